// P2M and L2P (Sec. 3), and the L2P gradient used by the backward pass (Sec. 4.1).
//
// Both kernels walk the cell-sorted points written by the counting sort, so every read of
// positions and weights is contiguous.
//
// P2M: one thread per finest cell sums its sources' scaled monomials
//        Mt(b) += w u^b / b!,  u = (p - z) / h,
// in registers (no atomics), then the block writes its cells' rows through shared memory
// as contiguous 16-byte stores.  Per source the work is the D power ladders plus one FMA
// per coefficient (Sec. 3.3 counts 2 FLOPs per coefficient for P2M).
//
// L2P: a CTA stages the coefficient rows of a segment of finest cells in shared memory, then
// one thread per sorted query of those cells evaluates
//        y = sum_k Lt(k) u^k / k!
// as nested sums over the exponents (a Horner-like factoring).  The gradient variant also
// returns grad y = (1/h) sum_k Lt(k + e_i) u^k / k!, times the point's weight (pbar of
// Sec. 4.1), and writes results back in input order through the sort permutation.
#include "dispatch.cuh"
#include "fc2t2_internal.cuh"
#include "tc_ptx.cuh"

namespace fc2t2 {

constexpr int kP2MThreads = 64;
// A P2M thread takes at most kP2MCap points of its cell; the points of a cell beyond its first
// kP2MCap (clustered sources, or the many samples of rays that cross a cell) are summed by a second
// kernel, in chunks of kOverChunk consecutive sorted points spread over the whole GPU, and added to
// the cell's row with float atomics.  So no thread waits on a cell much fuller than the mean.
constexpr int kP2MCap = 32;
// points per overflow chunk: one thread sums a chunk and adds it to its cell's row with one row of
// atomics, so longer chunks mean fewer atomics on the rows of the fullest cells
constexpr int kOverChunk = 128;

// acc += w u^b for one point (u = (x - z) / h per dimension); the factor 1 / b! is applied to the
// finished sums (p2m_scale)
template <int D, int RHO>
__device__ __forceinline__ void p2m_add(float (&acc)[ncoef(D, RHO)], const float4 r, const float (&z)[3], float inv_h) {
    const float xj[3] = {r.x, r.y, r.z};
    float pw[3][RHO + 1];
#pragma unroll
    for (int d = 0; d < D; ++d) powers<RHO>((xj[d] - z[d]) * inv_h, pw[d]);
    const float wj = r.w;
#pragma unroll
    for (int a0 = 0; a0 <= RHO; ++a0) {
        const float t0 = wj * pw[0][a0];
#pragma unroll
        for (int a1 = 0; a1 <= RHO; ++a1) {
            if (a0 + a1 > RHO) continue;
            if (D == 2) {
                acc[gidx2(a0, a1)] = fmaf(t0, pw[1][a1], acc[gidx2(a0, a1)]);
            } else {
                const float t01 = t0 * pw[1][a1];
#pragma unroll
                for (int a2 = 0; a2 <= RHO; ++a2) {
                    if (a0 + a1 + a2 > RHO) continue;
                    acc[gidx3(a0, a1, a2)] = fmaf(t01, pw[2][a2], acc[gidx3(a0, a1, a2)]);
                }
            }
        }
    }
}

// acc(b) *= 1 / b!
template <int D, int RHO>
__device__ __forceinline__ void p2m_scale(float (&acc)[ncoef(D, RHO)]) {
#pragma unroll
    for (int a0 = 0; a0 <= RHO; ++a0)
#pragma unroll
        for (int a1 = 0; a0 + a1 <= RHO; ++a1) {
            if (D == 2) {
                acc[gidx2(a0, a1)] *= inv_fact3(a0, a1, 0);
            } else {
#pragma unroll
                for (int a2 = 0; a0 + a1 + a2 <= RHO; ++a2) acc[gidx3(a0, a1, a2)] *= inv_fact3(a0, a1, a2);
            }
        }
}

// the records of [j0, j1) (j0 < j1) through f, the next record's load issued before each point's
// arithmetic
template <typename F>
__device__ __forceinline__ void walk_records(const float4 *__restrict__ rec, int j0, int j1, F f) {
    float4 r = __ldg(rec + j0);
    for (int j = j0; j < j1; ++j) {
        const float4 nx = j + 1 < j1 ? __ldg(rec + j + 1) : r;
        f(r);
        r = nx;
    }
}

template <int D>
__device__ __forceinline__ void cell_centre(int64_t c, int n, float lo, float h, float (&z)[3]) {
    z[0] = z[1] = z[2] = 0.0f;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        z[d] = lo + ((float)(int)(c % n) + 0.5f) * h;
        c /= n;
    }
}

template <int D, int RHO>
__global__ void __launch_bounds__(kP2MThreads) k_p2m(const float4 *__restrict__ rec,
                                                     const int *__restrict__ start, int n,
                                                     int64_t G, float lo, float h, float inv_h,
                                                     float *__restrict__ M, int *__restrict__ err,
                                                     int2 *__restrict__ over, unsigned long long *over_ctr,
                                                     int skip_empty) {
    constexpr int P = ncoef(D, RHO), Pp = pad4(P);
    extern __shared__ float4 smem4[];   // the block's sorted records, then its output rows
    __shared__ uint64_t staged;
    float *sm = reinterpret_cast<float *>(smem4);
    const int64_t c0 = (int64_t)blockIdx.x * kP2MThreads;
    const int64_t c = c0 + threadIdx.x;
    // The records of the block's cells are contiguous in the sort: one bulk asynchronous copy
    // stages them (as many as fit the output buffer) while the threads set up their cells; records
    // past the staged ones, or all of them if the bounded wait gives up, are read from memory.
    const int64_t c_end = (G - c0) < kP2MThreads ? G : c0 + kP2MThreads;
    const int jb0 = __ldg(start + c0), jb1 = __ldg(start + c_end);
    // (M2L over occupied cells: the rows of cells without sources are never read, so a block whose
    // cells hold no point leaves them as they are)
    if (skip_empty && jb1 == jb0) return;
    const int nst = min(jb1 - jb0, kP2MThreads * Pp / 4);
    if (nst > 0) {
        if (threadIdx.x == 0) tc::mbar_init(&staged, 1);
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::mbar_arrive_expect_tx(&staged, (uint32_t)nst * 16u);
            tc::bulk_g2s(smem4, rec + jb0, (uint32_t)nst * 16u, &staged);
        }
    }
    float acc[P];
#pragma unroll
    for (int k = 0; k < P; ++k) acc[k] = 0.0f;
    if (c < G) {
        float z[3];
        cell_centre<D>(c, n, lo, h, z);
        const int j0 = start[c], j1 = min(start[c + 1], j0 + kP2MCap);
        const bool have = nst > 0 && j1 > j0 && tc::mbar_wait(&staged, 0, err, 1024);
        for (int j = j0; j < j1; ++j) {
            const float4 r = (have && j - jb0 < nst) ? smem4[j - jb0] : __ldg(rec + j);
            p2m_add<D, RHO>(acc, r, z, inv_h);
        }
        p2m_scale<D, RHO>(acc);
    }
    __syncthreads();   // every staged record has been read before the buffer takes the output rows
#pragma unroll
    for (int k = 0; k < Pp; ++k) sm[threadIdx.x * Pp + k] = (k < P) ? acc[k] : 0.0f;
    __syncthreads();
    const int64_t ncell = (G - c0) < kP2MThreads ? (G - c0) : kP2MThreads;
    const int total4 = (int)(ncell * Pp / 4);
    float4 *dst = reinterpret_cast<float4 *>(M + c0 * Pp);
    for (int i = threadIdx.x; i < total4; i += kP2MThreads) dst[i] = smem4[i];

    // The cells of the block with points beyond their first kP2MCap append themselves to the
    // plan's overflow list: one 64-bit atomic per block reserves (entries, chunks) -- entry =
    // (cell, index of its first chunk of kOverChunk points in the list's chunk numbering) -- so the
    // entries come out ordered by chunk index.  k_p2m_over sums the chunks.
    const int cnt = c < G ? start[c + 1] - start[c] : 0;
    const int nch = cnt > kP2MCap ? (cnt - kP2MCap + kOverChunk - 1) / kOverChunk : 0;   // chunks past the first kP2MCap
    if (!__syncthreads_or(nch > 0)) return;
    __shared__ int s_warp[kP2MThreads / 32][2];
    __shared__ unsigned long long s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const unsigned heavy = __ballot_sync(0xffffffffu, nch > 0);
    if (lane == 31) { s_warp[warp][0] = incl; s_warp[warp][1] = __popc(heavy); }
    __syncthreads();
    int chunk_before = 0, entry_before = 0, chunks = 0, entries = 0;
#pragma unroll
    for (int v = 0; v < kP2MThreads / 32; ++v) {
        if (v < warp) { chunk_before += s_warp[v][0]; entry_before += s_warp[v][1]; }
        chunks += s_warp[v][0];
        entries += s_warp[v][1];
    }
    if (threadIdx.x == 0)
        s_base = atomicAdd(over_ctr, ((unsigned long long)entries << 32) | (unsigned long long)chunks);
    __syncthreads();
    if (nch > 0) {
        const int e = (int)(s_base >> 32) + entry_before + __popc(heavy & ((1u << lane) - 1u));
        over[e] = make_int2((int)c, (int)(s_base & 0xffffffffu) + chunk_before + incl - nch);
    }
}

// The overflow chunks of one P2M: a grid-stride loop over the list's chunks; chunk i belongs to the
// last entry whose first chunk is <= i (binary search), and covers kOverChunk consecutive sorted
// points of that cell past its first kP2MCap.  Each chunk's sum is added to the cell's row (written
// by k_p2m) with float atomics.  The last block to finish clears the list's counters for the next
// P2M; with an empty list every block leaves at once.
template <int D, int RHO>
__global__ void __launch_bounds__(128) k_p2m_over(const float4 *__restrict__ rec, const int *__restrict__ start,
                                                  int n, float lo, float h, float inv_h, float *__restrict__ M,
                                                  const int2 *__restrict__ over, unsigned long long *over_ctr) {
    constexpr int P = ncoef(D, RHO), Pp = pad4(P);
    const unsigned long long tot = *reinterpret_cast<volatile unsigned long long *>(over_ctr);
    if (tot == 0) return;
    const int nent = (int)(tot >> 32), nchunks = (int)(tot & 0xffffffffu);
    float acc[P];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nchunks; i += gridDim.x * blockDim.x) {
        int a = 0, b = nent;                         // over[a].y <= i < over[a + 1].y
        while (b - a > 1) {
            const int mid = (a + b) >> 1;
            if (__ldg(&over[mid].y) <= i) a = mid; else b = mid;
        }
        const int2 ent = __ldg(&over[a]);
        const int64_t cell = ent.x;
        const int jc = __ldg(start + cell) + kP2MCap + kOverChunk * (i - ent.y);
        const int jc1 = min(__ldg(start + cell + 1), jc + kOverChunk);
        float z[3];
        cell_centre<D>(cell, n, lo, h, z);
#pragma unroll
        for (int k = 0; k < P; ++k) acc[k] = 0.0f;
        walk_records(rec, jc, jc1, [&](const float4 r) { p2m_add<D, RHO>(acc, r, z, inv_h); });
        p2m_scale<D, RHO>(acc);
#pragma unroll
        for (int k = 0; k < P; ++k) atomicAdd(M + cell * Pp + k, acc[k]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(over_ctr + 1, 1ull) == gridDim.x - 1) {   // every block has read the counters
            over_ctr[0] = 0;
            over_ctr[1] = 0;
        }
    }
}

cudaError_t launch_p2m(const fc2t2_plan_s *pl, cudaStream_t s, const SortWork &w, float *M0) {
    const int64_t G = pl->lev[0].G;
    const unsigned blocks = (unsigned)((G + kP2MThreads - 1) / kP2MThreads);
    const size_t smem = sizeof(float) * kP2MThreads * pl->Pp;
    const float h = (float)pl->lev[0].h, inv_h = (float)(1.0 / pl->lev[0].h);
    cudaError_t err = cudaSuccess;
    pl->launches[FC2T2_STAGE_P2M] += 2;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned oblocks = (unsigned)(4 * (sms > 0 ? sms : 1));
    FC2T2_DISPATCH(pl->D, pl->rho,
                   (k_p2m<D_, R_><<<blocks, kP2MThreads, smem, s>>>(w.rec, w.start, pl->n, G, pl->lo_f, h, inv_h,
                                                                    M0, pl->d_flags + 2, pl->d_over,
                                                                    pl->d_over_ctr, pl->occ.enabled),
                    err = cudaGetLastError(),
                    err = err != cudaSuccess ? err
                                             : (k_p2m_over<D_, R_><<<oblocks, 128, 0, s>>>(w.rec, w.start, pl->n,
                                                                                          pl->lo_f, h, inv_h, M0,
                                                                                          pl->d_over, pl->d_over_ctr),
                                                cudaGetLastError())),
                   return cudaErrorInvalidValue)
    return err;
}

constexpr int kL2PThreads = 128;

// the outputs of one point: val[i] = value; grad[i] = (or += with accumulate) scale * g
template <int D, bool GRAD>
__device__ __forceinline__ void l2p_store(int64_t i, float value, const float (&g)[3], float scale, float *val,
                                          float *grad, int accumulate) {
    if (val) val[i] = value;
    if (GRAD && grad) {
        float *gi = grad + i * D;
        // (accumulate: the channels of one call add into the same gradient, one launch at a time)
        if (accumulate) {
            gi[0] += scale * g[0];
            gi[1] += scale * g[1];
            if (D == 3) gi[2] += scale * g[2];
        } else {
            gi[0] = scale * g[0];
            gi[1] = scale * g[1];
            if (D == 3) gi[2] = scale * g[2];
        }
    }
}

// The series of staged rows ra and rb (row index in units of P4 float4) at two points, into
// (va, ga) and (vb, gb); one shared pass over the row when both points use the same row.
template <int D, int RHO, bool GRAD>
__device__ __forceinline__ void l2p_rows(const float4 *rows, int P4, int ra, int rb, bool hasb,
                                         const float (&pa)[3][RHO + 1], const float (&pb)[3][RHO + 1], float &va,
                                         float (&ga)[3], float &vb, float (&gb)[3]) {
    constexpr int Pp = pad4(ncoef(D, RHO));
    float Lv[Pp];
    if (hasb && ra == rb) {
#pragma unroll
        for (int i = 0; i < Pp / 4; ++i) {
            const float4 v = rows[ra * P4 + i];
            Lv[4 * i] = v.x; Lv[4 * i + 1] = v.y; Lv[4 * i + 2] = v.z; Lv[4 * i + 3] = v.w;
        }
        series_add2<D, RHO, GRAD>(Lv, pa, pb, va, ga, vb, gb);
        return;
    }
#pragma unroll
    for (int i = 0; i < Pp / 4; ++i) {
        const float4 v = rows[ra * P4 + i];
        Lv[4 * i] = v.x; Lv[4 * i + 1] = v.y; Lv[4 * i + 2] = v.z; Lv[4 * i + 3] = v.w;
    }
    series_add<D, RHO, GRAD>(Lv, pa, va, ga);
    if (hasb) {
#pragma unroll
        for (int i = 0; i < Pp / 4; ++i) {
            const float4 v = rows[rb * P4 + i];
            Lv[4 * i] = v.x; Lv[4 * i + 1] = v.y; Lv[4 * i + 2] = v.z; Lv[4 * i + 3] = v.w;
        }
        series_add<D, RHO, GRAD>(Lv, pb, vb, gb);
    }
}

// L2P, staged: a CTA owns SC = min(32 or 64, n) consecutive finest cells of one x-line.  Their
// coefficient rows are contiguous in memory and are copied to shared memory with coalesced
// 16-byte loads (all in flight at once); the CTA then walks the cell-sorted points of those cells
// (a contiguous range of the sort), each thread evaluating its point from the staged row.  So no
// thread waits on a chain of dependent global loads (record, then row).
//
// TWO: the finest level's L2L has not run.  L2L is an exact re-centring of a local series of
// total degree <= rho, so the finest-level series after L2L equals the finest level's own M2L
// series plus level 1's complete local series (its M2L and everything L2L brought down to it),
// each about its own cell centre:
//     y(x) = sum_k Lt_0[c_0](k) u_0^k / k!  +  sum_k Lt_1[c_1](k) u_1^k / k!,
// c_1 = c_0 >> 1 per dimension (the tree's parent rule), u_l = (x - z_l) / h_l.  The SC / 2 parent
// rows of the segment are contiguous too and are staged beside the finest rows.
// cells a CTA stages: 64 with the parent rows (few targets per cell: twice the bytes in flight per
// CTA) where the rows fit the 48 KB of static shared memory, else 32
__host__ __device__ constexpr int l2p_stage_cells(int D, int rho, bool two) {
    return (two && 96 * pad4(ncoef(D, rho)) * 4 <= 48 * 1024) ? 64 : 32;
}

template <int D, int RHO, bool GRAD, bool TWO>
__global__ void __launch_bounds__(kL2PThreads) k_l2p_staged(const float4 *__restrict__ rec,
                                                            const int *__restrict__ perm,
                                                            const int *__restrict__ start,
                                                            const float *__restrict__ L0,
                                                            const float *__restrict__ L1, int n, float lo,
                                                            float scale, float h0, float inv_h0, float h1,
                                                            float inv_h1, float *__restrict__ val,
                                                            float *__restrict__ grad, int accumulate,
                                                            int *__restrict__ err) {
    constexpr int Pp = pad4(ncoef(D, RHO)), P4 = Pp / 4;
    constexpr int kStageCells = l2p_stage_cells(D, RHO, TWO);
    __shared__ alignas(16) float4 rows[(kStageCells + (TWO ? kStageCells / 2 : 0)) * P4];
    __shared__ uint64_t staged;   // mbarrier: the bulk copies of the rows have landed
    const int sc = n < kStageCells ? n : kStageCells;
    const int64_t c0 = (int64_t)blockIdx.x * sc;          // first cell (x0 = c0 mod n, a multiple of sc)
    const int x0 = (int)(c0 % n);
    const int j0 = __ldg(start + c0), j1 = __ldg(start + c0 + sc);
    if (j0 == j1) return;                                  // no points in the segment: nothing to stage
    // stage the segment's rows (and its parents' rows): both are contiguous in memory, so one
    // thread issues bulk asynchronous copies (16-byte aligned, multiples of 16 bytes) that complete
    // on an mbarrier, while every thread fetches its first point
    if (threadIdx.x == 0) tc::mbar_init(&staged, 1);
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t b0 = (uint32_t)(sc * Pp * sizeof(float));
        uint32_t b1 = 0;
        int64_t p0 = 0;
        if (TWO) {
            const int n1 = n >> 1;
            int64_t rest = c0 / n, mul = n1;               // (y, z) of the line, then the parent line
            for (int d = 1; d < D; ++d) {
                p0 += (rest % n >> 1) * mul;
                rest /= n;
                mul *= n1;
            }
            p0 += x0 >> 1;
            b1 = (uint32_t)((sc >> 1) * Pp * sizeof(float));
        }
        tc::mbar_arrive_expect_tx(&staged, b0 + b1);
        tc::bulk_g2s(rows, L0 + c0 * Pp, b0, &staged);
        if (TWO) tc::bulk_g2s(rows + sc * P4, L1 + p0 * Pp, b1, &staged);
    }
    // Without the parent rows (TWO false: many targets per cell) a thread takes two consecutive
    // sorted points per round -- mostly of one cell, whose series then share each row read; with
    // them (few targets per cell) one point, so that the CTA's threads all have work.  Records are
    // loaded one round ahead.
    constexpr int NPT = TWO ? 1 : 2;
    float4 rn[NPT];
    int in[NPT];                                           // and their places in the input order
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
        rn[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        in[u] = 0;
        if (j0 + NPT * (int)threadIdx.x + u < j1) {
            rn[u] = __ldg(rec + j0 + NPT * threadIdx.x + u);
            in[u] = __ldg(perm + j0 + NPT * threadIdx.x + u);
        }
    }
    if (!tc::mbar_wait(&staged, 0, err, 512)) return;     // (bounded; a timeout is reported by the plan)
    for (int j = j0 + NPT * (int)threadIdx.x; j < j1; j += NPT * kL2PThreads) {
        const bool hasb = NPT == 2 && j + 1 < j1;
        float4 r[NPT];
        int i_out[NPT];
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
            r[u] = rn[u];
            i_out[u] = in[u];
            if (j + NPT * kL2PThreads + u < j1) {   // the next records, one round ahead
                rn[u] = __ldg(rec + j + NPT * kL2PThreads + u);
                in[u] = __ldg(perm + j + NPT * kL2PThreads + u);
            }
        }
        int cd[NPT][3], lx[NPT];
        float pw[NPT][3][RHO + 1];
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
            const float xj[3] = {r[u].x, r[u].y, r[u].z};
#pragma unroll
            for (int d = 0; d < D; ++d) cd[u][d] = cell_of(xj[d], lo, scale, n);   // the sort's binning rule
            // the point's cell is in the segment (the sort used the same rule); clamped all the same
            const int l = cd[u][0] - x0;
            lx[u] = l < 0 ? 0 : (l >= sc ? sc - 1 : l);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const float z = lo + ((float)cd[u][d] + 0.5f) * h0;
                power_ladder<RHO>((xj[d] - z) * inv_h0, pw[u][d]);
            }
        }
        float value[2] = {0.0f, 0.0f}, g[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
        if constexpr (NPT == 2) {
            l2p_rows<D, RHO, GRAD>(rows, P4, lx[0], lx[1], hasb, pw[0], pw[1], value[0], g[0], value[1], g[1]);
        } else {
            float Lv[Pp];
#pragma unroll
            for (int i = 0; i < P4; ++i) {
                const float4 v = rows[lx[0] * P4 + i];
                Lv[4 * i] = v.x; Lv[4 * i + 1] = v.y; Lv[4 * i + 2] = v.z; Lv[4 * i + 3] = v.w;
            }
            series_add<D, RHO, GRAD>(Lv, pw[0], value[0], g[0]);
        }
        if (TWO) {
            // level 1's complete series about the parent cell (x0 is even): one point a thread
            const float xj[3] = {r[0].x, r[0].y, r[0].z};
            float pw1[3][RHO + 1];
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const float z = lo + ((float)(cd[0][d] >> 1) + 0.5f) * h1;
                power_ladder<RHO>((xj[d] - z) * inv_h1, pw1[d]);
            }
            float Lv[Pp];
            const int px = lx[0] >> 1;
#pragma unroll
            for (int i = 0; i < P4; ++i) {
                const float4 v = rows[(sc + px) * P4 + i];
                Lv[4 * i] = v.x; Lv[4 * i + 1] = v.y; Lv[4 * i + 2] = v.z; Lv[4 * i + 3] = v.w;
            }
            float v1 = 0.0f, g1[3] = {0.0f, 0.0f, 0.0f};
            series_add<D, RHO, GRAD>(Lv, pw1, v1, g1);
            value[0] += v1;
            if (GRAD) {
                // both gradients in x: the finest part scaled by 1/h0, level 1's by 1/h1
#pragma unroll
                for (int d = 0; d < 3; ++d) g[0][d] = fmaf(inv_h1 / inv_h0, g1[d], g[0][d]);
            }
        }
        l2p_store<D, GRAD>(i_out[0], value[0], g[0], r[0].w * inv_h0, val, grad, accumulate);
        if (NPT == 2 && hasb) l2p_store<D, GRAD>(i_out[NPT - 1], value[1], g[1], r[NPT - 1].w * inv_h0, val, grad, accumulate);
    }
}

template <bool TWO>
static cudaError_t launch_l2p_staged(const fc2t2_plan_s *pl, cudaStream_t s, const SortWork &w, int64_t m,
                                     float *val, float *grad_times_w, bool accumulate) {
    if (m == 0) return cudaSuccess;
    if (TWO && pl->nlev < 2) return cudaErrorInvalidValue;
    const int cells = l2p_stage_cells(pl->D, pl->rho, TWO);
    const int sc = pl->n < cells ? pl->n : cells;
    const unsigned blocks = (unsigned)(pl->lev[0].G / sc);
    const float h0 = (float)pl->lev[0].h, inv_h0 = (float)(1.0 / pl->lev[0].h);
    const float h1 = TWO ? (float)pl->lev[1].h : 1.0f, inv_h1 = TWO ? (float)(1.0 / pl->lev[1].h) : 1.0f;
    const float *L0 = pl->d_L + pl->lev[0].off * pl->Pp;
    const float *L1 = TWO ? pl->d_L + pl->lev[1].off * pl->Pp : nullptr;
    cudaError_t err = cudaSuccess;
    pl->launches[FC2T2_STAGE_L2P] += 1;
    if (grad_times_w) {
        FC2T2_DISPATCH(pl->D, pl->rho,
                       (k_l2p_staged<D_, R_, true, TWO><<<blocks, kL2PThreads, 0, s>>>(
                            w.rec, w.perm, w.start, L0, L1, pl->n, pl->lo_f, pl->scale0_f, h0, inv_h0, h1, inv_h1,
                            val, grad_times_w, accumulate ? 1 : 0, pl->d_flags + 2),
                        err = cudaGetLastError()),
                       return cudaErrorInvalidValue)
    } else {
        FC2T2_DISPATCH(pl->D, pl->rho,
                       (k_l2p_staged<D_, R_, false, TWO><<<blocks, kL2PThreads, 0, s>>>(
                            w.rec, w.perm, w.start, L0, L1, pl->n, pl->lo_f, pl->scale0_f, h0, inv_h0, h1, inv_h1,
                            val, nullptr, 0, pl->d_flags + 2),
                        err = cudaGetLastError()),
                       return cudaErrorInvalidValue)
    }
    return err;
}

cudaError_t launch_l2p(const fc2t2_plan_s *pl, cudaStream_t s, const SortWork &w, int64_t m, float *val,
                       float *grad_times_w, bool accumulate) {
    return launch_l2p_staged<false>(pl, s, w, m, val, grad_times_w, accumulate);
}

cudaError_t launch_l2p_two(const fc2t2_plan_s *pl, cudaStream_t s, const SortWork &w, int64_t m, float *val,
                           float *grad_times_w, bool accumulate) {
    return launch_l2p_staged<true>(pl, s, w, m, val, grad_times_w, accumulate);
}

}  // namespace fc2t2
