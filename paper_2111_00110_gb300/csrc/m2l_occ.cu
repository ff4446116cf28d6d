// M2L over occupied cells (Sec. 3: the M2L of a level sums, for every target cell t, the moments
// of the source cells of t's interaction list, translated by the kernel's derivatives at their
// offset).
//
//     Lt[t](k) = (-1)^|k| sum_{o in IL(t)} sum_{|b| <= rho-|k|} Dt[o](k+b) Mt[t+o](b)
//
// The moments of a cell that holds no source are zero, and the local series of a cell with no
// target below it is never read (L2L only hands a cell's series down to its children, L2P only
// reads the cells of the targets).  So the sum may run over the pairs of a target cell with
// targets below it and a source cell with sources below it: every local series that is read gets
// exactly the terms of the full M2L.  Where the points are clustered, most of the grid is empty
// and those pairs are a small part of all pairs.
//
// Occupancy: one byte per cell of every level (bit 0: sources below it, bit 1: targets below it).
// The finest level's byte comes from the two sorts' per-cell counts, each coarser level's is the
// OR of its 2^D children's.  The occupied targets of a level are appended to a list by parity
// class: bucket (level, class), where the lanes of a warp that fall in one bucket take one atomic
// together.  The order inside a bucket varies between runs; no result depends on it.
//
// The M2L is one persistent launch over a device work queue.  The work items are the chunks of 32
// targets of every bucket, of one plan or of every instance of a batched call, numbered by a
// prefix sum over the buckets (one small kernel).  Each CTA takes the next chunk with an atomic
// until none is left.  Within a CTA, each warp takes a group of the 2^D source parity classes (and,
// at orders 7-8, a range of the outputs), and each lane one target.  All targets of a chunk share
// its parity class, so a source class s' and a neighbour step delta in {-1, 0, 1}^D give one offset
// o = 2 delta + s' - s for the whole warp.  The offsets' derivative rows (all 2^D x 3^D of the
// class) are staged in shared memory once per chunk and read by broadcast.  Each lane reads its
// own source's moment row from global memory with 16-byte loads (the next offset's row prefetched
// into L1).  Offsets whose source cell is empty, outside the grid or (above the finest level) in
// the 3^D hole are skipped.  The multiply-adds are the direct form's compile-time list.  The
// partial sums of the source groups are added in shared memory in a fixed order, so the result
// does not depend on which CTA took which chunk.
#include <utility>

#include "dir_pairs.cuh"
#include "dispatch.cuh"
#include "fc2t2_internal.cuh"

namespace fc2t2 {

namespace {

// output ranges per warp: one thread cannot hold the 120 / 165 outputs of orders 7 / 8
__host__ __device__ constexpr int occ_splits(int D, int rho) { return D == 2 ? 1 : (rho <= 6 ? 1 : rho == 7 ? 2 : 4); }

template <int D, int RHO>
struct OccShape {
    static constexpr int NS = occ_splits(D, RHO);    // output ranges
    static constexpr int NC = 1 << D;                // source parity classes
    static constexpr int SPW = D == 2 ? 1 : NS;      // source classes per warp (8 warps per CTA in 3D)
    static constexpr int NG = NC / SPW;              // groups of source classes
    static constexpr int THREADS = 32 * NG * NS;     // 256 in 3D, 128 in 2D
    static constexpr int CHUNK = 32;                 // targets per work item: a lane each
    static constexpr int NV = D == 2 ? 9 : 27;       // offsets per source class
    static constexpr int P = ncoef(D, RHO), Pp = pad4(P);
    static constexpr int RP = P | 1;                 // pitch of the partial-sum rows (odd: no bank conflicts)
    static constexpr int DT_FLOATS = NC * NV * Pp;   // the class's staged derivative rows
    static constexpr size_t smem() { return ((size_t)DT_FLOATS + (size_t)NG * CHUNK * RP) * sizeof(float); }
};

template <int D, int RHO, int NS, int S>
struct OccSplit {
    static constexpr int K0 = dir_k0(D, RHO, NS, S), K1 = dir_k0(D, RHO, NS, S + 1);
    static constexpr int N = K1 - K0 > 0 ? K1 - K0 : 1;
};

// one pair: acc[k - K0] += Dt(m) Mt(b), the moment value from the source's row in global memory
// (16-byte read-only loads; repeated loads of one group are merged), the derivative value from the
// offset's staged row (a broadcast read)
template <int K0, int KB, int BB, int MB, int NACC>
__device__ __forceinline__ void occ_fma(const float *__restrict__ row, const float *__restrict__ drow,
                                        float (&acc)[NACC]) {
    const float4 mv4 = __ldg(reinterpret_cast<const float4 *>(row) + (BB >> 2));
    const float mv = (BB & 3) == 0 ? mv4.x : (BB & 3) == 1 ? mv4.y : (BB & 3) == 2 ? mv4.z : mv4.w;
    const float4 dv4 = *reinterpret_cast<const float4 *>(drow + (MB & ~3));
    const float dv = (MB & 3) == 0 ? dv4.x : (MB & 3) == 1 ? dv4.y : (MB & 3) == 2 ? dv4.z : dv4.w;
    acc[KB - K0] = fmaf(dv, mv, acc[KB - K0]);
}

template <int D, int RHO, int K0, int K1, int NACC, size_t... I>
__device__ __forceinline__ void occ_body_seq(const float *__restrict__ row, const float *__restrict__ drow,
                                             float (&acc)[NACC], std::index_sequence<I...>) {
    constexpr DirPairs<D, RHO, K0, K1> T{};
    (occ_fma<K0, T.k[I], T.b[I], T.m[I], NACC>(row, drow, acc), ...);
}

// sign (-1)^|k| and store of the outputs [K0, K1) into a partial-sum row
template <int D, int RHO, int K0, int K1, int NACC>
__device__ __forceinline__ void occ_store(float *red, const float (&acc)[NACC]) {
#pragma unroll
    for (int kd = 0; kd <= RHO; ++kd)
#pragma unroll
        for (int k0 = kd; k0 >= 0; --k0)
#pragma unroll
            for (int k1 = kd - k0; k1 >= 0; --k1) {
                const int k2 = kd - k0 - k1;
                if (D == 2 && k2 != 0) continue;
                const int ki = gidx<D>(k0, k1, k2);
                if (ki < K0 || ki >= K1) continue;
                red[ki] = (kd & 1) ? -acc[ki - K0] : acc[ki - K0];
            }
}

// L1 prefetch of a coefficient row of PP floats (16-byte aligned): every 128-byte line it touches
template <int PP>
__device__ __forceinline__ void prefetch_row(const float *row) {
    const char *a = reinterpret_cast<const char *>(row);
    const uintptr_t first = reinterpret_cast<uintptr_t>(a) & ~(uintptr_t)127;
    const uintptr_t last = (reinterpret_cast<uintptr_t>(a) + PP * 4 - 1) & ~(uintptr_t)127;
    for (uintptr_t l = first; l <= last; l += 128) asm volatile("prefetch.global.L1 [%0];" ::"l"(l));
}

// What a CTA knows about its current chunk (written by warp 0's first lane).
struct OccChunkInfo {
    const float *M;              // the level's moment rows
    float *L;                    // the level's local rows
    const float *dtab;           // the level's derivative rows [7^D][Pp]
    const unsigned char *act;    // the level's occupancy bytes
    const int *cells;            // the chunk's first target in its bucket
    int n, finest, cls, count, key, done;
};

// One warp's work for its source classes and output range, for its lane's target.  For each source
// class the warp runs the offsets that any of its lanes needs (the union of the lanes' masks of
// occupied, in-grid, non-hole source cells); a lane whose own source is empty sits the offset out.
template <int D, int RHO, int S>
__device__ __forceinline__ void occ_warp(const OccChunkInfo &ci, const float *s_dt, float *s_red, int g, int lane,
                                         bool valid, int cell) {
    using Sh = OccShape<D, RHO>;
    using Sp = OccSplit<D, RHO, Sh::NS, S>;
    float acc[Sp::N];
#pragma unroll
    for (int k = 0; k < Sp::N; ++k) acc[k] = 0.0f;
    const int n = ci.n, cls = ci.cls;
    const int tx = cell % n, ty = (cell / n) % n, tz = D == 3 ? cell / (n * n) : 0;
#pragma unroll 1
    for (int w = 0; w < Sh::SPW; ++w) {
        const int sp = g * Sh::SPW + w;
        // the offsets of this class whose source cell is in the grid and holds sources (all loads first)
        unsigned mask = 0;
        if (valid) {
#pragma unroll
            for (int j = 0; j < Sh::NV; ++j) {
                const int ox = 2 * (j % 3 - 1) + (sp & 1) - (cls & 1);
                const int oy = 2 * ((j / 3) % 3 - 1) + ((sp >> 1) & 1) - ((cls >> 1) & 1);
                const int oz = D == 3 ? 2 * (j / 9 - 1) + ((sp >> 2) & 1) - ((cls >> 2) & 1) : 0;
                const bool hole = !ci.finest && ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1;
                const int sx = tx + ox, sy = ty + oy, sz = tz + oz;
                const bool in = sx >= 0 && sx < n && sy >= 0 && sy < n && sz >= 0 && (D == 2 || sz < n);
                if (!hole && in && (__ldg(ci.act + (sx + n * (sy + n * sz))) & 1)) mask |= 1u << j;
            }
        }
        auto row_of = [&](int j) {
            const int ox = 2 * (j % 3 - 1) + (sp & 1) - (cls & 1);
            const int oy = 2 * ((j / 3) % 3 - 1) + ((sp >> 1) & 1) - ((cls >> 1) & 1);
            const int oz = D == 3 ? 2 * (j / 9 - 1) + ((sp >> 2) & 1) - ((cls >> 2) & 1) : 0;
            return ci.M + ((tx + ox) + (int64_t)n * ((ty + oy) + (int64_t)n * (tz + oz))) * Sh::Pp;
        };
        // the offsets in turn; while one row is worked on, the next one's cache lines are asked
        // for (an L1 prefetch: the loads of the next offset then wait on L1, not on L2)
        unsigned left = mask;
        if (left) prefetch_row<Sh::Pp>(row_of(__ffs(left) - 1));
#pragma unroll 1
        while (left) {
            const int j = __ffs(left) - 1;
            left &= left - 1;
            if (left) prefetch_row<Sh::Pp>(row_of(__ffs(left) - 1));
            occ_body_seq<D, RHO, Sp::K0, Sp::K1, Sp::N>(row_of(j), s_dt + (sp * Sh::NV + j) * Sh::Pp, acc,
                                                        std::make_index_sequence<DirPairs<D, RHO, Sp::K0, Sp::K1>::N>{});
        }
    }
    occ_store<D, RHO, Sp::K0, Sp::K1, Sp::N>(s_red + (g * Sh::CHUNK + lane) * Sh::RP, acc);
}

template <int D, int RHO>
__global__ void __launch_bounds__(OccShape<D, RHO>::THREADS, 1) k_m2l_occ(const OccQueue q) {
    using Sh = OccShape<D, RHO>;
    constexpr int NOFS = D == 3 ? 343 : 49;
    extern __shared__ __align__(16) float sm[];
    float *s_dt = sm;                         // [NC][NV][Pp]  derivative rows of the chunk's class
    float *s_red = sm + Sh::DT_FLOATS;        // [NG][32][RP]  partial sums of the source groups
    __shared__ OccChunkInfo ci;
    __shared__ int s_cell[Sh::CHUNK];
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const int g = warp / Sh::NS, split = warp % Sh::NS;   // warp-uniform
    const int nb = q.ninst * kOccBuckets;
    const int total = q.chunk_off[nb];
    int staged = -1;
    for (;;) {
        if (warp == 0) {
            int c = 0;
            if (lane == 0) c = atomicAdd(q.next, 1);
            c = __shfl_sync(0xffffffffu, c, 0);
            // the bucket b with chunk_off[b] <= c < chunk_off[b + 1] (a nonempty one): a 32-way
            // search, the lanes probing evenly spaced entries of the (non-decreasing) prefix
            int lo = 0, hi = nb;
            while (c < total && hi - lo > 1) {
                const int step = (hi - lo + 31) / 32;
                const int pos = lo + lane * step;
                const unsigned le = __ballot_sync(0xffffffffu, pos < hi && __ldg(q.chunk_off + pos) <= c);
                lo += (31 - __clz(le)) * step;   // lane 0 always holds (chunk_off[lo] <= c)
                hi = min(hi, lo + step);
            }
            if (lane == 0) ci.done = c >= total;
            if (lane == 0 && c < total) {
                const OccInst *in = q.inst[lo / kOccBuckets];
                const int j = lo % kOccBuckets, lvl = j >> 3, cls = j & 7;
                const int first = (c - q.chunk_off[lo]) * Sh::CHUNK;
                const int64_t off = in->off[lvl];
                const int n = in->n0 >> lvl;
                const int64_t G = D == 3 ? (int64_t)n * n * n : (int64_t)n * n;
                ci.M = in->M + off * Sh::Pp;
                ci.L = in->L + off * Sh::Pp;
                ci.dtab = in->dtab + (int64_t)lvl * NOFS * Sh::Pp;
                ci.act = in->act + off;
                ci.cells = in->list + off + cls * (G >> D) + first;
                ci.n = n;
                ci.finest = lvl == 0;
                ci.cls = cls;
                ci.count = min(Sh::CHUNK, in->cnt[j] - first);
                ci.key = lo;
            }
        }
        __syncthreads();
        if (ci.done) break;
        if (ci.key != staged) {   // (uniform) the class's 2^D x 3^D derivative rows
            const int cls = ci.cls;
            for (int i = (int)threadIdx.x; i < Sh::DT_FLOATS / 4; i += Sh::THREADS) {
                const int row = i / (Sh::Pp / 4), c4 = i - row * (Sh::Pp / 4);
                const int sp = row / Sh::NV, j = row - sp * Sh::NV;
                const int ox = 2 * (j % 3 - 1) + (sp & 1) - (cls & 1);
                const int oy = 2 * ((j / 3) % 3 - 1) + ((sp >> 1) & 1) - ((cls >> 1) & 1);
                const int oz = D == 3 ? 2 * (j / 9 - 1) + ((sp >> 2) & 1) - ((cls >> 2) & 1) : 0;
                const int olin = (ox + 3) + 7 * (oy + 3) + (D == 3 ? 49 * (oz + 3) : 0);
                reinterpret_cast<float4 *>(s_dt)[i] = __ldg(reinterpret_cast<const float4 *>(ci.dtab + olin * Sh::Pp) + c4);
            }
            staged = ci.key;
        }
        const bool valid = lane < ci.count;
        const int cell = valid ? ci.cells[lane] : 0;
        if (warp == 0) s_cell[lane] = cell;
        __syncthreads();
        if (Sh::NS == 1 || split == 0) occ_warp<D, RHO, 0>(ci, s_dt, s_red, g, lane, valid, cell);
        else if (Sh::NS >= 2 && split == 1) occ_warp<D, RHO, (Sh::NS >= 2 ? 1 : 0)>(ci, s_dt, s_red, g, lane, valid, cell);
        else if (Sh::NS >= 4 && split == 2) occ_warp<D, RHO, (Sh::NS >= 4 ? 2 : 0)>(ci, s_dt, s_red, g, lane, valid, cell);
        else if (Sh::NS >= 4) occ_warp<D, RHO, (Sh::NS >= 4 ? 3 : 0)>(ci, s_dt, s_red, g, lane, valid, cell);
        __syncthreads();
        // the groups' partial sums in a fixed order; coalesced row writes (padding columns zero)
        const int cnt = ci.count;
        float *L = ci.L;
        for (int i = (int)threadIdx.x; i < cnt * Sh::Pp; i += Sh::THREADS) {
            const int t = i / Sh::Pp, k = i - t * Sh::Pp;
            float v = 0.0f;
            if (k < Sh::P)
#pragma unroll
                for (int gg = 0; gg < Sh::NG; ++gg) v += s_red[(gg * Sh::CHUNK + t) * Sh::RP + k];
            L[(int64_t)s_cell[t] * Sh::Pp + k] = v;
        }
        __syncthreads();   // the chunk's shared state is read by every thread before the next claim
    }
}

// Number the chunks of every bucket of the queue's instances (exclusive prefix over the buckets,
// chunk_off[nb] = the total) and reset the work counter.  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_occ_queue(const OccQueue q) {
    const int nb = q.ninst * kOccBuckets;
    const int per = (nb + 1023) / 1024;
    const int b0 = (int)threadIdx.x * per;
    auto chunks = [&](int b) {
        const int c = q.inst[b / kOccBuckets]->cnt[b % kOccBuckets];
        return (c + q.chunk - 1) / q.chunk;
    };
    int local = 0;
    for (int i = 0; i < per; ++i)
        if (b0 + i < nb) local += chunks(b0 + i);
    __shared__ int s_warp[32];
    const int lane = (int)threadIdx.x & 31, warp = (int)threadIdx.x >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        s_warp[lane] = v;   // inclusive over the warps
    }
    __syncthreads();
    int run = incl - local + (warp > 0 ? s_warp[warp - 1] : 0);
    for (int i = 0; i < per; ++i)
        if (b0 + i < nb) {
            q.chunk_off[b0 + i] = run;
            run += chunks(b0 + i);
        }
    if (threadIdx.x == 1023) q.chunk_off[nb] = run;   // the last thread's running sum is the total
    if (threadIdx.x == 0) *q.next = 0;
}

// Append `cell` to bucket `cls` of a level's list when `want`: the lanes of a warp in one bucket
// take one atomic together.  Every lane of the warp must call it.
__device__ __forceinline__ void occ_append(int *list, int *cnt, int cls, int cap, int cell, bool want) {
    const unsigned wanting = __ballot_sync(0xffffffffu, want);
    if (!want) return;
    const unsigned peers = __match_any_sync(wanting, cls);
    const int lane = (int)threadIdx.x & 31, leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cnt + cls, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    list[(int64_t)cls * cap + base + __popc(peers & ((1u << lane) - 1u))] = cell;
}

// The cell of thread i of an occupancy kernel (n cells per dimension): the threads walk each
// parity class in turn, a class's cells in blocks of 4 x 4 x 2 class positions (8 x 4 in 2D), so a
// warp's appends -- and hence a work item's 32 consecutive targets -- are spatial neighbours.  Their
// sets of occupied source cells then nearly coincide (the M2L warp runs their union) and their
// source rows overlap in L1.
template <int D>
__device__ __forceinline__ int occ_cell(int i, int n, int G, int &cls) {
    const int per_cls = G >> D, h = n >> 1;   // class positions: h per dimension
    cls = i / per_cls;
    const int r = i - cls * per_cls;
    const int BX = min(D == 3 ? 4 : 8, h), BY = min(4, h), BZ = D == 3 ? min(2, h) : 1;
    const int per = BX * BY * BZ, b = r / per, w = r - b * per;
    const int nbx = h / BX, nby = h / BY;
    const int ax = (b % nbx) * BX + w % BX, ay = ((b / nbx) % nby) * BY + (w / BX) % BY;
    const int az = D == 3 ? (b / (nbx * nby)) * BZ + w / (BX * BY) : 0;
    return (2 * ax + (cls & 1)) + n * ((2 * ay + ((cls >> 1) & 1)) + n * (D == 3 ? 2 * az + ((cls >> 2) & 1) : 0));
}

// finest level: occupancy from the sorts' counts (NULL: every cell occupied) and the target list
template <int D>
__global__ void __launch_bounds__(256) k_occ_fine(const int *__restrict__ src_cnt, const int *__restrict__ tgt_cnt,
                                                  unsigned char *__restrict__ act, int *__restrict__ list,
                                                  int *__restrict__ cnt, int n, int G) {
    const int i = (int)(blockIdx.x * 256 + threadIdx.x);
    const bool live = i < G;
    int a = 0, cls = 0, c = 0;
    if (live) {
        c = occ_cell<D>(i, n, G, cls);
        a = ((src_cnt == nullptr || src_cnt[c] > 0) ? 1 : 0) | ((tgt_cnt == nullptr || tgt_cnt[c] > 0) ? 2 : 0);
        act[c] = (unsigned char)a;
    }
    occ_append(list, cnt, cls, G >> D, c, live && (a & 2));
}

// a coarser level (n cells per dimension): the OR of the children's bytes, and its target list
template <int D>
__global__ void __launch_bounds__(256) k_occ_up(const unsigned char *__restrict__ child, unsigned char *__restrict__ act,
                                                int *__restrict__ list, int *__restrict__ cnt, int n, int G) {
    const int i = (int)(blockIdx.x * 256 + threadIdx.x);
    const bool live = i < G;
    int a = 0, cls = 0, c = 0;
    if (live) {
        c = occ_cell<D>(i, n, G, cls);
        const int x = c % n, y = (c / n) % n, z = D == 3 ? c / (n * n) : 0;
        const int64_t nc = 2 * n;
#pragma unroll
        for (int k = 0; k < (D == 3 ? 2 : 1); ++k)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int64_t base = 2 * x + nc * ((2 * y + j) + nc * (D == 3 ? 2 * z + k : 0));
                a |= child[base] | child[base + 1];
            }
        act[c] = (unsigned char)a;
    }
    occ_append(list, cnt, cls, G >> D, c, live && (a & 2));
}

template <int D, int RHO>
cudaError_t occ_m2l_launch(const OccQueue &q, cudaStream_t s) {
    using Sh = OccShape<D, RHO>;
    constexpr size_t smem = Sh::smem();
    static_assert(smem <= 227 * 1024, "the staged rows exceed a CTA's shared memory");
    auto *fn = k_m2l_occ<D, RHO>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // persistent: as many CTAs as the device holds at once (per device, computed on first use)
    static int grid_of[64] = {};
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    int grid = dev < 64 ? grid_of[dev] : 0;
    if (grid == 0) {
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, Sh::THREADS, smem);
        grid = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
        if (dev < 64) grid_of[dev] = grid;
    }
    OccQueue qq = q;
    qq.chunk = Sh::CHUNK;
    k_occ_queue<<<1, 1024, 0, s>>>(qq);
    fn<<<grid, Sh::THREADS, smem, s>>>(qq);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_occupancy(const fc2t2_plan_s *pl, cudaStream_t s, const int *src_cnt, const int *tgt_cnt) {
    const auto &o = pl->occ;
    cudaError_t e = cudaMemsetAsync(o.cnt, 0, sizeof(int) * kOccBuckets, s);
    if (e != cudaSuccess) return e;
    pl->launches[FC2T2_STAGE_M2L] += pl->nlev;
    const int G0 = (int)pl->lev[0].G;
    if (pl->D == 2) k_occ_fine<2><<<(G0 + 255) / 256, 256, 0, s>>>(src_cnt, tgt_cnt, o.act, o.list, o.cnt, pl->n, G0);
    else k_occ_fine<3><<<(G0 + 255) / 256, 256, 0, s>>>(src_cnt, tgt_cnt, o.act, o.list, o.cnt, pl->n, G0);
    for (int l = 1; l < pl->nlev; ++l) {
        const Level &lv = pl->lev[l], &lc = pl->lev[l - 1];
        const int G = (int)lv.G;
        if (pl->D == 2)
            k_occ_up<2><<<(G + 255) / 256, 256, 0, s>>>(o.act + lc.off, o.act + lv.off, o.list + lv.off, o.cnt + 8 * l, lv.n, G);
        else
            k_occ_up<3><<<(G + 255) / 256, 256, 0, s>>>(o.act + lc.off, o.act + lv.off, o.list + lv.off, o.cnt + 8 * l, lv.n, G);
    }
    return cudaGetLastError();
}

cudaError_t launch_m2l_occ(const fc2t2_plan_s *const *plans, int nplan, cudaStream_t s) {
    if (nplan < 1 || nplan > kOccMaxInst) return cudaErrorInvalidValue;
    OccQueue q{};
    q.ninst = nplan;
    for (int i = 0; i < nplan; ++i) {
        if (plans[i]->D != plans[0]->D || plans[i]->rho != plans[0]->rho || !plans[i]->occ.enabled)
            return cudaErrorInvalidValue;
        q.inst[i] = plans[i]->occ.d_inst;
    }
    q.chunk_off = plans[0]->occ.chunk_off;
    q.next = plans[0]->occ.next;
    plans[0]->launches[FC2T2_STAGE_M2L] += 2;
    FC2T2_DISPATCH(plans[0]->D, plans[0]->rho, return (occ_m2l_launch<D_, R_>(q, s)), return cudaErrorInvalidValue);
    return cudaErrorInvalidValue;
}

}  // namespace fc2t2
