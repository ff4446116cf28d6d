// M2M, L2L and the CUDA-core M2L (Sec. 3).
//
// M2M (upward, level l -> l+1): one thread per (parent cell, multi-index a) sums the
// re-centred moments of its 2^D children,
//     Mt_{l+1}(a) = 2^-|a| sum_children sum_{b <= a} s^(a-b)/(a-b)! Mt_l(b),   s = +-1/2,
// the scaled form of the paper's M2M (Sec. 3, sum over k <= n).  The operator is the
// same at every level (the scaling absorbs h).  Padding columns are written as zeros.
//
// L2L (downward, level l+1 -> l): one thread per (child cell, k) adds the re-centred parent
// local expansion,  Lt_l(k) += sum_{g >= k} s^(g-k)/(g-k)! 2^-|g| Lt_{l+1}(g)
// (Sec. 3, L2L), after the M2L of level l has written Lt_l.
//
// M2L on the CUDA cores: target cells of one parity class and one output index k per
// block, so the interaction window (Sec. 3: the 6^D parity-dependent window, minus the
// 3^D hole above the finest level) and the operator rows are uniform across a warp.
//     Lt(k) = (-1)^|k| sum_{o in window} sum_{|b| <= rho-|k|} Dt[o](k+b) Mt[t+o](b)
#include "dispatch.cuh"
#include "fc2t2_internal.cuh"

namespace fc2t2 {

__device__ __forceinline__ void unravel_cell(int64_t lin, int n, int D, int (&c)[3]) {
    c[0] = c[1] = c[2] = 0;
    for (int d = 0; d < D; ++d) { c[d] = (int)(lin % n); lin /= n; }
}
__device__ __forceinline__ int64_t ravel_cell(const int (&c)[3], int n, int D) {
    int64_t lin = 0;
    for (int d = D - 1; d >= 0; --d) lin = lin * n + c[d];
    return lin;
}

// M2M and L2L: a block handles `pb` parent cells.  The rows it combines are staged in shared
// memory transposed ([coefficient][parent], stride pb + 1), so that a warp -- whose lanes are
// parents and which walks one output coefficient at a time -- reads conflict-free, while the
// pair list and the child shift tables are read as warp-wide broadcasts.  Results go through
// shared memory again so that global rows are written contiguously.
constexpr int kXThreads = 256;

struct XTables {
    const int *start;        // [P+1]
    const int2 *pairs;       // (row index, shift index)
    int npairs;
    const float *shift;      // [2^D][P]
    const float *pow2;       // [P]
};

struct XSmem {
    int *start;
    int2 *pairs;
    float *shift, *pow2;
    int64_t *cells;          // [pb][2^D] child (M2M, L2L) cell indices
    float *rows;             // transposed input rows
    float *out;              // staged output rows
};

__host__ __device__ inline size_t xsmem_bytes(int P, int Pp, int D, int npairs, int pb, bool l2l) {
    size_t b = ((sizeof(int) * (P + 1) + 15) & ~(size_t)15) + sizeof(int2) * npairs;
    b += sizeof(float) * (((size_t)P << D) + P);
    b = (b + 15) & ~(size_t)15;
    b += sizeof(int64_t) * pb * ((size_t)1 << D);
    const size_t nin = l2l ? (size_t)P : ((size_t)Pp << D);
    b += sizeof(float) * nin * (pb + 1);
    const size_t nout = l2l ? ((size_t)pb << D) * (Pp + 1) : (size_t)pb * (Pp + 1);
    b += sizeof(float) * nout;
    return b;
}

__device__ __forceinline__ XSmem xsmem_carve(unsigned char *base, const XTables &tb, int P, int Pp, int D, int pb,
                                             bool l2l) {
    XSmem s;
    s.start = reinterpret_cast<int *>(base);
    size_t off = (sizeof(int) * (P + 1) + 15) & ~(size_t)15;
    s.pairs = reinterpret_cast<int2 *>(base + off);
    off += sizeof(int2) * tb.npairs;
    s.shift = reinterpret_cast<float *>(base + off);
    off += sizeof(float) * ((size_t)P << D);
    s.pow2 = reinterpret_cast<float *>(base + off);
    off += sizeof(float) * P;
    off = (off + 15) & ~(size_t)15;
    s.cells = reinterpret_cast<int64_t *>(base + off);
    off += sizeof(int64_t) * pb * ((size_t)1 << D);
    s.rows = reinterpret_cast<float *>(base + off);
    off += sizeof(float) * (l2l ? (size_t)P : ((size_t)Pp << D)) * (pb + 1);
    s.out = reinterpret_cast<float *>(base + off);
    for (int i = threadIdx.x; i <= P; i += blockDim.x) s.start[i] = tb.start[i];
    for (int i = threadIdx.x; i < tb.npairs; i += blockDim.x) s.pairs[i] = tb.pairs[i];
    for (int i = threadIdx.x; i < (P << D); i += blockDim.x) s.shift[i] = tb.shift[i];
    for (int i = threadIdx.x; i < P; i += blockDim.x) s.pow2[i] = tb.pow2[i];
    return s;
}

// child cell indices of the block's parents (-1 past the end of the level)
__device__ __forceinline__ void child_cells(int64_t *cells, int64_t C0, int64_t Gp, int np, int D, int pb) {
    const int nch = 1 << D;
    for (int i = threadIdx.x; i < pb * nch; i += blockDim.x) {
        const int p = i / nch, ch = i % nch;
        const int64_t C = C0 + p;
        int64_t v = -1;
        if (C < Gp) {
            int cp[3];
            unravel_cell(C, np, D, cp);
            int cc[3] = {0, 0, 0};
            for (int d = 0; d < D; ++d) cc[d] = 2 * cp[d] + ((ch >> d) & 1);
            v = ravel_cell(cc, 2 * np, D);
        }
        cells[i] = v;
    }
}

__global__ void __launch_bounds__(kXThreads) k_m2m(const float *__restrict__ Mc, float *__restrict__ Mp, int np,
                                                   int D, int P, int Pp, int64_t Gp, int pb, XTables tb) {
    extern __shared__ __align__(16) unsigned char xs[];
    XSmem sm = xsmem_carve(xs, tb, P, Pp, D, pb, false);
    const int64_t C0 = (int64_t)blockIdx.x * pb;
    const int nch = 1 << D, ld = pb + 1;
    child_cells(sm.cells, C0, Gp, np, D, pb);
    __syncthreads();
    // rows[(ch * Pp + b) * ld + p] = Mt_child(p, ch)(b)
    for (int i = threadIdx.x; i < pb * nch * Pp; i += blockDim.x) {
        const int k = i % Pp, pc = i / Pp;            // pc = p * nch + ch
        const int64_t cell = sm.cells[pc];
        const int p = pc / nch, ch = pc % nch;
        sm.rows[(ch * Pp + k) * ld + p] = cell >= 0 ? Mc[cell * Pp + k] : 0.0f;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int pbase = 0; pbase < pb; pbase += 32) {
        const int p = pbase + lane;
        for (int a = warp; a < Pp; a += nwarps) {
            float acc = 0.0f;
            if (a < P && p < pb) {
                const int e0 = sm.start[a], e1 = sm.start[a + 1];
                for (int ch = 0; ch < nch; ++ch) {
                    const float *t = sm.shift + ch * P;
                    const float *r = sm.rows + ch * Pp * ld + p;
                    for (int e = e0; e < e1; ++e) {
                        const int2 pr = sm.pairs[e];
                        acc = fmaf(t[pr.y], r[pr.x * ld], acc);
                    }
                }
                acc *= sm.pow2[a];
            }
            if (p < pb) sm.out[p * (Pp + 1) + a] = acc;    // padding columns become zeros
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < pb * Pp; i += blockDim.x) {
        const int p = i / Pp, a = i % Pp;
        if (C0 + p < Gp) Mp[(C0 + p) * Pp + a] = sm.out[p * (Pp + 1) + a];
    }
}

static int x_parents(const fc2t2_plan_s *pl, int npairs, bool l2l, size_t &smem) {
    for (int pb = 32; pb >= 4; pb /= 2) {
        smem = xsmem_bytes(pl->P, pl->Pp, pl->D, npairs, pb, l2l);
        if (smem <= 200 * 1024) return pb;
    }
    smem = xsmem_bytes(pl->P, pl->Pp, pl->D, npairs, 4, l2l);
    return 4;
}

cudaError_t launch_m2m(const fc2t2_plan_s *pl, cudaStream_t s, int level) {
    cudaError_t rerr = cudaSuccess;
    if (launch_m2m_reg(pl, s, level, rerr)) return rerr;
    const Level &c = pl->lev[level], &p = pl->lev[level + 1];
    XTables tb{pl->d_m2m_start, pl->d_m2m_pairs, pl->n_m2m_pairs, pl->d_shift, pl->d_pow2};
    size_t smem = 0;
    const int pb = x_parents(pl, pl->n_m2m_pairs, false, smem);
    cudaFuncSetAttribute(k_m2m, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    pl->launches[FC2T2_STAGE_M2M] += 1;
    k_m2m<<<(unsigned)((p.G + pb - 1) / pb), kXThreads, smem, s>>>(
        pl->d_M + c.off * pl->Pp, pl->d_M + p.off * pl->Pp, p.n, pl->D, pl->P, pl->Pp, p.G, pb, tb);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kXThreads) k_l2l(const float *__restrict__ Lp, float *__restrict__ Lc, int np,
                                                   int D, int P, int Pp, int64_t Gp, int pb, XTables tb) {
    extern __shared__ __align__(16) unsigned char xs[];
    XSmem sm = xsmem_carve(xs, tb, P, Pp, D, pb, true);
    const int64_t C0 = (int64_t)blockIdx.x * pb;
    const int nch = 1 << D, ld = pb + 1;
    child_cells(sm.cells, C0, Gp, np, D, pb);
    __syncthreads();
    // rows[g * ld + p] = 2^-|g| Lt_parent(p)(g)
    for (int i = threadIdx.x; i < pb * P; i += blockDim.x) {
        const int p = i / P, g = i % P;
        sm.rows[g * ld + p] = (C0 + p < Gp) ? Lp[(C0 + p) * Pp + g] * sm.pow2[g] : 0.0f;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int pbase = 0; pbase < pb; pbase += 32) {
        const int p = pbase + lane;
        for (int task = warp; task < nch * P; task += nwarps) {
            const int ch = task / P, k = task % P;
            float acc = 0.0f;
            if (p < pb) {
                const float *t = sm.shift + ch * P;
                for (int e = sm.start[k]; e < sm.start[k + 1]; ++e) {
                    const int2 pr = sm.pairs[e];
                    acc = fmaf(t[pr.y], sm.rows[pr.x * ld + p], acc);
                }
                sm.out[(ch * pb + p) * (Pp + 1) + k] = acc;
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nch * pb * P; i += blockDim.x) {
        const int k = i % P, cp = i / P, p = cp / nch, ch = cp % nch;
        const int64_t cell = sm.cells[p * nch + ch];
        if (cell >= 0) Lc[cell * Pp + k] += sm.out[(ch * pb + p) * (Pp + 1) + k];
    }
}

cudaError_t launch_l2l(const fc2t2_plan_s *pl, cudaStream_t s, int level) {
    cudaError_t rerr = cudaSuccess;
    if (launch_l2l_reg(pl, s, level, rerr)) return rerr;
    const Level &p = pl->lev[level + 1], &c = pl->lev[level];
    XTables tb{pl->d_l2l_start, pl->d_l2l_pairs, pl->n_l2l_pairs, pl->d_shift, pl->d_pow2};
    size_t smem = 0;
    const int pb = x_parents(pl, pl->n_l2l_pairs, true, smem);
    cudaFuncSetAttribute(k_l2l, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    pl->launches[FC2T2_STAGE_L2L] += 1;
    k_l2l<<<(unsigned)((p.G + pb - 1) / pb), kXThreads, smem, s>>>(
        pl->d_L + p.off * pl->Pp, pl->d_L + c.off * pl->Pp, p.n, pl->D, pl->P, pl->Pp, p.G, pb, tb);
    return cudaGetLastError();
}

constexpr int kM2LThreads = 128;

__global__ void __launch_bounds__(kM2LThreads) k_m2l_simple(
    const float *__restrict__ M, float *__restrict__ L, int nl, int D, int Pp, int finest,
    const float *__restrict__ dtab, const int *__restrict__ pstart, const int2 *__restrict__ pairs) {
    const int k = blockIdx.y;
    const int half = nl >> 1;
    int64_t Gh = 1;
    for (int d = 0; d < D; ++d) Gh *= half;
    const int64_t nbp = (Gh + kM2LThreads - 1) / kM2LThreads;
    const int pi = (int)(blockIdx.x / nbp);
    const int64_t a = (int64_t)(blockIdx.x % nbp) * kM2LThreads + threadIdx.x;
    if (a >= Gh) return;
    int ac[3];
    unravel_cell(a, half, D, ac);
    int t[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, hiw[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) {
        t[d] = 2 * ac[d] + ((pi >> d) & 1);
        lo[d] = (t[d] & 1) ? -3 : -2;   // window [-3,+2] for odd, [-2,+3] for even indices
        hiw[d] = lo[d] + 5;
    }
    const int nz = (D == 3) ? nl : 1;
    const int e0 = pstart[k], e1 = pstart[k + 1];
    float acc = 0.0f;
    for (int oz = lo[2]; oz <= hiw[2]; ++oz) {
        const int sz = t[2] + oz;
        if (sz < 0 || sz >= nz) continue;
        for (int oy = lo[1]; oy <= hiw[1]; ++oy) {
            const int sy = t[1] + oy;
            if (sy < 0 || sy >= nl) continue;
            for (int ox = lo[0]; ox <= hiw[0]; ++ox) {
                const int sx = t[0] + ox;
                if (sx < 0 || sx >= nl) continue;
                // the hole: interactions within one cell are resolved at the finer level
                if (!finest && ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1)
                    continue;
                const int olin = (ox + 3) + 7 * (oy + 3) + (D == 3 ? 49 * (oz + 3) : 0);
                const int64_t slin = sx + (int64_t)nl * (sy + (int64_t)nl * sz);
                const float *Do = dtab + (int64_t)olin * Pp;
                const float *Ms = M + slin * Pp;
                for (int e = e0; e < e1; ++e) {
                    const int2 pr = pairs[e];
                    acc = fmaf(__ldg(Do + pr.y), __ldg(Ms + pr.x), acc);
                }
            }
        }
    }
    int deg = 0;
    while (((D == 2) ? (deg + 1) * (deg + 2) / 2 : (deg + 1) * (deg + 2) * (deg + 3) / 6) <= k) ++deg;
    const int64_t tlin = t[0] + (int64_t)nl * (t[1] + (int64_t)nl * t[2]);
    L[tlin * Pp + k] = (deg & 1) ? -acc : acc;
}

cudaError_t launch_m2l_simple(const fc2t2_plan_s *pl, cudaStream_t s, int level) {
    const Level &lv = pl->lev[level];
    const int half = lv.n >> 1;
    int64_t Gh = 1;
    for (int d = 0; d < pl->D; ++d) Gh *= half;
    const int64_t nbp = (Gh + kM2LThreads - 1) / kM2LThreads;
    const float *M = pl->d_M + lv.off * pl->Pp;
    float *L = pl->d_L + lv.off * pl->Pp;
    const int nofs = pl->D == 3 ? 343 : 49;
    const float *dt = pl->d_dtab + (int64_t)level * nofs * pl->Pp;
    dim3 grid((unsigned)(nbp << pl->D), (unsigned)pl->P);
    pl->launches[FC2T2_STAGE_M2L] += 1;
    k_m2l_simple<<<grid, kM2LThreads, 0, s>>>(M, L, lv.n, pl->D, pl->Pp, level == 0 ? 1 : 0, dt,
                                              pl->d_m2l_start, pl->d_m2l_pairs);
    return cudaGetLastError();
}

cudaError_t launch_m2l(const fc2t2_plan_s *pl, cudaStream_t s, int level) {
    return launch_m2l_simple(pl, s, level);
}

}  // namespace fc2t2
