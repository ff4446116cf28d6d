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

__global__ void __launch_bounds__(128) k_m2m(const float *__restrict__ Mc, float *__restrict__ Mp,
                                             int np, int D, int P, int Pp, int64_t Gp,
                                             const int *__restrict__ pstart,
                                             const int2 *__restrict__ pairs,
                                             const float *__restrict__ shift,
                                             const float *__restrict__ pow2) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t C = gid / Pp;
    const int a = (int)(gid % Pp);
    if (C >= Gp) return;
    if (a >= P) { Mp[C * Pp + a] = 0.0f; return; }
    int cp[3];
    unravel_cell(C, np, D, cp);
    const int nl = 2 * np;
    float acc = 0.0f;
    const int e0 = pstart[a], e1 = pstart[a + 1];
    for (int ch = 0; ch < (1 << D); ++ch) {
        int cc[3];
        for (int d = 0; d < 3; ++d) cc[d] = 2 * cp[d] + ((ch >> d) & 1);
        const float *m = Mc + ravel_cell(cc, nl, D) * Pp;
        const float *t = shift + ch * P;
        for (int e = e0; e < e1; ++e) {
            const int2 pr = pairs[e];
            acc = fmaf(t[pr.y], m[pr.x], acc);
        }
    }
    Mp[C * Pp + a] = acc * pow2[a];
}

cudaError_t launch_m2m(const fc2t2_plan_s *pl, cudaStream_t s, int level) {
    const Level &c = pl->lev[level], &p = pl->lev[level + 1];
    const int64_t threads = p.G * pl->Pp;
    pl->launches[FC2T2_STAGE_M2M] += 1;
    k_m2m<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(
        pl->d_M + c.off * pl->Pp, pl->d_M + p.off * pl->Pp, p.n, pl->D, pl->P, pl->Pp, p.G,
        pl->d_m2m_start, pl->d_m2m_pairs, pl->d_shift, pl->d_pow2);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(128) k_l2l(const float *__restrict__ Lp, float *__restrict__ Lc,
                                             int nl, int D, int P, int Pp, int64_t Gc,
                                             const int *__restrict__ pstart,
                                             const int2 *__restrict__ pairs,
                                             const float *__restrict__ shift,
                                             const float *__restrict__ pow2) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t c = gid / P;
    const int k = (int)(gid % P);
    if (c >= Gc) return;
    int cc[3];
    unravel_cell(c, nl, D, cc);
    int cp[3] = {0, 0, 0};
    int ch = 0;
    for (int d = 0; d < D; ++d) { cp[d] = cc[d] >> 1; ch |= (cc[d] & 1) << d; }
    const float *l = Lp + ravel_cell(cp, nl >> 1, D) * Pp;
    const float *t = shift + ch * P;
    float acc = 0.0f;
    for (int e = pstart[k]; e < pstart[k + 1]; ++e) {
        const int2 pr = pairs[e];
        acc = fmaf(t[pr.y] * pow2[pr.x], l[pr.x], acc);
    }
    Lc[c * Pp + k] += acc;
}

cudaError_t launch_l2l(const fc2t2_plan_s *pl, cudaStream_t s, int level) {
    const Level &c = pl->lev[level], &p = pl->lev[level + 1];
    const int64_t threads = c.G * pl->P;
    pl->launches[FC2T2_STAGE_L2L] += 1;
    k_l2l<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(
        pl->d_L + p.off * pl->Pp, pl->d_L + c.off * pl->Pp, c.n, pl->D, pl->P, pl->Pp, c.G,
        pl->d_l2l_start, pl->d_l2l_pairs, pl->d_shift, pl->d_pow2);
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
    if (pl->tc.enabled) return launch_m2l_tc(pl, s, level);
    return launch_m2l_simple(pl, s, level);
}

}  // namespace fc2t2
