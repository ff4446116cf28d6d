// M2M / L2L dispatch (the kernels are the register forms of shift_reg.cu) and the CUDA-core M2L
// (Sec. 3).
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

// M2M (level l -> l + 1) and L2L (level l + 1 -> l): the register kernels cover every dimension
// and order a plan accepts.
cudaError_t launch_m2m(const fc2t2_plan_s *pl, cudaStream_t s, int level) {
    cudaError_t err = cudaSuccess;
    return launch_m2m_reg(pl, s, level, err) ? err : cudaErrorInvalidValue;
}

cudaError_t launch_l2l(const fc2t2_plan_s *pl, cudaStream_t s, int level) {
    cudaError_t err = cudaSuccess;
    return launch_l2l_reg(pl, s, level, err) ? err : cudaErrorInvalidValue;
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
