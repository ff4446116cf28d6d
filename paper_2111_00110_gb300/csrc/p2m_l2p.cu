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
// L2P: one thread per sorted query loads its cell's coefficient row with 16-byte loads
// (queries of one cell are adjacent, so a warp touches few rows) and evaluates
//        y = sum_k Lt(k) u^k / k!
// as nested sums over the exponents (a Horner-like factoring).  The gradient variant also
// returns grad y = (1/h) sum_k Lt(k + e_i) u^k / k!, times the point's weight (pbar of
// Sec. 4.1), and writes results back in input order through the sort permutation.
#include "dispatch.cuh"
#include "fc2t2_internal.cuh"

namespace fc2t2 {

constexpr int kP2MThreads = 64;

template <int D, int RHO>
__global__ void __launch_bounds__(kP2MThreads) k_p2m(const float4 *__restrict__ rec,
                                                     const int *__restrict__ start, int n,
                                                     int64_t G, float lo, float h, float inv_h,
                                                     float *__restrict__ M) {
    constexpr int P = ncoef(D, RHO), Pp = pad4(P);
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const int64_t c0 = (int64_t)blockIdx.x * kP2MThreads;
    const int64_t c = c0 + threadIdx.x;
    float acc[P];
#pragma unroll
    for (int k = 0; k < P; ++k) acc[k] = 0.0f;
    if (c < G) {
        int cc[3] = {0, 0, 0};
        int64_t r = c;
#pragma unroll
        for (int d = 0; d < D; ++d) { cc[d] = (int)(r % n); r /= n; }
        float z[3];
#pragma unroll
        for (int d = 0; d < D; ++d) z[d] = lo + ((float)cc[d] + 0.5f) * h;
        const int j0 = start[c], j1 = start[c + 1];
        for (int j = j0; j < j1; ++j) {
            const float4 r = __ldg(rec + j);
            const float xj[3] = {r.x, r.y, r.z};
            float pw[3][RHO + 1];
#pragma unroll
            for (int d = 0; d < D; ++d) power_ladder<RHO>((xj[d] - z[d]) * inv_h, pw[d]);
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
    }
#pragma unroll
    for (int k = 0; k < Pp; ++k) sm[threadIdx.x * Pp + k] = (k < P) ? acc[k] : 0.0f;
    __syncthreads();
    const int64_t ncell = (G - c0) < kP2MThreads ? (G - c0) : kP2MThreads;
    const int total4 = (int)(ncell * Pp / 4);
    float4 *dst = reinterpret_cast<float4 *>(M + c0 * Pp);
    for (int i = threadIdx.x; i < total4; i += kP2MThreads) dst[i] = smem4[i];
}

cudaError_t launch_p2m(const fc2t2_plan_s *pl, cudaStream_t s, const SortWork &w, float *M0) {
    const int64_t G = pl->lev[0].G;
    const unsigned blocks = (unsigned)((G + kP2MThreads - 1) / kP2MThreads);
    const size_t smem = sizeof(float) * kP2MThreads * pl->Pp;
    const float h = (float)pl->lev[0].h, inv_h = (float)(1.0 / pl->lev[0].h);
    cudaError_t err = cudaSuccess;
    pl->launches[FC2T2_STAGE_P2M] += 1;
    FC2T2_DISPATCH(pl->D, pl->rho,
                   (k_p2m<D_, R_><<<blocks, kP2MThreads, smem, s>>>(w.rec, w.start, pl->n, G,
                                                                    pl->lo_f, h, inv_h, M0),
                    err = cudaGetLastError()),
                   return cudaErrorInvalidValue)
    return err;
}

constexpr int kL2PThreads = 128;

template <int D, int RHO, bool GRAD>
__global__ void __launch_bounds__(kL2PThreads) k_l2p(int64_t m, const float4 *__restrict__ rec,
                                                     const int *__restrict__ perm,
                                                     const float *__restrict__ L, int n, float lo, float scale,
                                                     float h, float inv_h, float *__restrict__ val,
                                                     float *__restrict__ grad, int accumulate) {
    constexpr int P = ncoef(D, RHO), Pp = pad4(P);
    const int64_t j = (int64_t)blockIdx.x * kL2PThreads + threadIdx.x;
    if (j >= m) return;
    const float4 r = __ldg(rec + j);
    const float xj[3] = {r.x, r.y, r.z};
    float pw[3][RHO + 1];
    int c = 0;
    {
        // the point's cell by the binning rule of the sort (same FP32 steps, same result)
        int cd[3];
#pragma unroll
        for (int d = 0; d < D; ++d) cd[d] = cell_of(xj[d], lo, scale, n);
#pragma unroll
        for (int d = D - 1; d >= 0; --d) c = c * n + cd[d];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const float z = lo + ((float)cd[d] + 0.5f) * h;
            power_ladder<RHO>((xj[d] - z) * inv_h, pw[d]);
        }
    }
    float Lv[Pp];
    const float4 *Lr = reinterpret_cast<const float4 *>(L + (int64_t)c * Pp);
#pragma unroll
    for (int i = 0; i < Pp / 4; ++i) {
        const float4 v = __ldg(Lr + i);
        Lv[4 * i] = v.x; Lv[4 * i + 1] = v.y; Lv[4 * i + 2] = v.z; Lv[4 * i + 3] = v.w;
    }
    float value = 0.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
#pragma unroll
    for (int a0 = 0; a0 <= RHO; ++a0) {
        float U = 0.0f, U1 = 0.0f, U2 = 0.0f;
#pragma unroll
        for (int a1 = 0; a1 <= RHO; ++a1) {
            if (a0 + a1 > RHO) continue;
            float T = 0.0f, T2 = 0.0f;
            if (D == 2) {
                T = Lv[gidx2(a0, a1)];
            } else {
#pragma unroll
                for (int a2 = 0; a2 <= RHO; ++a2) {
                    if (a0 + a1 + a2 > RHO) continue;
                    const float l = Lv[gidx3(a0, a1, a2)];
                    T = fmaf(pw[2][a2], l, T);
                    if (GRAD && a2 >= 1) T2 = fmaf(pw[2][a2 - 1], l, T2);
                }
            }
            U = fmaf(pw[1][a1], T, U);
            if (GRAD) {
                if (a1 >= 1) U1 = fmaf(pw[1][a1 - 1], T, U1);
                if (D == 3) U2 = fmaf(pw[1][a1], T2, U2);
            }
        }
        value = fmaf(pw[0][a0], U, value);
        if (GRAD) {
            if (a0 >= 1) g0 = fmaf(pw[0][a0 - 1], U, g0);
            g1 = fmaf(pw[0][a0], U1, g1);
            if (D == 3) g2 = fmaf(pw[0][a0], U2, g2);
        }
    }
    const int i = perm[j];
    if (val) val[i] = value;
    if (GRAD && grad) {
        const float s = r.w * inv_h;
        float *gi = grad + (int64_t)i * D;
        // (accumulate: the channels of one call add into the same gradient, one launch at a time)
        if (accumulate) {
            gi[0] += s * g0;
            gi[1] += s * g1;
            if (D == 3) gi[2] += s * g2;
        } else {
            gi[0] = s * g0;
            gi[1] = s * g1;
            if (D == 3) gi[2] = s * g2;
        }
    }
}

cudaError_t launch_l2p(const fc2t2_plan_s *pl, cudaStream_t s, const SortWork &w, int64_t m,
                       float *val, float *grad_times_w, bool accumulate) {
    if (m == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((m + kL2PThreads - 1) / kL2PThreads);
    const float h = (float)pl->lev[0].h, inv_h = (float)(1.0 / pl->lev[0].h);
    const float *L0 = pl->d_L + pl->lev[0].off * pl->Pp;
    cudaError_t err = cudaSuccess;
    pl->launches[FC2T2_STAGE_L2P] += 1;
    if (grad_times_w) {
        FC2T2_DISPATCH(pl->D, pl->rho,
                       (k_l2p<D_, R_, true><<<blocks, kL2PThreads, 0, s>>>(
                            m, w.rec, w.perm, L0, pl->n, pl->lo_f, pl->scale0_f, h, inv_h, val, grad_times_w,
                            accumulate ? 1 : 0),
                        err = cudaGetLastError()),
                       return cudaErrorInvalidValue)
    } else {
        FC2T2_DISPATCH(pl->D, pl->rho,
                       (k_l2p<D_, R_, false><<<blocks, kL2PThreads, 0, s>>>(
                            m, w.rec, w.perm, L0, pl->n, pl->lo_f, pl->scale0_f, h, inv_h, val, nullptr, 0),
                        err = cudaGetLastError()),
                       return cudaErrorInvalidValue)
    }
    return err;
}

}  // namespace fc2t2
