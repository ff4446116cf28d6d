// The accessor of an expansion (Sec. 3, "How to use the implementation?"): the field held as
// finest-level local series, queried at continuous positions for its value, first partials and
// second partials.
//
// With u = (x - z) / h in the cell that holds x and the scaled locals Lt(k) = h^|k| L(k),
//     y(x)                 = sum_k Lt(k) u^k / k!
//     d^s y / dx^s         = h^-|s| sum_k Lt(k + s) u^k / k!      (|k| <= rho - |s|)
// since d/du_i of u_i^a / a! is u_i^(a-1) / (a-1)!: a derivative lowers one exponent, so each
// partial is the series of the shifted coefficient row.  Each shifted sum is nested over the
// exponents (Horner-like) in the same order as the L2P kernel, so the value equals the forward
// transform's y at the same point.
//
// Two launch shapes: a list of points, walked in cell order through the counting sort (a warp
// touches few coefficient rows), and the meshgrid of per-axis coordinates (the paper's `vol`),
// where a thread derives its point from its output index -- consecutive outputs step along the
// last axis and stay in one or two cells, so no sort is needed.  The channel is blockIdx.y.
#include "dispatch.cuh"
#include "fc2t2_internal.cuh"

namespace fc2t2 {

constexpr int kEvalThreads = 128;

__host__ __device__ constexpr int eval_width(int D, int what) {
    return what == FC2T2_EVAL_VALUE ? 1 : what == FC2T2_EVAL_PARTIALS ? D : D * (D + 1) / 2;
}

// sum_{|k| <= rho - |s|} Lt(k + s) u^k / k!, nested over k0, k1, k2 (s = (S0, S1, S2))
template <int D, int RHO, int S0, int S1, int S2>
__device__ __forceinline__ float shifted_series(const float *Lv, const float (&pw)[3][RHO + 1]) {
    constexpr int R = RHO - S0 - S1 - S2;
    if constexpr (R < 0) {
        return 0.0f;
    } else {
        float acc = 0.0f;
#pragma unroll
        for (int a0 = 0; a0 <= R; ++a0) {
            float U = 0.0f;
#pragma unroll
            for (int a1 = 0; a0 + a1 <= R; ++a1) {
                float T;
                if constexpr (D == 2) {
                    T = Lv[gidx2(a0 + S0, a1 + S1)];
                } else {
                    T = 0.0f;
#pragma unroll
                    for (int a2 = 0; a0 + a1 + a2 <= R; ++a2)
                        T = fmaf(pw[2][a2], Lv[gidx3(a0 + S0, a1 + S1, a2 + S2)], T);
                }
                U = fmaf(pw[1][a1], T, U);
            }
            acc = fmaf(pw[0][a0], U, acc);
        }
        return acc;
    }
}

template <int D, int RHO, int WHAT>
__device__ __forceinline__ void series_outputs(const float *Lv, const float (&pw)[3][RHO + 1], float inv_h,
                                               float (&res)[eval_width(D, WHAT)]) {
    if constexpr (WHAT == FC2T2_EVAL_VALUE) {
        res[0] = shifted_series<D, RHO, 0, 0, 0>(Lv, pw);
    } else if constexpr (WHAT == FC2T2_EVAL_PARTIALS) {
        res[0] = inv_h * shifted_series<D, RHO, 1, 0, 0>(Lv, pw);
        res[1] = inv_h * shifted_series<D, RHO, 0, 1, 0>(Lv, pw);
        if constexpr (D == 3) res[2] = inv_h * shifted_series<D, RHO, 0, 0, 1>(Lv, pw);
    } else {
        const float s = inv_h * inv_h;
        if constexpr (D == 2) {
            res[0] = s * shifted_series<D, RHO, 2, 0, 0>(Lv, pw);
            res[1] = s * shifted_series<D, RHO, 1, 1, 0>(Lv, pw);
            res[2] = s * shifted_series<D, RHO, 0, 2, 0>(Lv, pw);
        } else {
            res[0] = s * shifted_series<D, RHO, 2, 0, 0>(Lv, pw);
            res[1] = s * shifted_series<D, RHO, 1, 1, 0>(Lv, pw);
            res[2] = s * shifted_series<D, RHO, 1, 0, 1>(Lv, pw);
            res[3] = s * shifted_series<D, RHO, 0, 2, 0>(Lv, pw);
            res[4] = s * shifted_series<D, RHO, 0, 1, 1>(Lv, pw);
            res[5] = s * shifted_series<D, RHO, 0, 0, 2>(Lv, pw);
        }
    }
}

struct EvalGeom {
    int n;                 // finest cells per dimension
    float lo, scale, h, inv_h;
    int64_t cstride;       // floats between channels' locals (G0 * Pp)
};

// the outputs at point x of channel c's locals
template <int D, int RHO, int WHAT>
__device__ __forceinline__ void eval_point(const float (&x)[3], const float *__restrict__ L, int c,
                                           const EvalGeom &g, float (&res)[eval_width(D, WHAT)]) {
    constexpr int Pp = pad4(ncoef(D, RHO));
    float pw[3][RHO + 1];
    int cell = 0, cd[3];
#pragma unroll
    for (int d = 0; d < D; ++d) cd[d] = cell_of(x[d], g.lo, g.scale, g.n);   // the sort's binning rule
#pragma unroll
    for (int d = D - 1; d >= 0; --d) cell = cell * g.n + cd[d];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float z = g.lo + ((float)cd[d] + 0.5f) * g.h;
        power_ladder<RHO>((x[d] - z) * g.inv_h, pw[d]);
    }
    if (D == 2) {
#pragma unroll
        for (int k = 0; k <= RHO; ++k) pw[2][k] = 0.0f;
    }
    float Lv[Pp];
    const float4 *Lr = reinterpret_cast<const float4 *>(L + (int64_t)c * g.cstride + (int64_t)cell * Pp);
#pragma unroll
    for (int i = 0; i < Pp / 4; ++i) {
        const float4 v = __ldg(Lr + i);
        Lv[4 * i] = v.x; Lv[4 * i + 1] = v.y; Lv[4 * i + 2] = v.z; Lv[4 * i + 3] = v.w;
    }
    series_outputs<D, RHO, WHAT>(Lv, pw, g.inv_h, res);
}

template <int D, int RHO, int WHAT>
__global__ void __launch_bounds__(kEvalThreads) k_eval_sorted(int64_t m, const float4 *__restrict__ rec,
                                                             const int *__restrict__ perm,
                                                             const float *__restrict__ L, EvalGeom g,
                                                             float *__restrict__ out) {
    constexpr int K = eval_width(D, WHAT);
    const int64_t j = (int64_t)blockIdx.x * kEvalThreads + threadIdx.x;
    if (j >= m) return;
    const int c = blockIdx.y;
    const float4 r = __ldg(rec + j);
    const float x[3] = {r.x, r.y, r.z};
    float res[K];
    eval_point<D, RHO, WHAT>(x, L, c, g, res);
    float *dst = out + ((int64_t)c * m + perm[j]) * K;
#pragma unroll
    for (int k = 0; k < K; ++k) dst[k] = res[k];
}

template <int D, int RHO, int WHAT>
__global__ void __launch_bounds__(kEvalThreads) k_eval_grid(const float *__restrict__ ax0,
                                                           const float *__restrict__ ax1,
                                                           const float *__restrict__ ax2, int64_t n1,
                                                           int64_t n2, int64_t total,
                                                           const float *__restrict__ L, EvalGeom g,
                                                           float *__restrict__ out) {
    constexpr int K = eval_width(D, WHAT);
    const int64_t idx = (int64_t)blockIdx.x * kEvalThreads + threadIdx.x;
    if (idx >= total) return;
    const int c = blockIdx.y;
    float x[3] = {0.0f, 0.0f, 0.0f};
    if (D == 2) {
        x[0] = __ldg(ax0 + idx / n1);
        x[1] = __ldg(ax1 + idx % n1);
    } else {
        const int64_t i2 = idx % n2, t = idx / n2;
        x[0] = __ldg(ax0 + t / n1);
        x[1] = __ldg(ax1 + t % n1);
        x[2] = __ldg(ax2 + i2);
    }
    float res[K];
    eval_point<D, RHO, WHAT>(x, L, c, g, res);
    float *dst = out + ((int64_t)c * total + idx) * K;
#pragma unroll
    for (int k = 0; k < K; ++k) dst[k] = res[k];
}

static EvalGeom geom_of(const fc2t2_plan_s *pl) {
    EvalGeom g;
    g.n = pl->n;
    g.lo = pl->lo_f;
    g.scale = pl->scale0_f;
    g.h = (float)pl->lev[0].h;
    g.inv_h = (float)(1.0 / pl->lev[0].h);
    g.cstride = pl->lev[0].G * pl->Pp;
    return g;
}

#define FC2T2_EVAL_WHAT(WHAT_VAR, LAUNCH)                                                    \
    switch (WHAT_VAR) {                                                                      \
        case FC2T2_EVAL_VALUE: { constexpr int W_ = FC2T2_EVAL_VALUE; LAUNCH; } break;       \
        case FC2T2_EVAL_PARTIALS: { constexpr int W_ = FC2T2_EVAL_PARTIALS; LAUNCH; } break; \
        case FC2T2_EVAL_PARTIALS2: { constexpr int W_ = FC2T2_EVAL_PARTIALS2; LAUNCH; } break; \
        default: return cudaErrorInvalidValue;                                               \
    }

cudaError_t launch_eval_sorted(const fc2t2_plan_s *pl, cudaStream_t s, const SortWork &w, int64_t m,
                               const float *L, int C, int what, float *out) {
    if (m == 0 || C == 0) return cudaSuccess;
    const dim3 grid((unsigned)((m + kEvalThreads - 1) / kEvalThreads), (unsigned)C);
    const EvalGeom g = geom_of(pl);
    cudaError_t err = cudaSuccess;
    pl->launches[FC2T2_STAGE_L2P] += 1;
    FC2T2_DISPATCH(pl->D, pl->rho,
                   FC2T2_EVAL_WHAT(what, (k_eval_sorted<D_, R_, W_><<<grid, kEvalThreads, 0, s>>>(
                                              m, w.rec, w.perm, L, g, out),
                                          err = cudaGetLastError())),
                   return cudaErrorInvalidValue)
    return err;
}

cudaError_t launch_eval_grid(const fc2t2_plan_s *pl, cudaStream_t s, const float *const *axis,
                             const int64_t *count, const float *L, int C, int what, float *out) {
    const int D = pl->D;
    int64_t total = 1;
    for (int d = 0; d < D; ++d) total *= count[d];
    if (total == 0 || C == 0) return cudaSuccess;
    const dim3 grid((unsigned)((total + kEvalThreads - 1) / kEvalThreads), (unsigned)C);
    const EvalGeom g = geom_of(pl);
    const float *a2 = D == 3 ? axis[2] : nullptr;
    const int64_t n2 = D == 3 ? count[2] : 1;
    cudaError_t err = cudaSuccess;
    pl->launches[FC2T2_STAGE_L2P] += 1;
    FC2T2_DISPATCH(D, pl->rho,
                   FC2T2_EVAL_WHAT(what, (k_eval_grid<D_, R_, W_><<<grid, kEvalThreads, 0, s>>>(
                                              axis[0], axis[1], a2, count[1], n2, total, L, g, out),
                                          err = cudaGetLastError())),
                   return cudaErrorInvalidValue)
    return err;
}

}  // namespace fc2t2
