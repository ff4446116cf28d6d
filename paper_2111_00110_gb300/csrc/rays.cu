// Ray integrals of the transform (Sec. 6, the integral-implicit layer): for rays x(t) = o + t r,
// t in [t0, t1],
//     forward   y_q = int f(o_q + t r_q) dt          (f: the finest-level local series)
//     adjoint   the rays as sources with weights ybar_q (ray2M): every segment of a ray inside a
//               finest cell adds ybar_q int u(t)^b / b! dt to the cell's moments, and the usual
//               M2M .. L2P then give wbar, pbar at the sources.
// A ray is clipped to the domain box and cut at the faces of the finest cells it crosses; each
// segment lies in one cell (found from its midpoint by the binning rule).  On a segment the
// integrand is a polynomial of degree rho in t (the cell's series, or the monomials of the
// moments), so Gauss-Legendre quadrature with ceil((rho + 1) / 2) nodes integrates it exactly up
// to rounding -- the same integrals the paper writes with the binomial expansions of line2poly and
// line2taylor, at a handful of series evaluations per segment.
//
// One thread per ray walks its segments in order (the next face crossing of each axis is kept and
// the smallest taken), so a ray's cells are visited once, with a bounded number of steps.  The
// adjoint adds each segment's moments to the cell's row with 16-byte float atomics: many rays
// cross a cell, in no fixed order, so those sums are not bit-reproducible from run to run.
#include <cmath>

#include "dispatch.cuh"
#include "fc2t2_internal.cuh"

namespace fc2t2 {

constexpr int kRayThreads = 128;
constexpr int kMaxNodes = (kMaxOrder + 2) / 2;

struct RayArgs {
    int n;                     // finest cells per dimension
    float lo, hi, h, inv_h, scale;
    int nodes;                 // Gauss-Legendre nodes per segment
    float gx[kMaxNodes], gw[kMaxNodes];   // nodes on [0, 1] and their weights (summing to 1)
};

// the segment walk: calls seg(cell, ta, tb, c[3]) for every segment of the ray inside the domain
template <typename F>
__device__ __forceinline__ void walk_ray(const float (&o)[3], const float (&r)[3], float t0, float t1,
                                         const RayArgs &g, F &&seg) {
    float ta = t0, tb = t1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {   // clip to the domain box (slabs)
        if (r[k] == 0.0f) {
            if (!(o[k] >= g.lo && o[k] < g.hi)) return;
            continue;
        }
        const float a = (g.lo - o[k]) / r[k], b = (g.hi - o[k]) / r[k];
        ta = fmaxf(ta, fminf(a, b));
        tb = fminf(tb, fmaxf(a, b));
    }
    if (!(tb > ta)) return;   // (also rejects NaN)
    // per axis: the index of the next interior plane (lo + j h, 1 <= j < n) the ray crosses after ta
    int j[3], step[3];
    float tn[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        step[k] = r[k] > 0.0f ? 1 : -1;
        tn[k] = INFINITY;
        if (r[k] == 0.0f) continue;
        // the entry point's cell index along k (unclamped); moving up, the next plane is its
        // upper face, moving down its lower face (entering at x = hi going down: plane n - 1)
        const float x = o[k] + ta * r[k];
        const float cx = floorf((x - g.lo) * g.scale);
        int jj = cx < -1.0f ? -1 : (cx > (float)g.n ? g.n : (int)cx);
        jj = r[k] > 0.0f ? max(jj + 1, 1) : min(jj, g.n - 1);
        // (rounding: step on until the crossing lies after ta)
        for (int it = 0; it < 3 && jj >= 1 && jj <= g.n - 1 && (g.lo + jj * g.h - o[k]) / r[k] <= ta; ++it) jj += step[k];
        j[k] = jj;
        if (jj >= 1 && jj <= g.n - 1) tn[k] = (g.lo + jj * g.h - o[k]) / r[k];
    }
    float tc = ta;
    const int max_steps = 3 * g.n + 4;   // at most n - 1 interior planes per axis
    for (int it = 0; it < max_steps && tc < tb; ++it) {
        const float te = fminf(tb, fminf(tn[0], fminf(tn[1], tn[2])));
        if (te > tc) {
            const float tm = 0.5f * (tc + te);
            int c[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) c[k] = cell_of(o[k] + tm * r[k], g.lo, g.scale, g.n);
            seg(((int64_t)c[2] * g.n + c[1]) * g.n + c[0], tc, te, c);
        }
        tc = te;
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (tn[k] <= tc) {
                j[k] += step[k];
                tn[k] = (j[k] >= 1 && j[k] <= g.n - 1) ? (g.lo + j[k] * g.h - o[k]) / r[k] : INFINITY;
            }
    }
}

__device__ __forceinline__ void load_ray(const float4 *rays, int64_t q, float (&o)[3], float (&r)[3], float &t0,
                                         float &t1) {
    const float4 a = __ldg(rays + 2 * q), b = __ldg(rays + 2 * q + 1);
    o[0] = a.x; o[1] = a.y; o[2] = a.z;
    r[0] = a.w; r[1] = b.x; r[2] = b.y;
    t0 = b.z; t1 = b.w;
}

template <int RHO>
__global__ void __launch_bounds__(kRayThreads) k_ray_forward(const float4 *__restrict__ rays, int64_t R,
                                                             const float *__restrict__ L0, RayArgs g,
                                                             float *__restrict__ y) {
    constexpr int Pp = pad4(ncoef(3, RHO));
    const int64_t q = (int64_t)blockIdx.x * kRayThreads + threadIdx.x;
    if (q >= R) return;
    float o[3], r[3], t0, t1;
    load_ray(rays, q, o, r, t0, t1);
    float acc = 0.0f;
    walk_ray(o, r, t0, t1, g, [&](int64_t cell, float ta, float tb, const int (&c)[3]) {
        float Lv[Pp];
        const float4 *row = reinterpret_cast<const float4 *>(L0 + cell * Pp);
#pragma unroll
        for (int i = 0; i < Pp / 4; ++i) {
            const float4 v = __ldg(row + i);
            Lv[4 * i] = v.x; Lv[4 * i + 1] = v.y; Lv[4 * i + 2] = v.z; Lv[4 * i + 3] = v.w;
        }
        const float s = tb - ta;
        float z[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) z[k] = g.lo + ((float)c[k] + 0.5f) * g.h;
#pragma unroll
        for (int i = 0; i < (RHO + 2) / 2; ++i) {   // g.nodes
            const float t = fmaf(s, g.gx[i], ta);
            float pw[3][RHO + 1];
#pragma unroll
            for (int k = 0; k < 3; ++k) power_ladder<RHO>((fmaf(t, r[k], o[k]) - z[k]) * g.inv_h, pw[k]);
            float v = 0.0f, gr[3] = {0.0f, 0.0f, 0.0f};
            series_add<3, RHO, false>(Lv, pw, v, gr);
            acc = fmaf(s * g.gw[i], v, acc);
        }
    });
    y[q] = acc;
}

template <int RHO>
__global__ void __launch_bounds__(kRayThreads) k_ray2m(const float4 *__restrict__ rays, int64_t R,
                                                       const float *__restrict__ ybar, float *__restrict__ M0,
                                                       RayArgs g) {
    constexpr int P = ncoef(3, RHO), Pp = pad4(P);
    const int64_t q = (int64_t)blockIdx.x * kRayThreads + threadIdx.x;
    if (q >= R) return;
    const float wq = __ldg(ybar + q);
    if (wq == 0.0f) return;
    float o[3], r[3], t0, t1;
    load_ray(rays, q, o, r, t0, t1);
    walk_ray(o, r, t0, t1, g, [&](int64_t cell, float ta, float tb, const int (&c)[3]) {
        const float s = tb - ta;
        float z[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) z[k] = g.lo + ((float)c[k] + 0.5f) * g.h;
        float m[P];
#pragma unroll
        for (int b = 0; b < P; ++b) m[b] = 0.0f;
#pragma unroll
        for (int i = 0; i < (RHO + 2) / 2; ++i) {   // g.nodes
            const float t = fmaf(s, g.gx[i], ta);
            float pw[3][RHO + 1];
#pragma unroll
            for (int k = 0; k < 3; ++k) power_ladder<RHO>((fmaf(t, r[k], o[k]) - z[k]) * g.inv_h, pw[k]);
            const float wt = wq * s * g.gw[i];
#pragma unroll
            for (int a0 = 0; a0 <= RHO; ++a0) {
                const float t0w = wt * pw[0][a0];
#pragma unroll
                for (int a1 = 0; a0 + a1 <= RHO; ++a1) {
                    const float t01 = t0w * pw[1][a1];
#pragma unroll
                    for (int a2 = 0; a0 + a1 + a2 <= RHO; ++a2)
                        m[gidx3(a0, a1, a2)] = fmaf(t01, pw[2][a2], m[gidx3(a0, a1, a2)]);
                }
            }
        }
        // 16-byte atomic adds into the row (four coefficients per atomic; the padding gets zeros)
        float4 *dst = reinterpret_cast<float4 *>(M0 + cell * Pp);
#pragma unroll
        for (int i = 0; i < Pp / 4; ++i)
            atomicAdd(dst + i, make_float4(4 * i < P ? m[4 * i] : 0.0f, 4 * i + 1 < P ? m[4 * i + 1] : 0.0f,
                                           4 * i + 2 < P ? m[4 * i + 2] : 0.0f, 4 * i + 3 < P ? m[4 * i + 3] : 0.0f));
    });
}

// Gauss-Legendre nodes and weights of k points, mapped to [0, 1] (weights summing to 1): the roots
// of the Legendre polynomial P_k by Newton's method on the three-term recurrence.
static void gauss_legendre01(int k, float *x, float *w) {
    for (int i = 0; i < k; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (k + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;   // P_0, P_1
            for (int m = 2; m <= k; ++m) {
                const double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
                p0 = p1;
                p1 = p2;
            }
            const double pk = k == 0 ? 1.0 : p1, pkm1 = p0;
            dp = k * (z * pk - pkm1) / (z * z - 1.0);
            const double dz = pk / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = (float)(0.5 * (1.0 + z));
        w[i] = (float)(1.0 / ((1.0 - z * z) * dp * dp));   // 2 / ((1 - z^2) P_k'(z)^2), halved for [0, 1]
    }
}

static RayArgs ray_args(const fc2t2_plan_s *pl) {
    RayArgs g{};
    g.n = pl->n;
    g.lo = pl->lo_f;
    g.hi = pl->hi_f;
    g.h = (float)pl->lev[0].h;
    g.inv_h = (float)(1.0 / pl->lev[0].h);
    g.scale = pl->scale0_f;
    g.nodes = (pl->rho + 2) / 2;
    gauss_legendre01(g.nodes, g.gx, g.gw);
    return g;
}

cudaError_t launch_ray_forward(const fc2t2_plan_s *pl, cudaStream_t s, const float *rays, int64_t R, float *y) {
    if (R == 0) return cudaSuccess;
    if (pl->D != 3) return cudaErrorInvalidValue;
    const RayArgs g = ray_args(pl);
    const unsigned blocks = (unsigned)((R + kRayThreads - 1) / kRayThreads);
    const float *L0 = pl->d_L + pl->lev[0].off * pl->Pp;
    cudaError_t err = cudaSuccess;
    pl->launches[FC2T2_STAGE_L2P] += 1;
    switch (pl->rho) {
#define FC2T2_RAY_F(R_)                                                                                           \
    case R_:                                                                                                      \
        k_ray_forward<R_><<<blocks, kRayThreads, 0, s>>>(reinterpret_cast<const float4 *>(rays), R, L0, g, y);    \
        err = cudaGetLastError();                                                                                 \
        break;
        FC2T2_RAY_F(1) FC2T2_RAY_F(2) FC2T2_RAY_F(3) FC2T2_RAY_F(4) FC2T2_RAY_F(5) FC2T2_RAY_F(6) FC2T2_RAY_F(7)
        FC2T2_RAY_F(8)
#undef FC2T2_RAY_F
        default: return cudaErrorInvalidValue;
    }
    return err;
}

cudaError_t launch_ray2m(const fc2t2_plan_s *pl, cudaStream_t s, const float *rays, int64_t R, const float *ybar,
                         float *M0) {
    if (R == 0) return cudaSuccess;
    if (pl->D != 3) return cudaErrorInvalidValue;
    const RayArgs g = ray_args(pl);
    const unsigned blocks = (unsigned)((R + kRayThreads - 1) / kRayThreads);
    cudaError_t err = cudaSuccess;
    pl->launches[FC2T2_STAGE_P2M] += 1;
    switch (pl->rho) {
#define FC2T2_RAY_B(R_)                                                                                           \
    case R_:                                                                                                      \
        k_ray2m<R_><<<blocks, kRayThreads, 0, s>>>(reinterpret_cast<const float4 *>(rays), R, ybar, M0, g);      \
        err = cudaGetLastError();                                                                                 \
        break;
        FC2T2_RAY_B(1) FC2T2_RAY_B(2) FC2T2_RAY_B(3) FC2T2_RAY_B(4) FC2T2_RAY_B(5) FC2T2_RAY_B(6) FC2T2_RAY_B(7)
        FC2T2_RAY_B(8)
#undef FC2T2_RAY_B
        default: return cudaErrorInvalidValue;
    }
    return err;
}

}  // namespace fc2t2
