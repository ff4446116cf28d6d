// M2M and L2L with the re-centring done in registers (every order up to 8).
//
// Re-centring a degree-rho polynomial by a per-dimension offset factorises over dimensions
// (Sec. 3: the M2M and L2L kernels are products of one-dimensional binomial shifts), and the
// total-degree truncation is preserved by every one-dimensional pass, so each shift is D
// in-place passes over the coefficient array held in registers:
//   moments (M2M):  a(..., n_d, ...) += sum_{k_d < n_d} t(n_d - k_d) a(..., k_d, ...)   (n_d descending)
//   locals  (L2L):  a(..., k_d, ...) += sum_{g_d > k_d} t(g_d - k_d) a(..., g_d, ...)   (k_d ascending)
// with t(j) = s^j / j!, s = +-1/2 the child centre's offset from the parent centre in child
// cell widths.  M2M: a parent thread (large levels) or the parent's 2^D child threads (small
// levels, summing by warp shuffles) shift the child rows and scale the sum by 2^-|a|.  L2L: a
// child thread loads its parent row, scales by 2^-|g|, shifts it and adds it to its own row.
// Rows move as 16-byte loads.
//
// With the M2L over occupied cells (`act`, the plan's occupancy bytes; NULL otherwise), rows that
// nothing reads are skipped: the moments of a parent without sources below it are not formed and
// a child without sources adds nothing (its row may be stale), and the locals of a child without
// targets below it are not formed.
#include "dispatch.cuh"
#include "fc2t2_internal.cuh"

namespace fc2t2 {

template <int D, int RHO, bool MOMENTS>
__device__ __forceinline__ void shift_axis(float (&a)[ncoef(D, RHO)], int axis, float s) {
    float t[RHO + 1];
    t[0] = 1.0f;
#pragma unroll
    for (int j = 1; j <= RHO; ++j) t[j] = t[j - 1] * (s * (1.0f / (float)j));
    // lines along `axis`: the other exponents fixed
#pragma unroll
    for (int u = 0; u <= RHO; ++u) {
#pragma unroll
        for (int v = 0; v <= RHO; ++v) {
            if (u + v > RHO) continue;
            if (D == 2 && v > 0) continue;
            const int len = RHO - u - v;   // exponent along the axis runs 0..len
            auto idx = [&](int n) {
                int e0, e1, e2;
                if (axis == 0) { e0 = n; e1 = u; e2 = v; }
                else if (axis == 1) { e0 = u; e1 = n; e2 = v; }
                else { e0 = u; e1 = v; e2 = n; }
                return D == 2 ? gidx2(e0, e1) : gidx3(e0, e1, e2);
            };
            if (MOMENTS) {
#pragma unroll
                for (int n = RHO; n >= 1; --n) {
                    if (n > len) continue;
                    float acc = a[idx(n)];
#pragma unroll
                    for (int k = 0; k < RHO; ++k)
                        if (k < n) acc = fmaf(t[n - k], a[idx(k)], acc);
                    a[idx(n)] = acc;
                }
            } else {
#pragma unroll
                for (int k = 0; k < RHO; ++k) {
                    if (k >= len) continue;
                    float acc = a[idx(k)];
#pragma unroll
                    for (int g = 1; g <= RHO; ++g)
                        if (g > k && g <= len) acc = fmaf(t[g - k], a[idx(g)], acc);
                    a[idx(k)] = acc;
                }
            }
        }
    }
}

template <int D, int RHO>
__device__ __forceinline__ void load_row(const float *__restrict__ src, float (&a)[ncoef(D, RHO)]) {
    constexpr int P = ncoef(D, RHO), Pp = pad4(P);
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
    for (int i = 0; i < Pp / 4; ++i) {
        const float4 v = __ldg(s4 + i);
        if (4 * i < P) a[4 * i] = v.x;
        if (4 * i + 1 < P) a[4 * i + 1] = v.y;
        if (4 * i + 2 < P) a[4 * i + 2] = v.z;
        if (4 * i + 3 < P) a[4 * i + 3] = v.w;
    }
}

template <int D, int RHO>
__device__ __forceinline__ void store_row(float *__restrict__ dst, const float (&a)[ncoef(D, RHO)]) {
    constexpr int P = ncoef(D, RHO), Pp = pad4(P);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int i = 0; i < Pp / 4; ++i)
        d4[i] = make_float4(4 * i < P ? a[4 * i] : 0.0f, 4 * i + 1 < P ? a[4 * i + 1] : 0.0f,
                            4 * i + 2 < P ? a[4 * i + 2] : 0.0f, 4 * i + 3 < P ? a[4 * i + 3] : 0.0f);
}

// total degree of the coefficient at graded index k (compile-time inside unrolled loops: a loop
// over the degrees with an inner loop over each degree's indices is not fully unrolled at orders
// 7-8, which leaves the row indexed at run time, i.e. in local memory)
__host__ __device__ constexpr int coef_degree(int D, int k) {
    int d = 0;
    while (ncoef(D, d) <= k) ++d;
    return d;
}

// M2M at large levels: one thread per parent cell, its children loaded and shifted in turn.
template <int D, int RHO>
__global__ void __launch_bounds__(128) k_m2m_reg(const float *__restrict__ Mc, float *__restrict__ Mp, int np,
                                                 int64_t Gp, const unsigned char *__restrict__ act_c,
                                                 const unsigned char *__restrict__ act_p) {
    constexpr int P = ncoef(D, RHO), Pp = pad4(P);
    const int64_t C = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (C >= Gp) return;
    if (act_p && !(act_p[C] & 1)) return;
    int cp[3] = {0, 0, 0};
    {
        int64_t r = C;
        for (int d = 0; d < D; ++d) { cp[d] = (int)(r % np); r /= np; }
    }
    const int nl = 2 * np;
    float acc[P];
#pragma unroll
    for (int k = 0; k < P; ++k) acc[k] = 0.0f;
    for (int ch = 0; ch < (1 << D); ++ch) {
        int64_t lin = 0;
        for (int d = D - 1; d >= 0; --d) lin = lin * nl + (2 * cp[d] + ((ch >> d) & 1));
        if (act_c && !(act_c[lin] & 1)) continue;
        float a[P];
        load_row<D, RHO>(Mc + lin * Pp, a);
#pragma unroll
        for (int d = 0; d < D; ++d) shift_axis<D, RHO, true>(a, d, ((ch >> d) & 1) ? 0.5f : -0.5f);
#pragma unroll
        for (int k = 0; k < P; ++k) acc[k] += a[k];
    }
    // 2^-|a| of the parent's larger cell width
#pragma unroll
    for (int k = 0; k < P; ++k) acc[k] *= 1.0f / (float)(1 << coef_degree(D, k));
    store_row<D, RHO>(Mp + C * Pp, acc);
}

// M2M at small levels: one thread per child cell, the 2^D children of a parent in consecutive
// lanes (at a few thousand parents one thread per parent leaves the GPU idle).  Each
// thread re-centres its child's row in registers; the parent's row is the sum over its lanes
// (butterfly shuffles), scaled by 2^-|a|; lane ch then writes the coefficients k = ch mod 2^D.
template <int D, int RHO>
__global__ void __launch_bounds__(256) k_m2m_child(const float *__restrict__ Mc, float *__restrict__ Mp, int np,
                                                 int64_t Gp, const unsigned char *__restrict__ act_c,
                                                 const unsigned char *__restrict__ act_p) {
    constexpr int P = ncoef(D, RHO), Pp = pad4(P), NCH = 1 << D;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t C = t >> D;
    const int ch = (int)(t & (NCH - 1));
    const bool valid = C < Gp;
    int64_t lin = 0;
    if (valid) {
        int cp[3] = {0, 0, 0};
        int64_t r = C;
        for (int d = 0; d < D; ++d) { cp[d] = (int)(r % np); r /= np; }
        const int nl = 2 * np;
        for (int d = D - 1; d >= 0; --d) lin = lin * nl + (2 * cp[d] + ((ch >> d) & 1));
    }
    const bool live = valid && (!act_c || (act_c[lin] & 1));   // (a child without sources adds zero)
    float a[P];
    if (live) {
        load_row<D, RHO>(Mc + lin * Pp, a);
#pragma unroll
        for (int d = 0; d < D; ++d) shift_axis<D, RHO, true>(a, d, ((ch >> d) & 1) ? 0.5f : -0.5f);
    } else {
#pragma unroll
        for (int k = 0; k < P; ++k) a[k] = 0.0f;
    }
    // every lane of the warp takes part in the shuffles (invalid lanes add zeros)
#pragma unroll
    for (int k = 0; k < P; ++k)
#pragma unroll
        for (int off = 1; off < NCH; off <<= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], off);
    if (!valid || (act_p && !(act_p[C] & 1))) return;
    float *dst = Mp + C * Pp;
#pragma unroll
    for (int k = 0; k < P; ++k)
        if ((k & (NCH - 1)) == ch) dst[k] = a[k] * (1.0f / (float)(1 << coef_degree(D, k)));
#pragma unroll
    for (int k = P; k < Pp; ++k)
        if ((k & (NCH - 1)) == ch) dst[k] = 0.0f;
}

template <int D, int RHO>
__global__ void __launch_bounds__(128) k_l2l_reg(const float *__restrict__ Lp, float *__restrict__ Lc, int nl,
                                                 int64_t Gc, const unsigned char *__restrict__ act_c) {
    constexpr int P = ncoef(D, RHO), Pp = pad4(P);
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= Gc) return;
    if (act_c && !(act_c[c] & 2)) return;
    int cc[3] = {0, 0, 0};
    {
        int64_t r = c;
        for (int d = 0; d < D; ++d) { cc[d] = (int)(r % nl); r /= nl; }
    }
    const int np = nl >> 1;
    int64_t plin = 0;
    for (int d = D - 1; d >= 0; --d) plin = plin * np + (cc[d] >> 1);
    float a[P];
    load_row<D, RHO>(Lp + plin * Pp, a);
#pragma unroll
    for (int k = 0; k < P; ++k) a[k] *= 1.0f / (float)(1 << coef_degree(D, k));
#pragma unroll
    for (int d = 0; d < D; ++d) shift_axis<D, RHO, false>(a, d, (cc[d] & 1) ? 0.5f : -0.5f);
    float4 *own = reinterpret_cast<float4 *>(Lc + c * Pp);
    if constexpr (RHO <= 6) {
        // all of the child's row in flight at once, then added and stored
        float o[P];
        load_row<D, RHO>(Lc + c * Pp, o);
#pragma unroll
        for (int k = 0; k < P; ++k) o[k] += a[k];
        store_row<D, RHO>(Lc + c * Pp, o);
    } else {
        // orders 7-8: add in batches of eight 16-byte chunks (a second row does not fit the
        // registers; eight loads stay in flight)
#pragma unroll
        for (int i0 = 0; i0 < Pp / 4; i0 += 8) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i0 + u < Pp / 4) v[u] = own[i0 + u];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u;
                if (i >= Pp / 4) break;
                if (4 * i < P) v[u].x += a[4 * i];
                if (4 * i + 1 < P) v[u].y += a[4 * i + 1];
                if (4 * i + 2 < P) v[u].z += a[4 * i + 2];
                if (4 * i + 3 < P) v[u].w += a[4 * i + 3];
                own[i] = v[u];
            }
        }
    }
}

template <int D, int RHO>
cudaError_t run_m2m_reg(const fc2t2_plan_s *pl, cudaStream_t s, int level) {
    {
        const Level &c = pl->lev[level], &p = pl->lev[level + 1];
        const unsigned char *act = pl->occ.enabled ? pl->occ.act : nullptr;
        // the per-parent form holds two rows in registers: orders <= 6 only
        bool done = false;
        if constexpr (RHO <= 6) {
            if (p.G > 4096) {
                const unsigned blocks = (unsigned)((p.G + 127) / 128);
                k_m2m_reg<D, RHO><<<blocks, 128, 0, s>>>(pl->d_M + c.off * pl->Pp, pl->d_M + p.off * pl->Pp, p.n, p.G,
                                                         act ? act + c.off : nullptr, act ? act + p.off : nullptr);
                done = true;
            }
        }
        if (!done) {
            const unsigned blocks = (unsigned)((p.G * (1 << D) + 255) / 256);
            k_m2m_child<D, RHO><<<blocks, 256, 0, s>>>(pl->d_M + c.off * pl->Pp, pl->d_M + p.off * pl->Pp, p.n, p.G,
                                                       act ? act + c.off : nullptr, act ? act + p.off : nullptr);
        }
    }
    return cudaGetLastError();
}

template <int D, int RHO>
cudaError_t run_l2l_reg(const fc2t2_plan_s *pl, cudaStream_t s, int level) {
    {
        const Level &p = pl->lev[level + 1], &c = pl->lev[level];
        const unsigned blocks = (unsigned)((c.G + 127) / 128);
        k_l2l_reg<D, RHO><<<blocks, 128, 0, s>>>(pl->d_L + p.off * pl->Pp, pl->d_L + c.off * pl->Pp, c.n, c.G,
                                                 pl->occ.enabled ? pl->occ.act + c.off : nullptr);
    }
    return cudaGetLastError();
}

bool launch_m2m_reg(const fc2t2_plan_s *pl, cudaStream_t s, int level, cudaError_t &err) {
    pl->launches[FC2T2_STAGE_M2M] += 1;
    FC2T2_DISPATCH(pl->D, pl->rho, (err = run_m2m_reg<D_, R_>(pl, s, level)), return false)
    return true;
}

bool launch_l2l_reg(const fc2t2_plan_s *pl, cudaStream_t s, int level, cudaError_t &err) {
    pl->launches[FC2T2_STAGE_L2L] += 1;
    FC2T2_DISPATCH(pl->D, pl->rho, (err = run_l2l_reg<D_, R_>(pl, s, level)), return false)
    return true;
}

}  // namespace fc2t2
