// Internal definitions of the FC2T2 CUDA library: the plan, multi-index arithmetic,
// the FP32 binning rule, and the kernel launchers shared between translation units.
//
// Representation on the device (scaled per level, which keeps every coefficient O(1)):
//   Mt_l[c](b) = sum_{i in c} w_i u_i^b / b!,        u_i = (p_i - z_l(c)) / h_l
//   Lt_l[c](k) = h_l^|k| L_l[c](k)
//   Dt_l[o](m) = h_l^|m| d^m psi(o h_l)              (o an integer cell offset)
// so that, with the paper's unscaled M, L (Sec. 3):
//   M2L  Lt(k) += (-1)^|k| sum_{|b| <= rho-|k|} Dt[o](k+b) Mt[t+o](b)
//   M2M  Mt_{l+1}(a) = 2^-|a| sum_children sum_{b<=a} s^(a-b)/(a-b)! Mt_l(b),  s = +-1/2
//   L2L  Lt_l(k) += sum_{g>=k} s^(g-k)/(g-k)! 2^-|g| Lt_{l+1}(g)
//   L2P  y = sum_k Lt_0(k) u^k / k!,  grad y = (1/h_0) sum_k Lt_0(k + e_i) u^k / k!
// Multi-indices are graded: degree, then the exponent of x_0 descending, then of x_1
// descending.  Coefficient rows are padded to Pp = P rounded up to 4 floats (16 bytes).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fc2t2.h"

namespace fc2t2 {

constexpr int kMaxDim = 3;
constexpr int kMaxOrder = 8;
constexpr int kMaxLevels = 10;

__host__ __device__ constexpr int ncoef(int D, int rho) {
    return D == 2 ? (rho + 1) * (rho + 2) / 2 : (rho + 1) * (rho + 2) * (rho + 3) / 6;
}
__host__ __device__ constexpr int pad4(int P) { return (P + 3) & ~3; }

// graded index of an exponent tuple
__host__ __device__ constexpr int gidx2(int a0, int a1) {
    int d = a0 + a1;
    return d * (d + 1) / 2 + (d - a0);
}
__host__ __device__ constexpr int gidx3(int a0, int a1, int a2) {
    int d = a0 + a1 + a2, r = d - a0;
    return d * (d + 1) * (d + 2) / 6 + r * (r + 1) / 2 + (r - a1);
}
template <int D>
__host__ __device__ constexpr int gidx(int a0, int a1, int a2) {
    return D == 2 ? gidx2(a0, a1) : gidx3(a0, a1, a2);
}

// The FP32 binning rule (every step rounded to FP32, no contraction).
__device__ __forceinline__ int cell_of(float x, float lo, float scale, int n) {
    float t = __fmul_rn(__fsub_rn(x, lo), scale);
    float f = floorf(t);
    int c = 0;
    if (f >= 0.0f) c = (f >= (float)n) ? n - 1 : (int)f;   // NaN and negatives -> 0
    return c;
}
__device__ __forceinline__ bool outside(float x, float lo, float scale, int n) {
    float t = __fmul_rn(__fsub_rn(x, lo), scale);
    return !(t >= 0.0f && t < (float)n);
}

// u^k / k! for k = 0..RHO (the monomials of P2M and L2P)
template <int RHO>
__device__ __forceinline__ void power_ladder(float u, float (&pw)[RHO + 1]) {
    pw[0] = 1.0f;
#pragma unroll
    for (int k = 1; k <= RHO; ++k) pw[k] = pw[k - 1] * (u * (1.0f / (float)k));
}

// u^k for k = 0..RHO (one multiply per power; the factorials are applied once per row instead)
template <int RHO>
__device__ __forceinline__ void powers(float u, float (&pw)[RHO + 1]) {
    pw[0] = 1.0f;
#pragma unroll
    for (int k = 1; k <= RHO; ++k) pw[k] = pw[k - 1] * u;
}

// 1 / (a0! a1! a2!) in FP32 (a compile-time constant where the exponents are)
__host__ __device__ constexpr float inv_fact3(int a0, int a1, int a2) {
    double f = 1.0;
    for (int i = 2; i <= a0; ++i) f *= i;
    for (int i = 2; i <= a1; ++i) f *= i;
    for (int i = 2; i <= a2; ++i) f *= i;
    return (float)(1.0 / f);
}

// The series of one coefficient row at u (power ladders pw): value, and with GRAD the three
// sums of the shifted rows sum_k Lt(k + e_i) u^k / k! (the gradient in u), nested over the
// exponents; the results are added to value, g[].
template <int D, int RHO, bool GRAD>
__device__ __forceinline__ void series_add(const float *Lv, const float (&pw)[3][RHO + 1], float &value,
                                           float (&g)[3]) {
    float val = 0.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
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
        val = fmaf(pw[0][a0], U, val);
        if (GRAD) {
            if (a0 >= 1) g0 = fmaf(pw[0][a0 - 1], U, g0);
            g1 = fmaf(pw[0][a0], U1, g1);
            if (D == 3) g2 = fmaf(pw[0][a0], U2, g2);
        }
    }
    value += val;
    g[0] += g0;
    g[1] += g1;
    g[2] += g2;
}

// series_add for two points on the same coefficient row: each coefficient is read once and feeds
// both points' sums (the row's reads are shared, and the two points' FMA chains interleave).
template <int D, int RHO, bool GRAD>
__device__ __forceinline__ void series_add2(const float *Lv, const float (&pa)[3][RHO + 1], const float (&pb)[3][RHO + 1],
                                            float &va, float (&ga)[3], float &vb, float (&gb)[3]) {
    float a_val = 0.0f, a0g = 0.0f, a1g = 0.0f, a2g = 0.0f;
    float b_val = 0.0f, b0g = 0.0f, b1g = 0.0f, b2g = 0.0f;
#pragma unroll
    for (int a0 = 0; a0 <= RHO; ++a0) {
        float Ua = 0.0f, U1a = 0.0f, U2a = 0.0f, Ub = 0.0f, U1b = 0.0f, U2b = 0.0f;
#pragma unroll
        for (int a1 = 0; a1 <= RHO; ++a1) {
            if (a0 + a1 > RHO) continue;
            float Ta = 0.0f, T2a = 0.0f, Tb = 0.0f, T2b = 0.0f;
            if (D == 2) {
                Ta = Tb = Lv[gidx2(a0, a1)];
            } else {
#pragma unroll
                for (int a2 = 0; a2 <= RHO; ++a2) {
                    if (a0 + a1 + a2 > RHO) continue;
                    const float l = Lv[gidx3(a0, a1, a2)];
                    Ta = fmaf(pa[2][a2], l, Ta);
                    Tb = fmaf(pb[2][a2], l, Tb);
                    if (GRAD && a2 >= 1) {
                        T2a = fmaf(pa[2][a2 - 1], l, T2a);
                        T2b = fmaf(pb[2][a2 - 1], l, T2b);
                    }
                }
            }
            Ua = fmaf(pa[1][a1], Ta, Ua);
            Ub = fmaf(pb[1][a1], Tb, Ub);
            if (GRAD) {
                if (a1 >= 1) {
                    U1a = fmaf(pa[1][a1 - 1], Ta, U1a);
                    U1b = fmaf(pb[1][a1 - 1], Tb, U1b);
                }
                if (D == 3) {
                    U2a = fmaf(pa[1][a1], T2a, U2a);
                    U2b = fmaf(pb[1][a1], T2b, U2b);
                }
            }
        }
        a_val = fmaf(pa[0][a0], Ua, a_val);
        b_val = fmaf(pb[0][a0], Ub, b_val);
        if (GRAD) {
            if (a0 >= 1) {
                a0g = fmaf(pa[0][a0 - 1], Ua, a0g);
                b0g = fmaf(pb[0][a0 - 1], Ub, b0g);
            }
            a1g = fmaf(pa[0][a0], U1a, a1g);
            b1g = fmaf(pb[0][a0], U1b, b1g);
            if (D == 3) {
                a2g = fmaf(pa[0][a0], U2a, a2g);
                b2g = fmaf(pb[0][a0], U2b, b2g);
            }
        }
    }
    va += a_val;
    ga[0] += a0g; ga[1] += a1g; ga[2] += a2g;
    vb += b_val;
    gb[0] += b0g; gb[1] += b1g; gb[2] += b2g;
}

// One counting sort of points into finest-level cells.
struct SortWork {
    int64_t cap = 0;
    int *count = nullptr;       // [G0]   points per cell
    int *start = nullptr;       // [G0+1] exclusive prefix sum
    int *key = nullptr;         // [cap]  cell of point i (input order)
    int *rank = nullptr;        // [cap]  position of point i within its cell
    int *perm = nullptr;        // [cap]  sorted position -> input index
    float4 *rec = nullptr;      // [cap]  sorted point: (x0, x1, x2 or 0, weight or 0)
    int *scan_tmp = nullptr;    // block sums of this sort's prefix scan (the two sorts may run at once)
    // what the workspace holds: the points and weights arrays (and count) it last sorted
    const float *held_x = nullptr, *held_w = nullptr;
    int64_t held_n = -1;
};

struct Level {
    int n;              // cells per dimension
    int64_t G;          // cells
    int64_t off;        // first cell of this level in the concatenated coefficient arrays
    double h;           // cell width
};

// M2L over occupied cells: one plan's arrays as the work queue's kernel reads them (kept in device
// memory, written once at plan creation), and the queue of one launch over one or more plans.
constexpr int kOccBuckets = kMaxLevels * 8;    // (level, parity class) buckets per plan
constexpr int kOccMaxInst = 64;                // plans per launch
struct OccInst {
    const float *M;              // moments of every level [G_total][Pp]
    float *L;                    // locals of every level
    const float *dtab;           // [nlev][7^D][Pp] scaled kernel derivatives
    const unsigned char *act;    // [G_total] bit 0: sources below the cell, bit 1: targets below it
    const int *list;             // [G_total] occupied targets: bucket (l, cls) at off[l] + cls * G_l / 2^D
    const int *cnt;              // [kOccBuckets] bucket sizes, (l, cls) at 8 l + cls
    int nlev, n0;                // levels, finest cells per dimension
    int64_t off[kMaxLevels];     // first cell of each level
};
struct OccQueue {
    const OccInst *inst[kOccMaxInst];
    int ninst;
    int chunk;                   // targets per work item (a chunk of one bucket)
    int *chunk_off;              // [ninst * kOccBuckets + 1] first chunk of every bucket, then the total
    int *next;                   // the next chunk to take
};

}  // namespace fc2t2

struct fc2t2_plan_s {
    fc2t2_plan_desc desc;
    std::vector<double> poly;
    int D = 0, n = 0, rho = 0, P = 0, Pp = 0, nlev = 0;
    fc2t2::Level lev[fc2t2::kMaxLevels];
    int64_t G_total = 0;
    float lo_f = 0.f, hi_f = 0.f, scale0_f = 0.f;

    // device memory
    float *d_M = nullptr;         // [G_total][Pp]
    float *d_L = nullptr;         // [G_total][Pp]
    int C = 1;                    // channels
    float *d_hold = nullptr;      // [C][G0][Pp] finest-level locals of every channel (C > 1)
    bool expansion_held = false;  // fc2t2_expand's expansion is in d_L (C = 1) or d_hold
    // separable M2L: the levels above the finest run on a second stream beside the finest level's
    // passes (fork / join by events on the call's stream)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_sorted = nullptr;
    // batched calls: the plan's instances run on its own stream, forked from and joined to the
    // call's stream (instances of different plans overlap)
    cudaStream_t run = nullptr;
    cudaEvent_t ev_run_fork = nullptr, ev_run_done = nullptr;
    uint64_t batch_mark = 0;
    float *d_dtab = nullptr;      // [nlev][7^D][Pp]  scaled kernel derivatives
    int *d_scan_tmp = nullptr;    // block sums of the prefix scan
    int64_t scan_tmp_len = 0;
    int *d_flags = nullptr;       // [4] device error flags
    int2 *d_over = nullptr;       // [G0] P2M's overflow list: (cell, first chunk) of cells past the cap
    unsigned long long *d_over_ctr = nullptr;   // [2] the list's (entries << 32 | chunks), blocks done
    fc2t2::SortWork src, qry;
    void *d_mma_ops = nullptr;    // tensor-core M2L operator images (TF32 / BF16 modes)
    size_t mma_ops_bytes = 0;
    struct TcInfo {
        int enabled = 0, mode = 0, img_bytes = 0, ncomp = 1, kbytes = 0, nchunks = 0;
        int ncls = 1;      // target parity classes one CTA accumulates (sharing its moment views)
        int ksc = 0;       // K-step capacity class of the kernel variant
        int kh = 0;        // coefficients per epilogue column half
        int pnb = 0;       // accumulator columns per TMEM buffer (2 * ncls * kh)
        int n0[24] = {}, N[24] = {}, K[24] = {}, b_off[24] = {};
        int nbuf = 1, nbslots = 2, smem = 0, tmem_cols = 32;
        double mma_flops = 0.0;                       // tensor-core work issued per transform
        double mma_flops_level[fc2t2::kMaxLevels] = {};
        int64_t packed_bytes = 0;
        void *packed[fc2t2::kMaxLevels] = {};         // moments in the tensor-core layout, per level
        int level_ok[fc2t2::kMaxLevels] = {};         // 1: this level runs on the tensor cores
        alignas(64) unsigned char maps[fc2t2::kMaxLevels][2][128] = {};   // TMA descriptors (hi, lo)
    } tc;

    struct SepInfo {             // separable-kernel M2L (Gaussian, 3D)
        int enabled = 0, q4p = 0;
        std::vector<float> dt_host;   // [nlev][7][rho + 1] scaled 1D derivatives dt_o(j)
        float *d_t = nullptr;     // intermediate 4-indexed rows
        size_t t_bytes = 0;
        int64_t t_off[fc2t2::kMaxLevels][2][2] = {};   // [level][buffer][chain], in floats
        int seg[fc2t2::kMaxLevels] = {};
        size_t smem = 0;
        double flops = 0.0;
    } sep;

    struct OccInfo {             // M2L over occupied cells
        int enabled = 0;
        unsigned char *act = nullptr;   // [G_total] occupancy bytes
        int *list = nullptr;            // [G_total] occupied targets by (level, class)
        int *cnt = nullptr;             // [kOccBuckets]
        int *chunk_off = nullptr;       // [kOccMaxInst * kOccBuckets + 1] (a batched launch uses its first plan's)
        int *next = nullptr;            // [1]
        fc2t2::OccInst *d_inst = nullptr;
    } occ;

    // diagnostics: kernel launches per stage, and (when enabled) event pairs per stage
    mutable int64_t launches[FC2T2_NUM_STAGES] = {};
    bool profiling = false;
    struct EventPair { int stage; cudaEvent_t a, b; };
    std::vector<EventPair> pending;
    std::vector<cudaEvent_t> event_pool;
    double stage_ms[FC2T2_NUM_STAGES] = {};
};

namespace fc2t2 {

// error reporting (thread-local message)
fc2t2_status set_error(fc2t2_status st, const std::string &msg);
fc2t2_status check_cuda(cudaError_t e, const char *what);

// launchers (return cudaGetLastError() of the launch)
cudaError_t launch_bin_count(const fc2t2_plan_s *pl, cudaStream_t s, const float *x, int64_t n,
                             SortWork &w);
cudaError_t launch_scan(const fc2t2_plan_s *pl, cudaStream_t s, const int *in, int *out, int64_t n, int *tmp);
cudaError_t launch_reweight(const fc2t2_plan_s *pl, cudaStream_t s, const float *wt, int64_t n, SortWork &w);
cudaError_t launch_scatter(const fc2t2_plan_s *pl, cudaStream_t s, const float *x, const float *wt,
                           int64_t n, SortWork &w);
cudaError_t launch_p2m(const fc2t2_plan_s *pl, cudaStream_t s, const SortWork &w, float *M0);
cudaError_t launch_m2m(const fc2t2_plan_s *pl, cudaStream_t s, int level);
cudaError_t launch_m2l(const fc2t2_plan_s *pl, cudaStream_t s, int level);
cudaError_t launch_l2l(const fc2t2_plan_s *pl, cudaStream_t s, int level);
// val[perm[j]] = the series at point j; grad_times_w[perm[j]] = (or += with accumulate) its
// gradient times the point's record weight
cudaError_t launch_l2p(const fc2t2_plan_s *pl, cudaStream_t s, const SortWork &w, int64_t m,
                       float *val, float *grad_times_w, bool accumulate = false);
// the same without the finest level's L2L: the finest level's own M2L series plus level 1's
// complete local series, both about the point's cells (needs two or more levels)
cudaError_t launch_l2p_two(const fc2t2_plan_s *pl, cudaStream_t s, const SortWork &w, int64_t m,
                           float *val, float *grad_times_w, bool accumulate = false);
// ray integrals (3D): rays [R][8] = (origin, direction, t0, t1); y[q] = the integral of the
// finest-level series along ray q; ray2M adds ybar_q times the rays' moment integrals to M0
cudaError_t launch_ray_forward(const fc2t2_plan_s *pl, cudaStream_t s, const float *rays, int64_t R, float *y);
cudaError_t launch_ray2m(const fc2t2_plan_s *pl, cudaStream_t s, const float *rays, int64_t R, const float *ybar,
                         float *M0);
// the accessor: channels [C] of finest-level locals L (channel stride G0 * Pp) evaluated at the
// sorted points of w (out [C][m][K]) or on the meshgrid of axis[0..D-1] (out [C][n0][n1]([n2])[K])
cudaError_t launch_eval_sorted(const fc2t2_plan_s *pl, cudaStream_t s, const SortWork &w, int64_t m,
                               const float *L, int C, int what, float *out);
cudaError_t launch_eval_grid(const fc2t2_plan_s *pl, cudaStream_t s, const float *const *axis,
                             const int64_t *count, const float *L, int C, int what, float *out);
cudaError_t launch_tc_pack(const fc2t2_plan_s *pl, cudaStream_t s);
fc2t2_status build_sep(fc2t2_plan_s *pl, const std::vector<double> &dtab64);
// part 0: every level; 1: the finest level; 2: the levels above it
cudaError_t launch_m2l_sep(const fc2t2_plan_s *pl, cudaStream_t s, int part = 0);
cudaError_t launch_m2l_tc_all(const fc2t2_plan_s *pl, cudaStream_t s);
// occupancy of every level from the finest cells' counts of the sources and targets (NULL: every
// cell occupied), and the occupied targets' lists
cudaError_t launch_occupancy(const fc2t2_plan_s *pl, cudaStream_t s, const int *src_cnt, const int *tgt_cnt);
// M2L over occupied cells of every level of `nplan` plans of one dimension and order, one
// persistent launch (after launch_occupancy and M2M of each)
cudaError_t launch_m2l_occ(const fc2t2_plan_s *const *plans, int nplan, cudaStream_t s);
// register-resident M2M / L2L for orders <= 6 (return false when not applicable)
bool launch_m2m_reg(const fc2t2_plan_s *pl, cudaStream_t s, int level, cudaError_t &err);
bool launch_l2l_reg(const fc2t2_plan_s *pl, cudaStream_t s, int level, cudaError_t &err);
fc2t2_status build_tc_operators(fc2t2_plan_s *pl, const std::vector<double> &dtab64);

}  // namespace fc2t2
