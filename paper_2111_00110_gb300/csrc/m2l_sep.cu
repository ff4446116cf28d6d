// Separable M2L for the Gaussian kernel (Sec. 3: M2L as a convolution over the parity window;
// Sec. 3, future work on decomposable kernels: chained one-dimensional convolutions when the
// kernel's derivatives factor per dimension, as the Gaussian's do).
//
// With Dt_o(m) = prod_i dt_{o_i}(m_i), dt_o(j) = h^j g^(j)(o h) the scaled 1D derivatives, the
// M2L of one level
//     Lt[t](k) = sum_{s in IL(t)} sum_{|b| <= rho-|k|} (-1)^|k| Dt_{s-t}(k+b) Mt[s](b)
// is evaluated as three one-dimensional passes, one per axis, over a box of offsets.  The
// interaction set of a level above the finest is the parity window W minus the 3^3 hole H; it is
// split into three disjoint boxes (W\H) x W x W, H x (W\H) x W and H x H x (W\H), so every box
// sum holds only genuine interactions (no large near-field terms cancel).  At the finest level
// the set is the whole window W^3 (near field included).
//
// The total-degree truncation |k| + |b| <= rho couples the axes; the passes carry the unused
// degree as a slack index e.  With one pass done the coefficient is 4-indexed:
//   X:  T1(kx, by, bz, e)   = (-1)^kx sum_{ox} sum_{bx <= e}  dt_ox(kx+bx) Mt[t+ox](bx, by, bz)
//   Y:  T2(kx, ky, bz, e')  = (-1)^ky sum_{oy} sum_{by <= e'} dt_oy(ky+by) T1[t+oy](kx, by, bz, e'-by)
//   Z:  Lt(kx, ky, kz)      = (-1)^kz sum_{oz} sum_{bz}       dt_oz(kz+bz) T2[t+oz](kx, ky, bz, rho-|k|-bz)
// with kx + by + bz + e <= rho and kx + ky + bz + e' <= rho.  A 4-indexed row holds C(rho+4, 4)
// values (210 at order 6), grouped by its two leading indices; each group is a triangle.
//
// Every pass is a line convolution: a CTA stages a segment of one grid line (up to 64 target
// cells at the finest level, 32 above it, plus the source cells their windows reach: 2 on each
// side at the finest level, 3 above it) of its input rows in shared memory with coalesced loads,
// computes its outputs from shared memory (a thread per pair of targets and task at the finest
// level, per target and task above it), and writes the segment's output rows coalesced.  The
// passes move far fewer flops than the dense M2L; their cost is instruction issue and the
// intermediate rows' memory traffic.  The finest level runs in one launch per pass, the levels
// above it in another.
#include <algorithm>
#include <cstring>

#include "dispatch.cuh"
#include "fc2t2_internal.cuh"

namespace fc2t2 {

// threads per CTA: 512 at orders 7-8, whose passes run one long-segment CTA per multiprocessor
// (more warps to hide latency: order-8 M2L 2.72 -> 2.55 ms per step), 256 below (at order 6, 512
// threads cost 14 % of the step)
__host__ __device__ constexpr int sep_threads(int rho) { return rho >= 7 ? 512 : 256; }
// input rows a warp loads at once while staging.  At orders <= 6, enough for one round (segments
// of up to 64 cells plus 2 halo cells on each side at the finest level, 32 plus 3 above it): every
// warp issues all of its loads before the first one returns (order-6 M2L 0.923 -> 0.876 ms per
// step against four rows a round).  At orders 7-8 the 16 warps of a CTA load four rows a round,
// one round but for the last four rows of a 64-cell segment (five rows each, order-8 M2L was
// 1.7 % slower: more registers at one CTA per multiprocessor).
__host__ __device__ constexpr int stage_rows(int rho, bool finest) {
    return rho >= 7 ? 4 : ((finest ? 68 : 38) + sep_threads(rho) / 32 - 1) / (sep_threads(rho) / 32);
}

__host__ __device__ constexpr int q4count(int rho) { return (rho + 1) * (rho + 2) * (rho + 3) * (rho + 4) / 24; }
__host__ __device__ constexpr int tri_count(int r) { return (r + 1) * (r + 2) / 2; }
// entry (i2, i3), i2 + i3 <= r, of a triangle stored row by row (row i2 holds r - i2 + 1 values)
__host__ __device__ constexpr int tri_idx(int r, int i2, int i3) { return i2 * (r + 1) - i2 * (i2 - 1) / 2 + i3; }

struct SepLevel {
    const float *in0, *in1;   // inputs of the pass (in1: second chain, levels above the finest)
    float *out0, *out1;       // outputs (out1: second chain of passes X and Y above the finest)
    int n;                    // cells per dimension
    int seg, nseg;            // target cells per CTA along the pass axis, segments per line
    int block0;
};

constexpr int kSepMaxSlots = 192;

struct SepArgs {
    SepLevel lv[kMaxLevels];
    int nlev;
    float dt[kMaxLevels][7][kMaxOrder + 1];   // dt_o(j) of each level of the launch, o = -3..3
    int goff[(kMaxOrder + 1) * (kMaxOrder + 1)];   // offset of group (i0, i1) in a 4-indexed row
    int nslot;                                     // task slots of the table (pairs plus empty slots)
    char2 pair[kSepMaxSlots];                      // task pair (i, j), i + j <= rho, by slot; (-1, -1): none
    int ahead;   // finest level: a block prefetches into L2 the input rows of block + ahead (0: none)
};

// bulk prefetch of `bytes` (a multiple of 16) from a 16-byte aligned global address into L2
__device__ __forceinline__ void prefetch_l2(const float *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(bytes) : "memory");
}

// In shared memory rows are padded to an odd number of floats so that the 32 lanes of a warp,
// which work on 32 consecutive cells, read 32 different banks.
__host__ __device__ constexpr int odd_pitch(int p) { return p | 1; }

template <int AXIS>
__device__ __forceinline__ void line_geometry(int line, int n, int64_t &base, int64_t &stride) {
    const int u = line % n, v = line / n;
    if (AXIS == 0) { base = (int64_t)n * (u + (int64_t)n * v); stride = 1; }
    else if (AXIS == 1) { base = (int64_t)u + (int64_t)n * n * v; stride = n; }
    else { base = (int64_t)u + (int64_t)n * v; stride = (int64_t)n * n; }
}

// The parity window of a target with coordinate t along the axis is [-3, 2] (t odd) or [-2, 3]
// (t even).  An even target t and the odd target t + 1 therefore read the same six source rows
// t - 2 .. t + 3: at the finest level a task owns such a pair of targets, loads each of the six rows once and applies
// it to both, with offset k - 2 for the even target and k - 3 for the odd one (k = 0..5).  So
// no lane computes an offset outside its window, and which offsets lie in the hole |o| <= 1 is
// known per row at compile time (or uniformly across the warp).

// offset sets of a pass: the whole window, the window minus the hole, the hole
enum { kSetW = 0, kSetWH = 1, kSetH = 2 };
__host__ __device__ constexpr bool in_set(int set, int off) {
    return set == kSetW ? true : set == kSetH ? (off >= -1 && off <= 1) : (off < -1 || off > 1);
}

// dt_o(j) of the even target (offset k - 2) and of the odd one (offset k - 3) for row k
__device__ __forceinline__ const float *dt_even(const float *s_dt, int k) { return s_dt + (k + 1) * (kMaxOrder + 1); }
__device__ __forceinline__ const float *dt_odd(const float *s_dt, int k) { return s_dt + k * (kMaxOrder + 1); }

// Per-task bodies, specialised on the task's degree budget R = rho - i - j (the two fixed
// indices of the task), so that every loop has exactly the trip count the budget allows.

// pass X, task (target pair tl, tl + 1; by, bz): T1(kx, by, bz, e) for kx + e <= R as running
// sums over e.  At the finest level the window goes to out0; above it the window minus the hole
// goes to out0 and the hole to out1.
template <int RHO, int R, bool FINEST>
__device__ __forceinline__ void sep_task_x(const float *in0, int tl, int by, int bz, const float *s_dt,
                                           const int *s_goff, float *out0, float *out1) {
    constexpr int PIN = odd_pitch(pad4(ncoef(3, RHO)));
    constexpr int POUT = odd_pitch(pad4(q4count(RHO)));
    float ae0[R + 1], ae1[R + 1], ao0[R + 1], ao1[R + 1];   // even / odd target, out0 / out1
    int g[R + 1];
#pragma unroll
    for (int kx = 0; kx <= R; ++kx) {
        ae0[kx] = ae1[kx] = ao0[kx] = ao1[kx] = 0.0f;
        g[kx] = s_goff[kx * (RHO + 1) + bz];
    }
    // e outermost: the inputs Mt[t-2..t+3](e, by, bz) feed every kx <= R - e
#pragma unroll
    for (int e = 0; e <= R; ++e) {
        float v[6];
        const int col = gidx3(e, by, bz);
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = in0[(tl + k) * PIN + col];
#pragma unroll
        for (int kx = 0; kx + e <= R; ++kx) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float te = dt_even(s_dt, k)[kx + e] * v[k];
                const float to = dt_odd(s_dt, k)[kx + e] * v[k];
                if (FINEST || in_set(kSetWH, k - 2)) ae0[kx] += te;
                else ae1[kx] += te;
                if (FINEST || in_set(kSetWH, k - 3)) ao0[kx] += to;
                else ao1[kx] += to;
            }
            const float sg = (kx & 1) ? -1.0f : 1.0f;
            const int idx = g[kx] + tri_idx(RHO - kx - bz, by, e);
            out0[tl * POUT + idx] = sg * ae0[kx];
            out0[(tl + 1) * POUT + idx] = sg * ao0[kx];
            if (!FINEST) {
                out1[tl * POUT + idx] = sg * ae1[kx];
                out1[(tl + 1) * POUT + idx] = sg * ao1[kx];
            }
        }
    }
}

// pass Y: adds sum_{oy in SET} sum_{by <= e'} dt_oy(ky+by) T1[t+oy](kx, by, bz, e'-by) into
// acc(ky, e') of both targets.  Each row element T1(by, f) is loaded once and feeds every
// (ky, e' = by + f) of both accumulators.  The row loop is not unrolled (unrolled, the
// budget-specialised bodies overflow the instruction cache); its hole tests are warp-uniform.
template <int RHO, int R, int SET>
__device__ __forceinline__ void sep_accum_y(float (&ae)[tri_count(R)], float (&ao)[tri_count(R)], const float *inb,
                                            int tl, int gin, const float *s_dt) {
    constexpr int PIN = odd_pitch(pad4(q4count(RHO)));
#pragma unroll 1
    for (int k = 0; k < 6; ++k) {
        const bool ue = in_set(SET, k - 2), uo = in_set(SET, k - 3);
        if (!ue && !uo) continue;
        const float *row = inb + (tl + k) * PIN + gin;
        float de[R + 1], dd[R + 1];
#pragma unroll
        for (int j = 0; j <= R; ++j) {
            de[j] = ue ? dt_even(s_dt, k)[j] : 0.0f;
            dd[j] = uo ? dt_odd(s_dt, k)[j] : 0.0f;
        }
#pragma unroll
        for (int by = 0; by <= R; ++by)
#pragma unroll
            for (int f = 0; by + f <= R; ++f) {
                const float x = row[tri_idx(R, by, f)];
#pragma unroll
                for (int ky = 0; ky + by + f <= R; ++ky) {
                    const int a = tri_idx(R, ky, by + f);
                    ae[a] = fmaf(de[ky + by], x, ae[a]);
                    ao[a] = fmaf(dd[ky + by], x, ao[a]);
                }
            }
    }
}

// T2(kx, ky, bz, e') for ky + e' <= R, stored at (bz, f = R - ky - e') of group (kx, ky) so that
// pass Z indexes it by (bz, kz)
template <int RHO, int R>
__device__ __forceinline__ void sep_store_y(float (&acc)[tri_count(R)], float *outb, int kx, int bz,
                                            const int *s_goff) {
#pragma unroll
    for (int ky = 0; ky <= R; ++ky) {
        const float sg = (ky & 1) ? -1.0f : 1.0f;
        const int rg = RHO - kx - ky;
        float *dst = outb + s_goff[kx * (RHO + 1) + ky];
#pragma unroll
        for (int ep = 0; ky + ep <= R; ++ep) dst[tri_idx(rg, bz, R - ky - ep)] = sg * acc[tri_idx(R, ky, ep)];
    }
}

// pass Y, task (target pair; kx, bz), one chain.  Finest level: the window on in0.  Above it (the
// chains are computed one after the other into the same shared-memory rows), chain 0 (U) = the
// window on in0 plus the window minus the hole on in1, chain 1 (V) = the hole on in1.
template <int RHO, int R, bool FINEST>
__device__ __forceinline__ void sep_task_y(const float *in0, const float *in1, int tl, int kx, int bz,
                                           const float *s_dt, const int *s_goff, float *out, int chain) {
    constexpr int POUT = odd_pitch(pad4(q4count(RHO)));
    const int gin = s_goff[kx * (RHO + 1) + bz];
    float ae[tri_count(R)], ao[tri_count(R)];
#pragma unroll
    for (int i = 0; i < tri_count(R); ++i) ae[i] = ao[i] = 0.0f;
    if (chain == 0) {
        sep_accum_y<RHO, R, kSetW>(ae, ao, in0, tl, gin, s_dt);
        if (!FINEST) sep_accum_y<RHO, R, kSetWH>(ae, ao, in1, tl, gin, s_dt);
    } else {
        sep_accum_y<RHO, R, kSetH>(ae, ao, in1, tl, gin, s_dt);
    }
    sep_store_y<RHO, R>(ae, out + tl * POUT, kx, bz, s_goff);
    sep_store_y<RHO, R>(ao, out + (tl + 1) * POUT, kx, bz, s_goff);
}

// pass Z: adds sum_{oz in SET} sum_{bz} dt_oz(kz+bz) T2[t+oz](kx, ky, bz, f = kz) into acc(kz) of
// both targets
template <int RHO, int R, int SET>
__device__ __forceinline__ void sep_accum_z(float (&ae)[R + 1], float (&ao)[R + 1], const float *inb, int tl, int gin,
                                            const float *s_dt) {
    constexpr int PIN = odd_pitch(pad4(q4count(RHO)));
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const bool ue = in_set(SET, k - 2), uo = in_set(SET, k - 3);
        if (!ue && !uo) continue;
        const float *row = inb + (tl + k) * PIN + gin;
#pragma unroll
        for (int bz = 0; bz <= R; ++bz)
#pragma unroll
            for (int kz = 0; kz + bz <= R; ++kz) {
                const float x = row[tri_idx(R, bz, kz)];
                if (ue) ae[kz] = fmaf(dt_even(s_dt, k)[kz + bz], x, ae[kz]);
                if (uo) ao[kz] = fmaf(dt_odd(s_dt, k)[kz + bz], x, ao[kz]);
            }
    }
}

// pass Z, task (target pair; kx, ky): Lt(kx, ky, kz) for kz <= R; the window on in0, plus the
// window minus the hole on in1 above the finest level
template <int RHO, int R, bool FINEST>
__device__ __forceinline__ void sep_task_z(const float *in0, const float *in1, int tl, int kx, int ky,
                                           const float *s_dt, const int *s_goff, float *out0) {
    constexpr int POUT = odd_pitch(pad4(ncoef(3, RHO)));
    const int gin = s_goff[kx * (RHO + 1) + ky];
    float ae[R + 1], ao[R + 1];
#pragma unroll
    for (int i = 0; i <= R; ++i) ae[i] = ao[i] = 0.0f;
    sep_accum_z<RHO, R, kSetW>(ae, ao, in0, tl, gin, s_dt);
    if (!FINEST) sep_accum_z<RHO, R, kSetWH>(ae, ao, in1, tl, gin, s_dt);
#pragma unroll
    for (int kz = 0; kz <= R; ++kz) {
        const float sg = (kz & 1) ? -1.0f : 1.0f;
        out0[tl * POUT + gidx3(kx, ky, kz)] = sg * ae[kz];
        out0[(tl + 1) * POUT + gidx3(kx, ky, kz)] = sg * ao[kz];
    }
}

template <int RHO, int AXIS, bool FINEST, int R>
__device__ __forceinline__ void sep_task(const float *in0, const float *in1, int tl, int2 pr, const float *s_dt,
                                         const int *s_goff, float *out0, float *out1, int chain) {
    if (AXIS == 0) sep_task_x<RHO, R, FINEST>(in0, tl, pr.x, pr.y, s_dt, s_goff, out0, out1);
    else if (AXIS == 1) sep_task_y<RHO, R, FINEST>(in0, in1, tl, pr.x, pr.y, s_dt, s_goff, out0, chain);
    else sep_task_z<RHO, R, FINEST>(in0, in1, tl, pr.x, pr.y, s_dt, s_goff, out0);
}

// ---- Levels above the finest: a task owns one target.  There the two targets of a pair would
// use different hole rows (a third of the paired work would be zeros), so a thread works on one
// target over the seven offsets -3..3 and zeroes the input of the one outside its window:
// [-3, 2] for odd t, [-2, 3] for even t.  The segment is staged with three source rows on each
// side (row o of target tl is source t + o - 3).
__device__ __forceinline__ bool excluded(int off, int par) { return par ? off == 3 : off == -3; }

// pass X, task (t, by, bz): T1(kx, by, bz, e) for kx + e <= R as running sums over e; the window
// minus the hole goes to out0 and the hole to out1.
template <int RHO, int R, bool FINEST>
__device__ __forceinline__ void cell_task_x(const float *in0, int tl, int par, int by, int bz, const float *s_dt,
                                           const int *s_goff, float *out0, float *out1) {
    constexpr int PIN = odd_pitch(pad4(ncoef(3, RHO)));
    float a0[R + 1], a1[R + 1];
    int g[R + 1];
#pragma unroll
    for (int kx = 0; kx <= R; ++kx) { a0[kx] = 0.0f; a1[kx] = 0.0f; g[kx] = s_goff[kx * (RHO + 1) + bz]; }
    // e outermost: the inputs Mt[t+o](e, by, bz) of the seven offsets feed every kx <= R - e
#pragma unroll
    for (int e = 0; e <= R; ++e) {
        float v[7];
        const int col = gidx3(e, by, bz);
#pragma unroll
        for (int o = 0; o < 7; ++o) v[o] = excluded(o - 3, par) ? 0.0f : in0[(tl + o) * PIN + col];
#pragma unroll
        for (int kx = 0; kx + e <= R; ++kx) {
#pragma unroll
            for (int o = 0; o < 7; ++o) {
                const float term = s_dt[o * (kMaxOrder + 1) + kx + e] * v[o];
                if (FINEST || in_set(kSetWH, o - 3)) a0[kx] += term;
                else a1[kx] += term;
            }
            const float sg = (kx & 1) ? -1.0f : 1.0f;
            const int idx = g[kx] + tri_idx(RHO - kx - bz, by, e);
            out0[idx] = sg * a0[kx];
            if (!FINEST) out1[idx] = sg * a1[kx];
        }
    }
}

// pass Y: adds sum_{oy in SET} sum_{by <= e'} dt_oy(ky+by) T1[t+oy](kx, by, bz, e'-by) into
// acc(ky, e'), one offset at a time.
template <int RHO, int R, int SET>
__device__ __forceinline__ void cell_accum_y(float (&acc)[tri_count(R)], const float *inb, int tl, int par, int gin,
                                            const float *s_dt) {
    constexpr int PIN = odd_pitch(pad4(q4count(RHO)));
#pragma unroll 1
    for (int o = 0; o < 7; ++o) {
        if (!in_set(SET, o - 3)) continue;
        const bool ex = excluded(o - 3, par);
        const float *row = inb + (tl + o) * PIN + gin;
        float tri[tri_count(R)], dr[R + 1];
#pragma unroll
        for (int i = 0; i < tri_count(R); ++i) tri[i] = row[i];
#pragma unroll
        for (int j = 0; j <= R; ++j) dr[j] = ex ? 0.0f : s_dt[o * (kMaxOrder + 1) + j];   // excluded: weight 0
#pragma unroll
        for (int ky = 0; ky <= R; ++ky)
#pragma unroll
            for (int ep = 0; ky + ep <= R; ++ep) {
                float sacc = acc[tri_idx(R, ky, ep)];
#pragma unroll
                for (int by = 0; by <= ep; ++by) sacc = fmaf(dr[ky + by], tri[tri_idx(R, by, ep - by)], sacc);
                acc[tri_idx(R, ky, ep)] = sacc;
            }
    }
}

// pass Y, task (t, kx, bz), one chain (computed one after the other into the same shared-memory
// rows): chain 0 (U) = the window on in0 plus the window minus the hole on in1, chain 1 (V) = the
// hole on in1.
template <int RHO, int R, bool FINEST>
__device__ __forceinline__ void cell_task_y(const float *in0, const float *in1, int tl, int par, int kx, int bz,
                                           const float *s_dt, const int *s_goff, float *out, int chain) {
    const int gin = s_goff[kx * (RHO + 1) + bz];
    float acc[tri_count(R)];
#pragma unroll
    for (int i = 0; i < tri_count(R); ++i) acc[i] = 0.0f;
    if (chain == 0) {
        cell_accum_y<RHO, R, kSetW>(acc, in0, tl, par, gin, s_dt);
        if (!FINEST) cell_accum_y<RHO, R, kSetWH>(acc, in1, tl, par, gin, s_dt);
    } else {
        cell_accum_y<RHO, R, kSetH>(acc, in1, tl, par, gin, s_dt);
    }
    sep_store_y<RHO, R>(acc, out, kx, bz, s_goff);
}

// pass Z: adds sum_{oz in SET} sum_{bz} dt_oz(kz+bz) T2[t+oz](kx, ky, bz, f = kz) into acc(kz)
template <int RHO, int R, int SET>
__device__ __forceinline__ void cell_accum_z(float (&acc)[R + 1], const float *inb, int tl, int par, int gin,
                                            const float *s_dt) {
    constexpr int PIN = odd_pitch(pad4(q4count(RHO)));
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        if (!in_set(SET, o - 3)) continue;
        const bool ex = excluded(o - 3, par);
        const float *row = inb + (tl + o) * PIN + gin;
        float tri[tri_count(R)], dr[R + 1];
#pragma unroll
        for (int i = 0; i < tri_count(R); ++i) tri[i] = row[i];
#pragma unroll
        for (int j = 0; j <= R; ++j) dr[j] = ex ? 0.0f : s_dt[o * (kMaxOrder + 1) + j];   // excluded: weight 0
#pragma unroll
        for (int kz = 0; kz <= R; ++kz) {
            float sacc = acc[kz];
#pragma unroll
            for (int bz = 0; bz + kz <= R; ++bz) sacc = fmaf(dr[kz + bz], tri[tri_idx(R, bz, kz)], sacc);
            acc[kz] = sacc;
        }
    }
}

// pass Z, task (t, kx, ky): Lt(kx, ky, kz) for kz <= R; the window on in0 plus the window minus
// the hole on in1
template <int RHO, int R, bool FINEST>
__device__ __forceinline__ void cell_task_z(const float *in0, const float *in1, int tl, int par, int kx, int ky,
                                           const float *s_dt, const int *s_goff, float *out0) {
    const int gin = s_goff[kx * (RHO + 1) + ky];
    float acc[R + 1];
#pragma unroll
    for (int i = 0; i <= R; ++i) acc[i] = 0.0f;
    cell_accum_z<RHO, R, kSetW>(acc, in0, tl, par, gin, s_dt);
    if (!FINEST) cell_accum_z<RHO, R, kSetWH>(acc, in1, tl, par, gin, s_dt);
#pragma unroll
    for (int kz = 0; kz <= R; ++kz) out0[gidx3(kx, ky, kz)] = ((kz & 1) ? -1.0f : 1.0f) * acc[kz];
}

template <int RHO, int AXIS, bool FINEST, int R>
__device__ __forceinline__ void cell_task(const float *in0, const float *in1, int tl, int par, int2 pr,
                                         const float *s_dt, const int *s_goff, float *out0, float *out1, int chain) {
    if (AXIS == 0) cell_task_x<RHO, R, FINEST>(in0, tl, par, pr.x, pr.y, s_dt, s_goff, out0, out1);
    else if (AXIS == 1) cell_task_y<RHO, R, FINEST>(in0, in1, tl, par, pr.x, pr.y, s_dt, s_goff, out0, chain);
    else cell_task_z<RHO, R, FINEST>(in0, in1, tl, par, pr.x, pr.y, s_dt, s_goff, out0);
}

template <int RHO, int AXIS>
struct SepPitch {
    static constexpr int in = AXIS == 0 ? pad4(ncoef(3, RHO)) : pad4(q4count(RHO));    // global row, floats
    static constexpr int out = AXIS == 2 ? pad4(ncoef(3, RHO)) : pad4(q4count(RHO));
    static constexpr int sin = odd_pitch(in), sout = odd_pitch(out);                 // shared-memory row
};

// Three CTAs of 256 threads per multiprocessor at orders <= 6 (registers permitting, without
// spills); one CTA of 512 threads at orders 7-8 (their long segments' shared memory).
template <int RHO, int AXIS, bool FINEST>
__global__ void __launch_bounds__(sep_threads(RHO), RHO >= 7 ? 1 : 3) k_m2l_sep(const SepArgs args) {
    constexpr int kSepThreads = sep_threads(RHO);
    constexpr int P = ncoef(3, RHO);
    using Pt = SepPitch<RHO, AXIS>;
    constexpr bool TWO_IN = !FINEST && AXIS > 0;
    constexpr bool TWO_OUT = !FINEST && AXIS == 0;       // pass X fills both chains at once
    constexpr int NCHAIN = (!FINEST && AXIS == 1) ? 2 : 1;   // pass Y: one chain after the other
    extern __shared__ float sm[];
    // the finest level is launched alone (its tables at compile-time offsets); the levels above
    // it share a launch, blocks ordered level by level
    int lvl = 0;
    if (!FINEST) {
#pragma unroll
        for (int i = 1; i < kMaxLevels; ++i)
            if (i < args.nlev && (int)blockIdx.x >= args.lv[i].block0) lvl = i;
    }
    const SepLevel lv = args.lv[lvl];
    const int n = lv.n;
    const int bl = (int)blockIdx.x - lv.block0;
    const int seg = bl % lv.nseg, line = bl / lv.nseg;
    int64_t base, stride;
    line_geometry<AXIS>(line, n, base, stride);
    const int t0 = seg * lv.seg;
    const int nt = min(lv.seg, n - t0);
    // sources t0 - 2 .. t0 + nt + 1 for target pairs (finest), t0 - 3 .. t0 + nt + 2 above
    constexpr int HALO = FINEST ? 2 : 3;
    const int nin = nt + 2 * HALO;

    // finest level at orders 7-8: the last warp asks L2 for the input rows of the block `ahead`
    // blocks on (a wave later), so that its staging finds them there (order-8 M2L 2.56 -> 2.40 ms
    // per step; at order 6, whose warps load all their rows in one round, it cost 2 %)
    if (FINEST && RHO >= 7 && args.ahead > 0 && threadIdx.x >= kSepThreads - 32) {
        const int b2 = bl + args.ahead;
        if (b2 < n * n * lv.nseg) {
            const int seg2 = b2 % lv.nseg, line2 = b2 / lv.nseg;
            int64_t base2, stride2;
            line_geometry<AXIS>(line2, n, base2, stride2);
            const int t02 = seg2 * lv.seg;
            const int lo = max(0, t02 - HALO), hi = min(n, t02 + min(lv.seg, n - t02) + HALO);
            for (int r = lo + (int)(threadIdx.x & 31); r < hi; r += 32)
                prefetch_l2(lv.in0 + (base2 + (int64_t)r * stride2) * Pt::in, Pt::in * (unsigned)sizeof(float));
        }
    }

    float *in0 = sm;
    float *in1 = in0 + nin * Pt::sin;
    float *out0 = in1 + (TWO_IN ? nin * Pt::sin : 0);
    float *out1 = out0 + nt * Pt::sout;

    // the level's derivative table and the group / pair tables live in the launch parameters
    const float *s_dt = &args.dt[lvl][0][0];
    const int *s_goff = args.goff;
    const char2 *s_pair = args.pair;

    // stage the input rows of sources t0 - HALO .. t0 + nt + HALO - 1 (zero outside the grid): a
    // warp per row, lanes across the row (coalesced scalar loads, conflict-free stores into the odd-pitch
    // rows), stage_rows(RHO, FINEST) rows per warp in flight
    bool nonzero = false;              // any staged input value nonzero (the CTA's outputs depend on no other)
    {
        constexpr int W = kSepThreads / 32, CPL = (Pt::in + 31) / 32;   // columns per lane
        constexpr int kStageRows = stage_rows(RHO, FINEST);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll 1
        for (int src = 0; src < (TWO_IN ? 2 : 1); ++src) {
            const float *gsrc = src == 0 ? lv.in0 : lv.in1;
            float *sdst = src == 0 ? in0 : in1;
#pragma unroll 1
            for (int r0 = warp * kStageRows; r0 < nin; r0 += W * kStageRows) {   // one round
                float buf[kStageRows][CPL];
#pragma unroll
                for (int u = 0; u < kStageRows; ++u) {
                    const int srow = t0 - HALO + r0 + u;
                    const bool ok = r0 + u < nin && srow >= 0 && srow < n;
                    const float *g = gsrc + (base + (int64_t)srow * stride) * Pt::in;
#pragma unroll
                    for (int k = 0; k < CPL; ++k) {
                        const int c = lane + 32 * k;
                        buf[u][k] = (ok && c < Pt::in) ? __ldg(g + c) : 0.0f;
                        if (AXIS == 0) nonzero |= buf[u][k] != 0.0f;
                    }
                }
#pragma unroll
                for (int u = 0; u < kStageRows; ++u) {
                    if (r0 + u >= nin) break;
                    float *d = sdst + (r0 + u) * Pt::sin;
#pragma unroll
                    for (int k = 0; k < CPL; ++k) {
                        const int c = lane + 32 * k;
                        if (c < Pt::in) d[c] = buf[u][k];
                    }
                }
            }
        }
    }
    // Pass X: a segment whose staged moments are all zero (no source within the windows of its
    // targets -- much of the grid for clustered points) has zero outputs: write them and skip the
    // arithmetic.  (Passes Y and Z read the window-dilated outputs of the pass before, which are
    // zero on few whole segments; they skip the test.)
    if (AXIS != 0) __syncthreads();
    else if (!__syncthreads_or(nonzero)) {
        constexpr int W = kSepThreads / 32, CPL = (Pt::out + 31) / 32;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        constexpr int NOUT = (TWO_OUT || NCHAIN > 1) ? 2 : 1;
#pragma unroll 1
        for (int o = 0; o < NOUT; ++o) {
            float *gout = o == 0 ? lv.out0 : lv.out1;
#pragma unroll 1
            for (int rr = warp; rr < nt; rr += W) {
                float *g0 = gout + (base + (int64_t)(t0 + rr) * stride) * Pt::out;
#pragma unroll
                for (int k = 0; k < CPL; ++k) {
                    const int c = lane + 32 * k;
                    if (c < Pt::out) g0[c] = 0.0f;
                }
            }
        }
        return;
    }

    // finest level: target pairs (2 tp, 2 tp + 1) of the segment (t0 and nt are even); a warp's
    // lanes cover 32 / np task slots, whose pairs the table groups by budget.  Above it: one
    // target per task, 32 / nt slots per warp.
    const int np = FINEST ? nt >> 1 : nt;
    const int lg_np = __ffs(np) - 1;   // np is a power of two
#pragma unroll 1
    for (int chain = 0; chain < NCHAIN; ++chain) {
        for (int task = threadIdx.x; task < np * args.nslot; task += blockDim.x) {
            const char2 pc = s_pair[task >> lg_np];
            const int2 pr = make_int2(pc.x, pc.y);   // (-1, -1): an empty slot (no budget matches)
            if constexpr (FINEST) {
                const int tl = 2 * (task & (np - 1));
                switch (RHO - pr.x - pr.y) {
#define FC2T2_SEP_R(R_)                                                                                 \
    case R_:                                                                                            \
        if constexpr (R_ <= RHO) sep_task<RHO, AXIS, FINEST, R_>(in0, in1, tl, pr, s_dt, s_goff, out0, out1, chain); \
        break;
                    FC2T2_SEP_R(0) FC2T2_SEP_R(1) FC2T2_SEP_R(2) FC2T2_SEP_R(3) FC2T2_SEP_R(4)
                    FC2T2_SEP_R(5) FC2T2_SEP_R(6) FC2T2_SEP_R(7) FC2T2_SEP_R(8)
#undef FC2T2_SEP_R
                    default: break;
                }
            } else {
                const int tl = task & (np - 1);
                const int par = (t0 + tl) & 1;
                float *o0 = out0 + tl * Pt::sout, *o1 = out1 + tl * Pt::sout;
                switch (RHO - pr.x - pr.y) {
#define FC2T2_SEP_R(R_)                                                                                 \
    case R_:                                                                                            \
        if constexpr (R_ <= RHO) cell_task<RHO, AXIS, false, R_>(in0, in1, tl, par, pr, s_dt, s_goff, o0, o1, chain); \
        break;
                    FC2T2_SEP_R(0) FC2T2_SEP_R(1) FC2T2_SEP_R(2) FC2T2_SEP_R(3) FC2T2_SEP_R(4)
                    FC2T2_SEP_R(5) FC2T2_SEP_R(6) FC2T2_SEP_R(7) FC2T2_SEP_R(8)
#undef FC2T2_SEP_R
                    default: break;
                }
            }
        }
        __syncthreads();

        // write the segment's output rows, a warp per row (padding columns of Lt rows are zero;
        // padding of the 4-indexed rows is never read)
        {
            constexpr int W = kSepThreads / 32, CPL = (Pt::out + 31) / 32;
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            float *gout0 = chain == 0 ? lv.out0 : lv.out1;
#pragma unroll 1
            for (int rr = warp; rr < nt; rr += W) {
                float *g0 = gout0 + (base + (int64_t)(t0 + rr) * stride) * Pt::out;
                const float *s0 = out0 + rr * Pt::sout;
#pragma unroll
                for (int k = 0; k < CPL; ++k) {
                    const int c = lane + 32 * k;
                    if (c < Pt::out) g0[c] = (AXIS == 2 && c >= P) ? 0.0f : s0[c];
                }
                if (TWO_OUT) {
                    float *g1 = lv.out1 + (base + (int64_t)(t0 + rr) * stride) * Pt::out;
                    const float *s1 = out1 + rr * Pt::sout;
#pragma unroll
                    for (int k = 0; k < CPL; ++k) {
                        const int c = lane + 32 * k;
                        if (c < Pt::out) g1[c] = s1[c];
                    }
                }
            }
        }
        if (NCHAIN > 1) __syncthreads();   // the next chain reuses the output rows
    }
}

namespace {

// shared memory of one CTA of a pass for `seg` target cells
size_t sep_smem(int axis, int seg, bool finest, int in_pitch, int out_pitch) {
    const int nin = seg + (finest ? 4 : 6);
    // two input chains above the finest level (passes Y, Z); two output rows per cell only for
    // pass X (pass Y computes its two chains one after the other into the same rows)
    const bool two = !finest && axis > 0, two_out = !finest && axis == 0;
    const size_t f = (size_t)nin * odd_pitch(in_pitch) * (two ? 2 : 1) +
                     (size_t)seg * odd_pitch(out_pitch) * (two_out ? 2 : 1);
    return f * sizeof(float);
}

}  // namespace

fc2t2_status build_sep(fc2t2_plan_s *pl, const std::vector<double> &dtab64) {
    const int rho = pl->rho, P = pl->P;
    const int Q4p = pad4(q4count(rho));
    pl->sep.q4p = Q4p;
    std::vector<float> dt((size_t)pl->nlev * 7 * (rho + 1));
    for (int l = 0; l < pl->nlev; ++l)
        for (int o = 0; o < 7; ++o)
            for (int j = 0; j <= rho; ++j)   // Dt at offset (o - 3, 0, 0), exponent (j, 0, 0)
                dt[((size_t)l * 7 + o) * (rho + 1) + j] =
                    (float)dtab64[((size_t)l * 343 + (size_t)o + 7 * 3 + 49 * 3) * P + gidx3(j, 0, 0)];
    pl->sep.dt_host = dt;   // passed to the kernels in their launch parameters
    // intermediate rows: pass X writes buffer 0, pass Y reads it and writes buffer 1 (a CTA's
    // halo rows belong to neighbouring segments, so a pass never writes its own input), pass Z
    // reads buffer 1; one chain at the finest level, two above it
    int64_t cells = 0;
    for (int l = 0; l < pl->nlev; ++l) cells += pl->lev[l].G * (l == 0 ? 1 : 2);
    pl->sep.t_bytes = (size_t)cells * 2 * Q4p * sizeof(float);
    if (cudaMalloc(&pl->sep.d_t, pl->sep.t_bytes) != cudaSuccess) {
        cudaGetLastError();
        pl->sep.d_t = nullptr;
        return set_error(FC2T2_ERR_OOM, "cudaMalloc failed for the separable M2L intermediates");
    }
    int64_t off = 0;
    for (int buf = 0; buf < 2; ++buf)
        for (int l = 0; l < pl->nlev; ++l)
            for (int chain = 0; chain < (l == 0 ? 1 : 2); ++chain) {
                pl->sep.t_off[l][buf][chain] = off;
                off += pl->lev[l].G * Q4p;
            }
    // segment length per level: the longest of 64 (finest level only: a warp's lanes then hold its
    // 32 target pairs), 32, 16, 8, 4 cells that keeps every pass's CTA within 116 KB of shared
    // memory at orders <= 6 (two or three CTAs per multiprocessor) and 220 KB at orders 7-8 (one:
    // there the longer segments' smaller halo share outweighs the lost CTA, order 8 M2L 2.99 ->
    // 2.72 ms per step); segments shorter than a warp split warps between tasks.  The plan's
    // `tile` caps the finest level's length (a tuning knob)
    size_t max_smem = 0;
    const size_t cap = (size_t)(pl->rho >= 7 ? 220 : 116) * 1024;
    for (int l = 0; l < pl->nlev; ++l) {
        const int n = pl->lev[l].n;
        int seg = 4;
        for (int cand : {64, 32, 16, 8}) {
            if (cand > n || (cand == 64 && l != 0)) continue;
            if (l == 0 && pl->desc.tile > 0 && cand > pl->desc.tile) continue;
            bool fits = true;
            for (int axis = 0; axis < 3; ++axis) {
                const int ip = axis == 0 ? pl->Pp : Q4p, op = axis == 2 ? pl->Pp : Q4p;
                if (sep_smem(axis, cand, l == 0, ip, op) > cap) fits = false;
            }
            if (fits) { seg = cand; break; }
        }
        if (seg > n) seg = n;
        pl->sep.seg[l] = seg;
        for (int axis = 0; axis < 3; ++axis) {
            const int ip = axis == 0 ? pl->Pp : Q4p, op = axis == 2 ? pl->Pp : Q4p;
            max_smem = std::max(max_smem, sep_smem(axis, seg, l == 0, ip, op));
        }
    }
    pl->sep.smem = max_smem;   // the largest CTA of any pass (each launch asks for its own)
    // flops of the three passes per transform (multiply-adds x 2), for performance accounting
    double fl = 0.0;
    for (int l = 0; l < pl->nlev; ++l) {
        double per = 0.0;
        for (int a = 0; a <= rho; ++a)
            for (int b = 0; a + b <= rho; ++b) {
                const int r = rho - a - b;
                per += 6.0 * tri_count(r);                 // pass X: one FMA per output and offset
                per += 6.0 * (double)(r + 1) * (r + 2) * (r + 3) / 6.0 * (l == 0 ? 1.0 : 1.5);   // pass Y
                per += 6.0 * tri_count(r) * (l == 0 ? 1.0 : 1.5);                                  // pass Z
            }
        fl += 2.0 * per * (double)pl->lev[l].G;
    }
    pl->sep.flops = fl;
    pl->sep.enabled = 1;
    return FC2T2_OK;
}

// The launch's small tables: each level's dt_o(j); the group offsets of the 4-indexed rows; the
// task pairs (i, j) by slot, dealt to the sep_threads(rho) / 32 warps as below.
static void fill_tables(const fc2t2_plan_s *pl, SepArgs &a, int l_begin, int l_end, int axis) {
    const int rho = pl->rho;
    for (int l = l_begin; l < l_end; ++l)
        for (int o = 0; o < 7; ++o)
            for (int j = 0; j <= rho; ++j) a.dt[l - l_begin][o][j] = pl->sep.dt_host[((size_t)l * 7 + o) * (rho + 1) + j];
    for (int i0 = 0; i0 <= rho; ++i0)
        for (int i1 = 0; i1 <= rho; ++i1) {
            int off = 0;
            for (int x = 0; x <= rho; ++x)
                for (int y = 0; x + y <= rho; ++y)
                    if (x < i0 || (x == i0 && y < i1)) off += tri_count(rho - x - y);
            a.goff[i0 * (rho + 1) + i1] = off;
        }
    // A task owns two targets at the finest level and one above it, so with segments of nt cells
    // a warp's lanes cover G = 64 / nt or 32 / nt consecutive task slots, and warp w takes the
    // slot groups w, w + W, w + 2W, ... (W warps).  Pass Y at the finest level, whose task costs
    // spread widest (C(R+3, 3) multiply-adds per row and target: 84 at R = 6, 1 at R = 0), and at
    // orders 7-8 every pass of the finest level (165 at R = 8): the pairs are grouped G at a time
    // by equal budget (lanes of different budgets would run one after the other), and the groups
    // are dealt longest first to the warp with the least work so far -- the CTA's compute phase
    // ends with its busiest warp.  Unfilled slots hold (-1, -1).
    const int W = sep_threads(pl->rho) / 32;
    const int seg = std::min(pl->sep.seg[l_begin], pl->lev[l_begin].n);
    const int G = std::max(1, (l_begin == 0 ? 64 : 32) / seg);
    struct Group { int cost; std::vector<int2> pairs; };
    std::vector<Group> groups;
    for (int R = rho; R >= 0; --R) {
        std::vector<int2> same;
        for (int i = 0; i <= rho - R; ++i) same.push_back(make_int2(i, rho - R - i));
        const int c = (R + 1) * (R + 2) * (R + 3) / 6;
        for (size_t k = 0; k < same.size(); k += G)
            groups.push_back({c, std::vector<int2>(same.begin() + k, same.begin() + std::min(same.size(), k + G))});
    }
    std::stable_sort(groups.begin(), groups.end(), [](const Group &x, const Group &y) { return x.cost > y.cost; });
    if (!(l_begin == 0 && (axis == 1 || pl->rho >= 7))) {
        // elsewhere (passes X and Z at orders <= 6, and the levels above the finest, where a
        // padded table's extra rounds cost more than the balance gains): the pairs in cost order, dealt to the
        // warps in a snake order (0, 1, .., W-1, W-1, .., 0, ...) G slots at a time
        const int T2 = tri_count(rho);
        std::vector<int> used(T2, 0);
        int k = 0;
        for (int d = 0; d <= rho; ++d)
            for (int i = 0; i <= d; ++i) {
                const int m = k / G, round = m / W, pos = m % W;
                const int w = (round & 1) ? W - 1 - pos : pos;
                int slot = round * G * W + G * w + k % G;
                if (slot >= T2) {   // the partial last round: the first free slot
                    slot = 0;
                    while (used[slot]) ++slot;
                }
                used[slot] = 1;
                a.pair[slot] = make_char2((char)i, (char)(d - i));
                ++k;
            }
        a.nslot = T2;
        return;
    }
    std::vector<int> load(W, 0);
    std::vector<std::vector<int>> dealt(W);
    for (int g = 0; g < (int)groups.size(); ++g) {
        int w = 0;
        for (int v = 1; v < W; ++v)
            if (load[v] < load[w] || (load[v] == load[w] && dealt[v].size() < dealt[w].size())) w = v;
        load[w] += groups[g].cost;
        dealt[w].push_back(g);
    }
    size_t rounds = 0;
    for (int w = 0; w < W; ++w) rounds = std::max(rounds, dealt[w].size());
    a.nslot = (int)rounds * W * G;
    if (a.nslot > kSepMaxSlots) {   // (not reached for orders <= 8): the pairs in cost order
        a.nslot = 0;
        for (const Group &g : groups)
            for (const int2 &pr : g.pairs) a.pair[a.nslot++] = make_char2((char)pr.x, (char)pr.y);
        return;
    }
    for (int i = 0; i < a.nslot; ++i) a.pair[i] = make_char2(-1, -1);
    for (size_t r = 0; r < rounds; ++r)
        for (int w = 0; w < W; ++w) {
            if (r >= dealt[w].size()) continue;
            const Group &g = groups[dealt[w][r]];
            for (size_t k = 0; k < g.pairs.size(); ++k)
                a.pair[(r * W + w) * G + k] = make_char2((char)g.pairs[k].x, (char)g.pairs[k].y);
        }
}

template <int RHO, int AXIS, bool FINEST>
static cudaError_t sep_launch(const SepArgs &a0, unsigned blocks, size_t smem, cudaStream_t s) {
    auto *fn = k_m2l_sep<RHO, AXIS, FINEST>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    SepArgs a = a0;
    a.ahead = 0;
    if (FINEST && RHO >= 7) {   // one wave ahead: the blocks resident at once
        int occ = 0, dev = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, sep_threads(RHO), smem);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        a.ahead = occ * sms;
    }
    fn<<<blocks, sep_threads(RHO), smem, s>>>(a);
    return cudaGetLastError();
}

template <int RHO>
static cudaError_t sep_launch_axis(int axis, bool finest, const SepArgs &a, unsigned blocks, size_t smem,
                                   cudaStream_t s) {
    if (finest) {
        if (axis == 0) return sep_launch<RHO, 0, true>(a, blocks, smem, s);
        if (axis == 1) return sep_launch<RHO, 1, true>(a, blocks, smem, s);
        return sep_launch<RHO, 2, true>(a, blocks, smem, s);
    }
    if (axis == 0) return sep_launch<RHO, 0, false>(a, blocks, smem, s);
    if (axis == 1) return sep_launch<RHO, 1, false>(a, blocks, smem, s);
    return sep_launch<RHO, 2, false>(a, blocks, smem, s);
}

// Per pass: one launch for the finest level, one for all levels above it.  `part` selects the
// finest level's three launches (1), the levels above (2) or both (0): the two parts read and
// write disjoint buffers and may run on different streams.
cudaError_t launch_m2l_sep(const fc2t2_plan_s *pl, cudaStream_t s, int part) {
    const int Q4p = pl->sep.q4p;
    for (int axis = 0; axis < 3; ++axis)
        for (int fin = 1; fin >= 0; --fin) {
            if ((part == 1 && !fin) || (part == 2 && fin)) continue;
            const int l_begin = fin ? 0 : 1, l_end = fin ? 1 : pl->nlev;
            if (l_begin >= l_end) continue;
            SepArgs a;
            std::memset(&a, 0, sizeof(a));
            a.nlev = l_end - l_begin;
            fill_tables(pl, a, l_begin, l_end, axis);
            int block = 0;
            size_t smem = 0;
            for (int l = l_begin; l < l_end; ++l) {
                SepLevel &v = a.lv[l - l_begin];
                const int n = pl->lev[l].n;
                float *x0 = pl->sep.d_t + pl->sep.t_off[l][0][0];
                float *x1 = l > 0 ? pl->sep.d_t + pl->sep.t_off[l][0][1] : nullptr;
                float *y0 = pl->sep.d_t + pl->sep.t_off[l][1][0];
                float *y1 = l > 0 ? pl->sep.d_t + pl->sep.t_off[l][1][1] : nullptr;
                if (axis == 0) { v.in0 = pl->d_M + pl->lev[l].off * pl->Pp; v.in1 = nullptr; v.out0 = x0; v.out1 = x1; }
                else if (axis == 1) { v.in0 = x0; v.in1 = x1; v.out0 = y0; v.out1 = y1; }
                else { v.in0 = y0; v.in1 = y1; v.out0 = pl->d_L + pl->lev[l].off * pl->Pp; v.out1 = nullptr; }
                v.n = n;
                v.seg = pl->sep.seg[l];
                v.nseg = (n + v.seg - 1) / v.seg;
                v.block0 = block;
                block += n * n * v.nseg;
                smem = std::max(smem, sep_smem(axis, v.seg, l == 0, axis == 0 ? pl->Pp : Q4p, axis == 2 ? pl->Pp : Q4p));
            }
            pl->launches[FC2T2_STAGE_M2L] += 1;
            cudaError_t err;
            switch (pl->rho) {
                case 1: err = sep_launch_axis<1>(axis, fin, a, block, smem, s); break;
                case 2: err = sep_launch_axis<2>(axis, fin, a, block, smem, s); break;
                case 3: err = sep_launch_axis<3>(axis, fin, a, block, smem, s); break;
                case 4: err = sep_launch_axis<4>(axis, fin, a, block, smem, s); break;
                case 5: err = sep_launch_axis<5>(axis, fin, a, block, smem, s); break;
                case 6: err = sep_launch_axis<6>(axis, fin, a, block, smem, s); break;
                case 7: err = sep_launch_axis<7>(axis, fin, a, block, smem, s); break;
                case 8: err = sep_launch_axis<8>(axis, fin, a, block, smem, s); break;
                default: return cudaErrorInvalidValue;
            }
            if (err != cudaSuccess) return err;
        }
    return cudaSuccess;
}

}  // namespace fc2t2
