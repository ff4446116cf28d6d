// M2M / L2L dispatch (the kernels are the register forms of shift_reg.cu) and the CUDA-core M2L
// (Sec. 3): the direct form, for any kernel (Gaussian, polynomial, least-squares fitted
// operators), 2D and 3D.
//
//     Lt[t](k) = (-1)^|k| sum_{o in window(t)} sum_{|b| <= rho-|k|} Dt[o](k+b) Mt[t+o](b)
//
// The window of target cell t is [-2, 3] per dimension where t is even and [-3, 2] where it is
// odd (Sec. 3: the children of the parent's neighbours), minus the 3^D hole above the finest
// level.  Split targets and sources into parity classes, t = 2a + s and t + o = 2(a + delta) + s'
// per dimension: then o = 2 delta + s' - s, and as s' runs over the 2^D source classes and delta
// over {-1, 0, 1}^D, o runs over the target's window exactly once.  So a CTA that owns a box of
// targets of one class stages, for one source class at a time, the moment rows of the sources
// at subgrid positions box + {-1, 0, 1}^D -- one copy serves all 3^D offsets that reach into it
// (a row-address shift per offset) -- together with the 3^D derivative rows Dt[o] of those
// offsets.  A thread owns one target and a compile-time range of output indices k: it loads an
// offset's derivative row into registers once (a broadcast read) and then, for every input b,
// one moment value that feeds all its outputs k with |k| + |b| <= rho.  Every index is known at
// compile time, so the inner work is a straight run of FMAs.
//
// Staging is by bulk asynchronous copies (one per row, completing on an mbarrier with a bounded
// wait); rows outside the grid are zero-filled.  The rows are stored at a pitch of an odd number
// of 16-byte units, so the 16-byte shared loads of eight neighbouring targets hit distinct banks.
#include <utility>

#include "dir_pairs.cuh"
#include "dispatch.cuh"
#include "fc2t2_internal.cuh"
#include "tc_ptx.cuh"

namespace fc2t2 {

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

namespace {

constexpr int kDirThreads = 256;

// Output ranges per thread: orders <= 6 keep all P outputs of a target in one thread; above, the
// outputs are split between NS threads (registers).
__host__ __device__ constexpr int dir_splits(int D, int rho) { return D == 2 ? 1 : (rho <= 6 ? 1 : rho == 7 ? 2 : 4); }

template <int D, int NS>
struct DirTile {
    static constexpr int T = kDirThreads / NS;                                   // targets per CTA
    static constexpr int X = D == 2 ? 16 : (NS == 4 ? 4 : 8);
    static constexpr int Y = D == 2 ? T / 16 : (NS == 1 ? 8 : 4);
    static constexpr int Z = D == 2 ? 1 : T / (X * Y);
    static constexpr int RX = X + 2, RY = Y + 2, RZ = D == 2 ? 1 : Z + 2;        // staged source rows
    static constexpr int NR = RX * RY * RZ;
    static constexpr int NV = D == 2 ? 9 : 27;                                   // offsets per source class
};

// shared-memory row pitch (floats): Pp, or Pp + 4 when Pp / 4 is even
__host__ __device__ constexpr int dir_pitch(int Pp) { return ((Pp / 4) & 1) ? Pp : Pp + 4; }

template <int D, int RHO>
__host__ __device__ constexpr size_t dir_smem() {
    constexpr int NS = dir_splits(D, RHO), Pp = pad4(ncoef(D, RHO));
    using Tl = DirTile<D, NS>;
    return (size_t)Tl::NR * dir_pitch(Pp) * 4 + (size_t)Tl::NV * Pp * 4 + 16;
}

// one pair: acc[k - K0] += Dt(m) Mt(b); the moment value comes from the 16-byte group of b and
// the derivative value from the offset's row (repeated reads of one address are merged)
template <int K0, int KB, int BB, int MB, int NACC>
__device__ __forceinline__ void dir_fma(const float *__restrict__ row, const float *__restrict__ drow,
                                        float (&acc)[NACC]) {
    const float4 mv4 = *reinterpret_cast<const float4 *>(row + (BB & ~3));
    const float mv = (BB & 3) == 0 ? mv4.x : (BB & 3) == 1 ? mv4.y : (BB & 3) == 2 ? mv4.z : mv4.w;
    const float4 dv4 = *reinterpret_cast<const float4 *>(drow + (MB & ~3));
    const float dv = (MB & 3) == 0 ? dv4.x : (MB & 3) == 1 ? dv4.y : (MB & 3) == 2 ? dv4.z : dv4.w;
    acc[KB - K0] = fmaf(dv, mv, acc[KB - K0]);
}

template <int D, int RHO, int K0, int K1, int NACC, size_t... I>
__device__ __forceinline__ void dir_body_seq(const float *__restrict__ row, const float *__restrict__ drow,
                                             float (&acc)[NACC], std::index_sequence<I...>) {
    constexpr DirPairs<D, RHO, K0, K1> T{};
    (dir_fma<K0, T.k[I], T.b[I], T.m[I], NACC>(row, drow, acc), ...);
}

// Outputs [K0, K1) of one target for one offset: acc[k - K0] += Dt(k + b) Mt(b) over
// |k| + |b| <= RHO.  `row` is the source's staged moment row, `drow` the offset's derivative row.
template <int D, int RHO, int K0, int K1, int NACC>
__device__ __forceinline__ void dir_body(const float *__restrict__ row, const float *__restrict__ drow,
                                         float (&acc)[NACC]) {
    dir_body_seq<D, RHO, K0, K1, NACC>(row, drow, acc, std::make_index_sequence<DirPairs<D, RHO, K0, K1>::N>{});
}

template <int D, int RHO, int NS, int S>
struct DirSplit {
    static constexpr int K0 = dir_k0(D, RHO, NS, S), K1 = dir_k0(D, RHO, NS, S + 1);
    static constexpr int N = K1 - K0 > 0 ? K1 - K0 : 1;
};

// One split's whole work for one target: every source class, every offset of its window.
template <int D, int RHO, int NS, int S>
__device__ __forceinline__ void dir_accumulate(const float *rows, const float *drow, int ix, int iy, int iz, int cls,
                                               int sp, bool finest, float (&acc)[DirSplit<D, RHO, NS, S>::N]) {
    using Tl = DirTile<D, NS>;
    constexpr int Pp = pad4(ncoef(D, RHO)), PITCH = dir_pitch(Pp);
#pragma unroll 1
    for (int j = 0; j < Tl::NV; ++j) {
        const int dx = j % 3 - 1, dy = (j / 3) % 3 - 1, dz = D == 3 ? j / 9 - 1 : 0;
        const int ox = 2 * dx + (sp & 1) - (cls & 1);
        const int oy = 2 * dy + ((sp >> 1) & 1) - ((cls >> 1) & 1);
        const int oz = D == 3 ? 2 * dz + ((sp >> 2) & 1) - ((cls >> 2) & 1) : 0;
        // the hole: interactions of near cells are resolved at the finer level
        if (!finest && ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
        const int r = (ix + dx + 1) + Tl::RX * ((iy + dy + 1) + Tl::RY * (D == 3 ? iz + dz + 1 : 0));
        dir_body<D, RHO, DirSplit<D, RHO, NS, S>::K0, DirSplit<D, RHO, NS, S>::K1, DirSplit<D, RHO, NS, S>::N>(
            rows + r * PITCH, drow + j * Pp, acc);
    }
}

template <int D, int RHO, int NS, int S>
__device__ __forceinline__ void dir_store(float *L, int64_t tlin, const float (&acc)[DirSplit<D, RHO, NS, S>::N]) {
    constexpr int P = ncoef(D, RHO), Pp = pad4(P);
    constexpr int K0 = DirSplit<D, RHO, NS, S>::K0, K1 = DirSplit<D, RHO, NS, S>::K1;
    float *dst = L + tlin * Pp;
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
                dst[ki] = (kd & 1) ? -acc[ki - K0] : acc[ki - K0];
            }
    if (K1 == P)
#pragma unroll
        for (int k = P; k < Pp; ++k) dst[k] = 0.0f;   // row padding stays zero
}

template <int D, int RHO, int NS, int S>
__device__ __forceinline__ void dir_run(const float *rows, const float *drow, uint64_t *bar, const float *M,
                                        float *L, const float *dtab, int n, int finest, int *err, int cls,
                                        int ox0, int oy0, int oz0, int ix, int iy, int iz, bool valid) {
    using Tl = DirTile<D, NS>;
    constexpr int Pp = pad4(ncoef(D, RHO)), PITCH = dir_pitch(Pp);
    const int half = n >> 1;
    float acc[DirSplit<D, RHO, NS, S>::N];
#pragma unroll
    for (int k = 0; k < DirSplit<D, RHO, NS, S>::N; ++k) acc[k] = 0.0f;
    // rows of the staged box that lie in the grid (the same for every source class)
    auto in_count = [&](int o0, int R) { return max(0, min(half, o0 - 1 + R) - max(0, o0 - 1)); };
    const uint32_t nin = (uint32_t)in_count(ox0, Tl::RX) * (uint32_t)in_count(oy0, Tl::RY) *
                         (uint32_t)(D == 3 ? in_count(oz0, Tl::RZ) : 1);
    const uint32_t bytes = (nin + Tl::NV) * (uint32_t)Pp * 4u;
#pragma unroll 1
    for (int sp = 0; sp < (1 << D); ++sp) {
        __syncthreads();                        // the previous class's rows are no longer read
        tc::fence_proxy_async_smem();           // (before the copies overwrite them)
        if (threadIdx.x == 0) tc::mbar_arrive_expect_tx(bar, bytes);
        __syncthreads();
        float *rws = const_cast<float *>(rows);
        for (int r = threadIdx.x; r < Tl::NR; r += kDirThreads) {
            const int rx = r % Tl::RX, ry = (r / Tl::RX) % Tl::RY, rz = r / (Tl::RX * Tl::RY);
            const int ax = ox0 + rx - 1, ay = oy0 + ry - 1, az = D == 3 ? oz0 + rz - 1 : 0;
            if (ax >= 0 && ax < half && ay >= 0 && ay < half && az >= 0 && (D == 2 || az < half)) {
                const int64_t cell = (2 * ax + (sp & 1)) +
                                     (int64_t)n * ((2 * ay + ((sp >> 1) & 1)) + (int64_t)n * (D == 3 ? 2 * az + ((sp >> 2) & 1) : 0));
                tc::bulk_g2s(rws + r * PITCH, M + cell * Pp, Pp * 4u, bar);
            } else {
                float4 *z = reinterpret_cast<float4 *>(rws + r * PITCH);
#pragma unroll
                for (int c = 0; c < Pp / 4; ++c) z[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        for (int j = threadIdx.x; j < Tl::NV; j += kDirThreads) {
            const int dx = j % 3 - 1, dy = (j / 3) % 3 - 1, dz = D == 3 ? j / 9 - 1 : 0;
            const int ox = 2 * dx + (sp & 1) - (cls & 1);
            const int oy = 2 * dy + ((sp >> 1) & 1) - ((cls >> 1) & 1);
            const int oz = D == 3 ? 2 * dz + ((sp >> 2) & 1) - ((cls >> 2) & 1) : 0;
            const int olin = (ox + 3) + 7 * (oy + 3) + (D == 3 ? 49 * (oz + 3) : 0);
            tc::bulk_g2s(const_cast<float *>(drow) + j * Pp, dtab + (int64_t)olin * Pp, Pp * 4u, bar);
        }
        const bool ok = tc::mbar_wait(bar, (uint32_t)(sp & 1), err, 2048);
        if (__syncthreads_or(!ok)) {
            // a copy did not land within the bounded wait: let the copies in flight finish (again
            // bounded) before the CTA's shared memory is released, and leave the outputs alone
            tc::mbar_wait(bar, (uint32_t)(sp & 1), err, 2048);
            return;
        }
        if (valid) dir_accumulate<D, RHO, NS, S>(rows, drow, ix, iy, iz, cls, sp, finest != 0, acc);
    }
    if (valid) {
        const int tx = 2 * (ox0 + ix) + (cls & 1), ty = 2 * (oy0 + iy) + ((cls >> 1) & 1);
        const int tz = D == 3 ? 2 * (oz0 + iz) + ((cls >> 2) & 1) : 0;
        dir_store<D, RHO, NS, S>(L, tx + (int64_t)n * (ty + (int64_t)n * tz), acc);
    }
}

template <int D, int RHO>
__global__ void __launch_bounds__(kDirThreads, 1) k_m2l_dir(const float *__restrict__ M, float *__restrict__ L,
                                                            const float *__restrict__ dtab, int n, int finest,
                                                            int *__restrict__ err) {
    constexpr int NS = dir_splits(D, RHO), Pp = pad4(ncoef(D, RHO));
    using Tl = DirTile<D, NS>;
    extern __shared__ __align__(16) float sm[];
    float *rows = sm;
    float *drow = rows + Tl::NR * dir_pitch(Pp);
    uint64_t *bar = reinterpret_cast<uint64_t *>(drow + Tl::NV * Pp);
    const int half = n >> 1;
    const int tx = (half + Tl::X - 1) / Tl::X, ty = (half + Tl::Y - 1) / Tl::Y;
    const int tz = D == 3 ? (half + Tl::Z - 1) / Tl::Z : 1;
    const int ntile = tx * ty * tz;
    const int cls = (int)blockIdx.x / ntile, tile = (int)blockIdx.x % ntile;
    const int ox0 = (tile % tx) * Tl::X, oy0 = ((tile / tx) % ty) * Tl::Y, oz0 = (tile / (tx * ty)) * Tl::Z;
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const int split = warp % NS;                               // warp-uniform
    const int i = (warp / NS) * 32 + lane;                     // target within the tile
    const int ix = i % Tl::X, iy = (i / Tl::X) % Tl::Y, iz = i / (Tl::X * Tl::Y);
    const bool valid = ox0 + ix < half && oy0 + iy < half && (D == 2 || oz0 + iz < half);
    if (threadIdx.x == 0) tc::mbar_init(bar, 1);
    __syncthreads();
    // every warp runs the same barriers; the split only selects the compile-time output range
    if (NS == 1 || split == 0)
        dir_run<D, RHO, NS, 0>(rows, drow, bar, M, L, dtab, n, finest, err, cls, ox0, oy0, oz0, ix, iy, iz, valid);
    else if (NS >= 2 && split == 1)
        dir_run<D, RHO, NS, (NS >= 2 ? 1 : 0)>(rows, drow, bar, M, L, dtab, n, finest, err, cls, ox0, oy0, oz0, ix, iy, iz, valid);
    else if (NS >= 4 && split == 2)
        dir_run<D, RHO, NS, (NS >= 4 ? 2 : 0)>(rows, drow, bar, M, L, dtab, n, finest, err, cls, ox0, oy0, oz0, ix, iy, iz, valid);
    else if (NS >= 4)
        dir_run<D, RHO, NS, (NS >= 4 ? 3 : 0)>(rows, drow, bar, M, L, dtab, n, finest, err, cls, ox0, oy0, oz0, ix, iy, iz, valid);
}

template <int D, int RHO>
cudaError_t dir_launch(const fc2t2_plan_s *pl, cudaStream_t s, int level) {
    constexpr int NS = dir_splits(D, RHO);
    using Tl = DirTile<D, NS>;
    constexpr size_t smem = dir_smem<D, RHO>();
    static_assert(smem <= 227 * 1024, "the staged rows exceed a CTA's shared memory");
    const Level &lv = pl->lev[level];
    const int half = lv.n >> 1;
    const int ntile = ((half + Tl::X - 1) / Tl::X) * ((half + Tl::Y - 1) / Tl::Y) *
                      (D == 3 ? (half + Tl::Z - 1) / Tl::Z : 1);
    const int nofs = D == 3 ? 343 : 49;
    auto *fn = k_m2l_dir<D, RHO>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    fn<<<(unsigned)(ntile << D), kDirThreads, smem, s>>>(pl->d_M + lv.off * pl->Pp, pl->d_L + lv.off * pl->Pp,
                                                          pl->d_dtab + (int64_t)level * nofs * pl->Pp, lv.n,
                                                          level == 0 ? 1 : 0, pl->d_flags + 2);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_m2l(const fc2t2_plan_s *pl, cudaStream_t s, int level) {
    pl->launches[FC2T2_STAGE_M2L] += 1;
    FC2T2_DISPATCH(pl->D, pl->rho, return (dir_launch<D_, R_>(pl, s, level)), return cudaErrorInvalidValue);
    return cudaErrorInvalidValue;
}

}  // namespace fc2t2
