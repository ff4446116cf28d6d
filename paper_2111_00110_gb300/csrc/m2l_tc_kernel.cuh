// Tensor-core M2L kernel (shared by the per-precision translation units that instantiate it).
// The method and the kernel's structure are described in m2l_tc.cu.
#pragma once
#include <cuda.h>

#include "fc2t2_internal.cuh"
#include "tc_ptx.cuh"

namespace fc2t2 {

using namespace tc;

constexpr int kTcEpiWarps = 8;                       // accumulate / write warps
constexpr int kTcThreads = 64 + 32 * kTcEpiWarps;    // + producer and MMA-issuer warps
constexpr int kAccHalf = 128;            // most accumulator columns one epilogue thread holds
constexpr int kSlabCells = 180;          // 10 x 18 cells
constexpr int kMaxChunks = 24;           // K-steps per operator (b up to 176 TF32 values)
constexpr int kMaxBSlots = 8;
constexpr int kMaxSlabSlots = 3;

struct TcChunk {
    int n0, N, K;     // k columns [n0, n0 + N) over the b range [k0, k0 + K) of one K-step
    int b_off;        // byte offset of the chunk's block inside one operator image
    int k0;
};

struct TcLevel {
    float *L;                     // this level's local coefficients
    const unsigned char *B;       // this level's operator images: [343][ncomp][img_bytes]
    int nl;                       // cells per dimension
    int finest;                   // 1: no hole
    int tiles_x, tiles_y;         // tiles per parity class along x, y (z: n/2)
    int block0;                   // first block of this level in the launch
};

struct TcMaps {
    CUtensorMap m[kMaxLevels][2];   // packed-moment descriptors (high, low part) per level
};

// All levels' M2L run in one launch (they are independent given the moments); blocks are
// ordered finest level first so the small coarse levels fill the tail of the last wave.
struct TcArgs {
    TcLevel lv[kMaxLevels];
    int nlev;
    int *err;
    int Pp;
    int nkc;                      // 16-byte chunks per slab row
    int img_bytes;                // one operator image (one component)
    int ncomp_b;                  // 1, or 2 for the split forms (hi, lo)
    int nchunks;
    int2 ch[kMaxChunks];          // (N, byte offset in the image) of each K-step
    int kh;                       // coefficients per epilogue column half
    int pnb;                      // accumulator columns per TMEM buffer (2 * classes * kh)
    uint32_t tmem_cols;
    int nslab;                    // slab ring slots
    int nbslots;                  // operator ring slots
};

template <int MODE>   // 0: BF16, 1: TF32, 2: TF32 x 3, 3: BF16 x 3
struct TcMode {
    static constexpr bool bf16 = MODE == 0 || MODE == 3;
    static constexpr bool split = MODE == 2 || MODE == 3;   // high + low parts, three products
    static constexpr int esz = bf16 ? 2 : 4;
    static constexpr int epc = 16 / esz;          // elements per 16-byte chunk
    static constexpr int eps = 32 / esz;          // elements per MMA K-step
    static constexpr int ncomp = split ? 2 : 1;
    static constexpr uint32_t fmt = bf16 ? 1u : 2u;
};

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// K-step capacity classes of the MMA issue loop (it is unrolled to the class's count and
// predicates off the steps a plan does not use): BF16 moves 16 values of b per step, TF32 8.
__host__ __device__ constexpr int tc_ksteps(bool bf16, int ksc) {
    return bf16 ? (ksc == 0 ? 4 : ksc == 1 ? 6 : ksc == 2 ? 8 : 11) : (ksc == 0 ? 7 : ksc == 1 ? 11 : ksc == 2 ? 15 : 21);
}
// (classes per CTA, capacity class) pairs that are instantiated: four classes only occur for
// P <= 56 (class 0), two for P <= 120 (classes 0-2), one for larger P or tight shared memory
// (classes 1-3)
__host__ __device__ constexpr bool tc_variant(int ncls, int ksc) {
    return ncls == 4 ? ksc == 0 : ncls == 2 ? (ksc >= 0 && ksc <= 2) : ncls == 1 ? (ksc >= 1 && ksc <= 3) : false;
}

// ------------------------------------------------------------------------------ M2L
template <int MODE, int NCLS, int KSTEPS>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_m2l_tc(const __grid_constant__ TcMaps maps, const TcArgs args) {
    using Md = TcMode<MODE>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar_bfull[kMaxBSlots], bar_bfree[kMaxBSlots], bar_sfull[kMaxSlabSlots], bar_sfree[kMaxSlabSlots];
    __shared__ uint64_t bar_accfull[2], bar_accfree[2], bar_done;
    __shared__ uint32_t tmem_base;
    __shared__ int2 s_chunk[kMaxChunks];         // (N, b_off) of each K-step

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int lvl = 0;
#pragma unroll
    for (int i = 1; i < kMaxLevels; ++i)
        if (i < args.nlev && (int)blockIdx.x >= args.lv[i].block0) lvl = i;
    const TcLevel lv = args.lv[lvl];
    const CUtensorMap *map_hi = &maps.m[lvl][0];
    const CUtensorMap *map_lo = &maps.m[lvl][1];
    const int half = lv.nl >> 1;
    const int tiles_per_group = lv.tiles_x * lv.tiles_y * half;
    const int bl = (int)blockIdx.x - lv.block0;
    int gb = bl / tiles_per_group;           // class group
    int tr = bl % tiles_per_group;
    const int tx = tr % lv.tiles_x;
    tr /= lv.tiles_x;
    const int ty = tr % lv.tiles_y;
    const int az = tr / lv.tiles_y;
    const int ax0 = tx * 8, ay0 = ty * 16;
    // parity of the group's class 0; class c of the group adds (c & 1, c >> 1, 0)
    const int pix0 = NCLS >= 2 ? 0 : (gb & 1);
    if (NCLS < 2) gb >>= 1;
    const int piy0 = NCLS >= 4 ? 0 : (gb & 1);
    if (NCLS < 4) gb >>= 1;
    const int piz = gb & 1;

    const int box_bytes = kSlabCells * 16 * args.nkc;           // bytes one TMA slab load delivers
    const int slab_bytes = (box_bytes + 1023) & ~1023;          // one component, 1024-aligned
    const int slab_stride = slab_bytes * Md::ncomp;              // one ring slot
    unsigned char *slabs = smem;
    unsigned char *bring = smem + ((args.nslab * slab_stride + 1023) & ~1023);
    const int bslot_bytes = args.img_bytes * args.ncomp_b;

    if (threadIdx.x < kMaxChunks) s_chunk[threadIdx.x] = args.ch[threadIdx.x];
    if (threadIdx.x == 0) {
        for (int i = 0; i < args.nbslots; ++i) { mbar_init(&bar_bfull[i], 1); mbar_init(&bar_bfree[i], 1); }
        for (int i = 0; i < args.nslab; ++i) { mbar_init(&bar_sfull[i], 1); mbar_init(&bar_sfree[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&bar_accfull[i], 1); mbar_init(&bar_accfree[i], 32 * kTcEpiWarps); }
        mbar_init(&bar_done, 1);
    }
    fence_proxy_async_smem();
    if (warp == 0) tmem_alloc(&tmem_base, args.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tacc = tmem_base;

    bool ok = true;
    // The view of step s = (sigma, dz) shifted by (dx, dy) meets class 0 at offset o; class c at
    // o - (c & 1, c >> 1, 0).  Above the finest level a view whose offsets all fall in the hole
    // is skipped (the operator image zeroes the classes for which only some do).
    auto op_of = [&](int s, int dx, int dy, int &olin) -> bool {
        const int sg = s / 3, dz = s % 3 - 1;
        const int ox = 2 * dx + (sg & 1) - pix0, oy = 2 * dy + ((sg >> 1) & 1) - piy0, oz = 2 * dz + (sg >> 2) - piz;
        if (!lv.finest && oz >= -1 && oz <= 1) {
            bool any = false;
#pragma unroll
            for (int c = 0; c < NCLS; ++c) {
                const int oxc = ox - (NCLS >= 2 ? (c & 1) : 0), oyc = oy - (NCLS >= 4 ? (c >> 1) : 0);
                if (oxc < -1 || oxc > 1 || oyc < -1 || oyc > 1) any = true;
            }
            if (!any) return false;
        }
        olin = (ox + 3) + 7 * (oy + 3) + 49 * (oz + 3);
        return true;
    };
    if (warp == 0) {
        // ---------------------------------------------------------------- producer (whole warp,
        // one elected lane issues the copies)
        int j = 0;
        for (int s = 0; s < 24 && ok; ++s) {
            const int slot = s % args.nslab, use = s / args.nslab;
            if (use >= 1 && !mbar_wait_warp(&bar_sfree[slot], (use - 1) & 1, args.err, 16)) { ok = false; break; }
            const int sg = s / 3, dz = s % 3 - 1;
            unsigned char *dst = slabs + slot * slab_stride;
            const int zc = sg * (half + 2) + (az + dz + 1);   // z plane index includes the zero plane below z = 0
            if (elect_one()) {
                mbar_arrive_expect_tx(&bar_sfull[slot], (uint32_t)(box_bytes * Md::ncomp));
                // innermost coordinate in bytes: (ax0 - 1) * 16, a multiple of 16 (may be -16: zero fill)
                tma_load_4d(dst, map_hi, (ax0 - 1) * 16, ay0 - 1, 0, zc, &bar_sfull[slot]);
                if (Md::split) tma_load_4d(dst + slab_bytes, map_lo, (ax0 - 1) * 16, ay0 - 1, 0, zc, &bar_sfull[slot]);
            }
            __syncwarp();
            for (int t9 = 0; t9 < 9 && ok; ++t9) {
                int olin;
                if (!op_of(s, t9 % 3 - 1, t9 / 3 - 1, olin)) continue;
                const int bslot = j % args.nbslots, buse = j / args.nbslots;
                if (buse >= 1 && !mbar_wait_warp(&bar_bfree[bslot], (buse - 1) & 1, args.err, 16)) { ok = false; break; }
                if (elect_one()) {
                    mbar_arrive_expect_tx(&bar_bfull[bslot], (uint32_t)bslot_bytes);
                    bulk_g2s(bring + bslot * bslot_bytes, lv.B + (size_t)olin * bslot_bytes, (uint32_t)bslot_bytes,
                             &bar_bfull[bslot]);
                }
                __syncwarp();
                ++j;
            }
        }
        // bounded drain of the last copies of every ring slot
        for (int jj = (j - args.nbslots > 0 ? j - args.nbslots : 0); jj < j; ++jj)
            mbar_wait_warp(&bar_bfull[jj % args.nbslots], (jj / args.nbslots) & 1, args.err, 128);
        for (int s = 24 - args.nslab; s < 24; ++s)
            mbar_wait_warp(&bar_sfull[s % args.nslab], (s / args.nslab) & 1, args.err, 128);
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer (whole warp,
        // one elected lane issues; every per-K-step quantity is precomputed)
        constexpr int kSteps = KSTEPS;
        const uint32_t lboA = kSlabCells * 16, sboA = 160;
        uint32_t c_idesc[kSteps];
        uint64_t c_bdesc[kSteps];          // B descriptor relative to the slot base
#pragma unroll
        for (int c = 0; c < kSteps; ++c) {
            const int2 cn = s_chunk[c];
            const int n = c < args.nchunks ? cn.x : 16;
            c_idesc[c] = instr_desc(Md::fmt, (uint32_t)n);
            c_bdesc[c] = smem_desc((uint32_t)cn.y, (uint32_t)(n / 8) * 128u, 128u);
        }
        const uint64_t a_lo = (uint64_t)((uint32_t)slab_bytes >> 4);      // A low part (split forms)
        const uint64_t b_lo = (uint64_t)((uint32_t)args.img_bytes >> 4);  // B low part
        const int nch = args.nchunks;
        int j = 0;
        for (int s = 0; s < 24 && ok; ++s) {
            const int slot = s % args.nslab, use = s / args.nslab;
            const int ab = s & 1;
            if (s >= 2 && !mbar_wait_warp(&bar_accfree[ab], ((s - 2) >> 1) & 1, args.err, 4)) { ok = false; break; }
            if (!mbar_wait_warp(&bar_sfull[slot], use & 1, args.err, 4)) { ok = false; break; }
            tc_fence_after();
            const uint32_t slab_a = smem_u32(slabs + slot * slab_stride);
            const uint32_t acc_col = tacc + (uint32_t)(ab * args.pnb);
            uint32_t accum0 = 0;              // the step's first MMA initialises the buffer
            for (int t9 = 0; t9 < 9; ++t9) {
                int olin;
                const int dx = t9 % 3 - 1, dy = t9 / 3 - 1;
                if (!op_of(s, dx, dy, olin)) continue;
                const int bslot = j % args.nbslots;
                if (!mbar_wait_warp(&bar_bfull[bslot], (j / args.nbslots) & 1, args.err, 8)) { ok = false; break; }
                tc_fence_after();
                const uint64_t bbase = (uint64_t)(smem_u32(bring + bslot * bslot_bytes) >> 4);
                const uint64_t abase = smem_desc(slab_a + (uint32_t)(((dy + 1) * 10 + (dx + 1)) * 16), lboA, sboA);
#pragma unroll
                for (int c = 0; c < kSteps; ++c) {
                    const uint32_t on = c < nch ? 1u : 0u;
                    const uint64_t ad = abase + (uint64_t)(((uint32_t)c * 2u * lboA) >> 4);
                    const uint64_t bd = c_bdesc[c] + bbase;
                    if (Md::bf16) {
                        mma_bf16_elect(on, acc_col, ad, bd, c_idesc[c], accum0 | (uint32_t)c);
                        if (Md::split) {
                            mma_bf16_elect(on, acc_col, ad, bd + b_lo, c_idesc[c], 1u);
                            mma_bf16_elect(on, acc_col, ad + a_lo, bd, c_idesc[c], 1u);
                        }
                    } else {
                        mma_tf32_elect(on, acc_col, ad, bd, c_idesc[c], accum0 | (uint32_t)c);
                        if (Md::split) {
                            mma_tf32_elect(on, acc_col, ad, bd + b_lo, c_idesc[c], 1u);
                            mma_tf32_elect(on, acc_col, ad + a_lo, bd, c_idesc[c], 1u);
                        }
                    }
                }
                accum0 = 1u;
                mma_commit_elect(&bar_bfree[bslot]);
                ++j;
            }
            if (!ok) break;
            mma_commit_elect(&bar_sfree[slot]);
            mma_commit_elect(&bar_accfull[ab]);
        }
        mma_commit_elect(&bar_done);
    } else {
        // ---------------------------------------------------------------- accumulate / write
        // Warps 2..9: warp w reads TMEM lane quarter w % 4 and column half (w - 2) / 4; column
        // n of a buffer holds coefficient n / NCLS of class n % NCLS.
        const int q = warp & 3;
        const int hh = (warp - 2) >> 2;
        const int colh = args.pnb >> 1;                // = NCLS * kh
        float acc[kAccHalf];
#pragma unroll
        for (int i = 0; i < kAccHalf; ++i) acc[i] = 0.0f;
        for (int u = 0; u < 24 && ok; ++u) {
            const int ab = u & 1;
            if (!mbar_wait_warp(&bar_accfull[ab], (u >> 1) & 1, args.err, 32)) { ok = false; break; }
            tc_fence_after();
            const uint32_t col = tacc + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * args.pnb + hh * colh);
#pragma unroll
            for (int c0 = 0; c0 < kAccHalf; c0 += 16) {
                if (c0 < colh) {
                    float v[16];
                    tmem_ld16(col + (uint32_t)c0, v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) acc[c0 + e] += v[e];
                }
            }
            tc_fence_before();
            mbar_arrive(&bar_accfree[ab]);
        }
        if (ok) {
            const int r = q * 32 + lane;            // tile row
            const int x = ax0 + (r & 7), y = ay0 + (r >> 3);
            if (x < half && y < half) {
#pragma unroll
                for (int c = 0; c < NCLS; ++c) {
                    const int cx = NCLS >= 2 ? (c & 1) : 0, cy = NCLS >= 4 ? (c >> 1) : 0;
                    const int64_t t = (int64_t)(2 * x + pix0 + cx) +
                                      (int64_t)lv.nl * ((2 * y + piy0 + cy) + (int64_t)lv.nl * (2 * az + piz));
                    float *Lrow = lv.L + t * args.Pp + hh * args.kh;
#pragma unroll
                    for (int jc = 0; jc < kAccHalf; jc += 4 * NCLS) {
                        const int k = hh * args.kh + jc / NCLS;
                        if (jc < colh && k + 4 <= args.Pp)
                            *reinterpret_cast<float4 *>(Lrow + jc / NCLS) =
                                make_float4(acc[jc + c], acc[jc + NCLS + c], acc[jc + 2 * NCLS + c],
                                            acc[jc + 3 * NCLS + c]);
                    }
                }
            }
        }
    }
    // every MMA issued must have completed before the accumulator is released
    mbar_wait(&bar_done, 0, args.err, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tacc, args.tmem_cols);
}

// Launches k_m2l_tc<MODE, ncls, tc_ksteps(MODE, ksc)>; defined per MODE in its own translation unit.
template <int MODE>
cudaError_t launch_m2l_tc_mode(int ncls, int ksc, unsigned blocks, int smem, cudaStream_t s, const TcMaps &maps,
                               const TcArgs &a);

#define FC2T2_TC_INSTANTIATE(MODE_)                                                                          \
    template <>                                                                                               \
    cudaError_t launch_m2l_tc_mode<MODE_>(int ncls, int ksc, unsigned blocks, int smem, cudaStream_t s,       \
                                          const TcMaps &maps, const TcArgs &a) {                              \
        constexpr bool bf = TcMode<MODE_>::bf16;                                                              \
        switch (ncls * 8 + ksc) {                                                                             \
            FC2T2_TC_CASE(MODE_, 4, 0) FC2T2_TC_CASE(MODE_, 2, 0) FC2T2_TC_CASE(MODE_, 2, 1)                  \
            FC2T2_TC_CASE(MODE_, 2, 2) FC2T2_TC_CASE(MODE_, 1, 1) FC2T2_TC_CASE(MODE_, 1, 2)                  \
            FC2T2_TC_CASE(MODE_, 1, 3)                                                                        \
            default: return cudaErrorInvalidValue;                                                            \
        }                                                                                                     \
        return cudaGetLastError();                                                                            \
    }
#define FC2T2_TC_CASE(MODE_, NCLS_, KSC_)                                                                     \
    case (NCLS_) * 8 + (KSC_): {                                                                              \
        auto *fn = k_m2l_tc<MODE_, NCLS_, tc_ksteps(bf, KSC_)>;                                               \
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);                          \
        fn<<<blocks, kTcThreads, smem, s>>>(maps, a);                                                         \
        break;                                                                                                \
    }

}  // namespace fc2t2
