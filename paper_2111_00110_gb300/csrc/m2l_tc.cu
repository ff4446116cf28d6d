// M2L on the tcgen05 tensor cores (Sec. 3: M2L as a convolution with a parity-dependent
// 6^D window and a 3^D hole; here as batched small dense contractions).
//
// For a target parity class pi and an offset o = 2 delta + sigma - pi (delta in {-1,0,1}^3,
// sigma the source parity) the M2L of every target of class pi is one GEMM
//     Lt[a, k] += sum_b  Mt_sigma[a + delta, b] * B_o[k, b],   B_o[k, b] = (-1)^|k| Dt_o[k+b]
// (|k| + |b| <= rho), with a the target's index in the half-resolution sub-grid.  A CTA owns
// 128 targets (8 x 16 sub-grid cells in x, y at one z) of one class: its accumulator is a
// 128 x Pn FP32 tile in tensor memory.
//
// Operands.  A pack kernel rewrites each level's moments once into the tensor-core layout:
// per source parity sigma and sub-grid z, 16-byte chunks of 8 BF16 (or 4 TF32) coefficients
// ordered [chunk][y][x] -- exactly the canonical no-swizzle K-major layout, so one TMA tensor
// load brings the 10 x 18 cell "slab" of sub-grid sigma around the tile into shared memory
// (cells outside the grid arrive as zeros).  The nine (delta_x, delta_y) A operands of a slab
// are views that differ only in their start address.  The operators B_o are precomputed per
// level as shared-memory images and fetched with bulk copies.  Because |k| + |b| <= rho, each
// MMA K-step (16 BF16 or 8 TF32 values of b) only reaches the k of degree <= rho - min|b| of
// the step, so its N shrinks with the degree of b (degree-block skipping): rho = 6, BF16 uses
// N = 96, 32, 16, 16, 16, 16 for its six K-steps -- 3072 of 9216 dense multiply-adds.  (An
// MMA instruction costs at least ~40 cycles whatever its size and runs at full rate only from
// N ~ 96, so one instruction per K-step is cheaper than splitting k into narrow chunks.)
//
// Precision: BF16 or TF32 operands with FP32 accumulation, or a split form (A_hi B_hi + A_hi B_lo
// + A_lo B_hi, the low parts being the rounding residues) in TF32 x 3 or BF16 x 3; both split
// forms are within the FP32 bar (1e-5 relative L2), BF16 x 3 with half the MMAs of TF32 x 3.  The tensor
// core's accumulation over thousands of MMAs loses low bits, so each step's partial sum is
// accumulated in its own TMEM buffer (two, alternating) and added into FP32 registers.
//
// Warp roles: warp 0 lane 0 fetches slabs (TMA) and operators (bulk copies), warp 1 lane 0
// issues the MMAs, warps 2-5 add each step's partial accumulator into FP32 registers (each
// warp reads its TMEM lane quarter) and finally write the Lt rows.  Every wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <vector>

#include "fc2t2_internal.cuh"
#include "tc_ptx.cuh"

namespace fc2t2 {

using namespace tc;

constexpr int kTcThreads = 192;
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
    int ncomp_b;                  // 1, or 2 for TF32 x 3 (hi, lo)
    int nchunks;
    TcChunk ch[kMaxChunks];
    int pn;                       // accumulator columns used
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

// ------------------------------------------------------------------------------ pack
// Mtc[comp][sigma][z + 1][kc][y][x] (16 bytes each) from Mt[cell][Pp]; z planes -1 and half
// stay zero.  comp 1 (TF32 x 3) holds the TF32 rounding residue of comp 0.
template <int MODE>
__global__ void __launch_bounds__(256) k_pack_tc(const float *__restrict__ M, unsigned char *__restrict__ out,
                                                 int nl, int Pp, int nkc) {
    using Md = TcMode<MODE>;
    const int half = nl >> 1;
    const int64_t plane = (int64_t)nkc * half * half;          // chunks per (sigma, z)
    const int64_t total = (int64_t)8 * half * plane;
    const int64_t comp_stride = (int64_t)8 * (half + 2) * plane * 16;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i;
        const int x = (int)(r % half); r /= half;
        const int y = (int)(r % half); r /= half;
        const int kc = (int)(r % nkc); r /= nkc;
        const int z = (int)(r % half);
        const int sg = (int)(r / half);
        const int64_t cell = (int64_t)(2 * x + (sg & 1)) +
                             (int64_t)nl * ((2 * y + ((sg >> 1) & 1)) + (int64_t)nl * (2 * z + (sg >> 2)));
        const float *row = M + cell * Pp;
        const int k0 = kc * Md::epc;
        float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int q4 = 0; q4 < Md::epc / 4; ++q4)
            if (k0 + 4 * q4 + 4 <= Pp) {
                const float4 f = __ldg(reinterpret_cast<const float4 *>(row + k0 + 4 * q4));
                v[4 * q4] = f.x; v[4 * q4 + 1] = f.y; v[4 * q4 + 2] = f.z; v[4 * q4 + 3] = f.w;
            }
        const int64_t o = ((((int64_t)sg * (half + 2) + (z + 1)) * nkc + kc) * half + y) * half + x;
        uint4 *dst = reinterpret_cast<uint4 *>(out + o * 16);
        if (Md::bf16) {
            float h[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) h[e] = round_bf16(v[e]);
            *dst = make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]), pack_bf16x2(h[4], h[5]),
                              pack_bf16x2(h[6], h[7]));
            if (MODE == 3)
                *reinterpret_cast<uint4 *>(out + comp_stride + o * 16) =
                    make_uint4(pack_bf16x2(v[0] - h[0], v[1] - h[1]), pack_bf16x2(v[2] - h[2], v[3] - h[3]),
                               pack_bf16x2(v[4] - h[4], v[5] - h[5]), pack_bf16x2(v[6] - h[6], v[7] - h[7]));
        } else {
            float h[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) h[e] = round_tf32(v[e]);
            *dst = make_uint4(__float_as_uint(h[0]), __float_as_uint(h[1]), __float_as_uint(h[2]), __float_as_uint(h[3]));
            if (MODE == 2)
                *reinterpret_cast<uint4 *>(out + comp_stride + o * 16) =
                    make_uint4(__float_as_uint(round_tf32(v[0] - h[0])), __float_as_uint(round_tf32(v[1] - h[1])),
                               __float_as_uint(round_tf32(v[2] - h[2])), __float_as_uint(round_tf32(v[3] - h[3])));
        }
    }
}

// ------------------------------------------------------------------------------ M2L
// most K-steps any order up to the one that needs PNMAX columns can have (BF16: 16 b per step,
// TF32: 8); the issue loop is unrolled to it and predicates off the steps a plan does not use
template <int MODE, int PNMAX>
constexpr int max_ksteps() {
    constexpr bool tf = !TcMode<MODE>::bf16;
    return PNMAX == 32 ? (tf ? 3 : 2)
         : PNMAX == 64 ? (tf ? 7 : 4)
         : PNMAX == 96 ? (tf ? 11 : 6)
         : PNMAX == 128 ? (tf ? 15 : 8)
                        : (tf ? 21 : 11);
}

template <int MODE, int PNMAX>
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
    const int tiles_per_class = lv.tiles_x * lv.tiles_y * half;
    const int bl = (int)blockIdx.x - lv.block0;
    const int pi = bl / tiles_per_class;
    int tr = bl % tiles_per_class;
    const int tx = tr % lv.tiles_x;
    tr /= lv.tiles_x;
    const int ty = tr % lv.tiles_y;
    const int az = tr / lv.tiles_y;
    const int ax0 = tx * 8, ay0 = ty * 16;
    const int pix = pi & 1, piy = (pi >> 1) & 1, piz = (pi >> 2) & 1;

    const int box_bytes = kSlabCells * 16 * args.nkc;           // bytes one TMA slab load delivers
    const int slab_bytes = (box_bytes + 1023) & ~1023;          // one component, 1024-aligned
    const int slab_stride = slab_bytes * Md::ncomp;              // one ring slot
    unsigned char *slabs = smem;
    unsigned char *bring = smem + ((args.nslab * slab_stride + 1023) & ~1023);
    const int bslot_bytes = args.img_bytes * args.ncomp_b;

    if (threadIdx.x < kMaxChunks) s_chunk[threadIdx.x] = make_int2(args.ch[threadIdx.x].N, args.ch[threadIdx.x].b_off);
    if (threadIdx.x == 0) {
        for (int i = 0; i < args.nbslots; ++i) { mbar_init(&bar_bfull[i], 1); mbar_init(&bar_bfree[i], 1); }
        for (int i = 0; i < args.nslab; ++i) { mbar_init(&bar_sfull[i], 1); mbar_init(&bar_sfree[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&bar_accfull[i], 1); mbar_init(&bar_accfree[i], 128); }
        mbar_init(&bar_done, 1);
    }
    fence_proxy_async_smem();
    if (warp == 0) tmem_alloc(&tmem_base, args.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tacc = tmem_base;

    bool ok = true;
    // operators of step s = (sigma, dz), then (dx, dy); the hole is skipped above the finest level
    auto op_of = [&](int s, int dx, int dy, int &olin) -> bool {
        const int sg = s / 3, dz = s % 3 - 1;
        const int ox = 2 * dx + (sg & 1) - pix, oy = 2 * dy + ((sg >> 1) & 1) - piy, oz = 2 * dz + (sg >> 2) - piz;
        if (!lv.finest && ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) return false;
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
        constexpr int kSteps = max_ksteps<MODE, PNMAX>();
        const uint32_t lboA = kSlabCells * 16, sboA = 160;
        uint32_t c_idesc[kSteps];
        uint64_t c_bdesc[kSteps];          // B descriptor relative to the slot base
        uint64_t c_adesc[kSteps];          // A descriptor relative to the view base
#pragma unroll
        for (int c = 0; c < kSteps; ++c) {
            const int2 cn = s_chunk[c];
            const int n = c < args.nchunks ? cn.x : 16;
            c_idesc[c] = instr_desc(Md::fmt, (uint32_t)n);
            c_bdesc[c] = smem_desc((uint32_t)cn.y, (uint32_t)(n / 8) * 128u, 128u);
            c_adesc[c] = (uint64_t)(((uint32_t)c * 2u * lboA) >> 4);
        }
        const uint64_t a_lo = (uint64_t)((uint32_t)slab_bytes >> 4);      // A low part (TF32 x 3)
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
            const uint32_t acc_col = tacc + (uint32_t)(ab * args.pn);
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
                    const uint64_t ad = abase + c_adesc[c];
                    const uint64_t bd = c_bdesc[c] + bbase;
                    if (Md::bf16) {
                        mma_bf16_elect(on, acc_col, ad, bd, c_idesc[c], accum0 | (uint32_t)c);
                        if (MODE == 3) {
                            mma_bf16_elect(on, acc_col, ad, bd + b_lo, c_idesc[c], 1u);
                            mma_bf16_elect(on, acc_col, ad + a_lo, bd, c_idesc[c], 1u);
                        }
                    } else {
                        mma_tf32_elect(on, acc_col, ad, bd, c_idesc[c], accum0 | (uint32_t)c);
                        if (MODE == 2) {
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
        const int q = warp & 3;                 // TMEM lane quarter of this warp
        float acc[PNMAX];
#pragma unroll
        for (int i = 0; i < PNMAX; ++i) acc[i] = 0.0f;
        for (int u = 0; u < 24 && ok; ++u) {
            const int ab = u & 1;
            if (!mbar_wait_warp(&bar_accfull[ab], (u >> 1) & 1, args.err, 32)) { ok = false; break; }
            tc_fence_after();
#pragma unroll
            for (int c0 = 0; c0 < PNMAX; c0 += 16) {
                if (c0 < args.pn) {
                    float v[16];
                    tmem_ld16(tacc + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * args.pn + c0), v);
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
                const int64_t t = (int64_t)(2 * x + pix) +
                                  (int64_t)lv.nl * ((2 * y + piy) + (int64_t)lv.nl * (2 * az + piz));
                float *Lrow = lv.L + t * args.Pp;
#pragma unroll
                for (int e = 0; e < PNMAX; e += 4)
                    if (e + 4 <= args.Pp)
                        *reinterpret_cast<float4 *>(Lrow + e) = make_float4(acc[e], acc[e + 1], acc[e + 2], acc[e + 3]);
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

// ------------------------------------------------------------------------------ host side

namespace {

int degree_of(int D, int k) {
    int d = 0;
    while (ncoef(D, d) <= k) ++d;
    return d;
}

// One chunk per MMA K-step of kg values of b: the step starting at b0 only reaches the k of
// degree <= rho - deg(b0), i.e. the first ncoef(rho - deg(b0)) columns (rounded up to 16).
void plan_chunks(int D, int rho, int P, int kg, std::vector<TcChunk> &out, int &pn, int &kfull) {
    pn = (P + 15) / 16 * 16;
    kfull = (P + kg - 1) / kg * kg;
    out.clear();
    for (int k0 = 0; k0 < kfull; k0 += kg) {
        const int d = degree_of(D, k0);
        const int need = ncoef(D, rho - d);
        TcChunk ch;
        ch.k0 = k0;
        ch.K = kg;
        ch.n0 = 0;
        ch.N = (need + 15) / 16 * 16;
        if (ch.N > pn) ch.N = pn;
        ch.b_off = 0;
        out.push_back(ch);
    }
}

uint16_t to_bf16(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float to_tf32(float x) {   // round half away from zero on the 13 dropped bits (as cvt.rna)
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x1000u;
    u &= 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

}  // namespace

// Build the tensor-core operator images of every level from the FP64 derivative table,
// the packed-moment buffers and their TMA descriptors.
fc2t2_status build_tc_operators(fc2t2_plan_s *pl, const std::vector<double> &dtab64) {
    pl->tc.enabled = 0;
    if (pl->D != 3) return FC2T2_OK;
    const int mode = pl->desc.m2l == FC2T2_M2L_BF16 ? 0 : pl->desc.m2l == FC2T2_M2L_TF32 ? 1
                   : pl->desc.m2l == FC2T2_M2L_TF32X3 ? 2 : 3;
    const bool bf16 = mode == 0 || mode == 3, split = mode == 2 || mode == 3;
    const int esz = bf16 ? 2 : 4, epc = 16 / esz, kg = 32 / esz;
    std::vector<TcChunk> ch;
    int pn = 0, kfull = 0;
    plan_chunks(pl->D, pl->rho, pl->P, kg, ch, pn, kfull);
    if (pn > 176 || (int)ch.size() > kMaxChunks) return FC2T2_OK;
    {
        const int cls = pn <= 32 ? 32 : pn <= 64 ? 64 : pn <= 96 ? 96 : pn <= 128 ? 128 : 176;
        const bool tf = !bf16;
        const int cap = cls == 32 ? (tf ? 3 : 2) : cls == 64 ? (tf ? 7 : 4) : cls == 96 ? (tf ? 11 : 6)
                      : cls == 128 ? (tf ? 15 : 8) : (tf ? 21 : 11);
        if ((int)ch.size() > cap) return FC2T2_OK;   // cannot happen for orders <= 8; keep the CUDA-core M2L
    }
    int off = 0;
    for (auto &c : ch) { c.b_off = off; off += c.N * c.K * esz; }
    const int img = off;
    const int ncomp = split ? 2 : 1;
    const int nofs = 343;
    const int nkc = kfull * esz / 16;
    // shared memory: slab ring + operator ring (two CTAs per SM when both fit in half of it)
    const int slab = ((kSlabCells * 16 * nkc + 1023) & ~1023) * ncomp;   // as in the kernel
    const int bslot = img * ncomp;
    // prefer two CTAs per SM, then a deep operator ring (bulk-copy latency), then more slab slots
    int nslab = 0, nbs = 0, smem = 0;
    for (int budget : {112 * 1024, 220 * 1024}) {
        for (int nb = kMaxBSlots; nb >= 4 && !nslab; --nb)
            for (int ns = kMaxSlabSlots; ns >= 1; --ns) {
                if (ns < 2 && budget <= 112 * 1024) continue;
                const int bytes = ((ns * slab + 1023) & ~1023) + nb * bslot;
                if (bytes <= budget) { nslab = ns; nbs = nb; smem = bytes; break; }
            }
        if (nslab) break;
    }
    if (!nslab) return FC2T2_OK;   // too large for shared memory: the CUDA-core M2L runs instead
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return FC2T2_OK;

    std::vector<int> deg(pl->P);
    for (int k = 0; k < pl->P; ++k) deg[k] = degree_of(pl->D, k);
    std::vector<int> ex(3 * pl->P);
    for (int a0 = 0; a0 <= pl->rho; ++a0)
        for (int a1 = 0; a0 + a1 <= pl->rho; ++a1)
            for (int a2 = 0; a0 + a1 + a2 <= pl->rho; ++a2) {
                const int g = gidx3(a0, a1, a2);
                ex[3 * g] = a0; ex[3 * g + 1] = a1; ex[3 * g + 2] = a2;
            }
    std::vector<unsigned char> host((size_t)pl->nlev * nofs * ncomp * img, 0);
    for (int l = 0; l < pl->nlev; ++l)
        for (int o = 0; o < nofs; ++o) {
            const double *Dt = dtab64.data() + ((size_t)l * nofs + o) * pl->P;
            unsigned char *base = host.data() + ((size_t)l * nofs + o) * ncomp * img;
            for (const TcChunk &c : ch)
                for (int n = 0; n < c.N; ++n)
                    for (int k = 0; k < c.K; ++k) {
                        const int kap = c.n0 + n, b = c.k0 + k;
                        double v = 0.0;
                        if (kap < pl->P && b < pl->P && deg[kap] + deg[b] <= pl->rho) {
                            const int m = gidx3(ex[3 * kap] + ex[3 * b], ex[3 * kap + 1] + ex[3 * b + 1],
                                                ex[3 * kap + 2] + ex[3 * b + 2]);
                            v = (deg[kap] & 1) ? -Dt[m] : Dt[m];
                        }
                        const size_t pos = (size_t)c.b_off + ((size_t)(k / epc) * (c.N / 8) + n / 8) * 128 +
                                           (n % 8) * 16 + (k % epc) * esz;
                        if (bf16) {
                            const uint16_t h = to_bf16((float)v);
                            std::memcpy(base + pos, &h, 2);
                            if (mode == 3) {
                                float hf;
                                const uint32_t u = (uint32_t)h << 16;
                                std::memcpy(&hf, &u, 4);
                                const uint16_t lo = to_bf16((float)(v - (double)hf));
                                std::memcpy(base + img + pos, &lo, 2);
                            }
                        } else {
                            const float hi = to_tf32((float)v);
                            std::memcpy(base + pos, &hi, 4);
                            if (mode == 2) {
                                const float lo = to_tf32((float)(v - (double)hi));
                                std::memcpy(base + img + pos, &lo, 4);
                            }
                        }
                    }
        }
    cudaError_t e = cudaMalloc(&pl->d_mma_ops, host.size());
    if (e != cudaSuccess) {
        cudaGetLastError();
        pl->d_mma_ops = nullptr;
        return set_error(FC2T2_ERR_OOM, "cudaMalloc failed for tensor-core operators");
    }
    pl->mma_ops_bytes = host.size();
    if ((e = cudaMemcpy(pl->d_mma_ops, host.data(), host.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return check_cuda(e, "upload tensor-core operators");

    // packed moments per level: [comp][sigma][half + 2][nkc][half][half] x 16 bytes, zeroed once
    for (int l = 0; l < pl->nlev; ++l) {
        const int half = pl->lev[l].n >> 1;
        const size_t comp_bytes = (size_t)8 * (half + 2) * nkc * half * half * 16;
        void *buf = nullptr;
        if ((e = cudaMalloc(&buf, comp_bytes * ncomp)) != cudaSuccess) {
            cudaGetLastError();
            return set_error(FC2T2_ERR_OOM, "cudaMalloc failed for packed moments");
        }
        pl->tc.packed[l] = buf;
        pl->tc.packed_bytes += (int64_t)(comp_bytes * ncomp);
        pl->tc.level_ok[l] = 1;
        if ((e = cudaMemset(buf, 0, comp_bytes * ncomp)) != cudaSuccess) return check_cuda(e, "clear packed moments");
        for (int comp = 0; comp < ncomp; ++comp) {
            // bytes of a row of x cells innermost (160-byte box rows), then y, chunk, (sigma, z)
            cuuint64_t dims[4] = {(cuuint64_t)16 * half, (cuuint64_t)half, (cuuint64_t)nkc, (cuuint64_t)8 * (half + 2)};
            cuuint64_t strides[3] = {(cuuint64_t)16 * half, (cuuint64_t)16 * half * half,
                                     (cuuint64_t)16 * half * half * nkc};
            cuuint32_t box[4] = {160, 18, (cuuint32_t)nkc, 1};
            cuuint32_t estr[4] = {1, 1, 1, 1};
            CUresult r = enc(reinterpret_cast<CUtensorMap *>(&pl->tc.maps[l][comp]), CU_TENSOR_MAP_DATA_TYPE_UINT8, 4,
                             static_cast<unsigned char *>(buf) + comp * comp_bytes, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            // a level whose grid the descriptor cannot describe keeps the CUDA-core M2L
            if (r != CUDA_SUCCESS) pl->tc.level_ok[l] = 0;
        }
        if (ncomp == 1) std::memcpy(&pl->tc.maps[l][1], &pl->tc.maps[l][0], sizeof(pl->tc.maps[l][0]));
    }
    pl->tc.mode = mode;
    pl->tc.img_bytes = img;
    pl->tc.ncomp = ncomp;
    pl->tc.pn = pn;
    pl->tc.kbytes = kfull * esz;
    pl->tc.nchunks = (int)ch.size();
    for (size_t i = 0; i < ch.size(); ++i) {
        pl->tc.n0[i] = ch[i].n0; pl->tc.N[i] = ch[i].N; pl->tc.K[i] = ch[i].K; pl->tc.b_off[i] = ch[i].b_off;
    }
    pl->tc.nbuf = nslab;
    pl->tc.nbslots = nbs;
    pl->tc.smem = smem;
    const int cols = 2 * pn;   // two accumulator buffers
    pl->tc.tmem_cols = cols <= 32 ? 32 : (cols <= 64 ? 64 : (cols <= 128 ? 128 : (cols <= 256 ? 256 : 512)));
    // MMA work issued per transform (2 x multiply-adds), for roofline reporting
    double per_op = 0.0;
    for (const TcChunk &c : ch) per_op += 2.0 * 128 * c.N * c.K * (split ? 3 : 1);
    double total = 0.0;
    for (int l = 0; l < pl->nlev; ++l) {
        const int half = pl->lev[l].n >> 1;
        const double tiles = 8.0 * ((half + 7) / 8) * ((half + 15) / 16) * half;
        pl->tc.mma_flops_level[l] = tiles * (l == 0 ? 216 : 189) * per_op;
        total += pl->tc.mma_flops_level[l];
    }
    pl->tc.mma_flops = total;
    pl->tc.enabled = 1;
    return FC2T2_OK;
}

// Pack every tensor-core level's moments, then run all those levels' M2L in one launch.
cudaError_t launch_m2l_tc_all(const fc2t2_plan_s *pl, cudaStream_t s) {
    const int nkc = pl->tc.kbytes / 16;
    TcArgs a;
    TcMaps maps;          // descriptors, copied into the launch parameters
    std::memset(&a, 0, sizeof(a));
    int nl_used = 0, block = 0;
    for (int level = 0; level < pl->nlev; ++level) {
        if (!pl->tc.level_ok[level]) continue;
        const Level &lv = pl->lev[level];
        const int half = lv.n >> 1;
        {
            const int64_t total = (int64_t)8 * half * half * half * nkc;
            const int64_t want = (total + 255) / 256;
            const unsigned blocks = (unsigned)(want < 152 * 16 ? want : 152 * 16);
            const float *M = pl->d_M + lv.off * pl->Pp;
            unsigned char *out = static_cast<unsigned char *>(pl->tc.packed[level]);
            pl->launches[FC2T2_STAGE_M2L] += 1;
            if (pl->tc.mode == 0) k_pack_tc<0><<<blocks, 256, 0, s>>>(M, out, lv.n, pl->Pp, nkc);
            else if (pl->tc.mode == 1) k_pack_tc<1><<<blocks, 256, 0, s>>>(M, out, lv.n, pl->Pp, nkc);
            else if (pl->tc.mode == 2) k_pack_tc<2><<<blocks, 256, 0, s>>>(M, out, lv.n, pl->Pp, nkc);
            else k_pack_tc<3><<<blocks, 256, 0, s>>>(M, out, lv.n, pl->Pp, nkc);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        TcLevel &t = a.lv[nl_used];
        t.L = pl->d_L + lv.off * pl->Pp;
        t.B = static_cast<const unsigned char *>(pl->d_mma_ops) + (size_t)level * 343 * pl->tc.ncomp * pl->tc.img_bytes;
        t.nl = lv.n;
        t.finest = level == 0 ? 1 : 0;
        t.tiles_x = (half + 7) / 8;
        t.tiles_y = (half + 15) / 16;
        t.block0 = block;
        std::memcpy(&maps.m[nl_used][0], &pl->tc.maps[level][0], sizeof(CUtensorMap));
        std::memcpy(&maps.m[nl_used][1], &pl->tc.maps[level][1], sizeof(CUtensorMap));
        block += 8 * t.tiles_x * t.tiles_y * half;
        ++nl_used;
    }
    if (nl_used == 0) return cudaSuccess;
    a.nlev = nl_used;
    a.err = pl->d_flags + 1;
    a.Pp = pl->Pp;
    a.nkc = nkc;
    a.img_bytes = pl->tc.img_bytes;
    a.ncomp_b = pl->tc.ncomp;
    a.nchunks = pl->tc.nchunks;
    for (int i = 0; i < kMaxChunks; ++i) {
        a.ch[i].n0 = 0; a.ch[i].N = pl->tc.N[i]; a.ch[i].K = 0; a.ch[i].b_off = pl->tc.b_off[i]; a.ch[i].k0 = 0;
    }
    a.pn = pl->tc.pn;
    a.tmem_cols = (uint32_t)pl->tc.tmem_cols;
    a.nslab = pl->tc.nbuf;
    a.nbslots = pl->tc.nbslots;
    const unsigned blocks = (unsigned)block;
    pl->launches[FC2T2_STAGE_M2L] += 1;
    const int key = pl->tc.mode * 8 + (a.pn <= 32 ? 0 : a.pn <= 64 ? 1 : a.pn <= 96 ? 2 : a.pn <= 128 ? 3 : 4);
#define FC2T2_TC_CASE(MODE_, IDX_, PN_)                                                                   \
    case (MODE_) * 8 + (IDX_):                                                                           \
        cudaFuncSetAttribute(k_m2l_tc<MODE_, PN_>, cudaFuncAttributeMaxDynamicSharedMemorySize, pl->tc.smem); \
        k_m2l_tc<MODE_, PN_><<<blocks, kTcThreads, pl->tc.smem, s>>>(maps, a);                            \
        break;
    switch (key) {
        FC2T2_TC_CASE(0, 0, 32) FC2T2_TC_CASE(0, 1, 64) FC2T2_TC_CASE(0, 2, 96) FC2T2_TC_CASE(0, 3, 128) FC2T2_TC_CASE(0, 4, 176)
        FC2T2_TC_CASE(1, 0, 32) FC2T2_TC_CASE(1, 1, 64) FC2T2_TC_CASE(1, 2, 96) FC2T2_TC_CASE(1, 3, 128) FC2T2_TC_CASE(1, 4, 176)
        FC2T2_TC_CASE(2, 0, 32) FC2T2_TC_CASE(2, 1, 64) FC2T2_TC_CASE(2, 2, 96) FC2T2_TC_CASE(2, 3, 128) FC2T2_TC_CASE(2, 4, 176)
        FC2T2_TC_CASE(3, 0, 32) FC2T2_TC_CASE(3, 1, 64) FC2T2_TC_CASE(3, 2, 96) FC2T2_TC_CASE(3, 3, 128) FC2T2_TC_CASE(3, 4, 176)
        default: return cudaErrorInvalidValue;
    }
#undef FC2T2_TC_CASE
    return cudaGetLastError();
}

}  // namespace fc2t2
