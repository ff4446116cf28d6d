// M2L on the tcgen05 tensor cores (Sec. 3: M2L as a convolution with a parity-dependent
// 6^D window and a 3^D hole; here as batched small dense contractions).
//
// For a target parity class pi and an offset o = 2 delta + sigma - pi (delta in {-1,0,1}^3,
// sigma the source parity) the M2L of every target of class pi is one GEMM
//     Lt[a, k] += sum_b  Mt_sigma[a + delta, b] * B_o[k, b],   B_o[k, b] = (-1)^|k| Dt_o[k+b]
// (|k| + |b| <= rho), with a the target's index in the half-resolution sub-grid.  A CTA owns
// 128 targets (8 x 16 sub-grid cells in x, y at one z) of one class: its accumulator is a
// 128 x Pn FP32 tile in tensor memory.  For each (sigma, delta_z) the CTA stages the 10 x 18
// cell "slab" of sub-grid sigma around its tile (converted to BF16 or TF32) in shared memory;
// the nine (delta_x, delta_y) operands are views of that slab that differ only in their start
// address.  The operators B_o are precomputed per level in the shared-memory image and fetched
// with bulk copies.  Because |k| + |b| <= rho, the k range is cut into chunks that only run
// over the b range they can reach (degree-block skipping), e.g. rho = 6: k in [0,16) x b < 96,
// [16,32) x b < 32, [32,96) x b < 16 -- 3072 of 9216 dense multiply-adds.
//
// Precision: BF16 or TF32 operands with FP32 accumulation, or TF32 x 3 (A_hi B_hi + A_hi B_lo
// + A_lo B_hi, the low parts being the TF32 rounding residues) which is accurate to FP32.
//
// Warp roles: warp 0 lane 0 issues bulk copies and MMAs; warps 1-4 stage slabs and, at the end,
// read the accumulator (each warp reads its TMEM lane quarter) and write Lt rows.
#include <cstring>
#include <vector>

#include "fc2t2_internal.cuh"
#include "tc_ptx.cuh"

namespace fc2t2 {

using namespace tc;

constexpr int kTcThreads = 160;
constexpr int kSlabCells = 180;          // 10 x 18 cells
constexpr int kMaxChunks = 4;
constexpr int kMaxBSlots = 8;

struct TcChunk {
    int n0, N, K;     // k columns [n0, n0 + N), b range [0, K)
    int b_off;        // byte offset of the chunk's block inside one operator image
};

struct TcArgs {
    const float *M;               // level coefficients [G][Pp]
    float *L;
    const unsigned char *B;       // operator images of this level: [343][ncomp][img_bytes]
    int *err;
    int nl;                       // cells per dimension at this level
    int Pp;
    int finest;                   // 1: no hole
    int kbytes;                   // bytes per slab row (covers the largest chunk K)
    int img_bytes;                // one operator image (one component)
    int ncomp_b;                  // 1, or 2 for TF32 x 3 (hi, lo)
    int nchunks;
    TcChunk ch[kMaxChunks];
    int pn;                       // accumulator columns used
    uint32_t tmem_cols;
    int nslab_buf;                // 1 or 2
    int nbslots;
    int tiles_x, tiles_y;         // tiles per parity class along x, y (z: half)
};

template <int MODE>   // 0: BF16, 1: TF32, 2: TF32 x 3
struct TcMode {
    static constexpr int esz = MODE == 0 ? 2 : 4;
    static constexpr int epc = 16 / esz;          // elements per 16-byte chunk
    static constexpr int eps = 32 / esz;          // elements per MMA K-step
    static constexpr int ncomp_a = MODE == 2 ? 2 : 1;
    static constexpr uint32_t fmt = MODE == 0 ? 1u : 2u;
};

template <int MODE, int PNMAX>
__global__ void __launch_bounds__(kTcThreads, 1) k_m2l_tc(const TcArgs args) {
    using Md = TcMode<MODE>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar_bfull[kMaxBSlots], bar_bfree[kMaxBSlots], bar_sfull[2], bar_sfree[2];
    __shared__ uint64_t bar_accfull[2], bar_accfree[2], bar_done;
    __shared__ uint32_t tmem_base;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int half = args.nl >> 1;
    // block -> (parity class, tile)
    const int tiles_per_class = args.tiles_x * args.tiles_y * half;
    const int pi = blockIdx.x / tiles_per_class;
    int tr = blockIdx.x % tiles_per_class;
    const int tx = tr % args.tiles_x;
    tr /= args.tiles_x;
    const int ty = tr % args.tiles_y;
    const int az = tr / args.tiles_y;
    const int ax0 = tx * 8, ay0 = ty * 16;
    const int pix = pi & 1, piy = (pi >> 1) & 1, piz = (pi >> 2) & 1;

    const int slab_bytes = kSlabCells * args.kbytes;             // one component
    const int slab_stride = slab_bytes * Md::ncomp_a;            // one buffer
    unsigned char *slabs = smem;
    unsigned char *bring = smem + ((args.nslab_buf * slab_stride + 1023) & ~1023);
    const int bslot_bytes = args.img_bytes * args.ncomp_b;

    if (threadIdx.x == 0) {
        for (int i = 0; i < args.nbslots; ++i) { mbar_init(&bar_bfull[i], 1); mbar_init(&bar_bfree[i], 1); }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar_sfull[i], 128);
            mbar_init(&bar_sfree[i], 1);
            mbar_init(&bar_accfull[i], 1);
            mbar_init(&bar_accfree[i], 128);
        }
        mbar_init(&bar_done, 1);
    }
    fence_proxy_async_smem();
    if (warp == 0) tmem_alloc(&tmem_base, args.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tacc = tmem_base;

    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------------------- issuer
            // operators in consumption order: step s = (sigma, dz), within a step (dx, dy);
            // above the finest level the 3^D hole is skipped
            int seq_o[216];
            unsigned char seq_step[216];
            int nseq = 0;
            for (int s = 0; s < 24; ++s) {
                const int sg = s / 3, dz = s % 3 - 1;
                const int sx = sg & 1, sy = (sg >> 1) & 1, sz = sg >> 2;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int ox = 2 * dx + sx - pix, oy = 2 * dy + sy - piy, oz = 2 * dz + sz - piz;
                        const bool hole = !args.finest && ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 &&
                                          oz <= 1;
                        if (hole) continue;
                        seq_o[nseq] = ((ox + 3) + 7 * (oy + 3) + 49 * (oz + 3)) | ((dx + 1) << 16) | ((dy + 1) << 20);
                        seq_step[nseq] = (unsigned char)s;
                        ++nseq;
                    }
            }
            int issued = 0;
            auto load_b = [&](int j) {
                issued = j + 1;
                const int slot = j % args.nbslots;
                const int olin = seq_o[j] & 0xFFFF;
                mbar_arrive_expect_tx(&bar_bfull[slot], (uint32_t)bslot_bytes);
                bulk_g2s(bring + slot * bslot_bytes, args.B + (size_t)olin * bslot_bytes, (uint32_t)bslot_bytes,
                         &bar_bfull[slot]);
            };
            const int pre = nseq < args.nbslots ? nseq : args.nbslots;
            for (int j = 0; j < pre; ++j) load_b(j);
            const uint32_t lboA = kSlabCells * 16, sboA = 160;
            int j = 0;
            for (int s = 0; s < 24 && ok; ++s) {
                const int buf = s % args.nslab_buf;
                const int use = s / args.nslab_buf;    // earlier fills of this slab buffer
                const int ab = s & 1;                  // accumulator buffer of this step
                if (s >= 2 && !mbar_wait(&bar_accfree[ab], ((s - 2) >> 1) & 1, args.err, 4)) { ok = false; break; }
                if (!mbar_wait(&bar_sfull[buf], use & 1, args.err, 4)) { ok = false; break; }
                tc_fence_after();
                const uint32_t slab_a = smem_u32(slabs + buf * slab_stride);
                const uint32_t acc_col = tacc + (uint32_t)(ab * args.pn);
                uint32_t started = 0;                  // bit c: chunk c written in this step
                for (; j < nseq && seq_step[j] == s; ++j) {
                    const int slot = j % args.nbslots;
                    if (!mbar_wait(&bar_bfull[slot], (j / args.nbslots) & 1, args.err, 8)) { ok = false; break; }
                    tc_fence_after();
                    const int dx = ((seq_o[j] >> 16) & 0xF) - 1, dy = ((seq_o[j] >> 20) & 0xF) - 1;
                    const uint32_t b_img = smem_u32(bring + slot * bslot_bytes);
                    const uint32_t a_view = slab_a + (uint32_t)(((dy + 1) * 10 + (dx + 1)) * 16);
                    for (int c = 0; c < args.nchunks; ++c) {
                        const TcChunk &chk = args.ch[c];
                        const uint32_t lboB = (uint32_t)(chk.N / 8) * 128u;
                        const uint32_t idesc = instr_desc(Md::fmt, (uint32_t)chk.N);
                        const uint32_t dcol = acc_col + (uint32_t)chk.n0;
                        const int nks = chk.K / Md::eps;
                        // passes: (A_hi, B_hi); for TF32 x 3 also (A_hi, B_lo), (A_lo, B_hi)
                        for (int pass = 0; pass < (MODE == 2 ? 3 : 1); ++pass) {
                            const uint32_t abase = a_view + (pass == 2 ? (uint32_t)slab_bytes : 0u);
                            const uint32_t bbase =
                                b_img + (uint32_t)chk.b_off + (pass == 1 ? (uint32_t)args.img_bytes : 0u);
                            for (int ks = 0; ks < nks; ++ks) {
                                const uint64_t ad = smem_desc(abase + (uint32_t)ks * 2u * lboA, lboA, sboA);
                                const uint64_t bd = smem_desc(bbase + (uint32_t)ks * 2u * lboB, lboB, 128u);
                                const uint32_t accum = (started >> c) & 1u;
                                if (MODE == 0) mma_bf16(dcol, ad, bd, idesc, accum);
                                else mma_tf32(dcol, ad, bd, idesc, accum);
                                started |= 1u << c;
                            }
                        }
                    }
                    mma_commit(&bar_bfree[slot]);
                    // refill the previous operator's slot once its MMAs have completed
                    if (j >= 1) {
                        const int jp = j - 1 + args.nbslots;
                        if (jp < nseq && jp >= args.nbslots) {
                            const int ps = (j - 1) % args.nbslots;
                            if (!mbar_wait(&bar_bfree[ps], ((j - 1) / args.nbslots) & 1, args.err, 16)) { ok = false; break; }
                            load_b(jp);
                        }
                    }
                }
                if (!ok) break;
                mma_commit(&bar_sfree[buf]);
                mma_commit(&bar_accfull[ab]);
            }
            mma_commit(&bar_done);
            // after an error, wait (bounded) for operator copies still in flight
            for (int jj = j; jj < issued; ++jj)
                mbar_wait(&bar_bfull[jj % args.nbslots], (jj / args.nbslots) & 1, args.err, 128);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- stagers / epilogue
        const int ts = threadIdx.x - 32;
        const int nkc = args.kbytes / 16;
        const int q = warp & 3;                 // TMEM lane quarter of this warp
        float acc[PNMAX];
#pragma unroll
        for (int i = 0; i < PNMAX; ++i) acc[i] = 0.0f;
        // add the partial sums of step u (accumulator buffer u & 1) into FP32 registers
        auto flush = [&](int u) {
            const int ab = u & 1;
            if (!mbar_wait(&bar_accfull[ab], (u >> 1) & 1, args.err, 32)) { ok = false; return; }
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
        };
        for (int s = 0; s < 24 && ok; ++s) {
            const int buf = s % args.nslab_buf;
            const int use = s / args.nslab_buf;
            if (use >= 1 && !mbar_wait(&bar_sfree[buf], (use - 1) & 1, args.err, 32)) { ok = false; break; }
            const int sg = s / 3, dz = s % 3 - 1;
            const int sx = sg & 1, sy = (sg >> 1) & 1, sz = sg >> 2;
            unsigned char *dst = slabs + buf * slab_stride;
            const int cz = az + dz;
            for (int idx = ts; idx < nkc * kSlabCells; idx += 128) {
                const int cell = idx % kSlabCells, kc = idx / kSlabCells;
                const int cx = ax0 - 1 + cell % 10, cy = ay0 - 1 + cell / 10;
                const bool in = cx >= 0 && cx < half && cy >= 0 && cy < half && cz >= 0 && cz < half;
                const int k0 = kc * Md::epc;
                float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                if (in) {
                    const int64_t lin = (int64_t)(2 * cx + sx) +
                                        (int64_t)args.nl * ((2 * cy + sy) + (int64_t)args.nl * (2 * cz + sz));
                    const float *row = args.M + lin * args.Pp;
#pragma unroll
                    for (int q4 = 0; q4 < Md::epc / 4; ++q4) {
                        if (k0 + 4 * q4 + 4 <= args.Pp) {
                            const float4 f = __ldg(reinterpret_cast<const float4 *>(row + k0 + 4 * q4));
                            v[4 * q4] = f.x; v[4 * q4 + 1] = f.y; v[4 * q4 + 2] = f.z; v[4 * q4 + 3] = f.w;
                        }
                    }
                }
                unsigned char *d16 = dst + ((size_t)kc * kSlabCells + cell) * 16;
                if (MODE == 0) {
                    *reinterpret_cast<uint4 *>(d16) = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]),
                                                                 pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
                } else {
                    float h[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) h[e] = round_tf32(v[e]);
                    *reinterpret_cast<uint4 *>(d16) = make_uint4(__float_as_uint(h[0]), __float_as_uint(h[1]),
                                                                 __float_as_uint(h[2]), __float_as_uint(h[3]));
                    if (MODE == 2)
                        *reinterpret_cast<uint4 *>(d16 + slab_bytes) = make_uint4(
                            __float_as_uint(round_tf32(v[0] - h[0])), __float_as_uint(round_tf32(v[1] - h[1])),
                            __float_as_uint(round_tf32(v[2] - h[2])), __float_as_uint(round_tf32(v[3] - h[3])));
                }
            }
            fence_proxy_async_smem();
            mbar_arrive(&bar_sfull[buf]);
            if (s >= 1) flush(s - 1);
        }
        if (ok) flush(23);
        // ---------------------------------------------------------------- write Lt rows
        if (ok) {
            const int r = q * 32 + lane;            // tile row
            const int x = ax0 + (r & 7), y = ay0 + (r >> 3);
            if (x < half && y < half) {
                const int64_t t = (int64_t)(2 * x + pix) +
                                  (int64_t)args.nl * ((2 * y + piy) + (int64_t)args.nl * (2 * az + piz));
                float *Lrow = args.L + t * args.Pp;
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

// Split [0, Pn) into at most kMaxChunks column chunks (multiples of 16) minimising the dense
// multiply-adds sum N_c K_c, where chunk c only needs b of degree <= rho - deg(first k).
void plan_chunks(int D, int rho, int P, int kg, std::vector<TcChunk> &out, int &pn, int &kfull) {
    pn = (P + 15) / 16 * 16;
    const int nb = pn / 16;
    auto kneed = [&](int n0) {
        const int d = degree_of(D, n0 < P ? n0 : P - 1);
        const int cnt = ncoef(D, rho - d);
        return (cnt + kg - 1) / kg * kg;
    };
    // dp[i][c]: best cost covering blocks [i, nb) with c chunks left
    const long INF = 1L << 60;
    std::vector<std::vector<long>> dp(nb + 1, std::vector<long>(kMaxChunks + 1, INF));
    std::vector<std::vector<int>> nxt(nb + 1, std::vector<int>(kMaxChunks + 1, -1));
    for (int c = 0; c <= kMaxChunks; ++c) dp[nb][c] = 0;
    for (int i = nb - 1; i >= 0; --i)
        for (int c = 1; c <= kMaxChunks; ++c)
            for (int e = i + 1; e <= nb; ++e) {
                const long cost = (long)(e - i) * 16 * kneed(16 * i) + dp[e][c - 1];
                if (cost < dp[i][c]) { dp[i][c] = cost; nxt[i][c] = e; }
            }
    out.clear();
    int i = 0, c = kMaxChunks;
    kfull = 0;
    while (i < nb) {
        const int e = nxt[i][c];
        TcChunk ch;
        ch.n0 = 16 * i;
        ch.N = 16 * (e - i);
        ch.K = kneed(16 * i);
        ch.b_off = 0;
        if (ch.K > kfull) kfull = ch.K;
        out.push_back(ch);
        i = e;
        --c;
    }
}

uint16_t to_bf16(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float to_tf32(float x) {   // round half away from zero on the 13 dropped bits (cvt.rna)
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x1000u;
    u &= 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

}  // namespace

// Build the tensor-core operator images of every level from the FP32/FP64 derivative table.
fc2t2_status build_tc_operators(fc2t2_plan_s *pl, const std::vector<double> &dtab64) {
    pl->tc.enabled = 0;
    if (pl->D != 3) return FC2T2_OK;
    const int mode = pl->desc.m2l == FC2T2_M2L_BF16 ? 0 : (pl->desc.m2l == FC2T2_M2L_TF32 ? 1 : 2);
    // a bounded issuer: remember in-flight operator loads to drain them on an error
    const int esz = mode == 0 ? 2 : 4, epc = 16 / esz, kg = 32 / esz;
    std::vector<TcChunk> ch;
    int pn = 0, kfull = 0;
    plan_chunks(pl->D, pl->rho, pl->P, kg, ch, pn, kfull);
    int off = 0;
    for (auto &c : ch) { c.b_off = off; off += c.N * c.K * esz; }
    const int img = off;
    const int ncomp = mode == 2 ? 2 : 1;
    const int nofs = 343;
    // degree of every graded index
    std::vector<int> deg(pl->P);
    for (int k = 0; k < pl->P; ++k) deg[k] = degree_of(pl->D, k);
    // graded index of k + b: via exponents
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
                        const int kap = c.n0 + n, b = k;
                        double v = 0.0;
                        if (kap < pl->P && b < pl->P && deg[kap] + deg[b] <= pl->rho) {
                            const int m = gidx3(ex[3 * kap] + ex[3 * b], ex[3 * kap + 1] + ex[3 * b + 1],
                                                ex[3 * kap + 2] + ex[3 * b + 2]);
                            v = (deg[kap] & 1) ? -Dt[m] : Dt[m];
                        }
                        const size_t pos = (size_t)c.b_off + ((size_t)(k / epc) * (c.N / 8) + n / 8) * 128 +
                                           (n % 8) * 16 + (k % epc) * esz;
                        if (mode == 0) {
                            const uint16_t h = to_bf16((float)v);
                            std::memcpy(base + pos, &h, 2);
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
    // remember the layout
    pl->tc.mode = mode;
    pl->tc.img_bytes = img;
    pl->tc.ncomp = ncomp;
    pl->tc.pn = pn;
    pl->tc.kbytes = kfull * esz;
    pl->tc.nchunks = (int)ch.size();
    for (size_t i = 0; i < ch.size(); ++i) {
        pl->tc.n0[i] = ch[i].n0; pl->tc.N[i] = ch[i].N; pl->tc.K[i] = ch[i].K; pl->tc.b_off[i] = ch[i].b_off;
    }
    // shared memory: slab buffers + operator ring
    const int ncomp_a = mode == 2 ? 2 : 1;
    const int slab = kSlabCells * pl->tc.kbytes * ncomp_a;
    const int bslot = img * ncomp;
    int best = -1;
    for (int nbuf = 2; nbuf >= 1 && best < 0; --nbuf)
        for (int nbs = kMaxBSlots; nbs >= 2; --nbs) {
            const size_t bytes = (size_t)((nbuf * slab + 1023) & ~1023) + (size_t)nbs * bslot;
            if (bytes <= 200 * 1024) { pl->tc.nbuf = nbuf; pl->tc.nbslots = nbs; pl->tc.smem = (int)bytes; best = 1; break; }
        }
    pl->tc.enabled = (best > 0 && pl->D == 3 && pn <= 256) ? 1 : 0;
    const int cols = 2 * pn;   // two accumulator buffers
    pl->tc.tmem_cols = cols <= 32 ? 32 : (cols <= 64 ? 64 : (cols <= 128 ? 128 : (cols <= 256 ? 256 : 512)));
    return FC2T2_OK;
}

cudaError_t launch_m2l_tc(const fc2t2_plan_s *pl, cudaStream_t s, int level) {
    const Level &lv = pl->lev[level];
    TcArgs a;
    a.M = pl->d_M + lv.off * pl->Pp;
    a.L = pl->d_L + lv.off * pl->Pp;
    a.B = static_cast<const unsigned char *>(pl->d_mma_ops) + (size_t)level * 343 * pl->tc.ncomp * pl->tc.img_bytes;
    a.err = pl->d_flags + 1;
    a.nl = lv.n;
    a.Pp = pl->Pp;
    a.finest = level == 0 ? 1 : 0;
    a.kbytes = pl->tc.kbytes;
    a.img_bytes = pl->tc.img_bytes;
    a.ncomp_b = pl->tc.ncomp;
    a.nchunks = pl->tc.nchunks;
    for (int i = 0; i < kMaxChunks; ++i) {
        a.ch[i].n0 = pl->tc.n0[i]; a.ch[i].N = pl->tc.N[i]; a.ch[i].K = pl->tc.K[i]; a.ch[i].b_off = pl->tc.b_off[i];
    }
    a.pn = pl->tc.pn;
    a.tmem_cols = (uint32_t)pl->tc.tmem_cols;
    a.nslab_buf = pl->tc.nbuf;
    a.nbslots = pl->tc.nbslots;
    const int half = lv.n >> 1;
    a.tiles_x = (half + 7) / 8;
    a.tiles_y = (half + 15) / 16;
    const unsigned blocks = (unsigned)(8 * a.tiles_x * a.tiles_y * half);
    pl->launches[FC2T2_STAGE_M2L] += 1;
    const int key = pl->tc.mode * 8 + (a.pn <= 32 ? 0 : a.pn <= 64 ? 1 : a.pn <= 96 ? 2 : a.pn <= 128 ? 3 : 4);
#define FC2T2_TC_CASE(MODE_, IDX_, PN_)                                                                   \
    case (MODE_) * 8 + (IDX_):                                                                           \
        cudaFuncSetAttribute(k_m2l_tc<MODE_, PN_>, cudaFuncAttributeMaxDynamicSharedMemorySize, pl->tc.smem); \
        k_m2l_tc<MODE_, PN_><<<blocks, kTcThreads, pl->tc.smem, s>>>(a);                                  \
        break;
    switch (key) {
        FC2T2_TC_CASE(0, 0, 32) FC2T2_TC_CASE(0, 1, 64) FC2T2_TC_CASE(0, 2, 96) FC2T2_TC_CASE(0, 3, 128) FC2T2_TC_CASE(0, 4, 176)
        FC2T2_TC_CASE(1, 0, 32) FC2T2_TC_CASE(1, 1, 64) FC2T2_TC_CASE(1, 2, 96) FC2T2_TC_CASE(1, 3, 128) FC2T2_TC_CASE(1, 4, 176)
        FC2T2_TC_CASE(2, 0, 32) FC2T2_TC_CASE(2, 1, 64) FC2T2_TC_CASE(2, 2, 96) FC2T2_TC_CASE(2, 3, 128) FC2T2_TC_CASE(2, 4, 176)
        default: return cudaErrorInvalidValue;
    }
#undef FC2T2_TC_CASE
    return cudaGetLastError();
}

}  // namespace fc2t2
