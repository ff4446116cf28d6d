// M2L on the tcgen05 tensor cores (Sec. 3: M2L as a convolution with a parity-dependent
// 6^D window and a 3^D hole; here as batched small dense contractions).
//
// For a target parity class pi and an offset o = 2 delta + sigma - pi (delta in {-1,0,1}^3,
// sigma the source parity) the M2L of every target of class pi is one GEMM
//     Lt[a, k] += sum_b  Mt_sigma[a + delta, b] * B_o[k, b],   B_o[k, b] = (-1)^|k| Dt_o[k+b]
// (|k| + |b| <= rho), with a the target's index in the half-resolution sub-grid.  The moment
// view Mt_sigma[a + delta] does not depend on pi: all eight classes read the same 216 views and
// differ only in the operator.  A CTA therefore owns 128 sub-grid cells (8 x 16 in x, y at one z)
// for a group of 1, 2 or 4 classes (pi_x, and pi_y, free), and each MMA multiplies one view by
// the operators of all classes of the group at once: its accumulator columns interleave the
// classes (column = classes * k + class), so one read of the A operand from shared memory -- the
// cost that bounds these narrow MMAs -- serves every class.  Orders <= 5 use four classes, 6 and
// 7 two (the two TMEM accumulator buffers must fit 512 columns and one MMA at most N = 256).
//
// Operands.  A pack kernel rewrites each level's moments once into the tensor-core layout:
// per source parity sigma and sub-grid z, 16-byte chunks of 8 BF16 (or 4 TF32) coefficients
// ordered [chunk][y][x] -- exactly the canonical no-swizzle K-major layout, so one TMA tensor
// load brings the 10 x 18 cell "slab" of sub-grid sigma around the tile into shared memory
// (cells outside the grid arrive as zeros).  The nine (delta_x, delta_y) A operands of a slab
// are views that differ only in their start address.  The operators of each class group and
// offset are precomputed per level as shared-memory images and fetched with bulk copies.
// Because |k| + |b| <= rho, each MMA K-step (16 BF16 or 8 TF32 values of b) only reaches the k of
// degree <= rho - min|b| of the step, so its N shrinks with the degree of b (degree-block
// skipping): rho = 6, BF16, two classes uses N = 176, 48, 32, 16, 16, 16 for its six K-steps.
//
// Precision: BF16 or TF32 operands with FP32 accumulation, or a split form (A_hi B_hi + A_hi B_lo
// + A_lo B_hi, the low parts being the rounding residues) in TF32 x 3 or BF16 x 3; both split
// forms are within the FP32 bar (1e-5 relative L2), BF16 x 3 with half the MMAs of TF32 x 3.  The tensor
// core's accumulation over thousands of MMAs loses low bits, so each step's partial sum is
// accumulated in its own TMEM buffer (two, alternating) and added into FP32 registers.
//
// Warp roles: warp 0 fetches slabs (TMA) and operators (bulk copies), warp 1 issues the MMAs
// (one elected lane, converged warp), warps 2-9 add each step's partial accumulator into FP32
// registers (a warp reads its TMEM lane quarter and one half of the columns) and finally write
// the Lt rows of every class.  Every wait is bounded in time.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "m2l_tc_kernel.cuh"

namespace fc2t2 {

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

// ------------------------------------------------------------------------------ host side

namespace {

int degree_of(int D, int k) {
    int d = 0;
    while (ncoef(D, d) <= k) ++d;
    return d;
}

// One chunk per MMA K-step of kg values of b: the step starting at b0 only reaches the k of
// degree <= rho - deg(b0), i.e. the first ncoef(rho - deg(b0)) coefficients of each of the ncls
// classes (accumulator columns interleave the classes), rounded up to 16 columns.
void plan_chunks(int D, int rho, int P, int kg, int ncls, int pnb, std::vector<TcChunk> &out, int &kfull) {
    kfull = (P + kg - 1) / kg * kg;
    out.clear();
    for (int k0 = 0; k0 < kfull; k0 += kg) {
        const int need = ncoef(D, rho - degree_of(D, k0)) * ncls;
        TcChunk ch;
        ch.k0 = k0;
        ch.K = kg;
        ch.n0 = 0;
        ch.N = (need + 15) / 16 * 16;
        if (ch.N > pnb) ch.N = pnb;
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
    const int P = pl->P;
    const int ncomp = split ? 2 : 1;
    const int nofs = 343;
    const int max_steps = bf16 ? 11 : 21;
    // Classes per CTA: as many as fit the MMA width (N <= 256) and two accumulator buffers in
    // TMEM (2 * pnb <= 512 columns), with a shared-memory plan of >= 2 slab and >= 3 operator
    // slots (one class: >= 1 and >= 2).  One CTA per SM when the buffers take all of TMEM.
    std::vector<TcChunk> ch;
    int kfull = 0, ncls = 0, kh = 0, pnb = 0, img = 0, nslab = 0, nbs = 0, smem = 0, nkc = 0, ksc = 0;
    for (int nc : {4, 2, 1}) {
        if (nc * P > 256) continue;
        const int kq = std::max(4, 16 / nc);
        const int khc = ((P + 1) / 2 + kq - 1) / kq * kq;
        const int pnbc = 2 * nc * khc;
        if (pnbc > 256) continue;
        std::vector<TcChunk> chc;
        int kf = 0;
        plan_chunks(pl->D, pl->rho, P, kg, nc, pnbc, chc, kf);
        if ((int)chc.size() > max_steps || (int)chc.size() > kMaxChunks) continue;
        int kscc = 0;
        while (kscc < 3 && tc_ksteps(bf16, kscc) < (int)chc.size()) ++kscc;
        if (!tc_variant(nc, kscc)) continue;
        int off = 0;
        for (auto &c : chc) { c.b_off = off; off += c.N * c.K * esz; }
        const int nkcc = kf * esz / 16;
        const int slab = ((kSlabCells * 16 * nkcc + 1023) & ~1023) * ncomp;   // as in the kernel
        const int bslot = off * ncomp;
        const int min_ns = nc == 1 ? 1 : 2, min_nb = nc == 1 ? 2 : 3;
        int ns_ok = 0, nb_ok = 0, bytes_ok = 0;
        // preference: two or three slab slots (the next slab loads during this one's MMAs) with
        // a deep operator ring (bulk-copy latency), then whatever fits above the minimum
        auto try_fit = [&](int ns, int nb) {
            const int bytes = ((ns * slab + 1023) & ~1023) + nb * bslot;
            if (ns_ok || ns < min_ns || nb < min_nb || bytes > 220 * 1024) return;
            ns_ok = ns; nb_ok = nb; bytes_ok = bytes;
        };
        for (int nb = kMaxBSlots; nb >= 4; --nb) { try_fit(3, nb); try_fit(2, nb); }
        try_fit(2, 3);
        try_fit(2, 2);
        for (int nb = kMaxBSlots; nb >= 2; --nb) try_fit(1, nb);
        if (!ns_ok) continue;
        ch = chc; kfull = kf; ncls = nc; kh = khc; pnb = pnbc; img = off; ksc = kscc;
        nslab = ns_ok; nbs = nb_ok; smem = bytes_ok; nkc = nkcc;
        break;
    }
    if (!ncls) return FC2T2_OK;   // too large for shared memory: the CUDA-core M2L runs instead
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
    // image o (offset of the group's class 0) holds, in row n = ncls * kappa + c, the operator of
    // class c at offset o - (c & 1, c >> 1, 0); zero where that offset is outside the 7^3 stencil
    // or, above the finest level, in the hole
    std::vector<unsigned char> host((size_t)pl->nlev * nofs * ncomp * img, 0);
    for (int l = 0; l < pl->nlev; ++l)
        for (int o = 0; o < nofs; ++o) {
            unsigned char *base = host.data() + ((size_t)l * nofs + o) * ncomp * img;
            const int ox = o % 7 - 3, oy = (o / 7) % 7 - 3, oz = o / 49 - 3;
            for (const TcChunk &c : ch)
                for (int n = 0; n < c.N; ++n)
                    for (int k = 0; k < c.K; ++k) {
                        const int kap = n / ncls, cls = n % ncls, b = c.k0 + k;
                        const int oxc = ox - (ncls >= 2 ? (cls & 1) : 0), oyc = oy - (ncls >= 4 ? (cls >> 1) : 0);
                        const bool inside = oxc >= -3 && oxc <= 3 && oyc >= -3 && oyc <= 3;
                        const bool hole = oxc >= -1 && oxc <= 1 && oyc >= -1 && oyc <= 1 && oz >= -1 && oz <= 1;
                        double v = 0.0;
                        if (inside && !(l > 0 && hole) && kap < P && b < P && deg[kap] + deg[b] <= pl->rho) {
                            const double *Dt =
                                dtab64.data() + ((size_t)l * nofs + (oxc + 3) + 7 * (oyc + 3) + 49 * (oz + 3)) * P;
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
    pl->tc.ncls = ncls;
    pl->tc.ksc = ksc;
    pl->tc.kh = kh;
    pl->tc.pnb = pnb;
    pl->tc.kbytes = kfull * esz;
    pl->tc.nchunks = (int)ch.size();
    for (size_t i = 0; i < ch.size(); ++i) {
        pl->tc.n0[i] = ch[i].n0; pl->tc.N[i] = ch[i].N; pl->tc.K[i] = ch[i].K; pl->tc.b_off[i] = ch[i].b_off;
    }
    pl->tc.nbuf = nslab;
    pl->tc.nbslots = nbs;
    const int cols = 2 * pnb;   // two accumulator buffers
    pl->tc.tmem_cols = cols <= 32 ? 32 : (cols <= 64 ? 64 : (cols <= 128 ? 128 : (cols <= 256 ? 256 : 512)));
    // a CTA that takes all of TMEM asks for more than half the shared memory, so that a second
    // CTA is never placed on its SM to wait in the TMEM allocation
    if (pl->tc.tmem_cols == 512 && smem < 116 * 1024) smem = 116 * 1024;
    pl->tc.smem = smem;
    // MMA work issued per transform (2 x multiply-adds), for roofline reporting: every class
    // group of a tile issues one MMA sequence per view it does not skip
    double per_view = 0.0;
    for (const TcChunk &c : ch) per_view += 2.0 * 128 * c.N * c.K * (split ? 3 : 1);
    double total = 0.0;
    for (int l = 0; l < pl->nlev; ++l) {
        const int half = pl->lev[l].n >> 1;
        const double tiles = (double)((half + 7) / 8) * ((half + 15) / 16) * half;
        double views = 0.0;
        for (int g = 0; g < 8 / ncls; ++g) {
            int gb = g;
            const int pix0 = ncls >= 2 ? 0 : (gb & 1);
            if (ncls < 2) gb >>= 1;
            const int piy0 = ncls >= 4 ? 0 : (gb & 1);
            if (ncls < 4) gb >>= 1;
            const int piz = gb & 1;
            for (int sg = 0; sg < 8; ++sg)
                for (int d = 0; d < 27; ++d) {
                    const int ox = 2 * (d % 3 - 1) + (sg & 1) - pix0, oy = 2 * ((d / 3) % 3 - 1) + ((sg >> 1) & 1) - piy0;
                    const int oz = 2 * (d / 9 - 1) + (sg >> 2) - piz;
                    bool any = l == 0 || oz < -1 || oz > 1;
                    for (int c = 0; c < ncls && !any; ++c) {
                        const int oxc = ox - (ncls >= 2 ? (c & 1) : 0), oyc = oy - (ncls >= 4 ? (c >> 1) : 0);
                        if (oxc < -1 || oxc > 1 || oyc < -1 || oyc > 1) any = true;
                    }
                    if (any) views += 1.0;
                }
        }
        pl->tc.mma_flops_level[l] = tiles * views * per_view;
        total += pl->tc.mma_flops_level[l];
    }
    pl->tc.mma_flops = total;
    pl->tc.enabled = 1;
    return FC2T2_OK;
}

// Rewrite every tensor-core level's moments into the packed operand layout.
cudaError_t launch_tc_pack(const fc2t2_plan_s *pl, cudaStream_t s) {
    const int nkc = pl->tc.kbytes / 16;
    for (int level = 0; level < pl->nlev; ++level) {
        if (!pl->tc.level_ok[level]) continue;
        const Level &lv = pl->lev[level];
        const int half = lv.n >> 1;
        const int64_t total = (int64_t)8 * half * half * half * nkc;
        const int64_t want = (total + 255) / 256;
        const unsigned blocks = (unsigned)(want < 152 * 16 ? want : 152 * 16);
        const float *M = pl->d_M + lv.off * pl->Pp;
        unsigned char *out = static_cast<unsigned char *>(pl->tc.packed[level]);
        pl->launches[FC2T2_STAGE_M2L_PACK] += 1;
        if (pl->tc.mode == 0) k_pack_tc<0><<<blocks, 256, 0, s>>>(M, out, lv.n, pl->Pp, nkc);
        else if (pl->tc.mode == 1) k_pack_tc<1><<<blocks, 256, 0, s>>>(M, out, lv.n, pl->Pp, nkc);
        else if (pl->tc.mode == 2) k_pack_tc<2><<<blocks, 256, 0, s>>>(M, out, lv.n, pl->Pp, nkc);
        else k_pack_tc<3><<<blocks, 256, 0, s>>>(M, out, lv.n, pl->Pp, nkc);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Run the M2L of every tensor-core level in one launch (the moments are packed already).
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
        block += (8 / pl->tc.ncls) * t.tiles_x * t.tiles_y * half;
        ++nl_used;
    }
    if (nl_used == 0) return cudaSuccess;
    a.nlev = nl_used;
    a.err = pl->d_flags + 2;
    a.Pp = pl->Pp;
    a.nkc = nkc;
    a.img_bytes = pl->tc.img_bytes;
    a.ncomp_b = pl->tc.ncomp;
    a.nchunks = pl->tc.nchunks;
    for (int i = 0; i < kMaxChunks; ++i) a.ch[i] = make_int2(pl->tc.N[i], pl->tc.b_off[i]);
    a.kh = pl->tc.kh;
    a.pnb = pl->tc.pnb;
    a.tmem_cols = (uint32_t)pl->tc.tmem_cols;
    a.nslab = pl->tc.nbuf;
    a.nbslots = pl->tc.nbslots;
    const unsigned blocks = (unsigned)block;
    pl->launches[FC2T2_STAGE_M2L] += 1;
    switch (pl->tc.mode) {
        case 0: return launch_m2l_tc_mode<0>(pl->tc.ncls, pl->tc.ksc, blocks, pl->tc.smem, s, maps, a);
        case 1: return launch_m2l_tc_mode<1>(pl->tc.ncls, pl->tc.ksc, blocks, pl->tc.smem, s, maps, a);
        case 2: return launch_m2l_tc_mode<2>(pl->tc.ncls, pl->tc.ksc, blocks, pl->tc.smem, s, maps, a);
        case 3: return launch_m2l_tc_mode<3>(pl->tc.ncls, pl->tc.ksc, blocks, pl->tc.smem, s, maps, a);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fc2t2
