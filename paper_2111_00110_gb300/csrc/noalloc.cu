// fc2t2_forward_noalloc: the forward transform without any device allocation.
//
// Some callers cannot call cudaMalloc at the moment they need a transform: code running
// inside a framework that owns all device memory through its own pool (and forbids foreign
// allocations), real-time or embedded loops that must not allocate after start-up, and
// callbacks that run while another component holds the allocator.  For them this entry
// point needs no plan: everything the transform keeps between kernels (the cell sort, the
// moment and local coefficients of every level, and the operator tables) lives in one
// file-scope device array, sized for small problems (limits below).
//
// The array is part of the library image: every GPU that loads the library holds it
// (kScratchBytes) until the process exits.  All calls share it, and it keeps the previous
// call's contents; everything that must start from zero is cleared by the call itself, and the
// operator tables are rebuilt on the device by every call (a small kernel, FP64 arithmetic), so
// no host memory is read after the call returns.  Two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array and give wrong results:
// issue them on one stream, one after the other.
//
// Host code cannot use the array's name as a device pointer.  Every call asks the runtime for
// the array's device address on the current device (cudaGetSymbolAddress; not a stream
// operation), so the address is never stale, even after a device reset.  The first call on a
// device also loads the library's device code there (set-up), so make the first call outside
// any CUDA stream capture.
#include <cmath>

#include "fc2t2_internal.cuh"

namespace fc2t2 {
namespace {

// Limits of the allocation-free path.
constexpr int kNaMaxCells = 4096;          // finest cells: 64^2 in 2D, 16^3 in 3D
constexpr int kNaMaxOrder = 4;             // P <= 35 (3D), Pp <= 36
constexpr int64_t kNaMaxPoints = 65536;    // sources and queries, each
constexpr int kNaMaxPp = 36;
constexpr int kNaMaxLevels = 5;            // 64^2: 64, 32, 16, 8, 4
constexpr int64_t kNaMaxCellsAllLevels = kNaMaxCells * 4 / 3 + 16;
constexpr int kNaOffsets = 343;            // 7^3 cell offsets

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr size_t kSortBytes =
    align256(sizeof(int) * kNaMaxCells) + align256(sizeof(int) * (kNaMaxCells + 1)) +
    3 * align256(sizeof(int) * kNaMaxPoints) + align256(sizeof(float4) * kNaMaxPoints);
constexpr size_t kScratchBytes =
    2 * align256(sizeof(float) * kNaMaxCellsAllLevels * kNaMaxPp) +                  // M, L
    align256(sizeof(float) * kNaMaxLevels * kNaOffsets * kNaMaxPp) +                 // dtab
    align256(sizeof(int) * 64) + align256(sizeof(int) * 4) +                         // scan, flags
    align256(sizeof(int2) * kNaMaxCells) + align256(sizeof(unsigned long long) * 2) + // P2M overflow list
    2 * kSortBytes;

}  // namespace

// The scratch array: kScratchBytes, about 6.1 MB.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

// Operator table on the device, as a plan builds it on the host (the same definition):
//   dtab[l][o][k] = h_l^|k| d^k psi(o h_l),  psi = exp(-|x|^2 / (2 sigma^2)),  o in {-3..3}^D,
// from the one-dimensional factors h^j g^(j)(x) (probabilists' Hermite recurrence in FP64).
// One block per (level, offset).
__device__ int na_exponents(int D, int rho, int k, int e[3]) {
    for (int d = 0; d <= rho; ++d)
        for (int a0 = d; a0 >= 0; --a0)
            for (int a1 = d - a0; a1 >= 0; --a1) {
                const int a2 = d - a0 - a1;
                if (D == 2 && a2) continue;
                if ((D == 2 ? gidx2(a0, a1) : gidx3(a0, a1, a2)) == k) {
                    e[0] = a0; e[1] = a1; e[2] = a2;
                    return d;
                }
            }
    e[0] = e[1] = e[2] = 0;
    return -1;
}

__global__ void k_na_tables(float *dtab, int D, int rho, int Pp, int nofs, double sigma, double h0) {
    const int l = blockIdx.x / nofs, o = blockIdx.x % nofs;
    const int P = ncoef(D, rho);
    const double h = h0 * (double)(1 << l);
    for (int k = threadIdx.x; k < Pp; k += blockDim.x) {
        float out = 0.0f;
        if (k < P) {
            int e[3];
            na_exponents(D, rho, k, e);
            double v = 1.0;
            int r = o;
            for (int d = 0; d < D; ++d) {
                const double x = (double)(r % 7 - 3) * h;
                r /= 7;
                const double t = x / sigma, g = exp(-0.5 * t * t), f = -h / sigma;
                double hem1 = 0.0, he = 1.0, fj = 1.0;     // He_j(t) and (-h/sigma)^j
                for (int j = 0; j < e[d]; ++j) {
                    const double hn = t * he - j * hem1;
                    hem1 = he; he = hn; fj *= f;
                }
                v *= fj * he * g;
            }
            out = (float)v;
        }
        dtab[(size_t)blockIdx.x * Pp + k] = out;
    }
}

template <typename T>
T *carve(unsigned char *base, size_t &off, size_t count) {
    T *p = reinterpret_cast<T *>(base + off);
    off += align256(sizeof(T) * count);
    return p;
}

}  // namespace
}  // namespace fc2t2

using namespace fc2t2;

extern "C" FC2T2_API fc2t2_status fc2t2_forward_noalloc(const fc2t2_plan_desc *desc, void *stream,
                                                        const float *p, const float *w, int64_t N,
                                                        const float *q, int64_t M, float *y) {
    if (!desc) return set_error(FC2T2_ERR_INVALID_ARG, "desc is NULL");
    if (desc->dim != 2 && desc->dim != 3) return set_error(FC2T2_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (desc->kernel != FC2T2_KERNEL_GAUSSIAN)
        return set_error(FC2T2_ERR_UNSUPPORTED, "the allocation-free path supports the Gaussian kernel only");
    if (!(desc->sigma > 0.0) || !std::isfinite(desc->sigma))
        return set_error(FC2T2_ERR_INVALID_ARG, "sigma must be positive");
    if (!(desc->hi > desc->lo) || !std::isfinite(desc->lo) || !std::isfinite(desc->hi))
        return set_error(FC2T2_ERR_INVALID_ARG, "domain must satisfy lo < hi");
    if (desc->channels != 1 || desc->m2l != FC2T2_M2L_FP32 || desc->fit != 0)
        return set_error(FC2T2_ERR_UNSUPPORTED, "the allocation-free path supports one channel, FP32 M2L, Taylor operators");
    if (desc->check_domain != 0)
        return set_error(FC2T2_ERR_UNSUPPORTED,
                         "the allocation-free path does not check the domain (points outside clamp to the edge cells); "
                         "set check_domain = 0 or use a plan");
    if (desc->grid < 4 || (desc->grid & (desc->grid - 1)))
        return set_error(FC2T2_ERR_INVALID_ARG, "grid must be a power of two >= 4");
    int64_t cells = 1;
    for (int d = 0; d < desc->dim; ++d) cells *= desc->grid;
    if (cells > kNaMaxCells)
        return set_error(FC2T2_ERR_INVALID_ARG,
                         "allocation-free path: grid^dim exceeds 4096 cells (64^2 or 16^3); use a plan");
    if (desc->order < 1 || desc->order > kNaMaxOrder)
        return set_error(FC2T2_ERR_INVALID_ARG, "allocation-free path: order must be in [1, 4]; use a plan");
    if (N < 0 || M < 0 || N > kNaMaxPoints || M > kNaMaxPoints)
        return set_error(FC2T2_ERR_INVALID_ARG,
                         "allocation-free path: N and M must be in [0, 65536]; use a plan");
    if (M == 0) return FC2T2_OK;
    if (!q || !y || (N > 0 && (!p || !w))) return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;

    // the array's device address on the current device (looked up on every call)
    void *addr = nullptr;
    fc2t2_status st = check_cuda(cudaGetSymbolAddress(&addr, g_noalloc_scratch), "cudaGetSymbolAddress");
    if (st != FC2T2_OK) return st;
    unsigned char *base = static_cast<unsigned char *>(addr);

    // a plan on the stack whose device pointers all point into the scratch array
    fc2t2_plan_s pl;
    pl.desc = *desc;
    pl.desc.poly_coef = nullptr;
    pl.D = desc->dim;
    pl.n = desc->grid;
    pl.rho = desc->order;
    pl.P = ncoef(pl.D, pl.rho);
    pl.Pp = pad4(pl.P);
    int lg = 0;
    while ((1 << lg) < pl.n) ++lg;
    pl.nlev = lg - 1;
    int64_t off_cells = 0;
    for (int l = 0; l < pl.nlev; ++l) {
        Level &lv = pl.lev[l];
        lv.n = pl.n >> l;
        lv.G = 1;
        for (int d = 0; d < pl.D; ++d) lv.G *= lv.n;
        lv.off = off_cells;
        lv.h = (desc->hi - desc->lo) / lv.n;
        off_cells += lv.G;
    }
    pl.G_total = off_cells;
    pl.lo_f = (float)desc->lo;
    pl.hi_f = (float)desc->hi;
    pl.scale0_f = (float)((double)pl.n / (desc->hi - desc->lo));

    size_t off = 0;
    pl.d_M = carve<float>(base, off, (size_t)kNaMaxCellsAllLevels * kNaMaxPp);
    pl.d_L = carve<float>(base, off, (size_t)kNaMaxCellsAllLevels * kNaMaxPp);
    pl.d_dtab = carve<float>(base, off, (size_t)kNaMaxLevels * kNaOffsets * kNaMaxPp);
    pl.d_scan_tmp = carve<int>(base, off, 64);
    pl.d_flags = carve<int>(base, off, 4);
    pl.d_over = carve<int2>(base, off, kNaMaxCells);
    pl.d_over_ctr = carve<unsigned long long>(base, off, 2);
    SortWork *sorts[2] = {&pl.src, &pl.qry};
    for (SortWork *sw : sorts) {
        sw->cap = kNaMaxPoints;
        sw->count = carve<int>(base, off, kNaMaxCells);
        sw->start = carve<int>(base, off, kNaMaxCells + 1);
        sw->key = carve<int>(base, off, kNaMaxPoints);
        sw->rank = carve<int>(base, off, kNaMaxPoints);
        sw->perm = carve<int>(base, off, kNaMaxPoints);
        sw->rec = carve<float4>(base, off, kNaMaxPoints);
    }
    if (off > kScratchBytes) return set_error(FC2T2_ERR_UNSUPPORTED, "scratch layout exceeds the array");

    // operator table, built on the device into the scratch array
    const int nofs = pl.D == 3 ? 343 : 49;
    k_na_tables<<<pl.nlev * nofs, 64, 0, s>>>(pl.d_dtab, pl.D, pl.rho, pl.Pp, nofs, desc->sigma, pl.lev[0].h);
    if ((st = check_cuda(cudaGetLastError(), "operator tables")) != FC2T2_OK) return st;
    if ((st = check_cuda(cudaMemsetAsync(pl.d_flags, 0, 4 * sizeof(int), s), "clear flags")) != FC2T2_OK) return st;
    if ((st = check_cuda(cudaMemsetAsync(pl.d_over_ctr, 0, 2 * sizeof(unsigned long long), s), "clear counters")) != FC2T2_OK)
        return st;
    if (N == 0) return check_cuda(cudaMemsetAsync(y, 0, sizeof(float) * M, s), "zero y");

    // the same kernels as fc2t2_forward, on scratch-array pointers
    if ((st = check_cuda(launch_bin_count(&pl, s, p, N, pl.src), "bin")) != FC2T2_OK) return st;
    if ((st = check_cuda(launch_scan(&pl, s, pl.src.count, pl.src.start, pl.lev[0].G, pl.d_scan_tmp), "scan")) != FC2T2_OK) return st;
    if ((st = check_cuda(launch_scatter(&pl, s, p, w, N, pl.src), "scatter")) != FC2T2_OK) return st;
    if ((st = check_cuda(launch_p2m(&pl, s, pl.src, pl.d_M), "p2m")) != FC2T2_OK) return st;
    for (int l = 0; l + 1 < pl.nlev; ++l)
        if ((st = check_cuda(launch_m2m(&pl, s, l), "m2m")) != FC2T2_OK) return st;
    for (int l = pl.nlev - 1; l >= 0; --l) {
        if ((st = check_cuda(launch_m2l(&pl, s, l), "m2l")) != FC2T2_OK) return st;
        if (l + 1 < pl.nlev && (st = check_cuda(launch_l2l(&pl, s, l), "l2l")) != FC2T2_OK) return st;
    }
    if ((st = check_cuda(launch_bin_count(&pl, s, q, M, pl.qry), "bin")) != FC2T2_OK) return st;
    if ((st = check_cuda(launch_scan(&pl, s, pl.qry.count, pl.qry.start, pl.lev[0].G, pl.d_scan_tmp), "scan")) != FC2T2_OK) return st;
    if ((st = check_cuda(launch_scatter(&pl, s, q, nullptr, M, pl.qry), "scatter")) != FC2T2_OK) return st;
    return check_cuda(launch_l2p(&pl, s, pl.qry, M, y, nullptr), "l2p");
}
