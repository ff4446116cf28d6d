// Binning of points into finest-level cells and a counting sort by cell
// (Sec. 3: P2M sorts source points into their boxes at the highest grid granularity;
// the paper's find_box computes int((p + 1) N / 2) per dimension, Sec. 3.3).
//
// Three passes, no atomics on coefficient data:
//   count   : cell of every point (FP32 rule), count[cell]++ (the returned old value is the
//             point's rank inside its cell)
//   scan    : exclusive prefix sum of the counts -> start[cell]        (reduce-then-scan)
//   scatter : sorted position = start[cell] + rank; writes the permutation and one 16-byte
//             record per point (coordinates and weight), so P2M and L2P read contiguous,
//             cell-ordered data; a consumer that needs a point's cell recomputes it from the
//             record with the same FP32 rule.
// The order of points inside one cell depends on the order in which the atomics resolved;
// every consumer only sums or evaluates per point, so results differ at most by rounding.
#include "fc2t2_internal.cuh"

namespace fc2t2 {

template <int D>
__global__ void __launch_bounds__(256) k_bin_count(const float *__restrict__ x, int64_t n, int grid,
                                                   float lo, float scale, int *__restrict__ key,
                                                   int *__restrict__ rank, int *__restrict__ count,
                                                   int *__restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < n;
    int lin = -1;                          // lanes past the end join no group of a real cell
    bool out = false;
    if (live) {
        lin = 0;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            float xd = x[i * D + d];
            out |= outside(xd, lo, scale, grid);
            lin = lin * grid + cell_of(xd, lo, scale, grid);
        }
    }
    if (out) atomicOr(flags, 1);
    // lanes of the warp that fall in the same cell take one atomic together: the group's lowest
    // lane adds the group's size, and each lane's rank is its position within the group (points
    // that arrive in runs along a cell -- samples along a ray -- no longer serialise on one counter)
    const unsigned peers = __match_any_sync(0xffffffffu, lin);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    const int before = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (live && lane == leader) base = atomicAdd(count + lin, __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!live) return;
    key[i] = lin;
    rank[i] = base + before;
}

cudaError_t launch_bin_count(const fc2t2_plan_s *pl, cudaStream_t s, const float *x, int64_t n,
                             SortWork &w) {
    cudaError_t e = cudaMemsetAsync(w.count, 0, sizeof(int) * pl->lev[0].G, s);
    if (e != cudaSuccess || n == 0) return e;
    unsigned blocks = (unsigned)((n + 255) / 256);
    pl->launches[FC2T2_STAGE_SORT] += 1;
    if (pl->D == 2)
        k_bin_count<2><<<blocks, 256, 0, s>>>(x, n, pl->n, pl->lo_f, pl->scale0_f, w.key, w.rank,
                                              w.count, pl->d_flags);
    else
        k_bin_count<3><<<blocks, 256, 0, s>>>(x, n, pl->n, pl->lo_f, pl->scale0_f, w.key, w.rank,
                                              w.count, pl->d_flags);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- prefix scan
// Block of 1024 threads scans 4096 ints (4 per thread).

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int *smem_warp, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) smem_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int ws = smem_warp[lane];
        int wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        smem_warp[lane] = wi - ws;   // exclusive prefix of warp sums
        if (lane == 31) smem_warp[32] = wi;
    }
    __syncthreads();
    total = smem_warp[32];
    return smem_warp[warp] + incl - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int *__restrict__ in, int64_t n,
                                                              int *__restrict__ sums) {
    __shared__ int sw[33];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) if (base + j < n) v += in[base + j];
    int tot;
    block_exclusive_scan(v, sw, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// exclusive scan of one tile per block, plus the tile's offset (offsets may be NULL);
// writes out[n] = grand total when the last tile is processed and `write_total` is set.
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const int *__restrict__ in, int64_t n,
                                                            const int *__restrict__ offsets,
                                                            int *__restrict__ out, int write_total) {
    __shared__ int sw[33];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = (base + j < n) ? in[base + j] : 0;
        sum += v[j];
    }
    int tot;
    int ex = block_exclusive_scan(sum, sw, tot);
    int off = offsets ? offsets[blockIdx.x] : 0;
    int run = off + ex;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = off + tot;
}

// Exclusive scan of in[0..n) into out[0..n], out[n] = total.  Recursive reduce-then-scan;
// the block sums of every level live in `tmp` (one workspace per sort).
static cudaError_t scan_rec(cudaStream_t s, const int *in, int *out, int64_t n, int *tmp,
                            bool write_total, int64_t &launches) {
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles <= 1) {
        k_scan_tile<<<1, kScanThreads, 0, s>>>(in, n, nullptr, out, write_total ? 1 : 0);
        launches += 1;
        return cudaGetLastError();
    }
    int *sums = tmp;
    int *sums_scanned = tmp + tiles;
    k_scan_reduce<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_rec(s, sums, sums_scanned, tiles, tmp + 2 * tiles + 1, false, launches);
    if (e != cudaSuccess) return e;
    k_scan_tile<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums_scanned, out, write_total ? 1 : 0);
    launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_scan(const fc2t2_plan_s *pl, cudaStream_t s, const int *in, int *out, int64_t n, int *tmp) {
    return scan_rec(s, in, out, n, tmp, true, pl->launches[FC2T2_STAGE_SORT]);
}

// ---------------------------------------------------------------- scatter

template <int D>
__global__ void __launch_bounds__(256) k_scatter(int64_t n, const int *__restrict__ key,
                                                 const int *__restrict__ rank,
                                                 const int *__restrict__ start,
                                                 const float *__restrict__ x,
                                                 const float *__restrict__ wt, int *__restrict__ perm,
                                                 float4 *__restrict__ rec) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t pos = (int64_t)start[key[i]] + rank[i];
    perm[pos] = (int)i;
    rec[pos] = make_float4(x[i * D], x[i * D + 1], D == 3 ? x[i * D + 2] : 0.0f, wt ? wt[i] : 0.0f);
}

cudaError_t launch_scatter(const fc2t2_plan_s *pl, cudaStream_t s, const float *x, const float *wt,
                           int64_t n, SortWork &w) {
    if (n == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((n + 255) / 256);
    pl->launches[FC2T2_STAGE_SORT] += 1;
    if (pl->D == 2)
        k_scatter<2><<<blocks, 256, 0, s>>>(n, w.key, w.rank, w.start, x, wt, w.perm, w.rec);
    else
        k_scatter<3><<<blocks, 256, 0, s>>>(n, w.key, w.rank, w.start, x, wt, w.perm, w.rec);
    return cudaGetLastError();
}

// New weights for an existing sort: rec[j].w = wt[perm[j]] (the points and their order kept).
__global__ void __launch_bounds__(256) k_reweight(int64_t n, const int *__restrict__ perm,
                                                  const float *__restrict__ wt, float4 *__restrict__ rec) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) rec[j].w = wt[perm[j]];
}

cudaError_t launch_reweight(const fc2t2_plan_s *pl, cudaStream_t s, const float *wt, int64_t n, SortWork &w) {
    if (n == 0) return cudaSuccess;
    pl->launches[FC2T2_STAGE_SORT] += 1;
    k_reweight<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, w.perm, wt, w.rec);
    w.held_w = wt;
    return cudaGetLastError();
}

}  // namespace fc2t2
