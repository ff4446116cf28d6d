// Direct evaluation of the transform, y_m = sum_n psi(p_n - q_m) w_n (Sec. 3, Eq. 1), by brute
// force in O(N M): the exact sum the series approximates.  Used to measure the truncation error of
// a plan on a sample of queries (the autotuner) -- not part of the transform's hot path.
//
// One thread per query; the sources stream through shared memory in tiles of 256; the sum is
// compensated (Kahan) in FP32, so its rounding error does not grow with N.
#include "fc2t2_internal.cuh"

namespace fc2t2 {

constexpr int kDirectThreads = 256;

template <int D>
__global__ void __launch_bounds__(kDirectThreads) k_direct(const float *__restrict__ p, const float *__restrict__ w,
                                                           int64_t N, const float *__restrict__ q, int64_t M,
                                                           float inv_2s2, float *__restrict__ y) {
    __shared__ float4 tile[kDirectThreads];
    const int64_t m = (int64_t)blockIdx.x * kDirectThreads + threadIdx.x;
    float qx[3] = {0.f, 0.f, 0.f};
    if (m < M)
#pragma unroll
        for (int d = 0; d < D; ++d) qx[d] = q[m * D + d];
    float sum = 0.0f, comp = 0.0f;
    for (int64_t n0 = 0; n0 < N; n0 += kDirectThreads) {
        const int64_t n = n0 + threadIdx.x;
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n < N) t = make_float4(p[n * D], p[n * D + 1], D == 3 ? p[n * D + 2] : 0.f, w[n]);
        tile[threadIdx.x] = t;
        __syncthreads();
        const int cnt = (N - n0) < kDirectThreads ? (int)(N - n0) : kDirectThreads;
        for (int j = 0; j < cnt; ++j) {
            const float4 s = tile[j];
            const float d0 = s.x - qx[0], d1 = s.y - qx[1], d2 = D == 3 ? s.z - qx[2] : 0.0f;
            const float term = s.w * expf(-(d0 * d0 + d1 * d1 + d2 * d2) * inv_2s2);
            const float yk = term - comp;
            const float tk = sum + yk;
            comp = (tk - sum) - yk;
            sum = tk;
        }
        __syncthreads();
    }
    if (m < M) y[m] = sum;
}

}  // namespace fc2t2

using namespace fc2t2;

extern "C" fc2t2_status fc2t2_direct(const fc2t2_plan_desc *desc, void *stream, const float *p, const float *w,
                                     int64_t N, const float *q, int64_t M, float *y) {
    if (!desc) return set_error(FC2T2_ERR_INVALID_ARG, "desc is NULL");
    if (desc->dim != 2 && desc->dim != 3) return set_error(FC2T2_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (desc->kernel != FC2T2_KERNEL_GAUSSIAN)
        return set_error(FC2T2_ERR_UNSUPPORTED, "the direct sum supports the Gaussian kernel");
    if (!(desc->sigma > 0.0)) return set_error(FC2T2_ERR_INVALID_ARG, "sigma must be positive");
    if (N < 0 || M < 0) return set_error(FC2T2_ERR_INVALID_ARG, "negative size");
    if (desc->channels < 1 || desc->channels > 4096)
        return set_error(FC2T2_ERR_INVALID_ARG, "channels must be in [1, 4096]");
    if ((N > 0 && (!p || !w)) || (M > 0 && (!q || !y))) return set_error(FC2T2_ERR_INVALID_ARG, "NULL array");
    if (M == 0) return FC2T2_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float inv_2s2 = (float)(1.0 / (2.0 * desc->sigma * desc->sigma));
    const unsigned blocks = (unsigned)((M + kDirectThreads - 1) / kDirectThreads);
    for (int c = 0; c < desc->channels; ++c) {   // w [C][N] -> y [C][M]
        const float *wc = w ? w + (int64_t)c * N : nullptr;
        float *yc = y + (int64_t)c * M;
        if (desc->dim == 2) k_direct<2><<<blocks, kDirectThreads, 0, s>>>(p, wc, N, q, M, inv_2s2, yc);
        else k_direct<3><<<blocks, kDirectThreads, 0, s>>>(p, wc, N, q, M, inv_2s2, yc);
        const fc2t2_status st = check_cuda(cudaGetLastError(), "direct sum");
        if (st != FC2T2_OK) return st;
    }
    return FC2T2_OK;
}
