// The unbiased MMD^2 estimator between two batches of paths (Sec. 3.1.1
// names it; read as the U-statistic with the diagonal terms left out):
//   MMD^2 = sum_{i!=j} Kxx_ij / (m(m-1)) + sum_{i!=j} Kyy_ij / (n(n-1))
//           - 2 sum_{i,j} Kxy_ij / (mn),
// summed in double by one thread block; and its gradient with respect to the
// three Gram matrices (constants times the incoming scalar gradient).
#include "sigk_internal.cuh"

namespace sigk {

namespace {

constexpr int MMD_THREADS = 1024;

template <typename T>
__global__ void __launch_bounds__(MMD_THREADS) mmd2_kernel(const T *Kxx, const T *Kyy, const T *Kxy,
                                                            int64_t m, int64_t n, T *out) {
    __shared__ double red[3][MMD_THREADS / 32];
    double sxx = 0, syy = 0, sxy = 0;
    for (int64_t i = threadIdx.x; i < m * m; i += blockDim.x)
        if (i / m != i % m) sxx += (double)Kxx[i];
    for (int64_t i = threadIdx.x; i < n * n; i += blockDim.x)
        if (i / n != i % n) syy += (double)Kyy[i];
    for (int64_t i = threadIdx.x; i < m * n; i += blockDim.x) sxy += (double)Kxy[i];
    for (int o = 16; o > 0; o >>= 1) {
        sxx += __shfl_down_sync(FULL, sxx, o);
        syy += __shfl_down_sync(FULL, syy, o);
        sxy += __shfl_down_sync(FULL, sxy, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = sxx; red[1][w] = syy; red[2][w] = sxy; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += red[0][i]; b += red[1][i]; c += red[2][i]; }
        const double md = (double)m, nd = (double)n;
        out[0] = (T)(a / (md * (md - 1)) + b / (nd * (nd - 1)) - 2.0 * c / (md * nd));
    }
}

template <typename T>
__global__ void mmd2_backward_kernel(const T *grad, int64_t m, int64_t n, T *gKxx, T *gKyy, T *gKxy) {
    const double g = (double)grad[0];
    const T axx = (T)(g / ((double)m * (double)(m - 1)));
    const T ayy = (T)(g / ((double)n * (double)(n - 1)));
    const T axy = (T)(-2.0 * g / ((double)m * (double)n));
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gKxx)
        for (int64_t i = t0; i < m * m; i += stride) gKxx[i] = (i / m == i % m) ? (T)0 : axx;
    if (gKyy)
        for (int64_t i = t0; i < n * n; i += stride) gKyy[i] = (i / n == i % n) ? (T)0 : ayy;
    if (gKxy)
        for (int64_t i = t0; i < m * n; i += stride) gKxy[i] = axy;
}

// g_out = grad[0] g_in: the chain rule through the scalar loss for input
// gradients formed with a unit upstream derivative.
template <typename T>
__global__ void scale_grad_kernel(const T *grad, const T *g_in, T *g_out, int64_t n) {
    const T g = grad[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        g_out[i] = g * g_in[i];
}

}  // namespace

cudaError_t launch_scale_grad(const void *grad, const void *g_in, void *g_out, int64_t n, int dtype,
                              cudaStream_t st) {
    const int grid = (int)((n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048);
    if (dtype == SIGK_F64)
        scale_grad_kernel<double><<<grid, 256, 0, st>>>((const double *)grad, (const double *)g_in,
                                                         (double *)g_out, n);
    else
        scale_grad_kernel<float><<<grid, 256, 0, st>>>((const float *)grad, (const float *)g_in,
                                                        (float *)g_out, n);
    return cudaGetLastError();
}

cudaError_t launch_mmd2(const void *Kxx, const void *Kyy, const void *Kxy, int64_t m, int64_t n,
                        int dtype, void *out, cudaStream_t st) {
    if (dtype == SIGK_F64)
        mmd2_kernel<double><<<1, MMD_THREADS, 0, st>>>((const double *)Kxx, (const double *)Kyy,
                                                       (const double *)Kxy, m, n, (double *)out);
    else
        mmd2_kernel<float><<<1, MMD_THREADS, 0, st>>>((const float *)Kxx, (const float *)Kyy,
                                                      (const float *)Kxy, m, n, (float *)out);
    return cudaGetLastError();
}

cudaError_t launch_mmd2_backward(const void *grad, int64_t m, int64_t n, int dtype, void *gKxx,
                                 void *gKyy, void *gKxy, cudaStream_t st) {
    int64_t big = m > n ? m : n;
    int grid = (int)((big * big + 255) / 256 < 1024 ? (big * big + 255) / 256 : 1024);
    if (dtype == SIGK_F64)
        mmd2_backward_kernel<double><<<grid, 256, 0, st>>>((const double *)grad, m, n, (double *)gKxx,
                                                           (double *)gKyy, (double *)gKxy);
    else
        mmd2_backward_kernel<float><<<grid, 256, 0, st>>>((const float *)grad, m, n, (float *)gKxx,
                                                          (float *)gKyy, (float *)gKxy);
    return cudaGetLastError();
}

}  // namespace sigk
