// Moments-matching reduction of the support of a discrete measure on paths
// (Sec. 5.3): given the signature-kernel Gram K of the support's N paths and
// the weights alpha, proximal gradient descent on
//   L(beta) + lam |beta|_1,  L(beta) = (alpha - beta)^T K (alpha - beta),
//   beta <- A_{gamma lam}(beta - gamma grad L(beta)),  grad L = -2 K (alpha - beta),
// A_tau the soft-thresholding operator (the proximal map of tau |.|_1).
//
// One thread block runs every iteration in one launch: the problem is small
// (the paper's example has N = 30) and each iteration depends on the last, so
// the work is latency-bound and a single block, synchronised by barriers
// only, keeps it free of launches and of waits between blocks.  Per
// iteration each warp takes Gram rows (lanes stride along the row: coalesced
// reads of K) and reduces g_i = sum_j K_ij (alpha_j - beta_j) by shuffles;
// the loss is L(beta) + lam |beta|_1 = (alpha - beta).g + lam |beta|_1.
#include "sigk_internal.cuh"

namespace sigk {

namespace {

constexpr int SR_THREADS = 1024;

template <typename T>
__device__ __forceinline__ T soft_threshold(T v, T tau) {
    return v > tau ? v - tau : (v < -tau ? v + tau : (T)0);
}

// KS: K is staged in shared memory once (N^2 elements fit), else read from
// global memory (L2) every iteration.  alpha and two copies of beta live in
// shared memory: step t reads beta^t from one copy and writes beta^{t+1} into
// the other, so one barrier per step orders everything (each warp forms
// r_j = alpha_j - beta_j inside its own dot products).  Each warp adds its
// rows' share of the loss of step t into loss[t] (zeroed by the launcher) with
// one atomic add, which keeps the sum off the step's critical path; the
// order of those adds, and so the last bits of the loss, may vary.
template <typename T, bool KS>
__global__ void __launch_bounds__(SR_THREADS) support_kernel(const T *K, const T *alpha, T *beta, int N,
                                                             T gamma, T lam, int iters, T *loss) {
    extern __shared__ __align__(16) unsigned char sr_sm[];
    T *al = reinterpret_cast<T *>(sr_sm);
    T *be0 = al + N, *be1 = be0 + N;
    T *Ks = be1 + N;                                           // [N][N] when KS
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const T tau = gamma * lam;
    for (int i = tid; i < N; i += blockDim.x) { al[i] = alpha[i]; be0[i] = beta[i]; }
    if constexpr (KS)
        for (int64_t i = tid; i < (int64_t)N * N; i += blockDim.x) Ks[i] = K[i];
    const T *Kb = KS ? Ks : K;
    __syncthreads();
    for (int t = 0; t <= iters; ++t) {
        const T *bc = (t & 1) ? be1 : be0;
        T *bn = (t & 1) ? be0 : be1;
        T lw = 0;
        for (int row = warp; row < N; row += nw) {
            const T *Kr = Kb + (int64_t)row * N;
            T acc = 0;
            for (int j = lane; j < N; j += 32) acc += Kr[j] * (al[j] - bc[j]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
            if (lane == 0) {
                const T b = bc[row];
                lw += (al[row] - b) * acc + lam * fabs(b);
                bn[row] = t < iters ? soft_threshold(b + 2 * gamma * acc, tau) : b;
            }
        }
        if (loss && lane == 0 && warp < N) atomicAdd(&loss[t], lw);
        __syncthreads();
    }
    const T *bf = ((iters + 1) & 1) ? be1 : be0;   // step iters copied beta^iters there
    for (int i = tid; i < N; i += blockDim.x) beta[i] = bf[i];
}

}  // namespace

// shared memory: alpha and two copies of beta [N] each, then K [N][N] when
// it fits
constexpr int64_t SR_SMEM = 200 * 1024;

int64_t support_max_n(int dtype) {
    const int64_t es = dtype == SIGK_F64 ? 8 : 4;
    return SR_SMEM / (3 * es);
}

template <typename T>
static cudaError_t launch_support_t(const T *K, const T *alpha, T *beta, int64_t N, T gamma, T lam, int iters,
                                    T *loss, cudaStream_t st) {
    if (loss) {
        cudaError_t z = cudaMemsetAsync(loss, 0, (size_t)(iters + 1) * sizeof(T), st);
        if (z != cudaSuccess) return z;
    }
    const int64_t base = 3 * N * (int64_t)sizeof(T);
    const bool ks = base + N * N * (int64_t)sizeof(T) <= SR_SMEM;
    const int smem = (int)(ks ? base + N * N * (int64_t)sizeof(T) : base);
    auto k = ks ? support_kernel<T, true> : support_kernel<T, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // a warp per Gram row up to 32 warps: fewer warps at a barrier for small N
    const int threads = (int)(N < 32 ? 32 * N : SR_THREADS);
    k<<<1, threads, smem, st>>>(K, alpha, beta, (int)N, gamma, lam, iters, loss);
    return cudaGetLastError();
}

cudaError_t launch_support(const void *K, const void *alpha, void *beta, int64_t N, double gamma,
                           double lam, int iters, int dtype, void *loss, cudaStream_t st) {
    if (dtype == SIGK_F64)
        return launch_support_t<double>((const double *)K, (const double *)alpha, (double *)beta, N, gamma, lam,
                                        iters, (double *)loss, st);
    return launch_support_t<float>((const float *)K, (const float *)alpha, (float *)beta, N, (float)gamma,
                                   (float)lam, iters, (float *)loss, st);
}

}  // namespace sigk
