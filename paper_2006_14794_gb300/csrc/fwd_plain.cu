// Forward sweep, "plain" form: one thread block per pair sweeps the grid's
// anti-diagonals (Sec. 3.1.1: the cells of an anti-diagonal do not depend on
// one another), keeping the two or three live diagonals in shared memory and
// forming each cell's coefficient from the paths in global memory.
//
// In double precision it runs the explicit scheme of Sec. 3.1 as printed:
//   K(a,b) = K(a,b-1) + K(a-1,b) - K(a-1,b-1) + c (K(a,b-1) + K(a-1,b)),
// c = 1/2 4^-lambda <dx_p, dy_q>, p = (a-1) >> lambda, q = (b-1) >> lambda.
// In single precision it runs the difference form (Q = K(a,b) - K(a,b-1)),
// like the chained kernel.  This kernel is the comparison baseline for the
// chained FP32 kernel and the general path for shapes that kernel has no
// instance for (uneven lengths, long pairs, high dyadic orders, wide d).
#include "sigk_internal.cuh"

namespace sigk {

namespace {

constexpr int PLAIN_THREADS = 512;

// The coarse cell's coefficient: <dx_p, dy_q>, or with the RBF lift (Sec. 2.2)
// the second difference of kappa over the cell's corners (rbf_s = 1/(2 sigma^2)).
template <typename T>
__device__ __forceinline__ T coef(const T *x, const T *y, int64_t d, int64_t p, int64_t q,
                                  T scale, int kernel, T rbf_s) {
    const T *x0 = x + p * d, *x1 = x0 + d;
    const T *y0 = y + q * d, *y1 = y0 + d;
    if (kernel == SIGK_KERNEL_RBF) {
        T uu = 0, ux = 0, uy = 0, xy = 0, nx = 0, ny = 0;
        for (int64_t c = 0; c < d; ++c) {
            const T u = x0[c] - y0[c], dx = x1[c] - x0[c], dy = y1[c] - y0[c];
            uu += u * u; ux += u * dx; uy += u * dy; xy += dx * dy; nx += dx * dx; ny += dy * dy;
        }
        return rbf_second_difference(uu, ux, uy, xy, nx, ny, rbf_s) * scale;
    }
    T g = 0;
    for (int64_t c = 0; c < d; ++c) g += (x1[c] - x0[c]) * (y1[c] - y0[c]);
    return g * scale;
}

// Q_FORM = false: the printed scheme (three diagonals of K).
// Q_FORM = true:  the difference form (K and Q on two diagonals each).
// surf (optional, pairs of uniform lengths only): the solution at the
// sample-grid nodes, node (i, j) of pair k at surf[k La Lb + i Lb + j] (i over
// the A path); the refined node (a, b) is one when both are multiples of 2^lambda.
template <typename T, bool Q_FORM>
__global__ void __launch_bounds__(PLAIN_THREADS) plain_kernel(PairSrc src, int64_t n_pairs,
                                                               int lam, int64_t wcap, T *out, T *surf) {
    extern __shared__ unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    const T scale = (T)0.5 / (T)(1LL << (2 * lam));
    const T rbf_s = (T)(0.5 / (src.sigma * src.sigma));
    for (int64_t k = blockIdx.x; k < n_pairs; k += gridDim.x) {
        const PairRef pr = pair_ref(src, k);
        if (pr.la < 2 || pr.lb < 2) {
            if (threadIdx.x == 0) {
                out[pr.out0] = (T)1;
                if (pr.out1 >= 0) out[pr.out1] = (T)1;
            }
            continue;
        }
        // rows index the shorter path (k(x,y) = k(y,x), Sec. 2 symmetry of <.,.>)
        const T *x = (const T *)src.A + pr.a_row0 * src.d;
        const T *y = (const T *)src.B + pr.b_row0 * src.d;
        int64_t la = pr.la, lb = pr.lb;
        const bool swapped = la > lb;
        if (swapped) {
            const T *t = x; x = y; y = t;
            int64_t tl = la; la = lb; lb = tl;
        }
        // surface strides of the sweep's rows and columns (rows index the A path unless swapped)
        T *sf = surf ? surf + pr.out0 * pr.la * pr.lb : nullptr;
        const int64_t sr = swapped ? 1 : pr.lb, sc = swapped ? pr.lb : 1;
        const int64_t smask = (1LL << lam) - 1;
        const int64_t Ni = (la - 1) << lam, Nj = (lb - 1) << lam;
        const int64_t W = Ni + 1;
        if (W > wcap) {
            // the caller's length bound was too small for this pair: no sweep,
            // the result is NaN rather than a write past the diagonals
            if (threadIdx.x == 0) {
                out[pr.out0] = (T)NAN;
                if (pr.out1 >= 0) out[pr.out1] = (T)NAN;
            }
            continue;
        }
        T *D0 = sm, *D1 = sm + W, *D2 = sm + 2 * W, *D3 = sm + 3 * W;
        // D0/D1: K on diagonals n-1 / n-2 (plain) or K, Q on n-1 (Q form);
        // diagonal 1: K(0,1) = K(1,0) = 1, Q = 0.
        for (int64_t a = threadIdx.x; a < W; a += blockDim.x) {
            D0[a] = (T)1;
            D1[a] = Q_FORM ? (T)0 : (T)1;
            D2[a] = (T)1;
            if (Q_FORM) D3[a] = (T)0;
        }
        __syncthreads();
        for (int64_t n = 2; n <= Ni + Nj; ++n) {
            const int64_t alo = n - Nj > 0 ? n - Nj : 0;
            const int64_t ahi = n < Ni ? n : Ni;
            for (int64_t a = alo + threadIdx.x; a <= ahi; a += blockDim.x) {
                const int64_t b = n - a;
                if (!Q_FORM) {
                    // D0 = diag n-1, D1 = diag n-2, D2 = new diag n
                    T v = (T)1;
                    if (a > 0 && b > 0) {
                        const T c = scheme_coef(coef(x, y, src.d, (a - 1) >> lam, (b - 1) >> lam, scale,
                                                     src.kernel, rbf_s),
                                                src.scheme);
                        const T kl = D0[a], ku = D0[a - 1], kd = D1[a - 1];
                        v = kl + ku - kd + c * (kl + ku);
                        if (sf && (a & smask) == 0 && (b & smask) == 0) sf[(a >> lam) * sr + (b >> lam) * sc] = v;
                    }
                    D2[a] = v;
                } else {
                    // D0 = K(n-1), D1 = Q(n-1), D2 = K(n), D3 = Q(n)
                    T kv = (T)1, qv = (T)0;
                    if (a > 0 && b > 0) {
                        const T c = scheme_coef(coef(x, y, src.d, (a - 1) >> lam, (b - 1) >> lam, scale,
                                                     src.kernel, rbf_s),
                                                src.scheme);
                        const T kl = D0[a], ku = D0[a - 1], qu = D1[a - 1];
                        qv = qu + c * (kl + ku);
                        kv = kl + qv;
                        if (sf && (a & smask) == 0 && (b & smask) == 0) sf[(a >> lam) * sr + (b >> lam) * sc] = kv;
                    }
                    D2[a] = kv;
                    D3[a] = qv;
                }
            }
            __syncthreads();
            if (!Q_FORM) {
                T *t = D1; D1 = D0; D0 = D2; D2 = t;
            } else {
                T *t0 = D0, *t1 = D1;
                D0 = D2; D1 = D3; D2 = t0; D3 = t1;
            }
        }
        if (threadIdx.x == 0) {
            out[pr.out0] = D0[Ni];
            if (pr.out1 >= 0) out[pr.out1] = D0[Ni];
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void fill_one_kernel(T *out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (T)1;
}

template <typename T, bool QF>
cudaError_t launch_plain_t(const PairSrc &src, int64_t n_pairs, int lam, T *out, cudaStream_t st,
                           int64_t min_len, T *surf) {
    const int64_t W = ((min_len > 1 ? min_len - 1 : 0) << lam) + 1;
    const int64_t smem = (QF ? 4 : 3) * W * (int64_t)sizeof(T);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    auto kern = plain_kernel<T, QF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PLAIN_THREADS, (int)smem);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sms * per_sm;
    if (grid > n_pairs) grid = n_pairs;
    kern<<<(int)grid, PLAIN_THREADS, (int)smem, st>>>(src, n_pairs, lam, W, out, surf);
    return cudaGetLastError();
}

}  // namespace

// The shared-memory diagonals are sized by the shorter path of a pair; for
// uneven lengths the caller passes in src.La the longest length any pair's
// shorter path can have.
cudaError_t launch_plain(const PairSrc &src, int64_t n_pairs, int lam, int dtype, void *out,
                         cudaStream_t st, void *surf) {
    if (n_pairs <= 0) return cudaSuccess;
    const int64_t min_len = src.mode == PM_VARLEN ? src.La : (src.La < src.Lb ? src.La : src.Lb);
    if (dtype == SIGK_F64)
        return launch_plain_t<double, false>(src, n_pairs, lam, (double *)out, st, min_len, (double *)surf);
    return launch_plain_t<float, true>(src, n_pairs, lam, (float *)out, st, min_len, (float *)surf);
}

cudaError_t launch_fill_one(void *out, int64_t n, int dtype, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    if (dtype == SIGK_F64)
        fill_one_kernel<double><<<grid, 256, 0, st>>>((double *)out, n);
    else
        fill_one_kernel<float><<<grid, 256, 0, st>>>((float *)out, n);
    return cudaGetLastError();
}

// Row 0 and column 0 of B surfaces [L][M]: the boundary value 1 (the sweeps
// write every other node).
template <typename T>
__global__ void surface_border_kernel(T *surf, int64_t B, int64_t L, int64_t M, bool col0) {
    const int64_t per = col0 ? L + M - 1 : M;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B * per;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / per, j = i - b * per;
        T *s = surf + b * L * M;
        if (j < M) s[j] = (T)1;                 // row 0
        else s[(j - M + 1) * M] = (T)1;         // column 0, rows 1 .. L-1
    }
}

cudaError_t launch_surface_border(void *surf, int64_t B, int64_t L, int64_t M, int dtype, cudaStream_t st,
                                  bool col0) {
    const int64_t n = B * (col0 ? L + M - 1 : M);
    if (n <= 0) return cudaSuccess;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    if (dtype == SIGK_F64)
        surface_border_kernel<double><<<grid, 256, 0, st>>>((double *)surf, B, L, M, col0);
    else
        surface_border_kernel<float><<<grid, 256, 0, st>>>((float *)surf, B, L, M, col0);
    return cudaGetLastError();
}

}  // namespace sigk
