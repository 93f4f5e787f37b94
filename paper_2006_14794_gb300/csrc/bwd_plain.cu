// Reverse-mode derivative of the scheme (the paper states no gradient; this
// is the exact derivative of the discrete scheme of Sec. 3.1), one thread
// block per pair:
//
//  1. G(p,q) = <dx_p, dy_q> into the block's workspace slot;
//  2. the forward sweep by anti-diagonals (as in fwd_plain.cu), writing every
//     K(a,b) of the (Ni+1) x (Nj+1) grid into the slot;
//  3. the adjoint A(a,b) = d k(Ni,Nj) / d K(a,b) by anti-diagonals from the
//     terminal corner:
//       A(a,b) = h(a,b+1) A(a,b+1) + h(a+1,b) A(a+1,b) - A(a+1,b+1),
//     h = 1 + c, out-of-grid terms zero, A(Ni,Nj) = 1; in FP32 in the
//     difference form (P(a,b) = A(a,b) - A(a,b+1)):
//       P(a,b) = P(a+1,b) + c(a,b+1) A(a,b+1) + c(a+1,b) A(a+1,b),
//       A(a,b) = A(a,b+1) + P(a,b),
//     seeded by a virtual P(Ni+1,Nj) = 1;
//     every cell adds A(a,b) (K(a,b-1) + K(a-1,b)) to Gbar of its coarse cell;
//  4. the chain rule: dk/d dx_p = 1/2 4^-lambda sum_q Gbar(p,q) dy_q (and the
//     mirror for y), scaled by the incoming gradient, then to the points:
//     dk/dx_i = dk/d dx_{i-1} - dk/d dx_i, added atomically into dX / dY
//     (a path appears in many pairs of a Gram).
#include <string.h>

#include "sigk_internal.cuh"

namespace sigk {

namespace {

constexpr int BWD_THREADS = 512;

struct BwdArgs {
    PairSrc src;
    const void *gout;       // [n] incoming gradient, indexed like the forward output
    void *dA, *dB;          // gradients of the A (row) and B (column) paths, or null
    unsigned char *ws;      // workspace: n_slots slots of slot_bytes
    int64_t slot_bytes;
    int64_t n_pairs;
    int lam;
};

template <typename T>
__device__ __forceinline__ T inc(const T *p, int64_t i, int64_t d, int64_t c) {
    return p[(i + 1) * d + c] - p[i * d + c];
}

template <typename T>
__device__ __forceinline__ void atomic_add(T *p, T v) { atomicAdd(p, v); }

template <typename T, bool QF>
__global__ void __launch_bounds__(BWD_THREADS) bwd_plain_kernel(BwdArgs a) {
    extern __shared__ unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    const T scale = (T)0.5 / (T)(1LL << (2 * a.lam));
    const int lam = a.lam;
    const bool rbf = a.src.kernel == SIGK_KERNEL_RBF;
    const T rbf_s = (T)(0.5 / (a.src.sigma * a.src.sigma));
    const int64_t d = a.src.d;
    unsigned char *slot = a.ws + (int64_t)blockIdx.x * a.slot_bytes;
    for (int64_t k = blockIdx.x; k < a.n_pairs; k += gridDim.x) {
        const PairRef pr = pair_ref(a.src, k);
        const T gk = ((const T *)a.gout)[pr.out0];
        if (pr.la < 2 || pr.lb < 2) continue;   // k = 1 identically: zero gradient
        // rows index the shorter path; its gradient goes to the matching output
        const T *x = (const T *)a.src.A + pr.a_row0 * d;
        const T *y = (const T *)a.src.B + pr.b_row0 * d;
        T *dx = a.dA ? (T *)a.dA + pr.a_row0 * d : nullptr;
        T *dy = a.dB ? (T *)a.dB + pr.b_row0 * d : nullptr;
        int64_t la = pr.la, lb = pr.lb;
        if (la > lb) {
            const T *t = x; x = y; y = t;
            T *td = dx; dx = dy; dy = td;
            int64_t tl = la; la = lb; lb = tl;
        }
        const int64_t nx = la - 1, ny = lb - 1;
        const int64_t Ni = nx << lam, Nj = ny << lam, W = Nj + 1;
        T *Gm = reinterpret_cast<T *>(slot);
        T *Gb = Gm + nx * ny;
        T *Kg = Gb + nx * ny;

        // 1. increment Gram (or the RBF lift's second differences), Gbar = 0
        for (int64_t idx = threadIdx.x; idx < nx * ny; idx += blockDim.x) {
            const int64_t p = idx / ny, q = idx - (idx / ny) * ny;
            T g = 0;
            if (rbf) {
                T uu = 0, ux = 0, uy = 0, xy = 0, snx = 0, sny = 0;
                for (int64_t c = 0; c < d; ++c) {
                    const T u = x[p * d + c] - y[q * d + c], dxv = inc(x, p, d, c), dyv = inc(y, q, d, c);
                    uu += u * u; ux += u * dxv; uy += u * dyv; xy += dxv * dyv;
                    snx += dxv * dxv; sny += dyv * dyv;
                }
                g = rbf_second_difference(uu, ux, uy, xy, snx, sny, rbf_s);
            } else {
                for (int64_t c = 0; c < d; ++c) g += inc(x, p, d, c) * inc(y, q, d, c);
            }
            Gm[idx] = scheme_coef(g * scale, a.src.scheme);
            Gb[idx] = 0;
        }
        __syncthreads();
#define COEF(aa, bb) Gm[(((aa) - 1) >> lam) * ny + (((bb) - 1) >> lam)]

        // 2. forward sweep, K grid into the slot
        {
            T *D0 = sm, *D1 = sm + (Ni + 1), *D2 = sm + 2 * (Ni + 1), *D3 = sm + 3 * (Ni + 1);
            for (int64_t i = threadIdx.x; i <= Ni; i += blockDim.x) {
                D0[i] = 1; D1[i] = QF ? (T)0 : (T)1; D2[i] = 1;
                if (QF) D3[i] = 0;
                Kg[i * W] = 1;   // column 0
            }
            for (int64_t b = threadIdx.x; b <= Nj; b += blockDim.x) Kg[b] = 1;   // row 0
            __syncthreads();
            for (int64_t n = 2; n <= Ni + Nj; ++n) {
                const int64_t alo = n - Nj > 0 ? n - Nj : 0;
                const int64_t ahi = n < Ni ? n : Ni;
                for (int64_t aa = alo + threadIdx.x; aa <= ahi; aa += blockDim.x) {
                    const int64_t bb = n - aa;
                    if (!QF) {
                        T v = 1;
                        if (aa > 0 && bb > 0) {
                            const T c = COEF(aa, bb);
                            const T kl = D0[aa], ku = D0[aa - 1], kd = D1[aa - 1];
                            v = kl + ku - kd + c * (kl + ku);
                            Kg[aa * W + bb] = v;
                        }
                        D2[aa] = v;
                    } else {
                        T kv = 1, qv = 0;
                        if (aa > 0 && bb > 0) {
                            const T c = COEF(aa, bb);
                            const T kl = D0[aa], ku = D0[aa - 1], qu = D1[aa - 1];
                            qv = qu + c * (kl + ku);
                            kv = kl + qv;
                            Kg[aa * W + bb] = kv;
                        }
                        D2[aa] = kv;
                        D3[aa] = qv;
                    }
                }
                __syncthreads();
                if (!QF) {
                    T *t = D1; D1 = D0; D0 = D2; D2 = t;
                } else {
                    T *t0 = D0, *t1 = D1;
                    D0 = D2; D1 = D3; D2 = t0; D3 = t1;
                }
            }
        }

        // 3. adjoint sweep from the terminal corner; diagonals indexed by a in [0, Ni+1]
        {
            const int64_t V = Ni + 2;
            // QF: E0/E1 = A, P on diagonal n+1; E2/E3 = A, P on diagonal n.
            // plain: E0 = A on n+1, E1 = A on n+2, E2 = A on n.
            T *E0 = sm, *E1 = sm + V, *E2 = sm + 2 * V, *E3 = sm + 3 * V;
            for (int64_t i = threadIdx.x; i < V; i += blockDim.x) {
                E0[i] = 0; E1[i] = 0; E2[i] = 0;
                if (QF) E3[i] = 0;
            }
            __syncthreads();
            for (int64_t n = Ni + Nj; n >= 2; --n) {
                const int64_t alo = n - Nj > 1 ? n - Nj : 1;
                const int64_t ahi = n - 1 < Ni ? n - 1 : Ni;
                for (int64_t aa = alo + threadIdx.x; aa <= ahi; aa += blockDim.x) {
                    const int64_t bb = n - aa;
                    // neighbours on diagonal n+1: (aa, bb+1) at row aa, (aa+1, bb) at row aa+1
                    const T Ar = (bb + 1 <= Nj) ? E0[aa] : (T)0;
                    const T Ad = (aa + 1 <= Ni) ? E0[aa + 1] : (T)0;
                    const T cr = (bb + 1 <= Nj) ? COEF(aa, bb + 1) : (T)0;
                    const T cd = (aa + 1 <= Ni) ? COEF(aa + 1, bb) : (T)0;
                    T An;
                    if (QF) {
                        T Pd;
                        if (aa + 1 <= Ni) Pd = E1[aa + 1];
                        else Pd = (bb == Nj) ? (T)1 : (T)0;   // virtual seed row
                        const T Pn = Pd + cr * Ar + cd * Ad;
                        An = Ar + Pn;
                        E3[aa] = Pn;
                    } else {
                        if (aa == Ni && bb == Nj) {
                            An = 1;
                        } else {
                            const T Add = (aa + 1 <= Ni && bb + 1 <= Nj) ? E1[aa + 1] : (T)0;
                            An = (1 + cr) * Ar + (1 + cd) * Ad - Add;
                        }
                    }
                    E2[aa] = An;
                    const T s = Kg[aa * W + bb - 1] + Kg[(aa - 1) * W + bb];
                    atomic_add(&Gb[((aa - 1) >> lam) * ny + ((bb - 1) >> lam)], An * s);
                }
                __syncthreads();
                if (QF) {
                    T *t0 = E0, *t1 = E1;
                    E0 = E2; E1 = E3; E2 = t0; E3 = t1;
                } else {
                    T *t = E1; E1 = E0; E0 = E2; E2 = t;
                }
            }
        }
#undef COEF
        if (a.src.scheme != SIGK_SCHEME_EXPLICIT) {
            // the sweeps used c' = scheme_coef(c): Gbar holds dk/dc', turn it into
            // dk/dc (the adjoint's last diagonal ended with a barrier)
            for (int64_t idx = threadIdx.x; idx < nx * ny; idx += blockDim.x)
                Gb[idx] *= scheme_dcoef(Gm[idx], a.src.scheme);
            __syncthreads();
        }

        const T f = gk * scale;
        if (rbf) {
            // 4'. chain rule through the second difference of kappa: the point
            // pair (i, j) enters G(p, q) for p in {i-1, i}, q in {j-1, j} with
            // weight W(i,j) = Gb(i-1,j-1) - Gb(i,j-1) - Gb(i-1,j) + Gb(i,j)
            // (terms outside the grid 0), and d kappa(a,b)/da = kappa (b - a) /
            // sigma^2 = -d kappa/db.  Z(i,j) = f W(i,j) kappa(x_i, y_j) / sigma^2
            // goes where the K grid was (no longer needed); then
            // dk/dx_i = sum_j Z(i,j) (y_j - x_i), dk/dy_j = sum_i Z(i,j) (x_i - y_j).
            T *Z = Kg;
            const int64_t la1 = nx + 1, lb1 = ny + 1;
            for (int64_t idx = threadIdx.x; idx < la1 * lb1; idx += blockDim.x) {
                const int64_t i = idx / lb1, j = idx - (idx / lb1) * lb1;
                T w = 0;
                if (i >= 1 && j >= 1) w += Gb[(i - 1) * ny + j - 1];
                if (i < nx && j >= 1) w -= Gb[i * ny + j - 1];
                if (i >= 1 && j < ny) w -= Gb[(i - 1) * ny + j];
                if (i < nx && j < ny) w += Gb[i * ny + j];
                T dd = 0;
                for (int64_t c = 0; c < d; ++c) {
                    const T u = x[i * d + c] - y[j * d + c];
                    dd += u * u;
                }
                Z[idx] = f * w * exp(-rbf_s * dd) * (2 * rbf_s);
            }
            __syncthreads();
            if (dx) {
                for (int64_t idx = threadIdx.x; idx < la1 * d; idx += blockDim.x) {
                    const int64_t i = idx / d, c = idx - (idx / d) * d;
                    T sacc = 0;
                    for (int64_t j = 0; j < lb1; ++j) sacc += Z[i * lb1 + j] * (y[j * d + c] - x[i * d + c]);
                    atomic_add(&dx[i * d + c], sacc);
                }
            }
            if (dy) {
                for (int64_t idx = threadIdx.x; idx < lb1 * d; idx += blockDim.x) {
                    const int64_t j = idx / d, c = idx - (idx / d) * d;
                    T sacc = 0;
                    for (int64_t i = 0; i < la1; ++i) sacc += Z[i * lb1 + j] * (x[i * d + c] - y[j * d + c]);
                    atomic_add(&dy[j * d + c], sacc);
                }
            }
            __syncthreads();
            continue;
        }

        // 4. chain rule through G(p,q) = <dx_p, dy_q>, into the points
        if (dx) {
            for (int64_t idx = threadIdx.x; idx < nx * d; idx += blockDim.x) {
                const int64_t p = idx / d, c = idx - (idx / d) * d;
                T s = 0;
                for (int64_t q = 0; q < ny; ++q) s += Gb[p * ny + q] * inc(y, q, d, c);
                s *= f;
                atomic_add(&dx[(p + 1) * d + c], s);
                atomic_add(&dx[p * d + c], -s);
            }
        }
        if (dy) {
            for (int64_t idx = threadIdx.x; idx < ny * d; idx += blockDim.x) {
                const int64_t q = idx / d, c = idx - (idx / d) * d;
                T s = 0;
                for (int64_t p = 0; p < nx; ++p) s += Gb[p * ny + q] * inc(x, p, d, c);
                s *= f;
                atomic_add(&dy[(q + 1) * d + c], s);
                atomic_add(&dy[q * d + c], -s);
            }
        }
        __syncthreads();
    }
}

template <typename T, bool QF>
int grid_of(int64_t n_pairs, int64_t smem) {
    auto kern = bwd_plain_kernel<T, QF>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BWD_THREADS, (int)smem) !=
        cudaSuccess)
        return 0;
    if (per_sm < 1) return 0;
    int64_t g = (int64_t)sms * per_sm;
    if (g > n_pairs) g = n_pairs;
    return (int)g;
}

}  // namespace

// Sizes of the plain backward's workspace for uniform lengths La x Lb:
// one slot per thread block in flight.
bool bwd_plain_plan(int64_t n_pairs, int64_t La, int64_t Lb, int64_t d, int lam, int dtype,
                    int64_t &grid, int64_t &slot_bytes, int64_t &smem) {
    (void)d;
    const int64_t la = La < Lb ? La : Lb, lb = La < Lb ? Lb : La;
    const int64_t nx = la > 1 ? la - 1 : 0, ny = lb > 1 ? lb - 1 : 0;
    const int64_t Ni = nx << lam, Nj = ny << lam;
    const int64_t es = dtype == SIGK_F64 ? 8 : 4;
    slot_bytes = ((2 * nx * ny + (Ni + 1) * (Nj + 1)) * es + 255) / 256 * 256;
    smem = (dtype == SIGK_F64 ? 3 : 4) * (Ni + 2) * es;
    if (smem > 227 * 1024) return false;
    if (n_pairs < 1) { grid = 0; return true; }
    grid = dtype == SIGK_F64 ? grid_of<double, false>(n_pairs, smem)
                             : grid_of<float, true>(n_pairs, smem);
    return grid > 0;
}

cudaError_t launch_bwd_plain(const PairSrc &src, int64_t n_pairs, int lam, int dtype,
                             const void *gout, void *dA, void *dB, void *ws, int64_t grid,
                             int64_t slot_bytes, int64_t smem, cudaStream_t st) {
    BwdArgs a;
    a.src = src;
    a.gout = gout;
    a.dA = dA;
    a.dB = dB;
    a.ws = (unsigned char *)ws;
    a.slot_bytes = slot_bytes;
    a.n_pairs = n_pairs;
    a.lam = lam;
    if (dtype == SIGK_F64)
        bwd_plain_kernel<double, false><<<(int)grid, BWD_THREADS, (int)smem, st>>>(a);
    else
        bwd_plain_kernel<float, true><<<(int)grid, BWD_THREADS, (int)smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace sigk

// ---------------------------------------------------------------------------
// sigk_pairs_backward_noalloc: the pairs backward above, with its per-block
// scratch taken from a fixed array in device memory instead of a caller
// workspace.  For callers that cannot allocate device memory at call time:
// a process whose device memory is all handed to its own pool at start-up,
// or that runs under a fixed memory budget, where an extra allocation fails
// or stalls the device.  The array is part of the library image: every GPU
// that loads the library holds SIGK_NOALLOC_SCRATCH_BYTES of it until the
// process exits.  Every call shares it, so calls that overlap on the GPU
// (two streams, or two host threads) race and must be serialised by the
// caller.  Each call writes every scratch element it reads before reading it
// (the kernel clears its dk/dG accumulator itself), so no state carries over
// from one call to the next.
// ---------------------------------------------------------------------------
#include <cuda.h>   // CUcontext / CUresult types; the two driver calls are fetched at run time
#include <mutex>

#define SIGK_NOALLOC_SCRATCH_BYTES (32u << 20)
#define SIGK_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char sigk_noalloc_scratch[SIGK_NOALLOC_SCRATCH_BYTES];

namespace {

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

std::mutex g_noalloc_mu;
struct NoallocSlot {
    void *ptr;                  // the array's device address in that context
    unsigned long long ctx_id;  // the context it was looked up in (0: unknown)
};
NoallocSlot g_noalloc[SIGK_NOALLOC_MAX_DEVICES];
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_ctx_fns_tried = false;

// Process-unique id of the calling thread's current context, 0 when there is
// none yet or the driver cannot say.  A device reset ends the context, and the
// library image (with the array) is loaded again in the next one, possibly at
// another address: the id tells a cached address from a stale one.
unsigned long long current_ctx_id() {
    if (!g_ctx_fns_tried) {
        g_ctx_fns_tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_id = (CtxGetIdFn)f;
    }
    if (!g_ctx_current || !g_ctx_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&c) != CUDA_SUCCESS || !c) return 0;
    if (g_ctx_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array on the current device: the host-side
// name is only a stand-in for it.  Set-up, once per device and context: the
// first call on a device, and the first after that device's context was
// reset, look the address up with cudaGetSymbolAddress; later calls in the
// same context reuse it.
int noalloc_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SIGK_ECUDA;
    if (dev < 0 || dev >= SIGK_NOALLOC_MAX_DEVICES) return SIGK_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocSlot &sl = g_noalloc[dev];
    const unsigned long long id = current_ctx_id();
    if (sl.ptr && id != 0 && sl.ctx_id == id) {
        *out = sl.ptr;
        return SIGK_OK;
    }
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, sigk_noalloc_scratch) != cudaSuccess || !p) return SIGK_ECUDA;
    // the look-up makes the device's context current if it was not yet
    sl.ptr = p;
    sl.ctx_id = id != 0 ? id : current_ctx_id();
    *out = p;
    return SIGK_OK;
}

}  // namespace

extern "C" int sigk_pairs_backward_noalloc(const void *grad_out, const void *X, const void *Y,
                                           int64_t B, int64_t L, int64_t M, int64_t d,
                                           int dyadic_order, int dtype, void *dX, void *dY,
                                           void *stream) {
    using namespace sigk;
    if (B < 0 || L < 1 || M < 1 || d < 1) return SIGK_EINVAL;
    if (dtype != SIGK_F32 && dtype != SIGK_F64) return SIGK_EINVAL;
    if (dyadic_order < 0) return SIGK_EINVAL;
    if (dyadic_order > 8) return SIGK_EUNSUPPORTED;
    if (B == 0) return SIGK_OK;
    if (!grad_out || !X || !Y) return SIGK_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t es = dtype == SIGK_F64 ? 8 : 4;
    int64_t grid = 0, slot = 0, smem = 0;
    if (!bwd_plain_plan(B, L, M, d, dyadic_order, dtype, grid, slot, smem)) return SIGK_EUNSUPPORTED;
    if (L >= 2 && M >= 2 && slot > (int64_t)SIGK_NOALLOC_SCRATCH_BYTES)
        return SIGK_EUNSUPPORTED;   // one pair's scratch does not fit the fixed array
    void *scratch = nullptr;
    int s = noalloc_scratch(&scratch);
    if (s != SIGK_OK) return s;
    if (dX && cudaMemsetAsync(dX, 0, (size_t)(B * L * d * es), st) != cudaSuccess) return SIGK_ECUDA;
    if (dY && cudaMemsetAsync(dY, 0, (size_t)(B * M * d * es), st) != cudaSuccess) return SIGK_ECUDA;
    if (L < 2 || M < 2 || (!dX && !dY)) return SIGK_OK;
    const int64_t fit = (int64_t)SIGK_NOALLOC_SCRATCH_BYTES / slot;
    if (grid > fit) grid = fit;
    PairSrc src;
    memset(&src, 0, sizeof(src));
    src.mode = PM_PAIRS;
    src.A = X; src.B = Y;
    src.La = L; src.Lb = M; src.d = d;
    return launch_bwd_plain(src, B, dyadic_order, dtype, grad_out, dX, dY, scratch, grid, slot, smem,
                            st) == cudaSuccess ? SIGK_OK : SIGK_ECUDA;
}
