/*
 * sigk.h — C ABI of libsigk: the signature kernel of two streams, computed
 * as the solution of its Goursat PDE on a dyadically refined grid.
 *
 * Paper: C. Salvi, T. Cass, J. Foster, T. Lyons, W. Yang, "The Signature
 * Kernel is the solution of a Goursat PDE" (arXiv 2006.14794).
 *
 *   k_{x,y}(s,t) = <S(x)_s, S(y)_t>                      (Def. "signature kernel")
 *   d^2 k / ds dt = <x'_s, y'_t> k,  k(u,.) = k(.,v) = 1  (Thm. "PDE")
 *
 * solved with the explicit finite-difference scheme of Sec. 3.1 on the grid
 * P_lambda, which splits every cell of the sample grid into
 * 2^lambda x 2^lambda cells (Def. of P_lambda).  On piecewise-linear paths the
 * refined increment inner product is 2^(-2 lambda) <dx_p, dy_q> (remark after
 * the scheme):
 *
 *   k(i+1,j+1) = k(i+1,j) + k(i,j+1) - k(i,j)
 *                + 1/2 <dx, dy> (k(i+1,j) + k(i,j+1)),   k(0,.) = k(.,0) = 1,
 *
 * and the kernel is the value at the terminal corner.  A path of L points
 * x_0..x_{L-1} in R^d gives L-1 increments; rows of P_lambda refine x
 * (Ni = 2^lambda (L-1)), columns refine y (Nj = 2^lambda (M-1)).
 *
 * Conventions for every call:
 *  - Every pointer is caller-owned DEVICE memory, row-major and contiguous
 *    (paths [B, L, d]; outputs [B] or [Bx, By]); 4-byte (f32) or 8-byte (f64)
 *    alignment.  Offsets of the uneven-length calls are device int64 arrays.
 *  - Calls are asynchronous on `stream` (0 = the legacy default stream).
 *    Argument errors are detected on the host, return an error code and
 *    launch nothing.  CUDA launch errors return SIGK_ECUDA.
 *  - A call needing scratch memory takes it from the caller-provided
 *    workspace `ws` of `ws_bytes` bytes; size it with sigk_workspace_bytes.
 *    Calls whose workspace size is 0 accept ws = NULL.
 *  - L = 1 or M = 1 (a single point) is valid and gives k = 1.  B = 0 is
 *    valid and launches nothing.  d >= 1.  0 <= dyadic_order <= 8.
 *  - NaN or Inf inputs propagate to the outputs; nothing traps.
 *  - Time augmentation and path scaling are the caller's job.
 *  - No C++ exception crosses this interface.
 */
#ifndef SIGK_H
#define SIGK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SIGK_OK = 0,
    SIGK_EINVAL = 1,        /* bad argument (null pointer, negative size, ...) */
    SIGK_ENOMEM_WS = 2,     /* workspace missing or smaller than required      */
    SIGK_ECUDA = 3,         /* a CUDA call failed (launch error, bad device)   */
    SIGK_ETIMEOUT = 4,      /* a device-side bounded wait expired              */
    SIGK_EUNSUPPORTED = 5   /* valid but unsupported (dyadic order > 8, ...)   */
} sigk_status;

typedef enum { SIGK_F32 = 0, SIGK_F64 = 1 } sigk_dtype;   /* storage AND arithmetic */

/* Recurrence form and schedule.
 *  CHAIN: the register-resident wavefront in the difference form of the
 *    scheme: for pairs of equal lengths whose refined rows fit one warp
 *    (2^lambda (L-1) <= 512 for the shorter path) each warp solves a chain
 *    of pairs; otherwise (long or uneven pairs, wide d) the strip path: the
 *    grid is cut into 512-row (f32) or 256-row (f64) strips solved by warps
 *    of a persistent kernel that hand bottom rows on behind bounded waits,
 *    with the coarse-cell coefficients formed first by a separate kernel.
 *    It needs workspace (sigk_workspace_bytes) and dyadic_order <= 3.
 *  PLAIN: one thread block per pair sweeping the anti-diagonals, the scheme
 *    as printed (f64) or its difference form (f32): the baseline.
 *  STRIP: the strip path even where the register chain would apply
 *    (SIGK_EUNSUPPORTED where the strip path has no instance).
 *  BAND (f32, equal lengths, 2^lambda (L-1) <= 512 for the shorter path,
 *    dyadic_order <= 3): the register chain reading coarse-cell coefficients
 *    that a contraction kernel first writes into a banded buffer in the
 *    workspace (4 bytes per coarse cell); CHAIN and AUTO take it for f32
 *    pairs that fit a warp but are too wide (d > 16) for inline products.
 *  AUTO: CHAIN for f32 (PLAIN when CHAIN has no instance), PLAIN for f64. */
typedef enum {
    SIGK_REC_AUTO = 0, SIGK_REC_CHAIN = 1, SIGK_REC_PLAIN = 2, SIGK_REC_STRIP = 3, SIGK_REC_BAND = 4
} sigk_rec;

typedef struct {
    int rec;          /* sigk_rec; 0 = auto                                   */
    int symmetric;    /* gram only: X == Y and Bx == By; fills the lower
                         triangle by mirroring the upper one                  */
    int fault_inject; /* test only, 0 otherwise: 1 makes the first strip of
                         the first pair of the strip path never publish its
                         bottom row, so the strip below waits out its bounded
                         wait (~1 s) and sigk_stream_status reports
                         SIGK_ETIMEOUT; nothing faults on the device          */
    int rows_per_lane;/* schedule: refined rows per lane (4, 8 or 16; 0 =
                         default).  Chained and band kernels: the band height
                         32 x rows_per_lane (default the smallest that fits).
                         Strip path (f32: 16 by default, 8 at dyadic order 0;
                         8 for dyadic order <= 2, 4 for <= 1 on request; f64:
                         8): the strip height.  A value
                         without an instance gives SIGK_EUNSUPPORTED; the
                         plain path ignores it                                */
    int coef_path;    /* strip path coefficients: 0 auto (split-TF32 on the
                         tcgen05 tensor cores for f32 with 32 <= d <= 64,
                         warp-level MMAs for larger d, FMA otherwise), 1 FMA
                         contraction, 2 split-TF32 warp-level MMAs (mma.sync),
                         3 split-TF32 tcgen05 MMAs (d <= 64); 2 and 3 are f32
                         only (f64 gives SIGK_EUNSUPPORTED).  Band form: 3
                         takes the tcgen05 contraction, anything else the FMA
                         one; in a Gram's backward 3 also takes the chain
                         rule (the contractions of dk/dc with the increments)
                         to the tcgen05 tensor cores.  Uneven lengths in the
                         band form always use the FMA contraction.  Other
                         paths ignore it                                      */
    int orient;       /* strip path: which path the rows refine.  0 auto (the
                         shorter path from 1024 pairs per call on, else the
                         longer), 1 the longer (more strips per pair: more
                         warps on few pairs), 2 the shorter (fewer virtual
                         rows and fill/drain steps per cell)                   */
    int scheme;       /* sigk_scheme: 0 the explicit scheme (Sec. 3.1), 1 the
                         implicit four-point scheme of the remark after it   */
    int static_kernel;/* sigk_static_kernel: 0 linear (the paths as given),
                         1 RBF lift with bandwidth `sigma` (Sec. 2.2)         */
    double sigma;     /* RBF bandwidth, > 0 (ignored for the linear kernel)   */
    int accumulate;   /* backward calls (sigk_pairs_backward, sigk_gram_backward,
                         sigk_gram_value_and_grad): 0 overwrites dX / dY, 1
                         adds the gradients to what dX / dY hold (a loss that
                         sums several Grams of the same paths)                */
    int reserved[1];  /* must be 0                                            */
} sigk_opts;          /* a NULL pointer means all-zero (automatic) options    */

/* Finite-difference scheme (Sec. 3.1).
 *  EXPLICIT: the scheme above.
 *  IMPLICIT: the remark after it, whose quadrature of the cell integral uses
 *    all four corners:
 *      k(i+1,j+1) = k(i+1,j) + k(i,j+1) - k(i,j)
 *                   + 1/4 <dx, dy> (k(i,j) + k(i+1,j) + k(i,j+1) + k(i+1,j+1)).
 *    Solved for k(i+1,j+1) it is the explicit update with 1 + <dx,dy>/2
 *    replaced by (1 + <dx,dy>/4) / (1 - <dx,dy>/4), so every schedule runs
 *    it; it is undefined where a refined cell has <dx, dy> = 4 (the inputs
 *    are then far too coarse for either scheme). */
typedef enum { SIGK_SCHEME_EXPLICIT = 0, SIGK_SCHEME_IMPLICIT = 1 } sigk_scheme;

/* Static kernel on the ambient space (Sec. 2.2).  The paths are lifted into
 * the kernel's feature space; the lifted PDE's coefficient on coarse cell
 * (p, q) is the second difference
 *   kappa(x_{p+1}, y_{q+1}) - kappa(x_p, y_{q+1}) - kappa(x_{p+1}, y_q) + kappa(x_p, y_q),
 * split over the cell's 4^lambda refined cells as for the linear kernel.
 *  LINEAR: kappa(a, b) = <a, b>: the coefficient is <dx_p, dy_q>.
 *  RBF: kappa(a, b) = exp(-|a - b|^2 / (2 sigma^2)). */
typedef enum { SIGK_KERNEL_LINEAR = 0, SIGK_KERNEL_RBF = 1 } sigk_static_kernel;

typedef enum {
    SIGK_OP_PAIRS = 0, SIGK_OP_GRAM = 1, SIGK_OP_PAIRS_VARLEN = 2,
    SIGK_OP_PAIRS_BACKWARD = 3, SIGK_OP_GRAM_BACKWARD = 4, SIGK_OP_PAIRS_SURFACE = 5
} sigk_op;

/* Bytes of device workspace the call `op` needs for these sizes (B_or_Bx is
 * B for pair calls; By is ignored for them).  For SIGK_OP_PAIRS_VARLEN pass
 * L = M = the longest path length.  Returns 0 when no workspace is needed.
 * Never fails; nonsense sizes give 0. */
size_t sigk_workspace_bytes(int op, int64_t B_or_Bx, int64_t By, int64_t L, int64_t M,
                            int64_t d, int dyadic_order, int dtype, const sigk_opts *opts);

/* out[b] = k(X_b, Y_b), b < B.   X: [B, L, d], Y: [B, M, d], out: [B].
 * Defines: Def. "signature kernel" + the explicit scheme of Sec. 3.1. */
int sigk_pairs(const void *X, const void *Y, int64_t B, int64_t L, int64_t M, int64_t d,
               int dyadic_order, int dtype, const sigk_opts *opts, void *out, void *ws,
               size_t ws_bytes, void *stream);

/* out[i * By + j] = k(X_i, Y_j).   X: [Bx, L, d], Y: [By, M, d], out: [Bx, By].
 * The Gram matrices used by the paper's kernel methods (Sec. 5). */
int sigk_gram(const void *X, const void *Y, int64_t Bx, int64_t By, int64_t L, int64_t M,
              int64_t d, int dyadic_order, int dtype, const sigk_opts *opts, void *out,
              void *ws, size_t ws_bytes, void *stream);

/* Pairs of uneven lengths.  Path b of X is rows x_off[b] .. x_off[b+1]-1 of
 * Xp [sum L, d]; likewise Y.  x_off, y_off: device int64 [B+1], nondecreasing,
 * x_off[0] = 0.  max_len: an upper bound on every path length (host value).
 * out: [B].  Same scheme as sigk_pairs, per pair.
 * f32 with rec CHAIN (default rows_per_lane, linear static kernel), d <= 16,
 * dyadic order <= 2 and max_len <= 513: warp stacks, each pair's rows
 * refining its shorter path in bands of 64 coarse rows, one warp a band, the
 * coefficients formed inside the sweep (no coefficient in memory); rec AUTO
 * takes them for d <= 8, or where the band form has no class for max_len.
 * Otherwise f32 with rec AUTO or BAND: the band form, when 2^lambda
 * (max_len - 1) refined rows fit its largest band (dyadic order 0: 512,
 * orders 1 and 2: 1024; orders above 2 have none); else the strip path (rec
 * BAND: then SIGK_EUNSUPPORTED).  Both forms plan every pair's geometry on the
 * device (no host round trip; CUDA-graph capturable) and run their stack
 * heights or band classes on library-owned streams forked from and joined to
 * `stream` by events, created on the first such call on a device. */
int sigk_pairs_varlen(const void *Xp, const int64_t *x_off, const void *Yp,
                      const int64_t *y_off, int64_t B, int64_t d, int64_t max_len,
                      int dyadic_order, int dtype, const sigk_opts *opts, void *out, void *ws,
                      size_t ws_bytes, void *stream);

/* The solution surface on the sample grid: surf[b][i][j] = the scheme's value
 * at the node (s_i, t_j) of the sample grid P_0 inside P_lambda, i.e. at
 * refined node (2^lambda i, 2^lambda j): the solution k_{x,y}(s_i, t_j) of the
 * Goursat problem on [u, s_i] x [v, t_j] (Sec. 3.1, the grids of Def. P_lambda
 * and Fig. "error"), for i < L over X_b's points and j < M over Y_b's.  Row 0
 * and column 0 are the boundary value 1; surf[b][L-1][M-1] = out[b] = k.
 * X: [B, L, d], Y: [B, M, d]; out: [B]; surf: [B, L, M] (both overwritten).
 * opts as for sigk_pairs (scheme and static kernel included).  f32 pairs
 * whose shorter path fits a warp (2^lambda (L-1) <= 512) run a chained sweep
 * that keeps the nodes in a band layout in the workspace, then an unpack
 * into surf (size the workspace with SIGK_OP_PAIRS_SURFACE): with the
 * coefficients formed inline (rec AUTO or CHAIN, explicit scheme, linear
 * static kernel, d <= 16 where the chained kernel has an instance), else
 * from the band form's coefficient band; others run the plain sweep without
 * a workspace.  SIGK_REC_STRIP gives SIGK_EUNSUPPORTED (the strip path keeps
 * no surface); SIGK_REC_BAND where the band form does not apply too.
 * Writes B L M elements: HBM-bound once the grid is small. */
int sigk_pairs_surface(const void *X, const void *Y, int64_t B, int64_t L, int64_t M, int64_t d,
                       int dyadic_order, int dtype, const sigk_opts *opts, void *out, void *surf,
                       void *ws, size_t ws_bytes, void *stream);

/* Reverse-mode derivative of sigk_pairs: dX[b] = grad_out[b] dk_b/dX_b and
 * dY[b] = grad_out[b] dk_b/dY_b (either output may be NULL to skip it).
 * The paper states no gradient; this is the exact derivative of the discrete
 * scheme (adjoint sweep from the terminal corner, then the chain rule through
 * <dx_p, dy_q>).  grad_out: [B]; dX: [B, L, d]; dY: [B, M, d] (overwritten).
 * opts->scheme selects the scheme differentiated.  With the RBF lift
 * (opts->static_kernel) the chain rule goes through the second difference of
 * kappa over the points (dk/dkappa(i,j) from four neighbouring dk/dc, then
 * dkappa/dx_i = kappa (y_j - x_i) / sigma^2): in f32 on the band form when
 * the pair fits it (the symmetric Gram backward included), else in the
 * one-block-per-pair backward; SIGK_REC_STRIP gives SIGK_EUNSUPPORTED. */
int sigk_pairs_backward(const void *grad_out, const void *X, const void *Y, int64_t B,
                        int64_t L, int64_t M, int64_t d, int dyadic_order, int dtype,
                        const sigk_opts *opts, void *dX, void *dY, void *ws, size_t ws_bytes,
                        void *stream);

/* Reverse-mode derivative of sigk_gram: dX[i] = sum_j grad_out[i,j] dk_ij/dX_i,
 * dY[j] = sum_i grad_out[i,j] dk_ij/dY_j (either may be NULL).
 * grad_out: [Bx, By].  dX, dY overwritten.
 * With opts->symmetric (X == Y: the caller passes the same paths, Bx == By,
 * L == M, dY NULL): dX = d/dX sum_ij grad_out[i,j] k(X_i, X_j), the derivative
 * through both arguments, from the pairs i <= j only (k(x,y) = k(y,x)).  f32
 * only, and only where the band form applies (SIGK_EUNSUPPORTED otherwise). */
int sigk_gram_backward(const void *grad_out, const void *X, const void *Y, int64_t Bx,
                       int64_t By, int64_t L, int64_t M, int64_t d, int dyadic_order,
                       int dtype, const sigk_opts *opts, void *dX, void *dY, void *ws,
                       size_t ws_bytes, void *stream);

/* sigk_gram and sigk_gram_backward in one pass, for a caller whose grad_out
 * does not depend on the Gram's values (a loss linear in the Gram, such as
 * the unbiased MMD^2 of Sec. 4, whose derivative with respect to each Gram is
 * a constant matrix).  out [Bx, By] receives the Gram's values, written by
 * the backward's own forward sweep (the band form, which also keeps the
 * checkpoints the adjoint needs; within rounding of sigk_gram's values where
 * sigk_gram picks another sweep), dX and dY what sigk_gram_backward computes
 * for grad_out; arguments, opts (symmetric included) and layouts as there.
 * The workspace is the backward's (size it with SIGK_OP_GRAM_BACKWARD).
 * Saves the separate forward call: its coefficient contraction and sweep.
 * Only where the backward runs in the band form (f32, the shorter path
 * fitting a warp, both lengths >= 2, the linear static kernel):
 * SIGK_EUNSUPPORTED otherwise, before any launch, and the caller then makes
 * the two calls. */
int sigk_gram_value_and_grad(const void *grad_out, const void *X, const void *Y, int64_t Bx,
                             int64_t By, int64_t L, int64_t M, int64_t d, int dyadic_order,
                             int dtype, const sigk_opts *opts, void *out, void *dX, void *dY,
                             void *ws, size_t ws_bytes, void *stream);

/* sigk_pairs_backward without a workspace argument: the paper has no
 * counterpart; this entry point exists for callers that cannot allocate
 * device memory at call time (a process that hands all device memory to its
 * own pool at start-up, or runs under a fixed memory budget, where one more
 * cudaMalloc fails or stalls the device).  It allocates nothing: the
 * per-block scratch of the adjoint sweep lives in a fixed 32 MiB array in the
 * library's device image, which every GPU that loads the library holds until
 * the process exits.  Arguments, layout and results are those of
 * sigk_pairs_backward (dX, dY may be NULL; both are overwritten).
 * Returns SIGK_EUNSUPPORTED when one pair's scratch,
 * (2 (L-1)(M-1) + (2^lambda (L-1) + 1)(2^lambda (M-1) + 1)) elements,
 * exceeds the array.  The first call on each device looks the array's device
 * address up (cudaGetSymbolAddress, with that device current) and keeps it
 * for that device's context; the first call after the context was reset
 * (cudaDeviceReset) looks it up again.  All calls share the array:
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.  No state carries over between calls. */
int sigk_pairs_backward_noalloc(const void *grad_out, const void *X, const void *Y, int64_t B,
                                int64_t L, int64_t M, int64_t d, int dyadic_order, int dtype,
                                void *dX, void *dY, void *stream);

/* The unbiased MMD^2 estimator between two batches (Sec. 3.1.1 names it; the
 * U-statistic form) from the three Gram matrices:
 *   out[0] = sum_{i!=j} Kxx_ij / (m(m-1)) + sum_{i!=j} Kyy_ij / (n(n-1))
 *            - 2 sum_{i,j} Kxy_ij / (mn).
 * Kxx [m,m], Kyy [n,n], Kxy [m,n]; out: one element.  m, n >= 2. */
int sigk_mmd2(const void *Kxx, const void *Kyy, const void *Kxy, int64_t m, int64_t n,
              int dtype, void *out, void *stream);

/* Gradient of sigk_mmd2 with respect to the three Gram matrices, scaled by
 * the scalar grad (device, one element): writes gKxx [m,m], gKyy [n,n],
 * gKxy [m,n] (any may be NULL). */
int sigk_mmd2_backward(const void *grad, int64_t m, int64_t n, int dtype, void *gKxx,
                       void *gKyy, void *gKxy, void *stream);

/* The chain rule through a scalar loss whose input gradients were formed
 * before its upstream derivative was known (sigk_gram_value_and_grad with a
 * constant dL/dK, as for the unbiased MMD^2, which is linear in the Grams):
 *   g_out[i] = grad[0] * g_in[i],  i < n.
 * grad: device, one element; g_in, g_out: device, n elements (may alias).
 * n >= 0.  Asynchronous on `stream`; no workspace. */
int sigk_scale_grad(const void *grad, const void *g_in, void *g_out, int64_t n, int dtype,
                    void *stream);

/* Moments-matching reduction of the support of a discrete measure on paths
 * (Sec. 5.3).  With K the signature-kernel Gram of the support's N paths
 * (e.g. sigk_gram of X with itself) and weights alpha, proximal gradient
 * descent on L(beta) + lam |beta|_1, L(beta) = (alpha - beta)^T K (alpha - beta):
 *   beta <- A_{gamma lam}(beta + 2 gamma K (alpha - beta)),
 * A_tau the paper's soft-thresholding operator (the proximal map of
 * tau |.|_1; the paper writes A_gamma with the penalty folded in).
 * K: [N, N] (symmetric), alpha: [N]; beta: [N], in: beta^0, out: beta after
 * `iters` steps; loss: [iters + 1] or NULL, L(beta^t) + lam |beta^t|_1 for
 * t = 0..iters.  gamma > 0 (convergence needs gamma <= 1 / (2 |K|)),
 * lam >= 0, iters >= 0.  One thread block runs every step in one launch,
 * with alpha and beta (and K, for N up to about 220 in f32) in shared memory;
 * N above 17066 (f32) or 8533 (f64) gives SIGK_EUNSUPPORTED.  No workspace.
 * The loss is summed with atomic adds: its last bits may vary run to run. */
int sigk_support_reduction(const void *K, const void *alpha, void *beta, int64_t N, double gamma,
                           double lam, int iters, int dtype, void *loss, void *stream);

/* Status word of the last strip-path call that used workspace `ws` on
 * `stream`: synchronises the stream, then returns SIGK_OK or SIGK_ETIMEOUT
 * (a bounded device wait expired; that call's results are meaningless).
 * SIGK_OK when ws is NULL.  Only meaningful after a call that took the strip
 * path (it needed workspace). */
int sigk_stream_status(void *stream, void *ws);

/* Static description of a status code (never NULL). */
const char *sigk_strerror(int status);

/* Library version, e.g. "sigk 0.1 sm_103a". */
const char *sigk_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SIGK_H */
