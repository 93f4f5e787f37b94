// Internal declarations shared by the libsigk CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sigk.h"

namespace sigk {

constexpr unsigned FULL = 0xffffffffu;

// How a flat pair index maps to (row path, column path, output slots).
// The grid's rows refine the "A" path and its columns the "B" path.
enum PairMode { PM_PAIRS = 0, PM_GRAM = 1, PM_GRAM_SYM = 2, PM_VARLEN = 3 };

struct PairSrc {
    int mode;
    const void *A;          // row paths
    const void *B;          // column paths
    const int64_t *a_off;   // varlen offsets (rows of A), [n+1]
    const int64_t *b_off;
    int64_t nb;             // gram: number of B paths (columns of the enumeration)
    int64_t La, Lb;         // uniform lengths (ignored for varlen)
    int64_t d;
    int64_t out_si, out_sj; // gram: out index = i*out_si + j*out_sj
    int64_t kbase;          // pair k of a launch is pair kbase + k of the call
    int scheme;             // sigk_scheme: how a cell's coefficient enters (scheme_coef)
    int kernel;             // sigk_static_kernel
    double sigma;           // RBF bandwidth
};

// The implicit scheme (Sec. 3.1, remark after the explicit scheme) solved for
// its unknown corner is k(a,b) = (k(a,b-1) + k(a-1,b)) (1 + g/4)/(1 - g/4) -
// k(a-1,b-1): the explicit update with the coefficient c = g/2 of the
// difference form replaced by c / (1 - c/2).  Every producer of coefficients
// passes c through this map, so every sweep runs either scheme.
__device__ __forceinline__ float scheme_coef(float c, int scheme) {
    return scheme == SIGK_SCHEME_IMPLICIT ? __fdividef(c, 1.f - 0.5f * c) : c;
}
__device__ __forceinline__ double scheme_coef(double c, int scheme) {
    return scheme == SIGK_SCHEME_IMPLICIT ? c / (1.0 - 0.5 * c) : c;
}
// The RBF lift (Sec. 2.2): the coarse cell's coefficient is the second
// difference of kappa(a,b) = exp(-|a-b|^2 / (2 sigma^2)) over its corners.
// From u = x_p - y_q, dx = x_{p+1} - x_p, dy = y_{q+1} - y_q and the channel
// sums uu = |u|^2, ux = <u,dx>, uy = <u,dy>, xy = <dx,dy>, nx = |dx|^2,
// ny = |dy|^2, with s = 1/(2 sigma^2):
//   kappa(x_p, y_q) = e = exp(-s uu),        kappa(x_p, y_{q+1}) = e exp(A),
//   kappa(x_{p+1}, y_q) = e exp(B),          kappa(x_{p+1}, y_{q+1}) = e exp(A + B + C),
// A = s (2 uy - ny), B = -s (2 ux + nx), C = 2 s xy (|u - dy|^2, |u + dx|^2 and
// |u + dx - dy|^2 expanded), so the second difference is
//   e (exp(A+B+C) - exp(A) - exp(B) + 1) = e (expm1(A) expm1(B) + exp(A+B) expm1(C)):
// no O(1) values cancel, and FP32 keeps the relative accuracy of the small
// coefficient that the plain four-term difference would lose.
// e^x - 1 in FP32 without cancellation: the Taylor series through x^8 / 8! for
// |x| <= 1/2 (truncation below 2e-8 relative, Horner in FMAs), e^x - 1 beyond,
// where the subtraction loses less than 4e-7 relative.  The lift's exponents
// are small differences of squared distances, so the series is the common case.
__device__ __forceinline__ float expm1_taylor(float x) {
    if (fabsf(x) > 0.5f) return expf(x) - 1.f;
    float p = 1.f / 40320.f;
    p = fmaf(p, x, 1.f / 5040.f);
    p = fmaf(p, x, 1.f / 720.f);
    p = fmaf(p, x, 1.f / 120.f);
    p = fmaf(p, x, 1.f / 24.f);
    p = fmaf(p, x, 1.f / 6.f);
    p = fmaf(p, x, 0.5f);
    p = fmaf(p, x, 1.f);
    return p * x;
}
// The two plain exponentials take the hardware exp2 (__expf): its error is a
// few 1e-7 relative for the moderate arguments here, and a cell whose points
// are many bandwidths apart has a negligible coefficient either way.
__device__ __forceinline__ float rbf_second_difference(float uu, float ux, float uy, float xy, float nx,
                                                       float ny, float s) {
    const float A = s * (2.f * uy - ny), B = -s * (2.f * ux + nx), C = 2.f * s * xy;
    return __expf(-s * uu) * (expm1_taylor(A) * expm1_taylor(B) + __expf(A + B) * expm1_taylor(C));
}
__device__ __forceinline__ double rbf_second_difference(double uu, double ux, double uy, double xy,
                                                        double nx, double ny, double s) {
    const double A = s * (2.0 * uy - ny), B = -s * (2.0 * ux + nx), C = 2.0 * s * xy;
    return exp(-s * uu) * (expm1(A) * expm1(B) + exp(A + B) * expm1(C));
}

// dc'/dc of that map, written through c' = c / (1 - c/2): (1 + c'/2)^2.  The
// adjoint sweeps use c' like the forward and so sum dk/dc'; times this factor
// per coarse cell it is dk/dc.
template <typename T>
__device__ __forceinline__ T scheme_dcoef(T cp, int scheme) {
    const T t = (T)1 + (T)0.5 * cp;
    return scheme == SIGK_SCHEME_IMPLICIT ? t * t : (T)1;
}

struct PairRef {
    int64_t a_row0, la;     // first point row of the A path, and its length
    int64_t b_row0, lb;
    int64_t out0, out1;     // output slots (out1 = -1 when only one)
};

// Upper-triangle enumeration (i <= j) of an n x n symmetric Gram matrix.
__host__ __device__ inline void sym_index(int64_t k, int64_t n, int64_t &i, int64_t &j) {
    // row i holds n - i entries, starting at off(i) = i*n - i*(i-1)/2
    double nn = (double)n;
    double disc = (2.0 * nn + 1.0) * (2.0 * nn + 1.0) - 8.0 * (double)k;
    int64_t ii = (int64_t)((2.0 * nn + 1.0 - sqrt(disc > 0 ? disc : 0.0)) * 0.5);
    if (ii < 0) ii = 0;
    if (ii > n - 1) ii = n - 1;
    while (ii > 0 && ii * n - ii * (ii - 1) / 2 > k) --ii;
    while (ii + 1 < n && (ii + 1) * n - (ii + 1) * ii / 2 <= k) ++ii;
    i = ii;
    j = ii + (k - (ii * n - ii * (ii - 1) / 2));
}

__host__ __device__ inline PairRef pair_ref(const PairSrc &s, int64_t k) {
    PairRef r;
    k += s.kbase;
    r.out1 = -1;
    if (s.mode == PM_PAIRS) {
        r.a_row0 = k * s.La; r.la = s.La;
        r.b_row0 = k * s.Lb; r.lb = s.Lb;
        r.out0 = k;
    } else if (s.mode == PM_GRAM) {
        int64_t i = k / s.nb, j = k - (k / s.nb) * s.nb;
        r.a_row0 = i * s.La; r.la = s.La;
        r.b_row0 = j * s.Lb; r.lb = s.Lb;
        r.out0 = i * s.out_si + j * s.out_sj;
    } else if (s.mode == PM_GRAM_SYM) {
        int64_t i, j;
        sym_index(k, s.nb, i, j);
        r.a_row0 = i * s.La; r.la = s.La;
        r.b_row0 = j * s.Lb; r.lb = s.Lb;
        r.out0 = i * s.nb + j;
        r.out1 = (i != j) ? j * s.nb + i : -1;
    } else {
        r.a_row0 = s.a_off[k]; r.la = s.a_off[k + 1] - s.a_off[k];
        r.b_row0 = s.b_off[k]; r.lb = s.b_off[k + 1] - s.b_off[k];
        r.out0 = k;
    }
    return r;
}

// ---- launchers (each returns a cudaError_t) --------------------------------

struct ChainPlan {
    int R, lam, D4;         // rows per lane, dyadic order, channel float4 chunks
    int Tper, vpad, vtop;   // period (refined columns incl. virtual), pads
    int NQ, NQV;            // coarse columns incl. virtual, virtual ones
    int nby, nbx, nout;     // per-warp column / row increment buffers, output slots
    int yunits, xunits;     // their sizes (float4 units)
    int warp_units;         // shared memory per warp (float4 units)
    int64_t ppw;            // pairs per warp
    int grid, smem_bytes;
};

// Geometry and shared memory of the chained kernel, with no device query;
// false when it has no instance for these sizes.
bool chain_geometry(int64_t La, int64_t Lb, int64_t d, int lam, ChainPlan &p, int rows_per_lane = 0);
// Returns false when the chained kernel has no instance for these sizes.
bool chain_plan(int64_t n_pairs, int64_t La, int64_t Lb, int64_t d, int lam, ChainPlan &p,
                int rows_per_lane = 0);
// sband (explicit scheme only): also the solution surface's sample-grid
// nodes in the band layout of the surface unpack (launch_surface_unpack),
// Tper/R + 1 slots of 32 (R/2^lambda)^2 floats a pair.
cudaError_t launch_chain_f32(const PairSrc &src, const ChainPlan &p, int64_t n_pairs,
                             float *out, cudaStream_t st, float *sband = nullptr);

// The band form (fwd_band.cu): the row chain reading coefficients that a
// contraction kernel formed beforehand into a banded buffer (the workspace).
struct BandPlan {
    int R, lam, NG;         // rows per lane, dyadic order, coarse rows per lane
    int TperR;              // macro-steps per pair
    int NQ, NQV, vrows;     // padded coarse columns, virtual columns, virtual coarse rows
    int64_t slot_floats;    // floats per (pair, position) slot row: 32 lanes x NG x NG
};
// Geometry only (no device query); false when the band form has no instance.
bool band_geometry(int64_t La, int64_t Lb, int lam, int rows_per_lane, BandPlan &p);
int64_t band_bytes(const BandPlan &p, int64_t n_pairs);
// with the solution surface: the band, then the surface values in the band layout
int64_t band_surface_offset(const BandPlan &p, int64_t n_pairs);
int64_t band_surface_bytes(const BandPlan &p, int64_t n_pairs);
// coef_path 3: coefficients on tcgen05 (d <= 64); otherwise the FMA contraction
// surf (optional): the solution surface, node (i, j) of pair k (of the call)
// at surf[k s_pair + i s_a + j s_b]; nodes on row or column 0 are not written.
// It needs band_surface_bytes of workspace instead of band_bytes.
cudaError_t launch_band_f32(const PairSrc &src, const BandPlan &p, int64_t n_pairs, float *out,
                            void *ws, cudaStream_t st, int coef_path, float *surf = nullptr,
                            int64_t s_pair = 0, int64_t s_a = 0, int64_t s_b = 0);
// The surface from its band-layout node values (written by a SURF sweep,
// band or chain, with geometry p) into surf[k s_pair + i s_a + j s_b].
cudaError_t launch_surface_unpack(const PairSrc &src, const BandPlan &p, int64_t n_pairs, const float *sband,
                                  float *surf, int64_t s_pair, int64_t s_a, int64_t s_b, cudaStream_t st);
// The band backward (reversible adjoint): pairs per launch (Gram: whole rows)
// under cap_bytes, with the workspace that needs (coef_path 3 adds a Gram's
// dense dk/dc for the tensor-core contraction); then the launches.  src is
// oriented (rows refine A); dA / dB (either may be null) are overwritten.
int64_t band_bwd_batch(const PairSrc &src, const BandPlan &p, int64_t n, int64_t cap_bytes,
                       int64_t &bytes, int coef_path);
// out: null, or where the forward sweep also writes the values; add: the
// gradients are added to what dA / dB hold instead of overwriting them
cudaError_t launch_band_bwd_f32(const PairSrc &src, const BandPlan &p, int64_t n, int64_t nbp,
                                const float *gout, float *dA, float *dB, void *ws, cudaStream_t st,
                                int coef_path, float *out = nullptr, bool add = false);

cudaError_t launch_plain(const PairSrc &src, int64_t n_pairs, int lam, int dtype, void *out,
                         cudaStream_t st, void *surf = nullptr);

cudaError_t launch_fill_one(void *out, int64_t n, int dtype, cudaStream_t st);
// row 0 and (col0) column 0 of B solution surfaces [L][M] set to 1
cudaError_t launch_surface_border(void *surf, int64_t B, int64_t L, int64_t M, int dtype, cudaStream_t st,
                                  bool col0 = true);

bool bwd_plain_plan(int64_t n_pairs, int64_t La, int64_t Lb, int64_t d, int lam, int dtype,
                    int64_t &grid, int64_t &slot_bytes, int64_t &smem);
cudaError_t launch_bwd_plain(const PairSrc &src, int64_t n_pairs, int lam, int dtype,
                             const void *gout, void *dA, void *dB, void *ws, int64_t grid,
                             int64_t slot_bytes, int64_t smem, cudaStream_t st);

bool strip_supported(int lam, int64_t d, int dtype);
// rowsA / rowsB: point rows of the src.A / src.B arrays (an upper bound for
// packed uneven paths, whose exact count the kernels read from the offsets)
// R: rows per lane (strip_has_R); shorter_rows: the rows refine the shorter path
bool strip_has_R(int R, int lam, int dtype);
int64_t strip_workspace_bytes(int64_t n, int64_t max_la, int64_t max_lb, int lam, int dtype,
                              int64_t rowsA, int64_t rowsB, int64_t d, int R, int shorter_rows);
cudaError_t launch_strip(const PairSrc &src, int64_t n, int lam, int dtype, void *ws, void *out,
                         long long wait_cycles, int fault_inject, cudaStream_t st, int64_t max_la,
                         int64_t max_lb, int64_t rowsA, int64_t rowsB, int coef_path, int R,
                         int shorter_rows);

// The band form for pairs of uneven lengths (vband.cu): pairs planned on the
// device into band-height classes and chains, f32, the linear static kernel.
// Supported when every path of at most max_len points fits the largest class.
bool vband_supported(int lam, int64_t d, int64_t max_len, int dtype, int kernel);
int64_t vband_workspace_bytes(int64_t n, int64_t max_len, int lam);
cudaError_t launch_vband(const PairSrc &src, int64_t n, int lam, int64_t max_len, float *out, void *ws,
                         cudaStream_t st);

// Pairs of uneven lengths with the coefficients formed inside the sweep
// (vstack.cu): stacks of warps, one 64-coarse-row band each, f32, the linear
// static kernel, d <= 16, dyadic order <= 2, shorter paths of <= 513 points.
bool vstack_supported(int lam, int64_t d, int64_t max_len, int dtype, int kernel);
int64_t vstack_workspace_bytes(int64_t n, int64_t max_len, int64_t d);
cudaError_t launch_vstack(const PairSrc &src, int64_t n, int lam, int64_t max_len, float *out, void *ws,
                          cudaStream_t st);

// The band backward's chain rule on the tcgen05 tensor cores (chain_tc5.cu):
// C = G B (trans = 0) or G^T B (trans = 1), G [M][K] (trans: [K][M]) with row
// stride g_ld, B [K][N], C [M][N]; add: C += instead of C =; tri_rb > 0: a
// symmetric Gram's blocks (tri_rb x tri_cb) below the diagonal are zero and
// skipped.  Split-TF32 products (FP32 accuracy), N <= 64.
struct ChainGemm {
    const float *G;
    int64_t g_ld;
    int trans;
    const float *Bm;
    float *C;
    int64_t M, K;
    int N, add;
    int64_t tri_rb, tri_cb;
};
bool chain_gemm_tc5_ok(int64_t M, int64_t K, int N);
cudaError_t launch_chain_gemm_tc5(const ChainGemm &g, int *status, cudaStream_t st);

// Point rows of the src.A and src.B arrays of a call of n_total pairs.
inline void src_rows(const PairSrc &s, int64_t n_total, int64_t &ra, int64_t &rb) {
    if (s.mode == PM_PAIRS) { ra = n_total * s.La; rb = n_total * s.Lb; }
    else if (s.mode == PM_GRAM) { ra = (n_total / s.nb) * s.La; rb = s.nb * s.Lb; }
    else if (s.mode == PM_GRAM_SYM) { ra = s.nb * s.La; rb = ra; }
    else { ra = n_total * s.La; rb = n_total * s.Lb; }   // packed: upper bounds
}
int read_status_word(void *ws, cudaStream_t st, int *status);
int64_t strip_bwd_workspace_bytes(int64_t n, int64_t max_la, int64_t max_lb, int lam, int dtype,
                                  int64_t rowsA, int64_t rowsB, int64_t d);
cudaError_t launch_strip_bwd(const PairSrc &src, int64_t n, int lam, int dtype, void *ws,
                             const void *gout, void *dA, void *dB, long long wait_cycles,
                             cudaStream_t st, int64_t max_la, int64_t max_lb, int64_t rowsA,
                             int64_t rowsB, int coef_path);

// Support reduction (support.cu): largest N one block holds, and the launch.
int64_t support_max_n(int dtype);
cudaError_t launch_support(const void *K, const void *alpha, void *beta, int64_t N, double gamma,
                           double lam, int iters, int dtype, void *loss, cudaStream_t st);

cudaError_t launch_mmd2(const void *Kxx, const void *Kyy, const void *Kxy, int64_t m, int64_t n,
                        int dtype, void *out, cudaStream_t st);
cudaError_t launch_scale_grad(const void *grad, const void *g_in, void *g_out, int64_t n, int dtype,
                              cudaStream_t st);
cudaError_t launch_mmd2_backward(const void *grad, int64_t m, int64_t n, int dtype, void *gKxx,
                                 void *gKyy, void *gKxy, cudaStream_t st);

}  // namespace sigk
