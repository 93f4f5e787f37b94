// libsigk C ABI: argument checks, kernel choice and launches.  No call here
// allocates memory; no C++ exception crosses the interface.
#include <stdio.h>
#include <string.h>

#include "sigk_internal.cuh"

using namespace sigk;

namespace {

bool opts_ok(const sigk_opts *o) {
    if (!o) return true;
    if (o->rec < SIGK_REC_AUTO || o->rec > SIGK_REC_BAND) return false;
    if (o->symmetric != 0 && o->symmetric != 1) return false;
    if (o->fault_inject != 0 && o->fault_inject != 1) return false;
    if (o->rows_per_lane != 0 && o->rows_per_lane != 4 && o->rows_per_lane != 8 &&
        o->rows_per_lane != 16)
        return false;
    if (o->coef_path < 0 || o->coef_path > 3) return false;
    if (o->orient < 0 || o->orient > 2) return false;
    if (o->scheme != SIGK_SCHEME_EXPLICIT && o->scheme != SIGK_SCHEME_IMPLICIT) return false;
    if (o->static_kernel != SIGK_KERNEL_LINEAR && o->static_kernel != SIGK_KERNEL_RBF) return false;
    if (o->static_kernel == SIGK_KERNEL_RBF && !(o->sigma > 0.0 && o->sigma < 1e300)) return false;
    if (o->accumulate != 0 && o->accumulate != 1) return false;
    if (o->reserved[0] != 0) return false;
    return true;
}

int rec_of(const sigk_opts *o) { return o ? o->rec : SIGK_REC_AUTO; }

// The scheme and static kernel a call solves, carried with its pairs.
void set_variant(PairSrc &s, const sigk_opts *o) {
    s.scheme = o ? o->scheme : SIGK_SCHEME_EXPLICIT;
    s.kernel = o ? o->static_kernel : SIGK_KERNEL_LINEAR;
    s.sigma = o && o->static_kernel == SIGK_KERNEL_RBF ? o->sigma : 1.0;
}

int common_checks(int64_t B, int64_t L, int64_t M, int64_t d, int lam, int dtype,
                  const sigk_opts *opts) {
    if (B < 0 || L < 1 || M < 1 || d < 1) return SIGK_EINVAL;
    if (dtype != SIGK_F32 && dtype != SIGK_F64) return SIGK_EINVAL;
    if (!opts_ok(opts)) return SIGK_EINVAL;
    if (lam < 0) return SIGK_EINVAL;
    if (lam > 8) return SIGK_EUNSUPPORTED;
    if (opts && opts->coef_path >= 2 && dtype != SIGK_F32) return SIGK_EUNSUPPORTED;
    if (opts && opts->coef_path == 3 && d > 64) return SIGK_EUNSUPPORTED;
    // the RBF lift forms its coefficients with its own kernel (no tensor-core path)
    if (opts && opts->static_kernel == SIGK_KERNEL_RBF && opts->coef_path >= 2) return SIGK_EUNSUPPORTED;
    return SIGK_OK;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SIGK_OK;
    if (e == cudaErrorInvalidConfiguration) return SIGK_EUNSUPPORTED;
    return SIGK_ECUDA;
}

// Bounded device waits of the strip path: ~1 s at the GB300's 2.07 GHz clock.
constexpr long long WAIT_CYCLES = 2000000000LL;
// Largest workspace the strip path asks for; bigger batches run in pieces.
constexpr int64_t STRIP_WS_CAP = 8LL << 30;
// the band backward's batches: a 128 x 128 Gram of 256-point paths (band,
// dense dk/dG and its band layout, about 13 GB) in one launch
constexpr int64_t BAND_BWD_WS_CAP = 16LL << 30;

int fault_of(const sigk_opts *o) { return o ? o->fault_inject : 0; }
// backward calls: add into dX / dY instead of overwriting them
bool accumulate_of(const sigk_opts *o) { return o && o->accumulate; }
int rows_of(const sigk_opts *o) { return o ? o->rows_per_lane : 0; }
int coef_of(const sigk_opts *o) { return o ? o->coef_path : 0; }
// the strip path's rows per lane (its default, or the requested one).  f32
// defaults to 512-row strips, 256-row ones at dyadic order 0: there every
// refined cell reads its own coefficient, and twice the strips (warps) hide
// that better (64 pairs of 4096 points: 5.3 against 6.2 ms; at order 1 the
// 512-row strips stay faster, 7.4 against 7.7 ms)
int strip_R_of(const sigk_opts *o, int dtype, int lam) {
    const int r = rows_of(o);
    return r != 0 ? r : (dtype == SIGK_F64 ? 8 : (lam == 0 ? 8 : 16));
}
// rows refine the shorter path: on request, or by default with many pairs
// in flight (parallelism then comes from the pairs, and fewer virtual rows
// and fill/drain steps per cell win)
int shorter_of(const sigk_opts *o, int64_t n_pairs) {
    const int v = o ? o->orient : 0;
    return v == 2 || (v == 0 && n_pairs >= 1024) ? 1 : 0;
}

// Pairs per strip-path launch and the workspace that needs.
void strip_batch(const PairSrc &src, int64_t n, int64_t la, int64_t lb, int lam, int dtype,
                 const sigk_opts *opts, int64_t &nb, int64_t &bytes) {
    int64_t ra, rb;
    src_rows(src, n, ra, rb);
    const int R = strip_R_of(opts, dtype, lam), sh = shorter_of(opts, n);
    nb = n;
    bytes = strip_workspace_bytes(nb, la, lb, lam, dtype, ra, rb, src.d, R, sh);
    while (nb > 1 && bytes > STRIP_WS_CAP) {
        nb = (nb + 1) / 2;
        bytes = strip_workspace_bytes(nb, la, lb, lam, dtype, ra, rb, src.d, R, sh);
    }
}

enum Path { P_FILL, P_CHAIN, P_BAND, P_STRIP, P_PLAIN };

// Pairs of uneven lengths in warp stacks with the coefficients formed in the
// sweep: f32, the linear static kernel, rec AUTO or CHAIN with the default
// rows, d <= 16, dyadic order <= 2 and every path of at most 513 points.
// AUTO takes them for d <= 8, or where the band form has no class for the
// longest path: at d = 16 the band form's separate FMA contraction is the
// faster of the two (4096 pairs of 16..512 points at dyadic order 1: 1.48
// against 1.94 ms), at d = 8 and below the stacks are (1.08 against 1.36 ms
// at d = 8, 0.87 against 1.40 ms at d = 3).
bool varlen_uses_band(int64_t d, int64_t max_len, int lam, int dtype, const sigk_opts *o);
bool varlen_uses_stack(int64_t d, int64_t max_len, int lam, int dtype, const sigk_opts *o) {
    const int rec = rec_of(o);
    if (rec != SIGK_REC_AUTO && rec != SIGK_REC_CHAIN) return false;
    if (rows_of(o) != 0) return false;
    if (!vstack_supported(lam, d, max_len, dtype, o ? o->static_kernel : SIGK_KERNEL_LINEAR)) return false;
    return rec == SIGK_REC_CHAIN || d <= 8 || !varlen_uses_band(d, max_len, lam, dtype, o);
}
// Pairs per stack launch and the workspace that needs.
void vstack_batch(int64_t n, int64_t max_len, int64_t d, int64_t &nb, int64_t &bytes) {
    nb = n;
    bytes = vstack_workspace_bytes(nb, max_len, d);
    while (nb > 1 && bytes > STRIP_WS_CAP) {
        nb = (nb + 1) / 2;
        bytes = vstack_workspace_bytes(nb, max_len, d);
    }
}

// Pairs of uneven lengths in the band form: f32, the linear static kernel,
// rec AUTO or BAND with the default band heights, and every path short enough
// for the largest band class.
bool varlen_uses_band(int64_t d, int64_t max_len, int lam, int dtype, const sigk_opts *o) {
    const int rec = rec_of(o);
    if (rec != SIGK_REC_AUTO && rec != SIGK_REC_BAND) return false;
    if (rows_of(o) != 0) return false;
    return vband_supported(lam, d, max_len, dtype, o ? o->static_kernel : SIGK_KERNEL_LINEAR);
}
// Pairs per varlen band launch and the workspace that needs.
void vband_batch(int64_t n, int64_t max_len, int lam, int64_t &nb, int64_t &bytes) {
    nb = n;
    bytes = vband_workspace_bytes(nb, max_len, lam);
    while (nb > 1 && bytes > STRIP_WS_CAP) {
        nb = (nb + 1) / 2;
        bytes = vband_workspace_bytes(nb, max_len, lam);
    }
}

// Band-form pairs per launch and the workspace (the coefficient band) that needs.
void band_batch(const BandPlan &bp, int64_t n, int64_t &nb, int64_t &bytes) {
    nb = n;
    bytes = band_bytes(bp, nb);
    while (nb > 1 && bytes > STRIP_WS_CAP) {
        nb = (nb + 1) / 2;
        bytes = band_bytes(bp, nb);
    }
}
// The same with the solution surface's band-layout values after the band.
void band_surface_batch(const BandPlan &bp, int64_t n, int64_t &nb, int64_t &bytes) {
    nb = n;
    bytes = band_surface_bytes(bp, nb);
    while (nb > 1 && bytes > STRIP_WS_CAP) {
        nb = (nb + 1) / 2;
        bytes = band_surface_bytes(bp, nb);
    }
}

Path choose_uniform(const PairSrc &src, int64_t n, int lam, int dtype, int rec, ChainPlan *cp,
                    int rows_per_lane = 0, BandPlan *bpo = nullptr) {
    if (src.La < 2 || src.Lb < 2) return P_FILL;
    if (rec == SIGK_REC_PLAIN) return P_PLAIN;
    if (rec == SIGK_REC_STRIP)
        return strip_supported(lam, src.d, dtype) &&
                       strip_has_R(rows_per_lane ? rows_per_lane : (dtype == SIGK_F64 ? 8 : (lam == 0 ? 8 : 16)),
                                   lam, dtype)
                   ? P_STRIP : P_FILL;
    if (rec == SIGK_REC_BAND && dtype != SIGK_F32) return P_FILL;
    if (dtype == SIGK_F64 && rec != SIGK_REC_CHAIN) return P_PLAIN;
    if (dtype == SIGK_F32) {
        int64_t la = src.La, lb = src.Lb;
        if (src.mode == PM_PAIRS && la > lb) { int64_t t = la; la = lb; lb = t; }
        BandPlan bp;
        const bool band = band_geometry(la, lb, lam, rows_per_lane, bp);
        if (band && bpo) *bpo = bp;
        if (rec == SIGK_REC_BAND) return band ? P_BAND : P_FILL;
        ChainPlan p;
        // the inline-product chain has no RBF lift: the band form forms its coefficients
        if (src.kernel == SIGK_KERNEL_LINEAR && chain_plan(n, la, lb, src.d, lam, p, rows_per_lane)) {
            if (cp) *cp = p;
            return P_CHAIN;
        }
        if (band) return P_BAND;
        if (rows_per_lane != 0) return P_FILL;   // the requested schedule has no instance
    }
    if (strip_supported(lam, src.d, dtype)) return P_STRIP;
    return rec == SIGK_REC_CHAIN ? P_FILL /* unsupported */ : P_PLAIN;
}

int run_strip(PairSrc src, int64_t n, int lam, int dtype, int64_t la, int64_t lb, const sigk_opts *opts,
              void *out, void *ws, size_t ws_bytes, cudaStream_t st) {
    int64_t nb, need, ra, rb;
    strip_batch(src, n, la, lb, lam, dtype, opts, nb, need);
    src_rows(src, n, ra, rb);
    if (!strip_has_R(strip_R_of(opts, dtype, lam), lam, dtype)) return SIGK_EUNSUPPORTED;
    if (!ws || (int64_t)ws_bytes < need) return SIGK_ENOMEM_WS;
    for (int64_t k0 = 0; k0 < n; k0 += nb) {
        PairSrc s = src;
        s.kbase = src.kbase + k0;
        const int64_t m = n - k0 < nb ? n - k0 : nb;
        cudaError_t e = launch_strip(s, m, lam, dtype, ws, out, WAIT_CYCLES,
                                     k0 == 0 ? fault_of(opts) : 0, st, la, lb, ra, rb, coef_of(opts),
                                     strip_R_of(opts, dtype, lam), shorter_of(opts, n));
        if (e != cudaSuccess) return cuda_status(e);
    }
    return SIGK_OK;
}

// Solve n_pairs pairs described by `src` (uniform lengths La x Lb).
int run_uniform(PairSrc src, int64_t n_pairs, int lam, int dtype, const sigk_opts *opts,
                void *out, void *ws, size_t ws_bytes, cudaStream_t st) {
    if (n_pairs == 0) return SIGK_OK;
    const int rec = rec_of(opts);
    ChainPlan p;
    BandPlan bp;
    switch (choose_uniform(src, n_pairs, lam, dtype, rec, &p, rows_of(opts), &bp)) {
        case P_FILL:
            if (src.La < 2 || src.Lb < 2) return cuda_status(launch_fill_one(out, n_pairs, dtype, st));
            return SIGK_EUNSUPPORTED;
        case P_CHAIN: {
            // the chained kernel wants the shorter path on the rows (k(x,y) = k(y,x));
            // sigk_gram already orders its batches, pairs are swapped here
            PairSrc s2 = src;
            if (s2.mode == PM_PAIRS && s2.La > s2.Lb) {
                const void *t = s2.A; s2.A = s2.B; s2.B = t;
                int64_t tl = s2.La; s2.La = s2.Lb; s2.Lb = tl;
            }
            return cuda_status(launch_chain_f32(s2, p, n_pairs, (float *)out, st));
        }
        case P_BAND: {
            PairSrc s2 = src;
            if (s2.mode == PM_PAIRS && s2.La > s2.Lb) {
                const void *t = s2.A; s2.A = s2.B; s2.B = t;
                int64_t tl = s2.La; s2.La = s2.Lb; s2.Lb = tl;
            }
            int64_t nb, need;
            band_batch(bp, n_pairs, nb, need);
            if (!ws || (int64_t)ws_bytes < need) return SIGK_ENOMEM_WS;
            for (int64_t k0 = 0; k0 < n_pairs; k0 += nb) {
                PairSrc s3 = s2;
                s3.kbase = s2.kbase + k0;
                const int64_t m = n_pairs - k0 < nb ? n_pairs - k0 : nb;
                cudaError_t e = launch_band_f32(s3, bp, m, (float *)out, ws, st, coef_of(opts));
                if (e != cudaSuccess) return cuda_status(e);
            }
            return SIGK_OK;
        }
        case P_STRIP:
            return run_strip(src, n_pairs, lam, dtype, src.La, src.Lb, opts, out, ws, ws_bytes, st);
        default:
            return cuda_status(launch_plain(src, n_pairs, lam, dtype, out, st));
    }
}


// The adjoint's path: the strip backward (f32 auto / chain, f64 chain), else
// the plain one-block-per-pair backward.
bool bwd_uses_strip(int lam, int64_t d, int dtype, int rec, int kernel) {
    // the RBF lift's chain rule runs in the plain backward only
    if (kernel != SIGK_KERNEL_LINEAR || !strip_supported(lam, d, dtype)) return false;
    if (rec == SIGK_REC_STRIP) return true;
    return dtype == SIGK_F32 ? rec != SIGK_REC_PLAIN : rec == SIGK_REC_CHAIN;
}

// The strip backward's batches: under 16 GiB, so that the 64 pairs of 4096
// points at dyadic order 1 (coefficient blocks and dk/dG, 9.7 GB) run as one
// launch, with all their strips' wavefronts in flight at once.
void bwd_strip_batch(const PairSrc &src, int64_t n, int lam, int dtype, int64_t &nb, int64_t &bytes) {
    int64_t ra, rb;
    src_rows(src, n, ra, rb);
    nb = n;
    bytes = strip_bwd_workspace_bytes(nb, src.La, src.Lb, lam, dtype, ra, rb, src.d);
    while (nb > 1 && bytes > BAND_BWD_WS_CAP) {
        nb = (nb + 1) / 2;
        bytes = strip_bwd_workspace_bytes(nb, src.La, src.Lb, lam, dtype, ra, rb, src.d);
    }
}

// The band backward's orientation: rows refine the shorter path.  For a Gram
// from sigk_gram_backward (A = X with out_si = nb, B = Y) the swap enumerates
// (Y path, X path) like sigk_gram does.
PairSrc band_orient(const PairSrc &src, int64_t n, bool &swapped) {
    PairSrc o = src;
    swapped = src.La > src.Lb;
    if (!swapped) return o;
    o.A = src.B; o.B = src.A;
    o.La = src.Lb; o.Lb = src.La;
    if (src.mode == PM_GRAM) {
        o.nb = n / src.nb;            // the X paths are now the columns
        o.out_si = 1;
        o.out_sj = src.nb;
    }
    return o;
}

bool bwd_uses_band(const PairSrc &src, int lam, int dtype, int rec, int rows, BandPlan &bp) {
    if (dtype != SIGK_F32 || rec == SIGK_REC_PLAIN || rec == SIGK_REC_STRIP) return false;
    if (src.kernel != SIGK_KERNEL_LINEAR && src.kernel != SIGK_KERNEL_RBF) return false;
    if (src.mode != PM_PAIRS && src.mode != PM_GRAM && src.mode != PM_GRAM_SYM) return false;
    const int64_t la = src.La < src.Lb ? src.La : src.Lb, lb = src.La < src.Lb ? src.Lb : src.La;
    return band_geometry(la, lb, lam, rows, bp);
}

int64_t backward_ws_bytes(const PairSrc &src, int64_t n, int lam, int dtype, int rec, int rows, int coef) {
    if (n == 0 || src.La < 2 || src.Lb < 2) return 0;
    BandPlan bp;
    if (bwd_uses_band(src, lam, dtype, rec, rows, bp)) {
        bool sw;
        const PairSrc o = band_orient(src, n, sw);
        int64_t bytes;
        band_bwd_batch(o, bp, n, BAND_BWD_WS_CAP, bytes, coef);
        return bytes;
    }
    if (rec == SIGK_REC_BAND || src.mode == PM_GRAM_SYM) return -1;
    if (src.kernel != SIGK_KERNEL_LINEAR && rec == SIGK_REC_STRIP) return -1;
    if (bwd_uses_strip(lam, src.d, dtype, rec, src.kernel)) {
        int64_t nb, need;
        bwd_strip_batch(src, n, lam, dtype, nb, need);
        return need;
    }
    int64_t grid, slot, smem;
    if (!bwd_plain_plan(n, src.La, src.Lb, src.d, lam, dtype, grid, slot, smem)) return -1;
    return grid * slot;
}

// out: when non-null, the band backward's forward sweep also writes the
// values (the caller has checked that the band form applies)
int run_backward(PairSrc src, int64_t n_pairs, int lam, int dtype, const sigk_opts *opts,
                 const void *gout, void *dX, void *dY, int64_t nX, int64_t nY, void *ws,
                 size_t ws_bytes, cudaStream_t st, void *out = nullptr) {
    const int64_t es = dtype == SIGK_F64 ? 8 : 4;
    // every path below adds into zeroed outputs (atomics), except the band
    // form, whose last kernel writes each output once (and adds on request)
    const bool acc = accumulate_of(opts);
    if (!acc && dX && cudaMemsetAsync(dX, 0, (size_t)(nX * es), st) != cudaSuccess) return SIGK_ECUDA;
    if (!acc && dY && cudaMemsetAsync(dY, 0, (size_t)(nY * es), st) != cudaSuccess) return SIGK_ECUDA;
    if (n_pairs == 0 || src.La < 2 || src.Lb < 2 || (!dX && !dY)) return SIGK_OK;
    const int rec = rec_of(opts);
    if (rec == SIGK_REC_STRIP && !strip_supported(lam, src.d, dtype)) return SIGK_EUNSUPPORTED;
    BandPlan bp;
    if (bwd_uses_band(src, lam, dtype, rec, rows_of(opts), bp)) {
        bool sw;
        const PairSrc o = band_orient(src, n_pairs, sw);
        int64_t bytes;
        const int64_t nbp = band_bwd_batch(o, bp, n_pairs, BAND_BWD_WS_CAP, bytes, coef_of(opts));
        if (!ws || (int64_t)ws_bytes < bytes) return SIGK_ENOMEM_WS;
        float *dA = (float *)(sw ? dY : dX), *dB = (float *)(sw ? dX : dY);
        return cuda_status(
            launch_band_bwd_f32(o, bp, n_pairs, nbp, (const float *)gout, dA, dB, ws, st, coef_of(opts),
                                (float *)out, acc));
    }
    // the symmetric backward exists in the band form only; the RBF lift's in
    // the band form (FP32, pairs that fit a warp) and the plain backward
    if (rec == SIGK_REC_BAND || src.mode == PM_GRAM_SYM) return SIGK_EUNSUPPORTED;
    if (src.kernel != SIGK_KERNEL_LINEAR && rec == SIGK_REC_STRIP) return SIGK_EUNSUPPORTED;
    if (bwd_uses_strip(lam, src.d, dtype, rec, src.kernel)) {
        int64_t nb, need, ra, rb;
        bwd_strip_batch(src, n_pairs, lam, dtype, nb, need);
        src_rows(src, n_pairs, ra, rb);
        if (!ws || (int64_t)ws_bytes < need) return SIGK_ENOMEM_WS;
        for (int64_t k0 = 0; k0 < n_pairs; k0 += nb) {
            PairSrc s = src;
            s.kbase = k0;
            const int64_t m = n_pairs - k0 < nb ? n_pairs - k0 : nb;
            cudaError_t e = launch_strip_bwd(s, m, lam, dtype, ws, gout, dX, dY, WAIT_CYCLES, st,
                                             src.La, src.Lb, ra, rb, coef_of(opts));
            if (e != cudaSuccess) return cuda_status(e);
        }
        return SIGK_OK;
    }
    int64_t grid, slot, smem;
    if (!bwd_plain_plan(n_pairs, src.La, src.Lb, src.d, lam, dtype, grid, slot, smem))
        return SIGK_EUNSUPPORTED;
    if (!ws || (int64_t)ws_bytes < grid * slot) return SIGK_ENOMEM_WS;
    return cuda_status(launch_bwd_plain(src, n_pairs, lam, dtype, gout, dX, dY, ws, grid, slot,
                                        smem, st));
}

// The surface's path: the band sweep's surface instance for f32 pairs whose
// shorter path fits a warp (rec AUTO, CHAIN or BAND), else the plain sweep.
// The surface in the chain schedule (inline coefficients, no coefficient
// band): f32, the linear static kernel, the explicit scheme, rec AUTO or
// CHAIN and a chained instance for the shape (d <= 16); bp is the same
// geometry as the surface unpack reads it.
bool surface_uses_chain(const PairSrc &src, int lam, int dtype, int rec, int rows, ChainPlan &cp,
                        BandPlan &bp) {
    if (dtype != SIGK_F32 || (rec != SIGK_REC_AUTO && rec != SIGK_REC_CHAIN)) return false;
    if (src.kernel != SIGK_KERNEL_LINEAR || src.scheme != SIGK_SCHEME_EXPLICIT) return false;
    const int64_t la = src.La < src.Lb ? src.La : src.Lb, lb = src.La < src.Lb ? src.Lb : src.La;
    if (!chain_geometry(la, lb, src.d, lam, cp, rows)) return false;
    bp.R = cp.R;
    bp.lam = lam;
    bp.NG = cp.R >> lam;
    bp.TperR = cp.Tper / cp.R;
    bp.NQ = cp.NQ;
    bp.NQV = cp.NQV;
    bp.vrows = cp.vtop >> lam;
    bp.slot_floats = 32LL * bp.NG * bp.NG;
    return true;
}
// Its workspace: a 256-byte header, then the nodes' band layout (TperR + 1
// slots a pair); pairs per launch under the cap.
int64_t chain_surface_bytes(const BandPlan &bp, int64_t n) {
    return 256 + (int64_t)sizeof(float) * n * (bp.TperR + 1) * bp.slot_floats;
}
void chain_surface_batch(const BandPlan &bp, int64_t n, int64_t &nb, int64_t &bytes) {
    nb = n;
    bytes = chain_surface_bytes(bp, nb);
    while (nb > 1 && bytes > STRIP_WS_CAP) {
        nb = (nb + 1) / 2;
        bytes = chain_surface_bytes(bp, nb);
    }
}

bool surface_uses_band(const PairSrc &src, int lam, int dtype, int rec, int rows, BandPlan &bp) {
    if (dtype != SIGK_F32 || rec == SIGK_REC_PLAIN || rec == SIGK_REC_STRIP) return false;
    const int64_t la = src.La < src.Lb ? src.La : src.Lb, lb = src.La < src.Lb ? src.Lb : src.La;
    return band_geometry(la, lb, lam, rows, bp);
}

}  // namespace

extern "C" {

const char *sigk_strerror(int s) {
    switch (s) {
        case SIGK_OK: return "ok";
        case SIGK_EINVAL: return "invalid argument";
        case SIGK_ENOMEM_WS: return "workspace missing or too small";
        case SIGK_ECUDA: return "CUDA error";
        case SIGK_ETIMEOUT: return "device-side wait timed out";
        case SIGK_EUNSUPPORTED: return "unsupported size or option";
        default: return "unknown status";
    }
}

const char *sigk_version(void) { return "sigk 0.1 sm_103a"; }

size_t sigk_workspace_bytes(int op, int64_t B_or_Bx, int64_t By, int64_t L, int64_t M, int64_t d,
                            int dyadic_order, int dtype, const sigk_opts *opts) {
    if (common_checks(B_or_Bx, L, M, d, dyadic_order, dtype, opts) != SIGK_OK) return 0;
    int64_t n_pairs;
    if (op == SIGK_OP_PAIRS || op == SIGK_OP_PAIRS_VARLEN || op == SIGK_OP_PAIRS_BACKWARD ||
        op == SIGK_OP_PAIRS_SURFACE)
        n_pairs = B_or_Bx;
    else if (op == SIGK_OP_GRAM || op == SIGK_OP_GRAM_BACKWARD)
        n_pairs = (By < 0) ? 0 : (opts && opts->symmetric ? B_or_Bx * (B_or_Bx + 1) / 2 : B_or_Bx * By);
    else
        return 0;
    if (n_pairs == 0 || L < 2 || M < 2) return 0;
    if (op == SIGK_OP_PAIRS_SURFACE) {
        PairSrc ss;
        memset(&ss, 0, sizeof(ss));
        set_variant(ss, opts);
        ss.mode = PM_PAIRS;
        ss.La = L; ss.Lb = M; ss.d = d;
        BandPlan bp;
        ChainPlan cp;
        int64_t nb, need;
        if (surface_uses_chain(ss, dyadic_order, dtype, rec_of(opts), rows_of(opts), cp, bp)) {
            chain_surface_batch(bp, n_pairs, nb, need);
            return (size_t)need;
        }
        if (!surface_uses_band(ss, dyadic_order, dtype, rec_of(opts), rows_of(opts), bp)) return 0;
        band_surface_batch(bp, n_pairs, nb, need);
        return (size_t)need;
    }
    if (op == SIGK_OP_PAIRS_BACKWARD || op == SIGK_OP_GRAM_BACKWARD) {
        PairSrc bs;
        memset(&bs, 0, sizeof(bs));
        set_variant(bs, opts);
        bs.mode = op == SIGK_OP_PAIRS_BACKWARD ? PM_PAIRS : PM_GRAM;
        bs.La = L; bs.Lb = M; bs.d = d;
        bs.nb = By;
        if (op == SIGK_OP_GRAM_BACKWARD && opts && opts->symmetric) {
            if (B_or_Bx != By || L != M) return 0;
            bs.mode = PM_GRAM_SYM;
            bs.nb = B_or_Bx;
        }
        const int64_t need = backward_ws_bytes(bs, n_pairs, dyadic_order, dtype, rec_of(opts), rows_of(opts),
                                               coef_of(opts));
        return need > 0 ? (size_t)need : 0;
    }
    int64_t nb, need;
    if (op == SIGK_OP_PAIRS_VARLEN) {
        if (varlen_uses_stack(d, L, dyadic_order, dtype, opts)) {
            vstack_batch(n_pairs, L, d, nb, need);
            return (size_t)need;
        }
        if (varlen_uses_band(d, L, dyadic_order, dtype, opts)) {
            vband_batch(n_pairs, L, dyadic_order, nb, need);
            return (size_t)need;
        }
        const int rec = rec_of(opts);
        if (rec == SIGK_REC_BAND) return 0;   // the call refuses it
        const bool strip = strip_supported(dyadic_order, d, dtype) &&
                           (rec == SIGK_REC_STRIP ||
                            (dtype == SIGK_F32 ? rec != SIGK_REC_PLAIN : rec == SIGK_REC_CHAIN));
        if (!strip) return 0;
        PairSrc vs;
        memset(&vs, 0, sizeof(vs));
        vs.mode = PM_VARLEN;
        vs.La = L; vs.Lb = M; vs.d = d;
        strip_batch(vs, n_pairs, L, M, dyadic_order, dtype, opts, nb, need);
        return (size_t)need;
    }
    PairSrc src;
    memset(&src, 0, sizeof(src));
    set_variant(src, opts);
    src.d = d;
    if (op == SIGK_OP_PAIRS) {
        src.mode = PM_PAIRS;
        src.La = L; src.Lb = M;
    } else if (opts && opts->symmetric) {
        src.mode = PM_GRAM_SYM;
        src.La = L; src.Lb = L;
        src.nb = B_or_Bx;
    } else {
        // the same orientation sigk_gram picks
        src.mode = PM_GRAM;
        src.La = L <= M ? L : M; src.Lb = L <= M ? M : L;
        src.nb = L <= M ? By : B_or_Bx;
    }
    BandPlan bp;
    const Path path = choose_uniform(src, n_pairs, dyadic_order, dtype, rec_of(opts), nullptr,
                                     rows_of(opts), &bp);
    if (path == P_BAND) {
        band_batch(bp, n_pairs, nb, need);
        return (size_t)need;
    }
    if (path != P_STRIP) return 0;
    strip_batch(src, n_pairs, src.La, src.Lb, dyadic_order, dtype, opts, nb, need);
    return (size_t)need;
}

int sigk_pairs(const void *X, const void *Y, int64_t B, int64_t L, int64_t M, int64_t d,
               int dyadic_order, int dtype, const sigk_opts *opts, void *out, void *ws,
               size_t ws_bytes, void *stream) {
    int s = common_checks(B, L, M, d, dyadic_order, dtype, opts);
    if (s) return s;
    if (opts && opts->symmetric) return SIGK_EINVAL;
    if (B == 0) return SIGK_OK;
    if (!X || !Y || !out) return SIGK_EINVAL;
    PairSrc src;
    memset(&src, 0, sizeof(src));
    set_variant(src, opts);
    src.mode = PM_PAIRS;
    src.A = X; src.B = Y;
    src.La = L; src.Lb = M; src.d = d;
    return run_uniform(src, B, dyadic_order, dtype, opts, out, ws, ws_bytes, (cudaStream_t)stream);
}

int sigk_gram(const void *X, const void *Y, int64_t Bx, int64_t By, int64_t L, int64_t M,
              int64_t d, int dyadic_order, int dtype, const sigk_opts *opts, void *out, void *ws,
              size_t ws_bytes, void *stream) {
    int s = common_checks(Bx, L, M, d, dyadic_order, dtype, opts);
    if (s) return s;
    if (By < 0) return SIGK_EINVAL;
    const bool sym = opts && opts->symmetric;
    if (sym && (Bx != By || L != M)) return SIGK_EINVAL;
    if (Bx == 0 || By == 0) return SIGK_OK;
    if (!X || !Y || !out) return SIGK_EINVAL;
    PairSrc src;
    memset(&src, 0, sizeof(src));
    set_variant(src, opts);
    src.d = d;
    if (sym) {
        src.mode = PM_GRAM_SYM;
        src.A = X; src.B = X;
        src.La = L; src.Lb = L;
        src.nb = Bx;
        return run_uniform(src, Bx * (Bx + 1) / 2, dyadic_order, dtype, opts, out, ws, ws_bytes,
                           (cudaStream_t)stream);
    }
    src.mode = PM_GRAM;
    if (L <= M) {
        // rows of each grid refine X: enumerate (i, j), out[i*By + j]
        src.A = X; src.B = Y;
        src.La = L; src.Lb = M;
        src.nb = By;
        src.out_si = By; src.out_sj = 1;
    } else {
        // rows refine the shorter Y paths: enumerate (j, i), out[i*By + j]
        src.A = Y; src.B = X;
        src.La = M; src.Lb = L;
        src.nb = Bx;
        src.out_si = 1; src.out_sj = By;
    }
    return run_uniform(src, Bx * By, dyadic_order, dtype, opts, out, ws, ws_bytes, (cudaStream_t)stream);
}

int sigk_pairs_varlen(const void *Xp, const int64_t *x_off, const void *Yp, const int64_t *y_off,
                      int64_t B, int64_t d, int64_t max_len, int dyadic_order, int dtype,
                      const sigk_opts *opts, void *out, void *ws, size_t ws_bytes, void *stream) {
    int s = common_checks(B, max_len < 1 ? 1 : max_len, 1, d, dyadic_order, dtype, opts);
    if (s) return s;
    if (max_len < 1) return SIGK_EINVAL;
    if (opts && opts->symmetric) return SIGK_EINVAL;
    if (B == 0) return SIGK_OK;
    if (!Xp || !Yp || !x_off || !y_off || !out) return SIGK_EINVAL;
    PairSrc src;
    memset(&src, 0, sizeof(src));
    set_variant(src, opts);
    src.mode = PM_VARLEN;
    src.A = Xp; src.B = Yp;
    src.a_off = x_off; src.b_off = y_off;
    src.La = max_len; src.Lb = max_len;
    src.d = d;
    const int rec = rec_of(opts);
    if (varlen_uses_stack(d, max_len, dyadic_order, dtype, opts)) {
        int64_t nb, need;
        vstack_batch(B, max_len, d, nb, need);
        if (!ws || (int64_t)ws_bytes < need) return SIGK_ENOMEM_WS;
        for (int64_t k0 = 0; k0 < B; k0 += nb) {
            PairSrc s2 = src;
            s2.kbase = k0;
            const int64_t m = B - k0 < nb ? B - k0 : nb;
            cudaError_t e = launch_vstack(s2, m, dyadic_order, max_len, (float *)out, ws, (cudaStream_t)stream);
            if (e != cudaSuccess) return cuda_status(e);
        }
        return SIGK_OK;
    }
    if (varlen_uses_band(d, max_len, dyadic_order, dtype, opts)) {
        int64_t nb, need;
        vband_batch(B, max_len, dyadic_order, nb, need);
        if (!ws || (int64_t)ws_bytes < need) return SIGK_ENOMEM_WS;
        for (int64_t k0 = 0; k0 < B; k0 += nb) {
            PairSrc s2 = src;
            s2.kbase = k0;
            const int64_t m = B - k0 < nb ? B - k0 : nb;
            cudaError_t e = launch_vband(s2, m, dyadic_order, max_len, (float *)out, ws, (cudaStream_t)stream);
            if (e != cudaSuccess) return cuda_status(e);
        }
        return SIGK_OK;
    }
    if (rec == SIGK_REC_BAND) return SIGK_EUNSUPPORTED;   // no band class holds the longest path
    const bool strip = strip_supported(dyadic_order, d, dtype) &&
                       (rec == SIGK_REC_STRIP ||
                        (dtype == SIGK_F32 ? rec != SIGK_REC_PLAIN : rec == SIGK_REC_CHAIN));
    if (strip)
        return run_strip(src, B, dyadic_order, dtype, max_len, max_len, opts, out, ws, ws_bytes,
                         (cudaStream_t)stream);
    if (rec == SIGK_REC_CHAIN || rec == SIGK_REC_STRIP) return SIGK_EUNSUPPORTED;
    return cuda_status(launch_plain(src, B, dyadic_order, dtype, out, (cudaStream_t)stream));
}


int sigk_pairs_surface(const void *X, const void *Y, int64_t B, int64_t L, int64_t M, int64_t d,
                       int dyadic_order, int dtype, const sigk_opts *opts, void *out, void *surf,
                       void *ws, size_t ws_bytes, void *stream) {
    int s = common_checks(B, L, M, d, dyadic_order, dtype, opts);
    if (s) return s;
    if (opts && opts->symmetric) return SIGK_EINVAL;
    if (B == 0) return SIGK_OK;
    if (!X || !Y || !out || !surf) return SIGK_EINVAL;
    const int rec = rec_of(opts);
    if (rec == SIGK_REC_STRIP) return SIGK_EUNSUPPORTED;   // the strip path has no surface
    cudaStream_t st = (cudaStream_t)stream;
    PairSrc src;
    memset(&src, 0, sizeof(src));
    set_variant(src, opts);
    src.mode = PM_PAIRS;
    src.A = X; src.B = Y;
    src.La = L; src.Lb = M; src.d = d;
    BandPlan bp;
    ChainPlan cp;
    const bool chain = surface_uses_chain(src, dyadic_order, dtype, rec, rows_of(opts), cp, bp);
    const bool band = !chain && surface_uses_band(src, dyadic_order, dtype, rec, rows_of(opts), bp);
    if (rec == SIGK_REC_BAND && !band) return SIGK_EUNSUPPORTED;
    if (chain || band) {
        int64_t nb, need;
        if (chain) chain_surface_batch(bp, B, nb, need);
        else band_surface_batch(bp, B, nb, need);
        if (!ws || (int64_t)ws_bytes < need) return SIGK_ENOMEM_WS;
    }
    // boundary nodes (row and column 0) are 1; the sweeps write the others
    if (L < 2 || M < 2) {
        cudaError_t e = launch_fill_one(surf, B * L * M, dtype, st);
        if (e != cudaSuccess) return cuda_status(e);
        return cuda_status(launch_fill_one(out, B, dtype, st));
    }
    // the unpack of the chain and band forms writes the sweep's column 0 at
    // dyadic orders >= 1 when the pairs have virtual left columns: the
    // surface's column 0 unless the rows refine Y
    const bool col0 = !(chain || band) || dyadic_order == 0 || bp.NQV == 0 || L > M;
    cudaError_t e = launch_surface_border(surf, B, L, M, dtype, st, col0);
    if (e != cudaSuccess) return cuda_status(e);
    if (!band && !chain) return cuda_status(launch_plain(src, B, dyadic_order, dtype, out, st, surf));
    // rows refine the shorter path: node (i, j) of the sweep is surface (i, j),
    // or (j, i) when X and Y swap places
    PairSrc s2 = src;
    int64_t sa = M, sb = 1;
    if (L > M) {
        s2.A = Y; s2.B = X;
        s2.La = M; s2.Lb = L;
        sa = 1; sb = M;
    }
    int64_t nb, need;
    if (chain) {
        // the chained sweep writes the nodes' band layout, the unpack the surface
        chain_surface_batch(bp, B, nb, need);
        float *sband = (float *)((unsigned char *)ws + 256);
        if ((e = cudaMemsetAsync(ws, 0, sizeof(int), st)) != cudaSuccess) return cuda_status(e);
        for (int64_t k0 = 0; k0 < B; k0 += nb) {
            PairSrc s3 = s2;
            s3.kbase = k0;
            const int64_t m = B - k0 < nb ? B - k0 : nb;
            ChainPlan c2;
            if (!chain_plan(m, s2.La, s2.Lb, d, dyadic_order, c2, rows_of(opts))) return SIGK_EUNSUPPORTED;
            if ((e = launch_chain_f32(s3, c2, m, (float *)out, st, sband)) != cudaSuccess) return cuda_status(e);
            if ((e = launch_surface_unpack(s3, bp, m, sband, (float *)surf, L * M, sa, sb, st)) != cudaSuccess)
                return cuda_status(e);
        }
        return SIGK_OK;
    }
    band_surface_batch(bp, B, nb, need);
    for (int64_t k0 = 0; k0 < B; k0 += nb) {
        PairSrc s3 = s2;
        s3.kbase = k0;
        const int64_t m = B - k0 < nb ? B - k0 : nb;
        e = launch_band_f32(s3, bp, m, (float *)out, ws, st, coef_of(opts), (float *)surf, L * M, sa, sb);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return SIGK_OK;
}

int sigk_pairs_backward(const void *grad_out, const void *X, const void *Y, int64_t B, int64_t L,
                        int64_t M, int64_t d, int dyadic_order, int dtype, const sigk_opts *opts,
                        void *dX, void *dY, void *ws, size_t ws_bytes, void *stream) {
    int s = common_checks(B, L, M, d, dyadic_order, dtype, opts);
    if (s) return s;
    if (opts && opts->symmetric) return SIGK_EINVAL;
    if (B == 0) return SIGK_OK;
    if (!grad_out || !X || !Y) return SIGK_EINVAL;
    PairSrc src;
    memset(&src, 0, sizeof(src));
    set_variant(src, opts);
    src.mode = PM_PAIRS;
    src.A = X; src.B = Y;
    src.La = L; src.Lb = M; src.d = d;
    return run_backward(src, B, dyadic_order, dtype, opts, grad_out, dX, dY, B * L * d, B * M * d,
                        ws, ws_bytes, (cudaStream_t)stream);
}

int sigk_gram_backward(const void *grad_out, const void *X, const void *Y, int64_t Bx, int64_t By,
                       int64_t L, int64_t M, int64_t d, int dyadic_order, int dtype,
                       const sigk_opts *opts, void *dX, void *dY, void *ws, size_t ws_bytes,
                       void *stream) {
    int s = common_checks(Bx, L, M, d, dyadic_order, dtype, opts);
    if (s) return s;
    if (By < 0) return SIGK_EINVAL;
    const bool sym = opts && opts->symmetric;
    if (sym && (Bx != By || L != M || dY)) return SIGK_EINVAL;
    if (Bx == 0 || By == 0) {
        const int64_t es = dtype == SIGK_F64 ? 8 : 4;
        if (accumulate_of(opts)) return SIGK_OK;
        if (dX && Bx && cudaMemsetAsync(dX, 0, (size_t)(Bx * L * d * es), (cudaStream_t)stream)) return SIGK_ECUDA;
        if (dY && By && cudaMemsetAsync(dY, 0, (size_t)(By * M * d * es), (cudaStream_t)stream)) return SIGK_ECUDA;
        return SIGK_OK;
    }
    if (!grad_out || !X || !Y) return SIGK_EINVAL;
    PairSrc src;
    memset(&src, 0, sizeof(src));
    set_variant(src, opts);
    src.mode = PM_GRAM;
    src.A = X; src.B = Y;
    src.La = L; src.Lb = M; src.d = d;
    src.nb = By;
    src.out_si = By; src.out_sj = 1;
    if (sym) {
        src.mode = PM_GRAM_SYM;
        src.B = X;
        src.nb = Bx;
        return run_backward(src, Bx * (Bx + 1) / 2, dyadic_order, dtype, opts, grad_out, dX, nullptr,
                            Bx * L * d, 0, ws, ws_bytes, (cudaStream_t)stream);
    }
    return run_backward(src, Bx * By, dyadic_order, dtype, opts, grad_out, dX, dY, Bx * L * d,
                        By * M * d, ws, ws_bytes, (cudaStream_t)stream);
}

int sigk_gram_value_and_grad(const void *grad_out, const void *X, const void *Y, int64_t Bx, int64_t By,
                             int64_t L, int64_t M, int64_t d, int dyadic_order, int dtype,
                             const sigk_opts *opts, void *out, void *dX, void *dY, void *ws, size_t ws_bytes,
                             void *stream) {
    int s = common_checks(Bx, L, M, d, dyadic_order, dtype, opts);
    if (s) return s;
    if (By < 0) return SIGK_EINVAL;
    const bool sym = opts && opts->symmetric;
    if (sym && (Bx != By || L != M || dY)) return SIGK_EINVAL;
    if (Bx == 0 || By == 0) return SIGK_OK;
    if (!grad_out || !X || !Y || !out) return SIGK_EINVAL;
    PairSrc src;
    memset(&src, 0, sizeof(src));
    set_variant(src, opts);
    src.mode = sym ? PM_GRAM_SYM : PM_GRAM;
    src.A = X; src.B = sym ? X : Y;
    src.La = L; src.Lb = M; src.d = d;
    src.nb = By;
    src.out_si = By; src.out_sj = 1;
    const int64_t n = sym ? Bx * (Bx + 1) / 2 : Bx * By;
    BandPlan bp;
    if (L < 2 || M < 2 || !bwd_uses_band(src, dyadic_order, dtype, rec_of(opts), rows_of(opts), bp))
        return SIGK_EUNSUPPORTED;
    return run_backward(src, n, dyadic_order, dtype, opts, grad_out, dX, sym ? nullptr : dY, Bx * L * d,
                        sym ? 0 : By * M * d, ws, ws_bytes, (cudaStream_t)stream, out);
}

int sigk_mmd2(const void *Kxx, const void *Kyy, const void *Kxy, int64_t m, int64_t n, int dtype,
              void *out, void *stream) {
    if (m < 2 || n < 2) return SIGK_EINVAL;
    if (dtype != SIGK_F32 && dtype != SIGK_F64) return SIGK_EINVAL;
    if (!Kxx || !Kyy || !Kxy || !out) return SIGK_EINVAL;
    return cuda_status(launch_mmd2(Kxx, Kyy, Kxy, m, n, dtype, out, (cudaStream_t)stream));
}

int sigk_mmd2_backward(const void *grad, int64_t m, int64_t n, int dtype, void *gKxx, void *gKyy,
                       void *gKxy, void *stream) {
    if (m < 2 || n < 2) return SIGK_EINVAL;
    if (dtype != SIGK_F32 && dtype != SIGK_F64) return SIGK_EINVAL;
    if (!grad) return SIGK_EINVAL;
    return cuda_status(launch_mmd2_backward(grad, m, n, dtype, gKxx, gKyy, gKxy, (cudaStream_t)stream));
}

int sigk_scale_grad(const void *grad, const void *g_in, void *g_out, int64_t n, int dtype, void *stream) {
    if (n < 0) return SIGK_EINVAL;
    if (dtype != SIGK_F32 && dtype != SIGK_F64) return SIGK_EINVAL;
    if (n == 0) return SIGK_OK;
    if (!grad || !g_in || !g_out) return SIGK_EINVAL;
    return cuda_status(launch_scale_grad(grad, g_in, g_out, n, dtype, (cudaStream_t)stream));
}

int sigk_support_reduction(const void *K, const void *alpha, void *beta, int64_t N, double gamma,
                           double lam, int iters, int dtype, void *loss, void *stream) {
    if (N < 0 || iters < 0) return SIGK_EINVAL;
    if (dtype != SIGK_F32 && dtype != SIGK_F64) return SIGK_EINVAL;
    if (!(gamma > 0.0 && gamma < 1e300) || !(lam >= 0.0 && lam < 1e300)) return SIGK_EINVAL;
    const int64_t es = dtype == SIGK_F64 ? 8 : 4;
    if (N == 0) {
        if (loss && cudaMemsetAsync(loss, 0, (size_t)(iters + 1) * es, (cudaStream_t)stream) != cudaSuccess)
            return SIGK_ECUDA;
        return SIGK_OK;
    }
    if (!K || !alpha || !beta) return SIGK_EINVAL;
    if (N > support_max_n(dtype)) return SIGK_EUNSUPPORTED;
    return cuda_status(launch_support(K, alpha, beta, N, gamma, lam, iters, dtype, loss, (cudaStream_t)stream));
}

int sigk_stream_status(void *stream, void *ws) {
    if (!ws) return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? SIGK_OK : SIGK_ECUDA;
    int st = 0;
    const int r = read_status_word(ws, (cudaStream_t)stream, &st);
    if (r != SIGK_OK) return r;
    return st == SIGK_ETIMEOUT ? SIGK_ETIMEOUT : SIGK_OK;
}

}  // extern "C"
