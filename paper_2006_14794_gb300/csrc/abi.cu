// libsigk C ABI: argument checks, kernel choice and launches.  No call here
// allocates memory; no C++ exception crosses the interface.
#include <stdio.h>
#include <string.h>

#include "sigk_internal.cuh"

using namespace sigk;

namespace {

bool opts_ok(const sigk_opts *o) {
    if (!o) return true;
    if (o->rec < SIGK_REC_AUTO || o->rec > SIGK_REC_PLAIN) return false;
    if (o->symmetric != 0 && o->symmetric != 1) return false;
    for (int i = 0; i < 6; ++i)
        if (o->reserved[i] != 0) return false;
    return true;
}

int rec_of(const sigk_opts *o) { return o ? o->rec : SIGK_REC_AUTO; }

int common_checks(int64_t B, int64_t L, int64_t M, int64_t d, int lam, int dtype,
                  const sigk_opts *opts) {
    if (B < 0 || L < 1 || M < 1 || d < 1) return SIGK_EINVAL;
    if (dtype != SIGK_F32 && dtype != SIGK_F64) return SIGK_EINVAL;
    if (!opts_ok(opts)) return SIGK_EINVAL;
    if (lam < 0) return SIGK_EINVAL;
    if (lam > 8) return SIGK_EUNSUPPORTED;
    return SIGK_OK;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SIGK_OK;
    if (e == cudaErrorInvalidConfiguration) return SIGK_EUNSUPPORTED;
    return SIGK_ECUDA;
}

// Solve n_pairs pairs described by `src` (uniform lengths La x Lb).
int run_uniform(PairSrc src, int64_t n_pairs, int lam, int dtype, int rec, void *out,
                cudaStream_t st) {
    if (n_pairs == 0) return SIGK_OK;
    if (src.La < 2 || src.Lb < 2) return cuda_status(launch_fill_one(out, n_pairs, dtype, st));
    if (dtype == SIGK_F32 && rec != SIGK_REC_PLAIN) {
        // the chained kernel wants the shorter path on the rows (k(x,y) = k(y,x));
        // sigk_gram already orders its batches, pairs are swapped here
        PairSrc s2 = src;
        if (s2.mode == PM_PAIRS && s2.La > s2.Lb) {
            const void *t = s2.A; s2.A = s2.B; s2.B = t;
            int64_t tl = s2.La; s2.La = s2.Lb; s2.Lb = tl;
        }
        ChainPlan p;
        if (chain_plan(n_pairs, s2.La, s2.Lb, s2.d, lam, p))
            return cuda_status(launch_chain_f32(s2, p, n_pairs, (float *)out, st));
        if (rec == SIGK_REC_CHAIN) return SIGK_EUNSUPPORTED;
    }
    return cuda_status(launch_plain(src, n_pairs, lam, dtype, out, st));
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
    (void)op; (void)B_or_Bx; (void)By; (void)L; (void)M; (void)d; (void)dyadic_order;
    (void)dtype; (void)opts;
    return 0;
}

int sigk_pairs(const void *X, const void *Y, int64_t B, int64_t L, int64_t M, int64_t d,
               int dyadic_order, int dtype, const sigk_opts *opts, void *out, void *ws,
               size_t ws_bytes, void *stream) {
    (void)ws; (void)ws_bytes;
    int s = common_checks(B, L, M, d, dyadic_order, dtype, opts);
    if (s) return s;
    if (opts && opts->symmetric) return SIGK_EINVAL;
    if (B == 0) return SIGK_OK;
    if (!X || !Y || !out) return SIGK_EINVAL;
    PairSrc src;
    memset(&src, 0, sizeof(src));
    src.mode = PM_PAIRS;
    src.A = X; src.B = Y;
    src.La = L; src.Lb = M; src.d = d;
    return run_uniform(src, B, dyadic_order, dtype, rec_of(opts), out, (cudaStream_t)stream);
}

int sigk_gram(const void *X, const void *Y, int64_t Bx, int64_t By, int64_t L, int64_t M,
              int64_t d, int dyadic_order, int dtype, const sigk_opts *opts, void *out, void *ws,
              size_t ws_bytes, void *stream) {
    (void)ws; (void)ws_bytes;
    int s = common_checks(Bx, L, M, d, dyadic_order, dtype, opts);
    if (s) return s;
    if (By < 0) return SIGK_EINVAL;
    const bool sym = opts && opts->symmetric;
    if (sym && (Bx != By || L != M)) return SIGK_EINVAL;
    if (Bx == 0 || By == 0) return SIGK_OK;
    if (!X || !Y || !out) return SIGK_EINVAL;
    PairSrc src;
    memset(&src, 0, sizeof(src));
    src.d = d;
    if (sym) {
        src.mode = PM_GRAM_SYM;
        src.A = X; src.B = X;
        src.La = L; src.Lb = L;
        src.nb = Bx;
        return run_uniform(src, Bx * (Bx + 1) / 2, dyadic_order, dtype, rec_of(opts), out,
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
    return run_uniform(src, Bx * By, dyadic_order, dtype, rec_of(opts), out, (cudaStream_t)stream);
}

int sigk_pairs_varlen(const void *Xp, const int64_t *x_off, const void *Yp, const int64_t *y_off,
                      int64_t B, int64_t d, int64_t max_len, int dyadic_order, int dtype,
                      const sigk_opts *opts, void *out, void *ws, size_t ws_bytes, void *stream) {
    (void)ws; (void)ws_bytes;
    int s = common_checks(B, max_len < 1 ? 1 : max_len, 1, d, dyadic_order, dtype, opts);
    if (s) return s;
    if (max_len < 1) return SIGK_EINVAL;
    if (opts && opts->symmetric) return SIGK_EINVAL;
    if (B == 0) return SIGK_OK;
    if (!Xp || !Yp || !x_off || !y_off || !out) return SIGK_EINVAL;
    if (opts && opts->rec == SIGK_REC_CHAIN) return SIGK_EUNSUPPORTED;
    PairSrc src;
    memset(&src, 0, sizeof(src));
    src.mode = PM_VARLEN;
    src.A = Xp; src.B = Yp;
    src.a_off = x_off; src.b_off = y_off;
    src.La = max_len; src.Lb = max_len;
    src.d = d;
    return cuda_status(launch_plain(src, B, dyadic_order, dtype, out, (cudaStream_t)stream));
}

int sigk_pairs_backward(const void *grad_out, const void *X, const void *Y, int64_t B, int64_t L,
                        int64_t M, int64_t d, int dyadic_order, int dtype, const sigk_opts *opts,
                        void *dX, void *dY, void *ws, size_t ws_bytes, void *stream) {
    (void)grad_out; (void)X; (void)Y; (void)B; (void)L; (void)M; (void)d; (void)dyadic_order;
    (void)dtype; (void)opts; (void)dX; (void)dY; (void)ws; (void)ws_bytes; (void)stream;
    return SIGK_EUNSUPPORTED;
}

int sigk_gram_backward(const void *grad_out, const void *X, const void *Y, int64_t Bx, int64_t By,
                       int64_t L, int64_t M, int64_t d, int dyadic_order, int dtype,
                       const sigk_opts *opts, void *dX, void *dY, void *ws, size_t ws_bytes,
                       void *stream) {
    (void)grad_out; (void)X; (void)Y; (void)Bx; (void)By; (void)L; (void)M; (void)d;
    (void)dyadic_order; (void)dtype; (void)opts; (void)dX; (void)dY; (void)ws; (void)ws_bytes;
    (void)stream;
    return SIGK_EUNSUPPORTED;
}

int sigk_mmd2(const void *Kxx, const void *Kyy, const void *Kxy, int64_t m, int64_t n, int dtype,
              void *out, void *stream) {
    (void)Kxx; (void)Kyy; (void)Kxy; (void)m; (void)n; (void)dtype; (void)out; (void)stream;
    return SIGK_EUNSUPPORTED;
}

int sigk_mmd2_backward(const void *grad, int64_t m, int64_t n, int dtype, void *gKxx, void *gKyy,
                       void *gKxy, void *stream) {
    (void)grad; (void)m; (void)n; (void)dtype; (void)gKxx; (void)gKyy; (void)gKxy; (void)stream;
    return SIGK_EUNSUPPORTED;
}

int sigk_stream_status(void *stream, void *ws) {
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return SIGK_ECUDA;
    (void)ws;
    return SIGK_OK;
}

}  // extern "C"
