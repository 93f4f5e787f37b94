/*
 * FP64 CPU oracle for the signature-kernel Goursat PDE solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this library.  The CUDA
 * product path never calls it, and the two share no code: only the seeded
 * input generators serve both.
 *
 * What it computes (Salvi et al., "The Signature Kernel is the solution of a
 * Goursat PDE", Sec. 3.1):
 *   - the coarse grid P_0 is the product of the two paths' sample partitions,
 *     and P_lambda splits every coarse cell into 2^lambda x 2^lambda cells
 *     (definition of P_lambda);
 *   - on piecewise-linear paths a refined cell's increment inner product is
 *     2^(-2 lambda) times the enclosing coarse cell's <dx_p, dy_q> (remark
 *     following the scheme);
 *   - the explicit finite-difference scheme on P_lambda:
 *       k(i+1,j+1) = k(i+1,j) + k(i,j+1) - k(i,j)
 *                    + 1/2 <dx, dy> (k(i+1,j) + k(i,j+1)),
 *     with k(0,.) = k(.,0) = 1 (the boundary of the Goursat problem, Thm.
 *     "PDE");
 *   - the kernel value is the scheme's value at the terminal corner
 *     (Definition of the signature kernel: k_{x,y}(u', v')).
 * The scheme runs in row order in the paper's operation order; nothing is
 * blocked, fused or reordered.
 *
 * Two variants the paper states beside it (the *_ex entry points):
 *   - the implicit scheme of the remark after the explicit one (Sec. 3.1),
 *     which puts all four corner values into the quadrature:
 *       k(i+1,j+1) = k(i+1,j) + k(i,j+1) - k(i,j)
 *                    + 1/4 <dx, dy> (k(i,j) + k(i+1,j) + k(i,j+1) + k(i+1,j+1)),
 *     solved here for the unknown k(i+1,j+1);
 *   - a static kernel kappa on the ambient space (Sec. 2.2): the lifted PDE's
 *     coefficient on coarse cell (p,q) is the second difference
 *       kappa(x_{p+1}, y_{q+1}) - kappa(x_p, y_{q+1}) - kappa(x_{p+1}, y_q) + kappa(x_p, y_q),
 *     which for the linear kernel kappa(a,b) = <a,b> is <dx_p, dy_q>; the
 *     RBF kernel is kappa(a,b) = exp(-|a-b|^2 / (2 sigma^2)).  The lifted
 *     path is read as piecewise linear between the lifted sample points, so
 *     a refined cell again gets 2^(-2 lambda) times its coarse cell's value.  Rows of P_lambda refine x's L-1 intervals
 * (Ni = 2^lambda (L-1)) and columns refine y's M-1 intervals.
 *
 * The gradient is the exact reverse-mode derivative of that discrete scheme
 * (the paper states no gradient): with A = d k(Ni,Nj) / d k(a,b),
 *   A(a,b) = h(a,b+1) A(a,b+1) + h(a+1,b) A(a+1,b) - A(a+1,b+1),
 * h = 1 + 1/2 <dx,dy>, out-of-grid terms zero and A(Ni,Nj) = 1; then
 *   dk/dG(p,q) = 1/2 4^-lambda sum over the refined cells (a,b) of coarse
 *                cell (p,q) of A(a,b) (k(a,b-1) + k(a-1,b)),
 *   dk/d dx_p = sum_q dk/dG(p,q) dy_q,   dk/dx_i = dk/d dx_{i-1} - dk/d dx_i.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no FMA
 * contraction, so the order of roundings is the one written here).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* G row p: G[q] = <x_{p+1} - x_p, y_{q+1} - y_q>, channels in ascending order. */
static void gram_row(const double *x, int64_t p, const double *y, int64_t M, int64_t d,
                     double *Grow) {
    for (int64_t q = 0; q + 1 < M; ++q) {
        double s = 0.0;
        for (int64_t c = 0; c < d; ++c) {
            double dx = x[(p + 1) * d + c] - x[p * d + c];
            double dy = y[(q + 1) * d + c] - y[q * d + c];
            s += dx * dy;
        }
        Grow[q] = s;
    }
}

static double pow4neg(int lam) {
    double f = 1.0;
    for (int i = 0; i < lam; ++i) f *= 0.25;
    return f;
}

/* RBF static kernel exp(-|a - b|^2 / (2 sigma^2)) of two points of R^d. */
static double rbf(const double *a, const double *b, int64_t d, double sigma) {
    double s = 0.0;
    for (int64_t c = 0; c < d; ++c) {
        double t = a[c] - b[c];
        s += t * t;
    }
    return exp(-s / (2.0 * sigma * sigma));
}

/* Coarse row p of the lifted coefficient (Sec. 2.2):
 * kernel 0 (linear): <dx_p, dy_q>; kernel 1 (RBF): the second difference of
 * kappa over the four corners of coarse cell (p, q). */
static void coef_row(const double *x, int64_t p, const double *y, int64_t M, int64_t d,
                     int kernel, double sigma, double *Grow) {
    if (kernel == 0) {
        gram_row(x, p, y, M, d, Grow);
        return;
    }
    for (int64_t q = 0; q + 1 < M; ++q) {
        const double *x0 = x + p * d, *x1 = x + (p + 1) * d;
        const double *y0 = y + q * d, *y1 = y + (q + 1) * d;
        Grow[q] = rbf(x1, y1, d, sigma) - rbf(x0, y1, d, sigma) - rbf(x1, y0, d, sigma)
                  + rbf(x0, y0, d, sigma);
    }
}

/* One step of the scheme: k(i+1,j+1) from k10 = k(i+1,j), k01 = k(i,j+1),
 * k00 = k(i,j) and the refined coefficient inc.
 * scheme 0: the explicit scheme; scheme 1: the implicit one, solved for
 * k(i+1,j+1) (it appears on both sides with weight 1 and inc/4). */
static double scheme_step(int scheme, double k10, double k01, double k00, double inc) {
    if (scheme == 0) return k10 + k01 - k00 + 0.5 * inc * (k10 + k01);
    return (k10 + k01 - k00 + 0.25 * inc * (k00 + k10 + k01)) / (1.0 - 0.25 * inc);
}

/* k_{x,y} on P_lambda with a choice of scheme (0 explicit, 1 implicit) and
 * static kernel (0 linear, 1 RBF of bandwidth sigma). */
double oracle_sigk_pair_ex(const double *x, int64_t L, const double *y, int64_t M, int64_t d,
                           int lam, int scheme, int kernel, double sigma) {
    if (L < 2 || M < 2) return 1.0;
    const int64_t s = (int64_t)1 << lam;
    const int64_t Ni = s * (L - 1), Nj = s * (M - 1);
    const double f = pow4neg(lam);
    double *prev = (double *)malloc(sizeof(double) * (size_t)(Nj + 1));
    double *cur = (double *)malloc(sizeof(double) * (size_t)(Nj + 1));
    double *Grow = (double *)malloc(sizeof(double) * (size_t)(M - 1));
    for (int64_t b = 0; b <= Nj; ++b) prev[b] = 1.0;          /* k(0, .) = 1 */
    int64_t pcur = -1;
    for (int64_t a = 1; a <= Ni; ++a) {
        int64_t p = (a - 1) >> lam;
        if (p != pcur) { coef_row(x, p, y, M, d, kernel, sigma, Grow); pcur = p; }
        cur[0] = 1.0;                                          /* k(., 0) = 1 */
        for (int64_t b = 1; b <= Nj; ++b)
            cur[b] = scheme_step(scheme, cur[b - 1], prev[b], prev[b - 1], f * Grow[(b - 1) >> lam]);
        double *t = prev; prev = cur; cur = t;
    }
    double k = prev[Nj];
    free(prev); free(cur); free(Grow);
    return k;
}

/* The solution surface on the sample grid P_0 (Sec. 3.1: k(s_i, t_j) at the
 * nodes of the coarse grid, the quantity of Fig. "error"): surf[i * M + j] =
 * the scheme's value at refined node (2^lambda i, 2^lambda j), i < L, j < M;
 * row 0 and column 0 are the boundary value 1.  Returns k = surf[L-1][M-1]. */
double oracle_sigk_pair_surface(const double *x, int64_t L, const double *y, int64_t M, int64_t d,
                                int lam, int scheme, int kernel, double sigma, double *surf) {
    for (int64_t j = 0; j < M; ++j) surf[j] = 1.0;
    for (int64_t i = 0; i < L; ++i) surf[i * M] = 1.0;
    if (L < 2 || M < 2) return 1.0;
    const int64_t s = (int64_t)1 << lam;
    const int64_t Ni = s * (L - 1), Nj = s * (M - 1);
    const double f = pow4neg(lam);
    double *prev = (double *)malloc(sizeof(double) * (size_t)(Nj + 1));
    double *cur = (double *)malloc(sizeof(double) * (size_t)(Nj + 1));
    double *Grow = (double *)malloc(sizeof(double) * (size_t)(M - 1));
    for (int64_t b = 0; b <= Nj; ++b) prev[b] = 1.0;
    int64_t pcur = -1;
    for (int64_t a = 1; a <= Ni; ++a) {
        int64_t p = (a - 1) >> lam;
        if (p != pcur) { coef_row(x, p, y, M, d, kernel, sigma, Grow); pcur = p; }
        cur[0] = 1.0;
        for (int64_t b = 1; b <= Nj; ++b)
            cur[b] = scheme_step(scheme, cur[b - 1], prev[b], prev[b - 1], f * Grow[(b - 1) >> lam]);
        if (a % s == 0)
            for (int64_t j = 1; j < M; ++j) surf[(a / s) * M + j] = cur[j * s];
        double *t = prev; prev = cur; cur = t;
    }
    double k = prev[Nj];
    free(prev); free(cur); free(Grow);
    return k;
}

void oracle_sigk_pairs_surface(const double *X, const double *Y, int64_t B, int64_t L, int64_t M,
                               int64_t d, int lam, int scheme, int kernel, double sigma,
                               double *out, double *surf) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < B; ++b)
        out[b] = oracle_sigk_pair_surface(X + b * L * d, L, Y + b * M * d, M, d, lam, scheme, kernel,
                                          sigma, surf + b * L * M);
}

void oracle_sigk_pairs_ex(const double *X, const double *Y, int64_t B, int64_t L, int64_t M,
                          int64_t d, int lam, int scheme, int kernel, double sigma, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < B; ++b)
        out[b] = oracle_sigk_pair_ex(X + b * L * d, L, Y + b * M * d, M, d, lam, scheme, kernel, sigma);
}

void oracle_sigk_gram_ex(const double *X, const double *Y, int64_t Bx, int64_t By, int64_t L,
                         int64_t M, int64_t d, int lam, int scheme, int kernel, double sigma,
                         double *out) {
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int64_t i = 0; i < Bx; ++i)
        for (int64_t j = 0; j < By; ++j)
            out[i * By + j] = oracle_sigk_pair_ex(X + i * L * d, L, Y + j * M * d, M, d, lam,
                                                  scheme, kernel, sigma);
}

void oracle_sigk_pairs_varlen_ex(const double *Xp, const int64_t *x_off, const double *Yp,
                                 const int64_t *y_off, int64_t B, int64_t d, int lam, int scheme,
                                 int kernel, double sigma, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < B; ++b)
        out[b] = oracle_sigk_pair_ex(Xp + x_off[b] * d, x_off[b + 1] - x_off[b],
                                     Yp + y_off[b] * d, y_off[b + 1] - y_off[b], d, lam, scheme,
                                     kernel, sigma);
}

/* One kernel value k_{x,y} on P_lambda. x: [L,d], y: [M,d] row-major. */
double oracle_sigk_pair(const double *x, int64_t L, const double *y, int64_t M, int64_t d,
                        int lam) {
    if (L < 2 || M < 2) return 1.0;
    const int64_t s = (int64_t)1 << lam;
    const int64_t Ni = s * (L - 1), Nj = s * (M - 1);
    const double f = pow4neg(lam);
    double *prev = (double *)malloc(sizeof(double) * (size_t)(Nj + 1));
    double *cur = (double *)malloc(sizeof(double) * (size_t)(Nj + 1));
    double *Grow = (double *)malloc(sizeof(double) * (size_t)(M - 1));
    for (int64_t b = 0; b <= Nj; ++b) prev[b] = 1.0;          /* k(0, .) = 1 */
    int64_t pcur = -1;
    for (int64_t a = 1; a <= Ni; ++a) {
        int64_t p = (a - 1) >> lam;
        if (p != pcur) { gram_row(x, p, y, M, d, Grow); pcur = p; }
        cur[0] = 1.0;                                          /* k(., 0) = 1 */
        for (int64_t b = 1; b <= Nj; ++b) {
            double inc = f * Grow[(b - 1) >> lam];             /* refined <dx, dy> */
            cur[b] = cur[b - 1] + prev[b] - prev[b - 1] + 0.5 * inc * (cur[b - 1] + prev[b]);
        }
        double *t = prev; prev = cur; cur = t;
    }
    double k = prev[Nj];
    free(prev); free(cur); free(Grow);
    return k;
}

/* out[b] = k(X_b, Y_b); X: [B,L,d], Y: [B,M,d]. */
void oracle_sigk_pairs(const double *X, const double *Y, int64_t B, int64_t L, int64_t M,
                       int64_t d, int lam, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < B; ++b)
        out[b] = oracle_sigk_pair(X + b * L * d, L, Y + b * M * d, M, d, lam);
}

/* out[i*By + j] = k(X_i, Y_j). */
void oracle_sigk_gram(const double *X, const double *Y, int64_t Bx, int64_t By, int64_t L,
                      int64_t M, int64_t d, int lam, double *out) {
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int64_t i = 0; i < Bx; ++i)
        for (int64_t j = 0; j < By; ++j)
            out[i * By + j] = oracle_sigk_pair(X + i * L * d, L, Y + j * M * d, M, d, lam);
}

/* Pairs of uneven lengths: pair b uses rows x_off[b]..x_off[b+1]-1 of Xp. */
void oracle_sigk_pairs_varlen(const double *Xp, const int64_t *x_off, const double *Yp,
                              const int64_t *y_off, int64_t B, int64_t d, int lam,
                              double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < B; ++b)
        out[b] = oracle_sigk_pair(Xp + x_off[b] * d, x_off[b + 1] - x_off[b],
                                  Yp + y_off[b] * d, y_off[b + 1] - y_off[b], d, lam);
}

/* gout * d kappa(a, b) / d a added into da (RBF: -kappa (a - b) / sigma^2) and
 * gout * d kappa(a, b) / d b into db, either may be NULL. */
static void rbf_grad(const double *a, const double *b, int64_t d, double sigma, double gout,
                     double *da, double *db) {
    const double k = rbf(a, b, d, sigma);
    for (int64_t c = 0; c < d; ++c) {
        const double t = gout * k * (a[c] - b[c]) / (sigma * sigma);
        if (da) da[c] -= t;
        if (db) db[c] += t;
    }
}

/*
 * Reverse-mode derivative of one kernel value (scheme and static kernel as in
 * oracle_sigk_pair_ex).  Adds gout * dk/dx into dx ([L,d], may be NULL) and
 * gout * dk/dy into dy ([M,d], may be NULL).  Returns k.  Keeps the whole
 * (Ni+1) x (Nj+1) grid: meant for test sizes.
 *
 * With A(a,b) = dk/dk(a,b): each k(a,b) enters k(a,b+1) and k(a+1,b) with
 * weight h = d k(a+1,b+1) / d k(a+1,b) (explicit: 1 + g/2; implicit, from
 * k (1 - g/4) = k10 + k01 - k00 + g/4 (k00 + k10 + k01): (1 + g/4) / (1 - g/4))
 * and k(a+1,b+1) with weight -1 (both schemes); a cell's own coefficient g
 * enters with dk(a,b)/dg = (k10 + k01)/2 (explicit) or
 * (k00 + k10 + k01 + k(a,b)) / (4 (1 - g/4)) (implicit).
 */
double oracle_sigk_pair_grad_ex(const double *x, int64_t L, const double *y, int64_t M,
                                int64_t d, int lam, int scheme, int kernel, double sigma,
                                double gout, double *dx, double *dy) {
    if (L < 2 || M < 2) return 1.0;
    const int64_t s = (int64_t)1 << lam;
    const int64_t Ni = s * (L - 1), Nj = s * (M - 1), W = Nj + 1;
    const double f = pow4neg(lam);
    double *G = (double *)malloc(sizeof(double) * (size_t)((L - 1) * (M - 1)));
    double *K = (double *)malloc(sizeof(double) * (size_t)((Ni + 1) * W));
    double *A = (double *)calloc((size_t)((Ni + 2) * (W + 1)), sizeof(double));
    double *Gb = (double *)calloc((size_t)((L - 1) * (M - 1)), sizeof(double));
    for (int64_t p = 0; p + 1 < L; ++p) coef_row(x, p, y, M, d, kernel, sigma, G + p * (M - 1));
#define Gc(a, b) G[(((a) - 1) >> lam) * (M - 1) + (((b) - 1) >> lam)]
#define Hc(a, b) (scheme == 0 ? 1.0 + 0.5 * f * Gc(a, b) \
                              : (1.0 + 0.25 * f * Gc(a, b)) / (1.0 - 0.25 * f * Gc(a, b)))
    for (int64_t b = 0; b <= Nj; ++b) K[b] = 1.0;
    for (int64_t a = 1; a <= Ni; ++a) {
        K[a * W] = 1.0;
        for (int64_t b = 1; b <= Nj; ++b)
            K[a * W + b] = scheme_step(scheme, K[a * W + b - 1], K[(a - 1) * W + b],
                                       K[(a - 1) * W + b - 1], f * Gc(a, b));
    }
    double k = K[Ni * W + Nj];
    /* adjoint grid, stride W+1 so that A(a, Nj+1) and A(Ni+1, b) exist and are 0 */
    const int64_t WA = W + 1;
    for (int64_t a = Ni; a >= 1; --a) {
        for (int64_t b = Nj; b >= 1; --b) {
            double v;
            if (a == Ni && b == Nj) {
                v = 1.0;
            } else {
                v = 0.0;
                if (b < Nj) v += Hc(a, b + 1) * A[a * WA + b + 1];
                if (a < Ni) v += Hc(a + 1, b) * A[(a + 1) * WA + b];
                if (a < Ni && b < Nj) v -= A[(a + 1) * WA + b + 1];
            }
            A[a * WA + b] = v;
            const double k10 = K[a * W + b - 1], k01 = K[(a - 1) * W + b];
            double dkdg;
            if (scheme == 0) {
                dkdg = 0.5 * (k10 + k01);
            } else {
                const double k00 = K[(a - 1) * W + b - 1], k11 = K[a * W + b];
                dkdg = (k00 + k10 + k01 + k11) / (4.0 * (1.0 - 0.25 * f * Gc(a, b)));
            }
            Gb[((a - 1) >> lam) * (M - 1) + ((b - 1) >> lam)] += f * v * dkdg;
        }
    }
#undef Hc
#undef Gc
    /* chain rule from the coarse coefficients to the points */
    for (int64_t p = 0; p + 1 < L; ++p) {
        for (int64_t q = 0; q + 1 < M; ++q) {
            double g = gout * Gb[p * (M - 1) + q];
            if (kernel == 0) {
                /* G(p,q) = sum_c dx_{p,c} dy_{q,c} */
                for (int64_t c = 0; c < d; ++c) {
                    double ddx = x[(p + 1) * d + c] - x[p * d + c];
                    double ddy = y[(q + 1) * d + c] - y[q * d + c];
                    if (dx) { dx[(p + 1) * d + c] += g * ddy; dx[p * d + c] -= g * ddy; }
                    if (dy) { dy[(q + 1) * d + c] += g * ddx; dy[q * d + c] -= g * ddx; }
                }
            } else {
                /* the four corners of the second difference, with their signs */
                const double *x0 = x + p * d, *x1 = x + (p + 1) * d;
                const double *y0 = y + q * d, *y1 = y + (q + 1) * d;
                rbf_grad(x1, y1, d, sigma, g, dx ? dx + (p + 1) * d : NULL, dy ? dy + (q + 1) * d : NULL);
                rbf_grad(x0, y1, d, sigma, -g, dx ? dx + p * d : NULL, dy ? dy + (q + 1) * d : NULL);
                rbf_grad(x1, y0, d, sigma, -g, dx ? dx + (p + 1) * d : NULL, dy ? dy + q * d : NULL);
                rbf_grad(x0, y0, d, sigma, g, dx ? dx + p * d : NULL, dy ? dy + q * d : NULL);
            }
        }
    }
    free(G); free(K); free(A); free(Gb);
    return k;
}

/* The explicit scheme with the linear kernel (the paper's main scheme). */
double oracle_sigk_pair_grad(const double *x, int64_t L, const double *y, int64_t M, int64_t d,
                             int lam, double gout, double *dx, double *dy) {
    return oracle_sigk_pair_grad_ex(x, L, y, M, d, lam, 0, 0, 1.0, gout, dx, dy);
}

/* Pairs: dX[b] = gout[b] dk_b/dX_b, dY likewise (either may be NULL). */
void oracle_sigk_pairs_grad_ex(const double *X, const double *Y, int64_t B, int64_t L, int64_t M,
                               int64_t d, int lam, int scheme, int kernel, double sigma,
                               const double *gout, double *dX, double *dY) {
    if (dX) memset(dX, 0, sizeof(double) * (size_t)(B * L * d));
    if (dY) memset(dY, 0, sizeof(double) * (size_t)(B * M * d));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < B; ++b)
        oracle_sigk_pair_grad_ex(X + b * L * d, L, Y + b * M * d, M, d, lam, scheme, kernel, sigma,
                                 gout[b], dX ? dX + b * L * d : NULL, dY ? dY + b * M * d : NULL);
}

void oracle_sigk_pairs_grad(const double *X, const double *Y, int64_t B, int64_t L, int64_t M,
                            int64_t d, int lam, const double *gout, double *dX, double *dY) {
    oracle_sigk_pairs_grad_ex(X, Y, B, L, M, d, lam, 0, 0, 1.0, gout, dX, dY);
}

/* Gram: dX[i] = sum_j gout[i,j] dk(X_i,Y_j)/dX_i; dY[j] = sum_i gout[i,j] dk/dY_j. */
void oracle_sigk_gram_grad_ex(const double *X, const double *Y, int64_t Bx, int64_t By, int64_t L,
                              int64_t M, int64_t d, int lam, int scheme, int kernel, double sigma,
                              const double *gout, double *dX, double *dY) {
    if (dX) {
        memset(dX, 0, sizeof(double) * (size_t)(Bx * L * d));
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t i = 0; i < Bx; ++i)
            for (int64_t j = 0; j < By; ++j)
                oracle_sigk_pair_grad_ex(X + i * L * d, L, Y + j * M * d, M, d, lam, scheme, kernel,
                                         sigma, gout[i * By + j], dX + i * L * d, NULL);
    }
    if (dY) {
        memset(dY, 0, sizeof(double) * (size_t)(By * M * d));
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t j = 0; j < By; ++j)
            for (int64_t i = 0; i < Bx; ++i)
                oracle_sigk_pair_grad_ex(X + i * L * d, L, Y + j * M * d, M, d, lam, scheme, kernel,
                                         sigma, gout[i * By + j], NULL, dY + j * M * d);
    }
}

void oracle_sigk_gram_grad(const double *X, const double *Y, int64_t Bx, int64_t By, int64_t L,
                           int64_t M, int64_t d, int lam, const double *gout, double *dX,
                           double *dY) {
    oracle_sigk_gram_grad_ex(X, Y, Bx, By, L, M, d, lam, 0, 0, 1.0, gout, dX, dY);
}

/* Number of OpenMP threads the oracle uses (1 without OpenMP). */
int oracle_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
