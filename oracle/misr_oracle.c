/*
 * FP64 CPU oracle: plain loops written from the paper's definitions.
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline of the benchmark).
 * See misr_oracle.h for the problem statement and the readings taken.
 *
 * Summation order is fixed: every reduction is a sequential sum per image row followed by
 * a sequential sum over rows, so results do not depend on the OpenMP thread count.
 */
#include "misr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int HRH(const orc_problem *P) { return P->f * P->h; }
static int HRW(const orc_problem *P) { return P->f * P->w; }

/* Set up a problem.  shifts_lr holds K pairs (dx, dy) in LR pixels (dx along columns).
 * Reading: the detector shift moves the sampling grid by t = f * s HR pixels (every shift
 * pattern of the paper, Sec. 3.2 and Sec. 4.1, is a multiple of 1/f LR px, so t is an integer
 * there); a non-integer t = n + a is modelled by bilinear interpolation between HR pixels
 * n and n + 1.  Returns 0, or a negative code for an invalid argument. */
int orc_init(orc_problem *P, int h, int w, int K, int f, const double *shifts_lr,
             const double *psf, int psf_size, double lambda, double btv_alpha, int btv_w,
             double eps, int reg) {
    memset(P, 0, sizeof(*P));
    if (h <= 0 || w <= 0 || f <= 0 || K <= 0 || K > ORC_MAXK) return -1;
    if (psf_size <= 0 || psf_size % 2 == 0 || psf_size > ORC_MAXPSF) return -2;
    if (btv_w < 1 || eps < 0 || lambda < 0) return -3;
    P->h = h; P->w = w; P->K = K; P->f = f;
    for (int k = 0; k < K; ++k) {
        double tx = f * shifts_lr[2 * k], ty = f * shifts_lr[2 * k + 1];
        if (!(fabs(tx) < 1e6 && fabs(ty) < 1e6)) return -4;
        double rx = floor(tx + 0.5), ry = floor(ty + 0.5);
        if (fabs(tx - rx) <= 1e-9) tx = rx;   /* integer shifts stay exact translations */
        if (fabs(ty - ry) <= 1e-9) ty = ry;
        P->tx[k] = (int)floor(tx);
        P->ty[k] = (int)floor(ty);
        P->fx[k] = tx - floor(tx);
        P->fy[k] = ty - floor(ty);
    }
    double s = 0;
    for (int i = 0; i < psf_size * psf_size; ++i) s += psf[i];
    if (!(s > 0)) return -5;
    P->psf_size = psf_size;
    for (int i = 0; i < psf_size * psf_size; ++i) P->psf[i] = psf[i] / s;
    P->lambda = lambda; P->btv_alpha = btv_alpha; P->btv_w = btv_w; P->eps = eps;
    P->reg = reg;
    return 0;
}

/* Data norm (reading: the paper's experiments use the L1 norm, Sec. 3.1; it is smoothed
 * like the prior's |.|, psi_d(t) = sqrt(t^2 + eps_d^2) - eps_d).  Returns 0, or -1 for an
 * unknown norm or eps_d <= 0 with the L1 norm. */
int orc_set_data_norm(orc_problem *P, int norm, double data_eps) {
    if (norm != ORC_NORM_L2 && norm != ORC_NORM_L1) return -1;
    if (norm == ORC_NORM_L1 && !(data_eps > 0)) return -1;
    P->data_norm = norm;
    P->data_eps = data_eps;
    return 0;
}

/* Decimation (reading: D samples phase 0 unless the binning of the synthetic study, Sec.
 * 4.1.1, is asked for).  Returns 0, or -1 for an unknown mode. */
int orc_set_decimation(orc_problem *P, int mode) {
    if (mode != ORC_DECIM_POINT && mode != ORC_DECIM_BIN) return -1;
    P->decim = mode;
    return 0;
}

/* FP32 storage of the SCG state as a perturbation model: with it on, orc_scg rounds x, r and
 * p to the nearest FP32 value after every update; every other operation stays FP64.  It
 * measures how far an implementation that keeps its state in FP32 must drift from the FP64
 * run.  Returns 0, or -1 for a value other than 0 or 1. */
int orc_set_state_f32(orc_problem *P, int on) {
    if (on != 0 && on != 1) return -1;
    P->state_f32 = on;
    return 0;
}

static void round_f32(double *v, long n) {
    for (long i = 0; i < n; ++i) v[i] = (double)(float)v[i];
}

/* (M_k x)(u, v) = sum_{p, q in {0, 1}} wy_p wx_q x(u + ty_k + p, v + tx_k + q), x zero outside
 * the grid, wy = (1 - fy_k, fy_k), wx = (1 - fx_k, fx_k): a translation for integer shifts,
 * bilinear interpolation otherwise.  The value at one pixel of B's input: */
static double motion_at(const orc_problem *P, int k, const double *x, int bu, int bv) {
    const int H = HRH(P), W = HRW(P);
    const double wy[2] = {1.0 - P->fy[k], P->fy[k]}, wx[2] = {1.0 - P->fx[k], P->fx[k]};
    double s = 0.0;
    for (int p = 0; p < 2; ++p) {
        const int u = bu + P->ty[k] + p;
        if (wy[p] == 0.0 || u < 0 || u >= H) continue;
        for (int q = 0; q < 2; ++q) {
            const int v = bv + P->tx[k] + q;
            if (wx[q] == 0.0 || v < 0 || v >= W) continue;
            s += wy[p] * wx[q] * x[(long)u * W + v];
        }
    }
    return s;
}

/* The adjoint of motion_at: pixel (bu, bv) of B's input scatters `val` back to x. */
static void motion_at_adj(const orc_problem *P, int k, double val, int bu, int bv, double *out) {
    const int H = HRH(P), W = HRW(P);
    const double wy[2] = {1.0 - P->fy[k], P->fy[k]}, wx[2] = {1.0 - P->fx[k], P->fx[k]};
    for (int p = 0; p < 2; ++p) {
        const int u = bu + P->ty[k] + p;
        if (wy[p] == 0.0 || u < 0 || u >= H) continue;
        for (int q = 0; q < 2; ++q) {
            const int v = bv + P->tx[k] + q;
            if (wx[q] == 0.0 || v < 0 || v >= W) continue;
            out[(long)u * W + v] += wy[p] * wx[q] * val;
        }
    }
}

/* (A_k x)(i, j) = (D B M_k x)(i, j)                                            Eq. 1
 *   (M_k x)(u, v) as above (x(u + ty_k, v + tx_k) for integer shifts), zero outside the grid;
 *   (B z)(u, v)   = sum_{a,b} h(a, b) z(u - a, v - b), z zero outside the grid;
 *   (D w)(i, j)   = w(f i, f j), or with binning
 *   (D w)(i, j)   = (1 / f^2) sum_{a', b' = 0}^{f-1} w(f i + a', f j + b').              */
void orc_forward(const orc_problem *P, int k, const double *x, double *out) {
    const int H = HRH(P), W = HRW(P), S = P->psf_size, R = S / 2, f = P->f;
    const int ty = P->ty[k], tx = P->tx[k];
    const int nb = P->decim == ORC_DECIM_BIN ? f : 1;   /* block side averaged by D */
    const double wd = 1.0 / ((double)nb * nb);
    const int frac = P->fy[k] != 0.0 || P->fx[k] != 0.0;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < P->h; ++i) {
        for (int j = 0; j < P->w; ++j) {
            double acc = 0.0;
            for (int a2 = 0; a2 < nb; ++a2) {
                for (int b2 = 0; b2 < nb; ++b2) {
                    const int cu = f * i + a2, cv = f * j + b2;   /* pixel of B's output */
                    double w = 0.0;
                    for (int a = -R; a <= R; ++a) {
                        int bu = cu - a;                 /* pixel of B's input, M_k x */
                        if (bu < 0 || bu >= H) continue;
                        for (int b = -R; b <= R; ++b) {
                            int bv = cv - b;
                            if (bv < 0 || bv >= W) continue;
                            if (frac) {
                                w += P->psf[(a + R) * S + (b + R)] * motion_at(P, k, x, bu, bv);
                                continue;
                            }
                            int u = bu + ty, v = bv + tx;   /* pixel of x read by M_k */
                            if (u < 0 || u >= H || v < 0 || v >= W) continue;
                            w += P->psf[(a + R) * S + (b + R)] * x[(long)u * W + v];
                        }
                    }
                    acc += wd * w;
                }
            }
            out[(long)i * P->w + j] = acc;
        }
    }
}

/* out = A_k^T e: the same loops as orc_forward with every multiply-add scattered back. */
void orc_adjoint(const orc_problem *P, int k, const double *e, double *out) {
    const int H = HRH(P), W = HRW(P), S = P->psf_size, R = S / 2, f = P->f;
    const int ty = P->ty[k], tx = P->tx[k];
    const int nb = P->decim == ORC_DECIM_BIN ? f : 1;
    const double wd = 1.0 / ((double)nb * nb);
    const int frac = P->fy[k] != 0.0 || P->fx[k] != 0.0;
    memset(out, 0, sizeof(double) * (size_t)H * W);
    for (int i = 0; i < P->h; ++i) {
        for (int j = 0; j < P->w; ++j) {
            const double ev = wd * e[(long)i * P->w + j];
            for (int a2 = 0; a2 < nb; ++a2) {
                for (int b2 = 0; b2 < nb; ++b2) {
                    const int cu = f * i + a2, cv = f * j + b2;
                    for (int a = -R; a <= R; ++a) {
                        int bu = cu - a;
                        if (bu < 0 || bu >= H) continue;
                        for (int b = -R; b <= R; ++b) {
                            int bv = cv - b;
                            if (bv < 0 || bv >= W) continue;
                            if (frac) {
                                motion_at_adj(P, k, P->psf[(a + R) * S + (b + R)] * ev, bu, bv, out);
                                continue;
                            }
                            int u = bu + ty, v = bv + tx;
                            if (u < 0 || u >= H || v < 0 || v >= W) continue;
                            out[(long)u * W + v] += P->psf[(a + R) * S + (b + R)] * ev;
                        }
                    }
                }
            }
        }
    }
}

/* Charbonnier smoothing of |t| used for the L1 norm of Eq. 8, and its derivatives. */
static double psi(double t, double eps) { return eps > 0 ? sqrt(t * t + eps * eps) - eps : fabs(t); }
static double dpsi(double t, double eps) {
    if (eps > 0) return t / sqrt(t * t + eps * eps);
    return (t > 0) - (t < 0);
}
static double d2psi(double t, double eps) {
    if (eps > 0) { double s = t * t + eps * eps; return eps * eps / (s * sqrt(s)); }
    return 0.0;
}

static double gamma_d(const orc_problem *P, int dx, int dy) { return pow(P->btv_alpha, dx + dy); }

static double sum_rows(const double *row_sums, int n) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += row_sums[i];
    return s;
}

/* Prior R(x).  BTV (Eq. 8): sum over d in [0, w-1]^2 \ {(0,0)} of
 * gamma(d) * sum_q psi(x_q - x_{q+d}), over pairs with q and q + d inside the grid.
 * (d = (0,0) contributes nothing; with ||.||_1 over valid pairs the direction of S_d is
 * immaterial because psi is even.)  Tikhonov: ||x||^2, used only by the tests. */
double orc_reg_value(const orc_problem *P, const double *x) {
    const int H = HRH(P), W = HRW(P);
    double *rows = (double *)calloc((size_t)H, sizeof(double));
    double total = 0.0;
    if (P->reg == ORC_REG_TIKHONOV) {
#pragma omp parallel for schedule(static)
        for (int u = 0; u < H; ++u) {
            double s = 0;
            for (int v = 0; v < W; ++v) s += x[(long)u * W + v] * x[(long)u * W + v];
            rows[u] = s;
        }
        total = sum_rows(rows, H);
        free(rows);
        return total;
    }
    for (int dy = 0; dy < P->btv_w; ++dy) {
        for (int dx = 0; dx < P->btv_w; ++dx) {
            if (dx == 0 && dy == 0) continue;
#pragma omp parallel for schedule(static)
            for (int u = 0; u < H; ++u) {
                double s = 0;
                if (u + dy < H)
                    for (int v = 0; v + dx < W; ++v)
                        s += psi(x[(long)u * W + v] - x[(long)(u + dy) * W + v + dx], P->eps);
                rows[u] = s;
            }
            total += gamma_d(P, dx, dy) * sum_rows(rows, H);
        }
    }
    free(rows);
    return total;
}

/* g = grad R(x) (overwrites g).  BTV: each valid pair adds gamma psi'(t) to q and
 * subtracts it from q + d, t = x_q - x_{q+d}. */
void orc_reg_grad(const orc_problem *P, const double *x, double *g) {
    const int H = HRH(P), W = HRW(P);
    if (P->reg == ORC_REG_TIKHONOV) {
        for (long i = 0; i < (long)H * W; ++i) g[i] = 2.0 * x[i];
        return;
    }
    memset(g, 0, sizeof(double) * (size_t)H * W);
    for (int dy = 0; dy < P->btv_w; ++dy)
        for (int dx = 0; dx < P->btv_w; ++dx) {
            if (dx == 0 && dy == 0) continue;
            const double gm = gamma_d(P, dx, dy);
            for (int u = 0; u + dy < H; ++u)
                for (int v = 0; v + dx < W; ++v) {
                    long q = (long)u * W + v, q2 = (long)(u + dy) * W + v + dx;
                    double d = gm * dpsi(x[q] - x[q2], P->eps);
                    g[q] += d;
                    g[q2] -= d;
                }
        }
}

/* out = H_R(x) p, the exact Hessian of the prior applied to p (overwrites out). */
void orc_reg_hessvec(const orc_problem *P, const double *x, const double *p, double *out) {
    const int H = HRH(P), W = HRW(P);
    if (P->reg == ORC_REG_TIKHONOV) {
        for (long i = 0; i < (long)H * W; ++i) out[i] = 2.0 * p[i];
        return;
    }
    memset(out, 0, sizeof(double) * (size_t)H * W);
    for (int dy = 0; dy < P->btv_w; ++dy)
        for (int dx = 0; dx < P->btv_w; ++dx) {
            if (dx == 0 && dy == 0) continue;
            const double gm = gamma_d(P, dx, dy);
            for (int u = 0; u + dy < H; ++u)
                for (int v = 0; v + dx < W; ++v) {
                    long q = (long)u * W + v, q2 = (long)(u + dy) * W + v + dx;
                    double c = gm * d2psi(x[q] - x[q2], P->eps) * (p[q] - p[q2]);
                    out[q] += c;
                    out[q2] -= c;
                }
        }
}

/* p . H_R(x) p in closed form: sum_d gamma(d) sum_q psi''(x_q - x_{q+d}) (p_q - p_{q+d})^2. */
double orc_reg_curvature(const orc_problem *P, const double *x, const double *p) {
    const int H = HRH(P), W = HRW(P);
    double *rows = (double *)calloc((size_t)H, sizeof(double));
    double total = 0.0;
    if (P->reg == ORC_REG_TIKHONOV) {
        for (int u = 0; u < H; ++u) {
            double s = 0;
            for (int v = 0; v < W; ++v) s += p[(long)u * W + v] * p[(long)u * W + v];
            rows[u] = s;
        }
        total = 2.0 * sum_rows(rows, H);
        free(rows);
        return total;
    }
    for (int dy = 0; dy < P->btv_w; ++dy)
        for (int dx = 0; dx < P->btv_w; ++dx) {
            if (dx == 0 && dy == 0) continue;
#pragma omp parallel for schedule(static)
            for (int u = 0; u < H; ++u) {
                double s = 0;
                if (u + dy < H)
                    for (int v = 0; v + dx < W; ++v) {
                        long q = (long)u * W + v, q2 = (long)(u + dy) * W + v + dx;
                        double dp = p[q] - p[q2];
                        s += d2psi(x[q] - x[q2], P->eps) * dp * dp;
                    }
                rows[u] = s;
            }
            total += gamma_d(P, dx, dy) * sum_rows(rows, H);
        }
    free(rows);
    return total;
}

/* the data term's value on a residual image: sum of squares (L2) or of psi_d (L1), rows
 * first */
static double data_value_lr(const orc_problem *P, const double *e) {
    double *rows = (double *)calloc((size_t)P->h, sizeof(double));
    const int l1 = P->data_norm == ORC_NORM_L1;
    const double ed = P->data_eps;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < P->h; ++i) {
        double s = 0;
        for (int j = 0; j < P->w; ++j) {
            const double t = e[(long)i * P->w + j];
            s += l1 ? psi(t, ed) : t * t;
        }
        rows[i] = s;
    }
    double t = sum_rows(rows, P->h);
    free(rows);
    return t;
}

/* sum of squares of an LR image, rows first */
static double sumsq_lr(const orc_problem *P, const double *e) {
    double *rows = (double *)calloc((size_t)P->h, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < P->h; ++i) {
        double s = 0;
        for (int j = 0; j < P->w; ++j) s += e[(long)i * P->w + j] * e[(long)i * P->w + j];
        rows[i] = s;
    }
    double t = sum_rows(rows, P->h);
    free(rows);
    return t;
}

/* J(x) = sum_k ||A_k x - y_k||^2 + lambda R(x)        Eq. 9 with p = 2 (Eq. 6),
 * or with the L1 data term sum_k sum_i psi_d((A_k x - y_k)_i).
 * y holds the K frames back to back, each h x w row-major. */
double orc_objective(const orc_problem *P, const double *x, const double *y) {
    const long m = (long)P->h * P->w;
    double *e = (double *)malloc(sizeof(double) * m);
    double data = 0.0;
    for (int k = 0; k < P->K; ++k) {
        orc_forward(P, k, x, e);
        for (long i = 0; i < m; ++i) e[i] -= y[k * m + i];
        data += data_value_lr(P, e);
    }
    free(e);
    return data + P->lambda * orc_reg_value(P, x);
}

/* g = grad J(x) = 2 sum_k A_k^T (A_k x - y_k) + lambda grad R(x)  (L2), or
 * sum_k A_k^T psi_d'(A_k x - y_k) + lambda grad R(x)  (L1); returns J(x). */
double orc_gradient(const orc_problem *P, const double *x, const double *y, double *g) {
    const long m = (long)P->h * P->w, n = (long)HRH(P) * HRW(P);
    double *e = (double *)malloc(sizeof(double) * m);
    double *t = (double *)malloc(sizeof(double) * n);
    double data = 0.0;
    orc_reg_grad(P, x, g);
    for (long i = 0; i < n; ++i) g[i] *= P->lambda;
    for (int k = 0; k < P->K; ++k) {
        orc_forward(P, k, x, e);
        for (long i = 0; i < m; ++i) e[i] -= y[k * m + i];
        data += data_value_lr(P, e);
        if (P->data_norm == ORC_NORM_L1) {
            for (long i = 0; i < m; ++i) e[i] = dpsi(e[i], P->data_eps);
            orc_adjoint(P, k, e, t);
            for (long i = 0; i < n; ++i) g[i] += t[i];
        } else {
            orc_adjoint(P, k, e, t);
            for (long i = 0; i < n; ++i) g[i] += 2.0 * t[i];
        }
    }
    free(e);
    free(t);
    return data + P->lambda * orc_reg_value(P, x);
}

/* out = H(x) p = 2 sum_k A_k^T A_k p + lambda H_R(x) p  (L2), or
 * sum_k A_k^T diag(psi_d''(A_k x - y_k)) A_k p + lambda H_R(x) p  (L1; y is read only then). */
void orc_hessvec(const orc_problem *P, const double *x, const double *y, const double *p, double *out) {
    const long m = (long)P->h * P->w, n = (long)HRH(P) * HRW(P);
    double *e = (double *)malloc(sizeof(double) * m);
    double *ex = (double *)malloc(sizeof(double) * m);
    double *t = (double *)malloc(sizeof(double) * n);
    const int l1 = P->data_norm == ORC_NORM_L1;
    orc_reg_hessvec(P, x, p, out);
    for (long i = 0; i < n; ++i) out[i] *= P->lambda;
    for (int k = 0; k < P->K; ++k) {
        orc_forward(P, k, p, e);
        if (l1) {
            orc_forward(P, k, x, ex);
            for (long i = 0; i < m; ++i) e[i] *= d2psi(ex[i] - y[k * m + i], P->data_eps);
        }
        orc_adjoint(P, k, e, t);
        for (long i = 0; i < n; ++i) out[i] += (l1 ? 1.0 : 2.0) * t[i];
    }
    free(e);
    free(ex);
    free(t);
}

/* p . H(x) p in closed form: 2 sum_k ||A_k p||^2 + lambda p . H_R(x) p  (L2), or
 * sum_k sum_i psi_d''((A_k x - y_k)_i) (A_k p)_i^2 + lambda p . H_R(x) p  (L1). */
double orc_curvature(const orc_problem *P, const double *x, const double *y, const double *p) {
    const long m = (long)P->h * P->w;
    double *e = (double *)malloc(sizeof(double) * m);
    double *ex = (double *)malloc(sizeof(double) * m);
    const int l1 = P->data_norm == ORC_NORM_L1;
    double data = 0.0;
    for (int k = 0; k < P->K; ++k) {
        orc_forward(P, k, p, e);
        if (l1) {
            orc_forward(P, k, x, ex);
            double *rows = (double *)calloc((size_t)P->h, sizeof(double));
            for (int i = 0; i < P->h; ++i) {
                double s = 0;
                for (int j = 0; j < P->w; ++j) {
                    const long o = (long)i * P->w + j;
                    s += d2psi(ex[o] - y[k * m + o], P->data_eps) * e[o] * e[o];
                }
                rows[i] = s;
            }
            data += sum_rows(rows, P->h);
            free(rows);
        } else {
            data += 2.0 * sumsq_lr(P, e);
        }
    }
    free(e);
    free(ex);
    return data + P->lambda * orc_reg_curvature(P, x, p);
}

/* Multi-image interpolation (Sec. 4.1.1): every LR sample is placed at the HR pixel it was
 * taken at, x0 = sum_k M_k^T D^T y_k / sum_k M_k^T D^T 1 with D the point sampling, and 0
 * where no sample falls.  With a non-integer shift M_k^T spreads a sample over the 2 x 2 HR
 * pixels around its position with the bilinear weights. */
void orc_shift_add(const orc_problem *P, const double *y, double *x0) {
    const int H = HRH(P), W = HRW(P), f = P->f;
    const long n = (long)H * W, m = (long)P->h * P->w;
    double *cnt = (double *)calloc((size_t)n, sizeof(double));
    memset(x0, 0, sizeof(double) * (size_t)n);
    for (int k = 0; k < P->K; ++k)
        for (int i = 0; i < P->h; ++i)
            for (int j = 0; j < P->w; ++j) {
                motion_at_adj(P, k, y[k * m + (long)i * P->w + j], f * i, f * j, x0);
                motion_at_adj(P, k, 1.0, f * i, f * j, cnt);
            }
    for (long i = 0; i < n; ++i) x0[i] = cnt[i] > 0 ? x0[i] / cnt[i] : 0.0;
    free(cnt);
}

/* Detector counts to attenuation line integrals (Beer-Lambert): y = ln I0 - ln max(c, 1). */
void orc_log_convert(const unsigned short *counts, long n, double flat_field, double *y) {
    for (long i = 0; i < n; ++i) {
        double c = counts[i] < 1 ? 1.0 : (double)counts[i];
        y[i] = log(flat_field) - log(c);
    }
}

static double dot(const double *a, const double *b, long n) {
    double s = 0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Moller's scaled conjugate gradient on J (Sec. 3.1 cites it for the local solves;
 * Algorithm 1 runs it for n_iter iterations, failed ones included; Table 1 lists its
 * scalars).  Step numbers follow Moller's description:
 *   1  x_1 = x0, p_1 = r_1 = -J'(x_1), sigma = 1e-4, lambda_1 = 1e-6, lambda_bar = 0,
 *      success = true
 *   2  if success: sigma_k = sigma / |p_k|, s_k = (J'(x_k + sigma_k p_k) - J'(x_k)) / sigma_k
 *      (HV mode FD) or s_k = H(x_k) p_k, its sigma -> 0 limit (HV mode EXACT);
 *      delta_k = p_k . s_k
 *   3  delta_k += (lambda_k - lambda_bar) |p_k|^2
 *   4  if delta_k <= 0: lambda_bar = 2 (lambda_k - delta_k / |p_k|^2),
 *      delta_k = -delta_k + lambda_k |p_k|^2, lambda_k = lambda_bar
 *   5  mu_k = p_k . r_k, alpha_k = mu_k / delta_k
 *   6  Delta_k = 2 delta_k (J(x_k) - J(x_k + alpha_k p_k)) / mu_k^2
 *   7  if Delta_k >= 0: x_{k+1} = x_k + alpha_k p_k, r_{k+1} = -J'(x_{k+1}), lambda_bar = 0,
 *      success = true, beta_k = (|r_{k+1}|^2 - r_{k+1} . r_k) / mu_k,
 *      p_{k+1} = r_{k+1} + beta_k p_k, and if Delta_k >= 0.75: lambda_k /= 4;
 *      else: lambda_bar = lambda_k, success = false
 *   8  if Delta_k < 0.25: lambda_k += delta_k (1 - Delta_k) / |p_k|^2
 *   9  stop when r = 0; otherwise next iteration.
 * Moller restarts with p = r every N iterations, N the number of unknowns; N exceeds
 * every iteration count used here, so no restart happens.
 * Returns the number of iterations run. */
int orc_scg(const orc_problem *P, const double *y, const double *x0, int iters, int hv_mode,
            double *x_out, orc_trace_row *trace) {
    const long n = (long)HRH(P) * HRW(P);
    double *x = x_out;
    double *r = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *s = (double *)malloc(sizeof(double) * n);
    double *xt = (double *)malloc(sizeof(double) * n);
    double *rt = (double *)malloc(sizeof(double) * n);
    const double sigma0 = 1e-4;
    double lam = 1e-6, lam_bar = 0.0, delta = 0.0, pn2 = 0.0;
    int success = 1, it;

    memcpy(x, x0, sizeof(double) * n);
    if (P->state_f32) round_f32(x, n);
    double E = orc_gradient(P, x, y, r);
    for (long i = 0; i < n; ++i) { r[i] = -r[i]; p[i] = r[i]; }
    if (P->state_f32) { round_f32(r, n); round_f32(p, n); }

    for (it = 0; it < iters; ++it) {
        if (success) {
            pn2 = dot(p, p, n);
            if (pn2 == 0.0) break;
            if (hv_mode == ORC_HV_FD) {
                double sig = sigma0 / sqrt(pn2);
                for (long i = 0; i < n; ++i) xt[i] = x[i] + sig * p[i];
                orc_gradient(P, xt, y, s);                      /* J'(x + sigma p) */
                for (long i = 0; i < n; ++i) s[i] = (s[i] + r[i]) / sig;  /* J'(x) = -r */
            } else {
                orc_hessvec(P, x, y, p, s);
            }
            delta = dot(p, s, n);
        }
        delta += (lam - lam_bar) * pn2;
        if (delta <= 0) {
            lam_bar = 2.0 * (lam - delta / pn2);
            delta = -delta + lam * pn2;
            lam = lam_bar;
        }
        const double mu = dot(p, r, n);
        const double alpha = mu / delta;
        for (long i = 0; i < n; ++i) xt[i] = x[i] + alpha * p[i];
        const double Et = orc_gradient(P, xt, y, rt);           /* J(x_t), J'(x_t) */
        const double Delta = 2.0 * delta * (E - Et) / (mu * mu);
        const double E_before = E;
        int accept = Delta >= 0;
        if (accept) {
            for (long i = 0; i < n; ++i) rt[i] = -rt[i];
            const double rr_new = dot(rt, rt, n), rr_cross = dot(rt, r, n);
            const double beta = (rr_new - rr_cross) / mu;
            memcpy(x, xt, sizeof(double) * n);
            for (long i = 0; i < n; ++i) { p[i] = rt[i] + beta * p[i]; r[i] = rt[i]; }
            if (P->state_f32) { round_f32(x, n); round_f32(r, n); round_f32(p, n); }
            E = Et;
            lam_bar = 0.0;
            success = 1;
            if (Delta >= 0.75) lam = lam / 4.0;
        } else {
            lam_bar = lam;
            success = 0;
        }
        if (Delta < 0.25) lam = lam + delta * (1.0 - Delta) / pn2;
        if (trace) {
            orc_trace_row *tr = &trace[it];
            tr->E = E_before; tr->J_trial = Et; tr->alpha = alpha; tr->delta = delta;
            tr->mu = mu; tr->lam = lam; tr->Delta = Delta; tr->pn2 = pn2;
            tr->rn2 = dot(r, r, n); tr->accept = accept;
        }
        if (accept && dot(r, r, n) == 0.0) { ++it; break; }
    }
    free(r); free(p); free(s); free(xt); free(rt);
    return it;
}
