/*
 * FP64 CPU oracle for the SCG solve of the multi-image super-resolution (MISR) objective.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg load this library.  It shares no code with the CUDA library.
 *
 * Problem (Sec. 3.1):
 *   image formation   y_k = A_k x + noise,  A_k = D B M_k             (Eq. 1)
 *   data term         sum_k || A_k x - y_k ||_2^2                      (Eq. 6, p = 2)
 *                     or sum_k sum_i psi_d((A_k x - y_k)_i), psi_d(t) = sqrt(t^2 + eps_d^2) - eps_d,
 *                     the L1 norm of the paper's experiments (Sec. 3.1) smoothed like the prior
 *   prior (BTV)       sum_d gamma(d) || x - S_d x ||_1,
 *                     d = (dx, dy), dx, dy in [0, w-1], gamma = alpha^(dx+dy)   (Eq. 8)
 *   objective         J(x) = data + lambda * prior                     (Eq. 9)
 *   solver            Moller's scaled conjugate gradient (Sec. 3.1, Algorithm 1, Table 1)
 *
 * Readings where the paper is silent (each is stated where it is used in the .c file):
 *   M_k  translation by the HR shift t_k = f * s_k (s_k in LR px), x zero outside; for a
 *        non-integer t_k = n_k + a_k (n_k integer, 0 < a_k < 1) per axis, bilinear
 *        interpolation: (M_k x)(u) = (1 - a_k) x(u + n_k) + a_k x(u + n_k + 1)
 *   B    convolution with the PSF h (normalised to sum 1), zero outside the HR grid
 *   D    sampling at HR position (f i, f j), or (ORC_DECIM_BIN) the mean of the f x f block
 *        whose first pixel is (f i, f j): the 2 x 2 binning of the synthetic study (Sec. 4.1.1)
 *   |.|  in the BTV term is smoothed as psi(t) = sqrt(t^2 + eps^2) - eps  (eps = 0: |t|)
 *   pairs (q, q + d) enter the BTV sum only when both pixels lie inside the grid
 *
 * Parity pins: tests/test_oracle_pins.py.  Every function here is pinned by at least one
 * check that does not call the oracle twice: a dense D*B*M product built from the textbook
 * matrices, closed-form BTV values, central finite differences, exact recovery, a dense
 * normal-equation solve and conjugate-gradient identities.
 * Moller's scale increase after a poor step (Delta < 0.25) is pinned through the identity it
 * implies after a rejected step: the next step's curvature is delta_k (2 - Delta_k) and its
 * step alpha_k / (2 - Delta_k).  The negative-curvature correction (delta <= 0) cannot run for
 * a convex J with Moller's lambda > 0 (delta is p.H p + lambda |p|^2 > 0 on a fresh direction
 * and grows after a rejection); the pins check that every first attempt along a direction has
 * delta_k = p_k.H p_k + lambda_{k-1} |p_k|^2, which a correction would break.
 */
#ifndef MISR_ORACLE_H
#define MISR_ORACLE_H

#define ORC_MAXK 64
#define ORC_MAXPSF 15

enum { ORC_REG_BTV = 0, ORC_REG_TIKHONOV = 1 };
enum { ORC_HV_EXACT = 0, ORC_HV_FD = 1 };
enum { ORC_NORM_L2 = 0, ORC_NORM_L1 = 1 };
enum { ORC_DECIM_POINT = 0, ORC_DECIM_BIN = 1 };

typedef struct {
    int h, w;                 /* LR frame size (rows, cols) */
    int K, f;                 /* number of frames, magnification factor */
    int ty[ORC_MAXK];         /* integer HR shift of frame k, rows */
    int tx[ORC_MAXK];         /* integer HR shift of frame k, cols */
    int psf_size;             /* odd */
    double psf[ORC_MAXPSF * ORC_MAXPSF];  /* row-major, normalised to sum 1 */
    double lambda;            /* regulariser weight */
    double btv_alpha;         /* spatial decay alpha of gamma(d) */
    int btv_w;                /* BTV window w */
    double eps;               /* Charbonnier smoothing of |.| */
    int reg;                  /* ORC_REG_BTV or ORC_REG_TIKHONOV */
    int data_norm;            /* ORC_NORM_L2 (default) or ORC_NORM_L1 */
    double data_eps;          /* Charbonnier smoothing of the L1 data term (> 0) */
    int decim;                /* ORC_DECIM_POINT (default) or ORC_DECIM_BIN */
    double fy[ORC_MAXK];      /* fractional part a_k of the HR shift, rows (ty = floor) */
    double fx[ORC_MAXK];      /* fractional part a_k of the HR shift, cols (tx = floor) */
    int state_f32;            /* 1: orc_scg rounds x, r and p to FP32 after every update (a
                                 model of FP32 storage of the SCG state, for sensitivity
                                 studies; 0, the default, keeps everything in FP64) */
} orc_problem;

/* one row of the SCG trace per iteration (failed iterations included) */
typedef struct {
    double E;        /* J(x_k) before the step */
    double J_trial;  /* J(x_k + alpha_k p_k) */
    double alpha, delta, mu;   /* step, scaled curvature, p.r */
    double lam;      /* Moller's lambda after the iteration's updates */
    double Delta;    /* comparison parameter */
    double pn2;      /* |p_k|^2 */
    double rn2;      /* |r|^2 after the iteration */
    double accept;   /* 1 accepted, 0 rejected */
} orc_trace_row;

#ifdef __cplusplus
extern "C" {
#endif

int orc_init(orc_problem *P, int h, int w, int K, int f, const double *shifts_lr,
             const double *psf, int psf_size, double lambda, double btv_alpha, int btv_w,
             double eps, int reg);
int orc_set_data_norm(orc_problem *P, int norm, double data_eps);
int orc_set_decimation(orc_problem *P, int mode);
int orc_set_state_f32(orc_problem *P, int on);
int orc_threads(void);
void orc_forward(const orc_problem *P, int k, const double *x, double *out);
void orc_adjoint(const orc_problem *P, int k, const double *e, double *out);
double orc_reg_value(const orc_problem *P, const double *x);
void orc_reg_grad(const orc_problem *P, const double *x, double *g);
void orc_reg_hessvec(const orc_problem *P, const double *x, const double *p, double *out);
double orc_reg_curvature(const orc_problem *P, const double *x, const double *p);
double orc_objective(const orc_problem *P, const double *x, const double *y);
double orc_gradient(const orc_problem *P, const double *x, const double *y, double *g);
void orc_hessvec(const orc_problem *P, const double *x, const double *y, const double *p, double *out);
double orc_curvature(const orc_problem *P, const double *x, const double *y, const double *p);
void orc_shift_add(const orc_problem *P, const double *y, double *x0);
void orc_log_convert(const unsigned short *counts, long n, double flat_field, double *y);
int orc_scg(const orc_problem *P, const double *y, const double *x0, int iters, int hv_mode,
            double *x_out, orc_trace_row *trace);

#ifdef __cplusplus
}
#endif
#endif
