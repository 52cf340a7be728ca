// Device code of the sm_103a MISR solver: the fused SCG pass, its scalar tail, and the
// prepare / forward / finalize kernels.
//
// Model (Sec. 3.1 of the paper): y_k = D B M_k x (Eq. 1), J(x) = sum_k ||A_k x - y_k||^2 +
// lambda * BTV(x) (Eq. 6, 8, 9), solved with Moller's scaled conjugate gradient (Algorithm 1).
//
// Layout of the data term on the HR grid.  Every frame k is shifted by an integer HR offset
// t_k in [0, f-1]^2, so its samples sit at HR pixels c = (f i + t_y, f j + t_x), and the
// phase (c_y mod f, c_x mod f) of a sample equals its frame's shift.  With one frame per
// phase, the K frames interleave into one HR image Y (NaN where no frame samples) and
//   A_k x (i, j) = (B_c x)(c),   B_c: convolution with the PSF whose taps that read x at a
//                                row < (c_y mod f) or a column < (c_x mod f) are dropped
// (the zero padding of B in front of the shift M_k; it only matters within f + R pixels of
// the top/left border).  So the data term of all K frames is one HR blur, one residual image
// E = B x - Y and one adjoint blur B^T E, whatever K is.
//
// HR images in the workspace are row-major with a row pitch that is a multiple of 4 floats,
// so that every row starts on a 16-byte boundary (TMA boxes, float4 stores).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tma.cuh"

namespace misr {

constexpr int MAXK = 64;
constexpr int MAXF = 8;
constexpr int PSF_R = 2;   // compiled PSF radius (5x5 taps); smaller PSFs are zero-padded
constexpr int BTV_W = 3;   // compiled BTV window; smaller windows get gamma = 0
constexpr int NPART = 10;
constexpr int TRACE_COLS = 10;
constexpr uint32_t TMA_WAIT_TRIES = 1u << 24;   // bounded wait for the tile loads

// per-tile partial sums of one pass (FP64)
enum { P_JD = 0, P_DJD, P_JB, P_RR, P_RRX, P_PR, P_PP, P_A, P_B, P_C };
enum { MODE_INIT = 0, MODE_ITER = 1, MODE_PROBE = 2 };
// device status codes (ScgState::status)
enum { DEV_OK = 0, DEV_TMA_TIMEOUT = 1 };

// Moller's SCG scalars of one projection, kept on the device between passes.
struct ScgState {
    double E;         // J(x_k)
    double E_btv;     // lambda * R(x_k)
    double lam, lam_bar;
    double delta;     // scaled curvature in effect for the coming step
    double mu;        // p_k . r_k
    double pn2;       // |p_k|^2
    double alpha;     // step of the coming pass
    double beta;      // p_k = r_k + beta * p_{k-1}, applied inside the coming pass
    double rn2;       // |r_k|^2
    double sums[NPART];
    int cur, pcur;    // which half of the X/R and P double buffers holds x_k, r_k / p_{k-1}
    int success, iter, accepted, done, status, iters;
};

struct DevProblem {
    CUtensorMap tmX[2], tmR[2], tmP[2], tmY;      // TMA maps of the workspace images
    int H, W, pitch, f, h, w, K;
    int tiles_x, tiles_y, n_tiles, iters, pad0;
    float hy[2 * PSF_R + 1], hx[2 * PSF_R + 1];  // separable PSF, h(a, b) = hy[a+R] hx[b+R]
    float lambda, eps, eps2, pad1;
    float gamma[BTV_W * BTV_W];                   // gamma(dx, dy) at [dy * BTV_W + dx]
    double eps_pairs;                             // eps * sum_d gamma_d * #pairs_d
    float *X[2], *Rv[2], *Pv[2];                  // x, r (double buffered), p (double buffered)
    float *Y;                                     // interleaved frames, NaN where unsampled
    double *partials;                             // [n_tiles][NPART]
    unsigned int *counter;                        // tiles finished in the current pass
    ScgState *st;
    double *trace;                                // [iters][TRACE_COLS]
    int ty[MAXK], tx[MAXK];
    int frame_of_phase[MAXF * MAXF];              // -1: no frame samples that phase
};

__device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ int ld_cg(const int *p) { return __ldcg(p); }

// ---------------------------------------------------------------------------------------
// SCG scalar tail, run by thread 0 of the last CTA of a pass with the pass totals S.
// Steps follow Moller's algorithm (the same order as Algorithm 1's loop body):
// comparison parameter, accept/reject, lambda updates, beta, then the scaling of the next
// curvature and the next step size.
__device__ inline void scg_tail(const DevProblem &P, ScgState *st, const double *S, int mode) {
    for (int i = 0; i < NPART; ++i) st->sums[i] = S[i];
    if (mode == MODE_PROBE) return;
    const double lambda = (double)P.lambda;
    const double Jb = lambda * (S[P_JB] - P.eps_pairs);   // lambda R(x')
    const double Jt = S[P_JD] + Jb;                        // J(x')
    const double rr = S[P_RR], rrx = S[P_RRX], pr = S[P_PR], pp = S[P_PP];
    double delta_raw = 0, mu_next = 0, pn2_next = 0;
    if (mode == MODE_INIT) {
        // x_1 = x0, r_1 = -J'(x_1), p_1 = r_1 (beta = 0 on a zero p_0)
        st->E = Jt; st->E_btv = Jb; st->rn2 = rr;
        st->lam = 1e-6; st->lam_bar = 0; st->success = 1;
        st->iter = 0; st->accepted = 0; st->beta = 0;
        delta_raw = S[P_A]; mu_next = rr; pn2_next = rr;
        st->cur ^= 1; st->pcur ^= 1;
        if (rr == 0.0 || st->iters <= 0) st->done = 1;
    } else {
        const double delta = st->delta, mu = st->mu, pn2 = st->pn2;
        // J(x') - J(x): data part from the per-pixel difference (accurate in FP32),
        // prior part from its two direct evaluations
        const double dE = S[P_DJD] + (Jb - st->E_btv);
        const double Delta = 2.0 * delta * (-dE) / (mu * mu);
        const double E_before = st->E;
        const int accept = Delta >= 0.0;
        if (accept) {
            const double beta = (rr - rrx) / mu;
            st->E = Jt; st->E_btv = Jb; st->rn2 = rr;
            delta_raw = S[P_A] + 2.0 * beta * S[P_B] + beta * beta * S[P_C];
            mu_next = rr + beta * pr;
            pn2_next = rr + 2.0 * beta * pr + beta * beta * pp;
            st->lam_bar = 0; st->success = 1;
            if (Delta >= 0.75) st->lam = st->lam / 4.0;
            st->cur ^= 1; st->pcur ^= 1;
            st->beta = beta;
            st->accepted += 1;
        } else {
            st->lam_bar = st->lam;
            st->success = 0;
        }
        if (Delta < 0.25) st->lam = st->lam + delta * (1.0 - Delta) / pn2;
        if (P.trace) {
            double *t = P.trace + (size_t)st->iter * TRACE_COLS;
            t[0] = E_before; t[1] = Jt; t[2] = st->alpha; t[3] = delta; t[4] = mu;
            t[5] = st->lam; t[6] = Delta; t[7] = pn2; t[8] = st->rn2; t[9] = accept;
        }
        st->iter += 1;
        if ((accept && rr == 0.0) || st->iter >= st->iters) st->done = 1;
    }
    // next step: Moller steps 2-5 (curvature, its scaling, step size)
    if (st->success) { st->delta = delta_raw; st->mu = mu_next; st->pn2 = pn2_next; }
    double delta = st->delta + (st->lam - st->lam_bar) * st->pn2;
    if (delta <= 0.0) {
        st->lam_bar = 2.0 * (st->lam - delta / st->pn2);
        delta = -delta + st->lam * st->pn2;
        st->lam = st->lam_bar;
    }
    st->delta = delta;
    st->alpha = st->mu / delta;
    if (!(st->pn2 > 0.0) || !isfinite(st->alpha)) st->done = 1;
}

// ---------------------------------------------------------------------------------------
// Tile geometry of the fused pass.  A CTA owns TH x TW HR pixels at (y0, x0).  Shared
// buffers, with their origin relative to (y0, x0) and their size:
//   XB, PB, RB  x' / p / r     origin (-6, -8)  (TH+12) x (TW+16)   TMA boxes (x first col
//                                                                    16-byte aligned)
//   YB          Y, then E      origin (-4, -4)  (TH+8)  x (TW+8)    TMA box, NaN outside
//   GB          2 B^T E, r'    origin (-2, -2)  (TH+4)  x (TW+4)
//   SC scratch: forward horizontal blur (TH+12) x (TW+8), adjoint horizontal blur
//               (TH+8) x (TW+4), three psi'(t_d) planes on origin (-4, -4) (TH+6) x (TW+8),
//               and the horizontal blurs of p for the curvature (TH+4) x TW
//   SMP         sampled flags of the owned pixels
template <int TH, int TW>
struct Geo {
    static_assert(PSF_R == 2 && BTV_W == 3, "halo layout assumes a 5x5 PSF and a 3x3 BTV window");
    static_assert(TW % 4 == 0 && TH % 2 == 0, "tile must be float4 wide and even high");
    static constexpr int XH = TH + 12, XW = TW + 16;
    static constexpr int EH = TH + 8, EW = TW + 8;
    static constexpr int GH = TH + 4, GW = TW + 4;
    static constexpr int DH = TH + 6, DW = TW + 8;
    static constexpr int CH = TH + 4, CW = TW;
    static constexpr int S1 = XH * EW, S2 = EH * GW, S3 = 3 * DH * DW, S4 = CH * CW;
    static constexpr int S12 = S1 > S2 ? S1 : S2, S34 = S3 > S4 ? S3 : S4;
    static constexpr int SC = S12 > S34 ? S12 : S34;
    static constexpr int FLOATS = 3 * XH * XW + EH * EW + GH * GW + SC;
    static constexpr size_t TMA_BYTES = sizeof(float) * (3 * XH * XW + EH * EW);
    static constexpr size_t SMEM_BYTES = 128 /*align slack*/ + sizeof(float) * FLOATS + TH * TW + 64;
};

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
__device__ __forceinline__ void ld8(const float *p, float *v) {   // p 16-byte aligned
    const float4 a = ld4(p), b = ld4(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void ld8_off2(const float *p, float *v) {   // p 8-byte aligned
    const float2 a = ld2(p), c = ld2(p + 6);
    const float4 b = ld4(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = b.z; v[5] = b.w; v[6] = c.x; v[7] = c.y;
}
__device__ __forceinline__ void ld4v(const float *p, float *v) {
    const float4 a = ld4(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void st4v(float *p, const float *v) { st4(p, make_float4(v[0], v[1], v[2], v[3])); }

// Frame mask of the forward blur at sample coordinate c (one axis) for tap offset a:
// the tap reads coordinate c - a, dropped when c - a < (c mod f).
__device__ __forceinline__ bool fwd_tap_ok(int c, int a, int f) { return c < 0 || (c - a) >= (c % f); }
// Frame mask of the adjoint blur at output coordinate u for tap offset a: the sample read
// sits at u + a; the tap exists when u >= ((u + a) mod f).
__device__ __forceinline__ bool adj_tap_ok(int u, int a, int f) { return (u + a) < 0 || u >= ((u + a) % f); }

struct PassAcc {
    float jd, dj, jb, rr, rrx, pr, pp, ad, bd, cd, ab, bb, cb;
};

// ---------------------------------------------------------------------------------------
// Body of the fused pass on one tile.  BORDER: the tile's halo reaches outside the image, so
// frame masks, BTV pair validity and image bounds are checked; interior tiles skip them.
template <int TH, int TW, int NT, bool BORDER>
__device__ __forceinline__ void pass_tile(const DevProblem &P, float *sm, unsigned char *smp, int y0, int x0,
                                          float alpha, float beta, float *Xn, float *Rn, float *Pn, PassAcc &A) {
    using G = Geo<TH, TW>;
    constexpr int XH = G::XH, XW = G::XW, EH = G::EH, EW = G::EW, GH = G::GH, GW = G::GW;
    constexpr int DH = G::DH, DW = G::DW, CH = G::CH, CW = G::CW;
    float *XB = sm;
    float *PB = XB + XH * XW;
    float *RB = PB + XH * XW;
    float *YB = RB + XH * XW;
    float *GB = YB + EH * EW;
    float *SC = GB + GH * GW;
    const int tid = threadIdx.x;
    const int H = P.H, W = P.W, f = P.f, pitch = P.pitch;
    float hx[5], hy[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) { hx[i] = P.hx[i]; hy[i] = P.hy[i]; }
    const float lambda = P.lambda, eps2 = P.eps2;

    // --- A: p = r + beta p_old, x' = x + alpha p on the X box; owned pixels go to HBM
    for (int it = tid; it < XH * XW / 4; it += NT) {
        const int r = it / (XW / 4), c4 = it - r * (XW / 4);
        const float4 rv = ld4(RB + 4 * it), pov = ld4(PB + 4 * it), xv = ld4(XB + 4 * it);
        float4 pv, xn;
        pv.x = fmaf(beta, pov.x, rv.x); pv.y = fmaf(beta, pov.y, rv.y);
        pv.z = fmaf(beta, pov.z, rv.z); pv.w = fmaf(beta, pov.w, rv.w);
        xn.x = fmaf(alpha, pv.x, xv.x); xn.y = fmaf(alpha, pv.y, xv.y);
        xn.z = fmaf(alpha, pv.z, xv.z); xn.w = fmaf(alpha, pv.w, xv.w);
        st4(PB + 4 * it, pv);
        st4(XB + 4 * it, xn);
        const int orow = r - 6, ocol = 4 * c4 - 8;
        if (orow >= 0 && orow < TH && ocol >= 0 && ocol < TW) {
            const int gy = y0 + orow, gx = x0 + ocol;
            if (!BORDER || (gy < H && gx + 3 < W)) {
                const size_t o = (size_t)gy * pitch + gx;
                st4(Xn + o, xn);
                st4(Pn + o, pv);
                A.pp += pv.x * pv.x + pv.y * pv.y + pv.z * pv.z + pv.w * pv.w;
            } else if (gy < H) {
                const float xs[4] = {xn.x, xn.y, xn.z, xn.w}, ps[4] = {pv.x, pv.y, pv.z, pv.w};
                for (int j = 0; j < 4 && gx + j < W; ++j) {
                    const size_t o = (size_t)gy * pitch + gx + j;
                    Xn[o] = xs[j];
                    Pn[o] = ps[j];
                    A.pp += ps[j] * ps[j];
                }
            }
        }
    }
    __syncthreads();

    // --- B1: forward horizontal blur of x' on (X rows) x (E cols)
    float *H1 = SC;
    for (int it = tid; it < XH * EW / 4; it += NT) {
        const int r = it / (EW / 4), e = 4 * (it - r * (EW / 4));
        float in[8];
        ld8_off2(XB + r * XW + e + 2, in);   // x' at E cols e-2 .. e+5
        float out[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float s = 0.f;
#pragma unroll
            for (int b = -2; b <= 2; ++b) {
                float v = in[j + 2 - b];
                if (BORDER && !fwd_tap_ok(x0 - 4 + e + j, b, f)) v = 0.f;
                s = fmaf(hx[b + 2], v, s);
            }
            out[j] = s;
        }
        st4v(H1 + r * EW + e, out);
    }
    __syncthreads();

    // --- B2: vertical blur -> Z, residual E = Z - Y (0 where Y is NaN: unsampled or outside)
    for (int it = tid; it < (EH / 2) * (EW / 4); it += NT) {
        const int m = it / (EW / 4), e = 4 * (it - m * (EW / 4)), n = 2 * m;
        float rows[6][4];
#pragma unroll
        for (int i = 0; i < 6; ++i) ld4v(H1 + (n + i) * EW + e, rows[i]);
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int gy = y0 - 4 + n + rr;
            float yv[4], ev[4];
            ld4v(YB + (n + rr) * EW + e, yv);
            const bool own_row = (n + rr - 4) >= 0 && (n + rr - 4) < TH;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float z = 0.f;
#pragma unroll
                for (int a = -2; a <= 2; ++a) {
                    float v = rows[rr + 2 - a][j];
                    if (BORDER && !fwd_tap_ok(gy, a, f)) v = 0.f;
                    z = fmaf(hy[a + 2], v, z);
                }
                const bool smp_ok = !isnan(yv[j]);
                ev[j] = smp_ok ? z - yv[j] : 0.f;
                const int oc = e + j - 4;
                if (own_row && oc >= 0 && oc < TW) {
                    smp[(n + rr - 4) * TW + oc] = smp_ok;
                    A.jd = fmaf(ev[j], ev[j], A.jd);
                }
            }
            st4v(YB + (n + rr) * EW + e, ev);
        }
    }
    __syncthreads();

    // --- C1: adjoint horizontal blur of E on (E rows) x (G cols)
    float *H2 = SC;
    for (int it = tid; it < EH * GW / 4; it += NT) {
        const int n = it / (GW / 4), g = 4 * (it - n * (GW / 4));
        float in[8];
        ld8(YB + n * EW + g, in);   // E at G cols g-2 .. g+5
        float out[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float s = 0.f;
#pragma unroll
            for (int b = -2; b <= 2; ++b) {
                float v = in[j + 2 + b];
                if (BORDER && !adj_tap_ok(x0 - 2 + g + j, b, f)) v = 0.f;
                s = fmaf(hx[b + 2], v, s);
            }
            out[j] = s;
        }
        st4v(H2 + n * GW + g, out);
    }
    __syncthreads();

    // --- C2: adjoint vertical blur -> GB = 2 B^T E
    for (int it = tid; it < (GH / 2) * (GW / 4); it += NT) {
        const int m = it / (GW / 4), g = 4 * (it - m * (GW / 4)), n = 2 * m;
        float rows[6][4];
#pragma unroll
        for (int i = 0; i < 6; ++i) ld4v(H2 + (n + i) * GW + g, rows[i]);
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int u = y0 - 2 + n + rr;
            float out[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float s = 0.f;
#pragma unroll
                for (int a = -2; a <= 2; ++a) {
                    float v = rows[rr + 2 + a][j];
                    if (BORDER && !adj_tap_ok(u, a, f)) v = 0.f;
                    s = fmaf(hy[a + 2], v, s);
                }
                out[j] = 2.f * s;
            }
            st4v(GB + (n + rr) * GW + g, out);
        }
    }
    // (no barrier needed here: D reads XB and writes the planes, which alias H2 only)
    __syncthreads();

    // --- D: BTV gradient.  Items are 4-pixel row groups of the D grid (origin (-4, -4));
    // the forward part sum_d gamma_d psi'(x_q - x_{q+d}) accumulates in registers, the
    // backward part sum_d gamma_d psi'(x_{q-d} - x_q) is read from psi' planes, one round
    // per row offset dy with a plane for each dx.
    constexpr int ND = DH * DW / 4;
    constexpr int NDI = (ND + NT - 1) / NT;
    float *PL = SC;   // 3 planes of DH x DW
    float facc[NDI][4], bacc[NDI][4];
#pragma unroll
    for (int i = 0; i < NDI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { facc[i][j] = 0.f; bacc[i][j] = 0.f; }
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
#pragma unroll
        for (int i = 0; i < NDI; ++i) {
            const int it = tid + i * NT;
            if (it >= ND) break;
            const int n = it / (DW / 4), e = 4 * (it - n * (DW / 4));
            float xq[4], xp[8];
            ld4v(XB + (n + 2) * XW + e + 4, xq);
            ld8(XB + (n + 2 + dy) * XW + e + 4, xp);
            const int qy = y0 - 4 + n;
            const bool own_row = (n - 4) >= 0 && (n - 4) < TH;
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                if (dx == 0 && dy == 0) continue;
                const float gam = P.gamma[dy * 3 + dx];
                float pv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float t = xq[j] - xp[j + dx];
                    const float s = fmaf(t, t, eps2);
                    const float rs = rsqrtf(s);
                    float psi1 = t * rs;
                    bool valid = true;
                    if (BORDER) {
                        const int qx = x0 - 4 + e + j;
                        valid = qy >= 0 && qx >= 0 && qy + dy < H && qx + dx < W;
                        if (!valid) psi1 = 0.f;
                    }
                    pv[j] = psi1;
                    facc[i][j] = fmaf(gam, psi1, facc[i][j]);
                    const int oc = e + j - 4;
                    if (own_row && oc >= 0 && oc < TW && valid) A.jb = fmaf(gam, s * rs, A.jb);
                }
                st4v(PL + dx * DH * DW + n * DW + e, pv);
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NDI; ++i) {
            const int it = tid + i * NT;
            if (it >= ND) break;
            const int n = it / (DW / 4), e = 4 * (it - n * (DW / 4));
            if (n < dy) continue;   // q - d above the plane: q is outside the R region
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                if (dx == 0 && dy == 0) continue;
                const float gam = P.gamma[dy * 3 + dx];
                const float *row = PL + dx * DH * DW + (n - dy) * DW;
                float v[8];
                if (e >= 4) ld8(row + e - 4, v);
                else { ld4v(row + e, v + 4); v[0] = v[1] = v[2] = v[3] = 0.f; }
#pragma unroll
                for (int j = 0; j < 4; ++j) bacc[i][j] = fmaf(gam, v[4 + j - dx], bacc[i][j]);
            }
        }
        __syncthreads();
    }

    // r' = -(2 B^T E + lambda grad BTV) on the R region (origin (-2, -2)); owned r' to HBM
#pragma unroll
    for (int i = 0; i < NDI; ++i) {
        const int it = tid + i * NT;
        if (it >= ND) break;
        const int n = it / (DW / 4), e = 4 * (it - n * (DW / 4));
        const int gn = n - 2;           // R-region row
        if (gn < 0 || gn >= GH) continue;
        const int gy = y0 - 4 + n;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gc = e + j - 2;    // R-region column
            if (gc < 0 || gc >= GW) continue;
            const int gx = x0 - 4 + e + j;
            float rv = -fmaf(lambda, facc[i][j] - bacc[i][j], GB[gn * GW + gc]);
            if (BORDER && !(gy >= 0 && gy < H && gx >= 0 && gx < W)) rv = 0.f;
            GB[gn * GW + gc] = rv;
            const int orow = gn - 2, ocol = gc - 2;
            if (orow >= 0 && orow < TH && ocol >= 0 && ocol < TW && (!BORDER || (gy < H && gx < W))) {
                Rn[(size_t)gy * pitch + gx] = rv;
                const float rold = RB[(orow + 6) * XW + ocol + 8];
                const float pq = PB[(orow + 6) * XW + ocol + 8];
                A.rr = fmaf(rv, rv, A.rr);
                A.rrx = fmaf(rv, rold, A.rrx);
                A.pr = fmaf(pq, rv, A.pr);
            }
        }
    }
    __syncthreads();

    // --- E1: forward horizontal blurs of r' and p on rows [-2, TH+2) x owned cols
    float *HR = RB;   // r is dead now
    float *HP = SC;
    for (int it = tid; it < CH * CW / 4; it += NT) {
        const int n = it / (CW / 4), o = 4 * (it - n * (CW / 4));
        float inr[8], inp[8];
        ld8(GB + n * GW + o, inr);                    // r' at owned cols o-2 .. o+5
        ld8_off2(PB + (n + 4) * XW + o + 6, inp);     // p  at owned cols o-2 .. o+5
        float outr[4], outp[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float sr = 0.f, sp = 0.f;
#pragma unroll
            for (int b = -2; b <= 2; ++b) {
                float vr = inr[j + 2 - b], vp = inp[j + 2 - b];
                if (BORDER && !fwd_tap_ok(x0 + o + j, b, f)) { vr = 0.f; vp = 0.f; }
                sr = fmaf(hx[b + 2], vr, sr);
                sp = fmaf(hx[b + 2], vp, sp);
            }
            outr[j] = sr;
            outp[j] = sp;
        }
        st4v(HR + n * CW + o, outr);
        st4v(HP + n * CW + o, outp);
    }
    __syncthreads();

    // --- E2: curvature forms on the owned pixels, two rows x four columns per item
    for (int it = tid; it < (TH / 2) * (TW / 4); it += NT) {
        const int m = it / (TW / 4), o = 4 * (it - m * (TW / 4)), n = 2 * m;
        // data part: (B r')(c), (B p)(c) at sampled c, and J_data(x') - J_data(x)
        {
            float hr[6][4], hp[6][4];
#pragma unroll
            for (int i = 0; i < 6; ++i) { ld4v(HR + (n + i) * CW + o, hr[i]); ld4v(HP + (n + i) * CW + o, hp[i]); }
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int gy = y0 + n + rr;
                float ev[4];
                ld4v(YB + (n + rr + 4) * EW + o + 4, ev);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float zr = 0.f, zp = 0.f;
#pragma unroll
                    for (int a = -2; a <= 2; ++a) {
                        float vr = hr[rr + 2 - a][j], vp = hp[rr + 2 - a][j];
                        if (BORDER && !fwd_tap_ok(gy, a, f)) { vr = 0.f; vp = 0.f; }
                        zr = fmaf(hy[a + 2], vr, zr);
                        zp = fmaf(hy[a + 2], vp, zp);
                    }
                    if (smp[(n + rr) * TW + o + j]) {
                        A.ad = fmaf(zr, zr, A.ad);
                        A.bd = fmaf(zr, zp, A.bd);
                        A.cd = fmaf(zp, zp, A.cd);
                        const float azp = alpha * zp;
                        A.dj = fmaf(azp, fmaf(2.f, ev[j], -azp), A.dj);
                    }
                }
            }
        }
        // prior part: sum_d gamma_d psi''(t_d) (dv_d)(dw_d) over valid pairs
        float xq[2][4], rq[2][4], pq[2][4];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            float tmp[8];
            ld4v(XB + (n + rr + 6) * XW + o + 8, xq[rr]);
            ld4v(PB + (n + rr + 6) * XW + o + 8, pq[rr]);
            ld8(GB + (n + rr + 2) * GW + o, tmp);
#pragma unroll
            for (int j = 0; j < 4; ++j) rq[rr][j] = tmp[j + 2];
        }
#pragma unroll
        for (int pr = 0; pr < 4; ++pr) {   // partner row n + pr
            float xr[8], rrow[8], prow[8];
            ld8(XB + (n + pr + 6) * XW + o + 8, xr);
            ld8(PB + (n + pr + 6) * XW + o + 8, prow);
            ld8(GB + (n + pr + 2) * GW + o, rrow);
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int dy = pr - rr;
                if (dy < 0 || dy > 2) continue;
                const int gy = y0 + n + rr;
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    if (dx == 0 && dy == 0) continue;
                    const float gam = P.gamma[dy * 3 + dx];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (BORDER) {
                            const int gx = x0 + o + j;
                            if (!(gy + dy < H && gx + dx < W)) continue;
                        }
                        const float t = xq[rr][j] - xr[j + dx];
                        const float rs = rsqrtf(fmaf(t, t, eps2));
                        const float wgt = gam * rs * rs * rs;
                        const float dr = rq[rr][j] - rrow[j + 2 + dx];
                        const float dp = pq[rr][j] - prow[j + dx];
                        const float wdr = wgt * dr;
                        A.ab = fmaf(wdr, dr, A.ab);
                        A.bb = fmaf(wdr, dp, A.bb);
                        A.cb = fmaf(wgt * dp, dp, A.cb);
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// The fused SCG pass.  One CTA owns a TH x TW tile of the HR grid and, for the step
//   p = r + beta p_old,  x' = x + alpha p,
// computes on chip (halos recomputed, nothing but the owned pixels leaves the CTA):
//   E = B x' - Y, the objective J(x') and J_data(x') - J_data(x),
//   r' = -(2 B^T E + lambda grad BTV(x')),
//   and the curvature forms r'.H(x')r', r'.H(x')p, p.H(x')p of the next direction
//   p_next = r' + beta_next p, whose beta_next is only known after the pass:
//   p_next.H p_next = a + 2 beta_next b + beta_next^2 c.
// It writes x', r', p for its tile and FP64 partial sums; the last CTA of the pass runs the
// SCG scalar tail.  Traffic: reads x, r, p_old, Y, writes x', r', p = 28 bytes per HR px.
template <int TH, int TW, int NT>
__global__ void __launch_bounds__(NT, 2) scg_pass_kernel(const DevProblem *__restrict__ probs,
                                                         const int2 *__restrict__ tile_map, int mode,
                                                         double probe_alpha, double probe_beta) {
    using Gm = Geo<TH, TW>;
    constexpr int NWARP = NT / 32;
    extern __shared__ unsigned char smem_raw[];
    float *sm = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    unsigned char *smp = reinterpret_cast<unsigned char *>(sm + Gm::FLOATS);
    __shared__ __align__(8) uint64_t bar;
    __shared__ float red[NWARP][13];
    __shared__ int s_last, s_fail;

    const int2 tm = tile_map[blockIdx.x];
    const DevProblem &P = probs[tm.x];
    ScgState *st = P.st;
    if (ld_cg(&st->done)) return;

    const int tid = threadIdx.x;
    const int cur = ld_cg(&st->cur), pcur = ld_cg(&st->pcur);
    const float alpha = (float)(mode == MODE_PROBE ? probe_alpha : ld_cg(&st->alpha));
    const float beta = (float)(mode == MODE_PROBE ? probe_beta : ld_cg(&st->beta));
    const int y0 = (tm.y / P.tiles_x) * TH, x0 = (tm.y % P.tiles_x) * TW;

    // tile loads: x, r, p_old boxes (zero outside the image) and the Y box (NaN outside)
    if (tid == 0) {
        s_fail = 0;
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar, (uint32_t)Gm::TMA_BYTES);
        tma_load_2d(sm, &P.tmX[cur], x0 - 8, y0 - 6, &bar);
        tma_load_2d(sm + Gm::XH * Gm::XW, &P.tmP[pcur], x0 - 8, y0 - 6, &bar);
        tma_load_2d(sm + 2 * Gm::XH * Gm::XW, &P.tmR[cur], x0 - 8, y0 - 6, &bar);
        tma_load_2d(sm + 3 * Gm::XH * Gm::XW, &P.tmY, x0 - 4, y0 - 4, &bar);
    }
    if (!mbar_wait_bounded(&bar, 0, TMA_WAIT_TRIES)) s_fail = 1;
    __syncthreads();
    if (s_fail) {
        // the loads did not complete in time: flag the state and stop this projection
        if (tid == 0) {
            atomicExch(&st->status, (int)DEV_TMA_TIMEOUT);
            atomicExch(&st->done, 1);
            mbar_wait_bounded(&bar, 0, TMA_WAIT_TRIES);   // let copies in flight land
        }
        return;
    }

    PassAcc A = {};
    float *Xn = P.X[cur ^ 1], *Rn = P.Rv[cur ^ 1], *Pn = P.Pv[pcur ^ 1];
    const bool border = (y0 - 6 < 0) || (x0 - 8 < 0) || (y0 + TH + 6 > P.H) || (x0 + TW + 8 > P.W);
    if (border) pass_tile<TH, TW, NT, true>(P, sm, smp, y0, x0, alpha, beta, Xn, Rn, Pn, A);
    else pass_tile<TH, TW, NT, false>(P, sm, smp, y0, x0, alpha, beta, Xn, Rn, Pn, A);

    // --- FP32 warp sums, FP64 across warps, per-tile partials; the last CTA runs the tail
    float v[13] = {A.jd, A.dj, A.jb, A.rr, A.rrx, A.pr, A.pp, A.ad, A.bd, A.cd, A.ab, A.bb, A.cb};
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int j = 0; j < 13; ++j) {
        float x = v[j];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) red[warp][j] = x;
    }
    __syncthreads();
    if (tid < NPART) {
        const double lam_eps2 = (double)P.lambda * (double)P.eps2;
        double s0 = 0, s1 = 0;
        const int j0 = tid < 7 ? tid : 7 + (tid - 7);   // data part index
        for (int w = 0; w < NWARP; ++w) {
            s0 += (double)red[w][j0];
            if (tid >= 7) s1 += (double)red[w][tid + 3];
        }
        const double val = tid < 7 ? s0 : 2.0 * s0 + lam_eps2 * s1;
        P.partials[(size_t)tm.y * NPART + tid] = val;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned int done_tiles = atomicAdd(P.counter, 1u);
        s_last = (done_tiles == (unsigned)(P.n_tiles - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // fixed-order FP64 sum over tiles: thread t sums tiles t, t+NT, ...; then a fixed tree
    __shared__ double redd[NWARP][NPART];
    double tot[NPART];
#pragma unroll
    for (int j = 0; j < NPART; ++j) tot[j] = 0.0;
    for (int t = tid; t < P.n_tiles; t += NT) {
#pragma unroll
        for (int j = 0; j < NPART; ++j) tot[j] += ld_cg(&P.partials[(size_t)t * NPART + j]);
    }
#pragma unroll
    for (int j = 0; j < NPART; ++j) {
        double x = tot[j];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) redd[warp][j] = x;
    }
    __syncthreads();
    if (tid == 0) {
        double S[NPART];
        for (int j = 0; j < NPART; ++j) {
            double s = 0;
            for (int w = 0; w < NWARP; ++w) s += redd[w][j];
            S[j] = s;
        }
        scg_tail(P, st, S, mode);
        *P.counter = 0u;
        __threadfence();
    }
}

// ---------------------------------------------------------------------------------------
// prepare: interleave the K frames into Y on the HR grid (converting u16 counts to line
// integrals), write the start point x_1 into X[0], zero r and p_0, and reset the state.
// flags: 1 = write x0, 2 = zero R[0] and P[0], 4 = reset the SCG state.  x_given is dense
// (row pitch W); the workspace images use P.pitch.
__global__ void prepare_kernel(const DevProblem *__restrict__ probs, int pidx, const void *__restrict__ y_in,
                               int in_dtype, float log_i0, const float *__restrict__ x_given, int x0_mode,
                               int flags) {
    const DevProblem &P = probs[pidx];
    const int H = P.H, W = P.W, f = P.f, pitch = P.pitch;
    const size_t n = (size_t)H * pitch;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (flags & 4)) {
        ScgState *st = P.st;
        st->cur = 0; st->pcur = 0; st->done = 0; st->iter = 0; st->accepted = 0;
        st->status = 0; st->alpha = 0.0; st->beta = 0.0; st->success = 1;
        st->lam = 1e-6; st->lam_bar = 0.0; st->iters = P.iters;
        *P.counter = 0u;
    }
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int cy = (int)(o / pitch), cx = (int)(o - (size_t)cy * pitch);
        float yv = __int_as_float(0x7fc00000);  // NaN: no frame samples this pixel
        float x0 = 0.f;
        if (cx < W) {
            const int k = P.frame_of_phase[(cy % f) * f + (cx % f)];
            if (k >= 0) {
                const size_t li = (size_t)k * P.h * P.w + (size_t)(cy / f) * P.w + (cx / f);
                if (in_dtype == 1) {
                    const unsigned short c = ((const unsigned short *)y_in)[li];
                    yv = log_i0 - logf((float)(c < 1 ? 1 : c));
                } else {
                    yv = ((const float *)y_in)[li];
                }
            }
            if (x0_mode == 1) x0 = (k >= 0) ? yv : 0.f;
            else if (x0_mode == 2) x0 = x_given[(size_t)cy * W + cx];
        }
        P.Y[o] = yv;
        if (flags & 1) P.X[0][o] = x0;
        if (flags & 2) {
            P.Rv[0][o] = 0.f;
            P.Pv[0][o] = 0.f;
        }
    }
}

// y_k(i, j) = (D B M_k x)(i, j) with the separable PSF; x dense (row pitch W); one thread
// per LR pixel and frame.
__global__ void forward_kernel(const DevProblem *__restrict__ probs, int pidx, const float *__restrict__ x,
                               float *__restrict__ y) {
    const DevProblem &P = probs[pidx];
    const int H = P.H, W = P.W, f = P.f, h = P.h, w = P.w;
    const size_t m = (size_t)h * w;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < m * P.K; t += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(t / m);
        const size_t li = t - (size_t)k * m;
        const int i = (int)(li / w), j = (int)(li - (size_t)i * w);
        const int cy = f * i + P.ty[k], cx = f * j + P.tx[k];
        float acc = 0.f;
        for (int a = -PSF_R; a <= PSF_R; ++a) {
            const int u = cy - a;
            if (u < P.ty[k] || u >= H) continue;   // B's zero padding in front of M_k / x outside
            float row = 0.f;
            for (int b = -PSF_R; b <= PSF_R; ++b) {
                const int v = cx - b;
                if (v < P.tx[k] || v >= W) continue;
                row = fmaf(P.hx[b + PSF_R], x[(size_t)u * W + v], row);
            }
            acc = fmaf(P.hy[a + PSF_R], row, acc);
        }
        y[t] = acc;
    }
}

// out (dense) = x_k, the iterate the state points at (end of a solve)
__global__ void finalize_kernel(const DevProblem *__restrict__ probs, int pidx, float *__restrict__ out) {
    const DevProblem &P = probs[pidx];
    const size_t n = (size_t)P.H * P.W;
    const float *src = P.X[ld_cg(&P.st->cur)];
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(o / P.W), x = (int)(o - (size_t)y * P.W);
        out[o] = src[(size_t)y * P.pitch + x];
    }
}

// out (dense, row pitch W) = sign * src (row pitch `pitch`)
__global__ void scale_copy_kernel(const float *__restrict__ src, int pitch, float sign, float *__restrict__ out,
                                  int H, int W) {
    const size_t n = (size_t)H * W;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(o / W), x = (int)(o - (size_t)y * W);
        out[o] = sign * src[(size_t)y * pitch + x];
    }
}

}  // namespace misr
