// Types shared by the device code and the host side of the sm_103a MISR solver: compile-time
// limits, the per-projection SCG state and the problem record the kernels read.
//
// Model (Sec. 3.1 of the paper): y_k = D B M_k x (Eq. 1), J(x) = sum_k ||A_k x - y_k||^2 +
// lambda * BTV(x) (Eq. 6, 8, 9), solved with Moller's scaled conjugate gradient (Algorithm 1).
// The L1 data term of the paper's experiments replaces ||e||^2 by sum_i psi_d(e_i),
// psi_d(t) = sqrt(t^2 + data_eps^2) - data_eps.
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
#include <stdint.h>

namespace misr {

constexpr int MAXK = 64;
constexpr int MAXF = 8;
constexpr int PSF_R = 2;   // compiled PSF radius (5x5 taps); smaller PSFs are zero-padded
constexpr int BTV_W = 3;   // compiled BTV window; smaller windows get gamma = 0
constexpr int NPART = 10;
constexpr int TRACE_COLS = 10;
constexpr uint32_t TMA_WAIT_TRIES = 1u << 24;   // bounded wait for the tile loads

// Shapes of the fused pass.  Tile shapes 0..2: TH x TW HR pixels per tile, NT threads per CTA
// (1024 / NT CTAs resident per SM).  STREAM_SHAPE: the row-streaming kernel, whose work item is
// a strip of SHAPE_TW = 112 columns by a height chosen per plan (SHAPE_TH 0: at run time), one
// warp each, NT = 256 threads (8 independent warps) per CTA.  The autotuner picks one per HR
// image size.  STREAM_LEFT_COST, STREAM_TOP_COST: time per row step of a streaming item of the
// left strip and of a top item, both on the path compiled with the border corrections,
// relative to an item on the interior path (per-warp globaltimer spans at 4096^2 HR: 2.56 and
// about 1.5 against 1.78 us per step), for the split of the items between the two paths.
constexpr int N_SHAPES = 4;
constexpr int N_TILE_SHAPES = 3;
constexpr int STREAM_SHAPE = 3;
constexpr int SHAPE_TH[N_SHAPES] = {32, 32, 16, 0};
constexpr int SHAPE_TW[N_SHAPES] = {64, 32, 64, 112};
constexpr int SHAPE_NT[N_SHAPES] = {512, 256, 256, 256};
constexpr double STREAM_LEFT_COST = 1.45, STREAM_TOP_COST = 1.0;
// Compiled variants of the fused pass per shape: bit 0 r and p stored as bf16, bit 1 the
// smoothed L1 data term, bit 2 per-phase blur taps (non-integer shifts; compiled for the
// 32x32 shape only).  The streaming shape has variants 0 to 3 (shared taps).
constexpr int N_VARIANTS = 8;
constexpr int PHASED_SHAPE = 1;
// per-phase tap tables of DevProblem::tph: full y taps, y taps of the bilinear's first part
// alone (the top border), full x taps, x taps of the first part alone (the left border), and
// the adjoint's full taps by output phase: AF[p][c + R] = F[(p + c) mod f][c + R] (the taps
// of the sample an adjoint tap c reads, from an output of phase p)
enum { TPH_FY = 0, TPH_PY = 1, TPH_FX = 2, TPH_PX = 3, TPH_AFY = 4, TPH_AFX = 5, N_TPH = 6 };

// partial sums of one pass (FP64)
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
    float alpha_f, beta_f;   // alpha and beta rounded once for the FP32 pass
};

struct DevProblem {
    CUtensorMap tmX[2], tmR[2], tmP[2], tmY;      // TMA maps of the workspace images
    int H, W, pitch, f, h, w, K;
    int tiles_x, tiles_y, n_tiles, iters;
    int rp_bf16;                                  // r and p stored as bf16 (x stays float)
    int l1;                                       // data term: 0 squared L2, 1 smoothed L1
    int phased;                                   // non-integer shifts: blur taps per phase
    int shape, tile_h, tile_w;                    // tile shape (index into SHAPE_*) and its size
    // Streaming shape: the edge items come first, the n_left items of the left strip (edge_h
    // rows each) and the n_top items at the top of the other strips (rows [0, edge_h)); then
    // those strips' remaining rows in items of tile_h rows (tiles_y per strip).  Only the edge
    // items meet the frame masks of the top and left borders.  edge_ctas: CTAs of a launch
    // over this problem alone that start on the edge items.
    int n_left, n_top, edge_h, edge_ctas;
    int wait_tries;                               // polls before a tile load is reported late
    float hy[2 * PSF_R + 1], hx[2 * PSF_R + 1];  // separable PSF, h(a, b) = hy[a+R] hx[b+R]
    float lambda, eps, eps2, data_eps;            // data_eps: the L1 data term's smoothing
    float gamma[BTV_W * BTV_W];                   // gamma(dx, dy) at [dy * BTV_W + dx]
    double eps_pairs;                             // eps * sum_d gamma_d * #pairs_d
    float *X[2], *Rv[2], *Pv[2];                  // x, r (double buffered), p (double buffered);
                                                  // Rv, Pv hold __nv_bfloat16 when rp_bf16
    float *Y;                                     // interleaved frames, NaN where unsampled
    // Fixed-order reduction of a pass's sums: every tile writes its sums; one warp per group of
    // `group` tiles sums the group in tile order, and the warp that finishes the last group sums
    // the groups in order and runs the SCG tail.  The tile kernel leaves this to reduce_kernel
    // after the pass; in the streaming pass the warp that completes a group does it.
    // Field-major arrays.
    float2 *partials;                             // [NPART][n_tiles] tile sums (hi, lo)
    float2 *gpartials;                            // [NPART][n_groups] group sums (hi, lo)
    unsigned int *counter;                        // groups finished in the current pass
    unsigned int *gcounter;                       // [n_groups] items finished per group (the
                                                  // streaming pass reduces in the pass itself)
    int group, n_groups;                          // tiles per group, groups
    ScgState *st;
    double *trace;                                // [iters][TRACE_COLS]
    int ty[MAXK], tx[MAXK];
    int frame_of_phase[MAXF * MAXF];              // -1: no frame samples that phase
    // non-integer shifts: fractional HR shift per row phase (ay) and column phase (ax), and
    // the blur taps per phase, tph[table][phase][c + PSF_R] for tap c in [-PSF_R, PSF_R]
    // (8 floats per phase so that a phase's taps start on a 16-byte boundary)
    float ay[MAXF], ax[MAXF];
    float tph[N_TPH][MAXF][8];
    // Frame-wise pass (general: the frames do not interleave into one HR image: several frames
    // on one phase, shifts outside [0, f), shifts off a product lattice, or a combined blur
    // wider than the compiled taps).  Frame k's operator is separable, A_k = G_y,k (x) G_x,k:
    // LR sample (i, j) reads x at rows f i + ty[k] - g_r + dy and columns f j + tx[k] - g_r + dx,
    // dy, dx in [0, g_tw), with weights Ty[k][i][dy] Tx[k][j][dx] that hold B, D, the bilinear
    // weights of M_k and every mask (ty, tx: the integer parts floor(t) of the HR shifts, any
    // sign; gfy, gfx: the fractional parts).  Each of the pass's kernels runs g_ctas CTAs (the
    // last one 2 g_ctas) and writes one tile of sums per CTA: n_tiles = GEN_TILES * g_ctas.
    int general, g_tw, g_r, g_nb, g_ctas;         // g_nb: the block side of D (f with binning, else 1)
    float gfy[MAXK], gfx[MAXK];                   // and 1 minus them, each rounded once from FP64
    float gfy0[MAXK], gfx0[MAXK];
    float *Yg;                                    // [K][h][w] frames (float; u16 converted)
    float *Ty, *Tx;                               // [K][h][g_tw], [K][w][g_tw] tap tables
    float *Eg;                                    // [K][h][w] DS psi_d'(e') of the trial point
    float *APg;                                   // [K][h][w] A_k p
    float *Wg;                                    // [K][h][w] psi_d''(e') (L1 data term)
    float *Tg;                                    // [K][h][W] the adjoint's horizontal part
    float *Hg[2];                                 // [K][H][w] the forward's horizontal parts
};
// taps per axis of a frame's D B M_k at most (binning f, PSF 2 PSF_R + 1, bilinear + 1); tiles
// of sums per CTA of the frame-wise pass's kernels
constexpr int GEN_TW = MAXF + 2 * PSF_R + 1;
constexpr int GEN_TILES = 5;

// Per-launch constants of the streaming pass (every problem of one launch shares them; the
// host splits launches where they differ).  They are kernel parameters, so the arithmetic
// reads them from the constant bank instead of holding them in registers.
struct StreamConsts {
    float hx[2 * PSF_R + 1], hy[2 * PSF_R + 1];   // forward taps, tap b at [b + R]
    float gam[BTV_W * BTV_W];                     // gamma(dx, dy) at [dy * 3 + dx]
    float lgam[BTV_W * BTV_W];                    // lambda gamma: the psi'' weight of a pair
    float eps2, lambda;
    float deps, deps2;                            // the L1 data term's smoothing eps_d and eps_d^2
    int f;
    unsigned fmag;                                // ceil(2^32 / f) (0 for f = 1), for c mod f
};

}  // namespace misr
