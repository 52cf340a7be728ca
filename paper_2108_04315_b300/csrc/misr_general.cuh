// The frame-wise SCG pass (sm_103a): the data term frame by frame, for frame sets that do not
// interleave into one HR image (several frames on one HR phase, such as the synthetic study's
// one-pixel shifts right, down, left and up, Sec. 4.1.1; shifts outside [0, f) HR pixels; non-
// integer shifts off a product lattice; a combined D B blur wider than the fused kernels'
// taps).  Included by misr_device.cuh.
//
// Model (Eq. 1, reading of M_k as bilinear interpolation for non-integer shifts): per axis,
// LR index i of frame k reads B's output at f i + a' (a' < f with binning, else 0), B's input
// pixel s = f i + a' - a for PSF tap a (s inside the grid: B's zero padding), and x at s + t_k
// + q, q in {0, 1} with the bilinear weights (x inside the grid).  Everything but x is a weight
// that depends on (k, i) alone, so A_k is separable, A_k x (i, j) = sum_{dy, dx} Ty[k][i][dy]
// Tx[k][j][dx] x(f i + ty_k - R + dy, f j + tx_k - R + dx), with the tables built on the host
// in FP64 from those definitions.  A_k^T gathers the same weights: HR pixel u takes the LR
// rows i with 0 <= u - (f i + ty_k - R) < g_tw.
//
// One pass computes what the fused pass computes (p = r + beta p_old, x' = x + alpha p,
// r' = -grad J(x'), and the ten sums J_data(x'), J_data(x') - J_data(x), R_BTV(x') + eps
// pairs, |r'|^2, r'.r, p.r', |p|^2, r'.H r', r'.H p, p.H p), in seven kernels:
//   gen_pass_a  (HR)  p, x', the BTV value and lambda grad BTV(x') into r's buffer; |p|^2
//   gen_pass_f1 (HR rows x LR columns)  the forward's horizontal part of x' and p, every frame
//   gen_pass_b  (LR)  its vertical part, A_k x', A_k p: the residual, J_data, dJ_data, the data
//                     part of p.H p; DS psi_d'(e'), A_k p and psi_d''(e') kept per sample
//   gen_pass_c1 (LR rows x HR columns)  the adjoint's horizontal part of every frame
//   gen_pass_c2 (HR)  its vertical part, r' = -(A^T DS psi_d' + lambda grad BTV); |r'|^2, r'.r, p.r'
//   gen_pass_f1 (HR rows x LR columns)  the forward's horizontal part of r'
//   gen_pass_d  (LR)  its vertical part, A_k r': the data parts of r'.H r' and r'.H p;
//               (HR)  the BTV parts of the three curvature forms (second half of its CTAs)
// then reduce_kernel sums the tiles and runs the SCG tail.  Each CTA writes one tile of sums
// (every field, zero where the kernel has no part), so the tail sees the same fields; a kernel
// runs at most g_ctas CTAs per role (as many as are resident at once), and the slots of CTAs it
// does not run hold the zeros the plan's workspace starts with.
// Per-thread sums are FP32 over the thread's grid-stride elements, the CTA sums FP64.
#pragma once

namespace misr {

constexpr int GEN_NT = 256;

// Checks of the bounds-checked build (MISR_BOUNDS_CHECK) on the frame-wise pass: the tap index
// of every adjoint gather (its LR row or column range comes from the division-free floor
// division) and every CTA's tile slot of sums (each role owns g_ctas slots).
enum GenBoundsCode { BC_GEN_TAP = 16, BC_GEN_TILE = 17 };

// floor(a / f) without a division, for a in [-2^21, 2^22] and 1 <= f <= 8: a + f 2^21 >= 0, and with
// m = ceil(2^32 / f), floor(n m / 2^32) = floor(n / f) for n < 2^25 (the error n (m f - 2^32) /
// (f 2^32) stays below 1 / f).  m = gen_fdiv_magic(f); f = 1 needs no division.
constexpr int GEN_DIV_OFF = 1 << 21;
__device__ __forceinline__ unsigned gen_fdiv_magic(int f) {
    return f > 1 ? (unsigned)((0x100000000ull + (unsigned)f - 1) / (unsigned)f) : 0u;
}
__device__ __forceinline__ int gen_fdiv(int a, int f, unsigned m) {
    return f == 1 ? a : (int)__umulhi((unsigned)(a + f * GEN_DIV_OFF), m) - GEN_DIV_OFF;
}

struct GenStep {
    int cur, pcur, done;
    float alpha, beta;
};
__device__ __forceinline__ GenStep gen_step(const DevProblem &P, int mode, double probe_alpha, double probe_beta) {
    GenStep g;
    g.done = ld_cg(&P.st->done);
    g.cur = ld_cg(&P.st->cur);
    g.pcur = ld_cg(&P.st->pcur);
    g.alpha = mode == MODE_PROBE ? (float)probe_alpha : __ldcg(&P.st->alpha_f);
    g.beta = mode == MODE_PROBE ? (float)probe_beta : __ldcg(&P.st->beta_f);
    return g;
}

// One tile of sums: the CTA's NF per-thread values of fields fld[] summed in FP64 in a fixed
// order (warp butterfly, then the warps in order), every other field zero.  Every thread of the
// CTA calls it.  tile = role * g_ctas + slot, slot < g_ctas.
template <int NF>
__device__ __forceinline__ void gen_write_sums(const DevProblem &P, int role, int slot, const int (&fld)[NF],
                                               const float (&v)[NF]) {
    const int tile = role * P.g_ctas + slot;
    __shared__ double red[GEN_NT / 32][NPART];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NF; ++j) {
        double d = (double)v[j];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
        if (lane == 0) red[warp][j] = d;
    }
    __syncthreads();
    if (threadIdx.x < NPART &&
        MISR_IN_BOUNDS(slot >= 0 && slot < P.g_ctas && tile < P.n_tiles, BC_GEN_TILE, role, slot)) {
        double s = 0.0;
        for (int j = 0; j < NF; ++j)
            if (fld[j] == (int)threadIdx.x)
                for (int w = 0; w < GEN_NT / 32; ++w) s += red[w][j];
        const float hi = (float)s, lo = (float)(s - (double)hi);
        P.partials[(size_t)threadIdx.x * P.n_tiles + tile] = make_float2(hi, lo);
    }
}

// A_k of one LR sample over two HR images a and b (row pitch `pitch`): (A_k a, A_k b)
__device__ __forceinline__ float2 gen_apply2(const DevProblem &P, int k, int i, int j, const float *__restrict__ a,
                                             const float *__restrict__ b, int pitch) {
    const int tw = P.g_tw, H = P.H, W = P.W;
    const float *ty = P.Ty + ((size_t)k * P.h + i) * tw, *tx = P.Tx + ((size_t)k * P.w + j) * tw;
    const int oy = P.f * i + P.ty[k] - P.g_r, ox = P.f * j + P.tx[k] - P.g_r;
    float za = 0.f, zb = 0.f;
    for (int dy = 0; dy < tw; ++dy) {
        const int u = oy + dy;
        const float wy = ty[dy];
        if (u < 0 || u >= H || wy == 0.f) continue;
        float ra = 0.f, rb = 0.f;
        for (int dx = 0; dx < tw; ++dx) {
            const int v = ox + dx;
            if (v < 0 || v >= W) continue;
            const float wx = tx[dx];
            const size_t o = (size_t)u * pitch + v;
            ra = fmaf(wx, a[o], ra);
            if (b) rb = fmaf(wx, b[o], rb);
        }
        za = fmaf(wy, ra, za);
        zb = fmaf(wy, rb, zb);
    }
    return make_float2(za, zb);
}

// Multi-image interpolation at HR pixel (u, v) for any shift set: sum_k M_k^T D^T y_k over
// sum_k M_k^T D^T 1 with point sampling (0 where no weight falls).  The sample (i, j) of frame
// k sits at B's input pixel (f i, f j) and spreads over x at (f i + ty_k + p, f j + tx_k + q),
// p, q in {0, 1}, with the bilinear weights; so (u, v) gathers the samples with
// f i = u - ty_k - p and f j = v - tx_k - q.
__device__ float gen_shift_add(const DevProblem &P, const void *__restrict__ y_in, int in_dtype, float log_i0, int u,
                               int v) {
    const int f = P.f;
    const size_t m = (size_t)P.h * P.w;
    float num = 0.f, den = 0.f;
    for (int k = 0; k < P.K; ++k) {
        for (int p = 0; p < 2; ++p) {
            const float wy = p ? P.gfy[k] : P.gfy0[k];
            const int fi = u - P.ty[k] - p;
            if (wy == 0.f || fi < 0 || fi % f != 0 || fi / f >= P.h) continue;
            for (int q = 0; q < 2; ++q) {
                const float wx = q ? P.gfx[k] : P.gfx0[k];
                const int fj = v - P.tx[k] - q;
                if (wx == 0.f || fj < 0 || fj % f != 0 || fj / f >= P.w) continue;
                const float wgt = wy * wx;
                num = fmaf(wgt, frame_value(y_in, in_dtype, log_i0, (size_t)k * m + (size_t)(fi / f) * P.w + fj / f), num);
                den += wgt;
            }
        }
    }
    return den > 0.f ? num / den : 0.f;
}

// prepare (frame-wise problems): the frames into Yg (u16 counts converted), the start point
// into X[0], r and p_0 zeroed, the state reset; flags as prepare_kernel's.
__global__ void __launch_bounds__(GEN_NT) gen_prepare_kernel(const DevProblem *__restrict__ probs, int pidx,
                                                             const void *__restrict__ y_in, int in_dtype, float log_i0,
                                                             const float *__restrict__ x_given, int x0_mode, int flags) {
    const DevProblem &P = probs[pidx];
    const int H = P.H, W = P.W, pitch = P.pitch;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (flags & 4)) {
        ScgState *st = P.st;
        st->cur = 0; st->pcur = 0; st->done = 0; st->iter = 0; st->accepted = 0;
        st->status = 0; st->alpha = 0.0; st->beta = 0.0; st->success = 1;
        st->alpha_f = 0.f; st->beta_f = 0.f;
        st->lam = 1e-6; st->lam_bar = 0.0; st->iters = P.iters;
        *P.counter = 0u;
    }
    const size_t stride = (size_t)gridDim.x * blockDim.x, t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t m = (size_t)P.K * P.h * P.w;
    for (size_t t = t0; t < m; t += stride) P.Yg[t] = frame_value(y_in, in_dtype, log_i0, t);
    const size_t n = (flags & 3) ? (size_t)H * pitch : 0;
    for (size_t o = t0; o < n; o += stride) {
        const int u = (int)(o / pitch), v = (int)(o - (size_t)u * pitch);
        float x0 = 0.f;
        if (v < W) {
            if (x0_mode == 1) x0 = gen_shift_add(P, y_in, in_dtype, log_i0, u, v);
            else if (x0_mode == 2) x0 = x_given[(size_t)u * W + v];
        }
        if (flags & 1) P.X[0][o] = x0;
        if (flags & 2) {
            P.Rv[0][o] = 0.f;
            P.Pv[0][o] = 0.f;
        }
    }
}

// y_k(i, j) = (D B M_k x)(i, j), x dense (row pitch W): one thread per LR sample and frame
__global__ void __launch_bounds__(GEN_NT) gen_forward_kernel(const DevProblem *__restrict__ probs, int pidx,
                                                             const float *__restrict__ x, float *__restrict__ y) {
    const DevProblem &P = probs[pidx];
    const size_t m = (size_t)P.h * P.w;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < m * P.K; t += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(t / m);
        const size_t li = t - (size_t)k * m;
        const int i = (int)(li / P.w), j = (int)(li - (size_t)i * P.w);
        y[t] = gen_apply2(P, k, i, j, x, nullptr, P.W).x;
    }
}

// multi-image interpolation (frame-wise problems), out dense
__global__ void __launch_bounds__(GEN_NT) gen_interpolate_kernel(const DevProblem *__restrict__ probs, int pidx,
                                                                 const void *__restrict__ y_in, int in_dtype,
                                                                 float log_i0, float *__restrict__ out) {
    const DevProblem &P = probs[pidx];
    const size_t n = (size_t)P.H * P.W;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
        const int u = (int)(o / P.W), v = (int)(o - (size_t)u * P.W);
        out[o] = gen_shift_add(P, y_in, in_dtype, log_i0, u, v);
    }
}

// HR tiles of the prior's stencils: GEN_TILE_H x GEN_TILE_W owned pixels, staged in shared memory
// with a halo of BTV_W - 1 pixels (both sides for the gradient, the far side for the forms)
constexpr int GEN_TILE_H = 16, GEN_TILE_W = 64, GEN_HALO = BTV_W - 1;
constexpr int GEN_RH = GEN_TILE_H + 2 * GEN_HALO, GEN_RW = GEN_TILE_W + 2 * GEN_HALO;
constexpr int GEN_FH = GEN_TILE_H + GEN_HALO, GEN_FW = GEN_TILE_W + GEN_HALO;
static_assert(GEN_TILE_H * GEN_TILE_W % GEN_NT == 0, "owned pixels per thread");

// A: p = r + beta p_old, x' = x + alpha p (to the other halves of the double buffers); the BTV
// prior at x': each pixel q takes the pairs (q, q + d) and (q - d, q) of every offset d of the
// window (Eq. 8), its gradient gamma_d psi'(x'_q - x'_{q+d}) - gamma_d psi'(x'_{q-d} - x'_q),
// and the value of the pairs it starts, gamma_d sqrt(t^2 + eps^2).  Per HR tile, x' of the tile
// and its halo is formed once into shared memory (0 outside the image, where no pair reads).
// lambda grad BTV(x') goes to r's buffer, which gen_pass_c2 completes to r'.  Tile blockIdx.x:
// |p|^2, the BTV value.
__global__ void __launch_bounds__(GEN_NT) gen_pass_a(const DevProblem *__restrict__ probs, int pidx, int mode,
                                                     double probe_alpha, double probe_beta) {
    __shared__ float xs[GEN_RH * GEN_RW];
    __shared__ float ps[GEN_TILE_H * GEN_TILE_W];
    const DevProblem &P = probs[pidx];
    const GenStep s = gen_step(P, mode, probe_alpha, probe_beta);
    if (s.done) return;
    const float *__restrict__ X = P.X[s.cur];
    const float *__restrict__ R = P.Rv[s.cur];
    const float *__restrict__ Po = P.Pv[s.pcur];
    float *__restrict__ Xn = P.X[s.cur ^ 1];
    float *__restrict__ Rn = P.Rv[s.cur ^ 1];
    float *__restrict__ Pn = P.Pv[s.pcur ^ 1];
    const int H = P.H, W = P.W, pitch = P.pitch;
    const float alpha = s.alpha, beta = s.beta, eps2 = P.eps2, lam = P.lambda;
    float gm[BTV_W * BTV_W];
#pragma unroll
    for (int d = 0; d < BTV_W * BTV_W; ++d) gm[d] = P.gamma[d];
    const int tiles_x = (W + GEN_TILE_W - 1) / GEN_TILE_W, n_t = tiles_x * ((H + GEN_TILE_H - 1) / GEN_TILE_H);
    float pp = 0.f, jb = 0.f;
    for (int t = blockIdx.x; t < n_t; t += gridDim.x) {
        const int y0 = (t / tiles_x) * GEN_TILE_H, x0 = (t % tiles_x) * GEN_TILE_W;
        for (int e = threadIdx.x; e < GEN_RH * GEN_RW; e += GEN_NT) {
            const int ry = e / GEN_RW, rx = e - ry * GEN_RW, u = y0 - GEN_HALO + ry, v = x0 - GEN_HALO + rx;
            float xv = 0.f, pv = 0.f;
            if (u >= 0 && u < H && v >= 0 && v < W) {
                const size_t o = (size_t)u * pitch + v;
                pv = fmaf(beta, Po[o], R[o]);
                xv = fmaf(alpha, pv, X[o]);
            }
            xs[e] = xv;
            const int oy = ry - GEN_HALO, ox = rx - GEN_HALO;
            if (oy >= 0 && oy < GEN_TILE_H && ox >= 0 && ox < GEN_TILE_W) ps[oy * GEN_TILE_W + ox] = pv;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < GEN_TILE_H * GEN_TILE_W / GEN_NT; ++q) {
            const int e = (int)threadIdx.x + GEN_NT * q, oy = e / GEN_TILE_W, ox = e - oy * GEN_TILE_W;
            const int u = y0 + oy, v = x0 + ox;
            if (u >= H || v >= W) continue;
            const float *c = xs + (oy + GEN_HALO) * GEN_RW + ox + GEN_HALO;
            const float xq = c[0], p = ps[e];
            pp = fmaf(p, p, pp);
            float g = 0.f, jq = 0.f;
#pragma unroll
            for (int dy = 0; dy < BTV_W; ++dy)
#pragma unroll
                for (int dx = 0; dx < BTV_W; ++dx) {
                    const float gd = gm[dy * BTV_W + dx];
                    if ((dx | dy) == 0 || gd == 0.f) continue;
                    if (u + dy < H && v + dx < W) {
                        const float d = xq - c[dy * GEN_RW + dx], q2 = fmaf(d, d, eps2), rq = rsqrtf(q2);
                        g = fmaf(gd, d * rq, g);
                        jq = fmaf(gd, q2 * rq, jq);   // sqrt(t^2 + eps^2)
                    }
                    if (u >= dy && v >= dx) {
                        const float d = c[-dy * GEN_RW - dx] - xq, q2 = fmaf(d, d, eps2);
                        g = fmaf(-gd, d * rsqrtf(q2), g);
                    }
                }
            jb += jq;
            const size_t o = (size_t)u * pitch + v;
            Xn[o] = xq;
            Pn[o] = p;
            Rn[o] = lam * g;
        }
        __syncthreads();
    }
    const int fld[2] = {P_PP, P_JB};
    const float val[2] = {pp, jb};
    gen_write_sums<2>(P, 0, (int)blockIdx.x, fld, val);
}

// The forward operator in two stages (no shared memory).  F1, the horizontal part for every HR
// row u of every frame and every LR column j: Hg[0][k][u][j] = sum_dx Tx[k][j][dx] a(u, f j + ox_k
// + dx) over the columns inside the grid (ox_k = tx_k - R), and Hg[1] the same of b (TWO: a = x',
// b = p for B; else a = r' for D).  F2, in B and D: the vertical part for the LR sample (i, j),
// sum_dy Ty[k][i][dy] Hg[k][f i + oy_k + dy][j] over the rows inside the grid.  Items: GEN_SEG
// columns of one row, thread t taking columns c0 + t + GEN_NT q, q < 4.
constexpr int GEN_SEG = 4 * GEN_NT;
template <int TWM, bool TWO>
__global__ void __launch_bounds__(GEN_NT) gen_pass_f1(const DevProblem *__restrict__ probs, int pidx, int mode,
                                                      double probe_alpha, double probe_beta) {
    const DevProblem &P = probs[pidx];
    const GenStep s = gen_step(P, mode, probe_alpha, probe_beta);
    if (s.done) return;
    const float *__restrict__ a = TWO ? P.X[s.cur ^ 1] : P.Rv[s.cur ^ 1];
    const float *__restrict__ b = P.Pv[s.pcur ^ 1];
    const int f = P.f, H = P.H, W = P.W, w = P.w, tw = P.g_tw, pitch = P.pitch;
    const int segs = (w + GEN_SEG - 1) / GEN_SEG, items = H * segs;
    // items by HR row segment, every frame inside: the frames' reads of the row hit L1
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int u = it / segs, c0 = (it - u * segs) * GEN_SEG;
        const float *__restrict__ ar = a + (size_t)u * pitch;
        const float *__restrict__ br = b + (size_t)u * pitch;
        for (int k = 0; k < P.K; ++k) {
            const int ox = P.tx[k] - P.g_r;
            const float *__restrict__ Txk = P.Tx + (size_t)k * w * tw;
            float *__restrict__ ha = P.Hg[0] + ((size_t)k * H + u) * w;
            float *__restrict__ hb = P.Hg[1] + ((size_t)k * H + u) * w;
#pragma unroll
            for (int q = 0; q < GEN_SEG / GEN_NT; ++q) {
                const int j = c0 + (int)threadIdx.x + GEN_NT * q;
                if (j >= w) continue;
                const int v0 = f * j + ox;
                float sa = 0.f, sb = 0.f;
#pragma unroll
                for (int dx = 0; dx < TWM; ++dx) {
                    const int v = v0 + dx;
                    if (dx < tw && v >= 0 && v < W) {
                        const float wx = __ldg(Txk + j * tw + dx);
                        sa = fmaf(wx, ar[v], sa);
                        if (TWO) sb = fmaf(wx, br[v], sb);
                    }
                }
                ha[j] = sa;
                if (TWO) hb[j] = sb;
            }
        }
    }
}

// The vertical part of A_k for the samples of LR row i of frame k (columns c0 + t + GEN_NT q):
// the row's taps once, then per column its rows of Hg[0] (and Hg[1]).
template <int TWM, bool TWO>
__device__ __forceinline__ void gen_f2_row(const DevProblem &P, int k, int i, int c0, float (&za)[GEN_SEG / GEN_NT],
                                           float (&zb)[GEN_SEG / GEN_NT]) {
    const int f = P.f, H = P.H, w = P.w, tw = P.g_tw;
    const int u0 = f * i + P.ty[k] - P.g_r;
    const float *Tyi = P.Ty + ((size_t)k * P.h + i) * tw;
#pragma unroll
    for (int q = 0; q < GEN_SEG / GEN_NT; ++q) { za[q] = 0.f; zb[q] = 0.f; }
#pragma unroll
    for (int dy = 0; dy < TWM; ++dy) {
        const int u = u0 + dy;
        if (dy >= tw || u < 0 || u >= H) continue;
        const float wy = __ldg(Tyi + dy);
        const float *__restrict__ ha = P.Hg[0] + ((size_t)k * H + u) * w;
        const float *__restrict__ hb = P.Hg[1] + ((size_t)k * H + u) * w;
#pragma unroll
        for (int q = 0; q < GEN_SEG / GEN_NT; ++q) {
            const int j = c0 + (int)threadIdx.x + GEN_NT * q;
            if (j < w) {
                za[q] = fmaf(wy, __ldcs(ha + j), za[q]);
                if (TWO) zb[q] = fmaf(wy, __ldcs(hb + j), zb[q]);
            }
        }
    }
}

// B: per LR sample of every frame, z = A_k x', zp = A_k p (F2 over F1's rows) and the residual
// e' = z - y; the data term's value psi_d(e') (e'^2 for L2), its change from x = x' - alpha p,
// psi_d(e') - psi_d(e' - alpha zp) (for L2 alpha zp (2 e' - alpha zp)), and the data part of p.H p,
// DS sum w zp^2 (w = 1 for L2, psi_d''(e') for L1; DS = 2 for L2, 1 for L1).  Kept per sample for
// C and D: DS psi_d'(e') (2 e' for L2), zp and w.  Tile g_ctas + blockIdx.x.
template <bool L1, int TWM>
__global__ void __launch_bounds__(GEN_NT) gen_pass_b(const DevProblem *__restrict__ probs, int pidx, int mode,
                                                     double probe_alpha, double probe_beta) {
    const DevProblem &P = probs[pidx];
    const GenStep s = gen_step(P, mode, probe_alpha, probe_beta);
    if (s.done) return;
    const float alpha = s.alpha, deps = P.data_eps, deps2 = deps * deps;
    const int h = P.h, w = P.w;
    constexpr int NQ = GEN_SEG / GEN_NT;
    const int segs = (w + GEN_SEG - 1) / GEN_SEG, items = P.K * h * segs;
    float jd = 0.f, dj = 0.f, cd = 0.f;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int r = it / segs, c0 = (it - r * segs) * GEN_SEG, k = r / h, i = r - k * h;
        float zx[NQ], zq[NQ];
        gen_f2_row<TWM, true>(P, k, i, c0, zx, zq);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int j = c0 + (int)threadIdx.x + GEN_NT * q;
            if (j >= w) continue;
            const size_t t = (size_t)r * w + j;
            const float e = zx[q] - P.Yg[t], zp = zq[q], abp = alpha * zp;
            const float de2 = abp * fmaf(2.f, e, -abp);   // e'^2 - (e' - alpha zp)^2
            if constexpr (L1) {
                // s = sqrt(e^2 + eps_d^2) as q rsqrt(q); psi_d(e') = e'^2 / (s1 + eps_d), psi_d' = e' / s1,
                // psi_d'' = eps_d^2 / s1^3, and the change (e'^2 - eb^2) / (s1 + s0)
                const float q1 = fmaf(e, e, deps2), r1 = rsqrtf(q1), s1 = q1 * r1;
                const float eb = e - abp, q0 = fmaf(eb, eb, deps2), s0 = q0 * rsqrtf(q0);
                jd += __fdividef(e * e, s1 + deps);
                dj += __fdividef(de2, s1 + s0);
                const float wd = deps2 * (r1 * r1 * r1);
                cd = fmaf(wd * zp, zp, cd);
                P.Eg[t] = e * r1;
                P.Wg[t] = wd;
            } else {
                jd = fmaf(e, e, jd);
                dj += de2;
                cd = fmaf(zp, zp, cd);
                P.Eg[t] = 2.f * e;
            }
            P.APg[t] = zp;
        }
    }
    const int fld[3] = {P_JD, P_DJD, P_C};
    const float val[3] = {jd, dj, (L1 ? 1.f : 2.f) * cd};
    gen_write_sums<3>(P, 1, (int)blockIdx.x, fld, val);
}

// C, in two stages (no shared memory).  C1, the adjoint's horizontal part for every LR row i of
// every frame and every HR column v: T[k][i][v] = sum_j Tx[k][j][v - f j - ox_k] DS psi_d'(e'_k)(i, j)
// over the j with 0 <= v - f j - ox_k < tw (ox_k = tx_k - R).  C2, the vertical part and r':
// r'(u, v) = -(sum_k sum_i Ty[k][i][u - f i - oy_k] T[k][i][v] + lambda grad BTV(x')(u, v)), the
// i with 0 <= u - f i - oy_k < tw; |r'|^2, r'.r, p.r' (tile 2 g_ctas + blockIdx.x).  Items of both:
// GEN_SEG columns of one row, thread t taking columns c0 + t + GEN_NT q, q < 4.
template <int TWM>
__global__ void __launch_bounds__(GEN_NT) gen_pass_c1(const DevProblem *__restrict__ probs, int pidx, int mode,
                                                      double probe_alpha, double probe_beta) {
    const DevProblem &P = probs[pidx];
    const GenStep s = gen_step(P, mode, probe_alpha, probe_beta);
    if (s.done) return;
    const int f = P.f, h = P.h, w = P.w, tw = P.g_tw, W = P.W;
    const unsigned fm = gen_fdiv_magic(f);
    const int segs = (W + GEN_SEG - 1) / GEN_SEG, items = P.K * h * segs;   // < 2^31 (plan check)
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int r = it / segs, c0 = (it - r * segs) * GEN_SEG, k = r / h;
        const int ox = P.tx[k] - P.g_r;
        const float *__restrict__ er = P.Eg + (size_t)r * w;
        const float *__restrict__ Txk = P.Tx + (size_t)k * w * tw;
        float *__restrict__ tr = P.Tg + (size_t)r * W;
#pragma unroll
        for (int q = 0; q < GEN_SEG / GEN_NT; ++q) {
            const int v = c0 + (int)threadIdx.x + GEN_NT * q;
            if (v >= W) continue;
            const int b = v - ox;
            const int jlo = max(gen_fdiv(b - tw + f, f, fm), 0), jhi = min(gen_fdiv(b, f, fm), w - 1);
            float sum = 0.f;
#pragma unroll
            for (int n = 0; n < TWM; ++n) {
                const int j = jlo + n;
                if (j <= jhi && MISR_IN_BOUNDS(j >= 0 && b - f * j >= 0 && b - f * j < tw, BC_GEN_TAP, v, j))
                    sum = fmaf(__ldg(Txk + j * tw + (b - f * j)), __ldg(er + j), sum);
            }
            tr[v] = sum;
        }
    }
}

template <int TWM>
__global__ void __launch_bounds__(GEN_NT) gen_pass_c2(const DevProblem *__restrict__ probs, int pidx, int mode,
                                                      double probe_alpha, double probe_beta) {
    const DevProblem &P = probs[pidx];
    const GenStep s = gen_step(P, mode, probe_alpha, probe_beta);
    if (s.done) return;
    const float *__restrict__ R = P.Rv[s.cur];
    const float *__restrict__ Pn = P.Pv[s.pcur ^ 1];
    float *__restrict__ Rn = P.Rv[s.cur ^ 1];
    const int f = P.f, h = P.h, tw = P.g_tw, H = P.H, W = P.W, K = P.K, pitch = P.pitch;
    const unsigned fm = gen_fdiv_magic(f);
    constexpr int NQ = GEN_SEG / GEN_NT;
    const int segs = (W + GEN_SEG - 1) / GEN_SEG, items = H * segs;
    float rr = 0.f, rrx = 0.f, pr = 0.f;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int u = it / segs, c0 = (it - u * segs) * GEN_SEG;
        float acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = 0.f;
        for (int k = 0; k < K; ++k) {   // the row's LR rows and weights of frame k, once for its columns
            const int a = u - (P.ty[k] - P.g_r);
            const int ilo = max(gen_fdiv(a - tw + f, f, fm), 0), ihi = min(gen_fdiv(a, f, fm), h - 1);
            const float *Tyk = P.Ty + (size_t)k * h * tw;
#pragma unroll
            for (int n = 0; n < TWM; ++n) {
                const int i = ilo + n;
                if (i > ihi) break;
                if (!MISR_IN_BOUNDS(i >= 0 && a - f * i >= 0 && a - f * i < tw, BC_GEN_TAP, u, i)) continue;
                const float wy = __ldg(Tyk + i * tw + (a - f * i));
                const float *__restrict__ tr = P.Tg + ((size_t)k * h + i) * W;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const int v = c0 + (int)threadIdx.x + GEN_NT * q;
                    if (v < W) acc[q] = fmaf(wy, __ldcs(tr + v), acc[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int v = c0 + (int)threadIdx.x + GEN_NT * q;
            if (v >= W) continue;
            const size_t o = (size_t)u * pitch + v;
            const float rn = -(acc[q] + Rn[o]);
            Rn[o] = rn;
            rr = fmaf(rn, rn, rr);
            rrx = fmaf(rn, R[o], rrx);
            pr = fmaf(Pn[o], rn, pr);
        }
    }
    const int fld[3] = {P_RR, P_RRX, P_PR};
    const float val[3] = {rr, rrx, pr};
    gen_write_sums<3>(P, 2, (int)blockIdx.x, fld, val);
}

// D, CTAs [0, g_ctas): per LR sample, zr = A_k r' (F2 over F1's rows of r'); the data parts of r'.H r' and r'.H p,
// DS sum w zr^2 and DS sum w zr zp.  CTAs [g_ctas, 2 g_ctas): per HR tile (x', r', p of the tile
// and its far-side halo in shared memory), the prior's parts of the three forms,
// lambda sum_d gamma_d sum_q psi''(x'_q - x'_{q+d}) (a_q - a_{q+d}) (b_q - b_{q+d}) for
// (a, b) = (r', r'), (r', p), (p, p), psi''(t) = eps^2 / (t^2 + eps^2)^(3/2).
// The grid is 2 half CTAs (half <= g_ctas); tiles 3 g_ctas + blockIdx.x and 4 g_ctas + blockIdx.x - half.
template <bool L1, int TWM>
__global__ void __launch_bounds__(GEN_NT) gen_pass_d(const DevProblem *__restrict__ probs, int pidx, int mode,
                                                     double probe_alpha, double probe_beta, int half) {
    __shared__ float xs[GEN_FH * GEN_FW], rs[GEN_FH * GEN_FW], qs[GEN_FH * GEN_FW];
    const DevProblem &P = probs[pidx];
    const GenStep s = gen_step(P, mode, probe_alpha, probe_beta);
    if (s.done) return;
    const float *__restrict__ Xn = P.X[s.cur ^ 1];
    const float *__restrict__ Rn = P.Rv[s.cur ^ 1];
    const float *__restrict__ Pn = P.Pv[s.pcur ^ 1];
    if ((int)blockIdx.x < half) {   // A_k r' by F2 over F1's rows of r'
        const int h = P.h, w = P.w;
        constexpr int NQ = GEN_SEG / GEN_NT;
        const int segs = (w + GEN_SEG - 1) / GEN_SEG, items = P.K * h * segs;
        float a = 0.f, b = 0.f;
        for (int it = blockIdx.x; it < items; it += half) {
            const int r = it / segs, c0 = (it - r * segs) * GEN_SEG, k = r / h, i = r - k * h;
            float zr[NQ], unused[NQ];
            gen_f2_row<TWM, false>(P, k, i, c0, zr, unused);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int j = c0 + (int)threadIdx.x + GEN_NT * q;
                if (j >= w) continue;
                const size_t t = (size_t)r * w + j;
                const float wzr = L1 ? P.Wg[t] * zr[q] : zr[q];
                a = fmaf(wzr, zr[q], a);
                b = fmaf(wzr, P.APg[t], b);
            }
        }
        const float ds = L1 ? 1.f : 2.f;
        const int fld[2] = {P_A, P_B};
        const float val[2] = {ds * a, ds * b};
        gen_write_sums<2>(P, 3, (int)blockIdx.x, fld, val);
        return;
    }
    const int H = P.H, W = P.W, pitch = P.pitch;
    const float eps2 = P.eps2;
    float gm[BTV_W * BTV_W];
#pragma unroll
    for (int d = 0; d < BTV_W * BTV_W; ++d) gm[d] = P.gamma[d];
    const int tiles_x = (W + GEN_TILE_W - 1) / GEN_TILE_W, n_t = tiles_x * ((H + GEN_TILE_H - 1) / GEN_TILE_H);
    float a = 0.f, b = 0.f, c = 0.f;
    for (int t = (int)blockIdx.x - half; t < n_t; t += half) {
        const int y0 = (t / tiles_x) * GEN_TILE_H, x0 = (t % tiles_x) * GEN_TILE_W;
        for (int e = threadIdx.x; e < GEN_FH * GEN_FW; e += GEN_NT) {
            const int ry = e / GEN_FW, rx = e - ry * GEN_FW, u = y0 + ry, v = x0 + rx;
            float xv = 0.f, rv = 0.f, pv = 0.f;
            if (u < H && v < W) {
                const size_t o = (size_t)u * pitch + v;
                xv = Xn[o]; rv = Rn[o]; pv = Pn[o];
            }
            xs[e] = xv; rs[e] = rv; qs[e] = pv;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < GEN_TILE_H * GEN_TILE_W / GEN_NT; ++q) {
            const int e = (int)threadIdx.x + GEN_NT * q, oy = e / GEN_TILE_W, ox = e - oy * GEN_TILE_W;
            const int u = y0 + oy, v = x0 + ox;
            if (u >= H || v >= W) continue;
            const int o = oy * GEN_FW + ox;
            const float xq = xs[o], rq = rs[o], pq = qs[o];
#pragma unroll
            for (int dy = 0; dy < BTV_W; ++dy)
#pragma unroll
                for (int dx = 0; dx < BTV_W; ++dx) {
                    const float gd = gm[dy * BTV_W + dx];
                    if ((dx | dy) == 0 || gd == 0.f || u + dy >= H || v + dx >= W) continue;
                    const int o2 = o + dy * GEN_FW + dx;
                    const float d = xq - xs[o2], q2 = fmaf(d, d, eps2), r3 = rsqrtf(q2);
                    const float w2 = gd * eps2 * (r3 * r3 * r3);
                    const float dr = rq - rs[o2], dp = pq - qs[o2], wdr = w2 * dr;
                    a = fmaf(wdr, dr, a);
                    b = fmaf(wdr, dp, b);
                    c = fmaf(w2 * dp, dp, c);
                }
        }
        __syncthreads();
    }
    const float lam = P.lambda;
    const int fld[3] = {P_A, P_B, P_C};
    const float val[3] = {lam * a, lam * b, lam * c};
    gen_write_sums<3>(P, 4, (int)blockIdx.x - half, fld, val);
}

}  // namespace misr
