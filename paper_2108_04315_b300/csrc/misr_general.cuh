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
// pairs, |r'|^2, r'.r, p.r', |p|^2, r'.H r', r'.H p, p.H p), in four kernels:
//   gen_pass_a  (HR)  p, x', the BTV value and lambda grad BTV(x') into r's buffer; |p|^2
//   gen_pass_b  (LR)  A_k x', A_k p: the residual, J_data, dJ_data, the data part of p.H p;
//                     DS psi_d'(e'), A_k p and psi_d''(e') kept per sample
//   gen_pass_c  (HR)  r' = -(A^T DS psi_d' + lambda grad BTV); |r'|^2, r'.r, p.r'
//   gen_pass_d  (LR)  A_k r': the data parts of r'.H r' and r'.H p;
//               (HR)  the BTV parts of the three curvature forms (second half of its CTAs)
// then reduce_kernel sums the tiles and runs the SCG tail.  Each CTA writes one tile of sums
// (every field, zero where the kernel has no part), so the tail sees the same fields.
// Per-thread sums are FP32 over the thread's grid-stride elements, the CTA sums FP64.
#pragma once

namespace misr {

constexpr int GEN_NT = 256;

// floor(a / f) for f > 0 and any sign of a
__device__ __forceinline__ int gen_floordiv(int a, int f) { return a >= 0 ? a / f : -((-a + f - 1) / f); }

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
// CTA calls it.
template <int NF>
__device__ __forceinline__ void gen_write_sums(const DevProblem &P, int tile, const int (&fld)[NF], const float (&v)[NF]) {
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
    if (threadIdx.x < NPART) {
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

// A: p = r + beta p_old, x' = x + alpha p (to the other halves of the double buffers); the BTV
// prior at x': each pixel q takes the pairs (q, q + d) and (q - d, q) of every offset d of the
// window (Eq. 8), its gradient gamma_d psi'(x'_q - x'_{q+d}) - gamma_d psi'(x'_{q-d} - x'_q),
// and the value of the pairs it starts, gamma_d sqrt(t^2 + eps^2).  A neighbour's x' is formed
// again from x, r and p_old with the same operations as its own thread's.  lambda grad BTV(x')
// goes to r's buffer, which gen_pass_c completes to r'.  Tile blockIdx.x: |p|^2, the BTV value.
__global__ void __launch_bounds__(GEN_NT) gen_pass_a(const DevProblem *__restrict__ probs, int pidx, int mode,
                                                     double probe_alpha, double probe_beta) {
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
    const float alpha = s.alpha, beta = s.beta, eps2 = P.eps2;
    auto xp = [&](int u, int v) {
        const size_t o = (size_t)u * pitch + v;
        return fmaf(alpha, fmaf(beta, Po[o], R[o]), X[o]);
    };
    float pp = 0.f, jb = 0.f;
    for (size_t t = (size_t)blockIdx.x * GEN_NT + threadIdx.x; t < (size_t)H * W; t += (size_t)gridDim.x * GEN_NT) {
        const int u = (int)(t / W), v = (int)(t - (size_t)u * W);
        const size_t o = (size_t)u * pitch + v;
        const float p = fmaf(beta, Po[o], R[o]);
        const float xq = fmaf(alpha, p, X[o]);
        pp = fmaf(p, p, pp);
        float g = 0.f, jq = 0.f;
        for (int dy = 0; dy < BTV_W; ++dy)
            for (int dx = 0; dx < BTV_W; ++dx) {
                const float gm = P.gamma[dy * BTV_W + dx];
                if ((dx | dy) == 0 || gm == 0.f) continue;
                if (u + dy < H && v + dx < W) {
                    const float d = xq - xp(u + dy, v + dx), q = fmaf(d, d, eps2);
                    g = fmaf(gm, d * rsqrtf(q), g);
                    jq = fmaf(gm, sqrtf(q), jq);
                }
                if (u >= dy && v >= dx) {
                    const float d = xp(u - dy, v - dx) - xq, q = fmaf(d, d, eps2);
                    g = fmaf(-gm, d * rsqrtf(q), g);
                }
            }
        jb += jq;
        Xn[o] = xq;
        Pn[o] = p;
        Rn[o] = P.lambda * g;
    }
    const int fld[2] = {P_PP, P_JB};
    const float val[2] = {pp, jb};
    gen_write_sums<2>(P, blockIdx.x, fld, val);
}

// B: per LR sample of every frame, z = A_k x', zp = A_k p and the residual e' = z - y; the data
// term's value psi_d(e') (e'^2 for L2), its change from x = x' - alpha p, psi_d(e') - psi_d(e'
// - alpha zp) (for L2 alpha zp (2 e' - alpha zp)), and the data part of p.H p, DS sum w zp^2
// (w = 1 for L2, psi_d''(e') for L1; DS = 2 for L2, 1 for L1).  Kept per sample for C and D:
// DS psi_d'(e') (2 e' for L2), zp and w.  Tile g_ctas + blockIdx.x.
template <bool L1>
__global__ void __launch_bounds__(GEN_NT) gen_pass_b(const DevProblem *__restrict__ probs, int pidx, int mode,
                                                     double probe_alpha, double probe_beta) {
    const DevProblem &P = probs[pidx];
    const GenStep s = gen_step(P, mode, probe_alpha, probe_beta);
    if (s.done) return;
    const float *__restrict__ Xn = P.X[s.cur ^ 1];
    const float *__restrict__ Pn = P.Pv[s.pcur ^ 1];
    const size_t m = (size_t)P.h * P.w;
    const float alpha = s.alpha, deps = P.data_eps, deps2 = deps * deps;
    float jd = 0.f, dj = 0.f, cd = 0.f;
    for (size_t t = (size_t)blockIdx.x * GEN_NT + threadIdx.x; t < m * P.K; t += (size_t)gridDim.x * GEN_NT) {
        const int k = (int)(t / m);
        const size_t li = t - (size_t)k * m;
        const int i = (int)(li / P.w), j = (int)(li - (size_t)i * P.w);
        const float2 z = gen_apply2(P, k, i, j, Xn, Pn, P.pitch);
        const float e = z.x - P.Yg[t], zp = z.y, abp = alpha * zp;
        const float de2 = abp * fmaf(2.f, e, -abp);   // e'^2 - (e' - alpha zp)^2
        if constexpr (L1) {
            const float s1 = sqrtf(fmaf(e, e, deps2)), eb = e - abp, s0 = sqrtf(fmaf(eb, eb, deps2));
            jd += e * e / (s1 + deps);                  // sqrt(e^2 + eps_d^2) - eps_d
            dj += de2 / (s1 + s0);
            const float w = deps2 / (s1 * s1 * s1);
            cd = fmaf(w * zp, zp, cd);
            P.Eg[t] = e / s1;
            P.Wg[t] = w;
        } else {
            jd = fmaf(e, e, jd);
            dj += de2;
            cd = fmaf(zp, zp, cd);
            P.Eg[t] = 2.f * e;
        }
        P.APg[t] = zp;
    }
    const int fld[3] = {P_JD, P_DJD, P_C};
    const float val[3] = {jd, dj, (L1 ? 1.f : 2.f) * cd};
    gen_write_sums<3>(P, P.g_ctas + blockIdx.x, fld, val);
}

// C: r'(u, v) = -(sum_k A_k^T (DS psi_d'(e'_k)) + lambda grad BTV(x')) by gathering, for each
// frame, the LR samples whose taps reach (u, v); |r'|^2, r'.r, p.r'.  Tile 2 g_ctas + blockIdx.x.
__global__ void __launch_bounds__(GEN_NT) gen_pass_c(const DevProblem *__restrict__ probs, int pidx, int mode,
                                                     double probe_alpha, double probe_beta) {
    const DevProblem &P = probs[pidx];
    const GenStep s = gen_step(P, mode, probe_alpha, probe_beta);
    if (s.done) return;
    const float *__restrict__ R = P.Rv[s.cur];
    const float *__restrict__ Pn = P.Pv[s.pcur ^ 1];
    float *__restrict__ Rn = P.Rv[s.cur ^ 1];
    const int H = P.H, W = P.W, f = P.f, h = P.h, w = P.w, tw = P.g_tw, gr = P.g_r;
    float rr = 0.f, rrx = 0.f, pr = 0.f;
    for (size_t t = (size_t)blockIdx.x * GEN_NT + threadIdx.x; t < (size_t)H * W; t += (size_t)gridDim.x * GEN_NT) {
        const int u = (int)(t / W), v = (int)(t - (size_t)u * W);
        const size_t o = (size_t)u * P.pitch + v;
        float acc = 0.f;
        for (int k = 0; k < P.K; ++k) {
            const int a = u - P.ty[k] + gr, b = v - P.tx[k] + gr;   // f i + dy, f j + dx
            const int ilo = max(gen_floordiv(a - tw + f, f), 0), ihi = min(gen_floordiv(a, f), h - 1);
            const int jlo = max(gen_floordiv(b - tw + f, f), 0), jhi = min(gen_floordiv(b, f), w - 1);
            for (int i = ilo; i <= ihi; ++i) {
                const float wy = P.Ty[((size_t)k * h + i) * tw + (a - f * i)];
                if (wy == 0.f) continue;
                const float *e = P.Eg + ((size_t)k * h + i) * w;
                float row = 0.f;
                for (int j = jlo; j <= jhi; ++j) row = fmaf(P.Tx[((size_t)k * w + j) * tw + (b - f * j)], e[j], row);
                acc = fmaf(wy, row, acc);
            }
        }
        const float rn = -(acc + Rn[o]);
        Rn[o] = rn;
        rr = fmaf(rn, rn, rr);
        rrx = fmaf(rn, R[o], rrx);
        pr = fmaf(Pn[o], rn, pr);
    }
    const int fld[3] = {P_RR, P_RRX, P_PR};
    const float val[3] = {rr, rrx, pr};
    gen_write_sums<3>(P, 2 * P.g_ctas + blockIdx.x, fld, val);
}

// D, CTAs [0, g_ctas): per LR sample, zr = A_k r'; the data parts of r'.H r' and r'.H p,
// DS sum w zr^2 and DS sum w zr zp.  CTAs [g_ctas, 2 g_ctas): the prior's parts of the three
// forms, lambda sum_d gamma_d sum_q psi''(x'_q - x'_{q+d}) (a_q - a_{q+d}) (b_q - b_{q+d}) for
// (a, b) = (r', r'), (r', p), (p, p), psi''(t) = eps^2 / (t^2 + eps^2)^(3/2).
// Tile 3 g_ctas + blockIdx.x.
template <bool L1>
__global__ void __launch_bounds__(GEN_NT) gen_pass_d(const DevProblem *__restrict__ probs, int pidx, int mode,
                                                     double probe_alpha, double probe_beta) {
    const DevProblem &P = probs[pidx];
    const GenStep s = gen_step(P, mode, probe_alpha, probe_beta);
    if (s.done) return;
    const float *__restrict__ Xn = P.X[s.cur ^ 1];
    const float *__restrict__ Rn = P.Rv[s.cur ^ 1];
    const float *__restrict__ Pn = P.Pv[s.pcur ^ 1];
    const int G = P.g_ctas;
    if ((int)blockIdx.x < G) {
        const size_t m = (size_t)P.h * P.w;
        float a = 0.f, b = 0.f;
        for (size_t t = (size_t)blockIdx.x * GEN_NT + threadIdx.x; t < m * P.K; t += (size_t)G * GEN_NT) {
            const int k = (int)(t / m);
            const size_t li = t - (size_t)k * m;
            const int i = (int)(li / P.w), j = (int)(li - (size_t)i * P.w);
            const float zr = gen_apply2(P, k, i, j, Rn, nullptr, P.pitch).x;
            const float wzr = L1 ? P.Wg[t] * zr : zr;
            a = fmaf(wzr, zr, a);
            b = fmaf(wzr, P.APg[t], b);
        }
        const float ds = L1 ? 1.f : 2.f;
        const int fld[2] = {P_A, P_B};
        const float val[2] = {ds * a, ds * b};
        gen_write_sums<2>(P, 3 * G + blockIdx.x, fld, val);
        return;
    }
    const int H = P.H, W = P.W, pitch = P.pitch;
    const float eps2 = P.eps2;
    float a = 0.f, b = 0.f, c = 0.f;
    for (size_t t = (size_t)(blockIdx.x - G) * GEN_NT + threadIdx.x; t < (size_t)H * W; t += (size_t)G * GEN_NT) {
        const int u = (int)(t / W), v = (int)(t - (size_t)u * W);
        const size_t o = (size_t)u * pitch + v;
        const float xq = Xn[o], rq = Rn[o], pq = Pn[o];
        for (int dy = 0; dy < BTV_W; ++dy)
            for (int dx = 0; dx < BTV_W; ++dx) {
                const float gm = P.gamma[dy * BTV_W + dx];
                if ((dx | dy) == 0 || gm == 0.f || u + dy >= H || v + dx >= W) continue;
                const size_t o2 = o + (size_t)dy * pitch + dx;
                const float d = xq - Xn[o2], q = fmaf(d, d, eps2), rs = rsqrtf(q);
                const float w2 = gm * eps2 * (rs * rs * rs);
                const float dr = rq - Rn[o2], dp = pq - Pn[o2], wdr = w2 * dr;
                a = fmaf(wdr, dr, a);
                b = fmaf(wdr, dp, b);
                c = fmaf(w2 * dp, dp, c);
            }
    }
    const float lam = P.lambda;
    const int fld[3] = {P_A, P_B, P_C};
    const float val[3] = {lam * a, lam * b, lam * c};
    gen_write_sums<3>(P, 3 * G + blockIdx.x, fld, val);
}

}  // namespace misr
