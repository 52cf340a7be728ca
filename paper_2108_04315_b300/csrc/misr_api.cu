// C ABI of the sm_103a MISR solver (declared in include/misr.h): plans, workspace, CUDA-graph
// replay of the SCG iteration, and the entry points.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "misr.h"
#include "misr_device.cuh"
#include "misr_internal.h"

using namespace misr;
using namespace misr_host;

namespace {
thread_local std::string g_err;
}  // namespace

misr_status misr_host::fail(misr_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

namespace {

// The compiled shapes of the fused pass (SHAPE_* in misr_types.cuh), dispatched at run time:
// the tile shapes (Geo), and the streaming shape (no shared-memory tile).
template <int S>
using ShapeGeo = Geo<SHAPE_TH[S < N_TILE_SHAPES ? S : 0], SHAPE_TW[S < N_TILE_SHAPES ? S : 0]>;
template <typename F>
auto with_shape(int s, F &&f) {
    static_assert(N_SHAPES == 4 && MISR_N_TILE_SHAPES == N_SHAPES && STREAM_SHAPE == 3, "one case per compiled shape");
    switch (s) {
    case 0: return f(std::integral_constant<int, 0>());
    case 1: return f(std::integral_constant<int, 1>());
    case 2: return f(std::integral_constant<int, 2>());
    default: return f(std::integral_constant<int, 3>());
    }
}
// the shape untuned geometries get (fastest on the B300 at 4096^2 and 768^2 HR)
constexpr int DEFAULT_SHAPE = 1;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

PFN_cuTensorMapEncodeTiled_v12000 g_encode_tiled = nullptr;

misr_status get_encode_tiled() {
    if (g_encode_tiled) return MISR_OK;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return fail(MISR_ECUDA, "cuTensorMapEncodeTiled unavailable: %s", cudaGetErrorString(e));
    g_encode_tiled = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return MISR_OK;
}

// 2-D float32 tensor map over an H x W image with the given row pitch (floats); box of
// box_w x box_h elements; out-of-bounds elements read as 0 or as NaN.
misr_status make_map(CUtensorMap *m, void *base, int W, int H, int pitch, int box_w, int box_h, bool nan_fill,
                     bool bf16 = false) {
    const size_t esz = bf16 ? 2 : sizeof(float);
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * esz};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode_tiled(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base,
                                dims, strides, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                nan_fill ? CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA
                                         : CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MISR_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return MISR_OK;
}

}  // namespace


static misr_status validate(const misr_desc *d) {
    if (!d) return fail(MISR_EINVAL, "desc is NULL");
    if (d->lr_h < 1 || d->lr_w < 1) return fail(MISR_EINVAL, "lr_h, lr_w must be >= 1");
    if (d->factor < 1 || d->factor > MAXF) return fail(MISR_EINVAL, "factor must be in [1, %d]", MAXF);
    if (d->K < 1 || d->K > MAXK) return fail(MISR_EINVAL, "K must be in [1, %d]", MAXK);
    if ((int64_t)d->factor * d->lr_h > (1 << 20) || (int64_t)d->factor * d->lr_w > (1 << 20))
        return fail(MISR_EINVAL, "HR image side above 2^20");
    if (!d->shifts) return fail(MISR_EINVAL, "shifts is NULL");
    if (!d->psf) return fail(MISR_EINVAL, "psf is NULL");
    if (d->psf_size < 1 || d->psf_size > 2 * PSF_R + 1 || d->psf_size % 2 == 0)
        return fail(MISR_EINVAL, "psf_size must be odd and <= %d", 2 * PSF_R + 1);
    if (!(d->lambda >= 0)) return fail(MISR_EINVAL, "lambda must be >= 0");
    if (!(d->eps >= 1e-15 && d->eps <= 1e15)) return fail(MISR_EINVAL, "eps must be in [1e-15, 1e15]");
    if (d->btv_w < 1 || d->btv_w > BTV_W) return fail(MISR_EINVAL, "btv_w must be in [1, %d]", BTV_W);
    if (!(d->btv_alpha >= 0)) return fail(MISR_EINVAL, "btv_alpha must be >= 0");
    if (d->iters < 0 || d->iters > 1000000) return fail(MISR_EINVAL, "iters must be in [0, 1e6]");
    if (d->x0_mode < 0 || d->x0_mode > 2) return fail(MISR_EINVAL, "bad x0_mode");
    if (d->in_dtype != MISR_F32 && d->in_dtype != MISR_U16) return fail(MISR_EINVAL, "in_dtype must be MISR_F32 or MISR_U16");
    if (d->in_dtype == MISR_U16 && !(d->flat_field > 0)) return fail(MISR_EINVAL, "flat_field must be > 0");
    if (d->iterate_dtype != MISR_F32 && d->iterate_dtype != MISR_BF16)
        return fail(MISR_EINVAL, "iterate_dtype must be MISR_F32 or MISR_BF16");
    if (d->tile_shape < MISR_TILE_AUTO || d->tile_shape > MISR_N_TILE_SHAPES)
        return fail(MISR_EINVAL, "tile_shape must be MISR_TILE_AUTO or a MISR_TILE_* shape");
    if (d->data_norm != MISR_NORM_L2 && d->data_norm != MISR_NORM_L1)
        return fail(MISR_EINVAL, "data_norm must be MISR_NORM_L2 or MISR_NORM_L1");
    if (d->data_norm == MISR_NORM_L1 && !(d->data_eps >= 1e-15 && d->data_eps <= 1e15))
        return fail(MISR_EINVAL, "data_eps must be in [1e-15, 1e15] for MISR_NORM_L1");
    if (d->decimation != MISR_DECIM_POINT && d->decimation != MISR_DECIM_BIN)
        return fail(MISR_EINVAL, "decimation must be MISR_DECIM_POINT or MISR_DECIM_BIN");
    return MISR_OK;
}

// The PSF normalised to sum 1 as its row sums rs and column sums cs.  h = u v^T with sum h = 1
// implies h = rs cs^T, so the PSF is accepted when it equals the outer product of its row and
// column sums.
static misr_status psf_factors(const misr_desc &d, std::vector<double> &rs, std::vector<double> &cs) {
    const int S = d.psf_size;
    double sum = 0;
    for (int i = 0; i < S * S; ++i) sum += d.psf[i];
    if (!(sum > 0)) return fail(MISR_EINVAL, "PSF must have a positive sum");
    std::vector<double> h(S * S);
    rs.assign(S, 0.0);
    cs.assign(S, 0.0);
    double hmax = 0;
    for (int i = 0; i < S * S; ++i) { h[i] = d.psf[i] / sum; hmax = std::max(hmax, std::fabs(h[i])); }
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b) { rs[a] += h[a * S + b]; cs[b] += h[a * S + b]; }
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b)
            if (std::fabs(h[a * S + b] - rs[a] * cs[b]) > 1e-6 * hmax)
                return fail(MISR_EINVAL, "PSF is not separable");
    return MISR_OK;
}

// Separable taps of the fused passes.  With binning, D B is one blur: per axis, (D_bin B z)(i) =
// (1/f) sum_{a'<f} (B z)(f i + a') = sum_c h'(c) z(f i - c) with h'(c) = (1/f) sum_{a'=0}^{f-1}
// h(c + a'), c in [-R-f+1, R]; the tap masks of the frames (B's zero padding in front of M_k:
// the input pixel f i - c >= 0) are those of the point-sampled blur with h' in place of h.
// hy, hx receive the taps at [c + R] (c in [-PSF_R, PSF_R], 0 outside the blur); *lowest the
// lowest tap c with a weight.  The caller has checked that the taps fit (R + f - 1 <= PSF_R
// with binning).
static void psf_taps(const misr_desc *d, const std::vector<double> &rs, const std::vector<double> &cs, double *hy,
                     double *hx, int *lowest) {
    const int S = d->psf_size, R = S / 2;
    for (int i = 0; i < 2 * PSF_R + 1; ++i) { hy[i] = 0.0; hx[i] = 0.0; }
    *lowest = -R;
    if (d->decimation == MISR_DECIM_BIN && d->factor > 1) {
        const int f = d->factor;
        for (int c = -R - f + 1; c <= R; ++c) {
            double sy = 0, sx = 0;
            for (int a2 = 0; a2 < f; ++a2)
                if (c + a2 >= -R && c + a2 <= R) { sy += rs[c + a2 + R]; sx += cs[c + a2 + R]; }
            hy[c + PSF_R] = sy / f;
            hx[c + PSF_R] = sx / f;
        }
        *lowest = -R - f + 1;
        return;
    }
    for (int a = -R; a <= R; ++a) { hy[a + PSF_R] = rs[a + R]; hx[a + PSF_R] = cs[a + R]; }
}

// The frames' geometry and the blur taps of a descriptor into the problem record.
// An HR shift t = f s (t within 1e-4 of an integer is that integer) is split per axis into
// t = n + a, n = floor(t), 0 <= a < 1.  A non-integer t is bilinear interpolation,
// (M x)(u) = (1 - a) x(u + n) + a x(u + n + 1).
//
// Interleaved frames (the fused passes): every n in [0, f - 1], one frame per phase (n_y, n_x),
// so the frame's samples sit at HR pixels f (i, j) + (n_y, n_x).  Per axis a frame's blur is
// then h_k(c) = (1 - a) h(c) + a h(c + 1), c in [lowest - 1, R], over x at s - c for a sample
// at s; at the top / left border the second part of the tap c = f i (s - c = n) reads B's
// input pixel -1, which B's zero padding drops: that tap weighs (1 - a) h(c) alone.  The taps
// of a frame must depend on one axis's phase only (a product lattice of shifts, as x and y
// stages give): a_y per row phase, a_x per column phase.  phased = 1 when some a is not 0.
// The combined taps must fit the compiled 2 PSF_R + 1.
//
// Any other frame set runs the frame-wise pass (general = 1): ty, tx hold n (any sign), gfy,
// gfx the fractional parts, and the tap tables are built by gen_tables.
// HR shift of frame k (within 1e-4 of an integer: that integer)
static void hr_shift(const misr_desc &d, int k, double *ty, double *tx) {
    *tx = (double)d.factor * d.shifts[2 * k];
    *ty = (double)d.factor * d.shifts[2 * k + 1];
    if (std::fabs(*tx - std::floor(*tx + 0.5)) <= 1e-4) *tx = std::floor(*tx + 0.5);
    if (std::fabs(*ty - std::floor(*ty + 0.5)) <= 1e-4) *ty = std::floor(*ty + 0.5);
}
static misr_status setup_geometry(const misr_desc &d, DevProblem &hp) {
    const int f = d.factor;
    for (int i = 0; i < MAXF * MAXF; ++i) hp.frame_of_phase[i] = -1;
    std::vector<double> rs, cs;
    misr_status s = psf_factors(d, rs, cs);
    if (s != MISR_OK) return s;
    double ay[MAXF], ax[MAXF];
    bool sy[MAXF] = {}, sx[MAXF] = {};
    for (int i = 0; i < MAXF; ++i) ay[i] = ax[i] = 0.0;
    bool frac_y = false, frac_x = false, interleaved = true, any_frac = false;
    double tys[MAXK], txs[MAXK];
    for (int k = 0; k < d.K; ++k) {
        double tx, ty;
        hr_shift(d, k, &ty, &tx);
        if (!std::isfinite(tx) || !std::isfinite(ty)) return fail(MISR_EINVAL, "frame %d: shift is not finite", k);
        if (std::fabs(tx) > (double)(1 << 20) || std::fabs(ty) > (double)(1 << 20))
            return fail(MISR_EINVAL, "frame %d: shift beyond 2^20 HR px", k);
        tys[k] = ty;
        txs[k] = tx;
        any_frac |= tx != std::floor(tx) || ty != std::floor(ty);
        if (!interleaved) continue;
        if (tx < 0 || tx >= f || ty < 0 || ty >= f) { interleaved = false; continue; }
        const int nx = (int)std::floor(tx), ny = (int)std::floor(ty);
        const double fx = tx - nx, fy = ty - ny;
        const int ph = ny * f + nx;
        if (hp.frame_of_phase[ph] >= 0 || (sy[ny] && std::fabs(ay[ny] - fy) > 1e-6) ||
            (sx[nx] && std::fabs(ax[nx] - fx) > 1e-6)) {
            interleaved = false;
            continue;
        }
        sy[ny] = sx[nx] = true;
        ay[ny] = fy; ax[nx] = fx;
        frac_y |= fy != 0.0;
        frac_x |= fx != 0.0;
        hp.frame_of_phase[ph] = k;
        hp.ty[k] = ny; hp.tx[k] = nx;
    }
    // the combined taps of the fused passes: binning widens the blur by f - 1, a non-integer
    // shift by 1
    const int R = d.psf_size / 2;
    const int lowest = d.decimation == MISR_DECIM_BIN && f > 1 ? -R - f + 1 : -R;
    if (interleaved && lowest - ((frac_y || frac_x) ? 1 : 0) < -PSF_R) interleaved = false;
    if (!interleaved) {
        if (d.iterate_dtype == MISR_BF16)
            return fail(MISR_ENOTIMPL, "frames that do not interleave into one HR image (several frames per phase, "
                                       "shifts outside [0, 1) LR px or off a product lattice, or a combined blur "
                                       "wider than %d taps) run the frame-wise pass, which keeps r and p in float",
                        2 * PSF_R + 1);
        hp.general = 1;
        hp.phased = 0;
        for (int i = 0; i < MAXF * MAXF; ++i) hp.frame_of_phase[i] = -1;
        for (int k = 0; k < d.K; ++k) {
            const double fy = std::floor(tys[k]), fx = std::floor(txs[k]);
            hp.ty[k] = (int)fy;
            hp.tx[k] = (int)fx;
            hp.gfy[k] = (float)(tys[k] - fy);
            hp.gfx[k] = (float)(txs[k] - fx);
            hp.gfy0[k] = (float)(1.0 - (tys[k] - fy));
            hp.gfx0[k] = (float)(1.0 - (txs[k] - fx));
        }
        const int nb = d.decimation == MISR_DECIM_BIN ? f : 1;
        hp.g_r = R;
        hp.g_nb = nb;
        hp.g_tw = nb + 2 * R + (any_frac ? 1 : 0);
        // the PSF's factors (the fused passes' tap slots; here they identify the model)
        for (int i = 0; i < 2 * PSF_R + 1; ++i) hp.hy[i] = hp.hx[i] = 0.f;
        for (int a = -R; a <= R; ++a) { hp.hy[a + PSF_R] = (float)rs[a + R]; hp.hx[a + PSF_R] = (float)cs[a + R]; }
        return MISR_OK;
    }
    hp.general = 0;
    double hy[2 * PSF_R + 1], hx[2 * PSF_R + 1];
    int low = 0;
    psf_taps(&d, rs, cs, hy, hx, &low);
    for (int i = 0; i < 2 * PSF_R + 1; ++i) { hp.hy[i] = (float)hy[i]; hp.hx[i] = (float)hx[i]; }
    hp.phased = frac_y || frac_x;
    if (!hp.phased) return MISR_OK;
    if (d.tile_shape != MISR_TILE_AUTO && d.tile_shape - 1 != PHASED_SHAPE)
        return fail(MISR_ENOTIMPL, "non-integer shifts on a product lattice run on the 32x32 tile shape only");
    for (int p = 0; p < f; ++p) {
        hp.ay[p] = (float)ay[p];
        hp.ax[p] = (float)ax[p];
        for (int c = -PSF_R; c <= PSF_R; ++c) {
            const double nyt = c + 1 <= PSF_R ? hy[c + 1 + PSF_R] : 0.0, nxt = c + 1 <= PSF_R ? hx[c + 1 + PSF_R] : 0.0;
            hp.tph[TPH_FY][p][c + PSF_R] = (float)((1.0 - ay[p]) * hy[c + PSF_R] + ay[p] * nyt);
            hp.tph[TPH_PY][p][c + PSF_R] = (float)((1.0 - ay[p]) * hy[c + PSF_R]);
            hp.tph[TPH_FX][p][c + PSF_R] = (float)((1.0 - ax[p]) * hx[c + PSF_R] + ax[p] * nxt);
            hp.tph[TPH_PX][p][c + PSF_R] = (float)((1.0 - ax[p]) * hx[c + PSF_R]);
        }
    }
    for (int p = 0; p < f; ++p)
        for (int c = -PSF_R; c <= PSF_R; ++c) {
            const int q = ((p + c) % f + f) % f;
            hp.tph[TPH_AFY][p][c + PSF_R] = hp.tph[TPH_FY][q][c + PSF_R];
            hp.tph[TPH_AFX][p][c + PSF_R] = hp.tph[TPH_FX][q][c + PSF_R];
        }
    return MISR_OK;
}

// Tap tables of the frame-wise pass, per axis (Eq. 1 with the readings of B, D and M_k): for
// LR index i of frame k, T[k][i][a' - a + q + R] accumulates h(a) w_q / nb over the block
// offsets a' < nb (nb = f with binning, else 1), the PSF taps a in [-R, R] whose input pixel
// s = f i + a' - a lies inside the grid, and the bilinear parts q in {0, 1} with weights
// (1 - frac, frac) whose x pixel s + n + q lies inside the grid (n = floor of the HR shift).
// Computed in FP64 and rounded once.
static void gen_axis_table(int n_lr, int f, int HR, int nb, int R, const std::vector<double> &h1, int n, double frac,
                           int tw, float *T) {
    std::vector<double> acc(tw);
    for (int i = 0; i < n_lr; ++i) {
        std::fill(acc.begin(), acc.end(), 0.0);
        for (int a2 = 0; a2 < nb; ++a2)
            for (int a = -R; a <= R; ++a) {
                const long s = (long)f * i + a2 - a;
                if (s < 0 || s >= HR) continue;
                for (int q = 0; q < 2; ++q) {
                    const double wq = q ? frac : 1.0 - frac;
                    const long u = s + n + q;
                    if (wq == 0.0 || u < 0 || u >= HR) continue;
                    acc[a2 - a + q + R] += h1[a + R] * wq / nb;
                }
            }
        for (int t = 0; t < tw; ++t) T[(size_t)i * tw + t] = (float)acc[t];
    }
}
static misr_status gen_tables(const misr_desc &d, const DevProblem &hp, std::vector<float> &Ty, std::vector<float> &Tx) {
    std::vector<double> rs, cs;
    misr_status s = psf_factors(d, rs, cs);
    if (s != MISR_OK) return s;
    const int f = d.factor, nb = d.decimation == MISR_DECIM_BIN ? f : 1, tw = hp.g_tw, R = hp.g_r;
    Ty.assign((size_t)d.K * hp.h * tw, 0.f);
    Tx.assign((size_t)d.K * hp.w * tw, 0.f);
    for (int k = 0; k < d.K; ++k) {
        double ty, tx;
        hr_shift(d, k, &ty, &tx);
        gen_axis_table(hp.h, f, hp.H, nb, R, rs, hp.ty[k], ty - std::floor(ty), tw, Ty.data() + (size_t)k * hp.h * tw);
        gen_axis_table(hp.w, f, hp.W, nb, R, cs, hp.tx[k], tx - std::floor(tx), tw, Tx.data() + (size_t)k * hp.w * tw);
    }
    return MISR_OK;
}

// Launch with programmatic stream serialization: the kernel may begin launching while the
// previous kernel on the stream finishes; it waits for it (griddepcontrol.wait) before reading
// what that kernel produced.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                              Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// the pass kernel of shape S and variant V (bit 0 bf16 r and p, bit 1 the L1 data term, bit 2
// per-phase taps), and its dynamic shared memory; the per-phase variants exist for the
// PHASED_SHAPE only
template <int S, int V>
constexpr bool compiled_variant() { return S == STREAM_SHAPE ? V < 4 : (V & 4) == 0 || S == PHASED_SHAPE; }
// whether a problem of variant v can run on shape sh
static bool shape_takes_variant(int sh, int v) { return sh == STREAM_SHAPE ? v < 4 : (v & 4) == 0 || sh == PHASED_SHAPE; }
template <int S, int V>
constexpr auto pass_kernel() {
    static_assert(compiled_variant<S, V>(), "variant not compiled for this shape");
    if constexpr (S == STREAM_SHAPE)
        return scg_stream_kernel<(V & 1) != 0, (V & 2) != 0>;
    else
        return scg_pass_kernel<SHAPE_TH[S], SHAPE_TW[S], SHAPE_NT[S], (V & 1) != 0, (V & 2) != 0, (V & 4) != 0>;
}
template <int S, int V>
constexpr size_t pass_smem() {
    if constexpr (S == STREAM_SHAPE) return SW_SMEM_BYTES;
    else return ShapeGeo<S>::smem_bytes((V & 2) != 0);
}
template <typename F>
auto with_variant(int v, F &&f) {
    static_assert(N_VARIANTS == 8, "one case per compiled variant");
    switch (v) {
    case 0: return f(std::integral_constant<int, 0>());
    case 1: return f(std::integral_constant<int, 1>());
    case 2: return f(std::integral_constant<int, 2>());
    case 3: return f(std::integral_constant<int, 3>());
    case 4: return f(std::integral_constant<int, 4>());
    case 5: return f(std::integral_constant<int, 5>());
    case 6: return f(std::integral_constant<int, 6>());
    default: return f(std::integral_constant<int, 7>());
    }
}

template <int S, int V>
static misr_status set_attrs_one() {
    if constexpr (!compiled_variant<S, V>()) {
        return MISR_OK;
    } else {
        auto *k = pass_kernel<S, V>();
        if constexpr (S == STREAM_SHAPE) {
            CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem<S, V>()));
            CK(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        } else {
            CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem<S, V>()));
            CK(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        }
        return MISR_OK;
    }
}

// Per-device state of the pass kernels: whether their attributes (dynamic shared memory above
// 48 KB, carveout) are set on that device, and their resident CTAs on the whole GPU per shape
// and variant (0: not measured yet).  Function attributes are per device, so every device a
// plan, batch, server or allocation-free call runs on sets them once, with it current.
constexpr int MAX_DEVICES = 64;
struct PassDeviceState {
    bool attrs = false;
    int resident[N_SHAPES][N_VARIANTS] = {};
};
std::mutex g_pass_dev_mu;
PassDeviceState g_pass_dev[MAX_DEVICES];

static misr_status current_device(int *dev) {
    CK(cudaGetDevice(dev));
    if (*dev < 0 || *dev >= MAX_DEVICES) return fail(MISR_EINVAL, "device %d out of range", *dev);
    return MISR_OK;
}

// Grid of a frame-wise kernel: at most `want` CTAs, at most as many as are resident at once on
// the current device (one wave); cached per device and kernel.
template <typename... A>
static int gen_grid(void (*kernel)(A...), int want) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(dev, reinterpret_cast<const void *>(kernel));
    auto it = cache.find(key);
    if (it == cache.end()) {
        int per_sm = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, GEN_NT, 0);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaGetLastError();
        it = cache.emplace(key, std::max(1, per_sm) * std::max(1, sms)).first;
    }
    return std::max(1, std::min(want, it->second));
}

// the frame-wise pass's kernels are compiled for at most 4, 8 or GEN_TW taps per axis
template <typename F>
auto with_gen_taps(int tw, F &&f) {
    if (tw <= 4) return f(std::integral_constant<int, 4>());
    if (tw <= 8) return f(std::integral_constant<int, 8>());
    return f(std::integral_constant<int, GEN_TW>());
}
// the occupancy of a frame-wise plan's kernels, queried once before any stream capture
static void gen_prime_grids(int tw) {
    gen_grid(gen_pass_a, 1);
    with_gen_taps(tw, [](auto T) {
        constexpr int t = decltype(T)::value;
        gen_grid(gen_pass_f1<t, true>, 1); gen_grid(gen_pass_f1<t, false>, 1);
        gen_grid(gen_pass_b<true, t>, 1); gen_grid(gen_pass_b<false, t>, 1);
        gen_grid(gen_pass_c1<t>, 1); gen_grid(gen_pass_c2<t>, 1);
        return 0;
    });
}

static misr_status set_pass_attrs() {
    int dev = 0;
    misr_status r = current_device(&dev);
    if (r != MISR_OK) return r;
    std::lock_guard<std::mutex> lock(g_pass_dev_mu);
    if (g_pass_dev[dev].attrs) return MISR_OK;
    for (int sh = 0; sh < N_SHAPES; ++sh)
        for (int v = 0; v < N_VARIANTS; ++v) {
            r = with_shape(sh, [v](auto S) {
                return with_variant(v, [](auto V) { return set_attrs_one<decltype(S)::value, decltype(V)::value>(); });
            });
            if (r != MISR_OK) return r;
        }
    g_pass_dev[dev].attrs = true;
    return MISR_OK;
}

// CTAs of the fused pass resident on the whole current GPU, per shape and variant (the L1 and
// per-phase variants take more shared memory)
static int resident_ctas(int shape, int variant) {
    int dev = 0;
    if (current_device(&dev) != MISR_OK) return 1;
    std::lock_guard<std::mutex> lock(g_pass_dev_mu);
    int &cached = g_pass_dev[dev].resident[shape][variant];
    if (cached > 0) return cached;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    with_shape(shape, [&](auto S) {
        return with_variant(variant, [&](auto V) {
            constexpr int s = decltype(S)::value, v = decltype(V)::value;
            if constexpr (compiled_variant<s, v>())
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pass_kernel<s, v>(), SHAPE_NT[s], pass_smem<s, v>());
            return 0;
        });
    });
    cudaGetLastError();
    cached = std::max(sms, 1) * std::max(per_sm, 1);
    return cached;
}

// persistent grid: one CTA per resident slot, at most one per tile
static int pass_grid(int shape, int variant, int n_tiles) {
    return std::max(1, std::min(n_tiles, resident_ctas(shape, variant)));
}

static misr_status launch_pass(misr_plan_t p, int mode, double alpha, double beta, cudaStream_t s) {
    return launch_pass_raw(p->dprob, p->dtile, p->segs, p->dgroup, p->hp.n_groups, p->work, mode, alpha, beta, s);
}

// The tile list of problem `pi` for a tile shape (border tiles first: they cost more, so a pass
// ends on interior tiles; the streaming shape's items are listed by build_pass_lists).  An entry is (problem, ty << 16 | tx); an HR side of at most 2^20 pixels
// keeps both tile coordinates below 2^16.
static void append_tiles(const DevProblem &hp, int pi, std::vector<int2> &tiles) {
    const int tx = hp.tiles_x, TH = hp.tile_h, TW = hp.tile_w;
    for (int pass = 0; pass < 2; ++pass)
        for (int t = 0; t < hp.n_tiles; ++t) {
            const int ty = t / tx, tc = t % tx, y0 = ty * TH, x0 = tc * TW;
            const bool border = y0 - 6 < 0 || x0 - 8 < 0 || y0 + TH + 6 > hp.H || x0 + TW + 8 > hp.W;
            if (border == (pass == 0)) tiles.push_back(make_int2(pi, (int)(((unsigned)ty << 16) | (unsigned)tc)));
        }
}

StreamConsts misr_host::stream_consts(const DevProblem &p) {
    StreamConsts k{};
    for (int i = 0; i < 2 * PSF_R + 1; ++i) { k.hx[i] = p.hx[i]; k.hy[i] = p.hy[i]; }
    for (int i = 0; i < BTV_W * BTV_W; ++i) {
        k.gam[i] = p.gamma[i];
        k.lgam[i] = p.lambda * p.gamma[i];
    }
    k.eps2 = p.eps2;
    k.lambda = p.lambda;
    k.deps = p.l1 ? p.data_eps : 0.f;
    k.deps2 = k.deps * k.deps;
    k.f = p.f;
    k.fmag = p.f > 1 ? (unsigned)((0x100000000ull + p.f - 1) / p.f) : 0u;
    return k;
}

bool misr_host::launch_alone(const DevProblem &p) {
    if (p.general) return true;
    if (p.shape != STREAM_SHAPE) return false;
    return 2L * p.n_tiles >= 8L * resident_ctas(STREAM_SHAPE, pass_variant(p));
}

void misr_host::build_pass_lists(const std::vector<const DevProblem *> &recs, const std::vector<int> &idx,
                                 std::vector<int2> &tiles, std::vector<int2> &groups, PassSegs &segs) {
    segs = PassSegs{};
    for (int sh = 0; sh < N_SHAPES; ++sh)
        for (int v = 0; v < N_VARIANTS; ++v) {
            if (sh == STREAM_SHAPE) {
                // runs of consecutive problems that share the launch constants
                std::vector<size_t> run;
                auto flush = [&]() {
                    if (run.empty()) return;
                    StreamRun r;
                    r.variant = v;
                    r.k = stream_consts(*recs[run[0]]);
                    // the run's edge items, then the rest
                    for (int part = 0; part < 2; ++part)
                        for (size_t i : run) {
                            const DevProblem &q = *recs[i];
                            const int ne = q.n_left + q.n_top;
                            for (int t = part ? ne : 0; t < (part ? q.n_tiles : ne); ++t)
                                tiles.push_back(make_int2(idx[i], t));
                            if (part) continue;
                            r.count += q.n_tiles;
                            r.n_edge += ne;
                            r.edge_work += (STREAM_LEFT_COST * q.n_left + STREAM_TOP_COST * q.n_top) *
                                           (std::min(q.edge_h, q.H) + 12);
                            r.int_work += (double)(q.n_tiles - ne) * (q.tile_h + 12);
                            r.edge_ctas_w += (double)q.edge_ctas * ((double)(q.n_tiles - ne) * (q.tile_h + 12) +
                                                                     (STREAM_LEFT_COST * q.n_left + STREAM_TOP_COST * q.n_top) *
                                                                         (std::min(q.edge_h, q.H) + 12));
                        }
                    r.edge_ctas = run.size() == 1 ? recs[run[0]]->edge_ctas : 0;
                    segs.n[sh][v] += r.count;
                    segs.runs.push_back(r);
                    run.clear();
                };
                // a problem whose items fill at least half the grid's warps gets a launch of its
                // own, split as planned (merged, such problems ran slower than one after another:
                // the launch's last items straggled); smaller ones share launches
                for (size_t i = 0; i < recs.size(); ++i) {
                    if (recs[i]->general || recs[i]->shape != sh || pass_variant(*recs[i]) != v) continue;
                    const bool alone = launch_alone(*recs[i]);
                    if (!run.empty()) {
                        const StreamConsts a = stream_consts(*recs[run[0]]), b = stream_consts(*recs[i]);
                        if (alone || std::memcmp(&a, &b, sizeof(a)) != 0) flush();
                    }
                    run.push_back(i);
                    if (alone) flush();
                }
                flush();
                continue;
            }
            for (size_t i = 0; i < recs.size(); ++i)
                if (!recs[i]->general && recs[i]->shape == sh && pass_variant(*recs[i]) == v) {
                    append_tiles(*recs[i], idx[i], tiles);
                    segs.n[sh][v] += recs[i]->n_tiles;
                }
        }
    // The reduction.  A step of one streaming launch and nothing else reduces in that launch
    // (no reduction launch, and the launch's last warps run the tail); a step of several
    // launches keeps the reduction kernel, which sums every problem's groups in parallel after
    // the last launch (reduced in each launch, the tails would run one after another).
    bool others = false;
    for (size_t i = 0; i < recs.size(); ++i) {
        others |= recs[i]->general || recs[i]->shape != STREAM_SHAPE;
        if (recs[i]->general) {
            GenRun g;
            g.pidx = idx[i];
            g.ctas = recs[i]->g_ctas;
            g.tw = recs[i]->g_tw;

            g.l1 = recs[i]->l1 != 0;
            segs.gen.push_back(g);
        }
    }
    const bool in_pass = !others && segs.runs.size() == 1;
    if (in_pass) segs.runs[0].reduce_in_pass = true;
    for (size_t i = 0; i < recs.size(); ++i) {
        if (in_pass && !recs[i]->general && recs[i]->shape == STREAM_SHAPE) continue;
        for (int g = 0; g < recs[i]->n_groups; ++g) groups.push_back(make_int2(idx[i], g));
        segs.n_reduce += recs[i]->n_groups;
    }
}

// The process's tuning: HR image size -> the time per pass misr_autotune measured for each shape
// (0: not timed, e.g. a shape the tuned descriptor's variant cannot run on).
std::mutex g_tuned_mu;
std::vector<std::pair<std::pair<int, int>, std::array<double, N_SHAPES>>> g_tuned;

// The shape of a plan: the descriptor's, else the tuned one for its HR size, else the default.
static int desc_variant(const misr_desc &d, bool phased) {
    return (d.iterate_dtype == MISR_BF16 ? 1 : 0) | (d.data_norm == MISR_NORM_L1 ? 2 : 0) | (phased ? 4 : 0);
}
// Untuned default: the streaming shape from STREAM_DEFAULT_PIXELS HR pixels up (where it can
// run the plan's variant), else 32 x 32 tiles.  Measured per pass, stream over the best tile
// shape: 1.10 at 2048^2, 0.91 at 2560^2, 0.90 at 3072^2, 0.86 at 3072 x 3840, 0.84 at 6144^2.
constexpr long STREAM_DEFAULT_PIXELS = 5000000;
static int pick_shape(const misr_desc &d, int variant) {
    if (d.tile_shape >= 1 && d.tile_shape <= N_SHAPES) return d.tile_shape - 1;
    const int H = d.factor * d.lr_h, W = d.factor * d.lr_w;
    std::lock_guard<std::mutex> lock(g_tuned_mu);
    for (auto &e : g_tuned)
        if (e.first.first == H && e.first.second == W) {
            int best = -1;
            for (int sh = 0; sh < N_SHAPES; ++sh)
                if (e.second[sh] > 0 && shape_takes_variant(sh, variant) && (best < 0 || e.second[sh] < e.second[best]))
                    best = sh;
            if (best >= 0) return best;
        }
    if ((long)H * W >= STREAM_DEFAULT_PIXELS && shape_takes_variant(STREAM_SHAPE, variant)) return STREAM_SHAPE;
    return DEFAULT_SHAPE;
}

// The data term of a descriptor (checked by check_desc).
static void set_data_norm(DevProblem &hp, const misr_desc &d) {
    hp.l1 = d.data_norm == MISR_NORM_L1;
    hp.data_eps = hp.l1 ? (float)d.data_eps : 0.f;
}

// Tile grid of a shape; the TMA maps of the workspace images with that shape's boxes.
static int resident_ctas(int shape, int variant);
// Finish time of the busiest of `warps` warps that take, in list order, n_left items of cost
// a and then n_top items of cost b, each warp taking the next item when it is free.  After the
// left items, r warps are free at (q + 1) a and the rest at q a; the top items then finish at
// the merged times q a + k b and (q + 1) a + k b, k >= 1, that many warps at each.
static double edge_makespan(long warps, long n_left, double a, long n_top, double b) {
    if (warps <= 0) return n_left + n_top > 0 ? 1e300 : 0.0;
    const long q = n_left / warps, r = n_left % warps;
    double end = (q + (r > 0 ? 1 : 0)) * a;
    long left = n_top, k0 = 1, k1 = 1;
    const long c0 = warps - r, c1 = r;
    while (left > 0) {
        const double t0 = q * a + k0 * b, t1 = c1 > 0 ? (q + 1) * a + k1 * b : 1e300;
        if (t0 <= t1) { left -= c0; ++k0; end = std::max(end, t0); }
        else { left -= c1; ++k1; end = std::max(end, t1); }
    }
    return end;
}

// Items of the streaming shape (DevProblem: n_left, n_top, edge_h, tile_h, tiles_y, edge_ctas).
// An item of r rows takes r + 12 row steps (its pipeline); a step of a left-strip item costs
// STREAM_LEFT_COST and one of a top item STREAM_TOP_COST of an interior step.  Over the
// resident warps (8 per CTA, the launch's full grid), the split picks the number of edge CTAs
// E, the edge item height and the interior item height that minimise the later of the two
// paths' finish times, the interior items in one wave; those start at row edge_h >= 24 (below
// every top frame mask).  For a launch over this problem alone.
static void stream_split(DevProblem &hp) {
    const int H = hp.H, strips = hp.tiles_x;
    const int G = std::max(1, resident_ctas(STREAM_SHAPE, pass_variant(hp)));
    const int n_top = strips > 1 ? strips - 1 : 0;
    double best = -1.0;
    int b_e = G, b_eh = std::max(24, H), b_th = 24;
    const int e_lo = strips > 1 && G > 1 ? 1 : G, e_hi = strips > 1 && G > 1 ? G - 1 : G;
    for (int E = e_lo; E <= e_hi; ++E) {
        const long we = 8L * E, wi = 8L * (G - E);
        // edge item heights: the lowest height for each count of left-strip items
        for (long nl = (H + 23) / 24; nl >= 1; --nl) {
            const int eh = std::max(24, (int)((H + nl - 1) / nl));
            if ((H + eh - 1) / eh != nl) continue;
            const double steps = std::min(eh, H) + 12;
            const double te = edge_makespan(we, nl, STREAM_LEFT_COST * steps, n_top, STREAM_TOP_COST * steps);
            if (best >= 0 && te >= best) {
                if (nl + n_top <= we) break;   // one wave: taller items only finish later
                continue;
            }
            double ti = 0.0;
            int th = 24;
            const long R = (long)H - eh;
            if (strips > 1 && R > 0) {
                if (wi <= 0) continue;
                th = (int)std::max(24L, (R * (strips - 1) + wi - 1) / wi);
                while (th < R && ((R + th - 1) / th) * (strips - 1) > wi) ++th;
                ti = (double)(std::min<long>(th, R) + 12);
            }
            const double c = std::max(te, ti);
            if (best < 0 || c < best) { best = c; b_e = E; b_eh = eh; b_th = th; }
        }
    }
    hp.edge_h = b_eh;
    hp.tile_h = b_th;
    hp.edge_ctas = b_e;
    hp.n_left = (H + b_eh - 1) / b_eh;
    hp.n_top = n_top;
    const long R = (long)H - b_eh;
    hp.tiles_y = strips > 1 && R > 0 ? (int)((R + b_th - 1) / b_th) : 0;
    hp.n_tiles = hp.n_left + hp.n_top + (strips - 1) * hp.tiles_y;
}
static void set_shape(DevProblem &hp, int shape) {
    hp.shape = shape;
    hp.tile_w = SHAPE_TW[shape];
    hp.tiles_x = (hp.W + hp.tile_w - 1) / hp.tile_w;
    if (shape == STREAM_SHAPE) {
        stream_split(hp);
        return;
    }
    hp.tile_h = SHAPE_TH[shape];
    hp.tiles_y = (hp.H + hp.tile_h - 1) / hp.tile_h;
    hp.n_tiles = hp.tiles_y * hp.tiles_x;
    hp.n_left = hp.n_top = hp.edge_h = hp.edge_ctas = 0;
}
static misr_status make_maps(DevProblem &hp) {
    int xw = 0, xh = 0, ew = 0, eh = 0;
    // (the streaming kernel uses no tensor maps; its problems get those of the 32 x 32 tiles)
    with_shape(hp.shape == STREAM_SHAPE ? 1 : hp.shape, [&](auto S) {
        using G = ShapeGeo<decltype(S)::value>;
        xw = G::XW; xh = G::XH; ew = G::EW; eh = G::EH;
        return 0;
    });
    misr_status ms = get_encode_tiled();
    for (int i = 0; i < 2 && ms == MISR_OK; ++i) {
        ms = make_map(&hp.tmX[i], hp.X[i], hp.W, hp.H, hp.pitch, xw, xh, false);
        if (ms == MISR_OK) ms = make_map(&hp.tmR[i], hp.Rv[i], hp.W, hp.H, hp.pitch, xw, xh, false, hp.rp_bf16);
        if (ms == MISR_OK) ms = make_map(&hp.tmP[i], hp.Pv[i], hp.W, hp.H, hp.pitch, xw, xh, false, hp.rp_bf16);
    }
    if (ms == MISR_OK) ms = make_map(&hp.tmY, hp.Y, hp.W, hp.H, hp.pitch, ew, eh, true);
    return ms;
}

// Groups of the pass reduction: at least 64 tiles, at most 128 groups (the last group's
// warp sums all groups).
static void set_groups(DevProblem &hp) {
    hp.group = 64;
    while ((hp.n_tiles + hp.group - 1) / hp.group > 128) hp.group *= 2;
    hp.n_groups = (hp.n_tiles + hp.group - 1) / hp.group;
}

int misr_host::row_pitch(int W) { return (W + 7) & ~7; }   // 16-byte rows for float and bf16 planes

// The problem record of a descriptor without its buffers: geometry, taps, prior and data-term
// constants, tile shape (`shape`, or -1 for the plan's choice) and reduction groups.  Plans and
// the allocation-free gradient both build their records here, so they cannot disagree.
static misr_status fill_problem(const misr_desc &d, int iters, int shape, DevProblem &hp) {
    const int f = d.factor;
    hp = DevProblem{};
    hp.h = d.lr_h; hp.w = d.lr_w; hp.f = f; hp.K = d.K;
    hp.H = f * d.lr_h; hp.W = f * d.lr_w;
    hp.pitch = row_pitch(hp.W);
    hp.wait_tries = (int)TMA_WAIT_TRIES;
    hp.iters = iters;
    misr_status s = setup_geometry(d, hp);
    if (s != MISR_OK) return s;
    hp.lambda = (float)d.lambda; hp.eps = (float)d.eps; hp.eps2 = (float)(d.eps * d.eps);
    set_data_norm(hp, d);
    double eps_pairs = 0;
    for (int dy = 0; dy < BTV_W; ++dy)
        for (int dx = 0; dx < BTV_W; ++dx) {
            const int dd = dy * BTV_W + dx;
            float g = 0.f;
            if (dd != 0 && dx < d.btv_w && dy < d.btv_w) g = (float)std::pow(d.btv_alpha, dx + dy);
            hp.gamma[dd] = g;
            if (dd != 0 && hp.H > dy && hp.W > dx) eps_pairs += (double)g * (double)(hp.H - dy) * (double)(hp.W - dx);
        }
    hp.eps_pairs = d.eps * eps_pairs;
    hp.rp_bf16 = d.iterate_dtype == MISR_BF16;
    if (hp.general) {
        // the frame-wise pass: GEN_TILES kernels' CTAs of g_ctas each (the last one 2 g_ctas),
        // at least 8 elements per thread of the larger of the HR image and the frames, at most
        // 8 CTAs of 256 threads per SM of a 148-SM GPU
        const size_t n_max = std::max((size_t)hp.H * hp.W, (size_t)d.K * hp.h * hp.w);
        // the kernels index their tiles (at least 256 elements each) in 32 bits
        const size_t segs = (size_t)(hp.W + 1023) / 1024;
        if ((size_t)d.K * ((hp.h + 7) / 8) * ((hp.w + 31) / 32) >= (1u << 31) ||
            (size_t)((hp.H + 15) / 16) * ((hp.W + 31) / 32) >= (1u << 31) ||
            (size_t)d.K * hp.h * segs >= (1u << 31) ||
            (size_t)d.K * hp.H * ((hp.w + 1023) / 1024) >= (1u << 31))
            return fail(MISR_EINVAL, "frame-wise pass: more than 2^31 tiles");
        set_shape(hp, DEFAULT_SHAPE);
        hp.g_ctas = (int)std::min<size_t>(148 * 8, std::max<size_t>(1, (n_max + 2047) / 2048));
        hp.n_tiles = GEN_TILES * hp.g_ctas;
        set_groups(hp);
        return MISR_OK;
    }
    const int variant = desc_variant(d, hp.phased);
    const int sh = hp.phased ? PHASED_SHAPE : shape >= 0 ? shape : pick_shape(d, variant);
    if (!shape_takes_variant(sh, variant))
        return fail(MISR_ENOTIMPL, "the streaming pass runs integer shifts only");
    set_shape(hp, sh);
    set_groups(hp);
    return MISR_OK;
}

// Byte offsets of a plan's workspace (one allocation): X[2], Y (float), R[2], P[2] (float or
// bf16) | tile and group sums, group counters, pass counter, launch tile counter | state |
// trace | problem | tile list | group list | frame-wise pass only: the frames, the per-sample
// buffers DS psi_d'(e'), A_k p and psi_d''(e'), the tap tables.
struct PlanLayout {
    size_t img, rp_img, o_img, o_part, o_gpart, o_cnt, o_work, o_st, o_tr, o_pr, o_tm, o_gl, total;
    size_t lr, o_gy, o_ge, o_gap, o_gw, o_gty, o_gtx, o_gt, o_gh;
};
static PlanLayout plan_layout(const misr_desc &d, const DevProblem &hp) {
    PlanLayout L{};
    const size_t n_pitched = (size_t)hp.H * hp.pitch;
    L.img = align_up(n_pitched * sizeof(float), 256);
    L.rp_img = d.iterate_dtype == MISR_BF16 ? align_up(n_pitched * 2, 256) : L.img;
    size_t off = 0;
    L.o_img = off; off += 3 * L.img + 4 * L.rp_img;
    L.o_part = off; off += align_up((size_t)hp.n_tiles * NPART * sizeof(float2), 256);
    L.o_gpart = off; off += align_up((size_t)hp.n_groups * NPART * sizeof(float2), 256);
    L.o_cnt = off; off += 1024;   // the group counter, then the per-group item counters
    L.o_work = off; off += 256;
    L.o_st = off; off += align_up(sizeof(ScgState), 256);
    L.o_tr = off; off += align_up((size_t)std::max(d.iters, 1) * TRACE_COLS * sizeof(double), 256);
    L.o_pr = off; off += align_up(sizeof(DevProblem), 256);
    L.o_tm = off; off += align_up((size_t)hp.n_tiles * sizeof(int2), 256);
    L.o_gl = off; off += align_up((size_t)hp.n_groups * sizeof(int2), 256);
    if (hp.general) {
        L.lr = align_up((size_t)d.K * hp.h * hp.w * sizeof(float), 256);
        L.o_gy = off; off += L.lr;
        L.o_ge = off; off += L.lr;
        L.o_gap = off; off += L.lr;
        L.o_gw = off; off += hp.l1 ? L.lr : 0;
        L.o_gty = off; off += align_up((size_t)d.K * hp.h * hp.g_tw * sizeof(float), 256);
        L.o_gtx = off; off += align_up((size_t)d.K * hp.w * hp.g_tw * sizeof(float), 256);
        L.o_gt = off; off += align_up((size_t)d.K * hp.h * hp.W * sizeof(float), 256);
        L.o_gh = off; off += 2 * align_up((size_t)d.K * hp.H * hp.w * sizeof(float), 256);
    }
    L.total = off;
    return L;
}

size_t misr_host::plan_bytes(const misr_desc &d) {
    DevProblem hp;
    if (fill_problem(d, d.iters, -1, hp) != MISR_OK) return 0;
    return plan_layout(d, hp).total;
}

int misr_host::grid_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    return (int)std::min<size_t>(std::max<size_t>(b, 1), 148 * 16);
}

static misr_status launch_prepare(misr_plan_t p, const void *y_dev, const float *x_given, int flags,
                                  cudaStream_t s) {
    return launch_prepare_raw(p->dprob, 0, p->hp, p->d, y_dev, x_given, p->d.x0_mode, flags, s);
}

// Edge CTAs of a streaming launch: the split planned for a problem alone, or for several
// problems the average of their planned splits weighted by their work (each planned for the
// full grid), scaled to the launch's grid; at least one CTA while there are edge items, and
// one left for the rest.
static int stream_edge_ctas(const StreamRun &run, int grid) {
    if (run.n_edge >= run.count) return grid;
    if (run.edge_ctas > 0 && run.edge_ctas <= grid) return run.edge_ctas;
    const double tot = run.edge_work + run.int_work;
    const int full = resident_ctas(STREAM_SHAPE, run.variant);
    int e = tot > 0 ? (int)std::lround(run.edge_ctas_w / tot * grid / std::max(full, 1)) : 1;
    e = std::max(e, 1);
    if (grid > 1) e = std::min(e, grid - 1);
    return e;
}

misr_status misr_host::launch_pass_raw(const DevProblem *probs, const int2 *tiles, const PassSegs &segs,
                                       const int2 *groups, int n_groups, unsigned *work, int mode, double alpha,
                                       double beta, cudaStream_t s) {
    if (segs.total() <= 0) return MISR_OK;
    misr_status r = set_pass_attrs();
    if (r != MISR_OK) return r;
    // frame-wise problems: their four kernels each, one after the other
    for (const GenRun &g : segs.gen) {
        // each kernel in one wave, at most its resident CTAs (measured faster for all but D, whose
        // two roles run g_ctas CTAs each: one wave of its own 4 per SM left each role too few)
        const int G = g.ctas;
        gen_pass_a<<<gen_grid(gen_pass_a, G), GEN_NT, 0, s>>>(probs, g.pidx, mode, alpha, beta);
        with_gen_taps(g.tw, [&](auto T) {
            constexpr int twm = decltype(T)::value;
            auto kb = g.l1 ? gen_pass_b<true, twm> : gen_pass_b<false, twm>;
            auto kd = g.l1 ? gen_pass_d<true, twm> : gen_pass_d<false, twm>;
            const int hd = G;
            gen_pass_f1<twm, true><<<gen_grid(gen_pass_f1<twm, true>, G), GEN_NT, 0, s>>>(probs, g.pidx, mode, alpha, beta);
            kb<<<gen_grid(kb, G), GEN_NT, 0, s>>>(probs, g.pidx, mode, alpha, beta);
            gen_pass_c1<twm><<<gen_grid(gen_pass_c1<twm>, G), GEN_NT, 0, s>>>(probs, g.pidx, mode, alpha, beta);
            gen_pass_c2<twm><<<gen_grid(gen_pass_c2<twm>, G), GEN_NT, 0, s>>>(probs, g.pidx, mode, alpha, beta);
            gen_pass_f1<twm, false><<<gen_grid(gen_pass_f1<twm, false>, G), GEN_NT, 0, s>>>(probs, g.pidx, mode, alpha,
                                                                                          beta);
            kd<<<2 * hd, GEN_NT, 0, s>>>(probs, g.pidx, mode, alpha, beta, hd);
            return 0;
        });
        CK(cudaGetLastError());
    }
    int off = 0;
    for (int sh = 0; sh < N_SHAPES; ++sh)
        for (int v = 0; v < N_VARIANTS; ++v) {
            const int n = segs.n[sh][v];
            if (n <= 0) continue;
            if (sh == STREAM_SHAPE) {   // one launch per run of shared constants
                for (const StreamRun &run : segs.runs) {
                    if (run.variant != v) continue;
                    const int2 *t = tiles + off;
                    off += run.count;
                    // a problem alone gets the full grid its items were split for
                    const int grid = run.edge_ctas > 0 ? resident_ctas(sh, v) : pass_grid(sh, v, (run.count + 7) / 8);
                    const int ne = stream_edge_ctas(run, grid);
                    auto kern = v == 0 ? scg_stream_kernel<false, false> : v == 1 ? scg_stream_kernel<true, false>
                              : v == 2 ? scg_stream_kernel<false, true> : scg_stream_kernel<true, true>;
                    CK(launch_pdl(kern, grid, SW_NT, SW_SMEM_BYTES, s, probs, t, run.n_edge, run.count, ne, work, mode,
                                  alpha, beta, run.k, run.reduce_in_pass ? 1 : 0));
                }
                continue;
            }
            const int2 *t = tiles + off;
            off += n;
            CK(with_shape(sh, [&](auto S) {
                return with_variant(v, [&](auto V) {
                    constexpr int k = decltype(S)::value, vv = decltype(V)::value;
                    if constexpr (!compiled_variant<k, vv>() || k == STREAM_SHAPE) {
                        return cudaErrorInvalidValue;   // plans with per-phase taps take the PHASED_SHAPE
                    } else {
                        return launch_pdl(pass_kernel<k, vv>(), pass_grid(k, vv, n), SHAPE_NT[k], pass_smem<k, vv>(), s,
                                          probs, t, n, work, mode, alpha, beta);
                    }
                });
            }));
        }
    (void)n_groups;   // the list's length is the segments' count
    if (segs.n_reduce > 0) CK(launch_pdl(reduce_kernel, segs.n_reduce, 32, 0, s, probs, groups, mode));
    return MISR_OK;
}

misr_status misr_host::launch_prepare_raw(const DevProblem *probs, int pidx, const DevProblem &hp, const misr_desc &d,
                                          const void *y_dev, const float *x_given, int x0_mode, int flags,
                                          cudaStream_t s) {
    const float log_i0 = d.in_dtype == MISR_U16 ? logf(d.flat_field) : 0.f;
    const size_t n_pitched = (size_t)hp.H * hp.pitch;
    if (hp.general) {
        const size_t n = std::max(n_pitched, (size_t)hp.K * hp.h * hp.w);
        gen_prepare_kernel<<<grid_for(n, GEN_NT), GEN_NT, 0, s>>>(probs, pidx, y_dev, d.in_dtype, log_i0, x_given,
                                                                  x0_mode, flags);
    } else {
        prepare_kernel<<<grid_for(n_pitched, 256), 256, 0, s>>>(probs, pidx, y_dev, d.in_dtype, log_i0, x_given,
                                                                x0_mode, flags);
    }
    CK(cudaGetLastError());
    return MISR_OK;
}

misr_status misr_host::launch_finalize_raw(const DevProblem *probs, int pidx, size_t n, float *out, cudaStream_t s) {
    finalize_kernel<<<grid_for(n, 256), 256, 0, s>>>(probs, pidx, out);
    CK(cudaGetLastError());
    return MISR_OK;
}

// Every check misr_plan_create makes before allocating (descriptor, shifts, PSF).
misr_status misr_host::check_desc(const misr_desc &d) {
    misr_status s = validate(&d);
    if (s != MISR_OK) return s;
    DevProblem hp{};
    hp.f = d.factor;
    return setup_geometry(d, hp);
}

extern "C" {

const char *misr_version(void) {
#ifdef MISR_BOUNDS_CHECK
    return "misr-b300 0.5 (sm_103a, fused SCG pass: row-streaming warps, or persistent TMA-fed tiles 32x64, 32x32, "
           "16x64; frame-wise pass for any shift set; bounds-checked)";
#else
    return "misr-b300 0.5 (sm_103a, fused SCG pass: row-streaming warps, or persistent TMA-fed tiles 32x64, 32x32, "
           "16x64; frame-wise pass for any shift set)";
#endif
}

const char *misr_last_error(void) { return g_err.c_str(); }

misr_status misr_plan_create(const misr_desc *desc, misr_plan_t *out) {
    if (!out) return fail(MISR_EINVAL, "out is NULL");
    *out = nullptr;
    misr_status s = validate(desc);
    if (s != MISR_OK) return s;
    const misr_desc &d = *desc;
    DevProblem hp;
    s = fill_problem(d, d.iters, -1, hp);
    if (s != MISR_OK) return s;

    misr_plan_t p = new (std::nothrow) misr_plan_s();
    if (!p) return fail(MISR_ENOMEM, "host allocation failed");
    p->d = d;
    p->d.shifts = nullptr;
    p->d.psf = nullptr;
    cudaGetDevice(&p->device);
    p->n = (size_t)hp.H * hp.W;
    p->n_pitched = (size_t)hp.H * hp.pitch;
    p->m_total = (size_t)d.K * d.lr_h * d.lr_w;

    const PlanLayout lay = plan_layout(d, hp);
    const size_t off = lay.total, img = lay.img, rp_img = lay.rp_img, o_img = lay.o_img;
    const size_t o_part = lay.o_part, o_gpart = lay.o_gpart, o_cnt = lay.o_cnt, o_work = lay.o_work;
    const size_t o_st = lay.o_st, o_tr = lay.o_tr, o_pr = lay.o_pr, o_tm = lay.o_tm, o_gl = lay.o_gl;
    p->ws_bytes = off;
    cudaError_t e = cudaMalloc((void **)&p->ws, off);
    if (e != cudaSuccess) {
        delete p;
        cudaGetLastError();
        return fail(MISR_ENOMEM, "cudaMalloc(%zu) failed: %s", off, cudaGetErrorString(e));
    }
    char *b = p->ws;
    for (int i = 0; i < 2; ++i) {
        hp.X[i] = (float *)(b + o_img + (0 + i) * img);
        hp.Rv[i] = (float *)(b + o_img + 3 * img + (0 + i) * rp_img);
        hp.Pv[i] = (float *)(b + o_img + 3 * img + (2 + i) * rp_img);
    }
    hp.Y = (float *)(b + o_img + 2 * img);
    hp.partials = (float2 *)(b + o_part);
    hp.gpartials = (float2 *)(b + o_gpart);
    hp.counter = (unsigned int *)(b + o_cnt);
    hp.gcounter = (unsigned int *)(b + o_cnt + 256);
    p->work = (unsigned int *)(b + o_work);
    hp.st = (ScgState *)(b + o_st);
    hp.trace = (double *)(b + o_tr);
    p->dprob = (DevProblem *)(b + o_pr);
    p->dtile = (int2 *)(b + o_tm);
    p->dgroup = (int2 *)(b + o_gl);
    if (hp.general) {
        hp.Yg = (float *)(b + lay.o_gy);
        hp.Eg = (float *)(b + lay.o_ge);
        hp.APg = (float *)(b + lay.o_gap);
        hp.Wg = hp.l1 ? (float *)(b + lay.o_gw) : nullptr;
        hp.Ty = (float *)(b + lay.o_gty);
        hp.Tx = (float *)(b + lay.o_gtx);
        hp.Tg = (float *)(b + lay.o_gt);
        hp.Hg[0] = (float *)(b + lay.o_gh);
        hp.Hg[1] = (float *)(b + lay.o_gh + align_up((size_t)d.K * hp.H * hp.w * sizeof(float), 256));
    }
    {
        const misr_status ms = make_maps(hp);
        if (ms != MISR_OK) {
            cudaFree(p->ws);
            delete p;
            return ms;
        }
    }
    p->hp = hp;

    std::vector<int2> tiles, groups;
    build_pass_lists({&p->hp}, {0}, tiles, groups, p->segs);
    misr_status rs = MISR_OK;
    do {
        if ((e = cudaMemset(p->ws, 0, off)) != cudaSuccess) break;
        if ((e = cudaMemcpy(p->dprob, &p->hp, sizeof(DevProblem), cudaMemcpyHostToDevice)) != cudaSuccess) break;
        if (!tiles.empty() &&
            (e = cudaMemcpy(p->dtile, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice)) != cudaSuccess)
            break;
        if (p->hp.general) {
            gen_prime_grids(p->hp.g_tw);
            std::vector<float> Ty, Tx;
            if ((rs = gen_tables(d, p->hp, Ty, Tx)) != MISR_OK) break;
            if ((e = cudaMemcpy(p->hp.Ty, Ty.data(), Ty.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) break;
            if ((e = cudaMemcpy(p->hp.Tx, Tx.data(), Tx.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) break;
        }
        if ((e = cudaMemcpy(p->dgroup, groups.data(), groups.size() * sizeof(int2), cudaMemcpyHostToDevice)) != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming)) != cudaSuccess) break;
        if ((e = cudaMallocHost((void **)&p->st_host, sizeof(ScgState))) != cudaSuccess) break;
        rs = set_pass_attrs();
    } while (0);
    if (e != cudaSuccess || rs != MISR_OK) {
        misr_status r = rs != MISR_OK ? rs : fail(MISR_ECUDA, "plan setup: %s", cudaGetErrorString(e));
        misr_plan_destroy(p);
        return r;
    }
    *out = p;
    return MISR_OK;
}

misr_status misr_plan_destroy(misr_plan_t p) {
    if (!p) return MISR_OK;
    DeviceGuard g(p->device);
    cudaDeviceSynchronize();
    if (p->chunk) cudaGraphExecDestroy(p->chunk);
    if (p->tail) cudaGraphExecDestroy(p->tail);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->done_ev) cudaEventDestroy(p->done_ev);
    if (p->st_host) cudaFreeHost(p->st_host);
    if (p->io_y) cudaFree(p->io_y);
    if (p->io_x) cudaFree(p->io_x);
    for (int b = 0; b < 2; ++b) {
        if (p->pio_y[b]) cudaFree(p->pio_y[b]);
        if (p->pio_x[b]) cudaFree(p->pio_x[b]);
        if (p->ev_in[b]) cudaEventDestroy(p->ev_in[b]);
        if (p->ev_done[b]) cudaEventDestroy(p->ev_done[b]);
        if (p->ev_out[b]) cudaEventDestroy(p->ev_out[b]);
    }
    if (p->cpy) cudaStreamDestroy(p->cpy);
    if (p->st_ring) cudaFree(p->st_ring);
    if (p->ws) cudaFree(p->ws);
    delete p;
    return MISR_OK;
}

misr_status misr_plan_set_wait_limit(misr_plan_t p, uint32_t tries) {
    if (!p) return fail(MISR_EINVAL, "plan is NULL");
    DeviceGuard g(p->device);
    p->hp.wait_tries = (int)std::min<uint32_t>(tries, 0x7fffffffu);
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(p->dprob, &p->hp, sizeof(DevProblem), cudaMemcpyHostToDevice));
    return MISR_OK;
}

misr_status misr_plan_workspace_bytes(misr_plan_t p, size_t *bytes) {
    if (!p || !bytes) return fail(MISR_EINVAL, "NULL argument");
    *bytes = p->ws_bytes;
    return MISR_OK;
}

misr_status misr_forward(misr_plan_t p, const float *x_dev, float *y_dev, misr_stream_t stream) {
    if (!p || !x_dev || !y_dev) return fail(MISR_EINVAL, "NULL argument");
    DeviceGuard g(p->device);
    if (p->hp.general)
        gen_forward_kernel<<<grid_for(p->m_total, GEN_NT), GEN_NT, 0, (cudaStream_t)stream>>>(p->dprob, 0, x_dev, y_dev);
    else
        forward_kernel<<<grid_for(p->m_total, 256), 256, 0, (cudaStream_t)stream>>>(p->dprob, 0, x_dev, y_dev);
    CK(cudaGetLastError());
    return MISR_OK;
}

}  // extern "C"

template <int F>
static cudaError_t launch_interpolate(const misr_plan_t p, const void *y_dev, float *x_dev, float log_i0,
                                      cudaStream_t s) {
    const int gx = (int)std::min<size_t>(((size_t)p->hp.w + 4 * 256 - 1) / (4 * 256), 64);
    const int gy = std::min(p->hp.H, 65535);
    interpolate_kernel<F><<<dim3(gx, gy), 256, 0, s>>>(p->dprob, 0, y_dev, p->d.in_dtype, log_i0, x_dev);
    return cudaGetLastError();
}

extern "C" {

misr_status misr_interpolate(misr_plan_t p, const void *y_dev, float *x_dev, misr_stream_t stream) {
    if (!p || !y_dev || !x_dev) return fail(MISR_EINVAL, "NULL argument");
    DeviceGuard g(p->device);
    const float log_i0 = p->d.in_dtype == MISR_U16 ? logf(p->d.flat_field) : 0.f;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->hp.general) {   // frame-wise problems: each pixel gathers every frame's samples
        gen_interpolate_kernel<<<grid_for(p->n, GEN_NT), GEN_NT, 0, s>>>(p->dprob, 0, y_dev, p->d.in_dtype, log_i0, x_dev);
        CK(cudaGetLastError());
        return MISR_OK;
    }
    if (p->hp.phased) {   // non-integer shifts: each pixel gathers its bilinear weights
        interpolate_phased_kernel<<<grid_for(p->n, 256), 256, 0, s>>>(p->dprob, 0, y_dev, p->d.in_dtype, log_i0, x_dev);
        CK(cudaGetLastError());
        return MISR_OK;
    }
    static_assert(MAXF == 8, "one case per factor");
    switch (p->hp.f) {
    case 1: CK(launch_interpolate<1>(p, y_dev, x_dev, log_i0, s)); break;
    case 2: CK(launch_interpolate<2>(p, y_dev, x_dev, log_i0, s)); break;
    case 3: CK(launch_interpolate<3>(p, y_dev, x_dev, log_i0, s)); break;
    case 4: CK(launch_interpolate<4>(p, y_dev, x_dev, log_i0, s)); break;
    case 5: CK(launch_interpolate<5>(p, y_dev, x_dev, log_i0, s)); break;
    case 6: CK(launch_interpolate<6>(p, y_dev, x_dev, log_i0, s)); break;
    case 7: CK(launch_interpolate<7>(p, y_dev, x_dev, log_i0, s)); break;
    default: CK(launch_interpolate<8>(p, y_dev, x_dev, log_i0, s)); break;
    }
    return MISR_OK;
}

misr_status misr_pass_probe(misr_plan_t p, const void *y_dev, const float *x_dev, const float *r_dev,
                            const float *p_old_dev, double alpha, double beta, float *x_out_dev,
                            float *r_out_dev, float *p_out_dev, double *sums, misr_stream_t stream) {
    if (!p || !y_dev || !x_dev || !r_dev || !p_old_dev || !sums) return fail(MISR_EINVAL, "NULL argument");
    if (!std::isfinite(alpha) || !std::isfinite(beta)) return fail(MISR_EINVAL, "alpha, beta must be finite");
    if (p->hp.rp_bf16) return fail(MISR_ENOTIMPL, "misr_pass_probe takes float r and p: use a MISR_F32 iterate plan");
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t wb = (size_t)p->hp.W * sizeof(float), pb = (size_t)p->hp.pitch * sizeof(float);
    const size_t hrows = (size_t)p->hp.H;
    misr_status r = launch_prepare(p, y_dev, nullptr, 4, s);
    if (r != MISR_OK) return r;
    CK(cudaMemcpy2DAsync(p->hp.X[0], pb, x_dev, wb, wb, hrows, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpy2DAsync(p->hp.Rv[0], pb, r_dev, wb, wb, hrows, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpy2DAsync(p->hp.Pv[0], pb, p_old_dev, wb, wb, hrows, cudaMemcpyDeviceToDevice, s));
    r = launch_pass(p, MODE_PROBE, alpha, beta, s);
    if (r != MISR_OK) return r;
    if (x_out_dev) CK(cudaMemcpy2DAsync(x_out_dev, wb, p->hp.X[1], pb, wb, hrows, cudaMemcpyDeviceToDevice, s));
    if (r_out_dev) CK(cudaMemcpy2DAsync(r_out_dev, wb, p->hp.Rv[1], pb, wb, hrows, cudaMemcpyDeviceToDevice, s));
    if (p_out_dev) CK(cudaMemcpy2DAsync(p_out_dev, wb, p->hp.Pv[1], pb, wb, hrows, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(p->st_host, p->hp.st, sizeof(ScgState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (p->st_host->status != DEV_OK) return fail(MISR_ETIMEOUT, "a tile load of the fused pass did not complete in time");
    for (int i = 0; i < NPART; ++i) sums[i] = p->st_host->sums[i];
    sums[P_JB] -= p->hp.eps_pairs;   // R_BTV(x') without lambda
    return MISR_OK;
}

misr_status misr_gradient(misr_plan_t p, const void *y_dev, const float *x_dev, float *g_dev, double *J_out,
                          misr_stream_t stream) {
    if (!p || !y_dev || !x_dev || !g_dev) return fail(MISR_EINVAL, "NULL argument");
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int saved = p->d.x0_mode;
    p->d.x0_mode = MISR_X0_GIVEN;
    misr_status r = launch_prepare(p, y_dev, x_dev, 1 | 2 | 4, s);
    p->d.x0_mode = saved;
    if (r != MISR_OK) return r;
    r = launch_pass(p, MODE_PROBE, 0.0, 0.0, s);
    if (r != MISR_OK) return r;
    if (p->hp.rp_bf16)
        scale_copy_kernel<<<grid_for(p->n, 256), 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(p->hp.Rv[1]),
                                                              p->hp.pitch, -1.f, g_dev, p->hp.H, p->hp.W);
    else
        scale_copy_kernel<<<grid_for(p->n, 256), 256, 0, s>>>(p->hp.Rv[1], p->hp.pitch, -1.f, g_dev, p->hp.H, p->hp.W);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(p->st_host, p->hp.st, sizeof(ScgState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (p->st_host->status != DEV_OK) return fail(MISR_ETIMEOUT, "a tile load of the fused pass did not complete in time");
    if (J_out) {
        const double *S = p->st_host->sums;
        *J_out = S[P_JD] + (double)p->hp.lambda * (S[P_JB] - p->hp.eps_pairs);
    }
    return MISR_OK;
}

// `len` SCG passes of the plan, captured on its private stream
static misr_status capture_passes(misr_plan_t p, int len, cudaGraphExec_t *exec) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
    misr_status r = MISR_OK;
    for (int i = 0; i < len && r == MISR_OK; ++i) r = launch_pass(p, MODE_ITER, 0.0, 0.0, p->cap);
    cudaError_t e = cudaStreamEndCapture(p->cap, &graph);
    if (r != MISR_OK) { if (graph) cudaGraphDestroy(graph); return r; }
    if (e != cudaSuccess) return fail(MISR_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(MISR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return MISR_OK;
}

// The plan's graphs: a chunk of GRAPH_CHUNK passes and the remainder of its iteration count, so
// that a solve launches exactly that many passes (none that would only find it done)
static misr_status ensure_graph(misr_plan_t p) {
    const int want = std::max(1, std::min(p->d.iters, GRAPH_CHUNK));
    const int tail = std::max(p->d.iters, 0) % want;
    if (p->chunk && p->chunk_len == want && p->tail_len == tail) return MISR_OK;
    if (p->chunk) { cudaGraphExecDestroy(p->chunk); p->chunk = nullptr; }
    if (p->tail) { cudaGraphExecDestroy(p->tail); p->tail = nullptr; }
    p->chunk_len = p->tail_len = 0;
    misr_status r = capture_passes(p, want, &p->chunk);
    if (r != MISR_OK) return r;
    if (tail > 0) r = capture_passes(p, tail, &p->tail);
    if (r != MISR_OK) { cudaGraphExecDestroy(p->chunk); p->chunk = nullptr; return r; }
    p->chunk_len = want;
    p->tail_len = tail;
    return MISR_OK;
}

// n SCG passes: whole chunks, then the tail graph when it is the rest, else single launches
static misr_status launch_iters(misr_plan_t p, int n, cudaStream_t s) {
    int done = 0;
    for (; done + p->chunk_len <= n; done += p->chunk_len) CK(cudaGraphLaunch(p->chunk, s));
    const int rest = n - done;
    if (rest > 0 && rest == p->tail_len) {
        CK(cudaGraphLaunch(p->tail, s));
        return MISR_OK;
    }
    for (int i = 0; i < rest; ++i) {
        const misr_status r = launch_pass(p, MODE_ITER, 0.0, 0.0, s);
        if (r != MISR_OK) return r;
    }
    return MISR_OK;
}

static misr_status fill_stats_from(const ScgState &h, misr_stats *st) {
    if (h.status == DEV_TMA_TIMEOUT) {
        st->status = MISR_ETIMEOUT;
        return fail(MISR_ETIMEOUT, "a tile load of the fused pass did not complete in time; the solve stopped");
    }
    st->iters_done = h.iter;
    st->accepted = h.accepted;
    st->status = MISR_OK;
    st->reserved = 0;
    st->J_final = h.E;
    st->rnorm2 = h.rn2;
    st->lambda_scg = h.lam;
    return MISR_OK;
}
static misr_status fill_stats(misr_plan_t p, misr_stats *st) { return fill_stats_from(*p->st_host, st); }

misr_status misr_solve(misr_plan_t p, const void *y_dev, float *x_dev, misr_stream_t stream, misr_stats *stats) {
    if (!p || !y_dev || !x_dev) return fail(MISR_EINVAL, "NULL argument");
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    misr_status r = ensure_graph(p);
    if (r != MISR_OK) return r;
    r = launch_prepare(p, y_dev, x_dev, 1 | 2 | 4, s);
    if (r != MISR_OK) return r;
    r = launch_pass(p, MODE_INIT, 0.0, 0.0, s);
    if (r != MISR_OK) return r;
    r = launch_iters(p, std::max(p->d.iters, 0), s);
    if (r != MISR_OK) return r;
    finalize_kernel<<<grid_for(p->n, 256), 256, 0, s>>>(p->dprob, 0, x_dev);
    CK(cudaGetLastError());
    CK(cudaEventRecord(p->done_ev, s));
    p->solved = true;
    if (stats) {
        CK(cudaMemcpyAsync(p->st_host, p->hp.st, sizeof(ScgState), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return fill_stats(p, stats);
    }
    return MISR_OK;
}

misr_status misr_solve_host(misr_plan_t p, const void *y_host, float *x_host, misr_stats *stats) {
    if (!p || !y_host || !x_host) return fail(MISR_EINVAL, "NULL argument");
    DeviceGuard g(p->device);
    misr_status gr = ensure_graph(p);   // capture on the private stream before it queues copies
    if (gr != MISR_OK) return gr;
    const size_t ybytes = p->m_total * (p->d.in_dtype == MISR_U16 ? 2 : 4);
    const size_t xbytes = p->n * sizeof(float);
    if (!p->io_y) {
        cudaError_t e = cudaMalloc(&p->io_y, ybytes);
        if (e != cudaSuccess) { cudaGetLastError(); return fail(MISR_ENOMEM, "cudaMalloc y: %s", cudaGetErrorString(e)); }
    }
    if (!p->io_x) {
        cudaError_t e = cudaMalloc((void **)&p->io_x, xbytes);
        if (e != cudaSuccess) { cudaGetLastError(); return fail(MISR_ENOMEM, "cudaMalloc x: %s", cudaGetErrorString(e)); }
    }
    cudaStream_t s = p->cap;
    CK(cudaMemcpyAsync(p->io_y, y_host, ybytes, cudaMemcpyHostToDevice, s));
    if (p->d.x0_mode == MISR_X0_GIVEN) CK(cudaMemcpyAsync(p->io_x, x_host, xbytes, cudaMemcpyHostToDevice, s));
    misr_status r = misr_solve(p, p->io_y, p->io_x, (misr_stream_t)s, nullptr);
    if (r != MISR_OK) return r;
    CK(cudaMemcpyAsync(x_host, p->io_x, xbytes, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(p->st_host, p->hp.st, sizeof(ScgState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (stats) return fill_stats(p, stats);
    return MISR_OK;
}

// The buffers, stream and events of misr_solve_host_many (kept with the plan).
static misr_status ensure_stream_io(misr_plan_t p, size_t ybytes, size_t xbytes, int n_states) {
    for (int b = 0; b < 2; ++b) {
        if (!p->pio_y[b] && cudaMalloc(&p->pio_y[b], ybytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(MISR_ENOMEM, "cudaMalloc of the frame buffers of misr_solve_host_many");
        }
        if (!p->pio_x[b] && cudaMalloc((void **)&p->pio_x[b], xbytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(MISR_ENOMEM, "cudaMalloc of the image buffers of misr_solve_host_many");
        }
        if (!p->ev_in[b]) CK(cudaEventCreateWithFlags(&p->ev_in[b], cudaEventDisableTiming));
        if (!p->ev_done[b]) CK(cudaEventCreateWithFlags(&p->ev_done[b], cudaEventDisableTiming));
        if (!p->ev_out[b]) CK(cudaEventCreateWithFlags(&p->ev_out[b], cudaEventDisableTiming));
    }
    if (!p->cpy) CK(cudaStreamCreateWithFlags(&p->cpy, cudaStreamNonBlocking));
    if (n_states > p->st_ring_cap) {
        if (p->st_ring) { cudaFree(p->st_ring); p->st_ring = nullptr; p->st_ring_cap = 0; }
        if (cudaMalloc((void **)&p->st_ring, sizeof(ScgState) * (size_t)n_states) != cudaSuccess) {
            cudaGetLastError();
            return fail(MISR_ENOMEM, "cudaMalloc of the state records of misr_solve_host_many");
        }
        p->st_ring_cap = n_states;
    }
    return MISR_OK;
}

misr_status misr_solve_host_many(misr_plan_t p, int32_t n, const void *const *y_host, float *const *x_host,
                                 misr_stats *stats) {
    if (!p || n < 0 || (n > 0 && (!y_host || !x_host))) return fail(MISR_EINVAL, "NULL plan or arrays, or n < 0");
    for (int32_t k = 0; k < n; ++k)
        if (!y_host[k] || !x_host[k]) return fail(MISR_EINVAL, "projection %d: NULL host buffer", (int)k);
    if (n == 0) return MISR_OK;
    DeviceGuard g(p->device);
    misr_status r = ensure_graph(p);   // captured on the plan's stream before work is queued on it
    if (r != MISR_OK) return r;
    const size_t ybytes = p->m_total * (p->d.in_dtype == MISR_U16 ? 2 : 4);
    const size_t xbytes = p->n * sizeof(float);
    r = ensure_stream_io(p, ybytes, xbytes, stats ? n : 0);
    if (r != MISR_OK) return r;
    cudaStream_t s = p->cap, c = p->cpy;
    const bool x_in = p->d.x0_mode == MISR_X0_GIVEN;
    // projection k uses buffer pair k & 1.  Copy stream: in(0), then for each k: in(k+1) once
    // solve k-1 has read pair (k+1) & 1, out(k) once solve k is done.  Plan stream: solve k
    // once in(k) has landed and out(k-2) has left pair k & 1.
    auto copy_in = [&](int32_t k) -> misr_status {
        const int b = k & 1;
        if (k >= 2) CK(cudaStreamWaitEvent(c, p->ev_done[b], 0));
        CK(cudaMemcpyAsync(p->pio_y[b], y_host[k], ybytes, cudaMemcpyHostToDevice, c));
        if (x_in) CK(cudaMemcpyAsync(p->pio_x[b], x_host[k], xbytes, cudaMemcpyHostToDevice, c));
        CK(cudaEventRecord(p->ev_in[b], c));
        return MISR_OK;
    };
    r = copy_in(0);
    for (int32_t k = 0; k < n && r == MISR_OK; ++k) {
        const int b = k & 1;
        CK(cudaStreamWaitEvent(s, p->ev_in[b], 0));
        if (k >= 2) CK(cudaStreamWaitEvent(s, p->ev_out[b], 0));
        r = misr_solve(p, p->pio_y[b], p->pio_x[b], (misr_stream_t)s, nullptr);
        if (r != MISR_OK) break;
        if (stats) CK(cudaMemcpyAsync(p->st_ring + k, p->hp.st, sizeof(ScgState), cudaMemcpyDeviceToDevice, s));
        CK(cudaEventRecord(p->ev_done[b], s));
        if (k + 1 < n) r = copy_in(k + 1);
        if (r != MISR_OK) break;
        CK(cudaStreamWaitEvent(c, p->ev_done[b], 0));
        CK(cudaMemcpyAsync(x_host[k], p->pio_x[b], xbytes, cudaMemcpyDeviceToHost, c));
        CK(cudaEventRecord(p->ev_out[b], c));
    }
    const cudaError_t e1 = cudaStreamSynchronize(s), e2 = cudaStreamSynchronize(c);
    if (r != MISR_OK) return r;
    if (e1 != cudaSuccess || e2 != cudaSuccess)
        return fail(MISR_ECUDA, "misr_solve_host_many: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    if (!stats) return MISR_OK;
    std::vector<ScgState> h((size_t)n);
    CK(cudaMemcpy(h.data(), p->st_ring, sizeof(ScgState) * (size_t)n, cudaMemcpyDeviceToHost));
    *p->st_host = h[(size_t)n - 1];
    misr_status worst = MISR_OK;
    for (int32_t k = 0; k < n; ++k) {
        const misr_status sk = fill_stats_from(h[(size_t)k], &stats[k]);
        if (sk != MISR_OK) worst = sk;
    }
    return worst;
}

misr_status misr_debug_bounds(uint32_t *bits, int32_t *first) {
    if (!bits) return fail(MISR_EINVAL, "bits is NULL");
#ifdef MISR_BOUNDS_CHECK
    CK(cudaDeviceSynchronize());
    unsigned int b = 0;
    int f[4] = {0, 0, 0, 0};
    CK(cudaMemcpyFromSymbol(&b, misr::g_bounds_bits, sizeof b));
    CK(cudaMemcpyFromSymbol(f, misr::g_bounds_first, sizeof f));
    const unsigned int zero = 0;
    const int zeros[4] = {0, 0, 0, 0};
    CK(cudaMemcpyToSymbol(misr::g_bounds_bits, &zero, sizeof zero));
    CK(cudaMemcpyToSymbol(misr::g_bounds_first, zeros, sizeof zeros));
    *bits = b;
    if (first) std::memcpy(first, f, sizeof f);
    return MISR_OK;
#else
    *bits = 0;
    if (first) std::memset(first, 0, 4 * sizeof(int32_t));
    return fail(MISR_ENOTIMPL, "this library was built without bounds checks (libmisr_check.so has them)");
#endif
}

// ---- checkpoint and resume
namespace {
struct CkptHeader {
    uint32_t magic, version, H, W, bf16, state_bytes, l1, model;
};
static_assert(sizeof(CkptHeader) == 32, "checkpoint header");
constexpr uint32_t CKPT_MAGIC = 0x4353524du, CKPT_VERSION = 3u;
// FNV-1a hash of the model a state belongs to: frames and shifts, blur taps (with binning and
// per-phase taps folded in), the prior's and the data term's constants.  A checkpoint resumes
// only on a plan of the same model (the iteration count may differ).
uint32_t model_hash(const DevProblem &hp) {
    uint32_t hsh = 2166136261u;
    auto mix = [&](const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) hsh = (hsh ^ b[i]) * 16777619u;
    };
    mix(&hp.f, sizeof hp.f);
    mix(&hp.K, sizeof hp.K);
    mix(hp.ty, sizeof(int) * hp.K);
    mix(hp.tx, sizeof(int) * hp.K);
    mix(hp.frame_of_phase, sizeof hp.frame_of_phase);
    mix(hp.hy, sizeof hp.hy);
    mix(hp.hx, sizeof hp.hx);
    mix(&hp.phased, sizeof hp.phased);
    mix(&hp.general, sizeof hp.general);
    if (hp.general) {   // the frame-wise pass: fractional shifts, D's block, the tap window
        mix(hp.gfy, sizeof(float) * hp.K);
        mix(hp.gfx, sizeof(float) * hp.K);
        mix(&hp.g_nb, sizeof hp.g_nb);
        mix(&hp.g_r, sizeof hp.g_r);
        mix(&hp.g_tw, sizeof hp.g_tw);
    }
    if (hp.phased) {
        mix(hp.ay, sizeof hp.ay);
        mix(hp.ax, sizeof hp.ax);
        mix(hp.tph, sizeof hp.tph);
    }
    mix(&hp.lambda, sizeof hp.lambda);
    mix(&hp.eps, sizeof hp.eps);
    mix(hp.gamma, sizeof hp.gamma);
    mix(&hp.l1, sizeof hp.l1);
    mix(&hp.data_eps, sizeof hp.data_eps);
    return hsh;
}
size_t ckpt_bytes(const misr_plan_t p) {
    const size_t n = (size_t)p->hp.H * p->hp.W, rp = p->hp.rp_bf16 ? 2 : 4;
    return sizeof(CkptHeader) + sizeof(ScgState) + n * 4 + 2 * n * rp;
}
}  // namespace

misr_status misr_state_bytes(misr_plan_t p, size_t *bytes) {
    if (!p || !bytes) return fail(MISR_EINVAL, "NULL argument");
    *bytes = ckpt_bytes(p);
    return MISR_OK;
}

misr_status misr_export_state(misr_plan_t p, void *buf, size_t bytes) {
    if (!p || !buf) return fail(MISR_EINVAL, "NULL argument");
    if (bytes < ckpt_bytes(p)) return fail(MISR_EINVAL, "checkpoint buffer of %zu bytes, %zu needed", bytes, ckpt_bytes(p));
    DeviceGuard g(p->device);
    CK(cudaDeviceSynchronize());
    ScgState st;
    CK(cudaMemcpy(&st, p->hp.st, sizeof(ScgState), cudaMemcpyDeviceToHost));
    const size_t W = p->hp.W, H = p->hp.H, pitch = p->hp.pitch, rp = p->hp.rp_bf16 ? 2 : 4;
    char *out = static_cast<char *>(buf);
    CkptHeader h{CKPT_MAGIC, CKPT_VERSION, (uint32_t)H, (uint32_t)W, (uint32_t)p->hp.rp_bf16, (uint32_t)sizeof(ScgState),
                 (uint32_t)p->hp.l1, model_hash(p->hp)};
    std::memcpy(out, &h, sizeof h);
    std::memcpy(out + sizeof h, &st, sizeof st);
    char *planes = out + sizeof h + sizeof st;
    CK(cudaMemcpy2D(planes, W * 4, p->hp.X[st.cur], pitch * 4, W * 4, H, cudaMemcpyDeviceToHost));
    planes += H * W * 4;
    CK(cudaMemcpy2D(planes, W * rp, p->hp.Rv[st.cur], pitch * rp, W * rp, H, cudaMemcpyDeviceToHost));
    planes += H * W * rp;
    CK(cudaMemcpy2D(planes, W * rp, p->hp.Pv[st.pcur], pitch * rp, W * rp, H, cudaMemcpyDeviceToHost));
    return MISR_OK;
}

misr_status misr_import_state(misr_plan_t p, const void *buf, size_t bytes) {
    if (!p || !buf) return fail(MISR_EINVAL, "NULL argument");
    if (bytes < sizeof(CkptHeader)) return fail(MISR_EINVAL, "checkpoint buffer too small");
    CkptHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (h.magic != CKPT_MAGIC || h.version != CKPT_VERSION) return fail(MISR_EINVAL, "not a checkpoint of this version");
    if (h.H != (uint32_t)p->hp.H || h.W != (uint32_t)p->hp.W || h.bf16 != (uint32_t)p->hp.rp_bf16 ||
        h.state_bytes != (uint32_t)sizeof(ScgState) || h.l1 != (uint32_t)p->hp.l1)
        return fail(MISR_EINVAL, "checkpoint of another geometry, storage type, data term or state layout");
    if (h.model != model_hash(p->hp))
        return fail(MISR_EINVAL, "checkpoint of another model (shifts, PSF, decimation or prior/data constants)");
    if (bytes < ckpt_bytes(p)) return fail(MISR_EINVAL, "checkpoint buffer of %zu bytes, %zu needed", bytes, ckpt_bytes(p));
    DeviceGuard g(p->device);
    CK(cudaDeviceSynchronize());
    const char *in = static_cast<const char *>(buf);
    ScgState st;
    std::memcpy(&st, in + sizeof h, sizeof st);
    const size_t W = p->hp.W, H = p->hp.H, pitch = p->hp.pitch, rp = p->hp.rp_bf16 ? 2 : 4;
    const char *planes = in + sizeof h + sizeof st;
    CK(cudaMemcpy2D(p->hp.X[0], pitch * 4, planes, W * 4, W * 4, H, cudaMemcpyHostToDevice));
    planes += H * W * 4;
    CK(cudaMemcpy2D(p->hp.Rv[0], pitch * rp, planes, W * rp, W * rp, H, cudaMemcpyHostToDevice));
    planes += H * W * rp;
    CK(cudaMemcpy2D(p->hp.Pv[0], pitch * rp, planes, W * rp, W * rp, H, cudaMemcpyHostToDevice));
    // the buffers now hold the checkpoint's halves at index 0; the iteration target is this
    // plan's, and a solve stopped only by its count is live again below it
    st.cur = 0;
    st.pcur = 0;
    st.iters = p->d.iters;
    st.done = (st.status != 0 || st.iter >= st.iters || !(st.pn2 > 0.0) || !std::isfinite(st.alpha)) ? 1 : 0;
    CK(cudaMemcpy(p->hp.st, &st, sizeof st, cudaMemcpyHostToDevice));
    CK(cudaMemset(p->hp.counter, 0, 1024));
    CK(cudaMemset(p->work, 0, 4 * sizeof(unsigned int)));
    CK(cudaMemset(p->hp.trace, 0, (size_t)std::max(p->d.iters, 1) * TRACE_COLS * sizeof(double)));
    *p->st_host = st;
    p->solved = true;
    return MISR_OK;
}

misr_status misr_resume(misr_plan_t p, const void *y_dev, float *x_dev, misr_stream_t stream, misr_stats *stats) {
    if (!p || !y_dev || !x_dev) return fail(MISR_EINVAL, "NULL argument");
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    misr_status r = ensure_graph(p);
    if (r != MISR_OK) return r;
    ScgState st;
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(&st, p->hp.st, sizeof(ScgState), cudaMemcpyDeviceToHost));
    // the frames again (Y only: no start point, no reset)
    r = launch_prepare_raw(p->dprob, 0, p->hp, p->d, y_dev, nullptr, MISR_X0_ZERO, 0, s);
    if (r != MISR_OK) return r;
    const int remaining = st.done ? 0 : std::max(st.iters - st.iter, 0);
    r = launch_iters(p, remaining, s);
    if (r != MISR_OK) return r;
    finalize_kernel<<<grid_for(p->n, 256), 256, 0, s>>>(p->dprob, 0, x_dev);
    CK(cudaGetLastError());
    CK(cudaEventRecord(p->done_ev, s));
    p->solved = true;
    if (stats) {
        CK(cudaMemcpyAsync(p->st_host, p->hp.st, sizeof(ScgState), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return fill_stats(p, stats);
    }
    return MISR_OK;
}

misr_status misr_get_trace(misr_plan_t p, double *out, int32_t max_rows, int32_t *rows) {
    if (!p || !out || !rows || max_rows < 0) return fail(MISR_EINVAL, "bad argument");
    DeviceGuard g(p->device);
    *rows = 0;
    if (!p->solved) return MISR_OK;
    CK(cudaEventSynchronize(p->done_ev));
    CK(cudaMemcpy(p->st_host, p->hp.st, sizeof(ScgState), cudaMemcpyDeviceToHost));
    const int n = std::min(p->st_host->iter, (int)max_rows);
    if (n > 0) CK(cudaMemcpy(out, p->hp.trace, (size_t)n * TRACE_COLS * sizeof(double), cudaMemcpyDeviceToHost));
    *rows = n;
    return MISR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Allocation-free objective/gradient (misr_gradient_noalloc).
//
// For callers that must not allocate device memory at all: a process whose device memory
// is already reserved by another allocator (a framework's caching pool or a detector
// pipeline that pre-reserves every byte), where cudaMalloc would fail or would force a
// device-wide synchronisation in the middle of a time-critical acquisition loop.  The
// workspace lives in the file-scope array below, sized for HR images up to
// NOALLOC_MAX_H x NOALLOC_MAX_W; every GPU that loads this library holds it until the
// process exits.  All calls share it, so calls that overlap on the GPU (other streams,
// other host threads) race.
namespace {

constexpr size_t na_align(size_t v, size_t a) { return (v + a - 1) / a * a; }
constexpr int NOALLOC_MAX_H = 512, NOALLOC_MAX_W = 512;
constexpr size_t NOALLOC_IMG = na_align(size_t(NOALLOC_MAX_H) * NOALLOC_MAX_W * sizeof(float), 256);
// (the allocation-free gradient runs the default shape)
constexpr int NOALLOC_MAX_TILES = ((NOALLOC_MAX_H + SHAPE_TH[DEFAULT_SHAPE] - 1) / SHAPE_TH[DEFAULT_SHAPE]) *
                                  ((NOALLOC_MAX_W + SHAPE_TW[DEFAULT_SHAPE] - 1) / SHAPE_TW[DEFAULT_SHAPE]);
constexpr int NOALLOC_MAX_GROUPS = 128;
constexpr size_t NA_O_IMG = 0;
constexpr size_t NA_O_PART = NA_O_IMG + 7 * NOALLOC_IMG;
constexpr size_t NA_O_GPART = NA_O_PART + na_align(size_t(NOALLOC_MAX_TILES) * NPART * sizeof(float2), 256);
constexpr size_t NA_O_CNT = NA_O_GPART + na_align(size_t(NOALLOC_MAX_GROUPS) * NPART * sizeof(float2), 256);
constexpr size_t NA_O_WORK = NA_O_CNT + 256;
constexpr size_t NA_O_ST = NA_O_WORK + 256;
constexpr size_t NA_O_PROB = NA_O_ST + na_align(sizeof(ScgState), 256);
constexpr size_t NA_O_TMAP = NA_O_PROB + na_align(sizeof(DevProblem), 256);
constexpr size_t NA_O_GLIST = NA_O_TMAP + na_align(size_t(NOALLOC_MAX_TILES) * sizeof(int2), 256);
constexpr size_t NOALLOC_BYTES = NA_O_GLIST + na_align(size_t(NOALLOC_MAX_GROUPS) * sizeof(int2), 256);

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {

struct NoallocDevice {
    bool ready = false;
    unsigned char *base = nullptr;   // device address of g_noalloc_scratch on this device
};
// polls of a tile-load wait before the allocation-free gradient reports it late
std::atomic<uint32_t> g_noalloc_wait_tries{TMA_WAIT_TRIES};
constexpr int NOALLOC_MAX_DEVICES = 64;
NoallocDevice g_noalloc_devices[NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mutex;

// Once per device, with that device current: the device address of the scratch array (the
// host-side symbol is only a stand-in) and the fused pass's shared-memory attributes.
misr_status noalloc_setup(unsigned char **base) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(MISR_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoallocDevice &d = g_noalloc_devices[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(MISR_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
        const misr_status r = set_pass_attrs();
        if (r != MISR_OK) return r;
        d.base = static_cast<unsigned char *>(ptr);
        d.ready = true;
    }
    *base = d.base;
    return MISR_OK;
}

// The problem record of the descriptor with its buffers inside the scratch array.
misr_status noalloc_problem(const misr_desc &d, unsigned char *base, DevProblem &hp) {
    misr_status s = fill_problem(d, 0, DEFAULT_SHAPE, hp);
    if (s != MISR_OK) return s;
    if (hp.general)
        return fail(MISR_ENOTIMPL, "frames that do not interleave into one HR image run the frame-wise pass, whose "
                                   "frame copies and tap tables need a plan's workspace: use misr_gradient");
    hp.wait_tries = (int)std::min<uint32_t>(g_noalloc_wait_tries.load(), 0x7fffffffu);
    for (int i = 0; i < 2; ++i) {
        hp.X[i] = reinterpret_cast<float *>(base + NA_O_IMG + (0 + i) * NOALLOC_IMG);
        hp.Rv[i] = reinterpret_cast<float *>(base + NA_O_IMG + (2 + i) * NOALLOC_IMG);
        hp.Pv[i] = reinterpret_cast<float *>(base + NA_O_IMG + (4 + i) * NOALLOC_IMG);
    }
    hp.Y = reinterpret_cast<float *>(base + NA_O_IMG + 6 * NOALLOC_IMG);
    hp.partials = reinterpret_cast<float2 *>(base + NA_O_PART);
    hp.gpartials = reinterpret_cast<float2 *>(base + NA_O_GPART);
    hp.counter = reinterpret_cast<unsigned int *>(base + NA_O_CNT);
    hp.gcounter = nullptr;   // (the allocation-free call runs the tile shape)
    hp.st = reinterpret_cast<ScgState *>(base + NA_O_ST);
    hp.trace = nullptr;
    return make_maps(hp);
}

}  // namespace

extern "C" misr_status misr_gradient_noalloc(const misr_desc *desc, const void *y_dev, const float *x_dev,
                                             float *g_dev, double *J_out, misr_stream_t stream) {
    if (!y_dev || !x_dev || !g_dev) return fail(MISR_EINVAL, "NULL argument");
    misr_status s = validate(desc);
    if (s != MISR_OK) return s;
    if (desc->iterate_dtype != MISR_F32)
        return fail(MISR_EINVAL, "the allocation-free gradient computes in FP32 only (iterate_dtype MISR_F32)");
    const int H = desc->factor * desc->lr_h, W = desc->factor * desc->lr_w;
    if (H > NOALLOC_MAX_H || W > NOALLOC_MAX_W)
        return fail(MISR_EINVAL, "HR image %d x %d exceeds the allocation-free limit %d x %d", H, W, NOALLOC_MAX_H,
                    NOALLOC_MAX_W);
    unsigned char *base = nullptr;
    s = noalloc_setup(&base);
    if (s != MISR_OK) return s;
    DevProblem hp;
    s = noalloc_problem(*desc, base, hp);
    if (s != MISR_OK) return s;
    std::vector<int2> tiles, groups;   // host lists (no device allocation)
    PassSegs segs;
    build_pass_lists({&hp}, {0}, tiles, groups, segs);
    DevProblem *dprob = reinterpret_cast<DevProblem *>(base + NA_O_PROB);
    int2 *dtile = reinterpret_cast<int2 *>(base + NA_O_TMAP);
    int2 *dgroup = reinterpret_cast<int2 *>(base + NA_O_GLIST);
    unsigned int *work = reinterpret_cast<unsigned int *>(base + NA_O_WORK);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(dprob, &hp, sizeof(DevProblem), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dtile, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dgroup, groups.data(), sizeof(int2) * groups.size(), cudaMemcpyHostToDevice, st));
    // (prepare's state reset zeroes the group counters and the pass counter; the tile counter
    // is zero in a fresh scratch array and zeroed again by every pass)
    const float log_i0 = desc->in_dtype == MISR_U16 ? logf(desc->flat_field) : 0.f;
    const size_t npitched = (size_t)hp.H * hp.pitch, n = (size_t)hp.H * hp.W;
    // x_1 = x (given), r = p_old = 0, state reset; then one pass with alpha = beta = 0
    prepare_kernel<<<grid_for(npitched, 256), 256, 0, st>>>(dprob, 0, y_dev, desc->in_dtype, log_i0, x_dev,
                                                           MISR_X0_GIVEN, 1 | 2 | 4);
    CK(cudaGetLastError());
    s = launch_pass_raw(dprob, dtile, segs, dgroup, hp.n_groups, work, MODE_PROBE, 0.0, 0.0, st);
    if (s != MISR_OK) return s;
    scale_copy_kernel<<<grid_for(n, 256), 256, 0, st>>>(hp.Rv[1], hp.pitch, -1.f, g_dev, hp.H, hp.W);
    CK(cudaGetLastError());
    ScgState hst;
    CK(cudaMemcpyAsync(&hst, hp.st, sizeof(ScgState), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hst.status != DEV_OK) return fail(MISR_ETIMEOUT, "a tile load of the fused pass did not complete in time");
    if (J_out) *J_out = hst.sums[P_JD] + (double)hp.lambda * (hst.sums[P_JB] - hp.eps_pairs);
    return MISR_OK;
}

extern "C" misr_status misr_noalloc_set_wait_limit(uint32_t tries) {
    g_noalloc_wait_tries.store(tries);
    return MISR_OK;
}

extern "C" misr_status misr_autotune(const misr_desc *desc, int32_t passes, int32_t *shape_out, double *ms_out) {
    if (!desc) return fail(MISR_EINVAL, "desc is NULL");
    if (passes < 1 || passes > 1000) return fail(MISR_EINVAL, "passes must be in [1, 1000]");
    misr_status st = check_desc(*desc);
    if (st != MISR_OK) return st;
    {   // non-integer shifts run on the PHASED_SHAPE only: nothing to choose
        DevProblem hp{};
        hp.f = desc->factor;
        misr_desc d = *desc;
        d.tile_shape = MISR_TILE_AUTO;
        if (setup_geometry(d, hp) == MISR_OK && hp.general) {   // one frame-wise pass: nothing to choose
            if (shape_out) *shape_out = MISR_TILE_AUTO;
            if (ms_out)
                for (int sh = 0; sh < N_SHAPES; ++sh) ms_out[sh] = 0.0;
            return MISR_OK;
        }
        if (hp.phased) {
            if (shape_out) *shape_out = PHASED_SHAPE + 1;
            if (ms_out)
                for (int sh = 0; sh < N_SHAPES; ++sh) ms_out[sh] = 0.0;
            return MISR_OK;
        }
    }
    const size_t in_bytes = (size_t)desc->K * desc->lr_h * desc->lr_w * (desc->in_dtype == MISR_U16 ? 2 : 4);
    void *y = nullptr;
    cudaError_t e = cudaMalloc(&y, in_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MISR_ENOMEM, "autotune frames: %s", cudaGetErrorString(e));
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double ms[N_SHAPES] = {};
    int best = DEFAULT_SHAPE;
    const int variant = desc_variant(*desc, false);
    do {
        if ((e = cudaMemset(y, 0, in_bytes)) != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaEventCreate(&e0)) != cudaSuccess) break;
        if ((e = cudaEventCreate(&e1)) != cudaSuccess) break;
        for (int sh = 0; sh < N_SHAPES && st == MISR_OK; ++sh) {
            if (!shape_takes_variant(sh, variant)) continue;   // not compiled for this variant
            misr_desc d = *desc;
            d.tile_shape = sh + 1;
            d.iters = 1;
            d.x0_mode = MISR_X0_ZERO;
            misr_plan_t p = nullptr;
            st = misr_plan_create(&d, &p);
            if (st != MISR_OK) break;
            // passes of the probe mode leave the state alone, so every launch is the same pass
            st = launch_prepare(p, y, nullptr, 1 | 2 | 4, s);
            for (int i = 0; i < 2 && st == MISR_OK; ++i) st = launch_pass(p, MODE_PROBE, 0.5, 0.5, s);
            if (st == MISR_OK && (e = cudaEventRecord(e0, s)) != cudaSuccess) st = fail(MISR_ECUDA, "event");
            for (int i = 0; i < passes && st == MISR_OK; ++i) st = launch_pass(p, MODE_PROBE, 0.5, 0.5, s);
            if (st == MISR_OK && (e = cudaEventRecord(e1, s)) != cudaSuccess) st = fail(MISR_ECUDA, "event");
            if (st == MISR_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) st = fail(MISR_ECUDA, "autotune run failed");
            float t = 0.f;
            if (st == MISR_OK) cudaEventElapsedTime(&t, e0, e1);
            ms[sh] = (double)t / passes;
            misr_plan_destroy(p);
        }
        if (st != MISR_OK) break;
        for (int sh = 0; sh < N_SHAPES; ++sh)
            if (ms[sh] > 0 && ms[sh] < ms[best]) best = sh;
    } while (0);
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (s) cudaStreamDestroy(s);
    cudaFree(y);
    if (st != MISR_OK) return st;
    if (e != cudaSuccess) return fail(MISR_ECUDA, "autotune: %s", cudaGetErrorString(e));
    {
        const int H = desc->factor * desc->lr_h, W = desc->factor * desc->lr_w;
        std::array<double, N_SHAPES> t{};
        for (int sh = 0; sh < N_SHAPES; ++sh) t[sh] = ms[sh];
        std::lock_guard<std::mutex> lock(g_tuned_mu);
        bool found = false;
        for (auto &en : g_tuned)
            if (en.first.first == H && en.first.second == W) {
                for (int sh = 0; sh < N_SHAPES; ++sh)
                    if (t[sh] > 0) en.second[sh] = t[sh];
                found = true;
            }
        if (!found) g_tuned.push_back({{H, W}, t});
    }
    if (shape_out) *shape_out = best + 1;
    if (ms_out)
        for (int sh = 0; sh < N_SHAPES; ++sh) ms_out[sh] = ms[sh];
    return MISR_OK;
}
