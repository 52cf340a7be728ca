// The fused SCG pass as a row-streaming kernel (sm_103a): one warp per work item, its row
// windows in registers, no block barriers.  Included by misr_device.cuh; it runs the shared-tap
// problems (integer shifts, point or binned D) with the squared L2 or the smoothed L1 data term.
//
// What one pass computes is the tile kernel's (Algorithm 1's loop body with Moller's curvature
// taken at the trial point): p = r + beta p_old, x' = x + alpha p, the residual of the
// interleaved frames E = B x' - Y (Eq. 1), r' = -(2 B^T E + lambda grad BTV(x')) (Eq. 6, 8, 9),
// and the ten sums of the pass (J_data(x'), J_data(x') - J_data(x), BTV(x'), |r'|^2, r'.r,
// p.r', |p|^2, r'.H r', r'.H p, p.H p).
//
// Work item: a strip of SW_OWN = 112 HR columns by `tile_h` rows.  Each lane holds 4
// consecutive columns of a 128-column window that starts SW_HALO = 8 columns left of the strip;
// the warp walks down the rows of its item, one row per step, from 6 rows above it to 5 below.
// Step n takes the input row n and advances every stage by one row:
//     x'(n), p(n)                         loads of row n
//     z = B x', B p     rows n-2 done     separable: horizontal blur of row n, then its five
//                                         vertical taps added into five pending rows
//     E(n-2) = z - Y, J_data, dJ_data, c (data part)
//     2 B^T E           row n-4 done      the adjoint the same way, from E(n-2)
//     BTV pairs of row n-4                each pair (q, q + d) once: psi' into both ends of the
//                                         gradient, psi'' kept for the curvature forms
//     r'(n-4), |r'|^2, r'.r, p.r'
//     B r'              row n-6 done      a, b (data part)
//     curvature of the BTV pairs of rows n-4 (d_y = 0), n-5 (d_y = 1), n-6 (d_y = 2)
// A stage's horizontal neighbours come from the neighbouring lanes by shuffles; the window's
// outer 8 columns on each side are computed but not owned (their values degrade inward by two
// columns per stage), so no warp depends on another.  Every register row window is a 5-slot
// array; at every step row n + off sits at slot off mod 5, and the windows move down one slot at
// the end of the step (register moves).  The loop body is one step: an unrolled body kept
// several copies of the step hot and overflowed the instruction cache.
//
// The image border is handled by the data, on the same code as the interior:
//   - outside the image x, r, p_old read as 0 (rows and lanes outside the row pitch are
//     zero-filled by the copies; the pitch's pad columns hold zeros) and Y as NaN ("no sample":
//     the pads hold NaN, the rest is written so), which is B's zero padding and the data mask;
//   - r' is set to 0 outside the image;
//   - the BTV's copy of x' holds SW_BIG outside the image: a pair with one end outside then has
//     t^2 = +inf, rsqrt = 0, and its psi', psi'' and value t psi' + eps^2 rsqrt are exactly 0,
//     which drops it as the prior's definition does (only pairs inside the image count).
// The frame masks (B's zero padding in front of the shift M_k, within f + R pixels of the top
// and left edges) are subtracted again from the blurs in correction blocks.  Those are compiled
// into the edge path only: the items that meet those edges run on the launch's first CTAs with
// that path, the rest on the others with a path without them (EDGE).  With one CTA per SM, an
// SM keeps one path in its instruction cache; present but unused, the blocks had cost the
// interior 20%.
//
// The pass's sums are reduced in the pass when its launch is the step's only one
// (stream_reduce), else by reduce_kernel after it.
#pragma once

namespace misr {

constexpr int SW_LANES = 32;
constexpr int SW_WIN = 4 * SW_LANES;   // window columns of a warp
constexpr int SW_HALO = 8;             // window columns left (and right) of the owned strip
constexpr int SW_OWN = SW_WIN - 2 * SW_HALO;
constexpr int SW_NT = 256;             // threads per CTA (8 independent warps)
constexpr int SW_U = 5;                // row-window slots
constexpr unsigned FULL = 0xffffffffu;
constexpr float SW_BIG = 1e20f;        // the BTV's x' outside the image ((SW_BIG - x)^2 = +inf)

// slot of row (n + off) when step n has slot k (compile time)
template <int K, int OFF>
struct Slot {
    static constexpr int v = ((K + OFF) % SW_U + SW_U) % SW_U;
};

// The per-lane state carried from step to step (register arrays with compile-time indices).
// Row windows:
//   xw[s][0..5]   the BTV's x' of a row: the lane's 4 columns and 2 of the next lane (rows n-4..n)
//   za[s], bpa[s] pending forward blurs of x' and p (rows n-2..n+2)
//   ga[s]         pending adjoint 2 B^T E (rows n-4..n)
//   gr[s][0..5]   pending BTV gradient, 2 columns of the next lane at [4], [5] (rows n-4..n-2)
//   bra[s]        pending B r' (rows n-6..n-2)
//   rw[s], pw[s]  r' and p with 2 columns of the next lane (rows n-6..n-4)
// Kept in the warp's shared-memory ring instead (written once, read once a few steps later,
// each lane its own 16-byte slots): the psi'' weights of the pairs with d_y = 1 and 2 of a row,
// until r' of the row d_y below exists, and the completed (masked) B p rows, for the data part
// of b four steps later.
struct StreamState {
    float xw[SW_U][6];
    float za[SW_U][4], bpa[SW_U][4], ga[SW_U][4], bra[SW_U][4];
    float gr[SW_U][6];
    float rw[SW_U][6], pw[SW_U][6];
    unsigned mbits;           // sample bits of rows n-6..n-2 (4 bits a row, newest lowest)
    // the lane's 16 bytes in the warp's shared-memory area (stages, then ring), and the byte
    // offsets of the current step's input stage and of the next step's, in flight
    unsigned char *wb;
    uint32_t cur, nxt;
    uint32_t w1o, w2o;        // this step's w1 and w2 slots (byte offsets)
    uint32_t bpo;             // the bpw slot of row n-2 (byte offset; row n-6's is the next one)
    // sums of the item (per lane); the prior's value, r.r', r'.r' and p.r' carry a
    // compensation term (two-sum) because Moller's comparison and beta take differences of them
    float s[NPART];
    float lo_jb, lo_rr, lo_rrx, lo_pr;
};

__device__ __forceinline__ void fast2sum_acc(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

// Item geometry of the lane.
struct SegGeo {
    int H, W, pitch;
    int y0, ye;          // owned rows [y0, ye)
    int v0;              // image column of the lane's first column
    bool own_lane;       // the lane's 4 columns belong to the owned strip (window cols 8..119)
    bool lane_in;        // the lane's 4 columns lie inside [0, pitch) (whole groups: v0, pitch % 4)
    bool all_in;         // all 4 inside [0, W)
    bool in0, in1, in2, in3;   // column v0 + j inside [0, W)
    bool left;           // the window meets the frame masks of the left edge
    __device__ __forceinline__ bool in(int j) const { return j == 0 ? in0 : j == 1 ? in1 : j == 2 ? in2 : in3; }
};

// Input rows of a step, staged in shared memory by cp.async one step ahead: per warp two stages
// of SW_ROWS rows of 128 floats (bf16 rows use the first 8 bytes of each lane's 16), each lane
// copying and reading only its own 16 bytes, so no warp synchronisation is needed.  Rows of
// step n: x(n), r(n), p_old(n), Y(n-2).
constexpr int SW_ROWS = 4;
constexpr uint32_t SW_ROW_BYTES = 4 * SW_WIN;
constexpr uint32_t SW_STAGE_BYTES = SW_ROWS * SW_ROW_BYTES;
enum { LR_X = 0, LR_R, LR_PO, LR_Y };
// the ring, per warp after its two stages: w1[slot][dx] (2 slots), w2[slot][dx] (3 slots),
// bpw[slot] (5 slots) and, for the L1 data term, wd[slot] (5 slots), each a row of 32 lanes x
// 16 bytes.  The slots rotate by step: w1 is read one step after it is written, w2 two steps
// after, bpw and wd four.  bpw holds the masked B p of a row (times psi_d''(e') with the L1
// term), wd the row's psi_d''(e') (0 where unsampled).  pr and rr (5 slots each) hold p(n) and
// r(n) of a row (as the pass uses them: rounded to bf16 when r and p are stored so), for the
// r' stage four steps on.
constexpr uint32_t SW_W_SLOT = 3 * SW_ROW_BYTES;
constexpr uint32_t SW_RING_W1 = 0, SW_RING_W2 = 2 * SW_W_SLOT, SW_RING_BP = 5 * SW_W_SLOT;
constexpr uint32_t SW_RING_WD = SW_RING_BP + SW_U * SW_ROW_BYTES;
constexpr uint32_t SW_RING_PR = SW_RING_WD + SW_U * SW_ROW_BYTES;
constexpr uint32_t SW_RING_RR = SW_RING_PR + SW_U * SW_ROW_BYTES;
constexpr uint32_t SW_RING_BYTES = SW_RING_RR + SW_U * SW_ROW_BYTES;
constexpr uint32_t SW_WARP_BYTES = 2 * SW_STAGE_BYTES + SW_RING_BYTES;
constexpr size_t SW_SMEM_BYTES = (size_t)(SW_NT / 32) * SW_WARP_BYTES;

constexpr uint32_t SW_RING = 2 * SW_STAGE_BYTES;   // the ring's offset in the warp's area
// the lane's 16 bytes at byte offset `o` of its warp's area (plain shared-memory accesses: the
// compiler orders them and may schedule them early)
__device__ __forceinline__ void sts4(unsigned char *wb, uint32_t o, const float *v) {
    *reinterpret_cast<float4 *>(wb + o) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void lds4(const unsigned char *wb, uint32_t o, float *v) {
    const float4 a = *reinterpret_cast<const float4 *>(wb + o);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

__device__ __forceinline__ void cp_async_n(uint32_t dst, const void *src, int bytes, uint32_t src_bytes) {
    if (bytes == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

// Copy the lane's 4 elements (float, or bf16 when BF) of row `row` into its slot at `dst`; a
// row outside the image or a lane outside the row pitch arrives as zeros (src-size 0, the
// address that of the image's first element), or as NaN for Y (NANF).
template <bool BF, bool NANF>
__device__ __forceinline__ void issue_row(const void *img, const SegGeo &g, int row, unsigned char *wb, uint32_t o) {
    const bool ok = row >= 0 && row < g.H && g.lane_in;
    if (NANF && !ok) {
        const float nan = __int_as_float(0x7fc00000);
        const float v[4] = {nan, nan, nan, nan};
        sts4(wb, o, v);
        return;
    }
    const size_t esz = BF ? 2 : 4;
    const char *src = static_cast<const char *>(img) + (ok ? ((size_t)row * g.pitch + g.v0) * esz : 0);
    cp_async_n(smem_addr(wb + o), src, BF ? 8 : 16, ok ? (BF ? 8u : 16u) : 0u);
}

template <bool RPB>
__device__ __forceinline__ void issue_step_rows(const SegGeo &g, unsigned char *wb, uint32_t o, int n, const float *X,
                                                const float *R, const float *PO, const float *Y) {
    issue_row<false, false>(X, g, n, wb, o + LR_X * SW_ROW_BYTES);
    issue_row<RPB, false>(R, g, n, wb, o + LR_R * SW_ROW_BYTES);
    issue_row<RPB, false>(PO, g, n, wb, o + LR_PO * SW_ROW_BYTES);
    issue_row<false, true>(Y, g, n - 2, wb, o + LR_Y * SW_ROW_BYTES);
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// The lane's 4 values of a staged row (byte offset o of its warp's area) as floats.
template <bool BF>
__device__ __forceinline__ void read_row4(const unsigned char *wb, uint32_t o, float *v) {
    if (BF) {
        const uint2 u = *reinterpret_cast<const uint2 *>(wb + o);
        v[0] = __uint_as_float(u.x << 16); v[1] = __uint_as_float(u.x & 0xffff0000u);
        v[2] = __uint_as_float(u.y << 16); v[3] = __uint_as_float(u.y & 0xffff0000u);
    } else {
        lds4(wb, o, v);
    }
}

// the lane's row vector with two columns of each neighbouring lane: e[0..7] = cols -2..5
__device__ __forceinline__ void with_ext(const float *v, float *e) {
    e[0] = __shfl_up_sync(FULL, v[2], 1);
    e[1] = __shfl_up_sync(FULL, v[3], 1);
    e[2] = v[0]; e[3] = v[1]; e[4] = v[2]; e[5] = v[3];
    e[6] = __shfl_down_sync(FULL, v[0], 1);
    e[7] = __shfl_down_sync(FULL, v[1], 1);
}

// Horizontal forward blur: out(v) = sum_b hx(b) e(v - b).  At the left edge the frame masks
// drop tap b of output v when b > fwd_lim(v): those taps are taken out again (an item whose
// window meets the edge enters that block; the rest skip it).  EDGE: compiled with the
// border corrections (the interior path leaves them out).
template <bool EDGE>
__device__ __forceinline__ void hblur_fwd(const StreamConsts &k, const SegGeo &g, const float *e, float *out) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float s = 0.f;
#pragma unroll
        for (int b = -2; b <= 2; ++b) s = fmaf(k.hx[b + 2], e[2 + j - b], s);
        out[j] = s;
    }
    if (EDGE && g.left) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int lim = fwd_lim(g.v0 + j, k.f, k.fmag);
#pragma unroll
            for (int b = -1; b <= 2; ++b)
                if (b > lim) out[j] = fmaf(-k.hx[b + 2], e[2 + j - b], out[j]);
        }
    }
}
// Horizontal adjoint blur: out(u) = sum_b hx(b) e(u + b); at the left edge the adjoint's frame
// masks (tap b dropped when !adj_tap_ok(u, b)) are taken out again.
template <bool EDGE>
__device__ __forceinline__ void hblur_adj(const StreamConsts &k, const SegGeo &g, const float *e, float *out) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float s = 0.f;
#pragma unroll
        for (int b = -2; b <= 2; ++b) s = fmaf(k.hx[b + 2], e[2 + j + b], s);
        out[j] = s;
    }
    if (EDGE && g.left) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int u = g.v0 + j;
#pragma unroll
            for (int b = -2; b <= 2; ++b)
                if (!adj_tap_ok(u, b, k.f, k.fmag)) out[j] = fmaf(-k.hx[b + 2], e[2 + j + b], out[j]);
        }
    }
}

// Vertical forward scatter of the horizontally blurred row `row` (values h, the row's slot
// K + OFF) into the pending rows row + a, a = -2..2.  Near the top edge (rows below
// 2 MAXF + 2) tap a of output row row + a is dropped when a > fwd_lim(row + a); it is taken out
// again there.
template <int K, int OFF, bool EDGE>
__device__ __forceinline__ void vscatter_fwd(const StreamConsts &k, float (*acc)[4], const float *h, int row) {
#pragma unroll
    for (int a = -2; a <= 2; ++a) {
        float *z = acc[((K + OFF + a) % SW_U + SW_U) % SW_U];
#pragma unroll
        for (int j = 0; j < 4; ++j) z[j] = fmaf(k.hy[a + 2], h[j], z[j]);
    }
    if (EDGE && row < 2 * MAXF + 2) {
#pragma unroll
        for (int a = -1; a <= 2; ++a) {
            if (a > fwd_lim(row + a, k.f, k.fmag)) {
                float *z = acc[((K + OFF + a) % SW_U + SW_U) % SW_U];
#pragma unroll
                for (int j = 0; j < 4; ++j) z[j] = fmaf(-k.hy[a + 2], h[j], z[j]);
            }
        }
    }
}

template <int NV>
__device__ __forceinline__ void rotate_rows(float (*w)[NV]) {
    float t[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) t[j] = w[0][j];
#pragma unroll
    for (int s = 0; s + 1 < SW_U; ++s)
#pragma unroll
        for (int j = 0; j < NV; ++j) w[s][j] = w[s + 1][j];
#pragma unroll
    for (int j = 0; j < NV; ++j) w[SW_U - 1][j] = t[j];
}

// One step of the item: input row n.  Row n + off sits at slot off mod 5 of every register
// window (K = 0; the windows are rotated at the end of the step).  RPB: r and p stored as bf16.
// EDGE: the path with the frame-mask corrections of the top and left borders (any item);
// without it, only items whose rows start at 24 or below and whose strip is not the first.
// L1: the smoothed L1 data term psi_d(e) = sqrt(e^2 + eps_d^2) - eps_d instead of e^2.
template <int K, bool RPB, bool EDGE, bool L1>
__device__ __forceinline__ void stream_step(StreamState &S, const StreamConsts &k, const SegGeo &g, int n,
                                            float alpha, float beta, const float *__restrict__ X,
                                            const float *__restrict__ R, const float *__restrict__ PO,
                                            const float *__restrict__ Y, float *__restrict__ Xn,
                                            float *__restrict__ Rn, float *__restrict__ Pn) {
    constexpr int sN = Slot<K, 0>::v, sN2 = Slot<K, -2>::v, sN4 = Slot<K, -4>::v, sN5 = Slot<K, -5>::v;
    constexpr int sN6 = Slot<K, -6>::v;
    const int lane = threadIdx.x & 31;
    const int H = g.H;

    // ---- this step's rows have landed (the lane's own copies); the next step's go out now into
    // the other stage, whose rows the previous step has read
    asm volatile("cp.async.wait_all;" ::: "memory");
    issue_step_rows<RPB>(g, S.wb, S.nxt, n + 1, X, R, PO, Y);

    // ---- row n: p, x'
    float p[4], xp[4];
    {
        float cx[4], cr[4], cpo[4];
        read_row4<false>(S.wb, S.cur + LR_X * SW_ROW_BYTES, cx);
        read_row4<RPB>(S.wb, S.cur + LR_R * SW_ROW_BYTES, cr);
        read_row4<RPB>(S.wb, S.cur + LR_PO * SW_ROW_BYTES, cpo);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            p[j] = fmaf(beta, cpo[j], cr[j]);
            if (RPB) p[j] = __bfloat162float(__float2bfloat16_rn(p[j]));
            xp[j] = fmaf(alpha, p[j], cx[j]);
        }
        // p(n) and r(n) for the r' stage of row n four steps on: row n's slot is two after row
        // n-2's (bpo)
        uint32_t o = S.bpo + 2 * SW_ROW_BYTES;
        if (o >= SW_U * SW_ROW_BYTES) o -= SW_U * SW_ROW_BYTES;
        sts4(S.wb, SW_RING + SW_RING_PR + o, p);
        sts4(S.wb, SW_RING + SW_RING_RR + o, cr);
    }
    const bool row_n_in = n >= 0 && n < H;
    if (n >= g.y0 && n < g.ye) {
        float pp = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) pp = fmaf(p[j], p[j], pp);   // p = 0 outside the image
        S.s[P_PP] += pp;
        if (g.own_lane) {
            const size_t o = (size_t)n * g.pitch + g.v0;
            if (g.all_in) {
                st4(Xn + o, make_float4(xp[0], xp[1], xp[2], xp[3]));
                if (RPB) st_bf4(reinterpret_cast<__nv_bfloat16 *>(Pn) + o, make_float4(p[0], p[1], p[2], p[3]));
                else st4(Pn + o, make_float4(p[0], p[1], p[2], p[3]));
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (g.in(j) && MISR_IN_BOUNDS(g.v0 + j < g.W, BC_A_STORE, n, g.v0 + j)) {
                        Xn[o + j] = xp[j];
                        if (RPB) reinterpret_cast<__nv_bfloat16 *>(Pn)[o + j] = __float2bfloat16_rn(p[j]);
                        else Pn[o + j] = p[j];
                    }
            }
        }
    }

    // ---- forward blurs of x'(n) and p(n): horizontal, then into the pending rows n-2 .. n+2;
    // the BTV's copy of x'(n), SW_BIG outside the image
    {
        float e[8], h[4];
        with_ext(xp, e);
        hblur_fwd<EDGE>(k, g, e, h);
        vscatter_fwd<K, 0, EDGE>(k, S.za, h, n);
#pragma unroll
        for (int j = 0; j < 4; ++j) S.xw[sN][j] = (row_n_in && g.in(j)) ? xp[j] : SW_BIG;
        S.xw[sN][4] = __shfl_down_sync(FULL, S.xw[sN][0], 1);
        S.xw[sN][5] = __shfl_down_sync(FULL, S.xw[sN][1], 1);
        with_ext(p, e);
        hblur_fwd<EDGE>(k, g, e, h);
        vscatter_fwd<K, 0, EDGE>(k, S.bpa, h, n);
    }

    // ---- row n-2: residual, J_data, dJ_data and the data part of c; then its adjoint.  With
    // the L1 term the adjoint takes psi_d'(e) = e / S(e), S(t) = sqrt(t^2 + eps_d^2), the sums
    // weigh by psi_d''(e) = eps_d^2 / S(e)^3, J_data sums psi_d(e) = e^2 / (S(e) + eps_d) and
    // J_data(x') - J_data(x) sums (e'^2 - e^2) / (S(e') + S(e)), so that no term cancels
    constexpr float DS = L1 ? 1.f : 2.f;   // d/de of the data term's e^2 (L2) or psi_d(e) (L1)
    {
        const int m = n - 2;
        float cy[4], E[4], bpm[4], wdm[4];
        read_row4<false>(S.wb, S.cur + LR_Y * SW_ROW_BYTES, cy);
        unsigned bits = 0;
        float jd = 0.f, dj = 0.f, cd = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool smp = !isnan(cy[j]);
            E[j] = smp ? S.za[sN2][j] - cy[j] : 0.f;
            const float bp = smp ? S.bpa[sN2][j] : 0.f;
            bits |= (smp ? 1u : 0u) << j;
            const float abp = alpha * bp;
            // e'^2 - e^2 = alpha (B p) (2 e' - alpha (B p)), e the residual at x = x' - alpha p
            if constexpr (L1) {
                const float de2 = abp * fmaf(2.f, E[j], -abp);
                const float q1 = fmaf(E[j], E[j], k.deps2), r1 = rsqrt_ftz(q1);
                const float eb = E[j] - abp;
                const float q0 = fmaf(eb, eb, k.deps2), r0 = rsqrt_ftz(q0);
                jd += __fdividef(E[j] * E[j], fmaf(q1, r1, k.deps));
                dj += __fdividef(de2, fmaf(q1, r1, q0 * r0));
                const float er = k.deps * r1;
                const float w = smp ? r1 * (er * er) : 0.f;   // psi_d''(e'), as (1/S) (eps_d/S)^2
                const float wbp = w * bp;
                cd = fmaf(wbp, bp, cd);
                bpm[j] = wbp;
                wdm[j] = w;
                E[j] *= r1;
            } else {
                bpm[j] = bp;                       // masked B p, for b at row n-2 four steps on
                jd = fmaf(E[j], E[j], jd);
                dj = fmaf(abp, fmaf(2.f, E[j], -abp), dj);
                cd = fmaf(bp, bp, cd);
            }
            S.za[sN2][j] = 0.f;
            S.bpa[sN2][j] = 0.f;
        }
        S.mbits = (S.mbits << 4) | bits;
        sts4(S.wb, SW_RING + SW_RING_BP + S.bpo, bpm);
        if constexpr (L1) sts4(S.wb, SW_RING + SW_RING_WD + S.bpo, wdm);
        if (m >= g.y0 && m < g.ye) {
            S.s[P_JD] += jd;
            S.s[P_DJD] += dj;
            S.s[P_C] = fmaf(DS, cd, S.s[P_C]);
        }
        float e[8], h[4];
        with_ext(E, e);
        hblur_adj<EDGE>(k, g, e, h);
#pragma unroll
        for (int a = -2; a <= 2; ++a) {
            // tap a of output row m - a reads sample row m
            float *ga = S.ga[((K - 2 - a) % SW_U + SW_U) % SW_U];
#pragma unroll
            for (int j = 0; j < 4; ++j) ga[j] = fmaf(DS * k.hy[a + 2], h[j], ga[j]);
        }
        if (EDGE && m < 2 * MAXF) {   // the adjoint's frame masks near the top: dropped when !adj_tap_ok(m - a, a)
#pragma unroll
            for (int a = -2; a <= 2; ++a)
                if (!adj_tap_ok(m - a, a, k.f, k.fmag)) {
                    float *ga = S.ga[((K - 2 - a) % SW_U + SW_U) % SW_U];
#pragma unroll
                    for (int j = 0; j < 4; ++j) ga[j] = fmaf(-DS * k.hy[a + 2], h[j], ga[j]);
                }
        }
    }

    // ---- BTV pairs (q, q + d) of row m = n-4: gradient at both ends, the prior's value over
    // owned q, the psi'' weights.  A pair with an end outside the image (its x' SW_BIG) has
    // rsqrt(t^2 + eps^2) = 0 and adds exactly nothing.
    const int m = n - 4;
    const bool own_m = m >= g.y0 && m < g.ye;
    float w0[2][4];   // weights of the d_y = 0 pairs (used below, this step)
    {
        float jbj[4] = {0.f, 0.f, 0.f, 0.f};   // per column, so that columns outside drop out
#pragma unroll
        for (int dy = 0; dy <= 2; ++dy) {
            constexpr int sq = Slot<K, -4>::v;
            const int sd = ((K - 4 + dy) % SW_U + SW_U) % SW_U;
#pragma unroll
            for (int dx = 0; dx <= 2; ++dx) {
                if (dx == 0 && dy == 0) continue;
                const float gam = k.gam[dy * 3 + dx], lgam = k.lgam[dy * 3 + dx];   // gamma, lambda gamma
                float wv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float t = S.xw[sq][j] - S.xw[sd][j + dx];
                    const float s2 = fmaf(t, t, k.eps2);
                    const float rs = rsqrt_ftz(s2);
                    const float tr = t * rs;                 // psi'(t)
                    const float gp = gam * tr;
                    S.gr[sq][j] += gp;
                    S.gr[sd][j + dx] -= gp;
                    const float e2rs = k.eps2 * rs;
                    jbj[j] = fmaf(gam, fmaf(t, tr, e2rs), jbj[j]);   // gamma sqrt(t^2 + eps^2)
                    const float w = (lgam * e2rs) * (rs * rs);         // lambda gamma psi''(t)
                    if (dy == 0) w0[dx - 1][j] = w;
                    else wv[j] = w;
                }
                if (dy == 1) sts4(S.wb, SW_RING + SW_RING_W1 + S.w1o + dx * SW_ROW_BYTES, wv);
                if (dy == 2) sts4(S.wb, SW_RING + SW_RING_W2 + S.w2o + dx * SW_ROW_BYTES, wv);
            }
        }
        // the next lane's share of row m's gradient (its columns 0, 1) is complete
        const float e0 = __shfl_up_sync(FULL, S.gr[sN4][4], 1), e1 = __shfl_up_sync(FULL, S.gr[sN4][5], 1);
        if (lane > 0) { S.gr[sN4][0] += e0; S.gr[sN4][1] += e1; }
        if (own_m) {
            float jb = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) jb += g.in(j) ? jbj[j] : 0.f;
            fast2sum_acc(S.s[P_JB], S.lo_jb, jb);
        }
    }

    // ---- r'(m) = -(2 B^T E + lambda grad BTV), zero outside the image; its sums and store
    float rv[4], p4[4], cr4[4];
    {
        const bool row_in = m >= 0 && m < H;
        {   // p and r of row m = n-4 as step m stored them (row m's slot: three after bpo)
            uint32_t o = S.bpo + 3 * SW_ROW_BYTES;
            if (o >= SW_U * SW_ROW_BYTES) o -= SW_U * SW_ROW_BYTES;
            lds4(S.wb, SW_RING + SW_RING_PR + o, p4);
            lds4(S.wb, SW_RING + SW_RING_RR + o, cr4);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float r = -fmaf(k.lambda, S.gr[sN4][j], S.ga[sN4][j]);
            if (!(row_in && g.in(j))) r = 0.f;
            if (RPB) r = __bfloat162float(__float2bfloat16_rn(r));
            rv[j] = r;
            S.ga[sN4][j] = 0.f;
        }
#pragma unroll
        for (int j = 0; j < 6; ++j) S.gr[sN4][j] = 0.f;
        if (own_m) {
            float rr = 0.f, rrx = 0.f, pr = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                rr = fmaf(rv[j], rv[j], rr);
                rrx = fmaf(rv[j], cr4[j], rrx);
                pr = fmaf(p4[j], rv[j], pr);
            }
            if (g.own_lane) {
                const size_t o = (size_t)m * g.pitch + g.v0;
                if (g.all_in) {
                    if (RPB) st_bf4(reinterpret_cast<__nv_bfloat16 *>(Rn) + o, make_float4(rv[0], rv[1], rv[2], rv[3]));
                    else st4(Rn + o, make_float4(rv[0], rv[1], rv[2], rv[3]));
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (g.in(j) && MISR_IN_BOUNDS(g.v0 + j < g.W, BC_C2_STORE, m, g.v0 + j)) {
                            if (RPB) reinterpret_cast<__nv_bfloat16 *>(Rn)[o + j] = __float2bfloat16_rn(rv[j]);
                            else Rn[o + j] = rv[j];
                        }
                }
            }
            fast2sum_acc(S.s[P_RR], S.lo_rr, rr);
            fast2sum_acc(S.s[P_RRX], S.lo_rrx, rrx);
            fast2sum_acc(S.s[P_PR], S.lo_pr, pr);
        }
    }

    // ---- B r'(m): horizontal, into the pending rows m-2 .. m+2; row n-6 done: a, b (data)
    {
        float e[8], h[4];
        with_ext(rv, e);
#pragma unroll
        for (int j = 0; j < 4; ++j) S.rw[sN4][j] = rv[j];
        S.rw[sN4][4] = e[6];
        S.rw[sN4][5] = e[7];
        hblur_fwd<EDGE>(k, g, e, h);
        vscatter_fwd<K, -4, EDGE>(k, S.bra, h, m);
        // p(m) with the next lane's two columns, for the BTV curvature
#pragma unroll
        for (int j = 0; j < 4; ++j) S.pw[sN4][j] = p4[j];
        S.pw[sN4][4] = __shfl_down_sync(FULL, p4[0], 1);
        S.pw[sN4][5] = __shfl_down_sync(FULL, p4[1], 1);

        const int m6 = n - 6;
        const unsigned b6 = (S.mbits >> 16) & 0xfu;   // rows n-6 .. n-2 sit at bits 16 .. 0
        float ad = 0.f, bd = 0.f, bp6[4], wd6[4];
        // row n-6's slot: written four steps ago, the one after this step's (mod 5)
        const uint32_t o6 = S.bpo == 4 * SW_ROW_BYTES ? 0 : S.bpo + SW_ROW_BYTES;
        lds4(S.wb, SW_RING + SW_RING_BP + o6, bp6);
        if constexpr (L1) lds4(S.wb, SW_RING + SW_RING_WD + o6, wd6);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float br = ((b6 >> j) & 1u) ? S.bra[sN6][j] : 0.f;
            ad = L1 ? fmaf(br * wd6[j], br, ad) : fmaf(br, br, ad);
            bd = fmaf(br, bp6[j], bd);
            S.bra[sN6][j] = 0.f;
        }
        if (m6 >= g.y0 && m6 < g.ye) {
            S.s[P_A] = fmaf(DS, ad, S.s[P_A]);
            S.s[P_B] = fmaf(DS, bd, S.s[P_B]);
        }
    }

    // ---- BTV curvature: lambda sum gamma psi''(t) (dv)(dw) over the pairs of rows n-4
    // (d_y = 0), n-5 (d_y = 1) and n-6 (d_y = 2), whose r' rows now all exist (r' and p are 0
    // outside the image, so a pair with both ends outside adds nothing)
    {
        float ca = 0.f, cb = 0.f, cc = 0.f;
        auto pair_terms = [&](const float *rq, const float *pq, const float *rd, const float *pd, const float *w,
                              int dx) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float dr = rq[j] - rd[j + dx], dp = pq[j] - pd[j + dx];
                const float wr = w[j] * dr, wp = w[j] * dp;
                ca = fmaf(wr, dr, ca);
                cb = fmaf(wr, dp, cb);
                cc = fmaf(wp, dp, cc);
            }
        };
        if (own_m) {
            pair_terms(S.rw[sN4], S.pw[sN4], S.rw[sN4], S.pw[sN4], w0[0], 1);
            pair_terms(S.rw[sN4], S.pw[sN4], S.rw[sN4], S.pw[sN4], w0[1], 2);
        }
        if (n - 5 >= g.y0 && n - 5 < g.ye) {
#pragma unroll
            for (int dx = 0; dx <= 2; ++dx) {
                float w[4];
                lds4(S.wb, SW_RING + SW_RING_W1 + (S.w1o ^ SW_W_SLOT) + dx * SW_ROW_BYTES, w);   // written last step
                pair_terms(S.rw[sN5], S.pw[sN5], S.rw[sN4], S.pw[sN4], w, dx);
            }
        }
        if (n - 6 >= g.y0 && n - 6 < g.ye) {
#pragma unroll
            for (int dx = 0; dx <= 2; ++dx) {
                float w[4];
                // written two steps ago: the slot after this step's
                lds4(S.wb, SW_RING + SW_RING_W2 + (S.w2o == 2 * SW_W_SLOT ? 0 : S.w2o + SW_W_SLOT) + dx * SW_ROW_BYTES, w);
                pair_terms(S.rw[sN6], S.pw[sN6], S.rw[sN4], S.pw[sN4], w, dx);
            }
        }
        S.s[P_A] += ca;
        S.s[P_B] += cb;
        S.s[P_C] += cc;
    }

    // ---- the stage issued above becomes the current one; the weight slots rotate
    const uint32_t t = S.cur;
    S.cur = S.nxt;
    S.nxt = t;
    S.w1o ^= SW_W_SLOT;
    S.w2o = S.w2o == 2 * SW_W_SLOT ? 0 : S.w2o + SW_W_SLOT;
    S.bpo = S.bpo == 4 * SW_ROW_BYTES ? 0 : S.bpo + SW_ROW_BYTES;
    // the register windows move down one row: slot s takes slot s + 1 (mod 5), so that the
    // next step finds row (n + 1) + off at slot off mod 5 (moves of dead slots are dropped)
    rotate_rows(S.xw);
    rotate_rows(S.za);
    rotate_rows(S.bpa);
    rotate_rows(S.ga);
    rotate_rows(S.bra);
    rotate_rows(S.gr);
    rotate_rows(S.rw);
    rotate_rows(S.pw);
}

// One item: steps n = y0 - 6 .. ye + 5.
template <bool RPB, bool EDGE, bool L1>
__device__ __forceinline__ void stream_item(StreamState &S, const StreamConsts &k, const SegGeo &g, float alpha,
                                            float beta, const float *__restrict__ X, const float *__restrict__ R,
                                            const float *__restrict__ PO, const float *__restrict__ Y,
                                            float *__restrict__ Xn, float *__restrict__ Rn, float *__restrict__ Pn) {
    // every window starts at zero (rows above the first are never owned)
#pragma unroll
    for (int s = 0; s < SW_U; ++s) {
#pragma unroll
        for (int j = 0; j < 6; ++j) { S.xw[s][j] = 0.f; S.gr[s][j] = 0.f; S.rw[s][j] = 0.f; S.pw[s][j] = 0.f; }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            S.za[s][j] = 0.f; S.bpa[s][j] = 0.f; S.ga[s][j] = 0.f; S.bra[s][j] = 0.f;
        }
    }
    {   // the ring starts at zero too (read before written on the item's first steps)
        const float z[4] = {0.f, 0.f, 0.f, 0.f};
        for (uint32_t o = 0; o < SW_RING_BYTES; o += SW_ROW_BYTES) sts4(S.wb, SW_RING + o, z);
    }
    S.mbits = 0;
    S.w1o = 0;
    S.w2o = 0;
    S.bpo = 0;
    const int n0 = g.y0 - 6;
    // the previous item's last (unused) stage is drained before its slots are written again
    asm volatile("cp.async.wait_all;" ::: "memory");
    // the first step's rows
    issue_step_rows<RPB>(g, S.wb, S.cur, n0, X, R, PO, Y);
    const int n_end = g.ye + 6;   // one past the last step
#pragma unroll 1
    for (int n = n0; n < n_end; ++n) stream_step<0, RPB, EDGE, L1>(S, k, g, n, alpha, beta, X, R, PO, Y, Xn, Rn, Pn);
}

// Geometry of item t of problem P (the item order of the problem record: the left strip's
// items, the top items of the other strips, then their remaining rows).
__device__ __forceinline__ void stream_item_rows(const DevProblem &P, int t, int &tx, int &y0, int &ye) {
    if (t < P.n_left) {
        tx = 0;
        y0 = t * P.edge_h;
        ye = min(y0 + P.edge_h, P.H);
    } else if (t < P.n_left + P.n_top) {
        tx = 1 + (t - P.n_left);
        y0 = 0;
        ye = min(P.edge_h, P.H);
    } else {
        const int u = t - P.n_left - P.n_top, sx = P.tiles_x - 1;
        const int c = u / sx;
        tx = 1 + (u - c * sx);
        y0 = P.edge_h + c * P.tile_h;
        ye = min(y0 + P.tile_h, P.H);
    }
}

// The pass's reduction, in the pass: after item t's sums are written, the warp that completes
// the item's group sums the group in item order into the group sums, and the warp that
// completes the problem's last group sums the groups in order and runs the SCG tail.  The sums
// and their order are reduce_kernel's, so the results are the same bit for bit; what goes is
// the reduction's launch and its wait for the whole pass.  A group's counter is reset by the
// warp that completes it, the problem's by the tail.  Not inlined: inlined into the item loop
// it cost the pass 7% (its registers and code in the loop's way), as a call 0.6% less than the
// reduction launch.
__device__ __noinline__ void stream_reduce(const DevProblem &P, int t, int mode) {
    const int lane = threadIdx.x & 31;
    const int g = t / P.group;
    const int gsize = min(P.group, P.n_tiles - g * P.group);
    // every lane's stores of the item's sums are made visible before the warp counts the item
    __threadfence();
    __syncwarp();
    unsigned old = 0;
    if (lane == 0) old = atomicAdd(&P.gcounter[g], 1u);
    old = __shfl_sync(FULL, old, 0);
    if (old != (unsigned)(gsize - 1)) return;
    __threadfence();
    if (lane == 0) P.gcounter[g] = 0u;
    const float2 v = warp_sum_fields(P.partials + (size_t)g * P.group, P.n_tiles, gsize);
    const int slot = lane >> 1;
    if ((lane & 1) == 0 && slot < NPART) P.gpartials[(size_t)slot * P.n_groups + g] = v;
    __threadfence();
    __syncwarp();
    if (lane == 0) old = atomicAdd(P.counter, 1u);
    old = __shfl_sync(FULL, old, 0);
    if (old != (unsigned)(P.n_groups - 1)) return;
    __threadfence();
    ScgState L;
    load_state(L, P.st);
    const float2 w = warp_sum_fields(P.gpartials, P.n_groups, P.n_groups);
    double S[NPART];
#pragma unroll
    for (int j = 0; j < NPART; ++j) {
        const float hi = __shfl_sync(FULL, w.x, 2 * j), lo = __shfl_sync(FULL, w.y, 2 * j);
        S[j] = (double)hi + (double)lo;
    }
    if (lane == 0) {
        scg_tail_local(P, &L, S, mode);
        *P.st = L;
        *P.counter = 0u;
        __threadfence();
    }
}

// One warp's share of the pass: items from the launch's lists until they run out.  The edge
// path (EDGE) first takes the edge items [0, n_edge) from counter work[0], then helps with the
// rest; the interior path takes only the items [n_edge, n_items), from counter work[2].  Every
// item's ten sums are written as (hi, lo) pairs at its index; reduce_kernel combines them after
// the pass as it does the tile sums.
template <bool RPB, bool EDGE, bool L1>
__device__ __forceinline__ void stream_worker(StreamState &S, const DevProblem *__restrict__ probs,
                                              const int2 *__restrict__ items, int n_edge, int n_items,
                                              unsigned *work, int mode, double probe_alpha, double probe_beta,
                                              const StreamConsts &k, int reduce) {
    const int lane = threadIdx.x & 31;
    bool edge_list = EDGE;
    for (;;) {
        unsigned it = 0;
        if (lane == 0) it = edge_list ? atomicAdd(&work[0], 1u) : (unsigned)n_edge + atomicAdd(&work[2], 1u);
        it = __shfl_sync(FULL, it, 0);
        if (edge_list && it >= (unsigned)n_edge) {
            edge_list = false;
            continue;
        }
        if (it >= (unsigned)n_items) break;
        const int2 wt = items[it];
        const DevProblem &P = probs[wt.x];
        const ScgState *st = P.st;
        if (ld_cg(&st->done)) continue;
        const int t = wt.y;
        if (!MISR_IN_BOUNDS(t >= 0 && t < P.n_tiles, BC_TILE, t, P.n_tiles)) continue;
        // the interior path takes no edge item (its list holds none; checked all the same)
        if (!EDGE && !MISR_IN_BOUNDS(t >= P.n_left + P.n_top, BC_TILE, t, P.n_left)) continue;
        int tx, y0, ye;
        stream_item_rows(P, t, tx, y0, ye);
        const int cur = ld_cg(&st->cur), pcur = ld_cg(&st->pcur);
        const float alpha = mode == MODE_PROBE ? (float)probe_alpha : __ldcg(&st->alpha_f);
        const float beta = mode == MODE_PROBE ? (float)probe_beta : __ldcg(&st->beta_f);
        SegGeo g;
        g.H = P.H; g.W = P.W; g.pitch = P.pitch;
        g.y0 = y0;
        g.ye = ye;
        const int x0 = tx * SW_OWN, c0 = x0 - SW_HALO;
        g.v0 = c0 + 4 * lane;
        g.own_lane = lane >= SW_HALO / 4 && lane < (SW_HALO + SW_OWN) / 4;
        g.lane_in = g.v0 >= 0 && g.v0 + 3 < g.pitch;
        g.in0 = g.v0 >= 0 && g.v0 < g.W;
        g.in1 = g.v0 + 1 >= 0 && g.v0 + 1 < g.W;
        g.in2 = g.v0 + 2 >= 0 && g.v0 + 2 < g.W;
        g.in3 = g.v0 + 3 >= 0 && g.v0 + 3 < g.W;
        g.all_in = g.in0 && g.in3;
        g.left = c0 < 2 * MAXF + 2;
        if (!MISR_IN_BOUNDS(g.y0 < g.ye && x0 < g.W, BC_IMAGE, g.y0, x0)) continue;
#pragma unroll
        for (int i = 0; i < NPART; ++i) S.s[i] = 0.f;
        S.lo_jb = S.lo_rr = S.lo_rrx = S.lo_pr = 0.f;
        stream_item<RPB, EDGE, L1>(S, k, g, alpha, beta, P.X[cur], P.Rv[cur], P.Pv[pcur], P.Y, P.X[cur ^ 1],
                               P.Rv[cur ^ 1], P.Pv[pcur ^ 1]);
        // the item's sums: lanes outside the owned strip drop theirs; then a fixed-order warp
        // sum of (hi, lo) pairs
        const bool keep = g.own_lane;
        float2 v[NPART];
#pragma unroll
        for (int i = 0; i < NPART; ++i) v[i] = make_float2(keep ? S.s[i] : 0.f, 0.f);
        v[P_JB].y = keep ? S.lo_jb : 0.f;
        v[P_RR].y = keep ? S.lo_rr : 0.f;
        v[P_RRX].y = keep ? S.lo_rrx : 0.f;
        v[P_PR].y = keep ? S.lo_pr : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int i = 0; i < NPART; ++i) v[i] = df_add(v[i], shfl_xor_f2(v[i], off));
        if (lane < NPART) {
            float2 mine = v[0];
#pragma unroll
            for (int i = 1; i < NPART; ++i)
                if (lane == i) mine = v[i];
            P.partials[(size_t)lane * P.n_tiles + t] = mine;
        }
        if (reduce) stream_reduce(P, t, mode);
    }
}

// The streaming pass.  The launch's item list holds its n_edge edge items, then the rest.  CTAs
// below n_edge_ctas run the edge path, the others the interior path: one CTA per SM, so an SM
// keeps one path in its instruction cache.  RPB: r and p stored as bf16; L1: the smoothed L1
// data term.  reduce: the launch reduces its problems' sums itself (stream_reduce), else
// reduce_kernel follows it.
template <bool RPB, bool L1>
__global__ void __launch_bounds__(SW_NT, 1) scg_stream_kernel(const DevProblem *__restrict__ probs,
                                                              const int2 *__restrict__ items, int n_edge,
                                                              int n_items, int n_edge_ctas, unsigned *work, int mode,
                                                              double probe_alpha, double probe_beta,
                                                              const StreamConsts k, int reduce) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    extern __shared__ __align__(16) unsigned char stream_smem[];   // SW_SMEM_BYTES
    asm volatile("griddepcontrol.wait;" ::: "memory");
    StreamState S;
    S.wb = stream_smem + warp * SW_WARP_BYTES + 16 * lane;
    S.cur = 0;
    S.nxt = SW_STAGE_BYTES;
    if ((int)blockIdx.x < n_edge_ctas)
        stream_worker<RPB, true, L1>(S, probs, items, n_edge, n_items, work, mode, probe_alpha, probe_beta, k, reduce);
    else
        stream_worker<RPB, false, L1>(S, probs, items, n_edge, n_items, work, mode, probe_alpha, probe_beta, k, reduce);
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // the last warp to stop zeroes the launch's counters for the next launch
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(&work[1], 1u) == gridDim.x * (SW_NT / 32) - 1) {
            work[0] = 0u;
            work[1] = 0u;
            work[2] = 0u;
            __threadfence();
        }
    }
}

}  // namespace misr
