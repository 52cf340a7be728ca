/*
 * misr.h -- C ABI of the B300 (sm_103a) multi-image super-resolution solver.
 *
 * The library solves, on one GPU, the MAP problem of Sec. 3.1 of the paper
 *     min_x  J(x) = sum_k || D B M_k x - y_k ||_2^2 + lambda * sum_d gamma(d) || x - S_d x ||_1
 * (Eq. 1 image formation, Eq. 6 data term, Eq. 8 BTV prior, Eq. 9 objective), or with the
 * smoothed L1 data term of the paper's experiments (misr_desc.data_norm), with Moller's
 * scaled conjugate gradient (Sec. 3.1, Algorithm 1, Table 1), for K low-resolution (LR)
 * frames taken with known subpixel detector shifts (Sec. 3.2).
 *
 * Conventions for every call:
 *  - Images are row-major, densely packed.  An LR frame is lr_h x lr_w; the K frames of one
 *    projection are stored back to back (K * lr_h * lr_w elements).  The HR image is
 *    (factor * lr_h) x (factor * lr_w) float32.
 *  - "_dev" pointers are CUDA device pointers on the device that was current when the plan
 *    was created; "_host" pointers are host memory.  The caller owns every buffer it passes;
 *    the library never frees or retains them past the call (asynchronous calls read them
 *    until the stream reaches that point).
 *  - misr_stream_t is a cudaStream_t (0 = the legacy default stream).
 *  - Every call returns a misr_status and never aborts; on failure misr_last_error() gives a
 *    thread-local description.  A call that fails leaves the caller's buffers untouched
 *    unless stated otherwise.
 *  - One plan runs one solve at a time: its workspace holds a single SCG state.  Calls on the
 *    same plan must be ordered (one stream, or synchronised).
 */
#ifndef MISR_H
#define MISR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MISR_OK = 0,
    MISR_EINVAL = 1,    /* invalid argument or descriptor */
    MISR_ENOMEM = 2,    /* device or host allocation failed */
    MISR_ECUDA = 3,     /* a CUDA runtime call failed */
    MISR_EAGAIN = 4,    /* not ready yet / no free slot */
    MISR_ETIMEOUT = 5,  /* a bounded wait ran out */
    MISR_ENOTIMPL = 6,  /* valid request this build does not support */
    MISR_ECANCELED = 7  /* a served request cancelled before it finished */
} misr_status;

/* element types of the LR frames and of the iterate */
enum { MISR_F32 = 0, MISR_U16 = 1, MISR_BF16 = 2 };

/* how the SCG start point x_1 is formed */
enum {
    MISR_X0_ZERO = 0,       /* x_1 = 0 */
    MISR_X0_SHIFT_ADD = 1,  /* multi-image interpolation (Sec. 4.1.1): each LR sample placed
                               at the HR pixel it was taken at (spread over the 2 x 2 pixels
                               around it with the bilinear weights for a non-integer shift),
                               several samples of one pixel averaged, 0 where none falls */
    MISR_X0_GIVEN = 2       /* x_1 = the caller's x buffer on entry */
};

/* Problem descriptor, copied by misr_plan_create (the pointers are read only during it). */
typedef struct misr_desc {
    int32_t lr_h, lr_w;      /* LR frame rows, columns (>= 1) */
    int32_t K;               /* number of frames, 1 <= K <= 64 */
    int32_t factor;          /* magnification f, 1 <= f <= 8; HR = f*lr_h x f*lr_w */
    const float *shifts;     /* host, K pairs (dx, dy) in LR px; the HR shift t = f*s (within 1e-4
                                of an integer counts as that integer), |t| <= 2^20.  M_k moves
                                the sampling grid by t, x zero outside the grid; a non-integer t
                                makes M_k a bilinear interpolation (reading of Eq. 1).
                                Two passes compute the same model.  The fused passes take frame
                                sets that interleave into one HR image: every t in [0, f) per
                                axis, one frame per HR phase floor(t), non-integer parts on a
                                product lattice (one fractional y shift per HR row phase, one x
                                shift per column phase, as x and y detector stages give; the
                                plan then runs the 32x32 tile shape, MISR_ENOTIMPL for another
                                explicit tile_shape), and a combined D B blur (psf_size, + f - 1
                                with binning, + 1 for non-integer shifts) of at most 5 taps per
                                axis.  Every other frame set (several frames on one phase, such
                                as the synthetic study's one-pixel shifts right, down, left and
                                up, Sec. 4.1.1; shifts outside [0, f); shifts off a product
                                lattice; a wider combined blur) runs the frame-wise pass,
                                whatever tile_shape asks; it keeps r and p in float
                                (iterate_dtype MISR_BF16: MISR_ENOTIMPL) and has no
                                allocation-free gradient */
    const float *psf;        /* host, psf_size^2 row-major PSF of B (Eq. 1); must be separable;
                                normalised to sum 1 by the plan; B is a convolution with it */
    int32_t psf_size;        /* odd, 1..5 */
    double lambda;           /* regulariser weight lambda of Eq. 9 (>= 0) */
    double btv_alpha;        /* decay alpha of gamma(d) = alpha^(dx+dy), Eq. 8 */
    int32_t btv_w;           /* BTV window w of Eq. 8, 1..3 */
    double eps;              /* in [1e-15, 1e15]: |t| of Eq. 8 is smoothed as sqrt(t^2+eps^2) - eps */
    int32_t iters;           /* SCG iterations, rejected ones included (Algorithm 1), 0..1e6 */
    int32_t x0_mode;         /* MISR_X0_* */
    int32_t in_dtype;        /* MISR_F32 frames, or MISR_U16 detector counts c converted on the
                                device to line integrals y = ln(flat_field) - ln(max(c, 1)) */
    float flat_field;        /* I0 for MISR_U16 (> 0) */
    int32_t iterate_dtype;   /* MISR_F32: x, r, p in float.  MISR_BF16: r and p (the gradient and
                                the search direction) stored in bf16, x kept in float as the master
                                copy (an alpha p update below the bf16 step of x is not lost);
                                stencils accumulate in float and the SCG scalars stay FP64 either
                                way.  misr_pass_probe needs MISR_F32. */
    int32_t tile_shape;      /* MISR_TILE_AUTO (0): the shape misr_autotune chose for this HR size
                                in this process, else the default (MISR_TILE_STREAM from 5e6 HR
                                pixels up where the plan's data term and shifts allow it,
                                MISR_TILE_32x32 otherwise); or one of MISR_TILE_* */
    int32_t data_norm;       /* MISR_NORM_L2 (0): the squared L2 data term of Eq. 6 above.
                                MISR_NORM_L1: the L1 data term of the paper's experiments
                                (Sec. 3.1), each residual t smoothed like the prior's |t|:
                                sum_k sum_i psi_d((A_k x - y_k)_i), psi_d(t) = sqrt(t^2 +
                                data_eps^2) - data_eps */
    double data_eps;         /* MISR_NORM_L1: the smoothing data_eps, in [1e-15, 1e15];
                                ignored for MISR_NORM_L2 */
    int32_t decimation;      /* MISR_DECIM_POINT (0): D samples HR pixel (f i, f j) of B M_k x.
                                MISR_DECIM_BIN: D is the mean of the f x f block starting there
                                (the 2 x 2 binning of the synthetic study, Sec. 4.1.1); D B is
                                then one blur whose taps span psf_size + f - 1 pixels per axis
                                (the fused passes take at most 5: psf_size 3 at f <= 2,
                                psf_size 1 at f <= 3, any PSF at f = 1; wider ones run the
                                frame-wise pass) */
} misr_desc;

/* data terms (misr_desc.data_norm) */
enum { MISR_NORM_L2 = 0, MISR_NORM_L1 = 1 };
/* decimation D (misr_desc.decimation) */
enum { MISR_DECIM_POINT = 0, MISR_DECIM_BIN = 1 };

/* Shapes of the fused pass.  MISR_TILE_32x64, _32x32, _16x64: HR pixels per CTA tile of the
 * persistent tile kernel (every model option).  MISR_TILE_STREAM: the row-streaming kernel, one
 * warp per strip of 112 HR columns walking its rows (integer shifts, either data term; a plan
 * with non-integer shifts on a product lattice gets MISR_ENOTIMPL).  Frame sets that do not
 * interleave (misr_desc.shifts) run the frame-wise pass whatever the shape.  The paper has no
 * counterpart: its partitions are whole sub-images per GPU (Sec. 3.1). */
enum { MISR_TILE_AUTO = 0, MISR_TILE_32x64 = 1, MISR_TILE_32x32 = 2, MISR_TILE_16x64 = 3, MISR_TILE_STREAM = 4,
       MISR_N_TILE_SHAPES = 4 };

/* Solve summary.  J_final, rnorm2 are FP64 reductions computed on the device. */
typedef struct misr_stats {
    int32_t iters_done;      /* SCG iterations run (rejected ones included) */
    int32_t accepted;        /* iterations whose step was accepted */
    int32_t status;          /* misr_status of the solve */
    int32_t reserved;
    double J_final;          /* J(x) at the returned x */
    double rnorm2;           /* |grad J(x)|^2 at the returned x */
    double lambda_scg;       /* Moller's scale parameter at the end */
} misr_stats;

typedef struct misr_plan_s *misr_plan_t;
typedef void *misr_stream_t;

/* Number of float64 columns per row of misr_get_trace, in this order:
 * E (J before the step), J_trial, alpha, delta, mu, lambda_scg, Delta, |p|^2, |r|^2, accept. */
#define MISR_TRACE_COLS 10
/* Number of float64 sums returned by misr_pass_probe, in this order:
 * J_data(x'), J_data(x') - J_data(x), R_BTV(x') (Eq. 8, without lambda), |r'|^2, r'.r,
 * p.r', |p|^2, r'.H(x')r', r'.H(x')p, p.H(x')p. */
#define MISR_PASS_SUMS 10

const char *misr_version(void);
/* Thread-local text of the last failure of a call made by this thread ("" if none). */
const char *misr_last_error(void);

/* Validate the descriptor and build a plan on the current device: the separable PSF taps,
 * the phase-to-frame table and the device workspace of one solve (7 HR float32 images plus
 * O(tiles) partial sums; for the frame-wise pass also a copy of the frames, three per-sample
 * buffers, the horizontal parts of the operator and of its adjoint (2 K H w + K h W floats) and
 * the per-frame, per-row tap tables of D B M_k, computed here in FP64), allocated here with
 * cudaMalloc.  The plan plays the part of the
 * system matrices that the paper builds once per scan and reuses for every rotation angle
 * (Sec. 3.2); no matrix is formed.
 * Errors: MISR_EINVAL (descriptor), MISR_ENOMEM, MISR_ECUDA, MISR_ENOTIMPL. */
misr_status misr_plan_create(const misr_desc *desc, misr_plan_t *out);

/* Synchronise the plan's work and free its workspace.  NULL is accepted. */
misr_status misr_plan_destroy(misr_plan_t plan);

/* Device bytes the plan holds. */
misr_status misr_plan_workspace_bytes(misr_plan_t plan, size_t *bytes);

/* Failure-path hook of the fused pass (for tests and diagnosis).  The wait for a tile's x, r
 * and p boxes gives up after `tries` polls and reports the tile late (the later wait for its
 * frames box keeps the default); the default, 2^24, is far beyond any healthy load.  A late load flags the projection: its SCG state is marked done and its
 * solve (or probe) returns MISR_ETIMEOUT; the copies already in flight are still waited for
 * (with the default limit) before the CTA stops, so the device context stays usable.
 * tries = 0 reports every load late without waiting.  Applies to solves of this plan launched
 * after the call; a batch or a server copies the plan's record when it is created or admits the
 * projection.  Synchronises the device.  Errors: MISR_EINVAL (NULL plan), MISR_ECUDA. */
misr_status misr_plan_set_wait_limit(misr_plan_t plan, uint32_t tries);

/* y_k = D B M_k x for every frame (Eq. 1 without noise, with the plan's decimation and
 * shifts): x_dev is the HR float32 image, y_dev receives K float32 frames.  Asynchronous on
 * stream.  Used to synthesise acquisitions. */
misr_status misr_forward(misr_plan_t plan, const float *x_dev, float *y_dev, misr_stream_t stream);

/* Multi-image interpolation (Sec. 4.1.1), the paper's non-iterative comparator: every LR
 * sample of y_dev (K frames, the plan's in_dtype; u16 counts are log-converted as for a solve)
 * is inserted at the HR pixel it was taken at, f*(i, j) + the frame's HR shift, and x_dev (HR
 * float32, dense) is 0 where no frame samples.  With non-integer shifts each sample is spread
 * over the 2 x 2 HR pixels around its position with the bilinear weights of M_k, and x is the
 * weighted mean there (sum_k M_k^T D^T y_k over sum_k M_k^T D^T 1).  It is also the start point of a
 * MISR_X0_SHIFT_ADD solve.  Reads only the plan's geometry: the plan's workspace and solve
 * state are not touched.  Asynchronous on stream.  Errors: MISR_EINVAL (NULL arguments),
 * MISR_ECUDA. */
misr_status misr_interpolate(misr_plan_t plan, const void *y_dev, float *x_dev, misr_stream_t stream);

/* Objective and gradient at x (Eq. 9 and its gradient 2 sum_k A_k^T (A_k x - y_k) +
 * lambda grad R; sum_k A_k^T psi_d'(A_k x - y_k) + lambda grad R with the L1 data term):
 * y_dev holds the K frames (in_dtype), x_dev the HR image, g_dev receives grad J(x) (HR
 * float32).  Blocking: *J_out (may be NULL) is valid on return. */
misr_status misr_gradient(misr_plan_t plan, const void *y_dev, const float *x_dev, float *g_dev,
                          double *J_out, misr_stream_t stream);

/* One fused SCG pass on explicit inputs (the per-iteration work of Algorithm 1):
 *   p' = r + beta * p_old,  x' = x + alpha * p',  r' = -grad J(x'),
 * and the sums listed at MISR_PASS_SUMS, where H(x') is the exact Hessian of J at x'.
 * All images are HR float32 device buffers; y_dev holds the K frames.  Blocking: sums
 * (host, MISR_PASS_SUMS doubles) is valid on return.  Exposed so that each pass can be
 * compared with an independent implementation. */
misr_status misr_pass_probe(misr_plan_t plan, const void *y_dev, const float *x_dev,
                            const float *r_dev, const float *p_old_dev, double alpha, double beta,
                            float *x_out_dev, float *r_out_dev, float *p_out_dev, double *sums,
                            misr_stream_t stream);

/* Full SCG solve (Algorithm 1 on one GPU, desc.iters iterations, failed ones included).
 * y_dev: K frames (in_dtype).  x_dev: HR float32 output (and the start point for
 * MISR_X0_GIVEN).  Asynchronous on stream unless stats is non-NULL, in which case the call
 * synchronises the stream and fills *stats. */
misr_status misr_solve(misr_plan_t plan, const void *y_dev, float *x_dev, misr_stream_t stream,
                       misr_stats *stats);

/* misr_solve on host buffers: copies y_host to the device, solves, copies x back to x_host,
 * all inside the call (blocking).  Page-locked host buffers give the fastest copies.  The
 * plan allocates the device copies on first use. */
misr_status misr_solve_host(misr_plan_t plan, const void *y_host, float *x_host, misr_stats *stats);

/* A stream of projections from host memory through one plan: solves projection k while the
 * frames of projection k+1 go to the device and the image of projection k-1 comes back, on a
 * copy stream beside the plan's stream, through two device buffer pairs the plan allocates on
 * first use and keeps.  The projections are solved one after another (same results as n calls
 * of misr_solve_host); only the copies overlap.  The CT setting of Sec. 3.2 reconstructs one
 * projection per rotation angle as they are acquired.
 * y_host[k]: frames of projection k (K x lr_h x lr_w, in_dtype, dense); x_host[k]: its HR image
 * (H x W float32, dense; also read as the start point under MISR_X0_GIVEN).  Page-locked host
 * buffers let the copies overlap the solves; pageable ones work but serialise.  The host
 * buffers must stay valid and unchanged until the call returns; it returns when every image
 * is in host memory.  stats: NULL or n records (projection k's in stats[k]).
 * Errors: MISR_EINVAL (NULL plan or arrays or entries, n < 0), MISR_ENOMEM, MISR_ECUDA,
 * MISR_ETIMEOUT (a tile load timed out in at least one projection: its record carries the
 * status, the others are complete). */
misr_status misr_solve_host_many(misr_plan_t plan, int32_t n, const void *const *y_host, float *const *x_host,
                                 misr_stats *stats);

/* Bounds-check record of the library's checked build (libmisr_check.so, compiled with
 * MISR_BOUNDS_CHECK, where every shared-memory item position, global store, tile or group
 * index and TMA x coordinate of the device code is checked, and a failed check is recorded and
 * its access skipped instead of made).  `bits` receives one bit per kind of check that failed
 * since the last call (0: none); `first` (4 ints, may be NULL) the first failure: the check,
 * two of its values and the block.  The record is then cleared.  Synchronises the device.
 * The normal build returns MISR_ENOTIMPL.  Errors: MISR_EINVAL (bits NULL), MISR_ECUDA. */
misr_status misr_debug_bounds(uint32_t *bits, int32_t *first);

/* ---- Checkpoint and resume ----------------------------------------------------------------
 * A projection's SCG solve can stop after any iteration and continue later, on the same plan or
 * on another plan of the same geometry and storage type (e.g. one with more iterations), with
 * the result bit for bit that of one uninterrupted solve.  A checkpoint holds the iterate x_k,
 * the gradient r_k, the previous direction p_{k-1} (float, or bf16 for MISR_BF16 plans) and
 * the SCG scalars of Algorithm 1 (Table 1): lambda, lambda-bar, delta, mu, |p|^2, E, beta,
 * alpha, success and the iteration count.  Layout (little-endian, host memory): a 32-byte
 * header (magic 0x4353524d, version 1, H, W, bf16 flag, state record size, 2 reserved words),
 * the state record, then x, r and p as dense H x W row-major planes.
 *
 * misr_state_bytes: the size of the plan's checkpoint.
 * misr_export_state: after a solve (or resume) of the plan has completed (synchronises the
 *   device), write its checkpoint to host memory `buf` of at least `bytes` bytes.
 * misr_import_state: load a checkpoint into the plan.  The iteration target becomes the plan's
 *   desc.iters; a checkpoint stopped by its iteration count is live again if that target is
 *   larger.  The plan's trace keeps rows only from iterations run on it.  Synchronises.
 * misr_resume: continue the plan's solve (after misr_import_state, or after a solve whose
 *   iteration target was reached) to its iteration target: y_dev gives the frames again (the
 *   plan does not keep them), x_dev receives the image.  Asynchronous on stream unless stats is
 *   non-NULL, as misr_solve.
 * Errors: MISR_EINVAL (NULL arguments, too small a buffer, a checkpoint of another geometry,
 * storage type, data term, model (shifts, PSF, decimation, the prior's and the data term's
 * constants; the iteration count may differ), state layout or version), MISR_ECUDA, and
 * misr_solve's. */
misr_status misr_state_bytes(misr_plan_t plan, size_t *bytes);
misr_status misr_export_state(misr_plan_t plan, void *buf, size_t bytes);
misr_status misr_import_state(misr_plan_t plan, const void *buf, size_t bytes);
misr_status misr_resume(misr_plan_t plan, const void *y_dev, float *x_dev, misr_stream_t stream,
                        misr_stats *stats);

/* Copy the per-iteration trace of the plan's last completed solve (MISR_TRACE_COLS doubles
 * per iteration) into out (host, max_rows rows); *rows receives the number written.
 * Synchronises with the plan's last solve. */
misr_status misr_get_trace(misr_plan_t plan, double *out, int32_t max_rows, int32_t *rows);

/* ---- Batched solves (many projections per launch) ---------------------------------------
 * A batch groups plans (uneven sizes, factors, frame counts, tile shapes, r/p storage types,
 * data terms, decimations and shift sets are fine; all on one device) so that every SCG step of
 * all of them is one fused-pass launch over the tiles of the projections that share launches
 * (one per tile shape and kernel variant present), then one reduction launch, while each
 * projection that fills the GPU on its own (or runs the frame-wise pass) takes its own plan's
 * pass on a stream of its own, forked and joined within the step; the steps are replayed as a
 * CUDA graph.  The CT setting of Sec. 3.2 produces one independent projection per
 * rotation angle; a batch advances many of them at once.  Each projection keeps its own
 * workspace, SCG state and fixed-order reductions, so its result equals its own misr_solve.
 * A plan may belong to several batches but runs one solve at a time. */
typedef struct misr_batch_s *misr_batch_t;

/* Build the batch tables (problem records, the shared tile and group lists, the streams of the
 * projections that launch alone) on the plans' device.
 * plans: n plans (host array, copied).  Errors: MISR_EINVAL, MISR_ENOMEM, MISR_ECUDA. */
misr_status misr_batch_create(int32_t n, const misr_plan_t *plans, misr_batch_t *out);

/* Synchronise and free the batch tables (the plans stay).  NULL is accepted. */
misr_status misr_batch_destroy(misr_batch_t batch);

/* Solve every projection of the batch: y_dev[i] (K_i frames, the plan's in_dtype) to x_dev[i]
 * (HR float32; also the start point of plans with MISR_X0_GIVEN).  Each projection runs its own
 * plan's iteration count.  Asynchronous on stream unless stats (n entries) is non-NULL, in
 * which case the call synchronises and fills stats[i] for plan i. */
misr_status misr_batch_solve(misr_batch_t batch, const void *const *y_dev, float *const *x_dev,
                             misr_stream_t stream, misr_stats *stats);

/* ---- Serving: continuous batching of projections as an acquisition produces them ----------
 * The CT setting of Sec. 3.2 reconstructs each rotation angle while the scan goes on.  A
 * server owns a worker thread, a private stream and a pool of slots.  A slot is a plan (its
 * workspace and its device-resident SCG state) of one geometry class.  Requests are admitted in
 * arrival order into free slots of their class.  A new slot is created when its workspace fits
 * the HBM budget, and idle slots of other classes are freed to make room.  Every tick runs
 * passes_per_tick fused-pass launches over the tiles of all live slots (one SCG iteration per
 * launch for each), so a request that arrives while others are on the GPU joins the next
 * launch; a slot whose projection fills the GPU on its own (or runs the frame-wise pass) takes
 * its passes on a stream of its own, which waits for the worker's stream once after the
 * slot's admission and is joined back within each tick, so that independent projections'
 * launches overlap; its state is copied on that stream after the tick's passes, and the
 * worker reads that copy, so the slot's next tick runs on at once.  The worker queues a tick
 * before it reads the states of the previous one, so the GPU does not wait for the host
 * between ticks.  Finished projections are copied out and their
 * slots reused.  Each projection keeps its own state and fixed-order reductions: its result is
 * the same alone and in the mix.  A request's frames are read once, when it is admitted (into
 * the slot's workspace), and its output is written once, when it finishes. */
typedef struct misr_server_s *misr_server_t;

typedef struct misr_server_cfg {
    int32_t max_slots;           /* most projections resident at once, 1..4096 */
    int32_t passes_per_tick;     /* SCG iterations between admission rounds, 0 = 4 */
    uint64_t hbm_budget_bytes;   /* > 0: slot workspaces use at most this many bytes */
    uint64_t hbm_reserve_bytes;  /* budget 0: admit while free device memory exceeds this */
    int32_t idle_spin_us;        /* once nothing is queued or running, the worker polls for new
                                    requests this many microseconds (0..1000000) before it
                                    sleeps: a request arriving meanwhile starts without a
                                    thread wake-up, at the cost of one busy CPU core; 0 = sleep
                                    at once */
    int32_t reserved;            /* 0 */
} misr_server_cfg;

/* Start a server on the current device.  Errors: MISR_EINVAL, MISR_ENOMEM. */
misr_status misr_server_create(const misr_server_cfg *cfg, misr_server_t *out);

/* Stop the worker after its current tick, then free every slot.  Requests still queued or
 * running are dropped (their buffers are no longer touched after this returns).  NULL is
 * accepted. */
misr_status misr_server_destroy(misr_server_t server);

/* Queue one projection: desc (copied; checked like misr_plan_create), y_dev its frames,
 * x_dev the HR output (and the start point for MISR_X0_GIVEN).  Both device buffers must stay
 * valid until misr_poll reports the ticket finished.  *ticket identifies the request. */
misr_status misr_submit(misr_server_t server, const misr_desc *desc, const void *y_dev, float *x_dev,
                        uint64_t *ticket);

/* MISR_EAGAIN while the request is queued or running.  Once it finished: its status (MISR_OK,
 * or the failure), *stats (may be NULL), times[3] = submit, start and end on the host's steady
 * clock in seconds (may be NULL); the ticket is then forgotten (a further poll gives
 * MISR_EINVAL). */
misr_status misr_poll(misr_server_t server, uint64_t ticket, misr_stats *stats, double *times);

/* Cancel a request.  Queued: it is dropped at once.  Running: it stops when the worker reads
 * the states of the tick in which it sees the cancel; x_dev is not written (passes already
 * queued may still run on the slot's own workspace, which the request no longer reads or
 * writes).  Either way the ticket finishes with MISR_ECANCELED, and its buffers may be released
 * once misr_poll (or misr_server_wait) reports that.  A ticket that already finished keeps its
 * result.  Errors: MISR_EINVAL (NULL server, unknown ticket). */
misr_status misr_cancel(misr_server_t server, uint64_t ticket);

/* Wait at most timeout_s seconds for the ticket to finish (then poll it).  MISR_OK when it
 * finished, MISR_ETIMEOUT otherwise, MISR_EINVAL for an unknown ticket. */
misr_status misr_server_wait(misr_server_t server, uint64_t ticket, double timeout_s);

/* Counters: out[0] queued requests, out[1] running, out[2] slots, out[3] slot workspace bytes,
 * out[4] fused-pass launches so far. */
misr_status misr_server_counters(misr_server_t server, int64_t *out);

/* Autotuner of the pass's shape.  Times `passes` fused passes of every compiled shape that can
 * run the descriptor (the three tile shapes and, for integer shifts, the streaming one) on the
 * geometry of `desc` (on zeroed device buffers it allocates and frees), and remembers the
 * fastest for plans of the same HR size created with tile_shape = MISR_TILE_AUTO in this
 * process.  shape_out (may be NULL): the chosen MISR_TILE_*; ms_out (may be NULL): the time per
 * pass of each shape, MISR_N_TILE_SHAPES values in MISR_TILE_* order.  passes: 1..1000.  A
 * descriptor with non-integer shifts on a product lattice runs on MISR_TILE_32x32 only: that
 * shape is returned at once, nothing is timed or remembered, and ms_out is zeroed.  A frame set
 * that runs the frame-wise pass has no shape to choose: MISR_TILE_AUTO is returned the same way,
 * before any device work.
 * Errors: MISR_EINVAL (descriptor, passes), MISR_ENOMEM, MISR_ECUDA. */
misr_status misr_autotune(const misr_desc *desc, int32_t passes, int32_t *shape_out, double *ms_out);

/* Allocation-free objective and gradient.  The paper has no counterpart: this is an
 * interface addition of the library.  It returns the same J(x) and grad J(x) as
 * misr_gradient for the problem in desc, without a plan and without allocating any device
 * memory.  It is for callers that cannot call cudaMalloc: a process whose device memory is
 * already fully reserved by another allocator (a framework's caching pool, a detector
 * pipeline that reserves all its buffers up front), or a time-critical acquisition loop
 * that cannot afford the implicit device synchronisation of cudaMalloc / cudaFree.
 * The workspace is a fixed array inside the library, sized for HR images of at most
 * 512 x 512 pixels (about 7 MB, held on every GPU that loads the library until the process
 * exits); larger problems return MISR_EINVAL.  It computes in FP32 only: a descriptor with
 * iterate_dtype other than MISR_F32 returns MISR_EINVAL, and a frame set that runs the
 * frame-wise pass (misr_desc.shifts: its frame copies and tap tables need a plan's workspace)
 * MISR_ENOTIMPL.  The first call on a device looks up
 * the array's device address and sets the pass kernel's attributes.  Every call uses the same
 * array, so calls that overlap on the GPU (other streams or host threads) race.  y_dev, x_dev,
 * g_dev as for misr_gradient.
 * Blocking: the call copies its problem record from host memory and synchronises `stream`
 * before it returns, so g_dev and *J_out (may be NULL) are valid on return; it must not be
 * called on a stream that is being captured into a CUDA graph.  A tile load that does not land
 * within the wait limit (misr_noalloc_set_wait_limit) returns MISR_ETIMEOUT; the next call
 * starts from a clean array. */
misr_status misr_gradient_noalloc(const misr_desc *desc, const void *y_dev, const float *x_dev, float *g_dev,
                                  double *J_out, misr_stream_t stream);

/* Polls of a tile-load wait before misr_gradient_noalloc reports the load late (the
 * counterpart of misr_plan_set_wait_limit for the plan-free call; process-wide, default
 * 2^24).  0 reports every load late, which the failure tests use to exercise the timeout path
 * without a fault.  Errors: none. */
misr_status misr_noalloc_set_wait_limit(uint32_t tries);

#ifdef __cplusplus
}
#endif
#endif /* MISR_H */
