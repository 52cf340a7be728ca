// Host-side internals shared by the translation units of the library: the plan record, error
// reporting and the launch helpers of the kernels (which live in misr_api.cu only, so that
// every kernel has one copy and one set of attributes).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "misr.h"
#include "misr_types.cuh"

namespace misr_host {

// record a thread-local error text and return s
misr_status fail(misr_status s, const char *fmt, ...);

#define CK(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return misr_host::fail(MISR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// passes captured per CUDA graph replay
constexpr int GRAPH_CHUNK = 50;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now = -1;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

int grid_for(size_t n, int threads);
// row pitch (elements) of the workspace images of an HR image W pixels wide
int row_pitch(int W);
// device bytes misr_plan_create allocates for a descriptor (0 if the descriptor is refused)
size_t plan_bytes(const misr_desc &d);
// every check misr_plan_create makes before allocating
misr_status check_desc(const misr_desc &d);
// one fused SCG pass (the pass kernel, then its reduction) over the tiles (problem index, tile)
// and the groups (problem index, group) of the problems in `probs`; every tile and every group
// of every problem named must be listed exactly once.  `work`: the launch's tile counter (two
// unsigned ints, zero before the first launch; every launch leaves them zero).  Launches that
// share a `work` must be stream-ordered.
// Tiles per pass kernel instantiation: the tile list holds segment (shape 0, variant 0),
// (shape 0, variant 1), ..., (shape 1, variant 0), ... in that order, n[shape][variant] tiles
// each (variant: bit 0 bf16 r and p, bit 1 the L1 data term, bit 2 per-phase taps, which only
// the PHASED_SHAPE has); one pass launch per non-empty segment.
// The streaming shape's tiles are further split into runs of problems that share their
// constants (kernel parameters of one launch): one launch per run, in list order.
struct StreamRun {
    int variant = 0, count = 0;
    int n_edge = 0;                      // the run's edge items (listed first)
    int edge_ctas = 0;                   // planned edge CTAs of a run of one problem, else 0
    double edge_work = 0, int_work = 0;  // row steps of the edge and the other items (edge weighted)
    double edge_ctas_w = 0;              // sum of the problems' planned edge CTAs times their work
    bool reduce_in_pass = false;         // the launch reduces its problems' sums itself
    misr::StreamConsts k{};
};
// A problem of the frame-wise pass (frames that do not interleave into one HR image): its
// kernels run per problem, before the fused launches, and its groups join the reduction.
struct GenRun {
    int pidx = 0, ctas = 0;
    int tw = 1;                          // taps per axis (the kernels' compiled bucket)
    bool l1 = false;
};
struct PassSegs {
    int n[misr::N_SHAPES][misr::N_VARIANTS] = {};
    std::vector<StreamRun> runs;
    std::vector<GenRun> gen;
    int n_reduce = 0;                    // groups of the reduction launch (tile-shape problems)
    int total() const {
        int t = (int)gen.size();
        for (auto &a : n)
            for (int v : a) t += v;
        return t;
    }
};
// the constants of the streaming pass for a problem
misr::StreamConsts stream_consts(const misr::DevProblem &p);
// the pass kernel variant of a problem
inline int pass_variant(const misr::DevProblem &p) { return (p.rp_bf16 ? 1 : 0) | (p.l1 ? 2 : 0) | (p.phased ? 4 : 0); }
misr_status launch_pass_raw(const misr::DevProblem *probs, const int2 *tiles, const PassSegs &segs,
                            const int2 *groups, int n_groups, unsigned *work, int mode, double alpha, double beta,
                            cudaStream_t s);
// Whether a problem's pass runs in launches of its own: a streaming problem whose items fill at
// least half the grid's warps (merged with others, such problems ran slower than one after
// another), or a problem of the frame-wise pass (its kernels are per problem).
bool launch_alone(const misr::DevProblem &p);
// The tile and group lists of a launch over problems recs[i] (problem index idx[i] in the
// launch's record array), ordered by segment, each problem's border tiles first.
void build_pass_lists(const std::vector<const misr::DevProblem *> &recs, const std::vector<int> &idx,
                      std::vector<int2> &tiles, std::vector<int2> &groups, PassSegs &segs);
// prepare problem `pidx` of `probs` (host mirror `hp`): interleave frames (or copy them for the
// frame-wise pass), start point, reset (flags as prepare_kernel)
misr_status launch_prepare_raw(const misr::DevProblem *probs, int pidx, const misr::DevProblem &hp, const misr_desc &d,
                               const void *y_dev, const float *x_given, int x0_mode, int flags, cudaStream_t s);
// copy problem `pidx`'s iterate out (dense H x W)
misr_status launch_finalize_raw(const misr::DevProblem *probs, int pidx, size_t n, float *out, cudaStream_t s);

}  // namespace misr_host

struct misr_plan_s {
    int device = 0;
    misr_desc d{};
    misr::DevProblem hp{};              // host mirror of the device problem record
    misr::DevProblem *dprob = nullptr;  // device problem record
    int2 *dtile = nullptr;              // tile list of the fused pass (0, tile)
    misr_host::PassSegs segs;           // its one segment
    int2 *dgroup = nullptr;             // group list of its reduction (0, group)
    unsigned int *work = nullptr;       // the fused pass's tile counter
    char *ws = nullptr;                 // one allocation for everything above and below
    size_t ws_bytes = 0;
    size_t n = 0, m_total = 0;          // HR pixels, LR samples of all frames
    size_t n_pitched = 0;               // H * pitch
    cudaStream_t cap = nullptr;         // private stream used for graph capture
    cudaGraphExec_t chunk = nullptr;    // GRAPH_CHUNK passes (or the iteration count, if fewer)
    int chunk_len = 0;
    cudaGraphExec_t tail = nullptr;     // the iteration count's remainder after whole chunks
    int tail_len = 0;
    cudaEvent_t done_ev = nullptr;
    bool solved = false;
    misr::ScgState *st_host = nullptr;  // page-locked copy of the state
    void *io_y = nullptr;               // device buffers of misr_solve_host
    float *io_x = nullptr;
    // misr_solve_host_many: two device buffer pairs, a copy stream and its events, and the
    // device copies of each projection's final state
    void *pio_y[2] = {nullptr, nullptr};
    float *pio_x[2] = {nullptr, nullptr};
    cudaStream_t cpy = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
    misr::ScgState *st_ring = nullptr;
    int st_ring_cap = 0;
};
