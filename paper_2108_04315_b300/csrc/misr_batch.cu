// Batched SCG solves: many independent projections (uneven sizes, magnification factors and
// frame counts) advanced together, one fused-pass launch per SCG step over the tiles of those
// that share launches and each of the others' own pass on a stream of its own, the step loop replayed
// as a CUDA graph.  Each projection keeps its own plan workspace,
// SCG state and fixed-order reductions, so its result is the same alone and in a batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "misr.h"
#include "misr_internal.h"

using namespace misr;
using namespace misr_host;

struct misr_batch_s {
    int device = 0;
    int n = 0;
    std::vector<misr_plan_t> plans;
    DevProblem *dprobs = nullptr;   // n problem records (copies of the plans' records)
    unsigned int *work = nullptr;   // the fused pass's tile counter
    void *mem = nullptr;
    int max_iters = 0;
    // Problems whose passes run in launches of their own (launch_alone) take them, in the step
    // graph, on a stream each (their plan's own pass: its lists and tile counter), forked from
    // the capture stream and joined back; the others share the step's launches.  Independent
    // problems' launches then overlap, the next one filling the SMs the last items of the
    // previous one leave idle.
    std::vector<int> own;           // indices of those problems
    PassSegs segs_shared;           // the step's launches over the others
    int shared_items = 0, shared_groups = 0;
    int2 *dshared = nullptr;        // their tile list, then their group list
    std::vector<cudaStream_t> own_streams;
    std::vector<cudaEvent_t> own_joins;
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;     // private stream used for graph capture
    cudaGraphExec_t chunk = nullptr;    // GRAPH_CHUNK steps (or max_iters, if fewer)
    int chunk_len = 0;
    cudaGraphExec_t tail = nullptr;     // the remainder of max_iters after whole chunks
    int tail_len = 0;
    ScgState *st_host = nullptr;    // n page-locked states
};

static size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

extern "C" misr_status misr_batch_destroy(misr_batch_t b) {
    if (!b) return MISR_OK;
    DeviceGuard g(b->device);
    cudaDeviceSynchronize();
    if (b->chunk) cudaGraphExecDestroy(b->chunk);
    if (b->tail) cudaGraphExecDestroy(b->tail);
    for (cudaStream_t st : b->own_streams)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->own_joins)
        if (ev) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->st_host) cudaFreeHost(b->st_host);
    if (b->mem) cudaFree(b->mem);
    delete b;
    return MISR_OK;
}

extern "C" misr_status misr_batch_create(int32_t n, const misr_plan_t *plans, misr_batch_t *out) {
    if (!out) return fail(MISR_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || !plans) return fail(MISR_EINVAL, "a batch needs n >= 1 plans");
    for (int i = 0; i < n; ++i) {
        if (!plans[i]) return fail(MISR_EINVAL, "plan %d is NULL", i);
        if (plans[i]->device != plans[0]->device) return fail(MISR_EINVAL, "plans %d and 0 are on different devices", i);
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return fail(MISR_EINVAL, "plan %d appears twice (a plan holds one solve)", i);
    }
    misr_batch_t b = new (std::nothrow) misr_batch_s();
    if (!b) return fail(MISR_ENOMEM, "host allocation failed");
    b->device = plans[0]->device;
    b->n = n;
    b->plans.assign(plans, plans + n);
    std::vector<DevProblem> recs(n);
    for (int i = 0; i < n; ++i) {
        recs[i] = plans[i]->hp;
        b->max_iters = std::max(b->max_iters, plans[i]->d.iters);
    }
    // the shared launches: one per (tile shape, kernel variant: r/p storage type, data term, tap
    // layout) present among the projections that do not launch alone
    std::vector<const DevProblem *> rps;
    std::vector<int> idxs;
    for (int i = 0; i < n; ++i) {
        if (launch_alone(plans[i]->hp)) b->own.push_back(i);
        else { rps.push_back(&plans[i]->hp); idxs.push_back(i); }
    }
    std::vector<int2> sitems, sgroups;
    if (!rps.empty()) build_pass_lists(rps, idxs, sitems, sgroups, b->segs_shared);
    b->shared_items = (int)sitems.size();
    b->shared_groups = (int)sgroups.size();
    sitems.insert(sitems.end(), sgroups.begin(), sgroups.end());
    DeviceGuard g(b->device);
    const size_t rec_bytes = round_up(sizeof(DevProblem) * n, 256);
    const size_t shared_bytes = round_up(sizeof(int2) * std::max<size_t>(sitems.size(), 1), 256);
    cudaError_t e = cudaMalloc(&b->mem, rec_bytes + 256 + shared_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(MISR_ENOMEM, "cudaMalloc for the batch tables failed: %s", cudaGetErrorString(e));
    }
    b->dprobs = static_cast<DevProblem *>(b->mem);
    b->work = reinterpret_cast<unsigned int *>(static_cast<char *>(b->mem) + rec_bytes);
    b->dshared = reinterpret_cast<int2 *>(static_cast<char *>(b->mem) + rec_bytes + 256);
    b->own_streams.assign(b->own.size(), nullptr);
    b->own_joins.assign(b->own.size(), nullptr);
    do {
        if (!sitems.empty() &&
            (e = cudaMemcpy(b->dshared, sitems.data(), sizeof(int2) * sitems.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
            break;
        if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess) break;
        for (size_t q = 0; q < b->own.size() && e == cudaSuccess; ++q) {
            e = cudaStreamCreateWithFlags(&b->own_streams[q], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->own_joins[q], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) break;
        if ((e = cudaMemcpy(b->dprobs, recs.data(), sizeof(DevProblem) * n, cudaMemcpyHostToDevice)) != cudaSuccess) break;
        if ((e = cudaMemset(b->work, 0, 256)) != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaMallocHost((void **)&b->st_host, sizeof(ScgState) * n)) != cudaSuccess) break;
    } while (0);
    if (e != cudaSuccess) {
        misr_status r = fail(MISR_ECUDA, "batch setup: %s", cudaGetErrorString(e));
        misr_batch_destroy(b);
        return r;
    }
    *out = b;
    return MISR_OK;
}

// One SCG step of every projection on stream s: the shared launches over the projections that
// share them, and each of the others' own pass on its stream, forked from s and joined back.
static misr_status batch_step(misr_batch_t b, int mode, cudaStream_t s) {
    if (!b->own.empty()) {
        CK(cudaEventRecord(b->fork, s));
        for (cudaStream_t st : b->own_streams) CK(cudaStreamWaitEvent(st, b->fork, 0));
    }
    misr_status r = MISR_OK;
    if (b->segs_shared.total() > 0)
        r = launch_pass_raw(b->dprobs, b->dshared, b->segs_shared, b->dshared + b->shared_items, b->shared_groups,
                            b->work, mode, 0.0, 0.0, s);
    for (size_t q = 0; q < b->own.size() && r == MISR_OK; ++q) {
        const misr_plan_t p = b->plans[b->own[q]];
        r = launch_pass_raw(p->dprob, p->dtile, p->segs, p->dgroup, p->hp.n_groups, p->work, mode, 0.0, 0.0,
                            b->own_streams[q]);
    }
    for (size_t q = 0; q < b->own.size(); ++q) {   // join (also after a failed launch: no stream left forked)
        CK(cudaEventRecord(b->own_joins[q], b->own_streams[q]));
        CK(cudaStreamWaitEvent(s, b->own_joins[q], 0));
    }
    return r;
}

// `len` SCG steps of the batch, captured on its private stream
static misr_status capture_steps(misr_batch_t b, int len, cudaGraphExec_t *exec) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    misr_status r = MISR_OK;
    for (int i = 0; i < len && r == MISR_OK; ++i) r = batch_step(b, MODE_ITER, b->cap);
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (r != MISR_OK) { if (graph) cudaGraphDestroy(graph); return r; }
    if (e != cudaSuccess) return fail(MISR_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(MISR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return MISR_OK;
}

// a chunk of GRAPH_CHUNK steps and the remainder of max_iters: a solve launches max_iters steps
static misr_status batch_graph(misr_batch_t b) {
    const int want = std::max(1, std::min(b->max_iters, GRAPH_CHUNK));
    const int tail = std::max(b->max_iters, 0) % want;
    if (b->chunk && b->chunk_len == want && b->tail_len == tail) return MISR_OK;
    if (b->chunk) { cudaGraphExecDestroy(b->chunk); b->chunk = nullptr; }
    if (b->tail) { cudaGraphExecDestroy(b->tail); b->tail = nullptr; }
    b->chunk_len = b->tail_len = 0;
    misr_status r = capture_steps(b, want, &b->chunk);
    if (r != MISR_OK) return r;
    if (tail > 0) r = capture_steps(b, tail, &b->tail);
    if (r != MISR_OK) { cudaGraphExecDestroy(b->chunk); b->chunk = nullptr; return r; }
    b->chunk_len = want;
    b->tail_len = tail;
    return MISR_OK;
}

extern "C" misr_status misr_batch_solve(misr_batch_t b, const void *const *y_dev, float *const *x_dev,
                                        misr_stream_t stream, misr_stats *stats) {
    if (!b || !y_dev || !x_dev) return fail(MISR_EINVAL, "NULL argument");
    for (int i = 0; i < b->n; ++i)
        if (!y_dev[i] || !x_dev[i]) return fail(MISR_EINVAL, "NULL frame or image pointer for projection %d", i);
    DeviceGuard g(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    misr_status r = batch_graph(b);
    if (r != MISR_OK) return r;
    for (int i = 0; i < b->n && r == MISR_OK; ++i) {
        const misr_plan_t p = b->plans[i];
        r = launch_prepare_raw(b->dprobs, i, p->hp, p->d, y_dev[i], x_dev[i], p->d.x0_mode, 1 | 2 | 4, s);
    }
    if (r == MISR_OK) r = batch_step(b, MODE_INIT, s);
    if (r != MISR_OK) return r;
    for (int done = 0; done + b->chunk_len <= b->max_iters; done += b->chunk_len) CK(cudaGraphLaunch(b->chunk, s));
    if (b->tail) CK(cudaGraphLaunch(b->tail, s));
    for (int i = 0; i < b->n && r == MISR_OK; ++i) r = launch_finalize_raw(b->dprobs, i, b->plans[i]->n, x_dev[i], s);
    if (r != MISR_OK) return r;
    for (int i = 0; i < b->n; ++i) {
        CK(cudaEventRecord(b->plans[i]->done_ev, s));
        b->plans[i]->solved = true;
    }
    if (!stats) return MISR_OK;
    for (int i = 0; i < b->n; ++i)
        CK(cudaMemcpyAsync(&b->st_host[i], b->plans[i]->hp.st, sizeof(ScgState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    misr_status worst = MISR_OK;
    for (int i = 0; i < b->n; ++i) {
        const ScgState &h = b->st_host[i];
        stats[i].iters_done = h.iter;
        stats[i].accepted = h.accepted;
        stats[i].status = h.status == DEV_OK ? MISR_OK : MISR_ETIMEOUT;
        stats[i].reserved = 0;
        stats[i].J_final = h.E;
        stats[i].rnorm2 = h.rn2;
        stats[i].lambda_scg = h.lam;
        if (stats[i].status != MISR_OK) worst = MISR_ETIMEOUT;
    }
    if (worst != MISR_OK) return fail(worst, "a tile load of the fused pass did not complete in time");
    return MISR_OK;
}
