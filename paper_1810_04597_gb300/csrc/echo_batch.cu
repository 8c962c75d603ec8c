// echo_batch.cu -- a batch of independent runs (e.g. a parameter sweep of
// tori of uneven sizes) advanced together, optionally replayed from one
// captured CUDA graph.  Three schedules (echo_batch_mode):
//   0  ONE persistent cooperative kernel per SSP-RK3 stage (below);
//   1  one ordinary launch per phase over the tiles of all runs;
//   2  run-major: each run's own launch sequence, so that the working set of
//      one run stays in L2 across its phases; the runs may be spread over
//      concurrent branches (side streams forked from the batch stream; in a
//      captured graph, parallel branches) so that small runs overlap.
//
// Inside the stage kernel the work of every phase of the stage -- ghost fill
// of faces (3 passes), c2p, ghost fill of primitives (3 passes), faces
// (x, y, z), EMFs (x, y, z), update -- is cut into tiles over all runs; the
// resident blocks take tiles round-robin or from an atomic queue, and
// grid.sync() separates dependent phases.  The cooperative launch guarantees
// that all blocks are co-resident, so the grid barrier cannot deadlock.
// Tiles never straddle two (run, kind) segments, so every warp calls one
// body with one set of template arguments (the bodies use warp-collective
// operations).  Each run keeps its own CFL dt.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "echo_ctx.h"
#include "echo_batch_kernels.cuh"

using namespace echo;

// ------------------------------------------------------------------ host side

struct echo_batch {
    std::vector<echo_ctx *> runs;
    int nruns = 0;
    int mk = 0;
    int precision = 64;
    bool mlp = false;
    int guess = 0;
    Phys ph;
    double cfl = 0.4;
    BatchPlan plan;
    size_t ws_need = 0;
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    bool bound = false;
    int grid_blocks = 0;
    int blocks_per_sm = 0;
    int phased = 0;       // 0 persistent kernel per stage, 1 one launch per phase, 2 run-major
    bool use_graph = false;
    int branches = 1;                       // run-major: concurrent branches
    std::vector<cudaStream_t> side;         // one per branch
    std::vector<cudaEvent_t> fork_join;     // [0] fork, [1 + k] join of branch k
    std::vector<int> branch_of;             // run -> branch
    cudaGraphExec_t gexec = nullptr;
    double graph_dt = 0.0;
    std::string err;
};

namespace {

int bfail(echo_batch *b, int code, const std::string &m)
{
    if (b)
        b->err = m;
    return code;
}

int bcheck(echo_batch *b, const char *where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return bfail(b, ECHO_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return ECHO_OK;
}

size_t a256(size_t v) { return (v + 255) / 256 * 256; }

long long phase_count(const Geom &g, int p, int kind)
{
    const long long n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    switch (p) {
    case PH_FILLF0:
    case PH_FILLP0:
        return fill_count(g, 0);
    case PH_FILLF1:
    case PH_FILLP1:
        return fill_count(g, 1);
    case PH_FILLF2:
    case PH_FILLP2:
        return fill_count(g, 2);
    case PH_C2P:
        return n0 * n1 * n2;
    case PH_FACES: {
        int cnt[3], off[3];
        faces_space(g, kind, cnt, off);
        return (long long)cnt[0] * cnt[1] * cnt[2];
    }
    case PH_EMF: {
        int cnt[3], off[3];
        emf_space(g, kind, cnt, off);
        return (long long)cnt[0] * cnt[1] * cnt[2];
    }
    default:
        return (n0 + 1) * (n1 + 1) * (n2 + 1);
    }
}

void build_plan(echo_batch *b, int tile, int dynamic)
{
    BatchPlan &P = b->plan;
    P.nruns = b->nruns;
    P.tile = tile;
    P.dynamic = dynamic;
    for (int p = 0; p < BATCH_NPHASE; ++p) {
        const int kinds = (p == PH_FACES || p == PH_EMF) ? 3 : 1;
        long long t = 0;
        int ns = 0;
        for (int r = 0; r < b->nruns; ++r)
            for (int k = 0; k < kinds; ++k) {
                const long long cnt = phase_count(b->runs[r]->geo, p, k);
                P.seg[p][ns] = Segment{t, cnt, r, k};
                t += (cnt + tile - 1) / tile;
                ++ns;
            }
        P.nseg[p] = ns;
        P.ntiles[p] = t;
    }
}

template <typename R>
FillList<R> faces_fill(const Arrays<R> &A)
{
    FillList<R> L{};
    for (int d = 0; d < 3; ++d) {
        L.a[d] = A.U[5 + d];
        L.comp[d] = d;
        L.face[d] = d;
        L.dens[d] = 1;
    }
    L.count = 3;
    return L;
}

template <typename R>
FillList<R> prims_fill(const Arrays<R> &A)
{
    FillList<R> L{};
    const int comps[8] = {-1, 0, 1, 2, -1, 0, 1, 2};
    for (int q = 0; q < 8; ++q) {
        L.a[q] = A.P[q];
        L.comp[q] = comps[q];
        L.face[q] = -1;
        L.dens[q] = 0;
    }
    L.count = 8;
    return L;
}

template <typename R>
size_t desc_bytes(int nruns) { return a256(sizeof(RunDesc<R>) * nruns); }

const void *stage_kernel(const echo_batch *b)
{
    return b->precision == 64 ? batch_stage_kernel<double>(b->mk, b->mlp) : batch_stage_kernel<float>(b->mk, b->mlp);
}

// the network's starts come from a pass of their own: no parameter block in
// the stage kernel's shared memory
size_t dyn_smem(const echo_batch *) { return 0; }

int occupancy(const echo_batch *b)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stage_kernel(b), 128, dyn_smem(b)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

int max_blocks_per_sm(echo_batch *b) { return occupancy(b); }

int upload(echo_batch *b)
{
    char *descs = b->ws;
    char *planp = b->ws + (b->precision == 64 ? desc_bytes<double>(b->nruns) : desc_bytes<float>(b->nruns));
    if (b->precision == 64) {
        std::vector<RunDesc<double>> d(b->nruns);
        for (int r = 0; r < b->nruns; ++r) {
            d[r].g = b->runs[r]->geo;
            d[r].A = b->runs[r]->ad;
            d[r].ff = faces_fill(d[r].A);
            d[r].fp = prims_fill(d[r].A);
        }
        if (cudaMemcpyAsync(descs, d.data(), sizeof(RunDesc<double>) * b->nruns, cudaMemcpyHostToDevice, b->stream)
            != cudaSuccess)
            return bcheck(b, "batch upload");
    } else {
        std::vector<RunDesc<float>> d(b->nruns);
        for (int r = 0; r < b->nruns; ++r) {
            d[r].g = b->runs[r]->geo;
            d[r].A = b->runs[r]->af;
            d[r].ff = faces_fill(d[r].A);
            d[r].fp = prims_fill(d[r].A);
        }
        if (cudaMemcpyAsync(descs, d.data(), sizeof(RunDesc<float>) * b->nruns, cudaMemcpyHostToDevice, b->stream)
            != cudaSuccess)
            return bcheck(b, "batch upload");
    }
    if (cudaMemcpyAsync(planp, &b->plan, sizeof(BatchPlan), cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
        return bcheck(b, "batch upload");
    // the host copies come from stack/heap buffers: finish before they go away
    if (cudaStreamSynchronize(b->stream) != cudaSuccess)
        return bcheck(b, "batch upload");
    return ECHO_OK;
}

int launch_stage(echo_batch *b, int stage, double dt)
{
    const size_t dsz = b->precision == 64 ? desc_bytes<double>(b->nruns) : desc_bytes<float>(b->nruns);
    void *descs = b->ws;
    BatchPlan *planp = reinterpret_cast<BatchPlan *>(b->ws + dsz);
    unsigned long long *qctr = reinterpret_cast<unsigned long long *>(b->ws + dsz + a256(sizeof(BatchPlan)));
    Phys ph = b->ph;
    double cfl = b->cfl;
    int guess = b->guess;
    if (b->mlp) {
        // the network's Newton starts of this stage, before the persistent
        // kernel (its features read the face field before the stage's own
        // ghost fill: a cell next to a periodic seam may start from a field
        // one stage old; Newton decides the result either way)
        if (b->precision == 64)
            batch_enqueue_guess<double>(b->mk, descs, planp, b->plan, ph.gr_f, b->stream);
        else
            batch_enqueue_guess<float>(b->mk, descs, planp, b->plan, ph.gr_f, b->stream);
    }
    void *args[] = {&descs, &planp, &qctr, &ph, &stage, &dt, &cfl, &guess};
    cudaError_t e = cudaLaunchCooperativeKernel(stage_kernel(b), dim3(b->grid_blocks), dim3(128), args, dyn_smem(b),
                                                b->stream);
    if (e != cudaSuccess)
        return bfail(b, ECHO_ECUDA, std::string("cooperative launch: ") + cudaGetErrorString(e));
    return ECHO_OK;
}

int enqueue_step(echo_batch *b, double dt)
{
    if (b->phased == 1) {
        const size_t dsz = b->precision == 64 ? desc_bytes<double>(b->nruns) : desc_bytes<float>(b->nruns);
        const BatchPlan *planp = reinterpret_cast<const BatchPlan *>(b->ws + dsz);
        if (b->precision == 64)
            batch_enqueue_phased<double>(b->mk, b->mlp, b->ws, planp, b->plan, b->nruns, b->ph, b->guess, dt, b->cfl,
                                         b->stream);
        else
            batch_enqueue_phased<float>(b->mk, b->mlp, b->ws, planp, b->plan, b->nruns, b->ph, b->guess, dt, b->cfl,
                                        b->stream);
        return bcheck(b, "phased step");
    }
    if (b->phased == 2) {
        // run-major: every run's own launch sequence; with several branches the
        // runs are split over side streams forked from and joined back into the
        // batch stream (in a captured graph: parallel branches)
        if (b->branches == 1) {
            for (echo_ctx *c : b->runs) {
                const int rc = echo_internal_enqueue_step(c, dt, b->stream);
                if (rc)
                    return bfail(b, rc, std::string("run step: ") + c->err);
            }
            return ECHO_OK;
        }
        if (cudaEventRecord(b->fork_join[0], b->stream) != cudaSuccess)
            return bcheck(b, "fork");
        for (int k = 0; k < b->branches; ++k)
            if (cudaStreamWaitEvent(b->side[k], b->fork_join[0], 0) != cudaSuccess)
                return bcheck(b, "fork");
        for (int r = 0; r < b->nruns; ++r) {
            echo_ctx *c = b->runs[r];
            const int rc = echo_internal_enqueue_step(c, dt, b->side[b->branch_of[r]]);
            if (rc)
                return bfail(b, rc, std::string("run step: ") + c->err);
        }
        for (int k = 0; k < b->branches; ++k) {
            if (cudaEventRecord(b->fork_join[1 + k], b->side[k]) != cudaSuccess
                || cudaStreamWaitEvent(b->stream, b->fork_join[1 + k], 0) != cudaSuccess)
                return bcheck(b, "join");
        }
        return ECHO_OK;
    }
    for (int st = 0; st < 3; ++st) {
        const int rc = launch_stage(b, st, dt);
        if (rc)
            return rc;
    }
    return ECHO_OK;
}

void drop_graph(echo_batch *b)
{
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
}

void drop_branches(echo_batch *b)
{
    for (cudaStream_t s : b->side)
        cudaStreamDestroy(s);
    for (cudaEvent_t e : b->fork_join)
        cudaEventDestroy(e);
    b->side.clear();
    b->fork_join.clear();
}

// Longest-processing-time assignment of runs (by zone count) to branches.
void assign_branches(echo_batch *b)
{
    std::vector<int> order(b->nruns);
    for (int r = 0; r < b->nruns; ++r)
        order[r] = r;
    auto zones = [b](int r) {
        const Geom &g = b->runs[r]->geo;
        return (long long)g.n[0] * g.n[1] * g.n[2];
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return zones(x) > zones(y); });
    std::vector<long long> load(b->branches, 0);
    b->branch_of.assign(b->nruns, 0);
    for (int r : order) {
        int k = 0;
        for (int q = 1; q < b->branches; ++q)
            if (load[q] < load[k])
                k = q;
        b->branch_of[r] = k;
        load[k] += zones(r);
    }
}

}  // namespace

extern "C" {

int echo_batch_create(echo_ctx *const *runs, int nruns, echo_batch **out)
{
    if (!out)
        return ECHO_EINVAL;
    *out = nullptr;
    if (!runs || nruns < 1 || nruns > BATCH_MAXRUNS)
        return ECHO_EINVAL;
    for (int r = 0; r < nruns; ++r) {
        const echo_ctx *c = runs[r];
        if (!c || !c->bound)
            return ECHO_ESTATE;
        if (c->metric.kind != runs[0]->metric.kind || c->precision != runs[0]->precision
            || c->eos.gamma != runs[0]->eos.gamma || c->cfl != runs[0]->cfl)
            return ECHO_EINVAL;
    }
    echo_batch *b = new (std::nothrow) echo_batch();
    if (!b)
        return ECHO_ENOMEM;
    b->runs.assign(runs, runs + nruns);
    b->nruns = nruns;
    b->mk = runs[0]->metric.kind;
    b->precision = runs[0]->precision;
    b->ph = runs[0]->ph;
    b->cfl = runs[0]->cfl;
    b->mlp = (runs[0]->c2p_guess & 3) == 1;
    b->guess = runs[0]->c2p_guess;
    build_plan(b, 256, 1);
    assign_branches(b);
    const size_t dsz = b->precision == 64 ? desc_bytes<double>(nruns) : desc_bytes<float>(nruns);
    b->ws_need = dsz + a256(sizeof(BatchPlan)) + a256(BATCH_NPHASE * sizeof(unsigned long long));
    *out = b;
    return ECHO_OK;
}

size_t echo_batch_workspace_bytes(const echo_batch *b) { return b ? b->ws_need : 0; }

int echo_batch_bind(echo_batch *b, void *ws, size_t bytes, void *stream)
{
    if (!b)
        return ECHO_EINVAL;
    if (!ws || ((uintptr_t)ws % 256) != 0)
        return bfail(b, ECHO_EINVAL, "batch workspace must be 256-byte aligned device memory");
    if (bytes < b->ws_need)
        return bfail(b, ECHO_ENOMEM, "batch workspace smaller than echo_batch_workspace_bytes");
    b->ws = static_cast<char *>(ws);
    b->stream = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(b->ws, 0, b->ws_need, b->stream) != cudaSuccess)
        return bcheck(b, "batch bind");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int m = occupancy(b);
    if (m < 1)
        return bfail(b, ECHO_ECUDA, "stage kernel cannot be resident");
    b->blocks_per_sm = m;
    b->grid_blocks = b->blocks_per_sm * sms;
    b->bound = true;
    drop_graph(b);
    return upload(b);
}

int echo_batch_mode(echo_batch *b, int phased)
{
    if (!b)
        return ECHO_EINVAL;
    if (phased < 0 || phased > 2)
        return bfail(b, ECHO_EINVAL, "batch mode: 0 persistent, 1 phased, 2 run-major");
    b->phased = phased;
    drop_graph(b);
    return ECHO_OK;
}

int echo_batch_config(echo_batch *b, int tile, int blocks_per_sm, int dynamic_queue)
{
    if (!b || !b->bound)
        return b ? bfail(b, ECHO_ESTATE, "bind the batch first") : ECHO_EINVAL;
    if (tile < 128 || tile % 128 != 0 || tile > 8192)
        return bfail(b, ECHO_EINVAL, "tile must be a multiple of 128 in [128, 8192]");
    if (blocks_per_sm < 1 || blocks_per_sm > occupancy(b))
        return bfail(b, ECHO_EINVAL, "blocks_per_sm must be in [1, max resident]");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->blocks_per_sm = blocks_per_sm;
    b->grid_blocks = blocks_per_sm * sms;
    build_plan(b, tile, dynamic_queue ? 1 : 0);
    drop_graph(b);
    return upload(b);
}

int echo_batch_max_blocks_per_sm(echo_batch *b) { return b ? max_blocks_per_sm(b) : 0; }

int echo_batch_branches(echo_batch *b, int branches)
{
    if (!b)
        return ECHO_EINVAL;
    if (branches < 1 || branches > b->nruns)
        return bfail(b, ECHO_EINVAL, "branches must be in [1, number of runs]");
    drop_graph(b);
    drop_branches(b);
    b->branches = branches;
    if (branches > 1) {
        b->side.assign(branches, nullptr);
        b->fork_join.assign(branches + 1, nullptr);
        for (int k = 0; k < branches; ++k)
            if (cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) != cudaSuccess) {
                b->side.resize(k);
                drop_branches(b);
                b->branches = 1;
                return bcheck(b, "branch streams");
            }
        for (int k = 0; k <= branches; ++k)
            if (cudaEventCreateWithFlags(&b->fork_join[k], cudaEventDisableTiming) != cudaSuccess) {
                b->fork_join.resize(k);
                drop_branches(b);
                b->branches = 1;
                return bcheck(b, "branch events");
            }
    }
    assign_branches(b);
    return ECHO_OK;
}

int echo_batch_graph(echo_batch *b, int enable)
{
    if (!b)
        return ECHO_EINVAL;
    if (enable && (b->stream == nullptr || b->stream == cudaStreamLegacy))
        return bfail(b, ECHO_EINVAL, "graph replay needs a created stream (the legacy default stream cannot be captured)");
    b->use_graph = enable != 0;
    if (!b->use_graph)
        drop_graph(b);
    return ECHO_OK;
}

int echo_batch_step(echo_batch *b, double dt)
{
    if (!b || !b->bound)
        return b ? bfail(b, ECHO_ESTATE, "bind the batch first") : ECHO_EINVAL;
    for (echo_ctx *c : b->runs) {
        if (!c->have_state)
            return bfail(b, ECHO_ESTATE, "every run needs a state");
        if (c->geo.order != 0 && b->phased != 2)
            return bfail(b, ECHO_EINVAL, "runs of order 1 need the run-major schedule (echo_batch_mode 2)");
    }
    // the runs' per-cell start codes, on the batch stream and outside any
    // capture: run-major inverts with each run's own guess mode, the other
    // schedules with the batch's (the network for every run, or none)
    for (echo_ctx *c : b->runs) {
        const int mode = b->phased == 2 ? c->c2p_guess : b->guess;
        const int rc = echo_internal_prepare_start(c, mode, b->stream);
        if (rc)
            return bfail(b, rc, std::string("start codes: ") + c->err);
    }
    if (!b->use_graph) {
        const int rc = enqueue_step(b, dt);
        return rc ? rc : bcheck(b, "echo_batch_step");
    }
    if (b->gexec && b->graph_dt != dt)
        drop_graph(b);
    if (!b->gexec) {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return bcheck(b, "graph capture begin");
        const int rc = enqueue_step(b, dt);
        const cudaError_t ee = cudaStreamEndCapture(b->stream, &graph);
        if (rc || ee != cudaSuccess) {
            if (graph)
                cudaGraphDestroy(graph);
            cudaGetLastError();
            b->use_graph = false;
            return rc ? rc : bfail(b, ECHO_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ee));
        }
        const cudaError_t ei = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            b->gexec = nullptr;
            b->use_graph = false;
            return bfail(b, ECHO_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
        }
        b->graph_dt = dt;
    }
    if (cudaGraphLaunch(b->gexec, b->stream) != cudaSuccess)
        return bcheck(b, "graph launch");
    return ECHO_OK;
}

const char *echo_batch_last_error(const echo_batch *b) { return b ? b->err.c_str() : "null batch"; }

void echo_batch_destroy(echo_batch *b)
{
    if (!b)
        return;
    drop_graph(b);
    drop_branches(b);
    delete b;
}

}  // extern "C"
