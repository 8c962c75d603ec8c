// echo_batch.cu -- a batch of independent runs (e.g. a parameter sweep of
// tori of uneven sizes) advanced by ONE persistent cooperative kernel per
// SSP-RK3 stage, optionally replayed from a captured CUDA graph.
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
#include <cooperative_groups.h>

#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "echo_ctx.h"
#include "echo_kernels.cuh"

namespace cg = cooperative_groups;
using namespace echo;

namespace echo {

constexpr int BATCH_MAXRUNS = 32;
constexpr int BATCH_NPHASE = 10;
constexpr int BATCH_MAXSEG = 3 * BATCH_MAXRUNS;

// phase kinds
enum { PH_FILLF0 = 0, PH_FILLF1, PH_FILLF2, PH_C2P, PH_FILLP0, PH_FILLP1, PH_FILLP2, PH_FACES, PH_EMF, PH_UPDATE };

template <typename R>
struct RunDesc {
    Geom g;
    Arrays<R> A;
    FillList<R> ff;   // face field
    FillList<R> fp;   // primitives
};

struct Segment {
    long long first_tile;   // global tile index of the segment's first tile
    long long count;        // work items
    int run;
    int kind;               // sub-kind: direction for fills/faces/emf
};

struct BatchPlan {
    int nruns;
    int tile;
    int dynamic;
    int nseg[BATCH_NPHASE];
    long long ntiles[BATCH_NPHASE];
    Segment seg[BATCH_NPHASE][BATCH_MAXSEG];
};

template <int MK, typename R, bool MLP>
__global__ void __launch_bounds__(128) k_batch_stage(const RunDesc<R> *__restrict__ runs, const BatchPlan *__restrict__ plan,
                                                     unsigned long long *qctr, Phys ph, int stage, double dt_fixed,
                                                     double cfl)
{
    cg::grid_group grid = cg::this_grid();
    __shared__ LimScratch<R> lsm;
    __shared__ long long s_tile;
    extern __shared__ float4 mlp_smem4[];
    const int nruns = plan->nruns;
    const int tile = plan->tile;
    const float *sm = nullptr;
    if constexpr (MLP) {
        float *Ps = reinterpret_cast<float *>(mlp_smem4);
        const float *src = runs[0].A.mlp;
        for (int q = threadIdx.x; q < MLP_BLOCK; q += blockDim.x)
            Ps[q] = src[q];
        __syncthreads();
        sm = Ps;
    }
    if (stage == 0 && blockIdx.x == 0 && (int)threadIdx.x < nruns) {
        DevScalars *sc = runs[threadIdx.x].A.scal;
        sc->rate_bits = 0ULL;
        sc->dt = dt_fixed > 0.0 ? dt_fixed : 0.0;
    }
    for (int p = 0; p < BATCH_NPHASE; ++p) {
        if (blockIdx.x == 0 && threadIdx.x == 0)
            qctr[(p + 1) % BATCH_NPHASE] = 0ULL;   // next phase's queue (visible after grid.sync)
        if (p == PH_FILLP0 && stage == 0 && dt_fixed <= 0.0 && blockIdx.x == 0 && (int)threadIdx.x < nruns) {
            DevScalars *sc = runs[threadIdx.x].A.scal;
            const double rate = __longlong_as_double((long long)sc->rate_bits);
            sc->totals[6] = rate;
            sc->dt = rate > 0.0 ? cfl / rate : 0.0;
        }
        const long long ntiles = plan->ntiles[p];
        const int nseg = plan->nseg[p];
        for (long long it = 0;; ++it) {
            long long tl;
            if (plan->dynamic) {
                if (threadIdx.x == 0)
                    s_tile = (long long)atomicAdd(&qctr[p], 1ULL);
                __syncthreads();
                tl = s_tile;
                __syncthreads();
            } else {
                tl = blockIdx.x + it * (long long)gridDim.x;
            }
            if (tl >= ntiles)
                break;
            int sgi = 0;
            while (sgi + 1 < nseg && plan->seg[p][sgi + 1].first_tile <= tl)
                ++sgi;
            const Segment sgm = plan->seg[p][sgi];
            const RunDesc<R> &rd = runs[sgm.run];
            const long long base = (tl - sgm.first_tile) * tile;
            for (int c = 0; c < tile; c += blockDim.x) {
                const long long t = base + c + threadIdx.x;
                switch (p) {
                case PH_FILLF0:
                case PH_FILLF1:
                case PH_FILLF2:
                    fill_body<R>(rd.g, p - PH_FILLF0, rd.ff, t);
                    break;
                case PH_C2P:
                    c2p_body<MK, R, MLP>(rd.g, ph, rd.A, 0, stage == 0 ? 1 : 0, t, sm);
                    break;
                case PH_FILLP0:
                case PH_FILLP1:
                case PH_FILLP2:
                    fill_body<R>(rd.g, p - PH_FILLP0, rd.fp, t);
                    break;
                case PH_FACES:
                    if (sgm.kind == 0)
                        faces_body<0, MK, R>(rd.g, ph, rd.A, t, lsm);
                    else if (sgm.kind == 1)
                        faces_body<1, MK, R>(rd.g, ph, rd.A, t, lsm);
                    else
                        faces_body<2, MK, R>(rd.g, ph, rd.A, t, lsm);
                    break;
                case PH_EMF:
                    if (sgm.kind == 0)
                        emf_body<0, MK, R>(rd.g, rd.A, t, lsm);
                    else if (sgm.kind == 1)
                        emf_body<1, MK, R>(rd.g, rd.A, t, lsm);
                    else
                        emf_body<2, MK, R>(rd.g, rd.A, t, lsm);
                    break;
                default:
                    update_body<MK, R>(rd.g, ph, rd.A, stage, nullptr, t);
                    break;
                }
            }
            __syncthreads();   // shared scratch reused by the next tile
        }
        grid.sync();
    }
}

}  // namespace echo

// ------------------------------------------------------------------ host side

struct echo_batch {
    std::vector<echo_ctx *> runs;
    int nruns = 0;
    int mk = 0;
    int precision = 64;
    bool mlp = false;
    Phys ph;
    double cfl = 0.4;
    BatchPlan plan;
    size_t ws_need = 0;
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    bool bound = false;
    int grid_blocks = 0;
    int blocks_per_sm = 0;
    bool use_graph = false;
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
    const long long p0 = g.np[0], p1 = g.np[1], p2 = g.np[2];
    switch (p) {
    case PH_FILLF0:
    case PH_FILLP0:
        return 2LL * NG * p1 * p2;
    case PH_FILLF1:
    case PH_FILLP1:
        return 2LL * NG * p0 * p2;
    case PH_FILLF2:
    case PH_FILLP2:
        return 2LL * NG * p0 * p1;
    case PH_C2P:
        return n0 * n1 * n2;
    case PH_FACES:
        return kind == 0 ? (n0 + 1) * p1 * p2 : (kind == 1 ? p0 * (n1 + 1) * p2 : p0 * p1 * (n2 + 1));
    case PH_EMF:
        return kind == 0 ? n0 * (n1 + 1) * (n2 + 1) : (kind == 1 ? (n0 + 1) * n1 * (n2 + 1) : (n0 + 1) * (n1 + 1) * n2);
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
    }
    L.count = 8;
    return L;
}

template <typename R>
size_t desc_bytes(int nruns) { return a256(sizeof(RunDesc<R>) * nruns); }

template <typename R>
const void *kernel_ptr(int mk, bool mlp)
{
    if (mk == 1)
        return mlp ? (const void *)k_batch_stage<1, R, true> : (const void *)k_batch_stage<1, R, false>;
    return mlp ? (const void *)k_batch_stage<0, R, true> : (const void *)k_batch_stage<0, R, false>;
}

const void *stage_kernel(const echo_batch *b)
{
    return b->precision == 64 ? kernel_ptr<double>(b->mk, b->mlp) : kernel_ptr<float>(b->mk, b->mlp);
}

size_t dyn_smem(const echo_batch *b) { return b->mlp ? MLP_BLOCK * sizeof(float) : 0; }

int max_blocks_per_sm(echo_batch *b)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stage_kernel(b), 128, dyn_smem(b)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

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
    void *args[] = {&descs, &planp, &qctr, &ph, &stage, &dt, &cfl};
    cudaError_t e = cudaLaunchCooperativeKernel(stage_kernel(b), dim3(b->grid_blocks), dim3(128), args, dyn_smem(b),
                                                b->stream);
    if (e != cudaSuccess)
        return bfail(b, ECHO_ECUDA, std::string("cooperative launch: ") + cudaGetErrorString(e));
    return ECHO_OK;
}

int enqueue_step(echo_batch *b, double dt)
{
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
    b->mlp = runs[0]->c2p_guess == 1;
    build_plan(b, 256, 1);
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
    const int mb = max_blocks_per_sm(b);
    if (mb < 1)
        return bfail(b, ECHO_ECUDA, "stage kernel cannot be resident");
    b->blocks_per_sm = mb;
    b->grid_blocks = mb * sms;
    b->bound = true;
    drop_graph(b);
    return upload(b);
}

int echo_batch_config(echo_batch *b, int tile, int blocks_per_sm, int dynamic_queue)
{
    if (!b || !b->bound)
        return b ? bfail(b, ECHO_ESTATE, "bind the batch first") : ECHO_EINVAL;
    if (tile < 128 || tile % 128 != 0 || tile > 8192)
        return bfail(b, ECHO_EINVAL, "tile must be a multiple of 128 in [128, 8192]");
    const int mb = max_blocks_per_sm(b);
    if (blocks_per_sm < 1 || blocks_per_sm > mb)
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
    for (echo_ctx *c : b->runs)
        if (!c->have_state)
            return bfail(b, ECHO_ESTATE, "every run needs a state");
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
    delete b;
}

}  // extern "C"
