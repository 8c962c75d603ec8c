// echo_batch_kernels.cuh -- device side of the batched runs (internal):
// run descriptors, the tile plan, the persistent cooperative stage kernel and
// the per-phase kernels.  Instantiated per storage type in
// echo_batch_f64.cu and echo_batch_f32.cu.
#pragma once

#include <cooperative_groups.h>

#include "echo_kernels.cuh"

namespace cg = cooperative_groups;

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

// The persistent kernel calls each phase body through a non-inlined
// wrapper: inlined into one switch the bodies' live ranges would be
// allocated together (~250 registers, 2 blocks per SM); called, the kernel
// needs only the largest body's registers.
template <typename R>
__device__ __noinline__ void nl_fill(const Geom &g, int d, const FillList<R> &L, long long t)
{
    fill_body<R>(g, d, L, t);
}
template <int MK, typename R, int NET>
__device__ __noinline__ void nl_c2p(const Geom &g, const Phys &ph, const Arrays<R> &A, int guess, int rate, long long t)
{
    c2p_body<MK, R, NET>(g, ph, A, guess, rate, t, nullptr);
}
template <int D, int MK, typename R>
__device__ __noinline__ void nl_faces(const Geom &g, const Phys &ph, const Arrays<R> &A, long long t,
                                      LimScratch<R> &lsm)
{
    faces_body<D, MK, R>(g, ph, A, t, lsm);
}
template <int E, int MK, typename R>
__device__ __noinline__ void nl_emf(const Geom &g, const Arrays<R> &A, long long t, LimScratch<R> &lsm)
{
    emf_body<E, MK, R>(g, A, t, lsm);
}
template <int MK, typename R>
__device__ __noinline__ void nl_update(const Geom &g, const Phys &ph, const Arrays<R> &A, int stage, long long t)
{
    update_body<MK, R>(g, ph, A, stage, nullptr, t);
}

// NET: 0 no network; 3 the network's Newton starts, written by
// k_bphase_guess_tc before the stage.
template <int MK, typename R, int NET, int MINB>
__global__ void __launch_bounds__(128, MINB) k_batch_stage(const RunDesc<R> *__restrict__ runs, const BatchPlan *__restrict__ plan,
                                                     unsigned long long *qctr, Phys ph, int stage, double dt_fixed,
                                                     double cfl, int guess_mode)
{
    cg::grid_group grid = cg::this_grid();
    __shared__ LimScratch<R> lsm;
    __shared__ long long s_tile;
    const int nruns = plan->nruns;
    const int tile = plan->tile;
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
                    nl_fill<R>(rd.g, p - PH_FILLF0, rd.ff, t);
                    break;
                case PH_C2P:
                    nl_c2p<MK, R, NET>(rd.g, ph, rd.A, guess_mode, stage == 0 ? 1 : 0, t);
                    break;
                case PH_FILLP0:
                case PH_FILLP1:
                case PH_FILLP2:
                    nl_fill<R>(rd.g, p - PH_FILLP0, rd.fp, t);
                    break;
                case PH_FACES:
                    if (sgm.kind == 0)
                        nl_faces<0, MK, R>(rd.g, ph, rd.A, t, lsm);
                    else if (sgm.kind == 1)
                        nl_faces<1, MK, R>(rd.g, ph, rd.A, t, lsm);
                    else
                        nl_faces<2, MK, R>(rd.g, ph, rd.A, t, lsm);
                    break;
                case PH_EMF:
                    if (sgm.kind == 0)
                        nl_emf<0, MK, R>(rd.g, rd.A, t, lsm);
                    else if (sgm.kind == 1)
                        nl_emf<1, MK, R>(rd.g, rd.A, t, lsm);
                    else
                        nl_emf<2, MK, R>(rd.g, rd.A, t, lsm);
                    break;
                default:
                    nl_update<MK, R>(rd.g, ph, rd.A, stage, t);
                    break;
                }
            }
            __syncthreads();   // shared scratch reused by the next tile
        }
        grid.sync();
    }
}

// ------------------------------------------------------------------ phased
// mode: one ordinary launch per phase over the tiles of all runs (each phase
// kernel keeps its own register allocation); a step is ~32 launches, usually
// replayed from a CUDA graph.

__device__ __forceinline__ int find_segment(const BatchPlan *plan, int p, long long tl)
{
    int sgi = 0;
    const int nseg = plan->nseg[p];
    while (sgi + 1 < nseg && plan->seg[p][sgi + 1].first_tile <= tl)
        ++sgi;
    return sgi;
}

template <typename R>
__global__ void __launch_bounds__(128) k_bphase_fill(const RunDesc<R> *__restrict__ runs, const BatchPlan *__restrict__ plan,
                                                     int p)
{
    const long long tl = blockIdx.x;
    const Segment sgm = plan->seg[p][find_segment(plan, p, tl)];
    const RunDesc<R> &rd = runs[sgm.run];
    const long long base = (tl - sgm.first_tile) * plan->tile;
    const int d = p < PH_C2P ? p - PH_FILLF0 : p - PH_FILLP0;
    for (int c = 0; c < plan->tile; c += blockDim.x)
        fill_body<R>(rd.g, d, p < PH_C2P ? rd.ff : rd.fp, base + c + threadIdx.x);
}

template <int MK, typename R, int NET>
__global__ void __launch_bounds__(128) k_bphase_c2p(const RunDesc<R> *__restrict__ runs, const BatchPlan *__restrict__ plan,
                                                    Phys ph, int guess_mode, int want_rate)
{
    const long long tl = blockIdx.x;
    const Segment sgm = plan->seg[PH_C2P][find_segment(plan, PH_C2P, tl)];
    const RunDesc<R> &rd = runs[sgm.run];
    const long long base = (tl - sgm.first_tile) * plan->tile;
    for (int c = 0; c < plan->tile; c += blockDim.x)
        c2p_body<MK, R, NET>(rd.g, ph, rd.A, guess_mode, want_rate, base + c + threadIdx.x, nullptr);
}

// The network's Newton starts for the cells every run's last inversion
// listed (tensor cores, echo_mlp_tc.cuh), as k_mlp_guess_tc does for one
// run: persistent CTAs walk the runs' lists in tiles of 128 cells, run after
// run (each CTA forms the tiles' prefix sums over the runs' list lengths),
// choose per cell between the network start and the previous-stage Z, and
// load the next tile's inputs during the current tile's MMA round trips.
// All runs use runs[0]'s network.
template <int MK, typename R>
__global__ void __launch_bounds__(128, 6) k_bphase_guess_tc(const RunDesc<R> *__restrict__ runs,
                                                         const BatchPlan *__restrict__ plan, float gr_f)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ long long s_first_tile[ECHO_BATCH_MAXRUNS + 1];
    const int nruns = plan->nruns;
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int r = 0; r < nruns; ++r) {
            s_first_tile[r] = acc;
            acc += ((long long)runs[r].A.scal->nlist_count + 127) / 128;
        }
        s_first_tile[nruns] = acc;
    }
    __syncthreads();
    const long long ntiles = s_first_tile[nruns];
    long long tile = blockIdx.x;
    if (tile >= ntiles)
        return;   // block-uniform: nothing listed for this CTA (nothing allocated yet)
    auto load = [&](long long tl, int &run, CellIn<R> &x) {
        run = 0;
        while (run + 1 < nruns && s_first_tile[run + 1] <= tl)
            ++run;
        const long long cnt = (long long)runs[run].A.scal->nlist_count;
        const long long r = (tl - s_first_tile[run]) * 128 + threadIdx.x;
        listed_cell_load<MK, R>(runs[run].g, runs[run].A, runs[run].A.nlist, cnt, r, x);
    };
    TcMlp tm;
    tc_setup(tm, tc_smem, runs[0].A.mlp);
    CellIn<R> x;
    int run = 0;
    load(tile, run, x);
    for (; tile < ntiles; tile += gridDim.x) {
        float f[MLP_NI], o[MLP_NO];
        const int cur = run;
        const float D = cell_in_features<MK, R>(runs[cur].A, x, f);
        const int id = x.id;
        const bool live = x.live;
        const long long next = tile + gridDim.x;
        if (next < ntiles)
            load(next, run, x);
        const bool ok = tc_tile(tm, f, o);
        if (live) {
            float z0 = -1.0f;
            if (ok) {
                const float Wg = expf(o[0]), pD = expf(o[1]);
                z0 = net_beats(o[2], runs[cur].A.ze[id]) ? D * Wg * (1.0f + gr_f * pD * Wg) : 0.0f;
            }
            runs[cur].A.zg[id] = z0;
        }
    }
    tc_teardown(tm);
}

// Empty every run's network-start list (after the network's pass, before
// the inversion that lists the cells again).
template <typename R>
__global__ void k_bphase_clear_lists(const RunDesc<R> *__restrict__ runs, int nruns)
{
    if ((int)threadIdx.x < nruns)
        runs[threadIdx.x].A.scal->nlist_count = 0ULL;
}

template <int MK, typename R>
__global__ void __launch_bounds__(128) k_bphase_faces(const RunDesc<R> *__restrict__ runs, const BatchPlan *__restrict__ plan,
                                                      Phys ph)
{
    __shared__ LimScratch<R> lsm;
    const long long tl = blockIdx.x;
    const Segment sgm = plan->seg[PH_FACES][find_segment(plan, PH_FACES, tl)];
    const RunDesc<R> &rd = runs[sgm.run];
    const long long base = (tl - sgm.first_tile) * plan->tile;
    for (int c = 0; c < plan->tile; c += blockDim.x) {
        const long long t = base + c + threadIdx.x;
        if (sgm.kind == 0)
            faces_body<0, MK, R>(rd.g, ph, rd.A, t, lsm);
        else if (sgm.kind == 1)
            faces_body<1, MK, R>(rd.g, ph, rd.A, t, lsm);
        else
            faces_body<2, MK, R>(rd.g, ph, rd.A, t, lsm);
    }
}

template <int MK, typename R>
__global__ void __launch_bounds__(128) k_bphase_emf(const RunDesc<R> *__restrict__ runs, const BatchPlan *__restrict__ plan)
{
    __shared__ LimScratch<R> lsm;
    const long long tl = blockIdx.x;
    const Segment sgm = plan->seg[PH_EMF][find_segment(plan, PH_EMF, tl)];
    const RunDesc<R> &rd = runs[sgm.run];
    const long long base = (tl - sgm.first_tile) * plan->tile;
    for (int c = 0; c < plan->tile; c += blockDim.x) {
        const long long t = base + c + threadIdx.x;
        if (sgm.kind == 0)
            emf_body<0, MK, R>(rd.g, rd.A, t, lsm);
        else if (sgm.kind == 1)
            emf_body<1, MK, R>(rd.g, rd.A, t, lsm);
        else
            emf_body<2, MK, R>(rd.g, rd.A, t, lsm);
    }
}

template <int MK, typename R>
__global__ void __launch_bounds__(128) k_bphase_update(const RunDesc<R> *__restrict__ runs, const BatchPlan *__restrict__ plan,
                                                       Phys ph, int stage)
{
    const long long tl = blockIdx.x;
    const Segment sgm = plan->seg[PH_UPDATE][find_segment(plan, PH_UPDATE, tl)];
    const RunDesc<R> &rd = runs[sgm.run];
    const long long base = (tl - sgm.first_tile) * plan->tile;
    for (int c = 0; c < plan->tile; c += blockDim.x)
        update_body<MK, R>(rd.g, ph, rd.A, stage, nullptr, base + c + threadIdx.x);
}

// per-run scalars: at the start of a step (rate reset, fixed dt) and after
// the first c2p (CFL dt)
template <typename R>
__global__ void k_bphase_scalars(const RunDesc<R> *__restrict__ runs, int nruns, int what, double dt_fixed, double cfl)
{
    const int r = threadIdx.x;
    if (r >= nruns)
        return;
    DevScalars *sc = runs[r].A.scal;
    if (what == 0) {
        sc->rate_bits = 0ULL;
        sc->dt = dt_fixed > 0.0 ? dt_fixed : 0.0;
    } else {
        const double rate = __longlong_as_double((long long)sc->rate_bits);
        sc->totals[6] = rate;
        if (dt_fixed <= 0.0)
            sc->dt = rate > 0.0 ? cfl / rate : 0.0;
    }
}


// Host-side entry points of one storage type R (defined in the per-type units).
template <typename R>
const void *batch_stage_kernel(int mk, bool mlp);
// the network's Newton starts of every run (guess modes 1, 5), before a stage
template <typename R>
void batch_enqueue_guess(int mk, const void *descs, const BatchPlan *plan_dev, const BatchPlan &plan, float gr_f,
                         cudaStream_t s);
template <typename R>
void batch_enqueue_phased(int mk, bool mlp, const void *descs, const BatchPlan *plan_dev, const BatchPlan &plan,
                          int nruns, const Phys &ph, int guess, double dt, double cfl, cudaStream_t s);
template <>
void batch_enqueue_guess<double>(int mk, const void *descs, const BatchPlan *plan_dev, const BatchPlan &plan,
                                 float gr_f, cudaStream_t s);
template <>
void batch_enqueue_guess<float>(int mk, const void *descs, const BatchPlan *plan_dev, const BatchPlan &plan,
                                float gr_f, cudaStream_t s);
template <>
const void *batch_stage_kernel<double>(int mk, bool mlp);
template <>
const void *batch_stage_kernel<float>(int mk, bool mlp);
template <>
void batch_enqueue_phased<double>(int mk, bool mlp, const void *descs, const BatchPlan *plan_dev,
                                  const BatchPlan &plan, int nruns, const Phys &ph, int guess, double dt, double cfl,
                                  cudaStream_t s);
template <>
void batch_enqueue_phased<float>(int mk, bool mlp, const void *descs, const BatchPlan *plan_dev, const BatchPlan &plan,
                                 int nruns, const Phys &ph, int guess, double dt, double cfl, cudaStream_t s);

}  // namespace echo
