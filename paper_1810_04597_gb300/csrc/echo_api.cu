// echo_api.cu -- extern "C" entry points of include/echo.h.
//
// Host-side orchestration only: validation, workspace layout, and the
// order of kernel launches for c2p, L(U) and one SSP-RK3 step.  Every
// operation on the state runs in the kernels of echo_kernels.cu.
#include <climits>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/echo.h"
#include "echo_device.cuh"
#include "echo_launch.h"
#include "echo_mlp.cuh"

using namespace echo;

#include "echo_ctx.h"

namespace {

constexpr size_t ALIGN = 256;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int fail(echo_ctx *c, int code, const std::string &msg)
{
    if (c)
        c->err = msg;
    return code;
}

int cuda_check(echo_ctx *c, const char *where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(c, ECHO_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return ECHO_OK;
}

// Walk the workspace in a fixed order; with base == nullptr only sizes.
template <typename R>
size_t layout(echo_ctx *c, char *base, Arrays<R> *A)
{
    size_t off = 0;
    const size_t cells = (size_t)c->geo.cells_padded;
    auto take = [&](size_t bytes) -> char * {
        off = align_up(off, ALIGN);
        char *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    auto arr = [&]() -> R * { return reinterpret_cast<R *>(take(cells * sizeof(R))); };
    for (int q = 0; q < 8; ++q)
        A->U[q] = arr();
    for (int q = 0; q < 8; ++q)
        A->U0[q] = arr();
    for (int q = 0; q < 8; ++q)
        A->P[q] = arr();
    for (int d = 0; d < 3; ++d) {
        for (int q = 0; q < 5; ++q)
            A->F[d][q] = arr();
        A->ap[d] = arr();
        A->am[d] = arr();
        for (int q = 0; q < 4; ++q)
            A->fv[d][q] = arr();
        A->E[d] = arr();
    }
    for (int d = 0; d < 3; ++d) {
        // order 1 only: corrected fluxes and EMFs
        for (int q = 0; q < 5; ++q)
            A->Fc[d][q] = c->geo.order ? arr() : nullptr;
        for (int w = 0; w < 2; ++w)
            A->Ec[d][w] = c->geo.order ? arr() : nullptr;
    }
    A->Z = reinterpret_cast<double *>(take(cells * sizeof(double)));
    A->zg = reinterpret_cast<float *>(take(cells * sizeof(float)));
    A->ze = reinterpret_cast<unsigned char *>(take(cells));
    A->nlist = reinterpret_cast<int *>(take((size_t)(c->ntiles * 128) * sizeof(int)));
    A->gmark = c->geo.order ? reinterpret_cast<unsigned char *>(take(cells)) : nullptr;
    A->mlp = reinterpret_cast<const float *>(take(MLP_BLOCK * sizeof(float)));
    A->met = MetTables{};
    A->met.np0 = c->geo.np[0];
    A->met.use_floors = c->eos.floors;
    if (c->metric.kind == ECHO_METRIC_KERR_SCHILD) {
        const size_t plane = (size_t)c->geo.np[0] * c->geo.np[1];
        A->met.C = reinterpret_cast<MetPt *>(take(plane * sizeof(MetPt)));
        A->met.F1 = reinterpret_cast<MetPt *>(take(plane * sizeof(MetPt)));
        A->met.F2 = reinterpret_cast<MetPt *>(take(plane * sizeof(MetPt)));
        A->met.K = reinterpret_cast<MetPt *>(take(plane * sizeof(MetPt)));
        A->met.dC = reinterpret_cast<MetDer *>(take(plane * sizeof(MetDer)));
        A->met.floors = reinterpret_cast<double *>(take((size_t)c->geo.np[0] * 2 * sizeof(double)));
        if (sizeof(R) == 4) {
            A->met.Cf = reinterpret_cast<MetPtF *>(take(plane * sizeof(MetPtF)));
            A->met.F1f = reinterpret_cast<MetPtF *>(take(plane * sizeof(MetPtF)));
            A->met.F2f = reinterpret_cast<MetPtF *>(take(plane * sizeof(MetPtF)));
            A->met.Kf = reinterpret_cast<MetPtF *>(take(plane * sizeof(MetPtF)));
            A->met.dCf = reinterpret_cast<MetDerF *>(take(plane * sizeof(MetDerF)));
        }
    }
    A->stage = reinterpret_cast<double *>(take(c->staging_count * sizeof(double)));
    A->partials = reinterpret_cast<double *>(take((size_t)c->nblk_red * 6 * sizeof(double)));
    A->scal = reinterpret_cast<DevScalars *>(take(sizeof(DevScalars)));
    return align_up(off, ALIGN);
}

// Bracket one launch with two events when profiling is enabled.
struct ProfScope {
    echo_ctx *c;
    size_t slot;
    bool on;
    ProfScope(echo_ctx *cc, int kind) : c(cc), slot(0), on(cc->prof)
    {
        if (!on)
            return;
        if (c->ev_used * 2 + 2 > c->ev.size()) {
            cudaEvent_t a, b;
            if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
                on = false;
                return;
            }
            c->ev.push_back(a);
            c->ev.push_back(b);
            c->ev_kind.push_back(kind);
        }
        slot = c->ev_used++;
        c->ev_kind[slot] = kind;
        cudaEventRecord(c->ev[2 * slot], c->stream);
    }
    ~ProfScope()
    {
        if (on)
            cudaEventRecord(c->ev[2 * slot + 1], c->stream);
    }
};
#define PROF(kind, stmt)              \
    do {                              \
        ProfScope _ps(c, (kind));     \
        stmt;                         \
    } while (0)

template <typename R>
FillList<R> face_list(const Arrays<R> &A)
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
FillList<R> prim_list(const Arrays<R> &A)
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
Arrays<R> &arrays(echo_ctx *c);
template <>
Arrays<double> &arrays<double>(echo_ctx *c) { return c->ad; }
template <>
Arrays<float> &arrays<float>(echo_ctx *c) { return c->af; }

// ---- operations, templated on the storage type

// The previous-Z error codes and the network-start list of the network
// modes' per-cell choice: after a new state an exact Newton memory (from p2c,
// or a Z the caller passed) needs no network start (codes "no change", list
// empty); a cold one (no Z) lists every cell with the code of an error of
// order one.
int reset_start_memory(echo_ctx *c, bool exact, cudaStream_t s)
{
    unsigned char *ze = c->precision == 64 ? c->ad.ze : c->af.ze;
    if (cudaMemsetAsync(ze, exact ? ZE_EXACT : 0, (size_t)c->geo.cells_padded, s) != cudaSuccess)
        return cuda_check(c, "start memory");
    if (exact) {
        DevScalars *ds = c->precision == 64 ? c->ad.scal : c->af.scal;
        if (cudaMemsetAsync(&ds->nlist_count, 0, sizeof(ds->nlist_count), s) != cudaSuccess)
            return cuda_check(c, "start memory");
    } else if (c->precision == 64) {
        launch_list_all<double>(c->geo, c->ad, s);
    } else {
        launch_list_all<float>(c->geo, c->af, s);
    }
    c->ze_valid = true;
    c->ze_refine = -1;
    return cuda_check(c, "start memory");
}

// Only the network modes' inversions keep the codes up to date: before one
// of them, codes left stale by plain-mode inversions are reset to "previous
// Z exact" (the plain method's start everywhere until the next inversion
// has measured the cells again).  So are the codes of a list made under the
// other gate (with or without the FP32 refinement): a cell consults the
// network's start only if the last inversion listed it.
int prepare_start(echo_ctx *c, int mode, cudaStream_t s)
{
    if ((mode & 3) != 1) {
        c->ze_valid = false;
        return ECHO_OK;
    }
    const int rf = (mode & 4) ? 1 : 0;
    if (c->ze_valid && (c->ze_refine < 0 || c->ze_refine == rf)) {
        c->ze_refine = rf;
        return ECHO_OK;
    }
    const int rc = reset_start_memory(c, true, s);
    c->ze_refine = rf;
    return rc;
}

template <int MK, typename R>
void enqueue_rhs_pass(echo_ctx *c, int stage, double *Lout, bool want_rate, double dt_fixed)
{
    Arrays<R> &A = arrays<R>(c);
    cudaStream_t s = c->stream;
    PROF(ECHO_K_FILL_FACES, launch_fill<R>(c->geo, face_list(A), s));
    PROF(ECHO_K_NETWORK, (launch_net_pass<MK, R>(c->geo, c->ph, A, c->c2p_guess, s)));
    PROF(ECHO_K_C2P, (launch_c2p<MK, R>(c->geo, c->ph, A, c->c2p_guess, want_rate ? 1 : 0, s)));
    if (want_rate)
        PROF(ECHO_K_SCALARS, launch_set_dt(A.scal, c->cfl, dt_fixed <= 0.0 ? 1 : 0, s));
    PROF(ECHO_K_FILL_PRIMS, launch_fill<R>(c->geo, prim_list(A), s));
    for (int d = 0; d < 3; ++d)
        PROF(ECHO_K_FACES_X + d, (launch_faces<MK, R>(c->geo, c->ph, A, d, s)));
    for (int e = 0; e < 3; ++e)
        PROF(ECHO_K_EMF_X + e, (launch_emf<MK, R>(c->geo, A, e, s)));
    if (c->geo.order) {
        PROF(ECHO_K_CORRECT, launch_correct<R>(c->geo, A, s));
        if (stage >= 0)
            PROF(ECHO_K_CORRECT, (launch_guard<MK, R>(c->geo, c->ph, A, stage, s)));
    }
    PROF(ECHO_K_UPDATE, (launch_update<MK, R>(c->geo, c->ph, A, stage, Lout, s)));
}

template <int MK, typename R>
int op_step(echo_ctx *c, double dt)
{
    Arrays<R> &A = arrays<R>(c);
    if (const int rc = prepare_start(c, c->c2p_guess, c->stream))
        return rc;
    PROF(ECHO_K_SCALARS, launch_step_begin(A.scal, dt > 0.0 ? dt : 0.0, c->stream));
    for (int st = 0; st < 3; ++st)
        enqueue_rhs_pass<MK, R>(c, st, nullptr, st == 0, dt);
    return cuda_check(c, "echo_step");
}

template <int MK, typename R>
int op_rhs(echo_ctx *c, double *Lout)
{
    Arrays<R> &A = arrays<R>(c);
    if (const int rc = prepare_start(c, c->c2p_guess, c->stream))
        return rc;
    launch_step_begin(A.scal, 0.0, c->stream);
    enqueue_rhs_pass<MK, R>(c, -1, Lout, true, 0.0);
    return cuda_check(c, "echo_rhs");
}

template <int MK, typename R>
int op_c2p(echo_ctx *c, int guess_mode)
{
    Arrays<R> &A = arrays<R>(c);
    if (const int rc = prepare_start(c, guess_mode, c->stream))
        return rc;
    PROF(ECHO_K_SCALARS, launch_step_begin(A.scal, 0.0, c->stream));
    PROF(ECHO_K_FILL_FACES, launch_fill<R>(c->geo, face_list(A), c->stream));
    PROF(ECHO_K_NETWORK, (launch_net_pass<MK, R>(c->geo, c->ph, A, guess_mode, c->stream)));
    PROF(ECHO_K_C2P, (launch_c2p<MK, R>(c->geo, c->ph, A, guess_mode, 1, c->stream)));
    PROF(ECHO_K_SCALARS, launch_set_dt(A.scal, c->cfl, 1, c->stream));
    return cuda_check(c, "echo_c2p");
}

// Dispatch an operation template on (metric kind, storage type).
#define ECHO_DISPATCH(c, fn, ...)                                                               \
    ((c)->metric.kind == ECHO_METRIC_KERR_SCHILD                                                \
         ? ((c)->precision == 64 ? fn<1, double>((c), __VA_ARGS__) : fn<1, float>((c), __VA_ARGS__)) \
         : ((c)->precision == 64 ? fn<0, double>((c), __VA_ARGS__) : fn<0, float>((c), __VA_ARGS__)))

int read_scalars(echo_ctx *c, DevScalars *hs)
{
    DevScalars *ds = c->precision == 64 ? c->ad.scal : c->af.scal;
    if (cudaMemcpyAsync(hs, ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return cuda_check(c, "read scalars");
    if (cudaStreamSynchronize(c->stream) != cudaSuccess)
        return cuda_check(c, "synchronize");
    return ECHO_OK;
}

// Guess modes: 0 previous Z, 1 network, 2 cold; +4 FP32 refinement; for the
// network +8 (FP32 on the CUDA cores) or +16 (tensor cores inside the c2p
// kernel) -- not both.
bool valid_guess(int mode)
{
    if (mode < 0 || mode > 31 || (mode & 3) == 3)
        return false;
    if ((mode & 24) && (mode & 3) != 1)
        return false;
    return (mode & 24) != 24;
}

const char *const kGuessModes =
    "guess mode: 0 previous Z, 1 network, 2 cold; +4 FP32 refinement; for the network +8 on the CUDA cores or +16 "
    "inside the c2p kernel";

int require_bound(echo_ctx *c, bool need_state)
{
    if (!c)
        return ECHO_EINVAL;
    if (!c->bound)
        return fail(c, ECHO_ESTATE, "context has no workspace: call echo_bind first");
    if (need_state && !c->have_state)
        return fail(c, ECHO_ESTATE, "no state: call echo_set_prims or echo_set_state first");
    return ECHO_OK;
}

}  // namespace

extern "C" {

int echo_init(const echo_grid *grid, const echo_metric *metric, const echo_eos *eos, int precision, double cfl,
              echo_ctx **out)
{
    if (!out)
        return ECHO_EINVAL;
    *out = nullptr;
    if (!grid || !metric || !eos)
        return ECHO_EINVAL;
    for (int d = 0; d < 3; ++d) {
        if (grid->n[d] < 1 || !(grid->dx[d] > 0.0))
            return ECHO_EINVAL;
        const int lo = grid->bc[2 * d], hi = grid->bc[2 * d + 1];
        if (lo < 0 || lo > 2 || hi < 0 || hi > 2)
            return ECHO_EINVAL;
        if ((lo == ECHO_BC_PERIODIC) != (hi == ECHO_BC_PERIODIC))
            return ECHO_EINVAL;
        if ((lo == ECHO_BC_AXIS || hi == ECHO_BC_AXIS) && grid->n[d] < NG)
            return ECHO_EINVAL;
    }
    if (metric->kind != ECHO_METRIC_FLAT && metric->kind != ECHO_METRIC_KERR_SCHILD)
        return ECHO_EINVAL;
    if (metric->kind == ECHO_METRIC_KERR_SCHILD && !(metric->spin >= 0.0 && metric->spin < 1.0))
        return ECHO_EINVAL;
    if (!(eos->gamma > 1.0) || !(cfl > 0.0) || (precision != 64 && precision != 32))
        return ECHO_EINVAL;
    // padded cells (n + 2 NG per axis, x rounded up to 8) below 2^31: the
    // kernels index every array with 32-bit offsets
    {
        long long padded = (long long)align_up((size_t)grid->n[0] + 2 * NG, 8);
        for (int d = 1; d < 3 && padded <= INT_MAX; ++d)
            padded *= (long long)grid->n[d] + 2 * NG;
        if (padded > INT_MAX)
            return ECHO_EINVAL;
    }

    echo_ctx *c = new (std::nothrow) echo_ctx();
    if (!c)
        return ECHO_ENOMEM;
    c->grid = *grid;
    c->metric = *metric;
    c->eos = *eos;
    c->precision = precision;
    c->cfl = cfl;
    Geom &g = c->geo;
    for (int d = 0; d < 3; ++d) {
        g.n[d] = grid->n[d];
        g.np[d] = grid->n[d] + 2 * NG;
        g.dx[d] = grid->dx[d];
        g.idx[d] = 1.0 / grid->dx[d];
        g.x0[d] = grid->x0[d];
        g.bc[2 * d] = grid->bc[2 * d];
        g.bc[2 * d + 1] = grid->bc[2 * d + 1];
        const bool per = grid->bc[2 * d] == ECHO_BC_PERIODIC;
        g.flo[d] = NG + (grid->bc[2 * d] == ECHO_BC_AXIS ? 1 : 0);
        g.fhi[d] = per ? NG + g.n[d] - 1 : NG + g.n[d] - (grid->bc[2 * d + 1] == ECHO_BC_AXIS ? 1 : 0);
    }
    g.px = (int)align_up((size_t)g.np[0], 8);
    g.pxy = g.px * g.np[1];
    g.cells_padded = (long long)g.pxy * g.np[2];
    c->ph.gamma = eos->gamma;
    c->ph.gr = eos->gamma / (eos->gamma - 1.0);
    c->ph.gm1g = (eos->gamma - 1.0) / eos->gamma;
    c->ph.cfl = cfl;
    c->ph.gamma_f = (float)c->ph.gamma;
    c->ph.gr_f = (float)c->ph.gr;
    for (int d = 0; d < 3; ++d)
        g.idx_f[d] = (float)g.idx[d];
    const size_t N = (size_t)grid->n[0] * grid->n[1] * grid->n[2];
    c->ntiles = (long long)((N + 127) / 128);
    c->nstate = 5 * N + (size_t)g.n[2] * g.n[1] * (g.n[0] + 1) + (size_t)g.n[2] * (g.n[1] + 1) * g.n[0]
                + (size_t)(g.n[2] + 1) * g.n[1] * g.n[0];
    c->staging_count = c->nstate > 8 * N ? c->nstate : 8 * N;
    c->nblk_red = 152 * 4;
    if (precision == 64)
        c->ws_need = layout<double>(c, nullptr, &c->ad);
    else
        c->ws_need = layout<float>(c, nullptr, &c->af);
    *out = c;
    return ECHO_OK;
}

int echo_set_order(echo_ctx *c, int order)
{
    if (!c)
        return ECHO_EINVAL;
    if (order != 0 && order != 1)
        return fail(c, ECHO_EINVAL, "order: 0 the scheme as read, 1 high order");
    if (c->bound)
        return fail(c, ECHO_ESTATE, "set the order before echo_bind");
    c->geo.order = order;
    if (c->precision == 64)
        c->ws_need = layout<double>(c, nullptr, &c->ad);
    else
        c->ws_need = layout<float>(c, nullptr, &c->af);
    return ECHO_OK;
}

size_t echo_workspace_bytes(const echo_ctx *c) { return c ? c->ws_need : 0; }

size_t echo_state_count(const echo_ctx *c) { return c ? c->nstate : 0; }

int echo_bind(echo_ctx *c, void *ws, size_t bytes, void *stream)
{
    if (!c)
        return ECHO_EINVAL;
    if (!ws || ((uintptr_t)ws % ALIGN) != 0)
        return fail(c, ECHO_EINVAL, "workspace must be a non-null 256-byte aligned device pointer");
    if (bytes < c->ws_need)
        return fail(c, ECHO_ENOMEM, "workspace smaller than echo_workspace_bytes");
    c->ws = static_cast<char *>(ws);
    c->stream = static_cast<cudaStream_t>(stream);
    if (c->precision == 64)
        layout<double>(c, c->ws, &c->ad);
    else
        layout<float>(c, c->ws, &c->af);
    if (cudaMemsetAsync(c->ws, 0, c->ws_need, c->stream) != cudaSuccess)
        return cuda_check(c, "echo_bind memset");
    if (c->metric.kind == ECHO_METRIC_KERR_SCHILD) {
        const MetTables &T = c->precision == 64 ? c->ad.met : c->af.met;
        launch_metric_tables(c->geo, c->metric.spin, T, c->eos.rho_floor, c->eos.rho_floor_pow, c->eos.p_floor,
                             c->eos.p_floor_pow, c->stream);
    }
    c->bound = true;
    c->have_state = false;
    return cuda_check(c, "echo_bind");
}

// Device address of page-locked host memory mapped into the device's
// address space, or null if p is not such memory.
static void *mapped_host(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

static const double *stage_input(echo_ctx *c, const double *src, size_t count, size_t at, int on_device,
                                 int *rc)
{
    *rc = ECHO_OK;
    if (on_device < 0 || on_device > 2) {
        *rc = fail(c, ECHO_EINVAL, "on_device: 0 host (staged), 1 device, 2 mapped page-locked host memory");
        return nullptr;
    }
    if (on_device == 1)
        return src;
    if (on_device == 2) {
        const double *d = static_cast<const double *>(mapped_host(src));
        if (!d)
            *rc = fail(c, ECHO_EINVAL, "on_device = 2 needs page-locked host memory mapped into the device");
        return d;
    }
    double *st = (c->precision == 64 ? c->ad.stage : c->af.stage) + at;
    if (cudaMemcpyAsync(st, src, count * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        *rc = cuda_check(c, "host to device copy");
    return st;
}

int echo_set_prims(echo_ctx *c, const double *prims5, const double *bface, int on_device)
{
    int rc = require_bound(c, false);
    if (rc)
        return rc;
    if (!prims5 || !bface)
        return fail(c, ECHO_EINVAL, "null pointer");
    const size_t N = (size_t)c->geo.n[0] * c->geo.n[1] * c->geo.n[2];
    const double *dp = stage_input(c, prims5, 5 * N, 0, on_device, &rc);
    if (rc)
        return rc;
    const double *df = stage_input(c, bface, c->nstate - 5 * N, 5 * N, on_device, &rc);
    if (rc)
        return rc;
    const bool ks = c->metric.kind == ECHO_METRIC_KERR_SCHILD;
    if (c->precision == 64) {
        launch_unpack_state<double>(c->geo, df, c->ad, 1, c->stream);
        launch_fill<double>(c->geo, face_list(c->ad), c->stream);
        if (ks)
            launch_p2c<1, double>(c->geo, c->ph, dp, c->ad, c->stream);
        else
            launch_p2c<0, double>(c->geo, c->ph, dp, c->ad, c->stream);
    } else {
        launch_unpack_state<float>(c->geo, df, c->af, 1, c->stream);
        launch_fill<float>(c->geo, face_list(c->af), c->stream);
        if (ks)
            launch_p2c<1, float>(c->geo, c->ph, dp, c->af, c->stream);
        else
            launch_p2c<0, float>(c->geo, c->ph, dp, c->af, c->stream);
    }
    rc = cuda_check(c, "echo_set_prims");
    if (rc == ECHO_OK)
        rc = reset_start_memory(c, true, c->stream);
    if (rc == ECHO_OK)
        c->have_state = true;
    return rc;
}

int echo_set_state(echo_ctx *c, const double *state, const double *Z, int on_device)
{
    int rc = require_bound(c, false);
    if (rc)
        return rc;
    if (!state)
        return fail(c, ECHO_EINVAL, "null state");
    const size_t N = (size_t)c->geo.n[0] * c->geo.n[1] * c->geo.n[2];
    const double *ds = stage_input(c, state, c->nstate, 0, on_device, &rc);
    if (rc)
        return rc;
    if (c->precision == 64)
        launch_unpack_state<double>(c->geo, ds, c->ad, 0, c->stream);
    else
        launch_unpack_state<float>(c->geo, ds, c->af, 0, c->stream);
    const double *dz = nullptr;
    if (Z) {
        // the staging area is free again once the unpack above has run
        dz = stage_input(c, Z, N, 0, on_device, &rc);
        if (rc)
            return rc;
    }
    if (c->precision == 64)
        launch_unpack_z<double>(c->geo, dz, c->ad, c->stream);
    else
        launch_unpack_z<float>(c->geo, dz, c->af, c->stream);
    rc = cuda_check(c, "echo_set_state");
    if (rc == ECHO_OK)
        rc = reset_start_memory(c, Z != nullptr, c->stream);
    if (rc == ECHO_OK)
        c->have_state = true;
    return rc;
}

// Where an output is written: the caller's device pointer (1), its mapped
// host memory (2), or the staging area copied out afterwards (0).
static double *output_target(echo_ctx *c, double *out, int on_device, int *rc)
{
    *rc = ECHO_OK;
    if (on_device < 0 || on_device > 2) {
        *rc = fail(c, ECHO_EINVAL, "on_device: 0 host (staged), 1 device, 2 mapped page-locked host memory");
        return nullptr;
    }
    if (on_device == 1)
        return out;
    if (on_device == 2) {
        double *d = static_cast<double *>(mapped_host(out));
        if (!d)
            *rc = fail(c, ECHO_EINVAL, "on_device = 2 needs page-locked host memory mapped into the device");
        return d;
    }
    return c->precision == 64 ? c->ad.stage : c->af.stage;
}

static int finish_output(echo_ctx *c, double *dst, const double *staged, size_t count, int on_device)
{
    if (on_device == 0) {
        if (cudaMemcpyAsync(dst, staged, count * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
            return cuda_check(c, "device to host copy");
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess)
        return cuda_check(c, "synchronize");
    return cuda_check(c, "output");
}

int echo_get_state(echo_ctx *c, double *out, int on_device)
{
    int rc = require_bound(c, true);
    if (rc)
        return rc;
    if (!out)
        return fail(c, ECHO_EINVAL, "null output");
    double *dst = output_target(c, out, on_device, &rc);
    if (rc)
        return rc;
    if (c->precision == 64) {
        launch_fill<double>(c->geo, face_list(c->ad), c->stream);
        launch_pack_state<double>(c->geo, c->ad, dst, c->stream);
    } else {
        launch_fill<float>(c->geo, face_list(c->af), c->stream);
        launch_pack_state<float>(c->geo, c->af, dst, c->stream);
    }
    return finish_output(c, out, dst, c->nstate, on_device);
}

int echo_get_prims(echo_ctx *c, double *out, int on_device)
{
    int rc = require_bound(c, true);
    if (rc)
        return rc;
    if (!out)
        return fail(c, ECHO_EINVAL, "null output");
    const size_t N = (size_t)c->geo.n[0] * c->geo.n[1] * c->geo.n[2];
    double *dst = output_target(c, out, on_device, &rc);
    if (rc)
        return rc;
    if (c->precision == 64)
        launch_pack_cells<double>(c->geo, c->ad, dst, 0, c->stream);
    else
        launch_pack_cells<float>(c->geo, c->af, dst, 0, c->stream);
    return finish_output(c, out, dst, 8 * N, on_device);
}

int echo_get_z(echo_ctx *c, double *out, int on_device)
{
    int rc = require_bound(c, true);
    if (rc)
        return rc;
    if (!out)
        return fail(c, ECHO_EINVAL, "null output");
    const size_t N = (size_t)c->geo.n[0] * c->geo.n[1] * c->geo.n[2];
    double *dst = output_target(c, out, on_device, &rc);
    if (rc)
        return rc;
    if (c->precision == 64)
        launch_pack_cells<double>(c->geo, c->ad, dst, 1, c->stream);
    else
        launch_pack_cells<float>(c->geo, c->af, dst, 1, c->stream);
    return finish_output(c, out, dst, N, on_device);
}

int echo_c2p(echo_ctx *c, int guess_mode, echo_totals *stats)
{
    int rc = require_bound(c, true);
    if (rc)
        return rc;
    if (!valid_guess(guess_mode))
        return fail(c, ECHO_EINVAL, kGuessModes);
    if ((guess_mode & 3) == 1 && !c->mlp_loaded)
        return fail(c, ECHO_ESTATE, "no c2p-guess network loaded: call echo_mlp_load first");
    rc = ECHO_DISPATCH(c, op_c2p, guess_mode);
    if (rc || !stats)
        return rc;
    DevScalars hs;
    rc = read_scalars(c, &hs);
    if (rc)
        return rc;
    stats->dt_cfl = hs.dt;
    stats->c2p_iters = (long long)hs.c2p_iters;
    stats->c2p_calls = (long long)hs.c2p_calls;
    stats->c2p_fail = (long long)hs.c2p_fail;
    stats->floor_hits = (long long)hs.floor_hits;
    stats->mlp_fallback = (long long)hs.mlp_fallback;
    stats->mlp_used = (long long)hs.mlp_used;
    for (int k = 0; k < ECHO_C2P_HIST; ++k)
        stats->c2p_iter_hist[k] = (long long)hs.c2p_hist[k];
    if (hs.fail_since_check) {
        DevScalars *ds = c->precision == 64 ? c->ad.scal : c->af.scal;
        cudaMemsetAsync(&ds->fail_since_check, 0, sizeof(unsigned long long), c->stream);
        if (!c->eos.floors)
            return fail(c, ECHO_EC2P, "conservative-to-primitive inversion failed in some cells");
    }
    return ECHO_OK;
}

int echo_rhs(echo_ctx *c, double *L, int on_device)
{
    int rc = require_bound(c, true);
    if (rc)
        return rc;
    if (!L)
        return fail(c, ECHO_EINVAL, "null output");
    double *dst = output_target(c, L, on_device, &rc);
    if (rc)
        return rc;
    rc = ECHO_DISPATCH(c, op_rhs, dst);
    if (rc)
        return rc;
    if (on_device != 1)
        return finish_output(c, L, dst, c->nstate, on_device);
    return ECHO_OK;
}

int echo_step(echo_ctx *c, double dt)
{
    int rc = require_bound(c, true);
    if (rc)
        return rc;
    return ECHO_DISPATCH(c, op_step, dt);
}

int echo_internal_prepare_start(echo_ctx *c, int mode, cudaStream_t s) { return prepare_start(c, mode, s); }

// Enqueue one step of context c on another stream (used by the run-major
// batch schedule); per-kernel timing is off while the batch records.
int echo_internal_enqueue_step(echo_ctx *c, double dt, cudaStream_t s)
{
    cudaStream_t own = c->stream;
    const bool prof = c->prof;
    c->stream = s;
    c->prof = false;
    const int rc = ECHO_DISPATCH(c, op_step, dt);
    c->stream = own;
    c->prof = prof;
    return rc;
}

int echo_reduce(echo_ctx *c, echo_totals *out)
{
    int rc = require_bound(c, true);
    if (rc)
        return rc;
    if (!out)
        return fail(c, ECHO_EINVAL, "null output");
    rc = ECHO_DISPATCH(c, op_c2p, 0);
    if (rc)
        return rc;
    if (c->precision == 64)
        PROF(ECHO_K_TOTALS, launch_totals<double>(c->geo, c->ad, c->nblk_red, c->stream));
    else
        PROF(ECHO_K_TOTALS, launch_totals<float>(c->geo, c->af, c->nblk_red, c->stream));
    rc = cuda_check(c, "echo_reduce");
    if (rc)
        return rc;
    DevScalars hs;
    rc = read_scalars(c, &hs);
    if (rc)
        return rc;
    out->dt_cfl = hs.dt;
    out->mass = hs.totals[0];
    out->energy = hs.totals[1];
    out->mom[0] = hs.totals[2];
    out->mom[1] = hs.totals[3];
    out->mom[2] = hs.totals[4];
    out->max_divb = hs.totals[5];
    out->c2p_iters = (long long)hs.c2p_iters;
    out->c2p_calls = (long long)hs.c2p_calls;
    out->c2p_fail = (long long)hs.c2p_fail;
    out->floor_hits = (long long)hs.floor_hits;
    out->fallback_faces = (long long)hs.fallback_faces;
    out->mlp_fallback = (long long)hs.mlp_fallback;
    out->mlp_used = (long long)hs.mlp_used;
    out->guard_faces = (long long)hs.guard_faces;
    for (int k = 0; k < ECHO_C2P_HIST; ++k)
        out->c2p_iter_hist[k] = (long long)hs.c2p_hist[k];
    if (hs.fail_since_check) {
        DevScalars *ds = c->precision == 64 ? c->ad.scal : c->af.scal;
        cudaMemsetAsync(&ds->fail_since_check, 0, sizeof(unsigned long long), c->stream);
        if (!c->eos.floors)
            return fail(c, ECHO_EC2P, "conservative-to-primitive inversion failed in some cells");
    }
    return ECHO_OK;
}

int echo_counters(echo_ctx *c, echo_totals *out)
{
    int rc = require_bound(c, false);
    if (rc)
        return rc;
    if (!out)
        return fail(c, ECHO_EINVAL, "null output");
    DevScalars hs;
    rc = read_scalars(c, &hs);
    if (rc)
        return rc;
    out->c2p_iters = (long long)hs.c2p_iters;
    out->c2p_calls = (long long)hs.c2p_calls;
    out->c2p_fail = (long long)hs.c2p_fail;
    out->floor_hits = (long long)hs.floor_hits;
    out->mlp_fallback = (long long)hs.mlp_fallback;
    out->mlp_used = (long long)hs.mlp_used;
    out->guard_faces = (long long)hs.guard_faces;
    out->fallback_faces = (long long)hs.fallback_faces;
    for (int k = 0; k < ECHO_C2P_HIST; ++k)
        out->c2p_iter_hist[k] = (long long)hs.c2p_hist[k];
    return ECHO_OK;
}

int echo_mlp_load(echo_ctx *c, const float *dev_state)
{
    int rc = require_bound(c, false);
    if (rc)
        return rc;
    if (!dev_state)
        return fail(c, ECHO_EINVAL, "null network block");
    float *dst = const_cast<float *>(c->precision == 64 ? c->ad.mlp : c->af.mlp);
    if (cudaMemcpyAsync(dst, dev_state, MLP_BLOCK * sizeof(float), cudaMemcpyDeviceToDevice, c->stream)
        != cudaSuccess)
        return cuda_check(c, "echo_mlp_load");
    // no Newton start of an earlier network survives: a cell the next
    // inversion consults under this network's gate, but that the list (made
    // under the old gate) did not hold, starts from its previous Z
    float *zg = c->precision == 64 ? c->ad.zg : c->af.zg;
    if (cudaMemsetAsync(zg, 0, (size_t)c->geo.cells_padded * sizeof(float), c->stream) != cudaSuccess)
        return cuda_check(c, "echo_mlp_load");
    c->mlp_loaded = true;
    return cuda_check(c, "echo_mlp_load");
}

int echo_set_c2p_guess(echo_ctx *c, int mode)
{
    if (!c)
        return ECHO_EINVAL;
    if (!valid_guess(mode))
        return fail(c, ECHO_EINVAL, kGuessModes);
    if ((mode & 3) == 1 && !c->mlp_loaded)
        return fail(c, ECHO_ESTATE, "no c2p-guess network loaded: call echo_mlp_load first");
    c->c2p_guess = mode;
    return ECHO_OK;
}

int echo_mlp_dataset(echo_ctx *c, float *X, float *Y, long long capacity, long long offset, long long stride)
{
    int rc = require_bound(c, true);
    if (rc)
        return rc;
    const long long N = (long long)c->geo.n[0] * c->geo.n[1] * c->geo.n[2];
    if (!X || !Y || offset < 0 || stride < 1 || offset + (N - 1) * stride >= capacity)
        return fail(c, ECHO_EINVAL, "dataset rows offset + (cells - 1) * stride must lie below capacity");
    rc = ECHO_DISPATCH(c, op_c2p, 0);
    if (rc)
        return rc;
    const bool ks = c->metric.kind == ECHO_METRIC_KERR_SCHILD;
    if (c->precision == 64) {
        if (ks)
            launch_mlp_dataset<1, double>(c->geo, c->ad, X, Y, offset, stride, c->stream);
        else
            launch_mlp_dataset<0, double>(c->geo, c->ad, X, Y, offset, stride, c->stream);
    } else {
        if (ks)
            launch_mlp_dataset<1, float>(c->geo, c->af, X, Y, offset, stride, c->stream);
        else
            launch_mlp_dataset<0, float>(c->geo, c->af, X, Y, offset, stride, c->stream);
    }
    return cuda_check(c, "echo_mlp_dataset");
}

int echo_profile(echo_ctx *c, int enable)
{
    if (!c)
        return ECHO_EINVAL;
    c->prof = enable != 0;
    return ECHO_OK;
}

int echo_profile_read(echo_ctx *c, double *ms, long long *launches, int nk)
{
    if (!c || !ms || !launches || nk < 0)
        return ECHO_EINVAL;
    for (int k = 0; k < nk; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    if (c->ev_used && cudaStreamSynchronize(c->stream) != cudaSuccess)
        return cuda_check(c, "echo_profile_read");
    for (size_t p = 0; p < c->ev_used; ++p) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, c->ev[2 * p], c->ev[2 * p + 1]) != cudaSuccess)
            return cuda_check(c, "echo_profile_read elapsed");
        const int k = c->ev_kind[p];
        if (k >= 0 && k < nk) {
            ms[k] += (double)t;
            launches[k] += 1;
        }
    }
    c->ev_used = 0;
    return ECHO_OK;
}

const char *echo_kernel_name(int k)
{
    static const char *names[ECHO_NK] = {"fill_faces", "c2p", "fill_prims", "faces_x", "faces_y", "faces_z",
                                         "emf_x", "emf_y", "emf_z", "update", "scalars", "totals", "correct",
                                         "network"};
    return (k >= 0 && k < ECHO_NK) ? names[k] : "";
}

const char *echo_last_error(const echo_ctx *c) { return c ? c->err.c_str() : "null context"; }

void echo_destroy(echo_ctx *c)
{
    if (!c)
        return;
    for (cudaEvent_t e : c->ev)
        cudaEventDestroy(e);
    delete c;
}

}  // extern "C"
