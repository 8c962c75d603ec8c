/*
 * echo.h -- C ABI of the GB300 library for the per-step update of the 3-D
 * finite-difference GRMHD scheme (ECHO-3DHPC method) on a fixed metric.
 *
 * The paper (introduction) describes ECHO-3DHPC as a code that solves the
 * equations of general-relativistic MHD with a 3-D finite-difference method
 * and high-order reconstruction; it prints no equation.  The update this
 * library computes restates published methods:
 *   conservative-to-primitive inversion by Newton iteration on Z = rho h W^2;
 *   MP5 reconstruction of primitives (Suresh & Huynh 1997);
 *   HLL fluxes with the approximate fast speed of the ECHO family;
 *   upwind constrained-transport (UCT-HLL) edge EMFs (Londrillo & Del Zanna
 *   2004);
 *   flux difference plus geometric sources of the 3+1 Valencia form, and the
 *   three-stage SSP Runge-Kutta scheme (Shu & Osher 1988).
 *
 * Conventions
 *   - Every entry point returns ECHO_OK (0) or a negative ECHO_E* code; the
 *     message of the last failure is echo_last_error(ctx).  No exception
 *     crosses the ABI.
 *   - The library never allocates device memory: the caller allocates the
 *     workspace (echo_workspace_bytes) and passes it to echo_bind together
 *     with a CUDA stream.  All work is enqueued on that stream.  Pointers
 *     stay owned by the caller.
 *   - Only echo_get_state, echo_get_prims, echo_c2p (with stats) and
 *     echo_reduce synchronise the bound stream.
 *   - Host-layout arrays are FP64 regardless of the internal precision.
 *     A state holds five cell arrays (D, S_x, S_y, S_z, tau), densitised by
 *     sqrt(gamma), each nz*ny*nx with x fastest, followed by the face field
 *     B~ = sqrt(gamma) B as Bx (nz, ny, nx+1), By (nz, ny+1, nx),
 *     Bz (nz+1, ny, nx), face i-1/2 at index i.  On a periodic axis the last
 *     face repeats the first (read: ignored; written: duplicated).
 *   - A pointer argument flagged "on_device" is a device pointer when the
 *     flag is 1; a host pointer copied through the library's staging area
 *     when it is 0; and, when it is 2, a host pointer into page-locked host
 *     memory mapped into the device's address space (cudaHostAlloc, torch
 *     pin_memory), which the library's kernels read or write directly over
 *     the host link with no staging copy -- the library checks the mapping
 *     with cudaPointerGetAttributes (ECHO_EINVAL if the memory is not
 *     mapped page-locked memory) but not the buffer's length, which must be
 *     the documented one.  A host input buffer must stay unchanged until the
 *     next synchronising call.  Other flag values: ECHO_EINVAL.
 */
#ifndef ECHO_H
#define ECHO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ECHO_OK 0
#define ECHO_EINVAL (-1)   /* bad argument or configuration */
#define ECHO_ECUDA (-2)    /* a CUDA runtime call or kernel launch failed */
#define ECHO_ENOMEM (-3)   /* workspace smaller than echo_workspace_bytes */
#define ECHO_EC2P (-4)     /* conservative-to-primitive inversion failed */
#define ECHO_ETIMEOUT (-5) /* a bounded device wait gave up */
#define ECHO_ESTATE (-6)   /* call out of order (e.g. not bound, no state) */
#define ECHO_ERANGE (-7)   /* size beyond a fixed maximum (echo_totals_static) */

/* boundary kinds (echo_grid.bc[2*d + side], side 0 lower, 1 upper) */
#define ECHO_BC_PERIODIC 0
#define ECHO_BC_OUTFLOW 1
#define ECHO_BC_AXIS 2

/* metric kinds */
#define ECHO_METRIC_FLAT 0
#define ECHO_METRIC_KERR_SCHILD 1 /* coordinates (ln r, theta, phi), M = 1 */

/* buckets of the Newton-iteration histogram in echo_totals */
#define ECHO_C2P_HIST 16

typedef struct echo_ctx echo_ctx; /* opaque, library-owned host object */

typedef struct {
    int n[3];      /* interior cells along x1, x2, x3 (each >= 1) */
    double x0[3];  /* coordinate of the lower face of the domain */
    double dx[3];  /* cell widths (> 0) */
    int bc[6];     /* ECHO_BC_* per axis and side */
} echo_grid;

typedef struct {
    int kind;      /* ECHO_METRIC_* */
    double spin;   /* a/M for Kerr-Schild */
} echo_metric;

typedef struct {
    double gamma;  /* ideal-gas adiabatic index, > 1 */
    int floors;    /* 1: atmosphere floors after c2p, failures fall back */
    double rho_floor, rho_floor_pow, p_floor, p_floor_pow; /* floor = f0 r^pow */
} echo_eos;

typedef struct {
    double dt_cfl;        /* CFL time step of the current state */
    double mass;          /* sum sqrt(g) D dV */
    double energy;        /* sum sqrt(g) tau dV */
    double mom[3];        /* sum sqrt(g) S_i dV */
    double max_divb;      /* max over cells |sum_d dB~^d / dx^d| */
    long long c2p_iters;  /* Newton iterations since bind (cumulative) */
    long long c2p_calls;  /* cell inversions since bind */
    long long c2p_fail;   /* failed inversions since bind */
    long long floor_hits; /* cells reset by floors since bind */
    long long fallback_faces; /* reconstructed face sides replaced by their cell
                               * (rho <= 0, p <= 0 or v^2 >= 1) since bind, on
                               * the faces that bound owned cells, each once */
    long long mlp_fallback;   /* network guesses that needed the previous-Z restart */
    /* cell inversions since bind by their Newton iterations: [k] took k
     * iterations (network attempt and restart together), [ECHO_C2P_HIST - 1]
     * that many or more; the entries sum to c2p_calls */
    long long c2p_iter_hist[ECHO_C2P_HIST];
    long long mlp_used;   /* inversions since bind started from the network's Newton start */
    long long guard_faces; /* order 1: faces the safeguard returned to the uncorrected flux since bind */
} echo_totals;

/* Method: the grid and equations of the paper's solver (introduction: a 3-D
 * finite-difference GRMHD code), read as the 3+1 Valencia form of ideal
 * GRMHD on a stationary metric (Banyuls et al. 1997; Del Zanna et al. 2007).
 * Create a context.  precision: 64 (FP64 everywhere) or 32 (FP32 storage
 * and stencil arithmetic; c2p, metric and reductions in FP64).  cfl: the
 * Courant number of the CFL time step.  Validates the configuration;
 * returns ECHO_EINVAL (and *out = NULL) on a bad one, and also when the
 * padded grid (n + 10 cells per axis, x rounded up to a multiple of 8) has
 * 2^31 cells or more: the kernels index each array with 32-bit offsets
 * (the limit is near 1278^3 cells, where the workspace of either
 * precision is already larger than the 288 GB of one GPU). */
int echo_init(const echo_grid *grid, const echo_metric *metric, const echo_eos *eos, int precision,
              double cfl, echo_ctx **out);

/* Method: the paper's "high-order reconstruction" (introduction), read as the
 * point-value finite-difference form with a flux-derivative correction
 * (Del Zanna et al. 2007).
 * Scheme order, before echo_bind (it changes the workspace size):
 * 0 (default) the scheme as read -- MP5 with the fifth-order interpolant of
 * cell averages on the point values, cell-centre B the mean of the two
 * faces, HLL fluxes and UCT EMFs differenced as they are; 1 high order --
 * MP5 with the fifth-order interpolant of point values, cell-centre B by
 * sixth-order interpolation of six faces, and the flux-derivative
 * correction F - D2/24 + 3 D4/640 (second and fourth differences of
 * neighbouring interface values) of every flux along its direction and of
 * every EMF along each of its two half-integer directions, so that the
 * differences are sixth-order derivatives (the scheme's "high-order"
 * finite differences).  With order 1 the divergence that stays constant is
 * the one built from corrected face differences (echo_reduce reports it).
 * Order 1 also runs a safeguard in every stage of echo_step: a cell whose
 * stage result (formed from L(U) with the corrected fluxes as the stage
 * forms it, with the current cell-centre field) the FP64 Newton inversion
 * cannot invert is flagged, every face of a flagged cell takes the
 * uncorrected flux (the same for both cells sharing it), and the check
 * repeats on the cells not yet flagged, three passes at most; the faces it
 * changed are counted (echo_totals.guard_faces).  echo_rhs has no step and
 * no safeguard.
 * ECHO_EINVAL for another value, ECHO_ESTATE after echo_bind. */
int echo_set_order(echo_ctx *ctx, int order);

/* Bytes of device workspace the context needs (all arrays, with 5 ghost
 * layers per side, plus staging and reduction scratch). */
size_t echo_workspace_bytes(const echo_ctx *ctx);

/* Number of doubles of a host-layout state. */
size_t echo_state_count(const echo_ctx *ctx);

/* Attach a caller-owned device workspace (>= echo_workspace_bytes bytes,
 * 256-byte aligned) and a CUDA stream (cudaStream_t, may be NULL for the
 * legacy default stream).  Resets the cumulative counters.  Returns
 * ECHO_ENOMEM if the workspace is too small, ECHO_EINVAL if misaligned. */
int echo_bind(echo_ctx *ctx, void *dev_workspace, size_t bytes, void *cuda_stream);

/* Method: primitive -> conserved map of the Valencia form (Anton et al. 2006).
 * Initial data: cell primitives (5, nz, ny, nx) = rho, v^x, v^y, v^z, p
 * (contravariant v) and the face field B~ in host face layout.  Converts
 * them to the conserved state on the device (cell-centre B = mean of the two
 * faces over sqrt(gamma)) and sets the Newton memory Z = rho h W^2. */
int echo_set_prims(echo_ctx *ctx, const double *prims5, const double *bface, int on_device);

/* Set the conserved state (host layout).  Z (nz*ny*nx doubles, may be NULL)
 * is the Newton guess memory; NULL selects the cold guess. */
int echo_set_state(echo_ctx *ctx, const double *state, const double *Z, int on_device);

/* Copy the conserved state out (host layout, periodic duplicate faces
 * filled).  Synchronises the stream. */
int echo_get_state(echo_ctx *ctx, double *state, int on_device);

/* Copy the primitives of the last c2p out: 8 cell arrays rho, v^x, v^y, v^z,
 * p, B^x, B^y, B^z (cell-centre B undensitised).  Synchronises. */
int echo_get_prims(echo_ctx *ctx, double *prims8, int on_device);

/* Copy the Newton memory Z (nz*ny*nx doubles) out.  Synchronises. */
int echo_get_z(echo_ctx *ctx, double *Z, int on_device);

/* Method: conservative-to-primitive inversion, a 1-D Newton iteration on
 * Z = rho h W^2 (as in Noble et al. 2006, one-dimensional form).
 * Conservative-to-primitive inversion of the current state on every owned
 * cell.  guess_mode: 0 = the stored Z of the cell (previous stage), 1 = the
 * c2p-guess network (see below), 2 = cold guess (Z = 0, replaced by the
 * admissibility rule); adding 4 refines the guess in FP32 first.  The
 * network (modes 1, 5) runs on the tensor cores in a pass of its own that
 * writes every cell's Newton start, followed by the plain c2p kernel; adding
 * 8 runs it in FP32 on the CUDA cores inside the c2p kernel instead, adding
 * 16 on the tensor cores inside the c2p kernel (the same starts, so the
 * same result as modes 1, 5).  The network modes choose the start per cell
 * as echo_set_c2p_guess describes.  Other values: ECHO_EINVAL.  If stats is non-NULL
 * the call synchronises and fills the counters and dt_cfl of stats (the
 * other fields are left untouched) and returns ECHO_EC2P if any cell failed. */
int echo_c2p(echo_ctx *ctx, int guess_mode, echo_totals *stats);

/* Method: the semi-discrete right-hand side of the finite-difference scheme:
 * MP5 reconstruction (Suresh & Huynh 1997), HLL fluxes (Harten, Lax & van
 * Leer 1983), UCT-HLL edge EMFs (Londrillo & Del Zanna 2004), Valencia
 * sources on a stationary metric.
 * L(U) of the current state: c2p, ghost fill, reconstruction, HLL fluxes,
 * UCT EMFs, flux difference + sources, and minus the curl of the EMFs for the
 * face field.  Written in host layout (state_count doubles) to L. */
int echo_rhs(echo_ctx *ctx, double *L, int on_device);

/* Method: the three-stage SSP Runge-Kutta scheme (Shu & Osher 1988) with the
 * CFL time step of the fastest characteristic speeds.
 * One SSP-RK3 step.  dt > 0: that step size; dt <= 0: the CFL step
 * cfl / max_cells sum_d max|lambda_d|/dx^d from the first-stage primitives. */
int echo_step(echo_ctx *ctx, double dt);

/* Method: volume sums of the conserved variables (conserved to rounding on
 * periodic grids by the flux form) and the discrete divergence of the
 * constrained-transport face field (Evans & Hawley 1988).
 * Totals of the current state (runs a c2p for dt_cfl), copied to *out.
 * Synchronises.  Returns ECHO_EC2P if an inversion failed since the last
 * call and floors are off. */
int echo_reduce(echo_ctx *ctx, echo_totals *out);

/* ---- c2p-guess network (a learned initial guess for the Newton solve) ----
 * A 9 -> 64 -> 64 -> 3 tanh network, FP32, maps scale-free features of the
 * conserved state and metric (log(tau/D), log(1+S^2/D^2), log(1+B^2/D),
 * (S.B)^2/(S^2 B^2), alpha, log sqrt(gamma), beta_i beta^i,
 * tr(gamma^ij)/3, log(D)/10) to log W, log(p/D) and the predicted log10
 * relative error of its guess Z0 = D W (1 + G/(G-1) (p/D) W).  The Newton
 * solve in FP64 stays the judge: from the network guess it may take at most
 * 8 iterations, else it restarts from the previous-stage Z (counted).
 * Float ECHO_MLP_GATE of the block (after the standardisation) holds the
 * network's gate (echo_mlp_calibrate).
 * A network "state" is ECHO_MLP_STATE floats of device memory: parameters
 * and standardisation block (ECHO_MLP_BLOCK floats: W1 64x9, b1, W2 64x64,
 * b2, W3 3x64, b3, feature mean/std (9+9), target mean/std (3+3)), then
 * the Adam moments m and v (ECHO_MLP_BLOCK floats each).  Datasets are row
 * major: features X (n x 9) and targets Y (n x 3: log W, log(p/D), log(Z/D)),
 * FP32 device arrays.  All buffers are caller-owned device memory. */
#define ECHO_MLP_NPARAM 4995
#define ECHO_MLP_BLOCK 5024
#define ECHO_MLP_STATE (3 * ECHO_MLP_BLOCK)

/* Method: Glorot & Bengio 2010 initialisation; splitmix64 generator.
 * Glorot-uniform weights (counter-based generator seeded by seed), zero
 * biases and moments, identity standardisation. */
int echo_mlp_init(float *dev_state, unsigned long long seed, void *cuda_stream);

/* Bytes of work buffer needed by echo_mlp_train/echo_mlp_grad/
 * echo_mlp_normalize for a batch size. */
size_t echo_mlp_work_bytes(int batch);

/* Standardisation of features and of the first two targets from n rows
 * (mean, std; constant columns keep std 1). */
int echo_mlp_normalize(float *dev_state, const float *X, const float *Y, long long n, void *dev_work,
                       size_t work_bytes, void *cuda_stream);

/* Method: Adam (Kingma & Ba 2015) on the squared-error loss of the network.
 * nsteps Adam steps (lr; b1 0.9, b2 0.999, eps 1e-8) on minibatches of
 * `batch` consecutive rows, step t (from step0) starting at row
 * (t * batch) mod n.  losses (device, may be NULL) receives each step's
 * mean batch loss. */
int echo_mlp_train(float *dev_state, const float *X, const float *Y, long long n, int batch, int nsteps,
                   long long step0, float lr, double gamma, void *dev_work, size_t work_bytes, float *losses,
                   void *cuda_stream);

/* Method: reverse-mode differentiation (backpropagation) of that loss.
 * Gradient (ECHO_MLP_NPARAM floats, device) and mean loss (device float, may
 * be NULL) of the batch loss over rows row0 .. row0+batch-1 (mod n). */
int echo_mlp_grad(const float *dev_state, const float *X, const float *Y, long long n, long long row0, int batch,
                  double gamma, float *dev_grad, float *dev_loss, void *dev_work, size_t work_bytes,
                  void *cuda_stream);

/* Standardised network outputs (n x 3, device) of n feature rows. */
int echo_mlp_forward(const float *dev_state, const float *X, long long n, float *out, void *cuda_stream);
/* The same with the products of layers 1 and 2 on the tensor cores
 * (tcgen05 MMA, BF16 inputs, FP32 accumulation; standardisation, tanh.approx
 * activations and layer 3 in FP32), as the network guess of c2p evaluates
 * it.  Rows whose tensor-core result did not arrive within about a second
 * get NaN. */
int echo_mlp_forward_tc(const float *dev_state, const float *X, long long n, float *out, void *cuda_stream);

/* Relative error |Z0 - Z| / Z of the network's Newton start Z0 on n rows
 * (features X, targets Y), for judging a trained network: the forward pass
 * (tensor_cores 0: echo_mlp_forward, 1: echo_mlp_forward_tc) writes the
 * standardised outputs to out (n x 3, device), then err (n floats, device)
 * receives the error of Z0 = D W (1 + G/(G-1) (p/D) W) against the target
 * Z = D exp(Y[:, 2]), evaluated in FP64 (gamma the adiabatic index). */
int echo_mlp_guess_error(const float *dev_state, const float *X, const float *Y, long long n, double gamma,
                         int tensor_cores, float *out, float *err, void *cuda_stream);

/* Method: training pairs that the inversion itself produces (the network
 * learns the Newton solve's converged answer).
 * Training rows from the current state: runs a c2p (previous-stage guess),
 * then writes for every owned cell its features and targets at row
 * offset + perm(cell) * stride of X/Y (perm: a fixed permutation of the
 * cells).  offset + (cells-1) * stride must be below capacity (rows). */
int echo_mlp_dataset(echo_ctx *ctx, float *X, float *Y, long long capacity, long long offset, long long stride);

/* The network's gate: writes to the state's block (float ECHO_MLP_GATE)
 * the mean over n rows (features X, targets Y, device) of log10 of its
 * Newton-start error, the network's typical error, below which a cell's
 * previous-stage Z is not expected to lose to it (see echo_set_c2p_guess).
 * out (n x 3) and err (n) are caller-owned device work arrays, as for
 * echo_mlp_guess_error (the tensor-core forward that c2p uses).  The gate
 * is 0 (an error of 1: only cold starts consult the network) until set. */
#define ECHO_MLP_GATE 5019
int echo_mlp_calibrate(float *dev_state, const float *X, const float *Y, long long n, double gamma, float *out,
                       float *err, void *cuda_stream);

/* Copy a trained network (the first ECHO_MLP_BLOCK floats of a state) into
 * the context; the Newton starts of an earlier network are discarded. */
int echo_mlp_load(echo_ctx *ctx, const float *dev_state);

/* Method: the initial guess of the Newton iteration (the iteration, not the
 * guess, decides the converged result).
 * Newton guess used by echo_step/echo_rhs: 0 previous-stage Z (default),
 * 1 network (requires echo_mlp_load), 2 cold (the guess of echo_c2p mode 2,
 * for measuring what the other guesses gain); adding 4 first refines that
 * guess by up to four Newton steps of the same residual in FP32 (the FP64
 * iterations that follow still decide convergence).  In the network modes
 * the start is chosen per cell: every inversion records how far each cell's
 * Z moved (an estimate of the error of the previous-stage Z as the next
 * start) and lists the cells that moved at least as much as the network's
 * calibrated typical error (echo_mlp_calibrate) -- with the FP32 refinement
 * (+4) only those that also moved by about 1/8 or more, since the refinement
 * brings any closer start to the same single FP64 iteration; the next inversion
 * evaluates the network for the listed cells only (packed into tiles of
 * 128), and a listed cell starts from it only where its predicted log10
 * error (third output) beats the previous Z's; all other cells start from
 * the previous-stage Z (not counted as a fallback).  After echo_set_prims,
 * or echo_set_state with Z, no cell is listed; after echo_set_state without
 * Z (a cold start) every cell is.  Inversions in the other modes keep no
 * record: the first network-mode inversion after them lists no cell; so
 * does one whose refinement flag (+4) differs from the previous one's.
 * The network's hidden layers run on the tensor cores (as
 * echo_mlp_forward_tc) in a pass before the c2p kernel; adding 8 to a network mode evaluates it in FP32 on the
 * CUDA cores inside the c2p kernel (modes 9, 13), adding 16 on the tensor
 * cores inside the c2p kernel (modes 17, 21).  Accepted: 0, 1, 2, 4, 5, 6,
 * 9, 13, 17, 21. */
int echo_set_c2p_guess(echo_ctx *ctx, int mode);

/* Copy the cumulative counters (c2p_iters, c2p_calls, c2p_fail, floor_hits,
 * mlp_fallback, fallback_faces, mlp_used, guard_faces, c2p_iter_hist) to *out without running anything; other
 * fields untouched.  Synchronises. */
int echo_counters(echo_ctx *ctx, echo_totals *out);

/* ---- batch of independent runs (parameter sweeps) ----
 * Method: independent runs of the scheme above, one time step of each per
 * call.  The paper motivates the cost of exploring many parameters; a batch advances
 * up to ECHO_BATCH_MAXRUNS independent runs (same metric kind, precision,
 * adiabatic index and CFL number; sizes may differ), by default with ONE
 * persistent cooperative kernel per SSP-RK3 stage.  Each stage's phases (ghost fills,
 * c2p, faces, EMFs, update) are cut into tiles over all runs and taken by
 * the resident blocks round-robin or from an atomic queue; grid-wide
 * barriers separate dependent phases (the cooperative launch keeps every
 * block resident, so they cannot deadlock).  Every run keeps its own CFL dt.
 * The runs must be bound contexts with a state; their workspaces and
 * counters are the runs' own.  In schedules 0 and 1, if run 0 uses the
 * network guess, all runs use run 0's guess mode and network, evaluated on
 * the tensor cores in a pass over all runs before each stage's c2p; schedule
 * 2 uses each run's own. */
#define ECHO_BATCH_MAXRUNS 32
typedef struct echo_batch echo_batch;

int echo_batch_create(echo_ctx *const *runs, int nruns, echo_batch **out);
/* Device bytes the batch needs (run descriptors, tile plan, queue). */
size_t echo_batch_workspace_bytes(const echo_batch *batch);
/* Attach a caller-owned 256-byte aligned workspace and the stream the stage
 * kernels run on (the runs' own streams are not used). */
int echo_batch_bind(echo_batch *batch, void *dev_workspace, size_t bytes, void *cuda_stream);
/* Tile size (multiple of 128 work items, <= 8192), resident blocks per SM
 * (1 .. echo_batch_max_blocks_per_sm) and queue kind (0 round-robin,
 * 1 atomic queue).  Default after bind: 256, the maximum, 1. */
int echo_batch_config(echo_batch *batch, int tile, int blocks_per_sm, int dynamic_queue);
int echo_batch_max_blocks_per_sm(echo_batch *batch);
/* Schedule: 0 (default) one persistent cooperative kernel per stage;
 * 1 one ordinary launch per phase over all runs' tiles (each phase with its
 * own register budget; blocks_per_sm and the queue kind do not apply);
 * 2 run-major: each run's own launch sequence (as echo_step) in turn, so a
 * run's working set stays in L2 across its phases (tile, blocks_per_sm and
 * queue kind do not apply).  ECHO_EINVAL for any other value.  Runs of
 * order 1 (echo_set_order) need schedule 2 (echo_batch_step returns
 * ECHO_EINVAL otherwise). */
int echo_batch_mode(echo_batch *batch, int mode);
/* Schedule 2 only: spread the runs over `branches` (1 .. number of runs)
 * concurrent streams forked from and joined back into the batch stream (in a
 * captured graph they become parallel branches), runs assigned
 * longest-first by zone count.  Default 1 (all runs on the batch stream). */
int echo_batch_branches(echo_batch *batch, int branches);
/* 1: capture one whole step (every launch of the schedule) into a CUDA graph
 * on first use and replay it; recaptured when dt or the configuration
 * changes.  Needs a created stream (ECHO_EINVAL on the legacy stream). */
int echo_batch_graph(echo_batch *batch, int enable);
/* One SSP-RK3 step of every run (dt > 0 for all, else each run's CFL dt). */
int echo_batch_step(echo_batch *batch, double dt);
const char *echo_batch_last_error(const echo_batch *batch);
void echo_batch_destroy(echo_batch *batch);

/* Method: IEEE 754 round-to-nearest-even binary64 -> binary32 conversion.
 * Self-check of the library's integer-pipe float <-> double conversions
 * against the hardware casts on n hashed test values (all float classes,
 * doubles over and beyond the float range, exact rounding ties): adds the
 * number of mismatches to *dev_mismatch (device, caller-zeroed). */
int echo_selftest_conversions(long long n, unsigned long long seed, unsigned long long *dev_mismatch,
                              void *cuda_stream);
/* Method: Newton-Raphson refinement r <- r + r (1 - d r) of a reciprocal.
 * Self-check of the library's Newton-Raphson FP64 reciprocal (used in the
 * c2p Newton solve in place of IEEE divisions) against the IEEE quotient on n
 * hashed values (both signs, exponents -300..300): atomically maxes the
 * largest distance in ulp into *dev_max_ulp (device, caller-zeroed). */
int echo_selftest_recip(long long n, unsigned long long seed, unsigned long long *dev_max_ulp, void *cuda_stream);
/* Method: one Newton-Raphson step r <- r + r (1 - d r) of a reciprocal.
 * The same check for the one-step reciprocal that forms the c2p Newton
 * step's quotient dZ = f / f' (its error perturbs only the next iterate):
 * the largest distance in ulp from the IEEE quotient into *dev_max_ulp
 * (device, caller-zeroed) over the same hashed values. */
int echo_selftest_recip1(long long n, unsigned long long seed, unsigned long long *dev_max_ulp,
                         void *cuda_stream);
/* Method: IEEE 754 binary64 exponent arithmetic (exact scaling by 2^k).
 * Self-check of the library's integer-pipe scaling by powers of two (the
 * exponent-field add the FP64 kernels use for alpha times a difference in
 * the MP5 test and for the halves and doublings of the c2p Newton step)
 * against the FP64 products x*4, x*2, x*0.5 on n hashed values (both signs,
 * exponents -1000..1000, and signed zeros): adds the number of bit-pattern
 * mismatches to *dev_mismatch (device, caller-zeroed). */
int echo_selftest_scale2(long long n, unsigned long long seed, unsigned long long *dev_mismatch, void *cuda_stream);
/* Method: the MP5 monotonicity test of Suresh & Huynh (1997), a b <= eps.
 * Self-check of the FP64 kernels' form of that test, decided from the signs
 * and binary exponents of a and b and multiplied out only near eps, against
 * the product test itself on n hashed pairs (exponent sums concentrated
 * around eps, both signs, zeros, subnormals, huge and infinite operands):
 * adds the number of differing decisions to *dev_mismatch (device,
 * caller-zeroed). */
int echo_selftest_mp5_accept(long long n, unsigned long long seed, unsigned long long *dev_mismatch,
                             void *cuda_stream);

/* Method: a register-only throughput probe (no counterpart in the paper).
 * FP64 fused multiply-add throughput probe: echo_selftest_dfma_blocks()
 * blocks of 256 threads (4 per SM of the current device; -1 if the device
 * cannot be queried), each thread running 8 independent chains of `iters`
 * (1 .. 2^31-1, else ECHO_EINVAL) FMAs c <- c * c - c in registers (one
 * source register per FMA, the form that issues at the FP64 pipe's full
 * rate), then writing one double per thread to dev_out (device,
 * at least 256 * blocks doubles, caller-owned).  *flops (host, may be NULL)
 * receives the launch's floating-point operations (2 per FMA), so that the
 * caller's event time around the launch gives the device's FP64 rate. */
int echo_selftest_dfma_blocks(void);
int echo_selftest_dfma(long long iters, double *dev_out, double *flops, void *cuda_stream);

/* Kernel classes timed by the profiling facility below (ECHO_K_NETWORK: the
 * network's own pass before c2p in guess modes 1 and 5). */
#define ECHO_K_FILL_FACES 0
#define ECHO_K_C2P 1
#define ECHO_K_FILL_PRIMS 2
#define ECHO_K_FACES_X 3
#define ECHO_K_FACES_Y 4
#define ECHO_K_FACES_Z 5
#define ECHO_K_EMF_X 6
#define ECHO_K_EMF_Y 7
#define ECHO_K_EMF_Z 8
#define ECHO_K_UPDATE 9
#define ECHO_K_SCALARS 10
#define ECHO_K_TOTALS 11
#define ECHO_K_CORRECT 12
#define ECHO_K_NETWORK 13
#define ECHO_NK 14

/* Enable (1) or disable (0) per-kernel timing: while enabled, every kernel
 * launch of echo_step/echo_rhs/echo_c2p/echo_reduce is bracketed by two
 * CUDA events recorded on the bound stream.  Not part of the numerics; adds
 * two event records per launch. */
int echo_profile(echo_ctx *ctx, int enable);

/* Synchronise, then write for each kernel class k < nk the summed device
 * time in milliseconds (ms[k]) and the number of launches (launches[k])
 * recorded since the last read, and reset the record. */
int echo_profile_read(echo_ctx *ctx, double *ms, long long *launches, int nk);

/* Name of kernel class k ("" if out of range). */
const char *echo_kernel_name(int k);

/* Totals of a state without allocating anything and without a context.
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory at the moment they want the numbers, such as an
 * application whose own memory manager has reserved all of HBM, or a
 * monitoring hook that must not change the device's memory footprint while
 * a large run sits near the HBM limit.
 *   state: device pointer, FP64 host layout of an n[0] x n[1] x n[2] grid
 *          (as written by echo_get_state with on_device = 1); its length
 *          (echo_state_count of such a grid) is not checked and must be
 *          the documented one.
 *   n, dx: host arrays of 3 (cells > 0, widths > 0).
 *   out6:  device pointer to 6 doubles, written with sum D dV, sum tau dV,
 *          sum S_x dV, sum S_y dV, sum S_z dV and max |div B~| (dV = dx dy dz),
 *          the same quantities echo_reduce reports.
 *   cuda_stream: stream to enqueue on (cudaStream_t, NULL = legacy stream).
 * state and out6 must be device (or managed) memory of the current device;
 * a host pointer or memory of another device returns ECHO_EINVAL with
 * nothing launched.  An error pending from earlier work on this thread is
 * reported as ECHO_ECUDA and left pending (not cleared), with nothing
 * launched.
 * The per-row partial sums live in one file-scope device array of
 * ECHO_STATIC_MAX_ROWS x 6 doubles (3 MiB) that every GPU loading the
 * library holds until the process exits; calls allocate nothing (no
 * cudaMalloc, no library allocator).  Rows = n[1] * n[2] above
 * ECHO_STATIC_MAX_ROWS return ECHO_ERANGE; bad arguments ECHO_EINVAL.  The
 * first call on a device looks up the array's device address (once per
 * device, with that device current) and caches it for the life of the
 * process -- the cached address does not survive a cudaDeviceReset of that
 * device; make that first call before any stream capture.  All calls share
 * the array: calls that overlap on the GPU race, so order them on one
 * stream.  Asynchronous: out6 is valid once the stream reaches the call. */
#define ECHO_STATIC_MAX_ROWS 65536
int echo_totals_static(const double *state, const int *n, const double *dx, double *out6, void *cuda_stream);

/* Message of the last failure on this context ("" if none). */
const char *echo_last_error(const echo_ctx *ctx);

/* Destroy a context (does not free the caller's workspace). */
void echo_destroy(echo_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* ECHO_H */
