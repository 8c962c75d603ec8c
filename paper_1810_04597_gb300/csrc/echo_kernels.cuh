// echo_kernels.cuh -- CUDA kernel templates of the GRMHD step (sm_103a).
//
// One pass of the hot path per RK stage:
//   fill(face B~) -> c2p (FP64 Newton) -> fill(primitives)
//   -> faces<x,y,z> (MP5 + HLL) -> emf<x,y,z> (UCT-HLL) -> update (flux
//   difference + sources + CT curl + SSP-RK3 combination).
// Templates over the metric kind MK (0 flat, 1 Kerr-Schild) and the storage
// type R are instantiated in echo_kernels_flat.cu and echo_kernels_ks.cu;
// metric-independent kernels live in echo_kernels_common.cu.
// Reductions (CFL rate, conserved totals, div B~) use warp shuffles and a
// fixed block tree, so results are bitwise reproducible run to run.
#pragma once

#include "echo_device.cuh"
#include "echo_launch.h"
#include "echo_mlp.cuh"
#include "echo_mlp_tc.cuh"

namespace echo {


// ------------------------------------------------------------------ helpers

__device__ __forceinline__ int stride_of(const Geom &g, int d)
{
    return d == 0 ? 1 : (d == 1 ? g.px : g.pxy);
}

template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Warp sum of small per-lane counts (32-bit: a 64-bit add issues on the
// FP64 pipe on GB300; the totals here stay far below 2^32).
__device__ __forceinline__ unsigned warp_sum_u32(unsigned v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------------ ghost fill

// Fill the ghost slab of axis d for a list of arrays, over the ghost layers
// the scheme reads (fill_layers: 3, order 1: 5).  Thread (s, t1, t2): s in
// [0, 2 L) selects the layer (lower NG-L..NG-1, upper NG+n..NG+n+L-1), t1/t2
// run over the same extent of the other axes (so that edges and corners
// are filled by the later axes).
template <typename R>
__device__ __forceinline__ void fill_body(const Geom &g, int d, const FillList<R> &L, long long t)
{
    const int d1 = d == 0 ? 1 : 0;
    const int d2 = d == 2 ? 1 : 2;
    const int nl = fill_layers(g);
    const int e1 = g.n[d1] + 2 * nl, e2 = g.n[d2] + 2 * nl;
    if (t >= (long long)2 * nl * e1 * e2)
        return;
    const int s = (int)(t % (2 * nl));
    const int t1 = (int)((t / (2 * nl)) % e1);
    const int t2 = (int)(t / (2 * nl) / e1);
    const int id_d = s < nl ? NG - nl + s : NG + g.n[d] + (s - nl);
    int ijk[3];
    ijk[d] = id_d;
    ijk[d1] = NG - nl + t1;
    ijk[d2] = NG - nl + t2;
    const int dst = gidx(g, ijk[0], ijk[1], ijk[2]);
    const int sd = stride_of(g, d);
    for (int a = 0; a < L.count; ++a) {
        bool flip;
        const int face = L.face[a] == d ? 1 : 0;
        const int src = bc_src(id_d, g.n[d], face, g.bc[2 * d], g.bc[2 * d + 1], flip);
        if (src == id_d)
            continue;
        R val = R(0);
        if (src >= 0) {
            val = L.a[a][dst + (src - id_d) * sd];
            // across a polar axis the component along d and the factor
            // sqrt(gamma) ~ sin(theta) are odd: negate if exactly one applies
            if (flip && ((L.comp[a] == d) != (L.dens[a] != 0)))
                val = -val;
        }
        L.a[a][dst] = val;
    }
}

template <typename R>
__global__ void k_fill(Geom g, int d, FillList<R> L)
{
    fill_body<R>(g, d, L, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// ------------------------------------------------------------------ c2p

// Conservative-to-primitive inversion of every owned cell (FP64 Newton);
// cell-centre B = mean of the two faces / sqrt(gamma).  Kerr-Schild runs with
// floors: a failed inversion keeps the cell's previous primitives, density
// and pressure are raised to the floors, and a cell changed that way has its
// conserved state reset from the floored primitives (counted in floor_hits).
// Optionally accumulates the CFL rate max (atomicMax on the bits of a
// non-negative double, order independent) and the Newton counters.
//
// With MLP the Newton guess comes from the c2p-guess network (weights staged
// in shared memory); Newton from that guess is capped at 8 iterations and
// falls back to the cell's previous-stage Z if it has not converged
// (counted in mlp_fallback).
// Body over the linear index t of the owned cells (x fastest); every lane of
// a warp must call it (warp-level counter reductions).  mlp_sm: the network
// block in shared memory when MLP.
// Densitised cell-centre B~ of the cell at padded index id: order 0 the
// mean of the two faces, order 1 the sixth-order interpolation of the faces
// i-2 .. i+3 along each axis.
template <typename R>
__device__ __forceinline__ void cell_centre_Bt(const Geom &g, const Arrays<R> &A, int id, double Bt[3])
{
    const int st[3] = {1, g.px, g.pxy};
    for (int d = 0; d < 3; ++d) {
        const R *__restrict__ f = A.U[5 + d];
        const int s = st[d];
        if (g.order)
            Bt[d] = ho_center(to_d(f[id - 2 * s]), to_d(f[id - s]), to_d(f[id]), to_d(f[id + s]),
                              to_d(f[id + 2 * s]), to_d(f[id + 3 * s]));
        else
            Bt[d] = 0.5 * (to_d(f[id]) + to_d(f[id + s]));
    }
}

// Inputs of the inversion at owned cell t (x fastest): undensitised D, S_i,
// tau, the cell-centre B (mean of the two faces), sqrt(gamma) and the metric
// point.  Returns false for t beyond the owned cells.
struct C2PCell {
    int id;
    int i, j;
    double B[3], S[3], Dc, tc, sg;
    const MetPt *mp;
};

template <int MK, typename R>
__device__ __forceinline__ bool c2p_cell(const Geom &g, const Arrays<R> &A, long long t, C2PCell &c)
{
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    if (t >= ncell)
        return false;
    // 32-bit decomposition: t < ncell < 2^31
    const unsigned u = (unsigned)t, n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
    const unsigned r = u / n0;
    c.i = NG + (int)(u - r * n0);
    const unsigned k0 = r / n1;
    c.j = NG + (int)(r - k0 * n1);
    const int k = NG + (int)k0;
    const int id = gidx(g, c.i, c.j, k);
    c.id = id;
    c.sg = 1.0;
    c.mp = nullptr;
    double Bt[3];
    cell_centre_Bt(g, A, id, Bt);
    if constexpr (MK == 1) {
        c.mp = &A.met.C[c.j * A.met.np0 + c.i];
        const double isg = c.mp->isg;
        c.sg = c.mp->sg;
        for (int q = 0; q < 3; ++q) {
            c.B[q] = Bt[q] * isg;
            c.S[q] = to_d(A.U[1 + q][id]) * isg;
        }
        c.Dc = to_d(A.U[0][id]) * isg;
        c.tc = to_d(A.U[4][id]) * isg;
    } else {
        for (int q = 0; q < 3; ++q) {
            c.B[q] = Bt[q];
            c.S[q] = to_d(A.U[1 + q][id]);
        }
        c.Dc = to_d(A.U[0][id]);
        c.tc = to_d(A.U[4][id]);
    }
    return true;
}

template <int MK>
__device__ __forceinline__ void c2p_cell_features(const C2PCell &c, float f[MLP_NI])
{
    if constexpr (MK == 1)
        mlp_features(c.Dc, c.S, c.tc, c.B, c.sg, MKS<double>(*c.mp), f);
    else
        mlp_features(c.Dc, c.S, c.tc, c.B, 1.0, MFlat<double>(), f);
}

// Newton start from the network outputs (log W, log(p/D)) of a cell with
// undensitised D: Z0 = D W (1 + G/(G-1) (p/D) W), in FP32.
__device__ __forceinline__ float net_z0(const float o[MLP_NO], double Dc, float gr_f)
{
    const float Wg = expf(o[0]), pD = expf(o[1]);
    return d2f(Dc) * Wg * (1.0f + gr_f * pD * Wg);
}

// MLPK: 0 no network; 1 network evaluated here (CUDA cores, parameter block
// mlp_sm in shared memory); 2 network outputs net[0..2] (log W, log(p/D),
// predicted log10 error) computed by the caller, usable if net_ok; 3 the
// Newton starts A.zg written by k_mlp_guess_tc.  Every network start is
// Z0 = D W (1 + G/(G-1) (p/D) W) in FP32 (net_z0): it only starts the Newton
// solve, and the FP64 pipe is the scarce one.
//
// Per-cell choice (network modes): only a cell the last inversion listed
// (its previous-Z error code A.ze within the network's gate) consults the
// network, and it takes the network start only where the network's
// predicted error beats its previous Z's (net_beats); every other cell
// starts from the previous-stage Z.
//
// Every inversion of the network modes writes the cell's new code A.ze and
// appends the cell to A.nlist when the new code is within the gate (the
// list the network's pass before the next inversion walks; the host empties
// it between that pass and the inversion).  The plain modes (MLPK 0) write
// neither; the host resets the codes before a network-mode inversion that
// follows them.  Every lane of a warp must call this.
template <int MK, typename R, int MLPK>
__device__ __forceinline__ void c2p_body(const Geom &g, const Phys &ph, const Arrays<R> &A, int guess_mode,
                                         int want_rate, long long t, const float *mlp_sm,
                                         const float *net = nullptr, bool net_ok = false)
{
    C2PCell c;
    const bool live = c2p_cell<MK, R>(g, A, t, c);
    double rate = 0.0;
    unsigned its = 0, calls = 0, fails = 0, floors = 0, mfb = 0, used = 0;
    bool want_net = false;
    int gate = 0;
    if constexpr (MLPK != 0)
        gate = ze_gate_mode(A.mlp[MLP_OGATE], guess_mode);
    if (live) {
        const int id = c.id;
        const int i = c.i;
        const MetPt *mp = c.mp;
        const double sg = c.sg;
        const double *B = c.B, *S = c.S;
        const double Dc = c.Dc, tc = c.tc;
        const int src = guess_mode & 3;
        const bool refine = (guess_mode & 4) != 0;
        const double zg = src == 2 ? 0.0 : A.Z[id];
        constexpr double tol = sizeof(R) == 4 ? NEWTON_TOL_BULK32 : NEWTON_TOL;
        C2PResult r;
        if constexpr (MLPK != 0) {
            // pick: 1 the network start z0f, 0 the previous-stage Z, -1 the
            // previous-stage Z because the network's result is missing (counted)
            int pick = 0;
            float z0f = 0.0f;
            const unsigned char code = A.ze[id];
            if ((int)code <= gate) {
                if constexpr (MLPK == 3) {
                    z0f = A.zg[id];
                    pick = z0f > 0.0f ? 1 : (z0f < 0.0f ? -1 : 0);
                } else {
                    float o[MLP_NO];
                    bool ok = true;
                    if constexpr (MLPK == 1) {
                        float f[MLP_NI];
                        c2p_cell_features<MK>(c, f);
                        mlp_infer(mlp_sm, f, o);
                    } else {
                        o[0] = net[0];
                        o[1] = net[1];
                        o[2] = net[2];
                        ok = net_ok;
                    }
                    if (!ok) {
                        pick = -1;
                    } else if (net_beats(o[2], code)) {
                        pick = 1;
                        z0f = net_z0(o, Dc, ph.gr_f);
                    }
                }
            }
            // the chosen start; after a network start that did not converge
            // in 8 iterations, the restart from the previous-stage Z (no FP32
            // refinement then; reloaded, so that no register holds it across
            // the first solve)
            double start = zg;
            int maxit = NEWTON_MAXIT;
            bool ref = refine;
            if (pick == 1) {
                used = 1;
                start = f2d(z0f);
                maxit = 8;
            } else if (pick == -1) {
                mfb = 1;
            }
            if constexpr (MK == 1)
                r = c2p_newton<sizeof(R) == 4>(Dc, S, tc, B, start, ph.gm1g, MKS<double>(*mp), maxit, ref, tol);
            else
                r = c2p_newton<sizeof(R) == 4>(Dc, S, tc, B, start, ph.gm1g, MFlat<double>(), maxit, ref, tol);
            if (!r.ok && pick == 1) {
                mfb = 1;
                const int first = r.iters;
                const double z1 = src == 2 ? 0.0 : __ldcg(&A.Z[id]);
                if constexpr (MK == 1)
                    r = c2p_newton(Dc, S, tc, B, z1, ph.gm1g, MKS<double>(*mp), NEWTON_MAXIT, false, tol);
                else
                    r = c2p_newton(Dc, S, tc, B, z1, ph.gm1g, MFlat<double>(), NEWTON_MAXIT, false, tol);
                r.iters += first;
            }
        } else {
            if constexpr (MK == 1)
                r = c2p_newton<sizeof(R) == 4>(Dc, S, tc, B, zg, ph.gm1g, MKS<double>(*mp), NEWTON_MAXIT, refine, tol);
            else
                r = c2p_newton<sizeof(R) == 4>(Dc, S, tc, B, zg, ph.gm1g, MFlat<double>(), NEWTON_MAXIT, refine, tol);
        }
        its = r.iters;
        calls = 1;
        fails = r.ok ? 0 : 1;
        double P8[8] = {r.rho, r.v[0], r.v[1], r.v[2], r.p, B[0], B[1], B[2]};
        double Z = r.Z;
        // the previous-stage Z again from memory, not held across the solve
        double zold = 0.0;
        if constexpr (MLPK != 0)
            zold = __ldcg(&A.Z[id]);
        if constexpr (MK == 1) {
            if (A.met.use_floors) {
                bool reset = !r.ok;
                if (reset)
                    for (int q = 0; q < 5; ++q)
                        P8[q] = to_d(A.P[q][id]);
                const double rf = A.met.floors[2 * i], pf = A.met.floors[2 * i + 1];
                if (!ile(rf, P8[0])) {
                    P8[0] = rf;
                    reset = true;
                }
                if (!ile(pf, P8[4])) {
                    P8[4] = pf;
                    reset = true;
                }
                if (reset) {
                    floors = 1;
                    double C5[5];
                    p2c_point(P8, ph.gr, MKS<double>(*mp), C5, Z);
                    for (int q = 0; q < 5; ++q)
                        A.U[q][id] = from_d<R>(C5[q] * sg);
                }
            }
        }
        for (int q = 0; q < 8; ++q)
            A.P[q][id] = from_d<R>(P8[q]);
        A.Z[id] = Z;
        if constexpr (MLPK != 0) {
            // the previous-Z error code for the next inversion, and whether
            // this cell may gain from the network there
            const unsigned char code = ze_code(Z, zold);
            A.ze[id] = code;
            want_net = (int)code <= ze_gate_mode(__ldg(&A.mlp[MLP_OGATE]), guess_mode);
        }
        if (want_rate) {
            if constexpr (sizeof(R) == 4) {
                float Pf[8];
                for (int q = 0; q < 8; ++q)
                    Pf[q] = d2f(P8[q]);
                const float idxf[3] = {d2f(g.idx[0]), d2f(g.idx[1]), d2f(g.idx[2])};
                float rf;
                if constexpr (MK == 1)
                    rf = cfl_rate(Pf, ph.gamma_f, ph.gr_f, idxf, MKS<float>(A.met.Cf[mp - A.met.C]));
                else
                    rf = cfl_rate(Pf, ph.gamma_f, ph.gr_f, idxf, MFlat<float>());
                rate = f2d(rf);
            } else {
                if constexpr (MK == 1)
                    rate = cfl_rate(P8, ph.gamma, ph.gr, g.idx, MKS<double>(*mp));
                else
                    rate = cfl_rate(P8, ph.gamma, ph.gr, g.idx, MFlat<double>());
            }
        }
    }
    // the cells the next inversion may start from the network
    if constexpr (MLPK != 0)
        list_append(want_net, live ? c.id : 0, A.nlist, &A.scal->nlist_count);
    // histogram of the iteration counts: one atomic per distinct count in the warp
    {
        const unsigned lmask = __ballot_sync(0xffffffffu, live);
        if (live) {
            const int b = its < (unsigned)(ECHO_C2P_HIST - 1) ? (int)its : ECHO_C2P_HIST - 1;
            const unsigned same = __match_any_sync(lmask, b);
            if ((int)(threadIdx.x & 31) == __ffs(same) - 1)
                atomicAdd(&A.scal->c2p_hist[b], (unsigned long long)__popc(same));
        }
    }
    // warp-aggregated counters
    its = warp_sum_u32(its);
    calls = warp_sum_u32(calls);
    fails = warp_sum_u32(fails);
    floors = warp_sum_u32(floors);
    if constexpr (MLPK != 0) {
        mfb = warp_sum_u32(mfb);
        used = warp_sum_u32(used);
    }
    if (want_rate)
        rate = warp_max(rate);
    if ((threadIdx.x & 31) == 0) {
        if (calls) {
            atomicAdd(&A.scal->c2p_iters, (unsigned long long)its);
            atomicAdd(&A.scal->c2p_calls, (unsigned long long)calls);
        }
        if (fails) {
            atomicAdd(&A.scal->c2p_fail, (unsigned long long)fails);
            atomicAdd(&A.scal->fail_since_check, (unsigned long long)fails);
        }
        if (floors)
            atomicAdd(&A.scal->floor_hits, (unsigned long long)floors);
        if constexpr (MLPK != 0) {
            if (mfb)
                atomicAdd(&A.scal->mlp_fallback, (unsigned long long)mfb);
            if (used)
                atomicAdd(&A.scal->mlp_used, (unsigned long long)used);
        }
        if (want_rate && rate > 0.0)
            atomicMax(&A.scal->rate_bits, (unsigned long long)__double_as_longlong(rate));
    }
}

// NET: 0 no network; 1 the FP32 network on the CUDA cores (parameter block
// staged in shared memory); 3 the Newton starts k_mlp_guess_tc wrote (that
// form through k_c2p_listed).
template <int MK, typename R, int NET>
__global__ void __launch_bounds__(128) k_c2p(Geom g, Phys ph, Arrays<R> A, int guess_mode, int want_rate)
{
    extern __shared__ float4 mlp_smem4[];
    const float *sm = nullptr;
    if constexpr (NET == 1) {
        float *Ps = reinterpret_cast<float *>(mlp_smem4);
        for (int q = threadIdx.x; q < MLP_BLOCK; q += blockDim.x)
            Ps[q] = A.mlp[q];
        __syncthreads();
        sm = Ps;
    }
    c2p_body<MK, R, NET>(g, ph, A, guess_mode, want_rate, (long long)blockIdx.x * blockDim.x + threadIdx.x, sm);
}

// c2p from the Newton starts k_mlp_guess_tc wrote for the listed cells
// (NET 3), held to the plain kernel's occupancy (flat: 7 blocks of 128
// threads per SM; Kerr-Schild: 4): the FP64-bound solve needs the warps more
// than the registers, and the Kerr-Schild solve spills below ~110.
template <int MK, typename R>
__global__ void __launch_bounds__(128, MK == 0 ? 7 : 4) k_c2p_listed(Geom g, Phys ph, Arrays<R> A, int guess_mode, int want_rate)
{
    c2p_body<MK, R, 3>(g, ph, A, guess_mode, want_rate, (long long)blockIdx.x * blockDim.x + threadIdx.x, nullptr);
}

// Inputs of one cell's network features, loaded one tile ahead of their use
// by k_mlp_guess_tc (the loads are in flight during the MMA round trips).
template <typename R>
struct CellIn {
    R u[5];          // D, S_i, tau (densitised)
    R bf[3][2];      // the two faces of each B~ component
    int id, i, j;
    bool live;
};

template <typename R>
__device__ __forceinline__ void cell_in_load(const Geom &g, const Arrays<R> &A, long long t, CellIn<R> &x)
{
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    x.live = t < ncell;
    const unsigned u = x.live ? (unsigned)t : 0u, n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
    const unsigned r = u / n0, k0 = r / n1;
    x.i = NG + (int)(u - r * n0);
    x.j = NG + (int)(r - k0 * n1);
    x.id = gidx(g, x.i, x.j, NG + (int)k0);
    const int st[3] = {1, g.px, g.pxy};
#pragma unroll
    for (int q = 0; q < 5; ++q)
        x.u[q] = A.U[q][x.id];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        x.bf[d][0] = A.U[5 + d][x.id];
        x.bf[d][1] = A.U[5 + d][x.id + st[d]];
    }
}

template <typename R>
__device__ __forceinline__ float to_f(R x);
template <>
__device__ __forceinline__ float to_f<float>(float x) { return x; }
template <>
__device__ __forceinline__ float to_f<double>(double x) { return d2f(x); }

// The network features of a loaded cell, in FP32 (cell-centre B the mean of
// the two faces, which the training pairs also use for the scheme of order
// 0; for order 1 the start changes by the difference of the two centre
// values, a few 1e-3 at most, and Newton decides as before); returns the
// undensitised D.
template <int MK, typename R>
__device__ __forceinline__ float cell_in_features(const Arrays<R> &A, const CellIn<R> &x, float f[MLP_NI])
{
    float isg = 1.0f, sg = 1.0f;
    float S[3], B[3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
        B[d] = 0.5f * (to_f(x.bf[d][0]) + to_f(x.bf[d][1]));
    if constexpr (MK == 1) {
        const MetPt &mp = A.met.C[x.j * A.met.np0 + x.i];
        isg = d2f(mp.isg);
        sg = d2f(mp.sg);
#pragma unroll
        for (int d = 0; d < 3; ++d)
            B[d] *= isg;
    }
    const float D = to_f(x.u[0]) * isg, tau = to_f(x.u[4]) * isg;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        S[q] = to_f(x.u[1 + q]) * isg;
    if constexpr (MK == 1)
        mlp_features_f(D, S, tau, B, sg, MKS<double>(A.met.C[x.j * A.met.np0 + x.i]), f);
    else
        mlp_features_f(D, S, tau, B, 1.0f, MFlat<float>(), f);
    return D;
}

// The network's Newton starts for the c2p kernel that follows (NET 3), both
// hidden layers on the tensor cores (echo_mlp_tc.cuh), for the cells the
// last inversion listed (A.nlist, A.scal->nlist_count entries): persistent
// CTAs of 128 threads walk the list in tiles of 128 cells.  A listed cell
// gets the start Z0 > 0 where the network's predicted error beats its
// previous Z's (net_beats), else 0; a tile whose tensor-core result did not
// arrive writes -1 (previous-stage Z, counted in mlp_fallback).  Unlisted
// cells are not touched (c2p does not read their start).  The next tile's
// inputs load during the current tile's MMA round trips.  Keeping the
// network out of the c2p kernel leaves that FP64-bound kernel at full
// occupancy and free of the per-tile barriers of the MMA round trips.
template <int MK, typename R>
__device__ __forceinline__ void listed_cell_load(const Geom &g, const Arrays<R> &A, const int *list, long long cnt,
                                                 long long r, CellIn<R> &x)
{
    const int id = list[r < cnt ? r : cnt - 1];
    // padded index -> (i, j, k); a lane past the end repeats the last cell
    const int k = id / g.pxy, rem = id - k * g.pxy;
    const int j = rem / g.px, i = rem - j * g.px;
    const long long t = ((long long)(k - NG) * g.n[1] + (j - NG)) * g.n[0] + (i - NG);
    cell_in_load(g, A, t, x);
    x.live = r < cnt;
}

template <int MK, typename R>
__global__ void __launch_bounds__(128, 6) k_mlp_guess_tc(Geom g, Arrays<R> A, float gr_f)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    const long long cnt = (long long)A.scal->nlist_count;
    const long long ntiles = (cnt + 127) / 128;
    long long tile = blockIdx.x;
    if (tile >= ntiles)
        return;   // block-uniform: nothing listed for this CTA (nothing allocated yet)
    TcMlp tm;
    tc_setup(tm, tc_smem, A.mlp);
    CellIn<R> x;
    listed_cell_load<MK, R>(g, A, A.nlist, cnt, tile * 128 + threadIdx.x, x);
    for (; tile < ntiles; tile += gridDim.x) {
        float f[MLP_NI], o[MLP_NO];
        const float D = cell_in_features<MK, R>(A, x, f);
        const int id = x.id;
        const bool live = x.live;
        const long long next = tile + gridDim.x;
        if (next < ntiles)
            listed_cell_load<MK, R>(g, A, A.nlist, cnt, next * 128 + threadIdx.x, x);
        const bool ok = tc_tile(tm, f, o);
        if (live) {
            float z0 = -1.0f;
            if (ok) {
                const float Wg = expf(o[0]), pD = expf(o[1]);
                z0 = net_beats(o[2], A.ze[id]) ? D * Wg * (1.0f + gr_f * pD * Wg) : 0.0f;
            }
            A.zg[id] = z0;
        }
    }
    tc_teardown(tm);
}

// c2p with the network evaluated inside it (guess mode +16), both hidden
// layers on the tensor cores (echo_mlp_tc.cuh): persistent CTAs of 128
// threads walk tiles of 128 cells; where a cell of the tile was listed by the
// last inversion, every thread computes its cell's features, the CTA runs the
// network (one tcgen05 MMA group), and the listed cells start from it where
// its predicted error beats the previous Z's; other tiles skip the network.
// A tile whose tensor-core result did not arrive falls back to the
// previous-stage guess (counted in mlp_fallback).
template <int MK, typename R>
__global__ void __launch_bounds__(128, 6) k_c2p_tc(Geom g, Phys ph, Arrays<R> A, int guess_mode, int want_rate,
                                                long long ntiles)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    TcMlp tm;
    tc_setup(tm, tc_smem, A.mlp);
    const int gate = ze_gate_mode(A.mlp[MLP_OGATE], guess_mode);
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long t = tile * 128 + threadIdx.x;
        C2PCell c;
        float f[MLP_NI], o[MLP_NO] = {0.0f, 0.0f, 0.0f};
        const bool have = c2p_cell<MK, R>(g, A, t, c);
        const bool listed = have && (int)A.ze[c.id] <= gate;
        bool ok = false;
        if (__syncthreads_or(listed ? 1 : 0)) {   // block-uniform
            if (have)
                c2p_cell_features<MK>(c, f);
            else
                for (int q = 0; q < MLP_NI; ++q)
                    f[q] = tm.P[TP_NORM + q];
            ok = tc_tile(tm, f, o);
        }
        c2p_body<MK, R, 2>(g, ph, A, guess_mode, want_rate, t, nullptr, o, ok);
    }
    tc_teardown(tm);
}

// ------------------------------------------------------------------ limiter
// compaction
//
// Each lane holds up to 16 reconstructions (slot = 2 m + side); `pend` marks
// those whose unlimited MP5 value was rejected.  The pending items are packed
// into a shared list (prefix sum of the counts: over the warp in FP32, over
// the block in FP64), processed 32 items per warp round -- a lane takes an
// item, loads the owning thread's stencil itself and evaluates the limited
// value -- and the results return through shared memory.  Rounds drop from
// the max over lanes of their pending count to ceil(total / 32).
constexpr int kWarpsPerBlock = 4;   // kernels using this run 128 threads

template <typename T>
struct LimScratch {
    T res[kWarpsPerBlock][32][16];
    unsigned short desc[kWarpsPerBlock * 32 * 16];
    int ids[kWarpsPerBlock * 32];   // FP64: each thread's unit, for items taken by another warp
    int wtot[kWarpsPerBlock];
};

// limited(id_of_owner, m, side, uor) -> T.  With PRE the owners have stored
// every unlimited value in their res slots before the call (uor passes the
// rejected item's one, so the limiter need not recompute it; FP64, where that
// saves five FP64-pipe instructions per item), else uor is 0.
//
// FP64 (PRE) packs the items of the whole block (128 threads): the last,
// partly filled round then occurs once per block rather than once per warp,
// which on the FP64 pipe is worth the block's three barriers.  Every thread
// of the block must call it then; the callers' units are block-uniform.
template <bool PRE, typename T, typename F>
__device__ __forceinline__ void compact_limit(unsigned pend, int id, LimScratch<T> &sm, F limited)
{
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int cnt = __popc(pend);
    int excl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, excl, o);
        if (lane >= o)
            excl += v;
    }
    const int wtotal = __shfl_sync(0xffffffffu, excl, 31);
    excl -= cnt;
    if constexpr (PRE) {
        sm.ids[threadIdx.x] = id;
        if (lane == 0)
            sm.wtot[w] = wtotal;
        __syncthreads();
        int wbase = 0, total = 0;
#pragma unroll
        for (int q = 0; q < kWarpsPerBlock; ++q) {
            const int v = sm.wtot[q];
            wbase += q < w ? v : 0;
            total += v;
        }
        if (total == 0)
            return;   // block-uniform
        {
            unsigned m = pend;
            int k = wbase + excl;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                sm.desc[k++] = (unsigned short)((threadIdx.x << 4) | b);
            }
        }
        __syncthreads();
        for (int base = w * 32; base < total; base += 32 * kWarpsPerBlock) {
            const int item = base + lane;
            if (item < total) {
                const unsigned d = sm.desc[item];
                const int o = (int)(d >> 4), b = (int)(d & 15);
                T &slot = sm.res[o >> 5][o & 31][b];
                slot = limited(sm.ids[o], b >> 1, b & 1, slot);
            }
        }
        __syncthreads();
    } else {
        const int total = wtotal;
        if (total == 0)
            return;
        unsigned short *desc = sm.desc + w * (32 * 16);
        {
            unsigned m = pend;
            int k = excl;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                desc[k++] = (unsigned short)((lane << 4) | b);
            }
        }
        __syncwarp();
        for (int base = 0; base < total; base += 32) {
            const int item = base + lane;
            const bool act = item < total;
            const unsigned d = act ? desc[item] : (unsigned)(lane << 4);
            const int o = (int)(d >> 4);
            const int ido = __shfl_sync(0xffffffffu, id, o);
            if (act) {
                const int b = (int)(d & 15);
                sm.res[w][o][b] = limited(ido, b >> 1, b & 1, T(0));
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ faces

// MP5 left/right states, HLL flux and speeds on the D-faces of the box
// faces_space gives: along D every face of an owned cell (order 1: two more
// per side for the flux correction), across D three rows into the ghosts
// (the EMF stencils read face data there; order 1: two more).  Threads map
// linearly onto that box so that warps stay full at row ends.  A reconstructed side with rho <= 0, p <= 0 or v^2 >= 1 takes
// the adjacent cell's primitives.
//
// The MP5 limiter is taken by ~10-15% of reconstructions; evaluated inline
// it would run for the whole warp at every one of the 14 calls.  Instead
// all unlimited values are computed first, a bitmask records the rejected
// ones, and compact_limit evaluates them packed 32 per warp round.
template <int D, int MK, typename R>
__device__ __forceinline__ void faces_body(const Geom &g, const Phys &ph, const Arrays<R> &A, long long t,
                                           LimScratch<R> &lsm)
{
    constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
    int cnt[3], off[3];
    faces_space(g, D, cnt, off);
    const long long tot = (long long)cnt[0] * cnt[1] * cnt[2];
    const bool live = t < tot;
    int ijk[3];
    {
        // 32-bit decomposition: the face box lies inside the padded array
        const unsigned tt = live ? (unsigned)t : 0u, c0 = (unsigned)cnt[0], c1 = (unsigned)cnt[1];
        const unsigned r = tt / c0, r2 = r / c1;
        ijk[0] = off[0] + (int)(tt - r * c0);
        ijk[1] = off[1] + (int)(r - r2 * c1);
        ijk[2] = off[2] + (int)r2;
    }
    const int order = g.order;
    const int id = gidx(g, ijk[0], ijk[1], ijk[2]);
    const int sd = stride_of(g, D);
    using T = R;
    const int qs[7] = {0, 1, 2, 3, 4, 5 + T1, 5 + T2};
    T Lv[7] = {}, Rv[7] = {};
    unsigned pend = 0;
    if (live) {
#pragma unroll
        for (int m = 0; m < 7; ++m) {
            const R *__restrict__ a = A.P[qs[m]];
            T q[6];
#pragma unroll
            for (int s = 0; s < 6; ++s)
                q[s] = a[id + (s - 3) * sd];
            bool okL, okR;
            const T d1 = q[2] - q[1], d2 = q[3] - q[2], d3 = q[4] - q[3];
            Lv[m] = mp5_try_d(q[0], q[1], q[2], q[3], q[4], d2, d1, okL, order);
            Rv[m] = mp5_try_d(q[5], q[4], q[3], q[2], q[1], -d2, -d3, okR, order);
            pend |= (okL ? 0u : 1u) << (2 * m);
            pend |= (okR ? 0u : 1u) << (2 * m + 1);
        }
    }
    // limiter on the rejected items, compacted across the warp
    constexpr bool PRE = sizeof(T) == 8;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if constexpr (PRE) {
#pragma unroll
        for (int m = 0; m < 7; ++m) {
            lsm.res[w][lane][2 * m] = Lv[m];
            lsm.res[w][lane][2 * m + 1] = Rv[m];
        }
    }
    compact_limit<PRE, T>(pend, id, lsm, [&](int ido, int m, int side, T uor) -> T {
        const R *__restrict__ a = A.P[qs[m]];
        // the item's own five-point stencil, oriented towards its face (the
        // right state's is the left one's mirror): one limiter evaluation
        const int s0 = side ? 2 * sd : -3 * sd, ds = side ? -sd : sd;
        T q[5];
#pragma unroll
        for (int s = 0; s < 5; ++s)
            q[s] = a[ido + s0 + s * ds];
        if constexpr (PRE)
            return mp5_limit_u(q[0], q[1], q[2], q[3], q[4], uor);
        else
            return mp5_limit(q[0], q[1], q[2], q[3], q[4], order);
    });
    if (!live)
        return;
#pragma unroll
    for (int m = 0; m < 7; ++m) {
        if (PRE || (pend & (1u << (2 * m))))
            Lv[m] = lsm.res[w][lane][2 * m];
        if (PRE || (pend & (1u << (2 * m + 1))))
            Rv[m] = lsm.res[w][lane][2 * m + 1];
    }
    // face metric (x1-faces: F1, x2-faces: F2, x3-faces: the cell-centre table)
    const MetPtOf<T> *mp = nullptr;   // the table of the storage type: no conversion
    T isgf = T(1);
    if constexpr (MK == 1) {
        const int ti = ijk[1] * A.met.np0 + ijk[0];
        const MetOf<T> M(A.met);
        mp = D == 0 ? &M.F1[ti] : (D == 1 ? &M.F2[ti] : &M.C[ti]);
        if (!(mp->sg > T(0))) {
            // polar-axis face: zero area, no flux
#pragma unroll
            for (int q = 0; q < 5; ++q)
                A.F[D][q][id] = T(0);
            A.ap[D][id] = T(0);
            A.am[D][id] = T(0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                A.fv[D][q][id] = T(0);
            return;
        }
        isgf = mp->isg;
    }
    T PL[8], PR[8];
#pragma unroll
    for (int m = 0; m < 7; ++m) {
        PL[qs[m]] = Lv[m];
        PR[qs[m]] = Rv[m];
    }
    const T Bn = A.U[5 + D][id] * isgf;
    PL[5 + D] = Bn;
    PR[5 + D] = Bn;
    // v^2 of each side, written as state_flux writes it (v_i v^i), which
    // then takes it instead of forming it again
    auto side_v2 = [&](const T *Ps) -> T {
        if constexpr (MK == 1) {
            const MKS<T> m(*mp);
            const T vv[3] = {Ps[1], Ps[2], Ps[3]};
            T vl[3];
            lower<T>(m, vv, vl);
            return vl[0] * vv[0] + vl[1] * vv[1] + vl[2] * vv[2];
        } else {
            const T vv[3] = {Ps[1], Ps[2], Ps[3]};
            return vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2];
        }
    };
    T v2s[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        T *Ps = side == 0 ? PL : PR;
        T v2 = side_v2(Ps);
        if (!is_pos(Ps[0]) || !is_pos(Ps[4]) || !ilt(v2, T(1))) {
            const int c = id + (side == 0 ? -sd : 0);
#pragma unroll
            for (int m = 0; m < 7; ++m)
                Ps[qs[m]] = A.P[qs[m]][c];
            v2 = side_v2(Ps);
            // counted on the faces that bound owned cells, each face once
            bool owned = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int top = NG + g.n[a] - 1 + ((a == D && g.bc[2 * D] != BC_PERIODIC) ? 1 : 0);
                owned = owned && ijk[a] >= NG && ijk[a] <= top;
            }
            if (owned)
                atomicAdd(&A.scal->fallback_faces, 1ULL);
        }
        v2s[side] = v2;
    }
    T FL[5], UL[5], FR[5], UR[5], npL, nmL, YL, npR, nmR, YR;
    if constexpr (MK == 1) {
        const MKS<T> m(*mp);
        state_flux<D>(PL, phys_gamma<T>(ph), phys_gr<T>(ph), m, FL, UL, npL, nmL, YL, &v2s[0]);
        state_flux<D>(PR, phys_gamma<T>(ph), phys_gr<T>(ph), m, FR, UR, npR, nmR, YR, &v2s[1]);
    } else {
        const MFlat<T> m;
        state_flux<D>(PL, phys_gamma<T>(ph), phys_gr<T>(ph), m, FL, UL, npL, nmL, YL, &v2s[0]);
        state_flux<D>(PR, phys_gamma<T>(ph), phys_gr<T>(ph), m, FR, UR, npR, nmR, YR, &v2s[1]);
    }
    // both states' 1/Y from one division in FP64
    T iYL, iYR;
    if constexpr (sizeof(T) == 8) {
        const T inv = T(1) / (YL * YR);
        iYL = inv * YR;
        iYR = inv * YL;
    } else {
        iYL = fast_recip(YL);
        iYR = fast_recip(YR);
    }
    const T lpL = npL * iYL, lmL = nmL * iYL, lpR = npR * iYR, lmR = nmR * iYR;
    const T ap = imax(T(0), imax(lpL, lpR));
    const T am = imax(T(0), imax(-lmL, -lmR));
    const T ssum = ap + am;
    if (is_pos(ssum)) {
        const T is = fast_recip(ssum);
        const T wL = ap * is, wR = am * is, wD = wL * am;
#pragma unroll
        for (int q = 0; q < 5; ++q)
            A.F[D][q][id] = wL * FL[q] + wR * FR[q] - wD * (UR[q] - UL[q]);
    } else {
#pragma unroll
        for (int q = 0; q < 5; ++q)
            A.F[D][q][id] = T(0.5) * (FL[q] + FR[q]);
    }
    A.ap[D][id] = ap;
    A.am[D][id] = am;
    A.fv[D][0][id] = PL[1 + D];
    A.fv[D][1][id] = PR[1 + D];
    A.fv[D][2][id] = PL[1 + T1];
    A.fv[D][3][id] = PR[1 + T1];
}

template <int D, int MK, typename R>
__global__ void __launch_bounds__(128) k_faces(Geom g, Phys ph, Arrays<R> A)
{
    __shared__ LimScratch<R> lsm;
    faces_body<D, MK, R>(g, ph, A, (long long)blockIdx.x * blockDim.x + threadIdx.x, lsm);
}

// ------------------------------------------------------------------ EMF

// UCT-HLL EMF on the edges along E; (a, b, E) cyclic.  The edge with index
// (i,j,k) sits at the lower half-integer positions along a and b.
//   E = [ap_a ap_b E_LL + ap_a am_b E_LR + am_a ap_b E_RL + am_a am_b E_RR]
//       / ((ap_a + am_a)(ap_b + am_b))
//     + ap_a am_a / (ap_a + am_a) (B~b_R - B~b_L) - ap_b am_b / (ap_b + am_b) (B~a_R - B~a_L),
//   E_st = -(v^a_st B~b_s - v^b_st B~a_t)   (s: a-side, t: b-side).
// v^a, v^b: a-face states (MP5 along a) reconstructed along b; B~b (b-faces)
// along a; B~a (a-faces) along b; speeds: max over the two adjacent faces.
// The 12 reconstructions use the same compacted limiter as k_faces.
template <typename R>
struct EmfSrc {
    const R *p[6];      // v^a_L, v^a_R, v^b_L, v^b_R (a-faces, along b), B~b (along a), B~a (along b)
    int st[6];          // stencil stride of each source
};

template <typename R>
__device__ __forceinline__ void emf_pick(const EmfSrc<R> &S, int m, const R *&p, int &st)
{
    p = S.p[0];
    st = S.st[0];
#pragma unroll
    for (int u = 1; u < 6; ++u)
        if (m == u) {
            p = S.p[u];
            st = S.st[u];
        }
}

template <int E, int MK, typename R>
__device__ __forceinline__ void emf_body(const Geom &g, const Arrays<R> &A, long long t, LimScratch<R> &lsm)
{
    constexpr int a = (E + 1) % 3, b = (E + 2) % 3;
    int cnt[3], off[3];
    emf_space(g, E, cnt, off);
    const long long tot = (long long)cnt[0] * cnt[1] * cnt[2];
    const bool live = t < tot;
    int id;
    int ei, ej;
    {
        // 32-bit decomposition: the edge box lies inside the padded array
        const unsigned tt = live ? (unsigned)t : 0u, c0 = (unsigned)cnt[0], c1 = (unsigned)cnt[1];
        const unsigned r = tt / c0, r2 = r / c1;
        ei = off[0] + (int)(tt - r * c0);
        ej = off[1] + (int)(r - r2 * c1);
        id = gidx(g, ei, ej, off[2] + (int)r2);
    }
    const int order = g.order;
    const int sa = stride_of(g, a);
    const int sb = stride_of(g, b);
    using T = R;
    EmfSrc<R> S;
    S.p[0] = A.fv[a][0];
    S.p[1] = A.fv[a][1];
    S.p[2] = A.fv[a][2];
    S.p[3] = A.fv[a][3];
    S.p[4] = A.U[5 + b];
    S.p[5] = A.U[5 + a];
    S.st[0] = S.st[1] = S.st[2] = S.st[3] = sb;
    S.st[4] = sa;
    S.st[5] = sb;
    T Lv[6] = {}, Rv[6] = {};
    unsigned pend = 0;
    if (live) {
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            T q[6];
#pragma unroll
            for (int s = 0; s < 6; ++s)
                q[s] = S.p[m][id + (s - 3) * S.st[m]];
            bool okL, okR;
            const T d1 = q[2] - q[1], d2 = q[3] - q[2], d3 = q[4] - q[3];
            Lv[m] = mp5_try_d(q[0], q[1], q[2], q[3], q[4], d2, d1, okL, order);
            Rv[m] = mp5_try_d(q[5], q[4], q[3], q[2], q[1], -d2, -d3, okR, order);
            pend |= (okL ? 0u : 1u) << (2 * m);
            pend |= (okR ? 0u : 1u) << (2 * m + 1);
        }
    }
    constexpr bool PRE = sizeof(T) == 8;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if constexpr (PRE) {
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            lsm.res[w][lane][2 * m] = Lv[m];
            lsm.res[w][lane][2 * m + 1] = Rv[m];
        }
    }
    compact_limit<PRE, T>(pend, id, lsm, [&](int ido, int m, int side, T uor) -> T {
        const R *p;
        int st;
        emf_pick(S, m, p, st);
        const int s0 = side ? 2 * st : -3 * st, ds = side ? -st : st;
        T q[5];
#pragma unroll
        for (int s = 0; s < 5; ++s)
            q[s] = p[ido + s0 + s * ds];
        if constexpr (PRE)
            return mp5_limit_u(q[0], q[1], q[2], q[3], q[4], uor);
        else
            return mp5_limit(q[0], q[1], q[2], q[3], q[4], order);
    });
    if (!live)
        return;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        if (PRE || (pend & (1u << (2 * m))))
            Lv[m] = lsm.res[w][lane][2 * m];
        if (PRE || (pend & (1u << (2 * m + 1))))
            Rv[m] = lsm.res[w][lane][2 * m + 1];
    }
    // va[s][t]: a-face side s (0 L, 1 R), reconstructed along b to side t
    const T va[2][2] = {{Lv[0], Rv[0]}, {Lv[1], Rv[1]}};
    const T vb[2][2] = {{Lv[2], Rv[2]}, {Lv[3], Rv[3]}};
    const T Bb[2] = {Lv[4], Rv[4]};
    const T Ba[2] = {Lv[5], Rv[5]};
    const T apa = imax(A.ap[a][id - sb], A.ap[a][id]);
    const T ama = imax(A.am[a][id - sb], A.am[a][id]);
    const T apb = imax(A.ap[b][id - sa], A.ap[b][id]);
    const T amb = imax(A.am[b][id - sa], A.am[b][id]);
    // transport velocity alpha v - beta at the edge (E_x1 edges sit at x2-face
    // positions of the (x1, x2) plane, E_x2 edges at x1-face positions, E_x3
    // edges at the corners)
    T al = T(1), bea = T(0), beb = T(0);
    if constexpr (MK == 1) {
        const int ti = ej * A.met.np0 + ei;
        const MetOf<T> M(A.met);
        const MetPtOf<T> &mp = E == 0 ? M.F2[ti] : (E == 1 ? M.F1[ti] : M.K[ti]);
        al = mp.al;
        bea = a == 0 ? mp.b1 : T(0);
        beb = b == 0 ? mp.b1 : T(0);
    }
    T Est[2][2];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if constexpr (MK == 1)
                Est[s][u] = -((al * va[s][u] - bea) * Bb[s] - (al * vb[s][u] - beb) * Ba[u]);
            else
                Est[s][u] = -(va[s][u] * Bb[s] - vb[s][u] * Ba[u]);
        }
    const T sA = apa + ama, sB = apb + amb;
    if (is_pos(sA) && is_pos(sB)) {
        // the whole expression over the common denominator sA sB, nested so
        // that the weights are never formed: one division, one final product
        const T t0 = fma(apb, Est[0][0], amb * Est[0][1]);
        const T t1 = fma(apb, Est[1][0], amb * Est[1][1]);
        T u = fma(apa, t0, ama * t1);
        u = fma(apa * ama * sB, Bb[1] - Bb[0], u);
        u = fma(-(apb * amb * sA), Ba[1] - Ba[0], u);
        A.E[E][id] = u * fast_recip(sA * sB);
    } else {
        const T da = is_pos(sA) ? apa * ama / sA : T(0);
        const T db = is_pos(sB) ? apb * amb / sB : T(0);
        A.E[E][id] = T(0.25) * (Est[0][0] + Est[0][1] + Est[1][0] + Est[1][1]) + da * (Bb[1] - Bb[0])
                     - db * (Ba[1] - Ba[0]);
    }
}

template <int E, int MK, typename R>
__global__ void __launch_bounds__(128) k_emf(Geom g, Arrays<R> A)
{
    __shared__ LimScratch<R> lsm;
    emf_body<E, MK, R>(g, A, (long long)blockIdx.x * blockDim.x + threadIdx.x, lsm);
}

// ------------------------------------------------------------------ sources

// Geometric sources of the Valencia form on the stationary Kerr-Schild metric
// at a cell centre, times sqrt(gamma) (only beta^1 is non-zero and nothing
// depends on x3):
//   S(S_i) = 1/2 alpha W^jk d_i gamma_jk + S_1 d_i beta^1 - U d_i alpha     (i = 1, 2)
//   S(tau) = 1/2 beta^1 W^ik d_1 gamma_ik + W_1^j d_j beta^1 - S^j d_j alpha
// with W^jk = (rho h + b^2) W^2 v^j v^k + (p + b^2/2) gamma^jk - b^j b^k.
template <typename T, typename MP, typename MD>
__device__ __forceinline__ void ks_sources(const T P[8], T gr, const MP &mp, const MD &md, T src[5])
{
    const MKS<T> m(mp);
    const T v[3] = {P[1], P[2], P[3]}, B[3] = {P[5], P[6], P[7]};
    T vl[3], Bl[3];
    lower<T>(m, v, vl);
    lower<T>(m, B, Bl);
    const T p = P[4];
    const T v2 = vl[0] * v[0] + vl[1] * v[1] + vl[2] * v[2];
    const T B2 = Bl[0] * B[0] + Bl[1] * B[1] + Bl[2] * B[2];
    const T vB = vl[0] * B[0] + vl[1] * B[1] + vl[2] * B[2];
    const T iW2 = T(1) - v2;
    const T W = rsqrt(iW2);
    const T iW = iW2 * W;
    const T W2 = W * W;
    const T rhoh = P[0] + gr * p;
    const T b2 = B2 * iW2 + vB * vB;
    const T Zw = rhoh * W2;
    const T ZB = Zw + B2;
    T bu[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        bu[c] = B[c] * iW + W * vB * v[c];
    const T hw = (rhoh + b2) * W2;
    const T pt = p + T(0.5) * b2;
    const T W11 = hw * v[0] * v[0] + pt * m.i11 - bu[0] * bu[0];
    const T W13 = hw * v[0] * v[2] + pt * m.i13 - bu[0] * bu[2];
    const T W22 = hw * v[1] * v[1] + pt * m.i22 - bu[1] * bu[1];
    const T W33 = hw * v[2] * v[2] + pt * m.i33 - bu[2] * bu[2];
    const T W12 = hw * v[0] * v[1] - bu[0] * bu[1];
    const T W32 = hw * v[2] * v[1] - bu[2] * bu[1];
    const T Sl[3] = {ZB * vl[0] - vB * Bl[0], ZB * vl[1] - vB * Bl[1], ZB * vl[2] - vB * Bl[2]};
    const T Uen = Zw - p + T(0.5) * (B2 + B2 * v2 - vB * vB);
    T s[2];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const T wdg = W11 * md.dg11[d] + T(2) * W13 * md.dg13[d] + W22 * md.dg22[d] + W33 * md.dg33[d];
        s[d] = T(0.5) * m.al * wdg + Sl[0] * md.db1[d] - Uen * md.dal[d];
    }
    const T wdg1 = W11 * md.dg11[0] + T(2) * W13 * md.dg13[0] + W22 * md.dg22[0] + W33 * md.dg33[0];
    const T W1_1 = m.g11 * W11 + m.g13 * W13;
    const T W1_2 = m.g11 * W12 + m.g13 * W32;
    const T Su1 = m.i11 * Sl[0] + m.i13 * Sl[2];
    const T Su2 = m.i22 * Sl[1];
    const T st = T(0.5) * m.b1 * wdg1 + W1_1 * md.db1[0] + W1_2 * md.db1[1] - Su1 * md.dal[0]
                 - Su2 * md.dal[1];
    src[0] = T(0);
    src[1] = s[0] * m.sg;
    src[2] = s[1] * m.sg;
    src[3] = T(0);
    src[4] = st * m.sg;
}

// ------------------------------------------------------------------ update

// Flux difference + CT curl + SSP-RK3 stage combination (Shu & Osher 1988):
//   stage 0: U = U0 + dt L (U0 saved);  stage 1: U = 3/4 U0 + 1/4 (U + dt L);
//   stage 2: U = 1/3 U0 + 2/3 (U + dt L).
// stage < 0: write L in host layout to Lout instead (faces NG..NG+n along
// their axis; a face that is not evolved, e.g. on the polar axis, gets 0).
// Body over the linear index t of the (n0+1)(n1+1)(n2+1) box of cells and
// faces, x fastest.
template <typename R>
__device__ __forceinline__ R geom_idx(const Geom &g, int d);
template <>
__device__ __forceinline__ double geom_idx<double>(const Geom &g, int d) { return g.idx[d]; }
template <>
__device__ __forceinline__ float geom_idx<float>(const Geom &g, int d) { return g.idx_f[d]; }

// L(U) of the five cell variables of owned cell (i, j, k) at padded index
// id: minus the flux differences (order 1: of the corrected fluxes) plus the
// sources.
template <int MK, typename R>
__device__ __forceinline__ void cell_rate(const Geom &g, const Phys &ph, const Arrays<R> &A, int id, int i, int j,
                                          R rate[5])
{
    const int st[3] = {1, g.px, g.pxy};
    R src[5] = {R(0), R(0), R(0), R(0), R(0)};
    if constexpr (MK == 1) {
        R P[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            P[q] = A.P[q][id];
        const int ti = j * A.met.np0 + i;
        const MetOf<R> M(A.met);
        ks_sources(P, phys_gr<R>(ph), M.C[ti], M.dC[ti], src);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        R r = R(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const R *__restrict__ F = g.order ? A.Fc[d][q] : A.F[d][q];
            r -= (F[id + st[d]] - F[id]) * geom_idx<R>(g, d);
        }
        rate[q] = r + src[q];
    }
}

template <int MK, typename R>
__device__ __forceinline__ void update_body(const Geom &g, const Phys &ph, const Arrays<R> &A, int stage,
                                            double *Lout, long long t)
{
    const long long e0 = g.n[0] + 1, e1 = g.n[1] + 1;
    if (t >= e0 * e1 * (g.n[2] + 1))
        return;
    // 32-bit decomposition: the box lies inside the padded array
    const unsigned u = (unsigned)t, r = u / (unsigned)e0, r2 = r / (unsigned)e1;
    const int ti = (int)(u - r * (unsigned)e0);
    const int tj = (int)(r - r2 * (unsigned)e1);
    const int tk = (int)r2;
    const int i = NG + ti, j = NG + tj, k = NG + tk;
    const int id = gidx(g, i, j, k);
    const int st[3] = {1, g.px, g.pxy};
    const int own[3] = {ti < g.n[0], tj < g.n[1], tk < g.n[2]};
    const int ijk[3] = {i, j, k};
    const R dt = stage >= 0 ? (R)A.scal->dt : R(0);
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];

    if (own[0] && own[1] && own[2]) {
        R rate[5];
        cell_rate<MK, R>(g, ph, A, id, i, j, rate);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const R r = rate[q];
            if (stage < 0) {
                Lout[q * N + ((long long)tk * g.n[1] + tj) * g.n[0] + ti] = (double)r;
            } else {
                const R u = A.U[q][id];
                R un;
                if (stage == 0) {
                    A.U0[q][id] = u;
                    un = u + dt * r;
                } else if (stage == 1) {
                    un = R(0.75) * A.U0[q][id] + R(0.25) * (u + dt * r);
                } else {
                    un = R(1.0 / 3.0) * A.U0[q][id] + R(2.0 / 3.0) * (u + dt * r);
                }
                A.U[q][id] = un;
            }
        }
    }
    long long off = 5 * N;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int a = (d + 1) % 3, b = (d + 2) % 3;
        int e[3] = {g.n[0], g.n[1], g.n[2]};
        e[d] += 1;
        const bool trans_own = own[a] && own[b];
        const bool evolved = ijk[d] >= g.flo[d] && ijk[d] <= g.fhi[d];
        // order 1: E_b corrected along a = (b+2)%3, E_a along b = (a+1)%3
        const R *__restrict__ Eb = g.order ? A.Ec[b][1] : A.E[b];
        const R *__restrict__ Ea = g.order ? A.Ec[a][0] : A.E[a];
        if (trans_own) {
            R l = R(0);
            if (evolved) {
                // dB~^d/dt = -(d_a E_b - d_b E_a)
                const R dEb = (Eb[id + st[a]] - Eb[id]) * geom_idx<R>(g, a);
                const R dEa = (Ea[id + st[b]] - Ea[id]) * geom_idx<R>(g, b);
                l = -(dEb - dEa);
            }
            if (stage < 0) {
                // periodic duplicate face: same EMF values as the first face
                if (ijk[d] <= NG + g.n[d]) {
                    const bool dup = ijk[d] == NG + g.n[d] && g.bc[2 * d] == BC_PERIODIC;
                    R lo = l;
                    if (dup) {
                        const R dEb = (Eb[id + st[a]] - Eb[id]) * geom_idx<R>(g, a);
                        const R dEa = (Ea[id + st[b]] - Ea[id]) * geom_idx<R>(g, b);
                        lo = -(dEb - dEa);
                    }
                    Lout[off + ((long long)tk * e[1] + tj) * e[0] + ti] = (double)lo;
                }
            } else if (evolved) {
                const R u = A.U[5 + d][id];
                R un;
                if (stage == 0) {
                    A.U0[5 + d][id] = u;
                    un = u + dt * l;
                } else if (stage == 1) {
                    un = R(0.75) * A.U0[5 + d][id] + R(0.25) * (u + dt * l);
                } else {
                    un = R(1.0 / 3.0) * A.U0[5 + d][id] + R(2.0 / 3.0) * (u + dt * l);
                }
                A.U[5 + d][id] = un;
            }
        }
        off += (long long)e[0] * e[1] * e[2];
    }
}

// Flat metric: 8 blocks of 256 per SM (32 registers, full occupancy; the
// FP32 form streams and needs the warps in flight).  Kerr-Schild (sources):
// FP32 8 blocks (32 registers, a 28-byte spill: the latency-bound kernel
// gains more from the warps than it loses to the spill), FP64 3 blocks (the
// occupancy its registers give anyway; that form is bound by the FP64 pipe).
template <int MK, typename R>
__global__ void __launch_bounds__(256, MK == 0 ? 8 : (sizeof(R) == 4 ? 8 : 3))
    k_update(Geom g, Phys ph, Arrays<R> A, int stage, double *Lout)
{
    update_body<MK, R>(g, ph, A, stage, Lout, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---- order 1: admissibility safeguard of the flux-derivative correction
//
// Pass `pass` (0 .. GUARD_PASSES-1) of a stage: every owned cell not yet
// flagged forms its stage result as k_update will (stage 0: U + dt L;
// 1: 3/4 U0 + 1/4 (U + dt L); 2: 1/3 U0 + 2/3 (U + dt L)) from L(U) with the
// current (corrected, or already returned) fluxes, with the cell-centre
// field of the current state, and is flagged if the FP64 Newton inversion
// from its Z cannot invert it; k_guard_revert then gives every face of a
// flagged cell its uncorrected flux.  A pass after one that flagged nothing
// returns at once.  The stage step dt is the device's.
constexpr int GUARD_PASSES = 3;

template <int MK, typename R>
__global__ void __launch_bounds__(128) k_guard_mark(Geom g, Phys ph, Arrays<R> A, int stage, int pass)
{
    if (pass > 0 && A.scal->guard_new[pass - 1] == 0ULL)
        return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    C2PCell c;
    if (!c2p_cell<MK, R>(g, A, t, c) || A.gmark[c.id])
        return;
    const int id = c.id;
    R rate[5];
    cell_rate<MK, R>(g, ph, A, id, c.i, c.j, rate);
    const R dt = (R)A.scal->dt;
    const R wa = stage == 0 ? R(0) : (stage == 1 ? R(0.75) : R(1.0 / 3.0));
    const R wb = stage == 0 ? R(1) : (stage == 1 ? R(0.25) : R(2.0 / 3.0));
    double u[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const R fe = A.U[q][id] + dt * rate[q];
        u[q] = to_d(stage == 0 ? fe : wa * A.U0[q][id] + wb * fe);
    }
    // undensitised, with the cell-centre field of the current state
    double S[3], B[3], Dc = u[0], tc = u[4];
    if constexpr (MK == 1) {
        const double isg = c.mp->isg;
        Dc *= isg;
        tc *= isg;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            S[q] = u[1 + q] * isg;
    } else {
#pragma unroll
        for (int q = 0; q < 3; ++q)
            S[q] = u[1 + q];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
        B[q] = to_d(A.P[5 + q][id]);
    constexpr double tol = sizeof(R) == 4 ? NEWTON_TOL_BULK32 : NEWTON_TOL;
    C2PResult r;
    if constexpr (MK == 1)
        r = c2p_newton(Dc, S, tc, B, A.Z[id], ph.gm1g, MKS<double>(*c.mp), NEWTON_MAXIT, false, tol);
    else
        r = c2p_newton(Dc, S, tc, B, A.Z[id], ph.gm1g, MFlat<double>(), NEWTON_MAXIT, false, tol);
    if (!r.ok) {
        A.gmark[id] = 1;
        atomicAdd(&A.scal->guard_new[pass], 1ULL);
    }
}

// Faces bounding a flagged cell (of the (n0+1)(n1+1)(n2+1) box, each
// direction's owned faces) take the uncorrected flux; a periodic axis pairs
// the faces across the seam with the cells they bound.  Counts the faces
// whose flux changed, the periodic duplicate face not again.
template <typename R>
__global__ void __launch_bounds__(256) k_guard_revert(Geom g, Arrays<R> A, int pass)
{
    if (A.scal->guard_new[pass] == 0ULL)
        return;
    const long long e0 = g.n[0] + 1, e1 = g.n[1] + 1;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= e0 * e1 * (g.n[2] + 1))
        return;
    const int tt[3] = {(int)(t % e0), (int)((t / e0) % e1), (int)(t / (e0 * e1))};
    unsigned long long changed = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        bool owned = true;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a != d && tt[a] >= g.n[a])
                owned = false;
        if (!owned)
            continue;
        const bool per = g.bc[2 * d] == BC_PERIODIC;
        bool f = false;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            int c[3] = {tt[0], tt[1], tt[2]};
            c[d] -= side == 0 ? 1 : 0;
            if (c[d] < 0 || c[d] >= g.n[d]) {
                if (!per)
                    continue;
                c[d] = (c[d] % g.n[d] + g.n[d]) % g.n[d];
            }
            f = f || A.gmark[gidx(g, NG + c[0], NG + c[1], NG + c[2])] != 0;
        }
        if (!f)
            continue;
        const int id = gidx(g, NG + tt[0], NG + tt[1], NG + tt[2]);
        bool ch = false;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const R v = A.F[d][q][id];
            ch = ch || A.Fc[d][q][id] != v;
            A.Fc[d][q][id] = v;
        }
        if (ch && !(per && tt[d] == g.n[d]))
            ++changed;
    }
    if (changed)
        atomicAdd(&A.scal->guard_faces, changed);
}

// Primitives (host layout, 5 arrays) + face B~ (already in U, ghosts
// filled) -> conserved cell variables (times sqrt(gamma)) and Z = rho h W^2.
template <int MK, typename R>
__global__ void k_p2c(Geom g, Phys ph, const double *prims5, Arrays<R> A)
{
    const int ti = blockIdx.x * blockDim.x + threadIdx.x;
    const int tj = blockIdx.y * blockDim.y + threadIdx.y;
    const int tk = blockIdx.z;
    if (ti >= g.n[0] || tj >= g.n[1] || tk >= g.n[2])
        return;
    const long long id = gidx(g, NG + ti, NG + tj, NG + tk);
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long h = ((long long)tk * g.n[1] + tj) * g.n[0] + ti;
    double isg = 1.0, sg = 1.0;
    const MetPt *mp = nullptr;
    if constexpr (MK == 1) {
        mp = &A.met.C[(NG + tj) * A.met.np0 + NG + ti];
        isg = mp->isg;
        sg = mp->sg;
    }
    double Bt[3];
    cell_centre_Bt(g, A, id, Bt);
    const double P8[8] = {prims5[h], prims5[N + h], prims5[2 * N + h], prims5[3 * N + h], prims5[4 * N + h],
                          Bt[0] * isg, Bt[1] * isg, Bt[2] * isg};
    double C5[5], Z;
    if constexpr (MK == 1)
        p2c_point(P8, ph.gr, MKS<double>(*mp), C5, Z);
    else
        p2c_point(P8, ph.gr, MFlat<double>(), C5, Z);
    for (int q = 0; q < 5; ++q)
        A.U[q][id] = (R)(C5[q] * sg);
    A.Z[id] = Z;
}

// ------------------------------------------------------------------ training
// pairs for the c2p-guess network

// One row per owned cell after a converged c2p: the network features of the
// conserved state and the targets log W, log(p/D), log(Z/D).  Rows go to
// offset + perm(c) * stride, with perm(c) = (c * 2654435761) mod N a
// permutation of the N cells (the multiplier is prime and larger than N),
// so one snapshot lands in a shuffled order.
template <int MK, typename R>
__global__ void k_mlp_dataset(Geom g, Arrays<R> A, float *X, float *Y, long long offset, long long stride)
{
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N)
        return;
    const int ti = (int)(c % g.n[0]);
    const long long rr = c / g.n[0];
    const int tj = (int)(rr % g.n[1]);
    const int tk = (int)(rr / g.n[1]);
    const int i = NG + ti, j = NG + tj, k = NG + tk;
    const long long id = gidx(g, i, j, k);
    const long long row = offset + (long long)(((unsigned long long)c * 2654435761ULL) % (unsigned long long)N) * stride;
    double isg = 1.0, sg = 1.0;
    const MetPt *mp = nullptr;
    if constexpr (MK == 1) {
        mp = &A.met.C[j * A.met.np0 + i];
        isg = mp->isg;
        sg = mp->sg;
    }
    const double B[3] = {0.5 * ((double)A.U[5][id] + (double)A.U[5][id + 1]) * isg,
                         0.5 * ((double)A.U[6][id] + (double)A.U[6][id + g.px]) * isg,
                         0.5 * ((double)A.U[7][id] + (double)A.U[7][id + g.pxy]) * isg};
    const double S[3] = {(double)A.U[1][id] * isg, (double)A.U[2][id] * isg, (double)A.U[3][id] * isg};
    const double Dc = (double)A.U[0][id] * isg, tc = (double)A.U[4][id] * isg;
    float f[MLP_NI];
    const double v[3] = {(double)A.P[1][id], (double)A.P[2][id], (double)A.P[3][id]};
    double vl[3];
    if constexpr (MK == 1) {
        mlp_features(Dc, S, tc, B, sg, MKS<double>(*mp), f);
        lower<double>(MKS<double>(*mp), v, vl);
    } else {
        mlp_features(Dc, S, tc, B, 1.0, MFlat<double>(), f);
        lower<double>(MFlat<double>(), v, vl);
    }
    for (int q = 0; q < MLP_NI; ++q)
        X[row * 9 + q] = f[q];
    const double v2 = vl[0] * v[0] + vl[1] * v[1] + vl[2] * v[2];
    const double W = 1.0 / sqrt(1.0 - v2);
    Y[row * 3 + 0] = (float)log(W);
    Y[row * 3 + 1] = (float)log((double)A.P[4][id] / Dc);
    Y[row * 3 + 2] = (float)log(A.Z[id] / Dc);
}

#ifdef ECHO_COMMON_KERNELS
// ------------------------------------------------------------------ scalars

__global__ void k_step_begin(DevScalars *s, double dt_fixed)
{
    s->rate_bits = 0ULL;
    s->dt = dt_fixed;
}

__global__ void k_set_dt(DevScalars *s, double cfl, int use_cfl)
{
    const double rate = __longlong_as_double((long long)s->rate_bits);
    s->totals[6] = rate;
    if (use_cfl)
        s->dt = rate > 0.0 ? cfl / rate : 0.0;
}

// ------------------------------------------------------------------ totals

// Sums of D, tau, S_i over owned cells and max |div B~|; per-block partials
// (6 per block) from a fixed shared-memory tree, then one block combines the
// partials in a fixed order.
template <typename R>
__global__ void __launch_bounds__(256) k_totals(Geom g, Arrays<R> A)
{
    __shared__ double sh[6][256];
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < N;
         t += (long long)gridDim.x * blockDim.x) {
        const int ti = (int)(t % g.n[0]);
        const long long r = t / g.n[0];
        const int tj = (int)(r % g.n[1]);
        const int tk = (int)(r / g.n[1]);
        const int id = gidx(g, NG + ti, NG + tj, NG + tk);
        acc[0] += (double)A.U[0][id];
        acc[1] += (double)A.U[4][id];
        acc[2] += (double)A.U[1][id];
        acc[3] += (double)A.U[2][id];
        acc[4] += (double)A.U[3][id];
        // div B~ from face differences (order 1: of the corrected face values,
        // the divergence that order keeps constant)
        double dv;
        if (g.order) {
            const int sd[3] = {1, g.px, g.pxy};
            dv = 0.0;
            for (int d = 0; d < 3; ++d) {
                const R *__restrict__ f = A.U[5 + d];
                const int s = sd[d];
                const double v[6] = {(double)f[id - 2 * s], (double)f[id - s], (double)f[id], (double)f[id + s],
                                     (double)f[id + 2 * s], (double)f[id + 3 * s]};
                dv += (ho_flux(v[1], v[2], v[3], v[4], v[5]) - ho_flux(v[0], v[1], v[2], v[3], v[4])) * g.idx[d];
            }
        } else {
            dv = ((double)A.U[5][id + 1] - (double)A.U[5][id]) * g.idx[0]
                 + ((double)A.U[6][id + g.px] - (double)A.U[6][id]) * g.idx[1]
                 + ((double)A.U[7][id + g.pxy] - (double)A.U[7][id]) * g.idx[2];
        }
        acc[5] = fmax(acc[5], fabs(dv));
    }
#pragma unroll
    for (int q = 0; q < 6; ++q)
        sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int q = 0; q < 5; ++q)
                sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
            sh[5][threadIdx.x] = fmax(sh[5][threadIdx.x], sh[5][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 6; ++q)
            A.partials[blockIdx.x * 6 + q] = sh[q][0];
}

__global__ void __launch_bounds__(256) k_totals_final(DevScalars *s, const double *partials, int nblk, double dV)
{
    __shared__ double sh[6][256];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
        for (int q = 0; q < 5; ++q)
            acc[q] += partials[b * 6 + q];
        acc[5] = fmax(acc[5], partials[b * 6 + 5]);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q)
        sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int q = 0; q < 5; ++q)
                sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
            sh[5][threadIdx.x] = fmax(sh[5][threadIdx.x], sh[5][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 5; ++q)
            s->totals[q] = sh[q][0] * dV;
        s->totals[5] = sh[5][0];
    }
}

// ------------------------------------------------------------------ layout

// Host layout (interior only, FP64) <-> padded arrays.  what: 0 = the five
// cell arrays and the three face arrays of U, 1 = the face arrays only.
template <typename R>
__global__ void k_unpack_state(Geom g, const double *src, Arrays<R> A, int what)
{
    const int ti = blockIdx.x * blockDim.x + threadIdx.x;
    const int tj = blockIdx.y * blockDim.y + threadIdx.y;
    const int tk = blockIdx.z;
    if (ti > g.n[0] || tj > g.n[1] || tk > g.n[2])
        return;
    const long long id = gidx(g, NG + ti, NG + tj, NG + tk);
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    const int t[3] = {ti, tj, tk};
    if (what == 0 && ti < g.n[0] && tj < g.n[1] && tk < g.n[2]) {
        const long long h = ((long long)tk * g.n[1] + tj) * g.n[0] + ti;
        for (int q = 0; q < 5; ++q)
            A.U[q][id] = (R)src[q * N + h];
    }
    const double *f = what == 0 ? src + 5 * N : src;
    for (int d = 0; d < 3; ++d) {
        int e[3] = {g.n[0], g.n[1], g.n[2]};
        e[d] += 1;
        if (t[0] < e[0] && t[1] < e[1] && t[2] < e[2])
            A.U[5 + d][id] = (R)f[((long long)tk * e[1] + tj) * e[0] + ti];
        f += (long long)e[0] * e[1] * e[2];
    }
}

template <typename R>
__global__ void k_pack_state(Geom g, Arrays<R> A, double *dst)
{
    const int ti = blockIdx.x * blockDim.x + threadIdx.x;
    const int tj = blockIdx.y * blockDim.y + threadIdx.y;
    const int tk = blockIdx.z;
    if (ti > g.n[0] || tj > g.n[1] || tk > g.n[2])
        return;
    const long long id = gidx(g, NG + ti, NG + tj, NG + tk);
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    const int t[3] = {ti, tj, tk};
    if (ti < g.n[0] && tj < g.n[1] && tk < g.n[2]) {
        const long long h = ((long long)tk * g.n[1] + tj) * g.n[0] + ti;
        for (int q = 0; q < 5; ++q)
            dst[q * N + h] = (double)A.U[q][id];
    }
    double *f = dst + 5 * N;
    for (int d = 0; d < 3; ++d) {
        int e[3] = {g.n[0], g.n[1], g.n[2]};
        e[d] += 1;
        if (t[0] < e[0] && t[1] < e[1] && t[2] < e[2])
            f[((long long)tk * e[1] + tj) * e[0] + ti] = (double)A.U[5 + d][id];
        f += (long long)e[0] * e[1] * e[2];
    }
}

// Cell arrays -> host layout: what 0 = primitives (8 arrays), 1 = Z.
template <typename R>
__global__ void k_pack_cells(Geom g, Arrays<R> A, double *dst, int what)
{
    const int ti = blockIdx.x * blockDim.x + threadIdx.x;
    const int tj = blockIdx.y * blockDim.y + threadIdx.y;
    const int tk = blockIdx.z;
    if (ti >= g.n[0] || tj >= g.n[1] || tk >= g.n[2])
        return;
    const long long id = gidx(g, NG + ti, NG + tj, NG + tk);
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long h = ((long long)tk * g.n[1] + tj) * g.n[0] + ti;
    if (what == 0) {
        for (int q = 0; q < 8; ++q)
            dst[q * N + h] = (double)A.P[q][id];
    } else {
        dst[h] = A.Z[id];
    }
}

// The network-start list of a cold start: every owned cell, in order.
template <typename R>
__global__ void k_list_all(Geom g, Arrays<R> A)
{
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0)
        A.scal->nlist_count = (unsigned long long)N;
    if (t >= N)
        return;
    const int i = (int)(t % g.n[0]), j = (int)((t / g.n[0]) % g.n[1]), k = (int)(t / ((long long)g.n[0] * g.n[1]));
    A.nlist[t] = gidx(g, NG + i, NG + j, NG + k);
}

template <typename R>
__global__ void k_unpack_z(Geom g, const double *src, Arrays<R> A)
{
    const int ti = blockIdx.x * blockDim.x + threadIdx.x;
    const int tj = blockIdx.y * blockDim.y + threadIdx.y;
    const int tk = blockIdx.z;
    if (ti >= g.n[0] || tj >= g.n[1] || tk >= g.n[2])
        return;
    const long long id = gidx(g, NG + ti, NG + tj, NG + tk);
    const long long h = ((long long)tk * g.n[1] + tj) * g.n[0] + ti;
    A.Z[id] = src ? src[h] : 0.0;
}

// ---- order 1: flux-derivative correction (ho_flux) of the fluxes along
// their direction on the owned faces, and of each EMF along each of its two
// half-integer directions on the edges of owned cells.
template <typename R>
__global__ void __launch_bounds__(256) k_fcorr(Geom g, Arrays<R> A, int d)
{
    const long long c0 = g.n[0] + (d == 0), c1 = g.n[1] + (d == 1), c2 = g.n[2] + (d == 2);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= c0 * c1 * c2)
        return;
    const int id = gidx(g, NG + (int)(t % c0), NG + (int)((t / c0) % c1), NG + (int)(t / (c0 * c1)));
    const int s = stride_of(g, d);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const R *__restrict__ F = A.F[d][q];
        A.Fc[d][q][id] = ho_flux(F[id - 2 * s], F[id - s], F[id], F[id + s], F[id + 2 * s]);
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_ecorr(Geom g, Arrays<R> A, int e)
{
    const long long c0 = g.n[0] + (e != 0), c1 = g.n[1] + (e != 1), c2 = g.n[2] + (e != 2);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= c0 * c1 * c2)
        return;
    const int id = gidx(g, NG + (int)(t % c0), NG + (int)((t / c0) % c1), NG + (int)(t / (c0 * c1)));
    const int st[3] = {1, g.px, g.pxy};
    const R *__restrict__ E = A.E[e];
#pragma unroll
    for (int w = 0; w < 2; ++w) {
        const int s = st[(e + 1 + w) % 3];
        A.Ec[e][w][id] = ho_flux(E[id - 2 * s], E[id - s], E[id], E[id + s], E[id + 2 * s]);
    }
}

template <typename R>
void launch_correct(const Geom &g, const Arrays<R> &A, cudaStream_t s)
{
    for (int d = 0; d < 3; ++d) {
        const long long n = (long long)(g.n[0] + (d == 0)) * (g.n[1] + (d == 1)) * (g.n[2] + (d == 2));
        k_fcorr<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, A, d);
    }
    for (int e = 0; e < 3; ++e) {
        const long long n = (long long)(g.n[0] + (e != 0)) * (g.n[1] + (e != 1)) * (g.n[2] + (e != 2));
        k_ecorr<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, A, e);
    }
}
template void launch_correct<double>(const Geom &, const Arrays<double> &, cudaStream_t);
template void launch_correct<float>(const Geom &, const Arrays<float> &, cudaStream_t);

#endif  // ECHO_COMMON_KERNELS

}  // namespace echo
