// echo_launch.h -- host-side launch entry points of the kernels (internal).
#pragma once

#include <cuda_runtime.h>

namespace echo {

struct Geom;
struct Phys;
struct DevScalars;
template <typename R>
struct Arrays;

// Arrays whose ghost layers one fill pass updates.  comp: vector component
// held (-1 scalar), face: face direction of a face-centred array (-1 cell),
// dens: 1 if the array carries the factor sqrt(gamma) (the densitised face
// field), which is odd about a polar axis like the component normal to it.
template <typename R>
struct FillList {
    R *a[12];
    int comp[12];
    int face[12];
    int dens[12];
    int count;
};

template <typename R>
void launch_fill(const Geom &g, const FillList<R> &L, cudaStream_t s);
template <int MK, typename R>
void launch_c2p(const Geom &g, const Phys &ph, const Arrays<R> &A, int guess_mode, int want_rate, cudaStream_t s);
// guess modes 1, 5: the network's pass writing the listed cells' Newton starts (before launch_c2p)
template <int MK, typename R>
void launch_net_pass(const Geom &g, const Phys &ph, const Arrays<R> &A, int guess_mode, cudaStream_t s);
template <int MK, typename R>
void launch_faces(const Geom &g, const Phys &ph, const Arrays<R> &A, int d, cudaStream_t s);
template <int MK, typename R>
void launch_emf(const Geom &g, const Arrays<R> &A, int e, cudaStream_t s);
template <int MK, typename R>
void launch_update(const Geom &g, const Phys &ph, const Arrays<R> &A, int stage, double *Lout, cudaStream_t s);
template <int MK, typename R>
void launch_p2c(const Geom &g, const Phys &ph, const double *prims5, const Arrays<R> &A, cudaStream_t s);
template <int MK, typename R>
void launch_mlp_dataset(const Geom &g, const Arrays<R> &A, float *X, float *Y, long long offset, long long stride,
                        cudaStream_t s);
template <typename R>
void launch_totals(const Geom &g, const Arrays<R> &A, int nblk, cudaStream_t s);
// order 1: corrected fluxes (Fc) and EMFs (Ec) from F and E (6 launches)
template <typename R>
void launch_correct(const Geom &g, const Arrays<R> &A, cudaStream_t s);
// order 1: the admissibility safeguard of stage `stage` (2 memsets, 6 launches)
template <int MK, typename R>
void launch_guard(const Geom &g, const Phys &ph, const Arrays<R> &A, int stage, cudaStream_t s);
// the network-start list of a cold start (every owned cell)
template <typename R>
void launch_list_all(const Geom &g, const Arrays<R> &A, cudaStream_t s);
template <typename R>
void launch_unpack_state(const Geom &g, const double *src, const Arrays<R> &A, int what, cudaStream_t s);
template <typename R>
void launch_pack_state(const Geom &g, const Arrays<R> &A, double *dst, cudaStream_t s);
template <typename R>
void launch_pack_cells(const Geom &g, const Arrays<R> &A, double *dst, int what, cudaStream_t s);
template <typename R>
void launch_unpack_z(const Geom &g, const double *src, const Arrays<R> &A, cudaStream_t s);
void launch_step_begin(DevScalars *sc, double dt_fixed, cudaStream_t s);
struct MetTables;
void launch_metric_tables(const Geom &g, double spin, const MetTables &T, double rho_floor, double rho_pow,
                          double p_floor, double p_pow, cudaStream_t s);
void launch_set_dt(DevScalars *sc, double cfl, int use_cfl, cudaStream_t s);

}  // namespace echo
