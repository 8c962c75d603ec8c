// echo_kernels_common.cu -- metric-independent kernels (ghost fill, device
// scalars, totals, layout conversion) and their launchers.
#define ECHO_COMMON_KERNELS
#include "echo_kernels.cuh"

namespace echo {

namespace {
inline dim3 grid3(int nx, int ny, int nz, dim3 blk)
{
    return dim3((unsigned)((nx + blk.x - 1) / blk.x), (unsigned)((ny + blk.y - 1) / blk.y), (unsigned)nz);
}
}  // namespace

template <typename R>
void launch_fill(const Geom &g, const FillList<R> &L, cudaStream_t s)
{
    for (int d = 0; d < 3; ++d) {
        const long long tot = fill_count(g, d);
        k_fill<R><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(g, d, L);
    }
}

void launch_step_begin(DevScalars *sc, double dt_fixed, cudaStream_t s)
{
    k_step_begin<<<1, 1, 0, s>>>(sc, dt_fixed);
}

void launch_set_dt(DevScalars *sc, double cfl, int use_cfl, cudaStream_t s)
{
    k_set_dt<<<1, 1, 0, s>>>(sc, cfl, use_cfl);
}

template <typename R>
void launch_totals(const Geom &g, const Arrays<R> &A, int nblk, cudaStream_t s)
{
    k_totals<R><<<nblk, 256, 0, s>>>(g, A);
    k_totals_final<<<1, 256, 0, s>>>(A.scal, A.partials, nblk, g.dx[0] * g.dx[1] * g.dx[2]);
}

template <typename R>
void launch_unpack_state(const Geom &g, const double *src, const Arrays<R> &A, int what, cudaStream_t s)
{
    dim3 blk(32, 8, 1);
    k_unpack_state<R><<<grid3(g.n[0] + 1, g.n[1] + 1, g.n[2] + 1, blk), blk, 0, s>>>(g, src, A, what);
}

template <typename R>
void launch_pack_state(const Geom &g, const Arrays<R> &A, double *dst, cudaStream_t s)
{
    dim3 blk(32, 8, 1);
    k_pack_state<R><<<grid3(g.n[0] + 1, g.n[1] + 1, g.n[2] + 1, blk), blk, 0, s>>>(g, A, dst);
}

template <typename R>
void launch_pack_cells(const Geom &g, const Arrays<R> &A, double *dst, int what, cudaStream_t s)
{
    dim3 blk(32, 8, 1);
    k_pack_cells<R><<<grid3(g.n[0], g.n[1], g.n[2], blk), blk, 0, s>>>(g, A, dst, what);
}

template <typename R>
void launch_unpack_z(const Geom &g, const double *src, const Arrays<R> &A, cudaStream_t s)
{
    dim3 blk(32, 8, 1);
    k_unpack_z<R><<<grid3(g.n[0], g.n[1], g.n[2], blk), blk, 0, s>>>(g, src, A);
}

template <typename R>
void launch_list_all(const Geom &g, const Arrays<R> &A, cudaStream_t s)
{
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    k_list_all<R><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(g, A);
}

#define ECHO_INSTANTIATE_COMMON(R)                                                                          \
    template void launch_list_all<R>(const Geom &, const Arrays<R> &, cudaStream_t);                       \
    template void launch_fill<R>(const Geom &, const FillList<R> &, cudaStream_t);                         \
    template void launch_totals<R>(const Geom &, const Arrays<R> &, int, cudaStream_t);                    \
    template void launch_unpack_state<R>(const Geom &, const double *, const Arrays<R> &, int, cudaStream_t); \
    template void launch_pack_state<R>(const Geom &, const Arrays<R> &, double *, cudaStream_t);           \
    template void launch_pack_cells<R>(const Geom &, const Arrays<R> &, double *, int, cudaStream_t);      \
    template void launch_unpack_z<R>(const Geom &, const double *, const Arrays<R> &, cudaStream_t);

ECHO_INSTANTIATE_COMMON(double)
ECHO_INSTANTIATE_COMMON(float)

}  // namespace echo
