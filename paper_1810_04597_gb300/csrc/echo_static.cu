// echo_static.cu -- conserved totals of a device state, with no allocation.
//
// Some callers cannot allocate device memory when they want these numbers:
// a host application whose memory manager has reserved all of HBM for its
// own pool, or a monitoring hook that must leave the device's memory
// footprint unchanged while a large run sits close to the HBM limit.  For
// them, echo_totals_static computes the same totals as echo_reduce without a
// context and without any workspace: the caller passes only the state and a
// 6-double output, and the per-row partial sums live in the file-scope
// device array below (every GPU that loads the library holds it until the
// process exits).
//
// Scratch: ECHO_STATIC_MAX_ROWS rows x 6 doubles (3 MiB).  Every call writes
// the partials of rows [0, ny*nz) before reading them, so nothing needs to
// start at zero; the array keeps the last call's contents.  Calls that
// overlap on the GPU (two streams, two host threads) share the array and
// race: order them on one stream.
#include <mutex>

#include "../../include/echo.h"

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_row_partials[ECHO_STATIC_MAX_ROWS * 6];

std::mutex g_mutex;
double *g_scratch[kMaxDevices] = {nullptr};

// One warp per (j, k) row of the host-layout state: sums of D, tau, S_x,
// S_y, S_z and the max of |div B~| over the row (fixed shuffle tree).
__global__ void __launch_bounds__(256) k_row_totals(const double *state, int nx, int ny, int nz, double idx,
                                                    double idy, double idz, double *rows)
{
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= (long long)ny * nz)
        return;  // warp-uniform
    const int j = (int)(warp % ny);
    const int k = (int)(warp / ny);
    const long long N = (long long)nx * ny * nz;
    const double *bx = state + 5 * N;
    const double *by = bx + (long long)nz * ny * (nx + 1);
    const double *bz = by + (long long)nz * (ny + 1) * nx;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = lane; i < nx; i += 32) {
        const long long h = ((long long)k * ny + j) * nx + i;
        acc[0] += state[h];
        acc[1] += state[4 * N + h];
        acc[2] += state[N + h];
        acc[3] += state[2 * N + h];
        acc[4] += state[3 * N + h];
        const long long fx = ((long long)k * ny + j) * (nx + 1) + i;
        const long long fy = ((long long)k * (ny + 1) + j) * nx + i;
        const long long fz = ((long long)k * ny + j) * nx + i;
        const double dv = (bx[fx + 1] - bx[fx]) * idx + (by[fy + nx] - by[fy]) * idy
                          + (bz[fz + (long long)ny * nx] - bz[fz]) * idz;
        acc[5] = fmax(acc[5], fabs(dv));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int q = 0; q < 5; ++q)
            acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        acc[5] = fmax(acc[5], __shfl_xor_sync(0xffffffffu, acc[5], o));
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 6; ++q)
            rows[warp * 6 + q] = acc[q];
}

// One block combines the row partials in a fixed order.
__global__ void __launch_bounds__(1024) k_rows_final(const double *rows, int nrows, double dV, double *out)
{
    __shared__ double sh[6][1024];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
#pragma unroll
        for (int q = 0; q < 5; ++q)
            acc[q] += rows[r * 6 + q];
        acc[5] = fmax(acc[5], rows[r * 6 + 5]);
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
            out[q] = sh[q][0] * dV;
        out[5] = sh[5][0];
    }
}

// Device address of the scratch array on the current device, looked up
// once per device (cudaGetSymbolAddress with that device current) and
// cached for the life of the process; the cache does not survive a
// cudaDeviceReset of that device.
int scratch_for_current_device(int dev, double **out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return ECHO_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_row_partials) != cudaSuccess || !p)
            return ECHO_ECUDA;
        g_scratch[dev] = static_cast<double *>(p);
    }
    *out = g_scratch[dev];
    return ECHO_OK;
}

// True if p is device memory (or managed memory) of device dev: the kernels
// below dereference it, so pageable or page-locked host memory and memory
// of another device are rejected before anything is launched.
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // clear the error this query raised
        return false;
    }
    if (a.type == cudaMemoryTypeManaged)
        return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" int echo_totals_static(const double *state, const int *n, const double *dx, double *out6,
                                  void *cuda_stream)
{
    if (!state || !n || !dx || !out6)
        return ECHO_EINVAL;
    for (int d = 0; d < 3; ++d)
        if (n[d] < 1 || !(dx[d] > 0.0))
            return ECHO_EINVAL;
    const long long rows = (long long)n[1] * n[2];
    if (rows > ECHO_STATIC_MAX_ROWS)
        return ECHO_ERANGE;
    // an error left pending by earlier work belongs to its owner: report it
    // without clearing it and launch nothing
    if (cudaPeekAtLastError() != cudaSuccess)
        return ECHO_ECUDA;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return ECHO_ECUDA;
    }
    if (!on_device(state, dev) || !on_device(out6, dev))
        return ECHO_EINVAL;
    double *scratch = nullptr;
    const int rc = scratch_for_current_device(dev, &scratch);
    if (rc != ECHO_OK) {
        cudaGetLastError();
        return rc;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const unsigned blocks = (unsigned)((rows * 32 + 255) / 256);
    k_row_totals<<<blocks, 256, 0, s>>>(state, n[0], n[1], n[2], 1.0 / dx[0], 1.0 / dx[1], 1.0 / dx[2], scratch);
    if (cudaGetLastError() != cudaSuccess)
        return ECHO_ECUDA;
    k_rows_final<<<1, 1024, 0, s>>>(scratch, (int)rows, dx[0] * dx[1] * dx[2], out6);
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}
