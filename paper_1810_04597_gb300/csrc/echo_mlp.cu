// echo_mlp.cu -- training of the c2p-guess network on the GPU: parameter
// initialisation, data standardisation, per-sample forward/backward,
// deterministic per-parameter gradient reduction, Adam (Kingma & Ba 2015),
// and a standalone forward pass.  All buffers are caller-owned.
//
// Loss per sample (standardised outputs o, targets t):
//   (o0 - t0)^2 + (o1 - t1)^2 + 0.1 (o2 - t2)^2, averaged over the batch,
// t0, t1 from log W and log(p/D) of the converged inversion; t2 is the log10
// relative error of the guess implied by o0, o1 (no gradient through t2).
#include <cstdint>

#include "../../include/echo.h"
#include "echo_mlp.cuh"
#include "echo_mlp_tc.cuh"

namespace echo {

static_assert(MLP_BLOCK == ECHO_MLP_BLOCK && MLP_STATE == ECHO_MLP_STATE && MLP_NPAR == ECHO_MLP_NPARAM,
              "network block layout of echo.h");
static_assert(MLP_OGATE == ECHO_MLP_GATE, "gate slot of echo.h");

constexpr int WS = 272;   // per-sample work floats
constexpr int W_XS = 0, W_H1 = 9, W_H2 = 73, W_D1 = 137, W_D2 = 201, W_D3 = 265, W_LOSS = 268;
constexpr float LOSS_W2 = 0.1f;
constexpr int NORM_BLOCKS = 304;

// splitmix64 (Steele, Lea & Flood 2014): a counter-based 64-bit generator.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    unsigned long long z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Glorot-uniform weights, zero biases, identity standardisation, zero Adam
// moments.
__global__ void k_mlp_init(float *S, unsigned long long seed)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= MLP_STATE)
        return;
    float v = 0.0f;
    if (p < MLP_NPAR) {
        int fan_in = 0, fan_out = 0;
        bool weight = true;
        if (p < MLP_OB1) {
            fan_in = MLP_NI;
            fan_out = MLP_NH;
        } else if (p < MLP_OW2) {
            weight = false;
        } else if (p < MLP_OB2) {
            fan_in = MLP_NH;
            fan_out = MLP_NH;
        } else if (p < MLP_OW3) {
            weight = false;
        } else if (p < MLP_OB3) {
            fan_in = MLP_NH;
            fan_out = MLP_NO;
        } else {
            weight = false;
        }
        if (weight) {
            const double u = (double)(splitmix64(seed ^ (0x5851f42d4c957f2dULL * (unsigned long long)(p + 1))) >> 11)
                             * (1.0 / 9007199254740992.0);
            const double a = sqrt(6.0 / (fan_in + fan_out));
            v = (float)((2.0 * u - 1.0) * a);
        }
    } else if (p < MLP_ONORM + MLP_NNORM) {
        const int q = p - MLP_ONORM;
        const bool is_std = (q >= MLP_NI && q < 2 * MLP_NI) || q >= 2 * MLP_NI + MLP_NO;
        v = is_std ? 1.0f : 0.0f;
    }
    S[p] = v;
}

// Per-block sums of x (9) and y (first 2) and their squares, in FP64.
__global__ void __launch_bounds__(256) k_mlp_moments(const float *x, const float *y, long long n, double *part)
{
    __shared__ double sh[22][256];
    double acc[22];
#pragma unroll
    for (int q = 0; q < 22; ++q)
        acc[q] = 0.0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double v = x[r * 9 + i];
            acc[i] += v;
            acc[11 + i] += v * v;
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const double v = y[r * 3 + i];
            acc[9 + i] += v;
            acc[20 + i] += v * v;
        }
    }
#pragma unroll
    for (int q = 0; q < 22; ++q)
        sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 22; ++q)
                sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 22; ++q)
            part[blockIdx.x * 22 + q] = sh[q][0];
}

// Combine the partials in a fixed order and write the standardisation block:
// mean and standard deviation of every feature and of log W, log(p/D); a
// (near-)constant column keeps std 1.  The error output is scaled as
// mean -4, std 2 (decades of relative error).
__global__ void k_mlp_moments_final(const double *part, int nblk, long long n, float *S)
{
    if (threadIdx.x != 0 || blockIdx.x != 0)
        return;
    double s[22];
    for (int q = 0; q < 22; ++q)
        s[q] = 0.0;
    for (int b = 0; b < nblk; ++b)
        for (int q = 0; q < 22; ++q)
            s[q] += part[b * 22 + q];
    for (int i = 0; i < 11; ++i) {
        const double mean = s[i] / (double)n;
        const double var = fmax(s[11 + i] / (double)n - mean * mean, 0.0);
        double sd = sqrt(var);
        if (!(sd > 1e-6 * fmax(1.0, fabs(mean))))
            sd = 1.0;
        if (i < 9) {
            S[MLP_ONORM + i] = (float)mean;
            S[MLP_ONORM + MLP_NI + i] = (float)sd;
        } else {
            S[MLP_ONORM + 2 * MLP_NI + (i - 9)] = (float)mean;
            S[MLP_ONORM + 2 * MLP_NI + MLP_NO + (i - 9)] = (float)sd;
        }
    }
    S[MLP_ONORM + 2 * MLP_NI + 2] = -4.0f;
    S[MLP_ONORM + 2 * MLP_NI + MLP_NO + 2] = 2.0f;
}

// Forward + backward of one sample per thread; rows row0 .. row0+batch-1
// (modulo n).  Stores standardised input, activations, deltas (already
// divided by the batch size) and the sample loss.
__global__ void __launch_bounds__(128) k_mlp_fwdbwd(const float *__restrict__ P, const float *__restrict__ x,
                                                    const float *__restrict__ y, long long n, long long row0,
                                                    int batch, float gr, float *__restrict__ work)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= batch)
        return;
    const long long r = (row0 + s) % n;
    float *w = work + (long long)s * WS;
    float xs[MLP_NI];
#pragma unroll
    for (int i = 0; i < MLP_NI; ++i) {
        xs[i] = (x[r * 9 + i] - P[MLP_ONORM + i]) / P[MLP_ONORM + MLP_NI + i];
        w[W_XS + i] = xs[i];
    }
    float h1[MLP_NH];
#pragma unroll
    for (int j = 0; j < MLP_NH; ++j) {
        float a = P[MLP_OB1 + j];
#pragma unroll
        for (int i = 0; i < MLP_NI; ++i)
            a = fmaf(P[MLP_OW1 + j * MLP_NI + i], xs[i], a);
        h1[j] = tanhf(a);
        w[W_H1 + j] = h1[j];
    }
    float o[MLP_NO] = {P[MLP_OB3], P[MLP_OB3 + 1], P[MLP_OB3 + 2]};
    for (int k = 0; k < MLP_NH; ++k) {
        float a = P[MLP_OB2 + k];
#pragma unroll
        for (int j = 0; j < MLP_NH; ++j)
            a = fmaf(P[MLP_OW2 + k * MLP_NH + j], h1[j], a);
        const float h2 = tanhf(a);
        w[W_H2 + k] = h2;
#pragma unroll
        for (int q = 0; q < MLP_NO; ++q)
            o[q] = fmaf(P[MLP_OW3 + q * MLP_NH + k], h2, o[q]);
    }
    const float *ym = P + MLP_ONORM + 2 * MLP_NI;
    const float *ys = ym + MLP_NO;
    float t[MLP_NO];
    t[0] = (y[r * 3 + 0] - ym[0]) / ys[0];
    t[1] = (y[r * 3 + 1] - ym[1]) / ys[1];
    {
        const double Wv = exp((double)(o[0] * ys[0] + ym[0]));
        const double pD = exp((double)(o[1] * ys[1] + ym[1]));
        const double z0 = Wv * (1.0 + (double)gr * pD * Wv);
        const double zs = exp((double)y[r * 3 + 2]);
        const double err = log10(fabs(z0 - zs) / zs + 1e-16);
        t[2] = (float)((err - (double)ym[2]) / (double)ys[2]);
    }
    const float wq[MLP_NO] = {1.0f, 1.0f, LOSS_W2};
    float d3[MLP_NO], loss = 0.0f;
    const float ib = 1.0f / (float)batch;
#pragma unroll
    for (int q = 0; q < MLP_NO; ++q) {
        const float e = o[q] - t[q];
        loss += wq[q] * e * e;
        d3[q] = 2.0f * wq[q] * e * ib;
        w[W_D3 + q] = d3[q];
    }
    w[W_LOSS] = loss * ib;
    // delta2 = (W3^T d3) (1 - h2^2)
    float d2[MLP_NH];
#pragma unroll
    for (int k = 0; k < MLP_NH; ++k) {
        const float h2 = w[W_H2 + k];
        float a = 0.0f;
#pragma unroll
        for (int q = 0; q < MLP_NO; ++q)
            a = fmaf(P[MLP_OW3 + q * MLP_NH + k], d3[q], a);
        d2[k] = a * (1.0f - h2 * h2);
        w[W_D2 + k] = d2[k];
    }
    // delta1 = (W2^T d2) (1 - h1^2)
    for (int j = 0; j < MLP_NH; ++j) {
        float a = 0.0f;
#pragma unroll
        for (int k = 0; k < MLP_NH; ++k)
            a = fmaf(P[MLP_OW2 + k * MLP_NH + j], d2[k], a);
        w[W_D1 + j] = a * (1.0f - h1[j] * h1[j]);
    }
}

// Gradient of the batch loss: one thread per parameter, summed over the
// batch in sample order (bitwise reproducible).
__global__ void __launch_bounds__(128) k_mlp_grad(const float *__restrict__ work, int batch, float *__restrict__ grad)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= MLP_NPAR)
        return;
    int od, oi;   // delta offset, input offset (-1: bias)
    if (p < MLP_OB1) {
        od = W_D1 + p / MLP_NI;
        oi = W_XS + p % MLP_NI;
    } else if (p < MLP_OW2) {
        od = W_D1 + (p - MLP_OB1);
        oi = -1;
    } else if (p < MLP_OB2) {
        const int q = p - MLP_OW2;
        od = W_D2 + q / MLP_NH;
        oi = W_H1 + q % MLP_NH;
    } else if (p < MLP_OW3) {
        od = W_D2 + (p - MLP_OB2);
        oi = -1;
    } else if (p < MLP_OB3) {
        const int q = p - MLP_OW3;
        od = W_D3 + q / MLP_NH;
        oi = W_H2 + q % MLP_NH;
    } else {
        od = W_D3 + (p - MLP_OB3);
        oi = -1;
    }
    float acc = 0.0f;
    for (int s = 0; s < batch; ++s) {
        const float *w = work + (long long)s * WS;
        acc = fmaf(w[od], oi >= 0 ? w[oi] : 1.0f, acc);
    }
    grad[p] = acc;
}

// Mean batch loss (fixed-order tree).
__global__ void __launch_bounds__(1024) k_mlp_loss(const float *work, int batch, float *loss)
{
    __shared__ double sh[1024];
    double a = 0.0;
    for (int s = threadIdx.x; s < batch; s += blockDim.x)
        a += work[(long long)s * WS + W_LOSS];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *loss = (float)sh[0];
}

// Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// theta -= lr (m/c1) / (sqrt(v/c2) + eps), c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void k_mlp_adam(float *S, const float *grad, float lr, float c1, float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= MLP_NPAR)
        return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float *m = S + MLP_BLOCK, *v = S + 2 * MLP_BLOCK;
    const float g = grad[p];
    const float mn = b1 * m[p] + (1.0f - b1) * g;
    const float vn = b2 * v[p] + (1.0f - b2) * g * g;
    m[p] = mn;
    v[p] = vn;
    S[p] -= lr * (mn / c1) / (sqrtf(vn / c2) + eps);
}

__global__ void __launch_bounds__(128) k_mlp_forward(const float *__restrict__ P, const float *__restrict__ x,
                                                     long long n, float *__restrict__ out)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n)
        return;
    float f[MLP_NI], o[MLP_NO];
#pragma unroll
    for (int i = 0; i < MLP_NI; ++i)
        f[i] = x[r * 9 + i];
    mlp_infer(P, f, o);
    // raw (standardised) outputs, as the oracle reports them
    for (int q = 0; q < MLP_NO; ++q)
        out[r * 3 + q] = (o[q] - P[MLP_ONORM + 2 * MLP_NI + q]) / P[MLP_ONORM + 2 * MLP_NI + MLP_NO + q];
}

// Forward pass with both hidden layers on the tensor cores (persistent CTAs
// of 128 rows); standardised outputs like k_mlp_forward, NaN where the
// tensor-core result did not arrive.
__global__ void __launch_bounds__(128) k_mlp_forward_tc(const float *__restrict__ P, const float *__restrict__ x,
                                                        long long n, float *__restrict__ out, long long ntiles)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    TcMlp t;
    tc_setup(t, tc_smem, P);
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long r = tile * 128 + threadIdx.x;
        float f[MLP_NI], o[MLP_NO];
#pragma unroll
        for (int i = 0; i < MLP_NI; ++i)
            f[i] = r < n ? x[r * 9 + i] : t.P[TP_NORM + i];
        const bool ok = tc_tile(t, f, o);
        if (r < n)
            for (int q = 0; q < MLP_NO; ++q)
                out[r * 3 + q] = ok ? (o[q] - t.P[TP_NORM + 2 * MLP_NI + q]) / t.P[TP_NORM + 2 * MLP_NI + MLP_NO + q]
                                    : __int_as_float(0x7fc00000);
    }
    tc_teardown(t);
}

// Relative error |Z0 - Z| / Z of the network's Newton start on each row,
// from its standardised outputs `out` (n x 3, as the forward kernels write
// them) and the rows' targets Y (log Z/D in column 2), in FP64:
// Z0 / D = W (1 + G/(G-1) (p/D) W) with the de-standardised log W, log(p/D).
__global__ void k_mlp_guess_error(const float *__restrict__ P, const float *__restrict__ out,
                                  const float *__restrict__ y, long long n, double gr, float *__restrict__ err)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n)
        return;
    const double lw = (double)out[r * 3] * P[MLP_ONORM + 2 * MLP_NI + MLP_NO] + P[MLP_ONORM + 2 * MLP_NI];
    const double lp = (double)out[r * 3 + 1] * P[MLP_ONORM + 2 * MLP_NI + MLP_NO + 1] + P[MLP_ONORM + 2 * MLP_NI + 1];
    const double W = exp(lw);
    const double z0 = W * (1.0 + gr * exp(lp) * W);
    const double z = exp((double)y[r * 3 + 2]);
    err[r] = (float)(fabs(z0 - z) / z);
}

// Mean of log10 of the rows' errors (clamped below at 1e-30) in FP64, one
// block in a fixed order, into the block's gate slot.
__global__ void __launch_bounds__(1024) k_mlp_gate(const float *__restrict__ err, long long n, float *S)
{
    __shared__ double sh[1024];
    double acc = 0.0;
    for (long long r = threadIdx.x; r < n; r += blockDim.x)
        acc += log10(fmax((double)err[r], 1e-30));
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        S[MLP_OGATE] = (float)(sh[0] / (double)n);
}

}  // namespace echo

using namespace echo;

namespace {
size_t work_floats(int batch) { return (size_t)batch * WS + MLP_BLOCK + 64; }
}  // namespace

extern "C" {

int echo_mlp_init(float *state, unsigned long long seed, void *stream)
{
    if (!state)
        return ECHO_EINVAL;
    k_mlp_init<<<(MLP_STATE + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(state, seed);
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}

size_t echo_mlp_work_bytes(int batch)
{
    const size_t a = work_floats(batch > 0 ? batch : 1) * sizeof(float);
    const size_t b = (size_t)NORM_BLOCKS * 22 * sizeof(double);
    return a > b ? a : b;
}

int echo_mlp_normalize(float *state, const float *x, const float *y, long long n, void *work, size_t work_bytes,
                       void *stream)
{
    if (!state || !x || !y || n < 1 || !work || work_bytes < (size_t)NORM_BLOCKS * 22 * sizeof(double))
        return ECHO_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *part = static_cast<double *>(work);
    k_mlp_moments<<<NORM_BLOCKS, 256, 0, s>>>(x, y, n, part);
    k_mlp_moments_final<<<1, 32, 0, s>>>(part, NORM_BLOCKS, n, state);
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}

int echo_mlp_grad(const float *state, const float *x, const float *y, long long n, long long row0, int batch,
                  double gamma, float *grad, float *loss, void *work, size_t work_bytes, void *stream)
{
    if (!state || !x || !y || !grad || n < 1 || batch < 1 || !work || work_bytes < echo_mlp_work_bytes(batch))
        return ECHO_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *w = static_cast<float *>(work);
    const float gr = (float)(gamma / (gamma - 1.0));
    k_mlp_fwdbwd<<<(batch + 127) / 128, 128, 0, s>>>(state, x, y, n, row0, batch, gr, w);
    k_mlp_grad<<<(MLP_NPAR + 127) / 128, 128, 0, s>>>(w, batch, grad);
    if (loss)
        k_mlp_loss<<<1, 1024, 0, s>>>(w, batch, loss);
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}

int echo_mlp_train(float *state, const float *x, const float *y, long long n, int batch, int nsteps, long long step0,
                   float lr, double gamma, void *work, size_t work_bytes, float *losses, void *stream)
{
    if (!state || !x || !y || n < 1 || batch < 1 || nsteps < 0 || step0 < 0 || !work
        || work_bytes < echo_mlp_work_bytes(batch))
        return ECHO_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *w = static_cast<float *>(work);
    float *grad = w + (size_t)batch * WS;
    const float gr = (float)(gamma / (gamma - 1.0));
    for (int it = 0; it < nsteps; ++it) {
        const long long t = step0 + it;
        const long long row0 = (t * (long long)batch) % n;
        k_mlp_fwdbwd<<<(batch + 127) / 128, 128, 0, s>>>(state, x, y, n, row0, batch, gr, w);
        k_mlp_grad<<<(MLP_NPAR + 127) / 128, 128, 0, s>>>(w, batch, grad);
        if (losses)
            k_mlp_loss<<<1, 1024, 0, s>>>(w, batch, losses + it);
        const double c1 = 1.0 - pow(0.9, (double)(t + 1));
        const double c2 = 1.0 - pow(0.999, (double)(t + 1));
        k_mlp_adam<<<(MLP_NPAR + 127) / 128, 128, 0, s>>>(state, grad, lr, (float)c1, (float)c2);
    }
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}

int echo_mlp_forward_tc(const float *state, const float *x, long long n, float *out, void *stream)
{
    if (!state || !x || !out || n < 0)
        return ECHO_EINVAL;
    if (n == 0)
        return ECHO_OK;
    static int resident = 0;
    if (resident == 0)
        resident = tc_resident_ctas((const void *)k_mlp_forward_tc, TC_SMEM);
    const long long ntiles = (n + 127) / 128;
    const long long grid = ntiles < resident ? ntiles : resident;
    k_mlp_forward_tc<<<(unsigned)grid, 128, TC_SMEM, static_cast<cudaStream_t>(stream)>>>(state, x, n, out, ntiles);
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}

int echo_mlp_forward(const float *state, const float *x, long long n, float *out, void *stream);

int echo_mlp_guess_error(const float *state, const float *x, const float *y, long long n, double gamma,
                         int tensor_cores, float *out, float *err, void *stream)
{
    if (!state || !x || !y || !out || !err || n < 0 || !(gamma > 1.0) || (tensor_cores != 0 && tensor_cores != 1))
        return ECHO_EINVAL;
    if (n == 0)
        return ECHO_OK;
    const int rc = tensor_cores ? echo_mlp_forward_tc(state, x, n, out, stream) : echo_mlp_forward(state, x, n, out, stream);
    if (rc != ECHO_OK)
        return rc;
    k_mlp_guess_error<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        state, out, y, n, gamma / (gamma - 1.0), err);
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}

int echo_mlp_calibrate(float *state, const float *x, const float *y, long long n, double gamma, float *out, float *err,
                       void *stream)
{
    if (n < 1)
        return ECHO_EINVAL;
    const int rc = echo_mlp_guess_error(state, x, y, n, gamma, 1, out, err, stream);
    if (rc != ECHO_OK)
        return rc;
    k_mlp_gate<<<1, 1024, 0, static_cast<cudaStream_t>(stream)>>>(err, n, state);
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}

int echo_mlp_forward(const float *state, const float *x, long long n, float *out, void *stream)
{
    if (!state || !x || !out || n < 0)
        return ECHO_EINVAL;
    if (n == 0)
        return ECHO_OK;
    k_mlp_forward<<<(unsigned)((n + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(state, x, n, out);
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}

}  // extern "C"
