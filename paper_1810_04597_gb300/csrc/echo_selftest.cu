// echo_selftest.cu -- self-check of device helpers that replace hardware
// instructions: the integer-pipe float <-> double conversions must equal the
// hardware casts bit for bit; the Newton-Raphson reciprocal must stay within
// 2 ulp of the IEEE quotient; the MP5 test decided from signs and exponents
// must agree with the product test.  Also a register-only FP64 FMA throughput probe
// whose measured rate is the FP64 roofline peak the benchmark reports
// against.
#include "../../include/echo.h"
#include "echo_device.cuh"

namespace echo {

__device__ __forceinline__ unsigned long long mix64(unsigned long long x)
{
    x += 0x9e3779b97f4a7c15ULL;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
    return x ^ (x >> 31);
}

// Thread i builds test values from a counter-based hash: random float bit
// patterns (every class), doubles spread over and beyond the float range,
// doubles exactly half-way between two floats, and signed zeros.
__global__ void k_check_conversions(long long n, unsigned long long seed, unsigned long long *mismatch)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const unsigned long long h = mix64(seed ^ (unsigned long long)i);
    unsigned long long bad = 0;
    // float -> double on an arbitrary float pattern
    {
        const float f = __uint_as_float((unsigned)h);
        const double a = f2d(f), b = (double)f;
        if (!(f != f)) {
            if (__double_as_longlong(a) != __double_as_longlong(b))
                ++bad;
        }
    }
    // double -> float: exponent near the float range, random mantissa
    {
        const unsigned long long e = 1023ULL - 160ULL + (h >> 52) % 320ULL;
        const unsigned long long m = mix64(h) & 0xfffffffffffffULL;
        const unsigned long long sgn = (h & 1ULL) << 63;
        const double x = __longlong_as_double((long long)(sgn | (e << 52) | m));
        if (__float_as_uint(d2f(x)) != __float_as_uint((float)x))
            ++bad;
        // exactly half-way between two floats (round-to-even case), and one ulp either side
        const unsigned long long tie = (m & ~0x1fffffffULL) | 0x10000000ULL;
        for (long long off = -1; off <= 1; ++off) {
            const double y = __longlong_as_double((long long)(sgn | (e << 52) | (tie + off)));
            if (__float_as_uint(d2f(y)) != __float_as_uint((float)y))
                ++bad;
        }
    }
    if (i == 0) {
        const double z[4] = {0.0, -0.0, 3.4028234663852886e38, -1.1754943508222875e-38};
        for (int k = 0; k < 4; ++k)
            if (__float_as_uint(d2f(z[k])) != __float_as_uint((float)z[k]))
                ++bad;
    }
    if (bad)
        atomicAdd(mismatch, bad);
}

// Largest distance in ulp between nr_recip(d) (STEPS 2) or nr_recip1(d)
// (STEPS 1) and the IEEE quotient 1/d over hashed d of both signs with
// exponents across [-300, 300].
template <int STEPS>
__global__ void k_check_recip(long long n, unsigned long long seed, unsigned long long *max_ulp)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const unsigned long long h = mix64(seed ^ (unsigned long long)i);
    const unsigned long long e = 1023ULL - 300ULL + (h >> 52) % 601ULL;
    const unsigned long long m = mix64(h) & 0xfffffffffffffULL;
    const double d = __longlong_as_double((long long)(((h & 1ULL) << 63) | (e << 52) | m));
    const double r = STEPS == 2 ? nr_recip(d) : nr_recip1(d);
    const long long a = __double_as_longlong(r), b = __double_as_longlong(1.0 / d);
    const unsigned long long dist = (unsigned long long)(a > b ? a - b : b - a);
    atomicMax(max_ulp, dist);
}

// scale2<E>(x) against the FP64 product x * 2^E for E = 2, 1, -1 on hashed
// x of both signs with exponents across [-1000, 1000] (products normal) and
// on signed zeros; counts the mismatching bit patterns.
__global__ void k_check_scale2(long long n, unsigned long long seed, unsigned long long *mismatch)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const unsigned long long h = mix64(seed ^ (unsigned long long)i);
    const unsigned long long e = 1023ULL - 1000ULL + (h >> 52) % 2001ULL;
    const unsigned long long m = mix64(h) & 0xfffffffffffffULL;
    const unsigned long long sign = (h & 1ULL) << 63;
    const double x = (i & 1023) == 0 ? __longlong_as_double((long long)sign)
                                      : __longlong_as_double((long long)(sign | (e << 52) | m));
    unsigned long long bad = 0;
    if (__double_as_longlong(scale2<2>(x)) != __double_as_longlong(x * 4.0))
        ++bad;
    if (__double_as_longlong(scale2<1>(x)) != __double_as_longlong(x * 2.0))
        ++bad;
    if (__double_as_longlong(scale2<-1>(x)) != __double_as_longlong(x * 0.5))
        ++bad;
    if (__double_as_longlong(alpha_times(x)) != __double_as_longlong(MP5_ALPHA * x))
        ++bad;
    if (bad)
        atomicAdd(mismatch, bad);
}

// mp5_accept<double>(a, b) (the MP5 test from signs and exponents) against
// the product test a * b <= eps on hashed pairs: exponent sums spread over
// [-60, 20] and concentrated on the band [-38, -31] around eps, both signs,
// random mantissas, and every 64th pair with a zero, a subnormal, a huge or
// a non-finite operand; counts the differing decisions.
__global__ void k_check_mp5_accept(long long n, unsigned long long seed, unsigned long long *mismatch)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const unsigned long long h = mix64(seed ^ (unsigned long long)i), g = mix64(h);
    const long long ea = -60 + (long long)((h >> 40) % 81ULL);
    const long long s = (h & 2ULL) ? -38 + (long long)((h >> 20) % 8ULL) : -60 + (long long)((h >> 20) % 81ULL);
    long long eb = s - ea;
    eb = eb < -1000 ? -1000 : (eb > 1000 ? 1000 : eb);
    const unsigned long long ma = g & 0xfffffffffffffULL, mb = mix64(g) & 0xfffffffffffffULL;
    double a = __longlong_as_double((long long)(((h & 1ULL) << 63) | ((unsigned long long)(1023 + ea) << 52) | ma));
    double b = __longlong_as_double((long long)(((h & 4ULL) << 61) | ((unsigned long long)(1023 + eb) << 52) | mb));
    if ((i & 63) == 0) {
        const int k = (int)((h >> 8) % 6ULL);
        const double sp[6] = {0.0, -0.0, 4.9e-324, 1e300, __longlong_as_double(0x7ff0000000000000LL),
                              __longlong_as_double((long long)0xfff0000000000000ULL)};
        if (h & 8ULL)
            a = sp[k];
        else
            b = sp[k];
    }
    if (mp5_accept<double>(a, b) != ile(a * b, MP5_EPS))
        atomicAdd(mismatch, 1ULL);
}

// FP64 fused multiply-add throughput: every thread runs 8 independent
// chains c <- c * c - c for `iters` rounds in registers (no memory traffic
// inside the loop) and writes one sum, so the compiler cannot drop the work.
// All three operands of each FMA are one register: FMAs that read three
// distinct 64-bit registers issue at 0.80-0.97 of the FP64 pipe's rate on
// GB300, this form at its full rate, which is the FP64 peak.  The chains
// start at (thread + chain + 1) * a with a small; two rounds map c to
// c - 2c^3 + c^4, so they shrink slowly towards 0 and stay finite and normal.
constexpr int kDfmaChains = 8;

// The loop counter is 32-bit (64-bit integer adds and compares can take
// FP64-pipe slots on GB300).
__global__ void __launch_bounds__(256) k_dfma_throughput(int iters, double a, double *out)
{
    double c[kDfmaChains];
#pragma unroll
    for (int q = 0; q < kDfmaChains; ++q)
        c[q] = (double)(threadIdx.x + q + 1) * a;
#pragma unroll 2
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kDfmaChains; ++q)
            c[q] = fma(c[q], c[q], -c[q]);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kDfmaChains; ++q)
        s += c[q];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace echo

extern "C" int echo_selftest_dfma_blocks(void)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)
                                                   != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return 4 * sms;
}

extern "C" int echo_selftest_dfma(long long iters, double *dev_out, double *flops, void *stream)
{
    const int blocks = echo_selftest_dfma_blocks();
    if (iters < 1 || iters > 0x7fffffffLL || !dev_out || blocks < 1)
        return ECHO_EINVAL;
    echo::k_dfma_throughput<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        (int)iters, 1e-6, dev_out);
    if (flops)
        *flops = 2.0 * echo::kDfmaChains * (double)iters * 256.0 * (double)blocks;
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}

extern "C" int echo_selftest_scale2(long long n, unsigned long long seed, unsigned long long *dev_mismatch,
                                    void *stream)
{
    if (n < 1 || !dev_mismatch)
        return ECHO_EINVAL;
    echo::k_check_scale2<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, seed,
                                                                                                   dev_mismatch);
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}

extern "C" int echo_selftest_mp5_accept(long long n, unsigned long long seed, unsigned long long *dev_mismatch,
                                        void *stream)
{
    if (n < 1 || !dev_mismatch)
        return ECHO_EINVAL;
    echo::k_check_mp5_accept<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n, seed, dev_mismatch);
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}

extern "C" int echo_selftest_recip(long long n, unsigned long long seed, unsigned long long *dev_max_ulp, void *stream)
{
    if (n < 1 || !dev_max_ulp)
        return ECHO_EINVAL;
    echo::k_check_recip<2><<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, seed,
                                                                                                    dev_max_ulp);
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}

extern "C" int echo_selftest_recip1(long long n, unsigned long long seed, unsigned long long *dev_max_ulp,
                                    void *stream)
{
    if (n < 1 || !dev_max_ulp)
        return ECHO_EINVAL;
    echo::k_check_recip<1><<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, seed,
                                                                                                    dev_max_ulp);
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}

extern "C" int echo_selftest_conversions(long long n, unsigned long long seed, unsigned long long *dev_mismatch,
                                         void *stream)
{
    if (n < 1 || !dev_mismatch)
        return ECHO_EINVAL;
    echo::k_check_conversions<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n, seed, dev_mismatch);
    return cudaGetLastError() == cudaSuccess ? ECHO_OK : ECHO_ECUDA;
}
