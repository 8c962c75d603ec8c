// echo_mlp_tc.cuh -- the c2p-guess network with the products of both
// hidden layers (9 -> 64 and 64 -> 64) on the 5th-generation tensor cores
// (tcgen05), for CTAs of 128 threads that each own one row (one cell or one
// feature row).
//
// Per tile of 128 rows:
//   1. every thread standardises its 9 features in FP32 and writes them as
//      BF16 (K padded to 16 with zeros) into row `threadIdx.x` of the layer-1
//      A operand in shared memory;
//   2. one thread issues one tcgen05.mma (M = 128, N = 64, K = 16, BF16
//      inputs, FP32 accumulation) of X (128 x 16) by W1^T (16 x 64) into 64
//      TMEM columns and commits it to an mbarrier;
//   3. every thread waits for the mbarrier (bounded), reads its own TMEM lane
//      (row = thread: warp w owns lanes 32w..32w+31) with tcgen05.ld, adds
//      b1, applies tanh and writes h1 as BF16 into its row of the layer-2 A
//      operand;
//   4. one thread issues four tcgen05.mma (K = 16 each) of H1 (128 x 64) by
//      W2^T (64 x 64) into the same TMEM columns and commits them;
//   5. every thread waits, reads its lane, adds b2, applies tanh and
//      evaluates layer 3 (64 -> 3) in FP32.
// Operands use the no-swizzle K-major layout: 8 x 8 BF16 core matrices of
// 128 contiguous bytes, core matrix (row group, k group) at
// (row_group * KG + k_group) * 128 bytes with KG = K / 8, so the
// leading-dimension (K) byte offset is 128 and the stride (M/N) byte offset
// is KG * 128 (1024 for the 64-wide operands, 256 for the 16-wide ones).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>
#include <cstdio>
#include <cstdlib>

#include "echo_mlp.cuh"

namespace echo {

// FP32 parameters the CUDA cores need, packed (W1 and W2 live only as BF16):
// b1 (64), b2 (64), W3 (3x64), b3 (3), feature mean/std (9+9), target
// mean/std (3+3).
constexpr int TP_B1 = 0, TP_B2 = TP_B1 + MLP_NH, TP_W3 = TP_B2 + MLP_NH,
              TP_B3 = TP_W3 + MLP_NO * MLP_NH, TP_NORM = TP_B3 + MLP_NO, TP_COUNT = TP_NORM + MLP_NNORM;
constexpr int TC_A_BYTES = 128 * 64 * 2;            // h1 of 128 rows, BF16 (layer-2 A)
constexpr int TC_B_BYTES = 64 * 64 * 2;             // W2, BF16 (layer-2 B)
constexpr int TC_X_OFF = TC_A_BYTES + TC_B_BYTES;   // features of 128 rows, BF16, K = 16 (layer-1 A)
constexpr int TC_W1_OFF = TC_X_OFF + 128 * 16 * 2;  // W1, BF16, K = 16 (layer-1 B)
constexpr int TC_P_OFF = TC_W1_OFF + 64 * 16 * 2;   // packed FP32 parameters
constexpr int TC_BAR_OFF = TC_P_OFF + ((TP_COUNT * 4 + 15) / 16) * 16;
constexpr int TC_SMEM = TC_BAR_OFF + 16;            // + mbarrier (8 B) + TMEM address slot
constexpr uint32_t TC_TMEM_COLS = 64;
// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
// Bounded waits: give up after about a second at 2 GHz.
constexpr long long TC_WAIT_CYCLES = 1LL << 31;

__device__ __forceinline__ uint32_t tc_smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row r, column k) of a 64-column K-major operand.
__device__ __forceinline__ int tc_off(int r, int k)
{
    return ((r >> 3) * 8 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// The same for a 16-column operand (two core matrices per row group).
__device__ __forceinline__ int tc_off16(int r, int k)
{
    return ((r >> 3) * 2 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset >> 4 (bits 16-29), stride byte offset >> 4 (bits 32-45), the
// fixed version field 1 (bits 46-47), base offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t sbo = 1024)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32)
           | (1ull << 46);
}

__device__ __forceinline__ uint32_t tc_pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// tanh of the hidden layers: the hardware approximation (tanh.approx.f32,
// one SFU instruction, relative error about 2^-11 by the PTX ISA) instead
// of the accurate library tanhf (two SFU instructions and a dozen FMAs).
// The network only supplies the Newton start; its outputs move by ~1e-3,
// well inside the guess's own error.
__device__ __forceinline__ float tc_tanh(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(d_tmem), "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar)
                 : "memory");
}

// Wait for the mbarrier phase with parity `phase`; false after TC_WAIT_CYCLES.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t phase)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done)
            return true;
        if (clock64() - t0 > TC_WAIT_CYCLES)
            return false;
    }
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcMlp {
    unsigned char *base;   // layer-2 A operand at offset 0, B at TC_A_BYTES, layer-1 A and B at TC_X_OFF, TC_W1_OFF
    const float *P;        // packed FP32 parameters (TP_*) in shared memory
    uint32_t a_addr, b_addr, x_addr, w1_addr, bar, tmem, phase;
    bool ok;               // false after a wait gave up: no further MMA is issued
    bool pending;          // a commit that never arrived (waited for again at teardown)
};

// Copy the parameters, build W1 and W2 as BF16 B operands, initialise the
// mbarrier and allocate the TMEM columns.  All threads of the CTA call it.
__device__ __forceinline__ void tc_setup(TcMlp &t, unsigned char *smem, const float *__restrict__ gP)
{
    float *Ps = reinterpret_cast<float *>(smem + TC_P_OFF);
    for (int q = threadIdx.x; q < TP_COUNT; q += blockDim.x) {
        int src;
        if (q < TP_B2)
            src = MLP_OB1 + q;                          // b1
        else if (q < TP_NORM)
            src = MLP_OB2 + (q - TP_B2);                // b2, W3, b3 (contiguous)
        else
            src = MLP_ONORM + (q - TP_NORM);
        // the feature standard deviations are only divided by: keep 1/std
        const bool fstd = q >= TP_NORM + MLP_NI && q < TP_NORM + 2 * MLP_NI;
        Ps[q] = fstd ? 1.0f / gP[src] : gP[src];
    }
    // B = W2^T as a K-major operand: row n (hidden-2 unit) holds W2[n][0..63]
    for (int idx = threadIdx.x; idx < 64 * 8; idx += blockDim.x) {
        const int n = idx >> 3, kg = idx & 7;
        const float *w = gP + MLP_OW2 + n * MLP_NH + kg * 8;
        uint4 v;
        v.x = tc_pack_bf16(w[0], w[1]);
        v.y = tc_pack_bf16(w[2], w[3]);
        v.z = tc_pack_bf16(w[4], w[5]);
        v.w = tc_pack_bf16(w[6], w[7]);
        *reinterpret_cast<uint4 *>(smem + TC_A_BYTES + tc_off(n, kg * 8)) = v;
    }
    // layer-1 B = W1^T, K-major: row n holds W1[n][0..8], zeros up to K = 16
    for (int idx = threadIdx.x; idx < 64 * 2; idx += blockDim.x) {
        const int n = idx >> 1, kg = idx & 1;
        float w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = kg * 8 + u;
            w[u] = k < MLP_NI ? gP[MLP_OW1 + n * MLP_NI + k] : 0.0f;
        }
        uint4 v;
        v.x = tc_pack_bf16(w[0], w[1]);
        v.y = tc_pack_bf16(w[2], w[3]);
        v.z = tc_pack_bf16(w[4], w[5]);
        v.w = tc_pack_bf16(w[6], w[7]);
        *reinterpret_cast<uint4 *>(smem + TC_W1_OFF + tc_off16(n, kg * 8)) = v;
    }
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + TC_BAR_OFF + 8);
    t.bar = tc_smem_addr(smem + TC_BAR_OFF);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(t.bar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(tc_smem_addr(slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    t.tmem = *slot;
    t.base = smem;
    t.P = Ps;
    t.a_addr = tc_smem_addr(smem);
    t.b_addr = tc_smem_addr(smem + TC_A_BYTES);
    t.x_addr = tc_smem_addr(smem + TC_X_OFF);
    t.w1_addr = tc_smem_addr(smem + TC_W1_OFF);
    t.phase = 0;
    t.ok = true;
    t.pending = false;
}

// One round of MMAs: make the CTA's operand writes visible to the tensor
// core, let thread 0 issue `issue()` and commit it, and wait (bounded) for
// the commit.  Returns false on every thread if the result did not arrive
// (then no further MMA is issued and the commit is waited for again at
// teardown).
template <typename Issue>
__device__ __forceinline__ bool tc_round(TcMlp &t, Issue issue)
{
    tc_fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && t.ok) {
        tc_fence_after();
        issue();
        tc_commit(t.bar);
    }
    bool got = false;
    if (t.ok)
        got = tc_wait(t.bar, t.phase);
    got = __syncthreads_and(got) != 0;
    if (!got) {
        if (t.ok)
            t.pending = true;
        t.ok = false;
        return false;
    }
    t.phase ^= 1u;
    tc_fence_after();
    return true;
}

// One tile: every thread of the CTA passes its 9 features and receives the
// de-standardised outputs (log W, log(p/D), log10 guess error).  Returns
// false (the same on every thread) if a tensor-core result did not arrive.
__device__ __forceinline__ bool tc_tile(TcMlp &t, const float f[MLP_NI], float out[MLP_NO])
{
    const float *__restrict__ P = t.P;
    const int r = threadIdx.x;
    {
        float x[16];
#pragma unroll
        for (int i = 0; i < 16; ++i)
            x[i] = i < MLP_NI ? (f[i] - P[TP_NORM + i]) * P[TP_NORM + MLP_NI + i] : 0.0f;   // (f - mean) / std
#pragma unroll
        for (int kg = 0; kg < 2; ++kg) {
            uint4 v;
            v.x = tc_pack_bf16(x[kg * 8 + 0], x[kg * 8 + 1]);
            v.y = tc_pack_bf16(x[kg * 8 + 2], x[kg * 8 + 3]);
            v.z = tc_pack_bf16(x[kg * 8 + 4], x[kg * 8 + 5]);
            v.w = tc_pack_bf16(x[kg * 8 + 6], x[kg * 8 + 7]);
            *reinterpret_cast<uint4 *>(t.base + TC_X_OFF + tc_off16(r, kg * 8)) = v;
        }
    }
    // layer 1: X (128 x 16) W1^T -> TMEM
    if (!tc_round(t, [&] { tc_mma(t.tmem, tc_desc(t.x_addr, 256), tc_desc(t.w1_addr, 256), 0u); }))
        return false;
    const uint32_t lane = t.tmem + ((uint32_t)((threadIdx.x >> 5) * 32) << 16);
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
        uint32_t v[32];
        tc_ld32(lane + (uint32_t)(c * 32), v);
#pragma unroll
        for (int kg = 0; kg < 4; ++kg) {
            float h[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int n = c * 32 + kg * 8 + u;
                h[u] = tc_tanh(__uint_as_float(v[kg * 8 + u]) + P[TP_B1 + n]);
            }
            uint4 w;
            w.x = tc_pack_bf16(h[0], h[1]);
            w.y = tc_pack_bf16(h[2], h[3]);
            w.z = tc_pack_bf16(h[4], h[5]);
            w.w = tc_pack_bf16(h[6], h[7]);
            *reinterpret_cast<uint4 *>(t.base + tc_off(r, c * 32 + kg * 8)) = w;
        }
    }
    // layer 2: H1 (128 x 64) W2^T -> the same TMEM columns (every lane's
    // tcgen05.ld above completed before the barrier in tc_round)
    if (!tc_round(t, [&] {
#pragma unroll
            for (int kb = 0; kb < 4; ++kb)
                tc_mma(t.tmem, tc_desc(t.a_addr + kb * 256), tc_desc(t.b_addr + kb * 256), kb > 0 ? 1u : 0u);
        }))
        return false;
    float o0 = P[TP_B3], o1 = P[TP_B3 + 1], o2 = P[TP_B3 + 2];
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
        uint32_t v[32];
        tc_ld32(lane + (uint32_t)(c * 32), v);
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            const int n = c * 32 + u;
            const float h2 = tc_tanh(__uint_as_float(v[u]) + P[TP_B2 + n]);
            o0 = fmaf(P[TP_W3 + n], h2, o0);
            o1 = fmaf(P[TP_W3 + MLP_NH + n], h2, o1);
            o2 = fmaf(P[TP_W3 + 2 * MLP_NH + n], h2, o2);
        }
    }
    // the next tile's MMA overwrites these columns only after a barrier
    tc_fence_before();
    out[0] = o0 * P[TP_NORM + 2 * MLP_NI + MLP_NO] + P[TP_NORM + 2 * MLP_NI];
    out[1] = o1 * P[TP_NORM + 2 * MLP_NI + MLP_NO + 1] + P[TP_NORM + 2 * MLP_NI + 1];
    out[2] = o2 * P[TP_NORM + 2 * MLP_NI + MLP_NO + 2] + P[TP_NORM + 2 * MLP_NI + 2];
    return true;
}

// Wait (bounded) for a commit that had not arrived, then free the TMEM
// columns.  All threads of the CTA call it.
__device__ __forceinline__ void tc_teardown(TcMlp &t)
{
    if (t.pending && threadIdx.x == 0)
        tc_wait(t.bar, t.phase);
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(t.tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// CTAs of a 128-thread tensor-core kernel that fit on the whole GPU at once:
// the fewest that the registers, the shared memory (with the 1 KB the driver
// reserves per CTA) and the 512 TMEM columns of an SM allow.  (The runtime's
// occupancy calculator answers 1 CTA per SM for kernels that use tcgen05,
// which would leave 4 warps per SM.)  Set ECHO_VERBOSE to print the figures.
inline int tc_resident_ctas(const void *kernel, int smem)
{
    int dev = 0, sms = 0, smem_sm = 0, regs_sm = 0, calc = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaFuncAttributes fa{};
    const cudaError_t ea = cudaFuncGetAttributes(&fa, kernel);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&calc, kernel, 128, (size_t)smem);
    cudaGetLastError();
    const int regs = ea == cudaSuccess && fa.numRegs > 0 ? ((fa.numRegs + 7) / 8) * 8 : 128;
    const int by_regs = regs_sm / (regs * 128);
    const int by_smem = smem_sm / (smem + (int)fa.sharedSizeBytes + 1024);
    const int by_tmem = 512 / (int)TC_TMEM_COLS;
    int per_sm = by_regs < by_smem ? by_regs : by_smem;
    if (per_sm > by_tmem)
        per_sm = by_tmem;
    if (per_sm < 1)
        per_sm = 1;
    if (getenv("ECHO_VERBOSE"))
        fprintf(stderr,
                "echo: tensor-core kernel: %d regs, %d B smem; CTAs/SM by regs %d, smem %d, TMEM %d "
                "(occupancy calculator %d): %d x %d SMs\n",
                fa.numRegs, smem, by_regs, by_smem, by_tmem, calc, per_sm, sms);
    return per_sm * (sms > 0 ? sms : 1);
}

}  // namespace echo
