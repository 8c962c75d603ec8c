// echo_mlp.cuh -- the c2p-guess network on the device: features of a
// conserved state and the fused FP32 forward pass used inside the c2p
// kernel.  Training kernels are in echo_mlp.cu.
//
// Network 9 -> 64 -> 64 -> 3 (tanh), FP32.  Parameter block (floats):
//   W1 64x9 | b1 64 | W2 64x64 | b2 64 | W3 3x64 | b3 3   (4995 values)
//   then feature mean 9 | feature std 9 | target mean 3 | target std 3.
// Outputs (standardised): log W, log(p/D), and the predicted log10
// relative error of the guess Z0 = D W (1 + G/(G-1) (p/D) W).
#pragma once

#include "echo_device.cuh"

namespace echo {

constexpr int MLP_NI = 9, MLP_NH = 64, MLP_NO = 3;
constexpr int MLP_OW1 = 0;
constexpr int MLP_OB1 = MLP_OW1 + MLP_NH * MLP_NI;
constexpr int MLP_OW2 = MLP_OB1 + MLP_NH;
constexpr int MLP_OB2 = MLP_OW2 + MLP_NH * MLP_NH;
constexpr int MLP_OW3 = MLP_OB2 + MLP_NH;
constexpr int MLP_OB3 = MLP_OW3 + MLP_NO * MLP_NH;
constexpr int MLP_NPAR = MLP_OB3 + MLP_NO;   // 4995
constexpr int MLP_ONORM = MLP_NPAR;
constexpr int MLP_NNORM = 2 * MLP_NI + 2 * MLP_NO;   // 24
// log10 of the network's typical guess error (its gate), written by
// echo_mlp_calibrate; 0 (an error of 1) until calibrated
constexpr int MLP_OGATE = MLP_ONORM + MLP_NNORM;     // 5019
constexpr int MLP_BLOCK = 5024;                      // params + norm + gate, padded to 32
// training state: [params+norm (MLP_BLOCK) | Adam m (MLP_BLOCK) | Adam v (MLP_BLOCK)]
constexpr int MLP_STATE = 3 * MLP_BLOCK;

// Scale-free features of an undensitised conserved state (D, S_i, tau),
// contravariant B and the metric:  log(tau/D), log(1 + S^2/D^2),
// log(1 + B^2/D), (S.B)^2 / (S^2 B^2), alpha, log sqrt(gamma), beta_i beta^i,
// (gamma^11 + gamma^22 + gamma^33)/3, log(D)/10.
// FP32 inputs; the metric's members are FP32 or FP64 (converted on the
// integer pipe).
__device__ __forceinline__ float as_f(float x) { return x; }
__device__ __forceinline__ float as_f(double x) { return d2f(x); }

template <typename M>
__device__ __forceinline__ void mlp_features_f(float D, const float Sf[3], float tauf, const float Bf[3],
                                               float sqrtgf, const M &m, float f[9])
{
    float Su[3], Bl[3];
    float al = 1.0f, bb = 0.0f, tr = 1.0f;
    if constexpr (M::flat) {
        Su[0] = Sf[0];
        Su[1] = Sf[1];
        Su[2] = Sf[2];
        Bl[0] = Bf[0];
        Bl[1] = Bf[1];
        Bl[2] = Bf[2];
    } else {
        const float i11 = as_f(m.i11), i13 = as_f(m.i13), i22 = as_f(m.i22), i33 = as_f(m.i33);
        const float g11 = as_f(m.g11), g13 = as_f(m.g13), g22 = as_f(m.g22), g33 = as_f(m.g33);
        const float b1 = as_f(m.b1);
        Su[0] = i11 * Sf[0] + i13 * Sf[2];
        Su[1] = i22 * Sf[1];
        Su[2] = i13 * Sf[0] + i33 * Sf[2];
        Bl[0] = g11 * Bf[0] + g13 * Bf[2];
        Bl[1] = g22 * Bf[1];
        Bl[2] = g13 * Bf[0] + g33 * Bf[2];
        al = as_f(m.al);
        bb = g11 * b1 * b1;
        tr = (i11 + i22 + i33) * (1.0f / 3.0f);
    }
    const float S2 = Sf[0] * Su[0] + Sf[1] * Su[1] + Sf[2] * Su[2];
    const float B2 = Bl[0] * Bf[0] + Bl[1] * Bf[1] + Bl[2] * Bf[2];
    const float SB = Sf[0] * Bf[0] + Sf[1] * Bf[1] + Sf[2] * Bf[2];
    const float iD = 1.0f / D;
    f[0] = logf(fmaxf(tauf * iD, 1e-30f));
    f[1] = log1pf(S2 * iD * iD);
    f[2] = log1pf(B2 * iD);
    f[3] = SB * SB / (S2 * B2 + 1e-30f);
    f[4] = al;
    f[5] = logf(sqrtgf);
    f[6] = bb;
    f[7] = tr;
    f[8] = fminf(fmaxf(logf(D), -30.0f), 30.0f) * 0.1f;
}

// FP64 inputs, converted to FP32 on the integer pipe (d2f): the FP64 pipe
// is the scarce one.
template <typename M>
__device__ __forceinline__ void mlp_features(double Dc, const double S[3], double tau, const double B[3], double sqrtg,
                                             const M &m, float f[9])
{
    const float Sf[3] = {d2f(S[0]), d2f(S[1]), d2f(S[2])};
    const float Bf[3] = {d2f(B[0]), d2f(B[1]), d2f(B[2])};
    mlp_features_f(d2f(Dc), Sf, d2f(tau), Bf, d2f(sqrtg), m, f);
}

// Forward pass with the parameter block in shared memory; returns the
// de-standardised outputs (log W, log(p/D), log10 error).
__device__ __forceinline__ void mlp_infer(const float *__restrict__ P, const float f[9], float out[3])
{
    float x[MLP_NI];
#pragma unroll
    for (int i = 0; i < MLP_NI; ++i)
        x[i] = (f[i] - P[MLP_ONORM + i]) / P[MLP_ONORM + MLP_NI + i];
    float h1[MLP_NH];
#pragma unroll
    for (int j = 0; j < MLP_NH; ++j) {
        float s = P[MLP_OB1 + j];
#pragma unroll
        for (int i = 0; i < MLP_NI; ++i)
            s = fmaf(P[MLP_OW1 + j * MLP_NI + i], x[i], s);
        h1[j] = tanhf(s);
    }
    float o[MLP_NO] = {P[MLP_OB3], P[MLP_OB3 + 1], P[MLP_OB3 + 2]};
#pragma unroll 4
    for (int k = 0; k < MLP_NH; ++k) {
        const float4 *w = reinterpret_cast<const float4 *>(P + MLP_OW2 + k * MLP_NH);
        float s = P[MLP_OB2 + k];
#pragma unroll
        for (int j4 = 0; j4 < MLP_NH / 4; ++j4) {
            const float4 wv = w[j4];
            s = fmaf(wv.x, h1[4 * j4], s);
            s = fmaf(wv.y, h1[4 * j4 + 1], s);
            s = fmaf(wv.z, h1[4 * j4 + 2], s);
            s = fmaf(wv.w, h1[4 * j4 + 3], s);
        }
        const float h2 = tanhf(s);
#pragma unroll
        for (int q = 0; q < MLP_NO; ++q)
            o[q] = fmaf(P[MLP_OW3 + q * MLP_NH + k], h2, o[q]);
    }
#pragma unroll
    for (int q = 0; q < MLP_NO; ++q)
        out[q] = o[q] * P[MLP_ONORM + 2 * MLP_NI + MLP_NO + q] + P[MLP_ONORM + 2 * MLP_NI + q];
}

// ---- per-cell choice of the Newton start
//
// The previous-stage Z of a cell is a good start when the state moved
// little since the last inversion.  Every network-mode inversion records,
// per cell, the code q of that movement: q = e(Z) - e(|Z - Z_prev|) from the binary
// exponents e of the new Z and of its change, i.e. -log2 of the relative
// change within one (0: a change of order one, 254: a change below 2^-254,
// 255: no change; a cold start, Z_prev = 0, gives 0).  It estimates the
// error of the previous Z as the next start.  The network's third output is
// its own predicted log10 relative error o2; a cell takes the network start
// iff -o2 log2(10) > q + 1/2, i.e. the network predicts a smaller error.
constexpr unsigned char ZE_EXACT = 255;

__device__ __forceinline__ unsigned char ze_code(double Z, double zprev)
{
    // binary exponents from the high words (32-bit integer work)
    const double dz = Z - zprev;
    const unsigned dh = (unsigned)__double2hiint(dz) & 0x7fffffffu;
    if ((dh | (unsigned)__double2loint(dz)) == 0u)
        return ZE_EXACT;
    const int ez = (int)(((unsigned)__double2hiint(Z) >> 20) & 0x7ffu);
    const int ed = (int)(dh >> 20);
    const int q = ez - ed;
    return (unsigned char)(q < 0 ? 0 : (q > 254 ? 254 : q));
}

// A cell whose previous Z is at least as far off as the network's typical
// error (gate, log10) may gain from the network: q <= floor(-gate log2 10);
// the inversion lists those cells (Arrays::nlist) for the network's pass
// before the next one, and only they consult the network there.
__device__ __forceinline__ int ze_gate(float gate_log10)
{
    const float g = -gate_log10 * 3.32192809f;
    return g <= 0.0f ? 0 : (g >= 254.0f ? 254 : (int)g);
}

// With the FP32 refinement (guess mode +4) every start that the four FP32
// Newton steps bring to FP32 accuracy costs the same one FP64 iteration, so
// only a previous Z that moved by about 1/8 or more (q <= 2) may gain from
// the network: from a relative error e the refinement leaves about e^16,
// which is below FP32 rounding for e < 1/4.
constexpr int ZE_REFINE_GATE = 2;

__device__ __forceinline__ int ze_gate_mode(float gate_log10, int guess_mode)
{
    const int g = ze_gate(gate_log10);
    return (guess_mode & 4) && g > ZE_REFINE_GATE ? ZE_REFINE_GATE : g;
}

__device__ __forceinline__ bool net_beats(float o2, unsigned char q)
{
    return q != ZE_EXACT && -o2 * 3.32192809f > (float)q + 0.5f;
}

// Append the padded index id of every lane with `want` to a list (one
// atomic per warp, lanes in lane order); every lane of the warp calls this.
__device__ __forceinline__ void list_append(bool want, int id, int *list, unsigned long long *count)
{
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m)
        return;
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == __ffs(m) - 1)
        base = atomicAdd(count, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    if (want)
        list[base + __popc(m & ((1u << lane) - 1u))] = id;
}

}  // namespace echo
