// echo_device.cuh -- device data structures and per-point physics of the
// GRMHD step on a flat or Kerr-Schild metric.  Included by the kernel
// translation units only.
//
// Arithmetic follows the published methods named in include/echo.h; it is
// written for the GPU (one division per reciprocal reused, rsqrt for the
// Lorentz factor, compile-time direction), so it differs from a textbook
// transcription only by rounding order.
#pragma once

#include <type_traits>

#include <cuda_runtime.h>
#include <stdint.h>

#include "echo.h"   // ECHO_C2P_HIST, the boundary's constants

namespace echo {

constexpr int NG = 5;              // ghost layers: MP5 needs 3 cells per side, the
                                   // high-order flux correction two more faces
constexpr double MP5_ALPHA = 4.0;  // Suresh & Huynh (1997) alpha
constexpr double MP5_EPS = 1e-10;  // Suresh & Huynh (1997) epsilon
constexpr double NEWTON_TOL = 1e-13;
// Stopping tolerance of the FP64 Newton iterations when the primitives are
// stored in FP32.  Newton converges quadratically: after a step with
// |dZ| <= 1e-6 Z the remaining relative error is O((dZ/Z)^2) ~ 1e-12 times
// the curvature factor, far below the 6e-8 rounding of the FP32 store, so
// the confirming iteration that the 1e-13 rule needs is skipped.
constexpr double NEWTON_TOL_BULK32 = 1e-6;
constexpr int NEWTON_MAXIT = 50;
constexpr int NEWTON_MAXHALF = 30;

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_AXIS = 2 };

// Geometry of the padded grid: every field (cell or face centred) is an
// array of np0*np1*np2 elements with row pitch px (>= np0) and plane pitch
// pxy = px*np1.  Face array d holds the face i-1/2 at index i along d.
struct Geom {
    int n[3];
    int np[3];
    // x and xy strides of the padded arrays; echo_init keeps cells_padded
    // below 2^31, so every offset into one array is an int
    int px, pxy;
    long long cells_padded;  // pxy * np2
    double dx[3];
    double idx[3];           // 1/dx
    float idx_f[3];          // 1/dx in FP32
    double x0[3];
    int bc[6];
    int flo[3], fhi[3];      // owned (evolved) face range along d, inclusive
    int order;               // 0 the scheme as read; 1 high order (flux-derivative correction)
};

__host__ __device__ __forceinline__ int gidx(const Geom &g, int i, int j, int k)
{
    return k * g.pxy + j * g.px + i;
}

// Ghost layers the scheme reads: 3 (MP5 stencils), 5 for order 1.
__host__ __device__ __forceinline__ int fill_layers(const Geom &g) { return 3 + 2 * g.order; }

// Threads of one ghost-fill launch along axis d (fill_body).
__host__ __device__ __forceinline__ long long fill_count(const Geom &g, int d)
{
    const int nl = fill_layers(g);
    const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
    return 2LL * nl * (g.n[d1] + 2 * nl) * (g.n[d2] + 2 * nl);
}

// Iteration space of the D-face kernel: cnt[a] indices from padded index
// off[a] on each axis.  Along D every face of an owned cell (order 1: two
// more on each side, for the flux correction); across, the faces whose
// velocities the EMF stencils (3 rows around the edges) read.
__host__ __device__ __forceinline__ void faces_space(const Geom &g, int D, int cnt[3], int off[3])
{
    const int w = 2 * g.order;
    for (int a = 0; a < 3; ++a) {
        cnt[a] = g.n[a] + 6 + 2 * w;
        off[a] = NG - 3 - w;
    }
    cnt[D] = g.n[D] + 1 + 2 * w;
    off[D] = NG - w;
}

// Iteration space of the E-edge kernel: the edges of owned cells (order 1:
// two more on each side across E, for the EMF correction).
__host__ __device__ __forceinline__ void emf_space(const Geom &g, int E, int cnt[3], int off[3])
{
    const int w = 2 * g.order;
    for (int a = 0; a < 3; ++a) {
        cnt[a] = g.n[a] + 1 + 2 * w;
        off[a] = NG - w;
    }
    cnt[E] = g.n[E];
    off[E] = NG;
}

// Flux-derivative correction at the middle of five interface values
// f_{-2} .. f_{+2}: f - D2/24 + 3 D4/640 (D2, D4 the second and fourth
// differences): the interface value of the function whose cell averages
// are the point values, so that its difference is the sixth-order
// derivative.
template <typename T>
__host__ __device__ __forceinline__ T ho_flux(T fm2, T fm1, T f0, T fp1, T fp2)
{
    const T d2 = fm1 - T(2) * f0 + fp1;
    const T d4 = fm2 - T(4) * fm1 + T(6) * f0 - T(4) * fp1 + fp2;
    return f0 - d2 * T(1.0 / 24.0) + d4 * T(3.0 / 640.0);
}

// Sixth-order interpolation to the midpoint of six equally spaced values:
// (3, -25, 150, 150, -25, 3) / 256.
template <typename T>
__host__ __device__ __forceinline__ T ho_center(T b0, T b1, T b2, T b3, T b4, T b5)
{
    return (T(3) * (b0 + b5) - T(25) * (b1 + b4) + T(150) * (b2 + b3)) * T(1.0 / 256.0);
}

struct Phys {
    double gamma;     // adiabatic index
    double gr;        // gamma / (gamma - 1)
    double gm1g;      // (gamma - 1) / gamma
    double cfl;
    float gamma_f, gr_f;   // the same constants in FP32 (no per-thread conversion)
};

template <typename T>
__device__ __forceinline__ T phys_gamma(const Phys &ph);
template <>
__device__ __forceinline__ double phys_gamma<double>(const Phys &ph) { return ph.gamma; }
template <>
__device__ __forceinline__ float phys_gamma<float>(const Phys &ph) { return ph.gamma_f; }
template <typename T>
__device__ __forceinline__ T phys_gr(const Phys &ph);
template <>
__device__ __forceinline__ double phys_gr<double>(const Phys &ph) { return ph.gr; }
template <>
__device__ __forceinline__ float phys_gr<float>(const Phys &ph) { return ph.gr_f; }

// Device-resident scalars of a context.
struct DevScalars {
    double dt;                   // dt of the running step
    unsigned long long rate_bits;  // max CFL rate (bits of a non-negative double)
    unsigned long long c2p_iters;
    unsigned long long c2p_calls;
    unsigned long long c2p_fail;
    unsigned long long floor_hits;
    unsigned long long fail_since_check;
    unsigned long long mlp_fallback;
    double totals[8];            // mass, energy, mom x3, max divB, rate, spare
    unsigned long long c2p_hist[ECHO_C2P_HIST];   // inversions by Newton iterations (last: that many or more)
    unsigned long long fallback_faces;  // first-order face fallbacks on faces bounding owned cells (sides)
    unsigned long long mlp_used;        // inversions started from the network's Newton start
    unsigned long long nlist_count;     // entries of Arrays::nlist
    unsigned long long guard_faces;     // order 1: faces the safeguard returned to the uncorrected flux
    unsigned long long guard_new[4];    // order 1: cells each safeguard pass of the running stage flagged
};

// Metric at one point of the axisymmetric (x1, x2) plane, FP64: lapse,
// shift^1 (the only non-zero shift component of Kerr-Schild), the non-zero
// spatial metric components gamma_11, _13, _22, _33, their inverse, and
// sqrt(gamma) with its reciprocal (0 on the polar axis).
struct MetPt {
    double al, b1, g11, g13, g22, g33, i11, i13, i22, i33, sg, isg;
};
// The same in FP32, for the FP32 kernels (rounded once when the tables are
// made, so that no kernel converts a metric value per cell).
struct MetPtF {
    float al, b1, g11, g13, g22, g33, i11, i13, i22, i33, sg, isg;
};

// d_1 and d_2 of alpha, beta^1, gamma_11, _13, _22, _33 at a cell centre
// (sixth-order centred differences of the closed form, step dx^d).
struct MetDer {
    double dal[2], db1[2], dg11[2], dg13[2], dg22[2], dg33[2];
};
struct MetDerF {
    float dal[2], db1[2], dg11[2], dg13[2], dg22[2], dg33[2];
};

// Tables over the padded (x1, x2) plane, index j * np0 + i: cell centres C,
// x1-faces F1 (i-1/2, j), x2-faces F2 (i, j-1/2), corners K (i-1/2, j-1/2);
// the x3-faces and x3-edges share C, F1/F2 and K positions.  floors: per i,
// the density and pressure floors at the cell centre.
struct MetTables {
    MetPt *C, *F1, *F2, *K;
    MetDer *dC;
    MetPtF *Cf, *F1f, *F2f, *Kf;   // FP32 copies (FP32 storage only, else null)
    MetDerF *dCf;
    double *floors;   // 2 * np0
    int np0;
    int use_floors;
};

// All device arrays of a context, R = storage type of the bulk fields.
template <typename R>
struct Arrays {
    R *U[8];       // conserved: D, S_x, S_y, S_z, tau (cell), B~x, B~y, B~z (faces)
    R *U0[8];      // RK base state
    double *Z;     // Newton memory (cell)
    float *zg;     // network Newton start per cell (> 0), or 0: the previous-stage Z chosen, < 0: the
                   // tensor-core result missing (previous Z, counted); written by k_mlp_guess_tc
    unsigned char *ze;     // per cell: code of the previous-Z error at the last inversion (ze_code)
    int *nlist;            // padded indices of the cells whose code reached the network's gate at the
                           // last inversion (the cells the next one may start from the network)
    unsigned char *gmark;  // order 1: cells the safeguard flagged in the running stage
    R *P[8];       // primitives rho, v^x, v^y, v^z, p, B^x, B^y, B^z (cell)
    R *F[3][5];    // HLL fluxes on d-faces
    R *ap[3];      // HLL a+ on d-faces
    R *am[3];      // HLL a- on d-faces
    R *fv[3][4];   // d-face states used by the EMFs: v^d_L, v^d_R, v^{d+1}_L, v^{d+1}_R
    R *E[3];       // edge EMFs: E_e at index (i,j,k) = edge at half-integer a, b
    R *Fc[3][5];   // order 1: corrected fluxes on the owned d-faces (else null)
    R *Ec[3][2];   // order 1: E_e corrected along (e+1)%3 [0] and (e+2)%3 [1]
    double *stage; // host-layout staging (FP64)
    double *partials;  // reduction partials
    DevScalars *scal;
    MetTables met; // Kerr-Schild tables (unused in flat space)
    const float *mlp;  // c2p-guess network block (params + standardisation)
};

// ------------------------------------------------------------------ exact
// comparisons on the integer pipe
//
// GB300 runs FP64 arithmetic, comparisons and min/max on a pipe ~70x slower
// than FP32, so sign tests, |x|, min/max and threshold tests are done on
// the IEEE-754 bit patterns instead (integer pipe).  For non-NaN values
// the map key(x) = bits ^ ((bits >> 63) & 0x7ff..f) is strictly monotonic
// in x (IEEE 754 total order of bit patterns), so every result below equals
// the floating-point comparison it replaces.  The FP64 forms work on the
// two 32-bit halves of the pattern (high word signed, low word unsigned,
// compared in that order): 64-bit integer compares, adds and masks issue on
// the FP64 pipe as well (ncu counts them with the DADDs), 32-bit ones on
// the integer ALU.

__device__ __forceinline__ long long bits_of(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ int bits_of(float x) { return __float_as_int(x); }

__device__ __forceinline__ long long okey(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ int okey(float x)
{
    const int b = __float_as_int(x);
    return b ^ ((b >> 31) & 0x7fffffff);
}
// key(x) as its two halves: (hi, lo), hi signed, lo unsigned
struct Key2 {
    int h;
    unsigned l;
};
__device__ __forceinline__ Key2 okey2(double x)
{
    const int h = __double2hiint(x);
    const unsigned l = (unsigned)__double2loint(x);
    const int s = h >> 31;
    return Key2{h ^ (s & 0x7fffffff), l ^ (unsigned)s};
}
__device__ __forceinline__ bool k2_lt(Key2 a, Key2 b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ bool k2_le(Key2 a, Key2 b) { return a.h < b.h || (a.h == b.h && a.l <= b.l); }
// x > 0 and x < 0 (strict; +0 and -0 are neither)
__device__ __forceinline__ bool is_pos(double x)
{
    const int h = __double2hiint(x);
    return h > 0 || (h == 0 && __double2loint(x) != 0);
}
__device__ __forceinline__ bool is_pos(float x) { return __float_as_int(x) > 0; }
__device__ __forceinline__ bool is_neg(double x)
{
    const int h = __double2hiint(x) ^ (int)0x80000000u;
    return h > 0 || (h == 0 && __double2loint(x) != 0);
}
__device__ __forceinline__ bool is_neg(float x) { return (__float_as_int(x) ^ (int)0x80000000u) > 0; }
__device__ __forceinline__ double iabs(double x)
{
    return __hiloint2double(__double2hiint(x) & 0x7fffffff, __double2loint(x));
}
__device__ __forceinline__ float iabs(float x) { return __int_as_float(__float_as_int(x) & 0x7fffffff); }
template <typename T>
__device__ __forceinline__ T imin(T a, T b) { return okey(a) < okey(b) ? a : b; }
template <typename T>
__device__ __forceinline__ T imax(T a, T b) { return okey(a) < okey(b) ? b : a; }
// a < b, a <= b
template <typename T>
__device__ __forceinline__ bool ilt(T a, T b) { return okey(a) < okey(b); }
template <typename T>
__device__ __forceinline__ bool ile(T a, T b) { return okey(a) <= okey(b); }
// FP32 has one-instruction min/max and comparisons on the fast pipes: use
// them (the integer form would cost 3-6 integer instructions each).  They
// differ from the integer forms only in the order of -0 and +0.
template <>
__device__ __forceinline__ float imin<float>(float a, float b) { return fminf(a, b); }
template <>
__device__ __forceinline__ float imax<float>(float a, float b) { return fmaxf(a, b); }
template <>
__device__ __forceinline__ bool ilt<float>(float a, float b) { return a < b; }
template <>
__device__ __forceinline__ bool ile<float>(float a, float b) { return a <= b; }
template <>
__device__ __forceinline__ double imin<double>(double a, double b) { return k2_lt(okey2(a), okey2(b)) ? a : b; }
template <>
__device__ __forceinline__ double imax<double>(double a, double b) { return k2_lt(okey2(a), okey2(b)) ? b : a; }
template <>
__device__ __forceinline__ bool ilt<double>(double a, double b) { return k2_lt(okey2(a), okey2(b)); }
template <>
__device__ __forceinline__ bool ile<double>(double a, double b) { return k2_le(okey2(a), okey2(b)); }
__device__ __forceinline__ double with_sign_of(double mag, double s)
{
    return __hiloint2double(__double2hiint(mag) | (__double2hiint(s) & (int)0x80000000u), __double2loint(mag));
}
__device__ __forceinline__ float with_sign_of(float mag, float s)
{
    return __int_as_float(__float_as_int(mag) | (__float_as_int(s) & (int)0x80000000u));
}

// Reciprocal 1/d by Newton-Raphson refinement of the hardware's approximate
// FP64 reciprocal (rcp.approx.ftz.f64): r <- r + r (1 - d r), two FMAs a
// step; each step squares the relative error, two reach the last bits of
// FP64 (within 2 ulp of the IEEE quotient, checked by
// echo_selftest_recip).  For normal, finite, non-zero d: 4 DFMA where an
// IEEE division costs about 8.6 DFMA slots on GB300.
__device__ __forceinline__ double nr_recip(double d)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

// 1/d after one refinement step of the same approximation: the step squares
// its relative error, leaving about 2^-39 (8773 ulp at most on 8 M hashed
// values, measured by echo_selftest_recip1).  For quotients whose accuracy
// only sets how fast an iteration converges, not what it converges to.
__device__ __forceinline__ double nr_recip1(double d)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    return fma(r, fma(-d, r, 1.0), r);
}

// n / d through nr_recip when |d| is safely normal, else the IEEE division.
// The product is rounded on its own (__dmul_rn is never fused into a
// neighbouring add), so, like a division, the result does not depend on how
// the compiler contracts the code around it (kernels that share this code
// stay bitwise equal).
__device__ __forceinline__ double nr_div(double n, double d)
{
    const double a = iabs(d);
    return (ilt(1e-200, a) && ilt(a, 1e200)) ? __dmul_rn(n, nr_recip(d)) : n / d;
}

// n / d through nr_recip1 (the same guards): a Newton step's quotient.
__device__ __forceinline__ double nr_step_div(double n, double d)
{
    const double a = iabs(d);
    return (ilt(1e-200, a) && ilt(a, 1e200)) ? __dmul_rn(n, nr_recip1(d)) : n / d;
}

// 1/x for the stencil: the IEEE division in FP64 (kernels that share the
// stencil code -- single runs and the batched schedules -- then agree
// bitwise); in FP32 the hardware reciprocal (MUFU, within 2 ulp for normal
// x) -- FP32 results are compared in L1 at 1e-5.
template <typename T>
__device__ __forceinline__ T fast_recip(T x);
template <>
__device__ __forceinline__ double fast_recip<double>(double x) { return 1.0 / x; }
template <>
__device__ __forceinline__ float fast_recip<float>(float x) { return __fdividef(1.0f, x); }


// ------------------------------------------------------------------ exact
// float <-> double conversions on the integer pipe
//
// GB300 executes F2F conversions on the FP64 pipe.  These build the IEEE 754
// binary64 / binary32 encodings directly (sign, re-biased exponent, shifted
// mantissa; round to nearest even when narrowing) and hand only zero-exponent
// (zero / subnormal), overflowing and non-finite values to the hardware
// conversion, so every result equals the hardware cast.  They work on the
// two 32-bit words of the binary64 encoding (64-bit integer operations
// would take the FP64 pipe too): the high word holds the sign, the exponent
// and the top 20 mantissa bits, the low word the other 32.

__device__ __forceinline__ double f2d(float x)
{
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) {
        if ((b & 0x7fffffffu) == 0u)
            return __hiloint2double((int)(b & 0x80000000u), 0);
        return (double)x;   // subnormal, inf, nan
    }
    // the 23 mantissa bits, shifted up by 29: the top 20 end the high word,
    // the low 3 start the low word
    const unsigned hi = (b & 0x80000000u) | ((e + (1023u - 127u)) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

__device__ __forceinline__ float d2f(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (e >= 1 && e <= 254) {
        // the top 23 of the 52 mantissa bits: 20 from the high word, 3 from the low
        unsigned r = (hi & 0x80000000u) | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
        const unsigned rem = lo & 0x1fffffffu;   // the 29 bits rounded away
        const unsigned half = 0x10000000u;
        r += (rem > half || (rem == half && (r & 1u))) ? 1u : 0u;   // carry may raise the exponent (to inf)
        return __uint_as_float(r);
    }
    if (((hi & 0x7fffffffu) | lo) == 0u)
        return __uint_as_float(hi & 0x80000000u);
    return (float)x;   // subnormal result, overflow, inf, nan
}

template <typename R>
__device__ __forceinline__ double to_d(R x) { return (double)x; }
template <>
__device__ __forceinline__ double to_d<float>(float x) { return f2d(x); }
template <typename R>
__device__ __forceinline__ R from_d(double x) { return (R)x; }
template <>
__device__ __forceinline__ float from_d<float>(double x) { return d2f(x); }

// ------------------------------------------------------------------ metric
// accessors.  MFlat is the Minkowski metric in Cartesian coordinates (every
// metric factor folds away at compile time); MKS holds one table point.

template <typename T>
struct MFlat {
    static constexpr bool flat = true;
};

template <typename T>
struct MKS {
    static constexpr bool flat = false;
    T al, b1, g11, g13, g22, g33, i11, i13, i22, i33, sg;
    // FP64 -> T through from_d (integer pipe for FP32)
    __device__ __forceinline__ explicit MKS(const MetPt &m)
        : al(from_d<T>(m.al)), b1(from_d<T>(m.b1)), g11(from_d<T>(m.g11)), g13(from_d<T>(m.g13)),
          g22(from_d<T>(m.g22)), g33(from_d<T>(m.g33)), i11(from_d<T>(m.i11)), i13(from_d<T>(m.i13)),
          i22(from_d<T>(m.i22)), i33(from_d<T>(m.i33)), sg(from_d<T>(m.sg))
    {
    }
    // from the FP32 copy of the table (no conversion in an FP32 kernel)
    __device__ __forceinline__ explicit MKS(const MetPtF &m)
        : al(m.al), b1(m.b1), g11(m.g11), g13(m.g13), g22(m.g22), g33(m.g33), i11(m.i11), i13(m.i13), i22(m.i22),
          i33(m.i33), sg(m.sg)
    {
    }
};

// The metric tables of storage type R: FP64 points for FP64 kernels, the
// FP32 copies for FP32 ones.
template <typename R>
using MetPtOf = std::conditional_t<sizeof(R) == 4, MetPtF, MetPt>;
template <typename R>
using MetDerOf = std::conditional_t<sizeof(R) == 4, MetDerF, MetDer>;
template <typename R>
struct MetOf {
    const MetPtOf<R> *C, *F1, *F2, *K;
    const MetDerOf<R> *dC;
    __device__ __forceinline__ explicit MetOf(const MetTables &T)
    {
        if constexpr (sizeof(R) == 4) {
            C = T.Cf;
            F1 = T.F1f;
            F2 = T.F2f;
            K = T.Kf;
            dC = T.dCf;
        } else {
            C = T.C;
            F1 = T.F1;
            F2 = T.F2;
            K = T.K;
            dC = T.dC;
        }
    }
};

template <typename T, typename M>
__device__ __forceinline__ void lower(const M &m, const T u[3], T d[3])
{
    if constexpr (M::flat) {
        d[0] = u[0];
        d[1] = u[1];
        d[2] = u[2];
    } else {
        d[0] = m.g11 * u[0] + m.g13 * u[2];
        d[1] = m.g22 * u[1];
        d[2] = m.g13 * u[0] + m.g33 * u[2];
    }
}

template <typename T, typename M>
__device__ __forceinline__ void raise(const M &m, const T d[3], T u[3])
{
    if constexpr (M::flat) {
        u[0] = d[0];
        u[1] = d[1];
        u[2] = d[2];
    } else {
        u[0] = m.i11 * d[0] + m.i13 * d[2];
        u[1] = m.i22 * d[1];
        u[2] = m.i13 * d[0] + m.i33 * d[2];
    }
}

// component D of gamma^{Dk} d_k
template <int D, typename T, typename M>
__device__ __forceinline__ T raise_c(const M &m, const T d[3])
{
    if constexpr (M::flat) {
        return d[D];
    } else {
        if constexpr (D == 0)
            return m.i11 * d[0] + m.i13 * d[2];
        else if constexpr (D == 1)
            return m.i22 * d[1];
        else
            return m.i13 * d[0] + m.i33 * d[2];
    }
}

template <int D, typename T, typename M>
__device__ __forceinline__ T gup(const M &m)
{
    if constexpr (M::flat)
        return T(1);
    else
        return D == 0 ? m.i11 : (D == 1 ? m.i22 : m.i33);
}

// ------------------------------------------------------------------ MP5

// minmod(a, b) = sign(a) min(|a|, |b|) if a, b have the same strict sign, else 0
template <typename T>
__device__ __forceinline__ T minmod2(T a, T b)
{
    const bool same = (is_pos(a) && is_pos(b)) || (is_neg(a) && is_neg(b));
    return same ? with_sign_of(imin(iabs(a), iabs(b)), a) : T(0);
}

// minmod of four: sign * min |.| if all four share a strict sign, else 0
template <typename T>
__device__ __forceinline__ T minmod4(T w, T x, T y, T z)
{
    const bool pos = is_pos(w) && is_pos(x) && is_pos(y) && is_pos(z);
    const bool neg = is_neg(w) && is_neg(x) && is_neg(y) && is_neg(z);
    const T m = imin(imin(iabs(w), iabs(x)), imin(iabs(y), iabs(z)));
    return (pos || neg) ? with_sign_of(m, w) : T(0);
}

// FP32 forms from one-instruction min/max (the integer sign tests above cost
// about a dozen integer instructions per call, and the FP32 stencil kernels
// are bound by the integer pipe): minmod of two is the median of (a, b, 0);
// minmod of four is max(min, 0) + min(max, 0), of which at most one term is
// non-zero.  Both select an argument exactly; only the sign of a zero result
// can differ from the forms above.
template <>
__device__ __forceinline__ float minmod2<float>(float a, float b)
{
    return fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.0f));
}

template <>
__device__ __forceinline__ float minmod4<float>(float w, float x, float y, float z)
{
    const float lo = fminf(fminf(w, x), fminf(y, z));
    const float hi = fmaxf(fmaxf(w, x), fmaxf(y, z));
    return fmaxf(lo, 0.0f) + fminf(hi, 0.0f);
}

// MP5 (Suresh & Huynh 1997): the interface value between u0 = u_j and
// up1 = u_{j+1}, biased to u_j -- the fifth-order interpolant of cell
// averages, kept inside the monotonicity- and accuracy-preserving interval.
// The GPU splits it for warp-uniform evaluation: mp5_try returns the
// unlimited value and whether the Suresh & Huynh test accepts it; mp5_limit
// returns the limited value for a rejected stencil (same uor).

// order 0: (2 u_{j-2} - 13 u_{j-1} + 47 u_j + 27 u_{j+1} - 3 u_{j+2}) / 60, the
// fifth-order interpolant of cell averages; order 1: (3, -20, 90, 60, -5) /
// 128, the fifth-order Lagrange interpolant of point values.  Weights
// pre-divided (5 FP64 operations).
template <typename T>
__device__ __forceinline__ T mp5_uor(T um2, T um1, T u0, T up1, T up2, int order)
{
    const T w0 = order ? T(3.0 / 128.0) : T(2.0 / 60.0);
    const T w1 = order ? T(-20.0 / 128.0) : T(-13.0 / 60.0);
    const T w2 = order ? T(90.0 / 128.0) : T(47.0 / 60.0);
    const T w3 = order ? T(60.0 / 128.0) : T(27.0 / 60.0);
    const T w4 = order ? T(-5.0 / 128.0) : T(-3.0 / 60.0);
    return fma(w0, um2, fma(w1, um1, fma(w2, u0, fma(w3, up1, w4 * up2))));
}

// Accept uor if (uor - u_j)(uor - u_mp) <= eps, u_mp = u_j + minmod(u_{j+1} - u_j,
// alpha (u_j - u_{j-1})); written with d0 = uor - u_j so that
// uor - u_mp = d0 - minmod(...).
// x 2^E for FP64 on the integer pipe, by adding E to the exponent field:
// the same bits as the FP64 product for zero and every normal x whose
// product is normal; a subnormal x (below 2^-1022 in magnitude, which none
// of the quantities scaled here ever is) gives a signed zero.  On GB300 an
// FP64 multiply takes a slot of the scarce FP64 pipe; where the product
// cannot fuse into an FMA this saves that slot.
template <int E>
__device__ __forceinline__ double scale2(double x)
{
    // on the high word only: the exponent field lies in it
    const int h = __double2hiint(x);
    const int l = __double2loint(x);
    const bool tiny = (h & 0x7ff00000) == 0;
    const int r = h + E * (1 << 20);
    return tiny ? __hiloint2double(h & (int)0x80000000u, 0) : __hiloint2double(r, l);
}

// alpha x for the MP5 test (alpha = 4 = 2^2): the product feeds a min/max,
// so it cannot fuse into an FMA.  FP64: scale2; FP32: the multiply.
static_assert(MP5_ALPHA == 4.0, "alpha_times assumes alpha = 4");
template <typename T>
__device__ __forceinline__ T alpha_times(T x) { return T(MP5_ALPHA) * x; }
template <>
__device__ __forceinline__ double alpha_times<double>(double x) { return scale2<2>(x); }

// dp = u_{j+1} - u_j and dm = u_j - u_{j-1} come from the caller, which
// shares them between the two states of a face: the right state's
// differences are the left stencil's negated (exact in IEEE arithmetic up to
// the sign of a zero, which minmod2 maps to 0 either way).
// The MP5 test a b <= eps with a = uor - u_j, b = a - minmod(...).  FP32:
// the product.  FP64: decided from the signs and binary exponents of a and b
// where that is exact -- a zero or opposite signs give a product <= 0; with
// unbiased exponents summing to s, |a b| lies in [2^s, 2^(s+2)), below eps
// (1e-10 > 2^-34) for s <= -36 and above it (2^-33 > 1e-10) for s >= -33 --
// and from the product itself only for s in {-35, -34} and non-normal
// operands, so the decision is the product's in every case.
template <typename T>
__device__ __forceinline__ bool mp5_accept(T a, T b) { return ile(a * b, T(MP5_EPS)); }
template <>
__device__ __forceinline__ bool mp5_accept<double>(double a, double b)
{
    static_assert(MP5_EPS == 1e-10, "the exponent bounds below assume eps = 1e-10");
    const int ha = __double2hiint(a), hb = __double2hiint(b);
    const bool za = ((ha & 0x7fffffff) | __double2loint(a)) == 0;
    const bool zb = ((hb & 0x7fffffff) | __double2loint(b)) == 0;
    if ((ha ^ hb) < 0 || za || zb)
        return true;
    const int ea = (ha >> 20) & 0x7ff, eb = (hb >> 20) & 0x7ff;
    if (ea != 0 && eb != 0 && ea != 0x7ff && eb != 0x7ff) {
        const int s = ea + eb - 2046;
        if (s <= -36)
            return true;
        if (s >= -33)
            return false;
    }
    return ile(a * b, MP5_EPS);
}

template <typename T>
__device__ __forceinline__ T mp5_try_d(T um2, T um1, T u0, T up1, T up2, T dp, T dm, bool &accept, int order)
{
    const T uor = mp5_uor(um2, um1, u0, up1, up2, order);
    const T d0 = uor - u0;
    const T mm = minmod2(dp, alpha_times(dm));
    accept = mp5_accept(d0, d0 - mm);
    return uor;
}

template <typename T>
__device__ __forceinline__ T mp5_try(T um2, T um1, T u0, T up1, T up2, bool &accept, int order)
{
    return mp5_try_d(um2, um1, u0, up1, up2, up1 - u0, u0 - um1, accept, order);
}

// The limited value given the unlimited one (uor = mp5_uor of the same stencil).
template <typename T>
__device__ __forceinline__ T mp5_limit_u(T um2, T um1, T u0, T up1, T up2, T uor)
{
    const T a4 = T(MP5_ALPHA) * (u0 - um1);
    const T dm1 = um2 - T(2) * um1 + u0;
    const T d0 = um1 - T(2) * u0 + up1;
    const T dp1 = u0 - T(2) * up1 + up2;
    const T dMp = minmod4(T(4) * d0 - dp1, T(4) * dp1 - d0, d0, dp1);
    const T dMm = minmod4(T(4) * d0 - dm1, T(4) * dm1 - d0, d0, dm1);
    const T uul = u0 + a4;
    const T uav = T(0.5) * (u0 + up1);
    const T umd = uav - T(0.5) * dMp;
    const T ulc = u0 + T(0.5) * (u0 - um1) + T(4.0 / 3.0) * dMm;
    const T umin = imax(imin(imin(u0, up1), umd), imin(imin(u0, uul), ulc));
    const T umax = imin(imax(imax(u0, up1), umd), imax(imax(u0, uul), ulc));
    return uor + minmod2(umin - uor, umax - uor);
}

template <typename T>
__device__ __forceinline__ T mp5_limit(T um2, T um1, T u0, T up1, T up2, int order)
{
    return mp5_limit_u(um2, um1, u0, up1, up2, mp5_uor(um2, um1, u0, up1, up2, order));
}

// ------------------------------------------------------------------ state

// Conserved vector, physical flux along D and HLL speeds of a primitive
// state P = (rho, v^1, v^2, v^3, p, B^1, B^2, B^3) (contravariant v, B),
// both vectors multiplied by sqrt(gamma) of the point (3+1 Valencia form):
//   D = rho W, S_j = (rho h W^2 + B^2) v_j - (v.B) B_j,
//   tau = rho h W^2 - p + (B^2 + B^2 v^2 - (v.B)^2)/2 - D;
//   F(D) = D (alpha v^d - beta^d),
//   F(S_j) = alpha [(rho h + b^2) W^2 v^d v_j + (p + b^2/2) delta^d_j - b^d b_j] - beta^d S_j,
//   F(tau) = alpha (S^d - D v^d) - beta^d tau,
// with b^i = B^i/W + W (v.B) v^i, b^2 = B^2/W^2 + (v.B)^2;
//   a^2 = c_s^2 + c_A^2 - c_s^2 c_A^2 = (G p + b^2)/(rho h + b^2),
//   lambda = alpha [v^d (1 - a^2) +- sqrt(a^2 (1-v^2)((1 - v^2 a^2) gamma^dd
//            - (1 - a^2)(v^d)^2))] / (1 - v^2 a^2) - beta^d.
// Returns the eigenvalues as lambda+- = np / Y, nm / Y (Y > 0 below), so
// that the caller can take the reciprocals of both states' Y with one
// division.
template <int D, typename T, typename M>
__device__ __forceinline__ void state_flux(const T P[8], T gam, T gr, const M &m, T F[5], T U[5], T &np, T &nm,
                                           T &Yout, const T *v2_known = nullptr)
{
    const T rho = P[0], p = P[4];
    const T v[3] = {P[1], P[2], P[3]};
    const T B[3] = {P[5], P[6], P[7]};
    T vl[3], Bl[3];
    lower<T>(m, v, vl);
    lower<T>(m, B, Bl);
    // v^2 as v_i v^i, or the caller's value of that same expression
    const T v2 = v2_known ? *v2_known : vl[0] * v[0] + vl[1] * v[1] + vl[2] * v[2];
    const T B2 = Bl[0] * B[0] + Bl[1] * B[1] + Bl[2] * B[2];
    const T vB = vl[0] * B[0] + vl[1] * B[1] + vl[2] * B[2];
    const T iW2 = T(1) - v2;
    const T W = rsqrt(iW2);
    const T iW = iW2 * W;
    const T W2 = W * W;
    const T rhoh = rho + gr * p;
    const T b2 = B2 * iW2 + vB * vB;
    const T Dn = rho * W;
    const T Zw = rhoh * W2;
    const T ZB = Zw + B2;
    U[0] = Dn;
#pragma unroll
    for (int j = 0; j < 3; ++j)
        U[1 + j] = ZB * vl[j] - vB * Bl[j];
    U[4] = Zw - p + T(0.5) * (B2 + B2 * v2 - vB * vB) - Dn;
    const T vd = v[D];
    const T Wvb = W * vB;
    const T bd = B[D] * iW + Wvb * vd;
    const T wt = (rhoh + b2) * W2 * vd;
    // With G = G p + b^2 and X = rho h + b^2 (a^2 = G/X), multiplying the
    // eigenvalue formula through by X leaves one division:
    //   lambda = alpha [v^d (rho h - G p) +- sqrt(G (1-v^2)(Y gamma^dd - (rho h - G p)(v^d)^2))] / Y
    //            - beta^d,  Y = X - v^2 G.
    const T Gs = gam * p + b2;
    const T Y = (rhoh + b2) - v2 * Gs;
    const T rmg = rhoh - gam * p;
    const T disc = Gs * iW2 * (Y * gup<D, T>(m) - rmg * vd * vd);
    // sqrt(disc) = disc rsqrt(disc): one rsqrt is cheaper than a sqrt
    const T sq = is_pos(disc) ? disc * rsqrt(disc) : T(0);
    const T base = vd * rmg;
    Yout = Y;
    // wt v_j - b^d b_j with b_j = B_j / W + W (v.B) v_j, regrouped as
    // c1 v_j - c2 B_j
    const T c1 = wt - bd * Wvb, c2 = bd * iW;
    if constexpr (M::flat) {
        F[0] = Dn * vd;
#pragma unroll
        for (int j = 0; j < 3; ++j)
            F[1 + j] = c1 * vl[j] - c2 * Bl[j] + (j == D ? p + T(0.5) * b2 : T(0));
        F[4] = U[1 + D] - Dn * vd;
        np = base + sq;
        nm = base - sq;
    } else {
        const T al = m.al;
        const T be = D == 0 ? m.b1 : T(0);
        F[0] = Dn * (al * vd - be);
#pragma unroll
        for (int j = 0; j < 3; ++j)
            F[1 + j] = al * (c1 * vl[j] - c2 * Bl[j] + (j == D ? p + T(0.5) * b2 : T(0))) - be * U[1 + j];
        const T Su[3] = {U[1], U[2], U[3]};
        F[4] = al * (raise_c<D, T>(m, Su) - Dn * vd) - be * U[4];
        np = al * (base + sq) - be * Y;
        nm = al * (base - sq) - be * Y;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            F[q] *= m.sg;
            U[q] *= m.sg;
        }
    }
}

// Sum over directions of max(|lambda+|, |lambda-|)/dx (CFL rate) of a cell
// (same eigenvalue form as state_flux) in T: FP64 for FP64 storage; with
// FP32 storage the speeds are evaluated in FP32 like the face speeds of that
// path, and only their max over cells (the reduction) is FP64.
template <typename M, typename T>
__device__ __forceinline__ T cfl_rate(const T P[8], T gam, T gr, const T idx[3], const M &m)
{
    const T v[3] = {P[1], P[2], P[3]}, B[3] = {P[5], P[6], P[7]};
    T vl[3], Bl[3];
    lower<T>(m, v, vl);
    lower<T>(m, B, Bl);
    const T p = P[4];
    const T v2 = vl[0] * v[0] + vl[1] * v[1] + vl[2] * v[2];
    const T B2 = Bl[0] * B[0] + Bl[1] * B[1] + Bl[2] * B[2];
    const T vB = vl[0] * B[0] + vl[1] * B[1] + vl[2] * B[2];
    const T iW2 = T(1) - v2;
    const T rhoh = P[0] + gr * p;
    const T b2 = B2 * iW2 + vB * vB;
    const T Gs = gam * p + b2;
    const T Y = (rhoh + b2) - v2 * Gs;
    const T rmg = rhoh - gam * p;
    const T iY = fast_recip(Y);
    T s = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        T gdd = T(1), al = T(1), be = T(0);
        if constexpr (!M::flat) {
            gdd = d == 0 ? m.i11 : (d == 1 ? m.i22 : m.i33);
            al = m.al;
            be = d == 0 ? m.b1 : T(0);
        }
        const T disc = Gs * iW2 * (Y * gdd - rmg * v[d] * v[d]);
        const T sq = is_pos(disc) ? disc * rsqrt(disc) : T(0);
        const T base = v[d] * rmg;
        T lp = (base + sq) * iY, lm = (base - sq) * iY;
        if constexpr (!M::flat) {
            lp = al * lp - be;
            lm = al * lm - be;
        }
        s += imax(iabs(lp), iabs(lm)) * idx[d];
    }
    return s;
}

// Conserved (undensitised, C5) and Z = rho h W^2 of cell primitives (FP64).
template <typename M>
__device__ __forceinline__ void p2c_point(const double P[8], double gr, const M &m, double C5[5], double &Z)
{
    const double v[3] = {P[1], P[2], P[3]}, B[3] = {P[5], P[6], P[7]};
    double vl[3], Bl[3];
    lower<double>(m, v, vl);
    lower<double>(m, B, Bl);
    const double v2 = vl[0] * v[0] + vl[1] * v[1] + vl[2] * v[2];
    const double B2 = Bl[0] * B[0] + Bl[1] * B[1] + Bl[2] * B[2];
    const double vB = vl[0] * B[0] + vl[1] * B[1] + vl[2] * B[2];
    const double W2 = 1.0 / (1.0 - v2);
    const double W = sqrt(W2);
    const double Zw = (P[0] + gr * P[4]) * W2;
    const double Dn = P[0] * W;
    C5[0] = Dn;
    for (int c = 0; c < 3; ++c)
        C5[1 + c] = (Zw + B2) * vl[c] - vB * Bl[c];
    C5[4] = Zw - P[4] + 0.5 * (B2 + B2 * v2 - vB * vB) - Dn;
    Z = Zw;
}

// ------------------------------------------------------------------ c2p

// Newton iteration on Z = rho h W^2 (FP64 always), with
// S^2 = gamma^ij S_i S_j, S.B = S_i B^i, B^2 = gamma_ij B^i B^j:
//   v^2(Z) = [S^2 Z^2 + (S.B)^2 (2Z + B^2)] / [Z^2 (Z + B^2)^2]
//   p(Z)   = (G-1)/G [Z (1 - v^2) - D sqrt(1 - v^2)]
//   f(Z)   = Z - p + (1 + v^2) B^2 / 2 - (S.B)^2 / (2 Z^2) - (tau + D)
// An inadmissible guess (Z <= 0 or v^2 >= 1) is replaced by doubling
// max(Z, tau + D); a step leaving the admissible set is halved (<= 30 times);
// stop at |dZ| <= tol Z (1e-13 by default) or after 50 iterations.
struct C2PResult {
    double rho, v[3], p, Z;
    int iters;
    bool ok;
};

// v^2 at Z from the reciprocals iZ = 1/Z, iZB = 1/(Z + B^2).
__device__ __forceinline__ double c2p_v2r(double Z, double iZ, double iZB, double S2, double SB2, double B2)
{
    return (S2 + SB2 * (2.0 * Z + B2) * iZ * iZ) * iZB * iZB;
}

// One division gives both reciprocals: 1/(Z (Z + B^2)).
__device__ __forceinline__ void c2p_recip(double Z, double B2, double &iZ, double &iZB)
{
    const double ZB = Z + B2;
    const double inv = nr_div(1.0, Z * ZB);
    iZ = inv * ZB;
    iZB = inv * Z;
}

// Optional FP32 pre-refinement of the guess: up to 4 Newton steps of the same
// residual in FP32 (stopping at |dZ| <= 4e-7 Z or at a step that leaves the
// admissible set).  It only moves the starting point; the FP64 iterations
// that follow decide convergence.  When it stops on the tolerance it also
// hands back f' and dv^2/dZ of its last step (fp_out, dv2_out), provided the
// terms of f' sum in absolute value to at most 1e3 |f'| (so that f' carries
// a relative error below about 1e-4); otherwise fp_out = 0.
__device__ __forceinline__ double c2p_refine_f32(double Zg, double S2d, double SB2d, double B2d, double Dd,
                                                 double Ud, double gm1gd, float &fp_out, float &dv2_out)
{
    const float S2 = d2f(S2d), SB2 = d2f(SB2d), B2 = d2f(B2d), D = d2f(Dd), U = d2f(Ud), gm1g = d2f(gm1gd);
    float Z = d2f(Zg);
    fp_out = 0.0f;
    dv2_out = 0.0f;
    for (int k = 0; k < 4; ++k) {
        const float iZ = 1.0f / Z, ZB = Z + B2, iZB = 1.0f / ZB;
        const float v2 = (S2 + SB2 * (2.0f * Z + B2) * iZ * iZ) * iZB * iZB;
        if (!(v2 < 1.0f) || !(Z > 0.0f))
            break;
        const float om = 1.0f - v2;
        const float isq = rsqrtf(om);
        const float p = gm1g * (Z * om - D * om * isq);
        const float f = Z - p + 0.5f * (1.0f + v2) * B2 - 0.5f * SB2 * iZ * iZ - U;
        const float dv2 = -2.0f * (S2 * Z * Z * Z + SB2 * (3.0f * Z * Z + 3.0f * Z * B2 + B2 * B2)) * iZ * iZ * iZ
                          * iZB * iZB * iZB;
        const float dp = gm1g * (om - Z * dv2 + 0.5f * D * dv2 * isq);
        const float fp = 1.0f - dp + 0.5f * B2 * dv2 + SB2 * iZ * iZ * iZ;
        const float dZ = f / fp;
        const float Zn = Z - dZ;
        if (!(Zn > 0.0f))
            break;
        if (fabsf(dZ) <= 4e-7f * Zn) {
            const float mag = 1.0f + gm1g * (om + fabsf(Z * dv2) + fabsf(0.5f * D * dv2 * isq))
                              + fabsf(0.5f * B2 * dv2) + SB2 * iZ * iZ * iZ;
            if (fabsf(fp) <= 1e35f && mag <= 1e3f * fabsf(fp)) {
                fp_out = fp;
                dv2_out = dv2;
            }
            Z = Zn;
            break;
        }
        Z = Zn;
    }
    return f2d(Z);
}

// F32D: the first FP64 step after an FP32 refinement that stopped on its
// tolerance takes f' and dv^2/dZ from that refinement (the FP32 storage
// path, tol 1e-6): an inexact Newton step on the FP64 residual, whose
// relative error e in f' (below about 1e-4) moves the result by at most
// e |dZ| <= e tol Z.  Later steps, and every step without it, evaluate
// both in FP64.
template <bool F32D = false, typename M>
__device__ __forceinline__ C2PResult c2p_newton(double Dc, const double S[3], double tau, const double B[3],
                                                double Zguess, double gm1g, const M &m, int maxit = NEWTON_MAXIT,
                                                bool refine = false, double tol = NEWTON_TOL)
{
    double Su[3], Bl[3];
    raise<double>(m, S, Su);
    lower<double>(m, B, Bl);
    const double S2 = S[0] * Su[0] + S[1] * Su[1] + S[2] * Su[2];
    const double SB = S[0] * B[0] + S[1] * B[1] + S[2] * B[2];
    const double SB2 = SB * SB;
    const double B2 = Bl[0] * B[0] + Bl[1] * B[1] + Bl[2] * B[2];
    const double Uen = tau + Dc;
    // halves used every iteration, exact on the integer pipe
    const double hB2 = scale2<-1>(B2), hSB2 = scale2<-1>(SB2), hD = scale2<-1>(Dc);
    C2PResult r;
    double Z = Zguess, iZ = 0.0, iZB = 0.0, v2 = 0.0;
    float fp32 = 0.0f, dv2_32 = 0.0f;
    if (refine && is_pos(Z))
        Z = c2p_refine_f32(Z, S2, SB2, B2, Dc, Uen, gm1g, fp32, dv2_32);
    int tries = 0;
    bool ok = true;
    for (;;) {
        if (is_pos(Z)) {
            c2p_recip(Z, B2, iZ, iZB);
            v2 = c2p_v2r(Z, iZ, iZB, S2, SB2, B2);
            if (ilt(v2, 1.0))
                break;
        }
        Z = 2.0 * imax(Z, Uen);
        if (++tries > 60) {
            ok = false;
            break;
        }
    }
    if (tries != 0)
        fp32 = 0.0f;        // the refinement's f' belongs to a Z since replaced
    int it = 0;
    bool conv = false;
    bool lin = false;       // the last step was taken to first order
    double sq_fin = 0.0;    // sqrt(1 - v^2) from that step
    while (ok && it < maxit) {
        ++it;
        const double om = 1.0 - v2;
        const double isq = rsqrt(om);
        const double sq = om * isq;
        const double p = gm1g * (Z * om - Dc * sq);
        const double iZ2 = iZ * iZ;
        const double f = Z - p + (1.0 + v2) * hB2 - hSB2 * iZ2 - Uen;
        double dv2, dZ;
        if (F32D && fp32 != 0.0f) {
            dv2 = f2d(dv2_32);
            dZ = f * f2d(__fdividef(1.0f, fp32));
            fp32 = 0.0f;
        } else {
            const double iZ3 = iZ2 * iZ;
            const double iZB3 = iZB * iZB * iZB;
            // dv^2/dZ = -2 (S^2 Z^3 + (S.B)^2 (3 Z^2 + 3 Z B^2 + B^4)) / (Z^3 (Z + B^2)^3)
            //         = -2 (S^2 + (S.B)^2 (Z (3 Z + 3 B^2) + B^4) / Z^3) / (Z + B^2)^3:
            // Z^3 cancels against 1/Z^3, both terms stay positive (no
            // cancellation), and 1/Z^3 serves f' below as well
            const double P3 = fma(3.0 * Z, Z + B2, B2 * B2);
            dv2 = -(scale2<1>(fma(SB2 * P3, iZ3, S2)) * iZB3);
            const double dp = gm1g * (om - Z * dv2 + hD * dv2 * isq);
            const double fp = 1.0 - dp + hB2 * dv2 + SB2 * iZ3;
            // the step's quotient to about 2^-39: its error only perturbs the
            // next iterate, which the iteration corrects, and at the final
            // step (|dZ| <= tol Z) it moves Z by about 2^-39 tol Z
            dZ = nr_step_div(f, fp);
        }
        // A step within the tolerance ends the iteration: Z, 1/Z, 1/(Z + B^2),
        // v^2 and sqrt(1 - v^2) move along their first derivatives instead of
        // being evaluated again at Z - dZ (one division, the v^2 formula and a
        // reciprocal square root fewer); the neglected terms are second order
        // in the step, below the error the stopping tolerance itself leaves.
        if (ile(iabs(dZ), tol * Z)) {
            const double dv = dv2 * dZ;
            const double Zl = Z - dZ, v2l = v2 - dv;
            if (is_pos(Zl) && ilt(v2l, 1.0)) {
                iZ = fma(iZ * dZ, iZ, iZ);
                iZB = fma(iZB * dZ, iZB, iZB);
                Z = Zl;
                v2 = v2l;
                sq_fin = fma(0.5 * isq, dv, sq);   // d sqrt(om) = d om / (2 sqrt(om)), d om = dv
                lin = true;
                conv = true;
                break;
            }
        }
        double Zn = Z - dZ, iZn = 0.0, iZBn = 0.0, v2n = 2.0;
        int h = 0;
        for (;;) {
            if (is_pos(Zn)) {
                c2p_recip(Zn, B2, iZn, iZBn);
                v2n = c2p_v2r(Zn, iZn, iZBn, S2, SB2, B2);
                if (ilt(v2n, 1.0))
                    break;
            }
            if (h >= NEWTON_MAXHALF)
                break;
            dZ *= 0.5;
            Zn = Z - dZ;
            ++h;
        }
        if (!is_pos(Zn) || !ilt(v2n, 1.0))
            break;
        Z = Zn;
        iZ = iZn;
        iZB = iZBn;
        v2 = v2n;
        if (ile(iabs(dZ), tol * Z)) {
            conv = true;
            break;
        }
    }
    const double om = 1.0 - v2;   // > 0: v2 < 1 on every accepted iterate
    const double sq = lin ? sq_fin : om * rsqrt(om);
    const double p = gm1g * (Z * om - Dc * sq);
    const double sbz = SB * iZ;
    double vl[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
        vl[j] = (S[j] + sbz * Bl[j]) * iZB;
    raise<double>(m, vl, r.v);
    r.rho = Dc * sq;
    r.p = p;
    r.Z = Z;
    r.iters = it;
    r.ok = ok && conv && is_pos(p) && is_pos(r.rho);
    return r;
}

// ------------------------------------------------------------------ bc

// Source index along one axis for padded index i (cell array: face = 0,
// d-face array: face = 1); returns i itself for an owned entry, -1 for the
// polar-axis face (value 0).  *flip: sign change under axis reflection.
__device__ __forceinline__ int bc_src(int i, int n, int face, int bclo, int bchi, bool &flip)
{
    flip = false;
    const int lo = NG;
    int hi = NG + n - 1 + face;
    if (face && bclo == BC_PERIODIC)
        hi = NG + n - 1;
    if (i >= lo && i <= hi)
        return i;
    const int side = i < lo ? 0 : 1;
    const int kind = side == 0 ? bclo : bchi;
    if (kind == BC_PERIODIC) {
        int r = (i - NG) % n;
        if (r < 0)
            r += n;
        return NG + r;
    }
    if (kind == BC_OUTFLOW)
        return side == 0 ? lo : hi;
    flip = true;
    if (face) {
        const int ax = side == 0 ? NG : NG + n;
        if (i == ax)
            return -1;
        return 2 * ax - i;
    }
    return side == 0 ? 2 * NG - 1 - i : 2 * (NG + n) - 1 - i;
}

}  // namespace echo
