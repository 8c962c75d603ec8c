/*
 * echo_oracle.c -- plain, slow, FP64 CPU oracle of the per-step update of the
 * 3-D finite-difference GRMHD scheme on a fixed metric.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load this file's library.  The CUDA library
 * shares no code, header, table or helper with it, and neither includes the
 * other.
 *
 * What it computes.  The paper (introduction, the paragraph that presents
 * ECHO-3DHPC) states only that the code solves the equations of
 * general-relativistic MHD with a 3-D finite-difference method and high-order
 * reconstruction, inherited from ECHO.  It prints no equation, so every step
 * below restates a published method, named where it is used:
 *   - 3+1 "Valencia" conservative form of ideal GRMHD on a stationary metric
 *     (Banyuls et al. 1997; Anton et al. 2006; Del Zanna et al. 2007, the
 *     ECHO paper);
 *   - conservative-to-primitive inversion by a 1-D Newton iteration on
 *     Z = rho h W^2;
 *   - MP5 reconstruction of primitives (Suresh & Huynh 1997), alpha = 4,
 *     eps = 1e-10;
 *   - HLL fluxes (Harten, Lax & van Leer 1983) with the approximate fast
 *     speed of the ECHO family;
 *   - upwind constrained transport (UCT-HLL) edge EMFs (Londrillo & Del
 *     Zanna 2004);
 *   - the three-stage SSP Runge-Kutta scheme of Shu & Osher (1988).
 * Readings of the paper's silence are listed in the design notes; each
 * function below states the one it follows.
 *
 * Style: one loop nest per step, no tiling, no fusion, arrays with 3 ghost
 * layers, FP64 everywhere, built with -O2 -ffp-contract=off.
 *
 * Host layout of a state (shared with the library only as a documented
 * format): five cell arrays (D, S_x, S_y, S_z, tau), all densitised by
 * sqrt(gamma), each nz*ny*nx (x fastest), then the face arrays
 *   Bx: nz*ny*(nx+1)   (face i-1/2 at index i, i = 0..nx)
 *   By: nz*(ny+1)*nx
 *   Bz: (nz+1)*ny*nx
 * holding B~ = sqrt(gamma) B^i.  On periodic axes the last face repeats the
 * first.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

/* Hooks of the operation-counting build (op_count.cpp compiles this file as
 * C++ with a number type that counts its arithmetic): OPC_PHASE(k) assigns
 * the operations that follow to step k of the scheme, OPC_UNIT() counts one
 * unit of that step (a cell, a face, an edge), OPC_UNCOUNTED opens a scope
 * whose arithmetic is not the method's own: evaluating the closed-form
 * metric and its derivatives (tabulated once for a fixed metric),
 * coordinates of grid points, and selections (min, max, minmod, which
 * return one of their arguments).  In this C build they do nothing. */
#ifndef OPC_PHASE
#define OPC_PHASE(k)
#define OPC_UNIT()
#define OPC_UNCOUNTED
#endif
enum { OPC_C2P, OPC_CFL, OPC_FACES, OPC_EMF, OPC_CORRECT, OPC_ASSEMBLE, OPC_CT, OPC_RK, OPC_OTHER, OPC_NPHASE };

#define NG 5                 /* ghost layers: MP5 needs 3 cells on each side, the
                                high-order flux correction two more faces */
#define MP5_ALPHA 4.0
#define MP5_EPS 1e-10
#define NEWTON_TOL 1e-13
#define NEWTON_MAXIT 50
#define NEWTON_MAXHALF 30

/* boundary kinds */
#define BC_PERIODIC 0
#define BC_OUTFLOW 1
#define BC_AXIS 2

typedef struct {
    int n[3];          /* interior cells along x1, x2, x3 */
    double x0[3];      /* coordinate of the lower face of the domain */
    double dx[3];      /* cell widths */
    int bc[6];         /* bc[2*d + side], side 0 = lower, 1 = upper */
    int metric;        /* 0: flat Cartesian; 1: Kerr-Schild, (ln r, theta, phi), M = 1 */
    double spin;       /* a/M */
    double gamma;      /* adiabatic index */
    double cfl;
    int floors;        /* 1: apply atmosphere floors after c2p */
    double rho_floor, rho_floor_pow, p_floor, p_floor_pow;  /* floor = f0 * r^pow */
    int order;         /* 0: the scheme as read (cell-average MP5 weights, second-order
                          cell-centre B, no flux correction); 1: high order (point-value
                          MP5 weights, sixth-order cell-centre B, flux-derivative
                          correction of the fluxes and the EMFs) */
} ocfg;

typedef struct {
    double alpha;
    double beta[3];    /* contravariant shift */
    double g[3][3];    /* gamma_ij */
    double gi[3][3];   /* gamma^ij */
    double sqrtg;      /* sqrt(det gamma_ij) */
} ometric;

typedef struct {
    long long c2p_iters;
    long long c2p_calls;
    long long c2p_fail;
    long long floor_hits;
    long long fallback_faces;
    long long guard_faces;    /* order 1: faces whose corrected fluxes the safeguard replaced */
} ostats;

/* ------------------------------------------------------------------ */
/* Metric                                                              */
/* ------------------------------------------------------------------ */

/* Inverse and determinant of a symmetric 3x3 matrix by cofactors. */
static double inv3(const double m[3][3], double out[3][3])
{
    OPC_UNCOUNTED;
    double c00 = m[1][1] * m[2][2] - m[1][2] * m[2][1];
    double c01 = m[1][2] * m[2][0] - m[1][0] * m[2][2];
    double c02 = m[1][0] * m[2][1] - m[1][1] * m[2][0];
    double det = m[0][0] * c00 + m[0][1] * c01 + m[0][2] * c02;
    if (det == 0.0) {
        memset(out, 0, 9 * sizeof(double));
        return 0.0;
    }
    out[0][0] = c00 / det;
    out[1][0] = c01 / det;
    out[2][0] = c02 / det;
    out[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) / det;
    out[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) / det;
    out[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) / det;
    out[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) / det;
    out[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) / det;
    out[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) / det;
    return det;
}

/* Lapse, shift and spatial metric at coordinate point x.
 * metric 0: Minkowski in Cartesian coordinates.
 * metric 1: Kerr in Kerr-Schild form (Boyer-Lindquist radius and polar angle,
 *   ingoing Kerr-Schild time), written in x1 = ln r, x2 = theta, x3 = phi:
 *   Sigma = r^2 + a^2 cos^2 theta, z = 2 r / Sigma,
 *   alpha = (1+z)^-1/2, beta^r = z/(1+z),
 *   gamma_rr = 1+z, gamma_rphi = -a(1+z) sin^2, gamma_thth = Sigma,
 *   gamma_phph = sin^2 [Sigma + a^2 (1+z) sin^2];
 *   dr = r dx1 scales the x1 row/column by r.  sqrt(gamma) is taken from the
 *   determinant, so the closed form alpha sqrt(gamma) = r Sigma sin(theta)
 *   is a test of the components. */
static void metric_components(const ocfg *c, const double x[3], double *alpha,
                              double beta[3], double g[3][3])
{
    OPC_UNCOUNTED;
    memset(g, 0, 9 * sizeof(double));
    beta[0] = beta[1] = beta[2] = 0.0;
    if (c->metric == 0) {
        *alpha = 1.0;
        g[0][0] = g[1][1] = g[2][2] = 1.0;
        return;
    }
    double r = exp(x[0]);
    double th = x[1];
    double a = c->spin;
    double cth = cos(th), sth = sin(th);
    double s2 = sth * sth;
    double sig = r * r + a * a * cth * cth;
    double z = 2.0 * r / sig;
    *alpha = 1.0 / sqrt(1.0 + z);
    beta[0] = z / (1.0 + z) / r;
    g[0][0] = (1.0 + z) * r * r;
    g[0][2] = g[2][0] = -a * (1.0 + z) * s2 * r;
    g[1][1] = sig;
    g[2][2] = s2 * (sig + a * a * (1.0 + z) * s2);
}

static void metric_eval(const ocfg *c, const double x[3], ometric *m)
{
    OPC_UNCOUNTED;
    metric_components(c, x, &m->alpha, m->beta, m->g);
    double det = inv3(m->g, m->gi);
    m->sqrtg = det > 0.0 ? sqrt(det) : 0.0;
}

/* Coordinate position of a cell centre (off = 0) or a face/edge (off = -1/2)
 * from padded indices. */
static double coord(const ocfg *c, int d, int ipad, double off)
{
    OPC_UNCOUNTED;
    return c->x0[d] + ((double)(ipad - NG) + 0.5 + off) * c->dx[d];
}

/* ------------------------------------------------------------------ */
/* Pointwise physics                                                   */
/* ------------------------------------------------------------------ */

static void lower3(const ometric *m, const double u[3], double d[3])
{
    for (int i = 0; i < 3; ++i)
        d[i] = m->g[i][0] * u[0] + m->g[i][1] * u[1] + m->g[i][2] * u[2];
}

static void raise3(const ometric *m, const double d[3], double u[3])
{
    for (int i = 0; i < 3; ++i)
        u[i] = m->gi[i][0] * d[0] + m->gi[i][1] * d[1] + m->gi[i][2] * d[2];
}

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Primitive -> conserved, Valencia variables (undensitised).
 * P = (rho, v^x, v^y, v^z, p, B^x, B^y, B^z), contravariant v and B.
 * D = rho W; S_j = (rho h W^2 + B^2) v_j - (v.B) B_j;
 * tau = rho h W^2 - p + (B^2 + B^2 v^2 - (v.B)^2)/2 - D. */
static void p2c_point(const ometric *m, double gam, const double *P, double *C)
{
    double v[3] = {P[1], P[2], P[3]}, B[3] = {P[5], P[6], P[7]};
    double vl[3], Bl[3];
    lower3(m, v, vl);
    lower3(m, B, Bl);
    double v2 = dot3(vl, v), B2 = dot3(Bl, B), vB = dot3(vl, B);
    double W = 1.0 / sqrt(1.0 - v2);
    double rho = P[0], p = P[4];
    double h = 1.0 + gam / (gam - 1.0) * p / rho;
    double Zw = rho * h * W * W;
    C[0] = rho * W;
    for (int j = 0; j < 3; ++j)
        C[1 + j] = (Zw + B2) * vl[j] - vB * Bl[j];
    double U = Zw - p + 0.5 * (B2 + B2 * v2 - vB * vB);
    C[4] = U - C[0];
}

/* v^2 as a function of the Newton unknown Z = rho h W^2 (derived from the
 * S_j definition: S.B = Z (v.B)). */
static double c2p_v2(double Z, double S2, double SB, double B2)
{
    double ZB = Z + B2;
    return (S2 * Z * Z + SB * SB * (2.0 * Z + B2)) / (Z * Z * ZB * ZB);
}

/* Conserved -> primitive: Newton iteration on Z = rho h W^2.
 * C = undensitised (D, S_j, tau), B = undensitised contravariant B^i.
 * Residual f(Z) = Z - p(Z) + (1 + v^2(Z)) B^2 / 2 - (S.B)^2 / (2 Z^2) - (tau + D),
 * p(Z) = (G-1)/G [Z (1 - v^2) - D sqrt(1 - v^2)].
 * Guess: Zguess; if it is not admissible (Z <= 0 or v^2 >= 1) it is replaced
 * by doubling max(Z, tau + D) until admissible.
 * Each step Z <- Z - f/f'; a step that leaves the admissible set is halved
 * (up to 30 times).  Stop when |dZ| <= 1e-13 Z, at most 50 iterations.
 * Output P5 = (rho, v^x, v^y, v^z, p).  Returns 0 on success, 1 on failure. */
static int c2p_point(const ometric *m, double gam, const double *C, const double B[3],
                     double Zguess, double *P5, double *Zout, int *iters)
{
    double D = C[0], tau = C[4];
    double S[3] = {C[1], C[2], C[3]};
    double Su[3], Bl[3];
    raise3(m, S, Su);
    lower3(m, B, Bl);
    double S2 = dot3(S, Su);
    double SB = dot3(S, B);
    double B2 = dot3(Bl, B);
    double U = tau + D;
    double gg = (gam - 1.0) / gam;

    double Z = Zguess;
    int tries = 0;
    while (!(Z > 0.0) || !(c2p_v2(Z, S2, SB, B2) < 1.0)) {
        double base = Z > U ? Z : U;
        Z = 2.0 * base;
        if (++tries > 60) {
            *iters = 0;
            return 1;
        }
    }

    int it = 0, ok = 0;
    while (it < NEWTON_MAXIT) {
        ++it;
        double v2 = c2p_v2(Z, S2, SB, B2);
        double sq = sqrt(1.0 - v2);
        double p = gg * (Z * (1.0 - v2) - D * sq);
        double f = Z - p + 0.5 * (1.0 + v2) * B2 - SB * SB / (2.0 * Z * Z) - U;
        double ZB = Z + B2;
        double dv2 = -2.0 * (S2 * Z * Z * Z + SB * SB * (3.0 * Z * Z + 3.0 * Z * B2 + B2 * B2))
                     / (Z * Z * Z * ZB * ZB * ZB);
        double dp = gg * ((1.0 - v2) - Z * dv2 + D * dv2 / (2.0 * sq));
        double fp = 1.0 - dp + 0.5 * B2 * dv2 + SB * SB / (Z * Z * Z);
        double dZ = f / fp;
        double Zn = Z - dZ;
        int h = 0;
        while ((!(Zn > 0.0) || !(c2p_v2(Zn, S2, SB, B2) < 1.0)) && h < NEWTON_MAXHALF) {
            dZ *= 0.5;
            Zn = Z - dZ;
            ++h;
        }
        if (!(Zn > 0.0) || !(c2p_v2(Zn, S2, SB, B2) < 1.0))
            break;
        Z = Zn;
        if (fabs(dZ) <= NEWTON_TOL * Z) {
            ok = 1;
            break;
        }
    }
    *iters = it;
    double v2 = c2p_v2(Z, S2, SB, B2);
    double sq = sqrt(1.0 - v2);
    double p = gg * (Z * (1.0 - v2) - D * sq);
    double vl[3];
    for (int j = 0; j < 3; ++j)
        vl[j] = (S[j] + SB * Bl[j] / Z) / (Z + B2);
    double vu[3];
    raise3(m, vl, vu);
    P5[0] = D * sq;
    P5[1] = vu[0];
    P5[2] = vu[1];
    P5[3] = vu[2];
    P5[4] = p;
    *Zout = Z;
    if (!ok || !(p > 0.0) || !(P5[0] > 0.0))
        return 1;
    return 0;
}

/* ---- MP5 (Suresh & Huynh 1997) ---- */

static double sgn(double a) { return (a > 0.0) - (a < 0.0); }

static double minmod2(double a, double b)
{
    OPC_UNCOUNTED;
    return 0.5 * (sgn(a) + sgn(b)) * fmin(fabs(a), fabs(b));
}

static double minmod4(double w, double x, double y, double z)
{
    OPC_UNCOUNTED;
    double s = 0.125 * (sgn(w) + sgn(x)) * fabs((sgn(w) + sgn(y)) * (sgn(w) + sgn(z)));
    return s * fmin(fmin(fabs(w), fabs(x)), fmin(fabs(y), fabs(z)));
}

/* Interface value between u0 = u_j and u1 = u_{j+1}, biased towards u_j,
 * from the five values um2 = u_{j-2}, um1, u0, up1, up2 = u_{j+2}.
 * The unlimited value is the fifth-order interpolant of cell averages,
 * (2, -13, 47, 27, -3)/60 (order 0), or the fifth-order Lagrange
 * interpolant of point values at the interface, (3, -20, 90, 60, -5)/128
 * (order 1); the limiter keeps it inside the monotonicity- and
 * accuracy-preserving interval of Suresh & Huynh. */
static double mp5_face(double um2, double um1, double u0, double up1, double up2, int order)
{
    double uor = order ? (3.0 * um2 - 20.0 * um1 + 90.0 * u0 + 60.0 * up1 - 5.0 * up2) / 128.0
                       : (2.0 * um2 - 13.0 * um1 + 47.0 * u0 + 27.0 * up1 - 3.0 * up2) / 60.0;
    double ump = u0 + minmod2(up1 - u0, MP5_ALPHA * (u0 - um1));
    if ((uor - u0) * (uor - ump) <= MP5_EPS)
        return uor;
    double dm1 = um2 - 2.0 * um1 + u0;
    double d0 = um1 - 2.0 * u0 + up1;
    double dp1 = u0 - 2.0 * up1 + up2;
    double dMp = minmod4(4.0 * d0 - dp1, 4.0 * dp1 - d0, d0, dp1);
    double dMm = minmod4(4.0 * d0 - dm1, 4.0 * dm1 - d0, d0, dm1);
    double uul = u0 + MP5_ALPHA * (u0 - um1);
    double uav = 0.5 * (u0 + up1);
    double umd = uav - 0.5 * dMp;
    double ulc = u0 + 0.5 * (u0 - um1) + 4.0 / 3.0 * dMm;
    double umin = fmax(fmin(fmin(u0, up1), umd), fmin(fmin(u0, uul), ulc));
    double umax = fmin(fmax(fmax(u0, up1), umd), fmax(fmax(u0, uul), ulc));
    return uor + minmod2(umin - uor, umax - uor);
}

/* Left and right states at the face between q[2] and q[3] of a 6-point
 * stencil q[0..5] = u_{f-3} .. u_{f+2}. */
static void mp5_lr(const double q[6], double *L, double *R, int order)
{
    *L = mp5_face(q[0], q[1], q[2], q[3], q[4], order);
    *R = mp5_face(q[5], q[4], q[3], q[2], q[1], order);
}

/* ---- high-order flux-derivative correction ----
 * For point values F_{j+1/2} of a flux at the interfaces, the corrected
 * flux  Fhat = F - D2/24 + 3 D4/640,  D2 = F_{-1} - 2 F_0 + F_{+1},
 * D4 = F_{-2} - 4 F_{-1} + 6 F_0 - 4 F_{+1} + F_{+2} (neighbouring
 * interfaces), makes (Fhat_{i+1/2} - Fhat_{i-1/2}) / h the sixth-order
 * derivative dF/dx at x_i: Fhat is the interface value of the function
 * whose cell averages are the point values F (F - h^2 F''/24 +
 * 7 h^4 F/5760), with F and F written as differences of the
 * interface values.  f5 = F_{-2} .. F_{+2}. */
static double ho_flux(const double f5[5])
{
    double d2 = f5[1] - 2.0 * f5[2] + f5[3];
    double d4 = f5[0] - 4.0 * f5[1] + 6.0 * f5[2] - 4.0 * f5[3] + f5[4];
    return f5[2] - d2 / 24.0 + 3.0 * d4 / 640.0;
}

/* Sixth-order Lagrange interpolation to the midpoint of six equally spaced
 * values b6 = b_{-5/2} .. b_{+5/2}: (3, -25, 150, 150, -25, 3)/256. */
static double ho_center(const double b6[6])
{
    return (3.0 * b6[0] - 25.0 * b6[1] + 150.0 * b6[2] + 150.0 * b6[3] - 25.0 * b6[4] + 3.0 * b6[5]) / 256.0;
}

/* ---- characteristic speeds (approximate fast magnetosonic speed) ----
 * c_s^2 = G p/(rho h), c_A^2 = b^2/(rho h + b^2), a^2 = c_s^2 + c_A^2 - c_s^2 c_A^2,
 * lambda_pm = alpha/(1 - v^2 a^2) { v^d (1-a^2) pm sqrt(a^2 (1-v^2)
 *             [(1 - v^2 a^2) gamma^dd - (1-a^2) (v^d)^2]) } - beta^d. */
static void speeds_point(const ometric *m, double gam, const double *P, int d,
                         double *lp, double *lm)
{
    double v[3] = {P[1], P[2], P[3]}, B[3] = {P[5], P[6], P[7]};
    double vl[3], Bl[3];
    lower3(m, v, vl);
    lower3(m, B, Bl);
    double v2 = dot3(vl, v), B2 = dot3(Bl, B), vB = dot3(vl, B);
    double W2 = 1.0 / (1.0 - v2);
    double rho = P[0], p = P[4];
    double rhoh = rho + gam / (gam - 1.0) * p;
    double b2 = B2 / W2 + vB * vB;
    double cs2 = gam * p / rhoh;
    double ca2 = b2 / (rhoh + b2);
    double a2 = cs2 + ca2 - cs2 * ca2;
    double vd = v[d];
    double disc = a2 * (1.0 - v2) * ((1.0 - v2 * a2) * m->gi[d][d] - (1.0 - a2) * vd * vd);
    double sq = sqrt(fmax(disc, 0.0));
    double den = 1.0 - v2 * a2;
    *lp = m->alpha / den * (vd * (1.0 - a2) + sq) - m->beta[d];
    *lm = m->alpha / den * (vd * (1.0 - a2) - sq) - m->beta[d];
}

/* Physical flux along direction d and conserved vector of a primitive
 * state, both multiplied by sqrt(gamma) of the point:
 *   F(D) = D (alpha v^d - beta^d)
 *   F(S_j) = alpha W^d_j - beta^d S_j,
 *     W^d_j = (rho h + b^2) W^2 v^d v_j + (p + b^2/2) delta^d_j - b^d b_j,
 *     b^i = B^i/W + W (v.B) v^i  (spatial projection of the comoving field)
 *   F(tau) = alpha (S^d - D v^d) - beta^d tau. */
static void flux_point(const ometric *m, double gam, const double *P, int d,
                       double F[5], double C[5])
{
    double v[3] = {P[1], P[2], P[3]}, B[3] = {P[5], P[6], P[7]};
    double vl[3], Bl[3];
    lower3(m, v, vl);
    lower3(m, B, Bl);
    double v2 = dot3(vl, v), B2 = dot3(Bl, B), vB = dot3(vl, B);
    double W = 1.0 / sqrt(1.0 - v2);
    double rho = P[0], p = P[4];
    double rhoh = rho + gam / (gam - 1.0) * p;
    double b2 = B2 / (W * W) + vB * vB;
    double bu[3], bl[3];
    for (int i = 0; i < 3; ++i)
        bu[i] = B[i] / W + W * vB * v[i];
    lower3(m, bu, bl);

    p2c_point(m, gam, P, C);
    double Su[3] = {0, 0, 0};
    double Sl[3] = {C[1], C[2], C[3]};
    raise3(m, Sl, Su);

    F[0] = C[0] * (m->alpha * v[d] - m->beta[d]);
    for (int j = 0; j < 3; ++j) {
        double Wdj = (rhoh + b2) * W * W * v[d] * vl[j] - bu[d] * bl[j];
        if (j == d)
            Wdj += p + 0.5 * b2;
        F[1 + j] = m->alpha * Wdj - m->beta[d] * C[1 + j];
    }
    F[4] = m->alpha * (Su[d] - C[0] * v[d]) - m->beta[d] * C[4];
    for (int q = 0; q < 5; ++q) {
        F[q] *= m->sqrtg;
        C[q] *= m->sqrtg;
    }
}

/* HLL combination of two states at a face (already multiplied by sqrt(gamma)).
 * a+ = max(0, l+_L, l+_R), a- = max(0, -l-_L, -l-_R),
 * F = (a+ F_L + a- F_R - a+ a- (U_R - U_L)) / (a+ + a-). */
static void hll(const double FL[5], const double FR[5], const double UL[5], const double UR[5],
                double ap, double am, double F[5])
{
    double s = ap + am;
    for (int q = 0; q < 5; ++q) {
        if (s > 0.0)
            F[q] = (ap * FL[q] + am * FR[q] - ap * am * (UR[q] - UL[q])) / s;
        else
            F[q] = 0.5 * (FL[q] + FR[q]);
    }
}

/* ------------------------------------------------------------------ */
/* Grid containers                                                     */
/* ------------------------------------------------------------------ */

typedef struct {
    int n[3];
    int np[3];          /* padded sizes n + 2 NG */
    size_t ncell;       /* np0*np1*np2 */
    double *U[5];       /* densitised cell conserved */
    double *B[3];       /* densitised face field, face i-1/2 at index i */
    double *Z;          /* Newton unknown memory (cell) */
    double *P[8];       /* cell primitives rho, v^x, v^y, v^z, p, B^x, B^y, B^z */
    /* face data per direction d: flux[5], a+, a-, reconstructed v (3) L/R */
    double *F[3][5];
    double *ap[3], *am[3];
    double *vL[3][3], *vR[3][3];   /* [face dir][component] */
    double *E[3];       /* edge EMFs */
    double *Fc[3][5];   /* order 1: corrected fluxes on the owned faces */
    double *Ec[3][2];   /* order 1: E_e corrected along (e+1)%3 [0] and (e+2)%3 [1] */
    double *LU[5], *LB[3];
    double *cellspeed;  /* per cell sum_d max|lambda_d|/dx_d */
    double *mark;       /* order 1: 1 for a cell the positivity safeguard flags */
} ogrid;

static size_t IDX(const ogrid *G, int i, int j, int k)
{
    return ((size_t)k * G->np[1] + (size_t)j) * G->np[0] + (size_t)i;
}

static double *zalloc(size_t n)
{
    double *p = (double *)calloc(n, sizeof(double));
    return p;
}

static int grid_alloc(ogrid *G, const int n[3])
{
    memset(G, 0, sizeof(*G));
    for (int d = 0; d < 3; ++d) {
        G->n[d] = n[d];
        G->np[d] = n[d] + 2 * NG;
    }
    G->ncell = (size_t)G->np[0] * G->np[1] * G->np[2];
    size_t N = G->ncell;
    int ok = 1;
#define A(p) do { (p) = zalloc(N); ok = ok && (p) != NULL; } while (0)
    for (int q = 0; q < 5; ++q) { A(G->U[q]); A(G->LU[q]); }
    for (int d = 0; d < 3; ++d) {
        A(G->B[d]); A(G->LB[d]); A(G->E[d]); A(G->ap[d]); A(G->am[d]);
        for (int q = 0; q < 5; ++q) { A(G->F[d][q]); A(G->Fc[d][q]); }
        A(G->Ec[d][0]); A(G->Ec[d][1]);
        for (int c = 0; c < 3; ++c) { A(G->vL[d][c]); A(G->vR[d][c]); }
    }
    for (int q = 0; q < 8; ++q) A(G->P[q]);
    A(G->Z);
    A(G->cellspeed);
    A(G->mark);
#undef A
    return ok ? 0 : -1;
}

static void grid_free(ogrid *G)
{
    for (int q = 0; q < 5; ++q) { free(G->U[q]); free(G->LU[q]); }
    for (int d = 0; d < 3; ++d) {
        free(G->B[d]); free(G->LB[d]); free(G->E[d]); free(G->ap[d]); free(G->am[d]);
        for (int q = 0; q < 5; ++q) { free(G->F[d][q]); free(G->Fc[d][q]); }
        free(G->Ec[d][0]); free(G->Ec[d][1]);
        for (int c = 0; c < 3; ++c) { free(G->vL[d][c]); free(G->vR[d][c]); }
    }
    for (int q = 0; q < 8; ++q) free(G->P[q]);
    free(G->Z);
    free(G->cellspeed);
    free(G->mark);
}

/* Number of doubles in a host state. */
static size_t state_count(const int n[3])
{
    size_t N = (size_t)n[0] * n[1] * n[2];
    return 5 * N + (size_t)n[2] * n[1] * (n[0] + 1) + (size_t)n[2] * (n[1] + 1) * n[0]
           + (size_t)(n[2] + 1) * n[1] * n[0];
}

/* Host face-array extents: face array d has n[d]+1 entries along d. */
static void face_extent(const int n[3], int d, int e[3])
{
    e[0] = n[0]; e[1] = n[1]; e[2] = n[2];
    e[d] += 1;
}

static void unpack_state(ogrid *G, const double *s)
{
    const int *n = G->n;
    size_t N = (size_t)n[0] * n[1] * n[2];
    for (int q = 0; q < 5; ++q)
        for (int k = 0; k < n[2]; ++k)
            for (int j = 0; j < n[1]; ++j)
                for (int i = 0; i < n[0]; ++i)
                    G->U[q][IDX(G, i + NG, j + NG, k + NG)] = s[q * N + ((size_t)k * n[1] + j) * n[0] + i];
    const double *f = s + 5 * N;
    for (int d = 0; d < 3; ++d) {
        int e[3];
        face_extent(n, d, e);
        for (int k = 0; k < e[2]; ++k)
            for (int j = 0; j < e[1]; ++j)
                for (int i = 0; i < e[0]; ++i)
                    G->B[d][IDX(G, i + NG, j + NG, k + NG)] = f[((size_t)k * e[1] + j) * e[0] + i];
        f += (size_t)e[0] * e[1] * e[2];
    }
}

static void pack_arrays(const ogrid *G, double *const *cellq, double *const *faced, double *s)
{
    const int *n = G->n;
    size_t N = (size_t)n[0] * n[1] * n[2];
    for (int q = 0; q < 5; ++q)
        for (int k = 0; k < n[2]; ++k)
            for (int j = 0; j < n[1]; ++j)
                for (int i = 0; i < n[0]; ++i)
                    s[q * N + ((size_t)k * n[1] + j) * n[0] + i] = cellq[q][IDX(G, i + NG, j + NG, k + NG)];
    double *f = s + 5 * N;
    for (int d = 0; d < 3; ++d) {
        int e[3];
        face_extent(n, d, e);
        for (int k = 0; k < e[2]; ++k)
            for (int j = 0; j < e[1]; ++j)
                for (int i = 0; i < e[0]; ++i)
                    f[((size_t)k * e[1] + j) * e[0] + i] = faced[d][IDX(G, i + NG, j + NG, k + NG)];
        f += (size_t)e[0] * e[1] * e[2];
    }
}

static void unpack_cell(const ogrid *G, const double *src, double *dst)
{
    const int *n = G->n;
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i)
                dst[IDX(G, i + NG, j + NG, k + NG)] = src[((size_t)k * n[1] + j) * n[0] + i];
}

static void pack_cell(const ogrid *G, const double *src, double *dst)
{
    const int *n = G->n;
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i)
                dst[((size_t)k * n[1] + j) * n[0] + i] = src[IDX(G, i + NG, j + NG, k + NG)];
}

/* ------------------------------------------------------------------ */
/* Boundary (ghost) fill                                               */
/* ------------------------------------------------------------------ */

/* Source index along dimension d for padded index i of a cell-centred
 * (face = 0) or d-face-centred (face = 1) array; *flip is set when the
 * value changes sign under an axis reflection; returns -1 for the polar
 * axis face itself (value 0).
 *   periodic: wrap into the owned range (cells and faces g..g+n-1);
 *   outflow:  copy the nearest owned cell / boundary face;
 *   axis:     mirror across the axis face. */
static int bc_source(const ocfg *c, int d, int i, int face, int *flip)
{
    int n = c->n[d];
    *flip = 0;
    int lo = NG, hi = NG + n - 1 + face;  /* owned range (inclusive) */
    if (face && (c->bc[2 * d] == BC_PERIODIC))
        hi = NG + n - 1;
    if (i >= lo && i <= hi)
        return i;
    int side = i < lo ? 0 : 1;
    int kind = c->bc[2 * d + side];
    if (kind == BC_PERIODIC) {
        int r = (i - NG) % n;
        if (r < 0)
            r += n;
        return NG + r;
    }
    if (kind == BC_OUTFLOW)
        return side == 0 ? lo : hi;
    /* axis */
    *flip = 1;
    if (face) {
        int ax = side == 0 ? NG : NG + n;
        if (i == ax)
            return -1;
        return 2 * ax - i;
    }
    return side == 0 ? 2 * NG - 1 - i : 2 * (NG + n) - 1 - i;
}

/* Fill the ghost layers of one padded array.  comp = the vector component
 * the array holds (0..2) or -1 for a scalar; face = -1 for a cell array,
 * else the face direction; dens = 1 if the array carries the factor
 * sqrt(gamma) (the densitised face field B~ = sqrt(gamma) B).  Under the
 * reflection across a polar axis along d the component along d changes
 * sign, and so does sqrt(gamma) ~ sin(theta), which is odd about the pole:
 * the ghost value is negated when exactly one of the two holds. */
static void fill_array(const ocfg *c, const ogrid *G, double *a, int comp, int face, int dens)
{
    for (int d = 0; d < 3; ++d) {
        int isface = face == d;
        /* sweep d over all padded indices; the other directions over their
         * full padded range so that edges and corners are filled too */
        for (int k = 0; k < G->np[2]; ++k)
            for (int j = 0; j < G->np[1]; ++j)
                for (int i = 0; i < G->np[0]; ++i) {
                    int idx[3] = {i, j, k};
                    int flip;
                    int s = bc_source(c, d, idx[d], isface, &flip);
                    if (s == idx[d])
                        continue;
                    double val;
                    if (s < 0) {
                        val = 0.0;
                    } else {
                        int sidx[3] = {i, j, k};
                        sidx[d] = s;
                        val = a[IDX(G, sidx[0], sidx[1], sidx[2])];
                        if (flip && ((comp == d) != (dens != 0)))
                            val = -val;
                    }
                    a[IDX(G, i, j, k)] = val;
                }
    }
}

static void fill_prims(const ocfg *c, ogrid *G)
{
    fill_array(c, G, G->P[0], -1, -1, 0);
    for (int q = 0; q < 3; ++q)
        fill_array(c, G, G->P[1 + q], q, -1, 0);
    fill_array(c, G, G->P[4], -1, -1, 0);
    for (int q = 0; q < 3; ++q)
        fill_array(c, G, G->P[5 + q], q, -1, 0);
}

/* The face field B~^d = sqrt(gamma) B^d: across a polar axis along theta the
 * theta-face array is even (B^theta and sqrt(gamma) both odd) and the r- and
 * phi-face arrays are odd. */
static void fill_faces(const ocfg *c, ogrid *G)
{
    for (int d = 0; d < 3; ++d)
        fill_array(c, G, G->B[d], d, d, 1);
}

/* ------------------------------------------------------------------ */
/* Grid steps                                                          */
/* ------------------------------------------------------------------ */

static double floor_value(double f0, double pw, const ocfg *c, double x1)
{
    OPC_UNCOUNTED;
    if (c->metric == 1)
        return f0 * pow(exp(x1), pw);
    return f0;
}

/* Cell-centre B of cell (i,j,k): order 0 the mean of the two faces, order 1
 * the sixth-order interpolation of the faces i-2 .. i+3 along each d; then
 * divided by the cell's sqrt(gamma). */
static void cell_centre_B(const ocfg *c, const ogrid *G, int i, int j, int k, double sqrtg, double Bc[3])
{
    for (int d = 0; d < 3; ++d) {
        if (c->order) {
            double b6[6];
            for (int s = 0; s < 6; ++s) {
                int t[3] = {i, j, k};
                t[d] += s - 2;
                b6[s] = G->B[d][IDX(G, t[0], t[1], t[2])];
            }
            Bc[d] = ho_center(b6) / sqrtg;
        } else {
            int t[3] = {i, j, k};
            t[d] += 1;
            Bc[d] = 0.5 * (G->B[d][IDX(G, i, j, k)] + G->B[d][IDX(G, t[0], t[1], t[2])]) / sqrtg;
        }
    }
}

/* c2p over the owned cells.  Cell-centre B from cell_centre_B.  With floors on, rho and p are raised
 * to the atmosphere floors and the conserved state is reset from the
 * floored primitives; a failed inversion keeps the cell's previous
 * primitives (floored) and is counted.  Without floors a failure is an
 * error. */
static int c2p_grid(const ocfg *c, ogrid *G, ostats *st)
{
    long long iters = 0, fails = 0, floors = 0, calls = 0;
    OPC_PHASE(OPC_C2P);
#pragma omp parallel for collapse(2) reduction(+ : iters, fails, floors, calls)
    for (int k = NG; k < NG + G->n[2]; ++k)
        for (int j = NG; j < NG + G->n[1]; ++j)
            for (int i = NG; i < NG + G->n[0]; ++i) {
                OPC_UNIT();
                size_t id = IDX(G, i, j, k);
                double x[3] = {coord(c, 0, i, 0), coord(c, 1, j, 0), coord(c, 2, k, 0)};
                ometric m;
                metric_eval(c, x, &m);
                double Bc[3];
                cell_centre_B(c, G, i, j, k, m.sqrtg, Bc);
                double C[5];
                for (int q = 0; q < 5; ++q)
                    C[q] = G->U[q][id] / m.sqrtg;
                double P5[5], Z;
                int it;
                int bad = c2p_point(&m, c->gamma, C, Bc, G->Z[id], P5, &Z, &it);
                iters += it;
                calls += 1;
                if (bad) {
                    fails += 1;
                    if (!c->floors)
                        continue;
                    for (int q = 0; q < 5; ++q)
                        P5[q] = G->P[q][id];
                }
                int reset = bad;
                if (c->floors) {
                    double rf = floor_value(c->rho_floor, c->rho_floor_pow, c, x[0]);
                    double pf = floor_value(c->p_floor, c->p_floor_pow, c, x[0]);
                    if (!(P5[0] >= rf)) { P5[0] = rf; reset = 1; }
                    if (!(P5[4] >= pf)) { P5[4] = pf; reset = 1; }
                    if (reset)
                        floors += 1;
                }
                for (int q = 0; q < 5; ++q)
                    G->P[q][id] = P5[q];
                for (int q = 0; q < 3; ++q)
                    G->P[5 + q][id] = Bc[q];
                if (reset) {
                    double Pf[8], Cf[5];
                    for (int q = 0; q < 5; ++q) Pf[q] = P5[q];
                    for (int q = 0; q < 3; ++q) Pf[5 + q] = Bc[q];
                    p2c_point(&m, c->gamma, Pf, Cf);
                    for (int q = 0; q < 5; ++q)
                        G->U[q][id] = Cf[q] * m.sqrtg;
                    double W2 = 0.0;
                    {
                        double v[3] = {Pf[1], Pf[2], Pf[3]}, vl[3];
                        lower3(&m, v, vl);
                        W2 = 1.0 / (1.0 - dot3(vl, v));
                    }
                    Z = (Pf[0] + c->gamma / (c->gamma - 1.0) * Pf[4]) * W2;
                }
                G->Z[id] = Z;
            }
    st->c2p_iters += iters;
    st->c2p_fail += fails;
    st->floor_hits += floors;
    st->c2p_calls += calls;
    if (fails && !c->floors)
        return -1;
    return 0;
}

/* Per-cell CFL rate sum_d max(|l+_d|, |l-_d|) / dx_d from cell primitives. */
static double cfl_rate_max(const ocfg *c, ogrid *G)
{
    OPC_PHASE(OPC_CFL);
#pragma omp parallel for collapse(2)
    for (int k = NG; k < NG + G->n[2]; ++k)
        for (int j = NG; j < NG + G->n[1]; ++j)
            for (int i = NG; i < NG + G->n[0]; ++i) {
                OPC_UNIT();
                size_t id = IDX(G, i, j, k);
                double x[3] = {coord(c, 0, i, 0), coord(c, 1, j, 0), coord(c, 2, k, 0)};
                ometric m;
                metric_eval(c, x, &m);
                double P[8];
                for (int q = 0; q < 8; ++q)
                    P[q] = G->P[q][id];
                double s = 0.0;
                for (int d = 0; d < 3; ++d) {
                    double lp, lm;
                    speeds_point(&m, c->gamma, P, d, &lp, &lm);
                    s += fmax(fabs(lp), fabs(lm)) / c->dx[d];
                }
                G->cellspeed[id] = s;
            }
    double mx = 0.0;
    for (int k = NG; k < NG + G->n[2]; ++k)
        for (int j = NG; j < NG + G->n[1]; ++j)
            for (int i = NG; i < NG + G->n[0]; ++i)
                mx = fmax(mx, G->cellspeed[IDX(G, i, j, k)]);
    return mx;
}

/* Face states, fluxes and HLL speeds on the d-faces.  Face index i along d
 * is the face between cells i-1 and i.  Computed on every face whose
 * 6-point stencil lies inside the padded array, i.e. along d for indices
 * NG..NG+n (all faces that bound an owned cell) and over the full padded
 * range transversally (the edge EMFs need faces 3 rows into the ghosts).
 * Reconstructed (MP5): rho, v^x, v^y, v^z, p and the two transverse
 * cell-centre B components; the normal component is the staggered B~^d
 * divided by the face sqrt(gamma).  If a reconstructed side has rho <= 0,
 * p <= 0 or v^2 >= 1, that side takes the adjacent cell's primitives
 * (first order); fallback_faces counts those replacements on the faces
 * that bound owned cells (each face once, both sides). */
static void faces_dir(const ocfg *c, ogrid *G, int d, ostats *st)
{
    int lo[3] = {0, 0, 0}, hi[3] = {G->np[0], G->np[1], G->np[2]};
    /* order 1: two more faces on each side for the flux correction */
    lo[d] = NG - 2 * c->order;
    hi[d] = NG + G->n[d] + 1 + 2 * c->order;
    /* transverse: indices whose face stencil (along d) exists; all */
    long long fb = 0;
    OPC_PHASE(OPC_FACES);
#pragma omp parallel for collapse(2) reduction(+ : fb)
    for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
            for (int i = lo[0]; i < hi[0]; ++i) {
                int idx[3] = {i, j, k};
                size_t id = IDX(G, i, j, k);
                double x[3] = {coord(c, 0, i, d == 0 ? -0.5 : 0.0), coord(c, 1, j, d == 1 ? -0.5 : 0.0),
                               coord(c, 2, k, d == 2 ? -0.5 : 0.0)};
                ometric m;
                metric_eval(c, x, &m);
                if (!(m.sqrtg > 0.0)) {
                    /* polar-axis face: zero area, no flux */
                    for (int q = 0; q < 5; ++q)
                        G->F[d][q][id] = 0.0;
                    G->ap[d][id] = 0.0;
                    G->am[d][id] = 0.0;
                    for (int cc = 0; cc < 3; ++cc) {
                        G->vL[d][cc][id] = 0.0;
                        G->vR[d][cc][id] = 0.0;
                    }
                    continue;
                }
                OPC_UNIT();
                /* counted fallbacks: faces that bound owned cells, each once (on a
                 * periodic axis the face NG+n repeats NG) */
                int owned = 1;
                for (int a = 0; a < 3; ++a) {
                    int top = NG + G->n[a] - 1;
                    if (a == d && c->bc[2 * d] != BC_PERIODIC)
                        top += 1;
                    if (idx[a] < NG || idx[a] > top)
                        owned = 0;
                }
                double PL[8], PR[8];
                /* gather stencil cells f-3..f+2 along d */
                size_t cid[6];
                for (int s = 0; s < 6; ++s) {
                    int t[3] = {idx[0], idx[1], idx[2]};
                    t[d] += s - 3;
                    cid[s] = IDX(G, t[0], t[1], t[2]);
                }
                for (int q = 0; q < 8; ++q) {
                    if (q == 5 + d)
                        continue;
                    double qq[6];
                    for (int s = 0; s < 6; ++s)
                        qq[s] = G->P[q][cid[s]];
                    mp5_lr(qq, &PL[q], &PR[q], c->order);
                }
                double Bn = G->B[d][id] / m.sqrtg;
                PL[5 + d] = Bn;
                PR[5 + d] = Bn;
                /* first-order fallback per side */
                for (int side = 0; side < 2; ++side) {
                    double *Ps = side == 0 ? PL : PR;
                    double v[3] = {Ps[1], Ps[2], Ps[3]}, vl[3];
                    lower3(&m, v, vl);
                    double v2 = dot3(vl, v);
                    if (!(Ps[0] > 0.0) || !(Ps[4] > 0.0) || !(v2 < 1.0)) {
                        size_t src = cid[side == 0 ? 2 : 3];
                        for (int q = 0; q < 8; ++q)
                            if (q != 5 + d)
                                Ps[q] = G->P[q][src];
                        fb += owned;
                    }
                }
                double FL[5], FR[5], UL[5], UR[5];
                flux_point(&m, c->gamma, PL, d, FL, UL);
                flux_point(&m, c->gamma, PR, d, FR, UR);
                double lpL, lmL, lpR, lmR;
                speeds_point(&m, c->gamma, PL, d, &lpL, &lmL);
                speeds_point(&m, c->gamma, PR, d, &lpR, &lmR);
                double ap = fmax(0.0, fmax(lpL, lpR));
                double am = fmax(0.0, fmax(-lmL, -lmR));
                double F[5];
                hll(FL, FR, UL, UR, ap, am, F);
                for (int q = 0; q < 5; ++q)
                    G->F[d][q][id] = F[q];
                G->ap[d][id] = ap;
                G->am[d][id] = am;
                for (int cc = 0; cc < 3; ++cc) {
                    G->vL[d][cc][id] = PL[1 + cc];
                    G->vR[d][cc][id] = PR[1 + cc];
                }
            }
    st->fallback_faces += fb;
}

/* UCT-HLL EMF at the edges parallel to direction e (Londrillo & Del Zanna
 * 2004).  With (a, b, e) cyclic, the edge with index (i,j,k) sits at
 * half-integer positions along a and b.  Velocities v^a, v^b come from a
 * two-step reconstruction: MP5 along a to the a-faces (stored by
 * faces_dir), then MP5 of those face values along b.  B~^b (on b-faces) is
 * reconstructed along a, B~^a (on a-faces) along b.  The four states are
 * labelled by (a-side, b-side):
 *   E_e = [ap_a ap_b E_LL + ap_a am_b E_LR + am_a ap_b E_RL + am_a am_b E_RR]
 *         / ((ap_a + am_a)(ap_b + am_b))
 *       + ap_a am_a/(ap_a + am_a) (B~^b_R - B~^b_L)
 *       - ap_b am_b/(ap_b + am_b) (B~^a_R - B~^a_L),
 *   E^{st} = -(vt^a_{st} B~^b_s - vt^b_{st} B~^a_t),  vt = alpha v - beta
 * at the edge.  ap_a, am_a are the maxima over the two a-faces adjacent to
 * the edge; likewise for b.  E_z uses (a, b) = (x, y), E_x (y, z), E_y (z, x). */
static void emf_dir(const ocfg *c, ogrid *G, int e)
{
    int a = (e + 1) % 3, b = (e + 2) % 3;
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = NG;
        hi[d] = NG + G->n[d];
    }
    hi[a] += 1;
    hi[b] += 1;
    /* order 1: two more edges on each side along a and b for the correction */
    lo[a] -= 2 * c->order;
    hi[a] += 2 * c->order;
    lo[b] -= 2 * c->order;
    hi[b] += 2 * c->order;
    OPC_PHASE(OPC_EMF);
#pragma omp parallel for collapse(2)
    for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
            for (int i = lo[0]; i < hi[0]; ++i) {
                OPC_UNIT();
                int idx[3] = {i, j, k};
                size_t id = IDX(G, i, j, k);
                /* stencils: along b on a-faces, along a on b-faces */
                size_t sb[6], sa[6];
                for (int s = 0; s < 6; ++s) {
                    int t[3] = {idx[0], idx[1], idx[2]};
                    t[b] += s - 3;
                    sb[s] = IDX(G, t[0], t[1], t[2]);
                    int u[3] = {idx[0], idx[1], idx[2]};
                    u[a] += s - 3;
                    sa[s] = IDX(G, u[0], u[1], u[2]);
                }
                double va[2][2], vb[2][2];  /* [a-side][b-side] */
                for (int sside = 0; sside < 2; ++sside) {
                    double *const *vs = sside == 0 ? G->vL[a] : G->vR[a];
                    double qa[6], qb[6];
                    for (int s = 0; s < 6; ++s) {
                        qa[s] = vs[a][sb[s]];
                        qb[s] = vs[b][sb[s]];
                    }
                    mp5_lr(qa, &va[sside][0], &va[sside][1], c->order);
                    mp5_lr(qb, &vb[sside][0], &vb[sside][1], c->order);
                }
                double Bb[2], Ba[2];
                {
                    double q[6];
                    for (int s = 0; s < 6; ++s)
                        q[s] = G->B[b][sa[s]];
                    mp5_lr(q, &Bb[0], &Bb[1], c->order);
                    for (int s = 0; s < 6; ++s)
                        q[s] = G->B[a][sb[s]];
                    mp5_lr(q, &Ba[0], &Ba[1], c->order);
                }
                size_t a0 = sb[2], a1 = sb[3];  /* a-faces at b-1, b */
                size_t b0 = sa[2], b1 = sa[3];  /* b-faces at a-1, a */
                double apa = fmax(G->ap[a][a0], G->ap[a][a1]);
                double ama = fmax(G->am[a][a0], G->am[a][a1]);
                double apb = fmax(G->ap[b][b0], G->ap[b][b1]);
                double amb = fmax(G->am[b][b0], G->am[b][b1]);
                double x[3] = {coord(c, 0, i, e == 0 ? 0.0 : -0.5), coord(c, 1, j, e == 1 ? 0.0 : -0.5),
                               coord(c, 2, k, e == 2 ? 0.0 : -0.5)};
                double alpha, beta[3], g[3][3];
                metric_components(c, x, &alpha, beta, g);
                double Est[2][2];
                for (int s = 0; s < 2; ++s)
                    for (int t = 0; t < 2; ++t) {
                        double vta = alpha * va[s][t] - beta[a];
                        double vtb = alpha * vb[s][t] - beta[b];
                        Est[s][t] = -(vta * Bb[s] - vtb * Ba[t]);
                    }
                double sa_ = apa + ama, sb_ = apb + amb;
                double wLL, wLR, wRL, wRR, da, db;
                if (sa_ > 0.0 && sb_ > 0.0) {
                    double den = sa_ * sb_;
                    wLL = apa * apb / den;
                    wLR = apa * amb / den;
                    wRL = ama * apb / den;
                    wRR = ama * amb / den;
                } else {
                    wLL = wLR = wRL = wRR = 0.25;
                }
                da = sa_ > 0.0 ? apa * ama / sa_ : 0.0;
                db = sb_ > 0.0 ? apb * amb / sb_ : 0.0;
                G->E[e][id] = wLL * Est[0][0] + wLR * Est[0][1] + wRL * Est[1][0] + wRR * Est[1][1]
                              + da * (Bb[1] - Bb[0]) - db * (Ba[1] - Ba[0]);
            }
}

/* Geometric source terms of the Valencia form on a stationary metric, at
 * the cell centre, multiplied by sqrt(gamma):
 *   S(S_i) = 1/2 alpha W^jk d_i gamma_jk + S_j d_i beta^j - U d_i alpha
 *   S(tau) = 1/2 W^ik beta^j d_j gamma_ik + W_i^j d_j beta^i - S^j d_j alpha
 * (the second is alpha K_ij W^ij - S^j d_j alpha with d_t gamma_ij = 0).
 * Metric derivatives: sixth-order centred differences of the closed-form
 * metric with step dx^d.  Zero in flat space. */
static void sources_point(const ocfg *c, const double x[3], const ometric *m, const double *P,
                          double src[5])
{
    for (int q = 0; q < 5; ++q)
        src[q] = 0.0;
    if (c->metric == 0)
        return;
    double dal[3], dbe[3][3], dg[3][3][3];
    for (int d = 0; d < 3; ++d) {
        OPC_UNCOUNTED;
        double h = c->dx[d];
        double wts[6] = {-1.0, 9.0, -45.0, 45.0, -9.0, 1.0};
        double offs[6] = {-3.0, -2.0, -1.0, 1.0, 2.0, 3.0};
        dal[d] = 0.0;
        for (int i = 0; i < 3; ++i) {
            dbe[d][i] = 0.0;
            for (int j = 0; j < 3; ++j)
                dg[d][i][j] = 0.0;
        }
        for (int s = 0; s < 6; ++s) {
            double y[3] = {x[0], x[1], x[2]};
            y[d] += offs[s] * h;
            double al, be[3], g[3][3];
            metric_components(c, y, &al, be, g);
            dal[d] += wts[s] * al;
            for (int i = 0; i < 3; ++i) {
                dbe[d][i] += wts[s] * be[i];
                for (int j = 0; j < 3; ++j)
                    dg[d][i][j] += wts[s] * g[i][j];
            }
        }
        dal[d] /= 60.0 * h;
        for (int i = 0; i < 3; ++i) {
            dbe[d][i] /= 60.0 * h;
            for (int j = 0; j < 3; ++j)
                dg[d][i][j] /= 60.0 * h;
        }
    }
    double v[3] = {P[1], P[2], P[3]}, B[3] = {P[5], P[6], P[7]};
    double vl[3], Bl[3];
    lower3(m, v, vl);
    lower3(m, B, Bl);
    double v2 = dot3(vl, v), B2 = dot3(Bl, B), vB = dot3(vl, B);
    double W = 1.0 / sqrt(1.0 - v2);
    double rho = P[0], p = P[4];
    double rhoh = rho + c->gamma / (c->gamma - 1.0) * p;
    double b2 = B2 / (W * W) + vB * vB;
    double bu[3];
    for (int i = 0; i < 3; ++i)
        bu[i] = B[i] / W + W * vB * v[i];
    double Wuu[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Wuu[i][j] = (rhoh + b2) * W * W * v[i] * v[j] + (p + 0.5 * b2) * m->gi[i][j] - bu[i] * bu[j];
    double C[5];
    p2c_point(m, c->gamma, P, C);
    double Sl[3] = {C[1], C[2], C[3]}, Su[3];
    raise3(m, Sl, Su);
    double U = C[4] + C[0];
    for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                s += 0.5 * m->alpha * Wuu[j][k] * dg[i][j][k];
        for (int j = 0; j < 3; ++j)
            s += Sl[j] * dbe[i][j];
        s -= U * dal[i];
        src[1 + i] = s * m->sqrtg;
    }
    double st = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j)
                st += 0.5 * Wuu[i][k] * m->beta[j] * dg[j][i][k];
    /* W_i^j d_j beta^i, W_i^j = gamma_ik W^kj */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double Wij = 0.0;
            for (int k = 0; k < 3; ++k)
                Wij += m->g[i][k] * Wuu[k][j];
            st += Wij * dbe[j][i];
        }
    for (int j = 0; j < 3; ++j)
        st -= Su[j] * dal[j];
    src[4] = st * m->sqrtg;
}

/* Owned face range along d for a d-face array: periodic g..g+n-1,
 * outflow g..g+n, axis faces are held at zero. */
static void owned_faces(const ocfg *c, int d, int *lo, int *hi)
{
    *lo = NG;
    *hi = NG + c->n[d] - 1;
    if (c->bc[2 * d] != BC_PERIODIC)
        *hi = NG + c->n[d];
    if (c->bc[2 * d] == BC_AXIS)
        *lo = NG + 1;
    if (c->bc[2 * d + 1] == BC_AXIS)
        *hi = NG + c->n[d] - 1;
}

/* Order 1: the flux-derivative correction (ho_flux) of the fluxes along
 * their own direction on the owned faces, and of each EMF E_e along each of
 * its two half-integer directions (the induction equation differences E_e
 * along both): Ec[e][0] along (e+1)%3, Ec[e][1] along (e+2)%3.  The 1-D
 * corrections along different axes commute, so the discrete divergence
 * built from the same corrected differences stays constant. */
static void ho_correct(const ocfg *c, ogrid *G)
{
    OPC_PHASE(OPC_CORRECT);
    for (int d = 0; d < 3; ++d) {
#pragma omp parallel for collapse(2)
        for (int k = NG; k < NG + G->n[2] + (d == 2); ++k)
            for (int j = NG; j < NG + G->n[1] + (d == 1); ++j)
                for (int i = NG; i < NG + G->n[0] + (d == 0); ++i) {
                    size_t id = IDX(G, i, j, k);
                    for (int q = 0; q < 5; ++q) {
                        double f5[5];
                        for (int s = 0; s < 5; ++s) {
                            int t[3] = {i, j, k};
                            t[d] += s - 2;
                            f5[s] = G->F[d][q][IDX(G, t[0], t[1], t[2])];
                        }
                        G->Fc[d][q][id] = ho_flux(f5);
                    }
                }
    }
    for (int e = 0; e < 3; ++e)
        for (int w = 0; w < 2; ++w) {
            int dir = (e + 1 + w) % 3;
            int hi[3] = {NG + G->n[0] + 1, NG + G->n[1] + 1, NG + G->n[2] + 1};
            hi[e] -= 1;
#pragma omp parallel for collapse(2)
            for (int k = NG; k < hi[2]; ++k)
                for (int j = NG; j < hi[1]; ++j)
                    for (int i = NG; i < hi[0]; ++i) {
                        double f5[5];
                        for (int s = 0; s < 5; ++s) {
                            int t[3] = {i, j, k};
                            t[dir] += s - 2;
                            f5[s] = G->E[e][IDX(G, t[0], t[1], t[2])];
                        }
                        G->Ec[e][w][IDX(G, i, j, k)] = ho_flux(f5);
                    }
        }
}

/* L(U): flux difference plus sources for the cell variables, minus the
 * curl of the edge EMFs for the face field (order 1: of the corrected
 * fluxes and EMFs). */
static void assemble(const ocfg *c, ogrid *G)
{
    OPC_PHASE(OPC_ASSEMBLE);
#pragma omp parallel for collapse(2)
    for (int k = NG; k < NG + G->n[2]; ++k)
        for (int j = NG; j < NG + G->n[1]; ++j)
            for (int i = NG; i < NG + G->n[0]; ++i) {
                OPC_UNIT();
                size_t id = IDX(G, i, j, k);
                size_t nb[3] = {IDX(G, i + 1, j, k), IDX(G, i, j + 1, k), IDX(G, i, j, k + 1)};
                double x[3] = {coord(c, 0, i, 0), coord(c, 1, j, 0), coord(c, 2, k, 0)};
                double src[5];
                if (c->metric != 0) {
                    ometric m;
                    metric_eval(c, x, &m);
                    double P[8];
                    for (int q = 0; q < 8; ++q)
                        P[q] = G->P[q][id];
                    sources_point(c, x, &m, P, src);
                } else {
                    for (int q = 0; q < 5; ++q)
                        src[q] = 0.0;
                }
                for (int q = 0; q < 5; ++q) {
                    double r = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        const double *F = c->order ? G->Fc[d][q] : G->F[d][q];
                        r -= (F[nb[d]] - F[id]) / c->dx[d];
                    }
                    G->LU[q][id] = r + src[q];
                }
            }
    /* face field: dB~^x/dt = -(dE_z/dy - dE_y/dz), cyclic */
    OPC_PHASE(OPC_CT);
    for (int d = 0; d < 3; ++d) {
        int a = (d + 1) % 3, b = (d + 2) % 3;
        int flo, fhi;
        owned_faces(c, d, &flo, &fhi);
        int lo[3] = {NG, NG, NG}, hi[3] = {NG + G->n[0] - 1, NG + G->n[1] - 1, NG + G->n[2] - 1};
        lo[d] = flo;
        hi[d] = fhi;
#pragma omp parallel for collapse(2)
        for (int k = lo[2]; k <= hi[2]; ++k)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int i = lo[0]; i <= hi[0]; ++i) {
                    OPC_UNIT();
                    int idx[3] = {i, j, k};
                    size_t id = IDX(G, i, j, k);
                    int ta[3] = {idx[0], idx[1], idx[2]};
                    ta[a] += 1;
                    int tb[3] = {idx[0], idx[1], idx[2]};
                    tb[b] += 1;
                    /* E_b varies along a: its edges at a+-1/2; E_a along b.  Order 1:
                     * E_b corrected along a = (b+2)%3, E_a along b = (a+1)%3 */
                    const double *Eb = c->order ? G->Ec[b][1] : G->E[b];
                    const double *Ea = c->order ? G->Ec[a][0] : G->E[a];
                    double dEb_da = (Eb[IDX(G, ta[0], ta[1], ta[2])] - Eb[id]) / c->dx[a];
                    double dEa_db = (Ea[IDX(G, tb[0], tb[1], tb[2])] - Ea[id]) / c->dx[b];
                    /* (curl E)^d = d_a E_b - d_b E_a */
                    G->LB[d][id] = -(dEb_da - dEa_db);
                }
    }
}

/* Order 1: admissibility safeguard of the flux-derivative correction, in up
 * to GUARD_PASSES passes after assemble has formed L(U) with the corrected
 * fluxes.  A pass forms every owned cell's stage result as the SSP-RK3
 * stage would form it (stage 0: U + dt L; 1: 3/4 U0 + 1/4 (U + dt L);
 * 2: 1/3 U0 + 2/3 (U + dt L)) for the five cell variables, with the
 * cell-centre field of the current state, and flags (for good) every cell
 * whose result the inversion (c2p_point, from the cell's Z) cannot invert;
 * every face of a flagged cell then takes the uncorrected flux (the scheme
 * of order 0) in place of the corrected one -- the same value for both
 * cells sharing it, a periodic axis pairing the faces across the seam with
 * the cells they bound -- and L(U) is assembled again.  A face replaced
 * changes the result of the neighbouring cell too, hence the further
 * passes; they stop when one flags no new cell.  U0: the stage base (the
 * state after the first stage's inversion).  Returns the faces replaced,
 * counted once each. */
#define GUARD_PASSES 3

static long long guard_mark(const ocfg *c, ogrid *G, double dt, int stage, double *const *U0)
{
    long long added = 0;
    const double wa = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
    const double wb = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
#pragma omp parallel for collapse(2) reduction(+ : added)
    for (int k = NG; k < NG + G->n[2]; ++k)
        for (int j = NG; j < NG + G->n[1]; ++j)
            for (int i = NG; i < NG + G->n[0]; ++i) {
                size_t id = IDX(G, i, j, k);
                if (G->mark[id] != 0.0)
                    continue;
                double x[3] = {coord(c, 0, i, 0), coord(c, 1, j, 0), coord(c, 2, k, 0)};
                ometric m;
                metric_eval(c, x, &m);
                double C[5];
                for (int q = 0; q < 5; ++q) {
                    double fe = G->U[q][id] + dt * G->LU[q][id];
                    double u = stage == 0 ? fe : wa * U0[q][id] + wb * fe;
                    C[q] = u / m.sqrtg;
                }
                double Bc[3] = {G->P[5][id], G->P[6][id], G->P[7][id]};
                double P5[5], Zc;
                int its;
                if (c2p_point(&m, c->gamma, C, Bc, G->Z[id], P5, &Zc, &its)) {
                    G->mark[id] = 1.0;
                    added += 1;
                }
            }
    return added;
}

/* Faces bounding a flagged cell take the uncorrected flux; returns the
 * owned faces that now differ from their corrected value, counted once. */
static long long guard_revert(const ocfg *c, ogrid *G)
{
    long long replaced = 0;
    for (int d = 0; d < 3; ++d) {
        int per = c->bc[2 * d] == BC_PERIODIC;
        int hi[3] = {NG + G->n[0] - 1, NG + G->n[1] - 1, NG + G->n[2] - 1};
        hi[d] = NG + G->n[d];
#pragma omp parallel for collapse(2) reduction(+ : replaced)
        for (int k = NG; k <= hi[2]; ++k)
            for (int j = NG; j <= hi[1]; ++j)
                for (int i = NG; i <= hi[0]; ++i) {
                    int idx[3] = {i, j, k};
                    /* the cells on the two sides of face idx along d */
                    int lo_c[3] = {i, j, k}, hi_c[3] = {i, j, k};
                    lo_c[d] -= 1;
                    int f = 0;
                    for (int side = 0; side < 2; ++side) {
                        int *t = side == 0 ? lo_c : hi_c;
                        if (t[d] < NG || t[d] >= NG + G->n[d]) {
                            if (!per)
                                continue;
                            t[d] = NG + ((t[d] - NG) % G->n[d] + G->n[d]) % G->n[d];
                        }
                        if (G->mark[IDX(G, t[0], t[1], t[2])] != 0.0)
                            f = 1;
                    }
                    if (!f)
                        continue;
                    size_t id = IDX(G, idx[0], idx[1], idx[2]);
                    int changed = 0;
                    for (int q = 0; q < 5; ++q) {
                        changed |= G->Fc[d][q][id] != G->F[d][q][id];
                        G->Fc[d][q][id] = G->F[d][q][id];
                    }
                    /* the periodic duplicate face NG + n is the face NG */
                    if (changed && !(per && idx[d] == NG + G->n[d]))
                        replaced += 1;
                }
    }
    return replaced;
}

static long long ho_guard(const ocfg *c, ogrid *G, double dt, int stage, double *const *U0)
{
    OPC_PHASE(OPC_CORRECT);
    memset(G->mark, 0, G->ncell * sizeof(double));
    long long replaced = 0;
    for (int pass = 0; pass < GUARD_PASSES; ++pass) {
        if (!guard_mark(c, G, dt, stage, U0))
            break;
        replaced += guard_revert(c, G);
        assemble(c, G);
    }
    return replaced;
}

/* One evaluation of L(U) on the grid G (U, B, Z set on owned cells).
 * save (may be NULL): 8 arrays that receive U and B~ right after the c2p,
 * i.e. after floors and failure fallbacks have reset the conserved state.
 * dt: the step the stage takes, for the safeguard of order 1 (ho_guard):
 * > 0 that step; < 0 the CFL step cfl / rate_max of this evaluation (rate_max
 * then non-NULL); 0 no safeguard (L(U) alone, with no step to check).
 * stage, U0: the SSP-RK3 stage (0..2) and its base state, for the same. */
static int eval_rhs(const ocfg *c, ogrid *G, ostats *st, double *rate_max, double *const *save, double dt,
                    int stage, double *const *U0)
{
    OPC_PHASE(OPC_OTHER);
    fill_faces(c, G);
    if (c2p_grid(c, G, st))
        return -1;
    if (save) {
        for (int q = 0; q < 5; ++q)
            memcpy(save[q], G->U[q], G->ncell * sizeof(double));
        for (int q = 0; q < 3; ++q)
            memcpy(save[5 + q], G->B[q], G->ncell * sizeof(double));
    }
    if (rate_max)
        *rate_max = cfl_rate_max(c, G);
    fill_prims(c, G);
    for (int d = 0; d < 3; ++d)
        faces_dir(c, G, d, st);
    for (int e = 0; e < 3; ++e)
        emf_dir(c, G, e);
    if (c->order)
        ho_correct(c, G);
    assemble(c, G);
    if (c->order && dt != 0.0) {
        double h = dt > 0.0 ? dt : c->cfl / *rate_max;
        st->guard_faces += ho_guard(c, G, h, stage, stage == 0 ? save : U0);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Exported API (ctypes)                                               */
/* ------------------------------------------------------------------ */

/* Pointwise functions, for tests that pin the physics. */
void oracle_metric_point(const ocfg *c, const double *x, double *out)
{
    /* out: alpha, beta[3], g[9], gi[9], sqrtg  (23 doubles) */
    ometric m;
    metric_eval(c, x, &m);
    out[0] = m.alpha;
    for (int i = 0; i < 3; ++i)
        out[1 + i] = m.beta[i];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            out[4 + 3 * i + j] = m.g[i][j];
            out[13 + 3 * i + j] = m.gi[i][j];
        }
    out[22] = m.sqrtg;
}

void oracle_p2c_point(const ocfg *c, const double *x, const double *P8, double *C5)
{
    ometric m;
    metric_eval(c, x, &m);
    p2c_point(&m, c->gamma, P8, C5);
}

int oracle_c2p_point(const ocfg *c, const double *x, const double *C5, const double *B3, double Zguess,
                     double *P5, double *Z, int *iters)
{
    ometric m;
    metric_eval(c, x, &m);
    return c2p_point(&m, c->gamma, C5, B3, Zguess, P5, Z, iters);
}

/* Residual f(Z) and its derivative, for the finite-difference pin. */
void oracle_c2p_residual(const ocfg *c, const double *x, const double *C5, const double *B3, double Z,
                         double *f, double *fp)
{
    ometric m;
    metric_eval(c, x, &m);
    double D = C5[0], tau = C5[4];
    double S[3] = {C5[1], C5[2], C5[3]}, Su[3], Bl[3];
    raise3(&m, S, Su);
    lower3(&m, B3, Bl);
    double S2 = dot3(S, Su), SB = dot3(S, B3), B2 = dot3(Bl, B3), U = tau + D;
    double gg = (c->gamma - 1.0) / c->gamma;
    double v2 = c2p_v2(Z, S2, SB, B2);
    double sq = sqrt(1.0 - v2);
    double p = gg * (Z * (1.0 - v2) - D * sq);
    *f = Z - p + 0.5 * (1.0 + v2) * B2 - SB * SB / (2.0 * Z * Z) - U;
    double ZB = Z + B2;
    double dv2 = -2.0 * (S2 * Z * Z * Z + SB * SB * (3.0 * Z * Z + 3.0 * Z * B2 + B2 * B2))
                 / (Z * Z * Z * ZB * ZB * ZB);
    double dp = gg * ((1.0 - v2) - Z * dv2 + D * dv2 / (2.0 * sq));
    *fp = 1.0 - dp + 0.5 * B2 * dv2 + SB * SB / (Z * Z * Z);
}

double oracle_mp5_face(const double *u5) { return mp5_face(u5[0], u5[1], u5[2], u5[3], u5[4], 0); }
double oracle_mp5_face_order(const double *u5, int order)
{
    return mp5_face(u5[0], u5[1], u5[2], u5[3], u5[4], order);
}
double oracle_ho_flux(const double *f5) { return ho_flux(f5); }
double oracle_ho_center(const double *b6) { return ho_center(b6); }

/* Ghost layers per side of every padded array. */
int oracle_ghosts(void) { return NG; }

/* Threads of the OpenMP loops from now on (n >= 1; no effect in a build
 * without OpenMP), for timing the oracle on a chosen number of cores. */
#ifdef _OPENMP
#include <omp.h>
#endif
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Ghost fill of one padded array (n[d] + 2 NG entries along each d, x
 * fastest; a face array holds face i-1/2 at index i) with the grid's
 * boundary conditions: the routine every step uses, exposed for the
 * boundary-condition pins.  comp, face and dens as in fill_array. */
void oracle_fill_padded(const ocfg *c, double *a, int comp, int face, int dens)
{
    ogrid G;
    memset(&G, 0, sizeof(G));
    for (int d = 0; d < 3; ++d) {
        G.n[d] = c->n[d];
        G.np[d] = c->n[d] + 2 * NG;
    }
    G.ncell = (size_t)G.np[0] * G.np[1] * G.np[2];
    fill_array(c, &G, a, comp, face, dens);
}

/* Unlimited fifth-order value, for the polynomial-exactness pin. */
double oracle_mp5_unlimited(const double *u5)
{
    return (2.0 * u5[0] - 13.0 * u5[1] + 47.0 * u5[2] + 27.0 * u5[3] - 3.0 * u5[4]) / 60.0;
}

void oracle_speeds_point(const ocfg *c, const double *x, const double *P8, int d, double *lp, double *lm)
{
    ometric m;
    metric_eval(c, x, &m);
    speeds_point(&m, c->gamma, P8, d, lp, lm);
}

void oracle_flux_point(const ocfg *c, const double *x, const double *P8, int d, double *F5, double *U5)
{
    ometric m;
    metric_eval(c, x, &m);
    flux_point(&m, c->gamma, P8, d, F5, U5);
}

void oracle_hll(const double *FL, const double *FR, const double *UL, const double *UR, double ap,
                double am, double *F)
{
    hll(FL, FR, UL, UR, ap, am, F);
}

void oracle_sources_point(const ocfg *c, const double *x, const double *P8, double *src5)
{
    ometric m;
    metric_eval(c, x, &m);
    sources_point(c, x, &m, P8, src5);
}

size_t oracle_state_count(const int *n) { return state_count(n); }

/* Primitives (rho, v^x, v^y, v^z, p; 5 cell arrays) and the face field B~
 * (host face layout) -> conserved state (host layout) and Z = rho h W^2. */
int oracle_p2c(const ocfg *c, const double *prims, const double *bface, double *state, double *Zout)
{
    ogrid G;
    if (grid_alloc(&G, c->n))
        return -2;
    const int *n = c->n;
    size_t N = (size_t)n[0] * n[1] * n[2];
    /* face field into the grid, then ghost fill for the cell average */
    double *tmp = (double *)calloc(state_count(n), sizeof(double));
    if (!tmp) {
        grid_free(&G);
        return -2;
    }
    memcpy(tmp + 5 * N, bface, (state_count(n) - 5 * N) * sizeof(double));
    unpack_state(&G, tmp);
    fill_faces(c, &G);
    for (int k = NG; k < NG + n[2]; ++k)
        for (int j = NG; j < NG + n[1]; ++j)
            for (int i = NG; i < NG + n[0]; ++i) {
                size_t id = IDX(&G, i, j, k);
                size_t h = ((size_t)(k - NG) * n[1] + (j - NG)) * n[0] + (i - NG);
                double x[3] = {coord(c, 0, i, 0), coord(c, 1, j, 0), coord(c, 2, k, 0)};
                ometric m;
                metric_eval(c, x, &m);
                double P[8];
                for (int q = 0; q < 5; ++q)
                    P[q] = prims[q * N + h];
                cell_centre_B(c, &G, i, j, k, m.sqrtg, P + 5);
                double C[5];
                p2c_point(&m, c->gamma, P, C);
                for (int q = 0; q < 5; ++q)
                    G.U[q][id] = C[q] * m.sqrtg;
                double v[3] = {P[1], P[2], P[3]}, vl[3];
                lower3(&m, v, vl);
                double W2 = 1.0 / (1.0 - dot3(vl, v));
                if (Zout)
                    Zout[h] = (P[0] + c->gamma / (c->gamma - 1.0) * P[4]) * W2;
            }
    pack_arrays(&G, G.U, G.B, state);
    free(tmp);
    grid_free(&G);
    return 0;
}

/* c2p of a state: outputs 8 cell arrays (rho, v^x, v^y, v^z, p, B^x, B^y,
 * B^z) and Z; Zguess may be NULL (then the cold guess tau + D is used via
 * the admissibility rule with Z = 0). stats: iters, calls, fails, floors. */
int oracle_c2p(const ocfg *c, const double *state, const double *Zguess, double *prims8, double *Zout,
               long long *stats4)
{
    ogrid G;
    if (grid_alloc(&G, c->n))
        return -2;
    unpack_state(&G, state);
    if (Zguess)
        unpack_cell(&G, Zguess, G.Z);
    fill_faces(c, &G);
    ostats st = {0, 0, 0, 0, 0, 0};
    int rc = c2p_grid(c, &G, &st);
    size_t N = (size_t)c->n[0] * c->n[1] * c->n[2];
    for (int q = 0; q < 8; ++q)
        pack_cell(&G, G.P[q], prims8 + q * N);
    if (Zout)
        pack_cell(&G, G.Z, Zout);
    if (stats4) {
        stats4[0] = st.c2p_iters;
        stats4[1] = st.c2p_calls;
        stats4[2] = st.c2p_fail;
        stats4[3] = st.floor_hits;
    }
    grid_free(&G);
    return rc;
}

/* L(U) of a state in host layout; Z (N values) is the Newton guess and is
 * updated in place.  rate_max (may be NULL) receives max_cells sum_d
 * max|lambda_d|/dx_d. */
int oracle_rhs(const ocfg *c, const double *state, double *Z, double *L, double *rate_max)
{
    ogrid G;
    if (grid_alloc(&G, c->n))
        return -2;
    unpack_state(&G, state);
    unpack_cell(&G, Z, G.Z);
    ostats st = {0, 0, 0, 0, 0, 0};
    int rc = eval_rhs(c, &G, &st, rate_max, NULL, 0.0, 0, NULL);
    if (rc == 0) {
        /* periodic axes: the duplicate last face repeats the first */
        for (int d = 0; d < 3; ++d)
            fill_array(c, &G, G.LB[d], d, d, 1);
        pack_arrays(&G, G.LU, G.LB, L);
        pack_cell(&G, G.Z, Z);
    }
    grid_free(&G);
    return rc;
}

/* nsteps SSP-RK3 steps (Shu & Osher 1988):
 *   U1 = U0 + dt L(U0)
 *   U2 = 3/4 U0 + 1/4 (U1 + dt L(U1))
 *   U3 = 1/3 U0 + 2/3 (U2 + dt L(U2)).
 * U0 is the state at the start of the step after the first stage's c2p
 * (floors and failure fallbacks reset the conserved variables there).
 * dt_in > 0: fixed dt; otherwise dt = cfl / max_cells sum_d max|lambda_d|/dx_d
 * from the primitives of the first stage of each step.  dts (may be NULL)
 * receives the dt of each step; stats6 (may be NULL): c2p iterations, c2p
 * calls, c2p failures, floor hits, first-order fallback faces, faces the
 * order-1 safeguard replaced.
 * The state (host layout) and Z are updated in place. */
int oracle_steps(const ocfg *c, double *state, double *Z, int nsteps, double dt_in, double *dts,
                 long long *stats6)
{
    ogrid G;
    if (grid_alloc(&G, c->n))
        return -2;
    unpack_state(&G, state);
    unpack_cell(&G, Z, G.Z);
    ostats st = {0, 0, 0, 0, 0, 0};
    size_t N = G.ncell;
    double *U0[8];
    for (int q = 0; q < 8; ++q)
        U0[q] = (double *)malloc(N * sizeof(double));
    double *const Ucur[8] = {G.U[0], G.U[1], G.U[2], G.U[3], G.U[4], G.B[0], G.B[1], G.B[2]};
    double *const Lcur[8] = {G.LU[0], G.LU[1], G.LU[2], G.LU[3], G.LU[4], G.LB[0], G.LB[1], G.LB[2]};
    int rc = 0;
    for (int step = 0; step < nsteps && rc == 0; ++step) {
        double dt = dt_in;
        for (int s = 0; s < 3 && rc == 0; ++s) {
            double rmax = 0.0;
            rc = eval_rhs(c, &G, &st, s == 0 && dt_in <= 0.0 ? &rmax : NULL, s == 0 ? U0 : NULL,
                          s == 0 && dt_in <= 0.0 ? -1.0 : dt, s, U0);
            if (rc)
                break;
            if (s == 0 && dt_in <= 0.0)
                dt = c->cfl / rmax;
            OPC_PHASE(OPC_RK);
            for (int q = 0; q < 8; ++q) {
                int isface = q >= 5;
                int d = q - 5;
                int lo[3] = {NG, NG, NG}, hi[3] = {NG + c->n[0] - 1, NG + c->n[1] - 1, NG + c->n[2] - 1};
                if (isface)
                    owned_faces(c, d, &lo[d], &hi[d]);
                double *u = Ucur[q], *l = Lcur[q], *u0 = U0[q];
                for (int k = lo[2]; k <= hi[2]; ++k)
                    for (int j = lo[1]; j <= hi[1]; ++j)
                        for (int i = lo[0]; i <= hi[0]; ++i) {
                            OPC_UNIT();
                            size_t id = IDX(&G, i, j, k);
                            if (s == 0)
                                u[id] = u0[id] + dt * l[id];
                            else if (s == 1)
                                u[id] = 0.75 * u0[id] + 0.25 * (u[id] + dt * l[id]);
                            else
                                u[id] = (1.0 / 3.0) * u0[id] + (2.0 / 3.0) * (u[id] + dt * l[id]);
                        }
            }
        }
        if (dts)
            dts[step] = dt;
    }
    if (rc == 0) {
        /* fill the periodic duplicate faces before packing */
        fill_faces(c, &G);
        pack_arrays(&G, G.U, G.B, state);
        pack_cell(&G, G.Z, Z);
    }
    if (stats6) {
        stats6[0] = st.c2p_iters;
        stats6[1] = st.c2p_calls;
        stats6[2] = st.c2p_fail;
        stats6[3] = st.floor_hits;
        stats6[4] = st.fallback_faces;
        stats6[5] = st.guard_faces;
    }
    for (int q = 0; q < 8; ++q)
        free(U0[q]);
    grid_free(&G);
    return rc;
}

/* Totals of a state: out[0] = sum D dV, out[1] = sum tau dV,
 * out[2..4] = sum S_i dV, out[5] = max |div B~| over owned cells, with
 * dV = dx dy dz and div B~ = sum_d (B~^d_{i+1/2} - B~^d_{i-1/2}) / dx^d. */
int oracle_reduce(const ocfg *c, const double *state, double *out)
{
    ogrid G;
    if (grid_alloc(&G, c->n))
        return -2;
    unpack_state(&G, state);
    fill_faces(c, &G);
    double dV = c->dx[0] * c->dx[1] * c->dx[2];
    double sD = 0.0, sT = 0.0, sS[3] = {0.0, 0.0, 0.0}, mdiv = 0.0;
    for (int k = NG; k < NG + c->n[2]; ++k)
        for (int j = NG; j < NG + c->n[1]; ++j)
            for (int i = NG; i < NG + c->n[0]; ++i) {
                size_t id = IDX(&G, i, j, k);
                sD += G.U[0][id] * dV;
                sT += G.U[4][id] * dV;
                for (int q = 0; q < 3; ++q)
                    sS[q] += G.U[1 + q][id] * dV;
                double dv = 0.0;
                for (int d = 0; d < 3; ++d) {
                    /* order 0: B~(i+1) - B~(i); order 1: the same difference of
                     * the corrected face values (the divergence that order 1
                     * keeps constant) */
                    double bf[2];
                    for (int side = 0; side < 2; ++side) {
                        int t[3] = {i, j, k};
                        t[d] += side;
                        if (c->order) {
                            double f5[5];
                            for (int s = 0; s < 5; ++s) {
                                int u[3] = {t[0], t[1], t[2]};
                                u[d] += s - 2;
                                f5[s] = G.B[d][IDX(&G, u[0], u[1], u[2])];
                            }
                            bf[side] = ho_flux(f5);
                        } else {
                            bf[side] = G.B[d][IDX(&G, t[0], t[1], t[2])];
                        }
                    }
                    dv += (bf[1] - bf[0]) / c->dx[d];
                }
                mdiv = fmax(mdiv, fabs(dv));
            }
    out[0] = sD;
    out[1] = sT;
    out[2] = sS[0];
    out[3] = sS[1];
    out[4] = sS[2];
    out[5] = mdiv;
    grid_free(&G);
    return 0;
}
