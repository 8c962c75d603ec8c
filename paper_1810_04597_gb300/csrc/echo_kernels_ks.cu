// echo_kernels_ks.cu -- instantiation of the metric-dependent kernels for the
// Kerr-Schild metric, plus the kernel that builds its FP64 tables.
#include "echo_kernels.cuh"
#define ECHO_MK 1
#include "echo_launch_mk.inc"

namespace echo {

// Kerr metric in Kerr-Schild form, coordinates (ln r, theta, phi), M = 1:
//   Sigma = r^2 + a^2 cos^2, z = 2 r / Sigma, alpha = (1 + z)^-1/2,
//   beta^r = z / (1 + z), gamma_rr = 1 + z, gamma_rphi = -a (1 + z) sin^2,
//   gamma_thth = Sigma, gamma_phph = sin^2 (Sigma + a^2 (1 + z) sin^2);
// dr = r dx1 scales the x1 row and column by r and beta^1 = beta^r / r.
__device__ void ks_components(double x1, double th, double a, double &al, double &b1, double &g11, double &g13,
                              double &g22, double &g33)
{
    const double r = exp(x1);
    const double c = cos(th), sn = sin(th);
    const double s2 = sn * sn;
    const double sig = r * r + a * a * c * c;
    const double z = 2.0 * r / sig;
    al = 1.0 / sqrt(1.0 + z);
    b1 = z / (1.0 + z) / r;
    g11 = (1.0 + z) * r * r;
    g13 = -a * (1.0 + z) * s2 * r;
    g22 = sig;
    g33 = s2 * (sig + a * a * (1.0 + z) * s2);
}

__device__ MetPt ks_point(double x1, double th, double a)
{
    MetPt m;
    ks_components(x1, th, a, m.al, m.b1, m.g11, m.g13, m.g22, m.g33);
    const double det2 = m.g11 * m.g33 - m.g13 * m.g13;
    const double det = det2 * m.g22;
    if (det > 0.0) {
        m.i11 = m.g33 / det2;
        m.i13 = -m.g13 / det2;
        m.i33 = m.g11 / det2;
        m.i22 = 1.0 / m.g22;
        m.sg = sqrt(det);
        m.isg = 1.0 / m.sg;
    } else {
        // polar axis: degenerate metric, zero face area
        m.i11 = m.i13 = m.i22 = m.i33 = 0.0;
        m.sg = m.isg = 0.0;
    }
    return m;
}

// One thread per (i, j) of the padded (x1, x2) plane: the four table
// positions, sixth-order centred derivatives at the cell centre
// ((f(-2h) - 8 f(-h) + 8 f(h) - f(2h)) / (12 h), h = dx^d), and per i the
// floors f0 r^pow at the cell centre.
__global__ void k_metric_tables(Geom g, double a, MetTables T, double rho_floor, double rho_pow, double p_floor,
                                double p_pow)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= g.np[0] || j >= g.np[1])
        return;
    const double xc = g.x0[0] + ((double)(i - NG) + 0.5) * g.dx[0];
    const double xf = g.x0[0] + ((double)(i - NG)) * g.dx[0];
    const double tc = g.x0[1] + ((double)(j - NG) + 0.5) * g.dx[1];
    const double tf = g.x0[1] + ((double)(j - NG)) * g.dx[1];
    const int id = j * T.np0 + i;
    T.C[id] = ks_point(xc, tc, a);
    T.F1[id] = ks_point(xf, tc, a);
    T.F2[id] = ks_point(xc, tf, a);
    T.K[id] = ks_point(xf, tf, a);
    MetDer dv;
    // sixth-order centred differences of the closed-form metric
    const double w[6] = {-1.0, 9.0, -45.0, 45.0, -9.0, 1.0};
    const double o[6] = {-3.0, -2.0, -1.0, 1.0, 2.0, 3.0};
    for (int d = 0; d < 2; ++d) {
        double acc[6] = {0, 0, 0, 0, 0, 0};
        const double h = g.dx[d];
        for (int s = 0; s < 6; ++s) {
            double v[6];
            const double x1 = d == 0 ? xc + o[s] * h : xc;
            const double th = d == 1 ? tc + o[s] * h : tc;
            ks_components(x1, th, a, v[0], v[1], v[2], v[3], v[4], v[5]);
            for (int c = 0; c < 6; ++c)
                acc[c] += w[s] * v[c];
        }
        dv.dal[d] = acc[0] / (60.0 * h);
        dv.db1[d] = acc[1] / (60.0 * h);
        dv.dg11[d] = acc[2] / (60.0 * h);
        dv.dg13[d] = acc[3] / (60.0 * h);
        dv.dg22[d] = acc[4] / (60.0 * h);
        dv.dg33[d] = acc[5] / (60.0 * h);
    }
    T.dC[id] = dv;
    if (T.Cf) {
        // the FP32 copies, rounded once here
        const MetPt *src[4] = {&T.C[id], &T.F1[id], &T.F2[id], &T.K[id]};
        MetPtF *dst[4] = {&T.Cf[id], &T.F1f[id], &T.F2f[id], &T.Kf[id]};
        for (int q = 0; q < 4; ++q) {
            const MetPt &m = *src[q];
            *dst[q] = MetPtF{(float)m.al,  (float)m.b1,  (float)m.g11, (float)m.g13, (float)m.g22, (float)m.g33,
                             (float)m.i11, (float)m.i13, (float)m.i22, (float)m.i33, (float)m.sg,  (float)m.isg};
        }
        MetDerF df;
        for (int d = 0; d < 2; ++d) {
            df.dal[d] = (float)dv.dal[d];
            df.db1[d] = (float)dv.db1[d];
            df.dg11[d] = (float)dv.dg11[d];
            df.dg13[d] = (float)dv.dg13[d];
            df.dg22[d] = (float)dv.dg22[d];
            df.dg33[d] = (float)dv.dg33[d];
        }
        T.dCf[id] = df;
    }
    if (j == 0) {
        T.floors[2 * i] = rho_floor * pow(exp(xc), rho_pow);
        T.floors[2 * i + 1] = p_floor * pow(exp(xc), p_pow);
    }
}

void launch_metric_tables(const Geom &g, double spin, const MetTables &T, double rho_floor, double rho_pow,
                          double p_floor, double p_pow, cudaStream_t s)
{
    dim3 blk(128, 1, 1);
    dim3 grd((unsigned)((g.np[0] + 127) / 128), (unsigned)g.np[1], 1);
    k_metric_tables<<<grd, blk, 0, s>>>(g, spin, T, rho_floor, rho_pow, p_floor, p_pow);
}

}  // namespace echo
