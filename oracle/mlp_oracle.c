/*
 * mlp_oracle.c -- plain FP64 CPU reference of the c2p-guess network and of
 * its training step.  TEST INFRASTRUCTURE ONLY (same rules as
 * echo_oracle.c): used by tests to check the GPU forward pass, the batch
 * gradient and the Adam update.
 *
 * Network: x (9 features) -> standardise -> h1 = tanh(W1 x + b1) (64)
 *          -> h2 = tanh(W2 h1 + b2) (64) -> o = W3 h2 + b3 (3).
 * Parameter vector layout (4995 values): W1 (64x9, row-major), b1 (64),
 * W2 (64x64), b2 (64), W3 (3x64), b3 (3); then the normalisation block:
 * feature mean (9), feature std (9), target mean (3), target std (3).
 *
 * Targets y (3 per sample): log W, log(p / D), log(Z / D) of the converged
 * inversion.  Outputs 0 and 1 regress the standardised log W and log(p/D);
 * output 2 regresses, with the first two held fixed (no gradient flows
 * through the target), the standardised log10 relative error of the guess
 *   Z0/D = W (1 + G/(G-1) (p/D) W)
 * that outputs 0 and 1 imply.  Loss per sample:
 *   (o0 - t0)^2 + (o1 - t1)^2 + w2 (o2 - t2)^2, averaged over the batch.
 * Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *   theta -= lr m/(1-b1^t) / (sqrt(v/(1-b2^t)) + eps).
 */
#include <math.h>
#include <string.h>

#define NI 9
#define NH 64
#define NO 3
#define OW1 0
#define OB1 (OW1 + NH * NI)
#define OW2 (OB1 + NH)
#define OB2 (OW2 + NH * NH)
#define OW3 (OB2 + NH)
#define OB3 (OW3 + NO * NH)
#define NPAR (OB3 + NO)
#define ONORM NPAR

int oracle_mlp_nparam(void) { return NPAR; }

/* Forward pass of one sample; h1, h2 (may be NULL) receive the hidden
 * activations; out receives the raw (standardised) outputs. */
static void forward(const double *P, const double *x, double *xs, double *h1, double *h2, double *out)
{
    const double *mu = P + ONORM, *sd = P + ONORM + NI;
    double a1[NH], a2[NH];
    for (int i = 0; i < NI; ++i)
        xs[i] = (x[i] - mu[i]) / sd[i];
    for (int j = 0; j < NH; ++j) {
        double s = P[OB1 + j];
        for (int i = 0; i < NI; ++i)
            s += P[OW1 + j * NI + i] * xs[i];
        a1[j] = tanh(s);
    }
    for (int k = 0; k < NH; ++k) {
        double s = P[OB2 + k];
        for (int j = 0; j < NH; ++j)
            s += P[OW2 + k * NH + j] * a1[j];
        a2[k] = tanh(s);
    }
    for (int o = 0; o < NO; ++o) {
        double s = P[OB3 + o];
        for (int k = 0; k < NH; ++k)
            s += P[OW3 + o * NH + k] * a2[k];
        out[o] = s;
    }
    if (h1)
        memcpy(h1, a1, sizeof(a1));
    if (h2)
        memcpy(h2, a2, sizeof(a2));
}

/* Standardised targets of one sample given the raw outputs. */
static void targets(const double *P, const double *y, const double *out, double gr, double *t)
{
    const double *ym = P + ONORM + 2 * NI, *ys = P + ONORM + 2 * NI + NO;
    t[0] = (y[0] - ym[0]) / ys[0];
    t[1] = (y[1] - ym[1]) / ys[1];
    double W = exp(out[0] * ys[0] + ym[0]);
    double pD = exp(out[1] * ys[1] + ym[1]);
    double z0 = W * (1.0 + gr * pD * W);
    double zs = exp(y[2]);
    double err = log10(fabs(z0 - zs) / zs + 1e-16);
    t[2] = (err - ym[2]) / ys[2];
}

/* Raw outputs of n samples (x: n x 9) into out (n x 3). */
void oracle_mlp_forward(const double *P, const double *x, int n, double *out)
{
    for (int s = 0; s < n; ++s) {
        double xs[NI];
        forward(P, x + (size_t)s * NI, xs, NULL, NULL, out + (size_t)s * NO);
    }
}

/* Standardised targets (n x 3) of n samples at parameters P. */
void oracle_mlp_targets(const double *P, const double *x, const double *y, int n, double gamma, double *t)
{
    double gr = gamma / (gamma - 1.0);
    for (int s = 0; s < n; ++s) {
        double xs[NI], o[NO];
        forward(P, x + (size_t)s * NI, xs, NULL, NULL, o);
        targets(P, y + (size_t)s * NO, o, gr, t + (size_t)s * NO);
    }
}

/* Mean loss of n samples and its gradient with respect to the NPAR
 * parameters (grad may be NULL).  t_fixed (may be NULL): standardised
 * targets to use instead of those implied by P (for derivative checks). */
double oracle_mlp_loss_grad(const double *P, const double *x, const double *y, int n, double gamma,
                            double w2, double *grad, const double *t_fixed)
{
    double gr = gamma / (gamma - 1.0);
    double loss = 0.0;
    if (grad)
        memset(grad, 0, NPAR * sizeof(double));
    for (int s = 0; s < n; ++s) {
        double xs[NI], h1[NH], h2[NH], o[NO], t[NO];
        forward(P, x + (size_t)s * NI, xs, h1, h2, o);
        if (t_fixed)
            memcpy(t, t_fixed + (size_t)s * NO, sizeof(t));
        else
            targets(P, y + (size_t)s * NO, o, gr, t);
        double wgt[NO] = {1.0, 1.0, w2};
        double d3[NO];
        for (int q = 0; q < NO; ++q) {
            double r = o[q] - t[q];
            loss += wgt[q] * r * r / n;
            d3[q] = 2.0 * wgt[q] * r / n;
        }
        if (!grad)
            continue;
        double d2[NH], d1[NH];
        for (int q = 0; q < NO; ++q) {
            grad[OB3 + q] += d3[q];
            for (int k = 0; k < NH; ++k)
                grad[OW3 + q * NH + k] += d3[q] * h2[k];
        }
        for (int k = 0; k < NH; ++k) {
            double s2 = 0.0;
            for (int q = 0; q < NO; ++q)
                s2 += P[OW3 + q * NH + k] * d3[q];
            d2[k] = s2 * (1.0 - h2[k] * h2[k]);
            grad[OB2 + k] += d2[k];
            for (int j = 0; j < NH; ++j)
                grad[OW2 + k * NH + j] += d2[k] * h1[j];
        }
        for (int j = 0; j < NH; ++j) {
            double s1 = 0.0;
            for (int k = 0; k < NH; ++k)
                s1 += P[OW2 + k * NH + j] * d2[k];
            d1[j] = s1 * (1.0 - h1[j] * h1[j]);
            grad[OB1 + j] += d1[j];
            for (int i = 0; i < NI; ++i)
                grad[OW1 + j * NI + i] += d1[j] * xs[i];
        }
    }
    return loss;
}

/* One Adam update of the NPAR parameters in place (t = 1, 2, ...). */
void oracle_mlp_adam(double *P, double *m, double *v, const double *g, int t, double lr, double b1, double b2,
                     double eps)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int i = 0; i < NPAR; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        P[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
