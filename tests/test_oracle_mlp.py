"""Pins of the oracle's c2p-guess network: the analytic gradient against
central finite differences (targets held fixed, as in training) and Adam's
closed-form first step."""
import numpy as np


def random_net(rng, scale=0.3):
    p = rng.normal(0.0, scale, size=4995 + 24)
    p[4995:4995 + 9] = rng.normal(0, 1, 9)          # feature mean
    p[4995 + 9:4995 + 18] = rng.uniform(0.5, 2, 9)  # feature std
    p[4995 + 18:4995 + 21] = rng.normal(0, 0.5, 3)  # target mean
    p[4995 + 21:4995 + 24] = rng.uniform(0.5, 2, 3)  # target std
    return p


def random_data(rng, n):
    x = rng.normal(0, 1, size=(n, 9))
    W = rng.uniform(1.0, 1.5, n)
    pD = rng.uniform(0.1, 2.0, n)
    z = W * (1 + 4.0 * pD * W)
    y = np.stack([np.log(W), np.log(pD), np.log(z)], axis=1)
    return x, y


def test_gradient_matches_finite_differences(orc):
    rng = np.random.default_rng(0)
    P = random_net(rng)
    x, y = random_data(rng, 16)
    t = orc.mlp_targets(P, x, y)
    loss, g = orc.mlp_loss_grad(P, x, y, w2=0.5, t_fixed=t)
    idx = rng.choice(4995, size=120, replace=False)
    idx = np.concatenate([idx, [0, 575, 576, 639, 640, 4735, 4736, 4799, 4800, 4991, 4992, 4994]])
    h = 1e-6
    for i in idx:
        Pp = P.copy()
        Pm = P.copy()
        Pp[i] += h
        Pm[i] -= h
        lp, _ = orc.mlp_loss_grad(Pp, x, y, w2=0.5, t_fixed=t)
        lm, _ = orc.mlp_loss_grad(Pm, x, y, w2=0.5, t_fixed=t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_target_of_third_output_is_the_guess_error(orc):
    """Output 2's target is log10 of the relative error of the guess
    Z0/D = W (1 + G/(G-1) (p/D) W) implied by outputs 0 and 1."""
    rng = np.random.default_rng(1)
    P = random_net(rng)
    x, y = random_data(rng, 8)
    o = orc.mlp_forward(P, x)
    t = orc.mlp_targets(P, x, y)
    ym, ys = P[4995 + 18:4995 + 21], P[4995 + 21:4995 + 24]
    W = np.exp(o[:, 0] * ys[0] + ym[0])
    pD = np.exp(o[:, 1] * ys[1] + ym[1])
    z0 = W * (1 + 4.0 * pD * W)
    err = np.log10(np.abs(z0 - np.exp(y[:, 2])) / np.exp(y[:, 2]) + 1e-16)
    assert np.allclose(t[:, 2], (err - ym[2]) / ys[2], rtol=1e-12, atol=1e-12)
    assert np.allclose(t[:, 0], (y[:, 0] - ym[0]) / ys[0], rtol=1e-14, atol=1e-14)


def test_adam_first_step_is_signed_learning_rate(orc):
    """With zero moments, the bias-corrected first Adam step is
    -lr g / (|g| + eps) per parameter."""
    rng = np.random.default_rng(2)
    P = rng.normal(size=4995)
    P0 = P.copy()
    g = rng.normal(size=4995)
    m = np.zeros(4995)
    v = np.zeros(4995)
    orc.mlp_adam(P, m, v, g, 1, lr=1e-2, eps=1e-8)
    assert np.allclose(P - P0, -1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_adam_steps_under_constant_gradient(orc):
    """With a constant gradient the bias-corrected moments are exactly g and
    g^2 at every t (m_t = (1 - b1^t) g, v_t = (1 - b2^t) g^2), so each of the
    first steps is again -lr g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    P = rng.normal(size=4995)
    g = rng.normal(size=4995)
    m = np.zeros(4995)
    v = np.zeros(4995)
    for t in range(1, 6):
        P0 = P.copy()
        orc.mlp_adam(P, m, v, g, t, lr=1e-2, eps=1e-8)
        assert np.allclose(P - P0, -1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-15), t


def test_loss_is_the_weighted_mean_square(orc):
    """The loss is the mean over samples of the squared standardised
    residuals, the third output's weighted by w2 (the first two by 1)."""
    rng = np.random.default_rng(4)
    P = random_net(rng)
    x, y = random_data(rng, 12)
    o = orc.mlp_forward(P, x)
    t = orc.mlp_targets(P, x, y)
    for w2 in (0.5, 0.1):
        loss, _ = orc.mlp_loss_grad(P, x, y, w2=w2)
        want = np.mean(np.sum((o - t) ** 2 * np.array([1.0, 1.0, w2]), axis=1))
        assert abs(loss - want) <= 1e-13 * want


def test_forward_is_the_layered_network(orc):
    """The forward pass is the 9 -> 64 -> 64 -> 3 tanh network of the
    parameter layout W1 (64x9) | b1 | W2 (64x64) | b2 | W3 (3x64) | b3, on
    features standardised by the stored mean and std (numpy products)."""
    rng = np.random.default_rng(5)
    P = random_net(rng)
    x, _ = random_data(rng, 10)
    o1 = 64 * 9
    W1, b1 = P[:o1].reshape(64, 9), P[o1:o1 + 64]
    o2 = o1 + 64
    W2, b2 = P[o2:o2 + 4096].reshape(64, 64), P[o2 + 4096:o2 + 4160]
    o3 = o2 + 4160
    W3, b3 = P[o3:o3 + 192].reshape(3, 64), P[o3 + 192:o3 + 195]
    mu, sd = P[4995:4995 + 9], P[4995 + 9:4995 + 18]
    h1 = np.tanh((x - mu) / sd @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    assert np.allclose(orc.mlp_forward(P, x), h2 @ W3.T + b3, rtol=1e-12, atol=1e-13)
