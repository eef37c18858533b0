"""Pins of the oracle's FP64 MLP (8 -> 32 ReLU -> 1 sigmoid, weighted BCE, Adam).

Gradients are checked against central finite differences of the oracle's own
loss and against the closed form of a one-sample network; Adam against its
defining update on the first step.
"""
import numpy as np

import oracle

IN, H = oracle.MLP_IN, oracle.MLP_H


def _params(rng):
    return (rng.standard_normal((H, IN)) * 0.4, rng.standard_normal(H) * 0.1,
            rng.standard_normal(H) * 0.3, 0.05)


def test_gradients_match_finite_differences(oracle_lib):
    rng = np.random.default_rng(7)
    X = rng.standard_normal((40, IN))
    y = (rng.uniform(size=40) < 0.3).astype(float)
    W1, b1, w2, b2 = _params(rng)
    L, gW1, gb1, gw2, gb2 = oracle.mlp_loss_grad(X, y, 3.0, W1, b1, w2, b2)
    eps = 1e-6

    def loss(W1_, b1_, w2_, b2_):
        return oracle.mlp_loss_grad(X, y, 3.0, W1_, b1_, w2_, b2_)[0]

    for (j, k) in [(0, 0), (5, 3), (31, 7), (12, 1)]:
        Wp = W1.copy(); Wp[j, k] += eps
        Wm = W1.copy(); Wm[j, k] -= eps
        fd = (loss(Wp, b1, w2, b2) - loss(Wm, b1, w2, b2)) / (2 * eps)
        assert abs(fd - gW1[j, k]) < 1e-7
    for j in [0, 9, 31]:
        bp = b1.copy(); bp[j] += eps
        bm = b1.copy(); bm[j] -= eps
        assert abs((loss(W1, bp, w2, b2) - loss(W1, bm, w2, b2)) / (2 * eps) - gb1[j]) < 1e-7
        wp = w2.copy(); wp[j] += eps
        wm = w2.copy(); wm[j] -= eps
        assert abs((loss(W1, b1, wp, b2) - loss(W1, b1, wm, b2)) / (2 * eps) - gw2[j]) < 1e-7
    assert abs((loss(W1, b1, w2, b2 + eps) - loss(W1, b1, w2, b2 - eps)) / (2 * eps) - gb2) < 1e-7


def test_one_sample_closed_form(oracle_lib):
    # one hidden unit active: z = w2_0 * (W1_0 . x + b1_0) + b2, dL/dz = p - y
    X = np.zeros((1, IN)); X[0, 2] = 1.5
    W1 = np.zeros((H, IN)); W1[0, 2] = 2.0
    b1 = np.zeros(H); b1[0] = 0.5
    b1[1:] = -1.0                      # every other unit inactive
    w2 = np.zeros(H); w2[0] = 0.7
    b2 = -0.2
    z, p = oracle.mlp_forward(X, W1, b1, w2, b2)
    a = 2.0 * 1.5 + 0.5
    assert abs(z[0] - (0.7 * a - 0.2)) < 1e-15
    y = np.array([1.0])
    L, gW1, gb1, gw2, gb2 = oracle.mlp_loss_grad(X, y, 1.0, W1, b1, w2, b2)
    pz = 1 / (1 + np.exp(-z[0]))
    assert abs(L - (-np.log(pz))) < 1e-14
    assert abs(gb2 - (pz - 1)) < 1e-15
    assert abs(gw2[0] - (pz - 1) * a) < 1e-14
    assert abs(gb1[0] - (pz - 1) * 0.7) < 1e-15
    assert abs(gW1[0, 2] - (pz - 1) * 0.7 * 1.5) < 1e-14
    assert np.all(gW1[1:] == 0) and np.all(gb1[1:] == 0)


def test_adam_first_step(oracle_lib):
    w = np.array([1.0, -2.0, 0.5]); g = np.array([0.3, -1e-3, 0.0])
    mo = np.zeros(3); ve = np.zeros(3)
    oracle.adam(w, g, mo, ve, 1, 0.01)
    # first step: m_hat = g, v_hat = g^2, so w moves by lr * g / (|g| + eps)
    ref = np.array([1.0, -2.0, 0.5]) - 0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(w, ref, rtol=0, atol=1e-15)


def test_adam_later_steps(oracle_lib):
    """Steps t >= 2, where beta2 and both bias corrections matter.
    Constant gradient g: m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so the
    bias-corrected moments are g and g^2 at every t and each step moves w by
    lr g / (|g| + eps).  Gradient +1 then -1: m_2 = 0.9 * 0.1 - 0.1 = -0.01,
    m_hat = -0.01 / (1 - 0.81) = -1/19; v_2 = 0.999 * 0.001 + 0.001 = 0.001999,
    v_hat = 0.001999 / (1 - 0.998001) = 1; so step 2 moves w by +lr/19 / (1 + eps)."""
    lr, eps = 0.01, 1e-8
    w = np.array([1.0, -2.0]); g = np.array([0.3, -0.02])
    mo = np.zeros(2); ve = np.zeros(2)
    for t in range(1, 6):
        oracle.adam(w, g, mo, ve, t, lr)
    ref = np.array([1.0, -2.0]) - 5 * lr * g / (np.abs(g) + eps)
    assert np.allclose(w, ref, rtol=0, atol=1e-14)

    w = np.array([0.5]); mo = np.zeros(1); ve = np.zeros(1)
    oracle.adam(w, np.array([1.0]), mo, ve, 1, lr)
    assert abs(w[0] - (0.5 - lr / (1.0 + eps))) < 1e-15
    oracle.adam(w, np.array([-1.0]), mo, ve, 2, lr)
    assert abs(mo[0] + 0.01) < 1e-17 and abs(ve[0] - 0.001999) < 1e-17
    assert abs(w[0] - (0.5 - lr / (1.0 + eps) + lr / 19.0 / (1.0 + eps))) < 1e-15
