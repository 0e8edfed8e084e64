"""Pins of the FP64 network reference: gradients against central finite differences, and the
Adam step against its closed form on a quadratic."""

import numpy as np

from oracle import mlp_oracle as MO


def _net(rng, i=3, h1=5, h2=4, d=7):
    return [rng.normal(size=(h1, i)), rng.normal(size=h1), rng.normal(size=(h2, h1)) * 0.5,
            rng.normal(size=h2), rng.normal(size=(d, h2)), rng.normal(size=d)]


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    params = _net(rng)
    Z = rng.normal(size=(6, 3))
    T = rng.normal(size=(6, 7))
    mu, sd = Z.mean(0), Z.std(0) + 0.5
    _, grads = MO.loss_and_grads(params, Z, T, mu, sd)
    h = 1e-6
    for pi, p in enumerate(params):
        flat = p.reshape(-1)
        for idx in range(flat.size):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = MO.loss_and_grads(params, Z, T, mu, sd)
            flat[idx] = old - h
            lm, _ = MO.loss_and_grads(params, Z, T, mu, sd)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[pi].reshape(-1)[idx]) <= 1e-7 * max(1.0, abs(fd)), (pi, idx)


def test_output_layer_is_least_squares_fit_at_stationarity():
    # with hidden layers frozen, the output-layer gradient vanishes exactly at the least-squares
    # solution of H2 [W3 b3]^T = T
    rng = np.random.default_rng(1)
    params = _net(rng)
    Z = rng.normal(size=(20, 3))
    T = rng.normal(size=(20, 7))
    mu, sd = np.zeros(3), np.ones(3)
    _, (_, _, H2) = MO.forward(params, Z, mu, sd)
    A = np.hstack([H2, np.ones((20, 1))])
    sol = np.linalg.lstsq(A, T, rcond=None)[0]
    params[4], params[5] = sol[:-1].T.copy(), sol[-1].copy()
    _, grads = MO.loss_and_grads(params, Z, T, mu, sd)
    assert np.abs(grads[4]).max() < 1e-12 and np.abs(grads[5]).max() < 1e-12


def test_adam_first_step_moves_by_lr_times_sign():
    # after one step from zero moments the bias-corrected update is lr * g / (|g| + eps)
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    m, v = [np.zeros(3)], [np.zeros(3)]
    out = MO.adam_step(p, g, m, v, 1, lr=0.1)
    assert np.allclose(out[0], p[0] - 0.1 * g[0] / (np.abs(g[0]) + 1e-8), rtol=0, atol=1e-15)
