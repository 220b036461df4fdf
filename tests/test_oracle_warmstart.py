"""Pins for the warm-start oracle: backpropagation against central finite differences, Adam
against its closed-form special cases, and training on a problem with a known solution."""
import numpy as np

import synth
from oracle import warmstart as ws


def _tiny(seed=0):
    p = synth.warmstart_params(5, 7, 6, 3, seed=seed)
    rng = np.random.default_rng(seed)
    for i in (1, 3, 5):
        p[i] = 0.1 * rng.standard_normal(p[i].shape)
    U = rng.standard_normal((4, 5))
    T = rng.standard_normal((4, 3))
    return p, U, T


def test_backprop_matches_finite_differences():
    p, U, T = _tiny()
    g = ws.grad(p, U, T)
    h = 1e-6
    for i, w in enumerate(p):
        fd = np.zeros_like(w)
        it = np.nditer(w, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = w[idx]
            w[idx] = old + h
            lp = ws.loss(p, U, T)
            w[idx] = old - h
            lm = ws.loss(p, U, T)
            w[idx] = old
            fd[idx] = (lp - lm) / (2 * h)
        assert np.allclose(g[i], fd, rtol=1e-6, atol=1e-9), i


def test_adam_first_step_is_lr_times_sign():
    """After bias correction, step 1 has mhat = g and vhat = g^2 for any beta1, beta2."""
    w = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    ws.adam_step(w, g, ws.init_state(w), 1, lr=0.01, beta1=0.7, beta2=0.95, eps=0.0)
    assert np.allclose(w[0], [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01], rtol=0, atol=1e-15)


def test_adam_without_momentum_is_sign_descent():
    w = [np.array([0.3, -0.2])]
    st = ws.init_state(w)
    for t in range(1, 5):
        g = [np.array([2.0 * t, -0.5])]
        ws.adam_step(w, g, st, t, lr=0.1, beta1=0.0, beta2=0.0, eps=0.0)
    assert np.allclose(w[0], [0.3 - 0.4, -0.2 + 0.4], atol=1e-14)


def test_training_recovers_a_linear_map():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3, 5)) * 0.5
    U = rng.standard_normal((256, 5))
    T = U @ A.T
    p = synth.warmstart_params(5, 32, 32, 3, seed=1)
    st = ws.init_state(p)
    l0 = ws.loss(p, U, T)
    for t in range(1, 801):
        ws.adam_step(p, ws.grad(p, U, T), st, t, lr=3e-3)
    assert ws.loss(p, U, T) < 1e-3 * l0
