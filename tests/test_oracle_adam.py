"""Pins of the oracle's Adam step (Kingma & Ba, ICLR 2015, Algorithm 1), which the GPU update
is checked against.

What pins it: from zero moments the first bias-corrected moments are g and g^2, so the step is
lr g / (|g| + eps); under a constant gradient the bias-corrected moments stay exactly g and g^2
at every step, so t steps move p by t lr g / (|g| + eps) (a missing or wrong bias correction, or
swapped betas, breaks this from the second step on); a zero gradient on zero moments leaves p
where it is; with eps = 0 the step is invariant to scaling the gradient by c > 0."""
import numpy as np

import oracle


def _g(seed=0, n=257):
    g = np.random.default_rng(seed).normal(size=n) * np.logspace(-4, 1, n)
    g[::17] = 0.0
    return g


def test_first_step_is_lr_g_over_abs_g_plus_eps():
    g = _g()
    p = np.linspace(-1.0, 1.0, g.size)
    z = np.zeros_like(g)
    p1, m1, v1 = oracle.adam(p, g, z, z, 0.01, 1)
    np.testing.assert_allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-15, atol=0)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12, atol=0)


def test_constant_gradient_moves_p_linearly():
    g = _g(1)
    p0 = np.random.default_rng(2).normal(size=g.size)
    p, m, v = p0.copy(), np.zeros_like(g), np.zeros_like(g)
    lr = np.full(g.size, 3e-3)
    for t in range(1, 41):
        p, m, v = oracle.adam(p, g, m, v, lr, t)
        np.testing.assert_allclose(p, p0 - t * lr * g / (np.abs(g) + 1e-8), rtol=1e-10, atol=1e-14)


def test_zero_gradient_keeps_p():
    p = np.arange(5.0)
    z = np.zeros(5)
    p1, m1, v1 = oracle.adam(p, z, z, z, 0.1, 1)
    assert np.array_equal(p1, p) and not m1.any() and not v1.any()


def test_step_is_invariant_to_gradient_scale_without_eps():
    g = _g(3)
    g = g[g != 0.0]
    p = np.zeros_like(g)
    z = np.zeros_like(g)
    a, b = (p.copy(), z.copy(), z.copy()), (p.copy(), z.copy(), z.copy())
    for t in range(1, 6):
        a = oracle.adam(a[0], g, a[1], a[2], 0.01, t, eps=0.0)
        b = oracle.adam(b[0], 37.5 * g, b[1], b[2], 0.01, t, eps=0.0)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-12, atol=1e-15)
