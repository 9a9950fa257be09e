"""Oracle pins: the Adam step (Section 3.3 optimises the parameters with Adam,
Kingma and Ba's update) and epsilon_v, the mean vertex error (Section 4.1).

Each pin is a consequence of the update that does not re-type it: the first step's
closed form, a constant gradient's closed form at every step, the moments as the
explicit weighted sums the recursions unroll to, sign symmetry, scale invariance,
linearity in the step size and the per-entry step-size pattern."""
import numpy as np
import pytest

import oracle

B1, B2, EPS = 0.9, 0.999, 1e-8


def _run(p0, grads, lr, eps=EPS, lr_scale=None):
    p, m, v = np.asarray(p0, np.float64), np.zeros(len(p0)), np.zeros(len(p0))
    out = []
    for t, g in enumerate(grads, start=1):
        p, m, v = oracle.adam_step(p, g, m, v, t, lr, B1, B2, eps, lr_scale=lr_scale)
        out.append((p, m, v))
    return out


def test_first_step_is_lr_times_sign():
    rng = np.random.default_rng(0)
    p0 = rng.normal(size=50)
    g = rng.normal(size=50) * np.logspace(-3, 3, 50)
    (p1, m1, v1), = _run(p0, [g], lr=0.01)
    # m_hat = g and v_hat = g^2 after one step: the move is lr g / (|g| + eps)
    assert np.allclose(p1 - p0, -0.01 * g / (np.abs(g) + EPS), rtol=1e-12, atol=0)
    # |move| = lr up to eps / |g|
    assert np.all(np.abs(np.abs(p1 - p0) - 0.01) <= 0.01 * 1.01 * EPS / np.abs(g))
    assert np.allclose(m1, (1 - B1) * g, rtol=1e-15)
    assert np.allclose(v1, (1 - B2) * g * g, rtol=1e-15)


def test_constant_gradient_moves_lr_per_step():
    # with g fixed, m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so the bias
    # corrections give m_hat = g and v_hat = g^2 at every step
    rng = np.random.default_rng(1)
    p0 = rng.normal(size=20)
    g = rng.normal(size=20)
    steps = _run(p0, [g] * 12, lr=0.003)
    for t, (p, m, v) in enumerate(steps, start=1):
        assert np.allclose(p, p0 - t * 0.003 * g / (np.abs(g) + EPS), rtol=0, atol=1e-14)
        assert np.allclose(m, (1 - B1 ** t) * g, rtol=1e-13)
        assert np.allclose(v, (1 - B2 ** t) * g * g, rtol=1e-13)


@pytest.mark.parametrize("t_max", [1, 2, 3, 7])
def test_moments_are_the_unrolled_weighted_sums(t_max):
    # m_t = (1 - b1) sum_i b1^(t-i) g_i; v_t likewise with g_i^2 and b2; the step at t
    # uses them divided by the sums of their weights, 1 - b^t
    rng = np.random.default_rng(2 + t_max)
    grads = [rng.normal(size=8) for _ in range(t_max)]
    p0 = rng.normal(size=8)
    steps = _run(p0, grads, lr=0.05)
    p_prev = p0
    for t in range(1, t_max + 1):
        w1 = np.array([(1 - B1) * B1 ** (t - i) for i in range(1, t + 1)])
        w2 = np.array([(1 - B2) * B2 ** (t - i) for i in range(1, t + 1)])
        G = np.stack(grads[:t])
        m_t, v_t = w1 @ G, w2 @ (G * G)
        p, m, v = steps[t - 1]
        assert np.allclose(m, m_t, rtol=1e-13, atol=0)
        assert np.allclose(v, v_t, rtol=1e-13, atol=0)
        assert np.isclose(w1.sum(), 1 - B1 ** t) and np.isclose(w2.sum(), 1 - B2 ** t)
        step = (m_t / w1.sum()) / (np.sqrt(v_t / w2.sum()) + EPS)
        assert np.allclose(p, p_prev - 0.05 * step, rtol=0, atol=1e-14)
        p_prev = p


def test_sign_symmetry_scale_invariance_and_zero_gradient():
    rng = np.random.default_rng(3)
    p0 = rng.normal(size=30)
    grads = [rng.normal(size=30) for _ in range(5)]
    base = _run(p0, grads, lr=0.02, eps=0.0)[-1][0]
    flipped = _run(p0, [-g for g in grads], lr=0.02, eps=0.0)[-1][0]
    scaled = _run(p0, [1e4 * g for g in grads], lr=0.02, eps=0.0)[-1][0]
    assert np.allclose(flipped - p0, -(base - p0), rtol=1e-12)
    assert np.allclose(scaled, base, rtol=0, atol=1e-12)
    still = _run(p0, [np.zeros(30)] * 3, lr=0.02)[-1][0]
    assert np.array_equal(still, p0)


def test_per_entry_step_sizes_repeat_and_scale_linearly():
    rng = np.random.default_rng(4)
    n, k = 61 * 3, 61
    scale = rng.uniform(0.0, 2.0, k)
    scale[::7] = 0.0                          # entries a phase keeps fixed
    p0 = rng.normal(size=n)
    grads = [rng.normal(size=n) for _ in range(4)]
    unit = _run(p0, grads, lr=1.0)
    scaled = _run(p0, grads, lr=0.5, lr_scale=scale)
    # the moments do not depend on the step size; the move of each step is lr * s_i
    # times the move with lr = 1 (both runs see the same m, v at every step)
    prev_u, prev_s = p0, p0
    for (pu, mu, vu), (ps, ms, vs) in zip(unit, scaled):
        assert np.array_equal(mu, ms) and np.array_equal(vu, vs)
        s_i = 0.5 * np.tile(scale, n // k)
        assert np.allclose(ps - prev_s, s_i * (pu - prev_u), rtol=1e-12, atol=1e-15)
        prev_u, prev_s = pu, ps
    fixed = np.tile(scale, n // k) == 0.0
    assert np.array_equal(scaled[-1][0][fixed], p0[fixed])


def test_step_count_starts_at_one():
    with pytest.raises(ValueError):
        oracle.adam_step(np.zeros(2), np.ones(2), np.zeros(2), np.zeros(2), 0, 0.1)


def test_vertex_error_closed_forms():
    rng = np.random.default_rng(5)
    a = rng.normal(size=(778, 3))
    # a rigid translation by (3, 4, 0) mm moves every vertex by exactly 5 mm
    assert abs(oracle.vertex_error_mm(a + np.array([3e-3, 4e-3, 0.0]), a) - 5.0) < 1e-9
    # one vertex moved by 2 cm: the mean is 20 mm / V
    b = a.copy()
    b[17] += np.array([0.0, 0.0, 0.02])
    assert abs(oracle.vertex_error_mm(b, a) - 20.0 / 778) < 1e-9
    assert oracle.vertex_error_mm(a, a) == 0.0
    assert oracle.vertex_error_mm(a, b) == oracle.vertex_error_mm(b, a)
