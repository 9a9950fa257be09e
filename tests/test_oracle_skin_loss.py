"""Oracle pins: skinning G_v (Section 3, the 61-parameter hand: shape beta(10),
pose theta(45), root rotation phi(3), root translation tau(3)), its adjoint, and
the masked photometric loss D_c (Eq. 4) with its adjoint."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2107_05509_gb300 import inputs as I


@pytest.fixture(scope="module")
def hand():
    return I.make_hand(0)


def test_rodrigues_matches_library_rotation():
    rng = np.random.default_rng(0)
    for r in list(rng.normal(0, 1.0, (20, 3))) + [np.zeros(3), np.array([1e-5, -2e-5, 3e-6])]:
        assert np.abs(oracle.rodrigues(r) - Rotation.from_rotvec(r).as_matrix()).max() < 1e-12


def test_rodrigues_gradient_fd():
    rng = np.random.default_rng(1)
    for r in list(rng.normal(0, 1.0, (10, 3))) + [np.array([1e-4, 2e-4, -1e-4]), np.zeros(3)]:
        G = rng.normal(size=(3, 3))
        g = oracle.rodrigues_grad(r, G)
        fd = np.zeros(3)
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-6
            fd[k] = ((G * oracle.rodrigues(r + e)).sum() - (G * oracle.rodrigues(r - e)).sum()) / 2e-6
        assert np.abs(g - fd).max() < 1e-7 * max(1.0, np.abs(fd).max())


def _wsum(hand):
    # float32 skin weights sum to 1 only up to rounding; LBS scales by the sum
    return hand.weights.astype(np.float64).sum(1, keepdims=True)


def test_zero_params_give_template(hand):
    v = oracle.skin(hand, np.zeros(61))
    assert np.abs(v - _wsum(hand) * hand.v_template).max() < 1e-12


def test_root_only_is_rigid(hand):
    x = np.zeros(61)
    x[55:58] = (0.3, -0.2, 0.5)
    x[58:61] = (0.01, -0.02, 0.03)
    R = Rotation.from_rotvec(x[55:58]).as_matrix()
    J0 = hand.j_template[0].astype(np.float64)
    expect = _wsum(hand) * ((hand.v_template - J0) @ R.T + J0) + x[58:61]
    assert np.abs(oracle.skin(hand, x) - expect).max() < 1e-12


def test_shape_only_is_linear(hand):
    x = np.zeros(61)
    x[0:10] = np.random.default_rng(2).normal(0, 1, 10)
    expect = _wsum(hand) * (hand.v_template + hand.shapedirs.astype(np.float64) @ x[0:10])
    assert np.abs(oracle.skin(hand, x) - expect).max() < 1e-12


def test_single_joint_rotates_its_subtree_about_the_joint(hand):
    # rotating joint j (middle finger MCP) moves a vertex weighted fully to it
    # exactly by R about the joint; vertices weighted to other fingers stay put
    j = 7
    x = np.zeros(61)
    x[10 + 3 * (j - 1):10 + 3 * j] = (0.4, 0.0, 0.1)
    v = oracle.skin(hand, x)
    R = Rotation.from_rotvec(x[10 + 3 * (j - 1):10 + 3 * j]).as_matrix()
    Jj = hand.j_template[j].astype(np.float64)
    w = hand.weights.astype(np.float64)
    sub = w[:, 7:10].sum(1)
    pred = (w[:, 7:10].sum(1, keepdims=True) * ((hand.v_template - Jj) @ R.T + Jj)
            + (w.sum(1) - sub)[:, None] * hand.v_template)
    assert np.abs(v - pred).max() < 1e-12
    other = w[:, 1:4].sum(1) > 0.999
    assert np.abs(v[other] - hand.v_template[other]).max() < 1e-6


def test_skin_adjoint_fd(hand):
    rng = np.random.default_rng(3)
    x = I.gt_params(1000).astype(np.float64)
    x[58:61] = (0.01, 0.02, -0.01)
    x[55:58] = (0.2, -0.1, 0.3)
    dV = rng.normal(size=(hand.V, 3))
    g = oracle.skin_bwd(hand, x, dV)
    fd = np.zeros(61)
    for k in range(61):
        e = np.zeros(61)
        e[k] = 1e-6
        fd[k] = ((dV * oracle.skin(hand, x + e)).sum() - (dV * oracle.skin(hand, x - e)).sum()) / 2e-6
    assert np.abs(g - fd).max() < 1e-6 * np.abs(fd).max()
    # translation gradient is exactly the sum of the vertex gradients
    assert np.array_equal(g[58:61], dV.sum(0))


def test_skin_adjoint_at_zero_pose(hand):
    rng = np.random.default_rng(4)
    dV = rng.normal(size=(hand.V, 3))
    x = np.zeros(61)
    g = oracle.skin_bwd(hand, x, dV)
    fd = np.zeros(61)
    for k in range(61):
        e = np.zeros(61)
        e[k] = 1e-6
        fd[k] = ((dV * oracle.skin(hand, x + e)).sum() - (dV * oracle.skin(hand, x - e)).sum()) / 2e-6
    assert np.abs(g - fd).max() < 1e-6 * np.abs(fd).max()


def test_loss_properties():
    rng = np.random.default_rng(5)
    R = rng.random((2, 6, 5, 3)).astype(np.float32)
    O = rng.random((2, 6, 5, 3)).astype(np.float32)
    M = (rng.random((2, 6, 5)) < 0.6).astype(np.uint8)
    # O == R: zero loss and zero adjoint (sign(0) = 0)
    L, A = oracle.loss(R, R, M)
    assert L == 0.0 and not A.any()
    # empty mask
    L, A = oracle.loss(R, O, np.zeros_like(M))
    assert L == 0.0 and not A.any()
    # closed form with a full mask: mean absolute difference over pixel-channels
    L, A = oracle.loss(R, O, np.ones_like(M))
    assert abs(L - np.abs(R.astype(np.float64) - O).mean()) < 1e-15
    # adjoint = finite difference of the loss (away from the kinks)
    L, A = oracle.loss(R, O, M)
    Rd = R.astype(np.float64)
    for idx in [(0, 1, 2, 0), (1, 5, 4, 2), (0, 0, 0, 1)]:
        e = np.zeros_like(Rd)
        e[idx] = 1e-7
        fd = (oracle.loss(Rd + e, O, M)[0] - oracle.loss(Rd - e, O, M)[0]) / 2e-7
        assert abs(fd - A[idx]) < 1e-9
    # masked-out pixels carry no adjoint; epsilon_b = 255 L in 0-255 levels
    assert not A[M == 0].any()


def test_joint_locations_and_their_adjoint():
    """G_J: at zero parameters the joints are the rest joints; a root translation moves
    every joint by it; the joint adjoint of skin_bwd matches central differences of the
    joint locations (all 61 parameters, a random upstream gradient)."""
    h = I.make_hand(0)
    x0 = np.zeros(61)
    assert np.allclose(oracle.skin_joints(h, x0), h.j_template.astype(np.float64))
    xt = x0.copy()
    xt[58:61] = (0.01, -0.02, 0.03)
    assert np.allclose(oracle.skin_joints(h, xt) - oracle.skin_joints(h, x0), xt[58:61])
    rng = np.random.default_rng(3)
    x = I.perturb_params(I.gt_params(5), 5).astype(np.float64)
    dJ = rng.normal(size=(h.j_template.shape[0], 3))
    g = oracle.skin_bwd(h, x, np.zeros((h.V, 3)), dJ)
    eps = 1e-6
    fd = np.zeros(61)
    for k in range(61):
        xp, xm = x.copy(), x.copy()
        xp[k] += eps
        xm[k] -= eps
        fd[k] = ((oracle.skin_joints(h, xp) - oracle.skin_joints(h, xm)) * dJ).sum() / (2 * eps)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-9 * np.abs(fd).max())


def test_joint_prior_smooth_l1():
    """f_2: quadratic inside gamma, linear outside, continuous with a continuous
    derivative at |x - y| = gamma; gradient = central differences."""
    gamma, lam = 0.005, 1e-3
    t = np.zeros((1, 3))
    for d, expect in ((0.002, 0.5 * 0.002 ** 2 / gamma), (0.008, 0.008 - 0.5 * gamma), (-0.008, 0.008 - 0.5 * gamma)):
        E, _ = oracle.joint_prior(np.array([[d, 0.0, 0.0]]), t, gamma, lam)
        assert abs(E - lam * expect) <= 1e-15
    a, _ = oracle.joint_prior(np.array([[gamma - 1e-9, 0, 0]]), t, gamma, 1.0)
    b, _ = oracle.joint_prior(np.array([[gamma + 1e-9, 0, 0]]), t, gamma, 1.0)
    assert abs(a - b) < 1e-8
    rng = np.random.default_rng(4)
    y = rng.normal(0, 0.006, (16, 3))
    x = rng.normal(0, 0.006, (16, 3))
    E, g = oracle.joint_prior(y, x, gamma, lam)
    for idx in [(0, 0), (3, 1), (9, 2), (15, 0)]:
        yp, ym = y.copy(), y.copy()
        yp[idx] += 1e-9
        ym[idx] -= 1e-9
        fd = (oracle.joint_prior(yp, x, gamma, lam)[0] - oracle.joint_prior(ym, x, gamma, lam)[0]) / 2e-9
        assert abs(fd - g[idx]) <= 1e-6 * max(abs(g[idx]), 1e-6)
