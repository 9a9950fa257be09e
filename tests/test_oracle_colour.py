"""Pins of the colour-transformed data term (Eq. 2, T_i applied to camera i's
rendering): identity transforms reduce it to the plain masked L1 term; the loss is
piecewise linear in T and in R, so central differences (steps that flip no sign) give
its gradients exactly."""
import numpy as np

import oracle


def _data(seed=0, N=2, H=6, W=5):
    rng = np.random.default_rng(seed)
    R = rng.uniform(0, 1, (N, H, W, 3)).astype(np.float32)
    O = rng.uniform(0, 1, (N, H, W, 3)).astype(np.float32)
    M = (rng.uniform(0, 1, (N, H, W)) > 0.3).astype(np.uint8)
    T = (np.eye(3)[None] + rng.normal(0, 0.1, (N, 3, 3))).reshape(N, 9).astype(np.float32)
    return R, O, M, T


def test_identity_transform_is_the_plain_loss():
    R, O, M, _ = _data()
    T = np.tile(np.eye(3).reshape(9), (R.shape[0], 1)).astype(np.float32)
    L, A, _ = oracle.loss_ct(R, O, M, T)
    L0, A0 = oracle.loss(R, O, M)
    assert abs(L - L0) <= 1e-12 * abs(L0) and np.allclose(A, A0, rtol=0, atol=1e-15)


def test_transform_and_render_gradients_are_exact_differences():
    R, O, M, T = _data(1)
    L, A, dT = oracle.loss_ct(R, O, M, T)
    h = 1e-4
    for n, k in [(0, 0), (0, 4), (1, 2), (1, 7), (0, 8)]:
        Tp, Tm = T.astype(np.float64).copy(), T.astype(np.float64).copy()
        Tp[n, k] += h
        Tm[n, k] -= h
        fd = (oracle.loss_ct(R, O, M, Tp.astype(np.float32))[0] -
              oracle.loss_ct(R, O, M, Tm.astype(np.float32))[0]) / (float(np.float32(Tp[n, k])) -
                                                                       float(np.float32(Tm[n, k])))
        assert abs(fd - dT[n, k]) <= 2e-3 * max(abs(dT[n, k]), 1e-3), (n, k, fd, dT[n, k])
    for idx in [(0, 1, 1, 0), (1, 3, 2, 2), (0, 5, 4, 1)]:
        Rp, Rm = R.astype(np.float64).copy(), R.astype(np.float64).copy()
        Rp[idx] += h
        Rm[idx] -= h
        fd = (oracle.loss_ct(Rp.astype(np.float32), O, M, T)[0] -
              oracle.loss_ct(Rm.astype(np.float32), O, M, T)[0]) / (float(np.float32(Rp[idx])) -
                                                                       float(np.float32(Rm[idx])))
        assert abs(fd - A[idx]) <= 2e-3 * max(abs(A[idx]), 1e-4), (idx, fd, A[idx])


def test_colour_map_upsampling_and_its_adjoint():
    """V_low enters every texel of its 64 x 64 block (nearest neighbour); the adjoint
    is the exact transpose: <up(a), b> = <a, blocksum(b)>."""
    rng = np.random.default_rng(2)
    lo = rng.normal(size=(8, 8, 3))
    hi = rng.normal(size=(512, 512, 3))
    V = oracle.colour_map(lo, hi)
    assert np.allclose(V[130, 70] - hi[130, 70], lo[2, 1]) and np.allclose(V[511, 0] - hi[511, 0], lo[7, 0])
    b = rng.normal(size=(512, 512, 3))
    lhs = ((V - hi) * b).sum()
    rhs = (lo * oracle.colour_map_bwd(b, lo.shape)).sum()
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
