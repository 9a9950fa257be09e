"""Pins of the edge-term oracle (Eq. 4's D_e with Canny's detector) against facts
fixed outside it: Gaussian tap ratios, the slope of a linear ramp, the closed-form
gradient of a step edge and where non-maximum suppression leaves it (vertical and
both diagonal edges), connected components from a library labelling, the impulse
response and constant response of K, the adjointness of every convolution and its
transpose (both border rules), and finite differences of the loss in the image and
in the colour transforms with the selection held fixed."""
import math

import numpy as np
import pytest

from oracle import edges as E


def _rgb(g):
    """An RGB image whose channels are all g (its gray value is g times the sum of the
    luma weights)."""
    return np.repeat(np.asarray(g, np.float32)[..., None], 3, axis=-1)


def test_gauss_weights():
    for r, s in ((2, 1.0), (5, 5.0)):
        w = E.gauss_weights(r, s).astype(np.float64)
        assert len(w) == 2 * r + 1
        assert abs(w.sum() - 1.0) < 1e-6
        assert np.array_equal(w, w[::-1])
        for k in range(1, r + 1):
            assert abs(w[r + k] / w[r] - math.exp(-k * k / (2 * s * s))) < 1e-6


def test_ramp_gives_its_slope():
    H, W = 20, 24
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    alpha, beta = 0.01, -0.02
    g = (0.3 + alpha * x + beta * y)[None]
    c = E.canny(_rgb(g))
    lum = float(np.float32(0.299) + np.float32(0.587) + np.float32(0.114))
    inner = (slice(None), slice(4, H - 4), slice(4, W - 4))
    assert np.allclose(c["gx"][inner], alpha * lum, rtol=0, atol=2e-7)
    assert np.allclose(c["gy"][inner], beta * lum, rtol=0, atol=2e-7)


def test_vertical_step_closed_form_and_suppression():
    H, W, x0, cval = 16, 20, 10, 0.8
    g = np.zeros((1, H, W))
    g[..., x0:] = cval
    c = E.canny(_rgb(g))
    w = E.gauss_weights(2, 1.0).astype(np.float64)
    lum = float(np.float32(0.299) + np.float32(0.587) + np.float32(0.114))

    def wk(k):
        return w[k + 2] if -2 <= k <= 2 else 0.0

    for x in range(3, W - 3):
        ref = 0.5 * cval * lum * (wk(x0 - x - 1) + wk(x0 - x))
        assert abs(c["gx"][0, 8, x] - ref) < 1e-6, x
    assert (c["gy"][0, 1:-1] == 0).all()
    kept = c["kept"][0]
    cols = np.nonzero(kept.any(0))[0]
    assert set(cols) <= {x0 - 1, x0}, cols
    assert kept.any(1).all()    # every row keeps the edge


@pytest.mark.parametrize("sign", [1, -1])
def test_diagonal_steps_are_thinned_along_the_diagonal(sign):
    H = W = 24
    y, x = np.mgrid[0:H, 0:W]
    k0 = 24 if sign > 0 else 0
    g = np.where(x + sign * y >= k0, 0.9, 0.1)[None].astype(np.float64)
    c = E.canny(_rgb(g))
    kept = c["kept"][0]
    inner = np.zeros_like(kept)
    inner[4:-4, 4:-4] = True
    ky, kx = np.nonzero(kept & inner)
    assert len(ky) > 0
    # within one diagonal step of the edge line x + sign y = k0 - 1/2
    assert (np.abs(kx + sign * ky - (k0 - 0.5)) <= 1.5).all()
    # suppression along the diagonal keeps at most two pixels per row
    for row in range(4, H - 4):
        assert kept[row, 4:-4].sum() <= 2
    # the direction was quantised to the diagonal (not to x or y) on the line
    gx, gy = c["gx"][0][kept], c["gy"][0][kept]
    assert (np.sign(gx) == sign * np.sign(gy)).all() and (gx != 0).all()


def test_hysteresis_matches_connected_components():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(4)
    for trial in range(5):
        cand = rng.random((2, 30, 40)) < 0.35
        strong = cand & (rng.random(cand.shape) < 0.03)
        kept = E.hysteresis(cand, strong)
        for n in range(2):
            lab, _ = ndimage.label(cand[n], structure=np.ones((3, 3)))
            good = np.unique(lab[strong[n]])
            ref = cand[n] & np.isin(lab, good[good > 0])
            assert np.array_equal(kept[n], ref), trial


def test_blur_k_impulse_and_constant():
    k = E.gauss_weights(5, 5.0)
    img = np.zeros((1, 31, 33), np.float32)
    img[0, 15, 16] = 1.0
    out = E.blur_k(img)
    ref = np.zeros_like(out)
    ref[0, 10:21, 11:22] = (k[:, None] * k[None, :]).astype(np.float32)
    assert np.array_equal(out, ref)
    const = E.blur_k(np.full((1, 31, 33), 0.5, np.float32))
    assert np.allclose(const[0, 5:-5, 5:-5], 0.5, atol=3e-7)
    assert const[0, 0, 0] < 0.5 * 0.6   # zero padding outside the image


@pytest.mark.parametrize("border", ["clamp", "zero"])
@pytest.mark.parametrize("axis", [1, 2])
def test_convolution_transposes_are_adjoints(border, axis):
    rng = np.random.default_rng(5)
    x = rng.normal(size=(2, 9, 13)).astype(np.float32)
    y = rng.normal(size=(2, 9, 13))
    for w in (E.gauss_weights(2, 1.0), np.array(E.DERIV, np.float32), E.gauss_weights(5, 5.0)):
        lhs = float((E.conv1d(x, w, axis, border).astype(np.float64) * y).sum())
        rhs = float((x.astype(np.float64) * E.conv1d_T(y, w, axis, border)).sum())
        assert abs(lhs - rhs) <= 1e-5 * max(1.0, abs(lhs)), (w, lhs, rhs)


def _scene(seed, N=2, H=28, W=32):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    R = np.empty((N, H, W, 3), np.float32)
    for n in range(N):
        disc = ((x - W / 2 - n) ** 2 + (y - H / 2) ** 2) < (7 + n) ** 2
        base = 0.2 + 0.1 * rng.random(3)
        fg = 0.8 - 0.1 * rng.random(3)
        R[n] = np.where(disc[..., None], fg, base) + rng.normal(0, 0.01, (H, W, 3))
    obs = R.copy()
    obs[:, :, 2:] = R[:, :, :-2]          # the observation's disc sits two pixels over
    mask = np.ones((N, H, W), np.uint8)
    mask[:, :3] = 0
    T = np.eye(3)[None] + rng.normal(0, 0.03, (N, 3, 3))
    return R, obs, mask, T.astype(np.float32)


def test_identity_transform_equals_no_transform():
    R, _, _, _ = _scene(6)
    eye = np.tile(np.eye(3, dtype=np.float32), (R.shape[0], 1, 1))
    assert np.array_equal(E.edges(R, eye), E.edges(R))


@pytest.mark.parametrize("with_T", [False, True])
def test_edge_loss_adjoint_matches_finite_differences(with_T):
    R, obs, mask, T = _scene(7)
    Tm = T if with_T else None
    Eo = E.edges(obs)
    L, A, dT, c, Eh = E.edge_loss(R, Tm, Eo, mask, weight=2.0)
    assert c["kept"].sum() > 20 and np.abs(A).max() > 0
    sel = c["kept"]
    # the float64 statement with the selection fixed agrees with the float32 forward
    assert abs(E.edge_loss_fixed(R, Tm, Eo, mask, sel, weight=2.0) - L) < 1e-5 * L
    rng = np.random.default_rng(8)
    h = 1e-4   # float64 round-off of the summed loss dominates below ~1e-5
    for _ in range(3):
        dR = rng.normal(size=R.shape)
        Lp = E.edge_loss_fixed(R + h * dR, Tm, Eo, mask, sel, weight=2.0)
        Lm = E.edge_loss_fixed(R - h * dR, Tm, Eo, mask, sel, weight=2.0)
        fd = (Lp - Lm) / (2 * h)
        an = float((A * dR).sum())
        assert abs(fd - an) <= 1e-4 * abs(an) + 1e-9, (fd, an)
    if with_T:
        for _ in range(3):
            dTd = rng.normal(size=T.shape)
            Lp = E.edge_loss_fixed(R, T + h * dTd, Eo, mask, sel, weight=2.0)
            Lm = E.edge_loss_fixed(R, T - h * dTd, Eo, mask, sel, weight=2.0)
            fd = (Lp - Lm) / (2 * h)
            an = float((dT.reshape(-1, 3, 3) * dTd).sum())
            assert abs(fd - an) <= 1e-4 * abs(an) + 1e-9, (fd, an)
