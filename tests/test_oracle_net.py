"""Pins of the proposal-network oracle (oracle/net.py) against definitions that do
not go through it: a direct loop convolution, the adjoint identity of im2col and
col2im, central finite differences of the float64 network, the first-maximum rule
of the view pooling, and the closed form of the vertex loss."""
import numpy as np
import pytest

from oracle import net as N


def test_im2col_matches_direct_strided_correlation():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(2, 8, 8, 3))
    W = rng.normal(size=(4, 3, 3, 3))     # [Cout][ky][kx][Cin]
    ref = np.zeros((2, 4, 4, 4))
    for n in range(2):
        for oy in range(4):
            for ox in range(4):
                for co in range(4):
                    s = 0.0
                    for ky in range(3):
                        for kx in range(3):
                            y, x = 2 * oy - 1 + ky, 2 * ox - 1 + kx
                            if 0 <= y < 8 and 0 <= x < 8:
                                s += W[co, ky, kx] @ X[n, y, x]
                    ref[n, oy, ox, co] = s
    Wk = np.zeros((4, 64))
    Wk[:, :27] = W.reshape(4, 27)          # k = (3 ky + kx) Cin + c
    got = (N.im2col(X, 3) @ Wk.T).reshape(2, 4, 4, 4)
    assert np.allclose(got, ref, atol=1e-12)


def test_col2im_is_the_adjoint_of_im2col():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(3, 16, 16, 5))
    D = rng.normal(size=(3 * 64, 64))
    D[:, 45:] = 0.0                        # padding columns carry no gradient
    lhs = (N.im2col(X, 5) * D).sum()
    rhs = (X * N.col2im(D, 3, 16, 5)).sum()
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def _setup(B=2, nv=2, seed=3):
    rng = np.random.default_rng(seed)
    p = N.init_params(seed).astype(np.float64)
    # non-zero biases so that every bias entry is exercised
    table, _ = N.offsets()
    for name, (w, b, n_out, K) in table.items():
        p[b:b + n_out] = rng.normal(0, 0.05, n_out)
    p[table["fc2"][1] + 61:table["fc2"][1] + 64] = 0.0
    X = rng.normal(0, 0.3, size=(B * nv, 128, 128, 8))
    X[..., 6:] = 0.0
    cams = rng.normal(size=(B * nv, 20))
    return p, X, cams


def test_network_gradient_matches_central_differences():
    B, nv = 2, 2
    p, X, cams = _setup(B, nv)
    rng = np.random.default_rng(4)
    c = rng.normal(size=(B, 61))
    out, cache = N.forward(p, X, cams, B, nv, bf16=False)
    g = N.backward(cache, c)
    table, _ = N.offsets()
    picks = []
    for name, (w, b, n_out, K) in table.items():
        n_real = 61 if name == "fc2" else n_out
        fan = 9 * N.CONV_IN[int(name[-1]) - 1] if name.startswith("conv") else {"view": 2060, "fc1": 256,
                                                                                   "fc2": 256}[name]
        for _ in range(3):
            picks.append(w + int(rng.integers(0, n_real)) * K + int(rng.integers(0, fan)))
        picks.append(b + int(rng.integers(0, n_real)))
    h = 1e-5
    for i in picks:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = ((N.forward(pp, X, cams, B, nv, bf16=False)[0] * c).sum() -
              (N.forward(pm, X, cams, B, nv, bf16=False)[0] * c).sum()) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(abs(fd), 1e-3), (i, fd, g[i])


def test_view_pooling_takes_the_first_maximum():
    B, nv = 1, 2
    p, X, cams = _setup(B, nv)
    X[1] = X[0]
    cams[1] = cams[0]                       # two identical views: every feature ties
    out, cache = N.forward(p, X, cams, B, nv, bf16=False)
    assert (cache["idx"] == 0).all()
    # the gradient then flows through view 0 only: same as a one-view instance
    c = np.ones((1, 61))
    g2 = N.backward(cache, c)
    out1, cache1 = N.forward(p, X[:1], cams[:1], 1, 1, bf16=False)
    assert np.allclose(out, out1)
    assert np.allclose(g2, N.backward(cache1, c))


def test_bf16_rounding_is_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5, 0.0], np.float64)
    got = N.bf16_round(x)
    assert got.tolist() == [1.0, 1.0, 1.0 + 4 * 2 ** -8, 1.0, -2.5, 0.0]


def test_vertex_mse_closed_form():
    a = np.zeros((2, 3, 3))
    b = np.zeros((2, 3, 3))
    a[0, 0] = [3.0, 4.0, 0.0]               # |d|^2 = 25 on one of 3 vertices
    a[1, 2] = [0.0, 0.0, 1.0]
    loss, grad = N.vertex_mse(a, b)
    assert np.allclose(loss, [25.0 / 3, 1.0 / 3])
    assert np.allclose(grad[0, 0], 2 * np.array([3.0, 4.0, 0.0]) / 6)
