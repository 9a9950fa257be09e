"""Oracle of the learned proposal network (test infrastructure only: used by tests/,
never by the product path).

A plain float64 NumPy statement of the network the CUDA library trains (an
extension of the paper's method: Section 3 refines by gradient descent alone; the
network proposes the first parameter updates from per-view residual images):

    X0   [NV][128][128][8]    inputs (given)
    Y_l  3x3 convolution, stride 2, padding 1, ReLU, l = 1..5:
         8->32, 32->64, 64->128, 128->128, 128->128   (128 -> 64 -> 32 -> 16 -> 8 -> 4)
    Z    [NV][2112] = Y5 flattened (y, x, c) | camera R (9) | centre / 0.6 (3) | zeros
    F    ReLU(Z Wv^T + bv)  [NV][256]
    P    max over the views of each instance (first maximum on ties)
    H    ReLU(P W1^T + b1)  [B][256]
    O    H W2^T + b2        [B][64]; delta[:, j] = s_j O[:, j] for j < 61

With bf16=True every stored tensor is rounded to bfloat16 where the CUDA path stores
bfloat16 (weights as GEMM operands, activations, back-propagated activation
gradients) and everything else is exact (float64), so the two agree up to the
float32 accumulation order and the bf16 rounding it can flip.  With bf16=False the
network is plain float64 (what the finite-difference pins check).

Parameter vector layout: per layer W [N][K] row-major then b [N]; conv K = 9 Cin
rounded up to 64 with k = (3 ky + kx) Cin + c; view layer K = 2112; W1 256x256;
W2 64x256 (rows 61-63 unused).
"""
from __future__ import annotations

import numpy as np

IN_SIDE, IN_CH = 128, 8
CONV_IN = (8, 32, 64, 128, 128)
CONV_OUT = (32, 64, 128, 128, 128)
FEAT, ZDIM, HID, NOUT, NOUT_PAD = 2048, 2112, 256, 61, 64
GROUP_SCALE = np.concatenate([np.full(10, 0.5), np.full(45, 0.1), np.full(3, 0.1), np.full(3, 0.005)])


def _pad64(k):
    return (k + 63) // 64 * 64


def layers():
    """(name, N, K) of every dense layer in parameter order."""
    out = [(f"conv{l + 1}", CONV_OUT[l], _pad64(9 * CONV_IN[l])) for l in range(5)]
    return out + [("view", HID, ZDIM), ("fc1", HID, HID), ("fc2", NOUT_PAD, HID)]


def offsets():
    off, table = 0, {}
    for name, N, K in layers():
        table[name] = (off, off + N * K, N, K)
        off += N * K + N
    return table, off


def param_count():
    return offsets()[1]


def unpack(params):
    table, _ = offsets()
    out = {}
    for name, (w, b, N, K) in table.items():
        out[name] = (np.asarray(params[w:w + N * K], np.float64).reshape(N, K),
                     np.asarray(params[b:b + N], np.float64))
    return out


def bf16_round(x):
    """Round to bfloat16 (nearest, ties to even) via float32, returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    a = ((a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return a.view(np.float32).astype(np.float64)


def init_params(seed=0):
    """He-normal weights on the real (unpadded) inputs, zero biases, zero padding."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 5150]))
    table, P = offsets()
    p = np.zeros(P, np.float64)
    fan = {f"conv{l + 1}": 9 * CONV_IN[l] for l in range(5)}
    fan.update(view=FEAT + 12, fc1=HID, fc2=HID)
    for name, (w, b, N, K) in table.items():
        W = np.zeros((N, K))
        n_real = NOUT if name == "fc2" else N
        std = np.sqrt(2.0 / fan[name]) if name != "fc2" else 0.1 * np.sqrt(1.0 / fan[name])
        W[:n_real, :fan[name]] = rng.normal(0.0, std, (n_real, fan[name]))
        p[w:w + N * K] = W.reshape(-1)
    return p.astype(np.float32)


def im2col(X, Cin):
    """[NV][H][H][Cin] -> [NV*(H/2)^2][pad64(9 Cin)] for the 3x3 / stride-2 / pad-1 taps."""
    NV, H = X.shape[0], X.shape[1]
    Ho = H // 2
    Xp = np.zeros((NV, H + 2, H + 2, Cin))
    Xp[:, 1:H + 1, 1:H + 1] = X
    K = _pad64(9 * Cin)
    cols = np.zeros((NV, Ho, Ho, K))
    for ky in range(3):
        for kx in range(3):
            t = ky * 3 + kx
            cols[..., t * Cin:(t + 1) * Cin] = Xp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Ho:2, :]
    return cols.reshape(NV * Ho * Ho, K)


def col2im(dcols, NV, H, Cin):
    """Adjoint of im2col: scatter-add the tap gradients back to the input pixels."""
    Ho = H // 2
    d = dcols.reshape(NV, Ho, Ho, -1)
    dXp = np.zeros((NV, H + 2, H + 2, Cin))
    for ky in range(3):
        for kx in range(3):
            t = ky * 3 + kx
            dXp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Ho:2, :] += d[..., t * Cin:(t + 1) * Cin]
    return dXp[:, 1:H + 1, 1:H + 1, :]


def camera_features(cams):
    c = np.asarray(cams, np.float64)
    f = np.zeros((c.shape[0], ZDIM - FEAT))
    f[:, :9] = c[:, 4:13]
    f[:, 9:12] = c[:, 16:19] / 0.6
    return f


def inputs(render, observed):
    """X0 from 256x256 renders and observations [NV][256][256][3]: 2x2 means,
    (R - O, O, 0, 0)."""
    R = np.asarray(render, np.float64)
    O = np.asarray(observed, np.float64)
    NV = R.shape[0]
    r = R.reshape(NV, 128, 2, 128, 2, 3).mean(axis=(2, 4))
    o = O.reshape(NV, 128, 2, 128, 2, 3).mean(axis=(2, 4))
    X = np.zeros((NV, 128, 128, IN_CH))
    X[..., 0:3] = r - o
    X[..., 3:6] = o
    return X


def forward(params, X0, cams, B, nv, bf16=True, base=None):
    """Returns (out [B][61], cache).  X0 [B*nv][128][128][8], cams [B*nv][20]."""
    rd = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    w = unpack(params)
    NV = B * nv
    acts = [rd(np.asarray(X0, np.float64))]
    cols_all = []
    for l in range(5):
        W, b = w[f"conv{l + 1}"]
        H = acts[-1].shape[1]
        cols = im2col(acts[-1], CONV_IN[l])
        cols_all.append(cols)
        Y = np.maximum(cols @ rd(W).T + b, 0.0)
        acts.append(rd(Y).reshape(NV, H // 2, H // 2, CONV_OUT[l]))
    Z = np.concatenate([acts[-1].reshape(NV, FEAT), rd(camera_features(cams))], axis=1)
    Wv, bv = w["view"]
    F = rd(np.maximum(Z @ rd(Wv).T + bv, 0.0))
    Fr = F.reshape(B, nv, HID)
    idx = np.argmax(Fr, axis=1)          # first maximum
    P = np.take_along_axis(Fr, idx[:, None, :], axis=1)[:, 0, :]
    W1, b1 = w["fc1"]
    Hh = rd(np.maximum(P @ rd(W1).T + b1, 0.0))
    W2, b2 = w["fc2"]
    O = Hh @ rd(W2).T + b2
    out = GROUP_SCALE * O[:, :NOUT]
    if base is not None:
        out = out + np.asarray(base, np.float64)
    cache = dict(acts=acts, cols=cols_all, Z=Z, F=F, idx=idx, P=P, H=Hh, w=w, B=B, nv=nv, bf16=bf16)
    return out, cache


def backward(cache, d_out):
    """Gradient of the parameter vector for d_out = dL/d delta [B][61]."""
    rd = bf16_round if cache["bf16"] else (lambda a: np.asarray(a, np.float64))
    w, B, nv = cache["w"], cache["B"], cache["nv"]
    NV = B * nv
    table, Ptot = offsets()
    g = np.zeros(Ptot)

    def put(name, dW, db):
        wo, bo, N, K = table[name]
        g[wo:wo + N * K] = dW.reshape(-1)
        g[bo:bo + N] = db

    dO = np.zeros((B, NOUT_PAD))
    dO[:, :NOUT] = rd(GROUP_SCALE * np.asarray(d_out, np.float64))
    W2, _ = w["fc2"]
    put("fc2", dO.T @ cache["H"], dO.sum(0))
    dH = rd(dO @ rd(W2))
    dPre = dH * (cache["H"] > 0)
    W1, _ = w["fc1"]
    put("fc1", dPre.T @ cache["P"], dPre.sum(0))
    dP = rd(dPre @ rd(W1))
    dF = np.zeros((B, nv, HID))
    np.put_along_axis(dF, cache["idx"][:, None, :], dP[:, None, :], axis=1)
    dF = dF.reshape(NV, HID)
    dPre = dF * (cache["F"] > 0)
    Wv, _ = w["view"]
    put("view", dPre.T @ cache["Z"], dPre.sum(0))
    dZ = rd(dPre @ rd(Wv))
    dY = dZ[:, :FEAT].reshape(cache["acts"][-1].shape)
    for l in range(4, -1, -1):
        Y = cache["acts"][l + 1]
        dPre = (dY * (Y > 0)).reshape(-1, CONV_OUT[l])
        W, _ = w[f"conv{l + 1}"]
        put(f"conv{l + 1}", dPre.T @ cache["cols"][l], dPre.sum(0))
        if l == 0:
            break
        dcols = rd(dPre @ rd(W))
        H = cache["acts"][l].shape[1]
        dY = rd(col2im(dcols, NV, H, CONV_IN[l]))
    return g


def vertex_mse(a, b):
    """loss_i = mean_v |a_i - b_i|^2 and d((1/n) sum_i loss_i)/da."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    n, V = a.shape[0], a.shape[1]
    d = a - b
    return (d ** 2).sum(axis=(1, 2)) / V, 2.0 * d / (V * n)
