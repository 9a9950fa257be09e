"""Oracle of the edge term D_e (test infrastructure only: used by tests/, never by the
product path).

Eq. 4 compares Canny edge maps of the observation o and of the rendering r, each
blurred by K, an 11 x 11 Gaussian of sigma 5:  D_e(o, r) = |Canny(o) * K - Canny(r) * K|.
The rendering that enters the data term is camera i's T_i R (Eq. 2), so Canny sees
T_i R.  Canny's detector (Canny 1986) is taken as its textbook steps:

  gray   g = w . (T R), w = (0.299, 0.587, 0.114) (Rec. 601 luma), evaluated as
         a . R with a = T^T w (a = w without a transform)
  smooth s = G5 (x) G5 g: separable 5-tap Gaussian, sigma 1, horizontal pass first,
         image border replicated (each pass reads clamped coordinates)
  Sobel  gx = D_x (S_y s), gy = D_y (S_x s): S = (1/4, 1/2, 1/4), D = (-1/2, 0, 1/2)
         (the Sobel operator / 8, so a linear ramp gives its slope), border replicated
  m      = sqrt(gx^2 + gy^2 + 1e-12)
  NMS    the gradient direction quantised to 0, 45, 90 or 135 degrees
         (|gy| <= tan(22.5) |gx|: along x; |gy| >= tan(67.5) |gx|: along y; else the
         diagonal with gx gy > 0 (x+1, y+1)/(x-1, y-1), or the other one); a pixel
         survives when m >= m at both neighbours along that direction (neighbour
         coordinates clamped to the image, each on its own)
  double threshold: candidates = survivors with m > low; strong = m > high
  hysteresis: a candidate is kept when its 8-connected component of candidates
         holds a strong pixel
  E      = m on kept pixels, 0 elsewhere (the detector's edge strength: the selection
         is piecewise constant in the image, so the derivative of D_e flows through
         m on the kept pixels and the selection is held fixed)
  E_hat  = K_y K_x E with zero padding (no edges outside the image)

Every forward quantity up to E_hat is float32 in a fixed operation order (each
convolution sums its taps from the most negative offset up, one rounding per
multiply and per add), because the selection (NMS, thresholds) and the sign of
E_hat_r - E_hat_o are decisions that the CUDA path must take on the same float32
values.  The loss and its adjoint are float64:

  L_e  = weight sum_p M_p |E_hat_r - E_hat_o| / sum_p M_p
  dL/dR_p = a gbar_p,   dL/dT_i[r][c] = w_r sum_{p in view i} gbar_p R_pc

with gbar = G5^T G5^T (S_y^T D_x^T (m_bar gx / m) + S_x^T D_y^T (m_bar gy / m)),
m_bar = kept ? (K^T K^T (weight M sign(d) / sum M)) : 0, each transpose the adjoint
of its forward pass including the border rule (a replicated border sends the
gradient of every clamped read back to the border pixel).
"""
from __future__ import annotations

import math
from collections import deque

import numpy as np

GRAY_W = (0.299, 0.587, 0.114)
PRE_RADIUS, PRE_SIGMA = 2, 1.0       # Canny's smoothing, 5 x 5
K_RADIUS, K_SIGMA = 5, 5.0           # K of Eq. 4, 11 x 11
SMOOTH = (0.25, 0.5, 0.25)
DERIV = (-0.5, 0.0, 0.5)
MAG_EPS = 1e-12
LOW, HIGH = 0.05, 0.1            # on the /8-normalised gradient: a step of contrast c peaks near 0.32 c


def gauss_weights(radius, sigma):
    """Normalised 1-D Gaussian taps at offsets -radius..radius: exp(-k^2 / (2 sigma^2))
    in float64, divided by their sum (added from offset -radius up), rounded to
    float32."""
    e = [math.exp(-(k * k) / (2.0 * sigma * sigma)) for k in range(-radius, radius + 1)]
    tot = 0.0
    for v in e:
        tot += v
    return np.array([v / tot for v in e], np.float32)


def _f32(x):
    return np.asarray(x, np.float32)


def conv1d(x, w, axis, border):
    """y[i] = sum_k w_k x[i + k] along `axis` (k = -r..r, w indexed from -r), float32,
    taps added in order; border 'clamp' reads x[clamp(i + k)], 'zero' reads 0 outside."""
    x = _f32(x)
    w = _f32(w)
    r = len(w) // 2
    n = x.shape[axis]
    idx = np.arange(n)
    acc = None
    for t in range(len(w)):
        j = idx + (t - r)
        if border == "clamp":
            src = np.take(x, np.clip(j, 0, n - 1), axis=axis)
        else:
            ok = (j >= 0) & (j < n)
            src = np.take(x, np.clip(j, 0, n - 1), axis=axis)
            shape = [1] * x.ndim
            shape[axis] = n
            src = np.where(ok.reshape(shape), src, np.float32(0.0)).astype(np.float32)
        term = (w[t] * src).astype(np.float32)
        acc = term if acc is None else (acc + term).astype(np.float32)
    return acc


def conv1d_T(y, w, axis, border):
    """The adjoint of conv1d (float64): every read x[c(i + k)] of the forward sends
    w_k y[i] back to c(i + k), with c the clamp (or nothing for a zero read)."""
    y = np.asarray(y, np.float64)
    w = np.asarray(w, np.float64)
    r = len(w) // 2
    n = y.shape[axis]
    idx = np.arange(n)
    out = np.zeros_like(y)
    lead = (slice(None),) * (axis % y.ndim)
    for t in range(len(w)):
        j = idx + (t - r)
        if border == "clamp":
            np.add.at(out, lead + (np.clip(j, 0, n - 1),), w[t] * y)
        else:
            ok = (j >= 0) & (j < n)
            np.add.at(out, lead + (j[ok],), w[t] * np.take(y, idx[ok], axis=axis))
    return out


def gray_weights(T=None, N=1):
    """a_i = T_i^T w per view in float32: a_c = (w_0 T[0][c] + w_1 T[1][c]) + w_2 T[2][c]."""
    w = _f32(GRAY_W)
    if T is None:
        return np.tile(w, (N, 1))
    T = _f32(T).reshape(-1, 3, 3)
    a = (w[0] * T[:, 0, :]).astype(np.float32)
    a = (a + (w[1] * T[:, 1, :]).astype(np.float32)).astype(np.float32)
    a = (a + (w[2] * T[:, 2, :]).astype(np.float32)).astype(np.float32)
    return a


def gray(R, a):
    """g = (a_0 R_0 + a_1 R_1) + a_2 R_2 per pixel, float32."""
    R = _f32(R)
    a = _f32(a)[:, None, None, :]
    g = (a[..., 0] * R[..., 0]).astype(np.float32)
    g = (g + (a[..., 1] * R[..., 1]).astype(np.float32)).astype(np.float32)
    return (g + (a[..., 2] * R[..., 2]).astype(np.float32)).astype(np.float32)


def hysteresis(cand, strong):
    """Candidates whose 8-connected component of candidates holds a strong pixel
    (breadth-first search from every strong pixel), per view."""
    cand = np.asarray(cand, bool)
    kept = np.zeros_like(cand)
    N, H, W = cand.shape
    for n in range(N):
        c, k = cand[n], kept[n]
        q = deque()
        for y, x in zip(*np.nonzero(np.asarray(strong[n], bool) & c)):
            if not k[y, x]:
                k[y, x] = True
                q.append((y, x))
            while q:
                cy, cx = q.popleft()
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        yy, xx = cy + dy, cx + dx
                        if 0 <= yy < H and 0 <= xx < W and c[yy, xx] and not k[yy, xx]:
                            k[yy, xx] = True
                            q.append((yy, xx))
    return kept


def canny(R, T=None, low=LOW, high=HIGH):
    """The detector's stages for images R [N][H][W][3]; returns a dict of the float32
    intermediates (g, s, gx, gy, m), the selections (cand, strong, kept) and E."""
    R = _f32(R)
    N = R.shape[0]
    a = gray_weights(T, N)
    g = gray(R, a)
    w5 = gauss_weights(PRE_RADIUS, PRE_SIGMA)
    s = conv1d(conv1d(g, w5, 2, "clamp"), w5, 1, "clamp")
    gx = conv1d(conv1d(s, SMOOTH, 1, "clamp"), DERIV, 2, "clamp")
    gy = conv1d(conv1d(s, SMOOTH, 2, "clamp"), DERIV, 1, "clamp")
    m2 = ((gx * gx).astype(np.float32) + (gy * gy).astype(np.float32)).astype(np.float32)
    m = np.sqrt((m2 + np.float32(MAG_EPS)).astype(np.float32)).astype(np.float32)
    ax, ay = np.abs(gx), np.abs(gy)
    t1 = np.float32(math.sqrt(2.0) - 1.0)
    t2 = np.float32(math.sqrt(2.0) + 1.0)
    along_x = ay <= (t1 * ax).astype(np.float32)
    along_y = ~along_x & (ay >= (t2 * ax).astype(np.float32))
    same = (gx > 0) == (gy > 0)
    # neighbours (x +- dx, y +- dy): along x (1, 0), along y (0, 1), diagonals (1, 1)
    # when gx and gy share a sign, else (1, -1)
    dx = np.where(along_y, 0, 1)
    dy = np.where(along_x, 0, np.where(along_y, 1, np.where(same, 1, -1)))
    _, H, W = m.shape
    n_i, y_i, x_i = np.meshgrid(np.arange(N), np.arange(H), np.arange(W), indexing="ij")
    m1 = m[n_i, np.clip(y_i + dy, 0, H - 1), np.clip(x_i + dx, 0, W - 1)]
    m_2 = m[n_i, np.clip(y_i - dy, 0, H - 1), np.clip(x_i - dx, 0, W - 1)]
    keep = (m >= m1) & (m >= m_2)
    cand = keep & (m > np.float32(low))
    strong = cand & (m > np.float32(high))
    kept = hysteresis(cand, strong)
    E = np.where(kept, m, np.float32(0.0)).astype(np.float32)
    return dict(a=a, g=g, s=s, gx=gx, gy=gy, m=m, cand=cand, strong=strong, kept=kept, E=E)


def blur_k(E):
    """E_hat = K_y K_x E, zero padding, float32 in the fixed tap order."""
    k = gauss_weights(K_RADIUS, K_SIGMA)
    return conv1d(conv1d(E, k, 2, "zero"), k, 1, "zero")


def edges(R, T=None, low=LOW, high=HIGH):
    """Canny(T R) * K per view, [N][H][W] float32."""
    return blur_k(canny(R, T, low, high)["E"])


def edge_loss(R, T, edges_obs, mask, low=LOW, high=HIGH, weight=1.0):
    """L_e and its adjoints (float64): returns (L, dL/dR [N][H][W][3], dL/dT [N][9] or
    None, the canny dict, E_hat of R)."""
    R = _f32(R)
    N = R.shape[0]
    c = canny(R, T, low, high)
    Eh = blur_k(c["E"])
    d = Eh.astype(np.float64) - np.asarray(edges_obs, np.float32).astype(np.float64)
    M = (np.asarray(mask) != 0).astype(np.float64)
    cnt = M.sum()
    scale = weight / cnt if cnt > 0 else 0.0
    L = float((M * np.abs(d)).sum() * scale)
    gE = M * np.sign(d) * scale
    k = gauss_weights(K_RADIUS, K_SIGMA)
    Ebar = conv1d_T(conv1d_T(gE, k, 1, "zero"), k, 2, "zero")
    mbar = np.where(c["kept"], Ebar, 0.0)
    m = c["m"].astype(np.float64)
    gxb = mbar * c["gx"].astype(np.float64) / m
    gyb = mbar * c["gy"].astype(np.float64) / m
    sbar = conv1d_T(conv1d_T(gxb, DERIV, 2, "clamp"), SMOOTH, 1, "clamp")
    sbar += conv1d_T(conv1d_T(gyb, DERIV, 1, "clamp"), SMOOTH, 2, "clamp")
    w5 = gauss_weights(PRE_RADIUS, PRE_SIGMA)
    gbar = conv1d_T(conv1d_T(sbar, w5, 1, "clamp"), w5, 2, "clamp")
    a = c["a"].astype(np.float64)
    A = gbar[..., None] * a[:, None, None, :]
    dT = None
    if T is not None:
        wv = np.asarray(_f32(GRAY_W), np.float64)
        S = np.einsum("nhw,nhwc->nc", gbar, R.astype(np.float64))
        dT = (wv[None, :, None] * S[:, None, :]).reshape(N, 9)
    return L, A, dT, c, Eh


def edge_loss_fixed(R, T, edges_obs, mask, sel, weight=1.0):
    """L_e in float64 with the selection `sel` (kept pixels) and the signs' reference
    held fixed: the smooth function whose derivative the adjoint is (finite-difference
    pins)."""
    R = np.asarray(R, np.float64)
    N = R.shape[0]
    w = np.asarray(GRAY_W, np.float64)
    if T is None:
        a = np.tile(w, (N, 1))
    else:
        a = np.einsum("r,nrc->nc", w, np.asarray(T, np.float64).reshape(-1, 3, 3))
    g = np.einsum("nhwc,nc->nhw", R, a)
    w5 = gauss_weights(PRE_RADIUS, PRE_SIGMA).astype(np.float64)

    def conv(x, wt, axis, border):
        r = len(wt) // 2
        n = x.shape[axis]
        out = np.zeros_like(x)
        for t in range(len(wt)):
            j = np.arange(n) + t - r
            if border == "clamp":
                out += wt[t] * np.take(x, np.clip(j, 0, n - 1), axis=axis)
            else:
                ok = (j >= 0) & (j < n)
                src = np.take(x, np.clip(j, 0, n - 1), axis=axis)
                shape = [1] * x.ndim
                shape[axis] = n
                out += wt[t] * np.where(ok.reshape(shape), src, 0.0)
        return out

    s = conv(conv(g, w5, 2, "clamp"), w5, 1, "clamp")
    gx = conv(conv(s, np.array(SMOOTH), 1, "clamp"), np.array(DERIV), 2, "clamp")
    gy = conv(conv(s, np.array(SMOOTH), 2, "clamp"), np.array(DERIV), 1, "clamp")
    m = np.sqrt(gx * gx + gy * gy + MAG_EPS)
    E = np.where(sel, m, 0.0)
    k = gauss_weights(K_RADIUS, K_SIGMA).astype(np.float64)
    Eh = conv(conv(E, k, 2, "zero"), k, 1, "zero")
    M = (np.asarray(mask) != 0).astype(np.float64)
    return float(weight * (M * np.abs(Eh - np.asarray(edges_obs, np.float64))).sum() / M.sum())
