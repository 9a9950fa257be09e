"""GPU parity of the edge term D_e (Eq. 4): the blurred Canny maps bit for bit (every
selection and every float32 value of the fixed-order forward agrees with the
oracle), the loss, and the adjoints into the image and the colour transforms, which
the kernels ADD to what the buffers hold.  Images come from the seeded input
generators (background plates, with bright discs standing in for the hand's
silhouette), at ragged sizes (neither side a multiple of the 32 x 8 tile), at the
paper's 8 x 512 x 384, and at degenerate sizes whose borders fold every tap."""
import numpy as np
import pytest

from oracle import edges as E
from paper_2107_05509_gb300 import inputs as I
from tests.gpu_common import grad_ok, require_gpu, torch

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _scene(seed, N, H, W):
    R = I.background(seed, N, H, W).astype(np.float32)
    obs = I.background(seed, N, H, W).astype(np.float32)
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    for n in range(N):
        cx, cy, r = W * rng.uniform(0.4, 0.6), H * rng.uniform(0.4, 0.6), min(H, W) * rng.uniform(0.15, 0.3)
        col = rng.uniform(0.6, 0.95, 3).astype(np.float32)
        R[n][(x - cx) ** 2 + (y - cy) ** 2 < r * r] = col
        obs[n][(x - cx - 2) ** 2 + (y - cy + 1) ** 2 < (r * 1.05) ** 2] = col * 0.97
    obs = I.add_noise(obs, seed, 0.01)
    mask = np.zeros((N, H, W), np.uint8)
    mask[:, H // 8:H - H // 8, W // 10:W - W // 10] = 1
    T = (np.eye(3)[None] + rng.normal(0, 0.04, (N, 3, 3))).astype(np.float32).reshape(N, 9)
    return R, obs, mask, T


def _run(seed, N, H, W, with_T=True, weight=1.5):
    from paper_2107_05509_gb300 import binding as B
    R, obs, mask, T = _scene(seed, N, H, W)
    Tm = T if with_T else None
    ctx = B.Context(8, 8, 8, N, W, H)
    e_obs = torch.empty((N, H, W), device="cuda")
    B.hr_edges(ctx, _t(obs), e_obs)
    ref_obs = E.edges(obs)
    assert np.array_equal(e_obs.cpu().numpy(), ref_obs), np.argwhere(e_obs.cpu().numpy() != ref_obs)[:5]
    e_r = torch.empty((N, H, W), device="cuda")
    B.hr_edges(ctx, _t(R), e_r, T=None if Tm is None else _t(Tm))
    L, A, dT, c, Eh = E.edge_loss(R, None if Tm is None else Tm.reshape(N, 3, 3), ref_obs, mask, weight=weight)
    assert np.array_equal(e_r.cpu().numpy(), Eh)
    adj = torch.zeros(R.shape, device="cuda")
    dTt = torch.zeros((N, 9), device="cuda")
    loss = torch.empty(1, device="cuda")

    def call():
        B.hr_edge_loss(ctx, _t(R), _t(ref_obs), _t(mask), loss, adj, T=None if Tm is None else _t(Tm),
                       dT=dTt if with_T else None, weight=weight)

    call()
    assert B.hr_get_status(ctx) == B.HR_OK
    got_L = float(loss.item())
    assert abs(got_L - L) <= 1e-5 * max(L, 1e-12), (got_L, L)
    ga = adj.cpu().numpy().astype(np.float64)
    ok = grad_ok(ga, A)
    assert ok.all(), (np.argwhere(~ok)[:5], ga[~ok][:5], A[~ok][:5])
    gT = dTt.cpu().numpy()
    if with_T:
        ok = grad_ok(gT.astype(np.float64), dT)
        assert ok.all(), (gT, dT)
    else:
        assert not gT.any()
    # a second call adds the same (deterministic) contributions to what the buffers hold
    a1, t1 = adj.clone(), dTt.clone()
    call()
    assert torch.equal(adj, 2 * a1) and torch.equal(dTt, 2 * t1)
    ctx.close()
    return c, L, A


@pytest.mark.parametrize("with_T", [False, True])
def test_ragged_views_match_oracle(with_T):
    require_gpu()
    c, L, A = _run(31, 3, 76, 100, with_T)
    assert c["kept"].sum() > 100 and c["strong"].sum() > 0 and (c["cand"] & ~c["kept"]).sum() > 0
    assert L > 0 and np.abs(A).max() > 0


def test_paper_size_matches_oracle():
    require_gpu()
    c, L, A = _run(32, 8, 384, 512, True)
    assert c["kept"].sum() > 1000


@pytest.mark.parametrize("H,W", [(1, 1), (1, 5), (3, 2), (9, 33)])
def test_degenerate_sizes_match_oracle(H, W):
    require_gpu()
    _run(33, 2, H, W, True)


def test_empty_mask_and_flat_image():
    require_gpu()
    from paper_2107_05509_gb300 import binding as B
    N, H, W = 2, 40, 48
    ctx = B.Context(8, 8, 8, N, W, H)
    flat = torch.full((N, H, W, 3), 0.5, device="cuda")
    e = torch.full((N, H, W), -1.0, device="cuda")
    B.hr_edges(ctx, flat, e)
    assert (e == 0).all()
    R, obs, mask, T = _scene(34, N, H, W)
    adj = torch.full((N, H, W, 3), 0.25, device="cuda")
    loss = torch.full((1,), -1.0, device="cuda")
    B.hr_edge_loss(ctx, _t(R), _t(E.edges(obs)), torch.zeros((N, H, W), dtype=torch.uint8, device="cuda"), loss,
                   adj)
    assert float(loss.item()) == 0.0 and (adj == 0.25).all()
    assert B.hr_get_status(ctx) == B.HR_OK
    with pytest.raises(B.HandrtError):
        B.hr_edges(ctx, flat, torch.empty((N, H, W + 1), device="cuda"))   # wider than the context
