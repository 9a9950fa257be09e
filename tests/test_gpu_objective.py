"""GPU parity of the paper's remaining objective terms against the oracle: the data
term with per-camera colour transforms (loss, adjoint with respect to the rendering,
transform gradient), the model's joint locations and their adjoint through the
kinematic chain, the smooth-L1 joint prior, and the two-level colour map with its
adjoint."""
import numpy as np
import pytest

import oracle
from paper_2107_05509_gb300 import inputs as I
from tests.gpu_common import grad_ok, hand, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    require_gpu()
    from paper_2107_05509_gb300 import binding
    return binding


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def test_colour_transformed_loss(B):
    rng = np.random.default_rng(0)
    N, H, W = 3, 40, 52
    R = rng.uniform(0, 1, (N, H, W, 3)).astype(np.float32)
    O = rng.uniform(0, 1, (N, H, W, 3)).astype(np.float32)
    M = (rng.uniform(0, 1, (N, H, W)) > 0.4).astype(np.uint8)
    T = (np.eye(3)[None] + rng.normal(0, 0.05, (N, 3, 3))).reshape(N, 9).astype(np.float32)
    L_ref, A_ref, dT_ref = oracle.loss_ct(R, O, M, T)
    h = hand()
    ctx = B.Context(h.V, h.F, h.E, N, W, H)
    loss = torch.zeros(1, device="cuda")
    adj = torch.empty((N, H, W, 3), device="cuda")
    dT = torch.empty((N, 9), device="cuda")
    for _ in range(2):   # deterministic: identical on repeat
        B.hr_loss_ct(ctx, _t(R), _t(O), _t(M), _t(T), loss, adj, dT)
        assert abs(loss.item() - L_ref) <= 1e-5 * abs(L_ref)
        a = adj.cpu().numpy()
        assert np.abs(a - A_ref).max() <= 1e-6 * np.abs(A_ref).max()
        assert grad_ok(dT.cpu().numpy(), dT_ref).all()
    # identity transforms: the plain loss
    Ti = np.tile(np.eye(3).reshape(9), (N, 1)).astype(np.float32)
    B.hr_loss_ct(ctx, _t(R), _t(O), _t(M), _t(Ti), loss, adj, None)
    L0, A0 = oracle.loss(R, O, M)
    assert abs(loss.item() - L0) <= 1e-5 * L0 and np.abs(adj.cpu().numpy() - A0).max() <= 1e-7 * np.abs(A0).max()
    assert B.hr_get_status(ctx) == B.HR_OK


def test_joints_and_prior(B):
    h = hand()
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, 1, 8, 8)
    x = I.perturb_params(I.gt_params(9), 9).astype(np.float32)
    verts = torch.empty((h.V, 3), device="cuda")
    joints = torch.empty((h.j_template.shape[0], 3), device="cuda")
    B.hr_skin_joints(ctx, model, _t(x), verts, joints)
    J_ref = oracle.skin_joints(h, x)
    assert np.abs(joints.cpu().numpy() - J_ref).max() < 2e-6
    target = (J_ref + np.random.default_rng(1).normal(0, 0.006, J_ref.shape)).astype(np.float32)
    loss = torch.empty(1, device="cuda")
    dj = torch.empty_like(joints)
    B.hr_joint_prior(joints, _t(target), 0.005, 1e-3, loss, dj)
    E_ref, g_ref = oracle.joint_prior(joints.cpu().numpy(), target, 0.005, 1e-3)
    assert abs(loss.item() - E_ref) <= 1e-5 * E_ref
    assert np.allclose(dj.cpu().numpy(), g_ref, rtol=1e-5, atol=1e-9)
    rng = np.random.default_rng(2)
    dV = rng.normal(0, 1, (h.V, 3)).astype(np.float32)
    dJ = rng.normal(0, 1, J_ref.shape).astype(np.float32)
    dp = torch.empty(61, device="cuda")
    B.hr_skin_bwd_joints(ctx, model, _t(x), _t(dV), _t(dJ), dp)
    ok = grad_ok(dp.cpu().numpy(), oracle.skin_bwd(h, x, dV, dJ))
    assert ok.all(), np.argwhere(~ok)
    assert B.hr_get_status(ctx) == B.HR_OK


def test_colour_map(B):
    rng = np.random.default_rng(3)
    lo = rng.normal(size=(8, 8, 3)).astype(np.float32)
    hi = rng.normal(size=(512, 512, 3)).astype(np.float32)
    out = torch.empty((512, 512, 3), device="cuda")
    B.hr_colour_map(_t(lo), _t(hi), out)
    assert np.allclose(out.cpu().numpy(), oracle.colour_map(lo, hi), rtol=0, atol=1e-6)
    d = rng.normal(size=(512, 512, 3)).astype(np.float32)
    dlo = torch.empty((8, 8, 3), device="cuda")
    B.hr_colour_map_bwd(_t(d), dlo)
    ref = oracle.colour_map_bwd(d, lo.shape)
    assert np.allclose(dlo.cpu().numpy(), ref, rtol=1e-5, atol=1e-4)
