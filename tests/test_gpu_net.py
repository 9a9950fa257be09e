"""The proposal network on the GPU (bf16 tensor-core GEMMs with float32
accumulation and the glue kernels around them) against the oracle's float64
statement of the same network with bf16 rounding at the same storage points.

Tolerance, from the arithmetic: every stored activation and back-propagated
activation gradient is rounded to bf16 (relative step 2^-8); the float32
accumulation order of the tensor cores differs from the oracle's float64 sums, so a
value that lies within ~1e-6 of a bf16 rounding boundary can round the other way
(one bf16 step, 0.4 %) and that difference propagates through the following layers.
Outputs and gradients therefore agree to a few bf16 steps: per entry |g - o| <=
0.03 |o| + 0.01 max|o| of its layer, and the direction of every layer's gradient to
cosine similarity >= 0.999."""
import numpy as np
import pytest

from oracle import net as N
from paper_2107_05509_gb300 import inputs as I
from tests.gpu_common import hand, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B_():
    require_gpu()
    from paper_2107_05509_gb300 import binding
    return binding


def _case(Bn=2, nv=2, seed=5):
    rng = np.random.default_rng(seed)
    p = N.init_params(seed).astype(np.float64)
    table, _ = N.offsets()
    for name, (w, b, n_out, K) in table.items():
        p[b:b + n_out] = rng.normal(0, 0.05, n_out)
    p[table["fc2"][1] + 61:table["fc2"][1] + 64] = 0.0
    p = p.astype(np.float32)
    # views of different magnitude, so that the maximum over views is decided by a
    # clear margin (a near-tie could be decided either way by one bf16 rounding, and
    # either routing of the gradient would be correct)
    scale = (1.0 + 0.5 * (np.arange(Bn * nv) % nv))[:, None, None, None]
    X = N.bf16_round(rng.normal(0, 0.3, size=(Bn * nv, 128, 128, 8)) * scale)
    X[..., 6:] = 0.0
    cfg = I.SceneConfig("net", views=nv, width=256, height=256, spp=1, edge_samples=0, elevation_deg=30.0,
                        azimuths_deg=tuple(360.0 * k / nv for k in range(nv)), seed=seed)
    cams = np.concatenate([I.pack_cameras(I.make_cameras(cfg, hand().v_template.mean(0)))] * Bn)
    return p, X, cams


def _layer_ok(g, o, name):
    g, o = np.ravel(g), np.ravel(o)
    err = np.abs(g - o)
    tol = 0.03 * np.abs(o) + 0.01 * np.abs(o).max()
    cos = float(g @ o / (np.linalg.norm(g) * np.linalg.norm(o) + 1e-30))
    assert (err <= tol).all() and cos >= 0.999, (name, err.max(), np.abs(o).max(), cos, int((err > tol).sum()))


@pytest.mark.parametrize("Bn,nv", [(2, 2), (1, 8)])
def test_net_forward_backward_match_oracle(B_, Bn, nv):
    p, X, cams = _case(Bn, nv)
    net = B_.Net(Bn, nv)
    assert net.P == N.param_count()
    dev = "cuda"
    net.set_params(torch.as_tensor(p, device=dev))
    net.set_inputs_bf16(torch.as_tensor(X.astype(np.float32), device=dev).to(torch.bfloat16))
    base = np.random.default_rng(6).normal(size=(Bn, 61)).astype(np.float32)
    out = torch.empty((Bn, 61), device=dev)
    net.forward(torch.as_tensor(cams, device=dev), out, base=torch.as_tensor(base, device=dev))
    ref, cache = N.forward(p, X, cams, Bn, nv, bf16=True, base=base)
    _layer_ok(out.cpu().numpy().astype(np.float64) - base, ref - base, "delta")
    d_out = np.random.default_rng(7).normal(size=(Bn, 61)).astype(np.float32)
    net.backward(torch.as_tensor(d_out, device=dev))
    g = torch.empty(net.P, device=dev)
    net.get_params(grads=g)
    g = g.cpu().numpy().astype(np.float64)
    o = N.backward(cache, d_out)
    table, _ = N.offsets()
    for name, (w, b, n_out, K) in table.items():
        _layer_ok(g[w:w + n_out * K], o[w:w + n_out * K], name + ".W")
        _layer_ok(g[b:b + n_out], o[b:b + n_out], name + ".b")
    assert net.status() == B_.HR_OK


def test_net_inputs_match_oracle(B_):
    """The input kernel (2x2 means of 256x256 render and observation) checked through
    a forward pass against the oracle's inputs."""
    Bn, nv = 1, 4
    p, _, cams = _case(Bn, nv, seed=8)
    rng = np.random.default_rng(9)
    R = rng.random((Bn * nv, 256, 256, 3), dtype=np.float32)
    O = rng.random((Bn * nv, 256, 256, 3), dtype=np.float32)
    net = B_.Net(Bn, nv)
    net.set_params(torch.as_tensor(p, device="cuda"))
    net.inputs(torch.as_tensor(R, device="cuda"), torch.as_tensor(O, device="cuda"))
    out = torch.empty((Bn, 61), device="cuda")
    net.forward(torch.as_tensor(cams, device="cuda"), out)
    ref, _ = N.forward(p, N.inputs(R, O), cams, Bn, nv, bf16=True)
    _layer_ok(out.cpu().numpy().astype(np.float64), ref, "delta")


def test_adam_moves_parameters_against_the_gradient(B_):
    Bn, nv = 1, 4
    p, X, cams = _case(Bn, nv, seed=10)
    net = B_.Net(Bn, nv)
    pt = torch.as_tensor(p, device="cuda")
    net.set_params(pt)
    net.set_inputs_bf16(torch.as_tensor(X.astype(np.float32), device="cuda").to(torch.bfloat16))
    out = torch.empty((Bn, 61), device="cuda")
    net.forward(torch.as_tensor(cams, device="cuda"), out)
    net.backward(torch.ones((Bn, 61), device="cuda"))
    g = torch.empty(net.P, device="cuda")
    net.get_params(grads=g)
    net.adam(1e-3, 1)
    q = torch.empty(net.P, device="cuda")
    net.get_params(params=q)
    step = (q - pt).cpu().numpy()
    gg = g.cpu().numpy()
    nz = np.abs(gg) > 1e-4
    # first Adam step: -lr g / (|g| + eps) = -lr sign(g) up to eps / |g|, zero where
    # the gradient is zero
    assert np.allclose(step[nz], -1e-3 * np.sign(gg[nz]), rtol=1e-3, atol=1e-6)
    assert (step[gg == 0] == 0).all()


def test_vertex_mse_select_best_and_noise(B_):
    rng = np.random.default_rng(11)
    a = rng.normal(size=(3, 50, 3)).astype(np.float32)
    b = rng.normal(size=(3, 50, 3)).astype(np.float32)
    loss = torch.empty(3, device="cuda")
    grad = torch.empty((3, 50, 3), device="cuda")
    B_.hr_vertex_mse(torch.as_tensor(a, device="cuda"), torch.as_tensor(b, device="cuda"), loss, grad)
    L, G = N.vertex_mse(a, b)
    assert np.allclose(loss.cpu().numpy(), L, rtol=1e-6)
    assert np.allclose(grad.cpu().numpy(), G, rtol=1e-6, atol=1e-9)
    cand = rng.normal(size=(4, 5, 61)).astype(np.float32)
    losses = rng.random((4, 5)).astype(np.float32)
    losses[2, 1] = losses[0, 1] = -1.0      # a tie: the earlier candidate wins
    out = torch.empty((5, 61), device="cuda")
    chosen = torch.empty(5, dtype=torch.int32, device="cuda")
    B_.hr_select_best(torch.as_tensor(cand, device="cuda"), torch.as_tensor(losses, device="cuda"), out, chosen)
    k = np.argmin(losses, axis=0)
    assert (chosen.cpu().numpy() == k).all() and k[1] == 0
    assert np.array_equal(out.cpu().numpy(), cand[k, np.arange(5)])
    img = torch.zeros(1 << 20, device="cuda")
    B_.hr_add_noise(img, 0.01, 1234)
    x = img.cpu().numpy().astype(np.float64)
    assert abs(x.mean()) < 4 * 0.01 / 1024 and abs(x.std() - 0.01) < 0.01 * 0.01
