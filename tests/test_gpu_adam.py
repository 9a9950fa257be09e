"""The Adam step on the GPU (Section 3.3: the parameters are optimised with Adam)
against the oracle's float64 Adam, element by element over several steps, for every
entry point that takes one: hr_adam_step (host step count), hr_adam_step_dev (device
step counter; one block for short vectors, a grid-stride launch plus a separate
counter advance for long ones; per-entry step sizes repeated or full-length), the
full objective's per-entry step vectors, and the proposal network's hr_net_adam.

Tolerance, from the arithmetic: the kernels take beta1, beta2, eps and lr as float32
(the oracle is given the same float32 values) and evaluate the bias corrections
1 - beta^t with powf, whose few-ulp error near 1 becomes a relative error of up to
~1e-4 in 1 - beta2^t = 0.002 at t = 2 (sqrt halves it in the step); the moments
carry a few ulp per step.  Per step and entry the move therefore agrees to
2e-4 lr_i (plus the float32 rounding of the parameter itself), and the moments to
1e-6 relative with a floor at the gradient's scale.  A wrong bias correction, a
swapped beta or a misindexed step size moves a parameter by O(lr_i) and fails."""
import numpy as np
import pytest

import oracle
from tests.gpu_common import require_gpu, torch

pytestmark = pytest.mark.gpu

F32 = lambda x: float(np.float32(x))
B1, B2, EPS = F32(0.9), F32(0.999), F32(1e-8)


@pytest.fixture(scope="module")
def B():
    require_gpu()
    from paper_2107_05509_gb300 import binding
    return binding


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def _grads(rng, n, steps):
    """Gradients spanning six decades, some entries exactly zero at every step."""
    mag = 10.0 ** rng.uniform(-3, 3, n)
    zero = rng.random(n) < 0.02
    out = []
    for _ in range(steps):
        g = (rng.normal(size=n) * mag).astype(np.float32)
        g[zero] = 0.0
        out.append(g)
    return out


def _check(p_gpu, m_gpu, v_gpu, p, m, v, lr_i, t, g_scale):
    """Cumulative bound after t steps (see the module docstring)."""
    tol_p = t * (2e-4 * lr_i + 2.0 ** -23 * np.abs(p))
    bad = np.abs(p_gpu - p) > tol_p
    assert not bad.any(), f"step {t}: {bad.sum()} params off, worst {np.abs(p_gpu - p)[bad].max():.3g}"
    assert np.all(np.abs(m_gpu - m) <= t * 1e-6 * (np.abs(m) + (1 - B1) * g_scale))
    assert np.all(np.abs(v_gpu - v) <= t * 1e-6 * (np.abs(v) + (1 - B2) * g_scale ** 2))


def _run_both(B, n, steps, lr, scale, dev_counter, seed):
    rng = np.random.default_rng(seed)
    p0 = rng.normal(size=n).astype(np.float32)
    grads = _grads(rng, n, steps)
    g_scale = np.max([np.abs(g) for g in grads], axis=0).astype(np.float64)
    pt, mt, vt = _t(p0), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    counter = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = None if scale is None else _t(scale)
    p, m, v = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    sc = None if scale is None else np.asarray(scale, np.float32).astype(np.float64)
    lr_i = np.full(n, F32(lr)) if sc is None else F32(lr) * sc[np.arange(n) % sc.size]
    for t, g in enumerate(grads, start=1):
        gt = _t(g)
        if dev_counter:
            B.hr_adam_step_dev(pt, gt, mt, vt, F32(lr), B1, B2, EPS, counter, lr_scale=st)
        else:
            B.hr_adam_step(pt, gt, mt, vt, F32(lr), B1, B2, EPS, t)
        p, m, v = oracle.adam_step(p, g, m, v, t, F32(lr), B1, B2, EPS, lr_scale=sc)
        torch.cuda.synchronize()
        _check(pt.cpu().numpy(), mt.cpu().numpy(), vt.cpu().numpy(), p, m, v, lr_i, t, g_scale)
        if dev_counter:
            assert int(counter.item()) == t
    # entries whose gradient was always zero never move
    zero = np.all([g == 0 for g in grads], axis=0)
    assert zero.any() and np.array_equal(pt.cpu().numpy()[zero], p0[zero])


@pytest.mark.parametrize("n", [61, 786757])
def test_adam_step_host_count_against_oracle(B, n):
    _run_both(B, n, steps=5, lr=0.01, scale=None, dev_counter=False, seed=1)


@pytest.mark.parametrize("n", [61, 4096, 4097, 786757])   # one block up to 4096 entries, then the grid path
def test_adam_step_dev_against_oracle(B, n):
    _run_both(B, n, steps=5, lr=0.01, scale=None, dev_counter=True, seed=2)


@pytest.mark.parametrize("n", [61, 61 * 64])
def test_adam_step_dev_group_steps_repeated_per_instance(B, n):
    # a batch's parameters [n / 61][61] share the per-group steps of one instance
    from paper_2107_05509_gb300 import pipeline as P
    scale = P.lr_scale_vector(device="cpu").numpy()
    assert scale.size == 61
    _run_both(B, n, steps=4, lr=1.0, scale=scale, dev_counter=True, seed=3)


def test_adam_step_dev_full_objective_step_vectors(B):
    """The warm-up and main phases' full-length per-entry step vectors (zeros for the
    entries a phase keeps fixed) on the 786,757-entry parameter vector of the paper
    workload's full objective, as the refiner builds them."""
    from paper_2107_05509_gb300 import inputs as I
    from paper_2107_05509_gb300 import pipeline as P
    from tests.gpu_common import hand
    cfg = I.PAPER
    N, H, W = cfg.views, cfg.height, cfg.width
    model = B.Model(hand())
    views = P.Views(cams=torch.zeros((N, 20), device="cuda"), background=torch.zeros((N, H, W, 3), device="cuda"),
                    observed=torch.zeros((N, H, W, 3), device="cuda"),
                    mask=torch.zeros((N, H, W), dtype=torch.uint8, device="cuda"), H=H, W=W)
    ref = P.PaperRefiner(model, views, cfg, edge_weight=0.0)
    assert ref.n == 786757
    for name, vec in (("warm", ref.scale_warm), ("main", ref.scale_main)):
        s = vec.cpu().numpy()
        assert s.size == ref.n and (s == 0).any() == (name == "warm")
        _run_both(B, ref.n, steps=3, lr=1.0, scale=s, dev_counter=True, seed=4)
    ref.ctx.close()


def test_net_adam_against_oracle(B):
    """hr_net_adam over the proposal network's 1.02 M float32 master weights: each
    step's gradient comes from a forward and backward of the network; the oracle
    steps the same weights with the same gradients and tracks the moments."""
    from tests.test_gpu_net import _case
    Bn, nv = 1, 4     # B * views a multiple of 4 (hr_net_create)
    p0, X, cams = _case(Bn, nv, seed=12)
    net = B.Net(Bn, nv)
    net.set_params(_t(p0))
    net.set_inputs_bf16(_t(X).to(torch.bfloat16))
    ct = _t(cams)
    out = torch.empty((Bn, 61), device="cuda")
    rng = np.random.default_rng(6)
    P = net.P
    p, m, v = p0.astype(np.float64), np.zeros(P), np.zeros(P)
    g_scale = np.zeros(P)
    lr = F32(1e-3)
    for t in range(1, 5):
        net.forward(ct, out)
        net.backward(_t(rng.normal(size=(Bn, 61))))
        gt = torch.empty(P, device="cuda")
        pt = torch.empty(P, device="cuda")
        net.get_params(params=pt, grads=gt)
        g = gt.cpu().numpy()
        g_scale = np.maximum(g_scale, np.abs(g))
        # the weights the step starts from are the oracle's previous result
        assert np.abs(pt.cpu().numpy() - p).max() <= t * (2e-4 * lr) + 1e-6
        net.adam(lr, t, B1, B2, EPS)
        p, m, v = oracle.adam_step(p, g, m, v, t, lr, B1, B2, EPS)
        q = torch.empty(P, device="cuda")
        net.get_params(params=q)
        got = q.cpu().numpy()
        tol = t * (2e-4 * lr + 2.0 ** -23 * np.abs(p))
        bad = np.abs(got - p) > tol
        assert not bad.any(), f"step {t}: {bad.sum()} weights off"
    assert net.status() == B.HR_OK
    net.close()
