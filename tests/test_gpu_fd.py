"""End-to-end gradient check of one refinement iteration on the GPU: the analytic
dL/dparams (interior + edge-sampling + vertex-normal adjoint, then the skinning
adjoint) against central finite differences of the loss, h = 1e-4, on 20 random
parameters of the paper-shaped workload (8 views 512x384).

The Monte Carlo estimator is piecewise constant in the parameters for fixed
samples, so both sides are random: for each of S sample seeds the finite difference
uses common random numbers (the same seed at x + h e_k and x - h e_k) and the
analytic gradient uses the same seed at x.  The seed means must agree within three
standard errors plus 2 % of the gradient's scale.
"""
import numpy as np
import pytest

from tests.gpu_common import hand, require_gpu, torch

pytestmark = pytest.mark.gpu


def test_param_gradient_matches_central_fd():
    require_gpu()
    from paper_2107_05509_gb300 import binding as B
    from paper_2107_05509_gb300 import inputs as I
    from paper_2107_05509_gb300 import pipeline as P
    cfg = I.PAPER
    h = hand()
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, cfg.views, cfg.width, cfg.height)
    x_gt = I.gt_params(cfg.seed)
    views, _ = P.make_views(cfg, model, x_gt, ctx=ctx)
    x0 = I.perturb_params(x_gt, cfg.seed).astype(np.float64)
    rng = np.random.default_rng(20)
    idx = np.sort(rng.choice(61, size=20, replace=False))
    hstep = 1e-4
    seeds = 24
    fd = np.zeros((seeds, len(idx)))
    an = np.zeros((seeds, len(idx)))
    for si in range(seeds):
        opts = P.opts_for(cfg, spp=16, seed=5000 + si)
        opts.edge_samples = 16384
        ref = P.Refiner(model, views, opts, ctx=ctx)
        p = torch.as_tensor(x0.astype(np.float32), device="cuda")
        _, g = ref.step(p)
        an[si] = g.cpu().numpy()[idx]
        for j, k in enumerate(idx):
            xp, xm = x0.copy(), x0.copy()
            xp[k] += hstep
            xm[k] -= hstep
            lp = float(ref.forward(torch.as_tensor(xp.astype(np.float32), device="cuda")).item())
            lm = float(ref.forward(torch.as_tensor(xm.astype(np.float32), device="cuda")).item())
            # the step actually taken in float32
            step = float(np.float32(xp[k])) - float(np.float32(xm[k]))
            fd[si, j] = (lp - lm) / step
    assert B.hr_get_status(ctx) == B.HR_OK
    m_fd, m_an = fd.mean(0), an.mean(0)
    se = np.sqrt(fd.var(0, ddof=1) / seeds + an.var(0, ddof=1) / seeds)
    scale = np.abs(m_an).max()
    tol = 3.0 * se + 0.02 * np.maximum(np.abs(m_an), 0.05 * scale)
    bad = np.abs(m_fd - m_an) > tol
    assert scale > 0
    assert not bad.any(), list(zip(idx[bad], m_fd[bad], m_an[bad], se[bad]))
    # the check has power: the gradient is resolved well above its noise for most entries
    assert (np.abs(m_an) > 3 * se).sum() >= 10
