"""The allocation-free skinning adjoint (hr_skin_bwd_noalloc) against the context
entry point (hr_skin_bwd) through the C ABI.

hr_skin_bwd_noalloc exists for callers that cannot let a library allocate device
memory (applications that own every device allocation through their own pool,
processes under a fixed device-memory quota, latency-bound loops that cannot take
cudaMalloc's implicit synchronisation); its scratch is a static device array in the
library, shared by all calls.  This file is collected last so that a failure here
leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

from tests.gpu_common import hand, require_gpu, torch

pytestmark = pytest.mark.gpu


def test_noalloc_skin_bwd_matches_context_entry_point_twice():
    require_gpu()
    from paper_2107_05509_gb300 import binding as B
    from paper_2107_05509_gb300 import inputs as I
    h = hand()
    model = B.Model(h)
    ctx = B.Context(h.V, h.F, h.E, 1, 8, 8)
    rng = np.random.default_rng(17)
    # two calls in a row with different inputs: the shared scratch must not leak
    # anything from one call into the next
    for trial, x in enumerate((I.perturb_params(I.gt_params(3), 3), np.zeros(61, np.float32))):
        dV = rng.normal(0, 1, (h.V, 3)).astype(np.float32)
        p = torch.as_tensor(np.ascontiguousarray(x, np.float32), device="cuda")
        g = torch.as_tensor(dV, device="cuda")
        ref = torch.empty(61, device="cuda")
        out = torch.full((61,), float("nan"), device="cuda")
        B.hr_skin_bwd(ctx, model, p, g, ref)
        B.hr_skin_bwd_noalloc(model, p, g, out)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.isfinite(o).all(), trial
        # the same kernel, block count and fixed-order reduction: bit-identical
        assert np.array_equal(o, r), (trial, o, r)
    assert B.hr_get_status(ctx) == B.HR_OK
    ctx.close()


def test_noalloc_rejects_models_beyond_its_scratch():
    require_gpu()
    from paper_2107_05509_gb300 import binding as B
    h = hand()
    model = B.Model(h)
    big = B.hr_model()
    ctypes.pointer(big)[0] = model.struct
    big.V = 16385    # one vertex more than the static scratch serves
    d = torch.zeros(61, device="cuda")
    code = B.lib().hr_skin_bwd_noalloc(ctypes.byref(big), ctypes.c_void_p(d.data_ptr()),
                                       ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()), None)
    assert code == B.HR_ERR_UNSUPPORTED
