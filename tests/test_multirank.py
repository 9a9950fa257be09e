"""The multi-rank path of bench.py on CPU: two gloo ranks launched like torchrun's
(RANK / WORLD_SIZE / MASTER_* in the environment, rendezvous on 127.0.0.1).  Each
rank gets its own hand instance and sample-stream field (weak scaling, no data
crossing ranks), the timings are the slowest rank's, every rank agrees on them, the
whole-job value counts every rank's units, and the reference arm leaves ranks other
than 0 without work."""
import json
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    from paper_2107_05509_gb300 import inputs as I
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.env_rank()
        seed, field = bench.rank_instance(1000, r)
        x = I.gt_params(seed)
        step_ms, e2e_ms = 1.0 + 0.5 * r, 3.0 - r          # each rank its own timings
        red = bench.reduce_max([step_ms, e2e_ms], dist, "cpu")

        class Args:
            steps, warmup = 1, 0
        ref_line = bench.run_reference(Args) if r != 0 else "rank 0 not run here"
        with open(out, "w") as f:
            json.dump({"rank": r, "world": w, "local": local, "seed": seed, "field": field, "x": x.tolist(),
                       "red": red, "ref": ref_line}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.distributed.is_available():
        pytest.skip("torch.distributed unavailable")
    import bench
    port = _free_port()
    ctx = mp.get_context("spawn")
    outs = [str(tmp_path / f"rank{r}.json") for r in range(2)]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, outs[r])) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = [json.load(open(o)) for o in outs]
    assert [q["rank"] for q in res] == [0, 1] and all(q["world"] == 2 for q in res)
    assert [q["local"] for q in res] == [0, 1]
    # distinct instances and sample streams per rank
    assert res[0]["seed"] != res[1]["seed"] and res[0]["field"] != res[1]["field"]
    assert not np.allclose(res[0]["x"], res[1]["x"])
    # every rank holds the slowest rank's timings
    assert res[0]["red"] == res[1]["red"] == [1.5, 3.0]
    # the reference arm: ranks other than 0 return without work
    assert res[1]["ref"] is None
    # whole-job value: both ranks' units over the slowest step
    assert abs(bench.job_value(2.0e6, 2, 1.5) - 2.0 * 2 / 1.5e-3) < 1e-9
