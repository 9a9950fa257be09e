"""Benchmark: render forward + backward throughput of one refinement iteration.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl handrt|reference]

Workload: the paper-shaped multiview hand capture -- 8 views of 512x384 on a ring at
0.6 m, 16 samples per pixel, 4096 silhouette-edge samples per view, the 778-vertex /
1538-triangle procedural hand (Section 3.3 times one iteration of this path: ~30 views,
16 spp forward and backward).  One step = one full iteration of the hot path:
skinning, BVH (rebuilt every 8th iteration, refitted in between) + vertex normals,
forward render, masked loss + adjoint, interior and edge-sampling backward with the
vertex-normal adjoint, skinning adjoint, Adam.

value: estimator samples resolved per second -- forward: every pixel sample of every
view (N x H x W x spp); backward: every sample of the pixels with a non-zero adjoint;
edges: the two rays of each edge sample that lands on such a pixel -- counted by the
library's HR_STATS pass.  The count is a property of the workload, not of how the
renderer finds each sample's closest hit (a sub-tile whose frustum misses the scene
resolves its samples without tracing them one by one; the counters report both).
Device-timed with CUDA events, inputs resident in HBM, L2 flushed between steps.  e2e:
the same rays per step through the public Python API (StreamedRefiner: the captured
step, Refiner.capture_step, on two input slots), every step's inputs and sample counter
copied from pinned host memory and its loss and gradient read back, the copy of step
k + 1 overlapping step k; serial_ms_per_step is the same without the overlap.

--impl reference times the CPU oracle (brute force, all host cores) on a bounded
sample of the same workload.  Under torchrun every rank refines its own hand instance
(weak scaling, no collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "render fwd+bwd Mrays/s"
UNIT = "Mrays/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 FMA peak: SMs (read from the device) x 128 FP32 lanes x 2 flop x clock
LANES = 128
# modelled FP32 work: per ray made (jitter, screen point, direction), per BVH node
# visited (two child boxes against a sub-tile frustum or a ray), per candidate
# screen-box test, per Moller-Trumbore test, per shaded hit (forward) or
# differentiated hit (backward)
FLOP_RAY, FLOP_NODE, FLOP_CAND, FLOP_TRI, FLOP_HIT, FLOP_HIT_GRAD = 40, 60, 4, 50, 60, 250
S_SAMPLES, S_RAYS, S_NODES, S_TRIS, S_HITS, S_CANDS = range(6)
FLOP_TRACE_NODE, FLOP_EDGE = 40, 120   # per-ray traversal node (two slab tests); edge-sample set-up
KERNEL_NAMES = {"fwd_gather": "k_bin_*", "fwd_shade": "k_shade_fwd", "bwd_gather": "k_items_bwd",
                "bwd_shade": "k_shade_bwd", "edge_samples": "k_edge_samples"}
# DRAM bytes (read + write) per launch from the ncu capture summarised under profiles/,
# with the hash of the render kernels' sources at that capture: a kernel whose source
# has changed since reports no traffic
NCU_TRAFFIC = {"k_shade_bwd": (4941824, "369d3913b55475c9"), "k_shade_fwd": (2931712, "369d3913b55475c9"),
               "k_edge_samples": (2455040, "369d3913b55475c9")}
NCU_TRAFFIC_SOURCES = ("paper_2107_05509_gb300/csrc/hr_render.cu", "paper_2107_05509_gb300/csrc/hr_device.cuh")


def render_source_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in NCU_TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """(bytes per launch, note) of the committed capture, or (None, why)."""
    rec = NCU_TRAFFIC.get(kernel)
    if rec is None:
        return None, "no capture of this kernel"
    nbytes, src = rec
    if src != render_source_hash():
        return None, "the kernel source changed since the capture"
    return nbytes, f"ncu dram__bytes_read.sum + dram__bytes_write.sum, sources {src}"
# kernels of one step: skin 1, BVH + normals 2, forward 7 (bin count, bin alloc,
# background, bin fill, bin sort, shade, overflow), loss 2, backward 8 (items, shade,
# overflow, reduce, silhouettes, edge samples, normal adjoint 2), skin adjoint 1, Adam 1
LAUNCHES_PER_STEP = 22
# a batched iteration: the same kernels (one launch each over all instances), the
# vertex-error kernel and the active-instance layout before the forward and backward
LAUNCHES_BATCH_ITER = 25


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def rank_instance(seed, rank):
    """Weak scaling: rank r refines its own hand instance, seeded seed + r, with Philox
    instance field r (independent sample streams); no data crosses ranks."""
    return seed + rank, rank


def reduce_max(values, dist, device):
    """The slowest rank's value of each entry (a MAX all-reduce when ranks exist)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_value(units_per_rank_step, world, ms_per_step):
    """Whole-job throughput in millions of units per second: the units all ranks
    processed in a step over the slowest rank's step time."""
    return units_per_rank_step * world / (ms_per_step * 1e-3) / 1e6


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"sm_max_mhz": 2070.0, "clocks_under_load": {"sm_mhz_median": 1492.0}}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for k, n in enumerate(names):
                if p[5 + k].lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def run_handrt(args):
    import torch

    from paper_2107_05509_gb300 import binding as B
    from paper_2107_05509_gb300 import inputs as I
    from paper_2107_05509_gb300 import pipeline as P

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    cfg = I.PAPER
    hand = I.make_hand(0)
    model = B.Model(hand, device=dev)
    inst_seed, inst_field = rank_instance(cfg.seed, rank)
    x_gt = I.gt_params(inst_seed)
    N, H, W = cfg.views, cfg.height, cfg.width
    ctx = B.Context(hand.V, hand.F, hand.E, N, W, H)
    views, _ = P.make_views(cfg, model, x_gt, device=dev, ctx=ctx)
    opts = P.opts_for(cfg)
    opts.instance = inst_field
    ref = P.Refiner(model, views, opts, ctx=ctx)
    x0 = torch.as_tensor(I.perturb_params(x_gt, inst_seed), device=dev)
    params = x0.clone()
    m1 = torch.zeros(61, device=dev)
    m2 = torch.zeros(61, device=dev)
    lr = 2e-3

    # work counters of one step (untimed pass)
    opts.flags = B.HR_STATS | B.HR_BWD_REUSE_FWD
    ref.step(params)
    stats = B.hr_get_stats(ctx).astype(np.float64)
    opts.flags = B.HR_BWD_REUSE_FWD
    rays_fwd, rays_bwd, rays_edge = stats[0, S_SAMPLES], stats[1, S_SAMPLES], stats[2, S_SAMPLES]
    rays_step = rays_fwd + rays_bwd + rays_edge

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    stages = ["skin", "bvh", "fwd", "loss", "bwd", "skin_bwd", "adam"]

    def one_step(step_idx, evs=None):
        def mark(i):
            if evs is not None:
                evs[i].record(stream)
        opts.iter = step_idx
        mark(0)
        B.hr_skin(ctx, model, params, ref.verts)
        mark(1)
        B.hr_build_bvh(ctx, model, ref.verts)
        mark(2)
        B.hr_render_fwd(ctx, model, ref.verts, views.cams, H, W, views.background, opts, ref.image)
        mark(3)
        B.hr_loss(ctx, ref.image, views.observed, views.mask, ref.loss, ref.adjoint)
        mark(4)
        B.hr_render_bwd(ctx, model, ref.verts, views.cams, H, W, views.background, opts, ref.adjoint, ref.d_verts)
        mark(5)
        B.hr_skin_bwd(ctx, model, params, ref.d_verts, ref.d_params)
        mark(6)
        B.hr_adam_step(params, ref.d_params, m1, m2, lr, 0.9, 0.999, 1e-8, step_idx + 1)
        mark(7)

    for w in range(args.warmup):
        one_step(w)
    torch.cuda.synchronize()

    # launch shapes of the render kernels for this workload (the project's autotuner;
    # untimed, before the graph is captured)
    tune_params = params.clone()
    tuning, tune_start_ms, tune_best_ms = P.autotune(
        ctx, lambda: ref.step(tune_params), P.workload_key(model, [(N, W, H, cfg.spp, cfg.edge_samples)]),
        cache=False)

    # the timed step: one whole iteration captured as a CUDA graph and replayed; the
    # sample streams and Adam's step number come from a device counter that the
    # Adam kernel advances, so every replay is a fresh iteration
    iter_dev = torch.full((1,), args.warmup, dtype=torch.int32, device=dev)
    gopts = P.opts_for(cfg, iter_dev=iter_dev)
    gopts.instance = rank

    def graph_step():
        B.hr_skin(ctx, model, params, ref.verts)
        B.hr_update_bvh(ctx, model, ref.verts, iter_dev, P.REBUILD_EVERY)
        B.hr_render_fwd(ctx, model, ref.verts, views.cams, H, W, views.background, gopts, ref.image)
        B.hr_loss(ctx, ref.image, views.observed, views.mask, ref.loss, ref.adjoint)
        B.hr_render_bwd(ctx, model, ref.verts, views.cams, H, W, views.background, gopts, ref.adjoint, ref.d_verts)
        B.hr_skin_bwd(ctx, model, params, ref.d_verts, ref.d_params)
        B.hr_adam_step_dev(params, ref.d_params, m1, m2, lr, 0.9, 0.999, 1e-8, iter_dev)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        graph_step()                     # one eager run on the capture stream first
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        graph_step()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        # the same replays for ~0.5 s before the timed region: the sampler starts and
        # records the clocks under this load (the timed region itself lasts only
        # steps x ~0.5 ms)
        t_end = time.time() + 0.5
        while time.time() < t_end:
            for _ in range(50):
                graph.replay()
            torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))        # evict L2 between timed steps (outside the events)
            ev[k][0].record(stream)
            graph.replay()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    ms_per_step = float(step_ms.mean())
    tot_ms = float(step_ms.sum())

    # stage breakdown (eager launches, events between the C-ABI calls; diagnostic)
    n_st = max(1, min(args.steps, 50))
    sev = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(n_st)]
    for k in range(n_st):
        flush.fill_(float(k))
        one_step(args.warmup + k, sev[k])
    torch.cuda.synchronize()
    st = np.array([[sev[k][i].elapsed_time(sev[k][i + 1]) for i in range(7)] for k in range(n_st)])
    status = B.hr_get_status(ctx)
    if status != B.HR_OK:
        raise RuntimeError(f"device status {B.status_string(status)}")

    # per-kernel device times: a second timed pass with CUDA events recorded by the
    # library between its internal kernels (HR_TIMING), L2 flushed between steps
    ktimes = {k: [] for k in B.KERNEL_TIMES}
    opts.flags = B.HR_TIMING | B.HR_BWD_REUSE_FWD
    n_kt = max(1, min(args.steps, 50))
    for k in range(n_kt):
        flush.fill_(float(k))
        one_step(args.warmup + args.steps + k)
        for name, ms in B.hr_kernel_times(ctx).items():
            if ms >= 0:
                ktimes[name].append(ms)
    opts.flags = B.HR_BWD_REUSE_FWD
    kt_mean = {k: float(np.mean(v)) for k, v in ktimes.items() if v}

    # end-to-end through the public API with host buffers
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()
    h_obs, h_mask, h_bg = pin(views.observed.cpu()), pin(views.mask.cpu()), pin(views.background.cpu())
    h_cams, h_x = pin(views.cams.cpu()), pin(x0.cpu())
    h_loss, h_grad = torch.empty(1).pin_memory(), torch.empty(61).pin_memory()
    e2e_views = P.Views(cams=torch.empty_like(views.cams), background=torch.empty_like(views.background),
                        observed=torch.empty_like(views.observed), mask=torch.empty_like(views.mask), H=H, W=W)
    # the public API's captured step (Refiner.capture_step): every step copies its
    # inputs and the sample-stream counter from pinned host memory, replays the graph
    # and reads the loss and the gradient back, one after another on one stream
    e_iter = torch.zeros(1, dtype=torch.int32, device=dev)
    # one pinned word per step: an asynchronous copy reads its host word when it runs
    h_iters = torch.arange(args.warmup + args.steps + 1, dtype=torch.int32).pin_memory()
    e2e_opts = P.opts_for(cfg, iter_dev=e_iter)
    e2e_opts.instance = inst_field
    e2e_ref = P.Refiner(model, e2e_views, e2e_opts, ctx=ctx)
    e_params = torch.empty(61, device=dev)
    for dst, src in ((e2e_views.observed, h_obs), (e2e_views.mask, h_mask), (e2e_views.background, h_bg),
                     (e2e_views.cams, h_cams), (e_params, h_x)):
        dst.copy_(src)
    e2e_graph = e2e_ref.capture_step(e_params)
    h2d = sum(t.numel() * t.element_size() for t in (h_obs, h_mask, h_bg, h_cams, h_x)) + 4
    d2h = h_loss.numel() * 4 + h_grad.numel() * 4

    def serial_step(i):
        e_iter.copy_(h_iters[i:i + 1], non_blocking=True)
        e2e_views.observed.copy_(h_obs, non_blocking=True)
        e2e_views.mask.copy_(h_mask, non_blocking=True)
        e2e_views.background.copy_(h_bg, non_blocking=True)
        e2e_views.cams.copy_(h_cams, non_blocking=True)
        e_params.copy_(h_x, non_blocking=True)
        e2e_graph.replay()
        h_loss.copy_(e2e_ref.loss, non_blocking=True)
        h_grad.copy_(e2e_ref.d_params, non_blocking=True)

    # the streamed public API (StreamedRefiner): the same copies, graph and read-back,
    # the copy of step k + 1 overlapping step k (two input slots)
    streamer = P.StreamedRefiner(model, e2e_views, e2e_opts, ctx=ctx, params=e_params)
    frames = [P.HostFrame(observed=h_obs, mask=h_mask, background=h_bg, cams=h_cams, params=h_x,
                          iter=h_iters[i:i + 1]) for i in range(args.warmup + args.steps)]
    h_losses = torch.empty(args.warmup + args.steps).pin_memory()
    h_grads = torch.empty(args.warmup + args.steps, 61).pin_memory()

    def streamed_step(i):
        streamer.submit(frames[i], h_losses[i:i + 1], h_grads[i], stream)

    def time_e2e(step_fn, tail):
        for w in range(args.warmup):
            step_fn(w)
        tail()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        e0.record(stream)
        streamer.order_after(stream)
        for k in range(args.steps):
            step_fn(args.warmup + k)
        tail()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    serial_ms = time_e2e(serial_step, lambda: None)
    e2e_ms = time_e2e(streamed_step, lambda: streamer.join(stream))
    opts.iter = 0

    if dist:
        tot_ms, e2e_ms, serial_ms = reduce_max([tot_ms, e2e_ms, serial_ms], dist, dev)
        ms_per_step = tot_ms / args.steps
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return None

    value = job_value(rays_step, world, ms_per_step)
    stage_ms = dict(zip(stages, st.mean(0).round(4).tolist()))
    pk, pk_kind = peaks()
    clocks = clk.summary()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = n_sm * LANES * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    fwd_row, bwd_row, edge_row = stats
    kflops = {
        "fwd_gather": FLOP_NODE * fwd_row[S_NODES],
        "fwd_shade": (FLOP_RAY * fwd_row[S_RAYS] + FLOP_CAND * fwd_row[S_CANDS] + FLOP_TRI * fwd_row[S_TRIS] +
                      FLOP_HIT * fwd_row[S_HITS]),
        "bwd_gather": FLOP_NODE * bwd_row[S_NODES],
        "bwd_shade": (FLOP_RAY * bwd_row[S_RAYS] + FLOP_CAND * bwd_row[S_CANDS] + FLOP_TRI * bwd_row[S_TRIS] +
                      FLOP_HIT_GRAD * bwd_row[S_HITS]),
        "edge_samples": (FLOP_RAY * edge_row[S_RAYS] + FLOP_TRACE_NODE * edge_row[S_NODES] +
                         FLOP_TRI * edge_row[S_TRIS] + FLOP_HIT * edge_row[S_HITS] + FLOP_EDGE * edge_row[S_RAYS] / 2),
    }
    dom = max((k for k in kflops if k in kt_mean), key=lambda k: kt_mean[k])
    achieved = kflops[dom] / (kt_mean[dom] * 1e-3) / 1e12
    kernel_name = KERNEL_NAMES[dom]
    traffic, traffic_note = ncu_traffic(kernel_name)
    roof = {"bound": "alu", "kernel": kernel_name, "achieved": round(achieved, 3), "peak": round(fp32_peak, 2),
            "unit": "TFLOP/s", "frac": round(achieved / fp32_peak, 4), "traffic": traffic,
            "traffic_note": traffic_note,
            "launch_ms": round(kt_mean[dom], 4), "flops_per_launch": float(kflops[dom]),
            "peak_note": f"FP32 FMA peak: {n_sm} SMs (cudaDevAttrMultiProcessorCount) x {LANES} lanes x 2 flop x "
                         f"{pk.get('sm_max_mhz', 2070.0):.0f} MHz (max SM clock, {pk_kind} clock data)",
            "flop_model": f"{FLOP_RAY}/ray made + {FLOP_CAND}/candidate box test + {FLOP_TRI}/Moller-Trumbore "
                          f"test + {FLOP_HIT}/shaded hit or {FLOP_HIT_GRAD}/differentiated hit; "
                          f"{FLOP_NODE}/frustum node visit",
            "kernel_ms": {k: round(v, 4) for k, v in kt_mean.items()},
            "frac_at_load_clock": None}
    if clocks:
        roof["frac_at_load_clock"] = round(achieved / (n_sm * LANES * 2 * clocks["sm_mhz"] * 1e6 / 1e12), 4)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded procedural hand, GPU-rendered observations)",
        "config": {"workload": cfg.name, "views": N, "width": W, "height": H, "spp": cfg.spp,
                   "edge_samples_per_view": cfg.edge_samples, "vertices": hand.V, "triangles": hand.F,
                   "rays_per_step": int(rays_step), "rays_fwd": int(rays_fwd), "rays_bwd": int(rays_bwd),
                   "rays_edge": int(rays_edge),
                   "work_counters": {k: {n: int(v) for n, v in zip(
                       ["samples", "rays", "bvh_nodes", "mt_tests", "hits", "cand_box_tests"], stats[i])}
                       for i, k in enumerate(["fwd", "bwd", "edge"])},
                   "stage_ms_eager": stage_ms, "step_ms_eager": round(float(st.sum(1).mean()), 4),
                   "timing": "CUDA graph of one whole iteration, replayed; events around each replay",
                   "tuning": tuning, "tuning_fwd_bwd_ms": {"default": round(tune_start_ms, 4),
                                                            "tuned": round(tune_best_ms, 4)},
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"{world} independent instance(s), one per GPU"},
        "e2e": {"value": round(job_value(rays_step, world, e2e_ms), 3), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_ms, 4),
                "api": "StreamedRefiner (copy of step k+1 overlaps step k): the public Python API; the C-ABI "
                       "calls take device pointers, the host copies are pinned-memory torch copies on a copy stream",
                "serial_ms_per_step": round(serial_ms, 4)},
        "gpu_launches": LAUNCHES_PER_STEP * args.steps,
        "roofline": roof,
        "clocks": clocks,
    }
    if clocks:
        clocks["window"] = "0.5 s of the same graph replays right before the timed region, then the timed region"
    if not args.no_refine and world == 1:
        line["paper_refinement"] = run_paper_refinement(dev)
        line["refinement"] = run_refinement(args, dev)
        line["tensor"] = run_tensor(dev)
        line["scale"] = run_scale(dev)
        line["paper_objective"] = run_paper_objective(dev)
        line["edge_term"] = run_edge_term(dev)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, budget_s=args.cpu_seconds)
    if dist:
        dist.destroy_process_group()
    return line


def _first_at_or_below(err_mm, thr=1.0):
    """first iteration whose error is <= thr (-1 if none)"""
    ok = np.nonzero(err_mm <= thr)[0]
    return int(ok[0]) if ok.size else -1


def refine_compare(cfgs, model, dev, iters, learned=None, proposal_steps=3, texture=None, proposal_layout="rig"):
    """Refine the instances of `cfgs` from the same initial estimates with the same
    sample streams: plain per-instance refinement through the single-instance calls,
    instance after instance (one CUDA graph each); all instances together through the
    batch calls (one CUDA graph per iteration); and, with `learned` parameters, the
    batch preceded by the learned proposal steps (proposal_layout "rig": computed on
    the proposal rig's views -- the instances' own views when they are the rig's, else
    the rig's cameras among them at reduced resolution; "ring": the ring network on
    each instance's views view_slots(k) area-resampled to 256 x 256).  The mean vertex
    error epsilon_v (Section 4.1) is recorded on the device every iteration.  texture:
    the model's albedo texture."""
    import torch

    from paper_2107_05509_gb300 import binding as B
    from paper_2107_05509_gb300 import inputs as I
    from paper_2107_05509_gb300 import pipeline as P

    n = len(cfgs)
    hand = model.hand
    x_gt = [I.gt_params(c.seed) for c in cfgs]
    x0 = torch.as_tensor(np.stack([I.perturb_params(x, c.seed) for x, c in zip(x_gt, cfgs)]), device=dev)
    views = P.make_batch_views(cfgs, model, x_gt, device=dev, texture=texture)
    bt = B.Batch(hand.V, hand.F, hand.E, [(c.views, c.width, c.height, c.spp, c.edge_samples, i)
                                          for i, c in enumerate(cfgs)])
    ref = torch.empty((n, hand.V, 3), device=dev)
    B.hr_skin_batch(bt, model, torch.as_tensor(np.stack(x_gt), device=dev), ref)
    R = P.BatchRefiner(model, bt, views, ref_verts=ref, max_iters=iters + 8, device=dev, texture=texture)
    # the same batch with converged instances retired on the device (the per-instance
    # criterion: an instance leaves the batch once its epsilon_v is <= 1 mm)
    Rr = P.BatchRefiner(model, bt, views, ref_verts=ref, max_iters=iters + 8, device=dev, retire="converged",
                        texture=texture)

    # work counters of one batched iteration
    R.reset(x0)
    R.opts.flags = B.HR_STATS | B.HR_BWD_REUSE_FWD
    R.iteration()
    stats = B.hr_get_stats(bt).astype(np.float64)
    R.opts.flags = B.HR_BWD_REUSE_FWD
    rays = float(stats[:, S_SAMPLES].sum())

    # launch shapes: the batch context and every plain context tuned by the same
    # autotuner (instances of one layout share the result)
    memo = {}

    def tune(ctx, run, layout):
        key = P.workload_key(model, layout)
        if key in memo:
            ctx.set_tuning(**memo[key])
        else:
            memo[key] = P.autotune(ctx, run, key, cache=False)[0]

    R.reset(x0)
    tune(bt, R.render_pass, [(c.views, c.width, c.height, c.spp, c.edge_samples) for c in cfgs])
    Rr.reset(x0)
    g_r = Rr.capture()
    R.reset(x0)
    g = R.capture()
    for _ in range(3):
        g.replay()

    def run_batch(pre=None, refiner=None, graph=None):
        refiner, graph = refiner or R, graph or g
        refiner.reset(x0)
        torch.cuda.synchronize()
        pre_ms = 0.0
        if pre is not None:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            pre()
            e1.record()
            torch.cuda.synchronize()
            pre_ms = e0.elapsed_time(e1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(iters + 1)]
        ev[0].record()
        for k in range(iters):
            graph.replay()
            ev[k + 1].record()
        torch.cuda.synchronize()
        dt = np.array([ev[k].elapsed_time(ev[k + 1]) for k in range(iters)])
        err = refiner.err[:iters].cpu().numpy() * 1e3
        status = B.hr_get_status(bt)
        if status != B.HR_OK:
            raise RuntimeError(f"batch device status {B.status_string(status)}")
        return err, dt, pre_ms

    err_b, dt_b, _ = run_batch()
    err_r, dt_r, _ = run_batch(refiner=Rr, graph=g_r)
    res_learned = res_learned_r = None
    if learned is not None:
        from paper_2107_05509_gb300 import proposal as PR
        rig_layout = proposal_layout == "rig" and all(
            (c.views, c.width, c.height) == (PR.RIG.views, PR.RIG.width, PR.RIG.height) for c in cfgs)
        if rig_layout:
            prop = PR.Proposer(R, learned, steps=proposal_steps)

            def propose(refiner):
                prop.r = refiner
                prop.run()
        else:
            # the proposal steps run on the network's views of these instances (a batch
            # of that layout); the refinement continues from the chosen candidates
            make = PR.rig_views if proposal_layout == "rig" else PR.ring_views
            rviews = make(cfgs, views, bt.view_offsets, bt.pixel_offsets)
            rbt = B.Batch(hand.V, hand.F, hand.E, [(PR.SLOTS, PR.NET_SIZE, PR.NET_SIZE, PR.RIG.spp,
                                                    PR.RIG.edge_samples, i) for i in range(n)])
            RR = P.BatchRefiner(model, rbt, rviews, device=dev, texture=texture)
            prop = PR.Proposer(RR, learned, steps=proposal_steps)

            def propose(refiner):
                RR.params.copy_(refiner.params)
                prop.run()
                refiner.params.copy_(RR.params)
        propose(R)                       # warm-up of the network's kernels
        err_l, dt_l, pre_ms = run_batch(lambda: propose(R))
        chosen = prop.chosen.cpu().numpy()
        if prop.net.status() != B.HR_OK:
            raise RuntimeError("proposal network status")
        res_learned = (err_l, dt_l, pre_ms, chosen)
        err_lr, dt_lr, pre_ms_r = run_batch(lambda: propose(Rr), refiner=Rr, graph=g_r)
        res_learned_r = (err_lr, dt_lr, pre_ms_r)

    # plain per-instance refinement, instance after instance
    err_p = np.full((iters, n), np.nan)
    dt_p = np.zeros((iters, n))
    vo, po = bt.view_offsets, bt.pixel_offsets
    for i, c in enumerate(cfgs):
        v1 = P.Views(cams=views.cams[vo[i]:vo[i + 1]].contiguous(),
                     background=views.background[po[i]:po[i + 1]].reshape(c.views, c.height, c.width, 3),
                     observed=views.observed[po[i]:po[i + 1]].reshape(c.views, c.height, c.width, 3),
                     mask=views.mask[po[i]:po[i + 1]].reshape(c.views, c.height, c.width), H=c.height, W=c.width)
        pr = P.PlainRefiner(model, v1, c, instance=i, ref_verts=ref[i], max_iters=iters + 8, device=dev,
                            texture=texture)
        pr.reset(x0[i])
        tune(pr.r.ctx, pr.render_pass, [(c.views, c.width, c.height, c.spp, c.edge_samples)])
        pr.reset(x0[i])
        gi = pr.capture()
        pr.reset(x0[i])
        evi = [torch.cuda.Event(enable_timing=True) for _ in range(iters + 1)]
        evi[0].record()
        for k in range(iters):
            gi.replay()
            evi[k + 1].record()
        torch.cuda.synchronize()
        dt_p[:, i] = [evi[k].elapsed_time(evi[k + 1]) for k in range(iters)]
        err_p[:, i] = pr.err[:iters, 0].cpu().numpy() * 1e3
        if B.hr_get_status(pr.r.ctx) != B.HR_OK:
            raise RuntimeError("plain refinement device status")
        pr.r.ctx.close()

    def summary(err, dt, sequential, pre_ms=0.0):
        mean = err.mean(1)
        k = _first_at_or_below(mean)
        firsts = np.array([_first_at_or_below(err[:, i]) for i in range(err.shape[1])])
        cap = np.where(firsts >= 0, firsts, err.shape[0] - 1)
        out = {"iters_to_mean_1mm": k, "mean_err_mm_at_start": round(float(mean[0]), 3),
               "mean_err_mm_at_end": round(float(mean[-1]), 4),
               "instances_at_or_below_1mm_at_end": int((err[-1] <= 1.0).sum()),
               "instances_never_1mm": int((firsts < 0).sum())}
        # plain: every instance runs its iterations instance after instance (dt [iters][n])
        out["time_to_mean_1mm_ms"] = round(pre_ms + float(dt[:k + 1].sum()), 2) if k >= 0 else None
        if sequential:
            out["time_to_each_1mm_ms"] = round(float(sum(dt[:cap[i] + 1, i].sum() for i in range(err.shape[1]))), 2)
        else:
            out["time_to_each_1mm_ms"] = round(pre_ms + float(dt[:int(cap.max()) + 1].sum()), 2)
        return out

    sb = summary(err_b, dt_b, False)
    sp = summary(err_p, dt_p, True)
    sb["ms_per_iter"] = round(float(np.median(dt_b)), 3)
    sb["value"] = round(rays / (float(np.median(dt_b)) * 1e-3) / 1e6, 1)
    sb["unit"] = UNIT
    sb["rays_per_iter"] = int(rays)
    sb["launches_per_iter"] = LAUNCHES_BATCH_ITER
    sp["ms_per_iter_sum_over_instances"] = round(float(np.median(dt_p.sum(1))), 3)
    sb["tuning"] = bt.get_tuning()
    res = {"instances": n, "views": int(bt.total_views), "pixels": int(bt.total_pixels), "iterations": iters,
           "plain_sequential": sp, "batched": sb}
    # with retirement the batch stops at the last instance's first iteration at or below
    # 1 mm (its iterations get cheaper as instances leave)
    sr = summary(err_r, dt_r, False)
    sr["ms_per_iter_first"] = round(float(dt_r[0]), 3)
    sr["ms_per_iter_last"] = round(float(dt_r[-1]), 3)
    res["batched_retiring"] = sr
    if res_learned is not None:
        err_l, dt_l, pre_ms, chosen = res_learned
        sl = summary(err_l, dt_l, False, pre_ms)
        sl["proposal_steps"] = proposal_steps
        sl["proposal_ms"] = round(pre_ms, 3)
        sl["instances_taking_a_proposal"] = int((chosen > 0).sum())
        res["batched_learned"] = sl
        err_lr, dt_lr, pre_ms_r = res_learned_r
        res["batched_learned_retiring"] = summary(err_lr, dt_lr, False, pre_ms_r)
    for name in ("batched", "batched_learned", "batched_retiring", "batched_learned_retiring"):
        if name in res and res[name]["time_to_mean_1mm_ms"] and sp["time_to_mean_1mm_ms"]:
            res[f"speedup_time_to_mean_1mm_{name}_vs_plain"] = round(
                sp["time_to_mean_1mm_ms"] / res[name]["time_to_mean_1mm_ms"], 3)
        if name in res and res[name]["time_to_each_1mm_ms"] and sp["time_to_each_1mm_ms"]:
            res[f"speedup_time_to_each_1mm_{name}_vs_plain"] = round(
                sp["time_to_each_1mm_ms"] / res[name]["time_to_each_1mm_ms"], 3)
    return res


def run_refinement(args, dev):
    """Time-to-1 mm on three batched workloads: (1) heterogeneous instances (4-16 views
    at 256x256 / 512x384 / 512x512, 8-32 spp): plain per-instance vs batched vs batched
    with the ring network's proposal steps first; (2) the
    learned proposal's rig (8 views at 256x256, 16 spp): plain vs batched vs batched
    with the learned proposal steps first; (3) instances of the scale workload: plain
    vs batched vs batched with the learned proposal steps first.  Each batched pipeline
    also runs with converged instances retired."""
    import torch

    from paper_2107_05509_gb300 import binding as B
    from paper_2107_05509_gb300 import inputs as I
    from paper_2107_05509_gb300 import pipeline as P
    from paper_2107_05509_gb300 import proposal as PR
    import dataclasses

    n, iters = args.batch_instances, args.refine_iters
    hand = I.make_hand(0)
    model = B.Model(hand, device=dev)
    ring, ring_meta = PR.load_weights(PR.WEIGHTS_RING)
    het = refine_compare(I.batch_configs(n), model, dev, iters, learned=ring, proposal_layout="ring")
    het["workload"] = f"batch-{n}x(4-16 views, 256x256|512x384|512x512, 8-32 spp, 4096 edge samples/view)"
    het["proposal"] = ("ring network: each instance's views view_slots(k) (8 of them, spread over its ring, "
                       "repeated when it has fewer) area-resampled to 256x256, intrinsics scaled per axis")
    het["proposal_training"] = {k: ring_meta[k] for k in ("pairs", "steps", "seconds", "layout", "heldout_eps_v_mm")
                                if k in ring_meta}
    rig = [dataclasses.replace(PR.RIG, seed=PR.RIG.seed + 100 + i, name=f"{PR.RIG.name}-{i}") for i in range(n)]
    learned, meta = PR.load_weights()
    lr = refine_compare(rig, model, dev, iters, learned=learned)
    lr["workload"] = f"rig-{n}x(8 views 256x256, 16 spp, 4096 edge samples/view)"
    lr["proposal_training"] = {k: meta[k] for k in ("pairs", "steps", "seconds", "heldout_eps_v_mm") if k in meta}
    # the scale workload (subdivided, textured, 16 x 1024^2 at 64 spp): a handful of
    # instances, plain vs batched vs batched with the learned proposal (on the rig's
    # views among the instances' own, at 256^2)
    sub = I.subdivide_hand(hand, 2)
    smodel = B.Model(sub, device=dev)
    tex = torch.as_tensor(I.texture(I.SCALE.seed, 256), device=dev)
    scfgs = [dataclasses.replace(I.SCALE, seed=I.SCALE.seed + i, name=f"{I.SCALE.name}-{i}")
             for i in range(args.scale_instances)]
    sc = refine_compare(scfgs, smodel, dev, args.scale_iters, learned=learned, texture=tex)
    sc["workload"] = (f"scale-{args.scale_instances}x(16 views 1024x1024, 64 spp, 32768 edge samples/view, "
                      f"12337 V / 24608 F, 256x256 texture)")
    return {"heterogeneous": het, "learned_rig": lr, "scale": sc,
            "adam_lr_per_group": {"shape": P.LR_GROUPS[0], "pose_rad": P.LR_GROUPS[1],
                                  "root_rot_rad": P.LR_GROUPS[2], "trans_m": P.LR_GROUPS[3]},
            "criterion": "time_to_mean_1mm: device time until the mean over instances of epsilon_v <= 1 mm "
                         "(plain: every instance refined that many iterations, one after another); "
                         "time_to_each_1mm: until every instance has been <= 1 mm (plain: per-instance "
                         "stopping), iteration cap counted for instances that never get there"}


def run_paper_refinement(dev, iters=300):
    """The paper-shaped workload refined as a plain Adam loop of 300 iterations from
    the perturbed estimate (each iteration one replay of the captured step, per-group
    step sizes), epsilon_v (Section 4.1) recorded on the device every iteration."""
    import torch

    from paper_2107_05509_gb300 import binding as B
    from paper_2107_05509_gb300 import inputs as I
    from paper_2107_05509_gb300 import pipeline as P

    cfg = I.PAPER
    hand = I.make_hand(0)
    model = B.Model(hand, device=dev)
    x_gt = I.gt_params(cfg.seed)
    views, v_gt = P.make_views(cfg, model, x_gt, device=dev)
    x0 = torch.as_tensor(I.perturb_params(x_gt, cfg.seed), device=dev)
    pr = P.PlainRefiner(model, views, cfg, ref_verts=v_gt, max_iters=iters + 8, device=dev)
    pr.reset(x0)
    g = pr.capture()
    pr.reset(x0)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(iters + 1)]
    ev[0].record()
    for k in range(iters):
        g.replay()
        ev[k + 1].record()
    torch.cuda.synchronize()
    dt = np.array([ev[k].elapsed_time(ev[k + 1]) for k in range(iters)])
    err = pr.err[:iters, 0].cpu().numpy() * 1e3
    if B.hr_get_status(pr.r.ctx) != B.HR_OK:
        raise RuntimeError("paper refinement device status")
    k1 = _first_at_or_below(err)
    pr.r.ctx.close()
    return {"workload": f"{cfg.name}, {iters} Adam iterations from the perturbed estimate",
            "eps_v_mm": {str(i): round(float(err[i]), 4) for i in list(range(0, iters, 25)) + [iters - 1]},
            "iters_to_1mm": k1, "time_to_1mm_ms": round(float(dt[:k1 + 1].sum()), 2) if k1 >= 0 else None,
            "ms_per_iter": round(float(np.median(dt)), 4), "total_ms": round(float(dt.sum()), 2),
            "adam_lr_per_group": {"shape": P.LR_GROUPS[0], "pose_rad": P.LR_GROUPS[1],
                                  "root_rot_rad": P.LR_GROUPS[2], "trans_m": P.LR_GROUPS[3]}}


def run_scale(dev, iters=10):
    """The scale workload: the hand Loop-subdivided twice (12,337 vertices, 24,608
    triangles; multi-block BVH build, float64-atomic backward sums) with a 256 x 256
    RGB albedo texture (bilinear lookup; its gradient is accumulated every iteration),
    16 views of 1024 x 1024, 64 spp, 32768 edge samples per view.  One refinement iteration
    (skinning, BVH update, forward, loss, backward, skinning adjoint, Adam) captured as
    a CUDA graph, replayed `iters` times; inputs (1.2 GB of images) exceed L2."""
    import torch

    from paper_2107_05509_gb300 import binding as B
    from paper_2107_05509_gb300 import inputs as I
    from paper_2107_05509_gb300 import pipeline as P

    cfg = I.SCALE
    hand = I.subdivide_hand(I.make_hand(0), 2)
    model = B.Model(hand, device=dev)
    x_gt = I.gt_params(cfg.seed)
    ctx = B.Context(hand.V, hand.F, hand.E, cfg.views, cfg.width, cfg.height)
    tex = torch.as_tensor(I.texture(cfg.seed, 256), device=dev)
    views, _ = P.make_views(cfg, model, x_gt, device=dev, ctx=ctx, texture=tex)
    ref = torch.empty((hand.V, 3), device=dev)
    B.hr_skin(ctx, model, torch.as_tensor(x_gt, device=dev), ref)
    pr = P.PlainRefiner(model, views, cfg, ctx=ctx, ref_verts=ref, max_iters=iters + 8, device=dev, texture=tex)
    d_tex = torch.zeros_like(tex)
    pr.r.opts.d_texture = d_tex.data_ptr()
    x0 = torch.as_tensor(I.perturb_params(x_gt, cfg.seed), device=dev)
    pr.reset(x0)
    tuning, t0, t1 = P.autotune(ctx, pr.render_pass,
                                P.workload_key(model, [(cfg.views, cfg.width, cfg.height, cfg.spp,
                                                        cfg.edge_samples)]), cache=False)
    pr.r.opts.flags = B.HR_STATS | B.HR_BWD_REUSE_FWD
    pr.render_pass()
    stats = B.hr_get_stats(ctx).astype(np.float64)
    pr.r.opts.flags = B.HR_BWD_REUSE_FWD
    rays = float(stats[:, S_SAMPLES].sum())
    pr.reset(x0)
    g = pr.capture()
    pr.reset(x0)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(iters)]
    for a, b in ev:
        a.record()
        g.replay()
        b.record()
    torch.cuda.synchronize()
    ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
    pr.r.opts.flags = B.HR_TIMING | B.HR_BWD_REUSE_FWD
    pr.render_pass()
    kt = B.hr_kernel_times(ctx)
    pr.r.opts.flags = B.HR_BWD_REUSE_FWD
    status = B.hr_get_status(ctx)
    if status != B.HR_OK:
        raise RuntimeError(f"scale device status {B.status_string(status)}")
    err = pr.err[:iters + 2, 0].cpu().numpy() * 1e3
    ctx.close()
    return {"workload": cfg.name, "vertices": hand.V, "triangles": hand.F, "texture": "256x256 RGB, bilinear",
            "views": cfg.views,
            "width": cfg.width, "height": cfg.height, "spp": cfg.spp, "edge_samples_per_view": cfg.edge_samples,
            "ms_per_iter": round(ms, 3), "rays_per_iter": int(rays), "value": round(rays / (ms * 1e-3) / 1e6, 1),
            "unit": UNIT, "kernel_ms": {k: round(v, 4) for k, v in kt.items() if v >= 0}, "tuning": tuning,
            "eps_v_mm_first_iters": [round(float(e), 3) for e in err[:4]]}


def run_paper_objective(dev):
    """The paper's whole objective and schedule on the paper-shaped workload (8 views
    of 512 x 384, 16 spp, 4096 edge samples per view): data term (colour differences
    and blurred Canny edge maps) with a 3x3 colour transform per camera, colour map
    V = upsample(V_low 8x8) + V_high 512x512 as the hand's texture, joint prior; 50 warm-up iterations (T and V_low only), then 150 of
    everything, each phase one captured CUDA graph.  Observations: the ground truth
    rendered with a 512x512 smooth-noise map, every camera's image through its own
    T_gt = I + N(0, 0.05), plus noise."""
    import torch

    from paper_2107_05509_gb300 import binding as B
    from paper_2107_05509_gb300 import inputs as I
    from paper_2107_05509_gb300 import pipeline as P

    cfg = I.PAPER
    hand = I.make_hand(0)
    model = B.Model(hand, device=dev)
    ctx = B.Context(hand.V, hand.F, hand.E, cfg.views, cfg.width, cfg.height)
    x_gt = I.gt_params(cfg.seed)
    rng = np.random.default_rng(cfg.seed + 3)
    T_gt = np.eye(3)[None] + rng.normal(0.0, 0.05, (cfg.views, 3, 3))
    views = P.make_paper_views(cfg, model, x_gt, I.texture(cfg.seed, 512), T_gt, device=dev, ctx=ctx)
    ref = torch.empty((hand.V, 3), device=dev)
    B.hr_skin(ctx, model, torch.as_tensor(x_gt, device=dev), ref)
    pr = P.PaperRefiner(model, views, cfg, tex_size=512, low_size=8, ref_verts=ref, max_iters=256, ctx=ctx,
                        device=dev)
    x0 = I.perturb_params(x_gt, cfg.seed).astype(np.float32)
    pr.capture()
    pr.reset(x0)
    T_err0 = float(np.abs(pr.T().cpu().numpy().reshape(-1, 3, 3) - T_gt).mean())
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    e[0].record()
    for _ in range(50):
        pr.graphs["warm"].replay()
    e[1].record()
    for _ in range(150):
        pr.graphs["main"].replay()
    e[2].record()
    torch.cuda.synchronize()
    warm_ms, main_ms = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    status = B.hr_get_status(ctx)
    if status != B.HR_OK:
        raise RuntimeError(f"paper-objective device status {B.status_string(status)}")
    err = pr.err[:200, 0].cpu().numpy() * 1e3
    T_err = float(np.abs(pr.T().cpu().numpy().reshape(-1, 3, 3) - T_gt).mean())
    hit = np.nonzero(err <= 1.0)[0]
    ctx.close()
    return {"workload": cfg.name + ", 512x512 colour map, per-camera colour transforms, edge term, joint prior",
            "schedule": "50 warm-up (T, V_low) + 150 full", "params": pr.n,
            "ms_per_iter_warmup": round(warm_ms / 50, 3), "ms_per_iter_full": round(main_ms / 150, 3),
            "schedule_ms": round(warm_ms + main_ms, 1),
            "eps_v_mm": {"start": round(float(err[0]), 3), "after_warmup": round(float(err[50]), 3),
                         "final": round(float(err[-1]), 3)},
            "iters_to_1mm": int(hit[0]) if len(hit) else None,
            "colour_transform_mean_abs_err": {"start": round(T_err0, 4), "final": round(T_err, 4)},
            "loss_final": {"colour": round(float(pr.loss.item()), 6), "edges": round(float(pr.edge_loss.item()), 6),
                           "prior": round(float(pr.prior.item()), 8)}}


def run_edge_term(dev, reps=20):
    """The edge term alone at the paper workload's size (8 views of 512 x 384):
    `hr_edges` (Canny + K of one image stack) and `hr_edge_loss` (the same plus the
    masked loss and the adjoint into the image and the colour transforms), event-timed
    over `reps` calls after 3 warm-up calls.  Images: the background plates with one
    bright disc per view (a silhouette's stand-in), transforms I + N(0, 0.04)."""
    import torch

    from paper_2107_05509_gb300 import binding as B
    from paper_2107_05509_gb300 import inputs as I

    N, H, W, seed = 8, 384, 512, 32
    R = I.background(seed, N, H, W).astype(np.float32)
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    for n in range(N):
        cx, cy, r = W * rng.uniform(0.4, 0.6), H * rng.uniform(0.4, 0.6), min(H, W) * rng.uniform(0.15, 0.3)
        R[n][(x - cx) ** 2 + (y - cy) ** 2 < r * r] = rng.uniform(0.6, 0.95, 3).astype(np.float32)
    obs = I.add_noise(R, seed, 0.01)
    mask = np.zeros((N, H, W), np.uint8)
    mask[:, H // 8:H - H // 8, W // 10:W - W // 10] = 1
    T = (np.eye(3)[None] + rng.normal(0, 0.04, (N, 3, 3))).astype(np.float32).reshape(N, 9)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    ctx = B.Context(8, 8, 8, N, W, H)
    Rt, Ot, Mt, Tt = t(R), t(obs), t(mask), t(T)
    eo = torch.empty((N, H, W), device=dev)
    B.hr_edges(ctx, Ot, eo)
    adj = torch.zeros((N, H, W, 3), device=dev)
    dT = torch.zeros((N, 9), device=dev)
    loss = torch.empty(1, device=dev)
    er = torch.empty((N, H, W), device=dev)
    calls = {"edge_loss": lambda: B.hr_edge_loss(ctx, Rt, eo, Mt, loss, adj, T=Tt, dT=dT),
             "edges": lambda: B.hr_edges(ctx, Rt, er, T=Tt)}
    out = {"workload": "8 x 512x384, plates with one disc per view", "ms": {}}
    for name, fn in calls.items():
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record()
            fn()
            b.record()
        torch.cuda.synchronize()
        out["ms"][name] = round(float(np.median([a.elapsed_time(b) for a, b in ev])), 4)
    status = B.hr_get_status(ctx)
    if status != B.HR_OK:
        raise RuntimeError(f"edge-term device status {B.status_string(status)}")
    ctx.close()
    return out


def run_tensor(dev, steps=20):
    """The bf16 tensor-core GEMM (tcgen05) on the proposal network's largest shapes and
    on a square product, and one training step of the network (B = 128 instances x 8
    views: two batched renders, forward, backward, Adam)."""
    import torch

    from paper_2107_05509_gb300 import binding as B
    from paper_2107_05509_gb300 import inputs as I
    from paper_2107_05509_gb300 import proposal as PR

    pk, pk_kind = peaks()
    ctx = B.Context(8, 8, 8, 1, 8, 8)
    out = {}
    shapes = {"conv1_fwd": (4194304, 32, 128), "conv4_fwd": (65536, 128, 1152), "view_fwd": (1024, 256, 2112),
              "square_8192": (8192, 8192, 8192)}
    g = torch.Generator(device=dev).manual_seed(0)
    for name, (M, N, K) in shapes.items():
        A = torch.randn(M, K, device=dev, generator=g).to(torch.bfloat16)
        Bm = torch.randn(N, K, device=dev, generator=g).to(torch.bfloat16)
        C = torch.empty(M, N, device=dev, dtype=torch.bfloat16)
        for _ in range(3):
            B.hr_gemm_bf16(ctx, A, Bm, C)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            a.record()
            B.hr_gemm_bf16(ctx, A, Bm, C)
            b.record()
        torch.cuda.synchronize()
        ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
        tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
        out[name] = {"M": M, "N": N, "K": K, "ms": round(ms, 4), "TFLOP/s": round(tf, 1)}
        del A, Bm, C
    if B.hr_get_status(ctx) != B.HR_OK:
        raise RuntimeError("gemm status")
    sq = out["square_8192"]
    peak = pk.get("bf16_tflops", 1900.0)
    roof = {"bound": "tensor", "kernel": "k_gemm_bf16<128>", "achieved": sq["TFLOP/s"], "peak": peak,
            "unit": "TFLOP/s", "frac": round(sq["TFLOP/s"] / peak, 4), "traffic": None,
            "peak_note": f"dense bf16, cuBLAS 8192^3 burst ({pk_kind})", "shape": "8192 x 8192 x 8192"}
    # one training step of the proposal network
    hand = I.make_hand(0)
    model = B.Model(hand, device=dev)
    tr = PR.Trainer(model, batch=128, seed=1)
    tr.set_params(PR.init_params(1))
    for _ in range(3):
        tr.step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_st = 10
    e0.record()
    for _ in range(n_st):
        tr.step()
    e1.record()
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / n_st
    ctx.close()
    return {"gemm": out, "roofline_tensor": roof,
            "proposal_train_step": {"instances": 128, "views": 8, "ms": round(step_ms, 3),
                                    "pairs_per_s": round(128 / (step_ms * 1e-3), 1)}}


def _oracle_sample(budget_s):
    """Time the oracle (forward + interior backward + edge samples) on a band of rows
    of the workload, grown until it has run about `budget_s` seconds."""
    import oracle
    from paper_2107_05509_gb300 import inputs as I

    cfg = I.PAPER
    hand = I.make_hand(0)
    x = I.perturb_params(I.gt_params(cfg.seed), cfg.seed)
    verts = oracle.skin(hand, x).astype(np.float32)
    normals = oracle.vertex_normals(verts, hand.faces, hand.vf_offsets, hand.vf_faces)
    cams = I.pack_cameras(I.make_cameras(cfg, hand.v_template.mean(0)))
    H, W = cfg.height, cfg.width
    bg = I.background(cfg.seed, cfg.views, H, W)
    o = oracle.make_opts(seed=cfg.seed * 7919 + 17, spp=cfg.spp, edge_samples=cfg.edge_samples, ka=I.K_AMBIENT,
                         kd=I.K_DIFFUSE, light_dir=I.LIGHT_DIR, light_rgb=I.LIGHT_RGB, edge_eps=I.EDGE_EPS_PX)
    rng = np.random.default_rng(0)
    A = (rng.choice([-1.0, 1.0], size=(cfg.views, H, W, 3)) * 1e-7).astype(np.float32)
    # bands of rows through the middle of each view (where the hand is), view after view
    rows_done, rays, secs = 0, 0.0, 0.0
    band = 4
    t_start = time.perf_counter()
    while time.perf_counter() - t_start < budget_s and rows_done < cfg.views * 96:
        view, k = divmod(rows_done, 96)
        r0 = view * H + H // 2 - 48 + k
        t0 = time.perf_counter()
        oracle.render_fwd(verts, hand.faces, normals, hand.albedo, cams, H, W, bg, o, rows=(r0, r0 + band))
        rmask = np.zeros_like(A)
        rv = rmask.reshape(cfg.views * H, W, 3)
        rv[r0:r0 + band] = A.reshape(cfg.views * H, W, 3)[r0:r0 + band]
        oracle.render_bwd_interior(verts, hand.faces, normals, hand.albedo, cams, H, W, bg, o, rmask,
                                   rows=(r0, r0 + band))
        secs += time.perf_counter() - t0
        rays += 2.0 * band * W * cfg.spp
        rows_done += band
    return rays, secs, rows_done


def cpu_baseline(args, budget_s=15.0):
    import oracle
    rays, secs, rows = _oracle_sample(budget_s)
    return {"value": round(rays / secs / 1e6, 5), "unit": UNIT, "cores": oracle.n_threads(), "kind": "oracle",
            "sample": f"forward + interior backward (brute force over all 1538 triangles, every pixel's adjoint "
                      f"non-zero) of {rows} rows x 512 px through the middle of the views at 16 spp, {secs:.1f} s"}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return None
    import oracle
    from paper_2107_05509_gb300 import inputs as I
    cfg = I.PAPER
    budget = max(1.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        _oracle_sample(budget)
    tot_rays, tot_s = 0.0, 0.0
    for _ in range(args.steps):
        r, s, rows = _oracle_sample(budget)
        tot_rays += r
        tot_s += s
    value = tot_rays / tot_s / 1e6
    cores = oracle.n_threads()
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * tot_s / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded procedural hand)",
            "config": {"workload": cfg.name, "views": cfg.views, "width": cfg.width, "height": cfg.height,
                       "spp": cfg.spp},
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: forward + interior backward of 4-row bands through the "
                                       f"middle of the views, about {budget:.0f} s of brute-force CPU work"},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="handrt", choices=["handrt", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-refine", action="store_true", help="skip the time-to-1 mm refinement comparison")
    ap.add_argument("--batch-instances", type=int, default=64)
    ap.add_argument("--refine-iters", type=int, default=150)
    ap.add_argument("--scale-instances", type=int, default=4)
    ap.add_argument("--scale-iters", type=int, default=60)
    ap.add_argument("--gemm-only", action="store_true", help="only the tensor-core GEMM timings (for profiling)")
    ap.add_argument("--objective-only", action="store_true", help="only the full-objective schedule")
    ap.add_argument("--edges-only", action="store_true", help="only the edge-term timings (for profiling)")
    ap.add_argument("--scale-only", action="store_true", help="only the scale workload (for profiling)")
    ap.add_argument("--refine-only", action="store_true", help="only the time-to-1 mm refinement comparison")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "handrt":
        args.warmup = 3
    if args.gemm_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(run_tensor(torch.device("cuda", 0))), flush=True)
        return
    if args.scale_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(run_scale(torch.device("cuda", 0))), flush=True)
        return
    if args.edges_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(run_edge_term(torch.device("cuda", 0))), flush=True)
        return
    if args.refine_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(run_refinement(args, torch.device("cuda", 0))), flush=True)
        return
    if args.objective_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(run_paper_objective(torch.device("cuda", 0))), flush=True)
        return
    line = run_reference(args) if args.impl == "reference" else run_handrt(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
