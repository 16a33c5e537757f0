#!/usr/bin/env python3
"""Benchmark: forward + backward samples/s of differentiable Monte Carlo ray
tracing with edge sampling on the direct-lighting workload.

Workload (one step): 256x256 image of a jittered icosphere (5120 triangles)
on a 2-triangle ground, lit by a 2-triangle area light; 64 samples per pixel
with one shadow ray each, 64 primary edge samples per pixel, one secondary
edge sample per interior sample.  A step is the whole hot path: vertex
update (LBVH rebuild, edge CDFs), render with a checkpoint tape, and the
backward pass (interior adjoint, secondary and primary edge terms, gradient
scatter).  Inputs are synthetic and seeded.

The second half of the metric, gradient variance x time of the learned
edge proposal against the plain edge sampler, comes from the proposal
module's protocol (train on logs of 20 scenes, score 4 held-out scenes) and
is reported under "variance_x_time" (N=1; --no-proposal skips it).  The
64-scene batched workload (persistent launches in a CUDA graph) is reported
under "batched", and the same with 64 small scenes under "batched_small"
(N=1; --no-batched skips both).  The secondary-edge hierarchy
(Sec. 5.3.1) and the importance-sampled point on an edge (Sec. 5.3.2)
against 3D length sampling with a uniform point, as gradient variance x
time, are reported under "secondary_samplers" (N=1; --no-hierarchy skips
it).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  For N > 1 (torchrun) every rank renders its
own replica and the value is the aggregate over ranks ("weak" scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd samples/sec and gradient variance x time vs plain edge sampler, 1 GB300"
UNIT = "samples/s"
W_IMG, H_IMG, SPP, EDGE_SPP = 256, 256, 64, 64
SCENE_SEED = 1236
BATCH_SEED, BATCH_SPP = 1238, 16
# Two triangles per BVH leaf: both timed workloads are direct lighting, whose
# rays are mostly coherent first-vertex rays (one per leaf suits path tracing).
BVH_LEAF = 2
WORKLOAD = ("direct lighting 256x256: jittered icosphere (5120 tris) + 2-tri ground + 2-tri area light; "
            "64 spp with 1 shadow ray, 64 primary edge spp, 1 secondary edge sample per path vertex; "
            "step = vertex update (LBVH + edge CDFs) + render + backward (all gradient terms)")
# FP32 lane-operations of one BVH node visit (two slab tests) and one
# watertight triangle test, counted from the kernels' arithmetic.
OPS_PER_NODE = 46
OPS_PER_TRI = 45
SMS, LANES, SM_MAX_MHZ = 152, 128, 2070.0


def peak_alu_tops():
    return SMS * LANES * SM_MAX_MHZ * 1e6 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def kernel_source_hash():
    h = hashlib.sha256()
    for rel in ("paper_1904_12228_gb300/csrc/render.cu", "paper_1904_12228_gb300/csrc/drt_device.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            t = json.load(f)
        ent = t.get(kernel)
        if ent and ent.get("source_hash") == kernel_source_hash():
            return ent.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device, self.proc = device, None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), max=float(f[2]), reasons=f[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = sorted({names[i] for r in rows for i, v in enumerate(r["reasons"]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["max"] for r in rows),
                "reasons": seen, "samples": len(rows)}


def run_batched(ctx, dev, replays=20, t_min=1000, t_max=100_000, resolutions=(128, 256, 512)):
    """64 procedural scenes (t_min-t_max triangles, log-uniform; square
    resolutions drawn from `resolutions`; direct lighting, 16 spp + 16 edge
    spp) as one batch step: persistent launches captured in a CUDA graph,
    launch shapes autotuned.  Median of `replays` graph replays, against the
    same scenes issued one render and one backward call at a time.  For the
    default workload the BVHs, tapes and sort buffers (several GB) exceed the
    129 MB L2, so no flush is needed between replays; the small-scene
    workload is reported as L2-resident."""
    import torch
    from paper_1904_12228_gb300 import drt
    from paper_1904_12228_gb300 import scenegen as sg
    scenes = sg.batch_workload(BATCH_SEED, t_min=t_min, t_max=t_max, resolutions=resolutions)
    up = [drt.Scene.from_arrays(ctx, sc, bvh_leaf_size=BVH_LEAF) for sc in scenes]
    d_images = [torch.from_numpy(sg.loss_adjoint(BATCH_SEED + k, sc.width, sc.height)).to(dev)
                for k, sc in enumerate(scenes)]
    imgs = [torch.zeros((sc.height, sc.width, 3), device=dev) for sc in scenes]

    def zeros_like_grads(sc):
        return dict(d_verts=torch.zeros((len(sc.verts), 3), device=dev),
                    d_albedo=torch.zeros((len(sc.tris), 3), device=dev), d_radiance=torch.zeros(3, device=dev),
                    d_cam_to_world=torch.zeros((3, 4), device=dev), d_cam_scale=torch.zeros(1, device=dev))
    grads = [zeros_like_grads(sc) for sc in scenes]
    opts = drt.make_opts(BATCH_SPP, BATCH_SPP, seed=7)
    t0 = time.perf_counter()
    b = drt.Batch(ctx, up, imgs, opts, d_images=d_images, grads=grads, use_graph=True, autotune=True)
    b.run()
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    for _ in range(2):
        b.run()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(replays)]
    for e0, e1 in ev:
        e0.record()
        b.run()
        e1.record()
    torch.cuda.synchronize()
    ms = statistics.median(e0.elapsed_time(e1) for e0, e1 in ev)
    code, info = ctx.check_device()
    if code != 0:
        raise RuntimeError("device error flag %d (%d) in the batched workload" % (code, info))
    # the same work as separate calls (same scene ids, tapes reused)
    tapes = [None] * len(scenes)
    for k, s in enumerate(up):
        tapes[k] = s.render(imgs[k], drt.make_opts(BATCH_SPP, BATCH_SPP, seed=7, scene_id=k), want_tape=True)
    single = []
    for rep in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k, s in enumerate(up):
            o = drt.make_opts(BATCH_SPP, BATCH_SPP, seed=7, scene_id=k)
            s.render(imgs[k], o, reuse=tapes[k])
            s.backward(d_images[k], o, tape=tapes[k], **grads[k])
        e1.record()
        torch.cuda.synchronize()
        single.append(e0.elapsed_time(e1))
    single_ms = statistics.median(single)
    samples = sum(sc.width * sc.height * BATCH_SPP for sc in scenes)
    inf = b.info()
    b.free()
    for t in tapes:
        t.free()
    return {"workload": "64 procedural scenes, triangles log-uniform in [%d,%d], resolution from {%s}, "
                        "direct lighting, 16 spp + 16 primary edge spp, all gradient terms"
                        % (t_min, t_max, ",".join(str(r) for r in resolutions)),
            "scenes": len(scenes), "triangles": int(sum(len(sc.tris) for sc in scenes)),
            "pixels": int(sum(sc.width * sc.height for sc in scenes)), "samples_per_step": samples,
            "ms_per_step": ms, "samples_per_s": samples / (ms / 1e3), "replays": replays,
            "single_calls_ms_per_step": single_ms, "speedup_vs_single_calls": single_ms / ms,
            "first_run_s": first_s, "launch_shapes": inf,
            "l2": "working set larger than L2 (no flush)" if t_min >= 1000 else "small scenes: L2-resident, no flush"}


def run_secondary_samplers(ctx, dev, K=24, samples=16):
    """Secondary edge term (Sec. 5.2.2) under three samplers, as gradient
    variance x time against the plain one (3D length CDF, uniform point): the
    edge hierarchy of Sec. 5.3.1 (`samples` root samples), and the
    importance-sampled point on the edge of Sec. 5.3.2 (clamped cosine over
    the edge's arc, mixed with uniform); the hierarchy also with 4 root
    samples.  Per scene, K runs with independent
    seeds; each run re-uploads the vertices (so the hierarchy is rebuilt
    inside the timed backward, as in an optimisation step), renders its tape
    (untimed) and times the backward pass of the secondary term alone.
    Variance: mean over vertex entries of the run variance, over the mean
    squared gradient; z2: mean squared z-score of the difference of a
    sampler's mean gradient and the plain one's (about 1 when both estimate
    the same term)."""
    import numpy as np
    import torch
    from paper_1904_12228_gb300 import drt
    from paper_1904_12228_gb300 import scenegen as sg
    out = []
    cases = (("direct lighting 256x256, 5124 tris, 64 spp", sg.direct_lighting(SCENE_SEED), 1, 64, 2),
             ("procedural 512x512, 200k tris, depth 3, 32 spp", sg.procedural(1237), 3, 32, 1))
    samplers = (("length", 0, 0), ("hierarchy", samples, 0), ("hierarchy_4", 4, 0), ("point", 0, 1))
    for name, sc, depth, spp, leaf in cases:
        S = drt.Scene.from_arrays(ctx, sc, bvh_leaf_size=leaf)
        verts = torch.from_numpy(sc.verts).to(dev)
        w = torch.from_numpy(sg.loss_adjoint(SCENE_SEED, sc.width, sc.height)).to(dev)
        img = torch.zeros((sc.height, sc.width, 3), device=dev)
        res = {}
        for label, tree, point in samplers:
            runs = torch.zeros((K, 3 * len(sc.verts)), device=dev)
            times = []
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for k in range(-2, K):  # two warm-up runs
                o = drt.make_opts(spp, 0, max_depth=depth, seed=7000 + k, terms=4, sec_tree_samples=tree,
                                  sec_point=point)
                S.update_vertices(verts)  # new scene version: the backward rebuilds the hierarchy
                tape = S.render(img, o, want_tape=True)
                dv = runs[max(k, 0)].view(-1, 3)
                dv.zero_()
                e0.record()
                S.backward(w, o, tape=tape, d_verts=dv)
                e1.record()
                e1.synchronize()
                if k >= 0:
                    times.append(e0.elapsed_time(e1))
            res[label] = (runs.double().cpu().numpy(), float(np.median(times)))
        ra, ta = res["length"]
        entry = {"scene": name, "triangles": len(sc.tris), "max_depth": depth, "spp": spp, "runs": K,
                 "var": {}, "ms": {}, "ratio": {}, "mean_z2": {}}
        mean_sq = {lab: (r.mean(0) ** 2).mean() for lab, (r, _) in res.items()}
        norm = float(np.mean(list(mean_sq.values()))) or 1.0
        va = float(ra.var(0, ddof=1).mean() / norm)
        for label, (rb, tb) in res.items():
            vb = float(rb.var(0, ddof=1).mean() / norm)
            entry["var"][label] = vb
            entry["ms"][label] = tb
            if label == "length":
                continue
            se2 = ra.var(0, ddof=1) / K + rb.var(0, ddof=1) / K
            ok = se2 > 0
            entry["mean_z2"][label] = float(np.mean((ra.mean(0)[ok] - rb.mean(0)[ok]) ** 2 / se2[ok])) if ok.any() else 0.0
            entry["ratio"][label] = (vb * tb) / max(va * ta, 1e-30)
        out.append(entry)
        S.free()
    geo = {lab: float(np.exp(np.mean([np.log(max(o["ratio"][lab], 1e-30)) for o in out])))
           for lab in ("hierarchy", "hierarchy_4", "point")}
    return {"ratio_geomean": geo, "root_samples": samples,
            "ratio_unit": "sampler/plain secondary-edge gradient variance x time (<1: the sampler wins); plain = "
                          "3D length CDF and uniform point; hierarchy = Sec. 5.3.1 with `root_samples` (hierarchy_4: "
                          "4) root samples; point = Sec. 5.3.2 (Lambertian)",
            "scenes": out}


def cpu_workload_sample(seconds_target, n_threads):
    """Time the CPU oracle on a bounded sample of the same workload: a block
    of pixels (all spp, interior + secondary edges) and a proportional range
    of primary edge samples.  Returns (samples/s, description, cores)."""
    import oracle
    from paper_1904_12228_gb300 import scenegen as sg
    scene = sg.direct_lighting(SCENE_SEED)
    w = sg.loss_adjoint(1, W_IMG, H_IMG)
    p0 = (H_IMG // 2) * W_IMG + W_IMG // 4

    def run(npix):
        t = time.perf_counter()
        oracle.render(scene, spp=SPP, seed=1, pixels=(p0, p0 + npix), n_threads=n_threads)
        oracle.backward(scene, w, spp=SPP, edge_spp=EDGE_SPP, seed=1, pixels=(p0, p0 + npix),
                        edges=(0, npix * EDGE_SPP), n_threads=n_threads)
        return time.perf_counter() - t

    n = 4
    dt = run(n)
    while dt < 0.15 * seconds_target and n < 4096:
        n *= 4
        dt = run(n)
    if dt < seconds_target and n < 4096:
        n2 = int(min(4096, n * seconds_target / max(dt, 1e-3)))
        if n2 > n:
            n, dt = n2, run(n2)
    samples = n * SPP
    desc = ("oracle, %d pixels x %d spp (render + backward with all terms) + %d primary edge samples of the "
            "256x256 workload, brute-force intersection over 5124 triangles" % (n, SPP, n * EDGE_SPP))
    return samples / dt, desc, n_threads, dt


def bench_config(triangles, world):
    return {"workload": WORKLOAD, "width": W_IMG, "height": H_IMG, "spp": SPP, "edge_spp": EDGE_SPP,
            "triangles": triangles, "bvh_leaf_size": BVH_LEAF, "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    from paper_1904_12228_gb300 import scenegen as sg
    oracle.build()
    cores = oracle.n_threads_default()
    per_step = max(1.0, 150.0 / max(1, args.steps + args.warmup))
    vals, times = [], []
    desc = ""
    for i in range(args.warmup + args.steps):
        v, desc, cores, dt = cpu_workload_sample(per_step, cores)
        if i >= args.warmup:
            vals.append(v)
            times.append(dt * 1e3)
    value = statistics.median(vals)
    config = bench_config(len(sg.direct_lighting(SCENE_SEED).tris), world)
    config["sample"] = desc
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-proposal", action="store_true", help="skip the learned-proposal variance x time part")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-scene batched workload")
    ap.add_argument("--no-hierarchy", action="store_true",
                    help="skip the secondary-edge sampler comparison (hierarchy, point sampling, length)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    from paper_1904_12228_gb300 import replicas
    rank, world, local = replicas.rank_info()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    from paper_1904_12228_gb300 import drt
    from paper_1904_12228_gb300 import scenegen as sg

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    ctx = drt.Context(local)
    scene_seed, adjoint_seed = replicas.replica_seeds(SCENE_SEED, 1, rank)
    scene = sg.direct_lighting(scene_seed)
    S = drt.Scene.from_arrays(ctx, scene, bvh_leaf_size=BVH_LEAF)
    V, T = len(scene.verts), len(scene.tris)
    verts = torch.from_numpy(scene.verts).to(dev)
    d_image = torch.from_numpy(sg.loss_adjoint(adjoint_seed, W_IMG, H_IMG)).to(dev)
    image = torch.zeros((H_IMG, W_IMG, 3), device=dev)
    g = dict(d_verts=torch.zeros((V, 3), device=dev), d_albedo=torch.zeros((T, 3), device=dev),
             d_radiance=torch.zeros(3, device=dev), d_cam_to_world=torch.zeros((3, 4), device=dev),
             d_cam_scale=torch.zeros(1, device=dev))
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    tape = S.render(image, drt.make_opts(SPP, EDGE_SPP, seed=0), want_tape=True)
    n_samples = W_IMG * H_IMG * SPP

    def step(k):
        opts = drt.make_opts(SPP, EDGE_SPP, seed=1000 + k)
        S.update_vertices(verts)
        S.render(image, opts, reuse=tape)
        S.backward(d_image, opts, tape=tape, **g)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    code, info = ctx.check_device()
    if code != 0:
        raise RuntimeError("device error flag %d (%d) during warm-up" % (code, info))
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ctx.profile(True)
    ctx.profile_read()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.zero_()                      # L2 flush between timed steps (not timed)
            starts[k].record()
            step(args.warmup + k)
            ends[k].record()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    prof = ctx.profile_read()
    ctx.profile(False)
    total_ms = replicas.max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), dist, dev)
    ms_per_step = total_ms / args.steps
    value = replicas.aggregate_throughput(n_samples, world, ms_per_step)

    # work counters of one extra (untimed) step
    ctx.counters(True)
    ctx.counters_read()
    step(0)
    cnt = ctx.counters_read()
    ctx.counters(False)
    rays = sum(c["closest_rays"] + c["shadow_rays"] for c in cnt.values())

    # dominant kernel and its roofline
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_launches) = dom
    avg_ms = dom_ms / dom_launches
    c = cnt.get(dom_name)
    roof = None
    if c:
        ops = OPS_PER_NODE * c["nodes"] + OPS_PER_TRI * c["tris"]
        achieved = ops / (avg_ms / 1e3) / 1e12
        peak = peak_alu_tops()
        traffic = ncu_traffic(dom_name)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": dom_name, "avg_launch_ms": avg_ms,
                "algorithmic_ops_per_launch": ops,
                "l1l2_bytes_per_launch": 64 * c["nodes"] + 48 * c["tris"],
                "peak_note": "152 SMs x 128 FP32 lanes x 2070 MHz (recipe unit counts and max clock)"}
    gpu_launches = sum(v[1] for v in prof.values())

    # end to end through the API with host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    h_verts = pin(scene.verts)
    h_dimg = pin(d_image.cpu().numpy())
    h_img = torch.zeros((H_IMG, W_IMG, 3)).pin_memory()
    hg = dict(d_verts=torch.zeros((V, 3)).pin_memory(), d_albedo=torch.zeros((T, 3)).pin_memory(),
              d_radiance=torch.zeros(3).pin_memory(), d_cam_to_world=torch.zeros((3, 4)).pin_memory(),
              d_cam_scale=torch.zeros(1).pin_memory())

    def e2e_step(k):
        opts = drt.make_opts(SPP, EDGE_SPP, seed=2000 + k)
        S.update_vertices(h_verts)
        S.render(h_img, opts, reuse=tape)
        S.backward(h_dimg, opts, tape=tape, **hg)

    for k in range(2):
        e2e_step(k)
    torch.cuda.synchronize()
    ke = max(3, args.steps // 4)
    t0 = time.perf_counter()
    for k in range(ke):
        e2e_step(k)
    torch.cuda.synchronize()
    e2e_ms = replicas.max_over_ranks((time.perf_counter() - t0) * 1e3 / ke, dist, dev)
    grad_bytes = 4 * (3 * V + 3 * T + 3 + 12 + 1)
    h2d = 12 * V + 12 * W_IMG * H_IMG + grad_bytes
    d2h = 12 * W_IMG * H_IMG + grad_bytes

    # the 64-scene batch (N=1 only), and the same with small scenes, where
    # per-call overheads dominate separate calls
    batched = batched_small = None
    if rank == 0 and world == 1 and not args.no_batched:
        batched = run_batched(ctx, dev)
        batched_small = run_batched(ctx, dev, t_min=300, t_max=3000, resolutions=(64, 96, 128))

    sec_h = None
    if rank == 0 and world == 1 and not args.no_hierarchy:
        sec_h = run_secondary_samplers(ctx, dev)

    # second half of the metric: gradient variance x time, learned proposal
    # against the plain edge sampler (N=1 only)
    vxt = None
    if rank == 0 and world == 1 and not args.no_proposal:
        from paper_1904_12228_gb300 import proposal
        vxt = proposal.protocol(ctx)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        v, desc, cores, dt = cpu_workload_sample(args.cpu_seconds, oracle.n_threads_default())
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc, "seconds": dt}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": bench_config(T, world),
                "rays_per_s": world * rays / (ms_per_step / 1e3),
                "roofline": roof, "cpu_baseline": cpu, "variance_x_time": vxt, "batched": batched,
                "batched_small": batched_small,
                "secondary_samplers": sec_h,
                "e2e": {"value": replicas.aggregate_throughput(n_samples, world, e2e_ms), "unit": UNIT,
                        "ms_per_step": e2e_ms,
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": gpu_launches,
                "kernels": {k: {"ms_total": v[0], "launches": v[1]} for k, v in prof.items()},
                "counters": cnt, "clocks": clocks.summary(),
                "peaks": {k: measured_peaks().get(k) for k in ("hbm_gbs", "bf16_tflops")}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
