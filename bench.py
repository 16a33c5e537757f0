#!/usr/bin/env python3
"""Benchmark: forward + backward samples/s of differentiable Monte Carlo ray
tracing with edge sampling.

Headline workload (one step): the procedural scene of about 200k triangles
(displaced icospheres and subdivided boxes on a ground quad, two area
lights), 512x512, path tracing with 3 scattering vertices and next-event
estimation at each, 32 samples per pixel, 32 primary edge samples per pixel
and one secondary edge sample per path vertex.  A step is the whole hot
path: vertex update (LBVH rebuild, edge CDFs), render with a checkpoint tape,
and the backward pass (interior adjoint, secondary and primary edge terms,
gradient scatter).  Inputs are synthetic and seeded.

Reported beside it (N=1): the direct-lighting workload (256x256, jittered
icosphere of 5120 triangles, 64 spp + 64 edge spp) under "direct_lighting";
the second half of the metric, gradient variance x time of the learned edge
proposal against the plain edge sampler (train on logs of 20 scenes, score 4
held-out scenes) under "variance_x_time" (--no-proposal skips it); the
64-scene batched workload (persistent launches in a CUDA graph) under
"batched", and the same with 64 small scenes under "batched_small"
(--no-batched skips both); the secondary-edge hierarchy (Sec. 5.3.1), the
importance-sampled point on an edge (Sec. 5.3.2) and next-event estimation
for edges (Sec. 5.3.3) against 3D length sampling with a uniform point, as
gradient variance x time, under "secondary_samplers" (--no-hierarchy skips
it); the tensor-core network's
BF16 rate under "mlp".

Roofline: the ray kernels are bound by issue slots and L1/L2 bandwidth (no
dense contraction, working set mostly in L2).  Per launch, the algorithmic
work of a kernel is 12 lane-operations per ray-box slab test (two per BVH
node visit) plus 26 per watertight triangle test, and its algorithmic bytes
64 per node visit plus 48 per triangle test, from the kernel's work
counters.  The peaks are measured in the same run by the library's probes
(FP32 FMA lane-operation rate; L2-resident copy bandwidth).

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


class Workload:
    def __init__(self, key, seed, spp, edge_spp, depth, leaf, desc):
        self.key, self.seed, self.spp, self.edge_spp, self.depth, self.leaf, self.desc = \
            key, seed, spp, edge_spp, depth, leaf, desc

    def scene(self, seed=None):
        from paper_1904_12228_gb300 import scenegen as sg
        s = self.seed if seed is None else seed
        if self.key == "procedural":
            return sg.procedural(s)
        if self.key == "procedural_small":
            return sg.procedural(s, n_target=50_000, width=256, height=256)
        return sg.direct_lighting(s)


# the inverse-rendering workload: 512x512, ~200k triangles, depth 3, 32 + 32 spp
PROCEDURAL = Workload("procedural", 1237, 32, 32, 3, 1,
                      "procedural 512x512: ~200k triangles (displaced icospheres + subdivided boxes) on a ground quad "
                      "with 2 area lights; path tracing depth 3 with NEE at every vertex, 32 spp, 32 primary edge spp, "
                      "1 secondary edge sample per path vertex; step = vertex update (LBVH + edge CDFs) + render + "
                      "backward (all gradient terms)")
# direct lighting: 256x256, icosphere 5120 triangles, 64 + 64 spp; two
# triangles per BVH leaf (coherent first-vertex rays)
DIRECT = Workload("direct", 1236, 64, 64, 1, 2,
                  "direct lighting 256x256: jittered icosphere (5120 tris) + 2-tri ground + 2-tri area light; "
                  "64 spp with 1 shadow ray, 64 primary edge spp, 1 secondary edge sample per path vertex; "
                  "step = vertex update (LBVH + edge CDFs) + render + backward (all gradient terms)")
# a reduced procedural case for profiler captures (same kernels, a few hundred MB on the device)
PROCEDURAL_SMALL = Workload("procedural_small", 1237, 32, 32, 3, 1,
                            "procedural 256x256: ~50k triangles, path tracing depth 3, 32 spp, 32 primary edge spp "
                            "(profiling case); step = vertex update + render + backward")
WORKLOADS = {"procedural": PROCEDURAL, "direct": DIRECT, "procedural_small": PROCEDURAL_SMALL}
HEADLINE = PROCEDURAL
BATCH_SEED, BATCH_SPP = 1238, 16
BVH_LEAF = 2  # batched direct-lighting workloads
# lane-operations and bytes of the algorithmic work units
OPS_PER_BOX = 12          # slab test: 6 FMA + 6 min/max
BOXES_PER_NODE = 2        # a BVH node visit tests both child boxes
OPS_PER_TRI = 26          # watertight test: shear and edge functions
BYTES_PER_NODE = 64
BYTES_PER_TRI = 48
# profiled kernel name -> work-counter slot
COUNTER_OF = {"render": "render", "render_first": "render", "render_bounce": "render_bounce",
              "backward_interior": "backward_interior", "backward_path": "backward_interior",
              "backward_primary_edges": "backward_primary_edges",
              "backward_secondary_edges": "backward_secondary_edges",
              "backward_secondary_sides": "backward_secondary_sides",
              "backward_secondary_bounce": "backward_secondary_bounce",
              "backward_primary_first": "backward_primary_edges",
              "backward_primary_bounce": "backward_primary_bounce"}


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


def ncu_traffic(workload, kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            t = json.load(f)
        ent = t.get(workload, {}).get(kernel)
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
    """Secondary edge term (Sec. 5.2.2) under four samplers, as gradient
    variance x time against the plain one (3D length CDF, uniform point): the
    edge hierarchy of Sec. 5.3.1 (`samples` root samples), the
    importance-sampled point on the edge of Sec. 5.3.2 (clamped cosine over
    the edge's arc, mixed with uniform), and next-event estimation for edges
    of Sec. 5.3.3 beside the plain sampler; the hierarchy also with 4 root
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
    cases = (("direct lighting 256x256, 5124 tris, 64 spp", sg.direct_lighting(DIRECT.seed), 1, 64, 2),
             ("direct lighting 256x256, 5124 tris, 64 spp, small light (0.1 x 0.1, same power)",
              sg.direct_lighting(DIRECT.seed, light_half=0.05), 1, 64, 2),
             ("procedural 512x512, 200k tris, depth 3, 32 spp", sg.procedural(1237), 3, 32, 1))
    samplers = (("length", 0, 0, 0), ("hierarchy", samples, 0, 0), ("hierarchy_4", 4, 0, 0), ("point", 0, 1, 0),
                ("nee", 0, 0, 1))
    for name, sc, depth, spp, leaf in cases:
        S = drt.Scene.from_arrays(ctx, sc, bvh_leaf_size=leaf)
        verts = torch.from_numpy(sc.verts).to(dev)
        w = torch.from_numpy(sg.loss_adjoint(DIRECT.seed, sc.width, sc.height)).to(dev)
        img = torch.zeros((sc.height, sc.width, 3), device=dev)
        res = {}
        for label, tree, point, nee in samplers:
            runs = torch.zeros((K, 3 * len(sc.verts)), device=dev)
            times = []
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for k in range(-2, K):  # two warm-up runs
                o = drt.make_opts(spp, 0, max_depth=depth, seed=7000 + k, terms=4, sec_tree_samples=tree,
                                  sec_point=point, sec_nee=nee)
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
           for lab in ("hierarchy", "hierarchy_4", "point", "nee")}
    return {"ratio_geomean": geo, "root_samples": samples,
            "ratio_unit": "sampler/plain secondary-edge gradient variance x time (<1: the sampler wins); plain = "
                          "3D length CDF and uniform point; hierarchy = Sec. 5.3.1 with `root_samples` (hierarchy_4: "
                          "4) root samples; point = Sec. 5.3.2 (Lambertian); nee = Sec. 5.3.3, billboard samples of "
                          "the shadow rays beside the length sampler (balance heuristic)",
            "scenes": out}


def cpu_workload_sample(wl, seconds_target, n_threads, n_fixed=None):
    """Time the CPU oracle on a bounded sample of workload wl: a block of
    pixels (all spp, interior + secondary edges) and a proportional range of
    primary edge samples, sized to about seconds_target (or n_fixed pixels).
    Returns (samples/s, description, cores, seconds, pixels)."""
    import oracle
    from paper_1904_12228_gb300 import scenegen as sg
    scene = wl.scene()
    W, H = scene.width, scene.height
    w = sg.loss_adjoint(1, W, H)
    p0 = (H // 2) * W + W // 4

    def run(npix):
        t = time.perf_counter()
        oracle.render(scene, spp=wl.spp, seed=1, max_depth=wl.depth, pixels=(p0, p0 + npix), n_threads=n_threads)
        oracle.backward(scene, w, spp=wl.spp, edge_spp=wl.edge_spp, seed=1, max_depth=wl.depth,
                        pixels=(p0, p0 + npix), edges=(0, npix * wl.edge_spp), n_threads=n_threads)
        return time.perf_counter() - t

    if n_fixed:
        n = n_fixed
        dt = run(n)
    else:
        n = max(1, n_threads)
        dt = run(n)
    while not n_fixed and dt < 0.15 * seconds_target and n < 4096:
        n *= 4
        dt = run(n)
    if not n_fixed and dt < seconds_target and n < 4096:
        n2 = int(min(4096, n * seconds_target / max(dt, 1e-3)))
        if n2 > n:
            n, dt = n2, run(n2)
    samples = n * wl.spp
    desc = ("oracle, %d pixels x %d spp (render + backward with all terms, depth %d) + %d primary edge samples of "
            "the %dx%d workload, brute-force intersection over %d triangles"
            % (n, wl.spp, wl.depth, n * wl.edge_spp, W, H, len(scene.tris)))
    return samples / dt, desc, n_threads, dt, n


def bench_config(wl, triangles, world):
    return {"workload": wl.desc, "width": 512 if wl.key == "procedural" else 256,
            "height": 512 if wl.key == "procedural" else 256, "spp": wl.spp, "edge_spp": wl.edge_spp,
            "max_depth": wl.depth, "triangles": triangles, "bvh_leaf_size": wl.leaf,
            "l2": "flushed between timed steps (256 MiB write); the step's working set (tape, sort and "
                  "secondary scratch) is also larger than L2",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = oracle.n_threads_default()
    # every step runs the same bounded sample, sized once so that the whole
    # run takes about 150 s of CPU work
    per_step = max(1.0, 150.0 / max(1, args.steps + args.warmup))
    _, _, _, _, n = cpu_workload_sample(HEADLINE, per_step, cores)
    vals, times = [], []
    desc = ""
    for i in range(args.warmup + args.steps):
        v, desc, cores, dt, _ = cpu_workload_sample(HEADLINE, per_step, cores, n_fixed=n)
        if i >= args.warmup:
            vals.append(v)
            times.append(dt * 1e3)
    value = statistics.median(vals)
    config = bench_config(HEADLINE, len(HEADLINE.scene().tris), world)
    config["sample"] = desc
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def kernel_rooflines(prof, cnt, steps, peak_ops, peak_l2):
    """Per ray kernel: algorithmic lane-operations and bytes per launch over
    its mean event-timed launch, against the measured FMA and L2 peaks."""
    out = {}
    for name, (ms, launches) in prof.items():
        slot = COUNTER_OF.get(name)
        c = cnt.get(slot) if slot else None
        if not c or c["nodes"] == 0 or launches == 0:
            continue
        per_step = max(1, round(launches / steps))
        avg_s = ms / launches / 1e3
        ops = (OPS_PER_BOX * BOXES_PER_NODE * c["nodes"] + OPS_PER_TRI * c["tris"]) / per_step
        nbytes = (BYTES_PER_NODE * c["nodes"] + BYTES_PER_TRI * c["tris"]) / per_step
        a_ops, a_l2 = ops / avg_s, nbytes / avg_s
        out[name] = {"avg_launch_ms": avg_s * 1e3, "launches_per_step": per_step,
                     "node_visits_per_launch": c["nodes"] / per_step, "tri_tests_per_launch": c["tris"] / per_step,
                     "alu": {"achieved": a_ops / 1e12, "peak": peak_ops / 1e12, "unit": "T lane-ops/s",
                             "frac": a_ops / peak_ops},
                     "l2": {"achieved": a_l2 / 1e9, "peak": peak_l2 / 1e9, "unit": "GB/s", "frac": a_l2 / peak_l2}}
    return out


def run_workload(ctx, dev, wl, steps, warmup, rank, world, dist, flush, timed_extras=True):
    """Time `steps` fwd+bwd steps of workload wl (inputs resident in HBM),
    then one counted step, then the same step end to end with host buffers."""
    import numpy as np
    import torch
    from paper_1904_12228_gb300 import drt
    from paper_1904_12228_gb300 import replicas
    from paper_1904_12228_gb300 import scenegen as sg
    scene_seed, adjoint_seed = replicas.replica_seeds(wl.seed, 1, rank)
    scene = wl.scene(scene_seed)
    W, H = scene.width, scene.height
    S = drt.Scene.from_arrays(ctx, scene, bvh_leaf_size=wl.leaf)
    V, T = len(scene.verts), len(scene.tris)
    verts = torch.from_numpy(scene.verts).to(dev)
    d_image = torch.from_numpy(sg.loss_adjoint(adjoint_seed, W, H)).to(dev)
    image = torch.zeros((H, W, 3), device=dev)
    g = dict(d_verts=torch.zeros((V, 3), device=dev), d_albedo=torch.zeros((T, 3), device=dev),
             d_radiance=torch.zeros(3, device=dev), d_cam_to_world=torch.zeros((3, 4), device=dev),
             d_cam_scale=torch.zeros(1, device=dev))
    opts0 = drt.make_opts(wl.spp, wl.edge_spp, max_depth=wl.depth, seed=0)
    tape = S.render(image, opts0, want_tape=True)
    n_samples = W * H * wl.spp

    def step(k):
        opts = drt.make_opts(wl.spp, wl.edge_spp, max_depth=wl.depth, seed=1000 + k)
        S.update_vertices(verts)
        S.render(image, opts, reuse=tape)
        S.backward(d_image, opts, tape=tape, **g)

    for k in range(warmup):
        step(k)
    torch.cuda.synchronize()
    code, info = ctx.check_device()
    if code != 0:
        raise RuntimeError("device error flag %d (%d) during warm-up" % (code, info))
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ctx.profile(True)
    ctx.profile_read()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index or 0) as clocks:
        for k in range(steps):
            flush.zero_()                      # L2 flush between timed steps (not timed)
            starts[k].record()
            step(warmup + k)
            ends[k].record()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    prof = ctx.profile_read()
    ctx.profile(False)
    code, info = ctx.check_device()
    if code != 0:
        raise RuntimeError("device error flag %d (%d) in the timed steps" % (code, info))
    total_ms = replicas.max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), dist, dev)
    ms_per_step = total_ms / steps
    value = replicas.aggregate_throughput(n_samples, world, ms_per_step)

    # work counters of one extra (untimed) step
    ctx.counters(True)
    ctx.counters_read()
    step(0)
    cnt = ctx.counters_read()
    ctx.counters(False)
    rays = sum(c["closest_rays"] + c["shadow_rays"] for c in cnt.values())

    # end to end through the API with host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    h_verts = pin(scene.verts)
    h_dimg = pin(d_image.cpu().numpy())
    h_img = torch.zeros((H, W, 3)).pin_memory()
    hg = dict(d_verts=torch.zeros((V, 3)).pin_memory(), d_albedo=torch.zeros((T, 3)).pin_memory(),
              d_radiance=torch.zeros(3).pin_memory(), d_cam_to_world=torch.zeros((3, 4)).pin_memory(),
              d_cam_scale=torch.zeros(1).pin_memory())

    def e2e_step(k):
        opts = drt.make_opts(wl.spp, wl.edge_spp, max_depth=wl.depth, seed=2000 + k)
        S.update_vertices(h_verts)
        S.render(h_img, opts, reuse=tape)
        S.backward(h_dimg, opts, tape=tape, **hg)

    for k in range(2):
        e2e_step(k)
    torch.cuda.synchronize()
    ke = max(3, steps // 4)
    t0 = time.perf_counter()
    for k in range(ke):
        e2e_step(k)
    torch.cuda.synchronize()
    e2e_ms = replicas.max_over_ranks((time.perf_counter() - t0) * 1e3 / ke, dist, dev)
    grad_bytes = 4 * (3 * V + 3 * T + 3 + 12 + 1)
    h2d = 12 * V + 12 * W * H + grad_bytes
    d2h = 12 * W * H + grad_bytes
    tape.free()
    S.free()
    return {"scene": scene, "triangles": T, "ms_per_step": ms_per_step, "value": value, "prof": prof,
            "counters": cnt, "rays": rays, "clocks": clocks.summary(),
            "e2e": {"value": replicas.aggregate_throughput(n_samples, world, e2e_ms), "unit": UNIT,
                    "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": sum(v[1] for v in prof.values())}


def roofline_of(res, steps, peaks, wl):
    """Roofline of the dominant kernel: the ray kernel (one with counted work)
    with the most event time.  Kernels on the second stream (the sample keys
    and their sort) are left out: their event times include waiting for the
    kernels beside them."""
    kr = kernel_rooflines(res["prof"], res["counters"], steps, peaks["alu_ops"], peaks["l2_bytes"])
    if not kr:
        return None, kr
    dom_name, (dom_ms, dom_launches) = max(((n, v) for n, v in res["prof"].items() if n in kr),
                                           key=lambda kv: kv[1][0])
    k = kr[dom_name]
    binding = "alu" if k["alu"]["frac"] >= k["l2"]["frac"] else "l2"
    b = k[binding]
    roof = {"bound": binding, "achieved": b["achieved"], "peak": b["peak"], "unit": b["unit"], "frac": b["frac"],
            "traffic": ncu_traffic(wl.key, dom_name), "kernel": dom_name, "avg_launch_ms": k["avg_launch_ms"],
            "share_of_step": dom_ms / steps / res["ms_per_step"],
            "alu": k["alu"], "l2": k["l2"],
            "algorithmic_ops_per_launch": OPS_PER_BOX * BOXES_PER_NODE * k["node_visits_per_launch"]
            + OPS_PER_TRI * k["tri_tests_per_launch"],
            "algorithmic_bytes_per_launch": BYTES_PER_NODE * k["node_visits_per_launch"]
            + BYTES_PER_TRI * k["tri_tests_per_launch"],
            "work_units": "12 lane-ops per ray-box slab test (2 per BVH node visit) + 26 per watertight triangle "
                          "test; 64 B per node visit + 48 B per triangle test; from the kernel's work counters",
            "peak_note": "peaks of measured: FP32 FMA lane-op rate (drt_probe_fma) and L2-resident copy "
                         "bandwidth (drt_probe_l2), same run; binding resource = the larger fraction"}
    return roof, kr


def run_mlp_rate(ctx, dev, m=1 << 22):
    """BF16 tensor-core rate of the edge-proposal network (tcgen05, FP32
    accumulation) on m rows: forward and backward, best of 5 launches each."""
    import torch
    from paper_1904_12228_gb300 import proposal
    net = proposal.EdgeProposal(ctx, seed=1)
    g = torch.Generator(device="cpu").manual_seed(2)
    x = torch.randn((m, proposal.N_IN), generator=g).to(dev).to(torch.bfloat16).view(torch.int16).contiguous()
    y = torch.empty(m, device=dev)
    target = torch.randn(m, device=dev)
    mask = torch.ones(m, device=dev)
    loss = torch.zeros(1, device=dev)

    def best(f):
        f()
        torch.cuda.synchronize()
        ts = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            f()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts)

    fwd_ms = best(lambda: ctx.mlp_forward(x, net._w, y))
    bwd_ms = best(lambda: ctx.mlp_backward(x, target, mask, 1.0 / m, net._w, net._gp, loss))
    i, h = proposal.N_IN, proposal.HIDDEN
    fwd_tc = 2.0 * m * (i * h + h * h)                    # the two tensor-core layers
    bwd_tc = 2.0 * m * (i * h + h * h) + 2.0 * m * (h * h) + 2.0 * m * (h * h + i * h)  # recompute, dz1, dW2, dW1
    peak = measured_peaks().get("bf16_tflops")
    out = {"rows": m, "forward_ms": fwd_ms, "backward_ms": bwd_ms,
           "forward_tflops": fwd_tc / (fwd_ms * 1e-3) / 1e12, "backward_tflops": bwd_tc / (bwd_ms * 1e-3) / 1e12,
           "input_gbs_forward": m * i * 2 / (fwd_ms * 1e-3) / 1e9,
           "peak_bf16_tflops": peak, "peak_note": "bf16_tflops of measured (cuBLAS burst)",
           "flops_note": "tensor-core flops only: 2 m (32x64 + 64x64) forward; backward adds the recompute, "
                         "dz1 = dz2 W2 and the weight gradients dW2, dW1"}
    if peak:
        out["forward_frac"] = out["forward_tflops"] / peak
        out["backward_frac"] = out["backward_tflops"] / peak
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-proposal", action="store_true", help="skip the learned-proposal variance x time part")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-scene batched workload")
    ap.add_argument("--no-hierarchy", action="store_true",
                    help="skip the secondary-edge sampler comparison (hierarchy, point sampling, length)")
    ap.add_argument("--no-direct", action="store_true", help="skip the direct-lighting workload")
    ap.add_argument("--workload", default="procedural", choices=sorted(WORKLOADS),
                    help="the timed workload (default: the 512x512 ~200k-triangle depth-3 scene)")
    args = ap.parse_args()
    global HEADLINE
    HEADLINE = WORKLOADS[args.workload]
    args.warmup = max(args.warmup, 3)
    from paper_1904_12228_gb300 import replicas
    rank, world, local = replicas.rank_info()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    from paper_1904_12228_gb300 import drt

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    ctx = drt.Context(local)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = {"alu_ops": ctx.probe_fma(), "l2_bytes": ctx.probe_l2(32 << 20), "sms": sms}

    res = run_workload(ctx, dev, HEADLINE, args.steps, args.warmup, rank, world, dist, flush)
    roof, kroof = roofline_of(res, args.steps, peaks, HEADLINE)

    direct = None
    if rank == 0 and world == 1 and not args.no_direct:
        d = run_workload(ctx, dev, DIRECT, args.steps, args.warmup, 0, 1, None, flush)
        droof, dk = roofline_of(d, args.steps, peaks, DIRECT)
        direct = {"workload": DIRECT.desc, "triangles": d["triangles"], "ms_per_step": d["ms_per_step"],
                  "samples_per_s": d["value"], "rays_per_s": d["rays"] / (d["ms_per_step"] / 1e3),
                  "e2e": d["e2e"], "roofline": droof, "kernels_roofline": dk, "clocks": d["clocks"],
                  "kernels": {k: {"ms_total": v[0], "launches": v[1]} for k, v in d["prof"].items()}}

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
    # against the plain edge sampler (N=1 only), and the network's BF16 rate
    vxt = mlp = None
    if rank == 0 and world == 1 and not args.no_proposal:
        from paper_1904_12228_gb300 import proposal
        vxt = proposal.protocol(ctx)
        mlp = run_mlp_rate(ctx, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        v, desc, cores, dt, _ = cpu_workload_sample(HEADLINE, args.cpu_seconds, oracle.n_threads_default())
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc, "seconds": dt}

    if rank == 0:
        mp = measured_peaks()
        line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": bench_config(HEADLINE, res["triangles"], world),
                "rays_per_s": world * res["rays"] / (res["ms_per_step"] / 1e3),
                "roofline": roof, "kernels_roofline": kroof, "cpu_baseline": cpu, "e2e": res["e2e"],
                "gpu_launches": res["gpu_launches"],
                "kernels": {k: {"ms_total": v[0], "launches": v[1]} for k, v in res["prof"].items()},
                "counters": res["counters"], "clocks": res["clocks"],
                "direct_lighting": direct, "variance_x_time": vxt, "mlp": mlp, "batched": batched,
                "batched_small": batched_small, "secondary_samplers": sec_h,
                "peaks": {"fma_lane_ops_per_s": peaks["alu_ops"], "l2_bytes_per_s": peaks["l2_bytes"],
                          "sms": sms, "hbm_gbs": mp.get("hbm_gbs"), "bf16_tflops": mp.get("bf16_tflops")}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
