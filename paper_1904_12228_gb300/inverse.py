"""Inverse rendering by gradient descent through the renderer (the
optimisation protocol of Sec. 5.4.1: start from perturbed parameters and
minimise the L2 image difference to a target with Adam).

    python -m paper_1904_12228_gb300.inverse [--steps 100] [--small]

Default: the 512x512 procedural scene of about 200k triangles, path tracing
with 3 scattering vertices at 32 spp; target rendered at the seed vertices,
start = vertices + N(0, 0.02), Adam (lr 1e-3) on the vertex tensor.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import scenegen as sg
from .autograd import Renderer


def run(scene, steps=100, lr=1e-3, spp=32, max_depth=3, target_spp=128, seed=0, device=0, log=None):
    """Returns a list of dicts (step, loss, vertex RMS error, ms)."""
    dev = torch.device("cuda", device)
    ren = Renderer(scene, device=device, spp=spp, max_depth=max_depth, seed=seed + 1)
    albedo = torch.from_numpy(scene.albedo).to(dev)
    rad = torch.from_numpy(scene.radiance).to(dev)
    cam = torch.from_numpy(scene.cam_to_world).to(dev)
    scale = torch.tensor([scene.cam_scale], dtype=torch.float32, device=dev)
    v_true = torch.from_numpy(scene.verts).to(dev)
    tgt_ren = Renderer(scene, device=device, spp=target_spp, max_depth=max_depth, seed=seed + 10_000_000,
                       ctx=ren.ctx)
    with torch.no_grad():
        target = tgt_ren(v_true, albedo, rad, cam, scale).clone()
    v = torch.from_numpy(sg.perturb_vertices(scene, seed)).to(dev).requires_grad_(True)
    opt = torch.optim.Adam([v], lr=lr)
    hist = []
    moved = None
    for k in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        img = ren(v, albedo, rad, cam, scale)
        loss = ((img - target) ** 2).mean()
        opt.zero_grad()
        loss.backward()
        if moved is None:
            moved = v.grad.abs().sum(1) > 0  # vertices the image depends on
        opt.step()
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        with torch.no_grad():
            err = (v - v_true)[moved].pow(2).sum(1).mean().sqrt().item() if moved.any() else 0.0
        rec = {"step": k, "loss": float(loss.item()), "vertex_rms_error": err, "ms": ms}
        hist.append(rec)
        if log:
            log(rec)
    return hist


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--small", action="store_true", help="20k triangles at 128x128, depth 2, 8 spp")
    ap.add_argument("--seed", type=int, default=1237)
    args = ap.parse_args()
    if args.small:
        scene = sg.procedural(args.seed, n_target=20_000, width=128, height=128)
        hist = run(scene, steps=args.steps, spp=8, max_depth=2, target_spp=64, lr=2e-3)
    else:
        scene = sg.procedural(args.seed)
        hist = run(scene, steps=args.steps)
    for h in hist[:: max(1, len(hist) // 10)] + hist[-1:]:
        print(json.dumps(h))
    ms = [h["ms"] for h in hist[3:]] or [h["ms"] for h in hist]
    print(json.dumps({"triangles": len(scene.tris), "width": scene.width, "height": scene.height,
                      "loss_first": hist[0]["loss"], "loss_last": hist[-1]["loss"],
                      "vertex_rms_first": hist[0]["vertex_rms_error"], "vertex_rms_last": hist[-1]["vertex_rms_error"],
                      "ms_per_step_median": float(np.median(ms))}))


if __name__ == "__main__":
    main()
