"""Inverse rendering by gradient descent through the renderer (the
optimisation protocol of Sec. 5.4.1: start from perturbed parameters and
minimise the L2 image difference to a target with Adam).

    python -m paper_1904_12228_gb300.inverse [--steps 100] [--small] [--objects]

Default: the 512x512 procedural scene of about 200k triangles, path tracing
with 3 scattering vertices at 32 spp; target rendered at the seed vertices,
start = vertices + N(0, 0.02), Adam (lr 1e-3) on the vertex tensor.
--objects: one translation per object (connected component of the mesh)
instead of free vertices, start = object + N(0, 0.05) per axis; the lights
and the ground stay fixed.

The vertex error is reported whole and split, per vertex, into its part
along the vertex normal of the true surface and its tangential part.
Moving a vertex along its surface leaves a smooth surface where it is and
changes the image only through the triangles' albedo and shading normals,
so with free vertices the tangential part is barely observable.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import scenegen as sg
from .autograd import Renderer


def vertex_normals(verts: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Area-weighted unit normals of the vertices (zero for isolated ones)."""
    v = verts.astype(np.float64)
    t = tris.astype(np.int64)
    fn = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])  # 2 x area x unit normal
    n = np.zeros_like(v)
    for k in range(3):
        np.add.at(n, t[:, k], fn)
    ln = np.linalg.norm(n, axis=1, keepdims=True)
    return np.where(ln > 0, n / np.maximum(ln, 1e-300), 0.0)


def components(verts: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Object label of every vertex: connected components of the mesh by
    union-find over the triangles' vertices, vertices at the same position
    counted as one (the faces of a box are separate sheets that meet at
    their borders); labels 0..k-1 in order of first vertex."""
    _, pos_id = np.unique(np.asarray(verts), axis=0, return_inverse=True)
    pos_id = pos_id.ravel()
    parent = np.arange(int(pos_id.max()) + 1 if len(pos_id) else 0)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for tri in pos_id[np.asarray(tris, np.int64)]:
        r0 = find(tri[0])
        for x in tri[1:]:
            r = find(x)
            if r != r0:
                lo, hi = min(r, r0), max(r, r0)
                parent[hi] = lo
                r0 = lo
    roots = np.array([find(p) for p in pos_id])
    _, labels = np.unique(roots, return_inverse=True)
    return labels.ravel()


def run(scene, steps=100, lr=1e-3, spp=32, max_depth=3, target_spp=128, seed=0, device=0, log=None,
        objects=False, sigma=None, decorrelate=False, lr_final=None):
    """Returns a list of dicts (step, loss, vertex RMS error whole, along the
    true vertex normals and tangential, ms).  objects=False: Adam on the free
    vertex tensor, start = vertices + N(0, sigma=0.02).  objects=True: Adam
    on one translation per object (every connected component except the
    lights and the widest one, the ground), start = N(0, sigma=0.05).

    decorrelate: the residual image - target comes from a second render with
    independent samples, and the gradient flows through the first.  The
    gradient of the L2 loss of one Monte Carlo image, 2 (I - T) dI/dtheta,
    pairs the image's noise with its own derivative; with I and dI from
    independent samples its mean is the gradient of |E[I] - T|^2, the
    quantity the optimisation means to lower.  lr_final: the learning rate
    falls from lr to lr_final by a cosine over the steps (default: constant)."""
    dev = torch.device("cuda", device)
    ren = Renderer(scene, device=device, spp=spp, max_depth=max_depth, seed=seed + 1)
    ren_res = Renderer(scene, device=device, spp=spp, max_depth=max_depth, seed=seed + 20_000_000,
                       ctx=ren.ctx) if decorrelate else None
    albedo = torch.from_numpy(scene.albedo).to(dev)
    rad = torch.from_numpy(scene.radiance).to(dev)
    cam = torch.from_numpy(scene.cam_to_world).to(dev)
    scale = torch.tensor([scene.cam_scale], dtype=torch.float32, device=dev)
    v_true = torch.from_numpy(scene.verts).to(dev)
    normals = torch.from_numpy(vertex_normals(scene.verts, scene.tris).astype(np.float32)).to(dev)
    tgt_ren = Renderer(scene, device=device, spp=target_spp, max_depth=max_depth, seed=seed + 10_000_000,
                       ctx=ren.ctx)
    with torch.no_grad():
        target = tgt_ren(v_true, albedo, rad, cam, scale).clone()
    if objects:
        label = components(scene.verts, scene.tris)
        n_obj = int(label.max()) + 1
        fixed = set(label[np.asarray(scene.tris)[np.asarray(scene.light_tris)].ravel()].tolist())
        extent = np.zeros(n_obj)
        for k in range(n_obj):
            pk = scene.verts[label == k]
            extent[k] = np.linalg.norm(pk.max(0) - pk.min(0))
        fixed.add(int(np.argmax(extent)))  # the ground
        free = np.array([k not in fixed for k in range(n_obj)])
        onehot = torch.zeros((len(scene.verts), n_obj), device=dev)
        onehot[torch.arange(len(scene.verts)), torch.from_numpy(label)] = 1.0
        onehot[:, torch.from_numpy(~free)] = 0.0
        rng = np.random.default_rng(seed + 7919)
        theta0 = rng.normal(0.0, 0.05 if sigma is None else sigma, size=(n_obj, 3)) * free[:, None]
        theta = torch.from_numpy(theta0.astype(np.float32)).to(dev).requires_grad_(True)
        params = [theta]

        def verts_now():
            return v_true + onehot @ theta
        label_t = torch.from_numpy(label).to(dev)
    else:
        v = torch.from_numpy(sg.perturb_vertices(scene, seed, 0.02 if sigma is None else sigma)).to(dev)
        v.requires_grad_(True)
        params = [v]

        def verts_now():
            return v
    moved = None
    opt = torch.optim.Adam(params, lr=lr)
    hist = []
    for k in range(steps):
        if lr_final is not None:
            for grp in opt.param_groups:
                grp["lr"] = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * k / max(steps - 1, 1)))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        img = ren(verts_now(), albedo, rad, cam, scale)
        if ren_res is not None:
            with torch.no_grad():
                res = ren_res(verts_now(), albedo, rad, cam, scale) - target
            loss = ((res + img - img.detach()) ** 2).mean()  # value of the second render, gradient 2 res dI
        else:
            loss = ((img - target) ** 2).mean()
        opt.zero_grad()
        loss.backward()
        if moved is None:  # vertices (objects) the image depends on
            moved = theta.grad.abs().sum(1)[label_t] > 0 if objects else v.grad.abs().sum(1) > 0
        with torch.no_grad():  # error before this step's update (step 0: the start)
            dv = (verts_now() - v_true)[moved]
            along = (dv * normals[moved]).sum(1)
            tang = dv - along[:, None] * normals[moved]
            n_m = max(int(moved.sum().item()), 1)
            err = dv.pow(2).sum().div(n_m).sqrt().item()
            err_n = along.pow(2).sum().div(n_m).sqrt().item()
            err_t = tang.pow(2).sum().div(n_m).sqrt().item()
        opt.step()
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        rec = {"step": k, "loss": float(loss.item()), "vertex_rms_error": err, "vertex_rms_normal": err_n,
               "vertex_rms_tangent": err_t, "ms": ms}
        hist.append(rec)
        if log:
            log(rec)
    return hist


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--small", action="store_true", help="20k triangles at 128x128, depth 2, 8 spp")
    ap.add_argument("--objects", action="store_true", help="one translation per object instead of free vertices")
    ap.add_argument("--lr", type=float, default=None)
    ap.add_argument("--lr-final", type=float, default=None, help="cosine decay of the learning rate to this value")
    ap.add_argument("--decorrelate", action="store_true",
                    help="residual from a second render with independent samples")
    ap.add_argument("--seed", type=int, default=1237)
    args = ap.parse_args()
    if args.small:
        scene = sg.procedural(args.seed, n_target=20_000, width=128, height=128)
        lr = args.lr or (5e-3 if args.objects else 2e-3)
        hist = run(scene, steps=args.steps, spp=8, max_depth=2, target_spp=64, lr=lr, objects=args.objects,
                   decorrelate=args.decorrelate, lr_final=args.lr_final)
    else:
        scene = sg.procedural(args.seed)
        lr = args.lr or (5e-3 if args.objects else 1e-3)
        hist = run(scene, steps=args.steps, lr=lr, objects=args.objects, decorrelate=args.decorrelate,
                   lr_final=args.lr_final)
    for h in hist[:: max(1, len(hist) // 10)] + hist[-1:]:
        print(json.dumps(h))
    ms = [h["ms"] for h in hist[3:]] or [h["ms"] for h in hist]
    summary = {"triangles": len(scene.tris), "width": scene.width, "height": scene.height,
               "parameters": "object translations" if args.objects else "free vertices", "lr": lr,
               "lr_final": args.lr_final, "decorrelate": args.decorrelate}
    for key in ("loss", "vertex_rms_error", "vertex_rms_normal", "vertex_rms_tangent"):
        summary[key + "_first"] = hist[0][key]
        summary[key + "_last"] = hist[-1][key]
    summary["ms_per_step_median"] = float(np.median(ms))
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
