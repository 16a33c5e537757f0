"""Pins of the oracle's equidistant fisheye camera (Sec. 5.2, "Cameras with
Non-linear Projections"), whose primary edges are sampled in 3D and whose
edge images are curves.

- The FP32 atan2 of the decision path against the library's within a few
  ulp, over the whole range it is used on.
- The camera ray and the projection invert each other, and the ray leaves at
  angle r * theta_half_height from the optical axis.
- The gradient of the fisheye image (interior, primary edges along the curved
  edge images, secondary edges) against central finite differences of the
  image with common random numbers, as a z-test over seeds, with a power
  check: without the primary edge term some probe misses by many standard
  errors.
"""
import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg

NT = oracle.n_threads_default()


def test_fp32_atan2_matches_the_library():
    rng = np.random.default_rng(3)
    ys = np.abs(rng.normal(size=4000)).astype(np.float32)
    xs = rng.normal(size=4000).astype(np.float32)
    extra = [(0.0, 1.0), (1.0, 0.0), (0.0, -1.0), (1.0, 1.0), (1.0, -1.0), (0.267949194, 1.0), (1e-30, -1.0)]
    for y, x in list(zip(ys, xs)) + extra:
        got = oracle.atan2_pos(float(y), float(x))
        want = float(np.arctan2(np.float64(np.float32(y)), np.float64(np.float32(x))))
        assert abs(got - want) <= 4 * np.spacing(np.float32(max(abs(want), 1e-30))) + 1e-38, (y, x, got, want)


def test_fisheye_ray_and_projection_invert_each_other():
    scene = sg.fisheye_view(3, width=64, height=48)
    W, H = scene.width, scene.height
    M = np.asarray(scene.cam_to_world, np.float64)
    axis = -M[:3, 2] / np.linalg.norm(M[:3, 2])
    rng = np.random.default_rng(4)
    for sx, sy in rng.uniform([0, 0], [W, H], size=(300, 2)):
        o, d = oracle.camera_ray(scene, float(sx), float(sy))
        assert np.allclose(o, M[:3, 3], atol=0)
        r = np.hypot((2 * sx - W) / H, (H - 2 * sy) / H)
        dd = d.astype(np.float64) / np.linalg.norm(d)
        assert abs(np.arccos(np.clip(dd @ axis, -1, 1)) - r * scene.cam_scale) < 2e-5
        back = oracle.fisheye_project(scene, (o.astype(np.float64) + 3.0 * dd).astype(np.float32))
        assert back is not None and abs(back[0] - sx) < 2e-3 and abs(back[1] - sy) < 2e-3, (sx, sy, back)


def _perturbed(scene, kind, idx, h):
    s = scene.copy()
    if kind == "verts":
        s.verts[idx] += h
    elif kind == "cam":
        s.cam_to_world[idx] += h
    else:
        s.cam_scale = float(np.float32(s.cam_scale + h))
    return s


def _pick(sp, kind, idx):
    if kind == "verts":
        return sp["verts"][idx]
    if kind == "cam":
        return sp["cam_to_world"][idx]
    return sp["cam_scale"][0]


@pytest.mark.slow
def test_fisheye_gradient_matches_central_differences():
    scene = sg.fisheye_view(5, width=24, height=18, subdiv=1)
    V = len(scene.verts)
    w = sg.loss_adjoint(6, scene.width, scene.height)
    probes = [("verts", (0, 0)), ("verts", (5, 1)), ("verts", (17, 2)), ("verts", (V - 6, 0)), ("cam", (0, 3)),
              ("cam", (1, 3)), ("cam", (0, 2)), ("scale", None)]
    K, spp, spp_fd, h = 8, 256, 1024, 1e-2
    rows, prim = [], []
    for k in range(K):
        g, _ = oracle.backward(scene, w, spp=spp, edge_spp=spp, seed=700 + k, n_threads=NT)
        sp = oracle.split_params(scene, g)
        rows.append([_pick(sp, kind, idx) for kind, idx in probes])
        gp, _ = oracle.backward(scene, w, spp=spp, edge_spp=spp, seed=700 + k, terms=oracle.TERM_PRIMARY,
                                n_threads=NT)
        spp_ = oracle.split_params(scene, gp)
        prim.append([_pick(spp_, kind, idx) for kind, idx in probes])
    ours, prim = np.array(rows), np.array(prim)
    fd = []
    for k in range(K):
        row = []
        for kind, idx in probes:
            hh = h if kind != "scale" else h / 4
            lp = float((oracle.render(_perturbed(scene, kind, idx, hh), spp=spp_fd, seed=1900 + k, n_threads=NT)
                        * w).sum())
            lm = float((oracle.render(_perturbed(scene, kind, idx, -hh), spp=spp_fd, seed=1900 + k, n_threads=NT)
                        * w).sum())
            row.append((lp - lm) / (2 * hh))
        fd.append(row)
    fd = np.array(fd)
    se = np.sqrt(ours.var(0, ddof=1) / K + fd.var(0, ddof=1) / K + (1e-3 * np.abs(fd.mean(0)).max()) ** 2)

    def z(est):
        return np.abs(est.mean(0) - fd.mean(0)) / se

    assert np.all(z(ours) < 4.5), list(zip(probes, ours.mean(0), fd.mean(0), se))
    assert z(ours - prim).max() > 8.0
