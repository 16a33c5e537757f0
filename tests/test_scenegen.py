"""The seeded synthetic inputs match their recipes: sizes, placements and
value ranges of the scenes the tests and the benchmark use."""
import math

import numpy as np

from paper_1904_12228_gb300 import scenegen as sg


def test_direct_lighting_scene():
    sc = sg.direct_lighting(1236)
    assert (sc.width, sc.height) == (256, 256)
    assert len(sc.tris) == 5120 + 4 and len(sc.light_tris) == 2
    sphere = sc.verts[:2562]
    r = np.linalg.norm(sphere, axis=1)
    assert abs(r.mean() - 1.0) < 0.01 and r.std() < 0.02          # unit sphere + N(0, 0.01) jitter
    assert np.all((sc.albedo >= 0.2) & (sc.albedo <= 0.8))
    assert np.allclose(sc.radiance, 10.0)
    assert np.allclose(sc.cam_to_world[:3, 3], [0, 1, 5])
    lt = sc.verts[sc.tris[sc.light_tris]].reshape(-1, 3)
    assert np.allclose(lt[:, 1], 3.0)                                # light quad at y = 3
    assert math.isclose(sc.cam_scale, math.tan(math.radians(22.5)), rel_tol=1e-6)


def test_procedural_scene():
    sc = sg.procedural(1237)
    assert 200_000 <= len(sc.tris) < 200_000 + 1280 + 8
    assert (sc.width, sc.height) == (512, 512) and len(sc.light_tris) == 4
    objs = sc.verts[:-12]
    assert np.all(np.abs(objs) <= 5.0 + 1e-3)                        # objects inside [-5,5]^3
    assert np.allclose(sc.radiance, 30.0)
    assert np.all((sc.albedo >= 0.2) & (sc.albedo <= 0.8))


def test_batch_workload():
    scenes = sg.batch_workload(1238, n=64)
    t = np.array([len(sc.tris) for sc in scenes])
    res = {sc.width for sc in scenes}
    assert len(scenes) == 64 and res <= {128, 256, 512} and len(res) == 3
    assert all(sc.width == sc.height for sc in scenes)
    assert t.min() >= 1000 and t.max() < 100_000 + 1280 + 8
    lt = np.log(t)
    assert lt.max() - lt.min() > 0.8 * math.log(100)                 # spread over the log range


def test_small_batch_workload():
    scenes = sg.batch_workload(1238, t_min=300, t_max=3000, resolutions=(64, 96, 128))
    t = np.array([len(sc.tris) for sc in scenes])
    assert len(scenes) == 64 and {sc.width for sc in scenes} <= {64, 96, 128}
    assert t.min() >= 300 and t.max() < 3000 + 1280 + 8


def test_loss_adjoint_and_perturbation():
    w = sg.loss_adjoint(3, 40, 30)
    assert w.shape == (30, 40, 3) and w.dtype == np.float32
    assert w.min() >= -1.0 and w.max() <= 1.0 and abs(w.mean()) < 0.05
    sc = sg.direct_lighting(1236, width=16, height=16, subdiv=1)
    v = sg.perturb_vertices(sc, 5, sigma=0.02)
    d = v - sc.verts
    assert abs(d.std() - 0.02) < 0.005 and np.array_equal(v, sg.perturb_vertices(sc, 5, sigma=0.02))
