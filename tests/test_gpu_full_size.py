"""Parity at full workload sizes, on outputs the oracle computes one at a
time (sampled pixels) and on properties that hold at any size.

- Procedural scene of about 200k triangles, 512x512, 32 spp, path tracing to
  depth 3 (the inverse-rendering workload).
- The 64-scene batch (1k-100k triangles, 128^2-512^2, 16 spp direct lighting)
  in the launch configuration the benchmark times: persistent launches in a
  CUDA graph with tuned shapes.
"""
import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NT = oracle.n_threads_default()


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12228_gb300 import drt
    return drt, drt.Context(0)


def _assert_pixel(got, want):
    assert np.all(np.abs(got - want) <= 1e-4 * np.abs(want) + 1e-7), (got, want)


def test_procedural_200k_depth3_sampled_pixels_and_invariants(env):
    drt, ctx = env
    scene = sg.procedural(1237)
    W, H, spp = scene.width, scene.height, 32
    s = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((H, W, 3), device="cuda")
    opts = drt.make_opts(spp, spp, max_depth=3, seed=4)
    tape = s.render(img, opts, want_tape=True)
    w = sg.loss_adjoint(1237, W, H)
    V, T = len(scene.verts), len(scene.tris)
    g = dict(d_verts=torch.zeros((V, 3), device="cuda"), d_albedo=torch.zeros((T, 3), device="cuda"),
             d_radiance=torch.zeros(3, device="cuda"), d_cam_to_world=torch.zeros((3, 4), device="cuda"),
             d_cam_scale=torch.zeros(1, device="cuda"))
    s.backward(torch.from_numpy(w).cuda(), opts, tape=tape, **g)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    got = img.double().cpu().numpy()
    rng = np.random.default_rng(2)
    for p in rng.choice(W * H, size=6, replace=False):
        want = oracle.render(scene, spp=spp, seed=4, max_depth=3, pixels=(int(p), int(p) + 1), n_threads=NT)
        y, x = divmod(int(p), W)
        _assert_pixel(got[y, x], want[y, x])
    # the image is linear in the light radiance (all bounces): sum Le dLe = sum w I
    dLe = g["d_radiance"].double().cpu().numpy()
    lhs = float((np.asarray(scene.radiance, np.float64) * dLe).sum())
    rhs = float((w.astype(np.float64) * got).sum())
    assert abs(lhs - rhs) <= 1e-4 * abs(rhs) + 1e-3, (lhs, rhs)
    # and invariant under a joint translation of scene and camera
    dv = g["d_verts"].double().cpu().numpy()
    dcam = g["d_cam_to_world"].double().cpu().numpy()
    total = dv.sum(0) + dcam[:, 3]
    assert np.all(np.abs(total) <= 2e-3 * np.abs(dv).sum(0) + 1e-3), total


def test_batch_of_64_scenes_sampled_pixels(env):
    drt, ctx = env
    scenes = sg.batch_workload(1238)
    up = [drt.Scene.from_arrays(ctx, sc) for sc in scenes]
    d_images = [torch.from_numpy(sg.loss_adjoint(1238 + k, sc.width, sc.height)).cuda() for k, sc in enumerate(scenes)]
    imgs = [torch.zeros((sc.height, sc.width, 3), device="cuda") for sc in scenes]
    grads = [dict(d_verts=torch.zeros((len(sc.verts), 3), device="cuda"),
                  d_albedo=torch.zeros((len(sc.tris), 3), device="cuda"), d_radiance=torch.zeros(3, device="cuda"),
                  d_cam_to_world=torch.zeros((3, 4), device="cuda"), d_cam_scale=torch.zeros(1, device="cuda"))
             for sc in scenes]
    b = drt.Batch(ctx, up, imgs, drt.make_opts(16, 16, seed=7), d_images=d_images, grads=grads, use_graph=True,
                  autotune=True)
    b.run()
    b.run()  # a graph replay
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    assert b.info()["graph"]
    rng = np.random.default_rng(3)
    picks = [0, int(np.argmax([len(sc.tris) for sc in scenes])), 63]
    for k in picks:
        sc = scenes[k]
        got = imgs[k].double().cpu().numpy()
        for p in rng.choice(sc.width * sc.height, size=3, replace=False):
            want = oracle.render(sc, spp=16, seed=7, scene_id=k, pixels=(int(p), int(p) + 1), n_threads=NT)
            y, x = divmod(int(p), sc.width)
            _assert_pixel(got[y, x], want[y, x])
    # gradients of two replays: every scene's image is linear in its radiance
    for k in picks:
        sc = scenes[k]
        dLe = grads[k]["d_radiance"].double().cpu().numpy()
        lhs = float((np.asarray(sc.radiance, np.float64) * dLe).sum())
        rhs = 2.0 * float((d_images[k].double().cpu().numpy() * imgs[k].double().cpu().numpy()).sum())
        assert abs(lhs - rhs) <= 1e-4 * abs(rhs) + 1e-3, (k, lhs, rhs)
    b.free()
