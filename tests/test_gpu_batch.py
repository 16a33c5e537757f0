"""Batched scenes: persistent launches, one screen sort, CUDA graph and
autotuner.  Scene k of a batch must reproduce the single-scene calls with
scene_id k: images bit for bit, gradients up to the order of floating-point
atomic additions."""
import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NT = oracle.n_threads_default()
GRAD_KEYS = ("d_verts", "d_albedo", "d_radiance", "d_cam_to_world", "d_cam_scale")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12228_gb300 import drt
    return drt, drt.Context(0)


def _scenes():
    return [sg.direct_lighting(301, width=40, height=28, subdiv=2),
            sg.procedural(302, n_target=3000, width=37, height=23),
            sg.direct_lighting(303, width=16, height=16, subdiv=1),
            sg.procedural(304, n_target=1500, width=48, height=48),
            sg.single_triangle(305, width=19, height=11)]


def _grads(sc):
    return dict(d_verts=torch.zeros((len(sc.verts), 3), device="cuda"),
                d_albedo=torch.zeros((len(sc.tris), 3), device="cuda"),
                d_radiance=torch.zeros(3, device="cuda"), d_cam_to_world=torch.zeros((3, 4), device="cuda"),
                d_cam_scale=torch.zeros(1, device="cuda"))


def _single(drt, ctx, scenes, uploaded, d_images, spp, edge_spp, depth, seed):
    imgs, grads = [], []
    for k, (sc, s) in enumerate(zip(scenes, uploaded)):
        o = drt.make_opts(spp, edge_spp, max_depth=depth, seed=seed, scene_id=k)
        img = torch.zeros((sc.height, sc.width, 3), device="cuda")
        tape = s.render(img, o, want_tape=True)
        g = _grads(sc)
        s.backward(d_images[k], o, tape=tape, **g)
        imgs.append(img)
        grads.append(g)
    torch.cuda.synchronize()
    return imgs, grads


def _assert_grads_close(gb, gs, what):
    for key in GRAD_KEYS:
        a = gb[key].double().cpu().numpy()
        b = gs[key].double().cpu().numpy()
        scale = max(np.abs(b).max(), 1e-12)
        assert np.allclose(a, b, rtol=1e-4, atol=1e-5 * scale), (what, key, np.abs(a - b).max(), scale)


@pytest.mark.parametrize("use_graph,autotune,depth", [(False, False, 1), (True, False, 1), (True, True, 1),
                                                      (True, False, 2)])
def test_batch_equals_single_scene_calls(env, use_graph, autotune, depth):
    drt, ctx = env
    scenes = _scenes()
    up = [drt.Scene.from_arrays(ctx, sc) for sc in scenes]
    d_images = [torch.from_numpy(sg.loss_adjoint(400 + k, sc.width, sc.height)).cuda() for k, sc in enumerate(scenes)]
    spp, edge_spp, seed = 5, 3, 77
    imgs_s, grads_s = _single(drt, ctx, scenes, up, d_images, spp, edge_spp, depth, seed)
    imgs_b = [torch.zeros((sc.height, sc.width, 3), device="cuda") for sc in scenes]
    grads_b = [_grads(sc) for sc in scenes]
    b = drt.Batch(ctx, up, imgs_b, drt.make_opts(spp, edge_spp, max_depth=depth, seed=seed), d_images=d_images,
                  grads=grads_b, use_graph=use_graph, autotune=autotune)
    b.run()
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    info = b.info()
    assert info["graph"] == use_graph and info["tuned"] == autotune
    for k in range(len(scenes)):
        assert torch.equal(imgs_b[k], imgs_s[k]), k
        _assert_grads_close(grads_b[k], grads_s[k], "scene %d" % k)
    if not autotune:  # same partial-sum rows and order: global gradients bit for bit
        for k in range(len(scenes)):
            for key in ("d_radiance", "d_cam_to_world", "d_cam_scale"):
                assert torch.equal(grads_b[k][key], grads_s[k][key]), (k, key)
    b.free()


def test_graph_replays_accumulate(env):
    drt, ctx = env
    scenes = _scenes()[:3]
    up = [drt.Scene.from_arrays(ctx, sc) for sc in scenes]
    d_images = [torch.from_numpy(sg.loss_adjoint(500 + k, sc.width, sc.height)).cuda() for k, sc in enumerate(scenes)]
    imgs_s, grads_s = _single(drt, ctx, scenes, up, d_images, 4, 4, 1, 5)
    imgs_b = [torch.zeros((sc.height, sc.width, 3), device="cuda") for sc in scenes]
    grads_b = [_grads(sc) for sc in scenes]
    b = drt.Batch(ctx, up, imgs_b, drt.make_opts(4, 4, seed=5), d_images=d_images, grads=grads_b, use_graph=True,
                  autotune=False)
    for _ in range(3):
        b.run()
    torch.cuda.synchronize()
    for k in range(3):
        assert torch.equal(imgs_b[k], imgs_s[k])
        for key in GRAD_KEYS:
            a = grads_b[k][key].double().cpu().numpy()
            want = 3.0 * grads_s[k][key].double().cpu().numpy()
            scale = max(np.abs(want).max(), 1e-12)
            assert np.allclose(a, want, rtol=1e-4, atol=1e-5 * scale), (k, key)


def test_vertex_updates_inside_the_batch(env):
    drt, ctx = env
    scenes = _scenes()[:2]
    moved = [sg.perturb_vertices(sc, 9 + k, sigma=0.01) for k, sc in enumerate(scenes)]
    # reference: update each scene, then single-scene calls
    ref = [drt.Scene.from_arrays(ctx, sc) for sc in scenes]
    for s, v in zip(ref, moved):
        s.update_vertices(torch.from_numpy(v).cuda())
    d_images = [torch.from_numpy(sg.loss_adjoint(600 + k, sc.width, sc.height)).cuda() for k, sc in enumerate(scenes)]
    imgs_s, grads_s = _single(drt, ctx, scenes, ref, d_images, 3, 2, 1, 11)
    up = [drt.Scene.from_arrays(ctx, sc) for sc in scenes]
    vt = [torch.from_numpy(v).cuda() for v in moved]
    imgs_b = [torch.zeros((sc.height, sc.width, 3), device="cuda") for sc in scenes]
    grads_b = [_grads(sc) for sc in scenes]
    b = drt.Batch(ctx, up, imgs_b, drt.make_opts(3, 2, seed=11), d_images=d_images, grads=grads_b, verts=vt,
                  use_graph=True, autotune=False)
    b.run()
    torch.cuda.synchronize()
    for k in range(2):
        assert torch.equal(imgs_b[k], imgs_s[k])
        _assert_grads_close(grads_b[k], grads_s[k], "moved scene %d" % k)


def test_forward_only_items_and_one_shot_call(env):
    drt, ctx = env
    scenes = _scenes()[:3]
    up = [drt.Scene.from_arrays(ctx, sc) for sc in scenes]
    d_images = [torch.from_numpy(sg.loss_adjoint(700 + k, sc.width, sc.height)).cuda() for k, sc in enumerate(scenes)]
    imgs_s, grads_s = _single(drt, ctx, scenes, up, d_images, 2, 2, 1, 3)
    imgs_b = [torch.zeros((sc.height, sc.width, 3), device="cuda") for sc in scenes]
    grads_b = [_grads(sc) for sc in scenes]
    drt.render_batch(ctx, up, imgs_b, drt.make_opts(2, 2, seed=3), d_images=d_images, grads=grads_b)
    for k in range(3):
        assert torch.equal(imgs_b[k], imgs_s[k])
        _assert_grads_close(grads_b[k], grads_s[k], "one-shot scene %d" % k)
    # images only: no backward pass, gradients untouched
    imgs_f = [torch.zeros((sc.height, sc.width, 3), device="cuda") for sc in scenes]
    gz = [_grads(sc) for sc in scenes]
    drt.render_batch(ctx, up, imgs_f, drt.make_opts(2, 2, seed=3), grads=gz)
    for k in range(3):
        assert torch.equal(imgs_f[k], imgs_s[k])
        assert all(float(v.abs().sum()) == 0.0 for v in gz[k].values())


def test_scene_counter_matches_the_oracle(env):
    drt, ctx = env
    sc = sg.direct_lighting(311, width=24, height=20, subdiv=1)
    s = drt.Scene.from_arrays(ctx, sc)
    img = torch.zeros((20, 24, 3), device="cuda")
    s.render(img, drt.make_opts(4, 4, seed=21, scene_id=6))
    torch.cuda.synchronize()
    want = oracle.render(sc, spp=4, seed=21, scene_id=6, n_threads=NT)
    got = img.double().cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-4 * np.abs(want) + 1e-7)
    other = oracle.render(sc, spp=4, seed=21, scene_id=0, n_threads=NT)
    assert not np.allclose(other, want)


def test_batch_autotuner_reports_its_shapes(env):
    drt, ctx = env
    scenes = _scenes()
    up = [drt.Scene.from_arrays(ctx, sc) for sc in scenes]
    d_images = [torch.from_numpy(sg.loss_adjoint(800 + k, sc.width, sc.height)).cuda() for k, sc in enumerate(scenes)]
    imgs = [torch.zeros((sc.height, sc.width, 3), device="cuda") for sc in scenes]
    grads = [_grads(sc) for sc in scenes]
    b = drt.Batch(ctx, up, imgs, drt.make_opts(6, 6, seed=1), d_images=d_images, grads=grads, use_graph=True,
                  autotune=True)
    b.run()
    torch.cuda.synchronize()
    info = b.info()
    assert info["tuned"] and info["graph"] and info["tune_ms"] > 0
    assert info["edge_per_thread_mult"] in (1, 2, 4)
    for nm, p in info["passes"].items():
        if p["items"] == 0:
            assert p["grid"] == 0
            continue
        assert 1 <= p["ctas_per_sm"] <= 16 and p["chunk"] in (1, 2, 4, 8)
        assert 1 <= p["grid"] <= p["items"]
    assert info["edge_samples"] == sum(6 * sc.width * sc.height for sc in scenes)
    # a second batch of the same class reuses the tuned shapes
    b2 = drt.Batch(ctx, up, imgs, drt.make_opts(6, 6, seed=1), d_images=d_images, grads=grads, use_graph=False,
                   autotune=True)
    assert b2.info()["tuned"]


def test_batch_rejects_bad_arguments(env):
    drt, ctx = env
    sc = sg.direct_lighting(321, width=8, height=8, subdiv=1)
    s = drt.Scene.from_arrays(ctx, sc)
    img = torch.zeros((8, 8, 3), device="cuda")
    n_seg = s.num_segments()
    w = torch.ones(n_seg, device="cuda")
    with pytest.raises(drt.DrtError):
        drt.Batch(ctx, [s], [img], drt.make_opts(2, 2, seg_weights=w))
    with pytest.raises(drt.DrtError):  # host image
        drt.Batch(ctx, [s], [torch.zeros((8, 8, 3))], drt.make_opts(2, 2))
    with pytest.raises(drt.DrtError):
        drt.Batch(ctx, [], [], drt.make_opts(2, 2))
