"""Element-wise gradient parity at full workload sizes, in the launch
configuration the benchmark times.

The backward pass takes evaluation ranges (drt_render_opts.pix_begin/pix_end
and edge_begin/edge_end): the kernels still launch over the whole image and
every primary edge sample, sort all samples by screen position and reduce all
partial-sum rows, but only the samples in the ranges contribute.  The oracle
evaluates the same samples one by one, so every gradient entry is compared
with the parity tolerance of the small cases:

- direct lighting, 256x256, 5124 triangles, 64 spp + 64 edge spp (4.19 M
  primary edge samples): a row of pixels and an edge-sample range from the
  middle of the sample order;
- the procedural scene of about 200k triangles, 512x512, depth 3, 32 spp +
  32 edge spp (8.39 M primary edge samples);
- one scene of a batch (persistent launches, one sort for all scenes) and the
  allocation-free backward, against the oracle directly.
"""
import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg
from parity import assert_grads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NT = oracle.n_threads_default()


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12228_gb300 import drt
    return drt, drt.Context(0)


def _zeros(scene):
    z = lambda *sh: torch.zeros(sh, dtype=torch.float32, device="cuda")  # noqa: E731
    return dict(d_verts=z(len(scene.verts), 3), d_albedo=z(len(scene.tris), 3), d_radiance=z(3),
                d_cam_to_world=z(3, 4), d_cam_scale=z(1))


def _flat(g):
    return np.concatenate([g[k].double().cpu().numpy().ravel()
                           for k in ("d_verts", "d_albedo", "d_radiance", "d_cam_to_world", "d_cam_scale")])


def _ranged(drt, ctx, scene, w, spp, edge_spp, depth, seed, pixels, edges, leaf=1):
    S = drt.Scene.from_arrays(ctx, scene, bvh_leaf_size=leaf)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    opts = drt.make_opts(spp, edge_spp, max_depth=depth, seed=seed, pixels=pixels, edges=edges)
    tape = S.render(img, opts, want_tape=True)
    g = _zeros(scene)
    S.backward(torch.from_numpy(w).cuda(), opts, tape=tape, **g)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    return _flat(g)


def test_direct_lighting_256_full_size_elementwise(env):
    drt, ctx = env
    scene = sg.direct_lighting(1236)
    W, H, spp = scene.width, scene.height, 64
    w = sg.loss_adjoint(1, W, H)
    n_edge = spp * W * H
    pixels = ((H // 2) * W, (H // 2) * W + 2 * W)          # two full rows in the middle of the image
    edges = (n_edge // 2 - 40000, n_edge // 2 + 40000)      # 80k samples from the middle of the order
    got = _ranged(drt, ctx, scene, w, spp, spp, 1, 21, pixels, edges, leaf=2)
    want, absum, c = oracle.backward(scene, w, spp=spp, edge_spp=spp, seed=21, pixels=pixels, edges=edges,
                                     n_threads=NT, contributions=True)
    assert_grads(got, want, absum, "direct lighting 256x256 64+64 spp, full size, ranged", c)
    assert np.count_nonzero(want) > 100


def test_procedural_200k_depth3_full_size_elementwise(env):
    drt, ctx = env
    scene = sg.procedural(1237)
    W, H, spp = scene.width, scene.height, 32
    w = sg.loss_adjoint(1237, W, H)
    n_edge = spp * W * H
    p0 = (H // 2) * W + W // 2 - 12
    pixels = (p0, p0 + 24)
    edges = (n_edge // 2, n_edge // 2 + 3000)
    got = _ranged(drt, ctx, scene, w, spp, spp, 3, 4, pixels, edges)
    want, absum, c = oracle.backward(scene, w, spp=spp, edge_spp=spp, seed=4, max_depth=3, pixels=pixels,
                                     edges=edges, n_threads=NT, contributions=True)
    assert_grads(got, want, absum, "procedural 200k 512x512 depth 3 32+32 spp, full size, ranged", c)
    assert np.count_nonzero(want) > 100


def test_batch_scene_gradient_against_the_oracle(env):
    """Scene k of a batch uses scene_id k: its gradient is the oracle's with
    scene_id k (persistent passes, the shared sort, a graph replay)."""
    drt, ctx = env
    scenes = [sg.procedural(302, n_target=3000, width=37, height=23),
              sg.direct_lighting(301, width=40, height=28, subdiv=2),
              sg.single_triangle(305, width=19, height=11)]
    up = [drt.Scene.from_arrays(ctx, sc) for sc in scenes]
    d_images = [sg.loss_adjoint(600 + k, sc.width, sc.height) for k, sc in enumerate(scenes)]
    imgs = [torch.zeros((sc.height, sc.width, 3), device="cuda") for sc in scenes]
    grads = [_zeros(sc) for sc in scenes]
    b = drt.Batch(ctx, up, imgs, drt.make_opts(5, 4, seed=31), d_images=[torch.from_numpy(d).cuda() for d in d_images],
                  grads=grads, use_graph=True, autotune=False)
    b.run()
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    for k, sc in enumerate(scenes):
        want, absum, c = oracle.backward(sc, d_images[k], spp=5, edge_spp=4, seed=31, scene_id=k, n_threads=NT,
                                         contributions=True)
        assert_grads(_flat(grads[k]), want, absum, "batch scene %d" % k, c)
    b.free()


@pytest.mark.parametrize("depth", [1, 2])
def test_noalloc_backward_against_the_oracle(env, depth):
    drt, ctx = env
    scene = sg.direct_lighting(1237, width=24, height=20, subdiv=1)
    S = drt.Scene.from_arrays(ctx, scene)
    opts = drt.make_opts(6, 6, max_depth=depth, seed=5)
    img = torch.zeros((20, 24, 3), device="cuda")
    tape = S.render(img, opts, want_tape=True)
    w = sg.loss_adjoint(4, 24, 20)
    g = _zeros(scene)
    S.backward_noalloc(torch.from_numpy(w).cuda(), opts, tape=tape, **g)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    want, absum, c = oracle.backward(scene, w, spp=6, edge_spp=6, seed=5, max_depth=depth, n_threads=NT,
                                     contributions=True)
    assert_grads(_flat(g), want, absum, "noalloc depth %d" % depth, c)
