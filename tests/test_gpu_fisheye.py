"""The equidistant fisheye camera on the GPU (Sec. 5.2, cameras with
non-linear projections) against the oracle: images, and gradients with the
primary edges sampled in 3D along the curved edge images, element by element
with the tolerance of the other parity tests."""
import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg
from parity import assert_grads, assert_pixels

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


@pytest.mark.parametrize("depth,terms,W,H", [(1, 7, 24, 18), (1, 2, 37, 23), (2, 7, 24, 18), (3, 2, 20, 16)])
def test_fisheye_image_and_gradient(env, depth, terms, W, H):
    drt, ctx = env
    scene = sg.fisheye_view(5, width=W, height=H, subdiv=2)
    S = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((H, W, 3), device="cuda")
    opts = drt.make_opts(6, 6, max_depth=depth, seed=17, terms=terms)
    tape = S.render(img, opts, want_tape=True)
    want_img = oracle.render(scene, spp=6, seed=17, max_depth=depth, n_threads=NT)
    assert_pixels(img.double().cpu().numpy(), want_img, "fisheye image depth %d" % depth)
    w = sg.loss_adjoint(18, W, H)
    g = _zeros(scene)
    S.backward(torch.from_numpy(w).cuda(), opts, tape=tape, **g)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    want, absum, c = oracle.backward(scene, w, spp=6, edge_spp=6, seed=17, max_depth=depth, terms=terms,
                                     n_threads=NT, contributions=True)
    assert_grads(_flat(g), want, absum, "fisheye depth %d terms %d %dx%d" % (depth, terms, W, H), c)
    assert np.abs(want).max() > 0


def test_fisheye_options_are_checked(env):
    drt, ctx = env
    scene = sg.fisheye_view(5, width=24, height=18, subdiv=1)
    bad = scene.copy()
    bad.cam_scale = 3.0  # the corners would look behind the camera
    with pytest.raises(drt.DrtError):
        drt.Scene.from_arrays(ctx, bad)
    S = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((18, 24, 3), device="cuda")
    with pytest.raises(drt.DrtError):
        S.segments()
    with pytest.raises(drt.DrtError):
        drt.Batch(ctx, [S], [img], drt.make_opts(2, 2))
    w = torch.ones_like(img)
    with pytest.raises(drt.DrtError):
        S.backward(w, drt.make_opts(2, 2, seg_weights=torch.ones(4, device="cuda"), terms=2),
                   d_verts=torch.zeros((len(scene.verts), 3), device="cuda"))
