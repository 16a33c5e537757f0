"""BVH leaf size is a per-scene choice that must not change any result: the
closest hit is decided exactly (ties to the lowest triangle id) and shadow
rays only ask whether any hit exists, so images agree bit for bit and
gradients up to the order of floating-point atomic additions."""
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


def _run(drt, ctx, sc, leaf, depth):
    s = drt.Scene.from_arrays(ctx, sc, bvh_leaf_size=leaf)
    o = drt.make_opts(6, 6, max_depth=depth, seed=13)
    img = torch.zeros((sc.height, sc.width, 3), device="cuda")
    tape = s.render(img, o, want_tape=True)
    g = dict(d_verts=torch.zeros((len(sc.verts), 3), device="cuda"),
             d_albedo=torch.zeros((len(sc.tris), 3), device="cuda"), d_radiance=torch.zeros(3, device="cuda"),
             d_cam_to_world=torch.zeros((3, 4), device="cuda"), d_cam_scale=torch.zeros(1, device="cuda"))
    s.backward(torch.from_numpy(sg.loss_adjoint(31, sc.width, sc.height)).cuda(), o, tape=tape, **g)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    return img, g


@pytest.mark.parametrize("depth", [1, 3])
@pytest.mark.parametrize("scene", ["direct", "procedural", "one"])
def test_leaf_sizes_agree(env, scene, depth):
    drt, ctx = env
    sc = {"direct": lambda: sg.direct_lighting(41, width=33, height=21, subdiv=2),
          "procedural": lambda: sg.procedural(42, n_target=4000, width=29, height=27),
          "one": lambda: sg.single_triangle(43, width=17, height=9)}[scene]()
    img1, g1 = _run(drt, ctx, sc, 1, depth)
    for leaf in (2, 3, 8):
        img, g = _run(drt, ctx, sc, leaf, depth)
        assert torch.equal(img, img1), leaf
        for key in g1:
            a, b = g[key].double().cpu().numpy(), g1[key].double().cpu().numpy()
            scale = max(np.abs(b).max(), 1e-12)
            assert np.allclose(a, b, rtol=1e-4, atol=1e-5 * scale), (leaf, key)
    if depth == 1:
        want = oracle.render(sc, spp=6, seed=13, max_depth=depth, n_threads=NT)
        got = img1.double().cpu().numpy()
        assert np.all(np.abs(got - want) <= 1e-4 * np.abs(want) + 1e-7)


def test_leaf_size_out_of_range_is_rejected(env):
    drt, ctx = env
    sc = sg.single_triangle(44, width=8, height=8)
    for bad in (-1, 9):
        with pytest.raises(drt.DrtError):
            drt.Scene.from_arrays(ctx, sc, bvh_leaf_size=bad)
