"""Importance-sampled point on a secondary edge (Sec. 5.3.2, Lambertian
case: the clamped cosine over the edge's arc, mixed with uniform) on the GPU
against the oracle, element by element, on the same seeded inputs.  The point
is an FP32 decision both sides take with the same operations; its density is
evaluated in FP64 on both sides.  Bound:

  |g_gpu - g_or| <= 1e-4 |g_or| + 1e-6 A   (A: the oracle's sum of |terms|)
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


def _assert_grads(got, want, absum, label="", contrib=None):
    assert_grads(got, want, absum, label, contrib)


def _zeros(scene):
    z = lambda *sh: torch.zeros(sh, dtype=torch.float32, device="cuda")  # noqa: E731
    return dict(d_verts=z(len(scene.verts), 3), d_albedo=z(len(scene.tris), 3), d_radiance=z(3),
                d_cam_to_world=z(3, 4), d_cam_scale=z(1))


def _flat(g):
    return np.concatenate([g[k].cpu().numpy().ravel().astype(np.float64)
                           for k in ("d_verts", "d_albedo", "d_radiance", "d_cam_to_world", "d_cam_scale")])


def _scene(name):
    if name == "direct":
        return sg.direct_lighting(1236, width=40, height=28, subdiv=2)
    return sg.procedural(41, n_target=3000, width=29, height=27)


CASES = [  # scene, depth, terms, hierarchy root samples, seed
    ("direct", 1, 4, 0, 11), ("direct", 1, 7, 0, 11), ("direct", 2, 4, 0, 11), ("direct", 1, 4, 16, 11),
    ("procedural", 1, 4, 0, 12), ("procedural", 3, 4, 0, 12), ("procedural", 3, 4, 16, 12),
]


@pytest.mark.parametrize("name,depth,terms,samples,seed", CASES)
def test_point_sampling_gradient_matches_oracle(env, name, depth, terms, samples, seed):
    drt, ctx = env
    scene = _scene(name)
    w = sg.loss_adjoint(3, scene.width, scene.height)
    S = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    opts = drt.make_opts(6, 6, max_depth=depth, seed=seed, terms=terms, sec_tree_samples=samples, sec_point=1)
    tape = S.render(img, opts, want_tape=True)
    g = _zeros(scene)
    S.backward(torch.from_numpy(w).cuda(), opts, tape=tape, **g)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    want, absum, c = oracle.backward(scene, w, spp=6, edge_spp=6, seed=seed, max_depth=depth, terms=terms,
                                     sec_tree_samples=samples, sec_point=1, n_threads=NT, contributions=True)
    _assert_grads(_flat(g), want, absum, "point %s depth %d terms %d S %d" % (name, depth, terms, samples), c)
    # the importance-sampled point changes the estimate
    plain, _ = oracle.backward(scene, w, spp=6, edge_spp=6, seed=seed, max_depth=depth, terms=4,
                               sec_tree_samples=samples, n_threads=NT)
    assert not np.allclose(plain, oracle.backward(scene, w, spp=6, edge_spp=6, seed=seed, max_depth=depth, terms=4,
                                                  sec_tree_samples=samples, sec_point=1, n_threads=NT)[0])


def test_noalloc_backward_with_point_sampling(env):
    drt, ctx = env
    scene = _scene("direct")
    w = torch.from_numpy(sg.loss_adjoint(6, scene.width, scene.height)).cuda()
    S = drt.Scene.from_arrays(ctx, scene)
    opts = drt.make_opts(4, 4, seed=8, sec_point=1)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    tape = S.render(img, opts, want_tape=True)
    got = _zeros(scene)
    S.backward_noalloc(w, opts, tape=tape, **got)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    want, absum, c = oracle.backward(scene, w.cpu().numpy(), spp=4, edge_spp=4, seed=8, sec_point=1, n_threads=NT,
                                     contributions=True)
    _assert_grads(_flat(got), want, absum, "point noalloc", c)


def test_point_sampling_options_are_checked(env):
    drt, ctx = env
    scene = sg.single_triangle(5, width=19, height=11)
    S = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    w = torch.ones_like(img)
    with pytest.raises(drt.DrtError):
        S.backward(w, drt.make_opts(2, 2, sec_point=2), d_verts=torch.zeros((3, 3), device="cuda"))
    with pytest.raises(drt.DrtError):  # a batch keeps the uniform point
        drt.Batch(ctx, [S], [img], drt.make_opts(2, 2, sec_point=1))
