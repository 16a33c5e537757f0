"""Secondary edges through the edge hierarchy (Sec. 5.3.1) on the GPU against
the oracle, element by element, on the same seeded inputs.  The hierarchy's
shape, every split and every pick are FP32 decisions both sides take with the
same operations, so the picked edges agree and the gradients meet the parity
tolerance of the length sampler:

  |g_gpu - g_or| <= 1e-4 |g_or| + 1e-6 A   (A: the oracle's sum of |terms|)
"""
import dataclasses

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


def _gpu(drt, ctx, scene, w, spp, edge_spp, seed, depth, terms, samples, S=None):
    s = S or drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    opts = drt.make_opts(spp, edge_spp, max_depth=depth, seed=seed, terms=terms, sec_tree_samples=samples)
    tape = s.render(img, opts, want_tape=True)
    g = _zeros(scene)
    s.backward(torch.from_numpy(w).cuda(), opts, tape=tape, **g)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    return _flat(g), s, tape, opts


CASES = [  # scene, depth, terms, root samples
    ("direct", 1, 4, 1), ("direct", 1, 4, 16), ("direct", 1, 7, 64), ("procedural", 1, 4, 16),
    ("direct", 2, 4, 16), ("direct", 3, 7, 4), ("procedural", 3, 4, 16), ("triangle", 1, 7, 16),
]


def _scene(name):
    if name == "direct":
        return sg.direct_lighting(1236, width=40, height=28, subdiv=2)
    if name == "procedural":
        return sg.procedural(41, n_target=3000, width=29, height=27)
    return sg.single_triangle(5, width=19, height=11)


@pytest.mark.parametrize("name,depth,terms,samples", CASES)
def test_hierarchy_gradient_matches_oracle(env, name, depth, terms, samples):
    drt, ctx = env
    scene = _scene(name)
    w = sg.loss_adjoint(3, scene.width, scene.height)
    got, _, _, _ = _gpu(drt, ctx, scene, w, 6, 6, 11, depth, terms, samples)
    want, absum, c = oracle.backward(scene, w, spp=6, edge_spp=6, seed=11, max_depth=depth, terms=terms,
                                     sec_tree_samples=samples, n_threads=NT, contributions=True)
    _assert_grads(got, want, absum, "hierarchy %s depth %d terms %d S %d" % (name, depth, terms, samples), c)
    if name != "triangle":
        # the hierarchy changes the estimate: not the length sampler's numbers
        plain, _ = oracle.backward(scene, w, spp=6, edge_spp=6, seed=11, max_depth=depth, terms=4, n_threads=NT)
        tree, _ = oracle.backward(scene, w, spp=6, edge_spp=6, seed=11, max_depth=depth, terms=4,
                                  sec_tree_samples=samples, n_threads=NT)
        assert not np.allclose(plain, tree)


def test_hierarchy_is_rebuilt_when_vertices_and_camera_change(env):
    drt, ctx = env
    scene = _scene("direct")
    w = sg.loss_adjoint(4, scene.width, scene.height)
    S = drt.Scene.from_arrays(ctx, scene)
    _gpu(drt, ctx, scene, w, 4, 4, 2, 1, 4, 16, S=S)
    moved = sg.perturb_vertices(scene, 3, sigma=0.02)
    S.update_vertices(torch.from_numpy(moved).cuda())
    cam = np.array(scene.cam_to_world, np.float32)
    cam[:3, 3] += np.array([0.05, -0.03, 0.02], np.float32)
    S.update_params(cam_to_world=torch.from_numpy(cam).cuda())
    got, _, _, _ = _gpu(drt, ctx, scene, w, 4, 4, 2, 1, 4, 16, S=S)
    scene2 = dataclasses.replace(scene, verts=moved, cam_to_world=cam)
    want, absum, c = oracle.backward(scene2, w, spp=4, edge_spp=4, seed=2, terms=4, sec_tree_samples=16, n_threads=NT,
                                     contributions=True)
    _assert_grads(got, want, absum, "hierarchy after update", c)


def test_noalloc_backward_with_the_hierarchy(env):
    drt, ctx = env
    scene = _scene("direct")
    w = torch.from_numpy(sg.loss_adjoint(6, scene.width, scene.height)).cuda()
    S = drt.Scene.from_arrays(ctx, scene)
    opts = drt.make_opts(4, 4, seed=8, sec_tree_samples=16)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    with pytest.raises(drt.DrtError):  # the hierarchy's buffers do not exist yet
        tape = S.render(img, opts, want_tape=True)
        S.backward_noalloc(w, opts, tape=tape, **_zeros(scene))
    torch.cuda.synchronize()
    tape = S.render(img, opts, want_tape=True)
    ref = _zeros(scene)
    S.backward(w, opts, tape=tape, **ref)
    got = _zeros(scene)
    S.backward_noalloc(w, opts, tape=tape, **got)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    want, absum, c = oracle.backward(scene, w.cpu().numpy(), spp=4, edge_spp=4, seed=8, sec_tree_samples=16,
                                     n_threads=NT, contributions=True)
    _assert_grads(_flat(got), want, absum, "hierarchy noalloc", c)
    _assert_grads(_flat(ref), want, absum, "hierarchy backward", c)


def test_hierarchy_options_are_checked(env):
    drt, ctx = env
    scene = _scene("triangle")
    S = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    w = torch.ones_like(img)
    with pytest.raises(drt.DrtError):
        S.backward(w, drt.make_opts(2, 2, sec_tree_samples=65), d_verts=torch.zeros((3, 3), device="cuda"))
    with pytest.raises(drt.DrtError):  # a batch samples secondary edges by length
        drt.Batch(ctx, [S], [img], drt.make_opts(2, 2, sec_tree_samples=4))


def test_noalloc_backward_rebuilds_the_hierarchy_after_an_update(env):
    """After the vertices and the camera change, the allocation-free backward
    rebuilds the hierarchy in place (kernel launches into the buffers an
    earlier backward allocated) and matches the oracle on the new scene."""
    drt, ctx = env
    scene = _scene("direct")
    w = sg.loss_adjoint(5, scene.width, scene.height)
    S = drt.Scene.from_arrays(ctx, scene)
    _gpu(drt, ctx, scene, w, 4, 4, 2, 1, 4, 16, S=S)  # allocates the hierarchy's buffers
    moved = sg.perturb_vertices(scene, 7, sigma=0.02)
    S.update_vertices(torch.from_numpy(moved).cuda())
    cam = np.array(scene.cam_to_world, np.float32)
    cam[:3, 3] += np.array([-0.04, 0.03, 0.01], np.float32)
    S.update_params(cam_to_world=torch.from_numpy(cam).cuda())
    opts = drt.make_opts(4, 4, seed=9, terms=4, sec_tree_samples=16)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    tape = S.render(img, opts, want_tape=True)
    got = _zeros(scene)
    S.backward_noalloc(torch.from_numpy(w).cuda(), opts, tape=tape, **got)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    scene2 = dataclasses.replace(scene, verts=moved, cam_to_world=cam)
    want, absum, c = oracle.backward(scene2, w, spp=4, edge_spp=4, seed=9, terms=4, sec_tree_samples=16, n_threads=NT,
                                     contributions=True)
    _assert_grads(_flat(got), want, absum, "hierarchy noalloc after update", c)
