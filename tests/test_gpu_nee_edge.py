"""Next-event estimation for edges (Sec. 5.3.3) on the GPU against the
oracle, element by element, on the same seeded inputs: the billboard
crossings, importances, race keys and the sample's point are FP32 decisions
both sides take with the same operations; the densities and the balance
heuristic's weights are FP64 on both sides (rounded to FP32 once on the GPU).
Bound:

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


CASES = [  # scene, depth, terms, billboard width (0: from the vertices), seed
    ("direct", 1, 4, 0.0, 11), ("direct", 1, 7, 0.0, 11), ("direct", 1, 4, 0.2, 13), ("direct", 2, 4, 0.0, 11),
    ("procedural", 1, 4, 0.0, 12), ("procedural", 2, 4, 0.5, 12), ("procedural", 3, 4, 0.0, 12),
    ("procedural", 3, 7, 0.0, 14),
]


@pytest.mark.parametrize("name,depth,terms,width,seed", CASES)
def test_billboard_sampling_gradient_matches_oracle(env, name, depth, terms, width, seed):
    drt, ctx = env
    scene = _scene(name)
    w = sg.loss_adjoint(3, scene.width, scene.height)
    S = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    opts = drt.make_opts(6, 6, max_depth=depth, seed=seed, terms=terms, sec_nee=1, nee_width=width)
    tape = S.render(img, opts, want_tape=True)
    g = _zeros(scene)
    S.backward(torch.from_numpy(w).cuda(), opts, tape=tape, **g)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    want, absum, c = oracle.backward(scene, w, spp=6, edge_spp=6, seed=seed, max_depth=depth, terms=terms,
                                     sec_nee=1, nee_width=width, n_threads=NT, contributions=True)
    assert_grads(_flat(g), want, absum, "nee %s depth %d terms %d width %g" % (name, depth, terms, width), c)
    # the billboard samples change the estimate
    plain, _ = oracle.backward(scene, w, spp=6, edge_spp=6, seed=seed, max_depth=depth, terms=4, n_threads=NT)
    nee, _ = oracle.backward(scene, w, spp=6, edge_spp=6, seed=seed, max_depth=depth, terms=4, sec_nee=1,
                             nee_width=width, n_threads=NT)
    assert not np.allclose(plain, nee)


def test_billboard_sampling_after_a_vertex_update(env):
    """The hierarchy the crossing queries walk and the derived width follow
    the scene's vertices."""
    drt, ctx = env
    scene = _scene("procedural")
    moved = scene.copy()
    moved.verts = sg.perturb_vertices(scene, 3, sigma=0.01)
    w = sg.loss_adjoint(4, scene.width, scene.height)
    S = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    opts = drt.make_opts(4, 4, max_depth=2, seed=21, terms=4, sec_nee=1)
    tape = S.render(img, opts, want_tape=True)
    S.backward(torch.from_numpy(w).cuda(), opts, tape=tape, **_zeros(scene))
    S.update_vertices(torch.from_numpy(moved.verts).cuda())
    tape = S.render(img, opts, want_tape=True)
    g = _zeros(scene)
    S.backward(torch.from_numpy(w).cuda(), opts, tape=tape, **g)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    want, absum, c = oracle.backward(moved, w, spp=4, edge_spp=4, seed=21, max_depth=2, terms=4, sec_nee=1,
                                     n_threads=NT, contributions=True)
    assert_grads(_flat(g), want, absum, "nee after update", c)


def test_billboard_options_are_checked(env):
    drt, ctx = env
    scene = _scene("direct")
    S = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    w = torch.ones_like(img)
    g = _zeros(scene)
    for bad in (dict(sec_nee=2), dict(sec_nee=1, sec_tree_samples=16), dict(sec_nee=1, sec_point=1),
                dict(sec_nee=1, nee_width=float("nan"))):
        with pytest.raises(drt.DrtError):
            S.backward(w, drt.make_opts(2, 2, **bad), **g)
    opts = drt.make_opts(2, 2, sec_nee=1)
    tape = S.render(img, opts, want_tape=True)
    with pytest.raises(drt.DrtError):  # no queue without allocation
        S.backward_noalloc(w, opts, tape=tape, **g)
    with pytest.raises(drt.DrtError):  # a batch keeps the length sampler alone
        drt.Batch(ctx, [S], [img], opts)
    assert ctx.check_device() == (0, 0)
