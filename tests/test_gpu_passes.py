"""Sample passes (spp_per_pass): the interior samples in spp / k passes of k
samples per pixel, pass p with the Philox key seed + p * 0x9E3779B97F4A7C15,
so the checkpoint tape holds one pass (Sec. 5.4 keeps every path vertex).
Against the oracle run pass by pass: the image is the mean of the passes'
images; the gradient is the sum of the passes' interior and secondary terms
with d_image / P, plus the primary edge term once with the full edge budget.
Bounds as in the other parity tests."""
import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg
from parity import assert_grads, assert_pixels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NT = oracle.n_threads_default()
GOLD = 0x9E3779B97F4A7C15


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


def _pass_seed(seed, p):
    return (seed + p * GOLD) & (2 ** 64 - 1)


@pytest.mark.parametrize("name,depth,spp,k", [("direct", 1, 6, 2), ("procedural", 3, 6, 3), ("procedural", 2, 4, 1)])
def test_passes_match_the_oracle_pass_by_pass(env, name, depth, spp, k):
    drt, ctx = env
    scene = sg.direct_lighting(1236, width=40, height=28, subdiv=2) if name == "direct" \
        else sg.procedural(41, n_target=3000, width=29, height=27)
    w = sg.loss_adjoint(3, scene.width, scene.height)
    seed, edge_spp, P = 31, 4, spp // k
    S = drt.Scene.from_arrays(ctx, scene)
    opts = drt.make_opts(spp, edge_spp, max_depth=depth, seed=seed, spp_per_pass=k)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    S.render(img, opts)
    g = _zeros(scene)
    S.backward(torch.from_numpy(w).cuda(), opts, **g)  # no tape: every pass is rendered again
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    want_img = np.mean([oracle.render(scene, spp=k, seed=_pass_seed(seed, p), max_depth=depth, n_threads=NT)
                        for p in range(P)], axis=0)
    assert_pixels(img.cpu().numpy(), want_img, "passes %s image" % name)
    want = np.zeros(oracle.num_params(scene))
    absum = np.zeros_like(want)
    contrib = np.zeros_like(want)
    for p in range(P):
        gp, ap, cp = oracle.backward(scene, w / P, spp=k, edge_spp=edge_spp, seed=_pass_seed(seed, p),
                                     max_depth=depth, terms=5, n_threads=NT, contributions=True)
        want += gp
        absum += ap
        contrib += cp
    gp, ap, cp = oracle.backward(scene, w, spp=k, edge_spp=edge_spp, seed=seed, max_depth=depth, terms=2,
                                 n_threads=NT, contributions=True)
    want += gp
    absum += ap
    contrib += cp
    assert_grads(_flat(g), want, absum, "passes %s depth %d spp %d per pass %d" % (name, depth, spp, k), contrib)


def test_pass_options_are_checked(env):
    drt, ctx = env
    scene = sg.single_triangle(5, width=19, height=11)
    S = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    for bad in (dict(spp_per_pass=-1), dict(spp_per_pass=4)):  # spp 6 is no multiple of 4
        with pytest.raises(drt.DrtError):
            S.render(img, drt.make_opts(6, 2, **bad))
    with pytest.raises(drt.DrtError):  # a batch takes one pass
        drt.Batch(ctx, [S], [img], drt.make_opts(6, 2, spp_per_pass=3))
    # k >= spp is one pass
    a = torch.zeros_like(img)
    S.render(a, drt.make_opts(6, 2, seed=4, spp_per_pass=6))
    b = torch.zeros_like(img)
    S.render(b, drt.make_opts(6, 2, seed=4))
    torch.cuda.synchronize()
    assert torch.equal(a, b)
