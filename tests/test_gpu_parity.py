"""CUDA path against the CPU oracle, element by element, on the same seeded
inputs (run on the GB300 machine: ``pytest -m gpu``).

Tolerances (floating point, FP32 kernels vs the oracle's FP64 smooth values
and FP64 sums, identical discrete decisions):
  pixels     |I_gpu - I_or| <= 1e-4 |I_or| + 1e-7
  gradients  |g_gpu - g_or| <= 1e-4 |g_or| + 1e-6 A,  A = the oracle's
             magnitude of the terms summed into that entry (the chain rule
             taken with absolute values, and |f_u|+|f_l| for an edge sample's
             radiance difference); the second term bounds FP32 rounding of
             contributions that are small by cancellation and of the
             unordered atomic sums.
"""
import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg
from parity import assert_grads, assert_pixels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NT = oracle.n_threads_default()


@pytest.fixture(scope="module")
def drt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12228_gb300 import drt as d
    d.load()
    return d


@pytest.fixture(scope="module")
def ctx(drt):
    return drt.Context(0)


def gpu_render(drt, ctx, scene, spp, seed, primary_only=False, edge_spp=None, want_tape=False, max_depth=1):
    s = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((scene.height, scene.width, 3), dtype=torch.float32, device="cuda")
    opts = drt.make_opts(spp, edge_spp, max_depth=max_depth, primary_only=primary_only, seed=seed)
    tape = s.render(img, opts, want_tape=want_tape)
    torch.cuda.synchronize()
    return s, img, tape, opts


def gpu_grads(drt, ctx, scene, d_image, spp, edge_spp, seed, primary_only=False, terms=7, use_tape=True):
    s, img, tape, _ = gpu_render(drt, ctx, scene, spp, seed, primary_only, edge_spp, want_tape=use_tape)
    opts = drt.make_opts(spp, edge_spp, primary_only=primary_only, seed=seed, terms=terms)
    dv = torch.zeros((len(scene.verts), 3), dtype=torch.float32, device="cuda")
    da = torch.zeros((len(scene.tris), 3), dtype=torch.float32, device="cuda")
    dr = torch.zeros(3, dtype=torch.float32, device="cuda")
    dc = torch.zeros((3, 4), dtype=torch.float32, device="cuda")
    ds = torch.zeros(1, dtype=torch.float32, device="cuda")
    w = torch.from_numpy(d_image).cuda()
    s.backward(w, opts, tape=tape if use_tape else None, d_verts=dv, d_albedo=da, d_radiance=dr, d_cam_to_world=dc,
               d_cam_scale=ds)
    torch.cuda.synchronize()
    code, info = ctx.check_device()
    assert code == 0, (code, info)
    flat = np.concatenate([x.cpu().numpy().ravel().astype(np.float64) for x in (dv, da, dr, dc, ds)])
    return flat, img.cpu().numpy()


# ---------------------------------------------------------------------------
def test_library_exports_and_context(drt, ctx):
    lib = drt.load()
    for name in drt.EXPORTED:
        assert hasattr(lib, name)
    assert b"sm_103a" in lib.drt_version()


def test_traversal_matches_brute_force(drt, ctx):
    scene = sg.direct_lighting(1236, width=8, height=8, subdiv=3)
    s = drt.Scene.from_arrays(ctx, scene)
    rng = np.random.default_rng(1)
    n = 20000
    o = (np.array([0.0, 1.0, 5.0]) + rng.normal(0, 0.2, (n, 3))).astype(np.float32)
    d = (rng.normal(0, 0.35, (n, 3)) + np.array([0, -0.2, -1.0])).astype(np.float32)
    # rays aimed exactly at vertices and edge midpoints stress the watertight test
    tgt = np.concatenate([scene.verts[:2000], 0.5 * (scene.verts[scene.tris[:2000, 0]] + scene.verts[scene.tris[:2000, 1]])])
    o2 = np.tile(np.array([0.3, 0.9, 4.0], np.float32), (len(tgt), 1))
    o = np.concatenate([o, o2]).astype(np.float32)
    d = np.concatenate([d, (tgt - o2)]).astype(np.float32)
    tri = torch.zeros(len(o), dtype=torch.int32, device="cuda")
    tb = torch.zeros((len(o), 3), dtype=torch.float32, device="cuda")
    s.closest(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), tri, tb)
    torch.cuda.synchronize()
    want_tri, want_tb = oracle.closest(scene, o, d, n_threads=NT)
    got_tri = tri.cpu().numpy()
    assert (got_tri == want_tri).all(), np.nonzero(got_tri != want_tri)[0][:10]
    hit = want_tri >= 0
    assert np.array_equal(tb.cpu().numpy()[hit], want_tb[hit])


@pytest.mark.parametrize("n_tris", [2, 3, 4, 5, 9, 300])
def test_traversal_small_and_random_soups(drt, ctx, n_tris):
    """Tiny meshes (the root itself may be a leaf range) and random triangle
    soups with overlaps: traversal returns exactly the brute-force hit."""
    rng = np.random.default_rng(n_tris)
    verts = rng.uniform(-1, 1, size=(3 * n_tris, 3))
    tris = np.arange(3 * n_tris).reshape(n_tris, 3)
    scene = sg.Scene(verts=verts, tris=tris, albedo=np.full((n_tris, 3), 0.5), light_tris=np.zeros(0, np.int32),
                     radiance=[0, 0, 0], cam_to_world=np.eye(4), cam_scale=1.0, cam_type=1, width=4, height=4)
    s = drt.Scene.from_arrays(ctx, scene)
    n = 5000
    o = rng.uniform(-2, 2, size=(n, 3)).astype(np.float32)
    d = (rng.uniform(-1, 1, size=(n, 3)) - 0.5 * o).astype(np.float32)
    tri = torch.zeros(n, dtype=torch.int32, device="cuda")
    tb = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    s.closest(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), tri, tb)
    torch.cuda.synchronize()
    want_tri, want_tb = oracle.closest(scene, o, d, n_threads=NT)
    assert (tri.cpu().numpy() == want_tri).all()
    hit = want_tri >= 0
    assert hit.any()
    assert np.array_equal(tb.cpu().numpy()[hit], want_tb[hit])


@pytest.mark.parametrize("seed", [1235, 7])
def test_single_triangle_image(drt, ctx, seed):
    scene = sg.single_triangle(seed)
    _, img, _, _ = gpu_render(drt, ctx, scene, 16, seed, primary_only=True)
    want = oracle.render(scene, spp=16, seed=seed, primary_only=True, n_threads=NT)
    assert_pixels(img.cpu().numpy().astype(np.float64), want)


@pytest.mark.parametrize("seed", [1235, 7])
def test_single_triangle_gradient(drt, ctx, seed):
    scene = sg.single_triangle(seed)
    w = sg.loss_adjoint(seed, scene.width, scene.height)
    got, _ = gpu_grads(drt, ctx, scene, w, 16, 16, seed, primary_only=True)
    want, absum, c = oracle.backward(scene, w, spp=16, edge_spp=16, seed=seed, primary_only=True, n_threads=NT,
                                     contributions=True)
    assert_grads(got, want, absum, "single triangle", c)
    assert np.abs(want[:9]).max() > 0


def _small_lit(seed=1236, W=40, H=28, subdiv=2):
    return sg.direct_lighting(seed, width=W, height=H, subdiv=subdiv)


def test_direct_lighting_image(drt, ctx):
    scene = _small_lit()
    _, img, _, _ = gpu_render(drt, ctx, scene, 8, 11)
    want = oracle.render(scene, spp=8, seed=11, n_threads=NT)
    assert_pixels(img.cpu().numpy().astype(np.float64), want)


@pytest.mark.parametrize("terms", [1, 2, 4, 7])
def test_direct_lighting_gradient_terms(drt, ctx, terms):
    scene = _small_lit()
    w = sg.loss_adjoint(3, scene.width, scene.height)
    got, _ = gpu_grads(drt, ctx, scene, w, 8, 8, 11, terms=terms)
    want, absum, c = oracle.backward(scene, w, spp=8, edge_spp=8, seed=11, terms=terms, n_threads=NT, contributions=True)
    assert_grads(got, want, absum, "direct lighting 40x28 terms=%d" % terms, c)


def gpu_grads_depth(drt, ctx, scene, d_image, spp, seed, depth, terms=7):
    s = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((scene.height, scene.width, 3), dtype=torch.float32, device="cuda")
    opts = drt.make_opts(spp, spp, max_depth=depth, seed=seed, terms=terms)
    tape = s.render(img, opts, want_tape=True)
    z = lambda *sh: torch.zeros(sh, dtype=torch.float32, device="cuda")  # noqa: E731
    dv, da, dr, dc, ds = z(len(scene.verts), 3), z(len(scene.tris), 3), z(3), z(3, 4), z(1)
    s.backward(torch.from_numpy(d_image).cuda(), opts, tape=tape, d_verts=dv, d_albedo=da, d_radiance=dr,
               d_cam_to_world=dc, d_cam_scale=ds)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    flat = np.concatenate([x.cpu().numpy().ravel().astype(np.float64) for x in (dv, da, dr, dc, ds)])
    return flat, img.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("depth", [2, 3])
def test_path_tracing_image(drt, ctx, depth):
    scene = _small_lit(W=24, H=18, subdiv=1)
    _, img = gpu_grads_depth(drt, ctx, scene, np.zeros((18, 24, 3), np.float32), 6, 4, depth)
    want = oracle.render(scene, spp=6, seed=4, max_depth=depth, n_threads=NT)
    assert_pixels(img, want)
    assert not np.allclose(want, oracle.render(scene, spp=6, seed=4, max_depth=1, n_threads=NT))


@pytest.mark.parametrize("depth,terms", [(2, 1), (2, 2), (2, 4), (3, 1), (3, 4), (3, 7)])
def test_path_tracing_gradient_terms(drt, ctx, depth, terms):
    scene = _small_lit(W=24, H=18, subdiv=1)
    w = sg.loss_adjoint(9, 24, 18)
    got, _ = gpu_grads_depth(drt, ctx, scene, w, 6, 4, depth, terms)
    want, absum, c = oracle.backward(scene, w, spp=6, edge_spp=6, seed=4, max_depth=depth, terms=terms, n_threads=NT,
                                     contributions=True)
    assert_grads(got, want, absum, "lit 24x18 depth %d terms %d" % (depth, terms), c)
    assert np.abs(want).max() > 0


@pytest.mark.parametrize("depth,seed", [(2, 12), (3, 12), (2, 11), (3, 11)])
def test_path_tracing_procedural(drt, ctx, depth, seed):
    # many short, distant edges: the secondary term's cross products of nearly
    # parallel vectors and near-cancelling side pairs
    scene = sg.procedural(41, n_target=3000, width=29, height=27)
    w = sg.loss_adjoint(3, scene.width, scene.height)
    got, _ = gpu_grads_depth(drt, ctx, scene, w, 6, seed, depth, 4)
    want, absum, c = oracle.backward(scene, w, spp=6, edge_spp=6, seed=seed, max_depth=depth, terms=4, n_threads=NT,
                                     contributions=True)
    assert_grads(got, want, absum, "procedural depth %d seed %d secondary" % (depth, seed), c)
    assert np.abs(want).max() > 0


def test_backward_without_tape_matches_with_tape(drt, ctx):
    scene = _small_lit(W=24, H=16)
    w = sg.loss_adjoint(5, scene.width, scene.height)
    a, _ = gpu_grads(drt, ctx, scene, w, 4, 4, 3, use_tape=True)
    b, _ = gpu_grads(drt, ctx, scene, w, 4, 4, 3, use_tape=False)
    want, absum, c = oracle.backward(scene, w, spp=4, edge_spp=4, seed=3, n_threads=NT, contributions=True)
    assert_grads(a, want, absum, "tape", c)
    assert_grads(b, want, absum, "no tape", c)


def test_ragged_sizes_and_spp(drt, ctx):
    """Odd image sizes, spp not a power of two, a single pixel, spp=1."""
    for (W, H, spp) in ((13, 7, 3), (1, 1, 5), (17, 9, 1), (5, 3, 33)):
        scene = _small_lit(W=W, H=H, subdiv=1)
        _, img, _, _ = gpu_render(drt, ctx, scene, spp, 5)
        want = oracle.render(scene, spp=spp, seed=5, n_threads=NT)
        assert_pixels(img.cpu().numpy().astype(np.float64), want)
        w = sg.loss_adjoint(W, W, H)
        got, _ = gpu_grads(drt, ctx, scene, w, spp, spp, 5)
        g, a, c = oracle.backward(scene, w, spp=spp, edge_spp=spp, seed=5, n_threads=NT, contributions=True)
        assert_grads(got, g, a, "%dx%d spp=%d" % (W, H, spp), c)


def test_render_is_deterministic(drt, ctx):
    scene = _small_lit(W=32, H=32)
    _, a, _, _ = gpu_render(drt, ctx, scene, 16, 9)
    _, b, _, _ = gpu_render(drt, ctx, scene, 16, 9)
    assert torch.equal(a, b)


def test_host_buffers_match_device_buffers(drt, ctx):
    scene = _small_lit(W=16, H=12, subdiv=1)
    s = drt.Scene.from_arrays(ctx, scene)
    opts = drt.make_opts(4, 4, seed=2)
    dev = torch.zeros((12, 16, 3), dtype=torch.float32, device="cuda")
    host = np.zeros((12, 16, 3), np.float32)
    s.render(dev, opts)
    s.render(host, opts)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), host)


def test_invalid_arguments_are_rejected(drt, ctx):
    scene = _small_lit(W=8, H=8, subdiv=1)
    bad = scene.copy()
    bad.tris = bad.tris.copy()
    bad.tris[0, 0] = len(bad.verts) + 5
    with pytest.raises(drt.DrtError) as e:
        drt.Scene.from_arrays(ctx, bad)
    assert e.value.status == 1
    s = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((8, 8, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(drt.DrtError):
        s.render(img, drt.make_opts(0))
    # a tape from another scene is refused
    s2 = drt.Scene.from_arrays(ctx, scene)
    tape = s2.render(img, drt.make_opts(2, seed=1), want_tape=True)
    with pytest.raises(drt.DrtError) as e:
        s.backward(torch.zeros_like(img), drt.make_opts(2, seed=1), tape=tape,
                   d_verts=torch.zeros((len(scene.verts), 3), device="cuda"))
    assert e.value.status == 6


def test_nonfinite_vertices_raise_the_device_flag(drt, ctx):
    scene = _small_lit(W=8, H=8, subdiv=1)
    bad = scene.copy()
    bad.verts[3, 1] = np.nan
    s = drt.Scene.from_arrays(ctx, bad)
    code, info = ctx.check_device()
    assert code == 2 and info == 3 * 3 + 1
    assert ctx.check_device() == (0, 0)
    del s


# ---------------------------------------------------------------------------
# Full-size direct-lighting workload (256x256, 5124 triangles, 64 spp)
# ---------------------------------------------------------------------------
def test_full_size_image_on_sampled_pixels(drt, ctx):
    scene = sg.direct_lighting(1236)
    _, img, _, _ = gpu_render(drt, ctx, scene, 64, 1)
    got = img.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(0)
    for p in rng.choice(scene.width * scene.height, size=24, replace=False):
        want = oracle.render(scene, spp=64, seed=1, pixels=(int(p), int(p) + 1), n_threads=NT)
        y, x = divmod(int(p), scene.width)
        assert_pixels(got[y, x], want[y, x])


def test_full_size_gradient_invariants(drt, ctx):
    """Properties that hold at any size: the image is invariant under a joint
    translation of the scene and camera, and linear in the light radiance."""
    scene = sg.direct_lighting(1236)
    w = sg.loss_adjoint(1, scene.width, scene.height)
    got, img = gpu_grads(drt, ctx, scene, w, 64, 64, 1)
    V, T = len(scene.verts), len(scene.tris)
    dv = got[:3 * V].reshape(V, 3)
    dcam = got[3 * V + 3 * T + 3:3 * V + 3 * T + 15].reshape(3, 4)
    total = dv.sum(0) + dcam[:, 3]
    assert np.all(np.abs(total) <= 2e-3 * np.abs(dv).sum(0) + 1e-3), total
    dLe = got[3 * V + 3 * T:3 * V + 3 * T + 3]
    lhs = float((scene.radiance * dLe).sum())
    rhs = float((w.astype(np.float64) * img).sum())
    assert abs(lhs - rhs) <= 1e-4 * abs(rhs) + 1e-3


# ---------------------------------------------------------------------------
# Learned-proposal estimator: tile segments and the mixture proposal
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("W,H", [(40, 28), (256, 256)])
def test_segments_match_oracle(drt, ctx, W, H):
    scene = _small_lit(W=W, H=H, subdiv=2)
    s = drt.Scene.from_arrays(ctx, scene)
    e, t, s01, ln = s.segments()
    we, wt, ws, wl = oracle.segments(scene)
    assert len(e) == len(we)
    assert np.array_equal(e, we) and np.array_equal(t, wt)
    assert np.array_equal(s01, ws)
    assert np.allclose(ln, wl, rtol=1e-15, atol=0)


@pytest.mark.parametrize("spp,mode", [(4, "weights"), (9, "weights"), (5, "scores")])
def test_mixture_proposal_gradient(drt, ctx, spp, mode):
    scene = _small_lit(W=40, H=28, subdiv=2)
    s = drt.Scene.from_arrays(ctx, scene)
    n_seg = len(s.segments()[0])
    rng = np.random.default_rng(spp)
    if mode == "weights":
        weights = (rng.exponential(size=n_seg) ** 2).astype(np.float32)
    else:  # network scores, some beyond the clamp range
        weights = (4.0 * rng.normal(size=n_seg)).astype(np.float32)
        weights[::17] = 55.0
        weights[5::17] = -70.0
    wt = torch.from_numpy(weights).cuda()
    img = torch.zeros((28, 40, 3), device="cuda")
    tape = s.render(img, drt.make_opts(spp, spp, seed=3), want_tape=True)
    dv = torch.zeros((len(scene.verts), 3), device="cuda")
    w = sg.loss_adjoint(8, 40, 28)
    kw = {"seg_weights": wt} if mode == "weights" else {"seg_scores": wt}
    s.backward(torch.from_numpy(w).cuda(), drt.make_opts(spp, spp, seed=3, terms=2, **kw), tape=tape, d_verts=dv)
    torch.cuda.synchronize()
    got = dv.double().cpu().numpy().ravel()
    okw = {"proposal_weights": weights} if mode == "weights" else {"proposal_scores": weights}
    g, a = oracle.backward(scene, w, spp=spp, edge_spp=spp, seed=3, terms=oracle.TERM_PRIMARY, n_threads=NT,
                           **okw)
    V = len(scene.verts)
    assert_grads(got, g[:3 * V], a[:3 * V], "mixture proposal")
    plain, _ = oracle.backward(scene, w, spp=spp, edge_spp=spp, seed=3, terms=oracle.TERM_PRIMARY, n_threads=NT)
    assert not np.allclose(plain[:3 * V], g[:3 * V])


# ---------------------------------------------------------------------------
# Per-pixel gradient image (drt_grads.dimage_dparam)
# ---------------------------------------------------------------------------
def _gpu_jacobian(drt, ctx, scene, w, spp, seed, params, depth=1, primary_only=False):
    s = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((scene.height, scene.width, 3), device="cuda")
    opts = drt.make_opts(spp, spp, max_depth=depth, primary_only=primary_only, seed=seed)
    tape = s.render(img, opts, want_tape=True)
    dv = torch.zeros((len(scene.verts), 3), device="cuda")
    jac = torch.zeros((len(params), scene.height, scene.width), device="cuda")
    z = lambda *sh: torch.zeros(sh, device="cuda")  # noqa: E731
    da, dr, dc, ds = z(len(scene.tris), 3), z(3), z(3, 4), z(1)
    s.backward(torch.from_numpy(w).cuda(), opts, tape=tape, d_verts=dv, d_albedo=da, d_radiance=dr,
               d_cam_to_world=dc, d_cam_scale=ds, dimage_dparam=jac, jac_params=params)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    flat = np.concatenate([x.cpu().numpy().ravel().astype(np.float64) for x in (dv, da, dr, dc, ds)])
    return jac.double().cpu().numpy(), flat


def _assert_jacobian(got, want, absum, label):
    """Per pixel within 1e-4 |J| + 1e-6 A_k, with A_k the oracle's magnitude
    of the terms summed into the whole gradient entry k (it bounds the terms
    of any one pixel)."""
    err = np.abs(got - want)
    bound = 1e-4 * np.abs(want) + 1e-6 * np.asarray(absum, np.float64)[:, None, None] + 1e-12
    bad = err > bound
    assert not bad.any(), "%s: %d of %d pixel entries off, worst %g (bound %g)" % (
        label, bad.sum(), bad.size, err.max(), bound.flat[np.argmax(err / bound)])


@pytest.mark.parametrize("seed", [1235, 7])
def test_single_triangle_pixel_gradient_image(drt, ctx, seed):
    """The six screen-plane vertex coordinates of the single-triangle case:
    the per-pixel gradient image against the oracle's (which is pinned to the
    per-pixel Reynolds boundary integral), and its sum over the pixels
    against the gradient."""
    scene = sg.single_triangle(seed)
    w = sg.loss_adjoint(seed, scene.width, scene.height)
    params = [3 * v + c for v in range(3) for c in range(2)]
    got, grad = _gpu_jacobian(drt, ctx, scene, w, 16, seed, params, primary_only=True)
    g, a, want = oracle.backward(scene, w, spp=16, edge_spp=16, seed=seed, primary_only=True, n_threads=NT,
                                 jacobian=params)
    _assert_jacobian(got, want, a[params], "single triangle")
    assert np.allclose(got.sum(axis=(1, 2)), grad[params], rtol=1e-4, atol=1e-6 * np.abs(grad).max())
    assert np.count_nonzero(want) > 10


@pytest.mark.parametrize("depth", [1, 2])
def test_lit_scene_pixel_gradient_image(drt, ctx, depth):
    """Vertex, albedo, radiance, camera and camera-scale entries of a lit
    scene with all gradient terms."""
    scene = _small_lit(W=24, H=18, subdiv=1)
    V, T = len(scene.verts), len(scene.tris)
    w = sg.loss_adjoint(6, scene.width, scene.height)
    params = [3 * 2 + 1, 3 * (V - 3) + 0, 3 * (V - 1) + 2, 3 * V + 3 * 4 + 1, 3 * V + 3 * T + 0,
              3 * V + 3 * T + 3 + 3, 3 * V + 3 * T + 3 + 5, 3 * V + 3 * T + 15]
    got, grad = _gpu_jacobian(drt, ctx, scene, w, 6, 4, params, depth=depth)
    g, a, want = oracle.backward(scene, w, spp=6, edge_spp=6, seed=4, max_depth=depth, n_threads=NT,
                                 jacobian=params)
    _assert_jacobian(got, want, a[params], "lit depth %d" % depth)
    assert np.allclose(got.sum(axis=(1, 2)), grad[params], rtol=1e-4, atol=1e-5 * np.abs(grad[params]).max())


# ---------------------------------------------------------------------------
# Geometry buffers (the AOV extension of Sec. 5.4)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("aov", [1, 2, 3, 4])
def test_geometry_buffer_image_and_gradient(drt, ctx, aov):
    scene = _small_lit(W=40, H=28, subdiv=2)
    s = drt.Scene.from_arrays(ctx, scene)
    img = torch.zeros((28, 40, 3), device="cuda")
    opts = drt.make_opts(8, 8, seed=13, aov=aov)
    tape = s.render(img, opts, want_tape=True)
    want_img = oracle.render(scene, spp=8, seed=13, aov=aov, n_threads=NT)
    assert_pixels(img.double().cpu().numpy(), want_img, "aov %d image" % aov)
    w = sg.loss_adjoint(14, 40, 28)
    z = lambda *sh: torch.zeros(sh, dtype=torch.float32, device="cuda")  # noqa: E731
    dv, da, dr, dc, ds = z(len(scene.verts), 3), z(len(scene.tris), 3), z(3), z(3, 4), z(1)
    s.backward(torch.from_numpy(w).cuda(), opts, tape=tape, d_verts=dv, d_albedo=da, d_radiance=dr,
               d_cam_to_world=dc, d_cam_scale=ds)
    torch.cuda.synchronize()
    assert ctx.check_device() == (0, 0)
    got = np.concatenate([x.cpu().numpy().ravel().astype(np.float64) for x in (dv, da, dr, dc, ds)])
    want, absum, c = oracle.backward(scene, w, spp=8, edge_spp=8, seed=13, aov=aov, n_threads=NT,
                                     contributions=True)
    assert_grads(got, want, absum, "aov %d gradient" % aov, c)
    assert np.abs(want).max() > 0
