"""Pins of the CPU oracle against facts fixed outside it.

Each test compares the oracle with something it cannot agree with by
construction: published known-answer values, an independent library, a
closed form from geometry or radiometry, or an exact invariant of the
estimator.  All run on the CPU (no GPU marker).
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg
from tests import closed_forms as cf

NT = oracle.n_threads_default()


# --------------------------------------------------------------------------
# Philox4x32-10
# --------------------------------------------------------------------------
def test_philox_known_answers():
    """Known-answer vectors of Philox4x32-10 (Salmon et al., SC'11; the
    Random123 reference distribution), stored under tests/golden."""
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    n = 0
    for line in open(path):
        line = line.split("#")[0].split()
        if not line:
            continue
        vals = [int(x, 16) for x in line]
        ctr, key, want = vals[0:4], vals[4:6], vals[6:10]
        got = oracle.philox(ctr, key)
        assert [int(x) for x in got] == want
        n += 1
    assert n >= 3


def _curand():
    for name in ("libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    """cuRAND's host-side Philox4_32_10 generator (a library run on the CPU)
    produces block i of a stream from counter (0,0,i,0) and key = seed."""
    cu = _curand()
    if cu is None:
        pytest.skip("libcurand not available")
    for seed in (0x123456789ABCDEF, 1234, 2**64 - 5):
        gen = ctypes.c_void_p()
        assert cu.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
        try:
            assert cu.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            n = 64
            out = (ctypes.c_uint * n)()
            assert cu.curandGenerate(gen, out, ctypes.c_size_t(n)) == 0
            got = np.array(out[:], np.uint32).reshape(-1, 4)
            key = [seed & 0xFFFFFFFF, seed >> 32]
            for i in range(len(got)):
                assert list(oracle.philox([0, 0, i, 0], key)) == list(got[i])
        finally:
            cu.curandDestroyGenerator(gen)


# --------------------------------------------------------------------------
# Own sin/cos and the cosine-weighted direction
# --------------------------------------------------------------------------
def test_sincos_accuracy():
    r = np.linspace(0, 1, 4097, endpoint=False).astype(np.float32)
    err = 0.0
    for x in r:
        c, s = oracle.sincos_2pi(float(x))
        err = max(err, abs(c - math.cos(2 * math.pi * float(x))), abs(s - math.sin(2 * math.pi * float(x))))
    assert err < 5e-7


# --------------------------------------------------------------------------
# Watertight intersection
# --------------------------------------------------------------------------
def test_watertight_closed_mesh_never_leaks():
    """Rays from inside a closed icosphere always hit it, including rays
    aimed exactly at vertices and edge midpoints (Woop et al. 2013)."""
    v, f = sg.icosphere(2)
    rng = np.random.default_rng(3)
    v = v + rng.normal(0, 0.01, v.shape)
    scene = sg.Scene(verts=v, tris=f, albedo=np.full((len(f), 3), 0.5), light_tris=np.zeros(0, np.int32),
                     radiance=[0, 0, 0], cam_to_world=np.eye(4), cam_scale=1.0, cam_type=1, width=1, height=1)
    origins = [np.zeros(3), np.array([0.1, -0.2, 0.05])]
    targets = list(scene.verts) + [0.5 * (scene.verts[a] + scene.verts[b]) for a, b, _ in f[:200]]
    targets += list(rng.normal(size=(500, 3)))
    for o in origins:
        d = np.array(targets, np.float64) - o
        tri, _ = oracle.closest(scene, np.tile(o, (len(d), 1)), d, n_threads=NT)
        assert (tri >= 0).all()


def test_closest_hit_matches_fp64_reference():
    """The FP32 closest hit equals an FP64 Moller-Trumbore brute force except
    where two candidates are within rounding of each other."""
    scene = sg.direct_lighting(1236, width=8, height=8, subdiv=2)
    rng = np.random.default_rng(5)
    n = 2000
    o = np.tile(np.array([0.0, 1.0, 5.0]), (n, 1)) + rng.normal(0, 0.1, (n, 3))
    d = rng.normal(0, 0.3, (n, 3)) + np.array([0, -0.2, -1.0])
    tri, tb = oracle.closest(scene, o, d, n_threads=NT)
    V = scene.verts.astype(np.float64)[scene.tris]
    o32 = o.astype(np.float32).astype(np.float64)
    d32 = d.astype(np.float32).astype(np.float64)
    e1, e2 = V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]
    checked = 0
    for i in range(n):
        pv = np.cross(d32[i], e2)
        det = np.einsum("ij,ij->i", e1, pv)
        tv = o32[i] - V[:, 0]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = np.einsum("ij,ij->i", tv, pv) / det
            qv = np.cross(tv, e1)
            w = np.einsum("j,ij->i", d32[i], qv) / det
            t = np.einsum("ij,ij->i", e2, qv) / det
        ok = (u >= 0) & (w >= 0) & (u + w <= 1) & (t > 0)
        if not ok.any():
            assert tri[i] == -1
            continue
        ts = np.where(ok, t, np.inf)
        order = np.argsort(ts)
        best = order[0]
        margin = min(u[best], w[best], 1 - u[best] - w[best])
        second = ts[order[1]] if ok.sum() > 1 else np.inf
        if margin < 1e-5 or second - ts[best] < 1e-5 * ts[best]:
            continue
        assert tri[i] == best
        assert abs(tb[i, 0] - ts[best]) <= 1e-5 * ts[best]
        assert abs(tb[i, 1] - u[best]) < 1e-4 and abs(tb[i, 2] - w[best]) < 1e-4
        checked += 1
    assert checked > n // 4


# --------------------------------------------------------------------------
# Single triangle: closed-form coverage and the Reynolds-transport gradient
# --------------------------------------------------------------------------
def _tri_pixels(scene):
    W, H = scene.width, scene.height
    xy = scene.verts[:, :2].astype(np.float64)
    return [np.array([(x + 1.0) * W / 2.0, (1.0 - y) * H / 2.0]) for x, y in xy]


@pytest.mark.parametrize("seed", [1235, 77])
def test_single_triangle_coverage(seed):
    """E[I_p] = 0.7 * area(T inside pixel p) (Eq. first with a box filter)."""
    scene = sg.single_triangle(seed)
    spp = 1024
    img = oracle.render(scene, spp=spp, seed=seed, primary_only=True, n_threads=NT)
    A = cf.coverage(_tri_pixels(scene), scene.width, scene.height)
    sigma = 0.7 * np.sqrt(A * (1 - A) / spp) + 1e-9
    z = np.abs(img[..., 0] - 0.7 * A) / sigma
    assert np.nanmax(np.where(A * (1 - A) > 0, z, 0)) < 6.0
    inside_or_out = A * (1 - A) == 0
    assert np.allclose(img[..., 0][inside_or_out], 0.7 * A[inside_or_out], atol=1e-12)


@pytest.mark.parametrize("seed", [1235, 91])
def test_single_triangle_edge_gradient_reynolds(seed):
    """The primary edge term is unbiased for the boundary derivative of the
    covered area (Reynolds transport, Sec. 5.2.4): mean over seeds agrees
    with the closed form within its standard error."""
    scene = sg.single_triangle(seed)
    W, H = scene.width, scene.height
    w = sg.loss_adjoint(seed, W, H)
    wsum = w.astype(np.float64).sum(axis=2)
    gpix = cf.coverage_gradient(_tri_pixels(scene), 0.7 * wsum, W, H)
    want = np.stack([gpix[:, 0] * W / 2.0, -gpix[:, 1] * H / 2.0], axis=1)
    runs = []
    for k in range(12):
        g, _ = oracle.backward(scene, w, spp=1, edge_spp=16, seed=1000 + k, primary_only=True,
                               terms=oracle.TERM_PRIMARY, n_threads=NT)
        runs.append(oracle.split_params(scene, g)["verts"][:, :2])
    runs = np.array(runs)
    mean, se = runs.mean(0), runs.std(0, ddof=1) / np.sqrt(len(runs))
    assert np.all(np.abs(mean - want) < 5 * se + 1e-3 * np.abs(want).max())
    # the z coordinate never moves the orthographic projection
    assert np.all(runs[:, :, :] == runs) and np.all(
        oracle.split_params(scene, g)["verts"][:, 2] == 0)


def test_single_triangle_pixel_gradient_image_reynolds():
    """The per-pixel gradient image of the six screen-plane vertex coordinates
    (each primary edge sample counted in the pixel that contains its point)
    is, in expectation, the Reynolds boundary integral over the part of the
    triangle's edges inside that pixel; pixels the edges do not cross get
    exactly zero; the image sums to the gradient."""
    scene = sg.single_triangle(1235)
    W, H = scene.width, scene.height
    w = sg.loss_adjoint(1235, W, H)
    wsum = w.astype(np.float64).sum(axis=2)
    gp = cf.coverage_gradient_pixels(_tri_pixels(scene), 0.7 * wsum, W, H)
    want = np.stack([gp[..., 0] * W / 2.0, -gp[..., 1] * H / 2.0], axis=-1)  # [H, W, 3, 2]
    params = [3 * v + c for v in range(3) for c in range(2)]
    runs = []
    for k in range(8):
        g, _, jac = oracle.backward(scene, w, spp=1, edge_spp=16, seed=2000 + k, primary_only=True,
                                    terms=oracle.TERM_PRIMARY, n_threads=NT, jacobian=params)
        assert np.allclose(jac.sum(axis=(1, 2)), g[params], rtol=1e-10, atol=1e-12)
        runs.append(jac)
    runs = np.array(runs)  # [K, 6, H, W]
    want6 = want.reshape(H, W, 6).transpose(2, 0, 1)
    crossed = np.abs(want6) > 0
    assert np.all(runs[:, ~crossed] == 0.0)
    mean, se = runs.mean(0), runs.std(0, ddof=1) / np.sqrt(len(runs))
    z = np.abs(mean - want6)[crossed] / (se[crossed] + 1e-3 * np.abs(want6).max())
    assert np.mean(z < 3.0) > 0.97 and z.max() < 6.0, (np.mean(z < 3.0), z.max())


def test_pixel_gradient_image_sums_to_the_gradient_at_depth_two():
    scene = sg.direct_lighting(1236, width=12, height=10, subdiv=1)
    V, T = len(scene.verts), len(scene.tris)
    w = sg.loss_adjoint(7, scene.width, scene.height)
    params = [0, 3 * 5 + 1, 3 * (V - 3) + 2, 3 * V + 4, 3 * V + 3 * T + 1, 3 * V + 3 * T + 3 + 3,
              3 * V + 3 * T + 15]
    g, _, jac = oracle.backward(scene, w, spp=4, edge_spp=4, seed=8, max_depth=2, n_threads=NT, jacobian=params)
    assert np.allclose(jac.sum(axis=(1, 2)), g[params], rtol=1e-10, atol=1e-12 * np.abs(g).max())
    assert np.count_nonzero(jac) > 0


def test_single_triangle_albedo_homogeneity():
    """Per seed, exactly: sum_c rho_c dL/drho_c = sum_p w_p . I_p."""
    scene = sg.single_triangle(5)
    w = sg.loss_adjoint(5, scene.width, scene.height)
    img = oracle.render(scene, spp=8, seed=3, primary_only=True, n_threads=NT)
    g, _ = oracle.backward(scene, w, spp=8, edge_spp=8, seed=3, primary_only=True, n_threads=NT)
    ga = oracle.split_params(scene, g)["albedo"]
    lhs = float((scene.albedo.astype(np.float64) * ga).sum())
    rhs = float((w.astype(np.float64) * img).sum())
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(rhs))


# --------------------------------------------------------------------------
# Next-event estimation and secondary visibility at one shading point
# --------------------------------------------------------------------------
P0 = np.array([0.1, 0.2, 0.0])
LIGHT_C, LIGHT_EX, LIGHT_EY = (0.3, -0.1, 1.0), (0.25, 0.0, 0.0), (0.0, -0.25, 0.0)
BLOCKER = np.array([[0.15, -0.15, 0.5], [0.275, 0.1, 0.5], [0.1, 0.125, 0.5]])
RHO = np.array([0.5, 0.6, 0.7])
LE = 5.0


def _point_scene(with_blocker, light_verts=None, blocker=None):
    rv, rf = sg.quad(P0, (0.3, 0, 0), (0, 0.3, 0))
    lv, lf = sg.quad(LIGHT_C, LIGHT_EX, LIGHT_EY)
    if light_verts is not None:
        lv = light_verts
    parts = [(rv, rf), (lv, lf)]
    if with_blocker:
        parts.append((BLOCKER if blocker is None else blocker, np.array([[0, 1, 2]])))
    verts, tris = sg._merge(parts)
    alb = np.tile(RHO, (len(tris), 1))
    cam = np.eye(4)
    cam[:3, 3] = [P0[0], P0[1], 3.0]
    return sg.Scene(verts=verts, tris=tris, albedo=alb, light_tris=[2, 3], radiance=[LE] * 3,
                    cam_to_world=cam, cam_scale=1e-4, cam_type=sg.CAM_ORTHO, width=1, height=1)


def _closed_radiance(light_verts, blocker=None):
    """Reflected radiance at P0: rho/pi * Le * projected solid angle of the
    visible part of the light; the blocker's shadow is its central
    projection from P0 onto the (planar) light, clipped to the light."""
    n = np.array([0.0, 0.0, 1.0])
    phi = cf.polygon_irradiance(P0, n, light_verts)
    if blocker is not None:
        zl = light_verts[0][2]
        proj = [P0 + (zl - P0[2]) / (b[2] - P0[2]) * (b - P0) for b in blocker]
        inter = cf.clip_convex(cf.ccw([p[:2] for p in proj]), cf.ccw([v[:2] for v in light_verts]))
        if len(inter) >= 3:
            phi -= cf.polygon_irradiance(P0, n, [np.array([x, y, zl]) for x, y in inter])
    return RHO / np.pi * LE * phi


def _seed_runs(scene, terms, k=8, spp=40000):
    imgs, grads = [], []
    w = np.ones((1, 1, 3), np.float32)
    for s in range(k):
        imgs.append(oracle.render(scene, spp=spp, seed=500 + s, n_threads=NT)[0, 0])
        g, _ = oracle.backward(scene, w, spp=spp, edge_spp=1, seed=500 + s, terms=terms, n_threads=NT)
        grads.append(g)
    return np.array(imgs), np.array(grads)


def _zcheck(samples, want, rel_floor):
    mean = samples.mean(0)
    se = samples.std(0, ddof=1) / np.sqrt(len(samples))
    bound = 5 * se + rel_floor * np.abs(want).max()
    assert np.all(np.abs(mean - want) <= bound), (mean, want, se)


@pytest.mark.slow
def test_nee_matches_lambert_irradiance_and_its_light_derivative():
    scene = _point_scene(False)
    lv = scene.verts[4:8].astype(np.float64)
    imgs, grads = _seed_runs(scene, oracle.TERM_INTERIOR | oracle.TERM_SECONDARY)
    _zcheck(imgs, _closed_radiance(list(lv)), 1e-4)
    # d(sum_c I_c)/d(light vertex coordinate), closed form by central differences (smooth)
    h = 1e-6
    want = np.zeros((4, 3))
    for i in range(4):
        for c in range(3):
            lp, lm = lv.copy(), lv.copy()
            lp[i, c] += h
            lm[i, c] -= h
            want[i, c] = (_closed_radiance(list(lp)).sum() - _closed_radiance(list(lm)).sum()) / (2 * h)
    got = np.array([oracle.split_params(scene, g)["verts"][4:8] for g in grads])
    _zcheck(got, want, 2e-3)


@pytest.mark.slow
def test_secondary_edges_match_blocker_closed_form():
    """Blocker-vertex derivatives come only from the secondary edge term and
    must equal the derivative of the clipped-polygon closed form; the light's
    in-plane derivatives are interior plus edge."""
    scene = _point_scene(True)
    lv = scene.verts[4:8].astype(np.float64)
    imgs, grads = _seed_runs(scene, oracle.TERM_INTERIOR | oracle.TERM_SECONDARY, k=10)
    _zcheck(imgs, _closed_radiance(list(lv), BLOCKER), 1e-4)
    h = 1e-6
    want_b = np.zeros((3, 3))
    for i in range(3):
        for c in range(3):
            bp, bm = BLOCKER.copy(), BLOCKER.copy()
            bp[i, c] += h
            bm[i, c] -= h
            want_b[i, c] = (_closed_radiance(list(lv), bp).sum() - _closed_radiance(list(lv), bm).sum()) / (2 * h)
    got_b = np.array([oracle.split_params(scene, g)["verts"][8:11] for g in grads])
    _zcheck(got_b, want_b, 3e-3)
    want_l = np.zeros((4, 2))
    for i in range(4):
        for c in range(2):
            lp, lm = lv.copy(), lv.copy()
            lp[i, c] += h
            lm[i, c] -= h
            want_l[i, c] = (_closed_radiance(list(lp), BLOCKER).sum() -
                            _closed_radiance(list(lm), BLOCKER).sum()) / (2 * h)
    got_l = np.array([oracle.split_params(scene, g)["verts"][4:8, :2] for g in grads])
    _zcheck(got_l, want_l, 3e-3)


def test_secondary_edge_area_and_solid_angle_forms_agree():
    """For the blocker's own vertices the area-measure form (Eq. dirac_3d_edge
    with the Jacobian of Appendix 5.A, reading m = p + tau omega) equals the
    solid-angle form of the same boundary integral."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        p = rng.normal(size=3)
        v0, v1 = p + rng.normal(size=3) + [0, 0, 2], p + rng.normal(size=3) + [0, 0, 2]
        nm = rng.normal(size=3)
        t = rng.uniform()
        w = v0 + t * (v1 - v0) - p
        # a plane beyond the edge point along w
        m_dist = rng.uniform(1.5, 4.0)
        plane_d = float(np.dot(p + m_dist * w, nm / np.linalg.norm(nm)))
        nmu = nm / np.linalg.norm(nm)
        if abs(np.dot(w / np.linalg.norm(w), nmu)) < 0.1:
            continue
        out = oracle.sec_edge_forms(p, v0, v1, t, nm, plane_d)
        assert np.allclose(out[:6], out[6:], rtol=1e-9, atol=1e-12 * np.abs(out).max())


# --------------------------------------------------------------------------
# Exact invariants on a small lit scene
# --------------------------------------------------------------------------
def _tiny_lit():
    return sg.direct_lighting(1236, width=12, height=10, subdiv=1)


def test_translation_invariance_of_the_gradient():
    """Moving every vertex and the camera together leaves the image unchanged,
    so sum_v dL/dv + dL/d(camera position) = 0 for every seed, term by term."""
    scene = _tiny_lit()
    w = sg.loss_adjoint(2, scene.width, scene.height)
    for terms in (oracle.TERM_INTERIOR, oracle.TERM_PRIMARY, oracle.TERM_SECONDARY):
        g, a = oracle.backward(scene, w, spp=4, edge_spp=4, seed=9, terms=terms, n_threads=NT)
        sp = oracle.split_params(scene, g)
        total = sp["verts"].sum(0) + sp["cam_to_world"][:, 3]
        scale = oracle.split_params(scene, a)["verts"].sum() + 1e-30
        assert np.all(np.abs(total) <= 1e-9 * scale), (terms, total, scale)
        assert np.abs(sp["verts"]).sum() > 0


def test_radiance_homogeneity():
    """Per seed, exactly: sum_c Le_c dL/dLe_c = sum_p w_p . I_p (the image is
    linear in the emitted radiance)."""
    scene = _tiny_lit()
    w = sg.loss_adjoint(3, scene.width, scene.height)
    img = oracle.render(scene, spp=4, seed=21, n_threads=NT)
    g, _ = oracle.backward(scene, w, spp=4, edge_spp=4, seed=21, terms=oracle.TERM_INTERIOR, n_threads=NT)
    gr = oracle.split_params(scene, g)["radiance"]
    lhs = float((scene.radiance.astype(np.float64) * gr).sum())
    rhs = float((w.astype(np.float64) * img).sum())
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(rhs))


# --------------------------------------------------------------------------
# Mixture proposal over tile segments (learned-proposal estimator)
# --------------------------------------------------------------------------
def test_segments_partition_the_clipped_edges():
    scene = sg.direct_lighting(1236, width=64, height=48, subdiv=2)
    edge, tile, s01, lens = oracle.segments(scene)
    pe = oracle.primary_edges(scene)
    per_edge = np.bincount(edge, weights=lens, minlength=len(pe))
    assert np.allclose(per_edge, pe[:, 6], rtol=0, atol=1e-9 * pe[:, 6].max())
    assert np.all(s01[:, 1] > s01[:, 0])
    assert tile.max() < 4 * 3 and tile.min() >= 0


@pytest.mark.parametrize("seed,mode", [(1235, "weights"), (91, "weights"), (77, "scores")])
def test_mixture_proposal_is_unbiased(seed, mode):
    """With arbitrary nonnegative segment weights m (or network scores s,
    m = len exp(s)), sampling segments by q = 1/2 len/L + 1/2 m/M and
    weighting by len/q keeps the primary edge term unbiased: its mean equals
    the Reynolds closed form."""
    scene = sg.single_triangle(seed)
    W, H = scene.width, scene.height
    w = sg.loss_adjoint(seed, W, H)
    gpix = cf.coverage_gradient(_tri_pixels(scene), 0.7 * w.astype(np.float64).sum(axis=2), W, H)
    want = np.stack([gpix[:, 0] * W / 2.0, -gpix[:, 1] * H / 2.0], axis=1)
    n_seg = len(oracle.segments(scene)[0])
    rng = np.random.default_rng(seed + 5)
    m = rng.exponential(size=n_seg).astype(np.float32) ** 3
    kw = {"proposal_weights": m} if mode == "weights" else {"proposal_scores": 3.0 * rng.normal(size=n_seg)}
    runs = []
    for k in range(12):
        g, _ = oracle.backward(scene, w, spp=1, edge_spp=16, seed=2000 + k, primary_only=True,
                               terms=oracle.TERM_PRIMARY, n_threads=NT, **kw)
        runs.append(oracle.split_params(scene, g)["verts"][:, :2])
    runs = np.array(runs)
    mean, se = runs.mean(0), runs.std(0, ddof=1) / np.sqrt(len(runs))
    assert np.all(np.abs(mean - want) < 5 * se + 1e-3 * np.abs(want).max())
