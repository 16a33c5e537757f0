"""Pins of the oracle's next-event estimation for edges (Sec. 5.3.3), against
definitions and closed forms, not against the oracle:

- its FP32 logarithm against numpy's;
- a billboard crossing is the closest approach of the shadow ray's line and
  the edge's line (FP64 least squares here), inside the half width, with the
  edge parameter in [0, 1] and the ray parameter before the light; the
  importance is length / distance for silhouettes seen from p (the face
  normals' orientation, computed here) and zero otherwise;
- the ray of an edge's family through (t, u) passes the edge's line at t at
  distance |u|, and the solid angle it sweeps per unit t and u is the closed
  form J |E| (central differences of directions built here from the
  definition: a point on the circle of radius |u| about the edge point whose
  offset is orthogonal to the ray);
- the race picks an edge with probability importance / sum (frequencies);
- the density: E[sum over crossed edges of P(e | S) / p_B] over light points
  drawn by area equals the measure of the (edge, t, u) whose rays reach the
  light with the edge before it (brute force over a grid here) -- the
  identity that makes 1 / p_B an unbiased weight;
- the combined secondary term (length sampler and billboard sampler, balance
  heuristic) has the plain sampler's expectation, matches the blocker's
  closed-form derivative with a small light, and has a lower variance there.
"""
import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg
from tests.test_oracle_pins import BLOCKER, P0, _closed_radiance, _point_scene, _zcheck

NT = oracle.n_threads_default()
F = np.float32


def test_ln32_is_the_logarithm():
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.uniform(0, 1, 4000), np.linspace(0.98, 1.0, 2000), 2.0 ** -np.arange(1, 24)])
    xs = xs[(xs > 0) & (xs < 1)].astype(F)
    got = np.array([oracle.ln32(float(x)) for x in xs])
    want = np.log(xs.astype(np.float64))
    assert np.all(np.abs(got - want) <= 3e-7 * np.abs(want)), np.max(np.abs(got - want) / np.abs(want))
    assert oracle.ln32(1.0) == 0.0


def _soup_scene(seed, n=40, spread=1.0):
    """Random triangles around the origin with a light above (an edge soup:
    every edge has one face)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-spread, spread, (n, 1, 3))
    v = (c + rng.normal(0, 0.3, (n, 3, 3))).reshape(-1, 3)
    lv, lf = sg.quad((0, 0, 3), (0.5, 0, 0), (0, -0.5, 0))
    verts, tris = sg._merge([(v, np.arange(3 * n).reshape(n, 3)), (lv, lf)])
    cam = np.eye(4)
    cam[:3, 3] = [0, 0, 6]
    return sg.Scene(verts=verts, tris=tris, albedo=np.full((len(tris), 3), 0.5), light_tris=[n, n + 1],
                    radiance=[5.0] * 3, cam_to_world=cam, cam_scale=0.5, cam_type=sg.CAM_PINHOLE, width=4, height=4)


def _edges_of(scene):
    """Unique undirected edges sorted by (min, max) vertex: the oracle's ids."""
    t = np.asarray(scene.tris)
    e = np.sort(np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]]), axis=1)
    return np.unique(e, axis=0)


def _closest(p, d, a, b):
    """FP64 closest points of the lines p + s d and a + t (b - a): (s, t, dist)."""
    E = b - a
    M = np.array([[d @ d, -(d @ E)], [d @ E, -(E @ E)]])
    rhs = np.array([(a - p) @ d, (a - p) @ E])
    s, t = np.linalg.solve(M, rhs)
    return s, t, np.linalg.norm(p + s * d - (a + t * E))


def test_crossing_is_the_closest_approach_of_the_two_lines():
    checked = 0
    for seed in range(6):
        scene = _soup_scene(seed)
        q = oracle.NeeQuery(scene)
        edges = _edges_of(scene)
        V = scene.verts.astype(np.float64)
        rng = np.random.default_rng(100 + seed)
        for _ in range(20):
            p = rng.uniform(-1, 1, 3).astype(F)
            y = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), 3.0], F)
            d = (y - p).astype(F)
            hw = 0.05
            n = (d / np.linalg.norm(d)).astype(F)
            eid, stui = q.crossings(p, n, d, 1.0, hw)
            got = dict(zip(eid.tolist(), stui))
            for k, (a, b) in enumerate(edges):
                s, t, dist = _closest(p.astype(np.float64), d.astype(np.float64), V[a], V[b])
                margin = min(abs(dist - hw) / hw, abs(t), abs(t - 1), abs(s), abs(s - 1))
                if margin < 1e-4:
                    continue  # a decision this close to its boundary is FP32's to take
                inside = dist < hw and 0 < t < 1 and 0 < s < 1
                assert (k in got) == inside, (seed, k, s, t, dist)
                if inside:
                    gs, gt, gu, gimp = got[k]
                    assert abs(gs - s) <= 1e-4 and abs(gt - t) <= 1e-4 * max(1.0, np.linalg.norm(V[b] - V[a]) ** -1)
                    assert abs(abs(gu) - dist) <= 1e-4 * hw + 1e-6
                    m = V[a] + t * (V[b] - V[a])
                    checked += 1
                    if a >= 3 * 40:
                        continue  # the light quad: its diagonal has two faces (the next test covers those)
                    # a soup edge has one face, so it is a silhouette; the point must lie above p's tangent
                    # plane and farther from p than the width
                    dist = np.linalg.norm(m - p)
                    want_imp = np.linalg.norm(V[b] - V[a]) / dist if n @ (m - p) > 0 and dist > 2 * hw else 0.0
                    if abs(dist - 2 * hw) < 1e-4 * hw:
                        continue
                    assert abs(gimp - want_imp) <= 1e-4 * want_imp
        q.close()
    assert checked > 50, checked


def test_importance_is_zero_off_the_silhouette():
    """On a closed icosphere seen from outside, an edge is a silhouette
    exactly when one of its faces faces p and the other does not."""
    v, f = sg.displaced_icosphere(np.random.default_rng(4))
    lv, lf = sg.quad((0, 0, 4), (0.5, 0, 0), (0, -0.5, 0))
    verts, tris = sg._merge([(v, f), (lv, lf)])
    cam = np.eye(4)
    cam[:3, 3] = [0, 0, 8]
    scene = sg.Scene(verts=verts, tris=tris, albedo=np.full((len(tris), 3), 0.5), light_tris=[len(f), len(f) + 1],
                     radiance=[5.0] * 3, cam_to_world=cam, cam_scale=0.5, cam_type=sg.CAM_PINHOLE, width=4, height=4)
    q = oracle.NeeQuery(scene)
    V = verts.astype(np.float64)
    faces_of = {}
    for ti, t in enumerate(np.asarray(f)):
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            faces_of.setdefault((min(a, b), max(a, b)), []).append(ti)
    edges = _edges_of(scene)
    rng = np.random.default_rng(5)
    n_sil = n_not = 0
    for _ in range(400):
        p = np.array([rng.uniform(-3, 3), rng.uniform(-3, 3), -3.0], F)
        y = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), 4.0], F)
        n = ((y - p) / np.linalg.norm(y - p)).astype(F)
        eid, stui = q.crossings(p, n, y - p, 1.0, 0.04)
        for k, x in zip(eid, stui):
            a, b = edges[k]
            fs = faces_of.get((a, b))
            if fs is None or len(fs) != 2:
                continue
            front = []
            for ti in fs:
                A, B, C = V[np.asarray(f)[ti]]
                fn = np.cross(B - A, C - A)
                front.append(fn @ (p - A) > 0)
            sil = front[0] != front[1]
            margin = min(abs(np.cross(V[np.asarray(f)[ti]][1] - V[np.asarray(f)[ti]][0],
                                      V[np.asarray(f)[ti]][2] - V[np.asarray(f)[ti]][0]) @ (p - V[np.asarray(f)[ti]][0]))
                         for ti in fs)
            if margin < 1e-5:
                continue
            assert (x[3] > 0) == sil, (k, x, front)
            n_sil += sil
            n_not += not sil
    q.close()
    assert n_sil > 10 and n_not > 10, (n_sil, n_not)


def _family_direction(p, a, b, t, u, branch=1):
    """Unit direction of the ray from p whose closest approach to the line of
    (a, b) is at parameter t, at distance u > 0, from the definition: the
    offset of that point from the edge point is orthogonal to the edge and to
    the ray; branch +1 or -1 picks one of the two such rays (FP64)."""
    E = b - a
    Eh = E / np.linalg.norm(E)
    m = a + t * E
    pm = p - m
    pm_perp = pm - (pm @ Eh) * Eh
    A = pm_perp / np.linalg.norm(pm_perp)
    B = np.cross(Eh, A)
    alpha, beta = pm @ A, pm @ B  # beta = 0
    R = np.hypot(alpha, beta)
    phi = np.arctan2(beta, alpha) + branch * np.arccos(u / R)
    off = u * (np.cos(phi) * A + np.sin(phi) * B)
    qpt = m + off
    assert abs(off @ (qpt - p)) < 1e-9 * (1 + np.linalg.norm(qpt - p))
    w = qpt - p
    return w / np.linalg.norm(w)


def test_family_ray_and_its_jacobian():
    scene = _soup_scene(7)
    q = oracle.NeeQuery(scene)
    edges = _edges_of(scene)
    V = scene.verts.astype(np.float64)
    rng = np.random.default_rng(8)
    checked = 0
    for _ in range(40):
        k = int(rng.integers(0, len(edges) - 5))
        a, b = V[edges[k][0]], V[edges[k][1]]
        p = rng.uniform(-1, 1, 3).astype(F)
        t = float(rng.uniform(0.05, 0.95))
        u = float(rng.uniform(0.01, 0.05))
        d = q.ray(k, p, t, u)
        if d is None:
            continue
        s, tt, dist = _closest(p.astype(np.float64), d.astype(np.float64), a, b)
        assert abs(s - 1) < 1e-4 and abs(tt - t) < 1e-4 and abs(dist - u) < 1e-4 * u + 1e-6, (s, tt, dist)
        # solid angle per unit t and u by central differences of the definition
        h_t, h_u = 1e-5, 1e-6
        pd = p.astype(np.float64)
        dt = (_family_direction(pd, a, b, t + h_t, u) - _family_direction(pd, a, b, t - h_t, u)) / (2 * h_t)
        du = (_family_direction(pd, a, b, t, u + h_u) - _family_direction(pd, a, b, t, u - h_u)) / (2 * h_u)
        want = np.linalg.norm(np.cross(dt, du))
        got = q.jacobian(k, p, t, u)
        assert abs(got - want) <= 1e-4 * want, (got, want)
        checked += 1
    q.close()
    assert checked >= 30


def test_race_picks_by_importance():
    scene = _soup_scene(9, n=60, spread=0.4)
    q = oracle.NeeQuery(scene)
    rng = np.random.default_rng(10)
    done = 0
    for _ in range(200):
        p = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), -1.5], F)
        y = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), 3.0], F)
        d = y - p
        n = (d / np.linalg.norm(d)).astype(F)
        eid, stui = q.crossings(p, n, d, 1.0, 0.08)
        pos = stui[:, 3] > 0
        if pos.sum() < 3:
            continue
        prob = stui[:, 3].astype(np.float64) / stui[:, 3].astype(np.float64).sum()
        draws = 6000
        picks = np.array([q.pick(p, n, d, 1.0, 0.08, int(k0), int(k1))
                          for k0, k1 in rng.integers(0, 2 ** 32, (draws, 2), dtype=np.uint64)])
        counts = np.array([(picks == e).sum() for e in eid])
        assert counts.sum() == draws and counts[~pos].sum() == 0
        eid, stui, counts, prob = eid[pos], stui[pos], counts[pos], prob[pos]
        exp = draws * prob
        chi2 = ((counts - exp) ** 2 / exp).sum()
        dof = len(eid) - 1
        assert chi2 < dof + 6 * np.sqrt(2 * dof), (chi2, dof, counts, exp)
        done += 1
        if done == 3:
            break
    q.close()
    assert done == 3


def _light_hit(p, d, tris):
    """FP64 ray/triangle test (Moller-Trumbore) against the light triangles:
    the smallest hit parameter in units of d, or inf."""
    best = np.inf
    for A, B, C in tris:
        e1, e2 = B - A, C - A
        h = np.cross(d, e2)
        det = e1 @ h
        if abs(det) < 1e-15:
            continue
        s = p - A
        uu = (s @ h) / det
        qv = np.cross(s, e1)
        vv = (d @ qv) / det
        if uu < 0 or vv < 0 or uu + vv > 1:
            continue
        tt = (e2 @ qv) / det
        if tt > 0:
            best = min(best, tt)
    return best


@pytest.mark.slow
def test_density_integrates_to_the_covered_measure():
    """With light points drawn by area and the race's probabilities as
    weights, the mean of sum_e P(e|S) / p_B is the measure of the (e, t, u)
    whose rays reach the light after crossing e's billboard."""
    scene = _point_scene(True)
    q = oracle.NeeQuery(scene)
    edges = _edges_of(scene)
    V = scene.verts.astype(np.float64)
    T = np.asarray(scene.tris)
    light = [V[T[j]] for j in scene.light_tris]
    areas = np.array([0.5 * np.linalg.norm(np.cross(B - A, C - A)) for A, B, C in light])
    # a receiver point off the receiver's diagonal; its normal is +z
    p = (P0 + np.array([0.04, 0.015, 0.0])).astype(F)
    nrm = np.array([0.0, 0.0, 1.0], F)
    hw = 0.01
    # Monte Carlo side: light points by area
    rng = np.random.default_rng(12)
    N = 40000
    tot = []
    for _ in range(N):
        j = rng.choice(len(light), p=areas / areas.sum())
        r1, r2 = rng.uniform(size=2)
        su = np.sqrt(r1)
        A, B, C = light[j]
        y = (1 - su) * A + su * (1 - r2) * B + su * r2 * C
        d = (y.astype(F) - p).astype(F)
        eid, stui = q.crossings(p, nrm, d, 1.0, hw)
        keep = stui[:, 3] > 0
        if not keep.any():
            tot.append(0.0)
            continue
        eid, stui = eid[keep], stui[keep]
        W = stui[:, 3].astype(np.float64).sum()
        dens = q.density(np.repeat(p[None], len(eid), 0), np.repeat(nrm[None], len(eid), 0),
                         np.repeat(d[None], len(eid), 0), eid, stui[:, 1], stui[:, 2], hw)
        tot.append(sum(stui[i, 3] / W / dens[i] for i in range(len(eid)) if dens[i] > 0))
    tot = np.array(tot)
    mc, se = tot.mean(), tot.std(ddof=1) / np.sqrt(N)
    # brute force side: the covered part of [0,1] x [-hw, hw] per edge
    nt, nu = 400, 40
    covered = 0.0
    faces_of = {}
    for t3 in T:
        for i in range(3):
            x, z = int(t3[i]), int(t3[(i + 1) % 3])
            faces_of.setdefault((min(x, z), max(x, z)), []).append(int(t3[(i + 2) % 3]))
    for k, (a, b) in enumerate(edges):
        A, B = V[a], V[b]
        thirds = faces_of[(int(a), int(b))]
        if len(thirds) == 2:  # two faces: a silhouette seen from p only if both lie on one side
            nplane = np.cross(A - p, B - p)
            if (V[thirds[0]] - p) @ nplane * ((V[thirds[1]] - p) @ nplane) < 0:
                continue
        cnt = 0
        for t in (np.arange(nt) + 0.5) / nt:
            for u in (np.arange(nu) + 0.5) / nu * 2 * hw - hw:
                m = A + t * (B - A)
                if (m - p) @ nrm <= 0 or np.linalg.norm(m - p) <= 2 * hw:
                    continue  # at or below p's tangent plane, or within the width of p: no importance
                if a < 4 and b < 4:
                    continue  # the receiver's own edges lie in that plane
                w = _family_direction(p.astype(np.float64), A, B, t, abs(u), 1 if u > 0 else -1)
                # the ray's parameter at its closest point, in units of |q - p|
                qdist = np.sqrt(max((m - p) @ (m - p) - u * u, 0.0))
                th = _light_hit(p.astype(np.float64), w, light)
                cnt += np.isfinite(th) and th > qdist
        covered += cnt / (nt * nu) * 2 * hw
    q.close()
    # only silhouette edges carry importance: the blocker's three edges and
    # the light's border; the light's diagonal and the receiver are not crossed
    assert covered > 0
    assert abs(mc - covered) <= 4 * se + 0.01 * covered, (mc, covered, se)


def _sec_grads(scene, w, depth, nee, seeds, spp=64):
    out = []
    for s in seeds:
        g, _ = oracle.backward(scene, w, spp=spp, edge_spp=1, seed=s, max_depth=depth,
                               terms=oracle.TERM_SECONDARY, sec_nee=nee, n_threads=NT)
        out.append(oracle.split_params(scene, g)["verts"].ravel())
    return np.array(out)


@pytest.mark.parametrize("depth", [1, 2])
def test_gradient_has_the_plain_samplers_expectation(depth):
    scene = sg.direct_lighting(11, width=16, height=16, subdiv=1)
    w = sg.loss_adjoint(5, 16, 16)
    seeds = range(100)
    a = _sec_grads(scene, w, depth, 0, seeds)
    b = _sec_grads(scene, w, depth, 1, seeds)
    ma, mb = a.mean(0), b.mean(0)
    se = np.sqrt(a.var(0, ddof=1) / len(a) + b.var(0, ddof=1) / len(b))
    floor = 1e-5 * np.abs(ma).max()
    z = (ma - mb) / np.sqrt(se ** 2 + floor ** 2)
    assert np.sqrt(np.mean(z ** 2)) < 1.5 and np.abs(z).max() < 5.0, (np.sqrt(np.mean(z ** 2)), np.abs(z).max())
    assert not np.allclose(a, b)


@pytest.mark.slow
def test_billboards_match_the_blocker_closed_form_with_less_variance():
    """A small light: the blocker's vertex derivatives (secondary term only)
    equal the clipped-polygon closed form with the billboard sampler added,
    and their variance drops."""
    # the light straddles the edge of the blocker's shadow (seen from P0)
    lv0, _ = sg.quad((0.4, -0.1, 1.0), (0.06, 0.0, 0.0), (0.0, -0.06, 0.0))
    scene = _point_scene(True, light_verts=lv0)
    lv = scene.verts[4:8].astype(np.float64)
    h = 1e-6
    want = np.zeros((3, 3))
    for i in range(3):
        for c in range(3):
            bp, bm = BLOCKER.copy(), BLOCKER.copy()
            bp[i, c] += h
            bm[i, c] -= h
            want[i, c] = (_closed_radiance(list(lv), bp).sum() - _closed_radiance(list(lv), bm).sum()) / (2 * h)
    assert np.abs(want).max() > 1e-3
    w = np.ones((1, 1, 3), np.float32)
    runs = {0: [], 1: []}
    for nee in (0, 1):
        for s in range(8):
            g, _ = oracle.backward(scene, w, spp=20000, edge_spp=1, seed=1300 + s, terms=oracle.TERM_SECONDARY,
                                   sec_nee=nee, n_threads=NT)
            runs[nee].append(oracle.split_params(scene, g)["verts"][8:11])
    _zcheck(np.array(runs[1]), want, 3e-3)
    v0 = np.array(runs[0]).reshape(8, -1).var(0, ddof=1).sum()
    v1 = np.array(runs[1]).reshape(8, -1).var(0, ddof=1).sum()
    assert v1 < 0.5 * v0, (v0, v1)
