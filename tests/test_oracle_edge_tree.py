"""Pins of the oracle's hierarchical secondary-edge selection (Sec. 5.3.1)
against geometry and probability, not against the oracle itself:

- the hierarchy holds every edge once, boxes bound their subtrees, total
  lengths add up, and the class split is the camera-silhouette test;
- the v-sphere test in Hough space never culls an edge that is a silhouette
  from the shading point (FP64 brute force over random points);
- the cosine bound bounds the cosine over sampled box points and is exact
  for a point box;
- the resampling weights make every positive-importance edge count once in
  expectation: E[w 1{pick = e}] = 1 (zero for edges the gate removes);
- the secondary-edge gradient through the hierarchy has the expectation of
  the length sampler's, and matches the blocker's closed-form derivative.
"""
import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg
from tests.test_oracle_pins import BLOCKER, _closed_radiance, _point_scene, _zcheck

NT = oracle.n_threads_default()


def _scene():
    return sg.direct_lighting(11, width=16, height=16, subdiv=1)


def _topology(scene):
    V = np.asarray(scene.verts, np.float64)
    faces = {}
    for t, tri in enumerate(np.asarray(scene.tris)):
        for k in range(3):
            a, b = int(tri[k]), int(tri[(k + 1) % 3])
            faces.setdefault((min(a, b), max(a, b)), []).append(t)
    return V, faces


def _third(scene, t, a, b):
    return [int(v) for v in scene.tris[t] if v != a and v != b][0]


def _silhouette64(scene, V, faces, ed, e, p):
    """Seen from p, a two-faced edge is not a silhouette when its faces lie
    strictly on opposite sides of the plane through p and the edge."""
    a, b = ed[e]
    f = faces[(a, b)]
    if len(f) != 2:
        return True
    c0, c1 = V[_third(scene, f[0], a, b)], V[_third(scene, f[1], a, b)]
    m = np.cross(V[a] - p, V[b] - p)
    return not ((m @ (c0 - p)) * (m @ (c1 - p)) < 0)


def _subtree(nodes, enc):
    if enc < 0:
        return [~enc]
    return _subtree(nodes, nodes[enc][0]) + _subtree(nodes, nodes[enc][1])


def test_hierarchy_structure_and_classes():
    scene = _scene()
    nodes, slots, leaves, root = oracle.edge_tree(scene)
    ed = oracle.edges(scene)
    E = len(ed)
    V, faces = _topology(scene)
    assert root == 0 and len(nodes) == E - 1
    assert sorted(leaves[:, 0].tolist()) == list(range(E))
    assert sorted(_subtree(nodes, root)) == list(range(E))
    O = np.asarray(scene.cam_to_world, np.float64)[:3, 3]
    lens = np.linalg.norm(V[ed[:, 1]] - V[ed[:, 0]], axis=1)
    for i in range(len(nodes)):
        for c in range(2):
            sub = _subtree(nodes, nodes[i][c])
            eids = leaves[sub, 0]
            pts = np.concatenate([V[ed[eids, 0]], V[ed[eids, 1]]])
            s = slots[i, c]
            assert np.all(s[0:3] <= pts.min(0)) and np.all(s[3:6] >= pts.max(0))
            assert abs(s[12] - lens[eids].sum()) <= 1e-5 * lens[eids].sum()
            assert bool(s[13]) == bool(np.all(leaves[sub, 1]))
    # class B: two faces, and O strictly on the same side of both (consistently oriented) face planes
    for pos in range(E):
        e, cls, bnd = leaves[pos]
        a, b = ed[e]
        f = faces[(a, b)]
        assert bool(bnd) == (len(f) != 2)
        if len(f) != 2:
            assert not cls
            continue
        c0, c1 = V[_third(scene, f[0], a, b)], V[_third(scene, f[1], a, b)]
        n0 = np.cross(V[b] - V[a], c0 - V[a])
        n1 = np.cross(V[a] - V[b], c1 - V[b])
        s0, s1 = n0 @ (O - V[a]), n1 @ (O - V[a])
        if abs(s0) > 1e-6 * np.linalg.norm(n0) and abs(s1) > 1e-6 * np.linalg.norm(n1):
            assert bool(cls) == (s0 * s1 > 0), pos
    # the class is the top key bit: the root separates the two hierarchies
    cls_left = leaves[_subtree(nodes, nodes[root][0]), 1]
    cls_right = leaves[_subtree(nodes, nodes[root][1]), 1]
    assert not cls_left.any() and cls_right.all()


def test_vsphere_never_culls_a_silhouette():
    scene = _scene()
    nodes, slots, leaves, _ = oracle.edge_tree(scene)
    ed = oracle.edges(scene)
    V, faces = _topology(scene)
    rng = np.random.default_rng(0)
    lo, hi = V.min(0), V.max(0)
    cleared = 0
    for _ in range(120):
        p = (lo + (hi - lo) * rng.random(3)).astype(np.float32)
        vs = oracle.edge_tree_vsphere(scene, p)
        for i, c in zip(*np.nonzero(vs)):
            cleared += 1
            for pos in _subtree(nodes, nodes[i][c]):
                assert not _silhouette64(scene, V, faces, ed, leaves[pos][0], p.astype(np.float64)), (p, i, c)
    assert cleared > 1000  # the test culls something


def test_cos_bound_bounds_the_cosine():
    rng = np.random.default_rng(1)
    for _ in range(400):
        p = rng.normal(size=3).astype(np.float32)
        n = rng.normal(size=3)
        n = (n / np.linalg.norm(n)).astype(np.float32)
        c = rng.normal(size=3) * 2
        h = np.abs(rng.normal(size=3)) * rng.choice([0.01, 0.3, 2.0])
        lo, hi = (c - h).astype(np.float32), (c + h).astype(np.float32)
        bound = oracle.edge_tree_cos_bound(p, n, lo, hi)
        x = lo + (hi - lo) * rng.random((2000, 3))
        corners = np.array([[(lo, hi)[(k >> j) & 1][j] for j in range(3)] for k in range(8)])
        x = np.concatenate([x, corners]).astype(np.float64)
        d = x - p.astype(np.float64)
        cos = (d @ n.astype(np.float64)) / np.linalg.norm(d, axis=1)
        assert bound >= cos.max() - 1e-5, (bound, cos.max())
    # a point box: the bound is the cosine itself
    for _ in range(100):
        p = rng.normal(size=3).astype(np.float32)
        n = rng.normal(size=3)
        n = (n / np.linalg.norm(n)).astype(np.float32)
        q = rng.normal(size=3).astype(np.float32)
        d = q.astype(np.float64) - p
        want = d @ n / np.linalg.norm(d)
        assert abs(oracle.edge_tree_cos_bound(p, n, q, q) - want) <= 1e-5


def _reaches_light(scene, V, p, pts, spread):
    """FP64 brute force: does a ray from p toward any of pts, or tilted by up
    to `spread` rad, hit a light triangle?  (Rays toward the light triangles'
    points within that angle of a ray through pts.)"""
    d = pts - p
    d = d / np.linalg.norm(d, axis=1)[:, None]
    rng = np.random.default_rng(0)
    for lt in np.asarray(scene.light_tris):
        a, b, c = (V[int(i)] for i in scene.tris[lt])
        uv = rng.random((4000, 2))
        flip = uv.sum(1) > 1
        uv[flip] = 1 - uv[flip]
        y = a + uv[:, :1] * (b - a) + uv[:, 1:] * (c - a)
        y = np.concatenate([y, np.array([a, b, c])])
        dy = y - p
        dy = dy / np.linalg.norm(dy, axis=1)[:, None]
        if (d @ dy.T).max() >= np.cos(spread):
            return True
    return False


@pytest.mark.parametrize("where,last,samples", [("ground", True, 1), ("ground", True, 16), ("ground", False, 4),
                                                 ("sphere", True, 16), ("sphere", False, 16)])
def test_resampling_weights_count_every_edge_once(where, last, samples):
    """E[w 1{pick = e}] = 1 for every edge the importance keeps; edges the
    silhouette gate or the horizon removes are never picked, and an edge the
    light-cone bound removes sends no ray to a light."""
    scene = _scene()
    V, faces = _topology(scene)
    ed = oracle.edges(scene)
    E = len(ed)
    if where == "ground":
        p = np.array([0.3, V[:, 1].min() + 1e-3, 0.2], np.float32)
        n = np.array([0.0, 1.0, 0.0], np.float32)
    else:  # a point on the sphere's lower half, facing down toward the ground
        k = int(np.argmin(V[:42, 1]))
        p = (V[k] * 0.999).astype(np.float32)
        n = (V[k] / np.linalg.norm(V[k])).astype(np.float32)
    N = 120000
    eid, w = oracle.edge_tree_picks(scene, p, n, last=last, samples=samples, n_picks=N, seed=3)
    contrib = np.zeros((E,))
    contrib2 = np.zeros((E,))
    np.add.at(contrib, eid[eid >= 0], w[eid >= 0])
    np.add.at(contrib2, eid[eid >= 0], w[eid >= 0].astype(np.float64) ** 2)
    est = contrib / N
    se = np.sqrt(np.maximum(contrib2 / N - est ** 2, 0) / N)
    p64, n64 = p.astype(np.float64), n.astype(np.float64)
    for e in range(E):
        a, b = V[ed[e, 0]], V[ed[e, 1]]
        ts = np.linspace(0, 1, 65)
        pts = a + ts[:, None] * (b - a)
        d = pts - p64
        cmax = ((d @ n64) / np.linalg.norm(d, axis=1)).max()
        sil = _silhouette64(scene, V, faces, ed, e, p64)
        if last and not sil:  # the silhouette gate: never picked
            assert est[e] == 0.0, (e, est[e])
            continue
        if last and est[e] == 0.0 and cmax > 1e-3:
            # the light-cone bound removed it: no ray from p through the edge
            # (nor 1e-3 rad around it) reaches a light triangle
            assert not _reaches_light(scene, V, p64, pts, 1e-3), e
            continue
        # clearly above the horizon edges must be kept; every kept edge counts once
        if cmax > 1e-3 or est[e] > 0.0:
            assert abs(est[e] - 1.0) <= 6 * se[e] + 0.02, (e, est[e], se[e], cmax)
    # the picks that exist are all finite and positive
    assert np.all(np.isfinite(w)) and np.all(w[eid >= 0] > 0)


def _secondary_grads(scene, w, depth, samples, seeds):
    out = []
    for s in seeds:
        g, _ = oracle.backward(scene, w, spp=64, edge_spp=1, seed=s, max_depth=depth,
                               terms=oracle.TERM_SECONDARY, sec_tree_samples=samples, n_threads=NT)
        out.append(oracle.split_params(scene, g)["verts"].ravel())
    return np.array(out)


@pytest.mark.parametrize("depth", [1, 2])
def test_hierarchy_gradient_has_the_length_samplers_expectation(depth):
    """Both samplers estimate the same secondary edge term.  They differ by
    O(eps) where the side rays of a non-silhouette edge graze one of its
    faces (the length sampler sees those, the silhouette gate skips them),
    hence the floor of 1e-5 of the largest entry."""
    scene = _scene()
    w = sg.loss_adjoint(5, 16, 16)
    seeds = range(120)
    a = _secondary_grads(scene, w, depth, 0, seeds)
    b = _secondary_grads(scene, w, depth, 16, seeds)
    ma, mb = a.mean(0), b.mean(0)
    se = np.sqrt(a.var(0, ddof=1) / len(a) + b.var(0, ddof=1) / len(b))
    floor = 1e-5 * np.abs(ma).max()
    z = (ma - mb) / np.sqrt(se ** 2 + floor ** 2)
    assert np.sqrt(np.mean(z ** 2)) < 1.5 and np.abs(z).max() < 5.0, (np.sqrt(np.mean(z ** 2)), np.abs(z).max())
    # and the hierarchy is the better sampler here
    assert b.var(0).sum() < 0.7 * a.var(0).sum()


@pytest.mark.slow
def test_hierarchy_matches_the_blocker_closed_form():
    """The blocker's vertex derivatives come only from the secondary edge
    term; through the hierarchy they must still equal the derivative of the
    clipped-polygon closed form."""
    scene = _point_scene(True)
    lv = scene.verts[4:8].astype(np.float64)
    h = 1e-6
    want_b = np.zeros((3, 3))
    for i in range(3):
        for c in range(3):
            bp, bm = BLOCKER.copy(), BLOCKER.copy()
            bp[i, c] += h
            bm[i, c] -= h
            want_b[i, c] = (_closed_radiance(list(lv), bp).sum() - _closed_radiance(list(lv), bm).sum()) / (2 * h)
    w = np.ones((1, 1, 3), np.float32)
    got = []
    for s in range(8):
        g, _ = oracle.backward(scene, w, spp=20000, edge_spp=1, seed=700 + s, terms=oracle.TERM_SECONDARY,
                               sec_tree_samples=8, n_threads=NT)
        got.append(oracle.split_params(scene, g)["verts"][8:11])
    _zcheck(np.array(got), want_b, 3e-3)
