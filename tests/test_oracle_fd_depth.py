"""Pins of the oracle's paths with two and three scattering vertices (CPU).

1. Central finite differences (the validation protocol of Sec. 5.4.1): the
   oracle's gradient, interior + primary edges + secondary edges, against
   central differences of its own image with common random numbers, as a
   z-test over independent seeds, on a scene lit only through reflections
   (scenegen.indirect_panel).  Its camera looks up at a panel the light cannot
   reach: every pixel's radiance comes through the cosine-hemisphere
   continuation, next-event estimation at the second and third vertex, and
   the secondary edge term in its solid-angle form (continuation) and area
   form (next event) at later vertices.
   The same seeds also give each term alone: dropping the secondary, the
   interior or (with the blocker's silhouette in view) the primary term must
   move some probe many standard errors away from the finite differences, so
   the test can tell a dropped term.
2. Exact identities at depth 3, per seed: translation invariance of every
   term and homogeneity in the emitted radiance.
"""
import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg

NT = oracle.n_threads_default()

# vertex ids of indirect_panel: floor 0-3, panel 4-7, light 8-11, blocker 12-14, wall 15-18
PROBES = [("verts", (12, 0)), ("verts", (13, 1)), ("verts", (14, 2)), ("verts", (13, 0)), ("verts", (9, 0)),
          ("verts", (1, 2)), ("verts", (5, 1)), ("verts", (16, 0)), ("cam", (0, 3)), ("scale", None)]


def _perturbed(scene, kind, idx, h):
    s = scene.copy()
    if kind == "verts":
        s.verts[idx] += h
    elif kind == "cam":
        s.cam_to_world[idx] += h
    else:
        s.cam_scale = float(np.float32(s.cam_scale + h))
    return s


def _pick(sp, kind, idx):
    if kind == "verts":
        return sp["verts"][idx]
    if kind == "cam":
        return sp["cam_to_world"][idx]
    return sp["cam_scale"][0]


@pytest.mark.slow
@pytest.mark.parametrize("view,depth", [("interior", 2), ("silhouette", 3)])
def test_gradient_matches_central_differences_beyond_depth_one(view, depth):
    scene = sg.indirect_panel(view)
    if depth == 3:  # the third vertex adds light (panel -> floor -> wall)
        assert not np.allclose(oracle.render(scene, spp=64, seed=1, max_depth=3, n_threads=NT),
                               oracle.render(scene, spp=64, seed=1, max_depth=2, n_threads=NT))
    w = np.ones((scene.height, scene.width, 3), np.float32)
    K, spp_g, spp_fd, h = 8, 1024, 1024, 0.02
    terms = {}
    for term in (oracle.TERM_INTERIOR, oracle.TERM_PRIMARY, oracle.TERM_SECONDARY):
        rows = []
        for k in range(K):
            g, _ = oracle.backward(scene, w, spp=spp_g, edge_spp=spp_g, seed=300 + k, max_depth=depth, terms=term,
                                   n_threads=NT)
            sp = oracle.split_params(scene, g)
            rows.append([_pick(sp, kind, idx) for kind, idx in PROBES])
        terms[term] = np.array(rows)
    ours = sum(terms.values())
    fd = []
    for k in range(K):
        row = []
        for kind, idx in PROBES:
            hh = h if kind != "scale" else h / 2
            lp = float((oracle.render(_perturbed(scene, kind, idx, hh), spp=spp_fd, seed=1700 + k, max_depth=depth,
                                      n_threads=NT) * w).sum())
            lm = float((oracle.render(_perturbed(scene, kind, idx, -hh), spp=spp_fd, seed=1700 + k, max_depth=depth,
                                      n_threads=NT) * w).sum())
            row.append((lp - lm) / (2 * hh))
        fd.append(row)
    fd = np.array(fd)
    se = np.sqrt(ours.var(0, ddof=1) / K + fd.var(0, ddof=1) / K)

    def z(est):
        return np.abs(est.mean(0) - fd.mean(0)) / se

    assert np.all(z(ours) < 4.5), list(zip(PROBES, ours.mean(0), fd.mean(0), se))
    # power: the test tells a dropped term
    assert z(ours - terms[oracle.TERM_SECONDARY]).max() > 8.0
    assert z(ours - terms[oracle.TERM_INTERIOR]).max() > 8.0
    if view == "silhouette":
        assert z(ours - terms[oracle.TERM_PRIMARY]).max() > 8.0


@pytest.mark.parametrize("scene_name", ["lit", "indirect"])
def test_translation_invariance_at_depth_three(scene_name):
    """Moving every vertex and the camera together leaves the image unchanged
    (the continuation directions are drawn about the surface normal, so they
    move with it): sum_v dL/dv + dL/d(camera position) = 0 per seed and per
    term, through three scattering vertices."""
    scene = sg.direct_lighting(1236, width=12, height=10, subdiv=1) if scene_name == "lit" \
        else sg.indirect_panel("silhouette", 10, 10)
    w = sg.loss_adjoint(2, scene.width, scene.height)
    for terms in (oracle.TERM_INTERIOR, oracle.TERM_PRIMARY, oracle.TERM_SECONDARY):
        g, a = oracle.backward(scene, w, spp=4, edge_spp=4, seed=9, max_depth=3, terms=terms, n_threads=NT)
        sp = oracle.split_params(scene, g)
        total = sp["verts"].sum(0) + sp["cam_to_world"][:, 3]
        scale = oracle.split_params(scene, a)["verts"].sum() + 1e-30
        assert np.all(np.abs(total) <= 1e-9 * scale), (terms, total, scale)
        assert np.abs(sp["verts"]).sum() > 0


@pytest.mark.parametrize("scene_name", ["lit", "indirect"])
def test_radiance_homogeneity_at_depth_three(scene_name):
    """Emission enters every path once (at the camera hit or through next-event
    estimation), so the image is linear in the radiance: per seed,
    sum_c Le_c dL/dLe_c = sum_p w_p . I_p at depth 3."""
    scene = sg.direct_lighting(1236, width=12, height=10, subdiv=1) if scene_name == "lit" \
        else sg.indirect_panel("silhouette", 10, 10)
    w = sg.loss_adjoint(3, scene.width, scene.height)
    img = oracle.render(scene, spp=4, seed=21, max_depth=3, n_threads=NT)
    g, _ = oracle.backward(scene, w, spp=4, edge_spp=4, seed=21, max_depth=3, terms=oracle.TERM_INTERIOR,
                           n_threads=NT)
    gr = oracle.split_params(scene, g)["radiance"]
    lhs = float((np.asarray(scene.radiance, np.float64) * gr).sum())
    rhs = float((w.astype(np.float64) * img).sum())
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(rhs))
    assert rhs != 0.0
