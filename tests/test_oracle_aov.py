"""Pins of the oracle's geometry buffers (the AOV extension of Sec. 5.4):
world position, shading normal and depth of the first hit.

Their gradient (interior derivative of the buffer at fixed screen samples
plus the primary edge term of the buffer's discontinuities) against central
finite differences of the buffer images with common random numbers, as a
z-test over seeds; the same seeds without the edge term must miss the finite
differences on some probe, so the test tells a dropped term.  And exact
identities per seed: a joint translation of scene and camera leaves the
normal and depth buffers unchanged and shifts the position buffer by the
translation."""
import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg

NT = oracle.n_threads_default()


def _scene():
    return sg.direct_lighting(1236, width=16, height=16, subdiv=1)


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


@pytest.mark.parametrize("aov", [oracle.AOV_POSITION, oracle.AOV_NORMAL, oracle.AOV_DEPTH])
def test_geometry_buffer_gradient_matches_central_differences(aov):
    scene = _scene()
    V = len(scene.verts)
    w = sg.loss_adjoint(11, scene.width, scene.height)
    probes = [("verts", (0, 0)), ("verts", (3, 1)), ("verts", (9, 2)), ("verts", (V - 7, 1)), ("cam", (0, 3)),
              ("cam", (2, 3)), ("scale", None)]
    K, spp, h = 8, 256, 1e-2
    interior, edge = [], []
    for k in range(K):
        for term, acc in ((oracle.TERM_INTERIOR, interior), (oracle.TERM_PRIMARY, edge)):
            g, _ = oracle.backward(scene, w, spp=spp, edge_spp=spp, seed=500 + k, terms=term, aov=aov, n_threads=NT)
            sp = oracle.split_params(scene, g)
            acc.append([_pick(sp, kind, idx) for kind, idx in probes])
    interior, edge = np.array(interior), np.array(edge)
    ours = interior + edge
    fd = []
    for k in range(K):
        row = []
        for kind, idx in probes:
            hh = h if kind != "scale" else h / 4
            lp = float((oracle.render(_perturbed(scene, kind, idx, hh), spp=1024, seed=900 + k, aov=aov,
                                      n_threads=NT) * w).sum())
            lm = float((oracle.render(_perturbed(scene, kind, idx, -hh), spp=1024, seed=900 + k, aov=aov,
                                      n_threads=NT) * w).sum())
            row.append((lp - lm) / (2 * hh))
        fd.append(row)
    fd = np.array(fd)
    # the two-sided evaluation a finite offset apart leaves an O(eps) bias on
    # edges whose sides see one smoothly varying surface (a hidden edge, whose
    # finite difference is exactly zero): a floor of 1e-3 of the largest
    # probe covers it
    se = np.sqrt(ours.var(0, ddof=1) / K + fd.var(0, ddof=1) / K + (1e-3 * np.abs(fd.mean(0)).max()) ** 2)

    def z(est):
        return np.abs(est.mean(0) - fd.mean(0)) / se

    assert np.all(z(ours) < 4.5), list(zip(probes, ours.mean(0), fd.mean(0), se))
    assert z(interior).max() > 8.0  # the edge term is needed
    assert np.abs(ours.mean(0)).max() > 0.01


def test_geometry_buffers_under_a_joint_translation():
    """Per seed, exactly (up to rounding): translating every vertex and the
    camera by the same vector leaves the depth and normal buffers unchanged,
    so sum_v dL/dv + dL/d(camera position) = 0; the position buffer moves
    with the translation, so the same sum equals the summed channel weights
    of the covered samples, i.e. sum_p w_p . (albedo-buffer image with unit
    albedo) per axis."""
    scene = _scene()
    scene.albedo = np.ones_like(scene.albedo)
    w = sg.loss_adjoint(12, scene.width, scene.height)
    cover = oracle.render(scene, spp=4, seed=3, aov=oracle.AOV_ALBEDO, n_threads=NT)  # 1 where a sample hits
    for aov in (oracle.AOV_NORMAL, oracle.AOV_DEPTH, oracle.AOV_POSITION):
        for terms in (oracle.TERM_INTERIOR, oracle.TERM_PRIMARY):
            g, a = oracle.backward(scene, w, spp=4, edge_spp=4, seed=3, terms=terms, aov=aov, n_threads=NT)
            sp = oracle.split_params(scene, g)
            total = sp["verts"].sum(0) + sp["cam_to_world"][:, 3]
            scale = oracle.split_params(scene, a)["verts"].sum() + 1e-30
            want = np.zeros(3)
            if aov == oracle.AOV_POSITION and terms == oracle.TERM_INTERIOR:
                want = (w.astype(np.float64) * cover).sum(axis=(0, 1))
            assert np.all(np.abs(total - want) <= 1e-9 * scale), (aov, terms, total, want)
