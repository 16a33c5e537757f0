"""Whole-method pin of the oracle: its gradient (interior + primary edges +
secondary edges) against central finite differences of its own image with
common random numbers, on a small lit scene (the validation protocol of
Sec. 5.4.1, "comparison with central finite differences").

Both sides are Monte Carlo estimates, so the check is a z-test over
independent seeds: for every probed parameter the two means agree within
4.5 combined standard errors.  A dropped term (edge or interior), a wrong
sign or a wrong measure shows up as a difference of many standard errors.
"""
import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg

NT = oracle.n_threads_default()


def _loss(scene, w, spp, seed, max_depth=1):
    return float((oracle.render(scene, spp=spp, seed=seed, max_depth=max_depth, n_threads=NT) * w).sum())


def _perturbed(scene, kind, idx, h):
    s = scene.copy()
    if kind == "verts":
        s.verts[idx] += h
    elif kind == "cam":
        s.cam_to_world[idx] += h
    elif kind == "scale":
        s.cam_scale = float(np.float32(s.cam_scale + h))
    return s


@pytest.mark.slow
def test_gradient_matches_central_differences():
    scene = sg.direct_lighting(1236, width=16, height=16, subdiv=1)
    V = len(scene.verts)
    w = sg.loss_adjoint(4, scene.width, scene.height)
    probes = [("verts", (0, 0)), ("verts", (0, 1)), ("verts", (V - 8, 1)), ("verts", (V - 3, 0)),
              ("verts", (V - 2, 2)), ("cam", (0, 3)), ("scale", None)]
    K = 8
    ours = []
    for k in range(K):
        g, _ = oracle.backward(scene, w, spp=1024, edge_spp=1024, seed=300 + k, n_threads=NT)
        sp = oracle.split_params(scene, g)
        row = []
        for kind, idx in probes:
            if kind == "verts":
                row.append(sp["verts"][idx])
            elif kind == "cam":
                row.append(sp["cam_to_world"][idx])
            else:
                row.append(sp["cam_scale"][0])
        ours.append(row)
    ours = np.array(ours)
    h = 1e-2
    fd = []
    for k in range(K):
        row = []
        for kind, idx in probes:
            hh = h if kind != "scale" else h / 2
            lp = _loss(_perturbed(scene, kind, idx, hh), w, 4096, 1700 + k)
            lm = _loss(_perturbed(scene, kind, idx, -hh), w, 4096, 1700 + k)
            row.append((lp - lm) / (2 * hh))
        fd.append(row)
    fd = np.array(fd)
    mo, mf = ours.mean(0), fd.mean(0)
    se = np.sqrt(ours.var(0, ddof=1) / K + fd.var(0, ddof=1) / K)
    z = np.abs(mo - mf) / se
    assert np.all(z < 4.5), list(zip(probes, mo, mf, se))
    # and the estimate is not trivially zero
    assert np.abs(mo).max() > 0.1
