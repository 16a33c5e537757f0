"""Pins of the oracle's importance sampling of the point on a secondary edge
(Sec. 5.3.2: the Lambertian case, where the linearly transformed cosine is
the clamped cosine itself), against its definition, not against the oracle:

- the density q(t) is 1/4 + 3/4 q_c(t), with q_c the clamped cosine
  (n . omega_hat)^+ times the arc measure d theta / dt of the edge seen from
  p, normalised by brute-force quadrature in FP64 here;
- the sampler's draws follow that density (Kolmogorov-Smirnov);
- degenerate configurations keep the uniform point (q = 1);
- the secondary-edge gradient with the sampler has the uniform point's
  expectation, and matches the blocker's closed-form derivative.
"""
import numpy as np
import pytest

import oracle
from paper_1904_12228_gb300 import scenegen as sg
from tests.test_oracle_pins import BLOCKER, _closed_radiance, _point_scene, _zcheck

NT = oracle.n_threads_default()


def _configs(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        p = rng.normal(size=3)
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        v0 = p + rng.normal(size=3) * rng.uniform(0.5, 5.0)
        v1 = v0 + rng.normal(size=3) * rng.uniform(0.01, 2.0)
        out.append(tuple(np.asarray(a, np.float32) for a in (p, nrm, v0, v1)))
    return out


def _clamped_cosine_arc(p, n, v0, v1, t):
    """(n . omega_hat)^+ d theta / dt at t, in FP64 from the definition."""
    p, n, v0, v1 = (np.asarray(a, np.float64) for a in (p, n, v0, v1))
    E = v1 - v0
    w = (v0 - p)[None, :] + t[:, None] * E[None, :]
    r = np.linalg.norm(w, axis=1)
    cos = (w @ n) / r
    dtheta = np.linalg.norm(np.cross(w, E[None, :]), axis=1) / r ** 2  # |omega x E| / |omega|^2
    return np.maximum(cos, 0.0) * dtheta


def test_density_is_the_mixture_with_the_normalised_clamped_cosine():
    M = 40000
    ts = (np.arange(M) + 0.5) / M
    checked = 0
    for p, n, v0, v1 in _configs(3, 40):
        g = _clamped_cosine_arc(p, n, v0, v1, ts)
        Z = g.mean()
        q = np.array([oracle.edge_point(p, n, v0, v1, float(t), 0.0)[1] for t in ts[::97]])
        if Z < 1e-6:
            assert np.all(q == 1.0)
            continue
        want = 0.25 + 0.75 * g[::97] / Z
        # midpoint quadrature of a function with one kink (the horizon)
        assert np.allclose(q, want, rtol=2e-4, atol=1e-9), (np.abs(q - want) / want).max()
        checked += 1
    assert checked >= 12


def test_draws_follow_the_density():
    rng = np.random.default_rng(9)
    M = 20000
    ts = (np.arange(M) + 0.5) / M
    for p, n, v0, v1 in _configs(5, 8):
        g = _clamped_cosine_arc(p, n, v0, v1, ts)
        if g.mean() < 1e-6:
            continue
        cdf = np.cumsum(g) / g.sum()
        us = rng.random(8000).astype(np.float32)
        draws = np.sort([oracle.edge_point(p, n, v0, v1, float(u), 0.9)[0] for u in us])
        emp = np.searchsorted(draws, ts) / len(draws)
        assert np.abs(emp - cdf).max() < 1.63 / np.sqrt(len(draws)) + 2e-3  # KS at 1 %
        # the uniform component returns the uniform number itself
        assert oracle.edge_point(p, n, v0, v1, 0.375, 0.1)[0] == 0.375


def test_degenerate_cases_keep_the_uniform_point():
    p = np.zeros(3, np.float32)
    v0 = np.array([1, -1, 2], np.float32)
    v1 = np.array([1, 1, 2], np.float32)
    # normal perpendicular to the plane of p and the edge
    n_perp = np.cross(v0, v1).astype(np.float64)
    n_perp = (n_perp / np.linalg.norm(n_perp)).astype(np.float32)
    assert oracle.edge_point(p, n_perp, v0, v1, 0.3, 0.9) == (pytest.approx(0.3), 1.0)
    # the whole edge below the horizon
    n_down = np.array([-1, 0, 0], np.float32)
    assert oracle.edge_point(p, n_down, v0, v1, 0.3, 0.9) == (pytest.approx(0.3), 1.0)
    # the edge's line through p
    on = np.array([0, 0, 1], np.float32), np.array([0, 0, 3], np.float32)
    assert oracle.edge_point(p, np.array([0, 0, 1], np.float32), *on, 0.3, 0.9) == (pytest.approx(0.3), 1.0)
    # symmetric edge straight above: the cosine branch's median is the foot
    n_up = np.array([1, 0, 0], np.float32)
    t, q = oracle.edge_point(p, n_up, v0, v1, 0.5, 0.9)
    assert abs(t - 0.5) < 1e-6 and q > 1.0


def _secondary_grads(scene, w, depth, point, seeds):
    out = []
    for s in seeds:
        g, _ = oracle.backward(scene, w, spp=64, edge_spp=1, seed=s, max_depth=depth, terms=oracle.TERM_SECONDARY,
                               sec_point=point, n_threads=NT)
        out.append(oracle.split_params(scene, g)["verts"].ravel())
    return np.array(out)


@pytest.mark.parametrize("depth", [1, 2])
def test_gradient_has_the_uniform_points_expectation(depth):
    scene = sg.direct_lighting(11, width=16, height=16, subdiv=1)
    w = sg.loss_adjoint(5, 16, 16)
    seeds = range(100)
    a = _secondary_grads(scene, w, depth, 0, seeds)
    b = _secondary_grads(scene, w, depth, 1, seeds)
    ma, mb = a.mean(0), b.mean(0)
    se = np.sqrt(a.var(0, ddof=1) / len(a) + b.var(0, ddof=1) / len(b))
    floor = 1e-5 * np.abs(ma).max()
    z = (ma - mb) / np.sqrt(se ** 2 + floor ** 2)
    assert np.sqrt(np.mean(z ** 2)) < 1.5 and np.abs(z).max() < 5.0, (np.sqrt(np.mean(z ** 2)), np.abs(z).max())
    assert not np.allclose(a, b)


@pytest.mark.slow
def test_point_sampling_matches_the_blocker_closed_form():
    """The blocker's vertex derivatives come only from the secondary edge
    term; with the importance-sampled point they must still equal the
    derivative of the clipped-polygon closed form."""
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
        g, _ = oracle.backward(scene, w, spp=20000, edge_spp=1, seed=900 + s, terms=oracle.TERM_SECONDARY,
                               sec_point=1, n_threads=NT)
        got.append(oracle.split_params(scene, g)["verts"][8:11])
    _zcheck(np.array(got), want_b, 3e-3)


def test_inverse_lands_where_the_cdf_reaches_u():
    """The closed-form inverse: the CDF of the clamped-cosine density at the
    returned t equals u (FP64 quadrature of the definition), up to FP32
    rounding of the inverse."""
    M = 200000
    ts = (np.arange(M) + 0.5) / M
    checked = 0
    for p, n, v0, v1 in _configs(11, 30):
        g = _clamped_cosine_arc(p, n, v0, v1, ts)
        if g.mean() < 1e-6:
            continue
        cdf = np.concatenate([[0.0], np.cumsum(g) / g.sum()])
        grid = np.concatenate([[0.0], (np.arange(M) + 1.0) / M])
        for u in (0.05, 0.3, 0.5, 0.77, 0.95):
            t, _ = oracle.edge_point(p, n, v0, v1, u, 0.9)
            assert abs(np.interp(t, grid, cdf) - u) < 2e-4, (u, t)  # measured worst 2.7e-5
        checked += 1
    assert checked >= 8
