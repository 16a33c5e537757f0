"""CPU oracle for differentiable Monte Carlo ray tracing through edge sampling.

TEST INFRASTRUCTURE ONLY: tests, the package smoke check and the benchmark's
CPU-baseline leg may use this module; the product path never does.

A thin ctypes wrapper over ``oracle.cpp`` (see its header for the method and
the precision rules).  Scenes are any object with the attributes of
``paper_1904_12228_gb300.scenegen.Scene`` (numpy arrays), so this module
imports nothing from the CUDA package.

Parameter layout of gradients (length ``3V + 3T + 16``):
  [0, 3V)            vertex positions, [V,3] row-major
  [3V, 3V+3T)        per-triangle albedo, [T,3]
  [3V+3T, +3)        light radiance (RGB)
  [.., +12)          camera-to-world rows 0..2 (4 entries each)
  [.., +1)           camera scale (tan(fov_y/2) or ortho half height)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build

TERM_INTERIOR = 1
TERM_PRIMARY = 2
TERM_SECONDARY = 4
TERMS_ALL = 7

EPS_REL = 2.0 ** -16

_LIB = None


class _Scene(ctypes.Structure):
    _fields_ = [("n_verts", ctypes.c_int32), ("n_tris", ctypes.c_int32), ("n_light_tris", ctypes.c_int32),
                ("cam_type", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("verts", ctypes.c_void_p), ("tris", ctypes.c_void_p), ("albedo", ctypes.c_void_p),
                ("light_tris", ctypes.c_void_p), ("radiance", ctypes.c_void_p), ("cam_to_world", ctypes.c_void_p),
                ("cam_scale", ctypes.c_float)]


class _Opts(ctypes.Structure):
    _fields_ = [("spp", ctypes.c_int32), ("edge_spp", ctypes.c_int32), ("max_depth", ctypes.c_int32),
                ("primary_only", ctypes.c_int32), ("seed", ctypes.c_uint64), ("eps_rel", ctypes.c_float),
                ("terms", ctypes.c_int32), ("pix_begin", ctypes.c_int32), ("pix_end", ctypes.c_int32),
                ("edge_begin", ctypes.c_int64), ("edge_end", ctypes.c_int64), ("n_threads", ctypes.c_int32),
                ("scene_id", ctypes.c_int32), ("proposal", ctypes.c_int32), ("seg_weights", ctypes.c_void_p),
                ("n_seg_weights", ctypes.c_int64), ("sec_sampler", ctypes.c_int32), ("sec_tree_samples", ctypes.c_int32),
                ("sec_point", ctypes.c_int32), ("n_jac", ctypes.c_int32), ("jac_param", ctypes.c_int64 * 8),
                ("aov", ctypes.c_int32), ("sec_nee", ctypes.c_int32), ("nee_width", ctypes.c_float)]


def lib():
    global _LIB
    if _LIB is None:
        _LIB = ctypes.CDLL(build())
    return _LIB


def n_threads_default() -> int:
    return max(1, len(os.sched_getaffinity(0)))


class _Pinned:
    """Keeps the numpy arrays alive while the C structure points at them."""

    def __init__(self, scene):
        self.arrays = [np.ascontiguousarray(a, dtype=t) for a, t in (
            (scene.verts, np.float32), (scene.tris, np.int32), (scene.albedo, np.float32),
            (scene.light_tris, np.int32), (scene.radiance, np.float32), (scene.cam_to_world, np.float32))]
        v, t, a, lt, r, c = self.arrays
        self.s = _Scene(len(v), len(t), len(lt), int(scene.cam_type), int(scene.width), int(scene.height),
                        v.ctypes.data, t.ctypes.data, a.ctypes.data, lt.ctypes.data, r.ctypes.data, c.ctypes.data,
                        float(scene.cam_scale))


AOV_ALBEDO, AOV_POSITION, AOV_NORMAL, AOV_DEPTH = 1, 2, 3, 4


def _opts(spp, edge_spp, max_depth, primary_only, seed, eps_rel, terms, pixels, edges, n_threads, scene_id,
          weights=None, mode=1, sec_tree_samples=0, sec_point=0, aov=0):
    pb, pe = pixels if pixels is not None else (0, 0)
    eb, ee = edges if edges is not None else (0, 0)
    wp, wn = (weights.ctypes.data, len(weights)) if weights is not None else (None, 0)
    o = _Opts(int(spp), int(edge_spp), int(max_depth), int(bool(primary_only) or aov > 0), int(seed) & (2 ** 64 - 1),
              float(eps_rel), int(terms), int(pb), int(pe), int(eb), int(ee),
              int(n_threads or n_threads_default()), int(scene_id), mode if weights is not None else 0, wp, wn,
              1 if sec_tree_samples > 0 else 0, int(sec_tree_samples), int(sec_point))
    o.aov = int(aov)
    return o


def num_params(scene) -> int:
    return 3 * len(scene.verts) + 3 * len(scene.tris) + 3 + 13


def split_params(scene, g: np.ndarray) -> dict:
    """Split a flat gradient into named parts."""
    V, T = len(scene.verts), len(scene.tris)
    o = 0
    out = {}
    for name, n, shape in (("verts", 3 * V, (V, 3)), ("albedo", 3 * T, (T, 3)), ("radiance", 3, (3,)),
                           ("cam_to_world", 12, (3, 4)), ("cam_scale", 1, (1,))):
        out[name] = g[o:o + n].reshape(shape)
        o += n
    return out


def render(scene, *, spp: int, seed: int, max_depth: int = 1, primary_only: bool = False,
           pixels=None, n_threads=None, scene_id: int = 0, aov: int = 0) -> np.ndarray:
    """Image [H,W,3] (FP64).  ``pixels=(begin,end)`` restricts to a linear
    pixel range; other pixels are NaN.  aov > 0 renders a geometry buffer of
    the first hit (AOV_ALBEDO, AOV_POSITION, AOV_NORMAL, AOV_DEPTH)."""
    P = _Pinned(scene)
    o = _opts(spp, spp, max_depth, primary_only, seed, EPS_REL, 0, pixels, None, n_threads, scene_id, aov=aov)
    img = np.full((scene.height, scene.width, 3), np.nan, np.float64)
    rc = lib().or_render(ctypes.byref(P.s), ctypes.byref(o), img.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise RuntimeError("oracle render failed (%d)" % rc)
    return img


def backward(scene, d_image: np.ndarray, *, spp: int, edge_spp: int, seed: int, max_depth: int = 1,
             primary_only: bool = False, terms: int = TERMS_ALL, eps_rel: float = EPS_REL, pixels=None,
             edges=None, n_threads=None, scene_id: int = 0, proposal_weights=None, proposal_scores=None,
             sec_tree_samples: int = 0, sec_point: int = 0, contributions: bool = False, jacobian=None,
             aov: int = 0, sec_nee: int = 0, nee_width: float = 0.0):
    """Gradient of sum(d_image * image) as a flat FP64 vector, and per entry
    the magnitude of the terms summed into it (absolute-value chain rule),
    which scales the rounding error an FP32 implementation may make.
    proposal_weights: per tile segment (see segments()), selects the mixture
    proposal for primary edges.  proposal_scores: per tile segment, network
    scores s_k; the mixture then weighs segment k by len_k * exp(s_k), with
    s_k clamped to [-40, 40].  sec_tree_samples > 0 picks secondary edges
    through the edge hierarchy with that many root samples (else by length).
    sec_point = 1 samples the point on a secondary edge by the clamped-cosine
    density over the edge's arc, mixed with uniform (else uniform).
    contributions=True also returns, per entry, the sum over samples of the
    magnitude of each sample's whole contribution, sum_k |c_k| (a third
    array).  jacobian: up to 8 flat parameter indices; then the per-pixel
    shares of those gradient entries, [n, H, W], are returned last.  aov > 0:
    the gradient of a geometry buffer of the first hit (see render).
    sec_nee = 1 adds next-event estimation for edges (Sec. 5.3.3): at every
    shading vertex one more secondary edge sample from the billboards its
    shadow ray crosses, both samples weighed by the balance heuristic (with
    the length sampler and the uniform point only); nee_width is the
    billboards' width (<= 0: 2 % of the vertices' mean absolute deviation
    per coordinate, combined in L2)."""
    if proposal_weights is not None and proposal_scores is not None:
        raise ValueError("give proposal_weights or proposal_scores, not both")
    P = _Pinned(scene)
    w = np.ascontiguousarray(d_image, dtype=np.float32).reshape(scene.height, scene.width, 3)
    mode, pw = 1, proposal_weights
    if proposal_scores is not None:
        mode, pw = 2, proposal_scores
    pw = None if pw is None else np.ascontiguousarray(pw, np.float32)
    o = _opts(spp, edge_spp, max_depth, primary_only, seed, eps_rel, terms, pixels, edges, n_threads, scene_id,
              pw, mode, sec_tree_samples, sec_point, aov)
    o.sec_nee = int(sec_nee)
    o.nee_width = float(nee_width)
    n = num_params(scene)
    g = np.zeros(n, np.float64)
    a = np.zeros(n, np.float64)
    c = np.zeros(n, np.float64) if contributions else None
    jac = None
    if jacobian is not None:
        idx = [int(i) for i in jacobian]
        if not 1 <= len(idx) <= 8 or min(idx) < 0 or max(idx) >= n:
            raise ValueError("jacobian takes 1 to 8 parameter indices in [0, %d)" % n)
        o.n_jac = len(idx)
        for k, i in enumerate(idx):
            o.jac_param[k] = i
        jac = np.zeros((len(idx), scene.height, scene.width), np.float64)
    rc = lib().or_backward4(ctypes.byref(P.s), ctypes.byref(o), w.ctypes.data_as(ctypes.c_void_p),
                            g.ctypes.data_as(ctypes.c_void_p), a.ctypes.data_as(ctypes.c_void_p),
                            c.ctypes.data_as(ctypes.c_void_p) if c is not None else None,
                            jac.ctypes.data_as(ctypes.c_void_p) if jac is not None else None)
    if rc != 0:
        raise RuntimeError("oracle backward failed (%d)" % rc)
    out = (g, a, c) if contributions else (g, a)
    return out + (jac,) if jac is not None else out


def edge_point(p, n, v0, v1, u: float, usel: float):
    """Point t on the edge v0 -> v1 seen from p with unit normal n, drawn by
    the clamped-cosine arc density mixed with uniform from the uniforms u
    (position) and usel (mixture component); returns (t, q(t))."""
    arrs = [np.ascontiguousarray(a, np.float32) for a in (p, n, v0, v1)]
    t = ctypes.c_float()
    q = ctypes.c_double()
    lib().or_edge_point(*[a.ctypes.data_as(ctypes.c_void_p) for a in arrs], ctypes.c_float(u), ctypes.c_float(usel),
                        ctypes.byref(t), ctypes.byref(q))
    return float(t.value), float(q.value)


def ln32(x: float) -> float:
    """The FP32 natural logarithm of next-event estimation for edges' race."""
    f = lib().or_ln32
    f.restype = ctypes.c_float
    return float(f(ctypes.c_float(x)))


def nee_half_width(scene) -> float:
    """Half the billboard width derived from the scene's vertices."""
    P = _Pinned(scene)
    f = lib().or_nee_half_width
    f.restype = ctypes.c_float
    return float(f(ctypes.byref(P.s)))


class NeeQuery:
    """Next-event estimation for edges (Sec. 5.3.3) on one scene: billboard
    crossings of a ray, the race's pick, the ray of an edge's family through
    (t, u), its Jacobian and the sampler's density."""

    def __init__(self, scene):
        self._pin = _Pinned(scene)
        L = lib()
        L.or_nee_open.restype = ctypes.c_void_p
        L.or_nee_jacobian.restype = ctypes.c_double
        self._h = ctypes.c_void_p(L.or_nee_open(ctypes.byref(self._pin.s)))

    def close(self):
        if self._h:
            lib().or_nee_close(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _f3(a):
        return np.ascontiguousarray(a, np.float32).reshape(3)

    def crossings(self, p, n, d, smax, hw, cap=4096):
        """(edge ids, [n, 4] of s, t, u, importance) of the billboards the ray
        p + s d crosses for s in (0, smax); n: the shading normal at p."""
        p, n, d = self._f3(p), self._f3(n), self._f3(d)
        eid = np.zeros(cap, np.int32)
        stui = np.zeros((cap, 4), np.float32)
        n = lib().or_nee_crossings(self._h, p.ctypes.data_as(ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p),
                                   d.ctypes.data_as(ctypes.c_void_p),
                                   ctypes.c_float(smax), ctypes.c_float(hw), eid.ctypes.data_as(ctypes.c_void_p),
                                   stui.ctypes.data_as(ctypes.c_void_p), cap)
        n = min(n, cap)
        return eid[:n].copy(), stui[:n].copy()

    def pick(self, p, n, d, smax, hw, key0, key1) -> int:
        p, n, d = self._f3(p), self._f3(n), self._f3(d)
        return int(lib().or_nee_pick(self._h, p.ctypes.data_as(ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p),
                                     d.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.c_float(smax), ctypes.c_float(hw), ctypes.c_uint32(key0),
                                     ctypes.c_uint32(key1)))

    def ray(self, eid, p, t, u):
        p = self._f3(p)
        d = np.zeros(3, np.float32)
        ok = lib().or_nee_ray(self._h, int(eid), p.ctypes.data_as(ctypes.c_void_p), ctypes.c_float(t),
                              ctypes.c_float(u), d.ctypes.data_as(ctypes.c_void_p))
        return d if ok else None

    def jacobian(self, eid, p, t, u) -> float:
        p = self._f3(p)
        return float(lib().or_nee_jacobian(self._h, int(eid), p.ctypes.data_as(ctypes.c_void_p), ctypes.c_float(t),
                                           ctypes.c_float(u)))

    def density(self, p, n, d, eid, t, u, hw) -> np.ndarray:
        """p_B at samples: p [n,3], normals n [n,3], d [n,3], eid [n], t [n], u [n]."""
        p = np.ascontiguousarray(p, np.float32).reshape(-1, 3)
        nrm = np.ascontiguousarray(n, np.float32).reshape(-1, 3)
        d = np.ascontiguousarray(d, np.float32).reshape(-1, 3)
        eid = np.ascontiguousarray(eid, np.int32).reshape(-1)
        t = np.ascontiguousarray(t, np.float32).reshape(-1)
        u = np.ascontiguousarray(u, np.float32).reshape(-1)
        out = np.zeros(len(eid), np.float64)
        lib().or_nee_density(self._h, len(eid), p.ctypes.data_as(ctypes.c_void_p),
                             nrm.ctypes.data_as(ctypes.c_void_p), d.ctypes.data_as(ctypes.c_void_p),
                             eid.ctypes.data_as(ctypes.c_void_p), t.ctypes.data_as(ctypes.c_void_p),
                             u.ctypes.data_as(ctypes.c_void_p), ctypes.c_float(hw),
                             out.ctypes.data_as(ctypes.c_void_p))
        return out


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox(c.ctypes.data_as(ctypes.c_void_p), k.ctypes.data_as(ctypes.c_void_p),
                    out.ctypes.data_as(ctypes.c_void_p))
    return out


def closest(scene, o: np.ndarray, d: np.ndarray, n_threads=None):
    """Brute-force closest hits for rays [N,3]: (tri [N], (t,b1,b2) [N,3])."""
    P = _Pinned(scene)
    o = np.ascontiguousarray(o, np.float32).reshape(-1, 3)
    d = np.ascontiguousarray(d, np.float32).reshape(-1, 3)
    n = len(o)
    tri = np.zeros(n, np.int32)
    tb = np.zeros((n, 3), np.float32)
    lib().or_closest_batch(ctypes.byref(P.s), ctypes.c_int(n), o.ctypes.data_as(ctypes.c_void_p),
                           d.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(n_threads or n_threads_default()),
                           tri.ctypes.data_as(ctypes.c_void_p), tb.ctypes.data_as(ctypes.c_void_p))
    return tri, tb


def edges(scene) -> np.ndarray:
    P = _Pinned(scene)
    cap = 3 * len(scene.tris)
    out = np.zeros((cap, 2), np.int32)
    n = lib().or_edges(ctypes.byref(P.s), out.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(cap))
    return out[:n]


def primary_edges(scene) -> np.ndarray:
    """[E,7] = (ax, ay, bx, by, t0, t1, clipped screen length)."""
    P = _Pinned(scene)
    cap = 3 * len(scene.tris)
    out = np.zeros((cap, 7), np.float64)
    n = lib().or_primary_edges(ctypes.byref(P.s), out.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(cap))
    return out[:n]


def segments(scene):
    """Tile segments of the clipped primary edges: (edge, tile) int arrays,
    (s0, s1) float32 parameters along the edge, FP64 screen lengths."""
    P = _Pinned(scene)
    cap = 3 * len(scene.tris) * (2 + (scene.width + scene.height) // 16)
    out = np.zeros((cap, 4), np.float64)
    lens = np.zeros(cap, np.float64)
    lib().or_segments.restype = ctypes.c_int64
    n = lib().or_segments(ctypes.byref(P.s), out.ctypes.data_as(ctypes.c_void_p),
                          lens.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(cap))
    out = out[:n]
    return out[:, 0].astype(np.int32), out[:, 1].astype(np.int32), out[:, 2:].astype(np.float32), lens[:n]


def atan2_pos(y: float, x: float) -> float:
    """FP32 atan2 for y >= 0 with the oracle's fixed operation order."""
    f = lib().or_atan2_pos
    f.restype = ctypes.c_float
    return float(f(ctypes.c_float(y), ctypes.c_float(x)))


def camera_ray(scene, sx: float, sy: float):
    """FP32 camera ray (origin, direction) through screen point (sx, sy)."""
    P = _Pinned(scene)
    o = np.zeros(3, np.float32)
    d = np.zeros(3, np.float32)
    lib().or_camera_ray(ctypes.byref(P.s), ctypes.c_float(sx), ctypes.c_float(sy), o.ctypes.data_as(ctypes.c_void_p),
                        d.ctypes.data_as(ctypes.c_void_p))
    return o, d


def fisheye_project(scene, v):
    """FP32 screen point of world point v under the fisheye camera, or None."""
    P = _Pinned(scene)
    va = np.ascontiguousarray(v, np.float32)
    sx, sy = ctypes.c_float(), ctypes.c_float()
    ok = lib().or_fisheye_project(ctypes.byref(P.s), va.ctypes.data_as(ctypes.c_void_p), ctypes.byref(sx),
                                  ctypes.byref(sy))
    return (sx.value, sy.value) if ok else None


def sincos_2pi(r: float):
    c = ctypes.c_float()
    s = ctypes.c_float()
    lib().or_sincos_2pi(ctypes.c_float(r), ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def sec_edge_forms(p, v0, v1, t, nm, plane_d) -> np.ndarray:
    """Area-form and solid-angle-form secondary edge weights (see oracle.cpp)."""
    arr = [np.ascontiguousarray(x, np.float64) for x in (p, v0, v1, nm)]
    out = np.zeros(12, np.float64)
    lib().or_sec_edge_forms(arr[0].ctypes.data_as(ctypes.c_void_p), arr[1].ctypes.data_as(ctypes.c_void_p),
                            arr[2].ctypes.data_as(ctypes.c_void_p), ctypes.c_double(t),
                            arr[3].ctypes.data_as(ctypes.c_void_p), ctypes.c_double(plane_d),
                            out.ctypes.data_as(ctypes.c_void_p))
    return out


def edge_tree(scene):
    """The secondary edge hierarchy: children [n,2] (>= 0 node, < 0 ~leaf
    position), slots [n,2,14] = (lo, hi, Hough lo, Hough hi, total length,
    all class B), leaves [E,3] = (edge id, class B, boundary), root code."""
    P = _Pinned(scene)
    cap = 3 * len(scene.tris)
    nodes = np.zeros((cap, 2), np.int32)
    slots = np.zeros((cap, 2, 14), np.float32)
    leaves = np.zeros((cap, 3), np.int32)
    root = ctypes.c_int32()
    n = lib().or_edge_tree(ctypes.byref(P.s), nodes.ctypes.data_as(ctypes.c_void_p),
                           slots.ctypes.data_as(ctypes.c_void_p), leaves.ctypes.data_as(ctypes.c_void_p),
                           ctypes.c_int(cap), ctypes.byref(root))
    n_edges = len(edges(scene))
    return nodes[:n], slots[:n], leaves[:n_edges], root.value


def edge_tree_vsphere(scene, p) -> np.ndarray:
    """[n,2] bool: the v-sphere of shading point p clears the slot's Hough box."""
    P = _Pinned(scene)
    nodes, _, _, _ = edge_tree(scene)
    out = np.zeros((max(1, len(nodes)), 2), np.uint8)
    pa = np.ascontiguousarray(p, np.float32)
    lib().or_edge_tree_vsphere(ctypes.byref(P.s), pa.ctypes.data_as(ctypes.c_void_p),
                               out.ctypes.data_as(ctypes.c_void_p))
    return out[:len(nodes)].astype(bool)


def edge_tree_cos_bound(p, n, lo, hi) -> float:
    arr = [np.ascontiguousarray(x, np.float32) for x in (p, n, lo, hi)]
    f = lib().or_edge_tree_cos_bound
    f.restype = ctypes.c_float
    return float(f(*[a.ctypes.data_as(ctypes.c_void_p) for a in arr]))


def edge_tree_picks(scene, p, n, *, last: bool, samples: int, n_picks: int, seed: int = 0, bounce: int = 0,
                    scene_id: int = 0, eps_rel: float = EPS_REL):
    """n_picks hierarchical picks at shading point p (unit normal n), with
    Philox counters (0, i): edge ids (-1: none) and resampling weights."""
    P = _Pinned(scene)
    pa = np.ascontiguousarray(p, np.float32)
    na = np.ascontiguousarray(n, np.float32)
    eid = np.zeros(n_picks, np.int32)
    w = np.zeros(n_picks, np.float32)
    lib().or_edge_tree_picks(ctypes.byref(P.s), pa.ctypes.data_as(ctypes.c_void_p), na.ctypes.data_as(ctypes.c_void_p),
                             ctypes.c_int(int(last)), ctypes.c_int(samples), ctypes.c_float(eps_rel),
                             ctypes.c_uint64(int(seed) & (2 ** 64 - 1)), ctypes.c_int(bounce), ctypes.c_int(scene_id),
                             ctypes.c_int(n_picks), eid.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p))
    return eid, w
