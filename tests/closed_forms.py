"""Closed-form references used to pin the oracle (FP64 numpy).

Each function restates a textbook result, independent of the oracle:
polygon clipping (Sutherland-Hodgman), the shoelace area, Liang-Barsky
segment clipping, Lambert's formula for the irradiance from a uniformly
emitting polygon, and the Reynolds transport theorem for the boundary
derivative of a moving polygon's area (Sec. 5.2.4).
"""
import numpy as np


def clip_polygon(poly, inside, intersect):
    """Sutherland-Hodgman clip of a polygon against one half-plane."""
    out = []
    n = len(poly)
    for i in range(n):
        cur, prev = poly[i], poly[i - 1]
        ci, pi = inside(cur), inside(prev)
        if ci:
            if not pi:
                out.append(intersect(prev, cur))
            out.append(cur)
        elif pi:
            out.append(intersect(prev, cur))
    return out


def clip_to_box(poly, x0, y0, x1, y1):
    def axis_clip(poly, k, bound, keep_ge):
        def inside(p):
            return p[k] >= bound if keep_ge else p[k] <= bound

        def intersect(a, b):
            t = (bound - a[k]) / (b[k] - a[k])
            return a + t * (b - a)
        return clip_polygon(poly, inside, intersect)
    for k, b, ge in ((0, x0, True), (0, x1, False), (1, y0, True), (1, y1, False)):
        poly = axis_clip(poly, k, b, ge)
        if not poly:
            return []
    return poly


def shoelace(poly):
    if len(poly) < 3:
        return 0.0
    p = np.array(poly)
    x, y = p[:, 0], p[:, 1]
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(np.roll(x, -1), y))


def clip_convex(subject, clipper):
    """Intersection of two convex 2D polygons (clipper counter-clockwise)."""
    out = [np.asarray(p, float) for p in subject]
    m = len(clipper)
    for i in range(m):
        a, b = np.asarray(clipper[i], float), np.asarray(clipper[(i + 1) % m], float)

        def side(p):
            return (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])

        def inside(p):
            return side(p) >= 0

        def intersect(p, q):
            sp, sq = side(p), side(q)
            return p + (sp / (sp - sq)) * (q - p)
        out = clip_polygon(out, inside, intersect)
        if not out:
            return []
    return out


def ccw(poly):
    p = np.array(poly)
    s = np.dot(p[:, 0], np.roll(p[:, 1], -1)) - np.dot(np.roll(p[:, 0], -1), p[:, 1])
    return list(poly) if s > 0 else list(poly)[::-1]


def segment_in_box(a, b, x0, y0, x1, y1):
    """Liang-Barsky parameter interval [s0,s1] of a+s(b-a) inside the box."""
    d = b - a
    s0, s1 = 0.0, 1.0
    for p, q in ((-d[0], a[0] - x0), (d[0], x1 - a[0]), (-d[1], a[1] - y0), (d[1], y1 - a[1])):
        if p == 0:
            if q < 0:
                return None
            continue
        r = q / p
        if p < 0:
            s0 = max(s0, r)
        else:
            s1 = min(s1, r)
    return (s0, s1) if s0 < s1 else None


def coverage(tri2d, width, height):
    """Area of the triangle inside every unit pixel, [H,W]."""
    tri = [np.asarray(p, float) for p in tri2d]
    A = np.zeros((height, width))
    xs, ys = [p[0] for p in tri], [p[1] for p in tri]
    for j in range(max(0, int(np.floor(min(ys)))), min(height, int(np.ceil(max(ys))) + 1)):
        for i in range(max(0, int(np.floor(min(xs)))), min(width, int(np.ceil(max(xs))) + 1)):
            A[j, i] = shoelace(clip_to_box(tri, i, j, i + 1, j + 1))
    return A


def coverage_gradient(tri2d, weight, width, height):
    """d/d(vertex) of sum_p weight[p] * area(T inside pixel p) by the
    Reynolds transport theorem: for each edge, the integral over the part of
    the edge inside the pixel of (velocity . outward normal)."""
    tri = [np.asarray(p, float) for p in tri2d]
    g = np.zeros((3, 2))
    for e in range(3):
        ia, ib, ic = e, (e + 1) % 3, (e + 2) % 3
        a, b, c = tri[ia], tri[ib], tri[ic]
        d = b - a
        L = np.hypot(d[0], d[1])
        n = np.array([d[1], -d[0]]) / L
        if np.dot(n, c - a) > 0:
            n = -n
        x0, x1 = min(a[0], b[0]), max(a[0], b[0])
        y0, y1 = min(a[1], b[1]), max(a[1], b[1])
        for j in range(max(0, int(np.floor(y0))), min(height, int(np.floor(y1)) + 1)):
            for i in range(max(0, int(np.floor(x0))), min(width, int(np.floor(x1)) + 1)):
                iv = segment_in_box(a, b, i, j, i + 1, j + 1)
                if iv is None:
                    continue
                s0, s1 = iv
                wa = (s1 - s0) - 0.5 * (s1 * s1 - s0 * s0)   # integral of (1-s)
                wb = 0.5 * (s1 * s1 - s0 * s0)               # integral of s
                g[ia] += weight[j, i] * wa * L * n
                g[ib] += weight[j, i] * wb * L * n
    return g


def coverage_gradient_pixels(tri2d, weight, width, height):
    """The terms of coverage_gradient pixel by pixel: [H, W, 3, 2], the
    boundary integral over the part of each edge inside pixel (j, i)."""
    tri = [np.asarray(p, float) for p in tri2d]
    g = np.zeros((height, width, 3, 2))
    for e in range(3):
        ia, ib, ic = e, (e + 1) % 3, (e + 2) % 3
        a, b, c = tri[ia], tri[ib], tri[ic]
        d = b - a
        L = np.hypot(d[0], d[1])
        n = np.array([d[1], -d[0]]) / L
        if np.dot(n, c - a) > 0:
            n = -n
        x0, x1 = min(a[0], b[0]), max(a[0], b[0])
        y0, y1 = min(a[1], b[1]), max(a[1], b[1])
        for j in range(max(0, int(np.floor(y0))), min(height, int(np.floor(y1)) + 1)):
            for i in range(max(0, int(np.floor(x0))), min(width, int(np.floor(x1)) + 1)):
                iv = segment_in_box(a, b, i, j, i + 1, j + 1)
                if iv is None:
                    continue
                s0, s1 = iv
                wa = (s1 - s0) - 0.5 * (s1 * s1 - s0 * s0)
                wb = 0.5 * (s1 * s1 - s0 * s0)
                g[j, i, ia] += weight[j, i] * wa * L * n
                g[j, i, ib] += weight[j, i] * wb * L * n
    return g


def polygon_irradiance(p, normal, poly3d):
    """Lambert's formula: integral over the polygon's solid angle of
    cos(theta) d omega = 1/2 sum_i Theta_i (n . Gamma_i)."""
    n = np.asarray(normal, float)
    u = [np.asarray(v, float) - p for v in poly3d]
    u = [x / np.linalg.norm(x) for x in u]
    s = 0.0
    for i in range(len(u)):
        a, b = u[i], u[(i + 1) % len(u)]
        c = np.cross(a, b)
        cn = np.linalg.norm(c)
        if cn == 0:
            continue
        theta = np.arctan2(cn, np.dot(a, b))
        s += theta * np.dot(n, c / cn)
    return 0.5 * abs(s)
