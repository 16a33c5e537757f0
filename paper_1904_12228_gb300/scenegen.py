"""Seeded synthetic scene generators.

These build the inputs that both the CUDA path and the CPU oracle consume:
triangle meshes, per-triangle albedo, area lights, cameras and loss adjoints.
They hold none of the rendering method's arithmetic (no projection, edge
extraction, shading or sampling); they only place geometry, the way the
thesis's scenes are built from lists of tensors (Sec. 5.4).

Every generator is deterministic in its ``seed``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

CAM_ORTHO = 0
CAM_PINHOLE = 1
CAM_FISHEYE = 2


@dataclasses.dataclass
class Scene:
    """A triangle-mesh scene in host memory (float32 / int32, C order).

    verts [V,3]; tris [T,3] (counter-clockwise seen from the front);
    albedo [T,3]; light_tris [L] indices of emitting triangles (front face
    only); radiance [3]; cam_to_world [4,4] row-major (camera looks down -z,
    y up); cam_scale = tan(fov_y/2) for a pinhole camera or the half height
    of the view for an orthographic one; image width x height.
    """

    verts: np.ndarray
    tris: np.ndarray
    albedo: np.ndarray
    light_tris: np.ndarray
    radiance: np.ndarray
    cam_to_world: np.ndarray
    cam_scale: float
    cam_type: int
    width: int
    height: int

    def __post_init__(self):
        self.verts = np.ascontiguousarray(self.verts, dtype=np.float32).reshape(-1, 3)
        self.tris = np.ascontiguousarray(self.tris, dtype=np.int32).reshape(-1, 3)
        self.albedo = np.ascontiguousarray(self.albedo, dtype=np.float32).reshape(-1, 3)
        self.light_tris = np.ascontiguousarray(self.light_tris, dtype=np.int32).reshape(-1)
        self.radiance = np.ascontiguousarray(self.radiance, dtype=np.float32).reshape(3)
        self.cam_to_world = np.ascontiguousarray(self.cam_to_world, dtype=np.float32).reshape(4, 4)
        self.cam_scale = float(np.float32(self.cam_scale))

    @property
    def n_params(self) -> int:
        return 3 * len(self.verts) + 3 * len(self.tris) + 3 + 13

    def copy(self) -> "Scene":
        return dataclasses.replace(self, verts=self.verts.copy(), tris=self.tris.copy(),
                                   albedo=self.albedo.copy(), light_tris=self.light_tris.copy(),
                                   radiance=self.radiance.copy(), cam_to_world=self.cam_to_world.copy())


def look_at(eye, target, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """Camera-to-world matrix whose -z axis points from eye to target."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    x = np.cross(f, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(x, f)
    m = np.eye(4)
    m[:3, 0], m[:3, 1], m[:3, 2], m[:3, 3] = x, y, -f, eye
    return m.astype(np.float32)


def icosphere(subdiv: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit icosphere by midpoint subdivision (20 * 4**subdiv faces)."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
             (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5),
             (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache: dict[tuple[int, int], int] = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts), np.array(faces, np.int64)


def quad(center, ex, ey) -> tuple[np.ndarray, np.ndarray]:
    """Two triangles spanning center +- ex +- ey; front normal = ex x ey."""
    c, ex, ey = (np.asarray(a, np.float64) for a in (center, ex, ey))
    v = np.array([c - ex - ey, c + ex - ey, c + ex + ey, c - ex + ey])
    return v, np.array([[0, 1, 2], [0, 2, 3]], np.int64)


def _merge(parts):
    verts, tris, off = [], [], 0
    for v, f in parts:
        verts.append(v)
        tris.append(f + off)
        off += len(v)
    return np.concatenate(verts), np.concatenate(tris)


def single_triangle(seed: int, width: int = 64, height: int = 64, color: float = 0.7) -> Scene:
    """One triangle with vertices uniform in [-1,1]^2 (z=0) under an
    orthographic camera at z=1 spanning [-1,1]^2; constant color over black."""
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-1.0, 1.0, size=(3, 2))
    verts = np.concatenate([xy, np.zeros((3, 1))], axis=1)
    cam = np.eye(4, dtype=np.float32)
    cam[2, 3] = 1.0
    return Scene(verts=verts, tris=[[0, 1, 2]], albedo=[[color] * 3], light_tris=np.zeros(0, np.int32),
                 radiance=[0, 0, 0], cam_to_world=cam, cam_scale=1.0, cam_type=CAM_ORTHO, width=width,
                 height=height)


def direct_lighting(seed: int, width: int = 256, height: int = 256, subdiv: int = 4,
                    jitter: float = 0.01, light_half: float = 0.5) -> Scene:
    """Jittered icosphere (radius 1) on a 2-triangle ground at y=-1 spanning
    [-4,4]^2, lit by a two-triangle square area light of half size
    light_half (default 0.5: 1x1) at y=3 facing down with radiance
    10 (0.5 / light_half)^2 (the same power for any size); per-triangle albedo
    uniform in [0.2,0.8]^3; pinhole camera at (0,1,5) looking at the origin,
    45 degree vertical field of view."""
    rng = np.random.default_rng(seed)
    sv, sf = icosphere(subdiv)
    sv = sv + rng.normal(0.0, jitter, size=sv.shape)
    gv, gf = quad((0, -1, 0), (0, 0, 4), (4, 0, 0))
    lv, lf = quad((0, 3, 0), (light_half, 0, 0), (0, 0, light_half))
    verts, tris = _merge([(sv, sf), (gv, gf), (lv, lf)])
    n = len(tris)
    albedo = rng.uniform(0.2, 0.8, size=(n, 3))
    light_tris = np.array([n - 2, n - 1], np.int32)
    le = 10.0 * (0.5 / light_half) ** 2
    return Scene(verts=verts, tris=tris, albedo=albedo, light_tris=light_tris, radiance=[le, le, le],
                 cam_to_world=look_at((0, 1, 5), (0, 0, 0)), cam_scale=math.tan(math.radians(22.5)),
                 cam_type=CAM_PINHOLE, width=width, height=height)


def loss_adjoint(seed: int, width: int, height: int) -> np.ndarray:
    """d loss / d image, uniform in [-1,1] per pixel and channel, [H,W,3]."""
    rng = np.random.default_rng(seed + 7919)
    return rng.uniform(-1.0, 1.0, size=(height, width, 3)).astype(np.float32)


def displaced_icosphere(rng, subdiv: int = 3, amp: float = 0.1, waves: int = 6):
    """Unit icosphere with a smooth seeded radial displacement of amplitude
    ``amp``: a sum of random cosine waves over the sphere, scaled to amp."""
    v, f = icosphere(subdiv)
    dirs = rng.normal(size=(waves, 3))
    freq = rng.uniform(1.0, 4.0, size=waves)
    phase = rng.uniform(0, 2 * np.pi, size=waves)
    d = np.cos((v @ dirs.T) * freq + phase).sum(axis=1)
    d = amp * d / max(1e-9, np.abs(d).max())
    return v * (1.0 + d)[:, None], f


def subdivided_box(n: int = 4):
    """Axis-aligned cube [-1,1]^3 with each face split into n x n quads
    (12 n^2 triangles; 192 for n = 4), faces wound outward."""
    verts, tris = [], []
    g = np.linspace(-1.0, 1.0, n + 1)
    for axis in range(3):
        for sign in (-1.0, 1.0):
            u, w = [a for a in range(3) if a != axis]
            base = len(verts)
            for i in range(n + 1):
                for j in range(n + 1):
                    p = np.zeros(3)
                    p[axis], p[u], p[w] = sign, g[i], g[j]
                    verts.append(p)
            for i in range(n):
                for j in range(n):
                    a, b = base + i * (n + 1) + j, base + (i + 1) * (n + 1) + j
                    c, d = b + 1, a + 1
                    tri = [[a, b, c], [a, c, d]]
                    if (sign > 0) != ((u, w) in ((1, 2), (2, 0), (0, 1))):
                        tri = [[a, c, b], [a, d, c]]
                    tris += tri
    return np.array(verts), np.array(tris, np.int64)


def procedural(seed: int, n_target: int = 200_000, width: int = 512, height: int = 512) -> Scene:
    """Displaced icospheres (1280 triangles each, radial noise amplitude 0.1)
    and subdivided boxes (192 triangles each), placed in [-5,5]^3 without
    overlap (rejection on bounding spheres) until the triangle count reaches
    n_target; a ground quad below and two area lights above (radiance 30);
    per-triangle albedo uniform in [0.2,0.8]^3; pinhole camera at (0,2,16)
    looking at (0,-0.5,0), 45 degree field of view."""
    rng = np.random.default_rng(seed)
    parts, centers, radii = [], [], []
    count = 6
    tries = 0
    while count < n_target and tries < 200000:
        tries += 1
        is_sphere = rng.uniform() < 0.5
        if is_sphere:
            r = rng.uniform(0.3, 0.6)
            bound = r * 1.1
        else:
            r = rng.uniform(0.25, 0.5)
            bound = r * np.sqrt(3.0)
        c = rng.uniform(-5.0 + bound, 5.0 - bound, size=3)
        if centers and np.any(np.linalg.norm(np.array(centers) - c, axis=1) < np.array(radii) + bound + 0.02):
            continue
        if is_sphere:
            v, f = displaced_icosphere(rng)
        else:
            v, f = subdivided_box()
        parts.append((v * r + c, f))
        centers.append(c)
        radii.append(bound)
        count += len(f)
    parts.append(quad((0, -5.5, 0), (0, 0, 8), (8, 0, 0)))
    l1 = quad((-2, 6, -2), (0.75, 0, 0), (0, 0, 0.75))
    l2 = quad((2, 6, 2), (0.75, 0, 0), (0, 0, 0.75))
    parts += [l1, l2]
    verts, tris = _merge(parts)
    n = len(tris)
    albedo = rng.uniform(0.2, 0.8, size=(n, 3))
    return Scene(verts=verts, tris=tris, albedo=albedo, light_tris=np.arange(n - 4, n, dtype=np.int32),
                 radiance=[30.0, 30.0, 30.0], cam_to_world=look_at((0, 2, 16), (0, -0.5, 0)),
                 cam_scale=math.tan(math.radians(22.5)), cam_type=CAM_PINHOLE, width=width, height=height)


def batch_workload(seed: int, n: int = 64, t_min: int = 1000, t_max: int = 100_000,
                   resolutions=(128, 256, 512)) -> list:
    """n procedural scenes (the generator above, direct lighting when
    rendered at depth 1): triangle count log-uniform in [t_min, t_max],
    square resolution drawn uniformly from `resolutions`."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        t = int(round(math.exp(rng.uniform(math.log(t_min), math.log(t_max)))))
        res = int(rng.choice(np.asarray(resolutions)))
        out.append(procedural(seed * 1000 + k, n_target=t, width=res, height=res))
    return out


def perturb_vertices(scene: Scene, seed: int, sigma: float = 0.02) -> np.ndarray:
    """Vertex positions + N(0, sigma) (the inverse-rendering start point)."""
    rng = np.random.default_rng(seed + 104729)
    return (scene.verts + rng.normal(0.0, sigma, size=scene.verts.shape)).astype(np.float32)


def indirect_panel(view: str = "interior", width: int = 12, height: int = 12) -> Scene:
    """A small scene for checking paths of two and three scattering vertices.

    A floor (albedo 0.9) and a side wall are lit by a small area light above;
    a panel hangs between the light and the floor, and a dark blocker
    triangle (albedo 0.05) sits between panel and floor.  An orthographic
    camera below the panel looks straight up at its underside, which the light
    cannot reach directly: every pixel is lit through the floor and the wall
    (two vertices) or through longer paths (three vertices: panel, floor,
    wall).  view="interior": the window shows the panel's underside only, no
    edge is in view, and the blocker acts through indirect shadows alone.
    view="silhouette": the window is centred under the blocker, whose
    silhouette against the panel is in view.  Both windows keep a margin of
    at least 0.05 to the panel's edges and the blocker's corners, so a small
    change of the window size brings no new edge into view."""
    floor = quad((0, 0, 0), (2, 0, 0), (0, 0, -2))
    panel = quad((0, 1.0, 0), (0.7, 0, 0), (0, 0, 0.7))
    light = quad((0, 2.0, 0), (0.3, 0, 0), (0, 0, 0.3))
    blocker = (np.array([[-0.5, 0.55, -0.3], [0.45, 0.5, 0.05], [-0.15, 0.6, 0.5]]), np.array([[0, 1, 2]]))
    wall = quad((-1.2, 0.75, 0), (0, 0.75, 0), (0, 0, 1.0))
    verts, tris = _merge([floor, panel, light, blocker, wall])
    alb = np.full((len(tris), 3), 0.9)
    alb[6] = 0.05
    if view == "interior":
        centre, half = (0.3, -0.35), 0.2
    elif view == "silhouette":
        centre, half = (-0.02, 0.1), 0.55
    else:
        raise ValueError("view must be 'interior' or 'silhouette'")
    cam = look_at((centre[0], 0.05, centre[1]), (centre[0], 1.0, centre[1]), up=(0, 0, -1))
    return Scene(verts=verts, tris=tris, albedo=alb, light_tris=[4, 5], radiance=[40, 40, 40], cam_to_world=cam,
                 cam_scale=half, cam_type=CAM_ORTHO, width=width, height=height)


def fisheye_view(seed: int, width: int = 64, height: int = 48, subdiv: int = 2, theta_half_height: float = 1.1
                 ) -> Scene:
    """The direct-lighting scene (jittered icosphere on a ground quad under an
    area light) seen through an equidistant fisheye from close by: the screen
    point at distance r from the centre, in units of half the image height,
    looks along the direction theta = r * theta_half_height from the optical
    axis (every pixel, corners included, sees a direction below pi)."""
    sc = direct_lighting(seed, width=width, height=height, subdiv=subdiv)
    return dataclasses.replace(sc, cam_to_world=look_at((0.4, 1.2, 2.6), (0.0, -0.2, 0.0)),
                               cam_scale=float(theta_half_height), cam_type=CAM_FISHEYE)


def gi_panel(width: int = 16, height: int = 16) -> Scene:
    """A scene lit mostly indirectly: a floor (albedo 0.85) lit by a small
    area light, a panel above the floor whose underside the camera sees (it
    receives light only by reflection from the floor), and a small dark
    blocker between floor and panel that casts an indirect shadow on the
    panel and a direct shadow on the floor."""
    floor = quad((0, 0, 0), (2, 0, 0), (0, 0, -2))
    panel = quad((0, 1.0, 0), (0.6, 0, 0), (0, 0, 0.6))
    light = quad((0, 2.0, 0), (0.3, 0, 0), (0, 0, 0.3))
    blocker = (np.array([[-0.3, 0.5, -0.2], [0.35, 0.5, 0.1], [-0.1, 0.5, 0.4]]), np.array([[0, 1, 2]]))
    verts, tris = _merge([floor, panel, light, blocker])
    alb = np.full((len(tris), 3), 0.85)
    alb[-1] = 0.3
    return Scene(verts=verts, tris=tris, albedo=alb, light_tris=[4, 5], radiance=[20, 20, 20],
                 cam_to_world=look_at((0.2, 0.25, 2.6), (0, 1.0, 0)), cam_scale=math.tan(math.radians(25)),
                 cam_type=CAM_PINHOLE, width=width, height=height)
