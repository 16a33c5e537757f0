/*
 * edge_tree.h -- part of the CPU oracle (TEST INFRASTRUCTURE ONLY; included
 * by oracle.cpp inside its anonymous namespace, after Prep).
 *
 * Hierarchical selection of the secondary edge at a shading point (Sec. 5.3.1),
 * written out plainly:
 *
 *  - Two hierarchies in the manner of Olson and Zhang's Hough-space silhouette
 *    search, joined under one root: edges that are silhouettes seen from the
 *    camera position O (or have one face, more than two, or a degenerate face)
 *    are grouped by their 3D position; the others by their 3D position and the
 *    Hough points of their two face planes (6D).  The Hough point of a plane
 *    n.x = n.c with unit n, taken about O, is ((c - O).n) n.
 *  - Construction: the binary radix tree over the sorted Morton codes of the
 *    box centroids (Karras 2012; Lauterbach et al. 2009), with the class as the
 *    top key bit so the root separates the two hierarchies.  The treelet SAH
 *    optimisation of Karras and Aila is not applied.
 *  - Light cone.  At the last vertex (next-event estimation) an edge's term is
 *    nonzero only where a side ray reaches a light, so a box whose cone of
 *    directions from the shading point misses the cone to the lights' bounding
 *    sphere (by more than 1e-3 rad) gets importance zero.  The thesis leaves
 *    incoming radiance to its next-event edge sampler; this bound is exact.
 *  - Node importance: total edge length x inverse distance from the shading
 *    point to the box centre x an upper bound of the clamped cosine over the box
 *    (Walter et al. 2005: the box in the frame of the shading normal; the
 *    linearly transformed cosine of a Lambertian surface is the cosine
 *    itself).  Zero when the node holds no silhouette (the v-sphere test in
 *    Hough space for 6D nodes, the exact test at leaves); both children get
 *    importance one when the shading point lies inside their parent's box.
 *  - Traversal: S samples start at the root and are split between the two
 *    children in proportion to their importance (stochastic rounding keeps the
 *    expected count of every leaf at S times the product of its branch
 *    probabilities); weighted reservoir sampling keeps one of the leaves
 *    reached.
 *
 * Readings where the text is silent:
 *  - Estimator.  The pick is a resampling step: leaf e reached c_e times, with
 *    branch-probability product P_e and importance I_e, has resampling weight
 *    c_e I_e / P_e; the chosen edge is weighted by (sum of those / S) / I_e.
 *    The edge term is then unbiased for any positive importances.
 *  - Silhouette gate.  A non-silhouette edge gives a zero edge term only where
 *    the integrand is visibility alone: at the last vertex (next-event
 *    estimation).  At a vertex that continues the path, flat shading makes
 *    every edge a discontinuity, and no gate applies.
 *  - Horizon.  Side rays leave up to eps |omega| above the edge direction, so
 *    the cosine bound gates a box only below -2 eps, and enters the importance
 *    as max(bound, eps).
 *  - Margins.  The v-sphere test rejects a box only when it clears the sphere by
 *    1e-4 (r + max |Hough coordinate|), so rounding cannot reject a silhouette.
 *
 * Every value that decides the tree's shape, a split or a pick is FP32 in the
 * operation order written here (the file is compiled with -ffp-contract=off).
 */

constexpr uint32_t K_EDGE_TREE = 5;  /* Philox stream kind of the tree's random numbers */

struct ETLeaf {
  float v0[3], v1[3], c0[3], c1[3];
  float len;
  int eid;
  bool boundary;  /* no two faces to compare: always a potential silhouette */
  bool classB;    /* not a silhouette seen from O: in the 6D hierarchy */
  float h0[3], h1[3];
};

struct ETSlot {  /* a child as its parent sees it */
  float lo[3], hi[3], hlo[3], hhi[3];
  float L;
  bool allB;
};

struct ETNode {
  int child[2];  /* >= 0: node index; < 0: ~(leaf position) */
  ETSlot slot[2];
};

struct EdgeTree {
  std::vector<ETLeaf> leaf;  /* in key order */
  std::vector<ETNode> node;
  int root = -1;             /* node index, or ~0 when there is a single edge */
  float O[3];
  bool has_light = false;    /* sphere around all light triangles (padded) */
  float lc[3], lr;
};

/* Sphere around a box: centre and padded half diagonal (FP32, fixed order). */
void et_sphere(const float lo[3], const float hi[3], float c[3], float* r) {
  float d[3];
  for (int i = 0; i < 3; ++i) { c[i] = (lo[i] + hi[i]) * 0.5f; d[i] = hi[i] - lo[i]; }
  *r = (0.5f * std::sqrt(dot32(d, d))) * 1.0001f + 1e-6f;
}

float et_min(float a, float b) { return b < a ? b : a; }
float et_max(float a, float b) { return b > a ? b : a; }

uint32_t et_quant(float x, float lo, float ext, uint32_t levels) {
  if (!(ext > 0.0f)) return 0;
  float f = ((x - lo) / ext) * (float)levels;
  if (!(f > 0.0f)) return 0;
  if (f >= (float)(levels - 1)) return levels - 1;
  return (uint32_t)f;
}

/* Unit normal of the plane through a, b, c (as cross(b - a, c - a)); false if
 * degenerate. */
bool et_unit_normal(const float* a, const float* b, const float* c, float n[3]) {
  float e1[3], e2[3];
  for (int i = 0; i < 3; ++i) { e1[i] = b[i] - a[i]; e2[i] = c[i] - a[i]; }
  float m[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  float l = std::sqrt(dot32(m, m));
  if (!(l > 0.0f)) return false;
  for (int i = 0; i < 3; ++i) n[i] = m[i] / l;
  return true;
}

void build_edge_tree(const Prep& P, EdgeTree& T) {
  const or_scene_t& sc = *P.sc;
  int E = (int)P.e0.size();
  for (int i = 0; i < 3; ++i) T.O[i] = sc.cam_to_world[4 * i + 3];
  T.has_light = sc.n_light_tris > 0;
  if (T.has_light) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int j = 0; j < sc.n_light_tris; ++j)
      for (int k = 0; k < 3; ++k) {
        const float* v = vtx(P, sc.tris[3 * sc.light_tris[j] + k]);
        for (int i = 0; i < 3; ++i) { lo[i] = et_min(lo[i], v[i]); hi[i] = et_max(hi[i], v[i]); }
      }
    et_sphere(lo, hi, T.lc, &T.lr);
  }
  /* faces of every edge, in increasing triangle order */
  std::vector<std::vector<int>> faces(E);
  for (int t = 0; t < P.T; ++t)
    for (int k = 0; k < 3; ++k) {
      int a = sc.tris[3 * t + k], b = sc.tris[3 * t + (k + 1) % 3];
      int lo = std::min(a, b), hi = std::max(a, b);
      /* edges are sorted by (lo, hi): binary search */
      int l = 0, h = E;
      while (l < h) {
        int m = (l + h) / 2;
        if (P.e0[m] < lo || (P.e0[m] == lo && P.e1[m] < hi)) l = m + 1; else h = m;
      }
      faces[l].push_back(t);
    }
  /* scene box and the Hough radius about O */
  float blo[3], bhi[3];
  for (int i = 0; i < 3; ++i) { blo[i] = sc.verts[i]; bhi[i] = sc.verts[i]; }
  for (int v = 1; v < P.V; ++v)
    for (int i = 0; i < 3; ++i) { blo[i] = et_min(blo[i], sc.verts[3 * v + i]); bhi[i] = et_max(bhi[i], sc.verts[3 * v + i]); }
  float R2 = 0.0f;
  {
    float q[3];
    for (int i = 0; i < 3; ++i) {
      float a = blo[i] - T.O[i], b = bhi[i] - T.O[i];
      q[i] = et_max(a * a, b * b);
    }
    R2 = (q[0] + q[1]) + q[2];
  }
  float R = std::sqrt(R2);
  std::vector<ETLeaf> lv(E);
  std::vector<std::pair<uint32_t, int>> keys(E);
  for (int e = 0; e < E; ++e) {
    ETLeaf& L = lv[e];
    const float *a = vtx(P, P.e0[e]), *b = vtx(P, P.e1[e]);
    for (int i = 0; i < 3; ++i) { L.v0[i] = a[i]; L.v1[i] = b[i]; L.c0[i] = 0.0f; L.c1[i] = 0.0f; L.h0[i] = 0.0f; L.h1[i] = 0.0f; }
    float d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    L.len = std::sqrt(dot32(d, d));
    L.eid = e;
    L.boundary = faces[e].size() != 2;
    L.classB = false;
    if (!L.boundary) {
      for (int f = 0; f < 2; ++f) {
        int t = faces[e][f];
        int third = sc.tris[3 * t];
        for (int k = 0; k < 3; ++k) {
          int v = sc.tris[3 * t + k];
          if (v != P.e0[e] && v != P.e1[e]) third = v;
        }
        const float* c = vtx(P, third);
        for (int i = 0; i < 3; ++i) (f == 0 ? L.c0 : L.c1)[i] = c[i];
      }
      /* face planes oriented consistently across the edge: (v0, v1, c0) and (v1, v0, c1) */
      float n0[3], n1[3];
      if (et_unit_normal(L.v0, L.v1, L.c0, n0) && et_unit_normal(L.v1, L.v0, L.c1, n1)) {
        float r0[3] = {L.v0[0] - T.O[0], L.v0[1] - T.O[1], L.v0[2] - T.O[2]};
        float t0 = dot32(n0, r0), t1 = dot32(n1, r0);
        for (int i = 0; i < 3; ++i) { L.h0[i] = t0 * n0[i]; L.h1[i] = t1 * n1[i]; }
        L.classB = (t0 > 0.0f && t1 > 0.0f) || (t0 < 0.0f && t1 < 0.0f);
      }
    }
    /* Morton code of the box centroid: 3D (10 bits per axis) or 6D (5 bits) */
    float mid[3];
    for (int i = 0; i < 3; ++i) mid[i] = (L.v0[i] + L.v1[i]) * 0.5f;
    uint32_t code = 0;
    if (!L.classB) {
      uint32_t q[3];
      for (int i = 0; i < 3; ++i) q[i] = et_quant(mid[i], blo[i], bhi[i] - blo[i], 1024u);
      for (int bit = 9; bit >= 0; --bit)
        for (int i = 0; i < 3; ++i) code = (code << 1) | ((q[i] >> bit) & 1u);
    } else {
      uint32_t q[6];
      for (int i = 0; i < 3; ++i) q[i] = et_quant(mid[i], blo[i], bhi[i] - blo[i], 32u);
      for (int i = 0; i < 3; ++i) {
        float hc = (L.h0[i] + L.h1[i]) * 0.5f;
        q[3 + i] = et_quant(hc, -R, R + R, 32u);
      }
      for (int bit = 4; bit >= 0; --bit)
        for (int i = 0; i < 6; ++i) code = (code << 1) | ((q[i] >> bit) & 1u);
    }
    keys[e] = {((L.classB ? 1u : 0u) << 30) | code, e};
  }
  std::stable_sort(keys.begin(), keys.end(),
                   [](const std::pair<uint32_t, int>& x, const std::pair<uint32_t, int>& y) { return x.first < y.first; });
  T.leaf.resize(E);
  for (int i = 0; i < E; ++i) T.leaf[i] = lv[keys[i].second];
  T.node.clear();
  if (E == 0) { T.root = -1; return; }
  if (E == 1) { T.root = ~0; return; }
  /* binary radix tree over (key, position): a range splits where the highest
   * bit in which its first and last augmented keys differ changes */
  auto aug = [&](int i) { return ((uint64_t)keys[i].first << 32) | (uint32_t)i; };
  auto clz64 = [](uint64_t x) { int n = 0; while (n < 64 && !(x & (1ull << (63 - n)))) ++n; return n; };
  std::function<ETSlot(int, int, int*)> build = [&](int lo, int hi, int* enc) -> ETSlot {
    ETSlot s;
    if (lo == hi) {
      const ETLeaf& L = T.leaf[lo];
      for (int i = 0; i < 3; ++i) {
        s.lo[i] = et_min(L.v0[i], L.v1[i]);
        s.hi[i] = et_max(L.v0[i], L.v1[i]);
        s.hlo[i] = L.classB ? et_min(L.h0[i], L.h1[i]) : INFINITY;
        s.hhi[i] = L.classB ? et_max(L.h0[i], L.h1[i]) : -INFINITY;
      }
      s.L = L.len;
      s.allB = L.classB;
      *enc = ~lo;
      return s;
    }
    int common = clz64(aug(lo) ^ aug(hi));
    int split = lo;
    for (int i = lo; i < hi; ++i)
      if (clz64(aug(lo) ^ aug(i)) > common) split = i;
    int id = (int)T.node.size();
    T.node.push_back(ETNode());
    int cl, cr;
    ETSlot a = build(lo, split, &cl);
    ETSlot b = build(split + 1, hi, &cr);
    ETNode& N = T.node[id];
    N.child[0] = cl; N.child[1] = cr;
    N.slot[0] = a; N.slot[1] = b;
    for (int i = 0; i < 3; ++i) {
      s.lo[i] = et_min(a.lo[i], b.lo[i]);
      s.hi[i] = et_max(a.hi[i], b.hi[i]);
      s.hlo[i] = et_min(a.hlo[i], b.hlo[i]);
      s.hhi[i] = et_max(a.hhi[i], b.hhi[i]);
    }
    s.L = a.L + b.L;
    s.allB = a.allB && b.allB;
    *enc = id;
    return s;
  };
  int root;
  build(0, E - 1, &root);
  T.root = root;
}

/* Shading point of one query: position, normal and the normal's frame. */
struct ETQuery {
  float p[3], n[3], t[3], u[3];
  float C[3], r;  /* v-sphere about O: centre (p - O)/2, radius |p - O|/2 */
  bool last;
  float eps;
};

/* Orthonormal frame of a unit normal (Duff et al., JCGT 2017). */
void et_frame(const float n[3], float t[3], float u[3]) {
  float sg = n[2] >= 0.0f ? 1.0f : -1.0f;
  float a = -1.0f / (sg + n[2]);
  float b = (n[0] * n[1]) * a;
  t[0] = 1.0f + (sg * (n[0] * n[0])) * a;
  t[1] = sg * b;
  t[2] = -(sg * n[0]);
  u[0] = b;
  u[1] = sg + (n[1] * n[1]) * a;
  u[2] = -n[1];
}

/* Upper bound of cos(n, x - p) over the box (Walter et al. 2005): the box's
 * bounds in the frame (t, u, n) about p. */
float et_cos_bound(const ETQuery& q, const float lo[3], const float hi[3]) {
  float c[3], h[3];
  for (int i = 0; i < 3; ++i) { c[i] = (lo[i] + hi[i]) * 0.5f - q.p[i]; h[i] = (hi[i] - lo[i]) * 0.5f; }
  float an[3] = {std::fabs(q.n[0]), std::fabs(q.n[1]), std::fabs(q.n[2])};
  float at[3] = {std::fabs(q.t[0]), std::fabs(q.t[1]), std::fabs(q.t[2])};
  float au[3] = {std::fabs(q.u[0]), std::fabs(q.u[1]), std::fabs(q.u[2])};
  float cz = dot32(q.n, c), ez = dot32(an, h);
  float cx = dot32(q.t, c), ex = dot32(at, h);
  float cy = dot32(q.u, c), ey = dot32(au, h);
  float zmax = cz + ez;
  float mx, my;
  if (zmax > 0.0f) {
    mx = et_max(std::fabs(cx) - ex, 0.0f);
    my = et_max(std::fabs(cy) - ey, 0.0f);
  } else {
    mx = std::fabs(cx) + ex;
    my = std::fabs(cy) + ey;
  }
  float den = std::sqrt((mx * mx + my * my) + zmax * zmax);
  if (!(den > 0.0f)) return 0.0f;
  return zmax / den;
}

/* True if the v-sphere clears the Hough box: then either every face plane
 * of the node separates O from p or none does, and no edge of the node is a
 * silhouette seen from p. */
bool et_vsphere_clears(const ETQuery& q, const ETSlot& s) {
  float dmin2 = 0.0f, dmax2 = 0.0f, hm = 0.0f;
  for (int i = 0; i < 3; ++i) {
    float a = s.hlo[i] - q.C[i], b = q.C[i] - s.hhi[i];
    float o = et_max(et_max(a, b), 0.0f);
    dmin2 = dmin2 + o * o;
    float fa_ = q.C[i] - s.hlo[i], fb = s.hhi[i] - q.C[i];
    dmax2 = dmax2 + et_max(fa_ * fa_, fb * fb);
    hm = et_max(hm, et_max(std::fabs(s.hlo[i]), std::fabs(s.hhi[i])));
  }
  float g = 1e-4f * (q.r + hm);
  float ri = q.r - g, ro = q.r + g;
  bool inside = ri > 0.0f && dmax2 < ri * ri;
  bool outside = dmin2 > ro * ro;
  return inside || outside;
}

/* Exact silhouette test of a leaf seen from p: false only when the two faces
 * lie strictly on opposite sides of the plane through p and the edge. */
bool et_silhouette(const ETQuery& q, const ETLeaf& L) {
  if (L.boundary) return true;
  float a0[3], a1[3], d0[3], d1[3];
  for (int i = 0; i < 3; ++i) {
    a0[i] = L.v0[i] - q.p[i]; a1[i] = L.v1[i] - q.p[i];
    d0[i] = L.c0[i] - q.p[i]; d1[i] = L.c1[i] - q.p[i];
  }
  float m[3] = {a0[1] * a1[2] - a0[2] * a1[1], a0[2] * a1[0] - a0[0] * a1[2], a0[0] * a1[1] - a0[1] * a1[0]};
  float s0 = dot32(m, d0), s1 = dot32(m, d1);
  return !((s0 > 0.0f && s1 < 0.0f) || (s0 < 0.0f && s1 > 0.0f));
}

/* At the last vertex only radiance that arrives from a light counts.  True
 * if the cone of directions from p to the box's sphere and the cone to the
 * lights' sphere are apart by more than 1e-3 rad (side rays leave an edge
 * point by about eps): then no edge of the box has a nonzero term. */
bool et_light_cone_clears(const EdgeTree& T, const ETQuery& q, const float lo[3], const float hi[3]) {
  float cb[3], rb, vb[3], vl[3];
  et_sphere(lo, hi, cb, &rb);
  for (int i = 0; i < 3; ++i) { vb[i] = cb[i] - q.p[i]; vl[i] = T.lc[i] - q.p[i]; }
  float db = std::sqrt(dot32(vb, vb)), dl = std::sqrt(dot32(vl, vl));
  if (!(db > rb) || !(dl > T.lr)) return false;
  float sb = rb / db, sl = T.lr / dl;
  float kb = std::sqrt(1.0f - sb * sb), kl = std::sqrt(1.0f - sl * sl);
  float cosA = kb * kl - sb * sl, sinA = sb * kl + kb * sl;  /* A = sum of the half-angles */
  float cosAm = cosA * 0.9999995f - sinA * 1e-3f, sinAm = sinA * 0.9999995f + cosA * 1e-3f;
  if (!(sinAm > 0.0f)) return false;
  float cg = dot32(vb, vl) / (db * dl);
  return cg < cosAm;
}

/* Importance of a child (slot s; leaf position `leaf` if a leaf, else -1)
 * of a parent with box [plo, phi]. */
float et_importance(const EdgeTree& T, const ETQuery& q, const ETSlot& s, int leaf, const float plo[3],
                    const float phi[3]) {
  if (q.last && T.has_light && et_light_cone_clears(T, q, s.lo, s.hi)) return 0.0f;
  if (q.last) {
    if (leaf >= 0) {
      if (!et_silhouette(q, T.leaf[leaf])) return 0.0f;
    } else if (s.allB && et_vsphere_clears(q, s)) {
      return 0.0f;
    }
  }
  float cb = et_cos_bound(q, s.lo, s.hi);
  if (cb <= -2.0f * q.eps) return 0.0f;
  bool inside = true;
  for (int i = 0; i < 3; ++i) inside = inside && plo[i] <= q.p[i] && q.p[i] <= phi[i];
  if (inside) return 1.0f;
  float c[3];
  for (int i = 0; i < 3; ++i) c[i] = (s.lo[i] + s.hi[i]) * 0.5f - q.p[i];
  float d = std::sqrt(dot32(c, c));
  return (s.L * et_max(cb, q.eps)) / et_max(d, 1e-30f);
}

ETQuery et_query(const EdgeTree& T, const float p[3], const float n[3], bool last, float eps) {
  ETQuery q;
  for (int i = 0; i < 3; ++i) { q.p[i] = p[i]; q.n[i] = n[i]; }
  et_frame(q.n, q.t, q.u);
  for (int i = 0; i < 3; ++i) q.C[i] = (p[i] - T.O[i]) * 0.5f;
  q.r = std::sqrt(dot32(q.C, q.C));
  q.last = last;
  q.eps = eps;
  return q;
}

/* Pick one secondary edge at the shading point with S root samples.  Random
 * numbers: one Philox block per popped item, counter (c0, c1, kind 5,
 * bounce, item ordinal, scene).  Out: edge id and the weight that replaces
 * 1/P(edge) of the length sampler.  False: no edge can contribute. */
bool et_pick(const EdgeTree& T, const ETQuery& q, int S, uint64_t seed, uint32_t c0, uint32_t c1, uint32_t bounce,
             uint32_t scene, int* eid, float* weight) {
  if (T.root == -1 || S <= 0) return false;
  struct Item { int enc, n; float P, I; };
  std::vector<Item> stack;
  if (T.root < 0) {
    /* a single edge: no parent box */
    float none_lo[3] = {INFINITY, INFINITY, INFINITY}, none_hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    const ETLeaf& L = T.leaf[0];
    ETSlot s;
    for (int i = 0; i < 3; ++i) { s.lo[i] = et_min(L.v0[i], L.v1[i]); s.hi[i] = et_max(L.v0[i], L.v1[i]); }
    s.L = L.len;
    s.allB = L.classB;
    float I = et_importance(T, q, s, 0, none_lo, none_hi);
    if (!(I > 0.0f)) return false;
    stack.push_back({~0, S, 1.0f, I});
  } else {
    stack.push_back({T.root, S, 1.0f, 0.0f});
  }
  float tot = 0.0f, chosen_I = 0.0f;
  int chosen = -1;
  uint32_t j = 0;
  while (!stack.empty()) {
    Item it = stack.back();
    stack.pop_back();
    uint32_t r[4];
    rng(seed, c0, c1, K_EDGE_TREE, bounce, j, scene, r);
    ++j;
    float u = u01f(r[0]);
    if (it.enc < 0) {
      if (!(it.P > 0.0f)) continue;
      float w = (float)it.n * (it.I / it.P);
      tot = tot + w;
      if (u * tot < w) { chosen = ~it.enc; chosen_I = it.I; }
      continue;
    }
    const ETNode& N = T.node[it.enc];
    float plo[3], phi[3];
    for (int i = 0; i < 3; ++i) {
      plo[i] = et_min(N.slot[0].lo[i], N.slot[1].lo[i]);
      phi[i] = et_max(N.slot[0].hi[i], N.slot[1].hi[i]);
    }
    float I0 = et_importance(T, q, N.slot[0], N.child[0] < 0 ? ~N.child[0] : -1, plo, phi);
    float I1 = et_importance(T, q, N.slot[1], N.child[1] < 0 ? ~N.child[1] : -1, plo, phi);
    float sum = I0 + I1;
    if (!(sum > 0.0f)) continue;
    float p0 = I0 / sum, p1 = I1 / sum;
    int n0;
    if (!(I0 > 0.0f)) {
      n0 = 0;
    } else if (!(I1 > 0.0f)) {
      n0 = it.n;
    } else {
      float x = (float)it.n * p0;
      float fl = std::floor(x);
      n0 = (int)fl + (u < x - fl ? 1 : 0);
      n0 = std::min(std::max(n0, 0), it.n);
    }
    int n1 = it.n - n0;
    if (n1 > 0) stack.push_back({N.child[1], n1, it.P * p1, I1});
    if (n0 > 0) stack.push_back({N.child[0], n0, it.P * p0, I0});
  }
  if (chosen < 0) return false;
  *eid = T.leaf[chosen].eid;
  *weight = (tot / (float)S) / chosen_I;
  return true;
}
