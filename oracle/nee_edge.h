/*
 * nee_edge.h -- next-event estimation for edges (Sec. 5.3.3), part of the CPU
 * oracle.  TEST INFRASTRUCTURE ONLY (see oracle.cpp); included by oracle.cpp
 * after edge_tree.h, whose leaves supply each edge's end points, the third
 * vertices of its faces and its length.
 *
 * The thesis reuses the shadow ray of next-event estimation at a shading
 * point p: every edge becomes a billboard of width w that faces the ray, the
 * billboards the ray crosses are collected, one of them is picked by its
 * importance, and the crossing point, projected onto the edge, is the edge
 * sample.  It gives no density for that sample.  The readings here:
 *
 *  - Billboard facing the ray.  It contains the edge's line and its normal is
 *    the part of the ray direction perpendicular to the edge.  The ray meets
 *    it at the ray's point closest to the edge's line, at distance |u| from
 *    that line, and the projection onto the edge is the line's closest point,
 *    at parameter t.  So the ray crosses the billboard exactly when the two
 *    lines pass within w/2 of each other with t in [0, 1] and the closest
 *    point of the ray between p and the light point, 0 < s < T (T: the
 *    light hit, in units of the ray direction d = y - p).
 *  - Width: w is the L2 norm over the three coordinates of 2 % of the mean
 *    absolute deviation of the vertex positions (the whole width; the
 *    crossing test uses w/2).
 *  - Importance of a crossed edge: length / distance from p to the crossing's
 *    point on the edge, zero unless the edge is a silhouette seen from p and
 *    that point lies above p's tangent plane and farther from p than the
 *    width w (the factors of Sec. 5.3.1 that differ between billboards along
 *    one ray).  The pick is an exponential race: each crossed edge draws a key
 *    -ln(U_e) / importance_e and the smallest key wins (ties to the lower
 *    edge id), which picks e with probability importance_e / sum over the
 *    crossed edges, whatever order the edges are visited in.  U_e comes from
 *    Philox4x32-10 with counter (edge id, 0, 0, 0) and a key drawn per
 *    (sample, vertex); ln is the FP32 series below, so both implementations
 *    compare the same keys.
 *  - Density.  For one edge the ray through p is fixed by (t, u).  With the
 *    edge on the z axis, rho the distance from p to the line and P_t the
 *    coordinate of p's projection, the ray's closest point is
 *    q = m(z) - (u^2/rho) e1 + u sqrt(1 - u^2/rho^2) e2 (e1 the unit vector
 *    from p's projection to the line, e2 = edge direction x e1), and the solid
 *    angle it sweeps is d omega = J dz du with
 *        J = sqrt(rho^2 - u^2) / ((z - P_t)^2 + rho^2 - u^2)^(3/2)
 *    (|d q/dz x d q/du . (q - p)| / |q - p|^3; the numerator reduces to
 *    sqrt(rho^2 - u^2) and |q - p|^2 to (z - P_t)^2 + rho^2 - u^2).  Light
 *    points are drawn by area (density 1/A over all lights), so a direction
 *    has density sum over the light hits k along it of r_k^2 / (A |cos_k|).
 *    The density of the sample (edge e, t, u) is
 *        p_B = |E| J sum_k r_k^2/(A |cos_k|) [s_e < T_k] P(e | S_k),
 *    S_k the billboards crossed before hit k and P(e | S_k) the race's
 *    probability.
 *  - Combination.  The plain sampler (edge by length, t uniform) is extended
 *    by an auxiliary u uniform in [-w/2, w/2], and the integrand by the
 *    factor 1/w on that interval; both samplers then draw (e, t, u) and the
 *    balance heuristic with one sample of each weighs a sample by
 *        1 / (p_A(e, t) + w p_B(e, t, u)),
 *    in place of 1 / p_A.  The plain sampler covers every (e, t), so the sum
 *    stays unbiased whatever p_B is, as long as it is the density the
 *    billboard sampler really has.
 */

constexpr uint32_t K_EDGE_NEE = 6;  /* Philox stream kind: auxiliary u and the race's key */

/* ln x for normal x > 0, FP32 in a fixed order (no library call): x = m 2^k
 * with m in [1, 2) from the bits, halved (k + 1) above sqrt 2 so that m is
 * in [sqrt(1/2), sqrt 2]; ln m = 2 atanh(z) with z = (m-1)/(m+1), |z| < 0.172,
 * by the series 2 z (1 + z^2/3 + ... + z^12/13) in Horner's form (first
 * omitted term below 1e-11 relative); then k ln 2 added. */
float ln32(float x) {
  uint32_t bits;
  std::memcpy(&bits, &x, 4);
  int k = (int)((bits >> 23) & 0xffu) - 127;
  uint32_t mb = (bits & 0x7fffffu) | 0x3f800000u;
  float m;
  std::memcpy(&m, &mb, 4);
  if (m > 1.41421354f) {
    m = m * 0.5f;
    k += 1;
  }
  float z = (m - 1.0f) / (m + 1.0f);
  float z2 = z * z;
  float s = 0.0769230798f;           /* 1/13 */
  s = z2 * s + 0.0909090936f;        /* 1/11 */
  s = z2 * s + 0.111111112f;         /* 1/9 */
  s = z2 * s + 0.142857149f;         /* 1/7 */
  s = z2 * s + 0.200000003f;         /* 1/5 */
  s = z2 * s + 0.333333343f;         /* 1/3 */
  s = z2 * s + 1.0f;
  float lm = (2.0f * z) * s;
  return (float)k * 0.693147182f + lm;
}

/* U in (0, 1) with 23 random bits, exact in FP32 (never 0: ln stays finite). */
float u01_open(uint32_t x) { return ((float)(x >> 9) + 0.5f) * 1.1920928955078125e-07f; }

/* Silhouette test seen from p (as the hierarchy's leaf test): false only when
 * the two faces lie strictly on opposite sides of the plane through p and
 * the edge. */
bool nee_silhouette(const ETLeaf& L, const float p[3]) {
  if (L.boundary) return true;
  float a0[3], a1[3], d0[3], d1[3];
  for (int i = 0; i < 3; ++i) {
    a0[i] = L.v0[i] - p[i]; a1[i] = L.v1[i] - p[i];
    d0[i] = L.c0[i] - p[i]; d1[i] = L.c1[i] - p[i];
  }
  float m[3] = {a0[1] * a1[2] - a0[2] * a1[1], a0[2] * a1[0] - a0[0] * a1[2], a0[0] * a1[1] - a0[1] * a1[0]};
  float s0 = dot32(m, d0), s1 = dot32(m, d1);
  return !((s0 > 0.0f && s1 < 0.0f) || (s0 < 0.0f && s1 > 0.0f));
}

struct NeeCross {
  int leaf;        /* position in the tree's leaf array */
  float s, t, u;   /* ray parameter (units of d), edge parameter, signed distance */
  float imp;       /* importance (0: not a silhouette from p) */
};

/* Crossing of the billboard of leaf L by the ray p + s d, s in (0, smax), with
 * half width hw (FP32, fixed order); n: the shading normal at p.  The
 * importance is zero unless the edge is a silhouette seen from p and the
 * crossing's point on the edge lies strictly above p's tangent plane and
 * farther from p than the billboard's width (edges in or below that plane,
 * such as those of p's own triangle, and edges of p's immediate surroundings
 * are left to the plain sampler: a shadow ray crosses their billboards at its
 * very start, where they bound no light).  The closest points of the two lines:
 * with r = v0 - p, E = v1 - v0 and c = d x E,
 *   s = ((r x E) . c) / |c|^2,  t = ((r x d) . c) / |c|^2,  u = (c . r) / |c|. */
bool nee_cross(const ETLeaf& L, const float p[3], const float n[3], const float d[3], float smax, float hw,
               NeeCross* out) {
  float E[3], r[3];
  for (int i = 0; i < 3; ++i) { E[i] = L.v1[i] - L.v0[i]; r[i] = L.v0[i] - p[i]; }
  float c[3] = {d[1] * E[2] - d[2] * E[1], d[2] * E[0] - d[0] * E[2], d[0] * E[1] - d[1] * E[0]};
  float cc = dot32(c, c);
  if (!(cc > 0.0f)) return false;
  float num = dot32(c, r);
  if (num * num > (hw * hw) * cc) return false;
  float rE[3] = {r[1] * E[2] - r[2] * E[1], r[2] * E[0] - r[0] * E[2], r[0] * E[1] - r[1] * E[0]};
  float rd[3] = {r[1] * d[2] - r[2] * d[1], r[2] * d[0] - r[0] * d[2], r[0] * d[1] - r[1] * d[0]};
  float s = dot32(rE, c) / cc;
  float t = dot32(rd, c) / cc;
  if (!(s > 0.0f && s < smax)) return false;
  if (!(t >= 0.0f && t <= 1.0f)) return false;
  out->s = s;
  out->t = t;
  out->u = num / std::sqrt(cc);
  out->imp = 0.0f;
  if (nee_silhouette(L, p)) {
    float dm[3];
    for (int i = 0; i < 3; ++i) dm[i] = r[i] + t * E[i];
    float dist = std::sqrt(dot32(dm, dm));
    if (dist > 2.0f * hw && dot32(n, dm) > 0.0f) out->imp = L.len / dist;
  }
  return true;
}

/* Every billboard the ray p + s d crosses for s in (0, smax). */
void nee_crossings(const EdgeTree& T, const float p[3], const float n[3], const float d[3], float smax, float hw,
                   std::vector<NeeCross>& out) {
  out.clear();
  for (int k = 0; k < (int)T.leaf.size(); ++k) {
    NeeCross x;
    if (nee_cross(T.leaf[k], p, n, d, smax, hw, &x)) {
      x.leaf = k;
      out.push_back(x);
    }
  }
}

struct NeeLightHit { int tri; float t; };

/* Light triangles hit by the ray p + s d, s > 0 (the watertight test). */
void nee_light_hits(const Prep& P, const float p[3], const float d[3], std::vector<NeeLightHit>& out) {
  out.clear();
  const or_scene_t& sc = *P.sc;
  Shear sh = make_shear(d);
  for (int j = 0; j < sc.n_light_tris; ++j) {
    int lt = sc.light_tris[j];
    float tt, b1, b2;
    if (watertight(sh, p, vtx(P, sc.tris[3 * lt]), vtx(P, sc.tris[3 * lt + 1]), vtx(P, sc.tris[3 * lt + 2]),
                   INFINITY, &tt, &b1, &b2))
      out.push_back(NeeLightHit{lt, tt});
  }
}

/* J(z, u) |E| of the header, FP64, for leaf L seen from p at (t, u); 0 where
 * no ray of the family exists (|u| >= rho). */
double nee_jacobian(const ETLeaf& L, const float p[3], float t, float u) {
  V3 v0{L.v0[0], L.v0[1], L.v0[2]}, v1{L.v1[0], L.v1[1], L.v1[2]}, P3{p[0], p[1], p[2]};
  V3 E = v1 - v0;
  double len = vlen(E);
  if (!(len > 0.0)) return 0.0;
  V3 Eh = (1.0 / len) * E;
  V3 a = P3 - v0;
  double Pt = vdot(a, Eh);
  double rho2 = vdot(a, a) - Pt * Pt;
  double uu = (double)u * (double)u;
  if (!(rho2 > uu)) return 0.0;
  double z = (double)t * len;
  double den = (z - Pt) * (z - Pt) + rho2 - uu;
  return len * std::sqrt(rho2 - uu) / (den * std::sqrt(den));
}

/* Density p_B of the billboard sampler at (leaf, t, u) for the ray p + s d
 * through that edge point.  The edge's crossing along d (recomputed) gives
 * its membership, importance and ray parameter; J is taken at the sample's
 * (t, u).  All light hits along d count, each with its own set of crossed
 * billboards. */
double nee_density(const Prep& P, const EdgeTree& T, const float p[3], const float n[3], const float d[3], int leaf,
                   float t, float u, float hw) {
  std::vector<NeeLightHit> hits;
  nee_light_hits(P, p, d, hits);
  if (hits.empty() || !(P.light_total > 0.0)) return 0.0;
  float smax = 0.0f;
  for (const NeeLightHit& h : hits) smax = std::max(smax, h.t);
  std::vector<NeeCross> xs;
  nee_crossings(T, p, n, d, smax, hw, xs);
  float imp_e = -1.0f, s_e = 0.0f;
  for (const NeeCross& x : xs)
    if (x.leaf == leaf) { imp_e = x.imp; s_e = x.s; }
  if (!(imp_e > 0.0f)) return 0.0;
  V3 dv{d[0], d[1], d[2]};
  double dl = vlen(dv);
  double dens = 0.0;
  for (const NeeLightHit& h : hits) {
    if (!(s_e < h.t)) continue;
    double W = 0.0;
    for (const NeeCross& x : xs)
      if (x.s < h.t) W += (double)x.imp;
    if (!(W > 0.0)) continue;
    const float *a = vtx(P, P.sc->tris[3 * h.tri]), *b = vtx(P, P.sc->tris[3 * h.tri + 1]),
                *c = vtx(P, P.sc->tris[3 * h.tri + 2]);
    V3 n = vcross(V3{(double)b[0] - a[0], (double)b[1] - a[1], (double)b[2] - a[2]},
                  V3{(double)c[0] - a[0], (double)c[1] - a[1], (double)c[2] - a[2]});
    double cosk = std::fabs(vdot(n, dv)) / (vlen(n) * dl);
    if (!(cosk > 0.0)) continue;
    double r = (double)h.t * dl;
    dens += r * r / (P.light_total * cosk) * ((double)imp_e / W);
  }
  return dens * nee_jacobian(T.leaf[leaf], p, t, u);
}

/* The ray from p through the point of leaf L's family at (t, u) (FP32, fixed
 * order): d = q - p with q the ray's closest point to the edge's line.  False
 * when |u| >= rho or the edge is degenerate. */
bool nee_ray(const ETLeaf& L, const float p[3], float t, float u, float d[3]) {
  float E[3], a[3];
  for (int i = 0; i < 3; ++i) { E[i] = L.v1[i] - L.v0[i]; a[i] = p[i] - L.v0[i]; }
  float len = std::sqrt(dot32(E, E));
  if (!(len > 0.0f)) return false;
  float Eh[3] = {E[0] / len, E[1] / len, E[2] / len};
  float Pt = dot32(a, Eh);
  float ap[3] = {a[0] - Pt * Eh[0], a[1] - Pt * Eh[1], a[2] - Pt * Eh[2]};
  float rho = std::sqrt(dot32(ap, ap));
  if (!(rho > std::fabs(u))) return false;
  float e1[3] = {-ap[0] / rho, -ap[1] / rho, -ap[2] / rho};
  float e2[3] = {Eh[1] * e1[2] - Eh[2] * e1[1], Eh[2] * e1[0] - Eh[0] * e1[2], Eh[0] * e1[1] - Eh[1] * e1[0]};
  float k = u / rho;
  float cq = std::sqrt(1.0f - k * k);
  float a1 = -(u * k), a2 = u * cq;
  for (int i = 0; i < 3; ++i) {
    float m = L.v0[i] + t * E[i];
    d[i] = ((m + a1 * e1[i]) + a2 * e2[i]) - p[i];
  }
  return true;
}

/* Exponential race over the crossings: smallest -ln(U_e) / imp_e wins, ties
 * to the lower edge id; returns the index into xs or -1 (nothing with a
 * positive importance). */
int nee_race(const EdgeTree& T, const std::vector<NeeCross>& xs, uint32_t key0, uint32_t key1) {
  int best = -1;
  float bk = 0.0f;
  for (int i = 0; i < (int)xs.size(); ++i) {
    if (!(xs[i].imp > 0.0f)) continue;
    int eid = T.leaf[xs[i].leaf].eid;
    uint32_t ctr[4] = {(uint32_t)eid, 0u, 0u, 0u}, key[2] = {key0, key1}, r[4];
    philox4x32_10(ctr, key, r);
    float kv = -ln32(u01_open(r[0])) / xs[i].imp;
    if (best < 0 || kv < bk || (kv == bk && eid < T.leaf[xs[best].leaf].eid)) {
      best = i;
      bk = kv;
    }
  }
  return best;
}

/* Billboard half width from the scene's vertices (FP64, rounded once): w/2,
 * w = |(0.02 MAD_x, 0.02 MAD_y, 0.02 MAD_z)|. */
float nee_half_width(const or_scene_t& sc) {
  if (sc.n_verts <= 0) return 0.0f;
  double mean[3] = {0, 0, 0}, mad[3] = {0, 0, 0};
  for (int i = 0; i < sc.n_verts; ++i)
    for (int c = 0; c < 3; ++c) mean[c] += sc.verts[3 * i + c];
  for (int c = 0; c < 3; ++c) mean[c] /= sc.n_verts;
  for (int i = 0; i < sc.n_verts; ++i)
    for (int c = 0; c < 3; ++c) mad[c] += std::fabs(sc.verts[3 * i + c] - mean[c]);
  double s2 = 0.0;
  for (int c = 0; c < 3; ++c) {
    double m = 0.02 * mad[c] / sc.n_verts;
    s2 += m * m;
  }
  return (float)(0.5 * std::sqrt(s2));
}
