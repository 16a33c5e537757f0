// Hierarchical selection of secondary edges (Sec. 5.3.1): device side.
//
// Two hierarchies under one root, after Olson and Zhang's Hough-space
// silhouette search.  Edges that are silhouettes seen from the camera position
// O (or lack a second face) are grouped by 3D position; the others by 3D
// position and the Hough points of their two face planes (6D).  The Hough
// point of a plane with unit normal n through c, taken about O, is
// ((c - O).n) n.  The tree is the binary radix tree over sorted 30-bit Morton
// codes of the box centroids (3D: 10 bits per axis; 6D: 5 bits per axis), with
// the class as the top key bit.
//
// At a shading point p with normal n, a child's importance is zero when it
// cannot hold a contributing edge (at the last vertex: its cone of directions
// from p misses the cone to the lights' bounding sphere, or it holds no
// silhouette seen from p, by the v-sphere test in Hough space for 6D nodes and
// exactly at leaves;
// anywhere: the whole box lies below the horizon by more than the side offset),
// one when p lies inside the parent's box, and otherwise total length x
// max(cosine bound, eps) / distance to the box centre.  S samples start at the
// root and split between the children in proportion to importance (stochastic
// rounding); weighted reservoir sampling over the leaves reached keeps one edge,
// weighted (sum of c_e I_e / P_e over the leaves) / (S I_e), which makes the
// edge term unbiased for any positive importances.
//
// Every value that decides the tree's shape, a split or a pick is FP32 with
// one rounding per operation (intrinsics that are never contracted).
#pragma once

#include "drt_device.cuh"

namespace drt {

constexpr int kEtStack = 64;
constexpr uint32_t kEdgeTree = 5;  // Philox stream kind of the hierarchy's random numbers
constexpr int kEtDefaultSamples = 16;
constexpr int kEtMaxSamples = 64;

// Internal node: 8 float4, child slot c at rows 4c..4c+3:
//   (lo.xyz, L), (hi.xyz, all-B as 0/1), (Hough lo.xyz, child code bits), (Hough hi.xyz, 0)
// Leaf record (key order): (v0.xyz, length), (v1.xyz, edge id bits),
//   (c0.xyz, flags bits: 1 boundary, 2 class B), (c1.xyz, 0)
constexpr int kEtNodeF4 = 8;
constexpr int kEtLeafF4 = 4;

__device__ __forceinline__ float et_min(float a, float b) { return b < a ? b : a; }
__device__ __forceinline__ float et_max(float a, float b) { return b > a ? b : a; }

struct EtLeafData {
  float v0[3], v1[3], c0[3], c1[3], h0[3], h1[3];
  float len;
  bool boundary, classB;
};

__device__ __forceinline__ bool et_unit_normal(const float* a, const float* b, const float* c, float* n) {
  float e1[3], e2[3];
  for (int i = 0; i < 3; ++i) { e1[i] = fs(b[i], a[i]); e2[i] = fs(c[i], a[i]); }
  float m[3] = {fs(fm(e1[1], e2[2]), fm(e1[2], e2[1])), fs(fm(e1[2], e2[0]), fm(e1[0], e2[2])),
                fs(fm(e1[0], e2[1]), fm(e1[1], e2[0]))};
  float l = fsq(dot3x(m, m));
  if (!(l > 0.0f)) return false;
  for (int i = 0; i < 3; ++i) n[i] = fdv(m[i], l);
  return true;
}

// Geometry and class of edge (v0, v1) with third vertices opp (-1: the edge
// does not have exactly two faces).  Face planes are oriented consistently
// across the edge: (v0, v1, c0) and (v1, v0, c1).
__device__ __forceinline__ void et_leaf_data(const float* verts, int2 ev, int2 opp, const float O[3], EtLeafData& L) {
  for (int i = 0; i < 3; ++i) {
    L.v0[i] = verts[3 * ev.x + i];
    L.v1[i] = verts[3 * ev.y + i];
    L.c0[i] = L.c1[i] = L.h0[i] = L.h1[i] = 0.0f;
  }
  float d[3] = {fs(L.v1[0], L.v0[0]), fs(L.v1[1], L.v0[1]), fs(L.v1[2], L.v0[2])};
  L.len = fsq(dot3x(d, d));
  L.boundary = opp.y < 0;
  L.classB = false;
  if (L.boundary) return;
  for (int i = 0; i < 3; ++i) { L.c0[i] = verts[3 * opp.x + i]; L.c1[i] = verts[3 * opp.y + i]; }
  float n0[3], n1[3];
  if (et_unit_normal(L.v0, L.v1, L.c0, n0) && et_unit_normal(L.v1, L.v0, L.c1, n1)) {
    float r0[3] = {fs(L.v0[0], O[0]), fs(L.v0[1], O[1]), fs(L.v0[2], O[2])};
    float t0 = dot3x(n0, r0), t1 = dot3x(n1, r0);
    for (int i = 0; i < 3; ++i) { L.h0[i] = fm(t0, n0[i]); L.h1[i] = fm(t1, n1[i]); }
    L.classB = (t0 > 0.0f && t1 > 0.0f) || (t0 < 0.0f && t1 < 0.0f);
  }
}

__device__ __forceinline__ uint32_t et_quant(float x, float lo, float ext, uint32_t levels) {
  if (!(ext > 0.0f)) return 0;
  float f = fm(fdv(fs(x, lo), ext), (float)levels);
  if (!(f > 0.0f)) return 0;
  if (f >= (float)(levels - 1)) return levels - 1;
  return (uint32_t)f;
}

// Key: class bit 30 above a 30-bit Morton code of the centroid (3D, or 6D
// with the Hough centroid in [-R, R]^3).
__device__ __forceinline__ uint32_t et_key(const EtLeafData& L, const float blo[3], const float bhi[3], float R) {
  float mid[3];
  for (int i = 0; i < 3; ++i) mid[i] = fm(fa(L.v0[i], L.v1[i]), 0.5f);
  uint32_t code = 0;
  if (!L.classB) {
    uint32_t q[3];
    for (int i = 0; i < 3; ++i) q[i] = et_quant(mid[i], blo[i], fs(bhi[i], blo[i]), 1024u);
    for (int bit = 9; bit >= 0; --bit)
      for (int i = 0; i < 3; ++i) code = (code << 1) | ((q[i] >> bit) & 1u);
  } else {
    uint32_t q[6];
    for (int i = 0; i < 3; ++i) q[i] = et_quant(mid[i], blo[i], fs(bhi[i], blo[i]), 32u);
    for (int i = 0; i < 3; ++i) q[3 + i] = et_quant(fm(fa(L.h0[i], L.h1[i]), 0.5f), -R, fa(R, R), 32u);
    for (int bit = 4; bit >= 0; --bit)
      for (int i = 0; i < 6; ++i) code = (code << 1) | ((q[i] >> bit) & 1u);
  }
  return ((L.classB ? 1u : 0u) << 30) | code;
}

// Radius about O of the scene box (bounds the Hough points).
__device__ __forceinline__ float et_hough_radius(const float blo[3], const float bhi[3], const float O[3]) {
  float q[3];
  for (int i = 0; i < 3; ++i) {
    float a = fs(blo[i], O[i]), b = fs(bhi[i], O[i]);
    q[i] = et_max(fm(a, a), fm(b, b));
  }
  return fsq(fa(fa(q[0], q[1]), q[2]));
}

struct EtSlot {
  float lo[3], hi[3], hlo[3], hhi[3];
  float L;
  bool allB;
  int child;
};

__device__ __forceinline__ void et_load_slot(const float4* nodes, int node, int c, EtSlot& s) {
  const float4* r = nodes + (size_t)kEtNodeF4 * node + 4 * c;
  float4 a = __ldg(r), b = __ldg(r + 1), h0 = __ldg(r + 2), h1 = __ldg(r + 3);
  s.lo[0] = a.x; s.lo[1] = a.y; s.lo[2] = a.z; s.L = a.w;
  s.hi[0] = b.x; s.hi[1] = b.y; s.hi[2] = b.z; s.allB = b.w != 0.0f;
  s.hlo[0] = h0.x; s.hlo[1] = h0.y; s.hlo[2] = h0.z; s.child = __float_as_int(h0.w);
  s.hhi[0] = h1.x; s.hhi[1] = h1.y; s.hhi[2] = h1.z;
}

struct EtQuery {
  float p[3], n[3], t[3], u[3];
  float C[3], r;  // v-sphere about O: centre (p - O)/2, radius |p - O|/2
  float lc[3], lr;  // sphere around the lights
  float eps;
  bool last, has_light;
};

// Sphere around a box: centre and padded half diagonal.
__device__ __forceinline__ void et_sphere(const float lo[3], const float hi[3], float c[3], float& r) {
  float d[3];
  for (int i = 0; i < 3; ++i) { c[i] = fm(fa(lo[i], hi[i]), 0.5f); d[i] = fs(hi[i], lo[i]); }
  r = fa(fm(fm(0.5f, fsq(dot3x(d, d))), 1.0001f), 1e-6f);
}

// At the last vertex only radiance that arrives from a light counts.  True if
// the cone of directions from p to the box's sphere and the cone to the
// lights' sphere are apart by more than 1e-3 rad (side rays leave an edge
// point by about eps): then no edge of the box has a nonzero term.
__device__ __forceinline__ bool et_light_cone_clears(const EtQuery& q, const float lo[3], const float hi[3]) {
  float cb[3], rb, vb[3], vl[3];
  et_sphere(lo, hi, cb, rb);
  for (int i = 0; i < 3; ++i) { vb[i] = fs(cb[i], q.p[i]); vl[i] = fs(q.lc[i], q.p[i]); }
  float db = fsq(dot3x(vb, vb)), dl = fsq(dot3x(vl, vl));
  if (!(db > rb) || !(dl > q.lr)) return false;
  float sb = fdv(rb, db), sl = fdv(q.lr, dl);
  float kb = fsq(fs(1.0f, fm(sb, sb))), kl = fsq(fs(1.0f, fm(sl, sl)));
  float cosA = fs(fm(kb, kl), fm(sb, sl)), sinA = fa(fm(sb, kl), fm(kb, sl));  // A = sum of the half-angles
  float cosAm = fs(fm(cosA, 0.9999995f), fm(sinA, 1e-3f)), sinAm = fa(fm(sinA, 0.9999995f), fm(cosA, 1e-3f));
  if (!(sinAm > 0.0f)) return false;
  float cg = fdv(dot3x(vb, vl), fm(db, dl));
  return cg < cosAm;
}

// Orthonormal frame of a unit normal (Duff et al., JCGT 2017).
__device__ __forceinline__ void et_frame(const float n[3], float t[3], float u[3]) {
  float sg = n[2] >= 0.0f ? 1.0f : -1.0f;
  float a = fdv(-1.0f, fa(sg, n[2]));
  float b = fm(fm(n[0], n[1]), a);
  t[0] = fa(1.0f, fm(fm(sg, fm(n[0], n[0])), a));
  t[1] = fm(sg, b);
  t[2] = -fm(sg, n[0]);
  u[0] = b;
  u[1] = fa(sg, fm(fm(n[1], n[1]), a));
  u[2] = -n[1];
}

__device__ __forceinline__ void et_query(const SceneView& s, const float p[3], const float n[3], bool last, float eps,
                                         EtQuery& q) {
  for (int i = 0; i < 3; ++i) { q.p[i] = p[i]; q.n[i] = n[i]; }
  et_frame(q.n, q.t, q.u);
  const float O[3] = {s.cam[3], s.cam[7], s.cam[11]};
  for (int i = 0; i < 3; ++i) q.C[i] = fm(fs(p[i], O[i]), 0.5f);
  q.r = fsq(dot3x(q.C, q.C));
  q.has_light = s.et_light != nullptr;
  if (q.has_light) {
    float4 l = __ldg(s.et_light);
    q.lc[0] = l.x; q.lc[1] = l.y; q.lc[2] = l.z; q.lr = l.w;
  }
  q.last = last;
  q.eps = eps;
}

// Upper bound of cos(n, x - p) over the box (Walter et al. 2005): the box's
// bounds in the frame (t, u, n) about p.
__device__ __forceinline__ float et_cos_bound(const EtQuery& q, const float lo[3], const float hi[3]) {
  float c[3], h[3];
  for (int i = 0; i < 3; ++i) { c[i] = fs(fm(fa(lo[i], hi[i]), 0.5f), q.p[i]); h[i] = fm(fs(hi[i], lo[i]), 0.5f); }
  float an[3] = {fabsf(q.n[0]), fabsf(q.n[1]), fabsf(q.n[2])};
  float at[3] = {fabsf(q.t[0]), fabsf(q.t[1]), fabsf(q.t[2])};
  float au[3] = {fabsf(q.u[0]), fabsf(q.u[1]), fabsf(q.u[2])};
  float cz = dot3x(q.n, c), ez = dot3x(an, h);
  float cx = dot3x(q.t, c), ex = dot3x(at, h);
  float cy = dot3x(q.u, c), ey = dot3x(au, h);
  float zmax = fa(cz, ez);
  float mx, my;
  if (zmax > 0.0f) {
    mx = et_max(fs(fabsf(cx), ex), 0.0f);
    my = et_max(fs(fabsf(cy), ey), 0.0f);
  } else {
    mx = fa(fabsf(cx), ex);
    my = fa(fabsf(cy), ey);
  }
  float den = fsq(fa(fa(fm(mx, mx), fm(my, my)), fm(zmax, zmax)));
  if (!(den > 0.0f)) return 0.0f;
  return fdv(zmax, den);
}

// True if the v-sphere clears the slot's Hough box (with a margin): no edge
// below is a silhouette seen from p.
__device__ __forceinline__ bool et_vsphere_clears(const EtQuery& q, const EtSlot& s) {
  float dmin2 = 0.0f, dmax2 = 0.0f, hm = 0.0f;
  for (int i = 0; i < 3; ++i) {
    float a = fs(s.hlo[i], q.C[i]), b = fs(q.C[i], s.hhi[i]);
    float o = et_max(et_max(a, b), 0.0f);
    dmin2 = fa(dmin2, fm(o, o));
    float xa = fs(q.C[i], s.hlo[i]), xb = fs(s.hhi[i], q.C[i]);
    dmax2 = fa(dmax2, et_max(fm(xa, xa), fm(xb, xb)));
    hm = et_max(hm, et_max(fabsf(s.hlo[i]), fabsf(s.hhi[i])));
  }
  float g = fm(1e-4f, fa(q.r, hm));
  float ri = fs(q.r, g), ro = fa(q.r, g);
  bool inside = ri > 0.0f && dmax2 < fm(ri, ri);
  bool outside = dmin2 > fm(ro, ro);
  return inside || outside;
}

// Exact silhouette test of the leaf at key position pos, seen from p.
__device__ __forceinline__ bool et_silhouette(const float4* leaf, int pos, const EtQuery& q) {
  const float4* r = leaf + (size_t)kEtLeafF4 * pos;
  float4 A = __ldg(r), B = __ldg(r + 1), C0 = __ldg(r + 2), C1 = __ldg(r + 3);
  if (__float_as_int(C0.w) & 1) return true;
  float a0[3] = {fs(A.x, q.p[0]), fs(A.y, q.p[1]), fs(A.z, q.p[2])};
  float a1[3] = {fs(B.x, q.p[0]), fs(B.y, q.p[1]), fs(B.z, q.p[2])};
  float d0[3] = {fs(C0.x, q.p[0]), fs(C0.y, q.p[1]), fs(C0.z, q.p[2])};
  float d1[3] = {fs(C1.x, q.p[0]), fs(C1.y, q.p[1]), fs(C1.z, q.p[2])};
  float m[3] = {fs(fm(a0[1], a1[2]), fm(a0[2], a1[1])), fs(fm(a0[2], a1[0]), fm(a0[0], a1[2])),
                fs(fm(a0[0], a1[1]), fm(a0[1], a1[0]))};
  float s0 = dot3x(m, d0), s1 = dot3x(m, d1);
  return !((s0 > 0.0f && s1 < 0.0f) || (s0 < 0.0f && s1 > 0.0f));
}

__device__ __forceinline__ float et_importance(const float4* leaf, const EtQuery& q, const EtSlot& s,
                                               const float plo[3], const float phi[3], bool has_parent) {
  if (q.last && q.has_light && et_light_cone_clears(q, s.lo, s.hi)) return 0.0f;
  if (q.last) {
    if (s.child < 0) {
      if (!et_silhouette(leaf, ~s.child, q)) return 0.0f;
    } else if (s.allB && et_vsphere_clears(q, s)) {
      return 0.0f;
    }
  }
  float cb = et_cos_bound(q, s.lo, s.hi);
  if (cb <= fm(-2.0f, q.eps)) return 0.0f;
  if (has_parent) {
    bool inside = true;
    for (int i = 0; i < 3; ++i) inside = inside && plo[i] <= q.p[i] && q.p[i] <= phi[i];
    if (inside) return 1.0f;
  }
  float c[3];
  for (int i = 0; i < 3; ++i) c[i] = fs(fm(fa(s.lo[i], s.hi[i]), 0.5f), q.p[i]);
  float d = fsq(dot3x(c, c));
  return fdv(fm(s.L, et_max(cb, q.eps)), et_max(d, 1e-30f));
}

// Pick one secondary edge for the query with S root samples.  Random numbers:
// one Philox block per popped item, counter (c0, c1, kind 5 | bounce | item
// ordinal, scene).  Out: edge id and the weight that replaces 1/P(edge) of the
// length sampler.  False: no edge can contribute.
static __device__ __noinline__ bool et_pick(const SceneView& s, const EtQuery& q, int S, uint2 key, uint32_t c0, uint32_t c1,
                                     uint32_t bounce, uint32_t scene, int& eid, float& weight) {
  if (s.et_root == -1 || S <= 0) return false;
  int st_enc[kEtStack], st_n[kEtStack];
  float st_P[kEtStack], st_I[kEtStack];
  int sp = 0;
  float nolo[3] = {0.0f, 0.0f, 0.0f};
  if (s.et_root < 0) {  // a single edge: its slot from the leaf record, no parent box
    const float4* r = s.et_leaf;
    float4 A = __ldg(r), B = __ldg(r + 1), C0 = __ldg(r + 2);
    EtSlot sl;
    sl.lo[0] = et_min(A.x, B.x); sl.lo[1] = et_min(A.y, B.y); sl.lo[2] = et_min(A.z, B.z);
    sl.hi[0] = et_max(A.x, B.x); sl.hi[1] = et_max(A.y, B.y); sl.hi[2] = et_max(A.z, B.z);
    sl.L = A.w;
    sl.allB = (__float_as_int(C0.w) & 2) != 0;
    sl.child = ~0;
    float I = et_importance(s.et_leaf, q, sl, nolo, nolo, false);
    if (!(I > 0.0f)) return false;
    st_enc[0] = ~0; st_n[0] = S; st_P[0] = 1.0f; st_I[0] = I;
  } else {
    st_enc[0] = s.et_root; st_n[0] = S; st_P[0] = 1.0f; st_I[0] = 0.0f;
  }
  sp = 1;
  float tot = 0.0f, chosen_I = 0.0f;
  int chosen = -1;
  uint32_t j = 0;
  // every node is pushed at most once per pick: more pops than the tree has
  // nodes and leaves means broken child links
  const uint32_t max_pops = 2u * (uint32_t)s.E + 1u;
  while (sp > 0) {
    if (j >= max_pops) {
      raise_flag(s.err, DRT_DEV_TRAVERSAL_CAP, s.E);
      return false;
    }
    --sp;
    int enc = st_enc[sp], n = st_n[sp];
    float P = st_P[sp], Ii = st_I[sp];
    uint4 r = rng4(key, c0, c1, kEdgeTree, bounce, j, scene);
    ++j;
    float u = u01f(r.x);
    if (enc < 0) {
      if (!(P > 0.0f)) continue;
      float w = fm((float)n, fdv(Ii, P));
      tot = fa(tot, w);
      if (fm(u, tot) < w) { chosen = ~enc; chosen_I = Ii; }
      continue;
    }
    EtSlot a, b;
    et_load_slot(s.et_nodes, enc, 0, a);
    et_load_slot(s.et_nodes, enc, 1, b);
    float plo[3], phi[3];
    for (int i = 0; i < 3; ++i) { plo[i] = et_min(a.lo[i], b.lo[i]); phi[i] = et_max(a.hi[i], b.hi[i]); }
    float I0 = et_importance(s.et_leaf, q, a, plo, phi, true);
    float I1 = et_importance(s.et_leaf, q, b, plo, phi, true);
    float sum = fa(I0, I1);
    if (!(sum > 0.0f)) continue;
    float p0 = fdv(I0, sum), p1 = fdv(I1, sum);
    int n0;
    if (!(I0 > 0.0f)) {
      n0 = 0;
    } else if (!(I1 > 0.0f)) {
      n0 = n;
    } else {
      float x = fm((float)n, p0);
      float fl = floorf(x);
      n0 = (int)fl + (u < fs(x, fl) ? 1 : 0);
      n0 = min(max(n0, 0), n);
    }
    int n1 = n - n0;
    if (sp + 2 > kEtStack) {
      raise_flag(s.err, DRT_DEV_STACK_OVERFLOW, enc);
      return false;
    }
    if (n1 > 0) { st_enc[sp] = b.child; st_n[sp] = n1; st_P[sp] = fm(P, p1); st_I[sp] = I1; ++sp; }
    if (n0 > 0) { st_enc[sp] = a.child; st_n[sp] = n0; st_P[sp] = fm(P, p0); st_I[sp] = I0; ++sp; }
  }
  if (chosen < 0) return false;
  eid = __float_as_int(__ldg(s.et_leaf + (size_t)kEtLeafF4 * chosen + 1).w);
  weight = fdv(fdv(tot, (float)S), chosen_I);
  return true;
}

}  // namespace drt
