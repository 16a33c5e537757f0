// Next-event estimation for edges (Sec. 5.3.3): device side.
//
// At a shading point p the shadow ray of next-event estimation (p toward the
// light point y drawn by area) is reused.  Every edge is a billboard of width
// w facing the ray: it contains the edge's line, and its normal is the part
// of the ray direction perpendicular to the edge, so the ray meets it at the
// ray's closest approach to the line.  The ray crosses it when the two lines
// pass within w/2 of each other, at an edge parameter t in [0, 1], with the
// closest point on the ray between p and the light point (0 < s < T, s and T
// in units of d = y - p).  The edge point at t is the sample.
//
// Importance of a crossed edge: length / distance from p to that point; zero
// unless the edge is a silhouette seen from p and the point lies strictly
// above p's tangent plane and farther from p than the width (a shadow ray
// crosses the billboards of p's immediate surroundings at its very start,
// where they bound no light; the length sampler keeps those edges).  One edge is picked by an exponential race (key
// -ln U_e / importance_e, the smallest wins, ties to the lower edge id; U_e
// from Philox4x32-10 with counter (edge id, 0, 0, 0) and a per-sample key),
// which picks e with probability importance_e / sum over the crossed edges in
// any traversal order.
//
// Density of a sample (edge e, t, u), u the signed distance of the lines:
//   p_B = |E| J(z, u) sum_k r_k^2 / (A |cos_k|) [s_e < T_k] imp_e / W_k,
//   J = sqrt(rho^2 - u^2) / ((z - P_t)^2 + rho^2 - u^2)^(3/2),
// the solid angle per unit edge length and offset of the rays whose closest
// point to the edge's line lies at z = t |E| and distance |u| (rho: distance
// from p to the line, P_t: the coordinate of p's projection), times the
// density of the light direction (area sampling, every light hit k along the
// ray, A the lights' total area) and the race probability with the edges W_k
// crossed before hit k.
//
// Crossings, importances and race keys are FP32 with one rounding per
// operation in a fixed order; densities are FP64.
#pragma once

#include "edge_tree.cuh"

namespace drt {

constexpr uint32_t kEdgeNee = 6;      // Philox stream kind: auxiliary offset and the race's key
constexpr int kNeeMaxLightHits = 8;   // light triangles along one ray that the density sums over

// ln x for normal x > 0 (own FP32 series, fixed order): x = m 2^k with m in
// [1, 2) from the bits, halved (k + 1) above sqrt 2; ln m = 2 atanh(z), z =
// (m - 1)/(m + 1), by the odd series to z^13 in Horner's form; plus k ln 2.
__device__ __forceinline__ float ln32(float x) {
  uint32_t bits = __float_as_uint(x);
  int k = (int)((bits >> 23) & 0xffu) - 127;
  float m = __uint_as_float((bits & 0x7fffffu) | 0x3f800000u);
  if (m > 1.41421354f) {
    m = fm(m, 0.5f);
    k += 1;
  }
  float z = fdv(fs(m, 1.0f), fa(m, 1.0f));
  float z2 = fm(z, z);
  float s = 0.0769230798f;
  s = fa(fm(z2, s), 0.0909090936f);
  s = fa(fm(z2, s), 0.111111112f);
  s = fa(fm(z2, s), 0.142857149f);
  s = fa(fm(z2, s), 0.200000003f);
  s = fa(fm(z2, s), 0.333333343f);
  s = fa(fm(z2, s), 1.0f);
  float lm = fm(fm(2.0f, z), s);
  return fa(fm((float)k, 0.693147182f), lm);
}

// U in (0, 1) with 23 random bits (never 0).
__device__ __forceinline__ float u01_open(uint32_t x) { return fm(fa((float)(x >> 9), 0.5f), 1.1920928955078125e-07f); }

// Silhouette seen from p: false only when the two faces lie strictly on
// opposite sides of the plane through p and the edge (leaf record at pos).
__device__ __forceinline__ bool nee_silhouette(const float4 A, const float4 B, const float4 C0, const float4 C1,
                                               const float p[3]) {
  if (__float_as_int(C0.w) & 1) return true;
  float a0[3] = {fs(A.x, p[0]), fs(A.y, p[1]), fs(A.z, p[2])};
  float a1[3] = {fs(B.x, p[0]), fs(B.y, p[1]), fs(B.z, p[2])};
  float d0[3] = {fs(C0.x, p[0]), fs(C0.y, p[1]), fs(C0.z, p[2])};
  float d1[3] = {fs(C1.x, p[0]), fs(C1.y, p[1]), fs(C1.z, p[2])};
  float m[3] = {fs(fm(a0[1], a1[2]), fm(a0[2], a1[1])), fs(fm(a0[2], a1[0]), fm(a0[0], a1[2])),
                fs(fm(a0[0], a1[1]), fm(a0[1], a1[0]))};
  float s0 = dot3x(m, d0), s1 = dot3x(m, d1);
  return !((s0 > 0.0f && s1 < 0.0f) || (s0 < 0.0f && s1 > 0.0f));
}

struct NeeCross {
  int eid;
  float s, t, u, imp;
};

// Crossing of the billboard of the leaf at key position pos by the ray
// p + s d, s in (0, smax), half width hw; n: shading normal at p.
__device__ __forceinline__ bool nee_cross(const float4* leaf, int pos, const float p[3], const float n[3],
                                          const float d[3], float smax, float hw, NeeCross& x) {
  const float4* r4 = leaf + (size_t)kEtLeafF4 * pos;
  float4 A = __ldg(r4), B = __ldg(r4 + 1);
  float E[3] = {fs(B.x, A.x), fs(B.y, A.y), fs(B.z, A.z)};
  float r[3] = {fs(A.x, p[0]), fs(A.y, p[1]), fs(A.z, p[2])};
  float c[3] = {fs(fm(d[1], E[2]), fm(d[2], E[1])), fs(fm(d[2], E[0]), fm(d[0], E[2])),
                fs(fm(d[0], E[1]), fm(d[1], E[0]))};
  float cc = dot3x(c, c);
  if (!(cc > 0.0f)) return false;
  float num = dot3x(c, r);
  if (fm(num, num) > fm(fm(hw, hw), cc)) return false;
  float rE[3] = {fs(fm(r[1], E[2]), fm(r[2], E[1])), fs(fm(r[2], E[0]), fm(r[0], E[2])),
                 fs(fm(r[0], E[1]), fm(r[1], E[0]))};
  float rd[3] = {fs(fm(r[1], d[2]), fm(r[2], d[1])), fs(fm(r[2], d[0]), fm(r[0], d[2])),
                 fs(fm(r[0], d[1]), fm(r[1], d[0]))};
  float s = fdv(dot3x(rE, c), cc);
  float t = fdv(dot3x(rd, c), cc);
  if (!(s > 0.0f && s < smax)) return false;
  if (!(t >= 0.0f && t <= 1.0f)) return false;
  x.eid = __float_as_int(B.w);
  x.s = s;
  x.t = t;
  x.u = fdv(num, fsq(cc));
  x.imp = 0.0f;
  float4 C0 = __ldg(r4 + 2), C1 = __ldg(r4 + 3);
  if (nee_silhouette(A, B, C0, C1, p)) {
    float dm[3] = {fa(r[0], fm(t, E[0])), fa(r[1], fm(t, E[1])), fa(r[2], fm(t, E[2]))};
    float dist = fsq(dot3x(dm, dm));
    if (dist > fm(2.0f, hw) && dot3x(n, dm) > 0.0f) x.imp = fdv(A.w, dist);
  }
  return true;
}

// The light triangles hit by the ray p + s d, s > 0, in light-list order (at
// most kNeeMaxLightHits; more raises the device flag and keeps the first).
struct NeeHits {
  int n;
  float t[kNeeMaxLightHits];
  double w[kNeeMaxLightHits];  // r_k^2 / (A |cos_k|)
};
__device__ __forceinline__ void nee_light_hits(const SceneView& s, const float p[3], const float d[3], NeeHits& h) {
  h.n = 0;
  if (s.L <= 0) return;
  Shear sh = make_shear(d);
  double A = s.light_cdf[s.L - 1];
  double dl = sqrt((double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2]);
  for (int j = 0; j < s.L; ++j) {
    const int32_t* id = s.tris + 3 * s.light_tris[j];
    float3 a = ld3(s.verts + 3 * id[0]), b = ld3(s.verts + 3 * id[1]), c = ld3(s.verts + 3 * id[2]);
    float tt, b1, b2;
    if (!watertight(sh, p, a, b, c, INFINITY, &tt, &b1, &b2)) continue;
    if (h.n >= kNeeMaxLightHits) {
      raise_flag(s.err, DRT_DEV_TRAVERSAL_CAP, j);
      break;
    }
    double e1[3] = {(double)b.x - a.x, (double)b.y - a.y, (double)b.z - a.z};
    double e2[3] = {(double)c.x - a.x, (double)c.y - a.y, (double)c.z - a.z};
    double nn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double nl = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    double cosk = fabs(nn[0] * d[0] + nn[1] * d[1] + nn[2] * d[2]) / (nl * dl);
    double rk = (double)tt * dl;
    h.t[h.n] = tt;
    h.w[h.n] = cosk > 0.0 ? rk * rk / (A * cosk) : 0.0;
    ++h.n;
  }
}

// One query of the billboards along the ray p + s d: every crossing with s
// below the largest of t_sel and the light hits' T_k.  Out: the race's
// winner among the crossings with s < t_sel (t_sel <= 0: no race), the sums
// W_k of the importances crossed before each light hit, and the importance
// and ray parameter of the target edge (-1 when it is not crossed).
struct NeeQuery {
  NeeCross win;
  float win_key;
  bool has_win;
  float timp, ts;
  double W[kNeeMaxLightHits];
};

__device__ __forceinline__ bool nee_box_hit(const float4 lo4, const float4 hi4, const float p[3], const float d[3],
                                            float smax, float pad) {
  // conservative: the exact crossing test at the leaves decides
  float lo[3] = {lo4.x, lo4.y, lo4.z}, hi[3] = {hi4.x, hi4.y, hi4.z};
  float tn = -1e-6f, tf = smax * 1.00001f + 1e-6f;
  for (int i = 0; i < 3; ++i) {
    float ext = fmaxf(fabsf(lo[i]), fabsf(hi[i]));
    float l = lo[i] - (pad + 1e-5f * ext), h = hi[i] + (pad + 1e-5f * ext);
    if (d[i] == 0.0f) {
      if (p[i] < l || p[i] > h) return false;
      continue;
    }
    float inv = 1.0f / d[i];
    float t0 = (l - p[i]) * inv, t1 = (h - p[i]) * inv;
    tn = fmaxf(tn, fminf(t0, t1));
    tf = fminf(tf, fmaxf(t0, t1));
  }
  return tn <= tf * 1.00001f + 1e-6f;
}

__device__ __noinline__ void nee_query(const SceneView& s, const float p[3], const float n[3], const float d[3],
                                       float hw, float t_sel, uint2 rkey, int target, const NeeHits& h,
                                       NeeQuery& o) {
  o.has_win = false;
  o.win_key = 0.0f;
  o.timp = -1.0f;
  o.ts = 0.0f;
  for (int k = 0; k < kNeeMaxLightHits; ++k) o.W[k] = 0.0;
  float smax = t_sel;
  for (int k = 0; k < h.n; ++k) smax = fmaxf(smax, h.t[k]);
  if (!(smax > 0.0f) || s.et_root == -1) return;
  // stack of children: >= 0 internal node, < 0 ~(leaf position)
  int stack[kEtStack];
  int sp = 0;
  stack[sp++] = s.et_root < 0 ? ~0 : s.et_root;
  // every node and leaf is pushed at most once: more pops means broken links
  const int max_pops = 2 * s.E + 2;
  int pops = 0;
  const float pad = fm(hw, 1.01f);
  while (sp > 0) {
    if (++pops > max_pops) {
      raise_flag(s.err, DRT_DEV_TRAVERSAL_CAP, s.E);
      break;
    }
    int enc = stack[--sp];
    if (enc < 0) {
      NeeCross x;
      if (!nee_cross(s.et_leaf, ~enc, p, n, d, smax, hw, x)) continue;
      for (int k = 0; k < h.n; ++k)
        if (x.s < h.t[k]) o.W[k] += (double)x.imp;
      if (x.eid == target) {
        o.timp = x.imp;
        o.ts = x.s;
      }
      if (x.s < t_sel && x.imp > 0.0f) {
        uint4 r = philox(make_uint4((uint32_t)x.eid, 0u, 0u, 0u), rkey);
        float key = fdv(-ln32(u01_open(r.x)), x.imp);
        if (!o.has_win || key < o.win_key || (key == o.win_key && x.eid < o.win.eid)) {
          o.win = x;
          o.win_key = key;
          o.has_win = true;
        }
      }
      continue;
    }
    for (int c = 0; c < 2; ++c) {
      const float4* r4 = s.et_nodes + (size_t)kEtNodeF4 * enc + 4 * c;
      float4 lo4 = __ldg(r4), hi4 = __ldg(r4 + 1);
      if (!nee_box_hit(lo4, hi4, p, d, smax, pad)) continue;
      if (sp >= kEtStack) {
        raise_flag(s.err, DRT_DEV_STACK_OVERFLOW, enc);
        continue;
      }
      stack[sp++] = __float_as_int(__ldg(r4 + 2).w);
    }
  }
}

// |E| J(z, u) of the header for the edge (v0, v1) seen from p at (t, u), FP64;
// 0 where no ray of the family exists (|u| >= rho).
__device__ __forceinline__ double nee_jacobian(float3 v0, float3 v1, const float p[3], float t, float u) {
  double E[3] = {(double)v1.x - v0.x, (double)v1.y - v0.y, (double)v1.z - v0.z};
  double len = sqrt(E[0] * E[0] + E[1] * E[1] + E[2] * E[2]);
  if (!(len > 0.0)) return 0.0;
  double a[3] = {(double)p[0] - v0.x, (double)p[1] - v0.y, (double)p[2] - v0.z};
  double Pt = (a[0] * E[0] + a[1] * E[1] + a[2] * E[2]) / len;
  double rho2 = (a[0] * a[0] + a[1] * a[1] + a[2] * a[2]) - Pt * Pt;
  double uu = (double)u * (double)u;
  if (!(rho2 > uu)) return 0.0;
  double z = (double)t * len;
  double den = (z - Pt) * (z - Pt) + rho2 - uu;
  return len * sqrt(rho2 - uu) / (den * sqrt(den));
}

// The ray d = q - p of the edge's family through (t, u): q the ray's point
// closest to the edge's line, at z = t |E| and distance |u| (FP32, fixed
// order).  False when |u| >= rho or the edge is degenerate.
__device__ __forceinline__ bool nee_ray(float3 v0, float3 v1, const float p[3], float t, float u, float d[3]) {
  float E[3] = {fs(v1.x, v0.x), fs(v1.y, v0.y), fs(v1.z, v0.z)};
  float a[3] = {fs(p[0], v0.x), fs(p[1], v0.y), fs(p[2], v0.z)};
  float len = fsq(dot3x(E, E));
  if (!(len > 0.0f)) return false;
  float Eh[3] = {fdv(E[0], len), fdv(E[1], len), fdv(E[2], len)};
  float Pt = dot3x(a, Eh);
  float ap[3] = {fs(a[0], fm(Pt, Eh[0])), fs(a[1], fm(Pt, Eh[1])), fs(a[2], fm(Pt, Eh[2]))};
  float rho = fsq(dot3x(ap, ap));
  if (!(rho > fabsf(u))) return false;
  float e1[3] = {fdv(-ap[0], rho), fdv(-ap[1], rho), fdv(-ap[2], rho)};
  float e2[3] = {fs(fm(Eh[1], e1[2]), fm(Eh[2], e1[1])), fs(fm(Eh[2], e1[0]), fm(Eh[0], e1[2])),
                 fs(fm(Eh[0], e1[1]), fm(Eh[1], e1[0]))};
  float k = fdv(u, rho);
  float cq = fsq(fs(1.0f, fm(k, k)));
  float a1 = -fm(u, k), a2 = fm(u, cq);
  float v0a[3] = {v0.x, v0.y, v0.z};
  for (int i = 0; i < 3; ++i) {
    float m = fa(v0a[i], fm(t, E[i]));
    d[i] = fs(fa(fa(m, fm(a1, e1[i])), fm(a2, e2[i])), p[i]);
  }
  return true;
}

// p_B of the target edge from a query along its ray, times |E| J (jac).
__device__ __forceinline__ double nee_density(const NeeQuery& o, const NeeHits& h, double jac) {
  if (!(o.timp > 0.0f)) return 0.0;
  double dens = 0.0;
  for (int k = 0; k < h.n; ++k) {
    if (!(o.ts < h.t[k]) || !(o.W[k] > 0.0)) continue;
    dens += h.w[k] * ((double)o.timp / o.W[k]);
  }
  return dens * jac;
}

// Billboard half width: w/2 with w the L2 norm over the coordinates of 2 % of
// the vertices' mean absolute deviation (one block of 1024 threads, FP64,
// strided sums then a fixed-order tree reduction, so every run takes the same
// value).
__global__ void __launch_bounds__(1024) k_nee_half_width(const float* verts, int V, float* out) {
  __shared__ double red[3][1024];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < V; i += 1024)
    for (int c = 0; c < 3; ++c) acc[c] += (double)verts[3 * i + c];
  for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
    __syncthreads();
  }
  double mean[3] = {red[0][0] / V, red[1][0] / V, red[2][0] / V};
  __syncthreads();
  for (int c = 0; c < 3; ++c) acc[c] = 0.0;
  for (int i = threadIdx.x; i < V; i += 1024)
    for (int c = 0; c < 3; ++c) acc[c] += fabs((double)verts[3 * i + c] - mean[c]);
  for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double s2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      double m = 0.02 * red[c][0] / V;
      s2 += m * m;
    }
    out[0] = V > 0 ? (float)(0.5 * sqrt(s2)) : 0.0f;
  }
}

}  // namespace drt
