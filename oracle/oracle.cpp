/*
 * oracle.cpp -- plain, slow CPU oracle for differentiable Monte Carlo ray
 * tracing through edge sampling (Li, "Differentiable Visual Computing",
 * Chapter 5).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and
 * the benchmark's CPU-baseline leg may load this file.  The CUDA library
 * shares no code, header, table or constant generator with it.
 *
 * What it computes (Sec. 5.2):
 *   - the image: per pixel, the box-filtered radiance integral (Eq. first),
 *     estimated by Monte Carlo (Eq. gradient_monte_carlo);
 *   - the gradient of sum_p w_p . I_p with respect to vertex positions,
 *     per-triangle albedo, light radiance and camera, as the sum of
 *       (a) the interior term: the second integral of Eq. redner_product_rule,
 *           by forward-mode dual numbers (Sec. 2.2.1) at fixed random numbers;
 *       (b) the primary-visibility edge term (Eq. dirac_rewrite, Eq. mc) with
 *           the edge-equation derivatives of Eq. redner_dirac_jacobian;
 *       (c) the secondary-visibility edge term (Eq. dirac_3d_edge with the
 *           Jacobian of Appendix 5.A and the alpha derivatives of
 *           Eq. alpha_3d) at every shading vertex.
 *
 * Precision.  Everything that decides a discrete outcome -- which triangle a
 * ray hits, whether a shadow ray is blocked, which edge or light triangle is
 * picked, where a sample point lies -- is FP32 in the operation order written
 * here: one IEEE rounding per operation and no contraction (compiled with
 * -ffp-contract=off).  Smooth values and all derivatives are FP64; sums are
 * FP64.  Sampling probabilities (edge and light-triangle pick, BSDF pdf) are
 * values, never differentiated: the derivative of an expectation whose
 * integrand is sampled from a parameter-dependent discrete or continuous pdf
 * is the expectation of d(integrand)/pdf with the pdf held fixed.
 *
 * Parity of which readings of the text are used is recorded in the project's
 * design notes; each function below names the passage it follows.
 */
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <functional>
#include <thread>
#include <vector>

namespace {

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based RNG (Salmon, Moraes, Dror, Shaw, SC'11).      */
/* ------------------------------------------------------------------------ */
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream kinds and passes of the counter layout. */
enum { K_CAMERA = 0, K_LIGHT = 1, K_BSDF = 2, K_EDGE_PRIMARY = 3, K_EDGE_SECONDARY = 4 };
enum { PASS_INTERIOR = 0, PASS_PRIMARY_EDGE = 1, PASS_SECONDARY_BASE = 2, PASS_NEE_BASE = 18 };

void rng(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t kind, uint32_t bounce, uint32_t pass,
         uint32_t scene, uint32_t out[4]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {c0, c1, (kind << 24) | ((bounce & 0xffu) << 16) | (pass & 0xffffu), scene};
  philox4x32_10(ctr, key, out);
}
/* u in [0,1) with 24 random bits, exact in FP32. */
float u01f(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-08f; }
/* u in [0,1) with 53 random bits, exact in FP64. */
double u01d(uint32_t x0, uint32_t x1) {
  return ((double)(x0 >> 5) * 67108864.0 + (double)(x1 >> 6)) * 1.1102230246251565e-16;
}

/* ------------------------------------------------------------------------ */
/* Sparse forward-mode dual numbers, FP64 (Sec. 2.2.1).                      */
/*                                                                           */
/* Beside each derivative d the dual carries ad, the same chain rule taken  */
/* with absolute values of every partial (|c_a| ad_a + |c_b| ad_b).  ad is  */
/* the magnitude of the terms that sum to d; where d is small by            */
/* cancellation (in-plane motion of a plane, an edge of the light seen from */
/* the light, an occluded edge whose two sides agree) an FP32              */
/* implementation of the same chain rule errs by about u * ad, not u * |d|, */
/* so parity tolerances are scaled by the sum of ad, not of |d|.            */
/* ------------------------------------------------------------------------ */
constexpr int MAXD = 192;
bool g_dual_overflow = false;

struct Dual {
  double v = 0.0;
  int n = 0;
  int32_t idx[MAXD];
  double d[MAXD];
  double ad[MAXD];
  Dual() {}
  Dual(double x) : v(x), n(0) {}
  Dual(const Dual& o) : v(o.v), n(o.n) {
    std::memcpy(idx, o.idx, sizeof(int32_t) * n);
    std::memcpy(d, o.d, sizeof(double) * n);
    std::memcpy(ad, o.ad, sizeof(double) * n);
  }
  Dual& operator=(const Dual& o) {
    v = o.v; n = o.n;
    std::memcpy(idx, o.idx, sizeof(int32_t) * n);
    std::memcpy(d, o.d, sizeof(double) * n);
    std::memcpy(ad, o.ad, sizeof(double) * n);
    return *this;
  }
  static Dual param(double x, int i, bool track) {
    Dual r(x);
    if (track) { r.n = 1; r.idx[0] = i; r.d[0] = 1.0; r.ad[0] = 1.0; }
    return r;
  }
};

/* r = value v, derivative ca*a' + cb*b' (merge of two sorted index lists). */
Dual lin(double v, double ca, const Dual& a, double cb, const Dual& b) {
  Dual r(v);
  int i = 0, j = 0, n = 0;
  double aa = std::fabs(ca), ab = std::fabs(cb);
  while (i < a.n || j < b.n) {
    int ia = i < a.n ? a.idx[i] : INT32_MAX;
    int ib = j < b.n ? b.idx[j] : INT32_MAX;
    double dv, av; int id;
    if (ia == ib) { id = ia; dv = ca * a.d[i] + cb * b.d[j]; av = aa * a.ad[i++] + ab * b.ad[j++]; }
    else if (ia < ib) { id = ia; dv = ca * a.d[i]; av = aa * a.ad[i++]; }
    else { id = ib; dv = cb * b.d[j]; av = ab * b.ad[j++]; }
    if (n >= MAXD) { g_dual_overflow = true; break; }
    r.idx[n] = id; r.d[n] = dv; r.ad[n] = av; ++n;
  }
  r.n = n;
  return r;
}
Dual scaled(double v, double c, const Dual& a) {
  Dual r(v);
  r.n = a.n;
  double ac = std::fabs(c);
  for (int i = 0; i < a.n; ++i) { r.idx[i] = a.idx[i]; r.d[i] = c * a.d[i]; r.ad[i] = ac * a.ad[i]; }
  return r;
}
Dual operator+(const Dual& a, const Dual& b) { return lin(a.v + b.v, 1.0, a, 1.0, b); }
Dual operator-(const Dual& a, const Dual& b) { return lin(a.v - b.v, 1.0, a, -1.0, b); }
Dual operator*(const Dual& a, const Dual& b) { return lin(a.v * b.v, b.v, a, a.v, b); }
Dual operator/(const Dual& a, const Dual& b) {
  double q = a.v / b.v;
  return lin(q, 1.0 / b.v, a, -q / b.v, b);
}
Dual operator-(const Dual& a) { return scaled(-a.v, -1.0, a); }
Dual operator*(double s, const Dual& a) { return scaled(s * a.v, s, a); }
Dual operator*(const Dual& a, double s) { return scaled(s * a.v, s, a); }
Dual operator/(const Dual& a, double s) { return scaled(a.v / s, 1.0 / s, a); }
Dual operator+(const Dual& a, double s) { Dual r(a); r.v += s; return r; }
Dual operator-(const Dual& a, double s) { Dual r(a); r.v -= s; return r; }
Dual operator-(double s, const Dual& a) { return scaled(s - a.v, -1.0, a); }
Dual dsqrt(const Dual& a) {
  double s = std::sqrt(a.v);
  return scaled(s, s > 0.0 ? 0.5 / s : 0.0, a);
}

Dual dsin(const Dual& a) { return scaled(std::sin(a.v), std::cos(a.v), a); }
Dual dcos(const Dual& a) { return scaled(std::cos(a.v), -std::sin(a.v), a); }
/* atan2(y, x) with d = (x dy - y dx) / (x^2 + y^2). */
Dual datan2(const Dual& y, const Dual& x) {
  double r2 = x.v * x.v + y.v * y.v;
  return lin(std::atan2(y.v, x.v), -y.v / r2, x, x.v / r2, y);
}

struct D3 { Dual x, y, z; };
D3 d3(double x, double y, double z) { return D3{Dual(x), Dual(y), Dual(z)}; }
/* The same tangents at another value (a rounded copy of the point). */
D3 at_value(const D3& a, const float v[3]) {
  D3 r = a;
  r.x.v = v[0];
  r.y.v = v[1];
  r.z.v = v[2];
  return r;
}
D3 operator+(const D3& a, const D3& b) { return D3{a.x + b.x, a.y + b.y, a.z + b.z}; }
D3 operator-(const D3& a, const D3& b) { return D3{a.x - b.x, a.y - b.y, a.z - b.z}; }
D3 operator*(const Dual& s, const D3& a) { return D3{s * a.x, s * a.y, s * a.z}; }
D3 operator*(double s, const D3& a) { return D3{s * a.x, s * a.y, s * a.z}; }
D3 operator/(const D3& a, const Dual& s) { return D3{a.x / s, a.y / s, a.z / s}; }
Dual dot(const D3& a, const D3& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
D3 cross(const D3& a, const D3& b) {
  return D3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
Dual length(const D3& a) { return dsqrt(dot(a, a)); }

/* Plain FP64 3-vectors for values that are never differentiated. */
struct V3 { double x, y, z; };
V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
double vdot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 vcross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double vlen(V3 a) { return std::sqrt(vdot(a, a)); }
V3 val(const D3& a) { return {a.x.v, a.y.v, a.z.v}; }

/* ------------------------------------------------------------------------ */
/* Scene and options as passed in from Python (all host memory).            */
/* ------------------------------------------------------------------------ */
}  // namespace

extern "C" {
typedef struct {
  int32_t n_verts, n_tris, n_light_tris, cam_type, width, height;
  const float* verts;        /* [V,3] */
  const int32_t* tris;       /* [T,3] */
  const float* albedo;       /* [T,3] */
  const int32_t* light_tris; /* [n_light_tris] indices into tris */
  const float* radiance;     /* [3] */
  const float* cam_to_world; /* [16] row-major; row 3 is (0,0,0,1) */
  float cam_scale;           /* pinhole: tan(fov_y/2); ortho: half height of the view */
} or_scene_t;

typedef struct {
  int32_t spp, edge_spp, max_depth, primary_only;
  uint64_t seed;
  float eps_rel;             /* edge side offset, relative to max(W,H) pixels / |omega| */
  int32_t terms;             /* bit0 interior, bit1 primary edges, bit2 secondary edges */
  int32_t pix_begin, pix_end;    /* interior pixel subset [begin,end); end<=0: all */
  int64_t edge_begin, edge_end;  /* primary edge sample subset; end<=0: all */
  int32_t n_threads;
  int32_t scene_id;          /* counter word c3 */
  int32_t proposal;          /* 0: edge by clipped length; 1: tile segments by the mixture of length and seg_weights;
                                2: the same with seg_weights read as network scores */
  const float* seg_weights;  /* [n_seg_weights] nonnegative weight per segment (proposal 1) */
  int64_t n_seg_weights;
  int32_t sec_sampler;       /* secondary edge: 0 by 3D length (Sec. 5.2.2); 1 the edge hierarchy (Sec. 5.3.1) */
  int32_t sec_tree_samples;  /* samples distributed from the hierarchy's root */
  int32_t sec_point;         /* point on a secondary edge: 0 uniform (Sec. 5.2.2); 1 the clamped-cosine
                                density over the edge's arc mixed with uniform (Sec. 5.3.2) */
  int32_t n_jac;             /* 0..8 parameters of the per-pixel gradient image */
  int64_t jac_param[8];      /* their flat indices in the gradient layout */
  int32_t aov;               /* with primary_only: 0, 1 albedo; 2 world position; 3 unit shading normal
                                (facing the ray); 4 distance from the ray origin (Sec. 5.4, geometry
                                buffers) */
  int32_t sec_nee;           /* 1: next-event estimation for edges (Sec. 5.3.3) beside the length sampler */
  float nee_width;           /* billboard width; <= 0: from the vertices' mean absolute deviation */
} or_opts_t;
}

namespace {

constexpr float NEAR_Z = 1e-4f;          /* camera-space depth below which a vertex is behind */
constexpr float SHADOW_TMAX = 0.9999f;   /* shadow rays stop short of the light point */
constexpr double INV_PI = 0.31830988618379067;

/* ---- FP32 decision-path primitives (fixed operation order) ------------- */

struct R32 { float o[3], d[3]; };

void sincos_2pi32(float r, float* c_out, float* s_out);

/* atan2(y, x) for y >= 0, in [0, pi], FP32 in a fixed order (no library
 * call, so both implementations take the same value): the ratio of the
 * smaller to the larger magnitude in [0, 1]; above tan(pi/12) it is reduced
 * by atan(a) = pi/6 + atan((sqrt(3) a - 1) / (a + sqrt(3))); then the Taylor
 * series of atan about 0 to z^13 by Horner's rule (|z| <= tan(pi/12), so the
 * first omitted term is below 2e-10); then the octant is restored. */
float atan2_pos32(float y, float x) {
  float ax = std::fabs(x);
  bool swap = y > ax;
  float num = swap ? ax : y, den = swap ? y : ax;
  float a = den > 0.0f ? num / den : 0.0f;
  bool red = a > 0.267949194f;
  float z = red ? (a * 1.73205078f - 1.0f) / (a + 1.73205078f) : a;
  float z2 = z * z;
  float p = 0.0769230798f;
  p = z2 * p + -0.0909090936f;
  p = z2 * p + 0.111111112f;
  p = z2 * p + -0.142857149f;
  p = z2 * p + 0.200000003f;
  p = z2 * p + -0.333333343f;
  float r = z + (z * z2) * p;
  if (red) r = 0.523598790f + r;
  if (swap) r = 1.57079637f - r;
  if (x < 0.0f) r = 3.14159274f - r;
  return r;
}

/* Camera ray through screen point (sx, sy) in pixel units, y down.  Sec. 5.2.1
 * restricts its screen-space edge sampling to cameras whose projection maps
 * lines to lines: pinhole (looks down -z, y up) and orthographic (spans
 * [-aspect*s, aspect*s] x [-s, s] in camera xy).  The equidistant fisheye
 * (cam_type 2, Sec. 5.2 "Cameras with Non-linear Projections") maps the
 * screen point at distance r from the centre (in units of half the image
 * height) to the direction at angle theta = r s from the optical axis (-z),
 * in the azimuth of the screen point; its edges are sampled in 3D. */
R32 camera_ray32(const or_scene_t& sc, float sx, float sy) {
  const float* M = sc.cam_to_world;
  float fw = (float)sc.width, fh = (float)sc.height;
  float xn = (2.0f * sx - fw) / fw;
  float yn = (fh - 2.0f * sy) / fh;
  float aspect = fw / fh;
  if (sc.cam_type == 2) {
    float a = xn * aspect, b = yn;
    float r = std::sqrt(a * a + b * b);
    float th = r * sc.cam_scale;
    float c, sn;
    sincos_2pi32(th * 0.159154937f, &c, &sn);
    float k = r > 0.0f ? sn / r : 0.0f;
    float dc[3] = {a * k, b * k, -c};
    R32 r32;
    for (int i = 0; i < 3; ++i) {
      r32.o[i] = M[4 * i + 3];
      r32.d[i] = (M[4 * i + 0] * dc[0] + M[4 * i + 1] * dc[1]) + M[4 * i + 2] * dc[2];
    }
    return r32;
  }
  float sxs = aspect * sc.cam_scale;
  float lx = xn * sxs;
  float ly = yn * sc.cam_scale;
  R32 r;
  for (int i = 0; i < 3; ++i) {
    if (sc.cam_type == 1) {
      r.o[i] = M[4 * i + 3];
      r.d[i] = (M[4 * i + 0] * lx + M[4 * i + 1] * ly) - M[4 * i + 2];
    } else {
      r.o[i] = (M[4 * i + 0] * lx + M[4 * i + 1] * ly) + M[4 * i + 3];
      r.d[i] = -M[4 * i + 2];
    }
  }
  return r;
}

/* Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2013), FP32, no FP64
 * fallback.  Returns true on a hit with t in (0, tmax); t, b1, b2 out. */
struct Shear { int kx, ky, kz; float Sx, Sy, Sz; };
Shear make_shear(const float d[3]) {
  int kz = 0;
  if (std::fabs(d[1]) > std::fabs(d[kz])) kz = 1;
  if (std::fabs(d[2]) > std::fabs(d[kz])) kz = 2;
  int kx = kz + 1; if (kx == 3) kx = 0;
  int ky = kx + 1; if (ky == 3) ky = 0;
  if (d[kz] < 0.0f) std::swap(kx, ky);
  Shear s;
  s.kx = kx; s.ky = ky; s.kz = kz;
  s.Sx = d[kx] / d[kz]; s.Sy = d[ky] / d[kz]; s.Sz = 1.0f / d[kz];
  return s;
}
bool watertight(const Shear& s, const float o[3], const float* v0, const float* v1, const float* v2,
                float tmax, float* t_out, float* b1_out, float* b2_out) {
  float A[3], B[3], C[3];
  for (int i = 0; i < 3; ++i) { A[i] = v0[i] - o[i]; B[i] = v1[i] - o[i]; C[i] = v2[i] - o[i]; }
  float Ax = A[s.kx] - s.Sx * A[s.kz], Ay = A[s.ky] - s.Sy * A[s.kz];
  float Bx = B[s.kx] - s.Sx * B[s.kz], By = B[s.ky] - s.Sy * B[s.kz];
  float Cx = C[s.kx] - s.Sx * C[s.kz], Cy = C[s.ky] - s.Sy * C[s.kz];
  float U = Cx * By - Cy * Bx;
  float V = Ax * Cy - Ay * Cx;
  float W = Bx * Ay - By * Ax;
  if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
  float det = (U + V) + W;
  if (det == 0.0f) return false;
  float Az = s.Sz * A[s.kz], Bz = s.Sz * B[s.kz], Cz = s.Sz * C[s.kz];
  float T = (U * Az + V * Bz) + W * Cz;
  float t = T / det;
  if (!(t > 0.0f && t < tmax)) return false;
  *t_out = t; *b1_out = V / det; *b2_out = W / det;
  return true;
}

/* FP32 face data and barycentric point (p = b0 v0 + b1 v1 + b2 v2, b0=(1-b1)-b2). */
void bary_point32(const float* v0, const float* v1, const float* v2, float b1, float b2, float p[3]) {
  float b0 = (1.0f - b1) - b2;
  for (int i = 0; i < 3; ++i) p[i] = (b0 * v0[i] + b1 * v1[i]) + b2 * v2[i];
}
void face_normal32(const float* v0, const float* v1, const float* v2, float n[3]) {
  float e1[3], e2[3];
  for (int i = 0; i < 3; ++i) { e1[i] = v1[i] - v0[i]; e2[i] = v2[i] - v0[i]; }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
}
float dot32(const float a[3], const float b[3]) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

/* Own sin/cos of 2*pi*r for r in [0,1): quadrant from 4r (exact), then the
 * Taylor series of sin and cos about 0 on [0, pi/2) by Horner's rule. */
void sincos_2pi32(float r, float* c_out, float* s_out) {
  float q4 = r * 4.0f;
  int q = (int)q4;
  if (q > 3) q = 3;
  float f = q4 - (float)q;
  float a = f * 1.57079637f;
  float a2 = a * a;
  float s = a2 * 1.60590444e-10f;
  s = a2 * (s - 2.50521084e-08f);
  s = a2 * (s + 2.75573192e-06f);
  s = a2 * (s - 1.98412698e-04f);
  s = a2 * (s + 8.33333377e-03f);
  s = a2 * (s - 1.66666672e-01f);
  s = a + a * s;
  float c = a2 * (-1.14707454e-11f);
  c = a2 * (c + 2.08767570e-09f);
  c = a2 * (c - 2.75573192e-07f);
  c = a2 * (c + 2.48015876e-05f);
  c = a2 * (c - 1.38888892e-03f);
  c = a2 * (c + 4.16666679e-02f);
  c = a2 * (c - 0.5f);
  c = 1.0f + c;
  switch (q) {
    case 0: *c_out = c; *s_out = s; break;
    case 1: *c_out = -s; *s_out = c; break;
    case 2: *c_out = -c; *s_out = -s; break;
    default: *c_out = s; *s_out = -c; break;
  }
}

/* Cosine-weighted hemisphere direction around unit normal n (FP32), with the
 * orthonormal basis of Duff et al., "Building an Orthonormal Basis,
 * Revisited", JCGT 2017. */
void cosine_dir32(const float n[3], float r1, float r2, float out[3]) {
  float rr = std::sqrt(r1);
  float c, s;
  sincos_2pi32(r2, &c, &s);
  float lx = rr * c, ly = rr * s;
  float lz = std::sqrt(std::max(0.0f, 1.0f - r1));
  float sgn = std::copysign(1.0f, n[2]);
  float a = -1.0f / (sgn + n[2]);
  float bb = (n[0] * n[1]) * a;
  float t[3] = {1.0f + ((sgn * n[0]) * n[0]) * a, sgn * bb, -(sgn * n[0])};
  float bt[3] = {bb, sgn + (n[1] * n[1]) * a, -n[1]};
  for (int i = 0; i < 3; ++i) out[i] = (lx * t[i] + ly * bt[i]) + lz * n[i];
}

/* ------------------------------------------------------------------------ */
/* Scene preparation.                                                        */
/* ------------------------------------------------------------------------ */
struct Prep {
  const or_scene_t* sc;
  int V, T, P;
  int pV, pA, pR, pC, pS;  /* parameter offsets: verts, albedo, radiance, camera(12), scale */
  float w2c[12];           /* world-to-camera rows (FP64 inverse, rounded once) */
  std::vector<int> light_of_tri;   /* -1 or index into light list */
  std::vector<double> light_cdf;   /* inclusive prefix of light-triangle areas */
  std::vector<double> light_area;
  double light_total = 0.0;
  /* unique undirected edges, sorted by (min vertex, max vertex) */
  std::vector<int32_t> e0, e1;
  /* primary edges: projected endpoints, clip interval, CDF */
  std::vector<float> pax, pay, pbx, pby, pt0, pt1;
  std::vector<double> pcdf; double ptotal = 0.0;
  /* secondary edges: 3D length CDF */
  std::vector<double> scdf; double stotal = 0.0;
  /* screen-tile segments of the clipped primary edges (learned proposal) */
  std::vector<int32_t> seg_edge, seg_tile;
  std::vector<float> seg_s0, seg_s1;
  std::vector<double> seg_len;
  std::vector<double> seg_cdf; double seg_total = 0.0;
};

constexpr float TILE = 16.0f;  /* screen tile size of the segment split, pixels */

const float* vtx(const Prep& P, int i) { return P.sc->verts + 3 * i; }

/* FP64 inverse of the camera's affine 3x4 (adjugate / determinant, in this
 * order), each entry rounded once to FP32. */
void world_to_cam64(const float* M, double out[12]) {
  double R[3][3], t[3];
  for (int i = 0; i < 3; ++i) { for (int j = 0; j < 3; ++j) R[i][j] = M[4 * i + j]; t[i] = M[4 * i + 3]; }
  double c00 = R[1][1] * R[2][2] - R[1][2] * R[2][1];
  double c01 = R[1][2] * R[2][0] - R[1][0] * R[2][2];
  double c02 = R[1][0] * R[2][1] - R[1][1] * R[2][0];
  double det = (R[0][0] * c00 + R[0][1] * c01) + R[0][2] * c02;
  double inv[3][3];
  inv[0][0] = c00 / det;
  inv[0][1] = (R[0][2] * R[2][1] - R[0][1] * R[2][2]) / det;
  inv[0][2] = (R[0][1] * R[1][2] - R[0][2] * R[1][1]) / det;
  inv[1][0] = c01 / det;
  inv[1][1] = (R[0][0] * R[2][2] - R[0][2] * R[2][0]) / det;
  inv[1][2] = (R[0][2] * R[1][0] - R[0][0] * R[1][2]) / det;
  inv[2][0] = c02 / det;
  inv[2][1] = (R[0][1] * R[2][0] - R[0][0] * R[2][1]) / det;
  inv[2][2] = (R[0][0] * R[1][1] - R[0][1] * R[1][0]) / det;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) out[4 * i + j] = inv[i][j];
    out[4 * i + 3] = -((inv[i][0] * t[0] + inv[i][1] * t[1]) + inv[i][2] * t[2]);
  }
}

/* Projection of a world point to screen pixels (FP32).  Returns false when
 * the point is not in front of the camera plane (camera z >= -NEAR_Z). */
bool project32(const Prep& P, const float v[3], float* sx, float* sy) {
  const float* W = P.w2c;
  float vc[3];
  for (int i = 0; i < 3; ++i) vc[i] = ((W[4 * i + 0] * v[0] + W[4 * i + 1] * v[1]) + W[4 * i + 2] * v[2]) + W[4 * i + 3];
  if (!(vc[2] < -NEAR_Z)) return false;
  const or_scene_t& sc = *P.sc;
  float fw = (float)sc.width, fh = (float)sc.height;
  float aspect = fw / fh;
  float px = vc[0], py = vc[1];
  if (sc.cam_type == 1) { float iz = -vc[2]; px = vc[0] / iz; py = vc[1] / iz; }
  float xn = px / (aspect * sc.cam_scale);
  float yn = py / sc.cam_scale;
  *sx = (xn + 1.0f) * (0.5f * fw);
  *sy = (1.0f - yn) * (0.5f * fh);
  return true;
}

/* Equidistant fisheye projection of a world point to screen pixels (FP32,
 * the inverse of camera_ray32 for cam_type 2).  False near the direction
 * opposite the optical axis (theta >= 3.1), which no pixel sees. */
bool fisheye_project32(const Prep& P, const float v[3], float* sx, float* sy) {
  const float* W = P.w2c;
  float vc[3];
  for (int i = 0; i < 3; ++i) vc[i] = ((W[4 * i + 0] * v[0] + W[4 * i + 1] * v[1]) + W[4 * i + 2] * v[2]) + W[4 * i + 3];
  const or_scene_t& sc = *P.sc;
  float rho = std::sqrt(vc[0] * vc[0] + vc[1] * vc[1]);
  float th = atan2_pos32(rho, -vc[2]);
  if (!(th < 3.1f)) return false;
  float k = rho > 0.0f ? th / (sc.cam_scale * rho) : 0.0f;
  float a = k * vc[0], b = k * vc[1];
  float fw = (float)sc.width, fh = (float)sc.height;
  float xn = a / (fw / fh);
  *sx = (xn + 1.0f) * (0.5f * fw);
  *sy = (1.0f - b) * (0.5f * fh);
  return true;
}

/* Liang-Barsky clip of a + t(b-a) to [0,W]x[0,H] (FP32, planes in the order
 * x>=0, x<=W, y>=0, y<=H).  Returns false when nothing is left. */
bool clip32(float ax, float ay, float bx, float by, float W, float H, float* t0o, float* t1o) {
  float dx = bx - ax, dy = by - ay;
  float t0 = 0.0f, t1 = 1.0f;
  float p[4] = {-dx, dx, -dy, dy};
  float q[4] = {ax, W - ax, ay, H - ay};
  for (int k = 0; k < 4; ++k) {
    if (p[k] == 0.0f) { if (q[k] < 0.0f) return false; continue; }
    float r = q[k] / p[k];
    if (p[k] < 0.0f) { if (r > t0) t0 = r; } else { if (r < t1) t1 = r; }
  }
  if (!(t0 < t1)) return false;
  *t0o = t0; *t1o = t1;
  return true;
}

/* Index of the first CDF entry strictly greater than target (upper bound);
 * if rounding leaves none, the last entry with positive mass. */
int cdf_pick(const std::vector<double>& cdf, double target) {
  int lo = 0, hi = (int)cdf.size();
  while (lo < hi) { int mid = (lo + hi) / 2; if (cdf[mid] > target) hi = mid; else lo = mid + 1; }
  if (lo >= (int)cdf.size()) {
    lo = (int)cdf.size() - 1;
    while (lo > 0 && cdf[lo] == cdf[lo - 1]) --lo;
  }
  return lo;
}

void prepare(const or_scene_t* sc, Prep& P) {
  P.sc = sc;
  P.V = sc->n_verts; P.T = sc->n_tris;
  P.pV = 0; P.pA = 3 * P.V; P.pR = P.pA + 3 * P.T; P.pC = P.pR + 3; P.pS = P.pC + 12;
  P.P = P.pS + 1;
  double w[12];
  world_to_cam64(sc->cam_to_world, w);
  for (int i = 0; i < 12; ++i) P.w2c[i] = (float)w[i];
  /* lights: FP64 areas from FP32 edge vectors, inclusive prefix in list order */
  P.light_of_tri.assign(P.T, -1);
  double acc = 0.0;
  for (int j = 0; j < sc->n_light_tris; ++j) {
    int t = sc->light_tris[j];
    P.light_of_tri[t] = j;
    const float *a = vtx(P, sc->tris[3 * t]), *b = vtx(P, sc->tris[3 * t + 1]), *c = vtx(P, sc->tris[3 * t + 2]);
    float e1[3], e2[3];
    for (int i = 0; i < 3; ++i) { e1[i] = b[i] - a[i]; e2[i] = c[i] - a[i]; }
    V3 E1{e1[0], e1[1], e1[2]}, E2{e2[0], e2[1], e2[2]};
    double area = 0.5 * vlen(vcross(E1, E2));
    P.light_area.push_back(area);
    acc += area;
    P.light_cdf.push_back(acc);
  }
  P.light_total = acc;
  /* unique undirected edges sorted by (min, max) */
  std::vector<uint64_t> keys;
  keys.reserve(3 * (size_t)P.T);
  for (int t = 0; t < P.T; ++t)
    for (int k = 0; k < 3; ++k) {
      uint32_t a = (uint32_t)sc->tris[3 * t + k], b = (uint32_t)sc->tris[3 * t + (k + 1) % 3];
      uint32_t lo = std::min(a, b), hi = std::max(a, b);
      keys.push_back(((uint64_t)lo << 32) | hi);
    }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  for (uint64_t k : keys) { P.e0.push_back((int32_t)(k >> 32)); P.e1.push_back((int32_t)(k & 0xffffffffu)); }
  int E = (int)keys.size();
  /* primary edges (Sec. 5.2.1: project, clip to the view, CDF of screen lengths) */
  P.pax.assign(E, 0); P.pay.assign(E, 0); P.pbx.assign(E, 0); P.pby.assign(E, 0);
  P.pt0.assign(E, 0); P.pt1.assign(E, 0); P.pcdf.assign(E, 0);
  acc = 0.0;
  for (int e = 0; e < E; ++e) {
    float ax, ay, bx, by, t0, t1;
    double len = 0.0;
    if (sc->cam_type == 2) {
      /* fisheye: edges are sampled in 3D, by the chord between the unit
       * directions from the camera to their end points (FP64) */
      const float *va = vtx(P, P.e0[e]), *vb = vtx(P, P.e1[e]);
      const float* M = sc->cam_to_world;
      double da_[3], db_[3];
      for (int i = 0; i < 3; ++i) { da_[i] = (double)va[i] - (double)M[4 * i + 3]; db_[i] = (double)vb[i] - (double)M[4 * i + 3]; }
      double la = std::sqrt((da_[0] * da_[0] + da_[1] * da_[1]) + da_[2] * da_[2]);
      double lb = std::sqrt((db_[0] * db_[0] + db_[1] * db_[1]) + db_[2] * db_[2]);
      if (la > 0.0 && lb > 0.0) {
        double u[3];
        for (int i = 0; i < 3; ++i) u[i] = da_[i] / la - db_[i] / lb;
        len = std::sqrt((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2]);
      }
    } else if (project32(P, vtx(P, P.e0[e]), &ax, &ay) && project32(P, vtx(P, P.e1[e]), &bx, &by) &&
        clip32(ax, ay, bx, by, (float)sc->width, (float)sc->height, &t0, &t1)) {
      P.pax[e] = ax; P.pay[e] = ay; P.pbx[e] = bx; P.pby[e] = by; P.pt0[e] = t0; P.pt1[e] = t1;
      float dx = bx - ax, dy = by - ay;
      len = ((double)t1 - (double)t0) * std::sqrt((double)dx * (double)dx + (double)dy * (double)dy);
    }
    acc += len;
    P.pcdf[e] = acc;
  }
  P.ptotal = acc;
  /* secondary edges: 3D length CDF over all edges */
  P.scdf.assign(E, 0);
  acc = 0.0;
  for (int e = 0; e < E; ++e) {
    const float *a = vtx(P, P.e0[e]), *b = vtx(P, P.e1[e]);
    float ex = b[0] - a[0], ey = b[1] - a[1], ez = b[2] - a[2];
    acc += std::sqrt((double)ex * ex + (double)ey * ey + (double)ez * ez);
    P.scdf[e] = acc;
  }
  P.stotal = acc;
  /* tile segments: split each clipped edge where it crosses the 16-pixel
   * tile grid (FP32 crossing parameters, merged in increasing t) */
  int tiles_x = (int)std::ceil(sc->width / TILE), tiles_y = (int)std::ceil(sc->height / TILE);
  for (int e = 0; e < E; ++e) {
    double le = P.pcdf[e] - (e > 0 ? P.pcdf[e - 1] : 0.0);
    if (!(le > 0.0) || sc->cam_type == 2) continue;  /* no screen segments for the fisheye */
    float ax = P.pax[e], ay = P.pay[e], t0 = P.pt0[e], t1 = P.pt1[e];
    float dx = P.pbx[e] - ax, dy = P.pby[e] - ay;
    std::vector<float> ts[2];
    for (int axis = 0; axis < 2; ++axis) {
      float a = axis == 0 ? ax : ay, d = axis == 0 ? dx : dy;
      if (d == 0.0f) continue;
      float c0 = a + t0 * d, c1 = a + t1 * d;
      float lo = std::min(c0, c1), hi = std::max(c0, c1);
      int m0 = (int)std::floor(lo / TILE) + 1, m1 = (int)std::floor(hi / TILE);
      for (int m = m0; m <= m1; ++m) {
        float t = ((float)m * TILE - a) / d;
        if (t > t0 && t < t1) ts[axis].push_back(t);
      }
      if (d < 0.0f) std::reverse(ts[axis].begin(), ts[axis].end());
    }
    std::vector<float> cuts;
    cuts.push_back(t0);
    size_t i = 0, j = 0;
    while (i < ts[0].size() || j < ts[1].size()) {
      float v;
      if (j >= ts[1].size() || (i < ts[0].size() && ts[0][i] <= ts[1][j])) v = ts[0][i++]; else v = ts[1][j++];
      if (v > cuts.back()) cuts.push_back(v);
    }
    if (t1 > cuts.back()) cuts.push_back(t1);
    double dl = std::sqrt((double)dx * (double)dx + (double)dy * (double)dy);
    for (size_t k = 0; k + 1 < cuts.size(); ++k) {
      float s0 = cuts[k], s1 = cuts[k + 1];
      float mid = s0 + 0.5f * (s1 - s0);
      float xm = ax + mid * dx, ym = ay + mid * dy;
      int tx = std::min(std::max((int)std::floor(xm / TILE), 0), tiles_x - 1);
      int ty = std::min(std::max((int)std::floor(ym / TILE), 0), tiles_y - 1);
      P.seg_edge.push_back(e);
      P.seg_tile.push_back(ty * tiles_x + tx);
      P.seg_s0.push_back(s0);
      P.seg_s1.push_back(s1);
      P.seg_len.push_back(((double)s1 - (double)s0) * dl);
    }
  }
}

/* Mixture proposal over segments: q = 1/2 len/L + 1/2 m/M (q = len/L when
 * every weight is zero); inclusive FP64 prefix of q in P.seg_cdf.
 * mode 1: m_k = max(0, w_k);  mode 2 (network scores s_k, a log density per
 * unit length): m_k = len_k * exp(min(max(s_k, -40), 40)), in FP64. */
void build_proposal(Prep& P, const float* w, int64_t n, int mode) {
  size_t ns = P.seg_len.size();
  std::vector<double> m(ns, 0.0);
  double L = 0.0, M = 0.0;
  for (size_t k = 0; k < ns; ++k) {
    L += P.seg_len[k];
    if ((int64_t)k < n) {
      if (mode == 2) m[k] = P.seg_len[k] * std::exp(std::min(std::max((double)w[k], -40.0), 40.0));
      else m[k] = (double)std::max(0.0f, w[k]);
    }
    M += m[k];
  }
  P.seg_cdf.assign(ns, 0.0);
  double acc = 0.0;
  for (size_t k = 0; k < ns; ++k) {
    double q = P.seg_len[k] / L;
    if (M > 0.0) q = 0.5 * q + 0.5 * m[k] / M;
    acc += q;
    P.seg_cdf[k] = acc;
  }
  P.seg_total = acc;
}

/* ---- brute-force visibility queries (all triangles, index order) -------- */
struct Hit { int tri = -1; float t = 0, b1 = 0, b2 = 0; };

Hit closest(const Prep& P, const float o[3], const float d[3], int exclude) {
  Shear s = make_shear(d);
  Hit h;
  float best = INFINITY;
  const or_scene_t& sc = *P.sc;
  for (int t = 0; t < P.T; ++t) {
    if (t == exclude) continue;
    float tt, b1, b2;
    if (watertight(s, o, vtx(P, sc.tris[3 * t]), vtx(P, sc.tris[3 * t + 1]), vtx(P, sc.tris[3 * t + 2]), best, &tt, &b1, &b2)) {
      best = tt; h.tri = t; h.t = tt; h.b1 = b1; h.b2 = b2;
    }
  }
  return h;
}
bool occluded(const Prep& P, const float o[3], const float d[3], float tmax, int ex0, int ex1) {
  Shear s = make_shear(d);
  const or_scene_t& sc = *P.sc;
  for (int t = 0; t < P.T; ++t) {
    if (t == ex0 || t == ex1) continue;
    float tt, b1, b2;
    if (watertight(s, o, vtx(P, sc.tris[3 * t]), vtx(P, sc.tris[3 * t + 1]), vtx(P, sc.tris[3 * t + 2]), tmax, &tt, &b1, &b2))
      return true;
  }
  return false;
}

/* ------------------------------------------------------------------------ */
/* Differentiable quantities (FP64 duals).                                   */
/* ------------------------------------------------------------------------ */
D3 vert_dual(const Prep& P, int i, bool track) {
  const float* v = vtx(P, i);
  return D3{Dual::param(v[0], P.pV + 3 * i, track), Dual::param(v[1], P.pV + 3 * i + 1, track),
            Dual::param(v[2], P.pV + 3 * i + 2, track)};
}
Dual cam_dual(const Prep& P, int r, int c, bool track) {
  return Dual::param(P.sc->cam_to_world[4 * r + c], P.pC + 4 * r + c, track);
}
Dual scale_dual(const Prep& P, bool track) { return Dual::param(P.sc->cam_scale, P.pS, track); }

/* Camera ray as a function of the camera parameters (same formulas as
 * camera_ray32, in FP64 duals). */
void camera_ray_dual(const Prep& P, float sx, float sy, bool track, D3* O, D3* D) {
  const or_scene_t& sc = *P.sc;
  double fw = sc.width, fh = sc.height;
  double xn = (2.0 * sx - fw) / fw, yn = (fh - 2.0 * sy) / fh;
  Dual S = scale_dual(P, track);
  if (sc.cam_type == 2) {
    double a = xn * (fw / fh), b = yn, r = std::sqrt(a * a + b * b);
    Dual th = r * S;
    Dual sn = dsin(th), cs = dcos(th);
    Dual dc[3] = {r > 0.0 ? (a / r) * sn : Dual(0.0), r > 0.0 ? (b / r) * sn : Dual(0.0), -cs};
    Dual Mo[3], Md[3];
    for (int i = 0; i < 3; ++i) {
      Dual m0 = cam_dual(P, i, 0, track), m1 = cam_dual(P, i, 1, track), m2 = cam_dual(P, i, 2, track),
           m3 = cam_dual(P, i, 3, track);
      Mo[i] = m3;
      Md[i] = m0 * dc[0] + m1 * dc[1] + m2 * dc[2];
    }
    *O = D3{Mo[0], Mo[1], Mo[2]};
    *D = D3{Md[0], Md[1], Md[2]};
    return;
  }
  Dual lx = (xn * (fw / fh)) * S, ly = yn * S;
  Dual Mo[3], Md[3];
  for (int i = 0; i < 3; ++i) {
    Dual m0 = cam_dual(P, i, 0, track), m1 = cam_dual(P, i, 1, track), m2 = cam_dual(P, i, 2, track),
         m3 = cam_dual(P, i, 3, track);
    if (sc.cam_type == 1) { Mo[i] = m3; Md[i] = m0 * lx + m1 * ly - m2; }
    else { Mo[i] = m0 * lx + m1 * ly + m3; Md[i] = -m2; }
  }
  *O = D3{Mo[0], Mo[1], Mo[2]};
  *D = D3{Md[0], Md[1], Md[2]};
}

/* Screen projection of a world point as a function of the point and the
 * camera (inverse of the camera matrix by adjugate, in duals). */
void project_dual(const Prep& P, const D3& v, bool track, Dual* sx, Dual* sy) {
  Dual R[3][3], t[3];
  for (int i = 0; i < 3; ++i) { for (int j = 0; j < 3; ++j) R[i][j] = cam_dual(P, i, j, track); t[i] = cam_dual(P, i, 3, track); }
  Dual c00 = R[1][1] * R[2][2] - R[1][2] * R[2][1];
  Dual c01 = R[1][2] * R[2][0] - R[1][0] * R[2][2];
  Dual c02 = R[1][0] * R[2][1] - R[1][1] * R[2][0];
  Dual det = R[0][0] * c00 + R[0][1] * c01 + R[0][2] * c02;
  Dual inv[3][3];
  inv[0][0] = c00 / det;
  inv[0][1] = (R[0][2] * R[2][1] - R[0][1] * R[2][2]) / det;
  inv[0][2] = (R[0][1] * R[1][2] - R[0][2] * R[1][1]) / det;
  inv[1][0] = c01 / det;
  inv[1][1] = (R[0][0] * R[2][2] - R[0][2] * R[2][0]) / det;
  inv[1][2] = (R[0][2] * R[1][0] - R[0][0] * R[1][2]) / det;
  inv[2][0] = c02 / det;
  inv[2][1] = (R[0][1] * R[2][0] - R[0][0] * R[2][1]) / det;
  inv[2][2] = (R[0][0] * R[1][1] - R[0][1] * R[1][0]) / det;
  D3 q{v.x - t[0], v.y - t[1], v.z - t[2]};
  Dual vc[3];
  for (int i = 0; i < 3; ++i) vc[i] = inv[i][0] * q.x + inv[i][1] * q.y + inv[i][2] * q.z;
  const or_scene_t& sc = *P.sc;
  double fw = sc.width, fh = sc.height;
  Dual S = scale_dual(P, track);
  Dual px = vc[0], py = vc[1];
  if (sc.cam_type == 1) { Dual iz = -vc[2]; px = vc[0] / iz; py = vc[1] / iz; }
  Dual xn = px / ((fw / fh) * S), yn = py / S;
  *sx = (xn + 1.0) * (0.5 * fw);
  *sy = (1.0 - yn) * (0.5 * fh);
}

/* Equidistant fisheye projection of a world point (duals; the smooth
 * counterpart of fisheye_project32). */
void project_fisheye_dual(const Prep& P, const D3& v, bool track, Dual* sx, Dual* sy) {
  Dual R[3][3], t[3];
  for (int i = 0; i < 3; ++i) { for (int j = 0; j < 3; ++j) R[i][j] = cam_dual(P, i, j, track); t[i] = cam_dual(P, i, 3, track); }
  Dual c00 = R[1][1] * R[2][2] - R[1][2] * R[2][1];
  Dual c01 = R[1][2] * R[2][0] - R[1][0] * R[2][2];
  Dual c02 = R[1][0] * R[2][1] - R[1][1] * R[2][0];
  Dual det = R[0][0] * c00 + R[0][1] * c01 + R[0][2] * c02;
  Dual inv[3][3];
  inv[0][0] = c00 / det;
  inv[0][1] = (R[0][2] * R[2][1] - R[0][1] * R[2][2]) / det;
  inv[0][2] = (R[0][1] * R[1][2] - R[0][2] * R[1][1]) / det;
  inv[1][0] = c01 / det;
  inv[1][1] = (R[0][0] * R[2][2] - R[0][2] * R[2][0]) / det;
  inv[1][2] = (R[0][2] * R[1][0] - R[0][0] * R[1][2]) / det;
  inv[2][0] = c02 / det;
  inv[2][1] = (R[0][1] * R[2][0] - R[0][0] * R[2][1]) / det;
  inv[2][2] = (R[0][0] * R[1][1] - R[0][1] * R[1][0]) / det;
  D3 q{v.x - t[0], v.y - t[1], v.z - t[2]};
  Dual vc[3];
  for (int i = 0; i < 3; ++i) vc[i] = inv[i][0] * q.x + inv[i][1] * q.y + inv[i][2] * q.z;
  const or_scene_t& sc = *P.sc;
  double fw = sc.width, fh = sc.height;
  Dual S = scale_dual(P, track);
  Dual rho = dsqrt(vc[0] * vc[0] + vc[1] * vc[1]);
  Dual th = datan2(rho, -vc[2]);
  Dual k = th / (S * rho);
  Dual a = k * vc[0], b = k * vc[1];
  *sx = (a / (fw / fh) + 1.0) * (0.5 * fw);
  *sy = (1.0 - b) * (0.5 * fh);
}

/* Ray/plane hit point of a fixed or moving ray with the (moving) triangle:
 * p = O + tau D, tau = ((v0 - O).N)/(D.N), N the unnormalised face normal. */
D3 hit_point_dual(const D3& O, const D3& D, const D3& V0, const D3& V1, const D3& V2) {
  D3 N = cross(V1 - V0, V2 - V0);
  Dual tau = dot(V0 - O, N) / dot(D, N);
  return O + tau * D;
}

#include "edge_tree.h"
#include "nee_edge.h"

struct Ctx {
  const Prep* P;
  const or_opts_t* opt;
  bool track;            /* accumulate derivatives */
  const float* w;        /* d_image [H,W,3] (backward) */
  double* g;             /* gradient accumulator [P] */
  double* ga;            /* sum of |contribution| per parameter [P] */
  const EdgeTree* tree = nullptr;  /* secondary edge hierarchy (sec_sampler 1) */
  double* gc = nullptr;  /* sum over accumulate calls of |coef x'| per parameter [P] (or null) */
  double* jac = nullptr; /* [n_jac, H, W] per-pixel share of the gradient (or null) */
  int64_t pix = 0;       /* pixel the current sample's contributions belong to */
  float nee_hw = 0.0f;   /* billboard half width of next-event estimation for edges (0: off) */
  const std::vector<int>* leaf_of_edge = nullptr;  /* edge id -> position in tree->leaf */
};

/* grad += coef * x';  tolerance scale += coef_abs * |x|' (see Dual).  Each
 * call adds one sample's contribution c_k (an interior path sample, a primary
 * edge sample, or a secondary edge sample); gc, if given, sums |c_k|. */
void accumulate(Ctx& C, double coef, double coef_abs, const Dual& x) {
  for (int i = 0; i < x.n; ++i) {
    C.g[x.idx[i]] += coef * x.d[i];
    C.ga[x.idx[i]] += coef_abs * x.ad[i];
    if (C.gc) C.gc[x.idx[i]] += std::fabs(coef * x.d[i]);
    if (C.jac)
      for (int k = 0; k < C.opt->n_jac; ++k)
        if (C.opt->jac_param[k] == x.idx[i])
          C.jac[(int64_t)k * C.P->sc->width * C.P->sc->height + C.pix] += coef * x.d[i];
  }
}

struct RGB { Dual c[3]; };

/* Triangle vertex data helpers. */
struct TriV { const float *v0, *v1, *v2; int i0, i1, i2; };
TriV tri_of(const Prep& P, int t) {
  const int32_t* id = P.sc->tris + 3 * t;
  return TriV{vtx(P, id[0]), vtx(P, id[1]), vtx(P, id[2]), id[0], id[1], id[2]};
}

/* Light point on light triangle j (Sec. 5.4 area lights): barycentric
 * (1-sqrt(r1), sqrt(r1) r2, sqrt(r1)(1-r2)), FP32 point, and its FP64 dual
 * with the barycentrics held fixed. */
void light_point(const Prep& P, int j, float r1, float r2, bool track, float y32[3], D3* Y, float bary[3]) {
  int lt = P.sc->light_tris[j];
  TriV L = tri_of(P, lt);
  float su = std::sqrt(r1);
  float b0 = 1.0f - su;
  float b1 = su * r2;
  float b2 = su - b1;
  for (int i = 0; i < 3; ++i) y32[i] = (b0 * L.v0[i] + b1 * L.v1[i]) + b2 * L.v2[i];
  bary[0] = b0; bary[1] = b1; bary[2] = b2;
  D3 A = vert_dual(P, L.i0, track), B = vert_dual(P, L.i1, track), Cc = vert_dual(P, L.i2, track);
  /* attachment weights summing to one in FP64, so the point moves rigidly */
  double w1 = b1, w2 = b2, w0 = 1.0 - w1 - w2;
  *Y = w0 * A + w1 * B + w2 * Cc;
}

/* ---- Secondary edge sample at a shading vertex (Sec. 5.2.2) -------------- */
/* Per side s the ray from p toward omega(t) +- eps |omega| n_h hits m_s.
 *  direct part (area measure on the lights, matching the area-sampled NEE):
 *     sign_s * h_s * |J_m(t)| / (|v0'xv1'| |n_m x n_h|) * d alpha(p, m_s)/d theta,
 *     alpha = (m-p).(v0-p)x(v1-p) with m attached to the light surface,
 *     J_m(t) = tau (e - omega (e.n_m)/(omega.n_m)), tau = ((m_s-p).n_m)/(omega.n_m),
 *     i.e. Appendix 5.A with m = p + tau omega;
 *  indirect part (solid-angle measure, matching cosine-sampled continuation):
 *     sign_s * f_r cos_p L_r,s / |omega|^2 * d alpha_dir/d theta,
 *     alpha_dir = omega_hat.(v0-p)x(v1-p) with omega_hat held fixed.
 * Everything is divided by P(E) = |E| / total length, or, with the edge
 * hierarchy (Sec. 5.3.1), multiplied by the pick's resampling weight.      */
/* Importance sampling of the point on a secondary edge (Sec. 5.3.2).  The
 * thesis integrates the BRDF over the edge as a linear light in the frame of a
 * fitted linearly transformed cosine and inverts the integral numerically.
 * For a Lambertian surface that distribution is the clamped cosine itself,
 * and its integral along the edge's arc (the edge seen from p as a piece of a
 * great circle) has a closed form with a closed-form inverse:
 *
 *   Let f be the unit vector from p to the foot of the perpendicular on the
 *   edge's line, e the edge direction, h the distance to the line and
 *   theta the angle from f toward e, so omega_hat = cos(theta) f + sin(theta) e
 *   and s = h tan(theta) along the line.  With n_p = n.f, n_e = n.e,
 *   rho = |(n_p, n_e)| and psi the angle of (n_p, n_e):
 *     n.omega_hat = rho cos(theta - psi),   d theta = h ds / r^2,
 *     G(theta) = n_p sin(theta) - n_e cos(theta) = rho sin(theta - psi)
 *   is an antiderivative of the cosine on its support, G = -rho and +rho at
 *   the support's ends.  A uniform y in [G(a), G(b)] gives sin(theta - psi) =
 *   y / rho, cos(theta - psi) = sqrt(1 - (y/rho)^2), hence cos(theta),
 *   sin(theta), s and t by rotation by psi: no angle is ever formed.
 *
 * The density in t is q_c(t) = (n.omega_hat)^+ h |E| / (r(t)^2 Z) with
 * Z = G(b) - G(a).  Mixed with uniform, q = 1/4 + 3/4 q_c, every point keeps a
 * positive density (also the sliver below the horizon that side rays offset
 * by eps can still reach).  The point t is an FP32 decision (fixed operation
 * order); q is evaluated in FP64 at that t.  Degenerate cases (the line
 * through p, n normal to the plane of p and the edge, an arc below the
 * horizon) keep t uniform with q = 1. */
struct EdgePoint {
  float t;
  double q;
};

EdgePoint edge_point_sample(const float p[3], const float n[3], const float v0[3], const float v1[3], float u,
                            float usel) {
  EdgePoint out{u, 1.0};
  float a0[3], E[3];
  for (int i = 0; i < 3; ++i) { a0[i] = v0[i] - p[i]; E[i] = v1[i] - v0[i]; }
  float N[3] = {a0[1] * E[2] - a0[2] * E[1], a0[2] * E[0] - a0[0] * E[2], a0[0] * E[1] - a0[1] * E[0]};
  float lE = std::sqrt(dot32(E, E)), nN = std::sqrt(dot32(N, N));
  if (!(lE > 0.0f) || !(nN > 0.0f)) return out;
  float h = nN / lE;
  float e[3] = {E[0] / lE, E[1] / lE, E[2] / lE};
  float k[3] = {e[1] * N[2] - e[2] * N[1], e[2] * N[0] - e[0] * N[2], e[0] * N[1] - e[1] * N[0]};
  float f[3] = {k[0] / nN, k[1] / nN, k[2] / nN};
  float s0 = dot32(a0, e), s1 = s0 + lE;
  float np = dot32(n, f), ne = dot32(n, e);
  float rho = std::sqrt(np * np + ne * ne);
  if (!(rho > 1e-6f)) return out;
  float r0 = std::sqrt(s0 * s0 + h * h), r1 = std::sqrt(s1 * s1 + h * h);
  float c0 = h / r0, g0 = s0 / r0, c1 = h / r1, g1 = s1 / r1;
  bool in0 = np * c0 + ne * g0 > 0.0f, in1 = np * c1 + ne * g1 > 0.0f;
  if (!in0 && !in1) return out;
  float Ga = in0 ? g0 * np - c0 * ne : -rho;
  float Gb = in1 ? g1 * np - c1 * ne : rho;
  float Z = Gb - Ga;
  if (!(Z > 1e-6f * rho)) return out;
  float t = u;
  if (!(usel < 0.25f)) {
    float Y = (Ga + u * Z) / rho;
    Y = std::min(std::max(Y, -1.0f), 1.0f);
    float C = std::sqrt(std::max(1.0f - Y * Y, 0.0f));
    float ct = (C * np - Y * ne) / rho;
    float st = (Y * np + C * ne) / rho;
    ct = std::max(ct, 1e-30f);
    float sl = (h * st) / ct;
    t = (sl - s0) / lE;
    t = std::min(std::max(t, 0.0f), 0.99999994f);
  }
  out.t = t;
  /* density at t, FP64 from the same FP32 inputs and clipping decisions */
  double A0[3], Ed[3];
  for (int i = 0; i < 3; ++i) { A0[i] = (double)v0[i] - p[i]; Ed[i] = (double)v1[i] - v0[i]; }
  V3 a0d{A0[0], A0[1], A0[2]}, Ev{Ed[0], Ed[1], Ed[2]}, nd{n[0], n[1], n[2]};
  V3 Nd = vcross(a0d, Ev);
  double lEd = vlen(Ev), nNd = vlen(Nd), hd = nNd / lEd;
  V3 ed = (1.0 / lEd) * Ev;
  V3 fd = (1.0 / nNd) * vcross(ed, Nd);
  double s0d = vdot(a0d, ed), s1d = s0d + lEd;
  double npd = vdot(nd, fd), ned = vdot(nd, ed), rhod = std::sqrt(npd * npd + ned * ned);
  double r0d = std::sqrt(s0d * s0d + hd * hd), r1d = std::sqrt(s1d * s1d + hd * hd);
  double Gad = in0 ? (s0d / r0d) * npd - (hd / r0d) * ned : -rhod;
  double Gbd = in1 ? (s1d / r1d) * npd - (hd / r1d) * ned : rhod;
  double Zd = Gbd - Gad;
  V3 w = a0d + (double)t * Ev;
  double r2 = vdot(w, w);
  double cw = vdot(nd, w) / std::sqrt(r2);
  double qc = cw > 0.0 ? cw * hd * lEd / (r2 * Zd) : 0.0;
  out.q = 0.25 + 0.75 * qc;
  return out;
}

void path_radiance(Ctx& C, int depth0, int max_depth, const float o32_in[3], const float d32_in[3],
                   const D3& O_in, const D3& D_in, int exclude_in, bool emission_first, uint32_t c0, uint32_t c1,
                   uint32_t pass, const double wscale[3], const double beta_in[3], bool backward, RGB* out);

void secondary_edge_eval(Ctx& C, int b, uint32_t c0, uint32_t c1, const float p32[3], const D3& Pd, V3 ns,
                         const float ns32[3], int k, const double albedo_k[3], const double beta[3],
                         const double wscale[3], int max_depth, int e, float t, double inv_pe,
                         uint32_t cont_pass);
void secondary_edge(Ctx& C, int b, uint32_t c0, uint32_t c1, uint32_t pass, const float p32[3], const D3& Pd,
                    V3 ns, const float ns32[3], int k, const double albedo_k[3], const double beta[3],
                    const double wscale[3], int max_depth) {
  const Prep& P = *C.P;
  if (P.stotal <= 0.0) return;
  uint32_t r[4];
  rng(C.opt->seed, c0, c1, K_EDGE_SECONDARY, (uint32_t)b, pass, (uint32_t)C.opt->scene_id, r);
  int e;
  double inv_pe;
  if (C.opt->sec_sampler == 1) {
    ETQuery q = et_query(*C.tree, p32, ns32, b + 1 >= max_depth, C.opt->eps_rel);
    float wgt;
    if (!et_pick(*C.tree, q, C.opt->sec_tree_samples, C.opt->seed, c0, c1, (uint32_t)b,
                 (uint32_t)C.opt->scene_id, &e, &wgt))
      return;
    inv_pe = (double)wgt;
  } else {
    e = cdf_pick(P.scdf, u01d(r[0], r[1]) * P.stotal);
    double le = P.scdf[e] - (e > 0 ? P.scdf[e - 1] : 0.0);
    if (le <= 0.0) return;
    inv_pe = P.stotal / le;
  }
  const float *v0 = vtx(P, P.e0[e]), *v1 = vtx(P, P.e1[e]);
  float t = u01f(r[2]);
  if (C.opt->sec_point == 1) {
    EdgePoint ep = edge_point_sample(p32, ns32, v0, v1, t, u01f(r[3]));
    t = ep.t;
    inv_pe = inv_pe / ep.q;
  }
  if (!(C.nee_hw > 0.0f)) {
    secondary_edge_eval(C, b, c0, c1, p32, Pd, ns, ns32, k, albedo_k, beta, wscale, max_depth, e, t, inv_pe,
                        PASS_SECONDARY_BASE + (uint32_t)b);
    return;
  }
  /* next-event estimation for edges (Sec. 5.3.3): the sample above and one
   * billboard sample, each weighed by the balance heuristic */
  const EdgeTree& T = *C.tree;
  const float hw = C.nee_hw;
  uint32_t rn[4];
  rng(C.opt->seed, c0, c1, K_EDGE_NEE, (uint32_t)b, pass, (uint32_t)C.opt->scene_id, rn);
  {
    float uA = hw * (2.0f * u01f(rn[0]) - 1.0f);
    int leaf = (*C.leaf_of_edge)[e];
    float d[3];
    double pB = 0.0;
    if (nee_ray(T.leaf[leaf], p32, t, uA, d)) pB = nee_density(P, T, p32, ns32, d, leaf, t, uA, hw);
    double pA = 1.0 / inv_pe;
    secondary_edge_eval(C, b, c0, c1, p32, Pd, ns, ns32, k, albedo_k, beta, wscale, max_depth, e, t,
                        1.0 / (pA + (2.0 * (double)hw) * pB), PASS_SECONDARY_BASE + (uint32_t)b);
  }
  if (!(P.light_total > 0.0)) return;
  /* the shadow ray of this vertex's next-event estimation, drawn again */
  uint32_t rl[4];
  rng(C.opt->seed, c0, c1, K_LIGHT, (uint32_t)b, pass, (uint32_t)C.opt->scene_id, rl);
  int j = cdf_pick(P.light_cdf, u01d(rl[0], rl[1]) * P.light_total);
  float y32[3], by[3];
  D3 Yunused;
  light_point(P, j, u01f(rl[2]), u01f(rl[3]), false, y32, &Yunused, by);
  float d[3] = {y32[0] - p32[0], y32[1] - p32[1], y32[2] - p32[2]};
  int lt = P.sc->light_tris[j];
  float Tj, tb1, tb2;
  if (!watertight(make_shear(d), p32, vtx(P, P.sc->tris[3 * lt]), vtx(P, P.sc->tris[3 * lt + 1]),
                  vtx(P, P.sc->tris[3 * lt + 2]), INFINITY, &Tj, &tb1, &tb2))
    return;
  std::vector<NeeCross> xs;
  nee_crossings(T, p32, ns32, d, Tj, hw, xs);
  int w = nee_race(T, xs, rn[2], rn[3]);
  if (w < 0) return;
  const NeeCross& x = xs[w];
  int eB = T.leaf[x.leaf].eid;
  double pB = nee_density(P, T, p32, ns32, d, x.leaf, x.t, x.u, hw);
  double le = P.scdf[eB] - (eB > 0 ? P.scdf[eB - 1] : 0.0);
  double pA = le / P.stotal;
  double den = pA + (2.0 * (double)hw) * pB;
  if (!(den > 0.0)) return;
  secondary_edge_eval(C, b, c0, c1, p32, Pd, ns, ns32, k, albedo_k, beta, wscale, max_depth, eB, x.t, 1.0 / den,
                      PASS_NEE_BASE + (uint32_t)b);
}

/* One secondary edge sample at edge e, parameter t, weighed by inv_pe (one
 * over its density); cont_pass: the pass of the side paths' continuation. */
void secondary_edge_eval(Ctx& C, int b, uint32_t c0, uint32_t c1, const float p32[3], const D3& Pd, V3 ns,
                         const float ns32[3], int k, const double albedo_k[3], const double beta[3],
                         const double wscale[3], int max_depth, int e, float t, double inv_pe,
                         uint32_t cont_pass) {
  const Prep& P = *C.P;
  const float *v0 = vtx(P, P.e0[e]), *v1 = vtx(P, P.e1[e]);
  float om[3], a0[3], a1[3];
  for (int i = 0; i < 3; ++i) {
    float ei = v1[i] - v0[i];
    om[i] = (v0[i] + t * ei) - p32[i];
    a0[i] = v0[i] - p32[i];
    a1[i] = v1[i] - p32[i];
  }
  float N32[3] = {a0[1] * a1[2] - a0[2] * a1[1], a0[2] * a1[0] - a0[0] * a1[2], a0[0] * a1[1] - a0[1] * a1[0]};
  float nlen = std::sqrt(dot32(N32, N32));
  if (!(nlen > 0.0f)) return;
  float nh32[3] = {N32[0] / nlen, N32[1] / nlen, N32[2] / nlen};
  float wl = std::sqrt(dot32(om, om));
  float sh = C.opt->eps_rel * wl;
  float du[3], dl[3];
  for (int i = 0; i < 3; ++i) { du[i] = om[i] + sh * nh32[i]; dl[i] = om[i] - sh * nh32[i]; }
  /* FP64 geometry of the sample for the weights */
  V3 p{p32[0], p32[1], p32[2]};
  V3 E{(double)v1[0] - v0[0], (double)v1[1] - v0[1], (double)v1[2] - v0[2]};
  V3 w{(double)v0[0] + t * E.x - p.x, (double)v0[1] + t * E.y - p.y, (double)v0[2] + t * E.z - p.z};
  V3 N = vcross(V3{v0[0] - p.x, v0[1] - p.y, v0[2] - p.z}, V3{v1[0] - p.x, v1[1] - p.y, v1[2] - p.z});
  double Nl = vlen(N);
  if (!(Nl > 0.0)) return;
  V3 nh = (1.0 / Nl) * N;
  double wl2 = vdot(w, w);
  V3 what = (1.0 / std::sqrt(wl2)) * w;
  D3 V0d = vert_dual(P, P.e0[e], C.track), V1d = vert_dual(P, P.e1[e], C.track);
  /* alpha and its derivatives are evaluated at the FP32 points the sample
   * uses (p32, and m32 below), the points the side rays leave from and hit;
   * the tangents are those of the exact hit points */
  D3 Ps = at_value(Pd, p32);
  D3 A0 = V0d - Ps, A1 = V1d - Ps;
  D3 Nd = cross(A0, A1);
  const float* Le = P.sc->radiance;
  /* both side rays first: which sides count */
  bool ok[2] = {false, false};
  Hit hs_[2];
  for (int side = 0; side < 2; ++side) {
    const float* ds = side == 0 ? du : dl;
    /* a side leaving below the shading horizon by more than 1e-5 |omega| is
     * not traced (FP32 decision, fixed order) */
    if (dot32(ns32, ds) < -1e-5f * wl) continue;
    Hit h = closest(P, p32, ds, k);
    if (h.tri < 0) continue;
    TriV M = tri_of(P, h.tri);
    float m32[3];
    bary_point32(M.v0, M.v1, M.v2, h.b1, h.b2, m32);
    float dm32[3] = {m32[0] - p32[0], m32[1] - p32[1], m32[2] - p32[2]};
    /* the hit must lie above the shading horizon (FP32 decision from the hit) */
    if (!(dot32(ns32, dm32) > 0.0f)) continue;
    ok[side] = true;
    hs_[side] = h;
  }
  /* Both sides on one triangle: the edge separates no surfaces at this point,
   * so the jump h_u - h_l of Eq. dirac_3d_edge is zero there; the difference
   * of the two evaluations a finite offset apart would be an O(eps) residue */
  if (ok[0] && ok[1] && hs_[0].tri == hs_[1].tri) return;
  for (int side = 0; side < 2; ++side) {
    if (!ok[side]) continue;
    const float* ds = side == 0 ? du : dl;
    double sgn = side == 0 ? 1.0 : -1.0;
    Hit h = hs_[side];
    TriV M = tri_of(P, h.tri);
    float m32[3];
    bary_point32(M.v0, M.v1, M.v2, h.b1, h.b2, m32);
    float dm32[3] = {m32[0] - p32[0], m32[1] - p32[1], m32[2] - p32[2]};
    float nf32[3];
    face_normal32(M.v0, M.v1, M.v2, nf32);
    /* the direct part needs the light's front face toward p (FP32 decision) */
    bool front = dot32(nf32, dm32) < 0.0f;
    V3 m{m32[0], m32[1], m32[2]};
    V3 dm = m - p;
    double r2 = vdot(dm, dm), rr = std::sqrt(r2);
    V3 wh = (1.0 / rr) * dm;
    double cos_p = vdot(ns, wh);
    V3 nm = V3{0, 0, 0};
    {
      V3 nn{nf32[0], nf32[1], nf32[2]};
      nm = (1.0 / vlen(nn)) * nn;
    }
    /* direct part: m on a light, front face toward p */
    int lj = P.light_of_tri[h.tri];
    if (front && lj >= 0) {
      double cos_m = -vdot(nm, wh);
      {
        double G = cos_p * cos_m / r2;
        double wn = vdot(w, nm);
        double tau = vdot(dm, nm) / wn;
        V3 J = tau * (E - (vdot(E, nm) / wn) * w);
        double cr = vlen(vcross(nm, nh));
        double hs = 0.0, hs_abs = 0.0;
        for (int c = 0; c < 3; ++c) {
          hs += wscale[c] * beta[c] * albedo_k[c] * INV_PI * Le[c] * G;
          hs_abs += std::fabs(wscale[c]) * beta[c] * albedo_k[c] * INV_PI * Le[c] * std::fabs(G);
        }
        if (cr > 0.0) {
          double W = vlen(J) / (Nl * cr);
          double w1 = h.b1, w2 = h.b2, w0 = 1.0 - w1 - w2;
          D3 Md = w0 * vert_dual(P, M.i0, C.track) + w1 * vert_dual(P, M.i1, C.track) +
                  w2 * vert_dual(P, M.i2, C.track);
          Dual alpha = dot(at_value(Md, m32) - Ps, Nd);
          accumulate(C, sgn * hs * W * inv_pe, hs_abs * W * inv_pe, alpha);
        }
      }
    }
    /* indirect part: reflected radiance at m with the remaining depth */
    if (b + 1 < max_depth) {
      D3 Oc = d3(p.x, p.y, p.z), Dc = d3(ds[0], ds[1], ds[2]);
      double one[3] = {1, 1, 1}, zero[3] = {0, 0, 0};
      RGB Lr;
      bool saved = C.track;
      C.track = false;
      path_radiance(C, b + 1, max_depth, p32, ds, Oc, Dc, k, false, c0, c1, cont_pass, zero, one, false, &Lr);
      C.track = saved;
      double hs = 0.0, hs_abs = 0.0;
      for (int c = 0; c < 3; ++c) {
        hs += wscale[c] * beta[c] * albedo_k[c] * INV_PI * cos_p * Lr.c[c].v;
        hs_abs += std::fabs(wscale[c] * beta[c] * albedo_k[c] * INV_PI * cos_p * Lr.c[c].v);
      }
      if (hs != 0.0) {
        Dual alpha = dot(d3(what.x, what.y, what.z), Nd);
        accumulate(C, sgn * hs / wl2 * inv_pe, hs_abs / wl2 * inv_pe, alpha);
      }
    }
  }
}

/* Radiance along a path (Sec. 5.4: path tracer with next-event estimation at
 * every vertex, emission seen directly only at the first camera hit).
 * depth0: index of the first scattering vertex; vertices depth0..max_depth-1
 * are shaded.  beta_in: throughput value before the first vertex (used only
 * for the secondary-edge weights); out: radiance duals (interior part). */
void path_radiance(Ctx& C, int depth0, int max_depth, const float o32_in[3], const float d32_in[3],
                   const D3& O_in, const D3& D_in, int exclude_in, bool emission_first, uint32_t c0, uint32_t c1,
                   uint32_t pass, const double wscale[3], const double beta_in[3], bool backward, RGB* out) {
  const Prep& P = *C.P;
  const or_scene_t& sc = *P.sc;
  const or_opts_t& op = *C.opt;
  for (int c = 0; c < 3; ++c) out->c[c] = Dual(0.0);
  float o32[3] = {o32_in[0], o32_in[1], o32_in[2]}, d32[3] = {d32_in[0], d32_in[1], d32_in[2]};
  D3 O = O_in, D = D_in;
  int exclude = exclude_in;
  Dual beta[3] = {Dual(1.0), Dual(1.0), Dual(1.0)};
  double betav[3] = {beta_in[0], beta_in[1], beta_in[2]};
  for (int b = depth0; b < max_depth; ++b) {
    Hit h = closest(P, o32, d32, exclude);
    if (h.tri < 0) break;
    int k = h.tri;
    TriV T = tri_of(P, k);
    float p32[3];
    bary_point32(T.v0, T.v1, T.v2, h.b1, h.b2, p32);
    D3 V0 = vert_dual(P, T.i0, C.track), V1 = vert_dual(P, T.i1, C.track), V2 = vert_dual(P, T.i2, C.track);
    D3 Pd = hit_point_dual(O, D, V0, V1, V2);
    float nu32[3];
    face_normal32(T.v0, T.v1, T.v2, nu32);
    float side = dot32(nu32, d32);
    D3 Nk = cross(V1 - V0, V2 - V0);
    Dual nkl = length(Nk);
    double flip = side > 0.0f ? -1.0 : 1.0;
    D3 ns{flip * (Nk.x / nkl), flip * (Nk.y / nkl), flip * (Nk.z / nkl)};
    Dual alb[3];
    for (int c = 0; c < 3; ++c) alb[c] = Dual::param(sc.albedo[3 * k + c], P.pA + 3 * k + c, C.track);
    if (op.primary_only) {
      /* geometry buffers of the first hit (Sec. 5.4): the value is a smooth
       * function of the hit point and triangle, discontinuous only where the
       * visible triangle changes, so the primary edge term covers its
       * discontinuities as for shaded images */
      if (op.aov == 2) {
        out->c[0] = out->c[0] + Pd.x;
        out->c[1] = out->c[1] + Pd.y;
        out->c[2] = out->c[2] + Pd.z;
      } else if (op.aov == 3) {
        out->c[0] = out->c[0] + ns.x;
        out->c[1] = out->c[1] + ns.y;
        out->c[2] = out->c[2] + ns.z;
      } else if (op.aov == 4) {
        D3 dv = Pd - O;
        Dual dist = length(dv);
        for (int c = 0; c < 3; ++c) out->c[c] = out->c[c] + dist;
      } else {
        for (int c = 0; c < 3; ++c) out->c[c] = out->c[c] + beta[c] * alb[c];
      }
      break;
    }
    Dual Le[3];
    for (int c = 0; c < 3; ++c) Le[c] = Dual::param(sc.radiance[c], P.pR + c, C.track);
    if (b == depth0 && emission_first && P.light_of_tri[k] >= 0 && side < 0.0f)
      for (int c = 0; c < 3; ++c) out->c[c] = out->c[c] + beta[c] * Le[c];
    /* next-event estimation: light triangle by area, uniform point, one shadow ray */
    if (P.light_total > 0.0) {
      uint32_t r[4];
      rng(op.seed, c0, c1, K_LIGHT, (uint32_t)b, pass, (uint32_t)op.scene_id, r);
      int j = cdf_pick(P.light_cdf, u01d(r[0], r[1]) * P.light_total);
      float y32[3], by[3];
      D3 Y;
      light_point(P, j, u01f(r[2]), u01f(r[3]), C.track, y32, &Y, by);
      int lt = sc.light_tris[j];
      float sd[3] = {y32[0] - p32[0], y32[1] - p32[1], y32[2] - p32[2]};
      if (!occluded(P, p32, sd, SHADOW_TMAX, k, lt)) {
        D3 Wv = Y - Pd;
        Dual r2 = dot(Wv, Wv);
        Dual rl = dsqrt(r2);
        D3 om = Wv / rl;
        Dual cos_p = dot(ns, om);
        TriV L = tri_of(P, lt);
        D3 L0 = vert_dual(P, L.i0, C.track), L1 = vert_dual(P, L.i1, C.track), L2 = vert_dual(P, L.i2, C.track);
        D3 Nl = cross(L1 - L0, L2 - L0);
        Dual nll = length(Nl);
        Dual cos_y = -(dot(Nl, om) / nll);
        if (cos_p.v > 0.0 && cos_y.v > 0.0) {
          Dual Aj = 0.5 * nll;
          double inv_pj = P.light_total / P.light_area[j];  /* 1 / P(j), a value */
          Dual G = cos_p * cos_y / r2;
          for (int c = 0; c < 3; ++c)
            out->c[c] = out->c[c] + beta[c] * (alb[c] * INV_PI) * Le[c] * G * Aj * inv_pj;
        }
      }
    }
    float nl32 = std::sqrt(dot32(nu32, nu32));
    float fl = side > 0.0f ? -1.0f : 1.0f;
    float ns32[3] = {fl * (nu32[0] / nl32), fl * (nu32[1] / nl32), fl * (nu32[2] / nl32)};
    if (backward && (op.terms & 4)) {
      double albv[3] = {sc.albedo[3 * k], sc.albedo[3 * k + 1], sc.albedo[3 * k + 2]};
      secondary_edge(C, b, c0, c1, pass, p32, Pd, val(ns), ns32, k, albv, betav, wscale, max_depth);
    }
    if (b + 1 >= max_depth) break;
    /* continuation: cosine-weighted direction, world direction held fixed */
    uint32_t r[4];
    rng(op.seed, c0, c1, K_BSDF, (uint32_t)b, pass, (uint32_t)op.scene_id, r);
    float nd[3];
    cosine_dir32(ns32, u01f(r[0]), u01f(r[1]), nd);
    D3 Dn = d3(nd[0], nd[1], nd[2]);
    Dual cosd = dot(ns, Dn);
    double pdf_cos = cosd.v;  /* pdf / (1/pi), a value */
    if (!(pdf_cos > 0.0)) break;
    for (int c = 0; c < 3; ++c) {
      beta[c] = beta[c] * alb[c] * (cosd / pdf_cos);
      betav[c] = betav[c] * sc.albedo[3 * k + c];
    }
    for (int i = 0; i < 3; ++i) { o32[i] = p32[i]; d32[i] = nd[i]; }
    O = Pd; D = Dn; exclude = k;
  }
}

/* Camera-path radiance for the interior sample (pix, s) or an edge side point. */
void camera_path(Ctx& C, float sx, float sy, uint32_t c0, uint32_t c1, uint32_t pass, const double wscale[3],
                 bool backward, RGB* out) {
  const Prep& P = *C.P;
  R32 r = camera_ray32(*P.sc, sx, sy);
  D3 O, D;
  camera_ray_dual(P, sx, sy, C.track, &O, &D);
  double one[3] = {1, 1, 1};
  int md = C.opt->primary_only ? 1 : C.opt->max_depth;
  path_radiance(C, 0, md, r.o, r.d, O, D, -1, true, c0, c1, pass, wscale, one, backward, out);
}

void jitter(const or_opts_t& op, int pix, int s, int W, float* sx, float* sy) {
  uint32_t r[4];
  rng(op.seed, (uint32_t)pix, (uint32_t)s, K_CAMERA, 0, PASS_INTERIOR, (uint32_t)op.scene_id, r);
  *sx = (float)(pix % W) + u01f(r[0]);
  *sy = (float)(pix / W) + u01f(r[1]);
}

/* Both side points of a primary edge sample see the same triangle first: the
 * edge bounds nothing visible there, so f is continuous across it and the
 * sample's term of Eq. mc is zero (the difference of the two evaluations a
 * finite offset apart would be an O(eps) residue). */
bool same_first_hit(const Prep& P, float xu, float yu, float xl, float yl) {
  R32 ru = camera_ray32(*P.sc, xu, yu), rl = camera_ray32(*P.sc, xl, yl);
  Hit hu = closest(P, ru.o, ru.d, -1), hl = closest(P, rl.o, rl.d, -1);
  return hu.tri >= 0 && hu.tri == hl.tri;
}

/* ---- primary edge sample of the fisheye (Sec. 5.2, non-linear projections) --
 * The image of an edge is a curve x(t) = pi(v0 + t (v1 - v0)).  The edge is
 * picked by its chord on the unit sphere of directions (prepare), t
 * uniformly in [0, 1), and the two sides are evaluated a small offset apart
 * across the curve (the offset direction perpendicular to the FP32 chord of
 * x(t - 1/1024) and x(t + 1/1024), clamped to the edge).  By Reynolds
 * transport over the pixel integral, a parameter moving the curve with
 * screen velocity V changes sum_p w_p I_p by -(f_u - f_l) (V . n_u) ds along
 * it; with ds n_u = perp(x'(t)) dt, the sample contributes
 * w (f_u - f_l) d(-perp(x'(t)) . x)/d theta / (P(e) N), perp(x') = (-x'_y,
 * x'_x) pointing to the u side.  Points outside the image contribute zero. */
void primary_edge_sample_fisheye(Ctx& C, int64_t jj, const uint32_t r[4]) {
  const Prep& P = *C.P;
  const or_scene_t& sc = *P.sc;
  const or_opts_t& op = *C.opt;
  uint32_t j = (uint32_t)jj;
  int e = cdf_pick(P.pcdf, u01d(r[0], r[1]) * P.ptotal);
  double pe = P.pcdf[e] - (e > 0 ? P.pcdf[e - 1] : 0.0);
  if (!(pe > 0.0)) return;
  const float *v0 = vtx(P, P.e0[e]), *v1 = vtx(P, P.e1[e]);
  float t = u01f(r[2]);
  auto point = [&](float tt, float out[3]) {
    for (int i = 0; i < 3; ++i) out[i] = v0[i] + tt * (v1[i] - v0[i]);
  };
  float p32[3], q0[3], q1[3];
  point(t, p32);
  float x, y, x0, y0, x1, y1;
  if (!fisheye_project32(P, p32, &x, &y)) return;
  float W = (float)sc.width, H = (float)sc.height;
  if (!(x >= 0.0f && x < W && y >= 0.0f && y < H)) return;
  float ta = t - 0.0009765625f, tb = t + 0.0009765625f;
  if (ta < 0.0f) ta = 0.0f;
  if (tb > 1.0f) tb = 1.0f;
  point(ta, q0);
  point(tb, q1);
  if (!fisheye_project32(P, q0, &x0, &y0) || !fisheye_project32(P, q1, &x1, &y1)) return;
  float cx = x1 - x0, cy = y1 - y0;
  float cl = std::sqrt(cx * cx + cy * cy);
  if (!(cl > 0.0f)) return;
  float nx = -cy / cl, ny = cx / cl;
  float eps = op.eps_rel * std::max(W, H);
  float xu = x + eps * nx, yu = y + eps * ny, xl = x - eps * nx, yl = y - eps * ny;
  int px = (int)std::floor(x), py = (int)std::floor(y);
  C.pix = (int64_t)py * sc.width + px;
  if (same_first_hit(P, xu, yu, xl, yl)) return;
  const float* w = C.w + 3 * ((size_t)py * sc.width + px);
  double zero[3] = {0, 0, 0};
  bool saved = C.track;
  C.track = false;
  RGB Lu, Ll;
  camera_path(C, xu, yu, j, 0, PASS_PRIMARY_EDGE, zero, false, &Lu);
  camera_path(C, xl, yl, j, 0, PASS_PRIMARY_EDGE, zero, false, &Ll);
  C.track = saved;
  double diff = 0.0, diff_abs = 0.0;
  for (int c = 0; c < 3; ++c) {
    diff += (double)w[c] * (Lu.c[c].v - Ll.c[c].v);
    diff_abs += std::fabs((double)w[c]) * (std::fabs(Lu.c[c].v) + std::fabs(Ll.c[c].v));
  }
  if (diff == 0.0) return;
  /* the curve point as a function of the parameters, and its tangent */
  D3 V0 = vert_dual(P, P.e0[e], C.track), V1 = vert_dual(P, P.e1[e], C.track);
  D3 Pt = V0 + (double)t * (V1 - V0);
  Dual X, Y;
  project_fisheye_dual(P, Pt, C.track, &X, &Y);
  D3 C0 = d3(v0[0], v0[1], v0[2]), C1 = d3(v1[0], v1[1], v1[2]);
  Dual tt = Dual::param((double)t, 0, true);
  D3 Pt_t = C0 + tt * (C1 - C0);
  Dual Xt, Yt;
  project_fisheye_dual(P, Pt_t, false, &Xt, &Yt);
  double dxt = Xt.n > 0 ? Xt.d[0] : 0.0, dyt = Yt.n > 0 ? Yt.d[0] : 0.0;
  Dual alpha = dyt * X - dxt * Y;  /* -perp(x') . x */
  int64_t N_edge = (int64_t)op.edge_spp * sc.width * sc.height;
  double k = (P.ptotal / pe) / (double)N_edge;
  accumulate(C, diff * k, diff_abs * k, alpha);
}

/* ---- primary edge sample j (Eq. mc with Eq. redner_dirac_jacobian) ------- */
void primary_edge_sample(Ctx& C, int64_t jj) {
  const Prep& P = *C.P;
  const or_scene_t& sc = *P.sc;
  const or_opts_t& op = *C.opt;
  if (P.ptotal <= 0.0) return;
  uint32_t j = (uint32_t)jj;
  uint32_t r[4];
  rng(op.seed, j, 0, K_EDGE_PRIMARY, 0, PASS_PRIMARY_EDGE, (uint32_t)op.scene_id, r);
  if (sc.cam_type == 2) {
    primary_edge_sample_fisheye(C, jj, r);
    return;
  }
  int e;
  float t0, t1;
  double inv_pdf_len;  /* 1 / (pdf of the point per unit length) = len_seg / q_seg, or L for the plain sampler */
  if (op.proposal >= 1) {
    if (P.seg_cdf.empty() || !(P.seg_total > 0.0)) return;
    int k = cdf_pick(P.seg_cdf, u01d(r[0], r[1]) * P.seg_total);
    double q = P.seg_cdf[k] - (k > 0 ? P.seg_cdf[k - 1] : 0.0);
    if (!(q > 0.0)) return;
    e = P.seg_edge[k];
    t0 = P.seg_s0[k];
    t1 = P.seg_s1[k];
    inv_pdf_len = P.seg_len[k] / (q / P.seg_total);
  } else {
    e = cdf_pick(P.pcdf, u01d(r[0], r[1]) * P.ptotal);
    t0 = P.pt0[e];
    t1 = P.pt1[e];
    inv_pdf_len = P.ptotal;
  }
  float ax = P.pax[e], ay = P.pay[e], bx = P.pbx[e], by = P.pby[e];
  float dx = bx - ax, dy = by - ay;
  float t = t0 + u01f(r[2]) * (t1 - t0);
  float x = ax + t * dx, y = ay + t * dy;
  float nlen = std::sqrt(dx * dx + dy * dy);
  float nx = -dy / nlen, ny = dx / nlen;
  float W = (float)sc.width, H = (float)sc.height;
  float eps = op.eps_rel * std::max(W, H);
  float xu = x + eps * nx, yu = y + eps * ny, xl = x - eps * nx, yl = y - eps * ny;
  int px = (int)std::floor(x), py = (int)std::floor(y);
  px = std::min(std::max(px, 0), sc.width - 1);
  py = std::min(std::max(py, 0), sc.height - 1);
  C.pix = (int64_t)py * sc.width + px;  /* the sample belongs to the pixel containing its point */
  if (same_first_hit(P, xu, yu, xl, yl)) return;
  const float* w = C.w + 3 * ((size_t)py * sc.width + px);
  double zero[3] = {0, 0, 0};
  bool saved = C.track;
  C.track = false;
  RGB Lu, Ll;
  camera_path(C, xu, yu, j, 0, PASS_PRIMARY_EDGE, zero, false, &Lu);
  camera_path(C, xl, yl, j, 0, PASS_PRIMARY_EDGE, zero, false, &Ll);
  C.track = saved;
  double diff = 0.0, diff_abs = 0.0;
  for (int c = 0; c < 3; ++c) {
    diff += (double)w[c] * (Lu.c[c].v - Ll.c[c].v);
    diff_abs += std::fabs((double)w[c]) * (std::fabs(Lu.c[c].v) + std::fabs(Ll.c[c].v));
  }
  if (diff == 0.0) return;
  Dual Ax, Ay, Bx, By;
  project_dual(P, vert_dual(P, P.e0[e], C.track), C.track, &Ax, &Ay);
  project_dual(P, vert_dual(P, P.e1[e], C.track), C.track, &Bx, &By);
  double X = x, Y = y;
  Dual alpha = (Ay - By) * X + (Bx - Ax) * Y + (Ax * By - Bx * Ay);
  double gl = std::sqrt((Ax.v - Bx.v) * (Ax.v - Bx.v) + (Ay.v - By.v) * (Ay.v - By.v));
  int64_t N_edge = (int64_t)op.edge_spp * sc.width * sc.height;
  double k = inv_pdf_len / (gl * (double)N_edge);
  accumulate(C, diff * k, diff_abs * k, alpha);
}

template <class F>
void parallel_for(int64_t begin, int64_t end, int n_threads, F f) {
  int64_t n = end - begin;
  if (n <= 0) return;
  int nt = (int)std::max<int64_t>(1, std::min<int64_t>(n_threads, n));
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) {
    int64_t b = begin + n * t / nt, e = begin + n * (t + 1) / nt;
    th.emplace_back([=]() { f(t, b, e); });
  }
  for (auto& x : th) x.join();
}

}  // namespace

extern "C" {

void or_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }

int or_num_params(const or_scene_t* sc) { return 3 * sc->n_verts + 3 * sc->n_tris + 3 + 13; }

/* Point on a secondary edge by the clamped-cosine density (test hook). */
void or_edge_point(const float* p, const float* n, const float* v0, const float* v1, float u, float usel, float* t,
                   double* q) {
  EdgePoint ep = edge_point_sample(p, n, v0, v1, u, usel);
  *t = ep.t;
  *q = ep.q;
}

/* Brute-force closest hit; returns the triangle index or -1. */
int or_closest(const or_scene_t* sc, const float* o, const float* d, int exclude, float* t_b1_b2) {
  Prep P;
  P.sc = sc; P.V = sc->n_verts; P.T = sc->n_tris;
  Hit h = closest(P, o, d, exclude);
  if (h.tri >= 0) { t_b1_b2[0] = h.t; t_b1_b2[1] = h.b1; t_b1_b2[2] = h.b2; }
  return h.tri;
}
int or_closest_batch(const or_scene_t* sc, int n, const float* o, const float* d, int n_threads, int* tri,
                     float* t_b1_b2) {
  Prep P;
  P.sc = sc; P.V = sc->n_verts; P.T = sc->n_tris;
  parallel_for(0, n, n_threads, [&](int, int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      Hit h = closest(P, o + 3 * i, d + 3 * i, -1);
      tri[i] = h.tri;
      t_b1_b2[3 * i] = h.t; t_b1_b2[3 * i + 1] = h.b1; t_b1_b2[3 * i + 2] = h.b2;
    }
  });
  return 0;
}

void or_sincos_2pi(float r, float* c, float* s) { sincos_2pi32(r, c, s); }
float or_atan2_pos(float y, float x) { return atan2_pos32(y, x); }

/* Camera ray through a screen point, and the fisheye projection of a world
 * point (test hooks; the projection returns 0 where no pixel sees the point). */
void or_camera_ray(const or_scene_t* sc, float sx, float sy, float* o, float* d) {
  R32 r = camera_ray32(*sc, sx, sy);
  for (int i = 0; i < 3; ++i) { o[i] = r.o[i]; d[i] = r.d[i]; }
}
int or_fisheye_project(const or_scene_t* sc, const float* v, float* sx, float* sy) {
  Prep P;
  prepare(sc, P);
  return fisheye_project32(P, v, sx, sy) ? 1 : 0;
}
void or_cosine_dir(const float* n, float r1, float r2, float* out) { cosine_dir32(n, r1, r2, out); }

/* Unique edges [E,2]; returns E (writes at most cap). */
int or_edges(const or_scene_t* sc, int32_t* out, int cap) {
  Prep P;
  prepare(sc, P);
  int E = (int)P.e0.size();
  for (int e = 0; e < E && e < cap; ++e) { out[2 * e] = P.e0[e]; out[2 * e + 1] = P.e1[e]; }
  return E;
}
/* Secondary edge hierarchy (Sec. 5.3.1), for the tests.
 * nodes [n_nodes, 2] children (>= 0 node, < 0 ~leaf position); slots
 * [n_nodes, 2, 14] = (lo[3], hi[3], hlo[3], hhi[3], L, allB); leaves [E, 3] =
 * (edge id, class B, boundary).  Returns the node count (writes at most cap)
 * and the root code in *root. */
int or_edge_tree(const or_scene_t* sc, int32_t* nodes, float* slots, int32_t* leaves, int cap, int32_t* root) {
  Prep P;
  prepare(sc, P);
  EdgeTree T;
  build_edge_tree(P, T);
  int n = (int)T.node.size();
  for (int i = 0; i < n && i < cap; ++i)
    for (int c = 0; c < 2; ++c) {
      nodes[2 * i + c] = T.node[i].child[c];
      const ETSlot& s = T.node[i].slot[c];
      float* o = slots + 28 * i + 14 * c;
      for (int k = 0; k < 3; ++k) { o[k] = s.lo[k]; o[3 + k] = s.hi[k]; o[6 + k] = s.hlo[k]; o[9 + k] = s.hhi[k]; }
      o[12] = s.L;
      o[13] = s.allB ? 1.0f : 0.0f;
    }
  for (size_t i = 0; i < T.leaf.size(); ++i) {
    leaves[3 * i] = T.leaf[i].eid;
    leaves[3 * i + 1] = T.leaf[i].classB;
    leaves[3 * i + 2] = T.leaf[i].boundary;
  }
  *root = T.root;
  return n;
}

/* For a shading point p: per node and child slot, 1 if the slot holds only
 * class-B edges and the v-sphere clears its Hough box. */
void or_edge_tree_vsphere(const or_scene_t* sc, const float* p, uint8_t* out) {
  Prep P;
  prepare(sc, P);
  EdgeTree T;
  build_edge_tree(P, T);
  float n[3] = {0.0f, 0.0f, 1.0f};
  ETQuery q = et_query(T, p, n, true, 0.0f);
  for (size_t i = 0; i < T.node.size(); ++i)
    for (int c = 0; c < 2; ++c)
      out[2 * i + c] = T.node[i].slot[c].allB && et_vsphere_clears(q, T.node[i].slot[c]);
}

/* Upper bound of the cosine over a box seen from p with unit normal n. */
float or_edge_tree_cos_bound(const float* p, const float* n, const float* lo, const float* hi) {
  EdgeTree T;
  for (int i = 0; i < 3; ++i) T.O[i] = 0.0f;
  ETQuery q = et_query(T, p, n, false, 0.0f);
  return et_cos_bound(q, lo, hi);
}

/* N picks at one shading point with counters (0, i): edge ids and weights
 * (-1 and 0 where no edge was picked). */
void or_edge_tree_picks(const or_scene_t* sc, const float* p, const float* n, int last, int S, float eps,
                        uint64_t seed, int bounce, int scene_id, int N, int32_t* eid, float* w) {
  Prep P;
  prepare(sc, P);
  EdgeTree T;
  build_edge_tree(P, T);
  ETQuery q = et_query(T, p, n, last != 0, eps);
  for (int i = 0; i < N; ++i) {
    int e;
    float x;
    if (et_pick(T, q, S, seed, 0u, (uint32_t)i, (uint32_t)bounce, (uint32_t)scene_id, &e, &x)) {
      eid[i] = e; w[i] = x;
    } else {
      eid[i] = -1; w[i] = 0.0f;
    }
  }
}

/* Primary edge table [E,7] = (ax, ay, bx, by, t0, t1, clipped length). */
int or_primary_edges(const or_scene_t* sc, double* out, int cap) {
  Prep P;
  prepare(sc, P);
  int E = (int)P.e0.size();
  for (int e = 0; e < E && e < cap; ++e) {
    double* o = out + 7 * e;
    o[0] = P.pax[e]; o[1] = P.pay[e]; o[2] = P.pbx[e]; o[3] = P.pby[e]; o[4] = P.pt0[e]; o[5] = P.pt1[e];
    o[6] = P.pcdf[e] - (e > 0 ? P.pcdf[e - 1] : 0.0);
  }
  return E;
}

/* Tile segments [n,4] = (edge, tile, s0, s1) as doubles plus [n] lengths;
 * returns n (writes at most cap). */
int64_t or_segments(const or_scene_t* sc, double* out, double* lens, int64_t cap) {
  Prep P;
  prepare(sc, P);
  int64_t n = (int64_t)P.seg_len.size();
  for (int64_t k = 0; k < n && k < cap; ++k) {
    out[4 * k] = P.seg_edge[k];
    out[4 * k + 1] = P.seg_tile[k];
    out[4 * k + 2] = P.seg_s0[k];
    out[4 * k + 3] = P.seg_s1[k];
    lens[k] = P.seg_len[k];
  }
  return n;
}

/* Image [H,W,3] in FP64 for pixels in [pix_begin, pix_end) (others untouched). */
int or_render(const or_scene_t* sc, const or_opts_t* op, double* image) {
  Prep P;
  prepare(sc, P);
  int npix = sc->width * sc->height;
  int pb = op->pix_begin, pe = op->pix_end > 0 ? op->pix_end : npix;
  g_dual_overflow = false;
  parallel_for(pb, pe, op->n_threads, [&](int, int64_t b, int64_t e) {
    Ctx C{&P, op, false, nullptr, nullptr, nullptr};
    double zero[3] = {0, 0, 0};
    for (int64_t pix = b; pix < e; ++pix) {
      double acc[3] = {0, 0, 0};
      for (int s = 0; s < op->spp; ++s) {
        float sx, sy;
        jitter(*op, (int)pix, s, sc->width, &sx, &sy);
        RGB L;
        camera_path(C, sx, sy, (uint32_t)pix, (uint32_t)s, PASS_INTERIOR, zero, false, &L);
        for (int c = 0; c < 3; ++c) acc[c] += L.c[c].v;
      }
      for (int c = 0; c < 3; ++c) image[3 * pix + c] = acc[c] / op->spp;
    }
  });
  return g_dual_overflow ? 2 : 0;
}

/* Gradient of sum_p w_p . I_p into grad[P] (FP64), and into abs_grad[P] the
 * magnitude of the terms that were summed (absolute-value chain rule, see
 * Dual) -- the scale of the rounding error an FP32 evaluation may make.
 * If contrib_abs is non-null it receives per entry sum_k |c_k| over the
 * samples' whole contributions c_k (the plain sum-of-magnitudes scale, which
 * the chain rule with absolute values bounds from above).  If jac is non-null
 * it receives [n_jac, H, W]: for each listed parameter, the contributions of
 * the samples of each pixel (interior and secondary samples by their camera
 * path's pixel, primary edge samples by the pixel containing their point),
 * which sum over the pixels to the gradient entry.  All outputs are
 * overwritten. */
int or_backward4(const or_scene_t* sc, const or_opts_t* op, const float* d_image, double* grad, double* abs_grad,
                 double* contrib_abs, double* jac) {
  Prep P;
  prepare(sc, P);
  int NP = P.P;
  int nt = std::max(1, op->n_threads);
  std::vector<std::vector<double>> g(nt, std::vector<double>(NP, 0.0)), ga(nt, std::vector<double>(NP, 0.0));
  std::vector<std::vector<double>> gc(contrib_abs ? nt : 0, std::vector<double>(NP, 0.0));
  int64_t npix_all = (int64_t)sc->width * sc->height;
  int n_jac = jac ? std::max(0, std::min(8, (int)op->n_jac)) : 0;
  std::vector<std::vector<double>> gj(n_jac > 0 ? nt : 0, std::vector<double>((size_t)n_jac * npix_all, 0.0));
  g_dual_overflow = false;
  int npix = sc->width * sc->height;
  EdgeTree tree;
  if (op->sec_nee && (op->sec_sampler != 0 || op->sec_point != 0)) return 3;  /* length sampler, uniform point */
  if (op->sec_sampler == 1 || op->sec_nee) build_edge_tree(P, tree);
  std::vector<int> leaf_of_edge(tree.leaf.size(), -1);
  for (int q = 0; q < (int)tree.leaf.size(); ++q) leaf_of_edge[tree.leaf[q].eid] = q;
  float nee_hw = !op->sec_nee ? 0.0f : (op->nee_width > 0.0f ? 0.5f * op->nee_width : nee_half_width(*sc));
  if (op->terms & 5) {
    int pb = op->pix_begin, pe = op->pix_end > 0 ? op->pix_end : npix;
    parallel_for(pb, pe, nt, [&](int tid, int64_t b, int64_t e) {
      Ctx C{&P, op, true, d_image, g[tid].data(), ga[tid].data(), &tree, contrib_abs ? gc[tid].data() : nullptr,
            n_jac > 0 ? gj[tid].data() : nullptr};
      C.nee_hw = nee_hw;
      C.leaf_of_edge = &leaf_of_edge;
      for (int64_t pix = b; pix < e; ++pix) {
        C.pix = pix;
        const float* w = d_image + 3 * pix;
        double ws[3] = {w[0] / (double)op->spp, w[1] / (double)op->spp, w[2] / (double)op->spp};
        for (int s = 0; s < op->spp; ++s) {
          float sx, sy;
          jitter(*op, (int)pix, s, sc->width, &sx, &sy);
          RGB L;
          C.track = (op->terms & 1) != 0;
          /* secondary edges need p's derivatives even when the interior term is off */
          if (op->terms & 4) C.track = true;
          camera_path(C, sx, sy, (uint32_t)pix, (uint32_t)s, PASS_INTERIOR, ws, true, &L);
          if (op->terms & 1) {
            Dual sc_ = ws[0] * L.c[0] + ws[1] * L.c[1] + ws[2] * L.c[2];
            accumulate(C, 1.0, 1.0, sc_);
          }
        }
      }
    });
  }
  if (op->proposal >= 1) build_proposal(P, op->seg_weights, op->n_seg_weights, op->proposal);
  if (op->terms & 2) {
    int64_t N = (int64_t)op->edge_spp * npix;
    int64_t eb = op->edge_begin, ee = op->edge_end > 0 ? op->edge_end : N;
    parallel_for(eb, ee, nt, [&](int tid, int64_t b, int64_t e) {
      Ctx C{&P, op, true, d_image, g[tid].data(), ga[tid].data(), nullptr, contrib_abs ? gc[tid].data() : nullptr,
            n_jac > 0 ? gj[tid].data() : nullptr};
      for (int64_t j = b; j < e; ++j) primary_edge_sample(C, j);
    });
  }
  for (int i = 0; i < NP; ++i) {
    double s = 0.0, a = 0.0, c = 0.0;
    for (int t = 0; t < nt; ++t) { s += g[t][i]; a += ga[t][i]; }
    if (contrib_abs)
      for (int t = 0; t < nt; ++t) c += gc[t][i];
    grad[i] = s; abs_grad[i] = a;
    if (contrib_abs) contrib_abs[i] = c;
  }
  for (int64_t q = 0; q < (int64_t)n_jac * npix_all; ++q) {
    double v = 0.0;
    for (int t = 0; t < nt; ++t) v += gj[t][q];
    jac[q] = v;
  }
  return g_dual_overflow ? 2 : 0;
}
int or_backward3(const or_scene_t* sc, const or_opts_t* op, const float* d_image, double* grad, double* abs_grad,
                 double* contrib_abs) {
  return or_backward4(sc, op, d_image, grad, abs_grad, contrib_abs, nullptr);
}
int or_backward(const or_scene_t* sc, const or_opts_t* op, const float* d_image, double* grad, double* abs_grad) {
  return or_backward4(sc, op, d_image, grad, abs_grad, nullptr, nullptr);
}

/* ---- next-event estimation for edges: pieces for the CPU pins ---------- */
float or_ln32(float x) { return ln32(x); }
float or_nee_half_width(const or_scene_t* sc) { return nee_half_width(*sc); }

/* Builds the scene's edge tree once and answers batches of queries. */
struct OrNee {
  Prep P;
  EdgeTree T;
  std::vector<int> leaf_of_edge;
};
void* or_nee_open(const or_scene_t* sc) {
  OrNee* q = new OrNee;
  prepare(sc, q->P);
  build_edge_tree(q->P, q->T);
  q->leaf_of_edge.assign(q->T.leaf.size(), -1);
  for (int k = 0; k < (int)q->T.leaf.size(); ++k) q->leaf_of_edge[q->T.leaf[k].eid] = k;
  return q;
}
void or_nee_close(void* h) { delete (OrNee*)h; }
/* Crossings of the ray p + s d, s in (0, smax): up to cap of (eid, s, t, u, imp);
 * returns their number. */
int or_nee_crossings(void* h, const float* p, const float* n, const float* d, float smax, float hw, int32_t* eid,
                     float* stui, int cap) {
  OrNee* q = (OrNee*)h;
  std::vector<NeeCross> xs;
  nee_crossings(q->T, p, n, d, smax, hw, xs);
  for (int i = 0; i < (int)xs.size() && i < cap; ++i) {
    eid[i] = q->T.leaf[xs[i].leaf].eid;
    stui[4 * i] = xs[i].s; stui[4 * i + 1] = xs[i].t; stui[4 * i + 2] = xs[i].u; stui[4 * i + 3] = xs[i].imp;
  }
  return (int)xs.size();
}
/* The race's pick among the crossings before smax: edge id or -1. */
int or_nee_pick(void* h, const float* p, const float* n, const float* d, float smax, float hw, uint32_t key0,
                uint32_t key1) {
  OrNee* q = (OrNee*)h;
  std::vector<NeeCross> xs;
  nee_crossings(q->T, p, n, d, smax, hw, xs);
  int w = nee_race(q->T, xs, key0, key1);
  return w < 0 ? -1 : q->T.leaf[xs[w].leaf].eid;
}
/* The ray of edge eid's family through (t, u): 1 and d, or 0. */
int or_nee_ray(void* h, int eid, const float* p, float t, float u, float* d) {
  OrNee* q = (OrNee*)h;
  return nee_ray(q->T.leaf[q->leaf_of_edge[eid]], p, t, u, d) ? 1 : 0;
}
double or_nee_jacobian(void* h, int eid, const float* p, float t, float u) {
  OrNee* q = (OrNee*)h;
  return nee_jacobian(q->T.leaf[q->leaf_of_edge[eid]], p, t, u);
}
/* p_B at n samples (eid, t, u) with their rays d. */
void or_nee_density(void* h, int n, const float* p, const float* nrm, const float* d, const int32_t* eid,
                    const float* t, const float* u, float hw, double* out) {
  OrNee* q = (OrNee*)h;
  for (int i = 0; i < n; ++i)
    out[i] = nee_density(q->P, q->T, p + 3 * i, nrm + 3 * i, d + 3 * i, q->leaf_of_edge[eid[i]], t[i], u[i], hw);
}

/* Self-check of the two secondary-edge measures at one edge point: for a
 * shading point p (normal ns), edge (v0, v1), parameter t and a light plane
 * point m with normal nm on the ray from p through the edge point, returns
 *   out[0..5]: area-form weight  x d alpha/d{v0, v1}
 *   out[6..11]: solid-angle form x d alpha_dir/d{v0, v1}
 * with the radiance factor left out (both multiply the same f_r Le cos_p). */
void or_sec_edge_forms(const double* p, const double* v0, const double* v1, double t, const double* nm_in,
                       double plane_d, double* out) {
  V3 P{p[0], p[1], p[2]}, A{v0[0], v0[1], v0[2]}, B{v1[0], v1[1], v1[2]}, nm{nm_in[0], nm_in[1], nm_in[2]};
  nm = (1.0 / vlen(nm)) * nm;
  V3 E = B - A;
  V3 w = (A + t * E) - P;
  V3 a0 = A - P, a1 = B - P;
  V3 N = vcross(a0, a1);
  double Nl = vlen(N);
  V3 nh = (1.0 / Nl) * N;
  /* m on the plane nm.x = plane_d along w */
  double tau = (plane_d - vdot(P, nm)) / vdot(w, nm);
  V3 m = P + tau * w;
  V3 dm = m - P;
  double r2 = vdot(dm, dm);
  V3 wh = (1.0 / std::sqrt(r2)) * dm;
  double cos_m = std::fabs(vdot(nm, wh));
  double h_area = cos_m / r2;  /* area-measure integrand without f_r Le cos_p */
  double wn = vdot(w, nm);
  V3 J = tau * (E - (vdot(E, nm) / wn) * w);
  double W = vlen(J) / (Nl * vlen(vcross(nm, nh)));
  V3 g0 = vcross(a1, dm), g1 = vcross(dm, a0);
  double s0 = h_area * W;
  out[0] = s0 * g0.x; out[1] = s0 * g0.y; out[2] = s0 * g0.z;
  out[3] = s0 * g1.x; out[4] = s0 * g1.y; out[5] = s0 * g1.z;
  double wl2 = vdot(w, w);
  V3 what = (1.0 / std::sqrt(wl2)) * w;
  V3 h0 = vcross(a1, what), h1 = vcross(what, a0);
  double s1 = 1.0 / wl2;
  out[6] = s1 * h0.x; out[7] = s1 * h0.y; out[8] = s1 * h0.z;
  out[9] = s1 * h1.x; out[10] = s1 * h1.y; out[11] = s1 * h1.z;
}

}  // extern "C"
