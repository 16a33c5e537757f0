// drt_device.cuh -- device-side building blocks of the GB300 edge-sampling
// differentiable ray tracer: counter RNG, the FP32 decision path, and the
// BVH traversal.
//
// Decision path.  Every value that decides a discrete outcome (which triangle
// a ray hits, whether a shadow ray is blocked, which edge or light triangle is
// picked, where a sample point lies) is computed with explicit
// round-to-nearest intrinsics (__fadd_rn, __fmul_rn, ...), which the compiler
// never contracts into FMAs, in a fixed operation order.  Two runs of the same
// estimator therefore take identical decisions on any IEEE machine that
// evaluates the same order, which is what makes per-sample comparison against
// an independent CPU implementation possible.  Smooth values (shading,
// derivatives) use ordinary FP32 arithmetic.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/drt.h"

namespace drt {

// ---------------------------------------------------------------------------
// Exact-order scalar arithmetic
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsq(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddv(double a, double b) { return __ddiv_rn(a, b); }

__device__ __forceinline__ float dot3x(const float* a, const float* b) {
  return fa(fa(fm(a[0], b[0]), fm(a[1], b[1])), fm(a[2], b[2]));
}

// ---------------------------------------------------------------------------
// Constants of the estimator
// ---------------------------------------------------------------------------
constexpr float kNearZ = 1e-4f;        // camera depth below which a vertex is behind
constexpr float kShadowTmax = 0.9999f; // shadow rays stop short of the light point
constexpr float kInvPi = 0.318309886f;
constexpr int kStackSize = 64;
constexpr int kTraceWarps = 8;  // warps per CTA that the warp-cooperative traversals support
constexpr float kTile = 16.0f;  // screen tile of the segment split, pixels
// BVH leaves hold up to a scene-chosen number (at most kLeafLimit) of
// consecutive triangles of the leaf-order soup; a leaf child is encoded as
// ~(first | (count-1) << 28).  One per leaf suits incoherent rays; two cut the
// node visits of coherent first-vertex rays by more than the extra tests cost.
constexpr int kLeafLimit = 8;
__host__ __device__ __forceinline__ int leaf_enc(int first, int count) { return ~(first | ((count - 1) << 28)); }
// float4 per closest-hit and any-hit pair record of the traversal pools
constexpr int kClosestRecF4 = 4;
constexpr int kAnyRecF4 = 5;
// device error-flag codes (mirrors the public enum in drt.h)


enum { kCamera = 0, kLight = 1, kBsdf = 2, kEdgePrimary = 3, kEdgeSecondary = 4 };
// passes of the counter layout: the continuation paths of a secondary sample at
// vertex b use kPassSecondaryBase + b, those of a billboard sample of next-event
// estimation for edges kPassNeeBase + b
enum { kPassInterior = 0, kPassPrimaryEdge = 1, kPassSecondaryBase = 2, kPassNeeBase = 18 };

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}
// Counter layout: (c0, c1, kind<<24 | bounce<<16 | pass, scene).
__device__ __forceinline__ uint4 rng4(uint2 key, uint32_t c0, uint32_t c1, uint32_t kind, uint32_t bounce,
                                      uint32_t pass, uint32_t scene) {
  return philox(make_uint4(c0, c1, (kind << 24) | ((bounce & 0xffu) << 16) | (pass & 0xffffu), scene), key);
}
__device__ __forceinline__ float u01f(uint32_t x) { return fm((float)(x >> 8), 5.9604644775390625e-08f); }
__device__ __forceinline__ double u01d(uint32_t x0, uint32_t x1) {
  return dm(da(dm((double)(x0 >> 5), 67108864.0), (double)(x1 >> 6)), 1.1102230246251565e-16);
}

// ---------------------------------------------------------------------------
// Device view of an uploaded scene (plain pointers into library buffers)
// ---------------------------------------------------------------------------
struct SceneView {
  const float* verts;        // [V,3]
  const int32_t* tris;       // [T,3]
  const float* albedo;       // [T,3]
  const float* radiance;     // [3]
  const float* cam;          // [16]
  const float* cam_scale;    // [1]
  const float* w2c;          // [12]  FP64 inverse of cam rows, rounded once
  const int32_t* light_tris; // [L]
  const int32_t* light_of_tri; // [T] index into light_tris or -1
  const double* light_cdf;   // [L] inclusive prefix of light areas
  const double* light_area;  // [L]
  const float* light_box;    // [6] padded bounding box of all light triangles (lo.xyz, hi.xyz)
  const float4* nodes;       // [4*(T-1)] BVH2 nodes, 64 B each
  const float4* soup;        // [3*T] triangles in BVH leaf order, w = original id bits
  const int2* edges;         // [E] unique edges (v0 < v1), sorted
  const float* pedge;        // [E,8] primary edge table: ax ay bx by t0 t1 (2 pad)
  const double* pcdf;        // [E] inclusive prefix of clipped screen lengths
  const double* scdf;        // [E] inclusive prefix of 3D edge lengths
  const int* pguide;         // [kGuide+1] guide table of pcdf
  const int* sguide;         // [kGuide+1] guide table of scdf
  int* err;                  // [2] device error flag (code, info)
  unsigned long long* counters;  // optional work counters [4] for this launch (or null)
  // learned-proposal mode (null otherwise): tile segments and their proposal CDF
  const double* seg_cdf;
  const int32_t* seg_edge;
  const float2* seg_s;
  const double* seg_len;
  // secondary edge hierarchy (Sec. 5.3.1), when built: internal nodes and
  // leaf records in key order (layouts in edge_tree.cuh)
  const float4* et_nodes;
  const float4* et_leaf;
  const float4* et_light;  // sphere around the light triangles (centre, padded radius), or null
  int n_seg;
  int V, T, L, E, W, H, cam_type, root;
  int et_root;  // 0: node 0; ~0: a single leaf; -1: not built
};

// Work counters (enabled per launch): rays traced by trace_closest, rays
// traced by trace_any, BVH nodes visited (two boxes each), triangle tests.
enum { kCntClosest = 0, kCntAny = 1, kCntNodes = 2, kCntTris = 3 };
// `rays` = rays this lane traced in the query (0, 1 or 2).
__device__ __forceinline__ void count_trace(const SceneView& s, int kind, int rays, int nodes, int tris) {
  if (s.counters == nullptr) return;
  unsigned m = __activemask();
  int lead = __ffs(m) - 1;
  unsigned nr = __reduce_add_sync(m, (unsigned)rays);
  unsigned tn = __reduce_add_sync(m, (unsigned)nodes), tt = __reduce_add_sync(m, (unsigned)tris);
  if ((int)(threadIdx.x & 31) == lead) {
    atomicAdd(s.counters + kind, (unsigned long long)nr);
    atomicAdd(s.counters + kCntNodes, (unsigned long long)tn);
    atomicAdd(s.counters + kCntTris, (unsigned long long)tt);
  }
}

struct Opts {
  int spp, edge_spp, max_depth, primary_only, terms, proposal;
  uint2 key;
  uint32_t scene_id;  // fourth Philox counter word (the scene's index in a batch)
  int sec_sampler;    // secondary edge: 0 by 3D length, 1 through the edge hierarchy
  int sec_samples;    // root samples of the hierarchy
  int sec_point;      // point on a secondary edge: 0 uniform, 1 clamped-cosine arc density mixed with uniform
  float eps_rel;
  float* seg_log;  // learned proposal training data: |w.(f_u - f_l)| summed per segment (or null)
  // debug restriction of the backward pass to sample ranges (full range by default)
  int pix_begin, pix_end;
  int64_t edge_begin, edge_end;
  int aov;  // with primary_only: 0, 1 albedo; 2 world position; 3 unit shading normal; 4 distance from the ray origin
  // next-event estimation for edges (Sec. 5.3.3): billboard half width, given
  // (nee_hw > 0) or computed on the device into *nee_hw_dev
  int nee;
  float nee_hw;
  const float* nee_hw_dev;
  // per-pixel gradient image of up to 8 parameters (n = 0: none)
  struct {
    float* out;         // [n, H, W]
    int n, npix;
    int64_t v3, t3;     // 3V, 3T: the albedo and global parameters start at v3 and v3 + t3
    int64_t param[8];   // flat parameter indices
  } jac;
};

// Passes of a batch, in launch order (a batch queues its secondary edge
// samples, so its secondary pass has no items).
enum BatchPhase { kPhaseRender = 0, kPhaseInterior = 1, kPhaseSecondary = 2, kPhasePath = 3, kPhasePrimary = 4,
                  kPhases = 5 };

// One scene of a batch (device array, one entry per scene): its view, its
// options and where its outputs go.  The persistent batch kernels copy the
// entry of the scene they work on into shared memory.
struct BatchScene {
  SceneView v;
  Opts op;
  float* image;            // [H,W,3]
  int32_t* tape_tri;       // this scene's tape (W*H*spp entries per bounce)
  float2* tape_bary;
  const float* d_image;    // [H,W,3] loss adjoint, or null (no backward pass)
  float* d_verts;
  float* d_albedo;
  float* partials;         // this scene's rows: interior rows, then primary edge rows
  float* d_radiance;
  float* d_cam;
  float* d_scale;
  const int32_t* order;    // screen order of the primary edge samples (null: sample order)
  int64_t rows_i;          // interior rows (0 when no pixel pass of the backward runs)
  int64_t n_edge;          // primary edge samples
  int64_t per_thread;      // primary edge samples per thread and virtual block
  int64_t blocks_e;        // primary edge virtual blocks
  int G;                   // lanes per pixel
  int rows_written;        // the secondary pass adds to rows the interior pass wrote
  int do_int;              // the pixel pass adds the interior term (else only secondary adjoints)
  int pad_;
  // secondary edge samples that need rays, queued and traced apart
  float* dp_sec;                  // [W*H*spp, depth] adjoint of each path vertex from its secondary sample
  unsigned long long* sec_queue;  // (sample << 3 | vertex) of the queued samples
  unsigned long long* sec_count;  // number queued per region [16]: region b < depth holds vertex b's samples in slots
                                  // [b n, b n + count); with next-event estimation for edges region depth + b
                                  // holds vertex b's billboard samples
  int2* sec_pick;                 // hierarchy sampler: (edge, weight bits) of each queued sample, or null
  int4* sec_nee;                  // next-event estimation for edges: (edge, weight bits, t bits, 0) per slot, or null
  int64_t sec_cap;                // queue capacity = W*H*spp*depth
  // beyond depth 1, the queued samples in stages (null: one fused kernel)
  int4* sec_hits;                 // [sec_cap, 2] side hits (tri, b1, b2, flags) per queue slot
  float* sec_lr;                  // [sec_cap, 6] radiance along the two continuation paths
  float4* sec_path[2];            // [sec_path_cap, 5] continuation states, ping-pong between bounces
  unsigned long long* sec_path_count;  // [2] entries in sec_path[0], sec_path[1]
  int64_t sec_path_cap;           // entries each state buffer holds = W*H*spp*(depth-1)
  // traversal pools of the continuation stages (null: the one-kernel continuation)
  float4* pool_crec;
  int4* pool_hits;
  float4* pool_arec;
  int* pool_occ;
  unsigned long long* pool_next;
  int64_t pool_cap;
};


__device__ __forceinline__ void raise_flag(int* err, int code, int info) {
  if (atomicCAS(err, 0, code) == 0) err[1] = info;
}

__device__ __forceinline__ const float* vtx(const SceneView& s, int i) { return s.verts + 3 * i; }

// ---------------------------------------------------------------------------
// FP32 decision path
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sincos_2pi(float r, float* c_out, float* s_out);

// atan2(y, x) for y >= 0, in [0, pi], FP32 with one rounding per operation
// in a fixed order (no library call: the fisheye's screen points are
// decisions): the ratio of the smaller to the larger magnitude in [0, 1];
// above tan(pi/12) reduced by atan(a) = pi/6 + atan((sqrt(3) a - 1) / (a +
// sqrt(3))); the Taylor series of atan about 0 to z^13 (coefficients
// (-1)^k / (2k + 1)) by Horner's rule; then the octant restored.
__device__ __forceinline__ float atan2_pos(float y, float x) {
  float ax = fabsf(x);
  bool swap = y > ax;
  float num = swap ? ax : y, den = swap ? y : ax;
  float a = den > 0.0f ? fdv(num, den) : 0.0f;
  bool red = a > 0.267949194f;
  float z = red ? fdv(fs(fm(a, 1.73205078f), 1.0f), fa(a, 1.73205078f)) : a;
  float z2 = fm(z, z);
  float p = 0.0769230798f;
  p = fa(fm(z2, p), -0.0909090936f);
  p = fa(fm(z2, p), 0.111111112f);
  p = fa(fm(z2, p), -0.142857149f);
  p = fa(fm(z2, p), 0.200000003f);
  p = fa(fm(z2, p), -0.333333343f);
  float r = fa(z, fm(fm(z, z2), p));
  if (red) r = fa(0.523598790f, r);
  if (swap) r = fs(1.57079637f, r);
  if (x < 0.0f) r = fs(3.14159274f, r);
  return r;
}

// Camera ray through screen point (sx, sy), pixel units, y down.  Pinhole
// and orthographic cameras map lines to lines (Sec. 5.2.1); the equidistant
// fisheye (Sec. 5.2, non-linear projections) sends the screen point at
// distance r from the centre, in units of half the image height, along the
// direction at angle r * cam_scale from the optical axis (-z).
__device__ __forceinline__ void camera_ray(const SceneView& s, float sx, float sy, float o[3], float d[3]) {
  const float* M = s.cam;
  float S = s.cam_scale[0];
  float fw = (float)s.W, fh = (float)s.H;
  float xn = fdv(fs(fm(2.0f, sx), fw), fw);
  float yn = fdv(fs(fh, fm(2.0f, sy)), fh);
  float aspect = fdv(fw, fh);
  if (s.cam_type == 2) {
    float a = fm(xn, aspect), b = yn;
    float r = fsq(fa(fm(a, a), fm(b, b)));
    float th = fm(r, S);
    float c, sn;
    sincos_2pi(fm(th, 0.159154937f), &c, &sn);
    float k = r > 0.0f ? fdv(sn, r) : 0.0f;
    float dc0 = fm(a, k), dc1 = fm(b, k), dc2 = -c;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      o[i] = M[4 * i + 3];
      d[i] = fa(fa(fm(M[4 * i], dc0), fm(M[4 * i + 1], dc1)), fm(M[4 * i + 2], dc2));
    }
    return;
  }
  float sxs = fm(aspect, S);
  float lx = fm(xn, sxs), ly = fm(yn, S);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float m0 = M[4 * i], m1 = M[4 * i + 1], m2 = M[4 * i + 2], m3 = M[4 * i + 3];
    if (s.cam_type == 1) {
      o[i] = m3;
      d[i] = fs(fa(fm(m0, lx), fm(m1, ly)), m2);
    } else {
      o[i] = fa(fa(fm(m0, lx), fm(m1, ly)), m3);
      d[i] = -m2;
    }
  }
}

// Equidistant fisheye projection of a world point (the inverse of
// camera_ray for cam_type 2); false near the direction opposite the optical
// axis (theta >= 3.1), which no pixel sees.
__device__ __forceinline__ bool fisheye_project(const SceneView& s, const float v[3], float* sx, float* sy) {
  const float* Wm = s.w2c;
  float vc[3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    vc[i] = fa(fa(fa(fm(Wm[4 * i], v[0]), fm(Wm[4 * i + 1], v[1])), fm(Wm[4 * i + 2], v[2])), Wm[4 * i + 3]);
  float rho = fsq(fa(fm(vc[0], vc[0]), fm(vc[1], vc[1])));
  float th = atan2_pos(rho, -vc[2]);
  if (!(th < 3.1f)) return false;
  float S = s.cam_scale[0];
  float k = rho > 0.0f ? fdv(th, fm(S, rho)) : 0.0f;
  float a = fm(k, vc[0]), b = fm(k, vc[1]);
  float fw = (float)s.W, fh = (float)s.H;
  float xn = fdv(a, fdv(fw, fh));
  *sx = fm(fa(xn, 1.0f), fm(0.5f, fw));
  *sy = fm(fs(1.0f, b), fm(0.5f, fh));
  return true;
}

// Screen projection with the FP32 world-to-camera rows; false if behind.
__device__ __forceinline__ bool project(const SceneView& s, const float v[3], float* sx, float* sy) {
  const float* Wm = s.w2c;
  float vc[3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
    vc[i] = fa(fa(fa(fm(Wm[4 * i], v[0]), fm(Wm[4 * i + 1], v[1])), fm(Wm[4 * i + 2], v[2])), Wm[4 * i + 3]);
  if (!(vc[2] < -kNearZ)) return false;
  float S = s.cam_scale[0];
  float fw = (float)s.W, fh = (float)s.H;
  float aspect = fdv(fw, fh);
  float px = vc[0], py = vc[1];
  if (s.cam_type == 1) {
    float iz = -vc[2];
    px = fdv(vc[0], iz);
    py = fdv(vc[1], iz);
  }
  float xn = fdv(px, fm(aspect, S));
  float yn = fdv(py, S);
  *sx = fm(fa(xn, 1.0f), fm(0.5f, fw));
  *sy = fm(fs(1.0f, yn), fm(0.5f, fh));
  return true;
}

// Liang-Barsky clip to [0,W]x[0,H]; planes x>=0, x<=W, y>=0, y<=H.
__device__ __forceinline__ bool clip_screen(float ax, float ay, float bx, float by, float W, float H, float* t0o,
                                            float* t1o) {
  float dx = fs(bx, ax), dy = fs(by, ay);
  float t0 = 0.0f, t1 = 1.0f;
  float p[4] = {-dx, dx, -dy, dy};
  float q[4] = {ax, fs(W, ax), ay, fs(H, ay)};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (p[k] == 0.0f) {
      if (q[k] < 0.0f) return false;
      continue;
    }
    float r = fdv(q[k], p[k]);
    if (p[k] < 0.0f) {
      if (r > t0) t0 = r;
    } else {
      if (r < t1) t1 = r;
    }
  }
  if (!(t0 < t1)) return false;
  *t0o = t0;
  *t1o = t1;
  return true;
}

// Upper bound in an inclusive CDF; falls back to the last entry with mass.
// Guide tables of the edge CDFs: g[b] = cdf_pick's answer for the target
// b * total / kGuide (b < kGuide), g[kGuide] = n.
constexpr int kGuide = 1024;

__device__ __forceinline__ int cdf_pick(const double* cdf, int n, double target) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cdf[mid] > target) hi = mid; else lo = mid + 1;
  }
  if (lo >= n) {
    lo = n - 1;
    while (lo > 0 && cdf[lo] == cdf[lo - 1]) --lo;
  }
  return lo;
}

// cdf_pick with the search narrowed by a guide table (same answer): the
// target's bucket, computed to within one bucket, and its neighbours bound
// the first index whose value exceeds the target (the thresholds of buckets
// b - 1 and b + 2 lie below and above it; the answer is monotone).
__device__ __forceinline__ int cdf_pick_guided(const double* cdf, int n, double target, const int* guide,
                                               double total) {
  int b = (int)(target * ((double)kGuide / total));
  b = min(max(b, 0), kGuide - 1);
  int lo = guide[max(b - 1, 0)], hi = guide[min(b + 2, kGuide)];
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cdf[mid] > target) hi = mid; else lo = mid + 1;
  }
  if (lo >= n) {
    lo = n - 1;
    while (lo > 0 && cdf[lo] == cdf[lo - 1]) --lo;
  }
  return lo;
}

// Watertight ray/triangle test (Woop, Benthin, Wald 2013), FP32.
struct Shear {
  unsigned char kx, ky, kz;
  float Sx, Sy, Sz;
};
__device__ __forceinline__ Shear make_shear(const float d[3]) {
  int kz = 0;
  if (fabsf(d[1]) > fabsf(d[kz])) kz = 1;
  if (fabsf(d[2]) > fabsf(d[kz])) kz = 2;
  int kx = kz + 1;
  if (kx == 3) kx = 0;
  int ky = kx + 1;
  if (ky == 3) ky = 0;
  if (d[kz] < 0.0f) {
    int t = kx; kx = ky; ky = t;
  }
  Shear sh;
  sh.kx = kx; sh.ky = ky; sh.kz = kz;
  sh.Sx = fdv(d[kx], d[kz]);
  sh.Sy = fdv(d[ky], d[kz]);
  sh.Sz = fdv(1.0f, d[kz]);
  return sh;
}
__device__ __forceinline__ float comp(const float3& v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ __forceinline__ bool watertight(const Shear& sh, const float o[3], float3 v0, float3 v1, float3 v2,
                                           float tmax, float* t_out, float* b1_out, float* b2_out) {
  float3 A = make_float3(fs(v0.x, o[0]), fs(v0.y, o[1]), fs(v0.z, o[2]));
  float3 B = make_float3(fs(v1.x, o[0]), fs(v1.y, o[1]), fs(v1.z, o[2]));
  float3 C = make_float3(fs(v2.x, o[0]), fs(v2.y, o[1]), fs(v2.z, o[2]));
  float Akz = comp(A, sh.kz), Bkz = comp(B, sh.kz), Ckz = comp(C, sh.kz);
  float Ax = fs(comp(A, sh.kx), fm(sh.Sx, Akz)), Ay = fs(comp(A, sh.ky), fm(sh.Sy, Akz));
  float Bx = fs(comp(B, sh.kx), fm(sh.Sx, Bkz)), By = fs(comp(B, sh.ky), fm(sh.Sy, Bkz));
  float Cx = fs(comp(C, sh.kx), fm(sh.Sx, Ckz)), Cy = fs(comp(C, sh.ky), fm(sh.Sy, Ckz));
  float U = fs(fm(Cx, By), fm(Cy, Bx));
  float V = fs(fm(Ax, Cy), fm(Ay, Cx));
  float Wv = fs(fm(Bx, Ay), fm(By, Ax));
  if ((U < 0.0f || V < 0.0f || Wv < 0.0f) && (U > 0.0f || V > 0.0f || Wv > 0.0f)) return false;
  float det = fa(fa(U, V), Wv);
  if (det == 0.0f) return false;
  float Az = fm(sh.Sz, Akz), Bz = fm(sh.Sz, Bkz), Cz = fm(sh.Sz, Ckz);
  float T = fa(fa(fm(U, Az), fm(V, Bz)), fm(Wv, Cz));
  float t = fdv(T, det);
  if (!(t > 0.0f && t < tmax)) return false;
  *t_out = t;
  *b1_out = fdv(V, det);
  *b2_out = fdv(Wv, det);
  return true;
}

__device__ __forceinline__ void bary_point(float3 v0, float3 v1, float3 v2, float b1, float b2, float p[3]) {
  float b0 = fs(fs(1.0f, b1), b2);
  p[0] = fa(fa(fm(b0, v0.x), fm(b1, v1.x)), fm(b2, v2.x));
  p[1] = fa(fa(fm(b0, v0.y), fm(b1, v1.y)), fm(b2, v2.y));
  p[2] = fa(fa(fm(b0, v0.z), fm(b1, v1.z)), fm(b2, v2.z));
}
__device__ __forceinline__ void face_normal(float3 v0, float3 v1, float3 v2, float n[3]) {
  float e1x = fs(v1.x, v0.x), e1y = fs(v1.y, v0.y), e1z = fs(v1.z, v0.z);
  float e2x = fs(v2.x, v0.x), e2y = fs(v2.y, v0.y), e2z = fs(v2.z, v0.z);
  n[0] = fs(fm(e1y, e2z), fm(e1z, e2y));
  n[1] = fs(fm(e1z, e2x), fm(e1x, e2z));
  n[2] = fs(fm(e1x, e2y), fm(e1y, e2x));
}

// Own sin/cos of 2*pi*r: quadrant from 4r, Taylor series of sin and cos on
// [0, pi/2) by Horner's rule (coefficients 1/n!).
__device__ __forceinline__ void sincos_2pi(float r, float* c_out, float* s_out) {
  float q4 = fm(r, 4.0f);
  int q = (int)q4;
  if (q > 3) q = 3;
  float f = fs(q4, (float)q);
  float a = fm(f, 1.57079637f);
  float a2 = fm(a, a);
  float s = fm(a2, 1.60590444e-10f);
  s = fm(a2, fs(s, 2.50521084e-08f));
  s = fm(a2, fa(s, 2.75573192e-06f));
  s = fm(a2, fs(s, 1.98412698e-04f));
  s = fm(a2, fa(s, 8.33333377e-03f));
  s = fm(a2, fs(s, 1.66666672e-01f));
  s = fa(a, fm(a, s));
  float c = fm(a2, -1.14707454e-11f);
  c = fm(a2, fa(c, 2.08767570e-09f));
  c = fm(a2, fs(c, 2.75573192e-07f));
  c = fm(a2, fa(c, 2.48015876e-05f));
  c = fm(a2, fs(c, 1.38888892e-03f));
  c = fm(a2, fa(c, 4.16666679e-02f));
  c = fm(a2, fs(c, 0.5f));
  c = fa(1.0f, c);
  if (q == 0) { *c_out = c; *s_out = s; }
  else if (q == 1) { *c_out = -s; *s_out = c; }
  else if (q == 2) { *c_out = -c; *s_out = -s; }
  else { *c_out = s; *s_out = -c; }
}

// Cosine-weighted direction around unit normal n; basis of Duff et al.,
// "Building an Orthonormal Basis, Revisited" (JCGT 2017).
__device__ __forceinline__ void cosine_dir(const float n[3], float r1, float r2, float out[3]) {
  float rr = fsq(r1);
  float c, s;
  sincos_2pi(r2, &c, &s);
  float lx = fm(rr, c), ly = fm(rr, s);
  float lz = fsq(fmaxf(0.0f, fs(1.0f, r1)));
  float sgn = copysignf(1.0f, n[2]);
  float a = fdv(-1.0f, fa(sgn, n[2]));
  float bb = fm(fm(n[0], n[1]), a);
  float t[3] = {fa(1.0f, fm(fm(fm(sgn, n[0]), n[0]), a)), fm(sgn, bb), -fm(sgn, n[0])};
  float bt[3] = {bb, fa(sgn, fm(fm(n[1], n[1]), a)), -n[1]};
#pragma unroll
  for (int i = 0; i < 3; ++i) out[i] = fa(fa(fm(lx, t[i]), fm(ly, bt[i])), fm(lz, n[i]));
}

// ---------------------------------------------------------------------------
// BVH traversal (BVH2, 64-byte nodes, stack in registers/local memory)
// ---------------------------------------------------------------------------
// Node n: f4[4n+0] = (loL.xyz, hiL.x), f4[4n+1] = (hiL.yz, loR.xy),
//         f4[4n+2] = (loR.z, hiR.xyz), f4[4n+3] = (childL, childR, -, -) as int.
// child >= 0: internal node; child < 0: leaf range (see leaf_enc).
// Boxes are enlarged when built so the slab test below never rejects a ray
// that the watertight test would accept.
struct Hit {
  int tri;
  float t, b1, b2;
};

// Three-input minimum / maximum (one instruction on sm_100 and later; exact,
// like the two-input forms).
__device__ __forceinline__ float fmax3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float fmin3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

struct RayPre {
  float o[3], inv[3];
  Shear sh;
};
__device__ __forceinline__ void ray_pre(RayPre& r, const float o[3], const float d[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r.o[i] = o[i];
    float di = fabsf(d[i]) < 1e-20f ? copysignf(1e-20f, d[i]) : d[i];
    r.inv[i] = 1.0f / di;
  }
  r.sh = make_shear(d);
}

__device__ __forceinline__ void slab2(const RayPre& r, const float4& a, const float4& b, const float4& c, float tmax,
                                      float* tl, bool* hl, float* tr, bool* hr) {
  // left box: lo=(a.x,a.y,a.z) hi=(a.w,b.x,b.y); right: lo=(b.z,b.w,c.x) hi=(c.y,c.z,c.w)
  float lx0 = (a.x - r.o[0]) * r.inv[0], lx1 = (a.w - r.o[0]) * r.inv[0];
  float ly0 = (a.y - r.o[1]) * r.inv[1], ly1 = (b.x - r.o[1]) * r.inv[1];
  float lz0 = (a.z - r.o[2]) * r.inv[2], lz1 = (b.y - r.o[2]) * r.inv[2];
  float tin = fmax3f(fminf(lx0, lx1), fminf(ly0, ly1), fmaxf(fminf(lz0, lz1), 0.0f));
  float tout = fmin3f(fmaxf(lx0, lx1), fmaxf(ly0, ly1), fminf(fmaxf(lz0, lz1), tmax));
  *tl = tin;
  *hl = tin <= tout * 1.00000024f;
  float rx0 = (b.z - r.o[0]) * r.inv[0], rx1 = (c.y - r.o[0]) * r.inv[0];
  float ry0 = (b.w - r.o[1]) * r.inv[1], ry1 = (c.z - r.o[1]) * r.inv[1];
  float rz0 = (c.x - r.o[2]) * r.inv[2], rz1 = (c.w - r.o[2]) * r.inv[2];
  float tin2 = fmax3f(fminf(rx0, rx1), fminf(ry0, ry1), fmaxf(fminf(rz0, rz1), 0.0f));
  float tout2 = fmin3f(fmaxf(rx0, rx1), fmaxf(ry0, ry1), fminf(fmaxf(rz0, rz1), tmax));
  *tr = tin2;
  *hr = tin2 <= tout2 * 1.00000024f;
}

// Closest hit with t in (0, tmax); ties on t go to the lowest triangle id;
// triangle `exclude` is skipped.  Returns tri = -1 on a miss.
__device__ __forceinline__ Hit trace_closest(const SceneView& s, const float o[3], const float d[3], float tmax,
                                             int exclude) {
  RayPre r;
  ray_pre(r, o, d);
  Hit h;
  h.tri = -1;
  h.t = tmax;
  h.b1 = h.b2 = 0.0f;
  int stack[kStackSize];
  int sp = 0;
  int node = s.root;
  // a tree has 2T-1 nodes and leaves, each visited at most once
  int budget = 2 * s.T + 8;
  int n_nodes = 0, n_tris = 0;
  while (true) {
    if (--budget < 0) {
      raise_flag(s.err, DRT_DEV_TRAVERSAL_CAP, s.T);
      break;
    }
    if (node >= 0) {
      ++n_nodes;
      const float4* n4 = s.nodes + 4 * node;
      float4 a = __ldg(n4), b = __ldg(n4 + 1), c = __ldg(n4 + 2);
      int4 ch = __ldg(reinterpret_cast<const int4*>(n4 + 3));
      float tl, tr;
      bool hl, hr;
      slab2(r, a, b, c, h.t, &tl, &hl, &tr, &hr);
      if (hl && hr) {
        int nearc = tl <= tr ? ch.x : ch.y, farc = tl <= tr ? ch.y : ch.x;
        if (sp < kStackSize) {
          stack[sp++] = farc;
        } else {
          raise_flag(s.err, DRT_DEV_STACK_OVERFLOW, node);
        }
        node = nearc;
        continue;
      } else if (hl) {
        node = ch.x;
        continue;
      } else if (hr) {
        node = ch.y;
        continue;
      }
    } else {
      int enc = ~node, first = enc & 0x0fffffff, count = (enc >> 28) + 1;
      for (int q = 0; q < count; ++q) {
        const float4* t4 = s.soup + 3 * (first + q);
        float4 p0 = __ldg(t4), p1 = __ldg(t4 + 1), p2 = __ldg(t4 + 2);
        int id = __float_as_int(p0.w);
        ++n_tris;
        if (id != exclude) {
          float t, b1, b2;
          // t must beat the best so far; a lower id also wins a tie on t
          float lim = (h.tri >= 0 && id < h.tri) ? __uint_as_float(__float_as_uint(h.t) + 1u) : h.t;
          if (watertight(r.sh, r.o, make_float3(p0.x, p0.y, p0.z), make_float3(p1.x, p1.y, p1.z),
                         make_float3(p2.x, p2.y, p2.z), lim, &t, &b1, &b2)) {
            h.tri = id; h.t = t; h.b1 = b1; h.b2 = b2;
          }
        }
      }
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  count_trace(s, kCntClosest, 1, n_nodes, n_tris);
  return h;
}

// Any hit with t in (0, tmax), skipping two triangle ids.
__device__ __forceinline__ bool trace_any(const SceneView& s, const float o[3], const float d[3], float tmax, int ex0,
                                          int ex1) {
  RayPre r;
  ray_pre(r, o, d);
  int stack[kStackSize];
  int sp = 0;
  int node = s.root;
  int budget = 2 * s.T + 8;
  int n_nodes = 0, n_tris = 0;
  bool found = false;
  while (true) {
    if (--budget < 0) {
      raise_flag(s.err, DRT_DEV_TRAVERSAL_CAP, s.T);
      break;
    }
    if (node >= 0) {
      ++n_nodes;
      const float4* n4 = s.nodes + 4 * node;
      float4 a = __ldg(n4), b = __ldg(n4 + 1), c = __ldg(n4 + 2);
      int4 ch = __ldg(reinterpret_cast<const int4*>(n4 + 3));
      float tl, tr;
      bool hl, hr;
      slab2(r, a, b, c, tmax, &tl, &hl, &tr, &hr);
      if (hl && hr) {
        if (sp < kStackSize) stack[sp++] = ch.y; else raise_flag(s.err, DRT_DEV_STACK_OVERFLOW, node);
        node = ch.x;
        continue;
      } else if (hl) {
        node = ch.x;
        continue;
      } else if (hr) {
        node = ch.y;
        continue;
      }
    } else {
      int enc = ~node, first = enc & 0x0fffffff, count = (enc >> 28) + 1;
      for (int q = 0; q < count && !found; ++q) {
        const float4* t4 = s.soup + 3 * (first + q);
        float4 p0 = __ldg(t4), p1 = __ldg(t4 + 1), p2 = __ldg(t4 + 2);
        int id = __float_as_int(p0.w);
        ++n_tris;
        if (id != ex0 && id != ex1) {
          float t, b1, b2;
          if (watertight(r.sh, r.o, make_float3(p0.x, p0.y, p0.z), make_float3(p1.x, p1.y, p1.z),
                         make_float3(p2.x, p2.y, p2.z), tmax, &t, &b1, &b2))
            found = true;
        }
      }
      if (found) break;
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  count_trace(s, kCntAny, 1, n_nodes, n_tris);
  return found;
}

// Two rays through one traversal: a node is visited when either active ray
// (with its own current closest t) enters one of its boxes, and every leaf
// triangle is tested against each active ray with that ray's own limits, so
// each result equals the ray's single traversal.  Used for the two side paths
// of an edge sample, which are a tiny offset apart and visit the same nodes.
__device__ __forceinline__ void trace_closest2(const SceneView& s, const float o0[3], const float d0[3],
                                               const float o1[3], const float d1[3], bool act0, bool act1, int ex0,
                                               int ex1, Hit& h0, Hit& h1) {
  RayPre r0, r1;
  ray_pre(r0, o0, d0);
  ray_pre(r1, o1, d1);
  h0.tri = -1; h0.t = INFINITY; h0.b1 = h0.b2 = 0.f;
  h1.tri = -1; h1.t = INFINITY; h1.b1 = h1.b2 = 0.f;
  if (!act0 && !act1) return;
  int stack[kStackSize];
  int sp = 0;
  int node = s.root;
  int budget = 2 * s.T + 8;
  int n_nodes = 0, n_tris = 0;
  while (true) {
    if (--budget < 0) {
      raise_flag(s.err, DRT_DEV_TRAVERSAL_CAP, s.T);
      break;
    }
    if (node >= 0) {
      ++n_nodes;
      const float4* n4 = s.nodes + 4 * node;
      float4 a = __ldg(n4), b = __ldg(n4 + 1), c = __ldg(n4 + 2);
      int4 ch = __ldg(reinterpret_cast<const int4*>(n4 + 3));
      float tl0, tr0, tl1, tr1;
      bool hl0, hr0, hl1, hr1;
      slab2(r0, a, b, c, h0.t, &tl0, &hl0, &tr0, &hr0);
      slab2(r1, a, b, c, h1.t, &tl1, &hl1, &tr1, &hr1);
      bool hl = (act0 && hl0) || (act1 && hl1), hr = (act0 && hr0) || (act1 && hr1);
      float tl = fminf(act0 && hl0 ? tl0 : INFINITY, act1 && hl1 ? tl1 : INFINITY);
      float tr = fminf(act0 && hr0 ? tr0 : INFINITY, act1 && hr1 ? tr1 : INFINITY);
      if (hl && hr) {
        int nearc = tl <= tr ? ch.x : ch.y, farc = tl <= tr ? ch.y : ch.x;
        if (sp < kStackSize) stack[sp++] = farc; else raise_flag(s.err, DRT_DEV_STACK_OVERFLOW, node);
        node = nearc;
        continue;
      } else if (hl) {
        node = ch.x;
        continue;
      } else if (hr) {
        node = ch.y;
        continue;
      }
    } else {
      int enc = ~node, first = enc & 0x0fffffff, count = (enc >> 28) + 1;
      for (int q = 0; q < count; ++q) {
      const float4* t4 = s.soup + 3 * (first + q);
      float4 p0 = __ldg(t4), p1 = __ldg(t4 + 1), p2 = __ldg(t4 + 2);
      int id = __float_as_int(p0.w);
      ++n_tris;
      float3 v0 = make_float3(p0.x, p0.y, p0.z), v1 = make_float3(p1.x, p1.y, p1.z), v2 = make_float3(p2.x, p2.y, p2.z);
      float t, b1, b2;
      if (act0 && id != ex0) {
        float lim = (h0.tri >= 0 && id < h0.tri) ? __uint_as_float(__float_as_uint(h0.t) + 1u) : h0.t;
        if (watertight(r0.sh, r0.o, v0, v1, v2, lim, &t, &b1, &b2)) { h0.tri = id; h0.t = t; h0.b1 = b1; h0.b2 = b2; }
      }
      if (act1 && id != ex1) {
        float lim = (h1.tri >= 0 && id < h1.tri) ? __uint_as_float(__float_as_uint(h1.t) + 1u) : h1.t;
        if (watertight(r1.sh, r1.o, v0, v1, v2, lim, &t, &b1, &b2)) { h1.tri = id; h1.t = t; h1.b1 = b1; h1.b2 = b2; }
      }
      }
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  count_trace(s, kCntClosest, (int)act0 + (int)act1, n_nodes, n_tris);
}

// Two any-hit queries through one traversal; occ0/occ1 report a hit with t in
// (0, tmax) that is not one of the ray's two skipped triangles.
__device__ __forceinline__ void trace_any2(const SceneView& s, const float o0[3], const float d0[3], int a0x, int a0y,
                                           const float o1[3], const float d1[3], int a1x, int a1y, bool act0,
                                           bool act1, float tmax, bool& occ0, bool& occ1) {
  occ0 = occ1 = false;
  if (!act0 && !act1) return;
  RayPre r0, r1;
  ray_pre(r0, o0, d0);
  ray_pre(r1, o1, d1);
  bool live0 = act0, live1 = act1;
  int stack[kStackSize];
  int sp = 0;
  int node = s.root;
  int budget = 2 * s.T + 8;
  int n_nodes = 0, n_tris = 0;
  while (live0 || live1) {
    if (--budget < 0) {
      raise_flag(s.err, DRT_DEV_TRAVERSAL_CAP, s.T);
      break;
    }
    if (node >= 0) {
      ++n_nodes;
      const float4* n4 = s.nodes + 4 * node;
      float4 a = __ldg(n4), b = __ldg(n4 + 1), c = __ldg(n4 + 2);
      int4 ch = __ldg(reinterpret_cast<const int4*>(n4 + 3));
      float tl, tr;
      bool hl0 = false, hr0 = false, hl1 = false, hr1 = false;
      if (live0) slab2(r0, a, b, c, tmax, &tl, &hl0, &tr, &hr0);
      if (live1) slab2(r1, a, b, c, tmax, &tl, &hl1, &tr, &hr1);
      bool hl = hl0 || hl1, hr = hr0 || hr1;
      if (hl && hr) {
        if (sp < kStackSize) stack[sp++] = ch.y; else raise_flag(s.err, DRT_DEV_STACK_OVERFLOW, node);
        node = ch.x;
        continue;
      } else if (hl) {
        node = ch.x;
        continue;
      } else if (hr) {
        node = ch.y;
        continue;
      }
    } else {
      int enc = ~node, first = enc & 0x0fffffff, count = (enc >> 28) + 1;
      for (int q = 0; q < count && (live0 || live1); ++q) {
        const float4* t4 = s.soup + 3 * (first + q);
        float4 p0 = __ldg(t4), p1 = __ldg(t4 + 1), p2 = __ldg(t4 + 2);
        int id = __float_as_int(p0.w);
        ++n_tris;
        float3 v0 = make_float3(p0.x, p0.y, p0.z), v1 = make_float3(p1.x, p1.y, p1.z),
               v2 = make_float3(p2.x, p2.y, p2.z);
        float t, b1, b2;
        if (live0 && id != a0x && id != a0y && watertight(r0.sh, r0.o, v0, v1, v2, tmax, &t, &b1, &b2)) {
          occ0 = true;
          live0 = false;
        }
        if (live1 && id != a1x && id != a1y && watertight(r1.sh, r1.o, v0, v1, v2, tmax, &t, &b1, &b2)) {
          occ1 = true;
          live1 = false;
        }
      }
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  count_trace(s, kCntAny, (int)act0 + (int)act1, n_nodes, n_tris);
}

// ---------------------------------------------------------------------------
// Warp-cooperative traversals.  The 32 lanes of a warp walk one tree
// traversal together: the union of the nodes their rays enter, in one order,
// with one stack in shared memory.  Control flow is uniform across the warp
// and every node is one broadcast load.  Each lane tracks whether its own
// rays enter the current node (a bit per stack entry) and tests only those
// boxes and triangles.  The results equal the per-lane traversals: the
// closest hit with ties to the lowest id, and the existence of an occluder,
// do not depend on the order in which nodes are visited.  All 32 lanes must
// call together, converged, in a CTA of at most kTraceWarps warps.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void trace_closest2_warp(const SceneView& s, const float o0[3], const float d0[3],
                                                    const float o1[3], const float d1[3], bool act0, bool act1,
                                                    int ex0, int ex1, Hit& h0, Hit& h1) {
  __shared__ int wstack[kTraceWarps][kStackSize];
  int* stk = wstack[threadIdx.x >> 5];
  const unsigned full = 0xffffffffu;
  const bool lane0 = (threadIdx.x & 31) == 0;
  RayPre r0, r1;
  ray_pre(r0, o0, d0);
  ray_pre(r1, o1, d1);
  h0.tri = -1; h0.t = INFINITY; h0.b1 = h0.b2 = 0.f;
  h1.tri = -1; h1.t = INFINITY; h1.b1 = h1.b2 = 0.f;
  if (!__any_sync(full, act0 || act1)) return;
  bool in = act0 || act1;       // this lane's rays enter the current node
  unsigned long long in_stk = 0;  // the same for every stacked node (bit = stack slot)
  int sp = 0;
  int node = s.root;
  int budget = 2 * s.T + 8;
  int n_nodes = 0, n_tris = 0;
  while (true) {
    if (--budget < 0) {
      if (lane0) raise_flag(s.err, DRT_DEV_TRAVERSAL_CAP, s.T);
      break;
    }
    if (node >= 0) {
      const float4* n4 = s.nodes + 4 * node;
      float4 a = __ldg(n4), b = __ldg(n4 + 1), c = __ldg(n4 + 2);
      int4 ch = __ldg(reinterpret_cast<const int4*>(n4 + 3));
      float tl0 = INFINITY, tr0 = INFINITY, tl1 = INFINITY, tr1 = INFINITY;
      bool hl0 = false, hr0 = false, hl1 = false, hr1 = false;
      if (in) {
        ++n_nodes;
        if (act0) slab2(r0, a, b, c, h0.t, &tl0, &hl0, &tr0, &hr0);
        if (act1) slab2(r1, a, b, c, h1.t, &tl1, &hl1, &tr1, &hr1);
      }
      bool hl = hl0 || hl1, hr = hr0 || hr1;
      float tl = fminf(hl0 ? tl0 : INFINITY, hl1 ? tl1 : INFINITY);
      float tr = fminf(hr0 ? tr0 : INFINITY, hr1 ? tr1 : INFINITY);
      unsigned ml = __ballot_sync(full, hl), mr = __ballot_sync(full, hr);
      if (ml && mr) {
        // the child most lanes reach first goes first
        unsigned pl = __ballot_sync(full, hl && (!hr || tl <= tr));
        unsigned pr = __ballot_sync(full, hr && (!hl || tr < tl));
        bool left_first = __popc(pl) >= __popc(pr);
        int nearc = left_first ? ch.x : ch.y, farc = left_first ? ch.y : ch.x;
        bool near_in = left_first ? hl : hr, far_in = left_first ? hr : hl;
        if (sp < kStackSize) {
          if (lane0) stk[sp] = farc;
          in_stk = far_in ? (in_stk | (1ull << sp)) : (in_stk & ~(1ull << sp));
          ++sp;
        } else if (lane0) {
          raise_flag(s.err, DRT_DEV_STACK_OVERFLOW, node);
        }
        node = nearc;
        in = near_in;
        continue;
      } else if (ml) {
        node = ch.x;
        in = hl;
        continue;
      } else if (mr) {
        node = ch.y;
        in = hr;
        continue;
      }
    } else if (in) {
      int enc = ~node, first = enc & 0x0fffffff, count = (enc >> 28) + 1;
      for (int q = 0; q < count; ++q) {
        const float4* t4 = s.soup + 3 * (first + q);
        float4 p0 = __ldg(t4), p1 = __ldg(t4 + 1), p2 = __ldg(t4 + 2);
        int id = __float_as_int(p0.w);
        ++n_tris;
        float3 v0 = make_float3(p0.x, p0.y, p0.z), v1 = make_float3(p1.x, p1.y, p1.z),
               v2 = make_float3(p2.x, p2.y, p2.z);
        float t, b1, b2;
        if (act0 && id != ex0) {
          float lim = (h0.tri >= 0 && id < h0.tri) ? __uint_as_float(__float_as_uint(h0.t) + 1u) : h0.t;
          if (watertight(r0.sh, r0.o, v0, v1, v2, lim, &t, &b1, &b2)) { h0.tri = id; h0.t = t; h0.b1 = b1; h0.b2 = b2; }
        }
        if (act1 && id != ex1) {
          float lim = (h1.tri >= 0 && id < h1.tri) ? __uint_as_float(__float_as_uint(h1.t) + 1u) : h1.t;
          if (watertight(r1.sh, r1.o, v0, v1, v2, lim, &t, &b1, &b2)) { h1.tri = id; h1.t = t; h1.b1 = b1; h1.b2 = b2; }
        }
      }
    }
    if (sp == 0) break;
    --sp;
    __syncwarp();
    node = stk[sp];
    in = (in_stk >> sp) & 1ull;
  }
  count_trace(s, kCntClosest, (int)act0 + (int)act1, n_nodes, n_tris);
}

// Warp-cooperative any-hit of two rays per lane (see trace_any2); the warp
// stops when no lane has a ray left to resolve.
__device__ __forceinline__ void trace_any2_warp(const SceneView& s, const float o0[3], const float d0[3], int a0x,
                                                int a0y, const float o1[3], const float d1[3], int a1x, int a1y,
                                                bool act0, bool act1, float tmax, bool& occ0, bool& occ1) {
  __shared__ int wstack[kTraceWarps][kStackSize];
  int* stk = wstack[threadIdx.x >> 5];
  const unsigned full = 0xffffffffu;
  const bool lane0 = (threadIdx.x & 31) == 0;
  occ0 = occ1 = false;
  RayPre r0, r1;
  ray_pre(r0, o0, d0);
  ray_pre(r1, o1, d1);
  bool live0 = act0, live1 = act1;
  bool in = live0 || live1;
  unsigned long long in_stk = 0;
  int sp = 0;
  int node = s.root;
  int budget = 2 * s.T + 8;
  int n_nodes = 0, n_tris = 0;
  while (__any_sync(full, live0 || live1)) {
    if (--budget < 0) {
      if (lane0) raise_flag(s.err, DRT_DEV_TRAVERSAL_CAP, s.T);
      break;
    }
    if (node >= 0) {
      const float4* n4 = s.nodes + 4 * node;
      float4 a = __ldg(n4), b = __ldg(n4 + 1), c = __ldg(n4 + 2);
      int4 ch = __ldg(reinterpret_cast<const int4*>(n4 + 3));
      float tl, tr;
      bool hl0 = false, hr0 = false, hl1 = false, hr1 = false;
      if (in && (live0 || live1)) {
        ++n_nodes;
        if (live0) slab2(r0, a, b, c, tmax, &tl, &hl0, &tr, &hr0);
        if (live1) slab2(r1, a, b, c, tmax, &tl, &hl1, &tr, &hr1);
      }
      bool hl = hl0 || hl1, hr = hr0 || hr1;
      unsigned ml = __ballot_sync(full, hl), mr = __ballot_sync(full, hr);
      if (ml && mr) {
        if (sp < kStackSize) {
          if (lane0) stk[sp] = ch.y;
          in_stk = hr ? (in_stk | (1ull << sp)) : (in_stk & ~(1ull << sp));
          ++sp;
        } else if (lane0) {
          raise_flag(s.err, DRT_DEV_STACK_OVERFLOW, node);
        }
        node = ch.x;
        in = hl;
        continue;
      } else if (ml) {
        node = ch.x;
        in = hl;
        continue;
      } else if (mr) {
        node = ch.y;
        in = hr;
        continue;
      }
    } else if (in) {
      int enc = ~node, first = enc & 0x0fffffff, count = (enc >> 28) + 1;
      for (int q = 0; q < count && (live0 || live1); ++q) {
        const float4* t4 = s.soup + 3 * (first + q);
        float4 p0 = __ldg(t4), p1 = __ldg(t4 + 1), p2 = __ldg(t4 + 2);
        int id = __float_as_int(p0.w);
        ++n_tris;
        float3 v0 = make_float3(p0.x, p0.y, p0.z), v1 = make_float3(p1.x, p1.y, p1.z),
               v2 = make_float3(p2.x, p2.y, p2.z);
        float t, b1, b2;
        if (live0 && id != a0x && id != a0y && watertight(r0.sh, r0.o, v0, v1, v2, tmax, &t, &b1, &b2)) {
          occ0 = true;
          live0 = false;
        }
        if (live1 && id != a1x && id != a1y && watertight(r1.sh, r1.o, v0, v1, v2, tmax, &t, &b1, &b2)) {
          occ1 = true;
          live1 = false;
        }
      }
    }
    if (sp == 0) break;
    --sp;
    __syncwarp();
    node = stk[sp];
    in = (in_stk >> sp) & 1ull;
  }
  count_trace(s, kCntAny, (int)act0 + (int)act1, n_nodes, n_tris);
}

__device__ __forceinline__ float3 ld3(const float* p) { return make_float3(p[0], p[1], p[2]); }

}  // namespace drt
