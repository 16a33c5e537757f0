// render.cu -- forward path tracing with next-event estimation (Eq. first via
// Eq. gradient_monte_carlo), and the backward pass: the reverse sweep over
// the checkpointed path (interior term of Eq. redner_product_rule), secondary
// edge samples at each shading vertex (Eq. dirac_3d_edge, Appendix 5.A,
// Eq. alpha_3d) and primary edge samples (Eq. mc, Eq. redner_dirac_jacobian).
//
// Thread mapping.  A warp owns 32/G pixels, G = min(32, spp rounded up to a
// power of two); lane l works on pixel l/G and samples l%G, l%G+G, ...  The
// 32 rays of a warp start in the same pixel, so traversal is coherent, and
// the per-pixel sum is a fixed-order butterfly (images are bit-reproducible).
#include <cstdio>
#include <cstring>

#include "drt_internal.h"
#include "edge_tree.cuh"
#include "nee_edge.cuh"
#include "trace_pool.cuh"

namespace drt {
namespace {

constexpr int kBlock = 256;
// Resident CTAs per SM the primary edge kernel is compiled for (its register
// cap is 65536 / (kBlock * this)).
#ifndef DRT_PRIMARY_MIN_BLOCKS
#define DRT_PRIMARY_MIN_BLOCKS 4
#endif
// Most blocks of the primary edge kernel: one sample per thread up to this
// many blocks (measured fastest: balanced blocks, no partial last wave), then
// several per thread.
#ifndef DRT_PRIMARY_BLOCK_CAP
#define DRT_PRIMARY_BLOCK_CAP (1 << 20)
#endif
// Resident CTAs per SM the interior and secondary edge passes are compiled for.
#ifndef DRT_PIXEL_MIN_BLOCKS
#define DRT_PIXEL_MIN_BLOCKS 2
#endif
// Screen keys of the primary edge samples resolve 1/DRT_KEY_SUB of a pixel.
#ifndef DRT_KEY_SUB
#define DRT_KEY_SUB 8
#endif
constexpr int kKeySub = DRT_KEY_SUB;
// Resident CTAs per SM of the kernel queueing secondary edge samples: with
// the length sampler, and with the edge hierarchy's pick (a per-thread stack).
#ifndef DRT_QUEUE_MIN_BLOCKS
#define DRT_QUEUE_MIN_BLOCKS 4
#endif
#ifndef DRT_TREE_QUEUE_MIN_BLOCKS
#define DRT_TREE_QUEUE_MIN_BLOCKS 4
#endif
// Resident CTAs per SM the render kernel is compiled for.
#ifndef DRT_RENDER_MIN_BLOCKS
#define DRT_RENDER_MIN_BLOCKS 4
#endif
// Resident CTAs per SM the kernel tracing the queued secondary edge samples
// is compiled for.
#ifndef DRT_SEC_MIN_BLOCKS
#define DRT_SEC_MIN_BLOCKS 2
#endif
// Resident CTAs per SM of the staged evaluation beyond depth 1: the side-ray
// stage of the secondary samples, the continuation stage (one launch per
// vertex) and the secondary contributions.
#ifndef DRT_SIDES_MIN_BLOCKS
#define DRT_SIDES_MIN_BLOCKS 4
#endif
#ifndef DRT_BOUNCE_MIN_BLOCKS
#define DRT_BOUNCE_MIN_BLOCKS 2
#endif
#ifndef DRT_FINISH_MIN_BLOCKS
#define DRT_FINISH_MIN_BLOCKS 2
#endif
// Resident CTAs per SM the depth > 1 path pass is compiled for (its variant
// with the secondary edge samples inside the pass stays at one: it spills).
#ifndef DRT_PATH_MIN_BLOCKS
#define DRT_PATH_MIN_BLOCKS 2
#endif
static_assert(kBlock / 32 <= kTraceWarps, "warp-cooperative traversals support at most kTraceWarps warps per CTA");
constexpr unsigned kFull = 0xffffffffu;
constexpr int kGlobals = 16;  // d_radiance[3], d_cam[12], d_cam_scale[1]

// ---- smooth float3 helpers (contraction allowed) ---------------------------
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float3 b) { return make_float3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ void operator+=(float3& a, float3 b) { a.x += b.x; a.y += b.y; a.z += b.z; }
__device__ __forceinline__ void operator-=(float3& a, float3 b) { a.x -= b.x; a.y -= b.y; a.z -= b.z; }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float len(float3 a) { return sqrtf(dot(a, a)); }
__device__ __forceinline__ float3 f3(const float p[3]) { return make_float3(p[0], p[1], p[2]); }
__device__ __forceinline__ float3 zero3() { return make_float3(0.f, 0.f, 0.f); }

// ---- warp-aggregated scatter (Sec. 5.4.6: reductions over pixels that hit
// the same object are the backward bottleneck).  All 32 lanes must call. ----
__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}
// Block-level gradient cache.  A few entities receive gradient from almost
// every pixel (the vertices of the light, of a floor, a floor's albedo); sent
// straight to global memory, their atomic additions all land in one L2 slice
// and serialise there, delaying every other access to that slice.  A block
// first adds warp sums into a direct-mapped table in shared memory (shared
// atomics; a key whose slot is taken goes to global memory directly) and
// sends each table entry once, when the block ends.
constexpr int kCacheSlots = 64;
struct GradCache {
  int key[kCacheSlots];
  float val[kCacheSlots][3];
};
// All threads of the block; __syncthreads() before the first scatter.
__device__ __forceinline__ void cache_init(GradCache& c) {
  for (int i = threadIdx.x; i < kCacheSlots; i += kBlock) {
    c.key[i] = -1;
    c.val[i][0] = c.val[i][1] = c.val[i][2] = 0.f;
  }
}
// All threads of the block, after a __syncthreads() that follows the last
// scatter; a __syncthreads() must separate it from the next cache_init.
__device__ __forceinline__ void cache_flush(const GradCache& c, float* arr) {
  if (arr == nullptr) return;
  for (int i = threadIdx.x; i < kCacheSlots; i += kBlock) {
    int k = c.key[i];
    if (k >= 0) {
      atomicAdd(arr + 3 * k, c.val[i][0]);
      atomicAdd(arr + 3 * k + 1, c.val[i][1]);
      atomicAdd(arr + 3 * k + 2, c.val[i][2]);
    }
  }
}

__device__ __forceinline__ void scatter3(float* arr, int id, float3 v, bool active, GradCache* cache = nullptr) {
  if (arr == nullptr) return;
  int lane = threadIdx.x & 31;
  unsigned pending = __ballot_sync(kFull, active);
  while (pending) {
    int leader = __ffs(pending) - 1;
    int key = __shfl_sync(kFull, id, leader);
    bool mine = active && id == key;
    unsigned peers = __ballot_sync(kFull, mine);
    float3 x = mine ? v : zero3();
    if (__popc(peers) > 1) {
      x.x = warp_sum(x.x);
      x.y = warp_sum(x.y);
      x.z = warp_sum(x.z);
    } else {
      x.x = __shfl_sync(kFull, x.x, leader);
      x.y = __shfl_sync(kFull, x.y, leader);
      x.z = __shfl_sync(kFull, x.z, leader);
    }
    if (lane == leader) {
      bool cached = false;
      if (cache) {
        int slot = key & (kCacheSlots - 1);
        int prev = atomicCAS(&cache->key[slot], -1, key);
        if (prev == -1 || prev == key) {
          atomicAdd(&cache->val[slot][0], x.x);
          atomicAdd(&cache->val[slot][1], x.y);
          atomicAdd(&cache->val[slot][2], x.z);
          cached = true;
        }
      }
      if (!cached) {
        atomicAdd(arr + 3 * key, x.x);
        atomicAdd(arr + 3 * key + 1, x.y);
        atomicAdd(arr + 3 * key + 2, x.z);
      }
    }
    pending &= ~peers;
  }
}

// The same as a called function: the path sweep scatters up to seven
// triples per vertex, and seven inlined copies made its loop too large for
// the instruction cache (warps stalled on instruction fetch; 6.9 -> 5.7 ms
// per launch on the 200k-triangle depth-3 step with the call).
__device__ __noinline__ void scatter3_call(float* arr, int id, float3 v, bool active, GradCache* cache) {
  scatter3(arr, id, v, active, cache);
}

// Per-pixel gradient image (drt_grads.dimage_dparam): a sample's
// contribution to a listed parameter is also added to the image of that
// parameter at the sample's pixel.  op.jac.n is uniform, so the hooks cost a
// branch when no image is asked for.
__device__ __forceinline__ void jac_add3(const Opts& op, int64_t base, int id, float3 v, int64_t pix, bool active) {
  if (op.jac.n == 0 || !active) return;
  for (int k = 0; k < op.jac.n; ++k) {
    int64_t q = op.jac.param[k] - base - 3 * (int64_t)id;
    if (q >= 0 && q < 3) atomicAdd(op.jac.out + (int64_t)k * op.jac.npix + pix, q == 0 ? v.x : (q == 1 ? v.y : v.z));
  }
}
__device__ __forceinline__ void jac_globals(const Opts& op, const float g[kGlobals], int64_t pix, bool active) {
  if (op.jac.n == 0 || !active) return;
  for (int k = 0; k < op.jac.n; ++k) {
    int64_t q = op.jac.param[k] - op.jac.v3 - op.jac.t3;
    if (q >= 0 && q < kGlobals) {
      float v = 0.f;
#pragma unroll
      for (int i = 0; i < kGlobals; ++i)
        if (i == q) v = g[i];
      if (v != 0.f) atomicAdd(op.jac.out + (int64_t)k * op.jac.npix + pix, v);
    }
  }
}

// Block reduction of the global parameters into one row of partials; the
// rows are summed in a fixed order by k_reduce_globals (deterministic).
__device__ __forceinline__ void block_globals(float g[kGlobals], float* row, bool add) {
  __shared__ float sm[kBlock / 32][kGlobals];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kGlobals; ++i) {
    float x = warp_sum(g[i]);
    if (lane == 0) sm[wid][i] = x;
  }
  __syncthreads();
  if (threadIdx.x < kGlobals) {
    float acc = 0.f;
    for (int w = 0; w < kBlock / 32; ++w) acc += sm[w][threadIdx.x];
    float* dst = row + threadIdx.x;
    *dst = add ? *dst + acc : acc;
  }
}

// Deterministic two-stage sum of the partial rows (the result does not depend
// on scheduling).  Stage 1: block c sums rows [c*kReduceRows, (c+1)*kReduceRows)
// per column in FP64, 16 row groups in a fixed stride, then the groups in
// order.  Stage 2: one warp per column sums the chunk totals in a fixed stride
// and a fixed butterfly.
constexpr int kReduceRows = 256;
__global__ void k_reduce_rows(const float* partials, int64_t rows, double* chunks) {
  __shared__ double sm[kBlock];
  int col = threadIdx.x & (kGlobals - 1), grp = threadIdx.x / kGlobals;  // kBlock / kGlobals = 16 groups
  int64_t r0 = (int64_t)blockIdx.x * kReduceRows;
  int64_t r1 = r0 + kReduceRows < rows ? r0 + kReduceRows : rows;
  double acc = 0.0;
  for (int64_t r = r0 + grp; r < r1; r += kBlock / kGlobals) acc += partials[r * kGlobals + col];
  sm[threadIdx.x] = acc;
  __syncthreads();
  if (grp == 0) {
    double t = 0.0;
    for (int g = 0; g < kBlock / kGlobals; ++g) t += sm[g * kGlobals + col];
    chunks[(int64_t)blockIdx.x * kGlobals + col] = t;
  }
}
__global__ void k_reduce_chunks(const double* chunks, int64_t n, float* d_radiance, float* d_cam, float* d_scale) {
  int i = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (i >= kGlobals) return;
  double acc = 0.0;
  for (int64_t c = lane; c < n; c += 32) acc += chunks[c * kGlobals + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  if (lane != 0) return;
  float v = (float)acc;
  if (i < 3) { if (d_radiance) d_radiance[i] += v; }
  else if (i < 15) { if (d_cam) d_cam[i - 3] += v; }
  else if (d_scale) d_scale[0] += v;
}

// ---- shading data of a hit -------------------------------------------------
struct Vertex {
  int k;
  float p[3];       // FP32 hit point (decision path)
  float nu[3];      // unnormalised face normal (decision path)
  float side;       // nu . d
  float3 v0, v1, v2;
};
__device__ __forceinline__ void load_vertex(const SceneView& s, int k, float b1, float b2, const float d[3], Vertex& x) {
  x.k = k;
  const int32_t* id = s.tris + 3 * k;
  x.v0 = ld3(s.verts + 3 * id[0]);
  x.v1 = ld3(s.verts + 3 * id[1]);
  x.v2 = ld3(s.verts + 3 * id[2]);
  bary_point(x.v0, x.v1, x.v2, b1, b2, x.p);
  face_normal(x.v0, x.v1, x.v2, x.nu);
  x.side = dot3x(x.nu, d);
}
// Flipped unit normal on the viewer side (decision-path FP32).
__device__ __forceinline__ void shading_normal32(const Vertex& x, float n[3]) {
  float nl = fsq(dot3x(x.nu, x.nu));
  float fl = x.side > 0.0f ? -1.0f : 1.0f;
  n[0] = fm(fl, fdv(x.nu[0], nl));
  n[1] = fm(fl, fdv(x.nu[1], nl));
  n[2] = fm(fl, fdv(x.nu[2], nl));
}

struct LightSample {
  int j, lt;
  float y[3];
  float w[3];  // barycentric weights
  float3 l0, l1, l2;
};
__device__ __forceinline__ void sample_light(const SceneView& s, uint4 r, LightSample& ls) {
  double total = s.light_cdf[s.L - 1];
  ls.j = cdf_pick(s.light_cdf, s.L, dm(u01d(r.x, r.y), total));
  ls.lt = s.light_tris[ls.j];
  const int32_t* id = s.tris + 3 * ls.lt;
  ls.l0 = ld3(s.verts + 3 * id[0]);
  ls.l1 = ld3(s.verts + 3 * id[1]);
  ls.l2 = ld3(s.verts + 3 * id[2]);
  float r1 = u01f(r.z), r2 = u01f(r.w);
  float su = fsq(r1);
  float b0 = fs(1.0f, su), b1 = fm(su, r2), b2 = fs(su, b1);
  ls.w[0] = b0; ls.w[1] = b1; ls.w[2] = b2;
  ls.y[0] = fa(fa(fm(b0, ls.l0.x), fm(b1, ls.l1.x)), fm(b2, ls.l2.x));
  ls.y[1] = fa(fa(fm(b0, ls.l0.y), fm(b1, ls.l1.y)), fm(b2, ls.l2.y));
  ls.y[2] = fa(fa(fm(b0, ls.l0.z), fm(b1, ls.l1.z)), fm(b2, ls.l2.z));
}

// NEE value at a vertex (factor multiplying rho/pi * Le): G * A_j / P(j).
__device__ __forceinline__ float nee_geometry(const SceneView& s, float3 p, float3 n, const LightSample& ls) {
  float3 W = f3(ls.y) - p;
  float r2 = dot(W, W);
  float r = sqrtf(r2);
  float3 w = (1.0f / r) * W;
  float cp = dot(n, w);
  float3 Nl = cross(ls.l1 - ls.l0, ls.l2 - ls.l0);
  float nll = len(Nl);
  float cy = -dot(Nl, w) / nll;
  if (!(cp > 0.f && cy > 0.f)) return 0.f;
  double total = s.light_cdf[s.L - 1];
  float invP = (float)(total / s.light_area[ls.j]);
  return cp * cy / r2 * (0.5f * nll) * invP;
}


// Geometry buffers of the first hit (Sec. 5.4): with primary_only the path's
// value is the hit's albedo, or (op.aov) its world position, its unit shading
// normal (facing the ray) or its distance from the ray origin o.
__device__ __forceinline__ float3 aov_value(const Opts& op, const Vertex& x, float3 alb, const float o[3]) {
  if (op.aov == 2) return f3(x.p);
  if (op.aov == 3) {
    float3 Nk = cross(x.v1 - x.v0, x.v2 - x.v0);
    float fl = x.side > 0.0f ? -1.f : 1.f;
    return (fl / len(Nk)) * Nk;
  }
  if (op.aov == 4) {
    float dd = len(f3(x.p) - f3(o));
    return make_float3(dd, dd, dd);
  }
  return alb;
}

// L += c * t with one rounding per component, written as an explicit FMA so
// that every evaluation of a path (in one kernel or in stages) rounds alike
// whatever the compiler would contract.
__device__ __forceinline__ void nee_add(float3& L, float c, float3 t) {
  L.x = __fmaf_rn(c, t.x, L.x);
  L.y = __fmaf_rn(c, t.y, L.y);
  L.z = __fmaf_rn(c, t.z, L.z);
}

// path_value of a camera path (from depth 0, first emission counted) for the
// 32 lanes of a warp together, traced by the warp-cooperative traversals.
// All lanes call; a lane with act = false traces nothing, writes no tape and
// returns 0.  Same values and tape entries as path_value.  pair_lanes: lanes
// 2k and 2k+1 hold the two sides of one edge sample, whose term is zero when
// both first hits are one triangle; such a pair stops after its first hit
// (first_tri is still reported, and the caller discards the value).
__device__ float3 path_value_warp(const SceneView& s, const Opts& op, const float o_in[3], const float d_in[3],
                                  bool act, uint32_t c0, uint32_t c1, uint32_t pass, int32_t* tape_tri,
                                  float2* tape_bary, int64_t n_idx, int64_t n_stride, int* first_tri = nullptr,
                                  bool pair_lanes = false) {
  const unsigned full = 0xffffffffu;
  float o[3] = {o_in[0], o_in[1], o_in[2]}, d[3] = {d_in[0], d_in[1], d_in[2]};
  float3 L = zero3(), beta = make_float3(1.f, 1.f, 1.f);
  int md = op.primary_only ? 1 : op.max_depth;
  const float3 Le = ld3(s.radiance);
  bool alive = act;
  int exclude = -1;
  int b_end = 0;  // first bounce whose tape entry is not written
  for (int b = 0; b < md; ++b) {
    if (!__any_sync(full, alive)) break;
    // the warp's camera rays are coherent; after a diffuse bounce its rays
    // point anywhere, and each lane traces its own
    Hit h;
    if (b == 0) {
      Hit h_unused;
      trace_closest2_warp(s, o, d, o, d, alive, false, exclude, -1, h, h_unused);
    } else if (alive) {
      h = trace_closest(s, o, d, INFINITY, exclude);
    } else {
      h.tri = -1;
      h.t = h.b1 = h.b2 = 0.f;
    }
    if (alive && h.tri < 0) alive = false;
    if (b == 0 && first_tri) *first_tri = alive ? h.tri : -1;
    if (b == 0 && pair_lanes) {
      int mine = alive ? h.tri : -1;
      int other = __shfl_xor_sync(full, mine, 1);  // every lane, before any branch on alive
      if (alive && mine == other) alive = false;
    }
    Vertex x;
    x.k = -1;
    x.p[0] = x.p[1] = x.p[2] = 0.f;
    float3 alb = zero3();
    float n32[3] = {0.f, 0.f, 1.f};
    if (alive) {
      load_vertex(s, h.tri, h.b1, h.b2, d, x);
      alb = ld3(s.albedo + 3 * x.k);
      if (op.primary_only) {
        L += beta * aov_value(op, x, alb, o);
        if (tape_tri) {
          tape_tri[b * n_stride + n_idx] = x.k;
          tape_bary[b * n_stride + n_idx] = make_float2(h.b1, h.b2);
        }
        b_end = b + 1;
        alive = false;
      } else {
        if (b == 0 && s.light_of_tri[x.k] >= 0 && x.side < 0.0f) L += beta * Le;
        shading_normal32(x, n32);
      }
    }
    if (op.primary_only) continue;
    int vis = 0;
    if (s.L > 0) {
      uint4 r = rng4(op.key, c0, c1, kLight, (uint32_t)b, pass, op.scene_id);
      LightSample ls;
      sample_light(s, r, ls);
      float sd[3] = {0.f, 0.f, 1.f};
      if (alive)
        for (int i = 0; i < 3; ++i) sd[i] = fs(ls.y[i], x.p[i]);
      bool occ = false, occ_unused;
      if (b == 0)
        trace_any2_warp(s, x.p, sd, x.k, ls.lt, x.p, sd, -1, -1, alive, false, kShadowTmax, occ, occ_unused);
      else if (alive)
        occ = trace_any(s, x.p, sd, kShadowTmax, x.k, ls.lt);
      if (alive && !occ) {
        vis = 1;
        float g = nee_geometry(s, f3(x.p), f3(n32), ls);
        nee_add(L, kInvPi * g, beta * alb * Le);
      }
    }
    if (alive) {
      if (tape_tri) {
        tape_tri[b * n_stride + n_idx] = x.k | (vis << 31);
        tape_bary[b * n_stride + n_idx] = make_float2(h.b1, h.b2);
      }
      b_end = b + 1;
    }
    if (b + 1 >= md) break;
    uint4 r = rng4(op.key, c0, c1, kBsdf, (uint32_t)b, pass, op.scene_id);
    if (alive) {
      float nd[3];
      cosine_dir(n32, u01f(r.x), u01f(r.y), nd);
      if (!(dot(f3(n32), f3(nd)) > 0.f)) {
        alive = false;
      } else {
        beta = beta * alb;
        for (int i = 0; i < 3; ++i) { o[i] = x.p[i]; d[i] = nd[i]; }
        exclude = x.k;
      }
    }
  }
  if (tape_tri && act)
    for (int b = b_end; b < md; ++b) tape_tri[b * n_stride + n_idx] = -1;
  return L;
}

// Vertex 0 of a camera path for the 32 lanes of a warp together, exactly as
// the first iteration of path_value_warp (all lanes call; warp-cooperative
// traversals): emission at the hit, next-event estimation, and, when the path
// goes on (cont), its continuation direction nd, the hit h0 and the hit's
// albedo (the throughput of what follows).
__device__ float3 path_first_vertex_warp(const SceneView& s, const Opts& op, const float o[3], const float d[3],
                                         bool act, uint32_t c0, uint32_t c1, uint32_t pass, bool& cont, Hit& h0,
                                         float nd[3], float3& alb, int* vis_out = nullptr, bool pair_lanes = false) {
  int md = op.primary_only ? 1 : op.max_depth;
  const float3 Le = ld3(s.radiance);
  float3 L = zero3();
  bool alive = act;
  cont = false;
  if (vis_out) *vis_out = 0;
  alb = zero3();
  nd[0] = nd[1] = 0.f;
  nd[2] = 1.f;
  Hit h, h_unused;
  trace_closest2_warp(s, o, d, o, d, alive, false, -1, -1, h, h_unused);
  if (alive && h.tri < 0) alive = false;
  h0 = h;
  // the two sides of an edge sample (lanes 2k, 2k+1) on one triangle: a zero
  // term, the caller discards this vertex; no shadow ray and no continuation
  if (pair_lanes) {
    int mine = alive ? h.tri : -1;
    int other = __shfl_xor_sync(0xffffffffu, mine, 1);  // every lane, before any branch on alive
    if (alive && mine == other) alive = false;
  }
  Vertex x;
  x.k = -1;
  x.p[0] = x.p[1] = x.p[2] = 0.f;
  float n32[3] = {0.f, 0.f, 1.f};
  if (alive) {
    load_vertex(s, h.tri, h.b1, h.b2, d, x);
    alb = ld3(s.albedo + 3 * x.k);
    if (s.light_of_tri[x.k] >= 0 && x.side < 0.0f) L += Le;
    shading_normal32(x, n32);
  }
  if (s.L > 0) {
    uint4 r = rng4(op.key, c0, c1, kLight, 0u, pass, op.scene_id);
    LightSample ls;
    sample_light(s, r, ls);
    float sd[3] = {0.f, 0.f, 1.f};
    if (alive)
      for (int i = 0; i < 3; ++i) sd[i] = fs(ls.y[i], x.p[i]);
    bool occ = false, occ_unused;
    trace_any2_warp(s, x.p, sd, x.k, ls.lt, x.p, sd, -1, -1, alive, false, kShadowTmax, occ, occ_unused);
    if (alive && !occ) {
      float g = nee_geometry(s, f3(x.p), f3(n32), ls);
      nee_add(L, kInvPi * g, alb * Le);
      if (vis_out) *vis_out = 1;
    }
  }
  if (alive && md > 1) {
    uint4 r = rng4(op.key, c0, c1, kBsdf, 0u, pass, op.scene_id);
    cosine_dir(n32, u01f(r.x), u01f(r.y), nd);
    cont = dot(f3(n32), f3(nd)) > 0.f;
  }
  return L;
}

// The two side paths of a secondary edge sample at path depth depth0 - 1,
// continued from their first hits h[q] (traced by the caller from the vertex
// along d[q], the vertex's triangle skipped): what path_value returns for each
// side with emission_first = false, both sides with the same random numbers,
// traced pairwise.  act[q] = false: side q contributes 0.
__device__ void path_value2_from(const SceneView& s, const Opts& op, const float d_in[2][3], const Hit h_in[2],
                                 const bool act[2], int depth0, uint32_t c0, uint32_t c1, uint32_t pass,
                                 float3 L[2]) {
  int md = op.primary_only ? 1 : op.max_depth;
  const float3 Le = ld3(s.radiance);
  bool alive[2] = {act[0], act[1]};
  float o[2][3], d[2][3];
  int exclude[2] = {-1, -1};
  for (int q = 0; q < 2; ++q)
    for (int i = 0; i < 3; ++i) { o[q][i] = 0.f; d[q][i] = d_in[q][i]; }
  float3 beta[2] = {make_float3(1.f, 1.f, 1.f), make_float3(1.f, 1.f, 1.f)};
  L[0] = L[1] = zero3();
  Hit h[2] = {h_in[0], h_in[1]};
  for (int b = depth0; b < md; ++b) {
    if (b > depth0)
      trace_closest2(s, o[0], d[0], o[1], d[1], alive[0], alive[1], exclude[0], exclude[1], h[0], h[1]);
    Vertex x[2];
    float3 alb[2];
    for (int q = 0; q < 2; ++q) {
      if (!alive[q]) continue;
      if (h[q].tri < 0) { alive[q] = false; continue; }
      load_vertex(s, h[q].tri, h[q].b1, h[q].b2, d[q], x[q]);
      alb[q] = ld3(s.albedo + 3 * x[q].k);
    }
    if (!alive[0] && !alive[1]) break;
    float n32[2][3];
    for (int q = 0; q < 2; ++q)
      if (alive[q]) shading_normal32(x[q], n32[q]);
    if (s.L > 0) {
      uint4 r = rng4(op.key, c0, c1, kLight, (uint32_t)b, pass, op.scene_id);
      LightSample ls;
      sample_light(s, r, ls);
      float sd[2][3];
      for (int q = 0; q < 2; ++q)
        if (alive[q])
          for (int i = 0; i < 3; ++i) sd[q][i] = fs(ls.y[i], x[q].p[i]);
      bool occ[2];
      trace_any2(s, x[0].p, sd[0], x[0].k, ls.lt, x[1].p, sd[1], x[1].k, ls.lt, alive[0], alive[1], kShadowTmax,
                 occ[0], occ[1]);
      for (int q = 0; q < 2; ++q)
        if (alive[q] && !occ[q]) {
          float g = nee_geometry(s, f3(x[q].p), f3(n32[q]), ls);
          nee_add(L[q], kInvPi * g, beta[q] * alb[q] * Le);
        }
    }
    if (b + 1 >= md) break;
    uint4 r = rng4(op.key, c0, c1, kBsdf, (uint32_t)b, pass, op.scene_id);
    for (int q = 0; q < 2; ++q) {
      if (!alive[q]) continue;
      float nd[3];
      cosine_dir(n32[q], u01f(r.x), u01f(r.y), nd);
      if (!(dot(f3(n32[q]), f3(nd)) > 0.f)) { alive[q] = false; continue; }
      beta[q] = beta[q] * alb[q];
      for (int i = 0; i < 3; ++i) { o[q][i] = x[q].p[i]; d[q][i] = nd[i]; }
      exclude[q] = x[q].k;
    }
    if (!alive[0] && !alive[1]) break;
  }
}

__device__ __forceinline__ void jitter(const Opts& op, int pix, int sidx, int W, float* sx, float* sy) {
  uint4 r = rng4(op.key, (uint32_t)pix, (uint32_t)sidx, kCamera, 0u, kPassInterior, op.scene_id);
  *sx = fa((float)(pix % W), u01f(r.x));
  *sy = fa((float)(pix / W), u01f(r.y));
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------
__device__ __forceinline__ void render_block(const SceneView& s, const Opts& op, float* image, int32_t* tape_tri,
                                                   float2* tape_bary, int G, int64_t blk) {
  int lane = threadIdx.x & 31;
  int64_t gw = (blk * kBlock + threadIdx.x) >> 5;
  int ppw = 32 / G;
  int64_t pix = gw * ppw + lane / G;
  int npix = s.W * s.H;
  bool active = pix < npix;
  int64_t n = (int64_t)npix * op.spp;
  float3 acc = zero3();
  // the warp traces its lanes' samples together: every lane runs the same
  // number of rounds
  int iters = (op.spp + G - 1) / G;
  for (int it = 0; it < iters; ++it) {
    int sidx = lane % G + it * G;
    bool act = active && sidx < op.spp;
    float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 1.f};
    if (act) {
      float sx, sy;
      jitter(op, (int)pix, sidx, s.W, &sx, &sy);
      camera_ray(s, sx, sy, o, d);
    }
    float3 v = path_value_warp(s, op, o, d, act, (uint32_t)pix, (uint32_t)sidx, kPassInterior, tape_tri, tape_bary,
                               pix * op.spp + sidx, n);
    if (act) acc += v;
  }
  for (int o = G >> 1; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(kFull, acc.x, o);
    acc.y += __shfl_xor_sync(kFull, acc.y, o);
    acc.z += __shfl_xor_sync(kFull, acc.z, o);
  }
  if (active && lane % G == 0) {
    float inv = 1.0f / (float)op.spp;
    image[3 * pix] = acc.x * inv;
    image[3 * pix + 1] = acc.y * inv;
    image[3 * pix + 2] = acc.z * inv;
  }
}
__global__ void __launch_bounds__(kBlock, DRT_RENDER_MIN_BLOCKS) k_render(SceneView s, Opts op, float* image, int32_t* tape_tri,
                                                   float2* tape_bary, int G) {
  render_block(s, op, image, tape_tri, tape_bary, G, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Backward helpers: camera adjoints
// ---------------------------------------------------------------------------
// Camera ray o, d as functions of the camera (same formulas as camera_ray):
// accumulate d loss/d(camera) given the adjoints do_, dd_.
__device__ __forceinline__ void camera_ray_adjoint(const SceneView& s, float sx, float sy, float3 do_, float3 dd_,
                                                   float g[kGlobals]) {
  const float* M = s.cam;
  float S = s.cam_scale[0];
  float fw = (float)s.W, fh = (float)s.H;
  float xn = (2.0f * sx - fw) / fw, yn = (fh - 2.0f * sy) / fh;
  float aspect = fw / fh;
  if (s.cam_type == 2) {
    // fisheye: d = M3 (a/r sin th, b/r sin th, -cos th), th = r S, o = t
    float a = xn * aspect, b = yn, r = sqrtf(a * a + b * b);
    float sn, cs;
    sincosf(r * S, &sn, &cs);
    float ar = r > 0.f ? a / r : 0.f, br = r > 0.f ? b / r : 0.f;
    float dc[3] = {ar * sn, br * sn, -cs}, dth[3] = {ar * cs, br * cs, sn};
    float dov[3] = {do_.x, do_.y, do_.z}, ddv[3] = {dd_.x, dd_.y, dd_.z};
    float gth = 0.f;
    for (int i = 0; i < 3; ++i) {
      float* gm = g + 3 + 4 * i;
      gm[3] += dov[i];
      for (int j = 0; j < 3; ++j) {
        gm[j] += ddv[i] * dc[j];
        gth += ddv[i] * M[4 * i + j] * dth[j];
      }
    }
    g[15] += gth * r;
    return;
  }
  float lx = xn * aspect * S, ly = yn * S;
  float dov[3] = {do_.x, do_.y, do_.z}, ddv[3] = {dd_.x, dd_.y, dd_.z};
  float dlx = 0.f, dly = 0.f;
  for (int r = 0; r < 3; ++r) {
    float* gm = g + 3 + 4 * r;
    if (s.cam_type == 1) {
      gm[3] += dov[r];
      gm[0] += ddv[r] * lx;
      gm[1] += ddv[r] * ly;
      gm[2] -= ddv[r];
      dlx += ddv[r] * M[4 * r];
      dly += ddv[r] * M[4 * r + 1];
    } else {
      gm[0] += dov[r] * lx;
      gm[1] += dov[r] * ly;
      gm[3] += dov[r];
      gm[2] -= ddv[r];
      dlx += dov[r] * M[4 * r];
      dly += dov[r] * M[4 * r + 1];
    }
  }
  g[15] += dlx * xn * aspect + dly * yn;
}

// Projection of world point v to the screen: given d loss/d(sx, sy), return
// d loss/dv and accumulate the camera adjoints (vc = R^-1 (v - t)).
__device__ __forceinline__ float3 project_adjoint(const SceneView& s, float3 v, float dsx, float dsy,
                                                  float g[kGlobals]) {
  const float* Wm = s.w2c;
  float vc[3];
  for (int i = 0; i < 3; ++i) vc[i] = Wm[4 * i] * v.x + Wm[4 * i + 1] * v.y + Wm[4 * i + 2] * v.z + Wm[4 * i + 3];
  float S = s.cam_scale[0];
  float fw = (float)s.W, fh = (float)s.H;
  float aspect = fw / fh;
  float px = vc[0], py = vc[1], iz = 1.f;
  if (s.cam_type == 1) {
    iz = -vc[2];
    px = vc[0] / iz;
    py = vc[1] / iz;
  }
  float xn = px / (aspect * S), yn = py / S;
  float dxn = dsx * (0.5f * fw), dyn = -dsy * (0.5f * fh);
  float dpx = dxn / (aspect * S), dpy = dyn / S;
  g[15] += -(dxn * xn + dyn * yn) / S;
  float dvc[3];
  if (s.cam_type == 1) {
    dvc[0] = dpx / iz;
    dvc[1] = dpy / iz;
    dvc[2] = (dpx * px + dpy * py) / iz;
  } else {
    dvc[0] = dpx; dvc[1] = dpy; dvc[2] = 0.f;
  }
  float3 dv;
  dv.x = Wm[0] * dvc[0] + Wm[4] * dvc[1] + Wm[8] * dvc[2];
  dv.y = Wm[1] * dvc[0] + Wm[5] * dvc[1] + Wm[9] * dvc[2];
  dv.z = Wm[2] * dvc[0] + Wm[6] * dvc[1] + Wm[10] * dvc[2];
  float dva[3] = {dv.x, dv.y, dv.z};
  for (int i = 0; i < 3; ++i) {
    float* gm = g + 3 + 4 * i;
    gm[3] -= dva[i];
    for (int j = 0; j < 3; ++j) gm[j] -= dva[i] * vc[j];
  }
  return dv;
}

// Fisheye projection of world point v (smooth FP32): given d loss/d(sx, sy),
// return d loss/dv and accumulate the camera and scale adjoints.  With the
// camera-space point (x, y, vz), rho = |(x, y)|, theta = atan2(rho, -vz) and
// k = theta / (S rho): a = k x, b = k y, sx = (a / aspect + 1) W / 2,
// sy = (1 - b) H / 2.
__device__ __forceinline__ float3 fisheye_project_adjoint(const SceneView& s, float3 v, float gx, float gy,
                                                          float g[kGlobals]) {
  const float* Wm = s.w2c;
  float vc[3];
  for (int i = 0; i < 3; ++i) vc[i] = Wm[4 * i] * v.x + Wm[4 * i + 1] * v.y + Wm[4 * i + 2] * v.z + Wm[4 * i + 3];
  float S = s.cam_scale[0];
  float x = vc[0], y = vc[1], zz = -vc[2];
  float rho2 = x * x + y * y, rho = sqrtf(rho2), R2 = rho2 + zz * zz;
  float th = atan2f(rho, zz);
  float k = th / (S * rho);
  float a = k * x, b = k * y;
  float hh = 0.5f * (float)s.H;
  float ga = gx * hh, gb = -gy * hh;
  float gk = ga * x + gb * y;
  float dthx = zz * x / (rho * R2), dthy = zz * y / (rho * R2), dthz = rho / R2;
  float dkx = dthx / (S * rho) - th * x / (S * rho * rho2), dky = dthy / (S * rho) - th * y / (S * rho * rho2);
  float dkz = dthz / (S * rho);
  float dvc[3] = {ga * k + gk * dkx, gb * k + gk * dky, gk * dkz};
  g[15] += -(ga * a + gb * b) / S;
  float3 dv;
  dv.x = Wm[0] * dvc[0] + Wm[4] * dvc[1] + Wm[8] * dvc[2];
  dv.y = Wm[1] * dvc[0] + Wm[5] * dvc[1] + Wm[9] * dvc[2];
  dv.z = Wm[2] * dvc[0] + Wm[6] * dvc[1] + Wm[10] * dvc[2];
  float dva[3] = {dv.x, dv.y, dv.z};
  for (int i = 0; i < 3; ++i) {
    float* gm = g + 3 + 4 * i;
    gm[3] -= dva[i];
    for (int j = 0; j < 3; ++j) gm[j] -= dva[i] * vc[j];
  }
  return dv;
}
// Tangent of the fisheye image of v + t dw with respect to t (smooth FP32).
__device__ __forceinline__ float2 fisheye_tangent(const SceneView& s, float3 v, float3 dw) {
  const float* Wm = s.w2c;
  float vc[3], dc[3];
  for (int i = 0; i < 3; ++i) {
    vc[i] = Wm[4 * i] * v.x + Wm[4 * i + 1] * v.y + Wm[4 * i + 2] * v.z + Wm[4 * i + 3];
    dc[i] = Wm[4 * i] * dw.x + Wm[4 * i + 1] * dw.y + Wm[4 * i + 2] * dw.z;
  }
  float S = s.cam_scale[0];
  float x = vc[0], y = vc[1], zz = -vc[2];
  float rho2 = x * x + y * y, rho = sqrtf(rho2), R2 = rho2 + zz * zz;
  float th = atan2f(rho, zz);
  float k = th / (S * rho);
  float drho = (x * dc[0] + y * dc[1]) / rho, dzz = -dc[2];
  float dth = (zz * drho - rho * dzz) / R2;
  float dk = dth / (S * rho) - th * drho / (S * rho2);
  float da_ = k * dc[0] + x * dk, db_ = k * dc[1] + y * dk;
  float hh = 0.5f * (float)s.H;
  return make_float2(hh * da_, -hh * db_);
}

// ---------------------------------------------------------------------------
// Backward: interior term (depth-1 paths) and secondary edge samples
// ---------------------------------------------------------------------------
struct Grads {
  float* verts;
  float* albedo;
  float* partials;
};

// The camera-path vertex of interior sample (pix, sidx): the tape gives the
// hit (and NEE visibility); without a tape the camera ray is traced again.
struct CamHit {
  float sx, sy, o[3], d[3];
  int k;
  bool vis;  // valid with a tape only
  float b1, b2;
};
__device__ __forceinline__ void camera_hit(const SceneView& s, const Opts& op, const int32_t* tape_tri,
                                           const float2* tape_bary, int64_t pix, int sidx, CamHit& c) {
  jitter(op, (int)pix, sidx, s.W, &c.sx, &c.sy);
  camera_ray(s, c.sx, c.sy, c.o, c.d);
  c.k = -1;
  c.vis = false;
  c.b1 = c.b2 = 0.f;
  if (tape_tri) {
    int64_t ti = pix * op.spp + sidx;
    int32_t tt = tape_tri[ti];
    if (tt != -1) {
      c.k = tt & 0x7fffffff;
      c.vis = (tt >> 31) & 1;
      float2 bb = tape_bary[ti];
      c.b1 = bb.x;
      c.b2 = bb.y;
    }
  } else {
    Hit h = trace_closest(s, c.o, c.d, INFINITY, -1);
    if (h.tri >= 0) {
      c.k = h.tri;
      c.b1 = h.b1;
      c.b2 = h.b2;
    }
  }
}

// Reverse sweep through the ray/plane hit point p = o + tau d of triangle k
// (and its flipped unit normal n): given d loss/dp and d loss/dn, add the
// triangle-vertex adjoints and the camera adjoints.
// Ray/plane hit p = o + tau d with the triangle of x moving: given d loss/dp
// and d loss/dn (flipped unit normal), add the vertex adjoints and return
// the adjoints of the ray origin and direction.
__device__ __forceinline__ void plane_hit_adjoint(const float o[3], const float d[3], const Vertex& x, float3 dp,
                                                  float3 dn, float3& dv0, float3& dv1, float3& dv2, float3& do_,
                                                  float3& dd_) {
  float3 ov = f3(o), dvv = f3(d);
  float3 e1 = x.v1 - x.v0, e2 = x.v2 - x.v0;
  float3 Nk = cross(e1, e2);
  float nkl = len(Nk);
  float flip = x.side > 0.0f ? -1.f : 1.f;
  float3 nhat = (1.f / nkl) * Nk;
  float num = dot(x.v0 - ov, Nk), den = dot(dvv, Nk);
  float tau = num / den;
  float3 dNk = zero3();
  float3 dnh = flip * dn;
  dNk += (1.f / nkl) * (dnh - dot(dnh, nhat) * nhat);
  float dtau = dot(dp, dvv);
  do_ = dp;
  dd_ = tau * dp;
  float dnum = dtau / den, dden = -dtau * tau / den;
  dv0 += dnum * Nk;
  do_ -= dnum * Nk;
  dNk += dnum * (x.v0 - ov);
  dd_ += dden * Nk;
  dNk += dden * dvv;
  float3 de1k = cross(e2, dNk), de2k = cross(dNk, e1);
  dv1 += de1k;
  dv2 += de2k;
  dv0 -= de1k + de2k;
}

__device__ __forceinline__ void hit_point_adjoint(const SceneView& s, const CamHit& c, const Vertex& x, float3 dp,
                                                  float3 dn, float3& dv0, float3& dv1, float3& dv2,
                                                  float g[kGlobals], float3 do_extra = float3{0.f, 0.f, 0.f}) {
  float3 ov = f3(c.o), dvv = f3(c.d);
  float3 e1 = x.v1 - x.v0, e2 = x.v2 - x.v0;
  float3 Nk = cross(e1, e2);
  float nkl = len(Nk);
  float flip = x.side > 0.0f ? -1.f : 1.f;
  float3 nhat = (1.f / nkl) * Nk;
  float num = dot(x.v0 - ov, Nk), den = dot(dvv, Nk);
  float tau = num / den;
  float3 dNk = zero3();
  float3 dnh = flip * dn;
  dNk += (1.f / nkl) * (dnh - dot(dnh, nhat) * nhat);
  float dtau = dot(dp, dvv);
  float3 do_ = dp + do_extra, dd_ = tau * dp;
  float dnum = dtau / den, dden = -dtau * tau / den;
  dv0 += dnum * Nk;
  do_ -= dnum * Nk;
  dNk += dnum * (x.v0 - ov);
  dd_ += dden * Nk;
  dNk += dden * dvv;
  float3 de1k = cross(e2, dNk), de2k = cross(dNk, e1);
  dv1 += de1k;
  dv2 += de2k;
  dv0 -= de1k + de2k;
  camera_ray_adjoint(s, c.sx, c.sy, do_, dd_, g);
}

__device__ __forceinline__ float3 shading_normal(const Vertex& x) {
  float3 Nk = cross(x.v1 - x.v0, x.v2 - x.v0);
  float flip = x.side > 0.0f ? -1.f : 1.f;
  return (flip / len(Nk)) * Nk;
}

// Interior term (second integral of Eq. redner_product_rule): emission and
// the NEE estimator F * A_j / P(j) at the camera hit, differentiated in
// reverse with the random numbers and the pick probability held fixed.
__device__ __forceinline__ void interior_block(const SceneView& s, const Opts& op, const int32_t* tape_tri,
                                               const float2* tape_bary, const float* d_image, Grads gr, int G,
                                               const float* dp_sec, int do_int, int64_t blk) {
  __shared__ GradCache cv, ca;
  cache_init(cv);
  cache_init(ca);
  __syncthreads();
  int lane = threadIdx.x & 31;
  int64_t gw = (blk * kBlock + threadIdx.x) >> 5;
  int ppw = 32 / G;
  int64_t pix = gw * ppw + lane / G;
  int npix = s.W * s.H;
  bool pix_ok = pix < npix && pix >= op.pix_begin && pix < op.pix_end;
  float g[kGlobals];
  for (int i = 0; i < kGlobals; ++i) g[i] = 0.f;
  float3 wpix = pix_ok ? ld3(d_image + 3 * pix) : zero3();
  float3 a = (1.0f / (float)op.spp) * wpix;  // adjoint of the sample radiance
  const float3 Le = ld3(s.radiance);
  int iters = (op.spp + G - 1) / G;
  for (int it = 0; it < iters; ++it) {
    int sidx = lane % G + it * G;
    bool active = pix_ok && sidx < op.spp;
    CamHit c;
    c.k = -1;
    if (active) camera_hit(s, op, tape_tri, tape_bary, pix, sidx, c);
    bool hit = active && c.k >= 0;
    float3 dv0 = zero3(), dv1 = zero3(), dv2 = zero3(), dl0 = zero3(), dl1 = zero3(), dl2 = zero3();
    float3 dalb = zero3();
    int vid0 = 0, vid1 = 0, vid2 = 0, lid0 = 0, lid1 = 0, lid2 = 0;
    bool have_light = false;
    if (hit) {
      Vertex x;
      load_vertex(s, c.k, c.b1, c.b2, c.d, x);
      const int32_t* vid = s.tris + 3 * c.k;
      vid0 = vid[0]; vid1 = vid[1]; vid2 = vid[2];
      float3 alb = ld3(s.albedo + 3 * c.k);
      if (op.primary_only) {
        if (do_int && op.aov <= 1) {
          dalb = a;
        } else if (do_int) {
          // geometry buffers: the value moves with the hit point, the face
          // normal or the ray origin (the albedo does not enter)
          float3 dp = zero3(), dn = zero3(), dox = zero3();
          if (op.aov == 2) {
            dp = a;
          } else if (op.aov == 3) {
            dn = a;
          } else {
            float3 u = f3(x.p) - f3(c.o);
            u = (1.f / len(u)) * u;
            float as = a.x + a.y + a.z;
            dp = as * u;
            dox = -as * u;
          }
          hit_point_adjoint(s, c, x, dp, dn, dv0, dv1, dv2, g, dox);
        }
      } else {
        if (do_int && s.light_of_tri[c.k] >= 0 && x.side < 0.0f) {
          g[0] += a.x; g[1] += a.y; g[2] += a.z;
        }
        float3 dp = zero3(), dn = zero3();
        if (do_int && s.L > 0) {
          uint4 r = rng4(op.key, (uint32_t)pix, (uint32_t)sidx, kLight, 0u, kPassInterior, op.scene_id);
          LightSample ls;
          sample_light(s, r, ls);
          bool vis = c.vis;
          if (!tape_tri) {
            float sd[3] = {fs(ls.y[0], x.p[0]), fs(ls.y[1], x.p[1]), fs(ls.y[2], x.p[2])};
            vis = !trace_any(s, x.p, sd, kShadowTmax, x.k, ls.lt);
          }
          float3 n = shading_normal(x);
          float3 p = f3(x.p);
          if (vis) {
            float3 W = f3(ls.y) - p;
            float r2 = dot(W, W);
            float rr = sqrtf(r2);
            float3 w = (1.f / rr) * W;
            float cp = dot(n, w);
            float3 el1 = ls.l1 - ls.l0, el2 = ls.l2 - ls.l0;
            float3 Nl = cross(el1, el2);
            float nll = len(Nl);
            float3 nl = (1.f / nll) * Nl;
            float cy = -dot(nl, w);
            if (cp > 0.f && cy > 0.f) {
              double total = s.light_cdf[s.L - 1];
              float invP = (float)(total / s.light_area[ls.j]);
              float Aj = 0.5f * nll;
              float Gf = cp * cy / r2;
              float common = kInvPi * Gf * Aj * invP;
              g[0] += a.x * alb.x * common;
              g[1] += a.y * alb.y * common;
              g[2] += a.z * alb.z * common;
              dalb = make_float3(a.x * Le.x * common, a.y * Le.y * common, a.z * Le.z * common);
              float Q = (a.x * alb.x * Le.x + a.y * alb.y * Le.y + a.z * alb.z * Le.z) * kInvPi * invP;
              float dG = Q * Aj, dA = Q * Gf;
              float dcp = dG * cy / r2, dcy = dG * cp / r2, dr2 = -dG * Gf / r2;
              dn += dcp * w;
              float3 dw = dcp * n - dcy * nl;
              float3 dnl = -dcy * w;
              float3 dW = (1.f / rr) * (dw - dot(dw, w) * w) + (2.f * dr2) * W;
              dp -= dW;
              float3 dy = dW;
              float3 dNl = (1.f / nll) * (dnl - dot(dnl, nl) * nl) + (0.5f * dA) * nl;
              float3 de1l = cross(el2, dNl), de2l = cross(dNl, el1);
              dl0 = ls.w[0] * dy - de1l - de2l;
              dl1 = ls.w[1] * dy + de1l;
              dl2 = ls.w[2] * dy + de2l;
              const int32_t* lid = s.tris + 3 * ls.lt;
              lid0 = lid[0]; lid1 = lid[1]; lid2 = lid[2];
              have_light = true;
            }
          }
        }
        // adjoint of the hit point from its secondary edge sample (traced apart)
        if (dp_sec) dp += ld3(dp_sec + 3 * (pix * op.spp + sidx));
        hit_point_adjoint(s, c, x, dp, dn, dv0, dv1, dv2, g);
      }
    }
    scatter3(gr.verts, vid0, dv0, hit, &cv);
    scatter3(gr.verts, vid1, dv1, hit, &cv);
    scatter3(gr.verts, vid2, dv2, hit, &cv);
    scatter3(gr.albedo, c.k, dalb, hit && do_int, &ca);
    scatter3(gr.verts, lid0, dl0, have_light, &cv);
    scatter3(gr.verts, lid1, dl1, have_light, &cv);
    scatter3(gr.verts, lid2, dl2, have_light, &cv);
    if (op.jac.n) {
      jac_add3(op, 0, vid0, dv0, pix, hit);
      jac_add3(op, 0, vid1, dv1, pix, hit);
      jac_add3(op, 0, vid2, dv2, pix, hit);
      jac_add3(op, op.jac.v3, c.k, dalb, pix, hit && do_int);
      jac_add3(op, 0, lid0, dl0, pix, have_light);
      jac_add3(op, 0, lid1, dl1, pix, have_light);
      jac_add3(op, 0, lid2, dl2, pix, have_light);
    }
  }
  __syncthreads();
  cache_flush(cv, gr.verts);
  cache_flush(ca, gr.albedo);
  jac_globals(op, g, pix, pix_ok);
  block_globals(g, gr.partials + blk * kGlobals, false);
}
__global__ void __launch_bounds__(kBlock, DRT_PIXEL_MIN_BLOCKS)
    k_backward_interior(SceneView s, Opts op, const int32_t* tape_tri, const float2* tape_bary, const float* d_image,
                        Grads gr, int G, const float* dp_sec, int do_int) {
  interior_block(s, op, tape_tri, tape_bary, d_image, gr, G, dp_sec, do_int, blockIdx.x);
}

// Could a ray from o along d reach a light triangle?  Conservative slab test
// against the lights' padded bounding box.
__device__ __forceinline__ bool may_reach_light(const SceneView& s, const float o[3], const float d[3]) {
  float t0 = 0.f, t1 = INFINITY;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float lo = s.light_box[i], hi = s.light_box[3 + i];
    if (d[i] == 0.f) {
      if (o[i] < lo || o[i] > hi) return false;
      continue;
    }
    float inv = 1.f / d[i];
    float ta = (lo - o[i]) * inv, tb = (hi - o[i]) * inv;
    t0 = fmaxf(t0, fminf(ta, tb));
    t1 = fminf(t1, fmaxf(ta, tb));
  }
  return t0 <= t1 * 1.0001f;
}


// ---------------------------------------------------------------------------
// Backward for paths with several scattering vertices (path tracing)
// ---------------------------------------------------------------------------
constexpr int kMaxDepth = 8;

// NEE at vertex x with throughput-weighted adjoint ab = a * beta: returns the
// NEE radiance value (per colour) and adds its reverse-mode adjoints.
__device__ __forceinline__ float3 nee_adjoint(const SceneView& s, const Opts& op, uint32_t c0, uint32_t c1, int b,
                                              const Vertex& x, float3 n, float3 alb, float3 ab, float3 Le,
                                              float g[kGlobals], float3& dalb, float3& dp, float3& dn, float3 dl[3],
                                              int lid[3], bool& have_light) {
  uint4 r = rng4(op.key, c0, c1, kLight, (uint32_t)b, kPassInterior, op.scene_id);
  LightSample ls;
  sample_light(s, r, ls);
  float3 p = f3(x.p);
  float3 W = f3(ls.y) - p;
  float r2 = dot(W, W);
  float rr = sqrtf(r2);
  float3 w = (1.f / rr) * W;
  float cp = dot(n, w);
  float3 el1 = ls.l1 - ls.l0, el2 = ls.l2 - ls.l0;
  float3 Nl = cross(el1, el2);
  float nll = len(Nl);
  float3 nl = (1.f / nll) * Nl;
  float cy = -dot(nl, w);
  if (!(cp > 0.f && cy > 0.f)) return zero3();
  double total = s.light_cdf[s.L - 1];
  float invP = (float)(total / s.light_area[ls.j]);
  float Aj = 0.5f * nll;
  float Gf = cp * cy / r2;
  float common = kInvPi * Gf * Aj * invP;
  g[0] += ab.x * alb.x * common;
  g[1] += ab.y * alb.y * common;
  g[2] += ab.z * alb.z * common;
  dalb += make_float3(ab.x * Le.x * common, ab.y * Le.y * common, ab.z * Le.z * common);
  float Q = (ab.x * alb.x * Le.x + ab.y * alb.y * Le.y + ab.z * alb.z * Le.z) * kInvPi * invP;
  float dG = Q * Aj, dA = Q * Gf;
  float dcp = dG * cy / r2, dcy = dG * cp / r2, dr2 = -dG * Gf / r2;
  dn += dcp * w;
  float3 dw = dcp * n - dcy * nl;
  float3 dnl = -dcy * w;
  float3 dW = (1.f / rr) * (dw - dot(dw, w) * w) + (2.f * dr2) * W;
  dp -= dW;
  float3 dNl = (1.f / nll) * (dnl - dot(dnl, nl) * nl) + (0.5f * dA) * nl;
  float3 de1l = cross(el2, dNl), de2l = cross(dNl, el1);
  dl[0] = ls.w[0] * dW - de1l - de2l;
  dl[1] = ls.w[1] * dW + de1l;
  dl[2] = ls.w[2] * dW + de2l;
  const int32_t* li = s.tris + 3 * ls.lt;
  lid[0] = li[0]; lid[1] = li[1]; lid[2] = li[2];
  have_light = true;
  return common * (alb * Le);
}

// Secondary edge sample at vertex b (Sec. 5.2.2) with both parts: the area
// form for radiance arriving from lights, and for b+1 < max_depth the
// solid-angle form for reflected radiance (a traced sub-path from the side
// hit with the remaining depth, the same counters on both sides).
// a - b exactly, as hi + lo (Knuth's TwoSum, operations never contracted).
__device__ __forceinline__ void two_diff(float a, float b, float& hi, float& lo) {
  hi = fs(a, b);
  float bv = fs(hi, a);
  float av = fs(hi, bv);
  lo = fa(fs(a, av), fs(-b, bv));
}
__device__ __forceinline__ void two_diff3(float3 a, float3 b, float3& hi, float3& lo) {
  two_diff(a.x, b.x, hi.x, lo.x);
  two_diff(a.y, b.y, hi.y, lo.y);
  two_diff(a.z, b.z, hi.z, lo.z);
}
// a b - c d to about one rounding of the result (Kahan's FMA form).
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
  float w = fm(c, d);
  float e = __fmaf_rn(c, d, -w);
  float f = __fmaf_rn(a, b, -w);
  return fs(f, e);
}
__device__ __forceinline__ float3 cross_comp(float3 a, float3 b) {
  return make_float3(diff_of_products(a.y, b.z, a.z, b.y), diff_of_products(a.z, b.x, a.x, b.z),
                     diff_of_products(a.x, b.y, a.y, b.x));
}

struct SecOut {
  float3 de0, de1, dm[2][3];
  int eid0, eid1, mid[2][3];
  bool have_edge, have_m[2];
};
// How a secondary edge is selected: by the 3D length CDF, through the edge
// hierarchy (Sec. 5.3.1), or taken from a hierarchy pick made earlier for the
// same sample (`pre`), or a pick of next-event estimation for edges made by
// the queue (`pre4`: edge, weight, point; Sec. 5.3.3).  A template parameter,
// so kernels of the length sampler carry no call into the hierarchy.
enum { kSelLength = 0, kSelTree = 1, kSelTreePre = 2, kSelNeePre = 3 };

// Secondary edge sample at path vertex b (Sec. 5.2.2): the edge (see above),
// the point on it, the side
// directions omega +- eps|omega| n_h, and which sides can contribute (above the
// shading horizon; at the last vertex only a side that may reach a light).
// False: nothing to evaluate.
struct SecGeom {
  int e;
  int2 ev;
  float invPE, wl, t;
  float3 ve0, ve1;
  float dsd[2][3];
  float n32[3];  // shading normal (decision path)
  int pt;        // point density: bit 0 clamped-cosine mixture in use, bits 1, 2 ends inside the support
  bool act[2], last;
};

// Point on a secondary edge by importance (Sec. 5.3.2).  For a Lambertian
// surface the linearly transformed cosine is the clamped cosine itself; its
// integral along the edge's arc seen from p has a closed form and a
// closed-form inverse.  With f the unit vector from p to the foot of the
// perpendicular on the edge's line, e the edge direction, h the distance to
// the line and theta the angle from f toward e (s = h tan theta along the
// line): n . omega_hat = n_p cos(theta) + n_e sin(theta) = rho cos(theta - psi)
// and G = n_p sin(theta) - n_e cos(theta) = rho sin(theta - psi) is its
// antiderivative over d theta = h ds / r^2 (G = -rho, +rho at the support's
// ends).  A uniform y in [G(a), G(b)] gives sin and cos of theta - psi, then
// of theta by a rotation, then s and t: no angle is formed.  Mixed 1/4 with
// uniform (usel < 1/4 keeps t = u).  Every step is FP32 with one rounding per
// operation: t is a decision.  Degenerate cases keep t = u with density 1.
__device__ __forceinline__ float edge_point_sample(const float p[3], const float n[3], float3 v0, float3 v1, float u,
                                                   float usel, int& pt) {
  pt = 0;
  float a0[3] = {fs(v0.x, p[0]), fs(v0.y, p[1]), fs(v0.z, p[2])};
  float E[3] = {fs(v1.x, v0.x), fs(v1.y, v0.y), fs(v1.z, v0.z)};
  float N[3] = {fs(fm(a0[1], E[2]), fm(a0[2], E[1])), fs(fm(a0[2], E[0]), fm(a0[0], E[2])),
                fs(fm(a0[0], E[1]), fm(a0[1], E[0]))};
  float lE = fsq(dot3x(E, E)), nN = fsq(dot3x(N, N));
  if (!(lE > 0.0f) || !(nN > 0.0f)) return u;
  float h = fdv(nN, lE);
  float e[3] = {fdv(E[0], lE), fdv(E[1], lE), fdv(E[2], lE)};
  float k[3] = {fs(fm(e[1], N[2]), fm(e[2], N[1])), fs(fm(e[2], N[0]), fm(e[0], N[2])),
                fs(fm(e[0], N[1]), fm(e[1], N[0]))};
  float f[3] = {fdv(k[0], nN), fdv(k[1], nN), fdv(k[2], nN)};
  float s0 = dot3x(a0, e), s1 = fa(s0, lE);
  float np = dot3x(n, f), ne = dot3x(n, e);
  float rho = fsq(fa(fm(np, np), fm(ne, ne)));
  if (!(rho > 1e-6f)) return u;
  float hh = fm(h, h);
  float r0 = fsq(fa(fm(s0, s0), hh)), r1 = fsq(fa(fm(s1, s1), hh));
  float c0 = fdv(h, r0), g0 = fdv(s0, r0), c1 = fdv(h, r1), g1 = fdv(s1, r1);
  bool in0 = fa(fm(np, c0), fm(ne, g0)) > 0.0f, in1 = fa(fm(np, c1), fm(ne, g1)) > 0.0f;
  if (!in0 && !in1) return u;
  float Ga = in0 ? fs(fm(g0, np), fm(c0, ne)) : -rho;
  float Gb = in1 ? fs(fm(g1, np), fm(c1, ne)) : rho;
  float Z = fs(Gb, Ga);
  if (!(Z > fm(1e-6f, rho))) return u;
  pt = 1 | (in0 ? 2 : 0) | (in1 ? 4 : 0);
  if (usel < 0.25f) return u;
  float Y = fdv(fa(Ga, fm(u, Z)), rho);
  Y = fminf(fmaxf(Y, -1.0f), 1.0f);
  float C = fsq(fmaxf(fs(1.0f, fm(Y, Y)), 0.0f));
  float ct = fdv(fs(fm(C, np), fm(Y, ne)), rho);
  float st = fdv(fa(fm(Y, np), fm(C, ne)), rho);
  ct = fmaxf(ct, 1e-30f);
  float sl = fdv(fm(h, st), ct);
  float t = fdv(fs(sl, s0), lE);
  return fminf(fmaxf(t, 0.0f), 0.99999994f);
}

// Density of that point at t: 1/4 + 3/4 (n.omega_hat)^+ h |E| / (r^2 Z), in
// FP64 from the same FP32 inputs and support decisions (pt).  Called only for
// samples with a traced side.
static __device__ __noinline__ double edge_point_pdf(const float p[3], const float n[3], float3 v0, float3 v1, float t,
                                                     int pt) {
  double a0[3] = {(double)v0.x - p[0], (double)v0.y - p[1], (double)v0.z - p[2]};
  double E[3] = {(double)v1.x - v0.x, (double)v1.y - v0.y, (double)v1.z - v0.z};
  double N[3] = {a0[1] * E[2] - a0[2] * E[1], a0[2] * E[0] - a0[0] * E[2], a0[0] * E[1] - a0[1] * E[0]};
  double lE = sqrt(E[0] * E[0] + E[1] * E[1] + E[2] * E[2]);
  double nN = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
  double h = nN / lE;
  double e[3] = {E[0] / lE, E[1] / lE, E[2] / lE};
  double k[3] = {e[1] * N[2] - e[2] * N[1], e[2] * N[0] - e[0] * N[2], e[0] * N[1] - e[1] * N[0]};
  double np = (n[0] * k[0] + n[1] * k[1] + n[2] * k[2]) / nN;
  double ne = n[0] * e[0] + n[1] * e[1] + n[2] * e[2];
  double rho = sqrt(np * np + ne * ne);
  double s0 = a0[0] * e[0] + a0[1] * e[1] + a0[2] * e[2], s1 = s0 + lE;
  double r0 = sqrt(s0 * s0 + h * h), r1 = sqrt(s1 * s1 + h * h);
  double Ga = (pt & 2) ? (s0 / r0) * np - (h / r0) * ne : -rho;
  double Gb = (pt & 4) ? (s1 / r1) * np - (h / r1) * ne : rho;
  double w[3] = {a0[0] + (double)t * E[0], a0[1] + (double)t * E[1], a0[2] + (double)t * E[2]};
  double r2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double cw = (n[0] * w[0] + n[1] * w[1] + n[2] * w[2]) / sqrt(r2);
  double qc = cw > 0.0 ? cw * h * lE / (r2 * (Gb - Ga)) : 0.0;
  return 0.25 + 0.75 * qc;
}
template <int kSel>
__device__ __forceinline__ bool secondary_sides(const SceneView& s, const Opts& op, uint32_t c0, uint32_t c1, int b,
                                                int md, const Vertex& x, float3 n, SecGeom& gm,
                                                const int2* pre = nullptr, const int4* pre4 = nullptr) {
  uint4 r = rng4(op.key, c0, c1, kEdgeSecondary, (uint32_t)b, kPassInterior, op.scene_id);
  int e;
  float inv_pe;
  if (kSel == kSelNeePre) {
    int4 pk = *pre4;
    e = pk.x;
    inv_pe = __int_as_float(pk.y);
    if (e < 0) return false;
  } else if (kSel == kSelTreePre) {
    int2 pk = *pre;
    e = pk.x;
    inv_pe = __int_as_float(pk.y);
    if (e < 0) return false;
  } else if (kSel == kSelTree) {
    float n32[3];
    shading_normal32(x, n32);
    EtQuery q;
    et_query(s, x.p, n32, b + 1 >= md, op.eps_rel, q);
    if (!et_pick(s, q, op.sec_samples, op.key, c0, c1, (uint32_t)b, op.scene_id, e, inv_pe)) return false;
  } else {
    double stotal = s.scdf[s.E - 1];
    e = cdf_pick_guided(s.scdf, s.E, dm(u01d(r.x, r.y), stotal), s.sguide, stotal);
    double le = s.scdf[e] - (e > 0 ? s.scdf[e - 1] : 0.0);
    if (!(le > 0.0)) return false;
    inv_pe = (float)(stotal / le);
  }
  float t = kSel == kSelNeePre ? __int_as_float(pre4->z) : u01f(r.z);
  int2 ev = s.edges[e];
  float3 ve0 = ld3(s.verts + 3 * ev.x), ve1 = ld3(s.verts + 3 * ev.y);
  // which sides are traced is a discrete decision: FP32 in a fixed order
  shading_normal32(x, gm.n32);
  gm.pt = 0;
  if (op.sec_point == 1) t = edge_point_sample(x.p, gm.n32, ve0, ve1, t, u01f(r.w), gm.pt);
  float om[3], a0[3], a1[3];
  om[0] = fs(fa(ve0.x, fm(t, fs(ve1.x, ve0.x))), x.p[0]);
  om[1] = fs(fa(ve0.y, fm(t, fs(ve1.y, ve0.y))), x.p[1]);
  om[2] = fs(fa(ve0.z, fm(t, fs(ve1.z, ve0.z))), x.p[2]);
  a0[0] = fs(ve0.x, x.p[0]); a0[1] = fs(ve0.y, x.p[1]); a0[2] = fs(ve0.z, x.p[2]);
  a1[0] = fs(ve1.x, x.p[0]); a1[1] = fs(ve1.y, x.p[1]); a1[2] = fs(ve1.z, x.p[2]);
  float N32[3] = {fs(fm(a0[1], a1[2]), fm(a0[2], a1[1])), fs(fm(a0[2], a1[0]), fm(a0[0], a1[2])),
                  fs(fm(a0[0], a1[1]), fm(a0[1], a1[0]))};
  float nlen32 = fsq(dot3x(N32, N32));
  if (!(nlen32 > 0.0f)) return false;
  gm.e = e;
  gm.ev = ev;
  gm.invPE = inv_pe;
  float nh32[3] = {fdv(N32[0], nlen32), fdv(N32[1], nlen32), fdv(N32[2], nlen32)};
  gm.wl = fsq(dot3x(om, om));
  float sh = fm(op.eps_rel, gm.wl);
  gm.t = t;
  gm.ve0 = ve0;
  gm.ve1 = ve1;
  gm.last = b + 1 >= md;
  for (int side = 0; side < 2; ++side) {
    for (int i = 0; i < 3; ++i)
      gm.dsd[side][i] = side == 0 ? fa(om[i], fm(sh, nh32[i])) : fs(om[i], fm(sh, nh32[i]));
    gm.act[side] = !(dot3x(gm.n32, gm.dsd[side]) < fm(-1e-5f, gm.wl)) &&
                   !(gm.last && !may_reach_light(s, x.p, gm.dsd[side]));
  }
  return gm.act[0] || gm.act[1];
}

// Which sides of a secondary edge sample count, given the side hits hms.
__device__ __forceinline__ bool secondary_side_decide(const SceneView& s, const Vertex& x, SecGeom& gm, Hit hms[2],
                                                      bool front[2]) {
  float (*dsd)[3] = gm.dsd;
  bool* act = gm.act;
  front[0] = front[1] = false;
  for (int side = 0; side < 2; ++side) {
    if (!act[side] || hms[side].tri < 0) { act[side] = false; continue; }
    Vertex mv;
    load_vertex(s, hms[side].tri, hms[side].b1, hms[side].b2, dsd[side], mv);
    float dm32[3] = {fs(mv.p[0], x.p[0]), fs(mv.p[1], x.p[1]), fs(mv.p[2], x.p[2])};
    if (!(dot3x(gm.n32, dm32) > 0.f)) act[side] = false;
    front[side] = dot3x(mv.nu, dm32) < 0.f;
  }
  // both sides on one triangle: the edge separates no surfaces at this point,
  // so the jump of Eq. dirac_3d_edge is zero (the difference of the two
  // evaluations a finite offset apart would be an O(eps) residue)
  if (act[0] && act[1] && hms[0].tri == hms[1].tri) act[0] = act[1] = false;
  return act[0] || act[1];
}

// The side rays of the secondary edge sample at vertex b: the sample's edge,
// point and side directions (secondary_sides), both side rays traced in one
// traversal, and which sides count: a side counts when its hit lies above
// the shading horizon and, for the direct part, on the front face of a
// light, both decided in FP32 in a fixed order from the hit point, so the
// oracle takes the same decisions.  False: no side counts.
template <int kSel>
__device__ __forceinline__ bool secondary_side_hits(const SceneView& s, const Opts& op, uint32_t c0, uint32_t c1,
                                                    int b, int md, const Vertex& x, float3 n, SecGeom& gm,
                                                    Hit hms[2], bool front[2], const int2* pre = nullptr,
                                                    const int4* pre4 = nullptr) {
  front[0] = front[1] = false;
  if (!secondary_sides<kSel>(s, op, c0, c1, b, md, x, n, gm, pre, pre4)) return false;
  trace_closest2(s, x.p, gm.dsd[0], x.p, gm.dsd[1], gm.act[0], gm.act[1], x.k, x.k, hms[0], hms[1]);
  return secondary_side_decide(s, x, gm, hms, front);
}

// The edge term's contributions of a secondary edge sample whose side hits
// (and, below the last vertex, the radiance Lr arriving along each side's
// continuation path) are known: edge vertices and light vertices into so,
// the adjoint of the vertex position into dp.
__device__ __forceinline__ void secondary_contrib(const SceneView& s, const Vertex& x, float3 n, float3 alb,
                                                  float3 ab, float3 Le, const SecGeom& gm, const Hit hms[2],
                                                  const bool front[2], const float3 Lr[2], float3& dp, SecOut& so) {
  const int2 ev = gm.ev;
  const bool last = gm.last;
  const float (*dsd)[3] = gm.dsd;
  const bool* act = gm.act;
  // Geometry of the sample.  The vectors a0, a1 from p to the edge's end
  // points are nearly parallel when the edge subtends a small angle at p, so
  // their cross product is taken in the equal, well-conditioned form
  // a0 x E (E = v1 - v0); with omega = a0 + t E the indirect part's
  // derivative vectors a1 x omega_hat and omega_hat x a0 are
  // -(1 - t) a0 x E / |omega| and -t a0 x E / |omega|.
  const float3 p = f3(x.p), E = gm.ve1 - gm.ve0;
  const float3 a0v = gm.ve0 - p, a1v = gm.ve1 - p;
  const float3 Ne = cross(a0v, E);
  const float Nlen = len(Ne);
  const float3 nh = (1.f / Nlen) * Ne;
  const float3 w = a0v + gm.t * E;
  const float wl2 = dot(w, w), wl = sqrtf(wl2);
  float invPE = gm.invPE;
  if (gm.pt & 1) invPE = (float)((double)invPE / edge_point_pdf(x.p, gm.n32, gm.ve0, gm.ve1, gm.t, gm.pt));
  for (int side = 0; side < 2; ++side) {
    if (!act[side]) continue;
    float sg = side == 0 ? 1.f : -1.f;
    const Hit& hm = hms[side];
    Vertex mv;
    load_vertex(s, hm.tri, hm.b1, hm.b2, dsd[side], mv);
    float3 m = f3(mv.p);
    float3 dmp = m - p;
    float mr2 = dot(dmp, dmp);
    float3 wh = (1.f / sqrtf(mr2)) * dmp;
    float cpm = dot(n, wh);
    if (front[side] && s.light_of_tri[hm.tri] >= 0) {
      float3 nmu = f3(mv.nu);
      float3 nm = (1.f / len(nmu)) * nmu;
      float cm = -dot(nm, wh);
      float wn = dot(w, nm);
      float cr = len(cross(nm, nh));
      if (cr > 0.f) {
        float Gm = cpm * cm / mr2;
        float hs = kInvPi * Gm * (ab.x * alb.x * Le.x + ab.y * alb.y * Le.y + ab.z * alb.z * Le.z);
        float tm = dot(dmp, nm) / wn;
        float3 J = tm * (E - (dot(E, nm) / wn) * w);
        float cc = sg * hs * (len(J) / (Nlen * cr)) * invPE;
        // a1 x (m - p) and (m - p) x a0 are cross products of nearly parallel
        // vectors: exact differences and the compensated form
        float3 a0h, a0l, a1h, a1l, dmh, dml;
        two_diff3(gm.ve0, p, a0h, a0l);
        two_diff3(gm.ve1, p, a1h, a1l);
        two_diff3(m, p, dmh, dml);
        float3 gv0 = cross_comp(a1h, dmh) + (cross(a1h, dml) + cross(a1l, dmh));
        float3 gv1 = cross_comp(dmh, a0h) + (cross(dmh, a0l) + cross(dml, a0h));
        so.de0 += cc * gv0;
        so.de1 += cc * gv1;
        dp -= cc * (Ne + gv0 + gv1);
        float bw1 = hm.b1, bw2 = hm.b2, bw0 = 1.f - bw1 - bw2;
        const int32_t* mid = s.tris + 3 * hm.tri;
        for (int i = 0; i < 3; ++i) so.mid[side][i] = mid[i];
        so.dm[side][0] = (cc * bw0) * Ne;
        so.dm[side][1] = (cc * bw1) * Ne;
        so.dm[side][2] = (cc * bw2) * Ne;
        so.have_m[side] = true;
        so.have_edge = true;
      }
    }
    if (!last) {
      float3 lr = Lr[side];
      float hs = kInvPi * cpm * (ab.x * alb.x * lr.x + ab.y * alb.y * lr.y + ab.z * alb.z * lr.z);
      if (hs != 0.f) {
        float cc = sg * hs / wl2 * invPE;
        float cw = cc / wl;
        so.de0 -= (cw * (1.f - gm.t)) * Ne;
        so.de1 -= (cw * gm.t) * Ne;
        dp += cw * Ne;
        so.have_edge = true;
      }
    }
  }
  so.eid0 = ev.x;
  so.eid1 = ev.y;
}

// Evaluate the secondary edge sample at vertex b: trace both side rays (one
// traversal), their continuation paths below the last vertex, and the edge
// term's contributions: edge vertices and light vertices into so, the
// adjoint of the vertex position into dp.
template <int kSel>
__device__ __forceinline__ void secondary_at_vertex(const SceneView& s, const Opts& op, uint32_t c0, uint32_t c1,
                                                    int b, int md, const Vertex& x, float3 n, float3 alb, float3 ab,
                                                    float3 Le, float3& dp, SecOut& so, const int2* pre = nullptr,
                                                    const int4* pre4 = nullptr,
                                                    uint32_t cont_pass = kPassSecondaryBase) {
  so.de0 = so.de1 = zero3();
  so.eid0 = so.eid1 = 0;
  so.have_edge = false;
  for (int q = 0; q < 2; ++q) {
    so.have_m[q] = false;
    for (int i = 0; i < 3; ++i) { so.dm[q][i] = zero3(); so.mid[q][i] = 0; }
  }
  SecGeom gm;
  Hit hms[2];
  bool front[2];
  if (!secondary_side_hits<kSel>(s, op, c0, c1, b, md, x, n, gm, hms, front, pre, pre4)) return;
  // radiance along both continuation paths, from the hits found above
  // (cont_pass: kPassSecondaryBase, or kPassNeeBase for a billboard sample)
  float3 Lr[2] = {zero3(), zero3()};
  if (!gm.last) path_value2_from(s, op, gm.dsd, hms, gm.act, b + 1, c0, c1, cont_pass + (uint32_t)b, Lr);
  secondary_contrib(s, x, n, alb, ab, Le, gm, hms, front, Lr, dp, so);
}

// Secondary edge samples at the camera hits (depth 1), evaluated inside the
// pixel pass: the form the allocation-free backward uses, having no scratch
// for the queue of k_sec_queue / k_sec_trace.  With one scattering vertex
// only radiance arriving from a light matters (area form, reading of the
// measure), so a side ray that cannot reach a light, or that leaves below the
// shading horizon by more than the side offset, contributes exactly nothing
// and is not traced (secondary_sides).
template <int kSel>
__device__ __forceinline__ void secondary_block(const SceneView& s, const Opts& op, const int32_t* tape_tri,
                                                               const float2* tape_bary, const float* d_image, Grads gr,
                                                               int G, int rows_written, int64_t blk) {
  int lane = threadIdx.x & 31;
  int64_t gw = (blk * kBlock + threadIdx.x) >> 5;
  int ppw = 32 / G;
  int64_t pix = gw * ppw + lane / G;
  int npix = s.W * s.H;
  bool pix_ok = pix < npix && pix >= op.pix_begin && pix < op.pix_end;
  float g[kGlobals];
  for (int i = 0; i < kGlobals; ++i) g[i] = 0.f;
  float3 wpix = pix_ok ? ld3(d_image + 3 * pix) : zero3();
  float3 a = (1.0f / (float)op.spp) * wpix;
  const float3 Le = ld3(s.radiance);
  int iters = (op.spp + G - 1) / G;
  for (int it = 0; it < iters; ++it) {
    int sidx = lane % G + it * G;
    bool active = pix_ok && sidx < op.spp && !op.primary_only;
    CamHit c;
    c.k = -1;
    if (active) camera_hit(s, op, tape_tri, tape_bary, pix, sidx, c);
    float3 dv0 = zero3(), dv1 = zero3(), dv2 = zero3(), de0 = zero3(), de1 = zero3();
    float3 dmv[2][3] = {{zero3(), zero3(), zero3()}, {zero3(), zero3(), zero3()}};
    int vid0 = 0, vid1 = 0, vid2 = 0, eid0 = 0, eid1 = 0, mids[2][3] = {{0, 0, 0}, {0, 0, 0}};
    bool have_edge = false, have_m[2] = {false, false};
    if (active && c.k >= 0) {
      Vertex x;
      load_vertex(s, c.k, c.b1, c.b2, c.d, x);
      float3 dp = zero3();
      SecOut so;
      secondary_at_vertex<kSel>(s, op, (uint32_t)pix, (uint32_t)sidx, 0, 1, x, shading_normal(x),
                          ld3(s.albedo + 3 * c.k), a, Le, dp, so);
      if (so.have_edge) {
        de0 = so.de0;
        de1 = so.de1;
        eid0 = so.eid0;
        eid1 = so.eid1;
        for (int sd = 0; sd < 2; ++sd) {
          have_m[sd] = so.have_m[sd];
          for (int q = 0; q < 3; ++q) {
            dmv[sd][q] = so.dm[sd][q];
            mids[sd][q] = so.mid[sd][q];
          }
        }
        have_edge = true;
        const int32_t* vid = s.tris + 3 * c.k;
        vid0 = vid[0]; vid1 = vid[1]; vid2 = vid[2];
        hit_point_adjoint(s, c, x, dp, zero3(), dv0, dv1, dv2, g);
      }
    }
    scatter3(gr.verts, eid0, de0, have_edge);
    scatter3(gr.verts, eid1, de1, have_edge);
    scatter3(gr.verts, vid0, dv0, have_edge);
    scatter3(gr.verts, vid1, dv1, have_edge);
    scatter3(gr.verts, vid2, dv2, have_edge);
    for (int sd = 0; sd < 2; ++sd)
      for (int q = 0; q < 3; ++q) scatter3(gr.verts, mids[sd][q], dmv[sd][q], have_m[sd]);
    if (op.jac.n) {
      jac_add3(op, 0, eid0, de0, pix, have_edge);
      jac_add3(op, 0, eid1, de1, pix, have_edge);
      jac_add3(op, 0, vid0, dv0, pix, have_edge);
      jac_add3(op, 0, vid1, dv1, pix, have_edge);
      jac_add3(op, 0, vid2, dv2, pix, have_edge);
      for (int sd = 0; sd < 2; ++sd)
        for (int q = 0; q < 3; ++q) jac_add3(op, 0, mids[sd][q], dmv[sd][q], pix, have_m[sd]);
    }
  }
  jac_globals(op, g, pix, pix_ok);
  block_globals(g, gr.partials + blk * kGlobals, rows_written != 0);
}
template <int kSel>
__global__ void __launch_bounds__(kBlock, DRT_PIXEL_MIN_BLOCKS) k_backward_secondary(SceneView s, Opts op, const int32_t* tape_tri,
                                                               const float2* tape_bary, const float* d_image, Grads gr,
                                                               int G, int rows_written) {
  secondary_block<kSel>(s, op, tape_tri, tape_bary, d_image, gr, G, rows_written, blockIdx.x);
}

// kInPass: the secondary edge samples are evaluated inside this pass (no
// scratch for the queue); else their vertex adjoints come in dp_sec.
template <bool kInPass, int kSel = kSelLength>
__device__ __forceinline__ void path_block(const SceneView& s, const Opts& op, const int32_t* tape_tri,
                                           const float2* tape_bary, const float* d_image, Grads gr, int G,
                                           const float* dp_sec, int64_t blk) {
  __shared__ GradCache cv, ca;
  cache_init(cv);
  cache_init(ca);
  __syncthreads();
  int lane = threadIdx.x & 31;
  int64_t gw = (blk * kBlock + threadIdx.x) >> 5;
  int ppw = 32 / G;
  int64_t pix = gw * ppw + lane / G;
  int npix = s.W * s.H;
  bool pix_ok = pix < npix && pix >= op.pix_begin && pix < op.pix_end;
  int64_t n = (int64_t)npix * op.spp;
  int md = min(op.max_depth, kMaxDepth);
  float g[kGlobals];
  for (int i = 0; i < kGlobals; ++i) g[i] = 0.f;
  float3 wpix = pix_ok ? ld3(d_image + 3 * pix) : zero3();
  float3 a = (1.0f / (float)op.spp) * wpix;
  const float3 Le = ld3(s.radiance);
  bool do_int = (op.terms & 1) != 0, do_sec = (op.terms & 4) != 0 && s.E > 0 && s.L > 0;
  int iters = (op.spp + G - 1) / G;
  for (int it = 0; it < iters; ++it) {
    int sidx = lane % G + it * G;
    bool active = pix_ok && sidx < op.spp;
    int64_t ti = pix * op.spp + sidx;
    // forward re-evaluation from the tape
    int kk[kMaxDepth];
    float bb1[kMaxDepth], bb2[kMaxDepth], din[kMaxDepth][3], orig[kMaxDepth][3];
    bool vis[kMaxDepth];
    float3 beta[kMaxDepth];
    int nv = 0;
    CamHit c;
    c.sx = c.sy = 0.f;
    if (active) {
      jitter(op, (int)pix, sidx, s.W, &c.sx, &c.sy);
      camera_ray(s, c.sx, c.sy, c.o, c.d);
      float d[3] = {c.d[0], c.d[1], c.d[2]}, o[3] = {c.o[0], c.o[1], c.o[2]};
      float3 bt = make_float3(1.f, 1.f, 1.f);
      for (int b = 0; b < md; ++b) {
        int32_t tt = tape_tri[b * n + ti];
        if (tt == -1) break;
        kk[b] = tt & 0x7fffffff;
        vis[b] = (tt >> 31) & 1;
        float2 bb = tape_bary[b * n + ti];
        bb1[b] = bb.x;
        bb2[b] = bb.y;
        for (int i = 0; i < 3; ++i) { din[b][i] = d[i]; orig[b][i] = o[i]; }
        beta[b] = bt;
        nv = b + 1;
        if (b + 1 >= md) break;
        Vertex x;
        load_vertex(s, kk[b], bb1[b], bb2[b], d, x);
        float n32[3];
        shading_normal32(x, n32);
        uint4 r = rng4(op.key, (uint32_t)pix, (uint32_t)sidx, kBsdf, (uint32_t)b, kPassInterior, op.scene_id);
        float nd[3];
        cosine_dir(n32, u01f(r.x), u01f(r.y), nd);
        if (!(dot(f3(n32), f3(nd)) > 0.f)) break;
        bt = bt * ld3(s.albedo + 3 * kk[b]);
        for (int i = 0; i < 3; ++i) { o[i] = x.p[i]; d[i] = nd[i]; }
      }
    }
    // reverse sweep (warp-uniform trip count for the scatter)
    float3 D_next = zero3(), pbar = zero3();
    for (int b = md - 1; b >= 0; --b) {
      bool av = active && b < nv;
      float3 dv0 = zero3(), dv1 = zero3(), dv2 = zero3(), dalb = zero3(), dl[3] = {zero3(), zero3(), zero3()};
      int vid[3] = {0, 0, 0}, lid[3] = {0, 0, 0};
      bool have_light = false;
      SecOut so;
      so.have_edge = false;
      so.have_m[0] = so.have_m[1] = false;
      so.eid0 = so.eid1 = 0;
      so.de0 = so.de1 = zero3();
      for (int q = 0; q < 2; ++q)
        for (int i = 0; i < 3; ++i) { so.dm[q][i] = zero3(); so.mid[q][i] = 0; }
      if (av) {
        Vertex x;
        load_vertex(s, kk[b], bb1[b], bb2[b], din[b], x);
        const int32_t* vi = s.tris + 3 * kk[b];
        vid[0] = vi[0]; vid[1] = vi[1]; vid[2] = vi[2];
        float3 alb = ld3(s.albedo + 3 * kk[b]);
        float3 n = shading_normal(x);
        float3 ab = a * beta[b];
        float3 Dv = zero3();
        float3 dp = pbar, dn = zero3();
        float gl[kGlobals];
        for (int i = 0; i < kGlobals; ++i) gl[i] = 0.f;
        if (do_int) {
          if (b == 0 && s.light_of_tri[kk[b]] >= 0 && x.side < 0.0f) {
            Dv += Le;
            gl[0] += ab.x; gl[1] += ab.y; gl[2] += ab.z;
          }
          if (s.L > 0 && vis[b]) {
            float3 dlt[3] = {zero3(), zero3(), zero3()};
            Dv += nee_adjoint(s, op, (uint32_t)pix, (uint32_t)sidx, b, x, n, alb, ab, Le, gl, dalb, dp, dn, dlt, lid,
                              have_light);
            for (int i = 0; i < 3; ++i) dl[i] = dlt[i];
          }
          if (b + 1 < nv) {
            // beta_{b+1} = beta_b * rho_b * cos(n_b, omega_b) / cos_value (pdf held fixed)
            float3 om = f3(din[b + 1]);
            float cbar = dot(n, om);
            dalb += ab * D_next;
            float cadj = (ab.x * alb.x * D_next.x + ab.y * alb.y * D_next.y + ab.z * alb.z * D_next.z) / cbar;
            dn += cadj * om;
            Dv += alb * D_next;
          }
        }
        if (do_sec) {
          if (kInPass)
            secondary_at_vertex<kSel>(s, op, (uint32_t)pix, (uint32_t)sidx, b, md, x, n, alb, ab, Le, dp, so);
          else if (dp_sec)  // evaluated apart (queued samples only)
            dp += ld3(dp_sec + 3 * (ti * md + b));
        }
        for (int i = 0; i < kGlobals; ++i) g[i] += gl[i];
        float3 do_, dd_;
        plane_hit_adjoint(orig[b], din[b], x, dp, dn, dv0, dv1, dv2, do_, dd_);
        if (b == 0) camera_ray_adjoint(s, c.sx, c.sy, do_, dd_, g);
        pbar = do_;  // the origin of ray b is vertex b-1 (its direction is held fixed)
        D_next = Dv;
      }
      scatter3_call(gr.verts, vid[0], dv0, av, &cv);
      scatter3_call(gr.verts, vid[1], dv1, av, &cv);
      scatter3_call(gr.verts, vid[2], dv2, av, &cv);
      scatter3_call(gr.albedo, av ? kk[b] : 0, dalb, av && do_int, &ca);
      for (int i = 0; i < 3; ++i) scatter3_call(gr.verts, lid[i], dl[i], have_light, &cv);
      scatter3_call(gr.verts, so.eid0, so.de0, so.have_edge, &cv);
      scatter3_call(gr.verts, so.eid1, so.de1, so.have_edge, &cv);
      for (int q = 0; q < 2; ++q)
        for (int i = 0; i < 3; ++i) scatter3_call(gr.verts, so.mid[q][i], so.dm[q][i], so.have_m[q], &cv);
      if (op.jac.n) {
        jac_add3(op, 0, vid[0], dv0, pix, av);
        jac_add3(op, 0, vid[1], dv1, pix, av);
        jac_add3(op, 0, vid[2], dv2, pix, av);
        jac_add3(op, op.jac.v3, av ? kk[b] : 0, dalb, pix, av && do_int);
        for (int i = 0; i < 3; ++i) jac_add3(op, 0, lid[i], dl[i], pix, have_light);
        jac_add3(op, 0, so.eid0, so.de0, pix, so.have_edge);
        jac_add3(op, 0, so.eid1, so.de1, pix, so.have_edge);
        for (int q = 0; q < 2; ++q)
          for (int i = 0; i < 3; ++i) jac_add3(op, 0, so.mid[q][i], so.dm[q][i], pix, so.have_m[q]);
      }
    }
  }
  __syncthreads();
  cache_flush(cv, gr.verts);
  cache_flush(ca, gr.albedo);
  jac_globals(op, g, pix, pix_ok);
  block_globals(g, gr.partials + blk * kGlobals, false);
}
template <int kSel>
__global__ void __launch_bounds__(kBlock, 1)
    k_backward_path_in_pass(SceneView s, Opts op, const int32_t* tape_tri, const float2* tape_bary,
                            const float* d_image, Grads gr, int G) {
  path_block<true, kSel>(s, op, tape_tri, tape_bary, d_image, gr, G, nullptr, blockIdx.x);
}
__global__ void __launch_bounds__(kBlock, DRT_PATH_MIN_BLOCKS)
    k_backward_path(SceneView s, Opts op, const int32_t* tape_tri, const float2* tape_bary, const float* d_image,
                    Grads gr, int G, const float* dp_sec) {
  path_block<false>(s, op, tape_tri, tape_bary, d_image, gr, G, dp_sec, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Secondary edge samples traced apart from the pixel passes.  Only a small
// share of them can contribute (most side rays leave below the shading
// horizon or, at the last vertex, cannot reach a light); traced inside the
// pixel passes, those few lanes hold back their warps and blocks.  A first
// pass queues the (sample, vertex) pairs that have a side to trace; a second
// traces only those, scatters the edge and light-vertex gradients and writes
// the adjoint of the vertex position, which the pixel pass adds where it
// chains hit-point adjoints back to the camera.  Same arithmetic as the
// evaluation inside the pixel passes.
// ---------------------------------------------------------------------------
// Vertex b of the camera path of sample (pix, sidx), re-evaluated from the
// tape (vertex 0 from the camera ray; traced when there is no tape, which
// only depth 1 allows).  beta = throughput before vertex b.  False: the path
// has no vertex b.
__device__ __forceinline__ bool tape_vertex(const SceneView& s, const Opts& op, const int32_t* tape_tri,
                                            const float2* tape_bary, int64_t pix, int sidx, int b, int md, Vertex& x,
                                            float3& beta) {
  CamHit c;
  camera_hit(s, op, tape_tri, tape_bary, pix, sidx, c);
  if (c.k < 0) return false;
  int64_t n = (int64_t)s.W * s.H * op.spp, ti = pix * op.spp + sidx;
  float d[3] = {c.d[0], c.d[1], c.d[2]};
  int k = c.k;
  float b1 = c.b1, b2 = c.b2;
  float3 bt = make_float3(1.f, 1.f, 1.f);
  for (int q = 0;; ++q) {
    load_vertex(s, k, b1, b2, d, x);
    if (q == b) {
      beta = bt;
      return true;
    }
    if (q + 1 >= md) return false;
    float n32[3];
    shading_normal32(x, n32);
    uint4 r = rng4(op.key, (uint32_t)pix, (uint32_t)sidx, kBsdf, (uint32_t)q, kPassInterior, op.scene_id);
    float nd[3];
    cosine_dir(n32, u01f(r.x), u01f(r.y), nd);
    if (!(dot(f3(n32), f3(nd)) > 0.f)) return false;
    bt = bt * ld3(s.albedo + 3 * k);
    for (int i = 0; i < 3; ++i) d[i] = nd[i];
    int32_t tt = tape_tri[(q + 1) * n + ti];
    if (tt == -1) return false;
    k = tt & 0x7fffffff;
    float2 bb = tape_bary[(q + 1) * n + ti];
    b1 = bb.x;
    b2 = bb.y;
  }
}

// Pass 1: one thread per sample walks its path and queues each vertex whose
// secondary sample has a side to trace (pixels with a zero loss adjoint
// contribute nothing and are skipped).  Warp-aggregated appends.
template <int kSel>
__global__ void __launch_bounds__(kBlock, kSel == kSelLength ? DRT_QUEUE_MIN_BLOCKS : DRT_TREE_QUEUE_MIN_BLOCKS) k_sec_queue(BatchScene bs) {
  const SceneView& s = bs.v;
  const Opts& op = bs.op;
  int lane = threadIdx.x & 31;
  int64_t n = (int64_t)s.W * s.H * op.spp;
  int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  int md = op.primary_only ? 1 : min(op.max_depth, kMaxDepth);
  bool alive = i < n;
  int64_t pix = alive ? i / op.spp : 0;
  int sidx = alive ? (int)(i % op.spp) : 0;
  alive = alive && pix >= op.pix_begin && pix < op.pix_end;
  if (alive) {
    float3 w = ld3(bs.d_image + 3 * pix);
    alive = w.x != 0.f || w.y != 0.f || w.z != 0.f;
  }
  CamHit c;
  c.k = -1;
  if (alive) {
    camera_hit(s, op, bs.tape_tri, bs.tape_bary, pix, sidx, c);
    alive = c.k >= 0;
  }
  float d[3] = {c.d[0], c.d[1], c.d[2]};
  int k = c.k;
  float b1 = c.b1, b2 = c.b2;
  for (int b = 0; b < md; ++b) {
    Vertex x;
    bool need = false;
    SecGeom gm;
    if (alive) {
      load_vertex(s, k, b1, b2, d, x);
      need = secondary_sides<kSel>(s, op, (uint32_t)pix, (uint32_t)sidx, b, md, x, shading_normal(x), gm);
    }
    unsigned m = __ballot_sync(kFull, need);
    if (m) {
      int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(bs.sec_count + b, (unsigned long long)__popc(m));
      base = __shfl_sync(kFull, base, leader);
      if (need) {
        // the queue holds one region of n slots per path vertex, so the
        // trace kernel's warps take samples of one vertex (equal remaining
        // depth, similar work) together
        unsigned long long slot = (unsigned long long)b * (unsigned long long)n + base +
                                  __popc(m & ((1u << lane) - 1u));
        bs.sec_queue[slot] = ((unsigned long long)i << 3) | (unsigned)b;
        if (kSel == kSelTree) bs.sec_pick[slot] = make_int2(gm.e, __float_as_int(gm.invPE));
      }
    }
    if (alive) {  // on to vertex b + 1
      if (b + 1 >= md) {
        alive = false;
      } else {
        float n32[3];
        shading_normal32(x, n32);
        uint4 r = rng4(op.key, (uint32_t)pix, (uint32_t)sidx, kBsdf, (uint32_t)b, kPassInterior, op.scene_id);
        float nd[3];
        cosine_dir(n32, u01f(r.x), u01f(r.y), nd);
        if (!(dot(f3(n32), f3(nd)) > 0.f)) {
          alive = false;
        } else {
          for (int q = 0; q < 3; ++q) d[q] = nd[q];
          int32_t tt = bs.tape_tri[(int64_t)(b + 1) * n + i];
          if (tt == -1) {
            alive = false;
          } else {
            k = tt & 0x7fffffff;
            float2 bb = bs.tape_bary[(int64_t)(b + 1) * n + i];
            b1 = bb.x;
            b2 = bb.y;
          }
        }
      }
    }
  }
}

// Queue of next-event estimation for edges (Sec. 5.3.3), beside the length
// sampler: per (sample, vertex) the length sample and the billboard sample
// of the vertex's shadow ray, each with its balance-heuristic weight
// 1 / (p_length + w p_billboard) and its point, into the regions of their
// kind (length: vertex b; billboard: depth + b).  The length sample's u is
// uniform in [-w/2, w/2]; its p_billboard comes from a query along the ray
// of its family through (t, u).  Same random numbers and arithmetic as the
// oracle's secondary edge sample with next-event estimation for edges.
__device__ __forceinline__ void sec_push(const BatchScene& bs, int region, unsigned long long n, bool need,
                                         unsigned long long item, int4 rec) {
  int lane = threadIdx.x & 31;
  unsigned m = __ballot_sync(kFull, need);
  if (!m) return;
  int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(bs.sec_count + region, (unsigned long long)__popc(m));
  base = __shfl_sync(kFull, base, leader);
  if (need) {
    unsigned long long slot = (unsigned long long)region * n + base + __popc(m & ((1u << lane) - 1u));
    bs.sec_queue[slot] = item;
    bs.sec_nee[slot] = rec;
  }
}

__global__ void __launch_bounds__(kBlock, DRT_TREE_QUEUE_MIN_BLOCKS) k_sec_queue_nee(BatchScene bs) {
  const SceneView& s = bs.v;
  const Opts& op = bs.op;
  int64_t n = (int64_t)s.W * s.H * op.spp;
  int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  int md = op.primary_only ? 1 : min(op.max_depth, kMaxDepth);
  bool alive = i < n;
  int64_t pix = alive ? i / op.spp : 0;
  int sidx = alive ? (int)(i % op.spp) : 0;
  alive = alive && pix >= op.pix_begin && pix < op.pix_end;
  if (alive) {
    float3 w = ld3(bs.d_image + 3 * pix);
    alive = w.x != 0.f || w.y != 0.f || w.z != 0.f;
  }
  CamHit c;
  c.k = -1;
  if (alive) {
    camera_hit(s, op, bs.tape_tri, bs.tape_bary, pix, sidx, c);
    alive = c.k >= 0;
  }
  const float hw = op.nee_hw > 0.0f ? op.nee_hw : (op.nee_hw_dev ? *op.nee_hw_dev : 0.0f);
  const double width = 2.0 * (double)hw;
  const double stotal = s.scdf[s.E - 1];
  float d[3] = {c.d[0], c.d[1], c.d[2]};
  int k = c.k;
  float b1 = c.b1, b2 = c.b2;
  for (int b = 0; b < md; ++b) {
    Vertex x;
    bool needA = false, needB = false;
    int4 recA = make_int4(-1, 0, 0, 0), recB = make_int4(-1, 0, 0, 0);
    if (alive) {
      load_vertex(s, k, b1, b2, d, x);
      float3 nrm = shading_normal(x);
      float n32[3];
      shading_normal32(x, n32);
      uint4 rn = rng4(op.key, (uint32_t)pix, (uint32_t)sidx, kEdgeNee, (uint32_t)b, kPassInterior, op.scene_id);
      SecGeom gm;
      needA = secondary_sides<kSelLength>(s, op, (uint32_t)pix, (uint32_t)sidx, b, md, x, nrm, gm);
      if (needA) {
        float uA = fm(hw, fs(fm(2.0f, u01f(rn.x)), 1.0f));
        double pB = 0.0;
        float dA[3];
        if (nee_ray(gm.ve0, gm.ve1, x.p, gm.t, uA, dA)) {
          NeeHits h;
          nee_light_hits(s, x.p, dA, h);
          if (h.n > 0) {
            NeeQuery o;
            nee_query(s, x.p, n32, dA, hw, 0.0f, make_uint2(0u, 0u), gm.e, h, o);
            pB = nee_density(o, h, nee_jacobian(gm.ve0, gm.ve1, x.p, gm.t, uA));
          }
        }
        double le = s.scdf[gm.e] - (gm.e > 0 ? s.scdf[gm.e - 1] : 0.0);
        recA = make_int4(gm.e, __float_as_int((float)(1.0 / (le / stotal + width * pB))), __float_as_int(gm.t), 0);
      }
      if (s.L > 0) {
        // the shadow ray of this vertex's next-event estimation, drawn again
        uint4 rl = rng4(op.key, (uint32_t)pix, (uint32_t)sidx, kLight, (uint32_t)b, kPassInterior, op.scene_id);
        LightSample ls;
        sample_light(s, rl, ls);
        float dB[3] = {fs(ls.y[0], x.p[0]), fs(ls.y[1], x.p[1]), fs(ls.y[2], x.p[2])};
        float Tj, tb1, tb2;
        if (watertight(make_shear(dB), x.p, ls.l0, ls.l1, ls.l2, INFINITY, &Tj, &tb1, &tb2)) {
          NeeHits h;
          nee_light_hits(s, x.p, dB, h);
          NeeQuery o;
          nee_query(s, x.p, n32, dB, hw, Tj, make_uint2(rn.z, rn.w), -1, h, o);
          if (o.has_win) {
            o.timp = o.win.imp;
            o.ts = o.win.s;
            int2 ev = s.edges[o.win.eid];
            float3 v0 = ld3(s.verts + 3 * ev.x), v1 = ld3(s.verts + 3 * ev.y);
            double pB = nee_density(o, h, nee_jacobian(v0, v1, x.p, o.win.t, o.win.u));
            double le = s.scdf[o.win.eid] - (o.win.eid > 0 ? s.scdf[o.win.eid - 1] : 0.0);
            double den = le / stotal + width * pB;
            if (den > 0.0) {
              recB = make_int4(o.win.eid, __float_as_int((float)(1.0 / den)), __float_as_int(o.win.t), 0);
              SecGeom gb;
              needB = secondary_sides<kSelNeePre>(s, op, (uint32_t)pix, (uint32_t)sidx, b, md, x, nrm, gb, nullptr,
                                                  &recB);
            }
          }
        }
      }
    }
    unsigned long long item = ((unsigned long long)i << 3) | (unsigned)b;
    sec_push(bs, b, (unsigned long long)n, needA, item, recA);
    sec_push(bs, md + b, (unsigned long long)n, needB, item, recB);
    if (alive) {  // on to vertex b + 1
      if (b + 1 >= md) {
        alive = false;
      } else {
        float n32[3];
        shading_normal32(x, n32);
        uint4 r = rng4(op.key, (uint32_t)pix, (uint32_t)sidx, kBsdf, (uint32_t)b, kPassInterior, op.scene_id);
        float nd[3];
        cosine_dir(n32, u01f(r.x), u01f(r.y), nd);
        if (!(dot(f3(n32), f3(nd)) > 0.f)) {
          alive = false;
        } else {
          for (int q = 0; q < 3; ++q) d[q] = nd[q];
          int32_t tt = bs.tape_tri[(int64_t)(b + 1) * n + i];
          if (tt == -1) {
            alive = false;
          } else {
            k = tt & 0x7fffffff;
            float2 bb = bs.tape_bary[(int64_t)(b + 1) * n + i];
            b1 = bb.x;
            b2 = bb.y;
          }
        }
      }
    }
  }
}

// regions of the secondary queue: one per path vertex, and as many again for
// the billboard samples of next-event estimation for edges
__device__ __forceinline__ int sec_regions(const Opts& op, int md) { return op.nee ? 2 * md : md; }
// queue slot of the qq-th queued sample (R regions of n slots, in order)
__device__ __forceinline__ unsigned long long sec_slot(const unsigned long long* cnt, int R, unsigned long long n,
                                                       unsigned long long qq) {
  for (int b = 0; b < R; ++b) {
    if (qq < cnt[b]) return (unsigned long long)b * n + qq;
    qq -= cnt[b];
  }
  return qq;
}

// Pass 2: the queued (sample, vertex) pairs, a block-stride loop over the
// vertex regions of the queue in order (first vertex first: its samples
// carry the longest continuation paths); vertex gradients through the block
// cache (the light's vertices take contributions from most samples).
template <int kSel>
__global__ void __launch_bounds__(kBlock, DRT_SEC_MIN_BLOCKS) k_sec_trace(BatchScene bs) {
  __shared__ GradCache cv;
  const SceneView& s = bs.v;
  const Opts& op = bs.op;
  int md = op.primary_only ? 1 : min(op.max_depth, kMaxDepth);
  const float3 Le = ld3(s.radiance);
  const unsigned long long n_region = (unsigned long long)s.W * s.H * op.spp;
  const int R = sec_regions(op, md);
  __shared__ unsigned long long cnt[2 * kMaxDepth];
  if (threadIdx.x < 2 * kMaxDepth) cnt[threadIdx.x] = (int)threadIdx.x < R ? bs.sec_count[threadIdx.x] : 0ull;
  __syncthreads();
  unsigned long long count = 0;
  for (int b = 0; b < R; ++b) count += cnt[b];
  for (unsigned long long base = (unsigned long long)blockIdx.x * kBlock; base < count;
       base += (unsigned long long)gridDim.x * kBlock) {
    cache_init(cv);
    __syncthreads();
    int64_t jpix = 0;  // pixel of the queued sample (per-pixel gradient image)
    // queue slot of the queued sample: region, offset within it
    unsigned long long q = sec_slot(cnt, R, n_region, base + threadIdx.x);
    SecOut so;
    so.have_edge = false;
    so.have_m[0] = so.have_m[1] = false;
    so.eid0 = so.eid1 = 0;
    so.de0 = so.de1 = zero3();
    for (int h = 0; h < 2; ++h)
      for (int j = 0; j < 3; ++j) { so.dm[h][j] = zero3(); so.mid[h][j] = 0; }
    if (base + threadIdx.x < count) {
      unsigned long long item = bs.sec_queue[q];
      int64_t i = (int64_t)(item >> 3);
      int b = (int)(item & 7u);
      int64_t pix = i / op.spp;
      jpix = pix;
      int sidx = (int)(i % op.spp);
      Vertex x;
      float3 beta;
      if (tape_vertex(s, op, bs.tape_tri, bs.tape_bary, pix, sidx, b, md, x, beta)) {
        float3 ab = ((1.0f / (float)op.spp) * ld3(bs.d_image + 3 * pix)) * beta;
        float3 dp = zero3();
        secondary_at_vertex<kSel>(s, op, (uint32_t)pix, (uint32_t)sidx, b, md, x, shading_normal(x),
                                  ld3(s.albedo + 3 * x.k), ab, Le, dp, so, bs.sec_pick + q, bs.sec_nee + q,
                                  q >= (unsigned long long)md * n_region ? kPassNeeBase : kPassSecondaryBase);
        // a vertex's length and billboard samples add to one slot (two
        // additions onto zero: the same sum in either order)
        float* o = bs.dp_sec + 3 * (i * md + b);
        atomicAdd(o, dp.x);
        atomicAdd(o + 1, dp.y);
        atomicAdd(o + 2, dp.z);
      }
    }
    scatter3(bs.d_verts, so.eid0, so.de0, so.have_edge, &cv);
    scatter3(bs.d_verts, so.eid1, so.de1, so.have_edge, &cv);
    for (int h = 0; h < 2; ++h)
      for (int j = 0; j < 3; ++j) scatter3(bs.d_verts, so.mid[h][j], so.dm[h][j], so.have_m[h], &cv);
    if (op.jac.n) {
      jac_add3(op, 0, so.eid0, so.de0, jpix, so.have_edge);
      jac_add3(op, 0, so.eid1, so.de1, jpix, so.have_edge);
      for (int h = 0; h < 2; ++h)
        for (int j = 0; j < 3; ++j) jac_add3(op, 0, so.mid[h][j], so.dm[h][j], jpix, so.have_m[h]);
    }
    __syncthreads();
    cache_flush(cv, bs.d_verts);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Queued secondary edge samples beyond depth 1, in stages.  With one thread
// per queued sample carrying both side paths to the last vertex, a warp's
// lanes trace from one to five traversals each (side rays, then next-event
// and continuation rays at every later vertex) and most lanes idle while a
// few finish their paths.  Here (1) k_sec_sides traces the side rays of every
// queued sample and stores the hits; (2) k_sec_bounce, launched once per
// remaining vertex, advances every live pair of continuation paths by one
// vertex (next-event ray pair, then the continuation ray pair) and adds the
// radiance they gather; (3) k_sec_finish evaluates the edge term from the
// stored hits and radiance.  Same random numbers and arithmetic as
// path_value2_from and secondary_at_vertex; the sample's geometry is
// recomputed in stage 3 (a pure function of the sample and its vertex).
// ---------------------------------------------------------------------------
struct SecPathState {
  float4 a;  // d0.xyz, beta0.x
  float4 b;  // d1.xyz, beta0.y
  float4 c;  // beta0.z, beta1.xyz
  float4 d;  // b1_0, b2_0, b1_1, b2_1
  int4 e;    // queue slot, tri0, tri1, vertex | alive0 << 8 | alive1 << 9
};
static_assert(sizeof(SecPathState) == 5 * sizeof(float4), "path state is five float4");

__device__ __forceinline__ void sec_push_path(const BatchScene& bs, int buf, bool push, const SecPathState& st) {
  int lane = threadIdx.x & 31;
  unsigned m = __ballot_sync(kFull, push);
  if (!m) return;
  int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(bs.sec_path_count + buf, (unsigned long long)__popc(m));
  base = __shfl_sync(kFull, base, leader);
  if (push) {
    unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
    reinterpret_cast<SecPathState*>(bs.sec_path[buf])[slot] = st;
  }
}

// Stage 1: side rays of every queued sample; samples above the last vertex
// start their continuation paths in state buffer 0.
template <int kSel>
__global__ void __launch_bounds__(kBlock, DRT_SIDES_MIN_BLOCKS) k_sec_sides(BatchScene bs) {
  const SceneView& s = bs.v;
  const Opts& op = bs.op;
  int md = op.primary_only ? 1 : min(op.max_depth, kMaxDepth);
  const unsigned long long n_region = (unsigned long long)s.W * s.H * op.spp;
  const int R = sec_regions(op, md);
  __shared__ unsigned long long cnt[2 * kMaxDepth];
  if (threadIdx.x < 2 * kMaxDepth) cnt[threadIdx.x] = (int)threadIdx.x < R ? bs.sec_count[threadIdx.x] : 0ull;
  __syncthreads();
  unsigned long long count = 0;
  for (int b = 0; b < R; ++b) count += cnt[b];
  for (unsigned long long base = (unsigned long long)blockIdx.x * kBlock; base < count;
       base += (unsigned long long)gridDim.x * kBlock) {
    bool in = base + threadIdx.x < count;
    unsigned long long q = in ? sec_slot(cnt, R, n_region, base + threadIdx.x) : 0ull;
    bool push = false;
    SecPathState st;
    if (in) {
      unsigned long long item = bs.sec_queue[q];
      int64_t i = (int64_t)(item >> 3);
      int b = (int)(item & 7u);
      int64_t pix = i / op.spp;
      int sidx = (int)(i % op.spp);
      Vertex x;
      float3 beta;
      int flags = 0;
      Hit hms[2];
      hms[0].tri = hms[1].tri = -1;
      hms[0].b1 = hms[0].b2 = hms[1].b1 = hms[1].b2 = 0.f;
      bool last = b + 1 >= md;
      if (tape_vertex(s, op, bs.tape_tri, bs.tape_bary, pix, sidx, b, md, x, beta)) {
        SecGeom gm;
        bool front[2];
        if (secondary_side_hits<kSel>(s, op, (uint32_t)pix, (uint32_t)sidx, b, md, x, shading_normal(x), gm, hms,
                                      front, bs.sec_pick + q, bs.sec_nee + q)) {
          flags = (gm.act[0] ? 1 : 0) | (gm.act[1] ? 2 : 0) | (front[0] ? 4 : 0) | (front[1] ? 8 : 0);
          if (!last) {
            push = true;
            st.a = make_float4(gm.dsd[0][0], gm.dsd[0][1], gm.dsd[0][2], 1.f);
            st.b = make_float4(gm.dsd[1][0], gm.dsd[1][1], gm.dsd[1][2], 1.f);
            st.c = make_float4(1.f, 1.f, 1.f, 1.f);
            st.d = make_float4(hms[0].b1, hms[0].b2, hms[1].b1, hms[1].b2);
            st.e = make_int4((int)(uint32_t)q, hms[0].tri, hms[1].tri,
                             (b + 1) | (gm.act[0] ? 256 : 0) | (gm.act[1] ? 512 : 0));
          }
        }
      }
      bs.sec_hits[2 * q] = make_int4(hms[0].tri, __float_as_int(hms[0].b1), __float_as_int(hms[0].b2), flags);
      bs.sec_hits[2 * q + 1] = make_int4(hms[1].tri, __float_as_int(hms[1].b1), __float_as_int(hms[1].b2), 0);
      if (!last) {
        float* lr = bs.sec_lr + 6 * q;
        for (int k = 0; k < 6; ++k) lr[k] = 0.f;
      }
    }
    sec_push_path(bs, 0, push, st);
  }
}

// Continuation paths in stages, shared by the secondary and the primary edge
// samples: one launch per path vertex advances every live pair of side paths
// (both sides of one edge sample, a tiny offset apart, with the same random
// numbers) by one vertex.  An entry holds either the hits at its vertex or,
// when `pending`, the rays leaving the previous vertex (origin = that
// vertex's FP32 hit point, recomputed from its triangle and barycentrics);
// pending rays are traced first, both sides in one traversal.
struct PathStage {
  float4* path[2];             // state buffers (SecPathState), ping-pong
  unsigned long long* count;   // [2] entries in each buffer
  float* lr;                   // [slots, 6] radiance gathered by each side
};
// sources of continuation paths: secondary edge samples (pairs of side
// paths), primary edge samples (pairs), camera paths of the render (one path
// per entry, side 1 unused; radiance per sample in lr[3 i], tape entries
// written at every vertex)
enum { kSrcSecondary = 0, kSrcPrimary = 1, kSrcRender = 2 };
constexpr int kPathPending = 1024;

__device__ __forceinline__ void path_push(const PathStage& ps, int buf, bool push, const SecPathState& st) {
  int lane = threadIdx.x & 31;
  unsigned m = __ballot_sync(kFull, push);
  if (!m) return;
  int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(ps.count + buf, (unsigned long long)__popc(m));
  base = __shfl_sync(kFull, base, leader);
  if (push) {
    unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
    reinterpret_cast<SecPathState*>(ps.path[buf])[slot] = st;
  }
}

// Every live pair in buffer `in`: (pending rays traced first) next-event
// estimation at its vertex, and above the last vertex the continuation
// directions, pushed as pending rays to the other buffer.  Random numbers:
// secondary samples use the counters of their queued (sample, vertex) and
// pass kPassSecondaryBase + vertex; primary samples (slot = position in
// screen order) the edge sample's index and kPassPrimaryEdge.
template <int kSrc>
__global__ void __launch_bounds__(kBlock, DRT_BOUNCE_MIN_BLOCKS) k_path_bounce(BatchScene bs, PathStage ps, int in) {
  const SceneView& s = bs.v;
  const Opts& op = bs.op;
  int md = op.primary_only ? 1 : min(op.max_depth, kMaxDepth);
  const float3 Le = ld3(s.radiance);
  unsigned long long count = ps.count[in];
  const SecPathState* src = reinterpret_cast<const SecPathState*>(ps.path[in]);
  for (unsigned long long base = (unsigned long long)blockIdx.x * kBlock; base < count;
       base += (unsigned long long)gridDim.x * kBlock) {
    unsigned long long e = base + threadIdx.x;
    bool push = false;
    SecPathState st;
    if (e < count) {
      st = src[e];
      unsigned long long q = (uint32_t)st.e.x;
      uint32_t c0, c1, pass;
      if (kSrc == kSrcSecondary) {
        unsigned long long item = bs.sec_queue[q];
        int64_t i = (int64_t)(item >> 3);
        c0 = (uint32_t)(i / op.spp);
        c1 = (uint32_t)(i % op.spp);
        // billboard samples (regions from md on) continue with their own pass
        bool nee_slot = q >= (unsigned long long)md * ((unsigned long long)s.W * s.H * op.spp);
        pass = (nee_slot ? kPassNeeBase : kPassSecondaryBase) + (uint32_t)(item & 7u);
      } else if (kSrc == kSrcPrimary) {
        c0 = bs.order ? (uint32_t)bs.order[q] : (uint32_t)q;
        c1 = 0u;
        pass = kPassPrimaryEdge;
      } else {
        c0 = (uint32_t)(q / (unsigned long long)op.spp);
        c1 = (uint32_t)(q % (unsigned long long)op.spp);
        pass = kPassInterior;
      }
      int bb = st.e.w & 255;
      bool alive[2] = {(st.e.w & 256) != 0, (st.e.w & 512) != 0};
      float d[2][3] = {{st.a.x, st.a.y, st.a.z}, {st.b.x, st.b.y, st.b.z}};
      float3 beta[2] = {make_float3(st.a.w, st.b.w, st.c.x), make_float3(st.c.y, st.c.z, st.c.w)};
      Hit h[2];
      h[0].tri = st.e.y; h[0].b1 = st.d.x; h[0].b2 = st.d.y; h[0].t = 0.f;
      h[1].tri = st.e.z; h[1].b1 = st.d.z; h[1].b2 = st.d.w; h[1].t = 0.f;
      if (st.e.w & kPathPending) {
        float o[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        int exclude[2] = {-1, -1};
        for (int k = 0; k < 2; ++k) {
          if (!alive[k]) continue;
          Vertex xo;
          load_vertex(s, h[k].tri, h[k].b1, h[k].b2, d[k], xo);
          for (int j = 0; j < 3; ++j) o[k][j] = xo.p[j];
          exclude[k] = h[k].tri;
        }
        trace_closest2(s, o[0], d[0], o[1], d[1], alive[0], alive[1], exclude[0], exclude[1], h[0], h[1]);
      }
      Vertex x[2];
      float3 alb[2];
      for (int k = 0; k < 2; ++k) {
        alb[k] = zero3();
        if (!alive[k]) continue;
        if (h[k].tri < 0) { alive[k] = false; continue; }
        load_vertex(s, h[k].tri, h[k].b1, h[k].b2, d[k], x[k]);
        alb[k] = ld3(s.albedo + 3 * x[k].k);
      }
      if (alive[0] || alive[1]) {
        int vis = 0;  // render: the vertex's next-event ray reached the light (tape bit)
        float n32[2][3];
        for (int k = 0; k < 2; ++k)
          if (alive[k]) shading_normal32(x[k], n32[k]);
        if (s.L > 0) {
          uint4 r = rng4(op.key, c0, c1, kLight, (uint32_t)bb, pass, op.scene_id);
          LightSample ls;
          sample_light(s, r, ls);
          float sd[2][3];
          for (int k = 0; k < 2; ++k)
            if (alive[k])
              for (int j = 0; j < 3; ++j) sd[k][j] = fs(ls.y[j], x[k].p[j]);
          bool occ[2];
          trace_any2(s, x[0].p, sd[0], x[0].k, ls.lt, x[1].p, sd[1], x[1].k, ls.lt, alive[0], alive[1],
                     kShadowTmax, occ[0], occ[1]);
          float* lr = ps.lr + (kSrc == kSrcRender ? 3 : 6) * q;
          for (int k = 0; k < 2; ++k)
            if (alive[k] && !occ[k]) {
              float g = nee_geometry(s, f3(x[k].p), f3(n32[k]), ls);
              float3 acc = make_float3(lr[3 * k], lr[3 * k + 1], lr[3 * k + 2]);
              nee_add(acc, kInvPi * g, beta[k] * alb[k] * Le);
              lr[3 * k] = acc.x;
              lr[3 * k + 1] = acc.y;
              lr[3 * k + 2] = acc.z;
              if (kSrc == kSrcRender) vis = 1;
            }
        }
        if (kSrc == kSrcRender && alive[0] && bs.tape_tri) {
          const int64_t n = (int64_t)s.W * s.H * op.spp;
          bs.tape_tri[(int64_t)bb * n + (int64_t)q] = x[0].k | (vis << 31);
          bs.tape_bary[(int64_t)bb * n + (int64_t)q] = make_float2(h[0].b1, h[0].b2);
        }
        if (bb + 1 < md) {
          uint4 r = rng4(op.key, c0, c1, kBsdf, (uint32_t)bb, pass, op.scene_id);
          for (int k = 0; k < 2; ++k) {
            if (!alive[k]) continue;
            float nd[3];
            cosine_dir(n32[k], u01f(r.x), u01f(r.y), nd);
            if (!(dot(f3(n32[k]), f3(nd)) > 0.f)) { alive[k] = false; continue; }
            beta[k] = beta[k] * alb[k];
            for (int j = 0; j < 3; ++j) d[k][j] = nd[j];
          }
          if (alive[0] || alive[1]) {
            push = true;
            st.a = make_float4(d[0][0], d[0][1], d[0][2], beta[0].x);
            st.b = make_float4(d[1][0], d[1][1], d[1][2], beta[0].y);
            st.c = make_float4(beta[0].z, beta[1].x, beta[1].y, beta[1].z);
            st.d = make_float4(h[0].b1, h[0].b2, h[1].b1, h[1].b2);
            st.e = make_int4(st.e.x, alive[0] ? h[0].tri : -1, alive[1] ? h[1].tri : -1,
                             (bb + 1) | (alive[0] ? 256 : 0) | (alive[1] ? 512 : 0) | kPathPending);
          }
        }
      }
    }
    path_push(ps, in ^ 1, push, st);
  }
}

// The continuation step of k_path_bounce split around two persistent
// traversal pools (trace_pool.cuh), so that the traversals of incoherent rays
// keep their lanes busy: phase 0 writes the pending rays of every entry (a
// closest-hit pair record), the pool traces them; phase 1 resolves the hits
// and writes the next-event rays (an any-hit pair record), the pool traces
// those; phase 2 adds the next-event radiance, writes the render's tape
// entries and pushes the continuation.  Same random numbers and arithmetic
// as k_path_bounce.
struct PoolBufs {
  float4* crec;   // [entries, kClosestRecF4]
  int4* hits;     // [entries, 2]
  float4* arec;   // [entries, kAnyRecF4]
  int* occ;       // [entries]
  unsigned long long* next;  // [2] fetch counters of the two pools
};

template <int kSrc, int kPhase>
__global__ void __launch_bounds__(kBlock) k_bounce_phase(BatchScene bs, PathStage ps, int in, PoolBufs pb) {
  const SceneView& s = bs.v;
  const Opts& op = bs.op;
  int md = op.primary_only ? 1 : min(op.max_depth, kMaxDepth);
  const float3 Le = ld3(s.radiance);
  unsigned long long count = ps.count[in];
  const SecPathState* src = reinterpret_cast<const SecPathState*>(ps.path[in]);
  for (unsigned long long base = (unsigned long long)blockIdx.x * kBlock; base < count;
       base += (unsigned long long)gridDim.x * kBlock) {
    unsigned long long e = base + threadIdx.x;
    bool push = false;
    SecPathState st;
    if (e < count) {
      st = src[e];
      unsigned long long q = (uint32_t)st.e.x;
      uint32_t c0, c1, pass;
      if (kSrc == kSrcSecondary) {
        unsigned long long item = bs.sec_queue[q];
        int64_t i = (int64_t)(item >> 3);
        c0 = (uint32_t)(i / op.spp);
        c1 = (uint32_t)(i % op.spp);
        bool nee_slot = q >= (unsigned long long)md * ((unsigned long long)s.W * s.H * op.spp);
        pass = (nee_slot ? kPassNeeBase : kPassSecondaryBase) + (uint32_t)(item & 7u);
      } else if (kSrc == kSrcPrimary) {
        c0 = bs.order ? (uint32_t)bs.order[q] : (uint32_t)q;
        c1 = 0u;
        pass = kPassPrimaryEdge;
      } else {
        c0 = (uint32_t)(q / (unsigned long long)op.spp);
        c1 = (uint32_t)(q % (unsigned long long)op.spp);
        pass = kPassInterior;
      }
      int bb = st.e.w & 255;
      bool pending = (st.e.w & kPathPending) != 0;
      bool alive[2] = {(st.e.w & 256) != 0, (st.e.w & 512) != 0};
      float d[2][3] = {{st.a.x, st.a.y, st.a.z}, {st.b.x, st.b.y, st.b.z}};
      float3 beta[2] = {make_float3(st.a.w, st.b.w, st.c.x), make_float3(st.c.y, st.c.z, st.c.w)};
      Hit h[2];
      h[0].tri = st.e.y; h[0].b1 = st.d.x; h[0].b2 = st.d.y; h[0].t = 0.f;
      h[1].tri = st.e.z; h[1].b1 = st.d.z; h[1].b2 = st.d.w; h[1].t = 0.f;
      if (kPhase == 0) {
        // the pending rays leave the previous vertex (its FP32 hit point)
        float4* r = pb.crec + (size_t)kClosestRecF4 * e;
        for (int k = 0; k < 2; ++k) {
          float o[3] = {0.f, 0.f, 0.f};
          bool act = pending && alive[k];
          if (act) {
            Vertex xo;
            load_vertex(s, h[k].tri, h[k].b1, h[k].b2, d[k], xo);
            for (int j = 0; j < 3; ++j) o[j] = xo.p[j];
          }
          r[2 * k] = make_float4(o[0], o[1], o[2], __int_as_float(act ? h[k].tri : -1));
          r[2 * k + 1] = make_float4(d[k][0], d[k][1], d[k][2], act ? 1.0f : 0.0f);
        }
      } else {
        if (pending)
          for (int k = 0; k < 2; ++k) {
            if (!alive[k]) continue;
            int4 hv = pb.hits[2 * e + k];
            h[k].tri = hv.x;
            h[k].t = __int_as_float(hv.y);
            h[k].b1 = __int_as_float(hv.z);
            h[k].b2 = __int_as_float(hv.w);
          }
        Vertex x[2];
        float3 alb[2];
        for (int k = 0; k < 2; ++k) {
          alb[k] = zero3();
          if (!alive[k]) continue;
          if (h[k].tri < 0) { alive[k] = false; continue; }
          load_vertex(s, h[k].tri, h[k].b1, h[k].b2, d[k], x[k]);
          alb[k] = ld3(s.albedo + 3 * x[k].k);
        }
        float n32[2][3];
        for (int k = 0; k < 2; ++k)
          if (alive[k]) shading_normal32(x[k], n32[k]);
        LightSample ls;
        float sd[2][3] = {{0.f, 0.f, 1.f}, {0.f, 0.f, 1.f}};
        if (s.L > 0 && (alive[0] || alive[1])) {
          uint4 r = rng4(op.key, c0, c1, kLight, (uint32_t)bb, pass, op.scene_id);
          sample_light(s, r, ls);
          for (int k = 0; k < 2; ++k)
            if (alive[k])
              for (int j = 0; j < 3; ++j) sd[k][j] = fs(ls.y[j], x[k].p[j]);
        }
        if (kPhase == 1) {
          float4* r = pb.arec + (size_t)kAnyRecF4 * e;
          bool act[2] = {s.L > 0 && alive[0], s.L > 0 && alive[1]};
          for (int k = 0; k < 2; ++k) {
            r[2 * k] = make_float4(act[k] ? x[k].p[0] : 0.f, act[k] ? x[k].p[1] : 0.f, act[k] ? x[k].p[2] : 0.f,
                                   __int_as_float(act[k] ? x[k].k : -1));
            r[2 * k + 1] = make_float4(sd[k][0], sd[k][1], sd[k][2], __int_as_float(act[k] ? ls.lt : -1));
          }
          r[4] = make_float4(act[0] ? 1.f : 0.f, act[1] ? 1.f : 0.f, 0.f, 0.f);
        } else {
          int vis = 0;
          if (s.L > 0 && (alive[0] || alive[1])) {
            int oc = pb.occ[e];
            bool occ[2] = {(oc & 1) != 0, (oc & 2) != 0};
            float* lr = ps.lr + (kSrc == kSrcRender ? 3 : 6) * q;
            for (int k = 0; k < 2; ++k)
              if (alive[k] && !occ[k]) {
                float g = nee_geometry(s, f3(x[k].p), f3(n32[k]), ls);
                float3 acc = make_float3(lr[3 * k], lr[3 * k + 1], lr[3 * k + 2]);
                nee_add(acc, kInvPi * g, beta[k] * alb[k] * Le);
                lr[3 * k] = acc.x;
                lr[3 * k + 1] = acc.y;
                lr[3 * k + 2] = acc.z;
                if (kSrc == kSrcRender) vis = 1;
              }
          }
          if (kSrc == kSrcRender && alive[0] && bs.tape_tri) {
            const int64_t n = (int64_t)s.W * s.H * op.spp;
            bs.tape_tri[(int64_t)bb * n + (int64_t)q] = x[0].k | (vis << 31);
            bs.tape_bary[(int64_t)bb * n + (int64_t)q] = make_float2(h[0].b1, h[0].b2);
          }
          if ((alive[0] || alive[1]) && bb + 1 < md) {
            uint4 r = rng4(op.key, c0, c1, kBsdf, (uint32_t)bb, pass, op.scene_id);
            for (int k = 0; k < 2; ++k) {
              if (!alive[k]) continue;
              float nd[3];
              cosine_dir(n32[k], u01f(r.x), u01f(r.y), nd);
              if (!(dot(f3(n32[k]), f3(nd)) > 0.f)) { alive[k] = false; continue; }
              beta[k] = beta[k] * alb[k];
              for (int j = 0; j < 3; ++j) d[k][j] = nd[j];
            }
            if (alive[0] || alive[1]) {
              push = true;
              st.a = make_float4(d[0][0], d[0][1], d[0][2], beta[0].x);
              st.b = make_float4(d[1][0], d[1][1], d[1][2], beta[0].y);
              st.c = make_float4(beta[0].z, beta[1].x, beta[1].y, beta[1].z);
              st.d = make_float4(h[0].b1, h[0].b2, h[1].b1, h[1].b2);
              st.e = make_int4(st.e.x, alive[0] ? h[0].tri : -1, alive[1] ? h[1].tri : -1,
                               (bb + 1) | (alive[0] ? 256 : 0) | (alive[1] ? 512 : 0) | kPathPending);
            }
          }
        }
      }
    }
    if (kPhase == 2) path_push(ps, in ^ 1, push, st);
  }
}

// Resident CTAs of the pool kernels on the device (a persistent launch).
template <bool kPair>
static int pool_grid_size() {
  static int g = 0;
  if (g == 0) {
    int dev = 0, sms = 0, b1 = 0, b2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_pool_closest<kPair>, 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_pool_any<kPair>, 256, 0);
    g = std::max(1, sms) * std::max(1, std::min(b1, b2));
  }
  return g;
}

// One continuation level through the pools: phase 0, closest-hit pool,
// phase 1, any-hit pool, phase 2 (entries read from buffer `in`).
template <int kSrc>
cudaError_t launch_bounce_level(const BatchScene& bs, const PathStage& ps, int in, const PoolBufs& pb,
                                int64_t grid, const char* name, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ps.count + (in ^ 1), 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(pb.next, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  unsigned g = (unsigned)std::max<int64_t>(grid, 1);
  ProfToken pt = prof_begin(name, st);
  k_bounce_phase<kSrc, 0><<<g, kBlock, 0, st>>>(bs, ps, in, pb);
  // a camera path is one ray per record; an edge sample's two side paths, two
  constexpr bool kPair = kSrc != kSrcRender;
  const int pool_grid = pool_grid_size<kPair>();
  k_pool_closest<kPair><<<pool_grid, 256, 0, st>>>(bs.v, pb.crec, ps.count + in, pb.hits, pb.next);
  k_bounce_phase<kSrc, 1><<<g, kBlock, 0, st>>>(bs, ps, in, pb);
  k_pool_any<kPair><<<pool_grid, 256, 0, st>>>(bs.v, pb.arec, ps.count + in, pb.occ, pb.next + 1);
  k_bounce_phase<kSrc, 2><<<g, kBlock, 0, st>>>(bs, ps, in, pb);
  prof_end(pt, st);
  return cudaGetLastError();
}


__host__ __forceinline__ PoolBufs pool_of(const BatchScene& b) {
  return PoolBufs{b.pool_crec, b.pool_hits, b.pool_arec, b.pool_occ, b.pool_next};
}

// The render beyond one vertex in stages.  k_render_first: the first vertex
// of every camera path with the warp-cooperative traversal (the lanes of a
// warp hold one pixel's samples, so their rays are coherent), its tape entry
// and radiance (emission and next-event estimation), and the continuation
// pushed as a pending ray.  k_path_bounce<kSrcRender>: one launch per later
// vertex over the live paths only, so a warp holds live paths whatever their
// pixels.  k_render_finish: the pixel means in the fused kernel's order.
// Same random numbers, tape entries and image as k_render.
__global__ void __launch_bounds__(kBlock, DRT_RENDER_MIN_BLOCKS)
    k_render_first(SceneView s, Opts op, int32_t* tape_tri, float2* tape_bary, int G, PathStage ps) {
  int lane = threadIdx.x & 31;
  int64_t gw = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
  int ppw = 32 / G;
  int64_t pix = gw * ppw + lane / G;
  int npix = s.W * s.H;
  bool active = pix < npix;
  int iters = (op.spp + G - 1) / G;
  for (int it = 0; it < iters; ++it) {
    int sidx = lane % G + it * G;
    bool act = active && sidx < op.spp;
    float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 1.f};
    if (act) {
      float sx, sy;
      jitter(op, (int)pix, sidx, s.W, &sx, &sy);
      camera_ray(s, sx, sy, o, d);
    }
    int64_t i = pix * op.spp + sidx;
    bool cont;
    Hit h0;
    float nd[3];
    float3 alb;
    int vis = 0;
    float3 L0 = path_first_vertex_warp(s, op, o, d, act, (uint32_t)pix, (uint32_t)sidx, kPassInterior, cont, h0, nd,
                                       alb, &vis);
    bool hit = act && h0.tri >= 0;
    if (act) {
      float* lr = ps.lr + 3 * i;
      lr[0] = L0.x;
      lr[1] = L0.y;
      lr[2] = L0.z;
      if (tape_tri) {
        tape_tri[i] = hit ? (h0.tri | (vis << 31)) : -1;
        tape_bary[i] = make_float2(hit ? h0.b1 : 0.f, hit ? h0.b2 : 0.f);
      }
    }
    bool push = act && cont;
    SecPathState st;
    if (push) {
      st.a = make_float4(nd[0], nd[1], nd[2], alb.x);
      st.b = make_float4(0.f, 0.f, 1.f, alb.y);
      st.c = make_float4(alb.z, 0.f, 0.f, 0.f);
      st.d = make_float4(h0.b1, h0.b2, 0.f, 0.f);
      st.e = make_int4((int)(uint32_t)i, h0.tri, -1, 1 | 256 | kPathPending);
    }
    path_push(ps, 0, push, st);
  }
}

__global__ void __launch_bounds__(kBlock) k_render_finish(SceneView s, Opts op, float* image, int G, const float* L) {
  int lane = threadIdx.x & 31;
  int64_t gw = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
  int ppw = 32 / G;
  int64_t pix = gw * ppw + lane / G;
  int npix = s.W * s.H;
  bool active = pix < npix;
  float3 acc = zero3();
  int iters = (op.spp + G - 1) / G;
  for (int it = 0; it < iters; ++it) {
    int sidx = lane % G + it * G;
    if (active && sidx < op.spp) {
      const float* l = L + 3 * (pix * op.spp + sidx);
      acc += make_float3(l[0], l[1], l[2]);
    }
  }
  for (int o = G >> 1; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(kFull, acc.x, o);
    acc.y += __shfl_xor_sync(kFull, acc.y, o);
    acc.z += __shfl_xor_sync(kFull, acc.z, o);
  }
  if (active && lane % G == 0) {
    float inv = 1.0f / (float)op.spp;
    image[3 * pix] = acc.x * inv;
    image[3 * pix + 1] = acc.y * inv;
    image[3 * pix + 2] = acc.z * inv;
  }
}

// Stage 3: the edge term of every queued sample from its stored side hits
// and continuation radiance; vertex gradients through the block cache.
template <int kSel>
__global__ void __launch_bounds__(kBlock, DRT_FINISH_MIN_BLOCKS) k_sec_finish(BatchScene bs) {
  __shared__ GradCache cv;
  const SceneView& s = bs.v;
  const Opts& op = bs.op;
  int md = op.primary_only ? 1 : min(op.max_depth, kMaxDepth);
  const float3 Le = ld3(s.radiance);
  const unsigned long long n_region = (unsigned long long)s.W * s.H * op.spp;
  const int R = sec_regions(op, md);
  __shared__ unsigned long long cnt[2 * kMaxDepth];
  if (threadIdx.x < 2 * kMaxDepth) cnt[threadIdx.x] = (int)threadIdx.x < R ? bs.sec_count[threadIdx.x] : 0ull;
  __syncthreads();
  unsigned long long count = 0;
  for (int b = 0; b < R; ++b) count += cnt[b];
  for (unsigned long long base = (unsigned long long)blockIdx.x * kBlock; base < count;
       base += (unsigned long long)gridDim.x * kBlock) {
    cache_init(cv);
    __syncthreads();
    SecOut so;
    so.have_edge = false;
    so.have_m[0] = so.have_m[1] = false;
    so.eid0 = so.eid1 = 0;
    so.de0 = so.de1 = zero3();
    for (int h = 0; h < 2; ++h)
      for (int j = 0; j < 3; ++j) { so.dm[h][j] = zero3(); so.mid[h][j] = 0; }
    int64_t jpix = 0;  // pixel of the queued sample (per-pixel gradient image)
    if (base + threadIdx.x < count) {
      unsigned long long q = sec_slot(cnt, R, n_region, base + threadIdx.x);
      int4 h0 = bs.sec_hits[2 * q], h1 = bs.sec_hits[2 * q + 1];
      int flags = h0.w;
      unsigned long long item = bs.sec_queue[q];
      int64_t i = (int64_t)(item >> 3);
      int b = (int)(item & 7u);
      int64_t pix = i / op.spp;
      jpix = pix;
      int sidx = (int)(i % op.spp);
      Vertex x;
      float3 beta;
      SecGeom gm;
      if ((flags & 3) && tape_vertex(s, op, bs.tape_tri, bs.tape_bary, pix, sidx, b, md, x, beta)) {
        float3 n = shading_normal(x);
        if (secondary_sides<kSel>(s, op, (uint32_t)pix, (uint32_t)sidx, b, md, x, n, gm, bs.sec_pick + q,
                                  bs.sec_nee + q)) {
          gm.act[0] = (flags & 1) != 0;
          gm.act[1] = (flags & 2) != 0;
          bool front[2] = {(flags & 4) != 0, (flags & 8) != 0};
          Hit hms[2];
          hms[0].tri = h0.x; hms[0].b1 = __int_as_float(h0.y); hms[0].b2 = __int_as_float(h0.z); hms[0].t = 0.f;
          hms[1].tri = h1.x; hms[1].b1 = __int_as_float(h1.y); hms[1].b2 = __int_as_float(h1.z); hms[1].t = 0.f;
          float3 Lr[2] = {zero3(), zero3()};
          if (!gm.last) {
            const float* lr = bs.sec_lr + 6 * q;
            Lr[0] = make_float3(lr[0], lr[1], lr[2]);
            Lr[1] = make_float3(lr[3], lr[4], lr[5]);
          }
          float3 ab = ((1.0f / (float)op.spp) * ld3(bs.d_image + 3 * pix)) * beta;
          float3 dp = zero3();
          secondary_contrib(s, x, n, ld3(s.albedo + 3 * x.k), ab, Le, gm, hms, front, Lr, dp, so);
          // length and billboard samples of a vertex share the slot (two
          // additions onto zero: the same sum in either order)
          float* o = bs.dp_sec + 3 * (i * md + b);
          atomicAdd(o, dp.x);
          atomicAdd(o + 1, dp.y);
          atomicAdd(o + 2, dp.z);
        }
      }
    }
    scatter3(bs.d_verts, so.eid0, so.de0, so.have_edge, &cv);
    scatter3(bs.d_verts, so.eid1, so.de1, so.have_edge, &cv);
    for (int h = 0; h < 2; ++h)
      for (int j = 0; j < 3; ++j) scatter3(bs.d_verts, so.mid[h][j], so.dm[h][j], so.have_m[h], &cv);
    if (op.jac.n) {
      jac_add3(op, 0, so.eid0, so.de0, jpix, so.have_edge);
      jac_add3(op, 0, so.eid1, so.de1, jpix, so.have_edge);
      for (int h = 0; h < 2; ++h)
        for (int j = 0; j < 3; ++j) jac_add3(op, 0, so.mid[h][j], so.dm[h][j], jpix, so.have_m[h]);
    }
    __syncthreads();
    cache_flush(cv, bs.d_verts);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Backward: primary edge samples (Eq. mc)
// ---------------------------------------------------------------------------
// Sample j: edge by the clipped-length CDF, uniform point on the clipped
// segment (exact decision-path arithmetic).
struct EdgeSample {
  int e, seg;
  bool valid;
  float ax, ay, bx, by, dx, dy, x, y;
  float t;             // fisheye: parameter of the point along the 3D edge
  double inv_pdf_len;  // 1 / (point density per unit screen length); fisheye: 1 / P(edge)
};
// An edge sample as four float4 (bit for bit), written by the key pass by
// sample index, gathered into screen order after the sort, and read there by
// the kernels that evaluate it.  The first float4 alone (point, direction;
// NaN point: no valid sample) is what the first vertex of the side paths
// needs.
__device__ __forceinline__ void store_sample(float4* rec, int64_t j, const EdgeSample& es) {
  float4* r = rec + 4 * j;
  r[0] = es.valid ? make_float4(es.x, es.y, es.dx, es.dy) : make_float4(NAN, NAN, NAN, NAN);
  r[1] = make_float4(es.ax, es.ay, es.bx, es.by);
  r[2] = make_float4(es.t, __int_as_float(es.e), __int_as_float(es.seg), es.valid ? 1.0f : 0.0f);
  r[3] = make_float4(__int_as_float(__double2loint(es.inv_pdf_len)), __int_as_float(__double2hiint(es.inv_pdf_len)),
                     0.0f, 0.0f);
}
__device__ __forceinline__ EdgeSample load_sample_point(const float4* pts, int64_t i) {
  float4 a = pts[i];
  EdgeSample es = {};
  es.x = a.x; es.y = a.y; es.dx = a.z; es.dy = a.w;
  es.valid = !isnan(a.x);
  return es;
}
// A point of a 3D edge, v0 + t (v1 - v0), FP32 in a fixed order.
__device__ __forceinline__ void edge_point3(float3 v0, float3 v1, float t, float p[3]) {
  p[0] = fa(v0.x, fm(t, fs(v1.x, v0.x)));
  p[1] = fa(v0.y, fm(t, fs(v1.y, v0.y)));
  p[2] = fa(v0.z, fm(t, fs(v1.z, v0.z)));
}
// Plain sampler: edge by clipped length, uniform point.  Learned proposal:
// tile segment by the mixture CDF, uniform point on the segment.
__device__ __forceinline__ EdgeSample primary_sample(const SceneView& s, const Opts& op, int64_t j, double ptotal) {
  uint4 r = rng4(op.key, (uint32_t)j, 0u, kEdgePrimary, 0u, kPassPrimaryEdge, op.scene_id);
  EdgeSample es;
  float t0, t1;
  es.valid = true;
  es.seg = -1;
  es.t = 0.f;
  if (s.cam_type == 2) {
    // fisheye (Sec. 5.2, non-linear projections): the edge by its chord on the
    // unit sphere of directions, t uniform in [0, 1), the point's image x(t)
    // on the curved edge image; the side offset runs perpendicular to the
    // FP32 chord of x(t - 1/1024) and x(t + 1/1024) (clamped to the edge)
    es.e = cdf_pick_guided(s.pcdf, s.E, dm(u01d(r.x, r.y), ptotal), s.pguide, ptotal);
    double pe = s.pcdf[es.e] - (es.e > 0 ? s.pcdf[es.e - 1] : 0.0);
    es.inv_pdf_len = pe > 0.0 ? ddv(ptotal, pe) : 0.0;
    es.ax = es.ay = es.bx = es.by = 0.f;
    es.t = u01f(r.z);
    int2 ev = s.edges[es.e];
    float3 v0 = ld3(s.verts + 3 * ev.x), v1 = ld3(s.verts + 3 * ev.y);
    float p[3], q0[3], q1[3];
    edge_point3(v0, v1, es.t, p);
    float ta = fmaxf(fs(es.t, 0.0009765625f), 0.0f), tb = fminf(fa(es.t, 0.0009765625f), 1.0f);
    edge_point3(v0, v1, ta, q0);
    edge_point3(v0, v1, tb, q1);
    float x0 = 0.f, y0 = 0.f, x1 = 0.f, y1 = 0.f;
    es.x = es.y = 0.f;
    bool ok = pe > 0.0 && fisheye_project(s, p, &es.x, &es.y) && fisheye_project(s, q0, &x0, &y0) &&
              fisheye_project(s, q1, &x1, &y1);
    ok = ok && es.x >= 0.0f && es.x < (float)s.W && es.y >= 0.0f && es.y < (float)s.H;
    es.dx = fs(x1, x0);
    es.dy = fs(y1, y0);
    es.valid = ok && fsq(fa(fm(es.dx, es.dx), fm(es.dy, es.dy))) > 0.0f;
    return es;
  }
  if (s.seg_cdf) {
    double qt = s.seg_cdf[s.n_seg - 1];
    int k = cdf_pick(s.seg_cdf, s.n_seg, dm(u01d(r.x, r.y), qt));
    double q = s.seg_cdf[k] - (k > 0 ? s.seg_cdf[k - 1] : 0.0);
    es.valid = q > 0.0;
    es.seg = k;
    es.e = s.seg_edge[k];
    float2 ss = s.seg_s[k];
    t0 = ss.x;
    t1 = ss.y;
    es.inv_pdf_len = ddv(s.seg_len[k], ddv(q, qt));
  } else {
    es.e = cdf_pick_guided(s.pcdf, s.E, dm(u01d(r.x, r.y), ptotal), s.pguide, ptotal);
    es.inv_pdf_len = ptotal;
  }
  const float4* row = reinterpret_cast<const float4*>(s.pedge + 8 * es.e);
  float4 r0 = row[0], r1 = row[1];
  es.ax = r0.x; es.ay = r0.y; es.bx = r0.z; es.by = r0.w;
  if (!s.seg_cdf) {
    t0 = r1.x;
    t1 = r1.y;
  }
  es.dx = fs(es.bx, es.ax);
  es.dy = fs(es.by, es.ay);
  float t = fa(t0, fm(u01f(r.z), fs(t1, t0)));
  es.x = fa(es.ax, fm(t, es.dx));
  es.y = fa(es.ay, fm(t, es.dy));
  return es;
}

__device__ __forceinline__ uint32_t spread_bits16(uint32_t x) {
  x &= 0xffffu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

// Screen-space Morton key of every primary edge sample, so the samples can be
// evaluated in screen order (coherent rays, aggregated scatter).  Only the
// evaluation order changes; each sample's arithmetic is the same.
// The samples in screen order (scattered reads once here, sequential reads
// in the kernels that evaluate them): sample order[i]'s first float4 (point
// and direction) to pts[i], its other three to rest[3 i .. 3 i + 2].
__global__ void k_gather_samples(const float4* rec, const int32_t* order, int64_t n, float4* pts, float4* rest) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // one float4 each
  if (k >= 4 * n) return;
  int64_t i = k >> 2;
  int c = (int)(k & 3);
  float4 v = rec[4 * (int64_t)order[i] + c];
  if (c == 0) pts[i] = v;
  else rest[3 * i + c - 1] = v;
}
// A sample in screen order from the gathered arrays.
__device__ __forceinline__ EdgeSample load_sorted_sample(const float4* pts, const float4* rest, int64_t i) {
  float4 a = pts[i], b = rest[3 * i], c = rest[3 * i + 1], d = rest[3 * i + 2];
  EdgeSample es;
  es.x = a.x; es.y = a.y; es.dx = a.z; es.dy = a.w;
  es.ax = b.x; es.ay = b.y; es.bx = b.z; es.by = b.w;
  es.t = c.x;
  es.e = __float_as_int(c.y);
  es.seg = __float_as_int(c.z);
  es.valid = c.w != 0.0f;
  es.inv_pdf_len = __hiloint2double(__float_as_int(d.y), __float_as_int(d.x));
  return es;
}
__global__ void k_primary_keys(SceneView s, Opts op, int64_t n_edge, uint32_t* keys, int32_t* vals, float4* rec) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_edge) return;
  double ptotal = s.pcdf[s.E - 1];
  uint32_t key = 0;
  if (ptotal > 0.0) {
    EdgeSample es = primary_sample(s, op, j, ptotal);
    if (rec) store_sample(rec, j, es);  // the evaluation reads it back
    // position at 1/kKeySub of a pixel
    int px = min(max((int)floorf(es.x * kKeySub), 0), s.W * kKeySub - 1);
    int py = min(max((int)floorf(es.y * kKeySub), 0), s.H * kKeySub - 1);
    key = spread_bits16((uint32_t)px) | (spread_bits16((uint32_t)py) << 1);
  }
  keys[j] = key;
  vals[j] = (int32_t)j;
}
// Two lanes per edge sample: the even lane traces the side at +eps, the odd
// lane the side at -eps, each a single-ray warp-cooperative path (as the
// camera paths of the forward pass); the pair exchanges radiance with one
// shuffle and the even lane forms the difference, the adjoint and the scatter.
constexpr int kPrimaryPerRound = kBlock / 2;  // edge samples per block and round
// kStage: the fused evaluation (kPrimFused); or, for paths beyond one
// vertex, the first vertex of both side paths with their continuation pushed
// to the path stages (kPrimFirst), and the edge term from the radiance the
// stages gathered (kPrimFinish).  Same samples, lanes and partial-sum rows.
enum { kPrimFused = 0, kPrimFirst = 1, kPrimFinish = 2 };
template <int kStage = kPrimFused>
__device__ __forceinline__ void primary_block(const SceneView& s, const Opts& op, const float* d_image, Grads gr,
                                              int64_t n_edge, int64_t per_thread, const int32_t* order,
                                              int64_t blk, PathStage ps = PathStage{},
                                              const float4* pts = nullptr, const float4* rest = nullptr) {
  float g[kGlobals];
  for (int i = 0; i < kGlobals; ++i) g[i] = 0.f;
  double ptotal = s.pcdf[s.E - 1];
  float W = (float)s.W, H = (float)s.H;
  float eps = fm(op.eps_rel, fmaxf(W, H));
  const double inv_n = 1.0 / (double)n_edge;  // Eq. mc averages over the N edge samples
  const int side = threadIdx.x & 1;
  for (int64_t it = 0; it < per_thread; ++it) {
    // consecutive lane pairs take consecutive entries of the screen-ordered list
    int64_t i = blk * kPrimaryPerRound * per_thread + it * kPrimaryPerRound + (threadIdx.x >> 1);
    int64_t j = i < n_edge ? (order ? (int64_t)order[i] : i) : n_edge;
    bool active = j < n_edge && ptotal > 0.0 && j >= op.edge_begin && j < op.edge_end;
    float3 da3 = zero3(), db3 = zero3();
    int ia = 0, ib = 0;
    int64_t jpix = 0;  // pixel containing the sample's point (per-pixel gradient image)
    float gs[kGlobals];  // this sample's share of the global parameters
    for (int q = 0; q < kGlobals; ++q) gs[q] = 0.f;
    EdgeSample es = {};
    if (active && side == 0) {
      // pts, rest: the samples in screen order (position i)
      es = !pts ? primary_sample(s, op, j, ptotal)
                : (kStage == kPrimFirst ? load_sample_point(pts, i) : load_sorted_sample(pts, rest, i));
      active = es.valid;
    }
    // the odd lane takes the sample's point and direction from its pair
    float x = __shfl_sync(kFull, es.x, threadIdx.x & ~1), y = __shfl_sync(kFull, es.y, threadIdx.x & ~1);
    float dx = __shfl_sync(kFull, es.dx, threadIdx.x & ~1), dy = __shfl_sync(kFull, es.dy, threadIdx.x & ~1);
    active = __shfl_sync(kFull, active, threadIdx.x & ~1);
    float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 1.f};
    float3 w = zero3();
    if (active) {
      float nlen = fsq(fa(fm(dx, dx), fm(dy, dy)));
      float nx = fdv(-dy, nlen), ny = fdv(dx, nlen);
      float xs = side == 0 ? fa(x, fm(eps, nx)) : fs(x, fm(eps, nx));
      float ys = side == 0 ? fa(y, fm(eps, ny)) : fs(y, fm(eps, ny));
      int px = min(max((int)floorf(x), 0), s.W - 1), py = min(max((int)floorf(y), 0), s.H - 1);
      jpix = (int64_t)py * s.W + px;
      w = ld3(d_image + 3 * jpix);
      if (kStage != kPrimFinish) camera_ray(s, xs, ys, o, d);
    }
    float3 Lme, Lot;
    if (kStage == kPrimFused) {
      int ftri = -1;
      Lme = path_value_warp(s, op, o, d, active, (uint32_t)j, 0u, kPassPrimaryEdge, nullptr, nullptr, 0, 0, &ftri,
                            true);
      Lot = make_float3(__shfl_xor_sync(kFull, Lme.x, 1), __shfl_xor_sync(kFull, Lme.y, 1),
                        __shfl_xor_sync(kFull, Lme.z, 1));
      // both sides see the same triangle first: the edge bounds nothing
      // visible there and the sample's term is zero
      int ftri_other = __shfl_xor_sync(kFull, ftri, 1);
      if (ftri >= 0 && ftri == ftri_other) Lme = Lot = zero3();
    } else if (kStage == kPrimFirst) {
      bool cont;
      Hit h0;
      float nd[3];
      float3 alb;
      float3 L0 = path_first_vertex_warp(s, op, o, d, active, (uint32_t)j, 0u, kPassPrimaryEdge, cont, h0, nd, alb,
                                         nullptr, true);
      // both sides see the same triangle first: the sample's term is zero
      // and its paths need not go on
      int ftri = active ? h0.tri : -1;
      int ftri_other = __shfl_xor_sync(kFull, ftri, 1);
      bool same = ftri >= 0 && ftri == ftri_other;
      if (same) L0 = zero3();
      if (active) {
        float* lr = ps.lr + 6 * i + 3 * side;
        lr[0] = L0.x;
        lr[1] = L0.y;
        lr[2] = L0.z;
      }
      // the pair's two continuation rays become one pending entry of the
      // path stages, pushed by the even lane
      cont = cont && active && !same;
      bool cont1 = __shfl_xor_sync(kFull, cont, 1);
      int tri1 = __shfl_xor_sync(kFull, h0.tri, 1);
      float b11 = __shfl_xor_sync(kFull, h0.b1, 1), b21 = __shfl_xor_sync(kFull, h0.b2, 1);
      float nd1[3] = {__shfl_xor_sync(kFull, nd[0], 1), __shfl_xor_sync(kFull, nd[1], 1),
                      __shfl_xor_sync(kFull, nd[2], 1)};
      float3 alb1 = make_float3(__shfl_xor_sync(kFull, alb.x, 1), __shfl_xor_sync(kFull, alb.y, 1),
                                __shfl_xor_sync(kFull, alb.z, 1));
      bool push = side == 0 && (cont || cont1);
      SecPathState st;
      if (push) {
        st.a = make_float4(nd[0], nd[1], nd[2], alb.x);
        st.b = make_float4(nd1[0], nd1[1], nd1[2], alb.y);
        st.c = make_float4(alb.z, alb1.x, alb1.y, alb1.z);
        st.d = make_float4(h0.b1, h0.b2, b11, b21);
        st.e = make_int4((int)(uint32_t)i, cont ? h0.tri : -1, cont1 ? tri1 : -1,
                         1 | (cont ? 256 : 0) | (cont1 ? 512 : 0) | kPathPending);
      }
      path_push(ps, 0, push, st);
      continue;
    } else {
      Lme = Lot = zero3();
      if (active && side == 0) {
        const float* lr = ps.lr + 6 * i;
        Lme = make_float3(lr[0], lr[1], lr[2]);
        Lot = make_float3(lr[3], lr[4], lr[5]);
      }
    }
    if (side != 0) active = false;
    if (active) {
      int e = es.e;
      float ax = es.ax, ay = es.ay, bx = es.bx, by = es.by;
      // w . (Lme - Lot) with every rounding written out: the fused and the
      // staged kernels must form the same value from the same radiance
      float diff = __fmaf_rn(w.z, __fsub_rn(Lme.z, Lot.z),
                             __fmaf_rn(w.y, __fsub_rn(Lme.y, Lot.y), __fmul_rn(w.x, __fsub_rn(Lme.x, Lot.x))));
      if (op.seg_log && es.seg >= 0) atomicAdd(op.seg_log + es.seg, fabsf(diff));
      if (diff != 0.f && s.cam_type == 2) {
        // the curved edge image: alpha = x'_y X - x'_x Y at the sample's
        // point (-perp(x') . x, perp pointing to the side at +eps)
        int2 ev = s.edges[e];
        ia = ev.x; ib = ev.y;
        float3 v0 = ld3(s.verts + 3 * ia), v1 = ld3(s.verts + 3 * ib);
        float pt[3];
        edge_point3(v0, v1, es.t, pt);
        float2 xt = fisheye_tangent(s, f3(pt), v1 - v0);
        float c = diff * (float)(es.inv_pdf_len * inv_n);
        float3 dvp = fisheye_project_adjoint(s, f3(pt), c * xt.y, -c * xt.x, gs);
        da3 = (1.f - es.t) * dvp;
        db3 = es.t * dvp;
        for (int q = 0; q < kGlobals; ++q) g[q] += gs[q];
      } else if (diff != 0.f) {
        float gl = sqrtf((ax - bx) * (ax - bx) + (ay - by) * (ay - by));
        float c = diff * (float)(es.inv_pdf_len * inv_n) / gl;
        float dax = c * (by - y), day = c * (x - bx), dbx = c * (y - ay), dby = c * (ax - x);
        int2 ev = s.edges[e];
        ia = ev.x; ib = ev.y;
        da3 = project_adjoint(s, ld3(s.verts + 3 * ia), dax, day, gs);
        db3 = project_adjoint(s, ld3(s.verts + 3 * ib), dbx, dby, gs);
        for (int q = 0; q < kGlobals; ++q) g[q] += gs[q];
      } else {
        active = false;
      }
    }
    scatter3(gr.verts, ia, da3, active);
    scatter3(gr.verts, ib, db3, active);
    if (op.jac.n) {
      jac_add3(op, 0, ia, da3, jpix, active);
      jac_add3(op, 0, ib, db3, jpix, active);
      jac_globals(op, gs, jpix, active);
    }
  }
  if (kStage != kPrimFirst) block_globals(g, gr.partials + blk * kGlobals, false);
}
__global__ void __launch_bounds__(kBlock, DRT_PRIMARY_MIN_BLOCKS) k_backward_primary(SceneView s, Opts op, const float* d_image, Grads gr,
                                                             int64_t n_edge, int64_t per_thread,
                                                             const int32_t* order, const float4* pts,
                                                             const float4* rest) {
  primary_block(s, op, d_image, gr, n_edge, per_thread, order, blockIdx.x, PathStage{}, pts, rest);
}
__global__ void __launch_bounds__(kBlock, DRT_PRIMARY_MIN_BLOCKS)
    k_primary_first(SceneView s, Opts op, const float* d_image, Grads gr, int64_t n_edge, int64_t per_thread,
                    const int32_t* order, PathStage ps, const float4* pts, const float4* rest) {
  primary_block<kPrimFirst>(s, op, d_image, gr, n_edge, per_thread, order, blockIdx.x, ps, pts, rest);
}
__global__ void __launch_bounds__(kBlock, DRT_PRIMARY_MIN_BLOCKS)
    k_primary_finish(SceneView s, Opts op, const float* d_image, Grads gr, int64_t n_edge, int64_t per_thread,
                     const int32_t* order, PathStage ps, const float4* pts, const float4* rest) {
  primary_block<kPrimFinish>(s, op, d_image, gr, n_edge, per_thread, order, blockIdx.x, ps, pts, rest);
}

__global__ void k_debug_closest(SceneView s, int64_t n, const float* o, const float* d, int32_t* tri, float* tb) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float oo[3] = {o[3 * i], o[3 * i + 1], o[3 * i + 2]}, dd[3] = {d[3 * i], d[3 * i + 1], d[3 * i + 2]};
  Hit h = trace_closest(s, oo, dd, INFINITY, -1);
  tri[i] = h.tri;
  tb[3 * i] = h.tri >= 0 ? h.t : 0.f;
  tb[3 * i + 1] = h.b1;
  tb[3 * i + 2] = h.b2;
}

int group_size(int spp) {
  int G = 1;
  while (G < spp && G < 32) G <<= 1;
  return G;
}

// ---------------------------------------------------------------------------
// Batched scenes: persistent kernels over (scene, virtual block) items.  A
// virtual block is exactly the work of one block of the single-scene launch
// (same pixels or samples, same partial-sum row), so every image and every
// partial row of a batch equals the single-scene result.  CTAs take chunks of
// items from an atomic counter until the items run out (no waiting).
// ---------------------------------------------------------------------------
// Scene of an item: the last k with prefix[k] <= item (prefix[0] = 0; a scene
// without items has prefix[k] == prefix[k+1] and is never returned).
__device__ __forceinline__ int batch_scene_of(const int64_t* prefix, int n, int64_t item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int PH>
struct PhaseMinBlocks {
  // resident CTAs per SM as the single-scene kernels have; the depth > 1
  // path pass needs more registers
  static constexpr int value =
      PH == kPhasePath ? DRT_PATH_MIN_BLOCKS
                       : (PH == kPhasePrimary ? DRT_PRIMARY_MIN_BLOCKS
                                              : (PH == kPhaseRender ? DRT_RENDER_MIN_BLOCKS : DRT_PIXEL_MIN_BLOCKS));
};

template <int PH>
__global__ void __launch_bounds__(kBlock, PhaseMinBlocks<PH>::value)
    k_batch(const BatchScene* bs, const int64_t* prefix, int n, int64_t n_items, int chunk,
            unsigned long long* counter) {
  __shared__ __align__(16) BatchScene sb;
  __shared__ long long s_item;
  int cur = -1;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, (unsigned long long)chunk);
    __syncthreads();
    long long it0 = s_item;
    if (it0 >= n_items) break;
    long long it1 = it0 + chunk < n_items ? it0 + chunk : n_items;
    for (long long it = it0; it < it1; ++it) {
      int sc = batch_scene_of(prefix, n, it);
      if (sc != cur) {  // same value in every thread
        __syncthreads();
        const int* src = reinterpret_cast<const int*>(bs + sc);
        int* dst = reinterpret_cast<int*>(&sb);
        for (int w = threadIdx.x; w < (int)(sizeof(BatchScene) / 4); w += kBlock) dst[w] = src[w];
        __syncthreads();
        cur = sc;
      }
      int64_t blk = it - prefix[sc];
      if (PH == kPhaseRender) {
        render_block(sb.v, sb.op, sb.image, sb.tape_tri, sb.tape_bary, sb.G, blk);
      } else if (PH == kPhaseInterior) {
        interior_block(sb.v, sb.op, sb.tape_tri, sb.tape_bary, sb.d_image, Grads{sb.d_verts, sb.d_albedo, sb.partials},
                       sb.G, sb.dp_sec, sb.do_int, blk);
      } else if (PH == kPhasePath) {
        path_block<false>(sb.v, sb.op, sb.tape_tri, sb.tape_bary, sb.d_image,
                          Grads{sb.d_verts, sb.d_albedo, sb.partials},
                   sb.G, sb.dp_sec, blk);
      } else {
        primary_block(sb.v, sb.op, sb.d_image, Grads{sb.d_verts, sb.d_albedo, sb.partials + sb.rows_i * kGlobals},
                      sb.n_edge, sb.per_thread, sb.order, blk);
      }
    }
  }
}

// Screen keys of the primary edge samples of all scenes, scene index in the
// high bits: one stable sort orders every scene's samples exactly as the
// single-scene sort does (with shift > 0, when the 32-bit key has no room
// for all screen bits, on a coarser grid).  vals = index of the sample
// within its scene.
__global__ void k_batch_keys(const BatchScene* bs, const int64_t* eprefix, int n, int64_t total, int pix_bits,
                             int shift, uint32_t* keys, int32_t* vals) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int sc = batch_scene_of(eprefix, n, g);
  const SceneView& s = bs[sc].v;
  int64_t j = g - eprefix[sc];
  double ptotal = s.pcdf[s.E - 1];
  uint32_t key = 0;
  if (ptotal > 0.0) {
    EdgeSample es = primary_sample(s, bs[sc].op, j, ptotal);
    // position at 1/kKeySub of a pixel
    int px = min(max((int)floorf(es.x * kKeySub), 0), s.W * kKeySub - 1);
    int py = min(max((int)floorf(es.y * kKeySub), 0), s.H * kKeySub - 1);
    key = spread_bits16((uint32_t)px) | (spread_bits16((uint32_t)py) << 1);
  }
  keys[g] = ((uint32_t)sc << pix_bits) | (key >> shift);
  vals[g] = (int32_t)j;
}

template <int PH>
cudaError_t launch_phase(const BatchScene* bs, const int64_t* prefix, int n, int64_t n_items, int grid, int chunk,
                         unsigned long long* counter, cudaStream_t st) {
  k_batch<PH><<<grid, kBlock, 0, st>>>(bs, prefix, n, n_items, chunk, counter);
  return cudaGetLastError();
}

template <int PH>
int phase_occupancy() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<PH>, kBlock, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

}  // namespace

int pixel_group(int spp) { return group_size(spp); }

int64_t pixel_blocks(int W, int H, int spp) {
  int G = group_size(spp);
  int64_t warps = ((int64_t)W * H + (32 / G) - 1) / (32 / G);
  return (warps * 32 + kBlock - 1) / kBlock;
}

void primary_blocks(int64_t n_edge, int64_t* blocks_e, int64_t* per_thread) {
  *blocks_e = std::min<int64_t>((n_edge + kPrimaryPerRound - 1) / kPrimaryPerRound, DRT_PRIMARY_BLOCK_CAP);
  *per_thread = *blocks_e > 0 ? (n_edge + *blocks_e * kPrimaryPerRound - 1) / (*blocks_e * kPrimaryPerRound) : 0;
}

int64_t primary_blocks_for(int64_t n_edge, int64_t per_thread) {
  return (n_edge + kPrimaryPerRound * per_thread - 1) / (kPrimaryPerRound * per_thread);
}

int screen_key_bits(int W, int H) {
  int bits = 2;
  while ((1 << (bits / 2)) < std::max(W, H) * kKeySub) bits += 2;
  return bits;
}

cudaError_t launch_batch_phase(int phase, const BatchScene* bs, const int64_t* prefix, int n, int64_t n_items,
                               int grid, int chunk, unsigned long long* counter, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  static const char* names[kPhases] = {"batch_render", "batch_backward_interior", "batch_backward_secondary_edges",
                                       "batch_backward_path", "batch_backward_primary_edges"};
  ProfToken pt = prof_begin(names[phase], st);
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    switch (phase) {
      case kPhaseRender: e = launch_phase<kPhaseRender>(bs, prefix, n, n_items, grid, chunk, counter, st); break;
      case kPhaseInterior: e = launch_phase<kPhaseInterior>(bs, prefix, n, n_items, grid, chunk, counter, st); break;
      case kPhaseSecondary:  // a batch queues its secondary edge samples (launch_secondary_apart)
        break;
      case kPhasePath: e = launch_phase<kPhasePath>(bs, prefix, n, n_items, grid, chunk, counter, st); break;
      default: e = launch_phase<kPhasePrimary>(bs, prefix, n, n_items, grid, chunk, counter, st); break;
    }
  }
  prof_end(pt, st);
  return e;
}

int batch_phase_occupancy(int phase) {
  switch (phase) {
    case kPhaseRender: return phase_occupancy<kPhaseRender>();
    case kPhaseInterior: return phase_occupancy<kPhaseInterior>();
    case kPhaseSecondary: return 1;
    case kPhasePath: return phase_occupancy<kPhasePath>();
    default: return phase_occupancy<kPhasePrimary>();
  }
}

cudaError_t launch_batch_keys(const BatchScene* bs, const int64_t* eprefix, int n, int64_t total, int pix_bits,
                              int shift, uint32_t* keys, int32_t* vals, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  DRT_PROF_LAUNCH("batch_primary_keys", st,
                  k_batch_keys<<<(unsigned)((total + kBlock - 1) / kBlock), kBlock, 0, st>>>(
                      bs, eprefix, n, total, pix_bits, shift, keys, vals));
  return cudaGetLastError();
}

int64_t partial_floats(int64_t rows) {
  int64_t chunks = (rows + kReduceRows - 1) / kReduceRows;
  return rows * kGlobals + 2 * kGlobals * chunks;  // rows, then FP64 chunk totals
}

cudaError_t launch_reduce_globals(float* partials, int64_t rows, float* d_radiance, float* d_cam, float* d_scale,
                                  cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  int64_t chunks = (rows + kReduceRows - 1) / kReduceRows;
  double* ch = reinterpret_cast<double*>(partials + rows * kGlobals);
  ProfToken pt = prof_begin("reduce_globals", st);
  k_reduce_rows<<<(unsigned)chunks, kBlock, 0, st>>>(partials, rows, ch);
  k_reduce_chunks<<<1, 32 * kGlobals, 0, st>>>(ch, chunks, d_radiance, d_cam, d_scale);
  prof_end(pt, st);
  return cudaGetLastError();
}

cudaError_t launch_render(const drt_scene* sc, const Opts& op, float* image, drt_tape* tape, const RenderScratch* rs,
                          cudaStream_t st) {
  SceneView s = sc->view();
  s.counters = counter_slot(kSlotRender);
  int npix = s.W * s.H;
  int G = group_size(op.spp);
  int64_t warps = ((int64_t)npix + (32 / G) - 1) / (32 / G);
  int64_t blocks = (warps * 32 + kBlock - 1) / kBlock;
  int md = op.primary_only ? 1 : std::min(op.max_depth, kMaxDepth);
  int64_t n = (int64_t)npix * op.spp;
  if (md > 1 && rs && rs->cap >= n && n < (int64_t(1) << 31)) {
    // paths beyond one vertex in stages (k_render_first, k_path_bounce, k_render_finish)
    int32_t* tt = tape ? tape->tri : nullptr;
    float2* tb = tape ? tape->bary : nullptr;
    cudaError_t e = cudaSuccess;
    if (tt) e = cudaMemsetAsync(tt + n, 0xff, sizeof(int32_t) * (size_t)n * (md - 1), st);  // -1: no vertex
    if (e == cudaSuccess) e = cudaMemsetAsync(rs->count, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    PathStage ps{{rs->path[0], rs->path[1]}, rs->count, rs->L};
    DRT_PROF_LAUNCH("render_first", st,
                    k_render_first<<<(unsigned)blocks, kBlock, 0, st>>>(s, op, tt, tb, G, ps));
    BatchScene bs;
    std::memset(&bs, 0, sizeof(bs));
    bs.v = s;
    bs.v.counters = counter_slot(kSlotRenderBounce);
    bs.op = op;
    bs.tape_tri = tt;
    bs.tape_bary = tb;
    int64_t grid_p = std::min<int64_t>((n + kBlock - 1) / kBlock, 152 * 8);
    const PoolScratch& pl = sc->pool;
    bool pooled = pl.cap >= n;
    if (pooled) {
      bs.pool_crec = pl.crec; bs.pool_hits = pl.hits; bs.pool_arec = pl.arec; bs.pool_occ = pl.occ;
      bs.pool_next = pl.next; bs.pool_cap = pl.cap;
    }
    for (int level = 0; level + 1 < md; ++level) {
      int in = level & 1;
      if (pooled) {
        e = launch_bounce_level<kSrcRender>(bs, ps, in, pool_of(bs), grid_p, "render_bounce", st);
        if (e != cudaSuccess) return e;
        continue;
      }
      e = cudaMemsetAsync(rs->count + (in ^ 1), 0, sizeof(unsigned long long), st);
      if (e != cudaSuccess) return e;
      DRT_PROF_LAUNCH("render_bounce", st,
                      k_path_bounce<kSrcRender><<<(unsigned)std::max<int64_t>(grid_p, 1), kBlock, 0, st>>>(
                          bs, ps, in));
    }
    DRT_PROF_LAUNCH("render_finish", st,
                    k_render_finish<<<(unsigned)blocks, kBlock, 0, st>>>(s, op, image, G, rs->L));
    return cudaGetLastError();
  }
  ProfToken pt = prof_begin("render", st);
  k_render<<<(unsigned)blocks, kBlock, 0, st>>>(s, op, image, tape ? tape->tri : nullptr, tape ? tape->bary : nullptr,
                                                G);
  prof_end(pt, st);
  return cudaGetLastError();
}

__global__ void k_axpy(float* out, const float* in, float scale, int64_t n, int first) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v = in[i] * scale;
  out[i] = first ? v : out[i] + v;
}

cudaError_t launch_axpy(float* out, const float* in, float scale, int64_t n, bool first, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_axpy<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, st>>>(out, in, scale, n, first ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_nee_half_width(const float* verts, int V, float* out, cudaStream_t st) {
  DRT_PROF_LAUNCH("nee_half_width", st, k_nee_half_width<<<1, 1024, 0, st>>>(verts, V, out));
  return cudaGetLastError();
}

int64_t secondary_capacity(int W, int H, const Opts& op) {
  int md = op.primary_only ? 1 : std::min(op.max_depth, kMaxDepth);
  return (int64_t)W * H * op.spp * md * (op.nee ? 2 : 1);
}

cudaError_t launch_secondary_apart(const BatchScene& b, cudaStream_t st) {
  int64_t n = (int64_t)b.v.W * b.v.H * b.op.spp;
  if (n <= 0) return cudaSuccess;
  BatchScene q = b;
  q.v.counters = nullptr;
  bool tree = b.op.sec_sampler == 1 && b.sec_pick;
  bool nee = b.op.nee != 0;
  if (nee && !b.sec_nee) return cudaErrorInvalidValue;
  unsigned gq = (unsigned)((n + kBlock - 1) / kBlock);
  if (nee)
    DRT_PROF_LAUNCH("backward_secondary_queue", st, k_sec_queue_nee<<<gq, kBlock, 0, st>>>(q));
  else if (tree)
    DRT_PROF_LAUNCH("backward_secondary_queue", st, k_sec_queue<kSelTree><<<gq, kBlock, 0, st>>>(q));
  else
    DRT_PROF_LAUNCH("backward_secondary_queue", st, k_sec_queue<kSelLength><<<gq, kBlock, 0, st>>>(q));
  BatchScene t = b;
  t.v.counters = counter_slot(kSlotBwdSecondary);
  int64_t grid = std::min<int64_t>((b.sec_cap + kBlock - 1) / kBlock, 152 * 8);
  int md = b.op.primary_only ? 1 : std::min(b.op.max_depth, kMaxDepth);
  bool staged = md > 1 && b.sec_hits && b.sec_lr && b.sec_path[0] && b.sec_path[1] && b.sec_path_count &&
                b.sec_cap < (int64_t(1) << 31);
  if (!staged) {
    if (nee)
      DRT_PROF_LAUNCH("backward_secondary_edges", st, k_sec_trace<kSelNeePre><<<(unsigned)grid, kBlock, 0, st>>>(t));
    else if (tree)
      DRT_PROF_LAUNCH("backward_secondary_edges", st,
                      k_sec_trace<kSelTreePre><<<(unsigned)grid, kBlock, 0, st>>>(t));
    else
      DRT_PROF_LAUNCH("backward_secondary_edges", st, k_sec_trace<kSelLength><<<(unsigned)grid, kBlock, 0, st>>>(t));
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(b.sec_path_count, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  t.v.counters = counter_slot(kSlotBwdSecSides);
  if (nee)
    DRT_PROF_LAUNCH("backward_secondary_sides", st, k_sec_sides<kSelNeePre><<<(unsigned)grid, kBlock, 0, st>>>(t));
  else if (tree)
    DRT_PROF_LAUNCH("backward_secondary_sides", st, k_sec_sides<kSelTreePre><<<(unsigned)grid, kBlock, 0, st>>>(t));
  else
    DRT_PROF_LAUNCH("backward_secondary_sides", st, k_sec_sides<kSelLength><<<(unsigned)grid, kBlock, 0, st>>>(t));
  int64_t grid_p = std::min<int64_t>((b.sec_path_cap + kBlock - 1) / kBlock, 152 * 8);
  t.v.counters = counter_slot(kSlotBwdSecBounce);
  PathStage ps{{b.sec_path[0], b.sec_path[1]}, b.sec_path_count, b.sec_lr};
  bool pooled = b.pool_crec && b.pool_cap >= b.sec_path_cap;
  for (int level = 0; level + 1 < md; ++level) {
    int in = level & 1;
    if (pooled) {
      e = launch_bounce_level<kSrcSecondary>(t, ps, in, pool_of(b), grid_p,
                                             "backward_secondary_bounce", st);
      if (e != cudaSuccess) return e;
      continue;
    }
    e = cudaMemsetAsync(b.sec_path_count + (in ^ 1), 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    DRT_PROF_LAUNCH("backward_secondary_bounce", st,
                    k_path_bounce<kSrcSecondary><<<(unsigned)std::max<int64_t>(grid_p, 1), kBlock, 0, st>>>(
                        t, ps, in));
  }
  BatchScene f = b;
  f.v.counters = nullptr;
  if (nee)
    DRT_PROF_LAUNCH("backward_secondary_finish", st, k_sec_finish<kSelNeePre><<<(unsigned)grid, kBlock, 0, st>>>(f));
  else if (tree)
    DRT_PROF_LAUNCH("backward_secondary_finish", st,
                    k_sec_finish<kSelTreePre><<<(unsigned)grid, kBlock, 0, st>>>(f));
  else
    DRT_PROF_LAUNCH("backward_secondary_finish", st, k_sec_finish<kSelLength><<<(unsigned)grid, kBlock, 0, st>>>(f));
  return cudaGetLastError();
}

int64_t secondary_path_capacity(int W, int H, const Opts& op) {
  int md = op.primary_only ? 1 : std::min(op.max_depth, kMaxDepth);
  return md > 1 ? (int64_t)W * H * op.spp * (md - 1) * (op.nee ? 2 : 1) : 0;
}

cudaError_t launch_backward(const drt_scene* sc, const Opts& op, const drt_tape* tape, const float* d_image,
                            float* d_verts, float* d_albedo, float* d_radiance, float* d_cam, float* d_cam_scale,
                            float* partials, const SortBuffers* sort, const SecScratch* secs, const PrimScratch* prims,
                            cudaStream_t st) {
  SceneView s = sc->view();
  if (op.proposal == 0) s.seg_cdf = nullptr;
  int npix = s.W * s.H;
  int G = group_size(op.spp);
  int64_t warps = ((int64_t)npix + (32 / G) - 1) / (32 / G);
  int64_t blocks_i = (warps * 32 + kBlock - 1) / kBlock;
  int64_t n_edge = (int64_t)op.edge_spp * npix;
  int64_t blocks_e = 0, per_thread = 0;
  if ((op.terms & 2) && s.E > 0 && n_edge > 0) primary_blocks(n_edge, &blocks_e, &per_thread);
  Grads gr{d_verts, d_albedo, partials};
  bool need_i = (op.terms & 5) != 0;
  // The screen keys of the primary edge samples and their sort depend on
  // nothing the other passes compute: they run on the context's side stream,
  // beside the secondary and interior passes, and are joined back before the
  // primary edge kernel.
  const int32_t* order = nullptr;
  const float4* pts = nullptr;   // the samples, kept by the key pass, in screen order
  const float4* rest = nullptr;
  bool forked = false;
  if (blocks_e > 0 && sort && sort->cap >= n_edge) {
    cudaStream_t ss = st;
    drt_context* cx = sc->ctx;
    if (cx && cx->side) {
      if (cudaEventRecord(cx->fork, st) == cudaSuccess && cudaStreamWaitEvent(cx->side, cx->fork, 0) == cudaSuccess) {
        ss = cx->side;
        forked = true;
      } else {
        cudaGetLastError();
      }
    }
    int bits = screen_key_bits(s.W, s.H);
    DRT_PROF_LAUNCH("primary_keys", ss,
                    k_primary_keys<<<(unsigned)((n_edge + kBlock - 1) / kBlock), kBlock, 0, ss>>>(
                        s, op, n_edge, sort->keys, sort->vals, sort->rec));
    bool alt = radix_sort_pairs(sort->keys, sort->vals, sort->keys2, sort->vals2, sort->hist, sort->hist_tmp,
                                (int)n_edge, bits, ss);
    order = alt ? sort->vals2 : sort->vals;
    if (sort->rec && sort->rec_sorted) {
      DRT_PROF_LAUNCH("primary_gather", ss,
                      k_gather_samples<<<(unsigned)((4 * n_edge + kBlock - 1) / kBlock), kBlock, 0, ss>>>(
                          sort->rec, order, n_edge, sort->rec_sorted, sort->rec_sorted + n_edge));
      pts = sort->rec_sorted;
      rest = sort->rec_sorted + n_edge;
    }
    if (forked) cudaEventRecord(cx->join, ss);
  }
  const int32_t* tt = tape ? tape->tri : nullptr;
  const float2* tb = tape ? tape->bary : nullptr;
  bool path = !op.primary_only && op.max_depth > 1;
  bool sec = !op.primary_only && (op.terms & 4) && s.E > 0 && s.L > 0;
  // secondary edge samples traced apart (queued) when scratch is given, else
  // inside the pixel passes
  bool apart = sec && secs != nullptr;
  const float* dps = nullptr;
  if (apart) {
    BatchScene bsd;
    std::memset(&bsd, 0, sizeof(bsd));
    bsd.v = s;
    bsd.op = op;
    bsd.tape_tri = const_cast<int32_t*>(tt);
    bsd.tape_bary = const_cast<float2*>(tb);
    bsd.d_image = d_image;
    bsd.d_verts = d_verts;
    bsd.dp_sec = secs->dp;
    bsd.sec_queue = secs->queue;
    bsd.sec_count = secs->count;
    bsd.sec_pick = op.sec_sampler == 1 ? secs->pick : nullptr;
    bsd.sec_nee = op.nee ? secs->nee : nullptr;
    bsd.sec_cap = secondary_capacity(sc->W, sc->H, op);
    if (secs->wave_cap >= bsd.sec_cap && secs->path_cap >= secondary_path_capacity(sc->W, sc->H, op)) {
      bsd.sec_hits = secs->hits;
      bsd.sec_lr = secs->lr;
      bsd.sec_path[0] = secs->path[0];
      bsd.sec_path[1] = secs->path[1];
      bsd.sec_path_count = secs->path_count;
      bsd.sec_path_cap = secondary_path_capacity(sc->W, sc->H, op);
      const PoolScratch& pl = sc->pool;
      if (pl.cap >= bsd.sec_path_cap) {
        bsd.pool_crec = pl.crec; bsd.pool_hits = pl.hits; bsd.pool_arec = pl.arec; bsd.pool_occ = pl.occ;
        bsd.pool_next = pl.next; bsd.pool_cap = pl.cap;
      }
    }
    cudaError_t e = cudaMemsetAsync(secs->dp, 0, sizeof(float) * 3 * bsd.sec_cap, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(secs->count, 0, sizeof(unsigned long long) * kSecCounters, st);
    if (e == cudaSuccess) e = launch_secondary_apart(bsd, st);
    if (e != cudaSuccess) return e;
    dps = secs->dp;
  }
  if (path && need_i) {
    s.counters = counter_slot(kSlotBwdInterior);
    ProfToken pt = prof_begin("backward_path", st);
    if (apart || !sec)
      k_backward_path<<<(unsigned)blocks_i, kBlock, 0, st>>>(s, op, tt, tb, d_image, gr, G, dps);
    else
      if (op.sec_sampler == 1)
        k_backward_path_in_pass<kSelTree><<<(unsigned)blocks_i, kBlock, 0, st>>>(s, op, tt, tb, d_image, gr, G);
      else
        k_backward_path_in_pass<kSelLength><<<(unsigned)blocks_i, kBlock, 0, st>>>(s, op, tt, tb, d_image, gr, G);
    prof_end(pt, st);
  } else if ((op.terms & 1) || apart) {
    s.counters = counter_slot(kSlotBwdInterior);
    ProfToken pt = prof_begin("backward_interior", st);
    k_backward_interior<<<(unsigned)blocks_i, kBlock, 0, st>>>(s, op, tt, tb, d_image, gr, G, dps, op.terms & 1);
    prof_end(pt, st);
  }
  if (path || apart) {
    // the path or interior pass covered the secondary term
  } else if (sec) {
    s.counters = counter_slot(kSlotBwdSecondary);
    ProfToken pt = prof_begin("backward_secondary_edges", st);
    if (op.sec_sampler == 1)
      k_backward_secondary<kSelTree><<<(unsigned)blocks_i, kBlock, 0, st>>>(s, op, tt, tb, d_image, gr, G,
                                                                             op.terms & 1);
    else
      k_backward_secondary<kSelLength><<<(unsigned)blocks_i, kBlock, 0, st>>>(s, op, tt, tb, d_image, gr, G,
                                                                               op.terms & 1);
    prof_end(pt, st);
  } else if (need_i && !(op.terms & 1)) {
    // secondary requested but nothing to sample: rows still need zeros
    cudaMemsetAsync(partials, 0, sizeof(float) * kGlobals * blocks_i, st);
  }
  Grads ge{d_verts, d_albedo, partials + (need_i ? blocks_i : 0) * kGlobals};
  int md = op.primary_only ? 1 : std::min(op.max_depth, kMaxDepth);
  bool prim_staged = blocks_e > 0 && md > 1 && prims && prims->cap >= n_edge && prims->lr && prims->path[0] &&
                     prims->path[1] && prims->count && n_edge < (int64_t(1) << 31);
  if (blocks_e > 0 && !prim_staged) {
    if (forked) cudaStreamWaitEvent(st, sc->ctx->join, 0);
    s.counters = counter_slot(kSlotBwdPrimary);
    ProfToken pt = prof_begin("backward_primary_edges", st);
    k_backward_primary<<<(unsigned)blocks_e, kBlock, 0, st>>>(s, op, d_image, ge, n_edge, per_thread, order, pts, rest);
    prof_end(pt, st);
  } else if (prim_staged) {
    // beyond one vertex: the first vertex of both side paths (coherent rays in
    // screen order, warp-cooperative traversal), the rest of the paths one
    // vertex per launch, then the edge term from the gathered radiance
    if (forked) cudaStreamWaitEvent(st, sc->ctx->join, 0);
    PathStage ps{{prims->path[0], prims->path[1]}, prims->count, prims->lr};
    cudaError_t e = cudaMemsetAsync(prims->count, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    s.counters = counter_slot(kSlotBwdPrimary);
    DRT_PROF_LAUNCH("backward_primary_first", st,
                    k_primary_first<<<(unsigned)blocks_e, kBlock, 0, st>>>(s, op, d_image, ge, n_edge, per_thread,
                                                                            order, ps, pts, rest));
    BatchScene t;
    std::memset(&t, 0, sizeof(t));
    t.v = s;
    t.v.counters = counter_slot(kSlotBwdPrimBounce);
    t.op = op;
    t.order = order;
    int64_t grid_p = std::min<int64_t>((n_edge + kBlock - 1) / kBlock, 152 * 8);
    const PoolScratch& pl = sc->pool;
    bool pooled = pl.cap >= n_edge;
    if (pooled) {
      t.pool_crec = pl.crec; t.pool_hits = pl.hits; t.pool_arec = pl.arec; t.pool_occ = pl.occ;
      t.pool_next = pl.next; t.pool_cap = pl.cap;
    }
    for (int level = 0; level + 1 < md; ++level) {
      int in = level & 1;
      if (pooled) {
        e = launch_bounce_level<kSrcPrimary>(t, ps, in, pool_of(t), grid_p,
                                             "backward_primary_bounce", st);
        if (e != cudaSuccess) return e;
        continue;
      }
      e = cudaMemsetAsync(prims->count + (in ^ 1), 0, sizeof(unsigned long long), st);
      if (e != cudaSuccess) return e;
      DRT_PROF_LAUNCH("backward_primary_bounce", st,
                      k_path_bounce<kSrcPrimary><<<(unsigned)std::max<int64_t>(grid_p, 1), kBlock, 0, st>>>(
                          t, ps, in));
    }
    s.counters = nullptr;
    DRT_PROF_LAUNCH("backward_primary_finish", st,
                    k_primary_finish<<<(unsigned)blocks_e, kBlock, 0, st>>>(s, op, d_image, ge, n_edge, per_thread,
                                                                             order, ps, pts, rest));
  }
  cudaError_t e = launch_reduce_globals(partials, (need_i ? blocks_i : 0) + blocks_e, d_radiance, d_cam, d_cam_scale,
                                        st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_debug_closest(const drt_scene* sc, int64_t n, const float* o, const float* d, int32_t* tri,
                                 float* tb, cudaStream_t st) {
  SceneView v = sc->view();
  v.counters = counter_slot(kSlotDebug);
  if (n > 0) k_debug_closest<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, st>>>(v, n, o, d, tri, tb);
  return cudaGetLastError();
}

int64_t backward_partial_rows(const drt_scene* sc, const Opts& op) {
  int npix = sc->W * sc->H;
  int G = group_size(op.spp);
  int64_t warps = ((int64_t)npix + (32 / G) - 1) / (32 / G);
  int64_t blocks_i = (warps * 32 + kBlock - 1) / kBlock;
  int64_t n_edge = (int64_t)op.edge_spp * npix;
  int64_t blocks_e = 0, per_thread = 0;
  primary_blocks(n_edge, &blocks_e, &per_thread);
  return blocks_i + blocks_e;
}

}  // namespace drt
