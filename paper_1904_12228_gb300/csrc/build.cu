// build.cu -- everything derived from the scene parameters, rebuilt whenever
// vertices change: the camera inverse, the light-area CDF, the LBVH over the
// triangles (Morton codes, LSD radix sort, Karras hierarchy, bottom-up refit)
// and the edge CDFs for primary (projected, clipped screen length) and
// secondary (3D length) edge sampling.
//
// Sec. 5.3.1 builds its edge hierarchies with this construction (a radix tree
// over sorted Morton codes of box centroids); here it serves the ray-casting
// BVH, which the thesis took from Embree / OptiX Prime, and the secondary
// edge hierarchy (built on demand, edge_tree.cuh).
#include <climits>
#include <cstdio>

#include <cuda_bf16.h>

#include "drt_internal.h"
#include "edge_tree.cuh"

namespace drt {
namespace {

constexpr int kBlock = 256;

// ---------------------------------------------------------------------------
// Validation and small FP64 prep (one thread: exact operation order)
// ---------------------------------------------------------------------------
__global__ void k_check_finite(const float* v, int n, int* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !isfinite(v[i])) raise_flag(err, DRT_DEV_NONFINITE_INPUT, i);
}

// World-to-camera rows: adjugate / determinant of the camera's 3x3 in FP64,
// translation -inv*t, each entry rounded once to FP32.
__global__ void k_world_to_cam(const float* M, float* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double R[3][3], t[3];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) R[i][j] = M[4 * i + j];
    t[i] = M[4 * i + 3];
  }
  double c00 = ds(dm(R[1][1], R[2][2]), dm(R[1][2], R[2][1]));
  double c01 = ds(dm(R[1][2], R[2][0]), dm(R[1][0], R[2][2]));
  double c02 = ds(dm(R[1][0], R[2][1]), dm(R[1][1], R[2][0]));
  double det = da(da(dm(R[0][0], c00), dm(R[0][1], c01)), dm(R[0][2], c02));
  double inv[3][3];
  inv[0][0] = ddv(c00, det);
  inv[0][1] = ddv(ds(dm(R[0][2], R[2][1]), dm(R[0][1], R[2][2])), det);
  inv[0][2] = ddv(ds(dm(R[0][1], R[1][2]), dm(R[0][2], R[1][1])), det);
  inv[1][0] = ddv(c01, det);
  inv[1][1] = ddv(ds(dm(R[0][0], R[2][2]), dm(R[0][2], R[2][0])), det);
  inv[1][2] = ddv(ds(dm(R[0][2], R[1][0]), dm(R[0][0], R[1][2])), det);
  inv[2][0] = ddv(c02, det);
  inv[2][1] = ddv(ds(dm(R[0][1], R[2][0]), dm(R[0][0], R[2][1])), det);
  inv[2][2] = ddv(ds(dm(R[0][0], R[1][1]), dm(R[0][1], R[1][0])), det);
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) out[4 * i + j] = __double2float_rn(inv[i][j]);
    double tt = da(da(dm(inv[i][0], t[0]), dm(inv[i][1], t[1])), dm(inv[i][2], t[2]));
    out[4 * i + 3] = __double2float_rn(-tt);
  }
}

// Light-triangle areas (FP64 from FP32 edge vectors) and their inclusive
// prefix in list order.
__global__ void k_light_cdf(const float* verts, const int32_t* tris, const int32_t* light_tris, int L, double* area,
                            double* cdf, float* box) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double acc = 0.0;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int j = 0; j < L; ++j) {
    int t = light_tris[j];
    const float *a = verts + 3 * tris[3 * t], *b = verts + 3 * tris[3 * t + 1], *c = verts + 3 * tris[3 * t + 2];
    for (int i = 0; i < 3; ++i) {
      lo[i] = fminf(lo[i], fminf(a[i], fminf(b[i], c[i])));
      hi[i] = fmaxf(hi[i], fmaxf(a[i], fmaxf(b[i], c[i])));
    }
    double e1x = fs(b[0], a[0]), e1y = fs(b[1], a[1]), e1z = fs(b[2], a[2]);
    double e2x = fs(c[0], a[0]), e2y = fs(c[1], a[1]), e2z = fs(c[2], a[2]);
    double cx = ds(dm(e1y, e2z), dm(e1z, e2y));
    double cy = ds(dm(e1z, e2x), dm(e1x, e2z));
    double cz = ds(dm(e1x, e2y), dm(e1y, e2x));
    double ar = dm(0.5, __dsqrt_rn(da(da(dm(cx, cx), dm(cy, cy)), dm(cz, cz))));
    area[j] = ar;
    acc = da(acc, ar);
    cdf[j] = acc;
  }
  // padded so the slab test stays conservative w.r.t. the watertight test
  float ext = 0.f;
  for (int i = 0; i < 3; ++i) ext = fmaxf(ext, fmaxf(hi[i] - lo[i], fmaxf(fabsf(lo[i]), fabsf(hi[i]))));
  float pad = 1e-3f * ext + 1e-6f;
  for (int i = 0; i < 3; ++i) {
    box[i] = lo[i] - pad;
    box[3 + i] = hi[i] + pad;
  }
}

// ---------------------------------------------------------------------------
// Edge tables (Sec. 5.2.1 primary, Sec. 5.2.2 secondary)
// ---------------------------------------------------------------------------
__global__ void k_edge_tables(SceneView s, float* pedge, double* plen, double* slen) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= s.E) return;
  int2 ev = s.edges[e];
  const float *a = vtx(s, ev.x), *b = vtx(s, ev.y);
  float ax, ay, bx, by, t0, t1;
  double len = 0.0;
  float row[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (s.cam_type == 2) {
    // fisheye: edges sampled in 3D, by the chord between the unit directions
    // from the camera to their end points (FP64, fixed order)
    double va[3], vb[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double ti = (double)s.cam[4 * i + 3];
      va[i] = ds((double)a[i], ti);
      vb[i] = ds((double)b[i], ti);
    }
    double la = __dsqrt_rn(da(da(dm(va[0], va[0]), dm(va[1], va[1])), dm(va[2], va[2])));
    double lb = __dsqrt_rn(da(da(dm(vb[0], vb[0]), dm(vb[1], vb[1])), dm(vb[2], vb[2])));
    if (la > 0.0 && lb > 0.0) {
      double u[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) u[i] = ds(ddv(va[i], la), ddv(vb[i], lb));
      len = __dsqrt_rn(da(da(dm(u[0], u[0]), dm(u[1], u[1])), dm(u[2], u[2])));
    }
  } else if (project(s, a, &ax, &ay) && project(s, b, &bx, &by) &&
      clip_screen(ax, ay, bx, by, (float)s.W, (float)s.H, &t0, &t1)) {
    row[0] = ax; row[1] = ay; row[2] = bx; row[3] = by; row[4] = t0; row[5] = t1;
    double dx = fs(bx, ax), dy = fs(by, ay);
    len = dm(ds((double)t1, (double)t0), __dsqrt_rn(da(dm(dx, dx), dm(dy, dy))));
  }
  float4* pr = reinterpret_cast<float4*>(pedge + 8 * e);
  pr[0] = make_float4(row[0], row[1], row[2], row[3]);
  pr[1] = make_float4(row[4], row[5], 0.0f, 0.0f);
  plen[e] = len;
  double ex = fs(b[0], a[0]), ey = fs(b[1], a[1]), ez = fs(b[2], a[2]);
  slen[e] = __dsqrt_rn(da(da(dm(ex, ex), dm(ey, ey)), dm(ez, ez)));
}

// ---------------------------------------------------------------------------
// Inclusive FP64 scan: per-block scan, scan of block totals, add.
// ---------------------------------------------------------------------------
constexpr int kScanItems = 4;
constexpr int kScanTile = kBlock * kScanItems;

__device__ double block_excl_scan(double x, double* total) {
  __shared__ double warp_sums[kBlock / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) warp_sums[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double w = lane < kBlock / 32 ? warp_sums[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      double y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kBlock / 32) warp_sums[lane] = w;
  }
  __syncthreads();
  double before = (wid > 0 ? warp_sums[wid - 1] : 0.0) + v - x;
  *total = warp_sums[kBlock / 32 - 1];
  __syncthreads();
  return before;
}

__global__ void k_scan_tiles(const double* in, double* out, double* tile_sums, int n) {
  int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  double v[kScanItems];
  double acc = 0.0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? in[base + i] : 0.0;
    acc += v[i];
    v[i] = acc;
  }
  double total;
  double before = block_excl_scan(acc, &total);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) out[base + i] = before + v[i];
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_sums(double* sums, int nt) {
  __shared__ double carry;
  if (threadIdx.x == 0) carry = 0.0;
  __syncthreads();
  for (int base = 0; base < nt; base += kBlock) {
    int i = base + threadIdx.x;
    double x = i < nt ? sums[i] : 0.0;
    double total;
    double before = block_excl_scan(x, &total);
    if (i < nt) sums[i] = carry + before + x;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
}

__global__ void k_scan_add(double* out, const double* sums, int n) {
  if (blockIdx.x == 0) return;
  double add = sums[blockIdx.x - 1];
  int base = blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += kBlock)
    if (base + i < n) out[base + i] += add;
}

cudaError_t scan_inclusive(const double* in, double* out, double* tmp, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int nt = (n + kScanTile - 1) / kScanTile;
  DRT_PROF_LAUNCH("scan_tiles", st, k_scan_tiles<<<nt, kBlock, 0, st>>>(in, out, tmp, n));
  if (nt > 1) {
    DRT_PROF_LAUNCH("scan_sums", st, k_scan_sums<<<1, kBlock, 0, st>>>(tmp, nt));
    DRT_PROF_LAUNCH("scan_add", st, k_scan_add<<<nt, kBlock, 0, st>>>(out, tmp, n));
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// LBVH: bounds, Morton codes, radix sort, Karras hierarchy, refit
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ord(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float unord(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_bounds_init(int* b) {
  if (threadIdx.x < 3) b[threadIdx.x] = INT_MAX;
  else if (threadIdx.x < 6) b[threadIdx.x] = INT_MIN;
}
__global__ void k_bounds(const float* v, int n, int* b) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int k = 0; k < 3; ++k) {
      lo[k] = fminf(lo[k], v[3 * i + k]);
      hi[k] = fmaxf(hi[k], v[3 * i + k]);
    }
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  }
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 3; ++k) {
      atomicMin(b + k, ord(lo[k]));
      atomicMax(b + 3 + k, ord(hi[k]));
    }
}

__device__ __forceinline__ uint32_t expand10(uint32_t x) {
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

// Key of a triangle: 30-bit Morton code of its centroid in the scene box,
// and above it one bit for triangles whose box is longer than 1/8 of the
// scene's longest extent (floors, walls, large lights).  The hierarchy then
// keeps those few large triangles in their own subtree below the root, so
// their boxes do not enlarge the boxes around the small geometry (a tree of
// Morton order alone places them by centroid, deep among small triangles).
__global__ void k_morton(SceneView s, const int* b, uint32_t* keys, int32_t* vals) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s.T) return;
  const int32_t* id = s.tris + 3 * t;
  float q[3];
  float tri_ext = 0.0f, scene_ext = 0.0f;
  for (int k = 0; k < 3; ++k) {
    float lo = unord(b[k]), hi = unord(b[3 + k]);
    float a = s.verts[3 * id[0] + k], bb = s.verts[3 * id[1] + k], cc = s.verts[3 * id[2] + k];
    float c = (a + bb + cc) * (1.0f / 3.0f);
    float ext = hi - lo;
    float u = ext > 0.0f ? (c - lo) / ext : 0.5f;
    q[k] = fminf(fmaxf(u * 1024.0f, 0.0f), 1023.0f);
    tri_ext = fmaxf(tri_ext, fmaxf(fmaxf(a, bb), cc) - fminf(fminf(a, bb), cc));
    scene_ext = fmaxf(scene_ext, ext);
  }
  uint32_t large = 8.0f * tri_ext > scene_ext ? 1u : 0u;
  keys[t] = (large << 30) | (expand10((uint32_t)q[0]) << 2) | (expand10((uint32_t)q[1]) << 1) | expand10((uint32_t)q[2]);
  vals[t] = t;
}

// One 8-bit LSD pass.  Tiles of kSortTile keys; per-tile digit histograms
// (digit-major), a global exclusive scan, then a stable scatter in which each
// warp ranks its 32 keys with __match_any_sync.
constexpr int kSortItems = 8;
constexpr int kSortTile = kBlock * kSortItems;

__global__ void k_sort_hist(const uint32_t* keys, int n, int shift, uint32_t* hist, int nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int base = blockIdx.x * kSortTile;
  for (int i = threadIdx.x; i < kSortTile; i += kBlock)
    if (base + i < n) atomicAdd(&h[(keys[base + i] >> shift) & 0xffu], 1u);
  __syncthreads();
  hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of the digit histograms (digit-major, tile-minor): tiles of
// kScanTile entries, a scan of the tile totals, then the carry-in.
__device__ uint32_t block_excl_scan_u32(uint32_t x, uint32_t* total) {
  __shared__ uint32_t warp_sums[kBlock / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) warp_sums[wid] = v;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < kBlock / 32 ? warp_sums[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kBlock / 32) warp_sums[lane] = w;
  }
  __syncthreads();
  uint32_t before = (wid > 0 ? warp_sums[wid - 1] : 0u) + v - x;
  *total = warp_sums[kBlock / 32 - 1];
  __syncthreads();
  return before;
}

__global__ void k_hist_scan_tiles(uint32_t* h, uint32_t* tile_sums, int m) {
  int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    uint32_t x = base + i < m ? h[base + i] : 0u;
    v[i] = acc;  // exclusive within the thread
    acc += x;
  }
  uint32_t total;
  uint32_t before = block_excl_scan_u32(acc, &total);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < m) h[base + i] = before + v[i];
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_hist_scan_sums(uint32_t* sums, int nt) {
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  for (int base = 0; base < nt; base += kBlock) {
    int i = base + threadIdx.x;
    uint32_t x = i < nt ? sums[i] : 0u;
    uint32_t total;
    uint32_t before = block_excl_scan_u32(x, &total);
    if (i < nt) sums[i] = carry + before;  // exclusive
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
}

__global__ void k_hist_scan_add(uint32_t* h, const uint32_t* sums, int m) {
  uint32_t add = sums[blockIdx.x];
  if (add == 0u) return;
  int base = blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += kBlock)
    if (base + i < m) h[base + i] += add;
}

__global__ void k_sort_scatter(const uint32_t* keys, const int32_t* vals, uint32_t* okeys, int32_t* ovals, int n,
                               int shift, const uint32_t* hist, int nblocks) {
  __shared__ uint32_t run[256];
  __shared__ uint32_t wcnt[kBlock / 32][256];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  run[threadIdx.x] = hist[threadIdx.x * nblocks + blockIdx.x];
  int base = blockIdx.x * kSortTile;
  for (int r = 0; r < kSortItems; ++r) {
    for (int k = 0; k < kBlock / 32; ++k) wcnt[k][threadIdx.x] = 0;
    __syncthreads();
    int i = base + r * kBlock + threadIdx.x;
    bool valid = i < n;
    uint32_t key = valid ? keys[i] : 0u;
    int32_t val = valid ? vals[i] : 0;
    uint32_t dig = valid ? (key >> shift) & 0xffu : 256u + lane;  // invalid lanes never match valid ones
    uint32_t peers = __match_any_sync(0xffffffffu, dig);
    uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[wid][dig] = __popc(peers);
    __syncthreads();
    // exclusive prefix over warps per digit; thread == digit
    uint32_t acc = 0;
    for (int k = 0; k < kBlock / 32; ++k) {
      uint32_t c = wcnt[k][threadIdx.x];
      wcnt[k][threadIdx.x] = acc;
      acc += c;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = run[dig] + wcnt[wid][dig] + rank;
      okeys[pos] = key;
      ovals[pos] = val;
    }
    __syncthreads();
    run[threadIdx.x] += acc;
    __syncthreads();
  }
}

__device__ __forceinline__ int delta(const uint32_t* k, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  uint32_t a = k[i], b = k[j];
  if (a == b) return 32 + __clz((uint32_t)(i ^ j));
  return __clz(a ^ b);
}

// Karras (HPG 2012): internal node i covers a key range; its split is the
// highest differing bit; children are leaves when the range has one key.
__global__ void k_karras(const uint32_t* keys, int n, int leaf_max, float4* nodes, int2* child_orig,
                         int32_t* parent, int32_t* leaf_parent) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = delta(keys, n, i, i - d);
  int lmax = 2;
  while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
  int j = i + l * d;
  int dnode = delta(keys, n, i, j);
  int s = 0;
  int len = l;
  for (int t = (len + 1) >> 1;; t = (t + 1) >> 1) {
    if (s + t < len + 1 && delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    if (t == 1) break;
  }
  int gamma = i + s * d + min(d, 0);
  int lo = min(i, j), hi = max(i, j);
  int left = (lo == gamma) ? ~gamma : gamma;
  int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
  // traversal sees a subtree of at most leaf_max triangles as one leaf range
  int lcount = gamma - lo + 1, rcount = hi - gamma;
  int left_enc = lcount <= leaf_max ? leaf_enc(lo, lcount) : left;
  int right_enc = rcount <= leaf_max ? leaf_enc(gamma + 1, rcount) : right;
  if (nodes) reinterpret_cast<int4*>(nodes)[4 * i + 3] = make_int4(left_enc, right_enc, 0, 0);
  child_orig[i] = make_int2(left, right);
  if (left < 0) leaf_parent[~left] = i; else parent[left] = i;
  if (right < 0) leaf_parent[~right] = i; else parent[right] = i;
  if (i == 0) parent[0] = -1;
}

// Triangle soup in leaf order and bottom-up refit with arrival counters.
__global__ void k_refit(SceneView s, const int32_t* vals, float4* nodes, float4* soup, const int2* child_orig,
                        const int32_t* parent, const int32_t* leaf_parent, int32_t* flags, int32_t* tsize) {
  int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= s.T) return;
  int t = vals[pos];
  const int32_t* id = s.tris + 3 * t;
  float3 v[3];
  for (int k = 0; k < 3; ++k) v[k] = ld3(s.verts + 3 * id[k]);
  soup[3 * pos + 0] = make_float4(v[0].x, v[0].y, v[0].z, __int_as_float(t));
  soup[3 * pos + 1] = make_float4(v[1].x, v[1].y, v[1].z, 0.0f);
  soup[3 * pos + 2] = make_float4(v[2].x, v[2].y, v[2].z, 0.0f);
  float lo[3], hi[3];
  float mag = 0.0f;
  for (int k = 0; k < 3; ++k) {
    float a = comp(v[0], k), b = comp(v[1], k), c = comp(v[2], k);
    lo[k] = fminf(a, fminf(b, c));
    hi[k] = fmaxf(a, fmaxf(b, c));
    mag = fmaxf(mag, fmaxf(fabsf(lo[k]), fabsf(hi[k])));
  }
  // enlarge so the FP32 slab test is conservative w.r.t. the watertight test
  float pad = mag * 3.0517578125e-05f + 1e-30f;
  for (int k = 0; k < 3; ++k) { lo[k] -= pad; hi[k] += pad; }
  if (s.T == 1) return;
  int child = ~pos;
  int node = leaf_parent[pos];
  int climb = 0;
  int size = 1;  // triangles below `child`
  while (node >= 0) {
    if (++climb > s.T) {  // deeper than the tree can be: parent links are broken
      raise_flag(s.err, DRT_DEV_REFIT_CAP, pos);
      return;
    }
    float4* n4 = nodes + 4 * node;
    bool is_left = child_orig[node].x == child;
    // write this child's box into its slot of the parent
    float* f = reinterpret_cast<float*>(n4);
    if (is_left) {
      f[0] = lo[0]; f[1] = lo[1]; f[2] = lo[2]; f[3] = hi[0]; f[4] = hi[1]; f[5] = hi[2];
    } else {
      f[6] = lo[0]; f[7] = lo[1]; f[8] = lo[2]; f[9] = hi[0]; f[10] = hi[1]; f[11] = hi[2];
    }
    __threadfence();
    // the first to arrive leaves its triangle count; the sibling finishes
    // this node with the sum
    int other = atomicAdd(flags + node, size);
    if (other == 0) return;
    __threadfence();
    size += other;
    tsize[node] = size;
    const float* o = reinterpret_cast<const float*>(n4) + (is_left ? 6 : 0);
    for (int k = 0; k < 3; ++k) {
      lo[k] = fminf(lo[k], __ldcg(o + k));
      hi[k] = fmaxf(hi[k], __ldcg(o + 3 + k));
    }
    child = node;
    node = parent[node];
  }
}

// Treelet restructuring of the refitted hierarchy (Karras and Aila, "Fast
// parallel construction of high-quality bounding volume hierarchies", HPG
// 2013).  A Morton-order hierarchy splits space, not cost: its nodes often
// have boxes much larger than a surface-area-guided split would give, and
// every ray that enters them pays for it.  Bottom-up, each node whose subtree
// holds at least `gamma` triangles takes a treelet: its two children, then
// repeatedly the treelet leaf with the largest box replaced by its two
// children, up to kTreeletLeaves leaves.  Over every subset of those leaves
// a dynamic program finds the binary topology with the least total surface
// area of internal nodes (the surface-area cost of the treelet, whose leaves
// keep their subtrees), and the treelet's internal nodes are rewritten with
// it.  Leaves, leaf ranges and every box of a leaf are unchanged, so the
// hierarchy holds the same triangles in the same boxes and every traversal
// finds the same hits; only the internal topology and its unions change.
// A pass starts one warp at every node it processes whose children it does
// not (subtree triangle counts from the refit, kept up to date by the
// rewrites); a warp climbs the parent links and processes each node once
// every child of it that the pass processes is done (the second of two to
// arrive goes on).  A treelet rewrites only its root and nodes below it, so
// a node keeps its children until it is processed, the set of nodes below
// it never changes, and the rewrites keep the links of the new topology for
// the next pass.
constexpr int kTreeletLeaves = 7;
// Passes over the hierarchy, the k-th on subtrees of 7 * 2^k triangles or
// more (of 1, 2 and 3 passes, 2 gave the fastest 200k-triangle depth-3 step;
// hierarchies with leaf ranges take one).
#ifndef DRT_TREELET_ROUNDS
#define DRT_TREELET_ROUNDS 2
#endif

__device__ __forceinline__ float box_area(const float b[6]) {
  float dx = fmaxf(b[3] - b[0], 0.0f), dy = fmaxf(b[4] - b[1], 0.0f), dz = fmaxf(b[5] - b[2], 0.0f);
  return dx * dy + dy * dz + dz * dx;
}

// child slot k (0 left, 1 right) of node n: box and encoding (L2 reads: other
// threads wrote the nodes below)
__device__ __forceinline__ void node_child(const float4* nodes, int n, int k, float b[6], int* enc) {
  const float* f = reinterpret_cast<const float*>(nodes + 4 * (size_t)n);
  for (int i = 0; i < 6; ++i) b[i] = __ldcg(f + 6 * k + i);
  int2 ch = __ldcg(reinterpret_cast<const int2*>(f + 12));
  *enc = k == 0 ? ch.x : ch.y;
}

// One treelet, by the 32 lanes of a warp together: every lane forms the
// same treelet (reads only); the subsets' areas, then their best splits, one
// size at a time, are spread over the lanes (cost, area and split in the
// warp's shared arrays); lane 0 rewrites the nodes.
// Triangles below a child reference: a leaf range's count, or the node's.
__device__ __forceinline__ int child_size(const int32_t* tsize, int enc) {
  return enc < 0 ? (((~enc) >> 28) + 1) : __ldcg(tsize + enc);
}

__device__ void restructure_treelet(float4* nodes, int32_t* parent, int32_t* tsize, int root, float* cost,
                                    float* area, unsigned char* split, int lane) {
  float lb[kTreeletLeaves][6];
  int le[kTreeletLeaves];
  int inner[kTreeletLeaves - 1];
  int nl = 2, ni = 1;
  inner[0] = root;
  node_child(nodes, root, 0, lb[0], &le[0]);
  node_child(nodes, root, 1, lb[1], &le[1]);
  while (nl < kTreeletLeaves) {
    int best = -1;
    float best_a = -1.0f;
    for (int i = 0; i < nl; ++i) {
      if (le[i] < 0) continue;  // a leaf range stays a leaf
      float a = box_area(lb[i]);
      if (a > best_a) { best_a = a; best = i; }
    }
    if (best < 0) break;
    int e = le[best];
    inner[ni++] = e;
    node_child(nodes, e, 0, lb[best], &le[best]);
    node_child(nodes, e, 1, lb[nl], &le[nl]);
    ++nl;
  }
  if (nl < 3) return;  // two leaves: one topology
  int lsz[kTreeletLeaves];
  for (int i = 0; i < nl; ++i) lsz[i] = child_size(tsize, le[i]);
  const int full = (1 << nl) - 1;
  for (int m = lane + 1; m <= full; m += 32) {
    cost[m] = 0.0f;  // one leaf: its subtree is fixed
    float b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < nl; ++i)
      if ((m >> i) & 1)
        for (int k = 0; k < 3; ++k) {
          b[k] = fminf(b[k], lb[i][k]);
          b[3 + k] = fmaxf(b[3 + k], lb[i][3 + k]);
        }
    area[m] = box_area(b);
  }
  __syncwarp();
  for (int size = 2; size <= nl; ++size) {
    for (int m = lane + 1; m <= full; m += 32) {
      if (__popc(m) != size) continue;
      // the two parts: p holds m's lowest leaf, q the rest (both non-empty)
      int low = m & -m, rest = m ^ low;
      float bc = INFINITY;
      int bp = low;
      for (int q = (rest - 1) & rest;; q = (q - 1) & rest) {
        int p = low | q;
        float c = cost[p] + cost[m ^ p];
        if (c < bc) { bc = c; bp = p; }
        if (q == 0) break;
      }
      cost[m] = area[m] + bc;
      split[m] = (unsigned char)bp;
    }
    __syncwarp();
  }
  if (lane == 0) {
    // the full set at the treelet root, each further set of two or more
    // leaves at the next internal node of the treelet
    int st_m[kTreeletLeaves], st_n[kTreeletLeaves];
    int sp = 0, next = 1;
    st_m[sp] = full;
    st_n[sp++] = root;
    while (sp > 0) {
      --sp;
      int m = st_m[sp], n = st_n[sp];
      int part[2] = {split[m], m ^ split[m]};
      float* f = reinterpret_cast<float*>(nodes + 4 * (size_t)n);
      int enc[2];
      for (int k = 0; k < 2; ++k) {
        int pm = part[k];
        float b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
        for (int i = 0; i < nl; ++i)
          if ((pm >> i) & 1)
            for (int j = 0; j < 3; ++j) {
              b[j] = fminf(b[j], lb[i][j]);
              b[3 + j] = fmaxf(b[3 + j], lb[i][3 + j]);
            }
        if ((pm & (pm - 1)) == 0) {
          enc[k] = le[__ffs(pm) - 1];
        } else {
          enc[k] = inner[next++];
          st_m[sp] = pm;
          st_n[sp++] = enc[k];
        }
        for (int i = 0; i < 6; ++i) f[6 * k + i] = b[i];
        // links and triangle counts of the new topology (for the climb and
        // a further pass)
        if (enc[k] >= 0) {
          parent[enc[k]] = n;
          int sz = 0;
          for (int i = 0; i < nl; ++i)
            if ((pm >> i) & 1) sz += lsz[i];
          tsize[enc[k]] = sz;
        }
      }
      reinterpret_cast<int4*>(f)[3] = make_int4(enc[0], enc[1], 0, 0);
    }
  }
  __syncwarp();
}

// One warp per binary internal node; lane 0 takes the arrival counters.
constexpr int kTreeletWarps = 4;
__global__ void __launch_bounds__(32 * kTreeletWarps) k_treelets(int T, int leaf_max, int gamma, float4* nodes,
                                                                 int32_t* parent, int32_t* tsize, int32_t* flags,
                                                                 int32_t* err) {
  __shared__ float s_cost[kTreeletWarps][1 << kTreeletLeaves];
  __shared__ float s_area[kTreeletWarps][1 << kTreeletLeaves];
  __shared__ unsigned char s_split[kTreeletWarps][1 << kTreeletLeaves];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int node = blockIdx.x * kTreeletWarps + w;
  if (node >= T - 1) return;  // uniform across the warp
  // a node the pass processes: a subtree of at least gamma triangles that is
  // not inside a leaf range (those are never traversed)
  auto takes = [&](int enc) { return enc >= 0 && child_size(tsize, enc) > leaf_max && child_size(tsize, enc) >= gamma; };
  if (!takes(node)) return;
  int2 ch = __ldcg(reinterpret_cast<const int2*>(nodes + 4 * (size_t)node + 3));
  if (takes(ch.x) || takes(ch.y)) return;  // a warp from below gets here
  int climb = 0;
  while (true) {
    if (++climb > T) {
      if (lane == 0 && err) raise_flag(err, DRT_DEV_REFIT_CAP, node);
      return;
    }
    restructure_treelet(nodes, parent, tsize, node, s_cost[w], s_area[w], s_split[w], lane);
    int p = __ldcg(parent + node);
    if (p < 0) return;
    int2 pc = __ldcg(reinterpret_cast<const int2*>(nodes + 4 * (size_t)p + 3));
    if (takes(pc.x) && takes(pc.y)) {  // two warps arrive: the second goes on
      int other = 0;
      if (lane == 0) {
        __threadfence();
        other = atomicAdd(flags + p, 1);
      }
      other = __shfl_sync(0xffffffffu, other, 0);
      if (other == 0) return;
      __threadfence();
    }
    node = p;
  }
}

// Tile segments of primary edge e (same crossing arithmetic as the oracle):
// calls emit(s0, s1) for each piece in increasing t.
template <class F>
__device__ __forceinline__ int for_each_segment(const SceneView& s, int e, F emit) {
  const float4* row = reinterpret_cast<const float4*>(s.pedge + 8 * e);
  float4 r0 = row[0], r1 = row[1];
  float ax = r0.x, ay = r0.y, t0 = r1.x, t1 = r1.y;
  float dx = fs(r0.z, ax), dy = fs(r0.w, ay);
  // crossing sequences along x and y, each monotone in t
  int mlo[2], mhi[2], dir[2];
  float av[2] = {ax, ay}, dv[2] = {dx, dy};
  for (int a = 0; a < 2; ++a) {
    mlo[a] = 1;
    mhi[a] = 0;
    dir[a] = 1;
    if (dv[a] == 0.0f) continue;
    float c0 = fa(av[a], fm(t0, dv[a])), c1 = fa(av[a], fm(t1, dv[a]));
    float lo = fminf(c0, c1), hi = fmaxf(c0, c1);
    mlo[a] = (int)floorf(fdv(lo, kTile)) + 1;
    mhi[a] = (int)floorf(fdv(hi, kTile));
    dir[a] = dv[a] > 0.0f ? 1 : -1;
  }
  int i[2] = {0, 0};
  int cnt[2] = {mhi[0] - mlo[0] + 1, mhi[1] - mlo[1] + 1};
  auto cross = [&](int a, int k) {
    int m = dir[a] > 0 ? mlo[a] + k : mhi[a] - k;
    return fdv(fs(fm((float)m, kTile), av[a]), dv[a]);
  };
  float last = t0;
  int nseg = 0;
  while (true) {
    // next valid crossing of each sequence
    float v[2];
    for (int a = 0; a < 2; ++a) {
      v[a] = INFINITY;
      while (i[a] < cnt[a]) {
        float t = cross(a, i[a]);
        if (t > t0 && t < t1) { v[a] = t; break; }
        ++i[a];
      }
    }
    float nv;
    if (v[0] == INFINITY && v[1] == INFINITY) break;
    if (v[1] == INFINITY || (v[0] != INFINITY && v[0] <= v[1])) { nv = v[0]; ++i[0]; } else { nv = v[1]; ++i[1]; }
    if (nv > last) {
      emit(nseg++, last, nv);
      last = nv;
    }
  }
  if (t1 > last) emit(nseg++, last, t1);
  return nseg;
}

__global__ void k_segment_count(SceneView s, const double* plen, uint32_t* counts) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= s.E) return;
  uint32_t n = 0;
  if (plen[e] > 0.0) n = (uint32_t)for_each_segment(s, e, [](int, float, float) {});
  counts[e] = n;
}

__global__ void k_segment_fill(SceneView s, const double* plen, const uint32_t* offsets, int32_t* seg_edge,
                               int32_t* seg_tile, float2* seg_s, double* seg_len) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= s.E || !(plen[e] > 0.0)) return;
  const float4* row = reinterpret_cast<const float4*>(s.pedge + 8 * e);
  float4 r0 = row[0];
  float ax = r0.x, ay = r0.y;
  float dx = fs(r0.z, ax), dy = fs(r0.w, ay);
  double dl = __dsqrt_rn(da(dm((double)dx, (double)dx), dm((double)dy, (double)dy)));
  int tiles_x = (int)ceilf((float)s.W / kTile), tiles_y = (int)ceilf((float)s.H / kTile);
  uint32_t base = offsets[e];
  for_each_segment(s, e, [&](int k, float s0, float s1) {
    float mid = fa(s0, fm(0.5f, fs(s1, s0)));
    float xm = fa(ax, fm(mid, dx)), ym = fa(ay, fm(mid, dy));
    int tx = min(max((int)floorf(fdv(xm, kTile)), 0), tiles_x - 1);
    int ty = min(max((int)floorf(fdv(ym, kTile)), 0), tiles_y - 1);
    seg_edge[base + k] = e;
    seg_tile[base + k] = ty * tiles_x + tx;
    seg_s[base + k] = make_float2(s0, s1);
    seg_len[base + k] = dm(ds((double)s1, (double)s0), dl);
  });
}

// Segment weights m_k of the mixture: max(0, w_k) (mode 1), or from network
// scores s_k, a log density per unit length: len_k exp(clamp(s_k, -40, 40))
// (mode 2), in FP64.
__global__ void k_weights_to_f64(const float* w, const double* len, int n, int mode, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = mode == 2 ? dm(len[i], exp(fmin(fmax((double)w[i], -40.0), 40.0))) : (double)fmaxf(0.0f, w[i]);
}

// q = 1/2 len/L + 1/2 m/M (q = len/L if M == 0), from inclusive prefixes of
// len and m (their last entries are L and M).
__global__ void k_proposal_q(const double* len, const double* len_cdf, const double* m, const double* m_cdf, int n,
                             double* q) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double L = len_cdf[n - 1], M = m_cdf[n - 1];
  double ql = ddv(len[i], L);
  q[i] = M > 0.0 ? da(dm(0.5, ql), dm(0.5, ddv(m[i], M))) : ql;
}

// Mean of |w_r|+|w_g|+|w_b| over each screen tile; the last entry receives
// the mean over tiles.
__global__ void k_tile_weights(const float* w, int W, int H, int tx, int ty, float* tile_w) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int nt = tx * ty;
  if (t < nt) {
    int x0 = (t % tx) * 16, y0 = (t / tx) * 16;
    float acc = 0.f;
    int n = 0;
    for (int y = y0; y < min(y0 + 16, H); ++y)
      for (int x = x0; x < min(x0 + 16, W); ++x, ++n) {
        const float* p = w + 3 * ((size_t)y * W + x);
        acc += fabsf(p[0]) + fabsf(p[1]) + fabsf(p[2]);
      }
    tile_w[t] = n > 0 ? acc / n : 0.f;
  }
}
__global__ void k_tile_weight_mean(float* tile_w, int nt) {
  __shared__ float sm[kBlock];
  float acc = 0.f;
  for (int i = threadIdx.x; i < nt; i += kBlock) acc += tile_w[i];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kBlock / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) tile_w[nt] = sm[0] / nt;
}

// 32 features per tile segment, stored as BF16 (zero-padded to 32).
__device__ __forceinline__ float3 pixel_at(const float* img, int W, int H, float x, float y) {
  int px = min(max((int)floorf(x), 0), W - 1), py = min(max((int)floorf(y), 0), H - 1);
  const float* p = img + 3 * ((size_t)py * W + px);
  return make_float3(p[0], p[1], p[2]);
}

__global__ void k_segment_features(SceneView s, const int32_t* seg_edge, const int32_t* seg_tile, const float2* seg_s,
                                   const double* seg_len, int n, const int2* edge_faces, const float* tile_w,
                                   const float* d_image, const float* image, __nv_bfloat16* x) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int e = seg_edge[k], tile = seg_tile[k];
  float2 ss = seg_s[k];
  const float4* row = reinterpret_cast<const float4*>(s.pedge + 8 * e);
  float4 r0 = row[0];
  float ax = r0.x, ay = r0.y, dx = r0.z - r0.x, dy = r0.w - r0.y;
  float W = (float)s.W, H = (float)s.H;
  int tx = (s.W + 15) / 16, ntiles = tx * ((s.H + 15) / 16);
  float f[32];
  for (int i = 0; i < 32; ++i) f[i] = 0.f;
  f[0] = ((tile % tx) + 0.5f) * 16.f / W;
  f[1] = ((tile / tx) + 0.5f) * 16.f / H;
  f[2] = (ax + ss.x * dx) / W;
  f[3] = (ay + ss.x * dy) / H;
  f[4] = (ax + ss.y * dx) / W;
  f[5] = (ay + ss.y * dy) / H;
  f[6] = (float)seg_len[k] / 16.f;
  float el = sqrtf(dx * dx + dy * dy);
  f[7] = el / fmaxf(W, H);
  int2 ev = s.edges[e];
  float3 v0 = ld3(s.verts + 3 * ev.x), v1 = ld3(s.verts + 3 * ev.y);
  float3 mid = make_float3(0.5f * (v0.x + v1.x), 0.5f * (v0.y + v1.y), 0.5f * (v0.z + v1.z));
  float3 cpos = make_float3(s.cam[3], s.cam[7], s.cam[11]);
  float3 view = make_float3(cpos.x - mid.x, cpos.y - mid.y, cpos.z - mid.z);
  int2 fc = edge_faces[e];
  float side[2] = {0.f, 0.f};
  for (int q = 0; q < 2; ++q) {
    int t = q == 0 ? fc.x : fc.y;
    if (t < 0) continue;
    const int32_t* id = s.tris + 3 * t;
    float3 a = ld3(s.verts + 3 * id[0]), b = ld3(s.verts + 3 * id[1]), c = ld3(s.verts + 3 * id[2]);
    float3 e1 = make_float3(b.x - a.x, b.y - a.y, b.z - a.z), e2 = make_float3(c.x - a.x, c.y - a.y, c.z - a.z);
    float3 nn = make_float3(e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x);
    float inv = rsqrtf(fmaxf(nn.x * nn.x + nn.y * nn.y + nn.z * nn.z, 1e-30f));
    nn = make_float3(nn.x * inv, nn.y * inv, nn.z * inv);
    for (int i = 0; i < 3; ++i)
      f[8 + 3 * q + i] = s.w2c[4 * i] * nn.x + s.w2c[4 * i + 1] * nn.y + s.w2c[4 * i + 2] * nn.z;
    side[q] = nn.x * view.x + nn.y * view.y + nn.z * view.z;
    if (s.light_of_tri[t] >= 0) f[19] = 1.f;
  }
  f[14] = (fc.y >= 0 && side[0] * side[1] < 0.f) ? 1.f : 0.f;
  f[15] = fc.y < 0 ? 1.f : 0.f;
  if (fc.x >= 0) {
    int t1 = fc.y >= 0 ? fc.y : fc.x;
    for (int i = 0; i < 3; ++i) f[16 + i] = fabsf(s.albedo[3 * fc.x + i] - (fc.y >= 0 ? s.albedo[3 * t1 + i] : 0.f));
  }
  float zc = s.w2c[8] * mid.x + s.w2c[9] * mid.y + s.w2c[10] * mid.z + s.w2c[11];
  f[20] = 1.f / fmaxf(-zc, 1e-3f);
  float wm = tile_w[ntiles];
  f[21] = wm > 0.f ? tile_w[tile] / wm : 0.f;
  f[22] = el > 0.f ? dx / el : 0.f;
  f[23] = el > 0.f ? dy / el : 0.f;
  // Visibility probes at the segment midpoint: a camera ray through it and
  // one half a pixel to each side of the edge.
  {
    float mid = 0.5f * (ss.x + ss.y);
    float xm = ax + mid * dx, ym = ay + mid * dy;
    float nx = el > 0.f ? -dy / el : 0.f, ny = el > 0.f ? dx / el : 0.f;
    float o[3], d[3];
    camera_ray(s, xm, ym, o, d);
    Hit hc = trace_closest(s, o, d, INFINITY, -1);
    // ray parameter of the closest approach to the edge's line
    float e3[3] = {v1.x - v0.x, v1.y - v0.y, v1.z - v0.z}, w0[3] = {o[0] - v0.x, o[1] - v0.y, o[2] - v0.z};
    float A = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], B = d[0] * e3[0] + d[1] * e3[1] + d[2] * e3[2];
    float C = e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2];
    float D = d[0] * w0[0] + d[1] * w0[1] + d[2] * w0[2], E = e3[0] * w0[0] + e3[1] * w0[1] + e3[2] * w0[2];
    float den = A * C - B * B;
    float te = den > 0.f ? (B * E - C * D) / den : 0.f;
    bool vis = hc.tri < 0 || hc.tri == fc.x || hc.tri == fc.y || hc.t >= te * (1.f - 1e-3f);
    f[24] = vis ? 1.f : 0.f;
    int side_tri[2];
    for (int q = 0; q < 2; ++q) {
      float sgn = q == 0 ? 0.5f : -0.5f;
      camera_ray(s, xm + sgn * nx, ym + sgn * ny, o, d);
      side_tri[q] = trace_closest(s, o, d, INFINITY, -1).tri;
    }
    f[25] = side_tri[0] != side_tri[1] ? 1.f : 0.f;
    f[26] = (side_tri[0] < 0) != (side_tri[1] < 0) ? 1.f : 0.f;
    float lum[2];
    for (int q = 0; q < 2; ++q) {
      int t = side_tri[q];
      lum[q] = t < 0 ? 0.f : (s.albedo[3 * t] + s.albedo[3 * t + 1] + s.albedo[3 * t + 2]) * (1.f / 3.f);
      if (t >= 0 && s.light_of_tri[t] >= 0) f[28] = 1.f;
    }
    f[27] = fabsf(lum[0] - lum[1]);
    // loss adjoint along the segment, over its image mean
    float wsum = 0.f;
    for (int q = 0; q < 4; ++q) {
      float u = ss.x + (ss.y - ss.x) * (0.125f + 0.25f * q);
      float3 wv = pixel_at(d_image, s.W, s.H, ax + u * dx, ay + u * dy);
      wsum += fabsf(wv.x) + fabsf(wv.y) + fabsf(wv.z);
    }
    f[29] = wm > 0.f ? 0.25f * wsum / wm : 0.f;
    // radiance contrast across the edge in the rendered image
    if (image) {
      float3 iu = pixel_at(image, s.W, s.H, xm + 1.5f * nx, ym + 1.5f * ny);
      float3 il = pixel_at(image, s.W, s.H, xm - 1.5f * nx, ym - 1.5f * ny);
      float dif = fabsf(iu.x - il.x) + fabsf(iu.y - il.y) + fabsf(iu.z - il.z);
      float sum = fabsf(iu.x) + fabsf(iu.y) + fabsf(iu.z) + fabsf(il.x) + fabsf(il.y) + fabsf(il.z);
      f[30] = dif / (sum + 1e-6f);
      f[31] = log1pf(dif);
    }
  }
  for (int i = 0; i < 32; ++i) x[(size_t)k * 32 + i] = __float2bfloat16_rn(f[i]);
}

// ---------------------------------------------------------------------------
// Secondary edge hierarchy (Sec. 5.3.1; layouts and arithmetic in edge_tree.cuh)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void et_frame_of_scene(const SceneView& s, const int* b, float O[3], float blo[3],
                                                  float bhi[3], float* R) {
  for (int k = 0; k < 3; ++k) {
    O[k] = s.cam[4 * k + 3];
    blo[k] = unord(b[k]);
    bhi[k] = unord(b[3 + k]);
  }
  *R = et_hough_radius(blo, bhi, O);
}

// One thread per edge: its key (class bit over the Morton code) and id.
// Sphere around all light triangles (the light-cone bound of the hierarchy).
__global__ void k_etree_light(const float* verts, const int32_t* tris, const int32_t* light_tris, int L, float4* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int j = 0; j < L; ++j)
    for (int k = 0; k < 3; ++k) {
      const float* v = verts + 3 * tris[3 * light_tris[j] + k];
      for (int i = 0; i < 3; ++i) { lo[i] = et_min(lo[i], v[i]); hi[i] = et_max(hi[i], v[i]); }
    }
  float c[3], r;
  et_sphere(lo, hi, c, r);
  *out = make_float4(c[0], c[1], c[2], r);
}

__global__ void k_etree_keys(SceneView s, const int2* opp, const int* b, uint32_t* keys, int32_t* vals, int spatial) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= s.E) return;
  float O[3], blo[3], bhi[3], R;
  et_frame_of_scene(s, b, O, blo, bhi, &R);
  EtLeafData L;
  et_leaf_data(s.verts, s.edges[e], opp[e], O, L);
  if (spatial) L.classB = false;  // one 3D hierarchy: compact boxes for segment queries
  keys[e] = et_key(L, blo, bhi, R);
  vals[e] = e;
}

__device__ __forceinline__ void et_store_slot(float4* nodes, int node, int c, const float lo[3], const float hi[3],
                                              const float hlo[3], const float hhi[3], float L, bool allB, int code) {
  float4* r = nodes + (size_t)kEtNodeF4 * node + 4 * c;
  r[0] = make_float4(lo[0], lo[1], lo[2], L);
  r[1] = make_float4(hi[0], hi[1], hi[2], allB ? 1.0f : 0.0f);
  r[2] = make_float4(hlo[0], hlo[1], hlo[2], __int_as_float(code));
  r[3] = make_float4(hhi[0], hhi[1], hhi[2], 0.0f);
}

// One thread per key position: the leaf record, then a bottom-up climb that
// writes each child's slot into its parent; the second child to arrive at a
// node merges both slots (left then right, so sums are order-independent of
// arrival) and continues.
__global__ void k_etree_refit(SceneView s, const int2* opp, const int32_t* vals, const int2* child,
                              const int32_t* parent, const int32_t* leaf_parent, int32_t* flags, float4* nodes,
                              float4* leaf) {
  int pos = blockIdx.x * blockDim.x + threadIdx.x;
  int E = s.E;
  if (pos >= E) return;
  int e = vals[pos];
  float O[3];
  for (int k = 0; k < 3; ++k) O[k] = s.cam[4 * k + 3];
  EtLeafData L;
  et_leaf_data(s.verts, s.edges[e], opp[e], O, L);
  float4* lr = leaf + (size_t)kEtLeafF4 * pos;
  lr[0] = make_float4(L.v0[0], L.v0[1], L.v0[2], L.len);
  lr[1] = make_float4(L.v1[0], L.v1[1], L.v1[2], __int_as_float(e));
  lr[2] = make_float4(L.c0[0], L.c0[1], L.c0[2], __int_as_float((L.boundary ? 1 : 0) | (L.classB ? 2 : 0)));
  lr[3] = make_float4(L.c1[0], L.c1[1], L.c1[2], 0.0f);
  if (E == 1) return;
  float lo[3], hi[3], hlo[3], hhi[3];
  for (int k = 0; k < 3; ++k) {
    lo[k] = et_min(L.v0[k], L.v1[k]);
    hi[k] = et_max(L.v0[k], L.v1[k]);
    hlo[k] = L.classB ? et_min(L.h0[k], L.h1[k]) : INFINITY;
    hhi[k] = L.classB ? et_max(L.h0[k], L.h1[k]) : -INFINITY;
  }
  float Ls = L.len;
  bool allB = L.classB;
  int code = ~pos;
  int node = leaf_parent[pos];
  int climb = 0;
  while (node >= 0) {
    if (++climb > E) {  // deeper than the tree can be: parent links are broken
      raise_flag(s.err, DRT_DEV_REFIT_CAP, pos);
      return;
    }
    int2 ch = child[node];
    int c = ch.x == code ? 0 : 1;
    et_store_slot(nodes, node, c, lo, hi, hlo, hhi, Ls, allB, code);
    __threadfence();
    if (atomicAdd(flags + node, 1) == 0) return;  // the sibling finishes this node
    __threadfence();
    const float* a = reinterpret_cast<const float*>(nodes + (size_t)kEtNodeF4 * node);
    const float* bq = a + 16;
    float aL = __ldcg(a + 3), bL = __ldcg(bq + 3);
    bool aB = __ldcg(a + 7) != 0.0f, bB = __ldcg(bq + 7) != 0.0f;
    for (int k = 0; k < 3; ++k) {
      lo[k] = et_min(__ldcg(a + k), __ldcg(bq + k));
      hi[k] = et_max(__ldcg(a + 4 + k), __ldcg(bq + 4 + k));
      hlo[k] = et_min(__ldcg(a + 8 + k), __ldcg(bq + 8 + k));
      hhi[k] = et_max(__ldcg(a + 12 + k), __ldcg(bq + 12 + k));
    }
    Ls = fa(aL, bL);
    allB = aB && bB;
    code = node;
    node = parent[node];
  }
}

}  // namespace

cudaError_t launch_segment_features(const drt_scene* s, const float* d_image, const float* image, void* x,
                                    cudaStream_t st) {
  int tx = (s->W + 15) / 16, ty = (s->H + 15) / 16, nt = tx * ty;
  DRT_PROF_LAUNCH("tile_weights", st, k_tile_weights<<<(nt + kBlock - 1) / kBlock, kBlock, 0, st>>>(
                                          d_image, s->W, s->H, tx, ty, s->tile_w));
  DRT_PROF_LAUNCH("tile_weight_mean", st, k_tile_weight_mean<<<1, kBlock, 0, st>>>(s->tile_w, nt));
  int n = (int)s->seg_n;
  if (n > 0)
    DRT_PROF_LAUNCH("segment_features", st, k_segment_features<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(
                                                s->view(), s->seg_edge, s->seg_tile, s->seg_s, s->seg_len, n,
                                                s->edge_faces, s->tile_w, d_image, image, (__nv_bfloat16*)x));
  return cudaGetLastError();
}

size_t scan_tmp_entries(int n) { return (size_t)(n + kScanTile - 1) / kScanTile + 1; }

cudaError_t scan_exclusive_u32(uint32_t* data, uint32_t* tmp, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int nt = (n + kScanTile - 1) / kScanTile;
  DRT_PROF_LAUNCH("scan_u32_tiles", st, k_hist_scan_tiles<<<nt, kBlock, 0, st>>>(data, tmp, n));
  DRT_PROF_LAUNCH("scan_u32_sums", st, k_hist_scan_sums<<<1, kBlock, 0, st>>>(tmp, nt));
  DRT_PROF_LAUNCH("scan_u32_add", st, k_hist_scan_add<<<nt, kBlock, 0, st>>>(data, tmp, n));
  return cudaGetLastError();
}

cudaError_t scan_inclusive_f64(const double* in, double* out, double* tmp, int n, cudaStream_t st) {
  return scan_inclusive(in, out, tmp, n, st);
}

cudaError_t launch_segment_count(const drt_scene* s, uint32_t* counts, cudaStream_t st) {
  if (s->E > 0)
    DRT_PROF_LAUNCH("segment_count", st, k_segment_count<<<(s->E + kBlock - 1) / kBlock, kBlock, 0, st>>>(
                                            s->view(), s->plen, counts));
  return cudaGetLastError();
}

cudaError_t launch_segment_fill(const drt_scene* s, const uint32_t* offsets, cudaStream_t st) {
  if (s->E > 0)
    DRT_PROF_LAUNCH("segment_fill", st, k_segment_fill<<<(s->E + kBlock - 1) / kBlock, kBlock, 0, st>>>(
                                           s->view(), s->plen, offsets, s->seg_edge, s->seg_tile, s->seg_s,
                                           s->seg_len));
  return cudaGetLastError();
}

cudaError_t launch_proposal_cdf(drt_scene* s, const float* weights, int mode, cudaStream_t st) {
  int n = (int)s->seg_n;
  if (n <= 0) return cudaSuccess;
  unsigned g = (unsigned)((n + kBlock - 1) / kBlock);
  cudaError_t e = scan_inclusive(s->seg_len, s->seg_a, s->seg_tmp, n, st);  // seg_a = cumulative length
  if (e != cudaSuccess) return e;
  DRT_PROF_LAUNCH("proposal_weights", st, k_weights_to_f64<<<g, kBlock, 0, st>>>(weights, s->seg_len, n, mode,
                                                                                  s->seg_b));
  e = scan_inclusive(s->seg_b, s->seg_cdf, s->seg_tmp, n, st);  // seg_cdf = cumulative weight (temporarily)
  if (e != cudaSuccess) return e;
  DRT_PROF_LAUNCH("proposal_q", st, k_proposal_q<<<g, kBlock, 0, st>>>(s->seg_len, s->seg_a, s->seg_b, s->seg_cdf,
                                                                       n, s->seg_b));
  return scan_inclusive(s->seg_b, s->seg_cdf, s->seg_tmp, n, st);
}

size_t radix_hist_entries(int n) { return 256 * (size_t)((n + kSortTile - 1) / kSortTile); }
size_t radix_hist_tmp_entries(int n) { return (radix_hist_entries(n) + kScanTile - 1) / kScanTile + 1; }

bool radix_sort_pairs(uint32_t* keys, int32_t* vals, uint32_t* keys2, int32_t* vals2, uint32_t* hist,
                      uint32_t* hist_tmp, int n, int bits, cudaStream_t st) {
  uint32_t *ka = keys, *kb = keys2;
  int32_t *va = vals, *vb = vals2;
  int nb = (n + kSortTile - 1) / kSortTile;
  int m = 256 * nb;
  int nt = (m + kScanTile - 1) / kScanTile;
  bool alt = false;
  for (int shift = 0; shift < bits; shift += 8) {
    DRT_PROF_LAUNCH("sort_hist", st, k_sort_hist<<<nb, kBlock, 0, st>>>(ka, n, shift, hist, nb));
    DRT_PROF_LAUNCH("sort_scan_tiles", st, k_hist_scan_tiles<<<nt, kBlock, 0, st>>>(hist, hist_tmp, m));
    DRT_PROF_LAUNCH("sort_scan_sums", st, k_hist_scan_sums<<<1, kBlock, 0, st>>>(hist_tmp, nt));
    DRT_PROF_LAUNCH("sort_scan_add", st, k_hist_scan_add<<<nt, kBlock, 0, st>>>(hist, hist_tmp, m));
    DRT_PROF_LAUNCH("sort_scatter", st, k_sort_scatter<<<nb, kBlock, 0, st>>>(ka, va, kb, vb, n, shift, hist, nb));
    std::swap(ka, kb);
    std::swap(va, vb);
    alt = !alt;
  }
  return alt;
}

cudaError_t check_finite(drt_scene* s, cudaStream_t st) {
  int n = 3 * s->V;
  if (n > 0) DRT_PROF_LAUNCH("check_finite", st, k_check_finite<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(s->verts, n, s->ctx->err));
  return cudaGetLastError();
}

cudaError_t build_bvh(drt_scene* s, cudaStream_t st) {
  SceneView v = s->view();
  int T = s->T;
  DRT_PROF_LAUNCH("bounds_init", st, k_bounds_init<<<1, 32, 0, st>>>(s->bounds));
  DRT_PROF_LAUNCH("bounds", st, k_bounds<<<std::min(1024, (s->V + kBlock - 1) / kBlock), kBlock, 0, st>>>(s->verts, s->V, s->bounds));
  DRT_PROF_LAUNCH("morton", st, k_morton<<<(T + kBlock - 1) / kBlock, kBlock, 0, st>>>(v, s->bounds, s->keys, s->vals));
  bool alt = radix_sort_pairs(s->keys, s->vals, s->keys2, s->vals2, s->hist, s->hist_tmp, T, 31, st);
  uint32_t* ka = alt ? s->keys2 : s->keys;
  int32_t* va = alt ? s->vals2 : s->vals;
  if (T > 1) {
    cudaMemsetAsync(s->flags, 0, sizeof(int32_t) * (T - 1), st);
    DRT_PROF_LAUNCH("karras", st, k_karras<<<(T - 1 + kBlock - 1) / kBlock, kBlock, 0, st>>>(ka, T, s->leaf_max, s->nodes, s->child_orig, s->parent, s->leaf_parent));
  }
  DRT_PROF_LAUNCH("refit", st, k_refit<<<(T + kBlock - 1) / kBlock, kBlock, 0, st>>>(v, va, s->nodes, s->soup, s->child_orig, s->parent, s->leaf_parent, s->flags, s->tsize));
  if (T > s->leaf_max && T >= kTreeletLeaves) {
    // a second pass pays with single-triangle leaves (the 200k-triangle
    // depth-3 step), not with two per leaf (the 5k-triangle direct-lighting
    // step: 6.62 -> 6.98 ms)
    int rounds = s->leaf_max == 1 ? DRT_TREELET_ROUNDS : 1;
    for (int r = 0; r < rounds; ++r) {
      cudaMemsetAsync(s->flags, 0, sizeof(int32_t) * (T - 1), st);
      DRT_PROF_LAUNCH("treelets", st, k_treelets<<<(T - 1 + kTreeletWarps - 1) / kTreeletWarps, 32 * kTreeletWarps, 0, st>>>(T, s->leaf_max, kTreeletLeaves << r, s->nodes, s->parent, s->tsize, s->flags, s->ctx->err));
    }
  }
  return cudaGetLastError();
}

// Guide table of an inclusive CDF: g[b] = first index whose value exceeds
// b * total / kGuide (b < kGuide), g[kGuide] = n.
__global__ void k_cdf_guide(const double* cdf, int n, int* guide) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > kGuide) return;
  if (b == kGuide) {
    guide[b] = n;
    return;
  }
  double thr = (double)b * (cdf[n - 1] / (double)kGuide);
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cdf[mid] > thr) hi = mid; else lo = mid + 1;
  }
  guide[b] = lo;
}

cudaError_t build_edge_cdfs(drt_scene* s, cudaStream_t st) {
  if (s->E <= 0) return cudaSuccess;
  DRT_PROF_LAUNCH("edge_tables", st, k_edge_tables<<<(s->E + kBlock - 1) / kBlock, kBlock, 0, st>>>(s->view(), s->pedge, s->plen, s->slen));
  cudaError_t e = scan_inclusive(s->plen, s->pcdf, s->scan_tmp, s->E, st);
  if (e != cudaSuccess) return e;
  e = scan_inclusive(s->slen, s->scdf, s->scan_tmp, s->E, st);
  if (e != cudaSuccess) return e;
  unsigned gb = (kGuide + 1 + kBlock - 1) / kBlock;
  DRT_PROF_LAUNCH("cdf_guides", st, k_cdf_guide<<<gb, kBlock, 0, st>>>(s->pcdf, s->E, s->pguide));
  DRT_PROF_LAUNCH("cdf_guides", st, k_cdf_guide<<<gb, kBlock, 0, st>>>(s->scdf, s->E, s->sguide));
  return cudaGetLastError();
}

cudaError_t build_edge_tree(drt_scene* s, cudaStream_t st, bool spatial) {
  int E = s->E;
  if (E <= 0) return cudaSuccess;
  SceneView v = s->view();
  if (s->L > 0)
    DRT_PROF_LAUNCH("etree_light", st, k_etree_light<<<1, 1, 0, st>>>(s->verts, s->tris, s->light_tris, s->L,
                                                                        s->et_leaf + (size_t)kEtLeafF4 * E));
  // the scene box (s->bounds) is the one the triangle LBVH build computed
  DRT_PROF_LAUNCH("etree_keys", st, k_etree_keys<<<(E + kBlock - 1) / kBlock, kBlock, 0, st>>>(
                                        v, s->edge_opp, s->bounds, s->et_keys, s->et_vals, spatial ? 1 : 0));
  bool alt = radix_sort_pairs(s->et_keys, s->et_vals, s->et_keys2, s->et_vals2, s->et_hist, s->et_hist_tmp, E, 31, st);
  uint32_t* ka = alt ? s->et_keys2 : s->et_keys;
  int32_t* va = alt ? s->et_vals2 : s->et_vals;
  if (E > 1) {
    cudaMemsetAsync(s->et_flags, 0, sizeof(int32_t) * (E - 1), st);
    DRT_PROF_LAUNCH("etree_karras", st, k_karras<<<(E - 1 + kBlock - 1) / kBlock, kBlock, 0, st>>>(
                                            ka, E, 1, nullptr, s->et_child, s->et_parent, s->et_leaf_parent));
  }
  DRT_PROF_LAUNCH("etree_refit", st, k_etree_refit<<<(E + kBlock - 1) / kBlock, kBlock, 0, st>>>(
                                         v, s->edge_opp, va, s->et_child, s->et_parent, s->et_leaf_parent,
                                         s->et_flags, s->et_nodes, s->et_leaf));
  return cudaGetLastError();
}

cudaError_t build_scene_derived(drt_scene* s, cudaStream_t st) {
  DRT_PROF_LAUNCH("world_to_cam", st, k_world_to_cam<<<1, 1, 0, st>>>(s->cam, s->w2c));
  if (s->L > 0) DRT_PROF_LAUNCH("light_cdf", st, k_light_cdf<<<1, 1, 0, st>>>(s->verts, s->tris, s->light_tris, s->L, s->light_area, s->light_cdf, s->light_box));
  cudaError_t e = build_bvh(s, st);
  if (e != cudaSuccess) return e;
  e = build_edge_cdfs(s, st);
  return e;
}

}  // namespace drt
