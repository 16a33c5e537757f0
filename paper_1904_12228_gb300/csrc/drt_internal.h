// drt_internal.h -- host-side structures and kernel launchers shared by the
// translation units of the library (not part of the public ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/drt.h"
#include "drt_device.cuh"

struct drt_context {
  int device = 0;
  int* err = nullptr;        // device error flag [2]
  int num_sms = 0;
  // second stream for work that can run beside the caller's stream, joined
  // back by events before its results are read
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

// NVTX range over one C-ABI call (header-only NVTX; a no-op unless a profiler
// is attached), so a timeline shows which library call launched what.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

namespace drt {
// Counters of the queue of secondary edge samples: one per region (one region
// per path vertex, max_depth <= 8, and as many again for the billboard
// samples of next-event estimation for edges).
constexpr int kSecCounters = 16;
// Scratch for the secondary edge samples traced apart: per (sample, vertex)
// the vertex adjoint, the queue of samples to trace and its length.
struct SecScratch {
  float* dp = nullptr;
  unsigned long long* queue = nullptr;
  unsigned long long* count = nullptr;
  int64_t cap = 0;  // (sample, vertex) pairs the buffers hold
  int2* pick = nullptr;  // edge hierarchy: (edge, weight bits) per queued pair
  int64_t pick_cap = 0;
  int4* nee = nullptr;   // next-event estimation for edges: (edge, weight, t, 0) per queued pair
  int64_t nee_cap = 0;
  // beyond depth 1: side hits and continuation radiance per queue slot, and
  // two buffers of continuation-path states (5 float4 each)
  int4* hits = nullptr;
  float* lr = nullptr;
  float4* path[2] = {nullptr, nullptr};
  unsigned long long* path_count = nullptr;
  int64_t wave_cap = 0, path_cap = 0;
};
// Scratch of the primary edge samples beyond depth 1, evaluated in stages:
// radiance of both side paths per sample (screen order) and two buffers of
// continuation-path states (5 float4 each).
struct PrimScratch {
  float* lr = nullptr;
  float4* path[2] = {nullptr, nullptr};
  unsigned long long* count = nullptr;
  int64_t cap = 0;  // edge samples the buffers hold
};
// Scratch of the render beyond depth 1, in stages: radiance per sample and
// two buffers of continuation-path states (5 float4 each).
struct RenderScratch {
  float* L = nullptr;
  float4* path[2] = {nullptr, nullptr};
  unsigned long long* count = nullptr;
  int64_t cap = 0;  // samples the buffers hold
};
// Records and results of the persistent traversal pools the continuation
// stages trace through (closest-hit and any-hit pair records per entry).
struct PoolScratch {
  float4* crec = nullptr;
  int4* hits = nullptr;
  float4* arec = nullptr;
  int* occ = nullptr;
  unsigned long long* next = nullptr;
  int64_t cap = 0;  // entries the buffers hold
};
// Scratch for sorting primary edge samples by screen position (key, index).
struct SortBuffers {
  uint32_t *keys = nullptr, *keys2 = nullptr, *hist = nullptr, *hist_tmp = nullptr;
  int32_t *vals = nullptr, *vals2 = nullptr;
  float4* rec = nullptr;         // [4 * cap] the samples themselves, by sample index (the key pass keeps them)
  float4* rec_sorted = nullptr;  // [4 * cap] the same in screen order: n points, then 3 n float4 of the rest
  int64_t cap = 0;  // samples the buffers hold
};
}  // namespace drt

struct drt_scene {
  drt_context* ctx = nullptr;
  int V = 0, T = 0, L = 0, E = 0, W = 0, H = 0, cam_type = 0;
  int leaf_max = 1;          // most triangles per BVH leaf range (1..kLeafLimit)
  uint64_t generation = 0;   // bumped on every update; tapes remember it
  // parameters (library copies)
  float *verts = nullptr, *albedo = nullptr, *radiance = nullptr, *cam = nullptr, *cam_scale = nullptr;
  int32_t *tris = nullptr, *light_tris = nullptr, *light_of_tri = nullptr;
  // derived
  float* w2c = nullptr;
  double *light_cdf = nullptr, *light_area = nullptr;
  float* light_box = nullptr;
  float4 *nodes = nullptr, *soup = nullptr;
  int2* edges = nullptr;
  int2* edge_faces = nullptr;  // up to two faces per edge (-1 if none)
  int2* edge_opp = nullptr;    // third vertices of the two faces (y = -1 unless exactly two faces)
  // secondary edge hierarchy (built on demand, rebuilt when the scene changes)
  float4 *et_nodes = nullptr, *et_leaf = nullptr;
  uint32_t *et_keys = nullptr, *et_keys2 = nullptr, *et_hist = nullptr, *et_hist_tmp = nullptr;
  int32_t *et_vals = nullptr, *et_vals2 = nullptr, *et_parent = nullptr, *et_leaf_parent = nullptr, *et_flags = nullptr;
  int2* et_child = nullptr;
  uint64_t et_generation = ~0ull;
  bool et_spatial = false;     // built with 3D keys for every edge (next-event estimation for edges)
  float* tile_w = nullptr;     // mean |d_image| per screen tile (features)
  float* pedge = nullptr;
  double *plen = nullptr, *pcdf = nullptr, *slen = nullptr, *scdf = nullptr, *scan_tmp = nullptr;
  int *pguide = nullptr, *sguide = nullptr;  // guide tables of pcdf and scdf
  // LBVH build scratch
  uint32_t *keys = nullptr, *keys2 = nullptr;
  int32_t *vals = nullptr, *vals2 = nullptr, *parent = nullptr, *leaf_parent = nullptr, *flags = nullptr,
          *tsize = nullptr;  // triangles below each internal node (refit, treelet passes)
  int2* child_orig = nullptr;  // Karras children before leaf collapsing (refit)
  uint32_t* hist = nullptr;
  uint32_t* hist_tmp = nullptr;
  int* bounds = nullptr;     // ordered-int AABB [6]
  float* partials = nullptr; // backward: per-block partial sums of global parameters
  size_t partials_cap = 0;
  drt::SortBuffers esort;    // backward: primary edge samples sorted by screen position
  drt::SecScratch sec;       // backward: secondary edge samples queued and traced apart
  drt::PrimScratch prim;     // backward: primary edge samples beyond depth 1 in stages
  drt::RenderScratch rnd;    // render: camera paths beyond depth 1 in stages
  drt::PoolScratch pool;     // render and backward: traversal pools of the continuation stages
  // tile segments of the primary edges (built on demand)
  int32_t *seg_edge = nullptr, *seg_tile = nullptr;
  uint32_t *seg_count = nullptr, *seg_scan_tmp = nullptr;
  float2* seg_s = nullptr;
  double *seg_len = nullptr, *seg_a = nullptr, *seg_b = nullptr, *seg_cdf = nullptr, *seg_tmp = nullptr;
  int64_t seg_cap = 0, seg_n = -1;
  uint64_t seg_generation = ~0ull;
  int sort_blocks = 0;
  float* nee_hw = nullptr;   // billboard half width derived from the vertices (next-event estimation for edges)
  // sample passes (spp_per_pass): one pass's image, the scaled loss adjoint and the pass tape
  float* pass_img = nullptr;
  float* pass_dimg = nullptr;
  drt_tape* pass_tape = nullptr;
  drt::SceneView view() const;
};

struct drt_tape {
  const drt_scene* scene = nullptr;
  uint64_t generation = 0;
  drt_render_opts opts{};
  int64_t n = 0;             // samples = W*H*spp
  int depth = 0;
  int32_t* tri = nullptr;    // [depth, n]  tri id | (nee visible << 31), -1 = none
  float2* bary = nullptr;    // [depth, n]
};

namespace drt {
void set_last_error(const char* msg);  // message returned by drt_last_error on this thread
// api.cu helpers shared with the other entry points
drt_status convert_opts(const drt_render_opts* o, Opts* op);  // validated device options
drt_status device_alloc(void** p, size_t bytes);              // cudaMalloc with fault injection
void device_free(void* p);
bool is_device_array(const void* p);
// prof.cu: event timing of launches (when enabled) and work-counter slots
struct ProfToken {
  const char* name;
  cudaEvent_t a, b;
};
ProfToken prof_begin(const char* name, cudaStream_t st);
void prof_end(const ProfToken& t, cudaStream_t st);
enum { kSlotRender = 0, kSlotBwdInterior = 1, kSlotBwdPrimary = 2, kSlotDebug = 3, kSlotBwdSecondary = 4,
       kSlotBwdSecSides = 5, kSlotBwdSecBounce = 6, kSlotBwdPrimBounce = 7, kSlotRenderBounce = 8, kKernelSlots = 9 };
unsigned long long* counter_slot(int kernel);  // null unless counters are enabled
#define DRT_PROF_LAUNCH(name, st, ...)                      \
  do {                                                      \
    ::drt::ProfToken t_ = ::drt::prof_begin(name, st);      \
    __VA_ARGS__;                                            \
    ::drt::prof_end(t_, st);                                \
  } while (0)
// build.cu
cudaError_t build_scene_derived(drt_scene* s, cudaStream_t st);   // w2c, lights, BVH, edge CDFs
// LSD radix sort of (key, value) pairs on the low `bits` bits; the result is
// in (keys2, vals2) when the return value is true, else in (keys, vals).
bool radix_sort_pairs(uint32_t* keys, int32_t* vals, uint32_t* keys2, int32_t* vals2, uint32_t* hist,
                      uint32_t* hist_tmp, int n, int bits, cudaStream_t st);
size_t radix_hist_entries(int n);
// Secondary edge hierarchy (Sec. 5.3.1) for the scene's current vertices and
// camera; the buffers must be allocated.  spatial: every edge keyed by the 3D
// Morton code of its centroid (no 6D class), the tree the billboard queries
// of next-event estimation for edges walk.
cudaError_t build_edge_tree(drt_scene* s, cudaStream_t st, bool spatial = false);
cudaError_t scan_exclusive_u32(uint32_t* data, uint32_t* tmp, int n, cudaStream_t st);
size_t scan_tmp_entries(int n);
cudaError_t scan_inclusive_f64(const double* in, double* out, double* tmp, int n, cudaStream_t st);
// tile segments: count per edge, fill from exclusive offsets, proposal CDF
cudaError_t launch_segment_count(const drt_scene* s, uint32_t* counts, cudaStream_t st);
cudaError_t launch_segment_fill(const drt_scene* s, const uint32_t* offsets, cudaStream_t st);
cudaError_t launch_proposal_cdf(drt_scene* s, const float* weights, int mode, cudaStream_t st);
cudaError_t launch_segment_features(const drt_scene* s, const float* d_image, const float* image, void* x,
                                    cudaStream_t st);
size_t radix_hist_tmp_entries(int n);
cudaError_t build_bvh(drt_scene* s, cudaStream_t st);
cudaError_t build_edge_cdfs(drt_scene* s, cudaStream_t st);
cudaError_t check_finite(drt_scene* s, cudaStream_t st);
// render.cu
cudaError_t launch_render(const drt_scene* s, const Opts& op, float* image, drt_tape* tape, const RenderScratch* rs,
                          cudaStream_t st);
cudaError_t launch_backward(const drt_scene* s, const Opts& op, const drt_tape* tape, const float* d_image,
                            float* d_verts, float* d_albedo, float* d_radiance, float* d_cam, float* d_cam_scale,
                            float* scratch_global, const SortBuffers* sort, const SecScratch* secs,
                            const PrimScratch* prims, cudaStream_t st);
// (sample, vertex) pairs of the secondary edge samples of a W x H image
int64_t secondary_capacity(int W, int H, const Opts& op);
// continuation-path states the staged secondary evaluation needs (0 at depth 1)
int64_t secondary_path_capacity(int W, int H, const Opts& op);
// queue the secondary edge samples that need rays and trace them (b.dp_sec
// and *b.sec_count zeroed by the caller)
cudaError_t launch_secondary_apart(const BatchScene& b, cudaStream_t st);
int64_t backward_partial_rows(const drt_scene* s, const Opts& op);
// out = in * scale (first) or out + in * scale, n floats
cudaError_t launch_axpy(float* out, const float* in, float scale, int64_t n, bool first, cudaStream_t st);
// billboard half width of next-event estimation for edges from the vertices
cudaError_t launch_nee_half_width(const float* verts, int V, float* out, cudaStream_t st);
cudaError_t launch_debug_closest(const drt_scene* s, int64_t n, const float* o, const float* d, int32_t* tri,
                                 float* tb, cudaStream_t st);
// the single-scene launch shapes the batch reproduces
int pixel_group(int spp);                          // lanes per pixel
int64_t pixel_blocks(int W, int H, int spp);       // blocks of the pixel passes
void primary_blocks(int64_t n_edge, int64_t* blocks_e, int64_t* per_thread);
int64_t primary_blocks_for(int64_t n_edge, int64_t per_thread);  // blocks at a given samples per thread
int screen_key_bits(int W, int H);                 // bits of a pixel's screen key
// batched scenes (persistent kernels; phase = BatchPhase)
cudaError_t launch_batch_phase(int phase, const BatchScene* bs, const int64_t* prefix, int n, int64_t n_items,
                               int grid, int chunk, unsigned long long* counter, cudaStream_t st);
int batch_phase_occupancy(int phase);              // resident CTAs per SM
cudaError_t launch_batch_keys(const BatchScene* bs, const int64_t* eprefix, int n, int64_t total, int pix_bits,
                              int shift, uint32_t* keys, int32_t* vals, cudaStream_t st);
// fixed-order sum of `rows` partial rows into the global gradients; the
// buffer holds partial_floats(rows) floats (the rows, then stage-1 totals)
int64_t partial_floats(int64_t rows);
cudaError_t launch_reduce_globals(float* partials, int64_t rows, float* d_radiance, float* d_cam, float* d_scale,
                                  cudaStream_t st);
}  // namespace drt
