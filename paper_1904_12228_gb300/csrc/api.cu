// api.cu -- the C ABI declared in include/drt.h: contexts, scene upload and
// update, render / backward orchestration, tapes and error reporting.
//
// Host-side rules: every call validates its arguments on the host and returns
// a status (nothing throws across the ABI); device work is enqueued on the
// caller's stream; caller arrays may be host or device memory.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>
#include <climits>

#include "drt_internal.h"
#include "edge_tree.cuh"

namespace {

thread_local std::string g_err;

drt_status fail(drt_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CUDA_TRY(x)                                                                  \
  do {                                                                               \
    cudaError_t e_ = (x);                                                            \
    if (e_ != cudaSuccess) return fail(DRT_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

#define DRT_TRY(x)                    \
  do {                                \
    drt_status s_ = (x);              \
    if (s_ != DRT_OK) return s_;      \
  } while (0)

// Allocation with host-side fault injection: DRT_FAULT_ALLOC_AT=n makes the
// n-th library allocation of the process fail with DRT_ERR_OOM.
long g_alloc_count = 0;
drt_status dalloc(void** p, size_t bytes) {
  *p = nullptr;
  ++g_alloc_count;
  const char* f = std::getenv("DRT_FAULT_ALLOC_AT");
  if (f && std::atol(f) == g_alloc_count) return fail(DRT_ERR_OOM, "injected allocation failure #%ld", g_alloc_count);
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? DRT_ERR_OOM : DRT_ERR_CUDA, "cudaMalloc(%zu): %s", bytes,
                cudaGetErrorString(e));
  }
  return DRT_OK;
}
template <class T>
drt_status dalloc_n(T** p, size_t n) {
  return dalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}
void dfree(void* p) {
  if (p) cudaFree(p);
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device staging buffers for host arrays, kept per device for the next call
// (a cudaMalloc and cudaFree per array and call cost more than the copies
// and synchronised the device).  A buffer returns to its pool only after the
// call that used it has synchronised its stream; drt_destroy releases the
// device's pool.
constexpr int kStageDevices = 64;
constexpr size_t kStageKeep = 16;  // buffers kept per device
std::mutex g_stage_mu;
std::vector<std::pair<void*, size_t>> g_stage_pool[kStageDevices];

int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return dev >= 0 && dev < kStageDevices ? dev : -1;
}
// The smallest pooled buffer of at least `bytes`, else a new one.
drt_status stage_get(void** p, size_t bytes) {
  int dev = current_device();
  if (dev >= 0) {
    std::lock_guard<std::mutex> lk(g_stage_mu);
    auto& pool = g_stage_pool[dev];
    int best = -1;
    for (int i = 0; i < (int)pool.size(); ++i)
      if (pool[i].second >= bytes && (best < 0 || pool[i].second < pool[best].second)) best = i;
    if (best >= 0) {
      *p = pool[best].first;
      pool.erase(pool.begin() + best);
      return DRT_OK;
    }
  }
  return dalloc(p, bytes);
}
void stage_put(void* p, size_t bytes) {
  if (!p) return;
  int dev = current_device();
  if (dev < 0) {
    dfree(p);
    return;
  }
  std::lock_guard<std::mutex> lk(g_stage_mu);
  auto& pool = g_stage_pool[dev];
  pool.emplace_back(p, bytes == 0 ? 16 : bytes);
  if (pool.size() > kStageKeep) {  // drop the smallest
    auto it = std::min_element(pool.begin(), pool.end(),
                               [](const std::pair<void*, size_t>& a, const std::pair<void*, size_t>& b) {
                                 return a.second < b.second;
                               });
    dfree(it->first);
    pool.erase(it);
  }
}
void stage_release_device(int dev) {
  if (dev < 0 || dev >= kStageDevices) return;
  std::lock_guard<std::mutex> lk(g_stage_mu);
  for (auto& b : g_stage_pool[dev]) dfree(b.first);
  g_stage_pool[dev].clear();
}

// A device view of a caller array: the array itself if it is device memory,
// else a device copy (inputs) or staging buffer (outputs) from the pool.
struct Staged {
  void* dev = nullptr;
  void* user = nullptr;
  size_t bytes = 0;
  bool temp = false;
  bool is_output = false;
};
drt_status stage(Staged& s, const void* user, size_t bytes, bool input, bool output, cudaStream_t st) {
  s.user = const_cast<void*>(user);
  s.bytes = bytes;
  s.is_output = output;
  if (!user) return DRT_OK;
  if (is_device_ptr(user)) {
    s.dev = s.user;
    return DRT_OK;
  }
  DRT_TRY(stage_get(&s.dev, bytes));
  s.temp = true;
  if (input) CUDA_TRY(cudaMemcpyAsync(s.dev, user, bytes, cudaMemcpyHostToDevice, st));
  return DRT_OK;
}
// Copy staged outputs back, synchronise, release temporaries.
drt_status unstage(Staged* arr, int n, cudaStream_t st) {
  bool any = false;
  for (int i = 0; i < n; ++i)
    if (arr[i].temp && arr[i].is_output) {
      CUDA_TRY(cudaMemcpyAsync(arr[i].user, arr[i].dev, arr[i].bytes, cudaMemcpyDeviceToHost, st));
      any = true;
    }
  bool anytemp = false;
  for (int i = 0; i < n; ++i) anytemp |= arr[i].temp;
  if (any || anytemp) CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < n; ++i)
    if (arr[i].temp) {
      stage_put(arr[i].dev, arr[i].bytes);
      arr[i].dev = nullptr;
      arr[i].temp = false;
    }
  return DRT_OK;
}

void free_scene_buffers(drt_scene* s) {
  void* bufs[] = {s->verts, s->albedo, s->radiance, s->cam, s->cam_scale, s->tris, s->light_tris, s->light_of_tri,
                  s->w2c, s->light_cdf, s->light_area, s->light_box, s->nodes, s->soup, s->edges, s->edge_faces,
                  s->tile_w, s->pedge, s->plen, s->pcdf,
                  s->slen, s->scdf, s->scan_tmp, s->keys, s->keys2, s->vals, s->vals2, s->parent, s->leaf_parent,
                  s->flags, s->tsize, s->child_orig, s->hist, s->hist_tmp, s->bounds, s->partials, s->esort.keys, s->esort.keys2, s->esort.rec, s->esort.rec_sorted,
                  s->esort.hist, s->esort.hist_tmp, s->esort.vals, s->esort.vals2, s->seg_edge, s->seg_tile,
                  s->seg_count, s->seg_scan_tmp, s->seg_s, s->seg_len, s->seg_a, s->seg_b, s->seg_cdf, s->seg_tmp,
                  s->sec.dp, s->sec.queue, s->sec.count, s->sec.pick, s->sec.nee, s->nee_hw, s->sec.hits, s->sec.lr,
                  s->sec.path[0],
                  s->sec.path[1], s->sec.path_count, s->prim.lr, s->prim.path[0], s->prim.path[1], s->prim.count,
                  s->rnd.L, s->rnd.path[0], s->rnd.path[1], s->rnd.count, s->pool.crec, s->pool.hits, s->pool.arec,
                  s->pool.occ, s->pool.next,
                  s->pguide, s->sguide, s->edge_opp,
                  s->et_nodes, s->et_leaf, s->et_keys, s->et_keys2, s->et_hist, s->et_hist_tmp, s->et_vals,
                  s->et_vals2, s->et_parent, s->et_leaf_parent, s->et_flags, s->et_child};
  for (void* b : bufs) dfree(b);
  dfree(s->pass_img);
  dfree(s->pass_dimg);
  drt_tape_free(nullptr, s->pass_tape);
}

drt_status make_opts(const drt_render_opts* o, drt::Opts* op) {
  if (!o) return fail(DRT_ERR_INVALID_ARG, "opts is NULL");
  if (o->spp < 1) return fail(DRT_ERR_INVALID_ARG, "spp must be >= 1 (got %d)", o->spp);
  if (o->edge_spp < 0) return fail(DRT_ERR_INVALID_ARG, "edge_spp must be >= 0");
  if (o->max_depth < 1 || o->max_depth > 8) return fail(DRT_ERR_INVALID_ARG, "max_depth must be in [1,8]");
  if (o->terms < 0 || o->terms > 7) return fail(DRT_ERR_INVALID_ARG, "terms must be a 3-bit mask");
  op->spp = o->spp;
  op->edge_spp = o->edge_spp;
  op->max_depth = o->max_depth;
  if (o->aov < 0 || o->aov > 4) return fail(DRT_ERR_INVALID_ARG, "aov must be in [0,4]");
  op->aov = o->aov;
  op->primary_only = (o->primary_only || o->aov > 0) ? 1 : 0;
  op->terms = o->terms == 0 ? 7 : o->terms;
  if (o->proposal < 0 || o->proposal > 2) return fail(DRT_ERR_INVALID_ARG, "proposal must be 0, 1 or 2");
  op->proposal = o->proposal;
  op->seg_log = o->proposal >= 1 ? o->seg_log : nullptr;
  op->key = make_uint2((uint32_t)o->seed, (uint32_t)(o->seed >> 32));
  if (o->scene_id < 0) return fail(DRT_ERR_INVALID_ARG, "scene_id must be >= 0");
  op->scene_id = (uint32_t)o->scene_id;
  op->eps_rel = o->eps_rel > 0.0f ? o->eps_rel : 1.52587890625e-05f;
  if (o->sec_sampler < 0 || o->sec_sampler > 1) return fail(DRT_ERR_INVALID_ARG, "sec_sampler must be 0 or 1");
  if (o->sec_tree_samples < 0 || o->sec_tree_samples > drt::kEtMaxSamples)
    return fail(DRT_ERR_INVALID_ARG, "sec_tree_samples must be in [0,%d]", drt::kEtMaxSamples);
  if (o->sec_point < 0 || o->sec_point > 1) return fail(DRT_ERR_INVALID_ARG, "sec_point must be 0 or 1");
  op->sec_sampler = o->sec_sampler;
  op->sec_point = o->sec_point;
  op->sec_samples = o->sec_tree_samples > 0 ? o->sec_tree_samples : drt::kEtDefaultSamples;
  // next-event estimation for edges: beside the length sampler and the uniform point only
  if (o->sec_nee < 0 || o->sec_nee > 1) return fail(DRT_ERR_INVALID_ARG, "sec_nee must be 0 or 1");
  if (o->sec_nee && (o->sec_sampler != 0 || o->sec_point != 0))
    return fail(DRT_ERR_INVALID_ARG, "sec_nee needs sec_sampler 0 and sec_point 0");
  if (!(o->nee_width == o->nee_width) || o->nee_width == INFINITY)
    return fail(DRT_ERR_INVALID_ARG, "nee_width must be finite");
  if (o->spp_per_pass < 0) return fail(DRT_ERR_INVALID_ARG, "spp_per_pass must be >= 0");
  if (o->spp_per_pass > 0 && o->spp_per_pass < o->spp && o->spp % o->spp_per_pass != 0)
    return fail(DRT_ERR_INVALID_ARG, "spp (%d) must be a multiple of spp_per_pass (%d)", o->spp, o->spp_per_pass);
  op->nee = o->sec_nee;
  op->nee_hw = o->nee_width > 0.0f ? 0.5f * o->nee_width : 0.0f;
  op->nee_hw_dev = nullptr;
  // which samples the backward pass evaluates (all by default)
  if (o->pix_begin < 0 || o->edge_begin < 0)
    return fail(DRT_ERR_INVALID_ARG, "pix_begin and edge_begin must be >= 0");
  op->pix_begin = o->pix_begin;
  op->pix_end = o->pix_end > 0 ? o->pix_end : INT32_MAX;
  op->edge_begin = o->edge_begin;
  op->edge_end = o->edge_end > 0 ? o->edge_end : INT64_MAX;
  op->jac.out = nullptr;
  op->jac.n = 0;
  op->jac.npix = 0;
  op->jac.v3 = op->jac.t3 = 0;
  for (int k = 0; k < 8; ++k) op->jac.param[k] = -1;
  return DRT_OK;
}

// Secondary edge hierarchy for the scene's current state: allocated on first
// use (unless alloc is false), rebuilt on the stream when the scene changed.
drt_status ensure_edge_tree(drt_scene* s, bool alloc, cudaStream_t st, bool spatial) {
  int E = s->E;
  if (E <= 0) return DRT_OK;
  if (!s->et_leaf) {
    if (!alloc) return fail(DRT_ERR_STATE, "the edge hierarchy is not allocated (run one backward with it first)");
    drt_status a = DRT_OK;
    size_t n = (size_t)E, m = (size_t)std::max(1, E - 1);
    if (a == DRT_OK) a = dalloc_n(&s->et_nodes, drt::kEtNodeF4 * m);
    if (a == DRT_OK) a = dalloc_n(&s->et_leaf, drt::kEtLeafF4 * n + 1);  // + the lights' sphere
    if (a == DRT_OK) a = dalloc_n(&s->et_keys, n);
    if (a == DRT_OK) a = dalloc_n(&s->et_keys2, n);
    if (a == DRT_OK) a = dalloc_n(&s->et_vals, n);
    if (a == DRT_OK) a = dalloc_n(&s->et_vals2, n);
    if (a == DRT_OK) a = dalloc_n(&s->et_hist, drt::radix_hist_entries(E));
    if (a == DRT_OK) a = dalloc_n(&s->et_hist_tmp, drt::radix_hist_tmp_entries(E));
    if (a == DRT_OK) a = dalloc_n(&s->et_child, m);
    if (a == DRT_OK) a = dalloc_n(&s->et_parent, m);
    if (a == DRT_OK) a = dalloc_n(&s->et_leaf_parent, n);
    if (a == DRT_OK) a = dalloc_n(&s->et_flags, m);
    if (a != DRT_OK) {
      void* bufs[] = {s->et_nodes, s->et_leaf, s->et_keys, s->et_keys2, s->et_vals, s->et_vals2, s->et_hist,
                      s->et_hist_tmp, s->et_child, s->et_parent, s->et_leaf_parent, s->et_flags};
      for (void* b : bufs) dfree(b);
      s->et_nodes = s->et_leaf = nullptr;
      s->et_keys = s->et_keys2 = s->et_hist = s->et_hist_tmp = nullptr;
      s->et_vals = s->et_vals2 = s->et_parent = s->et_leaf_parent = s->et_flags = nullptr;
      s->et_child = nullptr;
      return a;
    }
  }
  if (s->et_generation == s->generation && s->et_spatial == spatial) return DRT_OK;
  CUDA_TRY(drt::build_edge_tree(s, st, spatial));
  s->et_generation = s->generation;
  s->et_spatial = spatial;
  return DRT_OK;
}

// Tile segments for the scene's current state (synchronises to learn the count).
drt_status build_segments(drt_scene* s, cudaStream_t st) {
  if (s->seg_generation == s->generation && s->seg_n >= 0) return DRT_OK;
  int E = s->E;
  if (!s->seg_count) {
    DRT_TRY(dalloc_n(&s->seg_count, (size_t)E + 1));
    DRT_TRY(dalloc_n(&s->seg_scan_tmp, drt::scan_tmp_entries(E + 1)));
  }
  CUDA_TRY(cudaMemsetAsync(s->seg_count, 0, sizeof(uint32_t) * ((size_t)E + 1), st));
  CUDA_TRY(drt::launch_segment_count(s, s->seg_count, st));
  CUDA_TRY(drt::scan_exclusive_u32(s->seg_count, s->seg_scan_tmp, E + 1, st));
  uint32_t total = 0;
  CUDA_TRY(cudaMemcpyAsync(&total, s->seg_count + E, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if ((int64_t)total > s->seg_cap) {
    void* old[] = {s->seg_edge, s->seg_tile, s->seg_s, s->seg_len, s->seg_a, s->seg_b, s->seg_cdf, s->seg_tmp};
    for (void* p : old) dfree(p);
    s->seg_edge = s->seg_tile = nullptr;
    s->seg_s = nullptr;
    s->seg_len = s->seg_a = s->seg_b = s->seg_cdf = s->seg_tmp = nullptr;
    s->seg_cap = 0;
    size_t n = std::max<size_t>(1, total);
    DRT_TRY(dalloc_n(&s->seg_edge, n));
    DRT_TRY(dalloc_n(&s->seg_tile, n));
    DRT_TRY(dalloc_n(&s->seg_s, n));
    DRT_TRY(dalloc_n(&s->seg_len, n));
    DRT_TRY(dalloc_n(&s->seg_a, n));
    DRT_TRY(dalloc_n(&s->seg_b, n));
    DRT_TRY(dalloc_n(&s->seg_cdf, n));
    DRT_TRY(dalloc_n(&s->seg_tmp, n / 1024 + 2));
    s->seg_cap = (int64_t)n;
  }
  CUDA_TRY(drt::launch_segment_fill(s, s->seg_count, st));
  s->seg_n = total;
  s->seg_generation = s->generation;
  return DRT_OK;
}

}  // namespace

namespace drt {
void set_last_error(const char* msg) { g_err = msg; }
drt_status convert_opts(const drt_render_opts* o, Opts* op) { return make_opts(o, op); }
drt_status device_alloc(void** p, size_t bytes) { return dalloc(p, bytes); }
void device_free(void* p) { dfree(p); }
bool is_device_array(const void* p) { return is_device_ptr(p); }
}  // namespace drt

drt::SceneView drt_scene::view() const {
  drt::SceneView v;
  v.verts = verts; v.tris = tris; v.albedo = albedo; v.radiance = radiance; v.cam = cam; v.cam_scale = cam_scale;
  v.w2c = w2c; v.light_tris = light_tris; v.light_of_tri = light_of_tri; v.light_cdf = light_cdf;
  v.light_area = light_area; v.light_box = light_box; v.nodes = nodes; v.soup = soup; v.edges = edges; v.pedge = pedge; v.pcdf = pcdf;
  v.scdf = scdf; v.pguide = pguide; v.sguide = sguide; v.err = ctx->err; v.counters = nullptr;
  v.seg_cdf = seg_n > 0 ? seg_cdf : nullptr; v.seg_edge = seg_edge; v.seg_s = seg_s; v.seg_len = seg_len;
  v.n_seg = (int)std::max<int64_t>(0, seg_n);
  v.V = V; v.T = T; v.L = L; v.E = E; v.W = W; v.H = H; v.cam_type = cam_type;
  v.root = T > leaf_max ? 0 : drt::leaf_enc(0, T);
  v.et_nodes = et_nodes;
  v.et_leaf = et_leaf;
  v.et_light = (et_leaf && L > 0) ? et_leaf + (size_t)drt::kEtLeafF4 * E : nullptr;
  v.et_root = (et_leaf && et_generation == generation && E > 0) ? (E >= 2 ? 0 : ~0) : -1;
  return v;
}

extern "C" {

const char* drt_last_error(drt_context* ctx) {
  (void)ctx;
  return g_err.c_str();
}
const char* drt_version(void) { return "drt 0.1 (sm_103a)"; }

drt_status drt_create(int device, drt_context** out) {
  if (!out) return fail(DRT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int n = 0;
  CUDA_TRY(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(DRT_ERR_INVALID_ARG, "device %d out of range (%d devices)", device, n);
  CUDA_TRY(cudaSetDevice(device));
  drt_context* c = new drt_context();
  c->device = device;
  CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
  drt_status s = dalloc_n(&c->err, 2);
  if (s != DRT_OK) {
    delete c;
    return s;
  }
  CUDA_TRY(cudaMemset(c->err, 0, 2 * sizeof(int)));
  CUDA_TRY(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming));
  *out = c;
  return DRT_OK;
}

drt_status drt_destroy(drt_context* ctx) {
  if (!ctx) return DRT_OK;
  if (ctx->side) cudaStreamSynchronize(ctx->side);
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  if (ctx->join) cudaEventDestroy(ctx->join);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  dfree(ctx->err);
  stage_release_device(ctx->device);
  delete ctx;
  return DRT_OK;
}

drt_status drt_scene_upload(drt_context* ctx, const drt_scene_desc* d, void* stream, drt_scene** out) {
  NvtxRange nvtx_range("drt_scene_upload");
  if (!ctx || !d || !out) return fail(DRT_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (d->n_verts < 3 || d->n_tris < 1) return fail(DRT_ERR_INVALID_ARG, "need >= 3 vertices and >= 1 triangle");
  if (d->width < 1 || d->height < 1) return fail(DRT_ERR_INVALID_ARG, "bad image size %dx%d", d->width, d->height);
  if (d->cam_type != DRT_CAMERA_ORTHO && d->cam_type != DRT_CAMERA_PINHOLE && d->cam_type != DRT_CAMERA_FISHEYE)
    return fail(DRT_ERR_INVALID_ARG, "bad cam_type %d", d->cam_type);
  if (d->cam_type == DRT_CAMERA_FISHEYE) {
    double aspect = (double)d->width / (double)d->height;
    if (!((double)d->cam_scale * std::sqrt(aspect * aspect + 1.0) < 0.99 * 3.141592653589793))
      return fail(DRT_ERR_INVALID_ARG, "fisheye cam_scale %g reaches past the direction behind the camera",
                  (double)d->cam_scale);
  }
  if (!d->verts || !d->tris || !d->albedo || !d->radiance || !d->cam_to_world)
    return fail(DRT_ERR_INVALID_ARG, "NULL scene array");
  if (d->n_light_tris < 0 || (d->n_light_tris > 0 && !d->light_tris))
    return fail(DRT_ERR_INVALID_ARG, "bad light list");
  if (!(d->cam_scale > 0.0f)) return fail(DRT_ERR_INVALID_ARG, "cam_scale must be > 0");
  if (d->bvh_leaf_size < 0 || d->bvh_leaf_size > drt::kLeafLimit)
    return fail(DRT_ERR_INVALID_ARG, "bvh_leaf_size %d outside 0..%d", d->bvh_leaf_size, drt::kLeafLimit);
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(cudaSetDevice(ctx->device));
  // topology on the host: index validation and the unique edge list
  std::vector<int32_t> tris(3 * (size_t)d->n_tris);
  std::vector<int32_t> lts(d->n_light_tris);
  if (is_device_ptr(d->tris) || (d->n_light_tris > 0 && is_device_ptr(d->light_tris))) CUDA_TRY(cudaStreamSynchronize(st));
  CUDA_TRY(cudaMemcpy(tris.data(), d->tris, tris.size() * 4, cudaMemcpyDefault));
  if (d->n_light_tris > 0) CUDA_TRY(cudaMemcpy(lts.data(), d->light_tris, lts.size() * 4, cudaMemcpyDefault));
  for (size_t i = 0; i < tris.size(); ++i)
    if (tris[i] < 0 || tris[i] >= d->n_verts) return fail(DRT_ERR_INVALID_ARG, "triangle index %d out of range", tris[i]);
  std::vector<int32_t> light_of(d->n_tris, -1);
  for (int j = 0; j < d->n_light_tris; ++j) {
    if (lts[j] < 0 || lts[j] >= d->n_tris) return fail(DRT_ERR_INVALID_ARG, "light triangle %d out of range", lts[j]);
    light_of[lts[j]] = j;
  }
  // unique undirected edges sorted by (min, max) vertex, with their first two faces
  std::vector<std::pair<uint64_t, int32_t>> half(tris.size());
  for (int t = 0; t < d->n_tris; ++t)
    for (int k = 0; k < 3; ++k) {
      uint32_t a = (uint32_t)tris[3 * t + k], b = (uint32_t)tris[3 * t + (k + 1) % 3];
      half[3 * t + k] = {((uint64_t)std::min(a, b) << 32) | std::max(a, b), t};
    }
  std::sort(half.begin(), half.end());
  std::vector<int2> edges, edge_faces, edge_opp;
  auto third = [&](int t, int a, int b) {
    int v = tris[3 * (size_t)t];
    for (int k = 0; k < 3; ++k)
      if (tris[3 * (size_t)t + k] != a && tris[3 * (size_t)t + k] != b) v = tris[3 * (size_t)t + k];
    return v;
  };
  for (size_t i = 0; i < half.size();) {
    size_t j = i;
    while (j < half.size() && half[j].first == half[i].first) ++j;
    int a = (int)(half[i].first >> 32), b = (int)(half[i].first & 0xffffffffu);
    edges.push_back(make_int2(a, b));
    edge_faces.push_back(make_int2(half[i].second, j - i > 1 ? half[i + 1].second : -1));
    // the edge hierarchy compares exactly two faces (first in triangle order)
    edge_opp.push_back(j - i == 2 ? make_int2(third(half[i].second, a, b), third(half[i + 1].second, a, b))
                                  : make_int2(-1, -1));
    i = j;
  }

  drt_scene* s = new drt_scene();
  s->ctx = ctx;
  s->V = d->n_verts; s->T = d->n_tris; s->L = d->n_light_tris; s->E = (int)edges.size();
  s->W = d->width; s->H = d->height; s->cam_type = d->cam_type;
  s->leaf_max = d->bvh_leaf_size > 0 ? d->bvh_leaf_size : 1;
  int T = s->T, E = s->E;
  int nb = (T + 2047) / 2048;
  s->sort_blocks = nb;
  drt_status stt = DRT_OK;
#define ALLOC(ptr, n)                                        \
  if (stt == DRT_OK) stt = dalloc_n(&s->ptr, (size_t)(n));
  ALLOC(verts, 3 * (size_t)s->V) ALLOC(albedo, 3 * (size_t)T) ALLOC(radiance, 3) ALLOC(cam, 16)
  ALLOC(cam_scale, 1) ALLOC(tris, 3 * (size_t)T) ALLOC(light_tris, std::max(1, s->L)) ALLOC(light_of_tri, T)
  ALLOC(w2c, 12) ALLOC(light_cdf, std::max(1, s->L)) ALLOC(light_area, std::max(1, s->L)) ALLOC(light_box, 8)
  ALLOC(nodes, 4 * (size_t)std::max(1, T - 1)) ALLOC(soup, 3 * (size_t)T) ALLOC(edges, std::max(1, E))
  ALLOC(edge_faces, std::max(1, E)) ALLOC(edge_opp, std::max(1, E))
  ALLOC(tile_w, (size_t)((s->W + 15) / 16) * ((s->H + 15) / 16) + 1)
  ALLOC(pedge, 8 * (size_t)std::max(1, E)) ALLOC(plen, std::max(1, E)) ALLOC(pcdf, std::max(1, E))
  ALLOC(slen, std::max(1, E)) ALLOC(scdf, std::max(1, E)) ALLOC(scan_tmp, std::max(1, E / 1024 + 2))
  ALLOC(pguide, drt::kGuide + 1) ALLOC(sguide, drt::kGuide + 1)
  ALLOC(keys, T) ALLOC(keys2, T) ALLOC(vals, T) ALLOC(vals2, T) ALLOC(parent, std::max(1, T))
  ALLOC(leaf_parent, T) ALLOC(flags, std::max(1, T)) ALLOC(tsize, std::max(1, T)) ALLOC(child_orig, std::max(1, T)) ALLOC(hist, drt::radix_hist_entries(T))
  ALLOC(hist_tmp, drt::radix_hist_tmp_entries(T)) ALLOC(bounds, 8)
#undef ALLOC
  if (stt != DRT_OK) {
    free_scene_buffers(s);
    delete s;
    return stt;
  }
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st);
  };
  cp(s->verts, d->verts, 12 * (size_t)s->V);
  cp(s->albedo, d->albedo, 12 * (size_t)T);
  cp(s->radiance, d->radiance, 12);
  cp(s->cam, d->cam_to_world, 64);
  cp(s->cam_scale, &d->cam_scale, 4);
  cp(s->tris, tris.data(), 12 * (size_t)T);
  if (s->L > 0) cp(s->light_tris, lts.data(), 4 * (size_t)s->L);
  cp(s->light_of_tri, light_of.data(), 4 * (size_t)T);
  if (E > 0) cp(s->edges, edges.data(), sizeof(int2) * (size_t)E);
  if (E > 0) cp(s->edge_faces, edge_faces.data(), sizeof(int2) * (size_t)E);
  if (E > 0) cp(s->edge_opp, edge_opp.data(), sizeof(int2) * (size_t)E);
  // host vectors above are read by the copies; wait before they go away
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = drt::check_finite(s, st);
  if (e == cudaSuccess) e = drt::build_scene_derived(s, st);
  if (e != cudaSuccess) {
    free_scene_buffers(s);
    delete s;
    return fail(DRT_ERR_CUDA, "scene upload: %s", cudaGetErrorString(e));
  }
  *out = s;
  return DRT_OK;
}

drt_status drt_scene_update_vertices(drt_context* ctx, drt_scene* s, const float* verts, void* stream) {
  NvtxRange nvtx_range("drt_scene_update_vertices");
  if (!ctx || !s || !verts) return fail(DRT_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(s->verts, verts, 12 * (size_t)s->V, cudaMemcpyDefault, st));
  CUDA_TRY(drt::check_finite(s, st));
  CUDA_TRY(drt::build_scene_derived(s, st));
  ++s->generation;
  return DRT_OK;
}

drt_status drt_scene_update_params(drt_context* ctx, drt_scene* s, const float* albedo, const float* radiance,
                                   const float* cam_to_world, const float* cam_scale, void* stream) {
  NvtxRange nvtx_range("drt_scene_update_params");
  if (!ctx || !s) return fail(DRT_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (albedo) CUDA_TRY(cudaMemcpyAsync(s->albedo, albedo, 12 * (size_t)s->T, cudaMemcpyDefault, st));
  if (radiance) CUDA_TRY(cudaMemcpyAsync(s->radiance, radiance, 12, cudaMemcpyDefault, st));
  if (cam_to_world) CUDA_TRY(cudaMemcpyAsync(s->cam, cam_to_world, 64, cudaMemcpyDefault, st));
  if (cam_scale) CUDA_TRY(cudaMemcpyAsync(s->cam_scale, cam_scale, 4, cudaMemcpyDefault, st));
  if (cam_to_world || cam_scale) CUDA_TRY(drt::build_scene_derived(s, st));
  ++s->generation;
  return DRT_OK;
}

drt_status drt_scene_free(drt_context* ctx, drt_scene* s) {
  (void)ctx;
  if (!s) return DRT_OK;
  cudaDeviceSynchronize();
  free_scene_buffers(s);
  delete s;
  return DRT_OK;
}

drt_status drt_tape_free(drt_context* ctx, drt_tape* t) {
  (void)ctx;
  if (!t) return DRT_OK;
  dfree(t->tri);  // cudaFree waits for work that may still use the buffers
  dfree(t->bary);
  delete t;
  return DRT_OK;
}

// Records and results of the traversal pools for `cap` continuation entries.
drt_status ensure_pool(drt_scene* s, int64_t cap, cudaStream_t st) {
  if (cap <= s->pool.cap) return DRT_OK;
  cudaStreamSynchronize(st);
  drt::PoolScratch& b = s->pool;
  dfree(b.crec);
  dfree(b.hits);
  dfree(b.arec);
  dfree(b.occ);
  dfree(b.next);
  b = drt::PoolScratch();
  drt_status a = dalloc_n(&b.crec, (size_t)drt::kClosestRecF4 * cap);
  if (a == DRT_OK) a = dalloc_n(&b.hits, 2 * (size_t)cap);
  if (a == DRT_OK) a = dalloc_n(&b.arec, (size_t)drt::kAnyRecF4 * cap);
  if (a == DRT_OK) a = dalloc_n(&b.occ, (size_t)cap);
  if (a == DRT_OK) a = dalloc_n(&b.next, 2);  // the fetch counters of the two pools
  if (a != DRT_OK) {
    dfree(b.crec);
    dfree(b.hits);
    dfree(b.arec);
    dfree(b.occ);
    dfree(b.next);
    b = drt::PoolScratch();
    return a;
  }
  b.cap = cap;
  return DRT_OK;
}

// Philox key of sample pass p (spp_per_pass): the golden-ratio increment.
uint64_t pass_seed(uint64_t seed, int p) { return seed + (uint64_t)p * 0x9E3779B97F4A7C15ull; }

// One pass's image and the scaled loss adjoint, scene-owned.
drt_status ensure_pass_buffers(drt_scene* s, bool dimg) {
  size_t n = 3 * (size_t)s->W * s->H;
  if (!s->pass_img) DRT_TRY(dalloc_n(&s->pass_img, n));
  if (dimg && !s->pass_dimg) DRT_TRY(dalloc_n(&s->pass_dimg, n));
  return DRT_OK;
}

drt_status drt_render(drt_context* ctx, drt_scene* s, const drt_render_opts* opts, float* image, drt_tape** tape,
                      void* stream) {
  NvtxRange nvtx_range("drt_render");
  if (!ctx || !s || !image) return fail(DRT_ERR_INVALID_ARG, "NULL argument");
  drt::Opts op;
  DRT_TRY(make_opts(opts, &op));
  cudaStream_t st = (cudaStream_t)stream;
  if (opts->spp_per_pass > 0 && opts->spp_per_pass < opts->spp) {
    // sample passes: the image is the mean of the passes' images
    int P = opts->spp / opts->spp_per_pass;
    Staged img;
    DRT_TRY(stage(img, image, 12 * (size_t)s->W * s->H, false, true, st));
    drt_status r = ensure_pass_buffers(s, false);
    for (int p = 0; p < P && r == DRT_OK; ++p) {
      drt_render_opts o = *opts;
      o.spp = opts->spp_per_pass;
      o.spp_per_pass = 0;
      o.seed = pass_seed(opts->seed, p);
      r = drt_render(ctx, s, &o, s->pass_img, p + 1 == P ? tape : nullptr, stream);
      if (r == DRT_OK) {
        cudaError_t e = drt::launch_axpy((float*)img.dev, s->pass_img, (float)(1.0 / P),
                                         3 * (int64_t)s->W * s->H, p == 0, st);
        if (e != cudaSuccess) r = fail(DRT_ERR_CUDA, "pass accumulation: %s", cudaGetErrorString(e));
      }
    }
    drt_status u = unstage(&img, 1, st);
    return r != DRT_OK ? r : u;
  }
  drt_tape* tp = nullptr;
  if (tape) {
    int64_t n = (int64_t)s->W * s->H * op.spp;
    int depth = op.primary_only ? 1 : op.max_depth;
    if (*tape && (*tape)->scene == s && (*tape)->n * (*tape)->depth >= n * depth) {
      tp = *tape;  // reuse the caller's tape storage (no allocation, no sync)
    } else {
      if (*tape) drt_tape_free(ctx, *tape);
      *tape = nullptr;
      tp = new drt_tape();
      tp->scene = s;
      drt_status a = dalloc_n(&tp->tri, (size_t)(n * depth));
      if (a == DRT_OK) a = dalloc_n(&tp->bary, (size_t)(n * depth));
      if (a != DRT_OK) {
        dfree(tp->tri);
        delete tp;
        return a;
      }
    }
    tp->generation = s->generation;
    tp->opts = *opts;
    tp->n = n;
    tp->depth = depth;
  }
  Staged img;
  drt_status r = stage(img, image, 12 * (size_t)s->W * s->H, false, true, st);
  if (r != DRT_OK) {
    drt_tape_free(ctx, tp);
    return r;
  }
  // beyond depth 1 the camera paths are rendered in stages: radiance per
  // sample and continuation states
  const drt::RenderScratch* rs = nullptr;
  int64_t n_s = (int64_t)s->W * s->H * op.spp;
  if (!op.primary_only && op.max_depth > 1 && n_s < (int64_t(1) << 31)) {
    if (n_s > s->rnd.cap) {
      cudaStreamSynchronize(st);
      drt::RenderScratch& b = s->rnd;
      dfree(b.L);
      dfree(b.path[0]);
      dfree(b.path[1]);
      dfree(b.count);
      b = drt::RenderScratch();
      drt_status a = dalloc_n(&b.L, 3 * (size_t)n_s);
      if (a == DRT_OK) a = dalloc_n(&b.path[0], 5 * (size_t)n_s);
      if (a == DRT_OK) a = dalloc_n(&b.path[1], 5 * (size_t)n_s);
      if (a == DRT_OK) a = dalloc_n(&b.count, 2);
      if (a != DRT_OK) {
        unstage(&img, 1, st);
        drt_tape_free(ctx, tp);
        return a;
      }
      b.cap = n_s;
    }
    drt_status a = ensure_pool(s, n_s, st);
    if (a != DRT_OK) {
      unstage(&img, 1, st);
      drt_tape_free(ctx, tp);
      return a;
    }
    rs = &s->rnd;
  }
  cudaError_t e = drt::launch_render(s, op, (float*)img.dev, tp, rs, st);
  if (e != cudaSuccess) {
    unstage(&img, 1, st);
    drt_tape_free(ctx, tp);
    return fail(DRT_ERR_CUDA, "render launch: %s", cudaGetErrorString(e));
  }
  r = unstage(&img, 1, st);
  if (r != DRT_OK) {
    drt_tape_free(ctx, tp);
    return r;
  }
  if (tape) *tape = tp;
  return DRT_OK;
}

drt_status drt_render_backward(drt_context* ctx, drt_scene* s, const drt_tape* tape, const drt_render_opts* opts,
                               const float* d_image, const drt_grads* grads, void* stream) {
  NvtxRange nvtx_range("drt_render_backward");
  if (!ctx || !s || !d_image || !grads) return fail(DRT_ERR_INVALID_ARG, "NULL argument");
  drt::Opts op;
  DRT_TRY(make_opts(opts, &op));
  if (opts->spp_per_pass > 0 && opts->spp_per_pass < opts->spp) {
    // sample passes: the primary edge term once (full edge budget, key seed);
    // the interior and secondary terms per pass, each pass rendered again
    // into scene-owned scratch, with d_image / P
    cudaStream_t st = (cudaStream_t)stream;
    int P = opts->spp / opts->spp_per_pass;
    int terms = opts->terms == 0 ? 7 : opts->terms;
    if (terms & 2) {
      drt_render_opts o = *opts;
      o.spp_per_pass = 0;
      o.terms = 2;
      DRT_TRY(drt_render_backward(ctx, s, nullptr, &o, d_image, grads, stream));
    }
    if (!(terms & 5)) return DRT_OK;
    DRT_TRY(ensure_pass_buffers(s, true));
    Staged w;
    DRT_TRY(stage(w, d_image, 12 * (size_t)s->W * s->H, true, false, st));
    cudaError_t e = drt::launch_axpy(s->pass_dimg, (const float*)w.dev, (float)(1.0 / P), 3 * (int64_t)s->W * s->H,
                                     true, st);
    drt_status r = unstage(&w, 1, st);
    if (e != cudaSuccess) return fail(DRT_ERR_CUDA, "pass adjoint: %s", cudaGetErrorString(e));
    for (int p = 0; p < P && r == DRT_OK; ++p) {
      drt_render_opts o = *opts;
      o.spp = opts->spp_per_pass;
      o.spp_per_pass = 0;
      o.seed = pass_seed(opts->seed, p);
      o.terms = terms & 5;
      r = drt_render(ctx, s, &o, s->pass_img, &s->pass_tape, stream);
      if (r == DRT_OK) r = drt_render_backward(ctx, s, s->pass_tape, &o, s->pass_dimg, grads, stream);
    }
    return r;
  }
  if (!op.primary_only && op.max_depth > 1 && (op.terms & 5) && !tape)
    return fail(DRT_ERR_INVALID_ARG, "interior or secondary terms with max_depth > 1 need the tape of the forward pass");
  if (tape) {
    const drt_render_opts& t = tape->opts;
    if (tape->scene != s || tape->generation != s->generation)
      return fail(DRT_ERR_STATE, "tape belongs to another scene or an older version of this scene");
    if (t.spp != opts->spp || t.seed != opts->seed || t.max_depth != opts->max_depth ||
        (t.primary_only != 0) != (opts->primary_only != 0))
      return fail(DRT_ERR_STATE, "tape was recorded with different sampling options");
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (op.proposal >= 1 && s->cam_type == DRT_CAMERA_FISHEYE)
    return fail(DRT_ERR_INVALID_ARG, "the fisheye camera takes the length proposal (proposal 0)");
  if (op.proposal >= 1) {
    DRT_TRY(build_segments(s, st));
    if (!opts->seg_weights || opts->n_seg_weights != s->seg_n)
      return fail(DRT_ERR_INVALID_ARG, "proposal %d needs %lld segment weights (got %lld)", op.proposal,
                  (long long)s->seg_n, (long long)opts->n_seg_weights);
    if (!is_device_ptr(opts->seg_weights)) return fail(DRT_ERR_INVALID_ARG, "segment weights must be device memory");
    CUDA_TRY(drt::launch_proposal_cdf(s, opts->seg_weights, op.proposal, st));
  }
  // per-pixel gradient image of up to 8 listed parameters (optional)
  int64_t n_params = 3 * (int64_t)s->V + 3 * (int64_t)s->T + 16;
  if (grads->n_jac < 0 || grads->n_jac > 8 || (grads->n_jac > 0 && !grads->dimage_dparam))
    return fail(DRT_ERR_INVALID_ARG, "n_jac must be in [0,8] and needs dimage_dparam");
  for (int k = 0; k < grads->n_jac; ++k)
    if (grads->jac_param[k] < 0 || grads->jac_param[k] >= n_params)
      return fail(DRT_ERR_INVALID_ARG, "jac_param[%d] = %lld outside [0,%lld)", k, (long long)grads->jac_param[k],
                  (long long)n_params);
  Staged sg[7];
  size_t npix = (size_t)s->W * s->H;
  drt_status r = stage(sg[0], d_image, 12 * npix, true, false, st);
  if (r == DRT_OK) r = stage(sg[1], grads->d_verts, 12 * (size_t)s->V, true, true, st);
  if (r == DRT_OK) r = stage(sg[2], grads->d_albedo, 12 * (size_t)s->T, true, true, st);
  if (r == DRT_OK) r = stage(sg[3], grads->d_radiance, 12, true, true, st);
  if (r == DRT_OK) r = stage(sg[4], grads->d_cam_to_world, 48, true, true, st);
  if (r == DRT_OK) r = stage(sg[5], grads->d_cam_scale, 4, true, true, st);
  if (r == DRT_OK && grads->n_jac > 0)
    r = stage(sg[6], grads->dimage_dparam, 4 * npix * (size_t)grads->n_jac, true, true, st);
  if (grads->n_jac > 0) {
    op.jac.out = (float*)sg[6].dev;
    op.jac.n = grads->n_jac;
    op.jac.npix = (int)npix;
    op.jac.v3 = 3 * (int64_t)s->V;
    op.jac.t3 = 3 * (int64_t)s->T;
    for (int k = 0; k < grads->n_jac; ++k) op.jac.param[k] = grads->jac_param[k];
  }
  // per-block partial sums of the global parameters: scene-owned scratch,
  // grown on demand (the stream is drained before the old buffer is freed)
  int64_t rows = drt::backward_partial_rows(s, op);
  size_t need = (size_t)drt::partial_floats(rows);
  if (r == DRT_OK && need > s->partials_cap) {
    cudaStreamSynchronize(st);
    dfree(s->partials);
    s->partials = nullptr;
    s->partials_cap = 0;
    r = dalloc_n(&s->partials, need);
    if (r == DRT_OK) s->partials_cap = need;
  }
  if (r != DRT_OK) {
    unstage(sg, 7, st);
    return r;
  }
  // primary edge samples are evaluated in screen order: grow the sort scratch
  int64_t n_edge = (op.terms & 2) ? (int64_t)op.edge_spp * s->W * s->H : 0;
  const drt::SortBuffers* sort = nullptr;
  if (n_edge > 0 && n_edge < INT32_MAX) {
    if (n_edge > s->esort.cap) {
      cudaStreamSynchronize(st);
      drt::SortBuffers& b = s->esort;
      void* old[] = {b.keys, b.keys2, b.hist, b.hist_tmp, b.vals, b.vals2, b.rec, b.rec_sorted};
      for (void* p : old) dfree(p);
      b = drt::SortBuffers();
      int n = (int)n_edge;
      drt_status a = dalloc_n(&b.keys, n);
      if (a == DRT_OK) a = dalloc_n(&b.keys2, n);
      if (a == DRT_OK) a = dalloc_n(&b.vals, n);
      if (a == DRT_OK) a = dalloc_n(&b.vals2, n);
      if (a == DRT_OK) a = dalloc_n(&b.hist, drt::radix_hist_entries(n));
      if (a == DRT_OK) a = dalloc_n(&b.hist_tmp, drt::radix_hist_tmp_entries(n));
      if (a == DRT_OK) a = dalloc_n(&b.rec, 4 * (size_t)n);
      if (a == DRT_OK) a = dalloc_n(&b.rec_sorted, 4 * (size_t)n);
      if (a != DRT_OK) {
        unstage(sg, 7, st);
        return a;
      }
      b.cap = n_edge;
    }
    sort = &s->esort;
  }
  if ((op.sec_sampler == 1 || op.nee) && !op.primary_only && (op.terms & 4) && s->E > 0 && s->L > 0) {
    drt_status a = ensure_edge_tree(s, true, st, op.nee != 0);
    if (a != DRT_OK) {
      unstage(sg, 7, st);
      return a;
    }
  }
  // billboard half width of next-event estimation for edges from the
  // vertices (one block, fixed-order FP64 sums), when the caller gives none
  if (op.nee && !(op.nee_hw > 0.0f) && !op.primary_only && (op.terms & 4) && s->E > 0 && s->L > 0) {
    if (!s->nee_hw) {
      drt_status a = dalloc_n(&s->nee_hw, 1);
      if (a != DRT_OK) {
        unstage(sg, 7, st);
        return a;
      }
    }
    cudaError_t e = drt::launch_nee_half_width(s->verts, s->V, s->nee_hw, st);
    if (e != cudaSuccess) {
      unstage(sg, 7, st);
      return fail(DRT_ERR_CUDA, "billboard width: %s", cudaGetErrorString(e));
    }
    op.nee_hw_dev = s->nee_hw;
  }
  // secondary edge samples that need rays are queued and traced apart
  const drt::SecScratch* secs = nullptr;
  if (!op.primary_only && (op.terms & 4) && s->E > 0 && s->L > 0) {
    int64_t cap = drt::secondary_capacity(s->W, s->H, op);
    if (cap > s->sec.cap) {
      cudaStreamSynchronize(st);
      drt::SecScratch& b = s->sec;
      dfree(b.dp);
      dfree(b.queue);
      dfree(b.count);
      dfree(b.pick);
      dfree(b.nee);
      dfree(b.hits);
      dfree(b.lr);
      dfree(b.path[0]);
      dfree(b.path[1]);
      dfree(b.path_count);
      b = drt::SecScratch();
      drt_status a = dalloc_n(&b.dp, 3 * (size_t)cap);
      if (a == DRT_OK) a = dalloc_n(&b.queue, (size_t)cap);
      if (a == DRT_OK) a = dalloc_n(&b.count, drt::kSecCounters);
      if (a != DRT_OK) {
        unstage(sg, 7, st);
        return a;
      }
      b.cap = cap;
    }
    // beyond depth 1 the queued samples are evaluated in stages (side rays,
    // continuation paths one vertex per launch, contributions), which keep
    // per-sample hits and radiance and the continuation states
    int64_t pcap = drt::secondary_path_capacity(s->W, s->H, op);
    if (pcap > 0 && (cap > s->sec.wave_cap || pcap > s->sec.path_cap)) {
      cudaStreamSynchronize(st);
      drt::SecScratch& b = s->sec;
      dfree(b.hits);
      dfree(b.lr);
      dfree(b.path[0]);
      dfree(b.path[1]);
      dfree(b.path_count);
      b.hits = nullptr;
      b.lr = nullptr;
      b.path[0] = b.path[1] = nullptr;
      b.path_count = nullptr;
      b.wave_cap = b.path_cap = 0;
      drt_status a = dalloc_n(&b.hits, 2 * (size_t)cap);
      if (a == DRT_OK) a = dalloc_n(&b.lr, 6 * (size_t)cap);
      if (a == DRT_OK) a = dalloc_n(&b.path[0], 5 * (size_t)pcap);
      if (a == DRT_OK) a = dalloc_n(&b.path[1], 5 * (size_t)pcap);
      if (a == DRT_OK) a = dalloc_n(&b.path_count, 2);
      if (a != DRT_OK) {
        unstage(sg, 7, st);
        return a;
      }
      b.wave_cap = cap;
      b.path_cap = pcap;
    }
    if (op.nee && cap > s->sec.nee_cap) {
      cudaStreamSynchronize(st);
      dfree(s->sec.nee);
      s->sec.nee = nullptr;
      s->sec.nee_cap = 0;
      drt_status a = dalloc_n(&s->sec.nee, (size_t)cap);
      if (a != DRT_OK) {
        unstage(sg, 7, st);
        return a;
      }
      s->sec.nee_cap = cap;
    }
    if (op.sec_sampler == 1 && cap > s->sec.pick_cap) {
      cudaStreamSynchronize(st);
      dfree(s->sec.pick);
      s->sec.pick = nullptr;
      s->sec.pick_cap = 0;
      drt_status a = dalloc_n(&s->sec.pick, (size_t)cap);
      if (a != DRT_OK) {
        unstage(sg, 7, st);
        return a;
      }
      s->sec.pick_cap = cap;
    }
    secs = &s->sec;
  }
  // primary edge samples beyond depth 1 are evaluated in stages: radiance per
  // sample and side, continuation-path states
  const drt::PrimScratch* prims = nullptr;
  int md = op.primary_only ? 1 : std::min(op.max_depth, 8);
  if (sort && md > 1) {
    if (n_edge > s->prim.cap) {
      cudaStreamSynchronize(st);
      drt::PrimScratch& b = s->prim;
      dfree(b.lr);
      dfree(b.path[0]);
      dfree(b.path[1]);
      dfree(b.count);
      b = drt::PrimScratch();
      drt_status a = dalloc_n(&b.lr, 6 * (size_t)n_edge);
      if (a == DRT_OK) a = dalloc_n(&b.path[0], 5 * (size_t)n_edge);
      if (a == DRT_OK) a = dalloc_n(&b.path[1], 5 * (size_t)n_edge);
      if (a == DRT_OK) a = dalloc_n(&b.count, 2);
      if (a != DRT_OK) {
        unstage(sg, 7, st);
        return a;
      }
      b.cap = n_edge;
    }
    prims = &s->prim;
  }
  // the continuation stages trace through the pools
  int64_t pool_need = 0;
  if (prims) pool_need = std::max(pool_need, n_edge);
  if (secs) pool_need = std::max(pool_need, drt::secondary_path_capacity(s->W, s->H, op));
  if (pool_need > 0) {
    drt_status a = ensure_pool(s, pool_need, st);
    if (a != DRT_OK) {
      unstage(sg, 7, st);
      return a;
    }
  }
  cudaError_t e = drt::launch_backward(s, op, tape, (const float*)sg[0].dev, (float*)sg[1].dev, (float*)sg[2].dev,
                                       (float*)sg[3].dev, (float*)sg[4].dev, (float*)sg[5].dev, s->partials, sort,
                                       secs, prims, st);
  r = unstage(sg, 7, st);
  if (e != cudaSuccess) return fail(DRT_ERR_CUDA, "backward launch: %s", cudaGetErrorString(e));
  return r;
}

drt_status drt_scene_segments(drt_context* ctx, drt_scene* s, int64_t* n, int32_t* edge_tile, float* s01,
                              double* lens, int64_t cap, void* stream) {
  if (!ctx || !s || !n || cap < 0) return fail(DRT_ERR_INVALID_ARG, "bad argument");
  if (s->cam_type == DRT_CAMERA_FISHEYE) return fail(DRT_ERR_INVALID_ARG, "no screen segments for the fisheye camera");
  cudaStream_t st = (cudaStream_t)stream;
  DRT_TRY(build_segments(s, st));
  *n = s->seg_n;
  int64_t k = std::min<int64_t>(cap, s->seg_n);
  if (k <= 0) return DRT_OK;
  // edge_tile interleaves (edge, tile); s01 is the float2 array; lens the lengths
  if (edge_tile) {
    std::vector<int32_t> e(k), t(k), et(2 * k);
    CUDA_TRY(cudaMemcpyAsync(e.data(), s->seg_edge, 4 * k, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(t.data(), s->seg_tile, 4 * k, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < k; ++i) { et[2 * i] = e[i]; et[2 * i + 1] = t[i]; }
    CUDA_TRY(cudaMemcpy(edge_tile, et.data(), 8 * k, cudaMemcpyDefault));
  }
  if (s01) CUDA_TRY(cudaMemcpyAsync(s01, s->seg_s, 8 * k, cudaMemcpyDefault, st));
  if (lens) CUDA_TRY(cudaMemcpyAsync(lens, s->seg_len, 8 * k, cudaMemcpyDefault, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return DRT_OK;
}

drt_status drt_segment_features(drt_context* ctx, drt_scene* s, const float* d_image, const float* image, void* x,
                                void* stream) {
  NvtxRange nvtx_range("drt_segment_features");
  if (!ctx || !s || !d_image || !x) return fail(DRT_ERR_INVALID_ARG, "NULL argument");
  if (!is_device_ptr(d_image) || !is_device_ptr(x) || (image && !is_device_ptr(image)))
    return fail(DRT_ERR_INVALID_ARG, "device arrays only");
  if (s->cam_type == DRT_CAMERA_FISHEYE) return fail(DRT_ERR_INVALID_ARG, "no screen segments for the fisheye camera");
  cudaStream_t st = (cudaStream_t)stream;
  DRT_TRY(build_segments(s, st));
  CUDA_TRY(drt::launch_segment_features(s, d_image, image, x, st));
  return DRT_OK;
}

drt_status drt_debug_closest(drt_context* ctx, drt_scene* s, int64_t n, const float* o, const float* d,
                             int32_t* tri, float* tb1b2, void* stream) {
  if (!ctx || !s || n < 0 || (n > 0 && (!o || !d || !tri || !tb1b2))) return fail(DRT_ERR_INVALID_ARG, "bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  Staged sg[4];
  drt_status r = stage(sg[0], o, 12 * (size_t)n, true, false, st);
  if (r == DRT_OK) r = stage(sg[1], d, 12 * (size_t)n, true, false, st);
  if (r == DRT_OK) r = stage(sg[2], tri, 4 * (size_t)n, false, true, st);
  if (r == DRT_OK) r = stage(sg[3], tb1b2, 12 * (size_t)n, false, true, st);
  cudaError_t e = cudaSuccess;
  if (r == DRT_OK)
    e = drt::launch_debug_closest(s, n, (const float*)sg[0].dev, (const float*)sg[1].dev, (int32_t*)sg[2].dev,
                                  (float*)sg[3].dev, st);
  drt_status r2 = unstage(sg, 4, st);
  if (r != DRT_OK) return r;
  if (e != cudaSuccess) return fail(DRT_ERR_CUDA, "debug_closest: %s", cudaGetErrorString(e));
  return r2;
}

drt_status drt_check_device(drt_context* ctx, void* stream, int32_t* code, int32_t* info) {
  if (!ctx) return fail(DRT_ERR_INVALID_ARG, "NULL context");
  cudaStream_t st = (cudaStream_t)stream;
  int h[2] = {0, 0};
  CUDA_TRY(cudaStreamSynchronize(st));
  CUDA_TRY(cudaMemcpy(h, ctx->err, sizeof(h), cudaMemcpyDeviceToHost));
  if (code) *code = h[0];
  if (info) *info = h[1];
  if (h[0] != 0) {
    CUDA_TRY(cudaMemset(ctx->err, 0, sizeof(h)));
    return fail(DRT_ERR_DEVICE_FLAG, "device flag %d (info %d)", h[0], h[1]);
  }
  return DRT_OK;
}

}  // extern "C"
