// batch.cu -- many scenes per step: persistent launches over (scene, block)
// work items, one screen sort for the primary edge samples of all scenes, a
// CUDA graph for the whole step and an autotuner for the launch shapes.
//
// Plan.  Scene k of a batch does exactly the work of the single-scene calls
// with opts.scene_id = k: the same pixels per virtual block, the same
// partial-sum rows, the same sample order.  Each pass (render, interior or
// path, primary edges) is one launch of a persistent kernel; its CTAs take
// chunks of items from an atomic counter until none is left.  Secondary edge
// samples that need rays are queued and traced per scene between the render
// and the interior or path pass, as in the single-scene backward.
// The primary edge samples of all scenes are sorted once, with the scene
// index above the screen key, which orders every scene's samples as its own
// sort does.  Per-scene descriptors (scene view, options, output pointers)
// live in a device array; a CTA copies the entry of its current scene into
// shared memory.
//
// Autotuner.  On the first run it times each pass with candidate shapes:
// resident CTAs per SM (1 to the occupancy limit), items per counter
// increment (1, 2, 4, 8) and, for primary edges, the edge budget of a work
// item (samples per thread x 1, 2, 4).  Probe launches write gradients into
// scratch buffers.  The chosen shapes are kept per device and workload
// class for later batches.
//
// Graph.  The step (vertex copies and rebuilds when asked, every pass, the
// sort and the reductions) is captured once into a CUDA graph and replayed
// by each later run.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "drt_internal.h"

using drt::BatchScene;

namespace {

constexpr int kMaxBatch = 1 << 16;

drt_status bfail(drt_status st, const char* msg) {
  drt::set_last_error(msg);
  return st;
}

#define BATCH_CUDA(x)                                                      \
  do {                                                                     \
    cudaError_t e_ = (x);                                                  \
    if (e_ != cudaSuccess) {                                               \
      char m_[256];                                                        \
      std::snprintf(m_, sizeof(m_), "%s: %s", #x, cudaGetErrorString(e_)); \
      return bfail(DRT_ERR_CUDA, m_);                                      \
    }                                                                      \
  } while (0)

#define BATCH_TRY(x)               \
  do {                             \
    drt_status s_ = (x);           \
    if (s_ != DRT_OK) return s_;   \
  } while (0)

struct Shape {
  int ctas[drt::kPhases];   // resident CTAs per SM wanted
  int chunk[drt::kPhases];  // items per counter increment
  int edge_mult;            // primary edge samples per thread = single-scene value x edge_mult
};

Shape default_shape() {
  Shape s;
  for (int p = 0; p < drt::kPhases; ++p) {
    s.ctas[p] = 16;  // clamped to the occupancy limit
    s.chunk[p] = 1;
  }
  s.edge_mult = 1;
  return s;
}

// device, scenes, pixels, edge samples, spp, edge spp, depth, terms
using TuneKey = std::tuple<int, int, int64_t, int64_t, int, int, int, int>;
std::map<TuneKey, Shape> g_tuned;

}  // namespace

struct drt_batch {
  drt_context* ctx = nullptr;
  int n = 0;
  std::vector<drt_batch_item> items;
  drt::Opts op{};
  bool use_graph = false, autotune = false, tuned = false;
  double tune_ms = 0.0;
  Shape shape = default_shape();
  int occupancy[drt::kPhases] = {1, 1, 1, 1, 1};
  // plan
  std::vector<BatchScene> desc;
  std::vector<int64_t> prefix;   // kPhases x (n + 1)
  std::vector<int64_t> eprefix;  // n + 1
  int64_t n_items[drt::kPhases] = {};
  int64_t total_edge = 0, total_tape = 0, total_floats = 0, total_sec = 0;
  int pix_bits = 0, key_bits = 0;  // screen key bits; with the scene index above them
  int key_shift = 0;               // screen key bits dropped to fit 32-bit keys
  // device
  BatchScene* d_desc = nullptr;
  BatchScene* d_desc_tune = nullptr;
  int64_t* d_prefix = nullptr;
  int64_t* d_eprefix = nullptr;
  unsigned long long* d_counter = nullptr;
  int32_t* tape_tri = nullptr;
  float2* tape_bary = nullptr;
  float* partials = nullptr;
  float* scratch = nullptr;  // gradient sink of the autotuner's probes
  float* sec_dp = nullptr;   // secondary edge samples traced apart: vertex adjoints,
  unsigned long long* sec_queue = nullptr;   // queues
  unsigned long long* sec_counts = nullptr;  // and queue lengths (one per scene)
  uint32_t *keys = nullptr, *keys2 = nullptr, *hist = nullptr, *hist_tmp = nullptr;
  int32_t *vals = nullptr, *vals2 = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int runs = 0;
};

namespace {

// Work items, offsets and descriptors of every scene for the current shape.
// With `bind` false only the totals are computed (before allocation).
void plan(drt_batch* b, bool bind) {
  const int n = b->n;
  const drt::Opts& op = b->op;
  const bool path = !op.primary_only && op.max_depth > 1;
  const bool need_i = (op.terms & 5) != 0;
  const int depth = op.primary_only ? 1 : op.max_depth;
  b->prefix.assign((size_t)drt::kPhases * (n + 1), 0);
  b->eprefix.assign(n + 1, 0);
  b->desc.assign(n, BatchScene{});
  int64_t tape_off = 0, float_off = 0, sec_off = 0;
  int pix_bits = 2;
  for (int k = 0; k < n; ++k) {
    const drt_batch_item& it = b->items[k];
    const drt_scene* s = it.scene;
    BatchScene& d = b->desc[k];
    std::memset(&d, 0, sizeof(d));
    d.v = s->view();
    d.v.counters = nullptr;
    d.v.seg_cdf = nullptr;
    d.op = op;
    d.op.scene_id = (uint32_t)k;
    d.op.proposal = 0;
    d.op.seg_log = nullptr;
    d.image = it.image;
    d.G = drt::pixel_group(op.spp);
    const int64_t npix = (int64_t)s->W * s->H;
    const int64_t blocks_i = drt::pixel_blocks(s->W, s->H, op.spp);
    int64_t cnt[drt::kPhases] = {blocks_i, 0, 0, 0, 0};
    int64_t tape_here = tape_off;
    tape_off += npix * op.spp * depth;
    int64_t float_here = float_off;
    if (it.d_image) {
      d.d_image = it.d_image;
      d.d_verts = it.grads.d_verts;
      d.d_albedo = it.grads.d_albedo;
      d.d_radiance = it.grads.d_radiance;
      d.d_cam = it.grads.d_cam_to_world;
      d.d_scale = it.grads.d_cam_scale;
      // secondary edge samples are queued and traced apart; the pixel pass
      // (interior or path) adds their vertex adjoints
      const bool sec = !op.primary_only && (op.terms & 4) && s->E > 0 && s->L > 0;
      if (path && need_i) cnt[drt::kPhasePath] = blocks_i;
      else if (need_i) cnt[drt::kPhaseInterior] = blocks_i;
      d.rows_written = 0;
      d.do_int = op.terms & 1;
      d.rows_i = need_i ? blocks_i : 0;
      if (sec) {
        int64_t cap = drt::secondary_capacity(s->W, s->H, op);
        if (bind) {
          d.dp_sec = b->sec_dp + 3 * sec_off;
          d.sec_queue = b->sec_queue + sec_off;
          d.sec_count = b->sec_counts + (size_t)k * drt::kSecCounters;
        }
        d.sec_cap = cap;
        sec_off += cap;
      }
      const int64_t n_edge = (int64_t)op.edge_spp * npix;
      if ((op.terms & 2) && s->E > 0 && n_edge > 0) {
        int64_t be = 0, pt = 0;
        drt::primary_blocks(n_edge, &be, &pt);
        if (b->shape.edge_mult > 1) {
          pt *= b->shape.edge_mult;
          be = drt::primary_blocks_for(n_edge, pt);
        }
        d.n_edge = n_edge;
        d.per_thread = pt;
        d.blocks_e = be;
        cnt[drt::kPhasePrimary] = be;
        pix_bits = std::max(pix_bits, drt::screen_key_bits(s->W, s->H));
      }
      float_off += drt::partial_floats(d.rows_i + d.blocks_e);
    }
    for (int p = 0; p < drt::kPhases; ++p)
      b->prefix[(size_t)p * (n + 1) + k + 1] = b->prefix[(size_t)p * (n + 1) + k] + cnt[p];
    b->eprefix[k + 1] = b->eprefix[k] + d.n_edge;
    if (bind) {
      d.tape_tri = b->tape_tri + tape_here;
      d.tape_bary = b->tape_bary + tape_here;
      if (it.d_image) d.partials = b->partials + float_here;
    }
  }
  int sb = 0;
  while ((1 << sb) < n) ++sb;
  // the scene index goes above the screen key; drop low screen bits (a
  // coarser sample order) if both do not fit in 32 bits
  b->key_shift = std::max(0, pix_bits + sb - 32);
  b->pix_bits = pix_bits - b->key_shift;
  b->key_bits = b->pix_bits + sb;
  b->total_edge = b->eprefix[n];
  b->total_tape = tape_off;
  b->total_floats = float_off;
  b->total_sec = sec_off;
  for (int p = 0; p < drt::kPhases; ++p) b->n_items[p] = b->prefix[(size_t)p * (n + 1) + n];
  if (bind) {
    // the sort leaves its result in vals2 after an odd number of 8-bit passes
    const bool alt = ((b->key_bits + 7) / 8) % 2 == 1;
    int32_t* sorted = alt ? b->vals2 : b->vals;
    for (int k = 0; k < n; ++k)
      if (b->desc[k].n_edge > 0) b->desc[k].order = sorted + b->eprefix[k];
  }
}

drt_status upload_plan(drt_batch* b) {
  BATCH_CUDA(cudaMemcpy(b->d_desc, b->desc.data(), sizeof(BatchScene) * b->n, cudaMemcpyHostToDevice));
  BATCH_CUDA(cudaMemcpy(b->d_prefix, b->prefix.data(), sizeof(int64_t) * b->prefix.size(), cudaMemcpyHostToDevice));
  BATCH_CUDA(cudaMemcpy(b->d_eprefix, b->eprefix.data(), sizeof(int64_t) * b->eprefix.size(),
                        cudaMemcpyHostToDevice));
  if (b->d_desc_tune) {
    std::vector<BatchScene> t = b->desc;
    for (auto& d : t) {
      if (d.d_verts) d.d_verts = b->scratch;
      if (d.d_albedo) d.d_albedo = b->scratch;
    }
    BATCH_CUDA(cudaMemcpy(b->d_desc_tune, t.data(), sizeof(BatchScene) * b->n, cudaMemcpyHostToDevice));
  }
  return DRT_OK;
}

int grid_of(const drt_batch* b, int phase) {
  int per_sm = std::max(1, std::min(b->shape.ctas[phase], b->occupancy[phase]));
  int64_t g = (int64_t)b->ctx->num_sms * per_sm;
  int64_t need = (b->n_items[phase] + b->shape.chunk[phase] - 1) / b->shape.chunk[phase];
  return (int)std::max<int64_t>(1, std::min(g, need));
}

cudaError_t run_phase(drt_batch* b, int phase, const BatchScene* desc, cudaStream_t st) {
  return drt::launch_batch_phase(phase, desc, b->d_prefix + (size_t)phase * (b->n + 1), b->n, b->n_items[phase],
                                 grid_of(b, phase), b->shape.chunk[phase], b->d_counter + phase, st);
}

cudaError_t sort_edges(drt_batch* b, const BatchScene* desc, cudaStream_t st) {
  if (b->total_edge <= 0) return cudaSuccess;
  cudaError_t e = drt::launch_batch_keys(desc, b->d_eprefix, b->n, b->total_edge, b->pix_bits, b->key_shift, b->keys,
                                         b->vals, st);
  if (e != cudaSuccess) return e;
  drt::radix_sort_pairs(b->keys, b->vals, b->keys2, b->vals2, b->hist, b->hist_tmp, (int)b->total_edge,
                        b->key_bits, st);
  return cudaGetLastError();
}

// One step on stream st.
cudaError_t enqueue(drt_batch* b, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < b->n && e == cudaSuccess; ++k) {
    const drt_batch_item& it = b->items[k];
    if (!it.verts) continue;
    drt_scene* s = it.scene;
    e = cudaMemcpyAsync(s->verts, it.verts, 12 * (size_t)s->V, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = drt::check_finite(s, st);
    if (e == cudaSuccess) e = drt::build_scene_derived(s, st);
  }
  if (e == cudaSuccess) e = run_phase(b, drt::kPhaseRender, b->d_desc, st);
  if (b->total_sec > 0) {
    if (e == cudaSuccess) e = cudaMemsetAsync(b->sec_dp, 0, sizeof(float) * 3 * (size_t)b->total_sec, st);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(b->sec_counts, 0, sizeof(unsigned long long) * b->n * drt::kSecCounters, st);
    for (int k = 0; k < b->n && e == cudaSuccess; ++k)
      if (b->desc[k].dp_sec) e = drt::launch_secondary_apart(b->desc[k], st);
  }
  if (e == cudaSuccess) e = run_phase(b, drt::kPhasePath, b->d_desc, st);
  if (e == cudaSuccess) e = run_phase(b, drt::kPhaseInterior, b->d_desc, st);
  if (e == cudaSuccess) e = sort_edges(b, b->d_desc, st);
  if (e == cudaSuccess) e = run_phase(b, drt::kPhasePrimary, b->d_desc, st);
  for (int k = 0; k < b->n && e == cudaSuccess; ++k) {
    const BatchScene& d = b->desc[k];
    if (d.d_image)
      e = drt::launch_reduce_globals(d.partials, d.rows_i + d.blocks_e, d.d_radiance, d.d_cam, d.d_scale, st);
  }
  return e;
}

// Device time of one launch of a pass (milliseconds), median of three.
float time_phase(drt_batch* b, int phase, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  float t[3];
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0, st);
    run_phase(b, phase, b->d_desc_tune, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    t[r] = 0.f;
    cudaEventElapsedTime(&t[r], e0, e1);
  }
  std::sort(t, t + 3);
  return t[1];
}

drt_status autotune(drt_batch* b, cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  cudaEvent_t e0, e1;
  BATCH_CUDA(cudaEventCreate(&e0));
  BATCH_CUDA(cudaEventCreate(&e1));
  // tapes and the screen order must exist before the backward probes
  cudaError_t err = run_phase(b, drt::kPhaseRender, b->d_desc_tune, st);
  if (err == cudaSuccess) err = sort_edges(b, b->d_desc_tune, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  for (int p = 0; p < drt::kPhases && err == cudaSuccess; ++p) {
    if (b->n_items[p] == 0) continue;
    int best_c = 1;
    float best = 1e30f;
    for (int c = 1; c <= std::min(4, b->occupancy[p]); ++c) {
      b->shape.ctas[p] = c;
      b->shape.chunk[p] = 1;
      float t = time_phase(b, p, st, e0, e1);
      if (t < best) best = t, best_c = c;
    }
    b->shape.ctas[p] = best_c;
    int best_k = 1;
    for (int k : {2, 4, 8}) {
      b->shape.chunk[p] = k;
      float t = time_phase(b, p, st, e0, e1);
      if (t < best) best = t, best_k = k;
    }
    b->shape.chunk[p] = best_k;
    if (p == drt::kPhasePrimary) {
      int best_m = 1;
      for (int m : {2, 4}) {
        b->shape.edge_mult = m;
        plan(b, true);
        drt_status s = upload_plan(b);
        if (s != DRT_OK) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return s;
        }
        float t = time_phase(b, p, st, e0, e1);
        if (t < best) best = t, best_m = m;
      }
      b->shape.edge_mult = best_m;
      plan(b, true);
      drt_status s = upload_plan(b);
      if (s != DRT_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return s;
      }
    }
    err = cudaGetLastError();
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return bfail(DRT_ERR_CUDA, cudaGetErrorString(err));
  b->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  b->tuned = true;
  return DRT_OK;
}

TuneKey tune_key(const drt_batch* b) {
  int64_t pix = 0;
  for (const auto& it : b->items) pix += (int64_t)it.scene->W * it.scene->H;
  return TuneKey(b->ctx->device, b->n, pix, b->total_edge, b->op.spp, b->op.edge_spp, b->op.max_depth, b->op.terms);
}

void free_batch(drt_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  void* bufs[] = {b->d_desc, b->d_desc_tune, b->d_prefix, b->d_eprefix, b->d_counter, b->tape_tri, b->tape_bary,
                  b->partials, b->scratch, b->keys, b->keys2, b->hist, b->hist_tmp, b->vals, b->vals2,
                  b->sec_dp, b->sec_queue, b->sec_counts};
  for (void* p : bufs) drt::device_free(p);
  delete b;
}

template <class T>
drt_status balloc(T** p, size_t n) {
  return drt::device_alloc(reinterpret_cast<void**>(p), std::max<size_t>(1, n) * sizeof(T));
}

// A run that copies in new vertices changes those scenes: tapes and derived
// tables built for the old vertices no longer apply.
void bump_generations(drt_batch* b) {
  for (const auto& it : b->items)
    if (it.verts) ++it.scene->generation;
}

}  // namespace

extern "C" {

drt_status drt_batch_create(drt_context* ctx, const drt_batch_item* items, int32_t n, const drt_render_opts* opts,
                            int32_t use_graph, int32_t autotune, drt_batch** out) {
  if (!ctx || !items || !opts || !out) return bfail(DRT_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (n < 1 || n > kMaxBatch) return bfail(DRT_ERR_INVALID_ARG, "a batch holds 1 to 65536 scenes");
  drt::Opts op;
  BATCH_TRY(drt::convert_opts(opts, &op));
  if (op.proposal != 0) return bfail(DRT_ERR_INVALID_ARG, "a batch samples primary edges by length (proposal 0)");
  if (op.sec_sampler != 0) return bfail(DRT_ERR_INVALID_ARG, "a batch samples secondary edges by length (sec_sampler 0)");
  if (op.sec_point != 0) return bfail(DRT_ERR_INVALID_ARG, "a batch samples the point on a secondary edge uniformly (sec_point 0)");
  if (op.nee != 0) return bfail(DRT_ERR_INVALID_ARG, "a batch takes no next-event estimation for edges (sec_nee 0)");
  if (opts->spp_per_pass > 0 && opts->spp_per_pass < opts->spp)
    return bfail(DRT_ERR_INVALID_ARG, "a batch takes one sample pass (spp_per_pass 0)");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx->device)
    return bfail(DRT_ERR_STATE, "the context's device must be the current device");
  int64_t max_v = 1, max_t = 1;
  for (int k = 0; k < n; ++k) {
    const drt_batch_item& it = items[k];
    if (!it.scene || !it.image) return bfail(DRT_ERR_INVALID_ARG, "every batch item needs a scene and an image");
    if (it.grads.dimage_dparam || it.grads.n_jac != 0)
      return bfail(DRT_ERR_INVALID_ARG, "a batch writes no per-pixel gradient image");
    if (it.scene->cam_type == DRT_CAMERA_FISHEYE)
      return bfail(DRT_ERR_INVALID_ARG, "a batch takes pinhole and orthographic cameras");
    const void* arrays[] = {it.image, it.d_image, it.grads.d_verts, it.grads.d_albedo, it.grads.d_radiance,
                            it.grads.d_cam_to_world, it.grads.d_cam_scale, it.verts};
    for (const void* a : arrays)
      if (a && !drt::is_device_array(a)) return bfail(DRT_ERR_INVALID_ARG, "a batch takes device arrays only");
    max_v = std::max<int64_t>(max_v, it.scene->V);
    max_t = std::max<int64_t>(max_t, it.scene->T);
  }
  drt_batch* b = new drt_batch();
  b->ctx = ctx;
  b->n = n;
  b->items.assign(items, items + n);
  b->op = op;
  b->use_graph = use_graph != 0;
  b->autotune = autotune != 0;
  for (int p = 0; p < drt::kPhases; ++p) b->occupancy[p] = drt::batch_phase_occupancy(p);
  plan(b, false);  // totals at the largest edge budget
  if (b->total_edge > (int64_t)INT32_MAX || b->key_bits > 32) {
    free_batch(b);
    return bfail(DRT_ERR_INVALID_ARG, "batch too large: more than 2^31 primary edge samples");
  }
  drt_status s = balloc(&b->d_desc, n);
  if (s == DRT_OK && b->autotune) s = balloc(&b->d_desc_tune, n);
  if (s == DRT_OK && b->autotune) s = balloc(&b->scratch, 3 * (size_t)std::max(max_v, max_t));
  if (s == DRT_OK) s = balloc(&b->d_prefix, (size_t)drt::kPhases * (n + 1));
  if (s == DRT_OK) s = balloc(&b->d_eprefix, (size_t)n + 1);
  if (s == DRT_OK) s = balloc(&b->d_counter, drt::kPhases);
  if (s == DRT_OK) s = balloc(&b->tape_tri, (size_t)b->total_tape);
  if (s == DRT_OK) s = balloc(&b->tape_bary, (size_t)b->total_tape);
  if (s == DRT_OK) s = balloc(&b->partials, (size_t)b->total_floats);
  if (s == DRT_OK && b->total_sec > 0) {
    s = balloc(&b->sec_dp, 3 * (size_t)b->total_sec);
    if (s == DRT_OK) s = balloc(&b->sec_queue, (size_t)b->total_sec);
    if (s == DRT_OK) s = balloc(&b->sec_counts, (size_t)b->n * drt::kSecCounters);
  }
  size_t ne = (size_t)b->total_edge;
  if (s == DRT_OK && ne > 0) {
    s = balloc(&b->keys, ne);
    if (s == DRT_OK) s = balloc(&b->keys2, ne);
    if (s == DRT_OK) s = balloc(&b->vals, ne);
    if (s == DRT_OK) s = balloc(&b->vals2, ne);
    if (s == DRT_OK) s = balloc(&b->hist, drt::radix_hist_entries((int)ne));
    if (s == DRT_OK) s = balloc(&b->hist_tmp, drt::radix_hist_tmp_entries((int)ne));
  }
  if (s == DRT_OK) {
    auto hit = g_tuned.find(tune_key(b));
    if (hit != g_tuned.end()) {
      b->shape = hit->second;
      b->tuned = true;
    }
    plan(b, true);
    s = upload_plan(b);
  }
  if (s != DRT_OK) {
    free_batch(b);
    return s;
  }
  *out = b;
  return DRT_OK;
}

drt_status drt_batch_run(drt_context* ctx, drt_batch* b, void* stream) {
  NvtxRange nvtx_range("drt_batch_run");
  if (!ctx || !b || b->ctx != ctx) return bfail(DRT_ERR_INVALID_ARG, "NULL or foreign batch");
  cudaStream_t st = (cudaStream_t)stream;
  if (b->autotune && !b->tuned) {
    BATCH_TRY(autotune(b, st));
    g_tuned[tune_key(b)] = b->shape;
  }
  if (!b->use_graph) {
    BATCH_CUDA(enqueue(b, st));
    ++b->runs;
    bump_generations(b);
    return DRT_OK;
  }
  if (!b->exec) {
    BATCH_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    BATCH_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue(b, b->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      char m[256];
      std::snprintf(m, sizeof(m), "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
      return bfail(DRT_ERR_CUDA, m);
    }
    b->graph = g;
    BATCH_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  }
  BATCH_CUDA(cudaGraphLaunch(b->exec, st));
  ++b->runs;
  bump_generations(b);
  return DRT_OK;
}

drt_status drt_batch_get_info(drt_context* ctx, const drt_batch* b, drt_batch_info* info) {
  if (!ctx || !b || !info) return bfail(DRT_ERR_INVALID_ARG, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  for (int p = 0; p < drt::kPhases; ++p) {
    info->ctas_per_sm[p] = std::max(1, std::min(b->shape.ctas[p], b->occupancy[p]));
    info->chunk[p] = b->shape.chunk[p];
    info->items[p] = b->n_items[p];
    info->grid[p] = b->n_items[p] > 0 ? grid_of(b, p) : 0;
  }
  info->edge_per_thread_mult = b->shape.edge_mult;
  info->graph = b->exec != nullptr;
  info->tuned = b->tuned;
  info->edge_samples = b->total_edge;
  info->tune_ms = b->tune_ms;
  return DRT_OK;
}

drt_status drt_batch_free(drt_context* ctx, drt_batch* b) {
  if (!ctx) return bfail(DRT_ERR_INVALID_ARG, "NULL context");
  if (!b) return DRT_OK;
  cudaDeviceSynchronize();  // runs may still use the batch's buffers
  free_batch(b);
  return DRT_OK;
}

drt_status drt_render_batch(drt_context* ctx, drt_scene* const* scenes, int32_t n, const drt_render_opts* opts,
                            float* const* images, const float* const* d_images, const drt_grads* grads,
                            void* stream) {
  NvtxRange nvtx_range("drt_render_batch");
  if (!ctx || !scenes || !images || !opts) return bfail(DRT_ERR_INVALID_ARG, "NULL argument");
  if (n < 1 || n > kMaxBatch) return bfail(DRT_ERR_INVALID_ARG, "a batch holds 1 to 65536 scenes");
  std::vector<drt_batch_item> items((size_t)n);
  for (int k = 0; k < n; ++k) {
    std::memset(&items[k], 0, sizeof(drt_batch_item));
    items[k].scene = scenes[k];
    items[k].image = images[k];
    items[k].d_image = d_images ? d_images[k] : nullptr;
    if (grads) items[k].grads = grads[k];
  }
  drt_batch* b = nullptr;
  BATCH_TRY(drt_batch_create(ctx, items.data(), n, opts, 0, 0, &b));
  drt_status s = drt_batch_run(ctx, b, stream);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  free_batch(b);
  if (s != DRT_OK) return s;
  if (e != cudaSuccess) return bfail(DRT_ERR_CUDA, cudaGetErrorString(e));
  return DRT_OK;
}

}  // extern "C"
