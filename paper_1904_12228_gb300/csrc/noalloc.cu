// noalloc.cu -- a backward pass that allocates no memory.
//
// drt_render_backward keeps its scratch (one row of per-block partial sums of
// the global parameters per thread block, the screen sort of the primary edge
// samples, the queue of secondary edge samples) in scene-owned buffers that it
// grows with cudaMalloc, and copies host arrays through temporary device
// buffers.  Some callers cannot allow an allocation inside their step: a
// training or serving loop that reserved the device memory up front through
// its own caching allocator (a cudaMalloc there can fail, or make the cache
// give memory back and stall), or a process that runs under a fixed device
// memory budget.  drt_render_backward_noalloc serves them: its scratch lives
// in a fixed-size array compiled into this library, and it accepts device
// arrays only.  Without scratch for them, it evaluates the primary edge
// samples in sample order and the secondary edge samples inside the pixel
// passes (same arithmetic, other order of the floating-point sums).
#include <atomic>
#include <climits>
#include <cstdint>
#include <cstdio>

#include "drt_internal.h"
#include "edge_tree.cuh"

namespace {

// Capacity of the scratch: 2^22 floats = 16 MiB, about 2^18 partial-sum rows
// of 16 floats (one row per thread block of the pixel passes and of the
// primary edge pass) plus their stage-1 totals.  A 512x512 image at 64 spp
// and 64 edge samples per pixel needs 32768 + 65536 rows.
constexpr int64_t kNoAllocMaxFloats = int64_t(1) << 22;

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) float g_backward_scratch[kNoAllocMaxFloats];

// Device address of the array per device, looked up again on every call made
// outside stream capture (so a device whose primary context was destroyed and
// created again gets the new address); during capture the last address is
// used, which is why the first call on a device must come before any capture.
constexpr int kMaxDevices = 64;
std::atomic<float*> g_scratch_addr[kMaxDevices];

bool is_device_array(const void* p) {
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

drt_status fail_noalloc(drt_status st, const char* msg) {
  drt::set_last_error(msg);
  return st;
}

}  // namespace

extern "C" {

drt_status drt_render_backward_noalloc(drt_context* ctx, drt_scene* s, const drt_tape* tape,
                                       const drt_render_opts* opts, const float* d_image, const drt_grads* grads,
                                       void* stream) {
  NvtxRange nvtx_range("drt_render_backward_noalloc");
  if (!ctx || !s || !opts || !d_image || !grads) {
    return fail_noalloc(DRT_ERR_INVALID_ARG, "NULL argument");
  }
  drt::Opts op;
  // the option checks and defaults of drt_render_backward
  drt_status so = drt::convert_opts(opts, &op);
  if (so != DRT_OK) return so;
  if (opts->proposal != 0) return fail_noalloc(DRT_ERR_INVALID_ARG, "drt_render_backward_noalloc supports proposal 0");
  if (opts->sec_nee != 0)
    return fail_noalloc(DRT_ERR_INVALID_ARG, "drt_render_backward_noalloc supports sec_nee 0 (it has no queue)");
  if (opts->spp_per_pass > 0 && opts->spp_per_pass < opts->spp)
    return fail_noalloc(DRT_ERR_INVALID_ARG, "drt_render_backward_noalloc takes one sample pass (spp_per_pass 0)");
  op.proposal = 0;
  op.seg_log = nullptr;
  if (!op.primary_only && op.max_depth > 1 && (op.terms & 5) && !tape) {
    return fail_noalloc(DRT_ERR_INVALID_ARG,
                        "interior or secondary terms with max_depth > 1 need the tape of the forward pass");
  }
  if (tape) {
    const drt_render_opts& t = tape->opts;
    if (tape->scene != s || tape->generation != s->generation || t.spp != opts->spp || t.seed != opts->seed ||
        t.max_depth != opts->max_depth || (t.primary_only != 0) != (opts->primary_only != 0)) {
      return fail_noalloc(DRT_ERR_STATE, "tape does not match this scene and these options");
    }
  }
  if (grads->dimage_dparam || grads->n_jac != 0) {
    return fail_noalloc(DRT_ERR_INVALID_ARG, "drt_render_backward_noalloc writes no per-pixel gradient image");
  }
  const void* arrays[] = {d_image, grads->d_verts, grads->d_albedo, grads->d_radiance, grads->d_cam_to_world,
                          grads->d_cam_scale};
  for (const void* a : arrays)
    if (!is_device_array(a)) {
      return fail_noalloc(DRT_ERR_INVALID_ARG, "drt_render_backward_noalloc takes device arrays only");
    }
  int64_t rows = drt::backward_partial_rows(s, op);
  if (drt::partial_floats(rows) > kNoAllocMaxFloats) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "image too large for the fixed scratch: needs %lld floats, maximum %lld",
                  (long long)drt::partial_floats(rows), (long long)kNoAllocMaxFloats);
    return fail_noalloc(DRT_ERR_INVALID_ARG, buf);
  }
  // the device address of the array (a host-side name is not a device address)
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices || dev != ctx->device) {
    return fail_noalloc(DRT_ERR_STATE, "the context's device must be the current device");
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusNone;
  }
  float* scratch = g_scratch_addr[dev].load();
  if (cs == cudaStreamCaptureStatusNone || !scratch) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_backward_scratch);
    if (e != cudaSuccess || !p) {
      return fail_noalloc(DRT_ERR_CUDA, cudaGetErrorString(e));
    }
    scratch = static_cast<float*>(p);
    g_scratch_addr[dev].store(scratch);
  }
  // the edge hierarchy's buffers come from an earlier backward; a scene that
  // changed since is rebuilt in place (kernel launches only)
  if (op.sec_sampler == 1 && !op.primary_only && (op.terms & 4) && s->E > 0 && s->L > 0) {
    if (!s->et_leaf) {
      return fail_noalloc(DRT_ERR_STATE, "the edge hierarchy is not allocated: run one drt_render_backward with it first");
    }
    if (s->et_generation != s->generation || s->et_spatial) {
      cudaError_t eb = drt::build_edge_tree(s, (cudaStream_t)stream, false);
      if (eb != cudaSuccess) return fail_noalloc(DRT_ERR_CUDA, cudaGetErrorString(eb));
      s->et_generation = s->generation;
      s->et_spatial = false;
    }
  }
  cudaError_t e = drt::launch_backward(s, op, tape, d_image, grads->d_verts, grads->d_albedo, grads->d_radiance,
                                       grads->d_cam_to_world, grads->d_cam_scale, scratch,
                                       nullptr, nullptr, nullptr, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    return fail_noalloc(DRT_ERR_CUDA, cudaGetErrorString(e));
  }
  return DRT_OK;
}

}  // extern "C"
