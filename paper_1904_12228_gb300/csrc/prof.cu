// prof.cu -- per-kernel timing with CUDA events recorded on the launching
// stream, and per-kernel work counters.  Off by default; enabled through
// drt_profile_enable / drt_counters_enable.
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "drt_internal.h"

namespace drt {
namespace {

struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
bool g_prof = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

bool g_count = false;
unsigned long long* g_counters = nullptr;  // [kKernelSlots * 4]

}  // namespace

ProfToken prof_begin(const char* name, cudaStream_t st) {
  ProfToken t{nullptr, nullptr, nullptr};
  if (!g_prof) return t;
  // launches recorded into a CUDA graph are not timed per launch
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return t;
  }
  if (cs != cudaStreamCaptureStatusNone) return t;
  t.name = name;
  t.a = get_event();
  t.b = get_event();
  cudaEventRecord(t.a, st);
  return t;
}

void prof_end(const ProfToken& t, cudaStream_t st) {
  if (!t.name) return;
  cudaEventRecord(t.b, st);
  g_recs.push_back(Rec{t.name, t.a, t.b});
}

unsigned long long* counter_slot(int kernel) {
  if (!g_count || !g_counters) return nullptr;
  return g_counters + 4 * kernel;
}

}  // namespace drt

extern "C" {

drt_status drt_profile_enable(drt_context* ctx, int enable) {
  if (!ctx) return DRT_ERR_INVALID_ARG;
  drt::g_prof = enable != 0;
  return DRT_OK;
}

drt_status drt_profile_read(drt_context* ctx, int max, char* names, double* ms, int64_t* launches, int* n) {
  if (!ctx || !n || max < 0) return DRT_ERR_INVALID_ARG;
  std::map<std::string, std::pair<double, int64_t>> acc;
  std::vector<std::string> order;
  for (auto& r : drt::g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return DRT_ERR_CUDA;
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    if (!acc.count(r.name)) order.push_back(r.name);
    acc[r.name].first += t;
    acc[r.name].second += 1;
    drt::g_pool.push_back(r.a);
    drt::g_pool.push_back(r.b);
  }
  drt::g_recs.clear();
  int k = 0;
  for (auto& nm : order) {
    if (k >= max) break;
    if (names) {
      std::strncpy(names + 64 * k, nm.c_str(), 63);
      names[64 * k + 63] = 0;
    }
    if (ms) ms[k] = acc[nm].first;
    if (launches) launches[k] = acc[nm].second;
    ++k;
  }
  *n = k;
  return DRT_OK;
}

drt_status drt_counters_enable(drt_context* ctx, int enable) {
  if (!ctx) return DRT_ERR_INVALID_ARG;
  if (enable && !drt::g_counters) {
    if (cudaMalloc(&drt::g_counters, sizeof(unsigned long long) * 4 * drt::kKernelSlots) != cudaSuccess)
      return DRT_ERR_OOM;
    cudaMemset(drt::g_counters, 0, sizeof(unsigned long long) * 4 * drt::kKernelSlots);
  }
  drt::g_count = enable != 0;
  return DRT_OK;
}

drt_status drt_counters_read(drt_context* ctx, int64_t* out) {
  if (!ctx || !out) return DRT_ERR_INVALID_ARG;
  if (!drt::g_counters) {
    std::memset(out, 0, sizeof(int64_t) * 4 * drt::kKernelSlots);
    return DRT_OK;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return DRT_ERR_CUDA;
  cudaMemcpy(out, drt::g_counters, sizeof(int64_t) * 4 * drt::kKernelSlots, cudaMemcpyDeviceToHost);
  cudaMemset(drt::g_counters, 0, sizeof(unsigned long long) * 4 * drt::kKernelSlots);
  return DRT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// On-box peak probes: the denominators of the ray kernels' rooflines.  The
// traversal and shading kernels are bound by FP32/INT issue slots and by
// L1/L2 bandwidth, not by HBM or tensor cores, so the two peaks measured here
// are (1) the FP32 FMA lane-operation rate of a kernel with ample independent
// work per thread, and (2) the L2 bandwidth of a copy whose working set fits
// in L2, loads and stores bypassing L1 (.cg).
// ---------------------------------------------------------------------------
namespace drt {
namespace {

constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(256) k_probe_fma(float* out, int iters, float a, float b) {
  float x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = 1e-3f * (float)(threadIdx.x + c);
#pragma unroll 16
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += x[c];
  if (s == -1.2345f) out[blockIdx.x] = s;  // keeps the chains live; never true for these inputs
}

// passes alternate the direction (x -> y, then y -> x), so every pass reads
// what the previous one wrote
__global__ void __launch_bounds__(256) k_probe_copy(float4* x, float4* y, int64_t n, int passes) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int p = 0; p < passes; ++p) {
    const float4* src = (p & 1) ? y : x;
    float4* dst = (p & 1) ? x : y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) __stcg(dst + i, __ldcg(src + i));
  }
}

// Best of `reps` event-timed launches of f on st, in ms.
template <class F>
cudaError_t best_ms(cudaStream_t st, int reps, F f, float* best) {
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&b);
  if (e != cudaSuccess) {
    cudaEventDestroy(a);
    return e;
  }
  *best = 1e30f;
  f();  // warm-up
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(a, st);
    if (e == cudaSuccess) f();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && ms < *best) *best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e;
}

}  // namespace
}  // namespace drt

extern "C" {

drt_status drt_probe_fma(drt_context* ctx, double* lane_ops_per_s, void* stream) {
  if (!ctx || !lane_ops_per_s) return DRT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DRT_ERR_CUDA;
  int blocks = ctx->num_sms * 8;  // 2048 resident threads per SM
  const int iters = 1 << 16;
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * blocks) != cudaSuccess) {
    cudaGetLastError();
    return DRT_ERR_OOM;
  }
  float ms = 0.f;
  cudaError_t e = drt::best_ms(st, 5, [&] {
    drt::k_probe_fma<<<blocks, 256, 0, st>>>(out, iters, 0.99999994f, 1e-7f);
  }, &ms);
  cudaFree(out);
  if (e != cudaSuccess) {
    drt::set_last_error(cudaGetErrorString(e));
    return DRT_ERR_CUDA;
  }
  double ops = (double)blocks * 256.0 * iters * drt::kProbeChains;
  *lane_ops_per_s = ops / (ms * 1e-3);
  return DRT_OK;
}

drt_status drt_probe_l2(drt_context* ctx, int64_t bytes, double* bytes_per_s, void* stream) {
  if (!ctx || !bytes_per_s || bytes < (1 << 20) || bytes > ((int64_t)1 << 30)) return DRT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DRT_ERR_CUDA;
  int64_t n = bytes / 2 / (int64_t)sizeof(float4);  // two buffers of n float4 each
  float4* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(float4) * 2 * (size_t)n) != cudaSuccess) {
    cudaGetLastError();
    return DRT_ERR_OOM;
  }
  cudaError_t e = cudaMemsetAsync(buf, 0, sizeof(float4) * 2 * (size_t)n, st);
  int blocks = ctx->num_sms * 8;
  const int passes = 64;
  float ms = 0.f;
  if (e == cudaSuccess)
    e = drt::best_ms(st, 5, [&] { drt::k_probe_copy<<<blocks, 256, 0, st>>>(buf, buf + n, n, passes); }, &ms);
  cudaFree(buf);
  if (e != cudaSuccess) {
    drt::set_last_error(cudaGetErrorString(e));
    return DRT_ERR_CUDA;
  }
  *bytes_per_s = 2.0 * (double)n * sizeof(float4) * passes / (ms * 1e-3);
  return DRT_OK;
}

}  // extern "C"
