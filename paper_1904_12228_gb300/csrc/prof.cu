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
