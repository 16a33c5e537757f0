// mlp.cu -- the edge-proposal network on the 5th-generation tensor cores.
//
// A 3-layer MLP scores every screen-tile segment of the primary edges:
//   y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3,   x in R^32, hidden 64,
// BF16 weights and activations, FP32 accumulation.  The thesis importance-
// samples edges with a hierarchy and LTC bounds (Sec. 5.3.1); here a learned
// score takes that role, mixed with the length proposal so the estimator
// stays unbiased.
//
// Each CTA (128 threads) owns a tile of 128 rows.  Operands are staged in
// shared memory in the canonical K-major layout without swizzle: 8x8 BF16
// core matrices of 128 contiguous bytes, K-adjacent core matrices 128 B
// apart (LBO), 8-row groups (K/8)*128 B apart (SBO).  One thread issues
// tcgen05.mma (M=128, K=16 per instruction) into TMEM and commits to an
// mbarrier; all threads wait (bounded), then each warp reads its 32 TMEM
// lanes with tcgen05.ld.  Every wait has an iteration limit: on timeout the
// kernel raises the device error flag, frees its TMEM and returns.
#include <cmath>
#include <cstdint>
#include <vector>
#include <cuda_bf16.h>

#include "drt_internal.h"

namespace drt {
namespace {

constexpr int kRows = 128;
constexpr int kIn = 32;
constexpr int kHid = 64;
constexpr uint32_t kWaitLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (r, k) of an [R x K] K-major operand (no swizzle).
__device__ __forceinline__ uint32_t kmaj(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K)
// byte offset, stride (8-row group) byte offset, fixed version bits 46-48 =
// 0b001, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait on an mbarrier phase; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (uint32_t i = 0; i < kWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void st_bf16(uint8_t* base, uint32_t off, float x) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(x);
}

// Issue D[M=128 x N] (+)= A[128 x K] B[N x K]^T as K/16 MMAs from one thread.
__device__ __forceinline__ void gemm_issue(uint32_t d_tmem, uint32_t a_smem, uint32_t b_smem, int K, int N,
                                           bool accumulate_first) {
  uint32_t sbo = (uint32_t)(K >> 3) * 128u;
  uint32_t id = idesc_bf16(128, N);
  for (int ks = 0; ks < K / 16; ++ks) {
    uint64_t ad = sdesc(a_smem + ks * 256u, 128u, sbo);
    uint64_t bd = sdesc(b_smem + ks * 256u, 128u, sbo);
    mma_bf16(d_tmem, ad, bd, id, (ks > 0 || accumulate_first) ? 1u : 0u);
  }
}

struct MlpArgs {
  const __nv_bfloat16* x;  // [M, 32]
  const __nv_bfloat16* w1; // [64, 32]
  const float* b1;         // [64]
  const __nv_bfloat16* w2; // [64, 64]
  const float* b2;         // [64]
  const float* w3;         // [64]
  const float* b3;         // [1]
  int M;
  int* err;
};

// Forward: y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3.
// Dynamic shared memory is padded to kForwardSmem so at most 4 CTAs share an
// SM: 4 x 128 TMEM columns fit the 512 columns without a blocking alloc.
constexpr size_t kForwardSmem = 56 * 1024;
__global__ void __launch_bounds__(128) k_mlp_forward(MlpArgs a, float* y) {
  extern __shared__ __align__(1024) uint8_t fsm[];
  uint8_t* sA1 = fsm;                       // [128 x 32]
  uint8_t* sB1 = sA1 + kRows * kIn * 2;     // [64 x 32]
  uint8_t* sA2 = sB1 + kHid * kIn * 2;      // [128 x 64]
  uint8_t* sB2 = sA2 + kRows * kHid * 2;    // [64 x 64]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ int failed;
  int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int row0 = blockIdx.x * kRows;
  if (warp == 0) tmem_alloc(smem_u32(&tslot), 128);
  if (tid == 0) {
    mbar_init(smem_u32(&mbar), 1);
    failed = 0;
  }
  // stage X tile (zero rows past M) and the weights in the canonical layout
  for (int i = tid; i < kRows * kIn; i += 128) {
    int r = i / kIn, k = i % kIn;
    __nv_bfloat16 v = row0 + r < a.M ? a.x[(size_t)(row0 + r) * kIn + k] : __float2bfloat16_rn(0.f);
    *reinterpret_cast<__nv_bfloat16*>(sA1 + kmaj(r, k, kIn)) = v;
  }
  for (int i = tid; i < kHid * kIn; i += 128) *reinterpret_cast<__nv_bfloat16*>(sB1 + kmaj(i / kIn, i % kIn, kIn)) = a.w1[i];
  for (int i = tid; i < kHid * kHid; i += 128)
    *reinterpret_cast<__nv_bfloat16*>(sB2 + kmaj(i / kHid, i % kHid, kHid)) = a.w2[i];
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  uint32_t tmem = tslot;
  uint32_t mb = smem_u32(&mbar);
  // layer 1 into columns [0, 64)
  if (tid == 0) {
    gemm_issue(tmem, smem_u32(sA1), smem_u32(sB1), kIn, kHid, false);
    mma_commit(mb);
  }
  if (!mbar_wait(mb, 0)) failed = 1;
  tc_fence_after();
  __syncthreads();
  if (!failed) {
    int r = warp * 32 + lane;
    uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c = 0; c < kHid; c += 16) {
      float v[16];
      tmem_ld16(lane_addr + c, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) st_bf16(sA2, kmaj(r, c + i, kHid), fmaxf(v[i] + a.b1[c + i], 0.f));
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // layer 2 into columns [64, 128)
  if (!failed) {
    if (tid == 0) {
      gemm_issue(tmem + 64, smem_u32(sA2), smem_u32(sB2), kHid, kHid, false);
      mma_commit(mb);
    }
    if (!mbar_wait(mb, 1)) failed = 1;
    tc_fence_after();
  }
  __syncthreads();
  if (!failed) {
    int r = warp * 32 + lane;
    uint32_t lane_addr = tmem + 64 + ((uint32_t)(warp * 32) << 16);
    float acc = a.b3[0];
    for (int c = 0; c < kHid; c += 16) {
      float v[16];
      tmem_ld16(lane_addr + c, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) acc += a.w3[c + i] * fmaxf(v[i] + a.b2[c + i], 0.f);
    }
    if (row0 + r < a.M) y[row0 + r] = acc;
  } else if (tid == 0) {
    raise_flag(a.err, DRT_DEV_TIMEOUT, blockIdx.x);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 128);
}

// Backward of the mean-squared error L = 1/(2 n) sum_r mask_r (y_r - t_r)^2
// (n = number of masked rows, given): adds dL/dW1, db1, dW2, db2, dw3, db3
// into FP32 gradient buffers (atomics across CTAs).
__global__ void __launch_bounds__(128) k_mlp_backward(MlpArgs a, const float* target, const float* mask,
                                                      float inv_n, float* gw1, float* gb1, float* gw2, float* gb2,
                                                      float* gw3, float* gb3, float* loss) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sX = smem;                      // [128 x 32]     8 KB
  uint8_t* sXT = sX + 8192;                // [32 x 128]     8 KB
  uint8_t* sW1 = sXT + 8192;               // [64 x 32]      4 KB
  uint8_t* sW2 = sW1 + 4096;               // [64 x 64]      8 KB
  uint8_t* sW2T = sW2 + 8192;              // [64 x 64]      8 KB
  uint8_t* sH1 = sW2T + 8192;              // [128 x 64]    16 KB
  uint8_t* sH1T = sH1 + 16384;             // [64 x 128]    16 KB
  uint8_t* sD2 = sH1T + 16384;             // [128 x 64]    16 KB  dz2
  uint8_t* sD2T = sD2 + 16384;             // [128 x 128]   32 KB  dz2^T, rows 64..127 zero
  uint8_t* sD1T = sD2T + 32768;            // [128 x 128]   32 KB  dz1^T, rows 64..127 zero
  float* sRelu1 = reinterpret_cast<float*>(sD1T + 32768);  // [128 x 64] z1 > 0 mask as 0/1
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ int failed;
  __shared__ float red[4][kHid + 2];
  int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int row0 = blockIdx.x * kRows;
  int r = warp * 32 + lane;
  bool valid = row0 + r < a.M;
  if (warp == 0) tmem_alloc(smem_u32(&tslot), 256);
  if (tid == 0) {
    mbar_init(smem_u32(&mbar), 1);
    failed = 0;
  }
  for (int i = tid; i < kRows * kIn; i += 128) {
    int rr = i / kIn, k = i % kIn;
    __nv_bfloat16 v = row0 + rr < a.M ? a.x[(size_t)(row0 + rr) * kIn + k] : __float2bfloat16_rn(0.f);
    *reinterpret_cast<__nv_bfloat16*>(sX + kmaj(rr, k, kIn)) = v;
    *reinterpret_cast<__nv_bfloat16*>(sXT + kmaj(k, rr, kRows)) = v;
  }
  for (int i = tid; i < kHid * kIn; i += 128) *reinterpret_cast<__nv_bfloat16*>(sW1 + kmaj(i / kIn, i % kIn, kIn)) = a.w1[i];
  for (int i = tid; i < kHid * kHid; i += 128) {
    int o = i / kHid, k = i % kHid;
    *reinterpret_cast<__nv_bfloat16*>(sW2 + kmaj(o, k, kHid)) = a.w2[i];
    *reinterpret_cast<__nv_bfloat16*>(sW2T + kmaj(k, o, kHid)) = a.w2[i];
  }
  // zero the padding rows of the transposed dz operands
  for (int i = tid; i < 64 * kRows; i += 128) {
    int rr = 64 + i / kRows, k = i % kRows;
    *reinterpret_cast<__nv_bfloat16*>(sD2T + kmaj(rr, k, kRows)) = __float2bfloat16_rn(0.f);
    *reinterpret_cast<__nv_bfloat16*>(sD1T + kmaj(rr, k, kRows)) = __float2bfloat16_rn(0.f);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  uint32_t tmem = tslot, mb = smem_u32(&mbar);
  uint32_t lane_off = (uint32_t)(warp * 32) << 16;
  uint32_t phase = 0;
  auto run = [&](uint32_t d, uint8_t* A, uint8_t* B, int K, int N) {
    if (failed) return;
    if (tid == 0) {
      gemm_issue(d, smem_u32(A), smem_u32(B), K, N, false);
      mma_commit(mb);
    }
    if (!mbar_wait(mb, phase)) failed = 1;
    phase ^= 1u;
    tc_fence_after();
  };
  // forward: z1 -> cols [0,64)
  run(tmem, sX, sW1, kIn, kHid);
  __syncthreads();
  if (!failed)
    for (int c = 0; c < kHid; c += 16) {
      float v[16];
      tmem_ld16(tmem + lane_off + c, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        float z = v[i] + a.b1[c + i];
        float h = fmaxf(z, 0.f);
        sRelu1[r * kHid + c + i] = z > 0.f ? 1.f : 0.f;
        st_bf16(sH1, kmaj(r, c + i, kHid), h);
        st_bf16(sH1T, kmaj(c + i, r, kRows), h);
      }
    }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // z2 -> cols [64,128)
  run(tmem + 64, sH1, sW2, kHid, kHid);
  __syncthreads();
  // per-row output, loss and dz2
  float dy = 0.f, gw3l[kHid];
  if (!failed) {
    float z2[kHid];
    for (int c = 0; c < kHid; c += 16) {
      float v[16];
      tmem_ld16(tmem + 64 + lane_off + c, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) z2[c + i] = v[i] + a.b2[c + i];
    }
    float y = a.b3[0];
    for (int j = 0; j < kHid; ++j) y += a.w3[j] * fmaxf(z2[j], 0.f);
    float m = valid ? mask[row0 + r] : 0.f;
    float e = y - (valid ? target[row0 + r] : 0.f);
    dy = m * e * inv_n;
    if (valid && m != 0.f) atomicAdd(loss, 0.5f * m * e * e * inv_n);
    for (int j = 0; j < kHid; ++j) {
      float h2 = fmaxf(z2[j], 0.f);
      gw3l[j] = dy * h2;
      float dz = z2[j] > 0.f ? dy * a.w3[j] : 0.f;
      st_bf16(sD2, kmaj(r, j, kHid), dz);
      st_bf16(sD2T, kmaj(j, r, kRows), dz);
      z2[j] = dz;
    }
    // block sums of dw3, db3, db2 via warp shuffles then shared memory
    for (int j = 0; j < kHid; ++j) {
      float s3 = gw3l[j], s2 = z2[j];
      for (int o = 16; o > 0; o >>= 1) {
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      }
      if (lane == 0) {
        red[warp][j] = s3;
        atomicAdd(gb2 + j, s2);
      }
    }
    float sd = dy;
    for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
    if (lane == 0) red[warp][kHid] = sd;
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (!failed && tid < kHid) atomicAdd(gw3 + tid, red[0][tid] + red[1][tid] + red[2][tid] + red[3][tid]);
  if (!failed && tid == kHid) atomicAdd(gb3, red[0][kHid] + red[1][kHid] + red[2][kHid] + red[3][kHid]);
  // dh1 = dz2 W2 -> cols [0,64); dW2 = dz2^T h1 -> cols [128,192)
  run(tmem, sD2, sW2T, kHid, kHid);
  run(tmem + 128, sD2T, sH1T, kRows, kHid);
  __syncthreads();
  if (!failed) {
    for (int c = 0; c < kHid; c += 16) {
      float v[16];
      tmem_ld16(tmem + lane_off + c, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        float dz1 = v[i] * sRelu1[r * kHid + c + i];
        st_bf16(sD1T, kmaj(c + i, r, kRows), dz1);
        float s1 = dz1;
        for (int o = 16; o > 0; o >>= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        if (lane == 0) atomicAdd(gb1 + c + i, s1);
      }
    }
    if (warp < 2)  // TMEM lanes 0..63 hold dW2 rows
      for (int c = 0; c < kHid; c += 16) {
        float v[16];
        tmem_ld16(tmem + 128 + lane_off + c, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) atomicAdd(gw2 + r * kHid + c + i, v[i]);
      }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // dW1 = dz1^T x -> cols [192,224)
  run(tmem + 192, sD1T, sXT, kRows, kIn);
  __syncthreads();
  if (!failed && warp < 2)
    for (int c = 0; c < kIn; c += 16) {
      float v[16];
      tmem_ld16(tmem + 192 + lane_off + c, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) atomicAdd(gw1 + r * kIn + c + i, v[i]);
    }
  if (failed && tid == 0) raise_flag(a.err, DRT_DEV_TIMEOUT, blockIdx.x);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

// Adam (Kingma & Ba, with bias correction) on FP32 master parameters; the
// BF16 copies used by the tensor cores are refreshed in the same pass.
__global__ void k_adam(float* p, const float* g, float* m, float* v, __nv_bfloat16* p_bf16, int n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  if (p_bf16) p_bf16[i] = __float2bfloat16_rn(pi);
}

constexpr size_t kBackwardSmem = 8192 * 2 + 4096 + 8192 * 2 + 16384 * 3 + 32768 * 2 + kRows * kHid * 4;

// ---- training from logged edge contributions (drt_mlp_train) --------------
// Network parameters in the order w1, b1, w2, b2, w3, b3.
constexpr int kNumParamArrays = 6;
constexpr int kParamTotal = kHid * kIn + kHid + kHid * kHid + kHid + kHid + 1;

struct ParamArrays {
  float* p[kNumParamArrays];
  float* m1[kNumParamArrays];
  float* m2[kNumParamArrays];
  float* g[kNumParamArrays];
  __nv_bfloat16* w1b;
  __nv_bfloat16* w2b;
};

__device__ __forceinline__ int param_slot(int i, int* off) {
  const int sizes[kNumParamArrays] = {kHid * kIn, kHid, kHid * kHid, kHid, kHid, 1};
  int a = 0;
#pragma unroll
  for (int k = 0; k < kNumParamArrays; ++k) {
    if (i < sizes[k]) {
      a = k;
      break;
    }
    i -= sizes[k];
  }
  *off = i;
  return a;
}

__global__ void k_zero_grads(ParamArrays pa) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kParamTotal) return;
  int off;
  int a = param_slot(i, &off);
  pa.g[a][off] = 0.f;
}

// Adam on all six arrays at once (same update as k_adam).
__global__ void k_adam_all(ParamArrays pa, float lr, float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kParamTotal) return;
  int off;
  int a = param_slot(i, &off);
  float gi = pa.g[a][off];
  float mi = b1 * pa.m1[a][off] + (1.f - b1) * gi;
  float vi = b2 * pa.m2[a][off] + (1.f - b2) * gi * gi;
  pa.m1[a][off] = mi;
  pa.m2[a][off] = vi;
  float pi = pa.p[a][off] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  pa.p[a][off] = pi;
  if (a == 0) pa.w1b[off] = __float2bfloat16_rn(pi);
  if (a == 2) pa.w2b[off] = __float2bfloat16_rn(pi);
}

// Per logged scene: sum of the logged magnitudes and of the segment lengths,
// in FP64, in a fixed order (one block per scene).
__global__ void k_log_sums(const drt_mlp_log* logs, double* sums) {
  __shared__ double sa[256], sb[256];
  const drt_mlp_log& lg = logs[blockIdx.x];
  double a = 0.0, b = 0.0;
  for (int64_t r = threadIdx.x; r < lg.n; r += blockDim.x) {
    a += (double)lg.seg_log[r];
    b += lg.seg_len[r];
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      sa[threadIdx.x] += sa[threadIdx.x + h];
      sb[threadIdx.x] += sb[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sums[2 * blockIdx.x] = sa[0];
    sums[2 * blockIdx.x + 1] = sb[0];
  }
}

// Shuffle keys: a Philox draw per row (counter (row, 0, 0x4D4C5054, 0), key =
// seed), sorted with the row index as value.
__global__ void k_shuffle_keys(int64_t rows, uint2 key, uint32_t* keys, int32_t* vals) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  keys[r] = philox(make_uint4((uint32_t)r, 0u, 0x4D4C5054u, 0u), key).x;
  vals[r] = (int32_t)r;
}

// Training row p = concatenated row perm[p]: its features, and the target
// and weight of the regression.  For a segment of length len with logged
// magnitude S out of N logging samples over screen length L, S L / N
// estimates the segment's integral of |w . (f_u - f_l)|; the target is the
// log of that integral per unit length relative to the scene's mean density
// (sum S / N over all segments per unit length), offset by delta; the
// weight is the segment's length over the scene's mean segment length.
__global__ void k_training_rows(const drt_mlp_log* logs, const int64_t* offs, int n_logs, const double* sums,
                                const int32_t* perm, int64_t rows, float delta, __nv_bfloat16* x, float* target,
                                float* mask, int64_t* index_out) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= rows) return;
  int64_t r = perm[p];
  int k = 0;
  while (k + 1 < n_logs && r >= offs[k + 1]) ++k;
  const drt_mlp_log& lg = logs[k];
  int64_t j = r - offs[k];
  double S = sums[2 * k], L = sums[2 * k + 1];
  double N = lg.n_samples;
  double len = lg.seg_len[j];
  double dens = (double)lg.seg_log[j] * (L / N) / fmax(len, 1e-12);
  double mean = S / N;
  double rel = dens / fmax(mean, 1e-30);
  target[p] = (float)log(rel + (double)delta);
  mask[p] = (float)(len / (L / (double)lg.n));
  const uint4* src = reinterpret_cast<const uint4*>(reinterpret_cast<const __nv_bfloat16*>(lg.x) + j * kIn);
  uint4* dst = reinterpret_cast<uint4*>(x + p * kIn);
#pragma unroll
  for (int q = 0; q < kIn * 2 / 16; ++q) dst[q] = src[q];
  if (index_out) index_out[p] = r;
}

}  // namespace
}  // namespace drt

extern "C" {

drt_status drt_mlp_forward(drt_context* ctx, const void* x, int64_t m, const drt_mlp_weights* w, float* y,
                           void* stream) {
  NvtxRange nvtx_range("drt_mlp_forward");
  if (!ctx || !w || (m > 0 && (!x || !y)) || m < 0 || m > INT32_MAX) return DRT_ERR_INVALID_ARG;
  if (m == 0) return DRT_OK;
  drt::MlpArgs a{(const __nv_bfloat16*)x, (const __nv_bfloat16*)w->w1, w->b1, (const __nv_bfloat16*)w->w2, w->b2,
                 w->w3, w->b3, (int)m, ctx->err};
  cudaStream_t st = (cudaStream_t)stream;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(drt::k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)drt::kForwardSmem) != cudaSuccess)
      return DRT_ERR_CUDA;
    attr = true;
  }
  unsigned g = (unsigned)((m + drt::kRows - 1) / drt::kRows);
  DRT_PROF_LAUNCH("mlp_forward", st, drt::k_mlp_forward<<<g, 128, drt::kForwardSmem, st>>>(a, y));
  return cudaGetLastError() == cudaSuccess ? DRT_OK : DRT_ERR_CUDA;
}

drt_status drt_mlp_backward(drt_context* ctx, const void* x, const float* target, const float* mask, int64_t m,
                            float inv_n, const drt_mlp_weights* w, drt_mlp_grads* g, float* loss, void* stream) {
  NvtxRange nvtx_range("drt_mlp_backward");
  if (!ctx || !w || !g || !loss || m < 0 || m > INT32_MAX || (m > 0 && (!x || !target || !mask)))
    return DRT_ERR_INVALID_ARG;
  if (m == 0) return DRT_OK;
  drt::MlpArgs a{(const __nv_bfloat16*)x, (const __nv_bfloat16*)w->w1, w->b1, (const __nv_bfloat16*)w->w2, w->b2,
                 w->w3, w->b3, (int)m, ctx->err};
  cudaStream_t st = (cudaStream_t)stream;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(drt::k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)drt::kBackwardSmem) != cudaSuccess)
      return DRT_ERR_CUDA;
    attr = true;
  }
  unsigned gr = (unsigned)((m + drt::kRows - 1) / drt::kRows);
  DRT_PROF_LAUNCH("mlp_backward", st, drt::k_mlp_backward<<<gr, 128, drt::kBackwardSmem, st>>>(
                                          a, target, mask, inv_n, g->w1, g->b1, g->w2, g->b2, g->w3, g->b3, loss));
  return cudaGetLastError() == cudaSuccess ? DRT_OK : DRT_ERR_CUDA;
}

drt_status drt_mlp_train(drt_context* ctx, const drt_mlp_log* logs, int32_t n_logs, const drt_mlp_train_opts* o,
                         drt_mlp_state* state, void* stream) {
  NvtxRange nvtx_range("drt_mlp_train");
  if (!ctx || !logs || n_logs < 1 || !o || !state || o->steps < 0 || o->batch < 0)
    return DRT_ERR_INVALID_ARG;
  for (int k = 0; k < drt::kNumParamArrays; ++k)
    if (!state->p[k] || !state->m1[k] || !state->m2[k] || !state->g[k]) return DRT_ERR_INVALID_ARG;
  if (!state->w1_bf16 || !state->w2_bf16 || state->step < 0) return DRT_ERR_INVALID_ARG;
  std::vector<int64_t> offs(n_logs + 1, 0);
  for (int k = 0; k < n_logs; ++k) {
    const drt_mlp_log& lg = logs[k];
    if (lg.n < 1 || !lg.x || !lg.seg_log || !lg.seg_len || !(lg.n_samples > 0.0)) {
      drt::set_last_error("drt_mlp_train: every log needs n >= 1 rows, its arrays and n_samples > 0");
      return DRT_ERR_INVALID_ARG;
    }
    if (!drt::is_device_array(lg.x) || !drt::is_device_array(lg.seg_log) || !drt::is_device_array(lg.seg_len)) {
      drt::set_last_error("drt_mlp_train: the logs' arrays must be device memory");
      return DRT_ERR_INVALID_ARG;
    }
    offs[k + 1] = offs[k] + lg.n;
  }
  int64_t rows = offs[n_logs];
  if (rows > INT32_MAX) {
    drt::set_last_error("drt_mlp_train: more than 2^31 - 1 rows");
    return DRT_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int batch = o->batch > 0 ? o->batch : 16384;
  if (batch > rows) batch = (int)rows;
  float lr = o->lr > 0.f ? o->lr : 3e-3f;
  float delta = o->delta > 0.f ? o->delta : 1e-3f;
  // scratch of this call (training is not a hot path): the logs' table, the
  // per-log sums, the shuffle and the training rows
  void *d_logs = nullptr, *d_offs = nullptr, *d_sums = nullptr, *keys = nullptr, *keys2 = nullptr, *vals = nullptr,
       *vals2 = nullptr, *hist = nullptr, *hist_tmp = nullptr, *x = nullptr, *target = nullptr, *mask = nullptr,
       *loss_tmp = nullptr;
  auto release = [&]() {
    void* all[] = {d_logs, d_offs, d_sums, keys, keys2, vals, vals2, hist, hist_tmp, x, target, mask, loss_tmp};
    for (void* q : all) drt::device_free(q);
  };
  drt_status a = drt::device_alloc(&d_logs, sizeof(drt_mlp_log) * n_logs);
  if (a == DRT_OK) a = drt::device_alloc(&d_offs, sizeof(int64_t) * (n_logs + 1));
  if (a == DRT_OK) a = drt::device_alloc(&d_sums, sizeof(double) * 2 * n_logs);
  if (a == DRT_OK) a = drt::device_alloc(&keys, sizeof(uint32_t) * rows);
  if (a == DRT_OK) a = drt::device_alloc(&keys2, sizeof(uint32_t) * rows);
  if (a == DRT_OK) a = drt::device_alloc(&vals, sizeof(int32_t) * rows);
  if (a == DRT_OK) a = drt::device_alloc(&vals2, sizeof(int32_t) * rows);
  if (a == DRT_OK) a = drt::device_alloc(&hist, sizeof(uint32_t) * drt::radix_hist_entries((int)rows));
  if (a == DRT_OK) a = drt::device_alloc(&hist_tmp, sizeof(uint32_t) * drt::radix_hist_tmp_entries((int)rows));
  if (a == DRT_OK) a = drt::device_alloc(&x, sizeof(__nv_bfloat16) * drt::kIn * rows);
  if (a == DRT_OK) a = drt::device_alloc(&target, sizeof(float) * rows);
  if (a == DRT_OK) a = drt::device_alloc(&mask, sizeof(float) * rows);
  if (a == DRT_OK && !o->loss) a = drt::device_alloc(&loss_tmp, sizeof(float));
  if (a != DRT_OK) {
    release();
    return a;
  }
  cudaError_t e = cudaMemcpyAsync(d_logs, logs, sizeof(drt_mlp_log) * n_logs, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_offs, offs.data(), sizeof(int64_t) * (n_logs + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && loss_tmp) e = cudaMemsetAsync(loss_tmp, 0, sizeof(float), st);
  if (e == cudaSuccess) {
    drt::k_log_sums<<<n_logs, 256, 0, st>>>((const drt_mlp_log*)d_logs, (double*)d_sums);
    uint2 key = make_uint2((uint32_t)o->seed, (uint32_t)(o->seed >> 32));
    unsigned gr = (unsigned)((rows + 255) / 256);
    drt::k_shuffle_keys<<<gr, 256, 0, st>>>(rows, key, (uint32_t*)keys, (int32_t*)vals);
    bool alt = drt::radix_sort_pairs((uint32_t*)keys, (int32_t*)vals, (uint32_t*)keys2, (int32_t*)vals2,
                                     (uint32_t*)hist, (uint32_t*)hist_tmp, (int)rows, 32, st);
    const int32_t* perm = alt ? (const int32_t*)vals2 : (const int32_t*)vals;
    drt::k_training_rows<<<gr, 256, 0, st>>>((const drt_mlp_log*)d_logs, (const int64_t*)d_offs, n_logs,
                                             (const double*)d_sums, perm, rows, delta, (__nv_bfloat16*)x,
                                             (float*)target, (float*)mask, o->rows_index);
    if (o->rows_target) e = cudaMemcpyAsync(o->rows_target, target, sizeof(float) * rows, cudaMemcpyDefault, st);
    if (e == cudaSuccess && o->rows_mask)
      e = cudaMemcpyAsync(o->rows_mask, mask, sizeof(float) * rows, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  // mini-batch Adam over the shuffled rows, cosine decay to lr/10
  drt::ParamArrays pa;
  for (int k = 0; k < drt::kNumParamArrays; ++k) {
    pa.p[k] = state->p[k];
    pa.m1[k] = state->m1[k];
    pa.m2[k] = state->m2[k];
    pa.g[k] = state->g[k];
  }
  pa.w1b = (__nv_bfloat16*)state->w1_bf16;
  pa.w2b = (__nv_bfloat16*)state->w2_bf16;
  drt_mlp_weights w{state->w1_bf16, state->p[1], state->w2_bf16, state->p[3], state->p[4], state->p[5]};
  drt_mlp_grads g{state->g[0], state->g[1], state->g[2], state->g[3], state->g[4], state->g[5]};
  float* loss = o->loss ? o->loss : (float*)loss_tmp;
  int64_t nb = rows / batch > 0 ? rows / batch : 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  unsigned gp = (unsigned)((drt::kParamTotal + 255) / 256);
  drt_status r = DRT_OK;
  for (int i = 0; i < o->steps && e == cudaSuccess && r == DRT_OK; ++i) {
    int64_t b = i % nb;
    float lr_i = lr * (0.55f + 0.45f * cosf(3.14159265358979f * (float)i / (float)o->steps));
    drt::k_zero_grads<<<gp, 256, 0, st>>>(pa);
    r = drt_mlp_backward(ctx, (const __nv_bfloat16*)x + b * batch * drt::kIn, (const float*)target + b * batch,
                         (const float*)mask + b * batch, batch, 1.0f / (float)batch, &w, &g, loss, stream);
    int64_t step = state->step + 1;
    float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    DRT_PROF_LAUNCH("adam", st, drt::k_adam_all<<<gp, 256, 0, st>>>(pa, lr_i, b1, b2, eps, c1, c2));
    state->step = step;
    e = cudaGetLastError();
  }
  cudaError_t es = cudaStreamSynchronize(st);
  release();
  if (r != DRT_OK) return r;
  if (e != cudaSuccess || es != cudaSuccess) {
    drt::set_last_error(cudaGetErrorString(e != cudaSuccess ? e : es));
    return DRT_ERR_CUDA;
  }
  return DRT_OK;
}

drt_status drt_adam_step(drt_context* ctx, float* params, const float* grads, float* m1, float* m2, void* params_bf16,
                         int64_t n, float lr, float beta1, float beta2, float eps, int32_t step, void* stream) {
  NvtxRange nvtx_range("drt_adam_step");
  if (!ctx || n < 0 || n > INT32_MAX || step < 1 || (n > 0 && (!params || !grads || !m1 || !m2)))
    return DRT_ERR_INVALID_ARG;
  if (n == 0) return DRT_OK;
  float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  cudaStream_t st = (cudaStream_t)stream;
  DRT_PROF_LAUNCH("adam", st, drt::k_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                                  params, grads, m1, m2, (__nv_bfloat16*)params_bf16, (int)n, lr, beta1, beta2, eps,
                                  c1, c2));
  return cudaGetLastError() == cudaSuccess ? DRT_OK : DRT_ERR_CUDA;
}

}  // extern "C"
