// Persistent traversal pools for incoherent rays.
//
// A warp whose lanes each trace their own ray runs until its longest
// traversal ends, and after a diffuse bounce the lengths differ widely (about
// 6 of 32 lanes stayed active per instruction in the continuation kernels).
// Here the rays come from a buffer and every lane takes a new record as soon
// as its current one is done (one warp-aggregated atomic per refill), and the
// traversal advances one node visit or one leaf per loop iteration, so lanes
// are idle for at most one iteration between records.  The work per record
// is that of trace_closest2 / trace_any2 (a pair of rays traversing the
// union of the nodes either enters), with the same tests in the same order,
// so the results are the same: the closest hit with ties to the lowest id,
// and whether any occluder lies before tmax.
#pragma once

#include "drt_device.cuh"

namespace drt {

// Resident CTAs per SM of the one-ray pools (5: at most 51 registers; of 4,
// 5 and 6 the fastest on the 200k-triangle depth-3 step).  The two-ray pools
// run 4 (64 registers).
#ifndef DRT_POOL1_BLOCKS
#define DRT_POOL1_BLOCKS 5
#endif

// Closest-hit record: (o0.xyz, exclude0 bits), (d0.xyz, active0), (o1.xyz,
// exclude1 bits), (d1.xyz, active1); result: (tri, t bits, b1 bits, b2 bits)
// per ray, tri -1 for a miss or an inactive ray.
// Any-hit record: (o0.xyz, skip0a bits), (d0.xyz, skip0b bits), (o1.xyz,
// skip1a bits), (d1.xyz, skip1b bits), (active0, active1, 0, 0); result: bit
// 0 ray 0 occluded, bit 1 ray 1 occluded (tmax = kShadowTmax).
// (record sizes kClosestRecF4 and kAnyRecF4 in drt_device.cuh)

// Refill: every lane without a record and not yet exhausted takes the next
// one; returns false for a lane that found the buffer drained.
__device__ __forceinline__ void pool_fetch(unsigned long long* next, unsigned long long count, bool& have,
                                           bool& done, unsigned long long& idx) {
  int lane = threadIdx.x & 31;
  bool need = !have && !done;
  unsigned m = __ballot_sync(0xffffffffu, need);
  if (!m) return;
  int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(next, (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (need) {
    idx = base + __popc(m & ((1u << lane) - 1u));
    if (idx < count) have = true;
    else done = true;
  }
}

// kPair false: every record's second ray is inactive (the camera paths'
// continuation), and the kernel is compiled for one ray per record.
template <bool kPair>
__global__ void __launch_bounds__(256, kPair ? 4 : DRT_POOL1_BLOCKS) k_pool_closest(SceneView s, const float4* rec, const unsigned long long* count_ptr,
                                                      int4* hits, unsigned long long* next) {
  const unsigned long long count = *count_ptr;
  bool have = false, done = false;
  unsigned long long idx = 0;
  RayPre r0, r1;
  bool act0 = false, act1 = false;
  int ex0 = -1, ex1 = -1;
  Hit h0, h1;
  int stack[kStackSize];
  int sp = 0, node = 0, budget = 0, n_nodes = 0, n_tris = 0;
  while (true) {
    bool had = have;
    pool_fetch(next, count, have, done, idx);
    if (have && !had) {
      const float4* r = rec + (size_t)kClosestRecF4 * idx;
      float4 a = r[0], b = r[1], c = r[2], d = r[3];
      float o0[3] = {a.x, a.y, a.z}, d0[3] = {b.x, b.y, b.z}, o1[3] = {c.x, c.y, c.z}, d1[3] = {d.x, d.y, d.z};
      ray_pre(r0, o0, d0);
      if (kPair) ray_pre(r1, o1, d1);
      ex0 = __float_as_int(a.w);
      ex1 = __float_as_int(c.w);
      act0 = b.w != 0.0f;
      act1 = kPair && d.w != 0.0f;
      h0.tri = -1; h0.t = INFINITY; h0.b1 = h0.b2 = 0.f;
      h1.tri = -1; h1.t = INFINITY; h1.b1 = h1.b2 = 0.f;
      sp = 0;
      node = s.root;
      budget = 2 * s.T + 8;
      n_nodes = n_tris = 0;
    }
    if (!__any_sync(0xffffffffu, have)) break;
    if (!have) continue;
    bool finish = !act0 && !act1;
    if (!finish && --budget < 0) {
      raise_flag(s.err, DRT_DEV_TRAVERSAL_CAP, s.T);
      finish = true;
    }
    if (!finish) {
      bool pop = false;
      if (node >= 0) {
        ++n_nodes;
        const float4* n4 = s.nodes + 4 * node;
        float4 a = __ldg(n4), b = __ldg(n4 + 1), c = __ldg(n4 + 2);
        int4 ch = __ldg(reinterpret_cast<const int4*>(n4 + 3));
        float tl0, tr0, tl1, tr1;
        bool hl0, hr0, hl1, hr1;
        slab2(r0, a, b, c, h0.t, &tl0, &hl0, &tr0, &hr0);
        if (kPair) {
          slab2(r1, a, b, c, h1.t, &tl1, &hl1, &tr1, &hr1);
        } else {
          tl1 = tr1 = INFINITY;
          hl1 = hr1 = false;
        }
        bool hl = (act0 && hl0) || (act1 && hl1), hr = (act0 && hr0) || (act1 && hr1);
        float tl = fminf(act0 && hl0 ? tl0 : INFINITY, act1 && hl1 ? tl1 : INFINITY);
        float tr = fminf(act0 && hr0 ? tr0 : INFINITY, act1 && hr1 ? tr1 : INFINITY);
        if (hl && hr) {
          int nearc = tl <= tr ? ch.x : ch.y, farc = tl <= tr ? ch.y : ch.x;
          if (sp < kStackSize) stack[sp++] = farc; else raise_flag(s.err, DRT_DEV_STACK_OVERFLOW, node);
          node = nearc;
        } else if (hl) {
          node = ch.x;
        } else if (hr) {
          node = ch.y;
        } else {
          pop = true;
        }
      } else {
        int enc = ~node, first = enc & 0x0fffffff, cnt = (enc >> 28) + 1;
        for (int q = 0; q < cnt; ++q) {
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
        pop = true;
      }
      if (pop) {
        if (sp == 0) finish = true;
        else node = stack[--sp];
      }
    }
    if (finish) {
      hits[2 * idx] = make_int4(act0 ? h0.tri : -1, __float_as_int(h0.t), __float_as_int(h0.b1), __float_as_int(h0.b2));
      hits[2 * idx + 1] = make_int4(act1 ? h1.tri : -1, __float_as_int(h1.t), __float_as_int(h1.b1),
                                    __float_as_int(h1.b2));
      count_trace(s, kCntClosest, (int)act0 + (int)act1, n_nodes, n_tris);
      have = false;
    }
  }
}

template <bool kPair>
__global__ void __launch_bounds__(256, kPair ? 4 : DRT_POOL1_BLOCKS) k_pool_any(SceneView s, const float4* rec, const unsigned long long* count_ptr,
                                                  int* occ, unsigned long long* next) {
  const unsigned long long count = *count_ptr;
  const float tmax = kShadowTmax;
  bool have = false, done = false;
  unsigned long long idx = 0;
  RayPre r0, r1;
  bool act0 = false, act1 = false, live0 = false, live1 = false, occ0 = false, occ1 = false;
  int a0x = -1, a0y = -1, a1x = -1, a1y = -1;
  int stack[kStackSize];
  int sp = 0, node = 0, budget = 0, n_nodes = 0, n_tris = 0;
  while (true) {
    bool had = have;
    pool_fetch(next, count, have, done, idx);
    if (have && !had) {
      const float4* r = rec + (size_t)kAnyRecF4 * idx;
      float4 a = r[0], b = r[1], c = r[2], d = r[3], f = r[4];
      float o0[3] = {a.x, a.y, a.z}, d0[3] = {b.x, b.y, b.z}, o1[3] = {c.x, c.y, c.z}, d1[3] = {d.x, d.y, d.z};
      ray_pre(r0, o0, d0);
      if (kPair) ray_pre(r1, o1, d1);
      a0x = __float_as_int(a.w);
      a0y = __float_as_int(b.w);
      a1x = __float_as_int(c.w);
      a1y = __float_as_int(d.w);
      act0 = f.x != 0.0f;
      act1 = kPair && f.y != 0.0f;
      live0 = act0;
      live1 = act1;
      occ0 = occ1 = false;
      sp = 0;
      node = s.root;
      budget = 2 * s.T + 8;
      n_nodes = n_tris = 0;
    }
    if (!__any_sync(0xffffffffu, have)) break;
    if (!have) continue;
    bool finish = !live0 && !live1;
    if (!finish && --budget < 0) {
      raise_flag(s.err, DRT_DEV_TRAVERSAL_CAP, s.T);
      finish = true;
    }
    if (!finish) {
      bool pop = false;
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
        } else if (hl) {
          node = ch.x;
        } else if (hr) {
          node = ch.y;
        } else {
          pop = true;
        }
      } else {
        int enc = ~node, first = enc & 0x0fffffff, cnt = (enc >> 28) + 1;
        for (int q = 0; q < cnt && (live0 || live1); ++q) {
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
        pop = true;
      }
      if (pop && (live0 || live1)) {
        if (sp == 0) finish = true;
        else node = stack[--sp];
      } else if (!live0 && !live1) {
        finish = true;
      }
    }
    if (finish) {
      occ[idx] = (occ0 ? 1 : 0) | (occ1 ? 2 : 0);
      count_trace(s, kCntAny, (int)act0 + (int)act1, n_nodes, n_tris);
      have = false;
    }
  }
}

}  // namespace drt
