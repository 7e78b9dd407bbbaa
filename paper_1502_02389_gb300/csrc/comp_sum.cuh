// Compensated summation helpers shared by the mixed-precision and the
// compensated fp32 reductions: a (sum, compensation) pair updated with
// Knuth's TwoSum (the rounding error of every add is carried exactly in the
// compensation), merged pairwise across a warp and a CTA.
#pragma once
#include "lift_internal.cuh"

namespace lift {
namespace {

struct Comp {
  float s, c;
};

// s + v with the rounding error folded into c (TwoSum: 6 flops, no branch).
__device__ __forceinline__ void two_sum_add(Comp& a, float v) {
  const float t = __fadd_rn(a.s, v);
  const float bp = __fsub_rn(t, a.s);
  const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
  a.c = __fadd_rn(a.c, e);
  a.s = t;
}

__device__ __forceinline__ Comp comp_merge(Comp a, const Comp& b) {
  a.c = __fadd_rn(a.c, b.c);
  two_sum_add(a, b.s);
  return a;
}

__device__ __forceinline__ double comp_value(const Comp& a) {
  return isfinite(a.s) ? __dadd_rn((double)a.s, (double)a.c) : (double)a.s;
}

__device__ __forceinline__ Comp warp_comp(Comp v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Comp w;
    w.s = __shfl_down_sync(0xffffffffu, v.s, o);
    w.c = __shfl_down_sync(0xffffffffu, v.c, o);
    v = comp_merge(v, w);
  }
  return v;
}

template <int THREADS>
__device__ __forceinline__ Comp block_comp(Comp v) {
  __shared__ float rs[kWarp], rc[kWarp];
  v = warp_comp(v);
  if constexpr (THREADS > kWarp) {
    const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x / kWarp;
    if (lane == 0) {
      rs[warp] = v.s;
      rc[warp] = v.c;
    }
    __syncthreads();
    if (warp == 0) {
      v.s = lane < THREADS / kWarp ? rs[lane] : 0.f;
      v.c = lane < THREADS / kWarp ? rc[lane] : 0.f;
      v = warp_comp(v);
    }
  }
  return v;
}

}  // namespace
}  // namespace lift
