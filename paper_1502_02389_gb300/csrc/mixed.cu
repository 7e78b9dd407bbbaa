// Mixed-precision asum and dot: inputs stored as bf16, or as fp8-e4m3 with
// one fp32 scale per block of 4096 consecutive elements.
//
// The programs are those of Fig. 5 (asum = reduce(add,0) . map(abs),
// dot = reduce(add,0) . map(mult) . zip) over the stored values; the
// derivation is the fused form of Fig. 8 with the split at the scale block:
//
//   reduce(add64) . join . map-workgroup(tree_c . map-local(
//       reduce-seq(twoSum) . map-seq(scale_b . pairwise-sum . map(term))
//   )) . split^4096
//
//  * term: |q| (asum) or qx*qy (dot), exactly widened to fp32: bf16 -> fp32
//    is exact, fp8-e4m3 -> f16 -> fp32 is exact (cvt.rn.f16x2.e4m3x2), and
//    the product of two bf16 or two e4m3 values is exact in fp32;
//  * each thread takes E = 4096/THREADS consecutive elements of a block
//    (coalesced 16/32-byte loads) and sums its E terms with a halving tree
//    (pairwise, depth log2 E; for fp8 asum this sum is exact: E <= 64 values
//    on the 2^-9 grid below 2^15 need at most 24 bits, so the kernel adds
//    them in a cheaper order with the same value, see fp8_abs_sum);
//  * the block sum is multiplied once by the block scale (fp8: s_x, or
//    s_x * s_y for dot) and added into a (sum, compensation) pair with
//    Knuth's TwoSum;
//  * the CTA combines the pairs with TwoSum trees (warp shuffles, then
//    shared memory), writes sum + compensation as one FP64 partial, and the
//    last CTA (or a second kernel) adds the partials in FP64.
// A non-finite running sum is returned as it is (its compensation would be
// NaN), so Inf stays Inf and NaN stays NaN.
#include <cuda_fp16.h>

#include "comp_sum.cuh"

namespace lift {
namespace {

constexpr int kBlock = 4096;
enum { DT_BF16 = 1, DT_FP8 = 2 };

// --------------------------------------------------------------------------
// decoding
// --------------------------------------------------------------------------
__device__ __forceinline__ float2 e4m3x2_to_float2(uint32_t two_bytes) {
  uint32_t h;
  const uint16_t in = static_cast<uint16_t>(two_bytes);
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h) : "h"(in));
  __half2 hh = *reinterpret_cast<__half2*>(&h);
  return __half22float2(hh);
}

// Words (32-bit) of raw storage holding E elements.
template <int DT, int E>
struct Raw {
  static constexpr int W = DT == DT_FP8 ? E / 4 : E / 2;
  uint32_t w[W];
};

__device__ __forceinline__ void ld_words(const uint32_t* p, uint32_t* w, int count) {
  for (int i = 0; i < count; i += 8)
    asm("ld.global.nc.L1::no_allocate.L2::256B.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(w[i]), "=r"(w[i + 1]), "=r"(w[i + 2]), "=r"(w[i + 3]), "=r"(w[i + 4]),
          "=r"(w[i + 5]), "=r"(w[i + 6]), "=r"(w[i + 7])
        : "l"(p + i));
}
__device__ __forceinline__ void ld_words4(const uint32_t* p, uint32_t* w) {
  asm("ld.global.nc.L1::no_allocate.L2::256B.v4.b32 {%0,%1,%2,%3}, [%4];"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
      : "l"(p));
}

template <int DT, int E>
__device__ __forceinline__ void load_raw(const void* base, int64_t elem, Raw<DT, E>& r) {
  const uint32_t* p = reinterpret_cast<const uint32_t*>(
      static_cast<const uint8_t*>(base) + elem * (DT == DT_FP8 ? 1 : 2));
  if constexpr (Raw<DT, E>::W == 4) {
    ld_words4(p, r.w);
  } else {
    static_assert(Raw<DT, E>::W % 8 == 0, "load width");
#pragma unroll
    for (int i = 0; i < Raw<DT, E>::W; i += 8) ld_words(p + i, r.w + i, 8);
  }
}

template <int DT, int E>
__device__ __forceinline__ void decode(const Raw<DT, E>& r, float* v) {
  if constexpr (DT == DT_FP8) {
#pragma unroll
    for (int i = 0; i < E / 4; ++i) {
      const float2 a = e4m3x2_to_float2(r.w[i] & 0xffffu);
      const float2 b = e4m3x2_to_float2(r.w[i] >> 16);
      v[4 * i] = a.x;
      v[4 * i + 1] = a.y;
      v[4 * i + 2] = b.x;
      v[4 * i + 3] = b.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < E / 2; ++i) {
      v[2 * i] = __uint_as_float(r.w[i] << 16);
      v[2 * i + 1] = __uint_as_float(r.w[i] & 0xffff0000u);
    }
  }
}

// one stored element, for ragged tails and unaligned inputs
template <int DT>
__device__ __forceinline__ float decode_one(const void* base, int64_t i) {
  if constexpr (DT == DT_FP8) {
    const uint32_t b = static_cast<const uint8_t*>(base)[i];
    return e4m3x2_to_float2(b).x;
  } else {
    const uint32_t h = static_cast<const uint16_t*>(base)[i];
    return __uint_as_float(h << 16);
  }
}

template <int OP>
__device__ __forceinline__ float term(float a, float b) {
  if constexpr (OP == LIFT_OP_ASUM) return fabsf(a);
  else return __fmul_rn(a, b);  // exact for bf16 x bf16 and e4m3 x e4m3
}

// halving tree over E values in registers (pairwise summation)
template <int E>
__device__ __forceinline__ float pairwise(float* v) {
#pragma unroll
  for (int w = E / 2; w >= 1; w >>= 1)
#pragma unroll
    for (int i = 0; i < w; ++i) v[i] = __fadd_rn(v[i], v[i + w]);
  return v[0];
}

template <int OP, int DT>
__device__ __forceinline__ float block_scale(const float* xs, const float* ys, int64_t blk) {
  if constexpr (DT == DT_BF16) {
    return 1.0f;
  } else if constexpr (OP == LIFT_OP_ASUM) {
    return __ldg(xs + blk);
  } else {
    return __fmul_rn(__ldg(xs + blk), __ldg(ys + blk));
  }
}

// fp8 asum: a thread's E <= 64 magnitudes |q| lie on the 2^-9 grid below
// 448, so every partial sum of them is a multiple of 2^-9 below 2^15 and
// fits the 24-bit fp32 significand: any order of adding them gives the same
// exact value as the pairwise tree.  Here the sign bits are cleared on the
// raw bytes, e4m3 pairs are widened to f16 pairs (exact), and each f16 is
// added straight into an fp32 accumulator with the mixed-precision
// add.rn.f32.f16 (no separate f16 -> f32 conversion); four accumulators,
// one per byte position, are added at the end.
template <int E>
__device__ __forceinline__ float fp8_abs_sum(const uint32_t* w) {
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
  for (int i = 0; i < E / 4; ++i) {
    const uint32_t m = w[i] & 0x7f7f7f7fu;
    uint32_t lo, hi;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(lo) : "h"(static_cast<uint16_t>(m)));
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(hi) : "h"(static_cast<uint16_t>(m >> 16)));
    asm("{ .reg .f16 p, q; mov.b32 {p, q}, %2; add.rn.f32.f16 %0, p, %0; add.rn.f32.f16 %1, q, %1; }"
        : "+f"(a0), "+f"(a1) : "r"(lo));
    asm("{ .reg .f16 p, q; mov.b32 {p, q}, %2; add.rn.f32.f16 %0, p, %0; add.rn.f32.f16 %1, q, %1; }"
        : "+f"(a2), "+f"(a3) : "r"(hi));
  }
  return __fadd_rn(__fadd_rn(a0, a1), __fadd_rn(a2, a3));
}

template <int OP, int DT, int E>
__device__ __forceinline__ void fold_block(Comp& acc, const Raw<DT, E>& rx, const Raw<DT, E>& ry,
                                           float scale) {
  if constexpr (OP == LIFT_OP_ASUM && DT == DT_FP8) {
    static_assert(E <= 64, "the exact-sum argument needs at most 64 terms per thread");
    two_sum_add(acc, __fmul_rn(fp8_abs_sum<E>(rx.w), scale));
    return;
  }
  float vx[E], vy[E];
  decode<DT, E>(rx, vx);
  if constexpr (OP == LIFT_OP_DOT) decode<DT, E>(ry, vy);
#pragma unroll
  for (int i = 0; i < E; ++i) vx[i] = term<OP>(vx[i], OP == LIFT_OP_DOT ? vy[i] : 0.f);
  float bs = pairwise<E>(vx);
  if constexpr (DT == DT_FP8) bs = __fmul_rn(bs, scale);
  two_sum_add(acc, bs);
}

// element-wise (guarded) form of one block's share of a thread
template <int OP, int DT, int E>
__device__ __forceinline__ void fold_block_guarded(Comp& acc, const void* x, const void* y,
                                                   int64_t first, int64_t n, float scale) {
  float v[E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int64_t e = first + i;
    float a = 0.f, b = 0.f;
    if (e < n) {
      a = decode_one<DT>(x, e);
      if constexpr (OP == LIFT_OP_DOT) b = decode_one<DT>(y, e);
    }
    v[i] = term<OP>(a, b);
  }
  float bs = pairwise<E>(v);
  if constexpr (DT == DT_FP8) bs = __fmul_rn(bs, scale);
  two_sum_add(acc, bs);
}

// CONTIG: a CTA step takes U consecutive blocks (super-block sb covers
// blocks sb*U .. sb*U+U-1, CTAs take super-blocks round robin), so each step
// reads one contiguous U*4096-element run; otherwise the U blocks of a step
// are b, b+G, ..., b+(U-1)G.
template <int OP, int DT, int THREADS, int U, bool GUARDED, bool CONTIG = false>
__global__ void __launch_bounds__(THREADS)
    mixed_reduce(const void* __restrict__ x, const float* __restrict__ xs, const void* __restrict__ y,
                 const float* __restrict__ ys, int64_t n, double* __restrict__ partials,
                 unsigned* ticket, float* result, double* result64) {
  constexpr int E = kBlock / THREADS;
  pdl_wait();      // the previous kernel on the stream has completed
  const int t = threadIdx.x;
  const int64_t G = gridDim.x;
  const int64_t full = n / kBlock;
  Comp acc{0.f, 0.f};
  int64_t b = blockIdx.x;
  if constexpr (CONTIG && !GUARDED) {
    const int64_t nsb = full / U;
    for (int64_t sb = blockIdx.x; sb < nsb; sb += G) {
      Raw<DT, E> rx[U], ry[U];
      float sc[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t blk = sb * U + u;
        load_raw<DT, E>(x, blk * kBlock + (int64_t)t * E, rx[u]);
        if constexpr (OP == LIFT_OP_DOT) load_raw<DT, E>(y, blk * kBlock + (int64_t)t * E, ry[u]);
        sc[u] = block_scale<OP, DT>(xs, ys, blk);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) fold_block<OP, DT, E>(acc, rx[u], ry[u], sc[u]);
    }
    for (int64_t bb = nsb * U + blockIdx.x; bb < full; bb += G) {   // full blocks left over
      Raw<DT, E> rx, ry;
      load_raw<DT, E>(x, bb * kBlock + (int64_t)t * E, rx);
      if constexpr (OP == LIFT_OP_DOT) load_raw<DT, E>(y, bb * kBlock + (int64_t)t * E, ry);
      fold_block<OP, DT, E>(acc, rx, ry, block_scale<OP, DT>(xs, ys, bb));
    }
    b = full * kBlock < n && (int64_t)blockIdx.x == full % G ? full : n;   // the ragged block
  } else if constexpr (!GUARDED) {
    for (; b + (U - 1) * G < full; b += U * G) {
      Raw<DT, E> rx[U], ry[U];
      float sc[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t blk = b + u * G;
        load_raw<DT, E>(x, blk * kBlock + (int64_t)t * E, rx[u]);
        if constexpr (OP == LIFT_OP_DOT) load_raw<DT, E>(y, blk * kBlock + (int64_t)t * E, ry[u]);
        sc[u] = block_scale<OP, DT>(xs, ys, blk);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) fold_block<OP, DT, E>(acc, rx[u], ry[u], sc[u]);
    }
    for (; b < full; b += G) {
      Raw<DT, E> rx, ry;
      load_raw<DT, E>(x, b * kBlock + (int64_t)t * E, rx);
      if constexpr (OP == LIFT_OP_DOT) load_raw<DT, E>(y, b * kBlock + (int64_t)t * E, ry);
      fold_block<OP, DT, E>(acc, rx, ry, block_scale<OP, DT>(xs, ys, b));
    }
  }
  const int64_t nblocks = (n + kBlock - 1) / kBlock;
  for (; b < nblocks; b += G)
    fold_block_guarded<OP, DT, E>(acc, x, y, b * kBlock + (int64_t)t * E, n,
                                  block_scale<OP, DT>(xs, ys, b));

  pdl_trigger();   // streaming done: the next call's first kernel may be scheduled
  const Comp c = block_comp<THREADS>(acc);
  __shared__ bool is_last;
  __shared__ double red64[kWarp];
  if (t == 0) {
    partials[blockIdx.x] = comp_value(c);
    __threadfence();
    is_last = atomicAdd(ticket, 1u) == static_cast<unsigned>(G - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double s = 0.0;
  for (int64_t i = t; i < G; i += THREADS) s = __dadd_rn(s, __ldcg(partials + i));
  s = block_tree64<THREADS>(s, red64);
  if (t == 0) {
    *result = static_cast<float>(s);
    if (result64) *result64 = s;
    *ticket = 0u;
  }
}

template <int OP, int DT, int THREADS, int U, bool GUARDED, bool CONTIG = false>
struct Mixed {
  static const void* kernel() {
    return reinterpret_cast<const void*>(&mixed_reduce<OP, DT, THREADS, U, GUARDED, CONTIG>);
  }
  // persistent grid with the same number of blocks (super-blocks) for every CTA
  static int64_t grid(const Variant&, const Args& a) {
    int64_t nb = a.n > 0 ? (a.n + kBlock - 1) / kBlock : 1;
    if (CONTIG && nb >= U) nb /= U;
    const int64_t g = persistent_grid(kernel(), THREADS, 0, 1);
    if (g <= 0) return 0;
    const int64_t per = (nb + g - 1) / g;
    return (nb + per - 1) / per;
  }
  static lift_status launch(const Variant& v, const Args& a, cudaStream_t s) {
    DeviceState* st = current_state();
    const int64_t g = grid(v, a);
    if (g <= 0) return set_error(LIFT_ERR_CUDA, std::string("no resident CTA for ") + v.info.name);
    if (g > st->ws.capacity) return set_error(LIFT_ERR_UNSUPPORTED, "grid exceeds workspace");
    const void* x = a.x;
    const void* y = a.y;
    const float* xs = a.xscale;
    const float* ys = a.yscale;
    int64_t n = a.n;
    if (g > st->ws.capacity64) return set_error(LIFT_ERR_UNSUPPORTED, "grid exceeds workspace");
    double* partials = a.ws->partials64;
    unsigned* ticket = a.ws->tickets + 1;
    float* result = a.result;
    double* result64 = a.result64;
    void* args[] = {&x, &xs, &y, &ys, &n, &partials, &ticket, &result, &result64};
    return launch_config(kernel(), dim3((unsigned)g), dim3(THREADS), 0, 1, s, args, true);
  }
};

template <int OP, int DT, int THREADS, int U, bool GUARDED, bool CONTIG = false>
Variant mixed_variant(int opid, const char* name) {
  using K = Mixed<OP, DT, THREADS, U, GUARDED, CONTIG>;
  constexpr int E = kBlock / THREADS;
  Variant v{};
  v.info.op = opid;
  v.info.tile = kBlock;
  v.info.vw = E;
  v.info.threads = THREADS;
  v.info.stride = 0;
  v.info.tree = 1;
  v.info.cluster = 1;
  v.info.passes = 1;
  v.info.stages = 0;
  v.info.rows = U;
  v.info.final_threads = THREADS;
  snprintf(v.info.name, sizeof(v.info.name), "%s", name);
  v.launch = &K::launch;
  v.grid = &K::grid;
  v.align_bytes = GUARDED ? 1 : E * (DT == DT_FP8 ? 1 : 2);
  v.fallback = -1;
  return v;
}

template <int OP, int DT>
void register_one(std::vector<Variant>& L, int opid, const char* tag) {
  char nm[64];
  snprintf(nm, sizeof nm, "%s_t128_u2", tag);
  L.push_back(mixed_variant<OP, DT, 128, 2, false>(opid, nm));
  snprintf(nm, sizeof nm, "%s_t128_u4", tag);
  L.push_back(mixed_variant<OP, DT, 128, 4, false>(opid, nm));
  snprintf(nm, sizeof nm, "%s_t256_u4", tag);
  L.push_back(mixed_variant<OP, DT, 256, 4, false>(opid, nm));
  snprintf(nm, sizeof nm, "%s_t256_u8", tag);
  L.push_back(mixed_variant<OP, DT, 256, 8, false>(opid, nm));
  snprintf(nm, sizeof nm, "%s_t256_guarded", tag);
  L.push_back(mixed_variant<OP, DT, 256, 1, true>(opid, nm));
  const int guarded = static_cast<int>(L.size()) - 1;
  // 64 elements per thread per block: the block's decode, scale and
  // compensation work is spread over more elements
  snprintf(nm, sizeof nm, "%s_t64_u2", tag);
  L.push_back(mixed_variant<OP, DT, 64, 2, false>(opid, nm));
  snprintf(nm, sizeof nm, "%s_t64_u4", tag);
  L.push_back(mixed_variant<OP, DT, 64, 4, false>(opid, nm));
  // a CTA step over U consecutive blocks (one contiguous run per step)
  snprintf(nm, sizeof nm, "%s_t256_u4_c", tag);
  L.push_back(mixed_variant<OP, DT, 256, 4, false, true>(opid, nm));
  snprintf(nm, sizeof nm, "%s_t128_u4_c", tag);
  L.push_back(mixed_variant<OP, DT, 128, 4, false, true>(opid, nm));
  snprintf(nm, sizeof nm, "%s_t256_u8_c", tag);
  L.push_back(mixed_variant<OP, DT, 256, 8, false, true>(opid, nm));
  snprintf(nm, sizeof nm, "%s_t128_u2_c", tag);
  L.push_back(mixed_variant<OP, DT, 128, 2, false, true>(opid, nm));
  for (size_t i = 0; i < L.size(); ++i) {
    L[i].info.id = static_cast<int>(i);
    L[i].fallback = guarded;
  }
}

}  // namespace

void register_mixed(std::vector<Variant>* ops) {
  register_one<LIFT_OP_ASUM, DT_BF16>(ops[LIFT_OP_ASUM_BF16], LIFT_OP_ASUM_BF16, "asum_bf16");
  register_one<LIFT_OP_DOT, DT_BF16>(ops[LIFT_OP_DOT_BF16], LIFT_OP_DOT_BF16, "dot_bf16");
  register_one<LIFT_OP_ASUM, DT_FP8>(ops[LIFT_OP_ASUM_FP8], LIFT_OP_ASUM_FP8, "asum_fp8");
  register_one<LIFT_OP_DOT, DT_FP8>(ops[LIFT_OP_DOT_FP8], LIFT_OP_DOT_FP8, "dot_fp8");
}

}  // namespace lift
