// fp32 reduction kernel templates -- asum, dot, nrm2, sum (arXiv 1502.02389,
// Fig. 5; fused form of Fig. 8 eq. (8); device structure of Fig. 9a).
// Instantiated by reduce_f32.cu (the hand-picked variant space) and
// reduce_derived.cu (parameter sets emitted by the rule-driven enumeration).
//
// A variant evaluates the low-level expression
//
//   reduce-seq(add64) . join . map-workgroup(
//       tree . lanes . join . map-local(reduce-seq(vect^VW(f), 0))
//            . split^(K*J) . reorder-stride^THREADS . asVector^VW
//   ) . split^(K*TILE) . join . reorder-stride^G . split^TILE (x)
//
// with f = absAndPlus (asum) or lambda acc,(a,b): acc + a*b (dot):
//  * split^TILE and reorder-stride^G at tile level: CTA b of the G-CTA grid
//    takes tiles b, b+G, b+2G, ... (round robin);
//  * reorder-stride^THREADS (STRIDE) or a block-level stride (chunk): which
//    vectors of a tile thread t folds, and in which order;
//  * asVector^VW: 4-byte, 128-bit or 256-bit loads; VW lane accumulators;
//  * tree: lane sum, warp shuffle halving tree, shared-memory stage over
//    warps, and with CLUSTER > 1 a rank-ordered sum over the cluster's CTAs
//    read through distributed shared memory;
//  * the outer reduce: per-CTA fp32 partials summed in FP64 either by the
//    last CTA to finish (one pass, atomic ticket) or by a second kernel.
// Within a thread the fold is split at the tile (the partial reduction of
// Fig. 3d applied to the thread's reduce-seq): each tile's J vectors are
// folded from zero into VW lane sums, the lanes are added in order, and the
// thread adds its tile values with Neumaier's compensated step, so its error
// does not grow with the number of tiles it folds (the thread's value is
// sum + compensation).
// Every add and multiply is an explicit round-to-nearest fp32 operation
// (__fadd_rn / __fmul_rn), so the result is the expression's value bit for
// bit.  STAGES >= 2 stages full tiles through a ring of TMA bulk copies
// (cp.async.bulk + mbarrier); STAGES == 0 uses 128/256-bit direct loads
// with a one-tile register prefetch.  Ragged tails are read with guarded
// scalar loads (zero padding, the neutral element of add).
#pragma once
#include <cooperative_groups.h>

#include "lift_internal.cuh"

namespace cg = cooperative_groups;

namespace lift {
namespace {

// The fused reduction function lambda acc, x: acc + g(x) of each program
// (rule 3f applied to reduce(add, 0) . map(g)): g = abs (asum), mult over
// the zipped pair (dot), square (nrm2), none (sum).
template <int OP>
__device__ __forceinline__ float fold_term(float acc, float a, float b) {
  if constexpr (OP == LIFT_OP_ASUM) {
    return __fadd_rn(acc, fabsf(a));
  } else if constexpr (OP == LIFT_OP_DOT) {
    return __fadd_rn(acc, __fmul_rn(a, b));
  } else if constexpr (OP == LIFT_OP_NRM2) {
    return __fadd_rn(acc, __fmul_rn(a, a));
  } else {
    return __fadd_rn(acc, a);
  }
}

// map(post) over the FP64 reduce result: sqrt for nrm2 (correctly rounded)
template <int OP>
__device__ __forceinline__ double post(double s) {
  if constexpr (OP == LIFT_OP_NRM2) return __dsqrt_rn(s);
  return s;
}

template <int OP, int VW>
__device__ __forceinline__ void fold_vec(float* acc, const Vec<VW>& a, const Vec<VW>& b) {
#pragma unroll
  for (int l = 0; l < VW; ++l) acc[l] = fold_term<OP>(acc[l], a.v[l], b.v[l]);
}

// lane sum of a tile: ((l0 + l1) + l2) + ...
template <int VW>
__device__ __forceinline__ float lane_sum(const float* ts) {
  float r = ts[0];
#pragma unroll
  for (int l = 1; l < VW; ++l) r = __fadd_rn(r, ts[l]);
  return r;
}

// index (in vectors) of thread t's j-th vector inside a tile
template <int THREADS, int J, bool STRIDE>
__device__ __forceinline__ int vec_index(int t, int j) {
  return STRIDE ? t + THREADS * j : t * J + j;
}

// CTA result -> (cluster) -> partials -> (one pass) final FP64 combine.
template <int OP, int THREADS, int CLUSTER, bool ONEPASS>
__device__ __forceinline__ void finish(float r, float* red, double* red64, float* partials,
                                       unsigned* ticket, float* result, double* result64) {
  // two passes: the combine kernel (a programmatic dependent launch) may be
  // scheduled now; it waits for this grid to finish before it reads
  if constexpr (!ONEPASS) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  r = block_tree<THREADS>(r, red);
  int64_t pidx = blockIdx.x;
  bool leader = true;
  if constexpr (CLUSTER > 1) {
    __shared__ float cl_val;
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x == 0) cl_val = r;
    cl.sync();
    leader = cl.block_rank() == 0;
    if (leader && threadIdx.x == 0) {
      float p = cl_val;
      for (int q = 1; q < CLUSTER; ++q) p = __fadd_rn(p, *cl.map_shared_rank(&cl_val, q));
      r = p;
    }
    cl.sync();
    pidx = blockIdx.x / CLUSTER;
  }
  if (!leader) return;
  if (threadIdx.x == 0) partials[pidx] = r;
  if constexpr (ONEPASS) {
    __shared__ bool is_last;
    const int64_t P = gridDim.x / CLUSTER;
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned k = atomicAdd(ticket, 1u);
      is_last = (k == static_cast<unsigned>(P - 1));
    }
    __syncthreads();
    if (is_last) {
      __threadfence();
      const double s = post<OP>(combine_partials<THREADS>(partials, P, red64));
      if (threadIdx.x == 0) {
        *result = static_cast<float>(s);
        if (result64) *result64 = s;
        *ticket = 0u;  // ready for the next call (and for graph replays)
      }
    }
  }
}

// Ragged last tile (index n / TILE): guarded scalar loads, zero padded.
template <int OP, int THREADS, int TILE, int VW, bool STRIDE>
__device__ __forceinline__ void fold_tail(float* acc, const float* x, const float* y, int64_t n,
                                          int64_t tile) {
  constexpr int J = TILE / VW / THREADS;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int64_t first = tile * TILE + (int64_t)vec_index<THREADS, J, STRIDE>(threadIdx.x, j) * VW;
    Vec<VW> a, b;
    ld_guarded<VW>(x, first, n, a);
    if constexpr (OP == LIFT_OP_DOT) ld_guarded<VW>(y, first, n, b);
    fold_vec<OP, VW>(acc, a, b);
  }
}

template <int OP, int THREADS, int TILE, int VW, bool STRIDE, int CLUSTER, bool ONEPASS>
__global__ void __launch_bounds__(THREADS)
    reduce_ldg(const float* __restrict__ x, const float* __restrict__ y, int64_t n,
               float* __restrict__ partials, unsigned* ticket, float* result, double* result64,
               int* status, uint32_t polls) {
  constexpr int V = TILE / VW, J = V / THREADS;
  static_assert(V % THREADS == 0 && J >= 1, "tile too small for the CTA");
  __shared__ float red[kWarp];
  __shared__ double red64[kWarp];
  pdl_wait();   // the previous kernel on the stream has completed
  const int t = threadIdx.x;
  const int64_t full = n / TILE;
  float acc = 0.0f, cmp = 0.0f;

  Vec<VW> cx[J], cy[J];
  int64_t tile = blockIdx.x;
  if (tile < full) {
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int64_t e = tile * TILE + (int64_t)vec_index<THREADS, J, STRIDE>(t, j) * VW;
      ld_stream(x + e, cx[j]);
      if constexpr (OP == LIFT_OP_DOT) ld_stream(y + e, cy[j]);
    }
  }
  while (tile < full) {
    const int64_t nxt = tile + gridDim.x;
    Vec<VW> nx[J], ny[J];
    if (nxt < full) {
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int64_t e = nxt * TILE + (int64_t)vec_index<THREADS, J, STRIDE>(t, j) * VW;
        ld_stream(x + e, nx[j]);
        if constexpr (OP == LIFT_OP_DOT) ld_stream(y + e, ny[j]);
      }
    }
    float ts[VW];
#pragma unroll
    for (int l = 0; l < VW; ++l) ts[l] = 0.0f;
#pragma unroll
    for (int j = 0; j < J; ++j) fold_vec<OP, VW>(ts, cx[j], cy[j]);
    neumaier_add(acc, cmp, lane_sum<VW>(ts));
#pragma unroll
    for (int j = 0; j < J; ++j) {
      cx[j] = nx[j];
      if constexpr (OP == LIFT_OP_DOT) cy[j] = ny[j];
    }
    tile = nxt;
  }
  if (tile == full && full * TILE < n) {
    float ts[VW];
#pragma unroll
    for (int l = 0; l < VW; ++l) ts[l] = 0.0f;
    fold_tail<OP, THREADS, TILE, VW, STRIDE>(ts, x, y, n, tile);
    neumaier_add(acc, cmp, lane_sum<VW>(ts));
  }

  const float r = neumaier_value(acc, cmp);
  finish<OP, THREADS, CLUSTER, ONEPASS>(r, red, red64, partials, ticket, result, result64);
  (void)status;
  (void)polls;
}

template <int OP, int THREADS, int TILE, int VW, bool STRIDE, int STAGES, int CLUSTER, bool ONEPASS>
__global__ void __launch_bounds__(THREADS)
    reduce_tma(const float* __restrict__ x, const float* __restrict__ y, int64_t n,
               float* __restrict__ partials, unsigned* ticket, float* result, double* result64,
               int* status, uint32_t polls) {
  constexpr int V = TILE / VW, J = V / THREADS;
  constexpr int NIN = (OP == LIFT_OP_DOT) ? 2 : 1;
  constexpr uint32_t kTileBytes = TILE * sizeof(float);
  static_assert(V % THREADS == 0 && J >= 1, "tile too small for the CTA");
  static_assert(kTileBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* buf = reinterpret_cast<float*>(smem_raw);  // [STAGES][NIN][TILE]
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ float red[kWarp];
  __shared__ double red64[kWarp];
  const int t = threadIdx.x;
  const int64_t full = n / TILE;
  const int64_t G = gridDim.x;
  const int64_t myK = (int64_t)blockIdx.x < full ? (full - 1 - blockIdx.x) / G + 1 : 0;

  if (t == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&full_bar[s], 1);
    fence_mbar_init();
  }
  pdl_wait();   // the previous kernel on the stream has completed
  __syncthreads();
  auto issue = [&](int64_t k) {
    const int s = static_cast<int>(k % STAGES);
    const int64_t tl = blockIdx.x + k * G;
    float* dst = buf + (size_t)s * NIN * TILE;
    mbar_arrive_expect_tx(&full_bar[s], NIN * kTileBytes);
    bulk_g2s(dst, x + tl * TILE, kTileBytes, &full_bar[s]);
    if constexpr (OP == LIFT_OP_DOT) bulk_g2s(dst + TILE, y + tl * TILE, kTileBytes, &full_bar[s]);
  };
  if (t == 0)
    for (int64_t k = 0; k < STAGES && k < myK; ++k) issue(k);

  float acc = 0.0f, cmp = 0.0f;
  bool timed_out = false;
  int64_t k = 0;
  for (; k < myK; ++k) {
    const int s = static_cast<int>(k % STAGES);
    const bool ok = mbar_wait(&full_bar[s], static_cast<uint32_t>((k / STAGES) & 1), polls);
    if (ok) {
      const float* bx = buf + (size_t)s * NIN * TILE;
      float ts[VW];
#pragma unroll
      for (int l = 0; l < VW; ++l) ts[l] = 0.0f;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int idx = vec_index<THREADS, J, STRIDE>(t, j) * VW;
        Vec<VW> a, b;
        ld_smem<VW>(bx + idx, a);
        if constexpr (OP == LIFT_OP_DOT) ld_smem<VW>(bx + TILE + idx, b);
        fold_vec<OP, VW>(ts, a, b);
      }
      neumaier_add(acc, cmp, lane_sum<VW>(ts));
    }
    if (!__syncthreads_and(ok)) {
      // a copy did not complete in time: record it, wait (with the full
      // limit) for every copy still in flight into the ring -- the one
      // waited for included -- so none lands after the CTA has left, and
      // stop folding.  The CTA still takes its ticket below with a NaN
      // partial: the call's result is NaN, and the ticket returns to 0.
      if (t == 0) {
        report(status, LIFT_ERR_TIMEOUT);
        for (int64_t q = k; q < k + STAGES && q < myK; ++q)
          mbar_wait(&full_bar[q % STAGES], static_cast<uint32_t>((q / STAGES) & 1));
      }
      timed_out = true;
      break;
    }
    if (t == 0 && k + STAGES < myK) issue(k + STAGES);
  }
  const int64_t tail_owner = full % G;
  if (!timed_out && full * TILE < n && (int64_t)blockIdx.x == tail_owner) {
    float ts[VW];
#pragma unroll
    for (int l = 0; l < VW; ++l) ts[l] = 0.0f;
    fold_tail<OP, THREADS, TILE, VW, STRIDE>(ts, x, y, n, full);
    neumaier_add(acc, cmp, lane_sum<VW>(ts));
  }

  float r = neumaier_value(acc, cmp);
  if (timed_out) r = __int_as_float(0x7fc00000);
  finish<OP, THREADS, CLUSTER, ONEPASS>(r, red, red64, partials, ticket, result, result64);
}

template <int OP, int FT>
__global__ void __launch_bounds__(FT)
    combine_kernel(const float* __restrict__ partials, int64_t P, float* result, double* result64) {
  pdl_trigger();   // the next call's first kernel may be scheduled (it waits for this one)
  pdl_wait();      // the first pass has finished
  __shared__ double red64[kWarp];
  const double s = post<OP>(combine_partials<FT>(partials, P, red64));
  if (threadIdx.x == 0) {
    *result = static_cast<float>(s);
    if (result64) *result64 = s;
  }
}

constexpr int kCombineThreads = 256;

// The second pass, launched as a programmatic dependent of the first so that
// its launch overlaps the first pass's tail.
template <int OP>
lift_status launch_combine(const float* partials, int64_t P, float* result, double* result64,
                           cudaStream_t s) {
  void* args[] = {&partials, &P, &result, &result64};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1);
  cfg.blockDim = dim3(kCombineThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cuda_check(cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(&combine_kernel<OP, kCombineThreads>),
                                        args),
                    "combine launch");
}

template <int OP, int THREADS, int TILE, int VW, bool STRIDE, int STAGES, int CLUSTER, int PASSES>
struct ReduceF32 {
  static constexpr int NIN = (OP == LIFT_OP_DOT) ? 2 : 1;
  static const void* kernel() {
    if constexpr (STAGES == 0)
      return reinterpret_cast<const void*>(
          &reduce_ldg<OP, THREADS, TILE, VW, STRIDE, CLUSTER, PASSES == 1>);
    else
      return reinterpret_cast<const void*>(
          &reduce_tma<OP, THREADS, TILE, VW, STRIDE, STAGES, CLUSTER, PASSES == 1>);
  }
  static size_t smem() { return (size_t)STAGES * NIN * TILE * sizeof(float); }

  // Persistent grid, shrunk so that every CTA takes the same number of tiles
  // (ceil(T / G_max) each): no CTA runs a last tile alone.
  static int64_t grid(const Variant&, const Args& a) {
    const int64_t T = a.n > 0 ? (a.n + TILE - 1) / TILE : 1;
    int64_t g = persistent_grid(kernel(), THREADS, smem(), CLUSTER);
    if (g <= 0) return 0;
    const int64_t per = (T + g - 1) / g;
    g = (T + per - 1) / per;
    g = (g + CLUSTER - 1) / CLUSTER * CLUSTER;
    return g;
  }

  static lift_status launch(const Variant& v, const Args& a, cudaStream_t s) {
    DeviceState* st = current_state();
    const int64_t g = grid(v, a);
    if (g <= 0) return set_error(LIFT_ERR_CUDA, std::string("no resident CTA for ") + v.info.name);
    if (g > st->ws.capacity)
      return set_error(LIFT_ERR_UNSUPPORTED, "grid exceeds the partials workspace");
    const float* x = static_cast<const float*>(a.x);
    const float* y = static_cast<const float*>(a.y);
    int64_t n = a.n;
    float* partials = a.ws->partials;
    unsigned* ticket = a.ws->tickets;
    float* result = a.result;
    double* result64 = a.result64;
    int* status = st->ws.status;
    uint32_t polls = wait_polls();
    void* args[] = {&x, &y, &n, &partials, &ticket, &result, &result64, &status, &polls};
    lift_status rc =
        launch_config(kernel(), dim3((unsigned)g), dim3(THREADS), smem(), CLUSTER, s, args, true);
    if (rc != LIFT_OK || PASSES == 1) return rc;
    return launch_combine<OP>(partials, g / CLUSTER, a.result, a.result64, s);
  }
};

template <int OP, int THREADS, int TILE, int VW, bool STRIDE, int STAGES, int CLUSTER, int PASSES>
Variant make_variant(const char* name) {
  using K = ReduceF32<OP, THREADS, TILE, VW, STRIDE, STAGES, CLUSTER, PASSES>;
  Variant v{};
  v.info.op = OP;
  v.info.tile = TILE;
  v.info.vw = VW;
  v.info.threads = THREADS;
  v.info.stride = STRIDE ? 1 : 0;
  v.info.tree = CLUSTER > 1 ? 2 : (THREADS > kWarp ? 1 : 0);
  v.info.cluster = CLUSTER;
  v.info.passes = PASSES;
  v.info.stages = STAGES;
  v.info.final_threads = PASSES == 1 ? THREADS : kCombineThreads;
  const char* prefix = OP == LIFT_OP_ASUM ? "asum" : OP == LIFT_OP_DOT ? "dot" : OP == LIFT_OP_NRM2 ? "nrm2" : "sum";
  snprintf(v.info.name, sizeof(v.info.name), "%s_%s", prefix, name);
  v.launch = &K::launch;
  v.grid = &K::grid;
  v.align_bytes = STAGES > 0 ? 16 : VW * (int)sizeof(float);
  v.fallback = -1;
  return v;
}

}  // namespace
}  // namespace lift
