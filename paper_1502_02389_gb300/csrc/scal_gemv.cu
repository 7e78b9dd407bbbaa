// scal and gemv kernels (arXiv 1502.02389, Fig. 5; scal's low-level form is
// the vectorScal expression of Fig. 2b).
//
// scal = join . map-workgroup(asScalar . map-local(vect^VW(mult(alpha)))
//                             . asVector^VW) . split^TILE, tiles round robin
// over a persistent grid, or (GRID == 1) one work-group per tile, launched
// all at once and dealt to the SMs by the hardware as earlier ones finish:
// the same expression, scheduled the way an OpenCL global size of n would
// be.  One correctly rounded fp32 multiply per element
// (__fmul_rn), so the output is bit-exact whatever the variant.  STAGES >= 2
// stages tiles through a TMA bulk-copy ring, multiplies in shared memory and
// writes back with bulk shared->global copies.
//
// gemv: z = map(scal(alpha) . dot(x), A); y' = map(add) . zip(z, scal(beta, y)).
// One warp takes a row (map-workgroup over row groups, map-local over the
// 32 lanes); lane l folds vectors l, l+32, ... of the row zipped with x
// (reorder-stride^32 . asVector^VW), adds its vector lanes, then a warp
// halving tree; lane 0 writes fl(fl(alpha * d) + fl(beta * y)).  With
// beta == 0, y is not read (BLAS definition).
#include "lift_internal.cuh"

namespace lift {
namespace {

// ---------------------------------------------------------------------------
// scal
// ---------------------------------------------------------------------------
template <int VW>
__device__ __forceinline__ void mul_vec(float alpha, Vec<VW>& v) {
#pragma unroll
  for (int l = 0; l < VW; ++l) v.v[l] = __fmul_rn(alpha, v.v[l]);
}

template <int THREADS, int TILE, int VW>
__device__ __forceinline__ void scal_tail(int64_t n, float alpha, const float* x, float* y, int64_t tile) {
  constexpr int J = TILE / VW / THREADS;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int64_t first = tile * TILE + (int64_t)(threadIdx.x + THREADS * j) * VW;
#pragma unroll
    for (int l = 0; l < VW; ++l)
      if (first + l < n) y[first + l] = __fmul_rn(alpha, x[first + l]);
  }
}

template <int THREADS, int TILE, int VW>
__global__ void __launch_bounds__(THREADS)
    scal_ldg(int64_t n, float alpha, const float* x, float* y) {
  constexpr int J = TILE / VW / THREADS;
  static_assert(J >= 1 && (TILE / VW) % THREADS == 0, "tile too small");
  pdl_trigger();   // the next call's first kernel may be scheduled (it waits for this one)
  pdl_wait();      // the previous kernel on the stream has completed
  const int64_t full = n / TILE;
  int64_t tile = blockIdx.x;
  for (; tile < full; tile += gridDim.x) {
    Vec<VW> v[J];
#pragma unroll
    for (int j = 0; j < J; ++j)
      ld_stream(x + tile * TILE + (int64_t)(threadIdx.x + THREADS * j) * VW, v[j]);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      mul_vec<VW>(alpha, v[j]);
      st_stream(y + tile * TILE + (int64_t)(threadIdx.x + THREADS * j) * VW, v[j]);
    }
  }
  if (tile == full && full * TILE < n) scal_tail<THREADS, TILE, VW>(n, alpha, x, y, tile);
}

template <int THREADS, int TILE, int STAGES>
__global__ void __launch_bounds__(THREADS)
    scal_tma(int64_t n, float alpha, const float* x, float* y, int* status) {
  constexpr uint32_t kTileBytes = TILE * sizeof(float);
  static_assert(kTileBytes % 16 == 0 && TILE % (4 * THREADS) == 0, "tile shape");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* buf = reinterpret_cast<float*>(smem_raw);  // [STAGES][TILE]
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  const int t = threadIdx.x;
  const int64_t full = n / TILE, G = gridDim.x;
  const int64_t myK = (int64_t)blockIdx.x < full ? (full - 1 - blockIdx.x) / G + 1 : 0;
  if (t == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&full_bar[s], 1);
    fence_mbar_init();
  }
  pdl_trigger();   // the next call's first kernel may be scheduled (it waits for this one)
  pdl_wait();      // the previous kernel on the stream has completed
  __syncthreads();
  auto issue = [&](int64_t k) {
    const int s = static_cast<int>(k % STAGES);
    mbar_arrive_expect_tx(&full_bar[s], kTileBytes);
    bulk_g2s(buf + (size_t)s * TILE, x + (blockIdx.x + k * G) * TILE, kTileBytes, &full_bar[s]);
  };
  if (t == 0)
    for (int64_t k = 0; k < STAGES && k < myK; ++k) issue(k);
  for (int64_t k = 0; k < myK; ++k) {
    const int s = static_cast<int>(k % STAGES);
    const bool ok = mbar_wait(&full_bar[s], static_cast<uint32_t>((k / STAGES) & 1));
    float* b = buf + (size_t)s * TILE;
    if (ok) {
#pragma unroll
      for (int j = 0; j < TILE / (4 * THREADS); ++j) {
        Vec<4> v;
        ld_smem<4>(b + 4 * (t + THREADS * j), v);
        mul_vec<4>(alpha, v);
        st_smem<4>(b + 4 * (t + THREADS * j), v);
      }
      fence_proxy_async_smem();  // generic smem writes -> bulk copy reads
    }
    if (!__syncthreads_and(ok)) {
      if (t == 0) {
        report(status, LIFT_ERR_TIMEOUT);
        for (int64_t q = k; q < k + STAGES && q < myK; ++q)   // every copy still in flight
          mbar_wait(&full_bar[q % STAGES], static_cast<uint32_t>((q / STAGES) & 1));
        bulk_wait_all();
      }
      return;
    }
    if (t == 0) {
      bulk_s2g(y + (blockIdx.x + k * G) * TILE, b, kTileBytes);
      bulk_commit();
      if (k + STAGES < myK) {
        bulk_wait_read<0>();  // the store has read stage s before it is refilled
        issue(k + STAGES);
      }
    }
  }
  if (t == 0) bulk_wait_all();
  if (full * TILE < n && (int64_t)blockIdx.x == full % G)
    scal_tail<THREADS, TILE, 4>(n, alpha, x, y, full);
}

// Grid of a map over T tiles: one CTA per tile (GRID == 1; the kernels'
// tile loops then run once, and a grid capped at 2^31 - 1 still covers every
// tile), or a persistent grid with the same number of tiles for every CTA.
template <int GRID>
int64_t map_grid(const void* kernel, int threads, size_t smem, int64_t T) {
  if constexpr (GRID == 1) {
    return T < INT32_MAX ? T : INT32_MAX;
  } else {
    const int64_t g = persistent_grid(kernel, threads, smem, 1);
    if (g <= 0) return 0;
    const int64_t per = (T + g - 1) / g;
    return (T + per - 1) / per;
  }
}

template <int THREADS, int TILE, int VW, int STAGES, int GRID = 0>
struct Scal {
  static_assert(GRID == 0 || STAGES == 0, "a staged ring needs several tiles per CTA");
  static const void* kernel() {
    if constexpr (STAGES == 0)
      return reinterpret_cast<const void*>(&scal_ldg<THREADS, TILE, VW>);
    else
      return reinterpret_cast<const void*>(&scal_tma<THREADS, TILE, STAGES>);
  }
  static size_t smem() { return (size_t)STAGES * TILE * sizeof(float); }
  static int64_t grid(const Variant&, const Args& a) {
    const int64_t T = a.n > 0 ? (a.n + TILE - 1) / TILE : 1;
    return map_grid<GRID>(kernel(), THREADS, smem(), T);
  }
  static lift_status launch(const Variant& v, const Args& a, cudaStream_t s) {
    const int64_t g = grid(v, a);
    if (g <= 0) return set_error(LIFT_ERR_CUDA, std::string("no resident CTA for ") + v.info.name);
    int64_t n = a.n;
    float alpha = a.alpha;
    const float* x = static_cast<const float*>(a.x);
    float* y = a.out;
    int* status = current_state()->ws.status;
    if constexpr (STAGES == 0) {
      void* args[] = {&n, &alpha, &x, &y};
      return launch_config(kernel(), dim3((unsigned)g), dim3(THREADS), 0, 1, s, args, true);
    } else {
      void* args[] = {&n, &alpha, &x, &y, &status};
      return launch_config(kernel(), dim3((unsigned)g), dim3(THREADS), smem(), 1, s, args, true);
    }
  }
};

template <int THREADS, int TILE, int VW, int STAGES, int GRID = 0>
Variant scal_variant(const char* name) {
  using K = Scal<THREADS, TILE, VW, STAGES, GRID>;
  Variant v{};
  v.info.op = LIFT_OP_SCAL;
  v.info.tile = TILE;
  v.info.vw = STAGES ? 4 : VW;
  v.info.threads = THREADS;
  v.info.stride = 1;
  v.info.tree = 0;
  v.info.cluster = 1;
  v.info.passes = 1;
  v.info.stages = STAGES;
  v.info.grid = GRID;
  snprintf(v.info.name, sizeof(v.info.name), "scal_%s", name);
  v.launch = &K::launch;
  v.grid = &K::grid;
  v.align_bytes = STAGES ? 16 : VW * 4;
  v.fallback = 0;
  return v;
}

// ---------------------------------------------------------------------------
// axpy = map(add) . zip(map(mult(alpha), x), y): the scal map with a second
// zipped input; y_i <- fl(fl(alpha * x_i) + y_i), one rounding per operation
// ---------------------------------------------------------------------------
template <int THREADS, int TILE, int VW>
__global__ void __launch_bounds__(THREADS)
    axpy_ldg(int64_t n, float alpha, const float* x, float* y) {
  constexpr int J = TILE / VW / THREADS;
  static_assert(J >= 1 && (TILE / VW) % THREADS == 0, "tile too small");
  pdl_trigger();   // the next call's first kernel may be scheduled (it waits for this one)
  pdl_wait();      // the previous kernel on the stream has completed
  const int64_t full = n / TILE;
  int64_t tile = blockIdx.x;
  for (; tile < full; tile += gridDim.x) {
    Vec<VW> a[J], b[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int64_t e = tile * TILE + (int64_t)(threadIdx.x + THREADS * j) * VW;
      ld_stream(x + e, a[j]);
      ld_stream(y + e, b[j]);
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
#pragma unroll
      for (int l = 0; l < VW; ++l) b[j].v[l] = __fadd_rn(__fmul_rn(alpha, a[j].v[l]), b[j].v[l]);
      st_stream(y + tile * TILE + (int64_t)(threadIdx.x + THREADS * j) * VW, b[j]);
    }
  }
  if (tile == full && full * TILE < n) {
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int64_t first = tile * TILE + (int64_t)(threadIdx.x + THREADS * j) * VW;
#pragma unroll
      for (int l = 0; l < VW; ++l)
        if (first + l < n) y[first + l] = __fadd_rn(__fmul_rn(alpha, x[first + l]), y[first + l]);
    }
  }
}

template <int THREADS, int TILE, int VW, int GRID = 0>
struct Axpy {
  static const void* kernel() { return reinterpret_cast<const void*>(&axpy_ldg<THREADS, TILE, VW>); }
  static int64_t grid(const Variant&, const Args& a) {
    const int64_t T = a.n > 0 ? (a.n + TILE - 1) / TILE : 1;
    return map_grid<GRID>(kernel(), THREADS, 0, T);
  }
  static lift_status launch(const Variant& v, const Args& a, cudaStream_t s) {
    const int64_t g = grid(v, a);
    if (g <= 0) return set_error(LIFT_ERR_CUDA, std::string("no resident CTA for ") + v.info.name);
    int64_t n = a.n;
    float alpha = a.alpha;
    const float* x = static_cast<const float*>(a.x);
    float* y = a.out;
    void* args[] = {&n, &alpha, &x, &y};
    return launch_config(kernel(), dim3((unsigned)g), dim3(THREADS), 0, 1, s, args, true);
  }
};

template <int THREADS, int TILE, int VW, int GRID = 0>
Variant axpy_variant(const char* name) {
  using K = Axpy<THREADS, TILE, VW, GRID>;
  Variant v{};
  v.info.op = LIFT_OP_AXPY;
  v.info.tile = TILE;
  v.info.vw = VW;
  v.info.threads = THREADS;
  v.info.stride = 1;
  v.info.cluster = 1;
  v.info.passes = 1;
  v.info.grid = GRID;
  snprintf(v.info.name, sizeof(v.info.name), "axpy_%s", name);
  v.launch = &K::launch;
  v.grid = &K::grid;
  v.align_bytes = VW * 4;
  v.fallback = 0;
  return v;
}

// ---------------------------------------------------------------------------
// gemv
// ---------------------------------------------------------------------------
template <int VW>
__device__ __forceinline__ void ld_x(const float* p, Vec<VW>& o) {
  if constexpr (VW == 1) {
    o.v[0] = __ldg(p);
  } else {
#pragma unroll
    for (int q = 0; q < VW / 4; ++q) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(p) + q);
      o.v[4 * q] = t.x;
      o.v[4 * q + 1] = t.y;
      o.v[4 * q + 2] = t.z;
      o.v[4 * q + 3] = t.w;
    }
  }
}

template <int WARPS, int VW, int UNROLL>
__global__ void __launch_bounds__(WARPS * kWarp)
    gemv_warp(int64_t M, int64_t N, float alpha, const float* __restrict__ A, int64_t lda,
              const float* __restrict__ x, float beta, float* __restrict__ y) {
  constexpr int64_t kChunk = (int64_t)kWarp * VW;
  pdl_trigger();   // the next call's first kernel may be scheduled (it waits for this one)
  pdl_wait();      // the previous kernel on the stream has completed
  const int lane = threadIdx.x & (kWarp - 1);
  const int64_t gw = (int64_t)blockIdx.x * WARPS + threadIdx.x / kWarp;
  const int64_t total = (int64_t)gridDim.x * WARPS;
  const int64_t chunks = N / kChunk;
  static_assert(kGemvGroup % UNROLL == 0, "an unrolled step stays inside one group");
  for (int64_t row = gw; row < M; row += total) {
    const float* a = A + row * lda;
    GroupedDot<VW> acc;
    acc.init();
    int64_t c = 0;                     // the lane's vector index along the row
    for (; c + UNROLL <= chunks; c += UNROLL) {
      Vec<VW> va[UNROLL], vx[UNROLL];
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const int64_t e = (c + u) * kChunk + lane * VW;
        ld_stream(a + e, va[u]);
        ld_x<VW>(x + e, vx[u]);
      }
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) acc.add(va[u], vx[u]);
      if (((c + UNROLL) & (kGemvGroup - 1)) == 0) acc.flush();
    }
    for (; c < chunks; ++c) {
      Vec<VW> va, vx;
      const int64_t e = c * kChunk + lane * VW;
      ld_stream(a + e, va);
      ld_x<VW>(x + e, vx);
      acc.add(va, vx);
      if (((c + 1) & (kGemvGroup - 1)) == 0) acc.flush();
    }
    if (chunks * kChunk < N) {
      Vec<VW> va, vx;
      const int64_t e = chunks * kChunk + lane * VW;
      ld_guarded<VW>(a, e, N, va);
      ld_guarded<VW>(x, e, N, vx);
      acc.add(va, vx);
    }
    float r = warp_tree(acc.value());
    if (lane == 0) {
      const float z = __fmul_rn(alpha, r);
      y[row] = (beta == 0.0f) ? z : __fadd_rn(z, __fmul_rn(beta, y[row]));
    }
  }
}

// N == 0: every row's dot is the empty sum z = 0, so y <- fl(0 + fl(beta * y))
// (and y <- 0 when beta == 0).
__global__ void gemv_scale_y(int64_t M, float beta, float* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (beta == 0.0f) ? 0.0f : __fadd_rn(0.0f, __fmul_rn(beta, y[i]));
}

// GRID 0: at most the resident CTAs, each warp taking rows round robin;
// GRID 1: one CTA per WARPS rows (capped at 2^31 - 1 CTAs; the row loop
// still covers every row), dealt to the SMs by the hardware.
template <int WARPS, int VW, int UNROLL, int GRID = 0>
struct Gemv {
  static const void* kernel() { return reinterpret_cast<const void*>(&gemv_warp<WARPS, VW, UNROLL>); }
  static int64_t grid(const Variant&, const Args& a) {
    const int64_t need = (a.M + WARPS - 1) / WARPS;
    int64_t g = GRID == 1 ? INT32_MAX : persistent_grid(kernel(), WARPS * kWarp, 0, 1);
    if (need < g) g = need;
    return g < 1 ? 1 : g;
  }
  static lift_status launch(const Variant& v, const Args& a, cudaStream_t s) {
    if (a.M == 0) return LIFT_OK;
    float* y = a.out;
    if (a.N == 0) {
      gemv_scale_y<<<64, 256, 0, s>>>(a.M, a.beta, y);
      return cuda_check(cudaGetLastError(), "gemv_scale_y launch");
    }
    const int64_t g = grid(v, a);
    int64_t M = a.M, N = a.N, lda = a.lda;
    float alpha = a.alpha, beta = a.beta;
    const float* A = a.A;
    const float* x = static_cast<const float*>(a.x);
    void* args[] = {&M, &N, &alpha, &A, &lda, &x, &beta, &y};
    return launch_config(kernel(), dim3((unsigned)g), dim3(WARPS * kWarp), 0, 1, s, args, true);
  }
};

template <int WARPS, int VW, int UNROLL, int GRID = 0>
Variant gemv_variant(const char* name) {
  using K = Gemv<WARPS, VW, UNROLL, GRID>;
  Variant v{};
  v.info.op = LIFT_OP_GEMV;
  v.info.tile = 0;
  v.info.vw = VW;
  v.info.threads = WARPS * kWarp;
  v.info.stride = 1;
  v.info.tree = 0;
  v.info.cluster = 1;
  v.info.passes = 1;
  v.info.stages = 0;
  v.info.rows = WARPS;
  v.info.lanes = kWarp;
  v.info.grid = GRID;
  snprintf(v.info.name, sizeof(v.info.name), "gemv_%s", name);
  v.launch = &K::launch;
  v.grid = &K::grid;
  v.align_bytes = VW * 4;
  v.fallback = 0;
  return v;
}

}  // namespace

void register_scal(std::vector<Variant>& L) {
  L.push_back(scal_variant<256, 1024, 1, 0>("t1024_v1_ldg"));
  L.push_back(scal_variant<256, 256, 1, 0>("t256_v1_ldg"));
  L.push_back(scal_variant<256, 512, 1, 0>("t512_v1_ldg"));
  L.push_back(scal_variant<256, 2048, 1, 0>("t2048_v1_ldg"));
  L.push_back(scal_variant<256, 4096, 1, 0>("t4096_v1_ldg"));
  L.push_back(scal_variant<256, 1024, 4, 0>("t1024_v4_ldg"));
  L.push_back(scal_variant<256, 2048, 4, 0>("t2048_v4_ldg"));
  L.push_back(scal_variant<256, 4096, 4, 0>("t4096_v4_ldg"));
  L.push_back(scal_variant<256, 2048, 8, 0>("t2048_v8_ldg"));
  L.push_back(scal_variant<256, 4096, 8, 0>("t4096_v8_ldg"));
  L.push_back(scal_variant<256, 1024, 4, 4>("t1024_tma4"));
  L.push_back(scal_variant<256, 2048, 4, 4>("t2048_tma4"));
  L.push_back(scal_variant<256, 4096, 4, 4>("t4096_tma4"));
  L.push_back(scal_variant<256, 4096, 4, 2>("t4096_tma2"));
  L.push_back(scal_variant<256, 4096, 4, 6>("t4096_tma6"));
  // one CTA per tile (appended: earlier ids are stable)
  L.push_back(scal_variant<256, 2048, 4, 0, 1>("t2048_v4_ldg_pertile"));
  L.push_back(scal_variant<256, 4096, 4, 0, 1>("t4096_v4_ldg_pertile"));
  L.push_back(scal_variant<256, 4096, 8, 0, 1>("t4096_v8_ldg_pertile"));
  L.push_back(scal_variant<256, 8192, 8, 0, 1>("t8192_v8_ldg_pertile"));
  for (size_t i = 0; i < L.size(); ++i) L[i].info.id = static_cast<int>(i);
}

void register_axpy(std::vector<Variant>& L) {
  L.push_back(axpy_variant<256, 1024, 1>("t1024_v1_ldg"));
  L.push_back(axpy_variant<256, 1024, 4>("t1024_v4_ldg"));
  L.push_back(axpy_variant<256, 2048, 4>("t2048_v4_ldg"));
  L.push_back(axpy_variant<256, 4096, 4>("t4096_v4_ldg"));
  L.push_back(axpy_variant<256, 2048, 8>("t2048_v8_ldg"));
  L.push_back(axpy_variant<256, 2048, 4, 1>("t2048_v4_ldg_pertile"));
  L.push_back(axpy_variant<256, 4096, 4, 1>("t4096_v4_ldg_pertile"));
  L.push_back(axpy_variant<256, 4096, 8, 1>("t4096_v8_ldg_pertile"));
  for (size_t i = 0; i < L.size(); ++i) L[i].info.id = static_cast<int>(i);
}

void register_gemv(std::vector<Variant>& L) {
  L.push_back(gemv_variant<8, 1, 8>("w8_v1_u8"));
  L.push_back(gemv_variant<8, 4, 4>("w8_v4_u4"));
  L.push_back(gemv_variant<8, 4, 8>("w8_v4_u8"));
  L.push_back(gemv_variant<8, 8, 2>("w8_v8_u2"));
  L.push_back(gemv_variant<8, 8, 4>("w8_v8_u4"));
  L.push_back(gemv_variant<4, 4, 4>("w4_v4_u4"));
  L.push_back(gemv_variant<4, 8, 2>("w4_v8_u2"));
  L.push_back(gemv_variant<16, 4, 4>("w16_v4_u4"));
  for (size_t i = 0; i < L.size(); ++i) L[i].info.id = static_cast<int>(i);
}

// One CTA per WARPS rows; registered after every other gemv family so that
// earlier ids stay stable.
void register_gemv_pertile(std::vector<Variant>& L) {
  L.push_back(gemv_variant<8, 4, 4, 1>("w8_v4_u4_pertile"));
  L.push_back(gemv_variant<8, 8, 2, 1>("w8_v8_u2_pertile"));
  L.push_back(gemv_variant<8, 8, 4, 1>("w8_v8_u4_pertile"));
  L.push_back(gemv_variant<4, 8, 2, 1>("w4_v8_u2_pertile"));
  L.push_back(gemv_variant<4, 4, 4, 1>("w4_v4_u4_pertile"));
  for (size_t i = 0; i < L.size(); ++i) L[i].info.id = static_cast<int>(i);
}

}  // namespace lift
