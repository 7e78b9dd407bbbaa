// gemv-T: y <- alpha * A^T x + beta * y for a row-major M x N matrix A
// (x: M floats, y: N floats).
//
// In the pattern language the transpose is an index function: the columns
// of A are the rows of  split^M . reorder-stride^N . join (A)  (Sec. 3.2,
// "Reorder-stride"), so gemv-T is the Fig. 5 gemv over that reordered
// matrix:  z_j = alpha * dot(col_j, x),  y'_j = z_j + beta * y_j.
// The kernels evaluate, per column j,
//
//   map(mult(alpha)) . COMBINE . join . map(BLOCK) . split^B . pad-(RB*B)
//     . zip(col_j, x)
//   BLOCK = reduce-seq-comp . join . map(reduce-seq(lambda acc,(a,b):
//             acc + a*b, 0)) . split^32 . pad
// (reduce-seq-comp: Neumaier's compensated reduce-seq)
//
// i.e. the column is split into RB uniform blocks of B rows (the last one
// padded with zeros); CTA (cb, rb) folds the rows of block rb -- in groups
// of 32 rows folded in order, the group sums added with Neumaier's
// compensated step -- for
// its THREADS*VW consecutive columns (thread t owns VW adjacent columns, so
// a warp reads 32*VW*4 contiguous bytes of every row) and writes one fp32
// partial per column.  The two lowerings of COMBINE are a rewrite choice:
//   one pass:  reduce-seq-comp over the RB partials in block order, done
//              by the last CTA of each column block (an atomic ticket per
//              column block); row-major partials P[rb][j];
//   two pass:  a second kernel, one warp per column: lane l folds partials
//              l, l+32, ... , then a halving tree over the 32 lanes;
//              column-major partials P[j][rb] so that a warp's loads are
//              contiguous.  The second kernel is launched as a programmatic
//              dependent of the first and waits on it with
//              griddepcontrol.wait, which hides its launch latency.
// The combine is fp32: its rounding error (at most ceil(log2 RB) or RB - 1
// units of fp32 roundoff) is no larger than that of the B-row fold before
// it, and FP64 arithmetic runs at a small fraction of the fp32 rate on this
// part, which made an FP64 combine of the N x RB partials cost as much as
// streaming A.  The epilogue multiplies by alpha and adds fl(beta * y_j) (y
// is not read when beta == 0).
#include <cooperative_groups.h>

#include "lift_internal.cuh"

namespace cg = cooperative_groups;

namespace lift {

extern const int kTicketSlots;     // counters in the workspace (api.cu)

lift_status launch_rows_combine(int64_t n, int64_t per, float alpha, float beta,
                                const float* partials, float* y, cudaStream_t s);

namespace {

// Rows folded plainly before a compensated add (see fold_rows).
constexpr int kGroupRows = 32;

// Row block [r0, r1) of this thread's VW columns c0 .. c0+VW-1 (zero for an
// empty block): the rows in groups of kGroupRows, each group's products
// folded in row order from zero (U rows of loads in flight at a time), and
// the group sums added with Neumaier's compensated step (the partial
// reduction of Fig. 3d within the block's reduce-seq), so the error of a
// column's block value does not grow with the block length.
template <int VW, int U>
__device__ __forceinline__ void fold_rows(int64_t N, const float* __restrict__ A, int64_t lda,
                                          const float* __restrict__ x, int64_t c0, int64_t r0,
                                          int64_t r1, float* acc) {
  static_assert(kGroupRows % U == 0, "a group holds whole unrolled steps");
  float cmp[VW];
#pragma unroll
  for (int l = 0; l < VW; ++l) acc[l] = cmp[l] = 0.f;
  const bool full_cols = c0 + VW <= N;
  for (int64_t i = r0; i < r1;) {
    const int64_t ge = i + kGroupRows < r1 ? i + kGroupRows : r1;
    float gs[VW];
#pragma unroll
    for (int l = 0; l < VW; ++l) gs[l] = 0.f;
    if (full_cols) {
      for (; i + U <= ge; i += U) {
        Vec<VW> a[U];
        float xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) ld_stream(A + (i + u) * lda + c0, a[u]);
        if constexpr (VW >= 4 && U % 4 == 0) {
          // row blocks start at multiples of 4 rows and x is 16-byte aligned
          // for these variants: x[i .. i+U) in 16-byte loads
#pragma unroll
          for (int u = 0; u < U; u += 4) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(x + i + u));
            xv[u] = q.x;
            xv[u + 1] = q.y;
            xv[u + 2] = q.z;
            xv[u + 3] = q.w;
          }
        } else {
#pragma unroll
          for (int u = 0; u < U; ++u) xv[u] = __ldg(x + i + u);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int l = 0; l < VW; ++l) gs[l] = __fadd_rn(gs[l], __fmul_rn(a[u].v[l], xv[u]));
      }
      for (; i < ge; ++i) {
        Vec<VW> a;
        ld_stream(A + i * lda + c0, a);
        const float xv = __ldg(x + i);
#pragma unroll
        for (int l = 0; l < VW; ++l) gs[l] = __fadd_rn(gs[l], __fmul_rn(a.v[l], xv));
      }
    } else {
      for (; i < ge; ++i) {
        const float xv = __ldg(x + i);
#pragma unroll
        for (int l = 0; l < VW; ++l)
          if (c0 + l < N) gs[l] = __fadd_rn(gs[l], __fmul_rn(__ldg(A + i * lda + c0 + l), xv));
      }
    }
#pragma unroll
    for (int l = 0; l < VW; ++l) neumaier_add(acc[l], cmp[l], gs[l]);
  }
#pragma unroll
  for (int l = 0; l < VW; ++l) acc[l] = neumaier_value(acc[l], cmp[l]);
}

template <int THREADS, int VW, int U, int PASSES>
__global__ void __launch_bounds__(THREADS)
    gemv_t_kernel(int64_t M, int64_t N, float alpha, const float* __restrict__ A, int64_t lda,
                  const float* __restrict__ x, float beta, float* __restrict__ y, int64_t B,
                  float* __restrict__ partials, unsigned* __restrict__ tickets) {
  constexpr int CB = THREADS * VW;
  const int64_t cb = blockIdx.x, rb = blockIdx.y, RB = gridDim.y;
  const int64_t c0 = cb * CB + (int64_t)threadIdx.x * VW;
  const int64_t r0 = rb * B, r1 = (r0 + B < M) ? r0 + B : M;
  float acc[VW];
  fold_rows<VW, U>(N, A, lda, x, c0, r0, r1, acc);

  if constexpr (PASSES == 2) {
    // the combine kernel may start launching; it waits for this grid to end
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#pragma unroll
    for (int l = 0; l < VW; ++l)
      if (c0 + l < N) partials[(c0 + l) * RB + rb] = acc[l];
  } else {
#pragma unroll
    for (int l = 0; l < VW; ++l)
      if (c0 + l < N) partials[rb * N + c0 + l] = acc[l];

    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      is_last = atomicAdd(tickets + cb, 1u) == static_cast<unsigned>(RB - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
#pragma unroll
    for (int l = 0; l < VW; ++l) {
      const int64_t j = c0 + l;
      if (j >= N) continue;
      float s = 0.f, c = 0.f;              // block partials added in order, compensated
      int64_t q = 0;
      for (; q + 8 <= RB; q += 8) {        // eight loads in flight
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = __ldcg(partials + (q + k) * N + j);
#pragma unroll
        for (int k = 0; k < 8; ++k) neumaier_add(s, c, v[k]);
      }
      for (; q < RB; ++q) neumaier_add(s, c, __ldcg(partials + q * N + j));
      const float z = __fmul_rn(alpha, neumaier_value(s, c));
      y[j] = beta == 0.f ? z : __fadd_rn(z, __fmul_rn(beta, y[j]));
    }
    if (threadIdx.x == 0) tickets[cb] = 0u;   // ready for the next call
  }
}

// Second pass: column j's RB partials P[j][0..RB) -> y_j.  Warp w of the
// grid takes columns w, w + W, ...; lane l folds partials l, l+32, ...
// (eight loads in flight, added in order with Neumaier's compensated step),
// then a halving tree over the lanes (shuffle-down 16, 8, 4, 2, 1).
__global__ void __launch_bounds__(256)
    gemv_t_combine(int64_t N, int64_t RB, float alpha, float beta,
                   const float* __restrict__ partials, float* __restrict__ y) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int lane = threadIdx.x & (kWarp - 1);
  const int64_t W = (int64_t)gridDim.x * (blockDim.x / kWarp);
  for (int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp; j < N; j += W) {
    const float* p = partials + j * RB;
    float s = 0.f, c = 0.f;              // the lane's partials in order, compensated
    int64_t q = lane;
    for (; q + 7 * kWarp < RB; q += 8 * kWarp) {
      float v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = __ldcg(p + q + k * kWarp);
#pragma unroll
      for (int k = 0; k < 8; ++k) neumaier_add(s, c, v[k]);
    }
    for (; q < RB; q += kWarp) neumaier_add(s, c, __ldcg(p + q));
    s = neumaier_value(s, c);
#pragma unroll
    for (int o = kWarp / 2; o > 0; o >>= 1) s = __fadd_rn(s, __shfl_down_sync(0xffffffffu, s, o));
    if (lane == 0) {
      const float z = __fmul_rn(alpha, s);
      y[j] = beta == 0.f ? z : __fadd_rn(z, __fmul_rn(beta, y[j]));
    }
  }
}

// Cluster form (one launch): the RB row blocks of a column block are
// grouped CL to a thread-block cluster along gridDim.y.  Each CTA folds its
// block into shared memory; after a cluster barrier, CTA of rank q adds, for
// the columns of slice q (CB / CL of them), the CL block partials of its
// cluster in rank (= block) order through distributed shared memory, and
// writes one partial per column and cluster, P[c][j] (c = rb / CL).  The
// CTA that arrives last at the ticket of (column block, slice) adds the
// RB / CL cluster partials of the slice's columns in cluster order with
// Neumaier's compensated step (sixteen loads in flight) and writes y.  Per
// column:
//   s = reduce-seq-comp over clusters of reduce-seq(add, 0) over the CL
//       block partials of the cluster;   y_j = fl(alpha*s) (+ fl(beta*y_j)).
template <int THREADS, int VW, int U, int CL>
__global__ void __launch_bounds__(THREADS)
    gemv_t_cluster(int64_t M, int64_t N, float alpha, const float* __restrict__ A, int64_t lda,
                   const float* __restrict__ x, float beta, float* __restrict__ y, int64_t B,
                   float* __restrict__ partials, unsigned* __restrict__ tickets) {
  constexpr int CB = THREADS * VW, SL = CB / CL;
  static_assert(CB % CL == 0, "a slice holds whole columns");
  __shared__ __align__(16) float part[CB];
  __shared__ bool is_last;
  const int64_t cb = blockIdx.x, rb = blockIdx.y, RB = gridDim.y, RBC = RB / CL;
  const int64_t c0 = cb * CB + (int64_t)threadIdx.x * VW;
  const int64_t r0 = rb * B, r1 = (r0 + B < M) ? r0 + B : M;
  float acc[VW];
  fold_rows<VW, U>(N, A, lda, x, c0, r0, r1, acc);     // empty past M (padding blocks)
#pragma unroll
  for (int l = 0; l < VW; ++l) part[threadIdx.x * VW + l] = acc[l];

  cg::cluster_group cl = cg::this_cluster();
  cl.sync();                                    // every block partial of the cluster written
  const int q = static_cast<int>(cl.block_rank());
  const int64_t c = rb / CL;
  for (int k = threadIdx.x; k < SL; k += THREADS) {
    const int col = q * SL + k;
    float p = 0.f;
#pragma unroll
    for (int r = 0; r < CL; ++r) p = __fadd_rn(p, *cl.map_shared_rank(part + col, r));
    const int64_t j = cb * CB + col;
    if (j < N) partials[c * N + j] = p;
  }
  cl.sync();                                    // peers done reading this CTA's partials
  unsigned* ticket = tickets + cb * CL + q;
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(ticket, 1u) == static_cast<unsigned>(RBC - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int k = threadIdx.x; k < SL; k += THREADS) {
    const int64_t j = cb * CB + q * SL + k;
    if (j >= N) continue;
    float s = 0.f, c = 0.f;                     // cluster partials in order, compensated
    int64_t e = 0;
    for (; e + 16 <= RBC; e += 16) {            // sixteen loads in flight
      float v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] = __ldcg(partials + (e + u) * N + j);
#pragma unroll
      for (int u = 0; u < 16; ++u) neumaier_add(s, c, v[u]);
    }
    for (; e < RBC; ++e) neumaier_add(s, c, __ldcg(partials + e * N + j));
    const float z = __fmul_rn(alpha, neumaier_value(s, c));
    y[j] = beta == 0.f ? z : __fadd_rn(z, __fmul_rn(beta, y[j]));
  }
  if (threadIdx.x == 0) *ticket = 0u;           // ready for the next call
}

constexpr int kCombineThreads = 256;
constexpr int64_t kMaxRowBlocks2 = 512;   // two pass: at most 16 partials per lane

constexpr int kTicketBase = 64;    // gemv-T tickets follow the reductions' counters
constexpr int64_t kBlockAlign = 4; // rows per block: a multiple of 4 (16-byte x loads)

template <int THREADS, int VW, int U, int PASSES>
struct GemvT {
  static const void* kernel() {
    return reinterpret_cast<const void*>(&gemv_t_kernel<THREADS, VW, U, PASSES>);
  }
  // (column blocks, row blocks, rows per block): enough CTAs for one wave of
  // the persistent size, within the partials workspace (and, two pass, at
  // most kMaxRowBlocks2 row blocks)
  static void shape(const Args& a, int64_t& ncb, int64_t& RB, int64_t& B) {
    constexpr int CB = THREADS * VW;
    ncb = (a.N + CB - 1) / CB;
    const int64_t g = persistent_grid(kernel(), THREADS, 0, 1);
    int64_t want = g > ncb ? (g + ncb - 1) / ncb : 1;
    DeviceState* st = current_state();
    const int64_t cap = st ? st->ws.capacity / (a.N > 0 ? a.N : 1) : 1;
    if (want > cap) want = cap;
    if (PASSES == 2 && want > kMaxRowBlocks2) want = kMaxRowBlocks2;
    if (want > a.M) want = a.M;
    if (want < 1) want = 1;
    B = (a.M + want - 1) / want;
    B = (B + kBlockAlign - 1) / kBlockAlign * kBlockAlign;
    RB = (a.M + B - 1) / B;
  }
  static int64_t grid(const Variant&, const Args& a) {
    int64_t ncb, RB, B;
    shape(a, ncb, RB, B);
    return ncb * RB;
  }
  static lift_status launch(const Variant& v, const Args& a, cudaStream_t s) {
    DeviceState* st = current_state();
    if (a.N == 0) return LIFT_OK;
    if (a.M == 0) return set_error(LIFT_ERR_UNSUPPORTED, "gemv_t with M == 0 goes through gemv_t_scale");
    int64_t ncb, RB, B;
    shape(a, ncb, RB, B);
    if (PASSES == 1 && ncb > kTicketSlots - kTicketBase)
      return set_error(LIFT_ERR_UNSUPPORTED, "gemv_t: more column blocks than tickets");
    if (RB * a.N > st->ws.capacity)
      return set_error(LIFT_ERR_UNSUPPORTED, "gemv_t: N exceeds the partials workspace");
    int64_t M = a.M, N = a.N, lda = a.lda;
    float alpha = a.alpha, beta = a.beta;
    const float* A = a.A;
    const float* x = static_cast<const float*>(a.x);
    float* y = a.out;
    float* partials = a.ws->partials;
    unsigned* tickets = a.ws->tickets + kTicketBase;
    void* args[] = {&M, &N, &alpha, &A, &lda, &x, &beta, &y, &B, &partials, &tickets};
    lift_status r = launch_config(kernel(), dim3((unsigned)ncb, (unsigned)RB), dim3(THREADS), 0, 1, s, args);
    if (r != LIFT_OK || PASSES == 1) return r;
    return launch_rows_combine(N, RB, alpha, beta, partials, y, s);
  }
};

template <int THREADS, int VW, int U, int CL>
struct GemvTCluster {
  static constexpr int CB = THREADS * VW;
  static const void* kernel() {
    return reinterpret_cast<const void*>(&gemv_t_cluster<THREADS, VW, U, CL>);
  }
  // (column blocks, row blocks padded to a multiple of CL, rows per block):
  // about one wave of the persistent size, rounded down to whole clusters
  static void shape(const Args& a, int64_t& ncb, int64_t& RB, int64_t& B) {
    ncb = (a.N + CB - 1) / CB;
    const int64_t g = persistent_grid(kernel(), THREADS, 0, 1);
    int64_t want = g > ncb ? g / ncb : 1;
    want = want / CL * CL;
    DeviceState* st = current_state();
    const int64_t cap = st ? st->ws.capacity / (a.N > 0 ? a.N : 1) * CL : CL;
    if (want > cap) want = cap / CL * CL;
    if (want > a.M) want = a.M;
    if (want < 1) want = 1;
    B = (a.M + want - 1) / want;
    B = (B + kBlockAlign - 1) / kBlockAlign * kBlockAlign;
    RB = (a.M + B - 1) / B;
    RB = (RB + CL - 1) / CL * CL;
  }
  static int64_t grid(const Variant&, const Args& a) {
    int64_t ncb, RB, B;
    shape(a, ncb, RB, B);
    return ncb * RB;
  }
  static lift_status launch(const Variant& v, const Args& a, cudaStream_t s) {
    DeviceState* st = current_state();
    if (a.N == 0) return LIFT_OK;
    if (a.M == 0) return set_error(LIFT_ERR_UNSUPPORTED, "gemv_t with M == 0 goes through gemv_t_scale");
    int64_t ncb, RB, B;
    shape(a, ncb, RB, B);
    if (ncb * CL > kTicketSlots - kTicketBase)
      return set_error(LIFT_ERR_UNSUPPORTED, "gemv_t: more column slices than tickets");
    if (RB / CL * a.N > st->ws.capacity)
      return set_error(LIFT_ERR_UNSUPPORTED, "gemv_t: N exceeds the partials workspace");
    if (RB > 65535) return set_error(LIFT_ERR_UNSUPPORTED, "gemv_t: too many row blocks");
    int64_t M = a.M, N = a.N, lda = a.lda;
    float alpha = a.alpha, beta = a.beta;
    const float* A = a.A;
    const float* x = static_cast<const float*>(a.x);
    float* y = a.out;
    float* partials = a.ws->partials;
    unsigned* tickets = a.ws->tickets + kTicketBase;
    void* args[] = {&M, &N, &alpha, &A, &lda, &x, &beta, &y, &B, &partials, &tickets};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ncb, (unsigned)RB);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = CL;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cuda_check(cudaLaunchKernelExC(&cfg, kernel(), args), "gemv_t cluster launch");
  }
};

// M == 0: every column's dot is the empty sum, y <- fl(beta * y) (0 if beta == 0)
__global__ void gemv_t_scale(int64_t N, float beta, float* y) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x)
    y[j] = beta == 0.f ? 0.f : __fadd_rn(0.f, __fmul_rn(beta, y[j]));
}

template <int THREADS, int VW, int U, int PASSES>
Variant gemv_t_variant(const char* name) {
  using K = GemvT<THREADS, VW, U, PASSES>;
  Variant v{};
  v.info.op = LIFT_OP_GEMV_T;
  v.info.tile = THREADS * VW;
  v.info.vw = VW;
  v.info.threads = THREADS;
  v.info.stride = 1;
  v.info.cluster = 1;
  v.info.passes = PASSES;
  v.info.rows = U;
  v.info.lanes = 1;
  v.info.final_threads = PASSES == 2 ? kWarp : 1;
  snprintf(v.info.name, sizeof(v.info.name), "gemv_t_%s", name);
  v.launch = &K::launch;
  v.grid = &K::grid;
  v.align_bytes = VW * 4;
  v.fallback = 0;
  return v;
}

}  // namespace

// The second pass of gemv-T and of the split-row gemv: n outputs, each from
// `per` consecutive fp32 partials, launched as a programmatic dependent of
// the kernel before it on the stream.
lift_status launch_rows_combine(int64_t n, int64_t per, float alpha, float beta,
                                const float* partials, float* y, cudaStream_t s) {
  const void* k = reinterpret_cast<const void*>(&gemv_t_combine);
  const int64_t warps = kCombineThreads / kWarp;
  int64_t g = (n + warps - 1) / warps;
  const int64_t gmax = persistent_grid(k, kCombineThreads, 0, 1);
  if (g > gmax) g = gmax;
  if (g < 1) g = 1;
  void* args[] = {&n, &per, &alpha, &beta, &partials, &y};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g);
  cfg.blockDim = dim3(kCombineThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cuda_check(cudaLaunchKernelExC(&cfg, k, args), "partials combine launch");
}

lift_status gemv_t_empty_rows(int64_t N, float beta, float* y, cudaStream_t s) {
  if (N == 0) return LIFT_OK;
  gemv_t_scale<<<64, 256, 0, s>>>(N, beta, y);
  return cuda_check(cudaGetLastError(), "gemv_t_scale launch");
}

#define LIFT_GEMV_T_VARIANTS(X)      \
  X(256, 1, 8, 1, "t256_v1_u8")      \
  X(128, 4, 8, 1, "t128_v4_u8")      \
  X(256, 1, 8, 2, "t256_v1_u8_p2")   \
  X(256, 4, 4, 2, "t256_v4_u4_p2")   \
  X(256, 4, 8, 2, "t256_v4_u8_p2")   \
  X(128, 4, 8, 2, "t128_v4_u8_p2")   \
  X(128, 8, 4, 2, "t128_v8_u4_p2")   \
  X(64, 4, 8, 2, "t64_v4_u8_p2")

// cluster forms (appended after the others so that variant ids stay put)
#define LIFT_GEMV_T_CLUSTER_VARIANTS(X) \
  X(256, 4, 4, 8, "t256_v4_u4_c8")      \
  X(256, 4, 8, 8, "t256_v4_u8_c8")      \
  X(256, 4, 4, 4, "t256_v4_u4_c4")      \
  X(128, 4, 8, 8, "t128_v4_u8_c8")      \
  X(128, 8, 4, 8, "t128_v8_u4_c8")      \
  X(64, 4, 8, 8, "t64_v4_u8_c8")

template <int THREADS, int VW, int U, int CL>
Variant gemv_t_cluster_variant(const char* name) {
  using K = GemvTCluster<THREADS, VW, U, CL>;
  Variant v = gemv_t_variant<THREADS, VW, U, 1>(name);
  v.info.cluster = CL;
  v.info.tree = 2;
  v.launch = &K::launch;
  v.grid = &K::grid;
  return v;
}

void gemv_t_shape(int id, const Args& a, int64_t* B, int64_t* RB) {
  int64_t ncb = 0, rb = 0, b = 0;
  int k = 0;
#define X(T, V, U, P, NAME) \
  if (k++ == id) GemvT<T, V, U, P>::shape(a, ncb, rb, b);
  LIFT_GEMV_T_VARIANTS(X)
#undef X
#define X(T, V, U, CL, NAME) \
  if (k++ == id) GemvTCluster<T, V, U, CL>::shape(a, ncb, rb, b);
  LIFT_GEMV_T_CLUSTER_VARIANTS(X)
#undef X
  *B = b;
  *RB = rb;
}

void register_gemv_t(std::vector<Variant>& L) {
#define X(T, V, U, P, NAME) L.push_back(gemv_t_variant<T, V, U, P>(NAME));
  LIFT_GEMV_T_VARIANTS(X)
#undef X
#define X(T, V, U, CL, NAME) L.push_back(gemv_t_cluster_variant<T, V, U, CL>(NAME));
  LIFT_GEMV_T_CLUSTER_VARIANTS(X)
#undef X
  for (size_t i = 0; i < L.size(); ++i) L[i].info.id = static_cast<int>(i);
}

}  // namespace lift
