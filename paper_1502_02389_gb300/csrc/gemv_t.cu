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
  pdl_wait();      // the previous kernel on the stream has completed
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
  pdl_trigger();   // the next call's first kernel may be scheduled (it waits for this one)
  pdl_wait();      // the first pass has finished
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

// Staged form (the toLocal lowering of Fig. 4d applied to the column
// block's rows): the same expression and blocks as the two-pass kernel --
// per column, the block's rows in groups of 32 folded in row order from
// zero, the group sums added with Neumaier's compensated step, one partial
// per (column, block) written column-major for gemv_t_combine -- so both
// give the same bits.  Only the movement of A differs: one producer warp
// streams the block's rows, R at a time, into a ring of S shared-memory
// stages with one bulk copy per row segment (cw = min(CB, N - first
// column) floats, contiguous in A), a full mbarrier per stage counting the
// bytes in and an empty mbarrier counting the consumer warps that have read
// it; consumer thread t folds column quads t, t + THREADS, ... of every
// staged row (a warp reads 512 contiguous bytes of shared memory per quad).
// The copy engine moves whole row segments of 2-8 KB, where the direct
// kernel's warps each issue 512-byte pieces of rows lda apart.  Requires A
// and x 16-byte aligned and N, lda multiples of 4; R divides 32 so that no
// stage straddles a group.  A wait that runs out (the limit set with
// lift_set_wait_polls) records LIFT_ERR_TIMEOUT: a consumer warp stops as a
// whole and writes NaN partials, and the side that stops waits, with the
// full limit, for every copy that may still be in flight into the ring, so
// none lands after the CTA has left.
template <int THREADS, int VW, int R, int S>
__global__ void __launch_bounds__(THREADS + kWarp, 1)
    gemv_t_staged(int64_t M, int64_t N, const float* __restrict__ A, int64_t lda,
                  const float* __restrict__ x, int64_t B, float* __restrict__ partials,
                  int* status, uint32_t polls) {
  constexpr int CB = THREADS * VW, Q = VW / 4, WARPS = THREADS / kWarp;
  static_assert(VW % 4 == 0 && kGroupRows % R == 0 && R % 4 == 0, "quads; stages within groups");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* buf = reinterpret_cast<float*>(smem_raw);
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ __align__(8) uint64_t empty_bar[S];
  const int64_t cb = blockIdx.x, rb = blockIdx.y, RB = gridDim.y;
  const int64_t col0 = cb * CB;
  const int64_t cw = N - col0 < CB ? N - col0 : CB;
  const int64_t r0 = rb * B, r1 = (r0 + B < M) ? r0 + B : M;
  const int64_t steps = r1 > r0 ? (r1 - r0 + R - 1) / R : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], WARPS);
    }
    fence_mbar_init();
  }
  pdl_wait();      // the previous kernel on the stream has completed
  __syncthreads();

  if (threadIdx.x >= THREADS) {
    // producer warp: one lane streams the block's row segments into the ring
    if (threadIdx.x == THREADS) {
      const uint32_t bytes = static_cast<uint32_t>(cw * sizeof(float));
      for (int64_t k = 0; k < steps; ++k) {
        const int s = static_cast<int>(k % S);
        if (k >= S && !mbar_wait(&empty_bar[s], static_cast<uint32_t>(((k / S) - 1) & 1), polls)) {
          report(status, LIFT_ERR_TIMEOUT);
          for (int64_t q = k - S; q < k; ++q)       // steps whose copies may be in flight
            mbar_wait(&full_bar[q % S], static_cast<uint32_t>((q / S) & 1));
          return;
        }
        const int64_t i0 = r0 + k * R;
        const int rows = static_cast<int>(r1 - i0 < R ? r1 - i0 : R);
        float* st = buf + (size_t)s * R * CB;
        mbar_arrive_expect_tx(&full_bar[s], rows * bytes);
        for (int r = 0; r < rows; ++r)
          bulk_g2s(st + r * CB, A + (i0 + r) * lda + col0, bytes, &full_bar[s]);
      }
    }
    return;
  }

  const int lane = threadIdx.x & (kWarp - 1);
  float acc[VW], cmp[VW], gs[VW];
#pragma unroll
  for (int l = 0; l < VW; ++l) acc[l] = cmp[l] = gs[l] = 0.f;
  bool failed = false;
  for (int64_t k = 0; k < steps; ++k) {
    const int s = static_cast<int>(k % S);
    if (!__all_sync(0xffffffffu, mbar_wait(&full_bar[s], static_cast<uint32_t>((k / S) & 1), polls))) {
      // the producer issues no step past k + S - 1 before this warp's
      // arrival for step k, which never comes
      if (threadIdx.x == 0) {
        report(status, LIFT_ERR_TIMEOUT);
        for (int64_t q = k; q < k + S && q < steps; ++q)
          mbar_wait(&full_bar[q % S], static_cast<uint32_t>((q / S) & 1));
      }
      failed = true;
      break;
    }
    const int64_t i0 = r0 + k * R;
    const float* st = buf + (size_t)s * R * CB;
    if (i0 + R <= r1) {
      float xv[R];
#pragma unroll
      for (int u = 0; u < R; u += 4) {          // i0 is a multiple of 4, x 16-byte aligned
        const float4 q = __ldg(reinterpret_cast<const float4*>(x + i0 + u));
        xv[u] = q.x;
        xv[u + 1] = q.y;
        xv[u + 2] = q.z;
        xv[u + 3] = q.w;
      }
#pragma unroll
      for (int qd = 0; qd < Q; ++qd) {
        const int c = (qd * THREADS + threadIdx.x) * 4;
        if (c < cw) {
          Vec<4> a[R];
#pragma unroll
          for (int r = 0; r < R; ++r) ld_smem<4>(st + r * CB + c, a[r]);
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int l = 0; l < 4; ++l)
              gs[qd * 4 + l] = __fadd_rn(gs[qd * 4 + l], __fmul_rn(a[r].v[l], xv[r]));
        }
      }
    } else {
      const int rows = static_cast<int>(r1 - i0);
      for (int r = 0; r < rows; ++r) {
        const float xr = __ldg(x + i0 + r);
#pragma unroll
        for (int qd = 0; qd < Q; ++qd) {
          const int c = (qd * THREADS + threadIdx.x) * 4;
          if (c < cw) {
            Vec<4> a;
            ld_smem<4>(st + r * CB + c, a);
#pragma unroll
            for (int l = 0; l < 4; ++l)
              gs[qd * 4 + l] = __fadd_rn(gs[qd * 4 + l], __fmul_rn(a.v[l], xr));
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0)
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&empty_bar[s]))
                   : "memory");
    // a group of 32 rows ends here, or the block does
    if (((k + 1) * R) % kGroupRows == 0 || k + 1 == steps) {
#pragma unroll
      for (int l = 0; l < VW; ++l) {
        neumaier_add(acc[l], cmp[l], gs[l]);
        gs[l] = 0.f;
      }
    }
  }
  // the combine kernel may start launching; it waits for this grid to end
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#pragma unroll
  for (int qd = 0; qd < Q; ++qd) {
    const int64_t c = (qd * THREADS + threadIdx.x) * 4;
    if (c < cw) {
#pragma unroll
      for (int l = 0; l < 4; ++l)
        partials[(col0 + c + l) * RB + rb] =
            failed ? __int_as_float(0x7fc00000) : neumaier_value(acc[qd * 4 + l], cmp[qd * 4 + l]);
    }
  }
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
    lift_status r =
        launch_config(kernel(), dim3((unsigned)ncb, (unsigned)RB), dim3(THREADS), 0, 1, s, args, true);
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

template <int THREADS, int VW, int R, int S>
struct GemvTStaged {
  static constexpr int CB = THREADS * VW;
  static const void* kernel() {
    return reinterpret_cast<const void*>(&gemv_t_staged<THREADS, VW, R, S>);
  }
  static size_t smem() { return (size_t)S * R * CB * sizeof(float); }
  // at most one wave of the persistent size (row blocks rounded down: with
  // two to four CTAs per SM a second, nearly empty wave costs a whole
  // block's time), within the partials workspace and kMaxRowBlocks2 row
  // blocks
  static void shape(const Args& a, int64_t& ncb, int64_t& RB, int64_t& B) {
    ncb = (a.N + CB - 1) / CB;
    const int64_t g = persistent_grid(kernel(), THREADS + kWarp, smem(), 1);
    int64_t want = g > ncb ? g / ncb : 1;
    DeviceState* st = current_state();
    const int64_t cap = st ? st->ws.capacity / (a.N > 0 ? a.N : 1) : 1;
    if (want > cap) want = cap;
    if (want > kMaxRowBlocks2) want = kMaxRowBlocks2;
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
    if (a.N % 4 != 0 || a.lda % 4 != 0 || !aligned(a.A, 16) || !aligned(a.x, 16))
      return set_error(LIFT_ERR_UNSUPPORTED, "staged gemv_t: N, lda, A or x not in 16-byte granules");
    int64_t ncb, RB, B;
    shape(a, ncb, RB, B);
    if (RB * a.N > st->ws.capacity)
      return set_error(LIFT_ERR_UNSUPPORTED, "gemv_t: N exceeds the partials workspace");
    if (RB > 65535) return set_error(LIFT_ERR_UNSUPPORTED, "gemv_t: too many row blocks");
    int64_t M = a.M, N = a.N, lda = a.lda;
    const float* A = a.A;
    const float* x = static_cast<const float*>(a.x);
    float* partials = a.ws->partials;
    int* status = a.ws->status;
    uint32_t polls = wait_polls();
    void* args[] = {&M, &N, &A, &lda, &x, &B, &partials, &status, &polls};
    lift_status r = launch_config(kernel(), dim3((unsigned)ncb, (unsigned)RB), dim3(THREADS + kWarp),
                                  smem(), 1, s, args, true);
    if (r != LIFT_OK) return r;
    return launch_rows_combine(N, RB, a.alpha, a.beta, partials, a.out, s);
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

// staged forms (appended after the cluster forms): THREADS consumer threads,
// VW columns each, R rows per stage, S stages (16-32 KB stages, two to four
// CTAs per SM)
#define LIFT_GEMV_T_STAGED_VARIANTS(X) \
  X(64, 4, 32, 3, "t64_v4_r32_s3")     \
  X(128, 4, 16, 3, "t128_v4_r16_s3")   \
  X(128, 4, 16, 2, "t128_v4_r16_s2")   \
  X(128, 4, 8, 3, "t128_v4_r8_s3")     \
  X(32, 4, 32, 3, "t32_v4_r32_s3")     \
  X(64, 4, 16, 3, "t64_v4_r16_s3")

template <int THREADS, int VW, int R, int S>
Variant gemv_t_staged_variant(const char* name) {
  using K = GemvTStaged<THREADS, VW, R, S>;
  Variant v = gemv_t_variant<THREADS, VW, 1, 2>(name);
  v.info.threads = THREADS + kWarp;
  v.info.rows = R;
  v.info.stages = S;
  v.launch = &K::launch;
  v.grid = &K::grid;
  v.align_bytes = 16;
  return v;
}

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
#define X(T, V, R, S, NAME) \
  if (k++ == id) GemvTStaged<T, V, R, S>::shape(a, ncb, rb, b);
  LIFT_GEMV_T_STAGED_VARIANTS(X)
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
#define X(T, V, R, S, NAME) L.push_back(gemv_t_staged_variant<T, V, R, S>(NAME));
  LIFT_GEMV_T_STAGED_VARIANTS(X)
#undef X
  for (size_t i = 0; i < L.size(); ++i) L[i].info.id = static_cast<int>(i);
}

}  // namespace lift
