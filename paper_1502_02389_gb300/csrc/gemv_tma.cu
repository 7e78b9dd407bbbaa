// gemv with TMA bulk-copy staging (arXiv 1502.02389, Fig. 5 gemv; the
// toLocal lowering of Fig. 4d applied to the rows and to x).
//
// Same low-level expression as the warp-per-row kernel with 128-bit vectors:
// map-workgroup over blocks of WARPS rows, map-local over the 32 lanes of a
// row's warp, lane l folding vectors l, l+32, ... of the row zipped with x,
// lane sum, warp halving tree, epilogue fl(fl(alpha * d) + fl(beta * y)).
// Only the staging differs: each CTA owns a balanced contiguous range of
// rows, and one extra producer warp streams, block after block and chunk
// after chunk, the WARPS row segments of C columns plus the matching
// segment of x into a ring of S shared-memory stages with cp.async.bulk; a
// full mbarrier per stage counts the bytes in, an empty mbarrier per stage
// counts the consumer warps that have read it.  Requires A and x 16-byte
// aligned, lda and N multiples of 4 (the library uses the 4-byte-load kernel
// otherwise).
//
// With TMAP the producer moves a stage's WARPS row segments in one tensor
// copy (cp.async.bulk.tensor.3d) instead of one bulk copy per row: A is
// described to the copy engine as a 3-D tensor -- 256-float runs, the runs
// of a row, the rows (strides 1 KiB and lda * 4 bytes) -- and a stage is the
// box {256, C / 256, WARPS} at run C / 256 * chunk, row r0: the same
// [WARPS][C] layout in shared memory.  Rows past M and runs past N read as
// zeros; the box always lands whole, so a stage expects its full size.  It
// also needs N a multiple of 256.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "lift_internal.cuh"

namespace lift {
namespace {

// one tensor copy of box {256, C/256, WARPS} at (0, run, row) into dst
__device__ __forceinline__ void tensor_g2s(void* dst, const CUtensorMap* map, int run, int row,
                                           uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(run), "r"(row), "r"(smem_addr(bar))
      : "memory");
}

template <int WARPS, int C, int S, bool TMAP>
__global__ void __launch_bounds__((WARPS + 1) * kWarp, 1)
    gemv_tma(int64_t M, int64_t N, float alpha, const float* __restrict__ A, int64_t lda,
             const float* __restrict__ x, float beta, float* __restrict__ y, int* status,
             const __grid_constant__ CUtensorMap amap) {
  static_assert(C % 128 == 0, "a chunk holds whole 32-lane x float4 rows");
  constexpr int kStageFloats = WARPS * C + C;   // row segments, then x
  constexpr int J = C / 128;                    // float4 per lane per chunk
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* buf = reinterpret_cast<float*>(smem_raw);
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ __align__(8) uint64_t empty_bar[S];
  const int warp = threadIdx.x / kWarp, lane = threadIdx.x & (kWarp - 1);
  const int64_t G = gridDim.x, b = blockIdx.x;
  const int64_t r_begin = M * b / G, r_end = M * (b + 1) / G;
  const int64_t nblocks = (r_end - r_begin + WARPS - 1) / WARPS;
  const int64_t nchunks = (N + C - 1) / C;
  const int64_t total = nblocks * nchunks;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], WARPS);
    }
    fence_mbar_init();
  }
  pdl_trigger();   // the next call's first kernel may be scheduled (it waits for this one)
  pdl_wait();      // the previous kernel on the stream has completed
  __syncthreads();

  if (warp == WARPS) {
    // producer warp: one lane streams the row segments and x into the ring
    if (lane == 0) {
      for (int64_t k = 0; k < total; ++k) {
        const int s = static_cast<int>(k % S);
        if (k >= S && !mbar_wait(&empty_bar[s], static_cast<uint32_t>(((k / S) - 1) & 1))) {
          report(status, LIFT_ERR_TIMEOUT);
          for (int64_t q = k - S + 1; q < k; ++q)   // copies still in flight
            mbar_wait(&full_bar[q % S], static_cast<uint32_t>((q / S) & 1));
          return;
        }
        const int64_t blk = k / nchunks, ch = k % nchunks;
        const int64_t r0 = r_begin + blk * WARPS, c0 = ch * C;
        const int64_t cw = N - c0 < C ? N - c0 : C;
        const uint32_t bytes = static_cast<uint32_t>(cw * sizeof(float));
        const int nrows = static_cast<int>(r_end - r0 < WARPS ? r_end - r0 : WARPS);
        float* st = buf + (size_t)s * kStageFloats;
        if constexpr (TMAP) {
          mbar_arrive_expect_tx(&full_bar[s], (uint32_t)(WARPS * C * sizeof(float)) + bytes);
          tensor_g2s(st, &amap, static_cast<int>(ch * (C / 256)), static_cast<int>(r0),
                     &full_bar[s]);
        } else {
          mbar_arrive_expect_tx(&full_bar[s], (nrows + 1) * bytes);
          for (int r = 0; r < nrows; ++r)
            bulk_g2s(st + r * C, A + (r0 + r) * lda + c0, bytes, &full_bar[s]);
        }
        bulk_g2s(st + WARPS * C, x + c0, bytes, &full_bar[s]);
      }
    }
    return;
  }

  // consumer warps: warp w folds row (block start + w); lane l's vectors of
  // a row are l, l+32, ... (J per chunk), grouped kGemvGroup at a time
  static_assert(J % kGemvGroup == 0 || kGemvGroup % J == 0, "groups align with chunks");
  GroupedDot<4> acc;
  acc.init();
  for (int64_t k = 0; k < total; ++k) {
    const int s = static_cast<int>(k % S);
    if (!mbar_wait(&full_bar[s], static_cast<uint32_t>((k / S) & 1))) {
      report(status, LIFT_ERR_TIMEOUT);
      return;
    }
    const int64_t blk = k / nchunks, ch = k % nchunks;
    const int64_t row = r_begin + blk * WARPS + warp;
    const int64_t cw = N - ch * C < C ? N - ch * C : C;
    if (ch == 0) acc.init();
    if (row < r_end) {
      const float* st = buf + (size_t)s * kStageFloats;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int idx = (lane + kWarp * j) * 4;
        Vec<4> a, v;
        if (idx < cw) {
          ld_smem<4>(st + warp * C + idx, a);
          ld_smem<4>(st + WARPS * C + idx, v);
        } else {
          a.v[0] = a.v[1] = a.v[2] = a.v[3] = 0.f;
          v = a;
        }
        acc.add(a, v);
        if constexpr (J % kGemvGroup == 0) {
          if (((j + 1) & (kGemvGroup - 1)) == 0) acc.flush();
        }
      }
      if constexpr (J % kGemvGroup != 0) {   // a group spans several chunks
        if ((ch + 1) % (kGemvGroup / J) == 0) acc.flush();
      }
    }
    __syncwarp();
    if (lane == 0)
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&empty_bar[s]))
                   : "memory");
    if (ch == nchunks - 1 && row < r_end) {
      float r = warp_tree(acc.value());
      if (lane == 0) {
        const float z = __fmul_rn(alpha, r);
        y[row] = beta == 0.f ? z : __fadd_rn(z, __fmul_rn(beta, y[row]));
      }
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

template <int WARPS, int C, int S, bool TMAP>
struct GemvTma {
  static_assert(!TMAP || (C % 256 == 0 && C / 256 <= 256 && WARPS <= 256), "tensor box");
  static const void* kernel() {
    return reinterpret_cast<const void*>(&gemv_tma<WARPS, C, S, TMAP>);
  }
  // A as the 3-D tensor {256, N / 256, M} (strides 1 KiB, lda * 4 bytes)
  static lift_status encode(const Args& a, CUtensorMap* m) {
    auto fn = tensor_map_encoder();
    if (!fn) return set_error(LIFT_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    const cuuint64_t dims[3] = {256, (cuuint64_t)(a.N / 256), (cuuint64_t)a.M};
    const cuuint64_t strides[2] = {256 * sizeof(float), (cuuint64_t)a.lda * sizeof(float)};
    const cuuint32_t box[3] = {256, C / 256, WARPS};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(a.A), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? LIFT_OK : set_error(LIFT_ERR_CUDA, "tensor map encoding failed");
  }
  static size_t smem() { return (size_t)S * (WARPS * C + C) * sizeof(float); }
  static int64_t grid(const Variant&, const Args& a) {
    int64_t g = persistent_grid(kernel(), (WARPS + 1) * kWarp, smem(), 1);
    return g < 1 ? 1 : g;
  }
  static lift_status launch(const Variant& v, const Args& a, cudaStream_t s) {
    if (a.M == 0) return LIFT_OK;
    const int64_t g = grid(v, a);
    int64_t M = a.M, N = a.N, lda = a.lda;
    float alpha = a.alpha, beta = a.beta;
    const float* A = a.A;
    const float* x = static_cast<const float*>(a.x);
    float* y = a.out;
    int* status = current_state()->ws.status;
    alignas(64) CUtensorMap amap{};
    if constexpr (TMAP) {
      // the tensor form needs whole 256-float runs and 16-byte row strides
      if (a.N % 256 != 0 || a.lda % 4 != 0)
        return set_error(LIFT_ERR_UNSUPPORTED, "tensor-map gemv: N % 256 or lda % 4");
      const lift_status rc = encode(a, &amap);
      if (rc != LIFT_OK) return rc;
    }
    void* args[] = {&M, &N, &alpha, &A, &lda, &x, &beta, &y, &status, &amap};
    return launch_config(kernel(), dim3((unsigned)g), dim3((WARPS + 1) * kWarp), smem(), 1, s, args,
                         true);
  }
};

template <int WARPS, int C, int S, bool TMAP = false>
Variant gemv_tma_variant(const char* name) {
  using K = GemvTma<WARPS, C, S, TMAP>;
  Variant v{};
  v.info.op = LIFT_OP_GEMV;
  v.info.tile = C;
  v.info.vw = 4;
  v.info.threads = (WARPS + 1) * kWarp;
  v.info.stride = 1;
  v.info.tree = TMAP ? 3 : 0;     // 3: staged by tensor copies (needs N % 256 == 0)
  v.info.cluster = 1;
  v.info.passes = 1;
  v.info.stages = S;
  v.info.rows = WARPS;
  v.info.lanes = kWarp;
  snprintf(v.info.name, sizeof(v.info.name), "gemv_%s", name);
  v.launch = &K::launch;
  v.grid = &K::grid;
  v.align_bytes = 16;
  v.fallback = 0;
  return v;
}

}  // namespace

void register_gemv_tma(std::vector<Variant>& L) {
  const size_t first = L.size();
  L.push_back(gemv_tma_variant<8, 1024, 4>("tma_w8_c1024_s4"));
  L.push_back(gemv_tma_variant<8, 512, 8>("tma_w8_c512_s8"));
  L.push_back(gemv_tma_variant<8, 2048, 2>("tma_w8_c2048_s2"));
  L.push_back(gemv_tma_variant<4, 1024, 6>("tma_w4_c1024_s6"));
  L.push_back(gemv_tma_variant<8, 1024, 3>("tma_w8_c1024_s3"));
  L.push_back(gemv_tma_variant<16, 512, 6>("tma_w16_c512_s6"));
  for (size_t i = first; i < L.size(); ++i) L[i].info.id = static_cast<int>(i);
}

// variants added after the first sweeps: the tensor-copy forms and smaller
// rings (appended after every other gemv variant, so that the ids of the
// others stay those the timing data and the cost model know)
void register_gemv_tmap(std::vector<Variant>& L) {
  const size_t first = L.size();
  L.push_back(gemv_tma_variant<8, 1024, 3, true>("tmap_w8_c1024_s3"));
  L.push_back(gemv_tma_variant<8, 2048, 2, true>("tmap_w8_c2048_s2"));
  L.push_back(gemv_tma_variant<16, 1024, 2, true>("tmap_w16_c1024_s2"));
  // smaller rings: two or three CTAs per SM, each streaming its own rows
  L.push_back(gemv_tma_variant<8, 1024, 2>("tma_w8_c1024_s2"));
  L.push_back(gemv_tma_variant<4, 2048, 2>("tma_w4_c2048_s2"));
  L.push_back(gemv_tma_variant<4, 1024, 3>("tma_w4_c1024_s3"));
  L.push_back(gemv_tma_variant<2, 2048, 3>("tma_w2_c2048_s3"));
  L.push_back(gemv_tma_variant<4, 2048, 3>("tma_w4_c2048_s3"));
  L.push_back(gemv_tma_variant<4, 4096, 2>("tma_w4_c4096_s2"));
  for (size_t i = first; i < L.size(); ++i) L[i].info.id = static_cast<int>(i);
}

}  // namespace lift
