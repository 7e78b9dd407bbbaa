// gemv with the rows split across CTAs (arXiv 1502.02389, Fig. 5 gemv with
// the partial-reduction rule of Fig. 3 applied to each row's reduce).
//
// The warp-per-row kernels give a row to one warp, so a matrix with fewer
// rows than the GPU has warps leaves most of it idle; these variants give
// each row S segments of L elements (L a multiple of THREADS*VW) and one CTA
// per segment.  Per row r,
//
//   y'_r = epilogue . map(mult(alpha)) . COMBINE . join
//          . map-workgroup(block-tree . lane-sum . join
//                          . map-local(reduce-seq(vect-VW(lambda acc,(a,b): acc + a*b), 0))
//                          . split^J . reorder-stride^THREADS . asVector-VW)
//          . split^L . pad-(S*L) . zip(A_r, x)
//
// thread t of a segment's CTA folds vectors t, t+THREADS, ... in order, adds
// its VW lanes, and the CTA's halving tree (warp trees, then one warp over the
// warp results) gives the segment partial.  COMBINE is the warp-per-row fold
// of the S partials (lane l adds partials l, l+32, ..., then a halving tree
// over the lanes), run by the programmatically dependent second kernel that
// gemv-T uses; with S == 1 the CTA applies the epilogue itself.  The
// epilogue is fl(fl(alpha * d) + fl(beta * y_r)) (y not read when beta == 0).
#include "lift_internal.cuh"

namespace lift {

// second pass shared with gemv-T (gemv_t.cu): out_j from per[j*per .. +per)
lift_status launch_rows_combine(int64_t n, int64_t per, float alpha, float beta,
                                const float* partials, float* y, cudaStream_t s);
// y <- fl(0 + fl(beta * y)) (0 when beta == 0): the N == 0 case (gemv_t.cu)
lift_status gemv_t_empty_rows(int64_t N, float beta, float* y, cudaStream_t s);

namespace {

template <int VW>
__device__ __forceinline__ void ld_x_vec(const float* p, Vec<VW>& o) {
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

template <int THREADS, int VW, int U>
__global__ void __launch_bounds__(THREADS)
    gemv_split(int64_t M, int64_t N, float alpha, const float* __restrict__ A, int64_t lda,
               const float* __restrict__ x, float beta, float* __restrict__ y, int64_t L,
               int64_t S, float* __restrict__ partials) {
  constexpr int64_t kStep = (int64_t)THREADS * VW;
  __shared__ float red[kWarp];
  const int64_t r = blockIdx.x / S, seg = blockIdx.x % S;
  const int64_t c_end = (seg + 1) * L < N ? (seg + 1) * L : N;
  static_assert(kGemvGroup % U == 0, "an unrolled step stays inside one group");
  const float* row = A + r * lda;
  GroupedDot<VW> acc;
  acc.init();
  int64_t k = 0;             // the thread's vector index within the segment
  int64_t c = seg * L + (int64_t)threadIdx.x * VW;
  for (; c + (U - 1) * kStep + VW <= c_end; c += U * kStep, k += U) {
    Vec<VW> a[U], b[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      ld_stream(row + c + u * kStep, a[u]);
      ld_x_vec<VW>(x + c + u * kStep, b[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) acc.add(a[u], b[u]);
    if (((k + U) & (kGemvGroup - 1)) == 0) acc.flush();
  }
  for (; c + VW <= c_end; c += kStep, ++k) {
    Vec<VW> a, b;
    ld_stream(row + c, a);
    ld_x_vec<VW>(x + c, b);
    acc.add(a, b);
    if (((k + 1) & (kGemvGroup - 1)) == 0) acc.flush();
  }
  if (c < c_end) {           // the ragged last vector of the row
    Vec<VW> a, b;
    ld_guarded<VW>(row, c, c_end, a);
    ld_guarded<VW>(x, c, c_end, b);
    acc.add(a, b);
  }
  float d = block_tree<THREADS>(acc.value(), red);
  if (S > 1) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (threadIdx.x != 0) return;
  if (S > 1) {
    partials[r * S + seg] = d;
  } else {
    const float z = __fmul_rn(alpha, d);
    y[r] = beta == 0.f ? z : __fadd_rn(z, __fmul_rn(beta, y[r]));
  }
}

template <int THREADS, int VW, int U>
struct GemvSplit {
  static constexpr int64_t kStep = (int64_t)THREADS * VW;
  static const void* kernel() { return reinterpret_cast<const void*>(&gemv_split<THREADS, VW, U>); }
  // segment length L (a multiple of THREADS*VW) and segments per row S:
  // about one wave of the persistent size over all rows
  static void shape(const Args& a, int64_t& L, int64_t& S) {
    const int64_t g = persistent_grid(kernel(), THREADS, 0, 1);
    int64_t want = a.M > 0 ? (g + a.M - 1) / a.M : 1;
    if (want < 1) want = 1;
    DeviceState* st = current_state();
    const int64_t cap = st && a.M > 0 ? st->ws.capacity / a.M : 1;
    if (want > cap) want = cap > 0 ? cap : 1;
    const int64_t per = (a.N + want - 1) / want;
    L = (per + kStep - 1) / kStep * kStep;
    if (L < kStep) L = kStep;
    S = (a.N + L - 1) / L;
    if (S < 1) S = 1;
  }
  static int64_t grid(const Variant&, const Args& a) {
    int64_t L, S;
    shape(a, L, S);
    return a.M * S;
  }
  static lift_status launch(const Variant& v, const Args& a, cudaStream_t s) {
    if (a.M == 0) return LIFT_OK;
    if (a.N == 0) return gemv_t_empty_rows(a.M, a.beta, a.out, s);
    int64_t L, S;
    shape(a, L, S);
    if (a.M * S > 0x7fffffffLL) return set_error(LIFT_ERR_UNSUPPORTED, "gemv split: grid too large");
    DeviceState* st = current_state();
    if (S > 1 && a.M * S > st->ws.capacity)
      return set_error(LIFT_ERR_UNSUPPORTED, "gemv split: partials exceed the workspace");
    int64_t M = a.M, N = a.N, lda = a.lda;
    float alpha = a.alpha, beta = a.beta;
    const float* A = a.A;
    const float* x = static_cast<const float*>(a.x);
    float* y = a.out;
    float* partials = a.ws->partials;
    void* args[] = {&M, &N, &alpha, &A, &lda, &x, &beta, &y, &L, &S, &partials};
    lift_status r = launch_config(kernel(), dim3((unsigned)(M * S)), dim3(THREADS), 0, 1, s, args);
    if (r != LIFT_OK || S == 1) return r;
    return launch_rows_combine(M, S, alpha, beta, partials, y, s);
  }
};

template <int THREADS, int VW, int U>
Variant gemv_split_variant(const char* name) {
  using K = GemvSplit<THREADS, VW, U>;
  Variant v{};
  v.info.op = LIFT_OP_GEMV;
  v.info.tile = THREADS * VW;
  v.info.vw = VW;
  v.info.threads = THREADS;
  v.info.stride = 1;
  v.info.cluster = 1;
  v.info.passes = 2;
  v.info.rows = 1;
  v.info.lanes = THREADS;
  v.info.final_threads = kWarp;
  snprintf(v.info.name, sizeof(v.info.name), "gemv_%s", name);
  v.launch = &K::launch;
  v.grid = &K::grid;
  v.align_bytes = VW * 4;
  v.fallback = 0;
  return v;
}

}  // namespace

#define LIFT_GEMV_SPLIT_VARIANTS(X)  \
  X(256, 4, 4, "split_t256_v4_u4")   \
  X(128, 4, 4, "split_t128_v4_u4")   \
  X(256, 8, 2, "split_t256_v8_u2")

void gemv_split_shape(int k, const Args& a, int64_t* L, int64_t* S) {
  int64_t l = 0, s = 0;
  int i = 0;
#define X(T, V, U, NAME) \
  if (i++ == k) GemvSplit<T, V, U>::shape(a, l, s);
  LIFT_GEMV_SPLIT_VARIANTS(X)
#undef X
  *L = l;
  *S = s;
}

void register_gemv_split(std::vector<Variant>& L) {
  const size_t first = L.size();
#define X(T, V, U, NAME) L.push_back(gemv_split_variant<T, V, U>(NAME));
  LIFT_GEMV_SPLIT_VARIANTS(X)
#undef X
  for (size_t i = first; i < L.size(); ++i) L[i].info.id = static_cast<int>(i);
}

}  // namespace lift
