// Compensated fp32 asum and dot (arXiv 1502.02389, Fig. 5 programs, with the
// reduction's user function replaced by an error-free one).
//
// The fold of Fig. 8 eq. (8), reduce-seq(lambda acc, x. acc + g(x)), keeps
// one fp32 accumulator per lane and loses the rounding error of every add.
// Here a lane's accumulator is a (sum, compensation) pair: every term is
// added with TwoSum, whose exact rounding error goes into the compensation,
// and for dot the product's own rounding error, fma(x, y, -fl(x y)) (exact,
// TwoProduct with a fused multiply-add, as in Ogita, Rump and Oishi 2005),
// goes there too.  The structure is the fp32 kernels' (tiles of
// THREADS * VW * U elements dealt round robin to a persistent grid; work-item
// t takes vectors t, t + THREADS, ... of a tile; VW lane pairs per work-item),
// then the pairs are merged lane by lane, across the warp and the CTA with
// TwoSum, the CTA writes sum + compensation as one FP64 partial, and the last
// CTA adds the partials in FP64 and rounds once to fp32.  The result is then
// within about one unit of fp32 roundoff of the exact sum even when the sum
// cancels (|sum| much smaller than the sum of |terms|), where the plain fold's
// error bound grows with the sum of |terms|.
#include "comp_sum.cuh"

namespace lift {
namespace {

template <int OP, int VW>
__device__ __forceinline__ void fold_vec(Comp (&acc)[VW], const Vec<VW>& a, const Vec<VW>& b) {
#pragma unroll
  for (int l = 0; l < VW; ++l) {
    if constexpr (OP == LIFT_OP_ASUM) {
      two_sum_add(acc[l], fabsf(a.v[l]));
    } else {
      const float p = __fmul_rn(a.v[l], b.v[l]);
      const float e = __fmaf_rn(a.v[l], b.v[l], -p);     // x y - fl(x y), exact
      two_sum_add(acc[l], p);
      acc[l].c = __fadd_rn(acc[l].c, e);
    }
  }
}

template <int OP, int THREADS, int VW, int U>
__global__ void __launch_bounds__(THREADS)
    comp_reduce(const float* __restrict__ x, const float* __restrict__ y, int64_t n,
                double* __restrict__ partials, unsigned* ticket, float* result, double* result64) {
  constexpr int64_t kTile = (int64_t)THREADS * VW * U;
  pdl_wait();      // the previous kernel on the stream has completed
  const int t = threadIdx.x;
  const int64_t G = gridDim.x;
  const int64_t full = n / kTile;
  Comp acc[VW];
#pragma unroll
  for (int l = 0; l < VW; ++l) acc[l] = Comp{0.f, 0.f};
  int64_t tile = blockIdx.x;
  for (; tile < full; tile += G) {
    Vec<VW> a[U], b[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t e = tile * kTile + ((int64_t)u * THREADS + t) * VW;
      ld_stream(x + e, a[u]);
      if constexpr (OP == LIFT_OP_DOT) ld_stream(y + e, b[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) fold_vec<OP, VW>(acc, a[u], b[u]);
  }
  if (tile == full) {                       // the ragged last tile, element by element
    for (int u = 0; u < U; ++u) {
      const int64_t e = full * kTile + ((int64_t)u * THREADS + t) * VW;
      Vec<VW> a, b;
      ld_guarded<VW>(x, e, n, a);
      if constexpr (OP == LIFT_OP_DOT) ld_guarded<VW>(y, e, n, b);
      else b = a;
      fold_vec<OP, VW>(acc, a, b);
    }
  }
  pdl_trigger();   // streaming done: the next call's first kernel may be scheduled
  Comp c = acc[0];
#pragma unroll
  for (int l = 1; l < VW; ++l) c = comp_merge(c, acc[l]);
  c = block_comp<THREADS>(c);
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

constexpr int kCompTicket = 2;    // workspace counter of this family

template <int OP, int THREADS, int VW, int U>
struct CompReduce {
  static const void* kernel() {
    return reinterpret_cast<const void*>(&comp_reduce<OP, THREADS, VW, U>);
  }
  static int64_t grid(const Variant&, const Args& a) {
    constexpr int64_t kTile = (int64_t)THREADS * VW * U;
    const int64_t T = a.n > 0 ? (a.n + kTile - 1) / kTile : 1;
    const int64_t g = persistent_grid(kernel(), THREADS, 0, 1);
    if (g <= 0) return 0;
    const int64_t per = (T + g - 1) / g;
    return (T + per - 1) / per;
  }
  static lift_status launch(const Variant& v, const Args& a, cudaStream_t s) {
    DeviceState* st = current_state();
    const int64_t g = grid(v, a);
    if (g <= 0) return set_error(LIFT_ERR_CUDA, std::string("no resident CTA for ") + v.info.name);
    if (g > st->ws.capacity) return set_error(LIFT_ERR_UNSUPPORTED, "grid exceeds workspace");
    const float* x = static_cast<const float*>(a.x);
    const float* y = static_cast<const float*>(a.y);
    int64_t n = a.n;
    if (g > st->ws.capacity64) return set_error(LIFT_ERR_UNSUPPORTED, "grid exceeds workspace");
    double* partials = a.ws->partials64;
    unsigned* ticket = a.ws->tickets + kCompTicket;
    float* result = a.result;
    double* result64 = a.result64;
    void* args[] = {&x, &y, &n, &partials, &ticket, &result, &result64};
    return launch_config(kernel(), dim3((unsigned)g), dim3(THREADS), 0, 1, s, args, true);
  }
};

template <int OP, int THREADS, int VW, int U>
Variant comp_variant(int opid, const char* name) {
  using K = CompReduce<OP, THREADS, VW, U>;
  Variant v{};
  v.info.op = opid;
  v.info.tile = THREADS * VW * U;
  v.info.vw = VW;
  v.info.threads = THREADS;
  v.info.stride = 1;
  v.info.tree = 1;
  v.info.cluster = 1;
  v.info.passes = 1;
  v.info.rows = U;
  v.info.final_threads = THREADS;
  snprintf(v.info.name, sizeof(v.info.name), "%s", name);
  v.launch = &K::launch;
  v.grid = &K::grid;
  v.align_bytes = VW * 4;
  v.fallback = 0;
  return v;
}

template <int OP>
void register_comp_op(std::vector<Variant>& L, int opid, const char* tag) {
  char nm[64];
#define X(T, V, U)                                                \
  snprintf(nm, sizeof nm, "%s_t%d_v%d_u%d", tag, T, V, U);        \
  L.push_back(comp_variant<OP, T, V, U>(opid, nm));
  X(256, 1, 4)      // id 0: 4-byte loads, the guarded form for misaligned inputs
  X(256, 4, 2)
  X(256, 4, 4)
  X(128, 4, 4)
  X(256, 8, 2)
#undef X
  for (size_t i = 0; i < L.size(); ++i) L[i].info.id = static_cast<int>(i);
}

}  // namespace

void register_compensated(std::vector<Variant>& asum, std::vector<Variant>& dot) {
  register_comp_op<LIFT_OP_ASUM>(asum, LIFT_OP_ASUM_COMP, "asum_comp");
  register_comp_op<LIFT_OP_DOT>(dot, LIFT_OP_DOT_COMP, "dot_comp");
}

}  // namespace lift
