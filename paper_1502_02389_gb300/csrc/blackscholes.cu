// BlackScholes as a pure map (arXiv 1502.02389, Sec. 7 "Mathematical Finance
// Application", Fig. 6):  blackScholes(s) = map(BSComputation, s), one
// {call, put} pair per stock price.  The paper leaves compD1, compD2,
// compCall and compPut out; they are the Black-Scholes model for a European
// option with strike K, riskless rate r, volatility sigma and maturity T:
//
//   d1 = (ln(S/K) + (r + sigma^2/2) T) / (sigma sqrt(T)),  d2 = d1 - sigma sqrt(T)
//   call = S N(d1) - K e^{-rT} N(d2),  put = call - S + K e^{-rT}
//
// with N the standard normal distribution and the put taken from put-call
// parity.  The pair is stored as two arrays (the zip of the map's two
// outputs).  Two evaluations of N are variants of the user function:
//   CND = 0: N(x) = erfc(-x / sqrt(2)) / 2 with CUDA's erfcf;
//   CND = 1: the polynomial approximation 26.2.17 of Abramowitz and Stegun,
//            "Handbook of Mathematical Functions" (1964), after Hastings:
//            for x >= 0 the upper tail is Z(x) (b1 t + ... + b5 t^5),
//            t = 1 / (1 + p x), with |error| < 7.5e-8; N(x) is one minus
//            that tail, and N(-x) the tail itself;
//   CND = 2: the same polynomial on the approximate special-function
//            instructions (lg2.approx, ex2.approx, rcp.approx), with one
//            exponential per option: the model's identity
//            S phi(d1) = K e^{-rT} phi(d2) gives phi(d2) = phi(d1) S / (K e^{-rT}).
//            d1 = lg2(S/K) (ln 2 / (sigma sqrt T)) + (r + sigma^2/2) T / (sigma sqrt T)
//            is one fused multiply-add, and phi(d1) = 2^(d1 d1 (-1/(2 ln 2))
//            + log2(1/sqrt(2 pi))) one more and an ex2.  An error in d1 moves
//            the call by S phi(d1) - K e^{-rT} phi(d2) = 0 to first order (d2 is
//            formed from the same d1), so the logarithm's accuracy barely
//            reaches the prices; the exponential scales tails of at most 0.5.
//
// Lowering: the rule map(f) -> asScalar . map(vect^VW(f)) . asVector^VW
// (Fig. 4e), map-workgroup over tiles of THREADS*U vectors dealt round robin
// to a persistent grid (or, GRID == 1, one CTA per tile, dealt to the SMs by
// the hardware), map-local over the vectors of a tile.  Every variant
// with the same CND applies the same per-element function with explicitly
// rounded operations (no contraction), so they agree bit for bit.
#include <math.h>

#include "lift_internal.cuh"

namespace lift {
namespace {

struct BsConst {
  float inv_k;    // 1 / K
  float mu;       // (r + sigma^2 / 2) T
  float inv_sq;   // 1 / (sigma sqrt(T))
  float sq;       // sigma sqrt(T)
  float ke;       // K e^{-rT}
  float inv_ke;   // 1 / (K e^{-rT})
  float ln2_sq;   // ln 2 / (sigma sqrt(T))
  float mu_sq;    // (r + sigma^2 / 2) T / (sigma sqrt(T))
};

constexpr float kHalfLog2e = -0.72134752044448170368f;   // -1 / (2 ln 2)
constexpr float kLog2Rsqrt2Pi = -1.32574806473616f;      // log2(1 / sqrt(2 pi))

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr float kRsqrt2 = 0.70710678118654752440f;      // 1 / sqrt(2)
constexpr float kRsqrt2Pi = 0.39894228040143267794f;    // 1 / sqrt(2 pi)

template <int CND>
__device__ __forceinline__ float normal_cdf(float x) {
  if constexpr (CND == 0) {
    return __fmul_rn(0.5f, erfcf(__fmul_rn(-x, kRsqrt2)));
  } else {
    const float ax = fabsf(x);
    const float den = __fmaf_rn(0.2316419f, ax, 1.0f);
    const float arg = __fmul_rn(-0.5f, __fmul_rn(ax, ax));
    const float t = __frcp_rn(den);
    const float z = __fmul_rn(kRsqrt2Pi, expf(arg));
    float poly = 1.330274429f;
    poly = __fmaf_rn(poly, t, -1.821255978f);
    poly = __fmaf_rn(poly, t, 1.781477937f);
    poly = __fmaf_rn(poly, t, -0.356563782f);
    poly = __fmaf_rn(poly, t, 0.319381530f);
    const float tail = __fmul_rn(z, __fmul_rn(poly, t));
    return x >= 0.f ? __fsub_rn(1.0f, tail) : tail;
  }
}

// N(x) from the tail polynomial of A&S 26.2.17 and z = phi(x)
__device__ __forceinline__ float normal_cdf_poly(float x, float z) {
  const float t = rcp_approx(__fmaf_rn(0.2316419f, fabsf(x), 1.0f));
  float poly = 1.330274429f;
  poly = __fmaf_rn(poly, t, -1.821255978f);
  poly = __fmaf_rn(poly, t, 1.781477937f);
  poly = __fmaf_rn(poly, t, -0.356563782f);
  poly = __fmaf_rn(poly, t, 0.319381530f);
  const float tail = __fmul_rn(z, __fmul_rn(poly, t));
  return x >= 0.f ? __fsub_rn(1.0f, tail) : tail;
}

template <int CND>
__device__ __forceinline__ void bs_option(float S, const BsConst& c, float& call, float& put) {
  const float q = __fmul_rn(S, c.inv_k);
  float d1, n1, n2;
  if constexpr (CND == 2) {
    d1 = __fmaf_rn(lg2_approx(q), c.ln2_sq, c.mu_sq);
    const float d2 = __fsub_rn(d1, c.sq);
    const float z1 = ex2_approx(__fmaf_rn(d1, __fmul_rn(d1, kHalfLog2e), kLog2Rsqrt2Pi));
    const float z2 = __fmul_rn(__fmul_rn(z1, S), c.inv_ke);
    n1 = normal_cdf_poly(d1, z1);
    n2 = normal_cdf_poly(d2, z2);
  } else {
    d1 = __fmul_rn(__fadd_rn(logf(q), c.mu), c.inv_sq);
    const float d2 = __fsub_rn(d1, c.sq);
    n1 = normal_cdf<CND>(d1);
    n2 = normal_cdf<CND>(d2);
  }
  call = __fsub_rn(__fmul_rn(S, n1), __fmul_rn(c.ke, n2));
  put = __fadd_rn(__fsub_rn(call, S), c.ke);
}

template <int THREADS, int VW, int U, int CND>
__global__ void __launch_bounds__(THREADS)
    bs_map(int64_t n, const float* __restrict__ s, float* __restrict__ call,
           float* __restrict__ put, BsConst c) {
  pdl_trigger();   // the next call's first kernel may be scheduled (it waits for this one)
  pdl_wait();      // the previous kernel on the stream has completed
  const int64_t nv = n / VW;                         // whole vectors
  const int64_t stride = (int64_t)gridDim.x * THREADS * U;
  for (int64_t base = (int64_t)blockIdx.x * THREADS * U + threadIdx.x; base < nv; base += stride) {
    Vec<VW> S[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t v = base + (int64_t)u * THREADS;
      if (v < nv) ld_stream(s + v * VW, S[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t v = base + (int64_t)u * THREADS;
      if (v >= nv) continue;
      Vec<VW> C, P;
#pragma unroll
      for (int l = 0; l < VW; ++l) bs_option<CND>(S[u].v[l], c, C.v[l], P.v[l]);
      st_stream(call + v * VW, C);
      st_stream(put + v * VW, P);
    }
  }
  // the ragged tail (fewer than VW elements), one element per thread of CTA 0
  if (blockIdx.x == 0) {
    const int64_t i = nv * VW + threadIdx.x;
    if (i < n) bs_option<CND>(__ldg(s + i), c, call[i], put[i]);
  }
}

template <int THREADS, int VW, int U, int CND, int GRID = 0>
struct BlackScholes {
  static const void* kernel() { return reinterpret_cast<const void*>(&bs_map<THREADS, VW, U, CND>); }
  // one CTA per THREADS * U vectors (GRID == 1; the grid-stride loop still
  // covers every vector if the grid is capped), or at most the resident CTAs
  static int64_t grid(const Variant&, const Args& a) {
    const int64_t per = (int64_t)THREADS * U;
    const int64_t need = (a.n / VW + per - 1) / per;
    int64_t g = GRID == 1 ? INT32_MAX : persistent_grid(kernel(), THREADS, 0, 1);
    if (need < g) g = need;
    return g < 1 ? 1 : g;
  }
  // Args of this op: x = prices, out = call, result = put, and xscale points
  // at the host block {K, r, sigma, T}.
  static lift_status launch(const Variant& v, const Args& a, cudaStream_t s) {
    if (a.n == 0) return LIFT_OK;
    const float* p = a.xscale;
    const double K = p[0], r = p[1], sig = p[2], T = p[3];
    BsConst c;
    c.inv_k = (float)(1.0 / K);
    c.mu = (float)((r + 0.5 * sig * sig) * T);
    c.sq = (float)(sig * sqrt(T));
    c.inv_sq = (float)(1.0 / (sig * sqrt(T)));
    c.ke = (float)(K * exp(-r * T));
    c.inv_ke = (float)(1.0 / (K * exp(-r * T)));
    c.ln2_sq = (float)(log(2.0) / (sig * sqrt(T)));
    c.mu_sq = (float)((r + 0.5 * sig * sig) * T / (sig * sqrt(T)));
    int64_t n = a.n;
    const float* prices = static_cast<const float*>(a.x);
    float* call = a.out;
    float* put = a.result;
    void* args[] = {&n, &prices, &call, &put, &c};
    return launch_config(kernel(), dim3((unsigned)grid(v, a)), dim3(THREADS), 0, 1, s, args, true);
  }
};

// per CND, the id of its 4-byte-load variant (the guarded form)
constexpr int kFallback[3] = {0, 2, 5};

template <int THREADS, int VW, int U, int CND, int GRID = 0>
Variant bs_variant(const char* name) {
  using K = BlackScholes<THREADS, VW, U, CND, GRID>;
  Variant v{};
  v.info.op = LIFT_OP_BLACKSCHOLES;
  v.info.tile = THREADS * VW * U;
  v.info.vw = VW;
  v.info.threads = THREADS;
  v.info.stride = 1;
  v.info.cluster = 1;
  v.info.passes = 1;
  v.info.rows = U;
  v.info.lanes = 1;
  v.info.grid = GRID;
  snprintf(v.info.name, sizeof(v.info.name), "blackscholes_%s", name);
  v.launch = &K::launch;
  v.grid = &K::grid;
  v.info.tree = CND;      // the normal-distribution evaluation (0 erfcf, 1 A&S, 2 A&S fast)
  v.align_bytes = VW * 4;
  v.fallback = kFallback[CND];
  return v;
}

}  // namespace

void register_blackscholes(std::vector<Variant>& L) {
  L.push_back(bs_variant<256, 1, 4, 0>("t256_v1_u4"));
  L.push_back(bs_variant<256, 4, 2, 0>("t256_v4_u2"));
  L.push_back(bs_variant<256, 1, 4, 1>("t256_v1_u4_as"));
  L.push_back(bs_variant<256, 4, 2, 1>("t256_v4_u2_as"));
  L.push_back(bs_variant<256, 8, 1, 1>("t256_v8_u1_as"));
  L.push_back(bs_variant<256, 1, 4, 2>("t256_v1_u4_fast"));
  L.push_back(bs_variant<256, 4, 1, 2>("t256_v4_u1_fast"));
  L.push_back(bs_variant<256, 4, 2, 2>("t256_v4_u2_fast"));
  L.push_back(bs_variant<128, 4, 4, 2>("t128_v4_u4_fast"));
  L.push_back(bs_variant<256, 8, 1, 2>("t256_v8_u1_fast"));
  // one CTA per tile (appended: earlier ids are stable)
  L.push_back(bs_variant<256, 4, 1, 2, 1>("t256_v4_u1_fast_pertile"));
  L.push_back(bs_variant<256, 4, 2, 2, 1>("t256_v4_u2_fast_pertile"));
  L.push_back(bs_variant<128, 4, 4, 2, 1>("t128_v4_u4_fast_pertile"));
  L.push_back(bs_variant<256, 8, 1, 2, 1>("t256_v8_u1_fast_pertile"));
  L.push_back(bs_variant<256, 4, 2, 1, 1>("t256_v4_u2_as_pertile"));
  for (size_t i = 0; i < L.size(); ++i) L[i].info.id = static_cast<int>(i);
}

}  // namespace lift
