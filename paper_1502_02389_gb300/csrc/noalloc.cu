// lift_asum_noalloc: asum for callers that must not have the library
// allocate device memory.
//
// lift_asum keeps its per-CTA partial sums and its "last CTA" ticket in a
// workspace that lift_init obtains with cudaMalloc.  Some callers cannot let
// that happen: a process whose device memory is owned by its own pool
// allocator under a fixed budget (a framework's caching allocator, an
// embedded runtime) must not see a library take memory behind its back, and
// a latency-critical loop cannot pay for cudaFree, which synchronises the
// whole device.  This entry point runs the same kind of kernel (the
// one-pass, 256-thread, 4096-element-tile, 128-bit-load asum) but keeps its
// scratch in a fixed array in the library's own device image, so it needs
// neither lift_init nor any allocation.
//
// The scratch array holds kNoAllocSlots partial sums plus one ticket word
// (16 KiB + 256 B) and lives on every GPU that loads the library until the
// process exits.  Every call uses the same array:
//  * the ticket must be zero when a call starts, so each call clears it
//    with cudaMemsetAsync on its stream before the launch;
//  * calls whose kernels overlap on the GPU (different streams, or several
//    host threads) race on the array and give wrong results: order them.
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and caches it; make that
// first call before any stream capture.  A launch that would need more
// partial slots than the array holds is refused with LIFT_ERR_UNSUPPORTED.
// x needs only 4-byte alignment: a 16-byte aligned x is read with 128-bit
// loads, any other x element by element in the same order (same result).
// The cached address belongs to the device's current context: after
// cudaDeviceReset, call lift_finalize (which forgets it) before the next call.
#include <mutex>

#include "lift_internal.cuh"
#include "noalloc_plan.h"

namespace lift {
namespace {

using noalloc::kThreads;
using noalloc::kTile;
using noalloc::kVW;

struct NoAllocScratch {
  float partials[noalloc::kSlots];
  unsigned ticket;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// VEC: full tiles read with 128-bit loads (x 16-byte aligned), else with
// 4-byte loads of the same elements in the same order.
template <bool VEC>
__global__ void __launch_bounds__(kThreads)
    asum_noalloc_kernel(const float* __restrict__ x, int64_t n, NoAllocScratch* scratch,
                        float* result) {
  constexpr int J = kTile / kVW / kThreads;
  __shared__ float red[kWarp];
  __shared__ double red64[kWarp];
  __shared__ bool is_last;
  const int t = threadIdx.x;
  const int64_t full = n / kTile;
  float acc[kVW] = {0.f, 0.f, 0.f, 0.f};
  int64_t tile = blockIdx.x;
  for (; tile < full; tile += gridDim.x) {
    Vec<kVW> v[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const float* p = x + tile * kTile + (int64_t)(t + kThreads * j) * kVW;
      if constexpr (VEC) {
        ld_stream(p, v[j]);
      } else {
#pragma unroll
        for (int l = 0; l < kVW; ++l) v[j].v[l] = __ldg(p + l);
      }
    }
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int l = 0; l < kVW; ++l) acc[l] = __fadd_rn(acc[l], fabsf(v[j].v[l]));
  }
  if (tile == full && full * kTile < n) {
#pragma unroll
    for (int j = 0; j < J; ++j) {
      Vec<kVW> v;
      ld_guarded<kVW>(x, tile * kTile + (int64_t)(t + kThreads * j) * kVW, n, v);
#pragma unroll
      for (int l = 0; l < kVW; ++l) acc[l] = __fadd_rn(acc[l], fabsf(v.v[l]));
    }
  }
  float r = acc[0];
#pragma unroll
  for (int l = 1; l < kVW; ++l) r = __fadd_rn(r, acc[l]);
  r = block_tree<kThreads>(r, red);
  if (t == 0) {
    scratch->partials[blockIdx.x] = r;
    __threadfence();
    is_last = atomicAdd(&scratch->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const double s = combine_partials<kThreads>(scratch->partials, gridDim.x, red64);
  if (t == 0) {
    *result = static_cast<float>(s);
    scratch->ticket = 0u;
  }
}

struct PerDevice {
  NoAllocScratch* addr = nullptr;
  int sms = 0, per_sm = 0;   // CTAs per SM of the two forms (the smaller of them)
};

std::mutex g_mu;
std::vector<PerDevice> g_dev;   // per device ordinal, filled on first use

}  // namespace

// Forget the cached per-device addresses (lift_finalize; needed after a
// cudaDeviceReset, which unloads the module that holds the array).
void noalloc_forget() {
  std::lock_guard<std::mutex> lk(g_mu);
  g_dev.clear();
}

}  // namespace lift

using namespace lift;

extern "C" lift_status lift_asum_noalloc(const float* x, int64_t n, float* result, void* stream) {
  noalloc::Plan p;
  // arguments first, before any CUDA call (the device values do not matter yet)
  if (noalloc::plan(x, n, result != nullptr, 1, 1, &p) == noalloc::kBadArgs)
    return set_error(LIFT_ERR_INVALID_ARG, "asum_noalloc arguments");
  int dev = -1;
  lift_status rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc != LIFT_OK) return rc;
  PerDevice d;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_dev.size() <= dev) g_dev.resize(dev + 1);
    if (!g_dev[dev].addr) {
      // set-up, once per device, with that device current
      void* a = nullptr;
      rc = cuda_check(cudaGetSymbolAddress(&a, g_noalloc_scratch), "cudaGetSymbolAddress");
      if (rc != LIFT_OK) return rc;
      int sms = 0, v4 = 0, v1 = 0;
      rc = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
      if (rc == LIFT_OK)
        rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            &v4, asum_noalloc_kernel<true>, kThreads, 0), "occupancy");
      if (rc == LIFT_OK)
        rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            &v1, asum_noalloc_kernel<false>, kThreads, 0), "occupancy");
      if (rc != LIFT_OK) return rc;
      if (sms < 1 || v4 < 1 || v1 < 1)
        return set_error(LIFT_ERR_CUDA, "asum_noalloc: no CTA of the kernel fits on an SM");
      g_dev[dev].addr = static_cast<NoAllocScratch*>(a);
      g_dev[dev].sms = sms;
      g_dev[dev].per_sm = v4 < v1 ? v4 : v1;
    }
    d = g_dev[dev];
  }
  switch (noalloc::plan(x, n, true, d.sms, d.per_sm, &p)) {
    case noalloc::kOk: break;
    case noalloc::kTooLarge:
      return set_error(LIFT_ERR_UNSUPPORTED,
                       "asum_noalloc: the launch needs more partial slots than its fixed scratch "
                       "array holds (4096)");
    default: return set_error(LIFT_ERR_INVALID_ARG, "asum_noalloc arguments");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = cuda_check(cudaMemsetAsync(&d.addr->ticket, 0, sizeof(unsigned), s), "ticket clear");
  if (rc != LIFT_OK) return rc;
  if (p.vector_loads)
    asum_noalloc_kernel<true><<<(unsigned)p.grid, kThreads, 0, s>>>(x, n, d.addr, result);
  else
    asum_noalloc_kernel<false><<<(unsigned)p.grid, kThreads, 0, s>>>(x, n, d.addr, result);
  return cuda_check(cudaGetLastError(), "asum_noalloc launch");
}
