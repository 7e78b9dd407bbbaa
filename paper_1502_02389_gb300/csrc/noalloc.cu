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
#include <mutex>

#include "lift_internal.cuh"

namespace lift {
namespace {

constexpr int kNoAllocSlots = 4096;
constexpr int kThreads = 256, kTile = 4096, kVW = 4;

struct NoAllocScratch {
  float partials[kNoAllocSlots];
  unsigned ticket;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

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
    for (int j = 0; j < J; ++j) ld_stream(x + tile * kTile + (int64_t)(t + kThreads * j) * kVW, v[j]);
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

std::mutex g_mu;
std::vector<NoAllocScratch*> g_addr;   // per device, filled on first use
std::vector<int> g_grid;

}  // namespace
}  // namespace lift

using namespace lift;

extern "C" lift_status lift_asum_noalloc(const float* x, int64_t n, float* result, void* stream) {
  if (n < 0 || !result || (n > 0 && !x) || !aligned(x, 4))
    return set_error(LIFT_ERR_INVALID_ARG, "asum_noalloc arguments");
  int dev = -1;
  lift_status rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc != LIFT_OK) return rc;
  NoAllocScratch* scratch = nullptr;
  int per_device_grid = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_addr.size() <= dev) {
      g_addr.resize(dev + 1, nullptr);
      g_grid.resize(dev + 1, 0);
    }
    if (!g_addr[dev]) {
      // set-up, once per device, with that device current
      void* p = nullptr;
      rc = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
      if (rc != LIFT_OK) return rc;
      int sms = 0, per_sm = 0;
      rc = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
      if (rc != LIFT_OK) return rc;
      rc = cuda_check(
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, asum_noalloc_kernel, kThreads, 0),
          "occupancy");
      if (rc != LIFT_OK) return rc;
      g_addr[dev] = static_cast<NoAllocScratch*>(p);
      g_grid[dev] = sms * per_sm;
    }
    scratch = g_addr[dev];
    per_device_grid = g_grid[dev];
  }
  const int64_t tiles = n > 0 ? (n + kTile - 1) / kTile : 1;
  const int64_t grid = tiles < per_device_grid ? tiles : per_device_grid;
  if (grid > kNoAllocSlots || grid < 1)
    return set_error(LIFT_ERR_UNSUPPORTED,
                     "asum_noalloc: the launch needs more partial slots than its fixed scratch "
                     "array holds (4096)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = cuda_check(cudaMemsetAsync(&scratch->ticket, 0, sizeof(unsigned), s), "ticket clear");
  if (rc != LIFT_OK) return rc;
  asum_noalloc_kernel<<<(unsigned)grid, kThreads, 0, s>>>(x, n, scratch, result);
  return cuda_check(cudaGetLastError(), "asum_noalloc launch");
}
