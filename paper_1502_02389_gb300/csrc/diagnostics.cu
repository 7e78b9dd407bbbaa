// Failure-detection probe: the timeout path of the staged kernels, exercised
// without a fault.  Every bulk-copy pipeline waits on mbarrier phases with a
// bounded number of polls and, when they run out, records LIFT_ERR_TIMEOUT in
// the device status word and returns.  lift_wait_probe launches one warp
// whose first lane waits on an mbarrier nothing arrives at, with a
// caller-chosen poll limit, so that a test can watch the status word report
// the timeout and the context stay usable.
#include "lift_internal.cuh"

namespace lift {
namespace {

__global__ void wait_probe(uint32_t polls, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);                 // expects one arrival, which never comes
  fence_mbar_init();
  const uint32_t a = smem_addr(&bar);
  uint32_t ok = 0;
  for (uint32_t i = 0; i < polls && !ok; ++i)
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(a), "r"(0u)
        : "memory");
  if (!ok) report(status, LIFT_ERR_TIMEOUT);
}

}  // namespace
}  // namespace lift

extern "C" lift_status lift_wait_probe(uint32_t polls, void* stream) {
  using namespace lift;
  if (polls == 0 || polls > kWaitPolls) return set_error(LIFT_ERR_INVALID_ARG, "wait_probe polls");
  DeviceState* st = current_state();
  if (!st) return set_error(LIFT_ERR_NOT_INITIALIZED, "lift_init was not called for this device");
  wait_probe<<<1, kWarp, 0, static_cast<cudaStream_t>(stream)>>>(polls, st->ws.status);
  return cuda_check(cudaGetLastError(), "wait_probe launch");
}
