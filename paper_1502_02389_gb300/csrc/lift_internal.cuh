// Internal helpers shared by the liftblas translation units (device code for
// sm_103a and the host-side variant registry).  Not part of the C-ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lift.h"

namespace lift {

constexpr int kWarp = 32;
// Polls of an mbarrier before a wait gives up and reports LIFT_ERR_TIMEOUT.
// try_wait suspends for a hardware-defined interval per poll, so this bounds
// a stuck wait to well under a few seconds.
constexpr uint32_t kWaitPolls = 1u << 22;

// ---------------------------------------------------------------------------
// per-device state
// ---------------------------------------------------------------------------
struct Workspace {
  float* partials = nullptr;       // per-CTA fp32 partial sums
  double* partials64 = nullptr;    // per-CTA FP64 partials (sum, compensation pairs)
  unsigned* tickets = nullptr;     // one-pass "last CTA" counters (kept at 0 between calls)
  int* status = nullptr;           // device status word (0 = ok, else lift_status), shared
  int64_t capacity = 0;            // fp32 partial slots
  int64_t capacity64 = 0;          // FP64 partial slots
};

// Workspace slots per device: each stream that launches work gets its own
// slot (round robin once there are more streams than slots), so reductions
// running at the same time on different streams do not share partials or
// tickets.
constexpr int kWsSlots = 8;

struct DeviceState {
  int device = -1;
  int sm_count = 0;
  Workspace ws;                    // slot 0 (also the capacities and the status word)
  Workspace more[kWsSlots - 1];    // slots 1 ..
};

DeviceState* current_state();  // state of the current device, or nullptr
// The workspace slot of `stream` on the current device (assigned on first use).
Workspace* stream_workspace(DeviceState* st, cudaStream_t stream);
void noalloc_forget();          // drop lift_asum_noalloc's cached per-device addresses

lift_status set_error(lift_status s, const std::string& msg);
// Poll limit of the staged reductions' first wait on each copy
// (lift_set_wait_polls; kWaitPolls unless a test lowers it).
uint32_t wait_polls();
lift_status cuda_check(cudaError_t e, const char* what);

// ---------------------------------------------------------------------------
// call arguments and variant registry
// ---------------------------------------------------------------------------
struct Args {
  const void* x = nullptr;
  const void* y = nullptr;
  const float* xscale = nullptr;
  const float* yscale = nullptr;
  const float* A = nullptr;
  float* out = nullptr;            // scal / gemv output vector
  float* result = nullptr;         // reduction result
  double* result64 = nullptr;
  Workspace* ws = nullptr;         // the calling stream's workspace slot (set by the entry point)
  int64_t n = 0, M = 0, N = 0, lda = 0;
  float alpha = 0.f, beta = 0.f;
};

struct Variant;
typedef lift_status (*LaunchFn)(const Variant& v, const Args& a, cudaStream_t s);
typedef int64_t (*GridFn)(const Variant& v, const Args& a);

struct Variant {
  lift_variant_info info;
  LaunchFn launch;
  GridFn grid;
  int align_bytes;       // pointer alignment the vector/TMA form needs
  int fallback;          // id (same op) of the guarded scalar form, or -1
};

std::vector<Variant>& registry(int op);

void register_reduce_f32(std::vector<Variant>& asum, std::vector<Variant>& dot);
void register_scal(std::vector<Variant>& scal);
void register_gemv(std::vector<Variant>& gemv);
void register_mixed(std::vector<Variant>* ops);   // ops[LIFT_OP_*]

// Occupancy-derived persistent grid: SMs x resident CTAs per SM.
int64_t persistent_grid(const void* kernel, int threads, size_t smem, int cluster);

// pdl: launch as a programmatic dependent of the kernel before it on the
// stream (the kernel must execute griddepcontrol.wait before its first
// global memory access; see pdl_wait).
lift_status launch_config(const void* kernel, dim3 grid, dim3 block, size_t smem,
                          int cluster, cudaStream_t s, void** args, bool pdl = false);

// Programmatic dependent launch across calls.  A kernel launched with the
// pdl flag may be scheduled while the kernel before it on the stream is
// still running (once that kernel's CTAs have all executed pdl_trigger or
// exited); pdl_wait blocks until that kernel has completed and its memory
// operations are visible, so everything after it is ordered exactly as on a
// plain stream.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

inline bool aligned(const void* p, int bytes) {
  return (reinterpret_cast<uintptr_t>(p) % static_cast<uintptr_t>(bytes)) == 0;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
template <int VW>
struct Vec {
  float v[VW];
};

// Streaming loads: read-only path, no L1 allocation, 256-byte L2 prefetch.
__device__ __forceinline__ void ld_stream(const float* p, Vec<1>& o) {
  asm("ld.global.nc.L1::no_allocate.L2::256B.f32 %0, [%1];" : "=f"(o.v[0]) : "l"(p));
}
__device__ __forceinline__ void ld_stream(const float* p, Vec<4>& o) {
  asm("ld.global.nc.L1::no_allocate.L2::256B.v4.f32 {%0,%1,%2,%3}, [%4];"
      : "=f"(o.v[0]), "=f"(o.v[1]), "=f"(o.v[2]), "=f"(o.v[3])
      : "l"(p));
}
__device__ __forceinline__ void ld_stream(const float* p, Vec<8>& o) {
  asm("ld.global.nc.L1::no_allocate.L2::256B.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(o.v[0]), "=f"(o.v[1]), "=f"(o.v[2]), "=f"(o.v[3]), "=f"(o.v[4]), "=f"(o.v[5]),
        "=f"(o.v[6]), "=f"(o.v[7])
      : "l"(p));
}

__device__ __forceinline__ void st_stream(float* p, const Vec<1>& o) {
  asm volatile("st.global.cs.f32 [%0], %1;" ::"l"(p), "f"(o.v[0]) : "memory");
}
__device__ __forceinline__ void st_stream(float* p, const Vec<4>& o) {
  asm volatile("st.global.cs.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(o.v[0]), "f"(o.v[1]),
               "f"(o.v[2]), "f"(o.v[3])
               : "memory");
}
__device__ __forceinline__ void st_stream(float* p, const Vec<8>& o) {
  asm volatile("st.global.cs.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(o.v[0]),
               "f"(o.v[1]), "f"(o.v[2]), "f"(o.v[3]), "f"(o.v[4]), "f"(o.v[5]), "f"(o.v[6]),
               "f"(o.v[7])
               : "memory");
}

// Guarded scalar loads of a vector whose elements may run past n (zeros there).
template <int VW>
__device__ __forceinline__ void ld_guarded(const float* base, int64_t first, int64_t n, Vec<VW>& o) {
#pragma unroll
  for (int l = 0; l < VW; ++l) o.v[l] = (first + l < n) ? __ldg(base + first + l) : 0.0f;
}

template <int VW>
__device__ __forceinline__ void ld_smem(const float* p, Vec<VW>& o) {
  if constexpr (VW == 1) {
    o.v[0] = *p;
  } else {
#pragma unroll
    for (int q = 0; q < VW / 4; ++q) {
      float4 t = reinterpret_cast<const float4*>(p)[q];
      o.v[4 * q + 0] = t.x;
      o.v[4 * q + 1] = t.y;
      o.v[4 * q + 2] = t.z;
      o.v[4 * q + 3] = t.w;
    }
  }
}

template <int VW>
__device__ __forceinline__ void st_smem(float* p, const Vec<VW>& o) {
  if constexpr (VW == 1) {
    *p = o.v[0];
  } else {
#pragma unroll
    for (int q = 0; q < VW / 4; ++q)
      reinterpret_cast<float4*>(p)[q] =
          make_float4(o.v[4 * q], o.v[4 * q + 1], o.v[4 * q + 2], o.v[4 * q + 3]);
  }
}

// Neumaier's compensated step (Neumaier 1974): s + t rounded, and the
// rounding error of that add (exact: Fast2Sum with the larger operand
// first) added to the running compensation c.  A lane that adds its tile
// sums this way carries an error of about 2u|sum| however many tiles it
// folds, instead of one rounding per tile.
__device__ __forceinline__ void neumaier_add(float& s, float& c, float t) {
  const float u = __fadd_rn(s, t);
  const float d = fabsf(s) >= fabsf(t) ? __fadd_rn(__fsub_rn(s, u), t)
                                       : __fadd_rn(__fsub_rn(t, u), s);
  s = u;
  c = __fadd_rn(c, d);
}
// The compensated value s + c; a non-finite s (Inf or NaN among the terms)
// is returned as it is, so that Inf does not turn into NaN.
__device__ __forceinline__ float neumaier_value(float s, float c) {
  return isfinite(s) ? __fadd_rn(s, c) : s;
}

// Vectors a gemv lane (or thread) folds plainly before it adds their value
// to its compensated sum: its vectors k = 0, 1, ... of a row (or segment)
// form groups gG .. gG+G-1; a group's products are folded from zero over
// the VW lanes, the lanes added in order, and the group values added with
// neumaier_add, so a row's error does not grow with its length.
constexpr int kGemvGroup = 8;   // a power of two
static_assert((kGemvGroup & (kGemvGroup - 1)) == 0, "group masks need a power of two");

template <int VW>
struct GroupedDot {
  float gs[VW];        // the current group's lane sums
  float s, c;          // compensated sum of the finished groups
  bool closed;         // some group was closed before the last one
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int l = 0; l < VW; ++l) gs[l] = 0.f;
    s = c = 0.f;
    closed = false;
  }
  __device__ __forceinline__ void add(const Vec<VW>& a, const Vec<VW>& b) {
#pragma unroll
    for (int l = 0; l < VW; ++l) gs[l] = __fadd_rn(gs[l], __fmul_rn(a.v[l], b.v[l]));
  }
  // close the current group (a partial group is closed the same way: the
  // zeros that would pad it change nothing)
  __device__ __forceinline__ float lanes() const {
    float v = gs[0];
#pragma unroll
    for (int l = 1; l < VW; ++l) v = __fadd_rn(v, gs[l]);
    return v;
  }
  __device__ __forceinline__ void flush() {
    neumaier_add(s, c, lanes());
#pragma unroll
    for (int l = 0; l < VW; ++l) gs[l] = 0.f;
    closed = true;
  }
  // the value after the last vector (closes the last group); with a single
  // group the compensated sum is that group's value itself (0 + v is exact
  // and its correction is 0), so it is returned directly
  __device__ __forceinline__ float value() {
    if (!closed) return lanes();
    flush();
    return neumaier_value(s, c);
  }
};

// Halving tree over the 32 lanes of a warp: at offset o lane j adds lane
// j + o (iterate-5 of split-2 after reorder-stride with n = 2).  Lane 0 ends
// with the warp's value.
__device__ __forceinline__ float warp_tree(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_tree64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Whole-CTA tree: warp trees, then warp 0 over the warp results padded with
// zeros to 32.  `red` holds >= 32 floats of shared memory.  Valid in thread 0.
template <int THREADS>
__device__ __forceinline__ float block_tree(float v, float* red) {
  v = warp_tree(v);
  if constexpr (THREADS > kWarp) {
    const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x / kWarp;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
      v = lane < THREADS / kWarp ? red[lane] : 0.0f;
      v = warp_tree(v);
    }
  }
  return v;
}

template <int THREADS>
__device__ __forceinline__ double block_tree64(double v, double* red) {
  v = warp_tree64(v);
  if constexpr (THREADS > kWarp) {
    const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x / kWarp;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
      v = lane < THREADS / kWarp ? red[lane] : 0.0;
      v = warp_tree64(v);
    }
  }
  return v;
}

// Record the first error in the device status word.
__device__ __forceinline__ void report(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// mbarrier and TMA bulk copies (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait for phase `parity` of `bar`; false after `polls` polls
// (0: gives up at once).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          uint32_t polls = kWaitPolls) {
  const uint32_t a = smem_addr(bar);
  for (uint32_t i = 0; i < polls; ++i) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Bulk copy global -> shared (16-byte aligned addresses, size % 16 == 0),
// completion signalled on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Bulk copy shared -> global, tracked by bulk async-groups.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
// Make generic-proxy writes to shared memory visible to the async proxy.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------------------
// final FP64 combine of fp32 partials (shared by the one-pass last CTA and
// the two-pass second kernel): thread t sums partials t, t+FT, ... in FP64,
// then a block tree in FP64.  Valid in thread 0.
// ---------------------------------------------------------------------------
template <int FT>
__device__ __forceinline__ double combine_partials(const float* partials, int64_t P, double* red) {
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < P; i += FT) acc = __dadd_rn(acc, (double)__ldcg(partials + i));
  return block_tree64<FT>(acc, red);
}

}  // namespace lift
