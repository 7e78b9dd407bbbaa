// Batched persistent launch: many asum / dot / scal / gemv calls of uneven
// sizes in one graph-captured launch that pulls work items from a queue.
//
// Each op is split into work items (split^ITEM of its vector, or a block of
// gemv rows): map(op) over the batch becomes a map-workgroup over items
// handed out by an atomic queue head (largest items first, so the tail of
// the launch is made of small items).  A CTA processes an item exactly as
// the standalone kernels process their tiles (the item's tiles in order,
// thread t folding vectors t + THREADS*j of each tile, adding the tile's
// lanes, and adding the tile values with Neumaier's compensated step, then
// the block tree); for asum / dot
// each item leaves one fp32 partial, and the CTA that
// finishes an op's last item (an atomic per-op counter) adds that op's item
// partials in item order in FP64 (thread t takes partials t, t+256, ...,
// then an FP64 block tree) and writes the rounded result.  Nothing waits:
// the queue and the counters are atomics, reset by a memset node of the
// same graph before the kernel node.  The other schedule of the same
// map-workgroup launches one CTA per queue position instead of popping the
// queue, and lets the hardware deal the CTAs to the SMs as earlier ones
// retire; the items, their order and the combine are the same.
//
// Per op, the policy's variant choice (lift_pick: FIXED, TABLE or MLP) is
// mapped to a processing mode: vector ops take the (tile, vector width) of
// the chosen variant when the batch kernel has that mode, gemv takes its
// vector width.  A pointer that is not aligned for the mode's vector width
// gets the 4-byte mode.
#include <algorithm>
#include <string>
#include <vector>

#include "lift_internal.cuh"

namespace lift {
namespace {

constexpr int kThreads = 256;
constexpr int64_t kItemBytes = 256 * 1024;   // target bytes moved per work item

// vector-op processing modes: (VW, J) with TILE = kThreads * VW * J
struct VecMode {
  int vw, j;
};
constexpr VecMode kVecModes[] = {{1, 4}, {4, 1}, {4, 2}, {4, 4}, {8, 1}, {8, 2}};
constexpr int kNumVecModes = 6;
constexpr int kGemvVW[] = {1, 4, 8};

struct OpDev {
  int op;            // LIFT_OP_ASUM / DOT / SCAL / GEMV
  int mode;          // vector mode index, or gemv vw index
  int64_t n, M, N, lda;
  float alpha, beta;
  const float* x;
  const float* y;
  const float* A;
  float* out;
  int64_t first_item, num_items;
};

struct ItemDev {
  int op_index;
  int64_t begin, end;   // elements (vector ops) or rows (gemv)
};

struct BatchDev {
  const OpDev* ops;
  const ItemDev* items;
  const int64_t* order;       // queue position -> item index
  float* partials;            // per item
  unsigned* op_done;          // per op: items finished
  unsigned long long* head;   // queue head
  int64_t num_items;
};

template <int OP, int VW>
__device__ __forceinline__ void fold(float* acc, const Vec<VW>& a, const Vec<VW>& b) {
#pragma unroll
  for (int l = 0; l < VW; ++l)
    acc[l] = OP == LIFT_OP_ASUM ? __fadd_rn(acc[l], fabsf(a.v[l]))
                                : __fadd_rn(acc[l], __fmul_rn(a.v[l], b.v[l]));
}

// One reduction item: elements [begin, end) of op o, in tiles of
// kThreads*VW*J elements; returns the CTA's value in thread 0.
template <int OP, int VW, int J>
__device__ float reduce_item(const OpDev& o, int64_t begin, int64_t end, float* red) {
  constexpr int64_t TILE = (int64_t)kThreads * VW * J;
  const int t = threadIdx.x;
  float acc = 0.f, cmp = 0.f;  // sum of the tile values and its Neumaier compensation
  int64_t base = begin;
  for (; base + TILE <= end; base += TILE) {
    Vec<VW> a[J], b[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int64_t e = base + (int64_t)(t + kThreads * j) * VW;
      ld_stream(o.x + e, a[j]);
      if constexpr (OP == LIFT_OP_DOT) ld_stream(o.y + e, b[j]);
    }
    float ts[VW];
#pragma unroll
    for (int l = 0; l < VW; ++l) ts[l] = 0.f;
#pragma unroll
    for (int j = 0; j < J; ++j) fold<OP, VW>(ts, a[j], b[j]);
    float tv = ts[0];
#pragma unroll
    for (int l = 1; l < VW; ++l) tv = __fadd_rn(tv, ts[l]);
    neumaier_add(acc, cmp, tv);
  }
  if (base < end) {
    float ts[VW];
#pragma unroll
    for (int l = 0; l < VW; ++l) ts[l] = 0.f;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int64_t e = base + (int64_t)(t + kThreads * j) * VW;
      Vec<VW> a, b;
      ld_guarded<VW>(o.x, e, end, a);
      if constexpr (OP == LIFT_OP_DOT) ld_guarded<VW>(o.y, e, end, b);
      fold<OP, VW>(ts, a, b);
    }
    float tv = ts[0];
#pragma unroll
    for (int l = 1; l < VW; ++l) tv = __fadd_rn(tv, ts[l]);
    neumaier_add(acc, cmp, tv);
  }
  return block_tree<kThreads>(neumaier_value(acc, cmp), red);
}

template <int VW, int J>
__device__ void scal_item(const OpDev& o, int64_t begin, int64_t end) {
  constexpr int64_t TILE = (int64_t)kThreads * VW * J;
  const int t = threadIdx.x;
  int64_t base = begin;
  for (; base + TILE <= end; base += TILE) {
    Vec<VW> a[J];
#pragma unroll
    for (int j = 0; j < J; ++j) ld_stream(o.x + base + (int64_t)(t + kThreads * j) * VW, a[j]);
#pragma unroll
    for (int j = 0; j < J; ++j) {
#pragma unroll
      for (int l = 0; l < VW; ++l) a[j].v[l] = __fmul_rn(o.alpha, a[j].v[l]);
      st_stream(o.out + base + (int64_t)(t + kThreads * j) * VW, a[j]);
    }
  }
  for (int64_t e = base + t; e < end; e += kThreads) o.out[e] = __fmul_rn(o.alpha, o.x[e]);
}

template <int VW>
__device__ __forceinline__ void ld_x(const float* p, Vec<VW>& o) {
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

template <int VW>
__device__ void gemv_item(const OpDev& o, int64_t r0, int64_t r1) {
  constexpr int64_t kChunk = (int64_t)kWarp * VW;
  constexpr int U = VW == 1 ? 8 : (VW == 4 ? 4 : 2);
  const int lane = threadIdx.x & (kWarp - 1);
  const int64_t chunks = o.N / kChunk;
  static_assert(kGemvGroup % U == 0, "an unrolled step stays inside one group");
  for (int64_t row = r0 + threadIdx.x / kWarp; row < r1; row += kThreads / kWarp) {
    const float* a = o.A + row * o.lda;
    GroupedDot<VW> acc;
    acc.init();
    int64_t c = 0;                     // the lane's vector index along the row
    for (; c + U <= chunks; c += U) {
      Vec<VW> va[U], vx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t e = (c + u) * kChunk + lane * VW;
        ld_stream(a + e, va[u]);
        ld_x<VW>(o.x + e, vx[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) acc.add(va[u], vx[u]);
      if (((c + U) & (kGemvGroup - 1)) == 0) acc.flush();
    }
    for (; c < chunks; ++c) {
      Vec<VW> va, vx;
      const int64_t e = c * kChunk + lane * VW;
      ld_stream(a + e, va);
      ld_x<VW>(o.x + e, vx);
      acc.add(va, vx);
      if (((c + 1) & (kGemvGroup - 1)) == 0) acc.flush();
    }
    if (chunks * kChunk < o.N) {
      Vec<VW> va, vx;
      const int64_t e = chunks * kChunk + lane * VW;
      ld_guarded<VW>(a, e, o.N, va);
      ld_guarded<VW>(o.x, e, o.N, vx);
      acc.add(va, vx);
    }
    float r = warp_tree(acc.value());
    if (lane == 0) {
      const float z = __fmul_rn(o.alpha, r);
      o.out[row] = o.beta == 0.f ? z : __fadd_rn(z, __fmul_rn(o.beta, o.out[row]));
    }
  }
}

template <int OP>
__device__ float reduce_dispatch(const OpDev& o, int64_t b, int64_t e, float* red) {
  switch (o.mode) {
    case 0: return reduce_item<OP, 1, 4>(o, b, e, red);
    case 1: return reduce_item<OP, 4, 1>(o, b, e, red);
    case 2: return reduce_item<OP, 4, 2>(o, b, e, red);
    case 3: return reduce_item<OP, 4, 4>(o, b, e, red);
    case 4: return reduce_item<OP, 8, 1>(o, b, e, red);
    default: return reduce_item<OP, 8, 2>(o, b, e, red);
  }
}

// QUEUE: a persistent grid whose CTAs pop queue positions with an atomic;
// otherwise one CTA per queue position (CTA q takes position q), dealt to
// the SMs by the hardware in launch order as earlier CTAs retire.
template <bool QUEUE>
__device__ __forceinline__ void batch_body(const BatchDev& B) {
  __shared__ float red[kWarp];
  __shared__ double red64[kWarp];
  __shared__ int64_t s_item;
  __shared__ bool s_last;
  for (;;) {
    int64_t it;
    if constexpr (QUEUE) {
      if (threadIdx.x == 0) {
        const unsigned long long q = atomicAdd(B.head, 1ull);
        s_item = q < (unsigned long long)B.num_items ? B.order[q] : -1;
      }
      __syncthreads();
      it = s_item;
    } else {
      it = (int64_t)blockIdx.x < B.num_items ? B.order[blockIdx.x] : -1;
    }
    if (it < 0) return;
    const ItemDev item = B.items[it];
    const OpDev o = B.ops[item.op_index];
    if (o.op == LIFT_OP_ASUM || o.op == LIFT_OP_DOT) {
      const float r = o.op == LIFT_OP_ASUM ? reduce_dispatch<LIFT_OP_ASUM>(o, item.begin, item.end, red)
                                           : reduce_dispatch<LIFT_OP_DOT>(o, item.begin, item.end, red);
      if (threadIdx.x == 0) {
        B.partials[it] = r;
        __threadfence();
        s_last = atomicAdd(B.op_done + item.op_index, 1u) == (unsigned)(o.num_items - 1);
      }
      __syncthreads();
      if (s_last) {
        __threadfence();
        const double s = combine_partials<kThreads>(B.partials + o.first_item, o.num_items, red64);
        if (threadIdx.x == 0) *o.out = static_cast<float>(s);
      }
    } else if (o.op == LIFT_OP_SCAL) {
      switch (o.mode) {
        case 0: scal_item<1, 4>(o, item.begin, item.end); break;
        case 1: scal_item<4, 1>(o, item.begin, item.end); break;
        case 2: scal_item<4, 2>(o, item.begin, item.end); break;
        case 3: scal_item<4, 4>(o, item.begin, item.end); break;
        case 4: scal_item<8, 1>(o, item.begin, item.end); break;
        default: scal_item<8, 2>(o, item.begin, item.end); break;
      }
    } else {
      switch (o.mode) {
        case 0: gemv_item<1>(o, item.begin, item.end); break;
        case 1: gemv_item<4>(o, item.begin, item.end); break;
        default: gemv_item<8>(o, item.begin, item.end); break;
      }
    }
    if constexpr (!QUEUE) return;
    __syncthreads();   // shared state is reused by the next item
  }
}

// The kernels: batches of vector ops leave the register allocation to the
// compiler (64 registers, 4 CTAs per SM); batches with gemv ops ask for 5
// CTAs per SM (48 registers): their warp-per-row items keep more rows in
// flight with the extra warps (the 20,000-op workload: 8.89 ms against
// 9.44 ms), while vector ops alone ran about 1 % slower that way.
template <bool QUEUE>
__global__ void __launch_bounds__(kThreads) batch_kernel(BatchDev B) {
  batch_body<QUEUE>(B);
}

template <bool QUEUE>
__global__ void __launch_bounds__(kThreads, 5) batch_kernel_gemv(BatchDev B) {
  batch_body<QUEUE>(B);
}

}  // namespace
}  // namespace lift

struct lift_batch {
  int device = -1;
  int64_t count = 0, num_items = 0, bytes = 0;
  std::vector<lift::OpDev> ops_host;
  std::vector<int> mode;      // per op: the mode used
  std::vector<int> variant;   // per op: the policy's variant choice
  std::vector<int64_t> item;  // per op: elements (or rows) per work item
  lift::OpDev* ops = nullptr;
  lift::ItemDev* items = nullptr;
  int64_t* order = nullptr;
  float* partials = nullptr;
  unsigned* op_done = nullptr;
  unsigned long long* head = nullptr;
  int64_t grid = 0;           // CTAs of the persistent (queue) grid
  int schedule = LIFT_BATCH_QUEUE;
  bool gemv_occupancy = false;  // a gemv op is present: the 5-CTAs-per-SM kernel
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

using namespace lift;

namespace lift {
namespace {

int vec_mode_for(const lift_variant_info& v) {
  for (int m = 0; m < kNumVecModes; ++m)
    if (kThreads * kVecModes[m].vw * kVecModes[m].j == v.tile && kVecModes[m].vw == v.vw) return m;
  if (v.vw == 1) return 0;
  if (v.vw == 4) return v.tile >= 4096 ? 3 : (v.tile >= 2048 ? 2 : 1);
  return v.tile >= 4096 ? 5 : 4;
}

void free_batch(lift_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->ops);
  cudaFree(b->items);
  cudaFree(b->order);
  cudaFree(b->partials);
  cudaFree(b->op_done);
  cudaFree(b->head);
  delete b;
}

int64_t op_bytes(const lift_op_desc& d) {
  switch (d.op) {
    case LIFT_OP_ASUM: return 4 * d.n;
    case LIFT_OP_DOT: return 8 * d.n;
    case LIFT_OP_SCAL: return 8 * d.n;
    default: return 4 * d.M * d.N + 4 * d.N + (d.beta != 0.f ? 8 : 4) * d.M;
  }
}

}  // namespace
}  // namespace lift

extern "C" {

lift_status lift_batch_create(const lift_op_desc* descs, int64_t count, lift_batch** out) {
  if (!out || count < 0 || (count > 0 && !descs))
    return set_error(LIFT_ERR_INVALID_ARG, "batch_create arguments");
  *out = nullptr;
  // validate everything before touching the device
  for (int64_t i = 0; i < count; ++i) {
    const lift_op_desc& d = descs[i];
    const std::string at = "batch op " + std::to_string(i) + ": ";
    if (d.op != LIFT_OP_ASUM && d.op != LIFT_OP_DOT && d.op != LIFT_OP_SCAL && d.op != LIFT_OP_GEMV)
      return set_error(LIFT_ERR_INVALID_ARG, at + "op id out of range");
    if (d.variant < -1 || d.variant >= (int)registry(d.op).size())
      return set_error(LIFT_ERR_INVALID_ARG, at + "variant id out of range");
    if (!d.out) return set_error(LIFT_ERR_INVALID_ARG, at + "out is NULL");
    if (d.op == LIFT_OP_GEMV) {
      if (d.M < 0 || d.N < 0 || d.lda < d.N) return set_error(LIFT_ERR_INVALID_ARG, at + "gemv sizes");
      if (d.M > 0 && d.N > 0 && (!d.A || !d.x)) return set_error(LIFT_ERR_INVALID_ARG, at + "gemv A/x");
    } else {
      if (d.n < 0) return set_error(LIFT_ERR_INVALID_ARG, at + "n < 0");
      if (d.n > 0 && !d.x) return set_error(LIFT_ERR_INVALID_ARG, at + "x is NULL");
      if (d.op == LIFT_OP_DOT && d.n > 0 && !d.y) return set_error(LIFT_ERR_INVALID_ARG, at + "y is NULL");
    }
    const void* ptrs[] = {d.x, d.y, d.A, d.out};
    for (const void* p : ptrs)
      if (p && !aligned(p, 4)) return set_error(LIFT_ERR_INVALID_ARG, at + "pointer not 4-byte aligned");
  }
  DeviceState* st = current_state();
  if (!st) return set_error(LIFT_ERR_NOT_INITIALIZED, "lift_init was not called for this device");
  lift_batch* b = new lift_batch();
  cudaGetDevice(&b->device);
  b->count = count;
  b->ops_host.resize(count);
  b->mode.resize(count);
  b->variant.resize(count);
  b->item.resize(count);
  std::vector<ItemDev> items;
  std::vector<std::pair<int64_t, int64_t>> cost;   // (bytes, item) for the queue order
  for (int64_t i = 0; i < count; ++i) {
    const lift_op_desc& d = descs[i];
    OpDev o{};
    o.op = d.op;
    o.n = d.n;
    o.M = d.M;
    o.N = d.N;
    o.lda = d.lda;
    o.alpha = d.alpha;
    o.beta = d.beta;
    o.x = d.x;
    o.y = d.y;
    o.A = d.A;
    o.out = d.out;
    int v = d.variant;
    if (v < 0) lift_pick(d.op, d.n, d.M, d.N, &v);
    b->variant[i] = v;
    const lift_variant_info& info = registry(d.op)[v].info;
    o.first_item = (int64_t)items.size();
    if (d.op == LIFT_OP_GEMV) {
      int m = info.vw == 8 ? 2 : (info.vw == 4 ? 1 : 0);
      const int vw = kGemvVW[m];
      if (!aligned(d.A, 4 * vw) || !aligned(d.x, 4 * vw) || (d.lda * 4) % (4 * vw) != 0) m = 0;
      o.mode = m;
      const int64_t row_bytes = 4 * (d.N > 0 ? d.N : 1);
      int64_t rows = std::max<int64_t>(8, kItemBytes / row_bytes / 8 * 8);
      b->item[i] = rows;
      for (int64_t r = 0; r < d.M; r += rows) {
        const int64_t e = std::min(d.M, r + rows);
        cost.push_back({(e - r) * row_bytes, (int64_t)items.size()});
        items.push_back({(int)i, r, e});
      }
    } else {
      int m = vec_mode_for(info);
      const int vw = kVecModes[m].vw;
      const bool ok = aligned(d.x, 4 * vw) && (d.op != LIFT_OP_DOT || aligned(d.y, 4 * vw)) &&
                      (d.op != LIFT_OP_SCAL || aligned(d.out, 4 * vw));
      if (!ok) m = 0;
      o.mode = m;
      const int64_t tile = (int64_t)kThreads * kVecModes[m].vw * kVecModes[m].j;
      const int64_t esz = d.op == LIFT_OP_ASUM ? 4 : 8;
      const int64_t per = std::max<int64_t>(1, kItemBytes / (tile * esz)) * tile;
      b->item[i] = per;
      if (d.n == 0 && d.op != LIFT_OP_SCAL) {
        cost.push_back({0, (int64_t)items.size()});
        items.push_back({(int)i, 0, 0});   // one empty item: the combine writes 0
      }
      for (int64_t s = 0; s < d.n; s += per) {
        const int64_t e = std::min(d.n, s + per);
        cost.push_back({(e - s) * esz, (int64_t)items.size()});
        items.push_back({(int)i, s, e});
      }
    }
    o.num_items = (int64_t)items.size() - o.first_item;
    b->mode[i] = o.mode;
    b->ops_host[i] = o;
    b->bytes += op_bytes(d);
  }
  b->num_items = (int64_t)items.size();
  std::stable_sort(cost.begin(), cost.end(),
                   [](const std::pair<int64_t, int64_t>& a, const std::pair<int64_t, int64_t>& c) {
                     return a.first > c.first;
                   });
  std::vector<int64_t> order(items.size());
  for (size_t k = 0; k < cost.size(); ++k) order[k] = cost[k].second;

  const size_t ni = std::max<size_t>(1, items.size()), no = std::max<int64_t>(1, count);
  lift_status rc = cuda_check(cudaMalloc(&b->ops, no * sizeof(OpDev)), "batch alloc");
  if (rc == LIFT_OK) rc = cuda_check(cudaMalloc(&b->items, ni * sizeof(ItemDev)), "batch alloc");
  if (rc == LIFT_OK) rc = cuda_check(cudaMalloc(&b->order, ni * sizeof(int64_t)), "batch alloc");
  if (rc == LIFT_OK) rc = cuda_check(cudaMalloc(&b->partials, ni * sizeof(float)), "batch alloc");
  if (rc == LIFT_OK) rc = cuda_check(cudaMalloc(&b->op_done, no * sizeof(unsigned)), "batch alloc");
  if (rc == LIFT_OK) rc = cuda_check(cudaMalloc(&b->head, sizeof(unsigned long long)), "batch alloc");
  if (rc == LIFT_OK && count > 0)
    rc = cuda_check(cudaMemcpy(b->ops, b->ops_host.data(), count * sizeof(OpDev), cudaMemcpyHostToDevice),
                    "batch upload");
  if (rc == LIFT_OK && !items.empty())
    rc = cuda_check(cudaMemcpy(b->items, items.data(), items.size() * sizeof(ItemDev),
                               cudaMemcpyHostToDevice), "batch upload");
  if (rc == LIFT_OK && !items.empty())
    rc = cuda_check(cudaMemcpy(b->order, order.data(), order.size() * sizeof(int64_t),
                               cudaMemcpyHostToDevice), "batch upload");
  if (rc == LIFT_OK) {
    int per_sm = 0;
    b->gemv_occupancy = std::any_of(b->ops_host.begin(), b->ops_host.end(),
                                    [](const OpDev& o) { return o.op == LIFT_OP_GEMV; });
    rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                        &per_sm, b->gemv_occupancy ? batch_kernel_gemv<true> : batch_kernel<true>,
                        kThreads, 0),
                    "batch occupancy");
    b->grid = (int64_t)per_sm * st->sm_count;
    if (b->grid > b->num_items) b->grid = std::max<int64_t>(1, b->num_items);
  }
  if (rc != LIFT_OK) {
    free_batch(b);
    return rc;
  }
  *out = b;
  return LIFT_OK;
}

// The graph: memset(head, op counters) -> batch_kernel, captured once on a
// private stream, then launched on the caller's stream.
lift_status lift_batch_run(lift_batch* b, void* stream) {
  if (!b) return set_error(LIFT_ERR_INVALID_ARG, "batch is NULL");
  if (b->num_items == 0) return LIFT_OK;
  if (!b->exec) {
    cudaStream_t cap;
    lift_status rc = cuda_check(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "stream");
    if (rc != LIFT_OK) return rc;
    rc = cuda_check(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "capture");
    if (rc == LIFT_OK) {
      cudaMemsetAsync(b->head, 0, sizeof(unsigned long long), cap);
      cudaMemsetAsync(b->op_done, 0, std::max<int64_t>(1, b->count) * sizeof(unsigned), cap);
      BatchDev B{b->ops, b->items, b->order, b->partials, b->op_done, b->head, b->num_items};
      const bool q = b->schedule == LIFT_BATCH_QUEUE;
      const unsigned g = (unsigned)(q ? b->grid : b->num_items);
      if (q && b->gemv_occupancy) batch_kernel_gemv<true><<<g, kThreads, 0, cap>>>(B);
      else if (q) batch_kernel<true><<<g, kThreads, 0, cap>>>(B);
      else if (b->gemv_occupancy) batch_kernel_gemv<false><<<g, kThreads, 0, cap>>>(B);
      else batch_kernel<false><<<g, kThreads, 0, cap>>>(B);
      rc = cuda_check(cudaStreamEndCapture(cap, &b->graph), "end capture");
    }
    if (rc == LIFT_OK) rc = cuda_check(cudaGraphInstantiate(&b->exec, b->graph, 0), "instantiate");
    cudaStreamDestroy(cap);
    if (rc != LIFT_OK) return rc;
  }
  return cuda_check(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)), "graph launch");
}

lift_status lift_batch_set_schedule(lift_batch* b, int schedule) {
  if (!b) return set_error(LIFT_ERR_INVALID_ARG, "batch is NULL");
  if (schedule != LIFT_BATCH_QUEUE && schedule != LIFT_BATCH_PER_ITEM)
    return set_error(LIFT_ERR_INVALID_ARG, "batch schedule");
  if (schedule == LIFT_BATCH_PER_ITEM && b->num_items > INT32_MAX)
    return set_error(LIFT_ERR_UNSUPPORTED, "more work items than CTAs in a grid");
  if (schedule == b->schedule) return LIFT_OK;
  // the next run captures the graph again; a launch of the old one may still
  // be in flight on some stream, so let the device drain first
  if (b->exec) cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->schedule = schedule;
  return LIFT_OK;
}

int lift_batch_schedule(const lift_batch* b) { return b ? b->schedule : -1; }

lift_status lift_batch_info(const lift_batch* b, int64_t* items, int64_t* bytes, int64_t* grid) {
  if (!b) return set_error(LIFT_ERR_INVALID_ARG, "batch is NULL");
  if (items) *items = b->num_items;
  if (bytes) *bytes = b->bytes;
  if (grid) *grid = b->schedule == LIFT_BATCH_QUEUE ? b->grid : b->num_items;
  return LIFT_OK;
}

lift_status lift_batch_op_choice(const lift_batch* b, int64_t i, int* variant, int* mode,
                                 int64_t* item) {
  if (!b || i < 0 || i >= b->count) return set_error(LIFT_ERR_INVALID_ARG, "batch op index");
  if (variant) *variant = b->variant[i];
  if (mode) *mode = b->mode[i];
  if (item) *item = b->item[i];
  return LIFT_OK;
}

lift_status lift_batch_destroy(lift_batch* b) {
  if (!b) return LIFT_OK;
  cudaDeviceSynchronize();
  free_batch(b);
  return LIFT_OK;
}

}  // extern "C"
