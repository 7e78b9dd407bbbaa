// C-ABI of liftblas (include/lift.h): device state, argument validation,
// variant registry and policy, and the extern "C" entry points.
#include <dlfcn.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <tuple>

#include "lift_internal.cuh"

namespace lift {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

lift_status set_error(lift_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

static std::atomic<uint32_t> g_wait_polls{kWaitPolls};
uint32_t wait_polls() { return g_wait_polls.load(); }

lift_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LIFT_OK;
  return set_error(e == cudaErrorMemoryAllocation ? LIFT_ERR_NO_MEMORY : LIFT_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// device state
// ---------------------------------------------------------------------------
static std::mutex g_mu;
static std::map<int, DeviceState*> g_states;
constexpr int64_t kPartialCapacity = 1 << 22;   // fp32 partial slots per workspace slot (16 MiB)
constexpr int64_t kPartial64Capacity = 1 << 17; // FP64 partial slots per workspace slot (1 MiB)
extern const int kTicketSlots = 64 + 65536;     // counters: reductions, then gemv-T column blocks

DeviceState* current_state() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_states.find(dev);
  return it == g_states.end() ? nullptr : it->second;
}

static Workspace& slot(DeviceState* st, int i) { return i == 0 ? st->ws : st->more[i - 1]; }

// stream -> workspace slot, per device; a new stream takes the next slot
static std::map<std::pair<DeviceState*, cudaStream_t>, int> g_slot_of;
static std::map<DeviceState*, int> g_next_slot;

Workspace* stream_workspace(DeviceState* st, cudaStream_t stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto key = std::make_pair(st, stream);
  auto it = g_slot_of.find(key);
  if (it == g_slot_of.end()) {
    // a long-running process may see many short-lived streams: forget the
    // assignments once there are many (slots are then dealt afresh)
    if (g_slot_of.size() >= 4096) g_slot_of.clear();
    int& nx = g_next_slot[st];
    it = g_slot_of.emplace(key, nx).first;
    nx = (nx + 1) % kWsSlots;
  }
  return &slot(st, it->second);
}

static void free_slots(DeviceState* st) {
  for (int i = 0; i < kWsSlots; ++i) {
    Workspace& w = slot(st, i);
    cudaFree(w.partials);
    cudaFree(w.partials64);
    cudaFree(w.tickets);
    w = Workspace();
  }
}

// Serialises whole initialisations, so two threads that call lift_init for
// the same device at once set it up once (g_mu is held only around the
// table, not across the allocations).
static std::mutex g_init_mu;

static lift_status init_device(int device) {
  std::lock_guard<std::mutex> init_lk(g_init_mu);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_states.count(device)) return LIFT_OK;
  }
  int prev = -1;
  lift_status rc = cuda_check(cudaGetDevice(&prev), "cudaGetDevice");
  if (rc != LIFT_OK) return rc;
  rc = cuda_check(cudaSetDevice(device), "cudaSetDevice");
  if (rc != LIFT_OK) return rc;
  DeviceState* st = new DeviceState();
  st->device = device;
  rc = cuda_check(cudaDeviceGetAttribute(&st->sm_count, cudaDevAttrMultiProcessorCount, device),
                  "SM count");
  int* status = nullptr;
  if (rc == LIFT_OK) rc = cuda_check(cudaMalloc(&status, sizeof(int)), "workspace");
  if (rc == LIFT_OK) rc = cuda_check(cudaMemset(status, 0, sizeof(int)), "memset");
  for (int i = 0; i < kWsSlots && rc == LIFT_OK; ++i) {
    Workspace& w = slot(st, i);
    rc = cuda_check(cudaMalloc(&w.partials, kPartialCapacity * sizeof(float)), "workspace");
    if (rc == LIFT_OK)
      rc = cuda_check(cudaMalloc(&w.partials64, kPartial64Capacity * sizeof(double)), "workspace");
    if (rc == LIFT_OK)
      rc = cuda_check(cudaMalloc(&w.tickets, kTicketSlots * sizeof(unsigned)), "workspace");
    if (rc == LIFT_OK)
      rc = cuda_check(cudaMemset(w.tickets, 0, kTicketSlots * sizeof(unsigned)), "memset");
    w.status = status;
    w.capacity = kPartialCapacity;
    w.capacity64 = kPartial64Capacity;
  }
  if (rc == LIFT_OK) rc = cuda_check(cudaDeviceSynchronize(), "init sync");
  if (rc != LIFT_OK) {
    free_slots(st);
    cudaFree(status);
    delete st;
    cudaSetDevice(prev);
    return rc;
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_states[device] = st;
  }
  cudaSetDevice(prev);
  return LIFT_OK;
}

// ---------------------------------------------------------------------------
// registry
// ---------------------------------------------------------------------------
void register_gemv_tma(std::vector<Variant>& gemv);   // gemv_tma.cu
void register_gemv_tmap(std::vector<Variant>& gemv);  // gemv_tma.cu (tensor-copy forms)
void register_reduce_f32(std::vector<Variant>& asum, std::vector<Variant>& dot,
                         std::vector<Variant>& nrm2, std::vector<Variant>& sum);  // reduce_f32.cu
void register_axpy(std::vector<Variant>& axpy);       // scal_gemv.cu
void register_gemv_t(std::vector<Variant>& gemv_t);   // gemv_t.cu
void gemv_t_shape(int id, const Args& a, int64_t* B, int64_t* RB);
void register_gemv_split(std::vector<Variant>& gemv);  // gemv_split.cu
void register_gemv_pertile(std::vector<Variant>& gemv);  // scal_gemv.cu (one CTA per row group)
void register_blackscholes(std::vector<Variant>& bs);  // blackscholes.cu
void register_compensated(std::vector<Variant>& asum, std::vector<Variant>& dot);  // compensated.cu
void register_reduce_derived(std::vector<Variant>& asum, std::vector<Variant>& dot);  // reduce_derived.cu
void gemv_split_shape(int k, const Args& a, int64_t* L, int64_t* S);
lift_status gemv_t_empty_rows(int64_t N, float beta, float* y, cudaStream_t s);

static std::vector<Variant> g_ops[LIFT_NUM_OPS];
static std::once_flag g_reg_once;

static void build_registry() {
  register_reduce_f32(g_ops[LIFT_OP_ASUM], g_ops[LIFT_OP_DOT], g_ops[LIFT_OP_NRM2],
                      g_ops[LIFT_OP_SUM]);
  register_reduce_derived(g_ops[LIFT_OP_ASUM], g_ops[LIFT_OP_DOT]);
  register_scal(g_ops[LIFT_OP_SCAL]);
  register_gemv(g_ops[LIFT_OP_GEMV]);
  register_gemv_tma(g_ops[LIFT_OP_GEMV]);
  register_gemv_split(g_ops[LIFT_OP_GEMV]);
  register_gemv_tmap(g_ops[LIFT_OP_GEMV]);
  register_gemv_pertile(g_ops[LIFT_OP_GEMV]);
  register_mixed(g_ops);
  register_axpy(g_ops[LIFT_OP_AXPY]);
  register_gemv_t(g_ops[LIFT_OP_GEMV_T]);
  register_blackscholes(g_ops[LIFT_OP_BLACKSCHOLES]);
  register_compensated(g_ops[LIFT_OP_ASUM_COMP], g_ops[LIFT_OP_DOT_COMP]);
}

std::vector<Variant>& registry(int op) {
  std::call_once(g_reg_once, build_registry);
  return g_ops[op];
}

int64_t persistent_grid(const void* kernel, int threads, size_t smem, int cluster) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int64_t> cache;
  int dev = -1;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({dev, kernel});
    if (it != cache.end()) return it->second;
  }
  DeviceState* st = current_state();
  if (!st) return 0;
  if (smem > 0 &&
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess)
    return 0;
  int64_t g = (int64_t)per_sm * st->sm_count;
  g = g / cluster * cluster;
  std::lock_guard<std::mutex> lk(mu);
  cache[{dev, kernel}] = g;
  return g;
}

lift_status launch_config(const void* kernel, dim3 grid, dim3 block, size_t smem, int cluster,
                          cudaStream_t s, void** args, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  unsigned na = 0;
  if (cluster > 1) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = cluster;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  if (pdl) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = na ? attr : nullptr;
  cfg.numAttrs = na;
  return cuda_check(cudaLaunchKernelExC(&cfg, kernel, args), "kernel launch");
}

// ---------------------------------------------------------------------------
// policy
// ---------------------------------------------------------------------------
struct TableEntry {
  double ln, lm, lN;
  int variant;
};

struct Box {                         // trained range of one op, in log2(size + 1)
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};   // n (M*N for matrices), M, N
  bool known = false;
};

struct Mlp {
  Box box[LIFT_NUM_OPS];
  int d_in = 0, h1 = 0, h2 = 0, V = 0;
  int ops = 0;                       // op ids 0 .. ops-1 have an output slice
  int offsets[LIFT_MLP_OPS] = {0};
  std::vector<float> W1, b1, W2, b2, W3, b3;
};

static int g_policy = LIFT_POLICY_FIXED;
static int g_override[LIFT_NUM_OPS] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
static std::vector<TableEntry> g_table[LIFT_NUM_OPS];
static Mlp g_mlp;
static std::mutex g_policy_mu;

// Defaults of the FIXED policy: per op, a variant that is the autotuner's
// best or within a few per cent of it at the benchmark configurations of that
// op on the GB300 (the learned and table policies adapt to other shapes).
// Variant names; looked up at first use.
static const char* kDefaultName[LIFT_NUM_OPS] = {
    "asum_t4096_v4_ldg_p2", "dot_t4096_v4_ldg_p2", "scal_t2048_v4_ldg_pertile",
    "gemv_tma_w4_c1024_s3", "asum_bf16_t256_u4", "dot_bf16_t256_u4", "asum_fp8_t256_u8_c",
    "dot_fp8_t128_u2", "nrm2_t4096_v4_ldg_p2", "sum_t4096_v4_ldg_p2", "axpy_t2048_v4_ldg_pertile",
    "gemv_t_t128_v4_r16_s3", "blackscholes_t128_v4_u4_fast_pertile", "asum_comp_t256_v4_u4",
    "dot_comp_t256_v4_u4"};

static int find_variant(int op, const char* name) {
  auto& L = registry(op);
  if (name)
    for (size_t i = 0; i < L.size(); ++i)
      if (strcmp(L[i].info.name, name) == 0) return (int)i;
  return L.empty() ? -1 : 0;
}

}  // namespace lift

using namespace lift;

extern "C" {

// Features of a call for the cost model: one-hot op family (asum, dot,
// scal, gemv), log2(n+1)/32, log2(M+1)/16, log2(N+1)/16, one-hot dtype
// (fp32, bf16, fp8).  For gemv n = M*N.
lift_status lift_features(int op, int64_t n, int64_t M, int64_t N, float* out) {
  if (op < 0 || op >= LIFT_MLP_OPS || !out) return LIFT_ERR_INVALID_ARG;
  static const int fam[LIFT_MLP_OPS] = {0, 1, 2, 3, 0, 1, 0, 1, 0, 0, 2, 3, 2, 0, 1};
  static const int dt[LIFT_MLP_OPS] = {0, 0, 0, 0, 1, 1, 2, 2, 0, 0, 0, 0, 0, 0, 0};
  for (int i = 0; i < LIFT_NUM_FEATURES; ++i) out[i] = 0.f;
  out[fam[op]] = 1.f;
  const bool matrix = op == LIFT_OP_GEMV || op == LIFT_OP_GEMV_T;
  if (matrix) n = M * N;
  out[4] = (float)(log2((double)n + 1.0) / 32.0);
  out[5] = (float)(log2((double)M + 1.0) / 16.0);
  out[6] = (float)(log2((double)N + 1.0) / 16.0);
  out[7 + dt[op]] = 1.f;
  if (matrix) {                 // whole 16- and 32-byte vectors per dense row
    out[10] = N % 4 == 0 ? 1.f : 0.f;
    out[11] = N % 8 == 0 ? 1.f : 0.f;
  }
  return LIFT_OK;
}

}  // extern "C"

namespace lift {

static bool ptr_ok(const void* p, int bytes) { return p == nullptr || aligned(p, bytes); }

// Whether variant v runs as itself on these arguments: its vector loads need
// the pointers (and, gemv and gemv-T, the row pitch) aligned to its vector
// width, and the bulk-copy gemv and gemv-T need whole 16-byte row granules.  Otherwise
// the library runs the variant's guarded fallback instead.
static bool eligible(int op, const Variant& v, const Args& a) {
  const int al = v.align_bytes;
  bool ok = ptr_ok(a.x, al) && ptr_ok(a.y, al) && ptr_ok(a.A, al) && ptr_ok(a.out, al);
  if (op == LIFT_OP_BLACKSCHOLES) ok = ok && ptr_ok(a.result, al);   // the put array
  if (op == LIFT_OP_GEMV || op == LIFT_OP_GEMV_T) ok = ok && ((a.lda * 4) % al == 0);
  if ((op == LIFT_OP_GEMV || op == LIFT_OP_GEMV_T) && v.info.stages > 0)
    ok = ok && a.N > 0 && a.N % 4 == 0;
  // tensor copies: whole 256-float runs per row, 16-byte row strides
  if (op == LIFT_OP_GEMV && v.info.tree == 3) ok = ok && a.N % 256 == 0 && a.lda % 4 == 0;
  return ok;
}

// The learned ranking: (predicted log-time, variant) of every variant that
// runs as itself on these arguments, fastest first; the pick is the first.
static std::vector<std::pair<float, int>> mlp_rank(int op, const Args& a) {
  const Mlp& m = g_mlp;
  float f[LIFT_NUM_FEATURES];
  lift_features(op, a.n, a.M, a.N, f);
  std::vector<float> h1(m.h1), h2(m.h2);
  for (int j = 0; j < m.h1; ++j) {
    float s = m.b1[j];
    for (int i = 0; i < m.d_in; ++i) s += f[i] * m.W1[i * m.h1 + j];
    h1[j] = s > 0.f ? s : 0.f;
  }
  for (int j = 0; j < m.h2; ++j) {
    float s = m.b2[j];
    for (int i = 0; i < m.h1; ++i) s += h1[i] * m.W2[i * m.h2 + j];
    h2[j] = s > 0.f ? s : 0.f;
  }
  // variants the weights know: the file's slice of this op (a registry that
  // grew after training keeps its newer variants out of the pick)
  const int file_cnt = (op + 1 < m.ops ? m.offsets[op + 1] : m.V) - m.offsets[op];
  const auto& L = registry(op);
  const int cnt = std::min((int)L.size(), file_cnt);
  std::vector<std::pair<float, int>> r;   // empty: the caller falls back to the FIXED choice
  for (int v = 0; v < cnt; ++v) {
    const int o = m.offsets[op] + v;
    if (o >= m.V) break;
    if (!eligible(op, L[v], a)) continue;
    float s = m.b3[o];
    for (int i = 0; i < m.h2; ++i) s += h2[i] * m.W3[i * m.V + o];
    r.emplace_back(s, v);
  }
  std::stable_sort(r.begin(), r.end(),
                   [](const std::pair<float, int>& p, const std::pair<float, int>& q) {
                     return p.first < q.first;
                   });
  return r;
}

static int mlp_pick(int op, const Args& a) {
  const auto r = mlp_rank(op, a);
  return r.empty() ? -1 : r[0].second;
}

// The tuned table: the variant of the nearest tuned shape (log sizes) among
// the entries whose variant runs as itself on these arguments.
static int table_pick(int op, const Args& a) {
  const auto& T = g_table[op];
  if (T.empty()) return -1;
  const int64_t n = a.n, M = a.M, N = a.N;
  const double ln = log2((double)(op == LIFT_OP_GEMV ? M * N : n) + 1.0);
  const double lm = log2((double)M + 1.0), lN = log2((double)N + 1.0);
  const auto& L = registry(op);
  double best = INFINITY;
  int v = -1;
  for (const auto& e : T) {
    if (e.variant < 0 || e.variant >= (int)L.size() || !eligible(op, L[e.variant], a)) continue;
    const double d = (e.ln - ln) * (e.ln - ln) + (e.lm - lm) * (e.lm - lm) + (e.lN - lN) * (e.lN - lN);
    if (d < best) {
      best = d;
      v = e.variant;
    }
  }
  return v;
}

// ---------------------------------------------------------------------------
// MLP_TUNE: the learned pick, with exhaustive timing of candidates as its
// fallback where the model is unsure -- a call outside the box of shapes it
// was trained on, or (for working sets of at least twice the L2, which the
// timing reads cold like the autotuner does) one whose two best predicted
// times are within kTuneMargin of each other.  The candidates are the
// model's kTuneTopK best, the FIXED default and every variant added to the
// library after the model was trained; each is timed as the autotuner times
// (a CUDA graph of kTuneCalls back-to-back launches, replayed kTuneReps
// times, the candidates interleaved, median per candidate) on a private
// stream that waits for the call's stream, with the outputs sent to scratch
// so the caller's arrays are only read.  The winner is cached per (op,
// shape, alignment).  Inside stream capture, and in lift_pick, nothing is
// timed: a cached winner or the plain learned pick is used.
// ---------------------------------------------------------------------------
constexpr float kTuneMargin = 0.03f;   // in predicted log-time: about 3 %
constexpr int kTuneTopK = 3;
constexpr int kTuneCalls = 4;
constexpr int kTuneReps = 5;
constexpr double kBoxSlack = 0.1;      // log2 units beyond the trained range still inside

struct TuneKey {
  int op;
  int64_t n, M, N;
  uint64_t align;   // alignment_signature: which of the op's variants run as themselves
  bool operator<(const TuneKey& o) const {
    return std::tie(op, n, M, N, align) < std::tie(o.op, o.n, o.M, o.N, o.align);
  }
};
static std::map<TuneKey, int> g_tuned;
static std::map<TuneKey, int> g_picked;    // learned picks, memoised per call shape
constexpr size_t kPickCacheMax = 1 << 16;
static std::atomic<int64_t> g_tune_launches{0};
static std::mutex g_tune_mu;          // one timing at a time
static uint64_t g_policy_gen = 0;     // bumped whenever a policy is loaded

static bool in_box(int op, const Args& a) {
  const Box& b = g_mlp.box[op];
  if (!b.known) return true;
  const bool matrix = op == LIFT_OP_GEMV || op == LIFT_OP_GEMV_T;
  const double v[3] = {log2((double)(matrix ? a.M * a.N : a.n) + 1.0), log2((double)a.M + 1.0),
                       log2((double)a.N + 1.0)};
  for (int i = 0; i < (matrix ? 3 : 1); ++i)
    if (v[i] < b.lo[i] - kBoxSlack || v[i] > b.hi[i] + kBoxSlack) return false;
  return true;
}

// Bytes the call reads (its inputs): what decides whether repeated timing
// reads cold data.
static double input_bytes(int op, const Args& a) {
  switch (op) {
    case LIFT_OP_GEMV:
    case LIFT_OP_GEMV_T: return 4.0 * a.M * a.N;
    case LIFT_OP_DOT:
    case LIFT_OP_DOT_COMP:
    case LIFT_OP_AXPY: return 8.0 * a.n;
    case LIFT_OP_ASUM_BF16: return 2.0 * a.n;
    case LIFT_OP_DOT_BF16: return 4.0 * a.n;
    case LIFT_OP_ASUM_FP8: return 1.0 * a.n;
    case LIFT_OP_DOT_FP8: return 2.0 * a.n;
    default: return 4.0 * a.n;
  }
}

// What decides which variants run as themselves (see eligible): the
// pointers' residues modulo 32 bytes (the widest vector), and for the
// matrices the row pitch and width residues modulo 256 elements.
static uint64_t alignment_signature(int op, const Args& a) {
  auto r = [](const void* p) { return (uint64_t)(reinterpret_cast<uintptr_t>(p) % 32); };
  uint64_t sig = r(a.x) | r(a.y) << 5 | r(a.A) << 10 | r(a.out) << 15;
  if (op == LIFT_OP_BLACKSCHOLES) sig |= r(a.result) << 20;
  if (op == LIFT_OP_GEMV || op == LIFT_OP_GEMV_T)
    sig |= (uint64_t)(a.lda % 256) << 25 | (uint64_t)(a.N % 256) << 33 | (uint64_t)(a.N > 0) << 41;
  return sig;
}

static double l2_bytes() {
  int dev = 0, l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0.0;
  }
  return (double)l2;
}

static bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return true;       // unknown: do not time
  }
  return st != cudaStreamCaptureStatusNone;
}

// Time the candidates; returns the fastest, or -1 on any error.
static int tune_candidates(int op, const Args& a0, const std::vector<int>& cand, cudaStream_t s) {
  DeviceState* st = current_state();
  if (!st || cand.empty()) return -1;
  Args a = a0;
  // outputs to scratch: reductions write their scalar to the workspace's
  // spare slot; writing ops get a temporary output array
  int64_t outs = 0;
  if (op == LIFT_OP_SCAL || op == LIFT_OP_AXPY) outs = a.n;
  if (op == LIFT_OP_BLACKSCHOLES) outs = 2 * a.n;
  if (op == LIFT_OP_GEMV) outs = a.M;
  if (op == LIFT_OP_GEMV_T) outs = a.N;
  float* scratch = nullptr;
  if (outs > 0) {
    if (cudaMalloc(&scratch, outs * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    if (op == LIFT_OP_AXPY) a.y = scratch;     // y is read and written in place
    a.out = scratch;
    if (op == LIFT_OP_BLACKSCHOLES) a.result = scratch + a.n;
  } else {
    a.result = a.ws->partials + (a.ws->capacity - 1);
    a.result64 = nullptr;
  }
  const auto& L = registry(op);
  const size_t C = cand.size();
  std::vector<cudaGraphExec_t> exec(C, nullptr);
  std::vector<std::vector<float>> t(C);
  cudaStream_t p = nullptr;
  cudaEvent_t ready = nullptr, e0 = nullptr, e1 = nullptr;
  bool ok = cudaStreamCreateWithFlags(&p, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreate(&ready) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
            cudaEventCreate(&e1) == cudaSuccess && cudaEventRecord(ready, s) == cudaSuccess &&
            cudaStreamWaitEvent(p, ready, 0) == cudaSuccess;
  for (size_t c = 0; ok && c < C; ++c) {
    const Variant& v = L[cand[c]];
    ok = v.launch(v, a, p) == LIFT_OK;                   // warm-up: loads the kernel
    cudaGraph_t g = nullptr;
    ok = ok && cudaStreamBeginCapture(p, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      bool launched = true;
      for (int k = 0; k < kTuneCalls && launched; ++k) launched = v.launch(v, a, p) == LIFT_OK;
      ok = cudaStreamEndCapture(p, &g) == cudaSuccess && launched;
    }
    ok = ok && cudaGraphInstantiate(&exec[c], g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    ok = ok && cudaGraphLaunch(exec[c], p) == cudaSuccess;   // warm-up replay
    g_tune_launches += 1 + kTuneCalls;
  }
  for (int r = 0; ok && r < kTuneReps; ++r)
    for (size_t c = 0; ok && c < C; ++c) {
      float ms = 0.f;
      ok = cudaEventRecord(e0, p) == cudaSuccess && cudaGraphLaunch(exec[c], p) == cudaSuccess &&
           cudaEventRecord(e1, p) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
           cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      t[c].push_back(ms);
      g_tune_launches += kTuneCalls;
    }
  int best = -1;
  float best_ms = INFINITY;
  static const bool log = getenv("LIFT_TUNE_LOG") != nullptr;
  for (size_t c = 0; ok && c < C; ++c) {
    std::sort(t[c].begin(), t[c].end());
    const float med = t[c][t[c].size() / 2];
    if (log)
      fprintf(stderr, "lift tune: op %d n %lld M %lld N %lld  %-36s %.4f ms per call\n", op,
              (long long)(op == LIFT_OP_GEMV || op == LIFT_OP_GEMV_T ? a.M * a.N : a.n),
              (long long)a.M, (long long)a.N, L[cand[c]].info.name, med / kTuneCalls);
    if (med < best_ms) {
      best_ms = med;
      best = cand[c];
    }
  }
  if (p) cudaStreamSynchronize(p);
  for (auto& x : exec)
    if (x) cudaGraphExecDestroy(x);
  if (ready) cudaEventDestroy(ready);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (p) cudaStreamDestroy(p);
  if (scratch) cudaFree(scratch);
  if (!ok) {
    cudaGetLastError();
    return -1;
  }
  return best;
}

static int pick_variant(int op, const Args& a, cudaStream_t s = nullptr, bool may_tune = false) {
  std::unique_lock<std::mutex> lk(g_policy_mu);
  if (g_override[op] >= 0) return g_override[op];
  int v = -1;
  const bool learned = (g_policy == LIFT_POLICY_MLP || g_policy == LIFT_POLICY_MLP_TUNE) &&
                       g_mlp.V > 0 && op < g_mlp.ops;
  const bool matrix = op == LIFT_OP_GEMV || op == LIFT_OP_GEMV_T;   // shape = (M, N)
  const TuneKey key{op, matrix ? 0 : a.n, a.M, a.N, learned ? alignment_signature(op, a) : 0};
  if (learned) {
    auto it = g_tuned.find(key);              // a timed winner (MLP_TUNE)
    if (g_policy == LIFT_POLICY_MLP_TUNE && it != g_tuned.end()) return it->second;
    auto jt = g_picked.find(key);             // a pick made before for this shape
    if (jt != g_picked.end()) return jt->second;
  }
  auto memo = [&](int w) {
    if (g_picked.size() >= kPickCacheMax) g_picked.clear();
    g_picked[key] = w;
  };
  if (g_policy == LIFT_POLICY_MLP && learned) {
    v = mlp_pick(op, a);
    if (v >= 0) memo(v);
  }
  if (g_policy == LIFT_POLICY_MLP_TUNE && learned) {
    const auto r = mlp_rank(op, a);
    if (!r.empty()) {
      v = r[0].second;
      const bool unsure = !in_box(op, a) || (r.size() > 1 && r[1].first - r[0].first < kTuneMargin &&
                                             input_bytes(op, a) >= 2.0 * l2_bytes());
      if (!unsure) {
        memo(v);                               // no timing will ever be wanted here
      } else if (may_tune && !capturing(s)) {
        std::vector<int> cand;
        auto add = [&](int c) {
          if (c >= 0 && std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
        };
        for (size_t i = 0; i < r.size() && (int)i < kTuneTopK; ++i) add(r[i].second);
        const auto& L = registry(op);
        const int fixed = find_variant(op, kDefaultName[op]);
        if (fixed >= 0 && eligible(op, L[fixed], a)) add(fixed);
        const int known = (op + 1 < g_mlp.ops ? g_mlp.offsets[op + 1] : g_mlp.V) - g_mlp.offsets[op];
        for (int i = known; i < (int)L.size(); ++i)      // newer than the model
          if (eligible(op, L[i], a)) add(i);
        // time without holding the policy lock (other threads keep picking);
        // one timing at a time, and its winner kept only if the weights did
        // not change meanwhile
        const uint64_t gen = g_policy_gen;
        lk.unlock();
        int w = -1;
        {
          std::lock_guard<std::mutex> tk(g_tune_mu);
          w = tune_candidates(op, a, cand, s);
        }
        lk.lock();
        if (w >= 0) {
          if (g_policy_gen == gen) g_tuned[key] = w;
          v = w;
        }
      }
    }
  }
  if (g_policy == LIFT_POLICY_TABLE) v = table_pick(op, a);
  if (v < 0) v = find_variant(op, kDefaultName[op]);
  return v;
}

// Resolve the variant to run: explicit id or policy pick, then the guarded
// form when a pointer is not aligned for the chosen variant.
static lift_status resolve(int op, int variant, const Args& a, const Variant** out,
                           cudaStream_t s = nullptr, bool may_tune = false) {
  auto& L = registry(op);
  if (L.empty()) return set_error(LIFT_ERR_UNSUPPORTED, "no variants for op");
  if (variant < -1 || variant >= (int)L.size())
    return set_error(LIFT_ERR_INVALID_ARG, "variant id out of range");
  if (variant < 0) variant = pick_variant(op, a, s, may_tune);
  const Variant* v = &L[variant];
  if (!eligible(op, *v, a) && v->fallback >= 0) v = &L[v->fallback];
  *out = v;
  return LIFT_OK;
}

static lift_status run(int op, int variant, const Args& a0, void* stream) {
  DeviceState* st = current_state();
  if (!st) return set_error(LIFT_ERR_NOT_INITIALIZED, "lift_init was not called for this device");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  Args a = a0;
  a.ws = stream_workspace(st, s);
  const Variant* v = nullptr;
  lift_status rc = resolve(op, variant, a, &v, s, true);
  if (rc != LIFT_OK) return rc;
  return v->launch(*v, a, s);
}

static bool bad_n(int64_t n) { return n < 0; }

}  // namespace lift

extern "C" {

// Environment overrides, read once, at the first lift_init:
//   LIFT_POLICY  = fixed | table:<path> | mlp[:<path>] | mlp_tune[:<path>]
//                  (without a path the learned policies read the weights file
//                  that ships beside the library, data/mlp_gb300.txt)
//   LIFT_VARIANT = comma-separated variant names, each forced for its op
static std::string library_dir() {
  Dl_info info;
  if (!dladdr(reinterpret_cast<void*>(&lift_init), &info) || !info.dli_fname) return ".";
  std::string f(info.dli_fname);
  const size_t k = f.rfind('/');
  return k == std::string::npos ? "." : f.substr(0, k);
}

static lift_status apply_env() {
  const char* pol = getenv("LIFT_POLICY");
  if (pol && *pol) {
    std::string v(pol), kind = v, path;
    const size_t c = v.find(':');
    if (c != std::string::npos) {
      kind = v.substr(0, c);
      path = v.substr(c + 1);
    }
    int p = -1;
    if (kind == "fixed") p = LIFT_POLICY_FIXED;
    if (kind == "table") p = LIFT_POLICY_TABLE;
    if (kind == "mlp") p = LIFT_POLICY_MLP;
    if (kind == "mlp_tune") p = LIFT_POLICY_MLP_TUNE;
    if (p < 0) return set_error(LIFT_ERR_INVALID_ARG, "LIFT_POLICY: unknown policy " + kind);
    if (p == LIFT_POLICY_TABLE && path.empty())
      return set_error(LIFT_ERR_INVALID_ARG, "LIFT_POLICY: table needs table:<path>");
    if ((p == LIFT_POLICY_MLP || p == LIFT_POLICY_MLP_TUNE) && path.empty())
      path = library_dir() + "/data/mlp_gb300.txt";
    const lift_status rc = lift_set_policy(p, path.empty() ? nullptr : path.c_str());
    if (rc != LIFT_OK) return set_error(rc, "LIFT_POLICY: " + g_last_error);
  }
  const char* var = getenv("LIFT_VARIANT");
  if (var && *var) {
    std::stringstream ss(var);
    std::string name;
    while (std::getline(ss, name, ',')) {
      if (name.empty()) continue;
      int found = -1;
      for (int op = 0; op < LIFT_NUM_OPS && found < 0; ++op) {
        const auto& L = registry(op);
        for (size_t i = 0; i < L.size(); ++i)
          if (name == L[i].info.name) {
            found = op;
            lift_set_variant(op, (int)i);
            break;
          }
      }
      if (found < 0) return set_error(LIFT_ERR_INVALID_ARG, "LIFT_VARIANT: unknown variant " + name);
    }
  }
  return LIFT_OK;
}

lift_status lift_init(int device) {
  static std::once_flag once;
  static lift_status env_rc = LIFT_OK;
  static std::string env_msg;
  std::call_once(once, [] {
    env_rc = apply_env();
    if (env_rc != LIFT_OK) env_msg = g_last_error;
  });
  if (env_rc != LIFT_OK) return set_error(env_rc, env_msg);
  return init_device(device);
}

lift_status lift_finalize(void) {
  noalloc_forget();
  std::lock_guard<std::mutex> init_lk(g_init_mu);
  std::lock_guard<std::mutex> lk(g_mu);
  int prev = -1;
  cudaGetDevice(&prev);
  for (auto& kv : g_states) {
    cudaSetDevice(kv.first);
    cudaDeviceSynchronize();
    int* status = kv.second->ws.status;
    free_slots(kv.second);
    cudaFree(status);
    delete kv.second;
  }
  g_states.clear();
  g_slot_of.clear();
  g_next_slot.clear();
  if (prev >= 0) cudaSetDevice(prev);
  return LIFT_OK;
}

const char* lift_status_string(lift_status s) {
  switch (s) {
    case LIFT_OK: return "ok";
    case LIFT_ERR_INVALID_ARG: return "invalid argument";
    case LIFT_ERR_UNSUPPORTED: return "unsupported";
    case LIFT_ERR_CUDA: return "CUDA error";
    case LIFT_ERR_NO_MEMORY: return "out of device memory";
    case LIFT_ERR_TIMEOUT: return "device wait timed out";
    case LIFT_ERR_NOT_INITIALIZED: return "not initialised";
  }
  return "unknown status";
}

const char* lift_last_error(void) { return g_last_error.c_str(); }

int lift_sm_count(void) {
  DeviceState* st = current_state();
  return st ? st->sm_count : 0;
}

// device status word (timeouts recorded by kernels); reading it synchronises
int lift_read_status(int clear) {
  DeviceState* st = current_state();
  if (!st) return LIFT_ERR_NOT_INITIALIZED;
  int v = 0;
  if (cudaMemcpy(&v, st->ws.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return LIFT_ERR_CUDA;
  if (clear && v != 0) {
    // after a recorded failure, also return every "last CTA" ticket to 0
    // (a kernel that gave up still takes its ticket, so they should be; this
    // restores them whatever path the failure took).  Waits for the device.
    bool ok = cudaDeviceSynchronize() == cudaSuccess;
    for (int i = 0; i < kWsSlots && ok; ++i)
      ok = cudaMemset(slot(st, i).tickets, 0, kTicketSlots * sizeof(unsigned)) == cudaSuccess;
    ok = ok && cudaMemset(st->ws.status, 0, sizeof(int)) == cudaSuccess &&
         cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) return LIFT_ERR_CUDA;
  }
  return v;
}

lift_status lift_set_wait_polls(uint32_t polls) {
  if (polls > kWaitPolls) return set_error(LIFT_ERR_INVALID_ARG, "wait polls above the default limit");
  g_wait_polls.store(polls);
  return LIFT_OK;
}

lift_status lift_asum_v(int variant, const float* x, int64_t n, float* result, double* result_f64,
                        void* stream) {
  if (bad_n(n) || !result || (n > 0 && !x)) return set_error(LIFT_ERR_INVALID_ARG, "asum arguments");
  if (!aligned(x, 4)) return set_error(LIFT_ERR_INVALID_ARG, "x not 4-byte aligned");
  Args a;
  a.x = x;
  a.n = n;
  a.result = result;
  a.result64 = result_f64;
  return run(LIFT_OP_ASUM, variant, a, stream);
}

// The fp32 result of a shard call goes to the last fp32 workspace slot (no
// kernel uses it: grids and partial counts stay below the capacity).
static float* shard_discard(void* stream) {
  DeviceState* st = current_state();
  if (!st) return nullptr;
  Workspace* w = stream_workspace(st, static_cast<cudaStream_t>(stream));
  return w->partials + (w->capacity - 1);
}

lift_status lift_asum_partial(const float* x, int64_t n, double* partial, void* stream) {
  if (!partial) return set_error(LIFT_ERR_INVALID_ARG, "asum_partial: partial is NULL");
  float* r = shard_discard(stream);
  if (!r) return set_error(LIFT_ERR_NOT_INITIALIZED, "lift_init was not called for this device");
  return lift_asum_v(-1, x, n, r, partial, stream);
}

lift_status lift_dot_partial(const float* x, const float* y, int64_t n, double* partial,
                             void* stream) {
  if (!partial) return set_error(LIFT_ERR_INVALID_ARG, "dot_partial: partial is NULL");
  float* r = shard_discard(stream);
  if (!r) return set_error(LIFT_ERR_NOT_INITIALIZED, "lift_init was not called for this device");
  return lift_dot_v(-1, x, y, n, r, partial, stream);
}

lift_status lift_combine_partials(const double* partials, int64_t count, float* result,
                                  double* result_f64) {
  if (count < 0 || (count > 0 && !partials) || !result)
    return set_error(LIFT_ERR_INVALID_ARG, "combine_partials arguments");
  double s = 0.0;
  for (int64_t i = 0; i < count; ++i) s += partials[i];
  *result = static_cast<float>(s);
  if (result_f64) *result_f64 = s;
  return LIFT_OK;
}

lift_status lift_asum_comp_v(int variant, const float* x, int64_t n, float* result,
                             double* result_f64, void* stream) {
  if (bad_n(n) || !result || (n > 0 && !x))
    return set_error(LIFT_ERR_INVALID_ARG, "asum_comp arguments");
  if (!aligned(x, 4)) return set_error(LIFT_ERR_INVALID_ARG, "x not 4-byte aligned");
  Args a;
  a.x = x;
  a.n = n;
  a.result = result;
  a.result64 = result_f64;
  return run(LIFT_OP_ASUM_COMP, variant, a, stream);
}

lift_status lift_dot_comp_v(int variant, const float* x, const float* y, int64_t n, float* result,
                            double* result_f64, void* stream) {
  if (bad_n(n) || !result || (n > 0 && (!x || !y)))
    return set_error(LIFT_ERR_INVALID_ARG, "dot_comp arguments");
  if (!aligned(x, 4) || !aligned(y, 4))
    return set_error(LIFT_ERR_INVALID_ARG, "x/y not 4-byte aligned");
  Args a;
  a.x = x;
  a.y = y;
  a.n = n;
  a.result = result;
  a.result64 = result_f64;
  return run(LIFT_OP_DOT_COMP, variant, a, stream);
}

lift_status lift_asum_comp(const float* x, int64_t n, float* result, double* result_f64,
                           void* stream) {
  return lift_asum_comp_v(-1, x, n, result, result_f64, stream);
}

lift_status lift_dot_comp(const float* x, const float* y, int64_t n, float* result,
                          double* result_f64, void* stream) {
  return lift_dot_comp_v(-1, x, y, n, result, result_f64, stream);
}

lift_status lift_dot_v(int variant, const float* x, const float* y, int64_t n, float* result,
                       double* result_f64, void* stream) {
  if (bad_n(n) || !result || (n > 0 && (!x || !y)))
    return set_error(LIFT_ERR_INVALID_ARG, "dot arguments");
  if (!aligned(x, 4) || !aligned(y, 4)) return set_error(LIFT_ERR_INVALID_ARG, "x/y not 4-byte aligned");
  Args a;
  a.x = x;
  a.y = y;
  a.n = n;
  a.result = result;
  a.result64 = result_f64;
  return run(LIFT_OP_DOT, variant, a, stream);
}

lift_status lift_scal_v(int variant, int64_t n, float alpha, const float* x, float* y, void* stream) {
  if (bad_n(n) || (n > 0 && (!x || !y))) return set_error(LIFT_ERR_INVALID_ARG, "scal arguments");
  if (!aligned(x, 4) || !aligned(y, 4)) return set_error(LIFT_ERR_INVALID_ARG, "x/y not 4-byte aligned");
  if (n > 0 && x != y) {
    const char* xb = (const char*)x;
    const char* yb = (const char*)y;
    if (xb < yb + n * 4 && yb < xb + n * 4)
      return set_error(LIFT_ERR_INVALID_ARG, "x and y overlap without being equal");
  }
  if (n == 0) return LIFT_OK;
  Args a;
  a.x = x;
  a.out = y;
  a.n = n;
  a.alpha = alpha;
  return run(LIFT_OP_SCAL, variant, a, stream);
}

lift_status lift_gemv_v(int variant, int64_t M, int64_t N, float alpha, const float* A, int64_t lda,
                        const float* x, float beta, float* y, void* stream) {
  if (M < 0 || N < 0 || lda < N || lda < 0) return set_error(LIFT_ERR_INVALID_ARG, "gemv sizes");
  if (M > 0 && !y) return set_error(LIFT_ERR_INVALID_ARG, "gemv y is NULL");
  if (M > 0 && N > 0 && (!A || !x)) return set_error(LIFT_ERR_INVALID_ARG, "gemv A/x is NULL");
  if (!aligned(A, 4) || !aligned(x, 4) || !aligned(y, 4))
    return set_error(LIFT_ERR_INVALID_ARG, "gemv pointers not 4-byte aligned");
  Args a;
  a.A = A;
  a.x = x;
  a.out = y;
  a.M = M;
  a.N = N;
  a.lda = lda;
  a.n = M;
  a.alpha = alpha;
  a.beta = beta;
  return run(LIFT_OP_GEMV, variant, a, stream);
}

lift_status lift_asum(const float* x, int64_t n, float* result, void* stream) {
  return lift_asum_v(-1, x, n, result, nullptr, stream);
}
lift_status lift_dot(const float* x, const float* y, int64_t n, float* result, void* stream) {
  return lift_dot_v(-1, x, y, n, result, nullptr, stream);
}
lift_status lift_scal(int64_t n, float alpha, const float* x, float* y, void* stream) {
  return lift_scal_v(-1, n, alpha, x, y, stream);
}
lift_status lift_gemv(int64_t M, int64_t N, float alpha, const float* A, int64_t lda,
                      const float* x, float beta, float* y, void* stream) {
  return lift_gemv_v(-1, M, N, alpha, A, lda, x, beta, y, stream);
}

static lift_status mixed_args(lift_dtype t, const void* x, const float* xscale, int64_t n) {
  if (bad_n(n) || (n > 0 && !x)) return LIFT_ERR_INVALID_ARG;
  if (t == LIFT_BF16 && xscale) return LIFT_ERR_INVALID_ARG;
  if (t == LIFT_FP8_E4M3 && n > 0 && !xscale) return LIFT_ERR_INVALID_ARG;
  if (t != LIFT_BF16 && t != LIFT_FP8_E4M3) return LIFT_ERR_UNSUPPORTED;
  return LIFT_OK;
}

lift_status lift_asum_ex_v(int variant, lift_dtype t, const void* x, const float* xscale, int64_t n,
                           float* result, double* result_f64, void* stream) {
  if (t == LIFT_F32) return lift_asum_v(variant, (const float*)x, n, result, result_f64, stream);
  lift_status rc = mixed_args(t, x, xscale, n);
  if (rc != LIFT_OK || !result)
    return set_error(rc != LIFT_OK ? rc : LIFT_ERR_INVALID_ARG, "asum_ex arguments");
  Args a;
  a.x = x;
  a.xscale = xscale;
  a.n = n;
  a.result = result;
  a.result64 = result_f64;
  return run(t == LIFT_BF16 ? LIFT_OP_ASUM_BF16 : LIFT_OP_ASUM_FP8, variant, a, stream);
}

lift_status lift_dot_ex_v(int variant, lift_dtype t, const void* x, const float* xscale, const void* y,
                          const float* yscale, int64_t n, float* result, double* result_f64,
                          void* stream) {
  if (t == LIFT_F32)
    return lift_dot_v(variant, (const float*)x, (const float*)y, n, result, result_f64, stream);
  lift_status rc = mixed_args(t, x, xscale, n);
  if (rc == LIFT_OK) rc = mixed_args(t, y, yscale, n);
  if (rc != LIFT_OK || !result)
    return set_error(rc != LIFT_OK ? rc : LIFT_ERR_INVALID_ARG, "dot_ex arguments");
  Args a;
  a.x = x;
  a.y = y;
  a.xscale = xscale;
  a.yscale = yscale;
  a.n = n;
  a.result = result;
  a.result64 = result_f64;
  return run(t == LIFT_BF16 ? LIFT_OP_DOT_BF16 : LIFT_OP_DOT_FP8, variant, a, stream);
}

lift_status lift_asum_ex(lift_dtype t, const void* x, const float* xscale, int64_t n, float* result,
                         double* result_f64, void* stream) {
  return lift_asum_ex_v(-1, t, x, xscale, n, result, result_f64, stream);
}
lift_status lift_dot_ex(lift_dtype t, const void* x, const float* xscale, const void* y,
                        const float* yscale, int64_t n, float* result, double* result_f64,
                        void* stream) {
  return lift_dot_ex_v(-1, t, x, xscale, y, yscale, n, result, result_f64, stream);
}

lift_status lift_nrm2_v(int variant, const float* x, int64_t n, float* result, double* result_f64,
                        void* stream) {
  if (bad_n(n) || !result || (n > 0 && !x) || !aligned(x, 4))
    return set_error(LIFT_ERR_INVALID_ARG, "nrm2 arguments");
  Args a;
  a.x = x;
  a.n = n;
  a.result = result;
  a.result64 = result_f64;
  return run(LIFT_OP_NRM2, variant, a, stream);
}

lift_status lift_sum_v(int variant, const float* x, int64_t n, float* result, double* result_f64,
                       void* stream) {
  if (bad_n(n) || !result || (n > 0 && !x) || !aligned(x, 4))
    return set_error(LIFT_ERR_INVALID_ARG, "sum arguments");
  Args a;
  a.x = x;
  a.n = n;
  a.result = result;
  a.result64 = result_f64;
  return run(LIFT_OP_SUM, variant, a, stream);
}

lift_status lift_axpy_v(int variant, int64_t n, float alpha, const float* x, float* y, void* stream) {
  if (bad_n(n) || (n > 0 && (!x || !y))) return set_error(LIFT_ERR_INVALID_ARG, "axpy arguments");
  if (!aligned(x, 4) || !aligned(y, 4)) return set_error(LIFT_ERR_INVALID_ARG, "x/y not 4-byte aligned");
  if (n > 0 && x != y) {
    const char* xb = (const char*)x;
    const char* yb = (const char*)y;
    if (xb < yb + n * 4 && yb < xb + n * 4)
      return set_error(LIFT_ERR_INVALID_ARG, "x and y overlap without being equal");
  }
  if (n == 0) return LIFT_OK;
  Args a;
  a.x = x;
  a.out = y;
  a.n = n;
  a.alpha = alpha;
  return run(LIFT_OP_AXPY, variant, a, stream);
}

lift_status lift_gemv_t_v(int variant, int64_t M, int64_t N, float alpha, const float* A, int64_t lda,
                          const float* x, float beta, float* y, void* stream) {
  if (M < 0 || N < 0 || lda < N || lda < 0) return set_error(LIFT_ERR_INVALID_ARG, "gemv_t sizes");
  if (N > 0 && !y) return set_error(LIFT_ERR_INVALID_ARG, "gemv_t y is NULL");
  if (M > 0 && N > 0 && (!A || !x)) return set_error(LIFT_ERR_INVALID_ARG, "gemv_t A/x is NULL");
  if (!aligned(A, 4) || !aligned(x, 4) || !aligned(y, 4))
    return set_error(LIFT_ERR_INVALID_ARG, "gemv_t pointers not 4-byte aligned");
  if (!current_state()) return set_error(LIFT_ERR_NOT_INITIALIZED, "lift_init was not called for this device");
  if (M == 0) return gemv_t_empty_rows(N, beta, y, static_cast<cudaStream_t>(stream));
  Args a;
  a.A = A;
  a.x = x;
  a.out = y;
  a.M = M;
  a.N = N;
  a.lda = lda;
  a.n = M;
  a.alpha = alpha;
  a.beta = beta;
  return run(LIFT_OP_GEMV_T, variant, a, stream);
}

lift_status lift_gemv_t(int64_t M, int64_t N, float alpha, const float* A, int64_t lda,
                        const float* x, float beta, float* y, void* stream) {
  return lift_gemv_t_v(-1, M, N, alpha, A, lda, x, beta, y, stream);
}

lift_status lift_gemv_t_blocks(int variant, int64_t M, int64_t N, int64_t* rows_per_block,
                               int64_t* blocks) {
  if (variant < 0 || variant >= (int)registry(LIFT_OP_GEMV_T).size() || M < 1 || N < 1 ||
      !rows_per_block || !blocks)
    return set_error(LIFT_ERR_INVALID_ARG, "gemv_t_blocks arguments");
  if (!current_state()) return set_error(LIFT_ERR_NOT_INITIALIZED, "lift_init was not called for this device");
  Args a;
  a.M = M;
  a.N = N;
  gemv_t_shape(variant, a, rows_per_block, blocks);
  return LIFT_OK;
}

lift_status lift_blackscholes_v(int variant, int64_t n, const float* s, float strike, float rate,
                                float volatility, float years, float* call, float* put,
                                void* stream) {
  if (n < 0 || (n > 0 && (!s || !call || !put)))
    return set_error(LIFT_ERR_INVALID_ARG, "blackscholes arrays");
  if (!(strike > 0.f) || !isfinite(strike) || !(volatility > 0.f) || !isfinite(volatility) ||
      !(years > 0.f) || !isfinite(years) || !isfinite(rate))
    return set_error(LIFT_ERR_INVALID_ARG, "blackscholes parameters");
  if (!aligned(s, 4) || !aligned(call, 4) || !aligned(put, 4))
    return set_error(LIFT_ERR_INVALID_ARG, "blackscholes pointers not 4-byte aligned");
  const float params[4] = {strike, rate, volatility, years};
  Args a;
  a.n = n;
  a.x = s;
  a.out = call;
  a.result = put;
  a.xscale = params;      // host block read by the launcher
  return run(LIFT_OP_BLACKSCHOLES, variant, a, stream);
}

lift_status lift_blackscholes(int64_t n, const float* s, float strike, float rate, float volatility,
                              float years, float* call, float* put, void* stream) {
  return lift_blackscholes_v(-1, n, s, strike, rate, volatility, years, call, put, stream);
}

lift_status lift_gemv_segments(int variant, int64_t M, int64_t N, int64_t* seg_len,
                               int64_t* segments) {
  auto& L = registry(LIFT_OP_GEMV);
  if (variant < 0 || variant >= (int)L.size() || M < 1 || N < 0 || !seg_len || !segments)
    return set_error(LIFT_ERR_INVALID_ARG, "gemv_segments arguments");
  if (!current_state()) return set_error(LIFT_ERR_NOT_INITIALIZED, "lift_init was not called for this device");
  if (strncmp(L[variant].info.name, "gemv_split_", 11) != 0) {
    *seg_len = N;
    *segments = 1;
    return LIFT_OK;
  }
  int first = variant;
  while (first > 0 && strncmp(L[first - 1].info.name, "gemv_split_", 11) == 0) --first;
  Args a;
  a.M = M;
  a.N = N;
  gemv_split_shape(variant - first, a, seg_len, segments);
  return LIFT_OK;
}

lift_status lift_nrm2(const float* x, int64_t n, float* result, void* stream) {
  return lift_nrm2_v(-1, x, n, result, nullptr, stream);
}
lift_status lift_sum(const float* x, int64_t n, float* result, void* stream) {
  return lift_sum_v(-1, x, n, result, nullptr, stream);
}
lift_status lift_axpy(int64_t n, float alpha, const float* x, float* y, void* stream) {
  return lift_axpy_v(-1, n, alpha, x, y, stream);
}

int lift_variant_count(int op) {
  if (op < 0 || op >= LIFT_NUM_OPS) return 0;
  return (int)registry(op).size();
}

lift_status lift_variant_describe(int op, int id, lift_variant_info* out) {
  if (op < 0 || op >= LIFT_NUM_OPS || !out) return LIFT_ERR_INVALID_ARG;
  auto& L = registry(op);
  if (id < 0 || id >= (int)L.size()) return LIFT_ERR_INVALID_ARG;
  *out = L[id].info;
  return LIFT_OK;
}

lift_status lift_variant_grid(int op, int id, int64_t n, int64_t* grid) {
  if (op < 0 || op >= LIFT_NUM_OPS || !grid) return LIFT_ERR_INVALID_ARG;
  if (!current_state()) return LIFT_ERR_NOT_INITIALIZED;
  auto& L = registry(op);
  if (id < 0 || id >= (int)L.size()) return LIFT_ERR_INVALID_ARG;
  Args a;
  a.n = n;
  a.M = n;
  a.N = 1;
  *grid = L[id].grid(L[id], a);
  return LIFT_OK;
}

lift_status lift_set_variant(int op, int variant) {
  if (op < 0 || op >= LIFT_NUM_OPS) return LIFT_ERR_INVALID_ARG;
  if (variant < -1 || variant >= (int)registry(op).size()) return LIFT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_policy_mu);
  g_override[op] = variant;
  return LIFT_OK;
}

// Table file: one line per entry "op log2(n+1) log2(M+1) log2(N+1) variant"
// (gemv: n = M*N); '#' starts a comment.
// MLP file: "lift-mlp 2 d_in h1 h2 V", then "offsets K" and K integers (the
// first output of op ids 0 .. K-1; version 1 files have K = 8 without the
// count), then W1 b1 W2 b2 W3 b3 as whitespace-separated floats (W_k
// row-major [d_(k-1)][d_k]).
lift_status lift_set_policy(int policy, const char* path) {
  if (policy == LIFT_POLICY_FIXED) {
    std::lock_guard<std::mutex> lk(g_policy_mu);
    g_policy = policy;
    return LIFT_OK;
  }
  if (!path) return set_error(LIFT_ERR_INVALID_ARG, "policy file path is NULL");
  std::ifstream f(path);
  if (!f) return set_error(LIFT_ERR_INVALID_ARG, std::string("cannot open ") + path);
  if (policy == LIFT_POLICY_TABLE) {
    std::vector<TableEntry> T[LIFT_NUM_OPS];
    std::string line;
    while (std::getline(f, line)) {
      if (line.empty() || line[0] == '#') continue;
      std::istringstream is(line);
      int op, v;
      TableEntry e;
      if (!(is >> op >> e.ln >> e.lm >> e.lN >> v)) continue;
      if (op < 0 || op >= LIFT_NUM_OPS || v < 0 || v >= (int)registry(op).size())
        return set_error(LIFT_ERR_INVALID_ARG, "table entry out of range");
      e.variant = v;
      T[op].push_back(e);
    }
    std::lock_guard<std::mutex> lk(g_policy_mu);
    for (int i = 0; i < LIFT_NUM_OPS; ++i) g_table[i] = T[i];
    g_policy = policy;
    return LIFT_OK;
  }
  if (policy == LIFT_POLICY_MLP || policy == LIFT_POLICY_MLP_TUNE) {
    Mlp m;
    std::string tag, off;
    int ver;
    if (!(f >> tag >> ver >> m.d_in >> m.h1 >> m.h2 >> m.V) || tag != "lift-mlp" || m.d_in < 1 ||
        m.d_in > LIFT_NUM_FEATURES)
      return set_error(LIFT_ERR_INVALID_ARG, "bad MLP header");
    if (!(f >> off) || off != "offsets") return set_error(LIFT_ERR_INVALID_ARG, "bad MLP offsets");
    m.ops = 8;
    if (ver >= 2 && !(f >> m.ops)) return set_error(LIFT_ERR_INVALID_ARG, "bad MLP offsets");
    if (m.ops < 1 || m.ops > LIFT_MLP_OPS) return set_error(LIFT_ERR_INVALID_ARG, "bad MLP op count");
    for (int i = 0; i < m.ops; ++i)
      if (!(f >> m.offsets[i]) || m.offsets[i] < 0 || m.offsets[i] > m.V)
        return set_error(LIFT_ERR_INVALID_ARG, "bad MLP offsets");
    auto rd = [&](std::vector<float>& w, size_t cnt) {
      w.resize(cnt);
      for (size_t i = 0; i < cnt; ++i)
        if (!(f >> w[i])) return false;
      return true;
    };
    if (!rd(m.W1, (size_t)m.d_in * m.h1) || !rd(m.b1, m.h1) || !rd(m.W2, (size_t)m.h1 * m.h2) ||
        !rd(m.b2, m.h2) || !rd(m.W3, (size_t)m.h2 * m.V) || !rd(m.b3, m.V))
      return set_error(LIFT_ERR_INVALID_ARG, "truncated MLP weights");
    // optional: the trained range per op ("box <ops>" then op lo_n hi_n lo_M hi_M lo_N hi_N)
    std::string btag;
    int nb = 0;
    if (f >> btag) {
      if (btag != "box" || !(f >> nb) || nb < 0 || nb > LIFT_NUM_OPS)
        return set_error(LIFT_ERR_INVALID_ARG, "bad MLP box");
      for (int i = 0; i < nb; ++i) {
        int op;
        Box b;
        if (!(f >> op >> b.lo[0] >> b.hi[0] >> b.lo[1] >> b.hi[1] >> b.lo[2] >> b.hi[2]) ||
            op < 0 || op >= LIFT_NUM_OPS)
          return set_error(LIFT_ERR_INVALID_ARG, "bad MLP box");
        b.known = true;
        m.box[op] = b;
      }
    }
    std::lock_guard<std::mutex> lk(g_policy_mu);
    g_mlp = m;
    g_policy = policy;
    g_tuned.clear();
    g_picked.clear();
    ++g_policy_gen;
    return LIFT_OK;
  }
  return set_error(LIFT_ERR_INVALID_ARG, "unknown policy");
}

lift_status lift_tune_stats(int64_t* tuned_shapes, int64_t* timed_launches) {
  std::lock_guard<std::mutex> lk(g_policy_mu);
  if (tuned_shapes) *tuned_shapes = (int64_t)g_tuned.size();
  if (timed_launches) *timed_launches = g_tune_launches.load();
  return LIFT_OK;
}

lift_status lift_pick(int op, int64_t n, int64_t M, int64_t N, int* variant) {
  if (op < 0 || op >= LIFT_NUM_OPS || !variant) return LIFT_ERR_INVALID_ARG;
  if (registry(op).empty()) return LIFT_ERR_UNSUPPORTED;
  Args a;                 // a dense call: lda = N, aligned pointers
  a.n = n;
  a.M = M;
  a.N = N;
  a.lda = N;
  *variant = pick_variant(op, a);
  return LIFT_OK;
}

}  // extern "C"
