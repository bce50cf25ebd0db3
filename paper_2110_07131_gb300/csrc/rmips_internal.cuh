// Internal definitions shared by the librmips translation units.
//
// Index layout in device memory (n users, m items, d dims, sorted positions):
//   Qs     float [n][d]        users in descending-norm order (Algorithm 1)
//   Qh     bf16/fp16 [n][d]    reduced-precision copy for the online filter
//   Ps     float [m][d]        items in descending-norm order
//   unorm  float [n]           ||u|| rounded up (an upper bound of the exact norm)
//   pnorm  float [m]           ||p|| rounded up
//   permQ  int32 [n]           sorted position -> caller's user id
//   permP  int32 [m]           sorted position -> caller's item id
//   Lb     float2 [k_max][n]   (lo, hi): lo <= v_j(u) <= hi, v_j = j-th largest u.p
//                              over P' (hi = +inf when not proven)
//   cand   int32 [n][KC]       item positions whose set provably contains u's
//                              top-k_max (full-P index only)
//   cbnd   float2 [n][KC]      (lo, hi) with lo <= u.p <= hi for each candidate
//                              (float64 dot +- its error bound, rounded outward)
//   incomp uint8 [n]           1 when cand could not be proven complete
//   LB     float [k_max][nb]   block minima of lo (Equation 1)
//   hdr    float [nb]          upper bound of the first user's norm of each block
//   Qtc    [ceil(n/128)]       users in 128-row tiles of the tensor-core operand
//                              layout (K padded to 64 with zeros; TF32 = float32
//                              bits, or the BF16 / FP16 copy), for the batched filter
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <cfloat>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/rmips.h"
#include "ptr_class.h"

#define RMIPS_KC 32              // candidate slots per user (>= k_max + slack)
#define RMIPS_KMAX_LIMIT 28      // largest supported k_max
#define RMIPS_WS_MAXNS 12        // query stages of the batched tensor-core filter at most
#define RMIPS_WS_NMMA 4          // its MMA warps; the query stages are a multiple of this
#define RMIPS_DMAX 128           // largest supported dimension
#define MQ_MAXQ 16384            // queries per multi-query pass (14-bit index)
#define MQ_TQ 64                 // queries per tile
#define MQ_BIG_SLOTS 256         // concurrent large-result emitters (one id bitmap each)
// slots of a pass: the queries, each k-group padded to MQ_TQ, and two spare
// tiles so that a 128-slot read starting in the last tile stays in bounds
#define MQ_SLOTS (MQ_MAXQ + (RMIPS_KMAX_LIMIT + 3) * MQ_TQ)
// items of the tensor-core filter: chunks of up to 128 queries of one k-group
#define MQ_ITEMS (MQ_MAXQ / 128 + RMIPS_KMAX_LIMIT + 1)

#if defined(__CUDACC__)
#define RMIPS_HD __host__ __device__ __forceinline__
#else
#define RMIPS_HD inline
#endif

namespace rmips {

// ---------------------------------------------------------------------------
// Error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);

#define RMIPS_TRY_CUDA(expr)                                                           \
  do {                                                                                 \
    cudaError_t e__ = (expr);                                                          \
    if (e__ != cudaSuccess) {                                                          \
      ::rmips::set_error(std::string(#expr) + ": " + cudaGetErrorString(e__));         \
      return (e__ == cudaErrorMemoryAllocation) ? RMIPS_ERR_OOM : RMIPS_ERR_CUDA;      \
    }                                                                                  \
  } while (0)

// Device status word values (first error wins).  ST_PAIRS_FULL: a batched
// pass found more undecided (user, query) pairs than its list holds; the
// synchronous calls then run the batch again in smaller passes.
enum : int {
  ST_OK = 0, ST_K_RANGE = 2, ST_NONFINITE = 3, ST_CAPACITY = 5, ST_TIMEOUT = 6, ST_INTERNAL = 8, ST_PAIRS_FULL = 9
};

// Largest magnitude a value may have so that its copy in the filter's
// storage format (users of BF16 / FP16 indexes, and every query rounded for
// their filter) stays finite: FP16 65504, BF16 (1 - 2^-8) 2^128.
__host__ __device__ constexpr float filter_max_abs(int precision) {
  return precision == RMIPS_FP16 ? 65504.0f : (precision == RMIPS_BF16 ? 0x1.fep127f : FLT_MAX);
}

// Cycle counters of the tensor-core filter's roles (profiling only).
enum : int {
  WST_LOADER_WAIT = 0, WST_FEEDER_WAIT = 1, WST_MMA_WAIT_B = 2, WST_MMA_WAIT_T = 3, WST_EPI_WAIT = 4,
  WST_LOADER = 5, WST_FEEDER = 6, WST_MMA = 7, WST_EPI = 8, WST_TILES = 9,
  WST_MMA_WAIT_A = 10, WST_EPI_TMEM = 11, WST_ACTIVE = 12, WST_MMA_ISSUE = 13, WST_EPI_SLOW = 14,
  WST_EPI_SLOW_N = 15, WST_EPI_ATOM = 16, WST_N = 17
};

// Per-call device counters (int64 slots).
enum : int {
  C_YES = 0,        // users appended to the yes list
  C_TODO = 1,       // users appended to the todo list
  C_STATUS = 2,     // status word
  C_EXACT = 3,      // exact integer tie decisions
  C_PRUNED = 4,     // blocks pruned by Lemma 3
  C_TESTED = 5,     // users of unpruned blocks
  C_CURSOR = 6,     // running output offset (batches)
  C_YESFAST = 7,    // users decided yes by the O(1) tests
  C_TODOSUM = 8,    // users sent to the todo list (all queries of the call)
  C_NBIG = 9,       // queries of a batch pass with more than EMIT_SORT_CAP results
  C_DONE = 10,      // CTAs finished (one-launch query)
  C_NMID = 11,      // queries of a batch pass with 33 .. MEMIT_MID_CAP results
  C_TILE = 12,      // next user tile of the tensor-core filter (dynamic schedule)
  C_NCOUNTERS = 13
};

// ---------------------------------------------------------------------------
// Query workspace: scratch for one in-flight call.
// ---------------------------------------------------------------------------
struct Workspace {
  int32_t* yes = nullptr;       // [n] sorted positions decided yes
  int32_t* todo = nullptr;      // [n] sorted positions needing recheck / scan
  uint32_t* bitmap = nullptr;   // [n/32 + 1] all-zero between calls
  long long* ctr = nullptr;     // [C_NCOUNTERS] device counters
  long long* h_ctr = nullptr;   // pinned mirror of the counters
  float* dq = nullptr;          // [cap_q][d] staged queries
  int32_t* dk = nullptr;        // [cap_q] staged k
  float* dqn = nullptr;         // [cap_q] query norms rounded up
  float* deps = nullptr;        // [cap_q] absolute error slack per query
  long long* doffs = nullptr;   // [cap_q + 1] device offsets
  long long* h_offs = nullptr;  // [cap_q + 1] pinned offsets
  int64_t cap_q = 0;
  long long* dout = nullptr;    // [cap_out] device staging of result ids
  int64_t cap_out = 0;
  long long* h_out = nullptr;   // [n] pinned, device-mapped result staging
  int64_t cap_hout = 0;
  float* h_q = nullptr;          // [RMIPS_DMAX] pinned, device-mapped query staging
  long long* h_res = nullptr;    // [2 + C_NCOUNTERS] pinned, device-mapped status / count / counters
  long long* dres = nullptr;     // [2 + C_NCOUNTERS] device status / count / counters (asynchronous calls)
  bool ctr_dirty = false;        // counters may be non-zero (multi-kernel paths leave them so)
  // CUDA graphs of the batched pipeline, one (before, after the filter) pair
  // per pass, replayed while the pass's kernel arguments stay the same
  struct PassGraph {
    std::vector<unsigned char> key;   // arguments of the last pass seen
    cudaGraphExec_t pre = nullptr, post = nullptr;
    bool failed = false;              // capture failed for this key: launch directly
  };
  std::vector<PassGraph> pgraph;
  cudaStream_t cap_stream = nullptr;  // capture only (the legacy stream cannot capture)
  cudaEvent_t done_ev = nullptr; // recorded after the work of an asynchronous call
  bool done_pending = false;     // a later user joins done_ev on its own stream first
  cudaStream_t done_stream = nullptr;  // the stream done_ev was recorded on
  std::vector<cudaEvent_t> ev;   // profiling: start/stop pair per filter launch
  int64_t ev_used = 0;
  // batched (multi-query) path
  float* bq = nullptr;           // [MQ_SLOTS][d] queries grouped by k, descending norm
  int32_t* bk = nullptr;         // [MQ_SLOTS] k of each slot
  float* bqn = nullptr;          // [MQ_SLOTS] norm upper bound of each slot
  float* beps = nullptr;         // [MQ_SLOTS] absolute error slack of each slot
  int32_t* bidx = nullptr;       // [MQ_SLOTS] query index of each slot (-1: padding)
  int4* grp = nullptr;           // [RMIPS_KMAX_LIMIT + 1] (k, first slot, size, tiles); .x of the
                                 // last entry after the groups is 0
  int32_t* qcnt = nullptr;       // [MQ_MAXQ] results per query
  int32_t* qcur = nullptr;       // [MQ_MAXQ] scatter cursors
  unsigned long long* ypairs = nullptr;  // (query << 32 | position) decided yes
  int64_t cap_y = 0;
  unsigned long long* tpairs = nullptr;  // (query << 32 | position) to resolve
  int64_t cap_t = 0;
  int32_t* seg = nullptr;        // [cap_y] positions grouped by query
  unsigned long long* keys = nullptr;  // [MQ_MAXQ] query sort keys
  unsigned long long* runs = nullptr;  // [MQ_MAXQ] keys sorted in runs of 1024
  int* gfirst = nullptr;         // [RMIPS_KMAX_LIMIT + 2] first sorted position of each k
  int* gslot0 = nullptr;         // [RMIPS_KMAX_LIMIT + 2] first slot of each k-group
  int* hist = nullptr;           // [RMIPS_KMAX_LIMIT + 2] queries per k
  long long* dseglo = nullptr;   // [cap_seg] per-query id ranges of a batch
  long long* dseghi = nullptr;
  int64_t cap_seg = 0;
  float2* bcq = nullptr;         // [MQ_SLOTS] (error scale, absolute slack) of each slot
  unsigned char* bitems = nullptr;  // [MQ_ITEMS] packed items of the tensor-core filter
  int* gitem = nullptr;          // [RMIPS_KMAX_LIMIT + 2] first item of each k-group; [.. + 1] = items
  int2* itemg = nullptr;         // [MQ_ITEMS] (group, chunk) of each item
  int32_t* gpre = nullptr;       // [nb][k_max] Lemma 3 prefix of every (block, k-group)
  unsigned long long* wst = nullptr;  // [WST_N] role wait / busy cycles of the TC filter (profiling)
  int64_t cap_gpre = 0;
  int32_t* big = nullptr;        // [MQ_MAXQ] queries of a pass with large results
  int32_t* mid = nullptr;        // [MQ_MAXQ] queries of a pass with medium results
  int32_t* bslot = nullptr;      // [MQ_MAXQ] id-bitmap slot of a query with a large result, else -1
  int* bigcnt = nullptr;         // [MQ_BIG_SLOTS][chunks] ids per 1024-word chunk of a large result
  uint32_t* bigmaps = nullptr;   // [MQ_BIG_SLOTS][n/32 + 1] all-zero between uses
};

}  // namespace rmips

struct rmips_index {
  int64_t n = 0, m = 0;
  int d = 0, k_max = 0, bs = 32, precision = RMIPS_FP32;
  int64_t nb = 0, pp = 0;
  int full_p = 1;
  int batch_tc = 1;             // batched filter on tensor cores (TF32) when eligible
  int no_blocks = 0;            // Lemma 3 switched off (block bounds at -inf), for the ablation
  int device = 0;
  int64_t incomplete = 0;
  int64_t device_bytes = 0;
  double build_ms = 0.0;
  float pn0 = 0.f;              // largest item norm (rounded up)
  // launch choices of the autotuner (0: as many stages as fit in shared memory)
  int tune_ws_ns = 0;           // query stages of the batched tensor-core filter (even)
  int tune_q1_ns = 0;           // row stages of the one-launch single-query kernel
  int tuned = 0;                // 0 not tuned, 1 searched on the device, 2 read from a tune cache
  int build_kind = -1;          // operand kind of the tensor-core candidate selection (-1: CUDA cores)
  double tune_ms = 0.0;

  float* Qs = nullptr;
  void* Qh = nullptr;
  float* Ps = nullptr;
  float* unorm = nullptr;
  float* pnorm = nullptr;
  int32_t* permQ = nullptr;
  int32_t* permP = nullptr;
  float2* Lb = nullptr;
  int32_t* cand = nullptr;
  float2* cbnd = nullptr;
  uint8_t* incomp = nullptr;
  float* LB = nullptr;
  float* hdr = nullptr;
  unsigned char* Qtc = nullptr;  // user tiles of the batched tensor-core filter (null: not built)

  std::mutex mu;
  std::vector<rmips::Workspace*> pool;       // idle workspaces (their queued device work may still run)
  int n_ws = 0;                              // workspaces created for this index
  rmips_query_stats last_stats{};
  int prof_on = 0;
  rmips_profile prof{};
  std::vector<cudaEvent_t> pend_ev;          // filter event pairs of asynchronous calls, read on profile read
  unsigned long long* dprof = nullptr;       // [1] kept pairs of asynchronous calls (device)
  unsigned long long* dprof1 = nullptr;      // [4] asynchronous single queries: tested users, listed users,
                                             // pruned chunks, launches (device)
  std::vector<cudaEvent_t> pend_ev1;         // their filter event pairs
};

namespace rmips {

// Allocation helpers (tracked in idx->device_bytes).
template <class T>
cudaError_t dalloc(rmips_index* idx, T** p, size_t count) {
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e == cudaSuccess && idx) idx->device_bytes += (int64_t)bytes;
  return e;
}

bool is_device_ptr(const void* p);
// PTR_HOST, PTR_DEVICE (memory of `device`, or managed) or PTR_OTHER_DEVICE.
int ptr_class(const void* p, int device);
// RMIPS_ERR_ARG (with a message naming `what`) when p is device memory of a
// GPU other than `device`; RMIPS_OK otherwise (also for a null p).
rmips_status check_ptr_device(const void* p, int device, const char* what);

Workspace* acquire_workspace(rmips_index* idx, rmips_status* st);
// Batched run on a workspace whose ws->dq / ws->dk (and ws->dseglo/dseghi)
// already hold nq staged queries; results to `out` (device-visible),
// offsets to ws->doffs.  Asynchronous on `st`.
rmips_status batch_reserve(rmips_index* idx, Workspace* ws, int64_t nq);
rmips_status batch_launch(rmips_index* idx, Workspace* ws, int64_t nq, long long* out, long long capacity,
                          cudaStream_t st, bool with_segments);
rmips_status device_status(long long s);
// One query through the one-launch kernel (full-P index) on a workspace:
// device q, results to out (capacity ids), (status, count) to done.
rmips_status single_launch(rmips_index* idx, Workspace* ws, const float* q, int k, long long seg_lo,
                           long long seg_hi, long long* out, long long capacity, long long* done, cudaStream_t st);
void release_workspace(rmips_index* idx, Workspace* ws);
// Loads the module that holds rmips_query_noalloc's scratch array on the
// current device (called when an index is built or loaded).
rmips_status noalloc_prepare();
// Block arrays (Equation 1) for another block size, from the index's bounds.
rmips_status set_block_size(rmips_index* idx, int bs, cudaStream_t st);
// Autotuner timing hooks: milliseconds per run of the batched path on nq
// device-resident queries, and per one-launch single query.
rmips_status tune_time_batch(rmips_index* idx, const float* dq, const int32_t* dk, int64_t nq, int reps,
                             cudaStream_t st, float* ms);
rmips_status tune_time_single(rmips_index* idx, const float* dq, int64_t nq, int k, cudaStream_t st, float* ms);
// Largest number of query stages the batched tensor-core filter can use.
int max_batch_stages(const rmips_index* idx);
// Largest number of row stages the single-query kernel can use.
int max_single_stages(const rmips_index* idx);
// The autotuner: reads the choices from `cache` (may be NULL) or searches
// them on the device and appends them to `cache`.
rmips_status tune_index(rmips_index* idx, const char* cache, cudaStream_t st);
// Orders this stream after the last asynchronous call that used ws.
rmips_status ws_join(Workspace* ws, cudaStream_t st);
void destroy_workspace(Workspace* ws);

// ---------------------------------------------------------------------------
// Exact sign of u.a - u.b on float32 inputs.
//
// Every float32 is m * 2^e with an integer |m| < 2^24 and e in [-149, 104], so
// every product u_i a_i is an integer < 2^48 times 2^(e1 + e2), with
// e1 + e2 in [-298, 208].  The products are added into a fixed-point integer
// with its least significant bit at 2^-298, held as nine signed 128-bit limbs
// of 64-bit weight each; a limb receives at most 2d terms below 2^111, so no
// limb can overflow for d <= 256.  Carries are propagated once at the end and
// the sign is read off the top limb.  The result is exact: no rounding occurs.
// ---------------------------------------------------------------------------
RMIPS_HD void exact_acc_add(__int128* acc, float x, float y, bool negate) {
  uint32_t bx, by;
  memcpy(&bx, &x, 4);
  memcpy(&by, &y, 4);
  uint32_t ex = (bx >> 23) & 0xffu, ey = (by >> 23) & 0xffu;
  uint64_t mx = bx & 0x7fffffu, my = by & 0x7fffffu;
  if (ex) mx |= 0x800000u; else ex = 1;      // subnormal: m * 2^(1 - 150)
  if (ey) my |= 0x800000u; else ey = 1;
  if (mx == 0 || my == 0) return;
  uint64_t mag = mx * my;                    // < 2^48
  bool neg = (((bx ^ by) >> 31) != 0) != negate;
  int pos = (int)(ex + ey) - 2;              // exponent + 298, in [0, 506]
  int limb = pos >> 6, off = pos & 63;
  __int128 t = ((__int128)mag) << off;
  acc[limb] += neg ? -t : t;
}

RMIPS_HD int exact_acc_sign(__int128* acc) {
  const __int128 base = ((__int128)1) << 64;
  for (int i = 0; i < 8; ++i) {
    __int128 carry = acc[i] >> 64;           // floor division by 2^64
    acc[i] -= carry * base;                  // now 0 <= acc[i] < 2^64
    acc[i + 1] += carry;
  }
  if (acc[8] > 0) return 1;
  if (acc[8] < 0) return -1;
  for (int i = 7; i >= 0; --i)
    if (acc[i] != 0) return 1;
  return 0;
}

RMIPS_HD int exact_sign_diff(const float* u, const float* a, const float* b, int d) {
  __int128 acc[9];
  for (int i = 0; i < 9; ++i) acc[i] = 0;
  for (int i = 0; i < d; ++i) {
    exact_acc_add(acc, u[i], a[i], false);
    exact_acc_add(acc, u[i], b[i], true);
  }
  return exact_acc_sign(acc);
}

#if defined(__CUDACC__)
// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(long long* ctr, int st) {
  atomicCAS((unsigned long long*)&ctr[C_STATUS], 0ull, (unsigned long long)st);
}

// Sign of u.a - u.b: float64 when the difference clears its rounding bound
// (each float32 product is exact in float64; the sums carry at most
// gamma_d * sum|u_i x_i| error), else the exact integer accumulator.
__device__ __forceinline__ int cmp_dot(const float* __restrict__ u, const float* __restrict__ a,
                                       const float* __restrict__ b, int d, long long* ctr) {
  double sa = 0.0, sb = 0.0, aa = 0.0, ab = 0.0;
  for (int i = 0; i < d; ++i) {
    double ui = (double)u[i], ai = (double)a[i], bi = (double)b[i];
    sa = fma(ui, ai, sa);
    sb = fma(ui, bi, sb);
    aa = fma(fabs(ui), fabs(ai), aa);
    ab = fma(fabs(ui), fabs(bi), ab);
  }
  double diff = sa - sb;
  double bound = (4.0 * (d + 2) * 0x1p-53) * (aa + ab);
  if (diff > bound) return 1;
  if (diff < -bound) return -1;
  bool same = true;                                  // bit-identical vectors tie exactly
  for (int i = 0; i < d; ++i) same = same && (__float_as_uint(a[i]) == __float_as_uint(b[i]));
  if (same) return 0;
  if (ctr) atomicAdd((unsigned long long*)&ctr[C_EXACT], 1ull);
  return exact_sign_diff(u, a, b, d);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_cnt(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// 1-D bulk copy global -> shared (TMA engine), completion signalled on `bar`.
// dst, src 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after ~2^31 SM clocks (about
// one second) and reports false so the caller can flag a timeout and return.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1ll << 31)) return false;
  }
  return true;
}

template <class T>
__device__ __forceinline__ float to_f32(T x);
template <>
__device__ __forceinline__ float to_f32<float>(float x) { return x; }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <>
__device__ __forceinline__ float to_f32<__half>(__half x) { return __half2float(x); }
#endif  // __CUDACC__

}  // namespace rmips
