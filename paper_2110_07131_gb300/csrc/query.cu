// Online phase: Algorithm 3 ("Simpfer", Section 4.3) on the GPU.
//
// Per query q (with k):
//   k_qprep    ||q|| (float64, rounded up), finiteness check, error slack;
//   k_filter   Lemma 3 per block (prune iff ||u_first|| ||q|| < L^k(B)), then
//              for every user of a surviving block u.q with a rigorous error
//              bound e:  no  if u.q + e < lo_k(u)              (Lemma 1),
//                        yes if u.q - e >= hi_k(u)             (full-P index)
//                        yes if u.q - e >= ||u|| ||p_k||       (Lemma 2, P' index),
//              anything else goes to the todo list.  User rows are staged
//              32 at a time into shared memory by the TMA engine
//              (cp.async.bulk), double-buffered per warp;
//   k_resolve  todo users: exact count over the user's proven candidate list
//              (full-P index), else Algorithm 2 -- a norm-ordered scan of P
//              with Corollary 1 (stop once ||u|| ||p_j|| <= u.q) and
//              Corollary 2 (stop once k items are strictly above u.q);
//              comparisons within their rounding bound are decided exactly;
//   k_emit     sorted positions -> caller ids, optional segment filter,
//              ascending order, capacity check, CSR offsets.
#include <climits>
#include <cmath>
#include <cstdlib>

#include "rmips_internal.cuh"
#include "tc_common.cuh"

namespace rmips {
namespace {

constexpr float kInf = __builtin_huge_valf();
constexpr unsigned FULL = 0xffffffffu;
constexpr int FW = 4;                      // warps per filter CTA
constexpr int EMIT_THREADS = 1024;
constexpr int EMIT_SORT_CAP = 8192;       // single query: larger results use the id bitmap
constexpr int MEMIT_MID_CAP = 2048;       // batch: larger results use id bitmaps spread over the grid

// Relative error factor of a length-d float32 dot product whose inputs were
// rounded to a format with unit roundoff u_in (0 for float32 inputs):
// |fl(sum x_i q_i) - sum u_i q_i| <= (u_in + gamma_d (1 + u_in)) sum |u_i q_i|,
// gamma_d = d 2^-24 / (1 - d 2^-24); the computed sum |x_i q_i| is itself
// within (1 + u_in)(1 + gamma_d) of the exact one.  (d + 4) 2^-24 covers
// gamma_d and its own rounding for d <= 256.
inline float err_factor(int d, int precision) {
  double u_in = precision == RMIPS_BF16 ? 0x1p-8 : precision == RMIPS_FP16 ? 0x1p-11 : 0.0;
  double g = (d + 4) * 0x1p-24;
  double f = (u_in + g * (1.0 + u_in)) / (1.0 - u_in - g) * (1.0 + 0x1p-20);
  return (float)f;
}

struct Common {
  const float* Qs;
  const void* Qrows;           // Qs (float32) or the reduced-precision copy
  const float* Ps;
  const float2* Lb;
  const float* LB;
  const float* hdr;
  const float* unorm;
  const float* pnorm;
  const int32_t* cand;
  const float2* cbnd;
  const uint8_t* incomp;
  const int32_t* permQ;
  int64_t n, m, nb;
  int d, bs, k_max, full_p;
  float cg;                    // relative error factor of the filter dot product
  float cg32;                  // same for float32 inputs (verification)
  // query staging
  const float* dq;
  const int32_t* dk;
  float* dqn;
  float* deps;
  // workspace
  int32_t* yes;
  int32_t* todo;
  long long* ctr;
};

// Upper bound of ||q|| (float32, every step rounded up, so no float64 chain)
// and the absolute slack of the filter's error bound: float32 products below
// the normal range lose up to 2^-150 each, FP16 storage rounds values below
// 2^-14 with absolute error up to 2^-25 (BF16 below 2^-126: 2^-134).
__device__ __forceinline__ bool query_bounds(const float* q, int d, int precision, float* qn, float* eps) {
  float acc = 0.f, qmax = 0.f;
  bool fin = true;
  const float vmax = filter_max_abs(precision);
  for (int i = 0; i < d; ++i) {
    const float v = q[i];
    fin = fin && isfinite(v) && !(fabsf(v) > vmax);
    acc = __fmaf_ru(v, v, acc);
    qmax = fmaxf(qmax, fabsf(v));
  }
  *qn = __fsqrt_ru(acc);
  const float sub = (precision == RMIPS_FP16) ? 0x1p-25f : (precision == RMIPS_BF16 ? 0x1p-133f : 0.f);
  *eps = __fmul_ru((float)(d + 2), __fmaf_ru(sub, qmax, 0x1p-148f));
  return fin;
}

// --- query preparation ---------------------------------------------------------------
__global__ void k_qprep(Common c, int64_t nq, int precision) {
  const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= nq) return;
  const float* q = c.dq + j * c.d;
  if (lane == 0) {
    float qn, eps;
    const bool fin = query_bounds(q, c.d, precision, &qn, &eps);
    const int k = c.dk[j];
    if (!fin) atomicCAS((unsigned long long*)&c.ctr[C_STATUS], 0ull, (unsigned long long)ST_NONFINITE);
    if (k < 1 || k > c.k_max) atomicCAS((unsigned long long*)&c.ctr[C_STATUS], 0ull, (unsigned long long)ST_K_RANGE);
    c.dqn[j] = qn;
    c.deps[j] = eps;
  }
}

__device__ bool verify_scan(const float* __restrict__ u, float un, const Common& c, const float* sq, int k,
                            float qeps);
__device__ bool recheck_candidates(const float* __restrict__ u, const float* q, const int32_t* __restrict__ crow,
                                   const float2* __restrict__ cbrow, const float* __restrict__ Ps, int d, int k,
                                   float cg32, long long* ctr);

// --- filter ------------------------------------------------------------------------
// Lemmas 1-3 for one query over this CTA's share of 32-user chunks.  Warp w
// of the grid owns chunks w, w + W, w + 2W, ... (W = warps in the grid); it
// tests Lemma 3 for 32 of its chunks at once (one lane each), then streams
// the surviving chunks' rows into shared memory with 1-D TMA bulk copies,
// double-buffered, and tests every user.  Returns false if a TMA wait gave up.
template <class T, bool FULLP, bool INLINE = false>
__device__ bool filter_chunks(const Common& c, const float* sq, int k, float qn, float qeps, uint64_t* bars,
                              unsigned char* bufs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d = c.d;
  const int64_t n = c.n;
  const float pk = (k <= c.m) ? c.pnorm[k - 1] : -kInf;
  const uint32_t chunk_bytes = 32u * d * (uint32_t)sizeof(T);        // multiple of 16
  unsigned char* mybuf = bufs + (size_t)warp * 2 * chunk_bytes;
  const int64_t nchunks = (n + 31) / 32;
  const int nwarp = blockDim.x >> 5;
  const int64_t W = (int64_t)gridDim.x * nwarp;
  const int64_t w0 = (int64_t)blockIdx.x * nwarp + warp;
  const float* LBk = c.LB + (int64_t)(k - 1) * c.nb;
  const float2* Lbk = c.Lb + (int64_t)(k - 1) * n;

  int64_t gbase = 0;       // next group of 32 slots of this warp's chunk sequence
  int64_t gcur = 0;        // base of the group the mask belongs to
  uint32_t mask = 0;
  long long pruned = 0, tested = 0, yesfast = 0, todosum = 0;
  auto next_chunk = [&]() -> int64_t {
    while (mask == 0) {
      if (w0 + gbase * W >= nchunks) return -1;
      const int64_t ch = w0 + (gbase + lane) * W;
      bool ok = false;
      if (ch < nchunks) {
        const int64_t blk = (ch * 32) / c.bs;
        ok = !(__fmul_ru(c.hdr[blk], qn) < LBk[blk]);   // Lemma 3, strict
      }
      mask = __ballot_sync(FULL, ok);
      pruned += __popc(__ballot_sync(FULL, ch < nchunks && !ok));
      gcur = gbase;
      gbase += 32;
    }
    const int bit = __ffs(mask) - 1;
    mask &= mask - 1;
    return w0 + (gcur + bit) * W;
  };
  auto issue = [&](int64_t ch, int s) {
    if (lane == 0) {
      const int64_t rows = (n - ch * 32) < 32 ? (n - ch * 32) : 32;
      const uint32_t bytes = ((uint32_t)(rows * d * sizeof(T)) + 15u) & ~15u;
      fence_proxy_async();
      mbar_arrive_expect_tx(&bars[warp * 2 + s], bytes);
      bulk_g2s(mybuf + (size_t)s * chunk_bytes,
               reinterpret_cast<const unsigned char*>(c.Qrows) + (size_t)ch * chunk_bytes, bytes,
               &bars[warp * 2 + s]);
    }
  };

  uint32_t phase = 0;      // bit s = parity to wait for on buffer s
  int s = 0;
  bool good = true;
  int64_t cur = next_chunk();
  if (cur >= 0) issue(cur, 0);
  while (cur >= 0) {
    const int64_t nxt = next_chunk();
    if (nxt >= 0) issue(nxt, s ^ 1);
    const int64_t pos = cur * 32 + lane;
    const bool valid = pos < n;
    const float2 L = valid ? Lbk[pos] : make_float2(kInf, kInf);
    const float un = (!FULLP && valid) ? c.unorm[pos] : 0.f;
    bool ok = mbar_wait_bounded(&bars[warp * 2 + s], (phase >> s) & 1u);
    ok = __all_sync(FULL, ok);
    if (!ok) {
      set_status(c.ctr, ST_TIMEOUT);
      if (nxt >= 0) mbar_wait_bounded(&bars[warp * 2 + (s ^ 1)], (phase >> (s ^ 1)) & 1u);
      good = false;
      break;
    }
    phase ^= 1u << s;
    const T* row = reinterpret_cast<const T*>(mybuf + (size_t)s * chunk_bytes) + (size_t)lane * d;
    float g = 0.f, A = 0.f;
    int r = lane % d;                       // rotated start: lanes hit different banks
    for (int i = 0; i < d; ++i) {
      const float uv = to_f32<T>(row[r]);
      const float qv = sq[r];
      g = fmaf(uv, qv, g);
      A = fmaf(fabsf(uv), fabsf(qv), A);
      r = (r + 1 == d) ? 0 : r + 1;
    }
    __syncwarp();
    bool yes = false, todo = false;
    if (valid) {
      const float e = __fmaf_ru(A, c.cg, qeps);
      const float hi = __fadd_ru(g, e), lo = __fsub_rd(g, e);
      const bool no = hi < L.x;                                   // Lemma 1 (strict)
      if (!no) {
        yes = FULLP ? (lo >= L.y) : (lo >= __fmul_ru(un, pk));    // hi_k, or Lemma 2
        todo = !yes;
      }
    }
    uint32_t by = __ballot_sync(FULL, yes), bt = __ballot_sync(FULL, todo);
    const uint32_t lt = (1u << lane) - 1u;
    if (INLINE && bt) {
      // exact recheck right here, one user at a time, the warp's lanes on its candidates
      todosum += __popc(bt);
      for (uint32_t m = bt; m; m &= m - 1) {
        const int l = __ffs(m) - 1;
        const int64_t p = cur * 32 + l;
        const float* u = c.Qs + p * c.d;
        const bool ok_yes = !c.incomp[p]
                                ? recheck_candidates(u, sq, c.cand + p * RMIPS_KC, c.cbnd + p * RMIPS_KC, c.Ps, c.d,
                                                     k, c.cg32, c.ctr)
                                : verify_scan(u, c.unorm[p], c, sq, k, qeps);
        if (ok_yes && lane == l) yes = true;
      }
      by = __ballot_sync(FULL, yes);
      bt = 0;
    }
    if (by) {
      long long base = 0;
      if (lane == 0) base = atomicAdd((unsigned long long*)&c.ctr[C_YES], (unsigned long long)__popc(by));
      base = __shfl_sync(FULL, base, 0);
      if (yes) c.yes[base + __popc(by & lt)] = (int32_t)pos;
    }
    if (bt) {
      long long base = 0;
      if (lane == 0) base = atomicAdd((unsigned long long*)&c.ctr[C_TODO], (unsigned long long)__popc(bt));
      base = __shfl_sync(FULL, base, 0);
      if (todo) c.todo[base + __popc(bt & lt)] = (int32_t)pos;
    }
    tested += __popc(__ballot_sync(FULL, valid));
    yesfast += INLINE ? 0 : __popc(by);
    todosum += __popc(bt);
    cur = nxt;
    s ^= 1;
  }
  if (lane == 0) {
    if (pruned) atomicAdd((unsigned long long*)&c.ctr[C_PRUNED], (unsigned long long)pruned);
    if (tested) atomicAdd((unsigned long long*)&c.ctr[C_TESTED], (unsigned long long)tested);
    if (yesfast) atomicAdd((unsigned long long*)&c.ctr[C_YESFAST], (unsigned long long)yesfast);
    if (todosum) atomicAdd((unsigned long long*)&c.ctr[C_TODOSUM], (unsigned long long)todosum);
  }
  return good;
}

__device__ __forceinline__ void init_filter_barriers(uint64_t* bars) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    mbar_init(&bars[warp * 2 + 0], 1);
    mbar_init(&bars[warp * 2 + 1], 1);
    fence_mbar_init();
  }
}

template <class T, bool FULLP>
__global__ void __launch_bounds__(FW * 32) k_filter(Common c, int j) {
  extern __shared__ __align__(128) unsigned char smem[];
  float* sq = reinterpret_cast<float*>(smem);                        // [RMIPS_DMAX]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 512);          // [FW][2]
  unsigned char* bufs = smem + 512 + FW * 2 * 8;
  __shared__ int s_skip;
  if (threadIdx.x == 0) {
    const long long st0 = c.ctr[C_STATUS];
    s_skip = (st0 != 0 && st0 != ST_CAPACITY);                    // bad input: nothing to do
  }
  __syncthreads();
  if (s_skip) return;                                               // uniform across the CTA
  const int k = c.dk[j];
  const float* q = c.dq + (int64_t)j * c.d;
  for (int i = threadIdx.x; i < c.d; i += blockDim.x) sq[i] = q[i];
  init_filter_barriers(bars);
  __syncthreads();
  filter_chunks<T, FULLP>(c, sq, k, c.dqn[j], c.deps[j], bars, bufs);
}

// --- Algorithm 2 for one user, one warp ----------------------------------------------
__device__ bool verify_scan(const float* __restrict__ u, float un, const Common& c, const float* sq, int k,
                            float qeps) {
  const int lane = threadIdx.x & 31;
  const int d = c.d;
  float g = 0.f, A = 0.f;
  for (int i = 0; i < d; ++i) {
    g = fmaf(u[i], sq[i], g);
    A = fmaf(fabsf(u[i]), fabsf(sq[i]), A);
  }
  const float tiny = (d + 2) * 0x1p-148f;
  const float e = __fmaf_ru(A, c.cg32, qeps);
  const float gl = __fsub_rd(g, e), gh = __fadd_ru(g, e);
  int above = 0;
  for (int64_t j0 = 0; j0 < c.m; j0 += 32) {
    if (__fmul_ru(un, c.pnorm[j0]) <= gl) break;                 // Corollary 1
    const int64_t jj = j0 + lane;
    bool gt = false;
    if (jj < c.m && __fmul_ru(un, c.pnorm[jj]) > gl) {
      const float* p = c.Ps + jj * d;
      float sp = 0.f, B = 0.f;
      for (int i = 0; i < d; ++i) {
        sp = fmaf(u[i], p[i], sp);
        B = fmaf(fabsf(u[i]), fabsf(p[i]), B);
      }
      const float ep = __fmaf_ru(B, c.cg32, tiny);
      if (__fsub_rd(sp, ep) > gh) gt = true;
      else if (__fadd_ru(sp, ep) < gl) gt = false;
      else gt = cmp_dot(u, p, sq, d, c.ctr) > 0;
    }
    above += __popc(__ballot_sync(FULL, gt));
    if (above >= k) return false;                                 // Corollary 2
  }
  return true;
}


// Exact recheck of one user against its proven candidate list (one warp, one
// candidate per lane): u is a yes iff fewer than k candidates p have
// u.p > u.q.  Each comparison is taken at the cheapest level that decides it:
// float32 with its rounding bound, then "p is bit-identical to q" (an exact
// tie, q's own copy in P), then float64 with its bound, then the exact
// integer accumulator.  u.q is formed once per user, split across lanes.
__device__ bool recheck_candidates(const float* __restrict__ u, const float* q, const int32_t* __restrict__ crow,
                                   const float2* __restrict__ cbrow, const float* __restrict__ Ps, int d, int k,
                                   float cg32, long long* ctr) {
  const int lane = threadIdx.x & 31;
  float g32 = 0.f, a32 = 0.f;
  for (int i = lane; i < d; i += 32) {
    const float x = u[i], y = q[i];
    g32 = fmaf(x, y, g32);
    a32 = fmaf(fabsf(x), fabsf(y), a32);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    g32 += __shfl_xor_sync(FULL, g32, o);
    a32 += __shfl_xor_sync(FULL, a32, o);
  }
  const float tiny = (d + 2) * 0x1p-148f;
  const float eg = __fmaf_ru(a32, cg32, tiny);
  const float gl = __fsub_rd(g32, eg), gh = __fadd_ru(g32, eg);
  const int32_t it = crow[lane];
  bool gt = false, hard = false;
  // the index keeps an interval of every candidate's u.p: disjoint from that
  // of u.q it decides at once; only overlapping candidates read their row
  const float2 cb = it >= 0 ? cbrow[lane] : make_float2(-kInf, -kInf);
  if (it >= 0 && cb.x > gh) {
    gt = true;
  } else if (it >= 0 && !(cb.y < gl)) {
    const float* p = Ps + (int64_t)it * d;
    float sp = 0.f, B = 0.f;
    for (int i = 0; i < d; ++i) {
      sp = fmaf(u[i], p[i], sp);
      B = fmaf(fabsf(u[i]), fabsf(p[i]), B);
    }
    const float ep = __fmaf_ru(B, cg32, tiny);
    if (__fsub_rd(sp, ep) > gh) {
      gt = true;
    } else if (!(__fadd_ru(sp, ep) < gl)) {
      bool same = true;
      for (int i = 0; i < d; ++i) same = same && (__float_as_uint(p[i]) == __float_as_uint(q[i]));
      hard = !same;
    }
  }
  if (__any_sync(FULL, hard)) {
    // float64 u.q, formed once for the warp, only when some candidate needs it
    double g64 = 0.0, a64 = 0.0;
    for (int i = lane; i < d; i += 32) {
      const double x = (double)u[i], y = (double)q[i];
      g64 = fma(x, y, g64);
      a64 = fma(fabs(x), fabs(y), a64);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      g64 += __shfl_xor_sync(FULL, g64, o);
      a64 += __shfl_xor_sync(FULL, a64, o);
    }
    if (hard) {
      const float* p = Ps + (int64_t)it * d;
      double s64 = 0.0, b64 = 0.0;
      for (int i = 0; i < d; ++i) {
        s64 = fma((double)u[i], (double)p[i], s64);
        b64 = fma(fabs((double)u[i]), fabs((double)p[i]), b64);
      }
      const double diff = s64 - g64;
      const double bound = (4.0 * (d + 2) * 0x1p-53) * (b64 + a64);
      if (diff > bound) gt = true;
      else if (!(diff < -bound)) {
        if (ctr) atomicAdd((unsigned long long*)&ctr[C_EXACT], 1ull);
        gt = exact_sign_diff(u, p, q, d) > 0;
      }
    }
  }
  return __popc(__ballot_sync(FULL, gt)) < k;
}

// --- resolve the todo list ------------------------------------------------------------
__global__ void __launch_bounds__(256) k_resolve(Common c, int j) {
  __shared__ float sq[RMIPS_DMAX];
  __shared__ int s_skip;
  __shared__ long long s_cnt;
  const int d = c.d;
  for (int i = threadIdx.x; i < d; i += blockDim.x) sq[i] = c.dq[(int64_t)j * d + i];
  if (threadIdx.x == 0) {
    const long long st0 = c.ctr[C_STATUS];
    s_skip = (st0 != 0 && st0 != ST_CAPACITY);
    s_cnt = c.ctr[C_TODO];
  }
  __syncthreads();
  if (s_skip) return;                                               // uniform across the CTA
  const long long cnt = s_cnt;
  const int k = c.dk[j];
  const float qeps = c.deps[j];
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < cnt; t += nw) {
    const int32_t pos = c.todo[t];
    const float* u = c.Qs + (int64_t)pos * d;
    bool yes;
    if (c.full_p && !c.incomp[pos]) {
      // The candidate list holds every item that can reach u's k_max-th place,
      // so u is a yes iff fewer than k candidates are strictly above u.q.
      yes = recheck_candidates(u, sq, c.cand + (int64_t)pos * RMIPS_KC, c.cbnd + (int64_t)pos * RMIPS_KC, c.Ps, d, k,
                                 c.cg32, c.ctr);
    } else {
      yes = verify_scan(u, c.unorm[pos], c, sq, k, qeps);
    }
    if (lane == 0 && yes) {
      long long b = atomicAdd((unsigned long long*)&c.ctr[C_YES], 1ull);
      c.yes[b] = pos;
    }
  }
}

// --- emit ----------------------------------------------------------------------------
struct EmitArgs {
  const uint32_t* segmask;     // optional allowed-id bitmap (nullptr = all)
  int64_t seg_lo, seg_hi;      // allowed id range
  uint32_t* bitmap;            // [n/32 + 1] zero on entry and exit
  long long* out;              // result ids
  long long capacity;
  long long* offs;             // offsets (device-visible; entry j+1 written)
};

__device__ __forceinline__ bool seg_ok(const EmitArgs& e, int32_t id) {
  if (id < e.seg_lo || id >= e.seg_hi) return false;
  if (e.segmask && !((e.segmask[id >> 5] >> (id & 31)) & 1u)) return false;
  return true;
}

// Block-wide emit (any block size that is a multiple of 32): the cnt listed
// positions -> caller ids, segment filter, ascending order, written at
// e.out[base ..] when they fit in e.capacity.  keys: EMIT_SORT_CAP ints of
// shared memory; s_warp: 32 ints.  Returns the number of ids.
__device__ long long emit_block(const Common& c, const EmitArgs& e, long long cnt, long long base,
                                int32_t* keys, int* s_warp, long long* s_total) {
  const int tid = threadIdx.x, nt = blockDim.x, nwarp = nt >> 5;
  long long total = 0;
  if (cnt <= EMIT_SORT_CAP) {
    int N2 = 1;
    while (N2 < cnt) N2 <<= 1;
    for (int i = tid; i < N2; i += nt) {
      int32_t id = INT_MAX;
      if (i < cnt) {
        int32_t v = c.permQ[__ldcg(&c.yes[i])];
        if (seg_ok(e, v)) id = v;
      }
      keys[i] = id;
    }
    __syncthreads();
    for (int kk = 2; kk <= N2; kk <<= 1) {
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
        for (int t = tid; t < (N2 >> 1); t += nt) {
          const int i = 2 * t - (t & (jj - 1)), p = i + jj;
          const int32_t a = keys[i], b = keys[p];
          if ((a > b) == ((i & kk) == 0)) { keys[i] = b; keys[p] = a; }
        }
        __syncthreads();
      }
    }
    if (tid == 0) {
      int lo = 0, hi = N2;                 // first INT_MAX
      while (lo < hi) { int mid = (lo + hi) >> 1; if (keys[mid] == INT_MAX) hi = mid; else lo = mid + 1; }
      *s_total = lo;
    }
    __syncthreads();
    total = *s_total;
    if (base + total <= e.capacity) {
      for (int i = tid; i < total; i += nt) e.out[base + i] = keys[i];
    }
  } else {
    for (long long i = tid; i < cnt; i += nt) {
      int32_t v = c.permQ[__ldcg(&c.yes[i])];
      if (seg_ok(e, v)) atomicOr(&e.bitmap[v >> 5], 1u << (v & 31));
    }
    __syncthreads();
    const int64_t nw = (c.n + 31) / 32;
    const int64_t per = (nw + nt - 1) / nt;
    const int64_t w0 = tid * per, w1 = (w0 + per < nw) ? w0 + per : nw;
    int local = 0;
    for (int64_t w = w0; w < w1; ++w) local += __popc(__ldcg(&e.bitmap[w]));
    // block-wide exclusive scan of `local`
    int x = local;
    const int lane = tid & 31, wid = tid >> 5;
    for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(FULL, x, o); if (lane >= o) x += y; }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int v = lane < nwarp ? s_warp[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(FULL, v, o); if (lane >= o) v += y; }
      if (lane < nwarp) s_warp[lane] = v;
    }
    __syncthreads();
    const long long excl = (long long)(x - local) + (wid ? s_warp[wid - 1] : 0);
    total = s_warp[nwarp - 1];
    if (base + total <= e.capacity) {
      long long o = base + excl;
      for (int64_t w = w0; w < w1; ++w) {
        uint32_t word = __ldcg(&e.bitmap[w]);
        while (word) {
          int b = __ffs(word) - 1;
          word &= word - 1;
          e.out[o++] = w * 32 + b;
        }
      }
    }
    for (int64_t w = w0; w < w1; ++w) e.bitmap[w] = 0u;
  }
  return total;
}

__global__ void __launch_bounds__(EMIT_THREADS) k_emit(Common c, EmitArgs e, int j) {
  __shared__ int32_t keys[EMIT_SORT_CAP];
  __shared__ int s_warp[EMIT_THREADS / 32];
  __shared__ long long s_total, s_cnt, s_base;
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  if (tid == 0) {
    const long long st0 = c.ctr[C_STATUS];
    s_bad = (st0 != 0 && st0 != ST_CAPACITY);
    s_cnt = c.ctr[C_YES];
    s_base = c.ctr[C_CURSOR];
  }
  __syncthreads();
  const long long base = s_base;
  const bool bad = s_bad != 0;
  const long long total = bad ? 0 : emit_block(c, e, s_cnt, base, keys, s_warp, &s_total);
  __syncthreads();
  if (tid == 0) {
    if (!bad && base + total > e.capacity)
      atomicCAS((unsigned long long*)&c.ctr[C_STATUS], 0ull, (unsigned long long)ST_CAPACITY);
    e.offs[j + 1] = base + total;
    c.ctr[C_CURSOR] = base + total;
    c.ctr[C_YES] = 0;
    c.ctr[C_TODO] = 0;
  }
}

// Exact decision of up to four undecided users of one query per warp, eight
// lanes per user (four candidates per lane): float32 u.q with its bound
// against the index's interval of each candidate's u.p decides almost every
// user without reading an item row; overlapping candidates are settled one at
// a time with the whole warp (bit-identical to q: an exact tie; else float32
// u.p with its bound); what that leaves open goes to the whole-warp exact
// path (recheck_candidates, or verify_scan for users without a candidate
// proof).  pos: this lane's group's user (sorted position), or -1.  Returns
// the group's yes / no on every lane of the group.
__device__ bool q1_resolve4(const Common& c, const float* sq, float qeps, int k, int64_t pos) {
  const int lane = threadIdx.x & 31, sub = lane & 7;
  const int d = c.d;
  const float tiny = (d + 2) * 0x1p-148f;
  const bool have = pos >= 0;
  const bool quick = have && !c.incomp[pos];
  const float* u = c.Qs + (have ? pos : 0) * d;
  float g32 = 0.f, a32 = 0.f;
  for (int i = sub; quick && i < d; i += 8) {
    const float x = u[i], y = sq[i];
    g32 = fmaf(x, y, g32);
    a32 = fmaf(fabsf(x), fabsf(y), a32);
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {                 // within the eight lanes of the user
    g32 += __shfl_xor_sync(FULL, g32, o);
    a32 += __shfl_xor_sync(FULL, a32, o);
  }
  const float eg = __fmaf_ru(a32, c.cg32, tiny);
  const float gl = __fsub_rd(g32, eg), gh = __fadd_ru(g32, eg);
  int ngt = 0;
  uint32_t ovm = 0;                                  // this lane's candidates whose interval overlaps
  int32_t its[RMIPS_KC / 8] = {-1, -1, -1, -1};
  if (quick) {
    const int32_t* crow = c.cand + pos * RMIPS_KC;
    const float2* cbrow = c.cbnd + pos * RMIPS_KC;
    float2 cbs[RMIPS_KC / 8];
#pragma unroll
    for (int r = 0; r < RMIPS_KC / 8; ++r) {
      its[r] = crow[sub + 8 * r];
      cbs[r] = cbrow[sub + 8 * r];
    }
#pragma unroll
    for (int r = 0; r < RMIPS_KC / 8; ++r) {
      if (its[r] < 0) continue;
      if (cbs[r].x > gh) ++ngt;
      else if (!(cbs[r].y < gl)) ovm |= 1u << r;
    }
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) ngt += __shfl_xor_sync(FULL, ngt, o);
  bool hardg = false;
  for (unsigned pend = __ballot_sync(FULL, ovm != 0); pend; pend = __ballot_sync(FULL, ovm != 0)) {
    const int src = __ffs(pend) - 1;
    const uint32_t m = __shfl_sync(FULL, ovm, src);
    const int r = __ffs(m) - 1;
    if (lane == src) ovm &= ovm - 1;
    int32_t mine = its[0];
#pragma unroll
    for (int x = 1; x < RMIPS_KC / 8; ++x) mine = r == x ? its[x] : mine;
    const int32_t it = __shfl_sync(FULL, mine, src);
    const long long opos = __shfl_sync(FULL, (long long)pos, src);
    const float ogl = __shfl_sync(FULL, gl, src), ogh = __shfl_sync(FULL, gh, src);
    const float* op = c.Ps + (int64_t)it * d;
    const float* ou = c.Qs + opos * d;
    bool same = true;
    float sp = 0.f, sb = 0.f;
    for (int i = lane; i < d; i += 32) {
      const float pv = op[i], uv = ou[i];
      same = same && __float_as_uint(pv) == __float_as_uint(sq[i]);
      sp = fmaf(uv, pv, sp);
      sb = fmaf(fabsf(uv), fabsf(pv), sb);
    }
    same = __all_sync(FULL, same);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sp += __shfl_xor_sync(FULL, sp, o);
      sb += __shfl_xor_sync(FULL, sb, o);
    }
    const float ep = __fmaf_ru(sb, c.cg32, tiny);
    const bool ogt = !same && __fsub_rd(sp, ep) > ogh;
    const bool ohard = !same && !ogt && !(__fadd_ru(sp, ep) < ogl);
    if ((lane >> 3) == (src >> 3)) {
      ngt += ogt ? 1 : 0;
      hardg = hardg || ohard;
    }
  }
  bool yes = quick && !hardg && ngt < k;
  unsigned slow = __ballot_sync(FULL, sub == 0 && have && !(quick && !hardg));
  while (slow) {                                     // the users still open, one at a time with the warp
    const int src = __ffs(slow) - 1;
    slow &= slow - 1;
    const int64_t spos = __shfl_sync(FULL, (long long)pos, src);
    const float* su = c.Qs + spos * d;
    const bool y = !c.incomp[spos]
                       ? recheck_candidates(su, sq, c.cand + spos * RMIPS_KC, c.cbnd + spos * RMIPS_KC, c.Ps, d, k,
                                            c.cg32, c.ctr)
                       : verify_scan(su, c.unorm[spos], c, sq, k, qeps);
    if ((lane >> 3) == (src >> 3)) yes = y;
  }
  return yes;
}

// Public status code of a device status word (asynchronous calls write it).
__device__ __forceinline__ int status_code(long long s) {
  return s == ST_OK ? RMIPS_OK
       : s == ST_NONFINITE ? RMIPS_ERR_NONFINITE
       : s == ST_CAPACITY ? RMIPS_ERR_CAPACITY
       : s == ST_TIMEOUT ? RMIPS_ERR_TIMEOUT
       : s == ST_K_RANGE ? RMIPS_ERR_K_RANGE
       : s == ST_PAIRS_FULL ? RMIPS_ERR_OOM : RMIPS_ERR_INTERNAL;
}

// --- one launch per query (full-P index) ---------------------------------------------
// One CTA per SM.  The users are cut into spans of Q1_WARPS chunks of 32 rows
// (320 users); CTA c owns spans c, c + G, c + 2G, ... (G CTAs).  Warp
// Q1_WARPS is the producer: for 32 of its spans at a time (one per lane) it
// tests Lemma 3 for every block of the span, and for each span that keeps a
// chunk it takes a shared-memory stage, publishes (span, chunk mask), and
// copies every run of consecutive kept chunks with ONE bulk copy (a 1-D
// cp.async.bulk occupies the SM's copy engine for about the same time up to
// 64 KB, so a whole 64,000-byte span of float32 rows at d = 50 costs one
// copy, not ten).  Ten consumer warps measured faster than eight (three
// stages instead of four at d = 50) and than twelve.
// Consumer warp w handles chunk w of each stage: it prefetches its users'
// (lo_k, hi_k) while the rows land, forms u.q with its error bound (Lemma 1:
// no if u.q + e < lo_k; yes if u.q - e >= hi_k), rechecks undecided users
// exactly on the spot (one warp per user over its proven candidates), and
// frees the stage.  Stages are joined by mbarriers: full (the rows landed),
// info (span and mask published), empty (all consumers done).  Every wait is
// bounded; a CTA that gives up drains its own copies before it exits.
// The last CTA to finish (a device-wide counter taken after a memory fence)
// sorts and writes the ids, copies the status, count and counters to `res`
// (and status and count to `done` when given) and clears the counters.
constexpr int RES_STATUS = 0, RES_COUNT = 1, RES_CTR = 2;     // res layout: [2 + C_NCOUNTERS]
constexpr int Q1_WARPS = 10;                                   // consumer warps = chunks per span
constexpr int Q1_THREADS = (Q1_WARPS + 1) * 32;
constexpr int Q1_MAXNS = 6;                                    // stages at most
constexpr size_t Q1_HEAD = 1024;                               // q, barriers, stage info
constexpr int Q1_YCAP = 256;                                   // yes positions a warp buffers
constexpr int Q1_TCAP = 64;                                    // undecided positions past the CTA's list
constexpr int Q1_CTCAP = 1024;                                 // undecided positions the CTA lists
constexpr size_t Q1_BUFS =
    ((size_t)(Q1_WARPS + 1) * Q1_YCAP + (size_t)Q1_WARPS * Q1_TCAP + Q1_CTCAP) * sizeof(int32_t);

// Ascending sort of one value per lane (bitonic network over the warp).
__device__ __forceinline__ int32_t q1_warp_sort(int32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      const int32_t y = __shfl_xor_sync(FULL, x, j);
      const bool up = ((lane & kk) == 0);
      const bool lower = (lane & j) == 0;
      x = (lower == up) ? min(x, y) : max(x, y);
    }
  }
  return x;
}

__host__ __device__ inline size_t q1_stage_bytes(int d, int es) { return (size_t)Q1_WARPS * 32 * d * es; }

// query_bounds for one warp (every lane calls it, all get the result): the
// sum of squares rounded up in every step (any order gives an upper bound of
// ||q||^2), the largest |q_i|, finiteness and the format's range.
__device__ __forceinline__ bool query_bounds_warp(const float* q, int d, int precision, float* qn, float* eps) {
  const int lane = threadIdx.x & 31;
  float acc = 0.f, qmax = 0.f;
  bool fin = true;
  const float vmax = filter_max_abs(precision);
  for (int i = lane; i < d; i += 32) {
    const float v = q[i];
    fin = fin && isfinite(v) && !(fabsf(v) > vmax);
    acc = __fmaf_ru(v, v, acc);
    qmax = fmaxf(qmax, fabsf(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc = __fadd_ru(acc, __shfl_xor_sync(FULL, acc, o));
    qmax = fmaxf(qmax, __shfl_xor_sync(FULL, qmax, o));
  }
  *qn = __fsqrt_ru(acc);
  const float sub = (precision == RMIPS_FP16) ? 0x1p-25f : (precision == RMIPS_BF16 ? 0x1p-133f : 0.f);
  *eps = __fmul_ru((float)(d + 2), __fmaf_ru(sub, qmax, 0x1p-148f));
  return __all_sync(FULL, fin);
}

// u.q for this lane's row of a staged chunk (row-major, stride d).  With d
// even the row is read in pairs: 8-byte words of float32 rows (lane stride
// 25 words for d = 50: conflict-free per half-warp) or 4-byte pairs of 16-bit
// values, and q in pairs broadcast to the warp; two accumulators.  With d
// odd the rotated start r0 = lane mod d keeps the lanes on different banks.
// Any summation order is within the factor cg of the error bound.
template <class T>
__device__ __forceinline__ float q1_dot(const T* __restrict__ row, const float* __restrict__ sq, int d, int lane) {
  float g0 = 0.f, g1 = 0.f;
  if ((d & 1) == 0) {
    const float2* q2 = reinterpret_cast<const float2*>(sq);
    const int h = d >> 1;
    if (sizeof(T) == 4) {
      const float2* r2 = reinterpret_cast<const float2*>(row);
#pragma unroll 5
      for (int j = 0; j < h; ++j) {
        const float2 u = r2[j], q = q2[j];
        g0 = fmaf(u.x, q.x, g0);
        g1 = fmaf(u.y, q.y, g1);
      }
    } else {
      const uint32_t* r2 = reinterpret_cast<const uint32_t*>(row);
#pragma unroll 5
      for (int j = 0; j < h; ++j) {
        const uint32_t w = r2[j];
        T lo_h, hi_h;
        memcpy(&lo_h, &w, 2);
        const uint32_t wh = w >> 16;
        memcpy(&hi_h, &wh, 2);
        const float2 q = q2[j];
        g0 = fmaf(to_f32<T>(lo_h), q.x, g0);
        g1 = fmaf(to_f32<T>(hi_h), q.y, g1);
      }
    }
  } else {
    const int r0 = lane % d;
#pragma unroll 2
    for (int i = 0; i < d; ++i) {
      int r = r0 + i;
      r -= r >= d ? d : 0;
      g0 = fmaf(to_f32<T>(row[r]), sq[r], g0);
    }
  }
  return g0 + g1;
}

template <class T>
__global__ void __launch_bounds__(Q1_THREADS, 1) k_query1(Common c, EmitArgs e, const float* q_src, int k,
                                                          int precision, int ns, long long* res, long long* done,
                                                          unsigned long long* pacc, int res_host) {
  extern __shared__ __align__(128) unsigned char smem[];
  float* sq = reinterpret_cast<float*>(smem);                             // [RMIPS_DMAX]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 512);               // [Q1_MAXNS]
  uint64_t* info = full + Q1_MAXNS;                                       // [Q1_MAXNS]
  uint64_t* empty = info + Q1_MAXNS;                                      // [Q1_MAXNS]
  int2* sinfo = reinterpret_cast<int2*>(smem + 512 + 3 * Q1_MAXNS * 8);   // [Q1_MAXNS] (span, mask)
  int32_t* ybuf = reinterpret_cast<int32_t*>(smem + Q1_HEAD);            // [Q1_WARPS + 1][Q1_YCAP]
  int32_t* tbuf = ybuf + (Q1_WARPS + 1) * Q1_YCAP;                         // [Q1_WARPS][Q1_TCAP]
  int32_t* ctodo = tbuf + Q1_WARPS * Q1_TCAP;                              // [Q1_CTCAP]
  unsigned char* stages = smem + Q1_HEAD + Q1_BUFS;                        // ns x stage, later sort keys
  __shared__ float s_qn, s_eps;
  __shared__ int s_fin, s_last, s_abort, s_ntodo;
  __shared__ int s_fills[Q1_MAXNS];         // phases completed on full[s] by the producer
  __shared__ int s_warp[32];
  __shared__ long long s_total;
  __shared__ long long s_ctr[C_NCOUNTERS];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int d = c.d;
  const int64_t n = c.n;
  const uint32_t chunk_bytes = 32u * d * (uint32_t)sizeof(T);             // multiple of 16
  const size_t stage_bytes = (size_t)Q1_WARPS * chunk_bytes;
  const int64_t nchunks = (n + 31) / 32;
  const int64_t nspans = (nchunks + Q1_WARPS - 1) / Q1_WARPS;
  // Launched with programmatic stream serialization: the next launch on the
  // stream may start its CTAs as this one's leave their SMs; it prepares its
  // barriers and its first Lemma 3 loads (index data, read-only) and waits
  // for this grid's completion before it reads q or the workspace.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (tid == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&info[s], 1);
      mbar_init(&empty[s], Q1_WARPS);
    }
    fence_mbar_init();
    s_abort = 0;
    s_ntodo = 0;
    for (int s = 0; s < Q1_MAXNS; ++s) s_fills[s] = 0;
  }
  // the producer's first round of Lemma 3 loads is issued before the query's
  // norm is known (it only decides the comparison)
  const float* LBk = c.LB + (int64_t)(k - 1) * c.nb;
  const int64_t G = gridDim.x;
  float pre_h[Q1_WARPS], pre_l[Q1_WARPS];
  if (warp == Q1_WARPS) {
    const int64_t sp = blockIdx.x + (int64_t)lane * G;
#pragma unroll
    for (int i = 0; i < Q1_WARPS; ++i) {
      const int64_t ch = sp * Q1_WARPS + i;
      const bool in = sp < nspans && ch < nchunks;
      const int64_t blk = in ? (ch * 32) / c.bs : 0;
      pre_h[i] = in ? c.hdr[blk] : 0.f;
      pre_l[i] = in ? LBk[blk] : 0.f;
    }
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");               // the previous grid has completed
  for (int i = tid; i < d; i += blockDim.x) sq[i] = q_src[i];
  __syncthreads();
  if (warp == 0) {
    float qn0, eps0;
    const bool fin = query_bounds_warp(sq, d, precision, &qn0, &eps0);
    if (lane == 0) {
      s_qn = qn0;
      s_eps = eps0;
      s_fin = fin ? 1 : 0;
    }
  }
  __syncthreads();
  const float qn = s_qn, qeps = s_eps;
  const float2* Lbk = c.Lb + (int64_t)(k - 1) * n;
  long long pruned = 0, tested = 0, todosum = 0, yesfast = 0;
  // Yes positions go to the warp's own buffer in shared memory and reach the
  // global list with one reservation per 256 (every warp has one).
  int32_t* wy = ybuf + warp * Q1_YCAP;
  int ny = 0;                                                  // warp-uniform
  auto flush_yes = [&]() {
    __syncwarp();
    long long b0 = 0;
    if (lane == 0 && ny) b0 = atomicAdd((unsigned long long*)&c.ctr[C_YES], (unsigned long long)ny);
    b0 = __shfl_sync(FULL, b0, 0);
    for (int i = lane; i < ny; i += 32) c.yes[b0 + i] = wy[i];
    __syncwarp();
    ny = 0;
  };
  if (s_fin && warp == Q1_WARPS) {
    // ---------------- producer ----------------
    int stage = 0;
    uint32_t ph = 0;                   // bit s: parity of the next empty wait on stage s
    uint32_t used = 0;                 // bit s: stage s was filled at least once
    bool ok = true;
    for (int64_t base = 0; ok && blockIdx.x + base * G < nspans; base += 32) {
      const int64_t sp = blockIdx.x + (base + lane) * G;
      uint32_t mask = 0;
      if (sp < nspans) {
#pragma unroll
        for (int i = 0; i < Q1_WARPS; ++i) {
          const int64_t ch = sp * Q1_WARPS + i;
          if (ch < nchunks) {
            const int64_t blk = (ch * 32) / c.bs;
            const float h = base == 0 ? pre_h[i] : c.hdr[blk];
            const float lb = base == 0 ? pre_l[i] : LBk[blk];
            if (!(__fmul_ru(h, qn) < lb)) mask |= 1u << i;               // Lemma 3, strict
          }
        }
      }
      {
        const int64_t nch = sp < nspans ? ((nchunks - sp * Q1_WARPS) < Q1_WARPS ? (nchunks - sp * Q1_WARPS) : Q1_WARPS) : 0;
        int pr = (int)nch - __popc(mask);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pr += __shfl_xor_sync(FULL, pr, o);
        pruned += pr;                                          // warp-uniform
      }
      for (uint32_t live = __ballot_sync(FULL, mask != 0); live; live &= live - 1) {
        const int src = __ffs(live) - 1;
        const uint32_t m = __shfl_sync(FULL, mask, src);
        const int64_t s_sp = blockIdx.x + (base + src) * G;
        if (used & (1u << stage)) {                            // wait until the consumers freed it
          bool w = mbar_wait_bounded(&empty[stage], (ph >> stage) & 1u);
          w = __all_sync(FULL, w && !*(volatile int*)&s_abort);
          ph ^= 1u << stage;
          if (!w) { ok = false; break; }
        }
        used |= 1u << stage;
        if (lane == 0) {
          unsigned char* dst = stages + (size_t)stage * stage_bytes;
          const unsigned char* src_rows = reinterpret_cast<const unsigned char*>(c.Qrows) +
                                          (size_t)s_sp * Q1_WARPS * chunk_bytes;
          uint32_t tx = 0;
          for (uint32_t r = m; r;) {                           // runs of consecutive kept chunks
            const int a = __ffs(r) - 1;
            int b = a;
            while (b + 1 < Q1_WARPS && ((r >> (b + 1)) & 1u)) ++b;
            const int64_t last_row = (s_sp * Q1_WARPS + b + 1) * 32;
            const int64_t rows = (last_row < n ? last_row : n) - (s_sp * Q1_WARPS + a) * 32;
            tx += (((uint32_t)(rows * d * sizeof(T))) + 15u) & ~15u;
            r &= ~(((2u << b) - 1u) & ~((1u << a) - 1u));
          }
          sinfo[stage] = make_int2((int)(s_sp), (int)m);
          mbar_arrive(&info[stage]);
          fence_proxy_async();
          s_fills[stage] += 1;
          mbar_arrive_expect_tx(&full[stage], tx);
          for (uint32_t r = m; r;) {
            const int a = __ffs(r) - 1;
            int b = a;
            while (b + 1 < Q1_WARPS && ((r >> (b + 1)) & 1u)) ++b;
            const int64_t last_row = (s_sp * Q1_WARPS + b + 1) * 32;
            const int64_t rows = (last_row < n ? last_row : n) - (s_sp * Q1_WARPS + a) * 32;
            const uint32_t bytes = (((uint32_t)(rows * d * sizeof(T))) + 15u) & ~15u;
            bulk_g2s(dst + (size_t)a * chunk_bytes, src_rows + (size_t)a * chunk_bytes, bytes, &full[stage]);
            r &= ~(((2u << b) - 1u) & ~((1u << a) - 1u));
          }
        }
        __syncwarp();
        stage = stage + 1 == ns ? 0 : stage + 1;
      }
    }
    // end marker for the consumers (or, after a failed wait, the abort flag)
    if (ok && (used & (1u << stage))) {
      bool w = mbar_wait_bounded(&empty[stage], (ph >> stage) & 1u);
      w = __all_sync(FULL, w);
      ph ^= 1u << stage;
      ok = w;
    }
    if (lane == 0) {
      if (ok) {
        sinfo[stage] = make_int2(-1, 0);
        mbar_arrive(&info[stage]);
        s_fills[stage] += 1;
        mbar_arrive(&full[stage]);
      } else {
        set_status(c.ctr, ST_TIMEOUT);
        atomicExch(&s_abort, 1);
      }
    }
  } else if (s_fin && warp < Q1_WARPS) {
    // ---------------- consumers ----------------
    // The stream loop holds no round trip to global memory except the
    // prefetched bounds: yes positions go to the warp's buffer, undecided
    // positions to the CTA's list (resolved by every warp after the stream,
    // four users per warp), or, past its end, to the warp's own list
    // (rechecked by the warp when 64 have gathered).
    int32_t* wt = tbuf + warp * Q1_TCAP;
    int nt = 0;                                                 // warp-uniform
    const uint32_t lt = (1u << lane) - 1u;
    auto recheck = [&]() {                                      // whole warp, one user at a time
      __syncwarp();
      for (int t = 0; t < nt; ++t) {
        const int64_t p = wt[t];
        const float* u = c.Qs + p * d;
        const bool y = !c.incomp[p]
                           ? recheck_candidates(u, sq, c.cand + p * RMIPS_KC, c.cbnd + p * RMIPS_KC, c.Ps, d, k,
                                                c.cg32, c.ctr)
                           : verify_scan(u, c.unorm[p], c, sq, k, qeps);
        if (y) {
          if (ny == Q1_YCAP) flush_yes();
          if (lane == 0) wy[ny] = (int32_t)p;
          ++ny;
        }
      }
      __syncwarp();
      nt = 0;
    };
    int stage = 0;
    uint32_t ph = 0;
    while (true) {
      bool w = mbar_wait_bounded(&info[stage], ph);
      w = __all_sync(FULL, w);
      if (!w) { if (lane == 0) { set_status(c.ctr, ST_TIMEOUT); atomicExch(&s_abort, 1); } break; }
      const int2 si = sinfo[stage];
      if (si.x < 0) break;
      const bool mine = (si.y >> warp) & 1;
      const int64_t pos = ((int64_t)si.x * Q1_WARPS + warp) * 32 + lane;
      const bool valid = mine && pos < n;
      const float2 L = valid ? Lbk[pos] : make_float2(kInf, kInf);   // prefetched while the rows land
      const float un = valid ? c.unorm[pos] : 0.f;
      w = mbar_wait_bounded(&full[stage], ph);
      w = __all_sync(FULL, w);
      if (!w) { if (lane == 0) { set_status(c.ctr, ST_TIMEOUT); atomicExch(&s_abort, 1); } break; }
      if (mine) {
        const T* row = reinterpret_cast<const T*>(stages + (size_t)stage * stage_bytes + (size_t)warp * chunk_bytes) +
                       (size_t)lane * d;
        const float g = q1_dot<T>(row, sq, d, lane);
        bool yes = false, todo = false;
        if (valid) {
          // error bound from ||u|| ||q|| >= sum |u_i q_i| (both norms rounded up)
          const float e = __fmaf_ru(__fmul_ru(un, qn), c.cg, qeps);
          const float hi = __fadd_ru(g, e), lo = __fsub_rd(g, e);
          if (!(hi < L.x)) {                                              // Lemma 1 (strict)
            yes = lo >= L.y;                                              // above hi_k
            todo = !yes;
          }
        }
        const uint32_t by = __ballot_sync(FULL, yes), bt = __ballot_sync(FULL, todo);
        if (by) {
          if (ny + __popc(by) > Q1_YCAP) flush_yes();
          if (yes) wy[ny + __popc(by & lt)] = (int32_t)pos;
          ny += __popc(by);
        }
        if (bt) {
          int base = 0;
          if (lane == 0) base = atomicAdd(&s_ntodo, __popc(bt));
          base = __shfl_sync(FULL, base, 0);
          const int at = base + __popc(bt & lt);
          const uint32_t over = __ballot_sync(FULL, todo && at >= Q1_CTCAP);
          if (todo && at < Q1_CTCAP) ctodo[at] = (int32_t)pos;
          if (over) {                                  // past the CTA's list: the warp's own
            if (nt + __popc(over) > Q1_TCAP) recheck();
            if ((over >> lane) & 1u) wt[nt + __popc(over & lt)] = (int32_t)pos;
            nt += __popc(over);
          }
        }
        yesfast += __popc(by);
        tested += __popc(__ballot_sync(FULL, valid));
        todosum += __popc(bt);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[stage]);
      if (++stage == ns) { stage = 0; ph ^= 1u; }
    }
    recheck();
  }
  // every warp: the CTA's undecided users, four per warp at a time
  __syncthreads();
  if (s_fin && !s_abort) {
    const int ntodo = s_ntodo < Q1_CTCAP ? s_ntodo : Q1_CTCAP;
    for (int base = warp * 4; base < ntodo; base += (Q1_WARPS + 1) * 4) {
      const int at = base + (lane >> 3);
      const int64_t p = at < ntodo ? (int64_t)ctodo[at] : -1;
      const bool y = q1_resolve4(c, sq, qeps, k, p);
      const uint32_t by = __ballot_sync(FULL, (lane & 7) == 0 && p >= 0 && y);
      if (by) {
        if (ny + __popc(by) > Q1_YCAP) flush_yes();
        if ((by >> lane) & 1u) wy[ny + __popc(by & ((1u << lane) - 1u))] = (int32_t)p;
        ny += __popc(by);
      }
    }
  }
  flush_yes();
  if (lane == 0) {
    if (pruned) atomicAdd((unsigned long long*)&c.ctr[C_PRUNED], (unsigned long long)pruned);
    if (tested) atomicAdd((unsigned long long*)&c.ctr[C_TESTED], (unsigned long long)tested);
    if (todosum) atomicAdd((unsigned long long*)&c.ctr[C_TODOSUM], (unsigned long long)todosum);
    if (yesfast) atomicAdd((unsigned long long*)&c.ctr[C_YESFAST], (unsigned long long)yesfast);
  }
  __syncthreads();
  // a CTA that gave up waits (bounded) for the copies it may still have in
  // flight before its shared memory goes away: fill f of stage s is complete
  // once the phase of parity (f - 1) & 1 has completed
  if (s_abort && tid == 0) {
    for (int s = 0; s < ns; ++s)
      if (s_fills[s] > 0) mbar_wait_bounded(&full[s], (uint32_t)((s_fills[s] - 1) & 1));
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd((unsigned long long*)&c.ctr[C_DONE], 1ull) == (unsigned long long)(gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the counters, all at once (one thread each), then the result
  if (tid < C_NCOUNTERS) s_ctr[tid] = __ldcg(&c.ctr[tid]);
  __syncthreads();
  long long status = s_fin ? s_ctr[C_STATUS] : ST_NONFINITE;
  const long long cnt = s_ctr[C_YES];
  long long total = 0;
  if (status == 0 && cnt == 0) {
    // no result (most queries): nothing to sort or write
  } else if (status == 0 && cnt <= 32) {
    // a small result: one warp, one id per lane, sorted with shuffles
    if (warp == 0) {
      int32_t id = INT_MAX;
      if (lane < cnt) {
        const int32_t v = c.permQ[__ldcg(&c.yes[lane])];
        if (seg_ok(e, v)) id = v;
      }
      id = q1_warp_sort(id);
      const int tot = __popc(__ballot_sync(FULL, id != INT_MAX));
      if (tot <= e.capacity && id != INT_MAX) e.out[lane] = id;
      if (lane == 0) s_total = tot;
    }
    __syncthreads();
    total = s_total;
    if (total > e.capacity) status = ST_CAPACITY;
  } else if (status == 0) {
    total = emit_block(c, e, cnt, 0, reinterpret_cast<int32_t*>(stages), s_warp, &s_total);
    if (total > e.capacity) status = ST_CAPACITY;
  }
  __syncthreads();
  if (tid < C_NCOUNTERS) {
    res[RES_CTR + tid] = s_ctr[tid];
    c.ctr[tid] = 0;
  }
  if (tid == 0) {
    res[RES_STATUS] = status;
    res[RES_COUNT] = total;
    if (done) {
      done[0] = status == ST_OK ? RMIPS_OK : (long long)status_code(status);
      done[1] = total;
    }
    if (pacc) {                 // profiling of asynchronous calls: tested users, listed users, pruned chunks
      atomicAdd(&pacc[0], (unsigned long long)s_ctr[C_TESTED]);
      atomicAdd(&pacc[1], (unsigned long long)(s_ctr[C_YESFAST] + s_ctr[C_TODOSUM]));
      atomicAdd(&pacc[2], (unsigned long long)s_ctr[C_PRUNED]);
      atomicAdd(&pacc[3], 1ull);
    }
    if (res_host) __threadfence_system();                      // res is device-mapped host memory
  }
}

struct Launch {
  int filter_grid = 0;
  size_t filter_smem = 0;
  int resolve_grid = 0;
};

template <class T, bool FULLP>
cudaError_t launch_filter(const Common& c, int j, int grid, size_t smem, cudaStream_t st) {
  static thread_local bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_filter<T, FULLP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k_filter<T, FULLP><<<grid, FW * 32, smem, st>>>(c, j);
  return cudaGetLastError();
}

cudaError_t filter_dispatch(const rmips_index* idx, const Common& c, int j, int grid, size_t smem, cudaStream_t st) {
  const bool fp = idx->full_p != 0;
  switch (idx->precision) {
    case RMIPS_BF16:
      return fp ? launch_filter<__nv_bfloat16, true>(c, j, grid, smem, st)
                : launch_filter<__nv_bfloat16, false>(c, j, grid, smem, st);
    case RMIPS_FP16:
      return fp ? launch_filter<__half, true>(c, j, grid, smem, st) : launch_filter<__half, false>(c, j, grid, smem, st);
    default:
      return fp ? launch_filter<float, true>(c, j, grid, smem, st) : launch_filter<float, false>(c, j, grid, smem, st);
  }
}

int elem_bytes(int precision) { return precision == RMIPS_FP32 ? 4 : 2; }

Common make_common(const rmips_index* idx, Workspace* ws) {
  Common c;
  memset(&c, 0, sizeof(c));                        // padding too: graph keys compare the bytes
  c.Qs = idx->Qs;
  c.Qrows = idx->precision == RMIPS_FP32 ? (const void*)idx->Qs : idx->Qh;
  c.Ps = idx->Ps;
  c.Lb = idx->Lb;
  c.LB = idx->LB;
  c.hdr = idx->hdr;
  c.unorm = idx->unorm;
  c.pnorm = idx->pnorm;
  c.cand = idx->cand;
  c.cbnd = idx->cbnd;
  c.incomp = idx->incomp;
  c.permQ = idx->permQ;
  c.n = idx->n;
  c.m = idx->m;
  c.nb = idx->nb;
  c.d = idx->d;
  c.bs = idx->bs;
  c.k_max = idx->k_max;
  c.full_p = idx->full_p;
  c.cg = err_factor(idx->d, idx->precision);
  c.cg32 = err_factor(idx->d, RMIPS_FP32);
  c.dq = ws->dq;
  c.dk = ws->dk;
  c.dqn = ws->dqn;
  c.deps = ws->deps;
  c.yes = ws->yes;
  c.todo = ws->todo;
  c.ctr = ws->ctr;
  return c;
}

rmips_status ensure_queries(rmips_index* idx, Workspace* ws, int64_t nq) {
  if (ws->cap_q >= nq) return RMIPS_OK;
  int64_t cap = nq < 64 ? 64 : nq;
  cudaFree(ws->dq); cudaFree(ws->dk); cudaFree(ws->dqn); cudaFree(ws->deps); cudaFree(ws->doffs);
  cudaFreeHost(ws->h_offs);
  ws->dq = nullptr; ws->dk = nullptr; ws->dqn = nullptr; ws->deps = nullptr; ws->doffs = nullptr; ws->h_offs = nullptr;
  ws->cap_q = 0;
  RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->dq, cap * idx->d * sizeof(float)));
  RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->dk, cap * sizeof(int32_t)));
  RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->dqn, cap * sizeof(float)));
  RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->deps, cap * sizeof(float)));
  RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->doffs, (cap + 1) * sizeof(long long)));
  RMIPS_TRY_CUDA(cudaHostAlloc((void**)&ws->h_offs, (cap + 1) * sizeof(long long), cudaHostAllocDefault));
  ws->cap_q = cap;
  return RMIPS_OK;
}

rmips_status ensure_dout(Workspace* ws, int64_t cap) {
  if (ws->cap_out >= cap) return RMIPS_OK;
  cudaFree(ws->dout);
  ws->dout = nullptr;
  ws->cap_out = 0;
  RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->dout, (cap < 1024 ? 1024 : cap) * sizeof(long long)));
  ws->cap_out = cap < 1024 ? 1024 : cap;
  return RMIPS_OK;
}

rmips_status check_segment(const rmips_index* idx, const rmips_segment* seg) {
  if (!seg) return RMIPS_OK;
  if (seg->reserved != 0 || seg->kind < 0 || seg->kind > 2) { set_error("bad segment"); return RMIPS_ERR_ARG; }
  if (seg->kind == 1 && (seg->begin < 0 || seg->end < seg->begin)) { set_error("bad segment range"); return RMIPS_ERR_ARG; }
  if (seg->kind == 2) {
    if (seg->n_ids < 0 || (seg->n_ids > 0 && !seg->ids)) { set_error("bad segment list"); return RMIPS_ERR_ARG; }
    for (int64_t i = 0; i < seg->n_ids; ++i)
      if (seg->ids[i] < 0 || seg->ids[i] >= idx->n) { set_error("segment id out of range"); return RMIPS_ERR_ARG; }
  }
  return RMIPS_OK;
}

// Runs queries [0, nq) already staged in ws->dq / ws->dk.  Results go to
// `out` (device-visible), offsets to ws->doffs.
rmips_status run_queries(rmips_index* idx, Workspace* ws, int64_t nq, const rmips_segment* segs,
                         long long* out, long long capacity, cudaStream_t st) {
  ws->ctr_dirty = true;
  Common c = make_common(idx, ws);
  static thread_local int sm_count = 0;
  if (!sm_count) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (sm_count <= 0) sm_count = 1;
  }
  const size_t smem = 512 + FW * 2 * 8 + (size_t)FW * 2 * 32 * idx->d * elem_bytes(idx->precision);
  const int64_t nchunks = (idx->n + 31) / 32;
  int64_t want = (nchunks + FW - 1) / FW;
  int64_t per_sm = (int64_t)(228 * 1024) / (int64_t)(smem + 1024);
  if (per_sm > 8) per_sm = 8;
  if (per_sm < 1) per_sm = 1;
  int64_t cap = (int64_t)sm_count * per_sm;
  const int fgrid = (int)(want < cap ? want : cap);
  const int rgrid = sm_count;
  RMIPS_TRY_CUDA(cudaMemsetAsync(ws->ctr, 0, C_NCOUNTERS * sizeof(long long), st));
  k_qprep<<<(unsigned)((nq * 32 + 255) / 256), 256, 0, st>>>(c, nq, idx->precision);
  RMIPS_TRY_CUDA(cudaGetLastError());
  RMIPS_TRY_CUDA(cudaMemsetAsync(ws->doffs, 0, sizeof(long long), st));
  uint32_t* segmask = nullptr;
  std::vector<uint32_t> hmask;
  for (int64_t j = 0; j < nq; ++j) {
    EmitArgs e{};
    e.seg_lo = 0;
    e.seg_hi = INT64_MAX;
    e.segmask = nullptr;
    if (segs) {
      const rmips_segment& sg = segs[j];
      if (sg.kind == 1) { e.seg_lo = sg.begin; e.seg_hi = sg.end; }
      if (sg.kind == 2) {
        const int64_t nw = idx->n / 32 + 1;
        if (!segmask) RMIPS_TRY_CUDA(cudaMallocAsync((void**)&segmask, nw * sizeof(uint32_t), st));
        hmask.assign(nw, 0u);
        for (int64_t i = 0; i < sg.n_ids; ++i) hmask[sg.ids[i] >> 5] |= 1u << (sg.ids[i] & 31);
        RMIPS_TRY_CUDA(cudaMemcpyAsync(segmask, hmask.data(), nw * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
        RMIPS_TRY_CUDA(cudaStreamSynchronize(st));   // hmask is reused by the next query
        e.segmask = segmask;
      }
    }
    e.bitmap = ws->bitmap;
    e.out = out;
    e.capacity = capacity;
    e.offs = ws->doffs;
    const bool prof = idx->prof_on != 0;
    if (prof) {
      while ((int64_t)ws->ev.size() < 2 * (ws->ev_used + 1)) {
        cudaEvent_t ev;
        RMIPS_TRY_CUDA(cudaEventCreate(&ev));
        ws->ev.push_back(ev);
      }
      RMIPS_TRY_CUDA(cudaEventRecord(ws->ev[2 * ws->ev_used], st));
    }
    RMIPS_TRY_CUDA(filter_dispatch(idx, c, (int)j, fgrid, smem, st));
    if (prof) {
      RMIPS_TRY_CUDA(cudaEventRecord(ws->ev[2 * ws->ev_used + 1], st));
      ws->ev_used++;
    }
    k_resolve<<<rgrid, 256, 0, st>>>(c, (int)j);
    k_emit<<<1, EMIT_THREADS, 0, st>>>(c, e, (int)j);
    RMIPS_TRY_CUDA(cudaGetLastError());
  }
  if (segmask) RMIPS_TRY_CUDA(cudaFreeAsync(segmask, st));
  return RMIPS_OK;
}

rmips_status status_from_device(long long s) {
  switch ((int)s) {
    case ST_OK: return RMIPS_OK;
    case ST_K_RANGE: set_error("k outside [1, k_max]"); return RMIPS_ERR_K_RANGE;
    case ST_PAIRS_FULL:
      set_error("the undecided-pair list of a batched pass is full (RMIPS_PAIR_LIST_CAP)");
      return RMIPS_ERR_OOM;
    case ST_NONFINITE:
      set_error("non-finite value in a query (or, for a BF16 / FP16 index, one beyond that format's range)");
      return RMIPS_ERR_NONFINITE;
    case ST_CAPACITY: set_error("output capacity too small"); return RMIPS_ERR_CAPACITY;
    case ST_TIMEOUT: set_error("a device wait timed out"); return RMIPS_ERR_TIMEOUT;
    default: set_error("device-side consistency check failed"); return RMIPS_ERR_INTERNAL;
  }
}

template <class T>
cudaError_t launch_query1(const Common& c, const EmitArgs& e, const float* q, int k, int precision, int ns,
                          long long* res, long long* done, unsigned long long* pacc, int res_host, int grid,
                          size_t smem, cudaStream_t st) {
  static thread_local size_t configured = 0;
  if (configured < smem) {
    cudaError_t err = cudaFuncSetAttribute(k_query1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    configured = smem;
  }
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)grid);
  lc.blockDim = dim3(Q1_THREADS);
  lc.dynamicSmemBytes = smem;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, k_query1<T>, c, e, q, k, precision, ns, res, done, pacc, res_host);
}

// Launch shape of the one-launch query: one CTA per SM (fewer when there are
// fewer spans), as many row stages as fit in 220 KB (at most Q1_MAXNS), and
// room for the emit's sort keys.
struct Q1Plan {
  int grid = 1, ns = 1;
  size_t smem = 0;
};
Q1Plan q1_plan(const rmips_index* idx) {
  static thread_local int sm_count = 0;
  if (!sm_count) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (sm_count <= 0) sm_count = 1;
  }
  Q1Plan p;
  const size_t stage = q1_stage_bytes(idx->d, elem_bytes(idx->precision));
  const size_t budget = 220 * 1024 - Q1_HEAD - Q1_BUFS;
  p.ns = (int)(budget / stage);
  p.ns = p.ns > Q1_MAXNS ? Q1_MAXNS : (p.ns < 1 ? 1 : p.ns);
  if (idx->tune_q1_ns > 0 && idx->tune_q1_ns < p.ns) p.ns = idx->tune_q1_ns;    // the autotuner's choice
  int64_t keys = 1;
  while (keys < idx->n && keys < EMIT_SORT_CAP) keys <<= 1;
  const size_t body = (size_t)p.ns * stage;
  p.smem = Q1_HEAD + Q1_BUFS + (body > (size_t)keys * 4 ? body : (size_t)keys * 4);
  const int64_t nspans = ((idx->n + 31) / 32 + Q1_WARPS - 1) / Q1_WARPS;
  p.grid = (int)(nspans < sm_count ? nspans : sm_count);
  return p;
}

cudaError_t q1_dispatch(const rmips_index* idx, const Common& c, const EmitArgs& e, const float* q, int k,
                        long long* res, long long* done, unsigned long long* pacc, cudaStream_t st,
                        int res_host = 0) {
  const Q1Plan p = q1_plan(idx);
  switch (idx->precision) {
    case RMIPS_BF16:
      return launch_query1<__nv_bfloat16>(c, e, q, k, idx->precision, p.ns, res, done, pacc, res_host, p.grid,
                                          p.smem, st);
    case RMIPS_FP16:
      return launch_query1<__half>(c, e, q, k, idx->precision, p.ns, res, done, pacc, res_host, p.grid, p.smem, st);
    default:
      return launch_query1<float>(c, e, q, k, idx->precision, p.ns, res, done, pacc, res_host, p.grid, p.smem, st);
  }
}

// Single query in one launch; results land in device-mapped host memory.
rmips_status query_fused(rmips_index* idx, Workspace* ws, const float* q, int32_t k, const rmips_segment* seg,
                         int64_t* out_ids, int64_t capacity, int64_t* out_count, cudaStream_t st) {
  const int d = idx->d;
  const float* q_src = q;
  if (!is_device_ptr(q)) {                      // stage q in device-mapped pinned memory
    memcpy(ws->h_q, q, d * sizeof(float));
    q_src = ws->h_q;
  }
  Common c = make_common(idx, ws);
  const bool out_dev = capacity > 0 && is_device_ptr(out_ids);
  if (ws->ctr_dirty) {                           // the one-launch kernel needs zero counters
    RMIPS_TRY_CUDA(cudaMemsetAsync(ws->ctr, 0, C_NCOUNTERS * sizeof(long long), st));
    ws->ctr_dirty = false;
  }
  EmitArgs e{};
  e.seg_lo = (seg && seg->kind == 1) ? seg->begin : 0;
  e.seg_hi = (seg && seg->kind == 1) ? seg->end : INT64_MAX;
  e.segmask = nullptr;
  e.bitmap = ws->bitmap;
  e.out = out_dev ? (long long*)out_ids : ws->h_out;
  e.capacity = out_dev ? capacity : (capacity < ws->cap_hout ? capacity : ws->cap_hout);
  e.offs = nullptr;
  const bool prof = idx->prof_on != 0;
  if (prof) {
    while (ws->ev.size() < 2) {
      cudaEvent_t ev;
      RMIPS_TRY_CUDA(cudaEventCreate(&ev));
      ws->ev.push_back(ev);
    }
    RMIPS_TRY_CUDA(cudaEventRecord(ws->ev[0], st));
  }
  const cudaError_t err = q1_dispatch(idx, c, e, q_src, k, ws->h_res, nullptr, nullptr, st, 1);
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return RMIPS_ERR_CUDA; }
  if (prof) RMIPS_TRY_CUDA(cudaEventRecord(ws->ev[1], st));
  RMIPS_TRY_CUDA(cudaStreamSynchronize(st));
  const long long status = ws->h_res[RES_STATUS];
  if (prof) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ws->ev[0], ws->ev[1]);
    const long long* h = ws->h_res + RES_CTR;
    const int es = idx->precision == RMIPS_FP32 ? 4 : 2;
    std::lock_guard<std::mutex> lk(idx->mu);
    idx->prof.filter_launches += 1;
    idx->prof.filter_ms += ms;
    idx->prof.filter_alg_bytes += 8.0 * idx->nb + ((double)idx->d * es + 12.0) * h[C_TESTED] +
                                  4.0 * (double)(h[C_YESFAST] + h[C_TODOSUM]);
    idx->prof.users_tested += h[C_TESTED];
    idx->prof.blocks_pruned += h[C_PRUNED] * 32 / idx->bs;
    idx->prof.blocks_total += idx->nb;
  }
  const long long count = ws->h_res[RES_COUNT];
  *out_count = count;
  {
    std::lock_guard<std::mutex> lk(idx->mu);
    rmips_query_stats s{};
    s.blocks_total = idx->nb;
    s.blocks_pruned = ws->h_res[RES_CTR + C_PRUNED] * 32 / idx->bs;
    s.users_tested = ws->h_res[RES_CTR + C_TESTED];
    s.yes_fast = ws->h_res[RES_CTR + C_YESFAST];
    s.todo = ws->h_res[RES_CTR + C_TODOSUM];
    s.exact_calls = ws->h_res[RES_CTR + C_EXACT];
    s.result = count;
    idx->last_stats = s;
  }
  if (status == ST_TIMEOUT || status == ST_INTERNAL) ws->ctr_dirty = true;
  rmips_status s = status_from_device(status);
  if (s != RMIPS_OK) return s;
  if (!out_dev && count > 0) memcpy(out_ids, ws->h_out, count * sizeof(long long));
  return RMIPS_OK;
}

struct WsGuard {
  rmips_index* idx;
  Workspace* ws;
  ~WsGuard() { if (ws) release_workspace(idx, ws); }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev); else prev = -1;
  }
  ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

// Stage nq queries and ks into the workspace (one copy each).
rmips_status stage_inputs(rmips_index* idx, Workspace* ws, const float* qs, int64_t nq, const int32_t* ks,
                          cudaStream_t st) {
  RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->dq, qs, nq * idx->d * sizeof(float),
                                 is_device_ptr(qs) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->dk, ks, nq * sizeof(int32_t),
                                 is_device_ptr(ks) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  return RMIPS_OK;
}

void record_stats(rmips_index* idx, Workspace* ws, const long long* h, int64_t nq, bool batch = false) {
  std::lock_guard<std::mutex> lk(idx->mu);
  if (ws->ev_used > 0) {
    double ms = 0.0;
    for (int64_t i = 0; i < ws->ev_used; ++i) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ws->ev[2 * i], ws->ev[2 * i + 1]) == cudaSuccess) ms += t;
    }
    if (idx->prof_on && batch) {
      idx->prof.mfilter_launches += ws->ev_used;
      idx->prof.mfilter_ms += ms;
      idx->prof.mfilter_pairs += h[C_TESTED];
      idx->prof.mfilter_alg_flops += 2.0 * idx->d * (double)h[C_TESTED];
      unsigned long long w[WST_N] = {};
      if (idx->prof_on == 2 && ws->wst && cudaMemcpy(w, ws->wst, sizeof(w), cudaMemcpyDeviceToHost) == cudaSuccess) {
        idx->prof.mfilter_tiles += (int64_t)w[WST_TILES];
        for (int i = 0; i < 5; ++i) idx->prof.mfilter_wait[i] += (double)w[WST_LOADER_WAIT + i];
        idx->prof.mfilter_wait[5] += (double)w[WST_MMA_WAIT_A];
        idx->prof.mfilter_wait[6] += (double)w[WST_EPI_TMEM];
        idx->prof.mfilter_wait[7] += (double)w[WST_MMA_ISSUE];
        idx->prof.mfilter_wait[8] += (double)w[WST_EPI_SLOW];
        idx->prof.mfilter_wait[9] += (double)w[WST_EPI_SLOW_N];
        idx->prof.mfilter_wait[10] += (double)w[WST_EPI_ATOM];
        for (int i = 0; i < 4; ++i) idx->prof.mfilter_cycles[i] += (double)w[WST_LOADER + i];
        idx->prof.mfilter_active_tiles += (int64_t)w[WST_ACTIVE];
      }
    } else if (idx->prof_on) {
      const int es = idx->precision == RMIPS_FP32 ? 4 : 2;
      const double per_user = (double)idx->d * es + 8.0 + (idx->full_p ? 0.0 : 4.0);
      idx->prof.filter_launches += ws->ev_used;
      idx->prof.filter_ms += ms;
      idx->prof.filter_alg_bytes += 8.0 * idx->nb * ws->ev_used + per_user * h[C_TESTED] +
                                    4.0 * (double)(h[C_YESFAST] + h[C_TODOSUM]);
      idx->prof.users_tested += h[C_TESTED];
      idx->prof.blocks_pruned += h[C_PRUNED] * 32 / idx->bs;
      idx->prof.blocks_total += idx->nb * nq;
    }
    ws->ev_used = 0;
  }
  rmips_query_stats s{};
  s.blocks_total = idx->nb;
  s.blocks_pruned = batch ? 0 : h[C_PRUNED] * 32 / idx->bs;
  s.users_tested = h[C_TESTED];
  s.yes_fast = h[C_YESFAST];
  s.todo = h[C_TODOSUM];
  s.exact_calls = h[C_EXACT];
  idx->last_stats = s;
}



// One 128 x 64 x 64 tile through the layout, descriptors, MMA and TMEM loads
// used by the batched filter (test hook).  A [128][64], B [64][64] row-major
// float32 in global memory (rounded to nearest into BF16 / FP16 for those
// kinds); D [128][64] = A B^T.
template <int KIND>
__global__ void __launch_bounds__(128) k_debug_tc(const float* __restrict__ A, const float* __restrict__ B,
                                                  float* __restrict__ D, long long* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  constexpr uint32_t E = KIND == TCK_TF32 ? 4 : 2;
  unsigned char* sA = dsm;                          // 128 x 64
  unsigned char* sB = dsm + 128 * TC_K * E;         // 64 x 64
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t taddr_s;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < 192 * (int)TC_K; e += 128) {
    const bool isA = e < 128 * (int)TC_K;
    const int ee = isA ? e : e - 128 * (int)TC_K;
    const int r = ee / (int)TC_K, k = ee % (int)TC_K;
    const float v = isA ? A[ee] : B[ee];
    unsigned char* base = isA ? sA : sB;
    if (KIND == TCK_TF32) *reinterpret_cast<float*>(base + tc_off(r, k)) = v;
    else if (KIND == TCK_BF16) *reinterpret_cast<__nv_bfloat16*>(base + tc_off16(r, k)) = __float2bfloat16_rn(v);
    else *reinterpret_cast<__half*>(base + tc_off16(r, k)) = __float2half_rn(v);
  }
  if (warp == 0) {
    tmem_alloc(&taddr_s, 64);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    s_fail = 0;
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = taddr_s;
  if (tid == 0) {
    const uint32_t idesc = KIND == TCK_TF32 ? tc_idesc_tf32(128, 64) : tc_idesc_f16(128, 64, KIND == TCK_BF16);
    const uint32_t sbo = KIND == TCK_TF32 ? TC_SBO : TC_SBO16;
    for (uint32_t s = 0; s < TC_K * E / 32; ++s) {
      const uint64_t ad = tc_sdesc(smem_u32(sA) + s * 2 * TC_LBO, TC_LBO, sbo);
      const uint64_t bd = tc_sdesc(smem_u32(sB) + s * 2 * TC_LBO, TC_LBO, sbo);
      if (KIND == TCK_TF32) tc_mma_tf32(taddr, ad, bd, idesc, s > 0 ? 1u : 0u);
      else tc_mma_f16(taddr, ad, bd, idesc, s > 0 ? 1u : 0u);
    }
    tc_commit(&bar);
  }
  if (!mbar_wait_bounded(&bar, 0)) s_fail = 1;
  __syncthreads();
  if (s_fail) {
    if (tid == 0) set_status(status, ST_TIMEOUT);
  } else {
    tc_fence_after();
    float v[16];
    for (int c0 = 0; c0 < 64; c0 += 16) {
      tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      tmem_ld_wait();
      for (int i = 0; i < 16; ++i) D[(warp * 32 + lane) * 64 + c0 + i] = v[i];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, 64);
}

// ===========================================================================
// Batched path: up to MQ_MAXQ queries in one pass over the user rows.
//
//   k_mprep     query norms and checks; queries sorted by (k, descending
//               norm) and laid out in k-groups padded to MQ_TQ slots;
//   k_mfilter   persistent CTAs walk user tiles of MQ_TU users.  For every
//               k-group and every block of the tile, Lemma 3 keeps exactly a
//               prefix of the group (queries are in descending norm), found by
//               binary search; tiles with no surviving (block, query) pair
//               are skipped without reading their rows.  Surviving tiles are
//               multiplied in registers (8 users x 4 queries per thread) and
//               every surviving pair gets the per-user tests of Lemmas 1/2;
//   k_mresolve  exact decision of the undecided pairs (as k_resolve);
//   k_mscan / k_mscatter / k_memit   per-query CSR output, ids ascending.
// ===========================================================================
constexpr int MQ_TU = 128;
constexpr int MQ_THREADS = 256;
constexpr int MQ_US = MQ_TU + 4;       // row stride of the transposed user tile
constexpr int MQ_QS = MQ_TQ + 4;       // row stride of the transposed query tile

// A reserved but unused slot of a pair list (the tensor-core filter's
// epilogue warps reserve the lists in chunks); readers skip it.
constexpr unsigned long long PAIR_NONE = ~0ull;

struct Batch {
  const float* dq;        // [nq][d] staged queries (call order)
  const int32_t* dk;      // [nq]
  float* dqn;             // [nq] norm upper bounds (call order)
  float* deps;            // [nq]
  int nq;                 // queries in this pass (<= MQ_MAXQ)
  float* bq;
  int32_t* bk;
  float* bqn;
  float* beps;
  int32_t* bidx;
  int4* grp;
  int32_t* qcnt;
  int32_t* qcur;
  unsigned long long* ypairs;
  long long cap_y;
  unsigned long long* tpairs;
  long long cap_t;
  int32_t* seg;
  int tc_kind;            // TCK_* operand kind of the tensor-core filter
  float2* bcq;            // [slots] (error scale, absolute slack) of the TC filter
  unsigned char* bitems;  // [MQ_ITEMS] packed items of the TC filter (null: CUDA-core path)
  int* gitem;             // [RMIPS_KMAX_LIMIT + 2] first item of each group; [RMIPS_KMAX_LIMIT + 1] = items
  int2* itemg;            // [MQ_ITEMS] (group, chunk) of each item
  int32_t* gpre;          // [nb][ngroups] Lemma 3 prefix of each (block, group)
  unsigned long long* wst;  // [WST_N] role cycle counters of the TC filter (null: off)
  const long long* seglo;   // [nq] allowed id range per query (null: all users)
  const long long* seghi;
  unsigned long long* keys;  // [nq] sort keys
  unsigned long long* runs;  // [nruns * 1024] keys sorted in runs
  int* hist;              // [RMIPS_KMAX_LIMIT + 2] queries per k
  int* gfirst;            // [RMIPS_KMAX_LIMIT + 2] first sorted position of each k
  int* gslot0;            // [RMIPS_KMAX_LIMIT + 2] first slot of each k-group
  int32_t* big;           // queries with more than MEMIT_MID_CAP results
  int32_t* mid;           // queries with 33 .. MEMIT_MID_CAP results
  int32_t* bslot;         // [nq] id-bitmap slot of a query marked through k_mbig_mark, else -1
  uint32_t* bigmaps;      // MQ_BIG_SLOTS id bitmaps of nw words each
  int* bigcnt;            // [MQ_BIG_SLOTS][nwc] ids per 1024-word chunk of each bitmap
  int64_t nw;             // words per id bitmap
  int64_t nwc;            // 1024-word chunks per id bitmap
  long long* doffs;       // [nq + 1] offsets of this pass (absolute)
  long long* out;
  long long capacity;
};

// (a) per query: norm bound, slack, checks, sort key, k histogram.
__global__ void k_mprep_a(Common c, Batch b, int precision) {
  // eight lanes per query: the sum of squares rounded up in every step (any
  // order gives an upper bound of ||q||^2), the largest |q_i|, finiteness
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j = (int)(t >> 3), sub = (int)(t & 7);
  const int d = c.d;
  const bool live = j < b.nq;
  float acc = 0.f, qmax = 0.f;
  bool fin = true;
  const float vmax = filter_max_abs(precision);
  if (live) {
    const float* q = b.dq + (int64_t)j * d;
    for (int i = sub; i < d; i += 8) {
      const float v = q[i];
      fin = fin && isfinite(v) && !(fabsf(v) > vmax);
      acc = __fmaf_ru(v, v, acc);
      qmax = fmaxf(qmax, fabsf(v));
    }
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    acc = __fadd_ru(acc, __shfl_xor_sync(FULL, acc, o));
    qmax = fmaxf(qmax, __shfl_xor_sync(FULL, qmax, o));
  }
  const unsigned bad = __ballot_sync(FULL, !fin);
  if (!live || sub != 0) return;
  const float qn = __fsqrt_ru(acc);
  const float lsub = (precision == RMIPS_FP16) ? 0x1p-25f : (precision == RMIPS_BF16 ? 0x1p-133f : 0.f);
  const float eps = __fmul_ru((float)(d + 2), __fmaf_ru(lsub, qmax, 0x1p-148f));
  int k = b.dk[j];
  if ((bad >> (threadIdx.x & 24)) & 0xffu) set_status(c.ctr, ST_NONFINITE);
  if (k < 1 || k > c.k_max) { set_status(c.ctr, ST_K_RANGE); k = 1; }
  b.dqn[j] = qn;
  b.deps[j] = eps;
  b.qcnt[j] = 0;
  b.qcur[j] = 0;
  b.keys[j] = ((unsigned long long)k << 46) | ((unsigned long long)(~__float_as_uint(qn)) << 14) |
              (unsigned long long)j;
  atomicAdd(&b.hist[k], 1);
}

// (b) one CTA: k-group layout from the histogram (first sorted position and
// first slot of every k, group table, padding slots), counters of the pass.
__global__ void __launch_bounds__(256) k_mprep_groups(Common c, Batch b) {
  __shared__ int first[RMIPS_KMAX_LIMIT + 2];
  __shared__ int slot0[RMIPS_KMAX_LIMIT + 2];
  __shared__ int hist[RMIPS_KMAX_LIMIT + 2];
  const int tid = threadIdx.x;
  if (tid < RMIPS_KMAX_LIMIT + 2) hist[tid] = (tid >= 1 && tid <= RMIPS_KMAX_LIMIT) ? b.hist[tid] : 0;
  __syncthreads();
  if (tid == 0) {
    c.ctr[C_YES] = 0;
    c.ctr[C_TODO] = 0;
    c.ctr[C_NBIG] = 0;
    c.ctr[C_NMID] = 0;
    c.ctr[C_TILE] = 0;
    int f = 0, s = 0, g = 0, nit = 0;
    for (int k = 0; k <= RMIPS_KMAX_LIMIT + 1; ++k) {
      first[k] = f;
      slot0[k] = s;
      const int h = hist[k];
      if (h > 0) {
        const int tiles = (h + MQ_TQ - 1) / MQ_TQ;
        if (b.gitem) {                               // tensor-core items: chunks of 128 queries
          b.gitem[g] = nit;
          for (int t = 0; t * 128 < h; ++t) b.itemg[nit++] = make_int2(g, t);
        }
        b.grp[g++] = make_int4(k, s, h, tiles);
        f += h;
        s += tiles * MQ_TQ;
      }
    }
    if (b.gitem) b.gitem[RMIPS_KMAX_LIMIT + 1] = nit;
    for (; g <= RMIPS_KMAX_LIMIT; ++g) b.grp[g] = make_int4(0, s, 0, 0);   // empty groups; .y = total slots
  }
  __syncthreads();
  if (tid < RMIPS_KMAX_LIMIT + 2) {
    b.gfirst[tid] = first[tid];
    b.gslot0[tid] = slot0[tid];
  }
  for (int k = 1; k <= RMIPS_KMAX_LIMIT; ++k) {
    const int h = hist[k];
    if (h == 0) continue;
    const int pad = ((h + MQ_TQ - 1) / MQ_TQ) * MQ_TQ;
    for (int r = h + tid; r < pad; r += blockDim.x) {
      b.bidx[slot0[k] + r] = -1;
      b.bk[slot0[k] + r] = k;
      b.bqn[slot0[k] + r] = 0.f;
      b.beps[slot0[k] + r] = 0.f;
      if (b.bcq) b.bcq[slot0[k] + r] = make_float2(0.f, 0.f);
    }
  }
}

// (c) grid: every CTA sorts 1024 keys (k ascending, norm descending, query
// index) in shared memory; padding keys sort last.
constexpr int RUN = 1024;
__global__ void __launch_bounds__(RUN) k_mprep_runs(Batch b) {
  __shared__ unsigned long long keys[RUN];
  const int tid = threadIdx.x;
  const int64_t g = (int64_t)blockIdx.x * RUN + tid;
  keys[tid] = g < b.nq ? b.keys[g] : ~0ull;
  __syncthreads();
  for (int kk = 2; kk <= RUN; kk <<= 1) {
    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
      if (tid < RUN / 2) {
        const int i = 2 * tid - (tid & (jj - 1)), p = i + jj;
        const unsigned long long x = keys[i], y = keys[p];
        if ((x > y) == ((i & kk) == 0)) { keys[i] = y; keys[p] = x; }
      }
      __syncthreads();
    }
  }
  b.runs[g] = keys[tid];
}

// (d) one CTA per run: the final sorted position of each key is its position
// in its run plus, for every other run, the number of keys below it (keys are
// distinct), found by binary search in a shared-memory copy of that run (the
// next run's keys are loaded while the current one is searched); the position
// gives the query's slot in its k-group.
__global__ void __launch_bounds__(RUN) k_mprep_place(Common c, Batch b, int nruns) {
  __shared__ unsigned long long other[RUN];
  const int r = blockIdx.x, tid = threadIdx.x;
  const unsigned long long key = b.runs[(int64_t)r * RUN + tid];
  int64_t rank = tid;
  int o = r == 0 ? 1 : 0;
  unsigned long long nxt = o < nruns ? b.runs[(int64_t)o * RUN + tid] : 0ull;
  while (o < nruns) {                                 // uniform over the CTA
    other[tid] = nxt;
    int on = o + 1;
    if (on == r) ++on;
    if (on < nruns) nxt = b.runs[(int64_t)on * RUN + tid];
    __syncthreads();
    int lo = 0, hi = RUN;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (other[mid] < key) lo = mid + 1; else hi = mid;
    }
    rank += lo;
    __syncthreads();
    o = on;
  }
  if (key == ~0ull) return;                           // padding
  const int k = (int)(key >> 46);
  const int j = (int)(key & 16383ull);
  const int slot = b.gslot0[k] + (int)(rank - b.gfirst[k]);
  b.bidx[slot] = j;
  b.bk[slot] = k;
  const float qn = b.dqn[j], eps = b.deps[j];
  b.bqn[slot] = qn;
  b.beps[slot] = eps;
  if (b.bcq) {        // tensor-core error bound of (u, this query): ||u|| x + y, x = err ||q||,
                      // y covers operands below the normal range (||u|| <= ||u_0||)
    const float err = tc_rel_err(b.tc_kind);
    const float tiny = (c.d + 2) * tc_abs_unit(b.tc_kind);
    b.bcq[slot] = make_float2(__fmul_ru(qn, err), __fmaf_ru(__fadd_ru(qn, c.unorm[0]), tiny, eps));
  }
}

// (e) grid, CUDA-core path: gather the query vectors into slot order, row
// major (zeros in padding).
__global__ void k_mprep_c(Common c, Batch b) {
  const int total_slots = b.grp[RMIPS_KMAX_LIMIT].y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)total_slots * c.d; e += stride) {
    const int slot = (int)(e / c.d), i = (int)(e - (int64_t)slot * c.d);
    const int j = b.bidx[slot];
    b.bq[e] = j >= 0 ? b.dq[(int64_t)j * c.d + i] : 0.f;
  }
}

// (f) one CTA per tensor-core item: the item's 128 query rows in the filter's
// shared-memory operand layout (wf_off with rows of K = 64, zeros past d;
// rows past the group are zero), then their 128 (error scale, slack) pairs
// and 128 query indices (-1 past the group), contiguous so that one bulk copy
// moves the whole item.
__host__ __device__ constexpr uint32_t ws_pack_bytes(int nstep) { return wf_tile_bytes(nstep) + 128u * 12u; }
__global__ void __launch_bounds__(256) k_mprep_items(Common c, Batch b) {
  const int p = blockIdx.x;
  if (p >= b.gitem[RMIPS_KMAX_LIMIT + 1]) return;
  const int2 it = b.itemg[p];
  const int4 G = b.grp[it.x];
  const int r0 = it.y * 128;                       // first query of the item within its group
  const uint32_t esz = b.tc_kind == TCK_TF32 ? 4u : 2u;
  const int nstep = b.tc_kind == TCK_TF32 ? 8 : 4;      // rows of K = 64 (see k_mfilter_ws)
  const uint32_t sbo = wf_sbo(nstep);
  unsigned char* dst = b.bitems + (size_t)p * ws_pack_bytes(nstep);
  const int per = 16 / (int)esz;                   // values per 16-byte chunk
  for (int e = threadIdx.x; e < 128 * 2 * nstep; e += blockDim.x) {
    const int r = e & 127, k0 = (e >> 7) * per;
    const uint32_t off = wf_off(r, (e >> 7) * 16, sbo);
    const bool live = r0 + r < G.z;
    const int j = live ? b.bidx[G.y + r0 + r] : -1;
    const float* q = b.dq + (int64_t)(j < 0 ? 0 : j) * c.d;
    if (esz == 4) {
      float v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = (j >= 0 && k0 + i < c.d) ? q[k0 + i] : 0.f;
      *reinterpret_cast<float4*>(dst + off) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
      uint16_t h[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float v = (j >= 0 && k0 + i < c.d) ? q[k0 + i] : 0.f;
        h[i] = b.tc_kind == TCK_BF16 ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : __half_as_ushort(__float2half_rn(v));
      }
      uint4 w;
      w.x = h[0] | ((uint32_t)h[1] << 16);
      w.y = h[2] | ((uint32_t)h[3] << 16);
      w.z = h[4] | ((uint32_t)h[5] << 16);
      w.w = h[6] | ((uint32_t)h[7] << 16);
      *reinterpret_cast<uint4*>(dst + off) = w;
    }
  }
  float2* cq = reinterpret_cast<float2*>(dst + wf_tile_bytes(nstep));
  int* qj = reinterpret_cast<int*>(cq + 128);
  for (int r = threadIdx.x; r < 128; r += blockDim.x) {
    const bool live = r0 + r < G.z;
    cq[r] = live ? b.bcq[G.y + r0 + r] : make_float2(0.f, 0.f);
    qj[r] = live ? b.bidx[G.y + r0 + r] : -1;
  }
}

// True when the user at sorted position pos lies in query j's id range.
__device__ __forceinline__ bool in_segment(const Common& c, const Batch& b, int j, int64_t pos) {
  if (!b.seglo) return true;
  const long long id = c.permQ[pos];
  return id >= b.seglo[j] && id < b.seghi[j];
}

// Number of leading queries of group g (descending norm) kept by Lemma 3 for
// a block with header h and bound lb: the first r with fl_up(h qn_r) < lb.
__device__ __forceinline__ int lemma3_prefix(const float* __restrict__ qn, int slot0, int size, float h, float lb) {
  int lo = 0, hi = size;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__fmul_ru(h, qn[slot0 + mid]) < lb) hi = mid; else lo = mid + 1;
  }
  return lo;
}

template <class T, bool FULLP>
__global__ void __launch_bounds__(MQ_THREADS) k_mfilter(Common c, Batch b, int ngroups) {
  extern __shared__ __align__(16) float ms[];
  const int d = c.d;
  float* Ut = ms;                                        // [d][MQ_US]
  float* Qt = Ut + d * MQ_US;                            // [d][MQ_QS]
  float2* Lt = reinterpret_cast<float2*>(Qt + d * MQ_QS);  // [ngroups][MQ_TU]
  __shared__ float un_t[MQ_TU];
  __shared__ float qn_t[MQ_TQ], qe_t[MQ_TQ];
  __shared__ int qj_t[MQ_TQ];
  __shared__ int pre[RMIPS_KMAX_LIMIT][4];               // prefix length per (group, block of tile)
  __shared__ int gmax[RMIPS_KMAX_LIMIT];
  __shared__ int any_tile;
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t n = c.n;
  const int sub = c.bs < MQ_TU ? c.bs : MQ_TU;           // users of one block inside a tile
  const int nbt = MQ_TU / sub;                           // blocks (or block parts) per tile
  const int tu = tid & 15, tq = tid >> 4;                // 8 users x 4 queries per thread
  long long st_pairs = 0, st_users = 0, st_lrows = 0, st_yes = 0, st_todo = 0, st_skipped = 0;
  for (int64_t u0 = (int64_t)blockIdx.x * MQ_TU; u0 < n; u0 += (int64_t)gridDim.x * MQ_TU) {
    // 1. Lemma 3 prefixes for every (group, block) of this tile
    if (tid < ngroups * nbt) {
      const int g = tid / nbt, sb = tid - g * nbt;
      const int64_t ufirst = u0 + (int64_t)sb * sub;
      int r = 0;
      const int4 G = b.grp[g];
      if (ufirst < n && G.z > 0) {
        const int64_t blk = ufirst / c.bs;
        r = lemma3_prefix(b.bqn, G.y, G.z, c.hdr[blk], c.LB[(int64_t)(G.x - 1) * c.nb + blk]);
      }
      pre[g][sb] = r;
    }
    __syncthreads();
    if (tid < ngroups) {
      int mx = 0;
      for (int sb = 0; sb < nbt; ++sb) mx = max(mx, pre[tid][sb]);
      gmax[tid] = mx;
    }
    __syncthreads();
    if (tid == 0) {
      int a = 0;
      for (int g = 0; g < ngroups; ++g) a |= gmax[g];
      any_tile = a;
    }
    __syncthreads();
    const int64_t nvalid = (n - u0) < MQ_TU ? (n - u0) : MQ_TU;
    if (!any_tile) {
      if (tid == 0) st_skipped += 1;
      continue;
    }
    // 2. stage the user tile (transposed), norms and the needed bound rows
    const T* src = reinterpret_cast<const T*>(c.Qrows) + u0 * d;
    for (int e = tid; e < MQ_TU * d; e += MQ_THREADS) {
      const int uu = e / d, i = e - uu * d;
      Ut[i * MQ_US + uu] = uu < nvalid ? to_f32<T>(src[e]) : 0.f;
    }
    for (int uu = tid; uu < MQ_TU; uu += MQ_THREADS) un_t[uu] = uu < nvalid ? c.unorm[u0 + uu] : 0.f;
    for (int e = tid; e < ngroups * MQ_TU; e += MQ_THREADS) {
      const int g = e / MQ_TU, uu = e - g * MQ_TU;
      if (gmax[g] > 0 && uu < nvalid)
        Lt[e] = c.Lb[(int64_t)(b.grp[g].x - 1) * n + u0 + uu];
    }
    if (tid == 0) {
      st_users += nvalid;
      for (int g = 0; g < ngroups; ++g) {
        if (gmax[g] > 0) st_lrows += nvalid;
        for (int sb = 0; sb < nbt; ++sb) {
          const int64_t us = (int64_t)sb * sub;
          const int64_t cnt = nvalid - us < sub ? (nvalid - us > 0 ? nvalid - us : 0) : sub;
          st_pairs += (long long)pre[g][sb] * cnt;
        }
      }
    }
    __syncthreads();
    // 3. every surviving query tile of every group
    for (int g = 0; g < ngroups; ++g) {
      const int gm = gmax[g];
      if (gm == 0) continue;
      const int4 G = b.grp[g];
      const int k = G.x;
      const float pk = (k <= c.m) ? c.pnorm[k - 1] : -kInf;
      const int ntile = (gm + MQ_TQ - 1) / MQ_TQ;
      for (int t = 0; t < ntile; ++t) {
        const int s0 = G.y + t * MQ_TQ;
        __syncthreads();                                   // previous tile's readers are done
        for (int e = tid; e < MQ_TQ * d; e += MQ_THREADS) {
          const int qq = e / d, i = e - qq * d;
          Qt[i * MQ_QS + qq] = b.bq[(int64_t)s0 * d + e];
        }
        if (tid < MQ_TQ) {
          qn_t[tid] = b.bqn[s0 + tid];
          qe_t[tid] = b.beps[s0 + tid];
          qj_t[tid] = b.bidx[s0 + tid];
        }
        __syncthreads();
        float acc[8][4];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[a][q] = 0.f;
        for (int i = 0; i < d; ++i) {
          const float4 ua = *reinterpret_cast<const float4*>(&Ut[i * MQ_US + tu * 8]);
          const float4 ub = *reinterpret_cast<const float4*>(&Ut[i * MQ_US + tu * 8 + 4]);
          const float4 qv = *reinterpret_cast<const float4*>(&Qt[i * MQ_QS + tq * 4]);
          const float uv[8] = {ua.x, ua.y, ua.z, ua.w, ub.x, ub.y, ub.z, ub.w};
          const float qa[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[a][q] = fmaf(uv[a], qa[q], acc[a][q]);
        }
        // epilogue: Lemma 3 survivor test, then Lemmas 1 / 2
        uint32_t ymask = 0, tmask = 0;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int uu = tu * 8 + a;
          const int sb = uu / sub;
          const int lim = pre[g][sb];
          const float un = un_t[uu];
          const float2 L = Lt[g * MQ_TU + uu];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int r = t * MQ_TQ + tq * 4 + q;          // rank inside the group
            const bool live = uu < nvalid && r < lim && qj_t[tq * 4 + q] >= 0;
            if (!live) continue;
            const float e = __fmaf_ru(__fmul_ru(un, qn_t[tq * 4 + q]), c.cg, qe_t[tq * 4 + q]);
            const float hi = __fadd_ru(acc[a][q], e);
            if (hi < L.x) continue;                                  // Lemma 1
            const float lo = __fsub_rd(acc[a][q], e);
            const bool yes = FULLP ? (lo >= L.y) : (lo >= __fmul_ru(un, pk));   // hi_k / Lemma 2
            if (yes) ymask |= 1u << (a * 4 + q); else tmask |= 1u << (a * 4 + q);
          }
        }
        if (__any_sync(FULL, (ymask | tmask) != 0)) {
          const uint32_t lt = (1u << lane) - 1u;
          for (int p = 0; p < 32; ++p) {
            bool y = (ymask >> p) & 1u, tt = (tmask >> p) & 1u;
            if (!__any_sync(FULL, y || tt)) continue;
            const int a = p >> 2, q = p & 3;
            const unsigned long long pair =
                ((unsigned long long)(uint32_t)qj_t[tq * 4 + q] << 32) | (unsigned long long)(u0 + tu * 8 + a);
            if ((y || tt) && !in_segment(c, b, qj_t[tq * 4 + q], u0 + tu * 8 + a)) { y = false; tt = false; }
            const uint32_t by = __ballot_sync(FULL, y), bt = __ballot_sync(FULL, tt);
            if (by) {
              long long base = 0;
              if (lane == 0) base = atomicAdd((unsigned long long*)&c.ctr[C_YES], (unsigned long long)__popc(by));
              base = __shfl_sync(FULL, base, 0);
              if (y) {
                const long long at = base + __popc(by & lt);
                if (at < b.cap_y) b.ypairs[at] = pair;
                atomicAdd(&b.qcnt[qj_t[tq * 4 + q]], 1);
              }
            }
            if (bt) {
              long long base = 0;
              if (lane == 0) base = atomicAdd((unsigned long long*)&c.ctr[C_TODO], (unsigned long long)__popc(bt));
              base = __shfl_sync(FULL, base, 0);
              if (tt) {
                const long long at = base + __popc(bt & lt);
                if (at < b.cap_t) b.tpairs[at] = pair;
                else set_status(c.ctr, ST_PAIRS_FULL);
              }
            }
          }
          st_yes += __popc(ymask);
          st_todo += __popc(tmask);
        }
      }
    }
    __syncthreads();
  }
  // statistics (C_TESTED: surviving pairs; C_PRUNED: tiles skipped; C_TODOSUM; C_YESFAST)
  if (tid == 0) {
    atomicAdd((unsigned long long*)&c.ctr[C_TESTED], (unsigned long long)st_pairs);
    atomicAdd((unsigned long long*)&c.ctr[C_PRUNED], (unsigned long long)st_skipped);
  }
  if (st_yes) atomicAdd((unsigned long long*)&c.ctr[C_YESFAST], (unsigned long long)st_yes);
  if (st_todo) atomicAdd((unsigned long long*)&c.ctr[C_TODOSUM], (unsigned long long)st_todo);
  (void)st_users;
  (void)st_lrows;
}

// Four undecided pairs per warp, eight lanes per pair (four candidates per
// lane): float32 u.q with its bound against the index's interval of each
// candidate's u.p decides almost every pair without reading an item row.  A
// pair with an overlapping interval, or whose user has no candidate proof,
// goes to the whole-warp exact path (recheck_candidates / verify_scan).
// Four pairs in flight per warp hide the dependent loads (pair -> user and
// query rows -> candidate intervals); the yes pairs of a warp take one slot
// reservation together.
__global__ void __launch_bounds__(256) k_mresolve(Common c, Batch b) {
  __shared__ long long s_cnt;
  __shared__ int s_skip;
  if (threadIdx.x == 0) {
    const long long st0 = c.ctr[C_STATUS];
    s_skip = (st0 != 0 && st0 != ST_CAPACITY);
    s_cnt = c.ctr[C_TODO] < b.cap_t ? c.ctr[C_TODO] : b.cap_t;
  }
  __syncthreads();
  if (s_skip) return;
  const long long cnt = s_cnt;
  const int lane = threadIdx.x & 31, sub = lane & 7, grp = lane >> 3;
  const int d = c.d;
  const float tiny = (d + 2) * 0x1p-148f;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 4; t0 < cnt; t0 += nw * 4) {
    const int64_t t = t0 + grp;
    const unsigned long long pr = t < cnt ? b.tpairs[t] : PAIR_NONE;
    const bool have = pr != PAIR_NONE;
    const int j = (int)(pr >> 32);
    const int32_t pos = (int32_t)(pr & 0xffffffffull);
    const bool quick = have && c.full_p && !c.incomp[pos];
    const int k = have ? b.dk[j] : 0;
    const float* u = c.Qs + (int64_t)pos * d;
    const float* q = b.dq + (int64_t)j * d;
    float g32 = 0.f, a32 = 0.f;
    for (int i = sub; quick && i < d; i += 8) {
      const float x = u[i], y = q[i];
      g32 = fmaf(x, y, g32);
      a32 = fmaf(fabsf(x), fabsf(y), a32);
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {                 // within the eight lanes of the pair
      g32 += __shfl_xor_sync(FULL, g32, o);
      a32 += __shfl_xor_sync(FULL, a32, o);
    }
    const float eg = __fmaf_ru(a32, c.cg32, tiny);
    const float gl = __fsub_rd(g32, eg), gh = __fadd_ru(g32, eg);
    int ngt = 0;
    uint32_t ovm = 0;                                  // this lane's candidates whose interval overlaps
    int32_t its[RMIPS_KC / 8] = {-1, -1, -1, -1};
    if (quick) {
      const int32_t* crow = c.cand + (int64_t)pos * RMIPS_KC;
      const float2* cbrow = c.cbnd + (int64_t)pos * RMIPS_KC;
      float2 cbs[RMIPS_KC / 8];
#pragma unroll
      for (int r = 0; r < RMIPS_KC / 8; ++r) {
        its[r] = crow[sub + 8 * r];
        cbs[r] = cbrow[sub + 8 * r];
      }
#pragma unroll
      for (int r = 0; r < RMIPS_KC / 8; ++r) {
        if (its[r] < 0) continue;
        if (cbs[r].x > gh) ++ngt;
        else if (!(cbs[r].y < gl)) ovm |= 1u << r;
      }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) ngt += __shfl_xor_sync(FULL, ngt, o);
    // Overlapping candidates: each pair's eight lanes take its own, one at a
    // time, the warp's four pairs side by side.  Most are the query's own
    // copy in P (queries drawn from the items), an exact tie that the bitwise
    // comparison settles; otherwise float32 u.p with its bound.  What that
    // leaves open sends the pair to the exact path below.
    bool hardg = false;
    const unsigned gmask = 0xffu << (grp * 8);
    for (unsigned pend = __ballot_sync(FULL, ovm != 0); pend; pend = __ballot_sync(FULL, ovm != 0)) {
      const unsigned gp = pend & gmask;
      const bool act = gp != 0;                               // this pair has a candidate left
      const int src = act ? __ffs(gp) - 1 : lane;
      const uint32_t m = __shfl_sync(FULL, ovm, src);
      const int r = act ? __ffs(m) - 1 : 0;
      if (act && lane == src) ovm &= ovm - 1;
      int32_t mine = its[0];
#pragma unroll
      for (int x = 1; x < RMIPS_KC / 8; ++x) mine = r == x ? its[x] : mine;
      const int32_t it = __shfl_sync(FULL, mine, src);
      const float* op = c.Ps + (int64_t)(act ? it : 0) * d;
      bool same = true;
      float sp = 0.f, sb = 0.f;
      for (int i = sub; act && i < d; i += 8) {
        const float pv = op[i], uv = u[i];
        same = same && __float_as_uint(pv) == __float_as_uint(q[i]);
        sp = fmaf(uv, pv, sp);
        sb = fmaf(fabsf(uv), fabsf(pv), sb);
      }
      same = (__ballot_sync(FULL, !same) & gmask) == 0;        // all eight lanes of the pair
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        sp += __shfl_xor_sync(FULL, sp, o);
        sb += __shfl_xor_sync(FULL, sb, o);
      }
      const float ep = __fmaf_ru(sb, c.cg32, tiny);
      const bool ogt = act && !same && __fsub_rd(sp, ep) > gh;
      const bool ohard = act && !same && !ogt && !(__fadd_ru(sp, ep) < gl);
      ngt += ogt ? 1 : 0;
      hardg = hardg || ohard;
    }
    bool yes = quick && !hardg && ngt < k;
    // the pairs still undecided, one at a time with the whole warp
    unsigned slow = __ballot_sync(FULL, sub == 0 && have && !(quick && !hardg));
    while (slow) {
      const int src = __ffs(slow) - 1;
      slow &= slow - 1;
      const unsigned long long sp = __shfl_sync(FULL, pr, src);
      const int sj = (int)(sp >> 32);
      const int32_t spos = (int32_t)(sp & 0xffffffffull);
      const float* su = c.Qs + (int64_t)spos * d;
      const float* sq = b.dq + (int64_t)sj * d;
      const int sk = b.dk[sj];
      const bool y = (c.full_p && !c.incomp[spos])
                         ? recheck_candidates(su, sq, c.cand + (int64_t)spos * RMIPS_KC,
                                              c.cbnd + (int64_t)spos * RMIPS_KC, c.Ps, d, sk, c.cg32, c.ctr)
                         : verify_scan(su, c.unorm[spos], c, sq, sk, b.deps[sj]);
      if (lane == src) yes = y;
    }
    const unsigned ym = __ballot_sync(FULL, sub == 0 && yes);
    if (ym) {
      long long base = 0;
      if (lane == 0) base = atomicAdd((unsigned long long*)&c.ctr[C_YES], (unsigned long long)__popc(ym));
      base = __shfl_sync(FULL, base, 0);
      if (sub == 0 && yes) {
        const long long at = base + __popc(ym & ((1u << lane) - 1u));
        if (at < b.cap_y) b.ypairs[at] = pr;
        atomicAdd(&b.qcnt[j], 1);
      }
    }
  }
}

// Exclusive scan of per-query counts into absolute offsets.
__global__ void __launch_bounds__(1024) k_mscan(Common c, Batch b) {
  // One pass: thread t holds the counts of queries R t .. R t + R - 1; one
  // block scan gives each query's offset and each mid / large result its
  // place in the lists (the lists' counters are zero at the pass's start).
  constexpr int R = MQ_MAXQ / 1024;
  static_assert(R * 1024 == MQ_MAXQ && MQ_MAXQ < 65536, "ten queries per thread, list counts in 16 bits");
  __shared__ long long s_warp[32];
  __shared__ int s_wlist[32];
  __shared__ long long s_base;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_base = c.ctr[C_CURSOR];
  const int j0 = tid * R;
  int v[R];
  long long tsum = 0;
  int lists = 0;                                       // mid count | large count << 16
#pragma unroll
  for (int r = 0; r < R; ++r) {
    v[r] = j0 + r < b.nq ? b.qcnt[j0 + r] : 0;
    tsum += v[r];
    lists += v[r] > MEMIT_MID_CAP ? (1 << 16) : (v[r] > 32 ? 1 : 0);
  }
  long long x = tsum;
  int y = lists;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long xo = __shfl_up_sync(FULL, x, o);
    const int yo = __shfl_up_sync(FULL, y, o);
    if (lane >= o) { x += xo; y += yo; }
  }
  if (lane == 31) { s_warp[wid] = x; s_wlist[wid] = y; }
  __syncthreads();
  if (wid == 0) {
    long long w = s_warp[lane];
    int wl = s_wlist[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long wo = __shfl_up_sync(FULL, w, o);
      const int wlo = __shfl_up_sync(FULL, wl, o);
      if (lane >= o) { w += wo; wl += wlo; }
    }
    s_warp[lane] = w;
    s_wlist[lane] = wl;
  }
  __syncthreads();
  long long off = s_base + (x - tsum) + (wid ? s_warp[wid - 1] : 0);
  const int lbase = (y - lists) + (wid ? s_wlist[wid - 1] : 0);
  int nmid = lbase & 0xffff, nbig = lbase >> 16;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int j = j0 + r;
    if (j < b.nq) {
      b.doffs[j] = off;
      off += v[r];
      int32_t slot = -1;
      if (v[r] > MEMIT_MID_CAP) {
        b.big[nbig] = j;
        if (nbig < MQ_BIG_SLOTS) slot = nbig;
        ++nbig;
      } else if (v[r] > 32) {
        b.mid[nmid++] = j;
      }
      b.bslot[j] = slot;
    }
  }
  if (tid == 0) {
    const long long run = s_base + s_warp[31];
    b.doffs[b.nq] = run;
    c.ctr[C_CURSOR] = run;
    c.ctr[C_NMID] = s_wlist[31] & 0xffff;
    c.ctr[C_NBIG] = s_wlist[31] >> 16;
    if (run > b.capacity) set_status(c.ctr, ST_CAPACITY);
  }
}

__global__ void k_mscatter(Common c, Batch b) {
  const long long st0 = c.ctr[C_STATUS];
  if (st0 != 0) return;                                   // capacity or bad input: no output
  const long long cnt = c.ctr[C_YES];
  const long long base0 = b.doffs[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long pr = b.ypairs[i];
    if (pr == PAIR_NONE) continue;
    const int j = (int)(pr >> 32);
    if (b.bslot[j] >= 0) continue;                       // marked straight from the pair list
    const int slot = atomicAdd(&b.qcur[j], 1);
    b.seg[b.doffs[j] - base0 + slot] = (int32_t)(pr & 0xffffffffull);
  }
}

// Ascending sort of one int per lane across a warp (bitonic network).
__device__ __forceinline__ int32_t warp_sort_asc(int32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int32_t y = __shfl_xor_sync(FULL, x, j);
      const bool keep_min = (((lane & j) == 0) == ((lane & k) == 0));
      x = keep_min ? min(x, y) : max(x, y);
    }
  }
  return x;
}

// Positions -> ids, ascending, for queries with at most 32 results: one warp
// per query sorts in registers (8 queries per CTA).
constexpr int MEMIT_Q = 8;
__global__ void __launch_bounds__(256) k_memit(Common c, Batch b) {
  if (c.ctr[C_STATUS] != 0) return;                      // uniform: read-only here
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long base0 = b.doffs[0];
  const int j = blockIdx.x * MEMIT_Q + warp;
  if (j >= b.nq) return;
  const int cnt = b.qcnt[j];
  if (cnt > 0 && cnt <= 32) {
    const long long off = b.doffs[j];
    int32_t v = lane < cnt ? c.permQ[b.seg[off - base0 + lane]] : INT_MAX;
    v = warp_sort_asc(v);
    if (lane < cnt) b.out[off + lane] = v;
  }
}

// Queries with 33 .. MEMIT_MID_CAP results: one CTA per query, bitonic sort in
// shared memory.
__global__ void __launch_bounds__(256) k_memit_mid(Common c, Batch b) {
  __shared__ int32_t keys[MEMIT_MID_CAP];
  __shared__ long long s_n;
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_bad = c.ctr[C_STATUS] != 0;
    s_n = c.ctr[C_NMID];
  }
  __syncthreads();
  if (s_bad) return;
  const long long base0 = b.doffs[0];
  for (long long r = blockIdx.x; r < s_n; r += gridDim.x) {
    const int j = b.mid[r];
    const int cnt = b.qcnt[j];
    const long long off = b.doffs[j];
    int N2 = 64;
    while (N2 < cnt) N2 <<= 1;
    for (int i = tid; i < N2; i += blockDim.x) keys[i] = i < cnt ? c.permQ[b.seg[off - base0 + i]] : INT_MAX;
    __syncthreads();
    for (int kk = 2; kk <= N2; kk <<= 1) {
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
        for (int t = tid; t < (N2 >> 1); t += blockDim.x) {
          const int i = 2 * t - (t & (jj - 1)), p = i + jj;
          const int32_t x = keys[i], y = keys[p];
          if ((x > y) == ((i & kk) == 0)) { keys[i] = y; keys[p] = x; }
        }
        __syncthreads();
      }
    }
    for (int i = tid; i < cnt; i += blockDim.x) b.out[off + i] = keys[i];
    __syncthreads();                                     // keys consumed before the next query
  }
}

// Queries with more than MEMIT_MID_CAP results, the first MQ_BIG_SLOTS of
// them, each through an id bitmap of its own and spread over the grid:
//   mark   every yes pair of such a query sets its id's bit (straight from
//          the pair list: k_mscatter leaves these queries out);
//   count  ids per 1024-word chunk of every bitmap;
//   write  each chunk's ids, ascending, at the query's offset plus the ids of
//          the chunks before it, clearing the words.
__global__ void __launch_bounds__(256) k_mbig_mark(Common c, Batch b) {
  if (c.ctr[C_STATUS] != 0 || c.ctr[C_NBIG] == 0) return;
  const long long cnt = c.ctr[C_YES] < b.cap_y ? c.ctr[C_YES] : b.cap_y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long pr = b.ypairs[i];
    if (pr == PAIR_NONE) continue;
    const int r = b.bslot[(int)(pr >> 32)];
    if (r < 0) continue;
    const int32_t v = c.permQ[(int32_t)(pr & 0xffffffffull)];
    atomicOr(&b.bigmaps[(int64_t)r * b.nw + (v >> 5)], 1u << (v & 31));
  }
}

__device__ __forceinline__ int block_sum256(int x, int* s_red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  __syncthreads();
  if (lane == 0) s_red[wid] = x;
  __syncthreads();
  int t = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) t += s_red[w];
  return t;
}

__global__ void __launch_bounds__(256) k_mbig_count(Common c, Batch b) {
  __shared__ int s_red[8];
  if (c.ctr[C_STATUS] != 0) return;
  const long long nbig = c.ctr[C_NBIG] < MQ_BIG_SLOTS ? c.ctr[C_NBIG] : MQ_BIG_SLOTS;
  for (long long p = blockIdx.x; p < nbig * b.nwc; p += gridDim.x) {
    const long long r = p / b.nwc, ch = p - r * b.nwc;
    const uint32_t* bm = b.bigmaps + r * b.nw;
    int x = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long w = ch * 1024 + threadIdx.x * 4 + i;
      if (w < b.nw) x += __popc(__ldcg(&bm[w]));
    }
    x = block_sum256(x, s_red);
    if (threadIdx.x == 0) b.bigcnt[p] = x;
  }
}

__global__ void __launch_bounds__(256) k_mbig_write(Common c, Batch b) {
  __shared__ int s_red[8];
  __shared__ int s_scan[256];
  if (c.ctr[C_STATUS] != 0) return;
  const long long nbig = c.ctr[C_NBIG] < MQ_BIG_SLOTS ? c.ctr[C_NBIG] : MQ_BIG_SLOTS;
  const int tid = threadIdx.x;
  for (long long p = blockIdx.x; p < nbig * b.nwc; p += gridDim.x) {
    const long long r = p / b.nwc, ch = p - r * b.nwc;
    uint32_t* bm = b.bigmaps + r * b.nw;
    const int j = b.big[r];
    int before = 0;                                      // ids in the chunks before this one
    for (long long q = tid; q < ch; q += blockDim.x) before += b.bigcnt[r * b.nwc + q];
    before = block_sum256(before, s_red);
    uint32_t w4[4];
    int x = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long w = ch * 1024 + tid * 4 + i;
      w4[i] = w < b.nw ? __ldcg(&bm[w]) : 0u;
      x += __popc(w4[i]);
    }
    s_scan[tid] = x;                                     // exclusive scan over the CTA
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
      const int y = tid >= o ? s_scan[tid - o] : 0;
      __syncthreads();
      s_scan[tid] += y;
      __syncthreads();
    }
    long long o = b.doffs[j] + before + s_scan[tid] - x;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long w = ch * 1024 + tid * 4 + i;
      uint32_t word = w4[i];
      if (word) bm[w] = 0u;
      while (word) {
        const int bit = __ffs(word) - 1;
        word &= word - 1;
        b.out[o++] = w * 32 + bit;
      }
    }
    __syncthreads();
  }
}

// Large queries beyond the MQ_BIG_SLOTS handled above: each CTA owns one id
// bitmap and handles queries r = MQ_BIG_SLOTS + blockIdx.x, + gridDim.x, ...
// in turn: set one bit per result id, then read the bitmap back in order
// (block-wide prefix of per-thread bit counts), clearing it for the next one.
__global__ void __launch_bounds__(1024) k_memit_big(Common c, Batch b) {
  __shared__ int s_warp[32];
  __shared__ long long s_nbig;
  __shared__ int s_bad;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    s_bad = c.ctr[C_STATUS] != 0;
    s_nbig = c.ctr[C_NBIG];
  }
  __syncthreads();
  if (s_bad) return;
  uint32_t* bm = b.bigmaps + (int64_t)blockIdx.x * b.nw;
  const long long base0 = b.doffs[0];
  const int64_t per = (b.nw + 1023) / 1024;
  const int64_t w0 = tid * per, w1 = (w0 + per < b.nw) ? w0 + per : b.nw;
  for (long long r = MQ_BIG_SLOTS + blockIdx.x; r < s_nbig; r += gridDim.x) {
    const int j = b.big[r];
    const long long off = b.doffs[j];
    const int cnt = b.qcnt[j];
    for (int i = tid; i < cnt; i += 1024) {
      const int32_t v = c.permQ[b.seg[off - base0 + i]];
      atomicOr(&bm[v >> 5], 1u << (v & 31));
    }
    __syncthreads();
    int local = 0;
    for (int64_t w = w0; w < w1; ++w) local += __popc(__ldcg(&bm[w]));
    int x = local;
    for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(FULL, x, o); if (lane >= o) x += y; }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int v = s_warp[lane];
      for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(FULL, v, o); if (lane >= o) v += y; }
      s_warp[lane] = v;
    }
    __syncthreads();
    long long o = off + (x - local) + (wid ? s_warp[wid - 1] : 0);
    for (int64_t w = w0; w < w1; ++w) {
      uint32_t word = __ldcg(&bm[w]);
      bm[w] = 0u;
      while (word) {
        const int bit = __ffs(word) - 1;
        word &= word - 1;
        b.out[o++] = w * 32 + bit;
      }
    }
    __syncthreads();
  }
}


// Tile shapes of the batched tensor-core filter: user tiles of 128 rows (MMA
// M); query tiles of 64 slots as k_mprep lays them out, multiplied two at a
// time (MMA N up to 128); an epilogue warp owns 32 users x 32 queries.
constexpr int TCU = 128;                       // users per tile (MMA M)
constexpr int TCQ = MQ_TQ;                     // queries per laid-out tile
constexpr int WS_N = 2 * TCQ;                  // queries per item (largest MMA N)
__host__ __device__ constexpr uint32_t tc_esize(int kind) { return kind == TCK_TF32 ? 4u : 2u; }


// ===========================================================================
// Batched filter on tensor cores, warp-specialized.
//
// One persistent CTA per SM walks user tiles of 128 rows (round robin over the
// tiles).  The work of a tile is a list of items, one per (k-group, chunk of
// up to 128 queries) that Lemma 3 keeps for at least one block of the tile;
// the MMA's N is the chunk's query count rounded up to 16.  Four roles run as
// a pipeline joined by mbarriers only:
//   loader   (warp 16)  reads the tile's Lemma 3 prefixes (k_mprefix), skips a
//                       tile with no item, copies the users' norms and (lo, hi)
//                       bounds into one of two tile slots and starts the bulk
//                       copy of the pre-tiled user rows;
//   feeder   (warp 17)  bulk-copies each packed item (query rows, error
//                       constants, query indices) into a ring of stages, which
//                       the MMA commit frees;
//   mma      (warps 18, 19) one thread of each issues the 128 x N x K MMAs
//                       of alternate items into one of WS_NACC TMEM
//                       accumulator stages and commits;
//   epilogue (warps 0-15) warp w reads TMEM lanes 32 (w % 4) .. +31 and
//                       columns 32 (w / 4) .. +31 of a stage, frees the stage
//                       and classifies its 32 users x 32 queries (Lemma 1, then
//                       hi_k or Lemma 2), as k_mfilter does.
// K is rounded up to the MMA's K step (8 for TF32, 16 for BF16 / FP16), not to
// 64: the zero padding past d contributes nothing.  Every wait is bounded: on
// a timeout the CTA raises a flag, each role leaves its loop, waits for its
// copies in flight, and TMEM is freed.
// ===========================================================================
#ifndef RMIPS_WS_EPI
#define RMIPS_WS_EPI 16
#endif
constexpr int WS_EPI = RMIPS_WS_EPI;                   // epilogue warps: 2 sets x 4 lane quadrants x 2 column halves
constexpr int WS_NMMA = RMIPS_WS_NMMA;                 // MMA warps, taking items in turn
constexpr int WS_LOADER = WS_EPI, WS_FEEDER = WS_EPI + 1, WS_MMA = WS_EPI + 2;
constexpr int WS_THREADS = (WS_EPI + 2 + WS_NMMA) * 32;
constexpr int WS_NACC = 4;                             // TMEM accumulator stages of WS_N columns
static_assert(WS_NACC % WS_NMMA == 0 && WS_NACC % 2 == 0, "each MMA warp owns fixed accumulators");
constexpr int WS_MAXNS = RMIPS_WS_MAXNS;               // query stages at most (as many as fit are used)
constexpr int WS_LG = 4;                               // groups per tile whose bounds are staged
constexpr int WS_ESET = WS_EPI / 2;                    // epilogue warps per item: the two sets take alternate items
constexpr int WS_ECOLS = WS_N / (WS_ESET / 4);         // query columns per epilogue warp, read 32 at a time
static_assert(WS_ECOLS == 64 && WS_NACC % 2 == 0, "two sets of 8 epilogue warps, 64 columns each");
constexpr int WS_ESLOTS = 3;                           // tile slots of the epilogue's per-tile data
// Item record flags.  WI_END ends an epilogue set's loop.  WI_LAST (last
// item of its tile) and WI_NEWGROUP (first item of a (tile, group)) describe
// the record only: the epilogue sets see alternate items, so they key their
// per-tile state on (seq, ga) instead.
enum : int { WI_LAST = 1, WI_END = 2, WI_NEWGROUP = 4 };

struct WsTile {                                        // one tile slot, written by the loader
  long long u0;
  int nvalid, ngact, end, seq;
  int k[RMIPS_KMAX_LIMIT];                             // k of each active group
  int item0[RMIPS_KMAX_LIMIT];                         // first packed item of each active group
  int gmax[RMIPS_KMAX_LIMIT];                          // largest prefix over the tile's blocks
  int pre[RMIPS_KMAX_LIMIT][4];                        // prefix of each block of the tile
};
struct WsItem {                                        // one accumulator stage, written by the mma warp
  int seq, ga, t, item, flags;                         // seq: the tile's position in this CTA's sequence
  float2 c0;                                           // (error scale, slack) of the item's first query
};

size_t ws_smem_bytes(int tck, int ns) {
  const int ks = tck == TCK_TF32 ? 8 : 4;               // shared-memory rows of K = 64
  return 2 * (size_t)wf_tile_bytes(ks) + (size_t)ns * ws_pack_bytes(ks) + WS_ESLOTS * (size_t)WS_LG * TCU * 8 +
         WS_ESLOTS * (size_t)TCU * 4;
}

// Lemma 3 prefix of every (block, k-group): the leading queries of the group
// (descending norm) whose bound fl_up(h qn) is not below the block's LB.
// One thread per block.  The query norms of every group (descending) are
// sampled at every fourth slot into shared memory; the search over the
// samples leaves at most three norms between a sample that keeps its query
// and the next that does not, read at once from global memory.  The test is
// lemma3_prefix's, on the same values, so the prefix is the same.
constexpr int MPRE_STRIDE = 4;
__global__ void __launch_bounds__(256) k_mprefix(Common c, Batch b, int ngroups) {
  __shared__ float smp[(MQ_SLOTS + MPRE_STRIDE - 1) / MPRE_STRIDE];
  __shared__ int4 sg[RMIPS_KMAX_LIMIT + 1];
  const int tid = threadIdx.x;
  const int total = b.grp[RMIPS_KMAX_LIMIT].y;            // slots of all groups
  for (int i = tid; i * MPRE_STRIDE < total; i += blockDim.x) smp[i] = b.bqn[i * MPRE_STRIDE];
  for (int g = tid; g < ngroups; g += blockDim.x) sg[g] = b.grp[g];
  __syncthreads();
  const int64_t blk = blockIdx.x * (int64_t)blockDim.x + tid;
  if (blk >= c.nb) return;
  const float h = c.hdr[blk];
  for (int g = 0; g < ngroups; ++g) {
    const int4 G = sg[g];
    if (G.z <= 0) break;                                  // the non-empty groups come first
    const float lb = c.LB[(int64_t)(G.x - 1) * c.nb + blk];
    // samples inside the group: slots MPRE_STRIDE*i, i in [i0, i1)
    const int i0 = (G.y + MPRE_STRIDE - 1) / MPRE_STRIDE, i1 = (G.y + G.z + MPRE_STRIDE - 1) / MPRE_STRIDE;
    int lo = i0, hi = i1;                                 // first sample whose query Lemma 3 drops
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (__fmul_ru(h, smp[mid]) < lb) hi = mid; else lo = mid + 1;
    }
    const int rhi = lo < i1 ? lo * MPRE_STRIDE - G.y : G.z;           // dropped (or the group's end)
    const int rlo = lo > i0 ? (lo - 1) * MPRE_STRIDE - G.y : -1;      // kept (or before the start)
    float v[MPRE_STRIDE - 1];
#pragma unroll
    for (int t = 0; t < MPRE_STRIDE - 1; ++t) v[t] = rlo + 1 + t < rhi ? b.bqn[G.y + rlo + 1 + t] : 0.f;
    int r = rhi;
#pragma unroll
    for (int t = MPRE_STRIDE - 2; t >= 0; --t)
      if (rlo + 1 + t < rhi && __fmul_ru(h, v[t]) < lb) r = rlo + 1 + t;
    b.gpre[blk * ngroups + g] = r;
  }
}

// Queries of item t of a group whose tile prefix is gmax, rounded up to the
// MMA's N granularity (16).
__device__ __forceinline__ int ws_item_n(int gmax, int t) {
  const int q = min(WS_N, gmax - t * WS_N);
  return (q + 15) & ~15;
}

// v[q] for a run-time q in [0, 32) without local memory: a 5-level select tree.
__device__ __forceinline__ float ws_pick(const float* v, int q) {
  float a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = (q & 1) ? v[2 * i + 1] : v[2 * i];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (q & 2) ? a[2 * i + 1] : a[2 * i];
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = (q & 4) ? a[2 * i + 1] : a[2 * i];
#pragma unroll
  for (int i = 0; i < 2; ++i) a[i] = (q & 8) ? a[2 * i + 1] : a[2 * i];
  return (q & 16) ? a[1] : a[0];
}

// Pair lists without a shared counter per pair: an epilogue warp reserves
// slots at least a chunk at a time (one global atomic) and fills them in
// order; the slots left over in its last chunk hold PAIR_NONE, which every
// reader of the lists skips (fewer than a chunk per warp and list).  The
// undecided list is short and walked slot by slot by the recheck: its chunks
// are small.
constexpr int WS_CHUNK_Y = 16, WS_CHUNK_T = 4;
struct WsChunk {
  long long next;   // next free slot of the warp's current chunk
  int left;         // slots left in it
};
// The warp's n new entries (whole warp, uniform n > 0) take the rest of the
// current chunk, then a new one: entry e goes to slot at(e).
struct WsSlots {
  long long a, b;   // first slot of the old and of the new chunk
  int split;        // entries in the old chunk
  __device__ __forceinline__ long long at(int e) const { return e < split ? a + e : b + (e - split); }
};
template <int CHUNK>
__device__ __forceinline__ WsSlots ws_reserve(long long* ctr, int n, WsChunk& ch) {
  WsSlots s{ch.next, 0, ch.left};
  if (n > ch.left) {
    const int need = n - ch.left;
    const int r = need > CHUNK ? need : CHUNK;
    long long base = 0;
    if ((threadIdx.x & 31) == 0) base = (long long)atomicAdd((unsigned long long*)ctr, (unsigned long long)r);
    s.b = __shfl_sync(FULL, base, 0);
    ch.next = s.b + need;
    ch.left = r - need;
  } else {
    ch.next += n;
    ch.left -= n;
  }
  return s;
}

// Lemma 1 / hi_k / Lemma 2 classification of up to 32 accumulators v of one
// user (one lane) against 32 query columns (live leading ones; rows past the
// tile's users pass rowok = false).  Called by the whole warp.  Only columns
// at or above the fast threshold are tested one by one (a lane has one or
// two); their (error scale, slack) and query index come from the warp's copy
// in shared memory (sc, sj: lane l holds column l).  The yes and undecided
// pairs of the warp are appended together into the warp's own chunks of the
// two lists (ws_reserve).
template <bool PROF>
__device__ __forceinline__ void ws_classify(const Common& c, const Batch& b, const float* v, int live, bool rowok,
                                            float thr, float un, float2 L, int k, const float2* sc, const int* sj,
                                            int64_t pos, WsChunk& ych, WsChunk& tch, long long& st_yes,
                                            long long& st_todo, long long& w_atom) {
  const int lane = threadIdx.x & 31;
  uint32_t hit = 0;
#pragma unroll
  for (int q = 0; q < 32; ++q) hit |= (v[q] >= thr ? 1u : 0u) << q;
  if (live < 32) hit &= (1u << live) - 1u;
  if (!rowok) hit = 0;
  const float pkb = c.full_p ? 0.f : __fmul_ru(un, (k <= c.m) ? c.pnorm[k - 1] : -kInf);
  uint32_t ym = 0, tm = 0;
  while (hit) {
    const int q = __ffs(hit) - 1;
    hit &= hit - 1;
    const float2 e2 = sc[q];
    const float vq = ws_pick(v, q);
    const float e = __fmaf_ru(un, e2.x, e2.y);
    if (__fadd_ru(vq, e) < L.x) continue;                                  // decided no by Lemma 1
    if (!in_segment(c, b, sj[q], pos)) continue;
    const float lo = __fsub_rd(vq, e);
    if (c.full_p ? (lo >= L.y) : (lo >= pkb)) ym |= 1u << q;
    else tm |= 1u << q;
  }
  long long t_a = 0;
  if (PROF) t_a = clock64();
  // warp-wide exclusive prefix of both counts; the entries go to the warp's
  // own reserved chunks of the pair lists
  const int ny = __popc(ym), nt = __popc(tm);
  int sy = ny, stt = nt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int a = __shfl_up_sync(FULL, sy, o), bb = __shfl_up_sync(FULL, stt, o);
    if (lane >= o) { sy += a; stt += bb; }
  }
  const int ty = __shfl_sync(FULL, sy, 31), tt = __shfl_sync(FULL, stt, 31);
  const WsSlots wy = ty ? ws_reserve<WS_CHUNK_Y>(&c.ctr[C_YES], ty, ych) : WsSlots{0, 0, 0};
  const WsSlots wt = tt ? ws_reserve<WS_CHUNK_T>(&c.ctr[C_TODO], tt, tch) : WsSlots{0, 0, 0};
  int ey = sy - ny, et = stt - nt;                                  // this lane's first entries
  while (ym) {
    const int q = __ffs(ym) - 1;
    ym &= ym - 1;
    const int j = sj[q];
    const long long at = wy.at(ey++);
    if (at < b.cap_y) b.ypairs[at] = ((unsigned long long)(uint32_t)j << 32) | (unsigned long long)pos;
    atomicAdd(&b.qcnt[j], 1);
  }
  while (tm) {
    const int q = __ffs(tm) - 1;
    tm &= tm - 1;
    const long long at = wt.at(et++);
    if (at < b.cap_t) b.tpairs[at] = ((unsigned long long)(uint32_t)sj[q] << 32) | (unsigned long long)pos;
    else set_status(c.ctr, ST_PAIRS_FULL);
  }
  st_yes += ny;
  st_todo += nt;
  if (PROF) w_atom += clock64() - t_a;
}

template <int KIND, int NSTEP, bool PROF>
__global__ void __launch_bounds__(WS_THREADS, 1) k_mfilter_ws(Common c, Batch b, const unsigned char* __restrict__ qtc,
                                                               int ngroups, int ns) {
  // In shared memory, user tiles and query items have rows of K = 64 (the
  // 8-row groups 2048 / 1024 bytes apart, the stride the MMAs read fastest);
  // the index stores user tiles with rows of the MMA's K only (wf_nstep), and
  // the loader copies them one 8-row group at a time into the wider rows.
  constexpr int KS = KIND == TCK_TF32 ? 8 : 4;          // K steps of a shared-memory row
  static_assert(NSTEP <= KS, "K steps beyond the shared-memory row");
  constexpr uint32_t ABYTES = wf_tile_bytes(KS);       // a user tile in shared memory
  constexpr uint32_t SBO = wf_sbo(KS);
  constexpr uint32_t AGLOB = wf_tile_bytes(NSTEP), SBO_G = wf_sbo(NSTEP);   // a user tile in the index
  constexpr int KSTEP = 32 / (int)tc_esize(KIND);     // K of one MMA
  static_assert(NSTEP * KSTEP <= (int)TC_K, "K steps beyond the padded tile");
  constexpr uint32_t PACK = ws_pack_bytes(KS);        // one stage: an item as k_mprep_items packs it
  constexpr uint32_t BROWS = wf_tile_bytes(KS);        // its query rows; then WS_N (scale, slack), WS_N indices
  static_assert(PACK % 16 == 0 && SBO_G % 16 == 0 && WS_N == TCU, "item layout");
  extern __shared__ __align__(1024) unsigned char wsm[];
  unsigned char* sA = wsm;                             // 2 user tiles (MMA operand slots)
  unsigned char* sB = sA + 2 * ABYTES;                 // ns packed items
  float2* sL = reinterpret_cast<float2*>(sB + (size_t)ns * PACK);   // WS_ESLOTS tile slots of per-user data
  float* sUN = reinterpret_cast<float*>(sL + WS_ESLOTS * WS_LG * TCU);
  __shared__ WsTile tinfo[WS_ESLOTS];
  __shared__ WsItem items[WS_NACC];
  __shared__ int4 sgrp[RMIPS_KMAX_LIMIT];
  __shared__ int sgi[RMIPS_KMAX_LIMIT];
  __shared__ int lpre[RMIPS_KMAX_LIMIT][4];
  __shared__ __align__(8) uint64_t afull[2], aempty[2], eempty[WS_ESLOTS], bfull[WS_MAXNS], bempty[WS_MAXNS];
  __shared__ __align__(8) uint64_t tfull[WS_NACC], tempty[WS_NACC], mdone[WS_NMMA];
  __shared__ uint32_t taddr_s;
  __shared__ volatile int s_fail;
  __shared__ float2 s_ecq[WS_EPI][32];                  // per epilogue warp: 32 columns' (scale, slack)
  __shared__ int s_eqj[WS_EPI][32];                     // and query indices, for the per-pair tests
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sub = c.bs < TCU ? c.bs : TCU;             // users per block inside a tile
  const int nbt = TCU / sub;

  if (warp == 0) {
    tmem_alloc(&taddr_s, WS_NACC * WS_N);
    tmem_relinquish();
  }
  if (tid < ngroups) {
    sgrp[tid] = b.grp[tid];
    sgi[tid] = b.gitem[tid];
  }
  if (tid == 0) {
    // an operand slot is free once both MMA warps are through its tile; a
    // tile's per-user data once every epilogue warp has moved past the tile
    for (int i = 0; i < 2; ++i) { mbar_init(&afull[i], 1); mbar_init(&aempty[i], WS_NMMA); }
    for (int i = 0; i < WS_ESLOTS; ++i) mbar_init(&eempty[i], WS_EPI);
    for (int i = 0; i < ns; ++i) { mbar_init(&bfull[i], 1); mbar_init(&bempty[i], 1); }   // emptied by the MMA commit
    for (int i = 0; i < WS_NACC; ++i) { mbar_init(&tfull[i], 2); mbar_init(&tempty[i], WS_ESET); }
    for (int i = 0; i < WS_NMMA; ++i) mbar_init(&mdone[i], 1);
    fence_mbar_init();
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = taddr_s;
  // Warp-uniform bounded wait: one probe first; on a miss, a loop that gives
  // up after ~2^31 clocks or as soon as another role has failed.  False for
  // the whole warp on failure.  With PROF the cycles spent go to *spent.
  auto wwait = [&](uint64_t* bar, uint32_t parity, long long* spent) -> bool {
    long long t0 = 0;
    if (PROF) t0 = clock64();
    bool ok = __all_sync(FULL, mbar_try_wait(bar, parity));
    if (!ok) {
      const long long t1 = clock64();
      bool mine = false;
      while (!(mine = mbar_try_wait(bar, parity)))
        if (s_fail || clock64() - t1 > (1ll << 31)) break;
      ok = __all_sync(FULL, mine);
      if (!ok) s_fail = 1;
    }
    if (PROF) *spent += clock64() - t0;
    return ok;
  };
  long long t_start = 0;
  if (PROF) t_start = clock64();
  long long w_a = 0, w_b = 0;                          // this role's wait cycles (PROF)
  auto report = [&](int wait_a, int wait_b, int total) {
    if (!PROF || lane != 0) return;
    atomicAdd(&b.wst[wait_a], (unsigned long long)w_a);
    if (wait_b >= 0) atomicAdd(&b.wst[wait_b], (unsigned long long)w_b);
    atomicAdd(&b.wst[total], (unsigned long long)(clock64() - t_start));
  };

  if (warp == WS_LOADER) {
    // ---------------------------------------------------------------- loader
    const int64_t ntiles = (c.n + TCU - 1) / TCU;
    long long st_pairs = 0, st_skipped = 0, st_active = 0;
    uint32_t fpar = 0, fused = 0;           // per operand slot: parity of its fill count, filled at least once
    uint32_t epar = 0;                      // per data slot: parity of its fill count
    int ab = 0, es = 0, seq = 0;
    // Tiles in a snake order over the CTAs (the norm order puts the heaviest
    // first; CTA c takes tiles c, 2G - 1 - c, 2G + c, ... of G per round), so
    // no global counter sits on the loader's path.  A tile's Lemma 3 prefixes
    // are loaded one tile ahead, and its norms and bounds with every load
    // issued before the first store: one memory latency per tile.
    const int64_t G = gridDim.x;
    auto tile_at = [&](int64_t i) -> int64_t { return i * G + ((i & 1) ? G - 1 - blockIdx.x : blockIdx.x); };
    auto load_pre = [&](int64_t t, int* pf) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int e = lane + 32 * i;
        pf[i] = 0;
        if (t < ntiles && e < ngroups * nbt) {
          const int g = e / nbt, sb = e - g * nbt;
          const int64_t uf = t * TCU + (int64_t)sb * sub;
          if (uf < c.n && sgrp[g].z > 0) pf[i] = b.gpre[(uf / c.bs) * ngroups + g];
        }
      }
    };
    static_assert(RMIPS_KMAX_LIMIT * 4 <= 128, "prefixes of a tile: four per lane");
    int64_t iter = 0, tt = tile_at(0);
    int pf[4];
    load_pre(tt, pf);
    for (;;) {
      if (tt >= ntiles || s_fail) break;
      const int64_t tn = tile_at(iter + 1);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int e = lane + 32 * i;
        if (e < ngroups * nbt) lpre[e / nbt][e % nbt] = pf[i];
      }
      __syncwarp();
      load_pre(tn, pf);                                 // in flight while this tile is prepared
      const int64_t u0 = tt * TCU;
      const int nvalid = (int)((c.n - u0) < TCU ? (c.n - u0) : TCU);
      int gm = 0;
      if (lane < ngroups) {
        for (int sb = 0; sb < nbt; ++sb) {
          const int p = lpre[lane][sb];
          gm = max(gm, p);
          const int cnt = min(sub, max(0, nvalid - sb * sub));
          st_pairs += (long long)p * cnt;
        }
      }
      const unsigned act = __ballot_sync(FULL, gm > 0);
      ++iter;
      if (!act) {
        ++st_skipped;
        tt = tn;
        __syncwarp();
        continue;
      }
      if (!wwait(&aempty[ab], ((fpar >> ab) & 1u) ^ 1u, &w_a)) break;
      if (!wwait(&eempty[es], ((epar >> es) & 1u) ^ 1u, &w_a)) break;
      WsTile& T = tinfo[es];
      if (gm > 0) {
        const int ga = __popc(act & ((1u << lane) - 1u));
        T.k[ga] = sgrp[lane].x;
        T.item0[ga] = sgi[lane];
        T.gmax[ga] = gm;
        for (int sb = 0; sb < 4; ++sb) T.pre[ga][sb] = sb < nbt ? lpre[lane][sb] : 0;
      }
      if (lane == 0) {
        T.u0 = u0;
        T.nvalid = nvalid;
        T.ngact = __popc(act);
        T.end = 0;
        T.seq = seq;
      }
      __syncwarp();
      const int nstage = min(__popc(act), WS_LG);          // further groups' bounds are read from memory
      float unv[TCU / 32];
      float2 lbv[WS_LG][TCU / 32];
#pragma unroll
      for (int i = 0; i < TCU / 32; ++i) {
        const int r = lane + 32 * i;
        unv[i] = r < nvalid ? c.unorm[u0 + r] : 0.f;
      }
#pragma unroll
      for (int ga = 0; ga < WS_LG; ++ga) {
        const float2* src = c.Lb + (int64_t)((ga < nstage ? T.k[ga] : 1) - 1) * c.n + u0;
#pragma unroll
        for (int i = 0; i < TCU / 32; ++i) {
          const int r = lane + 32 * i;
          lbv[ga][i] = (ga < nstage && r < nvalid) ? src[r] : make_float2(kInf, kInf);
        }
      }
#pragma unroll
      for (int i = 0; i < TCU / 32; ++i) sUN[es * TCU + lane + 32 * i] = unv[i];
#pragma unroll
      for (int ga = 0; ga < WS_LG; ++ga)
        if (ga < nstage) {
          float2* dst = sL + ((size_t)es * WS_LG + ga) * TCU;
#pragma unroll
          for (int i = 0; i < TCU / 32; ++i) dst[lane + 32 * i] = lbv[ga][i];
        }
      __threadfence_block();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive_expect_tx(&afull[ab], AGLOB);
        if (SBO_G == SBO) {
          bulk_g2s(sA + (size_t)ab * ABYTES, qtc + (size_t)tt * AGLOB, AGLOB, &afull[ab]);
        } else {
#pragma unroll 1
          for (int g = 0; g < TCU / 8; ++g)                         // one 8-row group per copy
            bulk_g2s(sA + (size_t)ab * ABYTES + (size_t)g * SBO, qtc + (size_t)tt * AGLOB + (size_t)g * SBO_G, SBO_G,
                     &afull[ab]);
        }
      }
      fpar ^= 1u << ab;
      fused |= 1u << ab;
      epar ^= 1u << es;
      ab ^= 1;
      es = es + 1 == WS_ESLOTS ? 0 : es + 1;
      ++seq;
      ++st_active;
      tt = tn;
    }
    if (!s_fail && wwait(&aempty[ab], ((fpar >> ab) & 1u) ^ 1u, &w_a) &&
        wwait(&eempty[es], ((epar >> es) & 1u) ^ 1u, &w_a)) {            // end marker
      if (lane == 0) {
        tinfo[es].end = 1;
        __threadfence_block();
        mbar_arrive(&afull[ab]);
      }
      fpar ^= 1u << ab;
      fused |= 1u << ab;
    }
    for (int x = 0; x < 2; ++x)                                       // copies in flight
      if ((fused >> x) & 1u) mbar_wait_bounded(&afull[x], ((fpar >> x) & 1u) ^ 1u);
    for (int o = 16; o > 0; o >>= 1) st_pairs += __shfl_xor_sync(FULL, st_pairs, o);
    if (lane == 0) {
      atomicAdd((unsigned long long*)&c.ctr[C_TESTED], (unsigned long long)st_pairs);
      atomicAdd((unsigned long long*)&c.ctr[C_PRUNED], (unsigned long long)st_skipped);
    }
    report(WST_LOADER_WAIT, -1, WST_LOADER);
    if (PROF && lane == 0) atomicAdd(&b.wst[WST_ACTIVE], (unsigned long long)st_active);
  } else if (warp == WS_FEEDER) {
    // ---------------------------------------------------------------- feeder
    uint32_t wpar = 0;                      // per slot: parity of the next wait
    uint32_t epar = 0;                      // per stage: uses so far (parity)
    uint32_t armed = 0;                     // per stage: a copy was started
    int stg = 0, ab = 0, es = 0;
    for (;;) {
      if (!wwait(&afull[ab], (wpar >> ab) & 1u, &w_b)) break;
      wpar ^= 1u << ab;
      const WsTile& T = tinfo[es];
      if (T.end) break;
      bool ok = true;
      for (int ga = 0; ga < T.ngact && ok; ++ga) {
        const int gmax = T.gmax[ga], item0 = T.item0[ga];
        const int nt = (gmax + WS_N - 1) / WS_N;
        for (int t = 0; t < nt; ++t) {
          if (!wwait(&bempty[stg], ((epar >> stg) & 1u) ^ 1u, &w_a)) { ok = false; break; }
          epar ^= 1u << stg;
          if (lane == 0) {                     // one bulk copy per item: each costs the same up to 64 KB
            mbar_arrive_expect_tx(&bfull[stg], PACK);
            bulk_g2s(sB + (size_t)stg * PACK, b.bitems + (size_t)(item0 + t) * PACK, PACK, &bfull[stg]);
          }
          armed |= 1u << stg;
          stg = stg + 1 == ns ? 0 : stg + 1;
        }
      }
      if (!ok) break;
      ab ^= 1;
      es = es + 1 == WS_ESLOTS ? 0 : es + 1;
    }
    for (int x = 0; x < ns; ++x)                                      // copies in flight
      if ((armed >> x) & 1u) mbar_wait_bounded(&bfull[x], ((epar >> x) & 1u) ^ 1u);
    report(WST_FEEDER_WAIT, -1, WST_FEEDER);
  } else if (warp >= WS_MMA && warp < WS_MMA + WS_NMMA) {
    // ---------------------------------------------------------------- mma
    // The tensor core queues almost nothing: every cycle the issuing thread
    // spends between two MMAs (a barrier wait, loop control) leaves it idle.
    // WS_NMMA warps therefore issue items in turn -- the others wait while one
    // issues -- the MMAs go out as soon as the item's waits pass (its record
    // is written after them), and the K loop has a compile-time trip count.
    // Items keep the round-robin stage / accumulator order.  ns and WS_NACC
    // are multiples of WS_NMMA, so warp w owns the stages and accumulators
    // of items w, w + WS_NMMA, ... and waits on each of their barriers'
    // phases in order (a barrier is never tested one phase early).
    const int me = warp - WS_MMA;
    const uint64_t adesc0 = tc_sdesc(smem_u32(sA), TC_LBO, SBO);
    const uint64_t adesc1 = tc_sdesc(smem_u32(sA + ABYTES), TC_LBO, SBO);
    const uint64_t bdesc0 = tc_sdesc(smem_u32(sB), TC_LBO, SBO);
    constexpr uint64_t BSTEP = PACK >> 4;                 // descriptor units per stage
    uint32_t wpar = 0, fpar = 0, tpar = 0;                // parities: slots, stages, accumulators
    int stg = 0, acc = 0, ab = 0, it = 0, es = 0, seq = 0;
    long long w_c = 0, n_items = 0, w_issue = 0;
    for (;;) {
      if (!wwait(&afull[ab], (wpar >> ab) & 1u, &w_c)) break;
      wpar ^= 1u << ab;
      const WsTile& T = tinfo[es];
      if (T.end) break;
      const int ngact = T.ngact;
      bool ok = true, issued = false;
      for (int ga = 0; ga < ngact && ok; ++ga) {
        const int gmax = T.gmax[ga];
        const int nt = (gmax + WS_N - 1) / WS_N;
        for (int t = 0; t < nt; ++t, ++it) {
          const uint32_t fp = (fpar >> stg) & 1u, tp = (tpar >> acc) & 1u;
          fpar ^= 1u << stg;
          tpar ^= 1u << acc;
          if (it % WS_NMMA == me) {
            if (!wwait(&bfull[stg], fp, &w_a)) { ok = false; break; }
            if (!wwait(&tempty[acc], tp ^ 1u, &w_b)) { ok = false; break; }
            long long t_is = 0;
            if (PROF) t_is = clock64();
            if (lane == 0) {
              const int nq = ws_item_n(gmax, t);
              const uint32_t idesc = KIND == TCK_TF32 ? tc_idesc_tf32(TCU, (uint32_t)nq)
                                                      : tc_idesc_f16(TCU, (uint32_t)nq, KIND == TCK_BF16);
              const uint64_t ad0 = ab ? adesc1 : adesc0, bd0 = bdesc0 + (uint64_t)stg * BSTEP;
              const uint32_t d = taddr + (uint32_t)(acc * WS_N);
              tc_fence_after();
              // one K step is 32 bytes = 2 core-matrix columns = +16 in the
              // descriptors' 16-byte address field
#pragma unroll
              for (int s = 0; s < NSTEP; ++s) {
                if (KIND == TCK_TF32) tc_mma_tf32(d, ad0 + (uint64_t)(s * 16), bd0 + (uint64_t)(s * 16), idesc, s > 0 ? 1u : 0u);
                else tc_mma_f16(d, ad0 + (uint64_t)(s * 16), bd0 + (uint64_t)(s * 16), idesc, s > 0 ? 1u : 0u);
              }
              const float2 c0 = *reinterpret_cast<const float2*>(sB + (size_t)stg * PACK + BROWS);
              items[acc] = WsItem{seq, ga, t, T.item0[ga] + t,
                                  (ga == ngact - 1 && t == nt - 1 ? WI_LAST : 0) | (t == 0 ? WI_NEWGROUP : 0), c0};
              tc_commit(&bempty[stg]);           // the stage is free once these MMAs have read it
              tc_commit(&tfull[acc]);
              mbar_arrive(&tfull[acc]);
              if (PROF) w_issue += clock64() - t_is;
            }
            __syncwarp();
            issued = true;
            ++n_items;
          }
          stg = stg + 1 == ns ? 0 : stg + 1;
          acc = acc + 1 == WS_NACC ? 0 : acc + 1;
        }
      }
      if (!ok) break;
      // this warp is through the tile: its operand slot is free once its MMAs
      // have completed (none issued: at once -- earlier ones read other tiles)
      if (lane == 0) {
        if (issued) tc_commit(&aempty[ab]);
        else mbar_arrive(&aempty[ab]);
      }
      __syncwarp();
      ab ^= 1;
      es = es + 1 == WS_ESLOTS ? 0 : es + 1;
      ++seq;
    }
    // end markers in the next two accumulator stages, so that both epilogue
    // sets (alternate stages) see one, each written by the stage's owner
    if (me == acc % WS_NMMA || me == (acc + 1) % WS_NMMA) {
      const int ea = me == acc % WS_NMMA ? acc : (acc + 1) % WS_NACC;
      if (!s_fail && wwait(&tempty[ea], ((tpar >> ea) & 1u) ^ 1u, &w_b)) {
        if (lane == 0) {
          items[ea].flags = WI_END;
          mbar_arrive_cnt(&tfull[ea], 2);
        }
      }
    }
    if (lane == 0) {                                                  // this warp's MMAs in flight
      tc_commit(&mdone[me]);
      mbar_wait_bounded(&mdone[me], 0);
    }
    __syncwarp();
    if (me == 0) report(WST_MMA_WAIT_B, WST_MMA_WAIT_T, WST_MMA);
    if (PROF && lane == 0) {
      atomicAdd(&b.wst[WST_TILES], (unsigned long long)n_items);
      if (me == 0) atomicAdd(&b.wst[WST_MMA_WAIT_A], (unsigned long long)w_c);
      if (me == 0) atomicAdd(&b.wst[WST_MMA_ISSUE], (unsigned long long)w_issue);
    }
  } else if (warp < WS_EPI) {
    // ---------------------------------------------------------------- epilogue
    // Two sets of WS_ESET warps take alternate items (set s: accumulator
    // stages s, s + 2, ...), so each warp has two items' time for one.  In a
    // set, the warp of lane quadrant q4 and column half h classifies 32 users
    // x 64 query columns, read from TMEM 32 columns at a time; the stage is
    // released after both halves (the per-pair tests use the values).
    const int eset = warp / WS_ESET, q4 = warp & 3, col = ((warp >> 2) & 1) * WS_ECOLS;
    const int uu = q4 * 32 + lane;                                    // this thread's user row
    const uint32_t tl = taddr + ((uint32_t)(q4 * 32) << 16) + (uint32_t)col;
    long long st_yes = 0, st_todo = 0, w_slow = 0, n_slow = 0, w_atom = 0;
    WsChunk ych{0, 0}, tch{0, 0};                                    // this warp's chunks of the pair lists
    uint32_t tpar = 0;
    int acc = eset;
    int cur_seq = 0;                       // first tile whose data this warp has not released
    int c_seq = -1, c_ga = -1;             // (tile, group) of the constants held
    int pre_w = 0, nvalid = 0, kq = 1;
    long long u0 = 0;
    float un = 0.f;
    float2 L = make_float2(kInf, kInf);
    for (;;) {
      if (!wwait(&tfull[acc], (tpar >> acc) & 1u, &w_a)) break;
      tpar ^= 1u << acc;
      const WsItem itm = items[acc];
      if (itm.flags & WI_END) break;
      // items come in tile order: the tiles before this item's are done for
      // this warp, whether or not it had items in them
      for (; cur_seq < itm.seq; ++cur_seq)
        if (lane == 0) mbar_arrive(&eempty[cur_seq % WS_ESLOTS]);
      if (itm.seq != c_seq || itm.ga != c_ga) {
        const int es = itm.seq % WS_ESLOTS;
        const WsTile& T = tinfo[es];
        pre_w = T.pre[itm.ga][(q4 * 32) / sub];
        nvalid = T.nvalid;
        u0 = T.u0;
        kq = T.k[itm.ga];
        un = sUN[es * TCU + uu];
        L = itm.ga < WS_LG ? sL[((size_t)es * WS_LG + itm.ga) * TCU + uu]
                           : (uu < nvalid ? c.Lb[(int64_t)(kq - 1) * c.n + u0 + uu] : make_float2(kInf, kInf));
        c_seq = itm.seq;
        c_ga = itm.ga;
      }
      // live queries of this warp's columns for its block (warp-uniform)
      int live = pre_w - itm.t * WS_N - col;
      live = live < 0 ? 0 : (live > WS_ECOLS ? WS_ECOLS : live);
      const bool rowok = uu < nvalid;
      const int64_t pos = u0 + uu;
      // Fast Lemma 1: the item's first query has the largest error scale
      // and slack (descending norm), so acc < lo_k - e(u, q_0) proves "no".
      const float thr = __fsub_rd(L.x, __fmaf_ru(un, itm.c0.x, itm.c0.y));
#pragma unroll
      for (int h = 0; h < WS_ECOLS / 32; ++h) {
        int lh = live - 32 * h;
        if (lh <= 0) break;                                           // warp-uniform
        lh = lh > 32 ? 32 : lh;
        float v[32];
        long long t_ld = 0;
        if (PROF) t_ld = clock64();
        tc_fence_after();
        const float mx = tmem_ld32_max(tl + (uint32_t)(acc * WS_N + 32 * h), v);
        tmem_ld_wait();
        if (PROF) w_b += clock64() - t_ld;
        bool any = rowok;
        if (rowok && lh == 32) any = mx >= thr;
        if (__any_sync(FULL, any)) {
          long long t_sl = 0;
          if (PROF) t_sl = clock64();
          // (error scale, slack) and index of these 32 query columns, one
          // coalesced load each from the packed item in global memory (its
          // stage in shared memory may be refilled already)
          const float2* cq0 = reinterpret_cast<const float2*>(b.bitems + (size_t)itm.item * PACK + BROWS);
          s_ecq[warp][lane] = __ldg(cq0 + col + 32 * h + lane);
          s_eqj[warp][lane] = __ldg(reinterpret_cast<const int*>(cq0 + WS_N) + col + 32 * h + lane);
          __syncwarp();
          ws_classify<PROF>(c, b, v, lh, any, thr, un, L, kq, s_ecq[warp], s_eqj[warp], pos, ych, tch, st_yes,
                            st_todo, w_atom);
          __syncwarp();
          if (PROF) {
            w_slow += clock64() - t_sl;
            ++n_slow;
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
      acc = acc + 2 >= WS_NACC ? acc + 2 - WS_NACC : acc + 2;
    }
    // the unused rest of both chunks (fewer than a chunk each)
    if (lane < ych.left && ych.next + lane < b.cap_y) b.ypairs[ych.next + lane] = PAIR_NONE;
    if (lane < tch.left && tch.next + lane < b.cap_t) b.tpairs[tch.next + lane] = PAIR_NONE;
    for (int o = 16; o > 0; o >>= 1) {
      st_yes += __shfl_xor_sync(FULL, st_yes, o);
      st_todo += __shfl_xor_sync(FULL, st_todo, o);
    }
    if (lane == 0 && st_yes) atomicAdd((unsigned long long*)&c.ctr[C_YESFAST], (unsigned long long)st_yes);
    if (lane == 0 && st_todo) atomicAdd((unsigned long long*)&c.ctr[C_TODOSUM], (unsigned long long)st_todo);
    if (warp == 0) report(WST_EPI_WAIT, WST_EPI_TMEM, WST_EPI);
    if (PROF && warp == 0 && lane == 0) {
      atomicAdd(&b.wst[WST_EPI_SLOW], (unsigned long long)w_slow);
      atomicAdd(&b.wst[WST_EPI_SLOW_N], (unsigned long long)n_slow);
      atomicAdd(&b.wst[WST_EPI_ATOM], (unsigned long long)w_atom);
    }
  }
  if (s_fail && tid == 0) set_status(c.ctr, ST_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(taddr, WS_NACC * WS_N);
  }
}

template <int KIND, int NSTEP, bool PROF>
cudaError_t launch_ws_one(const Common& c, const Batch& b, const unsigned char* qtc, int ngroups, int grid, int ns,
                          size_t smem, cudaStream_t st) {
  static thread_local size_t cfg = 0;
  if (cfg < smem) {
    const cudaError_t e = cudaFuncSetAttribute(k_mfilter_ws<KIND, NSTEP, PROF>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cfg = smem;
  }
  k_mfilter_ws<KIND, NSTEP, PROF><<<grid, WS_THREADS, smem, st>>>(c, b, qtc, ngroups, ns);
  return cudaGetLastError();
}

// K steps of the MMA loop: the padded dimension in 32-byte steps, compiled for
// the common cases (d <= 32, d <= 56 for TF32) and for the full 64.
template <bool PROF>
cudaError_t launch_ws_prof(int kind, int d, const Common& c, const Batch& b, const unsigned char* qtc, int ngroups,
                           int grid, int ns, size_t smem, cudaStream_t st) {
  if (kind == TCK_TF32) {
    if (d <= 32) return launch_ws_one<TCK_TF32, 4, PROF>(c, b, qtc, ngroups, grid, ns, smem, st);
    if (d <= 56) return launch_ws_one<TCK_TF32, 7, PROF>(c, b, qtc, ngroups, grid, ns, smem, st);
    return launch_ws_one<TCK_TF32, 8, PROF>(c, b, qtc, ngroups, grid, ns, smem, st);
  }
  if (kind == TCK_BF16) {
    if (d <= 32) return launch_ws_one<TCK_BF16, 2, PROF>(c, b, qtc, ngroups, grid, ns, smem, st);
    return launch_ws_one<TCK_BF16, 4, PROF>(c, b, qtc, ngroups, grid, ns, smem, st);
  }
  if (d <= 32) return launch_ws_one<TCK_FP16, 2, PROF>(c, b, qtc, ngroups, grid, ns, smem, st);
  return launch_ws_one<TCK_FP16, 4, PROF>(c, b, qtc, ngroups, grid, ns, smem, st);
}

cudaError_t launch_mfilter_ws(int kind, const Common& c, const Batch& b, const unsigned char* qtc, int ngroups,
                              int grid, int ns, size_t smem, cudaStream_t st) {
  return b.wst ? launch_ws_prof<true>(kind, c.d, c, b, qtc, ngroups, grid, ns, smem, st)
               : launch_ws_prof<false>(kind, c.d, c, b, qtc, ngroups, grid, ns, smem, st);
}

// Entries of a workspace's undecided-pair list (8 bytes each): 16,777,216, or
// the value of the environment variable RMIPS_PAIR_LIST_CAP (at least 64) when
// a workspace is created.  A pass that finds more undecided pairs is run
// again in smaller passes by the synchronous calls.
int64_t pair_list_cap() {
  const char* v = getenv("RMIPS_PAIR_LIST_CAP");
  long long c = v ? atoll(v) : 0;
  if (c <= 0) return 16ll << 20;
  return c < 64 ? 64 : c;
}

rmips_status ensure_batch(rmips_index* idx, Workspace* ws, int64_t cap_y) {
  if (!ws->bq) {
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->bq, (size_t)MQ_SLOTS * idx->d * sizeof(float)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->bk, MQ_SLOTS * sizeof(int32_t)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->bqn, MQ_SLOTS * sizeof(float)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->beps, MQ_SLOTS * sizeof(float)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->bidx, MQ_SLOTS * sizeof(int32_t)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->grp, (RMIPS_KMAX_LIMIT + 2) * sizeof(int4)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->qcnt, MQ_MAXQ * sizeof(int32_t)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->qcur, MQ_MAXQ * sizeof(int32_t)));
    ws->cap_t = pair_list_cap();
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->tpairs, ws->cap_t * sizeof(unsigned long long)));
  }
  if (!ws->bitems && idx->d <= (int)TC_K) {
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->bcq, (size_t)MQ_SLOTS * sizeof(float2)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->bitems, (size_t)MQ_ITEMS * ws_pack_bytes(8)));   // the largest item
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->gitem, (RMIPS_KMAX_LIMIT + 2) * sizeof(int)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->itemg, (size_t)MQ_ITEMS * sizeof(int2)));
  }
  if (!ws->wst) RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->wst, WST_N * sizeof(unsigned long long)));
  if (ws->cap_gpre < idx->nb * idx->k_max) {
    cudaFree(ws->gpre);
    ws->gpre = nullptr;
    ws->cap_gpre = 0;
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->gpre, (size_t)idx->nb * idx->k_max * sizeof(int32_t)));
    ws->cap_gpre = idx->nb * idx->k_max;
  }
  if (!ws->keys) {
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->keys, MQ_MAXQ * sizeof(unsigned long long)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->runs, MQ_MAXQ * sizeof(unsigned long long)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->hist, (RMIPS_KMAX_LIMIT + 2) * sizeof(int)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->gfirst, (RMIPS_KMAX_LIMIT + 2) * sizeof(int)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->gslot0, (RMIPS_KMAX_LIMIT + 2) * sizeof(int)));
  }
  if (!ws->big) {
    const int64_t nw = idx->n / 32 + 1;
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->big, MQ_MAXQ * sizeof(int32_t)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->mid, MQ_MAXQ * sizeof(int32_t)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->bslot, MQ_MAXQ * sizeof(int32_t)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->bigcnt, (size_t)MQ_BIG_SLOTS * ((nw + 1023) / 1024) * sizeof(int)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->bigmaps, (size_t)MQ_BIG_SLOTS * nw * sizeof(uint32_t)));
    RMIPS_TRY_CUDA(cudaMemset(ws->bigmaps, 0, (size_t)MQ_BIG_SLOTS * nw * sizeof(uint32_t)));
  }
  if (cap_y < 4096) cap_y = 4096;
  if (ws->cap_y < cap_y) {
    cudaFree(ws->ypairs); cudaFree(ws->seg);
    ws->ypairs = nullptr; ws->seg = nullptr; ws->cap_y = 0;
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->ypairs, cap_y * sizeof(unsigned long long)));
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->seg, cap_y * sizeof(int32_t)));
    ws->cap_y = cap_y;
  }
  return RMIPS_OK;
}

template <class T, bool FULLP>
cudaError_t launch_mfilter(const Common& c, const Batch& b, int ngroups, int grid, size_t smem, cudaStream_t st) {
  static thread_local bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_mfilter<T, FULLP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k_mfilter<T, FULLP><<<grid, MQ_THREADS, smem, st>>>(c, b, ngroups);
  return cudaGetLastError();
}

cudaError_t mfilter_dispatch(const rmips_index* idx, const Common& c, const Batch& b, int ngroups, int grid,
                             size_t smem, cudaStream_t st) {
  const bool fp = idx->full_p != 0;
  switch (idx->precision) {
    case RMIPS_BF16:
      return fp ? launch_mfilter<__nv_bfloat16, true>(c, b, ngroups, grid, smem, st)
                : launch_mfilter<__nv_bfloat16, false>(c, b, ngroups, grid, smem, st);
    case RMIPS_FP16:
      return fp ? launch_mfilter<__half, true>(c, b, ngroups, grid, smem, st)
                : launch_mfilter<__half, false>(c, b, ngroups, grid, smem, st);
    default:
      return fp ? launch_mfilter<float, true>(c, b, ngroups, grid, smem, st)
                : launch_mfilter<float, false>(c, b, ngroups, grid, smem, st);
  }
}

// Batched run over queries [0, nq) staged in ws->dq / ws->dk; ws->doffs gets
// the nq + 1 absolute offsets, results go to `out`.
rmips_status ensure_segments(Workspace* ws, int64_t nq) {
  if (ws->cap_seg >= nq) return RMIPS_OK;
  cudaFree(ws->dseglo);
  cudaFree(ws->dseghi);
  ws->dseglo = ws->dseghi = nullptr;
  ws->cap_seg = 0;
  const int64_t cap = nq < 1024 ? 1024 : nq;
  RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->dseglo, cap * sizeof(long long)));
  RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->dseghi, cap * sizeof(long long)));
  ws->cap_seg = cap;
  return RMIPS_OK;
}

// Captures what `enqueue` puts on capture stream cs into an executable graph;
// false (and nothing kept) if any step of the capture fails.
template <class F>
bool capture_graph(cudaStream_t cs, F&& enqueue, cudaGraphExec_t* exec) {
  *exec = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
  enqueue(cs);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    if (*exec) cudaGraphExecDestroy(*exec);
    *exec = nullptr;
    cudaGetLastError();                            // clear the capture error
    return false;
  }
  return true;
}

rmips_status run_batch(rmips_index* idx, Workspace* ws, int64_t nq, long long* out, long long capacity,
                       cudaStream_t st, const long long* dseglo, const long long* dseghi, int pass_max = MQ_MAXQ) {
  ws->ctr_dirty = true;
  Common c = make_common(idx, ws);
  static thread_local int sm_count = 0;
  if (!sm_count) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (sm_count <= 0) sm_count = 1;
  }
  int64_t want_y = capacity < (int64_t)nq * idx->n ? capacity : (int64_t)nq * idx->n;
  // plus the slots the tensor-core filter's epilogue warps reserve but leave unused
  rmips_status s = ensure_batch(idx, ws, want_y + 1 + (int64_t)sm_count * WS_EPI * WS_CHUNK_Y);
  if (s != RMIPS_OK) return s;
  RMIPS_TRY_CUDA(cudaMemsetAsync(ws->ctr, 0, C_NCOUNTERS * sizeof(long long), st));
  if (idx->prof_on == 2) RMIPS_TRY_CUDA(cudaMemsetAsync(ws->wst, 0, WST_N * sizeof(unsigned long long), st));
  const int ngroups_max = idx->k_max;
  const bool use_tc = idx->batch_tc && idx->d <= (int)TC_K && idx->Qtc;
  const int tck = idx->precision == RMIPS_BF16 ? TCK_BF16 : (idx->precision == RMIPS_FP16 ? TCK_FP16 : TCK_TF32);
  const size_t smem = (size_t)idx->d * (MQ_US + MQ_QS) * sizeof(float) + (size_t)ngroups_max * MQ_TU * sizeof(float2);
  int ws_ns = max_batch_stages(idx);      // query stages that fit beside the user tiles and bounds
  if (idx->tune_ws_ns > 0 && idx->tune_ws_ns < ws_ns) ws_ns = idx->tune_ws_ns;   // the autotuner's choice
  ws_ns -= ws_ns % WS_NMMA;               // a multiple of the MMA warps: each owns fixed stages
  if (ws_ns < WS_NMMA) ws_ns = WS_NMMA;
  const size_t smem_ws = ws_smem_bytes(tck, ws_ns);
  const int64_t tc_tiles = (idx->n + TCU - 1) / TCU;
  const int tc_grid = (int)(tc_tiles < sm_count ? tc_tiles : sm_count);
  int64_t per_sm = (int64_t)(228 * 1024) / (int64_t)(smem + 4096);
  if (per_sm > 4) per_sm = 4;
  if (per_sm < 1) per_sm = 1;
  const int64_t tiles = (idx->n + MQ_TU - 1) / MQ_TU;
  const int fgrid = (int)(tiles < sm_count * per_sm ? tiles : sm_count * per_sm);
  if (pass_max < 1 || pass_max > MQ_MAXQ) pass_max = MQ_MAXQ;
  for (int64_t j0 = 0; j0 < nq; j0 += pass_max) {
    const int cnt = (int)((nq - j0) < pass_max ? (nq - j0) : pass_max);
    Batch b;
    memset(&b, 0, sizeof(b));                      // padding too: graph keys compare the bytes
    b.dq = ws->dq + j0 * idx->d;
    b.dk = ws->dk + j0;
    b.dqn = ws->dqn + j0;
    b.deps = ws->deps + j0;
    b.nq = cnt;
    b.bq = ws->bq; b.bk = ws->bk; b.bqn = ws->bqn; b.beps = ws->beps; b.bidx = ws->bidx; b.grp = ws->grp;
    b.qcnt = ws->qcnt; b.qcur = ws->qcur;
    b.ypairs = ws->ypairs; b.cap_y = ws->cap_y;
    b.tpairs = ws->tpairs; b.cap_t = ws->cap_t;
    b.seg = ws->seg;
    b.tc_kind = tck;
    b.bcq = use_tc ? ws->bcq : nullptr;
    b.bitems = use_tc ? ws->bitems : nullptr;
    b.gitem = use_tc ? ws->gitem : nullptr;
    b.itemg = use_tc ? ws->itemg : nullptr;
    b.gpre = ws->gpre;
    b.wst = idx->prof_on == 2 ? ws->wst : nullptr;
    b.keys = ws->keys;
    b.runs = ws->runs;
    b.hist = ws->hist;
    b.gfirst = ws->gfirst;
    b.gslot0 = ws->gslot0;
    b.seglo = dseglo ? dseglo + j0 : nullptr;
    b.seghi = dseghi ? dseghi + j0 : nullptr;
    b.big = ws->big;
    b.mid = ws->mid;
    b.bslot = ws->bslot;
    b.bigmaps = ws->bigmaps;
    b.bigcnt = ws->bigcnt;
    b.nw = idx->n / 32 + 1;
    b.nwc = (b.nw + 1023) / 1024;
    b.doffs = ws->doffs + j0;
    b.out = out;
    b.capacity = capacity;
    const int nruns = (cnt + RUN - 1) / RUN;
    auto pre = [&](cudaStream_t q) {
      cudaMemsetAsync(b.hist, 0, (RMIPS_KMAX_LIMIT + 2) * sizeof(int), q);
      k_mprep_a<<<(cnt * 8 + 255) / 256, 256, 0, q>>>(c, b, idx->precision);
      k_mprep_groups<<<1, 256, 0, q>>>(c, b);
      k_mprep_runs<<<nruns, RUN, 0, q>>>(b);
      k_mprep_place<<<nruns, RUN, 0, q>>>(c, b, nruns);
      if (!use_tc) k_mprep_c<<<sm_count * 4, 256, 0, q>>>(c, b);
      if (use_tc) k_mprep_items<<<MQ_ITEMS, 256, 0, q>>>(c, b);
      if (use_tc) k_mprefix<<<(unsigned)((idx->nb + 255) / 256), 256, 0, q>>>(c, b, ngroups_max);
    };
    auto post = [&](cudaStream_t q) {
      k_mresolve<<<sm_count * 4, 256, 0, q>>>(c, b);     // 64 registers: four CTAs per SM, one wave
      k_mscan<<<1, 1024, 0, q>>>(c, b);
      k_mscatter<<<sm_count * 4, 256, 0, q>>>(c, b);
      k_memit<<<(cnt + MEMIT_Q - 1) / MEMIT_Q, 256, 0, q>>>(c, b);
      k_memit_mid<<<sm_count * 4, 256, 0, q>>>(c, b);
      k_mbig_mark<<<sm_count * 4, 256, 0, q>>>(c, b);
      k_mbig_count<<<sm_count * 4, 256, 0, q>>>(c, b);
      k_mbig_write<<<sm_count * 4, 256, 0, q>>>(c, b);
      k_memit_big<<<MQ_BIG_SLOTS, 1024, 0, q>>>(c, b);
    };
    // replay the pass's graphs when every kernel argument is as captured
    const int pass = (int)(j0 / pass_max);
    if ((int)ws->pgraph.size() <= pass) ws->pgraph.resize(pass + 1);
    Workspace::PassGraph& pg = ws->pgraph[pass];
    std::vector<unsigned char> key(sizeof(Common) + sizeof(Batch) + 4 * sizeof(int));
    const int extra[4] = {cnt, use_tc ? 1 : 0, sm_count, ngroups_max};
    memcpy(key.data(), &c, sizeof(Common));
    memcpy(key.data() + sizeof(Common), &b, sizeof(Batch));
    memcpy(key.data() + sizeof(Common) + sizeof(Batch), extra, sizeof(extra));
    // (a pass seen for the first time runs directly; the second identical one
    // is captured, so a stream of differing batches never pays for captures)
    if (key != pg.key) {
      if (pg.pre) cudaGraphExecDestroy(pg.pre);
      if (pg.post) cudaGraphExecDestroy(pg.post);
      pg.pre = pg.post = nullptr;
      pg.failed = false;
      pg.key = key;
    } else if (!pg.pre && !pg.failed) {
      if (!ws->cap_stream) RMIPS_TRY_CUDA(cudaStreamCreateWithFlags(&ws->cap_stream, cudaStreamNonBlocking));
      if (!(capture_graph(ws->cap_stream, pre, &pg.pre) && capture_graph(ws->cap_stream, post, &pg.post))) {
        if (pg.pre) cudaGraphExecDestroy(pg.pre);
        if (pg.post) cudaGraphExecDestroy(pg.post);
        pg.pre = pg.post = nullptr;
        pg.failed = true;
      }
    }
    if (pg.pre) RMIPS_TRY_CUDA(cudaGraphLaunch(pg.pre, st));
    else pre(st);
    RMIPS_TRY_CUDA(cudaGetLastError());
    const bool prof = idx->prof_on != 0;
    if (prof) {
      while ((int64_t)ws->ev.size() < 2 * (ws->ev_used + 1)) {
        cudaEvent_t ev;
        RMIPS_TRY_CUDA(cudaEventCreate(&ev));
        ws->ev.push_back(ev);
      }
      RMIPS_TRY_CUDA(cudaEventRecord(ws->ev[2 * ws->ev_used], st));
    }
    if (use_tc) {
      RMIPS_TRY_CUDA(launch_mfilter_ws(tck, c, b, idx->Qtc, ngroups_max, tc_grid, ws_ns, smem_ws, st));
    } else {
      RMIPS_TRY_CUDA(mfilter_dispatch(idx, c, b, idx->k_max, fgrid, smem, st));
    }
    if (prof) {
      RMIPS_TRY_CUDA(cudaEventRecord(ws->ev[2 * ws->ev_used + 1], st));
      ws->ev_used++;
    }
    if (pg.post) RMIPS_TRY_CUDA(cudaGraphLaunch(pg.post, st));
    else post(st);
    RMIPS_TRY_CUDA(cudaGetLastError());
  }
  return RMIPS_OK;
}

}  // namespace
}  // namespace rmips

using namespace rmips;

extern "C" rmips_status rmips_query(rmips_index* idx, const float* q, int32_t k, const rmips_segment* seg,
                                    int64_t* out_ids, int64_t capacity, int64_t* out_count, void* stream) {
  if (!idx || !q || !out_count || (!out_ids && capacity > 0) || capacity < 0) {
    set_error("null argument or negative capacity");
    return RMIPS_ERR_ARG;
  }
  if (k < 1 || k > idx->k_max) { set_error("k outside [1, k_max]"); return RMIPS_ERR_K_RANGE; }
  rmips_status s = check_segment(idx, seg);
  if (s != RMIPS_OK) return s;
  if ((s = check_ptr_device(q, idx->device, "q")) != RMIPS_OK) return s;
  if (capacity > 0 && (s = check_ptr_device(out_ids, idx->device, "out_ids")) != RMIPS_OK) return s;
  DeviceGuard dg(idx->device);
  cudaStream_t st = (cudaStream_t)stream;
  s = RMIPS_OK;
  Workspace* ws = acquire_workspace(idx, &s);
  if (!ws) return s;
  WsGuard g{idx, ws};
  if ((s = ws_join(ws, st)) != RMIPS_OK) return s;
  if ((s = ensure_queries(idx, ws, 1)) != RMIPS_OK) return s;
  if (idx->full_p && (!seg || seg->kind != 2)) {
    s = query_fused(idx, ws, q, k, seg, out_ids, capacity, out_count, st);
    if (s != RMIPS_ERR_INTERNAL) return s;      // internal: fall through to the multi-kernel path
  }
  const bool out_dev = capacity > 0 && is_device_ptr(out_ids);
  long long* out;
  if (out_dev) out = (long long*)out_ids;
  else if (capacity <= ws->cap_hout) out = ws->h_out;            // device-mapped pinned host memory
  else {
    if ((s = ensure_dout(ws, capacity)) != RMIPS_OK) return s;
    out = ws->dout;
  }
  RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->dq, q, idx->d * sizeof(float),
                                 is_device_ptr(q) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->dk, &k, sizeof(int32_t), cudaMemcpyHostToDevice, st));
  if ((s = run_queries(idx, ws, 1, seg, out, capacity, st)) != RMIPS_OK) return s;
  RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->h_ctr, ws->ctr, C_NCOUNTERS * sizeof(long long), cudaMemcpyDeviceToHost, st));
  RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->h_offs, ws->doffs, 2 * sizeof(long long), cudaMemcpyDeviceToHost, st));
  RMIPS_TRY_CUDA(cudaStreamSynchronize(st));
  const long long count = ws->h_offs[1];
  *out_count = count;
  record_stats(idx, ws, ws->h_ctr, 1);
  {
    std::lock_guard<std::mutex> lk(idx->mu);
    idx->last_stats.result = count;
  }
  if ((s = status_from_device(ws->h_ctr[C_STATUS])) != RMIPS_OK) return s;
  if (!out_dev && count > 0) {
    if (out == ws->h_out) memcpy(out_ids, ws->h_out, count * sizeof(long long));
    else RMIPS_TRY_CUDA(cudaMemcpy(out_ids, ws->dout, count * sizeof(long long), cudaMemcpyDeviceToHost));
  }
  return RMIPS_OK;
}

namespace rmips {
namespace {
// Results of a batch (the first min(total, cap) ids; nothing after a failed
// pass) from the device buffer into device-mapped pinned host memory, 16 bytes
// per store.
__global__ void k_copy_results(const long long* __restrict__ src, long long* __restrict__ dst,
                               const long long* __restrict__ ctr, long long cap) {
  if (ctr[C_STATUS] != 0) return;
  const long long n = ctr[C_CURSOR] < cap ? ctr[C_CURSOR] : cap;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const longlong2* s2 = reinterpret_cast<const longlong2*>(src);
  longlong2* d2 = reinterpret_cast<longlong2*>(dst);
  for (long long i = t; i < n / 2; i += stride) d2[i] = s2[i];
  if (t == 0 && (n & 1)) dst[n - 1] = src[n - 1];
}

}  // namespace
}  // namespace rmips

extern "C" rmips_status rmips_query_batch(rmips_index* idx, const float* qs, int64_t nq, const int32_t* ks,
                                          const rmips_segment* segs, int64_t* out_ids, int64_t capacity,
                                          int64_t* out_offsets, void* stream) {
  if (!idx || nq < 0 || (nq > 0 && (!qs || !ks)) || !out_offsets || capacity < 0 || (!out_ids && capacity > 0)) {
    set_error("null argument or negative size");
    return RMIPS_ERR_ARG;
  }
  out_offsets[0] = 0;
  if (nq == 0) return RMIPS_OK;
  rmips_status s = RMIPS_OK;
  if ((s = check_ptr_device(qs, idx->device, "qs")) != RMIPS_OK) return s;
  if ((s = check_ptr_device(ks, idx->device, "ks")) != RMIPS_OK) return s;
  if (capacity > 0 && (s = check_ptr_device(out_ids, idx->device, "out_ids")) != RMIPS_OK) return s;
  if (segs)
    for (int64_t j = 0; j < nq; ++j)
      if ((s = check_segment(idx, &segs[j])) != RMIPS_OK) return s;
  if (!is_device_ptr(ks)) {
    for (int64_t j = 0; j < nq; ++j)
      if (ks[j] < 1 || ks[j] > idx->k_max) { set_error("k outside [1, k_max]"); return RMIPS_ERR_K_RANGE; }
  }
  DeviceGuard dg(idx->device);
  cudaStream_t st = (cudaStream_t)stream;
  Workspace* ws = acquire_workspace(idx, &s);
  if (!ws) return s;
  WsGuard g{idx, ws};
  if ((s = ws_join(ws, st)) != RMIPS_OK) return s;
  if ((s = ensure_queries(idx, ws, nq)) != RMIPS_OK) return s;
  const bool out_dev = capacity > 0 && is_device_ptr(out_ids);
  // host results: the emitters write a device buffer; one coalesced copy
  // kernel then streams it into device-mapped pinned memory (no second
  // device-to-host transfer after the sizes are known), and the host copies
  // that into the caller's buffer
  const bool out_mapped = !out_dev && capacity <= ws->cap_hout;
  long long* out;
  if (out_dev) out = (long long*)out_ids;
  else {
    if ((s = ensure_dout(ws, capacity)) != RMIPS_OK) return s;
    out = ws->dout;
  }
  if ((s = stage_inputs(idx, ws, qs, nq, ks, st)) != RMIPS_OK) return s;
  bool ranges_only = true;
  if (segs)
    for (int64_t j = 0; j < nq; ++j) ranges_only = ranges_only && segs[j].kind != 2;
  bool batched = ranges_only;
  const long long* dlo = nullptr;
  const long long* dhi = nullptr;
  if (batched && segs) {
    if ((s = ensure_segments(ws, nq)) != RMIPS_OK) return s;
    std::vector<long long> lo(nq), hi(nq);
    for (int64_t j = 0; j < nq; ++j) {
      lo[j] = segs[j].kind == 1 ? segs[j].begin : 0;
      hi[j] = segs[j].kind == 1 ? segs[j].end : INT64_MAX;
    }
    RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->dseglo, lo.data(), nq * sizeof(long long), cudaMemcpyHostToDevice, st));
    RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->dseghi, hi.data(), nq * sizeof(long long), cudaMemcpyHostToDevice, st));
    RMIPS_TRY_CUDA(cudaStreamSynchronize(st));        // lo / hi leave scope
    dlo = ws->dseglo;
    dhi = ws->dseghi;
  }
  // A pass whose undecided pairs overflow the pair list is run again with
  // passes of half the size; below 64 queries per pass the batch goes
  // through the per-query path, whose lists hold every user.
  for (int pass_max = MQ_MAXQ;;) {
    if (batched) {
      if ((s = run_batch(idx, ws, nq, out, capacity, st, dlo, dhi, pass_max)) != RMIPS_OK) return s;
    } else {
      if ((s = run_queries(idx, ws, nq, segs, out, capacity, st)) != RMIPS_OK) return s;
    }
    if (out_mapped && capacity > 0) {
      k_copy_results<<<256, 256, 0, st>>>(ws->dout, ws->h_out, ws->ctr, capacity);
      RMIPS_TRY_CUDA(cudaGetLastError());
    }
    RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->h_ctr, ws->ctr, C_NCOUNTERS * sizeof(long long), cudaMemcpyDeviceToHost, st));
    RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->h_offs, ws->doffs, (nq + 1) * sizeof(long long), cudaMemcpyDeviceToHost, st));
    RMIPS_TRY_CUDA(cudaStreamSynchronize(st));
    if (!batched || ws->h_ctr[C_STATUS] != ST_PAIRS_FULL) break;
    ws->ev_used = 0;                                  // this attempt's filter timing is not kept
    pass_max = (int)((pass_max < nq ? pass_max : nq) / 2);
    if (pass_max < 64) batched = false;
  }
  for (int64_t j = 0; j <= nq; ++j) out_offsets[j] = ws->h_offs[j];
  record_stats(idx, ws, ws->h_ctr, nq, batched);
  {
    std::lock_guard<std::mutex> lk(idx->mu);
    idx->last_stats.result = ws->h_offs[nq];
  }
  if ((s = status_from_device(ws->h_ctr[C_STATUS])) != RMIPS_OK) return s;
  const long long total = ws->h_offs[nq];
  if (!out_dev && total > 0) {
    if (out_mapped) memcpy(out_ids, ws->h_out, (size_t)total * sizeof(long long));
    else RMIPS_TRY_CUDA(cudaMemcpy(out_ids, ws->dout, total * sizeof(long long), cudaMemcpyDeviceToHost));
  }
  return RMIPS_OK;
}

// ===========================================================================
// Allocation-free single query.
//
// Some callers cannot let a library call cudaMalloc: a framework whose caching
// allocator has already reserved the device's free memory (a cudaMalloc
// behind its back fails or fragments the pool), or a latency-critical serving
// thread (cudaMalloc / cudaFree can synchronise the whole device and stall
// every other stream).  rmips_query_noalloc serves them: its scratch lives in
// one file-scope device array of fixed size, created when the library is
// loaded, and the call allocates nothing -- no device, pinned-host or
// workspace-pool memory.
// ===========================================================================
namespace rmips {
namespace {

constexpr int64_t NA_MAX_USERS = 1 << 20;                          // largest |Q| served
constexpr size_t NA_CTR = 0;                                         // C_NCOUNTERS x int64
constexpr size_t NA_Q = 256;                                         // RMIPS_DMAX floats
constexpr size_t NA_K = NA_Q + RMIPS_DMAX * sizeof(float);           // one int32
constexpr size_t NA_QN = NA_K + 16;                                  // one float
constexpr size_t NA_EPS = NA_QN + 16;                                // one float
constexpr size_t NA_OFFS = NA_EPS + 16;                              // two int64
constexpr size_t NA_YES = NA_OFFS + 256;                             // NA_MAX_USERS x int32
constexpr size_t NA_TODO = NA_YES + NA_MAX_USERS * sizeof(int32_t);  // NA_MAX_USERS x int32
constexpr size_t NA_BITMAP = NA_TODO + NA_MAX_USERS * sizeof(int32_t);  // NA_MAX_USERS/32 + 1 words
constexpr size_t NA_BYTES = NA_BITMAP + (NA_MAX_USERS / 32 + 64) * sizeof(uint32_t);

static_assert(NA_CTR + C_NCOUNTERS * sizeof(long long) <= NA_Q, "counter block overflows");

// Shared by every call on a device; kept for the life of the process.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_base[64] = {};

// Device address of the scratch array for the current device (looked up once
// per device; the host-side symbol is only a stand-in, never a device address).
rmips_status noalloc_base(int dev, unsigned char** out) {
  if (dev < 0 || dev >= 64) { set_error("device ordinal out of range"); return RMIPS_ERR_ARG; }
  if (!g_noalloc_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      return RMIPS_ERR_CUDA;
    }
    g_noalloc_base[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_base[dev]);
  return RMIPS_OK;
}

}  // namespace

// Looks the scratch array up on the current device.  The library's device
// code is loaded lazily, module by module, on first use; this lookup makes the
// CUDA runtime load this module (and so create the array) when an index is
// built or loaded, not in the middle of the first allocation-free call.
rmips_status noalloc_prepare() {
  int dev = 0;
  RMIPS_TRY_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  unsigned char* base = nullptr;
  return noalloc_base(dev, &base);
}

}  // namespace rmips

extern "C" rmips_status rmips_query_noalloc(rmips_index* idx, const float* q, int32_t k, int64_t* out_ids,
                                            int64_t capacity, int64_t* out_count, void* stream) {
  if (!idx || !q || !out_count || capacity < 0 || (capacity > 0 && !out_ids)) {
    set_error("null argument or negative capacity");
    return RMIPS_ERR_ARG;
  }
  if (idx->n > NA_MAX_USERS) {
    set_error("rmips_query_noalloc serves at most 1048576 users (its fixed scratch size); use rmips_query");
    return RMIPS_ERR_ARG;
  }
  if (k < 1 || k > idx->k_max) { set_error("k outside [1, k_max]"); return RMIPS_ERR_K_RANGE; }
  if (check_ptr_device(q, idx->device, "q") != RMIPS_OK) return RMIPS_ERR_ARG;
  if (capacity > 0 && check_ptr_device(out_ids, idx->device, "out_ids") != RMIPS_OK) return RMIPS_ERR_ARG;
  if (capacity > 0 && !is_device_ptr(out_ids)) {
    set_error("rmips_query_noalloc writes ids to device memory only");
    return RMIPS_ERR_ARG;
  }
  DeviceGuard dg(idx->device);
  cudaStream_t st = (cudaStream_t)stream;
  // All calls share one scratch array: hold the lock until the GPU work is done.
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  int dev = 0;
  RMIPS_TRY_CUDA(cudaGetDevice(&dev));
  unsigned char* base = nullptr;
  rmips_status s = noalloc_base(dev, &base);
  if (s != RMIPS_OK) return s;
  // Declared after the lock, so destroyed before it is released: an error
  // return after work was queued waits for that work first, so that the
  // next call cannot find the array still in use.
  struct DrainOnExit {
    cudaStream_t st;
    bool armed = false;
    ~DrainOnExit() { if (armed) cudaStreamSynchronize(st); }
  } drain{st};
  drain.armed = true;

  Workspace ws;                                    // views into the scratch array, nothing owned
  ws.ctr = reinterpret_cast<long long*>(base + NA_CTR);
  ws.dq = reinterpret_cast<float*>(base + NA_Q);
  ws.dk = reinterpret_cast<int32_t*>(base + NA_K);
  ws.dqn = reinterpret_cast<float*>(base + NA_QN);
  ws.deps = reinterpret_cast<float*>(base + NA_EPS);
  ws.doffs = reinterpret_cast<long long*>(base + NA_OFFS);
  ws.yes = reinterpret_cast<int32_t*>(base + NA_YES);
  ws.todo = reinterpret_cast<int32_t*>(base + NA_TODO);
  ws.bitmap = reinterpret_cast<uint32_t*>(base + NA_BITMAP);
  // The array keeps the previous call's contents: clear what must start at zero.
  RMIPS_TRY_CUDA(cudaMemsetAsync(ws.ctr, 0, C_NCOUNTERS * sizeof(long long), st));
  RMIPS_TRY_CUDA(cudaMemsetAsync(ws.doffs, 0, 2 * sizeof(long long), st));
  RMIPS_TRY_CUDA(cudaMemsetAsync(ws.bitmap, 0, (idx->n / 32 + 1) * sizeof(uint32_t), st));
  RMIPS_TRY_CUDA(cudaMemcpyAsync(ws.dq, q, idx->d * sizeof(float),
                                 is_device_ptr(q) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  RMIPS_TRY_CUDA(cudaMemcpyAsync(ws.dk, &k, sizeof(int32_t), cudaMemcpyHostToDevice, st));

  Common c = make_common(idx, &ws);
  int sm_count = 1;
  cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = 512 + FW * 2 * 8 + (size_t)FW * 2 * 32 * idx->d * elem_bytes(idx->precision);
  const int64_t nchunks = (idx->n + 31) / 32;
  int64_t per_sm = (int64_t)(228 * 1024) / (int64_t)(smem + 1024);
  per_sm = per_sm > 8 ? 8 : (per_sm < 1 ? 1 : per_sm);
  const int64_t want = (nchunks + FW - 1) / FW;
  const int fgrid = (int)(want < sm_count * per_sm ? want : sm_count * per_sm);
  EmitArgs e{};
  e.seg_lo = 0;
  e.seg_hi = INT64_MAX;
  e.segmask = nullptr;
  e.bitmap = ws.bitmap;
  e.out = reinterpret_cast<long long*>(out_ids);
  e.capacity = capacity;
  e.offs = ws.doffs;
  k_qprep<<<1, 32, 0, st>>>(c, 1, idx->precision);
  RMIPS_TRY_CUDA(cudaGetLastError());
  RMIPS_TRY_CUDA(filter_dispatch(idx, c, 0, fgrid, smem, st));
  k_resolve<<<sm_count, 256, 0, st>>>(c, 0);
  k_emit<<<1, EMIT_THREADS, 0, st>>>(c, e, 0);
  RMIPS_TRY_CUDA(cudaGetLastError());
  long long h[C_NCOUNTERS];
  long long offs[2];
  RMIPS_TRY_CUDA(cudaMemcpyAsync(h, ws.ctr, sizeof(h), cudaMemcpyDeviceToHost, st));
  RMIPS_TRY_CUDA(cudaMemcpyAsync(offs, ws.doffs, sizeof(offs), cudaMemcpyDeviceToHost, st));
  RMIPS_TRY_CUDA(cudaStreamSynchronize(st));
  drain.armed = false;
  *out_count = offs[1];
  return status_from_device(h[C_STATUS]);
}

// Status and result count of an asynchronous batch call, written on the stream.
__global__ void k_batch_done(const long long* __restrict__ ctr, const long long* __restrict__ doffs, int64_t nq,
                             int64_t* __restrict__ done, unsigned long long* __restrict__ dprof) {
  const long long s = ctr[C_STATUS];
  done[0] = s == ST_OK ? RMIPS_OK
          : s == ST_NONFINITE ? RMIPS_ERR_NONFINITE
          : s == ST_CAPACITY ? RMIPS_ERR_CAPACITY
          : s == ST_TIMEOUT ? RMIPS_ERR_TIMEOUT
          : s == ST_K_RANGE ? RMIPS_ERR_K_RANGE
          : s == ST_PAIRS_FULL ? RMIPS_ERR_OOM : RMIPS_ERR_INTERNAL;
  done[1] = doffs[nq];
  if (dprof) atomicAdd(dprof, (unsigned long long)ctr[C_TESTED]);
}

extern "C" rmips_status rmips_query_batch_async(rmips_index* idx, const float* qs, int64_t nq, const int32_t* ks,
                                                int64_t* out_ids, int64_t capacity, int64_t* out_offsets,
                                                int64_t* done, void* stream) {
  if (!idx || nq < 0 || !out_offsets || !done || capacity < 0 || (nq > 0 && (!qs || !ks)) ||
      (!out_ids && capacity > 0)) {
    set_error("null argument or negative size");
    return RMIPS_ERR_ARG;
  }
  {
    const int dv = idx->device;
    const auto here = [dv](const void* p) { return ptr_class(p, dv) == PTR_DEVICE; };
    if (!here(out_offsets) || !here(done) || (nq > 0 && (!here(qs) || !here(ks))) || (capacity > 0 && !here(out_ids))) {
      set_error("rmips_query_batch_async takes device buffers of the index's GPU only");
      return RMIPS_ERR_ARG;
    }
  }
  DeviceGuard dg(idx->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (nq == 0) {
    RMIPS_TRY_CUDA(cudaMemsetAsync(out_offsets, 0, sizeof(int64_t), st));
    RMIPS_TRY_CUDA(cudaMemsetAsync(done, 0, 2 * sizeof(int64_t), st));
    return RMIPS_OK;
  }
  rmips_status s = RMIPS_OK;
  Workspace* ws = acquire_workspace(idx, &s);
  if (!ws) return s;
  WsGuard g{idx, ws};
  if ((s = ws_join(ws, st)) != RMIPS_OK) return s;
  if (!ws->done_ev) RMIPS_TRY_CUDA(cudaEventCreateWithFlags(&ws->done_ev, cudaEventDisableTiming));
  if ((s = ensure_queries(idx, ws, nq)) != RMIPS_OK) return s;
  if ((s = stage_inputs(idx, ws, qs, nq, ks, st)) != RMIPS_OK) return s;
  if ((s = run_batch(idx, ws, nq, (long long*)out_ids, capacity, st, nullptr, nullptr)) != RMIPS_OK) return s;
  RMIPS_TRY_CUDA(cudaMemcpyAsync(out_offsets, ws->doffs, (nq + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  k_batch_done<<<1, 1, 0, st>>>(ws->ctr, ws->doffs, nq, done, idx->prof_on ? idx->dprof : nullptr);
  RMIPS_TRY_CUDA(cudaGetLastError());
  if (ws->ev_used > 0) {                                 // filter timing: read when the profile is read
    std::lock_guard<std::mutex> lk(idx->mu);
    idx->pend_ev.insert(idx->pend_ev.end(), ws->ev.begin(), ws->ev.begin() + 2 * ws->ev_used);
    ws->ev.erase(ws->ev.begin(), ws->ev.begin() + 2 * ws->ev_used);
    ws->ev_used = 0;
  }
  RMIPS_TRY_CUDA(cudaEventRecord(ws->done_ev, st));
  ws->done_pending = true;
  ws->done_stream = st;
  return RMIPS_OK;
}

extern "C" rmips_status rmips_query_async(rmips_index* idx, const float* q, int32_t k, int64_t* out_ids,
                                          int64_t capacity, int64_t* done, void* stream) {
  if (!idx || !q || !done || capacity < 0 || (capacity > 0 && !out_ids)) {
    set_error("null argument or negative capacity");
    return RMIPS_ERR_ARG;
  }
  if (k < 1 || k > idx->k_max) { set_error("k outside [1, k_max]"); return RMIPS_ERR_K_RANGE; }
  {
    const int dv = idx->device;
    if (ptr_class(q, dv) != PTR_DEVICE || ptr_class(done, dv) != PTR_DEVICE ||
        (capacity > 0 && ptr_class(out_ids, dv) != PTR_DEVICE)) {
      set_error("rmips_query_async takes device buffers of the index's GPU only");
      return RMIPS_ERR_ARG;
    }
  }
  DeviceGuard dg(idx->device);
  cudaStream_t st = (cudaStream_t)stream;
  rmips_status s = RMIPS_OK;
  Workspace* ws = acquire_workspace(idx, &s);
  if (!ws) return s;
  WsGuard g{idx, ws};
  if ((s = ws_join(ws, st)) != RMIPS_OK) return s;
  if (!ws->done_ev) RMIPS_TRY_CUDA(cudaEventCreateWithFlags(&ws->done_ev, cudaEventDisableTiming));
  if (!ws->dres) RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->dres, (2 + C_NCOUNTERS) * sizeof(long long)));
  if ((s = ensure_queries(idx, ws, 1)) != RMIPS_OK) return s;
  const bool prof = idx->prof_on != 0 && idx->dprof1;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (prof) {
    RMIPS_TRY_CUDA(cudaEventCreate(&ev[0]));
    RMIPS_TRY_CUDA(cudaEventCreate(&ev[1]));
    RMIPS_TRY_CUDA(cudaEventRecord(ev[0], st));
  }
  if (idx->full_p) {
    if (ws->ctr_dirty) {                         // the one-launch kernel needs zero counters
      RMIPS_TRY_CUDA(cudaMemsetAsync(ws->ctr, 0, C_NCOUNTERS * sizeof(long long), st));
      ws->ctr_dirty = false;
    }
    Common c = make_common(idx, ws);
    EmitArgs e{};
    e.seg_lo = 0;
    e.seg_hi = INT64_MAX;
    e.bitmap = ws->bitmap;
    e.out = (long long*)out_ids;
    e.capacity = capacity;
    const cudaError_t err = q1_dispatch(idx, c, e, q, k, ws->dres, (long long*)done, prof ? idx->dprof1 : nullptr, st);
    if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return RMIPS_ERR_CUDA; }
  } else {                                       // P' index: the multi-kernel path of Algorithm 3
    RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->dq, q, idx->d * sizeof(float), cudaMemcpyDeviceToDevice, st));
    RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->dk, &k, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    const int64_t ev_before = ws->ev_used;
    if ((s = run_queries(idx, ws, 1, nullptr, (long long*)out_ids, capacity, st)) != RMIPS_OK) return s;
    ws->ev_used = ev_before;                     // timed by the pair around the call
    k_batch_done<<<1, 1, 0, st>>>(ws->ctr, ws->doffs, 1, done, nullptr);
    RMIPS_TRY_CUDA(cudaGetLastError());
  }
  if (prof) {
    RMIPS_TRY_CUDA(cudaEventRecord(ev[1], st));
    std::lock_guard<std::mutex> lk(idx->mu);
    idx->pend_ev1.push_back(ev[0]);
    idx->pend_ev1.push_back(ev[1]);
  }
  RMIPS_TRY_CUDA(cudaEventRecord(ws->done_ev, st));
  ws->done_pending = true;
  ws->done_stream = st;
  return RMIPS_OK;
}

extern "C" rmips_status rmips_debug_tc_tile(const float* A, const float* B, float* D, int32_t kind,
                                           void* stream) {
  if (kind < TCK_TF32 || kind > TCK_FP16) { set_error("bad kind"); return RMIPS_ERR_ARG; }
  if (!A || !B || !D) {
    set_error("null argument");
    return RMIPS_ERR_ARG;
  }
  {
    int dv = 0;
    RMIPS_TRY_CUDA(cudaGetDevice(&dv));
    if (ptr_class(A, dv) != PTR_DEVICE || ptr_class(B, dv) != PTR_DEVICE || ptr_class(D, dv) != PTR_DEVICE) {
      set_error("A, B and D must be device memory of the current GPU");
      return RMIPS_ERR_ARG;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  long long* status = nullptr;
  RMIPS_TRY_CUDA(cudaMallocAsync((void**)&status, sizeof(long long), st));
  RMIPS_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(long long), st));
  const int dsmem = (int)(192 * TC_K * 4);
  if (kind == TCK_TF32) {
    RMIPS_TRY_CUDA(cudaFuncSetAttribute(k_debug_tc<TCK_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem));
    k_debug_tc<TCK_TF32><<<1, 128, dsmem, st>>>(A, B, D, status);
  } else if (kind == TCK_BF16) {
    RMIPS_TRY_CUDA(cudaFuncSetAttribute(k_debug_tc<TCK_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem));
    k_debug_tc<TCK_BF16><<<1, 128, dsmem, st>>>(A, B, D, status);
  } else {
    RMIPS_TRY_CUDA(cudaFuncSetAttribute(k_debug_tc<TCK_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem));
    k_debug_tc<TCK_FP16><<<1, 128, dsmem, st>>>(A, B, D, status);
  }
  RMIPS_TRY_CUDA(cudaGetLastError());
  long long h = 0;
  RMIPS_TRY_CUDA(cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, st));
  RMIPS_TRY_CUDA(cudaFreeAsync(status, st));
  RMIPS_TRY_CUDA(cudaStreamSynchronize(st));
  return status_from_device(h);
}

namespace rmips {
// Entry points for the serving loop (same translation-unit-local machinery).
rmips_status batch_reserve(rmips_index* idx, Workspace* ws, int64_t nq) {
  rmips_status s = ensure_queries(idx, ws, nq);
  if (s != RMIPS_OK) return s;
  return ensure_segments(ws, nq);
}
rmips_status batch_launch(rmips_index* idx, Workspace* ws, int64_t nq, long long* out, long long capacity,
                          cudaStream_t st, bool with_segments) {
  return run_batch(idx, ws, nq, out, capacity, st, with_segments ? ws->dseglo : nullptr,
                   with_segments ? ws->dseghi : nullptr);
}
rmips_status device_status(long long s) { return status_from_device(s); }

// One query through the one-launch kernel on a workspace, device buffers
// (the serving loop's small batches): q (device, d floats), results to out
// (capacity ids), (status, count) to done.  Full-P indexes only.
rmips_status single_launch(rmips_index* idx, Workspace* ws, const float* q, int k, long long seg_lo,
                           long long seg_hi, long long* out, long long capacity, long long* done, cudaStream_t st) {
  if (!ws->dres) RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->dres, (2 + C_NCOUNTERS) * sizeof(long long)));
  if (ws->ctr_dirty) {                           // the one-launch kernel needs zero counters
    RMIPS_TRY_CUDA(cudaMemsetAsync(ws->ctr, 0, C_NCOUNTERS * sizeof(long long), st));
    ws->ctr_dirty = false;
  }
  Common c = make_common(idx, ws);
  EmitArgs e{};
  e.seg_lo = seg_lo;
  e.seg_hi = seg_hi;
  e.bitmap = ws->bitmap;
  e.out = out;
  e.capacity = capacity;
  const cudaError_t err = q1_dispatch(idx, c, e, q, k, ws->dres, done, nullptr, st);
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return RMIPS_ERR_CUDA; }
  return RMIPS_OK;
}

int max_batch_stages(const rmips_index* idx) {
  const int tck = idx->precision == RMIPS_BF16 ? TCK_BF16 : (idx->precision == RMIPS_FP16 ? TCK_FP16 : TCK_TF32);
  int ns = WS_MAXNS;
  while (ns > WS_NMMA && ws_smem_bytes(tck, ns) > 220 * 1024) --ns;
  return ns - ns % WS_NMMA;
}

int max_single_stages(const rmips_index* idx) {
  const size_t stage = q1_stage_bytes(idx->d, elem_bytes(idx->precision));
  int ns = (int)((220 * 1024 - Q1_HEAD - Q1_BUFS) / stage);
  return ns > Q1_MAXNS ? Q1_MAXNS : (ns < 1 ? 1 : ns);
}

rmips_status tune_time_batch(rmips_index* idx, const float* dq, const int32_t* dk, int64_t nq, int reps,
                             cudaStream_t st, float* ms) {
  rmips_status s = RMIPS_OK;
  Workspace* ws = acquire_workspace(idx, &s);
  if (!ws) return s;
  WsGuard g{idx, ws};
  if ((s = ws_join(ws, st)) != RMIPS_OK) return s;
  if ((s = ensure_queries(idx, ws, nq)) != RMIPS_OK) return s;
  const int64_t cap = idx->n * nq < (8ll << 20) ? idx->n * nq : (8ll << 20);
  if ((s = ensure_dout(ws, cap)) != RMIPS_OK) return s;
  if ((s = stage_inputs(idx, ws, dq, nq, dk, st)) != RMIPS_OK) return s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RMIPS_TRY_CUDA(cudaEventCreate(&e0));
  cudaError_t err = cudaEventCreate(&e1);
  for (int r = -1; err == cudaSuccess && r < reps; ++r) {       // run -1 is untimed
    if (r == 0) err = cudaEventRecord(e0, st);
    if (err == cudaSuccess && (s = run_batch(idx, ws, nq, ws->dout, cap, st, nullptr, nullptr)) != RMIPS_OK) break;
  }
  ws->ev_used = 0;
  if (err == cudaSuccess && s == RMIPS_OK) err = cudaEventRecord(e1, st);
  if (err == cudaSuccess && s == RMIPS_OK) err = cudaEventSynchronize(e1);
  float t = 0.f;
  if (err == cudaSuccess && s == RMIPS_OK) err = cudaEventElapsedTime(&t, e0, e1);
  long long status = 0;
  if (err == cudaSuccess && s == RMIPS_OK) err = cudaMemcpy(&status, &ws->ctr[C_STATUS], sizeof(status), cudaMemcpyDeviceToHost);
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s != RMIPS_OK) return s;
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return RMIPS_ERR_CUDA; }
  if (status != ST_OK && status != ST_CAPACITY) return status_from_device(status);
  *ms = t / (reps > 0 ? reps : 1);
  return RMIPS_OK;
}

rmips_status tune_time_single(rmips_index* idx, const float* dq, int64_t nq, int k, cudaStream_t st, float* ms) {
  rmips_status s = RMIPS_OK;
  Workspace* ws = acquire_workspace(idx, &s);
  if (!ws) return s;
  WsGuard g{idx, ws};
  if ((s = ws_join(ws, st)) != RMIPS_OK) return s;
  if (!ws->dres) RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->dres, (2 + C_NCOUNTERS) * sizeof(long long)));
  if ((s = ensure_dout(ws, idx->n)) != RMIPS_OK) return s;
  if (ws->ctr_dirty) {
    RMIPS_TRY_CUDA(cudaMemsetAsync(ws->ctr, 0, C_NCOUNTERS * sizeof(long long), st));
    ws->ctr_dirty = false;
  }
  Common c = make_common(idx, ws);
  EmitArgs e{};
  e.seg_lo = 0;
  e.seg_hi = INT64_MAX;
  e.bitmap = ws->bitmap;
  e.out = ws->dout;
  e.capacity = idx->n;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RMIPS_TRY_CUDA(cudaEventCreate(&e0));
  cudaError_t err = cudaEventCreate(&e1);
  const int warm = 4;
  for (int64_t i = 0; err == cudaSuccess && i < nq + warm; ++i) {
    if (i == warm) err = cudaEventRecord(e0, st);
    if (err == cudaSuccess)
      err = q1_dispatch(idx, c, e, dq + (size_t)((i < warm ? i : i - warm) % nq) * idx->d, k, ws->dres, nullptr,
                        nullptr, st);
  }
  if (err == cudaSuccess) err = cudaEventRecord(e1, st);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  float t = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
  long long status = 0;
  if (err == cudaSuccess) err = cudaMemcpy(&status, &ws->dres[RES_STATUS], sizeof(status), cudaMemcpyDeviceToHost);
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return RMIPS_ERR_CUDA; }
  if (status != ST_OK) {
    if (status == ST_TIMEOUT || status == ST_INTERNAL) ws->ctr_dirty = true;
    return status_from_device(status);
  }
  *ms = t / (float)nq;
  return RMIPS_OK;
}
}  // namespace rmips
