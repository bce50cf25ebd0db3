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

#include "rmips_internal.cuh"
#include "tc_common.cuh"

namespace rmips {
namespace {

constexpr float kInf = __builtin_huge_valf();
constexpr unsigned FULL = 0xffffffffu;
constexpr int FW = 4;                      // warps per filter CTA
constexpr int EMIT_THREADS = 1024;
constexpr int EMIT_SORT_CAP = 8192;

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
  for (int i = 0; i < d; ++i) {
    const float v = q[i];
    fin = fin && isfinite(v);
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
    if (k < 1 || k > c.k_max) atomicCAS((unsigned long long*)&c.ctr[C_STATUS], 0ull, (unsigned long long)ST_INTERNAL);
    c.dqn[j] = qn;
    c.deps[j] = eps;
  }
}

__device__ bool verify_scan(const float* __restrict__ u, float un, const Common& c, const float* sq, int k,
                            float qeps);
__device__ bool recheck_candidates(const float* __restrict__ u, const float* q, const int32_t* __restrict__ crow,
                                   const float* __restrict__ Ps, int d, int k, float cg32, long long* ctr);

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
                                ? recheck_candidates(u, sq, c.cand + p * RMIPS_KC, c.Ps, c.d, k, c.cg32, c.ctr)
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
                                   const float* __restrict__ Ps, int d, int k, float cg32, long long* ctr) {
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
  if (it >= 0) {
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
      yes = recheck_candidates(u, sq, c.cand + (int64_t)pos * RMIPS_KC, c.Ps, d, k, c.cg32, c.ctr);
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

// --- one launch per query (full-P index) ---------------------------------------------
// Every CTA forms ||q|| itself and runs the filter on its chunks; the last CTA
// to finish (a device-wide counter taken after a memory fence, nothing waits)
// rechecks the undecided users, sorts and writes the ids, copies the status,
// count and counters to `res` (device-visible host memory) and clears the
// counters for the next call.
constexpr int RES_STATUS = 0, RES_COUNT = 1, RES_CTR = 2;     // res layout: [2 + C_NCOUNTERS]

template <class T>
__global__ void __launch_bounds__(FW * 32) k_query1(Common c, EmitArgs e, const float* q_src, int k, int precision,
                                                     long long* res) {
  extern __shared__ __align__(128) unsigned char smem[];
  float* sq = reinterpret_cast<float*>(smem);                        // [RMIPS_DMAX]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 512);          // [FW][2]
  unsigned char* bufs = smem + 512 + FW * 2 * 8;                     // TMA buffers, later sort keys
  __shared__ float s_qn, s_eps;
  __shared__ int s_fin, s_last;
  __shared__ int s_warp[32];
  __shared__ long long s_total;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int d = c.d;
  for (int i = tid; i < d; i += blockDim.x) sq[i] = q_src[i];
  init_filter_barriers(bars);
  __syncthreads();
  if (tid == 0) s_fin = query_bounds(sq, d, precision, &s_qn, &s_eps) ? 1 : 0;
  __syncthreads();
  if (s_fin) filter_chunks<T, true, true>(c, sq, k, s_qn, s_eps, bars, bufs);
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd((unsigned long long*)&c.ctr[C_DONE], 1ull) == (unsigned long long)(gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  long long status = s_fin ? __ldcg(&c.ctr[C_STATUS]) : ST_NONFINITE;
  long long total = 0;
  if (status == 0) {
    // exact recheck of the undecided users: one warp per user
    const long long ntodo = __ldcg(&c.ctr[C_TODO]);
    for (long long t = warp; t < ntodo; t += FW) {
      const int32_t pos = __ldcg(&c.todo[t]);
      const float* u = c.Qs + (int64_t)pos * d;
      const bool yes = !c.incomp[pos]
                           ? recheck_candidates(u, sq, c.cand + (int64_t)pos * RMIPS_KC, c.Ps, d, k, c.cg32, c.ctr)
                           : verify_scan(u, c.unorm[pos], c, sq, k, s_eps);
      if (lane == 0 && yes) {
        const long long b = atomicAdd((unsigned long long*)&c.ctr[C_YES], 1ull);
        c.yes[b] = pos;
      }
    }
    __threadfence_block();
    __syncthreads();
    total = emit_block(c, e, __ldcg(&c.ctr[C_YES]), 0, reinterpret_cast<int32_t*>(bufs), s_warp, &s_total);
    if (total > e.capacity) status = ST_CAPACITY;
  }
  __syncthreads();
  if (tid == 0) {
    res[RES_STATUS] = status;
    res[RES_COUNT] = total;
    for (int i = 0; i < C_NCOUNTERS; ++i) {
      res[RES_CTR + i] = c.ctr[i];
      c.ctr[i] = 0;
    }
    c.ctr[C_DONE] = 0;
    __threadfence_system();
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
  Common c{};
  c.Qs = idx->Qs;
  c.Qrows = idx->precision == RMIPS_FP32 ? (const void*)idx->Qs : idx->Qh;
  c.Ps = idx->Ps;
  c.Lb = idx->Lb;
  c.LB = idx->LB;
  c.hdr = idx->hdr;
  c.unorm = idx->unorm;
  c.pnorm = idx->pnorm;
  c.cand = idx->cand;
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
    case ST_NONFINITE: set_error("non-finite value in a query"); return RMIPS_ERR_NONFINITE;
    case ST_CAPACITY: set_error("output capacity too small"); return RMIPS_ERR_CAPACITY;
    case ST_TIMEOUT: set_error("a device wait timed out"); return RMIPS_ERR_TIMEOUT;
    default: set_error("device-side consistency check failed"); return RMIPS_ERR_INTERNAL;
  }
}

template <class T>
cudaError_t launch_query1(const Common& c, const EmitArgs& e, const float* q, int k, int precision, long long* res,
                          int grid, size_t smem, cudaStream_t st) {
  static thread_local bool configured = false;
  if (!configured) {
    cudaError_t err = cudaFuncSetAttribute(k_query1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (err != cudaSuccess) return err;
    configured = true;
  }
  k_query1<T><<<grid, FW * 32, smem, st>>>(c, e, q, k, precision, res);
  return cudaGetLastError();
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
  static thread_local int sm_count = 0;
  if (!sm_count) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (sm_count <= 0) sm_count = 1;
  }
  size_t smem = 512 + FW * 2 * 8 + (size_t)FW * 2 * 32 * d * elem_bytes(idx->precision);
  const size_t smem_keys = 512 + FW * 2 * 8 + EMIT_SORT_CAP * sizeof(int32_t);
  if (smem < smem_keys) smem = smem_keys;
  const int64_t nchunks = (idx->n + 31) / 32;
  int64_t per_sm = (int64_t)(228 * 1024) / (int64_t)(smem + 1024);
  per_sm = per_sm > 8 ? 8 : (per_sm < 1 ? 1 : per_sm);
  const int64_t want = (nchunks + FW - 1) / FW;
  const int grid = (int)(want < sm_count * per_sm ? want : sm_count * per_sm);
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
  cudaError_t err;
  switch (idx->precision) {
    case RMIPS_BF16: err = launch_query1<__nv_bfloat16>(c, e, q_src, k, idx->precision, ws->h_res, grid, smem, st); break;
    case RMIPS_FP16: err = launch_query1<__half>(c, e, q_src, k, idx->precision, ws->h_res, grid, smem, st); break;
    default: err = launch_query1<float>(c, e, q_src, k, idx->precision, ws->h_res, grid, smem, st); break;
  }
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
    idx->prof.filter_alg_bytes += 8.0 * idx->nb + ((double)idx->d * es + 8.0) * h[C_TESTED] +
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
                                                  float* __restrict__ D, uint32_t lbo, uint32_t sbo,
                                                  long long* __restrict__ status) {
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
    for (uint32_t s = 0; s < TC_K * E / 32; ++s) {
      const uint64_t ad = tc_sdesc(smem_u32(sA) + s * 2 * TC_LBO, lbo, sbo);
      const uint64_t bd = tc_sdesc(smem_u32(sB) + s * 2 * TC_LBO, lbo, sbo);
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
  unsigned char* bqt;     // query tiles in the UMMA layout (TC path), may be null
  int bqt_kind;           // TCK_* of the tiles
  const long long* seglo;   // [nq] allowed id range per query (null: all users)
  const long long* seghi;
  unsigned long long* keys;  // [nq] sort keys
  unsigned long long* runs;  // [nruns * 1024] keys sorted in runs
  int* hist;              // [RMIPS_KMAX_LIMIT + 2] queries per k
  int* gfirst;            // [RMIPS_KMAX_LIMIT + 2] first sorted position of each k
  int* gslot0;            // [RMIPS_KMAX_LIMIT + 2] first slot of each k-group
  int32_t* big;           // queries with more than EMIT_SORT_CAP results
  uint32_t* bigmaps;      // MQ_BIG_SLOTS id bitmaps of nw words each
  int64_t nw;             // words per id bitmap
  long long* doffs;       // [nq + 1] offsets of this pass (absolute)
  long long* out;
  long long capacity;
};

// (a) per query: norm bound, slack, checks, sort key, k histogram.
__global__ void k_mprep_a(Common c, Batch b, int precision) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= b.nq) return;
  float qn, eps;
  const bool fin = query_bounds(b.dq + (int64_t)j * c.d, c.d, precision, &qn, &eps);
  int k = b.dk[j];
  if (!fin) set_status(c.ctr, ST_NONFINITE);
  if (k < 1 || k > c.k_max) { set_status(c.ctr, ST_INTERNAL); k = 1; }
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
  const int tid = threadIdx.x;
  if (tid == 0) {
    c.ctr[C_YES] = 0;
    c.ctr[C_TODO] = 0;
    c.ctr[C_NBIG] = 0;
    int f = 0, s = 0, g = 0;
    for (int k = 0; k <= RMIPS_KMAX_LIMIT + 1; ++k) {
      first[k] = f;
      slot0[k] = s;
      const int h = (k >= 1 && k <= RMIPS_KMAX_LIMIT) ? b.hist[k] : 0;
      if (h > 0) {
        const int tiles = (h + MQ_TQ - 1) / MQ_TQ;
        b.grp[g++] = make_int4(k, s, h, tiles);
        f += h;
        s += tiles * MQ_TQ;
      }
    }
    for (; g <= RMIPS_KMAX_LIMIT; ++g) b.grp[g] = make_int4(0, s, 0, 0);   // empty groups; .y = total slots
  }
  __syncthreads();
  if (tid < RMIPS_KMAX_LIMIT + 2) {
    b.gfirst[tid] = first[tid];
    b.gslot0[tid] = slot0[tid];
  }
  for (int k = 1; k <= RMIPS_KMAX_LIMIT; ++k) {
    const int h = b.hist[k];
    if (h == 0) continue;
    const int pad = ((h + MQ_TQ - 1) / MQ_TQ) * MQ_TQ;
    for (int r = h + tid; r < pad; r += blockDim.x) {
      b.bidx[slot0[k] + r] = -1;
      b.bk[slot0[k] + r] = k;
      b.bqn[slot0[k] + r] = 0.f;
      b.beps[slot0[k] + r] = 0.f;
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

// (d) grid: the final sorted position of each key is its position in its run
// plus, for every other run, the number of keys below it (keys are distinct),
// found by binary search; the position gives the query's slot in its k-group.
__global__ void k_mprep_place(Batch b, int nruns) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= (int64_t)nruns * RUN) return;
  const unsigned long long key = b.runs[g];
  if (key == ~0ull) return;                        // padding
  const int r = (int)(g / RUN);
  int64_t rank = g - (int64_t)r * RUN;
  for (int o = 0; o < nruns; ++o) {
    if (o == r) continue;
    const unsigned long long* run = b.runs + (int64_t)o * RUN;
    int lo = 0, hi = RUN;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (run[mid] < key) lo = mid + 1; else hi = mid;
    }
    rank += lo;
  }
  const int k = (int)(key >> 46);
  const int j = (int)(key & 16383ull);
  const int slot = b.gslot0[k] + (int)(rank - b.gfirst[k]);
  b.bidx[slot] = j;
  b.bk[slot] = k;
  b.bqn[slot] = b.dqn[j];
  b.beps[slot] = b.deps[j];
}

// (e) grid: gather the query vectors into slot order (zeros in padding), row
// major for the CUDA-core path and in 64-query UMMA tiles for tensor cores.
__global__ void k_mprep_c(Common c, Batch b) {
  const int total_slots = b.grp[RMIPS_KMAX_LIMIT].y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)total_slots * c.d; e += stride) {
    const int slot = (int)(e / c.d), i = (int)(e - (int64_t)slot * c.d);
    const int j = b.bidx[slot];
    b.bq[e] = j >= 0 ? b.dq[(int64_t)j * c.d + i] : 0.f;
  }
  if (b.bqt) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)total_slots * TC_K; e += stride) {
      const int slot = (int)(e / TC_K), k = (int)(e - (int64_t)slot * TC_K);
      const int j = b.bidx[slot];
      const float v = (j >= 0 && k < c.d) ? b.dq[(int64_t)j * c.d + k] : 0.f;
      const size_t tile = (size_t)(slot / MQ_TQ);
      if (b.bqt_kind == TCK_TF32) {
        reinterpret_cast<float*>(b.bqt + tile * (MQ_TQ * TC_K * 4) + tc_off(slot % MQ_TQ, k))[0] = v;
      } else {
        unsigned char* dst = b.bqt + tile * (MQ_TQ * TC_K * 2) + tc_off16(slot % MQ_TQ, k);
        if (b.bqt_kind == TCK_BF16) *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v);
        else *reinterpret_cast<__half*>(dst) = __float2half_rn(v);
      }
    }
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
                else set_status(c.ctr, ST_INTERNAL);
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
  const int lane = threadIdx.x & 31;
  const int d = c.d;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < cnt; t += nw) {
    const unsigned long long pr = b.tpairs[t];
    const int j = (int)(pr >> 32);
    const int32_t pos = (int32_t)(pr & 0xffffffffull);
    const float* q = b.dq + (int64_t)j * d;
    const int k = b.dk[j];
    const float* u = c.Qs + (int64_t)pos * d;
    bool yes;
    if (c.full_p && !c.incomp[pos]) {
      yes = recheck_candidates(u, q, c.cand + (int64_t)pos * RMIPS_KC, c.Ps, d, k, c.cg32, c.ctr);
    } else {
      yes = verify_scan(u, c.unorm[pos], c, q, k, b.deps[j]);
    }
    if (lane == 0 && yes) {
      const long long at = atomicAdd((unsigned long long*)&c.ctr[C_YES], 1ull);
      if (at < b.cap_y) b.ypairs[at] = ((unsigned long long)(uint32_t)j << 32) | (uint32_t)pos;
      atomicAdd(&b.qcnt[j], 1);
    }
  }
}

// Exclusive scan of per-query counts into absolute offsets.
__global__ void __launch_bounds__(1024) k_mscan(Common c, Batch b) {
  __shared__ long long s_warp[32];
  __shared__ long long s_base;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_base = c.ctr[C_CURSOR];
  __syncthreads();
  const int per = (b.nq + 1023) / 1024;
  const int j0 = tid * per, j1 = min(b.nq, j0 + per);
  long long local = 0;
  for (int j = j0; j < j1; ++j) local += b.qcnt[j];
  long long x = local;
  for (int o = 1; o < 32; o <<= 1) { long long y = __shfl_up_sync(FULL, x, o); if (lane >= o) x += y; }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long v = s_warp[lane];
    for (int o = 1; o < 32; o <<= 1) { long long y = __shfl_up_sync(FULL, v, o); if (lane >= o) v += y; }
    s_warp[lane] = v;
  }
  __syncthreads();
  long long run = s_base + (x - local) + (wid ? s_warp[wid - 1] : 0);
  for (int j = j0; j < j1; ++j) {
    b.doffs[j] = run;
    run += b.qcnt[j];
    if (b.qcnt[j] > EMIT_SORT_CAP) {
      const long long r = atomicAdd((unsigned long long*)&c.ctr[C_NBIG], 1ull);
      b.big[r] = j;
    }
  }
  __syncthreads();
  if (tid == 0) {
    const long long total = s_warp[31];
    b.doffs[b.nq] = s_base + total;
    c.ctr[C_CURSOR] = s_base + total;
    if (s_base + total > b.capacity) set_status(c.ctr, ST_CAPACITY);
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
    const int j = (int)(pr >> 32);
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

// Positions -> ids, ascending, for queries with at most EMIT_SORT_CAP results.
// A CTA serves 8 consecutive queries: a result of at most 32 ids is sorted by
// one warp in registers; a larger one by the whole CTA in shared memory.
constexpr int MEMIT_Q = 8;
__global__ void __launch_bounds__(256) k_memit(Common c, Batch b) {
  __shared__ int32_t keys[EMIT_SORT_CAP];
  if (c.ctr[C_STATUS] != 0) return;                      // uniform: read-only here
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long base0 = b.doffs[0];
  const int j0 = blockIdx.x * MEMIT_Q;
  {
    const int j = j0 + warp;
    if (j < b.nq) {
      const int cnt = b.qcnt[j];
      if (cnt > 0 && cnt <= 32) {
        const long long off = b.doffs[j];
        int32_t v = lane < cnt ? c.permQ[b.seg[off - base0 + lane]] : INT_MAX;
        v = warp_sort_asc(v);
        if (lane < cnt) b.out[off + lane] = v;
      }
    }
  }
  for (int w = 0; w < MEMIT_Q; ++w) {
    const int j = j0 + w;
    if (j >= b.nq) break;
    const int cnt = b.qcnt[j];
    if (cnt <= 32 || cnt > EMIT_SORT_CAP) continue;      // small: done above; large: k_memit_big
    const long long off = b.doffs[j];
    int N2 = 64;
    while (N2 < cnt) N2 <<= 1;
    __syncthreads();                                     // keys of the previous query consumed
    for (int i = tid; i < N2; i += blockDim.x)
      keys[i] = i < cnt ? c.permQ[b.seg[off - base0 + i]] : INT_MAX;
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
  }
}

// Queries with large results: each CTA owns one id bitmap and handles the
// large queries r = blockIdx.x, blockIdx.x + gridDim.x, ... in turn: set one
// bit per result id, then read the bitmap back in order (block-wide prefix of
// per-thread bit counts), clearing it for the next query.
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
  for (long long r = blockIdx.x; r < s_nbig; r += gridDim.x) {
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


// ===========================================================================
// Batched filter on tensor cores (TF32, d <= 64).
//
// Same work decomposition as k_mfilter: a CTA owns a tile of 128 users, finds
// the Lemma 3 prefix of every k-group for every block of the tile, and skips
// the tile when nothing survives.  The users are written once into shared
// memory in the UMMA layout (K padded to 64 with zeros); the surviving
// 64-query tiles (laid out the same way by k_mprep) arrive by 1-D TMA, one
// ahead.  Thread 0 issues the 8 tcgen05.mma (128 x 64 x 8, TF32 in, FP32
// accumulate in TMEM) of a tile; every thread owns one user row, copies its
// 64 accumulators from TMEM into registers, after which the next tile's MMA
// runs while the row is classified (Lemma 1, then hi_k / Lemma 2).
//
// Error bound of a TF32 inner product: each operand is within 2^-10 of its
// float32 value (10 fraction bits, any rounding), each product of two TF32
// values is exact in float32, and the float32 accumulation over K = 64 terms
// (8 chained MMAs) is charged 65 * 2^-22 relative to sum |a_i b_i|; with
// sum |a_i b_i| <= ||u|| ||q|| the bound is TC_ERR ||u|| ||q|| plus the
// slack of operands below the normal range.
// ===========================================================================
constexpr int TCU = 128;                       // users per tile (MMA M)
constexpr int TCQ = MQ_TQ;                     // queries per tile (MMA N)
constexpr int TC_THREADS = 256;                // 8 warps: warp w and w + 4 share TMEM lanes 32 (w % 4) ...
constexpr int TC_HALF = TCQ / 2;               // ... and split the 64 query columns in halves
__host__ __device__ constexpr uint32_t tc_esize(int kind) { return kind == TCK_TF32 ? 4u : 2u; }
__host__ __device__ constexpr uint32_t tc_tile_bytes(int kind) { return TCQ * TC_K * tc_esize(kind); }
__host__ __device__ constexpr uint32_t tc_a_bytes(int kind) { return TCU * TC_K * tc_esize(kind); }

template <int KIND>
__global__ void __launch_bounds__(TC_THREADS, 3) k_mfilter_tc(Common c, Batch b, const unsigned char* __restrict__ bqt,
                                                               int ngroups) {
  constexpr uint32_t TC_TILE_BYTES = tc_tile_bytes(KIND);   // one query tile
  constexpr uint32_t TC_A_BYTES = tc_a_bytes(KIND);         // one user tile
  constexpr uint32_t SBO = KIND == TCK_TF32 ? TC_SBO : TC_SBO16;
  constexpr uint32_t NSTEP = TC_K * tc_esize(KIND) / 32;    // MMAs per tile (32 bytes of K each)
  constexpr float TC_ERR = tc_rel_err(KIND);
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* sA = tsm;
  unsigned char* sB = tsm + TC_A_BYTES;                      // 2 query tiles
  __shared__ __align__(8) uint64_t bar_b[2];     // query tile landed
  __shared__ __align__(8) uint64_t bar_m;        // MMA done
  __shared__ uint32_t taddr_s;
  __shared__ float un_s[TCU];
  __shared__ float2 cq_s[2][TCQ];                // (error scale, absolute slack) per query of a tile
  __shared__ int qj_s[2][TCQ];
  __shared__ int pre[RMIPS_KMAX_LIMIT][4];
  __shared__ int gmax[RMIPS_KMAX_LIMIT];
  __shared__ int any_tile, s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int uu = tid & (TCU - 1);                // this thread's user row (TMEM lane)
  const int half = tid >> 7;                     // which 32 query columns
  const int d = c.d;
  const int64_t n = c.n;
  const int sub = c.bs < TCU ? c.bs : TCU;
  const int nbt = TCU / sub;
  const float un0 = c.unorm[0];                  // largest user norm (users are sorted)
  const float tiny = (d + 2) * tc_abs_unit(KIND);            // operands below the normal range

  if (warp == 0) {
    tmem_alloc(&taddr_s, 64);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar_b[0], 1);
    mbar_init(&bar_b[1], 1);
    mbar_init(&bar_m, 1);
    fence_mbar_init();
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = taddr_s;
  const uint32_t tlane = taddr + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(half * TC_HALF);
  const uint32_t idesc = KIND == TCK_TF32 ? tc_idesc_tf32(TCU, TCQ) : tc_idesc_f16(TCU, TCQ, KIND == TCK_BF16);
  auto mma = [&](uint32_t bbase) {                 // one 128 x 64 x 64 tile, thread 0
    for (uint32_t s = 0; s < NSTEP; ++s) {
      const uint64_t ad = tc_sdesc(smem_u32(sA) + s * 2 * TC_LBO, TC_LBO, SBO);
      const uint64_t bd = tc_sdesc(bbase + s * 2 * TC_LBO, TC_LBO, SBO);
      if (KIND == TCK_TF32) tc_mma_tf32(taddr, ad, bd, idesc, s > 0 ? 1u : 0u);
      else tc_mma_f16(taddr, ad, bd, idesc, s > 0 ? 1u : 0u);
    }
    tc_commit(&bar_m);
  };
  uint32_t phb = 0, ph_m = 0;                    // parity of the next wait: bit x for bar_b[x] / bar_m
  long long st_pairs = 0, st_skipped = 0, st_yes = 0, st_todo = 0;

  for (int64_t u0 = (int64_t)blockIdx.x * TCU; u0 < n && !s_fail; u0 += (int64_t)gridDim.x * TCU) {
    // 1. Lemma 3 prefixes
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
    if (!any_tile) {
      if (tid == 0) st_skipped += 1;
      continue;
    }
    const int64_t nvalid = (n - u0) < TCU ? (n - u0) : TCU;
    // 2. user tile into the UMMA layout: one 16-byte chunk (4 consecutive k of
    //    one row) per store, consecutive threads on consecutive rows
    if (KIND == TCK_TF32) {
      const float* src = c.Qs + u0 * d;
      for (int e = tid; e < TCU * (int)(TC_K / 4); e += TC_THREADS) {
        const int r = e & (TCU - 1), k0 = (e >> 7) * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < nvalid) {
          const float* row = src + (int64_t)r * d;
          if (k0 + 0 < d) v.x = row[k0 + 0];
          if (k0 + 1 < d) v.y = row[k0 + 1];
          if (k0 + 2 < d) v.z = row[k0 + 2];
          if (k0 + 3 < d) v.w = row[k0 + 3];
        }
        *reinterpret_cast<float4*>(sA + tc_off(r, k0)) = v;
      }
    } else {                                       // the index's 16-bit copy, 8 values per chunk
      const uint16_t* src = reinterpret_cast<const uint16_t*>(c.Qrows) + u0 * d;
      for (int e = tid; e < TCU * (int)(TC_K / 8); e += TC_THREADS) {
        const int r = e & (TCU - 1), k0 = (e >> 7) * 8;
        uint16_t h[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) h[i] = (r < nvalid && k0 + i < d) ? src[(int64_t)r * d + k0 + i] : (uint16_t)0;
        uint4 v;
        v.x = h[0] | ((uint32_t)h[1] << 16);
        v.y = h[2] | ((uint32_t)h[3] << 16);
        v.z = h[4] | ((uint32_t)h[5] << 16);
        v.w = h[6] | ((uint32_t)h[7] << 16);
        *reinterpret_cast<uint4*>(sA + tc_off16(r, k0)) = v;
      }
    }
    if (tid < TCU) un_s[tid] = tid < nvalid ? c.unorm[u0 + tid] : 0.f;
    if (tid == 0) {
      for (int g = 0; g < ngroups; ++g)
        for (int sb = 0; sb < nbt; ++sb) {
          const int64_t us = (int64_t)sb * sub;
          const int64_t cnt = nvalid - us < sub ? (nvalid - us > 0 ? nvalid - us : 0) : sub;
          st_pairs += (long long)pre[g][sb] * cnt;
        }
    }
    fence_proxy_async();
    // 3. walk the (group, query tile) items of this user tile
    int nitems = 0;
    for (int g = 0; g < ngroups; ++g) nitems += (gmax[g] + TCQ - 1) / TCQ;
    int g_ld = 0, t_ld = 0;                       // next item to load
    auto advance = [&](int& g, int& t) {
      ++t;
      while (g < ngroups && t >= (gmax[g] + TCQ - 1) / TCQ) { ++g; t = 0; }
    };
    while (g_ld < ngroups && gmax[g_ld] == 0) ++g_ld;
    auto load_item = [&](int g, int t, int buf) {
      const int s0 = b.grp[g].y + t * TCQ;
      if (tid == 0) {
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar_b[buf], TC_TILE_BYTES);
        bulk_g2s(sB + (size_t)buf * TC_TILE_BYTES, bqt + (size_t)(s0 / TCQ) * TC_TILE_BYTES, TC_TILE_BYTES,
                 &bar_b[buf]);
      }
      if (tid < TCQ) {
        const float qn = b.bqn[s0 + tid];
        cq_s[buf][tid] = make_float2(__fmul_ru(qn, TC_ERR), __fmaf_ru(__fadd_ru(qn, un0), tiny, b.beps[s0 + tid]));
        qj_s[buf][tid] = b.bidx[s0 + tid];
      }
    };
    int g_cur = g_ld, t_cur = 0;
    load_item(g_ld, 0, 0);
    advance(g_ld, t_ld);
    __syncthreads();                               // user tile written, constants of item 0 visible
    if (tid == 0) {                                // MMA(0)
      if (mbar_wait_bounded(&bar_b[0], phb & 1u)) {
        tc_fence_after();
        mma(smem_u32(sB));
      } else {
        s_fail = 1;
      }
    }
    phb ^= 1u;
    int g_L = -1;                                  // group whose bounds are in L
    float2 L = make_float2(kInf, kInf);
    for (int it = 0; it < nitems; ++it) {
      const int buf = it & 1;
      // A. prefetch the next query tile (its buffer's last reader, MMA(it-1), is done)
      const bool has_next = it + 1 < nitems;
      if (has_next) load_item(g_ld, t_ld, buf ^ 1);
      // B. wait for MMA(it); copy this thread's 32 accumulators out of TMEM
      bool ok = s_fail ? false : mbar_wait_bounded(&bar_m, ph_m);
      ph_m ^= 1u;
      ok = __syncthreads_and(ok && !s_fail);
      if (!ok) {
        if (tid == 0) s_fail = 1;
        break;
      }
      tc_fence_after();
      float acc[TC_HALF];
      tmem_ld16(tlane, acc);
      tmem_ld16(tlane + 16, acc + 16);
      tmem_ld_wait();
      if (g_cur != g_L) {                          // this user's (lo, hi) for the group's k
        L = uu < nvalid ? c.Lb[(int64_t)(b.grp[g_cur].x - 1) * n + u0 + uu] : make_float2(kInf, kInf);
        g_L = g_cur;
      }
      tc_fence_before();
      __syncthreads();                             // TMEM consumed; next constants visible
      // C. MMA(it + 1) overlaps the epilogue below
      if (has_next && tid == 0) {
        if (mbar_wait_bounded(&bar_b[buf ^ 1], (phb >> (buf ^ 1)) & 1u)) {
          tc_fence_after();
          mma(smem_u32(sB) + (uint32_t)(buf ^ 1) * TC_TILE_BYTES);
        } else {
          s_fail = 1;
        }
      }
      if (has_next) phb ^= 1u << (buf ^ 1);
      // D. epilogue: (this user, 32 queries of item it)
      int live = pre[g_cur][uu / sub] - t_cur * TCQ - half * TC_HALF;
      live = live < 0 ? 0 : (live > TC_HALF ? TC_HALF : live);
      if (uu >= nvalid) live = 0;
      const float un = un_s[uu];
      // Fast Lemma 1: slots are in descending norm, so the tile's first query
      // carries the largest error scale and slack; with e_u >= e(u, q) for
      // every q of the tile, acc < lo_k - e_u (rounded down) proves "no".
      const float2 c0 = cq_s[buf][0];
      const float thr = __fsub_rd(L.x, __fmaf_ru(un, c0.x, c0.y));
      uint32_t hit = 0;
      if (live == TC_HALF) {                       // fast path: the row maximum decides alone
        float m0 = acc[0], m1 = acc[1], m2 = acc[2], m3 = acc[3];
#pragma unroll
        for (int q = 4; q < TC_HALF; q += 4) {
          m0 = fmaxf(m0, acc[q]);
          m1 = fmaxf(m1, acc[q + 1]);
          m2 = fmaxf(m2, acc[q + 2]);
          m3 = fmaxf(m3, acc[q + 3]);
        }
        if (fmaxf(fmaxf(m0, m1), fmaxf(m2, m3)) >= thr) {
#pragma unroll
          for (int q = 0; q < TC_HALF; ++q) hit |= (acc[q] >= thr ? 1u : 0u) << q;
        }
      } else if (live > 0) {
#pragma unroll
        for (int q = 0; q < TC_HALF; ++q) hit |= (acc[q] >= thr ? 1u : 0u) << q;
        hit &= (1u << live) - 1u;
      }
      uint32_t ym = 0, tm = 0;
      if (hit) {
        const int k = b.grp[g_cur].x;
        const float pkb = c.full_p ? 0.f : __fmul_ru(un, (k <= c.m) ? c.pnorm[k - 1] : -kInf);
#pragma unroll
        for (int q = 0; q < TC_HALF; ++q) {
          if ((hit >> q) & 1u) {
            const float2 cq = cq_s[buf][half * TC_HALF + q];
            const float e = __fmaf_ru(un, cq.x, cq.y);
            if (!(__fadd_ru(acc[q], e) < L.x)) {                  // not decided no by Lemma 1
              const float lo = __fsub_rd(acc[q], e);
              const bool yes = c.full_p ? (lo >= L.y) : (lo >= pkb);
              if (yes) ym |= 1u << q; else tm |= 1u << q;
            }
          }
        }
      }
      while (ym) {
        const int q = __ffs(ym) - 1;
        ym &= ym - 1;
        const int j = qj_s[buf][half * TC_HALF + q];
        if (!in_segment(c, b, j, u0 + uu)) continue;
        const long long at = atomicAdd((unsigned long long*)&c.ctr[C_YES], 1ull);
        if (at < b.cap_y) b.ypairs[at] = ((unsigned long long)(uint32_t)j << 32) | (unsigned long long)(u0 + uu);
        atomicAdd(&b.qcnt[j], 1);
        ++st_yes;
      }
      while (tm) {
        const int q = __ffs(tm) - 1;
        tm &= tm - 1;
        const int j = qj_s[buf][half * TC_HALF + q];
        if (!in_segment(c, b, j, u0 + uu)) continue;
        const long long at = atomicAdd((unsigned long long*)&c.ctr[C_TODO], 1ull);
        if (at < b.cap_t) b.tpairs[at] = ((unsigned long long)(uint32_t)j << 32) | (unsigned long long)(u0 + uu);
        else set_status(c.ctr, ST_INTERNAL);
        ++st_todo;
      }
      g_cur = g_ld;
      t_cur = t_ld;
      if (has_next) advance(g_ld, t_ld);
      __syncthreads();                             // constants of item it consumed
    }
    __syncthreads();
  }
  if (s_fail && tid == 0) set_status(c.ctr, ST_TIMEOUT);
  if (tid == 0) {
    atomicAdd((unsigned long long*)&c.ctr[C_TESTED], (unsigned long long)st_pairs);
    atomicAdd((unsigned long long*)&c.ctr[C_PRUNED], (unsigned long long)st_skipped);
  }
  if (st_yes) atomicAdd((unsigned long long*)&c.ctr[C_YESFAST], (unsigned long long)st_yes);
  if (st_todo) atomicAdd((unsigned long long*)&c.ctr[C_TODOSUM], (unsigned long long)st_todo);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, 64);
}

cudaError_t launch_mfilter_tc(int kind, const Common& c, const Batch& b, int ngroups, int grid, size_t smem,
                              cudaStream_t st) {
  static thread_local bool cfg[3] = {false, false, false};
  cudaError_t e = cudaSuccess;
  if (!cfg[kind]) {
    if (kind == TCK_TF32) e = cudaFuncSetAttribute(k_mfilter_tc<TCK_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else if (kind == TCK_BF16) e = cudaFuncSetAttribute(k_mfilter_tc<TCK_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else e = cudaFuncSetAttribute(k_mfilter_tc<TCK_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cfg[kind] = true;
  }
  if (kind == TCK_TF32) k_mfilter_tc<TCK_TF32><<<grid, TC_THREADS, smem, st>>>(c, b, b.bqt, ngroups);
  else if (kind == TCK_BF16) k_mfilter_tc<TCK_BF16><<<grid, TC_THREADS, smem, st>>>(c, b, b.bqt, ngroups);
  else k_mfilter_tc<TCK_FP16><<<grid, TC_THREADS, smem, st>>>(c, b, b.bqt, ngroups);
  return cudaGetLastError();
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
    ws->cap_t = 16ll << 20;
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->tpairs, ws->cap_t * sizeof(unsigned long long)));
  }
  if (!ws->bqt && idx->d <= (int)TC_K)
    RMIPS_TRY_CUDA(cudaMalloc((void**)&ws->bqt, (size_t)MQ_SLOTS * TC_K * sizeof(float)));
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

rmips_status run_batch(rmips_index* idx, Workspace* ws, int64_t nq, long long* out, long long capacity,
                       cudaStream_t st, const long long* dseglo, const long long* dseghi) {
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
  rmips_status s = ensure_batch(idx, ws, want_y + 1);
  if (s != RMIPS_OK) return s;
  RMIPS_TRY_CUDA(cudaMemsetAsync(ws->ctr, 0, C_NCOUNTERS * sizeof(long long), st));
  const int ngroups_max = idx->k_max;
  const bool use_tc = idx->batch_tc && idx->d <= (int)TC_K;
  const int tck = idx->precision == RMIPS_BF16 ? TCK_BF16 : (idx->precision == RMIPS_FP16 ? TCK_FP16 : TCK_TF32);
  const size_t smem = (size_t)idx->d * (MQ_US + MQ_QS) * sizeof(float) + (size_t)ngroups_max * MQ_TU * sizeof(float2);
  const size_t smem_tc = tc_a_bytes(tck) + 2 * tc_tile_bytes(tck);
  const int64_t tc_tiles = (idx->n + TCU - 1) / TCU;
  const int tc_grid = (int)(tc_tiles < sm_count * 3 ? tc_tiles : sm_count * 3);
  int64_t per_sm = (int64_t)(228 * 1024) / (int64_t)(smem + 4096);
  if (per_sm > 4) per_sm = 4;
  if (per_sm < 1) per_sm = 1;
  const int64_t tiles = (idx->n + MQ_TU - 1) / MQ_TU;
  const int fgrid = (int)(tiles < sm_count * per_sm ? tiles : sm_count * per_sm);
  for (int64_t j0 = 0; j0 < nq; j0 += MQ_MAXQ) {
    const int cnt = (int)((nq - j0) < MQ_MAXQ ? (nq - j0) : MQ_MAXQ);
    Batch b{};
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
    b.bqt = use_tc ? reinterpret_cast<unsigned char*>(ws->bqt) : nullptr;
    b.bqt_kind = tck;
    b.keys = ws->keys;
    b.runs = ws->runs;
    b.hist = ws->hist;
    b.gfirst = ws->gfirst;
    b.gslot0 = ws->gslot0;
    b.seglo = dseglo ? dseglo + j0 : nullptr;
    b.seghi = dseghi ? dseghi + j0 : nullptr;
    b.big = ws->big;
    b.bigmaps = ws->bigmaps;
    b.nw = idx->n / 32 + 1;
    b.doffs = ws->doffs + j0;
    b.out = out;
    b.capacity = capacity;
    const int nruns = (cnt + RUN - 1) / RUN;
    RMIPS_TRY_CUDA(cudaMemsetAsync(b.hist, 0, (RMIPS_KMAX_LIMIT + 2) * sizeof(int), st));
    k_mprep_a<<<(cnt + 255) / 256, 256, 0, st>>>(c, b, idx->precision);
    k_mprep_groups<<<1, 256, 0, st>>>(c, b);
    k_mprep_runs<<<nruns, RUN, 0, st>>>(b);
    k_mprep_place<<<(nruns * RUN + 255) / 256, 256, 0, st>>>(b, nruns);
    k_mprep_c<<<sm_count * 4, 256, 0, st>>>(c, b);
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
      RMIPS_TRY_CUDA(launch_mfilter_tc(tck, c, b, idx->k_max, tc_grid, smem_tc, st));
    } else {
      RMIPS_TRY_CUDA(mfilter_dispatch(idx, c, b, idx->k_max, fgrid, smem, st));
    }
    if (prof) {
      RMIPS_TRY_CUDA(cudaEventRecord(ws->ev[2 * ws->ev_used + 1], st));
      ws->ev_used++;
    }
    k_mresolve<<<sm_count * 2, 256, 0, st>>>(c, b);
    k_mscan<<<1, 1024, 0, st>>>(c, b);
    k_mscatter<<<sm_count * 4, 256, 0, st>>>(c, b);
    k_memit<<<(cnt + MEMIT_Q - 1) / MEMIT_Q, 256, 0, st>>>(c, b);
    k_memit_big<<<MQ_BIG_SLOTS, 1024, 0, st>>>(c, b);
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
  DeviceGuard dg(idx->device);
  cudaStream_t st = (cudaStream_t)stream;
  s = RMIPS_OK;
  Workspace* ws = acquire_workspace(idx, &s);
  if (!ws) return s;
  WsGuard g{idx, ws};
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
  if ((s = ensure_queries(idx, ws, nq)) != RMIPS_OK) return s;
  const bool out_dev = capacity > 0 && is_device_ptr(out_ids);
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
  const bool batched = ranges_only;
  if (batched) {
    const long long* dlo = nullptr;
    const long long* dhi = nullptr;
    if (segs) {
      if ((s = ensure_segments(ws, nq)) != RMIPS_OK) return s;
      std::vector<long long> lo(nq), hi(nq);
      for (int64_t j = 0; j < nq; ++j) {
        lo[j] = segs[j].kind == 1 ? segs[j].begin : 0;
        hi[j] = segs[j].kind == 1 ? segs[j].end : INT64_MAX;
      }
      RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->dseglo, lo.data(), nq * sizeof(long long), cudaMemcpyHostToDevice, st));
      RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->dseghi, hi.data(), nq * sizeof(long long), cudaMemcpyHostToDevice, st));
      dlo = ws->dseglo;
      dhi = ws->dseghi;
    }
    if ((s = run_batch(idx, ws, nq, out, capacity, st, dlo, dhi)) != RMIPS_OK) return s;
  } else {
    if ((s = run_queries(idx, ws, nq, segs, out, capacity, st)) != RMIPS_OK) return s;
  }
  RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->h_ctr, ws->ctr, C_NCOUNTERS * sizeof(long long), cudaMemcpyDeviceToHost, st));
  RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->h_offs, ws->doffs, (nq + 1) * sizeof(long long), cudaMemcpyDeviceToHost, st));
  RMIPS_TRY_CUDA(cudaStreamSynchronize(st));
  for (int64_t j = 0; j <= nq; ++j) out_offsets[j] = ws->h_offs[j];
  record_stats(idx, ws, ws->h_ctr, nq, batched);
  {
    std::lock_guard<std::mutex> lk(idx->mu);
    idx->last_stats.result = ws->h_offs[nq];
  }
  if (ws->h_ctr[C_STATUS] == ST_INTERNAL) { set_error("k outside [1, k_max]"); return RMIPS_ERR_K_RANGE; }
  if ((s = status_from_device(ws->h_ctr[C_STATUS])) != RMIPS_OK) return s;
  const long long total = ws->h_offs[nq];
  if (!out_dev && total > 0)
    RMIPS_TRY_CUDA(cudaMemcpy(out_ids, ws->dout, total * sizeof(long long), cudaMemcpyDeviceToHost));
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
  *out_count = offs[1];
  return status_from_device(h[C_STATUS]);
}

extern "C" rmips_status rmips_debug_tc_tile(const float* A, const float* B, float* D, int32_t kind, int32_t lbo,
                                           int32_t sbo, void* stream) {
  if (kind < TCK_TF32 || kind > TCK_FP16) { set_error("bad kind"); return RMIPS_ERR_ARG; }
  if (lbo == 0) lbo = (int32_t)TC_LBO;
  if (sbo == 0) sbo = (int32_t)(kind == TCK_TF32 ? TC_SBO : TC_SBO16);
  if (!A || !B || !D || lbo <= 0 || sbo <= 0 || lbo > 4096 || sbo > 4096 || (lbo & 15) || (sbo & 15)) {
    set_error("bad argument");
    return RMIPS_ERR_ARG;
  }
  if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(D)) {
    set_error("A, B and D must be device memory");
    return RMIPS_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  long long* status = nullptr;
  RMIPS_TRY_CUDA(cudaMallocAsync((void**)&status, sizeof(long long), st));
  RMIPS_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(long long), st));
  const int dsmem = (int)(192 * TC_K * 4);
  if (kind == TCK_TF32) {
    RMIPS_TRY_CUDA(cudaFuncSetAttribute(k_debug_tc<TCK_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem));
    k_debug_tc<TCK_TF32><<<1, 128, dsmem, st>>>(A, B, D, (uint32_t)lbo, (uint32_t)sbo, status);
  } else if (kind == TCK_BF16) {
    RMIPS_TRY_CUDA(cudaFuncSetAttribute(k_debug_tc<TCK_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem));
    k_debug_tc<TCK_BF16><<<1, 128, dsmem, st>>>(A, B, D, (uint32_t)lbo, (uint32_t)sbo, status);
  } else {
    RMIPS_TRY_CUDA(cudaFuncSetAttribute(k_debug_tc<TCK_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem));
    k_debug_tc<TCK_FP16><<<1, 128, dsmem, st>>>(A, B, D, (uint32_t)lbo, (uint32_t)sbo, status);
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
}  // namespace rmips
