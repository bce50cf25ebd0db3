// Offline index build: Algorithm 1 ("Pre-processing of Simpfer", Section 4.1).
//
//  1. norms of every user and item (float64, squares summed in index order);
//  2. users and items sorted by descending norm, ties by ascending id;
//  3. for every user, its top-KC items by float32 inner product over P'
//     (the first p' sorted items; all of P for a full-P index), kept with a
//     running threshold (one user per thread, items streamed through shared
//     memory);
//  4. the KC candidates re-dotted in float64 with a rounding bound, giving
//     lo_j <= v_j <= hi_j for the j-th largest inner product v_j, and a proof
//     that no item outside the candidates can reach the k_max-th place;
//  5. blocks of consecutive users with L^j(B) = min lo_j (Equation 1).
#include <chrono>
#include <climits>
#include <cmath>

#include "rmips_internal.cuh"
#include "tc_common.cuh"

namespace rmips {
namespace {

constexpr float kInf = __builtin_huge_valf();

// --- 1. norms ----------------------------------------------------------------
// bad |= 1 for a NaN or infinity, |= 2 for a finite value above vmax (the
// largest magnitude the filter's storage format holds without overflow).
__global__ void k_norms(const float* __restrict__ X, int64_t rows, int64_t rows_pad, int d, float vmax,
                        float* __restrict__ nrm_up, unsigned long long* __restrict__ key,
                        int32_t* __restrict__ ids, int* __restrict__ bad) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= rows_pad) return;
  if (r >= rows) {
    key[r] = ~0ull;
    ids[r] = INT_MAX;
    return;
  }
  const float* x = X + r * d;
  double acc = 0.0;
  bool fin = true, inrange = true;
  for (int i = 0; i < d; ++i) {
    float v = x[i];
    fin = fin && isfinite(v);
    inrange = inrange && !(fabsf(v) > vmax);
    double dv = (double)v;
    acc = fma(dv, dv, acc);   // dv*dv is exact, so this equals acc + dv*dv rounded once
  }
  if (!fin) atomicOr(bad, 1);
  else if (!inrange) atomicOr(bad, 2);
  double s = sqrt(acc);
  // Upper bound of the exact norm: the float64 value is within (d/2 + 2) ulps.
  nrm_up[r] = __double2float_ru(__dmul_ru(s, 1.0 + (d + 8) * 0x1p-52));
  key[r] = ~(unsigned long long)__double_as_longlong(s);   // s >= 0: ascending key = descending norm
  ids[r] = (int32_t)r;
}

// --- 2. sort: bitonic network over (key, id), both ascending ----------------------
__global__ void k_bitonic(unsigned long long* __restrict__ key, int32_t* __restrict__ id, int64_t N2,
                          int64_t j, int64_t kk) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N2) return;
  int64_t p = i ^ j;
  if (p <= i) return;
  unsigned long long a = key[i], b = key[p];
  int32_t ia = id[i], ib = id[p];
  bool gt = (a > b) || (a == b && ia > ib);
  bool up = (i & kk) == 0;
  if (gt == up) {
    key[i] = b; key[p] = a;
    id[i] = ib; id[p] = ia;
  }
}

// --- gather rows / norms into sorted order ----------------------------------------
__global__ void k_gather(const float* __restrict__ src, const int32_t* __restrict__ perm, int64_t rows, int d,
                         float* __restrict__ dst, const float* __restrict__ nsrc, float* __restrict__ ndst) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * d) return;
  int64_t r = e / d;
  int c = (int)(e - r * d);
  int64_t o = perm[r];
  dst[e] = src[o * d + c];
  if (c == 0) ndst[r] = nsrc[o];
}

__device__ __forceinline__ void store_rn(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void store_rn(__half* p, float v) { *p = __float2half_rn(v); }

template <class H>
__global__ void k_to_half(const float* __restrict__ src, int64_t count, H* __restrict__ dst) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= count) return;
  store_rn(dst + e, src[e]);
}

// Users in 128-row tiles of the batched filter's operand layout (wf_off:
// K-major core matrices, rows of nstep 32-byte K steps, zeros past d):
// 16-byte chunks, 4 float32 (TF32 kind) or 8 16-bit values; consecutive
// threads fill consecutive rows of a chunk column.  Rows past n are zero.
__global__ void k_user_tiles(const float* __restrict__ Qs, const uint16_t* __restrict__ Qh, int64_t n, int d,
                             int nstep, unsigned char* __restrict__ out) {
  const int per = Qh ? 8 : 4;                      // values per chunk
  const int64_t chunks = 128 * (int64_t)(2 * nstep);
  const uint32_t sbo = wf_sbo(nstep), tb = wf_tile_bytes(nstep);
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t tiles = (n + 127) / 128;
  if (e >= tiles * chunks) return;
  const int64_t t = e / chunks;
  const int rem = (int)(e - t * chunks);
  const int r = rem & 127, k0 = (rem >> 7) * per;
  const int64_t u = t * 128 + r;
  if (!Qh) {
    float v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = (u < n && k0 + i < d) ? Qs[u * d + k0 + i] : 0.f;
    *reinterpret_cast<float4*>(out + t * tb + wf_off(r, (rem >> 7) * 16, sbo)) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    uint16_t h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) h[i] = (u < n && k0 + i < d) ? Qh[u * d + k0 + i] : (uint16_t)0;
    uint4 w;
    w.x = h[0] | ((uint32_t)h[1] << 16);
    w.y = h[2] | ((uint32_t)h[3] << 16);
    w.z = h[4] | ((uint32_t)h[5] << 16);
    w.w = h[6] | ((uint32_t)h[7] << 16);
    *reinterpret_cast<uint4*>(out + t * tb + wf_off(r, (rem >> 7) * 16, sbo)) = w;
  }
}

// --- 3. top-KC candidates per user (float32, one user per thread) -----------------
// Items stream through shared memory in tiles of TP, stored transposed so that
// every thread reads the same float4 (a broadcast) holding component i of four
// consecutive items.  The KC best (value, position) pairs of each thread live
// in a shared-memory column; an item is inserted only when strictly above the
// current minimum, so every item left out has a value <= the final minimum.
constexpr int TP = 64;
constexpr int TS = TP + 4;
constexpr int TOPK_THREADS = 128;

template <int DP>
__global__ void __launch_bounds__(TOPK_THREADS) k_topk(const float* __restrict__ Qs, const float* __restrict__ Ps,
                                                       int64_t n, int64_t pp, int d, float* __restrict__ cval,
                                                       int32_t* __restrict__ cid, const int32_t* __restrict__ ulist,
                                                       int nseg) {
  // Item range of this CTA: segment blockIdx.y of nseg equal parts of P'.
  // The output row is the user (nseg = 1, no list) or (slot * nseg + segment).
  const int64_t segsize = (pp + nseg - 1) / nseg;
  const int64_t pa = (int64_t)blockIdx.y * segsize;
  const int64_t pb = pa + segsize < pp ? pa + segsize : pp;
  extern __shared__ __align__(16) float topk_smem[];
  float* tile = topk_smem;                                                   // [DP][TS]
  float (*lv)[TOPK_THREADS] = reinterpret_cast<float (*)[TOPK_THREADS]>(topk_smem + DP * TS);
  int32_t (*li)[TOPK_THREADS] =
      reinterpret_cast<int32_t (*)[TOPK_THREADS]>(topk_smem + DP * TS + RMIPS_KC * TOPK_THREADS);
  const int t = threadIdx.x;
  const int64_t slot = blockIdx.x * (int64_t)TOPK_THREADS + t;   // n = users to do (list length if ulist)
  const int64_t u = slot < n ? (ulist ? (int64_t)ulist[slot] : slot) : n;
  float ur[DP];
#pragma unroll
  for (int i = 0; i < DP; ++i) ur[i] = (slot < n && i < d) ? Qs[u * d + i] : 0.f;
#pragma unroll
  for (int s = 0; s < RMIPS_KC; ++s) {
    lv[s][t] = -kInf;
    li[s][t] = -1;
  }
  float thr = -kInf;
  int minslot = 0;
  for (int64_t p0 = pa; p0 < pb; p0 += TP) {
    __syncthreads();
    for (int e = t; e < DP * TP; e += TOPK_THREADS) {
      int i = e / TP, j = e % TP;
      int64_t p = p0 + j;
      tile[i * TS + j] = (i < d && p < pb) ? Ps[p * d + i] : 0.f;
    }
    __syncthreads();
    const int jmax = (int)((pb - p0) < TP ? (pb - p0) : TP);
    for (int j = 0; j < jmax; j += 4) {
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
      for (int i = 0; i < DP; ++i) {
        float4 pv = *reinterpret_cast<const float4*>(&tile[i * TS + j]);
        a0 = fmaf(ur[i], pv.x, a0);
        a1 = fmaf(ur[i], pv.y, a1);
        a2 = fmaf(ur[i], pv.z, a2);
        a3 = fmaf(ur[i], pv.w, a3);
      }
      float av[4] = {a0, a1, a2, a3};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (j + r < jmax && av[r] > thr) {
          lv[minslot][t] = av[r];
          li[minslot][t] = (int32_t)(p0 + j + r);
          thr = lv[0][t];
          minslot = 0;
          for (int s = 1; s < RMIPS_KC; ++s) {
            float v = lv[s][t];
            if (v < thr) { thr = v; minslot = s; }
          }
        }
      }
    }
  }
  if (slot < n) {
    const int64_t row = ulist ? slot * nseg + blockIdx.y : u;
    for (int s = 0; s < RMIPS_KC; ++s) {
      cval[row * RMIPS_KC + s] = lv[s][t];
      cid[row * RMIPS_KC + s] = li[s][t];
    }
  }
}

// Descending sort of one 64-bit key per lane across a warp (bitonic network).
__device__ __forceinline__ unsigned long long warp_sort_desc_u64(unsigned long long x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, j);
      const bool keep_max = (((lane & j) == 0) == ((lane & k) == 0));
      x = keep_max ? (x > y ? x : y) : (x < y ? x : y);
    }
  }
  return x;
}

// (value, item) as one key ordered by value: larger float -> larger key.
__device__ __forceinline__ unsigned long long vkey(float v, int32_t id) {
  const uint32_t b = __float_as_uint(v);
  const uint32_t k = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  return ((unsigned long long)k << 32) | (uint32_t)(id + 1);
}
__device__ __forceinline__ float vkey_value(unsigned long long key) {
  const uint32_t k = (uint32_t)(key >> 32);
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Merges the nseg per-segment top-KC lists of each listed user into its
// top-KC (one warp per user): each list is sorted, reversed and combined
// with the running top-KC by element-wise maximum, which leaves a bitonic
// sequence holding the KC largest of both; a half-cleaner network sorts it.
__global__ void k_merge_segments(const float* __restrict__ sval, const int32_t* __restrict__ sid,
                                 const int32_t* __restrict__ ulist, int64_t nlist, int nseg,
                                 float* __restrict__ cval, int32_t* __restrict__ cid) {
  const int64_t slot = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (slot >= nlist) return;
  unsigned long long cur = 0;
  for (int g = 0; g < nseg; ++g) {
    const int64_t r = (slot * nseg + g) * RMIPS_KC + lane;
    unsigned long long x = warp_sort_desc_u64(vkey(sval[r], sid[r]));
    if (g == 0) { cur = x; continue; }
    x = __shfl_sync(0xffffffffu, x, 31 - lane);              // ascending
    cur = cur > x ? cur : x;                                   // bitonic, the KC largest of both
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, cur, j);
      cur = ((lane & j) == 0) ? (cur > y ? cur : y) : (cur < y ? cur : y);
    }
  }
  const int64_t u = ulist[slot];
  cval[u * RMIPS_KC + lane] = vkey_value(cur);
  cid[u * RMIPS_KC + lane] = (int32_t)(cur & 0xffffffffull) - 1;
}

// Positions of the users whose candidate list is not proven complete.
__global__ void k_list_incomplete(const uint8_t* __restrict__ incomp, int64_t n, int32_t* __restrict__ list,
                                  unsigned long long* __restrict__ count) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u < n && incomp[u]) list[atomicAdd(count, 1ull)] = (int32_t)u;
}

// --- 3'. top-KC candidates per user on tensor cores (d <= 64) -------------------------
// Operands in TF32 (float32 index) or in the index's BF16 / FP16 format, FP32
// accumulation.  A CTA keeps 128 users (one per thread, TMEM lane = user) and
// streams every 64-item tile of P' through one 128 x 64 x 64 MMA chain; items
// arrive by 1-D TMA in the UMMA layout prepared by k_item_tiles.  Each thread
// keeps its user's KC best (value, position) in shared memory and `uex`, an
// upper bound on the exact inner product of every item it did not keep: a
// rejected item adds its tensor-core value plus ||u|| tc_rel_err(kind) ||p||
// and the absolute term of sub-normal 16-bit operands (for a whole tile, the
// tile's first item has the largest norm), an evicted item the same.  The
// float64 re-dot of the kept candidates (k_finalize) then makes the bounds
// rigorous whatever the selection's precision.
constexpr int TB_THREADS = 128;
constexpr int TB_TILE = 64;

template <int KIND>
__global__ void k_item_tiles(const float* __restrict__ Ps, const float* __restrict__ pnorm, int64_t pp, int d,
                             int64_t ntiles, unsigned char* __restrict__ Pt, float* __restrict__ cp) {
  constexpr uint32_t E = KIND == TCK_TF32 ? 4u : 2u;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < ntiles * TB_TILE * (int64_t)TC_K) {
    const int64_t tile = e / (TB_TILE * TC_K);
    const int r = (int)((e / TC_K) % TB_TILE), k = (int)(e % TC_K);
    const int64_t p = tile * TB_TILE + r;
    const float v = (p < pp && k < d) ? Ps[p * d + k] : 0.f;
    unsigned char* base = Pt + (size_t)tile * (TB_TILE * TC_K * E);
    if (KIND == TCK_TF32) *reinterpret_cast<float*>(base + tc_off(r, k)) = v;
    else if (KIND == TCK_BF16) *reinterpret_cast<__nv_bfloat16*>(base + tc_off16(r, k)) = __float2bfloat16_rn(v);
    else *reinterpret_cast<__half*>(base + tc_off16(r, k)) = __float2half_rn(v);
  }
  if (e < ntiles * TB_TILE) cp[e] = e < pp ? __fmul_ru(pnorm[e], tc_rel_err(KIND)) : 0.f;
}

template <int KIND>
__global__ void __launch_bounds__(TB_THREADS) k_topk_tc(const float* __restrict__ Qs,
                                                        const unsigned char* __restrict__ Pt,
                                                        const float* __restrict__ cp, const float* __restrict__ unorm,
                                                        int64_t n, int64_t pp, int d, float pn0,
                                                        float* __restrict__ cval, int32_t* __restrict__ cid,
                                                        float* __restrict__ uex_out, int* __restrict__ fail) {
  constexpr uint32_t E = KIND == TCK_TF32 ? 4u : 2u;
  constexpr uint32_t SBO = KIND == TCK_TF32 ? TC_SBO : TC_SBO16;
  extern __shared__ __align__(1024) unsigned char tb[];
  unsigned char* sA = tb;                                                          // 128 x 64 (at most 32 KB)
  unsigned char* sB = tb + 32768;                                                  // 2 x (64 x 64)
  float (*lv)[TB_THREADS] = reinterpret_cast<float (*)[TB_THREADS]>(tb + 65536);   // [KC][128]
  int32_t (*li)[TB_THREADS] = reinterpret_cast<int32_t (*)[TB_THREADS]>(tb + 65536 + RMIPS_KC * TB_THREADS * 4);
  __shared__ float cps[2][TB_TILE];
  __shared__ __align__(8) uint64_t bar_b[2];
  __shared__ __align__(8) uint64_t bar_m;
  __shared__ uint32_t taddr_s;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t TILE_BYTES = TB_TILE * TC_K * E;
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
  const uint32_t tlane = taddr + ((uint32_t)(warp * 32) << 16);
  const uint32_t idesc = KIND == TCK_TF32 ? tc_idesc_tf32(128, TB_TILE) : tc_idesc_f16(128, TB_TILE, KIND == TCK_BF16);
  const int64_t ntiles = (pp + TB_TILE - 1) / TB_TILE;
  uint32_t phb = 0, ph_m = 0;
  auto load_tile = [&](int64_t t, int buf) {
    if (tid == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(&bar_b[buf], TILE_BYTES);
      bulk_g2s(sB + (size_t)buf * TILE_BYTES, Pt + t * TILE_BYTES, TILE_BYTES, &bar_b[buf]);
    }
    if (tid < TB_TILE) cps[buf][tid] = cp[t * TB_TILE + tid];
  };
  auto issue_mma = [&](int buf) -> bool {        // thread 0 only
    if (!mbar_wait_bounded(&bar_b[buf], (phb >> buf) & 1u)) return false;
    tc_fence_after();
    const uint32_t bb = smem_u32(sB) + (uint32_t)buf * TILE_BYTES;
    // one MMA consumes 32 bytes of K per row (8 TF32 or 16 16-bit values)
    for (uint32_t s = 0; s < TC_K * E / 32; ++s) {
      const uint64_t ad = tc_sdesc(smem_u32(sA) + s * 2 * TC_LBO, TC_LBO, SBO);
      const uint64_t bd = tc_sdesc(bb + s * 2 * TC_LBO, TC_LBO, SBO);
      if (KIND == TCK_TF32) tc_mma_tf32(taddr, ad, bd, idesc, s > 0 ? 1u : 0u);
      else tc_mma_f16(taddr, ad, bd, idesc, s > 0 ? 1u : 0u);
    }
    tc_commit(&bar_m);
    return true;
  };
  for (int64_t u0 = (int64_t)blockIdx.x * TB_THREADS; u0 < n && !s_fail; u0 += (int64_t)gridDim.x * TB_THREADS) {
    const int64_t nvalid = (n - u0) < TB_THREADS ? (n - u0) : TB_THREADS;
    const float* src = Qs + u0 * d;
    if (KIND == TCK_TF32) {
      for (int e = tid; e < TB_THREADS * (int)(TC_K / 4); e += TB_THREADS) {
        const int r = e & (TB_THREADS - 1), k0 = (e >> 7) * 4;
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
    } else {                                       // the 16-bit copy, rounded to nearest
      for (int e = tid; e < TB_THREADS * (int)(TC_K / 8); e += TB_THREADS) {
        const int r = e & (TB_THREADS - 1), k0 = (e >> 7) * 8;
        uint16_t h[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float v = (r < nvalid && k0 + i < d) ? src[(int64_t)r * d + k0 + i] : 0.f;
          h[i] = KIND == TCK_BF16 ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : __half_as_ushort(__float2half_rn(v));
        }
        uint4 w;
        w.x = h[0] | ((uint32_t)h[1] << 16);
        w.y = h[2] | ((uint32_t)h[3] << 16);
        w.z = h[4] | ((uint32_t)h[5] << 16);
        w.w = h[6] | ((uint32_t)h[7] << 16);
        *reinterpret_cast<uint4*>(sA + tc_off16(r, k0)) = w;
      }
    }
    const float un = tid < nvalid ? unorm[u0 + tid] : 0.f;
    // absolute error of operands below the 16-bit format's normal range
    // (FP16: 2^-25 each), charged to every bound: (d + 2) unit (||u|| + max ||p||)
    const float ua = __fmul_ru((float)(d + 2), __fmul_ru(tc_abs_unit(KIND), __fadd_ru(un, pn0)));
    for (int s = 0; s < RMIPS_KC; ++s) {
      lv[s][tid] = -kInf;
      li[s][tid] = -1;
    }
    float thr = -kInf, uex = -kInf;
    int minslot = 0;
    fence_proxy_async();
    load_tile(0, 0);
    __syncthreads();
    if (tid == 0 && !issue_mma(0)) s_fail = 1;
    phb ^= 1u;
    for (int64_t t = 0; t < ntiles; ++t) {
      const int buf = (int)(t & 1);
      const bool has_next = t + 1 < ntiles;
      if (has_next) load_tile(t + 1, buf ^ 1);
      bool ok = s_fail ? false : mbar_wait_bounded(&bar_m, ph_m);
      ph_m ^= 1u;
      ok = __syncthreads_and(ok && !s_fail);
      if (!ok) {
        if (tid == 0) s_fail = 1;
        break;
      }
      tc_fence_after();
      float acc[TB_TILE];
      // the two loads also return the maxima of their 32 columns
      const float mx0 = tmem_ld32_max(tlane, acc), mx1 = tmem_ld32_max(tlane + 32u, acc + 32);
      tmem_ld_wait();
      tc_fence_before();
      __syncthreads();
      if (has_next && tid == 0 && !issue_mma(buf ^ 1)) s_fail = 1;
      if (has_next) phb ^= 1u << (buf ^ 1);
      // epilogue: reject against the current KC-th value, insert the rest
      const int live = (int)((pp - t * TB_TILE) < TB_TILE ? (pp - t * TB_TILE) : TB_TILE);
      bool done_fast = false;
      if (live == TB_TILE) {                       // fast path: the tile's maximum decides alone
        static_assert(TB_TILE == 64, "two 32-column loads per tile");
        const float vmax = fmaxf(mx0, mx1);
        if (!(vmax > thr)) {                       // every item of the tile is rejected
          uex = fmaxf(uex, __fadd_ru(__fmaf_ru(un, cps[buf][0], vmax), ua));
          done_fast = true;
        }
      }
      if (!done_fast) {
      uint64_t cand = 0;
      float vrej = -kInf;
#pragma unroll
      for (int q = 0; q < TB_TILE; ++q) {
        const bool in = q < live && acc[q] > thr;
        cand |= (uint64_t)in << q;
        vrej = (q < live && !in) ? fmaxf(vrej, acc[q]) : vrej;
      }
      if (vrej > -kInf) uex = fmaxf(uex, __fadd_ru(__fmaf_ru(un, cps[buf][0], vrej), ua));
      while (cand) {
        const int q = __ffsll((long long)cand) - 1;
        cand &= cand - 1;
        float v = acc[0];
#pragma unroll
        for (int i = 1; i < TB_TILE; ++i) v = (i == q) ? acc[i] : v;
        if (v > thr) {
          const int32_t old = li[minslot][tid];
          if (old >= 0) uex = fmaxf(uex, __fadd_ru(__fmaf_ru(un, cp[old], lv[minslot][tid]), ua));
          lv[minslot][tid] = v;
          li[minslot][tid] = (int32_t)(t * TB_TILE + q);
          thr = lv[0][tid];
          minslot = 0;
          for (int s = 1; s < RMIPS_KC; ++s) {
            const float w = lv[s][tid];
            if (w < thr) { thr = w; minslot = s; }
          }
        } else {
          uex = fmaxf(uex, __fadd_ru(__fmaf_ru(un, cps[buf][q], v), ua));
        }
      }
      }
      __syncthreads();                              // cps[buf] consumed before it is reloaded
    }
    if (tid < nvalid) {
      const int64_t u = u0 + tid;
      for (int s = 0; s < RMIPS_KC; ++s) {
        cval[u * RMIPS_KC + s] = lv[s][tid];
        cid[u * RMIPS_KC + s] = li[s][tid];
      }
      uex_out[u] = uex;
    }
    __syncthreads();
  }
  if (s_fail && tid == 0) atomicOr(fail, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, 64);
}

// Bitonic sort of one value per lane, descending across the warp.
__device__ __forceinline__ double warp_sort_desc(double x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      double y = __shfl_xor_sync(0xffffffffu, x, j);
      bool keep_max = (((lane & j) == 0) == ((lane & k) == 0));
      x = keep_max ? fmax(x, y) : fmin(x, y);
    }
  }
  return x;
}

// --- 4. float64 re-dot, bounds, completeness proof (one warp per user) ------------
__global__ void k_finalize(const float* __restrict__ Qs, const float* __restrict__ Ps,
                           const float* __restrict__ cval, const int32_t* __restrict__ cid,
                           const float* __restrict__ unorm, const float* __restrict__ uex_in, float pn0, int64_t n,
                           int64_t pp, int d, int dp, int k_max, int full_p, float2* __restrict__ Lb,
                           int32_t* __restrict__ cand, float2* __restrict__ cbnd, uint8_t* __restrict__ incomp,
                           unsigned long long* __restrict__ n_incomplete, const int32_t* __restrict__ ulist,
                           int64_t nlist) {
  const int64_t slot = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (slot >= (ulist ? nlist : n)) return;
  const int64_t w = ulist ? (int64_t)ulist[slot] : slot;
  const float v = cval[w * RMIPS_KC + lane];
  const int32_t id = cid[w * RMIPS_KC + lane];
  double lo = -INFINITY, hi = -INFINITY;
  if (id >= 0) {
    const float* u = Qs + w * d;
    const float* p = Ps + (int64_t)id * d;
    double s = 0.0, a = 0.0;
    for (int i = 0; i < d; ++i) {
      double x = (double)u[i], y = (double)p[i];
      s = fma(x, y, s);
      a = fma(fabs(x), fabs(y), a);
    }
    double beta = __dmul_ru(a, 2.0 * (d + 2) * 0x1p-53);
    lo = __dsub_rd(s, beta);
    hi = __dadd_ru(s, beta);
  }
  const double lo_s = warp_sort_desc(lo);
  const double hi_s = warp_sort_desc(hi);
  const double v_s = warp_sort_desc(id >= 0 ? (double)v : -INFINITY);
  // Items never kept have float32 value <= the KC-th kept value t_K; each float32
  // value is within E = (dp + 2) 2^-24 ||u|| max||p|| of the exact one, so if
  // t_K + E <= t_kmax - E, no item outside the list can exceed the k_max-th
  // largest exact value among the kept ones.
  // Every item left out has an exact inner product <= uex (an upper bound
  // from the selection: float32 selection, the KC-th kept value plus the
  // float32 error bound with the largest item norm; tensor-core selection,
  // tracked per rejected / evicted item).  If uex <= the float64 lower bound
  // of the k_max-th largest kept value, at least k_max kept items reach every
  // excluded one, so the list holds the top-k_max.
  bool complete = pp <= RMIPS_KC;
  if (!complete) {
    double ub;
    if (uex_in) {
      ub = (double)uex_in[w];
    } else {
      double tK = __shfl_sync(0xffffffffu, v_s, RMIPS_KC - 1);
      double E = __dmul_ru(__dmul_ru((double)(dp + 2) * 0x1p-24, (double)unorm[w]), (double)pn0);
      ub = __dadd_ru(tK, E);
    }
    const double lo_k = __shfl_sync(0xffffffffu, lo_s, k_max - 1);
    complete = ub <= lo_k;
  }
  if (lane < k_max) {
    float flo = __double2float_rd(lo_s);
    float fhi = (full_p && complete) ? __double2float_ru(hi_s) : kInf;
    Lb[(int64_t)lane * n + w] = make_float2(flo, fhi);
  }
  if (full_p) {
    cand[w * RMIPS_KC + lane] = id;
    cbnd[w * RMIPS_KC + lane] = id >= 0 ? make_float2(__double2float_rd(lo), __double2float_ru(hi))
                                        : make_float2(-kInf, -kInf);
    if (lane == 0) {
      incomp[w] = complete ? 0 : 1;
      if (!complete) atomicAdd(n_incomplete, 1ull);
    }
  }
}

// --- 5. blocks (Equation 1) --------------------------------------------------------
__global__ void k_blocks(const float2* __restrict__ Lb, const float* __restrict__ unorm, int64_t n, int bs,
                         int64_t nb, int k_max, float* __restrict__ LB, float* __restrict__ hdr, int no_blocks) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nb * k_max) return;
  int j = (int)(e / nb);
  int64_t b = e - (int64_t)j * nb;
  int64_t lo = b * bs, hi = lo + bs < n ? lo + bs : n;
  float mn = kInf;
  for (int64_t i = lo; i < hi; ++i) mn = fminf(mn, Lb[(int64_t)j * n + i].x);
  LB[(int64_t)j * nb + b] = no_blocks ? -kInf : mn;     // -inf: Lemma 3 never prunes (ablation)
  if (j == 0) hdr[b] = unorm[lo];
}

inline unsigned grid_for(int64_t work, int threads) { return (unsigned)((work + threads - 1) / threads); }

rmips_status sort_by_norm(const float* X, int64_t rows, int d, float vmax, cudaStream_t st, float* nrm_up,
                          int32_t* order, int* d_bad) {
  int64_t N2 = 1;
  while (N2 < rows) N2 <<= 1;
  unsigned long long* key = nullptr;
  int32_t* ids = nullptr;
  RMIPS_TRY_CUDA(cudaMallocAsync((void**)&key, N2 * sizeof(unsigned long long), st));
  RMIPS_TRY_CUDA(cudaMallocAsync((void**)&ids, N2 * sizeof(int32_t), st));
  k_norms<<<grid_for(N2, 256), 256, 0, st>>>(X, rows, N2, d, vmax, nrm_up, key, ids, d_bad);
  for (int64_t kk = 2; kk <= N2; kk <<= 1)
    for (int64_t j = kk >> 1; j > 0; j >>= 1)
      k_bitonic<<<grid_for(N2, 256), 256, 0, st>>>(key, ids, N2, j, kk);
  RMIPS_TRY_CUDA(cudaMemcpyAsync(order, ids, rows * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  RMIPS_TRY_CUDA(cudaFreeAsync(key, st));
  RMIPS_TRY_CUDA(cudaFreeAsync(ids, st));
  RMIPS_TRY_CUDA(cudaGetLastError());
  return RMIPS_OK;
}

template <int DP>
cudaError_t launch_topk(const float* Qs, const float* Ps, int64_t n, int64_t pp, int d, float* cval,
                        int32_t* cid, cudaStream_t st, const int32_t* ulist = nullptr, int nseg = 1) {
  const size_t smem = (size_t)(DP * TS + 2 * RMIPS_KC * TOPK_THREADS) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_topk<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (n <= 0) return cudaSuccess;
  dim3 grid(grid_for(n, TOPK_THREADS), nseg);
  k_topk<DP><<<grid, TOPK_THREADS, smem, st>>>(Qs, Ps, n, pp, d, cval, cid, ulist, nseg);
  return cudaGetLastError();
}

// Float32 selection for the listed users only (d <= 64): repairs users whose
// tensor-core selection could not be proven complete.
cudaError_t launch_topk_list(const float* Qs, const float* Ps, int64_t nlist, int64_t pp, int d, float* sval,
                             int32_t* sid, const int32_t* ulist, int nseg, cudaStream_t st, int* dp) {
  if (d <= 16) { *dp = 16; return launch_topk<16>(Qs, Ps, nlist, pp, d, sval, sid, st, ulist, nseg); }
  if (d <= 32) { *dp = 32; return launch_topk<32>(Qs, Ps, nlist, pp, d, sval, sid, st, ulist, nseg); }
  if (d <= 52) { *dp = 52; return launch_topk<52>(Qs, Ps, nlist, pp, d, sval, sid, st, ulist, nseg); }
  *dp = 64;
  return launch_topk<64>(Qs, Ps, nlist, pp, d, sval, sid, st, ulist, nseg);
}

}  // namespace

rmips_status set_block_size(rmips_index* idx, int bs, cudaStream_t st) {
  if (!(bs == 32 || bs == 64 || bs == 128 || bs == 256)) { set_error("block size must be 32, 64, 128 or 256"); return RMIPS_ERR_ARG; }
  if (bs == idx->bs) return RMIPS_OK;
  const int64_t nb = (idx->n + bs - 1) / bs;
  float *LB = nullptr, *hdr = nullptr;
  RMIPS_TRY_CUDA(cudaMalloc((void**)&LB, (size_t)idx->k_max * nb * sizeof(float)));
  cudaError_t e = cudaMalloc((void**)&hdr, (size_t)nb * sizeof(float));
  if (e != cudaSuccess) {
    cudaFree(LB);
    set_error(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? RMIPS_ERR_OOM : RMIPS_ERR_CUDA;
  }
  k_blocks<<<grid_for(nb * idx->k_max, 256), 256, 0, st>>>(idx->Lb, idx->unorm, idx->n, bs, nb, idx->k_max, LB, hdr,
                                                          idx->no_blocks);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(LB);
    cudaFree(hdr);
    set_error(cudaGetErrorString(e));
    return RMIPS_ERR_CUDA;
  }
  cudaFree(idx->LB);
  cudaFree(idx->hdr);
  idx->device_bytes += (int64_t)(idx->k_max + 1) * (nb - idx->nb) * (int64_t)sizeof(float);
  idx->LB = LB;
  idx->hdr = hdr;
  idx->bs = bs;
  idx->nb = nb;
  return RMIPS_OK;
}

}  // namespace rmips

using namespace rmips;

extern "C" rmips_status rmips_build_index(const float* Q, int64_t n, const float* P, int64_t m, int32_t d,
                                          const rmips_build_opts* opts, void* stream, rmips_index** out) {
  if (out) *out = nullptr;
  if (!Q || !P || !out || !opts) { set_error("null argument"); return RMIPS_ERR_ARG; }
  if (n < 1 || m < 1 || d < 1 || d > RMIPS_DMAX || n > INT_MAX / 2 || m > INT_MAX / 2) {
    set_error("n, m must be >= 1 and < 2^30, d in [1, 128]");
    return RMIPS_ERR_ARG;
  }
  int bs = opts->block_size == 0 ? 32 : opts->block_size;
  if (opts->k_max < 1 || opts->k_max > RMIPS_KMAX_LIMIT || !(bs == 32 || bs == 64 || bs == 128 || bs == 256) ||
      opts->p_prime < 0 || opts->precision < RMIPS_FP32 || opts->precision > RMIPS_FP16 ||
      (opts->flags & ~(RMIPS_FLAG_BATCH_CUDA_CORES | RMIPS_FLAG_BUILD_CUDA_CORES | RMIPS_FLAG_NO_BLOCK_FILTER |
                       RMIPS_FLAG_AUTOTUNE)) != 0) {
    set_error("invalid build options (k_max 1..28, block_size 32/64/128/256, precision 0..2)");
    return RMIPS_ERR_ARG;
  }
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)stream;
  rmips_index* idx = new rmips_index();
  idx->n = n; idx->m = m; idx->d = d; idx->k_max = opts->k_max; idx->bs = bs;
  idx->precision = opts->precision;
  idx->batch_tc = (opts->flags & RMIPS_FLAG_BATCH_CUDA_CORES) ? 0 : 1;
  idx->no_blocks = (opts->flags & RMIPS_FLAG_NO_BLOCK_FILTER) ? 1 : 0;
  idx->pp = (opts->p_prime == 0 || opts->p_prime >= m) ? m : opts->p_prime;
  idx->full_p = idx->pp == m ? 1 : 0;
  idx->nb = (n + bs - 1) / bs;
  cudaGetDevice(&idx->device);

  auto fail = [&](rmips_status s) { rmips_free_index(idx); return s; };
  {
    rmips_status pc = check_ptr_device(Q, idx->device, "Q");
    if (pc == RMIPS_OK) pc = check_ptr_device(P, idx->device, "P");
    if (pc != RMIPS_OK) return fail(pc);
  }
  const bool q_dev = is_device_ptr(Q), p_dev = is_device_ptr(P);
  float *Qin = nullptr, *Pin = nullptr, *qn = nullptr, *pn = nullptr, *cval = nullptr;
  unsigned char* Pt = nullptr;
  float *cpn = nullptr, *uex = nullptr;
  int32_t* ulist = nullptr;
  float* sval = nullptr;
  int32_t* sid = nullptr;
  int32_t* cid = nullptr;
  int *d_bad = nullptr;
  unsigned long long* d_incomp = nullptr;
  rmips_status s = RMIPS_OK;
#define TRY(expr)                                                                  \
  do {                                                                             \
    cudaError_t e__ = (expr);                                                      \
    if (e__ != cudaSuccess) {                                                      \
      set_error(std::string(#expr) + ": " + cudaGetErrorString(e__));              \
      s = (e__ == cudaErrorMemoryAllocation) ? RMIPS_ERR_OOM : RMIPS_ERR_CUDA;     \
      goto cleanup;                                                                \
    }                                                                              \
  } while (0)
  {
    const int64_t pad = 32 * (int64_t)d;  // one spare chunk so bulk copies of the tail stay in bounds
    TRY(dalloc(idx, &idx->Qs, n * d + pad));
    TRY(dalloc(idx, &idx->Ps, m * d + pad));
    TRY(cudaMemsetAsync(idx->Qs + n * d, 0, pad * sizeof(float), st));
    TRY(cudaMemsetAsync(idx->Ps + m * d, 0, pad * sizeof(float), st));
    TRY(dalloc(idx, &idx->unorm, n));
    TRY(dalloc(idx, &idx->pnorm, m));
    TRY(dalloc(idx, &idx->permQ, n));
    TRY(dalloc(idx, &idx->permP, m));
    TRY(dalloc(idx, &idx->Lb, (size_t)idx->k_max * n));
    TRY(dalloc(idx, &idx->LB, (size_t)idx->k_max * idx->nb));
    TRY(dalloc(idx, &idx->hdr, idx->nb));
    if (idx->full_p) {
      TRY(dalloc(idx, &idx->cand, (size_t)n * RMIPS_KC));
      TRY(dalloc(idx, &idx->cbnd, (size_t)n * RMIPS_KC));
      TRY(dalloc(idx, &idx->incomp, n));
    }
    TRY(cudaMallocAsync((void**)&qn, n * sizeof(float), st));
    TRY(cudaMallocAsync((void**)&pn, m * sizeof(float), st));
    TRY(cudaMallocAsync((void**)&d_bad, 16, st));
    TRY(cudaMallocAsync((void**)&d_incomp, 16, st));
    TRY(cudaMemsetAsync(d_bad, 0, 16, st));
    TRY(cudaMemsetAsync(d_incomp, 0, 16, st));
    const float* Qsrc = Q;
    const float* Psrc = P;
    if (!q_dev) {
      TRY(cudaMallocAsync((void**)&Qin, n * d * sizeof(float), st));
      TRY(cudaMemcpyAsync(Qin, Q, n * d * sizeof(float), cudaMemcpyHostToDevice, st));
      Qsrc = Qin;
    }
    if (!p_dev) {
      TRY(cudaMallocAsync((void**)&Pin, m * d * sizeof(float), st));
      TRY(cudaMemcpyAsync(Pin, P, m * d * sizeof(float), cudaMemcpyHostToDevice, st));
      Psrc = Pin;
    }
    // 1-2: norms and sort
    // the users also go into the filter's 16-bit copy (BF16 / FP16 indexes):
    // their values must stay finite there; the items stay in float32
    s = sort_by_norm(Qsrc, n, d, filter_max_abs(idx->precision), st, qn, idx->permQ, d_bad);
    if (s != RMIPS_OK) goto cleanup;
    s = sort_by_norm(Psrc, m, d, FLT_MAX, st, pn, idx->permP, d_bad);
    if (s != RMIPS_OK) goto cleanup;
    k_gather<<<grid_for(n * d, 256), 256, 0, st>>>(Qsrc, idx->permQ, n, d, idx->Qs, qn, idx->unorm);
    k_gather<<<grid_for(m * d, 256), 256, 0, st>>>(Psrc, idx->permP, m, d, idx->Ps, pn, idx->pnorm);
    TRY(cudaGetLastError());
    int h_bad = 0;
    TRY(cudaMemcpyAsync(&h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(&idx->pn0, idx->pnorm, sizeof(float), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    if (h_bad & 1) { set_error("non-finite value in Q or P"); s = RMIPS_ERR_NONFINITE; goto cleanup; }
    if (h_bad) {
      set_error(idx->precision == RMIPS_FP16 ? "a value of Q beyond +-65504 does not fit the FP16 filter copy"
                                             : "a value of Q beyond the BF16 range does not fit the filter copy");
      s = RMIPS_ERR_NONFINITE;
      goto cleanup;
    }
    if (idx->precision != RMIPS_FP32) {
      TRY(dalloc(idx, (uint16_t**)&idx->Qh, n * d + pad));
      TRY(cudaMemsetAsync((uint16_t*)idx->Qh + n * d, 0, pad * 2, st));
      if (idx->precision == RMIPS_BF16)
        k_to_half<__nv_bfloat16><<<grid_for(n * d, 256), 256, 0, st>>>(idx->Qs, n * d, (__nv_bfloat16*)idx->Qh);
      else
        k_to_half<__half><<<grid_for(n * d, 256), 256, 0, st>>>(idx->Qs, n * d, (__half*)idx->Qh);
    }
    if (idx->batch_tc && d <= (int)TC_K) {         // operand tiles of the batched tensor-core filter
      const int64_t tiles = (n + 127) / 128;
      const int nstep = wf_nstep(idx->precision == RMIPS_FP32, d);
      TRY(dalloc(idx, &idx->Qtc, (size_t)(tiles * wf_tile_bytes(nstep))));
      const int64_t chunks = tiles * 128 * 2 * nstep;
      k_user_tiles<<<grid_for(chunks, 256), 256, 0, st>>>(
          idx->Qs, idx->precision == RMIPS_FP32 ? nullptr : (const uint16_t*)idx->Qh, n, d, nstep, idx->Qtc);
      TRY(cudaGetLastError());
    }
    // 3: candidates
    TRY(cudaMallocAsync((void**)&cval, (size_t)n * RMIPS_KC * sizeof(float), st));
    TRY(cudaMallocAsync((void**)&cid, (size_t)n * RMIPS_KC * sizeof(int32_t), st));
    int dp = 0;
    const bool tc_build = d <= (int)TC_K && idx->pp > RMIPS_KC && !(opts->flags & RMIPS_FLAG_BUILD_CUDA_CORES);
    if (tc_build) {
      int dev = 0, sms = 1;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const int64_t ntiles = (idx->pp + TB_TILE - 1) / TB_TILE;
      // operand kind of the selection: TF32 for a float32 index, the index's
      // own 16-bit format otherwise (FP16 only while every item value fits it:
      // |p_i| <= ||p|| <= the largest item norm)
      TRY(cudaStreamSynchronize(st));                 // idx->pn0 has landed
      int kind = TCK_TF32;
      if (idx->precision == RMIPS_BF16) kind = TCK_BF16;
      if (idx->precision == RMIPS_FP16 && idx->pn0 <= 65504.0f) kind = TCK_FP16;
      idx->build_kind = kind;
      const uint32_t esz = kind == TCK_TF32 ? 4u : 2u;
      TRY(cudaMallocAsync((void**)&Pt, (size_t)ntiles * TB_TILE * TC_K * esz, st));
      TRY(cudaMallocAsync((void**)&cpn, (size_t)ntiles * TB_TILE * sizeof(float), st));
      TRY(cudaMallocAsync((void**)&uex, (size_t)n * sizeof(float), st));
      TRY(cudaMemsetAsync(d_bad, 0, 16, st));
      const unsigned tiles_grid = grid_for(ntiles * TB_TILE * TC_K, 256);
      if (kind == TCK_TF32) k_item_tiles<TCK_TF32><<<tiles_grid, 256, 0, st>>>(idx->Ps, idx->pnorm, idx->pp, d, ntiles, Pt, cpn);
      else if (kind == TCK_BF16) k_item_tiles<TCK_BF16><<<tiles_grid, 256, 0, st>>>(idx->Ps, idx->pnorm, idx->pp, d, ntiles, Pt, cpn);
      else k_item_tiles<TCK_FP16><<<tiles_grid, 256, 0, st>>>(idx->Ps, idx->pnorm, idx->pp, d, ntiles, Pt, cpn);
      const int smem_tc = 65536 + 2 * RMIPS_KC * TB_THREADS * 4;
      const int64_t utiles = (n + TB_THREADS - 1) / TB_THREADS;
      const int grid = (int)(utiles < 2 * sms ? utiles : 2 * sms);
      if (kind == TCK_TF32) {
        TRY(cudaFuncSetAttribute(k_topk_tc<TCK_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_tc));
        k_topk_tc<TCK_TF32><<<grid, TB_THREADS, smem_tc, st>>>(idx->Qs, Pt, cpn, idx->unorm, n, idx->pp, d, idx->pn0,
                                                               cval, cid, uex, d_bad);
      } else if (kind == TCK_BF16) {
        TRY(cudaFuncSetAttribute(k_topk_tc<TCK_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_tc));
        k_topk_tc<TCK_BF16><<<grid, TB_THREADS, smem_tc, st>>>(idx->Qs, Pt, cpn, idx->unorm, n, idx->pp, d, idx->pn0,
                                                               cval, cid, uex, d_bad);
      } else {
        TRY(cudaFuncSetAttribute(k_topk_tc<TCK_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_tc));
        k_topk_tc<TCK_FP16><<<grid, TB_THREADS, smem_tc, st>>>(idx->Qs, Pt, cpn, idx->unorm, n, idx->pp, d, idx->pn0,
                                                               cval, cid, uex, d_bad);
      }
      TRY(cudaGetLastError());
      int h_fail = 0;
      TRY(cudaMemcpyAsync(&h_fail, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
      TRY(cudaStreamSynchronize(st));
      if (h_fail) { set_error("tensor-core selection: a device wait timed out"); s = RMIPS_ERR_TIMEOUT; goto cleanup; }
    }
    else if (d <= 16) { dp = 16; TRY(launch_topk<16>(idx->Qs, idx->Ps, n, idx->pp, d, cval, cid, st)); }
    else if (d <= 32) { dp = 32; TRY(launch_topk<32>(idx->Qs, idx->Ps, n, idx->pp, d, cval, cid, st)); }
    else if (d <= 52) { dp = 52; TRY(launch_topk<52>(idx->Qs, idx->Ps, n, idx->pp, d, cval, cid, st)); }
    else if (d <= 64) { dp = 64; TRY(launch_topk<64>(idx->Qs, idx->Ps, n, idx->pp, d, cval, cid, st)); }
    else { dp = 128; TRY(launch_topk<128>(idx->Qs, idx->Ps, n, idx->pp, d, cval, cid, st)); }
    // 4: bounds
    k_finalize<<<grid_for(n * 32, 256), 256, 0, st>>>(idx->Qs, idx->Ps, cval, cid, idx->unorm, uex, idx->pn0,
                                                      n, idx->pp, d, dp, idx->k_max, idx->full_p, idx->Lb,
                                                      idx->cand, idx->cbnd, idx->incomp, d_incomp, nullptr, 0);
    if (tc_build && idx->full_p) {
      // users the TF32 selection could not prove complete: redo them in float32
      unsigned long long h_inc = 0;
      TRY(cudaMemcpyAsync(&h_inc, d_incomp, sizeof(h_inc), cudaMemcpyDeviceToHost, st));
      TRY(cudaStreamSynchronize(st));
      if (h_inc > 0) {
        TRY(cudaMallocAsync((void**)&ulist, (size_t)h_inc * sizeof(int32_t), st));
        TRY(cudaMemsetAsync(d_incomp, 0, 16, st));
        k_list_incomplete<<<grid_for(n, 256), 256, 0, st>>>(idx->incomp, n, ulist, d_incomp);
        TRY(cudaMemsetAsync(d_incomp, 0, 16, st));
        // split P' into segments so that even a handful of users fill the GPU, then merge
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t rows = ((int64_t)h_inc + TOPK_THREADS - 1) / TOPK_THREADS;
        int64_t nseg = (4 * (int64_t)sms + rows - 1) / rows;
        const int64_t seg_cap = idx->pp / (4 * TP) > 1 ? idx->pp / (4 * TP) : 1;
        if (nseg > seg_cap) nseg = seg_cap;
        if ((int64_t)h_inc * nseg * RMIPS_KC > (64ll << 20)) nseg = (64ll << 20) / ((int64_t)h_inc * RMIPS_KC);
        if (nseg < 1) nseg = 1;
        TRY(cudaMallocAsync((void**)&sval, (size_t)h_inc * nseg * RMIPS_KC * sizeof(float), st));
        TRY(cudaMallocAsync((void**)&sid, (size_t)h_inc * nseg * RMIPS_KC * sizeof(int32_t), st));
        int dp2 = 64;
        TRY(launch_topk_list(idx->Qs, idx->Ps, (int64_t)h_inc, idx->pp, d, sval, sid, ulist, (int)nseg, st, &dp2));
        k_merge_segments<<<grid_for((int64_t)h_inc * 32, 256), 256, 0, st>>>(sval, sid, ulist, (int64_t)h_inc,
                                                                              (int)nseg, cval, cid);
        k_finalize<<<grid_for((int64_t)h_inc * 32, 256), 256, 0, st>>>(
            idx->Qs, idx->Ps, cval, cid, idx->unorm, nullptr, idx->pn0, n, idx->pp, d, dp2, idx->k_max,
            idx->full_p, idx->Lb, idx->cand, idx->cbnd, idx->incomp, d_incomp, ulist, (int64_t)h_inc);
        TRY(cudaGetLastError());
      }
    }
    // 5: blocks
    k_blocks<<<grid_for(idx->nb * idx->k_max, 256), 256, 0, st>>>(idx->Lb, idx->unorm, n, bs, idx->nb,
                                                                   idx->k_max, idx->LB, idx->hdr, idx->no_blocks);
    TRY(cudaGetLastError());
    unsigned long long h_incomp = 0;
    TRY(cudaMemcpyAsync(&h_incomp, d_incomp, sizeof(h_incomp), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    idx->incomplete = (int64_t)h_incomp;
  }
cleanup:
  if (Qin) cudaFreeAsync(Qin, st);
  if (Pin) cudaFreeAsync(Pin, st);
  if (qn) cudaFreeAsync(qn, st);
  if (pn) cudaFreeAsync(pn, st);
  if (cval) cudaFreeAsync(cval, st);
  if (Pt) cudaFreeAsync(Pt, st);
  if (cpn) cudaFreeAsync(cpn, st);
  if (uex) cudaFreeAsync(uex, st);
  if (ulist) cudaFreeAsync(ulist, st);
  if (sval) cudaFreeAsync(sval, st);
  if (sid) cudaFreeAsync(sid, st);
  if (cid) cudaFreeAsync(cid, st);
  if (d_bad) cudaFreeAsync(d_bad, st);
  if (d_incomp) cudaFreeAsync(d_incomp, st);
#undef TRY
  if (s != RMIPS_OK) return fail(s);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("stream synchronisation failed after build");
    return fail(RMIPS_ERR_CUDA);
  }
  {
    const rmips_status ps = noalloc_prepare();       // the allocation-free call's scratch exists from here on
    if (ps != RMIPS_OK) return fail(ps);
  }
  if ((opts->flags & RMIPS_FLAG_AUTOTUNE) || opts->tune_cache) {
    const rmips_status ts = tune_index(idx, opts->tune_cache, st);
    if (ts != RMIPS_OK) return fail(ts);
  }
  idx->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = idx;
  return RMIPS_OK;
}
