// k-MIPS of every user over all items (Definition 1): the join whose top-k_max
// part the full-P index already holds.  For a user whose 32 candidates are
// proven to contain its top-k_max, one warp ranks the candidates (float64
// products with their error bounds, the exact integer comparison where two
// bounds overlap, equal products by ascending item id) and keeps the first k.
// A user without that proof is ranked by a scan over all items.
#include <climits>
#include <cmath>

#include "rmips_internal.cuh"

namespace rmips {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct Ranked {
  double s, b;        // float64 product and its error bound
  int32_t it;         // item position (-1: none)
  int32_t id;         // caller's item id
};

// True when x ranks before y: larger u.p, then smaller item id; "none" last.
__device__ __forceinline__ bool ranks_before(const Ranked& x, const Ranked& y, const float* u, const float* Ps,
                                             int d) {
  if (x.it < 0) return false;
  if (y.it < 0) return true;
  if (x.s - x.b > y.s + y.b) return true;
  if (y.s - y.b > x.s + x.b) return false;
  const int sg = exact_sign_diff(u, Ps + (int64_t)x.it * d, Ps + (int64_t)y.it * d, d);
  if (sg != 0) return sg > 0;
  return x.id < y.id;
}

__device__ __forceinline__ Ranked shfl_ranked(const Ranked& r, int src) {
  Ranked o;
  o.s = __shfl_sync(kFull, r.s, src);
  o.b = __shfl_sync(kFull, r.b, src);
  o.it = __shfl_sync(kFull, r.it, src);
  o.id = __shfl_sync(kFull, r.id, src);
  return o;
}

__device__ __forceinline__ void dot64(const float* u, const float* p, int d, double* s, double* a) {
  double x = 0.0, y = 0.0;
  for (int i = 0; i < d; ++i) {
    x = fma((double)u[i], (double)p[i], x);
    y = fma(fabs((double)u[i]), fabs((double)p[i]), y);
  }
  *s = x;
  *a = y;
}

// One warp per user (sorted position w); out row = the user's caller id.
__global__ void __launch_bounds__(256) k_topk_join(const float* __restrict__ Qs, const float* __restrict__ Ps,
                                                   const int32_t* __restrict__ cand, const uint8_t* __restrict__ incomp,
                                                   const int32_t* __restrict__ permQ, const int32_t* __restrict__ permP,
                                                   int64_t n, int64_t m, int d, int k, long long* __restrict__ out) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;                                   // warp-uniform
  const float* u = Qs + w * d;
  long long* orow = out + (int64_t)permQ[w] * k;
  const double bf = 2.0 * (d + 2) * 0x1p-53;            // float64 dot bound per unit of sum |u_i p_i|
  if (!incomp[w]) {
    Ranked me{-INFINITY, 0.0, -1, INT_MAX};
    const int32_t it = cand[w * RMIPS_KC + lane];
    if (it >= 0) {
      double s, a;
      dot64(u, Ps + (int64_t)it * d, d, &s, &a);
      me = Ranked{s, __dmul_ru(a, bf), it, permP[it]};
    }
    // bitonic network over the warp, first-ranked item to lane 0
#pragma unroll 1
    for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll 1
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
        // the lane that should keep the first-ranked of the pair takes the
        // other's entry unless its own ranks first; its partner gives its
        // entry away exactly when its own ranks first (the order is strict,
        // so the two decisions agree; two empty entries are alike)
        const Ranked other = shfl_ranked(me, lane ^ jj);
        const bool mine_first = ranks_before(me, other, u, Ps, d);
        const bool want_first = ((lane & jj) == 0) == ((lane & kk) == 0);
        if (want_first ? !mine_first : mine_first) me = other;
      }
    }
    if (lane < k) orow[lane] = me.id;
    return;
  }
  // No proof for this user: every lane keeps its best k of a strided scan of
  // all items (float64), then the warp merges the 32 lists.
  double tv[RMIPS_KMAX_LIMIT];
  int32_t ti[RMIPS_KMAX_LIMIT];
  for (int r = 0; r < k; ++r) { tv[r] = -INFINITY; ti[r] = -1; }
  for (int64_t j = lane; j < m; j += 32) {
    double s, a;
    dot64(u, Ps + j * d, d, &s, &a);
    if (s > tv[k - 1] || (s == tv[k - 1] && ti[k - 1] >= 0 && permP[j] < permP[ti[k - 1]])) {
      int r = k - 1;
      while (r > 0 && (s > tv[r - 1] || (s == tv[r - 1] && permP[j] < permP[ti[r - 1]]))) {
        tv[r] = tv[r - 1];
        ti[r] = ti[r - 1];
        --r;
      }
      tv[r] = s;
      ti[r] = (int32_t)j;
    }
  }
  int head = 0;
  for (int r = 0; r < k; ++r) {
    const double v = head < k ? tv[head] : -INFINITY;
    const int32_t id = (head < k && ti[head] >= 0) ? permP[ti[head]] : INT_MAX;
    double bv = v;
    int32_t bid = id, bl = lane;
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(kFull, bv, o);
      const int32_t oid = __shfl_xor_sync(kFull, bid, o);
      const int32_t ol = __shfl_xor_sync(kFull, bl, o);
      if (ov > bv || (ov == bv && oid < bid)) { bv = ov; bid = oid; bl = ol; }
    }
    if (lane == 0) orow[r] = bid;
    if (lane == bl) ++head;
  }
}

}  // namespace
}  // namespace rmips

using namespace rmips;

extern "C" rmips_status rmips_topk_join(const rmips_index* idx, int32_t k, int64_t* out_ids, void* stream) {
  if (!idx || !out_ids) { set_error("null argument"); return RMIPS_ERR_ARG; }
  if (!idx->full_p || !idx->cand) {
    set_error("the join needs a full-P index (p_prime = 0)");
    return RMIPS_ERR_ARG;
  }
  if (k < 1 || k > idx->k_max || k > idx->m) { set_error("k outside [1, min(k_max, m)]"); return RMIPS_ERR_K_RANGE; }
  if (check_ptr_device(out_ids, idx->device, "out_ids") != RMIPS_OK) return RMIPS_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != idx->device) cudaSetDevice(idx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev = is_device_ptr(out_ids);
  long long* dout = (long long*)out_ids;
  const size_t bytes = (size_t)idx->n * k * sizeof(long long);
  cudaError_t e = cudaSuccess;
  if (!dev) e = cudaMallocAsync((void**)&dout, bytes, st);
  if (e == cudaSuccess) {
    const int64_t threads = idx->n * 32;
    k_topk_join<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(idx->Qs, idx->Ps, idx->cand, idx->incomp,
                                                                   idx->permQ, idx->permP, idx->n, idx->m, idx->d,
                                                                   k, dout);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(out_ids, dout, bytes, cudaMemcpyDeviceToHost, st);
  if (!dev && dout) cudaFreeAsync(dout, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (prev != idx->device) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    set_error(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? RMIPS_ERR_OOM : RMIPS_ERR_CUDA;
  }
  return RMIPS_OK;
}
