// Index persistence and rebuild with another k_max.
//
// rmips_index_save / rmips_index_load write and read every device array of an
// index (with its sizes and options) so that a saved index answers exactly as
// the one built.  rmips_index_rebuild is the paper's path for k > k_max
// (Section 4.1: the bounds hold k_max ranks; a larger k needs Algorithm 1
// again): it restores Q and P in the caller's id order from the index's own
// sorted copies and builds anew.
#include <climits>
#include <cstdio>
#include <cstring>

#include "rmips_internal.cuh"
#include "tc_common.cuh"

namespace rmips {
namespace {

constexpr char kMagic[8] = {'R', 'M', 'I', 'P', 'S', 'I', 'X', '3'};

// File layout: this header, then for every array its byte count (int64), its
// bytes and their 64-bit FNV-1a hash.  96 bytes, no implicit padding.
struct FileHeader {
  char magic[8];
  int64_t n, m, nb, pp, incomplete;
  int32_t d, k_max, bs, precision, full_p, batch_tc, no_blocks, has_qh, has_qtc, narrays;
  float pn0;
  int32_t tune;            // autotuner choices: batch stages | single stages << 8 | tuned << 16
};
static_assert(sizeof(FileHeader) == 96, "index file header layout");

uint64_t fnv1a(const unsigned char* p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

// Every field the query kernels size or index with must be what a build of
// this library could have written; a file that fails is refused before any
// device call.
bool header_ok(const FileHeader& h, std::string* why) {
  auto bad = [&](const char* w) { *why = w; return false; };
  if (memcmp(h.magic, kMagic, sizeof(kMagic)) != 0) return bad("not an index file of this library");
  if (h.n < 1 || h.n > INT32_MAX || h.m < 1 || h.m > INT32_MAX) return bad("user or item count out of range");
  if (h.d < 1 || h.d > RMIPS_DMAX || h.k_max < 1 || h.k_max > RMIPS_KMAX_LIMIT) return bad("d or k_max out of range");
  if (h.bs != 32 && h.bs != 64 && h.bs != 128 && h.bs != 256) return bad("block size is not 32, 64, 128 or 256");
  if (h.nb != (h.n + h.bs - 1) / h.bs) return bad("block count does not match n and the block size");
  if (h.precision < RMIPS_FP32 || h.precision > RMIPS_FP16) return bad("unknown precision");
  if ((h.full_p != 0 && h.full_p != 1) || (h.batch_tc != 0 && h.batch_tc != 1) ||
      (h.no_blocks != 0 && h.no_blocks != 1) || (h.has_qh != 0 && h.has_qh != 1) ||
      (h.has_qtc != 0 && h.has_qtc != 1))
    return bad("flag field out of range");
  {
    const int ws_ns = h.tune & 0xff, q1_ns = (h.tune >> 8) & 0xff, tuned = (h.tune >> 16) & 0xff;
    if ((h.tune >> 24) != 0 || ws_ns > RMIPS_WS_MAXNS || (ws_ns & 1) || q1_ns > 8 || tuned > 2)
      return bad("autotuner field out of range");
  }
  if (h.pp < 1 || h.pp > h.m || (h.full_p == 1) != (h.pp == h.m)) return bad("|P'| does not match the index mode");
  if (h.has_qh != (h.precision != RMIPS_FP32 ? 1 : 0)) return bad("reduced-precision copy does not match the precision");
  if (h.has_qtc && h.d > 64) return bad("tensor-core tiles need d <= 64");
  if (h.incomplete < 0 || h.incomplete > h.n || (!h.full_p && h.incomplete != 0)) return bad("incomplete count out of range");
  if (!(h.pn0 >= 0.f) || !(h.pn0 <= FLT_MAX)) return bad("largest item norm is not finite");
  return true;
}

bool is_permutation(const unsigned char* bytes, int64_t n) {
  std::vector<unsigned char> seen((size_t)n, 0);
  for (int64_t i = 0; i < n; ++i) {
    int32_t v;
    memcpy(&v, bytes + 4 * i, 4);
    if (v < 0 || v >= n || seen[(size_t)v]) return false;
    seen[(size_t)v] = 1;
  }
  return true;
}

// The device arrays of an index in file order: pointer slot and byte size.
struct ArrayRef {
  void** ptr;
  int64_t bytes;
};

std::vector<ArrayRef> arrays(rmips_index* idx, bool has_qh, bool has_qtc) {
  const int64_t n = idx->n, m = idx->m, d = idx->d, pad = 32 * d;
  const int64_t tiles = (n + 127) / 128;
  const int64_t tile_bytes = wf_tile_bytes(wf_nstep(idx->precision == RMIPS_FP32, idx->d));
  std::vector<ArrayRef> a = {
      {(void**)&idx->Qs, (n * d + pad) * 4},     {(void**)&idx->Ps, (m * d + pad) * 4},
      {(void**)&idx->unorm, n * 4},              {(void**)&idx->pnorm, m * 4},
      {(void**)&idx->permQ, n * 4},              {(void**)&idx->permP, m * 4},
      {(void**)&idx->Lb, (int64_t)idx->k_max * n * 8},
      {(void**)&idx->LB, (int64_t)idx->k_max * idx->nb * 4},
      {(void**)&idx->hdr, idx->nb * 4},
  };
  if (idx->full_p) {
    a.push_back({(void**)&idx->cand, n * RMIPS_KC * 4});
    a.push_back({(void**)&idx->cbnd, n * RMIPS_KC * 8});
    a.push_back({(void**)&idx->incomp, n});
  }
  if (has_qh) a.push_back({(void**)&idx->Qh, (n * d + pad) * 2});
  if (has_qtc) a.push_back({(void**)&idx->Qtc, tiles * tile_bytes});
  return a;
}

// Restores rows in caller order: dst[perm[i]] = src[i] (rows of d floats).
__global__ void k_unsort_rows(const float* __restrict__ src, const int32_t* __restrict__ perm, int64_t rows, int d,
                              float* __restrict__ dst) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * d) return;
  const int64_t r = e / d;
  dst[(int64_t)perm[r] * d + (e - r * d)] = src[e];
}

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace rmips

using namespace rmips;

extern "C" rmips_status rmips_index_save(const rmips_index* cidx, const char* path) {
  if (!cidx || !path) { set_error("null argument"); return RMIPS_ERR_ARG; }
  rmips_index* idx = const_cast<rmips_index*>(cidx);
  DevGuard g(idx->device);
  FileHeader h{};
  memcpy(h.magic, kMagic, sizeof(kMagic));
  h.n = idx->n; h.m = idx->m; h.nb = idx->nb; h.pp = idx->pp; h.incomplete = idx->incomplete;
  h.d = idx->d; h.k_max = idx->k_max; h.bs = idx->bs; h.precision = idx->precision; h.full_p = idx->full_p;
  h.batch_tc = idx->batch_tc; h.no_blocks = idx->no_blocks; h.has_qh = idx->Qh != nullptr; h.has_qtc = idx->Qtc != nullptr;
  h.pn0 = idx->pn0;
  h.tune = (idx->tune_ws_ns & 0xff) | ((idx->tune_q1_ns & 0xff) << 8) | ((idx->tuned & 0xff) << 16);
  const std::vector<ArrayRef> a = arrays(idx, h.has_qh, h.has_qtc);
  h.narrays = (int32_t)a.size();
  if (cudaDeviceSynchronize() != cudaSuccess) { set_error("device error before save"); return RMIPS_ERR_CUDA; }
  FILE* f = fopen(path, "wb");
  if (!f) { set_error(std::string("cannot open ") + path + " for writing"); return RMIPS_ERR_ARG; }
  bool ok = fwrite(&h, sizeof(h), 1, f) == 1;
  std::vector<unsigned char> buf;
  for (const ArrayRef& r : a) {
    ok = ok && fwrite(&r.bytes, sizeof(r.bytes), 1, f) == 1;
    buf.resize((size_t)r.bytes);
    ok = ok && cudaMemcpy(buf.data(), *r.ptr, (size_t)r.bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && fwrite(buf.data(), 1, (size_t)r.bytes, f) == (size_t)r.bytes;
    const uint64_t hash = fnv1a(buf.data(), buf.size());
    ok = ok && fwrite(&hash, sizeof(hash), 1, f) == 1;
  }
  ok = (fclose(f) == 0) && ok;
  if (!ok) { set_error(std::string("writing ") + path + " failed"); return RMIPS_ERR_ARG; }
  return RMIPS_OK;
}

// Reads and checks the whole file on the host (header fields, array sizes,
// hashes, the two permutations and the candidate item positions) and only
// then uploads it, so a corrupted or foreign file never reaches a kernel.
extern "C" rmips_status rmips_index_load(const char* path, void* stream, rmips_index** out) {
  if (out) *out = nullptr;
  if (!path || !out) { set_error("null argument"); return RMIPS_ERR_ARG; }
  FILE* f = fopen(path, "rb");
  if (!f) { set_error(std::string("cannot open ") + path); return RMIPS_ERR_ARG; }
  FileHeader h{};
  std::string why;
  if (fread(&h, sizeof(h), 1, f) != 1) why = "shorter than an index header";
  else header_ok(h, &why);
  if (!why.empty()) {
    fclose(f);
    set_error(std::string(path) + ": " + why);
    return RMIPS_ERR_ARG;
  }
  rmips_index* idx = new rmips_index();
  idx->n = h.n; idx->m = h.m; idx->nb = h.nb; idx->pp = h.pp; idx->incomplete = h.incomplete;
  idx->d = h.d; idx->k_max = h.k_max; idx->bs = h.bs; idx->precision = h.precision; idx->full_p = h.full_p;
  idx->batch_tc = h.batch_tc; idx->no_blocks = h.no_blocks; idx->pn0 = h.pn0;
  idx->tune_ws_ns = h.tune & 0xff;
  idx->tune_q1_ns = (h.tune >> 8) & 0xff;
  idx->tuned = (h.tune >> 16) & 0xff;
  const std::vector<ArrayRef> a = arrays(idx, h.has_qh != 0, h.has_qtc != 0);
  std::vector<std::vector<unsigned char>> bufs(a.size());
  if ((int32_t)a.size() != h.narrays) why = "array count does not match its header";
  for (size_t i = 0; why.empty() && i < a.size(); ++i) {
    int64_t bytes = -1;
    uint64_t hash = 0;
    if (fread(&bytes, sizeof(bytes), 1, f) != 1 || bytes != a[i].bytes) { why = "array sizes do not match its header"; break; }
    bufs[i].resize((size_t)bytes);
    if (fread(bufs[i].data(), 1, (size_t)bytes, f) != (size_t)bytes || fread(&hash, sizeof(hash), 1, f) != 1) {
      why = "truncated";
      break;
    }
    if (hash != fnv1a(bufs[i].data(), bufs[i].size())) { why = "array contents do not match their hash"; break; }
  }
  if (why.empty() && fgetc(f) != EOF) why = "trailing bytes after the last array";
  fclose(f);
  // index arrays that address device memory: permutations, candidate positions
  for (size_t i = 0; why.empty() && i < a.size(); ++i) {
    if ((a[i].ptr == (void**)&idx->permQ && !is_permutation(bufs[i].data(), idx->n)) ||
        (a[i].ptr == (void**)&idx->permP && !is_permutation(bufs[i].data(), idx->m)))
      why = "a stored order is not a permutation";
    if (a[i].ptr == (void**)&idx->cand) {
      const int32_t* c = reinterpret_cast<const int32_t*>(bufs[i].data());
      for (size_t e = 0; e < bufs[i].size() / 4; ++e)
        if (c[e] < -1 || c[e] >= idx->m) { why = "a candidate item position is out of range"; break; }
    }
  }
  if (!why.empty()) {
    delete idx;
    set_error(std::string(path) + ": " + why);
    return RMIPS_ERR_ARG;
  }
  cudaGetDevice(&idx->device);
  rmips_status s = RMIPS_OK;
  for (size_t i = 0; s == RMIPS_OK && i < a.size(); ++i) {
    cudaError_t e = cudaMalloc(a[i].ptr, bufs[i].size());
    if (e == cudaSuccess) {
      idx->device_bytes += (int64_t)bufs[i].size();
      e = cudaMemcpy(*a[i].ptr, bufs[i].data(), bufs[i].size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
      set_error(cudaGetErrorString(e));
      s = e == cudaErrorMemoryAllocation ? RMIPS_ERR_OOM : RMIPS_ERR_CUDA;
    }
    std::vector<unsigned char>().swap(bufs[i]);
  }
  (void)stream;
  if (s == RMIPS_OK) s = noalloc_prepare();          // the allocation-free call's scratch exists from here on
  if (s != RMIPS_OK) {
    rmips_free_index(idx);
    return s;
  }
  *out = idx;
  return RMIPS_OK;
}

extern "C" rmips_status rmips_index_rebuild(const rmips_index* cidx, int32_t k_max, void* stream, rmips_index** out) {
  if (out) *out = nullptr;
  if (!cidx || !out) { set_error("null argument"); return RMIPS_ERR_ARG; }
  if (k_max < 1 || k_max > RMIPS_KMAX_LIMIT) { set_error("k_max outside [1, 28]"); return RMIPS_ERR_ARG; }
  rmips_index* idx = const_cast<rmips_index*>(cidx);
  DevGuard g(idx->device);
  cudaStream_t st = (cudaStream_t)stream;
  float *Q = nullptr, *P = nullptr;
  const int64_t n = idx->n, m = idx->m;
  const int d = idx->d;
  cudaError_t e = cudaMallocAsync((void**)&Q, (size_t)n * d * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&P, (size_t)m * d * sizeof(float), st);
  if (e == cudaSuccess) {
    k_unsort_rows<<<(unsigned)((n * d + 255) / 256), 256, 0, st>>>(idx->Qs, idx->permQ, n, d, Q);
    k_unsort_rows<<<(unsigned)((m * d + 255) / 256), 256, 0, st>>>(idx->Ps, idx->permP, m, d, P);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  rmips_status s = RMIPS_OK;
  if (e != cudaSuccess) {
    set_error(cudaGetErrorString(e));
    s = e == cudaErrorMemoryAllocation ? RMIPS_ERR_OOM : RMIPS_ERR_CUDA;
  } else {
    rmips_build_opts o{};
    o.k_max = k_max;
    o.block_size = idx->bs;
    o.p_prime = idx->full_p ? 0 : idx->pp;
    o.precision = idx->precision;
    o.flags = (idx->batch_tc ? 0 : RMIPS_FLAG_BATCH_CUDA_CORES) | (idx->no_blocks ? RMIPS_FLAG_NO_BLOCK_FILTER : 0);
    s = rmips_build_index(Q, n, P, m, d, &o, stream, out);
    if (s == RMIPS_OK) {                                 // the same launch choices
      (*out)->tune_ws_ns = idx->tune_ws_ns;
      (*out)->tune_q1_ns = idx->tune_q1_ns;
      (*out)->tuned = idx->tuned;
    }
  }
  if (Q) cudaFreeAsync(Q, st);
  if (P) cudaFreeAsync(P, st);
  cudaStreamSynchronize(st);
  return s;
}
