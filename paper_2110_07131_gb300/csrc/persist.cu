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

namespace rmips {
namespace {

constexpr char kMagic[8] = {'R', 'M', 'I', 'P', 'S', 'I', 'X', '1'};

struct FileHeader {
  char magic[8];
  int64_t n, m, nb, pp, incomplete;
  int32_t d, k_max, bs, precision, full_p, batch_tc, no_blocks, has_qh, has_qtc, narrays;
  float pn0;
};

// The device arrays of an index in file order: pointer slot and byte size.
struct ArrayRef {
  void** ptr;
  int64_t bytes;
};

std::vector<ArrayRef> arrays(rmips_index* idx, bool has_qh, bool has_qtc) {
  const int64_t n = idx->n, m = idx->m, d = idx->d, pad = 32 * d;
  const int64_t tiles = (n + 127) / 128;
  const int64_t tile_bytes = 128 * 64 * (idx->precision == RMIPS_FP32 ? 4 : 2);
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
  }
  ok = (fclose(f) == 0) && ok;
  if (!ok) { set_error(std::string("writing ") + path + " failed"); return RMIPS_ERR_ARG; }
  return RMIPS_OK;
}

extern "C" rmips_status rmips_index_load(const char* path, void* stream, rmips_index** out) {
  if (out) *out = nullptr;
  if (!path || !out) { set_error("null argument"); return RMIPS_ERR_ARG; }
  FILE* f = fopen(path, "rb");
  if (!f) { set_error(std::string("cannot open ") + path); return RMIPS_ERR_ARG; }
  FileHeader h{};
  if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, kMagic, sizeof(kMagic)) != 0 || h.n < 1 || h.m < 1 ||
      h.d < 1 || h.d > RMIPS_DMAX || h.k_max < 1 || h.k_max > RMIPS_KMAX_LIMIT) {
    fclose(f);
    set_error(std::string(path) + " is not an index file of this library");
    return RMIPS_ERR_ARG;
  }
  rmips_index* idx = new rmips_index();
  idx->n = h.n; idx->m = h.m; idx->nb = h.nb; idx->pp = h.pp; idx->incomplete = h.incomplete;
  idx->d = h.d; idx->k_max = h.k_max; idx->bs = h.bs; idx->precision = h.precision; idx->full_p = h.full_p;
  idx->batch_tc = h.batch_tc; idx->no_blocks = h.no_blocks; idx->pn0 = h.pn0;
  cudaGetDevice(&idx->device);
  const std::vector<ArrayRef> a = arrays(idx, h.has_qh != 0, h.has_qtc != 0);
  rmips_status s = RMIPS_OK;
  if ((int32_t)a.size() != h.narrays) {
    set_error(std::string(path) + ": array count does not match its header");
    s = RMIPS_ERR_ARG;
  }
  std::vector<unsigned char> buf;
  for (size_t i = 0; s == RMIPS_OK && i < a.size(); ++i) {
    int64_t bytes = -1;
    if (fread(&bytes, sizeof(bytes), 1, f) != 1 || bytes != a[i].bytes) {
      set_error(std::string(path) + ": array sizes do not match its header");
      s = RMIPS_ERR_ARG;
      break;
    }
    buf.resize((size_t)bytes);
    if (fread(buf.data(), 1, (size_t)bytes, f) != (size_t)bytes) {
      set_error(std::string(path) + " is truncated");
      s = RMIPS_ERR_ARG;
      break;
    }
    cudaError_t e = cudaMalloc(a[i].ptr, (size_t)bytes);
    if (e == cudaSuccess) {
      idx->device_bytes += bytes;
      e = cudaMemcpy(*a[i].ptr, buf.data(), (size_t)bytes, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
      set_error(cudaGetErrorString(e));
      s = e == cudaErrorMemoryAllocation ? RMIPS_ERR_OOM : RMIPS_ERR_CUDA;
    }
  }
  fclose(f);
  (void)stream;
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
  }
  if (Q) cudaFreeAsync(Q, st);
  if (P) cudaFreeAsync(P, st);
  cudaStreamSynchronize(st);
  return s;
}
