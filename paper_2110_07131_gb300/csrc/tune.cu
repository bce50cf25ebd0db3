// Autotuner: launch choices of an index, searched on the device and kept in a
// cache file.
//
// The paper leaves the block size open (Definition 4: O(log n) users per
// block) and runs one query at a time on CPU cores (Section 4.3).  On the GPU
// the block size and the pipeline depths of the two filter kernels decide
// the speed, never the answer (every choice returns the exact set).  The
// search measures them on the index itself:
//   * block size b in {32, 64, 128, 256} (the block arrays are rebuilt from
//     the index's bounds, Equation 1) x query stages of the batched
//     tensor-core filter in {4, 8, ...} (as many as fit): the batched path's
//     time on 1,024 items of P spread over the norm order, with k cycling
//     through 1..k_max;
//   * then row stages of the single-query kernel in {2, ..., as many as fit}:
//     the time of 64 single queries (k = min(10, k_max)) launched back to back.
// The fastest choice is kept.  With a cache file, a line for the same shape,
// precision, index mode and GPU is read instead of searching, and a search
// appends its result, so a later build or process reuses it.
#include <chrono>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "rmips_internal.cuh"

namespace rmips {
namespace {

std::mutex g_cache_mu;

std::string cache_key(const rmips_index* idx) {
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, idx->device);
  char buf[512];
  snprintf(buf, sizeof(buf), "rmips-tune-1 n=%lld m=%lld d=%d k_max=%d precision=%d p_prime=%lld batch_tc=%d "
           "no_blocks=%d gpu=%s sms=%d",
           (long long)idx->n, (long long)idx->m, idx->d, idx->k_max, idx->precision, (long long)idx->pp,
           idx->batch_tc, idx->no_blocks, prop.name, prop.multiProcessorCount);
  for (char* c = buf; *c; ++c)
    if (*c == '|' || *c == '\n') *c = '_';
  return buf;
}

struct Choice {
  int bs = 32, ws_ns = 0, q1_ns = 0;
  float batch_ms = 0.f, single_ms = 0.f;
};

bool cache_read(const char* path, const std::string& key, Choice* c) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    char* bar = strstr(line, " | ");
    if (!bar) continue;
    *bar = 0;
    if (key != line) continue;
    Choice t;
    if (sscanf(bar + 3, "bs=%d batch_stages=%d single_stages=%d batch_ms=%f single_ms=%f", &t.bs, &t.ws_ns,
               &t.q1_ns, &t.batch_ms, &t.single_ms) == 5 &&
        (t.bs == 32 || t.bs == 64 || t.bs == 128 || t.bs == 256) && t.ws_ns >= 0 && t.ws_ns <= RMIPS_WS_MAXNS && (t.ws_ns & 1) == 0 &&
        t.q1_ns >= 0 && t.q1_ns <= 8) {
      *c = t;                       // the last valid line for the key wins
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_append(const char* path, const std::string& key, const Choice& c) {
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s | bs=%d batch_stages=%d single_stages=%d batch_ms=%.5f single_ms=%.6f\n", key.c_str(), c.bs,
          c.ws_ns, c.q1_ns, c.batch_ms, c.single_ms);
  fclose(f);
}

rmips_status search(rmips_index* idx, cudaStream_t st, Choice* best) {
  const int64_t nq = idx->m < 1024 ? idx->m : 1024;
  const int d = idx->d;
  float* dq = nullptr;
  int32_t* dk = nullptr;
  RMIPS_TRY_CUDA(cudaMalloc((void**)&dq, (size_t)nq * d * sizeof(float)));
  cudaError_t e = cudaMalloc((void**)&dk, (size_t)nq * sizeof(int32_t));
  // nq items of P spread over the norm order (the index keeps P sorted)
  const int64_t step = idx->m / nq;
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(dq, d * sizeof(float), idx->Ps, (size_t)step * d * sizeof(float), d * sizeof(float),
                          (size_t)nq, cudaMemcpyDeviceToDevice, st);
  std::vector<int32_t> hk((size_t)nq);
  for (int64_t i = 0; i < nq; ++i) hk[i] = 1 + (int32_t)((i * 7) % idx->k_max);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dk, hk.data(), nq * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  rmips_status s = RMIPS_OK;
  if (e != cudaSuccess) {
    set_error(cudaGetErrorString(e));
    s = RMIPS_ERR_CUDA;
  }
  const int bs0 = idx->bs;
  const int ns_max = max_batch_stages(idx);
  const bool tc = idx->batch_tc && idx->d <= 64 && idx->Qtc;
  float best_ms = 1e30f;
  const int sizes[4] = {32, 64, 128, 256};
  for (int bi = 0; s == RMIPS_OK && bi < 4; ++bi) {
    if (idx->no_blocks && sizes[bi] != bs0) continue;          // no block bounds: the size does not matter
    if ((s = set_block_size(idx, sizes[bi], st)) != RMIPS_OK) break;
    for (int ns = RMIPS_WS_NMMA; s == RMIPS_OK && ns <= (tc ? ns_max : RMIPS_WS_NMMA); ns += RMIPS_WS_NMMA) {
      idx->tune_ws_ns = tc ? ns : 0;
      float ms = 0.f;
      if ((s = tune_time_batch(idx, dq, dk, nq, 3, st, &ms)) != RMIPS_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        best->bs = sizes[bi];
        best->ws_ns = tc ? ns : 0;
        best->batch_ms = ms;
      }
    }
  }
  if (s == RMIPS_OK) s = set_block_size(idx, best->bs, st);
  idx->tune_ws_ns = best->ws_ns;
  if (s == RMIPS_OK && idx->full_p) {
    const int q_max = max_single_stages(idx);
    const int k = idx->k_max < 10 ? idx->k_max : 10;
    const int64_t n1 = nq < 64 ? nq : 64;
    float best1 = 1e30f;
    for (int ns = 2 > q_max ? q_max : 2; s == RMIPS_OK && ns <= q_max; ++ns) {
      idx->tune_q1_ns = ns;
      float ms = 0.f;
      if ((s = tune_time_single(idx, dq, n1, k, st, &ms)) != RMIPS_OK) break;
      if (ms < best1) {
        best1 = ms;
        best->q1_ns = ns;
        best->single_ms = ms;
      }
    }
    idx->tune_q1_ns = best->q1_ns;
  }
  cudaFree(dq);
  cudaFree(dk);
  if (s != RMIPS_OK) {                 // leave the index as it was built
    idx->tune_ws_ns = idx->tune_q1_ns = 0;
    set_block_size(idx, bs0, st);
  }
  return s;
}

}  // namespace

rmips_status tune_index(rmips_index* idx, const char* cache, cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  const std::string key = cache_key(idx);
  Choice c;
  bool hit = false;
  if (cache) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    hit = cache_read(cache, key, &c);
  }
  rmips_status s = RMIPS_OK;
  if (hit) {
    if ((s = set_block_size(idx, c.bs, st)) != RMIPS_OK) return s;
    idx->tune_ws_ns = c.ws_ns > max_batch_stages(idx) ? max_batch_stages(idx) : c.ws_ns;
    idx->tune_q1_ns = c.q1_ns > max_single_stages(idx) ? max_single_stages(idx) : c.q1_ns;
    idx->tuned = 2;
  } else {
    if ((s = search(idx, st, &c)) != RMIPS_OK) return s;
    idx->tuned = 1;
    if (cache) {
      std::lock_guard<std::mutex> lk(g_cache_mu);
      cache_append(cache, key, c);
    }
  }
  idx->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return RMIPS_OK;
}

}  // namespace rmips

using namespace rmips;

extern "C" rmips_status rmips_index_tune(rmips_index* idx, const char* tune_cache, void* stream) {
  if (!idx) { set_error("null argument"); return RMIPS_ERR_ARG; }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != idx->device) cudaSetDevice(idx->device);
  const rmips_status s = tune_index(idx, tune_cache, (cudaStream_t)stream);
  if (prev != idx->device) cudaSetDevice(prev);
  return s;
}
