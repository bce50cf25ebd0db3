// C ABI glue: errors, workspaces, index inspection and release.
#include <cstdio>

#include "rmips_internal.cuh"

namespace rmips {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error state of the query
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int ptr_class(const void* p, int device) {
  cudaPointerAttributes a{};
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return PTR_HOST;
  }
  return ptr_class_of((int)a.type, a.device, device);
}

rmips_status check_ptr_device(const void* p, int device, const char* what) {
  if (ptr_class(p, device) != PTR_OTHER_DEVICE) return RMIPS_OK;
  set_error(std::string(what) + " is device memory of another GPU than the index's");
  return RMIPS_ERR_ARG;
}

void destroy_workspace(Workspace* ws) {
  if (!ws) return;
  if (ws->done_ev) cudaEventDestroy(ws->done_ev);
  for (auto& pg : ws->pgraph) {
    if (pg.pre) cudaGraphExecDestroy(pg.pre);
    if (pg.post) cudaGraphExecDestroy(pg.post);
  }
  ws->pgraph.clear();
  if (ws->cap_stream) cudaStreamDestroy(ws->cap_stream);
  cudaFree(ws->yes);
  cudaFree(ws->todo);
  cudaFree(ws->bitmap);
  cudaFree(ws->ctr);
  cudaFree(ws->dq);
  cudaFree(ws->dk);
  cudaFree(ws->dqn);
  cudaFree(ws->deps);
  cudaFree(ws->doffs);
  cudaFree(ws->dout);
  cudaFreeHost(ws->h_ctr);
  cudaFreeHost(ws->h_offs);
  cudaFreeHost(ws->h_out);
  cudaFreeHost(ws->h_q);
  cudaFreeHost(ws->h_res);
  cudaFree(ws->dres);
  for (cudaEvent_t e : ws->ev) cudaEventDestroy(e);
  cudaFree(ws->bq);
  cudaFree(ws->bk);
  cudaFree(ws->bqn);
  cudaFree(ws->beps);
  cudaFree(ws->bidx);
  cudaFree(ws->grp);
  cudaFree(ws->qcnt);
  cudaFree(ws->qcur);
  cudaFree(ws->ypairs);
  cudaFree(ws->tpairs);
  cudaFree(ws->seg);
  cudaFree(ws->keys);
  cudaFree(ws->runs);
  cudaFree(ws->gfirst);
  cudaFree(ws->gslot0);
  cudaFree(ws->dseglo);
  cudaFree(ws->dseghi);
  cudaFree(ws->hist);
  cudaFree(ws->big);
  cudaFree(ws->mid);
  cudaFree(ws->bslot);
  cudaFree(ws->bigcnt);
  cudaFree(ws->bigmaps);
  cudaFree(ws->bcq);
  cudaFree(ws->bitems);
  cudaFree(ws->gitem);
  cudaFree(ws->itemg);
  cudaFree(ws->gpre);
  cudaFree(ws->wst);
  delete ws;
}

// Idle workspaces are kept in the order they were released.  The oldest
// whose queued device work has finished is taken; while all of them still
// have work in flight (asynchronous batches queued back to back, e.g. on two
// streams in turn), a second workspace is created so that consecutive batches
// do not wait for each other; beyond that the oldest is taken and the call
// waits for its work (ws_join).  Taking the oldest keeps a stream of batches
// cycling through the workspaces in a fixed order, so each one replays its
// own captured graphs.
constexpr int kOverlapWorkspaces = 2;

Workspace* acquire_workspace(rmips_index* idx, rmips_status* st) {
  {
    std::lock_guard<std::mutex> lk(idx->mu);
    for (size_t i = 0; i < idx->pool.size(); ++i) {
      Workspace* ws = idx->pool[i];
      if (ws->done_pending && cudaEventQuery(ws->done_ev) != cudaSuccess) {
        cudaGetLastError();                    // "not ready" is not an error of the next call
        continue;
      }
      idx->pool.erase(idx->pool.begin() + (ptrdiff_t)i);
      return ws;
    }
    if (!idx->pool.empty() && idx->n_ws >= kOverlapWorkspaces) {
      Workspace* ws = idx->pool.front();
      idx->pool.erase(idx->pool.begin());
      return ws;
    }
    ++idx->n_ws;
  }
  Workspace* ws = new Workspace();
  const int64_t n = idx->n;
  const int64_t nw = n / 32 + 1;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc((void**)&ws->yes, n * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ws->todo, n * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ws->bitmap, nw * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ws->ctr, C_NCOUNTERS * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(ws->bitmap, 0, nw * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(ws->ctr, 0, C_NCOUNTERS * sizeof(long long));
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&ws->h_ctr, C_NCOUNTERS * sizeof(long long), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&ws->h_out, n * sizeof(long long), cudaHostAllocMapped);
  if (e == cudaSuccess) ws->cap_hout = n;
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&ws->h_q, RMIPS_DMAX * sizeof(float), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&ws->h_res, (2 + C_NCOUNTERS) * sizeof(long long), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    set_error(std::string("workspace allocation: ") + cudaGetErrorString(e));
    *st = e == cudaErrorMemoryAllocation ? RMIPS_ERR_OOM : RMIPS_ERR_CUDA;
    destroy_workspace(ws);
    std::lock_guard<std::mutex> lk(idx->mu);
    --idx->n_ws;
    return nullptr;
  }
  return ws;
}

rmips_status ws_join(Workspace* ws, cudaStream_t st) {
  if (ws->done_pending) {
    // on the stream that queued the work, stream order already joins it
    if (ws->done_stream != st) RMIPS_TRY_CUDA(cudaStreamWaitEvent(st, ws->done_ev, 0));
    ws->done_pending = false;
  }
  return RMIPS_OK;
}

void release_workspace(rmips_index* idx, Workspace* ws) {
  std::lock_guard<std::mutex> lk(idx->mu);
  idx->pool.push_back(ws);
}

}  // namespace rmips

using namespace rmips;

extern "C" const char* rmips_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* rmips_status_string(rmips_status s) {
  switch (s) {
    case RMIPS_OK: return "ok";
    case RMIPS_ERR_ARG: return "invalid argument";
    case RMIPS_ERR_K_RANGE: return "k outside [1, k_max]";
    case RMIPS_ERR_NONFINITE: return "non-finite input";
    case RMIPS_ERR_OOM: return "out of memory";
    case RMIPS_ERR_CAPACITY: return "output capacity too small";
    case RMIPS_ERR_TIMEOUT: return "device wait timed out";
    case RMIPS_ERR_CUDA: return "CUDA runtime error";
    case RMIPS_ERR_INTERNAL: return "internal consistency check failed";
    case RMIPS_ERR_BUSY: return "admission refused: too many requests pending";
  }
  return "unknown status";
}

extern "C" rmips_status rmips_index_get_info(const rmips_index* idx, rmips_index_info* out) {
  if (!idx || !out) { set_error("null argument"); return RMIPS_ERR_ARG; }
  rmips_index_info i{};
  i.n = idx->n;
  i.m = idx->m;
  i.d = idx->d;
  i.k_max = idx->k_max;
  i.block_size = idx->bs;
  i.precision = idx->precision;
  i.n_blocks = idx->nb;
  i.p_prime = idx->pp;
  i.incomplete = idx->incomplete;
  i.device_bytes = idx->device_bytes;
  i.build_ms = idx->build_ms;
  i.tuned = idx->tuned;
  i.batch_stages = idx->tune_ws_ns;
  i.single_stages = idx->tune_q1_ns;
  i.build_kind = idx->build_kind;
  i.tune_ms = idx->tune_ms;
  *out = i;
  return RMIPS_OK;
}

extern "C" rmips_status rmips_last_query_stats(const rmips_index* idx, rmips_query_stats* out) {
  if (!idx || !out) { set_error("null argument"); return RMIPS_ERR_ARG; }
  rmips_index* m = const_cast<rmips_index*>(idx);
  std::lock_guard<std::mutex> lk(m->mu);
  *out = m->last_stats;
  return RMIPS_OK;
}

extern "C" rmips_status rmips_index_export(const rmips_index* idx, int32_t field, void* dst, int64_t bytes) {
  if (!idx || !dst) { set_error("null argument"); return RMIPS_ERR_ARG; }
  const void* src = nullptr;
  int64_t need = 0;
  std::vector<float2> tmp;
  switch (field) {
    case 0: src = idx->permQ; need = idx->n * 4; break;
    case 1: src = idx->permP; need = idx->m * 4; break;
    case 2: case 3: need = (int64_t)idx->k_max * idx->n * 4; break;
    case 4: src = idx->LB; need = (int64_t)idx->k_max * idx->nb * 4; break;
    case 5: src = idx->hdr; need = idx->nb * 4; break;
    case 6: src = idx->unorm; need = idx->n * 4; break;
    case 7: src = idx->pnorm; need = idx->m * 4; break;
    case 8: src = idx->incomp; need = idx->full_p ? idx->n : 0; break;
    default: set_error("unknown field"); return RMIPS_ERR_ARG;
  }
  if (bytes != need) { set_error("byte count does not match the field size"); return RMIPS_ERR_ARG; }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != idx->device) cudaSetDevice(idx->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) {
    if (field == 2 || field == 3) {
      tmp.resize((size_t)idx->k_max * idx->n);
      e = cudaMemcpy(tmp.data(), idx->Lb, tmp.size() * sizeof(float2), cudaMemcpyDeviceToHost);
      float* f = (float*)dst;
      for (size_t i = 0; i < tmp.size(); ++i) f[i] = field == 2 ? tmp[i].x : tmp[i].y;
    } else if (need > 0) {
      e = cudaMemcpy(dst, src, need, cudaMemcpyDeviceToHost);
    }
  }
  if (prev != idx->device) cudaSetDevice(prev);
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return RMIPS_ERR_CUDA; }
  return RMIPS_OK;
}

extern "C" void rmips_free_index(rmips_index* idx) {
  if (!idx) return;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != idx->device) cudaSetDevice(idx->device);
  cudaDeviceSynchronize();
  for (Workspace* ws : idx->pool) destroy_workspace(ws);
  idx->pool.clear();
  cudaFree(idx->Qs);
  cudaFree(idx->Qh);
  cudaFree(idx->Ps);
  cudaFree(idx->unorm);
  cudaFree(idx->pnorm);
  cudaFree(idx->permQ);
  cudaFree(idx->permP);
  cudaFree(idx->Lb);
  cudaFree(idx->cand);
  cudaFree(idx->cbnd);
  cudaFree(idx->dprof);
  cudaFree(idx->dprof1);
  for (cudaEvent_t e : idx->pend_ev) cudaEventDestroy(e);
  idx->pend_ev.clear();
  for (cudaEvent_t e : idx->pend_ev1) cudaEventDestroy(e);
  idx->pend_ev1.clear();
  cudaFree(idx->incomp);
  cudaFree(idx->LB);
  cudaFree(idx->hdr);
  cudaFree(idx->Qtc);
  if (prev != idx->device) cudaSetDevice(prev);
  delete idx;
}

extern "C" int32_t rmips_exact_sign_host(const float* u, const float* a, const float* b, int32_t d) {
  if (!u || !a || !b || d < 1 || d > 256) return 0;
  return (int32_t)exact_sign_diff(u, a, b, d);
}

extern "C" rmips_status rmips_profile_enable(rmips_index* idx, int32_t enable) {
  if (!idx) { set_error("null argument"); return RMIPS_ERR_ARG; }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != idx->device) cudaSetDevice(idx->device);
  std::lock_guard<std::mutex> lk(idx->mu);
  idx->prof_on = enable == 2 ? 2 : (enable ? 1 : 0);
  idx->prof = rmips_profile{};
  for (cudaEvent_t e : idx->pend_ev) {
    cudaEventSynchronize(e);
    cudaEventDestroy(e);
  }
  idx->pend_ev.clear();
  for (cudaEvent_t e : idx->pend_ev1) {
    cudaEventSynchronize(e);
    cudaEventDestroy(e);
  }
  idx->pend_ev1.clear();
  cudaError_t e = cudaSuccess;
  if (!idx->dprof) e = cudaMalloc((void**)&idx->dprof, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(idx->dprof, 0, sizeof(unsigned long long));
  if (e == cudaSuccess && !idx->dprof1) e = cudaMalloc((void**)&idx->dprof1, 4 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(idx->dprof1, 0, 4 * sizeof(unsigned long long));
  if (prev != idx->device) cudaSetDevice(prev);
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return RMIPS_ERR_CUDA; }
  return RMIPS_OK;
}

// Folds the filter timing and kept-pair counts of asynchronous batch calls
// (event pairs and a device counter, waited for here) into the profile.
extern "C" rmips_status rmips_profile_read(const rmips_index* idx, rmips_profile* out) {
  if (!idx || !out) { set_error("null argument"); return RMIPS_ERR_ARG; }
  rmips_index* m = const_cast<rmips_index*>(idx);
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != m->device) cudaSetDevice(m->device);
  std::lock_guard<std::mutex> lk(m->mu);
  for (size_t i = 0; i + 1 < m->pend_ev.size(); i += 2) {
    float ms = 0.f;
    if (cudaEventSynchronize(m->pend_ev[i + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, m->pend_ev[i], m->pend_ev[i + 1]) == cudaSuccess) {
      m->prof.mfilter_launches += 1;
      m->prof.mfilter_ms += ms;
    }
  }
  for (cudaEvent_t e : m->pend_ev) cudaEventDestroy(e);
  m->pend_ev.clear();
  unsigned long long pairs = 0;
  if (m->dprof && cudaMemcpy(&pairs, m->dprof, sizeof(pairs), cudaMemcpyDeviceToHost) == cudaSuccess && pairs) {
    m->prof.mfilter_pairs += (int64_t)pairs;
    m->prof.mfilter_alg_flops += 2.0 * m->d * (double)pairs;
    cudaMemset(m->dprof, 0, sizeof(unsigned long long));
  }
  // asynchronous single queries: event pairs and the device counters
  for (size_t i = 0; i + 1 < m->pend_ev1.size(); i += 2) {
    float ms = 0.f;
    if (cudaEventSynchronize(m->pend_ev1[i + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, m->pend_ev1[i], m->pend_ev1[i + 1]) == cudaSuccess)
      m->prof.filter_ms += ms;
  }
  for (cudaEvent_t e : m->pend_ev1) cudaEventDestroy(e);
  m->pend_ev1.clear();
  unsigned long long acc[4] = {0, 0, 0, 0};
  if (m->dprof1 && cudaMemcpy(acc, m->dprof1, sizeof(acc), cudaMemcpyDeviceToHost) == cudaSuccess && acc[3]) {
    const int es = m->precision == RMIPS_FP32 ? 4 : 2;
    m->prof.filter_launches += (int64_t)acc[3];
    m->prof.filter_alg_bytes += 8.0 * m->nb * (double)acc[3] + ((double)m->d * es + 12.0) * (double)acc[0] +
                                4.0 * (double)acc[1];
    m->prof.users_tested += (int64_t)acc[0];
    m->prof.blocks_pruned += (int64_t)acc[2] * 32 / m->bs;
    m->prof.blocks_total += m->nb * (int64_t)acc[3];
    cudaMemset(m->dprof1, 0, sizeof(acc));
  }
  *out = m->prof;
  if (prev != m->device) cudaSetDevice(prev);
  return RMIPS_OK;
}
