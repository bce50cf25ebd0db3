// Serving loop: continuous batching of reverse k-MIPS requests.
//
// Requests (q, k, optional segment) are queued by rmips_server_submit.  A
// dispatcher thread closes a batch when it holds max_batch requests, when
// their result reservations fill a slot's result buffer, or when its oldest
// request has waited max_wait_us, and launches it on a free stream slot (each
// slot owns a workspace, pinned staging, a device result buffer and a pinned
// copy of it); requests that arrive in the meantime wait for the next batch,
// so up to `streams` batches overlap on the GPU.  Every segment kind is
// answered inside the batch: id ranges on the device, id lists and
// registered segments by intersecting the request's exact unrestricted
// result with the (sorted) list afterwards.  A completer thread finishes
// slots in launch order, copies each request's ids out and records its
// latency (submit to completion).
//
// Admission by device memory: every queued or running request reserves
// result slots in the slots' device result buffers (min(result_ids_per_request,
// its segment's size) ids of 8 bytes); a submission whose reservation would
// take the total past the buffers' capacity (streams x cap_out ids, sized
// from max_device_bytes, itself by default an eighth of the device's free
// memory at creation) is refused with RMIPS_ERR_BUSY, as is one past
// max_pending requests.  A batch whose actual results overflow its buffer
// (reservations are estimates) is answered one request at a time.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "rmips_internal.cuh"

using Clock = std::chrono::steady_clock;

namespace rmips {
namespace {

struct Request {
  std::vector<float> q;
  int32_t k = 1;
  int kind = 0;                 // 0 all users, 1 id range, 2 id list, 3 registered segment
  int64_t lo = 0, hi = INT64_MAX;
  std::vector<int64_t> list;    // kind 2: sorted, distinct ids
  int32_t handle = -1;          // kind 3
  int64_t reserve = 0;          // result ids reserved (admission)
  Clock::time_point t0;
  int state = 0;                // 0 queued, 1 running, 2 done
  rmips_status st = RMIPS_OK;
  std::vector<int64_t> ids;
  double ms = 0.0;
};

struct Slot {
  Workspace* ws = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  float* h_q = nullptr;         // pinned staging
  int32_t* h_k = nullptr;
  long long* h_lo = nullptr;
  long long* h_hi = nullptr;
  long long* h_offs = nullptr;
  long long* h_ctr = nullptr;
  long long* d_out = nullptr;   // device result ids of a batch
  long long* h_out = nullptr;   // pinned, device-mapped copy of them
  int64_t cap_out = 0;
  long long* d_done = nullptr;  // small batches: (status, count) per request, device
  long long* h_done = nullptr;  // and its pinned copy
  std::vector<int64_t> tickets;
  bool segments = false;
  bool small = false;           // run as one-launch single queries
  rmips_status launch = RMIPS_OK;
  bool busy = false;
};

constexpr size_t LAT_CAP = 1 << 20;

// Small batches: request i's ids (done[2i + 1] of them, when its status is
// RMIPS_OK) from its region of `per` ids into mapped host memory.
__global__ void k_serve_copy_regions(const long long* __restrict__ src, long long* __restrict__ dst,
                                     const long long* __restrict__ done, int nq, long long per) {
  for (int i = blockIdx.y; i < nq; i += gridDim.y) {
    if (done[2 * i] != RMIPS_OK) continue;
    const long long cnt = done[2 * i + 1] < per ? done[2 * i + 1] : per;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < cnt; j += (long long)gridDim.x * blockDim.x)
      dst[i * per + j] = src[i * per + j];
  }
}

// The first min(total, cap) result ids of a batch into mapped host memory.
__global__ void k_serve_copy(const long long* __restrict__ src, long long* __restrict__ dst,
                             const long long* __restrict__ ctr, long long cap) {
  if (ctr[C_STATUS] != 0) return;
  const long long n = ctr[C_CURSOR] < cap ? ctr[C_CURSOR] : cap;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

}  // namespace
}  // namespace rmips

struct rmips_server {
  rmips_index* idx = nullptr;
  rmips_server_opts o{};
  std::mutex mu;
  std::condition_variable cv_in, cv_slot, cv_fly, cv_done;
  std::atomic<uint64_t> ver{0};    // bumped on every change a waiter may be waiting for (spin_us)
  std::unordered_map<int64_t, rmips::Request*> reqs;
  std::deque<int64_t> queue;
  std::vector<rmips::Slot> slots;
  std::deque<int> inflight;
  std::vector<std::vector<int64_t>> segs;    // registered segments (sorted, distinct)
  int64_t next = 1, pending = 0;
  int64_t reserved = 0, capacity = 0;        // result ids reserved / reservable (admission)
  bool stop = false;
  std::thread disp, comp;
  int64_t submitted = 0, completed = 0, rejected = 0, batches = 0, batched = 0, one_by_one = 0;
  std::vector<double> lat;
  size_t lat_n = 0;
};

using namespace rmips;

namespace {

void record_latency(rmips_server* S, double ms) {
  if (S->lat.size() < LAT_CAP) S->lat.push_back(ms);
  else S->lat[S->lat_n % LAT_CAP] = ms;
  ++S->lat_n;
}

const std::vector<int64_t>* seg_list(const rmips_server* S, const Request* r) {
  if (r->kind == 2) return &r->list;
  if (r->kind == 3) return &S->segs[(size_t)r->handle];
  return nullptr;
}

// ids (ascending) restricted to the request's id list, if it has one.
void restrict_to_list(const rmips_server* S, const Request* r, std::vector<int64_t>& ids) {
  const std::vector<int64_t>* L = seg_list(S, r);
  if (!L) return;
  size_t w = 0;
  for (int64_t id : ids)
    if (std::binary_search(L->begin(), L->end(), id)) ids[w++] = id;
  ids.resize(w);
}

// One request through the single-query path (when a batch's results overflow).
void run_single(rmips_server* S, Request* r, std::vector<int64_t>& ids, rmips_status& st) {
  rmips_segment seg{};
  const std::vector<int64_t>* L = seg_list(S, r);
  seg.kind = L ? 2 : r->kind;
  seg.begin = r->lo;
  seg.end = r->hi;
  seg.ids = L ? L->data() : nullptr;
  seg.n_ids = L ? (int64_t)L->size() : 0;
  ids.resize((size_t)S->idx->n);
  int64_t cnt = 0;
  st = rmips_query(S->idx, r->q.data(), r->k, r->kind ? &seg : nullptr, ids.data(), S->idx->n, &cnt, nullptr);
  ids.resize(st == RMIPS_OK ? (size_t)cnt : 0);
}

void finish(rmips_server* S, Request* r, std::vector<int64_t>&& ids, rmips_status st, Clock::time_point now) {
  r->ids = std::move(ids);
  r->st = st;
  r->ms = std::chrono::duration<double, std::milli>(now - r->t0).count();
  r->state = 2;
  record_latency(S, r->ms);
  ++S->completed;
  --S->pending;
  S->reserved -= r->reserve;
}

rmips_status launch_slot(rmips_server* S, Slot& sl, int64_t nq) {
  rmips_index* idx = S->idx;
  Workspace* ws = sl.ws;
  cudaStream_t st = sl.stream;
  RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->dq, sl.h_q, nq * idx->d * sizeof(float), cudaMemcpyHostToDevice, st));
  RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->dk, sl.h_k, nq * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  if (sl.small) {                                   // one launch per request, on this slot's stream
    const long long per = sl.cap_out / nq;
    for (int64_t i = 0; i < nq; ++i) {
      rmips_status s = single_launch(idx, ws, ws->dq + i * idx->d, sl.h_k[i], sl.h_lo[i], sl.h_hi[i],
                                     sl.d_out + i * per, per, sl.d_done + 2 * i, st);
      if (s != RMIPS_OK) return s;
    }
    k_serve_copy_regions<<<dim3(16, (unsigned)nq), 256, 0, st>>>(sl.d_out, sl.h_out, sl.d_done, (int)nq, per);
    RMIPS_TRY_CUDA(cudaGetLastError());
    RMIPS_TRY_CUDA(cudaMemcpyAsync(sl.h_done, sl.d_done, 2 * nq * sizeof(long long), cudaMemcpyDeviceToHost, st));
    RMIPS_TRY_CUDA(cudaEventRecord(sl.done, st));
    return RMIPS_OK;
  }
  if (sl.segments) {
    RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->dseglo, sl.h_lo, nq * sizeof(long long), cudaMemcpyHostToDevice, st));
    RMIPS_TRY_CUDA(cudaMemcpyAsync(ws->dseghi, sl.h_hi, nq * sizeof(long long), cudaMemcpyHostToDevice, st));
  }
  rmips_status s = batch_launch(idx, ws, nq, sl.d_out, sl.cap_out, st, sl.segments);
  if (s != RMIPS_OK) return s;
  k_serve_copy<<<128, 256, 0, st>>>(sl.d_out, sl.h_out, ws->ctr, sl.cap_out);
  RMIPS_TRY_CUDA(cudaGetLastError());
  RMIPS_TRY_CUDA(cudaMemcpyAsync(sl.h_offs, ws->doffs, (nq + 1) * sizeof(long long), cudaMemcpyDeviceToHost, st));
  RMIPS_TRY_CUDA(cudaMemcpyAsync(sl.h_ctr, ws->ctr, C_NCOUNTERS * sizeof(long long), cudaMemcpyDeviceToHost, st));
  RMIPS_TRY_CUDA(cudaEventRecord(sl.done, st));
  return RMIPS_OK;
}

// Every notification of the server's condition variables goes through here,
// so that threads spinning on `ver` (spin_us > 0) see the change too.
void bump(rmips_server* S) { S->ver.fetch_add(1, std::memory_order_release); }

// With spin_us > 0: polls pred (under the lock, after each change of `ver`)
// for up to spin_us before the caller blocks.  Returns with the lock held;
// true when pred holds.
template <class P>
bool spin_for(rmips_server* S, std::unique_lock<std::mutex>& lk, P pred) {
  if (pred()) return true;
  if (S->o.spin_us <= 0) return false;
  const auto end = Clock::now() + std::chrono::microseconds(S->o.spin_us);
  uint64_t v = S->ver.load(std::memory_order_acquire);
  lk.unlock();
  for (;;) {
    const uint64_t w = S->ver.load(std::memory_order_acquire);
    if (w != v) {
      lk.lock();
      if (pred()) return true;
      lk.unlock();
      v = w;
    }
    if (Clock::now() >= end) break;
  }
  lk.lock();
  return pred();
}

void dispatcher(rmips_server* S) {
  cudaSetDevice(S->idx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    auto any_in = [&] { return S->stop || !S->queue.empty(); };
    if (!spin_for(S, lk, any_in)) S->cv_in.wait(lk, any_in);
    if (S->stop) break;
    // close the batch at once when no batch is on the device (waiting would
    // only add latency), else when it is full or its oldest request has
    // waited max_wait_us; requests arriving meanwhile join it
    const auto deadline = S->reqs[S->queue.front()]->t0 + std::chrono::microseconds(S->o.max_wait_us);
    while (!S->stop && !S->inflight.empty() && (int64_t)S->queue.size() < S->o.max_batch && Clock::now() < deadline)
      S->cv_in.wait_until(lk, deadline);
    if (S->stop) break;
    int si = -1;
    auto free_slot = [&] {
      if (S->stop) return true;
      for (int i = 0; i < (int)S->slots.size(); ++i)
        if (!S->slots[i].busy) { si = i; return true; }
      return false;
    };
    if (!spin_for(S, lk, free_slot)) S->cv_slot.wait(lk, free_slot);
    if (S->stop) break;
    Slot& sl = S->slots[si];
    sl.busy = true;
    sl.tickets.clear();
    sl.segments = false;
    std::vector<Request*> batch;
    int64_t ids_reserved = 0;
    while (!S->queue.empty() && (int64_t)batch.size() < S->o.max_batch) {
      const int64_t t = S->queue.front();
      Request* r = S->reqs[t];
      if (!batch.empty() && ids_reserved + r->reserve > sl.cap_out) break;   // the slot's result buffer is full
      S->queue.pop_front();
      r->state = 1;
      ids_reserved += r->reserve;
      sl.tickets.push_back(t);
      batch.push_back(r);
      sl.segments = sl.segments || r->kind == 1;
    }
    lk.unlock();
    const int64_t nq = (int64_t)batch.size();
    sl.small = S->idx->full_p && nq <= S->o.single_max;
    const int d = S->idx->d;
    for (int64_t i = 0; i < nq; ++i) {
      memcpy(sl.h_q + i * d, batch[i]->q.data(), d * sizeof(float));
      sl.h_k[i] = batch[i]->k;
      sl.h_lo[i] = batch[i]->kind == 1 ? batch[i]->lo : 0;
      sl.h_hi[i] = batch[i]->kind == 1 ? batch[i]->hi : INT64_MAX;
    }
    sl.launch = launch_slot(S, sl, nq);
    lk.lock();
    S->inflight.push_back(si);
    ++S->batches;
    S->batched += nq;
    S->cv_fly.notify_one();
    bump(S);
  }
  // stopped: fail whatever is still queued
  const auto now = Clock::now();
  while (!S->queue.empty()) {
    Request* r = S->reqs[S->queue.front()];
    S->queue.pop_front();
    finish(S, r, {}, RMIPS_ERR_ARG, now);
  }
  S->cv_done.notify_all();
  bump(S);
}

void completer(rmips_server* S) {
  cudaSetDevice(S->idx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    auto any_fly = [&] { return S->stop || !S->inflight.empty(); };
    if (!spin_for(S, lk, any_fly)) S->cv_fly.wait(lk, any_fly);
    if (S->inflight.empty()) {
      if (S->stop) break;
      continue;
    }
    const int si = S->inflight.front();
    S->inflight.pop_front();
    Slot& sl = S->slots[si];
    std::vector<Request*> rs;
    for (int64_t t : sl.tickets) rs.push_back(S->reqs[t]);
    lk.unlock();
    const int64_t nq = (int64_t)rs.size();
    rmips_status st = sl.launch;
    bool one_by_one = false;
    if (st == RMIPS_OK) {
      if (S->o.spin_us > 0) {                     // poll the batch's event before blocking on it
        const auto end = Clock::now() + std::chrono::microseconds(S->o.spin_us);
        while (cudaEventQuery(sl.done) == cudaErrorNotReady && Clock::now() < end) {
        }
      }
      if (cudaEventSynchronize(sl.done) != cudaSuccess) {
        set_error("batch failed on the device");
        st = RMIPS_ERR_CUDA;
      } else if (!sl.small) {
        // results past the buffer, or a full pair list (ties-heavy batch):
        // answered one request at a time (small batches carry a status per
        // request instead)
        one_by_one = sl.h_ctr[C_STATUS] == ST_PAIRS_FULL || sl.h_ctr[C_STATUS] == ST_CAPACITY;
        st = device_status(sl.h_ctr[C_STATUS]);
      }
    }
    std::vector<std::vector<int64_t>> res(nq);
    std::vector<rmips_status> sts(nq, st);
    if (st == RMIPS_OK && sl.small) {
      const long long per = sl.cap_out / nq;
      for (int64_t i = 0; i < nq; ++i) {
        const long long code = sl.h_done[2 * i], cnt = sl.h_done[2 * i + 1];
        if (code == RMIPS_OK) {
          res[i].assign(sl.h_out + i * per, sl.h_out + i * per + cnt);
          restrict_to_list(S, rs[i], res[i]);
        } else if (code == RMIPS_ERR_CAPACITY) {
          run_single(S, rs[i], res[i], sts[i]);
        } else {
          sts[i] = (rmips_status)code;
        }
      }
    } else if (st == RMIPS_OK) {
      for (int64_t i = 0; i < nq; ++i) {
        res[i].assign(sl.h_out + sl.h_offs[i], sl.h_out + sl.h_offs[i + 1]);
        restrict_to_list(S, rs[i], res[i]);
      }
    } else if (one_by_one) {
      for (int64_t i = 0; i < nq; ++i) run_single(S, rs[i], res[i], sts[i]);
    }
    const auto now = Clock::now();
    lk.lock();
    if (one_by_one) S->one_by_one += 1;
    for (int64_t i = 0; i < nq; ++i) finish(S, rs[i], std::move(res[i]), sts[i], now);
    sl.busy = false;
    S->cv_slot.notify_all();
    S->cv_done.notify_all();
    bump(S);
  }
}

// Validates a request; *segment_size receives the number of users its
// segment allows (for the result reservation).
rmips_status check_request(const rmips_server* S, const float* q, int32_t k, const rmips_segment* seg,
                           int64_t* segment_size) {
  const rmips_index* idx = S->idx;
  if (k < 1 || k > idx->k_max) { set_error("k outside [1, k_max]"); return RMIPS_ERR_K_RANGE; }
  // the same range rule as the filter: a value whose copy in the index's
  // filter format would overflow (FP16: |x| > 65504) is refused here, so that
  // it cannot fail the other requests of its batch
  const float vmax = filter_max_abs(idx->precision);
  for (int i = 0; i < idx->d; ++i)
    if (!std::isfinite(q[i]) || std::fabs(q[i]) > vmax) {
      set_error("non-finite value in a query (or, for a BF16 / FP16 index, one beyond that format's range)");
      return RMIPS_ERR_NONFINITE;
    }
  *segment_size = idx->n;
  if (seg) {
    if (seg->reserved != 0 || seg->kind < 0 || seg->kind > 3) { set_error("bad segment"); return RMIPS_ERR_ARG; }
    if (seg->kind == 1) {
      if (seg->begin < 0 || seg->end < seg->begin) { set_error("bad segment range"); return RMIPS_ERR_ARG; }
      const int64_t hi = seg->end < idx->n ? seg->end : idx->n;
      *segment_size = hi > seg->begin ? hi - seg->begin : 0;
    }
    if (seg->kind == 2) {
      if (seg->n_ids < 0 || (seg->n_ids > 0 && !seg->ids)) { set_error("bad segment list"); return RMIPS_ERR_ARG; }
      for (int64_t i = 0; i < seg->n_ids; ++i)
        if (seg->ids[i] < 0 || seg->ids[i] >= idx->n) { set_error("segment id out of range"); return RMIPS_ERR_ARG; }
      *segment_size = seg->n_ids;
    }
    if (seg->kind == 3) {
      if (seg->begin < 0 || seg->begin >= (int64_t)S->segs.size()) { set_error("unknown segment handle"); return RMIPS_ERR_ARG; }
      *segment_size = (int64_t)S->segs[(size_t)seg->begin].size();
    }
  }
  return RMIPS_OK;
}

Request* make_request(const rmips_server* S, const float* q, int32_t k, const rmips_segment* seg, int64_t seg_size) {
  Request* r = new Request();
  r->q.assign(q, q + S->idx->d);
  r->k = k;
  if (seg) {
    r->kind = seg->kind;
    r->lo = seg->begin;
    r->hi = seg->end;
    if (seg->kind == 2) {
      r->list.assign(seg->ids, seg->ids + seg->n_ids);
      std::sort(r->list.begin(), r->list.end());
      r->list.erase(std::unique(r->list.begin(), r->list.end()), r->list.end());
    }
    if (seg->kind == 3) r->handle = (int32_t)seg->begin;
  }
  const int64_t per = S->o.result_ids_per_request;
  r->reserve = seg_size < per ? (seg_size > 0 ? seg_size : 1) : per;
  r->t0 = Clock::now();
  return r;
}

}  // namespace

extern "C" rmips_status rmips_server_create(rmips_index* idx, const rmips_server_opts* opts, rmips_server** out) {
  if (!idx || !out) { set_error("null argument"); return RMIPS_ERR_ARG; }
  *out = nullptr;
  rmips_server_opts o{};
  o.max_batch = 4096;
  o.max_wait_us = 200;
  o.streams = 2;
  o.max_pending = 1 << 20;
  if (opts) o = *opts;
  if (o.max_batch < 1 || o.max_batch > MQ_MAXQ || o.max_wait_us < 0 || o.streams < 1 || o.streams > 16 ||
      o.max_pending < 1 || o.max_device_bytes < 0 || o.result_ids_per_request < 0 || o.single_max < -1 ||
      o.single_max > 64 || o.spin_us < 0 || o.spin_us > 100000 || o.reserved != 0) {
    set_error("bad server options (max_batch 1..16384, streams 1..16, spin_us 0..100000)");
    return RMIPS_ERR_ARG;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(idx->device);
  if (o.result_ids_per_request == 0) o.result_ids_per_request = 1024;
  if (o.single_max == 0) o.single_max = 4;
  if (o.single_max < 0) o.single_max = 0;
  if (o.max_device_bytes == 0) {               // an eighth of the free device memory, at most 256 MiB
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); fr = 0; }
    const size_t cap = (size_t)256 << 20;
    o.max_device_bytes = (int64_t)(fr / 8 < cap ? fr / 8 : cap);
  }
  // each slot's result buffer: its share of the budget, at least one request's reservation
  int64_t cap_out = o.max_device_bytes / (8 * (int64_t)o.streams);
  if (cap_out < o.result_ids_per_request) cap_out = o.result_ids_per_request;
  rmips_server* S = new rmips_server();
  S->idx = idx;
  S->o = o;
  S->capacity = cap_out * o.streams;
  S->slots.resize(o.streams);
  rmips_status st = RMIPS_OK;
  for (Slot& sl : S->slots) {
    sl.ws = acquire_workspace(idx, &st);
    if (!sl.ws) break;
    if ((st = batch_reserve(idx, sl.ws, o.max_batch)) != RMIPS_OK) break;
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && sl.ws->done_pending) {          // after an asynchronous call's work
      e = cudaStreamWaitEvent(sl.stream, sl.ws->done_ev, 0);
      sl.ws->done_pending = false;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&sl.h_q, (size_t)o.max_batch * idx->d * sizeof(float), 0);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&sl.h_k, o.max_batch * sizeof(int32_t), 0);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&sl.h_lo, o.max_batch * sizeof(long long), 0);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&sl.h_hi, o.max_batch * sizeof(long long), 0);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&sl.h_offs, (o.max_batch + 1) * sizeof(long long), 0);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&sl.h_ctr, C_NCOUNTERS * sizeof(long long), 0);
    if (e == cudaSuccess) e = cudaMalloc((void**)&sl.d_out, (size_t)cap_out * sizeof(long long));
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&sl.h_out, (size_t)cap_out * sizeof(long long), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaMalloc((void**)&sl.d_done, 2 * 64 * sizeof(long long));
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&sl.h_done, 2 * 64 * sizeof(long long), 0);
    sl.cap_out = cap_out;
    if (e != cudaSuccess) {
      set_error(std::string("server allocation: ") + cudaGetErrorString(e));
      st = e == cudaErrorMemoryAllocation ? RMIPS_ERR_OOM : RMIPS_ERR_CUDA;
      break;
    }
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (st != RMIPS_OK) {
    rmips_server_destroy(S);
    return st;
  }
  S->disp = std::thread(dispatcher, S);
  S->comp = std::thread(completer, S);
  *out = S;
  return RMIPS_OK;
}

extern "C" rmips_status rmips_server_add_segment(rmips_server* S, const int64_t* ids, int64_t n_ids, int32_t* handle) {
  if (!S || !handle || n_ids < 0 || (n_ids > 0 && !ids)) { set_error("null argument"); return RMIPS_ERR_ARG; }
  if (ptr_class(ids, S->idx->device) != PTR_HOST) { set_error("segment ids are given in host memory"); return RMIPS_ERR_ARG; }
  std::vector<int64_t> v(ids, ids + n_ids);
  for (int64_t id : v)
    if (id < 0 || id >= S->idx->n) { set_error("segment id out of range"); return RMIPS_ERR_ARG; }
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->segs.size() >= (size_t)INT32_MAX) { set_error("too many segments"); return RMIPS_ERR_ARG; }
  S->segs.push_back(std::move(v));
  *handle = (int32_t)(S->segs.size() - 1);
  return RMIPS_OK;
}

extern "C" rmips_status rmips_server_submit_many(rmips_server* S, const float* qs, int64_t nq, const int32_t* ks,
                                                 const rmips_segment* segs, int64_t* tickets) {
  if (!S || nq < 0 || (nq > 0 && (!qs || !ks || !tickets))) { set_error("null argument"); return RMIPS_ERR_ARG; }
  if (nq > 0 && (ptr_class(qs, S->idx->device) != PTR_HOST || ptr_class(ks, S->idx->device) != PTR_HOST)) {
    set_error("requests are submitted from host memory");
    return RMIPS_ERR_ARG;
  }
  const int d = S->idx->d;
  std::vector<int64_t> sizes((size_t)nq);
  {
    std::lock_guard<std::mutex> lk(S->mu);      // registered segments
    for (int64_t j = 0; j < nq; ++j) {
      rmips_status st = check_request(S, qs + j * d, ks[j], segs ? &segs[j] : nullptr, &sizes[j]);
      if (st != RMIPS_OK) return st;
    }
  }
  std::vector<Request*> rs(nq);
  int64_t need = 0;
  for (int64_t j = 0; j < nq; ++j) {
    rs[j] = make_request(S, qs + j * d, ks[j], segs ? &segs[j] : nullptr, sizes[j]);
    need += rs[j]->reserve;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      for (Request* r : rs) delete r;
      set_error("server is stopping");
      return RMIPS_ERR_ARG;
    }
    if (S->pending + nq > S->o.max_pending || S->reserved + need > S->capacity) {
      for (Request* r : rs) delete r;
      S->rejected += nq;
      set_error("admission refused: the pending requests' result reservations or count are at the limit");
      return RMIPS_ERR_BUSY;
    }
    for (int64_t j = 0; j < nq; ++j) {
      const int64_t t = S->next++;
      S->reqs[t] = rs[j];
      S->queue.push_back(t);
      tickets[j] = t;
    }
    S->pending += nq;
    S->reserved += need;
    S->submitted += nq;
  }
  S->cv_in.notify_one();
  bump(S);
  return RMIPS_OK;
}

extern "C" rmips_status rmips_server_submit(rmips_server* S, const float* q, int32_t k, const rmips_segment* seg,
                                            int64_t* ticket) {
  if (!q || !ticket) { set_error("null argument"); return RMIPS_ERR_ARG; }
  return rmips_server_submit_many(S, q, 1, &k, seg, ticket);
}

extern "C" rmips_status rmips_server_wait(rmips_server* S, int64_t ticket, int64_t* out_ids, int64_t capacity,
                                          int64_t* out_count, double* latency_ms, int32_t timeout_ms) {
  if (!S || !out_count || capacity < 0 || (capacity > 0 && !out_ids)) { set_error("null argument"); return RMIPS_ERR_ARG; }
  if (capacity > 0 && check_ptr_device(out_ids, S->idx->device, "out_ids") != RMIPS_OK) return RMIPS_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) { set_error("unknown ticket"); return RMIPS_ERR_ARG; }
  Request* r = it->second;
  auto done = [&] { return r->state == 2; };
  if (timeout_ms != 0 && spin_for(S, lk, done)) {
  } else if (timeout_ms < 0) S->cv_done.wait(lk, done);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    set_error("request not finished yet");
    return RMIPS_ERR_TIMEOUT;
  }
  *out_count = (int64_t)r->ids.size();
  if (latency_ms) *latency_ms = r->ms;
  const rmips_status st = r->st;
  if (st == RMIPS_OK && (int64_t)r->ids.size() > capacity) {
    set_error("output capacity too small");
    return RMIPS_ERR_CAPACITY;                   // the request is kept: wait again with more room
  }
  if (st == RMIPS_OK && !r->ids.empty()) {
    if (is_device_ptr(out_ids)) {
      lk.unlock();
      cudaError_t e = cudaMemcpy(out_ids, r->ids.data(), r->ids.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
      lk.lock();
      if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return RMIPS_ERR_CUDA; }
    } else {
      memcpy(out_ids, r->ids.data(), r->ids.size() * sizeof(int64_t));
    }
  }
  S->reqs.erase(ticket);
  delete r;
  return st;
}

extern "C" rmips_status rmips_server_wait_many(rmips_server* S, const int64_t* tickets, int64_t nt,
                                               int64_t* out_ids, int64_t capacity, int64_t* out_offsets,
                                               double* latency_ms, int32_t timeout_ms) {
  if (!S || nt < 0 || (nt > 0 && !tickets) || !out_offsets || capacity < 0 || (capacity > 0 && !out_ids)) {
    set_error("null argument");
    return RMIPS_ERR_ARG;
  }
  if (capacity > 0 && check_ptr_device(out_ids, S->idx->device, "out_ids") != RMIPS_OK) return RMIPS_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  std::vector<Request*> rs(nt);
  for (int64_t i = 0; i < nt; ++i) {
    auto it = S->reqs.find(tickets[i]);
    if (it == S->reqs.end()) { set_error("unknown ticket"); return RMIPS_ERR_ARG; }
    rs[i] = it->second;
  }
  auto all_done = [&] {
    for (Request* r : rs)
      if (r->state != 2) return false;
    return true;
  };
  if (timeout_ms != 0 && spin_for(S, lk, all_done)) {
  } else if (timeout_ms < 0) S->cv_done.wait(lk, all_done);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), all_done)) {
    set_error("requests not finished yet");
    return RMIPS_ERR_TIMEOUT;
  }
  out_offsets[0] = 0;
  rmips_status first = RMIPS_OK;
  for (int64_t i = 0; i < nt; ++i) {
    const int64_t c = rs[i]->st == RMIPS_OK ? (int64_t)rs[i]->ids.size() : 0;
    out_offsets[i + 1] = out_offsets[i] + c;
    if (first == RMIPS_OK && rs[i]->st != RMIPS_OK) first = rs[i]->st;
    if (latency_ms) latency_ms[i] = rs[i]->ms;
  }
  if (out_offsets[nt] > capacity) {
    set_error("output capacity too small");
    return RMIPS_ERR_CAPACITY;                   // tickets kept: wait again with more room
  }
  const bool dev = out_offsets[nt] > 0 && is_device_ptr(out_ids);
  for (int64_t i = 0; i < nt; ++i) {
    Request* r = rs[i];
    if (r->st == RMIPS_OK && !r->ids.empty()) {
      if (dev) {
        cudaError_t e = cudaMemcpy(out_ids + out_offsets[i], r->ids.data(), r->ids.size() * sizeof(int64_t),
                                   cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return RMIPS_ERR_CUDA; }
      } else {
        memcpy(out_ids + out_offsets[i], r->ids.data(), r->ids.size() * sizeof(int64_t));
      }
    }
  }
  for (int64_t i = 0; i < nt; ++i) {
    S->reqs.erase(tickets[i]);
    delete rs[i];
  }
  if (first != RMIPS_OK) set_error("a request of the set failed");
  return first;
}

extern "C" rmips_status rmips_server_get_stats(rmips_server* S, rmips_server_stats* out) {
  if (!S || !out) { set_error("null argument"); return RMIPS_ERR_ARG; }
  std::vector<double> v;
  rmips_server_stats s{};
  {
    std::lock_guard<std::mutex> lk(S->mu);
    v = S->lat;
    s.submitted = S->submitted;
    s.completed = S->completed;
    s.rejected = S->rejected;
    s.batches = S->batches;
    s.mean_batch = S->batches ? (double)S->batched / S->batches : 0.0;
    s.pending = S->pending;
    s.reserved_ids = S->reserved;
    s.reservable_ids = S->capacity;
    s.batches_one_by_one = S->one_by_one;
  }
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)std::floor(p * (v.size() - 1) + 0.5))]; };
    s.p50_ms = pct(0.50);
    s.p99_ms = pct(0.99);
    s.max_ms = v.back();
  }
  *out = s;
  return RMIPS_OK;
}

extern "C" void rmips_server_destroy(rmips_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_in.notify_all();
  S->cv_slot.notify_all();
  S->cv_fly.notify_all();
  bump(S);
  if (S->disp.joinable()) S->disp.join();
  if (S->comp.joinable()) S->comp.join();
  for (Slot& sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.ws) release_workspace(S->idx, sl.ws);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    cudaFreeHost(sl.h_q);
    cudaFreeHost(sl.h_k);
    cudaFreeHost(sl.h_lo);
    cudaFreeHost(sl.h_hi);
    cudaFreeHost(sl.h_offs);
    cudaFreeHost(sl.h_ctr);
    cudaFreeHost(sl.h_out);
    cudaFree(sl.d_out);
    cudaFree(sl.d_done);
    cudaFreeHost(sl.h_done);
  }
  for (auto& kv : S->reqs) delete kv.second;
  delete S;
}
