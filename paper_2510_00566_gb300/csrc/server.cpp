// Serving loop: continuous batching of single-query requests over the
// device-resident index.
//
// Requests enter a FIFO queue.  A worker thread owns `max_inflight` slots;
// each slot has its own stream, pinned host staging, device buffers for up to
// `max_batch` queries and a completion event.  Whenever a slot is free, the
// queue is non-empty and the memory budget admits the batch (its search
// workspace, estimated from the batch shape, plus the slot buffers), the
// worker moves up to max_batch queued requests into the slot, copies them to
// the device, enqueues the search, the copy-back of the results and of the
// search's device error word, and records the event.
// Batches in different slots overlap on the device; requests that arrive
// while batches run are admitted to the next free slot.  Finished slots are
// retired by polling their events: the error word decides the batch's status
// (a bounded device wait that gave up, or an FP8 query out of range, fails
// every request of the batch), results are handed to the waiting callers and
// the request latency (submit -> results on the host) recorded.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "search.h"

using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  uint64_t ticket;
  int32_t nprobe, k;
  Clock::time_point t_submit;
  std::vector<float> q;
};

struct Result {
  std::vector<int64_t> ids;
  std::vector<float> dists;
  bool done = false;
  int status = PANO_OK;
  double latency_us = 0.0;  // submit -> results on the host
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  float *d_q = nullptr, *h_q = nullptr;
  int32_t *d_np = nullptr, *h_np = nullptr, *d_k = nullptr, *h_k = nullptr;
  int64_t *d_ids = nullptr, *h_ids = nullptr;
  float *d_dists = nullptr, *h_dists = nullptr;
  int* h_err = nullptr;  // the batch's device error word (pinned), copied after its search
  std::vector<Request> reqs;
  bool busy = false;
  int64_t bytes = 0;  // admitted memory
  int status = PANO_OK;
};

}  // namespace

struct pano_server {
  const pano_index* idx = nullptr;
  pano_server_opts o{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::unordered_map<uint64_t, Result> results;
  std::vector<Slot> slots;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  int64_t in_flight_bytes = 0;
  // statistics
  int64_t submitted = 0, completed = 0, batches = 0, batched_queries = 0;
  std::vector<double> lat_us;  // ring of the most recent latencies
  size_t lat_pos = 0;
  Clock::time_point t_first{}, t_last{};

  ~pano_server();
  void run();
  int64_t batch_bytes(int nq, int nprobe_max) const;
};

int64_t pano_server::batch_bytes(int nq, int nprobe_max) const {
  // the search workspace of the batch, as the search carves it, plus the
  // slot buffers; the search's own layout at the largest stride if its
  // sizing fails (it then fails in the search as well)
  size_t ws = 0;
  if (pano::search_workspace_bytes(idx, nq, nprobe_max, o.k_max, &ws) != PANO_OK &&
      pano::search_workspace_bytes(idx, nq, idx->nlist, o.k_max, &ws) != PANO_OK)
    ws = 0;
  const int64_t d = idx->d, km = o.k_max;
  return (int64_t)ws + (int64_t)o.max_batch * (d * 4 + 8 + km * 12);
}

pano_server::~pano_server() {
  {
    std::lock_guard<std::mutex> lk(mu);
    stop = true;
  }
  cv_work.notify_all();
  if (worker.joinable()) worker.join();
  cudaSetDevice(device);
  for (Slot& s : slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    cudaFree(s.d_q);
    cudaFree(s.d_np);
    cudaFree(s.d_k);
    cudaFree(s.d_ids);
    cudaFree(s.d_dists);
    cudaFreeHost(s.h_q);
    cudaFreeHost(s.h_np);
    cudaFreeHost(s.h_k);
    cudaFreeHost(s.h_ids);
    cudaFreeHost(s.h_dists);
    cudaFreeHost(s.h_err);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.stream) cudaStreamDestroy(s.stream);
  }
}

void pano_server::run() {
  cudaSetDevice(device);
  const int d = idx->d, km = o.k_max;
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    // retire finished batches
    bool retired = false;
    for (Slot& s : slots) {
      if (!s.busy) continue;
      if (s.status == PANO_OK && cudaEventQuery(s.ev) == cudaErrorNotReady) continue;
      // a bounded device wait that gave up (partial top-k) or a query the
      // storage format cannot hold fails every request of the batch
      if (s.status == PANO_OK) s.status = pano::status_of_device_error(*s.h_err);
      const auto now = Clock::now();
      for (size_t i = 0; i < s.reqs.size(); ++i) {
        Result& r = results[s.reqs[i].ticket];
        r.ids.assign(s.h_ids + i * km, s.h_ids + (i + 1) * km);
        r.dists.assign(s.h_dists + i * km, s.h_dists + (i + 1) * km);
        r.status = s.status;
        r.done = true;
        const double us =
            std::chrono::duration<double, std::micro>(now - s.reqs[i].t_submit).count();
        r.latency_us = us;
        if (lat_us.size() < 1000000)
          lat_us.push_back(us);
        else
          lat_us[lat_pos++ % lat_us.size()] = us;
        ++completed;
      }
      t_last = now;
      in_flight_bytes -= s.bytes;
      s.reqs.clear();
      s.busy = false;
      s.status = PANO_OK;
      retired = true;
    }
    if (retired) cv_done.notify_all();
    // admit queued requests into free slots
    bool launched = false;
    for (Slot& s : slots) {
      if (queue.empty()) break;
      if (s.busy) continue;
      const int nb = (int)std::min<size_t>(queue.size(), (size_t)o.max_batch);
      int np_batch = 1;
      for (int i = 0; i < nb; ++i) np_batch = std::max(np_batch, queue[i].nprobe);
      const int64_t bytes = batch_bytes(nb, np_batch);
      const bool any_busy =
          std::any_of(slots.begin(), slots.end(), [](const Slot& x) { return x.busy; });
      if (any_busy && in_flight_bytes + bytes > o.memory_budget) break;  // wait for memory
      s.reqs.clear();
      int32_t np_max = 1;
      for (int i = 0; i < nb; ++i) {
        Request& r = queue.front();
        std::memcpy(s.h_q + (size_t)i * d, r.q.data(), (size_t)d * 4);
        s.h_np[i] = r.nprobe;
        s.h_k[i] = r.k;
        np_max = std::max(np_max, r.nprobe);
        s.reqs.push_back(std::move(r));
        queue.pop_front();
      }
      s.busy = true;
      s.bytes = bytes;
      in_flight_bytes += bytes;
      ++batches;
      batched_queries += nb;
      lk.unlock();
      int rc = PANO_OK;
      cudaError_t e = cudaMemcpyAsync(s.d_q, s.h_q, (size_t)nb * d * 4, cudaMemcpyHostToDevice, s.stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(s.d_np, s.h_np, nb * 4, cudaMemcpyHostToDevice, s.stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(s.d_k, s.h_k, nb * 4, cudaMemcpyHostToDevice, s.stream);
      if (e != cudaSuccess) rc = PANO_ECUDA;
      if (rc == PANO_OK) {
        pano_search_opts so{};
        so.synchronize = 0;
        *s.h_err = 0;
        rc = pano::search(idx, s.d_q, nb, s.d_np, std::min(np_max, idx->nlist), s.d_k, 0, km,
                          s.d_ids, s.d_dists, s.stream, &so, nullptr, 0, s.h_err);
      }
      if (rc == PANO_OK) {
        e = cudaMemcpyAsync(s.h_ids, s.d_ids, (size_t)nb * km * 8, cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(s.h_dists, s.d_dists, (size_t)nb * km * 4, cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess) e = cudaEventRecord(s.ev, s.stream);
        if (e != cudaSuccess) rc = PANO_ECUDA;
      }
      lk.lock();
      s.status = rc;
      launched = true;
    }
    if (stop && queue.empty() &&
        std::none_of(slots.begin(), slots.end(), [](const Slot& x) { return x.busy; }))
      break;
    const bool busy =
        std::any_of(slots.begin(), slots.end(), [](const Slot& x) { return x.busy; });
    if (!launched && !retired) {
      if (busy) {
        // poll the in-flight events without holding the lock
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      } else {
        cv_work.wait(lk, [&] { return stop || !queue.empty(); });
      }
    }
  }
}

using namespace pano;

extern "C" {

int panorama_server_create(const pano_index* idx, const pano_server_opts* opts,
                           pano_server** out) {
  clear_error();
  PANO_CHECK(idx && out, PANO_EINVAL, "null argument");
  auto s = std::make_unique<pano_server>();
  s->idx = idx;
  if (opts) s->o = *opts;
  if (s->o.max_batch <= 0) s->o.max_batch = 1024;
  if (s->o.max_inflight <= 0) s->o.max_inflight = 2;
  if (s->o.k_max <= 0) s->o.k_max = 10;
  if (s->o.memory_budget <= 0) s->o.memory_budget = (int64_t)1 << 30;
  PANO_CHECK(s->o.max_batch <= 65536 && s->o.max_inflight <= 16 && s->o.k_max <= 1024,
             PANO_EINVAL, "server options out of range");
  s->device = idx->device;
  PANO_CUDA(cudaSetDevice(s->device));
  const int d = idx->d, mb = s->o.max_batch, km = s->o.k_max;
  s->slots.resize(s->o.max_inflight);
  for (Slot& sl : s->slots) {
    PANO_CUDA(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
    PANO_CUDA(cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming));
    PANO_CUDA(cudaMalloc(&sl.d_q, (size_t)mb * d * 4));
    PANO_CUDA(cudaMalloc(&sl.d_np, mb * 4));
    PANO_CUDA(cudaMalloc(&sl.d_k, mb * 4));
    PANO_CUDA(cudaMalloc(&sl.d_ids, (size_t)mb * km * 8));
    PANO_CUDA(cudaMalloc(&sl.d_dists, (size_t)mb * km * 4));
    PANO_CUDA(cudaMallocHost(&sl.h_q, (size_t)mb * d * 4));
    PANO_CUDA(cudaMallocHost(&sl.h_np, mb * 4));
    PANO_CUDA(cudaMallocHost(&sl.h_k, mb * 4));
    PANO_CUDA(cudaMallocHost(&sl.h_ids, (size_t)mb * km * 8));
    PANO_CUDA(cudaMallocHost(&sl.h_dists, (size_t)mb * km * 4));
    PANO_CUDA(cudaMallocHost(&sl.h_err, sizeof(int)));
    *sl.h_err = 0;
  }
  pano_server* raw = s.get();
  s->worker = std::thread([raw] { raw->run(); });
  *out = s.release();
  return PANO_OK;
}

int panorama_server_submit(pano_server* s, const float* query, int32_t nprobe, int32_t k,
                           uint64_t* ticket) {
  PANO_CHECK(s && query && ticket, PANO_EINVAL, "null argument");
  PANO_CHECK(nprobe >= 1 && nprobe <= s->idx->nlist && k >= 0 && k <= s->o.k_max, PANO_EINVAL,
             "nprobe or k out of range");
  Request r;
  r.nprobe = nprobe;
  r.k = k;
  r.q.assign(query, query + s->idx->d);
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    PANO_CHECK(!s->stop, PANO_EINVAL, "server is shutting down");
    r.ticket = s->next_ticket++;
    *ticket = r.ticket;
    if (s->submitted == 0) s->t_first = r.t_submit;
    ++s->submitted;
    s->results[r.ticket];  // slot for the result
    s->queue.push_back(std::move(r));
  }
  s->cv_work.notify_one();
  return PANO_OK;
}

int panorama_server_wait(pano_server* s, uint64_t ticket, int32_t timeout_ms, int64_t* ids,
                         float* dists, double* latency_us) {
  PANO_CHECK(s && ids && dists, PANO_EINVAL, "null argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  PANO_CHECK(it != s->results.end(), PANO_EINVAL, "unknown ticket");
  const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 1 << 30 : timeout_ms),
                                      [&] { return s->results[ticket].done; });
  if (!ok) return fail(PANO_ETIMEOUT, "request not finished before the timeout");
  Result& r = s->results[ticket];
  const int status = r.status;
  if (latency_us) *latency_us = r.latency_us;
  std::memcpy(ids, r.ids.data(), r.ids.size() * 8);
  std::memcpy(dists, r.dists.data(), r.dists.size() * 4);
  s->results.erase(ticket);
  if (status) return fail(status, "the batch holding this request failed");
  return PANO_OK;
}

int panorama_server_stats(pano_server* s, pano_server_stats* out) {
  PANO_CHECK(s && out, PANO_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->batches = s->batches;
  out->mean_batch = s->batches ? (double)s->batched_queries / s->batches : 0.0;
  if (!s->lat_us.empty()) {
    std::vector<double> v = s->lat_us;
    auto q = [&](double f) {
      size_t i = std::min(v.size() - 1, (size_t)(f * (v.size() - 1) + 0.5));
      std::nth_element(v.begin(), v.begin() + i, v.end());
      return v[i];
    };
    out->p50_us = q(0.50);
    out->p99_us = q(0.99);
    out->max_us = *std::max_element(v.begin(), v.end());
  }
  const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
  out->qps = span > 0 ? s->completed / span : 0.0;
  return PANO_OK;
}

int panorama_server_run_trace(pano_server* s, const float* queries, int64_t nq,
                              const double* arrival_us, const int32_t* nprobe, const int32_t* k,
                              int64_t* out_ids, float* out_dists, double* latency_us) {
  clear_error();
  PANO_CHECK(s && queries && arrival_us && nprobe && k && out_ids && out_dists, PANO_EINVAL,
             "null argument");
  const int d = s->idx->d, km = s->o.k_max;
  std::vector<uint64_t> tickets(nq);
  const auto t0 = Clock::now();
  for (int64_t i = 0; i < nq; ++i) {  // open-loop arrivals at the given times
    const auto due = t0 + std::chrono::nanoseconds((int64_t)(arrival_us[i] * 1000.0));
    while (Clock::now() < due) {
    }
    int rc = panorama_server_submit(s, queries + i * d, nprobe[i], k[i], &tickets[i]);
    if (rc) return rc;
  }
  for (int64_t i = 0; i < nq; ++i) {
    int rc = panorama_server_wait(s, tickets[i], 600000, out_ids + i * km, out_dists + i * km,
                                  latency_us ? latency_us + i : nullptr);
    if (rc) return rc;
  }
  return PANO_OK;
}

void panorama_server_free(pano_server* s) { delete s; }

}  // extern "C"
