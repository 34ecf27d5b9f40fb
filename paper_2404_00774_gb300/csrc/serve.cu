// Continuous-batching serving loop over a resident index (an extension; the
// paper describes no serving system).
//
// Requests (one fp32 query, its own k and t) are queued by soar_server_submit
// from any thread, or as a trace of timed arrivals by soar_server_submit_many
// (a request becomes pending at its arrival time, and its latency counts from
// then).  A dispatcher thread keeps up to `streams` batches in flight:
// whenever a stream slot is free it takes pending requests in arrival order,
// keeping to one k class per batch (k <= 32 or k > 32, which the search
// serves with different list structures), admitting each while the batch
// stays within max_batch and the device-memory estimate of everything in
// flight stays within the budget;
// the batch then runs on that slot's stream (host-to-device copy of the
// queries, one soar_search with per-request probe counts and the batch's
// largest k, device-to-host copy of the results).  Requests that arrive while
// batches run join the next batch as soon as a slot and memory free up, so
// their work overlaps on the GPU with the batches already running.  Results
// are truncated to each request's own k (a top-k list is a prefix of the
// top-k' list for k <= k').
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"
#include "scan_common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id;
  std::vector<float> q;
  int k, t;
  Clock::time_point submitted;
  size_t bytes;
};

struct Done {
  std::vector<int64_t> ids;
  std::vector<float> scores;
  double latency_ms;
  soar_status status;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  float* q_host = nullptr;       // pinned [max_batch][d]
  int32_t* t_host = nullptr;     // pinned [max_batch]
  int64_t* ids_host = nullptr;   // pinned [max_batch][max_k]
  float* sc_host = nullptr;      // pinned [max_batch][max_k]
  float* q_dev = nullptr;
  int32_t* t_dev = nullptr;
  int64_t* ids_dev = nullptr;
  float* sc_dev = nullptr;
  bool busy = false;
  std::vector<Request> batch;
  int kmax = 0;
  size_t bytes = 0;
  soar_status status = SOAR_OK;
};

}  // namespace

struct soar_server {
  const soar_index* index = nullptr;
  soar_server_config cfg{};
  int device = 0;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work;   // dispatcher: new request or slot freed
  std::condition_variable cv_done;   // waiters: a request completed
  std::deque<Request> pending;
  std::multimap<Clock::time_point, Request> scheduled;   // future arrivals of submit_many
  std::unordered_map<uint64_t, Done> finished;
  uint64_t next_id = 1;
  size_t in_flight_bytes = 0;
  bool stop = false;
  std::thread worker;
  // statistics
  uint64_t batches = 0, completed = 0, queries_in_batches = 0;
  int max_in_flight = 0;
  std::vector<double> latencies;
};

namespace {

// Device scratch one request adds to a search: its centroid-score row, query
// row, probe lists, grouping pairs and per-probe candidate lists.
size_t request_bytes(const soar::IndexData& ix, int k, int t) {
  const size_t list = (size_t)std::max(k <= soar::kTcWideK ? soar::scan_tc_list_len(k) : 32, k) * 8;
  return (size_t)ix.c * 4 + (size_t)(ix.d + 16) * 4 + (size_t)t * (4 + 16 + 4 + 8 + list) + (size_t)k * 12 + 256;
}

void finish_slot(soar_server* sv, Slot& sl) {
  // called with sv->mu held, after sl.done completed
  const auto now = Clock::now();
  const int d = sv->index->data.d;
  (void)d;
  for (size_t i = 0; i < sl.batch.size(); ++i) {
    const Request& r = sl.batch[i];
    Done out;
    out.status = sl.status;
    out.ids.assign(sl.ids_host + i * sl.kmax, sl.ids_host + i * sl.kmax + r.k);
    out.scores.assign(sl.sc_host + i * sl.kmax, sl.sc_host + i * sl.kmax + r.k);
    out.latency_ms = std::chrono::duration<double, std::milli>(now - r.submitted).count();
    sv->latencies.push_back(out.latency_ms);
    sv->finished.emplace(r.id, std::move(out));
    ++sv->completed;
  }
  sv->in_flight_bytes -= sl.bytes;
  sl.batch.clear();
  sl.busy = false;
}

// Runs on a CUDA driver thread once a batch's copies and search are done:
// wakes the dispatcher (no CUDA calls are allowed here).
void CUDART_CB batch_done(void* arg) {
  soar_server* sv = static_cast<soar_server*>(arg);
  sv->cv_work.notify_one();
}

int k_class(int k) { return k <= 32 ? 0 : 1; }

void dispatcher(soar_server* sv) {
  cudaSetDevice(sv->device);
  const soar::IndexData& ix = sv->index->data;
  std::unique_lock<std::mutex> lock(sv->mu);
  while (true) {
    // scheduled requests whose arrival time has come become pending
    const auto now = Clock::now();
    while (!sv->scheduled.empty() && sv->scheduled.begin()->first <= now) {
      sv->pending.push_back(std::move(sv->scheduled.begin()->second));
      sv->scheduled.erase(sv->scheduled.begin());
    }
    // retire finished batches
    int busy = 0;
    for (Slot& sl : sv->slots) {
      if (!sl.busy) continue;
      if (cudaEventQuery(sl.done) == cudaSuccess) finish_slot(sv, sl);
      else ++busy;
    }
    if (busy == 0 && sv->stop && sv->pending.empty() && sv->scheduled.empty()) break;
    sv->cv_done.notify_all();
    // launch a batch into a free slot
    Slot* free_slot = nullptr;
    for (Slot& sl : sv->slots)
      if (!sl.busy) { free_slot = &sl; break; }
    if (free_slot && !sv->pending.empty()) {
      Slot& sl = *free_slot;
      size_t bytes = 0;
      const int cls = k_class(sv->pending.front().k);
      std::deque<Request> skipped;                 // other k class: stays pending, in order
      while (!sv->pending.empty() && (int)sl.batch.size() < sv->cfg.max_batch) {
        const Request& r = sv->pending.front();
        if (k_class(r.k) != cls) {
          skipped.push_back(std::move(sv->pending.front()));
          sv->pending.pop_front();
          continue;
        }
        // the first request of a batch is always admitted when nothing else runs
        const bool fits = sv->in_flight_bytes + bytes + r.bytes <= (size_t)sv->cfg.memory_budget;
        if (!fits && !(sl.batch.empty() && busy == 0)) break;
        bytes += r.bytes;
        sl.batch.push_back(std::move(sv->pending.front()));
        sv->pending.pop_front();
      }
      while (!skipped.empty()) {
        sv->pending.push_front(std::move(skipped.back()));
        skipped.pop_back();
      }
      if (!sl.batch.empty()) {
        const int nb = (int)sl.batch.size();
        int kmax = 1, tmax = 1;
        for (const Request& r : sl.batch) {
          kmax = std::max(kmax, r.k);
          tmax = std::max(tmax, r.t);
        }
        for (int i = 0; i < nb; ++i) {
          std::copy(sl.batch[i].q.begin(), sl.batch[i].q.end(), sl.q_host + (size_t)i * ix.d);
          sl.t_host[i] = sl.batch[i].t;
        }
        sl.kmax = kmax;
        sl.bytes = bytes;
        sl.busy = true;
        sv->in_flight_bytes += bytes;
        ++sv->batches;
        sv->queries_in_batches += nb;
        sv->max_in_flight = std::max(sv->max_in_flight, busy + 1);
        lock.unlock();
        soar_status st = SOAR_OK;
        cudaMemcpyAsync(sl.q_dev, sl.q_host, sizeof(float) * nb * ix.d, cudaMemcpyHostToDevice, sl.stream);
        cudaMemcpyAsync(sl.t_dev, sl.t_host, sizeof(int32_t) * nb, cudaMemcpyHostToDevice, sl.stream);
        st = soar_search(sv->index, sl.q_dev, SOAR_F32, nb, kmax, tmax, sl.t_dev, 0, sl.ids_dev, sl.sc_dev, sl.stream);
        cudaMemcpyAsync(sl.ids_host, sl.ids_dev, sizeof(int64_t) * nb * kmax, cudaMemcpyDeviceToHost, sl.stream);
        cudaMemcpyAsync(sl.sc_host, sl.sc_dev, sizeof(float) * nb * kmax, cudaMemcpyDeviceToHost, sl.stream);
        cudaEventRecord(sl.done, sl.stream);
        cudaLaunchHostFunc(sl.stream, batch_done, sv);
        lock.lock();
        sl.status = st;
        continue;   // look for more work right away
      }
    }
    // nothing to launch: sleep until a request arrives, a batch completes or
    // the next scheduled arrival is due
    auto until = Clock::now() + std::chrono::milliseconds(2);
    if (!sv->scheduled.empty()) until = std::min(until, sv->scheduled.begin()->first);
    sv->cv_work.wait_until(lock, until);
  }
  sv->cv_done.notify_all();
}

}  // namespace

extern "C" {

soar_status soar_server_create(const soar_index* index, const soar_server_config* cfg, soar_server** out) {
  if (!index || !cfg || !out) return SOAR_EINVAL;
  if (cfg->max_batch < 1 || cfg->max_batch > 4096 || cfg->streams < 1 || cfg->streams > 16 || cfg->max_k < 1 ||
      cfg->max_k > 1024 || cfg->memory_budget <= 0)
    return SOAR_EINVAL;
  if (index->data.mode != SOAR_SCORE_F32) return SOAR_EUNSUPPORTED;
  soar_server* sv = new soar_server;
  sv->index = index;
  sv->cfg = *cfg;
  cudaGetDevice(&sv->device);
  const int d = index->data.d, mb = cfg->max_batch, mk = cfg->max_k;
  sv->slots.resize(cfg->streams);
  bool ok = true;
  for (Slot& sl : sv->slots) {
    ok = ok && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&sl.q_host, sizeof(float) * mb * d) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&sl.t_host, sizeof(int32_t) * mb) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&sl.ids_host, sizeof(int64_t) * mb * mk) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&sl.sc_host, sizeof(float) * mb * mk) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&sl.q_dev, sizeof(float) * mb * d) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&sl.t_dev, sizeof(int32_t) * mb) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&sl.ids_dev, sizeof(int64_t) * mb * mk) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&sl.sc_dev, sizeof(float) * mb * mk) == cudaSuccess;
  }
  if (!ok) {
    soar_server_destroy(sv);
    return SOAR_ENOMEM;
  }
  sv->worker = std::thread(dispatcher, sv);
  *out = sv;
  return SOAR_OK;
}

soar_status soar_server_submit(soar_server* sv, const float* query, int32_t k, int32_t t, uint64_t* request_id) {
  if (!sv || !query || !request_id) return SOAR_EINVAL;
  const soar::IndexData& ix = sv->index->data;
  if (k < 1 || k > sv->cfg.max_k || t < 1 || t > ix.c || t > 8192) return SOAR_EINVAL;
  Request r;
  r.q.assign(query, query + ix.d);
  r.k = k;
  r.t = t;
  r.bytes = request_bytes(ix, k, t);
  r.submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    if (sv->stop) return SOAR_EINVAL;
    r.id = sv->next_id++;
    *request_id = r.id;
    sv->pending.push_back(std::move(r));
  }
  sv->cv_work.notify_one();
  return SOAR_OK;
}

soar_status soar_server_submit_many(soar_server* sv, const float* queries, int64_t n, const int32_t* ks,
                                   const int32_t* ts, const double* arrival_s, uint64_t* request_ids) {
  if (!sv || n < 0 || (n > 0 && (!queries || !ks || !ts || !request_ids))) return SOAR_EINVAL;
  const soar::IndexData& ix = sv->index->data;
  for (int64_t i = 0; i < n; ++i) {
    if (ks[i] < 1 || ks[i] > sv->cfg.max_k || ts[i] < 1 || ts[i] > ix.c || ts[i] > 8192) return SOAR_EINVAL;
    if (arrival_s && !(arrival_s[i] >= 0.0 && arrival_s[i] < 1e6)) return SOAR_EINVAL;
  }
  const auto t0 = Clock::now();
  std::vector<Request> reqs((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    Request& r = reqs[(size_t)i];
    r.q.assign(queries + i * ix.d, queries + (i + 1) * ix.d);
    r.k = ks[i];
    r.t = ts[i];
    r.bytes = request_bytes(ix, r.k, r.t);
    r.submitted = arrival_s ? t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[i]))
                            : t0;
  }
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    if (sv->stop) return SOAR_EINVAL;
    for (int64_t i = 0; i < n; ++i) {
      Request& r = reqs[(size_t)i];
      r.id = sv->next_id++;
      request_ids[i] = r.id;
      if (arrival_s) sv->scheduled.emplace(r.submitted, std::move(r));
      else sv->pending.push_back(std::move(r));
    }
  }
  sv->cv_work.notify_one();
  return SOAR_OK;
}

soar_status soar_server_wait_many(soar_server* sv, const uint64_t* request_ids, int64_t n, int32_t kstride,
                                  int64_t* ids_out, float* scores_out, double* latency_ms, int32_t timeout_ms) {
  if (!sv || n < 0 || kstride < 1 || (n > 0 && (!request_ids || !ids_out || !scores_out))) return SOAR_EINVAL;
  std::unique_lock<std::mutex> lock(sv->mu);
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
  soar_status worst = SOAR_OK;
  for (int64_t i = 0; i < n; ++i) {
    const uint64_t id = request_ids[i];
    if (id == 0 || id >= sv->next_id) return SOAR_EINVAL;
    while (true) {
      auto it = sv->finished.find(id);
      if (it != sv->finished.end()) {
        Done d = std::move(it->second);
        sv->finished.erase(it);
        const size_t kk = std::min(d.ids.size(), (size_t)kstride);
        std::copy(d.ids.begin(), d.ids.begin() + kk, ids_out + i * kstride);
        std::copy(d.scores.begin(), d.scores.begin() + kk, scores_out + i * kstride);
        std::fill(ids_out + i * kstride + kk, ids_out + (i + 1) * kstride, int64_t(-1));
        std::fill(scores_out + i * kstride + kk, scores_out + (i + 1) * kstride, -INFINITY);
        if (latency_ms) latency_ms[i] = d.latency_ms;
        if (d.status != SOAR_OK) worst = d.status;
        break;
      }
      if (sv->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && Clock::now() >= deadline)
        return SOAR_ETIMEOUT;
    }
  }
  return worst;
}

soar_status soar_server_wait(soar_server* sv, uint64_t request_id, int64_t* ids_out, float* scores_out,
                             double* latency_ms, int32_t timeout_ms) {
  if (!sv || !ids_out || !scores_out) return SOAR_EINVAL;
  std::unique_lock<std::mutex> lock(sv->mu);
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
  while (true) {
    auto it = sv->finished.find(request_id);
    if (it != sv->finished.end()) {
      Done d = std::move(it->second);
      sv->finished.erase(it);
      std::copy(d.ids.begin(), d.ids.end(), ids_out);
      std::copy(d.scores.begin(), d.scores.end(), scores_out);
      if (latency_ms) *latency_ms = d.latency_ms;
      return d.status;
    }
    if (request_id == 0 || request_id >= sv->next_id) return SOAR_EINVAL;
    if (sv->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && Clock::now() >= deadline)
      return SOAR_ETIMEOUT;
  }
}

soar_status soar_server_stats(soar_server* sv, soar_server_metrics* out) {
  if (!sv || !out) return SOAR_EINVAL;
  std::lock_guard<std::mutex> lock(sv->mu);
  out->batches = sv->batches;
  out->completed = sv->completed;
  out->queries_in_batches = sv->queries_in_batches;
  out->pending = sv->pending.size() + sv->scheduled.size();
  out->max_in_flight = sv->max_in_flight;
  std::vector<double> lat = sv->latencies;
  std::sort(lat.begin(), lat.end());
  auto pct = [&](double p) { return lat.empty() ? 0.0 : lat[std::min(lat.size() - 1, (size_t)(p * lat.size()))]; };
  out->p50_ms = pct(0.50);
  out->p99_ms = pct(0.99);
  return SOAR_OK;
}

soar_status soar_server_destroy(soar_server* sv) {
  if (!sv) return SOAR_OK;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (Slot& sl : sv->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    cudaFreeHost(sl.q_host);
    cudaFreeHost(sl.t_host);
    cudaFreeHost(sl.ids_host);
    cudaFreeHost(sl.sc_host);
    cudaFree(sl.q_dev);
    cudaFree(sl.t_dev);
    cudaFree(sl.ids_dev);
    cudaFree(sl.sc_dev);
  }
  delete sv;
  return SOAR_OK;
}

}  // extern "C"
