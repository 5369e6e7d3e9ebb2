// cc_server.cu -- serving loop with continuous batching (C ABI cc_server_*).
//
// Requests (graph, algorithm, eps, seed) are queued by cc_server_submit.  A
// dispatcher thread turns the queue into batched launches of the in-kernel
// pipeline (one thread block per job, see cc_rounds.cu) on a small set of
// streams: whenever a stream is free and the device-memory budget has room
// for the scratch of the next batch, the requests waiting at that moment
// form a batch and start, even while earlier batches still run on the other
// streams.  Graphs stay resident (they are the caller's cc_graph objects);
// each batch borrows scratch slots sized for its largest graph and returns
// them when its completion event fires.  A request's result is exactly the
// result of the same cc_cluster call: jobs never share state.
//
// Graphs above the one-block size limit are run on the whole GPU, one at a
// time, on the dispatcher thread.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/cc.h"
#include "cc_graph_impl.h"
#include "cc_internal.h"

using namespace ccg;

namespace {

constexpr int64_t kServeSmallN = 1 << 16;   // one thread block per job up to this size
constexpr int kStreams = 3;

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket;
  cc_graph* g;
  int algo;
  int64_t eps_ppm;
  double eps;
  uint64_t seed;
  int32_t* labels;       // device, may be null
  Clock::time_point t_submit;
};

struct Result {
  int status = CC_ERR_BUSY;    // CC_ERR_BUSY while pending
  int32_t rounds = 0;
  int64_t D = 0;
  double latency_ms = 0.0;
};

struct Flight {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  BatchJob* jobs_dev = nullptr;
  RoundBuffers* slots_dev = nullptr;
  std::vector<BatchJob> jobs;
  std::vector<int64_t> tickets;
  std::vector<Clock::time_point> t_submit;
};

}  // namespace

struct cc_server {
  int device = 0;
  size_t budget = 0;
  size_t in_use = 0;
  int max_batch = 0;
  int grid = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> pending;
  std::unordered_map<int64_t, Result> results;
  int64_t next_ticket = 1;
  bool stop = false;
  int fatal = CC_OK;
  Flight fl[kStreams];
  std::thread worker;
};

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return CC_OK;
  return e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA;
}

// Launch one batch on flight f.  Called without the lock held.
int start_batch(cc_server* sv, Flight& f, std::vector<Request>& reqs) {
  const int64_t n_max = std::max_element(reqs.begin(), reqs.end(), [](const Request& a, const Request& b) {
                          return a.g->n < b.g->n;
                        })->g->n;
  const int algo = reqs[0].algo;
  const int64_t ppm = reqs[0].eps_ppm;
  const int teams = std::min<int>((int)reqs.size(), sv->grid);
  const size_t slot = align_up(batch_slot_bytes(n_max, 1));
  f.ws_bytes = slot * (size_t)teams;
  cudaError_t e = pool_malloc(&f.ws, f.ws_bytes, f.stream);
  if (e != cudaSuccess) return cuda_status(e);
  std::vector<RoundBuffers> slots((size_t)teams);
  for (int t = 0; t < teams; ++t) {
    batch_slot_carve(static_cast<char*>(f.ws) + slot * (size_t)t, n_max, 1, &slots[(size_t)t]);
    if ((e = cudaMemsetAsync(slots[(size_t)t].ctl, 0, sizeof(Ctl), f.stream)) != cudaSuccess) return cuda_status(e);
  }
  f.jobs.assign(reqs.size(), BatchJob{});
  f.tickets.clear();
  f.t_submit.clear();
  // largest job first (the kernel deals jobs to blocks in order)
  std::sort(reqs.begin(), reqs.end(), [](const Request& a, const Request& b) { return a.g->n > b.g->n; });
  for (size_t q = 0; q < reqs.size(); ++q) {
    const cc_graph* g = reqs[q].g;
    BatchJob& jb = f.jobs[q];
    jb.off = g->off; jb.col = g->col; jb.nz = g->nz_row; jb.nz_n = g->nz_n;
    jb.dsort = g->dsort; jb.dge = g->dge;
    jb.n = g->n; jb.nnz = g->nnz; jb.max_deg = g->max_deg;
    jb.seed = reqs[q].seed;
    jb.labels = reqs[q].labels;
    jb.err = 1;
    f.tickets.push_back(reqs[q].ticket);
    f.t_submit.push_back(reqs[q].t_submit);
  }
  if ((e = pool_malloc(reinterpret_cast<void**>(&f.jobs_dev), sizeof(BatchJob) * f.jobs.size(), f.stream)) != cudaSuccess) return cuda_status(e);
  if ((e = pool_malloc(reinterpret_cast<void**>(&f.slots_dev), sizeof(RoundBuffers) * slots.size(), f.stream)) != cudaSuccess)
    return cuda_status(e);
  cudaMemcpyAsync(f.jobs_dev, f.jobs.data(), sizeof(BatchJob) * f.jobs.size(), cudaMemcpyHostToDevice, f.stream);
  cudaMemcpyAsync(f.slots_dev, slots.data(), sizeof(RoundBuffers) * slots.size(), cudaMemcpyHostToDevice, f.stream);
  if ((e = launch_batch_blocks(f.jobs_dev, (int)f.jobs.size(), f.slots_dev, teams, algo, ppm, f.stream)) != cudaSuccess)
    return cuda_status(e);
  cudaMemcpyAsync(f.jobs.data(), f.jobs_dev, sizeof(BatchJob) * f.jobs.size(), cudaMemcpyDeviceToHost, f.stream);
  if ((e = cudaEventRecord(f.done, f.stream)) != cudaSuccess) return cuda_status(e);
  f.busy = true;
  return CC_OK;
}

void finish_batch(cc_server* sv, Flight& f, std::unique_lock<std::mutex>& lk) {
  const auto now = Clock::now();
  cudaFreeAsync(f.jobs_dev, f.stream);
  cudaFreeAsync(f.slots_dev, f.stream);
  cudaFreeAsync(f.ws, f.stream);
  f.jobs_dev = nullptr;
  f.slots_dev = nullptr;
  f.ws = nullptr;
  sv->in_use -= f.ws_bytes;
  for (size_t q = 0; q < f.jobs.size(); ++q) {
    Result& r = sv->results[f.tickets[q]];
    r.status = f.jobs[q].err == 0 ? CC_OK : (f.jobs[q].err == CC_ERR_TIMEOUT ? CC_ERR_TIMEOUT : CC_ERR_INTERNAL);
    r.rounds = (int32_t)f.jobs[q].rounds;
    r.D = f.jobs[q].D;
    r.latency_ms = std::chrono::duration<double, std::milli>(now - f.t_submit[q]).count();
  }
  f.busy = false;
  (void)lk;
}

void dispatcher(cc_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    // reap finished batches
    for (auto& f : sv->fl) {
      if (f.busy && cudaEventQuery(f.done) == cudaSuccess) {
        finish_batch(sv, f, lk);
        sv->cv_done.notify_all();
      }
    }
    bool any_busy = false;
    for (auto& f : sv->fl) any_busy |= f.busy;
    if (sv->stop && sv->pending.empty() && !any_busy) break;
    // start a batch on a free stream if work and memory allow
    Flight* free_f = nullptr;
    for (auto& f : sv->fl)
      if (!f.busy) { free_f = &f; break; }
    if (free_f && !sv->pending.empty()) {
      Request head = sv->pending.front();
      if (head.g->n > kServeSmallN) {
        // large graph: whole GPU, synchronously
        sv->pending.pop_front();
        lk.unlock();
        int32_t r = 0;
        int64_t d = 0;
        const int st = cc_cluster(head.g, head.algo, head.eps, head.seed, head.labels, &r, &d);
        lk.lock();
        Result& res = sv->results[head.ticket];
        res.status = st;
        res.rounds = r;
        res.D = d;
        res.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - head.t_submit).count();
        sv->cv_done.notify_all();
        continue;
      }
      // gather the waiting small requests of the same algorithm and eps
      std::vector<Request> batch;
      int64_t n_max = 0;
      size_t need = 0;
      for (auto it = sv->pending.begin(); it != sv->pending.end() && (int)batch.size() < sv->max_batch;) {
        if (it->g->n > kServeSmallN || it->algo != head.algo || it->eps_ppm != head.eps_ppm) { ++it; continue; }
        const int64_t nm = std::max(n_max, it->g->n);
        const size_t nb = align_up(batch_slot_bytes(nm, 1)) * (size_t)std::min<int>((int)batch.size() + 1, sv->grid);
        if (sv->in_use + nb > sv->budget) {
          if (batch.empty() && !any_busy) {
            // this request alone exceeds the budget: it can never be admitted
            sv->results[it->ticket].status = CC_ERR_OOM;
            it = sv->pending.erase(it);
            sv->cv_done.notify_all();
            continue;
          }
          break;                                  // admit it when memory frees up
        }
        n_max = nm;
        need = nb;
        batch.push_back(*it);
        it = sv->pending.erase(it);
      }
      if (!batch.empty()) {
        sv->in_use += need;
        lk.unlock();
        const int st = start_batch(sv, *free_f, batch);
        lk.lock();
        if (st != CC_OK) {
          sv->in_use -= need;
          sv->fatal = st;
          for (auto& q : batch) sv->results[q.ticket].status = st;
          sv->cv_done.notify_all();
        }
        continue;
      }
    }
    // nothing to start: wait briefly for new work or completions
    sv->cv_work.wait_for(lk, std::chrono::microseconds(any_busy ? 20 : 2000));
  }
}

}  // namespace

extern "C" {

int cc_server_create(size_t mem_budget, int32_t max_batch, cc_server** out) {
  if (!out || mem_budget == 0 || max_batch < 1) return CC_ERR_INVALID_ARG;
  *out = nullptr;
  cc_server* sv = new (std::nothrow) cc_server();
  if (!sv) return CC_ERR_OOM;
  if (cudaGetDevice(&sv->device) != cudaSuccess) { delete sv; return CC_ERR_CUDA; }
  sv->budget = mem_budget;
  sv->max_batch = max_batch;
  sv->grid = batch_grid_size(sv->device);
  for (auto& f : sv->fl) {
    if (cudaStreamCreateWithFlags(&f.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming) != cudaSuccess) {
      for (auto& g : sv->fl) {
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.done) cudaEventDestroy(g.done);
      }
      delete sv;
      return CC_ERR_CUDA;
    }
  }
  sv->worker = std::thread(dispatcher, sv);
  *out = sv;
  return CC_OK;
}

int cc_server_submit(cc_server* sv, cc_graph* g, int algo, double eps, uint64_t seed, int32_t* labels_out,
                     int64_t* ticket) {
  if (!sv || !g || !ticket) return CC_ERR_INVALID_ARG;
  if (algo < CC_ALGO_C4 || algo > CC_ALGO_CLUSTERWILD_EST) return CC_ERR_INVALID_ARG;
  if (!(eps > 0.0) || !(eps <= 1.0)) return CC_ERR_INVALID_ARG;
  const long long ppm = std::llround(eps * 1e6);
  if (ppm < 1 || ppm > 1000000) return CC_ERR_INVALID_ARG;
  if (g->device != sv->device) return CC_ERR_INVALID_ARG;
  if (labels_out) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, labels_out) != cudaSuccess ||
        (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      return CC_ERR_INVALID_ARG;          // served labels go to device memory
    }
  }
  // the caller's work on the graph's stream must be visible to the server's streams
  if (cudaStreamSynchronize(g->stream) != cudaSuccess) return CC_ERR_CUDA;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stop) return CC_ERR_INVALID_ARG;
  if (sv->fatal != CC_OK) return sv->fatal;
  Request r;
  r.ticket = sv->next_ticket++;
  r.g = g;
  r.algo = algo;
  r.eps_ppm = ppm;
  r.eps = eps;
  r.seed = seed;
  r.labels = labels_out;
  r.t_submit = Clock::now();
  sv->pending.push_back(r);
  sv->results[r.ticket] = Result{};
  *ticket = r.ticket;
  sv->cv_work.notify_one();
  return CC_OK;
}

int cc_server_poll(cc_server* sv, int64_t ticket, int32_t* rounds, int64_t* disagreements, double* latency_ms) {
  if (!sv) return CC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->results.find(ticket);
  if (it == sv->results.end()) return CC_ERR_INVALID_ARG;
  if (it->second.status == CC_ERR_BUSY) return CC_ERR_BUSY;
  if (rounds) *rounds = it->second.rounds;
  if (disagreements) *disagreements = it->second.D;
  if (latency_ms) *latency_ms = it->second.latency_ms;
  return it->second.status;
}

int cc_server_wait(cc_server* sv, int64_t ticket, int32_t* rounds, int64_t* disagreements, double* latency_ms) {
  if (!sv) return CC_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->results.find(ticket);
  if (it == sv->results.end()) return CC_ERR_INVALID_ARG;
  const auto t0 = Clock::now();
  while (sv->results[ticket].status == CC_ERR_BUSY) {
    sv->cv_done.wait_for(lk, std::chrono::milliseconds(50));
    if (Clock::now() - t0 > std::chrono::seconds(600)) return CC_ERR_TIMEOUT;
  }
  const Result& r = sv->results[ticket];
  if (rounds) *rounds = r.rounds;
  if (disagreements) *disagreements = r.D;
  if (latency_ms) *latency_ms = r.latency_ms;
  return r.status;
}

int cc_server_destroy(cc_server* sv) {
  if (!sv) return CC_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv_work.notify_all();
  }
  if (sv->worker.joinable()) sv->worker.join();
  for (auto& f : sv->fl) {
    if (f.stream) {
      cudaStreamSynchronize(f.stream);
      cudaStreamDestroy(f.stream);
    }
    if (f.done) cudaEventDestroy(f.done);
  }
  delete sv;
  return CC_OK;
}

}  // extern "C"
