// cc_server.cu -- serving loop with continuous batching (C ABI cc_server_*).
//
// Requests (graph, algorithm, eps, seed) are queued by cc_server_submit.  A
// dispatcher thread turns the queue into launches of the in-kernel pipeline
// of cc_rounds.cu (a whole job -- permutation, rounds, objective, labels --
// inside one launch) and never waits for the GPU:
//
//   * small graphs (n <= batch_small_n of the batch settings, 2^16 by
//     default): one thread block per job, batched;
//   * medium graphs (n <= batch_team_n, 2^21): one team of batch_team_blocks
//     per job, batched in cooperative launches of at most kServeTeamMax teams,
//     kServeTeamFlights such launches in flight at a time (together at most
//     two thirds of the batched kernel's co-resident blocks, so that small
//     jobs always find room);
//   * larger graphs: the whole GPU per job (cc_cluster) on a worker thread of
//     their own, one at a time, so that they never hold up the dispatcher.
//
// Every batch runs on its own stream (kStreams of them).  Whenever a stream
// is free and the device-memory budget has room for a batch's scratch, the
// requests of one size class waiting at that moment form a batch and start,
// while earlier batches still run on the other streams: their work overlaps
// on the device.  Results come back into pinned host memory with an
// asynchronous copy, so starting a batch returns at once; the dispatcher
// notices completion by polling the batch's event.  A failed batch fails its
// own requests only.  A request's result is exactly that of the same
// cc_cluster call: jobs never share state.
#include <algorithm>
#include <chrono>
#include <cmath>
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
#include "cc_nvtx.h"

using namespace ccg;

namespace {

constexpr int kServeTeamMax = 16;            // teams per cooperative launch, at most
constexpr int kServeTeamFlights = 2;         // medium launches in flight at once
constexpr int kStreams = 16;             // launches in flight at once (one stream each)

using Clock = std::chrono::steady_clock;

enum Cls { kSmall = 0, kTeam = 1, kWhole = 2 };

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
  int64_t dev_t0 = -1, dev_t1 = -1;   // device clock at the job's start and end (batched jobs)
};

struct Flight {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  int cls = kSmall;
  size_t share = 0;              // bytes charged to the budget
  void* ws = nullptr;
  BatchJob* jobs_dev = nullptr;
  RoundBuffers* slots_dev = nullptr;
  BatchJob* jobs_host = nullptr; // pinned: the launch's jobs, then its results
  size_t jobs_cap = 0;
  RoundBuffers* slots_host = nullptr;   // pinned
  size_t slots_cap = 0;
  size_t njobs = 0;
  std::vector<int64_t> tickets;
  std::vector<Clock::time_point> t_submit;
};

}  // namespace

struct cc_server {
  int device = 0;
  size_t budget = 0;
  size_t in_use = 0;
  int max_batch = 0;
  int grid = 0;                  // co-resident blocks of the batched kernel
  // size classes and round settings (the batch settings when created):
  // one block per job up to small_n vertices, a team of team_blocks up to team_n
  int64_t small_n = 0, team_n = 0;
  int team_blocks = 0;
  Tuning tune;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_whole;
  std::deque<Request> pending;   // small and medium requests, in arrival order
  std::deque<Request> whole;     // requests for the whole-GPU worker
  std::unordered_map<int64_t, Result> results;
  int64_t next_ticket = 1;
  bool stop = false;
  bool whole_busy = false;
  Flight fl[kStreams];
  cudaStream_t whole_stream = nullptr;
  std::thread worker;            // dispatcher
  std::thread whole_worker;
};

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return CC_OK;
  return e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA;
}

int class_of(const cc_server* sv, int64_t n) { return n <= sv->small_n ? kSmall : (n <= sv->team_n ? kTeam : kWhole); }

int team_of(const cc_server* sv, int cls) { return cls == kSmall ? 1 : sv->team_blocks; }

// Teams of one launch: every job gets one while the launch stays co-resident
// (small: the batched kernel's whole grid; medium: kServeTeamMax teams).
int teams_for(const cc_server* sv, int cls, size_t jobs) {
  const int cap = cls == kSmall ? sv->grid
                                 : std::min(kServeTeamMax, sv->grid / sv->team_blocks / (kServeTeamFlights + 1));
  return (int)std::min<size_t>(jobs, (size_t)std::max(cap, 1));
}

size_t batch_bytes(const cc_server* sv, int cls, int64_t n_max, size_t jobs) {
  return align_up(batch_slot_bytes(n_max, team_of(sv, cls))) * (size_t)teams_for(sv, cls, jobs);
}

// Pinned host staging of a flight, grown when a batch needs more.
int ensure_host(Flight& f, size_t jobs, size_t slots) {
  if (f.jobs_cap < jobs) {
    if (f.jobs_host) cudaFreeHost(f.jobs_host);
    f.jobs_host = nullptr;
    f.jobs_cap = 0;
    if (cudaMallocHost(reinterpret_cast<void**>(&f.jobs_host), sizeof(BatchJob) * jobs) != cudaSuccess) {
      cudaGetLastError();
      return CC_ERR_OOM;
    }
    f.jobs_cap = jobs;
  }
  if (f.slots_cap < slots) {
    if (f.slots_host) cudaFreeHost(f.slots_host);
    f.slots_host = nullptr;
    f.slots_cap = 0;
    if (cudaMallocHost(reinterpret_cast<void**>(&f.slots_host), sizeof(RoundBuffers) * slots) != cudaSuccess) {
      cudaGetLastError();
      return CC_ERR_OOM;
    }
    f.slots_cap = slots;
  }
  return CC_OK;
}

void release_device(Flight& f) {
  if (f.jobs_dev) cudaFreeAsync(f.jobs_dev, f.stream);
  if (f.slots_dev) cudaFreeAsync(f.slots_dev, f.stream);
  if (f.ws) cudaFreeAsync(f.ws, f.stream);
  f.jobs_dev = nullptr;
  f.slots_dev = nullptr;
  f.ws = nullptr;
}

// Launch one batch of one size class on flight f; nothing here waits for the
// GPU.  Called without the lock held.  On failure everything the call
// allocated is released and the status returned.
int start_batch(cc_server* sv, Flight& f, int cls, std::vector<Request>& reqs) {
  NvtxRange range(cls == kSmall ? "cc_server batch: small" : "cc_server batch: team");
  const int64_t n_max = std::max_element(reqs.begin(), reqs.end(), [](const Request& a, const Request& b) {
                          return a.g->n < b.g->n;
                        })->g->n;
  const int algo = reqs[0].algo;
  const int64_t ppm = reqs[0].eps_ppm;
  const int team = team_of(sv, cls);
  const int teams = teams_for(sv, cls, reqs.size());
  const size_t slot = align_up(batch_slot_bytes(n_max, team));
  int rc = ensure_host(f, reqs.size(), (size_t)teams);
  if (rc != CC_OK) return rc;
  cudaError_t e = pool_malloc(&f.ws, slot * (size_t)teams, f.stream);
  if (e == cudaSuccess)
    e = pool_malloc(reinterpret_cast<void**>(&f.jobs_dev), sizeof(BatchJob) * reqs.size(), f.stream);
  if (e == cudaSuccess)
    e = pool_malloc(reinterpret_cast<void**>(&f.slots_dev), sizeof(RoundBuffers) * (size_t)teams, f.stream);
  for (int t = 0; t < teams && e == cudaSuccess; ++t) {
    batch_slot_carve(static_cast<char*>(f.ws) + slot * (size_t)t, n_max, team, &f.slots_host[t]);
    f.slots_host[t].tune = sv->tune;
    e = cudaMemsetAsync(f.slots_host[t].ctl, 0, sizeof(Ctl), f.stream);
  }
  if (e != cudaSuccess) {
    release_device(f);
    return cuda_status(e);
  }
  // largest job first (the kernel deals jobs to teams in order)
  std::sort(reqs.begin(), reqs.end(), [](const Request& a, const Request& b) { return a.g->n > b.g->n; });
  f.tickets.clear();
  f.t_submit.clear();
  for (size_t q = 0; q < reqs.size(); ++q) {
    const cc_graph* g = reqs[q].g;
    BatchJob& jb = f.jobs_host[q];
    jb = BatchJob{};
    jb.off = g->off; jb.col = g->col; jb.nz = g->nz_row; jb.nz_n = g->nz_n;
    jb.dsort = g->dsort; jb.dge = g->dge;
    jb.n = g->n; jb.nnz = g->nnz; jb.max_deg = g->max_deg;
    jb.seed = reqs[q].seed;
    jb.labels = reqs[q].labels;
    jb.err = 1;
    jb.t0 = jb.t1 = -1;
    f.tickets.push_back(reqs[q].ticket);
    f.t_submit.push_back(reqs[q].t_submit);
  }
  f.njobs = reqs.size();
  e = cudaMemcpyAsync(f.jobs_dev, f.jobs_host, sizeof(BatchJob) * f.njobs, cudaMemcpyHostToDevice, f.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(f.slots_dev, f.slots_host, sizeof(RoundBuffers) * (size_t)teams, cudaMemcpyHostToDevice,
                        f.stream);
  if (e == cudaSuccess) {
    e = cls == kSmall ? launch_batch_blocks(f.jobs_dev, (int)f.njobs, f.slots_dev, teams, algo, ppm, f.stream)
                      : launch_batch(f.jobs_dev, (int)f.njobs, f.slots_dev, team, teams * team, algo, ppm, f.stream);
  }
  // the results land in the pinned copy of the jobs: the copy is asynchronous
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(f.jobs_host, f.jobs_dev, sizeof(BatchJob) * f.njobs, cudaMemcpyDeviceToHost, f.stream);
  if (e == cudaSuccess) e = cudaEventRecord(f.done, f.stream);
  if (e != cudaSuccess) {
    // whatever was queued must finish before the staging is reused
    cudaStreamSynchronize(f.stream);
    cudaGetLastError();
    release_device(f);
    return cuda_status(e);
  }
  f.cls = cls;
  f.busy = true;
  return CC_OK;
}

void finish_batch(cc_server* sv, Flight& f, cudaError_t ev) {
  const auto now = Clock::now();
  release_device(f);
  sv->in_use -= f.share;
  f.share = 0;
  for (size_t q = 0; q < f.njobs; ++q) {
    Result& r = sv->results[f.tickets[q]];
    const BatchJob& jb = f.jobs_host[q];
    if (ev != cudaSuccess) r.status = cuda_status(ev);
    else r.status = jb.err == 0 ? CC_OK : (jb.err == CC_ERR_TIMEOUT ? CC_ERR_TIMEOUT : CC_ERR_INTERNAL);
    r.rounds = (int32_t)jb.rounds;
    r.D = jb.D;
    r.dev_t0 = jb.t0;
    r.dev_t1 = jb.t1;
    r.latency_ms = std::chrono::duration<double, std::milli>(now - f.t_submit[q]).count();
  }
  f.busy = false;
}

// Whole-GPU requests, one at a time, on their own thread.
void whole_worker(cc_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    sv->cv_whole.wait(lk, [&] { return sv->stop || !sv->whole.empty(); });
    if (sv->whole.empty()) {
      if (sv->stop) break;
      continue;
    }
    Request q = sv->whole.front();
    sv->whole.pop_front();
    sv->whole_busy = true;
    lk.unlock();
    int32_t r = 0;
    int64_t d = 0;
    // on the server's own stream (the graph's may be a blocking or the
    // legacy stream, which would serialise with the batches); the graph is
    // the server's while its request runs, and the call waits for its work
    cudaStream_t own = q.g->stream;
    q.g->stream = sv->whole_stream;
    const int st = cc_cluster(q.g, q.algo, q.eps, q.seed, q.labels, &r, &d);
    q.g->stream = own;
    lk.lock();
    Result& res = sv->results[q.ticket];
    res.status = st;
    res.rounds = r;
    res.D = d;
    res.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - q.t_submit).count();
    sv->whole_busy = false;
    sv->cv_done.notify_all();
  }
}

// Gather the waiting requests of size class cls that share the first one's
// algorithm and eps, as far as the budget allows.  Called with the lock held.
// Returns false when nothing can start now.
bool gather(cc_server* sv, int cls, bool any_busy, std::vector<Request>& batch, size_t* need) {
  batch.clear();
  *need = 0;
  int64_t n_max = 0;
  for (auto it = sv->pending.begin(); it != sv->pending.end() && (int)batch.size() < sv->max_batch;) {
    if (class_of(sv, it->g->n) != cls ||
        (!batch.empty() && (it->algo != batch.front().algo || it->eps_ppm != batch.front().eps_ppm))) {
      ++it;
      continue;
    }
    const int64_t nm = std::max(n_max, it->g->n);
    const size_t nb = batch_bytes(sv, cls, nm, batch.size() + 1);
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
    *need = nb;
    batch.push_back(*it);
    it = sv->pending.erase(it);
  }
  return !batch.empty();
}

void dispatcher(cc_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  std::vector<Request> batch;
  for (;;) {
    // reap finished batches
    for (auto& f : sv->fl) {
      if (!f.busy) continue;
      const cudaError_t q = cudaEventQuery(f.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) cudaGetLastError();
      finish_batch(sv, f, q);
      sv->cv_done.notify_all();
    }
    bool any_busy = false;
    int team_busy = 0;
    for (auto& f : sv->fl) {
      any_busy |= f.busy;
      team_busy += (f.busy && f.cls == kTeam) ? 1 : 0;
    }
    if (sv->stop && sv->pending.empty() && !any_busy) break;
    // start batches on free streams: small requests, and medium ones while
    // fewer than kServeTeamFlights medium launches are in flight
    bool started = false;
    for (int cls : {kSmall, kTeam}) {
      if (cls == kTeam && team_busy >= kServeTeamFlights) continue;
      Flight* free_f = nullptr;
      for (auto& f : sv->fl)
        if (!f.busy) { free_f = &f; break; }
      if (!free_f) break;
      size_t need = 0;
      if (!gather(sv, cls, any_busy, batch, &need)) continue;
      sv->in_use += need;
      free_f->share = need;
      free_f->busy = true;                    // reserved while the lock is released
      lk.unlock();
      const int st = start_batch(sv, *free_f, cls, batch);
      lk.lock();
      if (st != CC_OK) {
        // this batch's requests fail; the server carries on
        free_f->busy = false;
        sv->in_use -= need;
        free_f->share = 0;
        for (auto& q : batch) sv->results[q.ticket].status = st;
        sv->cv_done.notify_all();
      }
      started = true;
      any_busy = true;
      if (cls == kTeam) ++team_busy;
    }
    if (started) continue;
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
  sv->tune = batch_settings(&sv->small_n, &sv->team_n, &sv->team_blocks);
  for (auto& f : sv->fl) {
    if (cudaStreamCreateWithFlags(&f.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      for (auto& g : sv->fl) {
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.done) cudaEventDestroy(g.done);
      }
      delete sv;
      return CC_ERR_CUDA;
    }
  }
  if (cudaStreamCreateWithFlags(&sv->whole_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    for (auto& g : sv->fl) {
      cudaStreamDestroy(g.stream);
      cudaEventDestroy(g.done);
    }
    delete sv;
    return CC_ERR_CUDA;
  }
  sv->worker = std::thread(dispatcher, sv);
  sv->whole_worker = std::thread(whole_worker, sv);
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
  // no wait here: cc_graph_create returns with the graph on the device, and
  // the server only reads it
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stop) return CC_ERR_INVALID_ARG;
  Request r;
  r.ticket = sv->next_ticket++;
  r.g = g;
  r.algo = algo;
  r.eps_ppm = ppm;
  r.eps = eps;
  r.seed = seed;
  r.labels = labels_out;
  r.t_submit = Clock::now();
  sv->results[r.ticket] = Result{};
  *ticket = r.ticket;
  if (class_of(sv, g->n) == kWhole) {
    sv->whole.push_back(r);
    sv->cv_whole.notify_one();
  } else {
    sv->pending.push_back(r);
    sv->cv_work.notify_one();
  }
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
  while (it->second.status == CC_ERR_BUSY) {
    sv->cv_done.wait_for(lk, std::chrono::milliseconds(50));
    if (Clock::now() - t0 > std::chrono::seconds(600)) return CC_ERR_TIMEOUT;
  }
  const Result& r = it->second;
  if (rounds) *rounds = r.rounds;
  if (disagreements) *disagreements = r.D;
  if (latency_ms) *latency_ms = r.latency_ms;
  return r.status;
}

int cc_server_device_times(cc_server* sv, int64_t ticket, int64_t* start_ns, int64_t* end_ns) {
  if (!sv || !start_ns || !end_ns) return CC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->results.find(ticket);
  if (it == sv->results.end()) return CC_ERR_INVALID_ARG;
  if (it->second.status == CC_ERR_BUSY) return CC_ERR_BUSY;
  *start_ns = it->second.dev_t0;
  *end_ns = it->second.dev_t1;
  return CC_OK;
}

int cc_server_destroy(cc_server* sv) {
  if (!sv) return CC_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv_work.notify_all();
    sv->cv_whole.notify_all();
  }
  if (sv->worker.joinable()) sv->worker.join();
  if (sv->whole_worker.joinable()) sv->whole_worker.join();
  if (sv->whole_stream) cudaStreamDestroy(sv->whole_stream);
  for (auto& f : sv->fl) {
    if (f.stream) {
      cudaStreamSynchronize(f.stream);
      cudaStreamDestroy(f.stream);
    }
    if (f.done) cudaEventDestroy(f.done);
    if (f.jobs_host) cudaFreeHost(f.jobs_host);
    if (f.slots_host) cudaFreeHost(f.slots_host);
  }
  delete sv;
  return CC_OK;
}

}  // extern "C"
