// Serving loop: evolve requests of different n and T as they arrive, with their
// states resident on the device, admitted by free device memory, small
// instances batched into one launch, larger ones overlapped on a stream pool.
//
// Memory: the server reserves one device arena at creation and sub-allocates
// every request's state, clause tables, phase tables and reduction scratch from
// it with a host-side first-fit allocator, so serving never calls cudaMalloc or
// cudaFree (either can synchronise the whole device).  A request is admitted
// when its block fits in the arena and a result slot is free; it keeps its
// block until its observables are read back.
//
// Work: admitted requests with n <= 14 are gathered into one launch of the
// batched on-chip evolver (one CTA per request, whole run in shared memory);
// requests with 15 <= n <= 17 get one persistent cooperative launch each
// (persist.cu) on a few SMs, several running side by side; larger requests go
// to issuer threads, each with its own stream, which launch the streaming
// passes of the request's plan.  Completion is observed with one
// event per request; the worker then reads the FP64 observables from a pinned
// slot and releases the memory.
//
// Latency is measured on the host steady clock: t_submit (qaa_submit),
// t_admit (memory granted), t_done (results read back).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine_internal.h"
#include "qaa.h"
#include "qaa_internal.cuh"

namespace {

qaa_status sfail(int code, const std::string& msg) {
  qaa::set_last_error(msg);
  return static_cast<qaa_status>(code);
}

constexpr size_t kAlign = 256;
// Pinned staging per result slot for a request's two clause tables: copies
// from pinned memory are asynchronous, copies from pageable memory first
// synchronise the stream (which would stall the worker behind the device).
constexpr size_t kStageBytes = 2u * 16u * QAA_MAX_CLAUSES;
constexpr long long kPersistMaxSteps = 1ll << 16;
size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, size): free blocks by offset.
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    free_[0] = size;
    size_ = size;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t size() const { return size_; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0, used_ = 0;
};

enum Phase { kQueued, kAdmitted, kRunning, kDone };

struct Req {
  uint64_t ticket = 0;
  int n = 0, m = 0;
  double T = 0.0;
  long long K = 0;
  std::vector<qaa::ClauseMV> mv;
  std::vector<qaa::ClauseLP> lp;
  qaa::PassPlan plan;
  double t_submit = 0, t_admit = -1, t_done = -1;
  double t_dev_start = -1, t_dev_end = -1;  // device clock, seconds since the server's reference event
  int status = QAA_PENDING;
  double res[5] = {0, 0, 0, 0, 0};
  Phase phase = kQueued;
  bool cancel = false;
  // device block
  size_t off = 0, bytes = 0;
  int slot = -1;
  float2* psi = nullptr;
  qaa::ClauseMV* d_mv = nullptr;
  qaa::ClauseLP* d_lp = nullptr;
  float2* d_tab = nullptr;
  double* d_part = nullptr;
  double* d_res = nullptr;
  int* d_err = nullptr;
  long long chunk = 0;
  unsigned* d_bar = nullptr;
  unsigned* d_counts = nullptr;  // stored per-tile clause counts (streamed requests), else null
  size_t counts_bytes = 0;
  double* d_fold = nullptr;  // norm-fold slots of the low passes (streamed and persistent requests)
  cudaEvent_t done_ev = nullptr;
  cudaGraphExec_t gexec = nullptr;  // launch graph of a streamed request, kept until it completes
  bool persist = false;  // mid-size: one persistent cooperative launch for the whole run
  bool graph = false;    // streamed: one launch graph for the whole run
  bool small() const { return plan.onchip; }
  bool persistent() const { return persist; }
};

// Phase-table bytes of a request: the whole run for on-chip and persistent
// requests, the graph scratch (8 steps of rows) for launch-graph requests, a
// chunk of at most 1024 steps for per-pass launches.
size_t table_bytes(int n, int m, long long K, bool whole_run, bool graph) {
  if (graph) return qaa::graph_scratch_bytes(n, m);
  return 8u * qaa::table_entries(n, m, whole_run ? K : std::min(qaa::kChunkSteps, K));
}

// Device bytes of one request: state, clause tables, phase tables, reduction
// partials, results, an error word, a grid-barrier word pair and, beyond the
// on-chip sizes, the low passes' norm-fold slots.
size_t request_bytes(int n, int m, size_t tab_bytes, size_t counts_bytes, int num_sms) {
  size_t b = align_up((static_cast<size_t>(8) << n));
  b += align_up(counts_bytes);
  if (n > qaa::kOnchipMaxBits) b += align_up(qaa::kFoldBytes);
  b += align_up(16u * static_cast<size_t>(std::max(m, 1))) * 2;
  b += align_up(tab_bytes);
  b += align_up(8u * qaa::obs_partials_len(n, num_sms));
  b += align_up(64) + align_up(16) + align_up(16);
  return b;
}

double steady_now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct qaa_server {
  int device = 0, num_sms = 0;
  int max_slots = 0;
  char* arena_base = nullptr;
  Arena arena;
  std::vector<int> free_slots;
  // pinned, 8 doubles per slot: results [0..4], error word [5], the device
  // interval's start and end stamps [6], [7] (global_ns of the device)
  double* h_res = nullptr;
  unsigned char* h_stage = nullptr;  // pinned clause-table staging, kStageBytes per slot
  double t0 = 0;
  unsigned long long ref_ns = 0;  // device-clock origin of the requests' device intervals
  // submission (guarded by mu)
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> incoming;
  std::unordered_map<uint64_t, Req*> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  // worker-only lists
  std::vector<Req*> waiting, running, small_pending;
  // issuers (guarded by imu)
  std::mutex imu;
  std::condition_variable icv;
  std::deque<Req*> issue_q;
  std::vector<Req*> issued;
  std::vector<std::thread> issuers;
  std::vector<cudaStream_t> issue_streams;
  bool issue_stop = false;
  // mid-size requests: persistent launches, round robin over these streams
  std::vector<cudaStream_t> persist_streams;
  int persist_turn = 0;
  int persist_grid = 32;      // CTAs per persistent request, at most
  int persist_max_bits = 0;   // largest n served by a persistent launch (0: none)
  // Streamed requests as one launch graph each (QAA_SERVER_GRAPHS=1).  Off by
  // default: on the n ~ U{10..22} mix it measured 202-210 solves/s (4 or 8
  // issuers) against 219 with per-pass launches from 4 issuers -- the graph
  // makes one request's steps faster but several n = 20..22 requests then
  // contend for L2 and HBM at once.
  bool use_graphs = false;
  int graph_max_bits = 0;  // streamed requests with n <= this run as one launch graph
  // small-request batches
  cudaStream_t batch_stream = nullptr;
  qaa::OnchipJob* h_jobs[2] = {nullptr, nullptr};
  qaa::OnchipJob* d_jobs[2] = {nullptr, nullptr};
  cudaEvent_t jobs_ev[2] = {nullptr, nullptr};
  int jobs_turn = 0;
  std::thread worker;
  // statistics and test hooks (guarded by mu)
  long long batches = 0, batched = 0, streamed = 0, peak_used = 0;
  std::atomic<int> inject_delay_ms{0};
  std::atomic<int> inject_fail{0};
  std::atomic<int> inject_stuck_barrier{0};
  std::string fatal;
};

namespace {

void finish(qaa_server* s, Req* r, int status) {
  r->status = status;
  r->t_done = steady_now() - s->t0;
  r->phase = kDone;
}

void release(qaa_server* s, Req* r) {
  if (r->done_ev) {
    cudaEventDestroy(r->done_ev);
    r->done_ev = nullptr;
  }
  if (r->gexec) {
    cudaGraphExecDestroy(r->gexec);
    r->gexec = nullptr;
  }
  if (r->bytes) {
    s->arena.release(r->off, r->bytes);
    r->bytes = 0;
  }
  if (r->slot >= 0) {
    s->free_slots.push_back(r->slot);
    r->slot = -1;
  }
}

// Carve the request's device block and upload its clause tables (on `stream`).
bool place(qaa_server* s, Req* r) {
  r->chunk = (r->small() || r->persistent()) ? r->K : std::min(qaa::kChunkSteps, r->K);
  const size_t tb = table_bytes(r->n, r->m, r->K, r->small() || r->persistent(), r->graph);
  const size_t need = request_bytes(r->n, r->m, tb, r->counts_bytes, s->num_sms);
  if (s->free_slots.empty()) return false;
  size_t off = 0;
  if (!s->arena.alloc(need, &off)) return false;
  r->off = off;
  r->bytes = need;
  r->slot = s->free_slots.back();
  s->free_slots.pop_back();
  char* p = s->arena_base + off;
  auto take = [&](size_t b) {
    char* q = p;
    p += align_up(b);
    return q;
  };
  r->psi = reinterpret_cast<float2*>(take(static_cast<size_t>(8) << r->n));
  r->d_mv = reinterpret_cast<qaa::ClauseMV*>(take(16u * std::max(r->m, 1)));
  r->d_lp = reinterpret_cast<qaa::ClauseLP*>(take(16u * std::max(r->m, 1)));
  r->d_tab = reinterpret_cast<float2*>(take(tb));
  r->d_part = reinterpret_cast<double*>(take(8u * qaa::obs_partials_len(r->n, s->num_sms)));
  r->d_res = reinterpret_cast<double*>(take(64));
  r->d_err = reinterpret_cast<int*>(take(16));
  r->d_bar = reinterpret_cast<unsigned*>(take(16));
  r->d_counts = r->counts_bytes ? reinterpret_cast<unsigned*>(take(r->counts_bytes)) : nullptr;
  r->d_fold = r->n > qaa::kOnchipMaxBits ? reinterpret_cast<double*>(take(qaa::kFoldBytes)) : nullptr;
  return true;
}

cudaError_t upload_tables(qaa_server* s, Req* r, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (r->m > 0) {
    unsigned char* stage = s->h_stage + kStageBytes * static_cast<size_t>(r->slot);
    std::memcpy(stage, r->mv.data(), 16u * r->m);
    std::memcpy(stage + 16u * QAA_MAX_CLAUSES, r->lp.data(), 16u * r->m);
    e = cudaMemcpyAsync(r->d_mv, stage, 16u * r->m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r->d_lp, stage + 16u * QAA_MAX_CLAUSES, 16u * r->m, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(r->d_err, 0, sizeof(int), st);
  return e;
}

// The request's device-interval stamps, in its result block after the five
// results: [6] the start (global_ns before its first device work), [7] the end
// (written by the observables' last kernel).
unsigned long long* stamp_start(Req* r) { return reinterpret_cast<unsigned long long*>(r->d_res + 6); }
unsigned long long* stamp_end(Req* r) { return reinterpret_cast<unsigned long long*>(r->d_res + 7); }

// Observables of a finished evolution into the request's pinned slot (with
// the device-interval stamps), then the completion event.
cudaError_t observe_async(qaa_server* s, Req* r, cudaStream_t st) {
  const qaa::LaunchCtx lc{st, s->num_sms};
  cudaError_t e = qaa::launch_observables(lc, r->psi, r->n, r->m, r->d_lp, r->d_part, r->d_res, r->d_counts, r->d_err,
                                          stamp_end(r));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->h_res + 8 * r->slot, r->d_res, 8 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_res + 8 * r->slot + 5, r->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  // no timing: events with timing recorded on the persistent streams were
  // measured to serialise their cooperative launches (half the throughput)
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r->done_ev, st);
  return e;
}

// The start of a request's device interval: a stamp on its stream ahead of
// its first copy or kernel.
cudaError_t mark_start(qaa_server* s, Req* r, cudaStream_t st) {
  return qaa::launch_stamp(qaa::LaunchCtx{st, s->num_sms}, stamp_start(r));
}

// The streaming evolution of one request (issuer thread, its own stream):
// one launch graph for the whole run, or one launch per pass.

cudaError_t issue_streaming(qaa_server* s, Req* r, cudaStream_t st) {
  const qaa::LaunchCtx lc{st, s->num_sms};
  cudaError_t e = mark_start(s, r, st);
  if (e == cudaSuccess) e = upload_tables(s, r, st);
  if (e == cudaSuccess) e = qaa::launch_init_uniform(lc, r->psi, r->n);
  if (e == cudaSuccess && r->d_counts) e = qaa::launch_lp_counts(lc, r->d_counts, r->n, r->m, r->d_lp);
  const double dt = r->T / static_cast<double>(r->K);
  if (r->graph) {
    qaa::GraphSpec gs;
    gs.plan = &r->plan;
    gs.psi = r->psi;
    gs.m = r->m;
    gs.cl = r->d_lp;
    gs.err = r->d_err;
    gs.dt = dt;
    gs.K = r->K;
    gs.k0 = 0;
    gs.k1 = r->K;
    gs.num_sms = s->num_sms;
    gs.counts = r->d_counts;
    gs.fold = r->d_fold;
    qaa::graph_scratch_split(r->d_tab, r->m, gs);
    if (e == cudaSuccess) e = qaa::build_evolve_graph(gs, &r->gexec);
    if (e == cudaSuccess) e = cudaGraphLaunch(r->gexec, st);
    if (e == cudaSuccess) e = observe_async(s, r, st);
    return e;
  }
  float2* ptab = r->d_tab;
  float2* btab = r->d_tab + static_cast<size_t>(r->chunk + 1) * (r->m + 1);
  std::vector<qaa::Pass> passes;
  for (long long c0 = 0; e == cudaSuccess && c0 < r->K; c0 += r->chunk) {
    const long long c1 = std::min(r->K, c0 + r->chunk);
    e = qaa::launch_tables(lc, ptab, btab, r->n, r->m, dt, nullptr, r->K, 0, r->K, c0, c1,
                           r->plan.wht_kind == qaa::kRotationForm);
    qaa::build_passes(r->plan, 0, r->K, c0, c1, passes);
    for (const qaa::Pass& ps : passes) {
      if (e != cudaSuccess) break;
      e = qaa::launch_planned_pass(lc, r->plan, ps, r->psi, r->m, r->d_lp, ptab, btab, r->d_err, r->d_counts,
                                   r->d_fold);
    }
  }
  if (e == cudaSuccess) e = observe_async(s, r, st);
  return e;
}

// A mid-size request: tables for the whole run and one persistent cooperative
// launch on a few CTAs, so several such requests share the GPU at once.
cudaError_t issue_persistent(qaa_server* s, Req* r, cudaStream_t st) {
  const qaa::LaunchCtx lc{st, s->num_sms};
  cudaError_t e = mark_start(s, r, st);
  if (e == cudaSuccess) e = upload_tables(s, r, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(r->d_bar, 0, 2 * sizeof(unsigned), st);
  // injected fault: the arrival count starts at 2^32 - 1, so the first grid
  // barrier never sees all CTAs arrive; they give up after the bound, record
  // the error word and return (the request ends with QAA_E_TIMEOUT)
  if (e == cudaSuccess && s->inject_stuck_barrier.exchange(0)) e = cudaMemsetAsync(r->d_bar, 0xFF, sizeof(unsigned), st);
  if (e == cudaSuccess) e = qaa::launch_init_uniform(lc, r->psi, r->n);
  float2* ptab = r->d_tab;
  float2* btab = r->d_tab + static_cast<size_t>(r->K + 1) * (r->m + 1);
  if (e == cudaSuccess)
    e = qaa::launch_tables(lc, ptab, btab, r->n, r->m, r->T / static_cast<double>(r->K), nullptr, r->K, 0, r->K, 0,
                           r->K);
  qaa::PersistPlan pp{};
  pp.ng = static_cast<int>(r->plan.strided.size());
  pp.phase_group = r->plan.phase_group;
  for (int g = 0; g < pp.ng && g < 3; ++g) {
    pp.ga[g] = r->plan.strided[g].a;
    pp.gq[g] = r->plan.strided[g].q;
  }
  const int grid = static_cast<int>(std::min<long long>(1ll << std::max(r->n - 13, 0), s->persist_grid));
  if (e == cudaSuccess)
    e = qaa::launch_persist(lc, pp, r->psi, r->n, r->m, r->d_lp, ptab, btab, static_cast<int>(r->K), r->d_bar,
                            r->d_err, grid, r->d_fold);
  if (e == cudaSuccess) e = observe_async(s, r, st);
  return e;
}

void issuer_main(qaa_server* s, int idx) {
  cudaSetDevice(s->device);
  cudaStream_t st = s->issue_streams[idx];
  for (;;) {
    Req* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->imu);
      s->icv.wait(lk, [&] { return s->issue_stop || !s->issue_q.empty(); });
      if (s->issue_q.empty()) return;
      r = s->issue_q.front();
      s->issue_q.pop_front();
    }
    const cudaError_t e = issue_streaming(s, r, st);
    if (e != cudaSuccess) {
      cudaStreamSynchronize(st);  // work already queued must finish before the block is reused
      cudaGetLastError();
      r->status = QAA_E_CUDA;  // reported when the worker picks it up
    }
    {
      std::lock_guard<std::mutex> lk(s->imu);
      s->issued.push_back(r);
    }
    s->cv.notify_all();
  }
}

// One launch for every admitted small request.  Returns false (nothing
// launched) while the staging buffer is still read by an earlier batch; the
// worker never blocks on the device.
bool launch_batch(qaa_server* s, std::vector<Req*>& small) {
  if (small.empty()) return true;
  const int t = s->jobs_turn;
  if (cudaEventQuery(s->jobs_ev[t]) == cudaErrorNotReady) return false;
  cudaGetLastError();
  s->jobs_turn ^= 1;
  const qaa::LaunchCtx lc{s->batch_stream, s->num_sms};
  size_t smem = 0;
  int nj = 0;
  cudaError_t e = cudaSuccess;
  for (Req* r : small) {
    e = upload_tables(s, r, s->batch_stream);
    const double dt = r->T / static_cast<double>(r->K);
    float2* ptab = r->d_tab;
    float2* btab = r->d_tab + static_cast<size_t>(r->K + 1) * (r->m + 1);
    if (e == cudaSuccess) e = qaa::launch_tables(lc, ptab, btab, r->n, r->m, dt, nullptr, r->K, 0, r->K, 0, r->K);
    if (e != cudaSuccess) break;
    qaa::OnchipJob& j = s->h_jobs[t][nj++];
    j.psi = r->psi;
    j.cl = r->d_mv;
    j.ptab = ptab;
    j.btab = btab;
    j.n = r->n;
    j.m = r->m;
    j.nsteps = static_cast<int>(r->K);
    j.first_p = 1;
    j.init = 1;
    j.init_val = static_cast<float>(std::exp2(-0.5 * r->n));
    j.stamp = stamp_start(r);  // batched requests: the device interval starts with their CTA
    smem = std::max(smem, qaa::onchip_smem_bytes(r->n, r->m));
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_jobs[t], s->h_jobs[t], sizeof(qaa::OnchipJob) * nj, cudaMemcpyHostToDevice,
                        s->batch_stream);
  if (e == cudaSuccess) e = qaa::launch_onchip_batch(lc, s->d_jobs[t], nj, smem);
  if (e == cudaSuccess) e = cudaEventRecord(s->jobs_ev[t], s->batch_stream);
  for (Req* r : small) {
    if (e == cudaSuccess) e = observe_async(s, r, s->batch_stream);
    if (e != cudaSuccess) r->status = QAA_E_CUDA;
    r->phase = kRunning;
    s->running.push_back(r);
  }
  if (e != cudaSuccess) cudaGetLastError();
  std::lock_guard<std::mutex> lk(s->mu);
  s->batches += 1;
  s->batched += static_cast<long long>(small.size());
  return true;
}

void worker_main(qaa_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait_for(lk, std::chrono::microseconds(100), [&] { return s->stop || !s->incoming.empty(); });
      while (!s->incoming.empty()) {
        s->waiting.push_back(s->incoming.front());
        s->incoming.pop_front();
      }
      if (s->stop && s->waiting.empty() && s->running.empty() && s->small_pending.empty()) {
        std::lock_guard<std::mutex> ilk(s->imu);
        if (s->issue_q.empty() && s->issued.empty()) break;
      }
    }
    if (const int d = s->inject_delay_ms.exchange(0)) std::this_thread::sleep_for(std::chrono::milliseconds(d));

    // admission, in arrival order; a request that does not fit yet does not
    // hold back smaller ones behind it
    std::vector<Req*> still;
    std::vector<Req*>& small = s->small_pending;
    for (Req* r : s->waiting) {
      bool cancelled, stopping;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        cancelled = r->cancel;
        stopping = s->stop;
      }
      if (cancelled || stopping) {
        std::lock_guard<std::mutex> lk(s->mu);
        finish(s, r, QAA_E_STATE);
        continue;
      }
      if (!place(s, r)) {
        still.push_back(r);
        continue;
      }
      {
        std::lock_guard<std::mutex> lk(s->mu);
        r->t_admit = steady_now() - s->t0;
        r->phase = kAdmitted;
        s->peak_used = std::max<long long>(s->peak_used, static_cast<long long>(s->arena.used()));
      }
      if (s->inject_fail.exchange(0)) {
        std::lock_guard<std::mutex> lk(s->mu);
        release(s, r);
        finish(s, r, QAA_E_CUDA);  // injected host-side failure of this request only
        continue;
      }
      if (r->small()) {
        small.push_back(r);
      } else if (r->persistent()) {
        cudaStream_t st = s->persist_streams[s->persist_turn];
        s->persist_turn = (s->persist_turn + 1) % static_cast<int>(s->persist_streams.size());
        if (issue_persistent(s, r, st) != cudaSuccess) {
          cudaStreamSynchronize(st);
          cudaGetLastError();
          r->status = QAA_E_CUDA;
        }
        r->phase = kRunning;
        s->running.push_back(r);
        std::lock_guard<std::mutex> lk(s->mu);
        s->streamed += 1;
      } else {
        {
          std::lock_guard<std::mutex> lk(s->imu);
          s->issue_q.push_back(r);
        }
        s->icv.notify_one();
        std::lock_guard<std::mutex> lk(s->mu);
        s->streamed += 1;
      }
    }
    s->waiting.swap(still);
    if (launch_batch(s, small)) small.clear();
    {
      std::lock_guard<std::mutex> lk(s->imu);
      for (Req* r : s->issued) {
        r->phase = kRunning;
        s->running.push_back(r);
      }
      s->issued.clear();
    }
    // completions
    std::vector<Req*> keep;
    for (Req* r : s->running) {
      bool done = r->status != QAA_PENDING;
      if (!done && r->done_ev) {
        const cudaError_t q = cudaEventQuery(r->done_ev);
        if (q == cudaErrorNotReady) {
          keep.push_back(r);
          continue;
        }
        if (q != cudaSuccess) {
          cudaGetLastError();
          r->status = QAA_E_CUDA;
        }
      }
      std::lock_guard<std::mutex> lk(s->mu);
      if (r->status == QAA_PENDING) {
        unsigned long long a = 0, b = 0;
        std::memcpy(&a, s->h_res + 8 * r->slot + 6, sizeof(a));
        std::memcpy(&b, s->h_res + 8 * r->slot + 7, sizeof(b));
        if (a >= s->ref_ns && b >= a) {
          r->t_dev_start = 1e-9 * static_cast<double>(a - s->ref_ns);
          r->t_dev_end = 1e-9 * static_cast<double>(b - s->ref_ns);
        }
        std::memcpy(r->res, s->h_res + 8 * r->slot, 5 * sizeof(double));
        int err = 0;
        std::memcpy(&err, s->h_res + 8 * r->slot + 5, sizeof(int));
        finish(s, r, err ? QAA_E_TIMEOUT : QAA_OK);
      } else {
        finish(s, r, r->status);
      }
      release(s, r);
    }
    s->running.swap(keep);
  }
}

}  // namespace

extern "C" {

qaa_status qaa_server_create(size_t hbm_budget_bytes, int max_slots, qaa_server** out) {
  if (!out) return sfail(QAA_E_ARG, "out is null");
  *out = nullptr;
  if (max_slots < 1 || max_slots > 65536) return sfail(QAA_E_ARG, "max_slots out of range [1, 65536]");
  qaa_server* s = new (std::nothrow) qaa_server;
  if (!s) return sfail(QAA_E_NOMEM, "host allocation failed");
  auto bail = [&](int code, const std::string& msg) {
    if (s->arena_base) cudaFree(s->arena_base);
    if (s->h_res) cudaFreeHost(s->h_res);
    if (s->h_stage) cudaFreeHost(s->h_stage);
    for (int t = 0; t < 2; ++t) {
      if (s->h_jobs[t]) cudaFreeHost(s->h_jobs[t]);
      if (s->d_jobs[t]) cudaFree(s->d_jobs[t]);
      if (s->jobs_ev[t]) cudaEventDestroy(s->jobs_ev[t]);
    }
    if (s->batch_stream) cudaStreamDestroy(s->batch_stream);
    for (cudaStream_t st : s->issue_streams) cudaStreamDestroy(st);
    for (cudaStream_t st : s->persist_streams) cudaStreamDestroy(st);
    cudaGetLastError();
    delete s;
    return sfail(code, msg);
  };
  if (cudaGetDevice(&s->device) != cudaSuccess) return bail(QAA_E_CUDA, "no CUDA device");
  if (cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess)
    return bail(QAA_E_CUDA, "cannot query SM count");
  size_t budget = hbm_budget_bytes;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return bail(QAA_E_CUDA, "cannot query free memory");
    const size_t reserve = static_cast<size_t>(4) << 30;
    budget = fr > 2 * reserve ? std::min(fr - reserve, static_cast<size_t>(64) << 30) : fr / 2;
  }
  budget = align_up(budget);
  if (cudaMalloc(&s->arena_base, budget) != cudaSuccess) return bail(QAA_E_NOMEM, "cannot reserve the arena");
  s->arena.reset(budget);
  s->max_slots = max_slots;
  // Tuning overrides: QAA_PERSIST_MAX_BITS (0 turns persistent launches off),
  // QAA_PERSIST_GRID (CTAs per persistent request).
  // Default: persistent launches up to n = 17.  Measured on the n ~ U{10..22}
  // mix: n = 16 requests alone 2.0x and n = 18 1.24x faster than streamed, but
  // n = 20 and 22 slower (0.70x, 0.59x: a few SMs cannot pull a whole state's
  // bandwidth); whole mix 218.7 solves/s (n <= 17) vs 199.4 (streamed only).
  s->persist_max_bits = 17;
  if (const char* v = std::getenv("QAA_PERSIST_MAX_BITS")) s->persist_max_bits = std::min(std::atoi(v), qaa::kPersistMaxBits);
  if (const char* v = std::getenv("QAA_PERSIST_GRID")) s->persist_grid = std::max(1, std::atoi(v));
  if (const char* v = std::getenv("QAA_SERVER_GRAPHS")) s->use_graphs = std::atoi(v) != 0;
  if (const char* v = std::getenv("QAA_SERVER_GRAPH_BITS")) s->graph_max_bits = std::atoi(v);
  if (cudaMallocHost(&s->h_res, sizeof(double) * 8 * max_slots) != cudaSuccess ||
      cudaMallocHost(&s->h_stage, kStageBytes * static_cast<size_t>(max_slots)) != cudaSuccess)
    return bail(QAA_E_NOMEM, "cannot allocate result slots");
  for (int i = max_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
  for (int t = 0; t < 2; ++t) {
    if (cudaMallocHost(&s->h_jobs[t], sizeof(qaa::OnchipJob) * max_slots) != cudaSuccess ||
        cudaMalloc(&s->d_jobs[t], sizeof(qaa::OnchipJob) * max_slots) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->jobs_ev[t], cudaEventDisableTiming) != cudaSuccess)
      return bail(QAA_E_NOMEM, "cannot allocate batch staging");
  }
  // Batches of small requests get the higher stream priority: their CTAs each
  // need a large share of an SM's shared memory and would otherwise wait for
  // the streaming passes (which keep every SM busy) to drain.
  int lo_pri = 0, hi_pri = 0;
  cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri);
  if (cudaStreamCreateWithPriority(&s->batch_stream, cudaStreamNonBlocking, hi_pri) != cudaSuccess)
    return bail(QAA_E_CUDA, "cannot create streams");
  int nissuers = 4;  // QAA_SERVER_ISSUERS overrides (1..32)
  if (const char* v = std::getenv("QAA_SERVER_ISSUERS")) nissuers = std::min(32, std::max(1, std::atoi(v)));
  for (int i = 0; i < nissuers; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, lo_pri) != cudaSuccess)
      return bail(QAA_E_CUDA, "cannot create streams");
    s->issue_streams.push_back(st);
  }
  for (int i = 0; i < 8; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, lo_pri) != cudaSuccess)
      return bail(QAA_E_CUDA, "cannot create streams");
    s->persist_streams.push_back(st);
  }
  // the device clock's origin for the requests' device intervals, taken
  // before any request is issued (in the arena's first bytes, which no
  // request holds yet)
  {
    unsigned long long* d_ref = reinterpret_cast<unsigned long long*>(s->arena_base);
    if (qaa::launch_stamp(qaa::LaunchCtx{s->batch_stream, s->num_sms}, d_ref) != cudaSuccess ||
        cudaMemcpyAsync(&s->ref_ns, d_ref, sizeof(s->ref_ns), cudaMemcpyDeviceToHost, s->batch_stream) != cudaSuccess ||
        cudaStreamSynchronize(s->batch_stream) != cudaSuccess)
      return bail(QAA_E_CUDA, "cannot read the device clock");
  }
  s->t0 = steady_now();
  for (int i = 0; i < nissuers; ++i) s->issuers.emplace_back(issuer_main, s, i);
  s->worker = std::thread(worker_main, s);
  *out = s;
  return QAA_OK;
}

qaa_status qaa_submit(qaa_server* s, int n, const int32_t* clauses, int m, double T, int64_t steps, uint64_t* ticket) {
  if (!s || !ticket) return sfail(QAA_E_ARG, "null server or ticket");
  if (n < 1 || n > QAA_MAX_QUBITS) return sfail(QAA_E_ARG, "n out of range [1, 34]");
  if (m < 0 || m > QAA_MAX_CLAUSES) return sfail(QAA_E_ARG, "m out of range [0, 1023]");
  if (m > 0 && !clauses) return sfail(QAA_E_ARG, "clauses is null");
  if (!(T >= 0.0) || !std::isfinite(T) || steps < 1 || steps > (1ll << 30))
    return sfail(QAA_E_ARG, "need finite T >= 0 and 1 <= steps <= 2^30");
  Req* r = new (std::nothrow) Req;
  if (!r) return sfail(QAA_E_NOMEM, "host allocation failed");
  r->n = n;
  r->m = m;
  r->T = T;
  r->K = steps;
  std::string err;
  const int st = qaa::encode_clauses(n, clauses, m, r->mv, r->lp, err);
  if (st) {
    delete r;
    return sfail(st, err);
  }
  qaa::make_plan(n, r->plan);
  // Persistent launches keep the phase tables of the whole run resident, so
  // they take runs of at most kPersistMaxSteps steps.
  r->persist = !r->plan.onchip && n <= s->persist_max_bits && steps <= kPersistMaxSteps;
  if (r->persist) {
    qaa::make_plan(n, r->plan, 10);  // the persistent kernel's tiles hold at most 10 bits
    qaa::narrow_low_pass(r->plan, 10);
  }
  r->graph = !r->plan.onchip && !r->persist && (s->use_graphs || n <= s->graph_max_bits);
  // Streamed requests store the per-tile clause counts once (at most 1.25
  // bytes per amplitude) so the merged low passes read them instead of
  // counting each step.
  {
    const char* env = std::getenv("QAA_LP_COUNTS");
    if (!r->plan.onchip && !r->persist && r->plan.use_tma && n > qaa::kOnchipMaxBits && !(env && std::atoi(env) == 0))
      r->counts_bytes = qaa::lp_counts_bytes(n);
  }
  if (r->plan.onchip && qaa::onchip_smem_bytes(n, m) > 227u * 1024u) {
    delete r;
    return sfail(QAA_E_ARG, "instance too large for the on-chip evolver");
  }
  const size_t need =
      request_bytes(n, m, table_bytes(n, m, steps, r->plan.onchip || r->persist, r->graph), r->counts_bytes,
                    s->num_sms);
  if (need > s->arena.size()) {
    delete r;
    return sfail(QAA_E_NOMEM, "request needs " + std::to_string(need) + " device bytes, more than the server's " +
                                  std::to_string(s->arena.size()));
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete r;
      return sfail(QAA_E_STATE, "server is shutting down");
    }
    r->ticket = s->next_ticket++;
    r->t_submit = steady_now() - s->t0;
    s->all[r->ticket] = r;
    s->incoming.push_back(r);
    *ticket = r->ticket;
  }
  s->cv.notify_all();
  return QAA_OK;
}

qaa_status qaa_poll(qaa_server* s, uint64_t ticket, qaa_result* out) {
  if (!s || !out) return sfail(QAA_E_ARG, "null server or result");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return sfail(QAA_E_ARG, "unknown ticket");
  const Req* r = it->second;
  if (r->phase != kDone) return QAA_PENDING;
  out->success_prob = r->res[2];
  out->energy = r->res[1];
  out->norm = r->res[0];
  out->expect_hb = 0.5 * r->n * r->res[0] - r->res[4];
  out->ground_count = static_cast<int64_t>(std::llround(r->res[3]));
  out->t_submit = r->t_submit;
  out->t_admit = r->t_admit;
  out->t_done = r->t_done;
  out->t_dev_start = r->t_dev_start;
  out->t_dev_end = r->t_dev_end;
  out->n = r->n;
  out->steps = r->K;
  out->status = r->status;
  return QAA_OK;
}

qaa_status qaa_cancel(qaa_server* s, uint64_t ticket) {
  if (!s) return sfail(QAA_E_ARG, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return sfail(QAA_E_ARG, "unknown ticket");
  Req* r = it->second;
  if (r->phase != kQueued) return sfail(QAA_E_STATE, "request already admitted");
  r->cancel = true;
  return QAA_OK;
}

qaa_status qaa_server_stats(qaa_server* s, qaa_server_info* out) {
  if (!s || !out) return sfail(QAA_E_ARG, "null server or info");
  std::lock_guard<std::mutex> lk(s->mu);
  out->arena_bytes = s->arena.size();
  out->peak_used_bytes = static_cast<size_t>(s->peak_used);
  out->batches = s->batches;
  out->batched_requests = s->batched;
  out->streamed_requests = s->streamed;
  return QAA_OK;
}

qaa_status qaa_server_inject(qaa_server* s, int fault, int param) {
  if (!s) return sfail(QAA_E_ARG, "null server");
  if (fault == 1) {
    s->inject_delay_ms = std::max(param, 0);
  } else if (fault == 2) {
    s->inject_fail = 1;
  } else if (fault == 3) {
    s->inject_stuck_barrier = 1;
  } else {
    return sfail(QAA_E_ARG,
                 "unknown fault (1 = delay the worker, 2 = fail the next admission, 3 = stuck grid barrier)");
  }
  s->cv.notify_all();
  return QAA_OK;
}

qaa_status qaa_server_destroy(qaa_server* s) {
  if (!s) return QAA_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  {
    std::lock_guard<std::mutex> lk(s->imu);
    s->issue_stop = true;
  }
  s->icv.notify_all();
  for (auto& t : s->issuers) t.join();
  cudaSetDevice(s->device);
  for (cudaStream_t st : s->issue_streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (cudaStream_t st : s->persist_streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaStreamSynchronize(s->batch_stream);
  cudaStreamDestroy(s->batch_stream);
  for (int t = 0; t < 2; ++t) {
    cudaFreeHost(s->h_jobs[t]);
    cudaFree(s->d_jobs[t]);
    cudaEventDestroy(s->jobs_ev[t]);
  }
  cudaFree(s->arena_base);
  cudaFreeHost(s->h_res);
  cudaFreeHost(s->h_stage);
  for (auto& kv : s->all) {
    if (kv.second->done_ev) cudaEventDestroy(kv.second->done_ev);
    if (kv.second->gexec) cudaGraphExecDestroy(kv.second->gexec);
    delete kv.second;
  }
  delete s;
  return QAA_OK;
}

}  // extern "C"
