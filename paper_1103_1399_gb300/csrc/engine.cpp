// Handle API of include/qaa.h: device buffers of one instance, phase-table
// scheduling in chunks of steps, kernel launch order (the pass plan comes from
// plan.cpp), observables and launch profiling.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "engine_internal.h"
#include "qaa.h"
#include "qaa_internal.cuh"

namespace {

thread_local std::string g_last_error = "no error";

qaa_status fail(int code, const std::string& msg) {
  g_last_error = msg;
  return static_cast<qaa_status>(code);
}

#define QAA_CK(expr)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(QAA_E_CUDA, std::string(#expr) + " failed: " + cudaGetErrorString(e_)); \
  } while (0)

using qaa::kChunkSteps;

}  // namespace

struct qaa_ctx {
  int n = 0, m = 0, device = 0, num_sms = 0;
  cudaStream_t stream = nullptr;
  std::vector<qaa::ClauseMV> mv;
  std::vector<qaa::ClauseLP> lp;
  qaa::ClauseMV* d_mv = nullptr;
  qaa::ClauseLP* d_lp = nullptr;
  float2* d_tab = nullptr;
  size_t tab_cap = 0;  // float2 entries
  double* d_s = nullptr;
  size_t s_cap = 0;
  double* d_part = nullptr;
  size_t part_cap = 0;
  double* d_res = nullptr;
  double* h_res = nullptr;  // pinned
  int* d_err = nullptr;     // set by kernels whose bounded waits expired
  double* d_fold = nullptr; // norm-fold slots of the low passes (kFoldBytes)
  qaa::PassPlan plan;
  // launch graphs (QAA_LAUNCH_GRAPH): the last built graph and what it was built for
  int launch_mode = QAA_LAUNCH_PASSES;
  void* d_gscratch = nullptr;
  cudaGraphExec_t gexec = nullptr;
  struct GraphKey {
    const void* psi;
    double dt;
    const double* s_dev;
    const double* dt_dev;
    long long K, k0, k1;
    int wht_kind;
    cudaStream_t stream;
    bool operator==(const GraphKey& o) const {
      return psi == o.psi && std::memcmp(&dt, &o.dt, sizeof dt) == 0 && s_dev == o.s_dev && dt_dev == o.dt_dev &&
             K == o.K && k0 == o.k0 &&
             k1 == o.k1 && wht_kind == o.wht_kind && stream == o.stream;
    }
  } gkey{};
  // stored per-tile clause counts for the merged low passes: 0 = not yet
  // computed, 1 = valid, -1 = not used (no TMA passes, no memory, or
  // QAA_LP_COUNTS=0)
  unsigned* d_counts = nullptr;
  int counts_state = 0;
  // Lanczos workspace (qaa_lowest_eigenvalues), allocated on first use
  void* d_lz = nullptr;
  size_t lz_bytes = 0;
  // launch profiling
  bool prof = false;
  std::vector<cudaEvent_t> ev_free;
  struct Pending {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  long long prof_n[QAA_K_COUNT] = {};
  double prof_ms[QAA_K_COUNT] = {};
};

namespace {

qaa::LaunchCtx lctx(const qaa_ctx* h) { return {h->stream, h->num_sms}; }

cudaEvent_t take_event(qaa_ctx* h) {
  if (!h->ev_free.empty()) {
    cudaEvent_t e = h->ev_free.back();
    h->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Run `launch` (returns cudaError_t), bracketed by events when profiling.
template <class F>
cudaError_t timed(qaa_ctx* h, int kind, F&& launch) {
  if (!h->prof) return launch();
  cudaEvent_t a = take_event(h), b = take_event(h);
  if (a) cudaEventRecord(a, h->stream);
  const cudaError_t err = launch();
  if (b) cudaEventRecord(b, h->stream);
  if (a && b) {
    h->pending.push_back({kind, a, b});
  } else {
    if (a) h->ev_free.push_back(a);
    if (b) h->ev_free.push_back(b);
  }
  return err;
}

qaa_status fold_profile(qaa_ctx* h) {
  if (h->pending.empty()) return QAA_OK;
  QAA_CK(cudaStreamSynchronize(h->stream));
  for (const auto& p : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      h->prof_n[p.kind] += 1;
      h->prof_ms[p.kind] += ms;
    } else {
      cudaGetLastError();
    }
    h->ev_free.push_back(p.a);
    h->ev_free.push_back(p.b);
  }
  h->pending.clear();
  return QAA_OK;
}

qaa_status ensure_tab(qaa_ctx* h, size_t entries) {
  if (entries <= h->tab_cap) return QAA_OK;
  if (h->d_tab) {
    QAA_CK(cudaStreamSynchronize(h->stream));
    QAA_CK(cudaFree(h->d_tab));
    h->d_tab = nullptr;
    h->tab_cap = 0;
  }
  if (cudaMalloc(&h->d_tab, entries * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    return fail(QAA_E_NOMEM, "cannot allocate phase tables");
  }
  h->tab_cap = entries;
  return QAA_OK;
}

qaa_status check_handle(qaa_ctx* h) {
  if (!h) return fail(QAA_E_ARG, "null handle");
  QAA_CK(cudaSetDevice(h->device));
  return QAA_OK;
}

// After a stream synchronisation: report (and clear) an expired device wait.
qaa_status check_device_error(qaa_ctx* h) {
  int e = 0;
  QAA_CK(cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != 0) {
    QAA_CK(cudaMemset(h->d_err, 0, sizeof(int)));
    return fail(QAA_E_TIMEOUT, "a bounded wait on a TMA copy expired in a streaming pass");
  }
  return QAA_OK;
}

// Profiler kind of a pass: the rotation form's passes count as the low-pass
// and strided kinds they replace.
int prof_kind(int pass_kind) {
  switch (pass_kind) {
    case qaa::kLpPhase: return QAA_K_LOW_FIRST;
    case qaa::kLpRot: return QAA_K_LOW_MERGE;
    case qaa::kLpRot12: return QAA_K_LOW_MERGE;
    case qaa::kSpRot: return QAA_K_STRIDED;
    default: return pass_kind;
  }
}

// The stored per-tile clause counts, computed on the handle's stream the first
// time a streaming evolution needs them; null when they are not used.
const unsigned* stored_counts(qaa_ctx* h) {
  if (h->counts_state == 0) {
    const char* env = std::getenv("QAA_LP_COUNTS");
    // the tensor-core variant's low passes read the stored counts whatever QAA_LP_COUNTS says
    const bool tc = h->plan.wht_kind == 1 || h->plan.wht_kind == 2;
    const bool want = h->n > qaa::kOnchipMaxBits && (tc || (h->plan.use_tma && !(env && std::atoi(env) == 0)));
    h->counts_state = -1;
    if (want && cudaMalloc(&h->d_counts, qaa::lp_counts_bytes(h->n)) == cudaSuccess) {
      if (qaa::launch_lp_counts(lctx(h), h->d_counts, h->n, h->m, h->d_lp) == cudaSuccess) {
        h->counts_state = 1;
      } else {
        cudaGetLastError();
        cudaFree(h->d_counts);
        h->d_counts = nullptr;
      }
    } else {
      cudaGetLastError();
    }
  }
  return h->counts_state == 1 ? h->d_counts : nullptr;
}

// Streaming plan, launch-graph mode: build (or reuse) the graph of the whole
// range and launch it.  The graph is rebuilt when psi, the schedule, the range,
// the variant or the stream changes.
qaa_status evolve_graph(qaa_ctx* h, float2* psi, double dt, long long K, long long k0, long long k1, const double* s_dev,
                 const double* dt_dev) {
  if (!h->d_gscratch) {
    if (cudaMalloc(&h->d_gscratch, qaa::graph_scratch_bytes(h->n, h->m)) != cudaSuccess) {
      cudaGetLastError();
      return fail(QAA_E_NOMEM, "cannot allocate graph scratch");
    }
  }
  const qaa_ctx::GraphKey key{psi, dt, s_dev, dt_dev, K, k0, k1, h->plan.wht_kind, h->stream};
  if (!h->gexec || !(key == h->gkey)) {
    if (h->gexec) {
      QAA_CK(cudaStreamSynchronize(h->stream));
      QAA_CK(cudaGraphExecDestroy(h->gexec));
      h->gexec = nullptr;
    }
    qaa::GraphSpec gs;
    gs.plan = &h->plan;
    gs.psi = psi;
    gs.m = h->m;
    gs.cl = h->d_lp;
    gs.err = h->d_err;
    gs.dt = dt;
    gs.s_dev = s_dev;
    gs.dt_dev = dt_dev;
    gs.counts = stored_counts(h);
    gs.fold = h->d_fold;
    gs.K = K;
    gs.k0 = k0;
    gs.k1 = k1;
    gs.num_sms = h->num_sms;
    qaa::graph_scratch_split(h->d_gscratch, h->m, gs);
    QAA_CK(qaa::build_evolve_graph(gs, &h->gexec));
    h->gkey = key;
  }
  QAA_CK(timed(h, QAA_K_GRAPH, [&] { return cudaGraphLaunch(h->gexec, h->stream); }));
  return QAA_OK;
}

// s_host / dt_host (K entries each, optional): the caller's schedule and per-step
// lengths, copied to the device ahead of the launches on the handle's stream.
qaa_status evolve_impl(qaa_ctx* h, void* psi, double dt, long long K, long long k0, long long k1, const double* s_host,
                const double* dt_host = nullptr) {
  qaa_status st = check_handle(h);
  if (st) return st;
  if (!psi) return fail(QAA_E_ARG, "psi is null");
  if (reinterpret_cast<uintptr_t>(psi) % 16u) return fail(QAA_E_ARG, "psi must be 16-byte aligned");
  if (K < 1 || k0 < 0 || k1 < k0 || k1 > K) return fail(QAA_E_ARG, "bad step range");
  if (!std::isfinite(dt)) return fail(QAA_E_ARG, "dt must be finite");
  if (k0 == k1) return QAA_OK;
  const double* s_dev = nullptr;
  const double* dt_dev = nullptr;
  if (s_host || dt_host) {
    const size_t need = static_cast<size_t>(K) * 2;  // [0, K): s, [K, 2K): dt
    if (need > h->s_cap) {
      if (h->d_s) {
        QAA_CK(cudaStreamSynchronize(h->stream));
        QAA_CK(cudaFree(h->d_s));
        h->d_s = nullptr;
        h->s_cap = 0;
      }
      if (cudaMalloc(&h->d_s, need * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(QAA_E_NOMEM, "cannot allocate schedule");
      }
      h->s_cap = need;
    }
    if (s_host) {
      QAA_CK(cudaMemcpyAsync(h->d_s, s_host, K * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      s_dev = h->d_s;
    }
    if (dt_host) {
      QAA_CK(cudaMemcpyAsync(h->d_s + K, dt_host, K * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      dt_dev = h->d_s + K;
    }
  }
  if (h->launch_mode == QAA_LAUNCH_GRAPH && h->n > qaa::kOnchipMaxBits)
    return evolve_graph(h, static_cast<float2*>(psi), dt, K, k0, k1, s_dev, dt_dev);
  const long long chunk = std::min(kChunkSteps, k1 - k0);
  const size_t prow = static_cast<size_t>(h->m + 1), brow = static_cast<size_t>(h->n + 1);
  st = ensure_tab(h, static_cast<size_t>(chunk + 1) * prow + static_cast<size_t>(chunk) * brow);
  if (st) return st;
  float2* ptab = h->d_tab;
  float2* btab = h->d_tab + static_cast<size_t>(chunk + 1) * prow;
  const qaa::LaunchCtx lc = lctx(h);
  float2* p = static_cast<float2*>(psi);
  std::vector<qaa::Pass> passes;
  for (long long c0 = k0; c0 < k1; c0 += chunk) {
    const long long c1 = std::min(k1, c0 + chunk);
    QAA_CK(timed(h, QAA_K_TABLES, [&] {
      return qaa::launch_tables(lc, ptab, btab, h->n, h->m, dt, s_dev, K, k0, k1, c0, c1,
                                h->n > qaa::kOnchipMaxBits && h->plan.wht_kind == qaa::kRotationForm, dt_dev);
    }));
    if (h->n <= qaa::kOnchipMaxBits) {
      QAA_CK(timed(h, QAA_K_ONCHIP, [&] {
        return qaa::launch_onchip(lc, p, h->n, h->m, h->d_mv, ptab, btab, static_cast<int>(c1 - c0), c0 == k0);
      }));
    } else {
      qaa::build_passes(h->plan, k0, k1, c0, c1, passes);
      const unsigned* counts = stored_counts(h);
      for (const qaa::Pass& ps : passes)
        QAA_CK(timed(h, prof_kind(ps.kind), [&] {
          return qaa::launch_planned_pass(lc, h->plan, ps, p, h->m, h->d_lp, ptab, btab, h->d_err, counts,
                                          h->d_fold);
        }));
    }
  }
  return QAA_OK;
}

qaa_status observe(qaa_ctx* h, const void* psi, double out[5]) {
  qaa_status st = check_handle(h);
  if (st) return st;
  if (!psi) return fail(QAA_E_ARG, "psi is null");
  if (reinterpret_cast<uintptr_t>(psi) % 8u) return fail(QAA_E_ARG, "psi must be 8-byte aligned");
  const size_t need = qaa::obs_partials_len(h->n, h->num_sms);
  if (need > h->part_cap) {
    if (h->d_part) {
      QAA_CK(cudaStreamSynchronize(h->stream));
      QAA_CK(cudaFree(h->d_part));
      h->d_part = nullptr;
      h->part_cap = 0;
    }
    if (cudaMalloc(&h->d_part, need * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(QAA_E_NOMEM, "cannot allocate reduction partials");
    }
    h->part_cap = need;
  }
  QAA_CK(timed(h, QAA_K_OBSERVE, [&] {
    return qaa::launch_observables(lctx(h), static_cast<const float2*>(psi), h->n, h->m, h->d_lp, h->d_part, h->d_res,
                                   h->counts_state == 1 ? h->d_counts : nullptr, h->d_err);
  }));
  QAA_CK(cudaMemcpyAsync(h->h_res, h->d_res, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  QAA_CK(cudaStreamSynchronize(h->stream));
  std::memcpy(out, h->h_res, 5 * sizeof(double));
  return check_device_error(h);
}

}  // namespace

namespace qaa {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace qaa

extern "C" {

int qaa_version(void) { return 1; }

const char* qaa_last_error(void) { return g_last_error.c_str(); }

qaa_status qaa_create(int n, const int32_t* clauses, int m, qaa_handle* out) {
  if (!out) return fail(QAA_E_ARG, "out is null");
  *out = nullptr;
  if (n < 1 || n > QAA_MAX_QUBITS) return fail(QAA_E_ARG, "n out of range [1, 34]");
  if (m < 0 || m > QAA_MAX_CLAUSES) return fail(QAA_E_ARG, "m out of range [0, 1023]");
  if (m > 0 && !clauses) return fail(QAA_E_ARG, "clauses is null");
  qaa_ctx* h = new (std::nothrow) qaa_ctx;
  if (!h) return fail(QAA_E_NOMEM, "host allocation failed");
  h->n = n;
  h->m = m;
  {
    std::string err;
    const int st = qaa::encode_clauses(n, clauses, m, h->mv, h->lp, err);
    if (st) {
      delete h;
      return fail(st, err);
    }
  }
  auto cleanup = [&](int code, const std::string& msg) {
    qaa_destroy(h);
    return fail(code, msg);
  };
  if (cudaGetDevice(&h->device) != cudaSuccess) return cleanup(QAA_E_CUDA, "no CUDA device");
  if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
    return cleanup(QAA_E_CUDA, "cannot query SM count");
  const size_t mcap = static_cast<size_t>(std::max(m, 1));
  if (cudaMalloc(&h->d_mv, mcap * sizeof(qaa::ClauseMV)) != cudaSuccess ||
      cudaMalloc(&h->d_lp, mcap * sizeof(qaa::ClauseLP)) != cudaSuccess ||
      cudaMalloc(&h->d_res, 8 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->d_err, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->d_fold, qaa::kFoldBytes) != cudaSuccess ||
      cudaMallocHost(&h->h_res, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(QAA_E_NOMEM, "cannot allocate clause tables");
  }
  if (cudaMemset(h->d_err, 0, sizeof(int)) != cudaSuccess) return cleanup(QAA_E_CUDA, "cannot clear error word");
  qaa::make_plan(n, h->plan);
  if (m > 0) {
    if (cudaMemcpy(h->d_mv, h->mv.data(), m * sizeof(qaa::ClauseMV), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_lp, h->lp.data(), m * sizeof(qaa::ClauseLP), cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup(QAA_E_CUDA, "cannot upload clause tables");
  }
  *out = h;
  return QAA_OK;
}

qaa_status qaa_destroy(qaa_handle h) {
  if (!h) return QAA_OK;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  cudaFree(h->d_mv);
  cudaFree(h->d_lp);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  cudaFree(h->d_gscratch);
  cudaFree(h->d_lz);
  cudaFree(h->d_counts);
  cudaFree(h->d_tab);
  cudaFree(h->d_s);
  cudaFree(h->d_part);
  cudaFree(h->d_res);
  cudaFree(h->d_err);
  cudaFree(h->d_fold);
  if (h->h_res) cudaFreeHost(h->h_res);
  for (auto& p : h->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (cudaEvent_t e : h->ev_free) cudaEventDestroy(e);
  delete h;
  return QAA_OK;
}

qaa_status qaa_set_stream(qaa_handle h, void* cuda_stream) {
  if (!h) return fail(QAA_E_ARG, "null handle");
  const cudaStream_t next = static_cast<cudaStream_t>(cuda_stream);
  if (next != h->stream) {
    // the handle's tables, counts and scratch are reused by the next call: the
    // old stream's work on them must be done before another stream touches them
    qaa_status st = check_handle(h);
    if (st) return st;
    QAA_CK(cudaStreamSynchronize(h->stream));
  }
  h->stream = next;
  return QAA_OK;
}

qaa_status qaa_set_variant(qaa_handle h, int wht_kind, int q) {
  if (!h) return fail(QAA_E_ARG, "null handle");
  if (wht_kind < 0 || wht_kind > 3)
    return fail(QAA_E_ARG, "unknown wht_kind (0 = FP32, 1 = BF16x3, 2 = BF16x2, 3 = rotation form)");
  const int widest = (wht_kind == 1 || wht_kind == 2 || !h->plan.use_tma) ? 10 : 11;  // 11-bit tiles: TMA FP32 only
  if (q != 0 && (q < 5 || q > widest))
    return fail(QAA_E_ARG, "q (qubits per strided pass) must be 0 (automatic) or in [5, " + std::to_string(widest) +
                               "] for this variant");
  if (wht_kind == qaa::kRotationForm && h->n > qaa::kOnchipMaxBits && !h->plan.use_tma)
    return fail(QAA_E_ARG, "the rotation form needs the TMA passes (not available, or QAA_PASSES=classic)");
  // the low pass the plan will use: 12 bits only for the rotation form on TMA
  // passes with QAA_LOW_BITS=12 (and at least 5 bits above it)
  int low = qaa::kLowBits;
  if (wht_kind == qaa::kRotationForm && h->plan.use_tma) {
    const char* lb = std::getenv("QAA_LOW_BITS");
    if (lb && std::atoi(lb) == 12 && h->n - 12 >= 5) low = 12;
  }
  if (q != 0 && h->n > qaa::kOnchipMaxBits) {
    auto splits = [&](int L) {
      const int rest = h->n - L, ng = (rest + q - 1) / q;
      return 5 * ng <= rest;
    };
    // a 12-bit low pass that leaves no split into groups of 5..q bits falls back to 10 bits
    if (low == 12 && !splits(12)) low = qaa::kLowBits;
    if (!splits(low))
      return fail(QAA_E_ARG, "no split of the " + std::to_string(h->n - low) + " strided bits into groups of 5.." +
                                 std::to_string(q) + " bits");
  }
  if (q != 0)
    qaa::make_default_plan(h->n, h->plan, q, low);  // groups of at most q bits (the fewest such groups)
  else
    qaa::make_plan(h->n, h->plan, widest);
  // a plan made (or tuned) for the other form gets the run lengths of this one
  const bool same_form = (h->plan.wht_kind == qaa::kRotationForm) == (wht_kind == qaa::kRotationForm);
  h->plan.wht_kind = wht_kind;
  if (!same_form) qaa::set_default_run_c(h->plan);
  // the tensor-core passes need the stored counts: look again if they were turned off
  if ((wht_kind == 1 || wht_kind == 2) && h->counts_state == -1) h->counts_state = 0;
  // only the rotation form has a 12-bit low pass
  if (wht_kind != qaa::kRotationForm) qaa::narrow_low_pass(h->plan, q != 0 ? q : widest);
  return QAA_OK;
}

namespace {

// One timing of `plan` on the handle: init, `steps` Strang steps (dt = 0.1),
// the best of two runs, in ms per step; < 0 on a launch error.
// The candidate's own FP32 form (W.B.W or rotation) is timed; a handle on a
// tensor-core variant keeps that variant.
double time_plan(qaa_ctx* h, float2* psi, const qaa::PassPlan& plan, int steps, int tc_kind) {
  h->plan = plan;
  if (tc_kind) {
    h->plan.wht_kind = tc_kind;
    qaa::narrow_low_pass(h->plan, 10);
  }
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    return -1.0;
  }
  double best = -1.0;
  for (int rep = 0; rep < 3; ++rep) {
    if (qaa::launch_init_uniform(lctx(h), psi, h->n) != cudaSuccess) break;
    if (rep > 0) cudaEventRecord(a, h->stream);
    if (evolve_impl(h, psi, 0.1 * steps, steps, 0, steps, nullptr) != QAA_OK) break;
    if (rep > 0) {
      cudaEventRecord(b, h->stream);
      if (cudaEventSynchronize(b) != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      const double per = ms / steps;
      if (best < 0 || per < best) best = per;
    }
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess || check_device_error(h) != QAA_OK) best = -1.0;
  cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

}  // namespace

qaa_status qaa_autotune(qaa_handle h, void* psi, int steps, double budget_ms, char* report, size_t len) {
  qaa_status st = check_handle(h);
  if (st) return st;
  if (!psi) return fail(QAA_E_ARG, "psi is null");
  if (reinterpret_cast<uintptr_t>(psi) % 16u) return fail(QAA_E_ARG, "psi must be 16-byte aligned");
  if (steps < 1 || steps > 64) return fail(QAA_E_ARG, "steps must be in [1, 64]");
  std::string rep;
  auto finish = [&](int code) -> qaa_status {
    if (report && len > 0) {
      std::strncpy(report, rep.c_str(), len - 1);
      report[len - 1] = '\0';
    }
    return static_cast<qaa_status>(code);
  };
  if (h->n <= qaa::kOnchipMaxBits) {
    rep = "on-chip evolver: no pass plan to tune\n";
    return finish(QAA_OK);
  }
  if (!(budget_ms > 0)) budget_ms = 60000.0;
  const bool prof = h->prof;
  const int mode = h->launch_mode;
  h->prof = false;
  h->launch_mode = QAA_LAUNCH_PASSES;
  float2* p = static_cast<float2*>(psi);
  const auto t0 = std::chrono::steady_clock::now();
  auto spent = [&] {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  };
  const int tc_kind = (h->plan.wht_kind == 1 || h->plan.wht_kind == 2) ? h->plan.wht_kind : 0;
  qaa::PassPlan best;
  double best_ms = -1.0;
  auto consider = [&](const qaa::PassPlan& cand) {
    const double ms = time_plan(h, p, cand, steps, tc_kind);
    char line[64];
    std::snprintf(line, sizeof line, "%10.4f ms/step  ", ms);
    rep += std::string(line) + qaa::describe_plan(cand) + "\n";
    if (ms > 0 && (best_ms < 0 || ms < best_ms)) {
      best_ms = ms;
      best = cand;
    }
  };
  // stage 1: group widths and the phase group
  std::vector<qaa::PassPlan> cands;
  qaa::plan_candidates(h->n, cands);
  for (const auto& c : cands) {
    if (best_ms > 0 && spent() > budget_ms) break;
    consider(c);
  }
  if (best_ms < 0) {
    h->prof = prof;
    h->launch_mode = mode;
    qaa::make_plan(h->n, h->plan);
    return finish(fail(QAA_E_CUDA, "autotune: no candidate plan ran"));
  }
  // stage 2: run length of each group that has a choice (Q >= 7 on TMA passes)
  if (best.use_tma)
    for (size_t i = 0; i < best.strided.size() && spent() <= budget_ms; ++i) {
      if (best.strided[i].q < 7) continue;
      qaa::PassPlan c = best;
      c.run_c[i] = c.run_c[i] == 4 ? 0 : 4;
      consider(c);
    }
  // stage 3: two equal q-bit groups (q >= 10) recombined as {10..14, 15+q..} and {15..14+q}, or back
  if (best.use_tma && best.strided.size() == 2 && best.strided[0].q == best.strided[1].q && best.strided[0].q >= 10 &&
      spent() <= budget_ms) {
    qaa::PassPlan c = best;
    const int q = c.strided[0].q, L = c.low_bits;
    const bool split = c.strided[0].a2 != c.strided[0].a + 5;
    if (split) {
      c.strided[0] = {L, q, L + 5};
      c.strided[1] = {L + q, q, L + q + 5};
    } else {
      c.strided[0] = {L, q, L + q + 5};
      c.strided[1] = {L + 5, q, L + 10};
    }
    consider(c);
  }
  // stage 4: plain loads instead of TMA (groups of at most 10 bits, contiguous)
  bool narrow = true;
  for (const auto& g : best.strided) narrow = narrow && g.q <= 10;
  if (best.use_tma && narrow && best.low_bits == qaa::kLowBits && spent() <= budget_ms) {
    qaa::PassPlan c = best;
    c.use_tma = false;
    c.wht_kind = 0;  // plain loads: the W.B.W form only
    if (c.strided.size() == 2 && c.strided[0].a2 != c.strided[0].a + 5) {
      const int q = c.strided[0].q;
      c.strided[0] = {qaa::kLowBits, q, qaa::kLowBits + 5};
      c.strided[1] = {qaa::kLowBits + q, q, qaa::kLowBits + q + 5};
    }
    consider(c);
  }
  // stage 5: the rotation form of the H_B factor on the best plan (same step,
  // g instead of 2g - 2 round trips; FP32 CUDA-core passes only)
  if (!tc_kind && best.use_tma && spent() <= budget_ms) {
    qaa::PassPlan c = best;
    c.wht_kind = qaa::kRotationForm;
    consider(c);
    // its passes carry more arithmetic than a plain W pass, so the run lengths
    // that suit it can differ: toggle them again if it won
    if (best.wht_kind == qaa::kRotationForm)
      for (size_t i = 0; i < best.strided.size() && spent() <= budget_ms; ++i) {
        if (best.strided[i].q < 7) continue;
        qaa::PassPlan t = best;
        t.run_c[i] = t.run_c[i] == 4 ? 0 : 4;
        consider(t);
      }
  }
  h->plan = best;
  if (tc_kind) {
    h->plan.wht_kind = tc_kind;
    qaa::narrow_low_pass(h->plan, 10);
  }
  qaa::PassPlan rec = best;
  qaa::set_tuned_plan(rec);
  h->prof = prof;
  h->launch_mode = mode;
  char line[96];
  std::snprintf(line, sizeof line, "chosen (%.4f ms/step, %.0f ms spent): ", best_ms, spent());
  rep += std::string(line) + qaa::describe_plan(best) + "\n";
  return finish(QAA_OK);
}

int qaa_tune_candidates(int n, char* buf, size_t len) {
  if (n < 1 || n > QAA_MAX_QUBITS) return fail(QAA_E_ARG, "n out of range [1, 34]");
  std::vector<qaa::PassPlan> cands;
  qaa::plan_candidates(n, cands);
  std::string d;
  for (const auto& c : cands) d += qaa::describe_plan(c) + "\n";
  if (buf && len > 0) {
    std::strncpy(buf, d.c_str(), len - 1);
    buf[len - 1] = '\0';
  }
  return static_cast<int>(cands.size());
}

qaa_status qaa_forget_tuned_plans(void) {
  qaa::clear_tuned_plans();
  return QAA_OK;
}

namespace {

// Number of eigenvalues below x of the symmetric tridiagonal matrix with
// diagonal a[0..m) and off-diagonal b[1..m) (Sturm sequence of the LDL^T
// pivots).
int sturm_count(const std::vector<double>& a, const std::vector<double>& b, int first, int m, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = first; i < m; ++i) {
    const double off = i > first ? b[i] * b[i] : 0.0;
    q = a[i] - x - (i > first ? off / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// All eigenvalues (ascending) of the tridiagonal matrix rows [first, m) by bisection.
std::vector<double> tridiag_eigs(const std::vector<double>& a, const std::vector<double>& b, int first, int m) {
  double lo = 0.0, hi = 0.0;
  for (int i = first; i < m; ++i) {
    const double r = (i > first ? std::fabs(b[i]) : 0.0) + (i + 1 < m ? std::fabs(b[i + 1]) : 0.0);
    lo = i == first ? a[i] - r : std::min(lo, a[i] - r);
    hi = i == first ? a[i] + r : std::max(hi, a[i] + r);
  }
  const double span = std::max(1.0, hi - lo);
  std::vector<double> ev;
  for (int k = 0; k < m - first; ++k) {
    double l = lo - 1e-12 * span, r = hi + 1e-12 * span;
    for (int it = 0; it < 200 && r - l > 1e-15 * span; ++it) {
      const double mid = 0.5 * (l + r);
      if (sturm_count(a, b, first, m, mid) > k) r = mid; else l = mid;
    }
    ev.push_back(0.5 * (l + r));
  }
  return ev;
}

}  // namespace

qaa_status qaa_lowest_eigenvalues(qaa_handle h, double s, int k, int max_iter, int start, uint64_t seed, double* evals,
                           int* found, int* iters) {
  qaa_status st = check_handle(h);
  if (st) return st;
  if (!evals || !found) return fail(QAA_E_ARG, "evals or found is null");
  if (k < 1 || k > 8) return fail(QAA_E_ARG, "k must be in [1, 8]");
  if (max_iter < 2 || max_iter > 4000) return fail(QAA_E_ARG, "max_iter must be in [2, 4000]");
  if (start != 0 && start != 1) return fail(QAA_E_ARG, "start must be 0 (uniform) or 1 (random)");
  if (!std::isfinite(s)) return fail(QAA_E_ARG, "s must be finite");
  const size_t N = size_t{1} << h->n;
  const int P = qaa::lanczos_partials(h->num_sms);
  const size_t vec = N * sizeof(double);
  const size_t need = 3 * vec + ((N * sizeof(uint16_t) + 255) & ~size_t{255}) + sizeof(double) * (P + 2 * max_iter + 2);
  if (need > h->lz_bytes) {
    if (h->d_lz) {
      QAA_CK(cudaStreamSynchronize(h->stream));
      QAA_CK(cudaFree(h->d_lz));
      h->d_lz = nullptr;
      h->lz_bytes = 0;
    }
    if (cudaMalloc(&h->d_lz, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(QAA_E_NOMEM, "cannot allocate the Lanczos workspace (3 state vectors)");
    }
    h->lz_bytes = need;
  }
  char* base = static_cast<char*>(h->d_lz);
  qaa::LanczosArgs a;
  a.n = h->n;
  a.s = s;
  a.iters = max_iter;
  a.random_start = start;
  a.seed = seed;
  a.v = reinterpret_cast<double*>(base);
  a.vp = reinterpret_cast<double*>(base + vec);
  a.w = reinterpret_cast<double*>(base + 2 * vec);
  uint16_t* E = reinterpret_cast<uint16_t*>(base + 3 * vec);
  a.E = E;
  double* dbl = reinterpret_cast<double*>(base + 3 * vec + ((N * sizeof(uint16_t) + 255) & ~size_t{255}));
  a.partials = dbl;
  a.alpha = dbl + P;
  a.beta = dbl + P + max_iter;
  const qaa::LaunchCtx lc = lctx(h);
  QAA_CK(qaa::launch_hp_diag(lc, E, h->n, h->m, h->d_lp));
  int done = 0;
  QAA_CK(qaa::launch_lanczos(lc, a, &done));
  std::vector<double> alpha(static_cast<size_t>(max_iter)), beta(static_cast<size_t>(max_iter) + 1);
  QAA_CK(cudaMemcpyAsync(alpha.data(), a.alpha, sizeof(double) * max_iter, cudaMemcpyDeviceToHost, h->stream));
  QAA_CK(cudaMemcpyAsync(beta.data(), a.beta, sizeof(double) * (max_iter + 1), cudaMemcpyDeviceToHost, h->stream));
  QAA_CK(cudaStreamSynchronize(h->stream));
  // Krylov space exhausted: stop at the first vanishing beta
  double scale = 1.0;
  for (int j = 0; j < max_iter; ++j) scale = std::max(scale, std::fabs(alpha[j]));
  int m = max_iter;
  for (int j = 0; j < max_iter; ++j)
    if (!(beta[j + 1] > 1e-10 * scale)) {
      m = j + 1;
      break;
    }
  if (iters) *iters = m;
  // Ritz values, then the Cullum-Willoughby test: in finite precision the
  // Lanczos matrix T_m repeats converged eigenvalues and also has spurious
  // ones; a simple eigenvalue of T_m that is also an eigenvalue of T_m without
  // its first row and column is spurious, and repeated ones count once.
  const std::vector<double> ev = tridiag_eigs(alpha, beta, 0, m);
  const std::vector<double> evh = m > 1 ? tridiag_eigs(alpha, beta, 1, m) : std::vector<double>();
  double tnorm = 1.0;
  for (double x : ev) tnorm = std::max(tnorm, std::fabs(x));
  const double tol = 1e-9 * tnorm;  // FP64 vectors: converged copies agree far below this
  int nf = 0;
  for (size_t i = 0; i < ev.size() && nf < k;) {
    size_t j = i;
    while (j + 1 < ev.size() && ev[j + 1] - ev[i] <= tol) ++j;
    bool good = j > i;  // repeated: a converged eigenvalue
    if (!good) {
      good = true;
      for (double y : evh)
        if (std::fabs(y - ev[i]) <= tol) {
          good = false;
          break;
        }
    }
    if (good || m == 1) evals[nf++] = ev[i];
    i = j + 1;
  }
  *found = nf;
  return check_device_error(h);
}

qaa_status qaa_set_launch_mode(qaa_handle h, int mode) {
  if (!h) return fail(QAA_E_ARG, "null handle");
  if (mode != QAA_LAUNCH_PASSES && mode != QAA_LAUNCH_GRAPH)
    return fail(QAA_E_ARG, "unknown launch mode (0 = per-pass launches, 1 = launch graph)");
  h->launch_mode = mode;
  return QAA_OK;
}

qaa_status qaa_init_uniform(qaa_handle h, void* psi) {
  qaa_status st = check_handle(h);
  if (st) return st;
  if (!psi) return fail(QAA_E_ARG, "psi is null");
  QAA_CK(timed(h, QAA_K_INIT, [&] { return qaa::launch_init_uniform(lctx(h), static_cast<float2*>(psi), h->n); }));
  return QAA_OK;
}

qaa_status qaa_evolve(qaa_handle h, void* psi, double T, int64_t steps) {
  if (!(T >= 0.0) || !std::isfinite(T)) return fail(QAA_E_ARG, "T must be finite and >= 0");
  if (steps < 1) return fail(QAA_E_ARG, "steps must be >= 1");
  return evolve_impl(h, psi, T / static_cast<double>(steps), steps, 0, steps, nullptr);
}

qaa_status qaa_evolve_range(qaa_handle h, void* psi, double T, int64_t steps, int64_t k0, int64_t k1) {
  if (!(T >= 0.0) || !std::isfinite(T)) return fail(QAA_E_ARG, "T must be finite and >= 0");
  if (steps < 1) return fail(QAA_E_ARG, "steps must be >= 1");
  return evolve_impl(h, psi, T / static_cast<double>(steps), steps, k0, k1, nullptr);
}

qaa_status qaa_evolve_substeps(qaa_handle h, void* psi, const double* dt_values, const double* s_values, int64_t count) {
  if (!dt_values || !s_values) return fail(QAA_E_ARG, "dt_values or s_values is null");
  if (count < 1) return fail(QAA_E_ARG, "count must be >= 1");
  for (int64_t k = 0; k < count; ++k)
    if (!std::isfinite(dt_values[k]) || !std::isfinite(s_values[k]))
      return fail(QAA_E_ARG, "dt_values and s_values must be finite");
  return evolve_impl(h, psi, 0.0, count, 0, count, s_values, dt_values);
}

qaa_status qaa_evolve_order4(qaa_handle h, void* psi, double T, int64_t steps) {
  if (!(T >= 0.0) || !std::isfinite(T)) return fail(QAA_E_ARG, "T must be finite and >= 0");
  if (steps < 1 || steps > (1ll << 28)) return fail(QAA_E_ARG, "steps must be in [1, 2^28]");
  // Yoshida's triple jump: weights w1, w0, w1 with 2 w1 + w0 = 1, 2 w1^3 + w0^3 = 0
  const double w1 = 1.0 / (2.0 - std::cbrt(2.0)), w0 = 1.0 - 2.0 * w1;
  const double w[3] = {w1, w0, w1};
  const double dt = T / static_cast<double>(steps);
  std::vector<double> dts(static_cast<size_t>(3 * steps)), ss(static_cast<size_t>(3 * steps));
  for (int64_t k = 0; k < steps; ++k) {
    double t = static_cast<double>(k) * dt;
    for (int j = 0; j < 3; ++j) {
      const double h_j = w[j] * dt;
      dts[static_cast<size_t>(3 * k + j)] = h_j;
      ss[static_cast<size_t>(3 * k + j)] = T > 0.0 ? (t + 0.5 * h_j) / T : 0.5;
      t += h_j;
    }
  }
  return evolve_impl(h, psi, 0.0, 3 * steps, 0, 3 * steps, ss.data(), dts.data());
}

qaa_status qaa_evolve_schedule(qaa_handle h, void* psi, double dt, const double* s_values, int64_t steps) {
  if (!s_values) return fail(QAA_E_ARG, "s_values is null");
  if (steps < 1) return fail(QAA_E_ARG, "steps must be >= 1");
  for (int64_t k = 0; k < steps; ++k)
    if (!std::isfinite(s_values[k])) return fail(QAA_E_ARG, "s_values must be finite");
  return evolve_impl(h, psi, dt, steps, 0, steps, s_values);
}

qaa_status qaa_observables(qaa_handle h, const void* psi, qaa_obs* out) {
  if (!out) return fail(QAA_E_ARG, "out is null");
  double r[5];
  qaa_status st = observe(h, psi, r);
  if (st) return st;
  out->norm = r[0];
  out->expect_hp = r[1];
  out->ground_prob = r[2];
  out->ground_count = static_cast<int64_t>(std::llround(r[3]));
  out->expect_hb = 0.5 * h->n * r[0] - r[4];
  return QAA_OK;
}

qaa_status qaa_energy(qaa_handle h, const void* psi, double s, double* out) {
  if (!out) return fail(QAA_E_ARG, "out is null");
  qaa_obs o;
  qaa_status st = qaa_observables(h, psi, &o);
  if (st) return st;
  *out = (1.0 - s) * o.expect_hb + s * o.expect_hp;
  return QAA_OK;
}

qaa_status qaa_success_prob(qaa_handle h, const void* psi, double* out) {
  if (!out) return fail(QAA_E_ARG, "out is null");
  qaa_obs o;
  qaa_status st = qaa_observables(h, psi, &o);
  if (st) return st;
  *out = o.ground_prob;
  return QAA_OK;
}

qaa_status qaa_norm(qaa_handle h, const void* psi, double* out) {
  if (!out) return fail(QAA_E_ARG, "out is null");
  qaa_obs o;
  qaa_status st = qaa_observables(h, psi, &o);
  if (st) return st;
  *out = o.norm;
  return QAA_OK;
}

qaa_status qaa_hp_diagonal(qaa_handle h, uint16_t* out_dev) {
  qaa_status st = check_handle(h);
  if (st) return st;
  if (!out_dev) return fail(QAA_E_ARG, "out is null");
  if (reinterpret_cast<uintptr_t>(out_dev) % 2u) return fail(QAA_E_ARG, "out must be 2-byte aligned");
  QAA_CK(timed(h, QAA_K_DIAG, [&] { return qaa::launch_hp_diag(lctx(h), out_dev, h->n, h->m, h->d_lp); }));
  return QAA_OK;
}

qaa_status qaa_describe_plan(qaa_handle h, char* buf, size_t len) {
  if (!h) return fail(QAA_E_ARG, "null handle");
  if (!buf || len == 0) return fail(QAA_E_ARG, "buf is null or empty");
  const std::string d = qaa::describe_plan(h->plan);
  std::strncpy(buf, d.c_str(), len - 1);
  buf[len - 1] = '\0';
  return QAA_OK;
}

qaa_status qaa_profile_enable(qaa_handle h, int on) {
  qaa_status st = check_handle(h);
  if (st) return st;
  if (!on) {
    st = fold_profile(h);
    if (st) return st;
  }
  h->prof = on != 0;
  return QAA_OK;
}

qaa_status qaa_profile_reset(qaa_handle h) {
  qaa_status st = check_handle(h);
  if (st) return st;
  st = fold_profile(h);
  if (st) return st;
  for (int k = 0; k < QAA_K_COUNT; ++k) {
    h->prof_n[k] = 0;
    h->prof_ms[k] = 0.0;
  }
  return QAA_OK;
}

qaa_status qaa_profile_read(qaa_handle h, int kind, int64_t* launches, double* total_ms) {
  qaa_status st = check_handle(h);
  if (st) return st;
  if (kind < 0 || kind >= QAA_K_COUNT) return fail(QAA_E_ARG, "unknown kernel kind");
  st = fold_profile(h);
  if (st) return st;
  QAA_CK(cudaStreamSynchronize(h->stream));
  st = check_device_error(h);
  if (st) return st;
  if (launches) *launches = h->prof_n[kind];
  if (total_ms) *total_ms = h->prof_ms[kind];
  return QAA_OK;
}

}  // extern "C"
