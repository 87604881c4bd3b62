// Host engine behind the C ABI of include/qaa.h: clause encoding, pass
// planning, phase-table scheduling and kernel launch order.
//
// Clause encoding (Sec. 2.2 clauses, Sec. 4.3 energy): a clause over literals
// l_1..l_k is violated exactly when every literal is false, i.e. when
// (x & mask) == viol with mask the bits of its variables and viol the value of
// each variable that falsifies its literal (0 for x_i, 1 for NOT x_i).
//
// Pass plan for n >= 15 (state streamed from HBM): G1 = bits 0..9 (low pass),
// the remaining n-10 bits split into 1..3 strided groups of 5..10 bits.  Per
// Strang step: top group W B W, the middle groups downwards, the low pass
// W P W (merging the half phases of two steps), the middle groups upwards:
// 2g-2 HBM round trips for g groups.  n <= 14 runs entirely on chip.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "qaa.h"
#include "qaa_internal.cuh"

namespace {

thread_local std::string g_last_error = "no error";

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define QAA_CK(expr)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(QAA_E_CUDA, std::string(#expr) + " failed: " + cudaGetErrorString(e_)); \
  } while (0)

constexpr long long kChunkSteps = 1024;

struct Group {
  int a, q, a2;  // active bits [a, a+5) and [a2, a2+q-5); a2 == a + 5 for a contiguous group
};

}  // namespace

struct qaa_ctx {
  int n = 0, m = 0, device = 0, num_sms = 0;
  cudaStream_t stream = nullptr;
  int wht_kind = 0;
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
  bool use_tma = true;      // TMA-pipelined streaming passes (QAA_PASSES=classic selects the others)
  int phase_group = 1 << 20;  // strided group hosting the popcount phase (default: the top one)
  bool split_groups = true;   // recombine two 10-bit strided groups (see plan_groups)
  int run128_groups = -1;     // bit i set: strided group i uses 128-byte runs (-1: default policy)
  std::vector<Group> strided;  // ascending bit order; back() is the top group
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

int encode(qaa_ctx* h, const int32_t* clauses) {
  h->mv.resize(static_cast<size_t>(h->m));
  h->lp.resize(static_cast<size_t>(h->m));
  for (int c = 0; c < h->m; ++c) {
    unsigned long long mask = 0, viol = 0;
    int width = 0;
    for (int k = 0; k < 3; ++k) {
      const int32_t lit = clauses[3 * c + k];
      if (lit == 0) continue;
      const long long a = lit < 0 ? -static_cast<long long>(lit) : lit;
      if (a > h->n) return fail(QAA_E_ARG, "clause " + std::to_string(c) + ": literal beyond n");
      const unsigned long long bit = 1ull << (a - 1);
      if (mask & bit) return fail(QAA_E_ARG, "clause " + std::to_string(c) + ": variable repeated in a clause");
      mask |= bit;
      if (lit < 0) viol |= bit;
      ++width;
    }
    if (width == 0) return fail(QAA_E_ARG, "clause " + std::to_string(c) + ": no literals");
    h->mv[c] = {mask, viol};
    qaa::ClauseLP e;
    e.hi_mask = static_cast<unsigned>(mask >> qaa::kLowBits);
    e.hi_viol = static_cast<unsigned>(viol >> qaa::kLowBits);
    unsigned p0 = 0, p5 = 0;
    const unsigned m0 = static_cast<unsigned>(mask & 31u), v0 = static_cast<unsigned>(viol & 31u);
    const unsigned m5 = static_cast<unsigned>((mask >> 5) & 31u), v5 = static_cast<unsigned>((viol >> 5) & 31u);
    for (unsigned j = 0; j < 32; ++j) {
      if ((j & m0) == v0) p0 |= 1u << j;
      if ((j & m5) == v5) p5 |= 1u << j;
    }
    e.pat0 = p0;
    e.pat5 = p5;
    h->lp[c] = e;
  }
  return QAA_OK;
}

// Strided groups above the low pass: the n-10 remaining bits in groups of 5..10
// (as equal as possible), or the sizes given in QAA_GROUP_BITS ("10,8"), a
// tuning override.
void plan_groups(qaa_ctx* h) {
  h->strided.clear();
  if (h->n <= qaa::kOnchipMaxBits) return;
  const int rest = h->n - qaa::kLowBits;
  std::vector<int> sizes;
  if (const char* gb = std::getenv("QAA_GROUP_BITS")) {
    int sum = 0;
    bool ok = true;
    for (const char* p = gb; *p;) {
      const int q = std::atoi(p);
      if (q < 5 || q > 10) ok = false;
      sizes.push_back(q);
      sum += q;
      while (*p && *p != ',') ++p;
      if (*p == ',') ++p;
    }
    if (!ok || sum != rest) sizes.clear();
  }
  if (sizes.empty()) {
    const int ng = (rest + 9) / 10;
    const int base = rest / ng, extra = rest % ng;
    for (int g = 0; g < ng; ++g) sizes.push_back(base + (g < extra ? 1 : 0));
  }
  int a = qaa::kLowBits;
  for (int q : sizes) {
    h->strided.push_back({a, q, a + 5});
    a += q;
  }
  // Two 10-bit strided groups [10,20) and [20,30): recombine them as
  // {10..14, 25..29} and {15..24}.  With [20,30) as one group every tile has
  // 1024 rows 8 MiB apart, each on its own memory page; recombined, a tile
  // spans at most 128 pages.
  if (h->split_groups && h->strided.size() == 2 && h->strided[0].q == 10 && h->strided[1].q == 10) {
    const int b = qaa::kLowBits;
    h->strided[0] = {b, 10, b + 15};
    h->strided[1] = {b + 5, 10, b + 10};
  }
}

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

int fold_profile(qaa_ctx* h) {
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

int ensure_tab(qaa_ctx* h, size_t entries) {
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

// The popcount phase B needs every qubit in the Hadamard basis, so it is applied
// inside the pass of whichever strided group is transformed last (the "phase
// group"); the others are transformed before it (in ascending order) and after
// it (descending).
void build_passes(const qaa_ctx* h, long long k0, long long k1, long long c0, long long c1,
                  std::vector<qaa::Pass>& out) {
  out.clear();
  const int ng = static_cast<int>(h->strided.size());
  const int pg = h->phase_group < ng ? h->phase_group : ng - 1;
  const Group top = h->strided[pg];
  // Contiguous run per tile row: 128 bytes for the plain strided passes, 64
  // bytes (more CTAs per SM) for the heavier pass that hosts the phase.
  auto runc = [&](int i) {
    if (h->run128_groups >= 0) return ((h->run128_groups >> i) & 1) ? 4 : 0;
    return i == pg ? 0 : 4;
  };
  auto mid_up = [&]() {
    for (int i = 0; i < ng; ++i)
      if (i != pg) out.push_back({qaa::kSpW, h->strided[i].a, h->strided[i].q, 0, runc(i), 0, h->strided[i].a2});
  };
  auto mid_down = [&]() {
    for (int i = ng - 1; i >= 0; --i)
      if (i != pg) out.push_back({qaa::kSpW, h->strided[i].a, h->strided[i].q, 0, runc(i), 0, h->strided[i].a2});
  };
  if (c0 == k0) {
    out.push_back({qaa::kLpFirst, 0, 0, 0, 0, 0, 0});
    mid_up();
  }
  for (long long k = c0; k < c1; ++k) {
    out.push_back({qaa::kSpWBW, top.a, top.q, 0, runc(pg), static_cast<int>(k - c0), top.a2});
    mid_down();
    if (k == k1 - 1) {
      out.push_back({qaa::kLpLast, 0, 0, static_cast<int>(k + 1 - c0), 0, 0, 0});
    } else {
      out.push_back({qaa::kLpMerge, 0, 0, static_cast<int>(k + 1 - c0), 0, 0, 0});
      mid_up();
    }
  }
}

int check_handle(qaa_ctx* h) {
  if (!h) return fail(QAA_E_ARG, "null handle");
  QAA_CK(cudaSetDevice(h->device));
  return QAA_OK;
}

// After a stream synchronisation: report (and clear) an expired device wait.
int check_device_error(qaa_ctx* h) {
  int e = 0;
  QAA_CK(cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != 0) {
    QAA_CK(cudaMemset(h->d_err, 0, sizeof(int)));
    return fail(QAA_E_TIMEOUT, "a bounded wait on a TMA copy expired in a streaming pass");
  }
  return QAA_OK;
}

int evolve_impl(qaa_ctx* h, void* psi, double dt, long long K, long long k0, long long k1, const double* s_host) {
  int st = check_handle(h);
  if (st) return st;
  if (!psi) return fail(QAA_E_ARG, "psi is null");
  if (reinterpret_cast<uintptr_t>(psi) % 16u) return fail(QAA_E_ARG, "psi must be 16-byte aligned");
  if (K < 1 || k0 < 0 || k1 < k0 || k1 > K) return fail(QAA_E_ARG, "bad step range");
  if (!std::isfinite(dt)) return fail(QAA_E_ARG, "dt must be finite");
  if (k0 == k1) return QAA_OK;
  const double* s_dev = nullptr;
  if (s_host) {
    const size_t need = static_cast<size_t>(K);
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
    QAA_CK(cudaMemcpyAsync(h->d_s, s_host, need * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    s_dev = h->d_s;
  }
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
      return qaa::launch_tables(lc, ptab, btab, h->n, h->m, dt, s_dev, K, k0, k1, c0, c1);
    }));
    if (h->n <= qaa::kOnchipMaxBits) {
      QAA_CK(timed(h, QAA_K_ONCHIP, [&] {
        return qaa::launch_onchip(lc, p, h->n, h->m, h->d_mv, ptab, btab, static_cast<int>(c1 - c0), c0 == k0);
      }));
    } else {
      build_passes(h, k0, k1, c0, c1, passes);
      const bool tma = h->use_tma;
      const int tc_parts = h->wht_kind == 1 ? 3 : (h->wht_kind == 2 ? 2 : 0);
      for (const qaa::Pass& ps : passes)
        QAA_CK(timed(h, ps.kind, [&] {
          if (tc_parts) return qaa::launch_pass_tc(lc, ps, p, h->n, h->m, h->d_lp, ptab, btab, tc_parts);
          return tma ? qaa::launch_pass_tma(lc, ps, p, h->n, h->m, h->d_lp, ptab, btab, h->d_err)
                     : qaa::launch_pass(lc, ps, p, h->n, h->m, h->d_lp, ptab, btab);
        }));
    }
  }
  return QAA_OK;
}

int observe(qaa_ctx* h, const void* psi, double out[5]) {
  int st = check_handle(h);
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
    return qaa::launch_observables(lctx(h), static_cast<const float2*>(psi), h->n, h->m, h->d_lp, h->d_part, h->d_res);
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

int qaa_create(int n, const int32_t* clauses, int m, qaa_handle* out) {
  if (!out) return fail(QAA_E_ARG, "out is null");
  *out = nullptr;
  if (n < 1 || n > QAA_MAX_QUBITS) return fail(QAA_E_ARG, "n out of range [1, 34]");
  if (m < 0 || m > QAA_MAX_CLAUSES) return fail(QAA_E_ARG, "m out of range [0, 1023]");
  if (m > 0 && !clauses) return fail(QAA_E_ARG, "clauses is null");
  qaa_ctx* h = new (std::nothrow) qaa_ctx;
  if (!h) return fail(QAA_E_NOMEM, "host allocation failed");
  h->n = n;
  h->m = m;
  int st = encode(h, clauses);
  if (st) {
    delete h;
    return st;
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
      cudaMallocHost(&h->h_res, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(QAA_E_NOMEM, "cannot allocate clause tables");
  }
  if (cudaMemset(h->d_err, 0, sizeof(int)) != cudaSuccess) return cleanup(QAA_E_CUDA, "cannot clear error word");
  {
    const char* env = std::getenv("QAA_PASSES");
    h->use_tma = qaa::tma_available() && !(env && std::strcmp(env, "classic") == 0);
    const char* pg = std::getenv("QAA_PHASE_GROUP");
    if (pg) h->phase_group = std::atoi(pg);
    const char* rg = std::getenv("QAA_RUN128_GROUPS");
    if (rg) h->run128_groups = std::atoi(rg);
    const char* sg = std::getenv("QAA_SPLIT_GROUPS");
    h->split_groups = h->use_tma && !(sg && std::atoi(sg) == 0);
    plan_groups(h);
  }
  if (m > 0) {
    if (cudaMemcpy(h->d_mv, h->mv.data(), m * sizeof(qaa::ClauseMV), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_lp, h->lp.data(), m * sizeof(qaa::ClauseLP), cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup(QAA_E_CUDA, "cannot upload clause tables");
  }
  *out = h;
  return QAA_OK;
}

int qaa_destroy(qaa_handle h) {
  if (!h) return QAA_OK;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  cudaFree(h->d_mv);
  cudaFree(h->d_lp);
  cudaFree(h->d_tab);
  cudaFree(h->d_s);
  cudaFree(h->d_part);
  cudaFree(h->d_res);
  cudaFree(h->d_err);
  if (h->h_res) cudaFreeHost(h->h_res);
  for (auto& p : h->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (cudaEvent_t e : h->ev_free) cudaEventDestroy(e);
  delete h;
  return QAA_OK;
}

int qaa_set_stream(qaa_handle h, void* cuda_stream) {
  if (!h) return fail(QAA_E_ARG, "null handle");
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  return QAA_OK;
}

int qaa_set_variant(qaa_handle h, int wht_kind, int q) {
  if (!h) return fail(QAA_E_ARG, "null handle");
  if (wht_kind < 0 || wht_kind > 2) return fail(QAA_E_ARG, "unknown wht_kind (0 = FP32, 1 = BF16x3, 2 = BF16x2)");
  if (q != 0) return fail(QAA_E_ARG, "only automatic qubits-per-pass (q = 0) is available");
  h->wht_kind = wht_kind;
  return QAA_OK;
}

int qaa_init_uniform(qaa_handle h, void* psi) {
  int st = check_handle(h);
  if (st) return st;
  if (!psi) return fail(QAA_E_ARG, "psi is null");
  QAA_CK(timed(h, QAA_K_INIT, [&] { return qaa::launch_init_uniform(lctx(h), static_cast<float2*>(psi), h->n); }));
  return QAA_OK;
}

int qaa_evolve(qaa_handle h, void* psi, double T, int64_t steps) {
  if (!(T >= 0.0) || !std::isfinite(T)) return fail(QAA_E_ARG, "T must be finite and >= 0");
  if (steps < 1) return fail(QAA_E_ARG, "steps must be >= 1");
  return evolve_impl(h, psi, T / static_cast<double>(steps), steps, 0, steps, nullptr);
}

int qaa_evolve_range(qaa_handle h, void* psi, double T, int64_t steps, int64_t k0, int64_t k1) {
  if (!(T >= 0.0) || !std::isfinite(T)) return fail(QAA_E_ARG, "T must be finite and >= 0");
  if (steps < 1) return fail(QAA_E_ARG, "steps must be >= 1");
  return evolve_impl(h, psi, T / static_cast<double>(steps), steps, k0, k1, nullptr);
}

int qaa_evolve_schedule(qaa_handle h, void* psi, double dt, const double* s_values, int64_t steps) {
  if (!s_values) return fail(QAA_E_ARG, "s_values is null");
  if (steps < 1) return fail(QAA_E_ARG, "steps must be >= 1");
  for (int64_t k = 0; k < steps; ++k)
    if (!std::isfinite(s_values[k])) return fail(QAA_E_ARG, "s_values must be finite");
  return evolve_impl(h, psi, dt, steps, 0, steps, s_values);
}

int qaa_observables(qaa_handle h, const void* psi, qaa_obs* out) {
  if (!out) return fail(QAA_E_ARG, "out is null");
  double r[5];
  int st = observe(h, psi, r);
  if (st) return st;
  out->norm = r[0];
  out->expect_hp = r[1];
  out->ground_prob = r[2];
  out->ground_count = static_cast<int64_t>(std::llround(r[3]));
  out->expect_hb = 0.5 * h->n * r[0] - r[4];
  return QAA_OK;
}

int qaa_energy(qaa_handle h, const void* psi, double s, double* out) {
  if (!out) return fail(QAA_E_ARG, "out is null");
  qaa_obs o;
  int st = qaa_observables(h, psi, &o);
  if (st) return st;
  *out = (1.0 - s) * o.expect_hb + s * o.expect_hp;
  return QAA_OK;
}

int qaa_success_prob(qaa_handle h, const void* psi, double* out) {
  if (!out) return fail(QAA_E_ARG, "out is null");
  qaa_obs o;
  int st = qaa_observables(h, psi, &o);
  if (st) return st;
  *out = o.ground_prob;
  return QAA_OK;
}

int qaa_norm(qaa_handle h, const void* psi, double* out) {
  if (!out) return fail(QAA_E_ARG, "out is null");
  qaa_obs o;
  int st = qaa_observables(h, psi, &o);
  if (st) return st;
  *out = o.norm;
  return QAA_OK;
}

int qaa_hp_diagonal(qaa_handle h, uint16_t* out_dev) {
  int st = check_handle(h);
  if (st) return st;
  if (!out_dev) return fail(QAA_E_ARG, "out is null");
  if (reinterpret_cast<uintptr_t>(out_dev) % 2u) return fail(QAA_E_ARG, "out must be 2-byte aligned");
  QAA_CK(timed(h, QAA_K_DIAG, [&] { return qaa::launch_hp_diag(lctx(h), out_dev, h->n, h->m, h->d_lp); }));
  return QAA_OK;
}

int qaa_describe_plan(qaa_handle h, char* buf, size_t len) {
  if (!h) return fail(QAA_E_ARG, "null handle");
  if (!buf || len == 0) return fail(QAA_E_ARG, "buf is null or empty");
  std::string d;
  if (h->n <= qaa::kOnchipMaxBits) {
    d = "on-chip: whole run in one CTA's shared memory (n=" + std::to_string(h->n) + ")";
  } else {
    const int ng = static_cast<int>(h->strided.size());
    const int pg = h->phase_group < ng ? h->phase_group : ng - 1;
    const char* wk = h->wht_kind == 1 ? "tensor-core BF16x3" : (h->wht_kind == 2 ? "tensor-core BF16x2" : "FP32");
    d = "streaming, " + std::string(h->wht_kind ? "plain" : (h->use_tma ? "TMA" : "classic")) + " loads, " + wk +
        " WHT; low pass bits [0,10) W.P.W";
    for (int i = 0; i < ng; ++i) {
      const Group& g = h->strided[i];
      int c = i == pg ? 0 : 4;
      if (h->run128_groups >= 0) c = ((h->run128_groups >> i) & 1) ? 4 : 0;
      d += "; group bits [" + std::to_string(g.a) + "," + std::to_string(g.a + 5) + ")";
      if (g.q > 5) d += "+[" + std::to_string(g.a2) + "," + std::to_string(g.a2 + g.q - 5) + ")";
      d += i == pg ? " W.B.W" : " W";
      if (h->use_tma && !h->wht_kind) d += c == 4 ? " 128B runs" : " 64B runs";
    }
    d += "; " + std::to_string(2 * (ng + 1) - 2) + " HBM round trips per step";
  }
  std::strncpy(buf, d.c_str(), len - 1);
  buf[len - 1] = '\0';
  return QAA_OK;
}

int qaa_profile_enable(qaa_handle h, int on) {
  int st = check_handle(h);
  if (st) return st;
  if (!on) {
    st = fold_profile(h);
    if (st) return st;
  }
  h->prof = on != 0;
  return QAA_OK;
}

int qaa_profile_reset(qaa_handle h) {
  int st = check_handle(h);
  if (st) return st;
  st = fold_profile(h);
  if (st) return st;
  for (int k = 0; k < QAA_K_COUNT; ++k) {
    h->prof_n[k] = 0;
    h->prof_ms[k] = 0.0;
  }
  return QAA_OK;
}

int qaa_profile_read(qaa_handle h, int kind, int64_t* launches, double* total_ms) {
  int st = check_handle(h);
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
