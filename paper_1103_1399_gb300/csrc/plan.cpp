// Clause encoding and pass planning shared by the handle API and the server.
//
// Pass plan for n >= 15 (state streamed from HBM): G1 = bits 0..9 (low pass),
// the remaining n-10 bits in 1..3 strided groups of 5..10 bits.  The popcount
// phase B needs every qubit in the Hadamard basis, so it is fused into the pass
// of whichever strided group is transformed last (the phase group); the others
// are transformed before it (ascending) and after it (descending).  Per Strang
// step: phase group W B W, the other groups down, the low pass W P W (merging
// the half phases of two steps), the other groups up: 2g-2 HBM round trips for
// g groups.  n <= 14 runs entirely on chip.
#include <cstdlib>
#include <map>
#include <mutex>
#include <set>
#include <utility>
#include <cstring>
#include <string>
#include <vector>

#include "engine_internal.h"
#include "qaa.h"

namespace qaa {

int encode_clause(int n, const int32_t* lits, int c, ClauseMV& out, std::string& err) {
  unsigned long long mask = 0, viol = 0;
  int width = 0;
  for (int k = 0; k < 3; ++k) {
    const int32_t lit = lits[3 * c + k];
    if (lit == 0) continue;
    const long long a = lit < 0 ? -static_cast<long long>(lit) : lit;
    if (a > n) {
      err = "clause " + std::to_string(c) + ": literal beyond n";
      return QAA_E_ARG;
    }
    const unsigned long long bit = 1ull << (a - 1);
    if (mask & bit) {
      err = "clause " + std::to_string(c) + ": variable repeated in a clause";
      return QAA_E_ARG;
    }
    mask |= bit;
    if (lit < 0) viol |= bit;
    ++width;
  }
  if (width == 0) {
    err = "clause " + std::to_string(c) + ": no literals";
    return QAA_E_ARG;
  }
  out = {mask, viol};
  return QAA_OK;
}

ClauseLP clause_lp(const ClauseMV& mv) {
  ClauseLP e;
  e.hi_mask = static_cast<unsigned>(mv.mask >> kLowBits);
  e.hi_viol = static_cast<unsigned>(mv.viol >> kLowBits);
  unsigned p0 = 0, p5 = 0;
  const unsigned m0 = static_cast<unsigned>(mv.mask & 31u), v0 = static_cast<unsigned>(mv.viol & 31u);
  const unsigned m5 = static_cast<unsigned>((mv.mask >> 5) & 31u), v5 = static_cast<unsigned>((mv.viol >> 5) & 31u);
  for (unsigned j = 0; j < 32; ++j) {
    if ((j & m0) == v0) p0 |= 1u << j;
    if ((j & m5) == v5) p5 |= 1u << j;
  }
  e.pat0 = p0;
  e.pat5 = p5;
  return e;
}

int encode_clauses_lp(int n, const int32_t* lits, int m, ClauseLP* out, std::string& err) {
  for (int c = 0; c < m; ++c) {
    ClauseMV mv;
    const int st = encode_clause(n, lits, c, mv, err);
    if (st) return st;
    out[c] = clause_lp(mv);
  }
  return QAA_OK;
}

int encode_clauses(int n, const int32_t* lits, int m, std::vector<ClauseMV>& mv, std::vector<ClauseLP>& lp,
                   std::string& err) {
  mv.resize(static_cast<size_t>(m));
  lp.resize(static_cast<size_t>(m));
  for (int c = 0; c < m; ++c) {
    const int st = encode_clause(n, lits, c, mv[c], err);
    if (st) return st;
    lp[c] = clause_lp(mv[c]);
  }
  return QAA_OK;
}

namespace {
std::mutex g_tuned_mu;
std::map<std::pair<int, int>, PassPlan> g_tuned;  // (device, n) -> plan chosen by qaa_autotune

bool env_overrides() {
  for (const char* v :
       {"QAA_PASSES", "QAA_GROUP_BITS", "QAA_SPLIT_GROUPS", "QAA_PHASE_GROUP", "QAA_RUN128_GROUPS", "QAA_LOW_BITS"})
    if (std::getenv(v)) return true;
  return false;
}

int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return d;
}
}  // namespace

void set_tuned_plan(const PassPlan& plan) {
  std::lock_guard<std::mutex> lk(g_tuned_mu);
  g_tuned[{current_device(), plan.n}] = plan;
}

void clear_tuned_plans() {
  std::lock_guard<std::mutex> lk(g_tuned_mu);
  g_tuned.clear();
}

bool tuned_plan(int n, PassPlan& out) {
  std::lock_guard<std::mutex> lk(g_tuned_mu);
  auto it = g_tuned.find({current_device(), n});
  if (it == g_tuned.end()) return false;
  out = it->second;
  return true;
}

// Every split of `rest` bits into g ordered groups of 5..max_q bits.
static void compositions(int rest, int g, int max_q, std::vector<int>& cur, std::vector<std::vector<int>>& out) {
  if (g == 0) {
    if (rest == 0) out.push_back(cur);
    return;
  }
  for (int q = 5; q <= max_q && q <= rest; ++q) {
    cur.push_back(q);
    compositions(rest - q, g - 1, max_q, cur, out);
    cur.pop_back();
  }
}

void plan_with_groups(int n, const std::vector<int>& sizes, int phase_group, bool tma, PassPlan& plan) {
  plan = PassPlan();
  plan.n = n;
  plan.onchip = false;
  plan.use_tma = tma;
  int a = kLowBits;
  for (int q : sizes) {
    plan.strided.push_back({a, q, a + 5});
    a += q;
  }
  plan.phase_group = phase_group;
  plan.wht_kind = 0;  // stage 1 varies the W.B.W form's groups; stage 5 tries the rotation form
  set_default_run_c(plan);
}

void plan_candidates(int n, std::vector<PassPlan>& out) {
  out.clear();
  if (n <= kOnchipMaxBits) return;
  const int rest = n - kLowBits;
  const bool tma = tma_available();
  const int max_q = tma ? 11 : 10;
  const int g = (rest + max_q - 1) / max_q;
  std::vector<std::vector<int>> comps;
  std::vector<int> cur;
  compositions(rest, g, max_q, cur, comps);
  PassPlan def;
  make_default_plan(n, def);
  out.push_back(def);
  for (const auto& c : comps)
    for (int pg = 0; pg < g; ++pg) {
      PassPlan p;
      plan_with_groups(n, c, pg, tma, p);
      bool same = p.strided.size() == def.strided.size() && p.phase_group == def.phase_group;
      for (size_t i = 0; same && i < p.strided.size(); ++i)
        same = p.strided[i].a == def.strided[i].a && p.strided[i].q == def.strided[i].q &&
               p.strided[i].a2 == def.strided[i].a2;
      if (!same) out.push_back(p);
    }
  // the rotation form with a 12-bit low pass (kLpRot12), for states beyond L2
  if (tma && n >= 31) {
    PassPlan w;
    make_default_plan(n, w, max_q, 12);
    if (w.low_bits == 12 && def.low_bits != 12) out.push_back(w);
  }
}

static bool fits(const PassPlan& plan, int max_q) {
  for (const Group& g : plan.strided)
    if (g.q > max_q) return false;
  return true;
}

void make_plan(int n, PassPlan& plan, int max_q) {
  if (n > kOnchipMaxBits && !env_overrides() && tuned_plan(n, plan) && fits(plan, max_q)) return;
  make_default_plan(n, plan, max_q);
}

void make_default_plan(int n, PassPlan& plan, int max_q, int low) {
  plan = PassPlan();
  plan.n = n;
  plan.onchip = n <= kOnchipMaxBits;
  const char* env = std::getenv("QAA_PASSES");
  plan.use_tma = tma_available() && !(env && std::strcmp(env, "classic") == 0);
  if (plan.onchip) return;
  if (!plan.use_tma && max_q > 10) max_q = 10;  // 11-bit groups: TMA FP32 passes only
  // Low pass width: 10 bits, or 12 (kLpRot12, rotation form on TMA passes
  // only) when asked for here or by QAA_LOW_BITS.  Not the default: at n = 32
  // its two 10-bit groups with 128-byte runs ran 0.87 ms faster each than the
  // two 11-bit groups with 64-byte runs, but the 12-bit low pass itself took
  // 13.8 ms against 11.7 (its warp quads run in step and hide less latency):
  // 36.3 against 35.9 ms per step.  The autotuner offers it for n >= 31.
  if (low == 0) {
    const char* lb = std::getenv("QAA_LOW_BITS");
    low = lb ? std::atoi(lb) : kLowBits;
  }
  const int L = (low == 12 && plan.use_tma && n - 12 >= 5) ? 12 : kLowBits;
  plan.low_bits = L;
  const int rest = n - L;
  std::vector<int> sizes;
  if (const char* gb = std::getenv("QAA_GROUP_BITS")) {
    int sum = 0;
    bool ok = true;
    for (const char* p = gb; *p;) {
      const int q = std::atoi(p);
      if (q < 5 || q > max_q) ok = false;
      sizes.push_back(q);
      sum += q;
      while (*p && *p != ',') ++p;
      if (*p == ',') ++p;
    }
    if (!ok || sum != rest) sizes.clear();
  }
  if (sizes.empty()) {
    const int ng = (rest + max_q - 1) / max_q;
    const int base = rest / ng, extra = rest % ng;
    for (int g = 0; g < ng; ++g) sizes.push_back(base + (g < extra ? 1 : 0));
  }
  int a = L;
  for (int q : sizes) {
    plan.strided.push_back({a, q, a + 5});
    a += q;
  }
  // Two equal q-bit strided groups (q = 10 or 11: n = 30, 32), e.g. [10,20)
  // and [20,30): recombine them as {10..14, 25..29} and {15..24}.  With
  // [20,30) as one group every tile has 1024 rows 8 MiB apart, each on its own
  // memory page; recombined, a tile spans at most 128 pages (measured: 6.7 ms
  // -> 3.1 ms per pass at n = 30).
  const char* sg = std::getenv("QAA_SPLIT_GROUPS");
  const bool split = plan.use_tma && !(sg && std::atoi(sg) == 0);
  if (split && plan.strided.size() == 2 && plan.strided[0].q == plan.strided[1].q && plan.strided[0].q >= 10) {
    const int q = plan.strided[0].q;
    plan.strided[0] = {L, q, L + q + 5};
    plan.strided[1] = {L + 5, q, L + 10};
  }
  // Three groups at n = 33..34 (23..24 strided bits): contiguous 8-bit groups
  // put rows up to 512 MiB apart, 256 memory pages per tile.  Instead an 11-bit
  // group {L..L+4} + the top 6 bits, and the bits between in two contiguous
  // groups: at most 64 pages per tile.
  if (split && plan.strided.size() == 3 && max_q >= 11 && n >= 33 && L == kLowBits) {
    const int mid = n - 6 - (L + 5);  // bits [L+5, n-6) for the other two groups
    const int q1 = (mid + 1) / 2, q2 = mid - q1;
    if (q2 >= 5) {
      plan.strided[0] = {L, 11, n - 6};
      plan.strided[1] = {L + 5, q1, L + 10};
      plan.strided[2] = {L + 5 + q1, q2, L + 10 + q1};
    }
  }
  const int ng = static_cast<int>(plan.strided.size());
  plan.phase_group = ng - 1;
  if (const char* pg = std::getenv("QAA_PHASE_GROUP")) {
    const int v = std::atoi(pg);
    if (v >= 0 && v < ng) plan.phase_group = v;
  }
  // The form of the H_B factor: on the TMA FP32 passes the rotation form
  // (W.diag.W on every 5-qubit block inside each pass: g round trips per
  // step), otherwise the W.B.W form (2g - 2).
  plan.wht_kind = plan.use_tma ? kRotationForm : 0;
  set_default_run_c(plan);
}

void narrow_low_pass(PassPlan& plan, int max_q) {
  if (plan.onchip || plan.low_bits == kLowBits) return;
  const int wk = plan.wht_kind;
  make_default_plan(plan.n, plan, max_q, kLowBits);
  plan.wht_kind = wk;
  set_default_run_c(plan);
}

void set_default_run_c(PassPlan& plan) {
  // Contiguous run per tile row.  W.B.W form: 128 bytes for the plain strided
  // passes, 64 bytes (three CTAs per SM) for the heavier pass that hosts the
  // phase.  Rotation form: 128 bytes for every group (measured at n = 30: 8.97
  // ms per step, against 9.74 with 64 bytes for one group and 10.56 for both;
  // its passes start the next tile's copy before their second stage).
  const int ng = static_cast<int>(plan.strided.size());
  const char* rg = std::getenv("QAA_RUN128_GROUPS");
  const int rmask = rg ? std::atoi(rg) : -1;
  plan.run_c.resize(static_cast<size_t>(ng));
  for (int i = 0; i < ng; ++i) {
    if (rmask >= 0)
      plan.run_c[i] = ((rmask >> i) & 1) ? 4 : 0;
    else if (plan.wht_kind == kRotationForm)
      plan.run_c[i] = 4;
    else
      plan.run_c[i] = i == plan.phase_group ? 0 : 4;
  }
}

// Rotation form (variant 3): exp(-i theta H_B) = prod_i exp(-i theta (1 - sigma^x_i)/2),
// one-qubit factors on disjoint qubits, so every group is transformed once per
// step in any order and no pass changes basis.  A range starts with P alone;
// step k is the strided groups' rotations, then the low pass's rotations and
// the P phase at the boundary after step k (merged with the next step's first
// half, or the last half at the end of the range): g round trips per step.
static void build_rot_passes(const PassPlan& plan, long long k0, long long c0, long long c1, std::vector<Pass>& out) {
  if (c0 == k0) out.push_back({kLpPhase, 0, 0, 0, 0, 0, 0, -1});
  for (long long k = c0; k < c1; ++k) {
    const int brow = static_cast<int>(k - c0);
    for (size_t i = 0; i < plan.strided.size(); ++i) {
      const Group& g = plan.strided[i];
      out.push_back({kSpRot, g.a, g.q, 0, plan.run_c[i], brow, g.a2});
    }
    out.push_back({plan.low_bits == 12 ? kLpRot12 : kLpRot, 0, 0, static_cast<int>(k + 1 - c0), 0, brow, 0,
                   static_cast<int>(k - k0)});
  }
}

void build_passes(const PassPlan& plan, long long k0, long long k1, long long c0, long long c1,
                  std::vector<Pass>& out) {
  out.clear();
  if (plan.wht_kind == kRotationForm) {
    build_rot_passes(plan, k0, c0, c1, out);
    return;
  }
  const int ng = static_cast<int>(plan.strided.size());
  const int pg = plan.phase_group;
  const Group top = plan.strided[pg];
  auto other = [&](int i) {
    const Group& g = plan.strided[i];
    out.push_back({kSpW, g.a, g.q, 0, plan.run_c[i], 0, g.a2});
  };
  auto up = [&]() {
    for (int i = 0; i < ng; ++i)
      if (i != pg) other(i);
  };
  auto down = [&]() {
    for (int i = ng - 1; i >= 0; --i)
      if (i != pg) other(i);
  };
  if (c0 == k0) {
    out.push_back({kLpFirst, 0, 0, 0, 0, 0, 0, -1});
    up();
  }
  for (long long k = c0; k < c1; ++k) {
    out.push_back({kSpWBW, top.a, top.q, 0, plan.run_c[pg], static_cast<int>(k - c0), top.a2});
    down();
    const int rel = static_cast<int>(k - k0);
    if (k == k1 - 1) {
      out.push_back({kLpLast, 0, 0, static_cast<int>(k + 1 - c0), 0, 0, 0, rel});
    } else {
      out.push_back({kLpMerge, 0, 0, static_cast<int>(k + 1 - c0), 0, 0, 0, rel});
      up();
    }
  }
}

std::string describe_plan(const PassPlan& plan) {
  if (plan.onchip) return "on-chip: whole run in one CTA's shared memory (n=" + std::to_string(plan.n) + ")";
  const int ng = static_cast<int>(plan.strided.size());
  if (plan.wht_kind == kRotationForm) {
    std::string d = "streaming, TMA loads, rotation form (H_B per 5-qubit block: W.diag.W); low pass bits [0," +
                    std::to_string(plan.low_bits) + ") R.P";
    for (int i = 0; i < ng; ++i) {
      const Group& g = plan.strided[i];
      d += "; group bits [" + std::to_string(g.a) + "," + std::to_string(g.a + 5) + ")";
      if (g.q > 5) d += "+[" + std::to_string(g.a2) + "," + std::to_string(g.a2 + g.q - 5) + ")";
      d += " R " + std::to_string(tma_run_bytes(g.q, plan.run_c[i])) + "B runs";
    }
    return d + "; " + std::to_string(ng + 1) + " HBM round trips per step";
  }
  const char* wk = plan.wht_kind == 1 ? "tensor-core BF16x3" : (plan.wht_kind == 2 ? "tensor-core BF16x2" : "FP32");
  std::string d = "streaming, " + std::string(plan.wht_kind ? "plain" : (plan.use_tma ? "TMA" : "classic")) +
                  " loads, " + wk + " WHT; low pass bits [0,10) W.P.W";
  for (int i = 0; i < ng; ++i) {
    const Group& g = plan.strided[i];
    d += "; group bits [" + std::to_string(g.a) + "," + std::to_string(g.a + 5) + ")";
    if (g.q > 5) d += "+[" + std::to_string(g.a2) + "," + std::to_string(g.a2 + g.q - 5) + ")";
    d += i == plan.phase_group ? " W.B.W" : " W";
    if (plan.use_tma && !plan.wht_kind) d += " " + std::to_string(tma_run_bytes(g.q, plan.run_c[i])) + "B runs";
  }
  d += "; " + std::to_string(2 * ng) + " HBM round trips per step";
  return d;
}

cudaError_t allow_smem(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({dev, func})) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e == cudaSuccess) done.insert({dev, func});
  return e;
}

cudaError_t launch_planned_pass(const LaunchCtx& lc, const PassPlan& plan, const Pass& p, float2* psi, int m,
                                const ClauseLP* cl, const float2* ptab, const float2* btab, int* err, const unsigned* counts,
                                double* fold) {
  const NormFold nf = fold_for(fold, p, fold_period(plan.n));
  if (plan.wht_kind == kRotationForm) return launch_pass_tma(lc, p, psi, plan.n, m, cl, ptab, btab, err, counts, nf);
  if (plan.wht_kind)
    return launch_pass_tc(lc, p, psi, plan.n, m, cl, ptab, btab, plan.wht_kind == 1 ? 3 : 2, err, counts, nf);
  if (plan.use_tma) return launch_pass_tma(lc, p, psi, plan.n, m, cl, ptab, btab, err, counts, nf);
  return launch_pass(lc, p, psi, plan.n, m, cl, ptab, btab, nf);
}

}  // namespace qaa
