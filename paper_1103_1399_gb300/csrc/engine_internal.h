// Host-side pieces shared by the handle API (engine.cpp) and the serving loop
// (serve.cpp): clause encoding, pass planning and launch of a planned pass.
#pragma once

#include <string>
#include <vector>

#include "qaa_internal.cuh"

namespace qaa {

// Clause c over literals l_1..l_k (Sec. 2.2) is violated exactly when every
// literal is false (Sec. 4.3 counts such clauses): (x & mask) == viol, with
// mask the bits of its variables and viol, per variable, the value that makes
// its literal false.  Returns 0, or a nonzero code with a message.
int encode_clauses(int n, const int32_t* lits, int m, std::vector<ClauseMV>& mv, std::vector<ClauseLP>& lp,
                   std::string& err);
// Clause c of lits (three signed literals) -> (mask, viol).
int encode_clause(int n, const int32_t* lits, int c, ClauseMV& out, std::string& err);
// The 1024-amplitude tile record of a clause (ClauseLP in qaa_internal.cuh).
ClauseLP clause_lp(const ClauseMV& mv);
// Every clause's tile record into a caller-provided array of m records.
int encode_clauses_lp(int n, const int32_t* lits, int m, ClauseLP* out, std::string& err);

constexpr int kRotationForm = 3;  // PassPlan::wht_kind of the rotation form

struct Group {
  int a, q, a2;  // active bits [a, a+5) and [a2, a2+q-5); a2 == a + 5 for a contiguous group
};

// How an n-qubit state is evolved: on chip (n <= 14) or by streaming passes.
struct PassPlan {
  int n = 0;
  bool onchip = false;
  bool use_tma = true;       // TMA-pipelined passes (QAA_PASSES=classic: plain loads)
  int wht_kind = 0;          // 0 FP32 butterflies, 1/2 tensor-core BF16x3/x2, 3 rotation form
  std::vector<Group> strided;  // ascending bit order
  int phase_group = 0;         // strided group whose pass fuses W B W
  std::vector<int> run_c;      // per strided group: 4 = 128-byte runs, 0 = default
  int low_bits = kLowBits;     // bits of the low pass: 10, or 12 (rotation form, kLpRot12)
};

// Plan for n: the one qaa_autotune chose for n on the current device, if any
// and if no tuning override is set in the environment; otherwise the default.
// max_q: widest strided group allowed (11 on the TMA FP32 passes; 10 for the
// plain-load and tensor-core passes, which have no 11-bit tiles).
void make_plan(int n, PassPlan& plan, int max_q = 11);
// Default plan for n, with the tuning overrides QAA_PASSES, QAA_SPLIT_GROUPS,
// QAA_PHASE_GROUP, QAA_RUN128_GROUPS, QAA_GROUP_BITS and QAA_LOW_BITS read
// from the environment.  low: bits of the low pass, 10 or 12 (12 only for the
// rotation form on TMA passes); 0 = QAA_LOW_BITS, else 10.
void make_default_plan(int n, PassPlan& plan, int max_q = 11, int low = 0);
// Run lengths per group for the plan's form (QAA_RUN128_GROUPS overrides).
void set_default_run_c(PassPlan& plan);
// A plan with a 12-bit low pass becomes the default plan with a 10-bit one
// (same form): for the W.B.W, tensor-core and plain-load passes.
void narrow_low_pass(PassPlan& plan, int max_q = 11);

// Autotuner support.  First-stage candidates for n >= 15: the default plan,
// then every split of bits 10..n-1 into the fewest groups of 5..11 bits (5..10
// without TMA; the fewest HBM round trips) with every choice of phase group;
// run lengths 128 B for plain groups and 64 B for the phase group; for
// n >= 31 on TMA passes, last, the rotation form with a 12-bit low pass.
void plan_candidates(int n, std::vector<PassPlan>& out);
// Contiguous groups of the given widths from bit 10 up.
void plan_with_groups(int n, const std::vector<int>& sizes, int phase_group, bool tma, PassPlan& plan);
void set_tuned_plan(const PassPlan& plan);  // record for (current device, plan.n)
bool tuned_plan(int n, PassPlan& out);
void clear_tuned_plans();

// Passes for steps c0 <= k < c1 of the range [k0, k1): P rows are relative to
// the chunk (row k + 1 - c0 ends step k), B rows likewise (row k - c0).
void build_passes(const PassPlan& plan, long long k0, long long k1, long long c0, long long c1,
                  std::vector<Pass>& out);

std::string describe_plan(const PassPlan& plan);

// Launch one pass with the kernel family the plan selects.  fold: kFoldBytes
// of device scratch for the norm fold of the low passes (null: no fold).
cudaError_t launch_planned_pass(const LaunchCtx& lc, const PassPlan& plan, const Pass& p, float2* psi, int m,
                                const ClauseLP* cl, const float2* ptab, const float2* btab, int* err,
                                const unsigned* counts = nullptr, double* fold = nullptr);

constexpr long long kChunkSteps = 1024;

// Device-driven evolution of a step range in one CUDA graph (graph.cpp): a
// WHILE conditional node whose body is kGraphUnroll Strang steps, with the
// phase rows of each iteration computed on the device.
constexpr int kGraphUnroll = 8;
struct GraphSpec {
  const PassPlan* plan = nullptr;
  float2* psi = nullptr;
  int m = 0;
  const ClauseLP* cl = nullptr;
  int* err = nullptr;  // bounded-wait error word of the TMA passes
  double dt = 0;
  const double* s_dev = nullptr;  // caller schedule on the device, or null for s_k = (k + 1/2)/K
  const double* dt_dev = nullptr;  // per-step lengths on the device, or null for the uniform dt
  const unsigned* counts = nullptr;  // stored per-tile clause counts (launch_lp_counts), or null
  double* fold = nullptr;            // norm-fold slots (kFoldBytes), or null
  long long K = 0, k0 = 0, k1 = 0;
  int num_sms = 0;
  // graph scratch (graph_scratch_bytes): loop counter, kGraphUnroll + 1 P rows, kGraphUnroll B rows
  long long* ctr = nullptr;
  float2* prow = nullptr;
  float2* brow = nullptr;
};
size_t graph_scratch_bytes(int n, int m);
void graph_scratch_split(void* base, int m, GraphSpec& s);
// Build and instantiate the graph for s (streaming plans only).  The graph
// reads and writes s.psi and the scratch; launch it on any stream.
cudaError_t build_evolve_graph(const GraphSpec& s, cudaGraphExec_t* out);

// Bytes of phase tables for a chunk of `chunk` steps.
inline size_t table_entries(int n, int m, long long chunk) {
  return static_cast<size_t>(chunk + 1) * static_cast<size_t>(m + 1) + static_cast<size_t>(chunk) * (n + 1);
}

}  // namespace qaa
