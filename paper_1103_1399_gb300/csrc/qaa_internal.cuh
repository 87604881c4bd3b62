// Internal declarations shared by the kernels and the host engine.
//
// Data layout in HBM: the state is one caller-owned array of 2^n complex64
// (float2, re/im interleaved), psi[x] for the assignment x (x_i = bit i-1).
// Clause tables live in device memory owned by the handle:
//   ClauseMV  : {mask, viol} 64-bit pair; clause c is violated by x iff
//               (x & mask) == viol  (mask = its variables, viol = the value of
//               each that makes the literal false).  Sec. 2.2 / Sec. 4.3.
//   ClauseLP  : the same clause split for a 1024-amplitude tile (bits 0..9):
//               hi_mask/hi_viol over bits >= 10 (shifted down by 10), and two
//               32-bit truth tables pat0 / pat5: bit j of pat0 is set iff the
//               clause's literals on bits 0..4 are all false when those bits
//               equal j (all ones if the clause has none there); pat5 likewise
//               for bits 5..9.  Violated(x) = hi part false AND pat0 bit
//               (x & 31) AND pat5 bit ((x >> 5) & 31).
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

namespace qaa {

struct __align__(16) ClauseMV {
  unsigned long long mask;
  unsigned long long viol;
};

struct __align__(16) ClauseLP {
  unsigned hi_mask;
  unsigned hi_viol;
  unsigned pat0;
  unsigned pat5;
};

// Low-pass tile: bits 0..9 of the index, 1024 amplitudes, one warp.
constexpr int kLowBits = 10;
constexpr int kLowTile = 1 << kLowBits;

// In-register bit-sliced counters hold up to 10 bits (QAA_MAX_CLAUSES = 1023).
constexpr int kPlanes = 10;
constexpr int QAA_MAX_CLAUSES_DEV = 1023;

// ---- pass descriptors -------------------------------------------------------
enum PassKind : int {
  kLpFirst = 0,  // psi <- W_G1 P(row) psi                 (first pass of a range)
  kLpMerge = 1,  // psi <- W_G1 P(row) W_G1 psi            (step boundary, merged)
  kLpLast = 2,   // psi <- P(row) W_G1 psi                 (last pass of a range)
  kSpW = 3,      // psi <- W_G psi over a strided group G
  kSpWBW = 4,    // psi <- W_G B(row) W_G psi over the phase group
  // Rotation form of exp(-i theta H_B) (variant 3): a product of one-qubit
  // rotations, applied group by group, no change of basis.  TMA passes only.
  kLpPhase = 5,  // psi <- P(prow) psi                     (first pass of a range)
  kLpRot = 6,    // psi <- 2^-n P(prow) R_G1(brow) psi     (ends every step)
  kSpRot = 7,    // psi <- R_G(brow) psi over a strided group (unnormalised by 2^q)
  kLpRot12 = 8,  // kLpRot over bits 0..11: four 1024-amplitude tiles per warp quad
};

struct Pass {
  int kind;
  int a;      // strided passes: index bit of the group's lowest 5 active bits
  int q;      // active bits (strided passes)
  int prow;   // phase-table row for P (low passes)
  int run_c;  // strided passes: 4 = 128-byte contiguous runs per tile row, 0 = default
  int brow;   // popcount-phase row (kSpWBW)
  int a2;     // strided passes: index bit of active bits 5..q-1 (a + 5 for a contiguous group)
  // low passes: the step this pass ends, counted from the start of the range
  // (-1 for the first pass of a range, -2 for no norm fold); selects the
  // norm-fold slots below
  int rel = -2;
};

// ---- norm fold ---------------------------------------------------------------
// The exact evolution is unitary, but the FP32 state's norm performs a random
// walk of roundings (about 4e-6 after 3200 Strang steps at 20 qubits, most of it
// from the rounding of the few large amplitudes, so that the ground-state
// probability drifts with it).  A low pass therefore also sums |psi|^2 of its
// output (FP32 per 1024-amplitude tile, double-float FP32 pairs beyond -- an
// FP32 sum and its exact rounding error -- one partial per CTA), and the next
// one multiplies its P row by
//   c = sqrt(N_ref 2^j / N),
// N that sum, N_ref the sum taken by the first pass of the range and 2^j the
// power of two nearest to N / N_ref (the unnormalised Walsh-Hadamard stages and
// the 2^-n factor scale the norm by exact powers of two between passes).  Each
// correction restores the norm the range started with up to the rounding of
// the steps since the last one, so the corrections do not accumulate.  When
// the state has concentrated on a few amplitudes the norm's error is mostly
// theirs, so the correction also takes out most of their magnitude error.
// Period F (fold_period): a fold costs a few microseconds per low pass (the
// partials' reads and sums at its start, the per-tile sums, the block sum at
// its end; 3.6 us per step measured at n = 22), and the norm drifts by about
// 1e-7 per step from the phase tables' magnitude errors.  So F = 1 from
// n = 26 (steps of 0.5 ms and more: under 1 %), 2 at n = 24..25, 4 at
// n = 22..23 and 8 below, where steps last microseconds; F divides 8, so the
// launch-graph bodies of 8 steps stay uniform.
// Slots of kFoldSlot float pairs: [0].x = number of partials (integer bits),
// then one (sum, error) pair per CTA.  Slot 0 holds the range's reference;
// F = 1 alternates slots 1 and 2 by step parity (a pass reads one and writes
// the other), F > 1 uses slot 1 (written by step r when F divides r + 1, read
// by step r + 1).  All of it is FP32 arithmetic: GB300's FP64 rate is a small
// fraction of its FP32 rate, and the scalar FP64 work of an earlier version
// (sums, log2, sqrt on one thread) cost microseconds per pass.
constexpr int kFoldSlot = 2048;
constexpr size_t kFoldBytes = 3 * kFoldSlot * sizeof(float2);
__host__ __device__ inline int fold_period(int n) { return n >= 26 ? 1 : n >= 24 ? 2 : n >= 22 ? 4 : 8; }
struct NormFold {
  float2* out = nullptr;         // slot this launch writes (null: none)
  float2* out2 = nullptr;        // a second slot written with the same partials
  const float2* ref = nullptr;   // the range's reference slot (null: no correction)
  const float2* prev = nullptr;  // the slot of the step to correct for
};
// Slots of a low pass with relative step p.rel and period F: the first pass
// writes the reference and the slot step 0 reads (so that step 0's correction
// is exactly 1); step r reads when r is a multiple of F and measures when
// r + 1 is.
__host__ __device__ inline NormFold fold_for(double* slots, const Pass& p, int F) {
  NormFold f;
  if (!slots || p.rel < -1) return f;
  float2* base = reinterpret_cast<float2*>(slots);
  float2* s1 = base + kFoldSlot;
  float2* s2 = base + 2 * kFoldSlot;
  if (p.rel == -1) {
    f.out = base;
    f.out2 = F == 1 ? s2 : s1;
    return f;
  }
  if (F == 1) {
    f.ref = base;
    f.prev = (p.rel & 1) ? s1 : s2;
    f.out = (p.rel & 1) ? s2 : s1;
    return f;
  }
  if (p.rel % F == 0) {
    f.ref = base;
    f.prev = s1;
  }
  if ((p.rel + 1) % F == 0) f.out = s1;
  return f;
}

// ---- kernel launchers (defined in the .cu files) ----------------------------
struct LaunchCtx {
  cudaStream_t stream;
  int num_sms;
};

cudaError_t launch_init_uniform(const LaunchCtx& lc, float2* psi, int n);
// Phase tables for steps c0 <= k < c1 of the range [k0, k1) of a K-step run:
// c1-c0+1 P rows of m+1 entries and c1-c0 B rows of n+1 entries.
// rot: B rows in the rotation form's layout (entries q = 0..6 = exp(-i dt (1 - s_k) q), unscaled).
// dt_dev: per-step lengths (device, K entries) instead of the uniform dt.
cudaError_t launch_tables(const LaunchCtx& lc, float2* ptab, float2* btab, int n, int m, double dt,
                          const double* s_dev, long long K, long long k0, long long k1, long long c0, long long c1,
                          bool rot = false, const double* dt_dev = nullptr);
cudaError_t launch_pass(const LaunchCtx& lc, const Pass& p, float2* psi, int n, int m,
                        const ClauseLP* cl, const float2* ptab, const float2* btab, const NormFold& nf = NormFold());
// Launch-graph helpers: phase rows from the same entry functions as
// launch_tables (P positions p_first + j -> rows dst_p0 + j, B steps k_first + j
// -> rows j, both offset by *ctr when ctr is non-null), and the loop-body tail
// that advances *ctr by `step` and sets the WHILE condition to *ctr < limit.
cudaError_t launch_graph_rows(const LaunchCtx& lc, float2* prow, int dst_p0, long long p_first, int nprow, float2* brow,
                              long long k_first, int nbrow, const long long* ctr, int n, int m, double dt,
                              const double* s_dev, long long K, long long k0, long long k1, bool rot = false,
                              const double* dt_dev = nullptr);
cudaError_t launch_graph_advance(const LaunchCtx& lc, long long* ctr, long long step, long long limit,
                                 cudaGraphConditionalHandle h);
// n <= kOnchipMaxBits: the whole state stays in one CTA's shared memory for
// `nsteps` steps.  P row j (j = 0..nsteps) and B row j (j < nsteps) as produced
// by launch_tables; first_p = apply P row 0 before the first transform.
constexpr int kOnchipMaxBits = 14;
cudaError_t launch_onchip(const LaunchCtx& lc, float2* psi, int n, int m, const ClauseMV* cl,
                          const float2* ptab, const float2* btab, int nsteps, bool first_p);
size_t onchip_smem_bytes(int n, int m);
// Batched on-chip evolution: one CTA per job, dynamic shared memory = the
// largest onchip_smem_bytes of the batch.  jobs_dev is a device array.
struct OnchipJob {
  float2* psi;
  const ClauseMV* cl;
  const float2* ptab;
  const float2* btab;
  int n, m, nsteps, first_p;
  int init;        // nonzero: start from the uniform superposition instead of reading psi
  float init_val;  // that amplitude, 2^(-n/2) rounded to FP32 on the host
  unsigned long long* stamp;  // if not null: the device time at the job's start (global_ns)
};
cudaError_t launch_onchip_batch(const LaunchCtx& lc, const OnchipJob* jobs_dev, int njobs, size_t smem_bytes);
cudaError_t launch_hp_diag(const LaunchCtx& lc, uint16_t* out, int n, int m, const ClauseLP* cl);
// Observables: partials has room for obs_partials_len(n) doubles; result is 5 doubles
// {norm, <H_P>, ground_prob, ground_count, sum of pair correlations} on the device.
size_t obs_partials_len(int n, int num_sms);
// counts (optional): the stored per-tile clause counts of launch_lp_counts.
// err: the bounded-wait error word of the TMA correlation passes.
cudaError_t launch_observables(const LaunchCtx& lc, const float2* psi, int n, int m,
                               const ClauseLP* cl, double* partials, double* result,
                               const unsigned* counts = nullptr, int* err = nullptr,
                               unsigned long long* stamp = nullptr);
// One thread writes the device's nanosecond timer to *stamp (the start of a
// served request's device interval; the observables' last kernel writes its end).
cudaError_t launch_stamp(const LaunchCtx& lc, unsigned long long* stamp);
// Read-only TMA pass: pair correlations of the index bits [a, a+5) and
// [a2, a2+q-5) (a2 = a + 5: contiguous; 5 <= q <= 10), one partial per CTA in
// partials[0 .. nparts).
cudaError_t launch_corr_tma(const LaunchCtx& lc, const float2* psi, int n, int a, int a2, int q, double* partials,
                            int nparts, int* err);

// TMA-pipelined variants of the streaming passes (tma_kernels.cu).  err is a
// device word set to nonzero when a bounded wait expires.  psi must be 16-byte
// aligned.
bool tma_available();
// counts (optional): the stored per-tile violated-clause counts of
// launch_lp_counts, read by the merged low passes instead of counting again.
// Bytes per contiguous tile row of a q-bit TMA strided pass (run_c as in Pass).
int tma_run_bytes(int q, int run_c);
cudaError_t launch_pass_tma(const LaunchCtx& lc, const Pass& p, float2* psi, int n, int m, const ClauseLP* cl,
                            const float2* ptab, const float2* btab, int* err, const unsigned* counts = nullptr,
                            const NormFold& nf = NormFold());
// Per-tile bit-sliced violated-clause counts of every 1024-amplitude tile
// (lp_counts_bytes(n) bytes), computed once per instance.
size_t lp_counts_bytes(int n);
cudaError_t launch_lp_counts(const LaunchCtx& lc, unsigned* counts, int n, int m, const ClauseLP* cl);

// Tensor-core variant (tc_kernels.cu): the Walsh-Hadamard transforms of every
// streaming pass of the W.B.W form as 5-bit stages of tcgen05 GEMMs against
// H_32 on BF16-split operands (parts = 3: hi + mid + lo, parts = 2: hi + lo)
// with FP32 accumulation in tensor memory.  The low passes need n >= 13 and
// the stored per-tile counts; err is the bounded-wait error word.
cudaError_t launch_pass_tc(const LaunchCtx& lc, const Pass& p, float2* psi, int n, int m, const ClauseLP* cl,
                           const float2* ptab, const float2* btab, int parts, int* err, const unsigned* counts,
                           const NormFold& nf = NormFold());
size_t tc_smem_bytes(int parts);

// Persistent evolution of one instance with 15 <= n <= 24 in one cooperative
// launch (persist.cu): every pass of every step inside the kernel, separated by
// a bounded grid barrier (bar: two zeroed words).  Tables for the whole run
// (K + 1 P rows, K B rows).  Contiguous strided groups only.
constexpr int kPersistMaxBits = 24;
struct PersistPlan {
  int ng, phase_group;
  int ga[3], gq[3];
};
cudaError_t launch_persist(const LaunchCtx& lc, const PersistPlan& pp, float2* psi, int n, int m, const ClauseLP* cl,
                           const float2* ptab, const float2* btab, int K, unsigned* bar, int* err, int grid,
                           double* fold = nullptr);

// Lanczos on H(s) (lanczos.cu): `iters` iterations from the uniform state or a
// seeded random real vector; alpha[0..iters), beta[0..iters] (beta[0] = 0) in
// device memory.  v, vp, w: 2^n real FP64 each; E: the exported H_P diagonal;
// partials: lanczos_partials(num_sms) doubles.
struct LanczosArgs {
  int n = 0;
  double s = 0;
  int iters = 0;
  int random_start = 0;
  unsigned long long seed = 0;
  const uint16_t* E = nullptr;
  double *v = nullptr, *vp = nullptr, *w = nullptr;
  double* partials = nullptr;
  double* alpha = nullptr;
  double* beta = nullptr;
};
int lanczos_partials(int num_sms);
cudaError_t launch_lanczos(const LaunchCtx& lc, const LanczosArgs& a, int* done_iters);

// Raise a kernel's dynamic shared-memory limit to `bytes` (its worst case over
// every instance the library accepts) once per device.  Launches then request
// only what they need; a per-launch limit would race between threads that
// launch the same kernel with different sizes.
cudaError_t allow_smem(const void* func, size_t bytes);

// Store a message for qaa_last_error() on the calling thread.
void set_last_error(const std::string& msg);

}  // namespace qaa
