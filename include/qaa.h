/*
 * qaa.h -- C ABI of the GB300 adiabatic 3-SAT state-vector evolver.
 *
 * What it computes (the paper's method, restated):
 *   Eq. (1)   H(s) = (1 - s) H_B + s H_P,  s = t / T, swept linearly over [0, 1].
 *   Sec. 2.1  H_B is the beginning Hamiltonian whose ground state is the uniform
 *             superposition; it is taken as H_B = sum_i (1 - sigma^x_i) / 2.
 *   Sec. 4.3  H_P is diagonal: E(x) = number of clauses that assignment x leaves
 *             unsatisfied (energy proportional to that count, constant 1).
 *   Sec. 2.2  A K-SAT clause is a disjunction of literals x_i / NOT x_i.
 * The state psi (2^n amplitudes, complex64 = interleaved float re, im) evolves by
 * K second-order Strang steps of dt = T / K, step k frozen at s_k = (k + 1/2)/K:
 *   exp(-i dt/2 s_k H_P) W exp(-i dt (1 - s_k) popcount) W exp(-i dt/2 s_k H_P),
 * W the normalised Walsh-Hadamard transform (H_B = W diag(popcount) W).  The
 * half phases of adjacent steps are merged and E(x) comes from the clause bit
 * masks, bit exact (counted inside the kernels, or stored once per instance as
 * per-tile bit-sliced counts).  By default exp(-i theta H_B) is applied as a
 * Walsh-Hadamard sandwich W diag(exp(-i theta popcount)) W on every 5-qubit
 * block inside each pass (H_B is a sum of commuting one-qubit terms); the
 * whole-register form (the popcount phase between two transforms of all n
 * qubits) and tensor-core transforms are variants (qaa_set_variant).
 *
 * Index convention (Sec. 2.1, basis |q_n ... q_1>): amplitude psi[x] belongs to
 * the assignment with x_i = bit (i - 1) of x.
 *
 * Conventions for every entry point:
 *   - Return a qaa_status (qaa_version, qaa_tune_candidates and
 *     qaa_last_error return a version, a count and a message); no C++
 *     exception ever crosses this boundary.  On a failure qaa_last_error()
 *     returns a message for the calling thread.
 *   - Device pointers (psi, out_dev) are caller-owned CUDA device memory on the
 *     current device; the library never frees or keeps them after the call.
 *     psi must hold 2^n complex64 values; the evolution calls need it 16-byte
 *     aligned (as every cudaMalloc / PyTorch allocation is), the read-only
 *     calls 8-byte aligned.
 *   - Work is enqueued on the handle's stream (qaa_set_stream; default: the
 *     legacy default stream).  Calls that return a host value synchronise that
 *     stream; the others are asynchronous with respect to the host.
 *   - A handle is not thread safe: use one handle per host thread, or serialise.
 */
#ifndef QAA_H
#define QAA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qaa_ctx* qaa_handle;

typedef enum {
  QAA_OK = 0,
  QAA_PENDING = 1,      /* serving: the request has not finished yet            */
  QAA_E_ARG = -1,       /* invalid argument (sizes, literals, null pointers)     */
  QAA_E_NOMEM = -2,     /* device memory (or the configured budget) exhausted    */
  QAA_E_CUDA = -3,      /* a CUDA runtime call failed; see qaa_last_error()      */
  QAA_E_TIMEOUT = -4,   /* a bounded device wait gave up                         */
  QAA_E_UNSAT = -5,     /* reserved: instance has no satisfying assignment       */
  QAA_E_STATE = -6      /* call not valid in the object's current state          */
} qaa_status;

/* Largest number of qubits / variables accepted (2^34 complex64 = 128 GiB). */
#define QAA_MAX_QUBITS 34
/* Largest clause count accepted (energies must fit the 10-bit in-kernel counters). */
#define QAA_MAX_CLAUSES 1023

/* Library version, for the binding's sanity check. */
int qaa_version(void);

/* Thread-local message describing the last failure on this thread (never NULL). */
const char* qaa_last_error(void);

/*
 * qaa_create -- build a handle for one K-SAT instance (Sec. 2.2) on the current
 * CUDA device.
 *   n        number of variables = qubits, 1 <= n <= QAA_MAX_QUBITS.
 *   clauses  host array of m * 3 int32: clause c is clauses[3c .. 3c+2], each a
 *            signed 1-based literal (+i = x_i, -i = NOT x_i) or 0 for an unused
 *            slot (clauses of width 1..3).  Copied; the pointer is not kept.
 *   m        number of clauses, 0 <= m <= QAA_MAX_CLAUSES (0 gives H_P = 0).
 * Errors: QAA_E_ARG for n or m out of range, a literal with |lit| > n, a clause
 * naming the same variable twice, or an all-zero clause; QAA_E_NOMEM/QAA_E_CUDA
 * if the device tables cannot be allocated.  Repeated clauses are allowed and
 * count with multiplicity in E(x).
 */
qaa_status qaa_create(int n, const int32_t* clauses, int m, qaa_handle* out);

/* Release the handle and its device tables.  NULL is accepted. */
qaa_status qaa_destroy(qaa_handle h);

/* Bind a cudaStream_t (as void*) for all later work of this handle; NULL = default
 * stream.  Switching to a different stream first waits for the handle's work on
 * the old one (the handle's device tables are reused across calls). */
qaa_status qaa_set_stream(qaa_handle h, void* cuda_stream);

/*
 * qaa_set_variant -- choose the Walsh-Hadamard implementation of the
 * streaming passes (n >= 15; the on-chip path for n <= 14 is always FP32).
 *   wht_kind 0: FP32 CUDA-core butterflies, the whole-register W.B.W form.
 *            1: the W.B.W form with every transform on the tensor cores
 *               (tcgen05): each group of <= 10 qubits in two 5-qubit stages,
 *               each a GEMM against the exact +-1 block H_32 on BF16 operands,
 *               the amplitude split into three BF16 parts (hi + mid + lo),
 *               FP32 accumulation in tensor memory: about FP32 accuracy.  Its
 *               low passes read the stored per-tile clause counts (see
 *               qaa_evolve), which the handle then keeps whatever
 *               QAA_LP_COUNTS says.
 *            2: as 1 with two parts (hi + lo): about 16 mantissa bits.
 *            3: rotation form (the default on the TMA passes): exp(-i theta H_B)
 *               applied directly as the product
 *               of its n one-qubit factors (H_B = sum_i (1 - sigma^x_i)/2 is a
 *               sum of commuting one-qubit terms, Sec. 2.1), each
 *               (|+><+| + e^(-i theta) |-><-|), as complex butterflies inside
 *               the same passes; no Walsh-Hadamard change of basis, so g HBM
 *               round trips per step instead of 2g - 2 (3 instead of 4 at
 *               n = 30).  Same Strang step, FP32 butterflies; needs the TMA
 *               passes (QAA_E_ARG otherwise).
 *   q        qubits per strided pass: 0 = automatic (the plan qaa_autotune
 *            recorded for n, else the default: the fewest groups of at most 11
 *            bits); 5..11 = the fewest strided groups of at most q bits each
 *            (the 10 low bits always form one pass; 11 needs the TMA FP32
 *            passes, the tensor-core variants stop at 10).
 * Returns QAA_E_ARG for an unknown kind, a q outside those ranges, or a q for
 * which the n - 10 strided bits have no split into groups of 5..q bits.
 */
qaa_status qaa_set_variant(qaa_handle h, int wht_kind, int q);

/*
 * qaa_autotune -- choose the pass plan of a streaming-size handle (n >= 15)
 * by timing candidates on the GPU.  Stage 1 times the default plan and every
 * split of bits 10..n-1 into the fewest strided groups of 5..10 bits (qubits
 * per pass) with every choice of the group that hosts the popcount phase;
 * stage 2 toggles the contiguous run per tile row (64 or 128 bytes) of each
 * group of >= 7 bits; stage 3 tries recombining two 10-bit groups; stage 4
 * plain loads instead of TMA; stage 5 the rotation form of the H_B factor
 * (variant 3, see qaa_set_variant) on the best plan so far, and if it wins,
 * the run-length toggles of stage 2 again.  A handle on a
 * tensor-core variant (1, 2) keeps it and skips stage 5.  Each candidate is timed with CUDA events as the
 * best of two runs of `steps` Strang steps (1..64) after one untimed run.
 * Stages stop once budget_ms of host time is spent (<= 0: 60 s); stage 1's
 * first candidate always runs.
 *   psi      device complex64[2^n], 16-byte aligned: scratch, overwritten
 *            (re-initialise it afterwards).
 *   report   optional (NULL allowed): one line per timed candidate, then the
 *            choice; truncated to len - 1 bytes.
 * The fastest plan becomes this handle's plan and is recorded for n on the
 * current device, form included: every later qaa_create and server request
 * with the same n in this process uses it (unless a QAA_* plan override is set
 * in the environment); qaa_set_variant still switches a handle's form.  Results of different plans agree within FP32 rounding (the
 * butterfly order differs).  Synchronous.  For n <= 14 there is nothing to
 * tune (QAA_OK, report says so).  The paper has no counterpart.
 */
qaa_status qaa_autotune(qaa_handle h, void* psi, int steps, double budget_ms, char* report, size_t len);

/* Number of stage-1 autotune candidates for n (0 for n <= 14), with their
 * descriptions one per line in buf (NULL allowed).  Needs no GPU. */
int qaa_tune_candidates(int n, char* buf, size_t len);

/*
 * qaa_lowest_eigenvalues -- the k lowest levels of H(s) = (1 - s) H_B + s H_P
 * (Eq. (1)) by Lanczos: the gap E1 - E0 bounds how slowly the evolution of
 * Sec. 2.1 must sweep s to stay in the ground state.
 *   start 0: from the uniform state, so only levels reachable from the initial
 *            state of the evolution appear (the relevant gap); at s = 0 that is
 *            the ground level alone.
 *   start 1: from a real random vector (splitmix64 of the index and `seed`):
 *            every level, each distinct level once.
 *   max_iter Lanczos iterations (2..4000), fewer if the Krylov space is
 *            exhausted; *iters (may be NULL) receives the count used.
 *   evals    host array of k doubles: the lowest levels found, ascending;
 *            *found = how many (<= k).
 * FP64 real vectors (three arrays of 2^n doubles, allocated by the handle on
 * first use; QAA_E_NOMEM if they do not fit), FP64 recurrence scalars and host
 * tridiagonal eigenvalues (Sturm bisection); repeated and spurious Ritz values
 * of finite-precision Lanczos are removed by the Cullum-Willoughby test
 * (levels closer than 1e-9 ||T|| count as one).
 * Synchronous.  QAA_E_ARG for k outside [1, 8], max_iter outside [2, 4000], a
 * start other than 0 / 1 or a non-finite s.  The paper has no counterpart
 * (it evolves without computing the spectrum).
 */
qaa_status qaa_lowest_eigenvalues(qaa_handle h, double s, int k, int max_iter, int start, uint64_t seed, double* evals,
                           int* found, int* iters);

/* Forget every plan recorded by qaa_autotune in this process. */
qaa_status qaa_forget_tuned_plans(void);

/*
 * qaa_set_launch_mode -- how qaa_evolve* issue the streaming passes (n >= 15;
 * the on-chip path for n <= 14 is one launch per chunk either way).
 *   QAA_LAUNCH_PASSES (0, default): one kernel launch per pass from the host.
 *   QAA_LAUNCH_GRAPH  (1): one CUDA graph per step range, launched once: a
 *     WHILE conditional node whose body is 8 Strang steps, the phase rows of
 *     each iteration computed on the device from the same FP64 formulas, so
 *     the result is the same bit for bit.  The graph is kept and relaunched
 *     while psi, T, steps, the range, the schedule pointer, the variant and the
 *     stream stay the same; any change rebuilds it (a stream synchronisation
 *     and a few hundred microseconds of host time).  The handle allocates a
 *     small device scratch (the loop counter and 8 steps of phase rows) on the
 *     first graph launch.  The integrator is the paper's Eq. (1) Hamiltonian
 *     split as in qaa_evolve; the paper has no launch-graph counterpart.
 * Returns QAA_E_ARG for an unknown mode.
 */
#define QAA_LAUNCH_PASSES 0
#define QAA_LAUNCH_GRAPH 1
qaa_status qaa_set_launch_mode(qaa_handle h, int mode);

/* psi[x] = 2^(-n/2) for all x: the ground state of H_B (Sec. 2.1).  Asynchronous. */
qaa_status qaa_init_uniform(qaa_handle h, void* psi);

/*
 * qaa_evolve -- evolve psi in place from s = 0 to s = 1 over total time T with
 * `steps` Strang steps (dt = T/steps), Eq. (1) with the linear sweep s = t/T.
 * T >= 0, steps >= 1.  Asynchronous on the handle's stream.
 * For n >= 15 on the TMA passes the handle stores, on the first evolution,
 * the bit-sliced violated-clause counts of every 1024-amplitude tile (as many
 * bit planes as the instance's largest count needs, at most 10: 1.25 bytes
 * per amplitude, 0.88 for the 30-qubit benchmark instance), allocated once at
 * the largest size (1.25 GiB at n = 30), so that later low passes read them
 * instead of counting again; if that memory cannot be allocated the passes
 * count on the fly (the same values).  QAA_LP_COUNTS=0 turns the store off.
 * Norm fold: the exact evolution is unitary, and the low passes measure the
 * FP32 state's norm (|psi|^2 summed in the pass, no extra read; every step for
 * n >= 26, every 2, 4 or 8 steps below) so that a later one scales its phase row
 * back to the norm psi had at the start of the call (times the exact power of
 * two of the unnormalised transforms): the norm stays within about 1e-7 of
 * its starting value instead of drifting with the roundings (about 4e-6
 * after 3200 steps at n = 20).
 */
qaa_status qaa_evolve(qaa_handle h, void* psi, double T, int64_t steps);

/*
 * qaa_evolve_range -- only steps k0 <= k < k1 of the `steps`-step run of
 * qaa_evolve (0 <= k0 <= k1 <= steps).  The half phases at both ends are
 * applied unmerged, so running [0, j) then [j, K) reproduces [0, K) up to
 * floating-point rounding: this is checkpoint / resume (psi plus k is the
 * whole state of a run).  k0 == k1 is a no-op.
 */
qaa_status qaa_evolve_range(qaa_handle h, void* psi, double T, int64_t steps, int64_t k0, int64_t k1);

/*
 * qaa_evolve_schedule -- general schedule: `steps` Strang steps of length dt,
 * step k frozen at s = s_values[k] (host array of `steps` doubles, each in any
 * real range; 0..1 for the interpolation of Eq. (1)).  Used for non-linear
 * sweeps and for frozen-s closed-form checks.
 */
qaa_status qaa_evolve_schedule(qaa_handle h, void* psi, double dt, const double* s_values, int64_t steps);

/*
 * qaa_evolve_substeps -- `count` Strang sub-steps of individual length:
 * sub-step j has length dt_values[j] (any finite real, negative = backwards in
 * time) with H frozen at s = s_values[j] (host arrays of `count` doubles,
 * copied before return).  Adjacent half phases are merged with their own
 * lengths: exp(-i (dt_j s_j + dt_(j+1) s_(j+1))/2 H_P).  Equal lengths give
 * exactly qaa_evolve_schedule.  Asynchronous on the handle's stream.
 * QAA_E_ARG for null arrays, count < 1 or a non-finite entry.
 */
qaa_status qaa_evolve_substeps(qaa_handle h, void* psi, const double* dt_values, const double* s_values, int64_t count);

/*
 * qaa_evolve_order4 -- the linear schedule s = t/T of Eq. (1) in `steps`
 * fourth-order steps: each step of length dt = T/steps is Yoshida's triple
 * jump (Phys. Lett. A 150, 262 (1990)) of Strang sub-steps w1 dt, w0 dt, w1 dt
 * with w1 = 1/(2 - 2^(1/3)), w0 = 1 - 2 w1 (< 0), each frozen at s of its own
 * midpoint time; 3 x steps sub-steps through qaa_evolve_substeps.  The error
 * falls as dt^4 instead of dt^2 (the paper names no integrator; this is a
 * higher-order alternative to the Strang split of qaa_evolve).
 * QAA_E_ARG for T < 0 or not finite, steps outside [1, 2^28].
 */
qaa_status qaa_evolve_order4(qaa_handle h, void* psi, double T, int64_t steps);

/*
 * Observables, accumulated in FP64 from the complex64 state with a fixed
 * two-level reduction order (bit-identical run to run).  Synchronous.
 *   norm         sum_x |psi_x|^2
 *   expect_hp    <H_P> = sum_x E(x) |psi_x|^2
 *   expect_hb    <H_B> = n/2 norm - 1/2 sum_i Re sum_x conj(psi_x) psi_(x ^ 2^(i-1))
 *   ground_prob  sum over E(x) = 0 of |psi_x|^2  (Sec. 2.1: ground manifold)
 *   ground_count number of assignments with E(x) = 0 (the instance's solutions)
 */
typedef struct {
  double norm;
  double expect_hp;
  double expect_hb;
  double ground_prob;
  int64_t ground_count;
} qaa_obs;

qaa_status qaa_observables(qaa_handle h, const void* psi, qaa_obs* out);

/* <H(s)> = (1 - s) <H_B> + s <H_P> of Eq. (1), FP64, synchronous. */
qaa_status qaa_energy(qaa_handle h, const void* psi, double s, double* out);

/* Ground-state probability sum_{E(x)=0} |psi_x|^2, FP64, synchronous. */
qaa_status qaa_success_prob(qaa_handle h, const void* psi, double* out);

/* sum_x |psi_x|^2, FP64, synchronous. */
qaa_status qaa_norm(qaa_handle h, const void* psi, double* out);

/*
 * qaa_hp_diagonal -- write E(x) for every x (2^n uint16 values, caller-owned
 * device memory, 2-byte aligned) using the same in-kernel clause evaluation as
 * the evolution.  Exposed for bit-exact checks.  Asynchronous.
 */
qaa_status qaa_hp_diagonal(qaa_handle h, uint16_t* out_dev);

/*
 * qaa_describe_plan -- write a one-line, NUL-terminated description of how this
 * handle evolves a state (on-chip, or the streaming pass plan: groups of index
 * bits, run lengths, passes per step, load path) into buf (len bytes,
 * truncated to fit).  Host only; no CUDA work.  A library addition: the paper
 * has no counterpart.
 */
qaa_status qaa_describe_plan(qaa_handle h, char* buf, size_t len);

/*
 * qaa_observables_noalloc -- the same five observables as qaa_observables,
 * for callers that cannot allocate device memory.  A library addition: the
 * paper has no counterpart.
 *
 * Some callers cannot call cudaMalloc: their device memory belongs to another
 * allocator (a host framework's memory pool, a budget fixed at start-up), or
 * they run latency-critical loops in which cudaMalloc / cudaFree are not
 * acceptable because those calls can synchronise the whole device.  Such a
 * caller cannot create a qaa_handle (qaa_create allocates its clause tables),
 * so this entry point takes the instance directly and allocates nothing:
 *   n, clauses, m  the instance, exactly as for qaa_create (host array);
 *   psi            the caller's device state (2^n complex64, 8-byte aligned);
 *   cuda_stream    stream to run on (NULL = default stream); synchronised
 *                  before returning;
 *   out            host result.
 * Its scratch (encoded clause table, per-block partial sums, results) is one
 * static device array of about 80 KiB that every GPU which loads this library
 * holds until the process exits.  Limits: m <= QAA_MAX_CLAUSES, and the
 * partial sums a call needs, (5 + ceil((n - 10) / 5)) x 2 x (SM count) for
 * n > 10, must not exceed QAA_NOALLOC_MAX_PARTIALS; larger requests return
 * QAA_E_ARG with a message in qaa_last_error().
 * The first call made on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The address is kept for the life of the process: after cudaDeviceReset on a
 * device this entry point must not be used on it again (the reset unloads the
 * module, and the kept address belongs to the old context).
 * All calls share the one array and it keeps the last call's contents: calls
 * whose work can overlap on the GPU (from several threads or streams) race and
 * must be serialised by the caller.
 */
#define QAA_NOALLOC_MAX_PARTIALS 8192
qaa_status qaa_observables_noalloc(int n, const int32_t* clauses, int m, const void* psi, void* cuda_stream,
                            qaa_obs* out);

/*
 * Serving: a loop that evolves requests of different n and T as they arrive.
 * A library addition built on the same kernels (the paper evolves one instance
 * at a time).  Requests keep their states resident in a device arena that the
 * server reserves once, are admitted when their memory block and a result slot
 * are free, run in continuous batches (every admitted request with n <= 14 in
 * one launch of the batched on-chip evolver; larger ones as streaming passes on
 * a pool of streams, overlapped), and report host-clock timestamps for latency.
 * Each request evolves from the uniform superposition over T with `steps`
 * Strang steps (as qaa_evolve) and returns the observables of the final state.
 * All functions are thread safe.
 */
typedef struct qaa_server qaa_server;

typedef struct {
  double success_prob;   /* sum over E(x) = 0 of |psi_x|^2                        */
  double energy;         /* <H_P> = <H(1)>                                         */
  double norm;           /* sum |psi_x|^2                                          */
  double expect_hb;      /* <H_B>                                                  */
  int64_t ground_count;  /* number of assignments with E(x) = 0                    */
  double t_submit;       /* seconds on the server's steady clock                   */
  double t_admit;        /* memory granted (-1 if never admitted)                  */
  double t_done;         /* results available                                      */
  double t_dev_start;    /* the request's device interval, seconds on the device's */
  double t_dev_end;      /* global timer since the server's creation (-1 if not    */
                         /* run): from a stamp before its first copy or kernel     */
                         /* (batched requests: the start of their CTA) to the end  */
                         /* of its observables' last kernel, on the stream it ran  */
                         /* on; overlapping intervals = requests in flight together */
  int n;
  int64_t steps;
  int status;            /* QAA_OK, QAA_E_STATE (cancelled), QAA_E_CUDA, QAA_E_TIMEOUT */
} qaa_result;

typedef struct {
  size_t arena_bytes;        /* device memory reserved for request states         */
  size_t peak_used_bytes;    /* largest amount of it in use at once               */
  int64_t batches;           /* on-chip batch launches                            */
  int64_t batched_requests;  /* requests run in those batches                     */
  int64_t streamed_requests; /* requests run as streaming passes                  */
} qaa_server_info;

/* hbm_budget_bytes: arena size (0 = free memory minus 4 GiB, at most 64 GiB);
 * max_slots: requests admitted at once (1..65536).  Starts the worker threads. */
qaa_status qaa_server_create(size_t hbm_budget_bytes, int max_slots, qaa_server** out);
/* Copies the instance (as qaa_create) and returns a ticket at once.  QAA_E_NOMEM
 * if the request can never fit in the arena; QAA_E_ARG for invalid input. */
qaa_status qaa_submit(qaa_server* s, int n, const int32_t* clauses, int m, double T, int64_t steps, uint64_t* ticket);
/* QAA_PENDING until done, then QAA_OK with *out filled (its status field tells
 * how the request ended).  Results stay available until the server is destroyed. */
qaa_status qaa_poll(qaa_server* s, uint64_t ticket, qaa_result* out);
/* Cancel a request not yet admitted (QAA_E_STATE once admitted). */
qaa_status qaa_cancel(qaa_server* s, uint64_t ticket);
qaa_status qaa_server_stats(qaa_server* s, qaa_server_info* out);
/* Fault injection for tests: fault 1 delays the worker thread by param
 * milliseconds once; fault 2 fails the next admitted request (status
 * QAA_E_CUDA) without touching the device; fault 3 starts the next persistent
 * request (15 <= n <= 17 by default) with a grid barrier that can never
 * complete: its CTAs give up after the barrier's bounded wait (about a second),
 * record the error and return, and the request ends with QAA_E_TIMEOUT while
 * the server and the device stay usable.  No fault traps or faults the GPU. */
qaa_status qaa_server_inject(qaa_server* s, int fault, int param);
/* Finishes running requests, cancels queued ones, releases everything. */
qaa_status qaa_server_destroy(qaa_server* s);

/*
 * Launch profiling (tracing).  When enabled, the handle records a pair of CUDA
 * events on its stream around every kernel it launches and accumulates, per
 * kernel kind, the number of launches and their summed device time.
 * qaa_profile_read synchronises the stream, folds in every pending pair and
 * reports the totals since the last reset.  Event recording adds a few
 * microseconds of stream work per launch.
 */
typedef enum {
  QAA_K_LOW_FIRST = 0,     /* low pass: P then W over bits 0..9            */
  QAA_K_LOW_MERGE = 1,     /* low pass: W, merged P, W                      */
  QAA_K_LOW_LAST = 2,      /* low pass: W then P                            */
  QAA_K_STRIDED = 3,       /* strided group pass: W                         */
  QAA_K_STRIDED_PHASE = 4, /* top group pass: W, popcount phase, W          */
  QAA_K_TABLES = 5,        /* FP64 phase-table generation                   */
  QAA_K_ONCHIP = 6,        /* whole-run on-chip evolver (n <= 14)           */
  QAA_K_OBSERVE = 7,       /* observable reductions (all kernels of a call) */
  QAA_K_DIAG = 8,          /* E(x) export                                   */
  QAA_K_INIT = 9,          /* uniform-state initialisation                  */
  QAA_K_GRAPH = 10,        /* one launch-graph evolve (all its passes)      */
  QAA_K_COUNT = 11
} qaa_kernel_kind;

qaa_status qaa_profile_enable(qaa_handle h, int on);
qaa_status qaa_profile_reset(qaa_handle h);
/* kind in [0, QAA_K_COUNT); launches and total_ms may be NULL.  Synchronous. */
qaa_status qaa_profile_read(qaa_handle h, int kind, int64_t* launches, double* total_ms);

#ifdef __cplusplus
}
#endif

#endif /* QAA_H */
