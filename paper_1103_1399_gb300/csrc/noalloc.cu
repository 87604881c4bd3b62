// qaa_observables_noalloc: the observables reduction without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Who needs this: code whose device memory is owned by someone else (a host
// framework's pooled allocator, a fixed budget reserved at start-up), and
// latency-critical loops in which cudaMalloc / cudaFree are unacceptable
// because they can synchronise the whole device.  Such callers cannot create a
// qaa_handle (qaa_create allocates the clause tables), so this entry point
// takes the clause list directly.
//
// Its scratch -- the encoded clause table, the per-block partial sums and the
// five results -- lives in one file-scope __device__ array of fixed size that
// every GPU which loads the library holds until the process exits.  Host code
// must not use the array's name as a device address; the address is taken
// once per device with cudaGetSymbolAddress (on the first call made with that
// device current) and passed to the kernels.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "engine_internal.h"
#include "qaa.h"

namespace {

constexpr size_t kResultBytes = 64;  // 5 doubles, then the bounded-wait error word at byte 48
constexpr size_t kPartialBytes = static_cast<size_t>(QAA_NOALLOC_MAX_PARTIALS) * sizeof(double);
constexpr size_t kClauseBytes = static_cast<size_t>(QAA_MAX_CLAUSES) * sizeof(qaa::ClauseLP);
constexpr size_t kScratchBytes = kResultBytes + kPartialBytes + kClauseBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Messages go to the same thread-local slot that qaa_last_error() reports.
qaa_status noalloc_fail(int code, const std::string& msg) {
  qaa::set_last_error(msg);
  return static_cast<qaa_status>(code);
}

}  // namespace

extern "C" qaa_status qaa_observables_noalloc(int n, const int32_t* clauses, int m, const void* psi, void* cuda_stream,
                                       qaa_obs* out) {
  if (!out) return noalloc_fail(QAA_E_ARG, "out is null");
  if (n < 1 || n > QAA_MAX_QUBITS) return noalloc_fail(QAA_E_ARG, "n out of range [1, 34]");
  if (m < 0 || m > QAA_MAX_CLAUSES)
    return noalloc_fail(QAA_E_ARG, "m exceeds the static clause capacity of " + std::to_string(QAA_MAX_CLAUSES));
  if (m > 0 && !clauses) return noalloc_fail(QAA_E_ARG, "clauses is null");
  if (!psi) return noalloc_fail(QAA_E_ARG, "psi is null");
  if (reinterpret_cast<uintptr_t>(psi) % 8u) return noalloc_fail(QAA_E_ARG, "psi must be 8-byte aligned");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return noalloc_fail(QAA_E_CUDA, "no CUDA device");
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(QAA_E_ARG, "device ordinal beyond the supported range");
  int num_sms = 0;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return noalloc_fail(QAA_E_CUDA, "cannot query SM count");
  const size_t parts = qaa::obs_partials_len(n, num_sms);
  if (parts > static_cast<size_t>(QAA_NOALLOC_MAX_PARTIALS))
    return noalloc_fail(QAA_E_ARG, "this device needs " + std::to_string(parts) +
                                       " partial sums, above the static capacity of " +
                                       std::to_string(QAA_NOALLOC_MAX_PARTIALS));

  // Once per device, with that device current: the array's device address.
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (err != cudaSuccess || !p)
        return noalloc_fail(QAA_E_CUDA, std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(err));
      g_scratch_addr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_scratch_addr[dev]);
  }
  double* d_result = reinterpret_cast<double*>(base);
  double* d_partials = reinterpret_cast<double*>(base + kResultBytes);
  qaa::ClauseLP* d_clauses = reinterpret_cast<qaa::ClauseLP*>(base + kResultBytes + kPartialBytes);

  // the handle's own encoding (plan.cpp), into a per-thread host table
  static thread_local qaa::ClauseLP host_table[QAA_MAX_CLAUSES];
  {
    std::string msg;
    const int st = qaa::encode_clauses_lp(n, clauses, m, host_table, msg);
    if (st) return noalloc_fail(st, msg);
  }

  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  if (m > 0) {
    const cudaError_t err = cudaMemcpyAsync(d_clauses, host_table, static_cast<size_t>(m) * sizeof(qaa::ClauseLP),
                                            cudaMemcpyHostToDevice, stream);
    if (err != cudaSuccess) return noalloc_fail(QAA_E_CUDA, std::string("clause upload: ") + cudaGetErrorString(err));
  }
  // Every partial slot and result the kernels read is written earlier in the
  // same call; only the error word must start at zero.
  int* d_errword = reinterpret_cast<int*>(base + 48);
  cudaError_t err = cudaMemsetAsync(d_errword, 0, sizeof(int), stream);
  if (err != cudaSuccess) return noalloc_fail(QAA_E_CUDA, std::string("error word: ") + cudaGetErrorString(err));
  const qaa::LaunchCtx lc{stream, num_sms};
  err = qaa::launch_observables(lc, static_cast<const float2*>(psi), n, m, d_clauses, d_partials, d_result, nullptr,
                                d_errword);
  if (err != cudaSuccess) return noalloc_fail(QAA_E_CUDA, std::string("observables: ") + cudaGetErrorString(err));
  double r[8];
  err = cudaMemcpyAsync(r, d_result, sizeof(r), cudaMemcpyDeviceToHost, stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
  if (err != cudaSuccess) return noalloc_fail(QAA_E_CUDA, std::string("result read-back: ") + cudaGetErrorString(err));
  int werr = 0;
  std::memcpy(&werr, reinterpret_cast<const unsigned char*>(r) + 48, sizeof(int));
  if (werr != 0) return noalloc_fail(QAA_E_TIMEOUT, "a bounded wait on a TMA copy expired in a correlation pass");
  out->norm = r[0];
  out->expect_hp = r[1];
  out->ground_prob = r[2];
  out->ground_count = static_cast<int64_t>(std::llround(r[3]));
  out->expect_hb = 0.5 * n * r[0] - r[4];
  return QAA_OK;
}
