// Lanczos on H(s) = (1 - s) H_B + s H_P (Eq. (1)) for the lowest levels: the
// gap the adiabatic evolution of Sec. 2.1 must respect.
//
// H is real symmetric, so the Lanczos vectors are real; they are kept in FP64
// (8 bytes per amplitude, like a complex64 state), so loss of orthogonality
// and the end of the Krylov space show at the 1e-12 level.  One iteration is
// five launches and no host synchronisation: the recurrence scalars alpha_j,
// beta_j live in device memory, written by fixed-order FP64 reductions and
// read by the next kernels.
//   apply : w = H v, with H_B v = (n/2) v - 1/2 sum_i v(x ^ 2^(i-1)) gathered
//           directly (coalesced per warp for every i) and H_P v = E v from the
//           exported diagonal; FP64 partials of <v, w>
//   reduce: alpha_j
//   update: w -= alpha_j v + beta_j v_prev; FP64 partials of |w|^2
//   reduce: beta_(j+1) = sqrt
//   scale : v_next = w / beta_(j+1) (zero after a breakdown)
#include <cstdint>

#include "qaa_internal.cuh"

namespace qaa {

namespace {

constexpr int kLzThreads = 256;

__device__ __forceinline__ double lz_block_sum(double v, double* s_red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += s_red[w];
  return t;
}

// splitmix64: a counter-based generator (Steele, Lea, Flood 2014), used for a
// reproducible random start vector.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void __launch_bounds__(kLzThreads) lz_start_kernel(double* __restrict__ v, unsigned long long N, int random,
                                                              unsigned long long seed) {
  for (unsigned long long x = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x; x < N;
       x += static_cast<unsigned long long>(gridDim.x) * blockDim.x) {
    double r = 1.0;
    if (random) {
      const unsigned long long h = splitmix64(seed ^ splitmix64(x));
      r = static_cast<double>(h >> 11) * 0x1.0p-53 * 2.0 - 1.0;
    }
    v[x] = r;
  }
}

__global__ void __launch_bounds__(kLzThreads)
    lz_apply_kernel(double* __restrict__ w, const double* __restrict__ v, const uint16_t* __restrict__ E, int n,
                    unsigned long long N, double a_hb, double a_hp, double* __restrict__ partials) {
  __shared__ double s_red[kLzThreads / 32];
  double acc = 0.0;
  for (unsigned long long x = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x; x < N;
       x += static_cast<unsigned long long>(gridDim.x) * blockDim.x) {
    const double c = v[x];
    double sum = 0.0;
    for (int i = 0; i < n; ++i) sum += v[x ^ (1ull << i)];
    const double h = a_hb * (0.5 * n * c - 0.5 * sum) + a_hp * static_cast<double>(E[x]) * c;
    w[x] = h;
    acc += c * h;
  }
  const double t = lz_block_sum(acc, s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kLzThreads)
    lz_dot_kernel(const double* __restrict__ a, const double* __restrict__ b, unsigned long long N,
                  double* __restrict__ partials) {
  __shared__ double s_red[kLzThreads / 32];
  double acc = 0.0;
  for (unsigned long long x = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x; x < N;
       x += static_cast<unsigned long long>(gridDim.x) * blockDim.x)
    acc += a[x] * b[x];
  const double t = lz_block_sum(acc, s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// out = sum of the partials (fixed order), or its square root.
__global__ void __launch_bounds__(kLzThreads) lz_reduce_kernel(const double* __restrict__ partials, int np,
                                                               double* __restrict__ out, int take_sqrt) {
  __shared__ double s_red[kLzThreads / 32];
  double t = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) t += partials[i];
  t = lz_block_sum(t, s_red);
  if (threadIdx.x == 0) *out = take_sqrt ? sqrt(t > 0.0 ? t : 0.0) : t;
}

__global__ void __launch_bounds__(kLzThreads)
    lz_update_kernel(double* __restrict__ w, const double* __restrict__ v, const double* __restrict__ vp,
                     const double* __restrict__ alpha, const double* __restrict__ beta, unsigned long long N,
                     double* __restrict__ partials) {
  __shared__ double s_red[kLzThreads / 32];
  const double a = *alpha, b = *beta;
  double acc = 0.0;
  for (unsigned long long x = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x; x < N;
       x += static_cast<unsigned long long>(gridDim.x) * blockDim.x) {
    const double r = w[x] - a * v[x] - b * vp[x];
    w[x] = r;
    acc += r * r;
  }
  const double t = lz_block_sum(acc, s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kLzThreads) lz_scale_kernel(double* __restrict__ dst, const double* __restrict__ src,
                                                              const double* __restrict__ beta, unsigned long long N) {
  const double b = *beta;
  const double inv = b > 1e-300 ? 1.0 / b : 0.0;
  for (unsigned long long x = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x; x < N;
       x += static_cast<unsigned long long>(gridDim.x) * blockDim.x)
    dst[x] = src[x] * inv;
}

}  // namespace

int lanczos_partials(int num_sms) { return 4 * num_sms; }

cudaError_t launch_lanczos(const LaunchCtx& lc, const LanczosArgs& a, int* done_iters) {
  const unsigned long long N = 1ull << a.n;
  const int P = lanczos_partials(lc.num_sms);
  long long g = static_cast<long long>((N + kLzThreads - 1) / kLzThreads);
  const unsigned grid = static_cast<unsigned>(g < P ? g : P);
  // start vector, normalised; beta[0] = 0 and v_prev = 0
  lz_start_kernel<<<grid, kLzThreads, 0, lc.stream>>>(a.vp, N, a.random_start, a.seed);
  lz_dot_kernel<<<grid, kLzThreads, 0, lc.stream>>>(a.vp, a.vp, N, a.partials);
  lz_reduce_kernel<<<1, kLzThreads, 0, lc.stream>>>(a.partials, static_cast<int>(grid), a.beta, 1);
  lz_scale_kernel<<<grid, kLzThreads, 0, lc.stream>>>(a.v, a.vp, a.beta, N);
  cudaError_t e = cudaMemsetAsync(a.vp, 0, N * sizeof(double), lc.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.beta, 0, sizeof(double), lc.stream);
  if (e != cudaSuccess) return e;
  double *v = a.v, *vp = a.vp, *w = a.w;
  for (int j = 0; j < a.iters; ++j) {
    lz_apply_kernel<<<grid, kLzThreads, 0, lc.stream>>>(w, v, a.E, a.n, N, 1.0 - a.s, a.s, a.partials);
    lz_reduce_kernel<<<1, kLzThreads, 0, lc.stream>>>(a.partials, static_cast<int>(grid), a.alpha + j, 0);
    lz_update_kernel<<<grid, kLzThreads, 0, lc.stream>>>(w, v, vp, a.alpha + j, a.beta + j, N, a.partials);
    lz_reduce_kernel<<<1, kLzThreads, 0, lc.stream>>>(a.partials, static_cast<int>(grid), a.beta + j + 1, 1);
    // v_prev's buffer receives the next v; rotate (v_prev <- v, v <- next)
    lz_scale_kernel<<<grid, kLzThreads, 0, lc.stream>>>(vp, w, a.beta + j + 1, N);
    double* t = vp;
    vp = v;
    v = t;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  *done_iters = a.iters;
  return cudaGetLastError();
}

}  // namespace qaa
