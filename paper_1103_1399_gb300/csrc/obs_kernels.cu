// Read-only kernels: the exported H_P diagonal and the FP64 observables.
//
// Observables (ground state and its probability: Sec. 2.1; the result gathered
// from every thread and returned to the host: Sec. 4.2):
//   norm = sum |psi|^2, <H_P> = sum E |psi|^2, ground = sum_{E=0} |psi|^2,
//   count of E = 0, and C = sum_i sum_{x: bit i-1 clear} Re(conj psi_x psi_(x+2^(i-1)))
//   from which <H_B> = n/2 norm - C.
// norm, <H_P> and the ground probability: every product formed in FP64 from
// the FP32 amplitudes (exact) and summed in FP64.  The pair correlations C
// (n pair products per amplitude, the bulk of the arithmetic) are formed and
// summed in FP32 over one thread's share of one tile or column (at most 320
// products) and accumulated in FP64 beyond that: GB300's FP64 rate is a small
// fraction of its FP32 rate, and with FP64 pair products the reductions ran at
// ~2% of the HBM bound.  The FP32 stage adds at most ~320 ulp of the largest
// product to each partial; independent partials average out in the FP64 sum.
// Every sum runs in a fixed order (per thread, a fixed shuffle/shared-memory
// tree per block, the partials by one block): bit-identical run to run.
#include "device_common.cuh"

namespace qaa {

constexpr int kObsWarps = 8;
constexpr int kObsQuant = 5;  // norm, hp, ground, count, corr(low bits)

static size_t obs_low_smem(int m) {
  return 16u * static_cast<size_t>(m) + static_cast<size_t>(kObsWarps) * 8u * static_cast<size_t>(m + 16) + 64u * 8u;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block reduction of one double per thread; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* s_red) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += s_red[w];
  }
  return t;
}

__global__ void __launch_bounds__(kObsWarps * 32)
    diag_kernel(uint16_t* __restrict__ out, int n, int m, const ClauseLP* __restrict__ cl, long long ntiles) {
  extern __shared__ __align__(16) unsigned char smem[];
  ClauseLP* s_cl = reinterpret_cast<ClauseLP*>(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint2* s_act = reinterpret_cast<uint2*>(smem + 16u * m) + warp * (m + 16);
  for (int i = threadIdx.x; i < m; i += blockDim.x) s_cl[i] = cl[i];
  __syncthreads();
  const unsigned long long N = 1ull << n;
  for (long long tile = static_cast<long long>(blockIdx.x) * kObsWarps + warp; tile < ntiles;
       tile += static_cast<long long>(gridDim.x) * kObsWarps) {
    int nconst, npad;
    __syncwarp();
    fold_tile<false>(s_cl, m, static_cast<unsigned>(tile), lane, s_act, nconst, npad);
    int e[32];
    energies(e, s_act, npad, nconst, 1u << lane);
    const unsigned long long base = static_cast<unsigned long long>(tile) << kLowBits;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const unsigned long long x = base + lane + 32 * r;
      if (x < N) out[x] = static_cast<uint16_t>(e[r]);
    }
  }
}

__global__ void __launch_bounds__(kObsWarps * 32)
    obs_low_kernel(const float2* __restrict__ psi, int n, int m, const ClauseLP* __restrict__ cl, long long ntiles,
                   double* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char smem[];
  ClauseLP* s_cl = reinterpret_cast<ClauseLP*>(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint2* s_act = reinterpret_cast<uint2*>(smem + 16u * m) + warp * (m + 16);
  double* s_red = reinterpret_cast<double*>(smem + 16u * m + static_cast<size_t>(kObsWarps) * 8u * (m + 16));
  for (int i = threadIdx.x; i < m; i += blockDim.x) s_cl[i] = cl[i];
  __syncthreads();
  const unsigned long long N = 1ull << n;
  double a_norm = 0.0, a_hp = 0.0, a_gp = 0.0, a_gc = 0.0, a_corr = 0.0;
  for (long long tile = static_cast<long long>(blockIdx.x) * kObsWarps + warp; tile < ntiles;
       tile += static_cast<long long>(gridDim.x) * kObsWarps) {
    const unsigned long long base = static_cast<unsigned long long>(tile) << kLowBits;
    float2 v[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const unsigned long long x = base + lane + 32 * r;
      v[r] = x < N ? psi[x] : make_float2(0.0f, 0.0f);
    }
    int nconst, npad;
    __syncwarp();
    fold_tile<false>(s_cl, m, static_cast<unsigned>(tile), lane, s_act, nconst, npad);
    int e[32];
    energies(e, s_act, npad, nconst, 1u << lane);
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const double re = v[r].x, im = v[r].y;
      const double p = fma(re, re, im * im);
      a_norm += p;
      a_hp = fma(static_cast<double>(e[r]), p, a_hp);
      const bool valid = base + lane + 32 * r < N;
      if (e[r] == 0 && valid) {
        a_gp += p;
        a_gc += 1.0;
      }
    }
    float f_corr = 0.f;
    // pairs across register bits (index bits 5..9)
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      if (5 + b < n) {
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          if (!(r & (1 << b))) {
            const float2 u = v[r], w = v[r | (1 << b)];
            f_corr = fmaf(u.x, w.x, f_corr);
            f_corr = fmaf(u.y, w.y, f_corr);
          }
        }
      }
    }
    // pairs across lanes (index bits 0..4)
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      if (b < n) {
        const float keep = (lane & (1 << b)) ? 0.f : 1.f;  // count each pair once
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const float wx = __shfl_xor_sync(0xffffffffu, v[r].x, 1 << b);
          const float wy = __shfl_xor_sync(0xffffffffu, v[r].y, 1 << b);
          f_corr = fmaf(keep * v[r].x, wx, f_corr);
          f_corr = fmaf(keep * v[r].y, wy, f_corr);
        }
      }
    }
    a_corr += static_cast<double>(f_corr);
  }
  const double q[kObsQuant] = {a_norm, a_hp, a_gp, a_gc, a_corr};
#pragma unroll
  for (int k = 0; k < kObsQuant; ++k) {
    const double t = block_sum(q[k], s_red);
    if (threadIdx.x == 0) partials[static_cast<size_t>(k) * gridDim.x + blockIdx.x] = t;
  }
}

// Pair correlations for index bits [a, a+w) (a >= 10, w <= 5): one thread per
// column (the other index bits), coalesced over the low bits.
__global__ void __launch_bounds__(256)
    corr_kernel(const float2* __restrict__ psi, int a, int w, long long ncols, double* __restrict__ partials) {
  __shared__ double s_red[32];
  double acc = 0.0;
  const unsigned long long lo_mask = (1ull << a) - 1ull;
  for (long long col = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; col < ncols;
       col += static_cast<long long>(gridDim.x) * blockDim.x) {
    const unsigned long long uc = static_cast<unsigned long long>(col);
    const float2* g = psi + ((uc & lo_mask) | ((uc >> a) << (a + w)));
    float2 v[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = r < (1 << w) ? g[static_cast<unsigned long long>(r) << a] : make_float2(0.f, 0.f);
    float f = 0.f;  // at most 160 pair products of this column, then FP64
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      if (b < w) {
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          if (!(r & (1 << b)) && r < (1 << w)) {
            const float2 u = v[r], z = v[r | (1 << b)];
            f = fmaf(u.x, z.x, f);
            f = fmaf(u.y, z.y, f);
          }
        }
      }
    }
    acc += static_cast<double>(f);
  }
  const double t = block_sum(acc, s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// result[0..4] = norm, <H_P>, ground, count, C.  Regions 0..4 come from the low
// kernel; regions 5.. are the strided correlation kernels (added to C).
__global__ void __launch_bounds__(256)
    obs_reduce_kernel(const double* __restrict__ partials, int nparts, int nregions, double* __restrict__ result) {
  __shared__ double s[256];
  for (int q = 0; q < kObsQuant; ++q) {
    double t = 0.0;
    const int last = (q == kObsQuant - 1) ? nregions : q + 1;
    for (int reg = q; reg < last; ++reg) {
      for (int i = threadIdx.x; i < nparts; i += blockDim.x) t += partials[static_cast<size_t>(reg) * nparts + i];
    }
    s[threadIdx.x] = t;
    __syncthreads();
    for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
      if (static_cast<int>(threadIdx.x) < h) s[threadIdx.x] += s[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) result[q] = s[0];
    __syncthreads();
  }
}

static int obs_grid(int num_sms) { return 2 * num_sms; }

static int corr_kernels(int n) { return n > kLowBits ? (n - kLowBits + 4) / 5 : 0; }

size_t obs_partials_len(int n, int num_sms) {
  return static_cast<size_t>(kObsQuant + corr_kernels(n)) * obs_grid(num_sms);
}

cudaError_t launch_hp_diag(const LaunchCtx& lc, uint16_t* out, int n, int m, const ClauseLP* cl) {
  const long long ntiles = n > kLowBits ? (1ll << (n - kLowBits)) : 1ll;
  const size_t smem = 16u * static_cast<size_t>(m) + static_cast<size_t>(kObsWarps) * 8u * (m + 16);
  cudaError_t err = allow_smem(reinterpret_cast<const void*>(diag_kernel), 16u * QAA_MAX_CLAUSES_DEV + static_cast<size_t>(kObsWarps) * 8u * (QAA_MAX_CLAUSES_DEV + 16));
  if (err != cudaSuccess) return err;
  long long grid = (ntiles + kObsWarps - 1) / kObsWarps;
  if (grid > 4ll * lc.num_sms) grid = 4ll * lc.num_sms;
  diag_kernel<<<static_cast<unsigned>(grid), kObsWarps * 32, smem, lc.stream>>>(out, n, m, cl, ntiles);
  return cudaGetLastError();
}

cudaError_t launch_observables(const LaunchCtx& lc, const float2* psi, int n, int m, const ClauseLP* cl,
                               double* partials, double* result) {
  const int P = obs_grid(lc.num_sms);
  const long long ntiles = n > kLowBits ? (1ll << (n - kLowBits)) : 1ll;
  const size_t smem = obs_low_smem(m);
  cudaError_t err = allow_smem(reinterpret_cast<const void*>(obs_low_kernel), obs_low_smem(QAA_MAX_CLAUSES_DEV));
  if (err != cudaSuccess) return err;
  obs_low_kernel<<<P, kObsWarps * 32, smem, lc.stream>>>(psi, n, m, cl, ntiles, partials);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  const int nc = corr_kernels(n);
  for (int k = 0; k < nc; ++k) {
    const int a = kLowBits + 5 * k;
    const int w = (n - a) < 5 ? (n - a) : 5;
    const long long ncols = 1ll << (n - w);
    corr_kernel<<<P, 256, 0, lc.stream>>>(psi, a, w, ncols, partials + static_cast<size_t>(kObsQuant + k) * P);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  obs_reduce_kernel<<<1, 256, 0, lc.stream>>>(partials, P, kObsQuant + nc, result);
  return cudaGetLastError();
}

}  // namespace qaa
