// Persistent evolution of one mid-size instance (15 <= n <= 24) in a single
// cooperative launch on a few CTAs: every pass of every Strang step runs inside
// the kernel, separated by a grid barrier, instead of one kernel launch per
// pass.  The same passes and arithmetic as the streaming path (pass_kernels.cu):
// low pass W P W over bits 0..9 with on-the-fly clause counting, strided
// passes over groups of 5..10 bits, the phase group fused W B W.  Used by the
// serving loop, where many such requests run at once on disjoint sets of SMs.
//
// Strided tiles here always hold 2^13 amplitudes: 2^Q rows x 2^(13-Q)
// contiguous amplitudes, 256 threads, so one tile per CTA iteration for every
// group width Q.
//
// The grid barrier spins on a generation counter with an iteration limit
// (2^21 polls, about a second); on expiry it records an error word (reported
// as QAA_E_TIMEOUT) and the kernel returns.  Cooperative launch guarantees that all CTAs are resident.
#include "device_common.cuh"

namespace qaa {

constexpr int kPersistThreads = 256;
constexpr int kPersistWarps = kPersistThreads / 32;
constexpr int kRow = 33;
constexpr int kLpSlots = 32 * kRow;

struct PersistArgs {
  float2* psi;
  const ClauseLP* cl;
  const float2* ptab;  // K + 1 rows of m + 1 entries (the whole run)
  const float2* btab;  // K rows of n + 1 entries
  unsigned* bar;       // [0] arrivals, [1] generation; zeroed before launch
  int* err;
  double* fold;        // norm-fold slots (kFoldBytes), or null
  int n, m, K;
  int ng, phase_group;
  int ga[3], gq[3];  // contiguous strided groups [ga, ga + gq)
};

__device__ bool grid_barrier(unsigned* bar, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    s_ok = 1;
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*gen == g) {
        if (++it > (1ll << 21)) {  // about a second: every pass here takes milliseconds at most
          atomicExch(err, 2);
          s_ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------ low pass ------
__device__ __forceinline__ void x2y(float2 (&v)[32], float2* __restrict__ s, int lane) {
#pragma unroll
  for (int r = 0; r < 32; ++r) s[lane + kRow * r] = v[r];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 32; ++r) v[r] = s[kRow * lane + r];
  __syncwarp();
}
__device__ __forceinline__ void y2x(float2 (&v)[32], float2* __restrict__ s, int lane) {
#pragma unroll
  for (int r = 0; r < 32; ++r) s[kRow * lane + r] = v[r];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 32; ++r) v[r] = s[lane + kRow * r];
  __syncwarp();
}

// rel: the step this low pass ends (-1 for the first pass), selecting the
// norm-fold slots as for the streaming passes; the correction of the previous
// step is applied as a factor after the P phase (the P row stays in global
// memory here).
template <int KIND>
__device__ void low_pass(const PersistArgs& A, const ClauseLP* s_cl, float2* s_tile, uint2* s_act,
                         const float2* __restrict__ tab, int rel) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long ntiles = 1ll << (A.n - kLowBits);
  Pass fp{};
  fp.rel = rel;
  const NormFold nf = fold_for(A.fold, fp, fold_period(A.n));
  const float fd = fold_factor_block(nf);
  DFloat nacc{0.f, 0.f};
  for (long long tile = static_cast<long long>(blockIdx.x) * kPersistWarps + warp; tile < ntiles;
       tile += static_cast<long long>(gridDim.x) * kPersistWarps) {
    float2* g = A.psi + (tile << kLowBits);
    int nconst, npad;
    unsigned pl[kPlanes];
    __syncwarp();
    fold_tile<KIND != kLpFirst>(s_cl, A.m, static_cast<unsigned>(tile), lane, s_act, nconst, npad);
    count_active(s_act, npad, 1u << lane, pl);
    float2 v[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = g[lane + 32 * r];
    if (KIND == kLpFirst) {
      apply_p_phase(v, pl, nconst, tab);
      reg_wht<0, 5>(v);
      x2y(v, s_tile, lane);
      reg_wht<0, 5>(v);
      y2x(v, s_tile, lane);
    } else {
      reg_wht<0, 5>(v);
      x2y(v, s_tile, lane);
      reg_wht<0, 5>(v);
      apply_p_phase(v, pl, nconst, tab);
      if (fd != 0.0f) {
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = fold_apply(v[r], fd);
      }
      if (KIND == kLpMerge) reg_wht<0, 5>(v);
      y2x(v, s_tile, lane);
      if (KIND == kLpMerge) reg_wht<0, 5>(v);
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) g[lane + 32 * r] = v[r];
    if (nf.out) nacc = df_add1(nacc, tile_norm(v));
  }
  fold_store(nf, nacc);
}

// -------------------------------------------------------- strided pass ------
// Tile t = j + (i << C), C = 13 - Q, 256 threads.  Layout A: register = i bits
// 0..4, thread = (j, i bits 5..Q-1); layout B: register = i bits Q-5..Q-1,
// thread = (j, i bits 0..Q-6).  Shared slot: t + ((t >> (C+5)) << C).
template <int Q, bool WBW>
__device__ void strided_pass(const PersistArgs& A, int a, const float2* __restrict__ brow, float2* s_tile) {
  constexpr int C = 13 - Q;
  constexpr int QB = Q - 5;
  auto slot = [](int t) { return t + ((t >> (C + 5)) << C); };
  const int tid = threadIdx.x;
  const int j = tid & ((1 << C) - 1);
  const int th = tid >> C;
  const unsigned long long lo_mask = (1ull << (a - C)) - 1ull;
  const unsigned long long stride = 1ull << a;
  const long long ntiles = 1ll << (A.n - Q - C);
  for (long long T = blockIdx.x; T < ntiles; T += gridDim.x) {
    const unsigned long long ut = static_cast<unsigned long long>(T);
    const unsigned long long xbase = ((ut & lo_mask) << C) | ((ut >> (a - C)) << (a + Q));
    float2* g = A.psi + xbase + j;
    float2 v[32];
    {
      const float2* pa = g + (static_cast<unsigned long long>(th) << (a + 5));
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        v[r] = *pa;
        pa += stride;
      }
    }
    reg_wht<0, 5>(v);
    const int sa = j + (th << (C + 5)) + (QB > 0 ? (th << C) : 0);  // slot of (j, r = 0, th), layout A
    const int sb = slot(j + (th << C));
    if (QB > 0) {
#pragma unroll
      for (int r = 0; r < 32; ++r) s_tile[sa + (r << C)] = v[r];
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = s_tile[sb + slot((r << QB) << C)];
      __syncthreads();
      reg_wht<10 - Q, 5>(v);
    }
    if (WBW) {
      const int pc0 = __popcll(xbase) + __popc(j) + __popc(th);
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = cmul(v[r], __ldg(brow + pc0 + __popc(r)));
      if (QB > 0) {
        reg_wht<10 - Q, 5>(v);
#pragma unroll
        for (int r = 0; r < 32; ++r) s_tile[sb + slot((r << QB) << C)] = v[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = s_tile[sa + (r << C)];
        __syncthreads();
      }
      reg_wht<0, 5>(v);
      float2* pa = g + (static_cast<unsigned long long>(th) << (a + 5));
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        *pa = v[r];
        pa += stride;
      }
    } else {
      float2* pb = g + (static_cast<unsigned long long>(th) << a);
      const unsigned long long sbs = stride << QB;
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        *pb = v[r];
        pb += sbs;
      }
    }
  }
}

template <bool WBW>
__device__ void strided_dispatch(const PersistArgs& A, int a, int q, const float2* brow, float2* s_tile) {
  switch (q) {
    case 5: strided_pass<5, WBW>(A, a, brow, s_tile); break;
    case 6: strided_pass<6, WBW>(A, a, brow, s_tile); break;
    case 7: strided_pass<7, WBW>(A, a, brow, s_tile); break;
    case 8: strided_pass<8, WBW>(A, a, brow, s_tile); break;
    case 9: strided_pass<9, WBW>(A, a, brow, s_tile); break;
    default: strided_pass<10, WBW>(A, a, brow, s_tile); break;
  }
}

// smem: [clauses 16m | per-warp (padded tile, active list) ] ... strided tiles reuse
// the same space (8192 + 256 slots = 67584 bytes).
__host__ __device__ inline size_t persist_smem(int m) {
  const size_t lp = 16u * static_cast<size_t>(m) + static_cast<size_t>(kPersistWarps) * (8u * kLpSlots + 8u * (m + 16));
  const size_t sp = 16u * static_cast<size_t>(m) + 8u * (8192u + 256u);
  return lp > sp ? lp : sp;
}

__global__ void __launch_bounds__(kPersistThreads) persist_kernel(PersistArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  ClauseLP* s_cl = reinterpret_cast<ClauseLP*>(smem);
  unsigned char* work = smem + 16u * A.m;
  const int warp = threadIdx.x >> 5;
  float2* s_wtile = reinterpret_cast<float2*>(work) + warp * kLpSlots;
  uint2* s_act = reinterpret_cast<uint2*>(work + static_cast<size_t>(kPersistWarps) * 8u * kLpSlots) + warp * (A.m + 16);
  float2* s_tile = reinterpret_cast<float2*>(work);
  for (int i = threadIdx.x; i < A.m; i += blockDim.x) s_cl[i] = A.cl[i];
  __syncthreads();
  const int mp1 = A.m + 1, np1 = A.n + 1;
  const int pg = A.phase_group;
  auto sync = [&]() { return grid_barrier(A.bar, A.err); };
  // first pass of the run: P(row 0) then W over bits 0..9, then the other groups up
  low_pass<kLpFirst>(A, s_cl, s_wtile, s_act, A.ptab, -1);
  if (!sync()) return;
  for (int g = 0; g < A.ng; ++g) {
    if (g == pg) continue;
    strided_dispatch<false>(A, A.ga[g], A.gq[g], nullptr, s_tile);
    if (!sync()) return;
  }
  for (int k = 0; k < A.K; ++k) {
    strided_dispatch<true>(A, A.ga[pg], A.gq[pg], A.btab + static_cast<size_t>(k) * np1, s_tile);
    if (!sync()) return;
    for (int g = A.ng - 1; g >= 0; --g) {
      if (g == pg) continue;
      strided_dispatch<false>(A, A.ga[g], A.gq[g], nullptr, s_tile);
      if (!sync()) return;
    }
    const float2* prow = A.ptab + static_cast<size_t>(k + 1) * mp1;
    if (k == A.K - 1) {
      low_pass<kLpLast>(A, s_cl, s_wtile, s_act, prow, k);
      break;  // the kernel's end orders the final pass before any later work
    }
    low_pass<kLpMerge>(A, s_cl, s_wtile, s_act, prow, k);
    if (!sync()) return;
    for (int g = 0; g < A.ng; ++g) {
      if (g == pg) continue;
      strided_dispatch<false>(A, A.ga[g], A.gq[g], nullptr, s_tile);
      if (!sync()) return;
    }
  }
}

cudaError_t launch_persist(const LaunchCtx& lc, const PersistPlan& pp, float2* psi, int n, int m, const ClauseLP* cl,
                           const float2* ptab, const float2* btab, int K, unsigned* bar, int* err, int grid,
                           double* fold) {
  PersistArgs A;
  A.fold = fold;
  A.psi = psi;
  A.cl = cl;
  A.ptab = ptab;
  A.btab = btab;
  A.bar = bar;
  A.err = err;
  A.n = n;
  A.m = m;
  A.K = K;
  A.ng = pp.ng;
  A.phase_group = pp.phase_group;
  for (int g = 0; g < 3; ++g) {
    A.ga[g] = pp.ga[g];
    A.gq[g] = pp.gq[g];
  }
  if (pp.ng < 1 || pp.ng > 3 || pp.phase_group < 0 || pp.phase_group >= pp.ng) return cudaErrorInvalidValue;
  for (int g = 0; g < pp.ng; ++g)
    if (pp.gq[g] < 5 || pp.gq[g] > 10) return cudaErrorInvalidValue;  // strided tiles of 5..10 bits only
  const size_t smem = persist_smem(m);
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(persist_kernel), persist_smem(QAA_MAX_CLAUSES_DEV));
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persist_kernel, kPersistThreads, smem);
  if (e != cudaSuccess) return e;
  if (grid > occ * lc.num_sms) grid = occ * lc.num_sms;
  if (grid > kFoldSlot - 1) grid = kFoldSlot - 1;  // one norm-fold partial per CTA
  if (grid < 1) return cudaErrorInvalidConfiguration;
  void* params[] = {&A};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(persist_kernel), dim3(grid), dim3(kPersistThreads),
                                     params, smem, lc.stream);
}

}  // namespace qaa
