// Small-instance evolver (n <= 14): the whole complex64 state (<= 128 KiB) and
// its energies E(x) stay in one CTA's shared memory for every step of a run, so
// HBM is touched once on entry and once on exit.
//
// Same Strang step as the streaming path (Eq. (1) frozen at s_k; H_B applied as
// a popcount phase between two Walsh-Hadamard transforms, Sec. 2.1; H_P the
// violated-clause count, Sec. 4.3), with half phases of adjacent steps merged.
// The transform runs in "rounds" over groups of up to 5 index bits: each thread
// pulls a column of 2^w amplitudes into registers, applies the butterflies (and
// any phase due in that round) and writes it back.
//   step: [group 0: W] [groups 1..G-2: W] [group G-1: W B W] [groups G-2..1: W]
//         [group 0: W P(next) W(next step)]
// E(x) is evaluated once per launch from the clause bit masks (bit exact) and
// kept as uint16 in shared memory.
#include "device_common.cuh"

namespace qaa {

constexpr int kOnchipThreads = 512;

// Shared slot of amplitude x: rows of 32 padded to 33 (bank-conflict-free for
// columns along any 5-bit group, base + immediate addressing within a column).
__device__ __forceinline__ int oswz(int x) { return x + (x >> 5); }

enum : unsigned { kPreP = 1u, kW1 = 2u, kMidB = 4u, kW2 = 8u, kPostP = 16u, kW3 = 32u, kNorm = 64u };

template <int W>
__device__ __forceinline__ void col_wht(float2 (&v)[1 << W]) {
#pragma unroll
  for (int b = 0; b < W; ++b) {
#pragma unroll
    for (int r = 0; r < (1 << W); ++r) {
      if (!(r & (1 << b))) butterfly(v[r], v[r | (1 << b)]);
    }
  }
}

// kNorm: add |psi|^2 of the round's outputs to *nacc (FP32: at most one column
// per thread at n <= 14); cs = c - 1 scales the popcount phase (the norm fold of the
// previous step).
template <int W>
__device__ void onchip_round(float2* __restrict__ s_psi, const uint16_t* __restrict__ s_e, int n, int b0,
                             unsigned flags, const float2* __restrict__ prow_a, const float2* __restrict__ brow,
                             const float2* __restrict__ prow_b, float cs, float* nacc) {
  const int ncols = (1 << n) >> W;
  const int lo_mask = (1 << b0) - 1;
  for (int col = threadIdx.x; col < ncols; col += blockDim.x) {
    const int xb = (col & lo_mask) | ((col >> b0) << (b0 + W));
    // slot(xb + (r << b0)) = slot(xb) + r * rstep: xb has no bits in [b0, b0+W)
    // and, for b0 = 0, is a multiple of 32 (W = 5) or the whole index is < 32.
    const int sx = oswz(xb);
    const int rstep = (1 << b0) + (b0 >= 5 ? (1 << (b0 - 5)) : 0);
    float2 v[1 << W];
#pragma unroll
    for (int r = 0; r < (1 << W); ++r) v[r] = s_psi[sx + r * rstep];
    if (flags & kPreP) {
#pragma unroll
      for (int r = 0; r < (1 << W); ++r) v[r] = cmul(v[r], prow_a[s_e[sx + r * rstep]]);
    }
    if (flags & kW1) col_wht<W>(v);
    if (flags & kMidB) {
      const int pc = __popc(xb);
#pragma unroll
      for (int r = 0; r < (1 << W); ++r) v[r] = cmul(v[r], brow[pc + __popc(r)]);
      if (cs != 0.0f) {
#pragma unroll
        for (int r = 0; r < (1 << W); ++r) v[r] = fold_apply(v[r], cs);
      }
    }
    if (flags & kW2) col_wht<W>(v);
    if (flags & kPostP) {
#pragma unroll
      for (int r = 0; r < (1 << W); ++r) v[r] = cmul(v[r], prow_b[s_e[sx + r * rstep]]);
    }
    if (flags & kW3) col_wht<W>(v);
#pragma unroll
    for (int r = 0; r < (1 << W); ++r) s_psi[sx + r * rstep] = v[r];
    if (flags & kNorm) {
      // pairwise tree over the column (at most 5 levels of FP32 rounding)
      float p[1 << W];
#pragma unroll
      for (int r = 0; r < (1 << W); ++r) p[r] = fmaf(v[r].x, v[r].x, v[r].y * v[r].y);
#pragma unroll
      for (int h = (1 << W) >> 1; h > 0; h >>= 1) {
#pragma unroll
        for (int r = 0; r < h; ++r) p[r] += p[r + h];
      }
      *nacc += p[0];
    }
  }
}

__device__ __forceinline__ void round_dispatch(float2* s_psi, const uint16_t* s_e, int n, int g, unsigned flags,
                                               const float2* pa, const float2* br, const float2* pb, float cs,
                                               float* nacc) {
  const int b0 = 5 * g;
  const int w = (n - b0) < 5 ? (n - b0) : 5;
  switch (w) {
    case 1: onchip_round<1>(s_psi, s_e, n, b0, flags, pa, br, pb, cs, nacc); break;
    case 2: onchip_round<2>(s_psi, s_e, n, b0, flags, pa, br, pb, cs, nacc); break;
    case 3: onchip_round<3>(s_psi, s_e, n, b0, flags, pa, br, pb, cs, nacc); break;
    case 4: onchip_round<4>(s_psi, s_e, n, b0, flags, pa, br, pb, cs, nacc); break;
    default: onchip_round<5>(s_psi, s_e, n, b0, flags, pa, br, pb, cs, nacc); break;
  }
  __syncthreads();
}

// The norm fold of a step (as in the streaming low passes): the block's sum of
// one FP32 value per thread -- a fixed FP32 shuffle tree per warp, the warps'
// sums added as double-floats by thread 0 -- returned as a double-float pair
// when ref is null, else the correction c - 1 = fold_scale(ref, sum) in .hi.  Every
// thread gets the result.  Contains __syncthreads: every thread calls it.
__device__ DFloat onchip_fold(float v, const DFloat* ref) {
  __shared__ float s_w[kOnchipThreads / 32];
  __shared__ DFloat s_out;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) s_w[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    DFloat t{0.f, 0.f};
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t = df_add1(t, s_w[w]);
    s_out = ref ? DFloat{fold_scale(*ref, t), 0.f} : t;
  }
  __syncthreads();
  const DFloat out = s_out;
  __syncthreads();  // s_out is written again by the next call
  return out;
}

// Shared layout: [psi slots | E slots (uint16) | clauses], every region starting
// on a 16-byte boundary (the clause records are read with 128-bit loads).
struct OnchipLayout {
  size_t slots, off_e, off_cl, total;
  __host__ __device__ explicit OnchipLayout(int n, int m) {
    const size_t N = static_cast<size_t>(1) << n;
    slots = N + (N >> 5) + 1;
    off_e = (slots * 8u + 15u) & ~static_cast<size_t>(15);
    off_cl = off_e + ((slots * 2u + 15u) & ~static_cast<size_t>(15));
    total = off_cl + 16u * static_cast<size_t>(m);
  }
};

size_t onchip_smem_bytes(int n, int m) { return OnchipLayout(n, m).total; }

// One whole run (or chunk of a run) of one instance, by one CTA.
__device__ void onchip_run(float2* __restrict__ psi, int n, int m, const ClauseMV* __restrict__ cl,
                           const float2* __restrict__ ptab, const float2* __restrict__ btab, int nsteps, int first_p,
                           unsigned char* smem, bool init_uniform = false, float init_val = 0.0f) {
  const int N = 1 << n;
  const OnchipLayout L(n, m);
  float2* s_psi = reinterpret_cast<float2*>(smem);
  uint16_t* s_e = reinterpret_cast<uint16_t*>(smem + L.off_e);
  ClauseMV* s_cl = reinterpret_cast<ClauseMV*>(smem + L.off_cl);
  for (int i = threadIdx.x; i < m; i += blockDim.x) s_cl[i] = cl[i];
  // the uniform start state 2^(-n/2) (Sec. 2.1, value rounded on the host as
  // for qaa_init_uniform), or the caller's state
  const float2 u = make_float2(init_val, 0.0f);
  float racc = 0.0f;  // |psi|^2 of the input: the norm every step is folded back to
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    const float2 a = init_uniform ? u : psi[x];
    s_psi[oswz(x)] = a;
    racc += fmaf(a.x, a.x, a.y * a.y);  // at most 32 terms per thread (N <= 2^14)
  }
  const DFloat nref = onchip_fold(racc, nullptr);
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    int e = 0;
    for (int c = 0; c < m; ++c) {
      const unsigned mk = static_cast<unsigned>(s_cl[c].mask), vl = static_cast<unsigned>(s_cl[c].viol);
      e += (static_cast<unsigned>(x) & mk) == vl;
    }
    s_e[oswz(x)] = static_cast<uint16_t>(e);
  }
  __syncthreads();

  const int G = (n + 4) / 5;
  const int mp1 = m + 1;
  bool w0_done = false;
  float cs = 0.0f;  // norm fold c - 1 of the previous step, applied with the popcount phase
  for (int j = 0; j < nsteps; ++j) {
    const float2* p_first = ptab;  // row 0, only when first_p and j == 0
    const float2* p_next = ptab + static_cast<size_t>(j + 1) * mp1;
    const float2* brow = btab + static_cast<size_t>(j) * (n + 1);
    const bool last = j == nsteps - 1;
    const unsigned pre = (j == 0 && first_p) ? kPreP : 0u;
    // measure every fold_period(n)-th step; the factor corrects the step after it only
    const bool measure = !last && (j + 1) % fold_period(n) == 0;
    const unsigned nrm = measure ? kNorm : 0u;
    float nacc = 0.0f;
    if (G == 1) {
      const unsigned f = pre | (w0_done ? 0u : kW1) | kMidB | kW2 | kPostP | (last ? 0u : kW3) | nrm;
      round_dispatch(s_psi, s_e, n, 0, f, p_first, brow, p_next, cs, &nacc);
    } else {
      if (!w0_done) round_dispatch(s_psi, s_e, n, 0, pre | kW1, p_first, brow, p_next, cs, &nacc);
      for (int g = 1; g <= G - 2; ++g) round_dispatch(s_psi, s_e, n, g, kW1, p_first, brow, p_next, cs, &nacc);
      round_dispatch(s_psi, s_e, n, G - 1, kW1 | kMidB | kW2, p_first, brow, p_next, cs, &nacc);
      for (int g = G - 2; g >= 1; --g) round_dispatch(s_psi, s_e, n, g, kW1, p_first, brow, p_next, cs, &nacc);
      round_dispatch(s_psi, s_e, n, 0, kW1 | kPostP | (last ? 0u : kW3) | nrm, p_first, brow, p_next, cs, &nacc);
    }
    cs = measure ? onchip_fold(nacc, &nref).hi : 0.0f;
    w0_done = !last;
  }
  for (int x = threadIdx.x; x < N; x += blockDim.x) psi[x] = s_psi[oswz(x)];
}

__global__ void __launch_bounds__(kOnchipThreads)
    onchip_kernel(float2* __restrict__ psi, int n, int m, const ClauseMV* __restrict__ cl,
                  const float2* __restrict__ ptab, const float2* __restrict__ btab, int nsteps, int first_p) {
  extern __shared__ __align__(16) unsigned char smem[];
  onchip_run(psi, n, m, cl, ptab, btab, nsteps, first_p, smem);
}

// A batch of independent instances of uneven size and length: one CTA each.
__global__ void __launch_bounds__(kOnchipThreads) onchip_batch_kernel(const OnchipJob* __restrict__ jobs, int njobs) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (static_cast<int>(blockIdx.x) >= njobs) return;
  const OnchipJob jb = jobs[blockIdx.x];
  if (jb.stamp && threadIdx.x == 0) *jb.stamp = global_ns();
  onchip_run(jb.psi, jb.n, jb.m, jb.cl, jb.ptab, jb.btab, jb.nsteps, jb.first_p, smem, jb.init != 0, jb.init_val);
}

cudaError_t launch_onchip_batch(const LaunchCtx& lc, const OnchipJob* jobs_dev, int njobs, size_t smem_bytes) {
  if (njobs <= 0) return cudaSuccess;
  cudaError_t err =
      allow_smem(reinterpret_cast<const void*>(onchip_batch_kernel), onchip_smem_bytes(kOnchipMaxBits, QAA_MAX_CLAUSES_DEV));
  if (err != cudaSuccess) return err;
  onchip_batch_kernel<<<njobs, kOnchipThreads, smem_bytes, lc.stream>>>(jobs_dev, njobs);
  return cudaGetLastError();
}

cudaError_t launch_onchip(const LaunchCtx& lc, float2* psi, int n, int m, const ClauseMV* cl, const float2* ptab,
                          const float2* btab, int nsteps, bool first_p) {
  if (n > kOnchipMaxBits) return cudaErrorInvalidValue;
  const size_t smem = onchip_smem_bytes(n, m);
  cudaError_t err = allow_smem(reinterpret_cast<const void*>(onchip_kernel), onchip_smem_bytes(kOnchipMaxBits, QAA_MAX_CLAUSES_DEV));
  if (err != cudaSuccess) return err;
  onchip_kernel<<<1, kOnchipThreads, smem, lc.stream>>>(psi, n, m, cl, ptab, btab, nsteps, first_p ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace qaa
