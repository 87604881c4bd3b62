// Read-only kernels: the exported H_P diagonal and the FP64 observables.
//
// Observables (ground state and its probability: Sec. 2.1; the result gathered
// from every thread and returned to the host: Sec. 4.2):
//   norm = sum |psi|^2, <H_P> = sum E |psi|^2, ground = sum_{E=0} |psi|^2,
//   count of E = 0, and C = sum_i sum_{x: bit i-1 clear} Re(conj psi_x psi_(x+2^(i-1)))
//   from which <H_B> = n/2 norm - C.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so no per-amplitude
// work is done in FP64 here.  norm, <H_P> and the ground probability are formed
// exactly in FP32 pieces and summed as double-floats (an FP32 value plus its
// exact rounding error):
//   * |psi|^2 = re^2 + im^2: each square split into its FP32 product and the
//     product's exact error (one FMA), the two products added with Knuth's
//     TwoSum (exact result as sum + error);
//   * E |psi|^2: the same split of E times the FP32 part;
//   * each lane's running sums over its 32 amplitudes of a tile: TwoSum into a
//     (sum, error) pair, on packed f32x2 instructions for (norm, <H_P>);
//   * once per four tiles the pairs are added into the lane's FP64 totals.
// The result agrees with exact-product FP64 sums to about 1e-14 relative.
// The pair correlations C (n pair products per amplitude) are formed and
// summed in FP32 over one thread's share of one tile (at most 320 products)
// and accumulated in FP64 beyond that.  Every sum runs in a fixed order (per
// thread, a fixed shuffle/shared-memory tree per block, the partials by one
// block): bit-identical run to run.
//
// Passes over the state: the low kernel reads it once (bits 0..9 of the index
// in one warp's 1024-amplitude tile, brought in by a bulk copy for n > 10: the
// norm-type sums and the pair correlations of bits 0..9), and bits 10..n-1 are
// covered in groups of at most 10 bits by read-only strided-tile passes
// (corr_tma_kernel in tma_kernels.cu; plain loads in groups of 5 when TMA is
// unavailable): 3 reads of the state at n = 30.
#include "device_common.cuh"

namespace qaa {

constexpr int kObsWarps = 8;
constexpr int kObsQuant = 5;  // norm, hp, ground, count, corr(low bits)
constexpr int kObsRow = 33;   // padded transpose rows (as the low passes)

static size_t obs_low_smem(int m, bool stored) {
  const size_t tile = static_cast<size_t>(kObsWarps) * 8u * kObsRow * 32u;
  if (stored) return tile + 64u * 8u;
  return 16u * static_cast<size_t>(m) + tile + static_cast<size_t>(kObsWarps) * 8u * static_cast<size_t>(m + 16) +
         64u * 8u;
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

// ---- double-float accumulation ------------------------------------------------
__device__ __forceinline__ unsigned long long f2add(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2sub(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2fma(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// One lane's sums over a tile: (norm, <H_P>) as packed (sum, error) pairs, the
// ground probability as a scalar pair, the ground count.
struct ObsAcc {
  unsigned long long s = 0ull, e = 0ull;
  float gs = 0.f, ge = 0.f, gc = 0.f;
};

// Knuth's TwoSum: s + b = s' + err exactly; err added to e.
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float b) {
  const float t = s + b;
  const float bb = t - s;
  e += (s - (t - bb)) + (b - bb);
  s = t;
}

// Add |v|^2 (and E |v|^2, and |v|^2 to the ground sums when `ground`).
__device__ __forceinline__ void obs_add(ObsAcc& a, float2 v, float E, bool ground) {
  const unsigned long long vv = f2_bits(v);
  unsigned long long h;
  asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(h) : "l"(vv));
  const unsigned long long l = f2fma(vv, vv, h ^ 0x8000000080000000ull);  // exact errors of re^2, im^2
  const float2 hf = bits_f2(h), lf = bits_f2(l);
  // p = re^2 + im^2 = ph + pl (pl: TwoSum error of the two squares plus their errors)
  const float ph = hf.x + hf.y;
  const float bb = ph - hf.x;
  const float pl = ((hf.x - (ph - bb)) + (hf.y - bb)) + (lf.x + lf.y);
  const float eh = E * ph;
  const float el = fmaf(E, pl, fmaf(E, ph, -eh));  // E ph - eh exactly, plus E pl
  const unsigned long long t = f2_bits(make_float2(ph, eh));
  const unsigned long long s = f2add(a.s, t);
  const unsigned long long b2 = f2sub(s, a.s);
  const unsigned long long err = f2add(f2sub(a.s, f2sub(s, b2)), f2sub(t, b2));
  a.s = s;
  a.e = f2add(a.e, f2add(err, f2_bits(make_float2(pl, el))));
  if (ground) {
    two_sum_acc(a.gs, a.ge, ph);
    a.ge += pl;
    a.gc += 1.f;
  }
}

template <int R>
struct ObsAddUnroll {
  __device__ __forceinline__ static void run(ObsAcc& a, const float2 (&v)[32], const unsigned (&pl)[kPlanes],
                                             int nconst, int lane, int N) {
    const unsigned w = extract_pair<R>(pl);
    const int e0 = nconst + static_cast<int>(w & 0xffffu), e1 = nconst + static_cast<int>(w >> 16);
    // layout Y: register r holds index bits 0..4, the lane bits 5..9
    obs_add(a, v[R], static_cast<float>(e0), e0 == 0 && R + 32 * lane < N);
    obs_add(a, v[R + 16], static_cast<float>(e1), e1 == 0 && R + 16 + 32 * lane < N);
    ObsAddUnroll<R + 1>::run(a, v, pl, nconst, lane, N);
  }
};
template <>
struct ObsAddUnroll<16> {
  __device__ __forceinline__ static void run(ObsAcc&, const float2 (&)[32], const unsigned (&)[kPlanes], int, int,
                                             int) {}
};

// Pair products over register bits [0, 5) with index bit (b + shift) < n.
__device__ __forceinline__ unsigned long long reg_pairs(const float2 (&v)[32], int shift, int n,
                                                        unsigned long long c) {
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    if (b + shift < n) {
#pragma unroll
      for (int r = 0; r < 32; ++r)
        if (!(r & (1 << b))) c = f2fma(f2_bits(v[r]), f2_bits(v[r | (1 << b)]), c);
    }
  }
  return c;
}

// Low kernel: one 1024-amplitude tile per warp.  Loaded in layout X (lane =
// bits 0..4, register = bits 5..9): the pairs of bits 5..9; transposed to
// layout Y (register = bits 0..4, lane = bits 5..9): the pairs of bits 0..4
// and the norm-type sums with the energies of layout Y, read from the stored
// per-tile counts (STORED) or folded and counted from the clauses.  n < 10:
// one tile, amplitudes beyond 2^n read as zero and excluded from the count.
template <bool STORED>
__global__ void __launch_bounds__(kObsWarps * 32)
    obs_low_kernel(const float2* __restrict__ psi, int n, int m, const ClauseLP* __restrict__ cl,
                   const unsigned* __restrict__ counts, long long ntiles, double* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t cl_bytes = STORED ? 0u : 16u * static_cast<size_t>(m);
  ClauseLP* s_cl = reinterpret_cast<ClauseLP*>(smem);
  float2* s_tile = reinterpret_cast<float2*>(smem + cl_bytes) + warp * (kObsRow * 32);
  unsigned char* after_tiles = smem + cl_bytes + static_cast<size_t>(kObsWarps) * 8u * kObsRow * 32u;
  uint2* s_act = reinterpret_cast<uint2*>(after_tiles) + warp * (m + 16);
  double* s_red = reinterpret_cast<double*>(after_tiles + (STORED ? 0u : static_cast<size_t>(kObsWarps) * 8u * (m + 16)));
  if (!STORED) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) s_cl[i] = cl[i];
  }
  __syncthreads();
  const int N = n < kLowBits ? (1 << n) : (1 << kLowBits);  // amplitudes per tile that exist
  double d_norm = 0.0, d_hp = 0.0, d_gp = 0.0, d_gc = 0.0, d_corr = 0.0;
  for (long long tile = static_cast<long long>(blockIdx.x) * kObsWarps + warp; tile < ntiles;
       tile += static_cast<long long>(gridDim.x) * kObsWarps) {
    const float2* g = psi + (static_cast<unsigned long long>(tile) << kLowBits);
    float2 v[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = lane + 32 * r < N ? g[lane + 32 * r] : make_float2(0.0f, 0.0f);
    unsigned long long c2 = reg_pairs(v, 5, n, 0ull);  // index bits 5..9
    // layout X -> Y through the padded tile
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 32; ++r) s_tile[lane + kObsRow * r] = v[r];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = s_tile[kObsRow * lane + r];
    c2 = reg_pairs(v, 0, n, c2);  // index bits 0..4
    unsigned pl[kPlanes];
    int nconst;
    if (STORED) {
      load_counts(counts, tile, lane, pl, nconst);
    } else {
      int npad;
      fold_tile<true>(s_cl, m, static_cast<unsigned>(tile), lane, s_act, nconst, npad);
      count_active(s_act, npad, 1u << lane, pl);
    }
    ObsAcc a;
    ObsAddUnroll<0>::run(a, v, pl, nconst, lane, N);
    const float2 s = bits_f2(a.s), e = bits_f2(a.e), c = bits_f2(c2);
    d_norm += static_cast<double>(s.x) + static_cast<double>(e.x);
    d_hp += static_cast<double>(s.y) + static_cast<double>(e.y);
    if (a.gc != 0.f) {
      d_gp += static_cast<double>(a.gs) + static_cast<double>(a.ge);
      d_gc += static_cast<double>(a.gc);
    }
    d_corr += static_cast<double>(c.x + c.y);
  }
  const double q[kObsQuant] = {d_norm, d_hp, d_gp, d_gc, d_corr};
#pragma unroll
  for (int k = 0; k < kObsQuant; ++k) {
    const double t = block_sum(q[k], s_red);
    if (threadIdx.x == 0) partials[static_cast<size_t>(k) * gridDim.x + blockIdx.x] = t;
  }
}

// ---- bulk-copy pipelined low kernel (n > 10) ---------------------------------
__device__ __forceinline__ uint32_t obs_smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool obs_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(obs_smem(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool obs_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < (1ll << 24); ++it)
    if (obs_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void obs_bulk_load(void* dst, const void* src, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(obs_smem(bar)), "r"(8192u) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 8192, [%2];" ::"r"(
                   obs_smem(dst)),
               "l"(src), "r"(obs_smem(bar))
               : "memory");
}

struct ObsTmaLayout {
  size_t off_warp, per_warp, off_bar, off_red, total;
  __host__ __device__ ObsTmaLayout(int m, bool stored) {
    off_warp = stored ? 0 : ((16u * static_cast<size_t>(m) + 127u) & ~static_cast<size_t>(127));
    per_warp = 8u * kObsRow * 32u + (stored ? 0u : 8u * static_cast<size_t>(m + 16));
    per_warp = (per_warp + 127u) & ~static_cast<size_t>(127);
    off_bar = off_warp + per_warp * kObsWarps;
    off_red = off_bar + 8u * kObsWarps;
    total = off_red + 64u * 8u;
  }
};

// As obs_low_kernel for n > 10, with each warp's 1024-amplitude tile brought in
// by a 1-D cp.async.bulk into its shared buffer (mbarrier completion): the
// buffer is read into registers and reused for the transpose, and the next
// tile's copy is issued as soon as the transpose is read back, so that it is
// in flight during this tile's double-float sums.  The (norm, <H_P>) pairs
// are added into FP64 every other tile.
template <bool STORED>
__global__ void __launch_bounds__(kObsWarps * 32, 2)
    obs_tma_kernel(const float2* __restrict__ psi, int n, int m, const ClauseLP* __restrict__ cl,
                   const unsigned* __restrict__ counts, long long ntiles, double* __restrict__ partials,
                   int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const ObsTmaLayout L(m, STORED);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  ClauseLP* s_cl = reinterpret_cast<ClauseLP*>(smem);
  unsigned char* wbase = smem + L.off_warp + L.per_warp * warp;
  float2* s_buf = reinterpret_cast<float2*>(wbase);
  uint2* s_act = reinterpret_cast<uint2*>(wbase + 8u * kObsRow * 32u);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + L.off_bar) + warp;
  double* s_red = reinterpret_cast<double*>(smem + L.off_red);
  const long long step = static_cast<long long>(gridDim.x) * kObsWarps;
  const long long first = static_cast<long long>(blockIdx.x) * kObsWarps + warp;
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(obs_smem(s_bar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (lane == 0 && first < ntiles) obs_bulk_load(s_buf, psi + (first << kLowBits), s_bar);
  if (!STORED) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) s_cl[i] = cl[i];
  }
  __syncthreads();
  double d_norm = 0.0, d_hp = 0.0, d_gp = 0.0, d_gc = 0.0, d_corr = 0.0;
  ObsAcc a;
  int it = 0;
  bool ok = true;
  for (long long tile = first; tile < ntiles; tile += step, ++it) {
    ok = obs_wait(s_bar, static_cast<uint32_t>(it) & 1u);
    if (__any_sync(0xffffffffu, !ok)) break;
    float2 v[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = s_buf[lane + 32 * r];
    unsigned long long c2 = reg_pairs(v, 5, n, 0ull);  // index bits 5..9
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 32; ++r) s_buf[lane + kObsRow * r] = v[r];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = s_buf[kObsRow * lane + r];
    __syncwarp();
    const long long tn = tile + step;
    if (lane == 0 && tn < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      obs_bulk_load(s_buf, psi + (tn << kLowBits), s_bar);
    }
    c2 = reg_pairs(v, 0, n, c2);  // index bits 0..4
    unsigned pl[kPlanes];
    int nconst;
    if (STORED) {
      load_counts(counts, tile, lane, pl, nconst);
    } else {
      int npad;
      fold_tile<true>(s_cl, m, static_cast<unsigned>(tile), lane, s_act, nconst, npad);
      count_active(s_act, npad, 1u << lane, pl);
    }
    ObsAddUnroll<0>::run(a, v, pl, nconst, lane, 1 << kLowBits);
    const float2 c = bits_f2(c2);
    d_corr += static_cast<double>(c.x + c.y);
    if ((it & 3) == 3 || tn >= ntiles) {
      const float2 ss = bits_f2(a.s), ee = bits_f2(a.e);
      d_norm += static_cast<double>(ss.x) + static_cast<double>(ee.x);
      d_hp += static_cast<double>(ss.y) + static_cast<double>(ee.y);
      if (a.gc != 0.f) {
        d_gp += static_cast<double>(a.gs) + static_cast<double>(a.ge);
        d_gc += static_cast<double>(a.gc);
      }
      a = ObsAcc();
    }
  }
  if (!ok) {
    if (lane == 0) atomicExch(err, 1);
  } else if (lane == 0) {
    // a copy may be in flight if the loop was left early; wait for it (bounded)
    const long long t = first + static_cast<long long>(it) * step;
    if (t < ntiles && !obs_wait(s_bar, static_cast<uint32_t>(it) & 1u)) atomicExch(err, 1);
  }
  const double q[kObsQuant] = {d_norm, d_hp, d_gp, d_gc, d_corr};
#pragma unroll
  for (int k = 0; k < kObsQuant; ++k) {
    const double t = block_sum(q[k], s_red);
    if (threadIdx.x == 0) partials[static_cast<size_t>(k) * gridDim.x + blockIdx.x] = t;
  }
}

// Pair correlations for index bits [a, a+w) (a >= 10, w <= 5) with plain
// loads: one thread per column (the other index bits), coalesced over the low
// bits.  Used for n = 11..14 and when TMA is unavailable.
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
// kernel; regions 5.. are the strided correlation kernels (added to C).  With
// stamp, the device time at the end (global_ns) is written there.
__global__ void __launch_bounds__(256)
    obs_reduce_kernel(const double* __restrict__ partials, int nparts, int nregions, double* __restrict__ result,
                      unsigned long long* __restrict__ stamp) {
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
  if (stamp && threadIdx.x == 0) *stamp = global_ns();
}

static int obs_grid(int num_sms) { return 2 * num_sms; }

// Correlation passes over bits [10, n): contiguous groups of 5..10 bits (as
// even as possible) on the TMA tile passes, else groups of at most 5 bits with
// plain loads (and always for n - 10 < 5).
struct CorrPlan {
  int ng = 0;
  int a[8] = {}, a2[8] = {}, q[8] = {};
  bool tma = false;
};
static CorrPlan corr_plan(int n, bool allow_tma) {
  CorrPlan p;
  const int rest = n - kLowBits;
  if (rest <= 0) return p;
  p.tma = allow_tma && rest >= 5 && tma_available();
  const int widest = p.tma ? 10 : 5;
  p.ng = (rest + widest - 1) / widest;
  int a = kLowBits;
  for (int g = 0; g < p.ng; ++g) {
    p.q[g] = rest / p.ng + (g < rest % p.ng ? 1 : 0);
    p.a[g] = a;
    p.a2[g] = a + 5;
    a += p.q[g];
  }
  // two 10-bit groups (n = 30): {10..14, 25..29} and {15..24}, as the
  // evolution's plan, so that a tile's rows span at most 128 memory pages
  // (the contiguous group [20, 30) ran at a third of the read bandwidth)
  if (p.tma && p.ng == 2 && p.q[0] == 10 && p.q[1] == 10) {
    p.a[0] = kLowBits;
    p.a2[0] = kLowBits + 15;
    p.a[1] = kLowBits + 5;
    p.a2[1] = kLowBits + 10;
  }
  return p;
}

// Room for either plan (the plain-load one has more groups).
size_t obs_partials_len(int n, int num_sms) {
  return static_cast<size_t>(kObsQuant + corr_plan(n, false).ng) * obs_grid(num_sms);
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
                               double* partials, double* result, const unsigned* counts, int* err_word,
                               unsigned long long* stamp) {
  const int P = obs_grid(lc.num_sms);
  const long long ntiles = n > kLowBits ? (1ll << (n - kLowBits)) : 1ll;
  const bool stored = counts != nullptr && n > kLowBits;
  cudaError_t err;
  if (n > kLowBits && err_word != nullptr && reinterpret_cast<uintptr_t>(psi) % 16u == 0) {
    // whole tiles: the bulk-copy pipelined kernel
    auto kern = stored ? obs_tma_kernel<true> : obs_tma_kernel<false>;
    err = allow_smem(reinterpret_cast<const void*>(kern), ObsTmaLayout(QAA_MAX_CLAUSES_DEV, stored).total);
    if (err != cudaSuccess) return err;
    kern<<<P, kObsWarps * 32, ObsTmaLayout(m, stored).total, lc.stream>>>(psi, n, m, cl, counts, ntiles, partials,
                                                                          err_word);
  } else {
    auto kern = stored ? obs_low_kernel<true> : obs_low_kernel<false>;
    err = allow_smem(reinterpret_cast<const void*>(kern), obs_low_smem(QAA_MAX_CLAUSES_DEV, stored));
    if (err != cudaSuccess) return err;
    kern<<<P, kObsWarps * 32, obs_low_smem(m, stored), lc.stream>>>(psi, n, m, cl, counts, ntiles, partials);
  }
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  // the TMA passes need an error word for their bounded waits
  const CorrPlan cp = corr_plan(n, err_word != nullptr && reinterpret_cast<uintptr_t>(psi) % 16u == 0);
  for (int k = 0; k < cp.ng; ++k) {
    double* part = partials + static_cast<size_t>(kObsQuant + k) * P;
    if (cp.tma) {
      err = launch_corr_tma(lc, psi, n, cp.a[k], cp.a2[k], cp.q[k], part, P, err_word);
    } else {
      const long long ncols = 1ll << (n - cp.q[k]);
      corr_kernel<<<P, 256, 0, lc.stream>>>(psi, cp.a[k], cp.q[k], ncols, part);
      err = cudaGetLastError();
    }
    if (err != cudaSuccess) return err;
  }
  obs_reduce_kernel<<<1, 256, 0, lc.stream>>>(partials, P, kObsQuant + cp.ng, result, stamp);
  return cudaGetLastError();
}

}  // namespace qaa
