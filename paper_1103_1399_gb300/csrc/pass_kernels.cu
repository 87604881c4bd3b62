// Streaming passes of the Strang step for n >= 15 (state in HBM).
//
// One Strang step (Eq. (1) frozen at s_k, Sec. 2.1 / Sec. 4.3 Hamiltonians)
//   P(dt/2 s_k) . W . B(dt (1-s_k)) . W . P(dt/2 s_k)
// is executed as HBM round trips over qubit groups G1 = bits 0..9 (the "low
// pass", contiguous 1024-amplitude tiles, one warp each) and strided groups
// G2..Gg above it.  The Walsh-Hadamard transform factors over qubits, so every
// group can be transformed separately, and
//   * the popcount phase B is applied inside the top group's pass between its
//     two transforms (kSpWBW), and
//   * the violated-clause phase P is applied inside the low pass between the
//     inverse transform of step k and the forward transform of step k+1, with
//     the two half phases merged into one (kLpMerge).
// E(x) is never stored: each low-pass tile folds the clause list against its
// fixed high bits and counts the surviving clauses for 32 amplitudes at a time
// with bit-sliced carry-save adders (device_common.cuh).
#include "device_common.cuh"

namespace qaa {

// ---------------------------------------------------------------------------
// low pass: tile = 1024 consecutive amplitudes, one warp, 32 registers/lane.
// Layout X: lane = bits 0..4, register = bits 5..9 (coalesced global access).
// Layout Y: lane = bits 5..9, register = bits 0..4.
// Shared-memory slot of tile index t = lo5 + 32 hi5: 33 hi5 + lo5 (rows padded
// to 33 amplitudes).  Both layouts then touch 32 distinct bank pairs per warp
// access (the 2-wavefront minimum for 8-byte elements) with base + immediate
// addressing, so no per-register address has to stay live.
constexpr int kLpRow = 33;
constexpr int kLpTileSlots = 32 * kLpRow;
__device__ __forceinline__ void xpose_x2y(float2 (&v)[32], float2* __restrict__ s, int lane) {
  float2* w = s + lane;
#pragma unroll
  for (int r = 0; r < 32; ++r) w[kLpRow * r] = v[r];
  __syncwarp();
  const float2* q = s + kLpRow * lane;
#pragma unroll
  for (int r = 0; r < 32; ++r) v[r] = q[r];
  __syncwarp();
}
__device__ __forceinline__ void xpose_y2x(float2 (&v)[32], float2* __restrict__ s, int lane) {
  float2* w = s + kLpRow * lane;
#pragma unroll
  for (int r = 0; r < 32; ++r) w[r] = v[r];
  __syncwarp();
  const float2* q = s + lane;
#pragma unroll
  for (int r = 0; r < 32; ++r) v[r] = q[kLpRow * r];
  __syncwarp();
}

constexpr int kLpWarps = 8;

__host__ __device__ inline size_t lp_smem_bytes(int m) {
  size_t off = 16u * static_cast<size_t>(m) + ((8u * static_cast<size_t>(m + 1) + 15u) & ~static_cast<size_t>(15));
  return off + static_cast<size_t>(kLpWarps) * (8u * kLpTileSlots + 8u * static_cast<size_t>(m + 16));
}

template <int KIND>
__global__ void __launch_bounds__(kLpWarps * 32, 2)
    lp_kernel(float2* __restrict__ psi, int m, const ClauseLP* __restrict__ cl,
              const float2* __restrict__ prow, long long ntiles, const NormFold nf) {
  extern __shared__ __align__(16) unsigned char smem[];
  ClauseLP* s_cl = reinterpret_cast<ClauseLP*>(smem);
  float2* s_pt = reinterpret_cast<float2*>(smem + 16 * m);
  const size_t off = 16u * m + ((8u * (m + 1) + 15u) & ~15u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* s_tile = reinterpret_cast<float2*>(smem + off) + warp * kLpTileSlots;
  uint2* s_act = reinterpret_cast<uint2*>(smem + off + 8u * kLpTileSlots * kLpWarps) + warp * (m + 16);

  for (int i = threadIdx.x; i < m; i += blockDim.x) s_cl[i] = cl[i];
  const float fd = fold_factor_block(nf);  // norm correction c - 1 of the previous step (0 if none)
  for (int i = threadIdx.x; i <= m; i += blockDim.x)
    s_pt[i] = fold_apply(prow[i], fd);
  __syncthreads();

  DFloat nacc{0.f, 0.f};
  const long long step = static_cast<long long>(gridDim.x) * kLpWarps;
  for (long long tile = static_cast<long long>(blockIdx.x) * kLpWarps + warp; tile < ntiles; tile += step) {
    float2* g = psi + (tile << kLowBits);
    // Fold the clause list against this tile's high bits and count the active
    // clauses for all 32 register slots before the tile is loaded, so that the
    // counters and the amplitudes are never live at the same time.
    int nconst, npad;
    unsigned pl[kPlanes];
    __syncwarp();
    fold_tile<KIND != kLpFirst>(s_cl, m, static_cast<unsigned>(tile), lane, s_act, nconst, npad);
    count_active(s_act, npad, 1u << lane, pl);
    float2 v[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = g[lane + 32 * r];
    if (KIND == kLpFirst) {
      // P(theta_0) first (layout X: registers hold bits 5..9), then W over bits 0..9.
      apply_p_phase(v, pl, nconst, s_pt);
      reg_wht<0, 5>(v);
      xpose_x2y(v, s_tile, lane);
      reg_wht<0, 5>(v);
      xpose_y2x(v, s_tile, lane);
    } else {
      // W over bits 0..9, then P (layout Y: registers hold bits 0..4), then W again (merge).
      reg_wht<0, 5>(v);
      xpose_x2y(v, s_tile, lane);
      reg_wht<0, 5>(v);
      apply_p_phase(v, pl, nconst, s_pt);
      if (KIND == kLpMerge) reg_wht<0, 5>(v);
      xpose_y2x(v, s_tile, lane);
      if (KIND == kLpMerge) reg_wht<0, 5>(v);
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) g[lane + 32 * r] = v[r];
    if (nf.out) nacc = df_add1(nacc, tile_norm(v));
  }
  fold_store(nf, nacc);
}

// ---------------------------------------------------------------------------
// strided pass over active bits [a, a+Q) (5 <= Q <= 10), keeping the C lowest
// index bits inside the tile so that every global access covers 2^C
// consecutive amplitudes (8 * 2^C bytes).  Tile = 2^(Q+C) amplitudes, NT =
// 2^(Q+C-5) threads, 32 registers each.
// Layout A: register = i bits 0..4, thread = (j = low C bits, i bits 5..Q-1).
// Layout B: register = i bits Q-5..Q-1, thread = (j, i bits 0..Q-6).
// Shared slot of tile index t = j + (i << C): t + 2^C (t >> (C+5)), i.e. rows of
// 2^(C+5) amplitudes padded by 2^C.  Layout A writes then hit 32 distinct bank
// pairs per warp access; layout B reads are contiguous.  Both use base +
// immediate addressing.
__host__ __device__ constexpr int sp_c(int q) { return (10 - q) > 3 ? (10 - q) : 3; }

template <int Q, int C>
struct SpGeom {
  static constexpr int QB = Q - 5;
  static constexpr int NT = 1 << (Q + C - 5);
  static constexpr int TILE = 1 << (Q + C);
  static constexpr int SLOTS = TILE + (TILE >> 5);
  __host__ __device__ static constexpr int slot(int t) { return t + ((t >> (C + 5)) << C); }
};

template <int Q, int C, bool WBW>
__global__ void __launch_bounds__(SpGeom<Q, C>::NT, (SpGeom<Q, C>::NT >= 256 ? 2 : 4))
    sp_kernel(float2* __restrict__ psi, int n, int a, const float2* __restrict__ brow, long long ntiles) {
  using G = SpGeom<Q, C>;
  constexpr int QB = G::QB;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* s_tile = reinterpret_cast<float2*>(smem);
  float2* s_bt = s_tile + G::SLOTS;
  if (WBW) {
    for (int i = threadIdx.x; i <= n; i += blockDim.x) s_bt[i] = brow[i];
    __syncthreads();
  }
  const int tid = threadIdx.x;
  const int j = tid & ((1 << C) - 1);
  const int th = tid >> C;
  const unsigned long long lo_mask = (1ull << (a - C)) - 1ull;
  const unsigned long long stride = 1ull << a;
  // shared-memory bases: layout A slot(j + (r << C) + (th << (C+5))) = sa + slot(r << C);
  // layout B slot(j + (th << C) + (r << (QB+C))) = sb + slot(r << (QB+C)) (th < 2^QB, so
  // the row index (t >> (C+5)) of layout B depends on r and on th >> 5 only).
  const int sa = j + (th << (C + 5)) + (th << C);
  const int sb = G::slot(j + (th << C));

  for (long long T = blockIdx.x; T < ntiles; T += gridDim.x) {
    const unsigned long long ut = static_cast<unsigned long long>(T);
    const unsigned long long xbase = ((ut & lo_mask) << C) | ((ut >> (a - C)) << (a + Q));
    float2* g = psi + xbase + j;
    float2 v[32];
    // layout A: element r at g + (r + 32 th) 2^a, walked with one pointer
    {
      const float2* pa = g + (static_cast<unsigned long long>(th) << (a + 5));
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        v[r] = *pa;
        pa += stride;
      }
    }
    reg_wht<0, 5>(v);
    if (QB > 0) {
#pragma unroll
      for (int r = 0; r < 32; ++r) s_tile[sa + G::slot(r << C)] = v[r];
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = s_tile[sb + G::slot((r << QB) << C) - G::slot(0)];
      __syncthreads();
      reg_wht<10 - Q, 5>(v);  // i bits 5..Q-1 are register bits 10-Q..4 in layout B
    }
    if (WBW) {
      // 2^-n exp(-i phi popcount(x)) with x the full index (all bits in the Hadamard basis)
      const int pc0 = __popcll(xbase) + __popc(j) + __popc(th);
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = cmul(v[r], s_bt[pc0 + __popc(r)]);
      if (QB > 0) {
        reg_wht<10 - Q, 5>(v);
#pragma unroll
        for (int r = 0; r < 32; ++r) s_tile[sb + G::slot((r << QB) << C) - G::slot(0)] = v[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = s_tile[sa + G::slot(r << C)];
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
      // layout B (or A when Q == 5): element r at g + (th + (r << QB)) 2^a
      float2* pb = g + (static_cast<unsigned long long>(th) << a);
      const unsigned long long sb = stride << QB;
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        *pb = v[r];
        pb += sb;
      }
    }
  }
}

// ---------------------------------------------------------------------------
__global__ void stamp_kernel(unsigned long long* __restrict__ stamp) { *stamp = global_ns(); }

__global__ void init_uniform_kernel(float2* __restrict__ psi, unsigned long long count, float val) {
  const float2 z = make_float2(val, 0.0f);
  for (unsigned long long x = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x; x < count;
       x += static_cast<unsigned long long>(gridDim.x) * blockDim.x)
    psi[x] = z;
}

// Phase-table entries.  P row at boundary position p of a range [k0, k1) of a
// K-step run (p = 0 before step k0, p = k1 - k0 after the last step):
//   theta_p = dt/2 ( s_(k0+p-1) [p >= 1] + s_(k0+p) [p < k1-k0] ),  entry E: exp(-i theta_p E)
// B row of step k:  entry q: 2^-n exp(-i dt (1 - s_k) q)
// s_k = (k + 1/2)/K, or s_dev[k] for a caller-supplied schedule.  FP64 angles,
// FP64 sine/cosine, one rounding to FP32 per entry.  Every producer of phase
// rows (the chunk tables below, the per-iteration rows of a launch graph)
// calls these two functions, so the rows are identical whichever produced them.
__device__ __forceinline__ double sched_s(const double* s_dev, long long K, long long k) {
  return s_dev ? s_dev[k] : (static_cast<double>(k) + 0.5) / static_cast<double>(K);
}

// With dt_dev (sub-steps of individual length, e.g. the fourth-order triple
// jump) the two half phases are weighted by their own lengths:
//   theta_p = 1/2 ( dt_(k0+p-1) s_(k0+p-1) [p >= 1] + dt_(k0+p) s_(k0+p) [p < k1-k0] ).
__device__ __noinline__ float2 p_entry(double dt, const double* dt_dev, const double* s_dev, long long K, long long k0,
                                       long long k1, long long p, int e) {
  double th = 0.0;
  if (dt_dev) {
    if (p >= 1) th += dt_dev[k0 + p - 1] * sched_s(s_dev, K, k0 + p - 1);
    if (p < k1 - k0) th += dt_dev[k0 + p] * sched_s(s_dev, K, k0 + p);
    th *= 0.5;
  } else {
    if (p >= 1) th += sched_s(s_dev, K, k0 + p - 1);
    if (p < k1 - k0) th += sched_s(s_dev, K, k0 + p);
    th *= 0.5 * dt;
  }
  double sn, cs;
  sincos(th * static_cast<double>(e), &sn, &cs);
  return make_float2(static_cast<float>(cs), static_cast<float>(-sn));
}

// With rot set (rotation form) the row instead holds exp(-i dt (1 - s_k) q)
// unscaled for q = 0..6, the rest zero: the per-block popcount phases of the
// rotation form's 5- and 6-qubit Walsh-Hadamard sandwiches.
__device__ __noinline__ float2 b_entry(double dt, const double* dt_dev, const double* s_dev, long long K, long long k,
                                       int q, double scale, int rot) {
  const double s = sched_s(s_dev, K, k);
  if (dt_dev) dt = dt_dev[k];
  if (rot) {
    if (q > 6) return make_float2(0.f, 0.f);
    scale = 1.0;
  }
  const double ph = dt * (1.0 - s) * static_cast<double>(q);
  double sn, cs;
  sincos(ph, &sn, &cs);
  return make_float2(static_cast<float>(scale * cs), static_cast<float>(-scale * sn));
}

// Phase tables for the steps c0 <= k < c1 of a range [k0, k1): P row rho is
// position p = c0 - k0 + rho, B row rho is step k = c0 + rho.
__global__ void tables_kernel(float2* __restrict__ ptab, float2* __restrict__ btab, int n, int m, double dt,
                              const double* __restrict__ dt_dev, const double* __restrict__ s_dev, long long K,
                              long long k0, long long k1, long long c0, long long c1, double scale, int rot) {
  const long long prow_n = c1 - c0 + 1, brow_n = c1 - c0;
  const long long np = prow_n * (m + 1), nb = brow_n * (n + 1);
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < np + nb;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    if (i < np) {
      const long long rho = i / (m + 1);
      const int e = static_cast<int>(i - rho * (m + 1));
      ptab[i] = p_entry(dt, dt_dev, s_dev, K, k0, k1, c0 - k0 + rho, e);
    } else {
      const long long j = i - np;
      const long long rho = j / (n + 1);
      const int q = static_cast<int>(j - rho * (n + 1));
      btab[j] = b_entry(dt, dt_dev, s_dev, K, c0 + rho, q, scale, rot);
    }
  }
}

// Rows for a launch graph: P positions p_first + j into rows dst_p0 + j of
// prow (j < nprow), B rows of steps k_first + j into rows j of brow (j <
// nbrow); with ctr non-null both starts are offset by *ctr (the graph's loop
// counter, read by every thread; nothing here writes it).
__global__ void graph_rows_kernel(float2* __restrict__ prow, int dst_p0, long long p_first, int nprow,
                                  float2* __restrict__ brow, long long k_first, int nbrow,
                                  const long long* __restrict__ ctr, int n, int m, double dt,
                                  const double* __restrict__ dt_dev, const double* __restrict__ s_dev, long long K,
                                  long long k0, long long k1, double scale, int rot) {
  const long long off = ctr ? *ctr : 0;
  const long long np = static_cast<long long>(nprow) * (m + 1), nb = static_cast<long long>(nbrow) * (n + 1);
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < np + nb;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    if (i < np) {
      const long long j = i / (m + 1);
      const int e = static_cast<int>(i - j * (m + 1));
      prow[(dst_p0 + j) * (m + 1) + e] = p_entry(dt, dt_dev, s_dev, K, k0, k1, p_first + off + j, e);
    } else {
      const long long t = i - np;
      const long long j = t / (n + 1);
      const int q = static_cast<int>(t - j * (n + 1));
      brow[t] = b_entry(dt, dt_dev, s_dev, K, k_first + off + j, q, scale, rot);
    }
  }
}

// The last node of a graph loop body: advance the counter by `step` and keep
// looping while it is below `limit`.  The counter only grows, so the loop ends
// after at most limit / step iterations.
__global__ void graph_advance_kernel(long long* ctr, long long step, long long limit, cudaGraphConditionalHandle h) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const long long c = *ctr + step;
    *ctr = c;
    cudaGraphSetConditional(h, (c >= 0 && c < limit) ? 1u : 0u);
  }
}

// ---------------------------------------------------------------------------
template <int Q>
static cudaError_t launch_sp(const LaunchCtx& lc, float2* psi, int n, int a, bool wbw, const float2* brow) {
  constexpr int C = sp_c(Q);
  using G = SpGeom<Q, C>;
  const long long ntiles = 1ll << (n - Q - C);
  const size_t smem = static_cast<size_t>(G::SLOTS) * 8u + static_cast<size_t>(n + 1) * 8u;
  auto kern = wbw ? sp_kernel<Q, C, true> : sp_kernel<Q, C, false>;
  cudaError_t err = allow_smem(reinterpret_cast<const void*>(kern), static_cast<size_t>(G::SLOTS) * 8u + 64u * 8u);
  if (err != cudaSuccess) return err;
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, G::NT, smem);
  if (err != cudaSuccess) return err;
  if (occ < 1) occ = 1;
  long long grid = static_cast<long long>(occ) * lc.num_sms;
  if (grid > ntiles) grid = ntiles;
  kern<<<static_cast<unsigned>(grid), G::NT, smem, lc.stream>>>(psi, n, a, brow, ntiles);
  return cudaGetLastError();
}

template <int KIND>
static cudaError_t launch_lp(const LaunchCtx& lc, float2* psi, int n, int m, const ClauseLP* cl, const float2* prow,
                            const NormFold& nf) {
  const long long ntiles = 1ll << (n - kLowBits);
  const size_t smem = lp_smem_bytes(m);
  auto kern = lp_kernel<KIND>;
  cudaError_t err = allow_smem(reinterpret_cast<const void*>(kern), lp_smem_bytes(QAA_MAX_CLAUSES_DEV));
  if (err != cudaSuccess) return err;
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kLpWarps * 32, smem);
  if (err != cudaSuccess) return err;
  if (occ < 1) occ = 1;
  long long grid = static_cast<long long>(occ) * lc.num_sms;
  const long long need = (ntiles + kLpWarps - 1) / kLpWarps;
  if (grid > need) grid = need;
  if (grid > kFoldSlot - 1) grid = kFoldSlot - 1;  // one norm-fold partial per CTA
  kern<<<static_cast<unsigned>(grid), kLpWarps * 32, smem, lc.stream>>>(psi, m, cl, prow, ntiles, nf);
  return cudaGetLastError();
}

cudaError_t launch_pass(const LaunchCtx& lc, const Pass& p, float2* psi, int n, int m, const ClauseLP* cl,
                        const float2* ptab, const float2* btab, const NormFold& nf) {
  switch (p.kind) {
    case kLpFirst: return launch_lp<kLpFirst>(lc, psi, n, m, cl, ptab + static_cast<size_t>(p.prow) * (m + 1), nf);
    case kLpMerge: return launch_lp<kLpMerge>(lc, psi, n, m, cl, ptab + static_cast<size_t>(p.prow) * (m + 1), nf);
    case kLpLast: return launch_lp<kLpLast>(lc, psi, n, m, cl, ptab + static_cast<size_t>(p.prow) * (m + 1), nf);
    case kSpW:
    case kSpWBW: {
      const bool wbw = p.kind == kSpWBW;
      const float2* brow = btab + static_cast<size_t>(p.brow) * (n + 1);
      switch (p.q) {
        case 5: return launch_sp<5>(lc, psi, n, p.a, wbw, brow);
        case 6: return launch_sp<6>(lc, psi, n, p.a, wbw, brow);
        case 7: return launch_sp<7>(lc, psi, n, p.a, wbw, brow);
        case 8: return launch_sp<8>(lc, psi, n, p.a, wbw, brow);
        case 9: return launch_sp<9>(lc, psi, n, p.a, wbw, brow);
        case 10: return launch_sp<10>(lc, psi, n, p.a, wbw, brow);
        default: return cudaErrorInvalidValue;
      }
    }
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stamp(const LaunchCtx& lc, unsigned long long* stamp) {
  stamp_kernel<<<1, 1, 0, lc.stream>>>(stamp);
  return cudaGetLastError();
}

cudaError_t launch_init_uniform(const LaunchCtx& lc, float2* psi, int n) {
  const unsigned long long count = 1ull << n;
  const float val = static_cast<float>(exp2(-0.5 * n));
  long long grid = (static_cast<long long>(count) + 255) / 256;
  const long long cap = 8ll * lc.num_sms;
  if (grid > cap) grid = cap;
  init_uniform_kernel<<<static_cast<unsigned>(grid), 256, 0, lc.stream>>>(psi, count, val);
  return cudaGetLastError();
}

cudaError_t launch_graph_rows(const LaunchCtx& lc, float2* prow, int dst_p0, long long p_first, int nprow, float2* brow,
                              long long k_first, int nbrow, const long long* ctr, int n, int m, double dt,
                              const double* s_dev, long long K, long long k0, long long k1, bool rot,
                              const double* dt_dev) {
  const long long total = static_cast<long long>(nprow) * (m + 1) + static_cast<long long>(nbrow) * (n + 1);
  long long grid = (total + 127) / 128;
  if (grid > 2ll * lc.num_sms) grid = 2ll * lc.num_sms;
  if (grid < 1) grid = 1;
  graph_rows_kernel<<<static_cast<unsigned>(grid), 128, 0, lc.stream>>>(
      prow, dst_p0, p_first, nprow, brow, k_first, nbrow, ctr, n, m, dt, dt_dev, s_dev, K, k0, k1,
      exp2(-static_cast<double>(n)), rot ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_graph_advance(const LaunchCtx& lc, long long* ctr, long long step, long long limit,
                                 cudaGraphConditionalHandle h) {
  graph_advance_kernel<<<1, 32, 0, lc.stream>>>(ctr, step, limit, h);
  return cudaGetLastError();
}

cudaError_t launch_tables(const LaunchCtx& lc, float2* ptab, float2* btab, int n, int m, double dt,
                          const double* s_dev, long long K, long long k0, long long k1, long long c0, long long c1,
                          bool rot, const double* dt_dev) {
  const long long total = (c1 - c0 + 1) * (m + 1) + (c1 - c0) * (n + 1);
  long long grid = (total + 255) / 256;
  if (grid > 4ll * lc.num_sms) grid = 4ll * lc.num_sms;
  if (grid < 1) grid = 1;
  tables_kernel<<<static_cast<unsigned>(grid), 256, 0, lc.stream>>>(ptab, btab, n, m, dt, dt_dev, s_dev, K, k0, k1,
                                                                    c0, c1, exp2(-static_cast<double>(n)), rot ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace qaa
