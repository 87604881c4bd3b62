// TMA-pipelined streaming passes (n >= 15).  Same arithmetic as the passes in
// pass_kernels.cu; what changes is how the state moves between HBM and the SM.
//
// * Strided passes (W over a group of Q index bits, or W B W over the top
//   group): persistent CTAs, two dense 2^(Q+C)-amplitude tile buffers filled by
//   4-D cp.async.bulk.tensor loads that complete on an mbarrier.  While a tile
//   is transformed in registers, the TMA engine already fetches the tile after
//   next into the other buffer.  Results go straight from registers to HBM.
// * Low passes (W P W over bits 0..9): every warp owns two 8 KiB buffers filled
//   by 1-D cp.async.bulk copies; the clause fold and bit-sliced count for a tile
//   run while its data is still in flight.
//
// Every wait on an mbarrier is bounded; on expiry the kernel records an error
// word that the host reports as QAA_E_TIMEOUT, and all threads of the block (or
// lanes of the warp) leave together.
#include <cuda.h>

#include <cstdlib>

#include "device_common.cuh"

namespace qaa {

// ---------------------------------------------------------------- PTX -------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity to complete.
constexpr long long kWaitLimit = 1ll << 24;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

constexpr int kErrTimeout = 1;

// ------------------------------------------------------- strided pass -------
// Tile = 2^Q rows (active bits i, stride 2^a) x 2^C contiguous amplitudes j,
// written dense by the TMA engine at t = j + (i << C).
// Layout H: register r = i bits QB..QB+4 (QB = Q-5), thread = (j, i bits 0..QB-1):
//   reading the dense tile gives 32 consecutive amplitudes per warp access.
// Layout L: register r = i bits 0..4, thread = (j, i bits 5..Q-1).
// Once the tile is in registers the same buffer serves the transposes in a
// padded layout (rows of 2^(C+5) amplitudes padded by 2^C), and then receives
// the next tile while this one is stored: one buffer per CTA, several CTAs
// per SM, so the warps of other CTAs compute while a CTA waits for its load.
template <int Q, int C>
struct TmaGeom {
  static constexpr int QB = Q - 5;
  static constexpr int NT = 1 << (Q + C - 5);
  static constexpr int TILE = 1 << (Q + C);
  static constexpr int SLOTS = TILE + (TILE >> 5);
  __host__ __device__ static constexpr int slot(int t) { return t + ((t >> (C + 5)) << C); }
  static constexpr size_t off_bt = static_cast<size_t>(SLOTS) * 8;
  static constexpr size_t off_bar = off_bt + 64 * 8;  // room for n + 1 <= 64 entries
  static constexpr size_t smem = off_bar + 16;
};

__host__ __device__ constexpr int tma_c(int q) { return (10 - q) > 3 ? (10 - q) : 3; }

// Active bits: i bits 0..4 sit at index bits a1..a1+4 and i bits 5..Q-1 at
// a2..a2+Q-6 (a2 = a1 + 5 for a contiguous group; a split group, Q >= 10,
// takes a 5-bit range and a (Q-5)-bit range far apart so that the rows of one
// tile fall on fewer memory pages).  The tile's fixed bits are [C, a1),
// [a1+5, a2), [a2+Q-5, n).  Q = 11 (C = 3, 512 threads): the sixth bit of the
// layout-L stage is thread bit C, a lane bit, transformed by warp shuffles.
// MODE 0: W over the group; 1: W B W (the phase group); 2: the one-qubit
// rotations of exp(-i theta H_B) on the group's bits (rotation form: B row
// entries 0..6 = exp(-i theta p)), unnormalised by 2^Q.
//
// Butterflies over lane bit LB: (u, w) <- (u + w, u - w) across the two lanes.
template <int LB>
__device__ __forceinline__ void lane_wht(float2 (&v)[32], int lane) {
  const bool upper = (lane >> LB) & 1;
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const float px = __shfl_xor_sync(0xffffffffu, v[r].x, 1 << LB);
    const float py = __shfl_xor_sync(0xffffffffu, v[r].y, 1 << LB);
    v[r] = upper ? make_float2(px - v[r].x, py - v[r].y) : make_float2(v[r].x + px, v[r].y + py);
  }
}

// Layout-L stage over i bits 0..QB-1: registers hold i bits 0..4, a sixth bit
// (QB = 6) is lane bit C.  MODE 2 applies the rotation-form sandwich over all
// QB bits (its popcount counts the lane bit too).
template <int QB, int C, int MODE>
__device__ __forceinline__ void stage_l(float2 (&v)[32], const float2 (&rtab)[7], int lane) {
  if constexpr (QB <= 5) {
    if (MODE == 2) reg_rot<QB>(v, *reinterpret_cast<const float2(*)[6]>(&rtab)); else reg_wht<0, QB>(v);
  } else {
    static_assert(QB == 6 && C < 5, "a sixth layout-L bit must be a lane bit");
    reg_wht<0, 5>(v);
    lane_wht<C>(v, lane);
    if (MODE == 2) {
      const int hb = (lane >> C) & 1;
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = cmul(v[r], rtab[__builtin_popcount(r) + hb]);
      reg_wht<0, 5>(v);
      lane_wht<C>(v, lane);
    }
  }
}

template <int Q, int C, int MODE>
__global__ void __launch_bounds__(TmaGeom<Q, C>::NT, (TmaGeom<Q, C>::NT >= 512 ? 1 : (TmaGeom<Q, C>::NT >= 256 ? 3 : 4)))
    sp_tma_kernel(float2* __restrict__ psi, const __grid_constant__ CUtensorMap tmap, int n, int a1, int a2,
                  const float2* __restrict__ brow, long long ntiles, int* __restrict__ err) {
  using G = TmaGeom<Q, C>;
  constexpr int QB = G::QB;
  extern __shared__ __align__(1024) unsigned char smem[];
  float2* s_buf = reinterpret_cast<float2*>(smem);
  float2* s_bt = reinterpret_cast<float2*>(smem + G::off_bt);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + G::off_bar);

  const int tid = threadIdx.x;
  const int j = tid & ((1 << C) - 1);
  const int th = tid >> C;
  // tile index T -> (low, middle, high) fixed-bit fields
  const int lo_bits = a1 - C, mid_bits = a2 - a1 - 5;
  const unsigned long long lo_mask = (1ull << lo_bits) - 1ull, mid_mask = (1ull << mid_bits) - 1ull;
  const long long stride_t = gridDim.x;
  auto issue = [&](unsigned long long T) {
    mbar_expect_tx(s_bar, G::TILE * 8u);
    tma_load_5d(s_buf, &tmap, static_cast<int>((T & lo_mask) << C), 0, static_cast<int>((T >> lo_bits) & mid_mask), 0,
                static_cast<int>(T >> (lo_bits + mid_bits)), s_bar);
  };

  if (tid == 0) {
    mbar_init(s_bar, 1);
    fence_mbar_init();
  }
  constexpr bool WBW = MODE == 1;
  if (WBW) {
    for (int i = tid; i <= n; i += blockDim.x) s_bt[i] = brow[i];
  }
  float2 rtab[7];
#pragma unroll
  for (int p = 0; p < 7; ++p) rtab[p] = MODE == 2 ? brow[p] : make_float2(0.f, 0.f);
  const int lane = tid & 31;
  __syncthreads();
  if (tid == 0 && static_cast<long long>(blockIdx.x) < ntiles) issue(blockIdx.x);
  const int h_off = j + (th << C);                   // layout H in the dense tile
  const int sx_h = G::slot(j + (th << C));           // padded slot base, layout H
  const int sx_l = j + (th << (C + 5)) + (th << C);  // padded slot base, layout L
  const unsigned long long step_l = 1ull << a1;              // layout L: register r = i bits 0..4
  const unsigned long long step_h = 1ull << (a2 + QB - 5);    // layout H: register r = i bits QB..QB+4

  int it = 0;
  for (long long T = blockIdx.x; T < ntiles; T += stride_t, ++it) {
    const bool ok = mbar_wait_bounded(s_bar, static_cast<uint32_t>(it) & 1u);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(err, kErrTimeout);
      break;
    }
    const unsigned long long ut = static_cast<unsigned long long>(T);
    const unsigned long long xbase = ((ut & lo_mask) << C) | (((ut >> lo_bits) & mid_mask) << (a1 + 5)) |
                                     ((ut >> (lo_bits + mid_bits)) << (a2 + QB));
    float2 v[32];
    {
      const float2* src = s_buf + h_off;
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = src[(r << QB) << C];
    }
    if (MODE == 2) reg_rot<5>(v, *reinterpret_cast<const float2(*)[6]>(&rtab)); else reg_wht<0, 5>(v);  // i bits QB..QB+4
    // Passes that store from layout L (plain W and the rotation form) are done
    // with the buffer once layout L is read: the next tile's copy starts there,
    // before the second butterfly stage, instead of after it (measured at
    // n = 30: plain 3.08 -> 2.83 ms, rotation with 128-byte runs 2.70 ms).  A
    // rotation pass with three 256-thread CTAs per SM ran slower with the early
    // copy (3.67 -> 4.22 ms) and keeps the late one.
    constexpr bool kEarlyIssue = (MODE == 0 || (MODE == 2 && G::NT >= 512)) && QB > 0;
    auto issue_next = [&]() {
      __syncthreads();
      if (tid == 0) {
        const long long Tn = T + stride_t;
        if (Tn < ntiles) {
          fence_proxy_async();
          issue(static_cast<unsigned long long>(Tn));
        }
      }
    };
    if (QB > 0) {
      __syncthreads();  // dense tile fully read
#pragma unroll
      for (int r = 0; r < 32; ++r) s_buf[sx_h + G::slot((r << QB) << C)] = v[r];
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = s_buf[sx_l + (r << C)];
      if (kEarlyIssue) issue_next();
      stage_l<QB, C, MODE>(v, rtab, lane);  // i bits 0..QB-1
    }
    if (WBW) {
      // 2^-n exp(-i phi popcount(x)), x the full index
      const int pc0 = __popcll(xbase) + __popc(j) + __popc(th);
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = cmul(v[r], s_bt[pc0 + __popc(r)]);
      if (QB > 0) {
        stage_l<QB, C, 0>(v, rtab, lane);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 32; ++r) s_buf[sx_l + (r << C)] = v[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = s_buf[sx_h + G::slot((r << QB) << C)];
      }
      reg_wht<0, 5>(v);
    }
    // the buffer is free: fetch the next tile while this one is stored
    if (!kEarlyIssue) issue_next();
    if (WBW || QB == 0) {
      // layout H: i = th + (r << QB); th = i bits 0..QB-1: bits 0..4 lie at a1.., bit 5 (QB = 6) at a2
      float2* dst = psi + xbase + j + (static_cast<unsigned long long>(th & 31) << a1) +
                    (static_cast<unsigned long long>(th >> 5) << a2);
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        *dst = v[r];
        dst += step_h;
      }
    } else {
      // layout L: i = r + (th << 5); th = i bits 5..Q-1 lie at a2..
      float2* dst = psi + xbase + j + (static_cast<unsigned long long>(th) << a2);
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        *dst = v[r];
        dst += step_l;
      }
    }
  }
  // leave only when no copy issued by this block is still in flight
  if (tid == 0) {
    const long long T = blockIdx.x + static_cast<long long>(it) * stride_t;
    if (T < ntiles && !mbar_wait_bounded(s_bar, static_cast<uint32_t>(it) & 1u)) atomicExch(err, kErrTimeout);
  }
}

// ----------------------------------------------------------- low pass -------
// One 1024-amplitude tile per warp at a time, one buffer per warp: the TMA
// engine writes the tile dense, the warp reads it into registers (layout X),
// reuses the buffer for its two padded transposes, then asks for its next tile
// and folds and counts that tile's clauses while the copy is in flight.
constexpr int kLpRowT = 33;
constexpr int kLpSlotsT = 32 * kLpRowT;
constexpr int kLpTmaWarps = 8;

struct LpTmaLayout {
  size_t off_pt, off_warp, per_warp, off_bar, total;
  __host__ __device__ explicit LpTmaLayout(int m) {
    off_pt = 16u * static_cast<size_t>(m);
    off_warp = (off_pt + 8u * static_cast<size_t>(m + 1) + 127u) & ~static_cast<size_t>(127);
    per_warp = (8u * kLpSlotsT + 8u * static_cast<size_t>(m + 16) + 127u) & ~static_cast<size_t>(127);
    off_bar = off_warp + per_warp * kLpTmaWarps;
    total = off_bar + 8u * kLpTmaWarps;
  }
};

__device__ __forceinline__ void xpose_x2y_t(float2 (&v)[32], float2* __restrict__ s, int lane) {
  float2* w = s + lane;
#pragma unroll
  for (int r = 0; r < 32; ++r) w[kLpRowT * r] = v[r];
  __syncwarp();
  const float2* q = s + kLpRowT * lane;
#pragma unroll
  for (int r = 0; r < 32; ++r) v[r] = q[r];
  __syncwarp();
}
__device__ __forceinline__ void xpose_y2x_t(float2 (&v)[32], float2* __restrict__ s, int lane) {
  float2* w = s + kLpRowT * lane;
#pragma unroll
  for (int r = 0; r < 32; ++r) w[r] = v[r];
  __syncwarp();
  const float2* q = s + lane;
#pragma unroll
  for (int r = 0; r < 32; ++r) v[r] = q[kLpRowT * r];
  __syncwarp();
}

// KIND kLpPhase / kLpRot / kLpRot12: the rotation form (P alone; the
// rotations of bits 0..9, or 0..11 with warp quads, then 2^-n P), with B row
// entries 0..5 = exp(-i theta p).
// Stored per-tile counts: load_counts (device_common.cuh).

// Warp quads (kLpRot12): warps 4k..4k+3 of a CTA sync on named barrier 1 + k
// (immediate ids, so that only barriers 0..2 are reserved).
template <int ID>
__device__ __forceinline__ bool quad_any_id(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, 128, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(v)), "n"(ID)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ bool quad_any(bool v, int quad) { return quad ? quad_any_id<2>(v) : quad_any_id<1>(v); }
__device__ __forceinline__ void quad_sync(int quad) {
  if (quad)
    asm volatile("bar.sync 2, 128;" ::: "memory");
  else
    asm volatile("bar.sync 1, 128;" ::: "memory");
}

// exp(-i theta H_B) on index bits 10 and 11 of four 1024-amplitude tiles held
// in the quad's shared buffers (tile k of the quad = bits 10..11 equal to k):
// W diag(exp(-i theta popcount)) W on the two bits, up to the factor 4.
__device__ __forceinline__ void quad_rot2(float2* const (&b)[4], const float2 (&tab)[6], int t) {
#pragma unroll 2
  for (int o = t; o < 1024; o += 128) {
    float2 a0 = b[0][o], a1 = b[1][o], a2 = b[2][o], a3 = b[3][o];
    butterfly(a0, a1);
    butterfly(a2, a3);
    butterfly(a0, a2);
    butterfly(a1, a3);
    a0 = cmul(a0, tab[0]);
    a1 = cmul(a1, tab[1]);
    a2 = cmul(a2, tab[1]);
    a3 = cmul(a3, tab[2]);
    butterfly(a0, a1);
    butterfly(a2, a3);
    butterfly(a0, a2);
    butterfly(a1, a3);
    b[0][o] = a0;
    b[1][o] = a1;
    b[2][o] = a2;
    b[3][o] = a3;
  }
}

template <int KIND>
__global__ void __launch_bounds__(kLpTmaWarps * 32, 2)
    lp_tma_kernel(float2* __restrict__ psi, int m, const ClauseLP* __restrict__ cl, const float2* __restrict__ prow,
                  const float2* __restrict__ brow, int n, long long ntiles, int* __restrict__ err,
                  const unsigned* __restrict__ counts, const NormFold nf) {
  constexpr bool kRegLow = KIND != kLpFirst && KIND != kLpPhase;  // phase applied in layout Y
  extern __shared__ __align__(1024) unsigned char smem[];
  const LpTmaLayout L(m);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  ClauseLP* s_cl = reinterpret_cast<ClauseLP*>(smem);
  float2* s_pt = reinterpret_cast<float2*>(smem + L.off_pt);
  unsigned char* wbase = smem + L.off_warp + L.per_warp * warp;
  float2* s_buf = reinterpret_cast<float2*>(wbase);  // dense tile, then padded transposes
  uint2* s_act = reinterpret_cast<uint2*>(wbase + 8u * kLpSlotsT);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + L.off_bar) + warp;

  const long long step = static_cast<long long>(gridDim.x) * kLpTmaWarps;
  const long long first = static_cast<long long>(blockIdx.x) * kLpTmaWarps + warp;
  if (lane == 0) {
    mbar_init(s_bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (lane == 0 && first < ntiles) {
    mbar_expect_tx(s_bar, 8192u);
    bulk_load(s_buf, psi + (first << kLowBits), 8192u, s_bar);
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) s_cl[i] = cl[i];
  // the rotation form's last pass of a step also removes the 2^n of its rotations (exact)
  constexpr bool kRot = KIND == kLpRot || KIND == kLpRot12;
  constexpr bool kQuad = KIND == kLpRot12;
  // and every merged pass folds in the norm correction of the previous step
  const float fd = fold_factor_block(nf);
  const float psc = kRot ? __int_as_float((127 - n) << 23) : 1.0f;  // 2^-n exactly (n <= 34)
  for (int i = threadIdx.x; i <= m; i += blockDim.x) {
    const float2 pv = prow[i];
    s_pt[i] = fold_apply(make_float2(pv.x * psc, pv.y * psc), fd);
  }
  float2 rtab[6];
#pragma unroll
  for (int p = 0; p < 6; ++p) rtab[p] = kRot ? brow[p] : make_float2(0.f, 0.f);
  // kLpRot12: the quad's four tile buffers (tile first + k of the quad in warp 4q + k's buffer)
  const int quad = warp >> 2;
  float2* qbuf[4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    qbuf[k] = reinterpret_cast<float2*>(smem + L.off_warp + L.per_warp * (4 * quad + k));
  __syncthreads();

  int nconst = 0, npad = 0;
  unsigned pl[kPlanes];
  const bool stored = kRegLow && counts != nullptr;
  if (first < ntiles) {
    if (stored) {
      load_counts(counts, first, lane, pl, nconst);
    } else {
      fold_tile<kRegLow>(s_cl, m, static_cast<unsigned>(first), lane, s_act, nconst, npad);
      count_active(s_act, npad, 1u << lane, pl);
    }
  }
  int it = 0;
  DFloat nacc{0.f, 0.f};  // |psi|^2 of this lane's outputs (norm fold)
  for (long long tile = first; tile < ntiles; tile += step, ++it) {
    const bool ok = mbar_wait_bounded(s_bar, static_cast<uint32_t>(it) & 1u);
    // a quad leaves together (its four warps have the same tiles left)
    if (kQuad ? quad_any(!ok, quad) : __any_sync(0xffffffffu, !ok)) {
      if (lane == 0) atomicExch(err, kErrTimeout);
      break;
    }
    if (kQuad) {
      // all four tiles are in (the barrier above): bits 10..11 across them
      quad_rot2(qbuf, rtab, threadIdx.x & 127);
      fence_proxy_async();  // these writes precede the next bulk copies into the buffers
      quad_sync(quad);
    }
    float2 v[32];
    {
      const float2* src = s_buf + lane;
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = src[32 * r];
    }
    __syncwarp();
    if (KIND == kLpPhase) {
      apply_p_phase(v, pl, nconst, s_pt);
    } else if (kRot) {
      reg_rot<5>(v, rtab);
      xpose_x2y_t(v, s_buf, lane);
      reg_rot<5>(v, rtab);
      apply_p_phase(v, pl, nconst, s_pt);
      xpose_y2x_t(v, s_buf, lane);
    } else if (KIND == kLpFirst) {
      apply_p_phase(v, pl, nconst, s_pt);
      reg_wht<0, 5>(v);
      xpose_x2y_t(v, s_buf, lane);
      reg_wht<0, 5>(v);
      xpose_y2x_t(v, s_buf, lane);
    } else {
      reg_wht<0, 5>(v);
      xpose_x2y_t(v, s_buf, lane);
      reg_wht<0, 5>(v);
      apply_p_phase(v, pl, nconst, s_pt);
      if (KIND == kLpMerge) reg_wht<0, 5>(v);
      xpose_y2x_t(v, s_buf, lane);
      if (KIND == kLpMerge) reg_wht<0, 5>(v);
    }
    const long long tn = tile + step;
    if (lane == 0 && tn < ntiles) {
      fence_proxy_async();
      mbar_expect_tx(s_bar, 8192u);
      bulk_load(s_buf, psi + (tn << kLowBits), 8192u, s_bar);
    }
    float2* g = psi + (tile << kLowBits) + lane;
#pragma unroll
    for (int r = 0; r < 32; ++r) g[32 * r] = v[r];
    if (nf.out) nacc = df_add1(nacc, tile_norm(v));
    if (tn < ntiles) {
      if (stored) {
        load_counts(counts, tn, lane, pl, nconst);
      } else {
        __syncwarp();
        fold_tile<kRegLow>(s_cl, m, static_cast<unsigned>(tn), lane, s_act, nconst, npad);
        count_active(s_act, npad, 1u << lane, pl);
      }
    }
  }
  if (lane == 0) {
    const long long t = first + static_cast<long long>(it) * step;
    if (t < ntiles && !mbar_wait_bounded(s_bar, static_cast<uint32_t>(it) & 1u)) atomicExch(err, kErrTimeout);
  }
  fold_store(nf, nacc);
}

// ------------------------------------------------ correlation pass -------
// Read-only strided pass for the observables: the pair correlations
//   sum over x with bit i clear of Re(conj psi_x psi_(x + 2^i))
// of every index bit i of a contiguous group [a, a+Q), 5 <= Q <= 10 (the
// ground state and <H_B> of Sec. 2.1, gathered from every thread as in
// Sec. 4.2).  The tile and its layouts are those of sp_tma_kernel: in layout
// H the registers hold i bits QB..QB+4, in layout L i bits 0..4 (of which bits
// 0..QB-1 are new).  Products are summed in FP32 per thread and tile (at most
// 160 pairs), in FP64 beyond; one partial per CTA.
__device__ __forceinline__ unsigned long long pair_fma(const float2 (&v)[32], int b, unsigned long long c) {
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    if (!(r & (1 << b))) {
      const unsigned long long u = (static_cast<unsigned long long>(__float_as_uint(v[r].y)) << 32) |
                                   __float_as_uint(v[r].x);
      const unsigned long long w = (static_cast<unsigned long long>(__float_as_uint(v[r | (1 << b)].y)) << 32) |
                                   __float_as_uint(v[r | (1 << b)].x);
      asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(c) : "l"(u), "l"(w));
    }
  }
  return c;
}

template <int Q, int C>
__global__ void __launch_bounds__(TmaGeom<Q, C>::NT, (TmaGeom<Q, C>::NT >= 512 ? 1 : 3))
    corr_tma_kernel(const __grid_constant__ CUtensorMap tmap, int a1, int a2, long long ntiles,
                    double* __restrict__ partials, int nparts, int* __restrict__ err) {
  using G = TmaGeom<Q, C>;
  constexpr int QB = Q - 5;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ double s_red[32];
  float2* s_buf = reinterpret_cast<float2*>(smem);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + G::off_bar);
  const int tid = threadIdx.x;
  const int j = tid & ((1 << C) - 1);
  const int th = tid >> C;
  // tile index T -> (low, middle, high) fixed-bit fields, as sp_tma_kernel
  const int lo_bits = a1 - C, mid_bits = a2 - a1 - 5;
  const unsigned long long lo_mask = (1ull << lo_bits) - 1ull, mid_mask = (1ull << mid_bits) - 1ull;
  const long long stride_t = gridDim.x;
  auto issue = [&](unsigned long long T) {
    mbar_expect_tx(s_bar, G::TILE * 8u);
    tma_load_5d(s_buf, &tmap, static_cast<int>((T & lo_mask) << C), 0, static_cast<int>((T >> lo_bits) & mid_mask), 0,
                static_cast<int>(T >> (lo_bits + mid_bits)), s_bar);
  };
  if (tid == 0) {
    mbar_init(s_bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0 && static_cast<long long>(blockIdx.x) < ntiles) issue(blockIdx.x);
  const int h_off = j + (th << C);
  const int sx_h = G::slot(j + (th << C));
  const int sx_l = j + (th << (C + 5)) + (th << C);
  double acc = 0.0;
  int it = 0;
  for (long long T = blockIdx.x; T < ntiles; T += stride_t, ++it) {
    const bool ok = mbar_wait_bounded(s_bar, static_cast<uint32_t>(it) & 1u);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(err, kErrTimeout);
      break;
    }
    float2 v[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = s_buf[h_off + ((r << QB) << C)];
    unsigned long long c2 = 0ull;
#pragma unroll
    for (int b = 0; b < 5; ++b) c2 = pair_fma(v, b, c2);  // i bits QB..QB+4
    if (QB > 0) {
      __syncthreads();  // dense tile fully read
#pragma unroll
      for (int r = 0; r < 32; ++r) s_buf[sx_h + G::slot((r << QB) << C)] = v[r];
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = s_buf[sx_l + (r << C)];
    }
    __syncthreads();  // buffer free: the next tile's copy overlaps the rest of this one
    if (tid == 0 && T + stride_t < ntiles) {
      fence_proxy_async();
      issue(static_cast<unsigned long long>(T + stride_t));
    }
#pragma unroll
    for (int b = 0; b < 5; ++b)
      if (b < QB) c2 = pair_fma(v, b, c2);  // i bits 0..QB-1
    const float2 c = bits_f2(c2);
    acc += static_cast<double>(c.x + c.y);
  }
  if (tid == 0) {
    const long long T = blockIdx.x + static_cast<long long>(it) * stride_t;
    if (T < ntiles && !mbar_wait_bounded(s_bar, static_cast<uint32_t>(it) & 1u)) atomicExch(err, kErrTimeout);
  }
  // fixed-order block sum; CTAs beyond the grid's share write zero partials
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) s_red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += s_red[w];
    partials[blockIdx.x] = t;
    if (blockIdx.x == 0)
      for (int i = gridDim.x; i < nparts; ++i) partials[i] = 0.0;
  }
}

// ------------------------------------------------------------- host ---------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn lookup_encode() {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    return reinterpret_cast<EncodeTiledFn>(p);
  cudaGetLastError();
  return nullptr;
}

static EncodeTiledFn encode_fn() {
  static const EncodeTiledFn fn = lookup_encode();  // initialised once, thread safe
  return fn;
}

bool tma_available() { return encode_fn() != nullptr; }

// L2 sector promotion of the strided tiles' rows: 256 B for 128-byte runs,
// 128 B for 64-byte runs (measured at n = 30: the W.B.W phase pass 3.85 ms with
// 128 B against 3.99 ms with 256 B, which over-read DRAM by 11 %; 64 B: 5.6 ms).
// QAA_TMA_PROMO = 0 / 64 / 128 / 256 overrides it for every run length.
static CUtensorMapL2promotion l2_promotion(int c) {
  static const int env = [] {
    const char* v = std::getenv("QAA_TMA_PROMO");
    return v ? std::atoi(v) : -1;
  }();
  const int bytes = env >= 0 ? env : (c >= 4 ? 256 : 128);
  switch (bytes) {
    case 0: return CU_TENSOR_MAP_L2_PROMOTION_NONE;
    case 64: return CU_TENSOR_MAP_L2_PROMOTION_L2_64B;
    case 128: return CU_TENSOR_MAP_L2_PROMOTION_L2_128B;
    default: return CU_TENSOR_MAP_L2_PROMOTION_L2_256B;
  }
}

template <int Q, int C>
static cudaError_t launch_sp_tma_c(const LaunchCtx& lc, float2* psi, int n, int a1, int a2, int mode,
                                   const float2* brow, int* err) {
  using G = TmaGeom<Q, C>;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  constexpr int QB = Q - 5;
  if (a1 < C || a2 < a1 + 5 || a2 + QB > n || (a2 != a1 + 5 && QB < 5)) return cudaErrorInvalidValue;
  CUtensorMap map;
  // dims (innermost first): bits [0,a1), [a1,a1+5), [a1+5,a2), [a2,a2+QB), [a2+QB,n)
  const cuuint64_t dims[5] = {1ull << a1, 32ull, 1ull << (a2 - a1 - 5), 1ull << QB, 1ull << (n - a2 - QB)};
  const cuuint64_t strides[4] = {(1ull << a1) * 8ull, (1ull << (a1 + 5)) * 8ull, (1ull << a2) * 8ull,
                                 (1ull << (a2 + QB)) * 8ull};
  const cuuint32_t box[5] = {1u << C, 32u, 1u, 1u << QB, 1u};
  const cuuint32_t estr[5] = {1u, 1u, 1u, 1u, 1u};
  const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, psi, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, l2_promotion(C),
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const long long ntiles = 1ll << (n - Q - C);
  auto kern = mode == 1 ? sp_tma_kernel<Q, C, 1> : (mode == 2 ? sp_tma_kernel<Q, C, 2> : sp_tma_kernel<Q, C, 0>);
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(kern), G::smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, G::NT, G::smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  long long grid = static_cast<long long>(occ) * lc.num_sms;
  if (grid > ntiles) grid = ntiles;
  kern<<<static_cast<unsigned>(grid), G::NT, G::smem, lc.stream>>>(psi, map, n, a1, a2, brow, ntiles, err);
  return cudaGetLastError();
}

// The correlation pass over the bits [a, a+5) and [a2, a2+q-5) (a2 = a + 5 for
// a contiguous group; 5 <= q <= 10, a >= 10): one partial per CTA in
// partials[0 .. nparts).  Tiles of 2^q rows x 2^C contiguous amplitudes,
// C = max(10 - q, 3) as in the strided passes, so that a tile has at least
// 2^10 amplitudes and a CTA at least one whole warp.
template <int Q>
static cudaError_t launch_corr_q(const LaunchCtx& lc, const float2* psi, int n, int a, int a2, double* partials,
                                 int nparts, int* err) {
  constexpr int C = tma_c(Q);
  using G = TmaGeom<Q, C>;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  constexpr int QB = Q - 5;
  if (a < C || a2 < a + 5 || a2 + QB > n || (a2 != a + 5 && QB < 5)) return cudaErrorInvalidValue;
  CUtensorMap map;
  // dims (innermost first): bits [0,a), [a,a+5), [a+5,a2), [a2,a2+QB), [a2+QB,n)
  const cuuint64_t dims[5] = {1ull << a, 32ull, 1ull << (a2 - a - 5), 1ull << QB, 1ull << (n - a2 - QB)};
  const cuuint64_t strides[4] = {(1ull << a) * 8ull, (1ull << (a + 5)) * 8ull, (1ull << a2) * 8ull,
                                 (1ull << (a2 + QB)) * 8ull};
  const cuuint32_t box[5] = {1u << C, 32u, 1u, 1u << QB, 1u};
  const cuuint32_t estr[5] = {1u, 1u, 1u, 1u, 1u};
  const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, const_cast<float2*>(psi), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, l2_promotion(C),
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const long long ntiles = 1ll << (n - Q - C);
  auto kern = corr_tma_kernel<Q, C>;
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(kern), G::smem);
  if (e != cudaSuccess) return e;
  long long grid = nparts;
  if (grid > ntiles) grid = ntiles;
  kern<<<static_cast<unsigned>(grid), G::NT, G::smem, lc.stream>>>(map, a, a2, ntiles, partials, nparts, err);
  return cudaGetLastError();
}

cudaError_t launch_corr_tma(const LaunchCtx& lc, const float2* psi, int n, int a, int a2, int q, double* partials,
                            int nparts, int* err) {
  switch (q) {
    case 5: return launch_corr_q<5>(lc, psi, n, a, a2, partials, nparts, err);
    case 6: return launch_corr_q<6>(lc, psi, n, a, a2, partials, nparts, err);
    case 7: return launch_corr_q<7>(lc, psi, n, a, a2, partials, nparts, err);
    case 8: return launch_corr_q<8>(lc, psi, n, a, a2, partials, nparts, err);
    case 9: return launch_corr_q<9>(lc, psi, n, a, a2, partials, nparts, err);
    case 10: return launch_corr_q<10>(lc, psi, n, a, a2, partials, nparts, err);
    default: return cudaErrorInvalidValue;
  }
}

// Contiguous run per tile row: 2^C amplitudes.  C = 4 (128-byte runs) can be
// requested for groups whose rows lie far apart in memory (see the pass plan).
template <int Q>
static cudaError_t launch_sp_tma(const LaunchCtx& lc, float2* psi, int n, int a1, int a2, int mode,
                                 const float2* brow, int* err, int c_req) {
  constexpr int C0 = tma_c(Q);
  if constexpr (Q <= 10) {  // an 11-bit tile with 128-byte runs would not fit in shared memory
    if (c_req == 4 && C0 < 4 && a1 >= 4)
      return launch_sp_tma_c<Q, (C0 < 4 ? 4 : C0)>(lc, psi, n, a1, a2, mode, brow, err);
  }
  return launch_sp_tma_c<Q, C0>(lc, psi, n, a1, a2, mode, brow, err);
}

int tma_run_bytes(int q, int run_c) {
  const int c = (q <= 10 && run_c == 4 && tma_c(q) < 4) ? 4 : tma_c(q);
  return 8 << c;
}

// The stored counts of every tile (layout Y), computed once per instance in
// two launches of the same fold and count: MEASURE raises the header's plane
// count P to the bits of the largest count any lane holds, then the second
// launch stores P planes and the constant part of every tile.
template <bool MEASURE>
__global__ void __launch_bounds__(kLpTmaWarps * 32)
    lp_counts_kernel(int m, const ClauseLP* __restrict__ cl, unsigned* __restrict__ counts, long long ntiles,
                     unsigned planes_off) {
  extern __shared__ __align__(16) unsigned char smem[];
  ClauseLP* s_cl = reinterpret_cast<ClauseLP*>(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint2* s_act = reinterpret_cast<uint2*>(smem + 16u * m) + warp * (m + 16);
  for (int i = threadIdx.x; i < m; i += blockDim.x) s_cl[i] = cl[i];
  __syncthreads();
  const int P = MEASURE ? kPlanes : static_cast<int>(counts[0]);
  unsigned* planes = counts + planes_off;
  if (!MEASURE && blockIdx.x == 0 && threadIdx.x == 0) counts[1] = planes_off;
  unsigned used = 0u;  // OR of every plane word this lane computed, by plane
  for (long long tile = static_cast<long long>(blockIdx.x) * kLpTmaWarps + warp; tile < ntiles;
       tile += static_cast<long long>(gridDim.x) * kLpTmaWarps) {
    int nconst, npad;
    unsigned pl[kPlanes];
    __syncwarp();
    fold_tile<true>(s_cl, m, static_cast<unsigned>(tile), lane, s_act, nconst, npad);
    count_active(s_act, npad, 1u << lane, pl);
    if (MEASURE) {
#pragma unroll
      for (int b = 0; b < kPlanes; ++b) used |= pl[b] != 0u ? (1u << b) : 0u;
    } else {
      unsigned* c = planes + static_cast<size_t>(tile) * (32 * P) + lane;
#pragma unroll
      for (int b = 0; b < kPlanes; ++b)
        if (b < P) c[32 * b] = pl[b];
      if (lane == 0) counts[kCountHeaderWords + tile] = static_cast<unsigned>(nconst);
    }
  }
  if (MEASURE) {
    used = __reduce_or_sync(0xffffffffu, used);
    if (lane == 0 && used != 0u) atomicMax(counts, static_cast<unsigned>(32 - __clz(used)));
  }
}

static long long counts_planes_offset(long long ntiles) {
  return kCountHeaderWords + ((ntiles + 31) / 32) * 32;
}

size_t lp_counts_bytes(int n) {
  if (n <= kLowBits) return 0;
  const long long ntiles = 1ll << (n - kLowBits);
  return static_cast<size_t>(counts_planes_offset(ntiles) + ntiles * 32 * kPlanes) * sizeof(unsigned);
}

cudaError_t launch_lp_counts(const LaunchCtx& lc, unsigned* counts, int n, int m, const ClauseLP* cl) {
  const long long ntiles = 1ll << (n - kLowBits);
  const size_t smem = 16u * static_cast<size_t>(m) + static_cast<size_t>(kLpTmaWarps) * 8u * (m + 16);
  const size_t smem_max = 16u * QAA_MAX_CLAUSES_DEV + static_cast<size_t>(kLpTmaWarps) * 8u * (QAA_MAX_CLAUSES_DEV + 16);
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(lp_counts_kernel<true>), smem_max);
  if (e == cudaSuccess) e = allow_smem(reinterpret_cast<const void*>(lp_counts_kernel<false>), smem_max);
  if (e != cudaSuccess) return e;
  // the header's P is raised from 0 by the first launch; the second writes the planes' offset
  e = cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned), lc.stream);
  if (e != cudaSuccess) return e;
  const unsigned off = static_cast<unsigned>(counts_planes_offset(ntiles));
  long long grid = (ntiles + kLpTmaWarps - 1) / kLpTmaWarps;
  if (grid > 4ll * lc.num_sms) grid = 4ll * lc.num_sms;
  lp_counts_kernel<true><<<static_cast<unsigned>(grid), kLpTmaWarps * 32, smem, lc.stream>>>(m, cl, counts, ntiles, off);
  lp_counts_kernel<false><<<static_cast<unsigned>(grid), kLpTmaWarps * 32, smem, lc.stream>>>(m, cl, counts, ntiles, off);
  return cudaGetLastError();
}

template <int KIND>
static cudaError_t launch_lp_tma(const LaunchCtx& lc, float2* psi, int n, int m, const ClauseLP* cl,
                                 const float2* prow, const float2* brow, int* err, const unsigned* counts,
                                 const NormFold& nf) {
  const long long ntiles = 1ll << (n - kLowBits);
  const LpTmaLayout L(m);
  auto kern = lp_tma_kernel<KIND>;
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(kern), LpTmaLayout(QAA_MAX_CLAUSES_DEV).total);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kLpTmaWarps * 32, L.total);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  long long grid = static_cast<long long>(occ) * lc.num_sms;
  const long long need = (ntiles + kLpTmaWarps - 1) / kLpTmaWarps;
  if (grid > need) grid = need;
  if (grid > kFoldSlot - 1) grid = kFoldSlot - 1;  // one norm-fold partial per CTA
  kern<<<static_cast<unsigned>(grid), kLpTmaWarps * 32, L.total, lc.stream>>>(psi, m, cl, prow, brow, n, ntiles,
                                                                              err, counts, nf);
  return cudaGetLastError();
}

cudaError_t launch_pass_tma(const LaunchCtx& lc, const Pass& p, float2* psi, int n, int m, const ClauseLP* cl,
                            const float2* ptab, const float2* btab, int* err, const unsigned* counts,
                            const NormFold& nf) {
  const int c_req = p.run_c;
  const float2* prow = ptab + static_cast<size_t>(p.prow) * (m + 1);
  const float2* brow = btab + static_cast<size_t>(p.brow) * (n + 1);
  switch (p.kind) {
    case kLpFirst: return launch_lp_tma<kLpFirst>(lc, psi, n, m, cl, prow, nullptr, err, nullptr, nf);
    case kLpMerge: return launch_lp_tma<kLpMerge>(lc, psi, n, m, cl, prow, nullptr, err, counts, nf);
    case kLpLast: return launch_lp_tma<kLpLast>(lc, psi, n, m, cl, prow, nullptr, err, counts, nf);
    case kLpPhase: return launch_lp_tma<kLpPhase>(lc, psi, n, m, cl, prow, nullptr, err, nullptr, nf);
    case kLpRot: return launch_lp_tma<kLpRot>(lc, psi, n, m, cl, prow, brow, err, counts, nf);
    case kLpRot12:
      if (n < 12) return cudaErrorInvalidValue;
      return launch_lp_tma<kLpRot12>(lc, psi, n, m, cl, prow, brow, err, counts, nf);
    case kSpW:
    case kSpWBW:
    case kSpRot: {
      const int wbw = p.kind == kSpWBW ? 1 : (p.kind == kSpRot ? 2 : 0);
      switch (p.q) {
        case 5: return launch_sp_tma<5>(lc, psi, n, p.a, p.a2, wbw, brow, err, c_req);
        case 6: return launch_sp_tma<6>(lc, psi, n, p.a, p.a2, wbw, brow, err, c_req);
        case 7: return launch_sp_tma<7>(lc, psi, n, p.a, p.a2, wbw, brow, err, c_req);
        case 8: return launch_sp_tma<8>(lc, psi, n, p.a, p.a2, wbw, brow, err, c_req);
        case 9: return launch_sp_tma<9>(lc, psi, n, p.a, p.a2, wbw, brow, err, c_req);
        case 10: return launch_sp_tma<10>(lc, psi, n, p.a, p.a2, wbw, brow, err, c_req);
        case 11: return launch_sp_tma<11>(lc, psi, n, p.a, p.a2, wbw, brow, err, c_req);
        default: return cudaErrorInvalidValue;
      }
    }
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qaa
