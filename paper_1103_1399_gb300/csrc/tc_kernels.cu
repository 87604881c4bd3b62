// Tensor-core variant of the streaming passes: every Walsh-Hadamard transform
// over a group of index bits is applied as 16 x 16 Hadamard blocks on the
// tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation) instead
// of FP32 butterflies.  The complex64 amplitudes are split exactly enough into
// BF16 parts, x = hi + mid + lo (three products, ~FP32 accuracy) or x = hi + lo
// (two products, ~16 mantissa bits); the +-1 Hadamard entries are exact in
// BF16, so only the splitting and the FP32 accumulation round.
//
// One MMA stage transforms 4 index bits K of a shared-memory tile.  The A
// operand holds data: row g (g = lane / 4) is the real part, row g + 8 the
// imaginary part, of the amplitude whose 3 "other" bits O equal g; column k is
// the value of the K bits.  B is the Hadamard block (two 16 x 8 halves).  With
// the m16n8k16 fragment layouts, lane (g, t = lane % 4) supplies the inputs at
// k = 2t, 2t+1, 2t+8, 2t+9 and receives the outputs at exactly those k, so a
// stage works in place: 4 shared loads, the split, 6 (or 4) MMAs, 4 stores per
// lane and block of 16 x 8 amplitudes.  A stage may apply the Hadamard to a
// subset of K only (identity on the rest), which covers groups whose size is
// not a multiple of 4.
//
// Tiles are read and written with plain coalesced loads/stores and staged in
// shared memory under an XOR swizzle of the low address bits chosen so that
// every stage's access pattern, and the load/store layouts, touch 16 distinct
// bank pairs per warp access (the minimum for 8-byte elements).
#include <cuda_bf16.h>

#include "device_common.cuh"

namespace qaa {

// ---------------------------------------------------------------- MMA -------
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const unsigned short a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
  const unsigned short b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
  return static_cast<unsigned>(a) | (static_cast<unsigned>(b) << 16);
}
__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Hadamard block restricted to the bits in `hmask` (identity on the other K
// bits): M[k][k'] = prod_{b in hmask} (-1)^(k_b k'_b) * prod_{b not in hmask} [k_b == k'_b].
__device__ __forceinline__ float hblock(int k, int kp, int hmask) {
  if (((k ^ kp) & ~hmask & 15) != 0) return 0.0f;
  return (__popc(k & kp & hmask) & 1) ? -1.0f : 1.0f;
}

struct HFrag {
  unsigned b[2][2];  // [half][reg]
  __device__ __forceinline__ void init(int hmask, int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int col = 8 * h + g;
      b[h][0] = pack_bf16(hblock(2 * t, col, hmask), hblock(2 * t + 1, col, hmask));
      b[h][1] = pack_bf16(hblock(2 * t + 8, col, hmask), hblock(2 * t + 9, col, hmask));
    }
  }
};

// In-place transform of one 16 (K) x 8 (O) block of complex amplitudes.
// p[q] (q = 0..3) points at the amplitude with k = 2t, 2t+1, 2t+8, 2t+9.
// The tensor cores' FP32 accumulation drops low-order bits when small products
// are aligned to a large accumulator (a bias toward zero), so the hi part and
// the small parts (lo first, then mid) accumulate separately and are combined
// with one round-to-nearest FP32 addition.
template <int PARTS>
__device__ __forceinline__ void tc_block(float2* p0, float2* p1, float2* p2, float2* p3, const HFrag& H) {
  const float2 x0 = *p0, x1 = *p1, x2 = *p2, x3 = *p3;
  const float re[4] = {x0.x, x1.x, x2.x, x3.x}, im[4] = {x0.y, x1.y, x2.y, x3.y};
  float part_r[PARTS][4], part_i[PARTS][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float rr = re[q], ri = im[q];
#pragma unroll
    for (int p = 0; p < PARTS; ++p) {
      part_r[p][q] = (p == PARTS - 1) ? rr : bf16_round(rr);
      part_i[p][q] = (p == PARTS - 1) ? ri : bf16_round(ri);
      rr -= part_r[p][q];  // exact: the remainder of a round-to-nearest in FP32
      ri -= part_i[p][q];
    }
  }
  float h0[4] = {0.f, 0.f, 0.f, 0.f}, h1[4] = {0.f, 0.f, 0.f, 0.f};  // hi part
  float s0[4] = {0.f, 0.f, 0.f, 0.f}, s1[4] = {0.f, 0.f, 0.f, 0.f};  // small parts
#pragma unroll
  for (int p = PARTS - 1; p >= 0; --p) {
    // rows g (real) and g + 8 (imaginary); columns 2t, 2t+1 | 2t+8, 2t+9
    const unsigned a[4] = {pack_bf16(part_r[p][0], part_r[p][1]), pack_bf16(part_i[p][0], part_i[p][1]),
                           pack_bf16(part_r[p][2], part_r[p][3]), pack_bf16(part_i[p][2], part_i[p][3])};
    if (p == 0) {
      mma_bf16(h0, a, H.b[0][0], H.b[0][1]);
      mma_bf16(h1, a, H.b[1][0], H.b[1][1]);
    } else {
      mma_bf16(s0, a, H.b[0][0], H.b[0][1]);
      mma_bf16(s1, a, H.b[1][0], H.b[1][1]);
    }
  }
  *p0 = make_float2(h0[0] + s0[0], h0[2] + s0[2]);
  *p1 = make_float2(h0[1] + s0[1], h0[3] + s0[3]);
  *p2 = make_float2(h1[0] + s1[0], h1[2] + s1[2]);
  *p3 = make_float2(h1[1] + s1[1], h1[3] + s1[3]);
}

// ------------------------------------------------------- low pass (TC) ------
// Tile = 1024 consecutive amplitudes, one warp.  Stages: K = bits 0..3 (O =
// 4..6), K = bits 4..7 (O = 0..2), K = bits 6..9 with the Hadamard on 8, 9 only
// (O = 0..2).  Swizzle: address bits 0..3 XOR (t9^t4, t6, t7, t5^t8).
__device__ __forceinline__ int lp_swz(int t) {
  const int a0 = ((t >> 4) ^ (t >> 9)) & 1, a1 = (t >> 6) & 1, a2 = (t >> 7) & 1, a3 = ((t >> 5) ^ (t >> 8)) & 1;
  return t ^ (a0 | (a1 << 1) | (a2 << 2) | (a3 << 3));
}

template <int PARTS>
__device__ __forceinline__ void lp_tc_transform(float2* __restrict__ s, int lane, const HFrag& H4, const HFrag& H2) {
  const int g = lane >> 2, t = lane & 3;
  const int ks[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
  // stage 1: K = bits 0..3, O = bits 4..6, blocks = bits 7..9
#pragma unroll 1
  for (int blk = 0; blk < 8; ++blk) {
    const int base = (g << 4) | (blk << 7);
    tc_block<PARTS>(s + lp_swz(base | ks[0]), s + lp_swz(base | ks[1]), s + lp_swz(base | ks[2]),
                    s + lp_swz(base | ks[3]), H4);
  }
  __syncwarp();
  // stage 2: K = bits 4..7, O = bits 0..2, blocks = bits 3, 8, 9
#pragma unroll 1
  for (int blk = 0; blk < 8; ++blk) {
    const int base = g | ((blk & 1) << 3) | ((blk >> 1) << 8);
    tc_block<PARTS>(s + lp_swz(base | (ks[0] << 4)), s + lp_swz(base | (ks[1] << 4)), s + lp_swz(base | (ks[2] << 4)),
                    s + lp_swz(base | (ks[3] << 4)), H4);
  }
  __syncwarp();
  // stage 3: K = bits 6..9 (Hadamard on bits 8, 9), O = bits 0..2, blocks = bits 3..5
#pragma unroll 1
  for (int blk = 0; blk < 8; ++blk) {
    const int base = g | (blk << 3);
    tc_block<PARTS>(s + lp_swz(base | (ks[0] << 6)), s + lp_swz(base | (ks[1] << 6)), s + lp_swz(base | (ks[2] << 6)),
                    s + lp_swz(base | (ks[3] << 6)), H2);
  }
  __syncwarp();
}

constexpr int kTcWarps = 8;

template <int KIND, int PARTS>
__global__ void __launch_bounds__(kTcWarps * 32)
    lp_tc_kernel(float2* __restrict__ psi, int m, const ClauseLP* __restrict__ cl, const float2* __restrict__ prow,
                 long long ntiles) {
  extern __shared__ __align__(16) unsigned char smem[];
  ClauseLP* s_cl = reinterpret_cast<ClauseLP*>(smem);
  float2* s_pt = reinterpret_cast<float2*>(smem + 16 * m);
  const size_t off = 16u * m + ((8u * (m + 1) + 15u) & ~15u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* s_tile = reinterpret_cast<float2*>(smem + off) + warp * kLowTile;
  uint2* s_act = reinterpret_cast<uint2*>(smem + off + 8u * kLowTile * kTcWarps) + warp * (m + 16);
  for (int i = threadIdx.x; i < m; i += blockDim.x) s_cl[i] = cl[i];
  for (int i = threadIdx.x; i <= m; i += blockDim.x) s_pt[i] = prow[i];
  __syncthreads();
  HFrag H4, H2;
  H4.init(15, lane);
  H2.init(12, lane);  // bits 8, 9 are K bits 2, 3 of stage 3

  const long long step = static_cast<long long>(gridDim.x) * kTcWarps;
  for (long long tile = static_cast<long long>(blockIdx.x) * kTcWarps + warp; tile < ntiles; tile += step) {
    float2* g = psi + (tile << kLowBits);
    int nconst, npad;
    unsigned pl[kPlanes];
    __syncwarp();
    // P is applied with the registers holding bits 5..9 (layout X), as in the first low pass.
    fold_tile<false>(s_cl, m, static_cast<unsigned>(tile), lane, s_act, nconst, npad);
    count_active(s_act, npad, 1u << lane, pl);
    float2 v[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = g[lane + 32 * r];
    if (KIND == kLpFirst) apply_p_phase(v, pl, nconst, s_pt);
#pragma unroll
    for (int r = 0; r < 32; ++r) s_tile[lp_swz(lane + 32 * r)] = v[r];
    __syncwarp();
    lp_tc_transform<PARTS>(s_tile, lane, H4, H2);
    if (KIND != kLpFirst) {
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = s_tile[lp_swz(lane + 32 * r)];
      apply_p_phase(v, pl, nconst, s_pt);
      if (KIND == kLpMerge) {
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 32; ++r) s_tile[lp_swz(lane + 32 * r)] = v[r];
        __syncwarp();
        lp_tc_transform<PARTS>(s_tile, lane, H4, H2);
      }
    }
    if (KIND != kLpLast) {
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = s_tile[lp_swz(lane + 32 * r)];
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) g[lane + 32 * r] = v[r];
  }
}

// -------------------------------------------------- strided pass (TC) -------
// Tile t = j + (i << C): 2^Q rows i (active bits, i bits 0..4 at a1, 5..Q-1 at
// a2) x 2^C contiguous amplitudes j (C >= 3).  Stage list over i bits:
// [0,4) all new; [4,8) all new when Q >= 8; a last stage K = [Q-4, Q) with
// the Hadamard on the bits not yet transformed.  O = j bits 0..2.  Swizzle:
// address bit 3 XOR the parity of i bits in S, where S meets {b+1, b+2} of
// every stage start b (those two K bits vary across the lanes).
template <int Q, int C>
struct TcSp {
  static constexpr int NT = 256;
  static constexpr int TILE = 1 << (Q + C);
  static constexpr int S1 = 1, S2 = (Q >= 8) ? 5 : 1, S3 = (Q > 8 || (Q > 4 && Q < 8)) ? Q - 3 : 1;
  __device__ __forceinline__ static int swz(int t) {
    const int i = t >> C;
    int par = (i >> S1) & 1;
    if (S2 != S1) par ^= (i >> S2) & 1;
    if (S3 != S1 && S3 != S2) par ^= (i >> S3) & 1;
    return t ^ (par << 3);
  }
};

template <int Q, int C, int PARTS>
__device__ __forceinline__ void sp_tc_stage(float2* __restrict__ s, int b, const HFrag& H, int warp, int lane) {
  using G = TcSp<Q, C>;
  const int g = lane >> 2, t = lane & 3;
  constexpr int nblk = (1 << (Q + C)) >> 7;  // 128 amplitudes per block
  // block index enumerates j bits >= 3 and the i bits outside [b, b+4)
#pragma unroll 1
  for (int blk = warp; blk < nblk; blk += G::NT / 32) {
    const int jhi = blk & ((1 << (C - 3)) - 1);
    const int irest = blk >> (C - 3);  // Q-4 bits of i outside [b, b+4)
    const int i_base = (irest & ((1 << b) - 1)) | ((irest >> b) << (b + 4));
    const int base = g | (jhi << 3) | (i_base << C);
    tc_block<PARTS>(s + G::swz(base | ((2 * t) << (b + C))), s + G::swz(base | ((2 * t + 1) << (b + C))),
                    s + G::swz(base | ((2 * t + 8) << (b + C))), s + G::swz(base | ((2 * t + 9) << (b + C))), H);
  }
}

template <int Q, int C, bool WBW, int PARTS>
__global__ void __launch_bounds__(256)
    sp_tc_kernel(float2* __restrict__ psi, int n, int a1, int a2, const float2* __restrict__ brow, long long ntiles) {
  using G = TcSp<Q, C>;
  constexpr int QB = Q - 5;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* s_tile = reinterpret_cast<float2*>(smem);
  float2* s_bt = s_tile + G::TILE;
  if (WBW) {
    for (int i = threadIdx.x; i <= n; i += blockDim.x) s_bt[i] = brow[i];
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // stage list
  constexpr int NST = (Q <= 4) ? 1 : ((Q <= 8 && Q != 8) ? 2 : ((Q == 8) ? 2 : 3));
  int sb[3], hm[3];
  sb[0] = 0;
  hm[0] = 15;
  if (Q == 8) {
    sb[1] = 4;
    hm[1] = 15;
  } else if (Q < 8) {
    sb[1] = Q - 4;
    hm[1] = 15 & ~((1 << (8 - Q)) - 1);  // K bits >= 8-Q are the new bits 4..Q-1
  } else {
    sb[1] = 4;
    hm[1] = 15;
    sb[2] = Q - 4;
    hm[2] = 15 & ~((1 << (12 - Q)) - 1);  // new bits 8..Q-1
  }
  HFrag H[3];
#pragma unroll
  for (int s = 0; s < NST; ++s) H[s].init(hm[s], lane);

  const int lo_bits = a1 - C, mid_bits = a2 - a1 - 5;
  const unsigned long long lo_mask = (1ull << lo_bits) - 1ull, mid_mask = (1ull << mid_bits) - 1ull;
  // load/store layout: thread (j, th = i bits 5..Q-1), register r = i bits 0..4
  const int NTILE = 1 << (Q + C - 5);
  __syncthreads();
  for (long long T = blockIdx.x; T < ntiles; T += gridDim.x) {
    const unsigned long long ut = static_cast<unsigned long long>(T);
    const unsigned long long xbase = ((ut & lo_mask) << C) | (((ut >> lo_bits) & mid_mask) << (a1 + 5)) |
                                     ((ut >> (lo_bits + mid_bits)) << (a2 + QB));
    for (int u = threadIdx.x; u < NTILE; u += blockDim.x) {
      const int j = u & ((1 << C) - 1), th = u >> C;
      const float2* src = psi + xbase + j + (static_cast<unsigned long long>(th) << a2);
#pragma unroll 8
      for (int r = 0; r < 32; ++r) s_tile[G::swz(j + ((r + (th << 5)) << C))] = src[static_cast<unsigned long long>(r) << a1];
    }
    __syncthreads();
    for (int s = 0; s < NST; ++s) {
      sp_tc_stage<Q, C, PARTS>(s_tile, sb[s], H[s], warp, lane);
      __syncthreads();
    }
    if (WBW) {
      for (int e = threadIdx.x; e < G::TILE; e += blockDim.x) {
        const int j = e & ((1 << C) - 1), i = e >> C;
        const int pc = __popcll(xbase) + __popc(j) + __popc(i);
        const int a = G::swz(e);
        s_tile[a] = cmul(s_tile[a], s_bt[pc]);
      }
      __syncthreads();
      for (int s = 0; s < NST; ++s) {
        sp_tc_stage<Q, C, PARTS>(s_tile, sb[s], H[s], warp, lane);
        __syncthreads();
      }
    }
    for (int u = threadIdx.x; u < NTILE; u += blockDim.x) {
      const int j = u & ((1 << C) - 1), th = u >> C;
      float2* dst = psi + xbase + j + (static_cast<unsigned long long>(th) << a2);
#pragma unroll 8
      for (int r = 0; r < 32; ++r) dst[static_cast<unsigned long long>(r) << a1] = s_tile[G::swz(j + ((r + (th << 5)) << C))];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------- host ---------
template <int KIND, int PARTS>
static cudaError_t launch_lp_tc(const LaunchCtx& lc, float2* psi, int n, int m, const ClauseLP* cl, const float2* prow) {
  const long long ntiles = 1ll << (n - kLowBits);
  const size_t smem = 16u * m + ((8u * (m + 1) + 15u) & ~15u) + static_cast<size_t>(kTcWarps) * (8u * kLowTile + 8u * (m + 16));
  auto kern = lp_tc_kernel<KIND, PARTS>;
  const size_t worst = 16u * QAA_MAX_CLAUSES_DEV + ((8u * (QAA_MAX_CLAUSES_DEV + 1) + 15u) & ~15u) +
                       static_cast<size_t>(kTcWarps) * (8u * kLowTile + 8u * (QAA_MAX_CLAUSES_DEV + 16));
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(kern), worst);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTcWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  long long grid = static_cast<long long>(occ) * lc.num_sms;
  const long long need = (ntiles + kTcWarps - 1) / kTcWarps;
  if (grid > need) grid = need;
  kern<<<static_cast<unsigned>(grid), kTcWarps * 32, smem, lc.stream>>>(psi, m, cl, prow, ntiles);
  return cudaGetLastError();
}

template <int Q, int PARTS>
static cudaError_t launch_sp_tc(const LaunchCtx& lc, float2* psi, int n, int a1, int a2, bool wbw, const float2* brow) {
  constexpr int C = (10 - Q) > 3 ? (10 - Q) : 3;
  using G = TcSp<Q, C>;
  const long long ntiles = 1ll << (n - Q - C);
  const size_t smem = static_cast<size_t>(G::TILE) * 8u + 64u * 8u;
  auto kern = wbw ? sp_tc_kernel<Q, C, true, PARTS> : sp_tc_kernel<Q, C, false, PARTS>;
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, G::NT, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  long long grid = static_cast<long long>(occ) * lc.num_sms;
  if (grid > ntiles) grid = ntiles;
  kern<<<static_cast<unsigned>(grid), G::NT, smem, lc.stream>>>(psi, n, a1, a2, brow, ntiles);
  return cudaGetLastError();
}

template <int PARTS>
static cudaError_t launch_pass_tc_p(const LaunchCtx& lc, const Pass& p, float2* psi, int n, int m, const ClauseLP* cl,
                                    const float2* ptab, const float2* btab) {
  switch (p.kind) {
    case kLpFirst: return launch_lp_tc<kLpFirst, PARTS>(lc, psi, n, m, cl, ptab + static_cast<size_t>(p.prow) * (m + 1));
    case kLpMerge: return launch_lp_tc<kLpMerge, PARTS>(lc, psi, n, m, cl, ptab + static_cast<size_t>(p.prow) * (m + 1));
    case kLpLast: return launch_lp_tc<kLpLast, PARTS>(lc, psi, n, m, cl, ptab + static_cast<size_t>(p.prow) * (m + 1));
    case kSpW:
    case kSpWBW: {
      const bool wbw = p.kind == kSpWBW;
      const float2* brow = btab + static_cast<size_t>(p.brow) * (n + 1);
      switch (p.q) {
        case 5: return launch_sp_tc<5, PARTS>(lc, psi, n, p.a, p.a2, wbw, brow);
        case 6: return launch_sp_tc<6, PARTS>(lc, psi, n, p.a, p.a2, wbw, brow);
        case 7: return launch_sp_tc<7, PARTS>(lc, psi, n, p.a, p.a2, wbw, brow);
        case 8: return launch_sp_tc<8, PARTS>(lc, psi, n, p.a, p.a2, wbw, brow);
        case 9: return launch_sp_tc<9, PARTS>(lc, psi, n, p.a, p.a2, wbw, brow);
        case 10: return launch_sp_tc<10, PARTS>(lc, psi, n, p.a, p.a2, wbw, brow);
        default: return cudaErrorInvalidValue;
      }
    }
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pass_tc(const LaunchCtx& lc, const Pass& p, float2* psi, int n, int m, const ClauseLP* cl,
                           const float2* ptab, const float2* btab, int parts) {
  return parts == 2 ? launch_pass_tc_p<2>(lc, p, psi, n, m, cl, ptab, btab)
                    : launch_pass_tc_p<3>(lc, p, psi, n, m, cl, ptab, btab);
}

}  // namespace qaa
