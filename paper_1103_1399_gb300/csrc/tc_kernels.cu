// Tensor-core variant of the W.B.W form's passes on the fifth-generation tensor
// cores (tcgen05.mma, accumulators in tensor memory).
//
// Every Walsh-Hadamard transform over a group of up to 10 index bits is applied
// as at most two stages of 5 bits, each stage one GEMM against the 32 x 32
// Hadamard block H_32 (entries +-1, exact in BF16):
//   D[row][k'] = sum_k A[row][k] H_32[k][k'],
// a row being the 32 amplitudes (real or imaginary parts) that differ only in
// the stage's 5 bits.  The complex64 amplitudes are split into BF16 parts,
// x = hi + mid + lo (three products, about FP32 accuracy) or x = hi + lo (two
// products, about 16 mantissa bits); only the split and the FP32 accumulation
// round.  The hi part and the small parts accumulate in separate tensor-memory
// accumulators (the tensor cores' FP32 accumulation drops low-order bits of
// small addends added to a large accumulator) and are added in FP32 when read
// back.
//
// A CTA (256 threads, one per SM) owns a tile of 8192 amplitudes in shared
// memory: 2^Q rows of a strided group (Q <= 10) by 2^(13-Q) contiguous
// amplitudes, loaded by a cp.async.bulk.tensor box; or, for the low pass
// (bits 0..9), eight consecutive 1024-amplitude tiles loaded with cp.async.
// Tile index u (13 bits): stage 1 takes its K from a 5-bit field of u and
// stage 2 from u bits 8..12; the other 8 bits and re/im form 512 rows, four
// M = 128 units (two per component).  Per stage each thread reads its row's 32
// values from the tile, splits them and writes the BF16 parts in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix,
// LBO = 128 B along K, SBO = 512 B along M); one thread issues the MMAs
// (M = 128, N = 32, K = 16 each) and commits them to an mbarrier; every
// thread then reads its row's accumulators with tcgen05.ld (its warp's lane
// quarter) and writes the results back to the tile or, after the last stage,
// straight to global memory.  The phases between transforms (the popcount
// phase B, the merged P phase of the low pass, with the norm fold of the
// previous step) are applied on the way.  The next tile's load is issued as
// soon as the last stage has read the tile.
//
// Every mbarrier wait is bounded; on expiry the kernel records the handle's
// error word and all threads leave together, releasing tensor memory.
#include <cuda.h>

#include <cstring>

#include "device_common.cuh"

namespace qaa {

namespace {

// ---------------------------------------------------------------- PTX -------
__device__ __forceinline__ uint32_t tc_smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void tc_mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void tc_mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool tc_mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(tc_smem(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
constexpr long long kTcWaitLimit = 1ll << 24;
__device__ __forceinline__ bool tc_mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kTcWaitLimit; ++it)
    if (tc_mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tc_fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                               int c4, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(tc_smem(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(tc_smem(bar))
      : "memory");
}
__device__ __forceinline__ void tc_cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(tc_smem(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void tc_cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void tc_cp_async_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// tensor memory: allocation by one whole warp, the address written to shared memory
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// D (tensor memory) = A B^T (+ D when acc), A and B described in shared memory
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_smem(bar))
               : "memory");
}
// 32 consecutive FP32 columns of the calling thread's lane (its warp's quarter);
// the wait is in the same asm statement, so no use of the registers can be
// scheduled before the load has completed
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// two FP32 values rounded to BF16 and packed (the first in the low half)
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ float bf16_lo(uint32_t p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t p) { return __uint_as_float(p & 0xffff0000u); }

// ------------------------------------------------------------ geometry ------
constexpr int kTcThreads = 256;
constexpr int kTcTile = 8192;          // amplitudes per CTA tile
constexpr int kTcUnitBytes = 8192;     // one 128 x 32 BF16 operand unit
constexpr int kTcCols = 256;           // tensor-memory columns: 4 units x (hi 32 + small 32)
constexpr int kTcEStride = 33;         // energy buffer rows (padded)
constexpr uint32_t kTcLBO = 128, kTcSBO = 512;
// instruction descriptor: D F32, A and B BF16, both K-major, N = 32, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

struct TcLayout {
  size_t off_a, off_h, off_e, off_pt, off_bt, off_bar, total;
  __host__ __device__ explicit TcLayout(int parts) {
    off_a = static_cast<size_t>(kTcTile) * 8;
    off_h = off_a + static_cast<size_t>(parts) * 4 * kTcUnitBytes;
    off_e = off_h + 2 * 2048;
    off_pt = off_e + 8 * 32 * kTcEStride * 2;
    off_pt = (off_pt + 15) & ~static_cast<size_t>(15);
    off_bt = off_pt + 8 * (QAA_MAX_CLAUSES_DEV + 1);
    off_bar = off_bt + 64 * 8;
    total = off_bar + 32;
  }
};

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(kTcLBO >> 4) << 16) |
         (static_cast<uint64_t>(kTcSBO >> 4) << 32) | (1ull << 46);
}

// Tile index u of (row R, K index k) in stage 1 (K = u bits C..C+4) and stage 2
// (K = u bits 8..12).
__device__ __forceinline__ int u_stage1(int R, int k, int C) {
  return (R & ((1 << C) - 1)) | (k << C) | ((R >> C) << (C + 5));
}
__device__ __forceinline__ int u_stage2(int R, int k) { return (R & 255) | (k << 8); }
// Shared-memory slot of u: the low pass's tile is XOR-swizzled on bits 0..3 by
// bits 5..8 so that its loads and both stages' row accesses are conflict free;
// the strided tile is dense (as the TMA box writes it).
template <bool LOW>
__device__ __forceinline__ int tslot(int u) {
  return LOW ? (u ^ ((u >> 5) & 15)) : u;
}

// Hadamard block restricted to the K bits in hmask (identity on the others).
__device__ __forceinline__ float hentry(int k, int kp, int hmask) {
  if (((k ^ kp) & ~hmask & 31) != 0) return 0.0f;
  return (__popc(k & kp & hmask) & 1) ? -1.0f : 1.0f;
}

}  // namespace

// KIND: kSpW, kSpWBW (strided, Q bits), kLpFirst, kLpMerge, kLpLast (low pass, Q = 10).
template <int KIND, int Q, int PARTS>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_pass_kernel(float2* __restrict__ psi, const __grid_constant__ CUtensorMap tmap, int n, int a1, int a2,
                   long long ntiles, const float2* __restrict__ prow, const float2* __restrict__ brow,
                   const unsigned* __restrict__ counts, int m, int* __restrict__ err, const NormFold nf) {
  constexpr bool LOW = KIND == kLpFirst || KIND == kLpMerge || KIND == kLpLast;
  constexpr int C = LOW ? 0 : 13 - Q;  // stage-1 K field starts at u bit C
  constexpr int QB = Q - 5;
  constexpr bool TWO = Q > 5;          // two stages per transform (Q = 5: stage 2 alone)
  constexpr int NW = (KIND == kSpWBW || KIND == kLpMerge) ? 2 : 1;  // transforms per tile
  const TcLayout L(PARTS);
  extern __shared__ __align__(1024) unsigned char smem[];
  float2* s_t = reinterpret_cast<float2*>(smem);
  unsigned char* s_a = smem + L.off_a;
  unsigned char* s_h = smem + L.off_h;
  uint16_t* s_e = reinterpret_cast<uint16_t*>(smem + L.off_e);
  float2* s_pt = reinterpret_cast<float2*>(smem + L.off_pt);
  float2* s_bt = reinterpret_cast<float2*>(smem + L.off_bt);
  uint64_t* bar_tma = reinterpret_cast<uint64_t*>(smem + L.off_bar);
  uint64_t* bar_mma = bar_tma + 1;
  uint32_t* s_taddr = reinterpret_cast<uint32_t*>(bar_tma + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q4 = warp & 3, hh = warp >> 2;
  const int r = 32 * q4 + lane;  // tensor-memory lane = row within a unit
  const int R = r + 128 * hh;    // row (without re/im), 0..255

  // tensor memory, barriers, the two Hadamard operands (K-major, N x K)
  if (warp == 0) tmem_alloc(s_taddr, kTcCols);
  if (tid == 0) {
    tc_mbar_init(bar_tma, 1);
    tc_mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    const int hm2 = TWO ? (31 & ~((1 << (10 - Q)) - 1)) : 31;
    for (int e = tid; e < 2 * 32 * 16; e += kTcThreads) {
      const int s = e >> 9, nn = (e >> 4) & 31, kp = (e & 15) * 2;  // operand s, row n, columns kp, kp+1
      const int hm = s == 0 ? 31 : hm2;
      const uint32_t w = bf16x2(hentry(kp, nn, hm), hentry(kp + 1, nn, hm));
      const uint32_t off = s * 2048 + (nn >> 3) * kTcSBO + (kp >> 3) * kTcLBO + (nn & 7) * 16 + (kp & 7) * 2;
      *reinterpret_cast<uint32_t*>(s_h + off) = w;
    }
  }
  // phase rows: P (low passes; the norm fold of the previous step folded in), B (phase group)
  const float fd = fold_factor_block(nf);
  if (LOW) {
    for (int i = tid; i <= m; i += kTcThreads)
      s_pt[i] = fold_apply(prow[i], fd);
  }
  if (KIND == kSpWBW) {
    for (int i = tid; i <= n; i += kTcThreads) s_bt[i] = brow[i];
  }
  tc_fence_proxy_async();  // the Hadamard operands are read by the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *s_taddr;
  const uint32_t t_row = taddr + (static_cast<uint32_t>(32 * q4) << 16);  // this warp's lane quarter

  // strided tile T -> (low, middle, high) fixed-bit fields, as sp_tma_kernel
  const int lo_bits = LOW ? 0 : a1 - C, mid_bits = LOW ? 0 : a2 - a1 - 5;
  const unsigned long long lo_mask = (1ull << lo_bits) - 1ull, mid_mask = (1ull << mid_bits) - 1ull;
  auto xbase_of = [&](long long T) -> unsigned long long {
    const unsigned long long ut = static_cast<unsigned long long>(T);
    if (LOW) return ut * kTcTile;
    return ((ut & lo_mask) << C) | (((ut >> lo_bits) & mid_mask) << (a1 + 5)) |
           ((ut >> (lo_bits + mid_bits)) << (a2 + QB));
  };
  auto issue = [&](long long T) {
    if (LOW) {
      // eight consecutive 1024-amplitude tiles: x = base + i + 1024 j (i bits 0..4 = u bits 0..4,
      // j = u bits 5..7, i bits 5..9 = u bits 8..12)
      const float2* g = psi + xbase_of(T);
#pragma unroll 4
      for (int e = 0; e < kTcTile / kTcThreads; ++e) {
        const int x = tid + kTcThreads * e;
        const int u = (x & 31) | ((x >> 10) << 5) | (((x >> 5) & 31) << 8);
        tc_cp_async8(s_t + tslot<LOW>(u), g + x);
      }
      tc_cp_async_commit();
    } else if (tid == 0) {
      const unsigned long long ut = static_cast<unsigned long long>(T);
      tc_mbar_expect_tx(bar_tma, kTcTile * 8u);
      tc_tma_load_5d(s_t, &tmap, static_cast<int>((ut & lo_mask) << C), 0,
                     static_cast<int>((ut >> lo_bits) & mid_mask), 0, static_cast<int>(ut >> (lo_bits + mid_bits)),
                     bar_tma);
    }
  };

  DFloat nacc{0.f, 0.f};  // |psi|^2 of this thread's outputs (norm fold of the low passes)
  uint32_t mma_phase = 0;
  int it = 0;
  int pending = -1;  // strided: the iteration whose TMA load is in flight
  bool failed = false;
  if (static_cast<long long>(blockIdx.x) < ntiles) {
    issue(blockIdx.x);
    pending = 0;
  }
  for (long long T = blockIdx.x; T < ntiles; T += gridDim.x, ++it) {
    const unsigned long long xb = xbase_of(T);
    // energies of the low tile (stored per-tile counts, layout Y: lane = bits 5..9,
    // register = bits 0..4): warp w expands 1024-tile w of the eight
    if (LOW) {
      unsigned pl[kPlanes];
      int nconst;
      load_counts(counts, T * 8 + warp, lane, pl, nconst);
      int e[32];
      StoreCountUnroll<0>::run(e, pl, nconst);
      uint16_t* row = s_e + warp * 32 * kTcEStride + lane * kTcEStride;
#pragma unroll
      for (int rr = 0; rr < 32; ++rr) row[rr] = static_cast<uint16_t>(e[rr]);
    }
    // the tile
    bool ok = true;
    if (LOW) {
      tc_cp_async_wait();
    } else {
      ok = tc_mbar_wait(bar_tma, static_cast<uint32_t>(it) & 1u);
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    pending = -1;
    // kLpFirst: P before the transform (warp = 1024-tile j, lane = bits 0..4, k = bits 5..9)
    if (KIND == kLpFirst) {
#pragma unroll 4
      for (int k = 0; k < 32; ++k) {
        float2* p = s_t + tslot<LOW>(u_stage2(R, k));
        *p = cmul(*p, s_pt[s_e[warp * 32 * kTcEStride + k * kTcEStride + lane]]);
      }
      __syncthreads();
    }
    for (int w = 0; w < NW && !failed; ++w) {
      for (int st = TWO ? 1 : 2; st <= 2; ++st) {
        // ---- A: this thread's row, both components, split into BF16 parts
        {
          float2 x[32];
#pragma unroll
          for (int k = 0; k < 32; ++k) x[k] = s_t[tslot<LOW>(st == 1 ? u_stage1(R, k, C) : u_stage2(R, k))];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int unit = 2 * hh + c;
#pragma unroll
            for (int kb = 0; kb < 4; ++kb) {
              uint32_t ph[PARTS][4];
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                float v0 = c ? x[8 * kb + 2 * t].y : x[8 * kb + 2 * t].x;
                float v1 = c ? x[8 * kb + 2 * t + 1].y : x[8 * kb + 2 * t + 1].x;
#pragma unroll
                for (int p = 0; p < PARTS; ++p) {
                  const uint32_t b = bf16x2(v0, v1);
                  ph[p][t] = b;
                  v0 -= bf16_lo(b);  // exact: the remainder of a round-to-nearest in FP32
                  v1 -= bf16_hi(b);
                }
              }
#pragma unroll
              for (int p = 0; p < PARTS; ++p) {
                const uint32_t off = (p * 4 + unit) * kTcUnitBytes + (r >> 3) * kTcSBO + kb * kTcLBO + (r & 7) * 16;
                *reinterpret_cast<uint4*>(s_a + off) = make_uint4(ph[p][0], ph[p][1], ph[p][2], ph[p][3]);
              }
            }
          }
        }
        tc_fence_proxy_async();
        __syncthreads();
        // the tile has been read for the last time: the next tile's load can start
        if (w == NW - 1 && st == 2 && T + gridDim.x < ntiles) {
          if (!LOW && tid == 0) tc_fence_proxy_async();
          issue(T + gridDim.x);
          pending = it + 1;
        }
        // ---- MMAs: per unit, hi -> accumulator 0, the small parts -> accumulator 1
        if (tid == 0) {
          tc_fence_after();
          const uint32_t a0 = tc_smem(s_a), h0 = tc_smem(s_h) + (st == 1 ? 0u : 2048u);
#pragma unroll
          for (int unit = 0; unit < 4; ++unit) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
              const uint64_t bd = smem_desc(h0 + 256u * s);
#pragma unroll
              for (int p = 0; p < PARTS; ++p) {
                const uint64_t ad = smem_desc(a0 + (p * 4 + unit) * kTcUnitBytes + 256u * s);
                const uint32_t d = taddr + unit * 64 + (p == 0 ? 0 : 32);
                tc_mma(d, ad, bd, kTcIdesc, (s > 0 || p > 1) ? 1u : 0u);
              }
            }
          }
          tc_commit(bar_mma);
        }
        ok = tc_mbar_wait(bar_mma, mma_phase & 1u);
        ++mma_phase;
        if (__syncthreads_or(!ok)) {
          failed = true;
          break;
        }
        tc_fence_after();
        // ---- read back: y[k'] for this row, both components
        float2 y[32];
        {
          float hi[32], sm[32];
          tmem_ld32(t_row + (2 * hh) * 64, hi);
          tmem_ld32(t_row + (2 * hh) * 64 + 32, sm);
#pragma unroll
          for (int k = 0; k < 32; ++k) y[k].x = hi[k] + sm[k];
          tmem_ld32(t_row + (2 * hh + 1) * 64, hi);
          tmem_ld32(t_row + (2 * hh + 1) * 64 + 32, sm);
#pragma unroll
          for (int k = 0; k < 32; ++k) y[k].y = hi[k] + sm[k];
        }
        if (st == 2) {
          // phases due after a whole transform: B between the two transforms of
          // the phase group, P after the low pass's (first) transform
          if (KIND == kSpWBW && w == 0) {
            const int pc0 = __popcll(xb);
#pragma unroll
            for (int k = 0; k < 32; ++k) {
              const int u = u_stage2(R, k);
              y[k] = cmul(y[k], s_bt[pc0 + __popc(u & ((1 << C) - 1)) + __popc(u >> C)]);
            }
          }
          if ((KIND == kLpMerge && w == 0) || KIND == kLpLast) {
#pragma unroll
            for (int k = 0; k < 32; ++k) y[k] = cmul(y[k], s_pt[s_e[warp * 32 * kTcEStride + k * kTcEStride + lane]]);
          }
        }
        if (w == NW - 1 && st == 2) {
          // to global memory (x of u = R | k << 8)
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const int u = u_stage2(R, k);
            unsigned long long x;
            if (LOW) {
              x = xb + static_cast<unsigned long long>((u & 31) | ((u >> 8) << 5) | (((u >> 5) & 7) << 10));
            } else {
              const int j = u & ((1 << C) - 1), i = u >> C;
              x = xb + static_cast<unsigned long long>(j) + (static_cast<unsigned long long>(i & 31) << a1) +
                  (static_cast<unsigned long long>(i >> 5) << a2);
            }
            psi[x] = y[k];
          }
          if (LOW && nf.out) {
            float t = 0.0f;
#pragma unroll
            for (int k = 0; k < 32; ++k) t = fmaf(y[k].x, y[k].x, fmaf(y[k].y, y[k].y, t));
            nacc = df_add1(nacc, t);
          }
        } else {
#pragma unroll
          for (int k = 0; k < 32; ++k) s_t[tslot<LOW>(st == 1 ? u_stage1(R, k, C) : u_stage2(R, k))] = y[k];
        }
        tc_fence_before();
        __syncthreads();
      }
    }
    if (failed) break;
  }
  if (failed && tid == 0) atomicExch(err, 1);
  // leave only when no copy issued by this CTA is in flight
  if (LOW) {
    tc_cp_async_wait();
  } else if (tid == 0 && pending >= 0) {
    if (!tc_mbar_wait(bar_tma, static_cast<uint32_t>(pending) & 1u)) atomicExch(err, 1);
  }
  if (LOW) fold_store(nf, nacc);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(taddr, kTcCols);
  }
}

// ------------------------------------------------------------- host ---------
typedef CUresult (*TcEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static TcEncodeFn tc_encode() {
  static const TcEncodeFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<TcEncodeFn>(p);
    cudaGetLastError();
    return static_cast<TcEncodeFn>(nullptr);
  }();
  return fn;
}

size_t tc_smem_bytes(int parts) { return TcLayout(parts).total; }

template <int KIND, int Q, int PARTS>
static cudaError_t launch_tc_q(const LaunchCtx& lc, const Pass& p, float2* psi, int n, int m, const float2* prow,
                               const float2* brow, const unsigned* counts, int* err, const NormFold& nf) {
  constexpr bool LOW = KIND == kLpFirst || KIND == kLpMerge || KIND == kLpLast;
  constexpr int C = LOW ? 0 : 13 - Q;
  constexpr int QB = Q - 5;
  CUtensorMap map;
  std::memset(&map, 0, sizeof map);
  long long ntiles;
  int a1 = 0, a2 = 0;
  if (LOW) {
    if (n < 13 || !counts) return cudaErrorInvalidValue;  // eight 1024-amplitude tiles, stored counts
    ntiles = 1ll << (n - 13);
  } else {
    a1 = p.a;
    a2 = p.a2;
    if (a1 < C || a2 < a1 + 5 || a2 + QB > n || (a2 != a1 + 5 && QB < 5)) return cudaErrorInvalidValue;
    TcEncodeFn enc = tc_encode();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[5] = {1ull << a1, 32ull, 1ull << (a2 - a1 - 5), 1ull << QB, 1ull << (n - a2 - QB)};
    const cuuint64_t strides[4] = {(1ull << a1) * 8ull, (1ull << (a1 + 5)) * 8ull, (1ull << a2) * 8ull,
                                   (1ull << (a2 + QB)) * 8ull};
    const cuuint32_t box[5] = {1u << C, 32u, 1u, 1u << QB, 1u};
    const cuuint32_t estr[5] = {1u, 1u, 1u, 1u, 1u};
    const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, psi, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    ntiles = 1ll << (n - Q - C);
  }
  const TcLayout L(PARTS);
  auto kern = tc_pass_kernel<KIND, Q, PARTS>;
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(kern), L.total);
  if (e != cudaSuccess) return e;
  long long grid = lc.num_sms;  // one CTA per SM (shared memory and tensor memory)
  if (grid > ntiles) grid = ntiles;
  if (grid > kFoldSlot - 1) grid = kFoldSlot - 1;
  kern<<<static_cast<unsigned>(grid), kTcThreads, L.total, lc.stream>>>(psi, map, n, a1, a2, ntiles, prow, brow,
                                                                       counts, m, err, nf);
  return cudaGetLastError();
}

template <int KIND, int PARTS>
static cudaError_t launch_tc_sp(const LaunchCtx& lc, const Pass& p, float2* psi, int n, int m, const float2* brow,
                                int* err) {
  switch (p.q) {
    case 5: return launch_tc_q<KIND, 5, PARTS>(lc, p, psi, n, m, nullptr, brow, nullptr, err, NormFold());
    case 6: return launch_tc_q<KIND, 6, PARTS>(lc, p, psi, n, m, nullptr, brow, nullptr, err, NormFold());
    case 7: return launch_tc_q<KIND, 7, PARTS>(lc, p, psi, n, m, nullptr, brow, nullptr, err, NormFold());
    case 8: return launch_tc_q<KIND, 8, PARTS>(lc, p, psi, n, m, nullptr, brow, nullptr, err, NormFold());
    case 9: return launch_tc_q<KIND, 9, PARTS>(lc, p, psi, n, m, nullptr, brow, nullptr, err, NormFold());
    case 10: return launch_tc_q<KIND, 10, PARTS>(lc, p, psi, n, m, nullptr, brow, nullptr, err, NormFold());
    default: return cudaErrorInvalidValue;
  }
}

template <int PARTS>
static cudaError_t launch_pass_tc_p(const LaunchCtx& lc, const Pass& p, float2* psi, int n, int m, const float2* ptab,
                                    const float2* btab, int* err, const unsigned* counts, const NormFold& nf) {
  const float2* prow = ptab + static_cast<size_t>(p.prow) * (m + 1);
  const float2* brow = btab + static_cast<size_t>(p.brow) * (n + 1);
  switch (p.kind) {
    case kLpFirst: return launch_tc_q<kLpFirst, 10, PARTS>(lc, p, psi, n, m, prow, nullptr, counts, err, nf);
    case kLpMerge: return launch_tc_q<kLpMerge, 10, PARTS>(lc, p, psi, n, m, prow, nullptr, counts, err, nf);
    case kLpLast: return launch_tc_q<kLpLast, 10, PARTS>(lc, p, psi, n, m, prow, nullptr, counts, err, nf);
    case kSpW: return launch_tc_sp<kSpW, PARTS>(lc, p, psi, n, m, nullptr, err);
    case kSpWBW: return launch_tc_sp<kSpWBW, PARTS>(lc, p, psi, n, m, brow, err);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pass_tc(const LaunchCtx& lc, const Pass& p, float2* psi, int n, int m, const ClauseLP*,
                           const float2* ptab, const float2* btab, int parts, int* err, const unsigned* counts,
                           const NormFold& nf) {
  if (!err) return cudaErrorInvalidValue;
  return parts == 2 ? launch_pass_tc_p<2>(lc, p, psi, n, m, ptab, btab, err, counts, nf)
                    : launch_pass_tc_p<3>(lc, p, psi, n, m, ptab, btab, err, counts, nf);
}

}  // namespace qaa
