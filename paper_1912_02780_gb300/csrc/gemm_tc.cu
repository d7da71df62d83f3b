// Split-BF16 GEMM on the sm_103a tensor cores (tcgen05 + TMEM + TMA).
//
//   C(m, n) = alpha * sum_k A(m, k) * B(n, k)
//
// Both operands are K-major and split into bf16 planes (hi, lo [, lo2, lo3])
// so that a*b ~= sum over the plane pairs (i, j) with i + j <= nplanes - 1 of
// a_i * b_j.  This is how the O(D^7) contractions of the HOTRG step (SM
// Sec. B, HOTRG step equation) and of its adjoint run at tensor-core rate
// while keeping about 16, 24 or 32 significant bits per product (two, three
// or four planes).
//
// Structure (one persistent CTA per SM, or a cluster of two, 320 threads):
//   warp 8      TMA producer: per K slab (64 or 32 wide), one 3-D tensor-map
//               load per operand plane into a swizzled shared-memory stage.
//   warp 9      MMA issuer: tcgen05.mma kind::f16 (M = 128, or 256 across a
//               CTA pair; N = BN, K = 16) for every plane pair and K step,
//               hi*hi into its own exactly accumulated TMEM buffer, the other
//               products into a second; tcgen05.commit frees the stage and, at
//               the end of an accumulation chunk, hands the (double-buffered)
//               accumulators to the epilogue.
//   warps 0-7   epilogue: tcgen05.ld the accumulators (one TMEM lane per row,
//               half of the columns per warp), add the chunk into
//               float-float register sums, and write the tile through the
//               output index maps as FP32, FP64 or grid-split bf16 planes,
//               staged through a per-warp shared-memory transpose for
//               whole-sector stores.
// Every mbarrier wait is bounded; on timeout the error word gets kErrTimeout,
// the role stops, and all warps still meet at the final barrier, drain their
// MMAs and free TMEM.
#include <cuda.h>
#include <cstdio>
#include <mutex>
#include "gemm_tc.h"

namespace hotrg {

namespace {

constexpr int BM = 128;
// K slab per pipeline stage: 32 bf16 = 64-byte rows (64B swizzle, 4 stages of
// 48 KB for three planes) or 64 bf16 = 128-byte rows (128B swizzle, 2 stages).
constexpr long long kTimeoutCycles = 4000000000LL;   // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase with this parity completed, false (and
// the error word set) after about two seconds.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err,
                                       long long limit = kTimeoutCycles) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > limit) {
      report_error(err, kErrTimeout);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, uint32_t bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"((uint64_t)tm), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// ---- CTA-pair (cluster of two) helpers ------------------------------------
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cbar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cbar)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx_cluster(uint32_t cbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cluster.shared::cluster.b64 _, [%0], %1;" ::"r"(
                   cbar),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
// TMA load into this CTA's shared memory whose completion is counted on an
// mbarrier of either CTA of the pair (cbar: a shared::cluster address).
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap* tm,
                                                 uint32_t cbar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2 "
      "[%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"((uint64_t)tm), "r"(cbar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
// Pair MMA, issued by the even CTA: D (128 lanes in each CTA's TMEM) +=
// A (128 rows from each CTA) x B (N/2 rows from each CTA).
__device__ __forceinline__ void tc_mma_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on the mbarrier at offset `bar` of every CTA in `mask` once all pair
// MMAs issued so far by this thread have completed.
__device__ __forceinline__ void tc_commit_pair(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
      "[%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor for a K-major tile written by TMA with
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart (SBO),
// descriptor version 1, layout SWIZZLE_128B (= 2 in bits 61-63).  Advancing
// along K inside the 128-byte row is done by adding the byte offset to the
// start address (the swizzle is a function of the absolute address; tiles are
// 1024-byte aligned).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // version
  d |= (uint64_t)2 << 61;            // swizzle 128B
  return d;
}

// Same for 64-byte rows with 64-byte swizzle: 8-row groups 512 bytes apart,
// layout SWIZZLE_64B (= 4 in bits 61-63).
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

template <int BK>
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return BK == 64 ? sdesc_sw128(saddr) : sdesc_sw64(saddr);
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void named_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Named barrier with an AND-reduction of `pred` over the participating threads,
// so that every epilogue warp takes the same branch after a failed wait.
__device__ __forceinline__ bool named_bar_and(int id, int count, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "barrier.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Plane products formed for each K step: every pair (i, j) with
// i + j <= NP - 1, hi * hi first (its own, exactly accumulated TMEM buffer),
// then (0, 1), then the others smallest first.  hi * hi and (0, 1) share A
// plane 0 and sit side by side in TMEM ([hh | rest]) with B planes 0 and 1
// side by side in shared memory, so one CTA issues them as one N = 2 BN
// instruction.
template <int NP>
struct Pairs;
// (plane of A, plane of B) of product q, written out as selections so that
// they fold to constants in the unrolled issue loop
template <>
struct Pairs<2> {
  static constexpr int n = 3;
  __host__ __device__ static constexpr int a(int q) { return q == 2 ? 1 : 0; }
  __host__ __device__ static constexpr int b(int q) { return q == 1 ? 1 : 0; }
};
template <>
struct Pairs<3> {   // (0,0) (0,1) (2,0) (1,1) (0,2) (1,0)
  static constexpr int n = 6;
  __host__ __device__ static constexpr int a(int q) {
    return q == 2 ? 2 : (q == 3 || q == 5) ? 1 : 0;
  }
  __host__ __device__ static constexpr int b(int q) {
    return q == 1 ? 1 : q == 3 ? 1 : q == 4 ? 2 : 0;
  }
};
template <>
struct Pairs<4> {   // (0,0) (0,1) (3,0) (2,1) (1,2) (0,3) (2,0) (1,1) (0,2) (1,0)
  static constexpr int n = 10;
  __host__ __device__ static constexpr int a(int q) {
    return q == 2 ? 3 : (q == 3 || q == 6) ? 2 : (q == 4 || q == 7 || q == 9) ? 1 : 0;
  }
  __host__ __device__ static constexpr int b(int q) {
    return q == 5 ? 3 : (q == 4 || q == 8) ? 2 : (q == 1 || q == 3 || q == 7) ? 1 : 0;
  }
};

// Tile t of an MT x NT grid: M fastest (m_fast), N fastest, or (n_group > 0)
// in groups of n_group N-tiles: all M-tiles of one group of columns, N fastest
// inside the group, before the next group.  The persistent CTAs then work on
// one stripe of B at a time, which stays in L2 while A streams past it; A is
// read once per group.
__device__ __forceinline__ void tile_coords(long long t, int MT, int NT, int m_fast, int n_group,
                                            int& mt, int& nt) {
  if (m_fast) {
    nt = (int)(t / MT);
    mt = (int)(t - (long long)nt * MT);
  } else if (n_group > 0 && n_group < NT) {
    const long long per_group = (long long)MT * n_group;
    const int grp = (int)(t / per_group);
    const long long r = t - (long long)grp * per_group;
    const int n0 = grp * n_group;
    const int gw = (NT - n0) < n_group ? (NT - n0) : n_group;   // the last group may be narrower
    mt = (int)(r / gw);
    nt = n0 + (int)(r - (long long)mt * gw);
  } else {
    mt = (int)(t / NT);
    nt = (int)(t - (long long)mt * NT);
  }
}

// CG = 1: one CTA computes a BM x BN tile.  CG = 2: a cluster of two CTAs
// computes a (2 BM) x BN tile with pair MMAs (tcgen05 cta_group::2); each CTA
// loads its BM rows of A and BN / 2 rows of B, so a pipeline stage is 25 %
// smaller per CTA and three stages fit, and the tensor cores read a quarter
// less shared memory per flop.
template <int BN, int NP, int BK, int CG = 1>
struct Cfg {
  static constexpr int kBRows = BN / CG;                 // B rows loaded by each CTA
  static constexpr int kAPlane = BM * BK * 2;
  static constexpr int kBPlane = kBRows * BK * 2;
  static constexpr int kStage = NP * (kAPlane + kBPlane);
  // Epilogue: two warps per TMEM lane quadrant (a warp may only read the 32
  // lanes of its own sub-partition), each with half of the tile's columns.
  // Measured on GB300 (stage 2 at D_cut = 64, three planes): 8 epilogue warps
  // 40.1 ms, 16 warps 42.4 ms (less register pressure, but more warps
  // competing with the TMA and MMA warps for issue slots).
  static constexpr int kEpiPerQuad = 2;
  static constexpr int kEpiWarps = 4 * kEpiPerQuad;
  static constexpr int kThreads = (kEpiWarps + 2) * 32;  // + TMA warp + MMA warp
  static constexpr int kCols = BN / kEpiPerQuad;         // columns per epilogue thread
  // Shared memory after the pipeline stages (byte offsets from the 1024-aligned
  // base): mbarriers, column offsets (BN), contiguity flags, the TMEM address,
  // the segment-max / offset exchange of the grid-split epilogue (4 column
  // groups x 128 rows), and a 1 KB store-staging buffer per epilogue warp
  // (16-byte aligned: it is accessed as uint4).  CG = 2 keeps the exchange
  // inside the staging buffers (a barrier separates the two uses).
  static constexpr int kStageBytes = 1024;
  static constexpr int kXchg = kEpiPerQuad * BM * 12;    // offsets (8 B) + maxima (4 B)
  static constexpr int kExtra = 1024 + 17 * 8 + BN * 8 + BN / 16 * 4 + 32 +
                                (CG == 2 ? 0 : kXchg + 16) + kEpiWarps * kStageBytes;
  static constexpr int kFit = (232448 - kExtra) / kStage;
  static constexpr int kStages = kFit > 6 ? 6 : kFit;
  static constexpr int kBars = 2 * kStages + 5;
  static constexpr int kOffBars = kStages * kStage;
  static constexpr int kOffCn = kOffBars + kBars * 8;
  static constexpr int kOffCv = kOffCn + BN * 8;
  static constexpr int kOffTmem = kOffCv + BN / 16 * 4;
  static constexpr int kOffXo = (kOffTmem + 16 + 15) / 16 * 16;
  static constexpr int kOffXm = kOffXo + kEpiPerQuad * BM * 8;
  static constexpr int kOffStg =
      CG == 2 ? kOffXo : (kOffXm + kEpiPerQuad * BM * 4 + 15) / 16 * 16;
  static constexpr int kSmem = 1024 + kOffStg + kEpiWarps * kStageBytes;
  static_assert(kOffCn % 8 == 0 && kOffXo % 16 == 0 && kOffStg % 16 == 0, "smem alignment");
  static_assert(CG == 1 || kXchg <= kEpiWarps * kStageBytes, "exchange fits the staging");
  static_assert(kSmem <= 232448, "shared memory per CTA");
  static_assert(kCols % 16 == 0, "whole 16-column store groups per thread");
  // TMEM: per buffer (2) an exact hi*hi accumulator and a "rest" accumulator, BN columns each.
  static constexpr int kTmemCols = 4 * BN;
  static_assert(kStages >= 2, "need at least two pipeline stages");
  static_assert(kTmemCols <= 512, "TMEM holds 512 columns");
  static_assert(CG == 1 || CG == 2, "one CTA or a pair");
};
// Warp-cooperative store of 64 bytes per lane (each lane: one contiguous,
// 16-byte aligned destination run) through the warp's staging buffer: every
// store instruction then writes 8 runs x 64 bytes (whole 32-byte sectors)
// instead of 32 runs x 16 bytes.  The 16-byte chunk position is XOR-swizzled
// with the row so that both shared-memory passes are free of bank conflicts.
// With a 2 KB buffer all 32 rows go through at once; with 1 KB, in two halves
// of 16 rows.  All 32 lanes must take part.
template <int kBytes>
__device__ __forceinline__ void warp_store64(uint8_t* stage, const uint4 (&v)[4], char* dst,
                                             int lane) {
  constexpr int kRows = kBytes / 64;   // rows staged per pass (32 or 16)
  static_assert(kRows == 32 || kRows == 16, "2 KB or 1 KB staging");
  const int c = lane & 3;
#pragma unroll
  for (int h = 0; h < 32 / kRows; ++h) {
    if ((lane / kRows) == h) {
      const int lr = lane % kRows;
      const int sw = (lr >> 1) & 3;
      uint4* srow = reinterpret_cast<uint4*>(stage + lr * 64);
#pragma unroll
      for (int q = 0; q < 4; ++q) srow[q ^ sw] = v[q];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < kRows / 8; ++k) {
      const int lr = 8 * k + (lane >> 2);
      const int r = h * kRows + lr;
      char* d = reinterpret_cast<char*>(
          __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(dst), r));
      const uint4 x = reinterpret_cast<const uint4*>(stage + lr * 64)[c ^ ((lr >> 1) & 3)];
      *reinterpret_cast<uint4*>(d + c * 16) = x;
    }
    __syncwarp();
  }
}

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

template <int BN, int NP>
__device__ __forceinline__ void store_tile_chunk(const TcGemm& p, long long coff,
                                                 const long long* cn_s, int contig, int cc,
                                                 const float* hi, const float* lo) {
  const long long off0 = coff + cn_s[cc];
  // vector stores need the 16-byte alignment of the actual address
  const bool c16 = (reinterpret_cast<uintptr_t>(p.C) & 15) == 0;
  if (contig && c16 && off0 >= 0 && off0 + 15 < p.c_lim && !p.accumulate) {
    if (p.out_mode == kOutF32 && (off0 & 3) == 0) {
      float4* d = reinterpret_cast<float4*>(reinterpret_cast<float*>(p.C) + off0);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        d[q] = make_float4(p.alpha * (hi[4 * q] + lo[4 * q]), p.alpha * (hi[4 * q + 1] + lo[4 * q + 1]),
                           p.alpha * (hi[4 * q + 2] + lo[4 * q + 2]),
                           p.alpha * (hi[4 * q + 3] + lo[4 * q + 3]));
      return;
    }
    if (p.out_mode == kOutF64 && (off0 & 1) == 0) {
      double2* d = reinterpret_cast<double2*>(reinterpret_cast<double*>(p.C) + off0);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        d[q] = make_double2((double)p.alpha * ((double)hi[2 * q] + (double)lo[2 * q]),
                            (double)p.alpha * ((double)hi[2 * q + 1] + (double)lo[2 * q + 1]));
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    long long co = cn_s[cc + j];
    if (co < 0) continue;
    long long off = coff + co;
    if (off >= p.c_lim) {
      report_error(p.err, kErrBounds);
      continue;
    }
    if (p.out_mode == kOutF32) {
      float v = p.alpha * (hi[j] + lo[j]);
      float* c = reinterpret_cast<float*>(p.C) + off;
      if (p.accumulate) v += *c;
      *c = v;
    } else if (p.out_mode == kOutF64) {
      double v = (double)p.alpha * ((double)hi[j] + (double)lo[j]);
      double* c = reinterpret_cast<double*>(p.C) + off;
      if (p.accumulate) v += *c;
      *c = v;
    }
  }
}

// 320 threads: 10 warps, 3 on two of the SM's four sub-partitions, so at most
// 168 registers a thread (3 x 32 x 168 <= 16384).
// CG = 2: launched in clusters of two CTAs.  The even CTA's MMA warp issues
// the pair MMAs for both; each CTA's TMA warp loads its own halves and counts
// them on the even CTA's full barrier; the MMA completion is multicast to both
// CTAs' stage-empty and accumulator-full barriers; both CTAs' epilogue warps
// release an accumulator on the even CTA's barrier.
template <int BN, int NP, int BK, int CG>
__global__ void __launch_bounds__(Cfg<BN, NP, BK, CG>::kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcGemm p) {
  using C = Cfg<BN, NP, BK, CG>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kOffBars);
  long long* cn_s = reinterpret_cast<long long*>(smem + C::kOffCn);
  int* cv_s = reinterpret_cast<int*>(smem + C::kOffCv);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::kOffTmem);
  long long* xo_s = reinterpret_cast<long long*>(smem + C::kOffXo);
  float* xm_s = reinterpret_cast<float*>(smem + C::kOffXm);
  uint8_t* stg_s = smem + C::kOffStg;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int kProducer = C::kEpiWarps, kMma = C::kEpiWarps + 1;
  const uint32_t rank = CG == 2 ? cluster_rank() : 0u;   // 0: the CTA that issues the MMAs
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (C::kStages + s); };
  auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * C::kStages + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * C::kStages + 2 + a); };
  const uint32_t drain_bar = bar0 + 8u * (2 * C::kStages + 4);
  const uint32_t smem0 = smem_u32(smem);
  auto a_tile = [&](int s, int pl) { return smem0 + s * C::kStage + pl * C::kAPlane; };
  auto b_tile = [&](int s, int pl) {
    return smem0 + s * C::kStage + NP * C::kAPlane + pl * C::kBPlane;
  };

  if (warp == kProducer && lane == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(full_bar(s), CG);             // one expect_tx arrival per CTA of the pair
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), C::kEpiWarps * CG);
    }
    mbar_init(drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
  }
  if (warp == kMma) {
    if constexpr (CG == 2) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(C::kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(C::kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  if constexpr (CG == 2) cluster_sync();   // both CTAs' barriers are initialised
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // the even CTA's full / tempty barriers, as shared::cluster addresses
  auto lead = [&](uint32_t bar) { return CG == 2 ? map_to_rank(bar, 0) : bar; };

  // CG = 2: a tile is 2 BM rows; the pair (cluster) walks the tiles together
  // grouped launch: MTp row tiles per problem (its rows padded to a_pitch)
  const int bt = p.batch > 1 ? p.batch : 1;
  const int MTp = bt > 1 ? p.a_pitch / (BM * CG) : (p.M + BM * CG - 1) / (BM * CG);
  const int MT = MTp * bt, NT = (p.N + BN - 1) / BN;
  const long long t0 = blockIdx.x / CG, tstep = gridDim.x / CG;
  const long long tiles = (long long)MT * NT;
  const int KB = (p.K + BK - 1) / BK;
  // p.kchunk counts 64-wide K blocks; a chunk spans (64 / BK) slabs per unit
  const int kc_slabs = p.kchunk < 1 ? KB : p.kchunk * (64 / BK);
  const int kchunk = kc_slabs > KB ? KB : kc_slabs;
  const int nchunks = (KB + kchunk - 1) / kchunk;

  if (warp == kProducer) {
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      int issued[C::kStages];
      uint32_t last_par[C::kStages];
      for (int i = 0; i < C::kStages; ++i) { issued[i] = 0; last_par[i] = 0; }
      for (long long t = t0; t < tiles && ok; t += tstep) {
        int mt, nt;
        tile_coords(t, MT, NT, p.m_fast, p.n_group, mt, nt);
        const int bi = bt > 1 ? mt / MTp : 0;
        const int arow = mt * BM * CG + (int)rank * BM,
                  brow = nt * BN + (int)rank * C::kBRows + bi * p.b_pitch;
        for (int kb = 0; kb < KB; ++kb) {
          if (!mbar_wait(empty_bar(s), ph ^ 1u, p.err)) { ok = false; break; }
          if constexpr (CG == 2) {
            const uint32_t fb = lead(full_bar(s));
            mbar_expect_tx_cluster(fb, C::kStage);
#pragma unroll
            for (int pl = 0; pl < NP; ++pl)
              tma_load_3d_pair(a_tile(s, pl), &tmA, fb, kb * BK, arow, pl);
#pragma unroll
            for (int pl = 0; pl < NP; ++pl)
              tma_load_3d_pair(b_tile(s, pl), &tmB, fb, kb * BK, brow, pl);
          } else {
            mbar_expect_tx(full_bar(s), C::kStage);
#pragma unroll
            for (int pl = 0; pl < NP; ++pl)
              tma_load_3d(a_tile(s, pl), &tmA, full_bar(s), kb * BK, arow, pl);
#pragma unroll
            for (int pl = 0; pl < NP; ++pl)
              tma_load_3d(b_tile(s, pl), &tmB, full_bar(s), kb * BK, brow, pl);
          }
          issued[s] = 1;
          last_par[s] = ph;
          if (++s == C::kStages) { s = 0; ph ^= 1u; }
        }
      }
      if (!ok && rank == 0) {
        // Let copies already in flight land before the CTA can exit (the
        // odd CTA's copies are counted on the even CTA's barriers).
        for (int s2 = 0; s2 < C::kStages; ++s2)
          if (issued[s2]) mbar_wait(full_bar(s2), last_par[s2], p.err);
      }
    }
  } else if (warp == kMma) {
    if (lane == 0 && rank == 0) {
      using P = Pairs<NP>;
      constexpr uint32_t idesc = idesc_bf16(BM * CG, BN);
      constexpr uint32_t idesc2 = idesc_bf16(BM, 2 * BN);   // hh and (0, 1) together
      constexpr int q0 = CG == 1 ? 2 : 0;
      int s = 0;
      uint32_t ph = 0;
      int acc = 0;
      uint32_t acc_ph = 0;
      bool ok = true;
      for (long long t = t0; t < tiles && ok; t += tstep) {
        for (int c = 0; c < nchunks && ok; ++c) {
          if (!mbar_wait(tempty_bar(acc), acc_ph ^ 1u, p.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d_hh = tmem_base + (uint32_t)(acc * 2 * BN);
          const uint32_t d_rest = d_hh + BN;
          const int kb0 = c * kchunk, kb1 = min(KB, kb0 + kchunk);
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(full_bar(s), ph, p.err)) { ok = false; break; }
            tc_fence_after();
            const bool first = kb == kb0;   // the chunk's first slab resets both accumulators
            // descriptors of A and B plane 0 of this stage; a plane and a K step
            // are fixed byte offsets, added to the descriptor's address field
            // (address >> 4; stays below 2^14 inside shared memory)
            const uint64_t ad = sdesc<BK>(a_tile(s, 0)), bd = sdesc<BK>(b_tile(s, 0));
            if constexpr (CG == 1) {
              // hi * hi into hh and A0 * B1 into rest (= hh + BN): one N = 2 BN MMA
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk)
                tc_mma(d_hh, ad + 2 * kk, bd + 2 * kk, idesc2, (first && kk == 0) ? 0u : 1u);
            }
#pragma unroll
            for (int q = q0; q < P::n; ++q) {
              // product 0 (hi * hi) has its own, exactly accumulated, TMEM buffer
              const uint32_t d = (q == 0) ? d_hh : d_rest;
              const bool reset = first && q <= 1;
              const uint64_t aq = ad + (uint64_t)(P::a(q) * C::kAPlane / 16);
              const uint64_t bq = bd + (uint64_t)(P::b(q) * C::kBPlane / 16);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                if constexpr (CG == 2)
                  tc_mma_pair(d, aq + 2 * kk, bq + 2 * kk, idesc, (reset && kk == 0) ? 0u : 1u);
                else
                  tc_mma(d, aq + 2 * kk, bq + 2 * kk, idesc, (reset && kk == 0) ? 0u : 1u);
              }
            }
            if constexpr (CG == 2) tc_commit_pair(empty_bar(s), 3);   // both CTAs' stage s
            else tc_commit(empty_bar(s));
            if (++s == C::kStages) { s = 0; ph ^= 1u; }
          }
          if (!ok) break;
          if constexpr (CG == 2) tc_commit_pair(tfull_bar(acc), 3);
          else tc_commit(tfull_bar(acc));
          if (++acc == 2) { acc = 0; acc_ph ^= 1u; }
        }
      }
      // All MMAs issued by this thread (into both CTAs' TMEM) must finish
      // before TMEM is freed.
      if constexpr (CG == 2) tc_commit_pair(drain_bar, 1);
      else tc_commit(drain_bar);
      mbar_wait(drain_bar, 0, p.err);
    }
  } else {
    // Epilogue warps 0..15: warp w owns TMEM lanes [32 (w % 4), +32) (tile
    // rows) and column group cg = w / 4, columns [cg kCols, +kCols).  Chunk
    // sums hh + rest are added into a float-float running sum held in
    // registers.
    constexpr int kEpiThreads = C::kEpiWarps * 32;
    int acc = 0;
    uint32_t acc_ph = 0;
    bool ok = true;
    const int quad = warp & 3, cg = warp >> 2;
    const int row = quad * 32 + lane;
    const int col0 = cg * C::kCols;
    const uint32_t lane_base = tmem_base + ((uint32_t)(quad * 32) << 16);
    float rhi[C::kCols], rlo[C::kCols];
    for (long long t = t0; t < tiles && ok; t += tstep) {
      int mt, nt;
      tile_coords(t, MT, NT, p.m_fast, p.n_group, mt, nt);
      const int bi = bt > 1 ? mt / MTp : 0;
      const int m0 = (mt - bi * MTp) * BM * CG + (int)rank * BM, n0 = nt * BN;
      const int m = m0 + row;
      const bool mok = m < p.M;
      const long long coff = mok ? imap(p.cm, m) + bi * p.c_batch : 0;
      for (int c = 0; c < nchunks; ++c) {
        // warp-uniform wait: a lane that gave up stops its whole warp
        const bool w_ok = __all_sync(0xffffffffu, mbar_wait(tfull_bar(acc), acc_ph, p.err));
        if (!w_ok) { ok = false; break; }
        tc_fence_after();
        const uint32_t thh = lane_base + (uint32_t)(acc * 2 * BN + col0);
        const uint32_t trs = thh + BN;
        // 8 columns at a time keeps the live registers (the 2 x kCols running
        // sums plus the loaded chunk) under the 168-register budget
#pragma unroll
        for (int g = 0; g < C::kCols / 8; ++g) {
          float a[8], b[8];
          tmem_ld8(thh + g * 8, a);
          tmem_ld8(trs + g * 8, b);
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float& hi = rhi[g * 8 + j];
            float& lo = rlo[g * 8 + j];
            // float-float sum of the chunk's hh + rest into (hi, lo)
            float s, e;
            two_sum(a[j], b[j], s, e);
            if (c == 0) {
              hi = s;
              lo = e;
            } else {
              float u, f;
              two_sum(hi, s, u, f);
              f += lo + e;
              hi = u + f;
              lo = f - (hi - u);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if constexpr (CG == 2) mbar_arrive_cluster(lead(tempty_bar(acc)));
          else mbar_arrive(tempty_bar(acc));
        }
        if (++acc == 2) { acc = 0; acc_ph ^= 1u; }
      }
      // column offsets of this tile (shared by the epilogue warps); the
      // AND-barrier also makes every epilogue warp stop together after a failure
      ok = named_bar_and(1, kEpiThreads, ok);
      if (!ok) break;
      for (int j = threadIdx.x; j < BN; j += kEpiThreads)
        cn_s[j] = (n0 + j < p.N) ? imap(p.cn, n0 + j) : -1;
      named_bar(1, kEpiThreads);
      if (threadIdx.x < BN / 16) {
        int okc = cn_s[threadIdx.x * 16] >= 0;
        for (int j = 1; j < 16 && okc; ++j)
          okc = (cn_s[threadIdx.x * 16 + j] == cn_s[threadIdx.x * 16 + j - 1] + 1);
        cv_s[threadIdx.x] = okc;
      }
      named_bar(1, kEpiThreads);
      if (p.out_mode == kOutGridSplit) {
        // value as the FP32 output would hold it, and this thread's run start
        float mx = 0.f;
#pragma unroll
        for (int j = 0; j < C::kCols; ++j) {
          rhi[j] = p.alpha * (rhi[j] + rlo[j]);
          mx = fmaxf(mx, fabsf(rhi[j]));
        }
        // This thread's kCols columns are one run of an aligned 128-element
        // segment of the destination, made of two 64-element halves of kH
        // runs each: the other runs of its half belong to the column groups
        // next to it (same row), those of the partner half to the other
        // groups of the same row (seg_phalf) or the same groups of row ^
        // seg_prow.  The segment maximum sets the grid of plane 0.
        constexpr int kH = 64 / C::kCols;    // threads per 64-element half
        const int sub = cg % kH, hf = cg / kH;
        long long o = -1;
        if (mok) {
          o = coff + cn_s[col0];
          bool run = (o & 63) == C::kCols * sub && o >= 0 && o + C::kCols <= p.c_lim;
#pragma unroll
          for (int g = 0; g < C::kCols / 16; ++g)
            run = run && cv_s[col0 / 16 + g] && cn_s[col0 + 16 * g] == cn_s[col0] + 16 * g;
          if (!run) o = -1;
        }
        xm_s[cg * BM + row] = mx;
        xo_s[cg * BM + row] = o;
        named_bar(1, kEpiThreads);
        const long long hs = o - C::kCols * sub;   // start of this thread's half
        bool seg_ok = true;
        float pm = 0.f;
#pragma unroll
        for (int j = 0; j < kH; ++j) {
          const int own = (hf * kH + j) * BM + row;
          const int par = ((hf ^ p.seg_phalf) * kH + j) * BM + (row ^ p.seg_prow);
          pm = fmaxf(pm, fmaxf(xm_s[own], xm_s[par]));
          seg_ok = seg_ok && xo_s[own] == hs + C::kCols * j &&
                   xo_s[par] == (hs ^ 64) + C::kCols * j;
        }
        // CG = 2: the exchange lives in the staging buffers, which the stores
        // below overwrite: every warp must have read its partners first
        if constexpr (CG == 2) named_bar(1, kEpiThreads);
        const bool valid = mok && o >= 0 && seg_ok;
        if (mok && !valid) report_error(p.err, kErrBounds);
        // grid of the segment (the rule of kernels.cu: grid_split); v / g is
        // taken as v * (1/g), the same exactly rounded value (g a power of 2)
        const float smax = fmaxf(mx, pm);
        int e = 0;
        frexpf(smax, &e);
        const int ge = max(e - 8, -126);
        const float gq = (smax > 0.f) ? ldexpf(1.f, ge) : 1.f;
        const float gi = (smax > 0.f) ? ldexpf(1.f, -ge) : 1.f;
        const bool coop = __all_sync(0xffffffffu, valid);
        __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(p.C) + (valid ? o : 0);
        uint8_t* stage = stg_s + warp * C::kStageBytes;
        // plane by plane, 32 columns at a time: rhi holds the remainder still
        // to be split (v, then v - plane0, then v - plane0 - plane1)
#pragma unroll
        for (int hh = 0; hh < C::kCols / 32; ++hh) {
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            uint32_t pk[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              __nv_bfloat16 b[2];
#pragma unroll
              for (int t = 0; t < 2; ++t) {
                float& v = rhi[hh * 32 + 2 * i + t];
                b[t] = (q == 0) ? __float2bfloat16_rn(rintf(v * gi) * gq) : __float2bfloat16_rn(v);
                v = v - __bfloat162float(b[t]);
              }
              pk[i] = pack_bf16x2(b[0], b[1]);
            }
            uint4 v4[4];
#pragma unroll
            for (int c = 0; c < 4; ++c)
              v4[c] = make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
            char* d = reinterpret_cast<char*>(dst + q * p.out_plane_stride + hh * 32);
            if (coop) {
              warp_store64<C::kStageBytes>(stage, v4, d, lane);
            } else if (valid) {
#pragma unroll
              for (int c = 0; c < 4; ++c) reinterpret_cast<uint4*>(d)[c] = v4[c];
            }
          }
        }
      } else {
        // FP32 / FP64 output: 64-byte runs (16 floats or 8 doubles) through the
        // warp's staging buffer when every lane's run is contiguous and aligned
        uint8_t* stage = stg_s + warp * C::kStageBytes;
#pragma unroll
        for (int g = 0; g < C::kCols / 16; ++g) {
          const int cc = col0 + g * 16;
          const long long off0 = coff + cn_s[cc];
          const float* hi = rhi + g * 16;
          const float* lo = rlo + g * 16;
          const bool f32 = p.out_mode == kOutF32;
          const bool run = mok && cv_s[cc / 16] && !p.accumulate && off0 >= 0 &&
                           off0 + 15 < p.c_lim && (off0 & (f32 ? 3 : 1)) == 0 &&
                           (reinterpret_cast<uintptr_t>(p.C) & 15) == 0;
          if (__all_sync(0xffffffffu, run)) {
            if (f32) {
              uint4 v4[4];
#pragma unroll
              for (int c = 0; c < 4; ++c)
                v4[c] = make_uint4(__float_as_uint(p.alpha * (hi[4 * c] + lo[4 * c])),
                                   __float_as_uint(p.alpha * (hi[4 * c + 1] + lo[4 * c + 1])),
                                   __float_as_uint(p.alpha * (hi[4 * c + 2] + lo[4 * c + 2])),
                                   __float_as_uint(p.alpha * (hi[4 * c + 3] + lo[4 * c + 3])));
              warp_store64<C::kStageBytes>(
                  stage, v4, reinterpret_cast<char*>(reinterpret_cast<float*>(p.C) + off0), lane);
            } else {
#pragma unroll
              for (int hv = 0; hv < 2; ++hv) {
                uint4 v4[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                  const int j = hv * 8 + 2 * c;
                  const double d0 = (double)p.alpha * ((double)hi[j] + (double)lo[j]);
                  const double d1 = (double)p.alpha * ((double)hi[j + 1] + (double)lo[j + 1]);
                  const unsigned long long u0 = __double_as_longlong(d0),
                                           u1 = __double_as_longlong(d1);
                  v4[c] = make_uint4((uint32_t)u0, (uint32_t)(u0 >> 32), (uint32_t)u1,
                                     (uint32_t)(u1 >> 32));
                }
                warp_store64<C::kStageBytes>(
                    stage, v4,
                    reinterpret_cast<char*>(reinterpret_cast<double*>(p.C) + off0 + hv * 8), lane);
              }
            }
          } else if (mok) {
            store_tile_chunk<BN, NP>(p, coff, cn_s, cv_s[cc / 16], cc, hi, lo);
          }
        }
      }
    }
  }

  __syncwarp();
  tc_fence_before();
  // CG = 2: neither CTA frees its TMEM or exits while the pair's MMAs or the
  // other CTA's barrier arrivals may still reach it
  if constexpr (CG == 2) cluster_sync();
  else __syncthreads();
  tc_fence_after();
  if (warp == kMma) {
    if constexpr (CG == 2)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                   "r"(C::kTmemCols)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                   "r"(C::kTmemCols)
                   : "memory");
  }
}
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  });
  return fn;
}

bool make_map(CUtensorMap* tm, const TcOperand& op, int box_rows, int bk) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)op.K, (cuuint64_t)op.rows, (cuuint64_t)op.planes};
  cuuint64_t strides[2] = {(cuuint64_t)op.K * 2, (cuuint64_t)op.plane_stride * 2};
  cuuint32_t box[3] = {(cuuint32_t)bk, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(op.ptr), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN, int NP, int BK, int CG = 1>
cudaError_t launch(const TcOperand& A, const TcOperand& B, const TcGemm& g, cudaStream_t stream,
                   int num_sms) {
  using C = Cfg<BN, NP, BK, CG>;
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, BM, BK) || !make_map(&tb, B, C::kBRows, BK)) return cudaErrorInvalidValue;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<BN, NP, BK, CG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  long long mtiles = (g.M + BM * CG - 1) / (BM * CG);
  if (g.batch > 1) {
    if (g.a_pitch % (BM * CG) != 0 || g.a_pitch < g.M || g.b_pitch < g.N ||
        (long long)A.rows < (long long)g.batch * g.a_pitch ||
        (long long)B.rows < (long long)(g.batch - 1) * g.b_pitch + g.N)
      return cudaErrorInvalidValue;
    mtiles = (long long)g.batch * (g.a_pitch / (BM * CG));
  }
  const long long tiles = mtiles * ((g.N + BN - 1) / BN);
  count_launch();
  if constexpr (CG == 1) {
    int grid = (int)(tiles < num_sms ? tiles : num_sms);
    tc_gemm_kernel<BN, NP, BK, 1><<<grid, C::kThreads, C::kSmem, stream>>>(ta, tb, g);
    return cudaGetLastError();
  } else {
    // persistent clusters of two CTAs: one pair per two SMs (or per tile)
    const long long pairs = num_sms / 2 < tiles ? num_sms / 2 : tiles;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(2 * pairs), 1, 1);
    cfg.blockDim = dim3(C::kThreads, 1, 1);
    cfg.dynamicSmemBytes = C::kSmem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tc_gemm_kernel<BN, NP, BK, 2>, ta, tb, g);
  }
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing
// arrives at; the wait must give up after `limit` cycles and set kErrTimeout.
__global__ void bounded_wait_probe_kernel(int* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait(smem_u32(&bar), 0, err, limit);
  }
}

}  // namespace

cudaError_t bounded_wait_probe(int* err, long long limit_cycles, cudaStream_t stream) {
  count_launch();
  bounded_wait_probe_kernel<<<1, 32, 0, stream>>>(err, limit_cycles);
  return cudaGetLastError();
}

void tc_set_pairs(TcGemm& g, int nplanes) {
  // The kernel forms the products of Pairs<nplanes>; the list is recorded
  // here for the host-side checks and for callers that inspect it.
  g.nplanes = nplanes;
  auto take = [&](auto pairs) {
    using P = decltype(pairs);
    g.npairs = P::n;
    for (int i = 0; i < P::n; ++i) { g.pa[i] = P::a(i); g.pb[i] = P::b(i); }
  };
  if (nplanes == 4) take(Pairs<4>());
  else if (nplanes == 2) take(Pairs<2>());
  else take(Pairs<3>());
}

cudaError_t tc_gemm(const TcOperand& A, const TcOperand& B, const TcGemm& g, cudaStream_t stream,
                    int num_sms) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (A.K != B.K || A.K != g.K || A.K % 8 != 0 || A.rows < g.M || B.rows < g.N ||
      A.planes != g.nplanes || B.planes != g.nplanes || g.npairs < 1 || g.pa[0] != 0 ||
      g.pb[0] != 0)
    return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(A.ptr) | reinterpret_cast<uintptr_t>(B.ptr)) & 15)
    return cudaErrorInvalidValue;
  if (g.out_mode == kOutGridSplit &&
      (g.N <= 64 || g.M % BM != 0 || g.N % 128 != 0 || g.out_planes != 3 || g.accumulate ||
       g.seg_prow < 0 || g.seg_prow >= BM || g.seg_phalf < 0 || g.seg_phalf > 1 ||
       (g.seg_prow == 0 && g.seg_phalf == 0) || g.out_plane_stride % 64 != 0 ||
       (reinterpret_cast<uintptr_t>(g.C) & 15) != 0))
    return cudaErrorInvalidValue;
  // K slab: 64 (two 96 KB stages) for two and three planes, where it measured
  // faster (48.1 vs 57.4 ms per D = 64 stage-2 launch); 32 (three 64 KB stages)
  // for four planes, which lets them use 128-wide N tiles.
  const int bk = g.bk ? g.bk : (g.nplanes == 4 ? 32 : 64);
  if (bk == 64) {
    if (g.nplanes == 2) {
      if (g.N > 64) return launch<128, 2, 64>(A, B, g, stream, num_sms);
      return launch<64, 2, 64>(A, B, g, stream, num_sms);
    }
    if (g.nplanes == 3) {
      if (g.N > 64 && g.cta_pair && num_sms >= 2) return launch<128, 3, 64, 2>(A, B, g, stream, num_sms);
      if (g.N > 64) return launch<128, 3, 64>(A, B, g, stream, num_sms);
      return launch<64, 3, 64>(A, B, g, stream, num_sms);
    }
    if (g.nplanes == 4) return launch<64, 4, 64>(A, B, g, stream, num_sms);
    return cudaErrorInvalidValue;
  }
  if (g.nplanes == 2) {
    if (g.N > 64) return launch<128, 2, 32>(A, B, g, stream, num_sms);
    return launch<64, 2, 32>(A, B, g, stream, num_sms);
  }
  if (g.nplanes == 3) {
    if (g.N > 64) return launch<128, 3, 32>(A, B, g, stream, num_sms);
    return launch<64, 3, 32>(A, B, g, stream, num_sms);
  }
  if (g.nplanes == 4) {
    if (g.N > 64) return launch<128, 4, 32>(A, B, g, stream, num_sms);
    return launch<64, 4, 32>(A, B, g, stream, num_sms);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hotrg
