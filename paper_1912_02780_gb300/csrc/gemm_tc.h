// Split-BF16 tcgen05 GEMM (see gemm_tc.cu).
#pragma once
#include "common.cuh"

namespace hotrg {

// A K-major operand stored as `planes` bf16 planes [plane][rows][K] (K a
// multiple of 8 so that every row starts on a 16-byte boundary).
struct TcOperand {
  const __nv_bfloat16* ptr;
  int rows, K, planes;
  long long plane_stride;   // elements between planes (>= rows * K)
};

// kOutGridSplit: the tile is written as grid-aligned bf16 planes (the split
// the next GEMM reads, see kernels.cu: grid_split) of alpha * sum rounded to
// FP32, bit for bit what kOutF32 followed by grid_split would produce.  Each
// epilogue thread holds 64 consecutive columns of one row; they must map to 64
// contiguous destination elements, and together with the 64 of its partner
// (row ^ seg_prow, column half ^ seg_phalf) fill one aligned 128-element
// segment of the destination (checked on the device: kErrBounds otherwise).
enum TcOutMode : int { kOutF32 = 0, kOutF64 = 1, kOutGridSplit = 2 };

struct TcGemm {
  int M, N, K;
  int nplanes;               // operand planes (2 or 3)
  int npairs;                // products formed per K slab
  int pa[10], pb[10];        // plane of A / of B for each product (product 0 = hi * hi)
  int kchunk;                // K-blocks (of 64) per FP32 accumulation chunk; chunks are summed
                             // in compensated float-float; >= ceil(K/64) means one chunk
  IMap cm, cn;               // output element (m, n) at C + cm(m) + cn(n)
  int out_mode;              // TcOutMode
  int out_planes;            // planes written for kOutGridSplit (3)
  long long out_plane_stride;
  void* C;
  float alpha;               // output = alpha * sum
  int accumulate;            // kOutF32/kOutF64: C += output
  long long c_lim;           // elements per output plane: stores at or beyond are skipped
                             // and flagged (kErrBounds)
  int* err;                  // device error word
  int bk;                    // K slab per pipeline stage: 32 or 64 (0: 64 for two or three
                             // planes, 32 for four)
  int m_fast;                // tile order: 1 = consecutive tiles walk M (B tile reused from
                             // L2 by neighbouring CTAs), 0 = consecutive tiles walk N
  int n_group;               // with m_fast = 0 and n_group > 0: tiles in groups of n_group
                             // N-tiles (an L2-resident stripe of B), M-major inside
  int cta_pair;              // 1: run a three-plane, 64-wide-K, N > 64 GEMM on CTA pairs
                             // (tcgen05 cta_group::2, 256-row tiles); same results
  int seg_prow, seg_phalf;   // kOutGridSplit: segment partner of (row, half)
  int batch;                 // > 1: that many independent problems of this shape in one launch
                             // (a grouped launch): problem b reads A rows from b * a_pitch and
                             // B rows from b * b_pitch and writes at C + b * c_batch (plus the
                             // cm / cn offsets); a_pitch a multiple of the row tile, >= M;
                             // b_pitch >= N.  0 or 1: one problem.
  int a_pitch, b_pitch;
  long long c_batch;
};

// Set the products of a precision: all plane pairs (i, j) with
// i + j <= nplanes - 1 (3, 6 or 10 products for 2, 3 or 4 planes), hi * hi first.
void tc_set_pairs(TcGemm& g, int nplanes);

// Launch a single-thread kernel whose mbarrier wait can never complete; it
// gives up after limit_cycles and sets kErrTimeout in *err (self-test).
cudaError_t bounded_wait_probe(int* err, long long limit_cycles, cudaStream_t stream);

cudaError_t tc_gemm(const TcOperand& A, const TcOperand& B, const TcGemm& g, cudaStream_t stream,
                    int num_sms);

}  // namespace hotrg
