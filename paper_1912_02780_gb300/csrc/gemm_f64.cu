// FP64 GEMM on CUDA cores with mixed-radix operand maps.
//
//   C(m, n) = alpha * sum_k A(m, k) * B(n, k) + beta * C(m, n)
//
// A(m, k) lives at A + imap(am, m) + imap(ak, k), and likewise for B and C,
// so a HOTRG contraction (SM Sec. B, HOTRG step equation and its adjoints)
// runs directly on the tensors in their natural layout, without permuted
// copies.  This is the FP64 path; its speed is set by the FP64 pipe of the
// device (about 2 DFMA per clock per SM on GB300), not by memory, so the
// kernel keeps one 64x64 tile per 256-thread block with 4x4 outputs per
// thread and a 16-deep K slab in shared memory.  Very long K with a small
// output grid is split across blocks (split-K) when the caller provides a
// workspace for the partials, which are then summed in a fixed order, so the
// result never depends on the order in which blocks finish.
#include "common.cuh"
#include "gemm_f64.h"

namespace hotrg {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

__global__ void __launch_bounds__(256) gemm_f64_kernel(GemmF64 p, int k_per_split) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  __shared__ long long a_row[BM], b_row[BN], a_col[BK], b_col[BK];

  const int t = threadIdx.x;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int k_begin = blockIdx.z * k_per_split;
  const int k_end = min(p.K, k_begin + k_per_split);

  if (t < BM) a_row[t] = (m0 + t < p.M) ? imap(p.am, m0 + t) : -1;
  else if (t < BM + BN) b_row[t - BM] = (n0 + t - BM < p.N) ? imap(p.bn, n0 + t - BM) : -1;

  const int tx = t % 16, ty = t / 16;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int kb = k_begin; kb < k_end; kb += BK) {
    __syncthreads();
    if (t < BK) a_col[t] = (kb + t < k_end) ? imap(p.ak, kb + t) : -1;
    else if (t < 2 * BK) b_col[t - BK] = (kb + t - BK < k_end) ? imap(p.bk, kb + t - BK) : -1;
    __syncthreads();
    // 1024 elements of each operand tile, 4 per thread.
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int idx = t + e * 256;
      int kk, rr;
      if (p.a_kfast) { kk = idx % BK; rr = idx / BK; } else { rr = idx % BM; kk = idx / BM; }
      long long ro = a_row[rr], co = a_col[kk];
      double av = 0.0;
      if (ro >= 0 && co >= 0) {
        if (ro + co < p.a_lim) av = p.A[ro + co];
        else report_error(p.err, kErrBounds);
      }
      As[kk][rr] = av;
      if (p.b_kfast) { kk = idx % BK; rr = idx / BK; } else { rr = idx % BN; kk = idx / BN; }
      ro = b_row[rr]; co = b_col[kk];
      double bv = 0.0;
      if (ro >= 0 && co >= 0) {
        if (ro + co < p.b_lim) bv = p.B[ro + co];
        else report_error(p.err, kErrBounds);
      }
      Bs[kk][rr] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int m = m0 + ty + 16 * i;
    if (m >= p.M) continue;
    long long cr = imap(p.cm, m);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = n0 + tx + 16 * j;
      if (n >= p.N) continue;
      const long long off = cr + imap(p.cn, n);
      if (off < 0 || off >= p.c_lim) {
        report_error(p.err, kErrBounds);
        continue;
      }
      double* c = p.C + off;
      double v = p.alpha * acc[i][j];
      if (gridDim.z > 1) {
        p.ws[((long long)blockIdx.z * p.M + m) * p.N + n] = acc[i][j];
      } else {
        *c = (p.beta != 0.0) ? v + p.beta * *c : v;
      }
    }
  }
}

// Fixed-order sum of the split-K partials: C = alpha * sum_z ws[z] + beta * C.
__global__ void splitk_reduce_kernel(GemmF64 p, int splits) {
  long long total = (long long)p.M * p.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int m = (int)(i / p.N), n = (int)(i % p.N);
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += p.ws[(long long)z * total + i];
    const long long off = imap(p.cm, m) + imap(p.cn, n);
    if (off < 0 || off >= p.c_lim) {
      report_error(p.err, kErrBounds);
      continue;
    }
    double* c = p.C + off;
    *c = (p.beta != 0.0) ? p.alpha * s + p.beta * *c : p.alpha * s;
  }
}

__global__ void scale_out_kernel(GemmF64 p) {
  // beta-scaling pass used before a split-K launch (C <- beta * C).
  long long total = (long long)p.M * p.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int m = (int)(i / p.N), n = (int)(i % p.N);
    const long long off = imap(p.cm, m) + imap(p.cn, n);
    if (off < 0 || off >= p.c_lim) {
      report_error(p.err, kErrBounds);
      continue;
    }
    double* c = p.C + off;
    *c = (p.beta != 0.0) ? p.beta * *c : 0.0;
  }
}

}  // namespace

cudaError_t gemm_f64(const GemmF64& p, cudaStream_t stream, int num_sms) {
  if (p.M <= 0 || p.N <= 0) return cudaSuccess;
  dim3 grid((p.N + BN - 1) / BN, (p.M + BM - 1) / BM, 1);
  long long tiles = (long long)grid.x * grid.y;
  int splits = 1;
  long long target = 2LL * num_sms;
  if (tiles < target && p.K >= 4 * BK) {
    splits = (int)((target + tiles - 1) / tiles);
    int max_splits = (p.K + 4 * BK - 1) / (4 * BK);
    if (splits > max_splits) splits = max_splits;
    if (splits > 64) splits = 64;
    if (splits < 1) splits = 1;
  }
  int k_per_split = p.K;
  if (splits > 1) {
    k_per_split = ((p.K + splits - 1) / splits + BK - 1) / BK * BK;
    splits = (p.K + k_per_split - 1) / k_per_split;
  }
  if (splits > 1) {
    // as many splits as the workspace holds partials for (none: no split-K)
    const long long mn = (long long)p.M * p.N;
    const long long fit = p.ws ? p.ws_elems / mn : 0;
    if (fit < splits) {
      splits = fit >= 2 ? (int)fit : 1;
      k_per_split = splits > 1 ? ((p.K + splits - 1) / splits + BK - 1) / BK * BK : p.K;
      if (splits > 1) splits = (p.K + k_per_split - 1) / k_per_split;
    }
  }
  const bool det = splits > 1;
  if (splits > 1) grid.z = splits;
  if (p.K <= 0) {
    if (splits == 1) {
      GemmF64 q = p;
      long long total = (long long)p.M * p.N;
      int blocks = (int)((total + 255) / 256);
      if (blocks > 8 * num_sms) blocks = 8 * num_sms;
      count_launch();
      scale_out_kernel<<<blocks, 256, 0, stream>>>(q);
    }
    return cudaGetLastError();
  }
  GemmF64 q = p;
  count_launch();
  gemm_f64_kernel<<<grid, 256, 0, stream>>>(q, k_per_split);
  if (det) {
    long long total = (long long)p.M * p.N;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 8 * num_sms) blocks = 8 * num_sms;
    count_launch();
    splitk_reduce_kernel<<<blocks, 256, 0, stream>>>(p, splits);
  }
  return cudaGetLastError();
}

}  // namespace hotrg
