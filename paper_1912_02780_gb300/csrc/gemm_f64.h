// FP64 CUDA-core GEMM with mixed-radix operand maps (see gemm_f64.cu).
#pragma once
#include "common.cuh"

namespace hotrg {

struct GemmF64 {
  const double* A; IMap am, ak;   // A(m, k) = A[am(m) + ak(k)]
  const double* B; IMap bn, bk;   // B(n, k) = B[bn(n) + bk(k)]
  double* C; IMap cm, cn;         // C(m, n) = C[cm(m) + cn(n)]
  int M, N, K;
  double alpha, beta;             // C = alpha * A B^T + beta * C (beta = 0: C not read)
  int a_kfast, b_kfast;           // 1 if k is the operand's fastest index (load order hint)
  long long a_lim, b_lim, c_lim;  // element counts behind A, B, C: accesses at or beyond
                                  // them are skipped and flagged (kErrBounds)
  int* err;
  double* ws;                     // optional split-K workspace: split-K partials are summed in
  long long ws_elems;             // a fixed order; splits are limited to what it holds (none:
                                  // no split-K), so the result is always deterministic
};

cudaError_t gemm_f64(const GemmF64& p, cudaStream_t stream, int num_sms);

}  // namespace hotrg
