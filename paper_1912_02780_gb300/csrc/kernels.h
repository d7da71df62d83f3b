// Launchers of the memory-bound helper kernels (see kernels.cu).
#pragma once
#include "common.cuh"

namespace hotrg {

// dst planes [p][r][K] = bf16 split of src[rm(r) + km(k)]; source offsets at
// or beyond src_lim are read as 0 and flagged (kErrBounds).
cudaError_t gather_split(const double* src, long long src_lim, IMap rm, IMap km, int rows, int K,
                         int nplanes, long long plane_stride, __nv_bfloat16* dst, int* err,
                         cudaStream_t st, int sms);
// Grid-aligned bf16 split (segments of kGridSeg along K, see kernels.cu):
// the operand preparation the tensor-core GEMM's exact hi*hi accumulation needs.
constexpr int kGridSeg = 128;
cudaError_t grid_split(const double* src, long long src_lim, IMap rm, IMap km, int rows, int K,
                       int nplanes, long long plane_stride, __nv_bfloat16* dst, int* err,
                       cudaStream_t st, int sms);
cudaError_t grid_split(const float* src, long long src_lim, IMap rm, IMap km, int rows, int K,
                       int nplanes, long long plane_stride, __nv_bfloat16* dst, int* err,
                       cudaStream_t st, int sms);
cudaError_t ising_t0(double beta, double J, double h, double* T0, double* dT0, cudaStream_t st);
// x <- x / ||x||_F (FP64, deterministic), *log_norm = ln ||x||_F.
cudaError_t frob_normalize(double* x, long long n, double* partial, int max_partial,
                           double* log_norm, double* inv_scratch, int* err, cudaStream_t st,
                           int sms);
cudaError_t trace_lnz(const double* T, int P, int Q, const double* log_norms, int n, double* out,
                      double* trace_out, int* err, cudaStream_t st);
cudaError_t eig_desc(const double* asc, const double* w_asc, int N, int ncols, int rows_out,
                     double* desc, double* lam_desc, cudaStream_t st);
cudaError_t diag_trace(const double* G, int N, double* out, cudaStream_t st);
cudaError_t eig_diag(const double* lam, int nlam, int N, int Dp, const double* trace, double* trunc,
                     double* gap, cudaStream_t st);
// Kept Ritz pairs (rows of V, values lam descending) against Z = V G:
// *res = max_{a < Dp} ||Z_a - lam_a V_a||_2 / lam_0; *guard = max(*guard, code)
// when *res > tol.  row_scratch holds Dp doubles.
cudaError_t eig_residual(const double* Z, const double* V, const double* lam, int Dp, int N,
                         double tol, double* row_scratch, double* res, int* guard, int code,
                         cudaStream_t st);
cudaError_t eigh_info_check(const int* info, int* err, cudaStream_t st);
cudaError_t seed_trace_adjoint(double* E, int P, int Q, const double* tr, cudaStream_t st, int sms);
cudaError_t eigh_adj_scale(double* S, int nd, int Dp, const double* lam, double eta_rel,
                           cudaStream_t st, int sms);
cudaError_t symmetrize(double* G, int N, cudaStream_t st, int sms);
cudaError_t scale_copy(const double* x, double* y, long long n, double a, cudaStream_t st, int sms);
// x <- x * exp(-*logc)  (divide by a norm whose log lives on the device)
cudaError_t scale_exp_neg(double* x, long long n, const double* logc, cudaStream_t st, int sms);
cudaError_t fill_random(double* x, long long n, unsigned long long seed, cudaStream_t st, int sms);
// *x = v (if x) and *err |= bits (if err): used by the fault-injection hooks.
cudaError_t set_value(double* x, double v, int* err, int bits, cudaStream_t st);
cudaError_t dot_small(const double* a, const double* b, int n, double* out, cudaStream_t st);
// out[c][d][a][b] = in[a][b][c][d] for in of shape (P, P, Q, Q).
cudaError_t swap_pairs(const double* in, double* out, int P, int Q, cudaStream_t st, int sms);
// T0 (4 x 4 x 4 x 4) of the quantum XY chain's second-order Trotter MPO rho(tau).
cudaError_t xy_mpo(double tau, double J, double* T0, cudaStream_t st);
// *out = ||a - b||_F (n up to a few million).
cudaError_t diff_norm(const double* a, const double* b, long long n, double* out, cudaStream_t st);
// Scheme-(b) value of a depth-n chain, v = sum_k ln c_k / 2^k + lnlam / 2^(n+1):
// out (if not NULL) = [v, 1, ln c_1 .. ln c_n]; *step_out (if not NULL) = v.
cudaError_t chain_lnz(const double* log_norms, int n, const double* lnlam, double* out,
                      double* step_out, cudaStream_t st);
// w_rule 1: *side = (*trunc_l - *trunc_r > tie); dst = src where *flag.
cudaError_t w_rule_choose(const double* trunc_l, const double* trunc_r, double tie, int* side,
                          cudaStream_t st);
cudaError_t cond_copy(const int* flag, const double* src, double* dst, long long n,
                      cudaStream_t st, int sms);
// V = identity / sqrt(X) (X x X).
cudaError_t eye_unit(double* V, int X, cudaStream_t st, int sms);

}  // namespace hotrg
