// Quasi-Newton (L-BFGS) optimisation of one layer's isometry in the
// exponential parametrisation of SM Sec. D, on the device.
//
// The isometry of layer k is w(B) = Q exp(B) E: B antisymmetric N x N
// (N = X_k^2), E the first D' columns of the identity, Q an orthogonal N x N
// matrix whose first D' columns are the isometry at the start of the run (the
// complete Householder QR factor of w, columns sign-fixed), so that B = 0 is
// the starting point; the paper's w = exp(B) is the case Q = I.  The
// objective is f = ln Z / N of the plan's network with every other isometry
// fixed; its gradient in the variables b_ij (i > j) of B = b - b^T is
//     d f / d b_ij = G_ij - G_ji,   G = L_exp(B^T, Q^T wbar E^T),
// L_exp the Frechet derivative of the matrix exponential, read off the
// upper-right block of exp([[B^T, C], [0, B^T]]) (Higham, Functions of
// Matrices, Thm. 3.6), wbar = d f / d w_k from the plan's backward with every
// isometry held fixed (main-text Eq. (1)).
//
// Matrix exponentials: scaling and squaring, exp(A) = (T_16(A / 2^s))^(2^s)
// with ||A / 2^s||_1 <= 1/2 and T_16 the degree-16 Taylor polynomial
// (truncation below 1e-19 relative), evaluated by Horner's rule, every
// product on the FP64 GEMM.  The variables are kept as full antisymmetric
// matrices; the inner product of the packed variables is half the Frobenius
// product of those matrices.
//
// L-BFGS: the two-loop recursion (Nocedal and Wright, Numerical Optimization,
// Algorithm 7.4) with H_0 = (s^T y / y^T y) I, the first step along the
// gradient scaled to length step0, backtracking from the full step with the
// Armijo condition, pairs with s^T y <= 0 (for -f) not stored.
#include <cusolverDn.h>
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/hotrg.h"
#include "common.cuh"
#include "gemm_f64.h"
#include "kernels.h"
#include "plan_access.h"

using namespace hotrg;

namespace {

__device__ __forceinline__ long long gtid() {
  return blockIdx.x * (long long)blockDim.x + threadIdx.x;
}
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

int nblocks(long long n, int sms) {
  long long b = (n + 255) / 256, cap = 16LL * sms;
  return (int)std::max(1LL, std::min(b, cap));
}

__global__ void eye_kernel(double* __restrict__ R, int n) {
  const long long t = (long long)n * n;
  for (long long i = gtid(); i < t; i += gstride()) R[i] = (i / n == i % n) ? 1.0 : 0.0;
}

// X2 (2N x 2N, row-major) = [[B^T, 0], [0, B^T]]; the upper-right block is
// filled by a GEMM afterwards.
__global__ void block_kernel(const double* __restrict__ B, int N, double* __restrict__ X2) {
  const long long n2 = 2LL * N, t = n2 * n2;
  for (long long i = gtid(); i < t; i += gstride()) {
    const int r = (int)(i / n2), c = (int)(i % n2);
    double v = 0.0;
    if ((r < N) == (c < N)) v = B[(long long)(c % N) * N + (r % N)];
    X2[i] = v;
  }
}

// G = U - U^T with U the upper-right N x N block of E2 (2N x 2N).
__global__ void antisym_block_kernel(const double* __restrict__ E2, int N, double scale,
                                     double* __restrict__ G) {
  const long long t = (long long)N * N, n2 = 2LL * N;
  for (long long i = gtid(); i < t; i += gstride()) {
    const int r = (int)(i / N), c = (int)(i % N);
    G[i] = scale * (E2[r * n2 + N + c] - E2[(long long)c * n2 + N + r]);
  }
}

__global__ void axpy_kernel(const double* __restrict__ x, double* __restrict__ y, long long n,
                            double a) {
  for (long long i = gtid(); i < n; i += gstride()) y[i] += a * x[i];
}

__global__ void axpby_kernel(const double* __restrict__ x, const double* __restrict__ y,
                             double* __restrict__ z, long long n, double a, double b) {
  for (long long i = gtid(); i < n; i += gstride()) z[i] = a * x[i] + b * y[i];
}

// *out = sum a_i b_i (one block, fixed reduction order).
__global__ void dot_kernel(const double* __restrict__ a, const double* __restrict__ b, long long n,
                           double* __restrict__ out) {
  __shared__ double ws[32];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s = fma(a[i], b[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    *out = t;
  }
}

// *out = max_c sum_r |A[r][c]| (the 1-norm; one block).
__global__ void norm1_kernel(const double* __restrict__ A, int n, double* __restrict__ out) {
  __shared__ double ws[1024];
  double m = 0.0;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < n; ++r) s += fabs(A[(long long)r * n + c]);
    m = fmax(m, s);
  }
  ws[threadIdx.x] = m;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) ws[threadIdx.x] = fmax(ws[threadIdx.x], ws[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = ws[0];
}

// sgn[j] = sign of the diagonal entry R_jj of a column-major QR factor.
__global__ void diag_sign_kernel(const double* __restrict__ QR, int N, int Dp,
                                 double* __restrict__ sgn) {
  for (int j = threadIdx.x; j < Dp; j += blockDim.x) sgn[j] = QR[(long long)j * N + j] < 0 ? -1.0 : 1.0;
}

// Q[:, j] *= sgn[j] for j < Dp (column-major N x N).
__global__ void scale_cols_kernel(double* __restrict__ Q, int N, int Dp,
                                  const double* __restrict__ sgn) {
  const long long t = (long long)N * Dp;
  for (long long i = gtid(); i < t; i += gstride()) Q[i] *= sgn[i / N];
}

}  // namespace

struct hotrg_lbfgs_s {
  hotrg_plan plan = nullptr;
  int m = 10;
  int Nmax = 0, Dmax = 0;
  cudaStream_t st = nullptr;
  int sms = 1;
  cusolverDnHandle_t solver = nullptr;
  std::vector<void*> allocs;
  // N x N (Nmax^2): base point, variables, trial, gradients, direction, pairs
  double *Q = nullptr, *B = nullptr, *Bn = nullptr, *G = nullptr, *Gn = nullptr, *P = nullptr;
  std::vector<double*> S, Y;
  // 2N x 2N (4 Nmax^2): exponential workspace
  double *X2 = nullptr, *E1 = nullptr, *E2 = nullptr;
  double* Wacc = nullptr;   // accepted isometry (D' x N rows)
  double* small = nullptr;  // device scalars and the QR diagonal signs
  double* tau = nullptr;
  double* work = nullptr;
  int lwork = 0;
  int* info = nullptr;
  std::string err;
};

namespace {

#define LCK(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return plan_fail(o->plan, HOTRG_ECUDA, cudaGetErrorString(e_)); \
  } while (0)

GemmF64 gm(const hotrg_lbfgs_s* o, const double* A, IMap am, IMap ak, long long alim,
           const double* B, IMap bn, IMap bk, long long blim, double* C, IMap cm, IMap cn,
           long long clim, int M, int N, int K, double alpha, double beta) {
  GemmF64 g;
  g.A = A; g.am = am; g.ak = ak; g.a_lim = alim;
  g.B = B; g.bn = bn; g.bk = bk; g.b_lim = blim;
  g.C = C; g.cm = cm; g.cn = cn; g.c_lim = clim;
  g.M = M; g.N = N; g.K = K;
  g.alpha = alpha; g.beta = beta;
  g.a_kfast = ak.s0 == 1;
  g.b_kfast = bk.s0 == 1;
  g.err = plan_err(o->plan);
  g.ws = nullptr;
  g.ws_elems = 0;
  return g;
}

double host_scalar(hotrg_lbfgs_s* o, const double* dev, hotrg_status* st) {
  double v = 0;
  *st = HOTRG_OK;
  if (cudaMemcpyAsync(&v, dev, sizeof(double), cudaMemcpyDeviceToHost, o->st) != cudaSuccess ||
      cudaStreamSynchronize(o->st) != cudaSuccess)
    *st = plan_fail(o->plan, HOTRG_ECUDA, "device scalar read failed");
  return v;
}

// C = A B (n x n row-major) on the FP64 GEMM.
cudaError_t matmul(hotrg_lbfgs_s* o, const double* A, const double* B, double* C, int n,
                   double alpha, double beta) {
  const long long t = (long long)n * n;
  return gemm_f64(gm(o, A, map_lin(n), map_lin(1), t, B, map_lin(1), map_lin(n), t, C, map_lin(n),
                     map_lin(1), t, n, n, n, alpha, beta),
                  o->st, o->sms);
}

// exp(A) for A (n x n) held in `a` (overwritten); returns the buffer (one of a,
// b, c) that holds the result.
hotrg_status expm(hotrg_lbfgs_s* o, double* a, double* b, double* c, int n, double** result) {
  const long long t = (long long)n * n;
  count_launch();
  norm1_kernel<<<1, 1024, 0, o->st>>>(a, n, o->small);
  LCK(cudaGetLastError());
  hotrg_status st;
  const double nrm = host_scalar(o, o->small, &st);
  if (st != HOTRG_OK) return st;
  if (!std::isfinite(nrm)) return plan_fail(o->plan, HOTRG_ENONFINITE, "expm: non-finite input");
  int s = 0;
  while (std::ldexp(nrm, -s) > 0.5) ++s;
  if (s > 0) LCK(scale_copy(a, a, t, std::ldexp(1.0, -s), o->st, o->sms));
  // Horner: R = I; for j = 16..1: R <- I + (A / j) R
  double* R = b;
  double* Rn = c;
  count_launch();
  eye_kernel<<<nblocks(t, o->sms), 256, 0, o->st>>>(R, n);
  LCK(cudaGetLastError());
  for (int j = 16; j >= 1; --j) {
    count_launch();
    eye_kernel<<<nblocks(t, o->sms), 256, 0, o->st>>>(Rn, n);
    LCK(cudaGetLastError());
    LCK(matmul(o, a, R, Rn, n, 1.0 / j, 1.0));
    std::swap(R, Rn);
  }
  // squarings (the scaled input in `a` is no longer needed)
  double* spare = a;
  for (int i = 0; i < s; ++i) {
    LCK(matmul(o, R, R, spare, n, 1.0, 0.0));
    std::swap(R, spare);
  }
  *result = R;
  return HOTRG_OK;
}

double half_dot(hotrg_lbfgs_s* o, const double* x, const double* y, long long n,
                hotrg_status* st) {
  count_launch();
  dot_kernel<<<1, 1024, 0, o->st>>>(x, y, n, o->small + 1);
  if (cudaGetLastError() != cudaSuccess) {
    *st = plan_fail(o->plan, HOTRG_ECUDA, "dot kernel launch failed");
    return 0;
  }
  return 0.5 * host_scalar(o, o->small + 1, st);
}

// w = first D' columns of Q exp(B), written as D' rows of N into the plan's
// isometry of step k.
hotrg_status set_w(hotrg_lbfgs_s* o, int k, const double* Bm, int N, int Dp) {
  const long long t = (long long)N * N;
  LCK(cudaMemcpyAsync(o->X2, Bm, sizeof(double) * t, cudaMemcpyDeviceToDevice, o->st));
  double* ex = nullptr;
  hotrg_status r = expm(o, o->X2, o->E1, o->E2, N, &ex);
  if (r != HOTRG_OK) return r;
  // w[a][i] = sum_j exp(B)[j][a] Q[i][j]   (Q column-major: Q[i][j] at j N + i)
  LCK(gemm_f64(gm(o, ex, map_lin(1), map_lin(N), t, o->Q, map_lin(1), map_lin(N), t,
                  plan_isometry(o->plan, k), map_lin(N), map_lin(1), (long long)Dp * N, Dp, N, N,
                  1.0, 0.0),
               o->st, o->sms));
  return HOTRG_OK;
}

// f = ln Z / N of the network with the current isometries (forward on the
// plan's stored site tensor).
hotrg_status eval_f(hotrg_lbfgs_s* o, double* f) {
  hotrg_status r = hotrg_forward_device(o->plan, plan_T0(o->plan), nullptr);
  if (r != HOTRG_OK) return r;
  r = hotrg_sync(o->plan);
  if (r != HOTRG_OK) return r;
  *f = host_scalar(o, plan_lnz(o->plan), &r);
  return r;
}

// Gradient (full antisymmetric N x N) at the variables Bm, after eval_f there.
hotrg_status eval_g(hotrg_lbfgs_s* o, int k, const double* Bm, int N, int Dp, double* Gout) {
  hotrg_status r = hotrg_backward_device(o->plan, nullptr);
  if (r != HOTRG_OK) return r;
  const long long t = (long long)N * N, n2 = 2LL * N, t2 = n2 * n2;
  count_launch();
  block_kernel<<<nblocks(t2, o->sms), 256, 0, o->st>>>(Bm, N, o->X2);
  LCK(cudaGetLastError());
  // C = Q^T wbar E^T into the upper-right block (columns N .. N + D'), scaled
  // by 1/c (c = its largest entry) so that the exponential's scaling depends
  // on B alone; the Frechet derivative is linear in C.
  const double* wb = plan_wbar(o->plan, k);
  count_launch();
  dot_kernel<<<1, 1024, 0, o->st>>>(wb, wb, (long long)Dp * N, o->small + 2);
  LCK(cudaGetLastError());
  const double c2 = host_scalar(o, o->small + 2, &r);
  if (r != HOTRG_OK) return r;
  const double c = c2 > 0 ? std::sqrt(c2) : 1.0;
  // C[r][a] = sum_i Q[i][r] wbar[a][i]
  LCK(gemm_f64(gm(o, o->Q, map_lin(N), map_lin(1), t, wb, map_lin(N), map_lin(1),
                  (long long)Dp * N, o->X2 + N, map_lin(n2), map_lin(1), t2 - N, N, Dp, N, 1.0 / c,
                  0.0),
               o->st, o->sms));
  double* ex = nullptr;
  r = expm(o, o->X2, o->E1, o->E2, 2 * N, &ex);
  if (r != HOTRG_OK) return r;
  count_launch();
  antisym_block_kernel<<<nblocks(t, o->sms), 256, 0, o->st>>>(ex, N, c, Gout);
  LCK(cudaGetLastError());
  return HOTRG_OK;
}

// Base point of layer k: complete Householder QR of the current isometry.
hotrg_status base_point(hotrg_lbfgs_s* o, int k, int N, int Dp) {
  // the isometry's D' rows of N are the columns of a column-major N x D' matrix
  LCK(cudaMemcpyAsync(o->Q, plan_isometry(o->plan, k), sizeof(double) * (size_t)Dp * N,
                      cudaMemcpyDeviceToDevice, o->st));
  if (cusolverDnDgeqrf(o->solver, N, Dp, o->Q, N, o->tau, o->work, o->lwork, o->info) !=
      CUSOLVER_STATUS_SUCCESS)
    return plan_fail(o->plan, HOTRG_ECUDA, "cusolverDnDgeqrf failed");
  count_launch();
  diag_sign_kernel<<<1, 256, 0, o->st>>>(o->Q, N, Dp, o->small + 8);
  LCK(cudaGetLastError());
  if (cusolverDnDorgqr(o->solver, N, N, Dp, o->Q, N, o->tau, o->work, o->lwork, o->info) !=
      CUSOLVER_STATUS_SUCCESS)
    return plan_fail(o->plan, HOTRG_ECUDA, "cusolverDnDorgqr failed");
  count_launch();
  scale_cols_kernel<<<nblocks((long long)N * Dp, o->sms), 256, 0, o->st>>>(o->Q, N, Dp,
                                                                            o->small + 8);
  LCK(cudaGetLastError());
  return HOTRG_OK;
}

hotrg_status run_layer(hotrg_lbfgs_s* o, int k, int n_iter, double step0, double c1,
                       int max_bt, double* f_hist, int* n_acc, int* n_evals) {
  int X = 0, Y = 0, Dp = 0;
  hotrg_status r = hotrg_step_dims(o->plan, k, &X, &Y, &Dp);
  if (r != HOTRG_OK) return r;
  const int N = X * X;
  const long long t = (long long)N * N;
  if (N > o->Nmax || Dp > o->Dmax) return HOTRG_EINVAL;
  if (k > plan_steps_run(o->plan) || k > plan_given_steps(o->plan))
    return plan_fail(o->plan, HOTRG_ESTATE,
                     "L-BFGS layer must be run by the plan with its isometry given");
  r = base_point(o, k, N, Dp);
  if (r != HOTRG_OK) return r;
  LCK(cudaMemsetAsync(o->B, 0, sizeof(double) * t, o->st));
  double f = 0;
  if ((r = set_w(o, k, o->B, N, Dp)) != HOTRG_OK) return r;
  if ((r = eval_f(o, &f)) != HOTRG_OK) return r;
  if ((r = eval_g(o, k, o->B, N, Dp, o->G)) != HOTRG_OK) return r;
  LCK(cudaMemcpyAsync(o->Wacc, plan_isometry(o->plan, k), sizeof(double) * (size_t)Dp * N,
                      cudaMemcpyDeviceToDevice, o->st));
  int evals = 1, acc = 0;
  if (f_hist) f_hist[0] = f;
  int npairs = 0, head = 0;          // ring of stored pairs, oldest at (head - npairs)
  std::vector<double> rho(o->m);
  for (int it = 0; it < n_iter; ++it) {
    const double gg = half_dot(o, o->G, o->G, t, &r);
    if (r != HOTRG_OK) return r;
    if (!(gg > 0)) break;
    const double gn = std::sqrt(gg);
    double slope = 0;
    auto steepest = [&]() -> hotrg_status {
      LCK(scale_copy(o->G, o->P, t, step0 / gn, o->st, o->sms));
      slope = step0 * gn;
      return HOTRG_OK;
    };
    if (npairs == 0) {
      if ((r = steepest()) != HOTRG_OK) return r;
    } else {
      // two-loop recursion: P = H G
      LCK(cudaMemcpyAsync(o->P, o->G, sizeof(double) * t, cudaMemcpyDeviceToDevice, o->st));
      std::vector<double> alpha(npairs);
      for (int i = npairs - 1; i >= 0; --i) {
        const int slot = (head - npairs + i + o->m) % o->m;
        const double a = rho[slot] * half_dot(o, o->S[slot], o->P, t, &r);
        if (r != HOTRG_OK) return r;
        alpha[i] = a;
        count_launch();
        axpy_kernel<<<nblocks(t, o->sms), 256, 0, o->st>>>(o->Y[slot], o->P, t, -a);
        LCK(cudaGetLastError());
      }
      const int newest = (head - 1 + o->m) % o->m;
      const double sy = half_dot(o, o->S[newest], o->Y[newest], t, &r);
      if (r != HOTRG_OK) return r;
      const double yy = half_dot(o, o->Y[newest], o->Y[newest], t, &r);
      if (r != HOTRG_OK) return r;
      LCK(scale_copy(o->P, o->P, t, sy / yy, o->st, o->sms));
      for (int i = 0; i < npairs; ++i) {
        const int slot = (head - npairs + i + o->m) % o->m;
        const double b = rho[slot] * half_dot(o, o->Y[slot], o->P, t, &r);
        if (r != HOTRG_OK) return r;
        count_launch();
        axpy_kernel<<<nblocks(t, o->sms), 256, 0, o->st>>>(o->S[slot], o->P, t, alpha[i] - b);
        LCK(cudaGetLastError());
      }
      slope = half_dot(o, o->G, o->P, t, &r);
      if (r != HOTRG_OK) return r;
      if (!(slope > 0)) {            // not an ascent direction: drop the history
        npairs = 0;
        if ((r = steepest()) != HOTRG_OK) return r;
      }
    }
    // backtracking from the full step
    double a = 1.0, fn = 0;
    bool ok = false;
    for (int bt = 0; bt <= max_bt; ++bt) {
      count_launch();
      axpby_kernel<<<nblocks(t, o->sms), 256, 0, o->st>>>(o->B, o->P, o->Bn, t, 1.0, a);
      LCK(cudaGetLastError());
      if ((r = set_w(o, k, o->Bn, N, Dp)) != HOTRG_OK) return r;
      if ((r = eval_f(o, &fn)) != HOTRG_OK) return r;
      ++evals;
      if (fn >= f + c1 * a * slope) {
        ok = true;
        break;
      }
      a *= 0.5;
    }
    if (!ok) break;
    if ((r = eval_g(o, k, o->Bn, N, Dp, o->Gn)) != HOTRG_OK) return r;
    // pair: s = Bn - B, y = G - Gn (gradient change of -f), formed in the
    // spare slot m and stored (in place of the oldest pair) only if s^T y > 0
    double* s = o->S[o->m];
    double* y = o->Y[o->m];
    count_launch();
    axpby_kernel<<<nblocks(t, o->sms), 256, 0, o->st>>>(o->Bn, o->B, s, t, 1.0, -1.0);
    LCK(cudaGetLastError());
    count_launch();
    axpby_kernel<<<nblocks(t, o->sms), 256, 0, o->st>>>(o->G, o->Gn, y, t, 1.0, -1.0);
    LCK(cudaGetLastError());
    const double sy = half_dot(o, s, y, t, &r);
    if (r != HOTRG_OK) return r;
    if (sy > 0) {
      std::swap(o->S[head], o->S[o->m]);
      std::swap(o->Y[head], o->Y[o->m]);
      rho[head] = 1.0 / sy;
      head = (head + 1) % o->m;
      npairs = std::min(npairs + 1, o->m);
    }
    std::swap(o->B, o->Bn);
    std::swap(o->G, o->Gn);
    f = fn;
    ++acc;
    if (f_hist) f_hist[acc] = f;
    LCK(cudaMemcpyAsync(o->Wacc, plan_isometry(o->plan, k), sizeof(double) * (size_t)Dp * N,
                        cudaMemcpyDeviceToDevice, o->st));
  }
  // leave the accepted isometry in the plan (a rejected trial may be there)
  LCK(cudaMemcpyAsync(plan_isometry(o->plan, k), o->Wacc, sizeof(double) * (size_t)Dp * N,
                      cudaMemcpyDeviceToDevice, o->st));
  LCK(cudaStreamSynchronize(o->st));
  if (n_acc) *n_acc = acc;
  if (n_evals) *n_evals = evals;
  return HOTRG_OK;
}

}  // namespace

extern "C" {

hotrg_status hotrg_lbfgs_create(hotrg_plan plan, int history, hotrg_lbfgs* out) {
  if (!plan || !out || history < 1 || history > 64) return HOTRG_EINVAL;
  *out = nullptr;
  int n_steps = 0;
  {
    int X, Y, Xp;
    while (hotrg_step_dims(plan, n_steps + 1, &X, &Y, &Xp) == HOTRG_OK) ++n_steps;
  }
  if (n_steps == 0 || !plan_wbar(plan, 1) || !plan_w_given(plan))
    return plan_fail(plan, HOTRG_ESTATE, "L-BFGS needs a w_given plan with fixed-w gradients");
  if (!plan_has_forward(plan))
    return plan_fail(plan, HOTRG_ESTATE, "L-BFGS needs a forward first (it keeps that T0)");
  hotrg_lbfgs o = new hotrg_lbfgs_s();
  o->plan = plan;
  o->m = history;
  o->st = plan_stream(plan);
  o->sms = plan_sms(plan);
  for (int k = 1; k <= n_steps; ++k) {
    int X, Y, Xp;
    hotrg_step_dims(plan, k, &X, &Y, &Xp);
    o->Nmax = std::max(o->Nmax, X * X);
    o->Dmax = std::max(o->Dmax, Xp);
  }
  auto cleanup = [&](hotrg_status s) {
    hotrg_lbfgs_destroy(o);
    return s;
  };
  const long long t = (long long)o->Nmax * o->Nmax, t2 = 4 * t;
  auto al = [&](double** p, long long n) -> bool {
    void* v = nullptr;
    if (cudaMalloc(&v, sizeof(double) * (size_t)n) != cudaSuccess) return false;
    o->allocs.push_back(v);
    *p = static_cast<double*>(v);
    return true;
  };
  bool ok = al(&o->Q, t) && al(&o->B, t) && al(&o->Bn, t) && al(&o->G, t) && al(&o->Gn, t) &&
            al(&o->P, t) && al(&o->X2, t2) && al(&o->E1, t2) && al(&o->E2, t2) &&
            al(&o->Wacc, (long long)o->Dmax * o->Nmax) && al(&o->small, 16 + o->Dmax) &&
            al(&o->tau, o->Nmax);
  o->S.assign(o->m + 1, nullptr);   // m stored pairs and one spare
  o->Y.assign(o->m + 1, nullptr);
  for (int i = 0; ok && i <= o->m; ++i) ok = al(&o->S[i], t) && al(&o->Y[i], t);
  if (!ok) return cleanup(HOTRG_ENOMEM);
  void* iv = nullptr;
  if (cudaMalloc(&iv, sizeof(int)) != cudaSuccess) return cleanup(HOTRG_ENOMEM);
  o->allocs.push_back(iv);
  o->info = static_cast<int*>(iv);
  if (cusolverDnCreate(&o->solver) != CUSOLVER_STATUS_SUCCESS ||
      cusolverDnSetStream(o->solver, o->st) != CUSOLVER_STATUS_SUCCESS)
    return cleanup(HOTRG_ECUDA);
  int l1 = 0, l2 = 0;
  if (cusolverDnDgeqrf_bufferSize(o->solver, o->Nmax, o->Dmax, o->Q, o->Nmax, &l1) !=
          CUSOLVER_STATUS_SUCCESS ||
      cusolverDnDorgqr_bufferSize(o->solver, o->Nmax, o->Nmax, o->Dmax, o->Q, o->Nmax, o->tau,
                                  &l2) != CUSOLVER_STATUS_SUCCESS)
    return cleanup(HOTRG_ECUDA);
  o->lwork = std::max(l1, l2);
  if (!al(&o->work, o->lwork)) return cleanup(HOTRG_ENOMEM);
  *out = o;
  return HOTRG_OK;
}

hotrg_status hotrg_lbfgs_layer(hotrg_lbfgs opt, int step, int n_iter, double step0, double c1,
                               int max_backtracks, double* f_hist, int* n_accepted,
                               int* n_evals) {
  if (!opt || n_iter < 0 || !(step0 > 0) || !(c1 > 0 && c1 < 1) || max_backtracks < 0)
    return HOTRG_EINVAL;
  int X, Y, Xp;
  if (hotrg_step_dims(opt->plan, step, &X, &Y, &Xp) != HOTRG_OK) return HOTRG_EINVAL;
  return run_layer(opt, step, n_iter, step0, c1, max_backtracks, f_hist, n_accepted, n_evals);
}

void hotrg_lbfgs_destroy(hotrg_lbfgs opt) {
  if (!opt) return;
  if (opt->st) cudaStreamSynchronize(opt->st);
  if (opt->solver) cusolverDnDestroy(opt->solver);
  for (void* v : opt->allocs) cudaFree(v);
  delete opt;
}

}  // extern "C"
