// Memory-bound helper kernels of the HOTRG path: operand preparation
// (gather + bf16 split), the Ising site tensor, FP64 norms and traces, the
// eigenvector post-processing and the element-wise parts of the backward.
#include <math.h>
#include "kernels.h"

namespace hotrg {

namespace {

__device__ __forceinline__ long long gtid() {
  return blockIdx.x * (long long)blockDim.x + threadIdx.x;
}
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

int blocks_for(long long n, int num_sms) {
  long long b = (n + 255) / 256;
  long long cap = 16LL * num_sms;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// dst plane p, element (r, k) at dst + p * plane_stride + r * K + k.
__global__ void gather_split_kernel(const double* __restrict__ src, long long src_lim, IMap rm,
                                    IMap km, int rows, int K, int nplanes,
                                    long long plane_stride, __nv_bfloat16* __restrict__ dst,
                                    int* err) {
  const long long total = (long long)rows * K;
  for (long long i = gtid(); i < total; i += gstride()) {
    int r = (int)(i / K), k = (int)(i - (long long)r * K);
    const long long off = imap(rm, r) + imap(km, k);
    double v = 0.0;
    if (off >= 0 && off < src_lim) v = src[off];
    else report_error(err, kErrBounds);
    __nv_bfloat16 b[3];
    split_bf16_d(v, nplanes, b);
    dst[i] = b[0];
    if (nplanes > 1) dst[plane_stride + i] = b[1];
    if (nplanes > 2) dst[2 * plane_stride + i] = b[2];
  }
}

// Grid-aligned split for the tensor-core GEMM.  One warp per (row, K segment
// of `seg` <= 128 elements), kSplitSegs segments per warp iteration with all
// their loads issued before any is used (memory-level parallelism: the kernel
// streams the D^5 intermediates and is bound by HBM).  With three or four
// planes, plane 0 is the value rounded to the grid g = 2^(e-8),
// 2^(e-1) <= max|segment| < 2^e, so |plane0 / g| <= 256 is an integer that
// bf16 holds exactly; the further planes are the bf16 round-to-nearest of the
// remainders.  With every operand split this way, the products of the two
// plane-0 values of a segment are integers on the grid g_a g_b below 2^16, and
// their sum over a segment of 128 stays below 2^23: the FP32 tensor-core
// accumulation of those products is exact.  With two planes, plane 0 is the
// plain round-to-nearest bf16 of the value (a grid would cost the remainder
// plane bits on small elements).
constexpr int kSplitSegs = 4;

template <typename SrcT>
__device__ __forceinline__ void split_load4(const SrcT* __restrict__ src, long long src_lim,
                                            long long roff, const IMap& km, int k0, int contig,
                                            SrcT* vd, int* err) {
  const long long off0 = roff + imap(km, k0);
  if (contig && off0 >= 0 && off0 + 3 < src_lim && (off0 & (sizeof(SrcT) == 4 ? 3 : 1)) == 0) {
    if constexpr (sizeof(SrcT) == 4) {
      const float4 q = __ldcs(reinterpret_cast<const float4*>(src + off0));
      vd[0] = q.x; vd[1] = q.y; vd[2] = q.z; vd[3] = q.w;
    } else {
      const double2 a = *reinterpret_cast<const double2*>(src + off0);
      const double2 b = *reinterpret_cast<const double2*>(src + off0 + 2);
      vd[0] = a.x; vd[1] = a.y; vd[2] = b.x; vd[3] = b.y;
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long off = roff + imap(km, k0 + i);
    vd[i] = SrcT(0);
    if (off >= 0 && off < src_lim) vd[i] = src[off];
    else report_error(err, kErrBounds);
  }
}

// The split of one segment: lane holds its 4 consecutive elements vd (zeros
// when inactive); all 32 lanes take part in the segment-maximum reduction.
template <typename SrcT>
__device__ __forceinline__ void split_emit(const SrcT (&vd)[4], bool active, int nplanes,
                                           int gridded, long long plane_stride,
                                           __nv_bfloat16* __restrict__ dst, long long obase) {
  float v[4];
  float mx = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[i] = (float)vd[i];
    mx = fmaxf(mx, fabsf(v[i]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  // grid 2^(e-8) with 2^(e-1) <= max < 2^e, kept a normal float (tiny segments
  // get a coarser grid, which keeps the plane-0 integers even smaller)
  int e = 0;
  frexpf(mx, &e);
  const int ge = max(e - 8, -126);
  const float g = (mx > 0.f) ? ldexpf(1.f, ge) : 1.f;
  const float gi = (mx > 0.f) ? ldexpf(1.f, -ge) : 1.f;   // v / g == v * gi exactly
  if (!active) return;
  __nv_bfloat16 b[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __nv_bfloat16 b0;
    if (gridded) b0 = __float2bfloat16_rn(rintf(v[i] * gi) * g);
    else b0 = __double2bfloat16((double)vd[i]);
    b[0][i] = b0;
    if constexpr (sizeof(SrcT) == 4) {
      // float source: the remainders are exact in float
      const float rem = v[i] - __bfloat162float(b0);
      b[1][i] = __float2bfloat16_rn(rem);
      const float rem2 = rem - __bfloat162float(b[1][i]);
      b[2][i] = __float2bfloat16_rn(rem2);
      b[3][i] = __float2bfloat16_rn(rem2 - __bfloat162float(b[2][i]));
    } else {
      // double source: the first remainder as a float pair keeps the bits a
      // float would drop (enough for four planes), the rest in float
      const double remd = (double)vd[i] - (double)__bfloat162float(b0);
      const float rh = (float)remd;
      const float rl = (float)(remd - (double)rh);
      b[1][i] = __float2bfloat16_rn(rh);
      const float rem2 = (rh - __bfloat162float(b[1][i])) + rl;
      b[2][i] = __float2bfloat16_rn(rem2);
      b[3][i] = __float2bfloat16_rn(rem2 - __bfloat162float(b[2][i]));
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q >= nplanes) break;
    *reinterpret_cast<uint2*>(dst + q * plane_stride + obase) =
        *reinterpret_cast<const uint2*>(b[q]);
  }
}

template <typename SrcT>
__global__ void __launch_bounds__(256, sizeof(SrcT) == 4 ? 4 : 3)
    grid_split_kernel(const SrcT* __restrict__ src, long long src_lim, IMap rm,
                                  IMap km, int rows, int K, int seg, int nplanes, int gridded,
                                  int contig, long long plane_stride,
                                  __nv_bfloat16* __restrict__ dst, int* err) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int nseg = (K + seg - 1) / seg;
  const long long work = (long long)rows * nseg;
  for (long long w0 = warp0 * kSplitSegs; w0 < work; w0 += nwarps * kSplitSegs) {
    // lane handles the 4 consecutive elements k0 .. k0 + 3 of each segment
    SrcT vd[kSplitSegs][4];   // the source precision: float sources stay float
    long long obase[kSplitSegs];
    bool active[kSplitSegs];
#pragma unroll
    for (int s = 0; s < kSplitSegs; ++s) {
      const long long w = w0 + s;
      const int r = (int)(w / nseg), sg = (int)(w % nseg);
      const int k0 = sg * seg + 4 * lane;
      active[s] = w < work && 4 * lane < seg && k0 < K;   // K is a multiple of 8
      obase[s] = (long long)r * K + k0;                   // multiple of 4: 8-byte aligned
      if (active[s]) {
        split_load4(src, src_lim, imap(rm, r), km, k0, contig, vd[s], err);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) vd[s][i] = SrcT(0);
      }
    }
#pragma unroll
    for (int s = 0; s < kSplitSegs; ++s)
      split_emit(vd[s], active[s], nplanes, gridded, plane_stride, dst, obase[s]);
  }
}

// The same split for sources whose rows, not K, are contiguous (the first
// radix level of the row map has stride 1 and covers whole groups of 32 rows):
// a block stages 32 rows x one K segment in shared memory, read with
// consecutive lanes on consecutive rows (coalesced), then splits each row's
// segment exactly as grid_split_kernel does (same split_emit).
constexpr int kRowsTile = 32;
constexpr int kRowsPitch = kGridSeg + 2;   // elements per staged row (segments <= kGridSeg)

// rstep = 1: the tile is 32 consecutive rows; rstep > 1: the unit stride is on
// the second level (row = i + rstep q), and the tile is 32 consecutive q for
// one i.
template <typename SrcT>
__global__ void __launch_bounds__(256)
    grid_split_rows_kernel(const SrcT* __restrict__ src, long long src_lim, IMap rm, IMap km,
                           int rows, int K, int seg, int nplanes, int gridded, int rstep,
                           long long plane_stride, __nv_bfloat16* __restrict__ dst, int* err) {
  __shared__ __align__(16) SrcT tile[kRowsTile][kRowsPitch];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nseg = (K + seg - 1) / seg;
  const long long work = (long long)(rows / kRowsTile) * nseg;
  for (long long w = blockIdx.x; w < work; w += gridDim.x) {
    const int rb = (int)(w / nseg), sg = (int)(w % nseg);
    // first row of the tile and the row of lane l = rfirst + l * rstep
    const int rfirst = (rstep == 1) ? rb * kRowsTile
                                    : (rb % rstep) + rstep * (rb / rstep) * kRowsTile;
    const int k0 = sg * seg;
    const int kn = min(seg, K - k0);
    const long long roff = imap(rm, rfirst + lane * rstep);
    for (int kk = warp; kk < kn; kk += 8) {
      const long long off = roff + imap(km, k0 + kk);
      SrcT v = SrcT(0);
      if (off >= 0 && off < src_lim) v = src[off];
      else report_error(err, kErrBounds);
      tile[lane][kk] = v;
    }
    __syncthreads();
    for (int i = warp; i < kRowsTile; i += 8) {
      const bool active = 4 * lane < kn;
      SrcT vd[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) vd[j] = active ? tile[i][4 * lane + j] : SrcT(0);
      split_emit(vd, active, nplanes, gridded, plane_stride, dst,
                 (long long)(rfirst + i * rstep) * K + k0 + 4 * lane);
    }
    __syncthreads();
  }
}

// T0 and dT0/dbeta of the Ising model (one tensor per spin).
__global__ void ising_t0_kernel(double beta, double J, double h, double* T0, double* dT0) {
  int idx = threadIdx.x;   // 16 threads: (l, r, u, d) bits
  if (idx >= 16) return;
  const double k = beta * J;
  const double ch = cosh(k), sh = sinh(k);
  const double a = sqrt(ch), b = sqrt(sh);
  const double da = J * sh / (2.0 * a);
  const double db = (b > 0.0) ? J * ch / (2.0 * b) : 0.0;
  int leg[4] = {(idx >> 3) & 1, (idx >> 2) & 1, (idx >> 1) & 1, idx & 1};
  double t = 0.0, dt = 0.0;
  for (int si = 0; si < 2; ++si) {
    const double s = si == 0 ? 1.0 : -1.0;
    const double e = exp(beta * h * s), de = h * s * e;
    double W[4], dW[4];
    for (int q = 0; q < 4; ++q) {
      W[q] = leg[q] == 0 ? a : s * b;
      dW[q] = leg[q] == 0 ? da : s * db;
    }
    const double prod = W[0] * W[1] * W[2] * W[3];
    t += e * prod;
    double dprod = dW[0] * W[1] * W[2] * W[3] + W[0] * dW[1] * W[2] * W[3] +
                   W[0] * W[1] * dW[2] * W[3] + W[0] * W[1] * W[2] * dW[3];
    dt += de * prod + e * dprod;
  }
  T0[idx] = t;
  if (dT0) dT0[idx] = dt;
}

// Deterministic FP64 sum of squares: per-block partials, then one block.
__global__ void sumsq_partial_kernel(const double* __restrict__ x, long long n,
                                     double* __restrict__ partial) {
  double s = 0.0;
  for (long long i = gtid(); i < n; i += gstride()) s = fma(x[i], x[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

// c = sqrt(sum partials); log_norm = ln c; inv = 1/c stored in scal[0].
__global__ void norm_finalize_kernel(const double* __restrict__ partial, int np,
                                     double* __restrict__ log_norm, double* __restrict__ inv,
                                     int* err) {
  __shared__ double ws[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) {
      double c = sqrt(s);
      if (!(c > 0.0) || !isfinite(c)) {
        report_error(err, kErrNonFinite);
        c = 1.0;
      }
      *log_norm = log(c);
      *inv = 1.0 / c;
    }
  }
}

__global__ void scale_kernel(double* __restrict__ x, long long n, const double* __restrict__ s) {
  const double f = *s;
  for (long long i = gtid(); i < n; i += gstride()) x[i] *= f;
}

// out = [lnz, sign, log_norms...]; T stored as [a][a][b][b]-traceable tensor
// with leg dims (P, P, Q, Q).
__global__ void trace_lnz_kernel(const double* __restrict__ T, int P, int Q,
                                 const double* __restrict__ log_norms, int n,
                                 double* __restrict__ out, double* __restrict__ trace_out,
                                 int* err) {
  __shared__ double ws[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < P * Q; i += blockDim.x) {
    int a = i / Q, b = i % Q;
    s += T[((long long)(a * P + a) * Q + b) * Q + b];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tr += ws[w];
    double acc = 0.0, scale = 1.0;
    for (int k = 0; k < n; ++k) {
      scale *= 0.5;
      acc += log_norms[k] * scale;
    }
    if (!(fabs(tr) > 0.0) || !isfinite(tr)) report_error(err, kErrNonFinite);
    out[0] = acc + log(fabs(tr)) * scale;
    out[1] = tr >= 0.0 ? 1.0 : -1.0;
    for (int k = 0; k < n; ++k) out[2 + k] = log_norms[k];
    *trace_out = tr;
  }
}

// Eigen post-processing.  cuSOLVER returns `ncols` eigenvalues ascending (the
// largest ones) and their eigenvectors as the columns of a column-major
// matrix, i.e. eigenvector a is the contiguous row a of `asc`.  Write them
// descending: row alpha of `desc` is eigenvector ncols-1-alpha, flipped so
// that its largest-magnitude component (lowest index on ties) is positive.
// One block per eigenvector.
__global__ void eig_desc_kernel(const double* __restrict__ asc, const double* __restrict__ w_asc,
                                int N, int ncols, int rows_out, double* __restrict__ desc,
                                double* __restrict__ lam_desc) {
  const int alpha = blockIdx.x;
  if (alpha >= rows_out) return;
  const double* src = asc + (long long)(ncols - 1 - alpha) * N;
  double best = -1.0;
  int bi = 0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double v = fabs(src[i]);
    if (v > best) { best = v; bi = i; }
  }
  __shared__ double sb[256];
  __shared__ int si[256];
  sb[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double b2 = sb[threadIdx.x + o];
      int i2 = si[threadIdx.x + o];
      if (b2 > sb[threadIdx.x] || (b2 == sb[threadIdx.x] && i2 < si[threadIdx.x])) {
        sb[threadIdx.x] = b2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  const double sgn = src[si[0]] < 0.0 ? -1.0 : 1.0;
  double* dst = desc + (long long)alpha * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) dst[i] = sgn * src[i];
  if (alpha == 0)
    for (int i = threadIdx.x; i < ncols; i += blockDim.x) lam_desc[i] = w_asc[ncols - 1 - i];
}

// Trace of an N x N matrix (before the eigensolver overwrites it).
__global__ void diag_trace_kernel(const double* __restrict__ G, int N, double* out) {
  __shared__ double s[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) a += G[(long long)i * N + i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// trunc_err = sum of discarded eigenvalues / sum of all (= trace(G));
// gap = (lam[Dp-1] - lam[Dp]) / lam[0].  `nlam` eigenvalues (descending) are
// known; the discarded sum is trace - sum of the kept ones.
__global__ void eig_diag_kernel(const double* __restrict__ lam, int nlam, int N, int Dp,
                                const double* __restrict__ trace, double* trunc, double* gap) {
  __shared__ double s_all[256], s_cut[256];
  double a = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < Dp; i += blockDim.x) a += lam[i];
  s_all[threadIdx.x] = a;
  s_cut[threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_all[threadIdx.x] += s_all[threadIdx.x + o];
      s_cut[threadIdx.x] += s_cut[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double tot = *trace;
    *trunc = tot != 0.0 ? (tot - s_all[0]) / tot : 0.0;
    *gap = (Dp < N && Dp < nlam && lam[0] != 0.0) ? (lam[Dp - 1] - lam[Dp]) / lam[0] : 0.0;
  }
}

// Residual check of the kept Ritz pairs of the subspace eigensolver.
// Rows a < Dp of V hold the sign-fixed Ritz vectors (descending Ritz values
// lam), rows of Z = V G the products with the Gram matrix; the first kernel
// writes r_a = ||Z_a - lam_a V_a||_2 for each row (one block per row, fixed
// reduction order), the second max_a r_a / lam_0 to *res and raises *guard to
// `code` when that exceeds tol (or is not a number).
__global__ void eig_residual_rows_kernel(const double* __restrict__ Z,
                                         const double* __restrict__ V,
                                         const double* __restrict__ lam, int N,
                                         double* __restrict__ r) {
  const int a = blockIdx.x;
  const double la = lam[a];
  const double* z = Z + (long long)a * N;
  const double* v = V + (long long)a * N;
  double acc = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double d = z[i] - la * v[i];
    acc += d * d;
  }
  __shared__ double s[256];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) r[a] = sqrt(s[0]);
}

__global__ void eig_residual_max_kernel(const double* __restrict__ r, int Dp,
                                        const double* __restrict__ lam, double tol, double* res,
                                        int* guard, int code) {
  if (threadIdx.x != 0) return;
  double worst = 0.0;
  for (int a = 0; a < Dp; ++a) worst = fmax(worst, r[a]);
  const double l0 = lam[0];
  const double q = l0 > 0.0 ? worst / l0 : (worst > 0.0 ? INFINITY : 0.0);
  *res = q;
  if (!(q <= tol)) atomicMax(guard, code);
}

__global__ void eigh_info_kernel(const int* info, int* err) {
  if (threadIdx.x == 0 && *info != 0) report_error(err, kErrEigh);
}

// Backward seed: E = delta(a,a') delta(b,b') / trace on a (P, P, Q, Q) tensor.
__global__ void seed_kernel(double* __restrict__ E, int P, int Q, const double* __restrict__ tr) {
  const long long n = (long long)P * P * Q * Q;
  const double inv = 1.0 / *tr;
  for (long long i = gtid(); i < n; i += gstride()) {
    int d = (int)(i % Q);
    int u = (int)((i / Q) % Q);
    int r = (int)((i / ((long long)Q * Q)) % P);
    int l = (int)(i / ((long long)Q * Q * P));
    E[i] = (l == r && u == d) ? inv : 0.0;
  }
}

// F o S for the eigensolve adjoint: S[j][k] (j discarded, k kept) times
// (lam_k - lam_j) / ((lam_k - lam_j)^2 + eta), eta = eta_rel * lam_0^2.
__global__ void eigh_adj_scale_kernel(double* __restrict__ S, int nd, int Dp,
                                      const double* __restrict__ lam, double eta_rel) {
  const double eta = eta_rel * lam[0] * lam[0];
  const long long n = (long long)nd * Dp;
  for (long long i = gtid(); i < n; i += gstride()) {
    int j = (int)(i / Dp), k = (int)(i % Dp);
    double d = lam[k] - lam[Dp + j];
    S[i] *= d / (d * d + eta);
  }
}

// G <- (G + G^T) / 2 in place (N x N).
__global__ void symmetrize_kernel(double* __restrict__ G, int N) {
  const long long n = (long long)N * N;
  for (long long i = gtid(); i < n; i += gstride()) {
    int r = (int)(i / N), c = (int)(i % N);
    if (c > r) {
      double a = G[i], b = G[(long long)c * N + r];
      double m = 0.5 * (a + b);
      G[i] = m;
      G[(long long)c * N + r] = m;
    }
  }
}

__global__ void scale_copy_kernel(const double* __restrict__ x, double* __restrict__ y, long long n,
                                  double a) {
  for (long long i = gtid(); i < n; i += gstride()) y[i] = a * x[i];
}

__global__ void scale_exp_neg_kernel(double* __restrict__ x, long long n,
                                     const double* __restrict__ logc) {
  const double f = exp(-*logc);
  for (long long i = gtid(); i < n; i += gstride()) x[i] *= f;
}

// Deterministic pseudo-random fill in [-1, 1) (SplitMix64 of the index).
__global__ void fill_random_kernel(double* __restrict__ x, long long n, unsigned long long seed) {
  for (long long i = gtid(); i < n; i += gstride()) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    x[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

__global__ void set_value_kernel(double* x, double v, int* err, int bits) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (x) *x = v;
    if (err && bits) report_error(err, bits);
  }
}

__global__ void dot16_kernel(const double* __restrict__ a, const double* __restrict__ b, int n,
                             double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = fma(a[i], b[i], s);
    *out = s;
  }
}


// out[c][d][a][b] = in[a][b][c][d], in of shape (P, P, Q, Q): the exchange of
// the leg pairs (l, r) <-> (u, d).
__global__ void swap_pairs_kernel(const double* __restrict__ in, double* __restrict__ out, int P,
                                  int Q) {
  const long long n = (long long)P * P * Q * Q, q2 = (long long)Q * Q;
  for (long long i = gtid(); i < n; i += gstride()) {
    const long long ab = i / q2, cd = i - ab * q2;
    out[cd * P * P + ab] = in[i];
  }
}

// Density-matrix MPO cell of the quantum XY chain, rho(tau) to second order in
// tau: T0[l][r][(s1 s2)][(v1 v2)] = sum g_odd[(s1 s2),(t1 t2)] R_l[t1,t1']
// L_r[t2,t2'] g_odd[(t1' t2'),(v1 v2)], with g_odd = exp(-tau/2 h) on the cell's
// own bond and exp(-tau h) = sum_k L_k (x) R_k on the bond to the next cell.
// h = J (SxSx + SySy) flips |01> <-> |10> with amplitude J/2 (state 0 = up), so
// exp(-t h) is the identity on |00>, |11> and [[ch, -sh], [-sh, ch]] on
// (|01>, |10>), ch = cosh(t J / 2), sh = sinh(t J / 2).  In Pauli form
// exp(-t h) = (1+ch)/2 1(x)1 + (1-ch)/2 Z(x)Z - sh/2 X(x)X + sh/2 (iY)(x)(iY),
// (iY = [[0, 1], [-1, 0]]), an operator SVD across the bond:
// L_k = sqrt|c_k| P_k, R_k = sign(c_k) sqrt|c_k| P_k.
__device__ double xy_gate(double t, double J, int s1, int s2, int t1, int t2) {
  const int a = 2 * s1 + s2, b = 2 * t1 + t2;
  if (a == 0 || a == 3) return a == b ? 1.0 : 0.0;
  if (b == 0 || b == 3) return 0.0;
  return a == b ? cosh(0.5 * t * J) : -sinh(0.5 * t * J);
}

__device__ double pauli(int k, int a, int b) {
  switch (k) {
    case 0: return a == b ? 1.0 : 0.0;                       // 1
    case 1: return a == b ? (a == 0 ? 1.0 : -1.0) : 0.0;     // Z
    case 2: return a != b ? 1.0 : 0.0;                       // X
    default: return a == b ? 0.0 : (a == 0 ? 1.0 : -1.0);    // iY
  }
}

__global__ void xy_mpo_kernel(double tau, double J, double* __restrict__ T0) {
  const int idx = threadIdx.x;   // (l, r, s1, s2, v1, v2): 4 * 4 * 16 entries
  if (idx >= 256) return;
  const int l = idx >> 6, r = (idx >> 4) & 3, s1 = (idx >> 3) & 1, s2 = (idx >> 2) & 1,
            v1 = (idx >> 1) & 1, v2 = idx & 1;
  const double ch = cosh(0.5 * tau * J), sh = sinh(0.5 * tau * J);
  const double c[4] = {0.5 * (1.0 + ch), 0.5 * (1.0 - ch), -0.5 * sh, 0.5 * sh};
  const double sl = (c[l] < 0 ? -1.0 : 1.0) * sqrt(fabs(c[l]));   // R_l
  const double sr = sqrt(fabs(c[r]));                             // L_r
  double acc = 0.0;
  for (int t1 = 0; t1 < 2; ++t1)
    for (int t2 = 0; t2 < 2; ++t2) {
      const double top = xy_gate(0.5 * tau, J, s1, s2, t1, t2);
      if (top == 0.0) continue;
      for (int u1 = 0; u1 < 2; ++u1)
        for (int u2 = 0; u2 < 2; ++u2) {
          const double mid = sl * pauli(l, t1, u1) * sr * pauli(r, t2, u2);
          if (mid == 0.0) continue;
          acc += top * mid * xy_gate(0.5 * tau, J, u1, u2, v1, v2);
        }
    }
  T0[idx] = acc;
}

// *out = ||a - b||_F (one block; power-iteration convergence test).
__global__ void diff_norm_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                 long long n, double* __restrict__ out) {
  __shared__ double ws[32];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = a[i] - b[i];
    s = fma(d, d, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    *out = sqrt(t);
  }
}

// v = sum_k log_norms[k] / 2^(k+1) + lnlam / 2^(n+1); out (if given) =
// [v, 1, log_norms...]; *step_out (if given) = v.
__global__ void chain_lnz_kernel(const double* __restrict__ log_norms, int n,
                                 const double* __restrict__ lnlam, double* __restrict__ out,
                                 double* __restrict__ step_out) {
  if (threadIdx.x != 0) return;
  double acc = 0.0, scale = 1.0;
  for (int k = 0; k < n; ++k) {
    scale *= 0.5;
    acc += log_norms[k] * scale;
  }
  const double v = acc + *lnlam * scale * 0.5;
  if (out) {
    out[0] = v;
    out[1] = 1.0;
    for (int k = 0; k < n; ++k) out[2 + k] = log_norms[k];
  }
  if (step_out) *step_out = v;
}

// Identity matrix (X x X) scaled to unit Frobenius norm.
__global__ void eye_unit_kernel(double* __restrict__ V, int X) {
  const long long n = (long long)X * X;
  const double v = 1.0 / sqrt((double)X);
  for (long long i = gtid(); i < n; i += gstride()) V[i] = (i / X == i % X) ? v : 0.0;
}


// w_rule 1: *side = 1 when the right side's relative truncation error is
// smaller than the left one's by more than tie (a relative tie band: both
// Gram matrices have the same trace).
__global__ void w_rule_choose_kernel(const double* __restrict__ trunc_l,
                                     const double* __restrict__ trunc_r, double tie,
                                     int* __restrict__ side) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *side = (*trunc_l - *trunc_r > tie) ? 1 : 0;
}

// dst = src where *flag != 0 (the chosen side's eigenpairs).
__global__ void cond_copy_kernel(const int* __restrict__ flag, const double* __restrict__ src,
                                 double* __restrict__ dst, long long n) {
  if (*flag == 0) return;
  for (long long i = gtid(); i < n; i += gstride()) dst[i] = src[i];
}

}  // namespace

cudaError_t gather_split(const double* src, long long src_lim, IMap rm, IMap km, int rows, int K,
                         int nplanes, long long plane_stride, __nv_bfloat16* dst, int* err,
                         cudaStream_t st, int sms) {
  long long n = (long long)rows * K;
  if (n == 0) return cudaSuccess;
  if (n > plane_stride) return cudaErrorInvalidValue;
  count_launch();
  gather_split_kernel<<<blocks_for(n, sms), 256, 0, st>>>(src, src_lim, rm, km, rows, K, nplanes,
                                                          plane_stride, dst, err);
  return cudaGetLastError();
}

template <typename SrcT>
cudaError_t grid_split_t(const SrcT* src, long long src_lim, IMap rm, IMap km, int rows, int K,
                         int nplanes, long long plane_stride, __nv_bfloat16* dst, int* err,
                         cudaStream_t st, int sms) {
  // Plane 0 on the grid only for three planes; with two planes a floating
  // plane 0 keeps more bits for small elements (see the comment above).
  const int gridded = nplanes >= 3 ? 1 : 0;
  if (nplanes < 1 || nplanes > 4 || K % 8 != 0 || plane_stride % 4 != 0)
    return cudaErrorInvalidValue;
  // unit stride on K's first radix level, in runs of a multiple of 4: every
  // lane's 4 elements are contiguous (vector loads)
  const int contig = (km.s0 == 1 && km.r0 % 4 == 0) ? 1 : 0;
  const int seg = K < kGridSeg ? K : kGridSeg;
  const long long work = (long long)rows * ((K + seg - 1) / seg);
  if (work == 0) return cudaSuccess;
  if ((long long)rows * K > plane_stride) return cudaErrorInvalidValue;
  // rows contiguous, K strided: stage 32-row tiles through shared memory.
  // Unit stride on the rows' first level (32 consecutive rows), or on the
  // second level of a two-level row map (rows i + r0 q, 32 consecutive q).
  int rstep = 0;
  if (rm.s0 == 1 && rm.r0 % kRowsTile == 0 && rows % kRowsTile == 0) rstep = 1;
  else if (rm.r1 == kBig && rm.s1 == 1 && rm.r0 > 1 && rows % rm.r0 == 0 &&
           (rows / rm.r0) % kRowsTile == 0)
    rstep = rm.r0;
  if (!contig && rstep > 0 && seg <= kGridSeg) {
    long long rblocks = (long long)(rows / kRowsTile) * ((K + seg - 1) / seg);
    if (rblocks > 8LL * sms) rblocks = 8LL * sms;
    count_launch();
    grid_split_rows_kernel<SrcT><<<(int)rblocks, 256, 0, st>>>(
        src, src_lim, rm, km, rows, K, seg, nplanes, gridded, rstep, plane_stride, dst, err);
    return cudaGetLastError();
  }
  long long blocks = (work + 8 * kSplitSegs - 1) / (8 * kSplitSegs);   // 8 warps per block
  if (blocks > 16LL * sms) blocks = 16LL * sms;
  count_launch();
  grid_split_kernel<SrcT><<<(int)blocks, 256, 0, st>>>(src, src_lim, rm, km, rows, K, seg, nplanes,
                                                        gridded, contig, plane_stride, dst, err);
  return cudaGetLastError();
}

cudaError_t grid_split(const double* src, long long src_lim, IMap rm, IMap km, int rows, int K,
                       int nplanes, long long plane_stride, __nv_bfloat16* dst, int* err,
                       cudaStream_t st, int sms) {
  return grid_split_t<double>(src, src_lim, rm, km, rows, K, nplanes, plane_stride, dst, err, st,
                              sms);
}

cudaError_t grid_split(const float* src, long long src_lim, IMap rm, IMap km, int rows, int K,
                       int nplanes, long long plane_stride, __nv_bfloat16* dst, int* err,
                       cudaStream_t st, int sms) {
  return grid_split_t<float>(src, src_lim, rm, km, rows, K, nplanes, plane_stride, dst, err, st,
                             sms);
}

cudaError_t ising_t0(double beta, double J, double h, double* T0, double* dT0, cudaStream_t st) {
  count_launch();
  ising_t0_kernel<<<1, 32, 0, st>>>(beta, J, h, T0, dT0);
  return cudaGetLastError();
}

cudaError_t frob_normalize(double* x, long long n, double* partial, int max_partial,
                           double* log_norm, double* inv_scratch, int* err, cudaStream_t st,
                           int sms) {
  int b = blocks_for(n, sms);
  if (b > max_partial) b = max_partial;
  count_launch();
  sumsq_partial_kernel<<<b, 256, 0, st>>>(x, n, partial);
  count_launch();
  norm_finalize_kernel<<<1, 256, 0, st>>>(partial, b, log_norm, inv_scratch, err);
  count_launch();
  scale_kernel<<<blocks_for(n, sms), 256, 0, st>>>(x, n, inv_scratch);
  return cudaGetLastError();
}

cudaError_t trace_lnz(const double* T, int P, int Q, const double* log_norms, int n, double* out,
                      double* trace_out, int* err, cudaStream_t st) {
  count_launch();
  trace_lnz_kernel<<<1, 256, 0, st>>>(T, P, Q, log_norms, n, out, trace_out, err);
  return cudaGetLastError();
}

cudaError_t eig_desc(const double* asc, const double* w_asc, int N, int ncols, int rows_out,
                     double* desc, double* lam_desc, cudaStream_t st) {
  count_launch();
  eig_desc_kernel<<<rows_out, 256, 0, st>>>(asc, w_asc, N, ncols, rows_out, desc, lam_desc);
  return cudaGetLastError();
}

cudaError_t diag_trace(const double* G, int N, double* out, cudaStream_t st) {
  count_launch();
  diag_trace_kernel<<<1, 256, 0, st>>>(G, N, out);
  return cudaGetLastError();
}

cudaError_t eig_diag(const double* lam, int nlam, int N, int Dp, const double* trace, double* trunc,
                     double* gap, cudaStream_t st) {
  count_launch();
  eig_diag_kernel<<<1, 256, 0, st>>>(lam, nlam, N, Dp, trace, trunc, gap);
  return cudaGetLastError();
}

cudaError_t eig_residual(const double* Z, const double* V, const double* lam, int Dp, int N,
                         double tol, double* row_scratch, double* res, int* guard, int code,
                         cudaStream_t st) {
  count_launch();
  eig_residual_rows_kernel<<<Dp, 256, 0, st>>>(Z, V, lam, N, row_scratch);
  count_launch();
  eig_residual_max_kernel<<<1, 32, 0, st>>>(row_scratch, Dp, lam, tol, res, guard, code);
  return cudaGetLastError();
}

cudaError_t eigh_info_check(const int* info, int* err, cudaStream_t st) {
  count_launch();
  eigh_info_kernel<<<1, 32, 0, st>>>(info, err);
  return cudaGetLastError();
}

cudaError_t seed_trace_adjoint(double* E, int P, int Q, const double* tr, cudaStream_t st,
                               int sms) {
  count_launch();
  seed_kernel<<<blocks_for((long long)P * P * Q * Q, sms), 256, 0, st>>>(E, P, Q, tr);
  return cudaGetLastError();
}

cudaError_t eigh_adj_scale(double* S, int nd, int Dp, const double* lam, double eta_rel,
                           cudaStream_t st, int sms) {
  count_launch();
  eigh_adj_scale_kernel<<<blocks_for((long long)nd * Dp, sms), 256, 0, st>>>(S, nd, Dp, lam,
                                                                           eta_rel);
  return cudaGetLastError();
}

cudaError_t symmetrize(double* G, int N, cudaStream_t st, int sms) {
  count_launch();
  symmetrize_kernel<<<blocks_for((long long)N * N, sms), 256, 0, st>>>(G, N);
  return cudaGetLastError();
}

cudaError_t scale_copy(const double* x, double* y, long long n, double a, cudaStream_t st,
                       int sms) {
  count_launch();
  scale_copy_kernel<<<blocks_for(n, sms), 256, 0, st>>>(x, y, n, a);
  return cudaGetLastError();
}

cudaError_t scale_exp_neg(double* x, long long n, const double* logc, cudaStream_t st, int sms) {
  count_launch();
  scale_exp_neg_kernel<<<blocks_for(n, sms), 256, 0, st>>>(x, n, logc);
  return cudaGetLastError();
}

cudaError_t fill_random(double* x, long long n, unsigned long long seed, cudaStream_t st, int sms) {
  count_launch();
  fill_random_kernel<<<blocks_for(n, sms), 256, 0, st>>>(x, n, seed);
  return cudaGetLastError();
}

cudaError_t set_value(double* x, double v, int* err, int bits, cudaStream_t st) {
  count_launch();
  set_value_kernel<<<1, 32, 0, st>>>(x, v, err, bits);
  return cudaGetLastError();
}

cudaError_t dot_small(const double* a, const double* b, int n, double* out, cudaStream_t st) {
  count_launch();
  dot16_kernel<<<1, 32, 0, st>>>(a, b, n, out);
  return cudaGetLastError();
}

cudaError_t swap_pairs(const double* in, double* out, int P, int Q, cudaStream_t st, int sms) {
  count_launch();
  swap_pairs_kernel<<<blocks_for((long long)P * P * Q * Q, sms), 256, 0, st>>>(in, out, P, Q);
  return cudaGetLastError();
}

cudaError_t xy_mpo(double tau, double J, double* T0, cudaStream_t st) {
  count_launch();
  xy_mpo_kernel<<<1, 256, 0, st>>>(tau, J, T0);
  return cudaGetLastError();
}

cudaError_t diff_norm(const double* a, const double* b, long long n, double* out,
                      cudaStream_t st) {
  count_launch();
  diff_norm_kernel<<<1, 1024, 0, st>>>(a, b, n, out);
  return cudaGetLastError();
}

cudaError_t chain_lnz(const double* log_norms, int n, const double* lnlam, double* out,
                      double* step_out, cudaStream_t st) {
  count_launch();
  chain_lnz_kernel<<<1, 32, 0, st>>>(log_norms, n, lnlam, out, step_out);
  return cudaGetLastError();
}

cudaError_t eye_unit(double* V, int X, cudaStream_t st, int sms) {
  count_launch();
  eye_unit_kernel<<<blocks_for((long long)X * X, sms), 256, 0, st>>>(V, X);
  return cudaGetLastError();
}

cudaError_t w_rule_choose(const double* trunc_l, const double* trunc_r, double tie, int* side,
                          cudaStream_t st) {
  count_launch();
  w_rule_choose_kernel<<<1, 32, 0, st>>>(trunc_l, trunc_r, tie, side);
  return cudaGetLastError();
}

cudaError_t cond_copy(const int* flag, const double* src, double* dst, long long n,
                      cudaStream_t st, int sms) {
  count_launch();
  cond_copy_kernel<<<blocks_for(n, sms), 256, 0, st>>>(flag, src, dst, n);
  return cudaGetLastError();
}

}  // namespace hotrg
