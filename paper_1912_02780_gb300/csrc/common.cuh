// Internal header shared by the CUDA translation units of the HOTRG library.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace hotrg {

// Mixed-radix index map used to address a tensor operand or output by a
// flattened GEMM index i (row m, column n or contraction index k):
//   off(i) = (i % r0) * s0 + ((i / r0) % r1) * s1 + (i / (r0 * r1)) * s2
// One-level maps set r0 = r1 = 1 << 30 (so only s0 matters); two-level maps
// set r1 = 1 << 30.  Every HOTRG contraction is a plain GEMM once its free and
// summed tensor legs are grouped this way.
struct IMap {
  int r0, r1;
  long long s0, s1, s2;
};

constexpr int kBig = 1 << 30;

inline IMap map_lin(long long s) { return IMap{kBig, kBig, s, 0, 0}; }
inline IMap map2(int r0, long long s0, long long s1) { return IMap{r0, kBig, s0, s1, 0}; }
inline IMap map3(int r0, int r1, long long s0, long long s1, long long s2) {
  return IMap{r0, r1, s0, s1, s2};
}

__host__ __device__ __forceinline__ long long imap(const IMap& m, int i) {
  int q0 = i / m.r0;
  int i0 = i - q0 * m.r0;
  int q1 = q0 / m.r1;
  int i1 = q0 - q1 * m.r1;
  return (long long)i0 * m.s0 + (long long)i1 * m.s1 + (long long)q1 * m.s2;
}

// Device error word bits (set by kernels, read by the host after a sync).
enum : int {
  kErrTimeout = 1,      // a bounded mbarrier wait gave up
  kErrNonFinite = 2,    // a norm or trace was zero / NaN / inf
  kErrEigh = 4,         // the eigensolver reported failure (info != 0)
  kErrBounds = 8        // an index check failed (access skipped)
};

// Report a device-side failure: err[0] accumulates every bit seen, err[1]
// keeps the first one (the root cause when one failure leads to others).
// Every error word handed to a kernel is an array of two ints.
__device__ __forceinline__ void report_error(int* err, int bit) {
  atomicOr(err, bit);
  atomicCAS(err + 1, 0, bit);
}

// Split a float into bf16 planes: v ~= p0 + p1 (+ p2), each plane the
// round-to-nearest bf16 of the remainder left by the planes before it.
__device__ __forceinline__ void split_bf16(float v, int nplanes, __nv_bfloat16* out) {
  __nv_bfloat16 h = __float2bfloat16_rn(v);
  out[0] = h;
  float r = v - __bfloat162float(h);
  if (nplanes > 1) {
    __nv_bfloat16 m = __float2bfloat16_rn(r);
    out[1] = m;
    if (nplanes > 2) out[2] = __float2bfloat16_rn(r - __bfloat162float(m));
  }
}

// Same, from a double (the first residual is formed in double, later ones in
// float, which is exact enough for three bf16 planes).
__device__ __forceinline__ void split_bf16_d(double v, int nplanes, __nv_bfloat16* out) {
  __nv_bfloat16 h = __double2bfloat16(v);
  out[0] = h;
  double r = v - (double)__bfloat162float(h);
  if (nplanes > 1) {
    __nv_bfloat16 m = __double2bfloat16(r);
    out[1] = m;
    if (nplanes > 2) out[2] = __double2bfloat16(r - (double)__bfloat162float(m));
  }
}

}  // namespace hotrg

namespace hotrg {
// Host-side count of this library's kernel launches (for the benchmark's
// launch accounting); defined in hotrg_api.cu.
void count_launch();
}  // namespace hotrg
