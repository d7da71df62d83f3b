// Allocation-free variant of the split-BF16 tensor-core GEMM check.
//
// hotrg_gemm_split_check() stages the bf16 operand planes in device memory it
// obtains with cudaMalloc.  Some callers cannot allow that: their device
// memory belongs to another allocator (a framework's caching allocator or a
// fixed arena sized up front), or they run latency-critical loops in which a
// cudaMalloc/cudaFree pair would synchronise the device or fail under memory
// pressure in the middle of a request.  hotrg_gemm_split_noalloc() takes the
// caller's device buffers for A, B and C and keeps its scratch (the operand
// planes and an error word) in the file-scope array below, which every GPU
// that loads this library holds until the process exits.
#include <cstring>
#include <mutex>

#include "../../include/hotrg.h"
#include "common.cuh"
#include "gemm_tc.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = 8u << 20;   // 8 MiB per device
constexpr size_t kHeader = 256;              // error word, padded to 256 bytes

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct DeviceInfo {
  unsigned char* scratch = nullptr;   // device address of g_noalloc_scratch
  int sms = 0;                        // multiprocessor count
  bool supported = false;             // compute capability 10.3
};
DeviceInfo g_dev[kMaxDevices];

long long round_up64(long long v) { return (v + 63) / 64 * 64; }

// Set-up of the current device, done once and cached: the device address of
// the scratch array (its name in host code is only a host-side stand-in, so
// the address is looked up with the device current) and the two attributes
// the launch needs.
hotrg_status device_info(DeviceInfo* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HOTRG_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceInfo& d = g_dev[dev];
  if (!d.scratch) {
    void* p = nullptr;
    int major = 0, minor = 0, sms = 0;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
      return HOTRG_ECUDA;
    d.sms = sms;
    d.supported = major == 10 && minor == 3;
    d.scratch = static_cast<unsigned char*>(p);
  }
  *out = d;
  return HOTRG_OK;
}

hotrg_status run(int M, int N, int K, int planes, int kchunk, const double* A_dev,
                 const double* B_dev, double* C_dev, cudaStream_t s) {
  using namespace hotrg;
  const long long sa = round_up64((long long)M * K), sb = round_up64((long long)N * K);
  const long long need = (long long)kHeader + 2LL * planes * (sa + sb);
  if (need > (long long)kScratchBytes) return HOTRG_EINVAL;   // operands exceed the scratch
  DeviceInfo d;
  hotrg_status st = device_info(&d);
  if (st != HOTRG_OK) return st;
  if (!d.supported) return HOTRG_EUNSUPPORTED;
  int* err = reinterpret_cast<int*>(d.scratch);
  __nv_bfloat16* pa = reinterpret_cast<__nv_bfloat16*>(d.scratch + kHeader);
  __nv_bfloat16* pb = pa + (size_t)planes * sa;
  // The scratch keeps the previous call's contents: the error words (all bits
  // seen, first bit seen) must start at zero.
  if (cudaMemsetAsync(err, 0, 2 * sizeof(int), s) != cudaSuccess) return HOTRG_ECUDA;
  // Operand planes exactly as hotrg_gemm_split_check prepares them: plane 0
  // on the per-segment power-of-two grid that the exact hi*hi accumulation
  // of the GEMM relies on.
  if (grid_split(A_dev, (long long)M * K, map_lin(K), map_lin(1), M, K, planes, sa, pa, err, s,
                 d.sms) != cudaSuccess ||
      grid_split(B_dev, (long long)N * K, map_lin(K), map_lin(1), N, K, planes, sb, pb, err, s,
                 d.sms) != cudaSuccess)
    return HOTRG_ECUDA;
  TcGemm g;
  memset(&g, 0, sizeof(g));
  tc_set_pairs(g, planes);
  g.M = M; g.N = N; g.K = K; g.kchunk = kchunk;
  g.cm = map_lin(N); g.cn = map_lin(1);
  g.out_mode = kOutF64; g.out_planes = 1; g.C = C_dev; g.alpha = 1.f; g.err = err;
  g.c_lim = (long long)M * N;
  TcOperand a, b;
  a.ptr = pa; a.rows = M; a.K = K; a.planes = planes; a.plane_stride = sa;
  b.ptr = pb; b.rows = N; b.K = K; b.planes = planes; b.plane_stride = sb;
  if (tc_gemm(a, b, g, s, d.sms) != cudaSuccess) return HOTRG_ECUDA;
  int e = 0;
  if (cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return HOTRG_ECUDA;
  if (e & kErrTimeout) return HOTRG_ETIMEOUT;
  if (e) return HOTRG_ECUDA;
  return HOTRG_OK;
}

}  // namespace

extern "C" hotrg_status hotrg_gemm_split_noalloc(int M, int N, int K, int planes, int kchunk,
                                                 const double* A_dev, const double* B_dev,
                                                 double* C_dev, void* stream) {
  if (M < 1 || N < 1 || K < 8 || K % 8 != 0 || (planes != 2 && planes != 3) || !A_dev ||
      !B_dev || !C_dev)
    return HOTRG_EINVAL;
  const hotrg_status st =
      run(M, N, K, planes, kchunk, A_dev, B_dev, C_dev, reinterpret_cast<cudaStream_t>(stream));
  // A failed CUDA call leaves the runtime's last-error state set; clear it so
  // that a later, unrelated call of the caller does not report it.
  if (st != HOTRG_OK) cudaGetLastError();
  return st;
}
