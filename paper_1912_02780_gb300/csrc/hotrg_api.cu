// Plan / executor and C ABI of the HOTRG library (declared in include/hotrg.h).
//
// A plan fixes the bond-dimension schedule of every step, allocates all device
// memory once, and runs each coarse-graining step as a short sequence of
// kernels on one CUDA stream:
//
//   Gram (SM Sec. B: isometry from the local HOSVD of the merged pair)
//     A = T.T over (x1', y), B = T.T over (x2', y'), G = sum_{j j'} A B
//   FP64 eigensolve of G (cuSOLVER), descending order, sign fix
//   HOTRG step equation (SM Sec. B) as three GEMMs, chunked over the free leg y
//     S1: U[(y x1' a)][(x2 j)]   = sum_{x1} T[x1 x1' y j] w[x1 x2 a]
//     S2: V[(y a y')][(x1' x2')] = sum_{x2 j} U T[x2 x2' j y']
//     S3: T'[y][y'][a][b]        = sum_{x1' x2'} V w[x1' x2' b]
//     (written directly in the re-oriented layout used by the next step)
//   FP64 Frobenius normalisation and log-norm.
//
// Steps marked "split" run the Gram and S1-S3 on the tcgen05 split-BF16 GEMM;
// the others (and the whole FP64 precision mode) use the FP64 GEMM.  The
// backward (SM Sec. B recursion = SM Sec. E chain rule, main-text Eq. (1) for
// the adjoint of w, plus the adjoint of the truncated eigensolve and of the
// Gram assembly) recomputes U and V per step from the stored T_k and w_k.
#include <cusolverDn.h>
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hotrg.h"
#include "common.cuh"
#include "gemm_f64.h"
#include "gemm_tc.h"
#include "kernels.h"
#include "plan_access.h"

using namespace hotrg;

namespace {

constexpr long long kChunkF64 = 1LL << 27;     // FP64 stage chunk budget (elements)
constexpr long long kChunkSplit = 1LL << 30;   // split stage chunk budget (elements per plane)
constexpr int kMaxPartial = 4096;
constexpr long long kSplitK = 1LL << 25;       // FP64 split-K workspace (elements)

struct StepGeom {
  int X, Y, Xp;
  long long N;        // X * X
  bool split;
  int np;             // bf16 planes of the split GEMM operands (0: FP64 step)
  int yc64, ycs;      // y-chunk of the FP64 and split stage buffers
};

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

struct Layout {
  std::vector<StepGeom> g;
  long long maxT = 0, maxN = 0, maxN2 = 0, maxXp = 0;
  long long chunk64 = 0, chunkS = 0;       // elements
  long long splitT = 0, splitG = 0, splitW1 = 0, splitW3 = 0;   // elements per plane
  long long totalE = 0, totalT = 0, totalLam = 0;
  int np = 0;          // planes of the configured split precision
  int np_max = 0;      // most planes of any step (4 on the high-precision steps)
  bool any_split = false, any_hi = false;
};

int planes_of(int precision) {
  return precision == HOTRG_BF16X6 ? 3 : (precision == HOTRG_BF16X3 ? 2 : 0);
}

bool build_layout(const hotrg_config& c, Layout& L) {
  L = Layout();
  L.np = planes_of(c.precision);
  long long X = c.d0, Y = c.d0;
  for (int k = 1; k <= c.n_steps; ++k) {
    StepGeom s;
    s.X = (int)X;
    s.Y = (int)Y;
    s.N = X * X;
    long long Xp = s.N < c.d_cut ? s.N : c.d_cut;
    s.Xp = (int)Xp;
    s.split = L.np > 0 && k >= c.split_from_step && X % 8 == 0 && Y % 8 == 0 && Xp % 8 == 0;
    s.np = 0;
    if (s.split) {
      s.np = (L.np == 3 && k < c.split_from_step + c.hi_precision_steps) ? 4 : L.np;
      if (s.np > L.np_max) L.np_max = s.np;
      if (s.np == 4) L.any_hi = true;
    }
    long long per_y = X * X * Xp * Y;
    long long a = kChunkF64 / per_y;
    s.yc64 = (int)(a < 1 ? 1 : (a > Y ? Y : a));
    const long long chunk_split = c.split_chunk_elems > 0 ? c.split_chunk_elems : kChunkSplit;
    long long b = chunk_split / per_y;
    s.ycs = (int)(b < 1 ? 1 : (b > Y ? Y : b));
    if (s.N > (1LL << 31) / 2 || X * X * Y * Y > (1LL << 31) || per_y * Y > (1LL << 42)) return false;
    L.g.push_back(s);
    long long tin = X * X * Y * Y, tout = Y * Y * Xp * Xp;
    if (tin > L.maxT) L.maxT = tin;
    if (tout > L.maxT) L.maxT = tout;
    if (s.N > L.maxN) L.maxN = s.N;
    if (s.N * s.N > L.maxN2) L.maxN2 = s.N * s.N;
    if (Xp > L.maxXp) L.maxXp = Xp;
    L.totalT += tout;
    L.totalE += c.want_grad ? s.N * s.N : 0;
    L.totalLam += s.N;
    long long c64 = (long long)s.yc64 * per_y;
    if (c64 > L.chunk64) L.chunk64 = c64;
    if (s.split) {
      L.any_split = true;
      long long cs = (long long)s.ycs * per_y;
      if (cs > L.chunkS) L.chunkS = cs;
      if (tin > L.splitT) L.splitT = tin;
      if (X * X * Y * Y > L.splitG) L.splitG = X * X * Y * Y;
      if (Xp * X * X > L.splitW1) L.splitW1 = Xp * X * X;
      if (Xp * X * X > L.splitW3) L.splitW3 = Xp * X * X;
    }
    if (c.scheme == 1) {
      X = Xp;         // scheme (b): T' is stored (Xp, Xp, Y, Y), the vertical legs keep Y
    } else {
      Y = Xp;         // T' is (Xp, Xp, Y, Y), stored re-oriented as (Y, Y, Xp, Xp)
      X = s.Y;
    }
  }
  L.totalT += (long long)c.d0 * c.d0 * c.d0 * c.d0;
  L.chunkS = round_up(L.chunkS, 64);
  L.splitT = round_up(L.splitT, 64);
  L.splitG = round_up(L.splitG, 64);
  L.splitW1 = round_up(L.splitW1, 64);
  L.splitW3 = round_up(L.splitW3, 64);
  return true;
}

struct Bytes {
  size_t total = 0;
  void add(long long elems, size_t elsize) { total += round_up(elems * (long long)elsize, 256); }
};

}  // namespace

struct hotrg_plan_s {
  hotrg_config cfg;
  int n_run = 0;      // steps the forward and backward run (<= cfg.n_steps)
  Layout L;
  cudaStream_t stream = nullptr;
  cusolverDnHandle_t solver = nullptr;
  int sms = 152;
  int tc_sms = 152;   // CTAs of the persistent tensor-core GEMMs (sms - gemm_sm_reserve)
  std::vector<void*> allocs;
  std::vector<size_t> alloc_bytes;
  std::vector<double*> T, E, lam;
  double *Escr = nullptr, *wasc = nullptr, *work = nullptr;
  int lwork = 0;
  int* info = nullptr;
  double *Abuf = nullptr, *Bbuf = nullptr, *Abar = nullptr, *Bbar = nullptr;
  double *Ub = nullptr, *Vb = nullptr, *Pb = nullptr, *Qb = nullptr;
  double *Sb = nullptr, *Hb = nullptr, *wbT = nullptr, *Gb = nullptr;
  double *Ecur = nullptr, *Enext = nullptr, *Tbar = nullptr;
  double *dT0 = nullptr, *partial = nullptr, *scal = nullptr, *log_norms = nullptr, *out = nullptr;
  double *dtrunc = nullptr, *dgap = nullptr;
  double* dres = nullptr;     // per step: max relative residual of the kept Ritz pairs
  int* err = nullptr;         // [0] all error bits, [1] first bit, [2] residual guard code
  // subspace eigensolver guard, per step of the last forward: extra power
  // iterations it took, and whether the exact eigensolver had to finish it;
  // steps on which it fired over the plan's lifetime
  std::vector<int> guard_iters;
  std::vector<char> exact_step;
  long long fallbacks = 0;
  int* guard_host = nullptr;       // pinned host word the guard is read into
  // warm start of the subspace eigensolver: kept eigenvectors of the last two
  // steps (by step parity) and their shapes
  double* wkeep[2] = {nullptr, nullptr};
  int wkeep_n[2] = {0, 0}, wkeep_xp[2] = {0, 0};
  __nv_bfloat16 *pTA = nullptr, *pTB = nullptr, *pA = nullptr, *pB = nullptr, *pW1 = nullptr,
                *pT1 = nullptr, *pP = nullptr, *pW3 = nullptr, *pU = nullptr, *pV = nullptr;
  float* F32 = nullptr;   // FP32 GEMM output awaiting its grid-aligned split
  double* F64 = nullptr;  // same, FP64, for the four-plane steps
  double* splitk = nullptr;   // FP64 split-K partials (deterministic reduction)
  // randomized subspace eigensolver (eigh_mode 1)
  double *Qs = nullptr, *Zs = nullptr, *Hs = nullptr, *tau = nullptr, *swork = nullptr,
         *wsmall = nullptr;
  int kspace = 0, lswork = 0;
  bool have_fwd = false, fwd_ising = false, have_bwd = false, w_loaded = false;
  // gradient plans: d(ln Z/N)/d w_k of every step (rows = kept vectors)
  double* wbar_all = nullptr;
  std::vector<long long> w_off;        // offset of step k's Xp x N block
  // MERA update (SVD of the environment): workspace and status
  double* svd_work = nullptr;
  double* svd_rwork = nullptr;
  int svd_lwork = 0;
  // w_given plans: steps 1..given_steps use the stored isometries, later steps
  // take theirs from the Gram matrix (scheme (b) cooling, one new layer at a time)
  int given_steps = 0;
  int w_valid = 0;    // leading steps whose stored isometries are defined
  // scheme (b): dominant eigenvectors of the exact-product transfer operator
  // (right one of the last forward, left one of the backward), power-iteration
  // buffers, and out_k of every step
  double *chR = nullptr, *chW = nullptr, *chV = nullptr, *chZ = nullptr, *lnz_steps = nullptr;
  // w_rule 1: the right side's eigenpairs, truncation error and gap, and the
  // side each step took (device, and read on the host by the backward)
  double *Er = nullptr, *lamR = nullptr, *trR = nullptr;
  int* side_dev = nullptr;
  std::vector<int> side_host;
  std::string last_error;
  // optional per-stage CUDA-event timing
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> prof_rec;
};

namespace {

std::atomic<unsigned long long> g_launches{0};

// Host-side fault injection (tests of the error paths without a GPU fault):
// what = 1: the arg-th device allocation fails; 2: the eigensolver of step arg
// reports failure; 3: a NaN is written into the tensor of step arg.
std::atomic<int> g_inj_what{0}, g_inj_arg{0}, g_inj_count{0};
enum { kInjAlloc = 1, kInjEigh = 2, kInjNaN = 3 };

// Brackets one stage of the path with CUDA events on the plan's stream when
// profiling is on (slot = stage id, + 16 for the FP64 variant of a contraction).
struct Stage {
  hotrg_plan p;
  int slot;
  size_t idx;
  Stage(hotrg_plan p_, int slot_) : p(p_), slot(slot_), idx((size_t)-1) {
    if (p->prof && p->ev_used + 2 <= p->ev_pool.size()) {
      idx = p->ev_used;
      p->ev_used += 2;
      cudaEventRecord(p->ev_pool[idx], p->stream);
    }
  }
  ~Stage() {
    if (idx != (size_t)-1) {
      cudaEventRecord(p->ev_pool[idx + 1], p->stream);
      p->prof_rec.push_back({slot, idx});
    }
  }
};

hotrg_status fail(hotrg_plan p, hotrg_status s, const std::string& msg) {
  if (p) p->last_error = msg;
  return s;
}

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(p, HOTRG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define CK2(plan, call)                                                             \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(plan, HOTRG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
hotrg_status dalloc(hotrg_plan p, T** ptr, long long elems) {
  *ptr = nullptr;
  if (elems <= 0) return HOTRG_OK;
  void* v = nullptr;
  if (g_inj_what.load() == kInjAlloc && g_inj_count.fetch_add(1) + 1 == g_inj_arg.load())
    return fail(p, HOTRG_ENOMEM, "cudaMalloc failed (injected)");
  if (cudaMalloc(&v, (size_t)elems * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(p, HOTRG_ENOMEM, "cudaMalloc failed");
  }
  p->allocs.push_back(v);
  p->alloc_bytes.push_back((size_t)elems * sizeof(T));
  *ptr = reinterpret_cast<T*>(v);
  return HOTRG_OK;
}

// Elements of size `elsize` from ptr to the end of the plan allocation that
// holds it (0 if none does): the bound every kernel access is checked against.
long long lim_of(const hotrg_plan p, const void* ptr, size_t elsize) {
  const char* c = reinterpret_cast<const char*>(ptr);
  for (size_t i = 0; i < p->allocs.size(); ++i) {
    const char* b = reinterpret_cast<const char*>(p->allocs[i]);
    if (c >= b && c < b + p->alloc_bytes[i]) return (long long)((b + p->alloc_bytes[i] - c) / elsize);
  }
  return 0;
}

#define AL(ptr, n)                                \
  do {                                            \
    hotrg_status s_ = dalloc(p, &(ptr), (n));     \
    if (s_ != HOTRG_OK) return s_;                \
  } while (0)

hotrg_status validate(const hotrg_config* c) {
  if (!c) return HOTRG_EINVAL;
  if (c->d0 < 1 || c->d_cut < 1 || c->n_steps < 1 || c->n_steps > 200) return HOTRG_EINVAL;
  if (c->precision < HOTRG_FP64 || c->precision > HOTRG_BF16X6) return HOTRG_EINVAL;
  if (c->split_from_step < 1 || c->hi_precision_steps < 0) return HOTRG_EINVAL;
  if (c->eigh_mode < 0 || c->eigh_mode > 1) return HOTRG_EINVAL;
  if (c->split_chunk_elems < 0 || c->split_chunk_elems > (1LL << 34)) return HOTRG_EINVAL;
  if (c->w_given && (!c->want_grad || !c->fixed_w_grad)) return HOTRG_EINVAL;
  if (!std::isfinite(c->eigh_residual_tol) || c->eigh_residual_tol < 0) return HOTRG_EINVAL;
  if (c->stage2_n_group < 0) return HOTRG_EINVAL;
  if (c->gemm_sm_reserve < 0 || c->gemm_sm_reserve > 64) return HOTRG_EINVAL;
  if (c->eigh_warm_start < 0 || c->eigh_warm_start > 16) return HOTRG_EINVAL;
  if (c->scheme < 0 || c->scheme > 1 || c->chain_steps < 0 || c->chain_steps > 1)
    return HOTRG_EINVAL;
  if (c->scheme == 1 && c->d_cut > 4096) return HOTRG_EINVAL;
  if (c->w_rule < 0 || c->w_rule > 1 || (c->w_rule == 1 && c->w_given)) return HOTRG_EINVAL;
  return HOTRG_OK;
}

GemmF64 g64(const hotrg_plan p, const double* A, IMap am, IMap ak, const double* B, IMap bn,
            IMap bk, double* C, IMap cm, IMap cn, int M, int N, int K, double alpha, double beta) {
  GemmF64 g;
  g.a_lim = lim_of(p, A, sizeof(double));
  g.b_lim = lim_of(p, B, sizeof(double));
  g.c_lim = lim_of(p, C, sizeof(double));
  g.err = p->err;
  g.ws = p->splitk;
  g.ws_elems = kSplitK;
  g.A = A; g.am = am; g.ak = ak;
  g.B = B; g.bn = bn; g.bk = bk;
  g.C = C; g.cm = cm; g.cn = cn;
  g.M = M; g.N = N; g.K = K;
  g.alpha = alpha; g.beta = beta;
  g.a_kfast = (ak.s0 == 1) ? 1 : 0;
  g.b_kfast = (bk.s0 == 1) ? 1 : 0;
  return g;
}

TcGemm tcg(const hotrg_plan p, int np, int M, int N, int K, IMap cm, IMap cn, int mode, void* C,
           long long out_plane_stride) {
  TcGemm g;
  memset(&g, 0, sizeof(g));
  tc_set_pairs(g, np);
  g.M = M; g.N = N; g.K = K;
  g.kchunk = kGridSeg / 64;   // accumulation chunk = grid segment of the operand split
  g.cm = cm; g.cn = cn;
  g.out_mode = mode;
  g.out_planes = np;
  g.out_plane_stride = out_plane_stride;
  g.C = C;
  g.alpha = 1.f;
  g.accumulate = 0;
  g.c_lim = lim_of(p, C, mode == kOutF64 ? 8 : (mode == kOutF32 ? 4 : 2));
  if (mode == kOutGridSplit && out_plane_stride > 0 && g.c_lim > out_plane_stride)
    g.c_lim = out_plane_stride;
  g.err = p->err;
  return g;
}

// Operand preparation: grid-aligned bf16 planes (see kernels.cu: grid_split).
cudaError_t gsplit(const hotrg_plan p, const double* src, IMap rm, IMap km, int rows, int K,
                   int np, long long stride, __nv_bfloat16* dst) {
  return grid_split(src, lim_of(p, src, sizeof(double)), rm, km, rows, K, np, stride, dst, p->err,
                    p->stream, p->sms);
}
// Split a GEMM output kept in the staging buffer: FP32 for three planes, FP64
// for four (a float cannot feed more than three bf16 planes).
cudaError_t fsplit(const hotrg_plan p, int np, int rows, int K, long long stride,
                   __nv_bfloat16* dst) {
  if (np == 4)
    return grid_split(p->F64, lim_of(p, p->F64, sizeof(double)), map_lin(K), map_lin(1), rows, K,
                      np, stride, dst, p->err, p->stream, p->sms);
  return grid_split(p->F32, lim_of(p, p->F32, sizeof(float)), map_lin(K), map_lin(1), rows, K, np,
                    stride, dst, p->err, p->stream, p->sms);
}
// Output mode and buffer of a GEMM whose result is split again.
int stage_mode(int np) { return np == 4 ? kOutF64 : kOutF32; }
void* stage_buf(const hotrg_plan p, int np) {
  return np == 4 ? static_cast<void*>(p->F64) : static_cast<void*>(p->F32);
}

TcOperand opnd(const __nv_bfloat16* ptr, int rows, int K, int planes, long long stride) {
  TcOperand o;
  o.ptr = ptr; o.rows = rows; o.K = K; o.planes = planes; o.plane_stride = stride;
  return o;
}

// ---- forward pieces -------------------------------------------------------

enum StageId { kStGram = 0, kStEigh = 1, kStS1 = 2, kStS2 = 3, kStS3 = 4, kStNorm = 5,
               kStPrep = 6, kStBwdContract = 7, kStBwdEigh = 8, kStBwdGram = 9, kStS2Hi = 10,
               kStEighProd = 11, kStEighQR = 12, kStEighRR = 13, kStEighRes = 14,
               kStF64 = 16 };

// Strides of T's horizontal legs l and r: the Gram matrix of the right side
// (w_rule 1) is the left one of T with l and r exchanged, i.e. the same
// contractions with the two strides swapped.
void lr_strides(const StepGeom& s, bool right, long long& sl, long long& sr) {
  const long long XY2 = (long long)s.X * s.Y * s.Y, Y2 = (long long)s.Y * s.Y;
  sl = right ? Y2 : XY2;
  sr = right ? XY2 : Y2;
}

hotrg_status gram_f64(hotrg_plan p, const StepGeom& s, const double* T, double* A, double* B,
                      double* G, bool right = false) {
  Stage sc(p, kStGram + kStF64);
  const int X = s.X, Y = s.Y;
  const long long XY2 = (long long)X * Y * Y, Y2 = (long long)Y * Y;
  long long sl, sr;
  lr_strides(s, right, sl, sr);
  cudaStream_t st = p->stream;
  CK(gemm_f64(g64(p, T, map2(Y, 1, sl), map2(Y, Y, sr), T, map2(Y, 1, sl), map2(Y, Y, sr), A,
                  map2(Y, Y, XY2), map2(Y, 1, Y2), X * Y, X * Y, X * Y, 1.0, 0.0),
              st, p->sms));
  CK(gemm_f64(g64(p, T, map2(Y, Y, sl), map2(Y, 1, sr), T, map2(Y, Y, sl), map2(Y, 1, sr), B,
                  map2(Y, Y, XY2), map2(Y, 1, Y2), X * Y, X * Y, X * Y, 1.0, 0.0),
              st, p->sms));
  if (G)
    CK(gemm_f64(g64(p, A, map_lin(Y2), map_lin(1), B, map_lin(Y2), map_lin(1), G,
                    map2(X, X, (long long)X * X * X), map2(X, 1, (long long)X * X), X * X, X * X,
                    Y * Y, 1.0, 0.0),
                st, p->sms));
  return HOTRG_OK;
}

hotrg_status gram_split(hotrg_plan p, const StepGeom& s, const double* T, double* G,
                        bool right = false) {
  const int X = s.X, Y = s.Y, np = s.np;
  const long long XY2 = (long long)X * Y * Y, Y2 = (long long)Y * Y;
  long long sl, sr;
  lr_strides(s, right, sl, sr);
  cudaStream_t st = p->stream;
  const long long sT = p->L.splitT, sG = p->L.splitG;
  {
    Stage sc(p, kStPrep);
    CK(gsplit(p, T, map2(Y, 1, sl), map2(Y, Y, sr), X * Y, X * Y, np, sT, p->pTA));
    CK(gsplit(p, T, map2(Y, Y, sl), map2(Y, 1, sr), X * Y, X * Y, np, sT, p->pTB));
  }
  Stage sc(p, kStGram);
  TcOperand ta = opnd(p->pTA, X * Y, X * Y, np, sT), tb = opnd(p->pTB, X * Y, X * Y, np, sT);
  CK(tc_gemm(ta, ta, tcg(p, np, X * Y, X * Y, X * Y, map2(Y, Y, XY2), map2(Y, 1, Y2),
                         stage_mode(np), stage_buf(p, np), 0),
             st, p->tc_sms));
  CK(fsplit(p, np, X * X, Y * Y, sG, p->pA));
  CK(tc_gemm(tb, tb, tcg(p, np, X * Y, X * Y, X * Y, map2(Y, Y, XY2), map2(Y, 1, Y2),
                         stage_mode(np), stage_buf(p, np), 0),
             st, p->tc_sms));
  CK(fsplit(p, np, X * X, Y * Y, sG, p->pB));
  TcOperand a = opnd(p->pA, X * X, Y * Y, np, sG), b = opnd(p->pB, X * X, Y * Y, np, sG);
  CK(tc_gemm(a, b, tcg(p, np, X * X, X * X, Y * Y, map2(X, X, (long long)X * X * X),
                       map2(X, 1, (long long)X * X), kOutF64, G, 0),
             st, p->tc_sms));
  return HOTRG_OK;
}

hotrg_status contract_f64(hotrg_plan p, const StepGeom& s, const double* T, const double* Ek,
                          double* Tout) {
  const int X = s.X, Y = s.Y, Xp = s.Xp;
  const long long N = s.N, XY = (long long)X * Y, Y2 = (long long)Y * Y, XY2 = XY * Y;
  const long long Xp2 = (long long)Xp * Xp, X2 = (long long)X * X;
  cudaStream_t st = p->stream;
  for (int y0 = 0; y0 < Y; y0 += s.yc64) {
    const int yc = (Y - y0) < s.yc64 ? (Y - y0) : s.yc64;
    {
      Stage sc(p, kStS1 + kStF64);
      CK(gemm_f64(g64(p, Ek, map2(X, 1, N), map_lin(X), T + (long long)y0 * Y, map3(Y, X, 1, Y2, Y),
                      map_lin(XY2), p->Ub, map2(X, Y, XY), map3(Y, X, 1, Xp * XY, X * Xp * XY),
                      Xp * X, yc * X * Y, X, 1.0, 0.0),
                  st, p->sms));
    }
    {
      Stage sc(p, kStS2 + kStF64);
      CK(gemm_f64(g64(p, p->Ub, map_lin(XY), map_lin(1), T, map2(X, Y2, 1), map2(Y, Y, XY2), p->Vb,
                      map3(Xp, X, Y * X2, X, Xp * Y * X2), map2(X, 1, X2), yc * X * Xp, Y * X,
                      X * Y, 1.0, 0.0),
                  st, p->sms));
    }
    {
      Stage sc(p, kStS3 + kStF64);
      CK(gemm_f64(g64(p, p->Vb, map_lin(X2), map_lin(1), Ek, map_lin(N), map_lin(1),
                      Tout + (long long)y0 * Y * Xp2, map3(Y, Xp, Xp2, Xp, Y * Xp2), map_lin(1),
                      yc * Xp * Y, Xp, X * X, 1.0, 0.0),
                  st, p->sms));
    }
  }
  return HOTRG_OK;
}

// N-tiles per L2 raster group of the stage-2 GEMM (0 in the config: the
// default; >= the N-tile count: plain N-fastest order).
int stage2_group(const hotrg_config& c) { return c.stage2_n_group > 0 ? c.stage2_n_group : 16; }
// Stage-2 GEMM on CTA pairs (config: 0 = the default, off: the pair kernel
// measured slower on GB300, 46.4 vs 42.4 ms per D = 64 launch; > 0 = on).
int stage2_pair(const hotrg_config& c) { return c.stage2_pair > 0 ? 1 : 0; }

// Segment partner of the grid-split epilogue (see gemm_tc.h: kOutGridSplit)
// for an output whose 64-column half-runs are `run` consecutive destination
// elements of the consumer's K: the other half of a 128-segment is in the
// partner half of the same row (run = 128) or in the row `row_step` away
// (run = 64).  Returns false when the layout does not allow the fused split.
bool seg_partner(int run, long long row_step, int& prow, int& phalf) {
  prow = phalf = 0;
  if (run == 128) { phalf = 1; return true; }
  if (run == 64 && row_step > 0 && row_step < 128 && (row_step & (row_step - 1)) == 0) {
    prow = (int)row_step;
    return true;
  }
  return false;
}

hotrg_status contract_split(hotrg_plan p, const StepGeom& s, const double* T, const double* Ek,
                            double* Tout) {
  const int X = s.X, Y = s.Y, Xp = s.Xp, np = s.np;
  const long long N = s.N, XY = (long long)X * Y, Y2 = (long long)Y * Y, XY2 = XY * Y;
  const long long Xp2 = (long long)Xp * Xp, X2 = (long long)X * X;
  cudaStream_t st = p->stream;
  const long long sT = p->L.splitT, sW1 = p->L.splitW1, sW3 = p->L.splitW3, sC = p->L.chunkS;
  // operands shared by all y-chunks
  {
  Stage sc(p, kStPrep);
  CK(gsplit(p, Ek, map2(X, 1, N), map_lin(X), Xp * X, X, np, sW1, p->pW1));
  CK(gsplit(p, T, map3(Y, X, 1, Y2, Y), map_lin(XY2), Y * X * Y, X, np, sT, p->pT1));
  CK(gsplit(p, T, map2(X, Y2, 1), map2(Y, Y, XY2), Y * X, X * Y, np, sT, p->pP));
  CK(gsplit(p, Ek, map_lin(N), map_lin(1), Xp, X * X, np, sW3, p->pW3));
  }
  const TcOperand w1 = opnd(p->pW1, Xp * X, X, np, sW1);
  const TcOperand pp = opnd(p->pP, Y * X, X * Y, np, sT);
  const TcOperand w3 = opnd(p->pW3, Xp, X * X, np, sW3);
  // Three-plane steps write U and V as bf16 planes straight from the GEMM
  // epilogue where the layout allows it (bit-identical to the FP32 staging
  // buffer + grid split; saves their FP32 round trip through HBM).
  const bool fuse = np == 3 && p->cfg.epilogue_split != 0;
  int p1r = 0, p1h = 0, p2r = 0, p2h = 0;
  const bool fuse1 = fuse && (Xp * X) % 128 == 0 && (XY % 128) == 0 && X % 2 == 0 &&
                     seg_partner(Y, 1, p1r, p1h);            // S1: j runs, x2 partner = row ^ 1
  const bool fuse2 = fuse && (Y * X) % 128 == 0 && (X2 % 128) == 0 &&
                     seg_partner(X, Xp, p2r, p2h);           // S2: x2' runs, x1' partner = row ^ Xp
  for (int y0 = 0; y0 < Y; y0 += s.ycs) {
    const int yc = (Y - y0) < s.ycs ? (Y - y0) : s.ycs;
    const TcOperand t1 = opnd(p->pT1 + (long long)y0 * X * Y * X, yc * X * Y, X, np, sT);
    {
    Stage sc(p, kStS1);
    TcGemm g1 = tcg(p, np, Xp * X, yc * X * Y, X, map2(X, Y, XY),
                    map3(Y, X, 1, Xp * XY, X * Xp * XY),
                    fuse1 ? kOutGridSplit : stage_mode(np), fuse1 ? (void*)p->pU : stage_buf(p, np),
                    fuse1 ? sC : 0);
    g1.m_fast = 1;   // the W1 tiles stay in L2; each T1 tile is read from HBM once
    g1.seg_prow = p1r;
    g1.seg_phalf = p1h;
    CK(tc_gemm(w1, t1, g1, st, p->tc_sms));
    if (!fuse1) CK(fsplit(p, np, yc * X * Xp, X * Y, sC, p->pU));
    }
    const TcOperand u = opnd(p->pU, yc * X * Xp, X * Y, np, sC);
    {
    Stage sc(p, np == 4 ? kStS2Hi : kStS2);
    TcGemm g2 = tcg(p, np, yc * X * Xp, Y * X, X * Y, map3(Xp, X, Y * X2, X, Xp * Y * X2),
                    map2(X, 1, X2), fuse2 ? kOutGridSplit : stage_mode(np),
                    fuse2 ? (void*)p->pV : stage_buf(p, np), fuse2 ? sC : 0);
    g2.seg_prow = p2r;
    g2.seg_phalf = p2h;
    g2.n_group = stage2_group(p->cfg);
    g2.cta_pair = stage2_pair(p->cfg);
    CK(tc_gemm(u, pp, g2, st, p->tc_sms));
    }
    if (!fuse2) {
    Stage sc(p, kStPrep);
    CK(fsplit(p, np, yc * Xp * Y, X * X, sC, p->pV));
    }
    const TcOperand v = opnd(p->pV, yc * Xp * Y, X * X, np, sC);
    Stage sc(p, kStS3);
    CK(tc_gemm(v, w3,
               tcg(p, np, yc * Xp * Y, Xp, X * X, map3(Y, Xp, Xp2, Xp, Y * Xp2), map_lin(1), kOutF64,
                   Tout + (long long)y0 * Y * Xp2, 0),
               st, p->tc_sms));
  }
  return HOTRG_OK;
}

double* E_of(hotrg_plan p, int k) { return p->cfg.want_grad ? p->E[k - 1] : p->E[0]; }

// Block size of the subspace eigensolver at a step (D' + 1 at least: the
// kept vectors and one more for the gap).
int subspace_k(const hotrg_config& c, const StepGeom& s) {
  const int k = c.eigh_block > 0 ? c.eigh_block : 4 * s.Xp;
  return k > s.Xp + 1 ? k : s.Xp + 1;
}

bool subspace_applies(const hotrg_config& c, const StepGeom& s) {
  return c.eigh_mode == 1 && c.w_rule == 0 && (!c.want_grad || c.fixed_w_grad) &&
         (long long)subspace_k(c, s) < s.N;
}

bool use_subspace(const hotrg_plan p, const StepGeom& s) { return subspace_applies(p->cfg, s); }

// Ritz pairs the subspace eigensolver returns: the D' kept and one more.
int subspace_ritz(const StepGeom& s) { return s.Xp + 1; }

// Randomized subspace eigensolver for the leading eigenpairs of the symmetric
// PSD Gram matrix G (N x N, in p->Escr): a block of k vectors (eigh_block,
// default 4 D'), started from a deterministic pseudo-random block, is
// multiplied by G eigh_power_iters times with a Householder QR (cuSOLVER
// geqrf + orgqr) after each product, and the Rayleigh-Ritz problem Q^T G Q
// (k x k, cuSOLVER syevdx, the D' + 1 largest pairs) gives the Ritz pairs.  The random start is not orthonormalised: only the span
// of the block matters to the iteration.  On split steps the products G Q run
// on the tensor cores with four-plane operands (10 products, G split once per
// step, FP64 output); the QR, the projection Q^T (G Q), the small eigensolve and
// the Ritz vectors stay in FP64.  The block is stored as k contiguous vectors
// of length N, i.e. an N x k column-major matrix for cuSOLVER.  Output: the
// D' + 1 leading Ritz vectors (ascending Ritz values) in p->Zs as contiguous
// rows and their Ritz values in p->wasc, ready for eig_desc.
constexpr int kEighPlanes = 4;

// Residual bound of the kept Ritz pairs at step k, relative to the largest
// eigenvalue, above which the step's subspace eigensolve is refined.  The
// bound is on 2^-k r_k: an error made at step k enters ln Z / N with weight
// 2^-k (through ln c_k / 2^k and every later step of the same 2^k-site
// block).  Measured on GB300 (random d0 = 4 tensors with and without the
// reflection symmetry at D_cut = 16, 32, 64, Ising at beta_c, D_cut = 64): the
// ln Z / N error of a solve stayed below 0.05 times the sum over its steps of
// 2^-k r_k; with the bound at 1e-9 every benchmark seed (0-4, warm start) was
// within 1e-9 of the oracle, with 5e-9 seed 4 was not (1.05e-9).  The
// tensor-core products' own residual floor (about 1e-8 relative) passes it
// from step 4 on.
double residual_tol(const hotrg_config& c, int k) {
  const double t = c.eigh_residual_tol > 0 ? c.eigh_residual_tol : 1e-9;
  return std::ldexp(t, k);
}

bool subspace_on_tc(const hotrg_plan p, const StepGeom& s) {
  if (!s.split || !p->pU || !p->pV) return false;
  const long long N = s.N, K = subspace_k(p->cfg, s);
  const long long cap = p->L.chunkS * p->L.np_max;
  return N % 8 == 0 && kEighPlanes * round_up(N * N, 64) <= cap &&
         kEighPlanes * round_up(K * N, 64) <= cap;
}

// resume = true continues from the orthonormal block the previous call left
// in p->Qs with `iters` more power iterations (the accuracy guard's
// refinement) instead of starting from the random block.
hotrg_status eigh_subspace(hotrg_plan p, const StepGeom& s, int k_step, int iters, bool resume,
                           const double* warm = nullptr) {
  cudaStream_t st = p->stream;
  const int N = (int)s.N, K = subspace_k(p->cfg, s);
  const bool tc = subspace_on_tc(p, s);
  const long long sG = round_up((long long)N * N, 64), sQ = round_up((long long)K * N, 64);
  if (tc && !resume) {
    Stage sc(p, kStEighProd);
    CK(gsplit(p, p->Escr, map_lin(N), map_lin(1), N, N, kEighPlanes, sG, p->pV));
  }
  // Zs = G Qs, as rows: Z[a][i] = sum_j Q[a][j] G[i][j]
  auto product = [&]() -> hotrg_status {
    Stage sc(p, kStEighProd);
    if (tc) {
      CK(gsplit(p, p->Qs, map_lin(N), map_lin(1), K, N, kEighPlanes, sQ, p->pU));
      CK(tc_gemm(opnd(p->pU, K, N, kEighPlanes, sQ), opnd(p->pV, N, N, kEighPlanes, sG),
                 tcg(p, kEighPlanes, K, N, N, map_lin(N), map_lin(1), kOutF64, p->Zs, 0), st,
                 p->sms));
    } else {
      CK(gemm_f64(g64(p, p->Qs, map_lin(N), map_lin(1), p->Escr, map_lin(N), map_lin(1), p->Zs,
                      map_lin(N), map_lin(1), K, N, N, 1.0, 0.0),
                  st, p->sms));
    }
    return HOTRG_OK;
  };
  // Qs = orth(Zs): Householder QR (cuSOLVER geqrf + orgqr)
  auto householder = [&]() -> hotrg_status {
    CK(cudaMemcpyAsync(p->Qs, p->Zs, sizeof(double) * (size_t)K * N, cudaMemcpyDeviceToDevice,
                       st));
    if (cusolverDnDgeqrf(p->solver, N, K, p->Qs, N, p->tau, p->swork, p->lswork, p->info) !=
        CUSOLVER_STATUS_SUCCESS)
      return fail(p, HOTRG_ECUDA, "cusolverDnDgeqrf failed");
    CK(eigh_info_check(p->info, p->err, st));
    if (cusolverDnDorgqr(p->solver, N, K, K, p->Qs, N, p->tau, p->swork, p->lswork, p->info) !=
        CUSOLVER_STATUS_SUCCESS)
      return fail(p, HOTRG_ECUDA, "cusolverDnDorgqr failed");
    CK(eigh_info_check(p->info, p->err, st));
    return HOTRG_OK;
  };
  auto orth = [&]() -> hotrg_status {
    Stage sc(p, kStEighQR);
    return householder();
  };
  if (!resume) {
    CK(fill_random(p->Qs, (long long)K * N, 0x5EEDull + (unsigned long long)k_step, st, p->sms));
    // warm start: the first D' vectors of the block are the kept eigenvectors
    // of step k - 2 (same leg bases near the fixed point of the flow)
    if (warm)
      CK(cudaMemcpyAsync(p->Qs, warm, sizeof(double) * (size_t)s.Xp * N, cudaMemcpyDeviceToDevice,
                         st));
  }
  hotrg_status r;
  for (int it = 0; it < iters; ++it) {
    if ((r = product()) != HOTRG_OK) return r;
    if ((r = orth()) != HOTRG_OK) return r;
  }
  // Rayleigh-Ritz: Z = G Q, H[a][b] = sum_i Q[a][i] Z[b][i]
  if ((r = product()) != HOTRG_OK) return r;
  Stage sc(p, kStEighRR);
  CK(gemm_f64(g64(p, p->Qs, map_lin(N), map_lin(1), p->Zs, map_lin(N), map_lin(1), p->Hs,
                  map_lin(K), map_lin(1), K, K, N, 1.0, 0.0),
              st, p->sms));
  // only the D' + 1 largest Ritz pairs are used (D' kept, one more for the gap)
  const int nr = subspace_ritz(s);
  int meig = 0;
  if (cusolverDnDsyevdx(p->solver, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                        CUBLAS_FILL_MODE_LOWER, K, p->Hs, K, 0.0, 0.0, K - nr + 1, K, &meig,
                        p->wasc, p->swork, p->lswork, p->info) != CUSOLVER_STATUS_SUCCESS ||
      meig != nr)
    return fail(p, HOTRG_ECUDA, "cusolverDnDsyevdx (Rayleigh-Ritz) failed");
  CK(eigh_info_check(p->info, p->err, st));
  // Ritz vectors as rows: V[c][i] = sum_a S[a][c] Q[a][i]  (S column-major, first nr columns)
  CK(gemm_f64(g64(p, p->Hs, map_lin(K), map_lin(1), p->Qs, map_lin(1), map_lin(N), p->Zs,
                  map_lin(N), map_lin(1), nr, N, K, 1.0, 0.0),
              st, p->sms));
  return HOTRG_OK;
}

// Accuracy guard of the subspace eigensolver: the kept Ritz pairs (rows of
// Ek, values lk descending) are checked against the Gram matrix still in
// p->Escr, r = max_a ||G v_a - theta_a v_a|| / theta_1, bounded by
// residual_tol(k).  On split steps the products run on the four-plane
// tensor-core GEMM with the split of G the eigensolver made; otherwise in
// FP64.  A step over the bound sets the guard word err[2]; step_forward reads
// it (one host synchronisation per subspace step) and refines that step.
hotrg_status eigh_residual(hotrg_plan p, const StepGeom& s, int k) {
  Stage sc(p, kStEighRes);
  cudaStream_t st = p->stream;
  const int N = (int)s.N, Dp = s.Xp;
  const double* Ek = E_of(p, k);
  if (subspace_on_tc(p, s)) {
    const long long sE = round_up((long long)Dp * N, 64), sG = round_up((long long)N * N, 64);
    CK(gsplit(p, Ek, map_lin(N), map_lin(1), Dp, N, kEighPlanes, sE, p->pU));
    CK(tc_gemm(opnd(p->pU, Dp, N, kEighPlanes, sE), opnd(p->pV, N, N, kEighPlanes, sG),
               tcg(p, kEighPlanes, Dp, N, N, map_lin(N), map_lin(1), kOutF64, p->Zs, 0), st,
               p->sms));
  } else {
    CK(gemm_f64(g64(p, Ek, map_lin(N), map_lin(1), p->Escr, map_lin(N), map_lin(1), p->Zs,
                    map_lin(N), map_lin(1), Dp, N, N, 1.0, 0.0),
                st, p->sms));
  }
  CK(eig_residual(p->Zs, Ek, p->lam[k - 1], Dp, N, residual_tol(p->cfg, k), p->partial,
                  p->dres + (k - 1), p->err + 2, 1, st));
  return HOTRG_OK;
}

// Wait for the step's residual check and return (and clear) the guard word.
hotrg_status guard_fired(hotrg_plan p, bool* fired) {
  CK(cudaMemcpyAsync(p->guard_host, p->err + 2, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  *fired = *p->guard_host != 0;
  if (*fired) CK(cudaMemsetAsync(p->err + 2, 0, sizeof(int), p->stream));
  return HOTRG_OK;
}

// ---- scheme (b): the exact final product ---------------------------------
//
// Main text Fig. 1b leaves a one-dimensional structure that is contracted
// exactly.  For the depth-k chain T~_k[x][x'][y][j] (X x X x d x d) the free
// energy is evaluated as Tr[rho rho] of two copies of the chain, whose cell
// transfer operator acts on X x X matrices V as
//     (A V)[x1][x2] = sum_{y, j} sum_{x1', x2'} T[x1][x1'][y][j] V[x1'][x2'] T[x2][x2'][j][y],
// i.e. A V = sum_{y,j} T_yj V T_jy^T; the infinite chain contributes
// ln lambda_max(A) per cell, so out_k = sum_j ln c_j / 2^j + ln lambda_max / 2^(k+1).
// lambda_max and its eigenvectors come from power iteration in FP64 (two GEMMs
// per product, through the same mixed-radix index maps as the contractions).

constexpr int kChainMaxIters = 20000;   // power iterations before HOTRG_ENOTCONV
constexpr int kChainCheck = 8;          // iterations between convergence reads
constexpr double kChainTol = 1e-13;     // ||V_{i+1} - V_i||_F of unit vectors

// out = A in (left = false) or A^T in (left = true), in/out X x X row-major.
hotrg_status chain_apply(hotrg_plan p, const double* T, int X, int d, bool left, const double* in,
                         double* out) {
  cudaStream_t st = p->stream;
  const long long d2 = (long long)d * d, Xd2 = X * d2, dX = (long long)d * X;
  if (!left) {
    // Z[(x1 y j)][x2'] = sum_{x1'} T[x1][x1'][y][j] V[x1'][x2']
    CK(gemm_f64(g64(p, T, map3(d, d, 1, d, Xd2), map_lin(d2), in, map_lin(1), map_lin(X), p->chZ,
                    map_lin(X), map_lin(1), X * (int)d2, X, X, 1.0, 0.0),
                st, p->sms));
    // out[x1][x2] = sum_{x2' j y} Z[(x1 y j)][x2'] T[x2][x2'][j][y]
    CK(gemm_f64(g64(p, p->chZ, map_lin(d2 * X), map3(X, d, 1, X, dX), T, map_lin(Xd2),
                    map3(X, d, d2, d, 1), out, map_lin(X), map_lin(1), X, X, X * (int)d2, 1.0,
                    0.0),
                st, p->sms));
  } else {
    // Z[(x1' y j)][x2] = sum_{x1} T[x1][x1'][y][j] W[x1][x2]
    CK(gemm_f64(g64(p, T, map3(d, d, 1, d, d2), map_lin(Xd2), in, map_lin(1), map_lin(X), p->chZ,
                    map_lin(X), map_lin(1), X * (int)d2, X, X, 1.0, 0.0),
                st, p->sms));
    // out[x1'][x2'] = sum_{x2 j y} Z[(x1' y j)][x2] T[x2][x2'][j][y]
    CK(gemm_f64(g64(p, p->chZ, map_lin(d2 * X), map3(X, d, 1, X, dX), T, map_lin(d2),
                    map3(X, d, Xd2, d, 1), out, map_lin(X), map_lin(1), X, X, X * (int)d2, 1.0,
                    0.0),
                st, p->sms));
  }
  return HOTRG_OK;
}

// Dominant eigenvector (unit Frobenius norm) of A (or A^T) into V, ln lambda_max
// into p->scal[4].  Starts from the identity; fails with HOTRG_ENOTCONV when
// the iteration does not settle (a dominant eigenvalue that is not real,
// positive and simple).
hotrg_status chain_power(hotrg_plan p, const double* T, int X, int d, bool left, double* V) {
  cudaStream_t st = p->stream;
  const long long n = (long long)X * X;
  CK(eye_unit(V, X, st, p->sms));
  double* cur = V;
  double* nxt = p->chV;
  bool done = false;
  for (int it = 1; it <= kChainMaxIters && !done; ++it) {
    hotrg_status r = chain_apply(p, T, X, d, left, cur, nxt);
    if (r != HOTRG_OK) return r;
    CK(frob_normalize(nxt, n, p->partial, kMaxPartial, p->scal + 4, p->scal + 5, p->err, st,
                      p->sms));
    CK(diff_norm(nxt, cur, n, p->scal + 6, st));
    std::swap(cur, nxt);
    if (it % kChainCheck == 0) {
      double diff = 0;
      CK(cudaMemcpyAsync(&diff, p->scal + 6, sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (!(diff == diff)) return fail(p, HOTRG_ENONFINITE, "chain power iteration: not finite");
      done = diff < kChainTol;
    }
  }
  if (!done)
    return fail(p, HOTRG_ENOTCONV, "chain power iteration: no simple positive dominant eigenvalue");
  if (cur != V) CK(cudaMemcpyAsync(V, cur, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  return HOTRG_OK;
}

// out_k of the depth-k chain (T~_k in p->T[k]): the right eigenvector stays in
// p->chR for the backward; out_k goes to p->out (k = the run's last step) and
// to p->lnz_steps[k - 1].
hotrg_status chain_value(hotrg_plan p, int k) {
  const StepGeom& g = p->L.g[k - 1];
  hotrg_status r = chain_power(p, p->T[k], g.Xp, g.Y, false, p->chR);
  if (r != HOTRG_OK) return r;
  CK(chain_lnz(p->log_norms, k, p->scal + 4, k == p->n_run ? p->out : nullptr,
               p->lnz_steps + (k - 1), p->stream));
  return HOTRG_OK;
}

// E_n = 2^n d out_n / d T~_n = (1/2) d ln lambda / d T~_n
//     = [L T_vu R^T + L^T T_vu R][a][b] / (2 lambda <L, R>)   at [a][b][u][v],
// with R, L the right and left dominant eigenvectors (X x X) of A.
hotrg_status chain_seed(hotrg_plan p) {
  const int n = p->n_run;
  const StepGeom& g = p->L.g[n - 1];
  const int X = g.Xp, d = g.Y;
  const double* T = p->T[n];
  cudaStream_t st = p->stream;
  hotrg_status r = chain_power(p, T, X, d, true, p->chW);
  if (r != HOTRG_OK) return r;
  // the right eigenvector of the forward (the same tensor) is in p->chR
  const long long d2 = (long long)d * d, Xd2 = X * d2, dX = (long long)d * X;
  CK(dot_small(p->chW, p->chR, X * X, p->scal + 7, st));
  double h[2] = {0, 0};
  CK(cudaMemcpyAsync(&h[0], p->scal + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&h[1], p->scal + 7, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double lam = std::exp(h[0]), lr = h[1];
  if (!(lr != 0.0) || !std::isfinite(lam * lr))
    return fail(p, HOTRG_ENONFINITE, "chain seed: eigenvectors orthogonal or not finite");
  const double coef = 0.5 / (lam * lr);
  // term 1: Y[(x2 u v)][b] = sum_{x2'} T[x2][x2'][v][u] R[b][x2'];
  //         E[a][(b u v)]  = coef sum_{x2} L[a][x2] Y[(x2 u v)][b]
  CK(gemm_f64(g64(p, T, map3(d, d, d, 1, Xd2), map_lin(d2), p->chR, map_lin(X), map_lin(1),
                  p->chZ, map_lin(X), map_lin(1), X * (int)d2, X, X, 1.0, 0.0),
              st, p->sms));
  CK(gemm_f64(g64(p, p->chW, map_lin(X), map_lin(1), p->chZ, map3(d, d, X, dX, 1),
                  map_lin(d2 * X), p->Ecur, map_lin(Xd2), map3(d, d, 1, d, d2), X, X * (int)d2, X,
                  coef, 0.0),
              st, p->sms));
  // term 2: Y[(x1 u v)][b] = sum_{x1'} T[x1][x1'][v][u] R[x1'][b];
  //         E[a][(b u v)] += coef sum_{x1} L[x1][a] Y[(x1 u v)][b]
  CK(gemm_f64(g64(p, T, map3(d, d, d, 1, Xd2), map_lin(d2), p->chR, map_lin(1), map_lin(X),
                  p->chZ, map_lin(X), map_lin(1), X * (int)d2, X, X, 1.0, 0.0),
              st, p->sms));
  CK(gemm_f64(g64(p, p->chW, map_lin(1), map_lin(X), p->chZ, map3(d, d, X, dX, 1),
                  map_lin(d2 * X), p->Ecur, map_lin(Xd2), map3(d, d, 1, d, d2), X, X * (int)d2, X,
                  coef, 1.0),
              st, p->sms));
  return HOTRG_OK;
}

// Extra power iterations the guard may add to a step before it hands the
// step to the exact partial eigensolver (one iteration costs ~10 ms at
// D = 64, the exact solver ~350 ms).
constexpr int kGuardMaxIters = 4;
// w_rule 1: relative truncation errors closer than this count as a tie (left);
// where the two sides of a tensor have the same spectrum they differ by rounding.
constexpr double kWRuleTie = 1e-12;

// One forward step in three phases (the grouped forward runs each phase for
// every plan of a group, with the contractions of all plans in one launch per
// stage): the isometry (Gram matrix and eigensolve, or the given one), the
// three contractions, and the normalisation.
hotrg_status step_eigh(hotrg_plan p, int k) {
  const StepGeom& s = p->L.g[k - 1];
  cudaStream_t st = p->stream;
  const double* T = p->T[k - 1];
  double* Ek = E_of(p, k);
  double* lk = p->lam[k - 1];
  const int N = (int)s.N;
  hotrg_status r;
  if (p->cfg.w_given && k <= p->given_steps) {
    // the isometries are parameters (differentiable-TRG sweeps): no Gram, no
    // eigensolve; truncation diagnostics are not defined
    CK(set_value(p->dtrunc + (k - 1), std::nan(""), nullptr, 0, st));
    CK(set_value(p->dgap + (k - 1), std::nan(""), nullptr, 0, st));
  } else {
  if (s.split && k >= p->cfg.gram_split_from_step) r = gram_split(p, s, T, p->Escr);
  else r = gram_f64(p, s, T, p->Abuf, p->Bbuf, p->Escr);
  if (r != HOTRG_OK) return r;
  {
  Stage sc(p, kStEigh);
  CK(diag_trace(p->Escr, N, p->scal + 3, st));
  // forward only: the D'+1 largest eigenpairs (D' kept, one more for the gap)
  auto exact_partial = [&]() -> hotrg_status {
    int meig = 0;
    cusolverStatus_t cs = cusolverDnDsyevdx(p->solver, CUSOLVER_EIG_MODE_VECTOR,
                                            CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER, N,
                                            p->Escr, N, 0.0, 0.0, N - s.Xp, N, &meig, p->wasc,
                                            p->work, p->lwork, p->info);
    if (cs != CUSOLVER_STATUS_SUCCESS) return fail(p, HOTRG_ECUDA, "cusolverDnDsyevdx failed");
    return HOTRG_OK;
  };
  auto finish = [&](const double* evec, int ncols) -> hotrg_status {
    CK(eigh_info_check(p->info, p->err, st));
    if (g_inj_what.load() == kInjEigh && g_inj_arg.load() == k)
      CK(set_value(nullptr, 0.0, p->err, kErrEigh, st));
    // all N pairs where the backward's eigensolve adjoint needs the discarded
    // ones and the solver returned them; the D' kept ones otherwise
    CK(eig_desc(evec, p->wasc, N, ncols, (p->cfg.want_grad && ncols >= N) ? N : s.Xp, Ek, lk,
                st));
    CK(eig_diag(lk, ncols, N, s.Xp, p->scal + 3, p->dtrunc + (k - 1), p->dgap + (k - 1), st));
    return HOTRG_OK;
  };
  if (use_subspace(p, s)) {
    // randomized subspace eigensolver, checked on the device; where the check
    // fails, up to kGuardMaxIters more power iterations, then the exact solver
    int iters = p->cfg.eigh_power_iters > 0 ? p->cfg.eigh_power_iters : 4;
    const double* warm = nullptr;
    if (p->cfg.eigh_warm_start > 0 && k >= 3 && p->wkeep[k & 1] &&
        p->wkeep_n[k & 1] == N && p->wkeep_xp[k & 1] == s.Xp) {
      warm = p->wkeep[k & 1];
      iters = p->cfg.eigh_warm_start;
    }
    if ((r = eigh_subspace(p, s, k, iters, false, warm)) != HOTRG_OK) return r;
    if ((r = finish(p->Zs, subspace_ritz(s))) != HOTRG_OK) return r;
    if ((r = eigh_residual(p, s, k)) != HOTRG_OK) return r;
    bool fired = false;
    if ((r = guard_fired(p, &fired)) != HOTRG_OK) return r;
    if (fired) ++p->fallbacks;
    int extra = 0;
    while (fired && extra < kGuardMaxIters) {
      ++extra;
      if ((r = eigh_subspace(p, s, k, 1, true)) != HOTRG_OK) return r;
      if ((r = finish(p->Zs, subspace_ritz(s))) != HOTRG_OK) return r;
      if ((r = eigh_residual(p, s, k)) != HOTRG_OK) return r;
      if ((r = guard_fired(p, &fired)) != HOTRG_OK) return r;
    }
    p->guard_iters[k - 1] = extra;
    if (fired) {
      p->exact_step[k - 1] = 1;
      if ((r = exact_partial()) != HOTRG_OK) return r;
      if ((r = finish(p->Escr, s.Xp + 1)) != HOTRG_OK) return r;
      CK(set_value(p->dres + (k - 1), std::nan(""), nullptr, 0, st));
    }
  } else {
    int ncols = N;
    if (p->cfg.want_grad || s.Xp >= N) {
      // all eigenpairs (the backward's eigensolve adjoint needs the discarded ones)
      cusolverStatus_t cs = cusolverDnDsyevd(p->solver, CUSOLVER_EIG_MODE_VECTOR,
                                             CUBLAS_FILL_MODE_LOWER, N, p->Escr, N, p->wasc,
                                             p->work, p->lwork, p->info);
      if (cs != CUSOLVER_STATUS_SUCCESS) return fail(p, HOTRG_ECUDA, "cusolverDnDsyevd failed");
    } else {
      if ((r = exact_partial()) != HOTRG_OK) return r;
      ncols = s.Xp + 1;
    }
    if ((r = finish(p->Escr, ncols)) != HOTRG_OK) return r;
    CK(set_value(p->dres + (k - 1), std::nan(""), nullptr, 0, st));
    if (p->cfg.w_rule == 1 && s.Xp < N) {
      // Xie2012: the HOSVD along the right bond too; the side that discards
      // less (relative to the common trace) gives w, the left one on a tie
      if (s.split && k >= p->cfg.gram_split_from_step) r = gram_split(p, s, T, p->Escr, true);
      else r = gram_f64(p, s, T, p->Abuf, p->Bbuf, p->Escr, true);
      if (r != HOTRG_OK) return r;
      if (p->cfg.want_grad || s.Xp >= N) {
        cusolverStatus_t cs = cusolverDnDsyevd(p->solver, CUSOLVER_EIG_MODE_VECTOR,
                                               CUBLAS_FILL_MODE_LOWER, N, p->Escr, N, p->wasc,
                                               p->work, p->lwork, p->info);
        if (cs != CUSOLVER_STATUS_SUCCESS) return fail(p, HOTRG_ECUDA, "cusolverDnDsyevd failed");
      } else if ((r = exact_partial()) != HOTRG_OK) {
        return r;
      }
      CK(eigh_info_check(p->info, p->err, st));
      const int rows = (p->cfg.want_grad && ncols >= N) ? N : s.Xp;
      CK(eig_desc(p->Escr, p->wasc, N, ncols, rows, p->Er, p->lamR, st));
      CK(eig_diag(p->lamR, ncols, N, s.Xp, p->scal + 3, p->trR, p->trR + 1, st));
      CK(w_rule_choose(p->dtrunc + (k - 1), p->trR, kWRuleTie, p->side_dev + (k - 1), st));
      const int* f = p->side_dev + (k - 1);
      CK(cond_copy(f, p->Er, Ek, (long long)rows * N, st, p->sms));
      CK(cond_copy(f, p->lamR, lk, ncols, st, p->sms));
      CK(cond_copy(f, p->trR, p->dtrunc + (k - 1), 1, st, p->sms));
      CK(cond_copy(f, p->trR + 1, p->dgap + (k - 1), 1, st, p->sms));
    }
  }
  if (p->wkeep[k & 1]) {
    // this step's kept eigenvectors: the warm start of step k + 2
    CK(cudaMemcpyAsync(p->wkeep[k & 1], Ek, sizeof(double) * (size_t)s.Xp * N,
                       cudaMemcpyDeviceToDevice, st));
    p->wkeep_n[k & 1] = N;
    p->wkeep_xp[k & 1] = s.Xp;
  }
  }
  }
  return HOTRG_OK;
}

hotrg_status step_contract(hotrg_plan p, int k) {
  const StepGeom& s = p->L.g[k - 1];
  if (s.split) return contract_split(p, s, p->T[k - 1], E_of(p, k), p->T[k]);
  return contract_f64(p, s, p->T[k - 1], E_of(p, k), p->T[k]);
}

hotrg_status step_finish(hotrg_plan p, int k) {
  const StepGeom& s = p->L.g[k - 1];
  cudaStream_t st = p->stream;
  double* Tout = p->T[k];
  const long long n_out = (long long)s.Y * s.Y * s.Xp * s.Xp;
  if (g_inj_what.load() == kInjNaN && g_inj_arg.load() == k)
    CK(set_value(Tout, std::nan(""), nullptr, 0, st));
  {
  Stage sc(p, kStNorm);
  CK(frob_normalize(Tout, n_out, p->partial, kMaxPartial, p->log_norms + (k - 1), p->scal, p->err,
                    st, p->sms));
  }
  if (p->cfg.scheme == 1) {
    // scheme (b): no re-orientation, the next step merges vertically again
    CK(swap_pairs(Tout, p->Abuf, s.Y, s.Xp, st, p->sms));
    CK(cudaMemcpyAsync(Tout, p->Abuf, sizeof(double) * n_out, cudaMemcpyDeviceToDevice, st));
    if (p->cfg.chain_steps && k < p->n_run) return chain_value(p, k);
  }
  return HOTRG_OK;
}

hotrg_status step_forward(hotrg_plan p, int k) {
  hotrg_status r = step_eigh(p, k);
  if (r == HOTRG_OK) r = step_contract(p, k);
  if (r == HOTRG_OK) r = step_finish(p, k);
  return r;
}

hotrg_status forward_begin(hotrg_plan p) {
  cudaStream_t st = p->stream;
  if (p->cfg.w_given && std::min(p->given_steps, p->n_run) > p->w_valid)
    return fail(p, HOTRG_ESTATE, "w_given plan: load the isometries first");
  p->have_bwd = false;
  p->guard_iters.assign(p->cfg.n_steps, 0);
  p->wkeep_n[0] = p->wkeep_n[1] = 0;   // no warm start across forwards
  p->exact_step.assign(p->cfg.n_steps, 0);
  if (p->lnz_steps) CK(cudaMemsetAsync(p->lnz_steps, 0xff, sizeof(double) * p->cfg.n_steps, st));
  return HOTRG_OK;
}

hotrg_status forward_end(hotrg_plan p);

hotrg_status run_forward(hotrg_plan p) {
  hotrg_status r = forward_begin(p);
  if (r != HOTRG_OK) return r;
  for (int k = 1; k <= p->n_run; ++k) {
    r = step_forward(p, k);
    if (r != HOTRG_OK) return r;
  }
  return forward_end(p);
}

hotrg_status forward_end(hotrg_plan p) {
  cudaStream_t st = p->stream;
  // steps past given_steps of a w_given plan have just formed their isometries
  if (p->cfg.w_given && p->n_run > p->w_valid) p->w_valid = p->n_run;
  if (p->cfg.scheme == 1) return chain_value(p, p->n_run);
  const StepGeom& last = p->L.g[p->n_run - 1];
  CK(trace_lnz(p->T[p->n_run], last.Y, last.Xp, p->log_norms, p->n_run, p->out,
               p->scal + 1, p->err, st));
  return HOTRG_OK;
}

// ---- backward pieces ------------------------------------------------------

// One contraction of the backward: on the tensor cores (grid-aligned split of
// both operands from their FP64 sources through the same index maps, FP64
// output, optional accumulation) when the step runs split and the operands fit
// the plane buffers, else on the FP64 GEMM.
// f32 flags: bit 0 / 1 / 2 = A / B / C is an FP32 staging buffer (passed as a
// double pointer), which only the tensor-core path can read or write.
enum : unsigned { kA32 = 1, kB32 = 2, kC32 = 4 };

cudaError_t run_gemm(hotrg_plan p, int np, const GemmF64& g, unsigned f32 = 0) {
  const bool split = np > 0;
  const long long cap = p->L.chunkS;
  const bool ok = split && p->L.any_split && g.K % 8 == 0 && (g.beta == 0.0 || g.beta == 1.0) &&
                  (long long)g.M * g.K <= cap && (long long)g.N * g.K <= cap && g.K > 0;
  if (!ok) {
    if (f32) return cudaErrorInvalidValue;   // FP32 staging needs the tensor-core path
    return gemm_f64(g, p->stream, p->sms);
  }
  cudaError_t e;
  if (f32 & kA32) {
    const float* a = reinterpret_cast<const float*>(g.A);
    e = grid_split(a, lim_of(p, a, sizeof(float)), g.am, g.ak, g.M, g.K, np, cap, p->pU, p->err,
                   p->stream, p->sms);
  } else {
    e = grid_split(g.A, g.a_lim, g.am, g.ak, g.M, g.K, np, cap, p->pU, p->err, p->stream, p->sms);
  }
  if (e != cudaSuccess) return e;
  if (f32 & kB32) {
    const float* b = reinterpret_cast<const float*>(g.B);
    e = grid_split(b, lim_of(p, b, sizeof(float)), g.bn, g.bk, g.N, g.K, np, cap, p->pV, p->err,
                   p->stream, p->sms);
  } else {
    e = grid_split(g.B, g.b_lim, g.bn, g.bk, g.N, g.K, np, cap, p->pV, p->err, p->stream, p->sms);
  }
  if (e != cudaSuccess) return e;
  TcGemm t = tcg(p, np, g.M, g.N, g.K, g.cm, g.cn, (f32 & kC32) ? kOutF32 : kOutF64, g.C, 0);
  t.alpha = (float)g.alpha;
  t.accumulate = g.beta != 0.0 ? 1 : 0;
  return tc_gemm(opnd(p->pU, g.M, g.K, np, cap), opnd(p->pV, g.N, g.K, np, cap), t, p->stream,
                 p->tc_sms);
}

hotrg_status step_backward(hotrg_plan p, int k) {
  const StepGeom& s = p->L.g[k - 1];
  const bool sp = s.split;
  const int snp = s.np;
  // three-plane steps keep the D^5 intermediates U, V, P, Q in FP32 (they are
  // split into 24 bits anyway); FP64 steps and four-plane steps keep FP64
  const unsigned f = (snp == 3) ? 1u : 0u;
  const int X = s.X, Y = s.Y, Xp = s.Xp;
  const long long N = s.N, XY = (long long)X * Y, Y2 = (long long)Y * Y, XY2 = XY * Y;
  const long long Xp2 = (long long)Xp * Xp, X2 = (long long)X * X, YXp2 = (long long)Y * Xp2;
  cudaStream_t st = p->stream;
  const double* T = p->T[k - 1];
  const double* Ek = E_of(p, k);
  const double* lk = p->lam[k - 1];
  if (p->cfg.scheme == 1) {
    // scheme (b) keeps T~_k (and so E_k) as [a][b][y][y']: bring E_k into the
    // [y][y'][a][b] layout of the step's output index maps
    CK(swap_pairs(p->Ecur, p->Enext, Xp, Y, st, p->sms));
    double* t = p->Ecur;
    p->Ecur = p->Enext;
    p->Enext = t;
  }
  double* Eb = p->Ecur;                    // 2^k dL/dT~_k, stored layout [y][y'][a][b]
  CK(scale_exp_neg(Eb, Y2 * Xp2, p->log_norms + (k - 1), st, p->sms));   // -> dL/dT' (x 2^k)
  CK(cudaMemsetAsync(p->Tbar, 0, sizeof(double) * X2 * Y2, st));
  CK(cudaMemsetAsync(p->wbT, 0, sizeof(double) * Xp * N, st));
  {
  Stage sc(p, kStBwdContract + (sp ? 0 : kStF64));
  for (int y0 = 0; y0 < Y; y0 += s.yc64) {
    const int yc = (Y - y0) < s.yc64 ? (Y - y0) : s.yc64;
    const double* Ty = T + (long long)y0 * Y;
    const double* Eby = Eb + (long long)y0 * YXp2;
    // recompute U and V of this chunk (as in the forward)
    CK(run_gemm(p, snp, g64(p, Ek, map2(X, 1, N), map_lin(X), Ty, map3(Y, X, 1, Y2, Y), map_lin(XY2), p->Ub,
                    map2(X, Y, XY), map3(Y, X, 1, Xp * XY, X * Xp * XY), Xp * X, yc * X * Y, X,
                    1.0, 0.0), f * kC32));
    CK(run_gemm(p, snp, g64(p, p->Ub, map_lin(XY), map_lin(1), T, map2(X, Y2, 1), map2(Y, Y, XY2), p->Vb,
                    map3(Xp, X, Y * X2, X, Xp * Y * X2), map2(X, 1, X2), yc * X * Xp, Y * X,
                    X * Y, 1.0, 0.0), f * (kA32 | kC32)));
    // P[(y a i)][(k z)] = sum_b Tbar'[a b y z] w[i k b]
    CK(run_gemm(p, snp, g64(p, Eby, map3(Y, Xp, Xp2, Xp, YXp2), map_lin(1), Ek, map_lin(1), map_lin(N),
                    p->Pb, map3(Y, Xp, 1, X2 * Y, (long long)Xp * X2 * Y), map2(X, Y, XY),
                    yc * Xp * Y, X * X, Xp, 1.0, 0.0), f * kC32));
    // Q[(y a i)][(b j)] = sum_{k z} P T[b k j z]
    CK(run_gemm(p, snp, g64(p, p->Pb, map_lin(XY), map_lin(1), T, map2(Y, Y, XY2), map2(Y, 1, Y2), p->Qb,
                    map_lin(XY), map_lin(1), yc * Xp * X, X * Y, X * Y, 1.0, 0.0), f * (kA32 | kC32)));
    // upper copy: Tbar[a i y j] += sum_{A b} w[a b A] Q[y A i b j]
    CK(run_gemm(p, snp, g64(p, Ek, map_lin(X), map2(X, 1, N), p->Qb, map3(Y, X, 1, XY, (long long)Xp * X * XY),
                    map2(X, Y, X * XY), p->Tbar + (long long)y0 * Y, map_lin(XY2),
                    map3(Y, X, 1, Y2, Y), X, yc * X * Y, Xp * X, 1.0, 1.0), f * kB32));
    // lower copy: Tbar[b k j z] += sum_{y i A} U[y i A b j] P[y A z i k]
    CK(run_gemm(p, snp, g64(p, p->Ub, map2(Y, 1, Y), map3(Xp, X, XY, Xp * XY, (long long)X * Xp * XY), p->Pb,
                    map2(Y, 1, Y), map3(Xp, X, X * XY, XY, (long long)Xp * X * XY), p->Tbar,
                    map2(Y, Y, XY2), map2(Y, 1, Y2), X * Y, X * Y, yc * X * Xp, 1.0, 1.0), f * (kA32 | kB32)));
    // w carrying alpha: wbT[A][(a b)] += sum_{y i j} T[a i y j] Q[y A i b j]
    CK(run_gemm(p, snp, g64(p, Ty, map_lin(XY2), map3(Y, X, 1, Y2, Y), p->Qb, map2(X, Y, X * XY),
                    map3(Y, X, 1, XY, (long long)Xp * X * XY), p->wbT, map_lin(X), map2(X, 1, N),
                    X, Xp * X, yc * X * Y, 1.0, 1.0), f * kB32));
    // w carrying beta: wbT[B][(i k)] += sum_{y A z} V[y A z][(i k)] Tbar'[A B y z]
    CK(run_gemm(p, snp, g64(p, p->Vb, map_lin(1), map3(Y, Xp, X2, Y * X2, (long long)Xp * Y * X2), Eby,
                    map_lin(1), map3(Y, Xp, Xp2, Xp, YXp2), p->wbT, map_lin(1), map_lin(N),
                    X * X, Xp, yc * Xp * Y, 1.0, 1.0), f * kA32));
  }
  }
  if (!p->cfg.fixed_w_grad && Xp < N) {
    Stage sc(p, kStBwdEigh + (sp ? 0 : kStF64));
    long long sl, sr;
    lr_strides(s, p->side_host.size() >= (size_t)k && p->side_host[k - 1] != 0, sl, sr);
    const int nd = (int)(N - Xp);
    const double* Ud = Ek + (long long)Xp * N;
    // S[j][k] = sum_i U_d[i][j] wbar[i][k]
    CK(gemm_f64(g64(p, Ud, map_lin(N), map_lin(1), p->wbT, map_lin(N), map_lin(1), p->Sb,
                    map_lin(Xp), map_lin(1), nd, Xp, (int)N, 1.0, 0.0),
                st, p->sms));
    double eta = p->cfg.eigh_broadening > 0 ? p->cfg.eigh_broadening : 1e-12;
    CK(eigh_adj_scale(p->Sb, nd, Xp, lk, eta, st, p->sms));
    // H[i][k] = sum_j U_d[i][j] FS[j][k];  Gbar[i][i'] = sum_k H[i][k] U_k[i'][k]
    CK(gemm_f64(g64(p, Ud, map_lin(1), map_lin(N), p->Sb, map_lin(1), map_lin(Xp), p->Hb,
                    map_lin(Xp), map_lin(1), (int)N, Xp, nd, 1.0, 0.0),
                st, p->sms));
    CK(gemm_f64(g64(p, p->Hb, map_lin(Xp), map_lin(1), Ek, map_lin(1), map_lin(N), p->Gb,
                    map_lin(N), map_lin(1), (int)N, (int)N, Xp, 1.0, 0.0),
                st, p->sms));
    CK(symmetrize(p->Gb, (int)N, st, p->sms));
    {
      // Gram halves again (A, B of the forward, of the side that gave w), FP64 output
      const long long XY2g = (long long)X * Y * Y, Y2g = (long long)Y * Y;
      CK(run_gemm(p, snp, g64(p, T, map2(Y, 1, sl), map2(Y, Y, sr), T, map2(Y, 1, sl),
                             map2(Y, Y, sr), p->Abuf, map2(Y, Y, XY2g), map2(Y, 1, Y2g), X * Y,
                             X * Y, X * Y, 1.0, 0.0)));
      CK(run_gemm(p, snp, g64(p, T, map2(Y, Y, sl), map2(Y, 1, sr), T, map2(Y, Y, sl),
                             map2(Y, 1, sr), p->Bbuf, map2(Y, Y, XY2g), map2(Y, 1, Y2g), X * Y,
                             X * Y, X * Y, 1.0, 0.0)));
    }
    const long long X3 = X2 * X;
    // Abar[(x1 x1'')][(j j')] = sum_{x2 x2''} Gbar[x1 x2 x1'' x2''] B[(x2 x2'')][(j j')]
    CK(run_gemm(p, snp, g64(p, p->Gb, map2(X, X, X3), map2(X, 1, X2), p->Bbuf, map_lin(1), map_lin(Y2),
                    p->Abar, map_lin(Y2), map_lin(1), X * X, Y * Y, X * X, 1.0, 0.0)));
    CK(run_gemm(p, snp, g64(p, p->Gb, map2(X, 1, X2), map2(X, X, X3), p->Abuf, map_lin(1), map_lin(Y2),
                    p->Bbar, map_lin(Y2), map_lin(1), X * X, Y * Y, X * X, 1.0, 0.0)));
    // Tbar[a i y j] += 2 sum_{c k} Abar[a j c k] T[c i y k]   (l, r strides of the side)
    CK(run_gemm(p, snp, g64(p, p->Abar, map2(Y, Y, X * Y2), map2(Y, 1, Y2), T, map2(Y, Y, sr),
                    map2(Y, 1, sl), p->Tbar, map2(Y, 1, sl), map2(Y, Y, sr), X * Y, X * Y, X * Y,
                    2.0, 1.0)));
    // Tbar[b k j z] += 2 sum_{d m} Bbar[b j d m] T[d k m z]
    CK(run_gemm(p, snp, g64(p, p->Bbar, map2(Y, Y, XY2), map2(Y, 1, Y2), T, map2(Y, 1, sr),
                    map2(Y, Y, sl), p->Tbar, map2(Y, Y, sl), map2(Y, 1, sr), X * Y, X * Y, X * Y,
                    2.0, 1.0)));
  }
  // d(ln Z/N)/d w_k = wbT / 2^k (wbT carries the 2^k of E_k)
  if (p->wbar_all)
    CK(scale_copy(p->wbT, p->wbar_all + p->w_off[k - 1], (long long)Xp * N, std::ldexp(1.0, -k), st,
                  p->sms));
  // E_{k-1} = (1/2) Tbar (average of the two copies), in the layout of T_{k-1}
  CK(scale_copy(p->Tbar, p->Enext, X2 * Y2, 0.5, st, p->sms));
  double* tmp = p->Ecur;
  p->Ecur = p->Enext;
  p->Enext = tmp;
  return HOTRG_OK;
}

hotrg_status run_backward(hotrg_plan p) {
  const StepGeom& last = p->L.g[p->n_run - 1];
  if (p->side_dev) {
    p->side_host.assign(p->cfg.n_steps, 0);
    CK(cudaMemcpyAsync(p->side_host.data(), p->side_dev, sizeof(int) * p->n_run,
                       cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
  }
  if (p->cfg.scheme == 1) {
    hotrg_status r = chain_seed(p);
    if (r != HOTRG_OK) return r;
  } else {
    CK(seed_trace_adjoint(p->Ecur, last.Y, last.Xp, p->scal + 1, p->stream, p->sms));
  }
  for (int k = p->n_run; k >= 1; --k) {
    hotrg_status r = step_backward(p, k);
    if (r != HOTRG_OK) return r;
  }
  return HOTRG_OK;
}

hotrg_status device_status(hotrg_plan p, const int* w) {
  // the first failure recorded is the root cause; report it first
  const int e = w[1] ? w[1] : w[0];
  if (e & kErrTimeout) return fail(p, HOTRG_ETIMEOUT, "device wait timed out");
  if (e & kErrEigh) return fail(p, HOTRG_ENOTCONV, "eigensolver did not converge");
  if (e & kErrNonFinite) return fail(p, HOTRG_ENONFINITE, "norm or trace not finite");
  if (e & kErrBounds) return fail(p, HOTRG_ECUDA, "a kernel index check failed (access skipped)");
  if (e) return fail(p, HOTRG_ECUDA, "device error word set");
  return HOTRG_OK;
}

hotrg_status finish_sync(hotrg_plan p) {
  CK(cudaStreamSynchronize(p->stream));
  int w[2] = {0, 0};
  CK(cudaMemcpy(w, p->err, 2 * sizeof(int), cudaMemcpyDeviceToHost));
  return device_status(p, w);
}


// ---- grouped forward -------------------------------------------------------
//
// Several plans of the same shape run their forwards in lockstep on one
// stream: per step, each plan forms its isometry (Gram matrix, eigensolve),
// then the three contractions of all plans go out as ONE grouped tensor-core
// launch per stage (TcGemm::batch: problem b's operand rows at b * pitch of
// the group's buffers), then each plan normalises.  The group owns the batched
// operand buffers ([plane][problem][rows][K], each problem's rows padded to the
// 128-row tile where it is the first operand).  Results are bit-identical to
// each plan's own forward: the same kernels do the same arithmetic per problem.

struct GroupGeom {
  long long pW1, pT1, pP, pW3, pU, pV, pT;   // per-problem elements (padded rows x K)
  int aW1, aU, aV;                           // padded first-operand rows
};

GroupGeom group_geom(const StepGeom& s) {
  const long long X = s.X, Y = s.Y, Xp = s.Xp;
  GroupGeom g;
  g.aW1 = (int)round_up(Xp * X, 128);
  g.aU = (int)round_up(Y * X * Xp, 128);
  g.aV = (int)round_up(Y * Xp * Y, 128);
  g.pW1 = (long long)g.aW1 * X;
  g.pT1 = Y * X * Y * X;
  g.pP = Y * X * X * Y;
  g.pW3 = Xp * X * X;
  g.pU = (long long)g.aU * X * Y;
  g.pV = (long long)g.aV * X * X;
  g.pT = Y * Y * Xp * Xp;
  return g;
}

// A split step the group can run as grouped launches: the whole free leg in
// one chunk (small bond dimensions), so that every stage is one GEMM per plan.
bool groupable(const StepGeom& s) { return s.split && s.ycs >= s.Y; }

}  // namespace

struct hotrg_group_s {
  Layout L;
  int max_count = 0, np = 0;
  long long sW1 = 0, sT1 = 0, sP = 0, sW3 = 0, sU = 0, sV = 0, nT = 0, nF = 0;  // plane strides
  cudaStream_t stream = nullptr;
  std::vector<void*> allocs;
  __nv_bfloat16 *W1 = nullptr, *T1 = nullptr, *P = nullptr, *W3 = nullptr, *U = nullptr,
                *V = nullptr;
  float* F32 = nullptr;
  double* F64 = nullptr;
  double* Tg = nullptr;
  unsigned long long grouped_launches = 0;
  std::vector<cudaEvent_t> ev;     // per plan slot: its operands are prepared
  cudaEvent_t ev_done = nullptr;   // the grouped contractions of a step are issued
};

namespace {

TcOperand gopnd(const __nv_bfloat16* ptr, int count, int pitch_rows, int K, int np,
                long long stride) {
  return opnd(ptr, count * pitch_rows, K, np, stride);
}

// Operand preparation of plan q for its place `slot` of a grouped step k, on
// the plan's own stream: the four bf16-split operands of the three stages,
// written into the group's batched buffers.
hotrg_status group_prep(hotrg_group g, hotrg_plan q, int slot, int k) {
  hotrg_plan p = q;   // the plan errors are reported on
  const StepGeom& s = q->L.g[k - 1];
  const int X = s.X, Y = s.Y, Xp = s.Xp, np = s.np;
  const long long N = s.N, Y2 = (long long)Y * Y, XY2 = (long long)X * Y * Y;
  const GroupGeom gg = group_geom(s);
  Stage sc(q, kStPrep);
  const double* Ek = E_of(q, k);
  const double* T = q->T[k - 1];
  CK(gsplit(q, Ek, map2(X, 1, N), map_lin(X), Xp * X, X, np, g->sW1, g->W1 + slot * gg.pW1));
  CK(gsplit(q, T, map3(Y, X, 1, Y2, Y), map_lin(XY2), Y * X * Y, X, np, g->sT1,
            g->T1 + slot * gg.pT1));
  CK(gsplit(q, T, map2(X, Y2, 1), map2(Y, Y, XY2), Y * X, X * Y, np, g->sP, g->P + slot * gg.pP));
  CK(gsplit(q, Ek, map_lin(N), map_lin(1), Xp, X * X, np, g->sW3, g->W3 + slot * gg.pW3));
  return HOTRG_OK;
}

// The three contractions of step k of every plan in `ps` (prepared by
// group_prep) as one grouped launch per stage on the group's stream (mirrors
// contract_split for a single chunk), then each plan's new tensor copied home.
hotrg_status group_gemms(hotrg_group g, hotrg_plan* ps, int cnt, int k) {
  hotrg_plan p = ps[0];
  const StepGeom& s = p->L.g[k - 1];
  const int X = s.X, Y = s.Y, Xp = s.Xp, np = s.np;
  const long long XY = (long long)X * Y;
  const long long Xp2 = (long long)Xp * Xp, X2 = (long long)X * X;
  cudaStream_t st = g->stream;
  const GroupGeom gg = group_geom(s);
  const bool fuse = np == 3 && p->cfg.epilogue_split != 0;
  int p1r = 0, p1h = 0, p2r = 0, p2h = 0;
  const bool fuse1 = fuse && (Xp * X) % 128 == 0 && (XY % 128) == 0 && X % 2 == 0 &&
                     seg_partner(Y, 1, p1r, p1h);
  const bool fuse2 = fuse && (Y * X) % 128 == 0 && (X2 % 128) == 0 && seg_partner(X, Xp, p2r, p2h);
  auto staged = [&](int npl) -> void* {
    return npl == 4 ? static_cast<void*>(g->F64) : static_cast<void*>(g->F32);
  };
  auto batch = [&](TcGemm& t, int a_pitch, int b_pitch, long long c_batch, long long c_lim) {
    t.batch = cnt;
    t.a_pitch = a_pitch;
    t.b_pitch = b_pitch;
    t.c_batch = c_batch;
    t.c_lim = c_lim;
  };
  auto split_staged = [&](long long per, int rows, int K, long long plane, __nv_bfloat16* dst)
      -> cudaError_t {
    for (int i = 0; i < cnt; ++i) {
      const long long off = i * per;
      cudaError_t e = np == 4
          ? grid_split(g->F64 + off, g->nF - off, map_lin(K), map_lin(1), rows, K, np, plane,
                       dst + off, p->err, st, p->sms)
          : grid_split(g->F32 + off, g->nF - off, map_lin(K), map_lin(1), rows, K, np, plane,
                       dst + off, p->err, st, p->sms);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  // S1: U[(y x1' a)][(x2 j)] of every plan
  TcGemm g1 = tcg(p, np, Xp * X, Y * X * Y, X, map2(X, Y, XY), map3(Y, X, 1, Xp * XY, X * Xp * XY),
                  fuse1 ? kOutGridSplit : stage_mode(np), fuse1 ? (void*)g->U : staged(np),
                  fuse1 ? g->sU : 0);
  g1.m_fast = 1;
  g1.seg_prow = p1r;
  g1.seg_phalf = p1h;
  batch(g1, gg.aW1, Y * X * Y, gg.pU, fuse1 ? g->sU : g->nF);
  CK(tc_gemm(gopnd(g->W1, cnt, gg.aW1, X, np, g->sW1), gopnd(g->T1, cnt, Y * X * Y, X, np, g->sT1),
             g1, st, p->tc_sms));
  ++g->grouped_launches;
  if (!fuse1) CK(split_staged(gg.pU, Y * X * Xp, X * Y, g->sU, g->U));
  // S2: V[(y a y')][(x1' x2')] of every plan
  TcGemm g2 = tcg(p, np, Y * X * Xp, Y * X, X * Y, map3(Xp, X, Y * X2, X, Xp * Y * X2),
                  map2(X, 1, X2), fuse2 ? kOutGridSplit : stage_mode(np),
                  fuse2 ? (void*)g->V : staged(np), fuse2 ? g->sV : 0);
  g2.seg_prow = p2r;
  g2.seg_phalf = p2h;
  g2.n_group = stage2_group(p->cfg);
  batch(g2, gg.aU, Y * X, gg.pV, fuse2 ? g->sV : g->nF);
  CK(tc_gemm(gopnd(g->U, cnt, gg.aU, X * Y, np, g->sU), gopnd(g->P, cnt, Y * X, X * Y, np, g->sP),
             g2, st, p->tc_sms));
  ++g->grouped_launches;
  if (!fuse2) CK(split_staged(gg.pV, Y * Xp * Y, X * X, g->sV, g->V));
  // S3: T'[y][y'][a][b] of every plan into the group's buffer, then home
  TcGemm g3 = tcg(p, np, Y * Xp * Y, Xp, X * X, map3(Y, Xp, Xp2, Xp, Y * Xp2), map_lin(1), kOutF64,
                  g->Tg, 0);
  batch(g3, gg.aV, Xp, gg.pT, g->nT);
  CK(tc_gemm(gopnd(g->V, cnt, gg.aV, X * X, np, g->sV), gopnd(g->W3, cnt, Xp, X * X, np, g->sW3),
             g3, st, p->tc_sms));
  ++g->grouped_launches;
  for (int i = 0; i < cnt; ++i)
    CK(cudaMemcpyAsync(ps[i]->T[k], g->Tg + i * gg.pT, sizeof(double) * gg.pT,
                       cudaMemcpyDeviceToDevice, st));
  return HOTRG_OK;
}

// A reusable barrier for the group's host threads.
struct Barrier {
  std::mutex m;
  std::condition_variable cv;
  int n, count = 0;
  unsigned gen = 0;
  explicit Barrier(int n_) : n(n_) {}
  void wait() {
    std::unique_lock<std::mutex> l(m);
    const unsigned my = gen;
    if (++count == n) {
      count = 0;
      ++gen;
      cv.notify_all();
    } else {
      cv.wait(l, [&] { return gen != my; });
    }
  }
};

hotrg_status group_check(hotrg_group g, hotrg_plan* ps, int cnt) {
  if (!g || !ps || cnt < 1 || cnt > g->max_count) return HOTRG_EINVAL;
  for (int i = 0; i < cnt; ++i) {
    hotrg_plan q = ps[i];
    if (!q) return HOTRG_EINVAL;
    if (q->cfg.scheme != 0 || q->cfg.w_given || q->cfg.w_rule != 0 ||
        q->L.g.size() != g->L.g.size() || q->cfg.epilogue_split != ps[0]->cfg.epilogue_split ||
        q->cfg.stage2_n_group != ps[0]->cfg.stage2_n_group ||
        q->cfg.gemm_sm_reserve != ps[0]->cfg.gemm_sm_reserve)
      return fail(q, HOTRG_EINVAL, "grouped forward: plan shape differs from the group's");
    for (size_t j = 0; j < g->L.g.size(); ++j) {
      const StepGeom &a = q->L.g[j], &b = g->L.g[j];
      if (a.X != b.X || a.Y != b.Y || a.Xp != b.Xp || a.split != b.split || a.np != b.np ||
          a.ycs != b.ycs)
        return fail(q, HOTRG_EINVAL, "grouped forward: plan shape differs from the group's");
    }
    for (int j = 0; j < i; ++j)
      if (ps[j] == q) return fail(q, HOTRG_EINVAL, "grouped forward: a plan appears twice");
  }
  return HOTRG_OK;
}

// Lockstep forward of the plans (T0 already in each plan's T[0]).  One host
// thread per plan issues its work on the plan's own stream, so the plans'
// eigensolves (and their guards' host reads) overlap; per grouped step the
// threads meet twice: after each has formed its isometry and prepared its
// operands (an event on its stream), the first thread issues the grouped
// contractions on the group's stream after all those events; after them (one
// event) each plan normalises on its own stream.
hotrg_status group_run(hotrg_group g, hotrg_plan* ps, int cnt) {
  int kmax = 0;
  for (int i = 0; i < cnt; ++i) {
    hotrg_plan q = ps[i];
    q->have_fwd = false;
    CK2(q, cudaMemsetAsync(q->err, 0, 3 * sizeof(int), q->stream));
    hotrg_status r = forward_begin(q);
    if (r != HOTRG_OK) return r;
    kmax = std::max(kmax, q->n_run);
  }
  // the grouped work of step k must follow the copy-in and set-up above on
  // every plan's stream
  std::vector<hotrg_status> st(cnt, HOTRG_OK);
  hotrg_status lead = HOTRG_OK;
  std::atomic<bool> failed{false};
  Barrier bar(cnt);
  auto active_of = [&](int k, std::vector<int>& act) {
    act.clear();
    for (int i = 0; i < cnt; ++i)
      if (ps[i]->n_run >= k) act.push_back(i);
  };
  auto body = [&](int i) {
    hotrg_plan q = ps[i];
    std::vector<int> act;
    for (int k = 1; k <= kmax; ++k) {
      active_of(k, act);
      const bool grouped = act.size() > 1 && groupable(g->L.g[k - 1]);
      const bool mine = q->n_run >= k;
      if (mine && !failed.load()) {
        hotrg_status r = step_eigh(q, k);
        if (r == HOTRG_OK && grouped) {
          const int slot = (int)(std::find(act.begin(), act.end(), i) - act.begin());
          r = group_prep(g, q, slot, k);
          if (r == HOTRG_OK && cudaEventRecord(g->ev[i], q->stream) != cudaSuccess)
            r = fail(q, HOTRG_ECUDA, "cudaEventRecord failed");
        }
        if (r == HOTRG_OK && !grouped) r = step_contract(q, k);
        if (r != HOTRG_OK) {
          st[i] = r;
          failed = true;
        }
      }
      if (grouped) {
        bar.wait();
        if (i == 0 && !failed.load()) {
          hotrg_status r = HOTRG_OK;
          for (int j : act)
            if (cudaStreamWaitEvent(g->stream, g->ev[j], 0) != cudaSuccess)
              r = fail(ps[0], HOTRG_ECUDA, "cudaStreamWaitEvent failed");
          std::vector<hotrg_plan> ap;
          for (int j : act) ap.push_back(ps[j]);
          if (r == HOTRG_OK) r = group_gemms(g, ap.data(), (int)ap.size(), k);
          if (r == HOTRG_OK && cudaEventRecord(g->ev_done, g->stream) != cudaSuccess)
            r = fail(ps[0], HOTRG_ECUDA, "cudaEventRecord failed");
          if (r != HOTRG_OK) {
            lead = r;
            failed = true;
          }
        }
        bar.wait();
        if (mine && !failed.load() && cudaStreamWaitEvent(q->stream, g->ev_done, 0) != cudaSuccess) {
          st[i] = fail(q, HOTRG_ECUDA, "cudaStreamWaitEvent failed");
          failed = true;
        }
      }
      if (mine && !failed.load()) {
        hotrg_status r = step_finish(q, k);
        if (r != HOTRG_OK) {
          st[i] = r;
          failed = true;
        }
      }
    }
    if (!failed.load()) {
      hotrg_status r = forward_end(q);
      if (r != HOTRG_OK) {
        st[i] = r;
        failed = true;
      }
    }
  };
  // the plans live on the caller's current device; the helper threads use it too
  int dev = 0;
  CK2(ps[0], cudaGetDevice(&dev));
  std::vector<std::thread> th;
  for (int i = 1; i < cnt; ++i)
    th.emplace_back([&, i] {
      if (cudaSetDevice(dev) != cudaSuccess) {
        st[i] = HOTRG_ECUDA;
        failed = true;
      }
      body(i);
    });
  body(0);
  for (auto& t : th) t.join();
  if (lead != HOTRG_OK) return lead;
  for (int i = 0; i < cnt; ++i)
    if (st[i] != HOTRG_OK) return st[i];
  // grouped launches report device errors in the first plan's error word
  CK2(ps[0], cudaStreamSynchronize(g->stream));
  for (int i = 0; i < cnt; ++i) CK2(ps[i], cudaStreamSynchronize(ps[i]->stream));
  int w0[2] = {0, 0};
  CK2(ps[0], cudaMemcpy(w0, ps[0]->err, 2 * sizeof(int), cudaMemcpyDeviceToHost));
  for (int i = 0; i < cnt; ++i) {
    int w[2] = {0, 0};
    CK2(ps[i], cudaMemcpy(w, ps[i]->err, 2 * sizeof(int), cudaMemcpyDeviceToHost));
    w[0] |= w0[0];
    if (!w[1]) w[1] = w0[1];
    hotrg_status r = device_status(ps[i], w);
    if (r != HOTRG_OK) return r;
  }
  for (int i = 0; i < cnt; ++i) {
    ps[i]->have_fwd = true;
    ps[i]->fwd_ising = false;
  }
  return HOTRG_OK;
}

hotrg_status group_outputs(hotrg_plan* ps, int cnt, double* lnz) {
  for (int i = 0; i < cnt; ++i) {
    double v = 0;
    CK2(ps[i], cudaMemcpy(&v, ps[i]->out, sizeof(double), cudaMemcpyDeviceToHost));
    if (lnz) lnz[i] = v;
  }
  return HOTRG_OK;
}

}  // namespace

namespace hotrg {
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

cudaStream_t plan_stream(hotrg_plan p) { return p->stream; }
int plan_sms(hotrg_plan p) { return p->sms; }
int* plan_err(hotrg_plan p) { return p->err; }
double* plan_isometry(hotrg_plan p, int k) { return p->E[k - 1]; }
const double* plan_wbar(hotrg_plan p, int k) {
  return p->wbar_all ? p->wbar_all + p->w_off[k - 1] : nullptr;
}
const double* plan_T0(hotrg_plan p) { return p->T[0]; }
const double* plan_lnz(hotrg_plan p) { return p->out; }
bool plan_has_forward(hotrg_plan p) { return p->have_fwd; }
bool plan_w_given(hotrg_plan p) { return p->cfg.w_given != 0; }
int plan_given_steps(hotrg_plan p) { return p->given_steps; }
int plan_steps_run(hotrg_plan p) { return p->n_run; }
hotrg_status plan_fail(hotrg_plan p, hotrg_status s, const char* msg) { return fail(p, s, msg); }
}  // namespace hotrg

extern "C" {

unsigned long long hotrg_kernel_launches(void) { return g_launches.load(); }

hotrg_status hotrg_debug_inject(int what, int arg) {
  if (what < 0 || what > 3) return HOTRG_EINVAL;
  g_inj_count.store(0);
  g_inj_arg.store(arg);
  g_inj_what.store(what);
  return HOTRG_OK;
}

hotrg_status hotrg_check_bounded_wait(double timeout_ms) {
  if (!(timeout_ms > 0.0) || timeout_ms > 10000.0) return HOTRG_EINVAL;
  int dev = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0)
    return HOTRG_ECUDA;
  int* err = nullptr;
  if (cudaMalloc(&err, 2 * sizeof(int)) != cudaSuccess) return HOTRG_ENOMEM;
  hotrg_status st = HOTRG_OK;
  int e = 0;
  if (cudaMemset(err, 0, 2 * sizeof(int)) != cudaSuccess ||
      bounded_wait_probe(err, (long long)(timeout_ms * khz), 0) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    st = HOTRG_ECUDA;
  else if (e & kErrTimeout)
    st = HOTRG_ETIMEOUT;
  cudaFree(err);
  return st;
}

hotrg_status hotrg_profile_enable(hotrg_plan p, int enable) {
  if (!p) return HOTRG_EINVAL;
  if (enable && p->ev_pool.empty()) {
    p->ev_pool.resize(8192);
    for (auto& e : p->ev_pool)
      if (cudaEventCreate(&e) != cudaSuccess) {
        e = nullptr;
        return fail(p, HOTRG_ECUDA, "cudaEventCreate failed");
      }
  }
  p->prof = enable != 0;
  p->ev_used = 0;
  p->prof_rec.clear();
  return HOTRG_OK;
}

hotrg_status hotrg_profile_read(hotrg_plan p, double* ms, int* counts) {
  if (!p || !ms) return HOTRG_EINVAL;
  CK(cudaStreamSynchronize(p->stream));
  for (int i = 0; i < HOTRG_PROFILE_SLOTS; ++i) {
    ms[i] = 0.0;
    if (counts) counts[i] = 0;
  }
  for (const auto& r : p->prof_rec) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p->ev_pool[r.second], p->ev_pool[r.second + 1]) == cudaSuccess) {
      ms[r.first] += t;
      if (counts) counts[r.first] += 1;
    }
  }
  p->ev_used = 0;
  p->prof_rec.clear();
  return HOTRG_OK;
}

size_t hotrg_config_sizeof(void) { return sizeof(hotrg_config); }



void hotrg_config_default(hotrg_config* c, int d0, int d_cut, int n_steps) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->d0 = d0;
  c->d_cut = d_cut;
  c->n_steps = n_steps;
  c->precision = HOTRG_FP64;
  c->split_from_step = 1;
  c->want_grad = 1;
  c->fixed_w_grad = 0;
  c->eigh_broadening = 1e-12;
  c->gram_split_from_step = 0;
  c->hi_precision_steps = 2;
  c->eigh_mode = 0;
  c->eigh_power_iters = 4;
  c->eigh_block = 0;
  c->epilogue_split = 1;
  c->split_chunk_elems = 0;
  c->w_given = 0;
  c->eigh_residual_tol = 0.0;
  c->stage2_n_group = 0;
  c->stage2_pair = 0;
  c->gemm_sm_reserve = 0;
  c->eigh_warm_start = 0;
  c->scheme = 0;
  c->chain_steps = 0;
  c->w_rule = 0;
}

hotrg_status hotrg_plan_workspace_bytes(const hotrg_config* c, size_t* bytes) {
  if (validate(c) != HOTRG_OK || !bytes) return HOTRG_EINVAL;
  Layout L;
  if (!build_layout(*c, L)) return HOTRG_EINVAL;
  Bytes b;
  b.add(L.totalT, 8);
  b.add(c->want_grad ? L.totalE : L.maxN2, 8);
  b.add(L.totalLam, 8);
  b.add(L.maxN2, 8);          // Escr
  b.add(L.maxN, 8);           // wasc
  b.add(L.maxT, 8 * 4);       // Abuf Bbuf Abar Bbar
  b.add(L.chunk64, 8 * 2);    // Ub Vb
  if (c->want_grad) {
    long long wtot = 0;
    for (const StepGeom& g : L.g) wtot += (long long)g.Xp * g.N;
    b.add(wtot, 8);           // per-step isometry adjoints
    b.add(L.chunk64, 8 * 2);  // Pb Qb
    b.add(L.maxN * L.maxXp, 8 * 3);
    b.add(L.maxN2, 8);
    b.add(L.maxT, 8 * 3);
  }
  if (L.any_split) {
    b.add(L.splitT * L.np_max, 2 * 4);
    b.add(L.splitG * L.np_max, 2 * 2);
    b.add((L.splitW1 + L.splitW3) * L.np_max, 2);
    b.add(L.chunkS * L.np_max, 2 * 2);
    if (L.any_hi) b.add(L.chunkS > L.splitG ? L.chunkS : L.splitG, 8);
    b.add(L.chunkS > L.splitG ? L.chunkS : L.splitG, 4);
  }
  b.add(kSplitK, 8);
  {
    long long kmax = 0;   // subspace eigensolver blocks (two K x N, one K x K)
    for (const StepGeom& g : L.g)
      if (subspace_applies(*c, g) && subspace_k(*c, g) > kmax) kmax = subspace_k(*c, g);
    if (kmax > 0) {
      b.add(kmax * L.maxN, 8 * 2);
      b.add(kmax * kmax, 8);
    }
  }
  if (c->w_rule == 1) {
    b.add(L.maxN2, 8);                                    // right-side eigenvectors
    b.add(L.maxN + c->n_steps + 4, 8);
  }
  if (c->scheme == 1) {
    const long long Xm = L.maxXp > c->d0 ? L.maxXp : c->d0;
    b.add(Xm * Xm, 8 * 3);                                // chain eigenvectors
    b.add(Xm * Xm * (long long)c->d0 * c->d0, 8);         // chain GEMM buffer
    b.add(c->n_steps, 8);
  }
  b.total += (size_t)64 << 20;  // solver workspace and small buffers (estimate)
  *bytes = b.total;
  return HOTRG_OK;
}

hotrg_status hotrg_plan_create(const hotrg_config* cfg, void* cuda_stream, hotrg_plan* out) {
  if (!out) return HOTRG_EINVAL;
  *out = nullptr;
  if (validate(cfg) != HOTRG_OK) return HOTRG_EINVAL;
  hotrg_plan p = new hotrg_plan_s();
  p->cfg = *cfg;
  p->n_run = cfg->n_steps;
  p->given_steps = cfg->n_steps;
  if (!build_layout(*cfg, p->L)) {
    delete p;
    return HOTRG_EINVAL;
  }
  p->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  auto cleanup = [&](hotrg_status s) {
    hotrg_plan_destroy(p);
    return s;
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cleanup(HOTRG_ECUDA);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return cleanup(HOTRG_ECUDA);
  p->sms = prop.multiProcessorCount;
  p->tc_sms = std::max(1, p->sms - cfg->gemm_sm_reserve);
  if (p->L.any_split && !(prop.major == 10 && prop.minor == 3)) return cleanup(HOTRG_EUNSUPPORTED);
  const Layout& L = p->L;
  const int n = cfg->n_steps;
  hotrg_status s;
#define ALC(ptr, cnt)                          \
  do {                                         \
    s = dalloc(p, &(ptr), (cnt));              \
    if (s != HOTRG_OK) return cleanup(s);      \
  } while (0)
  p->T.resize(n + 1);
  ALC(p->T[0], (long long)cfg->d0 * cfg->d0 * cfg->d0 * cfg->d0);
  for (int k = 1; k <= n; ++k) {
    const StepGeom& g = L.g[k - 1];
    ALC(p->T[k], (long long)g.Y * g.Y * g.Xp * g.Xp);
  }
  if (cfg->want_grad) {
    p->E.resize(n);
    for (int k = 1; k <= n; ++k) ALC(p->E[k - 1], L.g[k - 1].N * L.g[k - 1].N);
  } else {
    p->E.resize(1);
    ALC(p->E[0], L.maxN2);
  }
  p->lam.resize(n);
  for (int k = 1; k <= n; ++k) ALC(p->lam[k - 1], L.g[k - 1].N);
  ALC(p->Escr, L.maxN2);
  ALC(p->wasc, L.maxN);
  ALC(p->Abuf, L.maxT);
  ALC(p->Bbuf, L.maxT);
  ALC(p->Ub, L.chunk64);
  ALC(p->Vb, L.chunk64);
  if (cfg->want_grad) {
    ALC(p->Pb, L.chunk64);
    ALC(p->Qb, L.chunk64);
    ALC(p->Abar, L.maxT);
    ALC(p->Bbar, L.maxT);
    ALC(p->Sb, L.maxN * L.maxXp);
    ALC(p->Hb, L.maxN * L.maxXp);
    ALC(p->wbT, L.maxN * L.maxXp);
    ALC(p->Gb, L.maxN2);
    {
      long long tot = 0;
      for (const StepGeom& g : L.g) {
        p->w_off.push_back(tot);
        tot += (long long)g.Xp * g.N;
      }
      ALC(p->wbar_all, tot);
    }
    ALC(p->Ecur, L.maxT);
    ALC(p->Enext, L.maxT);
    ALC(p->Tbar, L.maxT);
  }
  ALC(p->splitk, kSplitK);
  ALC(p->dT0, 64);
  ALC(p->partial, kMaxPartial);
  ALC(p->scal, 8);
  ALC(p->log_norms, n);
  ALC(p->out, n + 2);
  ALC(p->dtrunc, n);
  ALC(p->dgap, n);
  ALC(p->dres, n);
  ALC(p->err, 4);
  ALC(p->info, 4);
  if (L.any_split) {
    const int np = L.np_max;
    ALC(p->pTA, L.splitT * np);
    ALC(p->pTB, L.splitT * np);
    ALC(p->pT1, L.splitT * np);
    ALC(p->pP, L.splitT * np);
    ALC(p->pA, L.splitG * np);
    ALC(p->pB, L.splitG * np);
    ALC(p->pW1, L.splitW1 * np);
    ALC(p->pW3, L.splitW3 * np);
    ALC(p->pU, L.chunkS * np);
    ALC(p->pV, L.chunkS * np);
    ALC(p->F32, L.chunkS > L.splitG ? L.chunkS : L.splitG);
    if (L.any_hi) ALC(p->F64, L.chunkS > L.splitG ? L.chunkS : L.splitG);
  }
  if (cusolverDnCreate(&p->solver) != CUSOLVER_STATUS_SUCCESS) return cleanup(HOTRG_ECUDA);
  if (cusolverDnSetStream(p->solver, p->stream) != CUSOLVER_STATUS_SUCCESS)
    return cleanup(HOTRG_ECUDA);
  int lw = 0;
  for (const StepGeom& g : L.g) {
    int l = 0;
    if (cusolverDnDsyevd_bufferSize(p->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                    (int)g.N, p->Escr, (int)g.N, p->wasc, &l) !=
        CUSOLVER_STATUS_SUCCESS)
      return cleanup(HOTRG_ECUDA);
    if (l > lw) lw = l;
    if (!cfg->want_grad && g.Xp < g.N) {
      int meig = 0;
      l = 0;
      if (cusolverDnDsyevdx_bufferSize(p->solver, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                                       CUBLAS_FILL_MODE_LOWER, (int)g.N, p->Escr, (int)g.N, 0.0,
                                       0.0, (int)g.N - g.Xp, (int)g.N, &meig, p->wasc, &l) !=
          CUSOLVER_STATUS_SUCCESS)
        return cleanup(HOTRG_ECUDA);
      if (l > lw) lw = l;
    }
  }
  p->lwork = lw;
  ALC(p->work, (long long)lw);
  if (cfg->w_given) {
    int ls = 0;
    for (const StepGeom& g : L.g) {
      int l = 0;
      if (cusolverDnDgesvd_bufferSize(p->solver, (int)g.N, g.Xp, &l) != CUSOLVER_STATUS_SUCCESS)
        return cleanup(HOTRG_ECUDA);
      ls = std::max(ls, l);
    }
    p->svd_lwork = ls;
    ALC(p->svd_work, (long long)ls);
    ALC(p->svd_rwork, L.maxXp);
  }
  if (cfg->eigh_mode == 1 && !cfg->want_grad && cfg->eigh_warm_start > 0) {
    ALC(p->wkeep[0], L.maxN * L.maxXp);
    ALC(p->wkeep[1], L.maxN * L.maxXp);
  }
  if (cfg->eigh_mode == 1 && (!cfg->want_grad || cfg->fixed_w_grad)) {
    int kmax = 0;
    long long nmax = 0;
    for (const StepGeom& g : L.g)
      if (subspace_applies(*cfg, g) && subspace_k(*cfg, g) > kmax) kmax = subspace_k(*cfg, g);
    nmax = L.maxN;
    if (kmax > 0) {
      p->kspace = kmax;
      ALC(p->Qs, nmax * kmax);
      ALC(p->Zs, nmax * kmax);
      ALC(p->Hs, (long long)kmax * kmax);
      ALC(p->tau, kmax);
      int l1 = 0, l2 = 0, l3 = 0, ls = 0, meig_q = 0;
      for (const StepGeom& g : L.g) {
        if (!subspace_applies(*cfg, g)) continue;
        const int Kq = subspace_k(*cfg, g), Nq = (int)g.N;
        if (cusolverDnDgeqrf_bufferSize(p->solver, Nq, Kq, p->Qs, Nq, &l1) != CUSOLVER_STATUS_SUCCESS ||
            cusolverDnDorgqr_bufferSize(p->solver, Nq, Kq, Kq, p->Qs, Nq, p->tau, &l2) !=
                CUSOLVER_STATUS_SUCCESS ||
            cusolverDnDsyevdx_bufferSize(p->solver, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                                         CUBLAS_FILL_MODE_LOWER, Kq, p->Hs, Kq, 0.0, 0.0,
                                         Kq - subspace_ritz(g) + 1, Kq, &meig_q, p->wasc, &l3) !=
                CUSOLVER_STATUS_SUCCESS)
          return cleanup(HOTRG_ECUDA);
        ls = std::max(ls, std::max(l1, std::max(l2, l3)));
      }
      p->lswork = ls;
      ALC(p->swork, (long long)ls);
    }
  }
  if (cfg->w_rule == 1) {
    ALC(p->Er, L.maxN2);
    ALC(p->lamR, L.maxN);
    ALC(p->trR, 2);
    long long nint = (n + 1) / 2 + 1;          // n ints in doubles
    double* sd = nullptr;
    ALC(sd, nint);
    p->side_dev = reinterpret_cast<int*>(sd);
    if (cudaMemset(p->side_dev, 0, sizeof(int) * n) != cudaSuccess) return cleanup(HOTRG_ECUDA);
  }
  if (cfg->scheme == 1) {
    const long long Xm = L.maxXp > cfg->d0 ? L.maxXp : cfg->d0;
    const long long d2 = (long long)cfg->d0 * cfg->d0;
    ALC(p->chR, Xm * Xm);
    ALC(p->chW, Xm * Xm);
    ALC(p->chV, Xm * Xm);
    ALC(p->chZ, Xm * Xm * d2);
    ALC(p->lnz_steps, n);
  }
  if (cudaMallocHost(&p->guard_host, sizeof(int)) != cudaSuccess) {
    p->guard_host = nullptr;
    return cleanup(HOTRG_ENOMEM);
  }
  if (cudaMemset(p->err, 0, 3 * sizeof(int)) != cudaSuccess) return cleanup(HOTRG_ECUDA);
#undef ALC
  *out = p;
  return HOTRG_OK;
}

void hotrg_plan_destroy(hotrg_plan p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  else cudaDeviceSynchronize();
  if (p->solver) cusolverDnDestroy(p->solver);
  for (auto e : p->ev_pool)
    if (e) cudaEventDestroy(e);
  for (void* v : p->allocs) cudaFree(v);
  if (p->guard_host) cudaFreeHost(p->guard_host);
  delete p;
}

hotrg_status hotrg_forward_device(hotrg_plan p, const double* T0_dev, double* out_dev) {
  if (!p || !T0_dev) return fail(p, HOTRG_EINVAL, "null argument");
  const long long n0 = (long long)p->cfg.d0 * p->cfg.d0 * p->cfg.d0 * p->cfg.d0;
  p->have_fwd = false;
  CK(cudaMemsetAsync(p->err, 0, 3 * sizeof(int), p->stream));
  if (T0_dev != p->T[0])
    CK(cudaMemcpyAsync(p->T[0], T0_dev, sizeof(double) * n0, cudaMemcpyDeviceToDevice, p->stream));
  hotrg_status r = run_forward(p);
  if (r != HOTRG_OK) return r;
  if (out_dev)
    CK(cudaMemcpyAsync(out_dev, p->out, sizeof(double) * (p->n_run + 2),
                       cudaMemcpyDeviceToDevice, p->stream));
  p->have_fwd = true;
  p->fwd_ising = false;
  return HOTRG_OK;
}

static hotrg_status copy_out(hotrg_plan p, double* lnz, double* log_norms, int* sign) {
  std::vector<double> h(p->n_run + 2);
  CK(cudaMemcpyAsync(h.data(), p->out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                     p->stream));
  hotrg_status r = finish_sync(p);
  if (r != HOTRG_OK) {
    p->have_fwd = false;
    return r;
  }
  if (lnz) *lnz = h[0];
  if (sign) *sign = h[1] >= 0 ? 1 : -1;
  if (log_norms) memcpy(log_norms, h.data() + 2, sizeof(double) * p->n_run);
  return HOTRG_OK;
}

hotrg_status hotrg_forward_tensor(hotrg_plan p, const double* T0_host, double* lnz,
                                  double* log_norms, int* trace_sign) {
  if (!p || !T0_host) return fail(p, HOTRG_EINVAL, "null argument");
  const long long n0 = (long long)p->cfg.d0 * p->cfg.d0 * p->cfg.d0 * p->cfg.d0;
  for (long long i = 0; i < n0; ++i)
    if (!std::isfinite(T0_host[i])) return fail(p, HOTRG_EINVAL, "T0 has a non-finite entry");
  CK(cudaMemcpyAsync(p->T[0], T0_host, sizeof(double) * n0, cudaMemcpyHostToDevice, p->stream));
  hotrg_status r = hotrg_forward_device(p, p->T[0], nullptr);
  if (r != HOTRG_OK) return r;
  return copy_out(p, lnz, log_norms, trace_sign);
}

hotrg_status hotrg_forward_ising(hotrg_plan p, double beta, double J, double h, double* lnz,
                                 double* log_norms, int* trace_sign) {
  if (!p) return HOTRG_EINVAL;
  if (p->cfg.d0 != 2) return fail(p, HOTRG_EINVAL, "Ising tensor needs d0 == 2");
  if (!std::isfinite(beta) || !std::isfinite(J) || !std::isfinite(h) || beta * J < 0)
    return fail(p, HOTRG_EINVAL, "Ising parameters must be finite with beta*J >= 0");
  CK(ising_t0(beta, J, h, p->T[0], p->dT0, p->stream));
  hotrg_status r = hotrg_forward_device(p, p->T[0], nullptr);
  if (r != HOTRG_OK) return r;
  r = copy_out(p, lnz, log_norms, trace_sign);
  if (r == HOTRG_OK) p->fwd_ising = true;
  return r;
}

hotrg_status hotrg_backward_device(hotrg_plan p, double* grad_dev) {
  if (!p) return HOTRG_EINVAL;
  if (!p->cfg.want_grad) return fail(p, HOTRG_ESTATE, "plan created with want_grad = 0");
  if (!p->have_fwd) return fail(p, HOTRG_ESTATE, "backward needs a forward first");
  CK(cudaMemsetAsync(p->err, 0, 3 * sizeof(int), p->stream));
  hotrg_status r = run_backward(p);
  if (r != HOTRG_OK) return r;
  p->have_bwd = true;
  if (grad_dev) {
    const long long n0 = (long long)p->cfg.d0 * p->cfg.d0 * p->cfg.d0 * p->cfg.d0;
    CK(cudaMemcpyAsync(grad_dev, p->Ecur, sizeof(double) * n0, cudaMemcpyDeviceToDevice,
                       p->stream));
  }
  return HOTRG_OK;
}

hotrg_status hotrg_backward(hotrg_plan p, double* grad, double* dbeta) {
  if (!p) return HOTRG_EINVAL;
  if (dbeta && !p->fwd_ising) return fail(p, HOTRG_ESTATE, "d/dbeta needs hotrg_forward_ising");
  hotrg_status r = hotrg_backward_device(p, nullptr);
  if (r != HOTRG_OK) return r;
  const int n0 = p->cfg.d0 * p->cfg.d0 * p->cfg.d0 * p->cfg.d0;
  if (dbeta) CK(dot_small(p->Ecur, p->dT0, n0, p->scal + 2, p->stream));
  std::vector<double> h(n0);
  double db = 0;
  CK(cudaMemcpyAsync(h.data(), p->Ecur, sizeof(double) * n0, cudaMemcpyDeviceToHost, p->stream));
  if (dbeta) CK(cudaMemcpyAsync(&db, p->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  r = finish_sync(p);
  if (r != HOTRG_OK) return r;
  if (grad) memcpy(grad, h.data(), sizeof(double) * n0);
  if (dbeta) *dbeta = db;
  return HOTRG_OK;
}

hotrg_status hotrg_plan_set_stream(hotrg_plan p, void* cuda_stream) {
  if (!p) return HOTRG_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (s == p->stream) return HOTRG_OK;
  CK(cudaStreamSynchronize(p->stream));   // the plan's work on its old stream is done
  if (cusolverDnSetStream(p->solver, s) != CUSOLVER_STATUS_SUCCESS)
    return fail(p, HOTRG_ECUDA, "cusolverDnSetStream failed");
  p->stream = s;
  return HOTRG_OK;
}

hotrg_status hotrg_plan_set_steps(hotrg_plan p, int n_steps) {
  if (!p) return HOTRG_EINVAL;
  if (n_steps < 1 || n_steps > p->cfg.n_steps)
    return fail(p, HOTRG_EINVAL, "steps must be in [1, the plan's n_steps]");
  if (n_steps != p->n_run) p->have_fwd = p->have_bwd = false;
  p->n_run = n_steps;
  return HOTRG_OK;
}

hotrg_status hotrg_sync(hotrg_plan p) {
  if (!p) return HOTRG_EINVAL;
  return finish_sync(p);
}

hotrg_status hotrg_diagnostics(hotrg_plan p, double* trunc, double* gap, int* is_split) {
  if (!p) return HOTRG_EINVAL;
  const int n = p->cfg.n_steps;
  if (trunc) CK(cudaMemcpy(trunc, p->dtrunc, sizeof(double) * n, cudaMemcpyDeviceToHost));
  if (gap) CK(cudaMemcpy(gap, p->dgap, sizeof(double) * n, cudaMemcpyDeviceToHost));
  if (is_split)
    for (int k = 0; k < n; ++k) is_split[k] = p->L.g[k].split ? 1 : 0;
  return HOTRG_OK;
}

hotrg_status hotrg_eigh_diagnostics(hotrg_plan p, double* residual, int* extra_iters,
                                    int* exact_step, long long* guard_steps) {
  if (!p) return HOTRG_EINVAL;
  const int n = p->cfg.n_steps;
  if (residual) CK(cudaMemcpy(residual, p->dres, sizeof(double) * n, cudaMemcpyDeviceToHost));
  const bool have = (int)p->exact_step.size() == n;
  for (int k = 0; k < n; ++k) {
    if (extra_iters) extra_iters[k] = have ? p->guard_iters[k] : 0;
    if (exact_step) exact_step[k] = have ? p->exact_step[k] : 0;
  }
  if (guard_steps) *guard_steps = p->fallbacks;
  return HOTRG_OK;
}

hotrg_status hotrg_step_dims(hotrg_plan p, int step, int* X, int* Y, int* Xp) {
  if (!p || step < 1 || step > p->cfg.n_steps) return HOTRG_EINVAL;
  const StepGeom& g = p->L.g[step - 1];
  if (X) *X = g.X;
  if (Y) *Y = g.Y;
  if (Xp) *Xp = g.Xp;
  return HOTRG_OK;
}

hotrg_status hotrg_isometries(hotrg_plan p, double* w) {
  if (!p || !w) return HOTRG_EINVAL;
  if (!p->cfg.want_grad) return fail(p, HOTRG_ESTATE, "isometries are kept by gradient plans");
  if (!p->have_fwd && !p->w_loaded) return fail(p, HOTRG_ESTATE, "no forward yet");
  for (int k = 1; k <= p->cfg.n_steps; ++k) {
    const StepGeom& g = p->L.g[k - 1];
    CK(cudaMemcpyAsync(w + p->w_off[k - 1], p->E[k - 1], sizeof(double) * g.Xp * g.N,
                       cudaMemcpyDeviceToHost, p->stream));
  }
  return finish_sync(p);
}

hotrg_status hotrg_set_isometries(hotrg_plan p, const double* w) {
  if (!p || !w) return HOTRG_EINVAL;
  if (!p->cfg.w_given) return fail(p, HOTRG_ESTATE, "plan created with w_given = 0");
  for (int k = 1; k <= p->cfg.n_steps; ++k) {
    const StepGeom& g = p->L.g[k - 1];
    const long long n = (long long)g.Xp * g.N;
    for (long long i = 0; i < n; ++i)
      if (!std::isfinite(w[p->w_off[k - 1] + i]))
        return fail(p, HOTRG_EINVAL, "isometry entries must be finite");
    CK(cudaMemcpyAsync(p->E[k - 1], w + p->w_off[k - 1], sizeof(double) * n,
                       cudaMemcpyHostToDevice, p->stream));
  }
  hotrg_status r = finish_sync(p);
  if (r != HOTRG_OK) return r;
  p->w_loaded = true;
  p->w_valid = p->cfg.n_steps;
  p->have_fwd = p->have_bwd = false;
  return HOTRG_OK;
}

hotrg_status hotrg_isometry_adjoints(hotrg_plan p, double* wbar) {
  if (!p || !wbar) return HOTRG_EINVAL;
  if (!p->wbar_all || !p->have_bwd) return fail(p, HOTRG_ESTATE, "needs a backward first");
  const StepGeom& last = p->L.g.back();
  const long long tot = p->w_off.back() + (long long)last.Xp * last.N;
  CK(cudaMemcpyAsync(wbar, p->wbar_all, sizeof(double) * tot, cudaMemcpyDeviceToHost, p->stream));
  return finish_sync(p);
}

hotrg_status hotrg_plan_set_given_steps(hotrg_plan p, int k0) {
  if (!p) return HOTRG_EINVAL;
  if (!p->cfg.w_given) return fail(p, HOTRG_ESTATE, "plan created with w_given = 0");
  if (k0 < 0 || k0 > p->cfg.n_steps) return fail(p, HOTRG_EINVAL, "k0 must be in [0, n_steps]");
  if (k0 != p->given_steps) p->have_fwd = p->have_bwd = false;
  p->given_steps = k0;
  return HOTRG_OK;
}

hotrg_status hotrg_forward_xy(hotrg_plan p, double tau, double J, double* lnz, double* log_norms) {
  if (!p) return HOTRG_EINVAL;
  if (p->cfg.scheme != 1 || p->cfg.d0 != 4)
    return fail(p, HOTRG_EINVAL, "the XY-chain MPO needs scheme = 1 and d0 == 4");
  if (!std::isfinite(tau) || !std::isfinite(J) || tau <= 0)
    return fail(p, HOTRG_EINVAL, "tau must be finite and positive, J finite");
  CK(xy_mpo(tau, J, p->T[0], p->stream));
  hotrg_status r = hotrg_forward_device(p, p->T[0], nullptr);
  if (r != HOTRG_OK) return r;
  return copy_out(p, lnz, log_norms, nullptr);
}

// Buffer sizes of a group (per-plane strides, staging and output elements).
void group_sizes(hotrg_group_s* g) {
  long long mW1 = 0, mT1 = 0, mP = 0, mW3 = 0, mU = 0, mV = 0, mT = 0;
  int np = 0;
  for (const StepGeom& s : g->L.g) {
    if (!groupable(s)) continue;
    const GroupGeom gg = group_geom(s);
    np = std::max(np, s.np);
    mW1 = std::max(mW1, gg.pW1); mT1 = std::max(mT1, gg.pT1); mP = std::max(mP, gg.pP);
    mW3 = std::max(mW3, gg.pW3); mU = std::max(mU, gg.pU); mV = std::max(mV, gg.pV);
    mT = std::max(mT, gg.pT);
  }
  g->np = np;
  const long long c = g->max_count;
  g->sW1 = round_up(c * mW1, 64); g->sT1 = round_up(c * mT1, 64); g->sP = round_up(c * mP, 64);
  g->sW3 = round_up(c * mW3, 64); g->sU = round_up(c * mU, 64); g->sV = round_up(c * mV, 64);
  g->nT = c * mT;
  g->nF = c * std::max(mU, mV);
}

long long group_bytes(const hotrg_group_s* g) {
  if (g->np == 0) return 0;
  return 2LL * g->np * (g->sW1 + g->sT1 + g->sP + g->sW3 + g->sU + g->sV) + 4 * g->nF +
         (g->L.any_hi ? 8 * g->nF : 0) + 8 * g->nT;
}

hotrg_status hotrg_group_workspace_bytes(const hotrg_config* cfg, int max_count, size_t* bytes) {
  if (!bytes || validate(cfg) != HOTRG_OK || max_count < 1 || max_count > 64) return HOTRG_EINVAL;
  hotrg_group_s g;
  if (!build_layout(*cfg, g.L)) return HOTRG_EINVAL;
  g.max_count = max_count;
  group_sizes(&g);
  *bytes = (size_t)group_bytes(&g);
  return HOTRG_OK;
}

hotrg_status hotrg_group_create(const hotrg_config* cfg, int max_count, void* cuda_stream,
                                hotrg_group* out) {
  if (!out) return HOTRG_EINVAL;
  *out = nullptr;
  if (validate(cfg) != HOTRG_OK || max_count < 1 || max_count > 64) return HOTRG_EINVAL;
  if (cfg->scheme != 0 || cfg->w_given || cfg->w_rule != 0) return HOTRG_EINVAL;
  hotrg_group g = new hotrg_group_s();
  if (!build_layout(*cfg, g->L)) {
    delete g;
    return HOTRG_EINVAL;
  }
  g->max_count = max_count;
  g->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  group_sizes(g);
  const int np = g->np;
  auto alloc = [&](long long bytes, void** ptr) -> bool {
    if (bytes <= 0) { *ptr = nullptr; return true; }
    if (cudaMalloc(ptr, (size_t)bytes) != cudaSuccess) return false;
    g->allocs.push_back(*ptr);
    return true;
  };
  bool ok = true;
  if (np > 0) {
    void* v;
    ok = ok && alloc(2 * np * g->sW1, &v); g->W1 = static_cast<__nv_bfloat16*>(v);
    ok = ok && alloc(2 * np * g->sT1, &v); g->T1 = static_cast<__nv_bfloat16*>(v);
    ok = ok && alloc(2 * np * g->sP, &v); g->P = static_cast<__nv_bfloat16*>(v);
    ok = ok && alloc(2 * np * g->sW3, &v); g->W3 = static_cast<__nv_bfloat16*>(v);
    ok = ok && alloc(2 * np * g->sU, &v); g->U = static_cast<__nv_bfloat16*>(v);
    ok = ok && alloc(2 * np * g->sV, &v); g->V = static_cast<__nv_bfloat16*>(v);
    ok = ok && alloc(4 * g->nF, &v); g->F32 = static_cast<float*>(v);
    if (g->L.any_hi) { ok = ok && alloc(8 * g->nF, &v); g->F64 = static_cast<double*>(v); }
    ok = ok && alloc(8 * g->nT, &v); g->Tg = static_cast<double*>(v);
  }
  if (!ok) {
    hotrg_group_destroy(g);
    return HOTRG_ENOMEM;
  }
  g->ev.assign(max_count, nullptr);
  for (int i = 0; i < max_count; ++i)
    if (cudaEventCreateWithFlags(&g->ev[i], cudaEventDisableTiming) != cudaSuccess) ok = false;
  if (!ok || cudaEventCreateWithFlags(&g->ev_done, cudaEventDisableTiming) != cudaSuccess) {
    hotrg_group_destroy(g);
    return HOTRG_ECUDA;
  }
  *out = g;
  return HOTRG_OK;
}

void hotrg_group_destroy(hotrg_group g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  else cudaDeviceSynchronize();
  for (cudaEvent_t e : g->ev)
    if (e) cudaEventDestroy(e);
  if (g->ev_done) cudaEventDestroy(g->ev_done);
  for (void* v : g->allocs) cudaFree(v);
  delete g;
}

unsigned long long hotrg_group_launches(hotrg_group g) { return g ? g->grouped_launches : 0; }

hotrg_status hotrg_forward_group_tensor(hotrg_group g, hotrg_plan* plans, int count,
                                        const double* T0_host, double* lnz) {
  hotrg_status r = group_check(g, plans, count);
  if (r != HOTRG_OK) return r;
  if (!T0_host) return HOTRG_EINVAL;
  const long long n0 = (long long)plans[0]->cfg.d0 * plans[0]->cfg.d0 * plans[0]->cfg.d0 *
                       plans[0]->cfg.d0;
  for (long long i = 0; i < n0 * count; ++i)
    if (!std::isfinite(T0_host[i])) return fail(plans[0], HOTRG_EINVAL, "T0 has a non-finite entry");
  for (int i = 0; i < count; ++i)
    CK2(plans[i], cudaMemcpyAsync(plans[i]->T[0], T0_host + i * n0, sizeof(double) * n0,
                                  cudaMemcpyHostToDevice, plans[i]->stream));
  r = group_run(g, plans, count);
  if (r != HOTRG_OK) return r;
  return group_outputs(plans, count, lnz);
}

hotrg_status hotrg_forward_group_ising(hotrg_group g, hotrg_plan* plans, int count,
                                       const double* beta, const double* J, const double* h,
                                       double* lnz) {
  hotrg_status r = group_check(g, plans, count);
  if (r != HOTRG_OK) return r;
  if (!beta || !J || !h) return HOTRG_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (plans[i]->cfg.d0 != 2) return fail(plans[i], HOTRG_EINVAL, "Ising tensor needs d0 == 2");
    if (!std::isfinite(beta[i]) || !std::isfinite(J[i]) || !std::isfinite(h[i]) ||
        beta[i] * J[i] < 0)
      return fail(plans[i], HOTRG_EINVAL, "Ising parameters must be finite with beta*J >= 0");
  }
  for (int i = 0; i < count; ++i)
    CK2(plans[i], ising_t0(beta[i], J[i], h[i], plans[i]->T[0], plans[i]->dT0, plans[i]->stream));
  r = group_run(g, plans, count);
  if (r != HOTRG_OK) return r;
  for (int i = 0; i < count; ++i) plans[i]->fwd_ising = true;
  return group_outputs(plans, count, lnz);
}

hotrg_status hotrg_isometry_sides(hotrg_plan p, int* side) {
  if (!p || !side) return HOTRG_EINVAL;
  if (!p->have_fwd) return fail(p, HOTRG_ESTATE, "no forward yet");
  if (!p->side_dev) {
    for (int k = 0; k < p->n_run; ++k) side[k] = 0;
    return HOTRG_OK;
  }
  CK(cudaMemcpyAsync(side, p->side_dev, sizeof(int) * p->n_run, cudaMemcpyDeviceToHost,
                     p->stream));
  return finish_sync(p);
}

hotrg_status hotrg_chain_lnz_steps(hotrg_plan p, double* out) {
  if (!p || !out) return HOTRG_EINVAL;
  if (p->cfg.scheme != 1) return fail(p, HOTRG_ESTATE, "plan created with scheme = 0");
  if (!p->have_fwd) return fail(p, HOTRG_ESTATE, "no forward yet");
  CK(cudaMemcpyAsync(out, p->lnz_steps, sizeof(double) * p->n_run, cudaMemcpyDeviceToHost,
                     p->stream));
  return finish_sync(p);
}

hotrg_status hotrg_mera_update(hotrg_plan p, int k) {
  if (!p || k < 1 || k > p->n_run) return HOTRG_EINVAL;
  if (!p->cfg.w_given) return fail(p, HOTRG_ESTATE, "plan created with w_given = 0");
  if (!p->have_bwd) return fail(p, HOTRG_ESTATE, "the MERA update needs a backward first");
  const StepGeom& g = p->L.g[k - 1];
  const int N = (int)g.N, Xp = g.Xp;
  cudaStream_t st = p->stream;
  CK(cudaMemsetAsync(p->err, 0, 3 * sizeof(int), st));
  // E_w (rows = kept vectors) is the N x Xp column-major matrix cuSOLVER reads
  CK(cudaMemcpyAsync(p->Gb, p->wbar_all + p->w_off[k - 1], sizeof(double) * (size_t)Xp * N,
                     cudaMemcpyDeviceToDevice, st));
  if (cusolverDnDgesvd(p->solver, 'S', 'S', N, Xp, p->Gb, N, p->wasc, p->Hb, N, p->Sb, Xp,
                       p->svd_work, p->svd_lwork, p->svd_rwork, p->info) != CUSOLVER_STATUS_SUCCESS)
    return fail(p, HOTRG_ECUDA, "cusolverDnDgesvd failed");
  CK(eigh_info_check(p->info, p->err, st));
  // w = U V^T: w_k[a][i] = sum_c VT(c, a) U(i, c)   (U: N x Xp, VT: Xp x Xp, column-major)
  CK(gemm_f64(g64(p, p->Sb, map_lin(Xp), map_lin(1), p->Hb, map_lin(1), map_lin(N), p->E[k - 1],
                  map_lin(N), map_lin(1), Xp, N, Xp, 1.0, 0.0),
              st, p->sms));
  hotrg_status r = finish_sync(p);
  if (r != HOTRG_OK) return r;
  p->have_fwd = p->have_bwd = false;     // the network changed
  return HOTRG_OK;
}

const char* hotrg_status_string(hotrg_status s) {
  switch (s) {
    case HOTRG_OK: return "ok";
    case HOTRG_EINVAL: return "invalid argument";
    case HOTRG_ENOMEM: return "out of device memory";
    case HOTRG_ECUDA: return "CUDA error";
    case HOTRG_ENOTCONV: return "eigensolver did not converge";
    case HOTRG_ENONFINITE: return "non-finite norm or trace";
    case HOTRG_ETIMEOUT: return "device wait timed out";
    case HOTRG_ESTATE: return "call out of order";
    case HOTRG_EUNSUPPORTED: return "unsupported on this device";
  }
  return "unknown status";
}

const char* hotrg_last_error(hotrg_plan p) { return p ? p->last_error.c_str() : "null plan"; }

hotrg_status hotrg_device_supports_split(void) {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return HOTRG_ECUDA;
  }
  return (prop.major == 10 && prop.minor == 3) ? HOTRG_OK : HOTRG_EUNSUPPORTED;
}

hotrg_status hotrg_gemm_split_check(int M, int N, int K, int planes, int kchunk, int cta_pair,
                                    const double* A, const double* B, double* C) {
  if (M < 1 || N < 1 || K < 8 || K % 8 != 0 || planes < 2 || planes > 4 || !A || !B || !C)
    return HOTRG_EINVAL;
  hotrg_status status = HOTRG_OK;
  double *dA = nullptr, *dB = nullptr, *dC = nullptr;
  __nv_bfloat16 *pa = nullptr, *pb = nullptr;
  int* err = nullptr;
  const long long sa = round_up((long long)M * K, 64), sb = round_up((long long)N * K, 64);
  int sms = 152, dev = 0, e = 0;
  cudaDeviceProp prop;
  TcGemm g;
  memset(&g, 0, sizeof(g));
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    status = HOTRG_ECUDA;
    goto done;
  }
  sms = prop.multiProcessorCount;
  if (cudaMalloc(&dA, sizeof(double) * M * (size_t)K) != cudaSuccess ||
      cudaMalloc(&dB, sizeof(double) * N * (size_t)K) != cudaSuccess ||
      cudaMalloc(&dC, sizeof(double) * M * (size_t)N) != cudaSuccess ||
      cudaMalloc(&pa, 2 * sa * planes) != cudaSuccess ||
      cudaMalloc(&pb, 2 * sb * planes) != cudaSuccess ||
      cudaMalloc(&err, 2 * sizeof(int)) != cudaSuccess) {
    status = HOTRG_ENOMEM;
    goto done;
  }
  cudaMemcpy(dA, A, sizeof(double) * M * (size_t)K, cudaMemcpyHostToDevice);
  cudaMemcpy(dB, B, sizeof(double) * N * (size_t)K, cudaMemcpyHostToDevice);
  cudaMemset(err, 0, 2 * sizeof(int));
  grid_split(dA, (long long)M * K, map_lin(K), map_lin(1), M, K, planes, sa, pa, err, 0, sms);
  grid_split(dB, (long long)N * K, map_lin(K), map_lin(1), N, K, planes, sb, pb, err, 0, sms);
  tc_set_pairs(g, planes);
  g.M = M; g.N = N; g.K = K; g.kchunk = kchunk;
  g.cm = map_lin(N); g.cn = map_lin(1);
  g.out_mode = kOutF64; g.out_planes = 1; g.C = dC; g.alpha = 1.f; g.err = err;
  g.c_lim = (long long)M * N;
  g.cta_pair = cta_pair ? 1 : 0;
  if (tc_gemm(opnd(pa, M, K, planes, sa), opnd(pb, N, K, planes, sb), g, 0, sms) != cudaSuccess) {
    status = HOTRG_ECUDA;
    goto done;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) { status = HOTRG_ECUDA; goto done; }
  cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e & kErrTimeout) { status = HOTRG_ETIMEOUT; goto done; }
  if (e) { status = HOTRG_ECUDA; goto done; }
  if (cudaMemcpy(C, dC, sizeof(double) * M * (size_t)N, cudaMemcpyDeviceToHost) != cudaSuccess)
    status = HOTRG_ECUDA;
done:
  cudaFree(dA); cudaFree(dB); cudaFree(dC); cudaFree(pa); cudaFree(pb); cudaFree(err);
  cudaGetLastError();
  return status;
}

hotrg_status hotrg_gemm_f64_check(int M, int N, int K, const double* A, const double* B, double* C) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C) return HOTRG_EINVAL;
  hotrg_status status = HOTRG_OK;
  double *dA = nullptr, *dB = nullptr, *dC = nullptr;
  int* err = nullptr;
  int dev = 0, e = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return HOTRG_ECUDA;
  if (cudaMalloc(&dA, sizeof(double) * M * (size_t)K) != cudaSuccess ||
      cudaMalloc(&dB, sizeof(double) * N * (size_t)K) != cudaSuccess ||
      cudaMalloc(&dC, sizeof(double) * M * (size_t)N) != cudaSuccess ||
      cudaMalloc(&err, 2 * sizeof(int)) != cudaSuccess) {
    status = HOTRG_ENOMEM;
  } else {
    cudaMemcpy(dA, A, sizeof(double) * M * (size_t)K, cudaMemcpyHostToDevice);
    cudaMemcpy(dB, B, sizeof(double) * N * (size_t)K, cudaMemcpyHostToDevice);
    cudaMemset(err, 0, 2 * sizeof(int));
    GemmF64 g;
    g.A = dA; g.am = map_lin(K); g.ak = map_lin(1);
    g.B = dB; g.bn = map_lin(K); g.bk = map_lin(1);
    g.C = dC; g.cm = map_lin(N); g.cn = map_lin(1);
    g.M = M; g.N = N; g.K = K; g.alpha = 1.0; g.beta = 0.0; g.a_kfast = 1; g.b_kfast = 1;
    g.a_lim = (long long)M * K; g.b_lim = (long long)N * K; g.c_lim = (long long)M * N;
    g.err = err;
    g.ws = nullptr;
    g.ws_elems = 0;
    if (gemm_f64(g, 0, prop.multiProcessorCount) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
      status = HOTRG_ECUDA;
    else if (cudaMemcpy(C, dC, sizeof(double) * M * (size_t)N, cudaMemcpyDeviceToHost) != cudaSuccess)
      status = HOTRG_ECUDA;
    else if (cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || e)
      status = HOTRG_ECUDA;
  }
  cudaFree(dA); cudaFree(dB); cudaFree(dC); cudaFree(err);
  cudaGetLastError();
  return status;
}

}  // extern "C"
