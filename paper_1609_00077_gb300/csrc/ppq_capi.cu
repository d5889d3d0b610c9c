// ppq_capi.cu -- C ABI of the PQ solver (see include/ppq.h): argument checks,
// input staging, the per-device workspace, the residual pipeline and the
// Jacobi/DIIS solve loop (Implementation section: denominators, DIIS).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <type_traits>
#include <utility>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ppq.h"
#include "ppq_kernels.cuh"
#include "ppq_adjoint.cuh"
#include "ppq_tc.cuh"
#include "ppq_tc64.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(-100, "CUDA error %s at %s:%d", cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                       \
  } while (0)

constexpr int kDiisMax = 16;

// PPQ_TRACE=1 in the environment prints one line per residual evaluation
// (phase, precision, ||R||, E_c) to stderr.
bool trace_on() {
  static int on = -1;
  if (on < 0) {
    const char* e = getenv("PPQ_TRACE");
    on = (e && *e && *e != '0') ? 1 : 0;
  }
  return on == 1;
}
constexpr int kRedBlocks = 304;  // 2 x 152 SMs

// Per-kernel device time of one profiled call (opts.profile = 1): events are
// recorded on the launching stream after every kernel, and each kernel is
// charged the time since the previous event, so the classes add up to the
// stream time of the call (gaps between launches included).  Algorithmic
// bytes and FLOPs are summed per class beside the time.
struct KProf {
  bool on = false;
  struct Cls {
    std::string name;
    double ms = 0.0, bytes = 0.0, flops = 0.0;
    int n = 0;
  };
  struct Mark {
    cudaEvent_t ev;
    int cls;
    double bytes, flops;
  };
  std::vector<Cls> cls;
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t take() {
    cudaEvent_t e = nullptr;
    if (!pool.empty()) { e = pool.back(); pool.pop_back(); }
    else cudaEventCreate(&e);
    return e;
  }
  int id(const char* name) {
    for (size_t i = 0; i < cls.size(); ++i)
      if (cls[i].name == name) return (int)i;
    cls.push_back(Cls());
    cls.back().name = name;
    return (int)cls.size() - 1;
  }
  void reset(bool enable) {
    flush();
    on = enable;
    cls.clear();
  }
  // start of a timed region on stream s
  void start(cudaStream_t s) {
    if (!on) return;
    cudaEvent_t e = take();
    cudaEventRecord(e, s);
    marks.push_back({e, -1, 0.0, 0.0});
  }
  // after a kernel of class `name` (charged the time since the previous mark)
  void done(const char* name, cudaStream_t s, double bytes = 0.0, double flops = 0.0) {
    if (!on) return;
    if (marks.empty()) start(s);
    cudaEvent_t e = take();
    cudaEventRecord(e, s);
    marks.push_back({e, id(name), bytes, flops});
  }
  // accumulate the recorded segments (waits for the stream's events)
  void flush() {
    for (size_t i = 1; i < marks.size(); ++i) {
      if (marks[i].cls < 0) continue;
      cudaEventSynchronize(marks[i].ev);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, marks[i - 1].ev, marks[i].ev);
      Cls& c = cls[marks[i].cls];
      c.ms += ms; c.n++; c.bytes += marks[i].bytes; c.flops += marks[i].flops;
    }
    for (auto& m : marks) pool.push_back(m.ev);
    marks.clear();
  }
};
KProf g_prof;

// Per-device workspace, grown on demand and kept between calls.
struct Workspace {
  int N = 0;       // capacity in pairs
  size_t eri_cap = 0;
  int diis_cap = 0;
  // staged inputs
  double *h = nullptr, *eri = nullptr;  // only when the caller passes host pointers
  double *Bcd = nullptr, *Bt = nullptr;  // three-index factors (raw host copy, transposed)
  size_t cd_cap = 0;
  int *occ = nullptr, *vir = nullptr, *lab = nullptr;
  double *f = nullptr, *hp = nullptr, *fo = nullptr, *fv = nullptr;
  double *g1d = nullptr, *g2d = nullptr;
  float *g1f = nullptr, *g2f = nullptr;
  // amplitudes, residual
  double *t = nullptr, *r = nullptr, *dir = nullptr, *abuf = nullptr;
  // residual scratch (sized for double, reused as float)
  void *cl = nullptr, *hs = nullptr, *pg = nullptr, *pt7 = nullptr, *pc0 = nullptr;
  void *clT = nullptr, *gT = nullptr, *B9 = nullptr;  // quartic GEMM operands / output
  float2* clT2 = nullptr;                              // FP64 quartic epilogue: clT as float pairs
  void *pt7T = nullptr, *m7 = nullptr;                 // T7 GEMM operand / output
  // tensor-core quartic kernel (FP32 residual): split B operands, work list
  bool tc_allowed = false;  // set for workspaces that own their buffers
  int tc_N = 0, tc_Npad = 0, tc_Kc = 0, tc_nctas = 0;
  size_t tc_smem = 0;
  float* bpre = nullptr;
  int16_t* tc_chunk = nullptr;
  int* tc_cta = nullptr;
  int* tc_err = nullptr;
  int tc_nslot = 0;
  float* tc_part = nullptr;   // per-CTA row sums, [slot][p][29]
  // the same for the FP64 residual (exact-splitting tensor-core kernel)
  int tc64_N = 0, tc64_Npad = 0, tc64_Kc = 0, tc64_nctas = 0, tc64_nslot = 0;
  size_t tc64_smem = 0;
  float* bpre64 = nullptr;
  int* fexp64 = nullptr;
  int16_t* tc64_chunk = nullptr;
  int* tc64_cta = nullptr;
  double* tc64_part = nullptr;
  double* t9part = nullptr;   // per-work-item row sums of the SIMT kernel, [item][p][29]
  double* r1part = nullptr;   // k_r1 partial sums, [split][N][3]
  double* t9 = nullptr;
  double *tb = nullptr, *r64 = nullptr, *rb = nullptr, *del = nullptr, *rho = nullptr;
  unsigned long long* amax = nullptr;
  int* work9 = nullptr;
  int n_work9 = 0;
  double *esite = nullptr, *epair = nullptr;
  // reductions
  double *part = nullptr, *scal = nullptr, *coef = nullptr, *Bdiis = nullptr;
  int* ok = nullptr;
  int* order = nullptr;
  double* host = nullptr;  // pinned host scalars
  // DIIS ring: slots of t_new and of e
  double *slot_t = nullptr, *slot_e = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evq0 = nullptr, evq1 = nullptr;
  // optional timing of the quartic kernel (opts.profile)
  bool profile = false;
  double t_quartic_ms = 0.0;
  int n_quartic = 0;
  double t_quartic32_ms = 0.0;  // FP32 launches only
  int n_quartic32 = 0;
  int n_launches = 0;
  // adjoint (Lambda / gradient) buffers, allocated on first use
  int adjN = 0;
  double *clb = nullptr, *hsb = nullptr, *pgb = nullptr, *pt7b = nullptr, *pc0b = nullptr;
  double *dirb = nullptr, *abufb = nullptr, *t9b = nullptr, *gt = nullptr, *gu = nullptr;
  double *B9a = nullptr, *B9b = nullptr, *lam = nullptr;
  double *gb1 = nullptr, *gb2 = nullptr;                 // dL/d(gathered integrals)
  double *gh_raw = nullptr, *gh = nullptr, *gv_raw = nullptr, *gv = nullptr, *dk = nullptr, *ab = nullptr;
  size_t grad_n = 0;
  // captured residual pipeline per precision (index 0 FP64, 1 FP32)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int mt[2] = {1, 1};  // tuned GEMM micro-tile per precision for the current N
  int graph_N[2] = {0, 0};
  int graph_profile[2] = {0, 0};
  int graph_launches[2] = {0, 0};   // kernels in each captured pipeline
};

std::mutex g_mu;
std::map<int, Workspace*> g_ws;
std::map<int, std::vector<Workspace*>> g_batch_ws;  // per-thread workspaces of pq_solve_batched

size_t amp_len(int N) { return (size_t)3 * N + (size_t)PPQ_NA2 * N * N; }

// slice stride of the transposed link coefficients clT[c][X][Y]
inline int cl_ld(int N) { return (N * N + 3) & ~3; }

constexpr int kTcMaxN = 80;      // largest N of the tensor-core quartic kernel
constexpr int kR1Split = 8;      // blocks per output pair label in k_r1
constexpr int kTcMaxCtas = 1024;
constexpr int kTcPartRows = 152 * 128;  // slots x unordered pairs of the partial buffer

void free_ws(Workspace* w) {
  void* ps[] = {w->h, w->eri, w->Bcd, w->Bt, w->occ, w->vir, w->lab, w->f, w->hp, w->fo, w->fv, w->g1d, w->g2d,
                w->g1f, w->g2f, w->t, w->r, w->dir, w->abuf, w->cl, w->hs, w->pg, w->pt7, w->pc0,
                w->esite, w->epair, w->part, w->scal, w->coef, w->Bdiis, w->ok, w->order, w->slot_t, w->slot_e,
                w->clT, w->clT2, w->gT, w->B9, w->t9, w->work9, w->tb, w->r64, w->rb, w->del, w->rho,
                w->amax, w->pt7T, w->m7, w->bpre, w->tc_chunk, w->tc_cta, w->tc_err, w->tc_part, w->t9part,
                w->bpre64, w->fexp64, w->tc64_chunk, w->tc64_cta, w->tc64_part, w->r1part};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (w->host) cudaFreeHost(w->host);
  if (w->ev0) cudaEventDestroy(w->ev0);
  if (w->ev1) cudaEventDestroy(w->ev1);
  if (w->evq0) cudaEventDestroy(w->evq0);
  if (w->evq1) cudaEventDestroy(w->evq1);
  for (int i = 0; i < 2; ++i)
    if (w->graph[i]) cudaGraphExecDestroy(w->graph[i]);
  void* pa[] = {w->clb, w->hsb, w->pgb, w->pt7b, w->pc0b, w->dirb, w->abufb, w->t9b, w->gt, w->gu,
                w->B9a, w->B9b, w->lam, w->gb1, w->gb2, w->gh_raw, w->gh, w->gv_raw, w->gv, w->dk,
                w->ab};
  for (void* p : pa)
    if (p) cudaFree(p);
  *w = Workspace();
}

int grow(Workspace* w, int N, int diis) {
  if (N <= w->N && diis <= w->diis_cap && w->host) return 0;
  int n = 2 * N;
  int Nc = N > w->N ? N : w->N;
  int dc = diis > w->diis_cap ? diis : w->diis_cap;
  free_ws(w);
  size_t NN = (size_t)Nc * Nc, L = amp_len(Nc);
  n = 2 * Nc;
#define AL(ptr, bytes) CK(cudaMalloc((void**)&(ptr), (bytes) > 0 ? (bytes) : 8))
  AL(w->h, sizeof(double) * n * n);
  AL(w->occ, sizeof(int) * Nc); AL(w->vir, sizeof(int) * Nc); AL(w->lab, sizeof(int) * n);
  AL(w->f, sizeof(double) * n * n); AL(w->hp, sizeof(double) * n * n);
  AL(w->fo, sizeof(double) * Nc); AL(w->fv, sizeof(double) * Nc);
  AL(w->g1d, sizeof(double) * Nc * PPQ_NG1); AL(w->g2d, sizeof(double) * NN * PPQ_NG2);
  AL(w->g1f, sizeof(float) * Nc * PPQ_NG1); AL(w->g2f, sizeof(float) * NN * PPQ_NG2);
  AL(w->t, sizeof(double) * L); AL(w->r, sizeof(double) * L);
  AL(w->dir, sizeof(double) * NN * PPQ_NA2); AL(w->abuf, sizeof(double) * NN * PPQ_NA2);
  AL(w->cl, sizeof(double) * NN * PPQ_NS36); AL(w->hs, sizeof(double) * Nc * 256);
  AL(w->pg, sizeof(double) * NN * PPQ_NS36); AL(w->pt7, sizeof(double) * NN * PPQ_NT7E);
  AL(w->pc0, sizeof(double) * NN * PPQ_NCOL0);
  AL(w->clT, sizeof(double) * cl_ld(Nc) * PPQ_NS36); AL(w->gT, sizeof(double) * NN * PPQ_NS36);
  AL(w->clT2, sizeof(float2) * cl_ld(Nc) * PPQ_NS36);
  AL(w->tb, sizeof(double) * L); AL(w->r64, sizeof(double) * L); AL(w->rb, sizeof(double) * L);
  AL(w->del, sizeof(double) * L); AL(w->rho, sizeof(double) * L);
  AL(w->amax, sizeof(unsigned long long));
  AL(w->t9, sizeof(double) * NN * PPQ_NA2);
  AL(w->pt7T, sizeof(double) * NN * PPQ_NT7E); AL(w->m7, sizeof(double) * NN * PPQ_NK7);
  {
    int Nt = std::min(Nc, kTcMaxN);
    size_t npad = (size_t)(Nt + 15) / 16 * 16, kc = (size_t)(Nt + 7) / 8;
    AL(w->bpre, sizeof(float) * PPQ_NS36 * 2 * kc * npad * 8);
    AL(w->tc_chunk, sizeof(int16_t) * ppq::tc::kChunkFields * PPQ_NQ9);
    AL(w->tc_cta, sizeof(int) * 3 * kTcMaxCtas);
    AL(w->tc_err, sizeof(int));
    AL(w->tc_part, sizeof(float) * kTcPartRows * PPQ_NA2);
    AL(w->bpre64, sizeof(float) * PPQ_NS36 * ppq::tc::kSl * kc * npad * 8);
    AL(w->fexp64, sizeof(int) * PPQ_NS36 * npad);
    AL(w->tc64_chunk, sizeof(int16_t) * ppq::tc::kChunkFields * PPQ_NQ9);
    AL(w->tc64_cta, sizeof(int) * 3 * kTcMaxCtas);
    AL(w->tc64_part, sizeof(double) * kTcPartRows * PPQ_NA2);
    w->tc64_N = 0;
    CK(cudaMemset(w->tc_err, 0, sizeof(int)));
    w->tc_allowed = true;
    w->tc_N = 0;
  }
  {
    // quartic GEMM work items: chunks of at most 4 (c1, g) entries of one c2
    std::vector<int> wk;
    for (int c2 = 0; c2 < 30; ++c2)
      for (int a = ppq_q9cptr_h[c2]; a < ppq_q9cptr_h[c2 + 1]; a += 4) {
        wk.push_back(c2); wk.push_back(a); wk.push_back(std::min(a + 4, (int)ppq_q9cptr_h[c2 + 1]));
      }
    w->n_work9 = (int)wk.size() / 3;
    AL(w->work9, sizeof(int) * wk.size());
    CK(cudaMemcpy(w->work9, wk.data(), sizeof(int) * wk.size(), cudaMemcpyHostToDevice));
    AL(w->t9part, sizeof(double) * w->n_work9 * (NN - Nc) / 2 * PPQ_NA2);
    AL(w->r1part, sizeof(double) * kR1Split * 3 * Nc);
  }
  AL(w->esite, sizeof(double) * Nc); AL(w->epair, sizeof(double) * NN);
  AL(w->part, sizeof(double) * kRedBlocks * (kDiisMax + 2));
  AL(w->scal, sizeof(double) * (kDiisMax + 4)); AL(w->coef, sizeof(double) * kDiisMax);
  AL(w->Bdiis, sizeof(double) * kDiisMax * kDiisMax);
  AL(w->ok, sizeof(int) * 4); AL(w->order, sizeof(int) * kDiisMax);
  if (dc > 0) {
    AL(w->slot_t, sizeof(double) * L * dc);
    AL(w->slot_e, sizeof(double) * L * dc);
  }
#undef AL
  CK(cudaMallocHost((void**)&w->host, sizeof(double) * 64));
  CK(cudaEventCreate(&w->ev0));
  CK(cudaEventCreate(&w->ev1));
  CK(cudaEventCreate(&w->evq0));
  CK(cudaEventCreate(&w->evq1));
  w->N = Nc;
  w->diis_cap = dc;
  return 0;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// validate the pairing: a bijection onto 0..2N-1
int check_pairing(int N, const int* occ, const int* vir, std::vector<int>& lab) {
  if (N < 2) return fail(-1, "n_pairs must be >= 2 (got %d)", N);
  if (!occ || !vir) return fail(-2, "occ_of_pair / vir_of_pair must be non-null host arrays");
  int n = 2 * N;
  lab.assign(n, -1);
  for (int k = 0; k < N; ++k) {
    int o = occ[k], v = vir[k];
    if (o < 0 || o >= n || v < 0 || v >= n)
      return fail(-3, "orbital index out of range in pair %d", k);
    if (lab[o] >= 0 || lab[v] >= 0 || o == v)
      return fail(-3, "orbital listed twice in the pairing (pair %d)", k);
    lab[o] = k;
    lab[v] = k;
  }
  return 0;
}

__global__ void k_count_nonfinite(size_t L, const double* __restrict__ x, int* __restrict__ bad) {
  int b = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) b = 1;
  if (__syncthreads_or(b) && threadIdx.x == 0) atomicOr(bad, 1);
}

__global__ void k_fdiag(int N, int n, const double* __restrict__ f, const int* __restrict__ occ,
                        const int* __restrict__ vir, double* __restrict__ fo, double* __restrict__ fv) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  fo[k] = f[(size_t)occ[k] * n + occ[k]];
  fv[k] = f[(size_t)vir[k] * n + vir[k]];
}

__global__ void k_eref(int N, int n, const double* __restrict__ h, const double* __restrict__ f,
                       const int* __restrict__ occ, double* __restrict__ out) {
  if (threadIdx.x || blockIdx.x) return;
  double s = 0.0;
  for (int k = 0; k < N; ++k) s += h[(size_t)occ[k] * n + occ[k]] + f[(size_t)occ[k] * n + occ[k]];
  out[0] = s;
}

// multi-dot: row 0 = weighted norm^2 of x0; rows 1..m = <e_slot[order[j]], e_new>
__global__ void k_multidot(size_t L, int N, const double* __restrict__ x0, int m,
                           const double* __restrict__ slots, size_t ld, const int* __restrict__ order,
                           int inew, double* __restrict__ part) {
  __shared__ double red[32];
  int row = blockIdx.y;
  const double* a;
  const double* b;
  if (row == 0) { a = x0; b = x0; }
  else { a = slots + (size_t)order[row - 1] * ld; b = slots + (size_t)inew * ld; }
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (size_t)gridDim.x * blockDim.x)
    s += ppq::amp_weight(i, N) * a[i] * b[i];
  s = ppq::block_sum(s, red);
  if (threadIdx.x == 0) part[(size_t)row * gridDim.x + blockIdx.x] = s;
}

// out[r] = sum of part row r (r < rows), one block per row; block `rows`
// writes out[rows] = the energy, sum of the site and (halved) pair elements
__global__ void k_rowsum(int nb, int rows, const double* __restrict__ part, int N,
                         const double* __restrict__ esite, const double* __restrict__ epair,
                         double* __restrict__ out) {
  __shared__ double red[32];
  const int r = blockIdx.x;
  if (r < rows) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[(size_t)r * nb + i];
    s = ppq::block_sum(s, red);
    if (threadIdx.x == 0) out[r] = s;
    return;
  }
  double e = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) e += esite[i];
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) e += 0.5 * epair[i];
  e = ppq::block_sum(e, red);
  if (threadIdx.x == 0) out[rows] = e;
}

// The tensor-core quartic kernels bound every wait; on a timeout they stop,
// drain their copies and MMAs, flag tc_err and poison the residual with a NaN.
// After the stream has synchronised, the host reads the flag (copied beside
// the norm) and turns it into an error with its cause; the flag is cleared so
// the next call starts clean.
int check_tc_flag(Workspace* w, int flag, cudaStream_t s) {
  if (!flag) return 0;
  cudaMemsetAsync(w->tc_err, 0, sizeof(int), s);
  cudaStreamSynchronize(s);
  return fail(-9, "a tensor-core kernel's bounded wait timed out (about 1 s); the residual was poisoned and "
                  "the solve stopped; the device context is intact");
}

struct Problem {
  int N, n;
  const double* h;    // device
  const double* eri;  // device (nullptr when the integrals come as factors)
  const double* Bt = nullptr;  // device [n * n][naux] factors, (pq|rs) = B[pq] . B[rs]
  int naux = 0;
  ppq::EriSrc src() const { return ppq::EriSrc{eri, Bt, naux, n}; }
};

// stage integrals: Fock, h', gathers, denominators
int stage(Workspace* w, const Problem& P, cudaStream_t s) {
  int N = P.N, n = P.n;
  ppq::k_fock<<<(n * n + 127) / 128, 128, 0, s>>>(n, N, P.h, P.src(), w->occ, w->lab, w->f, w->hp);
  k_fdiag<<<1, 256, 0, s>>>(N, n, w->f, w->occ, w->vir, w->fo, w->fv);
  size_t tot = (size_t)N * N * PPQ_NG2 + (size_t)N * PPQ_NG1;
  unsigned nb = (unsigned)((tot + 255) / 256);
  ppq::k_gather<double><<<nb, 256, 0, s>>>(n, N, w->hp, P.src(), w->occ, w->vir, w->g1d, w->g2d);
  ppq::k_gather<float><<<nb, 256, 0, s>>>(n, N, w->hp, P.src(), w->occ, w->vir, w->g1f, w->g2f);
  CK(cudaGetLastError());
  return 0;
}

template <typename R, int MT>
int launch_t9_mt(Workspace* w, int N, cudaStream_t s) {
  int T = (N + MT - 1) / MT;           // thread grid T x T, micro-tile MT x MT
  int nth = ((T * T + 31) / 32) * 32;
  size_t npd = (size_t)T * MT;
  // GEMM tiles, then the [N][29] double row sums (16-byte aligned)
  size_t smem = ((2 * 16 * npd + npd * npd) * sizeof(R) + 15) / 16 * 16 + (size_t)N * PPQ_NA2 * sizeof(double);
  if (smem > 48 * 1024)
    CK(cudaFuncSetAttribute(ppq::k_t9_gemm<R, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid(w->n_work9, N);
  ppq::k_t9_gemm<R, MT><<<grid, nth, smem, s>>>(N, T, cl_ld(N), (const R*)w->clT, (const R*)w->gT,
                                                 w->work9, w->t9part);
  return 0;
}

template <typename R>
int launch_t9_mt_rt(Workspace* w, int N, int mt, cudaStream_t s) {
  switch (mt) {
    case 1: return launch_t9_mt<R, 1>(w, N, s);
    case 2: return launch_t9_mt<R, 2>(w, N, s);
    case 3: return launch_t9_mt<R, 3>(w, N, s);
    case 4: return launch_t9_mt<R, 4>(w, N, s);
    case 5: return launch_t9_mt<R, 5>(w, N, s);
    case 6: return launch_t9_mt<R, 6>(w, N, s);
    case 7: return launch_t9_mt<R, 7>(w, N, s);
    case 8: return launch_t9_mt<R, 8>(w, N, s);
    default: return fail(-5, "n_pairs > 128 is not supported by the quartic kernel");
  }
}

template <typename R, int MT>
int launch_t7_mt(Workspace* w, int N, cudaStream_t s) {
  int T = (N + MT - 1) / MT;
  int nth = ((T * T + 31) / 32) * 32;
  size_t smem = 2 * 16 * (size_t)T * MT * sizeof(R);
  ppq::k_t7_gemm<R, MT><<<PPQ_NK7, nth, smem, s>>>(N, T, cl_ld(N), (const R*)w->pt7T, (const R*)w->clT,
                                                   (R*)w->m7);
  return 0;
}

template <typename R>
int launch_t7_gemm(Workspace* w, int N, int mt, cudaStream_t s) {
  switch (mt) {
    case 1: return launch_t7_mt<R, 1>(w, N, s);
    case 2: return launch_t7_mt<R, 2>(w, N, s);
    case 3: return launch_t7_mt<R, 3>(w, N, s);
    case 4: return launch_t7_mt<R, 4>(w, N, s);
    case 5: return launch_t7_mt<R, 5>(w, N, s);
    case 6: return launch_t7_mt<R, 6>(w, N, s);
    case 7: return launch_t7_mt<R, 7>(w, N, s);
    case 8: return launch_t7_mt<R, 8>(w, N, s);
    default: return fail(-5, "n_pairs > 128 is not supported");
  }
}

// persistent pair closure: about two CTAs per SM, each looping over pairs
template <typename R>
int launch_pair_closure(int N, const R* g2, const double* t1, const double* t2, R* pg, R* pt7, R* pc0,
                        double* epair, R* pt7T, cudaStream_t s) {
  static std::once_flag attr[64];  // per device
  int dev;
  CK(cudaGetDevice(&dev));
  cudaError_t e = cudaSuccess;
  const size_t smem = ppq::ClosureSmem::total<R>();
  std::call_once(attr[dev & 63], [&] {
    e = cudaFuncSetAttribute(ppq::k_pair_closure_p<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return fail(-100, "k_pair_closure_p attribute: %s", cudaGetErrorString(e));
  // resident CTAs on the device, per precision and device (threads of the
  // batched solver may fill an entry concurrently with the same value)
  static std::atomic<int> per_dev[2][64];
  std::atomic<int>& slot = per_dev[sizeof(R) == 4][dev & 63];
  int ps = slot.load(std::memory_order_relaxed);
  if (ps == 0) {
    int nb = 0, nsm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ppq::k_pair_closure_p<R>, 256, smem));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    ps = std::max(1, nb) * std::max(1, nsm);
    slot.store(ps, std::memory_order_relaxed);
  }
  const int grid = std::min(N * N, ps);
  ppq::k_pair_closure_p<R><<<grid, 256, smem, s>>>(N, g2, t1, t2, pg, pt7, pc0, epair, pt7T);
  return 0;
}

// Work list of the tensor-core quartic kernel for N pairs.  A chunk is one
// link pair (c1, c2) with up to four of its g, as many as fit 256 TMEM
// columns at Npad = 16 ceil(N / 16) columns each; the rows (unordered pairs)
// come in tiles of 128, and each CTA takes one tile and a run of chunks of
// about equal cost, about one CTA per SM in all.  Host only.
struct TcPlan {
  int Npad = 0, Kc = 0, nchunks = 0;
  std::vector<int16_t> chunk;  // kChunkFields per chunk
  std::vector<int> cta;        // tile, first chunk, end chunk
};

int plan_tc(int N, TcPlan* pl, int g_cap = 4) {
  if (N < 1 || N > kTcMaxN) return fail(-5, "no tensor-core quartic kernel for n_pairs = %d", N);
  const int Npad = (N + 15) / 16 * 16, Kc = (N + 7) / 8;
  const int max_g = std::max(1, std::min(g_cap, ppq::tc::kMaxCols / Npad));
  pl->chunk.clear();
  pl->cta.clear();
  std::vector<double> cost;
  for (int q0 = 0; q0 < PPQ_NQ9;) {
    int p = ppq_q9_h[2 * q0], q1 = q0;
    while (q1 < PPQ_NQ9 && ppq_q9_h[2 * q1] == p) ++q1;
    int n = q1 - q0, parts = (n + max_g - 1) / max_g;
    for (int k = 0, a = q0; k < parts; ++k) {
      int ng = n / parts + (k < n % parts ? 1 : 0);
      int16_t rec[ppq::tc::kChunkFields] = {0};
      rec[0] = ppq_p9_h[2 * p]; rec[1] = ppq_p9_h[2 * p + 1];
      rec[2] = (int16_t)ng; rec[3] = (int16_t)(ng * Npad);
      int nch = 0;
      for (int j = 0; j < ng; ++j) {
        rec[4 + j] = ppq_q9_h[2 * (a + j) + 1];
        rec[8 + j] = (int16_t)(a + j);
        nch += ppq_c9qp_h[a + j + 1] - ppq_c9qp_h[a + j];
      }
      pl->chunk.insert(pl->chunk.end(), rec, rec + ppq::tc::kChunkFields);
      // MMA clocks (3 TF32 MMAs of 128 x n_cols x 8 per stage) + epilogue loads
      cost.push_back(3.0 * Kc * 128.0 * ng * Npad * 8 / 1620.0 + 8.0 * nch * N);
      a += ng;
    }
    q0 = q1;
  }
  const int nchunks = (int)cost.size();
  const int P = N * (N - 1) / 2, ntiles = (P + ppq::tc::kRows - 1) / ppq::tc::kRows;
  const int nsplit = std::max(1, std::min(nchunks, 152 / std::max(1, ntiles)));
  if (ntiles * nsplit > kTcMaxCtas) return fail(-5, "tensor-core work list too long");
  std::vector<double> pre(nchunks + 1, 0.0);
  for (int i = 0; i < nchunks; ++i) pre[i + 1] = pre[i] + cost[i];
  std::vector<int> bounds(nsplit + 1, 0);
  bounds[nsplit] = nchunks;
  for (int k = 1; k < nsplit; ++k) {
    double target = pre[nchunks] * k / nsplit;
    int i = (int)(std::lower_bound(pre.begin(), pre.end(), target) - pre.begin());
    bounds[k] = std::max(bounds[k - 1], std::min(i, nchunks));
  }
  for (int t = 0; t < ntiles; ++t)
    for (int k = 0; k < nsplit; ++k)
      if (bounds[k + 1] > bounds[k]) {
        pl->cta.push_back(t); pl->cta.push_back(bounds[k]); pl->cta.push_back(bounds[k + 1]);
      }
  pl->Npad = Npad;
  pl->Kc = Kc;
  pl->nchunks = nchunks;
  return 0;
}

int prepare_tc(Workspace* w, int N, cudaStream_t s) {
  TcPlan pl;
  int rc = plan_tc(N, &pl);
  if (rc) return rc;
  if (!pl.cta.empty())
    CK(cudaMemcpyAsync(w->tc_cta, pl.cta.data(), sizeof(int) * pl.cta.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w->tc_chunk, pl.chunk.data(), sizeof(int16_t) * pl.chunk.size(), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  w->tc_Npad = pl.Npad;
  w->tc_Kc = pl.Kc;
  w->tc_nctas = (int)pl.cta.size() / 3;
  const int P = N * (N - 1) / 2, ntiles = (P + ppq::tc::kRows - 1) / ppq::tc::kRows;
  w->tc_nslot = ntiles > 0 ? w->tc_nctas / ntiles : 0;
  if (w->tc_nslot * ntiles != w->tc_nctas || (size_t)w->tc_nslot * P > (size_t)kTcPartRows)
    return fail(-5, "tensor-core work list does not fit its partial buffer");
  // at least 120 KB, so that one CTA (holding all 512 TMEM columns) runs per SM
  w->tc_smem = std::max(ppq::tc::Smem::total(cl_ld(N)), (size_t)120 * 1024);
  w->tc_N = N;
  return 0;
}

template <int NW>
int launch_t9_tc_nw(Workspace* w, int N, cudaStream_t s) {
  static std::once_flag attr[64];  // per device
  int dev;
  CK(cudaGetDevice(&dev));
  cudaError_t e = cudaSuccess;
  std::call_once(attr[dev & 63], [&] {
    e = cudaFuncSetAttribute(ppq::tc::k_t9_tc<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ppq::tc::Smem::total(cl_ld(kTcMaxN)));
  });
  if (e != cudaSuccess) return fail(-100, "k_t9_tc attribute: %s", cudaGetErrorString(e));
  const int P = N * (N - 1) / 2;
  ppq::tc::k_t9_tc<NW><<<w->tc_nctas, ppq::tc::kThreads, w->tc_smem, s>>>(
      N, P, w->tc_Kc, cl_ld(N), (const float*)w->clT, w->bpre, w->tc_cta, w->tc_chunk, w->tc_nslot, w->tc_part,
      w->tc_err);
  return 0;
}

int launch_t9_tc(Workspace* w, int N, cudaStream_t s) {
  if (w->tc_nctas == 0) return 0;  // no unordered pairs
  switch (w->tc_Npad) {
    case 16: return launch_t9_tc_nw<16>(w, N, s);
    case 32: return launch_t9_tc_nw<32>(w, N, s);
    case 48: return launch_t9_tc_nw<48>(w, N, s);
    case 64: return launch_t9_tc_nw<64>(w, N, s);
    case 80: return launch_t9_tc_nw<80>(w, N, s);
    default: return fail(-5, "no tensor-core quartic kernel for n_pairs = %d", N);
  }
}

// FP64 residual: one g per chunk (six accumulator groups fill TMEM)
int prepare_tc64(Workspace* w, int N, cudaStream_t s) {
  TcPlan pl;
  int rc = plan_tc(N, &pl, 1);
  if (rc) return rc;
  if (!pl.cta.empty())
    CK(cudaMemcpyAsync(w->tc64_cta, pl.cta.data(), sizeof(int) * pl.cta.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w->tc64_chunk, pl.chunk.data(), sizeof(int16_t) * pl.chunk.size(), cudaMemcpyHostToDevice,
                     s));
  CK(cudaStreamSynchronize(s));
  w->tc64_Npad = pl.Npad;
  w->tc64_Kc = pl.Kc;
  w->tc64_nctas = (int)pl.cta.size() / 3;
  const int P = N * (N - 1) / 2, ntiles = (P + ppq::tc::kRows - 1) / ppq::tc::kRows;
  w->tc64_nslot = ntiles > 0 ? w->tc64_nctas / ntiles : 0;
  if (w->tc64_nslot * ntiles != w->tc64_nctas || (size_t)w->tc64_nslot * P > (size_t)kTcPartRows)
    return fail(-5, "tensor-core work list does not fit its partial buffer");
  w->tc64_smem = std::max(ppq::tc::Smem64::total(cl_ld(N)), (size_t)120 * 1024);
  w->tc64_N = N;
  return 0;
}

template <int NW>
int launch_t9_tc64_nw(Workspace* w, int N, cudaStream_t s) {
  static std::once_flag attr[64];  // per device
  int dev;
  CK(cudaGetDevice(&dev));
  cudaError_t e = cudaSuccess;
  std::call_once(attr[dev & 63], [&] {
    e = cudaFuncSetAttribute(ppq::tc::k_t9_tc64<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ppq::tc::Smem64::total(cl_ld(kTcMaxN)));
  });
  if (e != cudaSuccess) return fail(-100, "k_t9_tc64 attribute: %s", cudaGetErrorString(e));
  const int P = N * (N - 1) / 2;
  ppq::tc::k_t9_tc64<NW><<<w->tc64_nctas, ppq::tc::kThreads, w->tc64_smem, s>>>(
      N, P, w->tc64_Kc, cl_ld(N), (const double*)w->clT, w->clT2, w->bpre64, w->fexp64, w->tc64_cta,
      w->tc64_chunk, w->tc64_nslot, w->tc64_part, w->tc_err);
  return 0;
}

int launch_t9_tc64(Workspace* w, int N, cudaStream_t s) {
  if (w->tc64_nctas == 0) return 0;  // no unordered pairs
  switch (w->tc64_Npad) {
    case 16: return launch_t9_tc64_nw<16>(w, N, s);
    case 32: return launch_t9_tc64_nw<32>(w, N, s);
    case 48: return launch_t9_tc64_nw<48>(w, N, s);
    case 64: return launch_t9_tc64_nw<64>(w, N, s);
    case 80: return launch_t9_tc64_nw<80>(w, N, s);
    default: return fail(-5, "no tensor-core quartic kernel for n_pairs = %d", N);
  }
}

// Tile autotuner: the micro-tile MT of k_t9_gemm (thread grid ceil(N/MT)^2,
// at most 256 threads) is chosen per (N, precision) by timing every candidate
// once on the stream, the first time that size is seen on this device.
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tuned_mt;  // key (device * 1024 + N, precision)

template <typename R>
int tuned_mt(Workspace* w, int N, cudaStream_t s, int* mt_out) {
  int dev;
  CK(cudaGetDevice(&dev));
  int prec = std::is_same<R, float>::value ? 1 : 0;
  auto key = std::make_pair(dev * 1024 + N, prec);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned_mt.find(key);
    if (it != g_tuned_mt.end()) { *mt_out = it->second; return 0; }
  }
  int lo = (N + 15) / 16;
  if (lo > 8) return fail(-5, "n_pairs > 128 is not supported by the quartic kernel");
  int best = lo;
  float best_ms = 1e30f;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  for (int mt = lo; mt <= std::min(8, lo + 3); ++mt) {
    int rc = launch_t9_mt_rt<R>(w, N, mt, s);  // warm-up
    if (rc) return rc;
    CK(cudaEventRecord(a, s));
    if ((rc = launch_t9_mt_rt<R>(w, N, mt, s))) return rc;
    CK(cudaEventRecord(b, s));
    CK(cudaEventSynchronize(b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    if (ms < best_ms) { best_ms = ms; best = mt; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned_mt[key] = best;
  *mt_out = best;
  return 0;
}

double quartic_flops(int N);

// one residual evaluation at w->t into w->r; energy pieces into esite/epair
template <typename R>
int residual(Workspace* w, int N, cudaStream_t s) {
#define PN(x) (std::is_same<R, float>::value ? x " (FP32)" : x " (FP64)")
  int rc = 0;
  const R* g1 = std::is_same<R, double>::value ? (const R*)w->g1d : (const R*)w->g1f;
  const R* g2 = std::is_same<R, double>::value ? (const R*)w->g2d : (const R*)w->g2f;
  const double* t1 = w->t;
  const double* t2 = w->t + 3 * N;
  R* cl = (R*)w->cl;
  R* hs = (R*)w->hs;
  R* pg = (R*)w->pg;
  R* pt7 = (R*)w->pt7;
  R* pc0 = (R*)w->pc0;
  int NN = N * N;
  ppq::k_links<R><<<(NN + 63) / 64, 64, 0, s>>>(N, t2, cl);
  g_prof.done(PN("ppq::k_links"), s, 0.0, 2.0 * NN * PPQ_NSOP);
  ppq::k_site_closure<R><<<N, 64, 0, s>>>(N, g1, t1, hs, w->esite);
  g_prof.done(PN("ppq::k_site_closure"), s);
  if ((rc = launch_pair_closure<R>(N, g2, t1, t2, pg, pt7, pc0, w->epair, (R*)w->pt7T, s))) return rc;
  g_prof.done(PN("ppq::k_pair_closure_p"), s, 0.0, 2.0 * (NN - N) * (17792.0 + PPQ_PR_N + PPQ_PL_N));
  size_t T36 = (size_t)NN * PPQ_NS36;
  ppq::k_transpose_g<R><<<(unsigned)((T36 + 255) / 256), 256, 0, s>>>(N, pg, (R*)w->gT);
  g_prof.done(PN("ppq::k_transpose_g"), s);
  ppq::k_r1<R><<<dim3(N, kR1Split), 256, sizeof(R) * ppq::kR1Ld * N, s>>>(N, hs, pc0, cl, (const R*)w->gT,
                                                                        w->r1part);
  ppq::k_r1_reduce<R><<<(3 * N + 127) / 128, 128, 0, s>>>(N, kR1Split, hs, w->r1part, w->r);
  g_prof.done(PN("ppq::k_r1, k_r1_reduce"), s, 0.0, 2.0 * N * ((N - 1) * PPQ_NT3 + (double)(N - 1) * (N - 2) * PPQ_NT8));
  ppq::k_transpose_cl<R><<<(unsigned)((T36 + 255) / 256), 256, 0, s>>>(N, cl_ld(N), cl, (R*)w->clT);
  g_prof.done(PN("ppq::k_transpose_cl"), s);
  {
    // T7 as GEMMs over W
    int mt = std::max(1, (N + 15) / 16);
    if ((rc = launch_t7_gemm<R>(w, N, mt, s))) return rc;
  }
  g_prof.done(PN("ppq::k_t7_gemm"), s, 0.0, 2.0 * PPQ_NK7 * (double)N * N * N);
  {
    // staged rows of the T4 sum: 2 kR1Ld + 3 values per X (78.8 KB in FP64 at N = 128)
    static std::once_flag attr[64][2];
    int dev;
    CK(cudaGetDevice(&dev));
    cudaError_t e = cudaSuccess;
    std::call_once(attr[dev & 63][sizeof(R) == 8], [&] {
      e = cudaFuncSetAttribute(ppq::k_r2<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(sizeof(R) * 128 * (2 * ppq::kR1Ld + 3)));
    });
    if (e != cudaSuccess) return fail(-100, "k_r2 attribute: %s", cudaGetErrorString(e));
    ppq::k_r2<R><<<NN, 256, sizeof(R) * N * (2 * ppq::kR1Ld + 3), s>>>(N, hs, pc0, (const R*)w->m7, pg, cl, t2,
                                                                       w->dir, w->abuf);
  }
  g_prof.done(PN("ppq::k_r2"), s, 0.0, 2.0 * ((NN - N) / 2.0 * (N - 2) * PPQ_NT4 + (NN - N) * (double)(PPQ_NT2 + PPQ_NT7 + PPQ_NSOP)));
  // quartic term
  if (std::is_same<R, float>::value && w->tc_N == N) {
    // tensor cores: split B operands, then the fused MMA + W-contraction kernel
    size_t nb = (size_t)PPQ_NS36 * w->tc_Kc * w->tc_Npad * 8;
    ppq::tc::k_t9_bprep<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(N, w->tc_Npad, w->tc_Kc, (const float*)pg,
                                                                       w->bpre);
    g_prof.done(PN("tc::k_t9_bprep"), s);
    if (w->profile) CK(cudaEventRecord(w->evq0, s));
    if ((rc = launch_t9_tc(w, N, s))) return rc;
    if (w->profile) CK(cudaEventRecord(w->evq1, s));
    g_prof.done("tc::k_t9_tc (FP32 quartic, 3xTF32 tcgen05)", s, 0.0, quartic_flops(N));
    ppq::k_t9_reduce<float><<<(unsigned)((NN * PPQ_NA2 + 255) / 256), 256, 0, s>>>(N, w->tc_nslot, w->tc_part,
                                                                                   w->t9);
    g_prof.done(PN("ppq::k_t9_reduce"), s);
    w->n_launches += 3;
  } else if (std::is_same<R, double>::value && w->tc64_N == N) {
    // tensor cores, exact splitting: split B operands, then the MMA + W-contraction kernel
    ppq::tc::k_t9_bprep64<<<PPQ_NS36, 128, 0, s>>>(
        N, w->tc64_Npad, w->tc64_Kc, (const double*)pg, w->bpre64, w->fexp64);
    size_t ncl = (size_t)cl_ld(N) * PPQ_NS36;
    ppq::tc::k_split_cl<<<(unsigned)((ncl + 255) / 256), 256, 0, s>>>(ncl, (const double*)w->clT, w->clT2);
    g_prof.done(PN("tc::k_t9_bprep64"), s);
    if (w->profile) CK(cudaEventRecord(w->evq0, s));
    if ((rc = launch_t9_tc64(w, N, s))) return rc;
    if (w->profile) CK(cudaEventRecord(w->evq1, s));
    g_prof.done("tc::k_t9_tc64 (FP64 quartic, exact splitting on tcgen05)", s, 0.0, quartic_flops(N));
    ppq::k_t9_reduce<double><<<(unsigned)((NN * PPQ_NA2 + 255) / 256), 256, 0, s>>>(N, w->tc64_nslot,
                                                                                    w->tc64_part, w->t9);
    g_prof.done(PN("ppq::k_t9_reduce"), s);
    w->n_launches += 4;
  } else {
    // SIMT: GEMM over the transposed operands, W-contraction
    if (w->profile) CK(cudaEventRecord(w->evq0, s));
    if ((rc = launch_t9_mt_rt<R>(w, N, w->mt[std::is_same<R, float>::value ? 1 : 0], s))) return rc;
    if (w->profile) CK(cudaEventRecord(w->evq1, s));
    g_prof.done("ppq::k_t9_gemm (quartic, SIMT)", s, 0.0, quartic_flops(N));
    ppq::k_t9_reduce<double><<<(unsigned)((NN * PPQ_NA2 + 255) / 256), 256, 0, s>>>(N, w->n_work9, w->t9part,
                                                                                    w->t9);
    w->n_launches += 2;
  }
  size_t L2 = (size_t)NN * PPQ_NA2;
  ppq::k_assemble<<<(unsigned)((L2 + 255) / 256), 256, 0, s>>>(N, w->dir, w->abuf, w->t9, w->r + 3 * N);
  g_prof.done(PN("ppq::k_t9_reduce, k_assemble"), s);
  CK(cudaGetLastError());
  w->n_launches += 10;   // the launches common to the three quartic forms
  return 0;
#undef PN
}

// One residual evaluation.  On a non-default stream the pipeline is captured
// once per (workspace, N, precision) as a CUDA graph and replayed afterwards.
int run_residual(Workspace* w, int N, int precision, cudaStream_t s) {
  int rc;
  int p = precision ? 1 : 0;
  if (precision && w->tc_allowed && N <= kTcMaxN) {
    if (w->tc_N != N && (rc = prepare_tc(w, N, s))) return rc;
  } else if (!precision && w->tc_allowed && N <= kTcMaxN) {
    if (w->tc64_N != N && (rc = prepare_tc64(w, N, s))) return rc;
  } else if (precision) {
    if ((rc = tuned_mt<float>(w, N, s, &w->mt[1]))) return rc;
  } else {
    if ((rc = tuned_mt<double>(w, N, s, &w->mt[0]))) return rc;
  }
  if (s == 0 || g_prof.on) return precision ? residual<float>(w, N, s) : residual<double>(w, N, s);
  if (!w->graph[p] || w->graph_N[p] != N || w->graph_profile[p] != (int)w->profile) {
    if (w->graph[p]) { cudaGraphExecDestroy(w->graph[p]); w->graph[p] = nullptr; }
    cudaGraph_t g;
    int nl = w->n_launches;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    rc = precision ? residual<float>(w, N, s) : residual<double>(w, N, s);
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(-100, "graph capture failed: %s", cudaGetErrorString(e));
    CK(cudaGraphInstantiate(&w->graph[p], g, 0));
    cudaGraphDestroy(g);
    w->graph_N[p] = N;
    w->graph_profile[p] = (int)w->profile;
    w->graph_launches[p] = w->n_launches - nl;
    w->n_launches = nl;
  }
  CK(cudaGraphLaunch(w->graph[p], s));
  w->n_launches += w->graph_launches[p];
  return 0;
}

// algorithmic FLOPs of one k_t9_gemm launch: for each unordered pair Y < Z and
// each of the NQ9 (c1, c2, g) combinations, sum over X (N) for every W (N)
double quartic_flops(int N) {
  double n = N;
  return 2.0 * (n * (n - 1) / 2) * (PPQ_NQ9 * n * n + PPQ_NC9 * n);  // GEMM + fused W-contraction
}

double residual_flops(int N) {
  double n = N, pairs = n * (n - 1);
  double fma = 0.0;
  fma += pairs * PPQ_NSOP;                                                  // links
  fma += n * (PPQ_H1_NEL + 2 * 3 * 16 * 3);                                 // site closures (approx)
  fma += pairs * (17792.0 + PPQ_PR_N + PPQ_PL_N);                           // pair closures
  fma += n * ((n - 1) * PPQ_NT3 + (n - 1) * (n - 2) * PPQ_NT8);             // r1
  fma += pairs / 2 * (n - 2) * PPQ_NT4 + pairs * (PPQ_NT2 + PPQ_NT7 + PPQ_NSOP);  // r2
  fma += (double)PPQ_NK7 * n * n * n;                                        // T7 GEMMs
  fma += (pairs / 2) * (n * n * PPQ_NQ9 + n * PPQ_NC9);                      // quartic
  return 2.0 * fma;
}

// common entry preparation on a given workspace: pairing, staged inputs
int prepare_ws(Workspace* w, int N, const int* occ, const int* vir, const double* h,
               const double* eri, int diis, cudaStream_t s, Problem* P) {
  std::vector<int> lab;
  int rc = check_pairing(N, occ, vir, lab);
  if (rc) return rc;
  if (!h || !eri) return fail(-2, "h and eri must be non-null");
  if ((rc = grow(w, N, diis))) return rc;
  int n = 2 * N;
  CK(cudaMemcpyAsync(w->occ, occ, sizeof(int) * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w->vir, vir, sizeof(int) * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w->lab, lab.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
  P->N = N;
  P->n = n;
  size_t n4 = (size_t)n * n * n * n;
  if (is_device_ptr(h)) P->h = h;
  else {
    CK(cudaMemcpyAsync(w->h, h, sizeof(double) * n * n, cudaMemcpyHostToDevice, s));
    P->h = w->h;
  }
  void* mapped = nullptr;
  if (is_device_ptr(eri)) P->eri = eri;
  else if (cudaHostGetDevicePointer(&mapped, const_cast<double*>(eri), 0) == cudaSuccess && mapped) {
    // pinned host integrals mapped into the device address space: the screen
    // and the staging kernels read them over the host link, no n^4 copy
    P->eri = (const double*)mapped;
  } else {
    cudaGetLastError();   // pageable host memory: copy it
    if (w->eri_cap < n4) {
      if (w->eri) cudaFree(w->eri);
      w->eri = nullptr;
      CK(cudaMalloc((void**)&w->eri, sizeof(double) * n4));
      w->eri_cap = n4;
    }
    CK(cudaMemcpyAsync(w->eri, eri, sizeof(double) * n4, cudaMemcpyHostToDevice, s));
    P->eri = w->eri;
  }
  // non-finite screen
  CK(cudaMemsetAsync(w->ok, 0, sizeof(int), s));
  k_count_nonfinite<<<kRedBlocks, 256, 0, s>>>((size_t)n * n, P->h, w->ok);
  k_count_nonfinite<<<kRedBlocks * 4, 256, 0, s>>>(n4, P->eri, w->ok);
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, w->ok, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad) return 3;
  if ((rc = stage(w, *P, s))) return rc;
  return 0;
}

// the same on the per-device cached workspace
int prepare(int N, const int* occ, const int* vir, const double* h, const double* eri, int diis,
            cudaStream_t s, Workspace** pw, Problem* P) {
  std::vector<int> lab;
  int rc = check_pairing(N, occ, vir, lab);  // argument errors before any device call
  if (rc) return rc;
  int dev;
  CK(cudaGetDevice(&dev));
  Workspace*& w = g_ws[dev];
  if (!w) w = new Workspace();
  *pw = w;
  return prepare_ws(w, N, occ, vir, h, eri, diis, s, P);
}

// B[Q][pq] -> Bt[pq][Q] (the factor of one integral index pair contiguous)
__global__ void k_transpose_B(int naux, size_t n2, const double* __restrict__ B, double* __restrict__ Bt) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n2 * naux) return;
  size_t pq = i / naux, Q = i % naux;
  Bt[i] = B[Q * n2 + pq];
}

// entry preparation from three-index factors B[Q][p][q], (pq|rs) = sum_Q
// B[Q][p][q] B[Q][r][s]: pairing, h and B on the device (B transposed to
// [pq][Q]), non-finite screen, staging from the factors
int prepare_cd(int N, const int* occ, const int* vir, const double* h, const double* B, int naux, int diis,
               cudaStream_t s, Workspace** pw, Problem* P) {
  std::vector<int> lab;
  int rc = check_pairing(N, occ, vir, lab);
  if (rc) return rc;
  if (!h || !B) return fail(-2, "h and B must be non-null");
  if (naux < 1) return fail(-2, "naux must be >= 1");
  int dev;
  CK(cudaGetDevice(&dev));
  Workspace*& w = g_ws[dev];
  if (!w) w = new Workspace();
  *pw = w;
  if ((rc = grow(w, N, diis))) return rc;
  int n = 2 * N;
  size_t n2 = (size_t)n * n, nb = n2 * naux;
  CK(cudaMemcpyAsync(w->occ, occ, sizeof(int) * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w->vir, vir, sizeof(int) * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w->lab, lab.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
  P->N = N;
  P->n = n;
  P->eri = nullptr;
  if (is_device_ptr(h)) P->h = h;
  else {
    CK(cudaMemcpyAsync(w->h, h, sizeof(double) * n2, cudaMemcpyHostToDevice, s));
    P->h = w->h;
  }
  // factors: raw copy (when on the host) and the transposed working copy
  if (w->cd_cap < nb) {
    if (w->Bcd) cudaFree(w->Bcd);
    if (w->Bt) cudaFree(w->Bt);
    w->Bcd = w->Bt = nullptr;
    w->cd_cap = 0;
    CK(cudaMalloc((void**)&w->Bcd, sizeof(double) * nb));
    CK(cudaMalloc((void**)&w->Bt, sizeof(double) * nb));
    w->cd_cap = nb;
  }
  const double* Bd = B;
  if (!is_device_ptr(B)) {
    CK(cudaMemcpyAsync(w->Bcd, B, sizeof(double) * nb, cudaMemcpyHostToDevice, s));
    Bd = w->Bcd;
  }
  k_transpose_B<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(naux, n2, Bd, w->Bt);
  P->Bt = w->Bt;
  P->naux = naux;
  CK(cudaMemsetAsync(w->ok, 0, sizeof(int), s));
  k_count_nonfinite<<<kRedBlocks, 256, 0, s>>>(n2, P->h, w->ok);
  k_count_nonfinite<<<kRedBlocks, 256, 0, s>>>(nb, w->Bt, w->ok);
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, w->ok, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad) return 3;
  return stage(w, *P, s);
}

int copy_amps(double* dst, const double* src, size_t L, cudaStream_t s) {
  CK(cudaMemcpyAsync(dst, src, sizeof(double) * L, cudaMemcpyDefault, s));
  return 0;
}

}  // namespace

// ---------------------------------------------------------------- adjoint driver
int grow_adjoint(Workspace* w, int N) {
  if (w->adjN >= N) return 0;
  void** ps[] = {(void**)&w->clb, (void**)&w->hsb, (void**)&w->pgb, (void**)&w->pt7b, (void**)&w->pc0b,
                 (void**)&w->dirb, (void**)&w->abufb, (void**)&w->t9b, (void**)&w->gt, (void**)&w->gu,
                 (void**)&w->B9a, (void**)&w->B9b, (void**)&w->lam};
  for (void** p : ps)
    if (*p) { cudaFree(*p); *p = nullptr; }
  size_t NN = (size_t)N * N, L = amp_len(N);
  CK(cudaMalloc((void**)&w->clb, sizeof(double) * NN * PPQ_NS36));
  CK(cudaMalloc((void**)&w->hsb, sizeof(double) * N * 256));
  CK(cudaMalloc((void**)&w->pgb, sizeof(double) * NN * PPQ_NS36));
  CK(cudaMalloc((void**)&w->pt7b, sizeof(double) * NN * PPQ_NT7E));
  CK(cudaMalloc((void**)&w->pc0b, sizeof(double) * NN * PPQ_NCOL0));
  CK(cudaMalloc((void**)&w->dirb, sizeof(double) * NN * PPQ_NA2));
  CK(cudaMalloc((void**)&w->abufb, sizeof(double) * NN * PPQ_NA2));
  CK(cudaMalloc((void**)&w->t9b, sizeof(double) * NN * PPQ_NA2));
  CK(cudaMalloc((void**)&w->gt, sizeof(double) * L));
  CK(cudaMalloc((void**)&w->gu, sizeof(double) * L));
  CK(cudaMalloc((void**)&w->B9a, sizeof(double) * NN * N * PPQ_NQ9));
  CK(cudaMalloc((void**)&w->B9b, sizeof(double) * NN * N * PPQ_NQ9));
  CK(cudaMalloc((void**)&w->lam, sizeof(double) * L));
  w->adjN = N;
  return 0;
}

// grad_t L(t, lambda) for t = w->t, lambda = lam (stored layout, consistent
// copies) into w->gu (gradient w.r.t. unique amplitudes, in both copies);
// also leaves R(t) in w->r and the energy pieces (FP64 forward pass)
int lagrangian_gradient(Workspace* w, int N, const double* lam, cudaStream_t s,
                        bool integral_adjoints = false) {
  int rc = grow_adjoint(w, N);
  if (rc) return rc;
  size_t NN = (size_t)N * N, L = amp_len(N);
  if ((rc = run_residual(w, N, 0, s))) return rc;
  const double* t1 = w->t;
  const double* t2 = w->t + 3 * N;
  CK(cudaMemsetAsync(w->clb, 0, sizeof(double) * NN * PPQ_NS36, s));
  CK(cudaMemsetAsync(w->hsb, 0, sizeof(double) * N * 256, s));
  CK(cudaMemsetAsync(w->pgb, 0, sizeof(double) * NN * PPQ_NS36, s));
  CK(cudaMemsetAsync(w->pt7b, 0, sizeof(double) * NN * PPQ_NT7E, s));
  CK(cudaMemsetAsync(w->pc0b, 0, sizeof(double) * NN * PPQ_NCOL0, s));
  CK(cudaMemsetAsync(w->gt, 0, sizeof(double) * L, s));
  size_t L2 = NN * PPQ_NA2;
  unsigned b2 = (unsigned)((L2 + 255) / 256);
  const double* cl = (const double*)w->cl;
  const double* hs = (const double*)w->hs;
  const double* pg = (const double*)w->pg;
  const double* pt7 = (const double*)w->pt7;
  ppq::adj::k_assemble<<<b2, 256, 0, s>>>(N, lam + 3 * N, w->dirb, w->abufb, w->t9b);
  ppq::adj::k_r1<<<N, 256, 0, s>>>(N, lam, hs, cl, pg, w->hsb, w->pc0b, w->clb, w->pgb);
  ppq::adj::k_r2<<<(unsigned)NN, 128, 0, s>>>(N, w->dirb, w->abufb, t2, hs, cl, pt7, w->hsb, w->clb,
                                              w->pt7b, w->pc0b, w->gt + 3 * N);
  ppq::adj::k_b9<<<(unsigned)NN, 256, 0, s>>>(N, cl, pg, w->B9a);
  ppq::adj::k_t9_epi<<<(unsigned)NN, 256, 0, s>>>(N, w->t9b, w->B9a, cl, w->B9b, w->clb);
  unsigned bn = (unsigned)((NN + 63) / 64);
  ppq::adj::k_t9_gbar<<<bn, 64, 0, s>>>(N, w->B9b, cl, w->pgb);
  ppq::adj::k_t9_clbar<<<bn, 64, 0, s>>>(N, w->B9b, cl, pg, w->clb);
  size_t smem = 2 * sizeof(double) * PPQ_BLK;
  CK(cudaFuncSetAttribute(ppq::adj::k_pair_closure, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ppq::adj::k_pair_closure<<<(unsigned)NN, 256, smem, s>>>(N, w->g2d, t1, t2, w->pgb, w->pt7b, w->pc0b, w->gt,
                                                            integral_adjoints ? w->gb2 : nullptr);
  ppq::adj::k_site_closure<<<N, 64, 0, s>>>(N, w->g1d, t1, w->hsb, w->gt, integral_adjoints ? w->gb1 : nullptr);
  ppq::adj::k_links<<<bn, 64, 0, s>>>(N, t2, w->clb, w->gt + 3 * N);
  CK(cudaMemcpyAsync(w->gu, w->gt, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s));
  ppq::adj::k_unique<<<b2, 256, 0, s>>>(N, w->gt + 3 * N, w->gu + 3 * N);
  CK(cudaGetLastError());
  w->n_launches += 13;
  return 0;
}

// dE_total/dh, dE_total/d(pq|rs) and dE/dkappa at converged t (w->t) and
// lambda (w->lam): dL/d(gathered integrals) from the closure adjoints, the
// transposed gather, the chain rule through h' and E_ref, 8-fold symmetrisation
int integral_gradients(Workspace* w, const Problem& P, cudaStream_t s) {
  int N = P.N, n = P.n;
  size_t n2 = (size_t)n * n, n4 = n2 * n2, NN = (size_t)N * N;
  if (w->grad_n < (size_t)n) {
    void** ps[] = {(void**)&w->gb1, (void**)&w->gb2, (void**)&w->gh_raw, (void**)&w->gh,
                   (void**)&w->gv_raw, (void**)&w->gv, (void**)&w->dk, (void**)&w->ab};
    for (void** p : ps)
      if (*p) { cudaFree(*p); *p = nullptr; }
    CK(cudaMalloc((void**)&w->gb1, sizeof(double) * N * PPQ_NG1));
    CK(cudaMalloc((void**)&w->gb2, sizeof(double) * NN * PPQ_NG2));
    CK(cudaMalloc((void**)&w->gh_raw, sizeof(double) * n2));
    CK(cudaMalloc((void**)&w->gh, sizeof(double) * n2));
    CK(cudaMalloc((void**)&w->gv_raw, sizeof(double) * n4));
    CK(cudaMalloc((void**)&w->gv, sizeof(double) * n4));
    CK(cudaMalloc((void**)&w->dk, sizeof(double) * n2));
    CK(cudaMalloc((void**)&w->ab, sizeof(double) * 2 * n2));
    w->grad_n = n;
  }
  int rc = lagrangian_gradient(w, N, w->lam, s, true);
  if (rc) return rc;
  // dh' into gh (scratch), dv into gv_raw
  CK(cudaMemsetAsync(w->gh, 0, sizeof(double) * n2, s));
  CK(cudaMemsetAsync(w->gv_raw, 0, sizeof(double) * n4, s));
  size_t tot = NN * PPQ_NG2 + (size_t)N * PPQ_NG1;
  ppq::adj::k_scatter_gather<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, N, w->gb1, w->gb2, w->occ,
                                                                            w->vir, w->gh, w->gv_raw);
  ppq::adj::k_grad_chain<<<(unsigned)((n2 + 127) / 128), 128, 0, s>>>(n, N, w->gh, w->occ, w->lab,
                                                                      w->gh_raw, w->gv_raw, 1);
  ppq::adj::k_sym_h<<<(unsigned)((n2 + 127) / 128), 128, 0, s>>>(n, w->gh_raw, w->gh);
  ppq::adj::k_sym_v<<<(unsigned)((n4 + 255) / 256), 256, 0, s>>>(n, w->gv_raw, w->gv);
  ppq::adj::k_orbital_grad<<<(unsigned)((n2 + 127) / 128), 128, 0, s>>>(n, P.h, P.eri, w->gh, w->gv, w->ab);
  ppq::adj::k_orbital_final<<<(unsigned)((n2 + 127) / 128), 128, 0, s>>>(n, w->ab, w->dk);
  CK(cudaGetLastError());
  w->n_launches += 6;
  return 0;
}

// ---------------------------------------------------------------- solver pieces
__global__ void k_absmax(size_t L, const double* __restrict__ x, unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// t = tb + (eta / max|x|) x
__global__ void k_fd_point(size_t L, const double* __restrict__ tb, const double* __restrict__ x,
                           const unsigned long long* __restrict__ amax, double eta, double* __restrict__ t) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  double m = __longlong_as_double((long long)*amax);
  t[i] = tb[i] + (m > 0.0 ? eta / m : 0.0) * x[i];
}

// rho = r64 + (r - rb) * max|x| / eta   (r64 + J x by a forward difference)
__global__ void k_fd_rho(size_t L, const double* __restrict__ r64, const double* __restrict__ r,
                         const double* __restrict__ rb, const unsigned long long* __restrict__ amax,
                         double eta, double* __restrict__ rho) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  double m = __longlong_as_double((long long)*amax);
  rho[i] = r64[i] + (m > 0.0 ? (r[i] - rb[i]) * (m / eta) : 0.0);
}

__global__ void k_axpy_to(size_t L, const double* __restrict__ a, const double* __restrict__ b,
                          double* __restrict__ out) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L) out[i] = a[i] + b[i];
}

// Pulay DIIS on the device: B (kDiis x kDiis, by slot id) gains the new row
// from dots[1..m]; the bordered system [B -1; -1 0][c; l] = [0; -1] over the
// active slots (order[0..m), newest last) is solved in FP64 by one warp (a
// lane per row, partial pivoting; back-substitution by lane 0), the error
// block scaled by the power of two at or above its largest diagonal (exact;
// c unchanged).  Divisions are few (FP64 division is long on this part): one
// reciprocal of the pivot per column and one of each diagonal;
// coef = c, or the newest iterate alone if the system is singular or
// extrapolation is off.
__global__ void __launch_bounds__(32) k_diis_solve(int m, const int* __restrict__ order, int inew,
                                                   const double* __restrict__ dots, double* __restrict__ B, int ldb,
                                                   int extrap, double* __restrict__ coef) {
  // one warp: lane r owns row r of the bordered system (at most 17 rows)
  __shared__ double A[17][19];
  __shared__ int ord[16];
  const int lane = threadIdx.x;
  if (lane < m) ord[lane] = order[lane];
  __syncwarp();
  if (lane < m) {
    double d = dots[1 + lane];
    B[ord[lane] * ldb + inew] = d;
    B[inew * ldb + ord[lane]] = d;
  }
  __threadfence_block();
  __syncwarp();
  if (lane < m) coef[lane] = lane == m - 1 ? 1.0 : 0.0;
  if (!extrap || m < 2) return;
  const int nn = m + 1;
  double dd = lane < m ? fabs(B[ord[lane] * ldb + ord[lane]]) : 0.0;
  for (int o = 16; o > 0; o >>= 1) dd = fmax(dd, __shfl_xor_sync(0xffffffffu, dd, o));
  int ex = 0;
  if (dd > 0.0) frexp(dd, &ex);
  const double isc = ldexp(1.0, -ex);
  if (lane < nn) {
    for (int j = 0; j < m; ++j) A[lane][j] = lane < m ? B[ord[lane] * ldb + ord[j]] * isc : -1.0;
    A[lane][m] = lane < m ? -1.0 : 0.0;
    A[lane][nn] = lane < m ? 0.0 : -1.0;
  }
  __syncwarp();
  for (int col = 0; col < nn; ++col) {
    // partial pivot: the first row of largest |A[r][col]|, r >= col
    double v = (lane >= col && lane < nn) ? fabs(A[lane][col]) : -1.0;
    int idx = lane;
    for (int o = 16; o > 0; o >>= 1) {
      double v2 = __shfl_xor_sync(0xffffffffu, v, o);
      int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
      if (v2 > v || (v2 == v && i2 < idx)) { v = v2; idx = i2; }
    }
    if (fabs(A[idx][col]) < 1e-300) return;  // singular: keep the newest iterate
    if (idx != col && lane <= nn) {
      double x = A[col][lane];
      A[col][lane] = A[idx][lane];
      A[idx][lane] = x;
    }
    __syncwarp();
    const double ip = 1.0 / A[col][col];
    if (lane > col && lane < nn) {
      double f = A[lane][col] * ip;
      for (int q = col; q <= nn; ++q) A[lane][q] -= f * A[col][q];
    }
    __syncwarp();
  }
  __shared__ double idg[17];
  if (lane < nn) idg[lane] = 1.0 / A[lane][lane];
  __syncwarp();
  if (lane == 0) {
    double x[17];
    for (int r2 = nn - 1; r2 >= 0; --r2) {
      double s = A[r2][nn];
      for (int q = r2 + 1; q < nn; ++q) s -= A[r2][q] * x[q];
      x[r2] = s * idg[r2];
    }
    bool finite = true;
    for (int j = 0; j < m; ++j) finite = finite && isfinite(x[j]);
    if (finite)
      for (int j = 0; j < m; ++j) coef[j] = x[j];
  }
}

__global__ void k_extrap(size_t L, int m, const double* __restrict__ coef, const double* __restrict__ slots,
                         size_t ld, const int* __restrict__ order, double* __restrict__ t) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  double s = 0.0;
  for (int q = 0; q < m; ++q) s += coef[q] * slots[(size_t)order[q] * ld + i];
  t[i] = s;
}


// Pulay DIIS ring: slot ids, oldest first (the error-dot matrix lives on the
// device, indexed by slot id)
struct Diis {
  int m_max;
  std::vector<int> ring;
  explicit Diis(int m) : m_max(m) {}
  void reset() { ring.clear(); }
};

// The iteration machinery of pq_solve around the residual pipeline.
struct Solver {
  Workspace* w;
  int N;
  size_t L;
  ppq_opts o;
  cudaStream_t s;
  unsigned lb;
  int evals = 0, evals32 = 0, polish_evals = 0;
  double t_res_ms = 0.0;
  double last_outer = 0.0;
  double last_norm2 = 0.0;
  Solver(Workspace* w_, int N_, size_t L_, const ppq_opts& o_, cudaStream_t s_)
      : w(w_), N(N_), L(L_), o(o_), s(s_), lb((unsigned)((L_ + 255) / 256)) {}

  int cur_prec = 0;
  // residual at w->t (precision prec) into w->r; ||R|| and E_c to the host
  int eval(int prec, double* res, double* e) {
    cur_prec = prec;
    CK(cudaEventRecord(w->ev0, s));
    int rc = run_residual(w, N, prec, s);
    if (rc) return rc;
    CK(cudaEventRecord(w->ev1, s));
    dim3 g(kRedBlocks, 1);
    k_multidot<<<g, 256, 0, s>>>(L, N, w->r, 0, w->slot_e, L, w->order, 0, w->part);
    k_rowsum<<<2, 256, 0, s>>>(kRedBlocks, 1, w->part, N, w->esite, w->epair, w->scal);
    CK(cudaMemcpyAsync(w->host, w->scal, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(w->host + 60, w->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    g_prof.done("solver: norm, energy, device-to-host", s, 8.0 * L);
    CK(cudaStreamSynchronize(s));
    if (int rc2 = check_tc_flag(w, *(int*)(w->host + 60), s)) return rc2;
    w->n_launches += 2;
    account();
    evals++;
    if (prec) evals32++;
    last_norm2 = w->host[0];
    *res = sqrt(w->host[0]);
    *e = w->host[1];
    if (trace_on())
      fprintf(stderr, "ppq eval %4d %s |R| %.3e E_c %.12f\n", evals, prec ? "fp32" : "fp64", *res, *e);
    return 0;
  }

  void account() {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, w->ev0, w->ev1);
    t_res_ms += ms;
    if (w->profile) {
      float mq = 0.f;
      cudaEventElapsedTime(&mq, w->evq0, w->evq1);
      w->t_quartic_ms += mq;
      w->n_quartic++;
      if (cur_prec) {
        w->t_quartic32_ms += mq;
        w->n_quartic32++;
      }
    }
  }

  // Jacobi step x <- x + res / D with DIIS over the slots; `it` counts steps
  int diis_step(Diis& d, double* x, const double* res, int it) {
    int slot = (int)d.ring.size() < d.m_max ? (int)d.ring.size() : d.ring.front();
    double* st = w->slot_t + (size_t)slot * L;
    double* se = w->slot_e + (size_t)slot * L;
    ppq::k_jacobi<<<lb, 256, 0, s>>>(L, N, x, res, w->fo, w->fv, o.level_shift, st, se);
    std::vector<int> act;
    for (int id : d.ring) if (id != slot) act.push_back(id);
    if ((int)act.size() >= d.m_max) act.erase(act.begin());
    act.push_back(slot);
    int m = (int)act.size();
    memcpy(w->host + 48, act.data(), sizeof(int) * m);
    CK(cudaMemcpyAsync(w->order, w->host + 48, sizeof(int) * m, cudaMemcpyHostToDevice, s));
    dim3 g(kRedBlocks, 1 + m);
    k_multidot<<<g, 256, 0, s>>>(L, N, res, m, w->slot_e, L, w->order, slot, w->part);
    k_rowsum<<<m + 2, 256, 0, s>>>(kRedBlocks, 1 + m, w->part, N, w->esite, w->epair, w->scal);
    d.ring = act;
    // bordered least squares and extrapolation on the device (no host round trip)
    int extrap = o.diis_dim > 0 && it >= o.diis_start && m > 1;
    k_diis_solve<<<1, 32, 0, s>>>(m, w->order, slot, w->scal, w->Bdiis, kDiisMax, extrap, w->coef);
    k_extrap<<<lb, 256, 0, s>>>(L, m, w->coef, w->slot_t, L, w->order, x);
    w->n_launches += 5;
    g_prof.done("solver: Jacobi, DIIS, extrapolation", s, 8.0 * L * (4 + 2 * m));
    CK(cudaGetLastError());
    return 0;
  }

  int step_plain(Diis& d, int it) { return diis_step(d, w->t, w->r, it); }

  // Energy after one plain Jacobi step t + R / D (w->r holds R(t)), from the
  // closures alone: the site and pair closures in FP64 and the FP64 sum, about
  // a twentieth of a full FP64 residual.  Scratch: w->tb, w->del and the
  // closure buffers, all rewritten by the next evaluation.
  int jacobi_energy(double* e_next) {
    double* tn = w->tb;
    ppq::k_jacobi<<<lb, 256, 0, s>>>(L, N, w->t, w->r, w->fo, w->fv, o.level_shift, tn, w->del);
    ppq::k_site_closure<double><<<N, 64, 0, s>>>(N, w->g1d, tn, (double*)w->hs, w->esite);
    int rc = launch_pair_closure<double>(N, w->g2d, tn, tn + 3 * N, (double*)w->pg, (double*)w->pt7,
                                         (double*)w->pc0, w->epair, (double*)w->pt7T, s);
    if (rc) return rc;
    k_rowsum<<<1, 256, 0, s>>>(0, 0, w->part, N, w->esite, w->epair, w->scal);
    CK(cudaMemcpyAsync(w->host, w->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    g_prof.done("solver: energy of one more Jacobi step (closures, FP64)", s);
    CK(cudaStreamSynchronize(s));
    w->n_launches += 4;
    *e_next = w->host[0];
    if (trace_on()) fprintf(stderr, "ppq jacobi-step energy %.12f\n", *e_next);
    return 0;
  }

  // Lambda equations at the converged t in w->t: grad_t L(t, lambda) = 0 by
  // Jacobi steps lambda += grad / D with DIIS (FP64)
  int solve_lambda(double tol, int max_iter, double* res_out, int* iters_out) {
    int rc;
    CK(cudaMemsetAsync(w->lam, 0, sizeof(double) * L, s));
    Diis d(o.diis_dim > 0 ? o.diis_dim : 1);
    double res = 0.0;
    int it = 1;
    for (; it <= max_iter; ++it) {
      if ((rc = lagrangian_gradient(w, N, w->lam, s))) return rc;
      dim3 g(kRedBlocks, 1);
      k_multidot<<<g, 256, 0, s>>>(L, N, w->gu, 0, w->slot_e, L, w->order, 0, w->part);
      k_rowsum<<<2, 256, 0, s>>>(kRedBlocks, 1, w->part, N, w->esite, w->epair, w->scal);
      CK(cudaMemcpyAsync(w->host, w->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      res = sqrt(w->host[0]);
      if (trace_on()) fprintf(stderr, "ppq lambda %3d |grad_t L| %.3e\n", it, res);
      if (!isfinite(res) || res > 1e6) { *res_out = res; *iters_out = it; return 2; }
      if (res <= tol) break;
      if ((rc = diis_step(d, w->lam, w->gu, it))) return rc;
    }
    *res_out = res;
    *iters_out = it > max_iter ? max_iter : it;
    return it > max_iter ? 1 : 0;
  }

  // FP64 defect correction: w->r holds R_64(t) on entry.  Solves
  // r + J delta = 0 to a relative accuracy of 1e-3 with forward-difference
  // Jacobian products of FP32 residuals (perturbation eta = 1e-3 in max norm,
  // far above the FP32 resolution of t), then t <- t + delta.  The
  // finite-difference model itself is good to about 2e-3 on the PPP
  // workloads, so a tighter inner solve gains nothing per outer step.
  int defect_correction(int* inner_out, int* it_io) {
    const double eta = 1e-3, tol = 1e-3;
    double* tb = w->tb;
    double* r64 = w->r64;
    double* rb = w->rb;
    double* del = w->del;
    double* rho = w->rho;
    CK(cudaMemcpyAsync(tb, w->t, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(r64, w->r, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
    double r0 = sqrt(last_norm2), rn, ed;
    // FP32 residual at the base point
    int rc = eval(1, &rn, &ed);
    if (rc) return rc;
    CK(cudaMemcpyAsync(rb, w->r, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(del, 0, sizeof(double) * L, s));
    CK(cudaMemcpyAsync(rho, r64, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
    Diis d(w->diis_cap);
    int inner = 0;
    std::vector<double> hist;
    for (; inner < 30 && *it_io < o.max_iter; ++inner) {
      if ((rc = diis_step(d, del, rho, inner + 1))) return rc;
      // rho = r64 + J del by a forward difference at tb
      CK(cudaMemsetAsync(w->amax, 0, sizeof(unsigned long long), s));
      k_absmax<<<kRedBlocks, 256, 0, s>>>(L, del, w->amax);
      k_fd_point<<<lb, 256, 0, s>>>(L, tb, del, w->amax, eta, w->t);
      if ((rc = eval(1, &rn, &ed))) return rc;
      k_fd_rho<<<lb, 256, 0, s>>>(L, r64, w->r, rb, w->amax, eta, rho);
      w->n_launches += 3;
      g_prof.done("solver: defect-correction vectors", s, 8.0 * L * 6);
      (*it_io)++;
      // weighted norm of rho
      dim3 g(kRedBlocks, 1);
      k_multidot<<<g, 256, 0, s>>>(L, N, rho, 0, w->slot_e, L, w->order, 0, w->part);
      k_rowsum<<<2, 256, 0, s>>>(kRedBlocks, 1, w->part, N, w->esite, w->epair, w->scal);
      CK(cudaMemcpyAsync(w->host, w->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      w->n_launches += 2;
      double rr = sqrt(w->host[0]);
      if (trace_on()) fprintf(stderr, "ppq   inner %2d |r + J d| %.3e (target %.3e)\n", inner, rr, tol * r0);
      if (!isfinite(rr)) break;
      if (rr <= tol * r0) { inner++; break; }
      // stop at the finite-difference noise floor (< 10 % gain over 3 steps)
      hist.push_back(rr);
      size_t k = hist.size();
      if (k >= 4 && hist[k - 1] > 0.9 * hist[k - 4]) { inner++; break; }
    }
    k_axpy_to<<<lb, 256, 0, s>>>(L, tb, del, w->t);
    w->n_launches += 1;
    CK(cudaGetLastError());
    *inner_out = inner;
    return 0;
  }
};

extern "C" {

int ppq_default_opts(ppq_opts* o) {
  if (!o) return fail(-2, "null opts");
  o->K = 2; o->K_H = 0; o->precision = 0;
  o->switch_tol = 0.0; o->r_tol = 1e-10; o->e_tol = 1e-10;   // switch_tol 0: the solver's own default
  o->max_iter = 200; o->diis_dim = 8; o->diis_start = 3;
  o->level_shift = 0.0; o->guess = 0; o->profile = 0; o->polish = 1; o->max_rank = 0;
  return 0;
}

int ppq_amp_count(int K, int n_pairs, size_t* n_amp) {
  if ((K != 2 && K != 3) || n_pairs < 1 || !n_amp)
    return fail(-1, "ppq_amp_count: K must be 2 or 3 and n_pairs >= 1");
  size_t N = (size_t)n_pairs;
  *n_amp = amp_len(n_pairs) + (K == 3 ? (size_t)PPQ_NA3 * N * N * N : 0);
  return 0;
}

int ppq_amp_layout(int K, int* desc) {
  if ((K != 2 && K != 3) || !desc) return fail(-1, "ppq_amp_layout: K must be 2 or 3");
  if (K == 2)
    for (int i = 0; i < 3 * (PPQ_NA1 + PPQ_NA2); ++i) desc[i] = ppq_layout_desc[i];
  else
    for (int i = 0; i < 4 * (PPQ_NA1 + PPQ_NA2 + PPQ_NA3); ++i) desc[i] = ppq_layout_desc3[i];
  return 0;
}

int ppq_release(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  int dev;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  auto it = g_ws.find(dev);
  if (it != g_ws.end() && it->second) {
    free_ws(it->second);
    delete it->second;
    g_ws.erase(it);
  }
  return 0;
}

const char* ppq_last_error(void) { return g_err.c_str(); }

int ppq_profile_count(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_prof.flush();
  return (int)g_prof.cls.size();
}

int ppq_profile_entry(int i, char* name, int name_cap, double* ms, int* launches, double* bytes, double* flops) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_prof.flush();
  if (i < 0 || i >= (int)g_prof.cls.size()) return fail(-2, "ppq_profile_entry: index %d out of range", i);
  const KProf::Cls& c = g_prof.cls[i];
  if (name && name_cap > 0) {
    strncpy(name, c.name.c_str(), name_cap - 1);
    name[name_cap - 1] = 0;
  }
  if (ms) *ms = c.ms;
  if (launches) *launches = c.n;
  if (bytes) *bytes = c.bytes;
  if (flops) *flops = c.flops;
  return 0;
}

int ppq_tc_plan(int n_pairs, int16_t* chunks, int max_chunks, int* ctas, int max_ctas, int* n_chunks,
                int* n_ctas) {
  TcPlan pl;
  int rc = plan_tc(n_pairs, &pl);
  if (rc) return rc;
  int nc = pl.nchunks, nt = (int)pl.cta.size() / 3;
  if (n_chunks) *n_chunks = nc;
  if (n_ctas) *n_ctas = nt;
  if (chunks) {
    if (max_chunks < nc) return fail(-2, "ppq_tc_plan: %d chunks do not fit %d", nc, max_chunks);
    std::copy(pl.chunk.begin(), pl.chunk.end(), chunks);
  }
  if (ctas) {
    if (max_ctas < nt) return fail(-2, "ppq_tc_plan: %d CTAs do not fit %d", nt, max_ctas);
    std::copy(pl.cta.begin(), pl.cta.end(), ctas);
  }
  return 0;
}

int pq_residual(int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h,
                const double* eri, const double* t, double* r, double* e_corr, int precision,
                void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  if (!t || !r) return fail(-2, "t and r must be non-null");
  if (precision != 0 && precision != 1) return fail(-4, "precision must be 0 or 1");
  Workspace* w = nullptr;
  Problem P;
  int rc = prepare(n_pairs, occ_of_pair, vir_of_pair, h, eri, 0, s, &w, &P);
  if (rc) return rc;
  int N = n_pairs;
  size_t L = amp_len(N);
  if ((rc = copy_amps(w->t, t, L, s))) return rc;
  if ((rc = run_residual(w, N, precision, s))) return rc;
  k_rowsum<<<1, 256, 0, s>>>(1, 0, w->part, N, w->esite, w->epair, w->scal);
  if ((rc = copy_amps(r, w->r, L, s))) return rc;
  CK(cudaMemcpyAsync(w->host, w->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(w->host + 60, w->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if ((rc = check_tc_flag(w, *(int*)(w->host + 60), s))) return rc;
  if (e_corr) *e_corr = w->host[0];
  return 0;
}

}  // extern "C"

namespace {

int validate_opts(const ppq_opts& o, bool allow_full = false) {
  if (o.K != 2) return fail(-4, "pq_solve: K must be 2 (PQ)");
  if (o.guess < 0 || o.guess > 2 || (o.guess == 2 && !allow_full))
    return fail(-4, "guess must be 0 (zero), 1 (t_in) or 2 (single-pair start, pq_solve only)");
  if (o.K_H == -1 && !allow_full)
    return fail(-4, "K_H = -1 (untruncated integrals) is solved by pq_solve only");
  if (o.K_H != 0 && o.K_H != 2 && o.K_H != -1)
    return fail(-4, "pq_solve: K_H must be 0 or 2 (two-label integrals) or -1 (untruncated)");
  if (o.precision != 0 && o.precision != 1) return fail(-4, "precision must be 0 or 1");
  if (o.polish != 0 && o.polish != 1) return fail(-4, "polish must be 0 or 1");
  if (o.max_iter < 1 || o.diis_dim < 0 || o.diis_dim > kDiisMax)
    return fail(-4, "max_iter >= 1 and 0 <= diis_dim <= %d required", kDiisMax);
  if (o.max_rank < 0 || o.max_rank > 6) return fail(-4, "max_rank must be 0 (every rank) or 1..6");
  if (!(o.switch_tol >= 0.0)) return fail(-4, "switch_tol must be >= 0 (0: the solver's default)");
  if (o.max_rank != 0 && o.K_H != -1)
    return fail(-4, "max_rank needs the label-subset solver (ph_solve, or pq_solve with K_H = -1)");
  return 0;
}

int diis_slots(const ppq_opts& o) {
  int m_max = o.diis_dim > 0 ? o.diis_dim : 1;
  return (o.precision == 1 && o.polish == 1) ? kDiisMax : m_max;
}

int subset_solve(int K, int KH, int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h,
                 const double* eri, const double* B, int naux, double e_const, const ppq_opts& o,
                 const double* t_in, double* t_out, double* e_corr, double* e_total, ppq_info* info,
                 cudaStream_t s, std::chrono::steady_clock::time_point wall0);

// The solve of one system on a prepared workspace and stream.
int solve_core(Workspace* w, const Problem& P, double e_const, const ppq_opts& o,
               const double* t_in, double* t_out, double* e_corr, double* e_total, ppq_info* info,
               cudaStream_t s, std::chrono::steady_clock::time_point wall0) {
  int rc = 0;
  int m_max = o.diis_dim > 0 ? o.diis_dim : 1;
  int n_pairs = P.N;
  int N = n_pairs, n = 2 * N;
  size_t L = amp_len(N);
  w->profile = o.profile != 0;
  g_prof.reset(w->profile);
  struct ProfOff { ~ProfOff() { g_prof.on = false; } } prof_off;
  g_prof.start(s);
  w->t_quartic_ms = 0.0;
  w->n_quartic = 0;
  w->t_quartic32_ms = 0.0;
  w->n_quartic32 = 0;
  w->n_launches = 0;
  if (o.guess == 1) {
    if ((rc = copy_amps(w->t, t_in, L, s))) return rc;
    size_t L2 = (size_t)N * N * PPQ_NA2;
    ppq::k_symmetrize<<<(unsigned)((L2 + 255) / 256), 256, 0, s>>>(N, w->t + 3 * N);
  } else {
    CK(cudaMemsetAsync(w->t, 0, sizeof(double) * L, s));
  }
  k_eref<<<1, 1, 0, s>>>(N, n, P.h, w->f, w->occ, w->scal + kDiisMax + 2);
  CK(cudaMemcpyAsync(w->host + 40, w->scal + kDiisMax + 2, sizeof(double), cudaMemcpyDeviceToHost, s));

  Solver S(w, N, L, o, s);
  int prec = o.precision;
  int switched_at = prec ? -1 : 0;
  double e_old = 0.0, res = 0.0, e = 0.0;
  bool have_old = false;
  int status = 1, it = 0;
  Diis D(m_max);
  std::vector<double> hist;
  bool defect = false;  // FP64 defect-correction polish active
  for (it = 1; it <= o.max_iter; ++it) {
    if (defect) {
      // one outer step: FP64 residual and test, then J delta = -r by FP32
      // finite-difference Jacobian products (DIIS-accelerated Jacobi)
      if ((rc = S.eval(0, &res, &e))) return rc;
      S.polish_evals++;
      hist.push_back(res);
      if (!isfinite(res) || !isfinite(e) || res > 1e6) { status = 2; break; }
      if (have_old && res <= o.r_tol && fabs(e - e_old) <= o.e_tol) { status = 0; break; }
      if (S.last_outer > 0.0 && res > 0.1 * S.last_outer) {
        // the correction stopped paying: continue with plain FP64 iterations
        defect = false;
        D.reset();
        e_old = e;
        have_old = true;
        if ((rc = S.step_plain(D, it)) != 0) return rc;
        continue;
      }
      S.last_outer = res;
      e_old = e;
      have_old = true;
      if (res <= o.r_tol) {
        // only the energy test is left: converged if one more Jacobi step
        // would change E by at most e_tol (energy from the closures alone)
        double e_next = 0.0;
        if ((rc = S.jacobi_energy(&e_next)) != 0) return rc;
        if (fabs(e_next - e) <= o.e_tol) { status = 0; break; }
        D.reset();
        if ((rc = S.step_plain(D, 1)) != 0) return rc;
        continue;
      }
      int inner = 0;
      if ((rc = S.defect_correction(&inner, &it))) return rc;
      continue;
    }
    if ((rc = S.eval(prec, &res, &e))) return rc;
    if (prec == 0 && switched_at > 0) S.polish_evals++;
    hist.push_back(res);
    if (!isfinite(res) || !isfinite(e) || res > 1e6) { status = 2; break; }
    if (prec == 0 && have_old && res <= o.r_tol && fabs(e - e_old) <= o.e_tol) { status = 0; break; }
    if (prec == 1) {
      size_t k = hist.size();
      bool stagnant = k >= 4 && res < 1e-3 && hist[k - 1] > 0.9 * hist[k - 4];
      // default switch at 1e-4: the defect-correction polish takes the same three
      // FP64 steps from there as from 1e-5 on the C140H142 workload, with fewer
      // FP32 iterations before it (41 instead of 46 evaluations in all)
      if (res <= (o.switch_tol > 0.0 ? o.switch_tol : 1e-4) || stagnant) {
        prec = 0;
        switched_at = it;
        have_old = false;
        D.reset();
        if (o.polish == 1) defect = true;
        continue;  // re-evaluate at the same t in FP64
      }
    }
    e_old = e;
    have_old = true;
    if ((rc = S.step_plain(D, it)) != 0) return rc;
  }
  if (it > o.max_iter) it = o.max_iter;
  if (t_out) { if ((rc = copy_amps(t_out, w->t, L, s))) return rc; }
  CK(cudaStreamSynchronize(s));
  double e_ref = w->host[40];
  if (e_corr) *e_corr = e;
  if (e_total) *e_total = e + e_ref + e_const;
  if (info) {
    info->status = status;
    info->iters = S.evals;
    info->polish_iters = o.precision ? S.polish_evals : 0;
    info->switched_at = o.precision ? switched_at : -1;
    info->res_norm = res;
    info->e_corr = e;
    info->e_total = e + e_ref + e_const;
    info->t_residual_ms = S.t_res_ms;
    info->t_total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    info->residual_flops = residual_flops(N);
    info->quartic_flops = quartic_flops(N);
    info->t_quartic_ms = w->t_quartic_ms;
    info->n_quartic = w->n_quartic;
    info->n_launches = w->n_launches + 7;  // + staging kernels
    info->evals_fp32 = S.evals32;
    info->t_quartic32_ms = w->t_quartic32_ms;
    info->n_quartic32 = w->n_quartic32;
    info->evals_fp64 = S.evals - S.evals32;
  }
  return status;
}

}  // namespace

extern "C" {

int pq_solve(int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h,
             const double* eri, double e_const, const ppq_opts* opts, const double* t_in,
             double* t_out, double* e_corr, double* e_total, ppq_info* info, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  auto wall0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  ppq_opts o;
  if (opts) o = *opts; else ppq_default_opts(&o);
  int rc = validate_opts(o, true);
  if (rc) return rc;
  std::vector<double> pp;
  if (o.guess == 2) {
    // perfect-pairing-type start: solve the single-pair truncation (K = 1,
    // amplitudes inside one pairing label, two-label integrals) first and
    // start from its amplitudes (the two-pair block zero)
    ppq_opts o1 = o;
    o1.guess = 0;
    o1.profile = 0;
    o1.max_rank = o.max_rank == 1 ? 1 : 0;  // single-pair amplitudes have ranks 1 and 2
    size_t L = amp_len(n_pairs);
    pp.assign(L, 0.0);
    int rc1 = subset_solve(1, 2, n_pairs, occ_of_pair, vir_of_pair, h, eri, nullptr, 0, 0.0, o1, nullptr, pp.data(),
                           nullptr, nullptr, nullptr, s, wall0);
    if (rc1 < 0) return rc1;
    if (rc1 == 2 || rc1 == 3) pp.assign(L, 0.0);  // no usable start: zero amplitudes
    o.guess = 1;
    t_in = pp.data();
  }
  // untruncated integrals: terms reach K + 4 = 6 labels, evaluated by the
  // label-subset expansion
  if (o.K_H == -1)
    return subset_solve(2, 4, n_pairs, occ_of_pair, vir_of_pair, h, eri, nullptr, 0, e_const, o, t_in, t_out, e_corr,
                        e_total, info, s, wall0);
  if (o.guess == 1 && !t_in) return fail(-2, "guess = 1 needs t_in");
  Workspace* w = nullptr;
  Problem P;
  rc = prepare(n_pairs, occ_of_pair, vir_of_pair, h, eri, diis_slots(o), s, &w, &P);
  if (rc) {
    if (rc == 3 && info) { memset(info, 0, sizeof *info); info->status = 3; }
    return rc;
  }
  return solve_core(w, P, e_const, o, t_in, t_out, e_corr, e_total, info, s, wall0);
}

int pq_solve_cd(int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h, const double* B,
                int naux, double e_const, const ppq_opts* opts, const double* t_in, double* t_out, double* e_corr,
                double* e_total, ppq_info* info, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  auto wall0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  ppq_opts o;
  if (opts) o = *opts; else ppq_default_opts(&o);
  int rc = validate_opts(o, true);
  if (rc) return rc;
  if (o.guess == 1 && !t_in) return fail(-2, "guess = 1 needs t_in");
  if (!B) return fail(-2, "B must be non-null");
  if (o.K_H == -1)
    return subset_solve(2, 4, n_pairs, occ_of_pair, vir_of_pair, h, nullptr, B, naux, e_const, o, t_in, t_out, e_corr,
                        e_total, info, s, wall0);
  Workspace* w = nullptr;
  Problem P;
  rc = prepare_cd(n_pairs, occ_of_pair, vir_of_pair, h, B, naux, diis_slots(o), s, &w, &P);
  if (rc) {
    if (rc == 3 && info) { memset(info, 0, sizeof *info); info->status = 3; }
    return rc;
  }
  return solve_core(w, P, e_const, o, t_in, t_out, e_corr, e_total, info, s, wall0);
}

// Eigenvalues (and optionally eigenvectors, columns) of a symmetric n x n
// matrix by cyclic Jacobi rotations in one block's shared memory; the values
// sorted in descending order.  n <= kNatMax.
constexpr int kNatMax = 160;
__global__ void k_sym_eig(int n, const double* __restrict__ a_in, double* __restrict__ w_out,
                          double* __restrict__ v_out, int* __restrict__ sweeps_out) {
  extern __shared__ double sm[];
  double* A = sm;              // n x n
  double* V = sm + n * n;      // n x n (eigenvectors, only when v_out)
  __shared__ double cs[2];
  __shared__ double off;
  const bool vec = v_out != nullptr;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    A[i] = 0.5 * (a_in[i] + a_in[(i % n) * n + i / n]);
    if (vec) V[i] = (i / n == i % n) ? 1.0 : 0.0;
  }
  __syncthreads();
  int sweep = 0;
  for (; sweep < 64; ++sweep) {
    if (threadIdx.x == 0) off = 0.0;
    __syncthreads();
    double part = 0.0;
    for (int i = threadIdx.x; i < n * n; i += blockDim.x)
      if (i / n != i % n) part += A[i] * A[i];
    atomicAdd(&off, part);
    __syncthreads();
    double scale = 0.0;
    for (int i = 0; i < n; ++i) scale += A[i * n + i] * A[i * n + i];
    if (off <= 1e-30 * (scale + 1e-300)) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (threadIdx.x == 0) {
          double apq = A[p * n + q];
          double c = 1.0, sn = 0.0;
          if (fabs(apq) > 1e-300) {
            double th = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
            double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            sn = t * c;
          }
          cs[0] = c; cs[1] = sn;
        }
        __syncthreads();
        double c = cs[0], sn = cs[1];
        if (sn != 0.0) {
          // columns p, q
          for (int k = threadIdx.x; k < n; k += blockDim.x) {
            double akp = A[k * n + p], akq = A[k * n + q];
            A[k * n + p] = c * akp - sn * akq;
            A[k * n + q] = sn * akp + c * akq;
            if (vec) {
              double vkp = V[k * n + p], vkq = V[k * n + q];
              V[k * n + p] = c * vkp - sn * vkq;
              V[k * n + q] = sn * vkp + c * vkq;
            }
          }
          __syncthreads();
          // rows p, q
          for (int k = threadIdx.x; k < n; k += blockDim.x) {
            double apk = A[p * n + k], aqk = A[q * n + k];
            A[p * n + k] = c * apk - sn * aqk;
            A[q * n + k] = sn * apk + c * aqk;
          }
        }
        __syncthreads();
      }
  }
  if (threadIdx.x == 0) {
    // selection sort of the diagonal, descending (vectors follow)
    for (int i = 0; i < n; ++i) w_out[i] = A[i * n + i];
    int order[kNatMax];
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j)
        if (w_out[order[j]] > w_out[order[i]]) { int x = order[i]; order[i] = order[j]; order[j] = x; }
    double tmp[kNatMax];
    for (int i = 0; i < n; ++i) tmp[i] = w_out[order[i]];
    for (int i = 0; i < n; ++i) w_out[i] = tmp[i];
    if (vec)
      for (int k = 0; k < n; ++k)
        for (int i = 0; i < n; ++i) v_out[k * n + i] = V[k * n + order[i]];
    if (sweeps_out) *sweeps_out = sweep;
  }
}

int ppq_natural_occupations(int n_orb, const double* gamma, double* occ_out, double* vecs_out, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  if (n_orb < 1 || n_orb > kNatMax) return fail(-1, "ppq_natural_occupations: n_orb must be 1..%d", kNatMax);
  if (!gamma || !occ_out) return fail(-2, "gamma and occ_out must be non-null");
  if (vecs_out && n_orb > 120) return fail(-1, "ppq_natural_occupations: eigenvectors need n_orb <= 120");
  size_t nn = (size_t)n_orb * n_orb;
  double *dg = nullptr, *dw = nullptr, *dv = nullptr;
  CK(cudaMalloc((void**)&dg, sizeof(double) * nn));
  CK(cudaMalloc((void**)&dw, sizeof(double) * n_orb));
  if (vecs_out) CK(cudaMalloc((void**)&dv, sizeof(double) * nn));
  CK(cudaMemcpyAsync(dg, gamma, sizeof(double) * nn, cudaMemcpyDefault, s));
  size_t smem = sizeof(double) * nn * (vecs_out ? 2 : 1);
  if (smem > 227 * 1024) {
    cudaFree(dg); cudaFree(dw); if (dv) cudaFree(dv);
    return fail(-1, "ppq_natural_occupations: eigenvectors need n_orb <= 120");
  }
  if (smem > 48 * 1024) CK(cudaFuncSetAttribute(k_sym_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_sym_eig<<<1, 256, smem, s>>>(n_orb, dg, dw, dv, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(occ_out, dw, sizeof(double) * n_orb, cudaMemcpyDefault, s);
  if (e == cudaSuccess && vecs_out) e = cudaMemcpyAsync(vecs_out, dv, sizeof(double) * nn, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dg); cudaFree(dw); if (dv) cudaFree(dv);
  if (e != cudaSuccess) return fail(-100, "CUDA error %s in ppq_natural_occupations", cudaGetErrorString(e));
  return 0;
}

// Self-test of the bounded mbarrier wait used by the tensor-core kernels: one
// CTA initialises a barrier that expects one arrival, nobody arrives, and the
// wait gives up after `cycles` clock cycles and reports it.  No copy, MMA or
// tensor memory is involved, so the timeout leaves nothing in flight.
__global__ void k_wait_selftest(long long cycles, int* __restrict__ out) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    ppq::tc::mbar_init(&bar, 1);
    abort_flag = 0;
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  bool done = false;
  if (threadIdx.x == 0) {
    long long t0 = clock64();
    while (!(done = ppq::tc::mbar_try(&bar, 0)))
      if (clock64() - t0 > cycles) { abort_flag = 1; break; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = abort_flag;    // 1: the wait ran out
    out[1] = done ? 1 : 0;  // 1: the phase completed (it must not)
  }
}

int ppq_wait_selftest(long long cycles, int* timed_out, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  if (cycles < 1 || cycles > 4000000000LL) return fail(-2, "cycles must be in 1 .. 4e9");
  int dev;
  CK(cudaGetDevice(&dev));
  Workspace*& w = g_ws[dev];
  if (!w) w = new Workspace();
  int rc = grow(w, 2, 1);
  if (rc) return rc;
  k_wait_selftest<<<1, 32, 0, s>>>(cycles, w->ok);
  CK(cudaGetLastError());
  int host[2] = {0, 0};
  CK(cudaMemcpyAsync(host, w->ok, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (host[1]) return fail(-100, "wait self-test: a barrier phase completed without an arrival");
  if (timed_out) *timed_out = host[0];
  return 0;
}

int pq_solve_batched(int n_sys, const int* n_pairs, const int* const* occ_of_pair,
                     const int* const* vir_of_pair, const double* const* h,
                     const double* const* eri, const double* e_const, const ppq_opts* opts,
                     double* const* t_out, double* e_corr, double* e_total, ppq_info* info,
                     void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  if (n_sys < 1 || !n_pairs || !occ_of_pair || !vir_of_pair || !h || !eri)
    return fail(-2, "pq_solve_batched: n_sys >= 1 and non-null per-system arrays required");
  ppq_opts o;
  if (opts) o = *opts; else ppq_default_opts(&o);
  int rc = validate_opts(o);
  if (rc) return rc;
  if (o.guess == 1) return fail(-4, "pq_solve_batched starts from zero amplitudes (guess = 0)");
  int dev;
  CK(cudaGetDevice(&dev));
  const char* env = getenv("PPQ_BATCH_THREADS");
  int nthreads = env ? atoi(env) : 8;
  nthreads = std::max(1, std::min(nthreads, n_sys));
  auto& pool = g_batch_ws[dev];
  while ((int)pool.size() < nthreads) pool.push_back(new Workspace());
  // the batch starts after earlier work on the caller's stream and ends before return
  cudaStream_t caller = (cudaStream_t)stream;
  cudaEvent_t start_ev;
  CK(cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming));
  CK(cudaEventRecord(start_ev, caller));
  std::atomic<int> next(0);
  std::vector<int> codes(n_sys, 0);
  std::vector<std::string> msgs(nthreads);
  std::vector<int> worst(nthreads, 0);
  auto worker = [&](int tid) {
    cudaSetDevice(dev);
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      worst[tid] = -100;
      msgs[tid] = "cudaStreamCreate failed";
      return;
    }
    cudaStreamWaitEvent(s, start_ev, 0);
    Workspace* w = pool[tid];
    for (int i = next++; i < n_sys; i = next++) {
      auto wall0 = std::chrono::steady_clock::now();
      Problem P;
      ppq_info tmp;
      memset(&tmp, 0, sizeof tmp);
      int r = prepare_ws(w, n_pairs[i], occ_of_pair[i], vir_of_pair[i], h[i], eri[i],
                         diis_slots(o), s, &P);
      if (r == 0) {
        double ec = 0.0, et = 0.0;
        r = solve_core(w, P, e_const ? e_const[i] : 0.0, o, nullptr, t_out ? t_out[i] : nullptr,
                       &ec, &et, &tmp, s, wall0);
        if (e_corr) e_corr[i] = ec;
        if (e_total) e_total[i] = et;
      } else {
        tmp.status = r;
      }
      if (info) info[i] = tmp;
      codes[i] = r;
      if (r < 0 && worst[tid] == 0) { worst[tid] = r; msgs[tid] = g_err; }
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) th.emplace_back(worker, t);
  for (auto& t : th) t.join();
  cudaEventDestroy(start_ev);
  for (int t = 0; t < nthreads; ++t)
    if (worst[t] < 0) return fail(worst[t], "%s", msgs[t].c_str());
  int status = 0;
  for (int i = 0; i < n_sys; ++i) status = std::max(status, codes[i]);
  return status;  // 0 when every system converged, else the largest status
}

int pq_lagrangian_gradient(int n_pairs, const int* occ_of_pair, const int* vir_of_pair,
                           const double* h, const double* eri, const double* t, const double* lam,
                           double* grad, double* e_corr, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  if (!t || !lam || !grad) return fail(-2, "t, lam and grad must be non-null");
  Workspace* w = nullptr;
  Problem P;
  int rc = prepare(n_pairs, occ_of_pair, vir_of_pair, h, eri, 0, s, &w, &P);
  if (rc) return rc;
  int N = n_pairs;
  size_t L = amp_len(N);
  if ((rc = grow_adjoint(w, N))) return rc;
  if ((rc = copy_amps(w->t, t, L, s))) return rc;
  if ((rc = copy_amps(w->lam, lam, L, s))) return rc;
  if ((rc = lagrangian_gradient(w, N, w->lam, s))) return rc;
  k_rowsum<<<1, 256, 0, s>>>(1, 0, w->part, N, w->esite, w->epair, w->scal);
  if ((rc = copy_amps(grad, w->gu, L, s))) return rc;
  CK(cudaMemcpyAsync(w->host, w->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (e_corr) *e_corr = w->host[0];
  return 0;
}

int pq_lambda(int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h,
              const double* eri, const double* t, const ppq_opts* opts, double* lam_out,
              ppq_info* info, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  auto wall0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  if (!t || !lam_out) return fail(-2, "t and lam_out must be non-null");
  ppq_opts o;
  if (opts) o = *opts; else ppq_default_opts(&o);
  int rc = validate_opts(o);
  if (rc) return rc;
  Workspace* w = nullptr;
  Problem P;
  rc = prepare(n_pairs, occ_of_pair, vir_of_pair, h, eri, diis_slots(o), s, &w, &P);
  if (rc) return rc;
  int N = n_pairs;
  size_t L = amp_len(N);
  if ((rc = grow_adjoint(w, N))) return rc;
  if ((rc = copy_amps(w->t, t, L, s))) return rc;
  size_t L2 = (size_t)N * N * PPQ_NA2;
  ppq::k_symmetrize<<<(unsigned)((L2 + 255) / 256), 256, 0, s>>>(N, w->t + 3 * N);
  o.precision = 0;
  Solver S(w, N, L, o, s);
  double res = 0.0;
  int iters = 0;
  int status = S.solve_lambda(o.r_tol, o.max_iter, &res, &iters);
  if (status < 0) return status;
  if ((rc = copy_amps(lam_out, w->lam, L, s))) return rc;
  CK(cudaStreamSynchronize(s));
  if (info) {
    memset(info, 0, sizeof *info);
    info->status = status;
    info->iters = iters;
    info->res_norm = res;
    info->t_total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
  }
  return status;
}

int pq_gradient(int n_pairs, const int* occ_of_pair, const int* vir_of_pair, const double* h,
                const double* eri, double e_const, const ppq_opts* opts, double* t_out,
                double* lam_out, double* dE_dh, double* dE_deri, double* dE_dkappa,
                double* e_total, ppq_info* info, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  auto wall0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  ppq_opts o;
  if (opts) o = *opts; else ppq_default_opts(&o);
  int rc = validate_opts(o);
  if (rc) return rc;
  if (o.guess == 1) return fail(-4, "pq_gradient starts from zero amplitudes (guess = 0)");
  Workspace* w = nullptr;
  Problem P;
  rc = prepare(n_pairs, occ_of_pair, vir_of_pair, h, eri, diis_slots(o), s, &w, &P);
  if (rc) return rc;
  int N = n_pairs, n = 2 * N;
  size_t L = amp_len(N), n2 = (size_t)n * n;
  double ec = 0.0, et = 0.0;
  ppq_info si;
  int status = solve_core(w, P, e_const, o, nullptr, nullptr, &ec, &et, &si, s, wall0);
  if (status < 0) return status;
  if ((rc = grow_adjoint(w, N))) return rc;
  ppq_opts ol = o;
  ol.precision = 0;
  Solver S(w, N, L, ol, s);
  double lres = 0.0;
  int liters = 0;
  int lstat = S.solve_lambda(o.r_tol, o.max_iter, &lres, &liters);
  if (lstat < 0) return lstat;
  if ((rc = integral_gradients(w, P, s))) return rc;
  if (t_out) { if ((rc = copy_amps(t_out, w->t, L, s))) return rc; }
  if (lam_out) { if ((rc = copy_amps(lam_out, w->lam, L, s))) return rc; }
  if (dE_dh) CK(cudaMemcpyAsync(dE_dh, w->gh, sizeof(double) * n2, cudaMemcpyDefault, s));
  if (dE_deri) CK(cudaMemcpyAsync(dE_deri, w->gv, sizeof(double) * n2 * n2, cudaMemcpyDefault, s));
  if (dE_dkappa) CK(cudaMemcpyAsync(dE_dkappa, w->dk, sizeof(double) * n2, cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  if (e_total) *e_total = et;
  if (info) {
    *info = si;
    info->status = std::max(status, lstat);
    info->t_total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
  }
  return std::max(status, lstat);
}


}  // extern "C"

// ---------------------------------------------------------------- allocation-free residual
// pq_residual_static: the residual evaluation of pq_residual with every
// intermediate placed in one file-scope device array instead of the cached
// workspace, for callers that must not allocate device memory.
namespace {

// The array is sized for the stated maximum of 12 pairs: the intermediates
// grow as n_pairs^2 and take 4.4 MiB at 12 pairs; 8 MiB keeps headroom.
constexpr int kStaticMaxPairs = 12;
constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB on every device that loads the library
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
std::map<int, unsigned char*> g_static_addr;  // device address of g_static_scratch, per device

// Device address of the scratch array on the current device (looked up once
// per device; the host-side symbol is only a handle, never a device address).
int static_scratch_address(unsigned char** out) {
  int dev;
  CK(cudaGetDevice(&dev));
  auto it = g_static_addr.find(dev);
  if (it == g_static_addr.end()) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(-100, "cudaGetSymbolAddress(g_static_scratch) failed: %s", cudaGetErrorString(e));
    it = g_static_addr.emplace(dev, static_cast<unsigned char*>(p)).first;
  }
  *out = it->second;
  return 0;
}

struct Carver {
  unsigned char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += sizeof(T) * (count > 0 ? count : 1);
    return p;
  }
};

}  // namespace

extern "C" int pq_residual_static(int n_pairs, const int* occ_of_pair, const int* vir_of_pair,
                                  const double* h, const double* eri, const double* t, double* r,
                                  double* e_corr, int precision, void* stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  if (n_pairs > kStaticMaxPairs)
    return fail(-6, "pq_residual_static: n_pairs = %d exceeds the static scratch limit of %d pairs",
                n_pairs, kStaticMaxPairs);
  std::vector<int> lab;
  int rc = check_pairing(n_pairs, occ_of_pair, vir_of_pair, lab);
  if (rc) return rc;
  if (precision != 0 && precision != 1) return fail(-4, "precision must be 0 or 1");
  if (!h || !eri || !t || !r) return fail(-2, "h, eri, t and r must be non-null");
  if (!is_device_ptr(h) || !is_device_ptr(eri) || !is_device_ptr(t) || !is_device_ptr(r))
    return fail(-7, "pq_residual_static needs device pointers for h, eri, t and r");
  unsigned char* base = nullptr;
  if ((rc = static_scratch_address(&base))) return rc;
  int N = n_pairs, n = 2 * N;
  size_t NN = (size_t)N * N;
  Carver cv{base};
  Workspace w;  // pointers into the static array; nothing is allocated
  w.occ = cv.take<int>(N); w.vir = cv.take<int>(N); w.lab = cv.take<int>(n);
  w.f = cv.take<double>((size_t)n * n); w.hp = cv.take<double>((size_t)n * n);
  w.fo = cv.take<double>(N); w.fv = cv.take<double>(N);
  w.g1d = cv.take<double>((size_t)N * PPQ_NG1); w.g2d = cv.take<double>(NN * PPQ_NG2);
  w.g1f = cv.take<float>((size_t)N * PPQ_NG1); w.g2f = cv.take<float>(NN * PPQ_NG2);
  w.dir = cv.take<double>(NN * PPQ_NA2); w.abuf = cv.take<double>(NN * PPQ_NA2);
  w.cl = cv.take<double>(NN * PPQ_NS36); w.hs = cv.take<double>((size_t)N * 256);
  w.pg = cv.take<double>(NN * PPQ_NS36); w.pt7 = cv.take<double>(NN * PPQ_NT7E);
  w.pc0 = cv.take<double>(NN * PPQ_NCOL0);
  w.clT = cv.take<double>((size_t)cl_ld(N) * PPQ_NS36); w.gT = cv.take<double>(NN * PPQ_NS36);
  w.t9 = cv.take<double>(NN * PPQ_NA2);
  w.pt7T = cv.take<double>(NN * PPQ_NT7E); w.m7 = cv.take<double>(NN * PPQ_NK7);
  w.esite = cv.take<double>(N); w.epair = cv.take<double>(NN);
  w.part = cv.take<double>(kRedBlocks); w.scal = cv.take<double>(4);
  std::vector<int> wk;
  for (int c2 = 0; c2 < 30; ++c2)
    for (int a = ppq_q9cptr_h[c2]; a < ppq_q9cptr_h[c2 + 1]; a += 4) {
      wk.push_back(c2); wk.push_back(a); wk.push_back(std::min(a + 4, (int)ppq_q9cptr_h[c2 + 1]));
    }
  w.n_work9 = (int)wk.size() / 3;
  w.work9 = cv.take<int>(wk.size());
  w.t9part = cv.take<double>((size_t)w.n_work9 * (NN - N) / 2 * PPQ_NA2);
  w.r1part = cv.take<double>((size_t)kR1Split * 3 * N);
  if (cv.off > kStaticScratchBytes)
    return fail(-6, "pq_residual_static: %zu bytes of scratch needed, %zu available", cv.off,
                kStaticScratchBytes);
  // From the first enqueue on, every failure waits for the work already queued
  // on the stream before returning, so that no kernel of this call still uses
  // the array when the next call clears it.
  auto enqueue = [&]() -> int {
    // the array keeps the previous call's contents: clear the part this call uses
    CK(cudaMemsetAsync(base, 0, cv.off, s));
    CK(cudaMemcpyAsync(w.occ, occ_of_pair, sizeof(int) * N, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(w.vir, vir_of_pair, sizeof(int) * N, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(w.lab, lab.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(w.work9, wk.data(), sizeof(int) * wk.size(), cudaMemcpyHostToDevice, s));
    Problem P{N, n, h, eri};
    int rc2 = stage(&w, P, s);
    if (rc2) return rc2;
    w.t = const_cast<double*>(t);  // read only by the residual kernels
    w.r = r;
    // launched directly on any stream (capturing a graph here would
    // instantiate, i.e. allocate, one per call) with the fixed micro-tile
    // ceil(N / 16) of the SIMT quartic kernel: no autotuning, no events
    int mt = std::max(1, (N + 15) / 16);
    w.mt[0] = w.mt[1] = mt;
    return precision ? residual<float>(&w, N, s) : residual<double>(&w, N, s);
  };
  rc = enqueue();
  if (rc) {
    cudaStreamSynchronize(s);
    return rc;
  }
  k_rowsum<<<1, 256, 0, s>>>(1, 0, w.part, N, w.esite, w.epair, w.scal);
  double e = 0.0;
  CK(cudaMemcpyAsync(&e, w.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (e_corr) *e_corr = e;
  return 0;
}

#include "ph_engine.cuh"
#include "ph_adjoint.cuh"
