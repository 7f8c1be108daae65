// solver.cu -- host driver and C ABI (include/qnsch.h) of the GB300 q-NSCH solver:
// level hierarchy in device memory, one implicit time step of the primitive
// method (Sec. 6.1) solved by FAS V-cycles (Sec. 7.1), reductions for mass and
// energy (Thms. 6.1, 6.2).  Every step of the numerical path runs in the CUDA
// kernels of kernels.cu; this file only allocates, sequences and copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <type_traits>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "qnsch.h"

using qn::ErrForm;
using qn::FullForm;
using qn::ProjForm;
using qn::Lv;
using qn::Prm;

namespace {

// kernels queued into captured graphs (not executed at capture time) and
// kernels executed by graph replays, for qnsch_kernel_launches
std::atomic<long long> g_captured{0};
std::atomic<long long> g_replayed{0};

void* (*g_alloc)(size_t, void*) = nullptr;
void (*g_free)(void*, void*) = nullptr;
void* g_ctx = nullptr;
std::mutex g_alloc_mu;  // guards the three above

// the allocator a handle uses for its whole life: the one in effect when it
// was created (qnsch_set_allocator later changes only new handles)
struct Allocator {
  void* (*alloc)(size_t, void*) = nullptr;  // NULL: cudaMalloc / cudaFree
  void (*free)(void*, void*) = nullptr;
  void* ctx = nullptr;
};

void* dev_alloc(const Allocator& A, size_t bytes) {
  if (A.alloc) return A.alloc(bytes, A.ctx);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void dev_free(const Allocator& A, void* p) {
  if (!p) return;
  if (A.free) A.free(p, A.ctx);
  else cudaFree(p);
}

// process-wide device-memory budget (qnsch_set_budget; 0 = none) and the bytes
// reserved against it by live handles
std::atomic<size_t> g_budget{0};
std::atomic<size_t> g_reserved{0};

bool over_budget(size_t more) {
  size_t b = g_budget.load();
  return b != 0 && g_reserved.load() + more > b;
}

// reserve `bytes` against the budget, or fail without reserving anything
bool reserve_bytes(size_t bytes) {
  size_t cur = g_reserved.load();
  for (;;) {
    size_t b = g_budget.load();
    if (b != 0 && cur + bytes > b) return false;
    if (g_reserved.compare_exchange_weak(cur, cur + bytes)) return true;
  }
}

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

constexpr int NFIELD = 59;  // arrays per FP64 level (see Lv)
// doubles in s->scal and its pinned host mirror s->hbuf, and the offset of the
// device-side step loop's control block in them (layout in kernels.cu); its
// entry WAIT_FLAG is set by a bounded wait of the wavefront smoother that ran
// out of time
constexpr int NSCAL = 128;
constexpr int CTL = 64;
constexpr int CTL_LEN = 18;
constexpr int WAIT_FLAG = CTL + 17;
// bands of the wavefront smoother have at least this many rows
constexpr int WAVE_MIN_ROWS = 4;
// bytes of the wavefront's counters: a ticket and one count per band of the
// finest level at the smallest band height, rounded to 256 B
size_t wave_ctr_bytes(int m2) {
  size_t n = 2 + (size_t)(m2 + WAVE_MIN_ROWS - 1) / WAVE_MIN_ROWS;
  return (n * sizeof(unsigned) + 255) / 256 * 256;
}

// option "pdl": programmatic dependent launch of every kernel (process-wide)
static std::atomic<int> g_pdl_option{1};

// surface-tension ratio eta(rho1, rho2) of Sec. 8.1; near rho1 = rho2 the
// formula is 0/0 and the Taylor series of x^2 - 1 - 2x ln x in q = x - 1 is used
double eta_st(double r1, double r2) {
  double q = r2 / r1 - 1.0;
  if (std::fabs(q) < 0.1) {
    double S = 0.0, qn = 1.0;
    for (int n = 0; n < 24; ++n) {
      S += 2.0 * ((n & 1) ? -1.0 : 1.0) * qn / ((n + 2.0) * (n + 3.0));
      qn *= q;
    }
    return 1.0 / (2.0 * std::sqrt(2.0) * r1 * (1.0 + q) * S);
  }
  double d = r2 - r1;
  return d * d * d /
         (2.0 * std::sqrt(2.0) * r1 * r2 * (r2 * r2 - r1 * r1 - 2.0 * r1 * r2 * std::log(r2 / r1)));
}

// Vanka colours of a level: 5 (walls in x), 8 for (2i+j) mod 8 (periodic x,
// m1 = 0 mod 4), else the smallest divisor >= 5 of m1 for (i+2j) mod K
int colours_of(int m1, int px) {
  if (!px) return 5;
  if (m1 % 4 == 0) return 8;
  for (int K = 5; K <= m1; ++K)
    if (m1 % K == 0) return K;
  return m1;
}

// coarsen by 2 while both sizes are even: walls down to 2 cells; periodic x
// keeps the coarse m1 even (red-black across the seam) and >= 4
int max_levels(int m1, int m2, int px) {
  int n = 1;
  while (m1 % 2 == 0 && m2 % 2 == 0 && m2 / 2 >= 2 &&
         (px ? (m1 / 2 >= 4 && (m1 / 2) % 2 == 0) : m1 / 2 >= 2)) {
    m1 /= 2;
    m2 /= 2;
    ++n;
  }
  return n;
}

}  // namespace

struct qnsch_s {
  // physical parameters as given
  double rho1, rho2, mu1, mu2, Re, We, Pe, Cn, Fr_inv;
  double M, eta, eps_m;
  // options
  int nu1 = 2, nu2 = 2, nuc = 4, maxcyc = 50;
  // smoothing steps on the finest level of the V-cycle (-1: nu1, nu2)
  int nu1f = -1, nu2f = -1;
  double tol = 1e-9, omega = 1.0;
  // 0: FP64 FAS on the scheme itself; 1: FP64 defect correction around FP32 FAS
  // cycles on the error equation; 2: the same with FP64 error cycles
  int precision = 0;
  // levels with at most this many cells run as one fused single-block V-cycle
  // (0: never); separate thresholds for FP64 and FP32 levels
  int fuse64 = 128, fuse32 = 512;
  // blocks of the fused V-cycle's launch: 1, or a thread-block cluster of that
  // many blocks (a power of two up to 16 that the device accepts)
  int fuse_ctas = 1;
  // 0: the paper's separate CH and Vanka sweeps; 1: the coupled 7x7 block
  int coupled = 0;
  // 0: the primitive method (Sec. 6.1); 1: the projection method (Sec. 6.2)
  int scheme = 0;
  // FP64 levels with at most this many cells per Vanka colour smooth with four
  // lanes per block in the per-level launches, and with eight (half a
  // momentum row per lane) up to team8_max; team8_max > 0 also turns on the
  // eight-lane blocks of the single-block coarse V-cycle
  int team_max = 8192;
  int team8_max = 0;
  // FP64 full-iterate levels above team_max with at most this many cells per
  // Vanka colour smooth with a lane pair per block (x rows on one lane, y rows
  // on the other) in the per-level launches
  int pair_max = 0;
  // FP64 full-iterate single-lane Vanka launches: 0 as they are; 1 split a
  // colour between one lane per block and lane pairs where a cost model says
  // it is cheaper; >= 2 that many slots (a multiple of 32) one lane each
  int vsplit = 0;
  // the fused V-cycle of FP64 full-iterate levels in one block runs on a
  // shared-memory copy of its levels where it fits (1) or from global memory
  // (0); coarse_smem_used: whether the last fused launch did
  int coarse_smem = 1;
  int coarse_smem_used = 0;
  // the same for the CH smoother's per-level launches (cells per red-black colour)
  int ch_team_max = 4096, ch_team_max32 = 0;
  // the same on the error-equation levels of the defect correction (their
  // visits are latency-bound up to this size; larger levels stream from HBM)
  int team_max32 = 65536;
  // error-equation levels with at least this many cells run nu smoothing steps
  // as one banded wavefront launch (k_wave; 0: never), with bands of
  // wave_rows rows, waits bounded by wave_budget SM cycles; wave_stall is a
  // test hook that makes one wait run out
  long long wave_cells = 0;
  int wave_rows = 8;
  long long wave_budget = 1LL << 31;
  int wave_stall = 0;
  unsigned* wave_ctr = nullptr;  // 1 + bands of level 0 counters
  // error-equation levels with at least this many cells run nu smoothing steps
  // in the skewed-chunk schedule (k_skew; 0: never), chunks of skew_rows rows
  long long skew_cells = 0;
  int skew_rows = 32;
  // initial iterate of a step: 0 the committed state x^n; 1 or 2 its
  // extrapolation in time (Lagrange, at the new time) through x^n and the one
  // or two states committed before it.  hist[k] is the state committed k + 1
  // steps before the current one (c, mu, p, u, v, padded level-0 layout) and
  // hdt[k] the size of the step that left it; nhist of them are valid.
  // nhist = -1: the committed state was set by the caller, not computed by a
  // step (its mu and p are only guesses), so it is no node either
  int predictor = 0;
  int nhist = -1;
  double hdt[2] = {0.0, 0.0};
  double* hist[2][5] = {};
  // failure detection: a step stops once it has run this many seconds of wall
  // time (0: no limit), or once its residual has grown over this many
  // consecutive outer cycles (0: never)
  double time_limit = 0.0;
  int diverge = 0;
  // device bytes reserved against the process-wide budget
  size_t reserved = 0;
  // the allocator of every device block of this handle
  Allocator mem;
  // grid
  int m1, m2, px, nlev, kcol;
  double h;
  std::vector<Lv<double>> L;
  std::vector<Lv<float>> Ef;   // error-equation levels, FP32 (precision 1)
  std::vector<Lv<double>> Ed;  // error-equation levels, FP64 (precision 2)
  std::vector<void*> blocks;
  size_t level_elems0 = 0;
  // committed state, same padded layout as level 0
  double *sc = nullptr, *smu = nullptr, *sp = nullptr, *su = nullptr, *sv = nullptr;
  // scratch: block partials and small results
  double* part = nullptr;
  double* scal = nullptr;  // [0..9] norms, [16] p sum, [20..21] mass, [24] energy, [25] diss,
                           // [32..42] diagnostics
  double* hbuf = nullptr;  // pinned host mirror of scal
  double* stage = nullptr;  // device staging buffer for host-array I/O (one field)
  cudaStream_t stream = nullptr;       // work stream: the user's, else own_stream
  cudaStream_t user_stream = nullptr;  // set by qnsch_set_stream (NULL: legacy default stream)
  cudaStream_t own_stream = nullptr;   // non-blocking stream used when user_stream is NULL
  cudaEvent_t ev_entry = nullptr;      // orders own_stream after the legacy stream at entry
  cudaEvent_t ev_norms = nullptr;      // recorded after the norms' copy to hbuf (batch polling)
  int pending = 0;
  // one outer cycle captured as a CUDA graph and replayed (option "graphs")
  int use_graphs = 1;
  unsigned opt_version = 0;
  cudaGraphExec_t gexec = nullptr;
  double g_dt = -1.0;
  int g_precision = -1, g_prof = -1, g_ev_used = 0;
  unsigned g_opt = ~0u;
  long long g_nodes = 0;  // kernels in the captured graph
  // the whole step as one graph whose outer-cycle loop runs on the device:
  // the initial residual, a conditional WHILE node around the cycle, a
  // conditional IF node around the commit, one copy of the results to the
  // host (option "device_loop", off by default: it measured no faster for one
  // instance and slower for many at once, and kernels inside a graph with
  // conditional nodes cannot be profiled; off, or while profiling, the host
  // reads the norms after every cycle and queues the next one)
  int device_loop = 0;
  cudaGraphExec_t sexec = nullptr;
  double s_dt = -1.0;
  double s_w[3] = {0.0, 0.0, 0.0};  // the predictor's weights the graph was built with
  int s_precision = -1;
  unsigned s_opt = ~0u;
  long long s_pro = 0, s_body = 0, s_commit = 0;  // kernels in the graph's three parts
  // a step queued by qnsch_step_launch and not yet collected by
  // qnsch_step_poll: 1 on the device-side loop (events ev_s0/ev_s1 around it),
  // 2 already run by the host-driven loop (its outcome kept below)
  int async = 0;
  int a_status = 0, a_cycles = 0;
  double a_res = 0.0;
  cudaEvent_t ev_s0 = nullptr, ev_s1 = nullptr;
  // the host-driven step as a state machine (async == 2; qnsch_batch_step):
  // phase 1 waits for the norms of the initial residual, 2 for those of a
  // cycle, 3 for the commit; the stopping rules are qnsch_step's
  int hs_phase = 0, hs_k = 0, hs_grew = 0, hs_late = 0, hs_expired = 0;
  double hs_res = 0.0, hs_prev = 0.0;
  std::chrono::steady_clock::time_point hs_t0;
  // the FP64 residual arrays of level 0 hold r(x) of the current iterate
  int res_valid = 0;
  // optional CUDA-event timing of launches by kind (bit k of prof: kind k,
  // see PK_*); every event pair carries its kind and the cell visits of the
  // timed launch
  int prof = 0;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;
  std::vector<double> ev_visits;
  int ev_used = 0;
  long long prof_launches = 0;
  double prof_ms = 0.0;
  long long pk_n[6] = {0, 0, 0, 0, 0, 0};
  double pk_ms[6] = {0, 0, 0, 0, 0, 0}, pk_visits[6] = {0, 0, 0, 0, 0, 0};
  double dt = 0.0;
  double last_diss = 0.0;
};

namespace {

Prm<double> make_prm(const qnsch_s* s) {
  Prm<double> P;
  double alpha = (s->rho2 - s->rho1) / (s->rho1 * s->rho2);
  P.ia = alpha;
  P.ib = 1.0 / s->rho2;
  P.va = (s->mu2 - s->mu1) / (s->mu1 * s->mu2);
  P.vb = 1.0 / s->mu2;
  P.alpha = alpha;
  P.K = s->M * s->eta / (s->Cn * s->We);
  P.Lam = s->Cn * s->eta * s->M / s->We;
  P.iM = 1.0 / s->M;
  P.iRe = 1.0 / s->Re;
  P.iPe = 1.0 / s->Pe;
  P.Fr_inv = s->Fr_inv;
  P.eps_m = s->eps_m;
  P.idt = s->dt > 0 ? 1.0 / s->dt : 0.0;
  return P;
}

int cuda_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? QNSCH_OK : QNSCH_ECUDA;
}

int sync(const qnsch_s* s) {
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) {
    cudaGetLastError();
    return QNSCH_ECUDA;
  }
  return cuda_status();
}

size_t padded_elems(int m1, int m2, int* pitch) {
  int p = ((m1 + 3) + 31) / 32 * 32;
  *pitch = p;
  return (size_t)p * (size_t)(m2 + 3);
}

void free_all(qnsch_s* s) {
  // work still queued on the handle's own stream (the zero fills of a
  // creation that failed part way) ends before its memory goes back
  if (s->own_stream) cudaStreamSynchronize(s->own_stream);
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  s->gexec = nullptr;
  if (s->sexec) cudaGraphExecDestroy(s->sexec);
  s->sexec = nullptr;
  for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
  s->ev.clear();
  if (s->ev_entry) cudaEventDestroy(s->ev_entry);
  s->ev_entry = nullptr;
  if (s->ev_norms) cudaEventDestroy(s->ev_norms);
  s->ev_norms = nullptr;
  if (s->ev_s0) cudaEventDestroy(s->ev_s0);
  if (s->ev_s1) cudaEventDestroy(s->ev_s1);
  s->ev_s0 = s->ev_s1 = nullptr;
  if (s->own_stream) cudaStreamDestroy(s->own_stream);
  s->own_stream = nullptr;
  for (void* b : s->blocks) dev_free(s->mem, b);
  s->blocks.clear();
  g_reserved -= s->reserved;
  s->reserved = 0;
  if (s->hbuf) cudaFreeHost(s->hbuf);
  s->hbuf = nullptr;
}

int alloc_all(qnsch_s* s) {
  if (cudaStreamCreateWithFlags(&s->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_entry, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_norms, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&s->ev_s0) != cudaSuccess || cudaEventCreate(&s->ev_s1) != cudaSuccess) {
    cudaGetLastError();
    return QNSCH_ECUDA;
  }
  s->stream = s->own_stream;
  qn::coarse_smem_prepare();
  int a = s->m1, b = s->m2;
  double h = s->h;
  s->L.resize(s->nlev);
  for (int l = 0; l < s->nlev; ++l) {
    Lv<double>& L = s->L[l];
    int pitch;
    size_t n = padded_elems(a, b, &pitch);
    if (l == 0) s->level_elems0 = n;
    double* base = (double*)dev_alloc(s->mem, n * NFIELD * sizeof(double));
    if (!base) return QNSCH_ENOMEM;
    s->blocks.push_back(base);
    if (cudaMemsetAsync(base, 0, n * NFIELD * sizeof(double), s->stream) != cudaSuccess)
      return QNSCH_ECUDA;
    L.m1 = a;
    L.m2 = b;
    L.px = s->px;
    L.kcol = colours_of(a, s->px);
    L.c8 = s->px && a % 4 == 0;
    L.pitch = pitch;
    L.h = h;
    L.ih = 1.0 / h;
    L.ih2 = 1.0 / (h * h);
    double** f[NFIELD] = {&L.c,  &L.mu,  &L.p,    &L.u,    &L.v,    &L.fc, &L.fmu, &L.fp,
                          &L.fu, &L.fv,  &L.rc,   &L.rmu,  &L.rp,   &L.ru, &L.rv,  &L.sc,
                          &L.smu, &L.sp, &L.su,   &L.sv,   &L.cn,   &L.un, &L.vn,  &L.rhon,
                          &L.mobn, &L.visn, &L.Gn, &L.Aru, &L.Arv,  &L.Sx, &L.Sy,  &L.Qx,
                          &L.Qy, &L.Av,  &L.Tx,   &L.Ty,   &L.Dvu,  &L.Dvv, &L.T1u, &L.T1v,
                          &L.T0u, &L.T0v, &L.Dgu, &L.Dgv, &L.rhoc,
                          &L.Cu, &L.aPu, &L.aMu, &L.tPu, &L.tMu, &L.M0u, &L.M1u,
                          &L.Cv, &L.aPv, &L.aMv, &L.tPv, &L.tMv, &L.M0v, &L.M1v};
    for (int q = 0; q < NFIELD; ++q) *f[q] = base + (size_t)q * n + pitch + 1;  // origin (0,0)
    a /= 2;
    b /= 2;
    h *= 2.0;
  }
  size_t n0 = s->level_elems0;
  double* st = (double*)dev_alloc(s->mem, n0 * 5 * sizeof(double));
  if (!st) return QNSCH_ENOMEM;
  s->blocks.push_back(st);
  cudaMemsetAsync(st, 0, n0 * 5 * sizeof(double), s->stream);
  int pitch0 = s->L[0].pitch;
  s->sc = st + 0 * n0 + pitch0 + 1;
  s->smu = st + 1 * n0 + pitch0 + 1;
  s->sp = st + 2 * n0 + pitch0 + 1;
  s->su = st + 3 * n0 + pitch0 + 1;
  s->sv = st + 4 * n0 + pitch0 + 1;
  double* hs = (double*)dev_alloc(s->mem, n0 * 10 * sizeof(double));
  if (!hs) return QNSCH_ENOMEM;
  s->blocks.push_back(hs);
  cudaMemsetAsync(hs, 0, n0 * 10 * sizeof(double), s->stream);
  for (int k = 0; k < 2; ++k)
    for (int q = 0; q < 5; ++q) s->hist[k][q] = hs + (size_t)(5 * k + q) * n0 + pitch0 + 1;
  int rows = qn::partial_rows_needed(s->m1, s->m2);
  s->part = (double*)dev_alloc(s->mem, (size_t)rows * 10 * sizeof(double));
  if (!s->part) return QNSCH_ENOMEM;
  s->blocks.push_back(s->part);
  size_t nstage = (size_t)(s->m1 + 1) * (s->m2 + 1);
  s->stage = (double*)dev_alloc(s->mem, nstage * sizeof(double));
  if (!s->stage) return QNSCH_ENOMEM;
  s->blocks.push_back(s->stage);
  s->scal = (double*)dev_alloc(s->mem, NSCAL * sizeof(double));
  if (!s->scal) return QNSCH_ENOMEM;
  s->blocks.push_back(s->scal);
  s->wave_ctr = (unsigned*)dev_alloc(s->mem, wave_ctr_bytes(s->m2));
  if (!s->wave_ctr) return QNSCH_ENOMEM;
  s->blocks.push_back(s->wave_ctr);
  cudaMemsetAsync(s->scal, 0, NSCAL * sizeof(double), s->stream);
  if (cudaMallocHost(&s->hbuf, NSCAL * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return QNSCH_ENOMEM;
  }
  return sync(s);
}

// error-equation levels: the 38 arrays of a level without the per-step row
// coefficients, the assembled momentum stencils and rho(c) of the iterate
// (their operators use none of them), plus the base Bc, Bmu, Bu, Bv, Bdc
constexpr int NFIELD_ERR = NFIELD - 7 - 14 + 5;
static_assert(NFIELD_ERR == 43, "error-level arrays");

template <typename T>
int alloc_err_levels(qnsch_s* s, std::vector<Lv<T>>& E) {
  if (!E.empty()) return QNSCH_OK;
  size_t need = 0;
  for (int l = 0; l < s->nlev; ++l)
    need += (size_t)s->L[l].pitch * (size_t)(s->L[l].m2 + 3) * NFIELD_ERR * sizeof(T);
  if (!reserve_bytes(need)) return QNSCH_EBUDGET;
  std::vector<Lv<T>> out(s->nlev);
  std::vector<void*> got;
  auto fail = [&](int rc) {  // give back what this call took
    cudaStreamSynchronize(s->stream);
    for (void* b : got) dev_free(s->mem, b);
    g_reserved -= need;
    return rc;
  };
  for (int l = 0; l < s->nlev; ++l) {
    const Lv<double>& D = s->L[l];
    Lv<T>& L = out[l];
    size_t n = (size_t)D.pitch * (size_t)(D.m2 + 3);
    T* base = (T*)dev_alloc(s->mem, n * NFIELD_ERR * sizeof(T));
    if (!base) return fail(QNSCH_ENOMEM);
    got.push_back(base);
    if (cudaMemsetAsync(base, 0, n * NFIELD_ERR * sizeof(T), s->stream) != cudaSuccess) {
      cudaGetLastError();
      return fail(QNSCH_ECUDA);
    }
    L.m1 = D.m1;
    L.m2 = D.m2;
    L.px = D.px;
    L.kcol = D.kcol;
    L.c8 = D.c8;
    L.pitch = D.pitch;
    L.h = (T)D.h;
    L.ih = (T)D.ih;
    L.ih2 = (T)D.ih2;
    T** f[NFIELD_ERR] = {&L.c,   &L.mu,  &L.p,   &L.u,   &L.v,    &L.fc,  &L.fmu, &L.fp,
                         &L.fu,  &L.fv,  &L.rc,  &L.rmu, &L.rp,   &L.ru,  &L.rv,  &L.sc,
                         &L.smu, &L.sp,  &L.su,  &L.sv,  &L.cn,   &L.un,  &L.vn,  &L.rhon,
                         &L.mobn, &L.visn, &L.Gn, &L.Aru, &L.Arv, &L.Sx,  &L.Sy,  &L.Qx,
                         &L.Qy,  &L.Av,  &L.Tx,  &L.Ty,  &L.Dvu,  &L.Dvv, &L.Bc,  &L.Bmu,
                         &L.Bu,  &L.Bv,  &L.Bdc};
    for (int q = 0; q < NFIELD_ERR; ++q) *f[q] = base + (size_t)q * n + D.pitch + 1;
  }
  s->blocks.insert(s->blocks.end(), got.begin(), got.end());
  s->reserved += need;
  E.swap(out);
  return QNSCH_OK;
}

template <typename T>
Prm<T> cast_prm(const Prm<double>& P) {
  Prm<T> Q;
  Q.ia = (T)P.ia;
  Q.ib = (T)P.ib;
  Q.va = (T)P.va;
  Q.vb = (T)P.vb;
  Q.alpha = (T)P.alpha;
  Q.K = (T)P.K;
  Q.Lam = (T)P.Lam;
  Q.iM = (T)P.iM;
  Q.iRe = (T)P.iRe;
  Q.iPe = (T)P.iPe;
  Q.Fr_inv = (T)P.Fr_inv;
  Q.eps_m = (T)P.eps_m;
  Q.idt = (T)P.idt;
  return Q;
}

constexpr int MAX_PROF_EVENTS = 8192;
// kinds of timed launches (qnsch_profile's bit mask)
enum { PK_VANKA0 = 0, PK_VANKA = 1, PK_COARSE = 2, PK_CH = 3, PK_WAVE = 4, PK_SKEW = 5, PK_N = 6 };
static_assert(PK_N == sizeof(qnsch_s::pk_n) / sizeof(long long), "one total per profiling kind");

// cells of Vanka colour `colour` on an m1 x m2 level (the colourings of
// colours_of: (2i + j) mod 8 when c8, else (i + 2j) mod kcol)
long long colour_cells(int m1, int m2, int kcol, int c8, int colour) {
  auto in_row = [m1](int K, int r) -> long long {  // i in [1, m1] with i % K == r
    if (r == 0) return m1 / K;
    return r <= m1 ? (m1 - r) / K + 1 : 0;
  };
  long long n = 0;
  for (int j = 1; j <= m2; ++j) {
    if (c8) {
      int d = ((colour - j) % 8 + 8) % 8;
      if (!(d & 1)) n += in_row(4, d / 2);
    } else {
      n += in_row(kcol, ((colour - 2 * j) % kcol + kcol) % kcol);
    }
  }
  return n;
}

// record a timing event on s->stream; inside a stream capture as an external
// record (a plain record there only orders the captured work and is not
// replayed as an event record node)
void prof_record(qnsch_s* s, cudaEvent_t e) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, s->stream, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s->stream);
}

// open an event pair of `kind` around the launch queued next (-1: not timed)
int prof_open(qnsch_s* s, int kind, double visits) {
  if (!((s->prof >> kind) & 1) || s->ev_used + 2 > MAX_PROF_EVENTS) return -1;
  while ((int)s->ev.size() < s->ev_used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    s->ev.push_back(e);
  }
  const int pair = s->ev_used / 2;
  if ((int)s->ev_kind.size() <= pair) {
    s->ev_kind.resize(pair + 1);
    s->ev_visits.resize(pair + 1);
  }
  s->ev_kind[pair] = kind;
  s->ev_visits[pair] = visits;
  prof_record(s, s->ev[s->ev_used]);
  return s->ev_used;
}

void prof_close(qnsch_s* s, int q) {
  if (q < 0) return;
  prof_record(s, s->ev[q + 1]);
  s->ev_used = q + 2;
}

template <typename T, class Form>
void smooth(qnsch_s* s, const std::vector<Lv<T>>& Ls, const Prm<T>& P, int l) {
  const Lv<T>& L = Ls[l];
  const int ch_max = std::is_same<Form, ErrForm>::value ? s->ch_team_max32 : s->ch_team_max;
  if constexpr (std::is_same<Form, ProjForm>::value) {
    // projection method (Sec. 7.2): CH red-black, the intermediate-velocity
    // blocks over the Vanka colours, pressure Gauss-Seidel red-black
    const double ch_cells = 0.5 * (double)L.m1 * L.m2;
    for (int c = 0; c < 2; ++c) {
      int q = l == 0 ? prof_open(s, PK_CH, ch_cells) : -1;
      qn::launch_ch<T, Form>(P, L, c, s->stream, ch_max);
      prof_close(s, q);
    }
    for (int c = 0; c < L.kcol; ++c) {
      int q = prof_open(s, l == 0 ? PK_VANKA0 : PK_VANKA,
                        (double)colour_cells(L.m1, L.m2, L.kcol, L.c8, c));
      qn::launch_vanka4<T, Form>(P, L, c, (T)s->omega, s->stream, s->team_max);
      prof_close(s, q);
    }
    qn::launch_pgs<T>(P, L, 0, s->stream, ch_max);
    qn::launch_pgs<T>(P, L, 1, s->stream, ch_max);
    return;
  }
  if (!s->coupled) {
    const double ch_cells = 0.5 * (double)L.m1 * L.m2;
    for (int c = 0; c < 2; ++c) {
      int q = l == 0 ? prof_open(s, PK_CH, ch_cells) : -1;
      qn::launch_ch<T, Form>(P, L, c, s->stream, ch_max);
      prof_close(s, q);
    }
  }
  for (int c = 0; c < L.kcol; ++c) {
    int q = prof_open(s, l == 0 ? PK_VANKA0 : PK_VANKA,
                      (double)colour_cells(L.m1, L.m2, L.kcol, L.c8, c));
    if (s->coupled) qn::launch_coupled<T, Form>(P, L, c, (T)s->omega, s->stream,
                                                std::is_same<Form, ErrForm>::value ? s->team_max32 : s->team_max);
    else qn::launch_vanka<T, Form>(P, L, c, (T)s->omega, s->stream,
                                   std::is_same<Form, ErrForm>::value ? s->team_max32 : s->team_max,
                                   std::is_same<Form, ErrForm>::value ? 0 : s->team8_max,
                                   std::is_same<Form, ErrForm>::value ? 0 : s->pair_max,
                                   std::is_same<Form, ErrForm>::value ? 0 : s->vsplit);
    prof_close(s, q);
  }
}

// n smoothing steps on level l: on a large enough error-equation level the
// skewed-chunk schedule or one banded wavefront launch, else n times the
// per-colour launches of smooth()
template <typename T, class Form>
void smooth_steps(qnsch_s* s, const std::vector<Lv<T>>& Ls, const Prm<T>& P, int l, int n) {
  if constexpr (std::is_same<Form, ErrForm>::value) {
    const Lv<T>& L = Ls[l];
    if (n > 0 && s->skew_cells > 0 && (long long)L.m1 * L.m2 >= s->skew_cells) {
      int q = l == 0 ? prof_open(s, PK_SKEW, (double)L.m1 * L.m2 * n) : -1;
      qn::launch_skew<T, Form>(P, L, n, s->coupled, s->skew_rows, (T)s->omega, s->stream);
      prof_close(s, q);
      return;
    }
    const int rows = std::max(s->wave_rows, WAVE_MIN_ROWS);
    if (n > 0 && s->wave_cells > 0 && (long long)L.m1 * L.m2 >= s->wave_cells &&
        L.m2 >= 2 * rows) {
      qn::WavePlan W;
      W.coupled = s->coupled;
      W.rows = rows;
      W.nbands = (L.m2 + rows - 1) / rows;
      W.npass = n * (s->coupled ? L.kcol : L.kcol + 2);
      W.ch_team_max = s->ch_team_max32;
      W.vanka_team_max = s->team_max32;
      W.budget = s->wave_budget;
      W.stall = s->wave_stall;
      int q = l == 0 ? prof_open(s, PK_WAVE, (double)L.m1 * L.m2 * n) : -1;
      qn::launch_wave<T, Form>(P, L, W, (T)s->omega, s->wave_ctr, s->scal + WAIT_FLAG, s->stream);
      prof_close(s, q);
      return;
    }
  }
  for (int k = 0; k < n; ++k) smooth<T, Form>(s, Ls, P, l);
}

// first level of Ls whose V-cycle runs fused in one thread block
// smoothing steps before (pre) and after the coarse-grid correction on level l
int nu_pre(const qnsch_s* s, int l) { return l == 0 && s->nu1f >= 0 ? s->nu1f : s->nu1; }
int nu_post(const qnsch_s* s, int l) { return l == 0 && s->nu2f >= 0 ? s->nu2f : s->nu2; }

template <typename T>
int fused_from(const qnsch_s* s, const std::vector<Lv<T>>& Ls) {
  long long thr = sizeof(T) == 8 ? s->fuse64 : s->fuse32;
  // the fused V-cycle runs one pair of counts on all its levels: a finest
  // level with counts of its own stays out of it
  const bool own = nu_pre(s, 0) != s->nu1 || nu_post(s, 0) != s->nu2;
  for (int l = own ? 1 : 0; l < s->nlev; ++l)
    if ((long long)Ls[l].m1 * Ls[l].m2 <= thr && s->nlev - l <= QN_MAX_FUSED_LEVELS) return l;
  return s->nlev;
}

// Sweeps on the coarsest grid: nu_coarse on a grid at most 4 cells across,
// nu_coarse * ceil(n/4)^2 when its longest side n is larger (a periodic width
// that stopped coarsening under a tall domain), since the pressure and
// chemical-potential modes there decay at a rate set by n.
static int coarse_sweeps(const qnsch_s* s) {
  int n = std::max(s->L[s->nlev - 1].m1, s->L[s->nlev - 1].m2);
  int q = std::max(1, (n + 3) / 4);
  return s->nuc * q * q;
}

// FAS V-cycle (Sec. 7.1) from level l on the level set Ls
template <typename T, class Form>
void vcycle(qnsch_s* s, const std::vector<Lv<T>>& Ls, const Prm<T>& P, int l) {
  if (l >= fused_from(s, Ls)) {
    // visits of the Vanka (or coupled) block inside the fused V-cycle: every
    // cell once per smoothing step
    double visits = 0.0;
    for (int m = l; m < s->nlev; ++m)
      visits += (double)Ls[m].m1 * Ls[m].m2 *
                (m == s->nlev - 1 ? coarse_sweeps(s) : s->nu1 + s->nu2);
    int q = prof_open(s, PK_COARSE, visits);
    s->coarse_smem_used = qn::launch_coarse_vcycle<T, Form>(
        P, &Ls[l], s->nlev - l, s->nu1, s->nu2, coarse_sweeps(s), s->kcol, (T)s->omega, s->coupled,
        s->stream, s->team8_max > 0 ? 1 : 0, s->fuse_ctas, s->coarse_smem);
    prof_close(s, q);
    return;
  }
  if (l == s->nlev - 1) {
    smooth_steps<T, Form>(s, Ls, P, l, coarse_sweeps(s));
    return;
  }
  smooth_steps<T, Form>(s, Ls, P, l, nu_pre(s, l));
  const Lv<T>& F = Ls[l];
  const Lv<T>& C = Ls[l + 1];
  qn::launch_residual<T, Form>(P, F, (double*)nullptr, s->stream);
  qn::launch_restrict_state(P, F, C, s->stream);
  qn::launch_bc_unknowns(C, s->stream);
  qn::launch_restrict_res(F, C, s->stream);
  qn::launch_add_op<T, Form>(P, C, s->stream);
  vcycle<T, Form>(s, Ls, P, l + 1);
  qn::launch_prolong(P, F, C, s->stream);
  qn::launch_bc_unknowns(F, s->stream);
  smooth_steps<T, Form>(s, Ls, P, l, nu_post(s, l));
}

// fold the recorded event pairs into the totals (stream must be idle)
void prof_collect(qnsch_s* s) {
  for (int q = 0; q + 1 < s->ev_used; q += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s->ev[q], s->ev[q + 1]) == cudaSuccess) {
      s->prof_ms += ms;
      s->prof_launches += 1;
      const int k = s->ev_kind[q / 2];
      s->pk_ms[k] += ms;
      s->pk_n[k] += 1;
      s->pk_visits[k] += s->ev_visits[q / 2];
    }
  }
  cudaGetLastError();
  s->ev_used = 0;
}

// Work queued by a call runs on s->stream.  When the caller gave no stream,
// that is a private non-blocking stream, ordered here after everything the
// caller queued on the legacy default stream before the call.
void enter(qnsch_s* s) {
  if (!s->user_stream) {
    cudaEventRecord(s->ev_entry, 0);
    cudaStreamWaitEvent(s->stream, s->ev_entry, 0);
  }
}

// queue the finest FP64 residual, its norms and (to_host) their copy to
// s->hbuf[0..9]
void enqueue_norms(qnsch_s* s, const Prm<double>& P, bool to_host = true) {
  const Lv<double>& F = s->L[0];
  if (s->scheme) qn::launch_residual<double, ProjForm>(P, F, s->part, s->stream);
  else qn::launch_residual<double, FullForm>(P, F, s->part, s->stream);
  qn::launch_norms_finalize(F, s->part, s->scal, s->stream);
  if (to_host)
    cudaMemcpyAsync(s->hbuf, s->scal, (CTL + CTL_LEN) * sizeof(double), cudaMemcpyDeviceToHost,
                    s->stream);
}

void norms_from_host(const qnsch_s* s, double* norms10) {
  for (int q = 0; q < 5; ++q) {
    norms10[q] = std::sqrt(s->hbuf[5 + q]);
    norms10[5 + q] = s->hbuf[q];
  }
}

int read_norms(qnsch_s* s, double* norms10) {
  int rc = sync(s);
  if (rc) return rc;
  norms_from_host(s, norms10);
  return QNSCH_OK;
}

// batch polling: s->ev_norms marks the norms' arrival in s->hbuf.  Returns 1
// with norms10 filled once they have arrived, 0 while they are on their way,
// QNSCH_ECUDA if the work before the event failed.
int poll_norms(qnsch_s* s, double* norms10) {
  cudaError_t e = cudaEventQuery(s->ev_norms);
  if (e == cudaErrorNotReady) return 0;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return QNSCH_ECUDA;
  }
  if (s->prof) prof_collect(s);
  norms_from_host(s, norms10);
  return 1;
}

// finest residual + norms as [l2 x5, max x5]
int residual_norms(qnsch_s* s, const Prm<double>& P, double* norms10) {
  enqueue_norms(s, P);
  s->res_valid = 1;
  return read_norms(s, norms10);
}

double maxfam(const double* n10) {
  double m = 0.0;
  for (int q = 0; q < 5; ++q) {
    if (!(n10[q] == n10[q])) return NAN;
    m = n10[q] > m ? n10[q] : m;
  }
  return m;
}

// The host layout of a field (qnsch_get_fields) as a box of the padded level
// layout: kind 0 cells (m1 x m2 from (1,1)), 1 x-edges (m1 + 1 x m2 from
// (0,1)), 2 y-edges (m1 x m2 + 1 from (1,0)); rows of `width` bytes, `rows`
// of them, `dpitch` bytes apart on the device, contiguous on the host.
struct HostBox {
  double* dev;
  size_t dpitch, width, rows;
};
HostBox host_box(const Lv<double>& V, double* a, int kind) {
  const int i0 = kind == 1 ? 0 : 1, j0 = kind == 2 ? 0 : 1;
  HostBox b;
  b.dev = a + (size_t)j0 * V.pitch + i0;
  b.dpitch = (size_t)V.pitch * sizeof(double);
  b.width = (size_t)(kind == 1 ? V.m1 + 1 : V.m1) * sizeof(double);
  b.rows = (size_t)(kind == 2 ? V.m2 + 1 : V.m2);
  return b;
}

int copy_fields_in(qnsch_s* s, double* const dst[5], const double* const src[5], bool host) {
  Lv<double> V = s->L[0];
  const int kinds[5] = {0, 0, 1, 2, 0};  // c, mu, u, v, p
  for (int q = 0; q < 5; ++q) {
    if (host) {
      // host rows straight into the padded layout (one strided copy per field;
      // the sync below returns only once every copy has read the caller's arrays)
      const HostBox b = host_box(V, dst[q], kinds[q]);
      if (cudaMemcpy2DAsync(b.dev, b.dpitch, src[q], b.width, b.width, b.rows,
                            cudaMemcpyHostToDevice, s->stream) != cudaSuccess) {
        cudaGetLastError();
        sync(s);
        return QNSCH_ECUDA;
      }
    } else {
      qn::launch_pack_in(V, dst[q], src[q], kinds[q], s->stream);
    }
  }
  Lv<double> W = V;
  W.c = dst[0];
  W.mu = dst[1];
  W.u = dst[2];
  W.v = dst[3];
  W.p = dst[4];
  if (dst[0] != V.c) W.rhoc = nullptr;  // not the iterate: no density array beside it
  qn::launch_bc_unknowns(W, s->stream);
  if (dst[0] == V.c) qn::launch_rho_fill(make_prm(s), V, s->stream);
  return sync(s);
}

int copy_fields_out(const qnsch_s* s, double* const src[5], double* const dst[5], bool host) {
  const Lv<double>& V = s->L[0];
  const int kinds[5] = {0, 0, 1, 2, 0};
  int rc = QNSCH_OK;
  for (int q = 0; q < 5; ++q) {
    if (!dst[q]) continue;
    if (host) {
      const HostBox b = host_box(V, src[q], kinds[q]);
      if (cudaMemcpy2DAsync(dst[q], b.width, b.dev, b.dpitch, b.width, b.rows,
                            cudaMemcpyDeviceToHost, s->stream) != cudaSuccess) {
        cudaGetLastError();
        rc = QNSCH_ECUDA;
        break;
      }
    } else {
      qn::launch_pack_out(V, dst[q], src[q], kinds[q], s->stream);
    }
  }
  int rs = sync(s);
  return rc ? rc : rs;
}

// the error-equation levels of the precision in use (allocated once)
int alloc_err(qnsch_s* s) {
  if (s->precision == 1) return alloc_err_levels(s, s->Ef);
  if (s->precision == 2) return alloc_err_levels(s, s->Ed);
  return QNSCH_OK;
}

// the queued part of a step's start: the committed state into the iterate and
// the frozen level-n data, then the frozen data of every level (A2)
// Weights of the step's initial iterate w[0] x^n + w[1] x^(n-1) + w[2] x^(n-2):
// the Lagrange polynomial through the committed state (time t) and the
// predictor's earlier states (t - hdt[0], t - hdt[0] - hdt[1]) evaluated at
// t + dt; (1, 0, 0) without a predictor or without history.
void predictor_weights(const qnsch_s* s, double dt, double w[3]) {
  w[0] = 1.0;
  w[1] = w[2] = 0.0;
  const int n = std::min(s->predictor, s->nhist);
  if (n == 1) {
    const double a = s->hdt[0];
    w[0] = (dt + a) / a;
    w[1] = -dt / a;
  } else if (n == 2) {
    const double a = s->hdt[0], b = s->hdt[1];
    w[0] = (dt + a) * (dt + a + b) / (a * (a + b));
    w[1] = -dt * (dt + a + b) / (a * b);
    w[2] = dt * (dt + a) / ((a + b) * b);
  }
}

// after a committed step: the state it replaced becomes hist[0] (the copies
// were queued by queue_commit)
void note_commit(qnsch_s* s) {
  if (s->predictor <= 0) return;
  s->hdt[1] = s->hdt[0];
  s->hdt[0] = s->dt;
  s->nhist = std::min(s->nhist + 1, 2);
}

void queue_begin(qnsch_s* s, double dt) {
  s->dt = dt;
  s->res_valid = 0;
  cudaMemsetAsync(s->scal + WAIT_FLAG, 0, sizeof(double), s->stream);
  Prm<double> P = make_prm(s);
  Lv<double>& F = s->L[0];
  size_t bytes = s->level_elems0 * sizeof(double);
  double* src[5] = {s->sc, s->smu, s->sp, s->su, s->sv};
  double* dst[5] = {F.c, F.mu, F.p, F.u, F.v};
  int pitch = F.pitch;
  double w[3];
  predictor_weights(s, dt, w);
  if (w[1] == 0.0 && w[2] == 0.0) {
    for (int q = 0; q < 5; ++q)
      cudaMemcpyAsync(dst[q] - pitch - 1, src[q] - pitch - 1, bytes, cudaMemcpyDeviceToDevice,
                      s->stream);
  } else {
    qn::launch_predict(dst, src, s->hist[0], s->hist[1], w, s->level_elems0, pitch + 1,
                       s->stream);
  }
  cudaMemcpyAsync(F.cn - pitch - 1, s->sc - pitch - 1, bytes, cudaMemcpyDeviceToDevice, s->stream);
  cudaMemcpyAsync(F.un - pitch - 1, s->su - pitch - 1, bytes, cudaMemcpyDeviceToDevice, s->stream);
  cudaMemcpyAsync(F.vn - pitch - 1, s->sv - pitch - 1, bytes, cudaMemcpyDeviceToDevice, s->stream);
  qn::launch_rho_fill(P, F, s->stream);
  qn::launch_frozen(P, F, s->stream);
  for (int l = 1; l < s->nlev; ++l) {
    qn::launch_restrict_frozen(s->L[l - 1], s->L[l], s->stream);
    qn::launch_frozen(P, s->L[l], s->stream);
  }
  if (s->precision == 1) {
    for (int l = 0; l < s->nlev; ++l) qn::launch_cast_frozen(s->L[l], s->Ef[l], s->stream);
  } else if (s->precision == 2) {
    for (int l = 0; l < s->nlev; ++l) qn::launch_cast_frozen(s->L[l], s->Ed[l], s->stream);
  }
}

int begin(qnsch_s* s, double dt) {
  // the error-equation levels first: a refused allocation leaves nothing queued
  int rc = alloc_err(s);
  if (rc) return rc;
  queue_begin(s, dt);
  s->pending = 1;
  return cuda_status();
}

// one defect-correction cycle: e solves N(x + e) - N(x) = r(x) approximately by
// one FAS V-cycle on the error equation in precision T; then x += e.  Requires
// the FP64 residual of x in level 0's residual arrays.
template <typename T>
void correction_cycle(qnsch_s* s, std::vector<Lv<T>>& E) {
  Prm<double> P64 = make_prm(s);
  Prm<T> P = cast_prm<T>(P64);
  qn::launch_start_correction(s->L[0], E[0], s->stream);
  // the base state on every level; the single-block V-cycle restricts it to
  // the levels below its first one itself
  int f = fused_from(s, E);
  for (int l = 1; l < s->nlev && l <= f; ++l) qn::launch_restrict_base(E[l - 1], E[l], s->stream);
  vcycle<T, ErrForm>(s, E, P, 0);
  qn::launch_apply_correction(P64, s->L[0], E[0], s->stream);
}

// all work of one outer cycle: V-cycle (or defect-correction cycle), gauge,
// FP64 residual with norms and their copy to the host
void cycle_body(qnsch_s* s, const Prm<double>& P, bool to_host = true) {
  if (s->precision == 0) {
    if (s->scheme) vcycle<double, ProjForm>(s, s->L, P, 0);
    else vcycle<double, FullForm>(s, s->L, P, 0);
  } else {
    // the residual arrays hold r(x) of the current iterate (see one_cycle)
    if (s->precision == 1) correction_cycle<float>(s, s->Ef);
    else correction_cycle<double>(s, s->Ed);
  }
  qn::launch_gauge(s->L[0], s->part, s->scal + 16, s->stream);
  enqueue_norms(s, P, to_host);
}

void drop_graph(qnsch_s* s) {
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  s->gexec = nullptr;
}

// capture cycle_body once per (dt, precision, profiling, options) and replay it
int cycle_graph(qnsch_s* s, const Prm<double>& P) {
  bool fresh = s->gexec && s->g_dt == s->dt && s->g_precision == s->precision &&
               s->g_prof == s->prof && s->g_opt == s->opt_version;
  if (!fresh) {
    drop_graph(s);
    s->ev_used = 0;
    if (s->prof) {  // create the timing events before capture begins
      int pairs = 1;
      for (int l = 0; l < s->nlev; ++l)
        pairs += (s->L[l].kcol + 2) *
                 (l == s->nlev - 1 ? coarse_sweeps(s) : nu_pre(s, l) + nu_post(s, l));
      while ((int)s->ev.size() < 2 * pairs && (int)s->ev.size() < MAX_PROF_EVENTS) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
          cudaGetLastError();
          break;
        }
        s->ev.push_back(e);
      }
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return QNSCH_ECUDA;
    }
    long long before = qn::launches_issued();
    cycle_body(s, P);
    s->g_nodes = qn::launches_issued() - before;
    g_captured += s->g_nodes;
    cudaError_t e1 = cudaStreamEndCapture(s->stream, &g);
    cudaError_t e2 = e1 == cudaSuccess ? cudaGraphInstantiate(&s->gexec, g, 0) : e1;
    if (g) cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
      cudaGetLastError();
      s->gexec = nullptr;
      s->ev_used = 0;
      return QNSCH_ECUDA;
    }
    s->g_dt = s->dt;
    s->g_precision = s->precision;
    s->g_prof = s->prof;
    s->g_opt = s->opt_version;
    s->g_ev_used = s->ev_used;  // event pairs recorded by every replay
    s->ev_used = 0;
  }
  if (cudaGraphLaunch(s->gexec, s->stream) != cudaSuccess) {
    cudaGetLastError();
    return QNSCH_ECUDA;
  }
  g_replayed += s->g_nodes;
  s->ev_used = s->g_ev_used;
  return QNSCH_OK;
}

// queue one outer cycle (as a graph replay when possible); finish_cycle waits
// for it and reads the norms
void launch_cycle(qnsch_s* s) {
  Prm<double> P = make_prm(s);
  if (s->precision != 0 && !s->res_valid)
    qn::launch_residual<double, FullForm>(P, s->L[0], (double*)nullptr, s->stream);
  bool graphed = false;
  if (s->use_graphs) {
    graphed = cycle_graph(s, P) == QNSCH_OK;
    if (!graphed) s->use_graphs = 0;  // capture unavailable: run the launches directly
  }
  if (!graphed) cycle_body(s, P);
  s->res_valid = 1;  // cycle_body ends with the residual of the new iterate
}

int finish_cycle(qnsch_s* s, double* norms10) {
  int rc = read_norms(s, norms10);
  if (s->prof) prof_collect(s);
  return rc;
}

int one_cycle(qnsch_s* s, double* norms10) {
  launch_cycle(s);
  return finish_cycle(s, norms10);
}

// queue the dissipation of the step (Thm. 6.2), the copy of the iterate into
// the committed state and (to_host) the dissipation's copy to s->hbuf[25..26];
// finish_commit waits and records
void queue_commit(qnsch_s* s, bool to_host) {
  Prm<double> P = make_prm(s);
  const Lv<double>& F = s->L[0];
  double w_visc = s->dt / s->Re, w_div = s->dt / (3.0 * s->Re), w_ch = s->dt / (s->M * s->Pe);
  qn::launch_dissipation(P, F, w_visc, w_div, w_ch, s->part, s->scal + 25, s->stream);
  size_t bytes = s->level_elems0 * sizeof(double);
  int pitch = F.pitch;
  double* src[5] = {F.c, F.mu, F.p, F.u, F.v};
  double* dst[5] = {s->sc, s->smu, s->sp, s->su, s->sv};
  if (s->predictor > 0) {  // the state being replaced moves into the history
    for (int q = 0; q < 5; ++q) {
      cudaMemcpyAsync(s->hist[1][q] - pitch - 1, s->hist[0][q] - pitch - 1, bytes,
                      cudaMemcpyDeviceToDevice, s->stream);
      cudaMemcpyAsync(s->hist[0][q] - pitch - 1, dst[q] - pitch - 1, bytes,
                      cudaMemcpyDeviceToDevice, s->stream);
    }
  }
  int nq = s->scheme ? 3 : 5;  // projection: the velocity is u^{n+1} of (pj-num-pjx)
  for (int q = 0; q < nq; ++q)
    cudaMemcpyAsync(dst[q] - pitch - 1, src[q] - pitch - 1, bytes, cudaMemcpyDeviceToDevice,
                    s->stream);
  if (s->scheme) {
    qn::launch_proj_velocity(P, F, s->su, s->sv, s->stream);
    Lv<double> S = F;  // the committed arrays, to fill their ghosts
    S.c = s->sc;
    S.mu = s->smu;
    S.p = s->sp;
    S.u = s->su;
    S.v = s->sv;
    S.rhoc = nullptr;
    qn::launch_bc_unknowns(S, s->stream);
    qn::launch_proj_diss(P, F, s->su, s->sv, s->part, s->scal + 26, s->stream);
  }
  if (to_host)
    cudaMemcpyAsync(s->hbuf + 25, s->scal + 25, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                    s->stream);
}

void launch_commit(qnsch_s* s) { queue_commit(s, true); }

int finish_commit(qnsch_s* s) {
  int rc = sync(s);
  if (rc) return rc;
  s->last_diss = s->hbuf[25] + (s->scheme ? s->hbuf[26] : 0.0);
  s->pending = 0;
  note_commit(s);
  return QNSCH_OK;
}

int commit(qnsch_s* s) {
  launch_commit(s);
  return finish_commit(s);
}

void drop_step_graph(qnsch_s* s) {
  if (s->sexec) cudaGraphExecDestroy(s->sexec);
  s->sexec = nullptr;
}

// end a capture that a failure left open on s->stream
void abandon_capture(qnsch_s* s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s->stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(s->stream, &g);
    if (g) cudaGraphDestroy(g);
  }
  cudaGetLastError();
}

// Capture one whole step of size dt as a graph:
//   prologue: start time, begin (A2), initial FP64 residual and norms, loop
//             control (first = 1);
//   WHILE (hl): one outer cycle (cycle_body) and the loop control;
//   IF (hc): the commit (dissipation and the copy into the committed state);
//   epilogue: the scalars and the control block to the host.
// Returns QNSCH_ECUDA if the runtime refuses any part; nothing is then left
// captured and the caller runs the step with the host-driven loop.
int build_step_graph(qnsch_s* s, double dt) {
  drop_step_graph(s);
  int rc = alloc_err(s);
  if (rc) return rc;
  const auto mode = cudaStreamCaptureModeThreadLocal;
  double* ctl = s->scal + CTL;
  const double limit_ns = s->time_limit > 0.0 ? s->time_limit * 1e9 : 0.0;
  cudaGraph_t G = nullptr;
  cudaGraphConditionalHandle hl = 0, hc = 0;
  bool ok = cudaGraphCreate(&G, 0) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&hl, G, 0, cudaGraphCondAssignDefault) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&hc, G, 0, cudaGraphCondAssignDefault) == cudaSuccess;
  const long long c0 = qn::launches_issued();
  long long c1 = c0, c2 = c0, c3 = c0;
  std::vector<cudaGraphNode_t> deps;
  cudaGraphNode_t wn = nullptr, in = nullptr;
  // prologue
  if (ok) ok = cudaStreamBeginCaptureToGraph(s->stream, G, nullptr, nullptr, 0, mode) == cudaSuccess;
  if (ok) {
    qn::launch_loop_clock(ctl, s->stream);
    queue_begin(s, dt);
    Prm<double> P = make_prm(s);
    enqueue_norms(s, P, false);
    qn::launch_loop_ctl(s->scal, ctl, hl, hc, s->tol, s->maxcyc, s->diverge, limit_ns, 1, s->stream);
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    ok = cudaStreamGetCaptureInfo(s->stream, &cs, nullptr, nullptr, &d, nullptr, &nd) == cudaSuccess &&
         cs == cudaStreamCaptureStatusActive;
    if (ok) deps.assign(d, d + nd);
    cudaGraph_t g = G;
    ok = cudaStreamEndCapture(s->stream, &g) == cudaSuccess && ok;
    c1 = qn::launches_issued();
  }
  // WHILE: the outer cycle
  if (ok) {
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hl;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    ok = cudaGraphAddNode(&wn, G, deps.data(), nullptr, deps.size(), &wp) == cudaSuccess;
    cudaGraph_t body = ok ? wp.conditional.phGraph_out[0] : nullptr;
    if (ok) ok = cudaStreamBeginCaptureToGraph(s->stream, body, nullptr, nullptr, 0, mode) == cudaSuccess;
    if (ok) {
      Prm<double> P = make_prm(s);
      cycle_body(s, P, false);
      qn::launch_loop_ctl(s->scal, ctl, hl, hc, s->tol, s->maxcyc, s->diverge, limit_ns, 0,
                          s->stream);
      ok = cudaStreamEndCapture(s->stream, &body) == cudaSuccess;
      c2 = qn::launches_issued();
    }
  }
  // IF: the commit
  if (ok) {
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hc;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    ok = cudaGraphAddNode(&in, G, &wn, nullptr, 1, &ip) == cudaSuccess;
    cudaGraph_t body = ok ? ip.conditional.phGraph_out[0] : nullptr;
    if (ok) ok = cudaStreamBeginCaptureToGraph(s->stream, body, nullptr, nullptr, 0, mode) == cudaSuccess;
    if (ok) {
      queue_commit(s, false);
      ok = cudaStreamEndCapture(s->stream, &body) == cudaSuccess;
      c3 = qn::launches_issued();
    }
  }
  // epilogue: scalars (dissipation) and the control block to the host
  if (ok) ok = cudaStreamBeginCaptureToGraph(s->stream, G, &in, nullptr, 1, mode) == cudaSuccess;
  if (ok) {
    cudaMemcpyAsync(s->hbuf, s->scal, (CTL + CTL_LEN) * sizeof(double), cudaMemcpyDeviceToHost,
                    s->stream);
    cudaGraph_t g = G;
    ok = cudaStreamEndCapture(s->stream, &g) == cudaSuccess;
  }
  if (ok) ok = cudaGraphInstantiate(&s->sexec, G, 0) == cudaSuccess;
  const long long issued = qn::launches_issued() - c0;
  g_captured += issued;  // none of these ran: the graph's replays count them
  if (G) cudaGraphDestroy(G);
  if (!ok) {
    abandon_capture(s);
    s->sexec = nullptr;
    return QNSCH_ECUDA;
  }
  s->s_pro = c1 - c0;
  s->s_body = c2 - c1;
  s->s_commit = c3 - c2;
  s->s_dt = dt;
  predictor_weights(s, dt, s->s_w);
  s->s_precision = s->precision;
  s->s_opt = s->opt_version;
  return QNSCH_OK;
}

// the step runs as one graph when the handle allows it: graphs on, no
// profiling (event records cannot sit inside conditional bodies)
bool device_loop_on(const qnsch_s* s) { return s->device_loop && s->use_graphs && !s->prof; }

// queue one whole step as a graph replay; QNSCH_ECUDA if the graph cannot be
// built (the handle then falls back to the host-driven loop for good)
int launch_device_step(qnsch_s* s, double dt) {
  double w[3];
  predictor_weights(s, dt, w);
  const bool fresh = s->sexec && s->s_dt == dt && s->s_precision == s->precision &&
                     s->s_opt == s->opt_version && s->s_w[0] == w[0] && s->s_w[1] == w[1] &&
                     s->s_w[2] == w[2];
  if (!fresh) {
    int rc = build_step_graph(s, dt);
    if (rc == QNSCH_ECUDA) s->device_loop = 0;
    if (rc) return rc;
  }
  s->dt = dt;
  s->pending = 1;
  if (cudaGraphLaunch(s->sexec, s->stream) != cudaSuccess) {
    cudaGetLastError();
    s->pending = 0;
    return QNSCH_ECUDA;
  }
  return QNSCH_OK;
}

// wait for a step queued by launch_device_step and read its outcome; the
// status rules are those of the host-driven loop
int finish_device_step(qnsch_s* s, int* n_vcycles, double* final_residual) {
  int rc = sync(s);
  s->pending = 0;
  if (rc) return rc;
  const double* c = s->hbuf + CTL;
  const int k = (int)c[1];
  const double r = c[0];
  const bool late = c[3] != 0.0, committed = c[5] != 0.0;
  g_replayed += s->s_pro + (long long)k * s->s_body + (committed ? s->s_commit : 0);
  s->res_valid = 1;
  if (n_vcycles) *n_vcycles = k;
  if (final_residual) *final_residual = r;
  if (c[17] != 0.0) return QNSCH_ETIMEOUT;  // a bounded wait of the smoother ran out
  if (!(r == r)) return QNSCH_ENAN;
  if (late) return QNSCH_ETIMEOUT;
  if (!committed) return QNSCH_ENOTCONV;
  s->last_diss = s->hbuf[25] + (s->scheme ? s->hbuf[26] : 0.0);
  note_commit(s);
  return QNSCH_OK;
}

// Start a host-driven step: begin (A2), the initial residual with its norms
// on their way to the host.  t0 is the time the step's clock starts from.
int host_step_start(qnsch_s* s, double dt, std::chrono::steady_clock::time_point t0) {
  int rc = begin(s, dt);
  if (rc) return rc;
  enqueue_norms(s, make_prm(s));
  s->res_valid = 1;
  cudaEventRecord(s->ev_norms, s->stream);
  s->hs_phase = 1;
  s->hs_k = s->hs_grew = s->hs_late = s->hs_expired = 0;
  s->hs_res = HUGE_VAL;
  s->hs_t0 = t0;
  return QNSCH_OK;
}

// Advance a host-driven step without waiting: 0 while it runs (the next cycle
// or the commit queued when the norms allowed), 1 once it has ended, with
// *status as qnsch_step returns it and *k, *r its cycles and last residual.
int host_step_advance(qnsch_s* s, int* status, int* k, double* r) {
  if (s->hs_phase == 3) {  // the commit
    cudaError_t e = cudaEventQuery(s->ev_norms);
    if (e == cudaErrorNotReady) return 0;
    s->hs_phase = 0;
    if (e != cudaSuccess) {
      cudaGetLastError();
      s->pending = 0;
      *status = QNSCH_ECUDA;
    } else {
      *status = finish_commit(s);
    }
    *k = s->hs_k;
    *r = s->hs_res;
    return 1;
  }
  double nrm[10];
  int got = poll_norms(s, nrm);
  if (got == 0) return 0;
  auto end = [&](int st) {
    s->hs_phase = 0;
    s->pending = 0;
    *status = st;
    *k = s->hs_k;
    *r = s->hs_res;
    return 1;
  };
  if (got < 0) return end(got);
  s->hs_res = maxfam(nrm);
  if (s->hs_phase == 2) {  // a cycle has ended
    ++s->hs_k;
    if (s->hbuf[WAIT_FLAG] != 0.0) {  // a bounded wait of the smoother ran out
      s->hs_expired = 1;
      return end(QNSCH_ETIMEOUT);
    }
    s->hs_grew = s->hs_res > s->hs_prev ? s->hs_grew + 1 : 0;
  }
  const double rr = s->hs_res;
  const bool div = s->hs_phase == 2 && s->diverge > 0 && s->hs_grew >= s->diverge;
  if (!div && rr == rr && rr > s->tol && s->hs_k < s->maxcyc) {
    if (s->time_limit > 0.0 && seconds_since(s->hs_t0) > s->time_limit) {
      s->hs_late = 1;
      return end(QNSCH_ETIMEOUT);
    }
    s->hs_prev = rr;
    launch_cycle(s);
    cudaEventRecord(s->ev_norms, s->stream);
    s->hs_phase = 2;
    return 0;
  }
  if (!(rr == rr)) return end(QNSCH_ENAN);
  if (rr > s->tol) return end(QNSCH_ENOTCONV);
  launch_commit(s);
  cudaEventRecord(s->ev_norms, s->stream);
  s->hs_phase = 3;
  return 0;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

int qnsch_set_allocator(void* (*alloc)(size_t, void*), void (*free_fn)(void*, void*), void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return QNSCH_EINVAL;
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  g_alloc = alloc;
  g_free = free_fn;
  g_ctx = ctx;
  return QNSCH_OK;
}

int qnsch_create(const qnsch_grid* grid, double rho1, double rho2, double eta1, double eta2,
                 double Re, double We, double Pe, double Cn, double Fr, qnsch_t** out) {
  if (!grid || !out) return QNSCH_EINVAL;
  if (grid->m1 < 2 || grid->m2 < 2 || !(grid->Lx > 0) || !std::isfinite(grid->Lx) ||
      grid->periodic_y)
    return QNSCH_EINVAL;
  if (std::isnan(Fr)) return QNSCH_EINVAL;
  if (grid->periodic_x && (grid->m1 % 2 != 0 || grid->m1 < 4)) return QNSCH_EINVAL;
  if (!(rho1 > 0) || !(rho2 > 0) || !(eta1 > 0) || !(eta2 > 0) || !(Re > 0) || !(We > 0) ||
      !(Pe > 0) || !(Cn > 0))
    return QNSCH_EINVAL;
  int lmax = max_levels(grid->m1, grid->m2, grid->periodic_x);
  int lev = grid->levels <= 0 ? lmax : grid->levels;
  if (lev > lmax) return QNSCH_EINVAL;
  size_t need = 0;
  if (qnsch_footprint(grid, 0, &need) != QNSCH_OK) return QNSCH_EINVAL;
  if (over_budget(need)) return QNSCH_EBUDGET;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return QNSCH_ENODEV;
  }
  qnsch_s* s = new (std::nothrow) qnsch_s();
  if (!s) return QNSCH_ENOMEM;
  if (!reserve_bytes(need)) {
    delete s;
    return QNSCH_EBUDGET;
  }
  s->reserved = need;
  {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    s->mem.alloc = g_alloc;
    s->mem.free = g_free;
    s->mem.ctx = g_ctx;
  }
  s->rho1 = rho1;
  s->rho2 = rho2;
  s->mu1 = eta1;
  s->mu2 = eta2;
  s->Re = Re;
  s->We = We;
  s->Pe = Pe;
  s->Cn = Cn;
  s->Fr_inv = (std::isinf(Fr) || Fr <= 0) ? 0.0 : 1.0 / Fr;
  s->M = Cn;
  s->eps_m = Cn;
  s->eta = eta_st(rho1, rho2);
  s->m1 = grid->m1;
  s->m2 = grid->m2;
  s->px = grid->periodic_x ? 1 : 0;
  s->kcol = colours_of(grid->m1, s->px);
  s->nlev = lev;
  s->h = grid->Lx / grid->m1;
  int rc = alloc_all(s);
  if (rc) {
    free_all(s);
    delete s;
    return rc;
  }
  *out = s;
  return QNSCH_OK;
}

int qnsch_footprint(const qnsch_grid* grid, int precision, size_t* bytes) {
  if (!grid || !bytes || grid->m1 < 2 || grid->m2 < 2 || grid->periodic_y) return QNSCH_EINVAL;
  // the kernels index an array with 32-bit integers: its padded index space
  // must fit
  if (grid->m1 > (1 << 28) || grid->m2 > (1 << 28)) return QNSCH_EINVAL;
  {
    int pitch;
    if (padded_elems(grid->m1, grid->m2, &pitch) > (size_t)INT_MAX) return QNSCH_EINVAL;
  }
  if (grid->periodic_x && (grid->m1 % 2 != 0 || grid->m1 < 4)) return QNSCH_EINVAL;
  if (precision < 0 || precision > 2) return QNSCH_EINVAL;
  int lmax = max_levels(grid->m1, grid->m2, grid->periodic_x);
  int lev = grid->levels <= 0 ? lmax : grid->levels;
  if (lev > lmax) return QNSCH_EINVAL;
  size_t total = 0;
  int a = grid->m1, b = grid->m2;
  size_t elem_err = precision == 1 ? sizeof(float) : sizeof(double);
  size_t n0 = 0;
  for (int l = 0; l < lev; ++l) {
    int pitch;
    size_t n = padded_elems(a, b, &pitch);
    if (l == 0) n0 = n;
    total += n * NFIELD * sizeof(double);
    if (precision) total += n * NFIELD_ERR * elem_err;
    a /= 2;
    b /= 2;
  }
  total += n0 * 5 * sizeof(double);                                           // committed state
  total += n0 * 10 * sizeof(double);                                          // two earlier states
  total += (size_t)qn::partial_rows_needed(grid->m1, grid->m2) * 10 * sizeof(double);
  total += (size_t)(grid->m1 + 1) * (grid->m2 + 1) * sizeof(double);         // staging
  total += NSCAL * sizeof(double);
  total += wave_ctr_bytes(grid->m2);
  *bytes = total;
  return QNSCH_OK;
}

int qnsch_version(int* major, int* minor, int* patch) {
  if (major) *major = QNSCH_VERSION_MAJOR;
  if (minor) *minor = QNSCH_VERSION_MINOR;
  if (patch) *patch = QNSCH_VERSION_PATCH;
  return QNSCH_OK;
}

int qnsch_set_budget(size_t bytes) {
  g_budget = bytes;
  return QNSCH_OK;
}

int qnsch_budget(size_t* budget, size_t* in_use) {
  if (!budget && !in_use) return QNSCH_EINVAL;
  if (budget) *budget = g_budget.load();
  if (in_use) *in_use = g_reserved.load();
  return QNSCH_OK;
}

int qnsch_destroy(qnsch_t* s) {
  if (!s) return QNSCH_EINVAL;
  if (s->stream) cudaStreamSynchronize(s->stream);
  else cudaDeviceSynchronize();
  free_all(s);
  delete s;
  return QNSCH_OK;
}

namespace {

// an option that counts something: an integer in [lo, hi] (NaN, infinities
// and fractions are refused before any conversion)
bool count_of(double v, double lo, double hi, int* out) {
  if (!(v >= lo && v <= hi) || v != std::floor(v)) return false;
  *out = (int)v;
  return true;
}

bool positive(double v) { return v > 0.0 && std::isfinite(v); }

int set_option(qnsch_s* s, const std::string& k, double value) {
  if (std::isnan(value)) return QNSCH_EINVAL;
  int n = 0;
  const double imax = (double)INT_MAX;
  if (k == "nu1" || k == "nu2" || k == "nu_coarse") {
    if (!count_of(value, 0, 1000, &n)) return QNSCH_EINVAL;
    (k == "nu1" ? s->nu1 : k == "nu2" ? s->nu2 : s->nuc) = n;
  } else if (k == "nu1_fine" || k == "nu2_fine") {
    if (!count_of(value, -1, 1000, &n)) return QNSCH_EINVAL;
    (k == "nu1_fine" ? s->nu1f : s->nu2f) = n;
  } else if (k == "maxcyc") {
    if (!count_of(value, 0, 1e6, &n)) return QNSCH_EINVAL;
    s->maxcyc = n;
  } else if (k == "tol") {
    if (!(value >= 0.0) || !std::isfinite(value)) return QNSCH_EINVAL;
    s->tol = value;
  } else if (k == "omega_vanka") {
    if (!positive(value)) return QNSCH_EINVAL;
    s->omega = value;
  } else if (k == "M" || k == "eta_st" || k == "eps_mob") {
    if (!positive(value)) return QNSCH_EINVAL;
    (k == "M" ? s->M : k == "eta_st" ? s->eta : s->eps_m) = value;
  } else if (k == "graphs") {
    s->use_graphs = value != 0.0;
  } else if (k == "device_loop") {
    s->device_loop = value != 0.0;
  } else if (k == "wave_cells32") {
    if (!(value >= 0.0 && value <= 9.0e15 && value == std::floor(value))) return QNSCH_EINVAL;
    s->wave_cells = (long long)value;
  } else if (k == "wave_rows") {
    if (!count_of(value, WAVE_MIN_ROWS, 1 << 20, &n)) return QNSCH_EINVAL;
    s->wave_rows = n;
  } else if (k == "wave_wait_cycles") {
    if (!(value >= 0.0) || !(value <= 9.0e15) || value != std::floor(value)) return QNSCH_EINVAL;
    s->wave_budget = (long long)value;
  } else if (k == "wave_stall") {
    s->wave_stall = value != 0.0;
  } else if (k == "skew_cells32") {
    if (!(value >= 0.0 && value <= 9.0e15 && value == std::floor(value))) return QNSCH_EINVAL;
    s->skew_cells = (long long)value;
  } else if (k == "skew_rows") {
    if (!count_of(value, 1, 1 << 20, &n)) return QNSCH_EINVAL;
    s->skew_rows = n;
  } else if (k == "predictor") {
    if (!count_of(value, 0, 2, &n)) return QNSCH_EINVAL;
    if (s->pending) return QNSCH_ESTATE;
    s->predictor = n;
    s->nhist = std::min(s->nhist, 0);  // the history restarts with the next committed step
  } else if (k == "history") {  // read-only but for 0, which clears it
    if (value != 0.0) return QNSCH_EINVAL;
    if (s->pending) return QNSCH_ESTATE;
    s->nhist = std::min(s->nhist, 0);
  } else if (k == "step_time_limit") {
    if (!(value >= 0.0) || !std::isfinite(value)) return QNSCH_EINVAL;
    s->time_limit = value;
  } else if (k == "diverge_cycles") {
    if (!count_of(value, 0, 1e6, &n)) return QNSCH_EINVAL;
    s->diverge = n;
  } else if (k == "fuse_cells" || k == "fuse_cells32" || k == "vanka_team_max" ||
             k == "ch_team_max" || k == "ch_team_max32" || k == "vanka_team_max32" ||
             k == "vanka_team8_max" || k == "vanka_pair_max" || k == "vanka_split" ||
             k == "coarse_smem") {
    if (!count_of(value, 0, imax, &n)) return QNSCH_EINVAL;
    (k == "fuse_cells" ? s->fuse64 : k == "fuse_cells32" ? s->fuse32
     : k == "vanka_team_max" ? s->team_max : k == "ch_team_max" ? s->ch_team_max
     : k == "ch_team_max32" ? s->ch_team_max32 : k == "vanka_team8_max" ? s->team8_max
     : k == "vanka_pair_max" ? s->pair_max : k == "vanka_split" ? s->vsplit
     : k == "coarse_smem" ? s->coarse_smem : s->team_max32) = n;
  } else if (k == "fuse_ctas") {
    if (!count_of(value, 1, 16, &n) || (n & (n - 1))) return QNSCH_EINVAL;
    // the largest cluster at most n blocks wide that this device can launch
    s->fuse_ctas = qn::coarse_cluster_blocks(n);
  } else if (k == "coupled") {
    if (value != 0.0 && s->scheme) return QNSCH_EINVAL;  // a primitive-method smoother
    s->coupled = value != 0.0;
  } else if (k == "pdl") {
    g_pdl_option = value != 0.0;
    qn::set_pdl(g_pdl_option.load());
  } else if (k == "precision") {
    if (!count_of(value, 0, 2, &n)) return QNSCH_EINVAL;
    if (n != 0 && s->scheme) return QNSCH_EINVAL;  // the projection method runs in FP64
    if (s->pending) return QNSCH_ESTATE;
    s->precision = n;
  } else if (k == "scheme") {
    if (!count_of(value, 0, 1, &n)) return QNSCH_EINVAL;
    if (n == 1 && (s->coupled || s->precision != 0)) return QNSCH_EINVAL;
    if (s->pending) return QNSCH_ESTATE;
    s->scheme = n;
  } else {
    return QNSCH_EINVAL;
  }
  return QNSCH_OK;
}

}  // namespace

int qnsch_set_option(qnsch_t* s, const char* key, double value) {
  if (!s || !key) return QNSCH_EINVAL;
  int rc = set_option(s, std::string(key), value);
  if (rc == QNSCH_OK) ++s->opt_version;  // the next cycle recaptures its graph
  return rc;
}

int qnsch_get_option(const qnsch_t* s, const char* key, double* value) {
  if (!s || !key || !value) return QNSCH_EINVAL;
  std::string k(key);
  if (k == "nu1") *value = s->nu1;
  else if (k == "nu2") *value = s->nu2;
  else if (k == "nu1_fine") *value = s->nu1f;
  else if (k == "nu2_fine") *value = s->nu2f;
  else if (k == "nu_coarse") *value = s->nuc;
  else if (k == "maxcyc") *value = s->maxcyc;
  else if (k == "tol") *value = s->tol;
  else if (k == "omega_vanka") *value = s->omega;
  else if (k == "M") *value = s->M;
  else if (k == "eta_st") *value = s->eta;
  else if (k == "eps_mob") *value = s->eps_m;
  else if (k == "precision") *value = s->precision;
  else if (k == "graphs") *value = s->use_graphs;
  else if (k == "device_loop") *value = s->device_loop;
  else if (k == "wave_cells32") *value = (double)s->wave_cells;
  else if (k == "wave_rows") *value = s->wave_rows;
  else if (k == "wave_wait_cycles") *value = (double)s->wave_budget;
  else if (k == "wave_stall") *value = s->wave_stall;
  else if (k == "skew_cells32") *value = (double)s->skew_cells;
  else if (k == "skew_rows") *value = s->skew_rows;
  else if (k == "predictor") *value = s->predictor;
  else if (k == "history") *value = std::max(s->nhist, 0);
  else if (k == "step_time_limit") *value = s->time_limit;
  else if (k == "diverge_cycles") *value = s->diverge;
  else if (k == "fuse_cells") *value = s->fuse64;
  else if (k == "fuse_ctas") *value = s->fuse_ctas;
  else if (k == "coupled") *value = s->coupled;
  else if (k == "fuse_cells32") *value = s->fuse32;
  else if (k == "scheme") *value = s->scheme;
  else if (k == "vanka_team_max") *value = s->team_max;
  else if (k == "ch_team_max") *value = s->ch_team_max;
  else if (k == "ch_team_max32") *value = s->ch_team_max32;
  else if (k == "vanka_team_max32") *value = s->team_max32;
  else if (k == "vanka_team8_max") *value = s->team8_max;
  else if (k == "vanka_pair_max") *value = s->pair_max;
  else if (k == "vanka_split") *value = s->vsplit;
  else if (k == "coarse_smem") *value = s->coarse_smem;
  else if (k == "coarse_smem_used") *value = s->coarse_smem_used;
  else if (k == "pdl") *value = g_pdl_option.load();
  else return QNSCH_EINVAL;
  return QNSCH_OK;
}

int qnsch_set_stream(qnsch_t* s, void* stream) {
  if (!s) return QNSCH_EINVAL;
  if (sync(s)) return QNSCH_ECUDA;
  s->user_stream = (cudaStream_t)stream;
  s->stream = s->user_stream ? s->user_stream : s->own_stream;
  return QNSCH_OK;
}

int qnsch_profile(qnsch_t* s, int enable) {
  if (!s) return QNSCH_EINVAL;
  if (s->ev_used) {
    cudaStreamSynchronize(s->stream);
    prof_collect(s);
  }
  if (enable < 0 || enable >= (1 << PK_N)) return QNSCH_EINVAL;
  s->prof = enable;
  s->prof_launches = 0;
  s->prof_ms = 0.0;
  for (int k = 0; k < PK_N; ++k) {
    s->pk_n[k] = 0;
    s->pk_ms[k] = 0.0;
    s->pk_visits[k] = 0.0;
  }
  return QNSCH_OK;
}

int qnsch_profile_read_kind(qnsch_t* s, int kind, long long* launches, double* total_ms,
                            double* visits) {
  if (!s || kind < 0 || kind >= PK_N || !launches || !total_ms || !visits) return QNSCH_EINVAL;
  if (s->ev_used) {
    int rc = sync(s);
    if (rc) return rc;
    prof_collect(s);
  }
  *launches = s->pk_n[kind];
  *total_ms = s->pk_ms[kind];
  *visits = s->pk_visits[kind];
  return QNSCH_OK;
}

int qnsch_profile_read(qnsch_t* s, long long* launches, double* total_ms) {
  if (!s || !launches || !total_ms) return QNSCH_EINVAL;
  if (s->ev_used) {
    int rc = sync(s);
    if (rc) return rc;
    prof_collect(s);
  }
  *launches = s->prof_launches;
  *total_ms = s->prof_ms;
  return QNSCH_OK;
}

int qnsch_kernel_launches(long long* n) {
  if (!n) return QNSCH_EINVAL;
  *n = qn::launches_issued() - g_captured + g_replayed;
  return QNSCH_OK;
}

int qnsch_levels(const qnsch_t* s) { return s ? s->nlev : QNSCH_EINVAL; }
int qnsch_ncolours_vanka(const qnsch_t* s) { return s ? s->kcol : QNSCH_EINVAL; }

int qnsch_set_fields(qnsch_t* s, const double* c, const double* mu, const double* u,
                     const double* v, const double* p) {
  if (!s || !c || !mu || !u || !v || !p) return QNSCH_EINVAL;
  if (s->pending) return QNSCH_ESTATE;
  double* dst[5] = {s->sc, s->smu, s->su, s->sv, s->sp};
  const double* src[5] = {c, mu, u, v, p};
  s->nhist = -1;  // a state from the caller: no history, and no node itself
  return copy_fields_in(s, dst, src, true);
}

int qnsch_set_fields_device(qnsch_t* s, const double* c, const double* mu, const double* u,
                            const double* v, const double* p) {
  if (!s || !c || !mu || !u || !v || !p) return QNSCH_EINVAL;
  if (s->pending) return QNSCH_ESTATE;
  double* dst[5] = {s->sc, s->smu, s->su, s->sv, s->sp};
  const double* src[5] = {c, mu, u, v, p};
  s->nhist = -1;
  enter(s);
  return copy_fields_in(s, dst, src, false);
}

int qnsch_get_history(const qnsch_t* s, int k, double* dt, double* c, double* mu, double* u,
                      double* v, double* p) {
  if (!s || !dt || k < 0 || k >= s->nhist) return QNSCH_EINVAL;
  if (s->pending) return QNSCH_ESTATE;
  double* src[5] = {s->hist[k][0], s->hist[k][1], s->hist[k][3], s->hist[k][4], s->hist[k][2]};
  double* dst[5] = {c, mu, u, v, p};
  *dt = s->hdt[k];
  return copy_fields_out(s, src, dst, true);
}

int qnsch_set_history(qnsch_t* s, int k, double dt, const double* c, const double* mu,
                      const double* u, const double* v, const double* p) {
  if (!s || !c || !mu || !u || !v || !p || k < 0 || k > std::max(s->nhist, 0) || k > 1)
    return QNSCH_EINVAL;
  if (!(dt > 0.0) || !std::isfinite(dt)) return QNSCH_EINVAL;
  if (s->pending) return QNSCH_ESTATE;
  double* dst[5] = {s->hist[k][0], s->hist[k][1], s->hist[k][3], s->hist[k][4], s->hist[k][2]};
  const double* src[5] = {c, mu, u, v, p};
  int rc = copy_fields_in(s, dst, src, true);
  if (rc) return rc;
  s->hdt[k] = dt;
  if (k >= s->nhist) s->nhist = k + 1;  // the committed state is a node too
  return QNSCH_OK;
}

int qnsch_get_fields(const qnsch_t* s, double* c, double* mu, double* u, double* v, double* p) {
  if (!s) return QNSCH_EINVAL;
  double* src[5] = {s->sc, s->smu, s->su, s->sv, s->sp};
  double* dst[5] = {c, mu, u, v, p};
  return copy_fields_out(s, src, dst, true);
}

int qnsch_get_fields_device(const qnsch_t* s, double* c, double* mu, double* u, double* v,
                            double* p) {
  if (!s) return QNSCH_EINVAL;
  double* src[5] = {s->sc, s->smu, s->su, s->sv, s->sp};
  double* dst[5] = {c, mu, u, v, p};
  enter(const_cast<qnsch_s*>(s));
  return copy_fields_out(s, src, dst, false);
}

int qnsch_begin_step(qnsch_t* s, double dt) {
  if (!s || !(dt > 0) || !std::isfinite(dt)) return QNSCH_EINVAL;
  if (s->async) return QNSCH_ESTATE;
  int rc = begin(s, dt);
  if (rc) return rc;
  return sync(s);
}

int qnsch_vcycle(qnsch_t* s, double* norms10) {
  if (!s) return QNSCH_EINVAL;
  if (!s->pending || s->async) return QNSCH_ESTATE;
  double n[10];
  int rc = one_cycle(s, n);
  if (rc) return rc;
  if (norms10) std::memcpy(norms10, n, sizeof(n));
  return QNSCH_OK;
}

int qnsch_commit_step(qnsch_t* s) {
  if (!s) return QNSCH_EINVAL;
  if (!s->pending || s->async) return QNSCH_ESTATE;
  return commit(s);
}

int qnsch_step(qnsch_t* s, double dt, int* n_vcycles, double* final_residual) {
  if (!s || !(dt > 0) || !std::isfinite(dt)) return QNSCH_EINVAL;
  if (s->pending || s->async) return QNSCH_ESTATE;
  if (device_loop_on(s)) {
    int rc = launch_device_step(s, dt);
    if (rc == QNSCH_OK) return finish_device_step(s, n_vcycles, final_residual);
    if (rc != QNSCH_ECUDA || device_loop_on(s)) return rc;
    // the runtime refused the step graph: the host-driven loop below
  }
  const auto t0 = std::chrono::steady_clock::now();
  int rc = begin(s, dt);
  if (rc) return rc;
  Prm<double> P = make_prm(s);
  double n[10];
  rc = residual_norms(s, P, n);
  if (rc) return rc;
  int k = 0, grew = 0, late = 0, expired = 0;
  double r = maxfam(n);
  while (r == r && r > s->tol && k < s->maxcyc) {
    if (s->time_limit > 0.0 && seconds_since(t0) > s->time_limit) {
      late = 1;
      break;
    }
    const double prev = r;
    rc = one_cycle(s, n);
    if (rc) return rc;
    r = maxfam(n);
    ++k;
    if (s->hbuf[WAIT_FLAG] != 0.0) {  // a bounded wait of the smoother ran out
      expired = 1;
      break;
    }
    grew = r > prev ? grew + 1 : 0;
    if (s->diverge > 0 && grew >= s->diverge) break;
  }
  if (n_vcycles) *n_vcycles = k;
  if (final_residual) *final_residual = r;
  if (expired) {  // the cycle's result is not to be trusted, whatever its residual
    s->pending = 0;
    return QNSCH_ETIMEOUT;
  }
  if (!(r == r)) {
    s->pending = 0;
    return QNSCH_ENAN;
  }
  if (late) {
    s->pending = 0;
    return QNSCH_ETIMEOUT;
  }
  if (r > s->tol) {
    s->pending = 0;
    return QNSCH_ENOTCONV;
  }
  return commit(s);
}

int qnsch_step_launch(qnsch_t* s, double dt) {
  if (!s || !(dt > 0) || !std::isfinite(dt)) return QNSCH_EINVAL;
  if (s->pending || s->async) return QNSCH_ESTATE;
  if (device_loop_on(s)) {
    cudaEventRecord(s->ev_s0, s->stream);
    int rc = launch_device_step(s, dt);
    if (rc == QNSCH_OK) {
      cudaEventRecord(s->ev_s1, s->stream);
      s->async = 1;
      return QNSCH_OK;
    }
    if (rc != QNSCH_ECUDA || device_loop_on(s)) return rc;
  }
  // no device-side loop: a host-driven step that each poll advances
  cudaEventRecord(s->ev_s0, s->stream);
  int rc = host_step_start(s, dt, std::chrono::steady_clock::now());
  if (rc) return rc;
  s->async = 2;
  return QNSCH_OK;
}

int qnsch_step_poll(qnsch_t* s, int* done, int* n_vcycles, double* final_residual, int* status,
                    double* device_ms) {
  if (!s || !done) return QNSCH_EINVAL;
  if (!s->async) return QNSCH_ESTATE;
  int st = 0, k = 0;
  double r = 0.0;
  if (s->async == 2) {
    if (!host_step_advance(s, &st, &k, &r)) {
      *done = 0;
      return QNSCH_OK;
    }
    cudaEventRecord(s->ev_s1, s->stream);
    cudaEventSynchronize(s->ev_s1);  // the step's work has ended: immediate
  } else {
    cudaError_t e = cudaEventQuery(s->ev_s1);
    if (e == cudaErrorNotReady) {
      *done = 0;
      return QNSCH_OK;
    }
    if (e != cudaSuccess) cudaGetLastError();
    st = finish_device_step(s, &k, &r);
  }
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, s->ev_s0, s->ev_s1) != cudaSuccess) {
    cudaGetLastError();
    ms = -1.f;
  }
  s->async = 0;
  *done = 1;
  if (n_vcycles) *n_vcycles = k;
  if (final_residual) *final_residual = r;
  if (status) *status = st;
  if (device_ms) *device_ms = ms;
  return QNSCH_OK;
}

int qnsch_mass(const qnsch_t* s, double* mass_rho, double* mass_rhoc) {
  if (!s || !mass_rho || !mass_rhoc) return QNSCH_EINVAL;
  qnsch_s* m = const_cast<qnsch_s*>(s);
  Prm<double> P = make_prm(s);
  qn::launch_mass(P, s->L[0], (const double*)s->sc, s->part, s->scal + 20, s->stream);
  cudaMemcpyAsync(m->hbuf + 20, s->scal + 20, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                  s->stream);
  int rc = sync(s);
  if (rc) return rc;
  *mass_rho = m->hbuf[20];
  *mass_rhoc = m->hbuf[21];
  return QNSCH_OK;
}

int qnsch_diagnostics(const qnsch_t* s, double* out) {
  if (!s || !out) return QNSCH_EINVAL;
  qnsch_s* m = const_cast<qnsch_s*>(s);
  const Lv<double>& F = s->L[0];
  qn::launch_diag(F, s->sc, s->su, s->sv, s->part, s->scal + 32, s->stream);
  cudaMemcpyAsync(m->hbuf + 32, s->scal + 32, 11 * sizeof(double), cudaMemcpyDeviceToHost,
                  s->stream);
  int rc = sync(s);
  if (rc) return rc;
  const double* a = m->hbuf + 32;  // cells: max x3, sums x4; columns: max x2, sums x2
  double h = s->h, Ly = s->m2 * s->h;
  out[0] = a[4] / a[3];
  out[1] = a[5] / a[3];
  out[2] = a[0];
  out[3] = std::sqrt(h * h * a[6]);
  out[4] = a[1];
  out[5] = a[2];
  out[6] = 2.0 / s->m1 * a[9];
  bool any = a[10] > 0.0;
  out[7] = any ? a[7] : 0.0;
  out[8] = any ? Ly - a[8] : Ly;
  return QNSCH_OK;
}

int qnsch_divergence(const qnsch_t* s, double* div) {
  if (!s || !div) return QNSCH_EINVAL;
  const Lv<double>& F = s->L[0];
  qn::launch_div_field(F, s->su, s->sv, s->stage, s->stream);
  if (cudaMemcpyAsync(div, s->stage, (size_t)s->m1 * s->m2 * sizeof(double),
                      cudaMemcpyDeviceToHost, s->stream) != cudaSuccess) {
    cudaGetLastError();
    return QNSCH_ECUDA;
  }
  return sync(s);
}

static int energy_of(const qnsch_s* s, const double* c, const double* u, const double* v,
                     double* E) {
  qnsch_s* m = const_cast<qnsch_s*>(s);
  Prm<double> P = make_prm(s);
  double w_grad = s->Cn * s->eta / s->We;          // (eps eta / (2 We)) / (1/2)
  double w_bulk = s->eta / (s->Cn * s->We);
  double w_pot = s->Fr_inv;
  // k_energy sums rho [ (a_x u^2 + a_y v^2)/2 + w_grad G / 2 + w_bulk F + w_pot y ]:
  qn::launch_energy(P, s->L[0], c, u, v, 0.5 * w_grad, w_bulk, w_pot, s->part, s->scal + 24,
                    s->stream);
  cudaMemcpyAsync(m->hbuf + 24, s->scal + 24, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  int rc = sync(s);
  if (rc) return rc;
  *E = m->hbuf[24];
  return QNSCH_OK;
}

int qnsch_energy(const qnsch_t* s, double* E, double* last_dissipation) {
  if (!s || !E) return QNSCH_EINVAL;
  int rc = energy_of(s, s->sc, s->su, s->sv, E);
  if (rc) return rc;
  if (last_dissipation) *last_dissipation = s->last_diss;
  return QNSCH_OK;
}

int qnsch_iterate_energy(const qnsch_t* s, double* E, double* D) {
  if (!s || !E) return QNSCH_EINVAL;
  if (!s->pending || s->async) return QNSCH_ESTATE;
  const Lv<double>& F = s->L[0];
  int rc = energy_of(s, F.c, F.u, F.v, E);
  if (rc) return rc;
  if (D) {
    qnsch_s* m = const_cast<qnsch_s*>(s);
    Prm<double> P = make_prm(s);
    double w_visc = s->dt / s->Re, w_div = s->dt / (3.0 * s->Re), w_ch = s->dt / (s->M * s->Pe);
    qn::launch_dissipation(P, F, w_visc, w_div, w_ch, s->part, s->scal + 25, s->stream);
    cudaMemcpyAsync(m->hbuf + 25, s->scal + 25, sizeof(double), cudaMemcpyDeviceToHost,
                    s->stream);
    rc = sync(s);
    if (rc) return rc;
    *D = m->hbuf[25];
  }
  return QNSCH_OK;
}

int qnsch_set_iterate(qnsch_t* s, const double* c, const double* mu, const double* u,
                      const double* v, const double* p) {
  if (s) s->res_valid = 0;
  if (!s || !c || !mu || !u || !v || !p) return QNSCH_EINVAL;
  if (!s->pending || s->async) return QNSCH_ESTATE;
  const Lv<double>& F = s->L[0];
  double* dst[5] = {F.c, F.mu, F.u, F.v, F.p};
  const double* src[5] = {c, mu, u, v, p};
  return copy_fields_in(s, dst, src, true);
}

int qnsch_get_iterate(const qnsch_t* s, double* c, double* mu, double* u, double* v, double* p) {
  if (!s) return QNSCH_EINVAL;
  if (!s->pending || s->async) return QNSCH_ESTATE;
  const Lv<double>& F = s->L[0];
  double* src[5] = {F.c, F.mu, F.u, F.v, F.p};
  double* dst[5] = {c, mu, u, v, p};
  return copy_fields_out(s, src, dst, true);
}

int qnsch_residual(qnsch_t* s, double* rc_, double* rmu, double* rp, double* ru, double* rv,
                   double* norms10) {
  if (!s) return QNSCH_EINVAL;
  if (!s->pending || s->async) return QNSCH_ESTATE;
  Prm<double> P = make_prm(s);
  double n[10];
  int rc = residual_norms(s, P, n);
  if (rc) return rc;
  if (norms10) std::memcpy(norms10, n, sizeof(n));
  const Lv<double>& F = s->L[0];
  double* src[5] = {F.rc, F.rmu, F.ru, F.rv, F.rp};
  double* dst[5] = {rc_, rmu, ru, rv, rp};
  return copy_fields_out(s, src, dst, true);
}

int qnsch_smooth_ch(qnsch_t* s, int colour) {
  if (s) s->res_valid = 0;
  if (!s || colour < 0 || colour > 1) return QNSCH_EINVAL;
  if (!s->pending || s->async) return QNSCH_ESTATE;
  if (s->scheme) qn::launch_ch<double, ProjForm>(make_prm(s), s->L[0], colour, s->stream);
  else qn::launch_ch<double, FullForm>(make_prm(s), s->L[0], colour, s->stream, s->ch_team_max);
  return sync(s);
}

int qnsch_smooth_vanka(qnsch_t* s, int colour) {
  if (s) s->res_valid = 0;
  if (!s || colour < 0 || colour >= s->kcol) return QNSCH_EINVAL;
  if (!s->pending || s->async) return QNSCH_ESTATE;
  if (s->scheme)
    qn::launch_vanka4<double, ProjForm>(make_prm(s), s->L[0], colour, s->omega, s->stream, s->team_max);
  else qn::launch_vanka<double, FullForm>(make_prm(s), s->L[0], colour, s->omega, s->stream,
                                          s->team_max);
  return sync(s);
}

// ----------------------------------------------------------------------------
// batches of independent instances
// ----------------------------------------------------------------------------
struct qnsch_batch_s {
  std::vector<qnsch_s*> inst;
  // at most this many members step at once (0: all); the others start, in
  // member order, as running ones finish their steps
  int max_inflight = 0;
  // each member's last batch step on its stream: from the event before its
  // start to the event after its end (ms; -1 if not timed)
  std::vector<double> step_ms;
};

int qnsch_batch_create(int n, qnsch_t* const* insts, qnsch_batch_t** out) {
  if (n <= 0 || !insts || !out) return QNSCH_EINVAL;
  for (int a = 0; a < n; ++a) {
    if (!insts[a]) return QNSCH_EINVAL;
    for (int b = 0; b < a; ++b)
      if (insts[a] == insts[b] || (insts[a]->stream == insts[b]->stream)) return QNSCH_EINVAL;
  }
  qnsch_batch_s* B = new (std::nothrow) qnsch_batch_s();
  if (!B) return QNSCH_ENOMEM;
  B->inst.assign(insts, insts + n);
  *out = B;
  return QNSCH_OK;
}

int qnsch_batch_destroy(qnsch_batch_t* B) {
  if (!B) return QNSCH_EINVAL;
  delete B;
  return QNSCH_OK;
}

int qnsch_batch_size(const qnsch_batch_t* B) { return B ? (int)B->inst.size() : QNSCH_EINVAL; }

int qnsch_batch_step(qnsch_batch_t* B, const double* dt, int* status, int* n_vcycles) {
  if (!B || !dt || !status) return QNSCH_EINVAL;
  const int n = (int)B->inst.size();
  for (int a = 0; a < n; ++a) {
    if (!(dt[a] > 0) || !std::isfinite(dt[a]) || B->inst[a]->pending) return QNSCH_EINVAL;
    // a member moved onto another member's stream (qnsch_set_stream after
    // qnsch_batch_create) would serialise their cycles and share their events
    for (int b = 0; b < a; ++b)
      if (B->inst[a]->stream == B->inst[b]->stream) return QNSCH_EINVAL;
  }
  // Each member advances through its own host-driven step: its next cycle is
  // queued as soon as its norms arrive, so instances of different sizes do
  // not wait for one another.  (The members' whole-step graphs with the loop
  // on the device measured slower here: 64 such graphs on 64 streams took
  // 194 ms per batch step against 114 ms host-driven.)
  const auto t0 = std::chrono::steady_clock::now();
  const int cap = B->max_inflight > 0 ? std::min(B->max_inflight, n) : n;
  std::vector<char> running(n, 0);
  int next = 0, inflight = 0;
  B->step_ms.assign(n, -1.0);
  auto start_more = [&]() {
    while (inflight < cap && next < n) {
      const int a = next++;
      if (n_vcycles) n_vcycles[a] = 0;
      cudaEventRecord(B->inst[a]->ev_s0, B->inst[a]->stream);
      status[a] = host_step_start(B->inst[a], dt[a], t0);
      running[a] = status[a] == QNSCH_OK;
      inflight += running[a];
    }
  };
  start_more();
  while (inflight > 0) {
    for (int a = 0; a < next; ++a) {
      if (!running[a]) continue;
      int st = 0, k = 0;
      double r = 0.0;
      if (host_step_advance(B->inst[a], &st, &k, &r)) {
        running[a] = 0;
        --inflight;
        status[a] = st;
        if (n_vcycles) n_vcycles[a] = k;
        cudaEventRecord(B->inst[a]->ev_s1, B->inst[a]->stream);
        start_more();
      }
    }
  }
  for (int a = 0; a < n; ++a) {  // every member's work has ended: the events are done
    float ms = 0.f;
    if (cudaEventSynchronize(B->inst[a]->ev_s1) == cudaSuccess &&
        cudaEventElapsedTime(&ms, B->inst[a]->ev_s0, B->inst[a]->ev_s1) == cudaSuccess)
      B->step_ms[a] = ms;
    else
      cudaGetLastError();
  }
  return QNSCH_OK;
}

int qnsch_batch_step_times(const qnsch_batch_t* B, double* ms) {
  if (!B || !ms) return QNSCH_EINVAL;
  for (size_t a = 0; a < B->inst.size(); ++a)
    ms[a] = a < B->step_ms.size() ? B->step_ms[a] : -1.0;
  return QNSCH_OK;
}

int qnsch_batch_set_option(qnsch_batch_t* B, const char* key, double value) {
  if (!B || !key) return QNSCH_EINVAL;
  if (std::string(key) == "max_inflight") {
    if (!(value >= 0.0 && value <= 1e6 && value == std::floor(value))) return QNSCH_EINVAL;
    B->max_inflight = (int)value;
    return QNSCH_OK;
  }
  return QNSCH_EINVAL;
}

int qnsch_smooth(qnsch_t* s, int sweeps) {
  if (s) s->res_valid = 0;
  if (!s || sweeps < 0) return QNSCH_EINVAL;
  if (!s->pending || s->async) return QNSCH_ESTATE;
  Prm<double> P = make_prm(s);
  for (int k = 0; k < sweeps; ++k) {
    if (s->scheme) smooth<double, ProjForm>(s, s->L, P, 0);
    else smooth<double, FullForm>(s, s->L, P, 0);
  }
  return sync(s);
}

}  // extern "C"
