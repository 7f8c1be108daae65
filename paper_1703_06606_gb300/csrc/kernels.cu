// kernels.cu -- CUDA kernels (sm_103a) for one implicit step of the primitive
// q-NSCH scheme of arXiv:1703.06606: residual with fused norms (Sec. 6.1),
// CH 2x2 Newton Gauss-Seidel and 5x5 Vanka smoothers (Sec. 7.1), FAS
// transfers, frozen-data setup, ghost filling (App. A.6), and FP64 reductions
// for the norms, the mean of p, mass (Thm. 6.1) and energy (Thm. 6.2).
#include <cuda_runtime.h>
#include <math_constants.h>

#include <atomic>
#include <algorithm>
#include <type_traits>

#include "kernels.h"
#include "qnsch_dev.cuh"

namespace qn {

constexpr int BX = 32, BY = 8, NT = BX * BY;

static inline dim3 grid2(int nx, int ny) { return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY); }

// number of kernels issued by this library since load (host-side count;
// atomic, since host threads may drive different handles at once)
static std::atomic<long long> g_launches{0};
long long launches_issued() { return g_launches.load(); }

// Programmatic dependent launch (sm_90 and later).  Every kernel of the step is
// launched with programmatic stream serialisation: it is scheduled as the
// blocks of its predecessor in the stream exit, and its threads wait
// (griddepcontrol.wait) until the predecessor grid has completed and its
// memory is visible.  The wait comes before any access to global memory, so
// the order of effects is that of plain stream order; what is saved is part of
// the gap between dependent launches (measured: ~1.3 % of a droplet step).  An
// explicit early trigger (griddepcontrol.launch_dependents at kernel entry)
// measured 13 % slower: the successor's blocks were placed while the
// predecessor still held the SMs, and these latency-bound launches lost their
// even spread over the sub-partitions.
static std::atomic<int> g_pdl{1};
void set_pdl(int on) { g_pdl = on ? 1 : 0; }
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
template <typename... KArgs, typename... Args>
static void qlaunch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                    Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = g_pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// --------------------------------------------------------------------------
// block reduction helpers (fixed order: deterministic for a fixed launch shape)
// --------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum_store(double (&val)[NV], double* part, int nmax_first) {
  // first `nmax_first` values are reduced with max, the rest with sum.  The
  // max values are non-negative (or NaN), whose bit patterns order as the
  // values do (a NaN above everything), so the warp stage takes their max as
  // 64-bit integers, off the FP64 pipe.
  __shared__ double sh[NT / 32][NV];
  int lane = (threadIdx.y * BX + threadIdx.x) & 31, warp = (threadIdx.y * BX + threadIdx.x) >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double x = val[q];
    if (q < nmax_first) {
      long long b = __double_as_longlong(x);
      for (int o = 16; o > 0; o >>= 1) {
        long long c = __shfl_down_sync(0xffffffffu, b, o);
        b = c > b ? c : b;
      }
      x = __longlong_as_double(b);
    } else {
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    }
    if (lane == 0) sh[warp][q] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double x = lane < NT / 32 ? sh[lane][q] : (q < nmax_first ? 0.0 : 0.0);
      for (int o = 16; o > 0; o >>= 1) {
        double y = __shfl_down_sync(0xffffffffu, x, o);
        x = (q < nmax_first) ? fmax(x, y) : x + y;
      }
      if (lane == 0) part[(blockIdx.y * gridDim.x + blockIdx.x) * NV + q] = x;
    }
  }
}

// Sum (or max) nparts rows of NV partials in a fixed order; one block of 256.
__global__ void k_finalize(const double* part, int nparts, int nv, int nmax_first, double scale_sum,
                           double* out) {
  pdl_enter();
  __shared__ double sh[256];
  for (int q = 0; q < nv; ++q) {
    bool mx = q < nmax_first;
    double acc = 0.0;
    for (int p = threadIdx.x; p < nparts; p += 256) {
      double x = part[p * nv + q];
      acc = mx ? fmax(acc, x) : acc + x;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] = mx ? fmax(sh[threadIdx.x], sh[threadIdx.x + s])
                                                 : sh[threadIdx.x] + sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = mx ? sh[0] : sh[0] * scale_sum;
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// residual r = f - N(x) (mode 0, optional norms) or f += N(x) (mode 1)
// thread (i,j): cell families at (i,j), u-edge (i,j) and v-edge (i,j)
// --------------------------------------------------------------------------
// r = f - N(x) (MODE 0; val receives |r| and r^2 per family) or f += N(x) (MODE 1)
// at thread (i,j): cell families at (i,j), u-edge (i,j) and v-edge (i,j)
template <typename T, int MODE, class Form>
__device__ __forceinline__ void residual_cell(const Prm<T>& P, const Lv<T>& L, int i, int j,
                                              double (&val)[10]) {
  int k = L.at(i, j);
  bool hu = i <= L.uhi(), hv = j < L.m2;
  T nc, nm, np, nu, nv;
  if constexpr (std::is_same<Form, FullForm>::value) {
    // rho(c) of the cell and its neighbours, shared by the five rows
    const int W = L.pitch;
    const T* rc = L.rhoc;
    T rk = rc[k];
    const T rq[4] = {rc[k + 1], rc[k - 1], rc[k + W], rc[k - W]};
    nc = op_c(P, L, k, rk);
    nm = op_mu(P, L, k, rk, rq);
    np = op_p(P, L, k);
    nu = op_u(P, L, k, T(0.5) * (rk + rq[0]));  // also on boundary edges (padded arrays); masked below
    nv = op_v(P, L, k, T(0.5) * (rk + rq[2]));  // also on boundary edges (padded arrays); masked below
  } else if constexpr (std::is_same<Form, ProjForm>::value) {
    const int W = L.pitch;
    const T* rc = L.rhoc;
    T rk = rc[k];
    const T rq[4] = {rc[k + 1], rc[k - 1], rc[k + W], rc[k - W]};
    T w[4];
    proj_faces(P, L, i, j, rk, rq, w);
    nc = opp_c_w(P, L, k, rq, w);
    nm = op_mu_r(P, L, k, rk, rq, L.rhon[k]);
    np = opp_p_w(P, L, k, w);
    nu = op_u<T, false>(P, L, k, T(0.5) * (rk + rq[0]));  // also on boundary edges (padded arrays); masked below
    nv = op_v<T, false>(P, L, k, T(0.5) * (rk + rq[2]));  // also on boundary edges (padded arrays); masked below
  } else {
    nc = Form::Nc(P, L, k);
    nm = Form::Nmu(P, L, k);
    np = Form::Np(P, L, k);
    nu = Form::Nu(P, L, k);  // also on boundary edges (padded arrays); masked below
    nv = Form::Nv(P, L, k);  // also on boundary edges (padded arrays); masked below
  }
  if (MODE == 0) {
    T r[5] = {L.fc[k] - nc, L.fmu[k] - nm, L.fp[k] - np, hu ? L.fu[k] - nu : T(0),
              hv ? L.fv[k] - nv : T(0)};
    L.rc[k] = r[0];
    L.rmu[k] = r[1];
    L.rp[k] = r[2];
    if (hu) L.ru[k] = r[3];
    if (hv) L.rv[k] = r[4];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      double a = (double)r[q];
      val[q] = fabs(a);
      val[5 + q] = a * a;
    }
  } else {
    L.fc[k] += nc;
    L.fmu[k] += nm;
    L.fp[k] += np;
    if (hu) L.fu[k] += nu;
    if (hv) L.fv[k] += nv;
  }
}

// ROWS = 2 (large levels): each thread takes rows j and j + BY of a block of
// 2 BY rows, so that a 256x512 grid fits the GPU in one round of blocks and
// the norms' reduction is shared by two cells.
template <typename T, int MODE, class Form, int ROWS>
__global__ void k_residual(Prm<T> P, Lv<T> L, double* part) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x + 1;
  int j = blockIdx.y * (ROWS * BY) + threadIdx.y + 1;
  double val[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // max x5 then sum of squares x5
  if (i <= L.m1 && j <= L.m2) residual_cell<T, MODE, Form>(P, L, i, j, val);
  if (ROWS == 2 && i <= L.m1 && j + BY <= L.m2) {
    double v2[10];
    residual_cell<T, MODE, Form>(P, L, i, j + BY, v2);
    if (MODE == 0) {
#pragma unroll
      for (int q = 0; q < 5; ++q) {  // |r| >= 0 or NaN: the bit patterns order as the values
        long long a = __double_as_longlong(val[q]), b = __double_as_longlong(v2[q]);
        val[q] = __longlong_as_double(a > b ? a : b);
        val[5 + q] += v2[5 + q];
      }
    }
  }
  if (MODE == 0 && part) block_sum_store<10>(val, part, 5);
}

// rows per residual thread on level L: two on levels of at least 65536 cells
template <typename T>
static int residual_rows(const Lv<T>& L) {
  return (long long)L.m1 * L.m2 >= 65536 ? 2 : 1;
}

// --------------------------------------------------------------------------
// CH step 1 of Sec. 7.1: Newton step on the 2x2 system (N_c, N_mu) in (c, mu)
// of each cell with (i + j) % 2 == colour; neighbours frozen.  Faces on
// Neumann walls do not contribute (their ghost follows the cell).
// --------------------------------------------------------------------------
// The 2x2 CH system of cell (i,j): residuals R = N - f of (N_c, N_mu) and their
// Jacobian J in (c, mu), neighbours frozen, at the full values c, mu
template <typename T, class Form>
__device__ __forceinline__ void ch_system(const Prm<T>& P, const Lv<T>& L, int i, int j,
                                          T (&J)[2][2], T (&R)[2]) {
  const int W = L.pitch;
  int k = L.at(i, j);
  const int off[4] = {1, -1, W, -W};
  // rho(c) of the cell and its four neighbours, shared by N_c, N_mu and J
  T rho, rq4[4];
  rho = Form::rho(P, L, k);
#pragma unroll
  for (int f = 0; f < 4; ++f) rq4[f] = Form::rho(P, L, k + off[f]);
  T Rc, Rm;
  T wf[4];  // projection method: the face velocities u^{n+1} (E, W, N, S)
  if constexpr (std::is_same<Form, FullForm>::value) {
    Rc = op_c(P, L, k, rho) - L.fc[k];
    Rm = op_mu(P, L, k, rho, rq4) - L.fmu[k];
  } else if constexpr (std::is_same<Form, ProjForm>::value) {
    proj_faces(P, L, i, j, rho, rq4, wf);
    Rc = opp_c_w(P, L, k, rq4, wf) - L.fc[k];
    Rm = op_mu_r(P, L, k, rho, rq4, L.rhon[k]) - L.fmu[k];
  } else {
    Rc = Form::Nc(P, L, k) - L.fc[k];
    Rm = Form::Nmu(P, L, k) - L.fmu[k];
  }
  const T *cn = L.cn, *rn = L.rhon, *mob = L.mobn;
  // full values c, mu at which the local Jacobian is evaluated
  T ck = Form::val_c(L, k), cnk = cn[k], mk = Form::val_mu(L, k);
  T drho = -P.alpha * rho * rho;
  T rnk = rn[k];
  T rh = T(0.5) * (rho + rnk);
  T chk = ck + cnk;  // 2 c^{n+1/2}
  T r = -P.alpha * rho * rnk, dr = -P.alpha * drho * rnk;
  bool wall[4] = {!L.px && i == L.m1, !L.px && i == 1, j == L.m2, j == 1};
  T sm = 0, dG = 0, dd = 0, G2 = 0;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    int q = k + off[f];
    T cq = Form::val_c(L, q);
    T d = cq - ck;
    G2 += d * d;
    if (wall[f]) continue;
    sm += mob[k] + mob[q];
    dG -= d;
    T rq = T(0.5) * (rq4[f] + rn[q]);
    dd += T(0.5) * drho * ((cq + cn[q]) - chk) - (rh + rq);
  }
  // sm = 2 sum A m; dG = h^2 dG/dc; dd = 4 h^2 d(div)/dc; G2 = 2 h^2 G(c)
  T J11 = (rho + drho * (ck - cnk)) * P.idt;
  T J12 = T(0.5) * sm * P.iPe * L.ih2;
  T Gs = T(0.5) * G2 * L.ih2 + L.Gn[k];
  T dbulk = T(0.5) * drho * gsec(ck, cnk) + rh * gsec_da(ck, cnk) + T(0.5) * fdw(ck) * r +
            T(0.5) * (Fdw(ck) + Fdw(cnk)) * dr;
  T dgrad = T(0.25) * P.Lam * (dG * L.ih2 * r + Gs * dr);
  T J21 = drho * mk - P.K * dbulk - dgrad + P.Lam * T(0.25) * L.ih2 * dd;
  T J22 = rho;
  if constexpr (std::is_same<Form, ProjForm>::value) {
    // projection method: rho^n in the time derivative and in front of mu; the
    // advection a(rho(c) D c u^{n+1}) differentiated in c_ij through D c only,
    // with rho(c) of the neighbours and u^{n+1} at the iterate (the smoother's
    // choice; the fixed point is the scheme's)
    J11 = rnk * P.idt + T(0.5) * (-rq4[0] * wf[0] + rq4[1] * wf[1]) * L.ih +
          T(0.5) * (-rq4[2] * wf[2] + rq4[3] * wf[3]) * L.ih;
    J21 = -P.K * dbulk - dgrad + P.Lam * T(0.25) * L.ih2 * dd;
    J22 = rnk;
  }
  J[0][0] = J11;
  J[0][1] = J12;
  J[1][0] = J21;
  J[1][1] = J22;
  R[0] = Rc;
  R[1] = Rm;
}

template <typename T, class Form>
__device__ __forceinline__ void ch_cell(const Prm<T>& P, const Lv<T>& L, int i, int j) {
  T J[2][2], R[2];
  ch_system<T, Form>(P, L, i, j, J, R);
  T idet = qrcp(J[0][0] * J[1][1] - J[0][1] * J[1][0]);
  T dc = (J[1][1] * R[0] - J[0][1] * R[1]) * idet;
  T dm = (J[0][0] * R[1] - J[1][0] * R[0]) * idet;
  int k = L.at(i, j);
  T cnew = L.c[k] - dc;
  store_cell(L, L.c, i, j, cnew);
  if constexpr (!std::is_same<Form, ErrForm>::value) store_cell(L, L.rhoc, i, j, rho_of(P, cnew));
  store_cell(L, L.mu, i, j, L.mu[k] - dm);
}

// cells of CH colour `colour` ((i + j) % 2), packed: slot t -> row t / mpr + 1
template <typename T, class Form>
__global__ void __launch_bounds__(64) k_ch(Prm<T> P, Lv<T> L, int colour) {
  pdl_enter();
  int mpr = (L.m1 + 1) / 2;
  int t = blockIdx.x * 64 + threadIdx.x;
  if (t >= mpr * L.m2) return;
  int j = t / mpr + 1;
  int i = (((colour - j) & 1) ? 1 : 2) + 2 * (t % mpr);
  if (i > L.m1) return;
  ch_cell<T, Form>(P, L, i, j);
}

// sum over the four lanes of a team (lanes 4t .. 4t+3)
template <typename T>
__device__ __forceinline__ T team_sum(T v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v + __shfl_xor_sync(0xffffffffu, v, 2);
}

// u^{n+1} at face q (W, E, S, N) of cell k (0 on a wall face), as proj_faces
// gives it: rho(c) of the cell rk and of the face's neighbour rn
template <typename T>
__device__ __forceinline__ T proj_face_team(const Prm<T>& P, const Lv<T>& L, int k, int q, bool open, T rk,
                                            T rn) {
  const int d = q >> 1, off = d ? L.pitch : 1;
  const bool hi = q & 1;  // E or N: the face's velocity sits at k
  const int a = hi ? k : k - off;
  const T *vel = d ? L.v : L.u, *c = L.c, *mu = L.mu, *p = L.p;
  T ra = hi ? rk : rn, rb = hi ? rn : rk;
  T Ar = T(0.5) * (ra + rb);
  T dp = (p[a + off] - p[a]) * L.ih;
  T st = T(0.5) * (rb * mu[a] + ra * mu[a + off]) * (c[a + off] - c[a]) * L.ih;
  T grav = d ? P.Fr_inv / P.idt : T(0);
  return open ? vel[a] + (st - dp) * P.iM / (Ar * P.idt) - grav : T(0);
}

// The CH rows of cell (i,j) for a team of four lanes (lane & 3 = q: face W,
// E, S, N; open = face q is not a wall): residuals Rc = N_c - f_c,
// Rm = N_mu - f_mu and the 2x2 Jacobian of ch_system, and for the coupled
// block the open-face sum of A m, the diffusion flux sum, d rho/dc and face
// q's rho^n D c^n / 2.  Lane q evaluates face q's terms of N_c, N_mu (op_c and
// op_mu, or opd_c and opd_mu on error levels) and of the Jacobian's face
// sums; butterflies add them and every lane forms the cell terms.
template <typename T>
struct ChRows {
  T Rc, Rm, J11, J12, J21, J22;
  T sm, sflux, drho, gq;
};

template <typename T, class Form>
__device__ __forceinline__ ChRows<T> ch_team_rows(const Prm<T>& P, const Lv<T>& L, int i, int j, int q,
                                                  bool open) {
  const int W = L.pitch;
  const int d = q >> 1;
  const T ih2 = L.ih2;
  int k = L.at(i, j);
  const T *mob = L.mobn, *cn = L.cn, *rn = L.rhon;
  const int nq = k + (q == 0 ? -1 : q == 1 ? 1 : q == 2 ? -W : W);
  const int kf = q == 0 ? k - 1 : (q == 2 ? k - W : k);  // edge of face q
  // full values at the cell and at the face's neighbour
  T ck = Form::val_c(L, k), cnk = cn[k], mk = Form::val_mu(L, k), rnk = rn[k];
  T rho = Form::rho(P, L, k);
  T cq = Form::val_c(L, nq), rq = Form::rho(P, L, nq);
  T drho = -P.alpha * rho * rho;
  T rh = T(0.5) * (rho + rnk);
  T chk = ck + cnk;
  T am = mob[nq] + mob[k];
  T gq = rn[nq] * (d ? L.Ty[kf] : L.Tx[kf]);  // rho^n D c^n / 2 at face q
  T dlt = cq - ck;
  // face sums: diffusion flux (N_c and the mass row), sum A m over open faces,
  // advection of N_c, and the Jacobian's G, dG/dc and d(div)/dc terms
  T sflux = team_sum<T>(T(0.5) * am * ((L.mu[nq] - L.mu[k]) + P.alpha * (L.p[nq] - L.p[k])));
  T sm = team_sum<T>(open ? am : T(0));
  T sadv = team_sum<T>(gq * (d ? L.v[kf] : L.u[kf]));
  T G2 = team_sum<T>(dlt * dlt);
  T dG = team_sum<T>(open ? -dlt : T(0));
  T dd = team_sum<T>(open ? T(0.5) * drho * ((cq + cn[nq]) - chk) - (rh + T(0.5) * (rq + rn[nq])) : T(0));
  T Nc, Nm;
  T wq = T(0), sJ11 = T(0);  // projection method: u^{n+1} at face q, its advection Jacobian
  if constexpr (std::is_same<Form, ProjForm>::value) {
    wq = proj_face_team(P, L, k, q, open, rho, rq);
    // advection a(rho(c) D c u^{n+1}) of (pj-num-phase) by faces
    T sadvp = team_sum<T>(T(0.5) * rq * ((q & 1) ? (cq - ck) : (ck - cq)) * L.ih * wq);
    Nc = rnk * (ck - cnk) * P.idt + sadvp - P.iPe * ih2 * sflux;
    T sdv = team_sum<T>((rh + T(0.5) * (rq + rn[nq])) * ((cq + cn[nq]) - chk));
    T r = -P.alpha * rho * rnk;
    T bulk = rh * gsec(ck, cnk) + T(0.5) * (Fdw(ck) + Fdw(cnk)) * r;
    T grad = T(0.25) * P.Lam * (T(0.5) * G2 * ih2 + L.Gn[k]) * r;
    Nm = rnk * mk - P.K * bulk - grad + P.Lam * T(0.25) * ih2 * sdv;
    sJ11 = team_sum<T>(T(0.5) * ((q & 1) ? -rq * wq : rq * wq) * L.ih);
  } else if constexpr (std::is_same<Form, ErrForm>::value) {
    const T *e = L.c, *B = L.Bc;
    T ek = e[k], Ck = B[k];
    T rC = rho_of(P, Ck);
    Nc = ek * (rho + rsec_(P, rho, rC) * L.Bdc[k]) * P.idt + sadv - P.iPe * ih2 * sflux;
    T dC = B[nq] - Ck, de = e[nq] - ek;
    T rCq = rho_of(P, B[nq]);
    T dr = rsec_(P, rho, rC) * ek;
    T drq = rsec_(P, rq, rCq) * e[nq];
    T chP = Ck + cnk;
    T sdGe = team_sum<T>(de * (T(2) * dC + de));
    T sGC = team_sum<T>(dC * dC);
    T sddiv = team_sum<T>((rh + T(0.5) * (rq + rn[nq])) * de + T(0.5) * (dr + drq) * ((B[nq] + cn[nq]) - chP));
    T r_new = rsec_(P, rho, rnk);
    T d_r = -P.alpha * rnk * dr;
    T dF = gsec(ck, Ck) * ek;
    T dbulk = rh * dgsec(Ck, cnk, ek) + T(0.5) * dr * gsec(Ck, cnk) + T(0.5) * dF * r_new +
              T(0.5) * (Fdw(Ck) + Fdw(cnk)) * d_r;
    T dgrad = T(0.25) * P.Lam * (T(0.5) * sdGe * ih2 * r_new + (T(0.5) * sGC * ih2 + L.Gn[k]) * d_r);
    Nm = rho * L.mu[k] + dr * L.Bmu[k] - P.K * dbulk - dgrad + P.Lam * T(0.25) * ih2 * sddiv;
  } else {
    Nc = rho * (ck - cnk) * P.idt + sadv - P.iPe * ih2 * sflux;
    T sdv = team_sum<T>((rh + T(0.5) * (rq + rn[nq])) * ((cq + cn[nq]) - chk));
    T r = -P.alpha * rho * rnk;
    T bulk = rh * gsec(ck, cnk) + T(0.5) * (Fdw(ck) + Fdw(cnk)) * r;
    T grad = T(0.25) * P.Lam * (T(0.5) * G2 * ih2 + L.Gn[k]) * r;
    Nm = rho * mk - P.K * bulk - grad + P.Lam * T(0.25) * ih2 * sdv;
  }
  ChRows<T> R;
  R.Rc = Nc - L.fc[k];
  R.Rm = Nm - L.fmu[k];
  T r = -P.alpha * rho * rnk, drr = -P.alpha * drho * rnk;
  R.J11 = (rho + drho * (ck - cnk)) * P.idt;
  R.J12 = T(0.5) * sm * P.iPe * ih2;
  T Gs = T(0.5) * G2 * ih2 + L.Gn[k];
  T dbulkJ = T(0.5) * drho * gsec(ck, cnk) + rh * gsec_da(ck, cnk) + T(0.5) * fdw(ck) * r +
             T(0.5) * (Fdw(ck) + Fdw(cnk)) * drr;
  T dgradJ = T(0.25) * P.Lam * (dG * ih2 * r + Gs * drr);
  R.J21 = drho * mk - P.K * dbulkJ - dgradJ + P.Lam * T(0.25) * ih2 * dd;
  R.J22 = rho;
  if constexpr (std::is_same<Form, ProjForm>::value) {
    // ch_system's projection branch: rho^n in the time derivative and in front
    // of mu; the advection differentiated through D c only
    R.J11 = rnk * P.idt + sJ11;
    R.J21 = -P.K * dbulkJ - dgradJ + P.Lam * T(0.25) * ih2 * dd;
    R.J22 = rnk;
  }
  R.sm = sm;
  R.sflux = sflux;
  R.drho = drho;
  R.gq = gq;
  return R;
}

// CH step of cell (i,j) by a team of four lanes (ch_team_rows), every lane
// solving the 2x2 Newton step; lane 0 stores.  All 32 lanes of the warp call
// this (ok = false: a spare team on cell (1,1), no store).
template <typename T, class Form>
__device__ __forceinline__ void ch_team(const Prm<T>& P, const Lv<T>& L, int i, int j, bool ok) {
  const int q = threadIdx.x & 3;
  const bool open = q == 0 ? (L.px || i > 1) : q == 1 ? (L.px || i < L.m1) : q == 2 ? j > 1 : j < L.m2;
  ChRows<T> R = ch_team_rows<T, Form>(P, L, i, j, q, open);
  T idet = qrcp(R.J11 * R.J22 - R.J12 * R.J21);
  T dc = (R.J22 * R.Rc - R.J12 * R.Rm) * idet;
  T dm = (R.J11 * R.Rm - R.J21 * R.Rc) * idet;
  if (ok && q == 0) {
    int k = L.at(i, j);
    T cnew = L.c[k] - dc;
    store_cell(L, L.c, i, j, cnew);
    if constexpr (!std::is_same<Form, ErrForm>::value) store_cell(L, L.rhoc, i, j, rho_of(P, cnew));
    store_cell(L, L.mu, i, j, L.mu[k] - dm);
  }
}

// per-level CH launch with four lanes per cell (colour (i + j) % 2, packed)
template <typename T, class Form>
__global__ void __launch_bounds__(64) k_ch_team(Prm<T> P, Lv<T> L, int colour) {
  pdl_enter();
  int mpr = (L.m1 + 1) / 2;
  int n = mpr * L.m2;
  int t = blockIdx.x * 64 + threadIdx.x;
  if ((t & ~31) >= 4 * n) return;  // warp-uniform
  int s = t >> 2;
  int j = 1, i = 1;
  bool ok = false;
  if (s < n) {
    j = s / mpr + 1;
    i = (((colour - j) & 1) ? 1 : 2) + 2 * (s % mpr);
    ok = i <= L.m1;
  }
  if (!ok) i = j = 1;
  ch_team<T, Form>(P, L, i, j, ok);
}

// --------------------------------------------------------------------------
// Vanka step 2 of Sec. 7.1: exact solve of the 5x5 block of cell (i,j):
// unknowns (u_W, u_E, v_S, v_N, p), equations (N_u W, N_u E, N_v S, N_v N, N_p).
// Colours: (i + 2j) % 5 (walls in x) or (2i + j) % 8 (periodic x).
// --------------------------------------------------------------------------
// The 5x5 Vanka system of cell (i,j): A = Jacobian of (N_u W, N_u E, N_v S,
// N_v N, N_p) in (u_W, u_E, v_S, v_N, p), b = residuals N - f; rows and
// columns of wall edges (act = false) replaced by the identity
template <typename T, class Form>
__device__ __forceinline__ void vanka_system(const Prm<T>& P, const Lv<T>& L, int i, int j,
                                             T (&A)[5][5], T (&b)[5], bool (&act)[5]) {
  const int W = L.pitch;
  const T ih = L.ih, ih2 = L.ih2;
  const T* vis = L.visn;
  int k = L.at(i, j);
  int eW = (L.px && i == 1) ? L.m1 : i - 1;
  int kW = L.at(eW, j);
  act[0] = L.px || i > 1;
  act[1] = L.px || i < L.m1;
  act[2] = j > 1;
  act[3] = j < L.m2;
  act[4] = true;
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c < 5; ++c) A[r][c] = T(0);
  const T third = T(1.0 / 3.0);
  // density averages on the four edges from rho(c) of the cell and its four
  // neighbours (c at kW + 1 is c at k, exactly: ghosts are copies)
  T Arq[4];
  {
    T rk = Form::rho(P, L, k);
    Arq[0] = T(0.5) * (Form::rho(P, L, kW) + rk);
    Arq[1] = T(0.5) * (rk + Form::rho(P, L, k + 1));
    Arq[2] = T(0.5) * (Form::rho(P, L, k - W) + rk);
    Arq[3] = T(0.5) * (rk + Form::rho(P, L, k + W));
  }
  // x-edge rows: q = 0 (west edge, index kW), q = 1 (east edge, index k)
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    int ke = q == 0 ? kW : k;
    T Arn = L.Aru[ke];
    T Ar = Arq[q];
    T gt = (j == L.m2) ? T(2) : T(1), gb = (j == 1) ? T(2) : T(1);
    if constexpr (!std::is_same<Form, ErrForm>::value) {  // per-step coefficients
      A[q][q] = L.Dgu[ke] + T(0.5) * P.idt * Ar;
      continue;
    }
    A[q][q] = Arn * P.idt + T(0.5) * (Ar - Arn) * P.idt +
              T(0.5) * ih * (-L.Sx[ke + 1] + L.Sx[ke] - L.Qx[ke] * gt + L.Qx[ke - W] * gb) +
              L.Dvu[ke] +
              P.iRe * ih2 * ((vis[ke + 1] + vis[ke]) * (T(1) + third) + gt * L.Av[ke] +
                             gb * L.Av[ke - W]);
  }
  {
    T vc = vis[k];
    T v3 = vc * P.iRe * ih2 * third;
    A[0][1] = T(0.5) * L.Sx[k] * ih - vc * P.iRe * ih2 - v3;
    A[1][0] = -T(0.5) * L.Sx[k] * ih - vc * P.iRe * ih2 - v3;
    A[0][2] = v3;
    A[0][3] = -v3;
    A[1][2] = -v3;
    A[1][3] = v3;
    A[0][4] = ih * P.iM;
    A[1][4] = -ih * P.iM;
  }
  // y-edge rows: q = 2 (south edge, index k - W), q = 3 (north edge, index k)
#pragma unroll
  for (int q = 2; q < 4; ++q) {
    int ke = q == 2 ? k - W : k;
    T Arn = L.Arv[ke];
    T Ar = Arq[q];
    T ge = (!L.px && i == L.m1) ? T(2) : T(1), gw = (!L.px && i == 1) ? T(2) : T(1);
    if constexpr (!std::is_same<Form, ErrForm>::value) {  // per-step coefficients
      A[q][q] = L.Dgv[ke] + T(0.5) * P.idt * Ar;
      continue;
    }
    A[q][q] = Arn * P.idt + T(0.5) * (Ar - Arn) * P.idt +
              T(0.5) * ih * (-L.Qy[ke] * ge + L.Qy[ke - 1] * gw - L.Sy[ke + W] + L.Sy[ke]) +
              L.Dvv[ke] +
              P.iRe * ih2 * (ge * L.Av[ke] + gw * L.Av[ke - 1] +
                             (vis[ke + W] + vis[ke]) * (T(1) + third));
  }
  {
    T vc = vis[k];
    T v3 = vc * P.iRe * ih2 * third;
    A[2][3] = T(0.5) * L.Sy[k] * ih - vc * P.iRe * ih2 - v3;
    A[3][2] = -T(0.5) * L.Sy[k] * ih - vc * P.iRe * ih2 - v3;
    A[2][0] = v3;
    A[2][1] = -v3;
    A[3][0] = -v3;
    A[3][1] = v3;
    A[2][4] = ih * P.iM;
    A[3][4] = -ih * P.iM;
  }
  {
    const T* mob = L.mobn;
    bool wall[4] = {!L.px && i == L.m1, !L.px && i == 1, j == L.m2, j == 1};
    const int off[4] = {1, -1, W, -W};
    T sm = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f)
      if (!wall[f]) sm += mob[k] + mob[k + off[f]];
    A[4][0] = -ih;
    A[4][1] = ih;
    A[4][2] = -ih;
    A[4][3] = ih;
    A[4][4] = T(0.5) * P.alpha * P.alpha * P.iPe * sm * ih2;
  }
  if constexpr (std::is_same<Form, FullForm>::value) {
    {
      T nq = op_u(P, L, kW, Arq[0]);  // evaluated on wall edges too (padded arrays), then discarded
      b[0] = act[0] ? nq - L.fu[kW] : T(0);
    }
    {
      T nq = op_u(P, L, k, Arq[1]);  // evaluated on wall edges too (padded arrays), then discarded
      b[1] = act[1] ? nq - L.fu[k] : T(0);
    }
    {
      T nq = op_v(P, L, k - W, Arq[2]);  // evaluated on wall edges too (padded arrays), then discarded
      b[2] = act[2] ? nq - L.fv[k - W] : T(0);
    }
    {
      T nq = op_v(P, L, k, Arq[3]);  // evaluated on wall edges too (padded arrays), then discarded
      b[3] = act[3] ? nq - L.fv[k] : T(0);
    }
  } else if constexpr (std::is_same<Form, ProjForm>::value) {
    {
      T nq = op_u<T, false>(P, L, kW, Arq[0]);  // evaluated on wall edges too (padded arrays), then discarded
      b[0] = act[0] ? nq - L.fu[kW] : T(0);
    }
    {
      T nq = op_u<T, false>(P, L, k, Arq[1]);  // evaluated on wall edges too (padded arrays), then discarded
      b[1] = act[1] ? nq - L.fu[k] : T(0);
    }
    {
      T nq = op_v<T, false>(P, L, k - W, Arq[2]);  // evaluated on wall edges too (padded arrays), then discarded
      b[2] = act[2] ? nq - L.fv[k - W] : T(0);
    }
    {
      T nq = op_v<T, false>(P, L, k, Arq[3]);  // evaluated on wall edges too (padded arrays), then discarded
      b[3] = act[3] ? nq - L.fv[k] : T(0);
    }
  } else {
    {
      T nq = Form::Nu(P, L, kW);  // evaluated on wall edges too (padded arrays), then discarded
      b[0] = act[0] ? nq - L.fu[kW] : T(0);
    }
    {
      T nq = Form::Nu(P, L, k);  // evaluated on wall edges too (padded arrays), then discarded
      b[1] = act[1] ? nq - L.fu[k] : T(0);
    }
    {
      T nq = Form::Nv(P, L, k - W);  // evaluated on wall edges too (padded arrays), then discarded
      b[2] = act[2] ? nq - L.fv[k - W] : T(0);
    }
    {
      T nq = Form::Nv(P, L, k);  // evaluated on wall edges too (padded arrays), then discarded
      b[3] = act[3] ? nq - L.fv[k] : T(0);
    }
  }
  if constexpr (std::is_same<Form, ProjForm>::value) b[4] = T(0);  // the 4x4 block has no p row
  else b[4] = Form::Np(P, L, k) - L.fp[k];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (!act[q]) {
#pragma unroll
      for (int c = 0; c < 5; ++c) { A[q][c] = T(0); A[c][q] = T(0); }
      A[q][q] = T(1);
    }
}

// Exact solve of the Vanka system A d = b by its structure.  The velocity block
// is A_vv = B + v3 w w^T: every coupling between an x-edge and a y-edge of the
// cell is +-v3 (the grad-div term), w = (1, -1, 1, -1) on active edges and 0 on
// wall edges, and B is block-diagonal (the x pair and the y pair).  The
// pressure column is a w (a = 1/(M h)) and the pressure row -w/h.  With
// y = B^-1 b_v, z = B^-1 w, s = w.z, t = w.y, g = 1/(1 + v3 s)
// (Sherman-Morrison), p = (b_p + t g/h)/(A_pp + a s g/h) and
// d_v = y - z g (v3 t + a p): two 2x2 solves and three divisions in place of
// 5x5 elimination.  B is diagonally dominant and s, g > 0, so no pivoting.
// NP = 5 solves the full system, NP = 4 the velocity block alone.
template <typename T, int NP>
__device__ __forceinline__ void solve_vanka(const T (&A)[5][5], T (&b)[5], const bool (&act)[5],
                                            T v3, T a, T ih) {
  // w_q is +1, -1 or 0, so the products with w are selections
  T y[4], z[4];
#pragma unroll
  for (int blk = 0; blk < 4; blk += 2) {
    const int p0 = blk, p1 = blk + 1;
    const bool a0 = act[p0], a1 = act[p1];
    // B = A_vv - v3 w w^T on this pair: w_p0 w_p0 = a0, w_p1 w_p1 = a1, w_p0 w_p1 = -(a0 a1)
    T B00 = a0 ? A[p0][p0] - v3 : A[p0][p0];
    T B11 = a1 ? A[p1][p1] - v3 : A[p1][p1];
    T B01 = (a0 && a1) ? A[p0][p1] + v3 : A[p0][p1];
    T B10 = (a0 && a1) ? A[p1][p0] + v3 : A[p1][p0];
    T idet = qrcp(B00 * B11 - B01 * B10);
    y[p0] = (B11 * b[p0] - B01 * b[p1]) * idet;
    y[p1] = (B00 * b[p1] - B10 * b[p0]) * idet;
    // z = B^-1 w with w_p0 = a0 ? 1 : 0, w_p1 = a1 ? -1 : 0
    T zn0 = (a0 ? B11 : T(0)) + (a1 ? B01 : T(0));
    T zn1 = -((a1 ? B00 : T(0)) + (a0 ? B10 : T(0)));
    z[p0] = zn0 * idet;
    z[p1] = zn1 * idet;
  }
  // inactive entries of y and z are 0 (identity rows, b = 0, w = 0)
  T sdot = (z[0] - z[1]) + (z[2] - z[3]);
  T tdot = (y[0] - y[1]) + (y[2] - y[3]);
  T g = qrcp(T(1) + v3 * sdot);
  T pr = T(0);
  if constexpr (NP == 5) pr = (b[4] + ih * tdot * g) * qrcp(A[4][4] + ih * a * sdot * g);
  T f = g * (v3 * tdot + a * pr);
#pragma unroll
  for (int q = 0; q < 4; ++q) b[q] = y[q] - z[q] * f;
  if constexpr (NP == 5) b[4] = pr;
}

template <typename T, class Form>
__device__ __forceinline__ void vanka_cell(const Prm<T>& P, const Lv<T>& L, int i, int j, T omega) {
  T A[5][5], b[5];
  bool act[5];
  vanka_system<T, Form>(P, L, i, j, A, b, act);
  const int W = L.pitch;
  int k = L.at(i, j);
  solve_vanka<T, 5>(A, b, act, L.visn[k] * P.iRe * L.ih2 * T(1.0 / 3.0), L.ih * P.iM, L.ih);
  int eW = (L.px && i == 1) ? L.m1 : i - 1;
  int kW = L.at(eW, j);
  if (act[0]) store_u(L, eW, j, L.u[kW] - omega * b[0]);
  if (act[1]) store_u(L, i, j, L.u[k] - omega * b[1]);
  if (act[2]) store_v(L, i, j - 1, L.v[k - W] - omega * b[2]);
  if (act[3]) store_v(L, i, j, L.v[k] - omega * b[3]);
  store_cell(L, L.p, i, j, L.p[k] - omega * b[4]);
}

// Exact solve of the coupled 7x7 system of coupled_cell by blocks.  Its NS part
// A[2..6][2..6] is a Vanka block (see solve_vanka): it is factored once and
// applied to three right-hand sides, b_NS and the two columns through which c
// and mu enter the NS rows.  What remains for (dc, dmu) is the 2x2 Schur
// complement S = J_CH - C (A_NS^-1 C'), solved directly; the NS unknowns follow
// by back substitution.  Row 1 (N_mu) does not involve u, v or p, so its
// coupling entries are zero and its Schur row is that of J_CH.
template <typename T>
__device__ __forceinline__ void solve_coupled7(const T (&A)[7][7], T (&b)[7], const bool (&act)[5],
                                               T v3, T a, T ih) {
  T B00[2], B01[2], B10[2], B11[2], idet[2], z[4];
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    const int p0 = 2 * blk, p1 = p0 + 1;
    const bool a0 = act[p0], a1 = act[p1];
    B00[blk] = a0 ? A[2 + p0][2 + p0] - v3 : A[2 + p0][2 + p0];
    B11[blk] = a1 ? A[2 + p1][2 + p1] - v3 : A[2 + p1][2 + p1];
    B01[blk] = (a0 && a1) ? A[2 + p0][2 + p1] + v3 : A[2 + p0][2 + p1];
    B10[blk] = (a0 && a1) ? A[2 + p1][2 + p0] + v3 : A[2 + p1][2 + p0];
    idet[blk] = qrcp(B00[blk] * B11[blk] - B01[blk] * B10[blk]);
    z[p0] = ((a0 ? B11[blk] : T(0)) + (a1 ? B01[blk] : T(0))) * idet[blk];
    z[p1] = -((a1 ? B00[blk] : T(0)) + (a0 ? B10[blk] : T(0))) * idet[blk];
  }
  const T sdot = (z[0] - z[1]) + (z[2] - z[3]);
  const T g = qrcp(T(1) + v3 * sdot);
  const T iden = qrcp(A[6][6] + ih * a * sdot * g);
  // x = A_NS^-1 r for a right-hand side r over (u_W, u_E, v_S, v_N, p)
  auto apply = [&](const T (&r)[5], T (&x)[5]) {
    T y[4];
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
      const int p0 = 2 * blk, p1 = p0 + 1;
      y[p0] = (B11[blk] * r[p0] - B01[blk] * r[p1]) * idet[blk];
      y[p1] = (B00[blk] * r[p1] - B10[blk] * r[p0]) * idet[blk];
    }
    T t = (y[0] - y[1]) + (y[2] - y[3]);
    T pr = (r[4] + ih * t * g) * iden;
    T f = g * (v3 * t + a * pr);
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = y[q] - z[q] * f;
    x[4] = pr;
  };
  T r0[5], r1[5], r2[5], X0[5], X1[5], X2[5];
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    r0[m] = b[2 + m];
    r1[m] = A[2 + m][0];
    r2[m] = A[2 + m][1];
  }
  apply(r0, X0);
  apply(r1, X1);
  apply(r2, X2);
  T S00 = A[0][0], S01 = A[0][1], rhs0 = b[0];
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    S00 -= A[0][2 + m] * X1[m];
    S01 -= A[0][2 + m] * X2[m];
    rhs0 -= A[0][2 + m] * X0[m];
  }
  const T S10 = A[1][0], S11 = A[1][1], rhs1 = b[1];
  T id2 = qrcp(S00 * S11 - S01 * S10);
  T dc = (S11 * rhs0 - S01 * rhs1) * id2;
  T dm = (S00 * rhs1 - S10 * rhs0) * id2;
  b[0] = dc;
  b[1] = dm;
#pragma unroll
  for (int m = 0; m < 5; ++m) b[2 + m] = X0[m] - X1[m] * dc - X2[m] * dm;
}

// Coupled block (an option; the paper's smoother keeps the two blocks
// separate): one Newton step on the 7x7 system of (N_c, N_mu, N_u W, N_u E,
// N_v S, N_v N, N_p) in (c, mu, u_W, u_E, v_S, v_N, p).  It adds to the 2x2 CH
// and 5x5 Vanka blocks the couplings the separate smoothers treat explicitly:
// the CH advection (e1e2) and (alpha/Pe) grad.(A m grad p) in N_c, the
// (alpha/Pe) grad.(A m grad mu) term of N_p, and the rho(c) and surface-tension
// (e1e1) terms of the momentum rows.
template <typename T, class Form>
__device__ __forceinline__ void coupled_cell(const Prm<T>& P, const Lv<T>& L, int i, int j, T omega) {
  T A5[5][5], b5[5], J2[2][2], R2[2];
  bool act[5];
  vanka_system<T, Form>(P, L, i, j, A5, b5, act);
  ch_system<T, Form>(P, L, i, j, J2, R2);
  T A[7][7], b[7];
#pragma unroll
  for (int r = 0; r < 7; ++r)
#pragma unroll
    for (int c = 0; c < 7; ++c) A[r][c] = T(0);
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    b[2 + r] = b5[r];
#pragma unroll
    for (int c = 0; c < 5; ++c) A[2 + r][2 + c] = A5[r][c];
  }
  A[0][0] = J2[0][0];
  A[0][1] = J2[0][1];
  A[1][0] = J2[1][0];
  A[1][1] = J2[1][1];
  b[0] = R2[0];
  b[1] = R2[1];
  const int W = L.pitch;
  int k = L.at(i, j);
  int eW = (L.px && i == 1) ? L.m1 : i - 1;
  int kW = L.at(eW, j);
  const T *rn = L.rhon, *mob = L.mobn;
  bool wall[4] = {!L.px && i == L.m1, !L.px && i == 1, j == L.m2, j == 1};
  const int off[4] = {1, -1, W, -W};
  T sm = T(0);
#pragma unroll
  for (int f = 0; f < 4; ++f)
    if (!wall[f]) sm += mob[k] + mob[k + off[f]];
  T rho = Form::rho(P, L, k), drho = -P.alpha * rho * rho;
  // rho^n D c^n / 2 at the four faces of the cell, as in (e1e2) and (e1e1)
  T gW = rn[k - 1] * L.Tx[k - 1];
  T gE = rn[k + 1] * L.Tx[k];
  T gS = rn[k - W] * L.Ty[k - W];
  T gN = rn[k + W] * L.Ty[k];
  T diffc = T(0.5) * P.alpha * P.iPe * sm * L.ih2;
  A[0][2] = gW;
  A[0][3] = gE;
  A[0][4] = gS;
  A[0][5] = gN;
  A[0][6] = diffc;
  T half_idt = T(0.25) * drho * P.idt;  // d/dc of (A rho(c) - A rho^n) x / (2 dt), per edge
  A[2][0] = half_idt * Form::val_u(L, kW);
  A[3][0] = half_idt * Form::val_u(L, k);
  A[4][0] = half_idt * Form::val_v(L, k - W);
  A[5][0] = half_idt * Form::val_v(L, k);
  A[2][1] = -gW * P.iM;
  A[3][1] = -gE * P.iM;
  A[4][1] = -gS * P.iM;
  A[5][1] = -gN * P.iM;
  A[6][1] = diffc;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (!act[q]) {
#pragma unroll
      for (int c = 0; c < 7; ++c) {
        A[2 + q][c] = T(0);
        A[c][2 + q] = T(0);
      }
      A[2 + q][2 + q] = T(1);
    }
  solve_coupled7(A, b, act, L.visn[k] * P.iRe * L.ih2 * T(1.0 / 3.0), L.ih * P.iM, L.ih);
  T cnew = L.c[k] - omega * b[0];
  store_cell(L, L.c, i, j, cnew);
  if constexpr (!std::is_same<Form, ErrForm>::value) store_cell(L, L.rhoc, i, j, rho_of(P, cnew));
  store_cell(L, L.mu, i, j, L.mu[k] - omega * b[1]);
  if (act[0]) store_u(L, eW, j, L.u[kW] - omega * b[2]);
  if (act[1]) store_u(L, i, j, L.u[k] - omega * b[3]);
  if (act[2]) store_v(L, i, j - 1, L.v[k - W] - omega * b[4]);
  if (act[3]) store_v(L, i, j, L.v[k] - omega * b[5]);
  store_cell(L, L.p, i, j, L.p[k] - omega * b[6]);
}

// Vanka colour of cell (i,j): (2i + j) mod 8 (periodic x, m1 = 0 mod 4) or
// (i + 2j) mod kcol (kcol = 5 with walls, the smallest divisor >= 5 of m1 otherwise)
template <typename T>
__device__ __forceinline__ int vanka_colour(const Lv<T>& L, int i, int j) {
  return L.c8 ? (2 * i + j) & 7 : (i + 2 * j) % L.kcol;
}

// first cell i0 >= 1 of colour `colour` in row j and the stride between cells
// of that colour in the row; false if the row has none
template <typename T>
__device__ __forceinline__ bool colour_row(const Lv<T>& L, int colour, int j, int& i0, int& stride) {
  if (L.c8) {
    int d = (colour - j) & 7;
    if (d & 1) return false;
    i0 = d >> 1;
    if (i0 == 0) i0 = 4;
    stride = 4;
  } else {
    int K = L.kcol;
    i0 = ((colour - 2 * j) % K + K) % K;
    if (i0 == 0) i0 = K;
    stride = K;
  }
  return true;
}

// slots of Vanka colour `col`: slot t -> row j0 + rstep * (t / mpr), t % mpr-th
// cell of that row's colour
struct ColourSlots {
  int j0, rstep, mpr, n;
};

template <typename T>
__host__ __device__ __forceinline__ ColourSlots vanka_slots(const Lv<T>& L, int col) {
  ColourSlots cs;
  if (L.c8) {
    cs.j0 = ((col - 1) & 1) ? 2 : 1;  // rows with (col - j) even
    cs.rstep = 2;
    cs.mpr = (L.m1 + 3) / 4;
  } else {
    cs.j0 = 1;
    cs.rstep = 1;
    cs.mpr = (L.m1 + L.kcol - 1) / L.kcol;
  }
  cs.n = cs.j0 > L.m2 ? 0 : ((L.m2 - cs.j0) / cs.rstep + 1) * cs.mpr;
  return cs;
}

template <typename T>
__device__ __forceinline__ bool vanka_slot_cell(const Lv<T>& L, int col, const ColourSlots& cs, int t,
                                                int& i, int& j) {
  j = cs.j0 + cs.rstep * (t / cs.mpr);
  int i0, stride;
  if (!colour_row(L, col, j, i0, stride)) return false;
  i = i0 + stride * (t % cs.mpr);
  return i <= L.m1;
}

// per-level smoother launches: one thread per cell of the colour, packed into
// 64-thread blocks so that a level's warps spread over many SMs (on the FP64
// pipe a warp costs the same with 1 or 32 lanes busy)
constexpr int SNT = 64;

template <typename T, class Form>
__global__ void __launch_bounds__(SNT) k_vanka(Prm<T> P, Lv<T> L, int colour, T omega) {
  pdl_enter();
  ColourSlots cs = vanka_slots(L, colour);
  int t = blockIdx.x * SNT + threadIdx.x;
  int i, j;
  if (t >= cs.n || !vanka_slot_cell(L, colour, cs, t, i, j)) return;
  vanka_cell<T, Form>(P, L, i, j, omega);
}

template <typename T, class Form>
__global__ void __launch_bounds__(SNT) k_coupled(Prm<T> P, Lv<T> L, int colour, T omega) {
  pdl_enter();
  ColourSlots cs = vanka_slots(L, colour);
  int t = blockIdx.x * SNT + threadIdx.x;
  int i, j;
  if (t >= cs.n || !vanka_slot_cell(L, colour, cs, t, i, j)) return;
  coupled_cell<T, Form>(P, L, i, j, omega);
}

// --------------------------------------------------------------------------
// projection method (Sec. 7.2): the intermediate-velocity block, pressure
// Gauss-Seidel, the projected velocity and the projection dissipation
// --------------------------------------------------------------------------
// step 2: exact solve of the 4x4 block of the intermediate velocities
// (ut_W, ut_E, vt_S, vt_N) of cell (i,j) in the rows of (pj-num-mx)
template <typename T, class Form>
__device__ __forceinline__ void vanka4_cell(const Prm<T>& P, const Lv<T>& L, int i, int j, T omega) {
  T A5[5][5], b5[5];
  bool act[5];
  vanka_system<T, Form>(P, L, i, j, A5, b5, act);
  const int W = L.pitch;
  int k = L.at(i, j);
  solve_vanka<T, 4>(A5, b5, act, L.visn[k] * P.iRe * L.ih2 * T(1.0 / 3.0), L.ih * P.iM, L.ih);
  const T(&b)[5] = b5;
  int eW = (L.px && i == 1) ? L.m1 : i - 1;
  int kW = L.at(eW, j);
  if (act[0]) store_u(L, eW, j, L.u[kW] - omega * b[0]);
  if (act[1]) store_u(L, i, j, L.u[k] - omega * b[1]);
  if (act[2]) store_v(L, i, j - 1, L.v[k - W] - omega * b[2]);
  if (act[3]) store_v(L, i, j, L.v[k] - omega * b[3]);
}

template <typename T, class Form>
__global__ void __launch_bounds__(SNT) k_vanka4(Prm<T> P, Lv<T> L, int colour, T omega) {
  pdl_enter();
  ColourSlots cs = vanka_slots(L, colour);
  int t = blockIdx.x * SNT + threadIdx.x;
  int i, j;
  if (t >= cs.n || !vanka_slot_cell(L, colour, cs, t, i, j)) return;
  vanka4_cell<T, Form>(P, L, i, j, omega);
}

// step 3: Gauss-Seidel on (pj-num-mass) for p_ij.  The row is affine in p_ij:
// u^{n+1} on an open face carries -dt/(M h A rho(c)) times the pressure of each
// adjacent cell, plus the diffusion term (alpha^2/Pe) A m / h^2.
template <typename T>
__device__ __forceinline__ void pgs_cell(const Prm<T>& P, const Lv<T>& L, int i, int j) {
  const int W = L.pitch;
  int k = L.at(i, j);
  const T* rc = L.rhoc;
  T rk = rc[k];
  const T rq[4] = {rc[k + 1], rc[k - 1], rc[k + W], rc[k - W]};
  T w[4];
  proj_faces(P, L, i, j, rk, rq, w);
  T R = opp_p_w(P, L, k, w) - L.fp[k];
  const bool wall[4] = {!L.px && i == L.m1, !L.px && i == 1, j == L.m2, j == 1};
  const int off[4] = {1, -1, W, -W};
  T d = T(0);
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    if (wall[f]) continue;
    int q = k + off[f];
    T Ar = T(0.5) * (rk + rq[f]);
    d += P.iM / (Ar * P.idt) * L.ih2 + P.alpha * P.alpha * P.iPe * T(0.5) * (L.mobn[k] + L.mobn[q]) * L.ih2;
  }
  store_cell(L, L.p, i, j, L.p[k] - R / d);
}

// pgs_cell by a team of four lanes (lane & 3 = q: face W, E, S, N): lane q
// takes u^{n+1} at face q, its share of the mass row and of the row's
// derivative in p_ij; butterflies add them; lane 0 stores.
template <typename T>
__device__ __forceinline__ void pgs_team(const Prm<T>& P, const Lv<T>& L, int i, int j, bool ok) {
  const int W = L.pitch;
  const int q = threadIdx.x & 3;
  const bool open = q == 0 ? (L.px || i > 1) : q == 1 ? (L.px || i < L.m1) : q == 2 ? j > 1 : j < L.m2;
  int k = L.at(i, j);
  const int nq = k + (q == 0 ? -1 : q == 1 ? 1 : q == 2 ? -W : W);
  T rk = L.rhoc[k], rq = L.rhoc[nq];
  T wq = proj_face_team(P, L, k, q, open, rk, rq);
  T am = L.mobn[nq] + L.mobn[k];
  T sdiv = team_sum<T>((q & 1) ? wq : -wq);
  T sflux = team_sum<T>(T(0.5) * am * ((L.mu[nq] - L.mu[k]) + P.alpha * (L.p[nq] - L.p[k])));
  T Ar = T(0.5) * (rk + rq);
  T sd = team_sum<T>(open ? P.iM / (Ar * P.idt) * L.ih2 + P.alpha * P.alpha * P.iPe * T(0.5) * am * L.ih2 : T(0));
  T R = sdiv * L.ih - P.alpha * P.iPe * L.ih2 * sflux - L.fp[k];
  if (ok && q == 0) store_cell(L, L.p, i, j, L.p[k] - R / sd);
}

template <typename T>
__global__ void __launch_bounds__(64) k_pgs_team(Prm<T> P, Lv<T> L, int colour) {
  pdl_enter();
  int mpr = (L.m1 + 1) / 2;
  int n = mpr * L.m2;
  int t = blockIdx.x * 64 + threadIdx.x;
  if ((t & ~31) >= 4 * n) return;  // warp-uniform
  int s = t >> 2;
  int j = 1, i = 1;
  bool ok = false;
  if (s < n) {
    j = s / mpr + 1;
    i = (((colour - j) & 1) ? 1 : 2) + 2 * (s % mpr);
    ok = i <= L.m1;
  }
  if (!ok) i = j = 1;
  pgs_team<T>(P, L, i, j, ok);
}

// cells of colour (i + j) % 2 == colour, packed as in k_ch
template <typename T>
__global__ void __launch_bounds__(64) k_pgs(Prm<T> P, Lv<T> L, int colour) {
  pdl_enter();
  int mpr = (L.m1 + 1) / 2;
  int t = blockIdx.x * 64 + threadIdx.x;
  if (t >= mpr * L.m2) return;
  int j = t / mpr + 1;
  int i = (((colour - j) & 1) ? 1 : 2) + 2 * (t % mpr);
  if (i > L.m1) return;
  pgs_cell<T>(P, L, i, j);
}

// u^{n+1} on the x-edges i = 0..m1 (rows 1..m2) and v^{n+1} on the y-edges
// j = 0..m2 (columns 1..m1), into uo, vo (level layout); ghosts are filled after
template <typename T>
__global__ void k_proj_velocity(Prm<T> P, Lv<T> L, T* uo, T* vo) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x;
  int j = blockIdx.y * BY + threadIdx.y;
  if (i > L.m1 || j > L.m2) return;
  int k = L.at(i, j);
  if (j >= 1) uo[k] = proj_u(P, L, i, j);
  if (i >= 1) vo[k] = proj_v(P, L, i, j);
}

// the projection method's extra dissipation, 1/2 ||sqrt(rho(c)) (u^{n+1} - ut)||^2
// in the cell-averaged form of the kinetic energy; per cell before the h^2/2
template <typename T>
__global__ void k_proj_diss(Prm<T> P, Lv<T> L, const T* uo, const T* vo, double* part) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x + 1;
  int j = blockIdx.y * BY + threadIdx.y + 1;
  double val[1] = {0.0};
  if (i <= L.m1 && j <= L.m2) {
    const int W = L.pitch;
    int k = L.at(i, j);
    double r = 1.0 / ((double)P.ia * (double)L.c[k] + (double)P.ib);
    double a = (double)uo[k] - (double)L.u[k], b = (double)uo[k - 1] - (double)L.u[k - 1];
    double c = (double)vo[k] - (double)L.v[k], d = (double)vo[k - W] - (double)L.v[k - W];
    val[0] = r * (0.5 * (a * a + b * b) + 0.5 * (c * c + d * d));
  }
  block_sum_store<1>(val, part, 0);
}

// --------------------------------------------------------------------------
// ghost filling (App. A.6): every ghost entry computed from interior entries
// --------------------------------------------------------------------------
__device__ __forceinline__ int xsrc_cell(int I, int m1, int px) {
  if (I == 0) return px ? m1 : 1;
  if (I == m1 + 1) return px ? 1 : m1;
  return I;
}

// band: I = -1..m1+1 on rows J in {-1, 0, 1?}... we enumerate a 4-wide frame
__device__ __forceinline__ bool frame_pos(int t, int m1, int m2, int& I, int& J) {
  int NX = m1 + 3, NY = m2 + 3;
  if (t < 4 * NX) {
    int r = t / NX;
    I = t % NX - 1;
    J = r < 2 ? r - 1 : m2 + r - 2;  // rows -1, 0, m2, m2+1
    return true;
  }
  t -= 4 * NX;
  if (t < 4 * NY) {
    int cidx = t / NY;
    J = t % NY - 1;
    I = cidx < 2 ? cidx - 1 : m1 + cidx - 2;  // columns -1, 0, m1, m1+1
    return true;
  }
  return false;
}

template <typename T>
__device__ __forceinline__ void fill_cell_ghost(const Lv<T>& L, T* a, int I, int J) {
  if (I < 0 || J < 0) return;
  bool gx = (I == 0 || I == L.m1 + 1), gy = (J == 0 || J == L.m2 + 1);
  if (!gx && !gy) return;
  int si = xsrc_cell(I, L.m1, L.px);
  int sj = J == 0 ? 1 : (J == L.m2 + 1 ? L.m2 : J);
  a[L.at(I, J)] = a[L.at(si, sj)];
}

template <typename T>
__device__ __forceinline__ T u_interior_or_zero(const Lv<T>& L, const T* a, int I, int J) {
  // value of u(I, J) for J in 1..m2 after applying the x rule
  if (L.px) {
    int s = I;
    if (I == 0) s = L.m1;
    else if (I == -1) s = L.m1 - 1;
    else if (I == L.m1 + 1) s = 1;
    return a[L.at(s, J)];
  }
  if (I <= 0 || I >= L.m1) return T(0);
  return a[L.at(I, J)];
}

template <typename T>
__device__ __forceinline__ void fill_u_ghost(const Lv<T>& L, T* a, int I, int J) {
  if (J < 0) return;
  bool xg = L.px ? (I == 0 || I == -1 || I == L.m1 + 1) : (I <= 0 || I >= L.m1);
  bool yg = (J == 0 || J == L.m2 + 1);
  if (!xg && !yg) return;
  if (yg) {
    int sj = J == 0 ? 1 : L.m2;
    a[L.at(I, J)] = -u_interior_or_zero(L, a, I, sj);
  } else {
    a[L.at(I, J)] = u_interior_or_zero(L, a, I, J);
  }
}

template <typename T>
__device__ __forceinline__ T v_interior_or_zero(const Lv<T>& L, const T* a, int I, int J) {
  // value of v(I, J) for I in 1..m1 after applying the y (wall) rule
  if (J <= 0 || J >= L.m2) return T(0);
  return a[L.at(I, J)];
}

template <typename T>
__device__ __forceinline__ void fill_v_ghost(const Lv<T>& L, T* a, int I, int J) {
  if (I < 0) return;
  bool xg = (I == 0 || I == L.m1 + 1);
  bool yg = (J <= 0 || J >= L.m2);
  if (!xg && !yg) return;
  if (xg) {
    int si = xsrc_cell(I, L.m1, L.px);
    T s = v_interior_or_zero(L, a, si, J);
    a[L.at(I, J)] = L.px ? s : -s;
  } else {
    a[L.at(I, J)] = T(0);
  }
}

template <typename T>
__global__ void k_bc_unknowns(Lv<T> L) {
  pdl_enter();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int I, J;
  if (!frame_pos(t, L.m1, L.m2, I, J)) return;
  fill_cell_ghost(L, L.c, I, J);
  if (L.rhoc) fill_cell_ghost(L, L.rhoc, I, J);
  fill_cell_ghost(L, L.mu, I, J);
  fill_cell_ghost(L, L.p, I, J);
  fill_u_ghost(L, L.u, I, J);
  fill_v_ghost(L, L.v, I, J);
}

template <typename T>
__global__ void k_bc_frozen(Lv<T> L) {
  pdl_enter();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int I, J;
  if (!frame_pos(t, L.m1, L.m2, I, J)) return;
  fill_cell_ghost(L, L.cn, I, J);
  fill_u_ghost(L, L.un, I, J);
  fill_v_ghost(L, L.vn, I, J);
}

// rho(c^n), m(c^n), mu(c^n) on the whole ghosted cell range; G(c^n) inside
template <typename T>
__global__ void k_frozen_derived(Prm<T> P, Lv<T> L) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x;
  int j = blockIdx.y * BY + threadIdx.y;
  if (i > L.m1 + 1 || j > L.m2 + 1) return;
  int k = L.at(i, j);
  T c = L.cn[k];
  L.rhon[k] = rho_of(P, c);
  L.mobn[k] = mob_of(P, c);
  L.visn[k] = visc_of(P, c);
  if (i >= 1 && i <= L.m1 && j >= 1 && j <= L.m2) L.Gn[k] = G_h2(L.cn, k, L.pitch) * L.ih2;
}

// frozen coefficients of (pm-num-mx): cells and vertices (needs rho^n, mu(c^n), ghosts)
template <typename T>
__global__ void k_frozen_coef1(Lv<T> L) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x;
  int j = blockIdx.y * BY + threadIdx.y;
  if (i > L.m1 + 1 || j > L.m2 + 1) return;
  const int W = L.pitch;
  int k = L.at(i, j);
  const T *rn = L.rhon, *vis = L.visn, *un = L.un, *vn = L.vn, *cn = L.cn;
  L.Sx[k] = rn[k] * T(0.5) * (un[k] + un[k - 1]);   // cell (i,j)
  L.Sy[k] = rn[k] * T(0.5) * (vn[k] + vn[k - W]);
  if (i <= L.m1 && j <= L.m2) {  // vertex (i+1/2, j+1/2), edges (i+1/2, j), (i, j+1/2)
    T Ar = T(0.25) * (rn[k] + rn[k + 1] + rn[k + W] + rn[k + 1 + W]);
    L.Qx[k] = Ar * T(0.5) * (vn[k + 1] + vn[k]);
    L.Qy[k] = Ar * T(0.5) * (un[k + W] + un[k]);
    L.Av[k] = T(0.25) * (vis[k] + vis[k + 1] + vis[k + W] + vis[k + 1 + W]);
    L.Aru[k] = T(0.5) * (rn[k] + rn[k + 1]);
    L.Arv[k] = T(0.5) * (rn[k] + rn[k + W]);
    L.Tx[k] = T(0.5) * (cn[k + 1] - cn[k]) * L.ih;
    L.Ty[k] = T(0.5) * (cn[k + W] - cn[k]) * L.ih;
  }
}

// divergence corrections of (e1e1-2) on edges (needs k_frozen_coef1)
template <typename T>
__global__ void k_frozen_coef2(Lv<T> L) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x;
  int j = blockIdx.y * BY + threadIdx.y;
  if (i > L.m1 || j > L.m2) return;
  const int W = L.pitch;
  int k = L.at(i, j);
  if (j >= 1) L.Dvu[k] = T(0.5) * ((L.Sx[k + 1] - L.Sx[k]) + (L.Qx[k] - L.Qx[k - W])) * L.ih;
  if (i >= 1) L.Dvv[k] = T(0.5) * ((L.Qy[k] - L.Qy[k - 1]) + (L.Sy[k + W] - L.Sy[k])) * L.ih;
}

// The assembled stencil of one momentum row of (pm-num-mx) at edge k (mom_asm):
// s the stride along the edge normal, t across it; S the cell-centred and Q the
// vertex convection coefficients, Tf = D c^n / 2 on the edge, t1 the time
// term's coefficient T1.  With the differences of the row written out,
//   conv = 1/2 h^-1 (S[k+s] (a[k+s] - a) - S[k] (a - a[k-s]) ... )  and
//   visc = -h^-2/Re ((4/3)(vis[k+s] (a[k+s] - a) - vis[k] (a - a[k-s]))
//                    + Av[k] (a[k+t] - a) - Av[k-t] (a - a[k-t])) + cross terms,
// each neighbour's coefficient is the sum of its convective and viscous
// parts, and the edge's own coefficient is minus their sum plus t1.  Wall
// edges keep the undoubled coefficients: the row reads the reflected ghosts.
template <typename T>
__device__ __forceinline__ void assemble_row(const Prm<T>& P, const Lv<T>& L, int k, int s, int t,
                                             T t1, const T* S, const T* Q, const T* Tf, T* C,
                                             T* aP, T* aM, T* tP, T* tM, T* M0, T* M1) {
  const T* vis = L.visn;
  const T hc = T(0.5) * L.ih, hv = P.iRe * L.ih2, f43 = T(4.0 / 3.0);
  T vl = vis[k], vr = vis[k + s];
  T ap = hc * S[k + s] - f43 * hv * vr;
  T am = -hc * S[k] - f43 * hv * vl;
  T tp = hc * Q[k] - hv * L.Av[k];
  T tm = -hc * Q[k - t] - hv * L.Av[k - t];
  aP[k] = ap;
  aM[k] = am;
  tP[k] = tp;
  tM[k] = tm;
  C[k] = t1 + hc * (-S[k + s] + S[k] - Q[k] + Q[k - t]) +
         hv * (f43 * (vr + vl) + L.Av[k] + L.Av[k - t]);
  M0[k] = -L.rhon[k + s] * Tf[k] * P.iM;
  M1[k] = -L.rhon[k] * Tf[k] * P.iM;
}

// per-step row coefficients of the momentum rows (needs k_frozen_coef2): time =
// x T1 + T0 + A rho(c) x/(2dt); Dg = the iterate-independent part of the
// diagonal entry (the whole entry is Dg + A rho(c)/(2dt)), with the reflected
// no-slip ghosts doubling the tangential wall terms (g = 2)
template <typename T>
__global__ void k_frozen_coef3(Prm<T> P, Lv<T> L) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x;
  int j = blockIdx.y * BY + threadIdx.y;
  if (i > L.m1 || j > L.m2) return;
  const int W = L.pitch;
  int k = L.at(i, j);
  const T* vis = L.visn;
  const T third = T(1.0 / 3.0);
  if (j >= 1) {  // x-edge (i+1/2, j)
    T Arn = L.Aru[k];
    T gt = (j == L.m2) ? T(2) : T(1), gb = (j == 1) ? T(2) : T(1);
    T t1 = T(0.5) * Arn * P.idt + L.Dvu[k];
    L.T1u[k] = t1;
    L.T0u[k] = -Arn * L.un[k] * P.idt;
    L.Dgu[k] = t1 + T(0.5) * L.ih * (-L.Sx[k + 1] + L.Sx[k] - L.Qx[k] * gt + L.Qx[k - W] * gb) +
               P.iRe * L.ih2 * ((vis[k + 1] + vis[k]) * (T(1) + third) + gt * L.Av[k] + gb * L.Av[k - W]);
    assemble_row(P, L, k, 1, W, t1, L.Sx, L.Qx, L.Tx, L.Cu, L.aPu, L.aMu, L.tPu, L.tMu, L.M0u,
                 L.M1u);
  }
  if (i >= 1) {  // y-edge (i, j+1/2)
    T Arn = L.Arv[k];
    T ge = (!L.px && i == L.m1) ? T(2) : T(1), gw = (!L.px && i == 1) ? T(2) : T(1);
    T t1 = T(0.5) * Arn * P.idt + L.Dvv[k];
    L.T1v[k] = t1;
    L.T0v[k] = -Arn * L.vn[k] * P.idt;
    L.Dgv[k] = t1 + T(0.5) * L.ih * (-L.Qy[k] * ge + L.Qy[k - 1] * gw - L.Sy[k + W] + L.Sy[k]) +
               P.iRe * L.ih2 * (ge * L.Av[k] + gw * L.Av[k - 1] + (vis[k + W] + vis[k]) * (T(1) + third));
    assemble_row(P, L, k, W, 1, t1, L.Sy, L.Qy, L.Ty, L.Cv, L.aPv, L.aMv, L.tPv, L.tMv, L.M0v,
                 L.M1v);
  }
}

// --------------------------------------------------------------------------
// FAS transfers
// --------------------------------------------------------------------------
// coarse iterate = R x_h (cells: 4-mean; edges: mean of the 2 coincident fine edges),
// and a copy kept for the correction
template <typename T>
__device__ __forceinline__ void restrict_state_cell(const Prm<T>& P, const Lv<T>& F, const Lv<T>& C,
                                                    int I, int J) {
  int kc = C.at(I, J);
  if (I >= 1 && J >= 1) {
    int kf = F.at(2 * I - 1, 2 * J - 1), W = F.pitch;
    T a = T(0.25) * (F.c[kf] + F.c[kf + 1] + F.c[kf + W] + F.c[kf + W + 1]);
    T b = T(0.25) * (F.mu[kf] + F.mu[kf + 1] + F.mu[kf + W] + F.mu[kf + W + 1]);
    T d = T(0.25) * (F.p[kf] + F.p[kf + 1] + F.p[kf + W] + F.p[kf + W + 1]);
    C.c[kc] = a; C.sc[kc] = a;
    if (C.rhoc) C.rhoc[kc] = rho_of(P, a);
    C.mu[kc] = b; C.smu[kc] = b;
    C.p[kc] = d; C.sp[kc] = d;
  }
  if (J >= 1) {  // u edge (I, J), I = 0..M1
    int kf = F.at(2 * I, 2 * J - 1);
    T a = T(0.5) * (F.u[kf] + F.u[kf + F.pitch]);
    C.u[kc] = a; C.su[kc] = a;
  }
  if (I >= 1) {  // v edge (I, J), J = 0..M2
    int kf = F.at(2 * I - 1, 2 * J);
    T a = T(0.5) * (F.v[kf] + F.v[kf + 1]);
    C.v[kc] = a; C.sv[kc] = a;
  }
}

// coarse iterate = R x_h (cells: 4-mean; edges: mean of the 2 coincident fine edges),
// and a copy kept for the correction
template <typename T>
__global__ void k_restrict_state(Prm<T> P, Lv<T> F, Lv<T> C) {
  pdl_enter();
  int I = blockIdx.x * BX + threadIdx.x;
  int J = blockIdx.y * BY + threadIdx.y;
  if (I > C.m1 || J > C.m2) return;
  restrict_state_cell(P, F, C, I, J);
}

template <typename T>
__device__ __forceinline__ T ru_at(const Lv<T>& F, int i, int j) {
  if (F.px) {
    if (i > F.m1) i -= F.m1;
    if (i < 1) i += F.m1;
  } else if (i <= 0 || i >= F.m1) {
    return T(0);
  }
  return F.ru[F.at(i, j)];
}
template <typename T>
__device__ __forceinline__ T rv_at(const Lv<T>& F, int i, int j) {
  if (j <= 0 || j >= F.m2) return T(0);
  return F.rv[F.at(i, j)];
}

// coarse right-hand side f_H = R r_h (cells: 4-mean; edges: full weighting),
// to which k_residual<MODE 1> then adds N_H(R x_h)
template <typename T>
__device__ __forceinline__ void restrict_res_cell(const Lv<T>& F, const Lv<T>& C, int I, int J) {
  int kc = C.at(I, J);
  int kf = F.at(2 * I - 1, 2 * J - 1), W = F.pitch;
  C.fc[kc] = T(0.25) * (F.rc[kf] + F.rc[kf + 1] + F.rc[kf + W] + F.rc[kf + W + 1]);
  C.fmu[kc] = T(0.25) * (F.rmu[kf] + F.rmu[kf + 1] + F.rmu[kf + W] + F.rmu[kf + W + 1]);
  C.fp[kc] = T(0.25) * (F.rp[kf] + F.rp[kf + 1] + F.rp[kf + W] + F.rp[kf + W + 1]);
  if (I <= C.uhi()) {
    T s = T(0);
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      int jf = 2 * J - 1 + jj;
      s += T(0.25) * ru_at(F, 2 * I - 1, jf) + T(0.5) * ru_at(F, 2 * I, jf) +
           T(0.25) * ru_at(F, 2 * I + 1, jf);
    }
    C.fu[kc] = T(0.5) * s;
  }
  if (J < C.m2) {
    T s = T(0);
#pragma unroll
    for (int ii = 0; ii < 2; ++ii) {
      int ifn = 2 * I - 1 + ii;
      s += T(0.25) * rv_at(F, ifn, 2 * J - 1) + T(0.5) * rv_at(F, ifn, 2 * J) +
           T(0.25) * rv_at(F, ifn, 2 * J + 1);
    }
    C.fv[kc] = T(0.5) * s;
  }
}

template <typename T>
__global__ void k_restrict_res(Lv<T> F, Lv<T> C) {
  pdl_enter();
  int I = blockIdx.x * BX + threadIdx.x + 1;
  int J = blockIdx.y * BY + threadIdx.y + 1;
  if (I > C.m1 || J > C.m2) return;
  restrict_res_cell(F, C, I, J);
}

template <typename T>
__global__ void k_restrict_frozen(Lv<T> F, Lv<T> C) {
  pdl_enter();
  int I = blockIdx.x * BX + threadIdx.x;
  int J = blockIdx.y * BY + threadIdx.y;
  if (I > C.m1 || J > C.m2) return;
  int kc = C.at(I, J);
  if (I >= 1 && J >= 1) {
    int kf = F.at(2 * I - 1, 2 * J - 1), W = F.pitch;
    C.cn[kc] = T(0.25) * (F.cn[kf] + F.cn[kf + 1] + F.cn[kf + W] + F.cn[kf + W + 1]);
  }
  if (J >= 1) {
    int kf = F.at(2 * I, 2 * J - 1);
    C.un[kc] = T(0.5) * (F.un[kf] + F.un[kf + F.pitch]);
  }
  if (I >= 1) {
    int kf = F.at(2 * I - 1, 2 * J);
    C.vn[kc] = T(0.5) * (F.vn[kf] + F.vn[kf + 1]);
  }
}

// x_h += P(x_H - saved_H): cells piecewise constant; edges coincident or linear
// in the normal direction, constant in the tangential direction
template <typename T>
__device__ __forceinline__ void prolong_cell(const Prm<T>& P, const Lv<T>& F, const Lv<T>& C, int i,
                                             int j) {
  int k = F.at(i, j);
  int I = (i + 1) >> 1, J = (j + 1) >> 1;
  int kc = C.at(I, J);
  F.c[k] += C.c[kc] - C.sc[kc];
  if (F.rhoc) F.rhoc[k] = rho_of(P, F.c[k]);
  F.mu[k] += C.mu[kc] - C.smu[kc];
  F.p[k] += C.p[kc] - C.sp[kc];
  if (i <= F.uhi()) {
    T e;
    if ((i & 1) == 0) {
      int q = C.at(i >> 1, J);
      e = C.u[q] - C.su[q];
    } else {
      int q0 = C.at((i - 1) >> 1, J), q1 = C.at((i + 1) >> 1, J);
      e = T(0.5) * ((C.u[q0] - C.su[q0]) + (C.u[q1] - C.su[q1]));
    }
    F.u[k] += e;
  }
  if (j < F.m2) {
    T e;
    if ((j & 1) == 0) {
      int q = C.at(I, j >> 1);
      e = C.v[q] - C.sv[q];
    } else {
      int q0 = C.at(I, (j - 1) >> 1), q1 = C.at(I, (j + 1) >> 1);
      e = T(0.5) * ((C.v[q0] - C.sv[q0]) + (C.v[q1] - C.sv[q1]));
    }
    F.v[k] += e;
  }
}

template <typename T>
__global__ void k_prolong(Prm<T> P, Lv<T> F, Lv<T> C) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x + 1;
  int j = blockIdx.y * BY + threadIdx.y + 1;
  if (i > F.m1 || j > F.m2) return;
  prolong_cell(P, F, C, i, j);
}

// --------------------------------------------------------------------------
// the coarse end of a V-cycle in one launch: levels small enough for one SM,
// or for one thread-block cluster of up to 16 SMs, run their smoothing
// colours, residuals, transfers and ghost fills as group-stride loops
// separated by group barriers (__syncthreads(), or the cluster barrier), one
// launch instead of dozens.  Per-cell work is the same device code as the grid
// kernels above, in the same colour order, so the results are the same.
// --------------------------------------------------------------------------
// coarse base X_H = R X_h (cells: 4-mean; edges: 2 coincident fine edges), one entry
template <typename T>
__device__ __forceinline__ void restrict_base_cell(const Lv<T>& F, const Lv<T>& C, int I, int J) {
  int kc = C.at(I, J);
  if (I >= 1 && J >= 1) {
    int kf = F.at(2 * I - 1, 2 * J - 1), W = F.pitch;
    C.Bc[kc] = T(0.25) * (F.Bc[kf] + F.Bc[kf + 1] + F.Bc[kf + W] + F.Bc[kf + W + 1]);
    C.Bmu[kc] = T(0.25) * (F.Bmu[kf] + F.Bmu[kf + 1] + F.Bmu[kf + W] + F.Bmu[kf + W + 1]);
    C.Bdc[kc] = T(0.25) * (F.Bdc[kf] + F.Bdc[kf + 1] + F.Bdc[kf + W] + F.Bdc[kf + W + 1]);
  }
  if (J >= 1) {
    int kf = F.at(2 * I, 2 * J - 1);
    C.Bu[kc] = T(0.5) * (F.Bu[kf] + F.Bu[kf + F.pitch]);
  }
  if (I >= 1) {
    int kf = F.at(2 * I - 1, 2 * J);
    C.Bv[kc] = T(0.5) * (F.Bv[kf] + F.Bv[kf + 1]);
  }
}

// ghosts of the base arrays
template <typename T>
__device__ __forceinline__ void bc_base_cell(const Lv<T>& L, int I, int J) {
  fill_cell_ghost(L, L.Bc, I, J);
  fill_cell_ghost(L, L.Bmu, I, J);
  fill_cell_ghost(L, L.Bdc, I, J);
  fill_u_ghost(L, L.Bu, I, J);
  fill_v_ghost(L, L.Bv, I, J);
}

// The fused V-cycle runs in one thread block or in one thread-block cluster of
// gridDim.x blocks (the grid is the cluster).  Its loops and colour steps go
// over a rank of the whole group.  Warps are interleaved across the blocks:
// rank = ((warp * blocks + block) * 32 + lane), so the first 4 x blocks warps
// of a colour step sit on distinct SM sub-partitions (warp w of a block runs on
// sub-partition w mod 4), each of which owns one FP64 pipe.  The low five bits
// of the rank are the hardware lane, so four-lane teams stay inside a warp.
// One block: the rank is threadIdx.x and the step barrier is __syncthreads().
// A cluster: the barrier is the hardware cluster barrier, whose release and
// acquire order every block's global-memory writes before the next step's
// reads; every thread of the cluster reaches every barrier.
__device__ __forceinline__ int grp_rank() {
  return (((threadIdx.x >> 5) * gridDim.x + blockIdx.x) << 5) | (threadIdx.x & 31);
}
__device__ __forceinline__ int grp_size() { return gridDim.x * blockDim.x; }
__device__ __forceinline__ void grp_sync() {
  if (gridDim.x == 1) {
    __syncthreads();
  } else {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
  }
}

template <typename T>
struct CoarseLevels {
  Lv<T> L[QN_MAX_FUSED_LEVELS];
  int n;
  int base;  // error equation: restrict the base state to L[1..n-1] first
};

template <typename T>
__device__ __forceinline__ void bc_unknowns_block(const Lv<T>& L) {
  int n = 4 * (L.m1 + 3) + 4 * (L.m2 + 3);
  for (int t = grp_rank(); t < n; t += grp_size()) {
    int I, J;
    if (!frame_pos(t, L.m1, L.m2, I, J)) continue;
    fill_cell_ghost(L, L.c, I, J);
    if (L.rhoc) fill_cell_ghost(L, L.rhoc, I, J);
    fill_cell_ghost(L, L.mu, I, J);
    fill_cell_ghost(L, L.p, I, J);
    fill_u_ghost(L, L.u, I, J);
    fill_v_ghost(L, L.v, I, J);
  }
  grp_sync();
}

// --------------------------------------------------------------------------
// single-block smoothing of the coarse levels.  An FP64 warp instruction
// holds the SM sub-partition's FP64 pipe for about 64 cycles however many of
// its lanes are active, so a colour step on a small level costs (warp
// instructions per visit) x (warps per sub-partition): threads are packed onto
// the cells of the colour, and on the smallest levels four lanes share one
// Vanka block (one edge row each).
// --------------------------------------------------------------------------
// Momentum row of the full-form operator in one direction: d = 0 is the x row
// (op_u, unknown u), d = 1 the y row (op_v, unknown v).  Both directions run
// the same instructions on different arrays and strides (s along the edge
// normal, t across it).
template <typename T>
struct MomRow {
  const T *a, *b, *S, *Q, *Tf, *Arn, *Dv, *T1, *T0, *Dg, *B, *f;
  int s, t, d;
  T grav;
};

// FullForm uses the per-step row coefficients T1, T0, Dg; ErrForm (the error
// equation of the defect correction) has none of them, adds the base-state term
// of the time derivative and has no gravity (it cancels in N(X + e) - N(X))
template <typename T, class Form>
__device__ __forceinline__ MomRow<T> mom_row(const Prm<T>& P, const Lv<T>& L, int d) {
  MomRow<T> R;
  R.Dv = d ? L.Dvv : L.Dvu;
  R.B = d ? L.Bv : L.Bu;
  R.a = d ? L.v : L.u;
  R.b = d ? L.u : L.v;
  R.S = d ? L.Sy : L.Sx;
  R.Q = d ? L.Qy : L.Qx;
  R.Tf = d ? L.Ty : L.Tx;
  R.Arn = d ? L.Arv : L.Aru;
  R.T1 = d ? L.T1v : L.T1u;
  R.T0 = d ? L.T0v : L.T0u;
  R.Dg = d ? L.Dgv : L.Dgu;
  R.f = d ? L.fv : L.fu;
  R.s = d ? L.pitch : 1;
  R.t = d ? 1 : L.pitch;
  R.d = d;
  // gravity: the primitive momentum row only (the error equation cancels it,
  // the projection method puts it in the projection equation)
  R.grav = (d && std::is_same<Form, FullForm>::value) ? P.Fr_inv : T(0);
  return R;
}

// N - f of the momentum row at edge index k (op_u / op_v, or opd_u / opd_v for
// ErrForm), from rho(c) of the edge's two cells (full values) passed in
template <typename T, class Form>
__device__ __forceinline__ T mom_residual(const Prm<T>& P, const Lv<T>& L, const MomRow<T>& R, int k,
                                          T rl, T rr) {
  T Ar = T(0.5) * (rl + rr);
  // FP64 primitive rows: the per-step assembled stencil
  if constexpr (std::is_same<Form, FullForm>::value && sizeof(T) == 8)
    return mom_asm(P, L, R.d, k, Ar) - R.f[k];
  const int s = R.s, t = R.t;
  const T *a = R.a, *b = R.b, *vis = L.visn, *rn = L.rhon;
  T ae = a[k];
  T dl = (ae - a[k - s]) * L.ih, dr = (a[k + s] - ae) * L.ih;
  T dvl = dl + (b[k] - b[k - t]) * L.ih;
  T dvr = dr + (b[k + s] - b[k + s - t]) * L.ih;
  T Dp = (a[k + t] - ae) * L.ih, Dm = (ae - a[k - t]) * L.ih;
  T conv = T(0.5) * (R.S[k + s] * dr + R.S[k] * dl + R.Q[k] * Dp + R.Q[k - t] * Dm);
  T time;
  if constexpr (std::is_same<Form, ErrForm>::value) {
    // rho(X + e) - rho(X) of the two cells by the secant of rho, times the base velocity
    T dAr = T(0.5) * (rsec_(P, rl, rho_of(P, L.Bc[k])) * L.c[k] +
                      rsec_(P, rr, rho_of(P, L.Bc[k + s])) * L.c[k + s]);
    T Arn = R.Arn[k];
    time = Arn * ae * P.idt + T(0.5) * (Ar - Arn) * P.idt * ae + T(0.5) * dAr * P.idt * R.B[k] +
           R.Dv[k] * ae;
  } else {
    time = ae * R.T1[k] + R.T0[k] + T(0.5) * P.idt * Ar * ae;
  }
  T press = T(0), st = T(0);  // the projection method's intermediate-velocity row has neither
  if constexpr (!std::is_same<Form, ProjForm>::value) {
    press = (L.p[k + s] - L.p[k]) * L.ih * P.iM;
    st = -(rn[k + s] * L.mu[k] + rn[k] * L.mu[k + s]) * R.Tf[k] * P.iM;
  }
  T vl = vis[k], vr = vis[k + s];
  T visc = -P.iRe * L.ih * ((vr * dr - vl * dl) + (L.Av[k] * Dp - L.Av[k - t] * Dm) +
                            (vr * dvr - vl * dvl) * T(1.0 / 3.0));
  return time + conv + press + st + visc + R.grav * R.Arn[k] - R.f[k];
}

// Diagonal entry dq and residual bq = N - f (0 on a wall edge) of momentum row
// q of the Vanka block of cell (i,j), for lane q of a team: direction d (0:
// x-edge, 1: y-edge), edge index ke.  The x and y rows run the same
// instruction stream on different arrays and strides (mom_row).
template <typename T, class Form>
__device__ __forceinline__ void team_row(const Prm<T>& P, const Lv<T>& L, int i, int j, int d, int ke,
                                         bool mine, T& dq, T& bq) {
  const T ih = L.ih, ih2 = L.ih2, third = T(1.0 / 3.0);
  MomRow<T> R = mom_row<T, Form>(P, L, d);
  T rl = Form::rho(P, L, ke), rr = Form::rho(P, L, ke + R.s);
  T Ar = T(0.5) * (rl + rr);
  const T* vis = L.visn;
  if constexpr (std::is_same<Form, ErrForm>::value) {
    // the diagonal from the frozen arrays (error levels carry no row coefficients)
    T gp = d ? ((!L.px && i == L.m1) ? T(2) : T(1)) : ((j == L.m2) ? T(2) : T(1));
    T gm = d ? ((!L.px && i == 1) ? T(2) : T(1)) : ((j == 1) ? T(2) : T(1));
    T Arn = R.Arn[ke];
    dq = Arn * P.idt + T(0.5) * (Ar - Arn) * P.idt +
         T(0.5) * ih * (-R.S[ke + R.s] + R.S[ke] - R.Q[ke] * gp + R.Q[ke - R.t] * gm) + R.Dv[ke] +
         P.iRe * ih2 * ((vis[ke + R.s] + vis[ke]) * (T(1) + third) + gp * L.Av[ke] + gm * L.Av[ke - R.t]);
  } else {
    dq = R.Dg[ke] + T(0.5) * P.idt * Ar;
  }
  bq = mom_residual<T, Form>(P, L, R, ke, rl, rr);  // wall edges too (padded arrays), then discarded
  if (!mine) bq = T(0);
}

// The structured solve of solve_vanka, split over a team of four lanes.  The
// velocity block is B + v3 w w^T with B block diagonal over the pairs (W, E)
// and (S, N).  Lane q forms the 2x2 block of its pair (p0, p1) = (q & 2, q | 1)
// exactly as its partner does, and row q of z = B^-1 w; a butterfly gives
// s = w.z.  apply() then takes a right-hand side (row rq on lane q, pressure
// entry r4), forms row q of y = B^-1 r, t = w.y by a butterfly, and returns
// row q of the solution with the pressure in pr.  Rows of wall edges are
// identity rows with rq = 0.
template <typename T>
struct TeamSolve {
  T B00, B01, B10, B11, idet, z, g, iden, v3, a, ih;
  bool odd;
  // with_p = false: the 4x4 velocity block alone (the projection method's
  // intermediate-velocity block), solved as solve_vanka<T, 4> does
  __device__ __forceinline__ TeamSolve(const Prm<T>& P, const Lv<T>& L, int q, T dq, bool ap0, bool ap1,
                                       T S, T vc, T A44, bool with_p = true) {
    const unsigned FULL = 0xffffffffu;
    ih = L.ih;
    v3 = vc * P.iRe * L.ih2 * T(1.0 / 3.0);
    a = with_p ? L.ih * P.iM : T(0);
    odd = q & 1;
    T dqo = __shfl_xor_sync(FULL, dq, 1);
    T D0 = odd ? dqo : dq, D1 = odd ? dq : dqo;
    B00 = ap0 ? D0 - v3 : T(1);
    B11 = ap1 ? D1 - v3 : T(1);
    B01 = (ap0 && ap1) ? T(0.5) * S * ih - vc * P.iRe * L.ih2 : T(0);
    B10 = (ap0 && ap1) ? -T(0.5) * S * ih - vc * P.iRe * L.ih2 : T(0);
    idet = qrcp(B00 * B11 - B01 * B10);
    T zn = odd ? ((ap1 ? B00 : T(0)) + (ap0 ? B10 : T(0))) : ((ap0 ? B11 : T(0)) + (ap1 ? B01 : T(0)));
    z = (odd ? -zn : zn) * idet;
    T sdot = odd ? -z : z;
    sdot += __shfl_xor_sync(FULL, sdot, 1);
    sdot += __shfl_xor_sync(FULL, sdot, 2);
    g = qrcp(T(1) + v3 * sdot);
    iden = with_p ? qrcp(A44 + ih * a * sdot * g) : T(0);
  }
  __device__ __forceinline__ T apply(T rq, T r4, T& pr) const {
    const unsigned FULL = 0xffffffffu;
    T rqo = __shfl_xor_sync(FULL, rq, 1);
    T r0 = odd ? rqo : rq, r1 = odd ? rq : rqo;
    T y = ((odd ? B00 : B11) * (odd ? r1 : r0) - (odd ? B10 : B01) * (odd ? r0 : r1)) * idet;
    T tdot = odd ? -y : y;
    tdot += __shfl_xor_sync(FULL, tdot, 1);
    tdot += __shfl_xor_sync(FULL, tdot, 2);
    pr = (r4 + ih * tdot * g) * iden;
    return y - z * (g * (v3 * tdot + a * pr));
  }
};

// Vanka block of cell (i,j) by a team of four lanes (lane & 3 = q): lane q
// builds row q (diagonal entry and residual of edge q: W, E, S, N) and face
// q's share of the mass row; the team solves the 5x5 system together
// (TeamSolve); lane q writes edge q and lane 0 the pressure.  All 32 lanes of
// the warp call this (ok = false: a spare team, which computes on cell (1,1)
// and stores nothing).
template <typename T, class Form>
__device__ __forceinline__ void vanka_team(const Prm<T>& P, const Lv<T>& L, int i, int j, bool ok,
                                           T omega) {
  const int W = L.pitch;
  const int q = threadIdx.x & 3, d = q >> 1;
  const T ih = L.ih, ih2 = L.ih2;
  int k = L.at(i, j);
  int eW = (L.px && i == 1) ? L.m1 : i - 1;
  int kW = L.at(eW, j);
  bool a0 = L.px || i > 1, a1 = L.px || i < L.m1, a2 = j > 1, a3 = j < L.m2;
  bool mine = q == 0 ? a0 : q == 1 ? a1 : q == 2 ? a2 : a3;
  int ke = q == 0 ? kW : (q == 2 ? k - W : k);
  T dq, bq;
  team_row<T, Form>(P, L, i, j, d, ke, mine, dq, bq);
  // the mass row by faces: lane q takes face q (W, E, S, N) of the cell, the
  // face of its own edge: its velocity in d.u, its flux of
  // grad.(A m grad(mu + alpha p)) and, if open, its share of sum A m
  const T* mob = L.mobn;
  const int nq = k + (q == 0 ? -1 : q == 1 ? 1 : q == 2 ? -W : W);
  T am = mob[nq] + mob[k];
  T f0 = team_sum<T>((q & 1) ? (d ? L.v[k] : L.u[k]) : -(d ? L.v[k - W] : L.u[k - 1]));
  T f1 = team_sum<T>(T(0.5) * am * ((L.mu[nq] - L.mu[k]) + P.alpha * (L.p[nq] - L.p[k])));
  T f2 = team_sum<T>(mine ? am : T(0));
  T A44 = T(0.5) * P.alpha * P.alpha * P.iPe * f2 * ih2;
  T b4 = f0 * ih - P.alpha * P.iPe * ih2 * f1 - L.fp[k];
  TeamSolve<T> ts(P, L, q, dq, d ? a2 : a0, d ? a3 : a1, d ? L.Sy[k] : L.Sx[k], L.visn[k], A44);
  T pr;
  T x = ts.apply(bq, b4, pr);
  if (!ok) return;
  if (mine) {
    if (q == 0) store_u(L, eW, j, L.u[kW] - omega * x);
    else if (q == 1) store_u(L, i, j, L.u[k] - omega * x);
    else if (q == 2) store_v(L, i, j - 1, L.v[k - W] - omega * x);
    else store_v(L, i, j, L.v[k] - omega * x);
  }
  if (q == 0) store_cell(L, L.p, i, j, L.p[k] - omega * pr);
}

// One half of mom_residual for a lane pair of an eight-lane team: half 0 the
// time term, the convection, gravity and -f; half 1 the pressure gradient,
// the surface tension and the viscous terms.  The two halves sum to the
// momentum row's N - f (up to the order of the additions).  FullForm only.
template <typename T>
__device__ __forceinline__ T mom_residual_half(const Prm<T>& P, const Lv<T>& L, const MomRow<T>& R,
                                               int k, T rl, T rr, int half) {
  const int s = R.s, t = R.t;
  const T *a = R.a, *b = R.b;
  T ae = a[k];
  T dl = (ae - a[k - s]) * L.ih, dr = (a[k + s] - ae) * L.ih;
  T Dp = (a[k + t] - ae) * L.ih, Dm = (ae - a[k - t]) * L.ih;
  if (half == 0) {
    T Ar = T(0.5) * (rl + rr);
    T conv = T(0.5) * (R.S[k + s] * dr + R.S[k] * dl + R.Q[k] * Dp + R.Q[k - t] * Dm);
    T time = ae * R.T1[k] + R.T0[k] + T(0.5) * P.idt * Ar * ae;
    return time + conv + R.grav * R.Arn[k] - R.f[k];
  }
  const T *vis = L.visn, *rn = L.rhon;
  T dvl = dl + (b[k] - b[k - t]) * L.ih;
  T dvr = dr + (b[k + s] - b[k + s - t]) * L.ih;
  T press = (L.p[k + s] - L.p[k]) * L.ih * P.iM;
  T st = -(rn[k + s] * L.mu[k] + rn[k] * L.mu[k + s]) * R.Tf[k] * P.iM;
  T vl = vis[k], vr = vis[k + s];
  T visc = -P.iRe * L.ih * ((vr * dr - vl * dl) + (L.Av[k] * Dp - L.Av[k - t] * Dm) +
                            (vr * dvr - vl * dvl) * T(1.0 / 3.0));
  return press + st + visc;
}

// Vanka block of cell (i,j) by a team of eight lanes (FP64 full iterate): as
// vanka_team, with each momentum row's residual split over the lane pair
// (q, q + 4) (mom_residual_half) and summed by one shuffle, so that each lane
// evaluates half a row.  Both halves of the team then run the same solve;
// the lower half stores.  For levels whose colour leaves most of the GPU idle:
// the visit's chain of dependent instructions is what bounds them.
template <typename T>
__device__ __forceinline__ void vanka_team8(const Prm<T>& P, const Lv<T>& L, int i, int j, bool ok,
                                            T omega) {
  const int W = L.pitch;
  const int q = threadIdx.x & 3, d = q >> 1, half = (threadIdx.x >> 2) & 1;
  const T ih = L.ih, ih2 = L.ih2;
  int k = L.at(i, j);
  int eW = (L.px && i == 1) ? L.m1 : i - 1;
  int kW = L.at(eW, j);
  bool a0 = L.px || i > 1, a1 = L.px || i < L.m1, a2 = j > 1, a3 = j < L.m2;
  bool mine = q == 0 ? a0 : q == 1 ? a1 : q == 2 ? a2 : a3;
  int ke = q == 0 ? kW : (q == 2 ? k - W : k);
  MomRow<T> R = mom_row<T, FullForm>(P, L, d);
  T rl = L.rhoc[ke], rr = L.rhoc[ke + R.s];
  T dq = R.Dg[ke] + T(0.5) * P.idt * (T(0.5) * (rl + rr));
  T bq = mom_residual_half<T>(P, L, R, ke, rl, rr, half);
  bq += __shfl_xor_sync(0xffffffffu, bq, 4);
  if (!mine) bq = T(0);
  const T* mob = L.mobn;
  const int nq = k + (q == 0 ? -1 : q == 1 ? 1 : q == 2 ? -W : W);
  T am = mob[nq] + mob[k];
  T f0 = team_sum<T>((q & 1) ? (d ? L.v[k] : L.u[k]) : -(d ? L.v[k - W] : L.u[k - 1]));
  T f1 = team_sum<T>(T(0.5) * am * ((L.mu[nq] - L.mu[k]) + P.alpha * (L.p[nq] - L.p[k])));
  T f2 = team_sum<T>(mine ? am : T(0));
  T A44 = T(0.5) * P.alpha * P.alpha * P.iPe * f2 * ih2;
  T b4 = f0 * ih - P.alpha * P.iPe * ih2 * f1 - L.fp[k];
  TeamSolve<T> ts(P, L, q, dq, d ? a2 : a0, d ? a3 : a1, d ? L.Sy[k] : L.Sx[k], L.visn[k], A44);
  T pr;
  T x = ts.apply(bq, b4, pr);
  if (!ok || half) return;
  if (mine) {
    if (q == 0) store_u(L, eW, j, L.u[kW] - omega * x);
    else if (q == 1) store_u(L, i, j, L.u[k] - omega * x);
    else if (q == 2) store_v(L, i, j - 1, L.v[k - W] - omega * x);
    else store_v(L, i, j, L.v[k] - omega * x);
  }
  if (q == 0) store_cell(L, L.p, i, j, L.p[k] - omega * pr);
}

// The projection method's 4x4 intermediate-velocity block (vanka4_cell) by a
// team of four lanes: lane q builds row q (team_row without pressure, surface
// tension and gravity) and the team solves the block (TeamSolve without the
// pressure row); lane q writes edge q.
template <typename T>
__device__ __forceinline__ void vanka4_team(const Prm<T>& P, const Lv<T>& L, int i, int j, bool ok,
                                            T omega) {
  const int W = L.pitch;
  const int q = threadIdx.x & 3, d = q >> 1;
  int k = L.at(i, j);
  int eW = (L.px && i == 1) ? L.m1 : i - 1;
  int kW = L.at(eW, j);
  bool a0 = L.px || i > 1, a1 = L.px || i < L.m1, a2 = j > 1, a3 = j < L.m2;
  bool mine = q == 0 ? a0 : q == 1 ? a1 : q == 2 ? a2 : a3;
  int ke = q == 0 ? kW : (q == 2 ? k - W : k);
  T dq, bq;
  team_row<T, ProjForm>(P, L, i, j, d, ke, mine, dq, bq);
  TeamSolve<T> ts(P, L, q, dq, d ? a2 : a0, d ? a3 : a1, d ? L.Sy[k] : L.Sx[k], L.visn[k], T(0), false);
  T pr;
  T x = ts.apply(bq, T(0), pr);
  if (!ok || !mine) return;
  if (q == 0) store_u(L, eW, j, L.u[kW] - omega * x);
  else if (q == 1) store_u(L, i, j, L.u[k] - omega * x);
  else if (q == 2) store_v(L, i, j - 1, L.v[k - W] - omega * x);
  else store_v(L, i, j, L.v[k] - omega * x);
}

// Coupled 7x7 block of coupled_cell by a team of four lanes (lane & 3 = q:
// edge and face W, E, S, N).  Lane q builds momentum row q, face q's terms of
// the mass row, of N_c, N_mu and of the CH Jacobian's face sums, and the
// couplings of edge q; butterflies add the face terms and every lane forms
// the cell terms.  The solve follows solve_coupled7: the NS block's
// structured solve (TeamSolve) applied to three right-hand sides, then the
// 2x2 Schur system for (dc, dmu).  Lane q writes edge q, lane 0 c, mu, p.
template <typename T, class Form>
__device__ __forceinline__ void coupled_team(const Prm<T>& P, const Lv<T>& L, int i, int j, bool ok,
                                             T omega) {
  const int W = L.pitch;
  const int q = threadIdx.x & 3, d = q >> 1;
  const T ih = L.ih, ih2 = L.ih2;
  int k = L.at(i, j);
  int eW = (L.px && i == 1) ? L.m1 : i - 1;
  int kW = L.at(eW, j);
  bool a0 = L.px || i > 1, a1 = L.px || i < L.m1, a2 = j > 1, a3 = j < L.m2;
  bool mine = q == 0 ? a0 : q == 1 ? a1 : q == 2 ? a2 : a3;
  int ke = q == 0 ? kW : (q == 2 ? k - W : k);
  T dq, bq;
  team_row<T, Form>(P, L, i, j, d, ke, mine, dq, bq);
  ChRows<T> C = ch_team_rows<T, Form>(P, L, i, j, q, mine);
  T sdiv = team_sum<T>((q & 1) ? (d ? L.v[k] : L.u[k]) : -(d ? L.v[k - W] : L.u[k - 1]));
  T sm = C.sm, sflux = C.sflux, gq = C.gq;
  T J11 = C.J11, J12 = C.J12, J21 = C.J21, J22 = C.J22, Rc = C.Rc, Rm = C.Rm;
  // the mass row and the couplings of edge q: d N_q/dc, d N_q/dmu (rows of
  // the two CH columns), d N_c/d x_q = g_q (the CH row), d N_p/dmu = d N_c/dp
  T A44 = T(0.5) * P.alpha * P.alpha * P.iPe * sm * ih2;
  T b4 = sdiv * ih - P.alpha * P.iPe * ih2 * sflux - L.fp[k];
  T diffc = T(0.5) * P.alpha * P.iPe * sm * ih2;
  T gm = mine ? gq : T(0);
  T cq0 = mine ? T(0.25) * C.drho * P.idt * (d ? Form::val_v(L, ke) : Form::val_u(L, ke)) : T(0);
  T cq1 = mine ? -gq * P.iM : T(0);
  TeamSolve<T> ts(P, L, q, dq, d ? a2 : a0, d ? a3 : a1, d ? L.Sy[k] : L.Sx[k], L.visn[k], A44);
  T p0, p1, p2;
  T x0 = ts.apply(bq, b4, p0);
  T x1 = ts.apply(cq0, T(0), p1);
  T x2 = ts.apply(cq1, diffc, p2);
  T S00 = J11 - (team_sum<T>(gm * x1) + diffc * p1);
  T S01 = J12 - (team_sum<T>(gm * x2) + diffc * p2);
  T rhs0 = Rc - (team_sum<T>(gm * x0) + diffc * p0);
  T id2 = qrcp(S00 * J22 - S01 * J21);
  T dc = (J22 * rhs0 - S01 * Rm) * id2;
  T dm = (S00 * Rm - J21 * rhs0) * id2;
  T x = x0 - x1 * dc - x2 * dm;
  T pr = p0 - p1 * dc - p2 * dm;
  if (!ok) return;
  if (mine) {
    if (q == 0) store_u(L, eW, j, L.u[kW] - omega * x);
    else if (q == 1) store_u(L, i, j, L.u[k] - omega * x);
    else if (q == 2) store_v(L, i, j - 1, L.v[k - W] - omega * x);
    else store_v(L, i, j, L.v[k] - omega * x);
  }
  if (q == 0) {
    T cnew = L.c[k] - omega * dc;
    store_cell(L, L.c, i, j, cnew);
    if constexpr (!std::is_same<Form, ErrForm>::value) store_cell(L, L.rhoc, i, j, rho_of(P, cnew));
    store_cell(L, L.mu, i, j, L.mu[k] - omega * dm);
    store_cell(L, L.p, i, j, L.p[k] - omega * pr);
  }
}

// Per-level launch with four lanes per Vanka block (vanka_team): a level whose
// colour leaves most SM sub-partitions idle runs each block's critical path
// split over four lanes.  Whole warps past the last team return together, so
// every warp that calls vanka_team has all 32 lanes in it.
template <typename T>
__global__ void __launch_bounds__(SNT) k_vanka4_team(Prm<T> P, Lv<T> L, int colour, T omega) {
  pdl_enter();
  ColourSlots cs = vanka_slots(L, colour);
  int t = blockIdx.x * SNT + threadIdx.x;
  if ((t & ~31) >= 4 * cs.n) return;  // warp-uniform
  int i = 1, j = 1;
  bool ok = (t >> 2) < cs.n && vanka_slot_cell(L, colour, cs, t >> 2, i, j);
  if (!ok) i = j = 1;
  vanka4_team<T>(P, L, i, j, ok, omega);
}

template <typename T, class Form>
__global__ void __launch_bounds__(SNT) k_coupled_team(Prm<T> P, Lv<T> L, int colour, T omega) {
  pdl_enter();
  ColourSlots cs = vanka_slots(L, colour);
  int t = blockIdx.x * SNT + threadIdx.x;
  if ((t & ~31) >= 4 * cs.n) return;  // warp-uniform
  int i = 1, j = 1;
  bool ok = (t >> 2) < cs.n && vanka_slot_cell(L, colour, cs, t >> 2, i, j);
  if (!ok) i = j = 1;
  coupled_team<T, Form>(P, L, i, j, ok, omega);
}

// per-level launch with eight lanes per Vanka block (vanka_team8; FP64 full
// iterate)
__global__ void __launch_bounds__(SNT) k_vanka_team8(Prm<double> P, Lv<double> L, int colour,
                                                     double omega) {
  pdl_enter();
  ColourSlots cs = vanka_slots(L, colour);
  int t = blockIdx.x * SNT + threadIdx.x;
  if ((t & ~31) >= 8 * cs.n) return;  // warp-uniform
  int i = 1, j = 1;
  bool ok = (t >> 3) < cs.n && vanka_slot_cell(L, colour, cs, t >> 3, i, j);
  if (!ok) i = j = 1;
  vanka_team8<double>(P, L, i, j, ok, omega);
}

template <typename T, class Form>
__global__ void __launch_bounds__(SNT) k_vanka_team(Prm<T> P, Lv<T> L, int colour, T omega) {
  pdl_enter();
  ColourSlots cs = vanka_slots(L, colour);
  int t = blockIdx.x * SNT + threadIdx.x;
  if ((t & ~31) >= 4 * cs.n) return;  // warp-uniform
  int i = 1, j = 1;
  bool ok = (t >> 2) < cs.n && vanka_slot_cell(L, colour, cs, t >> 2, i, j);
  if (!ok) i = j = 1;
  vanka_team<T, Form>(P, L, i, j, ok, omega);
}

// Vanka block of cell (i,j) by a lane pair (FP64 full iterate; lane & 1 = d):
// lane 0 holds the x pair of the block (rows W, E), lane 1 the y pair (S, N).
// Each lane builds its two momentum rows (team_row) and its two faces of the
// mass row; one shuffle adds the faces.  The structured solve of solve_vanka
// then runs with each lane factoring only its own pair's 2x2 block B: s = w.z
// and t = w.y are the sums of the two pairs' shares, one shuffle each, and
// g, p and the pressure pivot are formed on both lanes alike.  Every sum is
// associated as in the four-lane team ((W + E) + (S + N)), so the arithmetic
// is the team's.  Against one lane per visit this halves each lane's FP64
// instructions, which is what bounds a launch whose colour fills the GPU
// more than once: the busiest sub-partition issues three warps of half a
// visit instead of two warps of a whole one.
template <typename T, class Form>
__device__ __forceinline__ void vanka_pair(const Prm<T>& P, const Lv<T>& L, int i, int j, bool ok,
                                           T omega) {
  const unsigned FULL = 0xffffffffu;
  const int W = L.pitch;
  const int d = threadIdx.x & 1;
  const T ih = L.ih, ih2 = L.ih2;
  int k = L.at(i, j);
  int eW = (L.px && i == 1) ? L.m1 : i - 1;
  int kW = L.at(eW, j);
  bool a0 = L.px || i > 1, a1 = L.px || i < L.m1, a2 = j > 1, a3 = j < L.m2;
  // this lane's edges: the low one (W or S) and the high one (E or N)
  bool ap0 = d ? a2 : a0, ap1 = d ? a3 : a1;
  int ke0 = d ? k - W : kW;
  T dq0, bq0, dq1, bq1;
  team_row<T, Form>(P, L, i, j, d, ke0, ap0, dq0, bq0);
  team_row<T, Form>(P, L, i, j, d, k, ap1, dq1, bq1);
  // the mass row by faces (as vanka_team): faces W, E on lane 0, S, N on lane 1
  const T* mob = L.mobn;
  const int off = d ? W : 1;
  const int n0 = k - off, n1 = k + off;
  T am0 = mob[n0] + mob[k], am1 = mob[n1] + mob[k];
  T fs0 = -(d ? L.v[k - W] : L.u[k - 1]) + (d ? L.v[k] : L.u[k]);
  T fs1 = T(0.5) * am0 * ((L.mu[n0] - L.mu[k]) + P.alpha * (L.p[n0] - L.p[k])) +
          T(0.5) * am1 * ((L.mu[n1] - L.mu[k]) + P.alpha * (L.p[n1] - L.p[k]));
  T fs2 = (ap0 ? am0 : T(0)) + (ap1 ? am1 : T(0));
  fs0 += __shfl_xor_sync(FULL, fs0, 1);
  fs1 += __shfl_xor_sync(FULL, fs1, 1);
  fs2 += __shfl_xor_sync(FULL, fs2, 1);
  T A44 = T(0.5) * P.alpha * P.alpha * P.iPe * fs2 * ih2;
  T b4 = fs0 * ih - P.alpha * P.iPe * ih2 * fs1 - L.fp[k];
  // this pair's block B = A_vv - v3 w w^T (TeamSolve, both rows on one lane)
  T vc = L.visn[k];
  T S = d ? L.Sy[k] : L.Sx[k];
  T v3 = vc * P.iRe * L.ih2 * T(1.0 / 3.0);
  T a = L.ih * P.iM;
  T B00 = ap0 ? dq0 - v3 : T(1);
  T B11 = ap1 ? dq1 - v3 : T(1);
  T B01 = (ap0 && ap1) ? T(0.5) * S * ih - vc * P.iRe * L.ih2 : T(0);
  T B10 = (ap0 && ap1) ? -T(0.5) * S * ih - vc * P.iRe * L.ih2 : T(0);
  T idet = qrcp(B00 * B11 - B01 * B10);
  T z0 = ((ap0 ? B11 : T(0)) + (ap1 ? B01 : T(0))) * idet;
  T z1 = -((ap1 ? B00 : T(0)) + (ap0 ? B10 : T(0))) * idet;
  T sdot = z0 + -z1;
  sdot += __shfl_xor_sync(FULL, sdot, 1);
  T g = qrcp(T(1) + v3 * sdot);
  T iden = qrcp(A44 + ih * a * sdot * g);
  T y0 = (B11 * bq0 - B01 * bq1) * idet;
  T y1 = (B00 * bq1 - B10 * bq0) * idet;
  T tdot = y0 + -y1;
  tdot += __shfl_xor_sync(FULL, tdot, 1);
  T pr = (b4 + ih * tdot * g) * iden;
  T f = g * (v3 * tdot + a * pr);
  T x0 = y0 - z0 * f, x1 = y1 - z1 * f;
  if (!ok) return;
  if (d == 0) {
    if (ap0) store_u(L, eW, j, L.u[kW] - omega * x0);
    if (ap1) store_u(L, i, j, L.u[k] - omega * x1);
    store_cell(L, L.p, i, j, L.p[k] - omega * pr);
  } else {
    if (ap0) store_v(L, i, j - 1, L.v[k - W] - omega * x0);
    if (ap1) store_v(L, i, j, L.v[k] - omega * x1);
  }
}

// per-level launch with a lane pair per Vanka block (vanka_pair; FP64 full
// iterate).  Whole warps past the last pair return together.
template <typename T, class Form>
__global__ void __launch_bounds__(SNT) k_vanka_pair(Prm<T> P, Lv<T> L, int colour, T omega) {
  pdl_enter();
  ColourSlots cs = vanka_slots(L, colour);
  int t = blockIdx.x * SNT + threadIdx.x;
  if ((t & ~31) >= 2 * cs.n) return;  // warp-uniform
  int i = 1, j = 1;
  bool ok = (t >> 1) < cs.n && vanka_slot_cell(L, colour, cs, t >> 1, i, j);
  if (!ok) i = j = 1;
  vanka_pair<T, Form>(P, L, i, j, ok, omega);
}

// per-level launch that splits a colour between one lane per block and lane
// pairs: slots [0, nsingle) one lane each (vanka_cell), the rest a lane pair
// each (vanka_pair), the single-lane warps first.  nsingle is a multiple of
// 32, so both branches are warp-uniform.  For a colour that fills the GPU's
// sub-partitions once and a fraction more (the finest level of the 256x512
// droplet: 820 warps on 608), a full round of single-lane warps followed by a
// round of pair warps for the remainder issues fewer FP64 instructions on the
// busiest sub-partition than a second, mostly empty single-lane round.
template <typename T, class Form>
__global__ void __launch_bounds__(SNT) k_vanka_split(Prm<T> P, Lv<T> L, int colour, T omega,
                                                     int nsingle) {
  pdl_enter();
  ColourSlots cs = vanka_slots(L, colour);
  int t = blockIdx.x * SNT + threadIdx.x;
  if (t < nsingle) {
    int i, j;
    if (t < cs.n && vanka_slot_cell(L, colour, cs, t, i, j)) vanka_cell<T, Form>(P, L, i, j, omega);
    return;
  }
  int u = t - nsingle;
  if ((u & ~31) >= 2 * (cs.n - nsingle)) return;  // warp-uniform
  int sl = nsingle + (u >> 1), i = 1, j = 1;
  bool ok = sl < cs.n && vanka_slot_cell(L, colour, cs, sl, i, j);
  if (!ok) i = j = 1;
  vanka_pair<T, Form>(P, L, i, j, ok, omega);
}

// teams of four lanes while the colour fits in four warps per block of the
// fused group (one warp per sub-partition)
constexpr int QN_TEAM_MAX_SLOTS = 32;

template <typename T, class Form>
__device__ void smooth_block(const Prm<T>& P, const Lv<T>& L, T omega, int coupled, int team8 = 0) {
  const int kcol = L.kcol;
  if constexpr (std::is_same<Form, ProjForm>::value) {
    // projection method (Sec. 7.2): CH red-black, intermediate-velocity blocks
    // over the Vanka colours, pressure Gauss-Seidel red-black
    const int mpr = (L.m1 + 1) / 2;
    // four lanes per cell while a colour fits the block in one pass
    const bool cteam = 4 * mpr * L.m2 <= grp_size();
    for (int col = 0; col < 2; ++col) {
      if (cteam) {
        int t = grp_rank(), sl = t >> 2, j = 1, i = 1;
        bool ok = false;
        if (sl < mpr * L.m2) {
          j = sl / mpr + 1;
          i = (((col - j) & 1) ? 1 : 2) + 2 * (sl % mpr);
          ok = i <= L.m1;
        }
        if (!ok) i = j = 1;
        if ((t & ~31) < 4 * mpr * L.m2) ch_team<T, Form>(P, L, i, j, ok);  // warp-uniform
      } else {
        for (int t = grp_rank(); t < mpr * L.m2; t += grp_size()) {
          int j = t / mpr + 1;
          int i = (((col - j) & 1) ? 1 : 2) + 2 * (t % mpr);
          if (i <= L.m1) ch_cell<T, Form>(P, L, i, j);
        }
      }
      grp_sync();
    }
    for (int col = 0; col < kcol; ++col) {
      ColourSlots cs = vanka_slots(L, col);
      if (sizeof(T) == 8 && cs.n <= QN_TEAM_MAX_SLOTS * (int)gridDim.x) {  // one warp per sub-partition
        int t = grp_rank();
        if ((t & ~31) < 4 * cs.n) {  // warp-uniform: the warp holds at least one team
          int i = 1, j = 1;
          bool ok = (t >> 2) < cs.n && vanka_slot_cell(L, col, cs, t >> 2, i, j);
          if (!ok) i = j = 1;
          vanka4_team<T>(P, L, i, j, ok, omega);
        }
      } else {
        for (int t = grp_rank(); t < cs.n; t += grp_size()) {
          int i, j;
          if (vanka_slot_cell(L, col, cs, t, i, j)) vanka4_cell<T, Form>(P, L, i, j, omega);
        }
      }
      grp_sync();
    }
    for (int col = 0; col < 2; ++col) {
      if (cteam) {
        int t = grp_rank(), sl = t >> 2, j = 1, i = 1;
        bool ok = false;
        if (sl < mpr * L.m2) {
          j = sl / mpr + 1;
          i = (((col - j) & 1) ? 1 : 2) + 2 * (sl % mpr);
          ok = i <= L.m1;
        }
        if (!ok) i = j = 1;
        if ((t & ~31) < 4 * mpr * L.m2) pgs_team<T>(P, L, i, j, ok);  // warp-uniform
      } else {
        for (int t = grp_rank(); t < mpr * L.m2; t += grp_size()) {
          int j = t / mpr + 1;
          int i = (((col - j) & 1) ? 1 : 2) + 2 * (t % mpr);
          if (i <= L.m1) pgs_cell<T>(P, L, i, j);
        }
      }
      grp_sync();
    }
  } else {  // primitive method (full iterate or error equation)
  if (coupled) {
    for (int col = 0; col < kcol; ++col) {
      ColourSlots cs = vanka_slots(L, col);
      // four lanes per block while the colour fits the block in one pass
      if (4 * cs.n <= grp_size()) {
        int t = grp_rank();
        if ((t & ~31) < 4 * cs.n) {  // warp-uniform: the warp holds at least one team
          int i = 1, j = 1;
          bool ok = (t >> 2) < cs.n && vanka_slot_cell(L, col, cs, t >> 2, i, j);
          if (!ok) i = j = 1;
          coupled_team<T, Form>(P, L, i, j, ok, omega);
        }
      } else {
        for (int t = grp_rank(); t < cs.n; t += grp_size()) {
          int i, j;
          if (vanka_slot_cell(L, col, cs, t, i, j)) coupled_cell<T, Form>(P, L, i, j, omega);
        }
      }
      grp_sync();
    }
    return;
  }
  const int mpr = (L.m1 + 1) / 2;
  constexpr bool team_ok = std::is_same<Form, FullForm>::value && sizeof(T) == 8;
  constexpr bool vteam_ok = team_ok || std::is_same<Form, ErrForm>::value;
  for (int col = 0; col < 2; ++col) {
    if (vteam_ok && 4 * mpr * L.m2 <= grp_size()) {
      int t = grp_rank();
      if ((t & ~31) < 4 * mpr * L.m2) {  // warp-uniform
        int sl = t >> 2, j = 1, i = 1;
        bool ok = false;
        if (sl < mpr * L.m2) {
          j = sl / mpr + 1;
          i = (((col - j) & 1) ? 1 : 2) + 2 * (sl % mpr);
          ok = i <= L.m1;
        }
        if (!ok) i = j = 1;
        ch_team<T, Form>(P, L, i, j, ok);
      }
    } else {
      for (int t = grp_rank(); t < mpr * L.m2; t += grp_size()) {
        int j = t / mpr + 1;
        int i = (((col - j) & 1) ? 1 : 2) + 2 * (t % mpr);
        if (i <= L.m1) ch_cell<T, Form>(P, L, i, j);
      }
    }
    grp_sync();
  }
  for (int col = 0; col < kcol; ++col) {
    ColourSlots cs = vanka_slots(L, col);
    // FP64: while the colour fits one warp per sub-partition of the group; the
    // latency-bound FP32 error levels: while it fits the group in one pass
    const int team_slots = team_ok ? QN_TEAM_MAX_SLOTS * (int)gridDim.x : grp_size() / 4;
    if (team_ok && team8 && 8 * cs.n <= grp_size()) {  // eight lanes per block
      int t = grp_rank();
      if ((t & ~31) < 8 * cs.n) {  // warp-uniform: the warp holds at least one team
        int i = 1, j = 1;
        bool ok = (t >> 3) < cs.n && vanka_slot_cell(L, col, cs, t >> 3, i, j);
        if (!ok) i = j = 1;
        if constexpr (team_ok) vanka_team8<double>(P, L, i, j, ok, omega);
      }
    } else if (vteam_ok && cs.n <= team_slots) {
      int t = grp_rank();
      if ((t & ~31) < 4 * cs.n) {  // warp-uniform: the warp holds at least one team
        int i = 1, j = 1;
        bool ok = (t >> 2) < cs.n && vanka_slot_cell(L, col, cs, t >> 2, i, j);
        if (!ok) i = j = 1;
        vanka_team<T, Form>(P, L, i, j, ok, omega);
      }
    } else {
      for (int t = grp_rank(); t < cs.n; t += grp_size()) {
        int i, j;
        if (vanka_slot_cell(L, col, cs, t, i, j)) vanka_cell<T, Form>(P, L, i, j, omega);
      }
    }
    grp_sync();
  }
  }  // primitive method
}

template <typename T, class Form>
__device__ __forceinline__ void coarse_vcycle_body(const Prm<T>& P, const CoarseLevels<T>& C, int nu1,
                                                   int nu2, int nuc, T omega, int coupled,
                                                   int team8) {
  const int n = C.n;
  double dummy[10];
  if (C.base) {
    for (int l = 1; l < n; ++l) {
      const Lv<T>& F = C.L[l - 1];
      const Lv<T>& G = C.L[l];
      for (int t = grp_rank(); t < (G.m1 + 1) * (G.m2 + 1); t += grp_size())
        restrict_base_cell(F, G, t % (G.m1 + 1), t / (G.m1 + 1));
      grp_sync();
      const int nf = 4 * (G.m1 + 3) + 4 * (G.m2 + 3);
      for (int t = grp_rank(); t < nf; t += grp_size()) {
        int I, J;
        if (frame_pos(t, G.m1, G.m2, I, J)) bc_base_cell(G, I, J);
      }
      grp_sync();
    }
  }
  for (int l = 0; l < n - 1; ++l) {
    const Lv<T>& F = C.L[l];
    const Lv<T>& G = C.L[l + 1];
    for (int s = 0; s < nu1; ++s) smooth_block<T, Form>(P, F, omega, coupled, team8);
    for (int t = grp_rank(); t < F.m1 * F.m2; t += grp_size())
      residual_cell<T, 0, Form>(P, F, t % F.m1 + 1, t / F.m1 + 1, dummy);
    grp_sync();
    for (int t = grp_rank(); t < (G.m1 + 1) * (G.m2 + 1); t += grp_size())
      restrict_state_cell(P, F, G, t % (G.m1 + 1), t / (G.m1 + 1));
    grp_sync();
    bc_unknowns_block(G);
    for (int t = grp_rank(); t < G.m1 * G.m2; t += grp_size())
      restrict_res_cell(F, G, t % G.m1 + 1, t / G.m1 + 1);
    grp_sync();
    for (int t = grp_rank(); t < G.m1 * G.m2; t += grp_size())
      residual_cell<T, 1, Form>(P, G, t % G.m1 + 1, t / G.m1 + 1, dummy);
    grp_sync();
  }
  for (int s = 0; s < nuc; ++s) smooth_block<T, Form>(P, C.L[n - 1], omega, coupled, team8);
  for (int l = n - 2; l >= 0; --l) {
    const Lv<T>& F = C.L[l];
    const Lv<T>& G = C.L[l + 1];
    for (int t = grp_rank(); t < F.m1 * F.m2; t += grp_size())
      prolong_cell(P, F, G, t % F.m1 + 1, t / F.m1 + 1);
    grp_sync();
    bc_unknowns_block(F);
    for (int s = 0; s < nu2; ++s) smooth_block<T, Form>(P, F, omega, coupled, team8);
  }
}

template <typename T, class Form, int NT>
__global__ void __launch_bounds__(NT) k_coarse_vcycle(Prm<T> P, CoarseLevels<T> C, int nu1, int nu2,
                                                      int nuc, int kcol, T omega, int coupled,
                                                      int team8) {
  pdl_enter();
  coarse_vcycle_body<T, Form>(P, C, nu1, nu2, nuc, omega, coupled, team8);
}

// --------------------------------------------------------------------------
// The fused V-cycle of the FP64 full-iterate levels on a shared-memory copy.
// Its colour steps are chains of dependent loads and FP64 instructions of one
// visit each; from shared memory the loads take tens of cycles instead of an
// L2 round trip.  The block copies every array of its levels (QN_LV_ARRAYS,
// the padded frame [-1, m1+1] x [-1, m2+1] that the device code reads and
// writes) into shared memory at the compact pitch m1 + 3, runs the V-cycle
// body unchanged on level descriptors that point into the copy, and writes
// back the arrays the V-cycle writes: the unknowns, sources, residuals and the
// kept restricted iterate (the first 20 arrays) and rho(c).  Same device code
// on the same values: the results are those of k_coarse_vcycle.
// --------------------------------------------------------------------------
constexpr int QN_LV_NARR = 59;     // arrays of QN_LV_ARRAYS
constexpr int QN_LV_WRITTEN = 20;  // arrays 0..19 are written; and rho(c):
constexpr int QN_LV_RHOC = 44;

struct CoarseSmem {
  int off[QN_MAX_FUSED_LEVELS];  // first element of level l's copy
  long long ng[QN_MAX_FUSED_LEVELS];  // elements per array in the global block
  int head;  // elements (doubles) before the first copy: the descriptors
};

// copy arrays [q0, q1) of one level between its global block (pitch pg, ng
// elements per array) and its compact copy (pitch cc, rr rows).  Thread t
// takes column t % cw (cw >= cc) of rows t / cw + k NT / cw.  IN: global to
// shared by asynchronous copies (cp.async, 8 bytes each, all of a thread's in
// flight at once; the caller waits for them with cp.async.wait_all); else
// shared to global by plain stores.
template <int NT, bool IN>
__device__ __forceinline__ void coarse_copy(double* __restrict__ g, int pg, long long ng,
                                            double* __restrict__ sh, int cc, int rr, int q0,
                                            int q1) {
  const int cw = cc <= 16 ? 16 : 32, tx = threadIdx.x % cw, rstep = NT / cw;
  if (tx >= cc) return;
  const int ns = cc * rr;
  for (int r = threadIdx.x / cw; r < rr; r += rstep) {
    double* __restrict__ gr = g + (long long)r * pg + tx;
    double* __restrict__ sr = sh + r * cc + tx;
#pragma unroll 8
    for (int q = q0; q < q1; ++q) {
      if (IN) {
        const unsigned sa = (unsigned)__cvta_generic_to_shared(sr + q * ns);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gr + q * ng)
                     : "memory");
      } else {
        gr[q * ng] = sr[q * ns];
      }
    }
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_coarse_vcycle_smem(Prm<double> P, CoarseLevels<double> C,
                                                           CoarseSmem M, int nu1, int nu2, int nuc,
                                                           double omega, int coupled, int team8) {
  extern __shared__ __align__(16) double qn_coarse_smem[];
  pdl_enter();
  CoarseLevels<double>* S = reinterpret_cast<CoarseLevels<double>*>(qn_coarse_smem);
  double* arr = qn_coarse_smem + M.head;
  const int n = C.n;
  for (int l = 0; l < n; ++l) {
    const Lv<double>& G = C.L[l];
    const int cc = G.m1 + 3, rr = G.m2 + 3;
    coarse_copy<NT, true>(G.c - (G.pitch + 1), G.pitch, M.ng[l], arr + M.off[l], cc, rr, 0,
                          QN_LV_NARR);
  }
  if (threadIdx.x < n) {  // the descriptor of level l, its arrays in the copy
    const int l = threadIdx.x;
    Lv<double> X = C.L[l];
    const int cc = X.m1 + 3, ns = cc * (X.m2 + 3);
    double* o = arr + M.off[l] + cc + 1;  // origin (0,0) of array 0
    int q = 0;
#define QN_REBASE(m) X.m = o + (q++) * ns;
    QN_LV_ARRAYS(QN_REBASE)
#undef QN_REBASE
    X.pitch = cc;
    S->L[l] = X;
  }
  if (threadIdx.x == 0) {
    S->n = n;
    S->base = 0;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  coarse_vcycle_body<double, FullForm>(P, *S, nu1, nu2, nuc, omega, coupled, team8);
  __syncthreads();
  for (int l = 0; l < n; ++l) {
    const Lv<double>& G = C.L[l];
    const int cc = G.m1 + 3, rr = G.m2 + 3;
    double* g = G.c - (G.pitch + 1);
    coarse_copy<NT, false>(g, G.pitch, M.ng[l], arr + M.off[l], cc, rr, 0, QN_LV_WRITTEN);
    coarse_copy<NT, false>(g, G.pitch, M.ng[l], arr + M.off[l], cc, rr, QN_LV_RHOC, QN_LV_RHOC + 1);
  }
}

// --------------------------------------------------------------------------
// banded wavefront of smoothing passes (one launch for nu smoothing steps on a
// level).  A smoothing step is a sequence of passes: CH red, CH black, then the
// Vanka colours (or the coupled block's colours).  Every visit reads and
// writes rows within 2 of its own, so with bands of at least 4 rows pass k on
// band b depends only on pass k - 1 on bands b - 1, b, b + 1.  Tickets are
// handed out in the order of t = b + 2k (then k), a topological order: a
// block takes a ticket, waits until each neighbouring band has finished pass
// k - 1 (per-band counters of finished passes), runs the pass's visits on its
// band and publishes the band's new count.  Each visit sees exactly the
// values it sees when every pass is a launch over the whole level and runs the
// same device code, so the results are those of the per-colour launches up to
// the compiler's contraction of multiply-adds, which may differ between the
// two kernels; what changes is that a band's arrays stay in L2 across its
// passes instead of every colour launch streaming the whole level.
// A ticket's dependencies hold earlier tickets, taken by blocks that are
// running or done, so the wavefront progresses whatever the number of
// resident blocks.  Waits are bounded: past `budget` SM cycles a wait sets
// *flag (the step then fails with QNSCH_ETIMEOUT) and every later wait
// returns at once.
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// the visits of pass `pass` on rows r0..r1 (1-based, inclusive)
template <typename T, class Form>
__device__ __forceinline__ void wave_pass(const Prm<T>& P, const Lv<T>& L, const WavePlan& W,
                                          int pass, int r0, int r1, T omega) {
  const int per = W.coupled ? L.kcol : L.kcol + 2;
  const int q = pass % per;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (!W.coupled && q < 2) {  // CH colour q: packed as in k_ch
    const int mpr = (L.m1 + 1) / 2;
    const int t_lo = (r0 - 1) * mpr, t_hi = r1 * mpr;
    if (mpr * L.m2 <= W.ch_team_max) {
      for (int base = t_lo; base < t_hi; base += nt / 4) {
        if (base + ((tid & ~31) >> 2) >= t_hi) continue;  // warp-uniform
        int t = base + (tid >> 2), i = 1, j = 1;
        bool ok = t < t_hi;
        if (ok) {
          j = t / mpr + 1;
          i = (((q - j) & 1) ? 1 : 2) + 2 * (t % mpr);
          ok = i <= L.m1;
        }
        if (!ok) i = j = 1;
        ch_team<T, Form>(P, L, i, j, ok);
      }
    } else {
      for (int t = t_lo + tid; t < t_hi; t += nt) {
        int j = t / mpr + 1;
        int i = (((q - j) & 1) ? 1 : 2) + 2 * (t % mpr);
        if (i <= L.m1) ch_cell<T, Form>(P, L, i, j);
      }
    }
    return;
  }
  const int col = W.coupled ? q : q - 2;
  ColourSlots cs = vanka_slots(L, col);
  // the slots whose row j0 + rstep * (t / mpr) lies in [r0, r1]
  if (r1 < cs.j0) return;
  const int qlo = r0 > cs.j0 ? (r0 - cs.j0 + cs.rstep - 1) / cs.rstep : 0;
  const int qhi = (r1 - cs.j0) / cs.rstep;
  const int t_lo = qlo * cs.mpr, t_hi = min((qhi + 1) * cs.mpr, cs.n);
  if (cs.n <= W.vanka_team_max) {
    for (int base = t_lo; base < t_hi; base += nt / 4) {
      if (base + ((tid & ~31) >> 2) >= t_hi) continue;  // warp-uniform
      int t = base + (tid >> 2), i = 1, j = 1;
      bool ok = t < t_hi && vanka_slot_cell(L, col, cs, t, i, j);
      if (!ok) i = j = 1;
      if (W.coupled) coupled_team<T, Form>(P, L, i, j, ok, omega);
      else vanka_team<T, Form>(P, L, i, j, ok, omega);
    }
  } else {
    for (int t = t_lo + tid; t < t_hi; t += nt) {
      int i, j;
      if (!vanka_slot_cell(L, col, cs, t, i, j)) continue;
      if (W.coupled) coupled_cell<T, Form>(P, L, i, j, omega);
      else vanka_cell<T, Form>(P, L, i, j, omega);
    }
  }
}

constexpr int WAVE_NT = 256;

template <typename T, class Form>
__global__ void __launch_bounds__(WAVE_NT) k_wave(Prm<T> P, Lv<T> L, WavePlan W, T omega,
                                                  unsigned* ctr, double* flag) {
  pdl_enter();
  __shared__ unsigned s_t;
  unsigned* done = ctr + 1;
  const int N = W.nbands, K = W.npass;
  // tickets run over the (t = b + 2k, k) grid, t in [0, N + 2K - 2]
  const unsigned tickets = (unsigned)(N + 2 * K - 1) * (unsigned)K;
  for (;;) {
    if (threadIdx.x == 0) s_t = atomicAdd(ctr, 1u);
    __syncthreads();
    const unsigned t = s_t;
    __syncthreads();
    if (t >= tickets) break;
    const int tau = (int)(t / (unsigned)K), k = (int)(t % (unsigned)K), b = tau - 2 * k;
    if (b < 0 || b >= N) continue;  // a ticket of the grid with no band
    if (threadIdx.x == 0 && k > 0) {
      // pass k - 1 done on this band and its neighbours (test hook: one
      // wait for a count that nothing reaches)
      const unsigned need = (W.stall && b == 0 && k == 1) ? 0xffffffffu : (unsigned)k;
      const long long t0 = clock64();
      for (int nb = max(b - 1, 0); nb <= min(b + 1, N - 1); ++nb) {
        while (ld_acquire_u32(done + nb) < need) {
          if (*(volatile double*)flag != 0.0) break;
          if (clock64() - t0 > W.budget) {
            *(volatile double*)flag = 1.0;
            break;
          }
        }
      }
    }
    __syncthreads();
    const int r0 = b * W.rows + 1, r1 = min((b + 1) * W.rows, L.m2);
    wave_pass<T, Form>(P, L, W, k, r0, r1, omega);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release_u32(done + b, (unsigned)(k + 1));
    }
  }
}

// --------------------------------------------------------------------------
// skewed-chunk schedule of the smoothing passes on a large error-equation
// level.  A colour launch over the whole level touches every sector of every
// array its visits read (the visits of one colour are spread over all rows
// and columns), so a level larger than L2 streams from DRAM once per pass.
// Here the passes of a smoothing block run together over chunks of H rows:
// launch d runs pass p on the rows [1 + (d - p) H - 2p, 1 + (d - p + 1) H - 2p)
// (clipped to the level), so each pass trails the one before it by a chunk
// and two rows, and the rows the launch touches stay in L2 between the
// passes.  A visit at row j reads rows j - 2 .. j + 1 and writes rows j - 1
// and j (and the ghost row beside row 1 or row m2), so within one launch no
// task reads or writes what another task writes, every row a task reads
// already holds the results of the earlier passes (they ran in earlier
// launches) and none holds a later pass's: each visit sees the values it sees
// when every pass is a launch over the whole level, with the same device code.
// No block waits for another; stream order orders the launches.
// --------------------------------------------------------------------------
template <typename T, class Form, bool COUPLED>
__global__ void __launch_bounds__(SNT) k_skew(Prm<T> P, Lv<T> L, SkewTasks S, T omega) {
  pdl_enter();
  const int b = blockIdx.x;
  int k = 0;
  while (k + 1 < S.n && S.boff[k + 1] <= b) ++k;
  const int t = S.t_lo[k] + (b - S.boff[k]) * SNT + threadIdx.x;
  if (t >= S.t_hi[k]) return;
  const int q = S.q[k];
  if constexpr (!COUPLED) {
    if (q < 2) {  // CH colour q, slots as in k_ch
      const int mpr = (L.m1 + 1) / 2;
      const int j = t / mpr + 1;
      const int i = (((q - j) & 1) ? 1 : 2) + 2 * (t % mpr);
      if (i <= L.m1) ch_cell<T, Form>(P, L, i, j);
      return;
    }
  }
  const int col = COUPLED ? q : q - 2;
  ColourSlots cs = vanka_slots(L, col);
  int i, j;
  if (!vanka_slot_cell(L, col, cs, t, i, j)) return;
  if constexpr (COUPLED) coupled_cell<T, Form>(P, L, i, j, omega);
  else vanka_cell<T, Form>(P, L, i, j, omega);
}

// --------------------------------------------------------------------------
// the predicted initial iterate of a step (option predictor): a Lagrange
// extrapolation in time of the committed state and the states before it,
// over the whole padded arrays (ghosts are linear in the values they copy,
// so the combination keeps them consistent)
// --------------------------------------------------------------------------
struct FiveArrays {
  double* p[5];
};

__global__ void k_predict(FiveArrays X, FiveArrays A, FiveArrays B, FiveArrays C, double w0,
                          double w1, double w2, long long n, int off) {
  pdl_enter();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int q = blockIdx.y;
  const long long i = t - off;
  X.p[q][i] = w0 * A.p[q][i] + w1 * B.p[q][i] + w2 * C.p[q][i];
}

// --------------------------------------------------------------------------
// defect correction (mixed precision): FP64 level <-> error-equation level
// --------------------------------------------------------------------------
// error-equation frozen data = rounded FP64 frozen data (whole padded arrays)
template <typename T>
__global__ void k_cast_frozen(Lv<double> D, Lv<T> E, long long n, int off) {
  pdl_enter();
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  long long q = t - off;  // origin-relative index
  E.cn[q] = (T)D.cn[q];
  E.un[q] = (T)D.un[q];
  E.vn[q] = (T)D.vn[q];
  E.rhon[q] = (T)D.rhon[q];
  E.mobn[q] = (T)D.mobn[q];
  E.visn[q] = (T)D.visn[q];
  E.Gn[q] = (T)D.Gn[q];
  E.Aru[q] = (T)D.Aru[q];
  E.Arv[q] = (T)D.Arv[q];
  E.Sx[q] = (T)D.Sx[q];
  E.Sy[q] = (T)D.Sy[q];
  E.Qx[q] = (T)D.Qx[q];
  E.Qy[q] = (T)D.Qy[q];
  E.Av[q] = (T)D.Av[q];
  E.Tx[q] = (T)D.Tx[q];
  E.Ty[q] = (T)D.Ty[q];
  E.Dvu[q] = (T)D.Dvu[q];
  E.Dvv[q] = (T)D.Dvv[q];
}

// base X = x (rounded), X.c - c^n formed in FP64, right-hand side = FP64 residual
// (rounded), correction e = 0
template <typename T>
__global__ void k_start_correction(Lv<double> D, Lv<T> E, long long n, int off) {
  pdl_enter();
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  long long q = t - off;
  E.Bc[q] = (T)D.c[q];
  E.Bmu[q] = (T)D.mu[q];
  E.Bu[q] = (T)D.u[q];
  E.Bv[q] = (T)D.v[q];
  E.Bdc[q] = (T)(D.c[q] - D.cn[q]);
  E.fc[q] = (T)D.rc[q];
  E.fmu[q] = (T)D.rmu[q];
  E.fp[q] = (T)D.rp[q];
  E.fu[q] = (T)D.ru[q];
  E.fv[q] = (T)D.rv[q];
  E.c[q] = T(0);
  E.mu[q] = T(0);
  E.p[q] = T(0);
  E.u[q] = T(0);
  E.v[q] = T(0);
}

// x += e on the whole padded arrays (ghost rules are linear, so ghosts stay valid)
template <typename T>
__global__ void k_apply_correction(Prm<double> P, Lv<double> D, Lv<T> E, long long n, int off) {
  pdl_enter();
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  long long q = t - off;
  D.c[q] += (double)E.c[q];
  D.rhoc[q] = rho_of(P, D.c[q]);
  D.mu[q] += (double)E.mu[q];
  D.p[q] += (double)E.p[q];
  D.u[q] += (double)E.u[q];
  D.v[q] += (double)E.v[q];
}

// rho(c) of the iterate over the whole padded array, after c was written in
// bulk (a new step's start, fields set from the host)
__global__ void k_rho_fill(Prm<double> P, Lv<double> L, long long n, int off) {
  pdl_enter();
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  long long q = t - off;
  L.rhoc[q] = rho_of(P, L.c[q]);
}

// coarse base X_H = R X_h (cells: 4-mean; edges: 2 coincident fine edges)
template <typename T>
__global__ void k_restrict_base(Lv<T> F, Lv<T> C) {
  pdl_enter();
  int I = blockIdx.x * BX + threadIdx.x;
  int J = blockIdx.y * BY + threadIdx.y;
  if (I > C.m1 || J > C.m2) return;
  restrict_base_cell(F, C, I, J);
}

template <typename T>
__global__ void k_bc_base(Lv<T> L) {
  pdl_enter();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int I, J;
  if (!frame_pos(t, L.m1, L.m2, I, J)) return;
  bc_base_cell(L, I, J);
}


// --------------------------------------------------------------------------
// reductions
// --------------------------------------------------------------------------
template <typename T>
__global__ void k_sum_p(Lv<T> L, double* part) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x + 1;
  int j = blockIdx.y * BY + threadIdx.y + 1;
  double val[1] = {0.0};
  if (i <= L.m1 && j <= L.m2) val[0] = (double)L.p[L.at(i, j)];
  block_sum_store<1>(val, part, 0);
}

template <typename T>
__global__ void k_sub_mean_p(Lv<T> L, const double* sum, double inv_n) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x;
  int j = blockIdx.y * BY + threadIdx.y;
  if (i > L.m1 + 1 || j > L.m2 + 1) return;
  L.p[L.at(i, j)] -= (T)(sum[0] * inv_n);
}

// mass: sum rho(c), sum rho(c) c over the cells (Thm. 6.1)
template <typename T>
__global__ void k_mass(Prm<T> P, Lv<T> L, const T* c, double* part) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x + 1;
  int j = blockIdx.y * BY + threadIdx.y + 1;
  double val[2] = {0.0, 0.0};
  if (i <= L.m1 && j <= L.m2) {
    double cc = (double)c[L.at(i, j)];
    double r = 1.0 / ((double)P.ia * cc + (double)P.ib);
    val[0] = r;
    val[1] = r * cc;
  }
  block_sum_store<2>(val, part, 0);
}

// --------------------------------------------------------------------------
// diagnostics of the experiments of Sec. 8 (FP64, committed state)
// --------------------------------------------------------------------------
// u_{i+1/2,j} for i = 0..m1 and v_{i,j+1/2} for j = 0..m2: zero on no-slip
// walls, period m1 in x
__device__ __forceinline__ double diag_u(const Lv<double>& L, const double* u, int i, int j) {
  if (!L.px && (i == 0 || i == L.m1)) return 0.0;
  if (L.px && i == 0) i = L.m1;
  return u[L.at(i, j)];
}
__device__ __forceinline__ double diag_v(const Lv<double>& L, const double* v, int i, int j) {
  if (j == 0 || j == L.m2) return 0.0;
  return v[L.at(i, j)];
}
// d_x u + d_y v of cell (i,j)
__device__ __forceinline__ double diag_div(const Lv<double>& L, const double* u, const double* v,
                                           int i, int j) {
  return (diag_u(L, u, i, j) - diag_u(L, u, i - 1, j)) / L.h +
         (diag_v(L, v, i, j) - diag_v(L, v, i, j - 1)) / L.h;
}

// per cell: [0] |div|, [1] max(div, 0), [2] max(-div, 0) (block maxima), then
// the sums [3] c, [4] c a_y(v), [5] c y, [6] div^2
__global__ void k_diag_cells(Lv<double> L, const double* c, const double* u, const double* v,
                             double* part) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x + 1;
  int j = blockIdx.y * BY + threadIdx.y + 1;
  double val[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (i <= L.m1 && j <= L.m2) {
    double d = diag_div(L, u, v, i, j);
    double cc = c[L.at(i, j)];
    double vbar = 0.5 * (diag_v(L, v, i, j) + diag_v(L, v, i, j - 1));
    val[0] = fabs(d);
    val[1] = fmax(d, 0.0);
    val[2] = fmax(-d, 0.0);
    val[3] = cc;
    val[4] = cc * vbar;
    val[5] = cc * ((j - 0.5) * L.h);
    val[6] = d * d;
  }
  block_sum_store<7>(val, part, 3);
}

// one thread per column i: eta_i = h sum_j c_ij and the upward crossings
// c_j >= 1/2 > c_{j+1} (linear between cell centres); [0] highest crossing,
// [1] Ly - lowest crossing (block maxima), then the sums [2] eta_i cos(2 pi
// x_i / Lx) and [3] columns with a crossing
__global__ void __launch_bounds__(NT) k_diag_cols(Lv<double> L, const double* c, double* part) {
  pdl_enter();
  int i = blockIdx.x * NT + threadIdx.x + 1;
  double val[4] = {0.0, 0.0, 0.0, 0.0};
  if (i <= L.m1) {
    const double h = L.h, Ly = L.m2 * h, Lx = L.m1 * h;
    const double pi = 3.14159265358979323846;
    double eta = 0.0, ytop = 0.0, ybot = Ly;
    bool found = false;
    double a = c[L.at(i, 1)];
    eta += a;
    for (int j = 1; j < L.m2; ++j) {
      double b = c[L.at(i, j + 1)];
      eta += b;
      if (a >= 0.5 && b < 0.5) {
        double y = (j - 0.5) * h + h * (a - 0.5) / (a - b);
        if (!found || y > ytop) ytop = y;
        if (!found || y < ybot) ybot = y;
        found = true;
      }
      a = b;
    }
    eta *= h;
    val[2] = eta * cos(2.0 * pi * ((i - 0.5) * h) / Lx);
    if (found) {
      val[0] = ytop;
      val[1] = Ly - ybot;
      val[3] = 1.0;
    }
  }
  block_sum_store<4>(val, part, 2);
}

// divergence field, packed out[(j-1)*m1 + (i-1)]
__global__ void k_div_field(Lv<double> L, const double* u, const double* v, double* out) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x + 1;
  int j = blockIdx.y * BY + threadIdx.y + 1;
  if (i > L.m1 || j > L.m2) return;
  out[(size_t)(j - 1) * L.m1 + (i - 1)] = diag_div(L, u, v, i, j);
}

// energy E_h (Thm. 6.2): per cell rho [a_x(u^2) + a_y(v^2)]/2 + (eps eta/(2We)) rho G(c)
// + (eta/(eps We)) rho F(c) + rho y / Fr; weights passed in w[0..2]
template <typename T>
__global__ void k_energy(Prm<T> P, Lv<T> L, const T* c, const T* u, const T* v, double w_grad,
                         double w_bulk, double w_pot, double* part) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x + 1;
  int j = blockIdx.y * BY + threadIdx.y + 1;
  double val[1] = {0.0};
  if (i <= L.m1 && j <= L.m2) {
    const int W = L.pitch;
    int k = L.at(i, j);
    double cc = (double)c[k];
    double r = 1.0 / ((double)P.ia * cc + (double)P.ib);
    double u0 = u[k], u1 = u[k - 1], v0 = v[k], v1 = v[k - W];
    double kin = 0.25 * (u0 * u0 + u1 * u1 + v0 * v0 + v1 * v1);
    double de = (double)c[k + 1] - cc, dw = cc - (double)c[k - 1];
    double dn = (double)c[k + W] - cc, ds = cc - (double)c[k - W];
    double G = 0.5 * (de * de + dw * dw + dn * dn + ds * ds) / ((double)L.h * (double)L.h);
    double F = 0.25 * cc * cc * (cc - 1.0) * (cc - 1.0);
    double y = (j - 0.5) * (double)L.h;
    val[0] = r * (kin + w_grad * G + w_bulk * F + w_pot * y);
  }
  block_sum_store<1>(val, part, 0);
}

// dissipation of Thm. 6.2 as sums of squares for the iterate against frozen data;
// thread (i,j) with i = 0..m1, j = 0..m2 handles vertex (i+1/2, j+1/2) and, for
// i, j >= 1, cell (i,j) and its east / north faces.  w: [dt/Re, dt/(3Re), dt/(M Pe)]
template <typename T>
__global__ void k_dissipation(Prm<T> P, Lv<T> L, double w_visc, double w_div, double w_ch,
                              double* part) {
  pdl_enter();
  int i = blockIdx.x * BX + threadIdx.x;
  int j = blockIdx.y * BY + threadIdx.y;
  double val[1] = {0.0};
  if (i <= L.m1 && j <= L.m2) {
    const int W = L.pitch;
    const double ih = 1.0 / (double)L.h;
    int k = L.at(i, j);
    double acc = 0.0;
    if (i >= 1 && j >= 1) {
      double rn = L.rhon[k], mv = L.visn[k];
      double du0 = (double)L.u[k] - L.un[k], du1 = (double)L.u[k - 1] - L.un[k - 1];
      double dv0 = (double)L.v[k] - L.vn[k], dv1 = (double)L.v[k - W] - L.vn[k - W];
      acc += 0.5 * rn * 0.5 * (du0 * du0 + du1 * du1 + dv0 * dv0 + dv1 * dv1);
      double dxu = ((double)L.u[k] - L.u[k - 1]) * ih, dyv = ((double)L.v[k] - L.v[k - W]) * ih;
      acc += w_visc * mv * (dxu * dxu + dyv * dyv) + w_div * mv * (dxu + dyv) * (dxu + dyv);
      double alpha = (double)P.alpha;
      double mc = (double)L.mu[k] + alpha * (double)L.p[k];
      if (L.px || i < L.m1) {
        double me = (double)L.mu[k + 1] + alpha * (double)L.p[k + 1];
        acc += w_ch * 0.5 * ((double)L.mobn[k] + L.mobn[k + 1]) * (me - mc) * (me - mc) * ih * ih;
      }
      if (j < L.m2) {
        double mn = (double)L.mu[k + W] + alpha * (double)L.p[k + W];
        acc += w_ch * 0.5 * ((double)L.mobn[k] + L.mobn[k + W]) * (mn - mc) * (mn - mc) * ih * ih;
      }
    }
    if (!L.px || i >= 1) {
      double Av = 0.25 * ((double)L.visn[k] + L.visn[k + 1] + L.visn[k + W] + L.visn[k + W + 1]);
      double Dyu = ((double)L.u[k + W] - L.u[k]) * ih;
      double Dxv = ((double)L.v[k + 1] - L.v[k]) * ih;
      double wy = (j == 0 || j == L.m2) ? 0.5 : 1.0;
      double wx = (!L.px && (i == 0 || i == L.m1)) ? 0.5 : 1.0;
      acc += w_visc * Av * (wy * Dyu * Dyu + wx * Dxv * Dxv);
    }
    val[0] = acc;
  }
  block_sum_store<1>(val, part, 0);
}

// --------------------------------------------------------------------------
// the outer-cycle loop of one step on the device (the step as one CUDA graph:
// a conditional WHILE node repeats the cycle, a conditional IF node commits).
// Control block ctl (doubles): [0] largest family residual r (scaled l2, NaN
// if any family is not finite), [1] cycles done k, [2] consecutive cycles the
// residual grew, [3] stopped by the time limit, [4] stopped by growth,
// [5] commit, [6..10] l2 norms, [11..15] max norms, [16] (as a 64-bit
// integer) the global timer in ns at the start of the step, [17] nonzero once
// a bounded wait of the wavefront smoother has run out.
// --------------------------------------------------------------------------
__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void k_loop_clock(double* ctl) {
  pdl_enter();
  *reinterpret_cast<long long*>(ctl + 16) = global_ns();
}

// nrm: the norms of k_finalize ([0..4] max, [5..9] h^2 sum r^2).  The stopping
// rule is the host loop's: continue while r is finite, r > tol and k < maxcyc;
// stop after `diverge` consecutive cycles of growth; before a further cycle,
// stop as late once the step has run longer than limit_ns.
__global__ void k_loop_ctl(const double* nrm, double* ctl, cudaGraphConditionalHandle hl,
                           cudaGraphConditionalHandle hc, double tol, int maxcyc, int diverge,
                           double limit_ns, int first) {
  pdl_enter();
  double r = 0.0;
  bool nan = false;
  for (int q = 0; q < 5; ++q) {
    double l2 = sqrt(nrm[5 + q]);
    ctl[6 + q] = l2;
    ctl[11 + q] = nrm[q];
    if (!(l2 == l2)) nan = true;
    else if (l2 > r) r = l2;
  }
  if (nan) r = CUDART_NAN;
  double k = 0.0, grew = 0.0;
  if (!first) {
    k = ctl[1] + 1.0;
    grew = r > ctl[0] ? ctl[2] + 1.0 : 0.0;
  }
  const bool div = !first && diverge > 0 && grew >= (double)diverge;
  bool cont = !div && r == r && r > tol && k < (double)maxcyc;
  // a bounded wait of the wavefront smoother ran out (ctl[17] set): the cycle's
  // result is not to be trusted, the step ends as late
  bool late = ctl[17] != 0.0;
  if (late) cont = false;
  if (cont && limit_ns > 0.0 &&
      (double)(global_ns() - *reinterpret_cast<const long long*>(ctl + 16)) > limit_ns) {
    cont = false;
    late = true;
  }
  const bool commit = !cont && r == r && !late && r <= tol;
  ctl[0] = r;
  ctl[1] = k;
  ctl[2] = grew;
  ctl[3] = late ? 1.0 : 0.0;
  ctl[4] = div ? 1.0 : 0.0;
  ctl[5] = commit ? 1.0 : 0.0;
  cudaGraphSetConditional(hl, cont ? 1u : 0u);
  cudaGraphSetConditional(hc, commit ? 1u : 0u);
}

// --------------------------------------------------------------------------
// host layout <-> padded layout
// --------------------------------------------------------------------------
// kind 0: cell (m2 x m1), 1: u (m2 x (m1+1)), 2: v ((m2+1) x m1)
template <typename T>
__global__ void k_pack_in(Lv<T> L, T* dst, const double* src, int kind) {
  pdl_enter();
  int a = blockIdx.x * BX + threadIdx.x;
  int b = blockIdx.y * BY + threadIdx.y;
  int nx = kind == 1 ? L.m1 + 1 : L.m1, ny = kind == 2 ? L.m2 + 1 : L.m2;
  if (a >= nx || b >= ny) return;
  int I = kind == 1 ? a : a + 1, J = kind == 2 ? b : b + 1;
  dst[L.at(I, J)] = (T)src[(size_t)b * nx + a];
}
template <typename T>
__global__ void k_pack_out(Lv<T> L, double* dst, const T* src, int kind) {
  pdl_enter();
  int a = blockIdx.x * BX + threadIdx.x;
  int b = blockIdx.y * BY + threadIdx.y;
  int nx = kind == 1 ? L.m1 + 1 : L.m1, ny = kind == 2 ? L.m2 + 1 : L.m2;
  if (a >= nx || b >= ny) return;
  int I = kind == 1 ? a : a + 1, J = kind == 2 ? b : b + 1;
  dst[(size_t)b * nx + a] = (double)src[L.at(I, J)];
}

// ==========================================================================
// launchers
// ==========================================================================
static int frame_threads(int m1, int m2) { return 4 * (m1 + 3) + 4 * (m2 + 3); }

template <typename T>
int nparts_cells(const Lv<T>& L) {
  dim3 g = grid2(L.m1, L.m2);
  return g.x * g.y;
}

template <typename T, class Form>
void launch_residual(const Prm<T>& P, const Lv<T>& L, double* part, cudaStream_t s) {
  if (residual_rows(L) == 2)
    qlaunch(&k_residual<T, 0, Form, 2>, grid2(L.m1, (L.m2 + 1) / 2), dim3(BX, BY), 0, s, P, L, part);
  else
    qlaunch(&k_residual<T, 0, Form, 1>, grid2(L.m1, L.m2), dim3(BX, BY), 0, s, P, L, part);
  ++g_launches;
}
template <typename T, class Form>
void launch_add_op(const Prm<T>& P, const Lv<T>& L, cudaStream_t s) {
  if (residual_rows(L) == 2)
    qlaunch(&k_residual<T, 1, Form, 2>, grid2(L.m1, (L.m2 + 1) / 2), dim3(BX, BY), 0, s, P, L, nullptr);
  else
    qlaunch(&k_residual<T, 1, Form, 1>, grid2(L.m1, L.m2), dim3(BX, BY), 0, s, P, L, nullptr);
  ++g_launches;
}
template <typename T, class Form>
void launch_ch(const Prm<T>& P, const Lv<T>& L, int colour, cudaStream_t s, int team_max) {
  int n = (L.m1 + 1) / 2 * L.m2;
  if (n <= 0) return;
  if constexpr (sizeof(T) == 8 || std::is_same<Form, ErrForm>::value) {
    if (n <= team_max) {  // four lanes per cell: shorter critical path per visit
      qlaunch(&k_ch_team<T, Form>, (4 * n + 63) / 64, 64, 0, s, P, L, colour);
      ++g_launches;
      return;
    }
  }
  qlaunch(&k_ch<T, Form>, (n + 63) / 64, 64, 0, s, P, L, colour);
  ++g_launches;
}
// SM sub-partitions of the current device (4 per SM)
static int sub_partitions() {
  static std::atomic<int> sms{0};
  if (!sms.load()) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    sms = n > 0 ? n : 1;
  }
  return 4 * sms.load();
}

// Slots of an n-slot FP64 Vanka colour that k_vanka_split runs one lane per
// block (the rest run as lane pairs).  split >= 2 forces split rounded down to
// a multiple of 32; split == 1 picks the count by a cost model of the busiest
// sub-partition: ceil(warps / sub-partitions) rounds of single-lane warps cost
// one unit each, rounds of pair warps VANKA_PAIR_ROUND each (the measured
// ratio of a pair round to a single-lane round on the 256x512 droplet's finest
// level, 7.5 us against 10.4 us), for colours that need two rounds or more.
// Returns n when no split is cheaper.  The model's premise, that the rounds of
// a sub-partition add up, did not hold on that level: the split it picks
// (19,456 single-lane blocks, the rest in pairs) took 22.8 us against 20.7 us
// for one lane per block, whose time is set by one visit's chain per round.
constexpr double VANKA_PAIR_ROUND = 0.72;
int vanka_split_single(int n, int split) {
  if (split >= 2) return std::min(n, split / 32 * 32);
  const long long S = sub_partitions();
  const long long ws = (n + 31) / 32, rounds = (ws + S - 1) / S;
  // one round is bound by the latency of a visit's chain, which pairs do not shorten
  if (rounds < 2) return n;
  double best = (double)rounds;
  int ns = n;
  for (long long k = 0; k < rounds; ++k) {
    const long long single = std::min<long long>(n, k * S * 32);
    const long long pw = (2 * (n - single) + 31) / 32;
    const double cost = (double)k + VANKA_PAIR_ROUND * (double)((pw + S - 1) / S);
    if (cost < best) { best = cost; ns = (int)single; }
  }
  return ns;
}

template <typename T, class Form>
void launch_vanka(const Prm<T>& P, const Lv<T>& L, int colour, T omega, cudaStream_t s,
                  int team_max, int team8_max, int pair_max, int split) {
  int n = vanka_slots(L, colour).n;
  if (n <= 0) return;
  if constexpr (std::is_same<Form, FullForm>::value && sizeof(T) == 8) {
    if (n <= team8_max) {  // eight lanes per block: half a momentum row per lane
      qlaunch(&k_vanka_team8, (8 * n + SNT - 1) / SNT, SNT, 0, s, P, L, colour, omega);
      ++g_launches;
      return;
    }
  }
  if constexpr ((std::is_same<Form, FullForm>::value && sizeof(T) == 8) ||
                std::is_same<Form, ErrForm>::value) {
    if (n <= team_max) {  // four lanes per block: shorter critical path per visit
      qlaunch(&k_vanka_team<T, Form>, (4 * n + SNT - 1) / SNT, SNT, 0, s, P, L, colour, omega);
      ++g_launches;
      return;
    }
  }
  if constexpr (std::is_same<Form, FullForm>::value && sizeof(T) == 8) {
    if (n <= pair_max) {  // a lane pair per block: half the FP64 instructions per lane
      qlaunch(&k_vanka_pair<T, Form>, (2 * n + SNT - 1) / SNT, SNT, 0, s, P, L, colour, omega);
      ++g_launches;
      return;
    }
    const int ns = split > 0 ? vanka_split_single(n, split) : n;
    if (ns < n) {  // one lane per block for slots [0, ns), a lane pair for the rest
      const long long threads = (long long)ns + 2LL * (n - ns);
      qlaunch(&k_vanka_split<T, Form>, (int)((threads + SNT - 1) / SNT), SNT, 0, s, P, L, colour,
              omega, ns);
      ++g_launches;
      return;
    }
  }
  qlaunch(&k_vanka<T, Form>, (n + SNT - 1) / SNT, SNT, 0, s, P, L, colour, omega);
  ++g_launches;
}
// Plan of the shared-memory copy of an FP64 full-iterate fused group: every
// level's arrays at their block's stride in QN_LV_ARRAYS order (checked
// pointer by pointer), columns within the copy kernel's 32-wide rows, and the
// whole copy within the device's opt-in shared memory per block.  Returns the
// dynamic shared-memory bytes, 0 if the group does not qualify.
static size_t coarse_smem_plan(const Lv<double>* levels, int n, CoarseSmem& M) {
  static std::atomic<int> optin{0};
  if (!optin.load()) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    optin = v > 0 ? v : 1;
  }
  const int head = (int)((sizeof(CoarseLevels<double>) + 15) / 16 * 2);
  long long elems = head;
  M.head = head;
  for (int l = 0; l < n; ++l) {
    const Lv<double>& L = levels[l];
    const int cc = L.m1 + 3, rr = L.m2 + 3;
    if (cc > 32 || !L.c) return 0;
    const long long ng = (long long)L.pitch * rr;
    int q = 0;
    bool ok = true;
#define QN_CHECK(m) ok = ok && L.m == L.c + (q++) * ng;
    QN_LV_ARRAYS(QN_CHECK)
#undef QN_CHECK
    if (!ok) return 0;
    M.ng[l] = ng;
    M.off[l] = (int)(elems - head);
    elems += (long long)QN_LV_NARR * cc * rr;
    elems = (elems + 1) / 2 * 2;  // 16-byte aligned copies
  }
  const size_t bytes = (size_t)elems * sizeof(double);
  return bytes <= (size_t)optin.load() ? bytes : 0;
}

void coarse_smem_prepare() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
      v > 0)
    cudaFuncSetAttribute(&k_coarse_vcycle_smem<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
  cudaGetLastError();
}

template <typename T, class Form>
int launch_coarse_vcycle(const Prm<T>& P, const Lv<T>* levels, int n, int nu1, int nu2, int nuc,
                         int kcol, T omega, int coupled, cudaStream_t s, int team8, int ctas,
                         int smem) {
  CoarseLevels<T> C;
  C.n = n;
  C.base = std::is_same<Form, ErrForm>::value;
  for (int l = 0; l < n; ++l) C.L[l] = levels[l];
  constexpr int NT = sizeof(T) == 8 ? 256 : 512;
  if constexpr (std::is_same<Form, FullForm>::value && sizeof(T) == 8) {
    if (smem && ctas <= 1) {
      CoarseSmem M = {};
      const size_t bytes = coarse_smem_plan(levels, n, M);
      if (bytes) {
        qlaunch(&k_coarse_vcycle_smem<NT>, 1, NT, bytes, s, P, C, M, nu1, nu2, nuc, omega, coupled,
                team8);
        ++g_launches;
        return 1;
      }
    }
  }
  if (ctas <= 1) {
    qlaunch(&k_coarse_vcycle<T, Form, NT>, 1, NT, 0, s, P, C, nu1, nu2, nuc, kcol, omega, coupled,
            team8);
  } else {  // one cluster of ctas blocks (a size coarse_cluster_blocks accepted)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(NT);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = g_pdl ? 2 : 1;
    cudaLaunchKernelEx(&cfg, &k_coarse_vcycle<T, Form, NT>, P, C, nu1, nu2, nuc, kcol, omega,
                       coupled, team8);
  }
  ++g_launches;
  return 0;
}

// largest cluster of at most `ctas` blocks (a power of two) in which the fused
// V-cycle of this form can run on the current device: a cluster is placed on
// the SMs of one GPC as a whole, and sizes above 8 need the non-portable
// cluster attribute, which the function must accept
template <typename T, class Form>
static int cluster_fit(int ctas) {
  constexpr int NT = sizeof(T) == 8 ? 256 : 512;
  auto kern = &k_coarse_vcycle<T, Form, NT>;
  if (ctas > 8 &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    ctas = 8;
  }
  for (; ctas > 1; ctas >>= 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(NT);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters > 0)
      break;
    cudaGetLastError();
  }
  return ctas < 1 ? 1 : ctas;
}

int coarse_cluster_blocks(int ctas) {
  int c = 1;
  while (c < 16 && 2 * c <= ctas) c *= 2;
  if (c == 1) return 1;
  c = cluster_fit<double, FullForm>(c);
  c = cluster_fit<double, ErrForm>(c);
  c = cluster_fit<float, ErrForm>(c);
  c = cluster_fit<double, ProjForm>(c);
  return c;
}

template <typename T, class Form>
void launch_vanka4(const Prm<T>& P, const Lv<T>& L, int colour, T omega, cudaStream_t s,
                   int team_max) {
  int n = vanka_slots(L, colour).n;
  if (n <= 0) return;
  if constexpr (std::is_same<Form, ProjForm>::value && sizeof(T) == 8) {
    if (n <= team_max) {  // four lanes per block: shorter critical path per visit
      qlaunch(&k_vanka4_team<T>, (4 * n + SNT - 1) / SNT, SNT, 0, s, P, L, colour, omega);
      ++g_launches;
      return;
    }
  }
  qlaunch(&k_vanka4<T, Form>, (n + SNT - 1) / SNT, SNT, 0, s, P, L, colour, omega);
  ++g_launches;
}
template <typename T>
void launch_pgs(const Prm<T>& P, const Lv<T>& L, int colour, cudaStream_t s, int team_max) {
  int n = (L.m1 + 1) / 2 * L.m2;
  if (n <= 0) return;
  if (n <= team_max) {  // four lanes per cell: shorter critical path per visit
    qlaunch(&k_pgs_team<T>, (4 * n + 63) / 64, 64, 0, s, P, L, colour);
    ++g_launches;
    return;
  }
  qlaunch(&k_pgs<T>, (n + 63) / 64, 64, 0, s, P, L, colour);
  ++g_launches;
}
template <typename T>
void launch_proj_velocity(const Prm<T>& P, const Lv<T>& L, T* uo, T* vo, cudaStream_t s) {
  qlaunch(&k_proj_velocity<T>, grid2(L.m1 + 1, L.m2 + 1), dim3(BX, BY), 0, s, P, L, uo, vo);
  ++g_launches;
}
template <typename T>
void launch_proj_diss(const Prm<T>& P, const Lv<T>& L, const T* uo, const T* vo, double* part,
                      double* out1, cudaStream_t s) {
  qlaunch(&k_proj_diss<T>, grid2(L.m1, L.m2), dim3(BX, BY), 0, s, P, L, uo, vo, part);
  ++g_launches;
  qlaunch(&k_finalize, 1, 256, 0, s, part, nparts_cells(L), 1, 0, 0.5 * (double)L.h * (double)L.h, out1);
  ++g_launches;
}
template <typename T, class Form>
void launch_coupled(const Prm<T>& P, const Lv<T>& L, int colour, T omega, cudaStream_t s,
                    int team_max) {
  int n = vanka_slots(L, colour).n;
  if (n <= 0) return;
  if (n <= team_max) {  // four lanes per block: shorter critical path per visit
    qlaunch(&k_coupled_team<T, Form>, (4 * n + SNT - 1) / SNT, SNT, 0, s, P, L, colour, omega);
    ++g_launches;
    return;
  }
  qlaunch(&k_coupled<T, Form>, (n + SNT - 1) / SNT, SNT, 0, s, P, L, colour, omega);
  ++g_launches;
}

static long long padded_n(int m1, int m2) {
  long long pitch = ((m1 + 3) + 31) / 32 * 32;
  return pitch * (m2 + 3);
}
template <typename T>
void launch_cast_frozen(const Lv<double>& D, const Lv<T>& E, cudaStream_t s) {
  long long n = padded_n(D.m1, D.m2);
  qlaunch(&k_cast_frozen<T>, (unsigned)((n + 255) / 256), 256, 0, s, D, E, n, D.pitch + 1);
  ++g_launches;
}
template <typename T>
void launch_start_correction(const Lv<double>& D, const Lv<T>& E, cudaStream_t s) {
  long long n = padded_n(D.m1, D.m2);
  qlaunch(&k_start_correction<T>, (unsigned)((n + 255) / 256), 256, 0, s, D, E, n, D.pitch + 1);
  ++g_launches;
}
template <typename T>
void launch_apply_correction(const Prm<double>& P, const Lv<double>& D, const Lv<T>& E,
                             cudaStream_t s) {
  long long n = padded_n(D.m1, D.m2);
  qlaunch(&k_apply_correction<T>, (unsigned)((n + 255) / 256), 256, 0, s, P, D, E, n, D.pitch + 1);
  ++g_launches;
}
void launch_rho_fill(const Prm<double>& P, const Lv<double>& L, cudaStream_t s) {
  long long n = padded_n(L.m1, L.m2);
  qlaunch(&k_rho_fill, (unsigned)((n + 255) / 256), 256, 0, s, P, L, n, L.pitch + 1);
  ++g_launches;
}
template <typename T>
void launch_restrict_base(const Lv<T>& F, const Lv<T>& C, cudaStream_t s) {
  qlaunch(&k_restrict_base<T>, grid2(C.m1 + 1, C.m2 + 1), dim3(BX, BY), 0, s, F, C);
  ++g_launches;
  int n = frame_threads(C.m1, C.m2);
  qlaunch(&k_bc_base<T>, (n + 255) / 256, 256, 0, s, C);
  ++g_launches;
}
template <typename T>
void launch_bc_unknowns(const Lv<T>& L, cudaStream_t s) {
  int n = frame_threads(L.m1, L.m2);
  qlaunch(&k_bc_unknowns<T>, (n + 255) / 256, 256, 0, s, L);
  ++g_launches;
}
template <typename T>
void launch_frozen(const Prm<T>& P, const Lv<T>& L, cudaStream_t s) {
  int n = frame_threads(L.m1, L.m2);
  qlaunch(&k_bc_frozen<T>, (n + 255) / 256, 256, 0, s, L);
  ++g_launches;
  qlaunch(&k_frozen_derived<T>, grid2(L.m1 + 2, L.m2 + 2), dim3(BX, BY), 0, s, P, L);
  ++g_launches;
  qlaunch(&k_frozen_coef1<T>, grid2(L.m1 + 2, L.m2 + 2), dim3(BX, BY), 0, s, L);
  ++g_launches;
  qlaunch(&k_frozen_coef2<T>, grid2(L.m1 + 1, L.m2 + 1), dim3(BX, BY), 0, s, L);
  if (L.T1u) {  // FP64 full-iterate levels
    qlaunch(&k_frozen_coef3<T>, grid2(L.m1 + 1, L.m2 + 1), dim3(BX, BY), 0, s, P, L);
    ++g_launches;
  }
  ++g_launches;
}
template <typename T>
void launch_restrict_state(const Prm<T>& P, const Lv<T>& F, const Lv<T>& C, cudaStream_t s) {
  qlaunch(&k_restrict_state<T>, grid2(C.m1 + 1, C.m2 + 1), dim3(BX, BY), 0, s, P, F, C);
  ++g_launches;
}
template <typename T>
void launch_restrict_res(const Lv<T>& F, const Lv<T>& C, cudaStream_t s) {
  qlaunch(&k_restrict_res<T>, grid2(C.m1, C.m2), dim3(BX, BY), 0, s, F, C);
  ++g_launches;
}
template <typename T>
void launch_restrict_frozen(const Lv<T>& F, const Lv<T>& C, cudaStream_t s) {
  qlaunch(&k_restrict_frozen<T>, grid2(C.m1 + 1, C.m2 + 1), dim3(BX, BY), 0, s, F, C);
  ++g_launches;
}
template <typename T>
void launch_prolong(const Prm<T>& P, const Lv<T>& F, const Lv<T>& C, cudaStream_t s) {
  qlaunch(&k_prolong<T>, grid2(F.m1, F.m2), dim3(BX, BY), 0, s, P, F, C);
  ++g_launches;
}
template <typename T>
void launch_gauge(const Lv<T>& L, double* part, double* scal, cudaStream_t s) {
  qlaunch(&k_sum_p<T>, grid2(L.m1, L.m2), dim3(BX, BY), 0, s, L, part);
  ++g_launches;
  qlaunch(&k_finalize, 1, 256, 0, s, part, nparts_cells(L), 1, 0, 1.0, scal);
  ++g_launches;
  qlaunch(&k_sub_mean_p<T>, grid2(L.m1 + 2, L.m2 + 2), dim3(BX, BY), 0, s, L, scal,
                                                                     1.0 / ((double)L.m1 * L.m2));
  ++g_launches;
}
template <typename T>
void launch_norms_finalize(const Lv<T>& L, double* part, double* out10, cudaStream_t s) {
  // part rows are [max x5, sum of squares x5]; out10 = [l2 x5, max x5] after the
  // host applies sqrt(h^2 *) to the sums; here: out[0..4] = max, out[5..9] = h^2 sum
  dim3 g = grid2(L.m1, (L.m2 + residual_rows(L) - 1) / residual_rows(L));  // k_residual's blocks
  qlaunch(&k_finalize, 1, 256, 0, s, part, (int)(g.x * g.y), 10, 5, (double)L.h * (double)L.h, out10);
  ++g_launches;
}
void launch_diag(const Lv<double>& L, const double* c, const double* u, const double* v,
                 double* part, double* out11, cudaStream_t s) {
  qlaunch(&k_diag_cells, grid2(L.m1, L.m2), dim3(BX, BY), 0, s, L, c, u, v, part);
  qlaunch(&k_finalize, 1, 256, 0, s, part, nparts_cells(L), 7, 3, 1.0, out11);
  int nb = (L.m1 + NT - 1) / NT;
  qlaunch(&k_diag_cols, nb, NT, 0, s, L, c, part);
  qlaunch(&k_finalize, 1, 256, 0, s, part, nb, 4, 2, 1.0, out11 + 7);
  g_launches += 4;
}
void launch_div_field(const Lv<double>& L, const double* u, const double* v, double* out,
                      cudaStream_t s) {
  qlaunch(&k_div_field, grid2(L.m1, L.m2), dim3(BX, BY), 0, s, L, u, v, out);
  ++g_launches;
}
template <typename T>
void launch_mass(const Prm<T>& P, const Lv<T>& L, const T* c, double* part, double* out2,
                 cudaStream_t s) {
  qlaunch(&k_mass<T>, grid2(L.m1, L.m2), dim3(BX, BY), 0, s, P, L, c, part);
  ++g_launches;
  qlaunch(&k_finalize, 1, 256, 0, s, part, nparts_cells(L), 2, 0, (double)L.h * (double)L.h, out2);
  ++g_launches;
}
template <typename T>
void launch_energy(const Prm<T>& P, const Lv<T>& L, const T* c, const T* u, const T* v,
                   double w_grad, double w_bulk, double w_pot, double* part, double* out1,
                   cudaStream_t s) {
  qlaunch(&k_energy<T>, grid2(L.m1, L.m2), dim3(BX, BY), 0, s, P, L, c, u, v, w_grad, w_bulk, w_pot,
                                                          part);
  ++g_launches;
  qlaunch(&k_finalize, 1, 256, 0, s, part, nparts_cells(L), 1, 0, (double)L.h * (double)L.h, out1);
  ++g_launches;
}
template <typename T>
void launch_dissipation(const Prm<T>& P, const Lv<T>& L, double w_visc, double w_div,
                        double w_ch, double* part, double* out1, cudaStream_t s) {
  dim3 g = grid2(L.m1 + 1, L.m2 + 1);
  qlaunch(&k_dissipation<T>, g, dim3(BX, BY), 0, s, P, L, w_visc, w_div, w_ch, part);
  ++g_launches;
  qlaunch(&k_finalize, 1, 256, 0, s, part, g.x * g.y, 1, 0, (double)L.h * (double)L.h, out1);
  ++g_launches;
}
template <typename T>
void launch_pack_in(const Lv<T>& L, T* dst, const double* src, int kind, cudaStream_t s) {
  int nx = kind == 1 ? L.m1 + 1 : L.m1, ny = kind == 2 ? L.m2 + 1 : L.m2;
  qlaunch(&k_pack_in<T>, grid2(nx, ny), dim3(BX, BY), 0, s, L, dst, src, kind);
  ++g_launches;
}
template <typename T>
void launch_pack_out(const Lv<T>& L, double* dst, const T* src, int kind, cudaStream_t s) {
  int nx = kind == 1 ? L.m1 + 1 : L.m1, ny = kind == 2 ? L.m2 + 1 : L.m2;
  qlaunch(&k_pack_out<T>, grid2(nx, ny), dim3(BX, BY), 0, s, L, dst, src, kind);
  ++g_launches;
}

template <typename T, class Form>
void launch_wave(const Prm<T>& P, const Lv<T>& L, const WavePlan& W, T omega, unsigned* ctr,
                 double* flag, cudaStream_t s) {
  static std::atomic<int> blocks_per_sm{0};
  static std::atomic<int> sms{0};
  if (!sms.load()) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    sms = n > 0 ? n : 1;
  }
  if (!blocks_per_sm.load()) {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_wave<T, Form>, WAVE_NT, 0);
    blocks_per_sm = b > 0 ? b : 1;
  }
  const long long tasks = (long long)W.nbands * W.npass;
  const int grid = (int)std::min<long long>((long long)sms.load() * blocks_per_sm.load(), tasks);
  cudaMemsetAsync(ctr, 0, (size_t)(1 + W.nbands) * sizeof(unsigned), s);
  qlaunch(&k_wave<T, Form>, grid, WAVE_NT, 0, s, P, L, W, omega, ctr, flag);
  ++g_launches;
}

template <typename T, class Form>
int launch_skew(const Prm<T>& P, const Lv<T>& L, int nsteps, int coupled, int rows, T omega,
                cudaStream_t s) {
  const int per = coupled ? L.kcol : L.kcol + 2;
  const int H = std::max(rows, 1);
  const int group = std::max(1, SKEW_MAX_TASKS / per);  // steps per schedule
  int launches = 0;
  for (int s0 = 0; s0 < nsteps; s0 += group) {
    const int npass = std::min(group, nsteps - s0) * per;
    // the last diagonal on which the last pass still has rows of the level
    const int D = npass + (L.m2 - 1 + (npass - 1) * SKEW_LAG) / H;
    for (int d = 0; d < D; ++d) {
      SkewTasks S;
      S.n = 0;
      int nb = 0;
      for (int p = 0; p < npass; ++p) {
        const int lo = std::max(1 + (d - p) * H - p * SKEW_LAG, 1);
        const int hi = std::min(1 + (d - p + 1) * H - p * SKEW_LAG, L.m2 + 1);
        if (lo >= hi) continue;
        const int q = p % per;
        int t_lo, t_hi;
        if (!coupled && q < 2) {
          const int mpr = (L.m1 + 1) / 2;
          t_lo = (lo - 1) * mpr;
          t_hi = (hi - 1) * mpr;
        } else {
          const ColourSlots cs = vanka_slots(L, coupled ? q : q - 2);
          const int r1 = hi - 1;  // rows lo .. r1
          if (r1 < cs.j0) continue;
          const int qlo = lo > cs.j0 ? (lo - cs.j0 + cs.rstep - 1) / cs.rstep : 0;
          const int qhi = (r1 - cs.j0) / cs.rstep;
          t_lo = qlo * cs.mpr;
          t_hi = std::min((qhi + 1) * cs.mpr, cs.n);
        }
        if (t_lo >= t_hi) continue;
        S.q[S.n] = q;
        S.t_lo[S.n] = t_lo;
        S.t_hi[S.n] = t_hi;
        S.boff[S.n] = nb;
        nb += (t_hi - t_lo + SNT - 1) / SNT;
        ++S.n;
      }
      S.boff[S.n] = nb;
      if (S.n == 0) continue;
      if (coupled) qlaunch(&k_skew<T, Form, true>, nb, SNT, 0, s, P, L, S, omega);
      else qlaunch(&k_skew<T, Form, false>, nb, SNT, 0, s, P, L, S, omega);
      ++g_launches;
      ++launches;
    }
  }
  return launches;
}

void launch_predict(double* const x[5], double* const a[5], double* const b[5],
                    double* const c[5], const double w[3], size_t n, int off, cudaStream_t s) {
  FiveArrays X, A, B, C;
  for (int q = 0; q < 5; ++q) {
    X.p[q] = x[q];
    A.p[q] = a[q];
    B.p[q] = b[q];
    C.p[q] = c[q];
  }
  const int NT = 256;
  dim3 grid((unsigned)((n + NT - 1) / NT), 5);
  qlaunch(&k_predict, grid, NT, 0, s, X, A, B, C, w[0], w[1], w[2], (long long)n, off);
  ++g_launches;
}

void launch_loop_clock(double* ctl, cudaStream_t s) {
  qlaunch(&k_loop_clock, 1, 1, 0, s, ctl);
  ++g_launches;
}
void launch_loop_ctl(const double* nrm, double* ctl, cudaGraphConditionalHandle hl,
                     cudaGraphConditionalHandle hc, double tol, int maxcyc, int diverge,
                     double limit_ns, int first, cudaStream_t s) {
  qlaunch(&k_loop_ctl, 1, 1, 0, s, nrm, ctl, hl, hc, tol, maxcyc, diverge, limit_ns, first);
  ++g_launches;
}

int partial_rows_needed(int m1, int m2) {
  dim3 g = grid2(m1 + 1, m2 + 1);
  return g.x * g.y;
}

#define QN_INSTANTIATE_FORM(T, F)                                                                \
  template int launch_coarse_vcycle<T, F>(const Prm<T>&, const Lv<T>*, int, int, int, int, int,   \
                                          T, int, cudaStream_t, int, int, int);                  \
  template void launch_coupled<T, F>(const Prm<T>&, const Lv<T>&, int, T, cudaStream_t, int);     \
  template void launch_residual<T, F>(const Prm<T>&, const Lv<T>&, double*, cudaStream_t);       \
  template void launch_add_op<T, F>(const Prm<T>&, const Lv<T>&, cudaStream_t);                  \
  template void launch_ch<T, F>(const Prm<T>&, const Lv<T>&, int, cudaStream_t, int);            \
  template void launch_vanka<T, F>(const Prm<T>&, const Lv<T>&, int, T, cudaStream_t, int, int, int, int);

#define QN_INSTANTIATE(T)                                                                        \
  template void launch_cast_frozen<T>(const Lv<double>&, const Lv<T>&, cudaStream_t);            \
  template void launch_start_correction<T>(const Lv<double>&, const Lv<T>&, cudaStream_t);       \
  template void launch_apply_correction<T>(const Prm<double>&, const Lv<double>&, const Lv<T>&,    \
                                            cudaStream_t);                                          \
  template void launch_restrict_base<T>(const Lv<T>&, const Lv<T>&, cudaStream_t);               \
  template void launch_bc_unknowns<T>(const Lv<T>&, cudaStream_t);                               \
  template void launch_frozen<T>(const Prm<T>&, const Lv<T>&, cudaStream_t);                     \
  template void launch_restrict_state<T>(const Prm<T>&, const Lv<T>&, const Lv<T>&, cudaStream_t); \
  template void launch_restrict_res<T>(const Lv<T>&, const Lv<T>&, cudaStream_t);                \
  template void launch_restrict_frozen<T>(const Lv<T>&, const Lv<T>&, cudaStream_t);             \
  template void launch_prolong<T>(const Prm<T>&, const Lv<T>&, const Lv<T>&, cudaStream_t);        \
  template void launch_gauge<T>(const Lv<T>&, double*, double*, cudaStream_t);                   \
  template void launch_norms_finalize<T>(const Lv<T>&, double*, double*, cudaStream_t);          \
  template void launch_mass<T>(const Prm<T>&, const Lv<T>&, const T*, double*, double*,          \
                               cudaStream_t);                                                    \
  template void launch_energy<T>(const Prm<T>&, const Lv<T>&, const T*, const T*, const T*,      \
                                 double, double, double, double*, double*, cudaStream_t);        \
  template void launch_dissipation<T>(const Prm<T>&, const Lv<T>&, double, double, double,       \
                                      double*, double*, cudaStream_t);                           \
  template void launch_pack_in<T>(const Lv<T>&, T*, const double*, int, cudaStream_t);           \
  template void launch_pack_out<T>(const Lv<T>&, double*, const T*, int, cudaStream_t);

QN_INSTANTIATE(double)
QN_INSTANTIATE(float)
QN_INSTANTIATE_FORM(double, FullForm)
QN_INSTANTIATE_FORM(double, ErrForm)
QN_INSTANTIATE_FORM(float, ErrForm)
template void launch_wave<float, ErrForm>(const Prm<float>&, const Lv<float>&, const WavePlan&,
                                          float, unsigned*, double*, cudaStream_t);
template void launch_wave<double, ErrForm>(const Prm<double>&, const Lv<double>&, const WavePlan&,
                                           double, unsigned*, double*, cudaStream_t);
template int launch_skew<float, ErrForm>(const Prm<float>&, const Lv<float>&, int, int, int, float,
                                         cudaStream_t);
template int launch_skew<double, ErrForm>(const Prm<double>&, const Lv<double>&, int, int, int, double,
                                          cudaStream_t);
// projection method (FP64, per-level launches)
template void launch_residual<double, ProjForm>(const Prm<double>&, const Lv<double>&, double*,
                                                cudaStream_t);
template int launch_coarse_vcycle<double, ProjForm>(const Prm<double>&, const Lv<double>*, int, int,
                                                    int, int, int, double, int, cudaStream_t, int,
                                                    int, int);
template void launch_add_op<double, ProjForm>(const Prm<double>&, const Lv<double>&, cudaStream_t);
template void launch_ch<double, ProjForm>(const Prm<double>&, const Lv<double>&, int, cudaStream_t,
                                          int);
template void launch_vanka4<double, ProjForm>(const Prm<double>&, const Lv<double>&, int, double,
                                               cudaStream_t, int);
template void launch_pgs<double>(const Prm<double>&, const Lv<double>&, int, cudaStream_t, int);
template void launch_proj_velocity<double>(const Prm<double>&, const Lv<double>&, double*, double*,
                                           cudaStream_t);
template void launch_proj_diss<double>(const Prm<double>&, const Lv<double>&, const double*,
                                       const double*, double*, double*, cudaStream_t);

}  // namespace qn
