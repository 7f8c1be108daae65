// qnsch_dev.cuh -- device data structures and the discrete operator of the
// primitive method (Guo, Lin, Lowengrub & Wise, arXiv:1703.06606, Sec. 6.1) on
// the staggered grid of Sec. 5 / App. A, for sm_103a.
//
// Layout: every array of a level lives in one padded 2-D index space with one
// ghost layer: entry (I, J), I = -1..m1+1, J = -1..m2+1, at origin[J*pitch + I];
// pitch is a multiple of 32 elements so that rows start 256-byte aligned.
//   cell (i,j)        -> (i, j)       i, j = 0..m1+1 / 0..m2+1 (with ghosts)
//   u_{i+1/2, j}      -> (i, j)       i = -1..m1+1
//   v_{i, j+1/2}      -> (i, j)       j = -1..m2+1
// A thread working at cell (i,j) therefore reads cell, u and v arrays at the same
// offset plus small constant displacements.
#pragma once
#include <cuda_runtime.h>

namespace qn {

template <typename T>
struct Prm {
  T ia, ib;        // rho(c) = 1 / (ia c + ib): ia = alpha = (rho2-rho1)/(rho1 rho2), ib = 1/rho2
  T va, vb;        // viscosity mu(c) = 1 / (va c + vb)
  T alpha;         // (rho2 - rho1) / (rho1 rho2), Sec. 2.1
  T K, Lam;        // M eta/(eps We) and eps eta M/We, coefficients of (pm-num-chem)
  T iM, iRe, iPe;  // 1/M, 1/Re, 1/Pe
  T Fr_inv;        // 1/Fr (0: no gravity)
  T eps_m;         // mobility regularisation, m(c) = sqrt(c^2 (1-c)^2 + eps_m)
  T idt;           // 1/dt
};

template <typename T>
struct Lv {
  int m1, m2, px, pitch;
  // Vanka colours of this level: kcol colours, (2i+j) mod 8 when c8 is set
  // (periodic x with m1 = 0 mod 4), else (i+2j) mod kcol
  int kcol, c8;
  T h, ih, ih2;
  T *c, *mu, *p, *u, *v;       // iterate
  T *fc, *fmu, *fp, *fu, *fv;  // FAS right-hand side
  T *rc, *rmu, *rp, *ru, *rv;  // residual f - N(x)
  T *sc, *smu, *sp, *su, *sv;  // restricted iterate kept for the correction
  T *cn, *un, *vn;             // frozen level-n data
  T *rhon, *mobn, *visn, *Gn;  // rho(c^n), m(c^n), mu(c^n), G(c^n)
  // coefficients of (pm-num-mx) that depend on frozen data only, built once
  // per step: A_x rho^n, A_y rho^n (edges); rho^n a_x u^n, rho^n a_y v^n
  // (cells); Acal rho^n Acal_x v^n, Acal rho^n Acal_y u^n, Acal mu(c^n)
  // (vertices (i+1/2, j+1/2) at (i,j)); D_x c^n / 2, D_y c^n / 2 (edges);
  // the divergence corrections 1/2[D_x(rho a_x u) + Dfrak_y(..)] (x-edges)
  // and 1/2[Dfrak_x(..) + D_y(rho a_y v)] (y-edges) of (e1e1-2)
  T *Aru, *Arv, *Sx, *Sy, *Qx, *Qy, *Av, *Tx, *Ty, *Dvu, *Dvv;
  // FP64 full-iterate levels only, built per step (they depend on dt): for each
  // momentum row (x-edges *u, y-edges *v) the time-term coefficients, time =
  // x T1 + T0 + (dt^-1/2) A rho(c) x with T1 = A rho^n/(2dt) + Dv and T0 =
  // -A rho^n x^n/dt, and Dg, the part of the row's diagonal entry that does not
  // depend on the iterate (the whole diagonal is Dg + A rho(c)/(2dt))
  T *T1u = nullptr, *T1v = nullptr, *T0u = nullptr, *T0v = nullptr, *Dgu = nullptr, *Dgv = nullptr;
  // FP64 full-iterate levels only: rho(c) of the iterate, ghosts included.
  // Every kernel that writes c writes rho(c) beside it, so the smoothers and
  // the residual read the density instead of dividing for it; the values are
  // those rho_of gives.
  T* rhoc = nullptr;
  // FP64 full-iterate levels only, built per step: the momentum rows of
  // (pm-num-mx) assembled as stencils.  Apart from the density term A rho(c)
  // u / (2dt), each row is linear in the iterate with coefficients that depend
  // on frozen data only.  For the x row at edge k (y row: u <-> v, strides
  // swapped): Cu multiplies u at the edge itself, aPu / aMu its neighbours
  // along x (k + 1, k - 1), tPu / tMu across (k + W, k - W), M0u / M1u the mu of
  // the cells k and k + 1.  Wall edges read their reflected ghosts, as the
  // unassembled row does.
  T *Cu = nullptr, *aPu = nullptr, *aMu = nullptr, *tPu = nullptr, *tMu = nullptr,
    *M0u = nullptr, *M1u = nullptr;
  T *Cv = nullptr, *aPv = nullptr, *aMv = nullptr, *tPv = nullptr, *tMv = nullptr,
    *M0v = nullptr, *M1v = nullptr;
  // error-equation (defect-correction) levels only: base state X the iterate
  // e is a correction to, and X.c - c^n formed in FP64 before rounding
  T *Bc = nullptr, *Bmu = nullptr, *Bu = nullptr, *Bv = nullptr, *Bdc = nullptr;
  __device__ __forceinline__ int at(int i, int j) const { return j * pitch + i; }
  // x-edge unknowns: walls exclude i = 0 and i = m1; periodic keeps i = m1 (= edge 0)
  __device__ __forceinline__ int uhi() const { return px ? m1 : m1 - 1; }
};

// The arrays of an FP64 full-iterate level in the order in which they sit in
// the level's block (one allocation, NFIELD arrays of the same padded size):
// X(member) for each.
#define QN_LV_ARRAYS(X)                                                                        \
  X(c) X(mu) X(p) X(u) X(v) X(fc) X(fmu) X(fp) X(fu) X(fv) X(rc) X(rmu) X(rp) X(ru) X(rv)     \
  X(sc) X(smu) X(sp) X(su) X(sv) X(cn) X(un) X(vn) X(rhon) X(mobn) X(visn) X(Gn) X(Aru)       \
  X(Arv) X(Sx) X(Sy) X(Qx) X(Qy) X(Av) X(Tx) X(Ty) X(Dvu) X(Dvv) X(T1u) X(T1v) X(T0u) X(T0v)  \
  X(Dgu) X(Dgv) X(rhoc) X(Cu) X(aPu) X(aMu) X(tPu) X(tMu) X(M0u) X(M1u) X(Cv) X(aPv) X(aMv)   \
  X(tPv) X(tMv) X(M0v) X(M1v)

// ---------------------------------------------------------------------------
// constitutive functions (Sec. 2.1) and secants (Sec. 4.1)
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T rho_of(const Prm<T>& P, T c) {
  return T(1) / (P.ia * c + P.ib);
}
// a / b: in FP32 (the error-equation smoothers) the fast division, within 2
// ulp, whose rounding the FP64 defect correction absorbs; IEEE division in FP64
template <typename T> __device__ __forceinline__ T qdiv(T a, T b) { return a / b; }
template <> __device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
// 1/x for the pivots of the local block solves.  FP32: the fast division, as
// qdiv.  FP64: the Newton-Raphson iteration r <- r + r (1 - x r) for the zero
// of 1/r - x, which squares the relative error of r at every step, started
// from the hardware's approximate reciprocal (rcp.approx.ftz.f64); after two
// steps the result is within a few units in the last place of 1/x (tested
// against IEEE division).  Normal-range x only: the pivots are determinants
// and diagonal sums of the local systems, far from the subnormal range.
template <typename T> __device__ __forceinline__ T qrcp(T x) { return qdiv(T(1), x); }
template <> __device__ __forceinline__ double qrcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
template <> __device__ __forceinline__ float rho_of(const Prm<float>& P, float c) {
  return qdiv(1.0f, P.ia * c + P.ib);
}
template <typename T> __device__ __forceinline__ T visc_of(const Prm<T>& P, T c) {
  return T(1) / (P.va * c + P.vb);
}
template <typename T> __device__ __forceinline__ T mob_of(const Prm<T>& P, T c) {
  T w = c * (T(1) - c);
  return sqrt(w * w + P.eps_m);
}
template <typename T> __device__ __forceinline__ T Fdw(T c) {
  T w = c * (c - T(1));
  return T(0.25) * w * w;
}
template <typename T> __device__ __forceinline__ T fdw(T c) { return c * (c - T(1)) * (c - T(0.5)); }
// g(a,b) with F(a) - F(b) = g(a,b) (a - b)
template <typename T> __device__ __forceinline__ T gsec(T a, T b) {
  return T(0.25) * (a * (a - T(1)) + b * (b - T(1))) * (a + b - T(1));
}
template <typename T> __device__ __forceinline__ T gsec_da(T a, T b) {
  return T(0.25) * ((T(2) * a - T(1)) * (a + b - T(1)) + a * (a - T(1)) + b * (b - T(1)));
}

// ---------------------------------------------------------------------------
// pieces of the discrete operator N(x) (Sec. 6.1)
// ---------------------------------------------------------------------------

// G(c) = a_x((D_x c)^2) + a_y((D_y c)^2) at cell k (times h^2)
template <typename T>
__device__ __forceinline__ T G_h2(const T* c, int k, int pitch) {
  T cc = c[k];
  T de = c[k + 1] - cc, dw = cc - c[k - 1], dn = c[k + pitch] - cc, ds = cc - c[k - pitch];
  return T(0.5) * (de * de + dw * dw + dn * dn + ds * ds);
}

// h^2 grad_d.(A kap grad_D phi) at cell k
template <typename T>
__device__ __forceinline__ T lap_h2(const T* kap, const T* phi, int k, int pitch) {
  T kc = kap[k], pc = phi[k];
  return T(0.5) * ((kap[k + 1] + kc) * (phi[k + 1] - pc) - (kc + kap[k - 1]) * (pc - phi[k - 1]) +
                   (kap[k + pitch] + kc) * (phi[k + pitch] - pc) -
                   (kc + kap[k - pitch]) * (pc - phi[k - pitch]));
}

// (pm-num-phase) with the advection (e1e2) of App. A.4
// (the overloads taking densities let a caller that already holds rho(c) of
// the cell and its neighbours skip the divisions; the values are the same)
template <typename T>
__device__ __forceinline__ T op_c(const Prm<T>& P, const Lv<T>& L, int k, T rho) {
  const int W = L.pitch;
  const T* cn = L.cn;
  const T* rn = L.rhon;
  T c = L.c[k], cnk = cn[k];
  T adv = rn[k + 1] * L.Tx[k] * L.u[k] + rn[k - 1] * L.Tx[k - 1] * L.u[k - 1] +
          rn[k + W] * L.Ty[k] * L.v[k] + rn[k - W] * L.Ty[k - W] * L.v[k - W];
  T diff = lap_h2(L.mobn, L.mu, k, W) + P.alpha * lap_h2(L.mobn, L.p, k, W);
  return rho * (c - cnk) * P.idt + adv - P.iPe * L.ih2 * diff;
}
template <typename T>
__device__ __forceinline__ T op_c(const Prm<T>& P, const Lv<T>& L, int k) {
  return op_c(P, L, k, rho_of(P, L.c[k]));
}

// (pm-num-chem) with the time-averaged gradient term (pointwise G)
// rq[f]: rho(c) of the neighbours k + 1, k - 1, k + W, k - W; rmu multiplies mu
// (rho(c) in (pm-num-chem), rho^n in the projection method's (pj-num-chem))
template <typename T>
__device__ __forceinline__ T op_mu_r(const Prm<T>& P, const Lv<T>& L, int k, T rho, const T (&rq)[4],
                                     T rmu) {
  const int W = L.pitch;
  const T* c = L.c;
  const T* cn = L.cn;
  const T* rn = L.rhon;
  T ck = c[k], cnk = cn[k];
  T rnk = rn[k];
  T rh = T(0.5) * (rho + rnk);
  T r = -P.alpha * rho * rnk;
  T bulk = rh * gsec(ck, cnk) + T(0.5) * (Fdw(ck) + Fdw(cnk)) * r;
  T grad = T(0.25) * P.Lam * (G_h2(c, k, W) * L.ih2 + L.Gn[k]) * r;
  // grad_d.(A rho^{n+1/2} grad_D c^{n+1/2})
  T chk = ck + cnk;
  T div = T(0);
  const int off[4] = {1, -1, W, -W};
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    int q = k + off[f];
    T rf = T(0.5) * (rq[f] + rn[q]);
    div += (rh + rf) * ((c[q] + cn[q]) - chk);
  }
  div *= T(0.25) * L.ih2;  // 1/2 (face average) * 1/2 (c^{n+1/2}) / h^2
  return rmu * L.mu[k] - P.K * bulk - grad + P.Lam * div;
}
template <typename T>
__device__ __forceinline__ T op_mu(const Prm<T>& P, const Lv<T>& L, int k, T rho, const T (&rq)[4]) {
  return op_mu_r(P, L, k, rho, rq, rho);
}
template <typename T>
__device__ __forceinline__ T op_mu(const Prm<T>& P, const Lv<T>& L, int k) {
  const int W = L.pitch;
  const T rq[4] = {rho_of(P, L.c[k + 1]), rho_of(P, L.c[k - 1]), rho_of(P, L.c[k + W]),
                   rho_of(P, L.c[k - W])};
  return op_mu(P, L, k, rho_of(P, L.c[k]), rq);
}

// (pm-num-mass)
template <typename T>
__device__ __forceinline__ T op_p(const Prm<T>& P, const Lv<T>& L, int k) {
  const int W = L.pitch;
  T dv = (L.u[k] - L.u[k - 1] + L.v[k] - L.v[k - W]) * L.ih;
  T diff = lap_h2(L.mobn, L.mu, k, W) + P.alpha * lap_h2(L.mobn, L.p, k, W);
  return dv - P.alpha * P.iPe * L.ih2 * diff;
}

// Momentum row d (0: x row at x-edge k, unknown u; 1: y row at y-edge k,
// unknown v) of (pm-num-mx) from the per-step assembled stencil (the arrays
// Cu.. / Cv.. of Lv): the same sum as op_u / op_v, term by term, regrouped by
// unknown.  Ar = A rho(c) on the edge.  s is the stride along the edge normal,
// t across it; a the row's own velocity, b the other one.
template <typename T>
__device__ __forceinline__ T mom_asm(const Prm<T>& P, const Lv<T>& L, int d, int k, T Ar) {
  const int s = d ? L.pitch : 1, t = d ? 1 : L.pitch;
  const T *a = d ? L.v : L.u, *b = d ? L.u : L.v;
  const T *C = d ? L.Cv : L.Cu, *aP = d ? L.aPv : L.aPu, *aM = d ? L.aMv : L.aMu;
  const T *tP = d ? L.tPv : L.tPu, *tM = d ? L.tMv : L.tMu;
  const T *M0 = d ? L.M0v : L.M0u, *M1 = d ? L.M1v : L.M1u;
  T ae = a[k];
  T r = (d ? L.T0v : L.T0u)[k] + (C[k] + T(0.5) * P.idt * Ar) * ae;
  r += aP[k] * a[k + s] + aM[k] * a[k - s] + tP[k] * a[k + t] + tM[k] * a[k - t];
  // the grad-div term's cross derivative of the other velocity
  T vl = L.visn[k], vr = L.visn[k + s];
  r -= (P.iRe * L.ih2 * T(1.0 / 3.0)) * (vr * (b[k + s] - b[k + s - t]) - vl * (b[k] - b[k - t]));
  r += (L.p[k + s] - L.p[k]) * (L.ih * P.iM) + M0[k] * L.mu[k] + M1[k] * L.mu[k + s];
  if (d) r += P.Fr_inv * L.Arv[k];
  return r;
}

// x row of (pm-num-mx) at edge u_{i+1/2,j} (array index k = at(i,j)); cells k (left), k+1 (right),
// vertices k (top, (i+1/2, j+1/2)) and k-W (bottom); (e1e1-1), (e1e1-2) and (e1e1)
// (Ar = (rho(c_k) + rho(c_{k+1})) / 2, the density average on the edge).  PST =
// false drops the pressure and surface-tension terms: the intermediate-velocity
// row of the projection method (pj-num-mx).
template <typename T, bool PST = true>
__device__ __forceinline__ T op_u(const Prm<T>& P, const Lv<T>& L, int k, T Ar) {
  if constexpr (PST && sizeof(T) == 8) return mom_asm(P, L, 0, k, Ar);  // FP64 primitive row
  const int W = L.pitch;
  const T *u = L.u, *vis = L.visn, *rn = L.rhon;
  T ue = u[k];
  T dxl = (ue - u[k - 1]) * L.ih, dxr = (u[k + 1] - ue) * L.ih;
  T dvl = dxl + (L.v[k] - L.v[k - W]) * L.ih;
  T dvr = dxr + (L.v[k + 1] - L.v[k + 1 - W]) * L.ih;
  T Dt = (u[k + W] - ue) * L.ih, Db = (ue - u[k - W]) * L.ih;
  T conv = T(0.5) * (L.Sx[k + 1] * dxr + L.Sx[k] * dxl + L.Qx[k] * Dt + L.Qx[k - W] * Db);
  T time = ue * L.T1u[k] + L.T0u[k] + T(0.5) * P.idt * Ar * ue;
  T r = time + conv;
  if constexpr (PST) {
    T press = (L.p[k + 1] - L.p[k]) * L.ih * P.iM;
    T st = -(rn[k + 1] * L.mu[k] + rn[k] * L.mu[k + 1]) * L.Tx[k] * P.iM;
    r = r + press + st;
  }
  T vl = vis[k], vr = vis[k + 1];
  T visc = -P.iRe * L.ih * ((vr * dxr - vl * dxl) + (L.Av[k] * Dt - L.Av[k - W] * Db) +
                            (vr * dvr - vl * dvl) * T(1.0 / 3.0));
  return r + visc;
}
template <typename T>
__device__ __forceinline__ T op_u(const Prm<T>& P, const Lv<T>& L, int k) {
  return op_u(P, L, k, T(0.5) * (rho_of(P, L.c[k]) + rho_of(P, L.c[k + 1])));
}

// y row of (pm-num-mx) at edge v_{i,j+1/2} (index k = at(i,j)); cells k (bottom), k+W (top),
// vertices k (east, (i+1/2, j+1/2)) and k-1 (west); plus gravity (1/Fr) A_y rho^n
// PST = false: the projection method's intermediate-velocity row, without
// pressure, surface tension and gravity (those act in (pj-num-pjx))
template <typename T, bool PST = true>
__device__ __forceinline__ T op_v(const Prm<T>& P, const Lv<T>& L, int k, T Ar) {
  if constexpr (PST && sizeof(T) == 8) return mom_asm(P, L, 1, k, Ar);  // FP64 primitive row
  const int W = L.pitch;
  const T *v = L.v, *vis = L.visn, *rn = L.rhon;
  T ve = v[k];
  T dyb = (ve - v[k - W]) * L.ih, dyt = (v[k + W] - ve) * L.ih;
  T dvb = dyb + (L.u[k] - L.u[k - 1]) * L.ih;
  T dvt = dyt + (L.u[k + W] - L.u[k + W - 1]) * L.ih;
  T De = (v[k + 1] - ve) * L.ih, Dw = (ve - v[k - 1]) * L.ih;
  T conv = T(0.5) * (L.Qy[k] * De + L.Qy[k - 1] * Dw + L.Sy[k + W] * dyt + L.Sy[k] * dyb);
  T time = ve * L.T1v[k] + L.T0v[k] + T(0.5) * P.idt * Ar * ve;
  T r = time + conv;
  if constexpr (PST) {
    T press = (L.p[k + W] - L.p[k]) * L.ih * P.iM;
    T st = -(rn[k + W] * L.mu[k] + rn[k] * L.mu[k + W]) * L.Ty[k] * P.iM;
    r = r + press + st;
  }
  T vb = vis[k], vt = vis[k + W];
  T visc = -P.iRe * L.ih * ((L.Av[k] * De - L.Av[k - 1] * Dw) + (vt * dyt - vb * dyb) +
                            (vt * dvt - vb * dvb) * T(1.0 / 3.0));
  if constexpr (PST) return r + visc + P.Fr_inv * L.Arv[k];
  return r + visc;
}
template <typename T>
__device__ __forceinline__ T op_v(const Prm<T>& P, const Lv<T>& L, int k) {
  return op_v(P, L, k, T(0.5) * (rho_of(P, L.c[k]) + rho_of(P, L.c[k + L.pitch])));
}

// ---------------------------------------------------------------------------
// projection method (Sec. 6.2): the iterate's u, v arrays hold the
// intermediate velocity; the new velocity follows from the projection
// equation (pj-num-pjx), A rho(c) (u - ut)/dt = -(1/M) D p + (1/M) ST(c, mu)
// [- (1/Fr) A_y rho(c) in y], ST the surface-tension pairing of (e1e1) at
// level n+1.  Gravity acts here, tested with u^{n+1} in the energy proof.
// ---------------------------------------------------------------------------
// u^{n+1} at edge (i+1/2, j), i = 0..m1; zero on no-slip walls
template <typename T>
__device__ __forceinline__ T proj_u(const Prm<T>& P, const Lv<T>& L, int i, int j) {
  if (!L.px && (i <= 0 || i >= L.m1)) return T(0);
  int k = L.at(i, j);
  T cl = L.c[k], cr = L.c[k + 1];
  T rl = rho_of(P, cl), rr = rho_of(P, cr);
  T Ar = T(0.5) * (rl + rr);
  T dp = (L.p[k + 1] - L.p[k]) * L.ih;
  T st = T(0.5) * (rr * L.mu[k] + rl * L.mu[k + 1]) * (cr - cl) * L.ih;
  return L.u[k] + (st - dp) * P.iM / (Ar * P.idt);
}
// v^{n+1} at edge (i, j+1/2), j = 0..m2; zero on the walls in y
template <typename T>
__device__ __forceinline__ T proj_v(const Prm<T>& P, const Lv<T>& L, int i, int j) {
  if (j <= 0 || j >= L.m2) return T(0);
  const int W = L.pitch;
  int k = L.at(i, j);
  T cb = L.c[k], ct = L.c[k + W];
  T rb = rho_of(P, cb), rt = rho_of(P, ct);
  T Ar = T(0.5) * (rb + rt);
  T dp = (L.p[k + W] - L.p[k]) * L.ih;
  T st = T(0.5) * (rt * L.mu[k] + rb * L.mu[k + W]) * (ct - cb) * L.ih;
  return L.v[k] + (st - dp) * P.iM / (Ar * P.idt) - P.Fr_inv / P.idt;
}
// The four face velocities u^{n+1} of cell (i,j) (E, W, N, S), from rho(c) of the
// cell (rk) and of its neighbours (rq[f] for k + 1, k - 1, k + W, k - W): the
// same values as proj_u / proj_v without re-evaluating the densities.
template <typename T>
__device__ __forceinline__ void proj_faces(const Prm<T>& P, const Lv<T>& L, int i, int j, T rk,
                                           const T (&rq)[4], T (&w)[4]) {
  const int W = L.pitch;
  int k = L.at(i, j);
  const T *c = L.c, *mu = L.mu, *p = L.p;
  const T g = P.Fr_inv / P.idt;
  // face between cells a (left/below) and b = a + off, velocity array at a
  auto face = [&](int a, int off, const T* vel, T ra, T rb, T grav) {
    T Ar = T(0.5) * (ra + rb);
    T dp = (p[a + off] - p[a]) * L.ih;
    T st = T(0.5) * (rb * mu[a] + ra * mu[a + off]) * (c[a + off] - c[a]) * L.ih;
    return vel[a] + (st - dp) * P.iM / (Ar * P.idt) - grav;
  };
  w[0] = (!L.px && i == L.m1) ? T(0) : face(k, 1, L.u, rk, rq[0], T(0));
  w[1] = (!L.px && i == 1) ? T(0) : face(k - 1, 1, L.u, rq[1], rk, T(0));
  w[2] = (j == L.m2) ? T(0) : face(k, W, L.v, rk, rq[2], g);
  w[3] = (j == 1) ? T(0) : face(k - W, W, L.v, rq[3], rk, g);
}
// (pj-num-phase): rho^n (c - c^n)/dt + a_x(rho_ew D_x c u^{n+1}) + a_y(...)
// - (1/Pe) grad_d.(A m^n grad_D mu) - (alpha/Pe) grad_d.(A m^n grad_D p), with
// rho = rho(c^{n+1}) and c^{n+1} in the advection; and (pj-num-mass): d_x u^{n+1}
// + d_y v^{n+1} - (alpha/Pe)(grad.(A m grad mu) + alpha grad.(A m grad p)).
// Both from the shared densities rq and the face velocities w of proj_faces.
template <typename T>
__device__ __forceinline__ T opp_c_w(const Prm<T>& P, const Lv<T>& L, int k, const T (&rq)[4],
                                     const T (&w)[4]) {
  const int W = L.pitch;
  const T* c = L.c;
  T ck = c[k];
  T t = L.rhon[k] * (ck - L.cn[k]) * P.idt;
  T ax = T(0.5) * (rq[0] * (c[k + 1] - ck) * L.ih * w[0] + rq[1] * (ck - c[k - 1]) * L.ih * w[1]);
  T ay = T(0.5) * (rq[2] * (c[k + W] - ck) * L.ih * w[2] + rq[3] * (ck - c[k - W]) * L.ih * w[3]);
  T diff = lap_h2(L.mobn, L.mu, k, W) + P.alpha * lap_h2(L.mobn, L.p, k, W);
  return t + ax + ay - P.iPe * L.ih2 * diff;
}
template <typename T>
__device__ __forceinline__ T opp_p_w(const Prm<T>& P, const Lv<T>& L, int k, const T (&w)[4]) {
  const int W = L.pitch;
  T dv = (w[0] - w[1] + w[2] - w[3]) * L.ih;
  T diff = lap_h2(L.mobn, L.mu, k, W) + P.alpha * lap_h2(L.mobn, L.p, k, W);
  return dv - P.alpha * P.iPe * L.ih2 * diff;
}

// (pj-num-chem): as (pm-num-chem) with rho^n in front of mu
template <typename T>
__device__ __forceinline__ T opp_mu(const Prm<T>& P, const Lv<T>& L, int k) {
  const int W = L.pitch;
  const T rq[4] = {rho_of(P, L.c[k + 1]), rho_of(P, L.c[k - 1]), rho_of(P, L.c[k + W]),
                   rho_of(P, L.c[k - W])};
  return op_mu_r(P, L, k, rho_of(P, L.c[k]), rq, L.rhon[k]);
}
template <typename T>
__device__ __forceinline__ T opp_u(const Prm<T>& P, const Lv<T>& L, int k) {
  return op_u<T, false>(P, L, k, T(0.5) * (rho_of(P, L.c[k]) + rho_of(P, L.c[k + 1])));
}
template <typename T>
__device__ __forceinline__ T opp_v(const Prm<T>& P, const Lv<T>& L, int k) {
  return op_v<T, false>(P, L, k, T(0.5) * (rho_of(P, L.c[k]) + rho_of(P, L.c[k + L.pitch])));
}

// ---------------------------------------------------------------------------
// stores that keep ghost copies consistent (App. A.6 boundary conditions)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void store_cell(const Lv<T>& L, T* a, int i, int j, T x) {
  const int W = L.pitch;
  int k = j * W + i;
  a[k] = x;
  if (i == 1) a[k + (L.px ? L.m1 : -1)] = x;       // ghost (m1+1, j) or (0, j)
  if (i == L.m1) a[k + (L.px ? -L.m1 : 1)] = x;    // ghost (0, j) or (m1+1, j)
  if (j == 1) a[k - W] = x;
  if (j == L.m2) a[k + W] = x;
}

template <typename T>
__device__ __forceinline__ void store_u(const Lv<T>& L, int e, int j, T x) {
  const int W = L.pitch;
  T* u = L.u;
  int cols[3] = {e, e, e};
  int n = 1;
  if (L.px) {
    if (e == L.m1) cols[n++] = 0;
    if (e == L.m1 - 1) cols[n++] = -1;
    if (e == 1) cols[n++] = L.m1 + 1;
  }
  for (int q = 0; q < n; ++q) {
    int k = j * W + cols[q];
    u[k] = x;
    if (j == 1) u[k - W] = -x;
    if (j == L.m2) u[k + W] = -x;
  }
}

template <typename T>
__device__ __forceinline__ void store_v(const Lv<T>& L, int i, int e, T x) {
  const int W = L.pitch;
  T* v = L.v;
  int k = e * W + i;
  v[k] = x;
  if (L.px) {
    if (i == L.m1) v[k - L.m1] = x;
    if (i == 1) v[k + L.m1] = x;
  } else {
    if (i == 1) v[k - 1] = -x;
    if (i == L.m1) v[k + 1] = -x;
  }
}

// ---------------------------------------------------------------------------
// error equation for defect correction: N_e(e) = N(X + e) - N(X) for the
// iterate e stored in c, mu, p, u, v of the level and the base X in Bc, Bmu, Bu,
// Bv.  Every nonlinear difference is written with the secant identities of
// Sec. 4.1 (rho(a) - rho(b) = r(a,b)(a-b), F(a) - F(b) = g(a,b)(a-b)) and the
// algebraic factorisations below, so that no term is a difference of two
// nearly equal numbers: in FP32 the result keeps the relative accuracy of e.
// ---------------------------------------------------------------------------

// r(a,b) = -alpha rho(a) rho(b)
template <typename T> __device__ __forceinline__ T rsec_(const Prm<T>& P, T ra, T rb) {
  return -P.alpha * ra * rb;
}
// g(a+e, b) - g(a, b) = e/4 [a(a-1) + b(b-1) + (2a - 1 + e)(a + b - 1 + e)]
template <typename T> __device__ __forceinline__ T dgsec(T a, T b, T e) {
  return T(0.25) * e * (a * (a - T(1)) + b * (b - T(1)) + (T(2) * a - T(1) + e) * (a + b - T(1) + e));
}

template <typename T>
__device__ __forceinline__ T opd_c(const Prm<T>& P, const Lv<T>& L, int k) {
  const int W = L.pitch;
  const T* cn = L.cn;
  const T* rn = L.rhon;
  T e = L.c[k], C = L.Bc[k];
  T rp = rho_of(P, C + e), rC = rho_of(P, C);
  (void)cn;
  T adv = rn[k + 1] * L.Tx[k] * L.u[k] + rn[k - 1] * L.Tx[k - 1] * L.u[k - 1] +
          rn[k + W] * L.Ty[k] * L.v[k] + rn[k - W] * L.Ty[k - W] * L.v[k - W];
  T diff = lap_h2(L.mobn, L.mu, k, W) + P.alpha * lap_h2(L.mobn, L.p, k, W);
  return e * (rp + rsec_(P, rp, rC) * L.Bdc[k]) * P.idt + adv - P.iPe * L.ih2 * diff;
}

template <typename T>
__device__ __forceinline__ T opd_mu(const Prm<T>& P, const Lv<T>& L, int k) {
  const int W = L.pitch;
  const T *e = L.c, *B = L.Bc, *cn = L.cn, *rn = L.rhon;
  T ek = e[k], Ck = B[k], cnk = cn[k], rnk = rn[k];
  T cp = Ck + ek;
  T rp = rho_of(P, cp), rC = rho_of(P, Ck);
  T dr = rsec_(P, rp, rC) * ek;             // rho(c') - rho(C)
  T rhp = T(0.5) * (rp + rnk);              // rho^{n+1/2} at c'
  T r_new = rsec_(P, rp, rnk);              // r(c', c^n)
  T d_r = -P.alpha * rnk * dr;              // r(c', c^n) - r(C, c^n)
  T dF = gsec(cp, Ck) * ek;                 // F(c') - F(C)
  T dbulk = rhp * dgsec(Ck, cnk, ek) + T(0.5) * dr * gsec(Ck, cnk) + T(0.5) * dF * r_new +
            T(0.5) * (Fdw(Ck) + Fdw(cnk)) * d_r;
  // G(c') - G(C) and G(C), both times h^2
  const int off[4] = {1, -1, W, -W};
  T dG = T(0), GC = T(0), ddiv = T(0);
  T chP = Ck + cnk;  // 2 c^{n+1/2} at C
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    int q = k + off[f];
    T dC = B[q] - Ck, de = e[q] - ek;
    dG += de * (T(2) * dC + de);
    GC += dC * dC;
    T rq = rho_of(P, B[q] + e[q]), rCq = rho_of(P, B[q]);
    T rhq = T(0.5) * (rq + rn[q]);
    T drq = rsec_(P, rq, rCq) * e[q];
    // div(A rho_h(c') grad(e/2)) + div(A d rho_h grad c^{n+1/2}(C)), per face
    ddiv += (rhp + rhq) * de + T(0.5) * (dr + drq) * ((B[q] + cn[q]) - chP);
  }
  dG *= T(0.5);
  GC *= T(0.5);
  T dgrad = T(0.25) * P.Lam * (dG * L.ih2 * r_new + (GC * L.ih2 + L.Gn[k]) * d_r);
  ddiv *= T(0.25) * L.ih2;
  return rp * L.mu[k] + dr * L.Bmu[k] - P.K * dbulk - dgrad + P.Lam * ddiv;
}

template <typename T>
__device__ __forceinline__ T opd_p(const Prm<T>& P, const Lv<T>& L, int k) { return op_p(P, L, k); }

// x row: the terms of op_u that are linear in (u, v, p, mu), applied to e, plus
// 1/2 (A_x rho(c') - A_x rho^n) e_u/dt + 1/2 A_x(rho(c') - rho(C)) U/dt
template <typename T>
__device__ __forceinline__ T opd_u(const Prm<T>& P, const Lv<T>& L, int k) {
  const int W = L.pitch;
  const T *u = L.u, *vis = L.visn, *rn = L.rhon;
  T ue = u[k];
  T cl = L.Bc[k] + L.c[k], cr = L.Bc[k + 1] + L.c[k + 1];
  T rpl = rho_of(P, cl), rpr = rho_of(P, cr);
  T Arp = T(0.5) * (rpl + rpr);
  T dAr = T(0.5) * (rsec_(P, rpl, rho_of(P, L.Bc[k])) * L.c[k] +
                    rsec_(P, rpr, rho_of(P, L.Bc[k + 1])) * L.c[k + 1]);
  T dxl = (ue - u[k - 1]) * L.ih, dxr = (u[k + 1] - ue) * L.ih;
  T dvl = dxl + (L.v[k] - L.v[k - W]) * L.ih;
  T dvr = dxr + (L.v[k + 1] - L.v[k + 1 - W]) * L.ih;
  T Dt = (u[k + W] - ue) * L.ih, Db = (ue - u[k - W]) * L.ih;
  T Arn = L.Aru[k];
  T conv = T(0.5) * (L.Sx[k + 1] * dxr + L.Sx[k] * dxl + L.Qx[k] * Dt + L.Qx[k - W] * Db);
  T time = Arn * ue * P.idt + T(0.5) * (Arp - Arn) * P.idt * ue + T(0.5) * dAr * P.idt * L.Bu[k] +
           L.Dvu[k] * ue;
  T press = (L.p[k + 1] - L.p[k]) * L.ih * P.iM;
  T st = -(rn[k + 1] * L.mu[k] + rn[k] * L.mu[k + 1]) * L.Tx[k] * P.iM;
  T vl = vis[k], vr = vis[k + 1];
  T visc = -P.iRe * L.ih * ((vr * dxr - vl * dxl) + (L.Av[k] * Dt - L.Av[k - W] * Db) +
                            (vr * dvr - vl * dvl) * T(1.0 / 3.0));
  return time + conv + press + st + visc;
}

template <typename T>
__device__ __forceinline__ T opd_v(const Prm<T>& P, const Lv<T>& L, int k) {
  const int W = L.pitch;
  const T *v = L.v, *vis = L.visn, *rn = L.rhon;
  T ve = v[k];
  T cb = L.Bc[k] + L.c[k], ct = L.Bc[k + W] + L.c[k + W];
  T rpb = rho_of(P, cb), rpt = rho_of(P, ct);
  T Arp = T(0.5) * (rpb + rpt);
  T dAr = T(0.5) * (rsec_(P, rpb, rho_of(P, L.Bc[k])) * L.c[k] +
                    rsec_(P, rpt, rho_of(P, L.Bc[k + W])) * L.c[k + W]);
  T dyb = (ve - v[k - W]) * L.ih, dyt = (v[k + W] - ve) * L.ih;
  T dvb = dyb + (L.u[k] - L.u[k - 1]) * L.ih;
  T dvt = dyt + (L.u[k + W] - L.u[k + W - 1]) * L.ih;
  T De = (v[k + 1] - ve) * L.ih, Dw = (ve - v[k - 1]) * L.ih;
  T Arn = L.Arv[k];
  T conv = T(0.5) * (L.Qy[k] * De + L.Qy[k - 1] * Dw + L.Sy[k + W] * dyt + L.Sy[k] * dyb);
  T time = Arn * ve * P.idt + T(0.5) * (Arp - Arn) * P.idt * ve + T(0.5) * dAr * P.idt * L.Bv[k] +
           L.Dvv[k] * ve;
  T press = (L.p[k + W] - L.p[k]) * L.ih * P.iM;
  T st = -(rn[k + W] * L.mu[k] + rn[k] * L.mu[k + W]) * L.Ty[k] * P.iM;
  T vb = vis[k], vt = vis[k + W];
  T visc = -P.iRe * L.ih * ((L.Av[k] * De - L.Av[k - 1] * Dw) + (vt * dyt - vb * dyb) +
                            (vt * dvt - vb * dvb) * T(1.0 / 3.0));
  return time + conv + press + st + visc;
}

// Two forms of the iterate: Full (x itself, Sec. 6.1) and Err (correction e to
// the base X of a defect-correction cycle).  val_c / val_mu return the full
// value c, mu that the local Jacobians of the smoothers are evaluated at.
struct FullForm {
  template <typename T> static __device__ __forceinline__ T val_c(const Lv<T>& L, int k) { return L.c[k]; }
  template <typename T> static __device__ __forceinline__ T rho(const Prm<T>&, const Lv<T>& L, int k) { return L.rhoc[k]; }
  template <typename T> static __device__ __forceinline__ T val_u(const Lv<T>& L, int k) { return L.u[k]; }
  template <typename T> static __device__ __forceinline__ T val_v(const Lv<T>& L, int k) { return L.v[k]; }
  template <typename T> static __device__ __forceinline__ T val_mu(const Lv<T>& L, int k) { return L.mu[k]; }
  template <typename T> static __device__ __forceinline__ T Nc(const Prm<T>& P, const Lv<T>& L, int k) { return op_c(P, L, k); }
  template <typename T> static __device__ __forceinline__ T Nmu(const Prm<T>& P, const Lv<T>& L, int k) { return op_mu(P, L, k); }
  template <typename T> static __device__ __forceinline__ T Np(const Prm<T>& P, const Lv<T>& L, int k) { return op_p(P, L, k); }
  template <typename T> static __device__ __forceinline__ T Nu(const Prm<T>& P, const Lv<T>& L, int k) { return op_u(P, L, k); }
  template <typename T> static __device__ __forceinline__ T Nv(const Prm<T>& P, const Lv<T>& L, int k) { return op_v(P, L, k); }
};
// The projection method on the full iterate (u, v arrays hold the intermediate
// velocity).  Its N_c and N_p need the cell's face velocities (proj_faces,
// which needs the cell index for the wall edges), so the kernels call
// opp_c_w / opp_p_w directly.
struct ProjForm {
  template <typename T> static __device__ __forceinline__ T val_c(const Lv<T>& L, int k) { return L.c[k]; }
  template <typename T> static __device__ __forceinline__ T rho(const Prm<T>&, const Lv<T>& L, int k) { return L.rhoc[k]; }
  template <typename T> static __device__ __forceinline__ T val_u(const Lv<T>& L, int k) { return L.u[k]; }
  template <typename T> static __device__ __forceinline__ T val_v(const Lv<T>& L, int k) { return L.v[k]; }
  template <typename T> static __device__ __forceinline__ T val_mu(const Lv<T>& L, int k) { return L.mu[k]; }
  template <typename T> static __device__ __forceinline__ T Nmu(const Prm<T>& P, const Lv<T>& L, int k) { return opp_mu(P, L, k); }
  template <typename T> static __device__ __forceinline__ T Nu(const Prm<T>& P, const Lv<T>& L, int k) { return opp_u(P, L, k); }
  template <typename T> static __device__ __forceinline__ T Nv(const Prm<T>& P, const Lv<T>& L, int k) { return opp_v(P, L, k); }
};
struct ErrForm {
  template <typename T> static __device__ __forceinline__ T val_c(const Lv<T>& L, int k) { return L.Bc[k] + L.c[k]; }
  template <typename T> static __device__ __forceinline__ T rho(const Prm<T>& P, const Lv<T>& L, int k) { return rho_of(P, val_c(L, k)); }
  template <typename T> static __device__ __forceinline__ T val_u(const Lv<T>& L, int k) { return L.Bu[k] + L.u[k]; }
  template <typename T> static __device__ __forceinline__ T val_v(const Lv<T>& L, int k) { return L.Bv[k] + L.v[k]; }
  template <typename T> static __device__ __forceinline__ T val_mu(const Lv<T>& L, int k) { return L.Bmu[k] + L.mu[k]; }
  template <typename T> static __device__ __forceinline__ T Nc(const Prm<T>& P, const Lv<T>& L, int k) { return opd_c(P, L, k); }
  template <typename T> static __device__ __forceinline__ T Nmu(const Prm<T>& P, const Lv<T>& L, int k) { return opd_mu(P, L, k); }
  template <typename T> static __device__ __forceinline__ T Np(const Prm<T>& P, const Lv<T>& L, int k) { return opd_p(P, L, k); }
  template <typename T> static __device__ __forceinline__ T Nu(const Prm<T>& P, const Lv<T>& L, int k) { return opd_u(P, L, k); }
  template <typename T> static __device__ __forceinline__ T Nv(const Prm<T>& P, const Lv<T>& L, int k) { return opd_v(P, L, k); }
};

}  // namespace qn
