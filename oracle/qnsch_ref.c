/*
 * qnsch_ref.c -- ORACLE: test infrastructure, not part of the product path.
 *
 * A plain, serial, FP64 CPU implementation of one implicit time step of the
 * primitive method of Guo, Lin, Lowengrub & Wise, "Mass conservative and energy
 * stable finite difference methods for the quasi-incompressible
 * Navier-Stokes-Cahn-Hilliard system" (arXiv:1703.06606):
 *   - fully discrete scheme: Sec. 6.1, Eqs. (pm-num-mx), (pm-num-mass),
 *     (pm-num-phase), (pm-num-chem), with the convective terms (e1e1-1),
 *     (e1e1-2), the surface tension (e1e1) and the CH advection (e1e2);
 *   - staggered-grid operators, inner products, norms and boundary conditions:
 *     Sec. 5 and Appendix A;
 *   - solver: Sec. 7.1 (CH nonlinear Gauss-Seidel, Vanka smoothing for the
 *     Navier-Stokes block, colour ordering, FAS V-cycle).
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.
 * It shares no code with the CUDA library.
 *
 * Readings of the paper that this file takes:
 *   R1 (e1e1-2): the divergence correction of the x-momentum row is
 *       1/2[D_x(rho a_x u^n) + Dfrak_y(Acal rho Acal_x v^n)] u, and of the
 *       y-row 1/2[Dfrak_x(Acal rho Acal_y u^n) + D_y(rho a_y v^n)] v; these are
 *       the pairings for which the skew-symmetry propositions of App. A hold.
 *   R2 (pm-num-chem): the gradient energy term is
 *       (eps eta M/(2We)) * 1/2 (G(c^{n+1}) + G(c^n)) r(c^{n+1},c^n), with the
 *       pointwise G(c) = a_x((D_x c)^2) + a_y((D_y c)^2), the time average of
 *       (grad c . grad c) used by the time-discrete scheme (mm-chem-1).
 *   R3 the mobility is m(c^n) = sqrt(c^2 (1-c)^2 + eps_m), eps_m = Cn.
 *   R4 M defaults to Cn (Sec. 8 sets M = eps in every example).
 *   R5 eta(rho1, rho2) from Sec. 8.1; at rho1 = rho2 the formula is 0/0 and the
 *       limit 3/(2 sqrt(2) rho1) is used (series for |rho2/rho1 - 1| < 0.1).
 *   R6 periodic edge data wrap with period m1 (u_{m1+1/2} = u_{1/2}).
 *   R7 smoother order: CH red-black, (i+j) mod 2; Vanka colours (i+2j) mod 5
 *       (walls in x), (2i+j) mod 8 (periodic x, m1 a multiple of 4) or
 *       (i+2j) mod K, K the smallest divisor >= 5 of m1 (other even periodic
 *       m1): any two cells whose 5x5 Vanka blocks couple are at L1 distance
 *       <= 2 and get distinct colours, also across the periodic seam.
 *   R8 transfers: cell data restricted by the 4-cell mean and prolongated
 *       piecewise constant; edge iterates restricted by the mean of the two
 *       coincident fine edges, edge residuals by full weighting (the transpose
 *       of the prolongation), edge corrections prolongated by coincidence /
 *       linear in the normal direction; coarse operator = the same scheme on the
 *       2h grid with restricted frozen data c^n, u^n, v^n; levels coarsen down
 *       to 2 cells (walls) or 4 cells (periodic x) in the shorter direction.
 *   R9 convergence: max over the five families of (h^2 sum r^2)^{1/2} <= tol;
 *       the mean of p is removed after every outer cycle.
 */
#include "qnsch_ref.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* parameters                                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
  double rho1, rho2, mu1, mu2; /* densities, viscosities of the two fluids */
  double Re, We, Pe, Cn, Fr_inv, M, eta, eps_m;
  double alpha; /* (rho2 - rho1)/(rho1 rho2), Sec. 2.1 */
  double K;     /* M eta / (eps We): coefficient of the bulk terms of (pm-num-chem) */
  double Lam;   /* eps eta M / We : coefficient of the gradient terms */
  int scheme;   /* 0: primitive method (Sec. 6.1); 1: projection method (Sec. 6.2) */
} ref_params;

/* rho(c) = rho1 rho2 / ((rho2 - rho1) c + rho1), Sec. 2.1 */
static double rho_of(const ref_params* P, double c) {
  return P->rho1 * P->rho2 / ((P->rho2 - P->rho1) * c + P->rho1);
}
/* viscosity mu(c) = mu1 mu2 / ((mu2 - mu1) c + mu1), Sec. 2.1 */
static double visc_of(const ref_params* P, double c) {
  return P->mu1 * P->mu2 / ((P->mu2 - P->mu1) * c + P->mu1);
}
/* regularised mobility, Sec. 6.1 (reading R3) */
static double mob_of(const ref_params* P, double c) {
  return sqrt(c * c * (1.0 - c) * (1.0 - c) + P->eps_m);
}
/* double well F(c) = c^2 (c-1)^2 / 4 and f = F', Sec. 2.1 */
static double Fdw(double c) { return 0.25 * c * c * (c - 1.0) * (c - 1.0); }
static double fdw(double c) { return c * (c - 1.0) * (c - 0.5); }
/* secant g(a,b) with F(a) - F(b) = g(a,b)(a-b), Sec. 4.1 */
static double gsec(double a, double b) {
  return 0.25 * (a * (a - 1.0) + b * (b - 1.0)) * (a + b - 1.0);
}
static double gsec_da(double a, double b) {
  return 0.25 * (2.0 * a - 1.0) * (a + b - 1.0) +
         0.25 * (a * (a - 1.0) + b * (b - 1.0));
}
/* secant r(a,b) = -alpha rho(a) rho(b) with rho(a) - rho(b) = r (a - b), (def-rhoal) */
static double rsec(const ref_params* P, double a, double b) {
  return -P->alpha * rho_of(P, a) * rho_of(P, b);
}

/* Surface-tension ratio eta(rho1, rho2), Sec. 8.1 (reading R5).  With
   x = rho2/rho1 = 1 + q,
     eta = (x-1)^3 / (2 sqrt2 rho1 x (x^2 - 1 - 2 x ln x)),
   and x^2 - 1 - 2x ln x = q^3 S(q), S(q) = sum_{n>=0} 2 (-1)^n q^n / ((n+2)(n+3))
   (from the Taylor series of ln(1+q)), so eta = 1 / (2 sqrt2 rho1 (1+q) S(q)).
   The series (24 terms) is used for |q| < 0.1, where the direct formula cancels. */
static double eta_of(double r1, double r2) {
  double q = r2 / r1 - 1.0;
  if (fabs(q) < 0.1) {
    double S = 0.0, qn = 1.0;
    for (int n = 0; n < 24; ++n) {
      S += 2.0 * ((n & 1) ? -1.0 : 1.0) * qn / ((n + 2.0) * (n + 3.0));
      qn *= q;
    }
    return 1.0 / (2.0 * sqrt(2.0) * r1 * (1.0 + q) * S);
  }
  double num = (r2 - r1) * (r2 - r1) * (r2 - r1);
  double den = 2.0 * sqrt(2.0) * r1 * r2 * (r2 * r2 - r1 * r1 - 2.0 * r1 * r2 * log(r2 / r1));
  return num / den;
}

static void derive_params(ref_params* P) {
  P->alpha = (P->rho2 - P->rho1) / (P->rho1 * P->rho2);
  P->K = P->M * P->eta / (P->Cn * P->We);
  P->Lam = P->Cn * P->eta * P->M / P->We;
}

/* ------------------------------------------------------------------------ */
/* grid storage                                                             */
/* ------------------------------------------------------------------------ */
/* Cell arrays: (m1+2) x (m2+2) with one ghost layer, entry (i,j), i,j = 0..m+1.
   u arrays: u_{i+1/2,j} for i = -1..m1+1, j = 0..m2+1.
   v arrays: v_{i,j+1/2} for i = 0..m1+1, j = -1..m2+1.                      */

typedef struct {
  int m1, m2, px;
  int kcol; /* number of Vanka colours on this level (reading R7) */
  double h;
  double *c, *mu, *p, *u, *v;       /* current iterate x */
  double *fc, *fmu, *fp, *fu, *fv;  /* FAS right-hand side f */
  double *rc, *rmu, *rp, *ru, *rv;  /* residual f - N(x) */
  double *sc, *smu, *sp, *su, *sv;  /* restricted iterate saved for the correction */
  double *cn, *un, *vn;             /* frozen level-n data */
  double *rhon, *mobn, *visn, *Gn;  /* rho(c^n), m(c^n), mu(c^n), G(c^n) */
} ref_level;

#define CI(L, i, j) ((size_t)(j) * (size_t)((L)->m1 + 2) + (size_t)(i))
#define UI(L, i, j) ((size_t)(j) * (size_t)((L)->m1 + 3) + (size_t)((i) + 1))
#define VI(L, i, j) ((size_t)((j) + 1) * (size_t)((L)->m1 + 2) + (size_t)(i))

static size_t ncell(const ref_level* L) { return (size_t)(L->m1 + 2) * (L->m2 + 2); }
static size_t nu_(const ref_level* L) { return (size_t)(L->m1 + 3) * (L->m2 + 2); }
static size_t nv_(const ref_level* L) { return (size_t)(L->m1 + 2) * (L->m2 + 3); }

/* first/last index of the u unknowns in x: walls exclude the boundary edges */
static int ulo(const ref_level* L) { (void)L; return 1; }
static int uhi(const ref_level* L) { return L->px ? L->m1 : L->m1 - 1; }

struct ref_solver {
  ref_params P;
  int nlev;
  ref_level* lev;
  int nu1, nu2, nuc, maxcyc, kcol, coupled;
  int nu1f, nu2f; /* smoothing steps on the finest level (-1: nu1, nu2) */
  double tol, omega, dt;
  int pending; /* 1 between begin_step and commit_step */
  /* committed state (finest level, ghosted) */
  double *c, *mu, *p, *u, *v;
  double last_res;
  /* option "predictor": the states committed 1 and 2 steps before the
     current one (ghosted, finest level), the sizes of the steps that left
     them, and how many are held; nhist = -1 while the committed state is the
     one the caller set (its mu and p are guesses, not a solution), which is
     then no node of the extrapolation either */
  int predictor, nhist;
  double hdt[2];
  double *hc[2], *hmu[2], *hp[2], *hu[2], *hv[2];
};

/* ------------------------------------------------------------------------ */
/* boundary conditions, App. A.6                                            */
/* ------------------------------------------------------------------------ */

/* cell-centred data: periodic or homogeneous Neumann in x (neubcx / pe-bcx),
   homogeneous Neumann in y (neubcy); corners follow from applying x then y */
static void bc_cell(const ref_level* L, double* a) {
  int m1 = L->m1, m2 = L->m2;
  for (int j = 1; j <= m2; ++j) {
    if (L->px) {
      a[CI(L, 0, j)] = a[CI(L, m1, j)];
      a[CI(L, m1 + 1, j)] = a[CI(L, 1, j)];
    } else {
      a[CI(L, 0, j)] = a[CI(L, 1, j)];
      a[CI(L, m1 + 1, j)] = a[CI(L, m1, j)];
    }
  }
  for (int i = 0; i <= m1 + 1; ++i) {
    a[CI(L, i, 0)] = a[CI(L, i, 1)];
    a[CI(L, i, m2 + 1)] = a[CI(L, i, m2)];
  }
}

/* east-west edge data: no-slip (u = 0 on x walls, a_y u = 0 on y walls through
   the reflected ghost, noslipbcx) or periodic in x (pecbcu, reading R6) */
static void bc_u(const ref_level* L, double* a) {
  int m1 = L->m1, m2 = L->m2;
  for (int j = 1; j <= m2; ++j) {
    if (L->px) {
      a[UI(L, 0, j)] = a[UI(L, m1, j)];
      a[UI(L, -1, j)] = a[UI(L, m1 - 1, j)];
      a[UI(L, m1 + 1, j)] = a[UI(L, 1, j)];
    } else {
      a[UI(L, 0, j)] = 0.0;
      a[UI(L, m1, j)] = 0.0;
      a[UI(L, -1, j)] = 0.0;
      a[UI(L, m1 + 1, j)] = 0.0;
    }
  }
  for (int i = -1; i <= m1 + 1; ++i) {
    a[UI(L, i, 0)] = -a[UI(L, i, 1)];
    a[UI(L, i, m2 + 1)] = -a[UI(L, i, m2)];
  }
}

/* north-south edge data: v = 0 on y walls (noslipbcy); in x either the
   reflected ghost (a_x v = 0 on x walls) or periodic (pecbcv) */
static void bc_v(const ref_level* L, double* a) {
  int m1 = L->m1, m2 = L->m2;
  for (int i = 1; i <= m1; ++i) {
    a[VI(L, i, 0)] = 0.0;
    a[VI(L, i, m2)] = 0.0;
    a[VI(L, i, -1)] = 0.0;
    a[VI(L, i, m2 + 1)] = 0.0;
  }
  for (int j = -1; j <= m2 + 1; ++j) {
    if (L->px) {
      a[VI(L, 0, j)] = a[VI(L, m1, j)];
      a[VI(L, m1 + 1, j)] = a[VI(L, 1, j)];
    } else {
      a[VI(L, 0, j)] = -a[VI(L, 1, j)];
      a[VI(L, m1 + 1, j)] = -a[VI(L, m1, j)];
    }
  }
}

static void bc_all(const ref_level* L) {
  bc_cell(L, L->c);
  bc_cell(L, L->mu);
  bc_cell(L, L->p);
  bc_u(L, L->u);
  bc_v(L, L->v);
}

/* ------------------------------------------------------------------------ */
/* frozen data: rho^n, m(c^n), mu(c^n), G(c^n) (Sec. 6.1)                   */
/* ------------------------------------------------------------------------ */

/* G(c)_{ij} = a_x((D_x c)^2) + a_y((D_y c)^2): the pointwise |grad_D c|^2 whose
   h^2-weighted rho-sum is ||sqrt(rho) grad_D c||_2^2 (App. A.7, reading R2) */
static double G_at(const ref_level* L, const double* c, int i, int j) {
  double h = L->h;
  double de = (c[CI(L, i + 1, j)] - c[CI(L, i, j)]) / h;
  double dw = (c[CI(L, i, j)] - c[CI(L, i - 1, j)]) / h;
  double dn = (c[CI(L, i, j + 1)] - c[CI(L, i, j)]) / h;
  double ds = (c[CI(L, i, j)] - c[CI(L, i, j - 1)]) / h;
  return 0.5 * (de * de + dw * dw) + 0.5 * (dn * dn + ds * ds);
}

static void frozen_derived(const ref_params* P, ref_level* L) {
  bc_cell(L, L->cn);
  bc_u(L, L->un);
  bc_v(L, L->vn);
  for (size_t k = 0; k < ncell(L); ++k) {
    L->rhon[k] = rho_of(P, L->cn[k]);
    L->mobn[k] = mob_of(P, L->cn[k]);
    L->visn[k] = visc_of(P, L->cn[k]);
  }
  for (int j = 1; j <= L->m2; ++j)
    for (int i = 1; i <= L->m1; ++i) L->Gn[CI(L, i, j)] = G_at(L, L->cn, i, j);
  bc_cell(L, L->Gn);
}

/* ------------------------------------------------------------------------ */
/* the discrete operator N(x) of Sec. 6.1, family by family                 */
/* ------------------------------------------------------------------------ */

/* grad_d . (A k grad_D phi) at cell (i,j): App. A.2 operators d, A, D */
static double div_A_grad(const ref_level* L, const double* k, const double* phi,
                         int i, int j) {
  double h2 = L->h * L->h;
  double fe = 0.5 * (k[CI(L, i + 1, j)] + k[CI(L, i, j)]) * (phi[CI(L, i + 1, j)] - phi[CI(L, i, j)]);
  double fw = 0.5 * (k[CI(L, i, j)] + k[CI(L, i - 1, j)]) * (phi[CI(L, i, j)] - phi[CI(L, i - 1, j)]);
  double fn = 0.5 * (k[CI(L, i, j + 1)] + k[CI(L, i, j)]) * (phi[CI(L, i, j + 1)] - phi[CI(L, i, j)]);
  double fs = 0.5 * (k[CI(L, i, j)] + k[CI(L, i, j - 1)]) * (phi[CI(L, i, j)] - phi[CI(L, i, j - 1)]);
  return (fe - fw + fn - fs) / h2;
}

/* (pm-num-phase) with the advection (e1e2) written out in App. A.4:
   N_c = rho(c)(c - c^n)/dt + a_x(rho^n_ew D_x c^n u) + a_y(rho^n_ns D_y c^n v)
         - (1/Pe) grad_d.(A m^n grad_D mu) - (alpha/Pe) grad_d.(A m^n grad_D p) */
static double N_c(const ref_params* P, const ref_level* L, double dt, int i, int j) {
  double h = L->h;
  const double *cn = L->cn, *rn = L->rhon;
  double c = L->c[CI(L, i, j)];
  double t = rho_of(P, c) * (c - cn[CI(L, i, j)]) / dt;
  double ax = 0.5 * (rn[CI(L, i + 1, j)] * (cn[CI(L, i + 1, j)] - cn[CI(L, i, j)]) / h * L->u[UI(L, i, j)] +
                     rn[CI(L, i - 1, j)] * (cn[CI(L, i, j)] - cn[CI(L, i - 1, j)]) / h * L->u[UI(L, i - 1, j)]);
  double ay = 0.5 * (rn[CI(L, i, j + 1)] * (cn[CI(L, i, j + 1)] - cn[CI(L, i, j)]) / h * L->v[VI(L, i, j)] +
                     rn[CI(L, i, j - 1)] * (cn[CI(L, i, j)] - cn[CI(L, i, j - 1)]) / h * L->v[VI(L, i, j - 1)]);
  double dmu = div_A_grad(L, L->mobn, L->mu, i, j);
  double dp = div_A_grad(L, L->mobn, L->p, i, j);
  return t + ax + ay - dmu / P->Pe - P->alpha / P->Pe * dp;
}

/* (pm-num-chem), reading R2:
   N_mu = rho(c) mu - K[rho^{n+1/2} g(c,c^n) + 1/2(F(c)+F(c^n)) r(c,c^n)]
          - (Lam/2) 1/2 (G(c) + G(c^n)) r(c,c^n)
          + Lam grad_d.(A rho^{n+1/2} grad_D c^{n+1/2}) */
static double N_mu(const ref_params* P, const ref_level* L, int i, int j) {
  double h2 = L->h * L->h;
  double c = L->c[CI(L, i, j)], cn = L->cn[CI(L, i, j)];
  double rho = rho_of(P, c), rhon = L->rhon[CI(L, i, j)];
  double rhalf = 0.5 * (rho + rhon);
  double r = rsec(P, c, cn);
  double bulk = rhalf * gsec(c, cn) + 0.5 * (Fdw(c) + Fdw(cn)) * r;
  double grad = 0.25 * P->Lam * (G_at(L, L->c, i, j) + L->Gn[CI(L, i, j)]) * r;
  /* grad_d . (A rho^{n+1/2} grad_D c^{n+1/2}) */
  static const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
  double div = 0.0;
  for (int f = 0; f < 4; ++f) {
    int a = i + di[f], b = j + dj[f];
    double rb = 0.5 * (rho_of(P, L->c[CI(L, a, b)]) + L->rhon[CI(L, a, b)]);
    double chb = 0.5 * (L->c[CI(L, a, b)] + L->cn[CI(L, a, b)]);
    double chp = 0.5 * (c + cn);
    div += 0.5 * (rhalf + rb) * (chb - chp);
  }
  div /= h2;
  /* (pj-num-chem) of the projection method has rho^n mu on the left */
  double rmu = P->scheme ? rhon : rho;
  return rmu * L->mu[CI(L, i, j)] - P->K * bulk - grad + P->Lam * div;
}

/* (pm-num-mass): N_p = d_x u + d_y v - (alpha/Pe) grad_d.(A m^n grad_D mu)
                         - (alpha^2/Pe) grad_d.(A m^n grad_D p) */
static double N_p(const ref_params* P, const ref_level* L, int i, int j) {
  double h = L->h;
  double du = (L->u[UI(L, i, j)] - L->u[UI(L, i - 1, j)]) / h;
  double dv = (L->v[VI(L, i, j)] - L->v[VI(L, i, j - 1)]) / h;
  double dmu = div_A_grad(L, L->mobn, L->mu, i, j);
  double dp = div_A_grad(L, L->mobn, L->p, i, j);
  return du + dv - P->alpha / P->Pe * dmu - P->alpha * P->alpha / P->Pe * dp;
}

/* index of the u unknown at x-edge index e (periodic: edge 0 is edge m1) */
static int uwrap(const ref_level* L, int e) { return (L->px && e == 0) ? L->m1 : e; }

/* centre-to-vertex average Acal phi at vertex (i+1/2, j+1/2), App. A.2 */
static double Avtx(const ref_level* L, const double* a, int i, int j) {
  return 0.25 * (a[CI(L, i, j)] + a[CI(L, i + 1, j)] + a[CI(L, i, j + 1)] + a[CI(L, i + 1, j + 1)]);
}

/* x row of (pm-num-mx) at edge (i+1/2, j), with (e1e1-1), (e1e1-2) [reading R1]
   and (e1e1) written out in App. A.5:
   N_u = A_x rho^n (u - u^n)/dt + A_x(rho^n a_x u^n d_x u) + Afrak_y(Acal rho^n Acal_x v^n Dcal_y u)
       + (A_x rho - A_x rho^n) u/(2dt) + 1/2[D_x(rho^n a_x u^n) + Dfrak_y(Acal rho^n Acal_x v^n)] u
       + (1/M) D_x p - (1/M) 1/2(rho^n_{i+1} mu_i + rho^n_i mu_{i+1}) D_x c^n
       - (1/Re)[D_x(mu^n d_x u) + Dfrak_y(Acal mu^n Dcal_y u)] - (1/(3Re)) D_x(mu^n (d_x u + d_y v)) */
static double N_u(const ref_params* P, const ref_level* L, double dt, int i, int j) {
  double h = L->h;
  const double *u = L->u, *un = L->un, *v = L->v, *vn = L->vn, *rn = L->rhon, *vis = L->visn;
  double ue = u[UI(L, i, j)];
  double Arn = 0.5 * (rn[CI(L, i, j)] + rn[CI(L, i + 1, j)]);
  double Ar = 0.5 * (rho_of(P, L->c[CI(L, i, j)]) + rho_of(P, L->c[CI(L, i + 1, j)]));
  /* cell quantities of the two cells i and i+1 adjacent to the edge */
  double axun_l = 0.5 * (un[UI(L, i, j)] + un[UI(L, i - 1, j)]);
  double axun_r = 0.5 * (un[UI(L, i + 1, j)] + un[UI(L, i, j)]);
  double dxu_l = (u[UI(L, i, j)] - u[UI(L, i - 1, j)]) / h;
  double dxu_r = (u[UI(L, i + 1, j)] - u[UI(L, i, j)]) / h;
  double divu_l = dxu_l + (v[VI(L, i, j)] - v[VI(L, i, j - 1)]) / h;
  double divu_r = dxu_r + (v[VI(L, i + 1, j)] - v[VI(L, i + 1, j - 1)]) / h;
  /* vertex quantities at (i+1/2, j+1/2) [top] and (i+1/2, j-1/2) [bottom] */
  double Ar_t = Avtx(L, rn, i, j), Ar_b = Avtx(L, rn, i, j - 1);
  double Av_t = Avtx(L, vis, i, j), Av_b = Avtx(L, vis, i, j - 1);
  double Axvn_t = 0.5 * (vn[VI(L, i + 1, j)] + vn[VI(L, i, j)]);
  double Axvn_b = 0.5 * (vn[VI(L, i + 1, j - 1)] + vn[VI(L, i, j - 1)]);
  double Dyu_t = (u[UI(L, i, j + 1)] - u[UI(L, i, j)]) / h;
  double Dyu_b = (u[UI(L, i, j)] - u[UI(L, i, j - 1)]) / h;

  double rl = rn[CI(L, i, j)], rr = rn[CI(L, i + 1, j)];
  double t_time = Arn * (ue - un[UI(L, i, j)]) / dt;
  double t_convx = 0.5 * (rr * axun_r * dxu_r + rl * axun_l * dxu_l);
  double t_convy = 0.5 * (Ar_t * Axvn_t * Dyu_t + Ar_b * Axvn_b * Dyu_b);
  double t_rho = (Ar - Arn) / (2.0 * dt) * ue;
  double t_div = 0.5 * ((rr * axun_r - rl * axun_l) / h + (Ar_t * Axvn_t - Ar_b * Axvn_b) / h) * ue;
  double t_p = (L->p[CI(L, i + 1, j)] - L->p[CI(L, i, j)]) / (P->M * h);
  double t_st = -0.5 * (rr * L->mu[CI(L, i, j)] + rl * L->mu[CI(L, i + 1, j)]) *
                (L->cn[CI(L, i + 1, j)] - L->cn[CI(L, i, j)]) / h / P->M;
  double t_visc = -((vis[CI(L, i + 1, j)] * dxu_r - vis[CI(L, i, j)] * dxu_l) / h +
                    (Av_t * Dyu_t - Av_b * Dyu_b) / h) / P->Re;
  double t_visc3 = -(vis[CI(L, i + 1, j)] * divu_r - vis[CI(L, i, j)] * divu_l) / h / (3.0 * P->Re);
  /* (pj-num-mx) of the projection method: the intermediate velocity's row has
     no pressure and no surface tension (they act in (pj-num-pjx)) */
  if (P->scheme) t_p = t_st = 0.0;
  return t_time + t_convx + t_convy + t_rho + t_div + t_p + t_st + t_visc + t_visc3;
}

/* y row of (pm-num-mx) at edge (i, j+1/2): mirror of N_u plus gravity (1/Fr) A_y rho^n */
static double N_v(const ref_params* P, const ref_level* L, double dt, int i, int j) {
  double h = L->h;
  const double *v = L->v, *vn = L->vn, *u = L->u, *un = L->un, *rn = L->rhon, *vis = L->visn;
  double ve = v[VI(L, i, j)];
  double Arn = 0.5 * (rn[CI(L, i, j)] + rn[CI(L, i, j + 1)]);
  double Ar = 0.5 * (rho_of(P, L->c[CI(L, i, j)]) + rho_of(P, L->c[CI(L, i, j + 1)]));
  double ayvn_b = 0.5 * (vn[VI(L, i, j)] + vn[VI(L, i, j - 1)]);
  double ayvn_t = 0.5 * (vn[VI(L, i, j + 1)] + vn[VI(L, i, j)]);
  double dyv_b = (v[VI(L, i, j)] - v[VI(L, i, j - 1)]) / h;
  double dyv_t = (v[VI(L, i, j + 1)] - v[VI(L, i, j)]) / h;
  double divu_b = (u[UI(L, i, j)] - u[UI(L, i - 1, j)]) / h + dyv_b;
  double divu_t = (u[UI(L, i, j + 1)] - u[UI(L, i - 1, j + 1)]) / h + dyv_t;
  /* vertices (i+1/2, j+1/2) [east] and (i-1/2, j+1/2) [west] */
  double Ar_e = Avtx(L, rn, i, j), Ar_w = Avtx(L, rn, i - 1, j);
  double Av_e = Avtx(L, vis, i, j), Av_w = Avtx(L, vis, i - 1, j);
  double Ayun_e = 0.5 * (un[UI(L, i, j + 1)] + un[UI(L, i, j)]);
  double Ayun_w = 0.5 * (un[UI(L, i - 1, j + 1)] + un[UI(L, i - 1, j)]);
  double Dxv_e = (v[VI(L, i + 1, j)] - v[VI(L, i, j)]) / h;
  double Dxv_w = (v[VI(L, i, j)] - v[VI(L, i - 1, j)]) / h;

  double rb = rn[CI(L, i, j)], rt = rn[CI(L, i, j + 1)];
  double t_time = Arn * (ve - vn[VI(L, i, j)]) / dt;
  double t_convx = 0.5 * (Ar_e * Ayun_e * Dxv_e + Ar_w * Ayun_w * Dxv_w);
  double t_convy = 0.5 * (rt * ayvn_t * dyv_t + rb * ayvn_b * dyv_b);
  double t_rho = (Ar - Arn) / (2.0 * dt) * ve;
  double t_div = 0.5 * ((Ar_e * Ayun_e - Ar_w * Ayun_w) / h + (rt * ayvn_t - rb * ayvn_b) / h) * ve;
  double t_p = (L->p[CI(L, i, j + 1)] - L->p[CI(L, i, j)]) / (P->M * h);
  double t_st = -0.5 * (rt * L->mu[CI(L, i, j)] + rb * L->mu[CI(L, i, j + 1)]) *
                (L->cn[CI(L, i, j + 1)] - L->cn[CI(L, i, j)]) / h / P->M;
  double t_visc = -((Av_e * Dxv_e - Av_w * Dxv_w) / h +
                    (vis[CI(L, i, j + 1)] * dyv_t - vis[CI(L, i, j)] * dyv_b) / h) / P->Re;
  double t_visc3 = -(vis[CI(L, i, j + 1)] * divu_t - vis[CI(L, i, j)] * divu_b) / h / (3.0 * P->Re);
  double t_grav = P->Fr_inv * Arn;
  /* projection method: pressure, surface tension and gravity act in the
     projection equation (reading R24) */
  if (P->scheme) t_p = t_st = t_grav = 0.0;
  return t_time + t_convx + t_convy + t_rho + t_div + t_p + t_st + t_visc + t_visc3 + t_grav;
}

/* ---- projection method (Sec. 6.2) ----------------------------------------
   The unknowns of a step are c, mu, p and the intermediate velocity (ut, vt),
   held in the u, v arrays of every level (same staggering, no-slip ghosts).
   The new velocity follows from the projection equation (pj-num-pjx),
     A rho(c) (u - ut)/dt = -(1/M) D p + (1/M) rho mu D c  [- (1/Fr) A_y rho(c) in y],
   with rho = rho(c^{n+1}) and the surface-tension pairing of (e1e1) at level
   n+1: 1/2 (rho_{i+1} mu_i + rho_i mu_{i+1}) D_x c.  Gravity sits in this
   equation, tested with u^{n+1} in the energy proof (reading R24). */

/* u^{n+1} at x-edge e (u_{e+1/2,j}); 0 on no-slip walls */
static double proj_u(const ref_params* P, const ref_level* L, double dt, int e, int j) {
  if (!L->px && (e <= 0 || e >= L->m1)) return 0.0;
  e = uwrap(L, e);
  double h = L->h;
  double cl = L->c[CI(L, e, j)], cr = L->c[CI(L, e + 1, j)];
  double rl = rho_of(P, cl), rr = rho_of(P, cr);
  double Ar = 0.5 * (rl + rr);
  double dp = (L->p[CI(L, e + 1, j)] - L->p[CI(L, e, j)]) / h;
  double st = 0.5 * (rr * L->mu[CI(L, e, j)] + rl * L->mu[CI(L, e + 1, j)]) * (cr - cl) / h;
  return L->u[UI(L, e, j)] + dt / Ar * (st - dp) / P->M;
}

/* v^{n+1} at y-edge e (v_{i,e+1/2}); 0 on the walls in y */
static double proj_v(const ref_params* P, const ref_level* L, double dt, int i, int e) {
  if (e <= 0 || e >= L->m2) return 0.0;
  double h = L->h;
  double cb = L->c[CI(L, i, e)], ct = L->c[CI(L, i, e + 1)];
  double rb = rho_of(P, cb), rt = rho_of(P, ct);
  double Ar = 0.5 * (rb + rt);
  double dp = (L->p[CI(L, i, e + 1)] - L->p[CI(L, i, e)]) / h;
  double st = 0.5 * (rt * L->mu[CI(L, i, e)] + rb * L->mu[CI(L, i, e + 1)]) * (ct - cb) / h;
  return L->v[VI(L, i, e)] + dt / Ar * (st - dp) / P->M - dt * P->Fr_inv;
}

/* (pj-num-phase): rho^n (c - c^n)/dt + a_x(rho_ew D_x c u^{n+1}) + a_y(rho_ns D_y c v^{n+1})
   - (1/Pe) grad_d.(A m^n grad_D mu) - (alpha/Pe) grad_d.(A m^n grad_D p),
   with rho = rho(c^{n+1}) and c = c^{n+1} in the advection (the (e1e2) form) */
static double Np_c(const ref_params* P, const ref_level* L, double dt, int i, int j) {
  double h = L->h;
  const double* c = L->c;
  double ck = c[CI(L, i, j)];
  double t = L->rhon[CI(L, i, j)] * (ck - L->cn[CI(L, i, j)]) / dt;
  double ax = 0.5 * (rho_of(P, c[CI(L, i + 1, j)]) * (c[CI(L, i + 1, j)] - ck) / h * proj_u(P, L, dt, i, j) +
                     rho_of(P, c[CI(L, i - 1, j)]) * (ck - c[CI(L, i - 1, j)]) / h * proj_u(P, L, dt, i - 1, j));
  double ay = 0.5 * (rho_of(P, c[CI(L, i, j + 1)]) * (c[CI(L, i, j + 1)] - ck) / h * proj_v(P, L, dt, i, j) +
                     rho_of(P, c[CI(L, i, j - 1)]) * (ck - c[CI(L, i, j - 1)]) / h * proj_v(P, L, dt, i, j - 1));
  double dmu = div_A_grad(L, L->mobn, L->mu, i, j);
  double dp = div_A_grad(L, L->mobn, L->p, i, j);
  return t + ax + ay - dmu / P->Pe - P->alpha / P->Pe * dp;
}

/* (pj-num-mass): d_x u^{n+1} + d_y v^{n+1} - (alpha/Pe) grad_d.(A m^n grad_D mu)
                  - (alpha^2/Pe) grad_d.(A m^n grad_D p) */
static double Np_p(const ref_params* P, const ref_level* L, double dt, int i, int j) {
  double h = L->h;
  double du = (proj_u(P, L, dt, i, j) - proj_u(P, L, dt, i - 1, j)) / h;
  double dv = (proj_v(P, L, dt, i, j) - proj_v(P, L, dt, i, j - 1)) / h;
  double dmu = div_A_grad(L, L->mobn, L->mu, i, j);
  double dp = div_A_grad(L, L->mobn, L->p, i, j);
  return du + dv - P->alpha / P->Pe * dmu - P->alpha * P->alpha / P->Pe * dp;
}

/* the cell families of the scheme in use */
static double Ncell_c(const ref_params* P, const ref_level* L, double dt, int i, int j) {
  return P->scheme ? Np_c(P, L, dt, i, j) : N_c(P, L, dt, i, j);
}
static double Ncell_p(const ref_params* P, const ref_level* L, double dt, int i, int j) {
  return P->scheme ? Np_p(P, L, dt, i, j) : N_p(P, L, i, j);
}

/* residual r = f - N(x) on all unknowns of a level; optional norms
   norms10 = [ (h^2 sum r^2)^{1/2} for c, mu, p, u, v ; max |r| for c, mu, p, u, v ] */
static void residual(const ref_params* P, ref_level* L, double dt, double* norms10) {
  double s[5] = {0, 0, 0, 0, 0}, mx[5] = {0, 0, 0, 0, 0};
  for (int j = 1; j <= L->m2; ++j)
    for (int i = 1; i <= L->m1; ++i) {
      size_t k = CI(L, i, j);
      L->rc[k] = L->fc[k] - Ncell_c(P, L, dt, i, j);
      L->rmu[k] = L->fmu[k] - N_mu(P, L, i, j);
      L->rp[k] = L->fp[k] - Ncell_p(P, L, dt, i, j);
      double a[3] = {L->rc[k], L->rmu[k], L->rp[k]};
      for (int q = 0; q < 3; ++q) {
        s[q] += a[q] * a[q];
        if (fabs(a[q]) > mx[q]) mx[q] = fabs(a[q]);
      }
    }
  for (int j = 1; j <= L->m2; ++j)
    for (int i = ulo(L); i <= uhi(L); ++i) {
      size_t k = UI(L, i, j);
      L->ru[k] = L->fu[k] - N_u(P, L, dt, i, j);
      s[3] += L->ru[k] * L->ru[k];
      if (fabs(L->ru[k]) > mx[3]) mx[3] = fabs(L->ru[k]);
    }
  for (int j = 1; j <= L->m2 - 1; ++j)
    for (int i = 1; i <= L->m1; ++i) {
      size_t k = VI(L, i, j);
      L->rv[k] = L->fv[k] - N_v(P, L, dt, i, j);
      s[4] += L->rv[k] * L->rv[k];
      if (fabs(L->rv[k]) > mx[4]) mx[4] = fabs(L->rv[k]);
    }
  if (norms10) {
    for (int q = 0; q < 5; ++q) {
      norms10[q] = sqrt(L->h * L->h * s[q]);
      norms10[5 + q] = mx[q];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* smoothers, Sec. 7.1                                                      */
/* ------------------------------------------------------------------------ */

/* copy cell (i,j) of a cell array into the ghosts that mirror it */
static void sync_cell(const ref_level* L, double* a, int i, int j) {
  int m1 = L->m1, m2 = L->m2;
  double x = a[CI(L, i, j)];
  if (i == 1) a[CI(L, L->px ? m1 + 1 : 0, j)] = x;
  if (i == m1) a[CI(L, L->px ? 0 : m1 + 1, j)] = x;
  if (j == 1) a[CI(L, i, 0)] = x;
  if (j == m2) a[CI(L, i, m2 + 1)] = x;
}

/* a Neumann wall face of cell (i,j) in direction f (0:E 1:W 2:N 3:S)? */
static int wall_face(const ref_level* L, int i, int j, int f) {
  if (f == 0) return !L->px && i == L->m1;
  if (f == 1) return !L->px && i == 1;
  if (f == 2) return j == L->m2;
  return j == 1;
}

/* 2x2 Jacobian of (N_c, N_mu) with respect to (c_ij, mu_ij), neighbours fixed;
   ghost cells follow their interior cell, so Neumann wall faces contribute 0 */
static void ch_jac(const ref_params* P, const ref_level* L, double dt, int i, int j, double J[4]) {
  static const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
  double h2 = L->h * L->h;
  double c = L->c[CI(L, i, j)], cn = L->cn[CI(L, i, j)], mu = L->mu[CI(L, i, j)];
  double rho = rho_of(P, c), drho = -P->alpha * rho * rho; /* rho' = -alpha rho^2 */
  double rhon = L->rhon[CI(L, i, j)];
  double rhalf = 0.5 * (rho + rhon), chp = 0.5 * (c + cn);
  double r = rsec(P, c, cn), dr = -P->alpha * drho * rhon;
  double g = gsec(c, cn), dg = gsec_da(c, cn);
  double sm = 0.0, dG = 0.0, ddiv = 0.0;
  for (int f = 0; f < 4; ++f) {
    if (wall_face(L, i, j, f)) continue;
    int a = i + di[f], b = j + dj[f];
    sm += 0.5 * (L->mobn[CI(L, i, j)] + L->mobn[CI(L, a, b)]);
    dG += (c - L->c[CI(L, a, b)]) / h2;
    double rb = 0.5 * (rho_of(P, L->c[CI(L, a, b)]) + L->rhon[CI(L, a, b)]);
    double chb = 0.5 * (L->c[CI(L, a, b)] + L->cn[CI(L, a, b)]);
    ddiv += 0.25 * drho * (chb - chp) - 0.25 * (rhalf + rb);
  }
  ddiv /= h2;
  double Gsum = G_at(L, L->c, i, j) + L->Gn[CI(L, i, j)];
  double dbulk = 0.5 * drho * g + rhalf * dg + 0.5 * fdw(c) * r + 0.5 * (Fdw(c) + Fdw(cn)) * dr;
  double dgrad = 0.25 * P->Lam * (dG * r + Gsum * dr);
  J[0] = (rho + drho * (c - cn)) / dt;
  J[1] = sm / (P->Pe * h2);
  J[2] = drho * mu - P->K * dbulk - dgrad + P->Lam * ddiv;
  J[3] = rho;
  if (P->scheme) {
    /* projection method: rho^n in the time derivative and in front of mu; the
       advection a(rho(c) D c u^{n+1}) differentiated in c_ij through D c only,
       with rho(c) of the neighbours and u^{n+1} held at the iterate (a choice
       of smoother; the fixed point is the scheme's) */
    double ue = proj_u(P, L, dt, i, j), uw = proj_u(P, L, dt, i - 1, j);
    double vn_ = proj_v(P, L, dt, i, j), vs = proj_v(P, L, dt, i, j - 1);
    double h = L->h;
    J[0] = rhon / dt + 0.5 * (-rho_of(P, L->c[CI(L, i + 1, j)]) * ue + rho_of(P, L->c[CI(L, i - 1, j)]) * uw) / h +
           0.5 * (-rho_of(P, L->c[CI(L, i, j + 1)]) * vn_ + rho_of(P, L->c[CI(L, i, j - 1)]) * vs) / h;
    J[2] = -P->K * dbulk - dgrad + P->Lam * ddiv;
    J[3] = rhon;
  }
}


/* write u_{e+1/2,j} and every ghost that mirrors it */
static void set_u(const ref_level* L, double* u, int e, int j, double x) {
  int m1 = L->m1, m2 = L->m2;
  int cols[3], nc = 0;
  cols[nc++] = e;
  if (L->px) {
    if (e == m1) cols[nc++] = 0;
    if (e == m1 - 1) cols[nc++] = -1;
    if (e == 1) cols[nc++] = m1 + 1;
  }
  for (int q = 0; q < nc; ++q) {
    u[UI(L, cols[q], j)] = x;
    if (j == 1) u[UI(L, cols[q], 0)] = -x;
    if (j == m2) u[UI(L, cols[q], m2 + 1)] = -x;
  }
}

/* write v_{i,e+1/2} and every ghost that mirrors it */
static void set_v(const ref_level* L, double* v, int i, int e, double x) {
  int m1 = L->m1;
  v[VI(L, i, e)] = x;
  if (L->px) {
    if (i == m1) v[VI(L, 0, e)] = x;
    if (i == 1) v[VI(L, m1 + 1, e)] = x;
  } else {
    if (i == 1) v[VI(L, 0, e)] = -x;
    if (i == m1) v[VI(L, m1 + 1, e)] = -x;
  }
}

/* The 5x5 Vanka block of cell (i,j) (Sec. 7.1 step 2): unknowns
   0:u_{i-1/2,j} 1:u_{i+1/2,j} 2:v_{i,j-1/2} 3:v_{i,j+1/2} 4:p_ij, equations
   N_u at the two x-edges, N_v at the two y-edges, N_p at the cell.  The NS
   block is affine in (u,v,p) for fixed (c,mu), so J is its exact Jacobian.
   A wall edge is not an unknown: its row and column are marked inactive.
   Reflected ghosts of an unknown (no-slip) double its weight in the
   tangential difference at the wall (gfac = 2). */
static void vanka_block(const ref_params* P, const ref_level* L, double dt, int i, int j,
                        double J[25], double R[5], int act[5]) {
  double h = L->h, h2 = h * h, iRe = 1.0 / P->Re;
  const double *rn = L->rhon, *vis = L->visn, *un = L->un, *vn = L->vn;
  int eW = uwrap(L, i - 1), eE = i;
  act[0] = L->px || i > 1;
  act[1] = L->px || i < L->m1;
  act[2] = j > 1;
  act[3] = j < L->m2;
  act[4] = 1;
  memset(J, 0, 25 * sizeof(double));
  /* x-edge equations: q = 0 (west edge, index eW), q = 1 (east edge, index eE) */
  for (int q = 0; q < 2; ++q) {
    int e = q == 0 ? eW : eE;
    /* diagonal of N_u at edge e: cells e (left) and e+1 (right) */
    double rl = rn[CI(L, e, j)], rr = rn[CI(L, e + 1, j)];
    double axl = 0.5 * (un[UI(L, e, j)] + un[UI(L, e - 1, j)]);
    double axr = 0.5 * (un[UI(L, e + 1, j)] + un[UI(L, e, j)]);
    double Arn = 0.5 * (rl + rr);
    double Ar = 0.5 * (rho_of(P, L->c[CI(L, e, j)]) + rho_of(P, L->c[CI(L, e + 1, j)]));
    double Art = Avtx(L, rn, e, j), Arb = Avtx(L, rn, e, j - 1);
    double Avt = Avtx(L, vis, e, j), Avb = Avtx(L, vis, e, j - 1);
    double At = 0.5 * (vn[VI(L, e + 1, j)] + vn[VI(L, e, j)]);
    double Ab = 0.5 * (vn[VI(L, e + 1, j - 1)] + vn[VI(L, e, j - 1)]);
    double gt = (j == L->m2) ? 2.0 : 1.0, gb = (j == 1) ? 2.0 : 1.0;
    double vl = vis[CI(L, e, j)], vr = vis[CI(L, e + 1, j)];
    double d = Arn / dt + 0.5 * (-rr * axr + rl * axl) / h + 0.5 * (-Art * At * gt + Arb * Ab * gb) / h +
               (Ar - Arn) / (2.0 * dt) + 0.5 * ((rr * axr - rl * axl) / h + (Art * At - Arb * Ab) / h) +
               iRe * ((vr + vl) / h2 + (gt * Avt + gb * Avb) / h2) + (vr + vl) / (3.0 * P->Re * h2);
    J[q * 5 + q] = d;
  }
  /* couplings through cell (i,j): it is the right cell of the west edge and the
     left cell of the east edge */
  {
    double rc = rn[CI(L, i, j)], vc = vis[CI(L, i, j)];
    double axc = 0.5 * (un[UI(L, i, j)] + un[UI(L, i - 1, j)]);
    J[0 * 5 + 1] = 0.5 * rc * axc / h - vc * iRe / h2 - vc / (3.0 * P->Re * h2);
    J[1 * 5 + 0] = -0.5 * rc * axc / h - vc * iRe / h2 - vc / (3.0 * P->Re * h2);
    J[0 * 5 + 3] = -vc / (3.0 * P->Re * h2);
    J[0 * 5 + 2] = +vc / (3.0 * P->Re * h2);
    J[1 * 5 + 3] = +vc / (3.0 * P->Re * h2);
    J[1 * 5 + 2] = -vc / (3.0 * P->Re * h2);
    J[0 * 5 + 4] = 1.0 / (P->M * h);
    J[1 * 5 + 4] = -1.0 / (P->M * h);
  }
  /* y-edge equations: q = 2 (south edge j-1), q = 3 (north edge j) */
  for (int q = 2; q < 4; ++q) {
    int e = q == 2 ? j - 1 : j;
    double rb = rn[CI(L, i, e)], rt = rn[CI(L, i, e + 1)];
    double ayb = 0.5 * (vn[VI(L, i, e)] + vn[VI(L, i, e - 1)]);
    double ayt = 0.5 * (vn[VI(L, i, e + 1)] + vn[VI(L, i, e)]);
    double Arn = 0.5 * (rb + rt);
    double Ar = 0.5 * (rho_of(P, L->c[CI(L, i, e)]) + rho_of(P, L->c[CI(L, i, e + 1)]));
    double Are = Avtx(L, rn, i, e), Arw = Avtx(L, rn, i - 1, e);
    double Ave = Avtx(L, vis, i, e), Avw = Avtx(L, vis, i - 1, e);
    double Ae = 0.5 * (un[UI(L, i, e + 1)] + un[UI(L, i, e)]);
    double Aw = 0.5 * (un[UI(L, i - 1, e + 1)] + un[UI(L, i - 1, e)]);
    double ge = (!L->px && i == L->m1) ? 2.0 : 1.0, gw = (!L->px && i == 1) ? 2.0 : 1.0;
    double vb = vis[CI(L, i, e)], vt = vis[CI(L, i, e + 1)];
    double d = Arn / dt + 0.5 * (-Are * Ae * ge + Arw * Aw * gw) / h + 0.5 * (-rt * ayt + rb * ayb) / h +
               (Ar - Arn) / (2.0 * dt) + 0.5 * ((Are * Ae - Arw * Aw) / h + (rt * ayt - rb * ayb) / h) +
               iRe * ((ge * Ave + gw * Avw) / h2 + (vt + vb) / h2) + (vt + vb) / (3.0 * P->Re * h2);
    J[q * 5 + q] = d;
  }
  {
    double rc = rn[CI(L, i, j)], vc = vis[CI(L, i, j)];
    double ayc = 0.5 * (vn[VI(L, i, j)] + vn[VI(L, i, j - 1)]);
    J[2 * 5 + 3] = 0.5 * rc * ayc / h - vc * iRe / h2 - vc / (3.0 * P->Re * h2);
    J[3 * 5 + 2] = -0.5 * rc * ayc / h - vc * iRe / h2 - vc / (3.0 * P->Re * h2);
    J[2 * 5 + 1] = -vc / (3.0 * P->Re * h2);
    J[2 * 5 + 0] = +vc / (3.0 * P->Re * h2);
    J[3 * 5 + 1] = +vc / (3.0 * P->Re * h2);
    J[3 * 5 + 0] = -vc / (3.0 * P->Re * h2);
    J[2 * 5 + 4] = 1.0 / (P->M * h);
    J[3 * 5 + 4] = -1.0 / (P->M * h);
  }
  /* mass row */
  {
    double sm = 0.0;
    static const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
    for (int f = 0; f < 4; ++f) {
      if (wall_face(L, i, j, f)) continue;
      sm += 0.5 * (L->mobn[CI(L, i, j)] + L->mobn[CI(L, i + di[f], j + dj[f])]);
    }
    J[4 * 5 + 0] = -1.0 / h;
    J[4 * 5 + 1] = 1.0 / h;
    J[4 * 5 + 2] = -1.0 / h;
    J[4 * 5 + 3] = 1.0 / h;
    J[4 * 5 + 4] = P->alpha * P->alpha / P->Pe * sm / h2;
  }
  /* local residuals N - f */
  R[0] = act[0] ? N_u(P, L, dt, eW, j) - L->fu[UI(L, eW, j)] : 0.0;
  R[1] = act[1] ? N_u(P, L, dt, eE, j) - L->fu[UI(L, eE, j)] : 0.0;
  R[2] = act[2] ? N_v(P, L, dt, i, j - 1) - L->fv[VI(L, i, j - 1)] : 0.0;
  R[3] = act[3] ? N_v(P, L, dt, i, j) - L->fv[VI(L, i, j)] : 0.0;
  R[4] = Ncell_p(P, L, dt, i, j) - L->fp[CI(L, i, j)];
  for (int q = 0; q < 5; ++q)
    if (!act[q])
      for (int k = 0; k < 5; ++k) {
        J[q * 5 + k] = (q == k) ? 1.0 : 0.0;
        J[k * 5 + q] = (q == k) ? 1.0 : 0.0;
      }
}

/* Gaussian elimination with partial pivoting on a dense n x n system (n <= 7) */
static void solve_dense(int n, double* A, double* b) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int r = k + 1; r < n; ++r)
      if (fabs(A[r * n + k]) > fabs(A[piv * n + k])) piv = r;
    if (piv != k) {
      for (int c = 0; c < n; ++c) {
        double t = A[k * n + c];
        A[k * n + c] = A[piv * n + c];
        A[piv * n + c] = t;
      }
      double t = b[k];
      b[k] = b[piv];
      b[piv] = t;
    }
    for (int r = k + 1; r < n; ++r) {
      double l = A[r * n + k] / A[k * n + k];
      for (int c = k; c < n; ++c) A[r * n + c] -= l * A[k * n + c];
      b[r] -= l * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double t = b[k];
    for (int c = k + 1; c < n; ++c) t -= A[k * n + c] * b[c];
    b[k] = t / A[k * n + k];
  }
}

/* Vanka colours (reading R7): walls in x: (i+2j) mod 5; periodic x with
   m1 = 0 mod 4: (2i+j) mod 8; other (even) periodic m1: (i+2j) mod K with K the
   smallest divisor of m1 that is >= 5.  The offsets of coupled blocks give
   i+2j differences in {+-1..+-4} and 2i+j differences in {+-1, +-2, +-3, +-4}
   with 2(i+m1)+j = 2i+j mod 8 when 4 | m1, so no two coupled cells share a
   colour, also across the periodic seam. */
static int colours_of(int m1, int px) {
  if (!px) return 5;
  if (m1 % 4 == 0) return 8;
  for (int K = 5; K <= m1; ++K)
    if (m1 % K == 0) return K;
  return m1;
}
static int vanka_colour(const ref_level* L, int kcol, int i, int j) {
  if (L->px && L->m1 % 4 == 0) return (2 * i + j) % 8;
  return (i + 2 * j) % kcol;
}

/* CH step 1 of Sec. 7.1 at cell (i,j): one Newton step on the 2x2 local system */
static void ch_point(const ref_params* P, ref_level* L, double dt, int i, int j) {
  size_t k = CI(L, i, j);
  double Rc = Ncell_c(P, L, dt, i, j) - L->fc[k];
  double Rm = N_mu(P, L, i, j) - L->fmu[k];
  double J[4];
  ch_jac(P, L, dt, i, j, J);
  double det = J[0] * J[3] - J[1] * J[2];
  L->c[k] -= (J[3] * Rc - J[1] * Rm) / det;
  L->mu[k] -= (J[0] * Rm - J[2] * Rc) / det;
  sync_cell(L, L->c, i, j);
  sync_cell(L, L->mu, i, j);
}

/* Vanka step 2 of Sec. 7.1 at cell (i,j): exact solve of the 5x5 block */
static void vanka_point(const ref_params* P, ref_level* L, double dt, int i, int j, double omega) {
  double J[25], R[5];
  int act[5];
  vanka_block(P, L, dt, i, j, J, R, act);
  solve_dense(5, J, R);
  int eW = uwrap(L, i - 1);
  if (act[0]) set_u(L, L->u, eW, j, L->u[UI(L, eW, j)] - omega * R[0]);
  if (act[1]) set_u(L, L->u, i, j, L->u[UI(L, i, j)] - omega * R[1]);
  if (act[2]) set_v(L, L->v, i, j - 1, L->v[VI(L, i, j - 1)] - omega * R[2]);
  if (act[3]) set_v(L, L->v, i, j, L->v[VI(L, i, j)] - omega * R[3]);
  L->p[CI(L, i, j)] -= omega * R[4];
  sync_cell(L, L->p, i, j);
}

/* Optional coupled block (not the paper's smoother, which decouples CH and NS):
   one Newton step on the 7x7 system of (N_c, N_mu, N_u west/east, N_v
   south/north, N_p) in (c, mu, u_W, u_E, v_S, v_N, p) of cell (i,j).  To the two
   blocks above it adds the couplings that the decoupled smoother treats
   explicitly: the CH advection and (alpha/Pe) grad.(A m grad p) in N_c,
   (alpha/Pe) grad.(A m grad mu) in N_p, and the rho(c) and surface-tension
   terms of N_u, N_v. */
static void coupled_point(const ref_params* P, ref_level* L, double dt, int i, int j, double omega) {
  double J5[25], R5[5], J2[4], J[49], R[7];
  int act[5];
  vanka_block(P, L, dt, i, j, J5, R5, act);
  ch_jac(P, L, dt, i, j, J2);
  memset(J, 0, sizeof(J));
  size_t k = CI(L, i, j);
  R[0] = N_c(P, L, dt, i, j) - L->fc[k];
  R[1] = N_mu(P, L, i, j) - L->fmu[k];
  for (int a = 0; a < 5; ++a) {
    R[2 + a] = R5[a];
    for (int b = 0; b < 5; ++b) J[(2 + a) * 7 + 2 + b] = J5[a * 5 + b];
  }
  J[0] = J2[0];
  J[1] = J2[1];
  J[7] = J2[2];
  J[8] = J2[3];
  double h = L->h, h2 = h * h;
  const double *rn = L->rhon, *cn = L->cn;
  static const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
  double sm = 0.0;
  for (int f = 0; f < 4; ++f)
    if (!wall_face(L, i, j, f)) sm += 0.5 * (L->mobn[k] + L->mobn[CI(L, i + di[f], j + dj[f])]);
  double rho = rho_of(P, L->c[k]), drho = -P->alpha * rho * rho;
  int eW = uwrap(L, i - 1);
  /* rho^n D c^n / 2 at the four faces of the cell, as in (e1e2) and (e1e1) */
  double gW = 0.5 * rn[CI(L, i - 1, j)] * (cn[k] - cn[CI(L, i - 1, j)]) / h;
  double gE = 0.5 * rn[CI(L, i + 1, j)] * (cn[CI(L, i + 1, j)] - cn[k]) / h;
  double gS = 0.5 * rn[CI(L, i, j - 1)] * (cn[k] - cn[CI(L, i, j - 1)]) / h;
  double gN = 0.5 * rn[CI(L, i, j + 1)] * (cn[CI(L, i, j + 1)] - cn[k]) / h;
  J[0 * 7 + 2] = gW;
  J[0 * 7 + 3] = gE;
  J[0 * 7 + 4] = gS;
  J[0 * 7 + 5] = gN;
  J[0 * 7 + 6] = P->alpha / P->Pe * sm / h2;
  J[2 * 7 + 0] = 0.5 * drho * L->u[UI(L, eW, j)] / (2.0 * dt);
  J[3 * 7 + 0] = 0.5 * drho * L->u[UI(L, i, j)] / (2.0 * dt);
  J[4 * 7 + 0] = 0.5 * drho * L->v[VI(L, i, j - 1)] / (2.0 * dt);
  J[5 * 7 + 0] = 0.5 * drho * L->v[VI(L, i, j)] / (2.0 * dt);
  J[2 * 7 + 1] = -gW / P->M;
  J[3 * 7 + 1] = -gE / P->M;
  J[4 * 7 + 1] = -gS / P->M;
  J[5 * 7 + 1] = -gN / P->M;
  J[6 * 7 + 1] = P->alpha / P->Pe * sm / h2;
  for (int q = 0; q < 5; ++q)
    if (!act[q])
      for (int b = 0; b < 7; ++b) {
        J[(2 + q) * 7 + b] = (b == 2 + q) ? 1.0 : 0.0;
        J[b * 7 + 2 + q] = (b == 2 + q) ? 1.0 : 0.0;
      }
  solve_dense(7, J, R);
  L->c[k] -= omega * R[0];
  L->mu[k] -= omega * R[1];
  sync_cell(L, L->c, i, j);
  sync_cell(L, L->mu, i, j);
  if (act[0]) set_u(L, L->u, eW, j, L->u[UI(L, eW, j)] - omega * R[2]);
  if (act[1]) set_u(L, L->u, i, j, L->u[UI(L, i, j)] - omega * R[3]);
  if (act[2]) set_v(L, L->v, i, j - 1, L->v[VI(L, i, j - 1)] - omega * R[4]);
  if (act[3]) set_v(L, L->v, i, j, L->v[VI(L, i, j)] - omega * R[5]);
  L->p[k] -= omega * R[6];
  sync_cell(L, L->p, i, j);
}

/* projection method, Sec. 7.2 step 2: exact solve of the 4x4 block of the
   intermediate velocities (ut_W, ut_E, vt_S, vt_N) of cell (i,j) in the rows of
   (pj-num-mx); the pressure is not part of the block */
static void vanka4_point(const ref_params* P, ref_level* L, double dt, int i, int j, double omega) {
  double J5[25], R5[5], J[16], R[4];
  int act[5];
  vanka_block(P, L, dt, i, j, J5, R5, act);
  for (int a = 0; a < 4; ++a) {
    R[a] = R5[a];
    for (int b = 0; b < 4; ++b) J[a * 4 + b] = J5[a * 5 + b];
  }
  solve_dense(4, J, R);
  int eW = uwrap(L, i - 1);
  if (act[0]) set_u(L, L->u, eW, j, L->u[UI(L, eW, j)] - omega * R[0]);
  if (act[1]) set_u(L, L->u, i, j, L->u[UI(L, i, j)] - omega * R[1]);
  if (act[2]) set_v(L, L->v, i, j - 1, L->v[VI(L, i, j - 1)] - omega * R[2]);
  if (act[3]) set_v(L, L->v, i, j, L->v[VI(L, i, j)] - omega * R[3]);
}

/* projection method, Sec. 7.2 step 3: Gauss-Seidel on (pj-num-mass) for p_ij.
   The row is affine in p_ij: u^{n+1} on an open face carries -dt/(M h A rho) p
   of each adjacent cell, and the diffusion term (alpha^2/Pe) A m / h^2 */
static void pgs_point(const ref_params* P, ref_level* L, double dt, int i, int j) {
  static const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
  double h2 = L->h * L->h;
  size_t k = CI(L, i, j);
  double R = Np_p(P, L, dt, i, j) - L->fp[k];
  double rk = rho_of(P, L->c[k]), d = 0.0;
  for (int f = 0; f < 4; ++f) {
    if (wall_face(L, i, j, f)) continue;
    size_t q = CI(L, i + di[f], j + dj[f]);
    double Ar = 0.5 * (rk + rho_of(P, L->c[q]));
    d += dt / (P->M * h2 * Ar) + P->alpha * P->alpha / P->Pe * 0.5 * (L->mobn[k] + L->mobn[q]) / h2;
  }
  L->p[k] -= R / d;
  sync_cell(L, L->p, i, j);
}

static void smooth_ch(const ref_params* P, ref_level* L, double dt, int colour) {
  for (int j = 1; j <= L->m2; ++j)
    for (int i = 1; i <= L->m1; ++i)
      if (((i + j) & 1) == colour) ch_point(P, L, dt, i, j);
}

static void smooth_vanka(const ref_params* P, ref_level* L, double dt, int kcol, int colour,
                         double omega) {
  for (int j = 1; j <= L->m2; ++j)
    for (int i = 1; i <= L->m1; ++i)
      if (vanka_colour(L, kcol, i, j) == colour) vanka_point(P, L, dt, i, j, omega);
}

static void smooth_coupled(const ref_params* P, ref_level* L, double dt, int kcol, int colour,
                           double omega) {
  for (int j = 1; j <= L->m2; ++j)
    for (int i = 1; i <= L->m1; ++i)
      if (vanka_colour(L, kcol, i, j) == colour) coupled_point(P, L, dt, i, j, omega);
}

/* one smoothing step.  Decoupled (Sec. 7.1): CH red, CH black, then the Vanka
   colours 0..K-1.  Coupled option: the 7x7 block over the K Vanka colours. */
static void smooth(const ref_solver* s, ref_level* L) {
  if (s->P.scheme) {
    /* projection method (Sec. 7.2): CH red-black, the intermediate-velocity
       blocks over the Vanka colours, pressure Gauss-Seidel red-black */
    smooth_ch(&s->P, L, s->dt, 0);
    smooth_ch(&s->P, L, s->dt, 1);
    for (int col = 0; col < L->kcol; ++col)
      for (int j = 1; j <= L->m2; ++j)
        for (int i = 1; i <= L->m1; ++i)
          if (vanka_colour(L, L->kcol, i, j) == col) vanka4_point(&s->P, L, s->dt, i, j, s->omega);
    for (int col = 0; col < 2; ++col)
      for (int j = 1; j <= L->m2; ++j)
        for (int i = 1; i <= L->m1; ++i)
          if (((i + j) & 1) == col) pgs_point(&s->P, L, s->dt, i, j);
    return;
  }
  if (s->coupled) {
    for (int col = 0; col < L->kcol; ++col) smooth_coupled(&s->P, L, s->dt, L->kcol, col, s->omega);
    return;
  }
  smooth_ch(&s->P, L, s->dt, 0);
  smooth_ch(&s->P, L, s->dt, 1);
  for (int col = 0; col < L->kcol; ++col) smooth_vanka(&s->P, L, s->dt, L->kcol, col, s->omega);
}

/* ------------------------------------------------------------------------ */
/* grid transfers (reading R8)                                              */
/* ------------------------------------------------------------------------ */

static void restrict_cell(const ref_level* F, const ref_level* C, const double* a, double* b) {
  for (int J = 1; J <= C->m2; ++J)
    for (int I = 1; I <= C->m1; ++I)
      b[CI(C, I, J)] = 0.25 * (a[CI(F, 2 * I - 1, 2 * J - 1)] + a[CI(F, 2 * I, 2 * J - 1)] +
                               a[CI(F, 2 * I - 1, 2 * J)] + a[CI(F, 2 * I, 2 * J)]);
}
static void restrict_u(const ref_level* F, const ref_level* C, const double* a, double* b) {
  for (int J = 1; J <= C->m2; ++J)
    for (int I = 0; I <= C->m1; ++I)
      b[UI(C, I, J)] = 0.5 * (a[UI(F, 2 * I, 2 * J - 1)] + a[UI(F, 2 * I, 2 * J)]);
}
static void restrict_v(const ref_level* F, const ref_level* C, const double* a, double* b) {
  for (int J = 0; J <= C->m2; ++J)
    for (int I = 1; I <= C->m1; ++I)
      b[VI(C, I, J)] = 0.5 * (a[VI(F, 2 * I - 1, 2 * J)] + a[VI(F, 2 * I, 2 * J)]);
}

/* Full-weighting restriction of edge residuals: the transpose of the edge
   prolongation below, scaled to preserve constants.  A coarse x-edge gathers the
   coincident fine edge (weight 1/2) and the two fine edges midway to its x
   neighbours (weight 1/4 each), in both fine rows of the coarse row (1/2 each). */
static double rwrap_u(const ref_level* F, const double* a, int i, int j) {
  if (F->px) {
    if (i > F->m1) i -= F->m1;
    if (i < 1) i += F->m1;
  } else if (i <= 0 || i >= F->m1) {
    return 0.0; /* wall edges carry no residual */
  }
  return a[UI(F, i, j)];
}
static void restrict_u_fw(const ref_level* F, const ref_level* C, const double* a, double* b) {
  for (int J = 1; J <= C->m2; ++J)
    for (int I = 0; I <= C->m1; ++I) {
      double s = 0.0;
      for (int jj = 2 * J - 1; jj <= 2 * J; ++jj)
        s += 0.5 * (0.25 * rwrap_u(F, a, 2 * I - 1, jj) + 0.5 * rwrap_u(F, a, 2 * I, jj) +
                    0.25 * rwrap_u(F, a, 2 * I + 1, jj));
      b[UI(C, I, J)] = s;
    }
}
static double rwrap_v(const ref_level* F, const double* a, int i, int j) {
  if (j <= 0 || j >= F->m2) return 0.0;
  return a[VI(F, i, j)];
}
static void restrict_v_fw(const ref_level* F, const ref_level* C, const double* a, double* b) {
  for (int J = 0; J <= C->m2; ++J)
    for (int I = 1; I <= C->m1; ++I) {
      double s = 0.0;
      for (int ii = 2 * I - 1; ii <= 2 * I; ++ii)
        s += 0.5 * (0.25 * rwrap_v(F, a, ii, 2 * J - 1) + 0.5 * rwrap_v(F, a, ii, 2 * J) +
                    0.25 * rwrap_v(F, a, ii, 2 * J + 1));
      b[VI(C, I, J)] = s;
    }
}

/* x_h += P(x_H - saved_H) */
static void prolong_correct(ref_level* F, const ref_level* C) {
  for (int j = 1; j <= F->m2; ++j)
    for (int i = 1; i <= F->m1; ++i) {
      size_t kc = CI(C, (i + 1) / 2, (j + 1) / 2), kf = CI(F, i, j);
      F->c[kf] += C->c[kc] - C->sc[kc];
      F->mu[kf] += C->mu[kc] - C->smu[kc];
      F->p[kf] += C->p[kc] - C->sp[kc];
    }
  for (int j = 1; j <= F->m2; ++j)
    for (int i = ulo(F); i <= uhi(F); ++i) {
      int J = (j + 1) / 2;
      double e;
      if ((i & 1) == 0) {
        size_t k = UI(C, i / 2, J);
        e = C->u[k] - C->su[k];
      } else {
        size_t k0 = UI(C, (i - 1) / 2, J), k1 = UI(C, (i + 1) / 2, J);
        e = 0.5 * ((C->u[k0] - C->su[k0]) + (C->u[k1] - C->su[k1]));
      }
      F->u[UI(F, i, j)] += e;
    }
  for (int j = 1; j <= F->m2 - 1; ++j)
    for (int i = 1; i <= F->m1; ++i) {
      int I = (i + 1) / 2;
      double e;
      if ((j & 1) == 0) {
        size_t k = VI(C, I, j / 2);
        e = C->v[k] - C->sv[k];
      } else {
        size_t k0 = VI(C, I, (j - 1) / 2), k1 = VI(C, I, (j + 1) / 2);
        e = 0.5 * ((C->v[k0] - C->sv[k0]) + (C->v[k1] - C->sv[k1]));
      }
      F->v[VI(F, i, j)] += e;
    }
  bc_all(F);
}

/* ------------------------------------------------------------------------ */
/* FAS V-cycle (Sec. 7.1; standard FAS)                                     */
/* ------------------------------------------------------------------------ */

/* Sweeps on the coarsest grid.  A fixed handful of sweeps only solves the
   coarsest problem when it is a few cells across; the pressure and chemical
   potential modes there converge at a rate set by the grid's longest side n,
   so a coarsest grid that could not coarsen further (periodic width 4 under a
   tall domain, or an odd periodic width) gets nu_coarse * ceil(n/4)^2 sweeps
   (Sec. 7.1 leaves the coarsest solve open). */
static int coarse_sweeps(const ref_solver* s) {
  const ref_level* C = &s->lev[s->nlev - 1];
  int n = C->m1 > C->m2 ? C->m1 : C->m2;
  int q = (n + 3) / 4;
  if (q < 1) q = 1;
  return s->nuc * q * q;
}

static void vcycle(ref_solver* s, int l) {
  ref_level* L = &s->lev[l];
  if (l == s->nlev - 1) {
    int nc = coarse_sweeps(s);
    for (int k = 0; k < nc; ++k) smooth(s, L);
    return;
  }
  int pre = (l == 0 && s->nu1f >= 0) ? s->nu1f : s->nu1;
  int post = (l == 0 && s->nu2f >= 0) ? s->nu2f : s->nu2;
  for (int k = 0; k < pre; ++k) smooth(s, L);
  residual(&s->P, L, s->dt, NULL);
  ref_level* C = &s->lev[l + 1];
  restrict_cell(L, C, L->c, C->c);
  restrict_cell(L, C, L->mu, C->mu);
  restrict_cell(L, C, L->p, C->p);
  restrict_u(L, C, L->u, C->u);
  restrict_v(L, C, L->v, C->v);
  bc_all(C);
  memcpy(C->sc, C->c, ncell(C) * sizeof(double));
  memcpy(C->smu, C->mu, ncell(C) * sizeof(double));
  memcpy(C->sp, C->p, ncell(C) * sizeof(double));
  memcpy(C->su, C->u, nu_(C) * sizeof(double));
  memcpy(C->sv, C->v, nv_(C) * sizeof(double));
  /* f_H = R r_h + N_H(R x_h) */
  restrict_cell(L, C, L->rc, C->fc);
  restrict_cell(L, C, L->rmu, C->fmu);
  restrict_cell(L, C, L->rp, C->fp);
  restrict_u_fw(L, C, L->ru, C->fu);
  restrict_v_fw(L, C, L->rv, C->fv);
  for (int J = 1; J <= C->m2; ++J)
    for (int I = 1; I <= C->m1; ++I) {
      size_t k = CI(C, I, J);
      C->fc[k] += Ncell_c(&s->P, C, s->dt, I, J);
      C->fmu[k] += N_mu(&s->P, C, I, J);
      C->fp[k] += Ncell_p(&s->P, C, s->dt, I, J);
    }
  for (int J = 1; J <= C->m2; ++J)
    for (int I = ulo(C); I <= uhi(C); ++I) C->fu[UI(C, I, J)] += N_u(&s->P, C, s->dt, I, J);
  for (int J = 1; J <= C->m2 - 1; ++J)
    for (int I = 1; I <= C->m1; ++I) C->fv[VI(C, I, J)] += N_v(&s->P, C, s->dt, I, J);
  vcycle(s, l + 1);
  prolong_correct(L, C);
  for (int k = 0; k < post; ++k) smooth(s, L);
}

/* mean of p removed (reading R9) */
static void gauge(ref_level* L) {
  double sum = 0.0;
  for (int j = 1; j <= L->m2; ++j)
    for (int i = 1; i <= L->m1; ++i) sum += L->p[CI(L, i, j)];
  double mean = sum / ((double)L->m1 * L->m2);
  for (int j = 1; j <= L->m2; ++j)
    for (int i = 1; i <= L->m1; ++i) L->p[CI(L, i, j)] -= mean;
  bc_cell(L, L->p);
}

/* ------------------------------------------------------------------------ */
/* reductions: mass (Thm. 6.1) and discrete energy / dissipation (Thm. 6.2)  */
/* ------------------------------------------------------------------------ */

static void mass_of(const ref_params* P, const ref_level* L, const double* c, double* mr, double* mrc) {
  double a = 0.0, b = 0.0;
  for (int j = 1; j <= L->m2; ++j)
    for (int i = 1; i <= L->m1; ++i) {
      double r = rho_of(P, c[CI(L, i, j)]);
      a += r;
      b += r * c[CI(L, i, j)];
    }
  *mr = L->h * L->h * a;
  *mrc = L->h * L->h * b;
}

/* E_h = 1/2||sqrt(rho) u||^2 + (eps eta/(2We))||sqrt(rho) grad_D c||^2
         + (eta h^2/(eps We))(rho F(c),1) + (h^2/Fr)(rho y,1)   (App. A.7 norms) */
static double energy_of(const ref_params* P, const ref_level* L, const double* c,
                        const double* u, const double* v) {
  double kin = 0.0, grad = 0.0, bulk = 0.0, pot = 0.0, h = L->h;
  for (int j = 1; j <= L->m2; ++j)
    for (int i = 1; i <= L->m1; ++i) {
      double r = rho_of(P, c[CI(L, i, j)]);
      double axu2 = 0.5 * (u[UI(L, i, j)] * u[UI(L, i, j)] + u[UI(L, i - 1, j)] * u[UI(L, i - 1, j)]);
      double ayv2 = 0.5 * (v[VI(L, i, j)] * v[VI(L, i, j)] + v[VI(L, i, j - 1)] * v[VI(L, i, j - 1)]);
      kin += r * (axu2 + ayv2);
      grad += r * G_at(L, c, i, j);
      bulk += r * Fdw(c[CI(L, i, j)]);
      pot += r * (j - 0.5) * h;
    }
  double h2 = h * h;
  return 0.5 * h2 * kin + P->Cn * P->eta / (2.0 * P->We) * h2 * grad +
         P->eta / (P->Cn * P->We) * h2 * bulk + P->Fr_inv * h2 * pot;
}

/* Dissipation of Thm. 6.2 for iterate x against frozen data, written as sums of
   squares: 1/2||sqrt(rho^n)(u - u^n)||^2 + (dt/Re)||sqrt(mu^n) grad_d u||^2
   + (dt/(3Re))||sqrt(mu^n) div_d u||^2 + (dt/(M Pe))||sqrt(m^n) grad_D(mu + alpha p)||^2.
   Vertex terms carry weight 1/2 on walls (vertex inner product, App. A.3),
   evaluated with the reflected ghosts. */
static double dissipation_of(const ref_params* P, const ref_level* L, double dt) {
  double h = L->h, h2 = h * h;
  double kin = 0.0, vc = 0.0, vv = 0.0, div = 0.0, ch = 0.0;
  for (int j = 1; j <= L->m2; ++j)
    for (int i = 1; i <= L->m1; ++i) {
      double rn = L->rhon[CI(L, i, j)], mv = L->visn[CI(L, i, j)];
      double du0 = L->u[UI(L, i, j)] - L->un[UI(L, i, j)];
      double du1 = L->u[UI(L, i - 1, j)] - L->un[UI(L, i - 1, j)];
      double dv0 = L->v[VI(L, i, j)] - L->vn[VI(L, i, j)];
      double dv1 = L->v[VI(L, i, j - 1)] - L->vn[VI(L, i, j - 1)];
      kin += rn * (0.5 * (du0 * du0 + du1 * du1) + 0.5 * (dv0 * dv0 + dv1 * dv1));
      double dxu = (L->u[UI(L, i, j)] - L->u[UI(L, i - 1, j)]) / h;
      double dyv = (L->v[VI(L, i, j)] - L->v[VI(L, i, j - 1)]) / h;
      vc += mv * (dxu * dxu + dyv * dyv);
      div += mv * (dxu + dyv) * (dxu + dyv);
    }
  /* vertices (i+1/2, j+1/2): periodic x counts columns 1..m1 once */
  int ilo = L->px ? 1 : 0;
  for (int j = 0; j <= L->m2; ++j)
    for (int i = ilo; i <= L->m1; ++i) {
      double Av = Avtx(L, L->visn, i, j);
      double Dyu = (L->u[UI(L, i, j + 1)] - L->u[UI(L, i, j)]) / h;
      double Dxv = (L->v[VI(L, i + 1, j)] - L->v[VI(L, i, j)]) / h;
      /* Dcal_y u lives on vertex rows; rows on the y walls get weight 1/2.
         Dcal_x v lives on vertex columns; columns on x walls get weight 1/2.
         (On an x wall u = 0, so Dcal_y u = 0 there; likewise Dcal_x v on y walls.) */
      double wy = (j == 0 || j == L->m2) ? 0.5 : 1.0;
      double wx = (!L->px && (i == 0 || i == L->m1)) ? 0.5 : 1.0;
      vv += Av * (wy * Dyu * Dyu + wx * Dxv * Dxv);
    }
  /* faces of mu_c = mu + alpha p */
  for (int j = 1; j <= L->m2; ++j)
    for (int i = 1; i <= L->m1; ++i) {
      double mc = L->mu[CI(L, i, j)] + P->alpha * L->p[CI(L, i, j)];
      if (L->px || i < L->m1) {
        double me = L->mu[CI(L, i + 1, j)] + P->alpha * L->p[CI(L, i + 1, j)];
        double Am = 0.5 * (L->mobn[CI(L, i, j)] + L->mobn[CI(L, i + 1, j)]);
        ch += Am * (me - mc) * (me - mc) / h2;
      }
      if (j < L->m2) {
        double mn = L->mu[CI(L, i, j + 1)] + P->alpha * L->p[CI(L, i, j + 1)];
        double Am = 0.5 * (L->mobn[CI(L, i, j)] + L->mobn[CI(L, i, j + 1)]);
        ch += Am * (mn - mc) * (mn - mc) / h2;
      }
    }
  return h2 * (0.5 * kin + dt / P->Re * (vc + vv) + dt / (3.0 * P->Re) * div +
               dt / (P->M * P->Pe) * ch);
}

/* u^{n+1}, v^{n+1} of the projection method on level L (interior edges from
   (pj-num-pjx), then the ghost rules of App. A.6) */
static void projected_velocity(const ref_params* P, const ref_level* L, double dt, double* u,
                               double* v) {
  for (int j = 1; j <= L->m2; ++j)
    for (int e = 0; e <= L->m1; ++e) u[UI(L, e, j)] = proj_u(P, L, dt, e, j);
  for (int e = 0; e <= L->m2; ++e)
    for (int i = 1; i <= L->m1; ++i) v[VI(L, i, e)] = proj_v(P, L, dt, i, e);
  bc_u(L, u);
  bc_v(L, v);
}

/* the extra dissipation of the projection method (Thm. 6.4):
   1/2 ||sqrt(rho(c)) (u^{n+1} - ut)||^2 over both velocity components, in the
   cell-averaged form of the kinetic energy */
static double projection_dissipation(const ref_params* P, const ref_level* L, const double* u,
                                     const double* v) {
  double s = 0.0;
  for (int j = 1; j <= L->m2; ++j)
    for (int i = 1; i <= L->m1; ++i) {
      double r = rho_of(P, L->c[CI(L, i, j)]);
      double a = u[UI(L, i, j)] - L->u[UI(L, i, j)], b = u[UI(L, i - 1, j)] - L->u[UI(L, i - 1, j)];
      double c = v[VI(L, i, j)] - L->v[VI(L, i, j)], d = v[VI(L, i, j - 1)] - L->v[VI(L, i, j - 1)];
      s += r * (0.5 * (a * a + b * b) + 0.5 * (c * c + d * d));
    }
  return 0.5 * L->h * L->h * s;
}

/* ------------------------------------------------------------------------ */
/* host-array packing                                                       */
/* ------------------------------------------------------------------------ */

static void pack_in(const ref_level* L, double* c, double* mu, double* p, double* u, double* v,
                    const double* hc, const double* hmu, const double* hp, const double* hu,
                    const double* hv) {
  int m1 = L->m1, m2 = L->m2;
  for (int j = 1; j <= m2; ++j)
    for (int i = 1; i <= m1; ++i) {
      size_t k = (size_t)(j - 1) * m1 + (i - 1);
      if (c) c[CI(L, i, j)] = hc[k];
      if (mu) mu[CI(L, i, j)] = hmu[k];
      if (p) p[CI(L, i, j)] = hp[k];
    }
  if (u)
    for (int j = 1; j <= m2; ++j)
      for (int i = 0; i <= m1; ++i) u[UI(L, i, j)] = hu[(size_t)(j - 1) * (m1 + 1) + i];
  if (v)
    for (int j = 0; j <= m2; ++j)
      for (int i = 1; i <= m1; ++i) v[VI(L, i, j)] = hv[(size_t)j * m1 + (i - 1)];
  if (c) bc_cell(L, c);
  if (mu) bc_cell(L, mu);
  if (p) bc_cell(L, p);
  if (u) bc_u(L, u);
  if (v) bc_v(L, v);
}

static void pack_out(const ref_level* L, const double* c, const double* mu, const double* p,
                     const double* u, const double* v, double* hc, double* hmu, double* hp,
                     double* hu, double* hv) {
  int m1 = L->m1, m2 = L->m2;
  for (int j = 1; j <= m2; ++j)
    for (int i = 1; i <= m1; ++i) {
      size_t k = (size_t)(j - 1) * m1 + (i - 1);
      if (hc) hc[k] = c[CI(L, i, j)];
      if (hmu) hmu[k] = mu[CI(L, i, j)];
      if (hp) hp[k] = p[CI(L, i, j)];
    }
  if (hu)
    for (int j = 1; j <= m2; ++j)
      for (int i = 0; i <= m1; ++i) hu[(size_t)(j - 1) * (m1 + 1) + i] = u[UI(L, i, j)];
  if (hv)
    for (int j = 0; j <= m2; ++j)
      for (int i = 1; i <= m1; ++i) hv[(size_t)j * m1 + (i - 1)] = v[VI(L, i, j)];
}

/* ------------------------------------------------------------------------ */
/* API                                                                      */
/* ------------------------------------------------------------------------ */

static double* zalloc(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

static int level_alloc(ref_level* L, int m1, int m2, int px, double h) {
  L->m1 = m1;
  L->m2 = m2;
  L->px = px;
  L->kcol = colours_of(m1, px);
  L->h = h;
  size_t nc = ncell(L), nu = nu_(L), nv = nv_(L);
  double** cells[] = {&L->c, &L->mu, &L->p, &L->fc, &L->fmu, &L->fp, &L->rc, &L->rmu, &L->rp,
                      &L->sc, &L->smu, &L->sp, &L->cn, &L->rhon, &L->mobn, &L->visn, &L->Gn};
  double** us[] = {&L->u, &L->fu, &L->ru, &L->su, &L->un};
  double** vs[] = {&L->v, &L->fv, &L->rv, &L->sv, &L->vn};
  for (size_t k = 0; k < sizeof(cells) / sizeof(cells[0]); ++k)
    if (!(*cells[k] = zalloc(nc))) return REF_ENOMEM;
  for (size_t k = 0; k < 5; ++k)
    if (!(*us[k] = zalloc(nu))) return REF_ENOMEM;
  for (size_t k = 0; k < 5; ++k)
    if (!(*vs[k] = zalloc(nv))) return REF_ENOMEM;
  return REF_OK;
}

static void level_free(ref_level* L) {
  double* a[] = {L->c, L->mu, L->p, L->fc, L->fmu, L->fp, L->rc, L->rmu, L->rp, L->sc, L->smu,
                 L->sp, L->cn, L->rhon, L->mobn, L->visn, L->Gn, L->u, L->fu, L->ru, L->su,
                 L->un, L->v, L->fv, L->rv, L->sv, L->vn};
  for (size_t k = 0; k < sizeof(a) / sizeof(a[0]); ++k) free(a[k]);
}

/* coarsen by 2 while both sizes stay even and >= 2 (walls in x) or the x size
   stays a multiple of 4 and >= 4 (periodic x, for the colouring of R7) */
static int max_levels(int m1, int m2, int px) {
  int n = 1;
  /* walls: down to 2 cells; periodic x: the coarse m1 stays even (red-black
     across the seam) and >= 4 */
  while (m1 % 2 == 0 && m2 % 2 == 0 && m2 / 2 >= 2 &&
         (px ? (m1 / 2 >= 4 && (m1 / 2) % 2 == 0) : m1 / 2 >= 2)) {
    m1 /= 2;
    m2 /= 2;
    ++n;
  }
  return n;
}

int qnsch_ref_create(int m1, int m2, double Lx, int periodic_x, int levels, double rho1,
                     double rho2, double eta1, double eta2, double Re, double We, double Pe,
                     double Cn, double Fr, ref_solver** out) {
  if (!out || m1 < 2 || m2 < 2 || !(Lx > 0) || !(rho1 > 0) || !(rho2 > 0) || !(eta1 > 0) ||
      !(eta2 > 0) || !(Re > 0) || !(We > 0) || !(Pe > 0) || !(Cn > 0))
    return REF_EINVAL;
  if (periodic_x && (m1 % 2 != 0 || m1 < 4)) return REF_EINVAL;
  int lmax = max_levels(m1, m2, periodic_x);
  if (levels <= 0) levels = lmax;
  if (levels > lmax) return REF_EINVAL;
  ref_solver* s = (ref_solver*)calloc(1, sizeof(ref_solver));
  if (!s) return REF_ENOMEM;
  s->P.rho1 = rho1;
  s->P.rho2 = rho2;
  s->P.mu1 = eta1;
  s->P.mu2 = eta2;
  s->P.Re = Re;
  s->P.We = We;
  s->P.Pe = Pe;
  s->P.Cn = Cn;
  s->P.Fr_inv = (isinf(Fr) || Fr <= 0) ? 0.0 : 1.0 / Fr;
  s->P.M = Cn;
  s->P.eps_m = Cn;
  s->P.eta = eta_of(rho1, rho2);
  derive_params(&s->P);
  s->nu1 = 2;
  s->nu2 = 2;
  s->nuc = 4;
  s->nu1f = -1;
  s->nu2f = -1;
  s->maxcyc = 50;
  s->tol = 1e-9;
  s->omega = 1.0;
  s->nhist = -1; /* no state set yet */
  s->kcol = colours_of(m1, periodic_x);
  s->nlev = levels;
  s->lev = (ref_level*)calloc((size_t)levels, sizeof(ref_level));
  double h = Lx / m1;
  int a = m1, b = m2;
  for (int l = 0; l < levels; ++l) {
    if (level_alloc(&s->lev[l], a, b, periodic_x, h) != REF_OK) {
      qnsch_ref_destroy(s);
      return REF_ENOMEM;
    }
    a /= 2;
    b /= 2;
    h *= 2.0;
  }
  ref_level* F = &s->lev[0];
  s->c = zalloc(ncell(F));
  s->mu = zalloc(ncell(F));
  s->p = zalloc(ncell(F));
  s->u = zalloc(nu_(F));
  s->v = zalloc(nv_(F));
  for (int k = 0; k < 2; ++k) {
    s->hc[k] = zalloc(ncell(F));
    s->hmu[k] = zalloc(ncell(F));
    s->hp[k] = zalloc(ncell(F));
    s->hu[k] = zalloc(nu_(F));
    s->hv[k] = zalloc(nv_(F));
  }
  *out = s;
  return REF_OK;
}

int qnsch_ref_destroy(ref_solver* s) {
  if (!s) return REF_EINVAL;
  if (s->lev)
    for (int l = 0; l < s->nlev; ++l) level_free(&s->lev[l]);
  free(s->lev);
  free(s->c);
  free(s->mu);
  free(s->p);
  free(s->u);
  free(s->v);
  for (int k = 0; k < 2; ++k) {
    free(s->hc[k]);
    free(s->hmu[k]);
    free(s->hp[k]);
    free(s->hu[k]);
    free(s->hv[k]);
  }
  free(s);
  return REF_OK;
}

int qnsch_ref_set_option(ref_solver* s, const char* key, double value) {
  if (!s || !key) return REF_EINVAL;
  if (!strcmp(key, "nu1")) s->nu1 = (int)value;
  else if (!strcmp(key, "nu2")) s->nu2 = (int)value;
  else if (!strcmp(key, "nu1_fine")) s->nu1f = (int)value;
  else if (!strcmp(key, "nu2_fine")) s->nu2f = (int)value;
  else if (!strcmp(key, "nu_coarse")) s->nuc = (int)value;
  else if (!strcmp(key, "scheme")) {
    if (s->pending || (value != 0.0 && value != 1.0) || (value == 1.0 && s->coupled)) return REF_EINVAL;
    s->P.scheme = (int)value;
  }
  else if (!strcmp(key, "maxcyc")) s->maxcyc = (int)value;
  else if (!strcmp(key, "tol")) s->tol = value;
  else if (!strcmp(key, "omega_vanka")) s->omega = value;
  else if (!strcmp(key, "M")) { s->P.M = value; derive_params(&s->P); }
  else if (!strcmp(key, "eta_st")) { s->P.eta = value; derive_params(&s->P); }
  else if (!strcmp(key, "eps_mob")) s->P.eps_m = value;
  else if (!strcmp(key, "coupled")) {
    if (value != 0.0 && s->P.scheme) return REF_EINVAL; /* the 7x7 block is a primitive-method smoother */
    s->coupled = value != 0.0;
  }
  else if (!strcmp(key, "predictor")) {
    if (s->pending || !(value == 0.0 || value == 1.0 || value == 2.0)) return REF_EINVAL;
    s->predictor = (int)value;
    if (s->nhist > 0) s->nhist = 0;
  }
  else if (!strcmp(key, "history")) {
    if (s->pending || value != 0.0) return REF_EINVAL;
    if (s->nhist > 0) s->nhist = 0;
  }
  else return REF_EINVAL;
  return REF_OK;
}

int qnsch_ref_get_option(const ref_solver* s, const char* key, double* value) {
  if (!s || !key || !value) return REF_EINVAL;
  if (!strcmp(key, "nu1")) *value = s->nu1;
  else if (!strcmp(key, "nu2")) *value = s->nu2;
  else if (!strcmp(key, "nu1_fine")) *value = s->nu1f;
  else if (!strcmp(key, "nu2_fine")) *value = s->nu2f;
  else if (!strcmp(key, "nu_coarse")) *value = s->nuc;
  else if (!strcmp(key, "scheme")) *value = s->P.scheme;
  else if (!strcmp(key, "maxcyc")) *value = s->maxcyc;
  else if (!strcmp(key, "tol")) *value = s->tol;
  else if (!strcmp(key, "omega_vanka")) *value = s->omega;
  else if (!strcmp(key, "M")) *value = s->P.M;
  else if (!strcmp(key, "eta_st")) *value = s->P.eta;
  else if (!strcmp(key, "eps_mob")) *value = s->P.eps_m;
  else if (!strcmp(key, "coupled")) *value = s->coupled;
  else if (!strcmp(key, "predictor")) *value = s->predictor;
  else if (!strcmp(key, "history")) *value = s->nhist > 0 ? s->nhist : 0;
  else return REF_EINVAL;
  return REF_OK;
}

int qnsch_ref_levels(const ref_solver* s) { return s ? s->nlev : REF_EINVAL; }
int qnsch_ref_ncolours_vanka(const ref_solver* s) { return s ? s->kcol : REF_EINVAL; }

int qnsch_ref_params(const ref_solver* s, double* out8) {
  if (!s || !out8) return REF_EINVAL;
  out8[0] = s->P.alpha;
  out8[1] = s->P.eta;
  out8[2] = s->P.K;
  out8[3] = s->P.Lam;
  out8[4] = s->P.M;
  out8[5] = s->P.Fr_inv;
  out8[6] = s->P.eps_m;
  out8[7] = s->lev[0].h;
  return REF_OK;
}

/* host layout <-> ghosted level array, for one family (0 cell, 1 u, 2 v) */
static void host_to_level(const ref_level* L, int fam, const double* h, double* a) {
  int m1 = L->m1, m2 = L->m2;
  if (fam == 0) {
    for (int j = 1; j <= m2; ++j)
      for (int i = 1; i <= m1; ++i) a[CI(L, i, j)] = h[(size_t)(j - 1) * m1 + (i - 1)];
  } else if (fam == 1) {
    for (int j = 1; j <= m2; ++j)
      for (int i = 0; i <= m1; ++i) a[UI(L, i, j)] = h[(size_t)(j - 1) * (m1 + 1) + i];
  } else {
    for (int j = 0; j <= m2; ++j)
      for (int i = 1; i <= m1; ++i) a[VI(L, i, j)] = h[(size_t)j * m1 + (i - 1)];
  }
}
static void level_to_host(const ref_level* L, int fam, const double* a, double* h) {
  int m1 = L->m1, m2 = L->m2;
  if (fam == 0) {
    for (int j = 1; j <= m2; ++j)
      for (int i = 1; i <= m1; ++i) h[(size_t)(j - 1) * m1 + (i - 1)] = a[CI(L, i, j)];
  } else if (fam == 1) {
    for (int j = 1; j <= m2; ++j)
      for (int i = 0; i <= m1; ++i) h[(size_t)(j - 1) * (m1 + 1) + i] = a[UI(L, i, j)];
  } else {
    for (int j = 0; j <= m2; ++j)
      for (int i = 1; i <= m1; ++i) h[(size_t)j * m1 + (i - 1)] = a[VI(L, i, j)];
  }
}
static size_t fam_size(const ref_level* L, int fam) {
  return fam == 0 ? ncell(L) : fam == 1 ? nu_(L) : nv_(L);
}

int qnsch_ref_transfer(const ref_solver* s, int l, int op, const double* in, double* out) {
  if (!s || !in || !out || l < 0 || l + 1 >= s->nlev || op < 0 || op > 7) return REF_EINVAL;
  const ref_level* F = &s->lev[l];
  const ref_level* C = &s->lev[l + 1];
  int fam = op >= 6 ? op - 5 : op % 3;
  if (op < 3 || op >= 6) { /* residual or state restriction, fine -> coarse */
    double* a = (double*)calloc(fam_size(F, fam), sizeof(double));
    double* b = (double*)calloc(fam_size(C, fam), sizeof(double));
    if (!a || !b) {
      free(a);
      free(b);
      return REF_ENOMEM;
    }
    host_to_level(F, fam, in, a);
    if (op == 6) restrict_u(F, C, a, b);
    else if (op == 7) restrict_v(F, C, a, b);
    else if (fam == 0) restrict_cell(F, C, a, b);
    else if (fam == 1) restrict_u_fw(F, C, a, b);
    else restrict_v_fw(F, C, a, b);
    level_to_host(C, fam, b, out);
    free(a);
    free(b);
    return REF_OK;
  }
  /* prolongation of a coarse correction, coarse -> fine, on copies of the two
     levels whose iterate and saved arrays are zero except the input */
  ref_level Ft = *F, Ct = *C;
  size_t nf[3] = {ncell(F), nu_(F), nv_(F)}, nc[3] = {ncell(C), nu_(C), nv_(C)};
  double* buf[4] = {NULL, NULL, NULL, NULL};
  buf[0] = (double*)calloc(3 * nf[0] + nf[1] + nf[2], sizeof(double)); /* fine x */
  buf[1] = (double*)calloc(3 * nc[0] + nc[1] + nc[2], sizeof(double)); /* coarse x */
  buf[2] = (double*)calloc(3 * nc[0] + nc[1] + nc[2], sizeof(double)); /* coarse saved */
  if (!buf[0] || !buf[1] || !buf[2]) {
    free(buf[0]);
    free(buf[1]);
    free(buf[2]);
    return REF_ENOMEM;
  }
  Ft.c = buf[0]; Ft.mu = Ft.c + nf[0]; Ft.p = Ft.mu + nf[0]; Ft.u = Ft.p + nf[0]; Ft.v = Ft.u + nf[1];
  Ct.c = buf[1]; Ct.mu = Ct.c + nc[0]; Ct.p = Ct.mu + nc[0]; Ct.u = Ct.p + nc[0]; Ct.v = Ct.u + nc[1];
  Ct.sc = buf[2]; Ct.smu = Ct.sc + nc[0]; Ct.sp = Ct.smu + nc[0]; Ct.su = Ct.sp + nc[0];
  Ct.sv = Ct.su + nc[1];
  host_to_level(C, fam, in, fam == 0 ? Ct.c : fam == 1 ? Ct.u : Ct.v);
  prolong_correct(&Ft, &Ct);
  level_to_host(F, fam, fam == 0 ? Ft.c : fam == 1 ? Ft.u : Ft.v, out);
  free(buf[0]);
  free(buf[1]);
  free(buf[2]);
  return REF_OK;
}

int qnsch_ref_secants(const ref_solver* s, double a, double b, double* out7) {
  if (!s || !out7) return REF_EINVAL;
  out7[0] = Fdw(a);
  out7[1] = Fdw(b);
  out7[2] = gsec(a, b);
  out7[3] = gsec_da(a, b);
  out7[4] = rho_of(&s->P, a);
  out7[5] = rho_of(&s->P, b);
  out7[6] = rsec(&s->P, a, b);
  return REF_OK;
}

int qnsch_ref_set_fields(ref_solver* s, const double* c, const double* mu, const double* u,
                         const double* v, const double* p) {
  if (!s || !c || !mu || !u || !v || !p) return REF_EINVAL;
  if (s->pending) return REF_ESTATE;
  pack_in(&s->lev[0], s->c, s->mu, s->p, s->u, s->v, c, mu, p, u, v);
  s->nhist = -1;
  return REF_OK;
}

/* the states the predictor extrapolates from (k = 0 the most recent) */
int qnsch_ref_get_history(const ref_solver* s, int k, double* dt, double* c, double* mu,
                          double* u, double* v, double* p) {
  if (!s || !dt || k < 0 || k >= s->nhist) return REF_EINVAL;
  pack_out(&s->lev[0], s->hc[k], s->hmu[k], s->hp[k], s->hu[k], s->hv[k], c, mu, p, u, v);
  *dt = s->hdt[k];
  return REF_OK;
}

int qnsch_ref_set_history(ref_solver* s, int k, double dt, const double* c, const double* mu,
                          const double* u, const double* v, const double* p) {
  if (!s) return REF_EINVAL;
  int held = s->nhist > 0 ? s->nhist : 0;
  if (!c || !mu || !u || !v || !p || k < 0 || k > 1 || k > held || !(dt > 0)) return REF_EINVAL;
  if (s->pending) return REF_ESTATE;
  pack_in(&s->lev[0], s->hc[k], s->hmu[k], s->hp[k], s->hu[k], s->hv[k], c, mu, p, u, v);
  s->hdt[k] = dt;
  if (k >= s->nhist) s->nhist = k + 1;
  return REF_OK;
}

/* Lagrange basis at tau = dt for the nodes tau_0 = 0 (the committed state),
   tau_1 = -hdt[0], tau_2 = -hdt[0] - hdt[1] (the earlier states), of the
   degree the option and the history allow: l_i(dt) = prod over j != i of
   (dt - tau_j) / (tau_i - tau_j); degree 0 gives the committed state. */
static void predict_weights(const ref_solver* s, double dt, double w[3]) {
  int m = s->predictor < s->nhist ? s->predictor : s->nhist;
  if (m < 0) m = 0;
  double tau[3];
  tau[0] = 0.0;
  tau[1] = -s->hdt[0];
  tau[2] = -s->hdt[0] - s->hdt[1];
  for (int i = 0; i < 3; ++i) w[i] = 0.0;
  for (int i = 0; i <= m; ++i) {
    double l = 1.0;
    for (int j = 0; j <= m; ++j)
      if (j != i) l *= (dt - tau[j]) / (tau[i] - tau[j]);
    w[i] = l;
  }
}

static void combine(double* x, size_t n, const double w[3], const double* a, const double* b,
                    const double* c) {
  for (size_t i = 0; i < n; ++i) x[i] = w[0] * a[i] + w[1] * b[i] + w[2] * c[i];
}

int qnsch_ref_get_fields(const ref_solver* s, double* c, double* mu, double* u, double* v,
                         double* p) {
  if (!s) return REF_EINVAL;
  pack_out(&s->lev[0], s->c, s->mu, s->p, s->u, s->v, c, mu, p, u, v);
  return REF_OK;
}

int qnsch_ref_begin_step(ref_solver* s, double dt) {
  if (!s || !(dt > 0)) return REF_EINVAL;
  s->dt = dt;
  ref_level* F = &s->lev[0];
  memcpy(F->c, s->c, ncell(F) * sizeof(double));
  memcpy(F->mu, s->mu, ncell(F) * sizeof(double));
  memcpy(F->p, s->p, ncell(F) * sizeof(double));
  memcpy(F->u, s->u, nu_(F) * sizeof(double));
  memcpy(F->v, s->v, nv_(F) * sizeof(double));
  {
    /* the initial iterate: x^n, or its extrapolation in time (predictor) */
    double w[3];
    predict_weights(s, dt, w);
    if (w[1] != 0.0 || w[2] != 0.0) {
      combine(F->c, ncell(F), w, s->c, s->hc[0], s->hc[1]);
      combine(F->mu, ncell(F), w, s->mu, s->hmu[0], s->hmu[1]);
      combine(F->p, ncell(F), w, s->p, s->hp[0], s->hp[1]);
      combine(F->u, nu_(F), w, s->u, s->hu[0], s->hu[1]);
      combine(F->v, nv_(F), w, s->v, s->hv[0], s->hv[1]);
    }
  }
  memcpy(F->cn, s->c, ncell(F) * sizeof(double));
  memcpy(F->un, s->u, nu_(F) * sizeof(double));
  memcpy(F->vn, s->v, nv_(F) * sizeof(double));
  memset(F->fc, 0, ncell(F) * sizeof(double));
  memset(F->fmu, 0, ncell(F) * sizeof(double));
  memset(F->fp, 0, ncell(F) * sizeof(double));
  memset(F->fu, 0, nu_(F) * sizeof(double));
  memset(F->fv, 0, nv_(F) * sizeof(double));
  bc_all(F);
  frozen_derived(&s->P, F);
  for (int l = 1; l < s->nlev; ++l) {
    ref_level *A = &s->lev[l - 1], *C = &s->lev[l];
    restrict_cell(A, C, A->cn, C->cn);
    restrict_u(A, C, A->un, C->un);
    restrict_v(A, C, A->vn, C->vn);
    frozen_derived(&s->P, C);
  }
  s->pending = 1;
  return REF_OK;
}

int qnsch_ref_vcycle(ref_solver* s, double* norms10) {
  if (!s) return REF_EINVAL;
  if (!s->pending) return REF_ESTATE;
  vcycle(s, 0);
  gauge(&s->lev[0]);
  double nrm[10];
  residual(&s->P, &s->lev[0], s->dt, nrm);
  if (norms10) memcpy(norms10, nrm, sizeof(nrm));
  return REF_OK;
}

int qnsch_ref_commit_step(ref_solver* s) {
  if (!s) return REF_EINVAL;
  if (!s->pending) return REF_ESTATE;
  ref_level* F = &s->lev[0];
  if (s->predictor > 0) {
    /* the state being replaced becomes the most recent earlier state */
    double* t;
#define ROTATE(h) (t = h[1], h[1] = h[0], h[0] = t)
    ROTATE(s->hc);
    ROTATE(s->hmu);
    ROTATE(s->hp);
    ROTATE(s->hu);
    ROTATE(s->hv);
#undef ROTATE
    memcpy(s->hc[0], s->c, ncell(F) * sizeof(double));
    memcpy(s->hmu[0], s->mu, ncell(F) * sizeof(double));
    memcpy(s->hp[0], s->p, ncell(F) * sizeof(double));
    memcpy(s->hu[0], s->u, nu_(F) * sizeof(double));
    memcpy(s->hv[0], s->v, nv_(F) * sizeof(double));
    s->hdt[1] = s->hdt[0];
    s->hdt[0] = s->dt;
    s->nhist = s->nhist < 2 ? s->nhist + 1 : 2;
  }
  memcpy(s->c, F->c, ncell(F) * sizeof(double));
  memcpy(s->mu, F->mu, ncell(F) * sizeof(double));
  memcpy(s->p, F->p, ncell(F) * sizeof(double));
  if (s->P.scheme) {
    /* projection method: the committed velocity is u^{n+1} of (pj-num-pjx) */
    projected_velocity(&s->P, F, s->dt, s->u, s->v);
  } else {
    memcpy(s->u, F->u, nu_(F) * sizeof(double));
    memcpy(s->v, F->v, nv_(F) * sizeof(double));
  }
  s->pending = 0;
  return REF_OK;
}

static double maxfam(const double* n10) {
  double m = 0.0;
  for (int q = 0; q < 5; ++q)
    if (n10[q] > m) m = n10[q];
  return m;
}

int qnsch_ref_step(ref_solver* s, double dt, int* n_vcycles, double* final_res) {
  int rc = qnsch_ref_begin_step(s, dt);
  if (rc) return rc;
  double nrm[10];
  residual(&s->P, &s->lev[0], s->dt, nrm);
  int k = 0;
  while (maxfam(nrm) > s->tol && k < s->maxcyc) {
    qnsch_ref_vcycle(s, nrm);
    ++k;
  }
  s->last_res = maxfam(nrm);
  if (n_vcycles) *n_vcycles = k;
  if (final_res) *final_res = s->last_res;
  if (s->last_res > s->tol) return REF_ENOTCONV;
  return qnsch_ref_commit_step(s);
}

int qnsch_ref_set_iterate(ref_solver* s, const double* c, const double* mu, const double* u,
                          const double* v, const double* p) {
  if (!s) return REF_EINVAL;
  if (!s->pending) return REF_ESTATE;
  ref_level* F = &s->lev[0];
  pack_in(F, c ? F->c : NULL, mu ? F->mu : NULL, p ? F->p : NULL, u ? F->u : NULL,
          v ? F->v : NULL, c, mu, p, u, v);
  return REF_OK;
}

int qnsch_ref_get_iterate(const ref_solver* s, double* c, double* mu, double* u, double* v,
                          double* p) {
  if (!s) return REF_EINVAL;
  if (!s->pending) return REF_ESTATE;
  const ref_level* F = &s->lev[0];
  pack_out(F, F->c, F->mu, F->p, F->u, F->v, c, mu, p, u, v);
  return REF_OK;
}

int qnsch_ref_residual(ref_solver* s, double* rc, double* rmu, double* rp, double* ru,
                       double* rv, double* norms10) {
  if (!s) return REF_EINVAL;
  if (!s->pending) return REF_ESTATE;
  ref_level* F = &s->lev[0];
  residual(&s->P, F, s->dt, norms10);
  pack_out(F, F->rc, F->rmu, F->rp, F->ru, F->rv, rc, rmu, rp, ru, rv);
  return REF_OK;
}

int qnsch_ref_smooth_ch(ref_solver* s, int colour) {
  if (!s || colour < 0 || colour > 1) return REF_EINVAL;
  if (!s->pending) return REF_ESTATE;
  smooth_ch(&s->P, &s->lev[0], s->dt, colour);
  return REF_OK;
}

int qnsch_ref_smooth_vanka(ref_solver* s, int colour) {
  if (!s || colour < 0 || colour >= s->kcol) return REF_EINVAL;
  if (!s->pending) return REF_ESTATE;
  smooth_vanka(&s->P, &s->lev[0], s->dt, s->kcol, colour, s->omega);
  return REF_OK;
}

int qnsch_ref_smooth(ref_solver* s, int sweeps) {
  if (!s) return REF_EINVAL;
  if (!s->pending) return REF_ESTATE;
  for (int k = 0; k < sweeps; ++k) smooth(s, &s->lev[0]);
  return REF_OK;
}

int qnsch_ref_ch_jacobian(ref_solver* s, int i, int j, double* J4, double* R2) {
  if (!s || !s->pending) return REF_ESTATE;
  ref_level* F = &s->lev[0];
  if (i < 1 || i > F->m1 || j < 1 || j > F->m2) return REF_EINVAL;
  ch_jac(&s->P, F, s->dt, i, j, J4);
  R2[0] = N_c(&s->P, F, s->dt, i, j) - F->fc[CI(F, i, j)];
  R2[1] = N_mu(&s->P, F, i, j) - F->fmu[CI(F, i, j)];
  return REF_OK;
}

int qnsch_ref_vanka_jacobian(ref_solver* s, int i, int j, double* J25, double* R5, int* active5) {
  if (!s || !s->pending) return REF_ESTATE;
  ref_level* F = &s->lev[0];
  if (i < 1 || i > F->m1 || j < 1 || j > F->m2) return REF_EINVAL;
  vanka_block(&s->P, F, s->dt, i, j, J25, R5, active5);
  return REF_OK;
}

int qnsch_ref_mass(const ref_solver* s, double* mass_rho, double* mass_rhoc) {
  if (!s || !mass_rho || !mass_rhoc) return REF_EINVAL;
  mass_of(&s->P, &s->lev[0], s->c, mass_rho, mass_rhoc);
  return REF_OK;
}

int qnsch_ref_energy(const ref_solver* s, double* E) {
  if (!s || !E) return REF_EINVAL;
  ref_level* F = &s->lev[0];
  *E = energy_of(&s->P, F, s->c, s->u, s->v);
  return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* Diagnostics of the experiments of Sec. 8, on the committed state          */
/* ------------------------------------------------------------------------ */

/* u_{i+1/2,j}, i = 0..m1: zero on no-slip walls, period m1 in x */
static double edge_u(const ref_solver* s, int i, int j) {
  const ref_level* L = &s->lev[0];
  if (!L->px && (i == 0 || i == L->m1)) return 0.0;
  if (L->px && i == 0) i = L->m1;
  return s->u[UI(L, i, j)];
}

/* v_{i,j+1/2}, j = 0..m2: zero on the no-slip walls in y */
static double edge_v(const ref_solver* s, int i, int j) {
  const ref_level* L = &s->lev[0];
  if (j == 0 || j == L->m2) return 0.0;
  return s->v[VI(L, i, j)];
}

/* discrete divergence d_x u + d_y v of cell (i,j) (Sec. 5; the quantity
   plotted for the rising droplet, Sec. 8.2) */
static double div_at(const ref_solver* s, int i, int j) {
  double h = s->lev[0].h;
  return (edge_u(s, i, j) - edge_u(s, i - 1, j)) / h + (edge_v(s, i, j) - edge_v(s, i, j - 1)) / h;
}

int qnsch_ref_divergence(const ref_solver* s, double* out) {
  if (!s || !out) return REF_EINVAL;
  const ref_level* L = &s->lev[0];
  for (int j = 1; j <= L->m2; ++j)
    for (int i = 1; i <= L->m1; ++i) out[(size_t)(j - 1) * L->m1 + (i - 1)] = div_at(s, i, j);
  return REF_OK;
}

/* out[0] rise velocity V_c = sum c a_y(v) / sum c (Sec. 8.2), a_y(v) the mean
   of the two ns edges of the cell; out[1] centroid height sum c y / sum c;
   out[2] max |div|, out[3] (h^2 sum div^2)^(1/2), out[4] max(div, 0),
   out[5] max(-div, 0); out[6] a1 = (2/m1) sum_i eta_i cos(2 pi x_i / Lx), the
   first cosine mode of the column height eta_i = h sum_j c_ij of the c = 1
   fluid: for an interface y0 + a cos(2 pi x / Lx) with c = 1 below, a1 = a
   (the capillary-wave amplitude of Sec. 8.1, where the paper's interface
   0.5 - H0 cos(2 pi x) has a1 = -H0); out[7], out[8] the highest and lowest
   upward crossing c_j >= 1/2 > c_{j+1} over all columns, by linear
   interpolation between cell centres (top of the rising and bottom of the
   falling fluid, Sec. 8.3); 0 and Ly when no column has a crossing. */
int qnsch_ref_diagnostics(const ref_solver* s, double* out) {
  if (!s || !out) return REF_EINVAL;
  const ref_level* L = &s->lev[0];
  const int m1 = L->m1, m2 = L->m2;
  const double h = L->h, Lx = m1 * h, Ly = m2 * h;
  const double pi = 3.14159265358979323846;
  double sc = 0.0, scv = 0.0, scy = 0.0, d2 = 0.0, dmax = 0.0, dpos = 0.0, dneg = 0.0;
  for (int j = 1; j <= m2; ++j)
    for (int i = 1; i <= m1; ++i) {
      double c = s->c[CI(L, i, j)];
      double vbar = 0.5 * (edge_v(s, i, j) + edge_v(s, i, j - 1));
      double d = div_at(s, i, j);
      sc += c;
      scv += c * vbar;
      scy += c * ((j - 0.5) * h);
      d2 += d * d;
      if (fabs(d) > dmax) dmax = fabs(d);
      if (d > dpos) dpos = d;
      if (-d > dneg) dneg = -d;
    }
  double Hs = 0.0, ytop = 0.0, ybot = Ly;
  int found = 0;
  for (int i = 1; i <= m1; ++i) {
    double eta = 0.0;
    for (int j = 1; j <= m2; ++j) eta += s->c[CI(L, i, j)];
    eta *= h;
    Hs += eta * cos(2.0 * pi * ((i - 0.5) * h) / Lx);
    for (int j = 1; j < m2; ++j) {
      double a = s->c[CI(L, i, j)], b = s->c[CI(L, i, j + 1)];
      if (a >= 0.5 && b < 0.5) {
        double y = (j - 0.5) * h + h * (a - 0.5) / (a - b);
        if (!found || y > ytop) ytop = y;
        if (!found || y < ybot) ybot = y;
        found = 1;
      }
    }
  }
  out[0] = scv / sc;
  out[1] = scy / sc;
  out[2] = dmax;
  out[3] = sqrt(h * h * d2);
  out[4] = dpos;
  out[5] = dneg;
  out[6] = 2.0 / m1 * Hs;
  out[7] = ytop;
  out[8] = ybot;
  return REF_OK;
}

int qnsch_ref_iterate_energy(const ref_solver* s, double* E) {
  if (!s || !E) return REF_EINVAL;
  if (!s->pending) return REF_ESTATE;
  const ref_level* F = &s->lev[0];
  if (s->P.scheme) {
    double *u = zalloc(nu_(F)), *v = zalloc(nv_(F));
    if (!u || !v) {
      free(u);
      free(v);
      return REF_ENOMEM;
    }
    projected_velocity(&s->P, F, s->dt, u, v);
    *E = energy_of(&s->P, F, F->c, u, v);
    free(u);
    free(v);
  } else {
    *E = energy_of(&s->P, F, F->c, F->u, F->v);
  }
  return REF_OK;
}

int qnsch_ref_iterate_dissipation(const ref_solver* s, double* D) {
  if (!s || !D) return REF_EINVAL;
  if (!s->pending) return REF_ESTATE;
  const ref_level* F = &s->lev[0];
  *D = dissipation_of(&s->P, F, s->dt);
  if (s->P.scheme) {
    double *u = zalloc(nu_(F)), *v = zalloc(nv_(F));
    if (!u || !v) {
      free(u);
      free(v);
      return REF_ENOMEM;
    }
    projected_velocity(&s->P, F, s->dt, u, v);
    *D += projection_dissipation(&s->P, F, u, v);
    free(u);
    free(v);
  }
  return REF_OK;
}

/* projection method: u^{n+1}, v^{n+1} of the current iterate in the host
   layout of qnsch_ref_get_fields */
int qnsch_ref_projected_velocity(const ref_solver* s, double* hu, double* hv) {
  if (!s || !hu || !hv) return REF_EINVAL;
  if (!s->pending || !s->P.scheme) return REF_ESTATE;
  const ref_level* F = &s->lev[0];
  double *u = zalloc(nu_(F)), *v = zalloc(nv_(F));
  if (!u || !v) {
    free(u);
    free(v);
    return REF_ENOMEM;
  }
  projected_velocity(&s->P, F, s->dt, u, v);
  pack_out(F, NULL, NULL, NULL, u, v, NULL, NULL, NULL, hu, hv);
  free(u);
  free(v);
  return REF_OK;
}
