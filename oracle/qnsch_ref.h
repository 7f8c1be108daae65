/*
 * qnsch_ref.h -- ORACLE (test infrastructure only).
 *
 * Plain, serial, FP64 CPU restatement of the fully discrete primitive scheme of
 * Guo, Lin, Lowengrub & Wise (arXiv:1703.06606), Sec. 6.1 (equations pm-num-mx,
 * pm-num-mass, pm-num-phase, pm-num-chem with e1e1-1, e1e1-2, e1e1, e1e2) on the
 * staggered MAC grid of Sec. 5 / Appendix A, and of the FAS multigrid of Sec. 7.1
 * (CH nonlinear Gauss-Seidel, Vanka smoothing for Navier-Stokes, V-cycle).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this library.  It shares no code with the CUDA path.
 *
 * Host array layouts (row-major, x fastest, no ghost cells):
 *   c, mu, p : m2 rows x m1       (cell centres (i,j), i=1..m1, j=1..m2)
 *   u        : m2 rows x (m1+1)   (u_{i+1/2,j}, i=0..m1)
 *   v        : (m2+1) rows x m1   (v_{i,j+1/2}, j=0..m2)
 * With walls in x the columns i=0 and i=m1 of u are zero; y is always bounded by
 * no-slip walls, so rows j=0 and j=m2 of v are zero.  With periodic x, u_{1/2}
 * and u_{m1+1/2} are one unknown; inputs take column m1 and outputs write both.
 */
#ifndef QNSCH_REF_H
#define QNSCH_REF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ref_solver ref_solver;

/* Status codes (same meaning as the product library's). */
#define REF_OK 0
#define REF_EINVAL (-1)
#define REF_ENOMEM (-3)
#define REF_ENOTCONV (-4)
#define REF_ESTATE (-8)

int qnsch_ref_create(int m1, int m2, double Lx, int periodic_x, int levels,
                     double rho1, double rho2, double eta1, double eta2,
                     double Re, double We, double Pe, double Cn, double Fr,
                     ref_solver** out);
int qnsch_ref_destroy(ref_solver* s);
int qnsch_ref_set_option(ref_solver* s, const char* key, double value);
int qnsch_ref_get_option(const ref_solver* s, const char* key, double* value);
int qnsch_ref_levels(const ref_solver* s);

/* committed state (time level n) */
int qnsch_ref_set_fields(ref_solver* s, const double* c, const double* mu,
                         const double* u, const double* v, const double* p);
int qnsch_ref_get_fields(const ref_solver* s, double* c, double* mu, double* u,
                         double* v, double* p);
/* option "predictor" (0, 1, 2): the initial iterate of a step extrapolated in
   time from the committed state and the last one or two states committed
   before it; these calls read and set those states (k = 0 the most recent)
   and the step sizes that left them */
int qnsch_ref_get_history(const ref_solver* s, int k, double* dt, double* c, double* mu,
                          double* u, double* v, double* p);
int qnsch_ref_set_history(ref_solver* s, int k, double dt, const double* c, const double* mu,
                          const double* u, const double* v, const double* p);

/* one time step = begin + outer V-cycles until tol + commit */
int qnsch_ref_step(ref_solver* s, double dt, int* n_vcycles, double* final_res);
int qnsch_ref_begin_step(ref_solver* s, double dt);
int qnsch_ref_vcycle(ref_solver* s, double* norms10);
int qnsch_ref_commit_step(ref_solver* s);

/* pending iterate x on the finest level (valid between begin and commit) */
int qnsch_ref_set_iterate(ref_solver* s, const double* c, const double* mu,
                          const double* u, const double* v, const double* p);
int qnsch_ref_get_iterate(const ref_solver* s, double* c, double* mu, double* u,
                          double* v, double* p);
/* r = f - N(x) on the finest level (f = 0 there); norms10 = [l2 x5, max x5] */
int qnsch_ref_residual(ref_solver* s, double* rc, double* rmu, double* rp,
                       double* ru, double* rv, double* norms10);
/* single smoother pieces on the finest level (tests) */
int qnsch_ref_smooth_ch(ref_solver* s, int colour);
int qnsch_ref_smooth_vanka(ref_solver* s, int colour);
int qnsch_ref_smooth(ref_solver* s, int sweeps);
int qnsch_ref_ncolours_vanka(const ref_solver* s);
/* local Jacobians at one cell of the finest level, row-major (tests) */
int qnsch_ref_ch_jacobian(ref_solver* s, int i, int j, double* J4, double* R2);
int qnsch_ref_vanka_jacobian(ref_solver* s, int i, int j, double* J25,
                             double* R5, int* active5);

/* diagnostics */
int qnsch_ref_mass(const ref_solver* s, double* mass_rho, double* mass_rhoc);
int qnsch_ref_energy(const ref_solver* s, double* E);
int qnsch_ref_iterate_energy(const ref_solver* s, double* E);
int qnsch_ref_iterate_dissipation(const ref_solver* s, double* D);
int qnsch_ref_params(const ref_solver* s, double* out8);
/* The pointwise functions of Sec. 2.1 and the secants of Sec. 4.1 at (a, b), for
   tests: F(a), F(b), g(a,b), dg/da(a,b), rho(a), rho(b), r(a,b). */
int qnsch_ref_secants(const ref_solver* s, double a, double b, double* out7);
/* The FAS grid transfers between level l and l+1 (reading R8), for tests, in
   the host layouts of qnsch_ref_get_fields: op 0, 1, 2 restrict a fine
   residual of cells, x-edges, y-edges to the coarse level (cell average;
   full weighting on edges); op 3, 4, 5 prolongate a coarse correction of
   cells, x-edges, y-edges to the fine level; op 6, 7 restrict the iterate's
   x-edges, y-edges (the mean of the two coincident fine edges; cells use op 0). */
int qnsch_ref_transfer(const ref_solver* s, int l, int op, const double* in, double* out);
/* Sec. 8 diagnostics of the committed state (see qnsch_ref.c): out9 = {V_c,
   centroid y, max|div|, l2 div, max expansion, max compression, a1, y_top,
   y_bottom}; divergence field out[(j-1)*m1 + (i-1)], m1*m2 values. */
int qnsch_ref_diagnostics(const ref_solver* s, double* out9);
/* projection method (option "scheme" = 1): u^{n+1}, v^{n+1} of the pending
   iterate, host layout of qnsch_ref_get_fields */
int qnsch_ref_projected_velocity(const ref_solver* s, double* hu, double* hv);
int qnsch_ref_divergence(const ref_solver* s, double* out);

#ifdef __cplusplus
}
#endif
#endif
