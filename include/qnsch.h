/*
 * qnsch.h -- C ABI of the GB300 library for one implicit time step of the
 * primitive method for the quasi-incompressible Navier-Stokes-Cahn-Hilliard
 * system of Guo, Lin, Lowengrub & Wise (arXiv:1703.06606).
 *
 * Problem (Sec. 6.1): given (c^n, mu^n, p^n, u^n, v^n) on an m1 x m2 staggered
 * MAC grid (Sec. 5, App. A) with spacing h = Lx/m1, find the level n+1 fields
 * solving the fully discrete primitive scheme, equations (pm-num-mx),
 * (pm-num-mass), (pm-num-phase) and (pm-num-chem).  mu is the paper's mu-bar_c
 * and p its p-bar.  The nonlinear system is solved by FAS multigrid V-cycles
 * (Sec. 7.1) until the largest of the five scaled residual norms
 * (h^2 sum r^2)^{1/2} is at most `tol`.
 *
 * Boundaries: y is bounded by no-slip walls (u = v = 0, Neumann data for c, mu, p;
 * App. A.6).  x is either periodic or bounded by the same walls.
 *
 * Host array layouts (row-major, x fastest, no ghost cells; all FP64):
 *   c, mu, p : m2 rows x m1 columns        (cell (i,j), i = 1..m1, j = 1..m2)
 *   u        : m2 rows x (m1+1) columns    (u_{i+1/2,j}, i = 0..m1)
 *   v        : (m2+1) rows x m1 columns    (v_{i,j+1/2}, j = 0..m2)
 * Wall entries (columns 0 and m1 of u with walls in x, rows 0 and m2 of v) are
 * ignored on input and returned as 0.  With periodic x, u_{1/2} and u_{m1+1/2}
 * are one unknown: inputs take column m1, outputs write both columns.
 *
 * Ownership: the handle owns all device memory it allocates, until
 * qnsch_destroy.  Arrays passed in are copied; the library keeps no pointer to
 * caller memory.  Device memory comes from the allocator set by
 * qnsch_set_allocator (cudaMalloc/cudaFree by default).  All work is issued on
 * the stream set by qnsch_set_stream; without one, on a private stream of the
 * handle that the device-array calls order after the caller's earlier work on
 * the legacy default stream.  Every call returns only after its work has
 * completed, unless stated.  Each outer V-cycle is captured once as a CUDA
 * graph and replayed, the host reading the norms between cycles (option
 * "graphs", default 1); with option "device_loop" = 1, qnsch_step instead runs
 * the whole step as one CUDA graph whose outer-cycle loop and convergence test
 * run on the device.  Graphs are recaptured when dt or an option changes.
 *
 * Every call returns an int status: 0 on success, a negative QNSCH_E* code on
 * failure.  On failure no output is written and, unless stated, the handle is
 * unchanged.
 */
#ifndef QNSCH_H
#define QNSCH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Version of this interface.  The major number changes when a call's meaning
   or signature changes, the minor number when calls or options are added. */
#define QNSCH_VERSION_MAJOR 1
#define QNSCH_VERSION_MINOR 0
#define QNSCH_VERSION_PATCH 0

#define QNSCH_OK 0
#define QNSCH_EINVAL (-1)   /* bad argument or option */
#define QNSCH_ENODEV (-2)   /* no CUDA device */
#define QNSCH_ENOMEM (-3)   /* allocation failed */
#define QNSCH_ENOTCONV (-4) /* maxcyc V-cycles without reaching tol; step not committed */
#define QNSCH_ENAN (-5)     /* non-finite residual; step not committed */
#define QNSCH_ETIMEOUT (-6) /* step_time_limit reached before tol; step not committed */
#define QNSCH_EBUDGET (-7)  /* the device-memory budget (qnsch_set_budget) would be exceeded */
#define QNSCH_ESTATE (-8)   /* call not valid in the current state (e.g. vcycle outside a step) */
#define QNSCH_ECUDA (-9)    /* a CUDA call failed */

/* The library's version (any pointer may be NULL): compare with the
   QNSCH_VERSION_* macros of the header a program was compiled against. */
int qnsch_version(int* major, int* minor, int* patch);

typedef struct qnsch_s qnsch_t;

typedef struct {
  int m1, m2;      /* cells in x and y; m1, m2 >= 2; periodic x needs m1 even, >= 4 */
  double Lx;       /* domain width; h = Lx / m1, height Ly = m2 h */
  int periodic_x;  /* 1: periodic in x; 0: no-slip walls in x */
  int periodic_y;  /* must be 0: y is always bounded by walls */
  int levels;      /* multigrid levels; 0 = deepest the grid allows */
} qnsch_grid;
/* Size limit: the padded index space of one array, (m1 + 3 rounded up to a
   multiple of 32) x (m2 + 3) elements, must not exceed 2^31 - 1, because the
   kernels index arrays with 32-bit integers; larger grids give QNSCH_EINVAL
   from qnsch_create and qnsch_footprint.
   Coarsening halves both sides.  A level is added while both sides of the
   current coarsest grid are even and the halved grid keeps at least 2 cells
   per side (periodic x: at least 4 cells across, an even number). */

/* Device allocator of the handles created from now on (process-wide).
   alloc(bytes, ctx) returns device memory or NULL; free(ptr, ctx) releases it.
   Passing NULL for both restores cudaMalloc/cudaFree.  A handle allocates and
   frees through the allocator in effect when it was created, for its whole
   life: changing the allocator affects only handles created afterwards. */
int qnsch_set_allocator(void* (*alloc)(size_t bytes, void* ctx),
                        void (*free_fn)(void* ptr, void* ctx), void* ctx);

/* Create a solver for one instance (Sec. 6.1 statement of the problem).
   rho1, rho2: densities of the fluids at c = 1 and c = 0 (Sec. 2.1);
   eta1, eta2: their viscosities (the paper's mu_1, mu_2);
   Re, We, Pe: Reynolds, Weber, Peclet numbers (Sec. 2.2); Cn: interface
   parameter epsilon; Fr: Froude number, INFINITY (or <= 0) for no gravity.
   Derived (Sec. 8): M = Cn, eta = eta(rho1, rho2) of Sec. 8.1, mobility
   regularisation eps = Cn; each can be overridden with qnsch_set_option.
   Returns QNSCH_EINVAL for an invalid grid or parameter (a non-finite Lx, a
   NaN Fr, a density, viscosity, Re, We, Pe or Cn that is not > 0), QNSCH_EBUDGET when
   the handle's footprint would exceed the budget (qnsch_set_budget), and
   QNSCH_ENODEV without a CUDA device, checked in that order. */
int qnsch_create(const qnsch_grid* grid, double rho1, double rho2, double eta1, double eta2,
                 double Re, double We, double Pe, double Cn, double Fr, qnsch_t** out);
int qnsch_destroy(qnsch_t* h);

/* Device-memory budget of the process (no counterpart in the paper; the limit a
   server admits work under).  qnsch_set_budget(bytes) sets it; 0 (the default)
   means none.  Every handle reserves its qnsch_footprint at creation
   (precision 0) and the error-equation levels' bytes when the first step at
   precision 1 or 2 allocates them; qnsch_destroy releases both.  A creation or
   a step whose reservation would take the reserved total above the budget
   fails with QNSCH_EBUDGET and allocates nothing (a step so refused is not
   started).  qnsch_create checks the budget before it looks for a device, so
   the refusal also comes without one.  Reservations are atomic, so threads
   creating handles at once never overshoot.  Lowering the budget below what
   is reserved frees nothing; it only refuses new reservations.
   qnsch_budget writes the budget and the bytes reserved (either pointer may be
   NULL, not both). */
int qnsch_set_budget(size_t bytes);
int qnsch_budget(size_t* budget, size_t* in_use);
/* Device bytes a handle for `grid` holds once created and stepped with the
   given "precision" option (0, 1 or 2), computed without allocating. */
int qnsch_footprint(const qnsch_grid* grid, int precision, size_t* bytes);

/* Options (key: default): "nu1": 2, "nu2": 2 (pre/post smoothing steps),
   "nu_coarse": 4 (smoothing steps on the coarsest level; a coarsest grid whose
   longest side n exceeds 4 cells gets nu_coarse * ceil(n/4)^2), "tol": 1e-9,
   "maxcyc": 50, "omega_vanka": 1, "M": Cn, "eta_st": eta(rho1, rho2),
   "eps_mob": Cn, "precision": 0, "graphs": 1, "fuse_cells": 128,
   "fuse_cells32": 512, "fuse_ctas": 1, "coupled": 0, "scheme": 0, "vanka_team_max": 8192,
   "vanka_team8_max": 0, "vanka_pair_max": 0, "vanka_split": 0, "coarse_smem": 1,
   "ch_team_max": 4096, "vanka_team_max32": 65536, "ch_team_max32": 0,
   "pdl": 1, "step_time_limit": 0, "diverge_cycles": 0, "device_loop": 0,
   "wave_cells32": 0, "wave_rows": 8, "wave_wait_cycles": 2147483648,
   "wave_stall": 0, "skew_cells32": 0, "skew_rows": 32, "predictor": 0,
   "nu1_fine": -1, "nu2_fine": -1.
   Unknown keys give QNSCH_EINVAL, and so do values out of range, which leave
   the option unchanged: NaN for any key; counts that are not integers in
   their range (nu1, nu2, nu_coarse: 0..1000; maxcyc, diverge_cycles:
   0..10^6; precision: 0..2; scheme: 0..1; fuse_ctas: 1, 2, 4, 8 or 16;
   fuse_cells, fuse_cells32 and the
   four team thresholds: 0..2^31 - 1); tol or step_time_limit negative or
   infinite; omega_vanka, M, eta_st or eps_mob not positive and finite.
   step_time_limit (seconds, >= 0; 0: none): before each outer cycle of a
   step, the step checks the time since it began (with device_loop, the GPU's
   global timer since the step's first kernel; without, the host's wall clock
   since the call began, or since qnsch_batch_step's call began) and, once it
   exceeds the limit with the residual still above tol, stops and returns
   QNSCH_ETIMEOUT without committing the step.  A cycle already running goes
   to its end, so a step can overrun the limit by one outer cycle.
   wave_cells32 (integer >= 0; 0: never): error-equation levels (precision 1
   and 2) with at least this many cells and at least 2 wave_rows rows run
   each block of nu smoothing steps as one banded wavefront launch instead of
   one launch per colour: the passes (CH red and black, then the Vanka or
   coupled colours) run band by band (bands of wave_rows >= 4 rows) in a
   skewed order, each band's pass waiting only for the previous pass on the
   band and its two neighbours, so a band stays in L2 across its passes.  The
   results are the per-colour launches' up to rounding (the same arithmetic on
   the same values).  Its waits are
   bounded by wave_wait_cycles SM clock cycles (integer >= 0); a wait that runs
   out ends the step with QNSCH_ETIMEOUT, uncommitted.  wave_stall (0 or 1) is
   a test hook for that path: with 1, one wait of every wavefront launch waits
   for a count nothing reaches.
   nu1_fine, nu2_fine (integers -1..1000; -1: nu1, nu2): the smoothing
   steps before and after the coarse-grid correction on the finest level
   only, so that the levels below can run fewer (nu1, nu2).  A finest level
   with counts of its own is never fused into the single-block coarse
   V-cycle.
   predictor (0, 1 or 2): the initial iterate of a step.  0 (the default):
   the committed state x^n.  1 or 2: the polynomial in time through x^n and
   the last one or two states committed before it (qnsch_get_history),
   evaluated at the new time t + dt, with the step sizes as they were
   (Lagrange interpolation on unequal nodes); with fewer states held, the
   highest order they allow.  The predicted iterate only moves the start of
   the outer cycles: the step still stops at the same residual tolerance.
   Setting the option clears the history; each committed step adds to it.
   history (read-only; 0 clears it): the number of earlier states held.
   skew_cells32 (integer >= 0; 0: never; checked before wave_cells32):
   error-equation levels with at least this many cells run each block of nu
   smoothing steps in the skewed-chunk schedule: launch d runs pass p (the
   passes of the nu steps as above) on the rows [1 + (d - p) R - 2p,
   1 + (d - p + 1) R - 2p) for R = skew_rows (integer >= 1), one lane per
   visit.  No block waits for another: every visit reads rows within 2 below
   and 1 above its own and writes within 1 below, so the tasks of one launch
   are independent and stream order orders the rest.  The results are those
   of the per-colour launches with one lane per visit, bit for bit (the same
   device code on the same values).  Measured on the 1024 x 4096 mixed
   workload: 1.7x less DRAM traffic per smoothing block and 1.25x more time.
   device_loop: 1 (with graphs = 1 and profiling off) runs qnsch_step and
   qnsch_step_launch as one graph per step: the initial residual, a
   conditional WHILE node around the outer cycle whose last kernel applies the
   stopping rules above (tol, maxcyc, diverge_cycles, step_time_limit) on the
   device, a conditional IF node around the commit, and one copy of the
   outcome to the host; no host round trip per cycle.  Results, cycle counts
   and statuses are those of the host-driven loop (0, the default).  Measured:
   no faster for one instance (the host keeps ahead of the GPU), slower for
   many instances stepping at once, and a graph with conditional nodes cannot
   be profiled kernel by kernel; hence off by default.  If the runtime refuses
   to build that graph the handle sets device_loop to 0 and steps with the
   host-driven loop.
   diverge_cycles (integer >= 0; 0: never): a step whose largest family
   residual has grown over this many consecutive outer cycles stops early and
   returns QNSCH_ENOTCONV without committing (failure detection for a step that
   would otherwise spend maxcyc cycles diverging).
   scheme: 0 the primitive method (Sec. 6.1); 1 the projection method
   (Sec. 6.2; precision 0 and coupled 0 only).
   vanka_team_max: FP64 levels with at most this many cells per Vanka colour
   run the per-level Vanka launches with four lanes per 5x5 block (same
   arithmetic, shorter critical path when the colour leaves most of the GPU
   idle); ch_team_max does the same for the CH 2x2 Newton launches (four lanes
   per cell, one face each); vanka_team_max32 for the Vanka launches on the
   error-equation levels of the defect correction (precision 1 and 2), which
   are latency-bound up to a few hundred thousand cells per colour, and
   ch_team_max32 for their CH launches.
   vanka_team_max and vanka_team_max32 also choose the four-lane launches of
   the coupled 7x7 block (coupled = 1).
   vanka_team8_max: FP64 full-iterate levels with at most this many cells per
   Vanka colour run the 5x5 blocks with eight lanes, each lane pair splitting
   one momentum row's residual in two halves (a shorter chain of dependent
   instructions per lane; same arithmetic up to the order of two additions);
   a value > 0 also uses eight lanes in the single-block coarse V-cycle where
   a colour fits the block in one pass.  0 (the default): never.
   vanka_pair_max: FP64 full-iterate levels above vanka_team_max with at most
   this many cells per Vanka colour run the 5x5 blocks with a lane pair, the
   x pair of rows (W, E) on one lane and the y pair (S, N) on the other, each
   lane factoring its own 2x2 block of the structured solve (half the FP64
   instructions per lane of one lane per block; the four-lane team's
   arithmetic).  0 (the default): never.
   vanka_split: FP64 full-iterate Vanka launches that would run one lane per
   block split their colour instead: the first slots one lane each (a whole
   number of warps, launched first), the rest as lane pairs.  1: where a cost
   model of the busiest SM sub-partition finds it cheaper, for colours that
   fill the sub-partitions more than once (the finest level of the 256x512
   droplet: one round of single-lane warps and one round of pair warps in
   place of two single-lane rounds, the second mostly empty); a value >= 2:
   that many slots, rounded down to a multiple of 32, one lane each; 0 (the
   default): never.  Each block is visited as vanka_cell or vanka_pair would.
   coarse_smem: 1 (the default) runs the fused V-cycle of the coarse FP64
   full-iterate levels (fuse_cells, in one thread block: fuse_ctas = 1) on a
   copy of those levels in shared memory, made at the start of the launch and
   written back at its end, wherever the copy fits the device's shared memory
   per block (about 151 KB for the 8x16, 4x8 and 2x4 levels); 0 runs it from
   global memory.  The same device code runs on the same values, so the
   results are the same.  Reading the key "coarse_smem_used" (get only) gives
   1 if the last fused launch ran on the shared-memory copy.
   pdl: 1 launches every kernel with programmatic dependent launch, so that
   a kernel is scheduled as its predecessor's blocks exit and waits on the GPU
   for the predecessor's results before touching memory (same results); 0
   launches in plain stream order.  It applies to every handle of the process
   and takes effect at the next graph capture.
   coupled: 0 smooths with the paper's separate sweeps (CH 2x2 red-black, then
   the Vanka 5x5 colours, Sec. 7.1); 1 replaces them by one sweep over the
   Vanka colours of a coupled 7x7 Newton block in (c, mu, u_W, u_E, v_S, v_N, p).
   Same fixed point; the coupled block keeps converging on fine grids where the
   separate sweeps stall (the CH/NS coupling through (alpha/Pe) div(m grad(mu +
   alpha p)) grows like 1/h^2).
   fuse_cells / fuse_cells32: the V-cycle on every FP64 / FP32 level with at
   most this many cells runs in one launch for all of them (same arithmetic
   and order as the per-level launches; 0 disables).
   fuse_ctas: that launch is one thread block (1) or one thread-block cluster
   of fuse_ctas blocks on as many SMs, its colour steps separated by the
   cluster barrier.  Sizes above 8 need the non-portable cluster size; the
   handle keeps the largest size not above the one asked for that the current
   device can launch (read it back with qnsch_get_option).  Set it outside
   stream capture: it queries the runtime.
   precision 0: FAS V-cycles in FP64 on the scheme itself.
   precision 1: mixed.  Each outer cycle forms the FP64 residual r = -N(x),
     runs one FAS V-cycle in FP32 on the error equation N(x + e) - N(x) = r
     (smoothing, transfers and coarse levels in FP32; every nonlinear
     difference written with the secant identities of Sec. 4.1, so nothing
     cancels in FP32), adds e to x in FP64 and removes the mean of p in FP64.
     Convergence is still judged on the FP64 residual, so the step meets the
     same tol.
   precision 2: as 1 with an FP64 error cycle (a check of the error form).
   "precision" cannot change between qnsch_begin_step and qnsch_commit_step. */
int qnsch_set_option(qnsch_t* h, const char* key, double value);
int qnsch_get_option(const qnsch_t* h, const char* key, double* value);
/* Issue the handle's work on `cuda_stream` (a cudaStream_t; NULL: the
   handle's private non-blocking stream, which the device-array calls order
   after the caller's earlier work on the legacy default stream).  Waits for
   the work queued so far on the previous stream. */
int qnsch_set_stream(qnsch_t* h, void* cuda_stream);
int qnsch_levels(const qnsch_t* h);          /* number of levels, or < 0 */
int qnsch_ncolours_vanka(const qnsch_t* h);  /* Vanka colours on the finest level */

/* Committed state (time level n, the fields of the scheme of Sec. 6.1): host
   arrays in the layouts above, copied in or out before the call returns.
   set_fields needs all five pointers (QNSCH_EINVAL) and no pending step
   (QNSCH_ESTATE); get_fields skips NULL pointers. */
int qnsch_set_fields(qnsch_t* h, const double* c, const double* mu, const double* u,
                     const double* v, const double* p);
int qnsch_get_fields(const qnsch_t* h, double* c, double* mu, double* u, double* v, double* p);
/* Same, with device pointers in the same (dense, ghost-free) layouts.  Without
   a stream set by qnsch_set_stream they are ordered after the caller's earlier
   work on the legacy default stream; with one, the caller orders its own work
   on that stream. */
int qnsch_set_fields_device(qnsch_t* h, const double* c, const double* mu, const double* u,
                            const double* v, const double* p);
int qnsch_get_fields_device(const qnsch_t* h, double* c, double* mu, double* u, double* v,
                            double* p);
/* The states committed before the current one, which the option "predictor"
   extrapolates from (k = 0 the most recent; get_option "history" gives how
   many are held, at most 2).  qnsch_get_history copies state k into host
   arrays in the layouts above (NULL pointers skipped) and its step size dt
   (the step that led from it to the next state); QNSCH_EINVAL if k is not
   below the count or dt is NULL.  qnsch_set_history sets state k and its dt
   (k at most the count, so k equal to the count appends; all five pointers;
   dt > 0 and finite; else QNSCH_EINVAL), for example to resume a run so that
   its next steps start from the same predicted iterates as the uninterrupted
   run's.  Both need no pending step (QNSCH_ESTATE).  qnsch_set_fields and
   qnsch_set_fields_device clear the history, and so do set_option
   "predictor" and set_option "history" = 0. */
int qnsch_get_history(const qnsch_t* h, int k, double* dt, double* c, double* mu, double* u,
                      double* v, double* p);
int qnsch_set_history(qnsch_t* h, int k, double dt, const double* c, const double* mu,
                      const double* u, const double* v, const double* p);

/* One time step of the scheme of Sec. 6.1 (primitive) or Sec. 6.2
   (projection, option scheme = 1), solved by the FAS V-cycles of Sec. 7.1 /
   7.2: qnsch_begin_step, then V-cycles until the largest scaled residual norm
   is <= tol, then qnsch_commit_step.  Writes the number of V-cycles and the
   final norm (either pointer may be NULL).  dt must be > 0 and finite
   (QNSCH_EINVAL); a step begun with qnsch_begin_step and not committed gives
   QNSCH_ESTATE.  Returns
   QNSCH_ENOTCONV, QNSCH_ENAN or QNSCH_ETIMEOUT, leaving the state at level n,
   when the iteration does not converge (maxcyc cycles, or diverge_cycles
   cycles of growth), turns non-finite or runs past step_time_limit; a
   refused budget reservation gives QNSCH_EBUDGET before any cycle. */
int qnsch_step(qnsch_t* h, double dt, int* n_vcycles, double* final_residual);
/* Freeze the level-n data of the step on every level (Sec. 6.1: restrict c^n,
   u^n, v^n; derive rho^n, m(c^n), mu(c^n), G(c^n) and the momentum rows'
   frozen coefficients) and start the iterate at the level-n fields.  dt > 0
   and finite, else QNSCH_EINVAL; a pending step is discarded and begun
   again. */
int qnsch_begin_step(qnsch_t* h, double dt);
/* One outer FAS V-cycle (Sec. 7.1; in mixed precision one defect-correction
   cycle) on the pending step, followed by removal of the mean of p; writes
   [scaled l2 norms of r_c, r_mu, r_p, r_u, r_v, then their max norms] after the
   cycle into host memory (NULL allowed).  QNSCH_ESTATE without a pending step. */
int qnsch_vcycle(qnsch_t* h, double* residual_norms10);
/* Accept the iterate as level n+1 (whatever its residual) and record the
   step's dissipation (Thm. 6.2).  QNSCH_ESTATE without a pending step. */
int qnsch_commit_step(qnsch_t* h);

/* Diagnostics of the experiments of Sec. 8, reduced in FP64 on the device from
   the committed state (the fields qnsch_get_fields returns) into host out[9]:
     out[0] V_c = sum c a_y(v) / sum c, the rise velocity of Sec. 8.2 (a_y(v)
            the mean of the cell's two ns edges);
     out[1] sum c y / sum c, the height of the c = 1 fluid's centroid;
     out[2] max |div|, out[3] (h^2 sum div^2)^(1/2), out[4] max(div, 0),
            out[5] max(-div, 0), div = d_x u + d_y v per cell (Sec. 8.2);
     out[6] a1 = (2/m1) sum_i eta_i cos(2 pi x_i / Lx), eta_i = h sum_j c_ij:
            the first cosine mode of the c = 1 column height; for an interface
            y0 + a cos(2 pi x / Lx) with c = 1 below, a1 = a (the capillary-wave
            amplitude of Sec. 8.1);
     out[7], out[8] the highest and lowest upward crossing c_j >= 1/2 > c_{j+1}
            over all columns, linear between cell centres: the top of the rising
            and the bottom of the falling fluid of Sec. 8.3 (0 and Ly if none).
   Wall-normal edge velocities count as zero; periodic edges wrap.  Blocks
   until the values are on the host. */
#define QNSCH_NDIAG 9
int qnsch_diagnostics(const qnsch_t* h, double* out);
/* d_x u + d_y v of the committed state into host div[(j-1)*m1 + (i-1)],
   m1*m2 doubles.  Blocks until copied. */
int qnsch_divergence(const qnsch_t* h, double* div);

/* Mass of the committed state (Thm. 6.1): h^2 sum rho(c), h^2 sum rho(c) c. */
int qnsch_mass(const qnsch_t* h, double* mass_rho, double* mass_rhoc);
/* Discrete energy E_h of the committed state (Thm. 6.2, norms of App. A.7), and
   the dissipation of the last committed step (0 before the first step). */
int qnsch_energy(const qnsch_t* h, double* E, double* last_dissipation);

/* Inspection of a pending step, host arrays in the layouts above (valid
   between begin_step and commit_step, else QNSCH_ESTATE; NULL arrays give
   QNSCH_EINVAL for set_iterate and are skipped by get_iterate). */
int qnsch_set_iterate(qnsch_t* h, const double* c, const double* mu, const double* u,
                      const double* v, const double* p);
int qnsch_get_iterate(const qnsch_t* h, double* c, double* mu, double* u, double* v, double* p);
/* r = f - N(x) on the finest level (f = 0 there; N the discrete operator of
   Sec. 6.1 or 6.2) into host arrays (NULL skips a family) and the ten norms of
   qnsch_vcycle.  QNSCH_ESTATE without a pending step. */
int qnsch_residual(qnsch_t* h, double* rc, double* rmu, double* rp, double* ru, double* rv,
                   double* norms10);
/* Smoother pieces on the finest level (Sec. 7.1): one colour of the CH
   nonlinear Gauss-Seidel (colour 0: (i+j) even), one colour of the Vanka
   smoother ((i+2j) mod 5 with walls in x; with periodic x (2i+j) mod 8 when
   m1 = 0 mod 4, else (i+2j) mod K, K the smallest divisor >= 5 of m1), or
   `sweeps` full smoothing steps (CH red, CH black, Vanka colours 0..K-1).
   A colour out of range or sweeps < 0 gives QNSCH_EINVAL, no pending step
   QNSCH_ESTATE. */
int qnsch_smooth_ch(qnsch_t* h, int colour);
int qnsch_smooth_vanka(qnsch_t* h, int colour);
int qnsch_smooth(qnsch_t* h, int sweeps);
/* Energy E_h of the pending iterate and the dissipation D_h of the step from
   the frozen data to it (Thm. 6.2).  QNSCH_ESTATE without a pending step. */
int qnsch_iterate_energy(const qnsch_t* h, double* E, double* D);

/* Measurement hooks (no counterpart in the paper).  qnsch_profile(h, mask)
   starts bracketing launches with pairs of CUDA events on the handle's stream
   (at most 4096 launches between reads) and resets the totals; mask 0 stops.
   Bit k of mask (0..63, else QNSCH_EINVAL) times the launches of kind k:
   0 the Vanka (or coupled, or projection 4x4) smoother on the finest level,
   1 the same smoother's per-level launches on the levels below it,
   2 the fused single-block V-cycle of the coarse levels, 3 the CH smoother on
   the finest level, 4 the banded wavefront launches on the finest level
   (wave_cells32; visits: cells x smoothing steps), 5 the skewed-chunk
   schedule on the finest level (skew_cells32; one timed entry per block of
   smoothing steps, however many launches it holds; visits: cells x
   smoothing steps).  Timing inserts event records into the replayed cycle
   graph, so while any bit is set qnsch_step drives its cycles from the host
   (device_loop is not used).  qnsch_profile_read synchronises the stream and
   returns the number of timed launches and their summed device time in
   milliseconds over all kinds; qnsch_profile_read_kind returns the same for
   one kind plus the cell visits those launches made (for the fused V-cycle:
   one visit per cell of each of its levels per smoothing step). */
int qnsch_profile(qnsch_t* h, int enable);
int qnsch_profile_read(qnsch_t* h, long long* launches, double* total_ms);
int qnsch_profile_read_kind(qnsch_t* h, int kind, long long* launches, double* total_ms,
                            double* visits);
/* Number of CUDA kernels this library has issued since it was loaded
   (process-wide, counted on the host at launch). */
int qnsch_kernel_launches(long long* n);
/* Asynchronous step (no counterpart in the paper; the interface a server
   uses to advance many instances without waiting for the slowest).
   qnsch_step_launch starts one step of size dt on the handle's stream and
   returns without waiting.  With device_loop on it queues the whole step graph;
   with device_loop = 0 it queues the step's start and initial residual, and
   each qnsch_step_poll that finds the latest norms arrived applies the
   stopping rules and queues the next outer cycle or the commit (the
   host-driven loop of qnsch_step, one cycle per poll at most).  Until
   qnsch_step_poll has reported the step done, the handle refuses other
   stepping calls with QNSCH_ESTATE.  qnsch_step_poll does not wait for the
   GPU: *done = 0 while the step runs; once it has ended, *done = 1 and
   n_vcycles, final_residual,
   status (what qnsch_step would have returned: 0, QNSCH_ENOTCONV, QNSCH_ENAN,
   QNSCH_ETIMEOUT, ...) and device_ms (the step's device time between CUDA
   events recorded around it on the handle's stream) receive the outcome;
   any of those four may be NULL.  qnsch_step_poll without a launched step
   gives QNSCH_ESTATE.  The result equals qnsch_step's on the same state. */
int qnsch_step_launch(qnsch_t* h, double dt);
int qnsch_step_poll(qnsch_t* h, int* done, int* n_vcycles, double* final_residual, int* status,
                    double* device_ms);

/* Batches of independent instances (no counterpart in the paper; the way a
   GPU runs many small problems at once).  A batch refers to n existing
   handles, each with its own stream (handles created without qnsch_set_stream
   each have a private one; two handles sharing a stream are rejected).
   qnsch_batch_step advances every instance by one step of size dt[a] with the
   host-driven loop: it polls the instances in turn and queues each one's next
   outer cycle as soon as that instance's norms have arrived, so the
   instances' kernels run concurrently on the GPU and none waits for another,
   and stops each instance at its own tolerance.  Every instance goes through exactly the arithmetic of
   qnsch_step on that handle, so its result does not depend on the batch.
   status[a] receives that instance's qnsch_step status (0, QNSCH_ENOTCONV,
   QNSCH_ENAN, ...), n_vcycles[a] (may be NULL) its V-cycle count.  The call
   returns QNSCH_OK unless its arguments are invalid: a dt that is not > 0 and
   finite, a member with a pending step, or two members that have come to
   share a stream (qnsch_set_stream after qnsch_batch_create) give
   QNSCH_EINVAL before any work is queued.  The batch does not own
   the handles; destroy it before them. */
typedef struct qnsch_batch_s qnsch_batch_t;
int qnsch_batch_create(int n, qnsch_t* const* insts, qnsch_batch_t** out);
int qnsch_batch_step(qnsch_batch_t* b, const double* dt, int* status, int* n_vcycles);
int qnsch_batch_size(const qnsch_batch_t* b);
/* Batch options: "max_inflight" (integer >= 0; 0, the default: all): at most
   this many members step at once; the others start, in member order, as
   running members finish their steps, so fewer instances share the L2 and
   the SMs at a time.  Results do not change.  Unknown keys and values out of
   range give QNSCH_EINVAL. */
int qnsch_batch_set_option(qnsch_batch_t* b, const char* key, double value);
/* Each member's last qnsch_batch_step on the GPU: ms[a] receives the device
   time from a CUDA event recorded on member a's stream before its step began
   to one recorded after it ended (the member's span inside the batch,
   including the time it shared the GPU with the others); -1 for a member
   not timed.  ms holds qnsch_batch_size(b) doubles. */
int qnsch_batch_step_times(const qnsch_batch_t* b, double* ms);
int qnsch_batch_destroy(qnsch_batch_t* b);

/* Mass reduction that allocates nothing (the paper has no counterpart: this is
   an interface for callers, not a step of the method).  It is meant for code
   that cannot allocate device memory when it needs the result: code running
   inside an allocator or memory-pool callback, where an allocation would
   re-enter the allocator; programs whose device memory is fully reserved up
   front by another framework; and loops that must not call cudaMalloc because
   it can synchronise the device.  It creates no handle and calls no
   cudaMalloc, cudaFree or allocating library routine.

   c: device pointer to the m2 x m1 cell array (layout above); h: cell size;
   rho1, rho2: the densities of qnsch_create; out2: device pointer to two
   doubles that receive h^2 sum rho(c) and h^2 sum rho(c) c (Thm. 6.1
   quantities, as qnsch_mass returns for a handle's state).  Work is queued on
   `stream` (NULL: legacy default stream) and the call returns without waiting:
   synchronise the stream before reading out2.

   Limit: m1 * m2 <= QNSCH_NOALLOC_MAX_CELLS, else QNSCH_EINVAL.  Its scratch is
   one file-scope device array of 64 KiB (QNSCH_NOALLOC_MAX_CELLS / 2048 pairs
   of doubles).  It is placed on a device when the library's device code is
   first loaded there (with lazy module loading, at this call's first use on
   that device) and stays until the process exits.  All calls share that
   array, so calls whose work overlaps on the GPU (other streams, other host
   threads) race and must be serialised by the caller; each call writes every
   entry it reads, so no clearing is needed.  The first call on a device looks
   up the array's device address (cudaGetSymbolAddress) with that device
   current and keeps it for the life of the process: make that first call
   before starting any stream capture, and do not call this entry point again
   after a reset of that device (cudaDeviceReset) in the same process. */
#define QNSCH_NOALLOC_MAX_CELLS 8388608
int qnsch_mass_noalloc(const double* c, int m1, int m2, double h, double rho1, double rho2,
                       double* out2, void* stream);

#ifdef __cplusplus
}
#endif
#endif
