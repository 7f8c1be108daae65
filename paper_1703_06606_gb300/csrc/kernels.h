// kernels.h -- host-side launchers of the CUDA kernels in kernels.cu.
#pragma once
#include <cuda_runtime.h>

#include "qnsch_dev.cuh"

namespace qn {

// most levels one fused coarse-level V-cycle launch can hold
#define QN_MAX_FUSED_LEVELS 10

// Form: FullForm (the iterate is x) or ErrForm (the iterate is a correction e to
// a base X; the operator is N(X + e) - N(X))
template <typename T, class Form> void launch_residual(const Prm<T>& P, const Lv<T>& L, double* part, cudaStream_t s);
template <typename T, class Form> void launch_add_op(const Prm<T>& P, const Lv<T>& L, cudaStream_t s);
// team_max: FP64 full-iterate levels with at most this many cells per colour
// use four lanes per cell
template <typename T, class Form>
void launch_ch(const Prm<T>& P, const Lv<T>& L, int colour, cudaStream_t s, int team_max = 0);
// team_max: FP64 full-iterate levels with at most this many cells per colour
// use four lanes per Vanka block; team8_max: FP64 full-iterate levels with at
// most this many cells per colour use eight (half a momentum row per lane);
// pair_max: FP64 full-iterate levels above team_max with at most this many
// cells per colour use two (the x pair of rows on one lane, the y pair on the
// other); split (FP64 full-iterate single-lane launches): 0 never, 1 split a
// colour between one lane per block and lane pairs where a cost model of the
// busiest sub-partition says it is cheaper, >= 2 that many slots (rounded
// down to a multiple of 32) one lane each and the rest as pairs
template <typename T, class Form>
void launch_vanka(const Prm<T>& P, const Lv<T>& L, int colour, T omega, cudaStream_t s,
                  int team_max = 0, int team8_max = 0, int pair_max = 0, int split = 0);
// slots of an n-slot colour that the split launch runs one lane each (n: no split)
int vanka_split_single(int n, int split);
// a banded wavefront of smoothing passes on one level (kernels.cu, k_wave):
// npass passes (per smoothing step: CH red, CH black and the kcol Vanka
// colours, or the kcol coupled colours), bands of `rows` rows, the same team
// thresholds as the per-colour launches, waits bounded by `budget` SM cycles;
// stall: test hook, one wait that nothing satisfies
struct WavePlan {
  int npass, coupled, rows, nbands;
  int ch_team_max, vanka_team_max;
  long long budget;
  int stall;
};
// ctr: 1 + nbands unsigned counters (zeroed by the launcher); flag: set to
// nonzero when a wait runs out
template <typename T, class Form>
void launch_wave(const Prm<T>& P, const Lv<T>& L, const WavePlan& W, T omega, unsigned* ctr,
                 double* flag, cudaStream_t s);
// the skewed-chunk schedule of nsteps smoothing steps on one error-equation
// level (kernels.cu, k_skew): the steps' passes (per step: CH red, CH black
// and the kcol Vanka colours, or the kcol coupled colours) over chunks of
// `rows` rows, pass p behind pass p - 1 by one chunk and SKEW_LAG rows; one
// launch per diagonal, stream order the only dependency.  One lane per visit.
// Returns the number of launches it queued.
constexpr int SKEW_MAX_TASKS = 32;
constexpr int SKEW_LAG = 2;
struct SkewTasks {
  int n;                         // tasks (pass on a row range) of one launch
  int q[SKEW_MAX_TASKS];         // pass within its step: CH colour 0/1, then Vanka colours
  int t_lo[SKEW_MAX_TASKS];      // the task's slots t_lo .. t_hi - 1
  int t_hi[SKEW_MAX_TASKS];
  int boff[SKEW_MAX_TASKS + 1];  // first block of each task; boff[n] = blocks
};
template <typename T, class Form>
int launch_skew(const Prm<T>& P, const Lv<T>& L, int nsteps, int coupled, int rows, T omega,
                cudaStream_t s);
// the predicted initial iterate of a step: x[q] = w[0] a[q] + w[1] b[q] +
// w[2] c[q] elementwise, q over the five unknowns (c, mu, p, u, v), each array
// n padded elements starting `off` elements before its origin pointer
void launch_predict(double* const x[5], double* const a[5], double* const b[5],
                    double* const c[5], const double w[3], size_t n, int off, cudaStream_t s);
// the V-cycle on levels[0..n-1] (levels[0] is its finest) in one launch: one
// thread block (ctas = 1) or one thread-block cluster of ctas blocks, a size
// coarse_cluster_blocks returned (team8: the FP64 full-iterate Vanka blocks use
// eight lanes where a colour fits the group in one pass).  smem: an FP64
// full-iterate group in one block runs on a shared-memory copy of its levels
// where the copy fits (k_coarse_vcycle_smem, same results).  Returns 1 if it
// ran on the shared-memory copy, else 0.
template <typename T, class Form>
int launch_coarse_vcycle(const Prm<T>& P, const Lv<T>* levels, int n, int nu1, int nu2, int nuc,
                         int kcol, T omega, int coupled, cudaStream_t s, int team8 = 0,
                         int ctas = 1, int smem = 0);
// lets the shared-memory fused V-cycle use the device's opt-in shared memory
// per block (call with the device current, outside stream capture)
void coarse_smem_prepare();
// the largest power of two not above ctas (and not above 16) at which every
// form of the fused V-cycle launches as one cluster on the current device; 1
// when ctas < 2 or no cluster fits.  Queries the runtime: call it outside
// stream capture
int coarse_cluster_blocks(int ctas);
// one colour of the coupled 7x7 smoother (option "coupled")
template <typename T, class Form>
void launch_coupled(const Prm<T>& P, const Lv<T>& L, int colour, T omega, cudaStream_t s,
                    int team_max = 0);
// projection method (Sec. 7.2): 4x4 intermediate-velocity blocks of one Vanka
// colour; pressure Gauss-Seidel on one red-black colour; the projected velocity
// u^{n+1}, v^{n+1} into uo, vo (level layout, interior and boundary edges); the
// extra dissipation 1/2||sqrt(rho)(u^{n+1} - ut)||^2 into out1
template <typename T, class Form>
void launch_vanka4(const Prm<T>& P, const Lv<T>& L, int colour, T omega, cudaStream_t s,
                   int team_max = 0);
template <typename T>
void launch_pgs(const Prm<T>& P, const Lv<T>& L, int colour, cudaStream_t s, int team_max = 0);
template <typename T>
void launch_proj_velocity(const Prm<T>& P, const Lv<T>& L, T* uo, T* vo, cudaStream_t s);
template <typename T>
void launch_proj_diss(const Prm<T>& P, const Lv<T>& L, const T* uo, const T* vo, double* part,
                      double* out1, cudaStream_t s);
// defect correction: E (error-equation level) from the FP64 level D
template <typename T> void launch_cast_frozen(const Lv<double>& D, const Lv<T>& E, cudaStream_t s);
template <typename T> void launch_start_correction(const Lv<double>& D, const Lv<T>& E, cudaStream_t s);
template <typename T>
void launch_apply_correction(const Prm<double>& P, const Lv<double>& D, const Lv<T>& E, cudaStream_t s);
// rho(c) of the iterate over the whole padded arrays of an FP64 full-iterate level
void launch_rho_fill(const Prm<double>& P, const Lv<double>& L, cudaStream_t s);
template <typename T> void launch_restrict_base(const Lv<T>& F, const Lv<T>& C, cudaStream_t s);
template <typename T> void launch_bc_unknowns(const Lv<T>& L, cudaStream_t s);
template <typename T> void launch_frozen(const Prm<T>& P, const Lv<T>& L, cudaStream_t s);
template <typename T> void launch_restrict_state(const Prm<T>& P, const Lv<T>& F, const Lv<T>& C, cudaStream_t s);
template <typename T> void launch_restrict_res(const Lv<T>& F, const Lv<T>& C, cudaStream_t s);
template <typename T> void launch_restrict_frozen(const Lv<T>& F, const Lv<T>& C, cudaStream_t s);
template <typename T> void launch_prolong(const Prm<T>& P, const Lv<T>& F, const Lv<T>& C, cudaStream_t s);
template <typename T> void launch_gauge(const Lv<T>& L, double* part, double* scal, cudaStream_t s);
template <typename T> void launch_norms_finalize(const Lv<T>& L, double* part, double* out10, cudaStream_t s);
// Sec. 8 diagnostics of (c, u, v) on level L: out11[0..6] from the cells
// (max|div|, max div+, max div-, sum c, sum c a_y v, sum c y, sum div^2),
// out11[7..10] from the columns (max y_top, max Ly - y_bot, sum eta cos, count)
void launch_diag(const Lv<double>& L, const double* c, const double* u, const double* v,
                 double* part, double* out11, cudaStream_t s);
void launch_div_field(const Lv<double>& L, const double* u, const double* v, double* out,
                      cudaStream_t s);
template <typename T>
void launch_mass(const Prm<T>& P, const Lv<T>& L, const T* c, double* part, double* out2, cudaStream_t s);
template <typename T>
void launch_energy(const Prm<T>& P, const Lv<T>& L, const T* c, const T* u, const T* v, double w_grad,
                   double w_bulk, double w_pot, double* part, double* out1, cudaStream_t s);
template <typename T>
void launch_dissipation(const Prm<T>& P, const Lv<T>& L, double w_visc, double w_div, double w_ch,
                        double* part, double* out1, cudaStream_t s);
template <typename T> void launch_pack_in(const Lv<T>& L, T* dst, const double* src, int kind, cudaStream_t s);
template <typename T> void launch_pack_out(const Lv<T>& L, double* dst, const T* src, int kind, cudaStream_t s);

// the outer-cycle loop of a step on the device: ctl is the loop's control
// block (layout in kernels.cu); launch_loop_clock records the step's start
// time, launch_loop_ctl (first = 1 after the initial residual, 0 after each
// cycle) updates the block from the norms nrm and sets the WHILE (hl) and
// commit IF (hc) conditions of the step graph
void launch_loop_clock(double* ctl, cudaStream_t s);
void launch_loop_ctl(const double* nrm, double* ctl, cudaGraphConditionalHandle hl,
                     cudaGraphConditionalHandle hc, double tol, int maxcyc, int diverge,
                     double limit_ns, int first, cudaStream_t s);

// kernels issued by this library since it was loaded
long long launches_issued();
// launch every kernel with programmatic dependent launch (1, the default) or
// in plain stream order (0); applies to all handles of the process
void set_pdl(int on);

// rows of block partials any reduction on an m1 x m2 level may write
int partial_rows_needed(int m1, int m2);

}  // namespace qn
