// Host-side launchers of the sm_103a kernels (one translation unit per phase).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace sedi {

// Launch variants of the substep kernel: threads per block and minimum resident
// blocks per SM (128/6, 64/12, 256/3 cap registers at 80 a thread, 128/8 at 64,
// 128/5 at 96), all with the warp-cooperative pair phase; variants 5-7 run the
// per-particle pair loop at 128/6, 128/8 and 64/12; variant 8 evaluates each listed
// pair once from a pair list (one thread per pair) and gathers the pair records per
// particle in slot order (two launches); variant 9 is variant 8 with the pairs taken
// in list order from a work counter (one wave of blocks claiming 128 consecutive
// pairs at a time) instead of a grid-stride sweep.  The FP64 parity form runs 128/6
// with the loop.
enum SubstepVariant {
  SUBSTEP_B128 = 0,
  SUBSTEP_B64 = 1,
  SUBSTEP_B256 = 2,
  SUBSTEP_B128_OCC8 = 3,
  SUBSTEP_B128_OCC5 = 4,
  SUBSTEP_B128_LOOP = 5,
  SUBSTEP_B128_OCC8_LOOP = 6,
  SUBSTEP_B64_LOOP = 7,
  SUBSTEP_PAIRS = 8,
  SUBSTEP_PAIRS_ORDERED = 9
};
constexpr int kSubstepVariants = 10;
inline bool pair_variant(int variant) {
  return variant == SUBSTEP_PAIRS || variant == SUBSTEP_PAIRS_ORDERED;
}
// launch shapes of the batched ensemble substep (every bed with the per-particle pair
// phase; the pair list is a single-bed mode)
constexpr int kEnsVariants = 4;
constexpr int kEnsVariant[kEnsVariants] = {SUBSTEP_B128_LOOP, SUBSTEP_B64_LOOP, SUBSTEP_B128_OCC8_LOOP,
                                           SUBSTEP_B128};
inline int substep_block(int variant) {
  return (variant == SUBSTEP_B64 || variant == SUBSTEP_B64_LOOP) ? 64 : variant == SUBSTEP_B256 ? 256 : 128;
}

// k_force.cu: one fused substep (integrate = true) or forces only into st.fdbg.
// The last block of an integrating launch sets ctl->need_rebuild and, when
// use_cond, the graph condition next_cond of the following rebuild node.
void launch_substep(int form, const DevState& st, const DevMesh& mesh, const DevParams& P,
                    int sub_off, bool integrate, int variant, unsigned long long next_cond,
                    int use_cond, cudaStream_t s);

// k_bin.cu: rebuild = bin, sort by (bin, caller index), gather into the other
// buffers, build lists, carry springs over.  `conditional` kernels return at once
// unless ctl->need_rebuild is set.  sub_off: substep offset of the state buffer.
void launch_rebuild(int form, const DevState& st, const DevParams& P, int sub_off, bool force,
                    cudaStream_t s);
// A rebuild now (not forced by new particles): lists from the current positions, the
// springs carried over, as at a rebuild due to motion.
void launch_rebuild_now(int form, const DevState& st, const DevParams& P, cudaStream_t s);
// Set ctl->need_rebuild from the displacement; optionally a graph conditional.
void launch_check(const DevState& st, const DevParams& P, unsigned long long cond_handle,
                  int use_cond, cudaStream_t s);
// ctl->st = (ctl->st + n) & 1 after n substeps.
void launch_advance_parity(const DevState& st, int n, cudaStream_t s);

// Ensembles: one launch per phase over every bed (grid.y = bed).
struct EnsLaunch {
  const BedView* views;  // [B] device table
  int32_t B;
  int32_t variant;       // substep launch shape (one of kEnsVariants; the autotuner's)
  int64_t max_n;         // largest bed (particles)
  int64_t max_bins;      // largest bin grid
  int64_t max_cells;     // largest mesh
  Ctl* ectl;             // ensemble control: completion counter, rebuild flag
};
void launch_check_ens(const EnsLaunch& e, unsigned long long cond_handle, int use_cond,
                      cudaStream_t s);
void launch_rebuild_ens(int form, const EnsLaunch& e, int sub_off, cudaStream_t s);
void launch_advance_ens(const EnsLaunch& e, int n, cudaStream_t s);
// every bed rebuilds at the next launch_rebuild_ens (autotuner)
void launch_force_need_ens(const EnsLaunch& e, cudaStream_t s);
// every bed's rebuild counter from rebuilds[B] (device)
void launch_set_rebuilds_ens(const EnsLaunch& e, const int64_t* rebuilds, cudaStream_t s);
void launch_ctl_gather_ens(const EnsLaunch& e, Ctl* out, cudaStream_t s);
// Substeps s0 .. n-1 of every bed in one persistent cooperative launch (no optional
// terms), stopping after the first substep that leaves a bed needing a list rebuild;
// *done (device) receives the substeps completed, or -1 when a grid-barrier wait ran
// out (SEDI_ETIMEOUT in e.ectl->error).  Nonzero when the launch was refused.
int launch_substeps_persist_ens(int form, const EnsLaunch& e, int s0, int n, long long spin_limit, int* done,
                                cudaStream_t s);
// ext: the beds run the optional terms (lift, tangential lubrication)
void launch_substep_ens(int form, const EnsLaunch& e, bool ext, int sub_off,
                        unsigned long long next_cond, int use_cond, cudaStream_t s);
// deposition of every bed (cleared first), fixed point -> smoothing word
void launch_deposit_ens(int form, const EnsLaunch& e, cudaStream_t s);
// smoothed eps of every bed -> the drag's mesh word
void launch_eps_out_ens(int form, const EnsLaunch& e, cudaStream_t s);

// Scatter/gather between the sorted device state and caller order.
void launch_export(int form, const DevState& st, int what, double* out, cudaStream_t s);
void launch_import(int form, const DevState& st, const double* x, const double* v,
                   const double* w, const double* d, const double* rho, const DevParams& P,
                   cudaStream_t s);
void launch_neighbors_export(const DevState& st, int64_t* counts, cudaStream_t s);
void launch_neighbors_fill(const DevState& st, const int64_t* offsets, int64_t* out,
                           cudaStream_t s);
// Imports by caller index: pair springs (m sorted pairs i < j, xi as seen from i) set
// as the current history; lagged accelerations (n x 3); wall springs [n][6][3]
// exported into out (in == null) or imported from in (out == null).
void launch_springs_in(int form, const DevState& st, int64_t m, const int64_t* ij, const double* xi,
                       cudaStream_t s);
void launch_accel_in(int form, const DevState& st, const double* a, cudaStream_t s);
void launch_wall_springs(int form, const DevState& st, double* out, const double* in, cudaStream_t s);
void launch_contacts_export(int form, const DevState& st, const DevParams& P,
                            unsigned long long* count, int64_t cap, int64_t* ij, double* xi,
                            cudaStream_t s);

// k_bin.cu: pair list of the current neighbour lists (after a checkpoint load), and
// the partner copies of the pair-mode springs (before the slots are read elsewhere).
void launch_pair_list(const DevState& st, const DevParams& P, cudaStream_t s);
void launch_spring_sync(int form, const DevState& st, cudaStream_t s);

// k_avg.cu: deposition, field conversion, outputs.
void launch_deposit(int form, const DevState& st, const DevMesh& mesh, const DevParams& P,
                    void* qfields, cudaStream_t s);
void launch_fields_from_fixed(int form, const void* q, const DevParams& P, void* phi,
                              int nf, cudaStream_t s);
// mesh words ufe (U; eps_s kept) and gfl (G) from the FP64 fields [C][3] on the device
void launch_fluid_prep(int form, const double* U, const double* gp, const double* du, int gp_default,
                       double c_add_rho_f, const double rho_g[3], const DevParams& P,
                       const DevMesh& mesh, cudaStream_t s);
// eps_s of the mesh from (to_mesh = 1) or to (0) FP64 cell values
void launch_eps_io(int form, double* eps, const DevMesh& mesh, int64_t C, int to_mesh, cudaStream_t s);
// cell vorticity (curl U, 0) of the FP64 velocity U [C][3] into the mesh's wfl
void launch_curl(int form, const double* U, const DevParams& P, const DevMesh& mesh,
                 cudaStream_t s);
// k_smooth.cu: the smoothing solve of a batch of meshes in one persistent launch.
constexpr int kMaxBeds = 1024;       // meshes in one smoothing launch
constexpr int kMaxStepsRound = 64;  // Chebyshev steps of one round at most (more: next round)

// Pseudo-time schemes of the smoothing (Sec. 2.4): backward Euler, or BDF2 whose
// first step is backward Euler.
enum { TAU_EULER = 0, TAU_BDF2 = 1 };

// Graded z mesh of a smoothing (all null / 0 on a uniform mesh): the z-face
// coefficients of every plane, [nz][2] (towards k - 1, towards k + 1), for the
// backward-Euler (0) and BDF2 (1) operators in FP64 and FP32; the plane weights
// h_k / mean h, their sum over the cells, and per operator the largest sum of a
// plane's two coefficients (for the Gershgorin bound of the spectrum).
struct SmoothZ {
  const double* cz[2];
  const float* czf[2];
  const double* w;
  double wsum;
  double zmax[2];
};

// One mesh of a smoothing batch, as the caller describes it.
struct SmoothMesh {
  void* phi;          // [nf][C] fields in the smoothing word of the form, in place
  const void* guess;  // [nf][C] initial guess of the first pseudo-step, or null
  void* work;         // smooth_mesh_bytes(form, C, nf, scheme) bytes of device scratch
  int* iters;         // [nf] device counters, incremented by the steps taken (or null)
  int64_t C;
  int32_t nc[3], per[3];
  int32_t nf;
  double coef[3];     // dtau * D_a / h_a^2 (z: unused on a graded mesh)
  SmoothZ z;
};

// The operator of one kind of pseudo-step, A = I - sum_a coef_a L_a, and the
// Chebyshev constants of its spectrum.
struct SmoothSpec {
  double coef[3];
  double theta, delta, sigma1, sig;  // spectrum [1, lmax]: centre, half width, ratio, rate
  double cheb[2][kMaxStepsRound];    // c1, c2 of Chebyshev steps 1..kMaxStepsRound of a round
  float chebf[2][kMaxStepsRound];    // the same rounded to FP32 (narrow recursion)
  float inv_theta_f;                 // 1 / theta in FP32
  float coef_hi[3], coef_lo[3];      // coef as an FP32 pair: hi = fl32(c), lo = fl32(c - hi)
};

// The same, as the kernel sees it (device table, built by launch_smooth_batch; the
// grid solver copies an entry to shared memory as 16-byte words).
struct alignas(16) SmoothMeshDev {
  void* x;
  const void* guess;
  void* b;           // [nf][C] right-hand side (wide word)
  void* xp;          // [nf][C] previous pseudo-step (wide word; BDF2 only, else null)
  void* q;           // [C][8] recursive residual (narrow word, fields interleaved)
  void* d[2];        // [C][8] directions; d[0] also holds the narrow true residual
  double* part;       // [units][8][3] per-unit sums
  int* iters;
  int64_t C, u0, nu;  // cells, first unit, units
  int32_t nc[3], per[3];
  uint64_t div_x, div_xy;            // ceil(2^64 / nx), ceil(2^64 / (nx ny)) (0: divisor 1)
  int32_t cl_size, cl_planes;        // cluster solver: CTAs, z-planes per CTA (0: grid solver)
  SmoothSpec sp[2];  // [0]: backward-Euler steps (coef); [1]: BDF2 steps (2/3 coef)
  SmoothZ z;         // graded z mesh (null: uniform)
};

struct SmoothBatchDev {
  const SmoothMeshDev* mesh;  // [B]
  const int32_t* unit_bed;    // [U] mesh of each unit
  void* pairs;                // [B] per-mesh solver state
  int32_t* gflag;             // [2] largest step count of a round (alternating slots)
  int64_t U;
  int32_t B, nf;
  double rtol2;
  int32_t max_iter, n_tau, scheme;
  Ctl* ctl;                   // grid barrier and cg_status
  long long spin_limit;       // polls of a grid-barrier wait before SEDI_ETIMEOUT
};

// Polls of one grid-barrier wait before the smoother gives up with SEDI_ETIMEOUT
// (~0.3 s).  A handle may lower it (environment variable SEDI_BARRIER_SPIN_LIMIT,
// read at sedi_create) so that tests can make the wait run out.
constexpr long long kBarrierSpins = 1ll << 22;

// Sizes shared by the smoothing solvers and the static scratch of sedi_smooth_static:
// cells per work unit of the grid solver, fields the solver keeps per cell, and the
// per-unit sums of each field (|r|^2, sum r, |b|^2, sum w r on a graded mesh).
constexpr int kSmoothUnitCells = 256;
constexpr int kSmoothMaxFields = 8;
constexpr int kSmoothSums = 4;

int64_t smooth_units(int64_t C);
// scratch of one mesh, and of the batch tables
size_t smooth_mesh_bytes(int form, int64_t C, int nf, int scheme);
size_t smooth_batch_bytes(int64_t B, int64_t U);
// Smooth every mesh's nf fields in place by n_tau pseudo-steps of the scheme;
// batch_work: smooth_batch_bytes(B, sum of units) bytes.  Returns 0, -1 (bad sizes)
// or -3 (launch failed).
int launch_smooth_batch(int form, const SmoothMesh* meshes, int B, int nf, void* batch_work,
                        double rtol, int max_iter, int n_tau, int scheme, Ctl* ctl,
                        int max_blocks, cudaStream_t s, long long spin_limit = kBarrierSpins);
// Single mesh: work holds smooth_work_bytes(form, C, nf, scheme) = mesh + batch scratch.
size_t smooth_work_bytes(int form, int64_t C, int nf, int scheme);
int launch_smooth(int form, const DevParams& P, void* phi, const void* guess, int nf,
                  void* work, const DevState& st, int* iters_dev, double rtol, int max_iter,
                  int n_tau, int scheme, const double coef[3], const SmoothZ* z,
                  cudaStream_t s, long long spin_limit = kBarrierSpins);
void launch_average_out(int form, const void* phi, const DevParams& P, void* ufe, double* eps,
                        double* Us, double* F, cudaStream_t s);
void launch_phi_convert(int form, const void* phi, double* out, int64_t n, int to_double,
                        cudaStream_t s);
void launch_phi_from_double(int form, const double* in, void* phi, int64_t n, cudaStream_t s);

// k_cnn.cu: learned warm start (3x3x3 CNN 4 -> 32 -> 32 -> 4, bf16 storage).
size_t cnn_param_count();
size_t cnn_work_bytes(int64_t n);
// network input from four channel rows (FP64 device arrays) divided by scale
void cnn_input(const DevParams& P, const double* const f[4], const float scale[4], void* work,
               cudaStream_t s);
// forward with the bf16-rounded copy of the FP32 master weights; *y_out: [v][4] FP32
void cnn_forward(const DevParams& P, const float* master, void* work, float** y_out,
                 cudaStream_t s);
// loss = mean (y - target)^2 ([v][4] FP32 target) and its gradient (FP32, packed order)
void cnn_loss_grad(const DevParams& P, const float* master, const float* target, float* grad,
                   double* loss, void* work, cudaStream_t s);
void cnn_adam(float* master, const float* grad, float* m, float* v, int64_t t, float lr,
              cudaStream_t s);
void cnn_chan_first_to_vec(const double* in, float* out, int64_t n, int nc, cudaStream_t s);
void cnn_vec_to_chan_first(const float* in, double* out, int64_t n, int nc, cudaStream_t s);
// guess = phi (+ scale * y on eps and F), in the smoothing word of the form
void cnn_guess(int form, const void* phi, const float* y, const float scale[4], void* guess,
               int64_t C, cudaStream_t s);

}  // namespace sedi
