/*
 * sedi.h -- C ABI of the GB300 particle-side hot path of the SediFoam CFD-DEM
 * method (Sun & Xiao, arXiv 1601.03801).
 *
 * The fluid is frozen: the caller prescribes cell-centred fluid fields on a
 * uniform Cartesian mesh.  Each DEM substep (sedi_step) does link-cell binning and
 * neighbour lists (Sec. 2.5), Hertz-Mindlin contact with tangential history
 * (Sec. 2.1, Eq. 1; Sec. 2.5), Ball-Melrose lubrication (Sec. 2.5), drag,
 * pressure-gradient and added-mass forces (Sec. 2.3, Eq. 3-8) and a leapfrog
 * velocity-Verlet update (Sec. 2.1, Eq. 1).  sedi_average does the diffusion-based
 * averaging (Sec. 2.4, Eq. 9-10): PCM deposition, then implicit diffusion
 * smoothing, each implicit step solved to a relative residual by Chebyshev
 * semi-iteration on the operator's known spectrum, organised as iterative
 * refinement (the linear systems and the stopping test are those of plain
 * conjugate gradients; the iteration differs, see sedi_average).
 *
 * Conventions for every call:
 *   - Return 0 on success or a negative SEDI_E* code; sedi_last_error() then
 *     holds a message (per handle, valid until the next call on that handle).
 *   - Vectors cross the boundary as row-major n x 3 (or C x 3) float64.
 *   - `mem` says where caller pointers live: SEDI_MEM_HOST or SEDI_MEM_DEVICE
 *     (device memory of the current CUDA device).  The library copies inputs and
 *     never keeps a caller pointer; outputs go to caller-owned buffers.
 *   - Particles are returned in the caller's order of sedi_set_particles.
 *   - Mesh fields are cell-centred, x fastest: cell (i, j, k) is
 *     (k * ny + j) * nx + i; cell (i, j, k) spans lo + [i, i+1) * (hi - lo) / n.
 *   - Work is queued on the handle's stream (sedi_set_stream).  Calls that
 *     return data to the caller synchronise that stream; a device-side error
 *     (neighbour capacity, non-finite state, unconverged smoothing, a bounded
 *     device wait that ran out) raised by queued work is reported by the next
 *     call that synchronises.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef SEDI_H
#define SEDI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SEDI_OK = 0,
  SEDI_EINVAL = -1,    /* bad argument or parameter */
  SEDI_ENOMEM = -2,    /* device allocation failed */
  SEDI_ECUDA = -3,     /* a CUDA runtime call failed */
  SEDI_EOVERFLOW = -4, /* a particle has more listed neighbours than nbr_capacity */
  SEDI_ERANGE = -5,    /* a deposited value does not fit the fixed-point format */
  SEDI_EDIVERGED = -6, /* smoothing solver hit cg_max_iter steps before cg_rtol */
  SEDI_ENONFINITE = -7,/* a force or position became NaN/Inf */
  SEDI_ETIMEOUT = -8,  /* a bounded device-side wait gave up */
  SEDI_ESTATE = -9,    /* calls in the wrong order (e.g. step before particles) */
  SEDI_EIO = -10       /* checkpoint file could not be read or written */
};

enum { SEDI_MEM_HOST = 0, SEDI_MEM_DEVICE = 1 };

/* sedi_average's bed argument for "every bed of an ensemble, in place". */
#define SEDI_ALL_BEDS (-1)

/* Arithmetic of the hot path.
 * SEDI_FORM_SPLIT (default): forces in FP32; positions, velocities, spins and
 *   tangential springs carried in FP64-class double-float (two FP32 words,
 *   48-bit significand) so every update runs on the FP32 pipes; contact overlap
 *   and gap evaluated in double-float; fixed-point deposition; smoothing with a
 *   double-float true residual and an FP32 Chebyshev recursion.
 * SEDI_FORM_PLAIN_FP32: everything FP32 (absolute FP32 positions, FP32 smoothing with
 *   its tolerance raised to at least 2e-6, float atomics for deposition) -- the
 *   comparison baseline.
 * SEDI_FORM_FP64: everything IEEE FP64, for parity checks against an FP64
 *   reference (slow on GB300: FP64 runs at a small fraction of the FP32 rate). */
enum { SEDI_FORM_SPLIT = 0, SEDI_FORM_PLAIN_FP32 = 1, SEDI_FORM_FP64 = 2 };

/* Contact laws.  SEDI_HERTZ_MINDLIN: Hertz normal force and Mindlin tangential
 * spring with Tsuji-type damping (E, poisson, restitution).  SEDI_LINEAR_SPRING: the
 * paper's linear spring-dashpot (Sec. 2.5, Table 1): normal stiffness kn_linear,
 * tangential stiffness kt_ratio * kn_linear, damping set by the restitution
 * coefficient (exactly e for a head-on collision). */
enum { SEDI_HERTZ_MINDLIN = 0, SEDI_LINEAR_SPRING = 1 };

/* Pseudo-time schemes of the diffusion smoothing (Sec. 2.4), n_tau steps of
 * dtau = 1 / n_tau.  SEDI_TAU_EULER: (I - dtau D L) phi^{m+1} = phi^m.  SEDI_TAU_BDF2:
 * the second-order implicit scheme, read as the two-step backward difference
 * (I - (2/3) dtau D L) phi^{m+1} = (4/3) phi^m - (1/3) phi^{m-1}, its first step
 * backward Euler.  Both keep sum(phi). */
enum { SEDI_TAU_EULER = 0, SEDI_TAU_BDF2 = 1 };

typedef struct sedi_handle sedi_handle; /* opaque, owned by the library */

/* All SI units.  Defaults from sedi_default_params() in brackets. */
typedef struct sedi_params {
  int32_t contact_law;                     /* SEDI_HERTZ_MINDLIN | SEDI_LINEAR_SPRING [Hertz] */
  double E, poisson, restitution, friction;/* particles and walls [1e7, 0.3, 0.9, 0.3] */
  double kn_linear, kt_ratio;              /* linear law: normal stiffness (N/m), tangential
                                              / normal stiffness [800 (Table 1), 2/7] */
  double rho_f, nu_f, g[3];                /* fluid density, kinematic viscosity, gravity
                                              [1000, 1e-6, (0, 0, -9.81)] */
  double lo[3], hi[3];                     /* box; axis a spans [lo, hi) */
  int32_t periodic[3];                     /* 1: axis wraps */
  int32_t wall_lo[3], wall_hi[3];          /* 1: plane wall at lo / hi (non-periodic axes) */
  double dt;                               /* DEM substep [1e-6] */
  double skin;                             /* neighbour-list skin [5e-5] */
  int32_t lubrication, drag, pressure_grad, added_mass; /* force switches [1, 1, 1, 1] */
  int32_t lift;                            /* Saffman lift (Sec. 2.3, Eq. 7), read as
                                              c_lift rho_f nu^0.5 d^2 |omega|^-0.5
                                              (w x omega), w = U_f - u_p, omega = curl U_f
                                              (central differences of U at the cell
                                              centres, interpolated trilinearly) [0] */
  int32_t lub_tangential;                  /* tangential (shear) lubrication terms of the
                                              Ball-Melrose model, with their torques
                                              (Sec. 2.5): leading log-gap term of the
                                              two-sphere resistance; needs lubrication [0] */
  double lub_h_in_frac, lub_h_out_frac;    /* lubrication gap limits as fractions of the
                                              pair-mean diameter [1e-3, 0.1] */
  double c_add;                            /* added-mass coefficient, Eq. 8 [0.5] */
  double c_lift;                           /* lift coefficient C_l, Eq. 7 [1.6] */
  double eps_max;                          /* clamp of eps_s in the drag law [0.9] */
  int32_t ncell[3];                        /* Eulerian mesh */
  double z_grading;                        /* graded mesh along z (Sec. 4.2: refined
                                              towards the bottom): cell heights grow
                                              geometrically from lo[2], top cell / bottom
                                              cell = z_grading; 1 = uniform.  Needs a
                                              non-periodic z axis with ncell[2] >= 2 [1] */
  double bandwidth[3];                     /* Gaussian bandwidth b per axis (Sec. 2.4) */
  int32_t n_tau;                           /* implicit pseudo-time steps [4] */
  int32_t tau_scheme;                      /* SEDI_TAU_EULER | SEDI_TAU_BDF2 [EULER];
                                              BDF2 excludes use_cnn_guess */
  double cg_rtol;                          /* ||r|| <= rtol ||b|| per pseudo-step [1e-8]
                                              (the names keep the usual CG vocabulary:
                                              the stopping test is the same) */
  int32_t cg_max_iter;                     /* most solver steps per field and pseudo-step
                                              [500] */
  int32_t shift_eps, shift_mom, shift_force; /* fixed-point exponents [40, 40, 32] */
  int32_t precision_form;                  /* SEDI_FORM_* [SPLIT] */
  int32_t nbr_capacity;                    /* listed neighbours per particle, <= 32 [32] */
  int32_t use_graphs;                      /* capture substeps in CUDA graphs [1] */
  int32_t substep_variant;                 /* launch shape of the substep:
                                              -1 = autotuned [-1]: the per-particle loop
                                              (5) runs until 200 substeps after the
                                              particles were set, then every shape is
                                              timed on integrating substeps (state
                                              restored) and the fastest kept;
                                              0: 128 threads, 6 blocks/SM; 1: 64 x 12;
                                              2: 256 x 3; 3: 128 x 8; 4: 128 x 5, all with
                                              the warp-cooperative pair phase; 5: 128 x 6,
                                              6: 128 x 8, 7: 64 x 12 with a per-particle
                                              pair loop; 8: the pair list (each listed
                                              pair evaluated once by one thread, then a
                                              per-particle gather; two launches); 9: the
                                              pair list with its pairs taken in list
                                              order from a work counter (one wave of
                                              blocks, 128 consecutive pairs a claim).  With
                                              lift or lub_tangential on the loop at
                                              128 x 6 runs.  The split form gives
                                              bit-identical results across variants, the
                                              plain form agrees to FP32 rounding.  The
                                              FP64 parity form always runs the loop. */
  int32_t n_beds;                          /* independent beds in this handle, 1..1024
                                              (see "Ensembles" below) [1] */
  int32_t profile;                         /* record CUDA events around each phase
                                              (see sedi_get_timings) [0] */
  int32_t use_cnn_guess;                   /* start every smoothing pseudo-step from
                                              the learned guess (sedi_cnn_*) [0] */
  int32_t ens_persistent;                  /* ensembles: run the substeps of a sedi_step
                                              call for all beds in one persistent
                                              cooperative launch (grid barrier between
                                              substeps; a list rebuild ends the launch and
                                              the next one resumes after it) instead of a
                                              CUDA graph of one batched launch per substep
                                              [0].  Same results either way; not with lift
                                              or tangential lubrication. */
  int32_t bin_order;                       /* storage order of the link-cell bins: -1 =
                                              autotuned with the launch shape (x fastest
                                              until then, and whenever substep_variant is
                                              fixed) [-1]; 0 = x fastest, 1 = z fastest.
                                              Changes no result. */
  int32_t bins_per_cutoff;                 /* link-cell bins per list cutoff of the list
                                              build: 0 = autotuned with the launch shape
                                              (1 until then, and whenever substep_variant
                                              is fixed) [0]; 1 or 2 = fixed (2: bins of
                                              half a cutoff, a 5 x 5 x 5 stencil; needs 5
                                              bins on every periodic axis).  Lists hold
                                              their partners in caller-index order, so
                                              the choice changes no result. */
  double cnn_scale[4];                     /* network input/output scale of eps_s and
                                              F_fp x, y, z [1, 1, 1, 1] */
  uint64_t seed;                           /* reserved for stochastic extensions [0] */
} sedi_params;

/* Per-handle counters since creation. */
typedef struct sedi_stats {
  int64_t substeps;       /* substeps advanced */
  int64_t rebuilds;       /* neighbour-list rebuilds */
  int64_t averages;       /* sedi_average calls */
  int64_t cg_iterations;  /* smoothing solver steps (Chebyshev steps plus one true-
                             residual evaluation per refinement round) summed over
                             fields and pseudo-steps */
  int32_t max_neighbors;  /* largest list length at the last rebuild */
  int32_t nbr_capacity;   /* capacity in use */
  int32_t substep_variant; /* launch variant of the substep kernel in use (-1: not yet tuned) */
  int32_t substep_block;   /* its threads per block (0: not yet tuned) */
  int32_t bins_per_cutoff; /* link-cell bins per list cutoff of the list build (1 or 2;
                              picked with the launch variant) */
  int32_t bin_order;       /* storage order of the bins: 0 x fastest, 1 z fastest
                              (picked with the launch variant) */
} sedi_stats;

/* Fill p with the defaults listed above (box 20 x 20 x 40 mm, periodic x/y,
   walls at z lo/hi, mesh 10 x 10 x 20, bandwidth 3 mm). */
void sedi_default_params(sedi_params* p);

/* Create a handle on the current CUDA device.  Checks the parameters and
   allocates the mesh fields and smoothing work space; particle buffers are
   allocated by sedi_set_particles.  (Sec. 2.5 advises dt <= t_c / 50 of the
   Hertz contact time; the caller chooses dt.)  *out is owned by the caller and
   released with sedi_destroy.  Errors: EINVAL, ENOMEM, ECUDA.  The environment
   variable SEDI_BARRIER_SPIN_LIMIT, read here, lowers the number of polls after
   which a wait at the grid-wide barrier of the smoother (meshes too large for one
   thread-block cluster) gives up and the averaging returns SEDI_ETIMEOUT (default
   2^22, about 0.3 s); it exists so tests can make that wait run out. */
int sedi_create(const sedi_params* p, sedi_handle** out);
void sedi_destroy(sedi_handle* h);

/* Queue all later work on `cuda_stream` (a cudaStream_t).  A new handle uses a
   non-blocking stream of its own.  NULL selects the legacy default stream, on
   which substeps run without CUDA graphs (stream capture needs a real stream).
   The stream must outlive its use by the handle. */
int sedi_set_stream(sedi_handle* h, void* cuda_stream);

/* ---- Ensembles (params.n_beds > 1) ----
 * The paper runs one bed per simulation; an ensemble holds n_beds independent
 * beds of uneven size (Sec. 2's method applied to each) so that small beds fill
 * the GPU together.  Each bed has its own particles, box and mesh (default: the
 * box and mesh of the parameters; sedi_set_bed changes them) and its own fluid
 * fields; the material, fluid, time step, bandwidth and solver parameters are
 * shared.  Every call that takes `bed` addresses one bed.  sedi_step advances all
 * beds with one launch per phase over all beds (one CUDA graph per fluid step);
 * sedi_average(h, SEDI_ALL_BEDS, NULL, NULL, NULL, mem) averages every bed in
 * batched launches and leaves the results on the device for the drag;
 * sedi_average(h, bed, ...) returns one bed's averaged fields (averaging all beds
 * first if a step happened since).  Every bed must have particles before the
 * first step.  A bed's results are bit-identical to running it alone in a
 * single-bed handle.  Not for ensembles: params.use_cnn_guess (learned warm
 * start) and the substep autotuner (ensembles run substep variant 5: 128-thread
 * blocks with the per-particle pair loop). */

/* Box [lo, hi) and mesh ncell of ensemble bed `bed`; resets that bed (its
   particles must be set again).  Errors: EINVAL (not an ensemble, bed out of
   range, bad box or mesh), ENOMEM. */
int sedi_set_bed(sedi_handle* h, int32_t bed, const double lo[3], const double hi[3],
                 const int32_t ncell[3]);

/* Set n particles of bed `bed` (0 <= bed < n_beds): ids (may be NULL: 0..n-1),
   positions x, half-step velocities v (Sec. 2.1: leapfrog), angular velocities
   omega (NULL = 0), diameters d and densities rho.  Positions on periodic axes
   must lie in [lo, hi).  Resets tangential history and the lagged acceleration,
   sorts the particles into link cells and builds neighbour lists (synchronous).
   Errors: EINVAL (n <= 0, d or rho <= 0, a position outside a periodic range, a
   periodic axis shorter than three list cutoffs), ENOMEM, EOVERFLOW. */
int sedi_set_particles(sedi_handle* h, int32_t bed, int64_t n, const int64_t* id,
                       const double* x, const double* v, const double* omega,
                       const double* d, const double* rho, int32_t mem);

/* Prescribed fluid fields on the ncell mesh (must equal params.ncell), each C x 3:
   U (NULL = 0), grad_p (NULL = rho_f g, hydrostatic), DUDt = dU/dt + U.grad U
   (NULL = 0) (Sec. 2.3).  The solid fraction seen by the drag (from the last
   sedi_average or sedi_set_eps, 0 initially) is kept.  Synchronous. */
int sedi_set_fluid(sedi_handle* h, int32_t bed, const int32_t ncell[3], const double* U,
                   const double* grad_p, const double* DUDt, int32_t mem);

/* Overwrite the smoothed solid fraction (C) that the drag law interpolates
   (normally written by sedi_average). */
int sedi_set_eps(sedi_handle* h, int32_t bed, const double* eps, int32_t mem);

/* Advance every bed by n_substeps DEM substeps (Sec. 2.1 Eq. 1, Sec. 2.3, 2.5):
   rebuild lists when a particle moved more than skin/2, then forces and the
   leapfrog update.  Asynchronous: returns after queueing. */
int sedi_step(sedi_handle* h, int32_t n_substeps);

/* Diffusion-based averaging of bed `bed` (Sec. 2.4, Eq. 9-10): PCM deposition of
   eps_s, eps_s U_s and the force density -f_fp / V_c on the fluid, then n_tau
   implicit diffusion steps, each solved to ||b - A x|| <= cg_rtol ||b||.  The
   solver: A = I - dtau div(D grad) has its spectrum in [1, 1 + 4 sum_a dtau D_a /
   dx_a^2], so Chebyshev semi-iteration needs no inner products; each refinement
   round forms the true residual in double-float (FP64 in SEDI_FORM_FP64), stops
   when it meets the tolerance, else runs a fixed number of Chebyshev steps on the
   correction in FP32.  The conserved sum of each field is kept as CG keeps it.  Outputs
   (any may be NULL): eps_s (C), U_s (C x 3), F_fp (C x 3).  The smoothed eps_s
   becomes the one the drag law sees.  bed = SEDI_ALL_BEDS (ensembles): every
   bed, outputs NULL.  Errors: ERANGE, EDIVERGED. */
int sedi_average(sedi_handle* h, int32_t bed, double* eps_s, double* U_s, double* F_fp,
                 int32_t mem);

/* Raw PCM deposition (Sec. 2.4, Eq. 9) as 64-bit fixed point, [7][C]:
   eps_s * 2^shift_eps, eps_s U_s * 2^shift_mom (x, y, z), F_fp * 2^shift_force
   (x, y, z), each rounded to nearest per particle and summed exactly.
   (The plain FP32 form sums floats and rounds the sum.) */
int sedi_deposit(sedi_handle* h, int32_t bed, int64_t* fixed_fields, int32_t mem);

/* Smooth n_fields caller fields [n_fields][C] with the averaging operator
   (Sec. 2.4, Eq. 10); guess (same shape or NULL) is projected onto the conserved
   sum and used as the first pseudo-step's initial iterate; iters (n_fields or
   NULL) receives the solver steps per field summed over pseudo-steps. */
int sedi_smooth(sedi_handle* h, int32_t bed, int32_t n_fields, const double* in, double* out,
                const double* guess, int32_t* iters, int32_t mem);

/* Current particle state in the caller's order: x (n x 3), v (half step),
   omega, a_prev (acceleration of the last substep); any may be NULL. */
int sedi_get_particles(sedi_handle* h, int32_t bed, double* x, double* v, double* omega,
                       double* a_prev, int32_t mem);

/* Forces and torque at the current state without advancing or touching the
   history (Sec. 2.1 Eq. 1 right-hand sides): contact (pairs + walls),
   lubrication, fluid (drag + pressure gradient + added mass), contact torque. */
int sedi_compute_forces(sedi_handle* h, int32_t bed, double* f_contact, double* f_lub,
                        double* f_fluid, double* torque, int32_t mem);

/* Current neighbour lists in the caller's numbering: offsets (n + 1) and sorted
   ids of each particle's listed partners.  Returns the number of entries, or
   SEDI_EOVERFLOW if cap is too small (offsets is still filled). */
int64_t sedi_get_neighbors(sedi_handle* h, int32_t bed, int64_t* offsets, int64_t* ids,
                           int64_t cap);

/* Tangential springs of the pairs in contact: ij (m x 2, caller indices, i < j)
   and xi (m x 3) as seen from i.  Returns m, or SEDI_EOVERFLOW if m > cap. */
int64_t sedi_get_contacts(sedi_handle* h, int32_t bed, int64_t cap, int64_t* ij, double* xi);

/* ---- State import (domain decomposition and restarts) ----
 * A bed split over several handles (one per GPU, e.g. x-slabs of the box with
 * ghost spheres copied from the neighbours) moves spheres between handles and
 * rebuilds a handle's particle set; these calls carry the state that
 * sedi_set_particles resets.  All take caller indices of the current particle set
 * (after sedi_set_particles) and synchronise the handle's stream. */

/* Tangential springs (Sec. 2.5, endured contacts) of m pairs: ij (m x 2, caller
   indices, i < j, each pair once) and xi (m x 3) as seen from i, as sedi_get_contacts
   returns them.  The given pairs that are in the current neighbour lists take these
   springs; every other listed pair has none.  Errors: EINVAL (index out of range,
   i >= j, a pair given twice). */
int sedi_set_contacts(sedi_handle* h, int32_t bed, int64_t m, const int64_t* ij, const double* xi,
                      int32_t mem);
/* Lagged accelerations a_prev (n x 3) used by the added-mass force (Sec. 2.3, Eq. 8),
   as sedi_get_particles returns them. */
int sedi_set_accel(sedi_handle* h, int32_t bed, const double* a_prev, int32_t mem);
/* Wall springs, [n][6][3]: walls lo x, hi x, lo y, hi y, lo z, hi z; a zero vector
   means no contact history with that wall. */
int sedi_get_wall_springs(sedi_handle* h, int32_t bed, double* xi_wall, int32_t mem);
int sedi_set_wall_springs(sedi_handle* h, int32_t bed, const double* xi_wall, int32_t mem);
/* The averaging of sedi_average (Sec. 2.4, Eq. 9-10) from a given PCM deposition q
   ([7][C] fixed point in the format of sedi_deposit, e.g. the sum of the depositions
   of several handles that share this mesh): smoothing, outputs, and the smoothed
   eps_s becomes the one the drag law sees.  Not in the plain FP32 form (EINVAL). */
int sedi_average_deposit(sedi_handle* h, int32_t bed, const int64_t* q, double* eps_s,
                         double* U_s, double* F_fp, int32_t mem);

/* ---- Learned warm start of the smoothing solve ----
 * A 3-layer 3x3x3 convolutional network 4 -> 32 -> 32 -> 4 (ReLU after the first
 * two; bfloat16 weights and activations, FP32 accumulation) maps one smoothing
 * pseudo-step's right-hand side phi^m of (eps_s, F_fp x, y, z), divided by
 * cnn_scale, to the predicted change (phi^{m+1} - phi^m) / cnn_scale.  With
 * params.use_cnn_guess = 1, sedi_average starts every pseudo-step's solve from
 * phi^m + cnn_scale * net(phi^m / cnn_scale), shifted to the conserved sum; the
 * solve still runs to cg_rtol, so only the iteration count changes.  The paper
 * has no learned component (Sec. 2.4 solves the diffusion equation directly).
 * Parameters are packed w1[32][4][27] b1[32] w2[32][32][27] b2[32] w3[4][32][27]
 * b3[4], tap t = (kz*3 + ky)*3 + kx at offset (kx-1, ky-1, kz-1); fields are
 * channels-first [4][C] float64; taps outside the mesh wrap on periodic axes and
 * read zero elsewhere.  Training runs on the GPU: forward, backward and Adam
 * (lr given, beta 0.9/0.999, eps 1e-8) on FP32 master weights. */
#define SEDI_CNN_PARAMS 34628
int sedi_cnn_set_params(sedi_handle* h, const double* params, int64_t n);  /* host array; resets Adam */
int sedi_cnn_get_params(sedi_handle* h, double* params, int64_t n);        /* host array */
/* y = net(x), x and y [4][C] */
int sedi_cnn_forward(sedi_handle* h, const double* x, double* y, int32_t mem);
/* loss = mean over [4][C] of (net(x) - target)^2 and d loss / d params (n doubles, host) */
int sedi_cnn_loss_grad(sedi_handle* h, const double* x, const double* target, double* grad,
                       double* loss, int32_t mem);
/* `steps` Adam steps cycling over n_pairs (x, target) pairs, each [4][C]; losses
   (steps doubles, host, or NULL) receives the loss before each step. */
int sedi_cnn_train(sedi_handle* h, int32_t n_pairs, const double* x, const double* target,
                   int32_t steps, double lr, double* losses, int32_t mem);

/* Checkpoint and restore of particles, lagged accelerations, tangential springs,
   fluid fields and the drag's solid fraction (binary, this library's format; an
   ensemble writes every bed, and restores into a handle with as many beds of the
   same meshes). */
int sedi_save_state(sedi_handle* h, const char* path);
int sedi_load_state(sedi_handle* h, const char* path);

/* Device time per phase since creation, from CUDA events recorded on the
   handle's stream (inside the CUDA graphs too) when params.profile = 1:
   ms[0] rebuild check + conditional rebuild, ms[1] fused force/update kernel,
   ms[2] deposition, ms[3] smoothing; ms[4..7] the number of timed launches of
   each phase.  Synchronises the stream.  Returns the number of values written
   (<= n), 0 when profiling is off. */
int sedi_get_timings(sedi_handle* h, double* ms_per_phase, int32_t n);
int sedi_get_stats(sedi_handle* h, sedi_stats* out);

/* ---- Smoothing without any device allocation ----
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc themselves or through this library -- e.g. code that
 * runs while a memory pool or a host framework owns all device memory, or a
 * plugin whose device allocations are forbidden after start-up.  It smooths
 * n_fields caller fields exactly like sedi_smooth (same operator, solver and
 * stopping test; the mesh, bandwidth, n_tau, tau_scheme, cg_rtol, cg_max_iter and
 * precision_form of *p), but keeps all scratch in one static device array of this
 * library, so it allocates nothing: no cudaMalloc/cudaFree, no allocating library
 * routine.
 *   p       : parameters (only the mesh, box, bandwidth, solver and form fields
 *             are read); no handle is needed.  A graded z mesh is rejected.
 *   in, out : DEVICE pointers (checked with cudaPointerGetAttributes; host memory
 *             is rejected), [n_fields][C] float64, C = prod(ncell); caller-owned.
 *   iters   : host array of n_fields (or NULL) receiving the solver steps.
 *   cuda_stream : stream to run on (NULL = legacy default stream).
 *   msg     : optional host buffer of msg_len bytes for an error message.
 * Limit: 8 * C <= SEDI_STATIC_MAX_WORDS, i.e. up to 131,072 cells with any
 * n_fields <= 8 (the solver keeps 8 words per cell); larger meshes return
 * SEDI_EINVAL.  The scratch (about 50 MB) lives on every GPU that loads the
 * library until the process exits.  Every call looks up the scratch's device
 * address on the current device (cudaGetSymbolAddress, which allocates nothing).
 * The call copies its status to the host and synchronises its stream, so it must
 * not be issued while the stream is being captured into a graph.  Every call
 * shares the one array and leaves its contents behind: calls whose GPU work
 * overlaps (two streams, two threads) race and must be serialised by the caller.
 * Each call ends by synchronising its stream and returns SEDI_OK, SEDI_EINVAL,
 * SEDI_EDIVERGED, SEDI_ETIMEOUT or SEDI_ECUDA. */
#define SEDI_STATIC_MAX_WORDS (1 << 20)
int sedi_smooth_static(const sedi_params* p, int32_t n_fields, const double* in, double* out,
                       int32_t* iters, void* cuda_stream, char* msg, int32_t msg_len);

/* Block until all queued work of the handle is done; returns its status. */
int sedi_sync(sedi_handle* h);

const char* sedi_last_error(const sedi_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* SEDI_H */
