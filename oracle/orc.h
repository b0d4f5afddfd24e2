/*
 * FP64 CPU oracle for the particle-side hot path of the SediFoam CFD-DEM method
 * (Sun & Xiao, "SediFoam: a general-purpose, open-source CFD-DEM solver for
 * particle-laden flow with emphasis on sediment transport", arXiv 1601.03801).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the plain, slow, obviously correct
 * restatement of the method that the CUDA library is checked against.  Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no header, helper, table or constant with the CUDA library.
 *
 * Everything here is IEEE binary64, evaluated in source order; the build passes
 * -ffp-contract=off so no multiply-add is fused.
 *
 * Sections of the paper followed:
 *   Sec. 2.1, Eq. (1a)-(1b)  Newton's equations for translation and rotation
 *   Sec. 2.3, Eq. (3)-(6)    drag (Syamlal-O'Brien correlation)
 *   Sec. 2.3, Eq. (8)        added mass (explicit, lagged particle acceleration)
 *   Sec. 2.4, Eq. (9)-(10)   PCM deposition and diffusion smoothing
 *   Sec. 2.5                 link-cell neighbour search, soft-sphere contact,
 *                            Ball-Melrose lubrication, rotation from torques
 * The readings of garbled or silent passages are listed beside each routine.
 */
#pragma once
#include <cstdint>

extern "C" {

/* Parameters of one oracle instance (all SI units). */
typedef struct {
  /* contact material (particles and walls share it) */
  double E, poisson, restitution, friction;
  /* fluid */
  double rho_f, nu_f, g[3];
  /* box: axis a spans [lo[a], hi[a]); periodic axes wrap, others may carry walls */
  double lo[3], hi[3];
  int32_t periodic[3], wall_lo[3], wall_hi[3];
  /* time step of one DEM substep */
  double dt;
  /* force switches */
  int32_t lubrication, drag, pressure_grad, added_mass;
  double lub_h_in_frac, lub_h_out_frac; /* fractions of the pair-mean diameter */
  double c_add;                         /* added-mass coefficient, 0.5 in Sec. 2.3 */
  double eps_max;                       /* clamp of the solid fraction seen by drag */
  /* Eulerian mesh (uniform, cell-centred, x fastest) covering the box */
  int32_t ncell[3];
  /* averaging: Gaussian bandwidth per axis, pseudo-time steps, CG control */
  double bandwidth[3];
  int32_t n_tau;
  double cg_rtol;
  int32_t cg_max_iter;
  /* fixed-point exponents of the deposited fields: solid fraction,
     momentum (eps*U) and force density */
  int32_t shift_eps, shift_mom, shift_force;
  /* contact law: 0 Hertz-Mindlin, 1 linear spring-dashpot (Sec. 2.5, Table 1) with
     normal stiffness kn_linear (N/m) and tangential stiffness kt_ratio * kn_linear */
  int32_t contact_law;
  double kn_linear, kt_ratio;
  /* pseudo-time scheme of the smoothing: 0 backward Euler, 1 second-order BDF
     (its first step backward Euler) */
  int32_t tau_scheme;
  /* Saffman lift (Sec. 2.3, Eq. 7) with coefficient c_lift (1.6), and the
     tangential (shear) lubrication terms of the Ball-Melrose model (Sec. 2.5) */
  int32_t lift;
  double c_lift;
  int32_t lub_tangential;
  /* graded mesh along z (Sec. 4.2: refined towards the bottom): ratio of the top
     cell's height to the bottom cell's; 1 = uniform */
  double z_grading;
} orc_params;

typedef struct orc_handle orc_handle;

orc_handle* orc_create(const orc_params* p);
void orc_destroy(orc_handle* h);

/* Particles: n, row-major n*3 arrays.  d = diameter, rho = density.
   v is the velocity at the half step behind the positions (leapfrog). */
int orc_set_particles(orc_handle* h, int64_t n, const double* x, const double* v,
                      const double* w, const double* d, const double* rho);
/* Optional lagged acceleration (n*3) used by the added-mass force. */
int orc_set_accel(orc_handle* h, const double* a_prev);
/* Fluid fields, C*3 row-major; NULL grad_p => rho_f*g (hydrostatic); NULL DUDt => 0. */
int orc_set_fluid(orc_handle* h, const double* U, const double* grad_p, const double* DUDt);
/* Smoothed solid fraction (C) seen by the drag law. */
int orc_set_eps(orc_handle* h, const double* eps);

/* Threads of the particle loops and of the smoothing (one field per thread); the
   results do not depend on the count.  Default 1. */
int orc_set_threads(orc_handle* h, int32_t threads);
/* Advance n_sub substeps (contact, lubrication, fluid forces, leapfrog). */
int orc_step(orc_handle* h, int32_t n_sub);
/* Forces at the current state, without advancing: each n*3 (NULL to skip). */
int orc_forces(orc_handle* h, double* f_contact, double* f_lub, double* f_fluid,
               double* torque);
int orc_get_particles(orc_handle* h, double* x, double* v, double* w, double* a_prev);

/* Tangential history: number of pairs in contact, and (i, j, xi[3]) for each,
   i < j by particle index.  Wall histories: n*6*3 (walls lo x, hi x, lo y, ...). */
int64_t orc_num_contacts(orc_handle* h);
int orc_get_contacts(orc_handle* h, int64_t cap, int64_t* ij, double* xi);
int orc_get_wall_history(orc_handle* h, double* xi_wall);

/* Set the tangential history: m pairs (i < j) with springs xi (m*3) as seen from i,
   and the wall springs (n*6*3).  Returns -1 on a bad pair. */
int orc_set_contacts(orc_handle* h, int64_t m, const int64_t* ij, const double* xi);
int orc_set_wall_history(orc_handle* h, const double* xi_wall);

/* Neighbour lists: every j != i with |x_j - x_i|^2 < (r_i + r_j + h_out + skin)^2.
   offsets has n+1 entries; idx receives sorted j per i.  Returns the total count,
   or -1 if cap is too small.  brute = 1: O(N^2) all pairs; 0: link-cell bins. */
int64_t orc_neighbors(orc_handle* h, double skin, int32_t brute, int64_t* offsets,
                      int64_t* idx, int64_t cap);

/* PCM deposition into 7 int64 fixed-point fields [7][C]:
   eps, eps*U (3), force density on the fluid (3). */
int orc_deposit(orc_handle* h, int64_t* q);
/* Diffusion smoothing of nf fields [nf][C] in place.  guess (nf*C or NULL) is an
   initial guess for the first pseudo-step, projected onto the conserved sum.
   iters receives the CG iterations per field, summed over pseudo-steps. */
int orc_smooth(orc_handle* h, int32_t nf, double* phi, const double* guess, int32_t* iters);
/* Deposition + smoothing; eps (C), Us (C*3), Ffp (C*3), any may be NULL.  The
   smoothed solid fraction becomes the one the drag law sees. */
int orc_average(orc_handle* h, double* eps, double* Us, double* Ffp);
/* The smoothing and outputs of orc_average from a given deposition q [7][C]. */
int orc_average_fixed(orc_handle* h, const int64_t* q, double* eps, double* Us, double* Ffp);

/* Single-particle helpers used by the pins. */
void orc_drag(const orc_params* p, double eps_s, const double w[3], double d,
              double out_f[3], double* Vr, double* Cd_times_w);
double orc_vr(double eps_f, double Re);
/* Faces of the z mesh (n_z + 1 values). */
void orc_z_faces(const orc_params* p, double* faces);
/* y = (I - dtau div(D grad)) x on one field (the operator of a smoothing step). */
void orc_smooth_operator(const orc_params* p, const double* x, double* y);
/* Vorticity curl U of a cell-centred field U (C*3) into omega (C*3). */
void orc_curl(const orc_params* p, const double* U, double* omega);
/* Lift force on a sphere of diameter d with slip w = U_f - u_p in vorticity omega. */
void orc_lift(const orc_params* p, const double w[3], const double omega[3], double d,
              double out_f[3]);
/* Lubrication on a for the pair (a, b), dx = x_b - x_a: force on a, torques on a
   and b (b receives -F). */
void orc_lub_pair(const orc_params* p, const double dx[3], double ra, double rb,
                  const double va[3], const double vb[3], const double wa[3],
                  const double wb[3], double F[3], double Ta[3], double Tb[3]);
/* Contact of the pair (a, b) with spring xi_old, dx = x_b - x_a: force on a, torques
   on a and b, updated spring.  Returns 1 if the spheres overlap, else 0 (outputs
   untouched). */
int orc_hm_pair(const orc_params* p, const double dx[3], double ra, double rb, double ma,
                double mb, const double va[3], const double vb[3], const double wa[3],
                const double wb[3], const double xi_old[3], double F[3], double Ta[3],
                double Tb[3], double xi_new[3]);
/* Lubrication against a wall: n unit normal towards the wall, dist centre-to-plane. */
void orc_lub_wall(const orc_params* p, const double n[3], double dist, double r,
                  const double v[3], const double w[3], double F[3], double T[3]);

}  /* extern "C" */
