/*
 * Oracle (test infrastructure only): diffusion-based averaging, Sec. 2.4.
 *
 * Deposition, Eq. (9) (particle centroid method): each particle adds to the cell
 * containing its centre
 *   eps_s        += V_p / V_c
 *   eps_s U_s    += V_p u_p / V_c
 *   F^fp         += -f_fp / V_c     (Sec. 2.2: per-particle forces summed to the
 *                                    cell scale; the fluid feels the reaction)
 * Reading: the sums are kept as 64-bit fixed point, q = llrint(value * 2^S)
 * (round to nearest even), one exponent S per field kind, so the result does not
 * depend on the order of the additions.  f_fp is the fluid force at the current
 * state (drag + pressure gradient + added mass); lubrication stays with the
 * particles.  The cell of a particle is floor((x - lo) * n / L), clamped.
 *
 * Smoothing, Eq. (10): d(phi)/d(tau) = div(D grad phi) up to unit pseudo-time,
 * D_a = b_a^2 / 4 per axis, which equals Gaussian-kernel averaging with
 * bandwidth b (kernel exp(-r^2/b^2)).  Readings: n_tau implicit steps of size
 * dtau = 1/n_tau, backward Euler  (I - dtau L) phi^{m+1} = phi^m  by default, or the
 * second-order implicit scheme the paper's OpenFOAM run uses (Sec. 2.4), read as
 * BDF2:  (I - (2/3) dtau L) phi^{m+1} = (4/3) phi^m - (1/3) phi^{m-1}, its first step
 * backward Euler (both keep sum(phi) since (4/3) - (1/3) = 1),
 * the 7-point finite-volume Laplacian with zero flux through non-periodic faces
 * (Sec. 2.4: "no-flux boundary condition ... conservative"), each step solved by
 * plain unpreconditioned conjugate gradients to ||r|| <= rtol ||b|| from
 * x0 = phi^m.  An initial guess is first shifted so its sum equals sum(b).
 * U_s = (eps_s U_s) / max(eps_s, 1e-12) after smoothing.
 *
 * Graded z mesh (z_grading != 1; Sec. 4.2 refines the mesh towards the bottom).
 * Reading: cell heights h_k grow geometrically from the floor (faces in
 * orc_internal.h); a particle's cell is the one whose faces enclose its centre;
 * V_c = h_x h_y h_k.  The finite-volume diffusion step on the graded mesh:
 *   (A x)_c = x_c - [c_x sum_x (x_nb - x_c) + c_y sum_y (x_nb - x_c)
 *                    + c-_k (x_{k-1} - x_c) + c+_k (x_{k+1} - x_c)],
 *   c-_k = dtau D_z / (h_k (zc_k - zc_{k-1})),  c+_k = dtau D_z / (h_k (zc_{k+1} - zc_k)),
 * i.e. V_c (x - b) / dtau = sum over faces of A_f D (x_nb - x_c) / |zc_nb - zc_c|,
 * which keeps sum(V_c x).  CG runs on the symmetric form W A x = W b,
 * W = diag(h_k / mean h), to ||W (b - A x)|| <= rtol ||W b||.
 */
#include <algorithm>
#include <cstring>

#include "orc_internal.h"

using orc::V3;

namespace {

int64_t cell_of(const orc_params& p, const orc::ZGrid& zg, V3 x) {
  int64_t c[3];
  for (int a = 0; a < 3; ++a) {
    if (a == 2 && zg.graded) {
      int64_t k = (int64_t)(std::upper_bound(zg.zf.begin(), zg.zf.end(), x.z) - zg.zf.begin()) - 1;
      if (k < 0) k = 0;
      if (k > p.ncell[2] - 1) k = p.ncell[2] - 1;
      c[2] = k;
      continue;
    }
    double inv = (double)p.ncell[a] / (p.hi[a] - p.lo[a]);
    double s = (orc::comp(x, a) - p.lo[a]) * inv;
    int64_t k = (int64_t)std::floor(s);
    if (k < 0) k = 0;
    if (k > p.ncell[a] - 1) k = p.ncell[a] - 1;
    c[a] = k;
  }
  return (c[2] * p.ncell[1] + c[1]) * p.ncell[0] + c[0];
}

double cell_volume(const orc_params& p, const orc::ZGrid& zg, int64_t kz) {
  double dx = (p.hi[0] - p.lo[0]) / p.ncell[0];
  double dy = (p.hi[1] - p.lo[1]) / p.ncell[1];
  double dz = zg.graded ? zg.hz[kz] : (p.hi[2] - p.lo[2]) / p.ncell[2];
  return dx * dy * dz;
}

/* The graded-mesh operator of one pseudo-step (coefficients times scale). */
struct GradedOp {
  double cx, cy;
  std::vector<double> czm, czp, w;
};

GradedOp graded_op(const orc_params& p, const orc::ZGrid& zg, double scale) {
  GradedOp op;
  const int64_t n = p.ncell[2];
  const double dtau = 1.0 / p.n_tau;
  const double hx = (p.hi[0] - p.lo[0]) / p.ncell[0], hy = (p.hi[1] - p.lo[1]) / p.ncell[1];
  const double D[3] = {0.25 * p.bandwidth[0] * p.bandwidth[0], 0.25 * p.bandwidth[1] * p.bandwidth[1],
                       0.25 * p.bandwidth[2] * p.bandwidth[2]};
  op.cx = scale * dtau * D[0] / (hx * hx);
  op.cy = scale * dtau * D[1] / (hy * hy);
  op.czm.assign(n, 0.0);
  op.czp.assign(n, 0.0);
  op.w.assign(n, 0.0);
  const double hmean = (p.hi[2] - p.lo[2]) / (double)n;
  for (int64_t k = 0; k < n; ++k) {
    if (k > 0) op.czm[k] = scale * dtau * D[2] / (zg.hz[k] * (zg.zc[k] - zg.zc[k - 1]));
    if (k < n - 1) op.czp[k] = scale * dtau * D[2] / (zg.hz[k] * (zg.zc[k + 1] - zg.zc[k]));
    op.w[k] = zg.hz[k] / hmean;
  }
  return op;
}

/* y = A x (weighted = false) or W A x on the graded mesh. */
void apply_graded(const orc_params& p, const GradedOp& op, const std::vector<double>& x,
                  std::vector<double>& y, bool weighted) {
  int64_t nx = p.ncell[0], ny = p.ncell[1], nz = p.ncell[2];
  const int64_t n[2] = {nx, ny};
  const double cxy[2] = {op.cx, op.cy};
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int64_t id[2] = {i, j};
        int64_t c = (k * ny + j) * nx + i;
        double lap = 0.0;
        for (int a = 0; a < 2; ++a) {
          for (int s = -1; s <= 1; s += 2) {
            int64_t t[2] = {i, j};
            t[a] = id[a] + s;
            if (t[a] < 0 || t[a] >= n[a]) {
              if (!p.periodic[a]) continue;
              t[a] = (t[a] + n[a]) % n[a];
            }
            lap += cxy[a] * (x[(k * ny + t[1]) * nx + t[0]] - x[c]);
          }
        }
        if (k > 0) lap += op.czm[k] * (x[c - nx * ny] - x[c]);
        if (k < nz - 1) lap += op.czp[k] * (x[c + nx * ny] - x[c]);
        y[c] = (weighted ? op.w[k] : 1.0) * (x[c] - lap);
      }
}

bool fixed(double v, int S, int64_t* q) {
  double s = std::ldexp(v, S);
  if (!(std::fabs(s) < 4.0e18)) return false;
  *q = (int64_t)std::llrint(s);
  return true;
}

/* y = (I - dtau div(D grad)) x on one field. */
void apply_A(const orc_params& p, const double coef[3], const std::vector<double>& x,
             std::vector<double>& y) {
  int64_t nx = p.ncell[0], ny = p.ncell[1], nz = p.ncell[2];
  int64_t n[3] = {nx, ny, nz};
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int64_t id[3] = {i, j, k};
        int64_t c = (k * ny + j) * nx + i;
        double lap = 0.0;
        for (int a = 0; a < 3; ++a) {
          for (int s = -1; s <= 1; s += 2) {
            int64_t t[3] = {i, j, k};
            t[a] = id[a] + s;
            if (t[a] < 0 || t[a] >= n[a]) {
              if (!p.periodic[a]) continue; /* no flux through this face */
              t[a] = (t[a] + n[a]) % n[a];
            }
            int64_t cn = (t[2] * ny + t[1]) * nx + t[0];
            lap += coef[a] * (x[cn] - x[c]);
          }
        }
        y[c] = x[c] - lap;
      }
}

double dotv(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

/* Plain CG on A x = b starting from x; returns iterations or -1. */
int cg(const orc_params& p, const double coef[3], const std::vector<double>& b,
       std::vector<double>& x) {
  size_t C = b.size();
  double bnorm = std::sqrt(dotv(b, b));
  if (!(bnorm > 0.0)) {
    x.assign(C, 0.0);
    return 0;
  }
  std::vector<double> r(C), q(C), pv(C);
  apply_A(p, coef, x, q);
  for (size_t i = 0; i < C; ++i) r[i] = b[i] - q[i];
  pv = r;
  double rr = dotv(r, r);
  if (std::sqrt(rr) <= p.cg_rtol * bnorm) return 0;
  for (int it = 1; it <= p.cg_max_iter; ++it) {
    apply_A(p, coef, pv, q);
    double alpha = rr / dotv(pv, q);
    for (size_t i = 0; i < C; ++i) {
      x[i] += alpha * pv[i];
      r[i] -= alpha * q[i];
    }
    double rr_new = dotv(r, r);
    if (std::sqrt(rr_new) <= p.cg_rtol * bnorm) return it;
    double beta = rr_new / rr;
    rr = rr_new;
    for (size_t i = 0; i < C; ++i) pv[i] = r[i] + beta * pv[i];
  }
  return -1;
}

/* Plain CG on the symmetric graded system W A x = W b starting from x. */
int cg_graded(const orc_params& p, const GradedOp& op, const std::vector<double>& b0,
              std::vector<double>& x) {
  const int64_t nxy = (int64_t)p.ncell[0] * p.ncell[1];
  size_t C = b0.size();
  std::vector<double> b(C);
  for (size_t i = 0; i < C; ++i) b[i] = op.w[i / nxy] * b0[i];
  double bnorm = std::sqrt(dotv(b, b));
  if (!(bnorm > 0.0)) {
    x.assign(C, 0.0);
    return 0;
  }
  std::vector<double> r(C), q(C), pv(C);
  apply_graded(p, op, x, q, true);
  for (size_t i = 0; i < C; ++i) r[i] = b[i] - q[i];
  pv = r;
  double rr = dotv(r, r);
  if (std::sqrt(rr) <= p.cg_rtol * bnorm) return 0;
  for (int it = 1; it <= p.cg_max_iter; ++it) {
    apply_graded(p, op, pv, q, true);
    double alpha = rr / dotv(pv, q);
    for (size_t i = 0; i < C; ++i) {
      x[i] += alpha * pv[i];
      r[i] -= alpha * q[i];
    }
    double rr_new = dotv(r, r);
    if (std::sqrt(rr_new) <= p.cg_rtol * bnorm) return it;
    double beta = rr_new / rr;
    rr = rr_new;
    for (size_t i = 0; i < C; ++i) pv[i] = r[i] + beta * pv[i];
  }
  return -1;
}

}  // namespace

extern "C" {

void orc_z_faces(const orc_params* p, double* faces) {
  const orc::ZGrid zg = orc::zgrid(*p);
  for (size_t k = 0; k < zg.zf.size(); ++k) faces[k] = zg.zf[k];
}

void orc_smooth_operator(const orc_params* p, const double* x, double* y) {
  const int64_t C = (int64_t)p->ncell[0] * p->ncell[1] * p->ncell[2];
  std::vector<double> xv(x, x + C), yv(C);
  const orc::ZGrid zg = orc::zgrid(*p);
  if (zg.graded) {
    apply_graded(*p, graded_op(*p, zg, 1.0), xv, yv, false);
  } else {
    double coef[3];
    for (int a = 0; a < 3; ++a) {
      const double h = (p->hi[a] - p->lo[a]) / p->ncell[a];
      coef[a] = (1.0 / p->n_tau) * (0.25 * p->bandwidth[a] * p->bandwidth[a]) / (h * h);
    }
    apply_A(*p, coef, xv, yv);
  }
  for (int64_t c = 0; c < C; ++c) y[c] = yv[c];
}

int orc_deposit(orc_handle* h, int64_t* q) {
  const orc_params& p = h->p;
  int64_t C = h->ncells();
  std::memset(q, 0, sizeof(int64_t) * 7 * C);
  const orc::ZGrid zg = orc::zgrid(p);
  double fluid[3];
  std::vector<double> ffp(3 * h->n);
  orc_forces(h, nullptr, nullptr, ffp.data(), nullptr);
  const int64_t nxy = (int64_t)p.ncell[0] * p.ncell[1];
  for (int64_t i = 0; i < h->n; ++i) {
    int64_t c = cell_of(p, zg, h->x[i]);
    double vc = cell_volume(p, zg, c / nxy);
    double d = h->d[i];
    double Vp = M_PI / 6.0 * d * d * d;
    double vfrac = Vp / vc;
    int64_t t;
    if (!fixed(vfrac, p.shift_eps, &t)) return -5;
    q[c] += t;
    for (int a = 0; a < 3; ++a) {
      if (!fixed(vfrac * orc::comp(h->v[i], a), p.shift_mom, &t)) return -5;
      q[(1 + a) * C + c] += t;
      fluid[a] = ffp[3 * i + a];
      if (!fixed(-fluid[a] / vc, p.shift_force, &t)) return -5;
      q[(4 + a) * C + c] += t;
    }
  }
  return 0;
}

int orc_smooth(orc_handle* h, int32_t nf, double* phi, const double* guess, int32_t* iters) {
  const orc_params& p = h->p;
  int64_t C = h->ncells();
  double dxs[3], coef[3];
  double dtau = 1.0 / p.n_tau;
  for (int a = 0; a < 3; ++a) {
    dxs[a] = (p.hi[a] - p.lo[a]) / p.ncell[a];
    double D = 0.25 * p.bandwidth[a] * p.bandwidth[a];
    coef[a] = dtau * D / (dxs[a] * dxs[a]);
  }
  const double coef2[3] = {2.0 / 3.0 * coef[0], 2.0 / 3.0 * coef[1], 2.0 / 3.0 * coef[2]};
  const orc::ZGrid zg = orc::zgrid(p);
  GradedOp gop, gop2;
  if (zg.graded) {
    gop = graded_op(p, zg, 1.0);
    gop2 = graded_op(p, zg, 2.0 / 3.0);
  }
  const int64_t nxy = (int64_t)p.ncell[0] * p.ncell[1];
  /* the fields are independent: one per thread with orc_set_threads(n > 1) */
  std::vector<int> fstatus(nf, 0);
#pragma omp parallel for schedule(dynamic, 1) num_threads(h->threads > 1 ? h->threads : 1)
  for (int32_t f = 0; f < nf; ++f) {
    std::vector<double> x(phi + f * C, phi + (f + 1) * C);
    std::vector<double> x_prev;
    int32_t total = 0;
    for (int32_t m = 0; m < p.n_tau; ++m) {
      const bool bdf2 = p.tau_scheme == 1 && m > 0;
      std::vector<double> b = x;
      if (bdf2)
        for (int64_t c = 0; c < C; ++c) b[c] = 4.0 / 3.0 * x[c] - 1.0 / 3.0 * x_prev[c];
      x_prev = x;
      if (m == 0 && guess) {
        x.assign(guess + f * C, guess + (f + 1) * C);
        double sb = 0.0, sx = 0.0, sw = 0.0;
        for (int64_t c = 0; c < C; ++c) {
          const double w = zg.graded ? gop.w[c / nxy] : 1.0;
          sb += w * b[c];
          sx += w * x[c];
          sw += w;
        }
        double shift = (sb - sx) / (zg.graded ? sw : (double)C);
        for (int64_t c = 0; c < C; ++c) x[c] += shift;
      }
      int it = zg.graded ? cg_graded(p, bdf2 ? gop2 : gop, b, x) : cg(p, bdf2 ? coef2 : coef, b, x);
      if (it < 0) {
        fstatus[f] = -6;
        it = p.cg_max_iter;
      }
      total += it;
    }
    std::memcpy(phi + f * C, x.data(), sizeof(double) * C);
    if (iters) iters[f] = total;
  }
  for (int32_t f = 0; f < nf; ++f)
    if (fstatus[f]) return fstatus[f];
  return 0;
}

int orc_average(orc_handle* h, double* eps, double* Us, double* Ffp) {
  std::vector<int64_t> q(7 * h->ncells());
  int st = orc_deposit(h, q.data());
  if (st) return st;
  return orc_average_fixed(h, q.data(), eps, Us, Ffp);
}

int orc_average_fixed(orc_handle* h, const int64_t* q, double* eps, double* Us, double* Ffp) {
  const orc_params& p = h->p;
  int64_t C = h->ncells();
  int st = 0;
  std::vector<double> phi(7 * C);
  int shifts[7] = {p.shift_eps, p.shift_mom, p.shift_mom, p.shift_mom,
                   p.shift_force, p.shift_force, p.shift_force};
  for (int f = 0; f < 7; ++f)
    for (int64_t c = 0; c < C; ++c) phi[f * C + c] = std::ldexp((double)q[f * C + c], -shifts[f]);
  st = orc_smooth(h, 7, phi.data(), nullptr, nullptr);
  for (int64_t c = 0; c < C; ++c) {
    double e = phi[c];
    if (eps) eps[c] = e;
    double den = e > 1e-12 ? e : 1e-12;
    for (int a = 0; a < 3; ++a) {
      if (Us) Us[3 * c + a] = phi[(1 + a) * C + c] / den;
      if (Ffp) Ffp[3 * c + a] = phi[(4 + a) * C + c];
    }
  }
  h->eps.assign(phi.begin(), phi.begin() + C);
  return st;
}

}  // extern "C"
