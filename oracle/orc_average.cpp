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
 */
#include <cstring>

#include "orc_internal.h"

using orc::V3;

namespace {

int64_t cell_of(const orc_params& p, V3 x) {
  int64_t c[3];
  for (int a = 0; a < 3; ++a) {
    double inv = (double)p.ncell[a] / (p.hi[a] - p.lo[a]);
    double s = (orc::comp(x, a) - p.lo[a]) * inv;
    int64_t k = (int64_t)std::floor(s);
    if (k < 0) k = 0;
    if (k > p.ncell[a] - 1) k = p.ncell[a] - 1;
    c[a] = k;
  }
  return (c[2] * p.ncell[1] + c[1]) * p.ncell[0] + c[0];
}

double cell_volume(const orc_params& p) {
  double dx = (p.hi[0] - p.lo[0]) / p.ncell[0];
  double dy = (p.hi[1] - p.lo[1]) / p.ncell[1];
  double dz = (p.hi[2] - p.lo[2]) / p.ncell[2];
  return dx * dy * dz;
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

}  // namespace

extern "C" {

int orc_deposit(orc_handle* h, int64_t* q) {
  const orc_params& p = h->p;
  int64_t C = h->ncells();
  std::memset(q, 0, sizeof(int64_t) * 7 * C);
  double vc = cell_volume(p);
  double fluid[3];
  std::vector<double> ffp(3 * h->n);
  orc_forces(h, nullptr, nullptr, ffp.data(), nullptr);
  for (int64_t i = 0; i < h->n; ++i) {
    int64_t c = cell_of(p, h->x[i]);
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
  int status = 0;
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
        double sb = 0.0, sx = 0.0;
        for (int64_t c = 0; c < C; ++c) {
          sb += b[c];
          sx += x[c];
        }
        double shift = (sb - sx) / (double)C;
        for (int64_t c = 0; c < C; ++c) x[c] += shift;
      }
      int it = cg(p, bdf2 ? coef2 : coef, b, x);
      if (it < 0) {
        status = -6;
        it = p.cg_max_iter;
      }
      total += it;
    }
    std::memcpy(phi + f * C, x.data(), sizeof(double) * C);
    if (iters) iters[f] = total;
  }
  return status;
}

int orc_average(orc_handle* h, double* eps, double* Us, double* Ffp) {
  const orc_params& p = h->p;
  int64_t C = h->ncells();
  std::vector<int64_t> q(7 * C);
  int st = orc_deposit(h, q.data());
  if (st) return st;
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
