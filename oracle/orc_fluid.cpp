/*
 * Oracle (test infrastructure only): fluid-particle forces, Sec. 2.3.
 *
 * Interpolation (Sec. 2.3 says only that U_f is "interpolated to the center of
 * particle i"; Sec. 2.2 says fluid fields are not smoothed before use).  Reading:
 * trilinear interpolation of the cell-centred fields; periodic axes wrap, other
 * axes clamp to the first/last cell centre.  On a graded z mesh (Sec. 4.2) the z
 * weight is the linear one between the two enclosing cell centres.
 *
 * Drag, Eq. (3)-(6), the Syamlal-O'Brien correlation of the MFIX documentation.
 * Readings of the garbled print:
 *   - C_d = (0.63 + 4.8 sqrt(V_r/Re))^2  (the print drops the square and a digit);
 *   - Re = d |u - U| / nu_f  (the print has rho_i and no viscosity);
 *   - beta carries eps_s eps_f, so f = V_p beta w / (eps_f eps_s) reduces to
 *       f_drag = (3/4) V_p C_d rho_f |w| w / (V_r^2 d),  w = U_f - u_p,
 *     i.e. the drag pulls the particle towards the fluid velocity;
 *   - eps_f = 1 - min(max(eps_s, 0), eps_max).
 * Pressure gradient / buoyancy (Sec. 2.3 lists it with no formula):
 *   f_pg = -V_p grad p, grad p = rho_f g when the caller supplies none.
 * Added mass, Eq. (8), with the physical sign:
 *   f_add = C_add rho_f V_p (DU_f/Dt - a_prev),
 * where a_prev is the particle's acceleration of the previous substep (the paper
 * uses the particle velocity of the previous time).
 * Lift, Eq. (7) (lift = 1), printed as C_l rho_f nu^0.5 D^2 (u_p - U_f) x grad U_f,
 * which is not a force dimensionally and whose sign would push a particle that lags
 * the flow towards slower fluid.  Reading: Saffman's (1965) shear lift, of which the
 * print is the scalar shear-flow form,
 *   f_lift = C_l rho_f nu^0.5 d^2 |omega|^(-1/2) (w x omega),  w = U_f - u_p,
 *   omega = curl U_f at the particle, C_l = 1.6,
 * so a sphere at rest in the shear flow U = (G z, 0, 0) feels
 * C_l rho_f nu^0.5 d^2 G^0.5 U_x along +z (towards the faster fluid); f_lift = 0
 * where omega = 0.  omega is the trilinear interpolant of the cell-centred vorticity
 * of U_f (the paper takes grad U_f from the fluid solver): second-order central
 * differences, wrapped on periodic axes, one-sided in the first and last cell of
 * other axes, zero along an axis of one cell; on a graded z mesh the z differences
 * divide by the distance between the centres used.  The lift is part of f_fp, so the
 * fluid also receives it through the deposition.
 */
#include <algorithm>

#include "orc_internal.h"

namespace orc {

ZGrid zgrid(const orc_params& p) {
  ZGrid g;
  const int64_t n = p.ncell[2];
  const double L = p.hi[2] - p.lo[2];
  g.graded = p.z_grading != 1.0 && n >= 2;
  g.zf.resize(n + 1);
  for (int64_t k = 0; k <= n; ++k) {
    if (g.graded) {
      const double lr = std::log(p.z_grading) / (double)(n - 1);  /* ln r */
      g.zf[k] = p.lo[2] + L * (std::expm1((double)k * lr) / std::expm1((double)n * lr));
    } else {
      g.zf[k] = p.lo[2] + L * (double)k / (double)n;
    }
  }
  g.zf[0] = p.lo[2];
  g.zf[n] = p.hi[2];
  g.zc.resize(n);
  g.hz.resize(n);
  for (int64_t k = 0; k < n; ++k) {
    g.zc[k] = 0.5 * (g.zf[k] + g.zf[k + 1]);
    g.hz[k] = g.zf[k + 1] - g.zf[k];
  }
  return g;
}

namespace {

struct Axis {
  int64_t i0, i1;
  double f;
};

Axis axis_weights(const orc_params& p, int a, double x) {
  int n = p.ncell[a];
  if (a == 2 && p.z_grading != 1.0 && n >= 2) {
    /* graded z: linear weight between the enclosing centres, clamped outside */
    const ZGrid g = zgrid(p);
    Axis ax;
    if (!(x > g.zc[0])) {
      ax.i0 = 0;
      ax.i1 = 1;
      ax.f = 0.0;
    } else if (!(x < g.zc[n - 1])) {
      ax.i0 = n - 2;
      ax.i1 = n - 1;
      ax.f = 1.0;
    } else {
      int64_t k = (int64_t)(std::upper_bound(g.zc.begin(), g.zc.end(), x) - g.zc.begin()) - 1;
      ax.i0 = k;
      ax.i1 = k + 1;
      ax.f = (x - g.zc[k]) / (g.zc[k + 1] - g.zc[k]);
    }
    return ax;
  }
  double inv = (double)n / (p.hi[a] - p.lo[a]);
  double s = (x - p.lo[a]) * inv - 0.5;
  Axis ax;
  if (p.periodic[a]) {
    double fl = std::floor(s);
    ax.f = s - fl;
    int64_t i0 = (int64_t)fl;
    i0 = ((i0 % n) + n) % n;
    ax.i0 = i0;
    ax.i1 = (i0 + 1) % n;
  } else {
    if (s < 0.0) s = 0.0;
    if (s > (double)(n - 1)) s = (double)(n - 1);
    int64_t i0 = (int64_t)std::floor(s);
    if (n >= 2 && i0 > n - 2) i0 = n - 2;
    if (n < 2) i0 = 0;
    ax.i0 = i0;
    ax.i1 = n >= 2 ? i0 + 1 : 0;
    ax.f = n >= 2 ? s - (double)i0 : 0.0;
  }
  return ax;
}

}  // namespace

double interp_scalar(const orc_params& p, const std::vector<double>& fld, int ncomp, int c,
                     V3 x) {
  Axis ax = axis_weights(p, 0, x.x), ay = axis_weights(p, 1, x.y), az = axis_weights(p, 2, x.z);
  int64_t nx = p.ncell[0], ny = p.ncell[1];
  double acc = 0.0;
  for (int kz = 0; kz < 2; ++kz) {
    int64_t iz = kz ? az.i1 : az.i0;
    double wz = kz ? az.f : 1.0 - az.f;
    for (int ky = 0; ky < 2; ++ky) {
      int64_t iy = ky ? ay.i1 : ay.i0;
      double wy = ky ? ay.f : 1.0 - ay.f;
      for (int kx = 0; kx < 2; ++kx) {
        int64_t ix = kx ? ax.i1 : ax.i0;
        double wx = kx ? ax.f : 1.0 - ax.f;
        int64_t cell = (iz * ny + iy) * nx + ix;
        acc += wz * wy * wx * fld[cell * ncomp + c];
      }
    }
  }
  return acc;
}

double vr_of(double eps_f, double Re) {
  double A1 = std::pow(eps_f, 4.14);
  double A2 = eps_f <= 0.85 ? 0.8 * std::pow(eps_f, 1.28) : std::pow(eps_f, 2.65);
  double t = 0.06 * Re;
  return 0.5 * (A1 - t + std::sqrt(t * t + 0.12 * Re * (2.0 * A2 - A1) + A1 * A1));
}

V3 drag_force(const orc_params& p, double eps_s, V3 w, double d, double* Vr_out,
              double* Cdw_out) {
  double es = eps_s < 0.0 ? 0.0 : eps_s;
  if (es > p.eps_max) es = p.eps_max;
  double eps_f = 1.0 - es;
  double wmag = norm(w);
  double Re = d * wmag / p.nu_f;
  double Vr = vr_of(eps_f, Re);
  if (Vr_out) *Vr_out = Vr;
  if (!(wmag > 0.0)) {
    if (Cdw_out) *Cdw_out = 0.0;
    return V3{0, 0, 0};
  }
  double c = 0.63 + 4.8 * std::sqrt(Vr / Re);
  double Cd = c * c;
  if (Cdw_out) *Cdw_out = Cd * wmag;
  double Vp = M_PI / 6.0 * d * d * d;
  return scl(0.75 * Cd * p.rho_f * wmag * Vp / (Vr * Vr * d), w);
}

void curl_cells(const orc_params& p, const std::vector<double>& U, std::vector<double>& out) {
  const int64_t n[3] = {p.ncell[0], p.ncell[1], p.ncell[2]};
  const int64_t C = n[0] * n[1] * n[2];
  out.assign(3 * C, 0.0);
  const ZGrid zg = zgrid(p);
  for (int64_t iz = 0; iz < n[2]; ++iz)
    for (int64_t iy = 0; iy < n[1]; ++iy)
      for (int64_t ix = 0; ix < n[0]; ++ix) {
        const int64_t idx[3] = {ix, iy, iz};
        /* g[a][b] = dU_b / dx_a at this cell */
        double g[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int a = 0; a < 3; ++a) {
          if (n[a] < 2) continue;
          const double h = (p.hi[a] - p.lo[a]) / (double)n[a];
          int64_t ip[3] = {ix, iy, iz}, im[3] = {ix, iy, iz};
          double den;
          if (p.periodic[a]) {
            ip[a] = (idx[a] + 1) % n[a];
            im[a] = (idx[a] + n[a] - 1) % n[a];
            den = 2.0 * h;
          } else if (idx[a] == 0) {
            ip[a] = 1;
            den = h;
          } else if (idx[a] == n[a] - 1) {
            im[a] = n[a] - 2;
            den = h;
          } else {
            ip[a] = idx[a] + 1;
            im[a] = idx[a] - 1;
            den = 2.0 * h;
          }
          if (a == 2 && zg.graded) den = zg.zc[ip[2]] - zg.zc[im[2]];
          const int64_t cp = (ip[2] * n[1] + ip[1]) * n[0] + ip[0];
          const int64_t cm = (im[2] * n[1] + im[1]) * n[0] + im[0];
          for (int b = 0; b < 3; ++b) g[a][b] = (U[3 * cp + b] - U[3 * cm + b]) / den;
        }
        const int64_t c = (iz * n[1] + iy) * n[0] + ix;
        out[3 * c + 0] = g[1][2] - g[2][1];
        out[3 * c + 1] = g[2][0] - g[0][2];
        out[3 * c + 2] = g[0][1] - g[1][0];
      }
}

V3 lift_force(const orc_params& p, V3 w, V3 omega, double d) {
  double om = norm(omega);
  if (!(om > 0.0)) return V3{0, 0, 0};
  return scl(p.c_lift * p.rho_f * std::sqrt(p.nu_f) * d * d / std::sqrt(om), cross(w, omega));
}

V3 fluid_force(const orc_params& p, const FluidFields& ff, V3 x, V3 u, V3 a_prev, double d) {
  double Vp = M_PI / 6.0 * d * d * d;
  V3 f{0, 0, 0};
  if (p.lift) {
    V3 U{interp_scalar(p, *ff.U, 3, 0, x), interp_scalar(p, *ff.U, 3, 1, x),
         interp_scalar(p, *ff.U, 3, 2, x)};
    V3 om{interp_scalar(p, *ff.curlU, 3, 0, x), interp_scalar(p, *ff.curlU, 3, 1, x),
          interp_scalar(p, *ff.curlU, 3, 2, x)};
    f = add(f, lift_force(p, sub(U, u), om, d));
  }
  if (p.drag) {
    V3 U{interp_scalar(p, *ff.U, 3, 0, x), interp_scalar(p, *ff.U, 3, 1, x),
         interp_scalar(p, *ff.U, 3, 2, x)};
    double es = interp_scalar(p, *ff.eps, 1, 0, x);
    f = add(f, drag_force(p, es, sub(U, u), d, nullptr, nullptr));
  }
  if (p.pressure_grad) {
    V3 gp{interp_scalar(p, *ff.gradp, 3, 0, x), interp_scalar(p, *ff.gradp, 3, 1, x),
          interp_scalar(p, *ff.gradp, 3, 2, x)};
    f = add(f, scl(-Vp, gp));
  }
  if (p.added_mass) {
    V3 Du{interp_scalar(p, *ff.DUDt, 3, 0, x), interp_scalar(p, *ff.DUDt, 3, 1, x),
          interp_scalar(p, *ff.DUDt, 3, 2, x)};
    f = add(f, scl(p.c_add * p.rho_f * Vp, sub(Du, a_prev)));
  }
  return f;
}

}  // namespace orc

extern "C" {

void orc_drag(const orc_params* p, double eps_s, const double w[3], double d, double out_f[3],
              double* Vr, double* Cd_times_w) {
  orc::V3 f = orc::drag_force(*p, eps_s, orc::V3{w[0], w[1], w[2]}, d, Vr, Cd_times_w);
  out_f[0] = f.x;
  out_f[1] = f.y;
  out_f[2] = f.z;
}

double orc_vr(double eps_f, double Re) { return orc::vr_of(eps_f, Re); }

void orc_curl(const orc_params* p, const double* U, double* omega) {
  const int64_t C = (int64_t)p->ncell[0] * p->ncell[1] * p->ncell[2];
  std::vector<double> u(U, U + 3 * C), out;
  orc::curl_cells(*p, u, out);
  for (int64_t k = 0; k < 3 * C; ++k) omega[k] = out[k];
}

void orc_lift(const orc_params* p, const double w[3], const double omega[3], double d,
              double out_f[3]) {
  orc::V3 f = orc::lift_force(*p, orc::load(w, 0), orc::load(omega, 0), d);
  orc::store(out_f, 0, f);
}

}  // extern "C"
