/*
 * Oracle (test infrastructure only): fluid-particle forces, Sec. 2.3.
 *
 * Interpolation (Sec. 2.3 says only that U_f is "interpolated to the center of
 * particle i"; Sec. 2.2 says fluid fields are not smoothed before use).  Reading:
 * trilinear interpolation of the cell-centred fields; periodic axes wrap, other
 * axes clamp to the first/last cell centre.
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
 */
#include "orc_internal.h"

namespace orc {

namespace {

struct Axis {
  int64_t i0, i1;
  double f;
};

Axis axis_weights(const orc_params& p, int a, double x) {
  int n = p.ncell[a];
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

V3 fluid_force(const orc_params& p, const FluidFields& ff, V3 x, V3 u, V3 a_prev, double d) {
  double Vp = M_PI / 6.0 * d * d * d;
  V3 f{0, 0, 0};
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

}  // extern "C"
