/*
 * Oracle (test infrastructure only): soft-sphere contact and lubrication.
 *
 * Contact.  Sec. 2.1 models particles as soft spheres with an elastic spring and a
 * viscous dashpot and cites Tsuji et al.; Sec. 2.5 adds that contacts persist
 * ("endured contacts") and Table 1 gives a friction coefficient.  The contact law
 * used here is Hertz-Mindlin with the Tsuji-type damping of Tsuji, Tanaka & Ishida
 * (1992) in the form published by Di Renzo & Di Maio (2004):
 *   E* = E / (2 (1 - nu^2)),  G* = G / (2 (2 - nu)),  G = E / (2 (1 + nu))
 *   beta = ln e / sqrt(ln^2 e + pi^2)
 *   S_n = 2 E* sqrt(R* delta),  S_t = 8 G* sqrt(R* delta)
 *   F_n = -(4/3) E* sqrt(R*) delta^(3/2) n  -  c_n v_n,   c_n = -2 sqrt(5/6) beta sqrt(S_n m*)
 *   F_t = -S_t xi - c_t v_t (capped at mu |F_n|),           c_t = -2 sqrt(5/6) beta sqrt(S_t m*)
 * The damping coefficients c_n, c_t are >= 0, so the dashpot opposes the
 * relative motion.  Readings where the paper is silent:
 *   - lever arms l = r - delta/2 (contact point mid-overlap), which makes the
 *     pair torques conserve angular momentum exactly;
 *   - the spring xi is first rotated onto the current tangent plane and rescaled
 *     to its old length, then incremented by v_t dt; after a Coulomb slip it is
 *     reset to the value that reproduces the capped force;
 *   - the spring is dropped when the overlap ends;
 *   - F_n is not clamped at zero (the damping may make it tensile).
 * A wall is a plane of the same material: R* = r, m* = m, same E*, G*.
 *
 * Lubrication.  Sec. 2.5: Ball & Melrose (1997), force proportional to the
 * relative velocity and inversely proportional to the gap.  Reading: the normal
 * squeeze term  F_a = -6 pi mu R_l^2 ((v_a - v_b).n) n / max(h, h_in),
 * R_l = r_a r_b / (r_a + r_b) (R_l = r for a wall), acting while the gap
 * h < h_out; h_in, h_out are fractions of the pair-mean diameter (the particle
 * diameter for a wall).  It also acts during overlap (with h_in).
 */
#include "orc_internal.h"

namespace orc {

V3 min_image(const orc_params& p, V3 xi, V3 xj) {
  V3 d = sub(xj, xi);
  for (int a = 0; a < 3; ++a) {
    if (!p.periodic[a]) continue;
    double L = p.hi[a] - p.lo[a];
    double s = comp(d, a);
    if (s > 0.5 * L) s = s - L;
    else if (s < -0.5 * L) s = s + L;
    set_comp(d, a, s);
  }
  return d;
}

namespace {

struct Material {
  double Es, Gs, beta;
};

Material material(const orc_params& p) {
  Material m;
  m.Es = p.E / (2.0 * (1.0 - p.poisson * p.poisson));
  double G = p.E / (2.0 * (1.0 + p.poisson));
  m.Gs = G / (2.0 * (2.0 - p.poisson));
  double lne = std::log(p.restitution);
  m.beta = lne / std::sqrt(lne * lne + M_PI * M_PI);
  return m;
}

/* Contact law for body a against partner b; n is the unit normal from a to b,
   delta > 0 the overlap, vrel the velocity of a's contact point relative to b's. */
void hm_core(const orc_params& p, V3 n, double delta, double Rs, double ms, V3 vrel, V3 xi_old,
             V3* F, V3* Ft_out, V3* xi_new) {
  Material mat = material(p);
  double sq = std::sqrt(Rs * delta);
  double Sn = 2.0 * mat.Es * sq;
  double St = 8.0 * mat.Gs * sq;
  double cn = -2.0 * std::sqrt(5.0 / 6.0) * mat.beta * std::sqrt(Sn * ms);
  double ct = -2.0 * std::sqrt(5.0 / 6.0) * mat.beta * std::sqrt(St * ms);
  double vn_s = dot(vrel, n);
  V3 vn = scl(vn_s, n);
  V3 vt = sub(vrel, vn);
  double kn = (4.0 / 3.0) * mat.Es * std::sqrt(Rs);
  V3 Fn = sub(scl(-kn * delta * std::sqrt(delta), n), scl(cn, vn));
  /* rotate the old spring onto the tangent plane, keep its length */
  double old_len = norm(xi_old);
  V3 xi = sub(xi_old, scl(dot(xi_old, n), n));
  double new_len = norm(xi);
  if (new_len > 0.0) xi = scl(old_len / new_len, xi);
  xi = add(xi, scl(p.dt, vt));
  V3 Ft = sub(scl(-St, xi), scl(ct, vt));
  double ft = norm(Ft), fn = norm(Fn);
  if (ft > p.friction * fn) {
    Ft = scl(p.friction * fn / ft, Ft);
    xi = scl(-1.0 / St, add(Ft, scl(ct, vt)));
  }
  *F = add(Fn, Ft);
  *Ft_out = Ft;
  *xi_new = xi;
}

}  // namespace

ContactOut hm_pair(const orc_params& p, V3 dx, double ra, double rb, double ma, double mb,
                   V3 va, V3 vb, V3 wa, V3 wb, V3 xi_old) {
  ContactOut out{};
  double dist = norm(dx);
  double delta = ra + rb - dist;
  if (!(delta > 0.0)) {
    out.active = false;
    return out;
  }
  out.active = true;
  V3 n = scl(1.0 / dist, dx);
  double Rs = ra * rb / (ra + rb);
  double ms = ma * mb / (ma + mb);
  double la = ra - 0.5 * delta, lb = rb - 0.5 * delta;
  /* contact-point velocity of a relative to b */
  V3 vrel = add(sub(va, vb), cross(add(scl(la, wa), scl(lb, wb)), n));
  V3 Ft;
  hm_core(p, n, delta, Rs, ms, vrel, xi_old, &out.F, &Ft, &out.xi);
  out.Ta = cross(scl(la, n), Ft);
  out.Tb = cross(scl(lb, n), Ft);
  return out;
}

ContactOut hm_wall(const orc_params& p, V3 n, double dist, double r, double m, V3 v, V3 w,
                   V3 xi_old) {
  ContactOut out{};
  double delta = r - dist;
  if (!(delta > 0.0)) {
    out.active = false;
    return out;
  }
  out.active = true;
  double l = r - 0.5 * delta;
  V3 vrel = add(v, cross(scl(l, w), n));
  V3 Ft;
  hm_core(p, n, delta, r, m, vrel, xi_old, &out.F, &Ft, &out.xi);
  out.Ta = cross(scl(l, n), Ft);
  out.Tb = V3{0, 0, 0};
  return out;
}

V3 lub_pair(const orc_params& p, V3 dx, double ra, double rb, V3 va, V3 vb) {
  double dist = norm(dx);
  double dbar = ra + rb; /* pair-mean diameter */
  double h = dist - ra - rb;
  double h_out = p.lub_h_out_frac * dbar;
  if (!(h < h_out)) return V3{0, 0, 0};
  double h_in = p.lub_h_in_frac * dbar;
  double mu = p.rho_f * p.nu_f;
  double Rl = ra * rb / (ra + rb);
  V3 n = scl(1.0 / dist, dx);
  double vn = dot(sub(va, vb), n);
  double hh = h > h_in ? h : h_in;
  return scl(-6.0 * M_PI * mu * Rl * Rl * vn / hh, n);
}

V3 lub_wall(const orc_params& p, V3 n, double dist, double r, V3 v) {
  double dbar = 2.0 * r;
  double h = dist - r;
  double h_out = p.lub_h_out_frac * dbar;
  if (!(h < h_out)) return V3{0, 0, 0};
  double h_in = p.lub_h_in_frac * dbar;
  double mu = p.rho_f * p.nu_f;
  double vn = dot(v, n);
  double hh = h > h_in ? h : h_in;
  return scl(-6.0 * M_PI * mu * r * r * vn / hh, n);
}

}  // namespace orc
