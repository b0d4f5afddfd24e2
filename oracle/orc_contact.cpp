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
 * Linear spring-dashpot (contact_law 1).  Sec. 2.5 states that the collision force
 * is a linear spring-dashpot (normal force proportional to the overlap) and Table 1
 * gives the stiffness (800 N/m), the normal restitution coefficient and the
 * friction coefficient.  Reading: S_n = k_n, S_t = kt_ratio k_n (2/7 by default),
 *   F_n = -k_n delta n - c_n v_n,  c_n = -2 beta sqrt(k_n m*),  c_t = -2 beta sqrt(S_t m*),
 * with the same spring history and Coulomb cap as above.  The normal motion is
 * then a damped linear oscillator with damping ratio zeta = -beta, which leaves
 * contact after half a damped period t_c = pi / (omega_0 sqrt(1 - zeta^2)),
 * omega_0 = sqrt(k_n / m*), with exactly the restitution coefficient e.
 *
 * Lubrication.  Sec. 2.5: Ball & Melrose (1997), force proportional to the
 * relative velocity and inversely proportional to the gap.  Reading: the normal
 * squeeze term  F_a = -6 pi mu R_l^2 ((v_a - v_b).n) n / max(h, h_in),
 * R_l = r_a r_b / (r_a + r_b) (R_l = r for a wall), acting while the gap
 * h < h_out; h_in, h_out are fractions of the pair-mean diameter (the particle
 * diameter for a wall).  It also acts during overlap (with h_in).
 * Tangential terms (lub_tangential = 1; Sec. 2.5 integrates a lubrication torque,
 * which the normal term alone does not give).  Reading: the leading shear term of
 * the two-sphere lubrication resistance (Jeffrey & Onishi 1984, the source of Ball
 * & Melrose's pair functions), whose leading squeeze term is the normal force above:
 *   F_a = -6 pi mu R_l (4/15) (2 + beta + 2 beta^2) / (1 + beta)^2 ln(1/xi) v_t,
 *   beta = r_b / r_a,  xi = 2 max(h, h_in) / (r_a + r_b),
 * where v_t is the tangential part of the velocity of a's surface relative to b's
 * at the gap midpoint, v_rel = v_a - v_b + (l_a w_a + l_b w_b) x n with lever
 * arms l = r + h/2 (r - delta/2 in overlap, as for contact); torques l n x F on
 * both spheres.  The factor is symmetric in (a, b), reduces to (1/6) ln(a/h) for
 * equal spheres and, as r_b -> infinity with r_a + r_b -> 2 r_a, to the sphere-wall
 * result (8/15) ln(r/h) (Goldman, Cox & Brenner 1967), which is the wall term.  The
 * logarithm is taken as 0 where it would be negative.
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
  double Sn, St, cn, ct, fel;  /* stiffnesses, damping coefficients, elastic normal force */
  if (p.contact_law == 1) {
    Sn = p.kn_linear;
    St = p.kt_ratio * p.kn_linear;
    cn = -2.0 * mat.beta * std::sqrt(Sn * ms);
    ct = -2.0 * mat.beta * std::sqrt(St * ms);
    fel = p.kn_linear * delta;
  } else {
    double sq = std::sqrt(Rs * delta);
    Sn = 2.0 * mat.Es * sq;
    St = 8.0 * mat.Gs * sq;
    cn = -2.0 * std::sqrt(5.0 / 6.0) * mat.beta * std::sqrt(Sn * ms);
    ct = -2.0 * std::sqrt(5.0 / 6.0) * mat.beta * std::sqrt(St * ms);
    double kn = (4.0 / 3.0) * mat.Es * std::sqrt(Rs);
    fel = kn * delta * std::sqrt(delta);
  }
  double vn_s = dot(vrel, n);
  V3 vn = scl(vn_s, n);
  V3 vt = sub(vrel, vn);
  V3 Fn = sub(scl(-fel, n), scl(cn, vn));
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

LubOut lub_pair(const orc_params& p, V3 dx, double ra, double rb, V3 va, V3 vb, V3 wa, V3 wb) {
  LubOut out{V3{0, 0, 0}, V3{0, 0, 0}, V3{0, 0, 0}};
  double dist = norm(dx);
  double dbar = ra + rb; /* pair-mean diameter */
  double h = dist - ra - rb;
  double h_out = p.lub_h_out_frac * dbar;
  if (!(h < h_out)) return out;
  double h_in = p.lub_h_in_frac * dbar;
  double mu = p.rho_f * p.nu_f;
  double Rl = ra * rb / (ra + rb);
  V3 n = scl(1.0 / dist, dx);
  double vn = dot(sub(va, vb), n);
  double hh = h > h_in ? h : h_in;
  out.F = scl(-6.0 * M_PI * mu * Rl * Rl * vn / hh, n);
  if (p.lub_tangential) {
    double la = ra + 0.5 * h, lb = rb + 0.5 * h;
    V3 vrel = add(sub(va, vb), cross(add(scl(la, wa), scl(lb, wb)), n));
    V3 vt = sub(vrel, scl(dot(vrel, n), n));
    double beta = rb / ra;
    double shape = (2.0 + beta + 2.0 * beta * beta) / ((1.0 + beta) * (1.0 + beta));
    double lg = std::log(dbar / (2.0 * hh));
    if (lg < 0.0) lg = 0.0;
    V3 Fs = scl(-6.0 * M_PI * mu * Rl * (4.0 / 15.0) * shape * lg, vt);
    out.F = add(out.F, Fs);
    out.Ta = cross(scl(la, n), Fs);
    out.Tb = cross(scl(lb, n), Fs);
  }
  return out;
}

LubOut lub_wall(const orc_params& p, V3 n, double dist, double r, V3 v, V3 w) {
  LubOut out{V3{0, 0, 0}, V3{0, 0, 0}, V3{0, 0, 0}};
  double dbar = 2.0 * r;
  double h = dist - r;
  double h_out = p.lub_h_out_frac * dbar;
  if (!(h < h_out)) return out;
  double h_in = p.lub_h_in_frac * dbar;
  double mu = p.rho_f * p.nu_f;
  double vn = dot(v, n);
  double hh = h > h_in ? h : h_in;
  out.F = scl(-6.0 * M_PI * mu * r * r * vn / hh, n);
  if (p.lub_tangential) {
    double l = r + 0.5 * h;
    V3 vrel = add(v, cross(scl(l, w), n));
    V3 vt = sub(vrel, scl(dot(vrel, n), n));
    double lg = std::log(r / hh);
    if (lg < 0.0) lg = 0.0;
    V3 Fs = scl(-6.0 * M_PI * mu * r * (8.0 / 15.0) * lg, vt);
    out.F = add(out.F, Fs);
    out.Ta = cross(scl(l, n), Fs);
  }
  return out;
}

}  // namespace orc

extern "C" {

void orc_lub_pair(const orc_params* p, const double dx[3], double ra, double rb,
                  const double va[3], const double vb[3], const double wa[3],
                  const double wb[3], double F[3], double Ta[3], double Tb[3]) {
  orc::LubOut o = orc::lub_pair(*p, orc::load(dx, 0), ra, rb, orc::load(va, 0), orc::load(vb, 0),
                                orc::load(wa, 0), orc::load(wb, 0));
  orc::store(F, 0, o.F);
  orc::store(Ta, 0, o.Ta);
  orc::store(Tb, 0, o.Tb);
}

int orc_hm_pair(const orc_params* p, const double dx[3], double ra, double rb, double ma,
                double mb, const double va[3], const double vb[3], const double wa[3],
                const double wb[3], const double xi_old[3], double F[3], double Ta[3],
                double Tb[3], double xi_new[3]) {
  orc::ContactOut o = orc::hm_pair(*p, orc::load(dx, 0), ra, rb, ma, mb, orc::load(va, 0),
                                   orc::load(vb, 0), orc::load(wa, 0), orc::load(wb, 0),
                                   orc::load(xi_old, 0));
  if (!o.active) return 0;
  orc::store(F, 0, o.F);
  orc::store(Ta, 0, o.Ta);
  orc::store(Tb, 0, o.Tb);
  orc::store(xi_new, 0, o.xi);
  return 1;
}

void orc_lub_wall(const orc_params* p, const double n[3], double dist, double r,
                  const double v[3], const double w[3], double F[3], double T[3]) {
  orc::LubOut o = orc::lub_wall(*p, orc::load(n, 0), dist, r, orc::load(v, 0), orc::load(w, 0));
  orc::store(F, 0, o.F);
  orc::store(T, 0, o.Ta);
}

}  // extern "C"
