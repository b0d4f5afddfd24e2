/*
 * Oracle (test infrastructure only): one DEM substep, Sec. 2.1 Eq. (1a)-(1b).
 *
 *   m du/dt = f_col + f_lub + f_fp + m g,     I dPsi/dt = T_col + T_lub (+ T_fp = 0)
 *
 * T_fp = 0: Sec. 2.5 says the interaction of particle rotation and fluid is not
 * considered.  Time integration (LAMMPS's velocity Verlet, written in its
 * equivalent leapfrog form): forces are evaluated at x^n with the half-step
 * velocity v^(n-1/2); then
 *   a^n = F/m + g,  v^(n+1/2) = v^(n-1/2) + dt a^n,  w likewise with I = 0.4 m r^2,
 *   x^(n+1) = x^n + dt v^(n+1/2), wrapped into [lo, hi) on periodic axes,
 * and a^n becomes the lagged acceleration of the added-mass force.
 * Pairs are visited in increasing (i, j), i < j; each pair is evaluated once with
 * i as body "a"; j receives the opposite force.
 */
#include <cstring>

#include "orc_internal.h"

using orc::V3;

namespace {

struct Forces {
  std::vector<V3> fc, fl, ff, tq;
};

void evaluate(orc_handle* h, Forces& out,
              std::map<std::pair<int64_t, int64_t>, V3>* new_hist,
              std::vector<V3>* new_whist) {
  const orc_params& p = h->p;
  int64_t n = h->n;
  std::vector<double> r(n), m(n);
  for (int64_t i = 0; i < n; ++i) {
    r[i] = 0.5 * h->d[i];
    m[i] = h->rho[i] * (M_PI / 6.0 * h->d[i] * h->d[i] * h->d[i]);
  }
  out.fc.assign(n, V3{0, 0, 0});
  out.fl.assign(n, V3{0, 0, 0});
  out.ff.assign(n, V3{0, 0, 0});
  out.tq.assign(n, V3{0, 0, 0});
  std::vector<std::pair<int64_t, int64_t>> pairs;
  double frac = p.lubrication ? p.lub_h_out_frac : 0.0;
  orc::find_pairs(p, h->x, r, frac, 0.0, n <= 4096, pairs);
  for (auto& pr : pairs) {
    int64_t i = pr.first, j = pr.second;
    V3 dx = orc::min_image(p, h->x[i], h->x[j]);
    V3 xi_old{0, 0, 0};
    auto it = h->hist.find(pr);
    if (it != h->hist.end()) xi_old = it->second;
    orc::ContactOut c =
        orc::hm_pair(p, dx, r[i], r[j], m[i], m[j], h->v[i], h->v[j], h->w[i], h->w[j], xi_old);
    if (c.active) {
      out.fc[i] = orc::add(out.fc[i], c.F);
      out.fc[j] = orc::sub(out.fc[j], c.F);
      out.tq[i] = orc::add(out.tq[i], c.Ta);
      out.tq[j] = orc::add(out.tq[j], c.Tb);
      if (new_hist) (*new_hist)[pr] = c.xi;
    }
    if (p.lubrication) {
      orc::LubOut l = orc::lub_pair(p, dx, r[i], r[j], h->v[i], h->v[j], h->w[i], h->w[j]);
      out.fl[i] = orc::add(out.fl[i], l.F);
      out.fl[j] = orc::sub(out.fl[j], l.F);
      out.tq[i] = orc::add(out.tq[i], l.Ta);
      out.tq[j] = orc::add(out.tq[j], l.Tb);
    }
  }
  if (new_whist) new_whist->assign(n * 6, V3{0, 0, 0});
  orc::FluidFields ff{&h->U, &h->gradp, &h->DUDt, &h->eps, &h->curlU};
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) {
      if (p.periodic[a]) continue;
      for (int side = 0; side < 2; ++side) {
        if (side == 0 && !p.wall_lo[a]) continue;
        if (side == 1 && !p.wall_hi[a]) continue;
        V3 nrm{0, 0, 0};
        orc::set_comp(nrm, a, side == 0 ? -1.0 : 1.0);
        double xa = orc::comp(h->x[i], a);
        double dist = side == 0 ? xa - p.lo[a] : p.hi[a] - xa;
        int slot = 2 * a + side;
        orc::ContactOut c =
            orc::hm_wall(p, nrm, dist, r[i], m[i], h->v[i], h->w[i], h->whist[i * 6 + slot]);
        if (c.active) {
          out.fc[i] = orc::add(out.fc[i], c.F);
          out.tq[i] = orc::add(out.tq[i], c.Ta);
          if (new_whist) (*new_whist)[i * 6 + slot] = c.xi;
        }
        if (p.lubrication) {
          orc::LubOut l = orc::lub_wall(p, nrm, dist, r[i], h->v[i], h->w[i]);
          out.fl[i] = orc::add(out.fl[i], l.F);
          out.tq[i] = orc::add(out.tq[i], l.Ta);
        }
      }
    }
    out.ff[i] = orc::fluid_force(p, ff, h->x[i], h->v[i], h->a_prev[i], h->d[i]);
  }
}

}  // namespace

extern "C" {

orc_handle* orc_create(const orc_params* p) {
  orc_handle* h = new orc_handle();
  h->p = *p;
  int64_t C = h->ncells();
  h->U.assign(C * 3, 0.0);
  h->gradp.assign(C * 3, 0.0);
  for (int64_t c = 0; c < C; ++c)
    for (int a = 0; a < 3; ++a) h->gradp[3 * c + a] = p->rho_f * p->g[a];
  h->DUDt.assign(C * 3, 0.0);
  h->eps.assign(C, 0.0);
  h->curlU.assign(C * 3, 0.0);
  return h;
}

void orc_destroy(orc_handle* h) { delete h; }

int orc_set_particles(orc_handle* h, int64_t n, const double* x, const double* v,
                      const double* w, const double* d, const double* rho) {
  h->n = n;
  h->x.resize(n);
  h->v.resize(n);
  h->w.resize(n);
  h->a_prev.assign(n, V3{0, 0, 0});
  h->d.assign(d, d + n);
  h->rho.assign(rho, rho + n);
  for (int64_t i = 0; i < n; ++i) {
    h->x[i] = orc::load(x, i);
    h->v[i] = v ? orc::load(v, i) : V3{0, 0, 0};
    h->w[i] = w ? orc::load(w, i) : V3{0, 0, 0};
  }
  h->hist.clear();
  h->whist.assign(n * 6, V3{0, 0, 0});
  return 0;
}

int orc_set_accel(orc_handle* h, const double* a) {
  for (int64_t i = 0; i < h->n; ++i) h->a_prev[i] = orc::load(a, i);
  return 0;
}

int orc_set_fluid(orc_handle* h, const double* U, const double* gp, const double* Du) {
  int64_t C = h->ncells();
  if (U) {
    h->U.assign(U, U + 3 * C);
    orc::curl_cells(h->p, h->U, h->curlU);
  }
  if (gp) h->gradp.assign(gp, gp + 3 * C);
  if (Du) h->DUDt.assign(Du, Du + 3 * C);
  return 0;
}

int orc_set_eps(orc_handle* h, const double* eps) {
  h->eps.assign(eps, eps + h->ncells());
  return 0;
}

int orc_forces(orc_handle* h, double* fc, double* fl, double* ff, double* tq) {
  Forces F;
  evaluate(h, F, nullptr, nullptr);
  for (int64_t i = 0; i < h->n; ++i) {
    if (fc) orc::store(fc, i, F.fc[i]);
    if (fl) orc::store(fl, i, F.fl[i]);
    if (ff) orc::store(ff, i, F.ff[i]);
    if (tq) orc::store(tq, i, F.tq[i]);
  }
  return 0;
}

int orc_step(orc_handle* h, int32_t n_sub) {
  const orc_params& p = h->p;
  for (int32_t s = 0; s < n_sub; ++s) {
    Forces F;
    std::map<std::pair<int64_t, int64_t>, V3> new_hist;
    std::vector<V3> new_whist;
    evaluate(h, F, &new_hist, &new_whist);
    for (int64_t i = 0; i < h->n; ++i) {
      double d = h->d[i], r = 0.5 * d;
      double m = h->rho[i] * (M_PI / 6.0 * d * d * d);
      double I = 0.4 * m * r * r;
      V3 ftot = orc::add(orc::add(F.fc[i], F.fl[i]), F.ff[i]);
      V3 a = orc::add(orc::scl(1.0 / m, ftot), V3{p.g[0], p.g[1], p.g[2]});
      h->v[i] = orc::add(h->v[i], orc::scl(p.dt, a));
      h->w[i] = orc::add(h->w[i], orc::scl(p.dt / I, F.tq[i]));
      V3 xn = orc::add(h->x[i], orc::scl(p.dt, h->v[i]));
      for (int ax = 0; ax < 3; ++ax) {
        if (!p.periodic[ax]) continue;
        double L = p.hi[ax] - p.lo[ax];
        double c = orc::comp(xn, ax);
        if (c < p.lo[ax]) c = c + L;
        else if (c >= p.hi[ax]) c = c - L;
        orc::set_comp(xn, ax, c);
      }
      h->x[i] = xn;
      h->a_prev[i] = a;
    }
    h->hist.swap(new_hist);
    h->whist.swap(new_whist);
  }
  return 0;
}

int orc_get_particles(orc_handle* h, double* x, double* v, double* w, double* a) {
  for (int64_t i = 0; i < h->n; ++i) {
    if (x) orc::store(x, i, h->x[i]);
    if (v) orc::store(v, i, h->v[i]);
    if (w) orc::store(w, i, h->w[i]);
    if (a) orc::store(a, i, h->a_prev[i]);
  }
  return 0;
}

int64_t orc_num_contacts(orc_handle* h) { return (int64_t)h->hist.size(); }

int orc_get_contacts(orc_handle* h, int64_t cap, int64_t* ij, double* xi) {
  int64_t k = 0;
  for (auto& kv : h->hist) {
    if (k >= cap) return -1;
    ij[2 * k] = kv.first.first;
    ij[2 * k + 1] = kv.first.second;
    orc::store(xi, k, kv.second);
    ++k;
  }
  return 0;
}

int orc_get_wall_history(orc_handle* h, double* xw) {
  for (int64_t i = 0; i < h->n * 6; ++i) orc::store(xw, i, h->whist[i]);
  return 0;
}

}  // extern "C"
