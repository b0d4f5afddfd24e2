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
 * i as body "a"; j receives the opposite force.  With orc_set_threads(n > 1) the
 * particle loops run on n threads and give the same bits (see pair_forces).
 */
#include <algorithm>
#include <cstring>

#include "orc_internal.h"

using orc::V3;

namespace {

struct Forces {
  std::vector<V3> fc, fl, ff, tq;
};

/* Pair forces.  Serial: pairs in increasing (i, j), each evaluated once with i as
   body "a"; i receives +F, j receives -F.  Parallel (threads > 1): every particle
   walks its own partners in increasing index and evaluates each of its pairs with
   the lower index as body "a", adding +F (it is "a") or -F (it is "b") -- the same
   evaluations, added to each particle in the same order as the serial loop, so the
   two give identical bits; each pair is evaluated from both sides. */
void pair_forces(orc_handle* h, const std::vector<double>& r, const std::vector<double>& m,
                 Forces& out, std::vector<orc::HistEntry>* new_hist) {
  const orc_params& p = h->p;
  int64_t n = h->n;
  std::vector<std::pair<int64_t, int64_t>> pairs;
  double frac = p.lubrication ? p.lub_h_out_frac : 0.0;
  orc::find_pairs(p, h->x, r, frac, 0.0, n <= 4096, pairs, h->threads);
  const orc::HistIndex hix = orc::hist_index(h->hist, n);
  if (h->threads <= 1) {
    for (auto& pr : pairs) {
      int64_t i = pr.first, j = pr.second;
      V3 dx = orc::min_image(p, h->x[i], h->x[j]);
      const V3* old = orc::hist_find(hix, i, j);
      V3 xi_old = old ? *old : V3{0, 0, 0};
      orc::ContactOut c =
          orc::hm_pair(p, dx, r[i], r[j], m[i], m[j], h->v[i], h->v[j], h->w[i], h->w[j], xi_old);
      if (c.active) {
        out.fc[i] = orc::add(out.fc[i], c.F);
        out.fc[j] = orc::sub(out.fc[j], c.F);
        out.tq[i] = orc::add(out.tq[i], c.Ta);
        out.tq[j] = orc::add(out.tq[j], c.Tb);
        if (new_hist) new_hist->push_back(orc::HistEntry{i, j, c.xi});
      }
      if (p.lubrication) {
        orc::LubOut l = orc::lub_pair(p, dx, r[i], r[j], h->v[i], h->v[j], h->w[i], h->w[j]);
        out.fl[i] = orc::add(out.fl[i], l.F);
        out.fl[j] = orc::sub(out.fl[j], l.F);
        out.tq[i] = orc::add(out.tq[i], l.Ta);
        out.tq[j] = orc::add(out.tq[j], l.Tb);
      }
    }
    return;
  }
  /* full partner lists, sorted: partners below k come from pairs (j, k), above from
     (k, j); pid is the pair's index in `pairs` */
  const int64_t np = (int64_t)pairs.size();
  std::vector<int64_t> off(n + 1, 0), nb(2 * np), pid(2 * np);
  for (auto& pr : pairs) {
    ++off[pr.first + 1];
    ++off[pr.second + 1];
  }
  for (int64_t i = 0; i < n; ++i) off[i + 1] += off[i];
  {
    std::vector<int64_t> fill(off.begin(), off.end() - 1);
    for (int64_t e = 0; e < np; ++e) {  /* increasing first index */
      pid[fill[pairs[e].second]] = e;
      nb[fill[pairs[e].second]++] = pairs[e].first;
    }
    for (int64_t e = 0; e < np; ++e) {  /* then increasing second index */
      pid[fill[pairs[e].first]] = e;
      nb[fill[pairs[e].first]++] = pairs[e].second;
    }
  }
  /* the spring of pair e, written by its first particle; kept in pair order below */
  std::vector<orc::HistEntry> slot(new_hist ? np : 0);
  std::vector<char> live(new_hist ? np : 0, 0);
#pragma omp parallel for schedule(dynamic, 1024) num_threads(h->threads)
  for (int64_t k = 0; k < n; ++k) {
    for (int64_t e = off[k]; e < off[k + 1]; ++e) {
      const int64_t q = nb[e];
      const int64_t i = k < q ? k : q, j = k < q ? q : k;
      const bool is_a = i == k;
      V3 dx = orc::min_image(p, h->x[i], h->x[j]);
      const V3* old = orc::hist_find(hix, i, j);
      V3 xi_old = old ? *old : V3{0, 0, 0};
      orc::ContactOut c =
          orc::hm_pair(p, dx, r[i], r[j], m[i], m[j], h->v[i], h->v[j], h->w[i], h->w[j], xi_old);
      if (c.active) {
        out.fc[k] = is_a ? orc::add(out.fc[k], c.F) : orc::sub(out.fc[k], c.F);
        out.tq[k] = orc::add(out.tq[k], is_a ? c.Ta : c.Tb);
        if (new_hist && is_a) {
          slot[pid[e]] = orc::HistEntry{i, j, c.xi};
          live[pid[e]] = 1;
        }
      }
      if (p.lubrication) {
        orc::LubOut l = orc::lub_pair(p, dx, r[i], r[j], h->v[i], h->v[j], h->w[i], h->w[j]);
        out.fl[k] = is_a ? orc::add(out.fl[k], l.F) : orc::sub(out.fl[k], l.F);
        out.tq[k] = orc::add(out.tq[k], is_a ? l.Ta : l.Tb);
      }
    }
  }
  if (new_hist)
    for (int64_t e = 0; e < np; ++e)
      if (live[e]) new_hist->push_back(slot[e]);
}

void evaluate(orc_handle* h, Forces& out, std::vector<orc::HistEntry>* new_hist,
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
  pair_forces(h, r, m, out, new_hist);
  if (new_whist) new_whist->assign(n * 6, V3{0, 0, 0});
  orc::FluidFields ff{&h->U, &h->gradp, &h->DUDt, &h->eps, &h->curlU};
  /* walls and fluid: each particle on its own */
#pragma omp parallel for schedule(static) num_threads(h->threads > 1 ? h->threads : 1)
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
    std::vector<orc::HistEntry> new_hist;
    std::vector<V3> new_whist;
    evaluate(h, F, &new_hist, &new_whist);
#pragma omp parallel for schedule(static) num_threads(h->threads > 1 ? h->threads : 1)
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
  for (auto& e : h->hist) {
    if (k >= cap) return -1;
    ij[2 * k] = e.i;
    ij[2 * k + 1] = e.j;
    orc::store(xi, k, e.xi);
    ++k;
  }
  return 0;
}

int orc_set_contacts(orc_handle* h, int64_t m, const int64_t* ij, const double* xi) {
  std::vector<orc::HistEntry> e(m);
  for (int64_t k = 0; k < m; ++k) {
    if (ij[2 * k] < 0 || ij[2 * k] >= ij[2 * k + 1] || ij[2 * k + 1] >= h->n) return -1;
    e[k] = orc::HistEntry{ij[2 * k], ij[2 * k + 1], orc::load(xi, k)};
  }
  std::sort(e.begin(), e.end(), [](const orc::HistEntry& a, const orc::HistEntry& b) {
    return a.i < b.i || (a.i == b.i && a.j < b.j);
  });
  h->hist.swap(e);
  return 0;
}

int orc_set_wall_history(orc_handle* h, const double* xw) {
  for (int64_t i = 0; i < h->n * 6; ++i) h->whist[i] = orc::load(xw, i);
  return 0;
}

int orc_set_threads(orc_handle* h, int32_t threads) {
  h->threads = threads < 1 ? 1 : threads;
  return 0;
}

int orc_get_wall_history(orc_handle* h, double* xw) {
  for (int64_t i = 0; i < h->n * 6; ++i) orc::store(xw, i, h->whist[i]);
  return 0;
}

}  // extern "C"
