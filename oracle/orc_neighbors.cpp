/*
 * Oracle (test infrastructure only): neighbour search, Sec. 2.5 (LAMMPS's
 * neighbour lists with link-cell binning, Hockney & Eastwood).
 *
 * The paper gives no predicate; the reading used here:
 *   pair (i, j) is listed iff  d2 < rc^2  with
 *     d2 = (dx*dx + dy*dy) + dz*dz                (in this order, no fused multiply-add)
 *     rc = ((r_i + r_j) + h_out_frac * (r_i + r_j)) + skin
 *   and dx the minimum-image difference.  Strict "<".
 * Two methods produce the same set: brute force over all pairs, and link-cell
 * bins of edge >= the largest rc (27 bins around each particle).
 */
#include <algorithm>
#include <cstdio>

#include "orc_internal.h"

namespace orc {

namespace {

bool listed(const orc_params& p, V3 xi, V3 xj, double ri, double rj, double frac, double skin) {
  V3 dx = min_image(p, xi, xj);
  double d2 = dx.x * dx.x;
  d2 = d2 + dx.y * dx.y;
  d2 = d2 + dx.z * dx.z;
  double s = ri + rj;
  double rc = s + frac * s;
  rc = rc + skin;
  return d2 < rc * rc;
}

}  // namespace

void find_pairs(const orc_params& p, const std::vector<V3>& x, const std::vector<double>& r,
                double frac, double skin, bool brute,
                std::vector<std::pair<int64_t, int64_t>>& out) {
  out.clear();
  int64_t n = (int64_t)x.size();
  double rmax = 0.0;
  for (double ri : r) rmax = std::max(rmax, ri);
  double rc_max = (2.0 * rmax) * (1.0 + frac) + skin;
  int nb[3];
  for (int a = 0; a < 3; ++a) {
    double L = p.hi[a] - p.lo[a];
    nb[a] = std::max(1, (int)std::floor(L / (rc_max * (1.0 + 1e-9))));
    if (p.periodic[a] && nb[a] < 3) brute = true;
  }
  if (brute) {
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = i + 1; j < n; ++j)
        if (listed(p, x[i], x[j], r[i], r[j], frac, skin)) out.emplace_back(i, j);
    return;
  }
  auto bin_of = [&](V3 xi, int a) {
    double L = p.hi[a] - p.lo[a];
    int b = (int)std::floor((comp(xi, a) - p.lo[a]) / L * nb[a]);
    if (b < 0) b = 0;
    if (b > nb[a] - 1) b = nb[a] - 1;
    return b;
  };
  int64_t nbins = (int64_t)nb[0] * nb[1] * nb[2];
  std::vector<std::vector<int64_t>> bins(nbins);
  std::vector<int64_t> bi(n);
  for (int64_t i = 0; i < n; ++i) {
    int b0 = bin_of(x[i], 0), b1 = bin_of(x[i], 1), b2 = bin_of(x[i], 2);
    bi[i] = ((int64_t)b2 * nb[1] + b1) * nb[0] + b0;
    bins[bi[i]].push_back(i);
  }
  for (int64_t i = 0; i < n; ++i) {
    int c[3] = {(int)(bi[i] % nb[0]), (int)((bi[i] / nb[0]) % nb[1]),
                (int)(bi[i] / ((int64_t)nb[0] * nb[1]))};
    for (int oz = -1; oz <= 1; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          int o[3] = {ox, oy, oz};
          int t[3];
          bool ok = true;
          for (int a = 0; a < 3; ++a) {
            t[a] = c[a] + o[a];
            if (p.periodic[a]) t[a] = (t[a] + nb[a]) % nb[a];
            else if (t[a] < 0 || t[a] >= nb[a]) ok = false;
          }
          if (!ok) continue;
          int64_t b = ((int64_t)t[2] * nb[1] + t[1]) * nb[0] + t[0];
          for (int64_t j : bins[b])
            if (j > i && listed(p, x[i], x[j], r[i], r[j], frac, skin)) out.emplace_back(i, j);
        }
  }
  std::sort(out.begin(), out.end());
}

}  // namespace orc

extern "C" int64_t orc_neighbors(orc_handle* h, double skin, int32_t brute, int64_t* offsets,
                                 int64_t* idx, int64_t cap) {
  std::vector<double> r(h->n);
  for (int64_t i = 0; i < h->n; ++i) r[i] = 0.5 * h->d[i];
  std::vector<std::pair<int64_t, int64_t>> pairs;
  orc::find_pairs(h->p, h->x, r, h->p.lub_h_out_frac, skin, brute != 0, pairs);
  int64_t total = 2 * (int64_t)pairs.size();
  if (total > cap) return -1;
  std::vector<std::vector<int64_t>> lists(h->n);
  for (auto& pr : pairs) {
    lists[pr.first].push_back(pr.second);
    lists[pr.second].push_back(pr.first);
  }
  int64_t k = 0;
  for (int64_t i = 0; i < h->n; ++i) {
    offsets[i] = k;
    std::sort(lists[i].begin(), lists[i].end());
    for (int64_t j : lists[i]) idx[k++] = j;
  }
  offsets[h->n] = k;
  return total;
}
