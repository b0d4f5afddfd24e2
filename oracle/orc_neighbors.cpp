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

HistIndex hist_index(const std::vector<HistEntry>& h, int64_t n) {
  HistIndex ix{&h, std::vector<int64_t>(n + 1, 0)};
  for (const HistEntry& e : h) ++ix.first[e.i + 1];
  for (int64_t i = 0; i < n; ++i) ix.first[i + 1] += ix.first[i];
  return ix;
}

const V3* hist_find(const HistIndex& ix, int64_t i, int64_t j) {
  for (int64_t k = ix.first[i]; k < ix.first[i + 1]; ++k)
    if ((*ix.h)[k].j == j) return &(*ix.h)[k].xi;
  return nullptr;
}

void find_pairs(const orc_params& p, const std::vector<V3>& x, const std::vector<double>& r,
                double frac, double skin, bool brute,
                std::vector<std::pair<int64_t, int64_t>>& out, int threads) {
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
  /* particles of each bin, in increasing index (counting sort) */
  int64_t nbins = (int64_t)nb[0] * nb[1] * nb[2];
  std::vector<int64_t> bi(n), bstart(nbins + 1, 0), bitems(n);
  for (int64_t i = 0; i < n; ++i) {
    int b0 = bin_of(x[i], 0), b1 = bin_of(x[i], 1), b2 = bin_of(x[i], 2);
    bi[i] = ((int64_t)b2 * nb[1] + b1) * nb[0] + b0;
    ++bstart[bi[i] + 1];
  }
  for (int64_t b = 0; b < nbins; ++b) bstart[b + 1] += bstart[b];
  {
    std::vector<int64_t> fill(bstart.begin(), bstart.end() - 1);
    for (int64_t i = 0; i < n; ++i) bitems[fill[bi[i]]++] = i;
  }
  /* the partners j > i of particle i, sorted, appended in increasing i: the pairs come
     out sorted by (i, j).  Threads take contiguous ranges of i and their outputs are
     joined in order. */
  if (threads < 1) threads = 1;
  std::vector<std::vector<std::pair<int64_t, int64_t>>> part(threads);
#pragma omp parallel for schedule(static) num_threads(threads)
  for (int t = 0; t < threads; ++t) {
    const int64_t i0 = n * t / threads, i1 = n * (t + 1) / threads;
    std::vector<int64_t> js;
    for (int64_t i = i0; i < i1; ++i) {
      js.clear();
      int c[3] = {(int)(bi[i] % nb[0]), (int)((bi[i] / nb[0]) % nb[1]),
                  (int)(bi[i] / ((int64_t)nb[0] * nb[1]))};
      for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            int o[3] = {ox, oy, oz};
            int cb[3];
            bool ok = true;
            for (int a = 0; a < 3; ++a) {
              cb[a] = c[a] + o[a];
              if (p.periodic[a]) cb[a] = (cb[a] + nb[a]) % nb[a];
              else if (cb[a] < 0 || cb[a] >= nb[a]) ok = false;
            }
            if (!ok) continue;
            int64_t b = ((int64_t)cb[2] * nb[1] + cb[1]) * nb[0] + cb[0];
            for (int64_t q = bstart[b]; q < bstart[b + 1]; ++q) {
              const int64_t j = bitems[q];
              if (j > i && listed(p, x[i], x[j], r[i], r[j], frac, skin)) js.push_back(j);
            }
          }
      std::sort(js.begin(), js.end());
      for (int64_t j : js) part[t].emplace_back(i, j);
    }
  }
  size_t total = 0;
  for (auto& pt : part) total += pt.size();
  out.reserve(total);
  for (auto& pt : part) out.insert(out.end(), pt.begin(), pt.end());
}

}  // namespace orc

extern "C" int64_t orc_neighbors(orc_handle* h, double skin, int32_t brute, int64_t* offsets,
                                 int64_t* idx, int64_t cap) {
  std::vector<double> r(h->n);
  for (int64_t i = 0; i < h->n; ++i) r[i] = 0.5 * h->d[i];
  std::vector<std::pair<int64_t, int64_t>> pairs;
  orc::find_pairs(h->p, h->x, r, h->p.lub_h_out_frac, skin, brute != 0, pairs, h->threads);
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
