/* Internal declarations of the FP64 oracle (test infrastructure only). */
#pragma once
#include "orc.h"
#include <cmath>
#include <map>
#include <utility>
#include <vector>

namespace orc {

struct V3 {
  double x, y, z;
};
inline V3 v3(double x, double y, double z) { return V3{x, y, z}; }
inline V3 add(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 sub(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 scl(double s, V3 a) { return V3{s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 cross(V3 a, V3 b) {
  return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline V3 load(const double* p, int64_t i) { return V3{p[3 * i], p[3 * i + 1], p[3 * i + 2]}; }
inline void store(double* p, int64_t i, V3 a) {
  p[3 * i] = a.x;
  p[3 * i + 1] = a.y;
  p[3 * i + 2] = a.z;
}
inline double comp(V3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }
inline void set_comp(V3& a, int k, double s) {
  if (k == 0) a.x = s; else if (k == 1) a.y = s; else a.z = s;
}

/* Minimum-image difference x_j - x_i on periodic axes (positions are kept in
   [lo, hi), so one shift of the box length is enough). */
V3 min_image(const orc_params& p, V3 xi, V3 xj);

/* Result of one contact evaluation for the body "a" of a pair (a, b). */
struct ContactOut {
  V3 F;       /* normal + tangential contact force on a */
  V3 Ta, Tb;  /* contact torques on a and on b */
  V3 xi;      /* updated tangential spring */
  bool active;
};

/* Hertz-Mindlin pair: dx = x_b - x_a (minimum image). */
ContactOut hm_pair(const orc_params& p, V3 dx, double ra, double rb, double ma, double mb,
                   V3 va, V3 vb, V3 wa, V3 wb, V3 xi_old);
/* Hertz-Mindlin sphere-plane: n is the unit normal from the centre towards the
   wall, dist the centre-to-plane distance. */
ContactOut hm_wall(const orc_params& p, V3 n, double dist, double r, double m, V3 v, V3 w,
                   V3 xi_old);
/* Ball-Melrose lubrication on a for the pair (a, b): force on a, torques on a
   and on b (b receives -F). */
struct LubOut {
  V3 F, Ta, Tb;
};
LubOut lub_pair(const orc_params& p, V3 dx, double ra, double rb, V3 va, V3 vb, V3 wa, V3 wb);
LubOut lub_wall(const orc_params& p, V3 n, double dist, double r, V3 v, V3 w);

/* Fluid-particle force at one particle (Sec. 2.3). */
struct FluidFields {
  const std::vector<double>* U;     /* C*3 */
  const std::vector<double>* gradp; /* C*3 */
  const std::vector<double>* DUDt;  /* C*3 */
  const std::vector<double>* eps;   /* C */
  const std::vector<double>* curlU; /* C*3, vorticity of U */
};
/* The z mesh.  Uniform unless z_grading != 1: then cell heights grow geometrically
   from the floor, h_k = h_0 r^k, r = z_grading^(1/(n_z - 1)) (z_grading is the ratio
   of the top cell's height to the bottom cell's), faces
   z_k = lo + L (r^k - 1) / (r^n - 1), written with expm1 so a ratio near 1 keeps
   its accuracy. */
struct ZGrid {
  bool graded;
  std::vector<double> zf, zc, hz; /* faces (n + 1), centres, heights (n) */
};
ZGrid zgrid(const orc_params& p);

/* Vorticity of a cell-centred velocity field (C*3 in, C*3 out). */
void curl_cells(const orc_params& p, const std::vector<double>& U, std::vector<double>& out);
V3 lift_force(const orc_params& p, V3 w, V3 omega, double d);
double interp_scalar(const orc_params& p, const std::vector<double>& f, int ncomp, int comp,
                     V3 x);
V3 fluid_force(const orc_params& p, const FluidFields& ff, V3 x, V3 u, V3 a_prev, double d);
V3 drag_force(const orc_params& p, double eps_s, V3 w, double d, double* Vr_out,
              double* Cdw_out);

/* Pairs (i < j) with |x_j - x_i| < r_i + r_j + extra(i, j), sorted by (i, j).  With
   threads > 1 the link-cell search runs over particles in parallel (same result). */
void find_pairs(const orc_params& p, const std::vector<V3>& x, const std::vector<double>& r,
                double h_out_frac, double skin, bool brute,
                std::vector<std::pair<int64_t, int64_t>>& out, int threads = 1);

/* Tangential spring of one pair in contact, i < j. */
struct HistEntry {
  int64_t i, j;
  V3 xi;
};
/* Springs sorted by (i, j) with the index of each particle's first entry:
   entries of particle i are [first[i], first[i + 1]). */
struct HistIndex {
  const std::vector<HistEntry>* h;
  std::vector<int64_t> first;
};
HistIndex hist_index(const std::vector<HistEntry>& h, int64_t n);
/* Spring of the pair (i, j), i < j; null if the pair has none. */
const V3* hist_find(const HistIndex& ix, int64_t i, int64_t j);

}  // namespace orc

struct orc_handle {
  orc_params p;
  int64_t n = 0;
  std::vector<orc::V3> x, v, w, a_prev;
  std::vector<double> d, rho;
  /* tangential spring of each pair in contact, i < j, sorted by (i, j) */
  std::vector<orc::HistEntry> hist;
  /* threads of the particle loops (orc_set_threads); 1 = the serial pair loop */
  int threads = 1;
  /* tangential spring of each particle against each of the six walls */
  std::vector<orc::V3> whist; /* n*6 */
  std::vector<double> U, gradp, DUDt, eps;
  std::vector<double> curlU; /* C*3, curl of U (lift force) */
  int64_t ncells() const { return (int64_t)p.ncell[0] * p.ncell[1] * p.ncell[2]; }
};
