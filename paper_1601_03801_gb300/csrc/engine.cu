// Host engine behind include/sedi.h: parameter checks, device buffers, CUDA-graph
// capture of the substep sequence (rebuild under a graph IF node decided on the
// device), orchestration of the averaging, import/export in caller order and
// checkpoints.  All arithmetic of the method runs in the kernels of k_*.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sedi.h"
#include "common.cuh"
#include "kernels.h"

using namespace sedi;

struct sedi_handle {
  sedi_params prm{};
  std::string err;
  long long barrier_spins = kBarrierSpins;  // grid-barrier polls before SEDI_ETIMEOUT
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;  // capture of conditional bodies
  cudaStream_t own = nullptr;   // default stream of the handle (graphs need a real stream)
  int form = FORM_SPLIT;
  int64_t N = 0;
  bool have_particles = false;
  std::vector<int64_t> ids;
  std::vector<double> d_host, rho_host;
  std::vector<double> U, gp, du, eps;  // host copies of the fluid fields (checkpoint)
  bool gp_default = true;
  DevState st{};
  DevParams P{};
  DevMesh mesh{};
  std::vector<void*> part_allocs;  // per-particle buffers
  std::vector<void*> bin_allocs;   // link-cell bins (resized when the bin size changes)
  std::vector<void*> mesh_allocs;
  double rc_max = 0.0;             // largest list cutoff 2 r_max (1 + f) + skin
  int64_t since_set = 0;               // substeps since the particles were set
  bool is_bed = false;                 // a bed of an ensemble (stepped by the ensemble)
  double* fdev = nullptr;              // FP64 U, grad p, DU/Dt [3][C][3] on the device
  double* edev = nullptr;              // FP64 staging of eps_s [C]
  bool fluid_host_stale = false;       // host copies (U, gp, du, eps) behind the device
  SmoothZ zs{};                        // graded z mesh: smoothing tables (device) and bounds
  void* qfix = nullptr;   // [7][C] int64 (plain: float phi)
  void* phi = nullptr;    // [8][C] smoothing word
  void* work = nullptr;
  size_t work_bytes = 0;
  int* iters_dev = nullptr;
  double* dstage = nullptr;  // [max(7C, 4*3N)] doubles
  size_t dstage_n = 0;
  double coef[3] = {0, 0, 0};
  std::map<int, cudaGraphExec_t> graphs;
  sedi_stats stats{};
  int variant = SUBSTEP_B128;  // substep launch variant in use
  std::string tuned_key;       // workload the variant was tuned for (empty: not tuned)
  std::string key_cache;       // the workload key of the current particles (empty: stale)
  // profiling: events per captured substep (A: before check, B: before the
  // substep kernel, C: after it) and around deposition / smoothing
  struct GraphEv {
    std::vector<cudaEvent_t> a, b, c;
  };
  std::map<int, GraphEv> gev;
  std::vector<cudaEvent_t> avg_ev;  // 3 events: before deposit, after deposit, after smooth
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  double ms[4] = {0, 0, 0, 0};
  double cnt[4] = {0, 0, 0, 0};
  // learned warm start: FP32 master weights, Adam moments, gradient, work space
  float* cnn_master = nullptr;
  float* cnn_m = nullptr;
  float* cnn_v = nullptr;
  float* cnn_grad = nullptr;
  float* cnn_target = nullptr;  // [v][4]
  double* cnn_loss = nullptr;   // device scalars (one per training step)
  void* cnn_work = nullptr;
  int64_t cnn_steps = 0;
  bool cnn_set = false;
  // ensemble (n_beds > 1): one single-bed handle per bed, stepped and averaged by
  // batched launches over all beds (grid.y = bed)
  std::vector<sedi_handle*> beds;
  BedView* ens_views = nullptr;   // device table of the beds' views
  void* ens_smooth = nullptr;     // smoothing batch tables
  int* ens_iters = nullptr;       // [B][8] smoother step counts
  Ctl* ens_ctl = nullptr;         // [B] gathered control blocks
  EnsLaunch ens{};
  bool ens_dirty = true;          // a bed's buffers changed: rebuild the table
  int ens_variant = SUBSTEP_B128_LOOP;  // launch shape of the batched substep
  int* ens_done = nullptr;        // substeps completed by the last persistent launch
  bool ens_fresh = false;         // the batched averaging is newer than the last step
};

namespace {

size_t word_bytes(int form) { return form == FORM_PLAIN ? 4 : 8; }
size_t quad_bytes(int form) { return form == FORM_PLAIN ? 16 : 32; }
size_t fquad_bytes(int form) { return form == FORM_FP64 ? 32 : 16; }

int fail(sedi_handle* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(h, SEDI_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
  } while (0)

int dmalloc(sedi_handle* h, std::vector<void*>& list, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return fail(h, SEDI_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  list.push_back(*p);
  return 0;
}

void free_list(std::vector<void*>& list) {
  for (void* p : list) cudaFree(p);
  list.clear();
}

void clear_graphs(sedi_handle* h) {
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  h->pending.clear();
  for (auto& kv : h->gev)
    for (auto* v : {&kv.second.a, &kv.second.b, &kv.second.c})
      for (cudaEvent_t e : *v) cudaEventDestroy(e);
  h->gev.clear();
}

// Accumulate the elapsed times of recorded event pairs (profile mode).
void harvest(sedi_handle* h) {
  if (h->pending.empty()) return;
  cudaEventSynchronize(h->pending.back().second.second);
  for (auto& p : h->pending) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, p.second.first, p.second.second) == cudaSuccess) {
      h->ms[p.first] += t;
      h->cnt[p.first] += 1.0;
    } else {
      cudaGetLastError();  // a pair that was not recorded is skipped, not sticky
    }
  }
  h->pending.clear();
}

cudaEvent_t new_event() {
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void split_double(double x, dd* out) {
  float hi = (float)x;
  float lo = (float)(x - (double)hi);
  *out = dd{hi, lo};
}

template <class F>
void fill_consts(const sedi_params& p, ForceConsts<F>& K) {
  const double Es = p.E / (2.0 * (1.0 - p.poisson * p.poisson));
  const double G = p.E / (2.0 * (1.0 + p.poisson));
  const double Gs = G / (2.0 * (2.0 - p.poisson));
  const double lne = std::log(p.restitution);
  const double beta = lne / std::sqrt(lne * lne + M_PI * M_PI);
  K.Es = (F)Es;
  K.Gs = (F)Gs;
  K.cdamp = (F)(-2.0 * std::sqrt(5.0 / 6.0) * beta);
  K.kn_fac = (F)(4.0 / 3.0 * Es);
  K.ct_ratio = (F)std::sqrt(4.0 * Gs / Es);
  K.ct_ratio_lin = (F)std::sqrt(p.kt_ratio);
  K.law = p.contact_law;
  K.kn_lin = (F)p.kn_linear;
  K.kt_lin = (F)(p.kt_ratio * p.kn_linear);
  K.cdamp_lin = (F)(-2.0 * beta);
  K.mu = (F)p.friction;
  K.dt = (F)p.dt;
  K.lub_in = (F)p.lub_h_in_frac;
  K.lub_out = (F)p.lub_h_out_frac;
  K.six_pi_mu = (F)(6.0 * M_PI * p.rho_f * p.nu_f);
  K.lift_c = (F)(p.c_lift * p.rho_f * std::sqrt(p.nu_f));
  K.rho_f = (F)p.rho_f;
  K.nu_f = (F)p.nu_f;
  K.c_add_rho_f = (F)(p.c_add * p.rho_f);
  K.eps_max = (F)p.eps_max;
  for (int a = 0; a < 3; ++a) {
    const double L = p.hi[a] - p.lo[a];
    K.g[a] = (F)p.g[a];
    K.lo[a] = (F)p.lo[a];
    K.L[a] = (F)L;
    K.halfL[a] = (F)(0.5 * L);
    K.inv_h[a] = (F)((double)p.ncell[a] / L);
  }
}

void fill_params(sedi_handle* h) {
  const sedi_params& p = h->prm;
  DevParams& P = h->P;
  for (int a = 0; a < 3; ++a) {
    P.lo[a] = p.lo[a];
    P.hi[a] = p.hi[a];
    P.L[a] = p.hi[a] - p.lo[a];
    P.periodic[a] = p.periodic[a] ? 1 : 0;
    P.wall_lo[a] = (!p.periodic[a] && p.wall_lo[a]) ? 1 : 0;
    P.wall_hi[a] = (!p.periodic[a] && p.wall_hi[a]) ? 1 : 0;
    P.nc[a] = p.ncell[a];
    P.inv_h[a] = (double)p.ncell[a] / (p.hi[a] - p.lo[a]);
    P.bf.lo[a] = (float)p.lo[a];
    P.bf.hi[a] = (float)p.hi[a];
    P.bf.L[a] = (float)P.L[a];
    P.bdb.lo[a] = p.lo[a];
    P.bdb.hi[a] = p.hi[a];
    P.bdb.L[a] = P.L[a];
    split_double(p.lo[a], &P.bdd.lo[a]);
    split_double(p.hi[a], &P.bdd.hi[a]);
    split_double(P.L[a], &P.bdd.L[a]);
    const double hc = P.L[a] / p.ncell[a];
    P.bf.h[a] = (float)hc;
    P.bdb.h[a] = hc;
    split_double(hc, &P.bdd.h[a]);
  }
  P.lubrication = p.lubrication ? 1 : 0;
  P.drag = p.drag ? 1 : 0;
  P.pressure_grad = p.pressure_grad ? 1 : 0;
  P.added_mass = p.added_mass ? 1 : 0;
  P.lift = p.lift ? 1 : 0;
  P.lub_tangential = (p.lubrication && p.lub_tangential) ? 1 : 0;
  P.graded = p.z_grading != 1.0 ? 1 : 0;
  fill_consts<float>(p, P.cf);
  fill_consts<double>(p, P.cd);
  P.C = (int64_t)p.ncell[0] * p.ncell[1] * p.ncell[2];
  const double dx = (p.hi[0] - p.lo[0]) / p.ncell[0];
  const double dy = (p.hi[1] - p.lo[1]) / p.ncell[1];
  const double dz = (p.hi[2] - p.lo[2]) / p.ncell[2];
  P.vc = dx * dy * dz;
  P.cap = p.nbr_capacity;
  P.skin = p.skin;
  P.lub_out_frac = p.lub_h_out_frac;
  P.half_skin_f = (float)(0.5 * p.skin);
  P.lub_out_f = (float)p.lub_h_out_frac;
  P.shift[0] = p.shift_eps;
  P.shift[1] = p.shift_mom;
  P.shift[2] = p.shift_force;
  for (int k = 0; k < 3; ++k) P.two_shift[k] = std::ldexp(1.0, P.shift[k]);
  P.two_shift_f = (float)P.two_shift[2];
  P.inv_vc_f = (float)(1.0 / P.vc);
  const double dtau = 1.0 / p.n_tau;
  const double hs[3] = {dx, dy, dz};
  for (int a = 0; a < 3; ++a) {
    const double D = 0.25 * p.bandwidth[a] * p.bandwidth[a];
    h->coef[a] = dtau * D / (hs[a] * hs[a]);
  }
}

int check_params(sedi_handle* h, const sedi_params& p) {
  if (p.contact_law != SEDI_HERTZ_MINDLIN && p.contact_law != SEDI_LINEAR_SPRING)
    return fail(h, SEDI_EINVAL, "contact_law must be SEDI_HERTZ_MINDLIN or SEDI_LINEAR_SPRING");
  if (p.contact_law == SEDI_LINEAR_SPRING && (!(p.kn_linear > 0) || !(p.kt_ratio >= 0)))
    return fail(h, SEDI_EINVAL, "linear contact law needs kn_linear > 0 and kt_ratio >= 0");
  if (!(p.E > 0) || !(p.poisson >= 0 && p.poisson < 0.5)) return fail(h, SEDI_EINVAL, "E > 0 and 0 <= poisson < 0.5 required");
  if (!(p.restitution > 0 && p.restitution <= 1)) return fail(h, SEDI_EINVAL, "restitution must be in (0, 1]");
  if (!(p.friction >= 0)) return fail(h, SEDI_EINVAL, "friction must be >= 0");
  if (!(p.c_lift >= 0)) return fail(h, SEDI_EINVAL, "c_lift must be >= 0");
  if (!(p.z_grading > 0) || !std::isfinite(p.z_grading)) return fail(h, SEDI_EINVAL, "z_grading must be > 0");
  if (p.z_grading != 1.0 && (p.periodic[2] || p.ncell[2] < 2))
    return fail(h, SEDI_EINVAL, "a graded z mesh needs a non-periodic z axis with ncell[2] >= 2");
  if (!(p.rho_f > 0) || !(p.nu_f > 0)) return fail(h, SEDI_EINVAL, "rho_f, nu_f must be > 0");
  if (!(p.dt > 0) || !(p.skin >= 0)) return fail(h, SEDI_EINVAL, "dt > 0 and skin >= 0 required");
  for (int a = 0; a < 3; ++a) {
    if (!(p.hi[a] > p.lo[a])) return fail(h, SEDI_EINVAL, "box hi must exceed lo on axis %d", a);
    if (p.ncell[a] < 1) return fail(h, SEDI_EINVAL, "ncell must be >= 1");
    if (!(p.bandwidth[a] >= 0)) return fail(h, SEDI_EINVAL, "bandwidth must be >= 0");
  }
  if (!(p.lub_h_in_frac > 0) || !(p.lub_h_out_frac > p.lub_h_in_frac)) return fail(h, SEDI_EINVAL, "need 0 < lub_h_in_frac < lub_h_out_frac");
  if (p.n_tau < 1 || !(p.cg_rtol > 0) || p.cg_max_iter < 1) return fail(h, SEDI_EINVAL, "n_tau, cg_rtol, cg_max_iter must be positive");
  if (p.tau_scheme != SEDI_TAU_EULER && p.tau_scheme != SEDI_TAU_BDF2)
    return fail(h, SEDI_EINVAL, "tau_scheme must be SEDI_TAU_EULER or SEDI_TAU_BDF2");
  if (p.tau_scheme == SEDI_TAU_BDF2 && p.use_cnn_guess)
    return fail(h, SEDI_EINVAL, "the learned warm start runs backward-Euler pseudo-steps only");
  if (p.precision_form < 0 || p.precision_form > 2) return fail(h, SEDI_EINVAL, "unknown precision_form");
  if (p.bins_per_cutoff < 0 || p.bins_per_cutoff > 2) return fail(h, SEDI_EINVAL, "bins_per_cutoff must be 0, 1 or 2");
  if (p.bin_order < -1 || p.bin_order > 1) return fail(h, SEDI_EINVAL, "bin_order must be -1, 0 or 1");
  if (p.nbr_capacity < 1 || p.nbr_capacity > kMaxCap) return fail(h, SEDI_EINVAL, "nbr_capacity must be in [1, %d]", kMaxCap);
  if (p.n_beds < 1 || p.n_beds > kMaxBeds) return fail(h, SEDI_EINVAL, "n_beds must be in [1, %d]", kMaxBeds);
  if (p.substep_variant < -1 || p.substep_variant >= kSubstepVariants)
    return fail(h, SEDI_EINVAL, "substep_variant must be -1 (tuned) or in [0, %d]", kSubstepVariants - 1);
  for (int k = 0; k < 3; ++k) {
    int s = k == 0 ? p.shift_eps : (k == 1 ? p.shift_mom : p.shift_force);
    if (s < 0 || s > 60) return fail(h, SEDI_EINVAL, "fixed-point shifts must be in [0, 60]");
  }
  return 0;
}

int copy_in(sedi_handle* h, void* dst, const void* src, size_t bytes, int mem) {
  CK(cudaMemcpyAsync(dst, src, bytes, mem == SEDI_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  return 0;
}

int copy_out(sedi_handle* h, void* dst, const void* src, size_t bytes, int mem) {
  CK(cudaMemcpyAsync(dst, src, bytes, mem == SEDI_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  return 0;
}

int ensure_stage(sedi_handle* h, size_t n) {
  if (h->dstage_n >= n) return 0;
  if (h->dstage) cudaFree(h->dstage);
  h->dstage = nullptr;
  h->dstage_n = 0;
  CK(cudaMalloc((void**)&h->dstage, n * sizeof(double)));
  h->dstage_n = n;
  return 0;
}

// Read the device control block; map device-side errors to status codes.
int sync_status(sedi_handle* h) {
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  if (!h->st.ctl) return 0;
  Ctl c;
  CK(cudaMemcpy(&c, h->st.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  h->stats.rebuilds = c.rebuilds;
  h->stats.max_neighbors = c.max_nn;
  if (c.error == SEDI_EOVERFLOW)
    return fail(h, SEDI_EOVERFLOW, "a particle has %d listed neighbours > nbr_capacity %d", c.overflow_nn, h->P.cap);
  if (c.error == SEDI_ENONFINITE) return fail(h, SEDI_ENONFINITE, "non-finite force or state");
  if (c.error) return fail(h, c.error, "device error %d", c.error);
  return 0;
}

// Graded z mesh (Sec. 4.2): cell heights h_k = h_0 r^k from the floor,
// r = z_grading^(1/(nz - 1)), faces z_k = lo + L (r^k - 1) / (r^nz - 1) (expm1 keeps a
// ratio near 1 accurate); centres, cell volumes h_x h_y h_k, and per plane the
// finite-volume z-face coefficients of one smoothing step,
// c-_k = dtau D_z / (h_k (zc_k - zc_{k-1})), c+_k = dtau D_z / (h_k (zc_{k+1} - zc_k))
// (0 at the floor and lid), times 2/3 for BDF2 steps; plane weights h_k / mean h.
// One device buffer; nothing on a uniform mesh.
int build_zgrid(sedi_handle* h) {
  const sedi_params& p = h->prm;
  if (!h->P.graded) return 0;
  const int64_t n = p.ncell[2], nxy = (int64_t)p.ncell[0] * p.ncell[1];
  const double L = p.hi[2] - p.lo[2];
  const double lr = std::log(p.z_grading) / (double)(n - 1);
  std::vector<double> zf(n + 1), zc(n), hz(n);
  for (int64_t k = 0; k <= n; ++k) zf[k] = p.lo[2] + L * (std::expm1((double)k * lr) / std::expm1((double)n * lr));
  zf[0] = p.lo[2];
  zf[n] = p.hi[2];
  for (int64_t k = 0; k < n; ++k) {
    zc[k] = 0.5 * (zf[k] + zf[k + 1]);
    hz[k] = zf[k + 1] - zf[k];
  }
  const double dx = (p.hi[0] - p.lo[0]) / p.ncell[0], dy = (p.hi[1] - p.lo[1]) / p.ncell[1];
  const double dtau = 1.0 / p.n_tau, Dz = 0.25 * p.bandwidth[2] * p.bandwidth[2], hmean = L / (double)n;
  // doubles: zf, zc, vc, cz[0], cz[1], w; floats: zcf, czf[0], czf[1]
  const size_t nd = (n + 1) + n + n + 2 * n + 2 * n + n, nfl = n + 2 * n + 2 * n;
  std::vector<double> dv(nd, 0.0);
  std::vector<float> fv(nfl, 0.0f);
  double* d_zf = dv.data();
  double* d_zc = d_zf + (n + 1);
  double* d_vc = d_zc + n;
  double* d_cz0 = d_vc + n;
  double* d_cz1 = d_cz0 + 2 * n;
  double* d_w = d_cz1 + 2 * n;
  float* f_zc = fv.data();
  float* f_cz0 = f_zc + n;
  float* f_cz1 = f_cz0 + 2 * n;
  double zmax[2] = {0.0, 0.0}, wsum = 0.0;
  for (int64_t k = 0; k <= n; ++k) d_zf[k] = zf[k];
  for (int64_t k = 0; k < n; ++k) {
    d_zc[k] = zc[k];
    f_zc[k] = (float)zc[k];
    d_vc[k] = dx * dy * hz[k];
    d_w[k] = hz[k] / hmean;
    wsum += d_w[k] * (double)nxy;
    for (int s = 0; s < 2; ++s) {
      const double scale = s == 0 ? 1.0 : 2.0 / 3.0;
      double* cz = s == 0 ? d_cz0 : d_cz1;
      float* czf = s == 0 ? f_cz0 : f_cz1;
      cz[2 * k] = k > 0 ? scale * dtau * Dz / (hz[k] * (zc[k] - zc[k - 1])) : 0.0;
      cz[2 * k + 1] = k < n - 1 ? scale * dtau * Dz / (hz[k] * (zc[k + 1] - zc[k])) : 0.0;
      czf[2 * k] = (float)cz[2 * k];
      czf[2 * k + 1] = (float)cz[2 * k + 1];
      zmax[s] = std::max(zmax[s], cz[2 * k] + cz[2 * k + 1]);
    }
  }
  void* buf = nullptr;
  const size_t dbytes = (nd * 8 + 255) & ~(size_t)255;
  int rc = dmalloc(h, h->mesh_allocs, &buf, dbytes + nfl * 4);
  if (rc) return rc;
  CK(cudaMemcpy(buf, dv.data(), nd * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy((char*)buf + dbytes, fv.data(), nfl * 4, cudaMemcpyHostToDevice));
  const double* bd = (const double*)buf;
  const float* bf = (const float*)((char*)buf + dbytes);
  h->mesh.zf = bd;
  h->mesh.zc = bd + (n + 1);
  h->mesh.vcz = bd + (n + 1) + n;
  h->mesh.zcf = bf;
  h->zs.cz[0] = bd + (n + 1) + 2 * n;
  h->zs.cz[1] = bd + (n + 1) + 4 * n;
  h->zs.w = bd + (n + 1) + 6 * n;
  h->zs.czf[0] = bf + n;
  h->zs.czf[1] = bf + 3 * n;
  h->zs.wsum = wsum;
  h->zs.zmax[0] = zmax[0];
  h->zs.zmax[1] = zmax[1];
  return 0;
}

// Mesh words of the fluid fields from the FP64 fields kept on the device (fdev:
// U, grad p, DU/Dt); the vorticity too when the lift is on and U changed.
int upload_mesh(sedi_handle* h, bool velocity = true) {
  const int64_t C = h->P.C;
  const sedi_params& p = h->prm;
  const double rho_g[3] = {p.rho_f * p.g[0], p.rho_f * p.g[1], p.rho_f * p.g[2]};
  launch_fluid_prep(h->form, h->fdev, h->fdev + 3 * C, h->fdev + 6 * C, h->gp_default ? 1 : 0,
                    p.c_add * p.rho_f, rho_g, h->P, h->mesh, h->stream);
  if (velocity && h->P.lift) launch_curl(h->form, h->fdev, h->P, h->mesh, h->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return 0;
}

// Link-cell bins of edge >= rc_max / R (R bins per list cutoff, with margin): the list
// build visits the (2R + 1)^3 bins around a particle's bin.  Lists hold their partners
// in caller-index order whatever the bins, so R changes no result, only the cost.
// Nonzero when a periodic axis is shorter than 2R + 1 bins or the bins would not fit
// 31-bit indices.
int bins_for(const sedi_handle* h, int R, int32_t nb[3], int64_t* nbins) {
  const sedi_params& p = h->prm;
  const double hb = h->rc_max * 1.001 / R;
  *nbins = 1;
  for (int a = 0; a < 3; ++a) {
    const double L = p.hi[a] - p.lo[a];
    int64_t n = (int64_t)std::floor(L / hb);
    if (n < 1) n = 1;
    if (p.periodic[a] && n < 2 * R + 1) return 1;
    if (n > ((int64_t)1 << 30)) return 2;
    nb[a] = (int32_t)n;
    *nbins *= n;
    if (*nbins > ((int64_t)1 << 31) - 2) return 2;
  }
  return 0;
}

int set_bins(sedi_handle* h, int R) {
  int32_t nb[3];
  int64_t nbins = 0;
  if (const int why = bins_for(h, R, nb, &nbins)) {
    if (R == 1 && why == 1)
      return fail(h, SEDI_EINVAL, "a periodic axis is shorter than 3 list cutoffs (%g m)", 3 * h->rc_max * 1.001);
    return fail(h, SEDI_EINVAL, "%d bins per list cutoff do not fit this box", R);
  }
  free_list(h->bin_allocs);
  DevState& st = h->st;
  for (int a = 0; a < 3; ++a) {
    h->P.nb[a] = nb[a];
    h->P.bin_inv[a] = (float)((double)nb[a] / (h->prm.hi[a] - h->prm.lo[a]));
  }
  h->P.nbins = nbins;
  h->P.bin_reach = R;
  const int64_t nblk = (nbins + 1023) / 1024 + 1;
  int rc;
  if ((rc = dmalloc(h, h->bin_allocs, (void**)&st.bin_count, 4 * nbins)) ||
      (rc = dmalloc(h, h->bin_allocs, (void**)&st.bin_start, 4 * (nbins + 1))) ||
      (rc = dmalloc(h, h->bin_allocs, (void**)&st.bin_fill, 4 * nbins)) ||
      (rc = dmalloc(h, h->bin_allocs, (void**)&st.scan_blk, 4 * nblk)))
    return rc;
  return 0;
}

int alloc_particles(sedi_handle* h, int64_t N, double rmax) {
  clear_graphs(h);
  h->key_cache.clear();
  free_list(h->part_allocs);
  DevState& st = h->st;
  Ctl* ctl = st.ctl;
  st = DevState{};
  st.ctl = ctl;
  st.N = N;
  const int form = h->form;
  const size_t q = quad_bytes(form), fq = fquad_bytes(form), w = word_bytes(form);
  const int64_t cap = h->P.cap;
  int rc;
  for (int b = 0; b < 2; ++b) {
    if ((rc = dmalloc(h, h->part_allocs, &st.pos[b], q * N))) return rc;
    if ((rc = dmalloc(h, h->part_allocs, &st.vel[b], q * N))) return rc;
    if ((rc = dmalloc(h, h->part_allocs, &st.omg[b], q * N))) return rc;
    if ((rc = dmalloc(h, h->part_allocs, &st.acc[b], fq * N))) return rc;
    if ((rc = dmalloc(h, h->part_allocs, (void**)&st.uid[b], 4 * N))) return rc;
    if ((rc = dmalloc(h, h->part_allocs, (void**)&st.r64[b], 8 * N))) return rc;
    if ((rc = dmalloc(h, h->part_allocs, (void**)&st.vfrac[b], 8 * N))) return rc;
    if ((rc = dmalloc(h, h->part_allocs, (void**)&st.xb[b], 16 * N))) return rc;
    if ((rc = dmalloc(h, h->part_allocs, &st.whist[b], (size_t)kWalls * 3 * w * N))) return rc;
    if ((rc = dmalloc(h, h->part_allocs, (void**)&st.wmask[b], 4 * N))) return rc;
    if ((rc = dmalloc(h, h->part_allocs, (void**)&st.nbr[b], 4 * cap * N))) return rc;
    if ((rc = dmalloc(h, h->part_allocs, (void**)&st.nn[b], 4 * N))) return rc;
    if ((rc = dmalloc(h, h->part_allocs, &st.hist[b], q * cap * N))) return rc;
    if ((rc = dmalloc(h, h->part_allocs, (void**)&st.cmask[b], 4 * N))) return rc;
  }
  if (form != FORM_FP64 && !h->is_bed && cap * N / 2 + 1 < ((int64_t)1 << 31)) {
    // pair list (substep variants SUBSTEP_PAIRS*; not for ensemble beds, which the
    // ensemble steps with the per-particle loop): every listed pair once, cap N / 2 at
    // most (pair ids share a word with the first-particle bit, so fewer than 2^31)
    st.pcap = cap * N / 2 + 1;
    if ((rc = dmalloc(h, h->part_allocs, (void**)&st.pairs, 16 * st.pcap)) ||
        (rc = dmalloc(h, h->part_allocs, (void**)&st.pid, 4 * cap * N)) ||
        (rc = dmalloc(h, h->part_allocs, (void**)&st.prec, 32 * st.pcap)) ||
        (rc = dmalloc(h, h->part_allocs, (void**)&st.pstart, 4 * (N + 1))) ||
        (rc = dmalloc(h, h->part_allocs, (void**)&st.pscan_blk, 4 * ((N + 1023) / 1024 + 1))))
      return rc;
    CK(cudaMemset(st.pairs, 0, 16 * st.pcap));
    CK(cudaMemset(st.pid, 0, 4 * cap * N));
    CK(cudaMemset(st.prec, 0, 32 * st.pcap));
  }
  // bins: R = 1 (edge >= the largest list cutoff) until the autotuner picks otherwise;
  // a tuned R is kept while it fits the new particles
  h->rc_max = (2.0 * rmax) * (1.0 + h->prm.lub_h_out_frac) + h->prm.skin;
  if (h->prm.bin_order >= 0) h->P.bin_zfast = h->prm.bin_order;
  if (h->prm.bins_per_cutoff > 0) {
    if ((rc = set_bins(h, h->prm.bins_per_cutoff))) return rc;
  } else {
    int R = h->P.bin_reach > 1 ? h->P.bin_reach : 1;
    int32_t nb[3];
    int64_t nbins = 0;
    if (R > 1 && bins_for(h, R, nb, &nbins)) R = 1;
    if ((rc = set_bins(h, R))) return rc;
  }
  if ((rc = dmalloc(h, h->part_allocs, (void**)&st.bin_of, 4 * N))) return rc;
  if ((rc = dmalloc(h, h->part_allocs, (void**)&st.order, 4 * N))) return rc;
  if ((rc = dmalloc(h, h->part_allocs, (void**)&st.fdbg, 8 * 12 * N))) return rc;
  CK(cudaMemsetAsync(st.cmask[0], 0, 4 * N, h->stream));
  CK(cudaMemsetAsync(st.cmask[1], 0, 4 * N, h->stream));
  CK(cudaMemsetAsync(st.wmask[0], 0, 4 * N, h->stream));
  CK(cudaMemsetAsync(st.wmask[1], 0, 4 * N, h->stream));
  CK(cudaMemsetAsync(st.nn[0], 0, 4 * N, h->stream));
  CK(cudaMemsetAsync(st.nn[1], 0, 4 * N, h->stream));
  return ensure_stage(h, std::max<size_t>((size_t)12 * N, (size_t)8 * h->P.C));
}

int build_graph(sedi_handle* h, int n, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  sedi_handle::GraphEv ev;
  if (h->prm.profile)
    for (int s = 0; s < n; ++s) {
      ev.a.push_back(new_event());
      ev.b.push_back(new_event());
      ev.c.push_back(new_event());
    }
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  // one IF node per substep: the first condition comes from a check kernel, every
  // later one from the last block of the previous substep kernel
  std::vector<cudaGraphConditionalHandle> ch(n);
  for (int s = 0; s < n; ++s) CK(cudaGraphConditionalHandleCreate(&ch[s], g, 0, cudaGraphCondAssignDefault));
  // inside a capture only the External flag makes an event-record node
  if (h->prm.profile) CK(cudaEventRecordWithFlags(ev.a[0], h->stream, cudaEventRecordExternal));
  launch_check(h->st, h->P, (unsigned long long)ch[0], 1, h->stream);
  for (int s = 0; s < n; ++s) {
    if (h->prm.profile && s > 0) CK(cudaEventRecordWithFlags(ev.a[s], h->stream, cudaEventRecordExternal));
    CK(cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &g, &deps, nullptr, &nd));
    // the struct has a union of non-trivial members: zero raw storage instead
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    std::memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams* cp = reinterpret_cast<cudaGraphNodeParams*>(raw);
    cp->type = cudaGraphNodeTypeConditional;
    cp->conditional.handle = ch[s];
    cp->conditional.type = cudaGraphCondTypeIf;
    cp->conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, cp));
    CK(cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = cp->conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(h->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch_rebuild(h->form, h->st, h->P, s, false, h->side);
    CK(cudaStreamEndCapture(h->side, &body));
    if (h->prm.profile) CK(cudaEventRecordWithFlags(ev.b[s], h->stream, cudaEventRecordExternal));
    const bool more = s + 1 < n;
    launch_substep(h->form, h->st, h->mesh, h->P, s, true, h->variant,
                   more ? (unsigned long long)ch[s + 1] : 0ull, more ? 1 : 0, h->stream);
    if (h->prm.profile) CK(cudaEventRecordWithFlags(ev.c[s], h->stream, cudaEventRecordExternal));
  }
  launch_advance_parity(h->st, n, h->stream);
  CK(cudaStreamEndCapture(h->stream, &graph));
  if (h->prm.profile) h->gev[n] = ev;
  cudaError_t e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(h, SEDI_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  return 0;
}

int need_particles(sedi_handle* h) {
  if (!h) return SEDI_EINVAL;
  if (!h->have_particles) return fail(h, SEDI_ESTATE, "no particles set");
  return 0;
}


// Ensembles: a per-bed call goes to that bed's single-bed handle.
#define ENS_FORWARD(CALL)                                                                 \
  do {                                                                                    \
    if (!h->beds.empty()) {                                                               \
      if (bed < 0 || bed >= (int32_t)h->beds.size())                                      \
        return fail(h, SEDI_EINVAL, "bed %d out of range", bed);                          \
      sedi_handle* sub = h->beds[bed];                                                    \
      const auto rc_ = (CALL);                                                            \
      if (rc_ < 0) h->err = sub->err;                                                     \
      return rc_;                                                                         \
    }                                                                                     \
  } while (0)

// The fluid fields and the drag's solid fraction live on the device; the host
// copies serve checkpoints only and are brought up to date here.
int refresh_fluid_host(sedi_handle* h) {
  if (!h->fluid_host_stale) return 0;
  const int64_t C = h->P.C;
  launch_eps_io(h->form, h->edev, h->mesh, C, 0, h->stream);
  CK(cudaMemcpyAsync(h->U.data(), h->fdev, 24 * C, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->gp.data(), h->fdev + 3 * C, 24 * C, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->du.data(), h->fdev + 6 * C, 24 * C, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->eps.data(), h->edev, 8 * C, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->fluid_host_stale = false;
  return 0;
}

int rebuild_now(sedi_handle* h) {
  launch_rebuild(h->form, h->st, h->P, 0, true, h->stream);
  return sync_status(h);
}

// ---------------------------------------------------------------- autotuner
// The launch variant of the substep kernel (threads per block x resident blocks,
// which sets the register budget, the pair phase, or the pair list) and the bin size
// of the list build (R = 1 or 2 bins per list cutoff) are picked per workload.  For
// each R the bins are resized and the lists rebuilt at once from the current
// positions (springs carried over, as at any rebuild); then one integrating substep of
// every variant is timed with events in interleaved rounds.  A substep reads the
// state buffer the step starts from and writes the other one, so only the arrays it
// updates in place (springs and their masks, wall springs, lagged accelerations, the
// control block) are copied aside first and put back after every timed launch.  The
// cost of a pair (R, variant) is its median substep plus the rebuild time of R times
// the rebuilds per substep seen so far; the cheapest wins.  Neither choice changes a
// result (lists are sorted by caller index, every variant adds the same terms in the
// same order, and an extra rebuild lists the same interacting pairs), so tuning
// leaves the trajectory as it found it.  Results are keyed by (GPU, N, diameter
// range, form, terms), kept for the process and, when the environment variable
// SEDI_AUTOTUNE_CACHE names a file, in that file as one JSON object per line.

constexpr int kTuneRounds = 5;
// Springs and lubrication gaps form over the first substeps after the particles are
// set (a fresh state has no tangential history); the launch shapes are compared on
// a state that has them.  Until then the per-particle loop at 128 x 6 runs.
constexpr int64_t kTuneAfter = 200;

// A bin configuration: R bins per list cutoff and the storage order of the bins.
struct BinCfg {
  int reach = 1;  // 1 or 2
  int zfast = 0;  // 0: x fastest, 1: z fastest
  bool operator==(const BinCfg& o) const { return reach == o.reach && zfast == o.zfast; }
  bool operator!=(const BinCfg& o) const { return !(*this == o); }
};

BinCfg bin_cfg(const sedi_handle* h) {
  BinCfg c;
  c.reach = h->P.bin_reach > 1 ? h->P.bin_reach : 1;
  c.zfast = h->P.bin_zfast ? 1 : 0;
  return c;
}

struct TuneChoice {
  int variant = -1;
  BinCfg bins;
};

std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune_cache;

// The workload key, computed once per particle set (it reads every diameter).
std::string tune_key(sedi_handle* h) {
  if (!h->key_cache.empty()) return h->key_cache;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) std::snprintf(prop.name, sizeof(prop.name), "device%d", dev);
  double dmin = 1e300, dmax = 0.0;
  for (double d : h->d_host) {
    dmin = std::min(dmin, d);
    dmax = std::max(dmax, d);
  }
  // the force terms that change a pair's cost belong to the workload too
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s sm%d|N=%lld|d=%.3e..%.3e|form=%d|law=%d|lub=%d|fluid=%d%d%d",
                prop.name, prop.multiProcessorCount, (long long)h->N, dmin, dmax, h->form,
                h->prm.contact_law, h->P.lubrication, h->P.drag, h->P.pressure_grad, h->P.added_mass);
  h->key_cache = buf;
  return h->key_cache;
}

TuneChoice tune_file_lookup(const std::string& key) {
  TuneChoice found;
  const char* path = std::getenv("SEDI_AUTOTUNE_CACHE");
  if (!path || !*path) return found;
  FILE* f = std::fopen(path, "r");
  if (!f) return found;
  char line[2048];
  const std::string want = "\"key\": \"" + key + "\"";
  while (std::fgets(line, sizeof(line), f)) {
    const char* k = std::strstr(line, want.c_str());
    const char* v = std::strstr(line, "\"variant\": ");
    const char* r = std::strstr(line, "\"bins_per_cutoff\": ");
    const char* o = std::strstr(line, "\"bin_order\": \"");
    if (!k || !v || !r || !o) continue;
    const int var = std::atoi(v + 11), reach = std::atoi(r + 19);
    if (var >= 0 && var < kSubstepVariants && (reach == 1 || reach == 2)) {
      found.variant = var;  // the last entry wins
      found.bins.reach = reach;
      found.bins.zfast = o[14] == 'z' ? 1 : 0;
    }
  }
  std::fclose(f);
  return found;
}

void tune_file_store(const std::string& key, const TuneChoice& best, const std::vector<BinCfg>& cfgs,
                     const std::vector<std::vector<double>>& us, const std::vector<double>& rebuild_us) {
  const char* path = std::getenv("SEDI_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "{\"key\": \"%s\", \"variant\": %d, \"bins_per_cutoff\": %d, \"bin_order\": \"%c\", "
               "\"block\": %d, \"median_us\": {",
               key.c_str(), best.variant, best.bins.reach, best.bins.zfast ? 'z' : 'x', substep_block(best.variant));
  for (size_t r = 0; r < cfgs.size(); ++r) {
    std::fprintf(f, "%s\"R%d%c\": [", r ? ", " : "", cfgs[r].reach, cfgs[r].zfast ? 'z' : 'x');
    for (int v = 0; v < kSubstepVariants; ++v) std::fprintf(f, "%s%.3f", v ? ", " : "", us[r][v]);
    std::fprintf(f, "]");
  }
  std::fprintf(f, "}, \"rebuild_us\": [");
  for (size_t r = 0; r < rebuild_us.size(); ++r) std::fprintf(f, "%s%.3f", r ? ", " : "", rebuild_us[r]);
  std::fprintf(f, "]}\n");
  std::fclose(f);
}

// The bins of a configuration (graphs cleared when it changes: they bake in the bin
// arrays and parameters).
int apply_bins(sedi_handle* h, const BinCfg& b) {
  if (b == bin_cfg(h)) return 0;
  clear_graphs(h);
  int rc;
  if (b.reach != h->P.bin_reach && (rc = set_bins(h, b.reach))) return rc;
  h->P.bin_zfast = b.zfast;
  return 0;
}

// Bins of a configuration and a rebuild at once; the rebuild counter is left as it
// was (the tuner's rebuilds are not the run's).
int retune_bins(sedi_handle* h, const BinCfg& b) {
  Ctl c;
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(&c, h->st.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  const int64_t rebuilds = c.rebuilds;
  int rc;
  if ((rc = apply_bins(h, b))) return rc;
  launch_rebuild_now(h->form, h->st, h->P, h->stream);
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(&c, h->st.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  c.rebuilds = rebuilds;
  CK(cudaMemcpy(h->st.ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice));
  return sync_status(h);
}

// Choose h->variant and the bin size for the current particles (no-op when fixed or
// up to date).
int autotune(sedi_handle* h) {
  if (h->prm.substep_variant >= 0 || h->form == FORM_FP64) return 0;
  if (h->P.lift || h->P.lub_tangential) {
    // the optional terms run one launch shape (the per-particle loop at 128 x 6)
    h->variant = SUBSTEP_B128_LOOP;
    return 0;
  }
  if (h->since_set < kTuneAfter) return 0;
  const std::string key = tune_key(h);
  if (key == h->tuned_key) return 0;
  TuneChoice best;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) best = it->second;
  }
  if (best.variant < 0) best = tune_file_lookup(key);
  if (best.variant < 0) {
    int rc;
    Ctl c0;
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy(&c0, h->st.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    const double rate = (double)std::max<int64_t>(c0.rebuilds, 1) / (double)std::max<int64_t>(h->since_set, 1);
    // R = 2 only while its bins stay few next to the particles (a sweep of the bin
    // arrays per rebuild: 32 per particle at most); a fixed bins_per_cutoff is the only
    // candidate
    std::vector<int> reaches = {1};
    if (h->prm.bins_per_cutoff > 0) {
      reaches = {h->prm.bins_per_cutoff};
    } else {
      int32_t nb[3];
      int64_t nbins = 0;
      if (!bins_for(h, 2, nb, &nbins) && nbins <= std::max<int64_t>(32 * h->N, (int64_t)1 << 22))
        reaches.push_back(2);
    }
    // every bin size in both storage orders, the current configuration last (a single
    // candidate then needs no extra resize)
    std::vector<BinCfg> cfgs;
    for (int R : reaches)
      for (int z = 0; z < 2; ++z) {
        if (h->prm.bin_order >= 0 && z != h->prm.bin_order) continue;
        BinCfg c;
        c.reach = R;
        c.zfast = z;
        if (c != bin_cfg(h)) cfgs.push_back(c);
      }
    if (std::find(reaches.begin(), reaches.end(), bin_cfg(h).reach) != reaches.end() &&
        (h->prm.bin_order < 0 || bin_cfg(h).zfast == h->prm.bin_order))
      cfgs.push_back(bin_cfg(h));
    std::vector<std::vector<double>> med(cfgs.size(), std::vector<double>(kSubstepVariants, 1e30));
    std::vector<double> rebuild_us(cfgs.size(), 0.0);
    const int64_t N = h->N, cap = h->P.cap;
    const size_t q = quad_bytes(h->form), fq = fquad_bytes(h->form), w = word_bytes(h->form);
    cudaEvent_t rb[2];
    CK(cudaEventCreate(&rb[0]));
    CK(cudaEventCreate(&rb[1]));
    std::vector<cudaEvent_t> ev(2 * kSubstepVariants * kTuneRounds, nullptr);
    for (auto& e : ev) CK(cudaEventCreate(&e));
    rc = 0;
    for (size_t ri = 0; ri < cfgs.size() && !rc; ++ri) {
      // the bins of this configuration and lists built from the current positions (timed)
      if ((rc = apply_bins(h, cfgs[ri]))) break;
      {
        Ctl c;
        CK(cudaMemcpy(&c, h->st.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
        const int64_t rebuilds = c.rebuilds;
        CK(cudaEventRecord(rb[0], h->stream));
        launch_rebuild_now(h->form, h->st, h->P, h->stream);
        CK(cudaEventRecord(rb[1], h->stream));
        if ((rc = sync_status(h))) break;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, rb[0], rb[1]) == cudaSuccess) rebuild_us[ri] = 1e3 * ms;
        CK(cudaMemcpy(&c, h->st.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
        c.rebuilds = rebuilds;
        CK(cudaMemcpy(h->st.ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice));
      }
      // the arrays an integrating substep updates in place, and their saved copies
      Ctl c;
      CK(cudaMemcpy(&c, h->st.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
      struct Item { void* p; size_t n; };
      const std::vector<Item> live = {
          {h->st.hist[c.nl], q * cap * N}, {h->st.cmask[c.nl], 4 * (size_t)N},
          {h->st.acc[c.pb], fq * N}, {h->st.whist[c.pb], (size_t)kWalls * 3 * w * N},
          {h->st.wmask[c.pb], 4 * (size_t)N}, {h->st.ctl, sizeof(Ctl)}};
      size_t total = 0;
      for (const auto& it : live) total += (it.n + 255) & ~(size_t)255;
      char* save = nullptr;
      if (cudaMalloc((void**)&save, total) != cudaSuccess) {
        // no room for the saved copies: keep this bin size and the current launch shape
        cudaGetLastError();
        best.variant = h->variant;
        best.bins = cfgs[ri];
        cfgs.resize(ri + 1);
        med.resize(ri + 1);
        rebuild_us.resize(ri + 1);
        med[ri].assign(kSubstepVariants, 1e30);
        med[ri][h->variant] = 0.0;
        break;
      }
      auto copy_all = [&](bool to_save) {
        size_t off = 0;
        for (const auto& it : live) {
          if (to_save) cudaMemcpyAsync(save + off, it.p, it.n, cudaMemcpyDeviceToDevice, h->stream);
          else cudaMemcpyAsync(it.p, save + off, it.n, cudaMemcpyDeviceToDevice, h->stream);
          off += (it.n + 255) & ~(size_t)255;
        }
      };
      copy_all(true);
      for (int v = 0; v < kSubstepVariants; ++v) {  // warm-up: first launch of each variant
        launch_substep(h->form, h->st, h->mesh, h->P, 0, true, v, 0ull, 0, h->stream);
        copy_all(false);
      }
      for (int r = 0; r < kTuneRounds; ++r)
        for (int v = 0; v < kSubstepVariants; ++v) {
          cudaEvent_t* e = &ev[2 * (r * kSubstepVariants + v)];
          CK(cudaEventRecord(e[0], h->stream));
          launch_substep(h->form, h->st, h->mesh, h->P, 0, true, v, 0ull, 0, h->stream);
          CK(cudaEventRecord(e[1], h->stream));
          copy_all(false);
        }
      rc = sync_status(h);
      cudaFree(save);
      for (int v = 0; v < kSubstepVariants && !rc; ++v) {
        std::vector<double> t;
        for (int r = 0; r < kTuneRounds; ++r) {
          float ms = 0.0f;
          cudaEvent_t* e = &ev[2 * (r * kSubstepVariants + v)];
          if (cudaEventElapsedTime(&ms, e[0], e[1]) != cudaSuccess) ms = 1e30f;
          t.push_back(1e3 * ms);
        }
        std::sort(t.begin(), t.end());
        med[ri][v] = t[kTuneRounds / 2];
      }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    cudaEventDestroy(rb[0]);
    cudaEventDestroy(rb[1]);
    if (rc) return rc;
    double best_cost = 1e300;
    for (size_t ri = 0; ri < cfgs.size(); ++ri)
      for (int v = 0; v < kSubstepVariants; ++v) {
        const double cost = med[ri][v] + rebuild_us[ri] * rate;
        if (cost < best_cost) {
          best_cost = cost;
          best.variant = v;
          best.bins = cfgs[ri];
        }
      }
    tune_file_store(key, best, cfgs, med, rebuild_us);
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  // the chosen bins (lists rebuilt at once when they change)
  if (best.bins != bin_cfg(h)) {
    const int rc = retune_bins(h, best.bins);
    if (rc) return rc;
  }
  if (best.variant != h->variant) clear_graphs(h);  // graphs bake in the launch shape
  // leaving the pair mode: the other variants read the partner copies of the springs
  if (pair_variant(h->variant) && !pair_variant(best.variant)) launch_spring_sync(h->form, h->st, h->stream);
  h->variant = best.variant;
  h->tuned_key = key;
  return 0;
}

}  // namespace

extern "C" {

void sedi_default_params(sedi_params* p) {
  std::memset(p, 0, sizeof(*p));
  p->contact_law = SEDI_HERTZ_MINDLIN;
  p->E = 1.0e7;
  p->poisson = 0.3;
  p->restitution = 0.9;
  p->friction = 0.3;
  p->kn_linear = 800.0;
  p->kt_ratio = 2.0 / 7.0;
  p->rho_f = 1000.0;
  p->nu_f = 1.0e-6;
  p->g[2] = -9.81;
  p->hi[0] = 20e-3;
  p->hi[1] = 20e-3;
  p->hi[2] = 40e-3;
  p->periodic[0] = p->periodic[1] = 1;
  p->wall_lo[2] = p->wall_hi[2] = 1;
  p->dt = 1.0e-6;
  p->skin = 0.05e-3;
  p->lubrication = p->drag = p->pressure_grad = p->added_mass = 1;
  p->lub_h_in_frac = 1.0e-3;
  p->lub_h_out_frac = 0.1;
  p->c_add = 0.5;
  p->c_lift = 1.6;
  p->z_grading = 1.0;
  p->eps_max = 0.9;
  p->ncell[0] = 10;
  p->ncell[1] = 10;
  p->ncell[2] = 20;
  p->bandwidth[0] = p->bandwidth[1] = p->bandwidth[2] = 3e-3;
  p->n_tau = 4;
  p->tau_scheme = SEDI_TAU_EULER;
  p->cg_rtol = 1e-8;
  p->cg_max_iter = 500;
  p->shift_eps = 40;
  p->shift_mom = 40;
  p->shift_force = 32;
  p->precision_form = SEDI_FORM_SPLIT;
  p->nbr_capacity = 32;
  p->use_graphs = 1;
  p->substep_variant = -1;
  p->bin_order = -1;
  p->n_beds = 1;
  p->cnn_scale[0] = p->cnn_scale[1] = p->cnn_scale[2] = p->cnn_scale[3] = 1.0;
}

int sedi_create(const sedi_params* p, sedi_handle** out) {
  if (!p || !out) return SEDI_EINVAL;
  *out = nullptr;
  sedi_handle* h = new sedi_handle();
  h->prm = *p;
  int rc = check_params(h, *p);
  if (rc) {
    std::string msg = h->err;
    delete h;
    (void)msg;
    return rc;
  }
  h->form = p->precision_form;
  h->variant = p->substep_variant >= 0 && h->form != FORM_FP64 ? p->substep_variant : SUBSTEP_B128_LOOP;
  // a lower limit on the smoother's grid-barrier waits, for failure-detection tests
  if (const char* lim = std::getenv("SEDI_BARRIER_SPIN_LIMIT")) {
    const long long v = std::atoll(lim);
    if (v > 0) h->barrier_spins = v;
  }
  fill_params(h);
  const int64_t C = h->P.C;
  h->U.assign(3 * C, 0.0);
  h->gp.assign(3 * C, 0.0);
  h->du.assign(3 * C, 0.0);
  h->eps.assign(C, 0.0);
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc((void**)&h->st.ctl, sizeof(Ctl)) != cudaSuccess) {
    delete h;
    return SEDI_ECUDA;
  }
  cudaMemset(h->st.ctl, 0, sizeof(Ctl));
  h->stream = h->own;
  h->mesh.C = C;
  const size_t fq = fquad_bytes(h->form);
  if ((rc = dmalloc(h, h->mesh_allocs, &h->mesh.ufe, fq * C)) ||
      (rc = dmalloc(h, h->mesh_allocs, &h->mesh.gfl, fq * C)) ||
      (rc = dmalloc(h, h->mesh_allocs, &h->mesh.wfl, fq * C)) ||
      (rc = dmalloc(h, h->mesh_allocs, (void**)&h->fdev, 72 * C)) ||
      (rc = dmalloc(h, h->mesh_allocs, (void**)&h->edev, 8 * C)) ||
      (rc = dmalloc(h, h->mesh_allocs, &h->qfix, 8 * 7 * C)) ||
      (rc = dmalloc(h, h->mesh_allocs, &h->phi, 8 * 8 * C)) ||
      (rc = dmalloc(h, h->mesh_allocs, (void**)&h->iters_dev, 4 * 8))) {
    sedi_destroy(h);
    return rc;
  }
  cudaMemset(h->mesh.wfl, 0, fq * C);  // no vorticity until a velocity field with lift
  cudaMemset(h->mesh.ufe, 0, fq * C);  // U = 0, eps_s = 0
  cudaMemset(h->fdev, 0, 72 * C);
  if ((rc = build_zgrid(h))) {
    sedi_destroy(h);
    return rc;
  }
  h->work_bytes = smooth_work_bytes(h->form, C, 8, h->prm.tau_scheme);
  if ((rc = dmalloc(h, h->mesh_allocs, &h->work, h->work_bytes))) {
    sedi_destroy(h);
    return rc;
  }
  if ((rc = upload_mesh(h))) {
    sedi_destroy(h);
    return rc;
  }
  if (p->n_beds > 1) {
    // one single-bed handle per bed, all on this handle's stream
    sedi_params q = *p;
    q.n_beds = 1;
    h->beds.assign(p->n_beds, nullptr);
    for (int b = 0; b < p->n_beds; ++b) {
      if ((rc = sedi_create(&q, &h->beds[b]))) {
        sedi_destroy(h);
        return rc;
      }
      h->beds[b]->stream = h->stream;
      h->beds[b]->is_bed = true;
    }
  }
  *out = h;
  return 0;
}

void sedi_destroy(sedi_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  clear_graphs(h);
  for (sedi_handle* b : h->beds) {
    if (!b) continue;
    b->stream = b->own;  // the shared stream belongs to the ensemble handle
    sedi_destroy(b);
  }
  h->beds.clear();
  for (void* p : {(void*)h->ens_views, h->ens_smooth, (void*)h->ens_iters, (void*)h->ens_ctl,
                  (void*)h->ens_done})
    if (p) cudaFree(p);
  for (cudaEvent_t e : h->avg_ev) cudaEventDestroy(e);
  free_list(h->part_allocs);
  free_list(h->bin_allocs);
  free_list(h->mesh_allocs);
  if (h->dstage) cudaFree(h->dstage);
  for (void* p : {(void*)h->cnn_master, (void*)h->cnn_m, (void*)h->cnn_v, (void*)h->cnn_grad,
                  (void*)h->cnn_target, (void*)h->cnn_loss, h->cnn_work})
    if (p) cudaFree(p);
  if (h->st.ctl) cudaFree(h->st.ctl);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->own) cudaStreamDestroy(h->own);
  delete h;
}

int sedi_set_stream(sedi_handle* h, void* s) {
  if (!h) return SEDI_EINVAL;
  if ((cudaStream_t)s != h->stream) clear_graphs(h);
  h->stream = (cudaStream_t)s;
  for (sedi_handle* b : h->beds) sedi_set_stream(b, s);
  return 0;
}

int sedi_set_bed(sedi_handle* h, int32_t bed, const double lo[3], const double hi[3],
                 const int32_t ncell[3]) {
  if (!h || !lo || !hi || !ncell) return SEDI_EINVAL;
  h->err.clear();
  if (h->beds.empty())
    return fail(h, SEDI_EINVAL, "sedi_set_bed needs n_beds > 1 (one bed takes its box from the parameters)");
  if (bed < 0 || bed >= (int32_t)h->beds.size()) return fail(h, SEDI_EINVAL, "bed %d out of range", bed);
  sedi_params q = h->beds[bed]->prm;
  for (int a = 0; a < 3; ++a) {
    q.lo[a] = lo[a];
    q.hi[a] = hi[a];
    q.ncell[a] = ncell[a];
  }
  sedi_handle* nb = nullptr;
  const int rc = sedi_create(&q, &nb);
  if (rc) return fail(h, rc, "bed %d: invalid box or mesh", bed);
  nb->stream = h->stream;
  nb->is_bed = true;
  sedi_handle* old = h->beds[bed];
  old->stream = old->own;
  cudaStreamSynchronize(h->stream);
  sedi_destroy(old);
  h->beds[bed] = nb;
  h->ens_dirty = true;
  h->ens_fresh = false;
  h->key_cache.clear();
  clear_graphs(h);
  return 0;
}

int sedi_set_particles(sedi_handle* h, int32_t bed, int64_t n, const int64_t* id, const double* x,
                       const double* v, const double* omega, const double* d, const double* rho,
                       int32_t mem) {
  if (!h) return SEDI_EINVAL;
  h->err.clear();
  if (!h->beds.empty()) {
    h->ens_dirty = true;
    h->ens_fresh = false;
    h->key_cache.clear();
    clear_graphs(h);
  }
  ENS_FORWARD(sedi_set_particles(sub, 0, n, id, x, v, omega, d, rho, mem));
  if (bed != 0) return fail(h, SEDI_EINVAL, "bed %d out of range", bed);
  if (n <= 0 || n > ((int64_t)1 << 31) - 1) return fail(h, SEDI_EINVAL, "n must be in [1, 2^31)");
  if (!x || !d || !rho) return fail(h, SEDI_EINVAL, "x, d and rho are required");
  // host copies of d, rho (bin size, checkpoint) and the caller's ids
  h->d_host.resize(n);
  h->rho_host.resize(n);
  std::vector<double> xh;
  if (mem == SEDI_MEM_DEVICE) {
    CK(cudaMemcpy(h->d_host.data(), d, 8 * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(h->rho_host.data(), rho, 8 * n, cudaMemcpyDeviceToHost));
    xh.resize(3 * n);
    CK(cudaMemcpy(xh.data(), x, 24 * n, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(h->d_host.data(), d, 8 * n);
    std::memcpy(h->rho_host.data(), rho, 8 * n);
    xh.assign(x, x + 3 * n);
  }
  double rmax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (!(h->d_host[i] > 0) || !(h->rho_host[i] > 0)) return fail(h, SEDI_EINVAL, "particle %lld: d and rho must be > 0", (long long)i);
    rmax = std::max(rmax, 0.5 * h->d_host[i]);
    for (int a = 0; a < 3; ++a) {
      const double c = xh[3 * i + a];
      if (!std::isfinite(c)) return fail(h, SEDI_EINVAL, "particle %lld: non-finite position", (long long)i);
      if (h->prm.periodic[a] && (c < h->prm.lo[a] || c >= h->prm.hi[a]))
        return fail(h, SEDI_EINVAL, "particle %lld: position outside [lo, hi) on periodic axis %d", (long long)i, a);
    }
  }
  h->ids.clear();
  if (id) {
    h->ids.resize(n);
    if (mem == SEDI_MEM_DEVICE) {
      CK(cudaMemcpy(h->ids.data(), id, 8 * n, cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(h->ids.data(), id, 8 * n);
    }
  }
  h->have_particles = false;
  int rc = alloc_particles(h, n, rmax);
  if (rc) return rc;
  h->N = n;
  // stage inputs (x, v, w, d, rho) in device doubles
  double* tmp = nullptr;
  CK(cudaMalloc((void**)&tmp, 8 * 11 * n));
  double *tx = tmp, *tv = tmp + 3 * n, *tw = tmp + 6 * n, *td = tmp + 9 * n, *tr = tmp + 10 * n;
  rc = copy_in(h, tx, xh.data(), 24 * n, SEDI_MEM_HOST);
  if (!rc && v) rc = copy_in(h, tv, v, 24 * n, mem);
  if (!rc && omega) rc = copy_in(h, tw, omega, 24 * n, mem);
  if (!rc) rc = copy_in(h, td, h->d_host.data(), 8 * n, SEDI_MEM_HOST);
  if (!rc) rc = copy_in(h, tr, h->rho_host.data(), 8 * n, SEDI_MEM_HOST);
  if (rc) {
    cudaFree(tmp);
    return rc;
  }
  Ctl zero{};
  cudaMemcpyAsync(h->st.ctl, &zero, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream);
  launch_import(h->form, h->st, tx, v ? tv : nullptr, omega ? tw : nullptr, td, tr, h->P, h->stream);
  rc = rebuild_now(h);
  cudaFree(tmp);
  if (rc) return rc;
  h->have_particles = true;
  h->since_set = 0;
  return 0;
}

int sedi_set_fluid(sedi_handle* h, int32_t bed, const int32_t ncell[3], const double* U,
                   const double* grad_p, const double* DUDt, int32_t mem) {
  if (!h) return SEDI_EINVAL;
  h->err.clear();
  ENS_FORWARD(sedi_set_fluid(sub, 0, ncell, U, grad_p, DUDt, mem));
  if (bed != 0) return fail(h, SEDI_EINVAL, "bed %d out of range", bed);
  if (!ncell || ncell[0] != h->prm.ncell[0] || ncell[1] != h->prm.ncell[1] || ncell[2] != h->prm.ncell[2])
    return fail(h, SEDI_EINVAL, "ncell must equal params.ncell");
  const int64_t C = h->P.C;
  // the caller's fields straight to the device (a pinned host buffer copies by DMA)
  const cudaMemcpyKind kind = mem == SEDI_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (U) CK(cudaMemcpyAsync(h->fdev, U, 24 * C, kind, h->stream));
  else CK(cudaMemsetAsync(h->fdev, 0, 24 * C, h->stream));
  h->gp_default = grad_p == nullptr;
  if (grad_p) CK(cudaMemcpyAsync(h->fdev + 3 * C, grad_p, 24 * C, kind, h->stream));
  if (DUDt) CK(cudaMemcpyAsync(h->fdev + 6 * C, DUDt, 24 * C, kind, h->stream));
  else CK(cudaMemsetAsync(h->fdev + 6 * C, 0, 24 * C, h->stream));
  h->fluid_host_stale = true;
  return upload_mesh(h);
}

int sedi_set_eps(sedi_handle* h, int32_t bed, const double* eps, int32_t mem) {
  if (!h || !eps) return SEDI_EINVAL;
  h->err.clear();
  ENS_FORWARD(sedi_set_eps(sub, 0, eps, mem));
  if (bed != 0) return fail(h, SEDI_EINVAL, "bed %d out of range", bed);
  const int64_t C = h->P.C;
  const cudaMemcpyKind kind = mem == SEDI_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(h->edev, eps, 8 * C, kind, h->stream));
  launch_eps_io(h->form, h->edev, h->mesh, C, 1, h->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  h->fluid_host_stale = true;
  return 0;
}

static int ens_step(sedi_handle* h, int n);
static int ens_status(sedi_handle* h);

int sedi_step(sedi_handle* h, int32_t n) {
  if (!h) return SEDI_EINVAL;
  h->err.clear();
  if (n < 0) return fail(h, SEDI_EINVAL, "n_substeps must be >= 0");
  if (!h->beds.empty()) return n == 0 ? 0 : ens_step(h, n);
  int rc = need_particles(h);
  if (rc) return rc;
  if (n == 0) return 0;
  if ((rc = autotune(h))) return rc;
  if (h->prm.profile) harvest(h);
  // stream capture needs a real stream: the legacy NULL stream runs without graphs
  if (h->prm.use_graphs && h->stream != nullptr) {
    auto it = h->graphs.find(n);
    cudaGraphExec_t ex;
    if (it == h->graphs.end()) {
      if ((rc = build_graph(h, n, &ex))) return rc;
      h->graphs[n] = ex;
    } else {
      ex = it->second;
    }
    CK(cudaGraphLaunch(ex, h->stream));
    if (h->prm.profile) {
      auto& ev = h->gev[n];
      for (int s = 0; s < n; ++s) {
        h->pending.push_back({0, {ev.a[s], ev.b[s]}});
        h->pending.push_back({1, {ev.b[s], ev.c[s]}});
      }
    }
  } else {
    if (h->prm.profile && h->gev.find(-n) == h->gev.end()) {
      sedi_handle::GraphEv ev;
      for (int s = 0; s < n; ++s) {
        ev.a.push_back(new_event());
        ev.b.push_back(new_event());
        ev.c.push_back(new_event());
      }
      h->gev[-n] = ev;
    }
    for (int s = 0; s < n; ++s) {
      if (h->prm.profile) CK(cudaEventRecord(h->gev[-n].a[s], h->stream));
      // the substep kernel's last block sets need_rebuild for the next substep
      if (s == 0) launch_check(h->st, h->P, 0ull, 0, h->stream);
      launch_rebuild(h->form, h->st, h->P, s, false, h->stream);
      if (h->prm.profile) CK(cudaEventRecord(h->gev[-n].b[s], h->stream));
      launch_substep(h->form, h->st, h->mesh, h->P, s, true, h->variant, 0ull, 0, h->stream);
      if (h->prm.profile) {
        CK(cudaEventRecord(h->gev[-n].c[s], h->stream));
        h->pending.push_back({0, {h->gev[-n].a[s], h->gev[-n].b[s]}});
        h->pending.push_back({1, {h->gev[-n].b[s], h->gev[-n].c[s]}});
      }
    }
    launch_advance_parity(h->st, n, h->stream);
  }
  CK(cudaGetLastError());
  h->stats.substeps += n;
  h->since_set += n;
  return 0;
}

int sedi_sync(sedi_handle* h) {
  if (!h) return SEDI_EINVAL;
  if (!h->beds.empty()) return ens_status(h);
  return sync_status(h);
}

// Deposition into h->qfix (split/FP64: int64; plain: float phi directly).
static int deposit_dev(sedi_handle* h) {
  const int64_t C = h->P.C;
  if (h->form == FORM_PLAIN) {
    CK(cudaMemsetAsync(h->phi, 0, 4 * 7 * C, h->stream));
    launch_deposit(h->form, h->st, h->mesh, h->P, h->phi, h->stream);
  } else {
    CK(cudaMemsetAsync(h->qfix, 0, 8 * 7 * C, h->stream));
    launch_deposit(h->form, h->st, h->mesh, h->P, h->qfix, h->stream);
  }
  CK(cudaGetLastError());
  return 0;
}

static int smooth_dev(sedi_handle* h, int nf, const void* guess, int n_tau = -1, bool zero_iters = true) {
  if (zero_iters) CK(cudaMemsetAsync(h->iters_dev, 0, 4 * 8, h->stream));
  // FP32 words cannot reach a relative residual much below 1e-6
  const double rtol = h->form == FORM_PLAIN ? std::max(h->prm.cg_rtol, 2e-6) : h->prm.cg_rtol;
  int rc = launch_smooth(h->form, h->P, h->phi, guess, nf, h->work, h->st, h->iters_dev,
                         rtol, h->prm.cg_max_iter, n_tau > 0 ? n_tau : h->prm.n_tau,
                         h->prm.tau_scheme, h->coef, h->P.graded ? &h->zs : nullptr,
                         h->stream, h->barrier_spins);
  if (rc) return fail(h, SEDI_ECUDA, "cooperative launch of the smoother failed: %s", cudaGetErrorString(cudaGetLastError()));
  return 0;
}

static int ensure_cnn(sedi_handle* h) {
  if (h->cnn_master) return 0;
  const size_t np = cnn_param_count();
  CK(cudaMalloc((void**)&h->cnn_master, np * sizeof(float)));
  CK(cudaMalloc((void**)&h->cnn_m, np * sizeof(float)));
  CK(cudaMalloc((void**)&h->cnn_v, np * sizeof(float)));
  CK(cudaMalloc((void**)&h->cnn_grad, np * sizeof(float)));
  CK(cudaMalloc((void**)&h->cnn_target, (size_t)h->P.C * 4 * sizeof(float)));
  CK(cudaMalloc(&h->cnn_work, cnn_work_bytes(h->P.C)));
  CK(cudaMemsetAsync(h->cnn_master, 0, np * sizeof(float), h->stream));
  CK(cudaMemsetAsync(h->cnn_m, 0, np * sizeof(float), h->stream));
  CK(cudaMemsetAsync(h->cnn_v, 0, np * sizeof(float), h->stream));
  return 0;
}

// One pseudo-step at a time: guess = phi + scale * net(phi / scale) on (eps, F),
// projected onto the conserved sum by the smoother, then solve to cg_rtol.
static int smooth_warm(sedi_handle* h) {
  int rc = ensure_cnn(h);
  if (rc) return rc;
  const int64_t C = h->P.C;
  const float scale[4] = {(float)h->prm.cnn_scale[0], (float)h->prm.cnn_scale[1],
                          (float)h->prm.cnn_scale[2], (float)h->prm.cnn_scale[3]};
  CK(cudaMemsetAsync(h->iters_dev, 0, 4 * 8, h->stream));
  for (int m = 0; m < h->prm.n_tau; ++m) {
    launch_phi_convert(h->form, h->phi, h->dstage, 7 * C, 1, h->stream);
    const double* f[4] = {h->dstage, h->dstage + 4 * C, h->dstage + 5 * C, h->dstage + 6 * C};
    cnn_input(h->P, f, scale, h->cnn_work, h->stream);
    float* y = nullptr;
    cnn_forward(h->P, h->cnn_master, h->cnn_work, &y, h->stream);
    cnn_guess(h->form, h->phi, y, scale, h->qfix, C, h->stream);
    if ((rc = smooth_dev(h, 7, h->qfix, 1, false))) return rc;
  }
  return 0;
}

static int smooth_status(sedi_handle* h, int nf) {
  int it[8] = {0};
  CK(cudaMemcpyAsync(it, h->iters_dev, 4 * 8, cudaMemcpyDeviceToHost, h->stream));
  int rc = sync_status(h);
  if (rc) return rc;
  Ctl c;
  CK(cudaMemcpy(&c, h->st.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  for (int f = 0; f < nf; ++f) h->stats.cg_iterations += it[f];
  int st = c.cg_status;
  int dr = c.deposit_range;
  if (st || dr) {
    int z = 0;
    cudaMemcpy((char*)h->st.ctl + offsetof(Ctl, deposit_range), &z, 4, cudaMemcpyHostToDevice);
    cudaMemcpy((char*)h->st.ctl + offsetof(Ctl, cg_status), &z, 4, cudaMemcpyHostToDevice);
  }
  if (dr) return fail(h, SEDI_ERANGE, "a deposited value does not fit the fixed-point format");
  if (st == SEDI_ETIMEOUT) return fail(h, SEDI_ETIMEOUT, "smoother grid barrier timed out");
  if (st == SEDI_EDIVERGED) return fail(h, SEDI_EDIVERGED, "smoothing CG reached cg_max_iter");
  return 0;
}


// ---------------------------------------------------------------- ensembles
// n_beds > 1: every bed is a single-bed handle (its own particles, box, mesh and
// control block); a step and an averaging are batched launches over all beds, the
// beds' views gathered in one device table.

// every bed shares the physics switches of the ensemble's parameters
static bool ens_ext(const sedi_handle* h) { return h->P.lift || h->P.lub_tangential; }

static int ens_finalize(sedi_handle* h) {
  for (size_t b = 0; b < h->beds.size(); ++b)
    if (!h->beds[b]->have_particles) return fail(h, SEDI_ESTATE, "bed %zu has no particles", b);
  if (!h->ens_dirty) return 0;
  const int B = (int)h->beds.size();
  std::vector<BedView> v(B);
  int64_t max_n = 0, max_bins = 0, max_c = 0, U = 0;
  for (int b = 0; b < B; ++b) {
    sedi_handle* sb = h->beds[b];
    v[b].st = sb->st;
    v[b].mesh = sb->mesh;
    v[b].P = sb->P;
    v[b].qfix = sb->qfix;
    v[b].phi = sb->phi;
    max_n = std::max(max_n, sb->N);
    max_bins = std::max(max_bins, sb->P.nbins);
    max_c = std::max(max_c, sb->P.C);
    U += smooth_units(sb->P.C);
  }
  for (void* p : {(void*)h->ens_views, h->ens_smooth, (void*)h->ens_iters, (void*)h->ens_ctl})
    if (p) cudaFree(p);
  h->ens_views = nullptr;
  h->ens_smooth = nullptr;
  h->ens_iters = nullptr;
  h->ens_ctl = nullptr;
  CK(cudaMalloc((void**)&h->ens_views, sizeof(BedView) * B));
  CK(cudaMalloc(&h->ens_smooth, smooth_batch_bytes(B, U)));
  CK(cudaMalloc((void**)&h->ens_iters, sizeof(int) * 8 * B));
  CK(cudaMalloc((void**)&h->ens_ctl, sizeof(Ctl) * B));
  CK(cudaMemcpy(h->ens_views, v.data(), sizeof(BedView) * B, cudaMemcpyHostToDevice));
  h->ens.views = h->ens_views;
  h->ens.B = B;
  h->ens.variant = h->ens_variant;
  h->ens.max_n = max_n;
  h->ens.max_bins = max_bins;
  h->ens.max_cells = max_c;
  h->ens.ectl = h->st.ctl;
  clear_graphs(h);
  h->ens_dirty = false;
  return 0;
}

// Synchronise; read every bed's control block; map device-side errors.
static int ens_status(sedi_handle* h) {
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  if (h->ens_dirty) return 0;
  const int B = h->ens.B;
  std::vector<Ctl> c(B);
  launch_ctl_gather_ens(h->ens, h->ens_ctl, h->stream);
  CK(cudaMemcpyAsync(c.data(), h->ens_ctl, sizeof(Ctl) * B, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int b = 0; b < B; ++b) {
    sedi_handle* sb = h->beds[b];
    sb->stats.rebuilds = c[b].rebuilds;
    sb->stats.max_neighbors = c[b].max_nn;
    if (c[b].error == SEDI_EOVERFLOW)
      return fail(h, SEDI_EOVERFLOW, "bed %d: a particle has %d listed neighbours > nbr_capacity %d", b,
                  c[b].overflow_nn, sb->P.cap);
    if (c[b].error == SEDI_ENONFINITE) return fail(h, SEDI_ENONFINITE, "bed %d: non-finite force or state", b);
    if (c[b].error) return fail(h, c[b].error, "bed %d: device error %d", b, c[b].error);
  }
  return 0;
}

// Ensembles: the launch shape of the batched substep (kEnsVariant) and the bins of
// every bed (R per list cutoff), tuned as for a single bed.  For each R every bed's
// bins are resized and all lists rebuilt at once (the batched rebuild, timed), then
// one batched substep of every shape is timed in interleaved rounds, the arrays it
// updates in place put back after each; cost = median substep + rebuild time x the
// largest rebuild rate of a bed.  No choice changes a result (lists in caller-index
// order, the same terms in the same order in every shape), so every bed keeps the bits
// it has alone.  Keyed by (GPU, beds, particles, diameter range, form, terms).
static int ens_autotune(sedi_handle* h) {
  if (h->prm.substep_variant >= 0 || h->form == FORM_FP64 || ens_ext(h)) return 0;
  const int B = (int)h->beds.size();
  int64_t since = INT64_MAX;
  for (sedi_handle* b : h->beds) since = std::min(since, b->since_set);
  if (since < kTuneAfter) return 0;
  // the key is computed once per set of beds (it reads every diameter)
  if (!h->key_cache.empty() && h->key_cache == h->tuned_key) return 0;
  int64_t ntot = 0, nmin = INT64_MAX, nmax = 0;
  double dmin = 1e300, dmax = 0.0;
  for (sedi_handle* b : h->beds) {
    ntot += b->N;
    nmin = std::min(nmin, b->N);
    nmax = std::max(nmax, b->N);
    for (double d : b->d_host) {
      dmin = std::min(dmin, d);
      dmax = std::max(dmax, d);
    }
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) std::snprintf(prop.name, sizeof(prop.name), "device%d", dev);
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s sm%d|ensemble B=%d|N=%lld (%lld..%lld)|d=%.3e..%.3e|form=%d|law=%d|lub=%d|fluid=%d%d%d",
                prop.name, prop.multiProcessorCount, B, (long long)ntot, (long long)nmin, (long long)nmax, dmin,
                dmax, h->form, h->prm.contact_law, h->P.lubrication, h->P.drag, h->P.pressure_grad,
                h->P.added_mass);
  const std::string key = buf;
  h->key_cache = key;
  if (key == h->tuned_key) return 0;
  int rc = ens_finalize(h);
  if (rc) return rc;
  TuneChoice best;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) best = it->second;
  }
  if (best.variant < 0) best = tune_file_lookup(key);
  // the rebuild counters as they stand (the tuner's rebuilds are not the run's)
  std::vector<Ctl> c(B);
  launch_ctl_gather_ens(h->ens, h->ens_ctl, h->stream);
  CK(cudaMemcpyAsync(c.data(), h->ens_ctl, sizeof(Ctl) * B, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  std::vector<int64_t> rebuilds(B);
  double rate = 0.0;
  for (int b = 0; b < B; ++b) {
    rebuilds[b] = c[b].rebuilds;
    rate = std::max(rate, (double)std::max<int64_t>(c[b].rebuilds, 1) / (double)std::max<int64_t>(h->beds[b]->since_set, 1));
  }
  int64_t* rb_dev = nullptr;
  CK(cudaMalloc((void**)&rb_dev, 8 * B));
  CK(cudaMemcpy(rb_dev, rebuilds.data(), 8 * B, cudaMemcpyHostToDevice));
  // every bed on the bins of a configuration, rebuilt now; returns the rebuild time (us)
  auto bins_and_rebuild = [&](const BinCfg& cfg, double* us) -> int {
    bool changed = false;
    for (sedi_handle* b : h->beds)
      if (bin_cfg(b) != cfg) {
        int r2 = apply_bins(b, cfg);
        if (r2) return fail(h, r2, "bed bins: %s", b->err.c_str());
        changed = true;
      }
    if (changed) {
      h->ens_dirty = true;
      int r2 = ens_finalize(h);
      if (r2) return r2;
    }
    cudaEvent_t e0 = new_event(), e1 = new_event();
    launch_force_need_ens(h->ens, h->stream);
    CK(cudaEventRecord(e0, h->stream));
    launch_rebuild_ens(h->form, h->ens, 0, h->stream);
    CK(cudaEventRecord(e1, h->stream));
    launch_set_rebuilds_ens(h->ens, rb_dev, h->stream);
    int r2 = ens_status(h);
    float ms = 0.0f;
    if (us) *us = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess ? 1e3 * ms : 0.0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return r2;
  };
  if (best.variant < 0) {
    std::vector<int> reaches = {1};
    bool two = h->prm.bins_per_cutoff == 0;
    for (sedi_handle* b : h->beds) {
      int32_t nb[3];
      int64_t nbins = 0;
      if (bins_for(b, 2, nb, &nbins) || nbins > std::max<int64_t>(16 * b->N, (int64_t)1 << 16)) two = false;
    }
    if (two) reaches.push_back(2);
    if (h->prm.bins_per_cutoff > 0) reaches = {h->prm.bins_per_cutoff};
    const BinCfg cur = bin_cfg(h->beds[0]);
    std::vector<BinCfg> cfgs;
    for (int R : reaches)
      for (int z = 0; z < 2; ++z) {
        if (h->prm.bin_order >= 0 && z != h->prm.bin_order) continue;
        BinCfg c;
        c.reach = R;
        c.zfast = z;
        if (c != cur) cfgs.push_back(c);
      }
    if (std::find(reaches.begin(), reaches.end(), cur.reach) != reaches.end() &&
        (h->prm.bin_order < 0 || cur.zfast == h->prm.bin_order))
      cfgs.push_back(cur);
    std::vector<std::vector<double>> med(cfgs.size(), std::vector<double>(kSubstepVariants, 1e30));
    std::vector<double> rebuild_us(cfgs.size(), 0.0);
    std::vector<cudaEvent_t> ev(2 * kEnsVariants * kTuneRounds, nullptr);
    for (auto& e : ev) e = new_event();
    for (size_t ri = 0; ri < cfgs.size() && !rc; ++ri) {
      if ((rc = bins_and_rebuild(cfgs[ri], &rebuild_us[ri]))) break;
      launch_ctl_gather_ens(h->ens, h->ens_ctl, h->stream);
      CK(cudaMemcpyAsync(c.data(), h->ens_ctl, sizeof(Ctl) * B, cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      // the arrays a substep updates in place, of every bed, and their saved copies
      struct Item { void* p; size_t n; };
      std::vector<Item> live;
      for (int b = 0; b < B; ++b) {
        sedi_handle* sb = h->beds[b];
        const int64_t N = sb->N, cap = sb->P.cap;
        const size_t q = quad_bytes(sb->form), fq = fquad_bytes(sb->form), w = word_bytes(sb->form);
        live.push_back({sb->st.hist[c[b].nl], q * cap * N});
        live.push_back({sb->st.cmask[c[b].nl], 4 * (size_t)N});
        live.push_back({sb->st.acc[c[b].pb], fq * N});
        live.push_back({sb->st.whist[c[b].pb], (size_t)kWalls * 3 * w * N});
        live.push_back({sb->st.wmask[c[b].pb], 4 * (size_t)N});
        live.push_back({sb->st.ctl, sizeof(Ctl)});
      }
      size_t total = 0;
      for (const auto& it : live) total += (it.n + 255) & ~(size_t)255;
      char* save = nullptr;
      if (cudaMalloc((void**)&save, total) != cudaSuccess) {
        cudaGetLastError();
        best.variant = h->ens_variant;
        best.bins = cfgs[ri];
        cfgs.resize(ri + 1);
        med.resize(ri + 1);
        rebuild_us.resize(ri + 1);
        med[ri].assign(kSubstepVariants, 1e30);
        med[ri][h->ens_variant] = 0.0;
        break;
      }
      auto copy_all = [&](bool to_save) {
        size_t off = 0;
        for (const auto& it : live) {
          if (to_save) cudaMemcpyAsync(save + off, it.p, it.n, cudaMemcpyDeviceToDevice, h->stream);
          else cudaMemcpyAsync(it.p, save + off, it.n, cudaMemcpyDeviceToDevice, h->stream);
          off += (it.n + 255) & ~(size_t)255;
        }
      };
      copy_all(true);
      EnsLaunch e = h->ens;
      for (int v = 0; v < kEnsVariants; ++v) {  // warm-up
        e.variant = kEnsVariant[v];
        launch_substep_ens(h->form, e, false, 0, 0ull, 0, h->stream);
        copy_all(false);
      }
      for (int r = 0; r < kTuneRounds; ++r)
        for (int v = 0; v < kEnsVariants; ++v) {
          cudaEvent_t* ee = &ev[2 * (r * kEnsVariants + v)];
          e.variant = kEnsVariant[v];
          CK(cudaEventRecord(ee[0], h->stream));
          launch_substep_ens(h->form, e, false, 0, 0ull, 0, h->stream);
          CK(cudaEventRecord(ee[1], h->stream));
          copy_all(false);
        }
      rc = ens_status(h);
      cudaFree(save);
      for (int v = 0; v < kEnsVariants && !rc; ++v) {
        std::vector<double> t;
        for (int r = 0; r < kTuneRounds; ++r) {
          float ms = 0.0f;
          cudaEvent_t* ee = &ev[2 * (r * kEnsVariants + v)];
          if (cudaEventElapsedTime(&ms, ee[0], ee[1]) != cudaSuccess) ms = 1e30f;
          t.push_back(1e3 * ms);
        }
        std::sort(t.begin(), t.end());
        med[ri][kEnsVariant[v]] = t[kTuneRounds / 2];
      }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (!rc) {
      double best_cost = 1e300;
      for (size_t ri = 0; ri < cfgs.size(); ++ri)
        for (int v = 0; v < kEnsVariants; ++v) {
          const double cost = med[ri][kEnsVariant[v]] + rebuild_us[ri] * rate;
          if (cost < best_cost) {
            best_cost = cost;
            best.variant = kEnsVariant[v];
            best.bins = cfgs[ri];
          }
        }
      tune_file_store(key, best, cfgs, med, rebuild_us);
    }
  }
  if (!rc && bin_cfg(h->beds[0]) != best.bins) rc = bins_and_rebuild(best.bins, nullptr);
  cudaFree(rb_dev);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  if (best.variant != h->ens_variant) clear_graphs(h);  // graphs bake in the launch shape
  h->ens_variant = best.variant;
  h->ens.variant = best.variant;
  h->tuned_key = key;
  return 0;
}

static int build_graph_ens(sedi_handle* h, int n, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  // one IF node per substep: rebuild the beds that need it (any bed -> condition)
  std::vector<cudaGraphConditionalHandle> ch(n);
  for (int s = 0; s < n; ++s) CK(cudaGraphConditionalHandleCreate(&ch[s], g, 0, cudaGraphCondAssignDefault));
  launch_check_ens(h->ens, (unsigned long long)ch[0], 1, h->stream);
  for (int s = 0; s < n; ++s) {
    CK(cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &g, &deps, nullptr, &nd));
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    std::memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams* cp = reinterpret_cast<cudaGraphNodeParams*>(raw);
    cp->type = cudaGraphNodeTypeConditional;
    cp->conditional.handle = ch[s];
    cp->conditional.type = cudaGraphCondTypeIf;
    cp->conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, cp));
    CK(cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = cp->conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(h->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch_rebuild_ens(h->form, h->ens, s, h->side);
    CK(cudaStreamEndCapture(h->side, &body));
    const bool more = s + 1 < n;
    launch_substep_ens(h->form, h->ens, ens_ext(h), s, more ? (unsigned long long)ch[s + 1] : 0ull, more ? 1 : 0,
                       h->stream);
  }
  launch_advance_ens(h->ens, n, h->stream);
  CK(cudaStreamEndCapture(h->stream, &graph));
  cudaError_t e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(h, SEDI_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  return 0;
}

static int ens_step(sedi_handle* h, int n) {
  int rc = ens_finalize(h);
  if (rc) return rc;
  if ((rc = ens_autotune(h))) return rc;
  if (h->prm.profile) {
    harvest(h);
    if (h->avg_ev.empty())
      for (int k = 0; k < 5; ++k) h->avg_ev.push_back(new_event());
    CK(cudaEventRecord(h->avg_ev[3], h->stream));
  }
  if (h->prm.ens_persistent && !ens_ext(h)) {
    // persistent launches: rebuild the beds that need it, then run substeps until one
    // leaves a bed needing a rebuild (or all are done)
    if (!h->ens_done) CK(cudaMalloc((void**)&h->ens_done, sizeof(int)));
    launch_check_ens(h->ens, 0ull, 0, h->stream);
    int s = 0;
    while (s < n) {
      launch_rebuild_ens(h->form, h->ens, s, h->stream);
      if (launch_substeps_persist_ens(h->form, h->ens, s, n, h->barrier_spins, h->ens_done, h->stream))
        return fail(h, SEDI_ECUDA, "persistent ensemble launch refused: %s", cudaGetErrorString(cudaGetLastError()));
      int done = 0;
      CK(cudaMemcpyAsync(&done, h->ens_done, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      if (done < 0) return fail(h, SEDI_ETIMEOUT, "persistent ensemble launch: a grid-barrier wait ran out");
      if (done <= s) return fail(h, SEDI_ECUDA, "persistent ensemble launch made no progress");
      s = done;
    }
    launch_advance_ens(h->ens, n, h->stream);
  } else if (h->prm.use_graphs && h->stream != nullptr) {
    auto it = h->graphs.find(n);
    cudaGraphExec_t ex;
    if (it == h->graphs.end()) {
      if ((rc = build_graph_ens(h, n, &ex))) return rc;
      h->graphs[n] = ex;
    } else {
      ex = it->second;
    }
    CK(cudaGraphLaunch(ex, h->stream));
  } else {
    launch_check_ens(h->ens, 0ull, 0, h->stream);
    for (int s = 0; s < n; ++s) {
      launch_rebuild_ens(h->form, h->ens, s, h->stream);
      launch_substep_ens(h->form, h->ens, ens_ext(h), s, 0ull, 0, h->stream);
    }
    launch_advance_ens(h->ens, n, h->stream);
  }
  if (h->prm.profile) {
    CK(cudaEventRecord(h->avg_ev[4], h->stream));
    h->pending.push_back({1, {h->avg_ev[3], h->avg_ev[4]}});
  }
  CK(cudaGetLastError());
  h->stats.substeps += n;
  for (sedi_handle* b : h->beds) {
    b->stats.substeps += n;
    b->since_set += n;
  }
  h->ens_fresh = false;
  return 0;
}

// Deposition and smoothing of every bed in batched launches; the smoothed eps
// feeds each bed's drag.  Outputs stay on the device.
static int ens_average(sedi_handle* h) {
  int rc = ens_finalize(h);
  if (rc) return rc;
  const int B = h->ens.B;
  if (h->prm.profile) {
    harvest(h);
    if (h->avg_ev.empty())
      for (int k = 0; k < 5; ++k) h->avg_ev.push_back(new_event());
    CK(cudaEventRecord(h->avg_ev[0], h->stream));
  }
  launch_deposit_ens(h->form, h->ens, h->stream);
  if (h->prm.profile) CK(cudaEventRecord(h->avg_ev[1], h->stream));
  std::vector<SmoothMesh> m(B);
  for (int b = 0; b < B; ++b) {
    sedi_handle* sb = h->beds[b];
    SmoothMesh& x = m[b];
    x.phi = sb->phi;
    x.guess = nullptr;
    x.work = sb->work;
    x.iters = h->ens_iters + 8 * b;
    x.C = sb->P.C;
    x.nf = 7;
    for (int a = 0; a < 3; ++a) {
      x.nc[a] = sb->P.nc[a];
      x.per[a] = sb->P.periodic[a];
      x.coef[a] = sb->coef[a];
    }
    x.z = sb->zs;
  }
  CK(cudaMemsetAsync(h->ens_iters, 0, sizeof(int) * 8 * B, h->stream));
  const double rtol = h->form == FORM_PLAIN ? std::max(h->prm.cg_rtol, 2e-6) : h->prm.cg_rtol;
  if (launch_smooth_batch(h->form, m.data(), B, 7, h->ens_smooth, rtol, h->prm.cg_max_iter,
                          h->prm.n_tau, h->prm.tau_scheme, h->st.ctl, 1 << 30, h->stream,
                          h->barrier_spins))
    return fail(h, SEDI_ECUDA, "cooperative launch of the batched smoother failed: %s",
                cudaGetErrorString(cudaGetLastError()));
  launch_eps_out_ens(h->form, h->ens, h->stream);
  if (h->prm.profile) {
    CK(cudaEventRecord(h->avg_ev[2], h->stream));
    h->pending.push_back({2, {h->avg_ev[0], h->avg_ev[1]}});
    h->pending.push_back({3, {h->avg_ev[1], h->avg_ev[2]}});
  }
  std::vector<int> it(8 * B);
  CK(cudaMemcpyAsync(it.data(), h->ens_iters, sizeof(int) * 8 * B, cudaMemcpyDeviceToHost, h->stream));
  if ((rc = ens_status(h))) return rc;
  Ctl ec;
  CK(cudaMemcpy(&ec, h->st.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  std::vector<Ctl> c(B);
  CK(cudaMemcpy(c.data(), h->ens_ctl, sizeof(Ctl) * B, cudaMemcpyDeviceToHost));
  int range_bed = -1;
  for (int b = 0; b < B; ++b) {
    sedi_handle* sb = h->beds[b];
    int64_t sum = 0;
    for (int f = 0; f < 7; ++f) sum += it[8 * b + f];
    sb->stats.cg_iterations += sum;
    h->stats.cg_iterations += sum;
    sb->stats.averages += 1;
    sb->fluid_host_stale = true;
    if (c[b].deposit_range) {
      range_bed = b;
      int z = 0;
      cudaMemcpy((char*)sb->st.ctl + offsetof(Ctl, deposit_range), &z, 4, cudaMemcpyHostToDevice);
    }
  }
  h->stats.averages += 1;
  if (ec.cg_status) {
    int z = 0;
    cudaMemcpy((char*)h->st.ctl + offsetof(Ctl, cg_status), &z, 4, cudaMemcpyHostToDevice);
  }
  if (range_bed >= 0) return fail(h, SEDI_ERANGE, "bed %d: a deposited value does not fit the fixed-point format", range_bed);
  if (ec.cg_status == SEDI_ETIMEOUT) return fail(h, SEDI_ETIMEOUT, "smoother grid barrier timed out");
  if (ec.cg_status == SEDI_EDIVERGED) return fail(h, SEDI_EDIVERGED, "smoothing reached cg_max_iter");
  h->ens_fresh = true;
  return 0;
}

// Outputs of the last averaging of a single-bed handle (smoothing word -> FP64).
static int average_outputs(sedi_handle* h, double* eps, double* Us, double* F, int32_t mem) {
  const int64_t C = h->P.C;
  double* de = h->dstage;
  double* du = h->dstage + C;
  double* dF = h->dstage + 4 * C;
  int rc;
  launch_average_out(h->form, h->phi, h->P, h->mesh.ufe, de, du, dF, h->stream);
  if (eps && (rc = copy_out(h, eps, de, 8 * C, mem))) return rc;
  if (Us && (rc = copy_out(h, Us, du, 24 * C, mem))) return rc;
  if (F && (rc = copy_out(h, F, dF, 24 * C, mem))) return rc;
  if ((rc = sync_status(h))) return rc;
  h->fluid_host_stale = true;
  return 0;
}

static int average_from_fixed(sedi_handle* h, double* eps, double* Us, double* F, int32_t mem);

int sedi_average(sedi_handle* h, int32_t bed, double* eps, double* Us, double* F, int32_t mem) {
  if (!h) return SEDI_EINVAL;
  h->err.clear();
  if (!h->beds.empty()) {
    if (bed == SEDI_ALL_BEDS) {
      if (eps || Us || F) return fail(h, SEDI_EINVAL, "SEDI_ALL_BEDS averages in place: outputs must be NULL");
      return ens_average(h);
    }
    if (bed < 0 || bed >= (int32_t)h->beds.size()) return fail(h, SEDI_EINVAL, "bed %d out of range", bed);
    int rc = h->ens_fresh ? 0 : ens_average(h);
    if (rc) return rc;
    sedi_handle* sb = h->beds[bed];
    rc = average_outputs(sb, eps, Us, F, mem);
    if (rc) h->err = sb->err;
    return rc;
  }
  int rc = need_particles(h);
  if (rc) return rc;
  if (bed != 0) return fail(h, SEDI_EINVAL, "bed %d out of range", bed);
  if (h->prm.profile) {
    harvest(h);
    if (h->avg_ev.empty())
      for (int k = 0; k < 3; ++k) h->avg_ev.push_back(new_event());
    CK(cudaEventRecord(h->avg_ev[0], h->stream));
  }
  if ((rc = deposit_dev(h))) return rc;
  return average_from_fixed(h, eps, Us, F, mem);
}

// The averaging after the deposition (in qfix, or phi in the plain form): fixed
// point -> smoothing word, n_tau smoothing steps, outputs.
static int average_from_fixed(sedi_handle* h, double* eps, double* Us, double* F, int32_t mem) {
  int rc = 0;
  const int64_t C = h->P.C;
  launch_fields_from_fixed(h->form, h->qfix, h->P, h->phi, 7, h->stream);
  if (h->prm.profile) CK(cudaEventRecord(h->avg_ev[1], h->stream));
  if (h->prm.use_cnn_guess && h->cnn_set) {
    if ((rc = smooth_warm(h))) return rc;
  } else if ((rc = smooth_dev(h, 7, nullptr))) {
    return rc;
  }
  if (h->prm.profile) {
    CK(cudaEventRecord(h->avg_ev[2], h->stream));
    h->pending.push_back({2, {h->avg_ev[0], h->avg_ev[1]}});
    h->pending.push_back({3, {h->avg_ev[1], h->avg_ev[2]}});
  }
  double* de = h->dstage;
  double* du = h->dstage + C;
  double* dF = h->dstage + 4 * C;
  launch_average_out(h->form, h->phi, h->P, h->mesh.ufe, de, du, dF, h->stream);
  if (eps && (rc = copy_out(h, eps, de, 8 * C, mem))) return rc;
  if (Us && (rc = copy_out(h, Us, du, 24 * C, mem))) return rc;
  if (F && (rc = copy_out(h, F, dF, 24 * C, mem))) return rc;
  h->stats.averages += 1;
  rc = smooth_status(h, 7);
  h->fluid_host_stale = true;
  return rc;
}

int sedi_average_deposit(sedi_handle* h, int32_t bed, const int64_t* q, double* eps, double* Us,
                         double* F, int32_t mem) {
  if (!h) return SEDI_EINVAL;
  h->err.clear();
  ENS_FORWARD(sedi_average_deposit(sub, 0, q, eps, Us, F, mem));
  int rc = need_particles(h);
  if (rc) return rc;
  if (bed != 0 || !q) return fail(h, SEDI_EINVAL, "bad bed or null deposit");
  if (h->form == FORM_PLAIN) return fail(h, SEDI_EINVAL, "the plain FP32 form deposits floats, not fixed point");
  if (h->prm.profile) {
    harvest(h);
    if (h->avg_ev.empty())
      for (int k = 0; k < 3; ++k) h->avg_ev.push_back(new_event());
    CK(cudaEventRecord(h->avg_ev[0], h->stream));
  }
  if ((rc = copy_in(h, h->qfix, q, 8 * 7 * h->P.C, mem))) return rc;
  return average_from_fixed(h, eps, Us, F, mem);
}

// ---------------------------------------------------------------- state import
int sedi_set_contacts(sedi_handle* h, int32_t bed, int64_t m, const int64_t* ij, const double* xi,
                      int32_t mem) {
  if (!h) return SEDI_EINVAL;
  h->err.clear();
  ENS_FORWARD(sedi_set_contacts(sub, 0, m, ij, xi, mem));
  int rc = need_particles(h);
  if (rc) return rc;
  if (bed != 0 || m < 0 || (m > 0 && (!ij || !xi))) return fail(h, SEDI_EINVAL, "bad contact table");
  std::vector<int64_t> hij(2 * m);
  std::vector<double> hxi(3 * m);
  if (m > 0) {
    if (mem == SEDI_MEM_DEVICE) {
      CK(cudaMemcpy(hij.data(), ij, 16 * m, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(hxi.data(), xi, 24 * m, cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(hij.data(), ij, 16 * m);
      std::memcpy(hxi.data(), xi, 24 * m);
    }
  }
  std::vector<int64_t> order(m);
  for (int64_t k = 0; k < m; ++k) {
    if (hij[2 * k] < 0 || hij[2 * k] >= hij[2 * k + 1] || hij[2 * k + 1] >= h->N)
      return fail(h, SEDI_EINVAL, "contact %lld: need 0 <= i < j < n", (long long)k);
    order[k] = k;
  }
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return hij[2 * a] != hij[2 * b] ? hij[2 * a] < hij[2 * b] : hij[2 * a + 1] < hij[2 * b + 1];
  });
  std::vector<int64_t> sij(2 * m);
  std::vector<double> sxi(3 * m);
  for (int64_t k = 0; k < m; ++k) {
    const int64_t o = order[k];
    if (k > 0 && hij[2 * o] == sij[2 * k - 2] && hij[2 * o + 1] == sij[2 * k - 1])
      return fail(h, SEDI_EINVAL, "contact (%lld, %lld) given twice", (long long)hij[2 * o], (long long)hij[2 * o + 1]);
    sij[2 * k] = hij[2 * o];
    sij[2 * k + 1] = hij[2 * o + 1];
    for (int a = 0; a < 3; ++a) sxi[3 * k + a] = hxi[3 * o + a];
  }
  int64_t* dij = nullptr;
  double* dxi = nullptr;
  CK(cudaMalloc((void**)&dij, 16 * std::max<int64_t>(m, 1)));
  CK(cudaMalloc((void**)&dxi, 24 * std::max<int64_t>(m, 1)));
  if (m > 0) {
    CK(cudaMemcpyAsync(dij, sij.data(), 16 * m, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(dxi, sxi.data(), 24 * m, cudaMemcpyHostToDevice, h->stream));
  }
  launch_springs_in(h->form, h->st, m, dij, dxi, h->stream);
  rc = sync_status(h);
  cudaFree(dij);
  cudaFree(dxi);
  return rc;
}

int sedi_set_accel(sedi_handle* h, int32_t bed, const double* a, int32_t mem) {
  if (!h) return SEDI_EINVAL;
  h->err.clear();
  ENS_FORWARD(sedi_set_accel(sub, 0, a, mem));
  int rc = need_particles(h);
  if (rc) return rc;
  if (bed != 0 || !a) return fail(h, SEDI_EINVAL, "bad bed or null accelerations");
  if ((rc = copy_in(h, h->dstage, a, 24 * h->N, mem))) return rc;
  launch_accel_in(h->form, h->st, h->dstage, h->stream);
  return sync_status(h);
}

static int wall_springs_io(sedi_handle* h, double* out, const double* in, int32_t mem) {
  int rc = need_particles(h);
  if (rc) return rc;
  double* tmp = nullptr;
  CK(cudaMalloc((void**)&tmp, 8 * 18 * h->N));
  if (in) rc = copy_in(h, tmp, in, 8 * 18 * h->N, mem);
  if (!rc) launch_wall_springs(h->form, h->st, in ? nullptr : tmp, in ? tmp : nullptr, h->stream);
  if (!rc && out) rc = copy_out(h, out, tmp, 8 * 18 * h->N, mem);
  if (!rc) rc = sync_status(h);
  cudaFree(tmp);
  return rc;
}

int sedi_get_wall_springs(sedi_handle* h, int32_t bed, double* xi_wall, int32_t mem) {
  if (!h) return SEDI_EINVAL;
  h->err.clear();
  ENS_FORWARD(sedi_get_wall_springs(sub, 0, xi_wall, mem));
  if (bed != 0 || !xi_wall) return fail(h, SEDI_EINVAL, "bad bed or null output");
  return wall_springs_io(h, xi_wall, nullptr, mem);
}

int sedi_set_wall_springs(sedi_handle* h, int32_t bed, const double* xi_wall, int32_t mem) {
  if (!h) return SEDI_EINVAL;
  h->err.clear();
  ENS_FORWARD(sedi_set_wall_springs(sub, 0, xi_wall, mem));
  if (bed != 0 || !xi_wall) return fail(h, SEDI_EINVAL, "bad bed or null input");
  return wall_springs_io(h, nullptr, xi_wall, mem);
}

int sedi_deposit(sedi_handle* h, int32_t bed, int64_t* q, int32_t mem) {
  if (!h) return SEDI_EINVAL;
  ENS_FORWARD(sedi_deposit(sub, 0, q, mem));
  int rc = need_particles(h);
  if (rc) return rc;
  h->err.clear();
  if (bed != 0 || !q) return fail(h, SEDI_EINVAL, "bad bed or null output");
  const int64_t C = h->P.C;
  if ((rc = deposit_dev(h))) return rc;
  if (h->form == FORM_PLAIN) {
    std::vector<float> f(7 * C);
    CK(cudaMemcpyAsync(f.data(), h->phi, 4 * 7 * C, cudaMemcpyDeviceToHost, h->stream));
    if ((rc = sync_status(h))) return rc;
    std::vector<int64_t> qq(7 * C);
    for (int k = 0; k < 7; ++k) {
      const double sc = h->P.two_shift[k == 0 ? 0 : (k < 4 ? 1 : 2)];
      for (int64_t c = 0; c < C; ++c) qq[k * C + c] = (int64_t)std::llrint((double)f[k * C + c] * sc);
    }
    if (mem == SEDI_MEM_DEVICE) {
      CK(cudaMemcpy(q, qq.data(), 8 * 7 * C, cudaMemcpyHostToDevice));
    } else {
      std::memcpy(q, qq.data(), 8 * 7 * C);
    }
    return 0;
  }
  if ((rc = copy_out(h, q, h->qfix, 8 * 7 * C, mem))) return rc;
  rc = sync_status(h);
  if (rc) return rc;
  Ctl c;
  CK(cudaMemcpy(&c, h->st.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  if (c.deposit_range) {
    int z = 0;
    cudaMemcpy((char*)h->st.ctl + offsetof(Ctl, deposit_range), &z, 4, cudaMemcpyHostToDevice);
    return fail(h, SEDI_ERANGE, "a deposited value does not fit the fixed-point format");
  }
  return 0;
}

int sedi_smooth(sedi_handle* h, int32_t bed, int32_t nf, const double* in, double* out,
                const double* guess, int32_t* iters, int32_t mem) {
  if (!h) return SEDI_EINVAL;
  ENS_FORWARD(sedi_smooth(sub, 0, nf, in, out, guess, iters, mem));
  if (!h) return SEDI_EINVAL;
  h->err.clear();
  if (bed != 0 || nf < 1 || nf > 8 || !in || !out) return fail(h, SEDI_EINVAL, "bad smoothing arguments (1 <= n_fields <= 8)");
  const int64_t C = h->P.C;
  const int64_t n = (int64_t)nf * C;
  int rc = ensure_stage(h, 2 * n);
  if (rc) return rc;
  const size_t wb = h->form == FORM_PLAIN ? 4 : 8;
  if ((rc = copy_in(h, h->dstage, in, 8 * n, mem))) return rc;
  launch_phi_from_double(h->form, h->dstage, h->phi, n, h->stream);
  void* gdev = nullptr;
  if (guess) {
    if ((rc = copy_in(h, h->dstage + n, guess, 8 * n, mem))) return rc;
    gdev = h->qfix;  // [7][C] int64 space reused as the guess buffer
    if (nf * C * wb > (size_t)8 * 7 * C) return fail(h, SEDI_EINVAL, "guess supports at most 7 fields");
    launch_phi_from_double(h->form, h->dstage + n, gdev, n, h->stream);
  }
  if ((rc = smooth_dev(h, nf, gdev))) return rc;
  launch_phi_convert(h->form, h->phi, h->dstage, n, 1, h->stream);
  if ((rc = copy_out(h, out, h->dstage, 8 * n, mem))) return rc;
  int it[8] = {0};
  CK(cudaMemcpyAsync(it, h->iters_dev, 4 * 8, cudaMemcpyDeviceToHost, h->stream));
  rc = smooth_status(h, nf);
  if (iters)
    for (int f = 0; f < nf; ++f) iters[f] = it[f];
  return rc;
}

int sedi_get_particles(sedi_handle* h, int32_t bed, double* x, double* v, double* w, double* a,
                       int32_t mem) {
  if (!h) return SEDI_EINVAL;
  ENS_FORWARD(sedi_get_particles(sub, 0, x, v, w, a, mem));
  int rc = need_particles(h);
  if (rc) return rc;
  h->err.clear();
  if (bed != 0) return fail(h, SEDI_EINVAL, "bed %d out of range", bed);
  const int64_t N = h->N;
  double* outs[4] = {x, v, w, a};
  for (int k = 0; k < 4; ++k) {
    if (!outs[k]) continue;
    launch_export(h->form, h->st, k, h->dstage + 3 * N * k, h->stream);
    if ((rc = copy_out(h, outs[k], h->dstage + 3 * N * k, 24 * N, mem))) return rc;
  }
  return sync_status(h);
}

int sedi_compute_forces(sedi_handle* h, int32_t bed, double* fc, double* fl, double* ff,
                        double* tq, int32_t mem) {
  if (!h) return SEDI_EINVAL;
  ENS_FORWARD(sedi_compute_forces(sub, 0, fc, fl, ff, tq, mem));
  int rc = need_particles(h);
  if (rc) return rc;
  h->err.clear();
  if (bed != 0) return fail(h, SEDI_EINVAL, "bed %d out of range", bed);
  const int64_t N = h->N;
  // lists must cover the current positions
  launch_check(h->st, h->P, 0ull, 0, h->stream);
  launch_rebuild(h->form, h->st, h->P, 0, false, h->stream);
  // pair-mode springs (ensembles, variant 8) to both slots: any variant may evaluate
  launch_spring_sync(h->form, h->st, h->stream);
  launch_substep(h->form, h->st, h->mesh, h->P, 0, false, h->variant, 0ull, 0, h->stream);
  // fdbg is in sorted order: scatter to caller order through the host
  std::vector<double> dbg(12 * N);
  std::vector<int32_t> uid(N);
  CK(cudaMemcpyAsync(dbg.data(), h->st.fdbg, 8 * 12 * N, cudaMemcpyDeviceToHost, h->stream));
  if ((rc = sync_status(h))) return rc;
  Ctl c;
  CK(cudaMemcpy(&c, h->st.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(uid.data(), h->st.uid[c.pb], 4 * N, cudaMemcpyDeviceToHost));
  double* outs[4] = {fc, fl, ff, tq};
  std::vector<double> tmp(3 * N);
  for (int k = 0; k < 4; ++k) {
    if (!outs[k]) continue;
    for (int64_t i = 0; i < N; ++i)
      for (int a = 0; a < 3; ++a) tmp[3 * uid[i] + a] = dbg[3 * N * k + 3 * i + a];
    if (mem == SEDI_MEM_DEVICE) {
      CK(cudaMemcpy(outs[k], tmp.data(), 24 * N, cudaMemcpyHostToDevice));
    } else {
      std::memcpy(outs[k], tmp.data(), 24 * N);
    }
  }
  return 0;
}

int64_t sedi_get_neighbors(sedi_handle* h, int32_t bed, int64_t* offsets, int64_t* ids, int64_t cap) {
  if (!h) return SEDI_EINVAL;
  ENS_FORWARD(sedi_get_neighbors(sub, 0, offsets, ids, cap));
  int rc = need_particles(h);
  if (rc) return rc;
  h->err.clear();
  if (bed != 0 || !offsets) return fail(h, SEDI_EINVAL, "bad arguments");
  const int64_t N = h->N;
  int64_t* dcnt = nullptr;
  CK(cudaMalloc((void**)&dcnt, 8 * (N + 1)));
  launch_neighbors_export(h->st, dcnt, h->stream);
  std::vector<int64_t> cnt(N);
  cudaMemcpyAsync(cnt.data(), dcnt, 8 * N, cudaMemcpyDeviceToHost, h->stream);
  if ((rc = sync_status(h))) {
    cudaFree(dcnt);
    return rc;
  }
  offsets[0] = 0;
  for (int64_t i = 0; i < N; ++i) offsets[i + 1] = offsets[i] + cnt[i];
  const int64_t total = offsets[N];
  if (!ids || total > cap) {
    cudaFree(dcnt);
    return ids ? fail(h, SEDI_EOVERFLOW, "cap %lld < %lld entries", (long long)cap, (long long)total) : total;
  }
  int64_t* dout = nullptr;
  if (cudaMalloc((void**)&dout, 8 * std::max<int64_t>(total, 1)) != cudaSuccess) {
    cudaFree(dcnt);
    return fail(h, SEDI_ENOMEM, "neighbour export buffer");
  }
  cudaMemcpyAsync(dcnt, offsets, 8 * (N + 1), cudaMemcpyHostToDevice, h->stream);
  launch_neighbors_fill(h->st, dcnt, dout, h->stream);
  cudaMemcpyAsync(ids, dout, 8 * total, cudaMemcpyDeviceToHost, h->stream);
  rc = sync_status(h);
  cudaFree(dout);
  cudaFree(dcnt);
  if (rc) return rc;
  if (!h->ids.empty())
    for (int64_t k = 0; k < total; ++k) ids[k] = h->ids[ids[k]];
  return total;
}

int64_t sedi_get_contacts(sedi_handle* h, int32_t bed, int64_t cap, int64_t* ij, double* xi) {
  if (!h) return SEDI_EINVAL;
  ENS_FORWARD(sedi_get_contacts(sub, 0, cap, ij, xi));
  int rc = need_particles(h);
  if (rc) return rc;
  h->err.clear();
  if (bed != 0) return fail(h, SEDI_EINVAL, "bad bed");
  unsigned long long* dc = nullptr;
  int64_t* dij = nullptr;
  double* dxi = nullptr;
  const int64_t c2 = std::max<int64_t>(cap, 1);
  CK(cudaMalloc((void**)&dc, 8));
  CK(cudaMalloc((void**)&dij, 16 * c2));
  CK(cudaMalloc((void**)&dxi, 24 * c2));
  cudaMemsetAsync(dc, 0, 8, h->stream);
  launch_spring_sync(h->form, h->st, h->stream);  // pair-mode springs to both slots
  launch_contacts_export(h->form, h->st, h->P, dc, cap, dij, dxi, h->stream);
  unsigned long long m = 0;
  cudaMemcpyAsync(&m, dc, 8, cudaMemcpyDeviceToHost, h->stream);
  rc = sync_status(h);
  std::vector<int64_t> vij;
  std::vector<double> vxi;
  if (!rc && (int64_t)m <= cap && m > 0) {
    vij.resize(2 * m);
    vxi.resize(3 * m);
    cudaMemcpy(vij.data(), dij, 16 * m, cudaMemcpyDeviceToHost);
    cudaMemcpy(vxi.data(), dxi, 24 * m, cudaMemcpyDeviceToHost);
  }
  cudaFree(dc);
  cudaFree(dij);
  cudaFree(dxi);
  if (rc) return rc;
  if ((int64_t)m > cap) return fail(h, SEDI_EOVERFLOW, "%llu contacts > cap", m);
  std::vector<int64_t> order(m);
  for (int64_t k = 0; k < (int64_t)m; ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return vij[2 * a] != vij[2 * b] ? vij[2 * a] < vij[2 * b] : vij[2 * a + 1] < vij[2 * b + 1];
  });
  for (int64_t k = 0; k < (int64_t)m; ++k) {
    const int64_t o = order[k];
    if (ij) {
      ij[2 * k] = vij[2 * o];
      ij[2 * k + 1] = vij[2 * o + 1];
    }
    if (xi)
      for (int a = 0; a < 3; ++a) xi[3 * k + a] = vxi[3 * o + a];
  }
  return (int64_t)m;
}

// ---------------------------------------------------------------- checkpoints
// Raw device words of the current buffers, so a resumed run is bit-identical.
namespace {
struct CkHeader {
  char magic[8];
  int32_t version, form, cap;
  int32_t bins_per_cutoff;  // R | z-fastest << 8 of the stored order (0 in older files: 1, x)
  int64_t N, C, nbins;
  sedi_stats stats;
};

int ck_write(FILE* f, const void* p, size_t n) { return fwrite(p, 1, n, f) == n ? 0 : -1; }
int ck_read(FILE* f, void* p, size_t n) { return fread(p, 1, n, f) == n ? 0 : -1; }

int dev_io(sedi_handle* h, FILE* f, void* dptr, size_t bytes, bool save) {
  std::vector<char> buf(bytes);
  if (save) {
    CK(cudaMemcpy(buf.data(), dptr, bytes, cudaMemcpyDeviceToHost));
    if (ck_write(f, buf.data(), bytes)) return fail(h, SEDI_EIO, "checkpoint write failed");
  } else {
    if (ck_read(f, buf.data(), bytes)) return fail(h, SEDI_EIO, "checkpoint read failed");
    CK(cudaMemcpy(dptr, buf.data(), bytes, cudaMemcpyHostToDevice));
  }
  return 0;
}

int state_io(sedi_handle* h, FILE* f, bool save) {
  const int64_t N = h->N, C = h->P.C, cap = h->P.cap;
  const size_t q = quad_bytes(h->form), fq = fquad_bytes(h->form), w = word_bytes(h->form);
  Ctl c;
  CK(cudaMemcpy(&c, h->st.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  int rc;
  DevState& s = h->st;
  struct Item { void* p; size_t n; };
  std::vector<Item> items = {
      {s.pos[c.st], q * N}, {s.vel[c.st], q * N}, {s.omg[c.st], q * N},
      {s.acc[c.pb], fq * N}, {s.uid[c.pb], 4 * (size_t)N}, {s.r64[c.pb], 8 * (size_t)N},
      {s.vfrac[c.pb], 8 * (size_t)N}, {s.xb[c.pb], 16 * (size_t)N},
      {s.whist[c.pb], (size_t)kWalls * 3 * w * N}, {s.wmask[c.pb], 4 * (size_t)N},
      {s.nbr[c.nl], 4 * (size_t)cap * N}, {s.nn[c.nl], 4 * (size_t)N},
      {s.hist[c.nl], q * cap * N}, {s.cmask[c.nl], 4 * (size_t)N},
      {h->mesh.ufe, fq * C}, {h->mesh.gfl, fq * C}, {h->mesh.wfl, fq * C}};
  for (auto& it : items)
    if ((rc = dev_io(h, f, it.p, it.n, save))) return rc;
  if (save) {
    if (ck_write(f, &c, sizeof(Ctl))) return fail(h, SEDI_EIO, "checkpoint write failed");
  } else {
    Ctl in;
    if (ck_read(f, &in, sizeof(Ctl))) return fail(h, SEDI_EIO, "checkpoint read failed");
    // keep the buffer parities of this handle (data were loaded into them)
    in.st = c.st;
    in.pb = c.pb;
    in.nl = c.nl;
    CK(cudaMemcpy(h->st.ctl, &in, sizeof(Ctl), cudaMemcpyHostToDevice));
  }
  return 0;
}
}  // namespace

static int save_to(sedi_handle* h, FILE* f) {
  int rc = need_particles(h);
  if (rc) return rc;
  launch_spring_sync(h->form, h->st, h->stream);  // pair-mode springs to both slots
  if ((rc = sync_status(h)) || (rc = refresh_fluid_host(h))) return rc;
  CkHeader hd{};
  std::memcpy(hd.magic, "SEDICK01", 8);
  hd.version = 1;
  hd.form = h->form;
  hd.cap = h->P.cap;
  hd.N = h->N;
  hd.C = h->P.C;
  hd.nbins = h->P.nbins;
  hd.bins_per_cutoff = bin_cfg(h).reach | (bin_cfg(h).zfast << 8);
  hd.stats = h->stats;
  rc = ck_write(f, &hd, sizeof(hd)) ? fail(h, SEDI_EIO, "write failed") : 0;
  if (!rc) rc = ck_write(f, h->d_host.data(), 8 * h->N) || ck_write(f, h->rho_host.data(), 8 * h->N) ? fail(h, SEDI_EIO, "write failed") : 0;
  int64_t nid = (int64_t)h->ids.size();
  if (!rc) rc = ck_write(f, &nid, 8) ? fail(h, SEDI_EIO, "write failed") : 0;
  if (!rc && nid) rc = ck_write(f, h->ids.data(), 8 * nid) ? fail(h, SEDI_EIO, "write failed") : 0;
  const int64_t C = h->P.C;
  if (!rc) rc = (ck_write(f, h->U.data(), 24 * C) || ck_write(f, h->gp.data(), 24 * C) ||
                 ck_write(f, h->du.data(), 24 * C) || ck_write(f, h->eps.data(), 8 * C))
                    ? fail(h, SEDI_EIO, "write failed") : 0;
  int gpd = h->gp_default ? 1 : 0;
  if (!rc) rc = ck_write(f, &gpd, 4) ? fail(h, SEDI_EIO, "write failed") : 0;
  if (!rc) rc = state_io(h, f, true);
  return rc;
}

static int load_from(sedi_handle* h, FILE* f) {
  CkHeader hd{};
  int rc = 0;
  if (ck_read(f, &hd, sizeof(hd)) || std::memcmp(hd.magic, "SEDICK01", 8) != 0) rc = fail(h, SEDI_EIO, "not a checkpoint of this library");
  if (!rc && (hd.form != h->form || hd.C != h->P.C))
    rc = fail(h, SEDI_EINVAL, "checkpoint form/mesh differ from this handle");
  std::vector<double> d, rho;
  std::vector<int64_t> ids;
  if (!rc) {
    d.resize(hd.N);
    rho.resize(hd.N);
    if (ck_read(f, d.data(), 8 * hd.N) || ck_read(f, rho.data(), 8 * hd.N)) rc = fail(h, SEDI_EIO, "read failed");
  }
  int64_t nid = 0;
  if (!rc && ck_read(f, &nid, 8)) rc = fail(h, SEDI_EIO, "read failed");
  if (!rc && nid) {
    ids.resize(nid);
    if (ck_read(f, ids.data(), 8 * nid)) rc = fail(h, SEDI_EIO, "read failed");
  }
  const int64_t C = h->P.C;
  int gpd = 1;
  if (!rc && (ck_read(f, h->U.data(), 24 * C) || ck_read(f, h->gp.data(), 24 * C) ||
              ck_read(f, h->du.data(), 24 * C) || ck_read(f, h->eps.data(), 8 * C) || ck_read(f, &gpd, 4)))
    rc = fail(h, SEDI_EIO, "read failed");
  if (!rc) {
    h->gp_default = gpd != 0;
    // the fluid fields back on the device (the mesh words come with the state below)
    CK(cudaMemcpy(h->fdev, h->U.data(), 24 * C, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->fdev + 3 * C, h->gp.data(), 24 * C, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->fdev + 6 * C, h->du.data(), 24 * C, cudaMemcpyHostToDevice));
    h->fluid_host_stale = false;
    double rmax = 0;
    for (double di : d) rmax = std::max(rmax, 0.5 * di);
    h->P.cap = hd.cap;
    h->have_particles = false;
    rc = alloc_particles(h, hd.N, rmax);
    // the stored order and lists follow the stored bins
    BinCfg stored;
    stored.reach = (hd.bins_per_cutoff & 0xff) > 0 ? (hd.bins_per_cutoff & 0xff) : 1;
    stored.zfast = (hd.bins_per_cutoff >> 8) & 1;
    if (!rc) rc = apply_bins(h, stored);
    if (!rc && h->P.nbins != hd.nbins) rc = fail(h, SEDI_EINVAL, "checkpoint binning differs");
  }
  if (!rc) {
    h->N = hd.N;
    h->d_host = d;
    h->rho_host = rho;
    h->ids = ids;
    Ctl zero{};
    cudaMemcpy(h->st.ctl, &zero, sizeof(Ctl), cudaMemcpyHostToDevice);
    rc = state_io(h, f, false);
  }
  if (rc) return rc;
  // the pair list follows the loaded neighbour lists
  launch_pair_list(h->st, h->P, h->stream);
  CK(cudaStreamSynchronize(h->stream));
  h->stats = hd.stats;
  h->have_particles = true;
  return 0;
}

// Ensemble checkpoints: a header with the bed count, then every bed's checkpoint.
struct EnsHeader {
  char magic[8];
  int32_t beds, pad;
  sedi_stats stats;
};

int sedi_save_state(sedi_handle* h, const char* path) {
  if (!h || !path) return SEDI_EINVAL;
  h->err.clear();
  int rc = h->beds.empty() ? need_particles(h) : ens_status(h);
  if (rc) return rc;
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(h, SEDI_EIO, "cannot open %s", path);
  if (h->beds.empty()) {
    rc = save_to(h, f);
  } else {
    EnsHeader eh{};
    std::memcpy(eh.magic, "SEDIEN01", 8);
    eh.beds = (int32_t)h->beds.size();
    eh.stats = h->stats;
    rc = ck_write(f, &eh, sizeof(eh)) ? fail(h, SEDI_EIO, "write failed") : 0;
    for (size_t b = 0; !rc && b < h->beds.size(); ++b)
      if ((rc = save_to(h->beds[b], f))) h->err = h->beds[b]->err;
  }
  std::fclose(f);
  return rc;
}

int sedi_load_state(sedi_handle* h, const char* path) {
  if (!h || !path) return SEDI_EINVAL;
  h->err.clear();
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(h, SEDI_EIO, "cannot open %s", path);
  int rc = 0;
  if (h->beds.empty()) {
    rc = load_from(h, f);
  } else {
    EnsHeader eh{};
    if (ck_read(f, &eh, sizeof(eh)) || std::memcmp(eh.magic, "SEDIEN01", 8) != 0)
      rc = fail(h, SEDI_EIO, "not an ensemble checkpoint of this library");
    else if (eh.beds != (int32_t)h->beds.size())
      rc = fail(h, SEDI_EINVAL, "checkpoint has %d beds, this handle %zu", eh.beds, h->beds.size());
    for (size_t b = 0; !rc && b < h->beds.size(); ++b)
      if ((rc = load_from(h->beds[b], f))) h->err = h->beds[b]->err;
    if (!rc) h->stats = eh.stats;
    h->ens_dirty = true;
    h->ens_fresh = false;
    h->key_cache.clear();
    clear_graphs(h);
  }
  std::fclose(f);
  return rc;
}

int sedi_cnn_set_params(sedi_handle* h, const double* params, int64_t n) {
  if (!h || !params) return SEDI_EINVAL;
  h->err.clear();
  if (n != (int64_t)cnn_param_count()) return fail(h, SEDI_EINVAL, "expected %zu parameters", cnn_param_count());
  int rc = ensure_cnn(h);
  if (rc) return rc;
  std::vector<float> f(n);
  for (int64_t k = 0; k < n; ++k) f[k] = (float)params[k];
  CK(cudaMemcpyAsync(h->cnn_master, f.data(), n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemsetAsync(h->cnn_m, 0, n * sizeof(float), h->stream));
  CK(cudaMemsetAsync(h->cnn_v, 0, n * sizeof(float), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->cnn_steps = 0;
  h->cnn_set = true;
  return 0;
}

int sedi_cnn_get_params(sedi_handle* h, double* params, int64_t n) {
  if (!h || !params) return SEDI_EINVAL;
  h->err.clear();
  if (n != (int64_t)cnn_param_count()) return fail(h, SEDI_EINVAL, "expected %zu parameters", cnn_param_count());
  if (!h->cnn_set) return fail(h, SEDI_ESTATE, "no network parameters set");
  std::vector<float> f(n);
  CK(cudaMemcpyAsync(f.data(), h->cnn_master, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int64_t k = 0; k < n; ++k) params[k] = f[k];
  return 0;
}

static int cnn_stage_input(sedi_handle* h, const double* x, int32_t mem) {
  const int64_t C = h->P.C;
  int rc = ensure_stage(h, 8 * C);
  if (rc) return rc;
  if ((rc = copy_in(h, h->dstage, x, 8 * 4 * C, mem))) return rc;
  const double* f[4] = {h->dstage, h->dstage + C, h->dstage + 2 * C, h->dstage + 3 * C};
  const float one[4] = {1, 1, 1, 1};
  cnn_input(h->P, f, one, h->cnn_work, h->stream);
  return 0;
}

int sedi_cnn_forward(sedi_handle* h, const double* x, double* y, int32_t mem) {
  if (!h || !x || !y) return SEDI_EINVAL;
  h->err.clear();
  if (!h->cnn_set) return fail(h, SEDI_ESTATE, "no network parameters set");
  const int64_t C = h->P.C;
  int rc = cnn_stage_input(h, x, mem);
  if (rc) return rc;
  float* yd = nullptr;
  cnn_forward(h->P, h->cnn_master, h->cnn_work, &yd, h->stream);
  cnn_vec_to_chan_first(yd, h->dstage + 4 * C, C, 4, h->stream);
  if ((rc = copy_out(h, y, h->dstage + 4 * C, 8 * 4 * C, mem))) return rc;
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  return 0;
}

int sedi_cnn_loss_grad(sedi_handle* h, const double* x, const double* target, double* grad,
                       double* loss, int32_t mem) {
  if (!h || !x || !target) return SEDI_EINVAL;
  h->err.clear();
  if (!h->cnn_set) return fail(h, SEDI_ESTATE, "no network parameters set");
  const int64_t C = h->P.C;
  int rc = cnn_stage_input(h, x, mem);
  if (rc) return rc;
  if ((rc = copy_in(h, h->dstage + 4 * C, target, 8 * 4 * C, mem))) return rc;
  cnn_chan_first_to_vec(h->dstage + 4 * C, h->cnn_target, C, 4, h->stream);
  if (!h->cnn_loss) CK(cudaMalloc((void**)&h->cnn_loss, 8 * 4096));
  cnn_loss_grad(h->P, h->cnn_master, h->cnn_target, h->cnn_grad, h->cnn_loss, h->cnn_work, h->stream);
  const size_t np = cnn_param_count();
  std::vector<float> g(np);
  double l = 0;
  CK(cudaMemcpyAsync(g.data(), h->cnn_grad, np * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&l, h->cnn_loss, 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  if (grad)
    for (size_t k = 0; k < np; ++k) grad[k] = g[k];
  if (loss) *loss = l;
  return 0;
}

int sedi_cnn_train(sedi_handle* h, int32_t n_pairs, const double* x, const double* target,
                   int32_t steps, double lr, double* losses, int32_t mem) {
  if (!h || !x || !target || n_pairs < 1 || steps < 0) return SEDI_EINVAL;
  h->err.clear();
  if (!h->cnn_set) return fail(h, SEDI_ESTATE, "no network parameters set");
  const int64_t C = h->P.C;
  double* dx = nullptr;
  double* dt = nullptr;
  if (!h->cnn_loss) CK(cudaMalloc((void**)&h->cnn_loss, 8 * 4096));
  CK(cudaMalloc((void**)&dx, 8 * 4 * C * (size_t)n_pairs));
  CK(cudaMalloc((void**)&dt, 8 * 4 * C * (size_t)n_pairs));
  int rc = copy_in(h, dx, x, 8 * 4 * C * (size_t)n_pairs, mem);
  if (!rc) rc = copy_in(h, dt, target, 8 * 4 * C * (size_t)n_pairs, mem);
  std::vector<double> lh(steps);
  const float one[4] = {1, 1, 1, 1};
  for (int32_t k = 0; k < steps && !rc; k += 4096) {
    const int32_t kn = std::min<int32_t>(steps - k, 4096);
    for (int32_t j = 0; j < kn; ++j) {
      const int64_t pr = (k + j) % n_pairs;
      const double* xp = dx + pr * 4 * C;
      const double* f[4] = {xp, xp + C, xp + 2 * C, xp + 3 * C};
      cnn_input(h->P, f, one, h->cnn_work, h->stream);
      cnn_chan_first_to_vec(dt + pr * 4 * C, h->cnn_target, C, 4, h->stream);
      cnn_loss_grad(h->P, h->cnn_master, h->cnn_target, h->cnn_grad, h->cnn_loss + j, h->cnn_work, h->stream);
      cnn_adam(h->cnn_master, h->cnn_grad, h->cnn_m, h->cnn_v, ++h->cnn_steps, (float)lr, h->stream);
    }
    if (cudaMemcpyAsync(lh.data() + k, h->cnn_loss, 8 * kn, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
      rc = fail(h, SEDI_ECUDA, "loss copy failed");
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = fail(h, SEDI_ECUDA, "training step failed");
  }
  cudaFree(dx);
  cudaFree(dt);
  if (rc) return rc;
  CK(cudaGetLastError());
  if (losses)
    for (int32_t k = 0; k < steps; ++k) losses[k] = lh[k];
  return 0;
}

int sedi_get_timings(sedi_handle* h, double* ms, int32_t n) {
  if (!h || !ms) return SEDI_EINVAL;
  if (!h->prm.profile) return 0;
  harvest(h);
  int k = 0;
  for (; k < n && k < 8; ++k) ms[k] = k < 4 ? h->ms[k] : h->cnt[k - 4];
  return k;
}

int sedi_get_stats(sedi_handle* h, sedi_stats* out) {
  if (!h || !out) return SEDI_EINVAL;
  if (!h->beds.empty()) {
    // ensemble: substeps, averages and smoother steps of the whole ensemble, list
    // rebuilds summed and the longest list over the beds
    const int rc = ens_status(h);
    sedi_stats st = h->stats;
    st.rebuilds = 0;
    st.max_neighbors = 0;
    for (sedi_handle* b : h->beds) {
      st.rebuilds += b->stats.rebuilds;
      st.max_neighbors = std::max(st.max_neighbors, b->stats.max_neighbors);
    }
    st.nbr_capacity = h->P.cap;
    st.substep_variant = h->ens_variant;
    st.substep_block = substep_block(h->ens_variant);
    st.bins_per_cutoff = bin_cfg(h->beds[0]).reach;
    st.bin_order = bin_cfg(h->beds[0]).zfast;
    *out = st;
    return rc;
  }
  int rc = h->have_particles ? sync_status(h) : 0;
  h->stats.nbr_capacity = h->P.cap;
  const bool tuned = h->prm.substep_variant >= 0 || h->form == FORM_FP64 || !h->tuned_key.empty();
  h->stats.substep_variant = tuned ? h->variant : -1;
  h->stats.substep_block = tuned ? substep_block(h->variant) : 0;
  h->stats.bins_per_cutoff = bin_cfg(h).reach;
  h->stats.bin_order = bin_cfg(h).zfast;
  *out = h->stats;
  return rc;
}

const char* sedi_last_error(const sedi_handle* h) { return h ? h->err.c_str() : "null handle"; }

}  // extern "C"
