// Diffusion-based averaging (Sec. 2.4, Eq. 9-10).
//
// Deposition (Eq. 9, PCM): each particle adds V_p/V_c, V_p u_p/V_c and
// -f_fp/V_c to the cell holding its centre.  The split and FP64 forms round each
// value to 64-bit fixed point (round to nearest even, one exponent per field kind)
// and add with integer atomics, so the sums do not depend on the order of the
// additions and match an exact integer sum bit for bit.  The plain FP32 form adds
// floats.
//
// Smoothing (Eq. 10) runs in k_smooth.cu; this file also converts the fixed-point
// sums to the smoothing word and writes the outputs.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "../../include/sedi.h"
#include "common.cuh"
#include "fluid.cuh"
#include "kernels.h"

namespace sedi {

namespace {

constexpr int kMaxF = 8;

// ---------------------------------------------------------------- deposition
template <int FORM>
__device__ __forceinline__ void deposit_body(const DevState& st, const DevMesh& mesh,
                                             const DevParams& P, void* qout) {
  using S = typename Traits<FORM>::S;
  using F = typename Traits<FORM>::F;
  using NS = Num<S>;
  const ForceConsts<F>& K = fconsts<F>(P);
  const int sb = st.ctl->st, pb = st.ctl->pb;
  const int64_t C = P.C;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < st.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Quad<S> p = ldq((const Quad<S>*)st.pos[sb] + i);
    const Quad<S> v = ldq((const Quad<S>*)st.vel[sb] + i);
    const Quad<F> acc = ldq((const Quad<F>*)st.acc[pb] + i);
    const S xs[3] = {p.a, p.b, p.c};
    int64_t cc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == 2 && P.graded) {
        // graded z: the cell whose FP64 faces enclose z (the last face <= z)
        const double z = NS::d(xs[2]);
        int lo = 0, hi = P.nc[2];  // faces zf[lo] <= z < zf[hi] once clamped
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (mesh.zf[mid] <= z) lo = mid;
          else hi = mid;
        }
        cc[2] = lo;
        continue;
      }
      // the cell must equal floor((x - lo) * n / L) in FP64; FP32 decides unless x
      // lies within ~1e-4 of a cell face, where the FP64 product is formed
      int64_t k;
      const float sf = (float)NS::f(NS::sub(xs[a], sbox<S>(P).lo[a])) * P.cf.inv_h[a];
      const float fl = floorf(sf);
      const float fr = sf - fl;
      if (FORM != FORM_FP64 && fr > 1e-4f && fr < 1.0f - 1e-4f) {
        k = (int64_t)fl;
      } else {
        const double s = __dmul_rn(__dsub_rn(NS::d(xs[a]), P.lo[a]), P.inv_h[a]);
        k = (int64_t)floor(s);
      }
      if (k < 0) k = 0;
      if (k > P.nc[a] - 1) k = P.nc[a] - 1;
      cc[a] = k;
    }
    const int64_t cell = (cc[2] * P.nc[1] + cc[1]) * P.nc[0] + cc[0];
    const F vf[3] = {NS::f(v.a), NS::f(v.b), NS::f(v.c)};
    const F ap[3] = {acc.a, acc.b, acc.c};
    F ff[3];
    fluid_force<S, F>(P, K, (const Quad<F>*)mesh.ufe, (const Quad<F>*)mesh.gfl,
                      (const Quad<F>*)mesh.wfl, zcent<F>(mesh), xs, NS::f(p.d), vf,
                      ap, ff);
    // graded mesh: the stored value is V_p, divided here by the volume of the cell
    const double vfrac = P.graded ? __ddiv_rn(st.vfrac[pb][i], mesh.vcz[cc[2]]) : st.vfrac[pb][i];
    if (FORM == FORM_PLAIN) {
      float* q = (float*)qout;
      const float vf32 = (float)vfrac;
      const float inv_vc = P.graded ? (float)(1.0 / mesh.vcz[cc[2]])
                                    : P.cf.inv_h[0] * P.cf.inv_h[1] * P.cf.inv_h[2];
      atomicAdd(q + cell, vf32);
      atomicAdd(q + 1 * C + cell, vf32 * vf[0]);
      atomicAdd(q + 2 * C + cell, vf32 * vf[1]);
      atomicAdd(q + 3 * C + cell, vf32 * vf[2]);
#pragma unroll
      for (int a = 0; a < 3; ++a) atomicAdd(q + (4 + a) * C + cell, -(float)ff[a] * inv_vc);
    } else {
      // eps and eps*U: exact FP64 products, scaled by 2^S (exact) and rounded to
      // nearest, bit-identical to an FP64 evaluation
      double val[4];
      val[0] = vfrac;
      val[1] = __dmul_rn(vfrac, NS::d(v.a));
      val[2] = __dmul_rn(vfrac, NS::d(v.b));
      val[3] = __dmul_rn(vfrac, NS::d(v.c));
      unsigned long long* q = (unsigned long long*)qout;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const double t = __dmul_rn(val[f], P.two_shift[f == 0 ? 0 : 1]);
        if (!(fabs(t) < 4.0e18)) {
          atomicCAS((int*)&st.ctl->deposit_range, 0, 1);
          continue;
        }
        atomicAdd(q + f * C + cell, (unsigned long long)__double2ll_rn(t));
      }
      // force density -f_fp / V_c in the force word, then to fixed point
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        long long qi;
        bool ok;
        if (FORM == FORM_FP64) {
          const double t = __dmul_rn(__ddiv_rn(-(double)ff[a], P.graded ? mesh.vcz[cc[2]] : P.vc),
                                     P.two_shift[2]);
          ok = fabs(t) < 4.0e18;
          qi = ok ? __double2ll_rn(t) : 0;
        } else {
          const float inv_vc = P.graded ? (float)(1.0 / mesh.vcz[cc[2]]) : P.inv_vc_f;
          const float t = -(float)ff[a] * inv_vc * P.two_shift_f;
          ok = fabsf(t) < 4.0e18f;
          qi = ok ? __float2ll_rn(t) : 0;
        }
        if (!ok) {
          atomicCAS((int*)&st.ctl->deposit_range, 0, 1);
          continue;
        }
        atomicAdd(q + (4 + a) * C + cell, (unsigned long long)qi);
      }
    }
  }
}

template <int FORM>
__global__ void k_deposit(DevState st, DevMesh mesh, DevParams P, void* qout) {
  deposit_body<FORM>(st, mesh, P, qout);
}

// Ensemble (blockIdx.y = bed): clear the deposition words, then deposit.
template <int FORM>
__global__ void k_deposit_zero_e(const BedView* v) {
  const BedView& b = v[blockIdx.y];
  const int64_t n = 7 * b.P.C;
  if (FORM == FORM_PLAIN) {
    float* q = (float*)b.phi;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
      q[k] = 0.0f;
  } else {
    long long* q = (long long*)b.qfix;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
      q[k] = 0;
  }
}
template <int FORM>
__global__ void k_deposit_e(const BedView* v) {
  if ((int64_t)blockIdx.x * blockDim.x >= v[blockIdx.y].st.N) return;
  const BedView& b = bed_view(v);
  deposit_body<FORM>(b.st, b.mesh, b.P, FORM == FORM_PLAIN ? b.phi : b.qfix);
}

// ---------------------------------------------------------------- CG words
template <class T>
struct CgA;
template <>
struct CgA<double> {
  __device__ static double zero() { return 0.0; }
  __device__ static double add(double a, double b) { return a + b; }
  __device__ static double sub(double a, double b) { return a - b; }
  __device__ static double mul(double a, double b) { return a * b; }
  __device__ static double from_d(double a) { return a; }
  __device__ static double to_d(double a) { return a; }
  __device__ static double shfl_xor(double a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
  __device__ static double addq(double a, double b) { return a + b; }
  __device__ static double subq(double a, double b) { return a - b; }
};
template <>
struct CgA<float> {
  __device__ static float zero() { return 0.0f; }
  __device__ static float add(float a, float b) { return a + b; }
  __device__ static float sub(float a, float b) { return a - b; }
  __device__ static float mul(float a, float b) { return a * b; }
  __device__ static float from_d(double a) { return __double2float_rn(a); }
  __device__ static double to_d(float a) { return (double)a; }
  __device__ static float shfl_xor(float a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
  __device__ static float addq(float a, float b) { return a + b; }
  __device__ static float subq(float a, float b) { return a - b; }
};
template <>
struct CgA<dd> {
  __device__ static dd zero() { return dd{0.0f, 0.0f}; }
  __device__ static dd add(dd a, dd b) { return dd_add(a, b); }
  __device__ static dd sub(dd a, dd b) { return dd_sub(a, b); }
  __device__ static dd mul(dd a, dd b) { return dd_mul(a, b); }
  __device__ static dd from_d(double a) { return dd_from_double(a); }
  __device__ static double to_d(dd a) { return dd_to_double(a); }
  __device__ static dd shfl_xor(dd a, int o) {
    return dd{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
  }
  // additions with error ~2^-44 of the operands (see dd_add_fast)
  __device__ static dd addq(dd a, dd b) { return dd_add_fast(a, b); }
  __device__ static dd subq(dd a, dd b) { return dd_sub_fast(a, b); }
};

// ---------------------------------------------------------------- conversions
template <class T>
__device__ __forceinline__ T t_from_fixed(long long q, double scale, float scalef);
template <>
__device__ __forceinline__ double t_from_fixed<double>(long long q, double scale, float) {
  return (double)q * scale;
}
template <>
__device__ __forceinline__ dd t_from_fixed<dd>(long long q, double, float s) {
  // exact split of the integer, then an exact power-of-two scaling of both words
  const float hi = __ll2float_rn(q);
  const long long rest = q - (long long)hi;
  const float lo = __ll2float_rn(rest);
  return quick_two_sum(hi * s, lo * s);
}
template <>
__device__ __forceinline__ float t_from_fixed<float>(long long q, double, float s) {
  return __ll2float_rn(q) * s;
}

template <class T>
__global__ void k_from_fixed(const long long* q, T* phi, int64_t C, double s0, double s1,
                             double s2, float f0, float f1, float f2, int nf) {
  const int64_t n = (int64_t)nf * C;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(k / C);
    const double s = f == 0 ? s0 : (f < 4 ? s1 : s2);
    const float sf = f == 0 ? f0 : (f < 4 ? f1 : f2);
    phi[k] = t_from_fixed<T>(q[k], s, sf);
  }
}

template <class T>
__global__ void k_to_double(const T* phi, double* out, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = CgA<T>::to_d(phi[k]);
}

template <class T>
__global__ void k_from_double(const double* in, T* phi, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    phi[k] = CgA<T>::from_d(in[k]);
}

// eps_s, U_s = (eps U)/max(eps, 1e-12), F_fp; eps also into the drag's mesh word.
template <class T, class F>
__global__ void k_average_out(const T* phi, int64_t C, Quad<F>* ufe, double* eps, double* Us,
                              double* Ff) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
       c += (int64_t)gridDim.x * blockDim.x) {
    const double e = CgA<T>::to_d(phi[c]);
    if (eps) eps[c] = e;
    const double den = e > 1e-12 ? e : 1e-12;
    for (int a = 0; a < 3; ++a) {
      if (Us) Us[3 * c + a] = CgA<T>::to_d(phi[(1 + a) * C + c]) / den;
      if (Ff) Ff[3 * c + a] = CgA<T>::to_d(phi[(4 + a) * C + c]);
    }
    ufe[c].d = (F)e;
  }
}

template <class T>
__global__ void k_from_fixed_e(const BedView* v) {
  const BedView& b = v[blockIdx.y];
  const int64_t C = b.P.C, n = 7 * C;
  const double s0 = 1.0 / b.P.two_shift[0], s1 = 1.0 / b.P.two_shift[1], s2 = 1.0 / b.P.two_shift[2];
  const float f0 = (float)s0, f1 = (float)s1, f2 = (float)s2;
  const long long* q = (const long long*)b.qfix;
  T* phi = (T*)b.phi;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(k / C);
    const double sc = f == 0 ? s0 : (f < 4 ? s1 : s2);
    const float sf = f == 0 ? f0 : (f < 4 ? f1 : f2);
    phi[k] = t_from_fixed<T>(q[k], sc, sf);
  }
}

// smoothed eps -> the drag's mesh word, every bed
template <class T, class F>
__global__ void k_eps_out_e(const BedView* v) {
  const BedView& b = v[blockIdx.y];
  const int64_t C = b.P.C;
  const T* phi = (const T*)b.phi;
  Quad<F>* ufe = (Quad<F>*)b.mesh.ufe;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x)
    ufe[c].d = (F)CgA<T>::to_d(phi[c]);
}

// Cell vorticity omega = curl U of the cell-centred fluid velocity U (FP64, C x 3),
// for the lift force (Sec. 2.3, Eq. 7): central differences, wrapped on periodic
// axes, one-sided in the first and last cell of other axes, zero along an axis of
// one cell (on a graded z mesh the z differences divide by the distance between
// the centres used); stored as (omega, 0) in the form's word.
template <class F>
__global__ void k_curl(const double* __restrict__ U, DevParams P, const double* __restrict__ zc,
                       Quad<F>* __restrict__ wfl) {
  const int64_t nx = P.nc[0], ny = P.nc[1], nz = P.nc[2];
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < P.C;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx[3] = {c % nx, (c / nx) % ny, c / (nx * ny)};
    const int64_t n[3] = {nx, ny, nz};
    double g[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // g[a][b] = dU_b / dx_a
    for (int a = 0; a < 3; ++a) {
      if (n[a] < 2) continue;
      const double h = (P.hi[a] - P.lo[a]) / (double)n[a];
      int64_t ip[3] = {idx[0], idx[1], idx[2]}, im[3] = {idx[0], idx[1], idx[2]};
      double den;
      if (P.periodic[a]) {
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
      if (a == 2 && P.graded) den = zc[ip[2]] - zc[im[2]];
      const int64_t cp = (ip[2] * ny + ip[1]) * nx + ip[0];
      const int64_t cm = (im[2] * ny + im[1]) * nx + im[0];
      for (int b = 0; b < 3; ++b) g[a][b] = (U[3 * cp + b] - U[3 * cm + b]) / den;
    }
    wfl[c] = Quad<F>{(F)(g[1][2] - g[2][1]), (F)(g[2][0] - g[0][2]), (F)(g[0][1] - g[1][0]), F(0)};
  }
}

// Mesh words of the fluid fields (Sec. 2.3): ufe = (U, eps_s) keeps its eps_s, gfl =
// G = -grad p + C_add rho_f DU/Dt (grad p = rho_f g when none is given), from the FP64
// fields [C][3] on the device.
template <class F>
__global__ void k_fluid_prep(const double* __restrict__ U, const double* __restrict__ gp,
                             const double* __restrict__ du, int64_t C, int pressure_grad,
                             int added_mass, int gp_default, double c_add_rho_f, double rgx,
                             double rgy, double rgz, Quad<F>* __restrict__ ufe,
                             Quad<F>* __restrict__ gfl) {
  const double rg[3] = {rgx, rgy, rgz};
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
       c += (int64_t)gridDim.x * blockDim.x) {
    double g[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double v = 0.0;
      if (pressure_grad) v -= gp_default ? rg[a] : gp[3 * c + a];
      if (added_mass) v += c_add_rho_f * du[3 * c + a];
      g[a] = v;
    }
    Quad<F> u = ufe[c];
    u.a = (F)U[3 * c];
    u.b = (F)U[3 * c + 1];
    u.c = (F)U[3 * c + 2];
    ufe[c] = u;
    gfl[c] = Quad<F>{(F)g[0], (F)g[1], (F)g[2], F(0)};
  }
}

// eps_s of the drag law from FP64 cell values.
template <class F>
__global__ void k_eps_in(const double* __restrict__ eps, int64_t C, Quad<F>* __restrict__ ufe) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
       c += (int64_t)gridDim.x * blockDim.x)
    ufe[c].d = (F)eps[c];
}

// eps_s of the drag law as FP64 cell values (checkpoints).
template <class F>
__global__ void k_eps_out(const Quad<F>* __restrict__ ufe, int64_t C, double* __restrict__ eps) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < C;
       c += (int64_t)gridDim.x * blockDim.x)
    eps[c] = (double)ufe[c].d;
}

inline unsigned grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)g;
}

}  // namespace

void launch_deposit(int form, const DevState& st, const DevMesh& mesh, const DevParams& P,
                    void* q, cudaStream_t s) {
  const unsigned g = grid_for(st.N, 256);
  switch (form) {
    case FORM_SPLIT: k_deposit<FORM_SPLIT><<<g, 256, 0, s>>>(st, mesh, P, q); break;
    case FORM_PLAIN: k_deposit<FORM_PLAIN><<<g, 256, 0, s>>>(st, mesh, P, q); break;
    default: k_deposit<FORM_FP64><<<g, 256, 0, s>>>(st, mesh, P, q); break;
  }
}

void launch_fluid_prep(int form, const double* U, const double* gp, const double* du, int gp_default,
                       double c_add_rho_f, const double rho_g[3], const DevParams& P,
                       const DevMesh& mesh, cudaStream_t s) {
  const unsigned g = grid_for(P.C, 256);
  if (form == FORM_FP64)
    k_fluid_prep<double><<<g, 256, 0, s>>>(U, gp, du, P.C, P.pressure_grad, P.added_mass, gp_default,
                                           c_add_rho_f, rho_g[0], rho_g[1], rho_g[2],
                                           (Quad<double>*)mesh.ufe, (Quad<double>*)mesh.gfl);
  else
    k_fluid_prep<float><<<g, 256, 0, s>>>(U, gp, du, P.C, P.pressure_grad, P.added_mass, gp_default,
                                          c_add_rho_f, rho_g[0], rho_g[1], rho_g[2],
                                          (Quad<float>*)mesh.ufe, (Quad<float>*)mesh.gfl);
}

void launch_eps_io(int form, double* eps, const DevMesh& mesh, int64_t C, int to_mesh, cudaStream_t s) {
  const unsigned g = grid_for(C, 256);
  if (form == FORM_FP64) {
    if (to_mesh) k_eps_in<double><<<g, 256, 0, s>>>(eps, C, (Quad<double>*)mesh.ufe);
    else k_eps_out<double><<<g, 256, 0, s>>>((const Quad<double>*)mesh.ufe, C, eps);
  } else {
    if (to_mesh) k_eps_in<float><<<g, 256, 0, s>>>(eps, C, (Quad<float>*)mesh.ufe);
    else k_eps_out<float><<<g, 256, 0, s>>>((const Quad<float>*)mesh.ufe, C, eps);
  }
}

void launch_curl(int form, const double* U, const DevParams& P, const DevMesh& mesh,
                 cudaStream_t s) {
  const unsigned g = grid_for(P.C, 256);
  if (form == FORM_FP64) k_curl<double><<<g, 256, 0, s>>>(U, P, mesh.zc, (Quad<double>*)mesh.wfl);
  else k_curl<float><<<g, 256, 0, s>>>(U, P, mesh.zc, (Quad<float>*)mesh.wfl);
}

void launch_fields_from_fixed(int form, const void* q, const DevParams& P, void* phi, int nf,
                              cudaStream_t s) {
  const double s0 = 1.0 / P.two_shift[0], s1 = 1.0 / P.two_shift[1], s2 = 1.0 / P.two_shift[2];
  const float f0 = (float)s0, f1 = (float)s1, f2 = (float)s2;  // exact powers of two
  const unsigned g = grid_for((int64_t)nf * P.C, 256);
  if (form == FORM_SPLIT)
    k_from_fixed<dd><<<g, 256, 0, s>>>((const long long*)q, (dd*)phi, P.C, s0, s1, s2, f0, f1, f2, nf);
  else if (form == FORM_FP64)
    k_from_fixed<double><<<g, 256, 0, s>>>((const long long*)q, (double*)phi, P.C, s0, s1, s2, f0, f1, f2, nf);
  // the plain form deposits floats straight into phi
}

void launch_average_out(int form, const void* phi, const DevParams& P, void* ufe, double* eps,
                        double* Us, double* F, cudaStream_t s) {
  const unsigned g = grid_for(P.C, 256);
  if (form == FORM_SPLIT)
    k_average_out<dd, float><<<g, 256, 0, s>>>((const dd*)phi, P.C, (Quad<float>*)ufe, eps, Us, F);
  else if (form == FORM_PLAIN)
    k_average_out<float, float><<<g, 256, 0, s>>>((const float*)phi, P.C, (Quad<float>*)ufe, eps, Us, F);
  else
    k_average_out<double, double><<<g, 256, 0, s>>>((const double*)phi, P.C, (Quad<double>*)ufe, eps, Us, F);
}

void launch_phi_convert(int form, const void* phi, double* out, int64_t n, int to_double,
                        cudaStream_t s) {
  const unsigned g = grid_for(n, 256);
  (void)to_double;
  if (form == FORM_SPLIT) k_to_double<dd><<<g, 256, 0, s>>>((const dd*)phi, out, n);
  else if (form == FORM_PLAIN) k_to_double<float><<<g, 256, 0, s>>>((const float*)phi, out, n);
  else k_to_double<double><<<g, 256, 0, s>>>((const double*)phi, out, n);
}

void launch_phi_from_double(int form, const double* in, void* phi, int64_t n, cudaStream_t s) {
  const unsigned g = grid_for(n, 256);
  if (form == FORM_SPLIT) k_from_double<dd><<<g, 256, 0, s>>>(in, (dd*)phi, n);
  else if (form == FORM_PLAIN) k_from_double<float><<<g, 256, 0, s>>>(in, (float*)phi, n);
  else k_from_double<double><<<g, 256, 0, s>>>(in, (double*)phi, n);
}


void launch_deposit_ens(int form, const EnsLaunch& e, cudaStream_t s) {
  auto g = [](int64_t n) {
    int64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 64 ? 64 : b));
  };
  const dim3 gc(g(7 * e.max_cells), (unsigned)e.B), gp((unsigned)((e.max_n + 255) / 256), (unsigned)e.B);
  switch (form) {
    case FORM_SPLIT:
      k_deposit_zero_e<FORM_SPLIT><<<gc, 256, 0, s>>>(e.views);
      k_deposit_e<FORM_SPLIT><<<gp, 256, 0, s>>>(e.views);
      k_from_fixed_e<dd><<<gc, 256, 0, s>>>(e.views);
      break;
    case FORM_PLAIN:
      k_deposit_zero_e<FORM_PLAIN><<<gc, 256, 0, s>>>(e.views);
      k_deposit_e<FORM_PLAIN><<<gp, 256, 0, s>>>(e.views);
      break;
    default:
      k_deposit_zero_e<FORM_FP64><<<gc, 256, 0, s>>>(e.views);
      k_deposit_e<FORM_FP64><<<gp, 256, 0, s>>>(e.views);
      k_from_fixed_e<double><<<gc, 256, 0, s>>>(e.views);
      break;
  }
}

void launch_eps_out_ens(int form, const EnsLaunch& e, cudaStream_t s) {
  int64_t b = (e.max_cells + 255) / 256;
  const dim3 g((unsigned)(b < 1 ? 1 : (b > 64 ? 64 : b)), (unsigned)e.B);
  if (form == FORM_SPLIT) k_eps_out_e<dd, float><<<g, 256, 0, s>>>(e.views);
  else if (form == FORM_PLAIN) k_eps_out_e<float, float><<<g, 256, 0, s>>>(e.views);
  else k_eps_out_e<double, double><<<g, 256, 0, s>>>(e.views);
}
}  // namespace sedi

// ---------------------------------------------------------------- no-allocation smoothing
// sedi_smooth_static: the smoothing solve of sedi_smooth without a handle and
// without any device allocation.  Its scratch is the file-scope array below,
// sized for SEDI_STATIC_MAX_WORDS field words, which every GPU that loads this
// library holds until the process exits.  Host code must not pass the array's
// name to a kernel (on the host it is only a stand-in): every call looks the
// device address up with cudaGetSymbolAddress (no allocation; after a device reset
// it names the reloaded module's array) and passes it instead.

using namespace sedi;

namespace {

constexpr int64_t kStaticWords = SEDI_STATIC_MAX_WORDS;
// The solver keeps 8 narrow words per cell whatever n_fields is, so the limit is
// 8 * cells <= kStaticWords (n_fields <= 8).  Upper bound of the solver scratch then
// (FP64 form with BDF2, the largest case): the wide right-hand side and the BDF2
// previous step (n_fields * cells <= kStaticWords words of 8 bytes each), three
// narrow [cells][8] arrays (8-byte words), kSmoothSums per-unit sums of every field
// for up to kStaticWords / (8 * 256) + 1 units of 256 cells, the unit table (4 bytes a
// unit), and 64 KB for the batch tables of one mesh and the 256-byte alignment of
// each part.
constexpr int64_t kStaticUnits = kStaticWords / (kSmoothMaxFields * kSmoothUnitCells) + 1;
constexpr int64_t kStaticWork =
    ((8 * 5 * kStaticWords + kStaticUnits * kSmoothMaxFields * kSmoothSums * 8 + 4 * kStaticUnits +
      64 * 1024) + 255) / 256 * 256;
static_assert(kMaxF == kSmoothMaxFields, "the static limit assumes the solver's field count");
static_assert(2 * sizeof(SmoothMeshDev) + 8 * 256 <= 64 * 1024,
              "the batch tables of one mesh must fit the static slack");
// layout: phi [W words] | solver scratch | iters[8] | ctl, every part 256-byte aligned
// (the control block holds 8-byte words that the compiler may access in pairs)
constexpr int64_t kStaticBytes = 8 * kStaticWords + kStaticWork + 256 + (int64_t)sizeof(Ctl) + 256;
static_assert(kStaticWork % 256 == 0 && (8 * kStaticWords) % 256 == 0,
              "parts of the static scratch must stay 256-byte aligned");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

void put_msg(char* msg, int32_t len, const char* text) {
  if (msg && len > 0) std::snprintf(msg, (size_t)len, "%s", text);
}

}  // namespace

extern "C" int sedi_smooth_static(const sedi_params* p, int32_t nf, const double* in, double* out,
                                  int32_t* iters, void* cuda_stream, char* msg, int32_t msg_len) {
  if (!p || !in || !out || nf < 1 || nf > kMaxF) {
    put_msg(msg, msg_len, "sedi_smooth_static: null pointer or n_fields outside [1, 8]");
    return SEDI_EINVAL;
  }
  const int64_t C = (int64_t)p->ncell[0] * p->ncell[1] * p->ncell[2];
  if (p->ncell[0] < 1 || p->ncell[1] < 1 || p->ncell[2] < 1 || p->n_tau < 1 || !(p->cg_rtol > 0) ||
      p->cg_max_iter < 1 || p->precision_form < 0 || p->precision_form > 2 ||
      (p->tau_scheme != SEDI_TAU_EULER && p->tau_scheme != SEDI_TAU_BDF2)) {
    put_msg(msg, msg_len, "sedi_smooth_static: invalid mesh or solver parameters");
    return SEDI_EINVAL;
  }
  if ((int64_t)kMaxF * C > kStaticWords) {
    char buf[256];
    std::snprintf(buf, sizeof(buf),
                  "sedi_smooth_static: 8 * cells = %lld exceeds the static scratch limit "
                  "SEDI_STATIC_MAX_WORDS = %lld",
                  (long long)kMaxF * C, (long long)kStaticWords);
    put_msg(msg, msg_len, buf);
    return SEDI_EINVAL;
  }
  // both buffers must be device memory (a host pointer would be read by the kernels)
  for (const void* ptr : {(const void*)in, (const void*)out}) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();  // clear a sticky "invalid value" from the query
      put_msg(msg, msg_len, "sedi_smooth_static: in and out must be device memory");
      return SEDI_EINVAL;
    }
  }
  unsigned char* base = nullptr;
  {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      put_msg(msg, msg_len, "sedi_smooth_static: cudaGetSymbolAddress of the scratch failed");
      return SEDI_ECUDA;
    }
    base = (unsigned char*)ptr;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int form = p->precision_form;
  const size_t W = (size_t)kStaticWords * 8;
  unsigned char* phi = base;
  unsigned char* work = base + W;  // solver scratch
  int* iters_dev = (int*)(base + W + kStaticWork);
  Ctl* ctl = (Ctl*)(base + W + kStaticWork + 256);
  if (p->z_grading != 1.0) {
    put_msg(msg, msg_len, "sedi_smooth_static: a graded z mesh needs a handle (sedi_smooth)");
    return SEDI_EINVAL;
  }
  if (smooth_work_bytes(p->precision_form, C, nf, p->tau_scheme) > (size_t)kStaticWork) {
    put_msg(msg, msg_len, "sedi_smooth_static: internal scratch bound exceeded");
    return SEDI_EINVAL;
  }
  // what must start at zero: the counters, the barrier and the status word
  if (cudaMemsetAsync(iters_dev, 0, 8 * sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(ctl, 0, sizeof(Ctl), s) != cudaSuccess) {
    put_msg(msg, msg_len, "sedi_smooth_static: clearing the scratch failed");
    return SEDI_ECUDA;
  }
  DevParams P{};
  for (int a = 0; a < 3; ++a) {
    P.nc[a] = p->ncell[a];
    P.periodic[a] = p->periodic[a] ? 1 : 0;
  }
  P.C = C;
  double coef[3];
  const double dtau = 1.0 / p->n_tau;
  for (int a = 0; a < 3; ++a) {
    const double h = (p->hi[a] - p->lo[a]) / p->ncell[a];
    coef[a] = dtau * 0.25 * p->bandwidth[a] * p->bandwidth[a] / (h * h);
  }
  DevState st{};
  st.ctl = ctl;
  const double rtol = form == FORM_PLAIN ? (p->cg_rtol > 2e-6 ? p->cg_rtol : 2e-6) : p->cg_rtol;
  const int64_t n = (int64_t)nf * C;
  launch_phi_from_double(form, in, phi, n, s);
  const int rc = launch_smooth(form, P, phi, nullptr, nf, work, st, iters_dev, rtol,
                               p->cg_max_iter, p->n_tau, p->tau_scheme, coef, nullptr, s);
  if (rc) {
    put_msg(msg, msg_len, "sedi_smooth_static: cooperative launch of the smoother failed");
    return SEDI_ECUDA;
  }
  launch_phi_convert(form, phi, out, n, 1, s);
  int it[8] = {0};
  Ctl c{};
  if (cudaMemcpyAsync(it, iters_dev, 8 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&c, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    put_msg(msg, msg_len, "sedi_smooth_static: CUDA error while smoothing");
    return SEDI_ECUDA;
  }
  if (iters)
    for (int f = 0; f < nf; ++f) iters[f] = it[f];
  if (c.cg_status == SEDI_ETIMEOUT) {
    put_msg(msg, msg_len, "sedi_smooth_static: grid barrier timed out");
    return SEDI_ETIMEOUT;
  }
  if (c.cg_status == SEDI_EDIVERGED) {
    put_msg(msg, msg_len, "sedi_smooth_static: cg_max_iter reached before cg_rtol");
    return SEDI_EDIVERGED;
  }
  put_msg(msg, msg_len, "");
  return 0;
}
