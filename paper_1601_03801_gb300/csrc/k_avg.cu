// Diffusion-based averaging (Sec. 2.4, Eq. 9-10).
//
// Deposition (Eq. 9, PCM): each particle adds V_p/V_c, V_p u_p/V_c and
// -f_fp/V_c to the cell holding its centre.  The split and FP64 forms round each
// value to 64-bit fixed point (round to nearest even, one exponent per field kind)
// and add with integer atomics, so the sums do not depend on the order of the
// additions and match an exact integer sum bit for bit.  The plain FP32 form adds
// floats.
//
// Smoothing (Eq. 10): n_tau backward-Euler steps (I - dtau div D grad) x = b of
// the 7-point finite-volume Laplacian (zero flux through non-periodic faces),
// each solved to ||r|| <= rtol ||b|| for all fields at once in ONE persistent
// cooperative launch.  The solver is Chebyshev semi-iteration on the known
// spectrum of the operator (see k_smooth): one grid barrier per iteration and no
// inner products except the final residual check.  Every block reduces the
// per-block partials in the same fixed order, so all blocks take identical
// decisions and the result is run-to-run deterministic.
// The grid barrier spins at most ~0.3 s, then records SEDI_ETIMEOUT and returns;
// the other blocks see the record and return at their next barrier.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/sedi.h"
#include "common.cuh"
#include "fluid.cuh"
#include "kernels.h"

namespace sedi {

namespace {

constexpr int kMaxF = 8;
constexpr int kSmoothThreads = 512;

// ---------------------------------------------------------------- deposition
template <int FORM>
__global__ void k_deposit(DevState st, DevMesh mesh, DevParams P, void* qout) {
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
    fluid_force<S, F>(P, K, (const Quad<F>*)mesh.ufe, (const Quad<F>*)mesh.gfl, xs, NS::f(p.d), vf,
                      ap, ff);
    const double vfrac = st.vfrac[pb][i];
    if (FORM == FORM_PLAIN) {
      float* q = (float*)qout;
      const float vf32 = (float)vfrac;
      const float inv_vc = P.cf.inv_h[0] * P.cf.inv_h[1] * P.cf.inv_h[2];
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
          const double t = __dmul_rn(__ddiv_rn(-(double)ff[a], P.vc), P.two_shift[2]);
          ok = fabs(t) < 4.0e18;
          qi = ok ? __double2ll_rn(t) : 0;
        } else {
          const float t = -(float)ff[a] * P.inv_vc_f * P.two_shift_f;
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

struct SmoothArgs;
template <class T>
__device__ __forceinline__ T coef_word(const SmoothArgs& a, int k);

struct SmoothArgs {
  void* x;            // [nf][C] in: fields, out: smoothed
  void* b;            // [nf][C] right-hand side of the current pseudo-step
  void* r;            // [nf][C]
  void* p[2];         // [nf][C] search directions (double-buffered)
  void* q;            // [nf][C] A p
  const void* guess;  // [nf][C] or null
  double* part;       // [2][kMaxF][grid]
  int* iters;         // [nf]
  int nf;
  int64_t C;
  int nc[3];
  int per[3];
  double coef[3];     // dtau * D_a / h_a^2
  dd coef_dd[3];      // the same, split into two FP32 words on the host
  double lmax;        // upper bound of the spectrum of A (1 + 4 sum coef)
  double rtol2;
  int max_iter;
  int n_tau;
  Ctl* ctl;
};

template <>
__device__ __forceinline__ double coef_word<double>(const SmoothArgs& a, int k) {
  return a.coef[k];
}
template <>
__device__ __forceinline__ float coef_word<float>(const SmoothArgs& a, int k) {
  return a.coef_dd[k].hi;
}
template <>
__device__ __forceinline__ dd coef_word<dd>(const SmoothArgs& a, int k) {
  return a.coef_dd[k];
}

// Bounded grid barrier (co-residency guaranteed by the cooperative launch).
__device__ bool grid_barrier(Ctl* ctl, unsigned nblocks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &ctl->bar_gen;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      long long spins = 0;
      while (*gen == g) {
        if (++spins > (1ll << 22)) {  // ~0.3 s
          atomicCAS((int*)&ctl->cg_status, 0, -8);
          break;
        }
        // another block gave up: stop waiting too
        if ((spins & 1023) == 0 && *((volatile int*)&ctl->cg_status) == -8) break;
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *((volatile int*)&ctl->cg_status) != -8;
}

// Block-reduce nf per-thread partials (fixed order), thread 0 writes part[f][blk].
template <class T>
__device__ void block_partials(T* acc, int nf, double* part_slot, unsigned nblk) {
  using A = CgA<T>;
  __shared__ double wred[kMaxF][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int f = 0; f < nf; ++f) {
    T v = acc[f];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = A::add(v, A::shfl_xor(v, o));
    if (lane == 0) wred[f][wid] = A::to_d(v);
  }
  __syncthreads();
  if (wid == 0) {
    for (int f = 0; f < nf; ++f) {
      double v = lane < nw ? wred[f][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) part_slot[(int64_t)f * nblk + blockIdx.x] = v;
    }
  }
  __syncthreads();
}

// Every block sums part[f][0..nblk) in the same order; result in out[f] (shared).
__device__ void grid_sums(const double* part_slot, int nf, unsigned nblk, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid == 0) {
    for (int f = 0; f < nf; ++f) {
      double v = 0.0;
      for (unsigned b = lane; b < nblk; b += 32) v += __ldcg(part_slot + (int64_t)f * nblk + b);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) out[f] = v;
    }
  }
  __syncthreads();
}

// Loads of words written by other blocks of the same launch: L2 only (ld.cg),
// so no stale L1 line is read after a grid barrier.
__device__ __forceinline__ double ldx(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldx(const float* p) { return __ldcg(p); }
__device__ __forceinline__ dd ldx(const dd* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return dd{v.x, v.y};
}

// Cell coordinates and the six face neighbours (-1: zero-flux face).
struct Stencil {
  int32_t nb[6];
};

__device__ __forceinline__ Stencil stencil_of(const SmoothArgs& a, int64_t c) {
  const uint32_t nx = a.nc[0], ny = a.nc[1], nz = a.nc[2];
  const uint32_t cc = (uint32_t)c;
  const uint32_t ix = cc % nx;
  const uint32_t t = cc / nx;
  const uint32_t iy = t % ny;
  const uint32_t iz = t / ny;
  const uint32_t idx[3] = {ix, iy, iz};
  const uint32_t n[3] = {nx, ny, nz};
  const int32_t stride[3] = {1, (int32_t)nx, (int32_t)(nx * ny)};
  Stencil s;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int32_t base = (int32_t)cc - (int32_t)idx[ax] * stride[ax];
    // minus face
    if (idx[ax] > 0) s.nb[2 * ax] = (int32_t)cc - stride[ax];
    else s.nb[2 * ax] = a.per[ax] ? base + (int32_t)(n[ax] - 1) * stride[ax] : -1;
    // plus face
    if (idx[ax] + 1 < n[ax]) s.nb[2 * ax + 1] = (int32_t)cc + stride[ax];
    else s.nb[2 * ax + 1] = a.per[ax] ? base : -1;
  }
  return s;
}

// (A v)(c) = v_c - sum_faces coef_a (v_nb - v_c) for one field
template <class T>
__device__ __forceinline__ T apply_A(const Stencil& st, const T* cf, const T* v, int64_t c) {
  using A = CgA<T>;
  const T vc = ldx(v + c);
  T lap = A::zero();
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    // both faces of one axis share the coefficient: coef * ((v- - vc) + (v+ - vc))
    T sa = A::zero();
    bool any = false;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int32_t nb = st.nb[2 * ax + side];
      if (nb < 0) continue;
      sa = any ? A::addq(sa, A::subq(ldx(v + nb), vc)) : A::subq(ldx(v + nb), vc);
      any = true;
    }
    if (any) lap = A::addq(lap, A::mul(cf[ax], sa));
  }
  return A::subq(vc, lap);
}

// Chebyshev semi-iteration for A x = b, spectrum of A in [1, lmax] (A = I - dtau L
// with the zero-flux / periodic 7-point Laplacian: lambda_min = 1 exactly,
// lambda_max <= 1 + 4 sum_a coef_a by Gershgorin).  Three-term recurrence:
//   r0 = b - A x0, d0 = r0 / theta, rho0 = delta / theta
//   x += d ; r -= A d ; rho' = 1 / (2 theta/delta - rho) ; d = rho' rho d + (2 rho'/delta) r
// (theta, delta: centre and half-width of the spectrum).  The residual obeys
// ||r_k|| <= 2 sigma^k ||r_0||, sigma = (sqrt(kappa)-1)/(sqrt(kappa)+1), so the
// iteration count is fixed up front from ||r_0|| / ||b|| and confirmed by one
// residual reduction; no dot product inside the loop, one grid barrier per
// iteration.  With x0 = b (or a guess shifted to sum(b)), 1^T r = 0 and 1^T d = 0
// throughout, so every iterate keeps sum(x) = sum(b).
template <class T>
__global__ void __launch_bounds__(kSmoothThreads) k_smooth(SmoothArgs a) {
  using A = CgA<T>;
  const unsigned G = gridDim.x;
  const int64_t nthr = (int64_t)G * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int nf = a.nf;
  const int64_t C = a.C;
  T* X = (T*)a.x;
  T* Bv = (T*)a.b;
  T* R = (T*)a.r;
  T* Q = (T*)a.q;
  const T cf[3] = {coef_word<T>(a, 0), coef_word<T>(a, 1), coef_word<T>(a, 2)};
  __shared__ double s_bb[kMaxF], s_rr[kMaxF], s_tmp[kMaxF], s_tmp2[kMaxF];
  __shared__ T s_word[kMaxF];
  __shared__ int s_active[kMaxF];
  __shared__ T s_c1, s_c2, s_inv_theta;
  __shared__ int s_kmin[kMaxF];
  int iters[kMaxF];
  for (int f = 0; f < kMaxF; ++f) iters[f] = 0;
  T acc[kMaxF], acc2[kMaxF];
  double* part0 = a.part;
  double* part1 = a.part + (int64_t)kMaxF * G;
  // spectral constants: FP64 scalars used by thread 0 only
  double theta = 0.0, delta = 0.0, sigma1 = 0.0, sig = 0.0;
  if (threadIdx.x == 0) {
    theta = 0.5 * (a.lmax + 1.0);
    delta = 0.5 * (a.lmax - 1.0);
    sigma1 = theta / delta;
    const double sq = sqrt(a.lmax);
    sig = (sq - 1.0) / (sq + 1.0);
    s_inv_theta = A::from_d(1.0 / theta);
  }
  __syncthreads();

  for (int m = 0; m < a.n_tau; ++m) {
    const bool use_guess = (m == 0 && a.guess != nullptr);
    for (int f = 0; f < nf; ++f) { acc[f] = A::zero(); acc2[f] = A::zero(); }
    for (int64_t c = tid; c < C; c += nthr)
      for (int f = 0; f < nf; ++f) {
        const T xv = ldx(X + f * C + c);
        Bv[f * C + c] = xv;
        if (use_guess) {
          acc[f] = A::add(acc[f], xv);
          acc2[f] = A::add(acc2[f], ldx((const T*)a.guess + f * C + c));
        }
      }
    if (use_guess) {
      block_partials<T>(acc, nf, part0, G);
      block_partials<T>(acc2, nf, part1, G);
      if (!grid_barrier(a.ctl, G)) return;
      grid_sums(part0, nf, G, s_tmp);
      grid_sums(part1, nf, G, s_tmp2);
      if (threadIdx.x < nf)
        s_word[threadIdx.x] = A::from_d((s_tmp[threadIdx.x] - s_tmp2[threadIdx.x]) / (double)C);
      __syncthreads();
      for (int64_t c = tid; c < C; c += nthr)
        for (int f = 0; f < nf; ++f)
          X[f * C + c] = A::add(ldx((const T*)a.guess + f * C + c), s_word[f]);
    }
    if (!grid_barrier(a.ctl, G)) return;
    // r = b - A x ; d = r / theta ; partials b.b and r.r
    for (int f = 0; f < nf; ++f) { acc[f] = A::zero(); acc2[f] = A::zero(); }
    T* D0 = (T*)a.p[0];
    for (int64_t c = tid; c < C; c += nthr) {
      const Stencil sc = stencil_of(a, c);
      for (int f = 0; f < nf; ++f) {
        const T ax = apply_A<T>(sc, cf, X + f * C, c);
        const T bv = ldx(Bv + f * C + c);
        const T rv = A::sub(bv, ax);
        R[f * C + c] = rv;
        D0[f * C + c] = A::mul(rv, s_inv_theta);
        acc[f] = A::add(acc[f], A::mul(bv, bv));
        acc2[f] = A::add(acc2[f], A::mul(rv, rv));
      }
    }
    block_partials<T>(acc, nf, part0, G);
    block_partials<T>(acc2, nf, part1, G);
    if (!grid_barrier(a.ctl, G)) return;
    grid_sums(part0, nf, G, s_bb);
    grid_sums(part1, nf, G, s_rr);
    if (threadIdx.x == 0) {
      for (int f = 0; f < nf; ++f) {
        s_active[f] = (s_bb[f] > 0.0) && (s_rr[f] > a.rtol2 * s_bb[f]);
        s_kmin[f] = 0;
        if (s_active[f]) {
          // ||r_k|| <= 2 sig^k ||r_0||  ->  k >= log(rtol ||b|| / (2 ||r_0||)) / log(sig)
          const double need = 0.5 * sqrt(a.rtol2 * s_bb[f] / s_rr[f]);
          int k = sig > 0.0 ? (int)ceil(log(need) / log(sig)) : 1;
          s_kmin[f] = k < 1 ? 1 : k;
        }
      }
    }
    __syncthreads();
    for (int f = 0; f < nf; ++f)
      if (!(s_bb[f] > 0.0))
        for (int64_t c = tid; c < C; c += nthr) X[f * C + c] = A::zero();
    int any = 0;
    for (int f = 0; f < nf; ++f) any |= s_active[f];
    // each field is first checked at its own a-priori count, then every 2 iterations
    int kcheck[kMaxF];
    for (int f = 0; f < kMaxF; ++f) kcheck[f] = f < nf ? s_kmin[f] : 0;
    double rho = 1.0 / sigma1;  // advanced by thread 0 only (FP64 is slow here)
    int it = 0;
    while (any && it < a.max_iter) {
      ++it;
      // scalars of this iteration (block thread 0, broadcast)
      if (threadIdx.x == 0) {
        const double rho_new = 1.0 / (2.0 * sigma1 - rho);
        s_c1 = A::from_d(rho_new * rho);
        s_c2 = A::from_d(2.0 * rho_new / delta);
        rho = rho_new;
      }
      __syncthreads();
      const T c1 = s_c1, c2 = s_c2;
      const T* Dold = (const T*)a.p[(it - 1) & 1];
      T* Dnew = (T*)a.p[it & 1];
      bool check = false;
      for (int f = 0; f < nf; ++f) check |= s_active[f] && it >= kcheck[f];
      for (int f = 0; f < nf; ++f) acc[f] = A::zero();
      for (int64_t c = tid; c < C; c += nthr) {
        const Stencil sc = stencil_of(a, c);
        for (int f = 0; f < nf; ++f) {
          if (!s_active[f]) continue;
          const int64_t k = f * C + c;
          const T dv = ldx(Dold + k);
          const T ad = apply_A<T>(sc, cf, Dold + f * C, c);
          X[k] = A::addq(ldx(X + k), dv);
          const T rv = A::subq(ldx(R + k), ad);
          R[k] = rv;
          Dnew[k] = A::addq(A::mul(c1, dv), A::mul(c2, rv));
          if (check) acc[f] = A::add(acc[f], A::mul(rv, rv));
        }
      }
      if (check) block_partials<T>(acc, nf, part0, G);
      if (!grid_barrier(a.ctl, G)) return;
      if (check) {
        grid_sums(part0, nf, G, s_tmp);
        if (threadIdx.x == 0)
          for (int f = 0; f < nf; ++f)
            if (s_active[f] && it >= kcheck[f] && s_tmp[f] <= a.rtol2 * s_bb[f]) s_active[f] = -it;
        __syncthreads();
        any = 0;
        for (int f = 0; f < nf; ++f) {
          if (s_active[f] < 0) iters[f] += -s_active[f];
          any |= s_active[f] > 0;
        }
        __syncthreads();
        if (threadIdx.x < nf && s_active[threadIdx.x] < 0) s_active[threadIdx.x] = 0;
        __syncthreads();
        for (int f = 0; f < nf; ++f)
          if (it >= kcheck[f]) kcheck[f] = it + 2;
      }
    }
    for (int f = 0; f < nf; ++f)
      if (s_active[f]) {
        iters[f] += a.max_iter;
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS((int*)&a.ctl->cg_status, 0, -6);
      }
    if (!grid_barrier(a.ctl, G)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int f = 0; f < nf; ++f) a.iters[f] += iters[f];
  (void)Q;
}

__global__ void k_bar_reset(Ctl* ctl) {
  ctl->bar_count = 0u;
  ctl->bar_gen = 0u;
}

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

inline unsigned grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)g;
}

template <class T>
int smooth_impl_sized(const DevParams& P, void* phi, const void* guess, int nf, void* work,
                      size_t stride_bytes, const DevState& st, int* iters_dev, double rtol,
                      int max_iter, int n_tau, const double coef[3], int max_blocks,
                      cudaStream_t s);

template <class T>
int smooth_impl(const DevParams& P, void* phi, const void* guess, int nf, void* work,
                const DevState& st, int* iters_dev, double rtol, int max_iter, int n_tau,
                const double coef[3], cudaStream_t s) {
  return smooth_impl_sized<T>(P, phi, guess, nf, work, (size_t)nf * P.C * sizeof(T), st, iters_dev,
                              rtol, max_iter, n_tau, coef, 152 * 8, s);
}

template <class T>
int smooth_impl_sized(const DevParams& P, void* phi, const void* guess, int nf, void* work,
                      size_t stride_bytes, const DevState& st, int* iters_dev, double rtol,
                      int max_iter, int n_tau, const double coef[3], int max_blocks,
                      cudaStream_t s) {
  const int64_t C = P.C;
  int dev = 0;
  cudaGetDevice(&dev);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smooth<T>, kSmoothThreads, 0);
  if (per_sm < 1) return -3;
  if (per_sm > 2) per_sm = 2;
  unsigned G = (unsigned)(nsm * per_sm);
  if ((int)G > max_blocks) G = (unsigned)max_blocks;
  SmoothArgs a{};
  char* w = (char*)work;
  const size_t fb = stride_bytes;
  a.x = phi;
  a.b = w;
  a.r = w + fb;
  a.p[0] = w + 2 * fb;
  a.p[1] = w + 3 * fb;
  a.q = w + 4 * fb;
  a.part = (double*)(w + 5 * fb);
  a.guess = guess;
  a.iters = iters_dev;
  a.nf = nf;
  a.C = C;
  for (int k = 0; k < 3; ++k) {
    a.nc[k] = P.nc[k];
    a.per[k] = P.periodic[k];
    a.coef[k] = coef[k];
    const float hi = (float)coef[k];
    a.coef_dd[k] = dd{hi, (float)(coef[k] - (double)hi)};
  }
  a.lmax = 1.0 + 4.0 * (coef[0] + coef[1] + coef[2]);
  if (a.lmax < 1.0 + 1e-12) a.lmax = 1.0 + 1e-12;
  a.rtol2 = rtol * rtol;
  a.max_iter = max_iter;
  a.n_tau = n_tau;
  a.ctl = st.ctl;
  k_bar_reset<<<1, 1, 0, s>>>(st.ctl);
  void* args[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_smooth<T>, dim3(G),
                                              dim3(kSmoothThreads), args, 0, s);
  return e == cudaSuccess ? 0 : -3;
}

}  // namespace

size_t smooth_work_bytes(int form, int64_t C, int nf) {
  const size_t w = form == FORM_PLAIN ? sizeof(float) : (form == FORM_FP64 ? sizeof(double) : sizeof(dd));
  return 5 * (size_t)nf * C * w + 2 * (size_t)kMaxF * 152 * 8 * sizeof(double) + 256;
}

void launch_deposit(int form, const DevState& st, const DevMesh& mesh, const DevParams& P,
                    void* q, cudaStream_t s) {
  const unsigned g = grid_for(st.N, 256);
  switch (form) {
    case FORM_SPLIT: k_deposit<FORM_SPLIT><<<g, 256, 0, s>>>(st, mesh, P, q); break;
    case FORM_PLAIN: k_deposit<FORM_PLAIN><<<g, 256, 0, s>>>(st, mesh, P, q); break;
    default: k_deposit<FORM_FP64><<<g, 256, 0, s>>>(st, mesh, P, q); break;
  }
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

int launch_smooth(int form, const DevParams& P, void* phi, const void* guess, int nf, void* work,
                  const DevState& st, int* iters_dev, double rtol, int max_iter, int n_tau,
                  const double coef[3], cudaStream_t s) {
  if (nf > kMaxF) return -1;
  switch (form) {
    case FORM_SPLIT:
      return smooth_impl<dd>(P, phi, guess, nf, work, st, iters_dev, rtol, max_iter, n_tau, coef, s);
    case FORM_PLAIN:
      return smooth_impl<float>(P, phi, guess, nf, work, st, iters_dev, rtol, max_iter, n_tau, coef, s);
    default:
      return smooth_impl<double>(P, phi, guess, nf, work, st, iters_dev, rtol, max_iter, n_tau, coef, s);
  }
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

}  // namespace sedi

// ---------------------------------------------------------------- no-allocation smoothing
// sedi_smooth_static: the smoothing solve of sedi_smooth without a handle and
// without any device allocation.  Its scratch is the file-scope array below,
// sized for SEDI_STATIC_MAX_WORDS field words, which every GPU that loads this
// library holds until the process exits.  Host code must not pass the array's
// name to a kernel (on the host it is only a stand-in): the device address is
// taken once per device with cudaGetSymbolAddress and passed instead.

using namespace sedi;

namespace {

constexpr int64_t kStaticWords = SEDI_STATIC_MAX_WORDS;
constexpr int kStaticMaxBlocks = 1216;  // partial sums of up to 1216 blocks
// layout (8-byte words): phi[W] b[W] r[W] p0[W] p1[W] q[W] part[2*kMaxF*1216] iters[8] ctl
constexpr int64_t kStaticBytes =
    8 * (6 * kStaticWords + 2 * (int64_t)kMaxF * kStaticMaxBlocks + 8) + (int64_t)sizeof(Ctl) + 256;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

struct StaticSlot {
  unsigned char* base = nullptr;  // device address of g_static_scratch on this device
};
std::mutex g_static_mutex;
StaticSlot g_static_slots[64];

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
      p->cg_max_iter < 1 || p->precision_form < 0 || p->precision_form > 2) {
    put_msg(msg, msg_len, "sedi_smooth_static: invalid mesh or solver parameters");
    return SEDI_EINVAL;
  }
  if ((int64_t)nf * C > kStaticWords) {
    char buf[256];
    std::snprintf(buf, sizeof(buf),
                  "sedi_smooth_static: n_fields * cells = %lld exceeds the static scratch limit "
                  "SEDI_STATIC_MAX_WORDS = %lld",
                  (long long)nf * C, (long long)kStaticWords);
    put_msg(msg, msg_len, buf);
    return SEDI_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    put_msg(msg, msg_len, "sedi_smooth_static: no current CUDA device");
    return SEDI_ECUDA;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_slots[dev].base) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess || !ptr) {
        put_msg(msg, msg_len, "sedi_smooth_static: cudaGetSymbolAddress of the scratch failed");
        return SEDI_ECUDA;
      }
      g_static_slots[dev].base = (unsigned char*)ptr;
    }
    base = g_static_slots[dev].base;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int form = p->precision_form;
  const size_t W = (size_t)kStaticWords * 8;
  unsigned char* phi = base;
  unsigned char* work = base + W;  // b, r, p0, p1, q, then the partial sums
  int* iters_dev = (int*)(base + 6 * W + 8 * 2 * (size_t)kMaxF * kStaticMaxBlocks);
  Ctl* ctl = (Ctl*)(base + 6 * W + 8 * (2 * (size_t)kMaxF * kStaticMaxBlocks + 8));
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
  int rc = -3;
  switch (form) {
    case FORM_SPLIT:
      rc = smooth_impl_sized<dd>(P, phi, nullptr, nf, work, W, st, iters_dev, rtol, p->cg_max_iter,
                                 p->n_tau, coef, kStaticMaxBlocks, s);
      break;
    case FORM_PLAIN:
      rc = smooth_impl_sized<float>(P, phi, nullptr, nf, work, W, st, iters_dev, rtol,
                                    p->cg_max_iter, p->n_tau, coef, kStaticMaxBlocks, s);
      break;
    default:
      rc = smooth_impl_sized<double>(P, phi, nullptr, nf, work, W, st, iters_dev, rtol,
                                     p->cg_max_iter, p->n_tau, coef, kStaticMaxBlocks, s);
      break;
  }
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
