// Fluid-particle force at one particle, shared by the substep and the
// deposition kernels so both evaluate f_fp with the same code.
#pragma once
#include "common.cuh"
#include "fmath.cuh"

namespace sedi {

// Per-axis trilinear weights of a cell-centred field (periodic wrap, else clamp).
template <class F>
__device__ __forceinline__ void axis_w(F s, int n, int per, int* i0, int* i1, F* f) {
  if (per) {
    // positions lie in [lo, hi), so s is in [-0.5, n - 0.5) and k in [-1, n - 1]
    F fl = xfloor(s);
    *f = s - fl;
    int k = (int)fl;
    if (k < 0) k += n;
    if (k >= n) k -= n;
    *i0 = k;
    *i1 = (k + 1 == n) ? 0 : k + 1;
  } else {
    if (s < F(0)) s = F(0);
    if (s > F(n - 1)) s = F(n - 1);
    int k = (int)xfloor(s);
    if (n >= 2 && k > n - 2) k = n - 2;
    if (n < 2) k = 0;
    *i0 = k;
    *i1 = n >= 2 ? k + 1 : 0;
    *f = n >= 2 ? s - F(k) : F(0);
  }
}

// The same weights from the integer part kf = floor(s) and a fraction f that may lie
// within rounding outside [0, 1) (the cell-relative form below).
template <class F>
__device__ __forceinline__ void axis_w_kf(F kf, F f, int n, int per, int* i0, int* i1, F* fo) {
  int k = (int)kf;
  if (f < F(0)) {
    k -= 1;
    f += F(1);
  } else if (f >= F(1)) {
    k += 1;
    f -= F(1);
  }
  if (per) {
    if (k < 0) k += n;
    if (k >= n) k -= n;
    *i0 = k;
    *i1 = (k + 1 == n) ? 0 : k + 1;
    *fo = f;
  } else if (n < 2) {
    *i0 = 0;
    *i1 = 0;
    *fo = F(0);
  } else {
    // s = k + f clamped to [0, n - 1]
    if (k < 0) {
      k = 0;
      f = F(0);
    }
    if (k > n - 2) {
      k = n - 2;
      f = F(1);
    }
    *i0 = k;
    *i1 = k + 1;
    *fo = f;
  }
}

// Fluid force on one particle (Sec. 2.3): drag (Eq. 3-6, Syamlal-O'Brien), the
// pressure-gradient force, added mass (Eq. 8) and, when switched on, Saffman lift
// (Eq. 7, read as C_l rho_f nu^0.5 d^2 |omega|^-0.5 (w x omega), w = U_f - u_p).
// The mesh carries G = -grad p + C_add rho_f DU/Dt so both linear terms come from
// one interpolation, and the cell vorticity omega = curl U_f for the lift.  Drag is
// written in a form without 1/Re:
//   C_d |w| = (0.63 sqrt|w| + 4.8 sqrt(V_r nu / d))^2.
// z centres of a graded mesh in the force word
template <class F>
__device__ __forceinline__ const F* zcent(const DevMesh& m);
template <>
__device__ __forceinline__ const float* zcent<float>(const DevMesh& m) {
  return m.zcf;
}
template <>
__device__ __forceinline__ const double* zcent<double>(const DevMesh& m) {
  return m.zc;
}

template <class S, class F, bool LIFT = true>
__device__ __forceinline__ void fluid_force(const DevParams& P, const ForceConsts<F>& K,
                                            const Quad<F>* ufe, const Quad<F>* gfl,
                                            const Quad<F>* wfl, const F* zc, const S* x, F r,
                                            const F v[3], const F a_prev[3], F out[3]) {
  using NS = Num<S>;
  const BoxS<S>& B = sbox<S>(P);
  int i0[3], i1[3];
  F fr[3];
  for (int a = 0; a < 3; ++a) {
    if (a == 2 && P.graded) {
      // graded z: linear weight between the enclosing cell centres, clamped outside
      const F z = NS::f(x[2]);
      const int n = P.nc[2];
      if (!(z > zc[0])) {
        i0[2] = 0, i1[2] = 1, fr[2] = F(0);
      } else if (!(z < zc[n - 1])) {
        i0[2] = n - 2, i1[2] = n - 1, fr[2] = F(1);
      } else {
        int lo = 0, hi = n - 1;  // zc[lo] < z < zc[hi]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (zc[mid] <= z) lo = mid;
          else hi = mid;
        }
        i0[2] = lo, i1[2] = lo + 1, fr[2] = (z - zc[lo]) / (zc[lo + 1] - zc[lo]);
      }
      continue;
    }
    F rel = NS::dif(x[a], B.lo[a]);
    F s = rel * K.inv_h[a] - F(0.5);
    if constexpr (NS::kExtended) {
      // cell-relative: the cell k = floor(s) from FP32 (a wrong guess by one is
      // corrected below), the fraction from the double-float offset x - c_k to that
      // cell's centre, so the weight keeps ~1e-7 of a cell on any box (s itself
      // carries ~n 6e-8 of rounding)
      const F kf = xfloor(s);
      const S ck = NS::addq(B.lo[a], NS::mul_f(B.h[a], kf + F(0.5)));
      const F f = NS::f(NS::subq(x[a], ck)) * K.inv_h[a];
      axis_w_kf<F>(kf, f, P.nc[a], P.periodic[a], &i0[a], &i1[a], &fr[a]);
    } else {
      axis_w<F>(s, P.nc[a], P.periodic[a], &i0[a], &i1[a], &fr[a]);
    }
  }
  F U[3] = {0, 0, 0}, G[3] = {0, 0, 0}, Om[3] = {0, 0, 0}, eps = 0;
  const int64_t nx = P.nc[0], ny = P.nc[1];
  for (int kz = 0; kz < 2; ++kz) {
    int iz = kz ? i1[2] : i0[2];
    F wz = kz ? fr[2] : F(1) - fr[2];
    for (int ky = 0; ky < 2; ++ky) {
      int iy = ky ? i1[1] : i0[1];
      F wy = ky ? fr[1] : F(1) - fr[1];
      for (int kx = 0; kx < 2; ++kx) {
        int ix = kx ? i1[0] : i0[0];
        F wx = kx ? fr[0] : F(1) - fr[0];
        int64_t c = ((int64_t)iz * ny + iy) * nx + ix;
        F w = wz * wy * wx;
        Quad<F> u = ldq(ufe + c);
        U[0] += w * u.a;
        U[1] += w * u.b;
        U[2] += w * u.c;
        eps += w * u.d;
        if (P.pressure_grad || P.added_mass) {
          Quad<F> g = ldq(gfl + c);
          G[0] += w * g.a;
          G[1] += w * g.b;
          G[2] += w * g.c;
        }
        if (LIFT && P.lift) {
          Quad<F> o = ldq(wfl + c);
          Om[0] += w * o.a;
          Om[1] += w * o.b;
          Om[2] += w * o.c;
        }
      }
    }
  }
  F d = F(2) * r;
  F Vp = F(0.52359877559829887) * d * d * d;  // pi/6 d^3
  out[0] = Vp * G[0];
  out[1] = Vp * G[1];
  out[2] = Vp * G[2];
  if (P.added_mass) {
    out[0] -= K.c_add_rho_f * Vp * a_prev[0];
    out[1] -= K.c_add_rho_f * Vp * a_prev[1];
    out[2] -= K.c_add_rho_f * Vp * a_prev[2];
  }
  if (P.drag) {
    F es = eps < F(0) ? F(0) : eps;
    if (es > K.eps_max) es = K.eps_max;
    F ef = F(1) - es;
    F w0 = U[0] - v[0], w1 = U[1] - v[1], w2 = U[2] - v[2];
    F wm = xsqrt_pos(w0 * w0 + w1 * w1 + w2 * w2);
    F Re = xdiv(d * wm, K.nu_f);
    F A1 = xpow_drag(ef, F(4.14));
    F A2 = ef <= F(0.85) ? F(0.8) * xpow_drag(ef, F(1.28)) : xpow_drag(ef, F(2.65));
    F t = F(0.06) * Re;
    F Vr = F(0.5) * (A1 - t + xsqrt_pos(t * t + F(0.12) * Re * (F(2) * A2 - A1) + A1 * A1));
    F c = F(0.63) * xsqrt_pos(wm) + F(4.8) * xsqrt_pos(xdiv(Vr * K.nu_f, d));
    F coef = xdiv(F(0.75) * Vp * K.rho_f * c * c, Vr * Vr * d);
    out[0] += coef * w0;
    out[1] += coef * w1;
    out[2] += coef * w2;
  }
  if (LIFT && P.lift) {
    const F om = xsqrt(Om[0] * Om[0] + Om[1] * Om[1] + Om[2] * Om[2]);
    if (om > F(0)) {
      const F s = K.lift_c * d * d * xrsqrt(om);
      const F w0 = U[0] - v[0], w1 = U[1] - v[1], w2 = U[2] - v[2];
      out[0] += s * (w1 * Om[2] - w2 * Om[1]);
      out[1] += s * (w2 * Om[0] - w0 * Om[2]);
      out[2] += s * (w0 * Om[1] - w1 * Om[0]);
    }
  }
}

}  // namespace sedi
