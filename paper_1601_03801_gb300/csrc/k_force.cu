// Fused DEM substep: for every particle (one thread, cell-sorted order) visit its
// neighbour list, evaluate Hertz-Mindlin contact with the tangential spring and
// Ball-Melrose lubrication (Sec. 2.1 Eq. 1, Sec. 2.5), then wall contact, then
// the fluid forces at the particle (Sec. 2.3, Eq. 3-8), then the leapfrog
// velocity-Verlet update (Sec. 2.1, Eq. 1).
//
// Each pair is evaluated from both sides in canonical order (lower caller index
// first) by the same code, so F_ji = -F_ij bit for bit and both sides keep
// identical copies of the pair's spring; no atomics and no second pass.
// Particle state is double-buffered (read buffer, write buffer) so neighbours are
// read at the old time level.
#include "../../include/sedi.h"
#include "common.cuh"
#include "fluid.cuh"
#include "fmath.cuh"
#include "kernels.h"

namespace sedi {

namespace {

template <class F>
struct V3 {
  F x, y, z;
};

// Contact on body "a" (Sec. 2.5 soft spheres): Hertz-Mindlin with Tsuji-type damping,
// or the linear spring-dashpot of Sec. 2.5 / Table 1 (K.law == 1).
// n: unit normal a -> b; delta > 0 overlap; vrel: contact-point velocity of a
// relative to b; xi_old: spring (valid if has_old).  Returns the force on a and
// writes the tangential part and the updated spring.
template <class S, class F>
__device__ __forceinline__ V3<F> hm_core(const ForceConsts<F>& K, V3<F> n, F delta, F Rs, F ms,
                                         V3<F> vrel, const S* xi_old, bool has_old, V3<F>* Ft_out,
                                         S* xi_new) {
  using NS = Num<S>;
  F Sn, St, cn, ct, fel;  // stiffnesses, damping coefficients, elastic normal force
  // both laws: the tangential damping coefficient is the normal one times
  // sqrt(S_t / S_n), a constant of the material (sqrt(4 G* / E*), or sqrt(k_t / k_n))
  if (K.law == 1) {
    // linear spring-dashpot (Sec. 2.5, Table 1)
    Sn = K.kn_lin;
    St = K.kt_lin;
    cn = K.cdamp_lin * xsqrt_pos(Sn * ms);
    ct = cn * K.ct_ratio_lin;
    fel = K.kn_lin * delta;
  } else {
    // sqrt(R* delta) = sqrt(R*) sqrt(delta): two roots serve S_n, S_t and F_el
    const F sr = xsqrt_pos(Rs), sd = xsqrt_pos(delta);
    const F sq = sr * sd;
    Sn = F(2) * K.Es * sq;
    St = F(8) * K.Gs * sq;
    cn = K.cdamp * xsqrt_pos(Sn * ms);
    ct = cn * K.ct_ratio;
    fel = K.kn_fac * sr * delta * sd;
  }
  F vn = vrel.x * n.x + vrel.y * n.y + vrel.z * n.z;
  V3<F> vt{vrel.x - vn * n.x, vrel.y - vn * n.y, vrel.z - vn * n.z};
  F fn_s = -fel - cn * vn;  // F_n = fn_s * n
  // spring: rotate onto the tangent plane, keep the length, add v_t dt.  A substep's
  // change, -(xi.n) n + (1/sqrt(1-t) - 1)(xi - (xi.n) n) + v_t dt, is formed in the
  // force word (n, v_t and the projection carry force-word rounding already; a wrong
  // normal part is projected out at the next substep) and added to the spring in the
  // state word, so the history accumulates without losing small changes
  S xi[3];
  F inc[3] = {K.dt * vt.x, K.dt * vt.y, K.dt * vt.z};
  if (has_old) {
    const F xf[3] = {NS::f(xi_old[0]), NS::f(xi_old[1]), NS::f(xi_old[2])};
    const F proj = xf[0] * n.x + xf[1] * n.y + xf[2] * n.z;
    const F len2 = xf[0] * xf[0] + xf[1] * xf[1] + xf[2] * xf[2];
    const F pr[3] = {xf[0] - proj * n.x, xf[1] - proj * n.y, xf[2] - proj * n.z};
    F scm1 = F(0);  // 1/sqrt(1-t) - 1, t = (xi.n)^2 / |xi|^2
    if (len2 > F(0)) {
      const F t = xdiv(proj * proj, len2);
      if (t < F(1)) {
        const F s1 = xsqrt_pos(F(1) - t);
        scm1 = xdiv(t, s1 * (F(1) + s1));
      }
    }
    inc[0] = (scm1 * pr[0] - proj * n.x) + inc[0];
    inc[1] = (scm1 * pr[1] - proj * n.y) + inc[1];
    inc[2] = (scm1 * pr[2] - proj * n.z) + inc[2];
    xi[0] = NS::add_f(xi_old[0], inc[0]);
    xi[1] = NS::add_f(xi_old[1], inc[1]);
    xi[2] = NS::add_f(xi_old[2], inc[2]);
  } else {
    xi[0] = NS::from_f(inc[0]);
    xi[1] = NS::from_f(inc[1]);
    xi[2] = NS::from_f(inc[2]);
  }
  V3<F> Ft{-St * NS::f(xi[0]) - ct * vt.x, -St * NS::f(xi[1]) - ct * vt.y,
           -St * NS::f(xi[2]) - ct * vt.z};
  // Coulomb limit |F_t| <= mu |F_n|, tested on the squares (no root unless sliding)
  const F ft2 = Ft.x * Ft.x + Ft.y * Ft.y + Ft.z * Ft.z;
  const F lim = K.mu * xabs(fn_s);
  if (ft2 > lim * lim) {
    F sc = lim * xrsqrt(ft2);
    Ft.x *= sc;
    Ft.y *= sc;
    Ft.z *= sc;
    F inv = xdiv(F(-1), St);
    xi[0] = NS::from_f((Ft.x + ct * vt.x) * inv);
    xi[1] = NS::from_f((Ft.y + ct * vt.y) * inv);
    xi[2] = NS::from_f((Ft.z + ct * vt.z) * inv);
  }
  xi_new[0] = xi[0];
  xi_new[1] = xi[1];
  xi_new[2] = xi[2];
  *Ft_out = Ft;
  return V3<F>{fn_s * n.x + Ft.x, fn_s * n.y + Ft.y, fn_s * n.z + Ft.z};
}

template <class F>
__device__ __forceinline__ V3<F> cross(V3<F> a, V3<F> b) {
  return V3<F>{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Contribution of one listed partner (list entry e in slot k of owner i) to the
// owner's accumulators: fa (contact force, signed for the owner), t (contact torque
// on the owner), l (lubrication force on the owner).  The pair is evaluated in
// canonical order (lower caller index first), so both sides get bitwise opposite
// forces.  When INTEGRATE, the owner's tangential spring of slot k is updated.
template <class F>
struct PairOut {
  V3<F> fa, t, l, lt;  // contact force (on i), contact torque, lubrication force and torque
  V3<F> G;             // n x F_t in canonical order: the contact torque is lever x G
  F hd;                // delta / 2 (the lever of either sphere is its radius minus it)
  bool contact, lub;
  bool first;          // the owner comes first in the pair (canonical order)
};

// The force of a pair on its owner as the integrating substep adds it: contact plus
// lubrication as one term, summed in canonical order (on the first particle) and
// negated for the second, so that every launch variant adds the same value per slot
// (the pair list stores the canonical sum in the pair's record).
template <class F>
__device__ __forceinline__ V3<F> pair_total(const PairOut<F>& o) {
  const V3<F> z{F(0), F(0), F(0)};
  const V3<F> a = o.contact ? (o.first ? o.fa : V3<F>{-o.fa.x, -o.fa.y, -o.fa.z}) : z;
  const V3<F> b = o.lub ? (o.first ? o.l : V3<F>{-o.l.x, -o.l.y, -o.l.z}) : z;
  const V3<F> c{a.x + b.x, a.y + b.y, a.z + b.z};
  return o.first ? c : V3<F>{-c.x, -c.y, -c.z};
}

// EXT: the optional terms (tangential lubrication here, lift in the fluid force)
// are compiled in; without it the kernel carries none of their registers.
template <int FORM, bool INTEGRATE, bool EXT>
__device__ __forceinline__ PairOut<typename Traits<FORM>::F> pair_eval(
    const DevParams& P, const Quad<typename Traits<FORM>::S>& Pi,
    const typename Traits<FORM>::F* vi, const typename Traits<FORM>::F* vil,
    const typename Traits<FORM>::F* wi, typename Traits<FORM>::F mi, int32_t e, int k, bool has,
    int64_t i, int64_t N,
    const Quad<typename Traits<FORM>::S>* pos, const Quad<typename Traits<FORM>::S>* vel,
    const Quad<typename Traits<FORM>::S>* omg, Quad<typename Traits<FORM>::S>* hist) {
  using S = typename Traits<FORM>::S;
  using F = typename Traits<FORM>::F;
  using NS = Num<S>;
  const ForceConsts<F>& K = fconsts<F>(P);
  const BoxS<S>& B = sbox<S>(P);
  PairOut<F> o;
  o.t = o.lt = o.G = V3<F>{F(0), F(0), F(0)};
  o.hd = F(0);
  o.contact = o.lub = false;
  const int j = nbr_index(e);
  const Quad<S> Pj = ldq(pos + j);
  const bool i_lo = nbr_first(e);
  o.first = i_lo;
  const Quad<S>& A = i_lo ? Pi : Pj;
  const Quad<S>& Bq = i_lo ? Pj : Pi;
  // precise geometry in canonical order: dx = x_B - x_A (minimum image)
  S dxs[3] = {NS::subq(Bq.a, A.a), NS::subq(Bq.b, A.b), NS::subq(Bq.c, A.c)};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!P.periodic[a]) continue;
    // across the periodic face: one shift by a box length toward zero
    const F c = NS::f(dxs[a]);
    if (xabs(c) > K.halfL[a]) dxs[a] = NS::addq(dxs[a], c > F(0) ? NS::neg(B.L[a]) : B.L[a]);
  }
  S d2 = NS::addq(NS::addq(NS::mul(dxs[0], dxs[0]), NS::mul(dxs[1], dxs[1])), NS::mul(dxs[2], dxs[2]));
  S ssum = NS::addq(A.d, Bq.d);
  S num = NS::subq(NS::mul(ssum, ssum), d2);
  const F d2f = NS::f(d2);
  const F inv_d = xrsqrt(d2f);
  const F dist = d2f > F(0) ? d2f * inv_d : F(0);
  const F sF = NS::f(ssum);
  // r_A + r_B - |dx| without cancellation: (s^2 - d^2) / (s + d)
  const F delta = NS::kExtended ? xdiv(NS::f(num), sF + dist) : sF - dist;
  const F dxf[3] = {NS::f(dxs[0]), NS::f(dxs[1]), NS::f(dxs[2])};
  o.contact = delta > F(0);
  o.lub = P.lubrication && (-delta < K.lub_out * sF);
  if (!o.contact && !o.lub) return o;
  const V3<F> n{dxf[0] * inv_d, dxf[1] * inv_d, dxf[2] * inv_d};
  const Quad<S> Vj = ldq(vel + j);
  const F vj[3] = {NS::f(Vj.a), NS::f(Vj.b), NS::f(Vj.c)};
  const F vjl[3] = {NS::lo(Vj.a), NS::lo(Vj.b), NS::lo(Vj.c)};
  // velocity of A relative to B from both words of each velocity: neighbours in a
  // moving bed differ by far less than their speed, so rounding each velocity to one
  // word first would cost the difference most of its digits.  Formed as i minus j and
  // negated when j comes first (exact: rounding is symmetric under negation).
  F dv[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const F d = (vi[a] - vj[a]) + (vil[a] - vjl[a]);
    dv[a] = i_lo ? d : -d;
  }
  F wj[3] = {F(0), F(0), F(0)};
  if (o.contact || (EXT && o.lub && P.lub_tangential)) {
    const Quad<S> Wj = ldq(omg + j);
    wj[0] = NS::f(Wj.a);
    wj[1] = NS::f(Wj.b);
    wj[2] = NS::f(Wj.c);
  }
  const F* wA = i_lo ? wi : wj;
  const F* wB = i_lo ? wj : wi;
  if (o.contact) {
    const F rA = NS::f(A.d), rB = NS::f(Bq.d);
    const F mA = i_lo ? mi : NS::f(Vj.d);
    const F mB = i_lo ? NS::f(Vj.d) : mi;
    const F Rs = xdiv(rA * rB, rA + rB);
    const F ms = xdiv(mA * mB, mA + mB);
    o.hd = F(0.5) * delta;
    const F la = rA - o.hd, lb = rB - o.hd;
    V3<F> om{la * wA[0] + lb * wB[0], la * wA[1] + lb * wB[1], la * wA[2] + lb * wB[2]};
    V3<F> wxn = cross(om, n);
    V3<F> vrel{dv[0] + wxn.x, dv[1] + wxn.y, dv[2] + wxn.z};
    S xo[3], xn_[3];
    if (has) {
      const Quad<S> h = ldq(hist + (int64_t)k * N + i);
      xo[0] = h.a;
      xo[1] = h.b;
      xo[2] = h.c;
    }
    V3<F> Ft;
    V3<F> FA = hm_core<S, F>(K, n, delta, Rs, ms, vrel, xo, has, &Ft, xn_);
    if (INTEGRATE) stq(hist + (int64_t)k * N + i, Quad<S>{xn_[0], xn_[1], xn_[2], NS::from_f(F(0))});
    const F lev = i_lo ? la : lb;
    o.G = cross(n, Ft);
    o.t = V3<F>{lev * o.G.x, lev * o.G.y, lev * o.G.z};
    o.fa = i_lo ? FA : V3<F>{-FA.x, -FA.y, -FA.z};
  }
  if (o.lub) {
    const F h = -delta;
    const F hin = K.lub_in * sF;
    const F hh = h > hin ? h : hin;
    const F rA = NS::f(A.d), rB = NS::f(Bq.d);
    const F Rl = xdiv(rA * rB, rA + rB);
    const F vn = dv[0] * n.x + dv[1] * n.y + dv[2] * n.z;
    F sl = xdiv(-K.six_pi_mu * Rl * Rl * vn, hh);
    if (!i_lo) sl = -sl;
    o.l = V3<F>{sl * n.x, sl * n.y, sl * n.z};
    if (EXT && P.lub_tangential) {
      // shear term: -6 pi mu R_l (4/15) (2 + b + 2 b^2)/(1 + b)^2 ln((r_A + r_B) / 2h) v_t,
      // b = r_B / r_A, v_t the tangential surface velocity of A relative to B at the
      // gap midpoint (lever arms r + h/2); torque l n x F on both spheres
      const F la = rA + F(0.5) * h, lb = rB + F(0.5) * h;
      const V3<F> om{la * wA[0] + lb * wB[0], la * wA[1] + lb * wB[1], la * wA[2] + lb * wB[2]};
      const V3<F> wxn = cross(om, n);
      const V3<F> vr{dv[0] + wxn.x, dv[1] + wxn.y, dv[2] + wxn.z};
      const F vrn = vr.x * n.x + vr.y * n.y + vr.z * n.z;
      const F b = rB / rA;
      const F shape = (F(2) + b + F(2) * b * b) / ((F(1) + b) * (F(1) + b));
      F lg = xlog(sF / (F(2) * hh));
      if (lg < F(0)) lg = F(0);
      const F ct = -K.six_pi_mu * Rl * F(4.0 / 15.0) * shape * lg;
      const V3<F> Ft{ct * (vr.x - vrn * n.x), ct * (vr.y - vrn * n.y), ct * (vr.z - vrn * n.z)};
      const F lev = i_lo ? la : lb;
      o.lt = cross(V3<F>{lev * n.x, lev * n.y, lev * n.z}, Ft);
      if (i_lo) {
        o.l.x += Ft.x; o.l.y += Ft.y; o.l.z += Ft.z;
      } else {
        o.l.x -= Ft.x; o.l.y -= Ft.y; o.l.z -= Ft.z;
      }
    }
  }
  return o;
}

}  // namespace

// Pair forces from the pair list: one thread per listed pair, from the particle
// that comes first in it.  The same FP32 cull and the same pair evaluation as the
// per-particle loop.  Every listed pair's record is written each substep, in pair
// order (one 32-byte sector per pair, so the writes are sequential and whole):
// {F, delta/2} {G, flags} with F the pair force on the first particle, G = n x F_t,
// and zero flags for a pair that does not interact.  The spring goes to the first
// particle's slot.  The pairs run independently, so the order in which they are
// taken does not change any result.  Integrating substeps only: the force export
// runs the per-particle loop, which keeps contact and lubrication apart.
//
// Two schedules.  Grid-stride (ORDERED false): thread t of a fixed grid takes pairs
// t, t + T, t + 2T, ...; with more blocks than fit on the GPU at once, each wave of
// resident blocks sweeps the whole list, so a particle's records are fetched again by
// every wave that reaches one of its pairs.  Ordered (ORDERED true): one wave of
// blocks takes blockDim.x consecutive pairs at a time from a counter (the next chunk
// claimed while the current one runs), so the pairs in flight are one narrow window
// of the list and the partners' records read by a pair are mostly still in L2 when
// the partners' own pairs come up (on the 10M bed: 34% fewer DRAM reads, 6% shorter
// substep launch; on beds whose lists fit in L2 the claims cost a little instead).
// The last block to finish resets the counter for the next launch.
// The arrays of one pair pass (the pair kernel's views of the current substep).
template <int FORM>
struct PairPass {
  using S = typename Traits<FORM>::S;
  const Quad<S>* pos;
  const Quad<S>* vel;
  const Quad<S>* omg;
  const uint32_t* cmask;
  Quad<S>* hist;
  float4* prec;
  const int4* pairs;
  int64_t N, M;  // particles; listed pairs
  float fac;     // the FP32 cull's cutoff factor (lubrication range)
};

template <int FORM>
__device__ __forceinline__ PairPass<FORM> pair_pass(const DevState& st, const DevParams& P, int sub_off) {
  using S = typename Traits<FORM>::S;
  const Ctl* ctl = st.ctl;
  const int sb = (ctl->st + sub_off) & 1;
  const int nl = ctl->nl;
  PairPass<FORM> pp;
  pp.pos = (const Quad<S>*)st.pos[sb];
  pp.vel = (const Quad<S>*)st.vel[sb];
  pp.omg = (const Quad<S>*)st.omg[sb];
  pp.cmask = st.cmask[nl];
  pp.hist = (Quad<S>*)st.hist[nl];
  pp.prec = st.prec;
  pp.pairs = st.pairs;
  pp.N = st.N;
  pp.M = (int64_t)ctl->npair < st.pcap ? (int64_t)ctl->npair : st.pcap;
  pp.fac = P.lubrication ? (1.0f + P.lub_out_f) : 1.0f;
  return pp;
}

// Listed pair m: its record (and the first particle's spring).
template <int FORM>
__device__ __forceinline__ void pair_record(const PairPass<FORM>& pp, const DevParams& P, const int64_t m) {
  using S = typename Traits<FORM>::S;
  using F = typename Traits<FORM>::F;
  using NS = Num<S>;
  static_assert(sizeof(F) == 4, "pair records hold FP32 force words");
  const Quad<S>* pos = pp.pos;
  const Quad<S>* vel = pp.vel;
  const Quad<S>* omg = pp.omg;
  Quad<S>* hist = pp.hist;
  const int64_t N = pp.N;
  const float fac = pp.fac;
  const int4 pr = pp.pairs[m];
  const int64_t i = pr.x;
  const Quad<S> Pi = ldq(pos + i);
  const Quad<S> Pv = ldq(pos + pr.z);
  const uint32_t cm = pp.cmask[i];
  // the records an interacting pair reads next, fetched with the positions
  prefetch_l1(vel + i);
  prefetch_l1(omg + i);
  prefetch_l1(vel + pr.z);
  prefetch_l1(omg + pr.z);
  float dx = (float)NS::dif(Pv.a, Pi.a), dy = (float)NS::dif(Pv.b, Pi.b), dz = (float)NS::dif(Pv.c, Pi.c);
  if (P.periodic[0]) dx = dx > P.cf.halfL[0] ? dx - P.cf.L[0] : (dx < -P.cf.halfL[0] ? dx + P.cf.L[0] : dx);
  if (P.periodic[1]) dy = dy > P.cf.halfL[1] ? dy - P.cf.L[1] : (dy < -P.cf.halfL[1] ? dy + P.cf.L[1] : dy);
  if (P.periodic[2]) dz = dz > P.cf.halfL[2] ? dz - P.cf.L[2] : (dz < -P.cf.halfL[2] ? dz + P.cf.L[2] : dz);
  const float cut = ((float)NS::f(Pi.d) + (float)NS::f(Pv.d)) * fac;
  float4 r0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), r1 = r0;
  if (dx * dx + dy * dy + dz * dz <= cut * cut * 1.0002f) {
    const int k = pr.y;
    const bool has = (cm >> k) & 1u;
    if (has) prefetch_l1(hist + (int64_t)k * N + i);
    const Quad<S> Vi = ldq(vel + i), Wi = ldq(omg + i);
    const F vi[3] = {NS::f(Vi.a), NS::f(Vi.b), NS::f(Vi.c)};
    const F vil[3] = {NS::lo(Vi.a), NS::lo(Vi.b), NS::lo(Vi.c)};
    const F wi[3] = {NS::f(Wi.a), NS::f(Wi.b), NS::f(Wi.c)};
    // the first particle of a listed pair is pr.x, so its list entry is the partner
    // with the first bit set
    const PairOut<F> o = pair_eval<FORM, true, false>(
        P, Pi, vi, vil, wi, NS::f(Vi.d), (int32_t)((uint32_t)pr.z | kFirstBit), k, has, i, N, pos,
        vel, omg, hist);
    const uint32_t fg = (o.contact || o.lub ? kSlotForce : 0u) | (o.contact ? kSlotContact : 0u);
    if (fg) {
      const V3<F> f = pair_total(o);
      r0 = make_float4(f.x, f.y, f.z, o.hd);
      r1 = make_float4(o.G.x, o.G.y, o.G.z, __uint_as_float(fg));
    }
  }
  pp.prec[2 * m] = r0;
  pp.prec[2 * m + 1] = r1;
}

template <int FORM, bool ORDERED>
__device__ __forceinline__ void pair_forces_body(const DevState& st, const DevParams& P, int sub_off) {
  Ctl* ctl = st.ctl;
  const PairPass<FORM> pp = pair_pass<FORM>(st, P, sub_off);
  const int64_t M = pp.M;
  if constexpr (ORDERED) {
    // chunk claims, two ahead of use: s_base[it % 3] is this round's chunk,
    // s_base[(it + 1) % 3] the next one (claimed last round), and thread 0 claims the
    // one after into the slot every thread finished reading before the last barrier
    __shared__ int64_t s_base[3];
    const int64_t chunk = blockDim.x;
    if (threadIdx.x == 0) {
      s_base[0] = (int64_t)atomicAdd(&ctl->pair_next, 1u) * chunk;
      s_base[1] = (int64_t)atomicAdd(&ctl->pair_next, 1u) * chunk;
    }
    __syncthreads();
    for (int it = 0;; ++it) {
      const int64_t base = s_base[it % 3];
      if (base >= M) break;  // the same value for the whole block
      if (threadIdx.x == 0) s_base[(it + 2) % 3] = (int64_t)atomicAdd(&ctl->pair_next, 1u) * chunk;
      const int64_t m = base + threadIdx.x;
      if (m < M) pair_record<FORM>(pp, P, m);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      // this block's claims are ordered before its completion count; the last block
      // to finish sees every claim and resets the counter
      __threadfence();
      if (atomicAdd(&ctl->pair_done, 1u) == gridDim.x - 1) {
        atomicExch(&ctl->pair_next, 0u);
        atomicExch(&ctl->pair_done, 0u);
      }
    }
  } else {
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x)
      pair_record<FORM>(pp, P, m);
  }
}

template <int FORM, bool ORDERED>
__global__ void __launch_bounds__(128, 7) k_pair_forces(DevState st, DevParams P, int sub_off) {
  pair_forces_body<FORM, ORDERED>(st, P, sub_off);
}

// BS threads per block, at least MINB resident blocks per SM (which caps the
// registers a thread may use); the variant is chosen per workload by the engine's
// autotuner.
// Body of the fused substep for one bed: blk is the block's index within the bed,
// nblk the bed's block count; ectl (ensembles only) collects the rebuild decision
// of all nbeds beds for the graph condition of the next substep.
// GATHER: the pair forces come from the pair list (k_pair_forces ran before); each
// particle adds its pairs' records in slot order, the same additions in the same
// order as the per-particle loop.
template <int FORM, bool INTEGRATE, int BS, bool COOP, bool EXT, bool GATHER = false>
__device__ __forceinline__ void substep_body(const DevState& st, const DevMesh& mesh,
                                             const DevParams& P, int sub_off,
                                             cudaGraphConditionalHandle next, int use_cond,
                                             int64_t blk, unsigned nblk, Ctl* ectl, int nbeds) {
  using S = typename Traits<FORM>::S;
  using F = typename Traits<FORM>::F;
  using NS = Num<S>;
  const ForceConsts<F>& K = fconsts<F>(P);
  const BoxS<S>& B = sbox<S>(P);
  const Ctl* ctl = st.ctl;
  const int sb = (ctl->st + sub_off) & 1;
  const int pb = ctl->pb;
  const int nl = ctl->nl;
  const int64_t N = st.N;
  const int64_t i = blk * BS + threadIdx.x;
  const bool valid = i < N;
  float my_disp2 = 0.0f;
  const Quad<S>* pos = (const Quad<S>*)st.pos[sb];
  const Quad<S>* vel = (const Quad<S>*)st.vel[sb];
  const Quad<S>* omg = (const Quad<S>*)st.omg[sb];
  Quad<F>* accp = (Quad<F>*)st.acc[pb];
  const int32_t* nbr = st.nbr[nl];
  Quad<S>* hist = (Quad<S>*)st.hist[nl];
  Quad<S> Pi{}, Vi{}, Wi{};
  Quad<F> Ai{};
  F ri = F(0), mi = F(0);
  F vi[3] = {F(0), F(0), F(0)}, wi[3] = {F(0), F(0), F(0)}, vil[3] = {F(0), F(0), F(0)};
  V3<F> fc{0, 0, 0}, fl{0, 0, 0}, tq{0, 0, 0};
  uint32_t mask = 0, nmask = 0, live = 0;
  // the particle's own records (loaded before the pair phase in every mode: in the
  // gather mode their loads overlap the first pair records' round trip)
  auto load_own = [&]() {
    Pi = ldq(pos + i);
    Vi = ldq(vel + i);
    Wi = ldq(omg + i);
    Ai = ldq(accp + i);
    ri = NS::f(Pi.d);
    mi = NS::f(Vi.d);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      vi[a] = NS::f(a == 0 ? Vi.a : (a == 1 ? Vi.b : Vi.c));
      vil[a] = NS::lo(a == 0 ? Vi.a : (a == 1 ? Vi.b : Vi.c));
      wi[a] = NS::f(a == 0 ? Wi.a : (a == 1 ? Wi.b : Wi.c));
    }
  };
  if (valid) {
    load_own();
    const int nn = st.nn[nl][i];
    mask = st.cmask[nl][i];
    if constexpr (GATHER) {
      (void)nn;  // the slots come from the pair kernel's masks
    } else {
    const float lub_out_f = P.lub_out_f;
    // phase 1: cheap FP32 cull of every listed partner (relative margin; the exact
    // test follows); four candidates per round so their gathers overlap
    const float rif = (float)ri;
    const float fac = P.lubrication ? (1.0f + lub_out_f) : 1.0f;
    for (int k0 = 0; k0 < nn; k0 += 4) {
      int32_t ev[4];
      Quad<S> Pv[4];
      const int32_t* ep = nbr + (int64_t)k0 * N + i;
#pragma unroll
      for (int u = 0; u < 4; ++u) ev[u] = k0 + u < nn ? ep[u * N] : 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) Pv[u] = ldq(pos + (k0 + u < nn ? nbr_index(ev[u]) : (int)i));
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float dx = (float)NS::dif(Pv[u].a, Pi.a), dy = (float)NS::dif(Pv[u].b, Pi.b),
              dz = (float)NS::dif(Pv[u].c, Pi.c);
        if (P.periodic[0]) dx = dx > P.cf.halfL[0] ? dx - P.cf.L[0] : (dx < -P.cf.halfL[0] ? dx + P.cf.L[0] : dx);
        if (P.periodic[1]) dy = dy > P.cf.halfL[1] ? dy - P.cf.L[1] : (dy < -P.cf.halfL[1] ? dy + P.cf.L[1] : dy);
        if (P.periodic[2]) dz = dz > P.cf.halfL[2] ? dz - P.cf.L[2] : (dz < -P.cf.halfL[2] ? dz + P.cf.L[2] : dz);
        const float cut = (rif + (float)NS::f(Pv[u].d)) * fac;
        if (k0 + u < nn && dx * dx + dy * dy + dz * dz <= cut * cut * 1.0002f) live |= 1u << (k0 + u);
      }
    }
    }
  }
  // phase 2: interacting pairs only, in slot order.  An integrating substep adds each
  // pair's force (contact plus lubrication, pair_total) to fc as one term; the force
  // export keeps contact (fc) and lubrication (fl) apart.
  if constexpr (GATHER) {
    static_assert(INTEGRATE, "the pair list serves integrating substeps only");
    // the pair records of this particle's slots, in slot order: the slot's pair id
    // (slot-major rows: a warp reads contiguous words), then the pair's sector
    const int nn = valid ? st.nn[nl][i] : 0;
    const int32_t* pid = st.pid;
    const float4* prec = st.prec;
    for (int k = 0; k < nn; ++k) prefetch_l1(pid + (int64_t)k * N + i);
    constexpr int kGatherBatch = 4;
    for (int k0 = 0; k0 < nn; k0 += kGatherBatch) {
      int32_t e[kGatherBatch];
#pragma unroll
      for (int u = 0; u < kGatherBatch; ++u) e[u] = k0 + u < nn ? pid[(int64_t)(k0 + u) * N + i] : -1;
      float4 ra[kGatherBatch], rb[kGatherBatch];
#pragma unroll
      for (int u = 0; u < kGatherBatch; ++u) {
        const int64_t m = (int64_t)nbr_index(e[u]);
        const bool ok = e[u] != -1 && m < st.pcap;
        ra[u] = ok ? prec[2 * m] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        rb[u] = ok ? prec[2 * m + 1] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
#pragma unroll
      for (int u = 0; u < kGatherBatch; ++u) {
        const uint32_t fg = __float_as_uint(rb[u].w);
        // the record holds the force on the first particle; the partner gets minus it
        if (fg & kSlotForce) {
          if (nbr_first(e[u])) {
            fc.x += ra[u].x; fc.y += ra[u].y; fc.z += ra[u].z;
          } else {
            fc.x += -ra[u].x; fc.y += -ra[u].y; fc.z += -ra[u].z;
          }
        }
        if (fg & kSlotContact) {
          const F lev = ri - ra[u].w;
          tq.x += lev * rb[u].x; tq.y += lev * rb[u].y; tq.z += lev * rb[u].z;
          nmask |= 1u << (k0 + u);
        }
      }
    }
  } else if constexpr (COOP) {
    // warp-cooperative: the warp's (owner lane, slot) pairs are queued in slot order
    // and evaluated 32 at a time, one per lane; each owner then adds its results in
    // queue order, i.e. the same additions in the same order as the loop below
    constexpr int W = BS / 32;
    __shared__ uint16_t q_pair[W][1024];
    __shared__ Quad<S> q_pi[W][32];
    __shared__ F q_vw[W][32][12];  // vi, wi, mi, (pad), low words of vi, (pad)
    __shared__ uint32_t q_mask[W][32];
    __shared__ F q_res[W][32][EXT ? 12 : 9];
    __shared__ uint8_t q_flag[W][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int cnt = __popc(live);
    int off = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, off, o);
      if (lane >= o) off += t;
    }
    const int total = __shfl_sync(0xffffffffu, off, 31);
    off -= cnt;  // exclusive prefix
    q_pi[wid][lane] = Pi;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      q_vw[wid][lane][a] = vi[a];
      q_vw[wid][lane][3 + a] = wi[a];
      q_vw[wid][lane][8 + a] = vil[a];
    }
    q_vw[wid][lane][6] = mi;
    q_mask[wid][lane] = mask;
    {
      uint32_t lv = live;
      int t = off;
      while (lv) {
        const int k = __ffs(lv) - 1;
        lv &= lv - 1;
        q_pair[wid][t++] = (uint16_t)((lane << 8) | k);
      }
    }
    __syncwarp();
    const int64_t i0 = i - lane;  // particle of lane 0
    for (int base = 0; base < total; base += 32) {
      const int p = base + lane;
      if (p < total) {
        const int e = q_pair[wid][p];
        const int L = e >> 8, k = e & 255;
        const int64_t iL = i0 + L;
        const F* vw = q_vw[wid][L];
        const PairOut<F> o = pair_eval<FORM, INTEGRATE, EXT>(P, q_pi[wid][L], vw, vw + 8, vw + 3, vw[6],
                                                        nbr[(int64_t)k * N + iL], k,
                                                        (q_mask[wid][L] >> k) & 1u, iL, N, pos, vel,
                                                        omg, hist);
        F* r = q_res[wid][lane];
        const V3<F> f0 = INTEGRATE ? pair_total(o) : o.fa;
        r[0] = f0.x; r[1] = f0.y; r[2] = f0.z;
        r[3] = o.t.x; r[4] = o.t.y; r[5] = o.t.z;
        r[6] = o.l.x; r[7] = o.l.y; r[8] = o.l.z;
        if constexpr (EXT) {
          r[9] = o.lt.x; r[10] = o.lt.y; r[11] = o.lt.z;
        }
        q_flag[wid][lane] = (uint8_t)((o.contact ? 1 : 0) | (o.lub ? 2 : 0));
      }
      __syncwarp();
      // this lane's queue entries inside the round, in order
      const int q0 = off > base ? off : base;
      const int q1 = off + cnt < base + 32 ? off + cnt : base + 32;
      for (int q = q0; q < q1; ++q) {
        const F* r = q_res[wid][q - base];
        const int fg = q_flag[wid][q - base];
        if (INTEGRATE) {
          if (fg & 3) {
            fc.x += r[0]; fc.y += r[1]; fc.z += r[2];
          }
        } else {
          if (fg & 1) {
            fc.x += r[0]; fc.y += r[1]; fc.z += r[2];
          }
          if (fg & 2) {
            fl.x += r[6]; fl.y += r[7]; fl.z += r[8];
          }
        }
        if (fg & 1) {
          tq.x += r[3]; tq.y += r[4]; tq.z += r[5];
          if (INTEGRATE) nmask |= 1u << (q_pair[wid][q] & 255);
        }
        if (fg & 2) {
          if constexpr (EXT) {
            if (P.lub_tangential) {
              tq.x += r[9]; tq.y += r[10]; tq.z += r[11];
            }
          }
        }
      }
      __syncwarp();
    }
  } else {
      while (live) {
        const int k = __ffs(live) - 1;
        live &= live - 1;
        const PairOut<F> o = pair_eval<FORM, INTEGRATE, EXT>(P, Pi, vi, vil, wi, mi, nbr[(int64_t)k * N + i], k,
                                                        (mask >> k) & 1u, i, N, pos, vel, omg, hist);
        if (INTEGRATE) {
          if (o.contact || o.lub) {
            const V3<F> f = pair_total(o);
            fc.x += f.x; fc.y += f.y; fc.z += f.z;
          }
        } else {
          if (o.contact) {
            fc.x += o.fa.x; fc.y += o.fa.y; fc.z += o.fa.z;
          }
          if (o.lub) {
            fl.x += o.l.x; fl.y += o.l.y; fl.z += o.l.z;
          }
        }
        if (o.contact) {
          tq.x += o.t.x; tq.y += o.t.y; tq.z += o.t.z;
          if (INTEGRATE) nmask |= 1u << k;
        }
        if (o.lub) {
          if (EXT && P.lub_tangential) {
            tq.x += o.lt.x; tq.y += o.lt.y; tq.z += o.lt.z;
          }
        }
      }
  }
  if (valid) {
    // walls (planes of the same material)
    uint32_t wmask_old = st.wmask[pb][i], wmask_new = 0;
    S* whist = (S*)st.whist[pb];
    const S xi_s[3] = {Pi.a, Pi.b, Pi.c};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (P.periodic[a]) continue;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        if (side == 0 ? !P.wall_lo[a] : !P.wall_hi[a]) continue;
        // overlap r - dist in the state word (dist = x - lo or hi - x)
        S dist_s = side == 0 ? NS::subq(xi_s[a], B.lo[a]) : NS::subq(B.hi[a], xi_s[a]);
        const F delta = NS::f(NS::subq(Pi.d, dist_s));
        V3<F> n{0, 0, 0};
        const F sgn = side == 0 ? F(-1) : F(1);
        if (a == 0) n.x = sgn; else if (a == 1) n.y = sgn; else n.z = sgn;
        const int w = 2 * a + side;
        if (delta > F(0)) {
          const F l = ri - F(0.5) * delta;
          V3<F> wxn = cross(V3<F>{l * wi[0], l * wi[1], l * wi[2]}, n);
          V3<F> vrel{vi[0] + wxn.x, vi[1] + wxn.y, vi[2] + wxn.z};
          S xo[3], xn_[3];
          const bool has = (wmask_old >> w) & 1u;
          if (has) {
#pragma unroll
            for (int c = 0; c < 3; ++c) xo[c] = whist[((int64_t)w * 3 + c) * N + i];
          }
          V3<F> Ft;
          V3<F> FA = hm_core<S, F>(K, n, delta, ri, mi, vrel, xo, has, &Ft, xn_);
          if (INTEGRATE) {
#pragma unroll
            for (int c = 0; c < 3; ++c) whist[((int64_t)w * 3 + c) * N + i] = xn_[c];
            wmask_new |= 1u << w;
          }
          V3<F> T = cross(V3<F>{l * n.x, l * n.y, l * n.z}, Ft);
          fc.x += FA.x; fc.y += FA.y; fc.z += FA.z;
          tq.x += T.x; tq.y += T.y; tq.z += T.z;
        }
        if (P.lubrication) {
          const F dbar = F(2) * ri;
          const F h = -delta;
          if (h < K.lub_out * dbar) {
            const F hin = K.lub_in * dbar;
            const F hh = h > hin ? h : hin;
            const F vn = vi[0] * n.x + vi[1] * n.y + vi[2] * n.z;
            const F s = xdiv(-K.six_pi_mu * ri * ri * vn, hh);
            fl.x += s * n.x; fl.y += s * n.y; fl.z += s * n.z;
            if (EXT && P.lub_tangential) {
              // shear term against the plane: -6 pi mu r (8/15) ln(r / h) v_t
              const F l = ri + F(0.5) * h;
              const V3<F> wxn = cross(V3<F>{l * wi[0], l * wi[1], l * wi[2]}, n);
              const V3<F> vr{vi[0] + wxn.x, vi[1] + wxn.y, vi[2] + wxn.z};
              const F vrn = vr.x * n.x + vr.y * n.y + vr.z * n.z;
              F lg = xlog(ri / hh);
              if (lg < F(0)) lg = F(0);
              const F ct = -K.six_pi_mu * ri * F(8.0 / 15.0) * lg;
              const V3<F> Ft{ct * (vr.x - vrn * n.x), ct * (vr.y - vrn * n.y), ct * (vr.z - vrn * n.z)};
              const V3<F> T = cross(V3<F>{l * n.x, l * n.y, l * n.z}, Ft);
              fl.x += Ft.x; fl.y += Ft.y; fl.z += Ft.z;
              tq.x += T.x; tq.y += T.y; tq.z += T.z;
            }
          }
        }
      }
    }
    // fluid forces at the particle
    F ff[3];
    const F ap[3] = {Ai.a, Ai.b, Ai.c};
    fluid_force<S, F, EXT>(P, K, (const Quad<F>*)mesh.ufe, (const Quad<F>*)mesh.gfl,
                           (const Quad<F>*)mesh.wfl, zcent<F>(mesh), xi_s, ri, vi, ap, ff);
    if (!INTEGRATE) {
      double* o = st.fdbg;
      o[3 * i + 0] = (double)fc.x; o[3 * i + 1] = (double)fc.y; o[3 * i + 2] = (double)fc.z;
      o += 3 * N;
      o[3 * i + 0] = (double)fl.x; o[3 * i + 1] = (double)fl.y; o[3 * i + 2] = (double)fl.z;
      o += 3 * N;
      o[3 * i + 0] = (double)ff[0]; o[3 * i + 1] = (double)ff[1]; o[3 * i + 2] = (double)ff[2];
      o += 3 * N;
      o[3 * i + 0] = (double)tq.x; o[3 * i + 1] = (double)tq.y; o[3 * i + 2] = (double)tq.z;
    } else {
      // leapfrog: v += dt a, w += dt T / I, x += dt v (state word)
      const F inv_m = xdiv(F(1), mi);
      F acc[3] = {xfma(fc.x + fl.x + ff[0], inv_m, K.g[0]), xfma(fc.y + fl.y + ff[1], inv_m, K.g[1]),
                  xfma(fc.z + fl.z + ff[2], inv_m, K.g[2])};
      const F inv_I = xdiv(F(2.5), mi * ri * ri);
      F alp[3] = {tq.x * inv_I, tq.y * inv_I, tq.z * inv_I};
      S vn[3] = {NS::fmaq(Vi.a, K.dt, acc[0]), NS::fmaq(Vi.b, K.dt, acc[1]),
                 NS::fmaq(Vi.c, K.dt, acc[2])};
      S wn[3] = {NS::fmaq(Wi.a, K.dt, alp[0]), NS::fmaq(Wi.b, K.dt, alp[1]),
                 NS::fmaq(Wi.c, K.dt, alp[2])};
      S xn[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        S x = NS::addq(xi_s[a], NS::mul_f(vn[a], K.dt));
        if (P.periodic[a]) {
          if (NS::lt(x, B.lo[a])) x = NS::add(x, B.L[a]);
          else if (!NS::lt(x, B.hi[a])) x = NS::sub(x, B.L[a]);
        }
        xn[a] = x;
      }
      if (!(xisfinite(acc[0]) && xisfinite(acc[1]) && xisfinite(acc[2]) &&
            xisfinite(alp[0]) && xisfinite(alp[1]) && xisfinite(alp[2])))
        atomicCAS((int*)&st.ctl->error, 0, -7);
      const int ob = sb ^ 1;
      stq((Quad<S>*)st.pos[ob] + i, Quad<S>{xn[0], xn[1], xn[2], Pi.d});
      stq((Quad<S>*)st.vel[ob] + i, Quad<S>{vn[0], vn[1], vn[2], Vi.d});
      stq((Quad<S>*)st.omg[ob] + i, Quad<S>{wn[0], wn[1], wn[2], Wi.d});
      stq(accp + i, Quad<F>{acc[0], acc[1], acc[2], F(0)});
      st.cmask[nl][i] = nmask;
      st.wmask[pb][i] = wmask_new;
      // displacement since the last rebuild (FP32, minimum image)
      const float4 b = st.xb[pb][i];
      float e[3] = {(float)NS::f(xn[0]) - b.x, (float)NS::f(xn[1]) - b.y,
                    (float)NS::f(xn[2]) - b.z};
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (P.periodic[a]) {
          if (e[a] > P.cf.halfL[a]) e[a] -= P.cf.L[a];
          else if (e[a] < -P.cf.halfL[a]) e[a] += P.cf.L[a];
        }
      my_disp2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
      if (!(my_disp2 < 3.0e38f)) my_disp2 = 3.0e38f;
    }
  }
  if (INTEGRATE) {
    // block max of the squared displacement -> one atomic per block
    float m = my_disp2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wmax[BS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wmax[wid] = m;
    __syncthreads();
    if (wid == 0) {
      m = lane < (int)(blockDim.x >> 5) ? wmax[lane] : 0.0f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0 && m > 0.0f) atomicMax(&st.ctl->disp_max_bits, __float_as_uint(m));
    }
    // the last block to finish decides whether the lists must be rebuilt before the
    // next substep (and sets the graph condition of that substep's rebuild node)
    // (thread 0 made this block's displacement atomic above; its fence orders it
    // before the completion count)
    __shared__ bool last;
    if (threadIdx.x == 0) {
      __threadfence();
      last = atomicAdd(&st.ctl->blocks_done, 1u) == nblk - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
      __threadfence();
      const float mx = __uint_as_float(atomicAdd(&st.ctl->disp_max_bits, 0u));
      const int need = mx > P.half_skin_f * P.half_skin_f ? 1 : 0;
      st.ctl->need_rebuild = need;
      st.ctl->blocks_done = 0u;
      if (ectl) {
        // the last bed to finish sets the condition: rebuild if any bed needs it
        if (need) atomicOr(&ectl->need_rebuild, 1);
        __threadfence();
        if (atomicAdd(&ectl->blocks_done, 1u) == (unsigned)nbeds - 1) {
          __threadfence();
          const int any = atomicExch(&ectl->need_rebuild, 0);
          ectl->blocks_done = 0u;
          ectl->ens_rebuild = any;
          if (use_cond) cudaGraphSetConditional(next, any ? 1u : 0u);
        }
      } else if (use_cond) {
        cudaGraphSetConditional(next, need ? 1u : 0u);
      }
    }
  }
}

template <int FORM, bool INTEGRATE, int BS, int MINB, bool COOP, bool EXT, bool GATHER = false>
__global__ void __launch_bounds__(BS, MINB) k_substep(DevState st, DevMesh mesh, DevParams P,
                                                         int sub_off, cudaGraphConditionalHandle next,
                                                         int use_cond) {
  substep_body<FORM, INTEGRATE, BS, COOP, EXT, GATHER>(st, mesh, P, sub_off, next, use_cond,
                                                       blockIdx.x, gridDim.x, nullptr, 1);
}

// Ensemble: blockIdx.y is the bed, blockIdx.x the block within it (blocks past the
// bed's particles return at once).
template <int FORM, int BS, int MINB, bool COOP, bool EXT>
__global__ void __launch_bounds__(BS, MINB) k_substep_e(const BedView* v, int nbeds, Ctl* ectl,
                                                           int sub_off, cudaGraphConditionalHandle next,
                                                           int use_cond) {
  const int64_t N = v[blockIdx.y].st.N;
  const unsigned nblk = (unsigned)((N + BS - 1) / BS);
  if (blockIdx.x >= nblk) return;
  const BedView& b = bed_view(v);
  substep_body<FORM, true, BS, COOP, EXT>(b.st, b.mesh, b.P, sub_off, next, use_cond, blockIdx.x,
                                          nblk, ectl, nbeds);
}

template <int FORM, int BS, int MINB, bool COOP, bool EXT = false>
static void launch_bs(const DevState& st, const DevMesh& mesh, const DevParams& P, int sub_off,
                      bool integrate, unsigned long long next, int use_cond, cudaStream_t s) {
  const int64_t grid = (st.N + BS - 1) / BS;
  const cudaGraphConditionalHandle h = (cudaGraphConditionalHandle)next;
  if (integrate)
    k_substep<FORM, true, BS, MINB, COOP, EXT><<<(unsigned)grid, BS, 0, s>>>(st, mesh, P, sub_off, h, use_cond);
  else
    k_substep<FORM, false, BS, MINB, COOP, EXT><<<(unsigned)grid, BS, 0, s>>>(st, mesh, P, sub_off, h, 0);
}

// Pair list: the pair forces (on a fixed grid: the pair count lives on the device),
// then the per-particle kernel gathering the records.  The ordered schedule runs one
// wave of blocks (every block resident at once, each claiming chunks until the list
// is done); the grid-stride schedule up to 32 blocks per SM.
template <int FORM>
static void launch_pairs(const DevState& st, const DevMesh& mesh, const DevParams& P, int sub_off,
                         bool ordered, unsigned long long next, int use_cond, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int64_t g = (st.pcap + 127) / 128;
  if (ordered) {
    static int per_sm = 0;  // resident blocks of the ordered kernel per SM (one device)
    if (per_sm <= 0 &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair_forces<FORM, true>, 128, 0) != cudaSuccess)
      per_sm = 1;
    if (per_sm <= 0) per_sm = 1;
    g = (int64_t)nsm * per_sm;
  } else {
    const int64_t gmax = (int64_t)nsm * 8 * 4;
    if (g > gmax) g = gmax;
  }
  if (g < 1) g = 1;
  const int64_t grid = (st.N + 127) / 128;
  const cudaGraphConditionalHandle h = (cudaGraphConditionalHandle)next;
  if (ordered) k_pair_forces<FORM, true><<<(unsigned)g, 128, 0, s>>>(st, P, sub_off);
  else k_pair_forces<FORM, false><<<(unsigned)g, 128, 0, s>>>(st, P, sub_off);
  k_substep<FORM, true, 128, 6, false, false, true><<<(unsigned)grid, 128, 0, s>>>(st, mesh, P, sub_off, h, use_cond);
}

template <int FORM>
static void launch_one(const DevState& st, const DevMesh& mesh, const DevParams& P, int sub_off,
                       bool integrate, int variant, unsigned long long next, int use_cond,
                       cudaStream_t s) {
  // the optional terms (lift, tangential lubrication) and the parity form run the
  // per-particle pair loop at 128 threads
  if (P.lift || P.lub_tangential) {
    launch_bs<FORM, 128, 6, false, true>(st, mesh, P, sub_off, integrate, next, use_cond, s);
    return;
  }
  if constexpr (FORM != FORM_FP64) {
    switch (variant) {
      case SUBSTEP_B64: launch_bs<FORM, 64, 12, true>(st, mesh, P, sub_off, integrate, next, use_cond, s); return;
      case SUBSTEP_B256: launch_bs<FORM, 256, 3, true>(st, mesh, P, sub_off, integrate, next, use_cond, s); return;
      case SUBSTEP_B128_OCC8: launch_bs<FORM, 128, 8, true>(st, mesh, P, sub_off, integrate, next, use_cond, s); return;
      case SUBSTEP_B128_OCC5: launch_bs<FORM, 128, 5, true>(st, mesh, P, sub_off, integrate, next, use_cond, s); return;
      case SUBSTEP_B128_LOOP: launch_bs<FORM, 128, 6, false>(st, mesh, P, sub_off, integrate, next, use_cond, s); return;
      case SUBSTEP_B128_OCC8_LOOP: launch_bs<FORM, 128, 8, false>(st, mesh, P, sub_off, integrate, next, use_cond, s); return;
      case SUBSTEP_B64_LOOP: launch_bs<FORM, 64, 12, false>(st, mesh, P, sub_off, integrate, next, use_cond, s); return;
      case SUBSTEP_PAIRS:
      case SUBSTEP_PAIRS_ORDERED:
        // the force export (not integrating) runs the per-particle loop
        if (st.pairs && integrate)
          launch_pairs<FORM>(st, mesh, P, sub_off, variant == SUBSTEP_PAIRS_ORDERED, next, use_cond, s);
        else
          launch_bs<FORM, 128, 6, false>(st, mesh, P, sub_off, integrate, next, use_cond, s);
        return;
      default: launch_bs<FORM, 128, 6, true>(st, mesh, P, sub_off, integrate, next, use_cond, s); return;
    }
  } else {
    launch_bs<FORM, 128, 6, false>(st, mesh, P, sub_off, integrate, next, use_cond, s);
  }
}

void launch_substep(int form, const DevState& st, const DevMesh& mesh, const DevParams& P,
                    int sub_off, bool integrate, int variant, unsigned long long next_cond,
                    int use_cond, cudaStream_t s) {
  if (st.N <= 0) return;
  switch (form) {
    case FORM_SPLIT:
      launch_one<FORM_SPLIT>(st, mesh, P, sub_off, integrate, variant, next_cond, use_cond, s);
      break;
    case FORM_PLAIN:
      launch_one<FORM_PLAIN>(st, mesh, P, sub_off, integrate, variant, next_cond, use_cond, s);
      break;
    default:
      launch_one<FORM_FP64>(st, mesh, P, sub_off, integrate, variant, next_cond, use_cond, s);
      break;
  }
}


// Bounded grid barrier of the persistent ensemble launch (co-residency guaranteed by
// the cooperative launch): a waiting block gives up after spin_limit polls, records
// SEDI_ETIMEOUT and returns; the others see the record and return at their next wait.
__device__ bool ens_grid_barrier(Ctl* ctl, unsigned nblocks, long long spin_limit) {
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
        if (++spins > spin_limit) {
          atomicCAS(&ctl->error, 0, (int)SEDI_ETIMEOUT);
          break;
        }
        if ((spins & 1023) == 0 && *((volatile int*)&ctl->error) == (int)SEDI_ETIMEOUT) break;
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *((volatile int*)&ctl->error) != (int)SEDI_ETIMEOUT;
}

__global__ void k_ens_bar_reset(Ctl* ctl) {
  ctl->bar_count = 0u;
  ctl->bar_gen = 0u;
  ctl->error = 0;
  ctl->ens_rebuild = 0;
}

// Persistent ensemble launch: substeps s0 .. n-1 of every bed in one cooperative launch
// (every block resident).  The (bed, block) items of a substep are spread over the CTAs
// -- each item runs the same body, with the same arguments, as the batched launch's
// block (bed, blk) -- and a bounded grid barrier separates substeps.  The launch stops
// after the first substep that leaves a bed needing a list rebuild (the host rebuilds
// and launches again from the next substep).  *done receives the substeps completed
// (-1 when a barrier wait ran out).
template <int FORM, int BS, int MINB, bool COOP>
__global__ void __launch_bounds__(BS, MINB) k_substeps_persist_e(const BedView* v, int nbeds, Ctl* ectl,
                                                                   int s0, int n, int maxblk,
                                                                   long long spin_limit, int* done) {
  __shared__ BedView s_view;
  __shared__ int s_stop;
  const int64_t items = (int64_t)nbeds * maxblk;
  int s = s0;
  bool ok = true;
  while (s < n) {
    for (int64_t t = blockIdx.x; t < items; t += gridDim.x) {
      const int bed = (int)(t / maxblk), blk = (int)(t % maxblk);
      const int64_t N = v[bed].st.N;
      const unsigned nblk = (unsigned)((N + BS - 1) / BS);
      if ((unsigned)blk >= nblk) continue;  // the same for the whole CTA
      __syncthreads();                      // the previous item's readers of s_view are done
      const int4* src = reinterpret_cast<const int4*>(v + bed);
      int4* dst = reinterpret_cast<int4*>(&s_view);
      for (int k = threadIdx.x; k < (int)(sizeof(BedView) / 16); k += blockDim.x) dst[k] = src[k];
      __syncthreads();
      substep_body<FORM, true, BS, COOP, false>(s_view.st, s_view.mesh, s_view.P, s, 0ull, 0, blk, nblk,
                                                ectl, nbeds);
    }
    if (!ens_grid_barrier(ectl, gridDim.x, spin_limit)) {
      ok = false;
      break;
    }
    ++s;
    // the last bed of the substep left the any-bed rebuild decision
    if (threadIdx.x == 0) s_stop = *((volatile int*)&ectl->ens_rebuild);
    __syncthreads();
    if (s_stop) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *done = ok ? s : -1;
}

template <int FORM, int BS, int MINB, bool COOP>
static int launch_persist_shape(const EnsLaunch& e, int s0, int n, long long spin_limit, int* done,
                                cudaStream_t s) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_substeps_persist_e<FORM, BS, MINB, COOP>, BS, 0) !=
          cudaSuccess || per_sm < 1)
    return -1;
  int maxblk = (int)((e.max_n + BS - 1) / BS);
  int64_t G = (int64_t)nsm * per_sm;
  if (G > (int64_t)e.B * maxblk) G = (int64_t)e.B * maxblk;
  if (G < 1) G = 1;
  k_ens_bar_reset<<<1, 1, 0, s>>>(e.ectl);
  const BedView* views = e.views;
  int B = e.B;
  Ctl* ectl = e.ectl;
  void* args[] = {(void*)&views, (void*)&B, (void*)&ectl, (void*)&s0, (void*)&n, (void*)&maxblk,
                  (void*)&spin_limit, (void*)&done};
  return cudaLaunchCooperativeKernel((const void*)k_substeps_persist_e<FORM, BS, MINB, COOP>, dim3((unsigned)G),
                                     dim3(BS), args, 0, s) == cudaSuccess ? 0 : -1;
}

template <int FORM>
static int launch_persist(const EnsLaunch& e, int s0, int n, long long spin_limit, int* done, cudaStream_t s) {
  if constexpr (FORM != FORM_FP64) {
    switch (e.variant) {
      case SUBSTEP_B64_LOOP: return launch_persist_shape<FORM, 64, 12, false>(e, s0, n, spin_limit, done, s);
      case SUBSTEP_B128_OCC8_LOOP: return launch_persist_shape<FORM, 128, 8, false>(e, s0, n, spin_limit, done, s);
      case SUBSTEP_B128: return launch_persist_shape<FORM, 128, 6, true>(e, s0, n, spin_limit, done, s);
      default: break;
    }
  }
  return launch_persist_shape<FORM, 128, 6, false>(e, s0, n, spin_limit, done, s);
}

template <int FORM, int BS, int MINB, bool COOP, bool EXT>
static void launch_ens_shape(const EnsLaunch& e, int sub_off, unsigned long long next_cond, int use_cond,
                             cudaStream_t s) {
  const dim3 grid((unsigned)((e.max_n + BS - 1) / BS), (unsigned)e.B);
  const cudaGraphConditionalHandle h = (cudaGraphConditionalHandle)next_cond;
  k_substep_e<FORM, BS, MINB, COOP, EXT><<<grid, BS, 0, s>>>(e.views, e.B, e.ectl, sub_off, h, use_cond);
}

template <int FORM>
static void launch_ens(const EnsLaunch& e, bool ext, int sub_off, unsigned long long next_cond, int use_cond,
                       cudaStream_t s) {
  // the optional terms and the parity form: the per-particle loop at 128 x 6
  if (ext) {
    launch_ens_shape<FORM, 128, 6, false, true>(e, sub_off, next_cond, use_cond, s);
    return;
  }
  if constexpr (FORM != FORM_FP64) {
    switch (e.variant) {
      case SUBSTEP_B64_LOOP: launch_ens_shape<FORM, 64, 12, false, false>(e, sub_off, next_cond, use_cond, s); return;
      case SUBSTEP_B128_OCC8_LOOP: launch_ens_shape<FORM, 128, 8, false, false>(e, sub_off, next_cond, use_cond, s); return;
      case SUBSTEP_B128: launch_ens_shape<FORM, 128, 6, true, false>(e, sub_off, next_cond, use_cond, s); return;
      default: break;
    }
  }
  launch_ens_shape<FORM, 128, 6, false, false>(e, sub_off, next_cond, use_cond, s);
}

int launch_substeps_persist_ens(int form, const EnsLaunch& e, int s0, int n, long long spin_limit, int* done,
                                cudaStream_t s) {
  switch (form) {
    case FORM_SPLIT: return launch_persist<FORM_SPLIT>(e, s0, n, spin_limit, done, s);
    case FORM_PLAIN: return launch_persist<FORM_PLAIN>(e, s0, n, spin_limit, done, s);
    default: return launch_persist<FORM_FP64>(e, s0, n, spin_limit, done, s);
  }
}

void launch_substep_ens(int form, const EnsLaunch& e, bool ext, int sub_off,
                        unsigned long long next_cond, int use_cond, cudaStream_t s) {
  switch (form) {
    case FORM_SPLIT: launch_ens<FORM_SPLIT>(e, ext, sub_off, next_cond, use_cond, s); break;
    case FORM_PLAIN: launch_ens<FORM_PLAIN>(e, ext, sub_off, next_cond, use_cond, s); break;
    default: launch_ens<FORM_FP64>(e, ext, sub_off, next_cond, use_cond, s); break;
  }
}

}  // namespace sedi
