// Diffusion smoothing of the averaged fields (Sec. 2.4, Eq. 10): n_tau implicit
// pseudo-steps A x = b of the 7-point finite-volume Laplacian L (zero flux through
// non-periodic faces), each solved to ||b - A x|| <= rtol ||b|| for every field of
// every mesh of a batch, in ONE persistent launch.  Backward Euler:
// A = I - dtau D L, b = x^m.  BDF2 (the paper's second-order implicit scheme, read
// as the two-step backward difference): A = I - (2/3) dtau D L,
// b = (4/3) x^m - (1/3) x^{m-1} = x^m + (x^m - x^{m-1}) / 3, its first step backward
// Euler; x^{m-1} is kept in the wide word.
//
// Solver: Chebyshev semi-iteration on the known spectrum of A (lambda_min = 1 from
// the constant mode, lambda_max <= 1 + 4 sum_a coef_a by Gershgorin), organised as
// iterative refinement:
//   round:  r = b - A x in the wide word (df64 in the split form), kept as a narrow
//           copy, with the sums |r|^2, sum r (and |b|^2 in the first round)
//           reduced per work unit;
//           the constant shift s = sum(r) / C restores sum(x) = sum(b) (1^T A = 1^T,
//           so A 1 = 1 and the shifted residual has |r - s|^2 = |r|^2 - (sum r)^2/C);
//           if |r - s| <= rtol |b| the field is done, otherwise k Chebyshev steps
//           follow, k fixed up front from |r_k| <= 2 sigma^k |r_0|,
//           sigma = (sqrt(kappa) - 1) / (sqrt(kappa) + 1);
//   steps:  d_0 = (r - s) / theta;  x += d;  q -= A d;  d = c1 d + c2 q
//           with the direction d and the recursive residual q in the narrow word
//           (FP32 in the split form, the 8 fields of a cell interleaved so they load
//           as two 16-byte vectors) and x accumulated in the wide word;
//           rho' = 1 / (2 theta/delta - rho), c1 = rho' rho, c2 = 2 rho'/delta.
// A round that ends with the narrow recursion's rounding floor above the tolerance
// is followed by another round from the true residual, so every field finishes
// with a true df64 residual below rtol and sum(x) = sum(b) to df64 rounding.  The
// narrow steps do about a sixth of the work of df64 steps.
//
// Work units: 256 consecutive cells of one mesh (one per thread).  Every reduction
// is a per-unit partial sum followed by a per-mesh sum over its units in unit
// order, so a mesh's result does not depend on the grid size or on the other
// meshes of the batch: a batch of beds gives the same bits as each bed alone.
// The grid barrier spins at most ~0.3 s, then records SEDI_ETIMEOUT and returns;
// the other blocks see the record and return at their next barrier.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/sedi.h"
#include "common.cuh"
#include "kernels.h"

namespace sedi {

namespace {

constexpr int kThreads = kSmoothUnitCells;  // threads per block = cells per work unit
constexpr int kMaxF = kSmoothMaxFields;
constexpr int kQ = kSmoothSums;  // per-unit sums: |r|^2, sum r, |b|^2, sum w r (graded mesh)
constexpr int kMaxRounds = 64;

// ---------------------------------------------------------------- words
// T: wide word (x, b, r); N: narrow word (d, q); Acc: unit sums.
template <class T>
struct Wide;
template <>
struct Wide<dd> {
  using N = float;
  using Acc = float;
  static constexpr double kFloor = 1.0e-6;  // reduction one narrow round can reach
  __device__ static dd zero() { return dd{0.0f, 0.0f}; }
  __device__ static dd from_d(double a) { return dd_from_double(a); }
  __device__ static float narrow(dd a) { return __fadd_rn(a.hi, a.lo); }
  __device__ static dd add(dd a, dd b) { return dd_add(a, b); }
  __device__ static dd addq(dd a, dd b) { return dd_add_fast(a, b); }
  __device__ static dd subq(dd a, dd b) { return dd_sub_fast(a, b); }
  __device__ static dd mul(dd a, dd b) { return dd_mul(a, b); }
  __device__ static dd add_n(dd a, float b) { return dd_add_f(a, b); }
  __device__ static dd ld(const dd* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return dd{v.x, v.y};
  }
};
template <>
struct Wide<float> {
  using N = float;
  using Acc = float;
  static constexpr double kFloor = 1.0e-6;
  __device__ static float zero() { return 0.0f; }
  __device__ static float from_d(double a) { return __double2float_rn(a); }
  __device__ static float narrow(float a) { return a; }
  __device__ static float add(float a, float b) { return a + b; }
  __device__ static float addq(float a, float b) { return a + b; }
  __device__ static float subq(float a, float b) { return a - b; }
  __device__ static float mul(float a, float b) { return a * b; }
  __device__ static float add_n(float a, float b) { return a + b; }
  __device__ static float ld(const float* p) { return __ldcg(p); }
};
template <>
struct Wide<double> {
  using N = double;
  using Acc = double;
  static constexpr double kFloor = 0.0;
  __device__ static double zero() { return 0.0; }
  __device__ static double from_d(double a) { return a; }
  __device__ static double narrow(double a) { return a; }
  __device__ static double add(double a, double b) { return a + b; }
  __device__ static double addq(double a, double b) { return a + b; }
  __device__ static double subq(double a, double b) { return a - b; }
  __device__ static double mul(double a, double b) { return a * b; }
  __device__ static double add_n(double a, double b) { return a + b; }
  __device__ static double ld(const double* p) { return __ldcg(p); }
};

// The operator coefficients in the wide and the narrow word (converted on the host,
// so the kernels run no FP64 conversion per cell).
template <class T>
__device__ __forceinline__ T coef_w(const SmoothSpec& sp, int a);
template <>
__device__ __forceinline__ dd coef_w<dd>(const SmoothSpec& sp, int a) {
  return dd{sp.coef_hi[a], sp.coef_lo[a]};
}
template <>
__device__ __forceinline__ float coef_w<float>(const SmoothSpec& sp, int a) {
  return sp.coef_hi[a];
}
template <>
__device__ __forceinline__ double coef_w<double>(const SmoothSpec& sp, int a) {
  return sp.coef[a];
}

// Loads of words written by other blocks of the same launch go to L2 (ld.cg), so
// no stale L1 line is read after a grid barrier.
__device__ __forceinline__ int ldi(const int* p) { return __ldcg(p); }
__device__ __forceinline__ double ldd(const double* p) { return __ldcg(p); }

// Bounded grid barrier (co-residency guaranteed by the cooperative launch).
__device__ bool grid_barrier(Ctl* ctl, unsigned nblocks, long long spin_limit) {
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
        if (++spins > spin_limit) {  // ~0.3 s at the default kBarrierSpins
          atomicCAS((int*)&ctl->cg_status, 0, SEDI_ETIMEOUT);
          break;
        }
        // another block gave up: stop waiting too
        if ((spins & 1023) == 0 && *((volatile int*)&ctl->cg_status) == SEDI_ETIMEOUT) break;
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *((volatile int*)&ctl->cg_status) != SEDI_ETIMEOUT;
}

// Cell coordinates -> the six face neighbours (-1: zero-flux face).
struct Stencil {
  int32_t nb[6];
};

// n / d for 32-bit n from M = ceil(2^64 / d) (M = 0 for d = 1): floor(n M / 2^64) is
// exact, the excess n (M - 2^64/d) / 2^64 < 2^-32 <= 1/d.
__device__ __forceinline__ uint32_t div_magic(uint32_t n, uint64_t M) {
  return M ? (uint32_t)__umul64hi((uint64_t)n, M) : n;
}

__device__ __forceinline__ Stencil stencil_of(const SmoothMeshDev& m, int64_t c) {
  const uint32_t nx = m.nc[0], ny = m.nc[1], nz = m.nc[2];
  const uint32_t cc = (uint32_t)c;
  const uint32_t t = div_magic(cc, m.div_x);
  const uint32_t iz = div_magic(cc, m.div_xy);
  const uint32_t ix = cc - t * nx;
  const uint32_t iy = t - iz * ny;
  const uint32_t idx[3] = {ix, iy, iz};
  const uint32_t n[3] = {nx, ny, nz};
  const int32_t stride[3] = {1, (int32_t)nx, (int32_t)(nx * ny)};
  Stencil s;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int32_t base = (int32_t)cc - (int32_t)idx[ax] * stride[ax];
    if (idx[ax] > 0) s.nb[2 * ax] = (int32_t)cc - stride[ax];
    else s.nb[2 * ax] = m.per[ax] ? base + (int32_t)(n[ax] - 1) * stride[ax] : -1;
    if (idx[ax] + 1 < n[ax]) s.nb[2 * ax + 1] = (int32_t)cc + stride[ax];
    else s.nb[2 * ax + 1] = m.per[ax] ? base : -1;
  }
  return s;
}

// (A v)(c) = v_c - sum_axes coef_a ((v_- - v_c) + (v_+ - v_c)), faces that exist only.
// V is the word of the operand, get(k) loads (or forms) its value at cell k.
template <class V, class Sub, class Add, class Mul, class Get>
__device__ __forceinline__ V apply_A(const Stencil& st, const V* cf, V vc, Sub sub, Add add,
                                     Mul mul, Get get) {
  V lap{};
  bool any_axis = false;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    V sa{};
    bool any = false;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int32_t nb = st.nb[2 * ax + side];
      if (nb < 0) continue;
      const V t = sub(get(nb), vc);
      sa = any ? add(sa, t) : t;
      any = true;
    }
    if (any) {
      const V t = mul(cf[ax], sa);
      lap = any_axis ? add(lap, t) : t;
      any_axis = true;
    }
  }
  return any_axis ? sub(vc, lap) : vc;
}

// Graded z mesh: as apply_A, the z faces with their own coefficients (cz_m towards
// the plane below, cz_p towards the plane above).
template <class V, class Sub, class Add, class Mul, class Get>
__device__ __forceinline__ V apply_A_graded(const Stencil& st, const V* cf, V czm, V czp, V vc,
                                            Sub sub, Add add, Mul mul, Get get) {
  V lap{};
  bool any_axis = false;
#pragma unroll
  for (int ax = 0; ax < 2; ++ax) {
    V sa{};
    bool any = false;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int32_t nb = st.nb[2 * ax + side];
      if (nb < 0) continue;
      const V t = sub(get(nb), vc);
      sa = any ? add(sa, t) : t;
      any = true;
    }
    if (any) {
      const V t = mul(cf[ax], sa);
      lap = any_axis ? add(lap, t) : t;
      any_axis = true;
    }
  }
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int32_t nb = st.nb[4 + side];
    if (nb < 0) continue;
    const V t = mul(side ? czp : czm, sub(get(nb), vc));
    lap = any_axis ? add(lap, t) : t;
    any_axis = true;
  }
  return any_axis ? sub(vc, lap) : vc;
}

// Eight narrow words of one cell (the fields of the narrow recursion are stored
// interleaved, [C][8], so one cell's fields load as two 16-byte vectors).
template <class N>
struct V8 {
  N v[8];
};
__device__ __forceinline__ V8<float> ld8(const float* p) {
  const float4 a = __ldcg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldcg(reinterpret_cast<const float4*>(p) + 1);
  return V8<float>{{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w}};
}
__device__ __forceinline__ void st8(float* p, const V8<float>& x) {
  reinterpret_cast<float4*>(p)[0] = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
  reinterpret_cast<float4*>(p)[1] = make_float4(x.v[4], x.v[5], x.v[6], x.v[7]);
}
__device__ __forceinline__ V8<double> ld8(const double* p) {
  V8<double> r;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 a = __ldcg(reinterpret_cast<const double2*>(p) + k);
    r.v[2 * k] = a.x;
    r.v[2 * k + 1] = a.y;
  }
  return r;
}
__device__ __forceinline__ void st8(double* p, const V8<double>& x) {
#pragma unroll
  for (int k = 0; k < 4; ++k) reinterpret_cast<double2*>(p)[k] = make_double2(x.v[2 * k], x.v[2 * k + 1]);
}

// Per-mesh solver state published by the owner block of each mesh.
struct alignas(16) MeshState {
  int32_t k[kMaxF];      // Chebyshev steps of the current round per field (0: none)
  int32_t done[kMaxF];   // converged, zero or stopped
  int32_t zero[kMaxF];   // b == 0: x = 0
  int32_t total[kMaxF];  // steps taken in this pseudo-step
  double shift[kMaxF];   // projection shift of the current round
  double bb[kMaxF];      // |b|^2
};

// Per-block reduction of the kQ sums of nf fields for one unit (fixed order).  The
// warp stage is a butterfly reduce-scatter of the 32 (field, sum) slots: at each of
// five rounds a lane keeps half of its slots and adds its partner's copy of them, so
// lane l ends with the warp's sum of slot l after 31 additions (a plain shuffle
// reduction of every slot would take 5 x 32; the FP64 pipe is the narrow one).
template <class Acc>
__device__ __forceinline__ void unit_sums(const Acc (&v)[kMaxF][kQ], int nf, double* out) {
  static_assert(kMaxF * kQ == 32, "one slot per lane");
  __shared__ Acc red[kThreads / 32][kMaxF * kQ];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Acc a[32];
#pragma unroll
  for (int f = 0; f < kMaxF; ++f)
#pragma unroll
    for (int q = 0; q < kQ; ++q) a[f * kQ + q] = v[f][q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < o; ++k) {
      const Acc mine = up ? a[k + o] : a[k];
      const Acc give = up ? a[k] : a[k + o];
      a[k] = mine + __shfl_xor_sync(0xffffffffu, give, o);
    }
  }
  red[wid][lane] = a[0];
  __syncthreads();
  if (threadIdx.x < nf * kQ) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += (double)red[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Right-hand side of pseudo-step m from x^m (xv): x^m itself (backward Euler, and
// the first BDF2 step), or x^m + (x^m - x^{m-1}) / 3 with x^{m-1} read from *xp.
// BDF2 also stores x^m in *xp for the next step.
template <class T>
__device__ __forceinline__ T rhs_of(int scheme, int m, T xv, T* xp) {
  using W = Wide<T>;
  if (scheme != TAU_BDF2) return xv;
  T bv = xv;
  if (m > 0) bv = W::add(xv, W::mul(W::from_d(1.0 / 3.0), W::subq(xv, W::ld(xp))));
  *xp = xv;
  return bv;
}

// Resident blocks per SM of the grid solver: 3 for the double-float and FP32 words (80
// registers, no spills; 17% faster than 2 on a 2M-cell mesh), 2 for FP64 (which would
// spill at 80).
template <class T>
constexpr int smooth_blocks_per_sm() {
  return sizeof(T) == 8 && !std::is_same<T, dd>::value ? 2 : 3;
}

// GR: graded z mesh (per-plane z coefficients, volume-weighted projection shift).
template <class T, bool GR>
__global__ void __launch_bounds__(kThreads, smooth_blocks_per_sm<T>()) k_smooth(SmoothBatchDev a) {
  using W = Wide<T>;
  using N = typename W::N;
  using Acc = typename W::Acc;
  const unsigned G = gridDim.x;
  const int nf = a.nf;
  const int64_t U = a.U;
  const int64_t u_begin = (int64_t)blockIdx.x * U / G, u_end = (int64_t)(blockIdx.x + 1) * U / G;
  MeshState* ms = (MeshState*)a.pairs;
  __shared__ double s_sums[(kThreads / 32) * kQ];
  __shared__ int s_K;
  // the mesh of the units being walked and its solver state for the current pass, in
  // shared memory (every thread of a block walks the same units, so a change of mesh is
  // seen by the whole block at once)
  static_assert(sizeof(SmoothMeshDev) % 16 == 0, "mesh entries are copied as 16-byte words");
  __shared__ SmoothMeshDev s_md;
  __shared__ int s_kf[kMaxF], s_zero[kMaxF], s_done[kMaxF];
  __shared__ double s_shd[kMaxF];
  auto load_mesh = [&](int bi) {
    __syncthreads();
    const int4* src = reinterpret_cast<const int4*>(a.mesh + bi);
    int4* dst = reinterpret_cast<int4*>(&s_md);
    for (int q = threadIdx.x; q < (int)(sizeof(SmoothMeshDev) / 16); q += blockDim.x) dst[q] = src[q];
    if (threadIdx.x < kMaxF) {
      const int f = threadIdx.x;
      const MeshState& st = ms[bi];
      s_kf[f] = f < nf ? ldi(&st.k[f]) : 0;
      s_zero[f] = f < nf ? ldi(&st.zero[f]) : 0;
      s_done[f] = f < nf ? ldi(&st.done[f]) : 1;
      s_shd[f] = f < nf ? ldd(&st.shift[f]) : 0.0;
    }
    __syncthreads();
  };
  int slot = 0;

  for (int m = 0; m < a.n_tau; ++m) {
    const bool use_guess = (m == 0);
    const int ph = (a.scheme == TAU_BDF2 && m > 0) ? 1 : 0;  // operator of this step
    // ---- b from the previous pseudo-step's result; x = guess on the first
    for (int64_t u = u_begin; u < u_end; ++u) {
      const SmoothMeshDev& md = a.mesh[a.unit_bed[u]];
      const int64_t c = (u - md.u0) * kThreads + threadIdx.x;
      if (c >= md.C) continue;
      for (int f = 0; f < nf; ++f) {
        const int64_t k = f * md.C + c;
        const T xv = W::ld((const T*)md.x + k);
        ((T*)md.b)[k] = rhs_of<T>(a.scheme, m, xv, (T*)md.xp + (md.xp ? k : 0));
        if (use_guess && md.guess) ((T*)md.x)[k] = W::ld((const T*)md.guess + k);
      }
    }
    if (!grid_barrier(a.ctl, G, a.spin_limit)) return;
    for (int round = 0; round < kMaxRounds; ++round) {
      // ---- true residual r = b - A x (wide), its narrow copy (interleaved, in d[0])
      //      and the unit sums |r|^2, sum r, |b|^2
      int cur_bi = -1;
      for (int64_t u = u_begin; u < u_end; ++u) {
        const int bi = a.unit_bed[u];
        if (bi != cur_bi) {
          load_mesh(bi);
          cur_bi = bi;
        }
        const SmoothMeshDev& md = s_md;
        const int64_t c = (u - md.u0) * kThreads + threadIdx.x;
        const bool in = c < md.C;
        Acc v[kMaxF][kQ];
        V8<N> rn;
        const SmoothSpec& sp = md.sp[ph];
        const T cf[3] = {coef_w<T>(sp, 0), coef_w<T>(sp, 1), coef_w<T>(sp, 2)};
        const Stencil sc = stencil_of(md, in ? c : 0);
        T czm{}, czp{};
        Acc wz = Acc(1);
        if constexpr (GR) {
          const int kz = (int)div_magic((uint32_t)(in ? c : 0), md.div_xy);
          czm = W::from_d(md.z.cz[ph][2 * kz]);
          czp = W::from_d(md.z.cz[ph][2 * kz + 1]);
          wz = (Acc)md.z.w[kz];
        }
#pragma unroll
        for (int f = 0; f < kMaxF; ++f) {
          v[f][0] = v[f][1] = v[f][2] = v[f][3] = Acc(0);
          rn.v[f] = N(0);
          if (f >= nf || !in || (round > 0 && s_done[f])) continue;
          const T* X = (const T*)md.x + f * md.C;
          const T xc = W::ld(X + c);
          auto subq = [](T p, T q) { return W::subq(p, q); };
          auto addq = [](T p, T q) { return W::addq(p, q); };
          auto mul = [](T p, T q) { return W::mul(p, q); };
          auto get = [&](int32_t k) { return W::ld(X + k); };
          T ax;
          if constexpr (GR) ax = apply_A_graded<T>(sc, cf, czm, czp, xc, subq, addq, mul, get);
          else ax = apply_A<T>(sc, cf, xc, subq, addq, mul, get);
          const T bv = W::ld((const T*)md.b + f * md.C + c);
          const T rv = W::subq(bv, ax);
          const N r_n = W::narrow(rv);
          rn.v[f] = r_n;
          v[f][0] = (Acc)r_n * (Acc)r_n;
          v[f][1] = (Acc)r_n;
          if constexpr (GR) v[f][3] = wz * (Acc)r_n;
          if (round == 0) {
            const Acc bn = (Acc)W::narrow(bv);
            v[f][2] = bn * bn;
          }
        }
        if (in) st8((N*)md.d[0] + c * kMaxF, rn);
        unit_sums<Acc>(v, nf, md.part + (u - md.u0) * (kMaxF * kQ));
      }
      if (!grid_barrier(a.ctl, G, a.spin_limit)) return;
      // ---- owners: one block per (mesh, field): the field's sums over the mesh's units
      //      (thread t adds units t, t + 256, ... in order, then a fixed tree: the same
      //      association whatever the grid or the batch), then its decisions
      for (int64_t it = blockIdx.x; it < (int64_t)a.B * nf; it += G) {
        const int bi = (int)(it / nf), f = (int)(it % nf);
        const SmoothMeshDev& md = a.mesh[bi];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        double sq[kQ] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t u = threadIdx.x; u < md.nu; u += kThreads) {
          const double* pu = md.part + u * (kMaxF * kQ) + f * kQ;
#pragma unroll
          for (int q = 0; q < kQ; ++q) sq[q] += ldd(pu + q);
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          double v = sq[q];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) s_sums[wid * kQ + q] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          double tot[kQ];
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            tot[q] = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) tot[q] += s_sums[w * kQ + q];
          }
          MeshState& st = ms[bi];
          int k = 0, done = 1, zero = 0, total = 0;
          double shift = 0.0, bb = 0.0;
          done = round == 0 ? 0 : st.done[f];
          zero = round == 0 ? 0 : st.zero[f];
          total = round == 0 ? 0 : st.total[f];
          bb = round == 0 ? tot[2] : st.bb[f];
          if (round == 0) zero = !(bb > 0.0);
          if (!done) {
            const double rr = tot[0], sr = tot[1];
            const double Cd = (double)md.C;
            if (zero) {
              done = 1;
            } else {
              double rrp;
              if (GR) {
                // the shift keeps sum(w x) = sum(w b); |r - s|^2 = |r|^2 - 2 s sum r + C s^2
                shift = tot[3] / md.z.wsum;
                rrp = fmax(rr - 2.0 * shift * sr + Cd * shift * shift, 0.0);
              } else {
                shift = sr / Cd;
                rrp = fmax(rr - sr * sr / Cd, 0.0);
              }
              if (rrp <= a.rtol2 * bb) {
                done = 1;
              } else {
                // |r_k| <= 2 sig^k |r_0|: enough steps for the tolerance, or for the
                // reduction the narrow word can deliver in one round
                const double need = fmax(0.5 * sqrt(a.rtol2 * bb / rrp), W::kFloor);
                const double sig = md.sp[ph].sig;
                k = sig > 0.0 ? (int)ceil(log(need) / log(sig)) : 1;
                if (k < 1) k = 1;
                if (k > kMaxStepsRound) k = kMaxStepsRound;
                if (total + k > a.max_iter) k = a.max_iter - total;
                if (k <= 0) {
                  k = 0;
                  done = 1;
                  atomicCAS((int*)&a.ctl->cg_status, 0, SEDI_EDIVERGED);
                } else {
                  total += k;
                }
              }
            }
            if (done && md.iters) atomicAdd(md.iters + f, total);
          }
          st.k[f] = k;
          st.done[f] = done;
          st.zero[f] = zero;
          st.total[f] = total;
          st.shift[f] = shift;
          st.bb[f] = bb;
          if (k > 0) atomicMax(a.gflag + slot, k);
        }
        __syncthreads();
      }
      // the slot of the next round was last read before the previous barrier
      if (blockIdx.x == 0 && threadIdx.x == 0) a.gflag[slot ^ 1] = 0;
      if (!grid_barrier(a.ctl, G, a.spin_limit)) return;
      if (threadIdx.x == 0) s_K = ldi(a.gflag + slot);
      __syncthreads();
      const int K = s_K;
      slot ^= 1;
      // ---- Chebyshev steps j = 1..K; step 1 also applies the shift (or zeroes x)
      const int J = K > 0 ? K : 1;
      for (int j = 1; j <= J; ++j) {
        int cur_bi = -1;
        for (int64_t u = u_begin; u < u_end; ++u) {
          const int bi = a.unit_bed[u];
          if (bi != cur_bi) {
            load_mesh(bi);
            cur_bi = bi;
          }
          const SmoothMeshDev& md = s_md;
          const int64_t c = (u - md.u0) * kThreads + threadIdx.x;
          if (c >= md.C) continue;
          int kf[kMaxF];
          N sh[kMaxF];
          bool any = false;
#pragma unroll
          for (int f = 0; f < kMaxF; ++f) sh[f] = N(0);
#pragma unroll
          for (int f = 0; f < kMaxF; ++f) {
            kf[f] = s_kf[f];
            any |= kf[f] >= j;
          }
          if (j == 1) {
            // projection shift (and zero fields) for every field, then the first step
            T* X = (T*)md.x;
#pragma unroll
            for (int f = 0; f < kMaxF; ++f) {
              if (f >= nf) continue;
              const double s = s_shd[f];
              sh[f] = (N)s;
              if (kf[f] == 0) {
                if (round == 0 && s_zero[f]) X[f * md.C + c] = W::zero();
                else if (s != 0.0) X[f * md.C + c] = W::add(W::ld(X + f * md.C + c), W::from_d(s));
              }
            }
          }
          if (!any) continue;
          const SmoothSpec& sp = md.sp[ph];
          const N cfn[3] = {coef_w<N>(sp, 0), coef_w<N>(sp, 1), coef_w<N>(sp, 2)};
          N c1, c2, inv_theta;
          if constexpr (sizeof(N) == 4) {
            c1 = sp.chebf[0][j - 1];
            c2 = sp.chebf[1][j - 1];
            inv_theta = sp.inv_theta_f;
          } else {
            c1 = (N)sp.cheb[0][j - 1];
            c2 = (N)sp.cheb[1][j - 1];
            inv_theta = (N)(1.0 / sp.theta);
          }
          const Stencil sc = stencil_of(md, c);
          // step 1 reads the narrow residual (d[0]) and forms d0 = (r - s) / theta at
          // every stencil point; later steps read the previous direction
          const N* Dold = (const N*)md.d[(j - 1) & 1];
          N* Dnew = (N*)md.d[j & 1];
          N* Q = (N*)md.q;
          auto dir = [&](const V8<N>& raw) {
            V8<N> d = raw;
            if (j == 1) {
#pragma unroll
              for (int f = 0; f < kMaxF; ++f) d.v[f] = (raw.v[f] - sh[f]) * inv_theta;
            }
            return d;
          };
          const V8<N> dc = dir(ld8(Dold + c * kMaxF));
          V8<N> lap;
          bool any_axis = false;
          N czn[2] = {N(0), N(0)};
          if constexpr (GR) {
            const int kz = (int)div_magic((uint32_t)c, md.div_xy);
            if constexpr (sizeof(N) == 4) {
              czn[0] = md.z.czf[ph][2 * kz];
              czn[1] = md.z.czf[ph][2 * kz + 1];
            } else {
              czn[0] = (N)md.z.cz[ph][2 * kz];
              czn[1] = (N)md.z.cz[ph][2 * kz + 1];
            }
          }
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) {
            if (GR && ax == 2) {
              // graded z: each face with its own coefficient
#pragma unroll
              for (int side = 0; side < 2; ++side) {
                const int32_t nb = sc.nb[4 + side];
                if (nb < 0) continue;
                const V8<N> dn = dir(ld8(Dold + (int64_t)nb * kMaxF));
#pragma unroll
                for (int f = 0; f < kMaxF; ++f) {
                  const N t = czn[side] * (dn.v[f] - dc.v[f]);
                  lap.v[f] = any_axis ? lap.v[f] + t : t;
                }
                any_axis = true;
              }
              continue;
            }
            V8<N> sa;
            bool any_side = false;
#pragma unroll
            for (int side = 0; side < 2; ++side) {
              const int32_t nb = sc.nb[2 * ax + side];
              if (nb < 0) continue;
              const V8<N> dn = dir(ld8(Dold + (int64_t)nb * kMaxF));
#pragma unroll
              for (int f = 0; f < kMaxF; ++f) {
                const N t = dn.v[f] - dc.v[f];
                sa.v[f] = any_side ? sa.v[f] + t : t;
              }
              any_side = true;
            }
            if (any_side) {
#pragma unroll
              for (int f = 0; f < kMaxF; ++f) {
                const N t = cfn[ax] * sa.v[f];
                lap.v[f] = any_axis ? lap.v[f] + t : t;
              }
              any_axis = true;
            }
          }
          // q: the narrow residual r - s (step 1) or the recursive residual
          V8<N> q = j == 1 ? ld8(Dold + c * kMaxF) : ld8(Q + c * kMaxF);
          V8<N> dn;
          T* X = (T*)md.x;
#pragma unroll
          for (int f = 0; f < kMaxF; ++f) {
            dn.v[f] = N(0);
            if (kf[f] < j) continue;
            const N ad = any_axis ? dc.v[f] - lap.v[f] : dc.v[f];
            const int64_t k = f * md.C + c;
            T xv = W::ld(X + k);
            if (j == 1) {
              xv = W::add(xv, W::from_d(s_shd[f]));  // projection shift
              q.v[f] = q.v[f] - sh[f];                         // narrow r - s
            }
            q.v[f] = q.v[f] - ad;
            dn.v[f] = c1 * dc.v[f] + c2 * q.v[f];
            X[k] = W::add_n(xv, dc.v[f]);
          }
          st8(Q + c * kMaxF, q);
          st8(Dnew + c * kMaxF, dn);
        }
        if (!grid_barrier(a.ctl, G, a.spin_limit)) return;
      }
      if (K == 0) break;
    }
  }
}

// ---------------------------------------------------------------- cluster solver
// Meshes whose z-planes fit 8192 cells per CTA on at most 16 CTAs (split and plain
// forms): a thread-block cluster solves one (mesh, field) pair at a time.  CTA r
// holds whole z-planes [r P, (r + 1) P) of the field and its narrow recursion in
// shared memory (x in the wide word, the narrow residual and two directions), so a
// step touches no global memory; the z-neighbours of a CTA's first and last plane
// are read from the adjacent CTAs through distributed shared memory.  Pairs are
// independent, so there is no grid-wide barrier: each step ends with the hardware
// cluster barrier and each field runs its own step count.  Same iteration as the
// grid solver (rounds of a wide true residual, then narrow Chebyshev steps); the
// sums of a round are reduced per CTA, then over the CTAs in rank order.  The
// cluster shape is a function of the mesh alone, so a bed smooths the same way in
// any batch.
namespace cg = cooperative_groups;
constexpr int kClThreads = 1024;
constexpr int kClCells = 8192;   // cells per CTA at most
constexpr size_t kClSmem = 212 * 1024;  // dynamic shared memory of a CTA at most: 20 B a cell
constexpr int kClMaxCta = 16;

// A stencil neighbour: index in the owning CTA's arrays, and that CTA (-1: this one).
struct Nb {
  int32_t l;
  int32_t r;
};

template <class T, bool GR>
__global__ void __launch_bounds__(kClThreads, 1) k_smooth_cl(SmoothBatchDev a) {
  using W = Wide<T>;
  using N = typename W::N;
  using Acc = typename W::Acc;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ double s_part[kClMaxCta][kQ];  // every CTA's sums, pushed by each CTA
  __shared__ double s_red[kClThreads / 32][kQ];
  __shared__ double s_shift;
  __shared__ int s_k, s_zero;
  cg::cluster_group cl = cg::this_cluster();
  const int csize = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int64_t ncl = gridDim.x / csize, cid = blockIdx.x / csize;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t items = (int64_t)a.B * a.nf;
  for (int64_t w = cid; w < items; w += ncl) {
    const int bi = (int)(w / a.nf), f = (int)(w % a.nf);
    const SmoothMeshDev& md = a.mesh[bi];
    const int64_t C = md.C;
    const int nx = md.nc[0], ny = md.nc[1], nz = md.nc[2], nxy = nx * ny;
    const int P = md.cl_planes;                                  // planes of a full CTA
    const int z0 = rank * P;
    const int planes = z0 + P <= nz ? P : nz - z0;               // this CTA's planes
    const int last_planes = nz - (csize - 1) * P;
    const int ncell = planes * nxy;
    const int64_t c0 = (int64_t)z0 * nxy;
    T* Xs = (T*)s_dyn;                      // [P nxy] x
    N* dA = (N*)(Xs + P * nxy);             // narrow true residual, then even directions
    N* dB = dA + P * nxy;                   // odd directions
    N* Qs = dB + P * nxy;                   // recursive residual

    T* Xg = (T*)md.x + f * C;
    T* Bg = (T*)md.b + f * C;
    T* XPg = md.xp ? (T*)md.xp + f * C : nullptr;
    // Work layout: thread t owns the (x, y) columns t, t + kClThreads, ... of the plane
    // and walks each column through this CTA's planes with a rolling window in z, so
    // the in-plane neighbours are fixed offsets per column and only the first and
    // last plane read a z-neighbour from another CTA (distributed shared memory,
    // both loaded before the walk).
    const bool pz = md.per[2] != 0;
    // z-neighbour below plane 0 / above the last plane of column s in array `arr`
    // (has = false: zero-flux face)
    auto z_below = [&](auto* arr, int s, bool& has) {
      using V = typename std::remove_const<typename std::remove_pointer<decltype(arr)>::type>::type;
      has = true;
      if (z0 > 0) return (V)cl.map_shared_rank(arr, (unsigned)(rank - 1))[(P - 1) * nxy + s];
      if (pz) {
        if (csize > 1) return (V)cl.map_shared_rank(arr, (unsigned)(csize - 1))[(last_planes - 1) * nxy + s];
        return (V)arr[(planes - 1) * nxy + s];
      }
      has = false;
      return V{};
    };
    auto z_above = [&](auto* arr, int s, bool& has) {
      using V = typename std::remove_const<typename std::remove_pointer<decltype(arr)>::type>::type;
      has = true;
      if (z0 + planes < nz) return (V)cl.map_shared_rank(arr, (unsigned)(rank + 1))[s];
      if (pz) {
        if (csize > 1) return (V)cl.map_shared_rank(arr, 0u)[s];
        return (V)arr[s];
      }
      has = false;
      return V{};
    };
    // in-plane neighbour offsets of column s (has[k] = false: zero-flux face)
    struct Col {
      int off[4];
      bool has[4];
    };
    auto col_of = [&](int sidx) {
      Col c;
      const int ix = sidx % nx, iy = sidx / nx;
      c.has[0] = ix > 0 || md.per[0];
      c.off[0] = ix > 0 ? -1 : nx - 1;
      c.has[1] = ix < nx - 1 || md.per[0];
      c.off[1] = ix < nx - 1 ? 1 : -(nx - 1);
      c.has[2] = iy > 0 || md.per[1];
      c.off[2] = iy > 0 ? -nx : (ny - 1) * nx;
      c.has[3] = iy < ny - 1 || md.per[1];
      c.off[3] = iy < ny - 1 ? nx : -(ny - 1) * nx;
      return c;
    };
    for (int m = 0; m < a.n_tau; ++m) {
      const int ph = (a.scheme == TAU_BDF2 && m > 0) ? 1 : 0;
      const SmoothSpec& sp = md.sp[ph];
      const T cf[3] = {coef_w<T>(sp, 0), coef_w<T>(sp, 1), coef_w<T>(sp, 2)};
      const N cfn[3] = {coef_w<N>(sp, 0), coef_w<N>(sp, 1), coef_w<N>(sp, 2)};
      N inv_theta;
      if constexpr (sizeof(N) == 4) inv_theta = sp.inv_theta_f;
      else inv_theta = (N)(1.0 / sp.theta);
      // ---- b (global) from the previous pseudo-step's result; x (or the guess)
      //      into shared memory
      for (int l = threadIdx.x; l < ncell; l += kClThreads) {
        const T xv = W::ld(Xg + c0 + l);
        Bg[c0 + l] = rhs_of<T>(a.scheme, m, xv, XPg ? XPg + c0 + l : nullptr);
        Xs[l] = (m == 0 && md.guess) ? W::ld((const T*)md.guess + f * C + c0 + l) : xv;
      }
      cl.sync();
      int total = 0, zero = 0;
      double bb = 0.0;
      for (int round = 0; round < kMaxRounds; ++round) {
        // ---- true residual (wide), its narrow copy in dA, sums
        Acc v[kQ] = {Acc(0), Acc(0), Acc(0), Acc(0)};
        // (A x)(c) = x_c - sum_a coef_a ((x_- - x_c) + (x_+ - x_c)), faces that exist
        auto wpair = [](bool h0, T v0, bool h1, T v1, T c) {
          if (h0 && h1) return W::addq(W::subq(v0, c), W::subq(v1, c));
          if (h0) return W::subq(v0, c);
          if (h1) return W::subq(v1, c);
          return W::zero();
        };
        for (int sidx = threadIdx.x; sidx < nxy; sidx += kClThreads) {
          const Col col = col_of(sidx);
          bool hb, hl;
          // both remote z-neighbours of the column are loaded before the walk
          T below = z_below(Xs, sidx, hb);
          const T top = z_above(Xs, sidx, hl);
          T cur = Xs[sidx];
          for (int izl = 0; izl < planes; ++izl) {
            const int l = izl * nxy + sidx;
            const bool ha = izl + 1 < planes || hl;
            const T above = izl + 1 < planes ? Xs[l + nxy] : top;
            const T sx = wpair(col.has[0], col.has[0] ? Xs[l + col.off[0]] : cur, col.has[1],
                               col.has[1] ? Xs[l + col.off[1]] : cur, cur);
            const T sy = wpair(col.has[2], col.has[2] ? Xs[l + col.off[2]] : cur, col.has[3],
                               col.has[3] ? Xs[l + col.off[3]] : cur, cur);
            T zt;
            if constexpr (GR) {
              // graded z: each face with its plane's own coefficient
              const double* cz = md.z.cz[ph] + 2 * (z0 + izl);
              zt = W::zero();
              if (hb) zt = W::mul(W::from_d(cz[0]), W::subq(below, cur));
              if (ha) zt = W::addq(zt, W::mul(W::from_d(cz[1]), W::subq(above, cur)));
            } else {
              zt = W::mul(cf[2], wpair(hb, below, ha, above, cur));
            }
            const T lap = W::addq(W::addq(W::mul(cf[0], sx), W::mul(cf[1], sy)), zt);
            const T ax = W::subq(cur, lap);
            const T bv = W::ld(Bg + c0 + l);
            const N rn = W::narrow(W::subq(bv, ax));
            dA[l] = rn;
            v[0] += (Acc)rn * (Acc)rn;
            v[1] += (Acc)rn;
            if constexpr (GR) v[3] += (Acc)md.z.w[z0 + izl] * (Acc)rn;
            if (round == 0) {
              const Acc bn = (Acc)W::narrow(bv);
              v[2] += bn * bn;
            }
            below = cur;
            hb = true;
            cur = above;
          }
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          // warp sums in the accumulation word (as the grid solver's units), the
          // CTA's sum of the 32 warp sums in FP64
          Acc t = v[q];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          if (lane == 0) s_red[wid][q] = (double)t;
        }
        __syncthreads();
        // this CTA's sums, pushed into every CTA's shared memory (stores do not wait)
        if (threadIdx.x < csize * kQ) {
          const int r = threadIdx.x / kQ, q = threadIdx.x % kQ;
          double t = 0.0;
          for (int k = 0; k < kClThreads / 32; ++k) t += s_red[k][q];
          cl.map_shared_rank(&s_part[0][0], (unsigned)r)[rank * kQ + q] = t;
        }
        cl.sync();
        // one thread of every CTA sums the parts in rank order and decides: every CTA
        // takes the same decision
        if (threadIdx.x == 0) {
          double tot[kQ] = {0.0, 0.0, 0.0, 0.0};
          for (int r = 0; r < csize; ++r)
#pragma unroll
            for (int q = 0; q < kQ; ++q) tot[q] += s_part[r][q];
          if (round == 0) {
            bb = tot[2];
            zero = !(bb > 0.0);
          }
          const double Cd = (double)C;
          double shift, rrp;
          if (GR) {
            // the shift keeps sum(w x) = sum(w b); |r - s|^2 = |r|^2 - 2 s sum r + C s^2
            shift = zero ? 0.0 : tot[3] / md.z.wsum;
            rrp = fmax(tot[0] - 2.0 * shift * tot[1] + Cd * shift * shift, 0.0);
          } else {
            shift = zero ? 0.0 : tot[1] / Cd;
            rrp = fmax(tot[0] - tot[1] * tot[1] / Cd, 0.0);
          }
          int k = 0;
          if (!zero && !(rrp <= a.rtol2 * bb)) {
            // the step count only has to be about right (the next round checks the true
            // residual), so it is formed in FP32
            const float need = fmaxf(0.5f * sqrtf((float)(a.rtol2 * bb / rrp)), (float)W::kFloor);
            k = sp.sig > 0.0 ? (int)ceilf(logf(need) / logf((float)sp.sig)) : 1;
            if (k < 1) k = 1;
            if (k > kMaxStepsRound) k = kMaxStepsRound;
            if (total + k > a.max_iter) k = a.max_iter - total;
            if (k <= 0) {
              k = 0;
              if (rank == 0) atomicCAS((int*)&a.ctl->cg_status, 0, SEDI_EDIVERGED);
            }
          }
          s_k = k;
          s_shift = shift;
          s_zero = zero;
        }
        __syncthreads();
        const int k = s_k;
        const double shift = s_shift;
        zero = s_zero;
        total += k;
        if (k == 0) {
          // converged (or zero, or stopped): apply the projection shift, write x back
          const T sw = W::from_d(shift);
          for (int l = threadIdx.x; l < ncell; l += kClThreads) {
            T xv = Xs[l];
            if (zero) xv = W::zero();
            else if (shift != 0.0) xv = W::add(xv, sw);
            Xg[c0 + l] = xv;
          }
          break;
        }
        const N shn = (N)shift;
        const T sw = W::from_d(shift);
        // ---- Chebyshev steps (step 1 applies the shift and forms d0 = (r - s) / theta)
        for (int j = 1; j <= k; ++j) {
          N* Dold = (j & 1) ? dA : dB;
          N* Dnew = (j & 1) ? dB : dA;
          N c1s, c2s;
          if constexpr (sizeof(N) == 4) {
            c1s = sp.chebf[0][j - 1];
            c2s = sp.chebf[1][j - 1];
          } else {
            c1s = (N)sp.cheb[0][j - 1];
            c2s = (N)sp.cheb[1][j - 1];
          }
          // One step over this CTA's columns.  FIRST (step 1) reads the narrow true
          // residual r and forms d0 = (r - s) / theta at every point it touches; x and
          // the recursion take the shift.  FULL: all four in-plane faces exist (the
          // common case), so the loop has no per-face selects.
          auto step = [&](auto first_tag, auto full_tag, int sidx, const Col& col) {
            constexpr bool FIRST = decltype(first_tag)::value;
            constexpr bool FULL = decltype(full_tag)::value;
            auto tr = [&](N raw) {
              if constexpr (FIRST) return (raw - shn) * inv_theta;
              else return raw;
            };
            auto face = [&](bool h, int l, int off, N cur) {
              if constexpr (FULL) return tr(Dold[l + off]) - cur;
              else return h ? tr(Dold[l + off]) - cur : N(0);
            };
            bool hb, hl;
            // both remote z-neighbours of the column are loaded before the walk
            N below = tr(z_below(Dold, sidx, hb));
            const N top = tr(z_above(Dold, sidx, hl));
            N cur = tr(Dold[sidx]);
            for (int izl = 0; izl < planes; ++izl) {
              const int l = izl * nxy + sidx;
              const bool up = izl + 1 < planes;
              const N above = up ? tr(Dold[l + nxy]) : top;
              const N sx = face(col.has[0], l, col.off[0], cur) + face(col.has[1], l, col.off[1], cur);
              const N sy = face(col.has[2], l, col.off[2], cur) + face(col.has[3], l, col.off[3], cur);
              N zt;
              if constexpr (GR) {
                const float* cz = md.z.czf[ph] + 2 * (z0 + izl);
                zt = (hb ? (N)cz[0] * (below - cur) : N(0)) + ((up || hl) ? (N)cz[1] * (above - cur) : N(0));
              } else {
                zt = cfn[2] * ((hb ? below - cur : N(0)) + ((up || hl) ? above - cur : N(0)));
              }
              const N ad = cur - ((cfn[0] * sx + cfn[1] * sy) + zt);
              T xv = Xs[l];
              N q;
              if constexpr (FIRST) {
                xv = W::add(xv, sw);
                q = Dold[l] - shn;
              } else {
                q = Qs[l];
              }
              q = q - ad;
              Qs[l] = q;
              Dnew[l] = c1s * cur + c2s * q;
              Xs[l] = W::add_n(xv, cur);
              below = cur;
              hb = true;
              cur = above;
            }
          };
          for (int sidx = threadIdx.x; sidx < nxy; sidx += kClThreads) {
            const Col col = col_of(sidx);
            const bool full = col.has[0] && col.has[1] && col.has[2] && col.has[3];
            if (j == 1) {
              if (full) step(std::true_type{}, std::true_type{}, sidx, col);
              else step(std::true_type{}, std::false_type{}, sidx, col);
            } else {
              if (full) step(std::false_type{}, std::true_type{}, sidx, col);
              else step(std::false_type{}, std::false_type{}, sidx, col);
            }
          }
          cl.sync();
        }
      }
      if (rank == 0 && threadIdx.x == 0 && md.iters) atomicAdd(md.iters + f, total);
    }
  }
}

__global__ void k_bar_reset(Ctl* ctl) {
  ctl->bar_count = 0u;
  ctl->bar_gen = 0u;
}

template <class T>
size_t word() {
  return sizeof(T);
}

template <class T, bool GR>
int launch_impl(const SmoothBatchDev& a, int max_blocks, cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smooth<T, GR>, kThreads, 0);
  if (per_sm < 1) return -3;
  if (per_sm > smooth_blocks_per_sm<T>()) per_sm = smooth_blocks_per_sm<T>();
  int G = nsm * per_sm;
  if (G > max_blocks) G = max_blocks;
  if (G < 1) G = 1;
  k_bar_reset<<<1, 1, 0, s>>>(a.ctl);
  SmoothBatchDev args = a;
  void* p[] = {&args};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_smooth<T, GR>, dim3(G), dim3(kThreads), p, 0, s);
  return e == cudaSuccess ? 0 : -3;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace

int64_t smooth_units(int64_t C) { return (C + kThreads - 1) / kThreads; }

size_t smooth_mesh_bytes(int form, int64_t C, int nf, int scheme) {
  const size_t w = form == FORM_PLAIN ? 4 : 8;             // wide word
  const size_t n = form == FORM_FP64 ? 8 : 4;              // narrow word
  const size_t wide = align256((size_t)nf * C * w);        // b, and x^{m-1} for BDF2
  return (scheme == TAU_BDF2 ? 2 : 1) * wide + 3 * align256((size_t)kMaxF * C * n) +
         align256((size_t)smooth_units(C) * kMaxF * kQ * 8) + 256;
}

size_t smooth_work_bytes(int form, int64_t C, int nf, int scheme) {
  return align256(smooth_mesh_bytes(form, C, nf, scheme)) + smooth_batch_bytes(1, smooth_units(C));
}

int launch_smooth(int form, const DevParams& P, void* phi, const void* guess, int nf, void* work,
                  const DevState& st, int* iters_dev, double rtol, int max_iter, int n_tau,
                  int scheme, const double coef[3], const SmoothZ* z, cudaStream_t s,
                  long long spin_limit) {
  SmoothMesh m{};
  m.phi = phi;
  m.guess = guess;
  m.work = work;
  m.iters = iters_dev;
  m.C = P.C;
  m.nf = nf;
  for (int k = 0; k < 3; ++k) {
    m.nc[k] = P.nc[k];
    m.per[k] = P.periodic[k];
    m.coef[k] = coef[k];
  }
  if (z) m.z = *z;
  void* batch = (char*)work + align256(smooth_mesh_bytes(form, P.C, nf, scheme));
  return launch_smooth_batch(form, &m, 1, nf, batch, rtol, max_iter, n_tau, scheme, st.ctl,
                             1 << 30, s, spin_limit);
}

size_t smooth_batch_bytes(int64_t B, int64_t U) {
  return 2 * align256((size_t)B * sizeof(SmoothMeshDev)) + align256((size_t)U * 4) +
         align256((size_t)B * sizeof(MeshState)) + 256;
}

// Spectrum [1, lmax] of A = I - sum_a coef_a L_a (lmax <= 1 + 4 sum_a coef_a by
// Gershgorin; on a graded z mesh the z term is 2 max_k (c-_k + c+_k), zmax > 0) and
// the Chebyshev coefficients of steps 1..kMaxStepsRound (the same in every round):
// rho_1 = 1 / sigma1, rho' = 1 / (2 sigma1 - rho), c1 = rho' rho, c2 = 2 rho' / delta.
static void smooth_spec(const double coef[3], double scale, double zmax, SmoothSpec* sp) {
  for (int k = 0; k < 3; ++k) {
    sp->coef[k] = scale * coef[k];
    sp->coef_hi[k] = (float)sp->coef[k];
    sp->coef_lo[k] = (float)(sp->coef[k] - (double)sp->coef_hi[k]);
  }
  double lmax = zmax > 0.0 ? 1.0 + 4.0 * (sp->coef[0] + sp->coef[1]) + 2.0 * zmax
                           : 1.0 + 4.0 * (sp->coef[0] + sp->coef[1] + sp->coef[2]);
  if (lmax < 1.0 + 1e-12) lmax = 1.0 + 1e-12;
  sp->theta = 0.5 * (lmax + 1.0);
  sp->delta = 0.5 * (lmax - 1.0);
  sp->sigma1 = sp->theta / sp->delta;
  sp->inv_theta_f = (float)(1.0 / sp->theta);
  const double sq = std::sqrt(lmax);
  sp->sig = (sq - 1.0) / (sq + 1.0);
  double rho = 1.0 / sp->sigma1;
  for (int j = 0; j < kMaxStepsRound; ++j) {
    const double rho_new = 1.0 / (2.0 * sp->sigma1 - rho);
    sp->cheb[0][j] = rho_new * rho;
    sp->cheb[1][j] = 2.0 * rho_new / sp->delta;
    sp->chebf[0][j] = (float)sp->cheb[0][j];
    sp->chebf[1][j] = (float)sp->cheb[1][j];
    rho = rho_new;
  }
}

static void smooth_mesh_layout(int form, int scheme, const SmoothMesh& in, SmoothMeshDev* out) {
  const size_t w = form == FORM_PLAIN ? 4 : 8;
  const size_t n = form == FORM_FP64 ? 8 : 4;
  char* p = (char*)in.work;
  SmoothMeshDev& m = *out;
  std::memset(&m, 0, sizeof(m));
  m.x = in.phi;
  m.guess = in.guess;
  m.b = p;  // [nf][C] wide
  p += align256((size_t)in.nf * in.C * w);
  if (scheme == TAU_BDF2) {
    m.xp = p;  // [nf][C] wide
    p += align256((size_t)in.nf * in.C * w);
  }
  const size_t nar = align256((size_t)kMaxF * in.C * n);  // [C][8] narrow
  m.q = p;
  m.d[0] = p + nar;
  m.d[1] = p + 2 * nar;
  p += 3 * nar;
  m.part = (double*)p;
  m.iters = in.iters;
  m.C = in.C;
  m.nu = smooth_units(in.C);
  for (int k = 0; k < 3; ++k) {
    m.nc[k] = in.nc[k];
    m.per[k] = in.per[k];
  }
  auto magic = [](uint64_t d) -> uint64_t { return d <= 1 ? 0 : ~(uint64_t)0 / d + 1; };
  m.div_x = magic((uint64_t)in.nc[0]);
  m.div_xy = magic((uint64_t)in.nc[0] * (uint64_t)in.nc[1]);
  m.z = in.z;
  const bool gr = in.z.cz[0] != nullptr;
  smooth_spec(in.coef, 1.0, gr ? in.z.zmax[0] : 0.0, &m.sp[0]);
  smooth_spec(in.coef, scheme == TAU_BDF2 ? 2.0 / 3.0 : 1.0, gr ? in.z.zmax[scheme == TAU_BDF2 ? 1 : 0] : 0.0,
              &m.sp[1]);
}

namespace {

template <class T, bool GR>
int launch_cluster(const SmoothBatchDev& a, int csize, cudaStream_t s) {
  using N = typename Wide<T>::N;
  const size_t smem = kClSmem;
  if (cudaFuncSetAttribute(k_smooth_cl<T, GR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return -3;
  if (csize > 8 && cudaFuncSetAttribute(k_smooth_cl<T, GR>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return -3;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kClThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(csize * 64);
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, (void*)k_smooth_cl<T, GR>, &cfg) != cudaSuccess || ncl < 1) return -3;
  const int64_t items = (int64_t)a.B * a.nf;
  if (ncl > items) ncl = (int)items;
  cfg.gridDim = dim3(csize * ncl);
  return cudaLaunchKernelEx(&cfg, k_smooth_cl<T, GR>, a) == cudaSuccess ? 0 : -3;
}

// Cluster plan of a mesh (whole z-planes per CTA, <= kClCells cells each), or
// csize 0 when the mesh does not fit the cluster solver.
void cluster_plan(int form, const SmoothMeshDev& m, int* csize, int* planes) {
  *csize = 0;
  *planes = 0;
  if (form == FORM_FP64) return;
  const int64_t nxy = (int64_t)m.nc[0] * m.nc[1];
  // per CTA: P planes of x (8 B) and three narrow words (4 B)
  const int64_t room = (int64_t)kClSmem / 4;  // in 4-byte words
  if (room < 5 * nxy) return;
  int pmax = (int)(room / (5 * nxy));
  if ((int64_t)pmax * nxy > kClCells) pmax = (int)(kClCells / nxy);
  if (pmax < 1) return;
  const int nz = m.nc[2];
  int cs = (nz + pmax - 1) / pmax;
  if (cs > kClMaxCta) return;
  const int p = (nz + cs - 1) / cs;
  cs = (nz + p - 1) / p;  // every CTA gets at least one plane
  *csize = cs;
  *planes = p;
}

}  // namespace

int launch_smooth_batch(int form, const SmoothMesh* meshes, int B, int nf, void* batch_work,
                        double rtol, int max_iter, int n_tau, int scheme, Ctl* ctl,
                        int max_blocks, cudaStream_t s, long long spin_limit) {
  if (B < 1 || B > kMaxBeds || nf < 1 || nf > kMaxF || (scheme != TAU_EULER && scheme != TAU_BDF2))
    return -1;
  // every mesh of a batch is graded or none is (one kernel instantiation per launch)
  const bool gr = meshes[0].z.cz[0] != nullptr;
  for (int b = 1; b < B; ++b)
    if ((meshes[b].z.cz[0] != nullptr) != gr) return -1;
  // meshes that fit the cluster solver take it; the rest take the grid solver.  The
  // choice depends on the mesh alone, so a bed smooths the same way in any batch.
  std::vector<SmoothMeshDev> mg, mc;
  int64_t U = 0;
  for (int b = 0; b < B; ++b) {
    SmoothMeshDev m;
    smooth_mesh_layout(form, scheme, meshes[b], &m);
    int cs, pl;
    cluster_plan(form, m, &cs, &pl);
    if (cs > 0) {
      m.cl_size = cs;
      m.cl_planes = pl;
      mc.push_back(m);
    } else {
      m.u0 = U;
      U += m.nu;
      mg.push_back(m);
    }
  }
  // cluster meshes grouped by cluster size (one launch per size)
  std::stable_sort(mc.begin(), mc.end(),
                   [](const SmoothMeshDev& x, const SmoothMeshDev& y) { return x.cl_size < y.cl_size; });
  char* p = (char*)batch_work;
  SmoothBatchDev a{};
  a.nf = nf;
  a.rtol2 = rtol * rtol;
  a.max_iter = max_iter;
  a.n_tau = n_tau;
  a.scheme = scheme;
  a.ctl = ctl;
  a.spin_limit = spin_limit > 0 ? spin_limit : 1;
  SmoothMeshDev* tab_g = (SmoothMeshDev*)p;
  p += align256((size_t)B * sizeof(SmoothMeshDev));
  SmoothMeshDev* tab_c = (SmoothMeshDev*)p;
  p += align256((size_t)B * sizeof(SmoothMeshDev));
  int rc = 0;
  if (!mc.empty()) {
    if (cudaMemcpyAsync(tab_c, mc.data(), mc.size() * sizeof(SmoothMeshDev), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return -3;
    for (size_t i0 = 0; i0 < mc.size();) {
      size_t i1 = i0;
      while (i1 < mc.size() && mc[i1].cl_size == mc[i0].cl_size) ++i1;
      SmoothBatchDev c = a;
      c.mesh = tab_c + i0;
      c.B = (int32_t)(i1 - i0);
      if (gr)
        rc = form == FORM_SPLIT ? launch_cluster<dd, true>(c, mc[i0].cl_size, s)
                                : launch_cluster<float, true>(c, mc[i0].cl_size, s);
      else
        rc = form == FORM_SPLIT ? launch_cluster<dd, false>(c, mc[i0].cl_size, s)
                                : launch_cluster<float, false>(c, mc[i0].cl_size, s);
      if (rc) {
        // a device without this cluster shape: these meshes take the grid solver
        cudaGetLastError();
        for (size_t i = i0; i < i1; ++i) {
          SmoothMeshDev m = mc[i];
          m.cl_size = m.cl_planes = 0;
          m.u0 = U;
          U += m.nu;
          mg.push_back(m);
        }
        rc = 0;
      }
      i0 = i1;
    }
  }
  if (!mg.empty()) {
    std::vector<int32_t> ub(U);
    for (size_t b = 0; b < mg.size(); ++b)
      for (int64_t u = 0; u < mg[b].nu; ++u) ub[mg[b].u0 + u] = (int32_t)b;
    a.mesh = tab_g;
    a.unit_bed = (int32_t*)p;
    p += align256((size_t)U * 4);
    a.pairs = p;
    p += align256((size_t)mg.size() * sizeof(MeshState));
    a.gflag = (int32_t*)p;
    a.B = (int32_t)mg.size();
    a.U = U;
    if (cudaMemcpyAsync(tab_g, mg.data(), mg.size() * sizeof(SmoothMeshDev), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync((void*)a.unit_bed, ub.data(), U * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(a.gflag, 0, 2 * sizeof(int32_t), s) != cudaSuccess)
      return -3;
    switch (form) {
      case FORM_SPLIT: rc = gr ? launch_impl<dd, true>(a, max_blocks, s) : launch_impl<dd, false>(a, max_blocks, s); break;
      case FORM_PLAIN: rc = gr ? launch_impl<float, true>(a, max_blocks, s) : launch_impl<float, false>(a, max_blocks, s); break;
      default: rc = gr ? launch_impl<double, true>(a, max_blocks, s) : launch_impl<double, false>(a, max_blocks, s); break;
    }
  }
  return rc;
}

}  // namespace sedi
