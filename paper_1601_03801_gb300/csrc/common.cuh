// Shared device-side definitions of the sm_103a hot path: number traits for the
// three arithmetic forms, packed per-particle records, the device control block
// and the launch-time parameter block.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "dd.cuh"

namespace sedi {

// ---------------------------------------------------------------- forms
enum Form { FORM_SPLIT = 0, FORM_PLAIN = 1, FORM_FP64 = 2 };

// Packed record of four state words: (x, y, z, r), (vx, vy, vz, m) or
// (wx, wy, wz, -).  16 bytes for FP32, 32 bytes (one sector) otherwise.
template <class S>
struct alignas(sizeof(S) * 4 >= 32 ? 32 : 16) Quad {
  S a, b, c, d;
};

// Device control block: buffer parities, rebuild trigger, error word, counters.
struct Ctl {
  int32_t st;              // particle-state buffer read at substep offset 0
  int32_t pb;              // buffer of per-particle arrays permuted on rebuild
  int32_t nl;              // buffer of neighbour lists / springs
  int32_t need_rebuild;    // set when max displacement > skin/2
  uint32_t disp_max_bits;  // max |x - x_build| since the last rebuild (float bits)
  int32_t error;           // first SEDI_E* raised on the device (0 = none)
  int32_t max_nn;          // longest list at the last rebuild
  int32_t overflow_nn;     // longest list that did not fit
  int64_t rebuilds;
  int32_t deposit_range;   // a deposited value overflowed the fixed-point format
  int32_t cg_status;       // 0 or SEDI_EDIVERGED / SEDI_ETIMEOUT from the smoother
  uint32_t bar_count, bar_gen;  // grid barrier of the persistent smoother
  uint32_t blocks_done;    // completion counter of the substep kernel
  uint32_t npair;          // interaction pairs of the current lists (pair list)
  int32_t ens_rebuild;     // ensembles: some bed needs a list rebuild after the last substep
  uint32_t pair_next;      // ordered pair schedule: next chunk of the pair list to claim
  uint32_t pair_done;      // ordered pair schedule: blocks finished (the last resets both)
};

// Constants of the force arithmetic, precomputed on the host in the force word
// F so the FP32 path performs no FP64 conversion.
template <class F>
struct ForceConsts {
  F Es, Gs, cdamp, kn_fac, mu, dt;     // contact: E*, G*, -2 sqrt(5/6) beta, (4/3)E*, friction
  F ct_ratio;                          // sqrt(S_t / S_n) = sqrt(4 G* / E*) (tangential damping)
  int32_t law;                         // 0 Hertz-Mindlin, 1 linear spring-dashpot
  F kn_lin, kt_lin, cdamp_lin;         // linear law: k_n, k_t, -2 beta
  F ct_ratio_lin;                      // linear law: sqrt(k_t / k_n)
  F lub_in, lub_out, six_pi_mu;        // lubrication limits (fractions of mean diameter), 6 pi mu_f
  F lift_c;                            // lift: C_l rho_f sqrt(nu_f)
  F rho_f, nu_f, c_add_rho_f, eps_max; // fluid
  F g[3];
  F lo[3], L[3], halfL[3], inv_h[3];   // box and mesh spacing (1/h = ncell/L)
};

// Box bounds in the state word S (for wrapping and wall distances).
template <class S>
struct BoxS {
  S lo[3], hi[3], L[3];
  S h[3];  // uniform cell size (hi - lo) / ncell per axis
};

// Launch-time parameters (precomputed on the host from sedi_params).
struct DevParams {
  double lo[3], hi[3], L[3];
  int32_t periodic[3], wall_lo[3], wall_hi[3];
  int32_t lubrication, drag, pressure_grad, added_mass;
  int32_t lift, lub_tangential;
  int32_t graded;                  // graded z mesh (tables in DevMesh)
  ForceConsts<float> cf;
  ForceConsts<double> cd;
  BoxS<float> bf;
  BoxS<double> bdb;
  BoxS<dd> bdd;
  // mesh
  int32_t nc[3];
  int64_t C;
  double inv_h[3];                 // ncell / L per axis (FP64, deposition cells)
  double vc;                       // cell volume
  // neighbour lists
  int32_t cap;                     // listed neighbours per particle
  double skin, lub_out_frac;
  float half_skin_f;
  float lub_out_f;
  int32_t nb[3];                   // bins per axis
  int64_t nbins;
  float bin_inv[3];                // bins per metre
  int32_t bin_reach;               // R: bins per list cutoff (the stencil spans +-R bins)
  int32_t bin_zfast;               // bin storage order: 0 x fastest, 1 z fastest
  // deposition
  int32_t shift[3];                // eps, momentum, force
  double two_shift[3];             // 2^shift
  float two_shift_f;               // 2^shift[2] (exact in FP32)
  float inv_vc_f;                  // 1 / V_c in FP32
};

template <class F>
__device__ __forceinline__ const ForceConsts<F>& fconsts(const DevParams& P);
template <>
__device__ __forceinline__ const ForceConsts<float>& fconsts<float>(const DevParams& P) {
  return P.cf;
}
template <>
__device__ __forceinline__ const ForceConsts<double>& fconsts<double>(const DevParams& P) {
  return P.cd;
}
template <class S>
__device__ __forceinline__ const BoxS<S>& sbox(const DevParams& P);
template <>
__device__ __forceinline__ const BoxS<float>& sbox<float>(const DevParams& P) {
  return P.bf;
}
template <>
__device__ __forceinline__ const BoxS<double>& sbox<double>(const DevParams& P) {
  return P.bdb;
}
template <>
__device__ __forceinline__ const BoxS<dd>& sbox<dd>(const DevParams& P) {
  return P.bdd;
}

// ---------------------------------------------------------------- numbers
// S: state word; F: force word.  Ops needed by the generic kernels.
template <class S>
struct Num;

template <>
struct Num<float> {
  __device__ static float f(float a) { return a; }
  __device__ static float lo(float) { return 0.0f; }
  __device__ static double d(float a) { return (double)a; }
  __device__ static float from_f(float a) { return a; }
  __device__ static float add(float a, float b) { return a + b; }
  __device__ static float sub(float a, float b) { return a - b; }
  __device__ static float mul(float a, float b) { return a * b; }
  __device__ static float add_f(float a, float b) { return a + b; }
  __device__ static float mul_f(float a, float b) { return a * b; }
  __device__ static float fma_ff(float a, float b, float c) { return fmaf(b, c, a); }
  __device__ static bool lt(float a, float b) { return a < b; }
  __device__ static float dif(float a, float b) { return a - b; }
  __device__ static float addq(float a, float b) { return a + b; }
  __device__ static float subq(float a, float b) { return a - b; }
  __device__ static float fmaq(float a, float b, float c) { return fmaf(b, c, a); }
  __device__ static float neg(float a) { return -a; }
  static constexpr bool kExtended = false;  // no wider word than the force word
};

template <>
struct Num<double> {
  __device__ static double f(double a) { return a; }
  __device__ static double lo(double) { return 0.0; }
  __device__ static double d(double a) { return a; }
  __device__ static double from_f(double a) { return a; }
  __device__ static double add(double a, double b) { return a + b; }
  __device__ static double sub(double a, double b) { return a - b; }
  __device__ static double mul(double a, double b) { return a * b; }
  __device__ static double add_f(double a, double b) { return a + b; }
  __device__ static double mul_f(double a, double b) { return a * b; }
  __device__ static double fma_ff(double a, double b, double c) { return a + b * c; }
  __device__ static bool lt(double a, double b) { return a < b; }
  __device__ static double dif(double a, double b) { return a - b; }
  __device__ static double addq(double a, double b) { return a + b; }
  __device__ static double subq(double a, double b) { return a - b; }
  __device__ static double fmaq(double a, double b, double c) { return a + b * c; }
  __device__ static double neg(double a) { return -a; }
  static constexpr bool kExtended = false;
};

template <>
struct Num<dd> {
  __device__ static float f(dd a) { return a.hi; }
  __device__ static float lo(dd a) { return a.lo; }  // the low word (f() is the high one)
  __device__ static double d(dd a) { return dd_to_double(a); }
  __device__ static dd from_f(float a) { return dd{a, 0.0f}; }
  __device__ static dd add(dd a, dd b) { return dd_add(a, b); }
  __device__ static dd sub(dd a, dd b) { return dd_sub(a, b); }
  __device__ static dd mul(dd a, dd b) { return dd_mul(a, b); }
  __device__ static dd add_f(dd a, float b) { return dd_add_f(a, b); }
  __device__ static dd mul_f(dd a, float b) { return dd_mul_f(a, b); }
  __device__ static dd fma_ff(dd a, float b, float c) { return dd_fma_ff(a, b, c); }
  __device__ static bool lt(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
  // approximate difference a - b in FP32 (for culling)
  __device__ static float dif(dd a, dd b) {
    return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo));
  }
  // additions whose error is relative to the operands (see dd_add_fast)
  __device__ static dd addq(dd a, dd b) { return dd_add_fast(a, b); }
  __device__ static dd subq(dd a, dd b) { return dd_sub_fast(a, b); }
  __device__ static dd fmaq(dd a, float b, float c) { return dd_add_fast(a, two_prod(b, c)); }
  __device__ static dd neg(dd a) { return dd_neg(a); }
  static constexpr bool kExtended = true;   // state word wider than the force word
};

template <class S>
__device__ __forceinline__ S s_zero() {
  return S{};
}

// Loads and stores of Quad records as vector words.
__device__ __forceinline__ Quad<float> ldq(const Quad<float>* p) {
  float4 v = *reinterpret_cast<const float4*>(p);
  return Quad<float>{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ void stq(Quad<float>* p, const Quad<float>& q) {
  *reinterpret_cast<float4*>(p) = make_float4(q.a, q.b, q.c, q.d);
}
__device__ __forceinline__ Quad<dd> ldq(const Quad<dd>* p) {
  const float4* v = reinterpret_cast<const float4*>(p);
  float4 u = v[0], w = v[1];
  return Quad<dd>{dd{u.x, u.y}, dd{u.z, u.w}, dd{w.x, w.y}, dd{w.z, w.w}};
}
__device__ __forceinline__ void stq(Quad<dd>* p, const Quad<dd>& q) {
  float4* v = reinterpret_cast<float4*>(p);
  v[0] = make_float4(q.a.hi, q.a.lo, q.b.hi, q.b.lo);
  v[1] = make_float4(q.c.hi, q.c.lo, q.d.hi, q.d.lo);
}
__device__ __forceinline__ Quad<double> ldq(const Quad<double>* p) {
  const double2* v = reinterpret_cast<const double2*>(p);
  double2 u = v[0], w = v[1];
  return Quad<double>{u.x, u.y, w.x, w.y};
}
__device__ __forceinline__ void stq(Quad<double>* p, const Quad<double>& q) {
  double2* v = reinterpret_cast<double2*>(p);
  v[0] = make_double2(q.a, q.b);
  v[1] = make_double2(q.c, q.d);
}

// Form -> (state word, force word, spring word).
template <int FORM>
struct Traits;
template <>
struct Traits<FORM_SPLIT> {
  using S = dd;
  using F = float;
};
template <>
struct Traits<FORM_PLAIN> {
  using S = float;
  using F = float;
};
template <>
struct Traits<FORM_FP64> {
  using S = double;
  using F = double;
};

// Device arrays of one handle (type-erased; kernels cast by form).
struct DevState {
  int64_t N;
  void* pos[2];       // Quad<S> (x, y, z, r)
  void* vel[2];       // Quad<S> (vx, vy, vz, m)
  void* omg[2];       // Quad<S> (wx, wy, wz, 0)
  void* acc[2];       // Quad<F> lagged acceleration (pb parity)
  int32_t* uid[2];    // caller index (pb parity)
  double* r64[2];     // FP64 radius (pb parity)
  double* vfrac[2];   // V_p / V_c in FP64 (pb parity)
  float4* xb[2];      // position at the last rebuild (pb parity)
  void* whist[2];     // S [6 walls][3][N] springs (pb parity)
  uint32_t* wmask[2]; // bit w: wall spring w in use (pb parity)
  int32_t* nbr[2];    // [cap][N] list entry: partner index | first-in-pair bit (nl parity)
  int32_t* nn[2];     // [N] list length (nl parity)
  void* hist[2];      // Quad<S> [cap][N] pair springs (x, y, z, 0) (nl parity)
  uint32_t* cmask[2]; // bit k: slot k holds a spring (nl parity)
  // pair list of the current lists (null: not kept): every listed pair once, from the
  // particle that comes first in it.  Each substep the pair kernel writes every listed
  // pair's record (one 32-byte sector per pair, in pair order, so the writes are
  // sequential): {F, delta/2} {G, flags}, with F the pair force on the first particle
  // (contact plus lubrication), G = n x F_t (the contact torque on either particle is
  // its lever r - delta/2 times G) and the kSlot* flags as the bits of the last word.
  // In the pair mode only the first particle's slot holds the pair's spring (see
  // launch_spring_sync).
  int4* pairs;        // [cap N / 2] (i, slot of j in i's list, j, slot of i in j's list)
  int32_t* pstart;    // [N + 1] first pair of each appending particle (its count before the scan)
  int32_t* pscan_blk; // tile sums of that scan
  int32_t* pid;       // [cap][N] pair of each list slot | kFirstBit if the owner is first
  float4* prec;       // [cap N / 2][2] the pair records of the current substep
  int64_t pcap;       // capacity of the pair arrays (cap N / 2)
  // binning scratch
  int32_t* bin_of;    // [N]
  int32_t* bin_count; // [nbins]
  int32_t* bin_start; // [nbins + 1]
  int32_t* bin_fill;  // [nbins]
  int32_t* order;     // [N] new -> old
  int32_t* scan_blk;  // block sums of the scan
  // debug forces (compute_forces)
  double* fdbg;       // [4][N][3]
  Ctl* ctl;
};

// Mesh arrays (type-erased Quad<F>): ufe = (Ux, Uy, Uz, eps_s), gfl = G where
// the pressure-gradient + fluid-acceleration part of f_fp is V_p * G, wfl =
// (curl U, 0) for the lift force.  Graded z mesh only (null otherwise): faces
// zf [nz + 1], centres zc [nz] (FP64) and zcf (FP32), cell volumes vcz [nz].
struct DevMesh {
  void* ufe;
  void* gfl;
  void* wfl;
  const double* zf;
  const double* zc;
  const float* zcf;
  const double* vcz;
  int64_t C;
};

constexpr int kWalls = 6;
constexpr int kMaxCap = 32;  // listed neighbours per particle at most (slot masks are 32-bit)

// One bed of an ensemble as the kernels see it: the single-bed views of its arrays
// and parameters.  Batched launches take a device table of these and pick the bed
// of a block from blockIdx.y.
struct alignas(16) BedView {
  DevState st;
  DevMesh mesh;
  DevParams P;
  void* qfix;  // [7][C] fixed-point deposition (split/FP64 forms)
  void* phi;   // [8][C] smoothing word (the plain form deposits here)
};

#ifdef __CUDACC__
// Copy the view of this block's bed (blockIdx.y) into shared memory.
__device__ __forceinline__ const BedView& bed_view(const BedView* views) {
  __shared__ BedView s_view;
  const int4* src = reinterpret_cast<const int4*>(views + blockIdx.y);
  int4* dst = reinterpret_cast<int4*>(&s_view);
  for (int k = threadIdx.x; k < (int)(sizeof(BedView) / 16); k += blockDim.x) dst[k] = src[k];
  __syncthreads();
  return s_view;
}
#endif

// Flags of a pair record: the pair interacts (the record holds its force: contact
// plus lubrication), and it is in contact (the record holds the contact torque, and
// the pair's spring is live).
constexpr uint8_t kSlotForce = 1, kSlotContact = 2;

// A list entry holds the partner index in bits 0-30 and, in bit 31, whether the
// owner comes first in canonical pair order (lower caller index).
constexpr uint32_t kFirstBit = 0x80000000u;
// Bring the line of p into L1 ahead of its use (no register is held while in flight).
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__host__ __device__ __forceinline__ int32_t nbr_index(int32_t e) { return e & 0x7fffffff; }
__host__ __device__ __forceinline__ bool nbr_first(int32_t e) { return ((uint32_t)e & kFirstBit) != 0; }

}  // namespace sedi
