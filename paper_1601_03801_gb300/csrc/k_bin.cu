// Neighbour-list rebuild (Sec. 2.5: link-cell binning + neighbour lists, O(N)).
//
//   check    : rebuild when the largest displacement since the last build
//              exceeds skin/2 (lists hold pairs within cutoff + skin)
//   bin      : bin of each particle, counts per bin
//   scan     : exclusive prefix sum of the counts (three-kernel block scan)
//   scatter  : particle -> slot of its bin; per-bin sort by caller index makes the
//              order deterministic
//   gather   : permute every per-particle array into the other buffer
//   build    : one thread per particle scans the (2R + 1)^3 surrounding bins (R bins
//              per list cutoff, 1 or 2); FP32 test with a relative margin, exact FP64
//              predicate
//                 d2 = (dx*dx + dy*dy) + dz*dz  <  ((r_i + r_j)(1 + f) + skin)^2
//              (no fused multiply-add) only when the FP32 test is inconclusive,
//              so lists are bit-identical to an FP64 evaluation of the predicate;
//              each list holds its partners in caller-index order, so neither the bin
//              size nor the bin order changes a list (nor any sum over one)
//   remap    : every new (i, k) entry looks its partner's caller index up in the
//              particle's old list and carries the tangential spring over
//   flip     : switch buffers, reset the displacement
// Every kernel of the sequence returns at once when ctl->need_rebuild is 0, so the
// sequence can be queued unconditionally or placed under a graph conditional.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace sedi {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ bool skip(const Ctl* ctl, bool force) {
  return !force && !ctl->need_rebuild;
}

__global__ void k_check(Ctl* ctl, float thresh2, cudaGraphConditionalHandle h, int use_cond) {
  float m = __uint_as_float(ctl->disp_max_bits);
  int need = (m > thresh2) ? 1 : 0;
  ctl->need_rebuild = need;
  if (use_cond) cudaGraphSetConditional(h, need ? 1u : 0u);
}

__global__ void k_force_need(Ctl* ctl) { ctl->need_rebuild = 1; }

__device__ __forceinline__ void zero_bins_body(const DevState& st, int64_t nbins, bool force) {
  if (skip(st.ctl, force)) return;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbins;
       b += (int64_t)gridDim.x * blockDim.x) {
    st.bin_count[b] = 0;
    st.bin_fill[b] = 0;
  }
}

template <class S>
__device__ __forceinline__ int bin_axis(S x, const DevParams& P, int a) {
  float rel = (float)Num<S>::f(Num<S>::sub(x, sbox<S>(P).lo[a]));
  int b = (int)floorf(rel * P.bin_inv[a]);
  if (b < 0) b = 0;
  if (b > P.nb[a] - 1) b = P.nb[a] - 1;
  return b;
}

// Storage order of the bins (the autotuner's choice): x fastest, then y, then z; or z
// fastest, then y, then x, which keeps a thin bed's vertical neighbours next to each
// other in memory (13% less DRAM traffic for the pair list on the 10M bed).  The order
// changes no list: every list is sorted by caller index.
__device__ __forceinline__ int64_t bin_key(int bx, int by, int bz, const DevParams& P) {
  if (P.bin_zfast) return ((int64_t)bx * P.nb[1] + by) * P.nb[2] + bz;
  return ((int64_t)bz * P.nb[1] + by) * P.nb[0] + bx;
}

template <class S>
__device__ __forceinline__ int64_t bin_index(const Quad<S>& p, const DevParams& P) {
  int bx = bin_axis<S>(p.a, P, 0), by = bin_axis<S>(p.b, P, 1), bz = bin_axis<S>(p.c, P, 2);
  return bin_key(bx, by, bz, P);
}

template <int FORM>
__device__ __forceinline__ void bin_count_body(const DevState& st, const DevParams& P, int sub_off,
                                               bool force) {
  if (skip(st.ctl, force)) return;
  using S = typename Traits<FORM>::S;
  const int sb = (st.ctl->st + sub_off) & 1;
  const Quad<S>* pos = (const Quad<S>*)st.pos[sb];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < st.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = bin_index<S>(ldq(pos + i), P);
    st.bin_of[i] = (int32_t)b;
    atomicAdd(&st.bin_count[b], 1);
  }
}

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of a thread value across the block; returns the block total.
__device__ __forceinline__ int block_excl_scan(int v, int* total) {
  __shared__ int wsum[32];
  __shared__ int wtot;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = warp_incl_scan(v);
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    int s = lane < nw ? wsum[lane] : 0;
    int si = warp_incl_scan(s);
    if (lane < nw) wsum[lane] = si - s;
    if (lane == nw - 1) wtot = si;
  }
  __syncthreads();
  int r = incl - v + wsum[wid];
  *total = wtot;
  __syncthreads();
  return r;
}

// Exclusive scan of cnt[0, n) into start[0, n] (start[n] = the total) in three
// launches: tile sums (scan1), the tiles' prefix in one block (scan2), the tile
// offsets added (scan3).  cnt and start may be the same array.
__device__ __forceinline__ void scan1_of(const int32_t* cnt, int32_t* start, int32_t* blk, int64_t n) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t b = base + k;
    v[k] = b < n ? cnt[b] : 0;
    s += v[k];
  }
  int total;
  int ex = block_excl_scan(s, &total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t b = base + k;
    if (b < n) start[b] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) blk[blockIdx.x] = total;
}

__device__ __forceinline__ void scan2_of(int32_t* blk, int64_t nblk, int32_t* start, int64_t n) {
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nblk; base += blockDim.x) {
    int64_t b = base + threadIdx.x;
    int v = b < nblk ? blk[b] : 0;
    int total;
    int ex = block_excl_scan(v, &total);
    if (b < nblk) blk[b] = ex + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) start[n] = carry;
}

__device__ __forceinline__ void scan3_of(int32_t* start, const int32_t* blk, int64_t n) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const int add = blk[blockIdx.x];
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
    int64_t b = base + k;
    if (b < n) start[b] += add;
  }
}

__device__ __forceinline__ void scan1_body(const DevState& st, int64_t nbins, bool force) {
  if (skip(st.ctl, force)) return;
  scan1_of(st.bin_count, st.bin_start, st.scan_blk, nbins);
}

__device__ __forceinline__ void scan2_body(const DevState& st, int64_t nblk, int64_t nbins, bool force) {
  if (skip(st.ctl, force)) return;
  scan2_of(st.scan_blk, nblk, st.bin_start, nbins);
}

__device__ __forceinline__ void scan3_body(const DevState& st, int64_t nbins, bool force) {
  if (skip(st.ctl, force)) return;
  scan3_of(st.bin_start, st.scan_blk, nbins);
}

__device__ __forceinline__ void scatter_body(const DevState& st, bool force) {
  if (skip(st.ctl, force)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < st.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    int b = st.bin_of[i];
    int slot = atomicAdd(&st.bin_fill[b], 1);
    st.order[st.bin_start[b] + slot] = (int32_t)i;
  }
}

// Insertion sort of each bin's entries by caller index (bins hold a few particles).
__device__ __forceinline__ void sort_bins_body(const DevState& st, int64_t nbins, bool force) {
  if (skip(st.ctl, force)) return;
  const int32_t* uid = st.uid[st.ctl->pb];
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbins;
       b += (int64_t)gridDim.x * blockDim.x) {
    int n = st.bin_count[b];
    if (n < 2) continue;
    int32_t* o = st.order + st.bin_start[b];
    for (int a = 1; a < n; ++a) {
      int32_t v = o[a];
      int32_t key = uid[v];
      int c = a - 1;
      while (c >= 0 && uid[o[c]] > key) {
        o[c + 1] = o[c];
        --c;
      }
      o[c + 1] = v;
    }
  }
}

template <int FORM>
__device__ __forceinline__ void gather_body(const DevState& st, int sub_off, bool force) {
  if (skip(st.ctl, force)) return;
  using S = typename Traits<FORM>::S;
  using F = typename Traits<FORM>::F;
  const int sb = (st.ctl->st + sub_off) & 1, ob = sb ^ 1;
  const int pb = st.ctl->pb, qb = pb ^ 1;
  const int64_t N = st.N;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = st.order[k];
    Quad<S> p = ldq((const Quad<S>*)st.pos[sb] + o);
    stq((Quad<S>*)st.pos[ob] + k, p);
    stq((Quad<S>*)st.vel[ob] + k, ldq((const Quad<S>*)st.vel[sb] + o));
    stq((Quad<S>*)st.omg[ob] + k, ldq((const Quad<S>*)st.omg[sb] + o));
    stq((Quad<F>*)st.acc[qb] + k, ldq((const Quad<F>*)st.acc[pb] + o));
    st.uid[qb][k] = st.uid[pb][o];
    st.r64[qb][k] = st.r64[pb][o];
    st.vfrac[qb][k] = st.vfrac[pb][o];
    const uint32_t wm = st.wmask[pb][o];
    st.wmask[qb][k] = wm;
    if (wm) {
      const S* wh = (const S*)st.whist[pb];
      S* wq = (S*)st.whist[qb];
      for (int w = 0; w < kWalls; ++w)
        if ((wm >> w) & 1u)
          for (int c = 0; c < 3; ++c) wq[((int64_t)w * 3 + c) * N + k] = wh[((int64_t)w * 3 + c) * N + o];
    }
    st.xb[qb][k] = make_float4((float)Num<S>::f(p.a), (float)Num<S>::f(p.b),
                               (float)Num<S>::f(p.c), 0.0f);
  }
}

__device__ __forceinline__ double min_image_d(double d, int per, double L) {
  if (!per) return d;
  if (d > 0.5 * L) return d - L;
  if (d < -0.5 * L) return d + L;
  return d;
}

// Exact FP64 list predicate (no contraction).
__device__ __forceinline__ bool listed_exact(const double xi[3], const double xj[3], double ri,
                                             double rj, const DevParams& P) {
  double d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = min_image_d(__dsub_rn(xj[a], xi[a]), P.periodic[a], P.L[a]);
  double d2 = __dmul_rn(d[0], d[0]);
  d2 = __dadd_rn(d2, __dmul_rn(d[1], d[1]));
  d2 = __dadd_rn(d2, __dmul_rn(d[2], d[2]));
  double s = __dadd_rn(ri, rj);
  double rc = __dadd_rn(s, __dmul_rn(P.lub_out_frac, s));
  rc = __dadd_rn(rc, P.skin);
  return d2 < __dmul_rn(rc, rc);
}

template <int FORM>
__device__ __forceinline__ void build_body(const DevState& st, const DevParams& P, int sub_off,
                                           bool force) {
  if (skip(st.ctl, force)) return;
  using S = typename Traits<FORM>::S;
  using NS = Num<S>;
  // after the gather the sorted state sits in the other buffers
  const int sb = ((st.ctl->st + sub_off) & 1) ^ 1;
  const int qb = st.ctl->pb ^ 1;
  const int ql = st.ctl->nl ^ 1;
  const int64_t N = st.N;
  const Quad<S>* pos = (const Quad<S>*)st.pos[sb];
  const double* r64 = st.r64[qb];
  const int32_t* uid = st.uid[qb];
  int32_t* nbr = st.nbr[ql];
  const float fr = (float)P.lub_out_frac, sk = (float)P.skin;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Quad<S> pi = ldq(pos + i);
    const double ri = r64[i];
    const int32_t ui = uid[i];
    const float rif = (float)ri;
    int c[3] = {bin_axis<S>(pi.a, P, 0), bin_axis<S>(pi.b, P, 1), bin_axis<S>(pi.c, P, 2)};
    // the partners found so far, ordered by caller index (insertion), so the list
    // order does not depend on the bins
    int32_t ent[kMaxCap], key[kMaxCap];
    int n = 0;
    const int R = P.bin_reach;
    // the candidates of sorted positions [s0, s1): FP32 test with a relative margin on
    // the stored words (the radius from the position record), the exact FP64 predicate
    // inside the margin
    auto visit = [&](int s0, int s1) {
      for (int j = s0; j < s1; ++j) {
        if (j == i) continue;
        const Quad<S> pj = ldq(pos + j);
        float d[3] = {(float)NS::dif(pj.a, pi.a), (float)NS::dif(pj.b, pi.b), (float)NS::dif(pj.c, pi.c)};
#pragma unroll
        for (int a = 0; a < 3; ++a)
          if (P.periodic[a])
            d[a] = d[a] > P.cf.halfL[a] ? d[a] - P.cf.L[a] : (d[a] < -P.cf.halfL[a] ? d[a] + P.cf.L[a] : d[a]);
        const float d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const float s = rif + (float)NS::f(pj.d);
        const float rc = s + fr * s + sk;
        const float rc2 = rc * rc;
        bool in;
        if (d2 < rc2 * (1.0f - 2e-4f)) in = true;
        else if (d2 > rc2 * (1.0f + 2e-4f)) in = false;
        else {
          const double xi[3] = {NS::d(pi.a), NS::d(pi.b), NS::d(pi.c)};
          const double xj[3] = {NS::d(pj.a), NS::d(pj.b), NS::d(pj.c)};
          in = listed_exact(xi, xj, ri, r64[j], P);
        }
        if (in) {
          if (n < P.cap) {
            const int32_t uj = uid[j];
            int k = n;
            while (k > 0 && key[k - 1] > uj) {
              key[k] = key[k - 1];
              ent[k] = ent[k - 1];
              --k;
            }
            key[k] = uj;
            ent[k] = j | (ui < uj ? (int32_t)kFirstBit : 0);
          }
          ++n;
        }
      }
    };
    // the stencil as runs along the bins' fastest axis: 2R + 1 consecutive bins are
    // one range of sorted positions unless the run wraps a periodic face
    const int fa = P.bin_zfast ? 2 : 0;           // fastest axis
    const int sa = 1, ta = P.bin_zfast ? 0 : 2;  // the other two
    for (int ot = -R; ot <= R; ++ot) {
      int ct = c[ta] + ot;
      if (P.periodic[ta]) ct = (ct + P.nb[ta]) % P.nb[ta];
      else if (ct < 0 || ct >= P.nb[ta]) continue;
      for (int os = -R; os <= R; ++os) {
        int cs = c[sa] + os;
        if (P.periodic[sa]) cs = (cs + P.nb[sa]) % P.nb[sa];
        else if (cs < 0 || cs >= P.nb[sa]) continue;
        int t[3];
        t[ta] = ct;
        t[sa] = cs;
        const int lo = c[fa] - R, hi = c[fa] + R;
        if (P.periodic[fa] && (lo < 0 || hi >= P.nb[fa])) {
          for (int of = lo; of <= hi; ++of) {
            t[fa] = (of + P.nb[fa]) % P.nb[fa];
            const int64_t bk = bin_key(t[0], t[1], t[2], P);
            visit(st.bin_start[bk], st.bin_start[bk] + st.bin_count[bk]);
          }
        } else {
          t[fa] = lo > 0 ? lo : 0;
          const int64_t b0 = bin_key(t[0], t[1], t[2], P);
          t[fa] = hi < P.nb[fa] - 1 ? hi : P.nb[fa] - 1;
          const int64_t b1 = bin_key(t[0], t[1], t[2], P);
          visit(st.bin_start[b0], st.bin_start[b1] + st.bin_count[b1]);
        }
      }
    }
    const int nk = n < P.cap ? n : P.cap;
    for (int k = 0; k < nk; ++k) nbr[(int64_t)k * N + i] = ent[k];
    st.nn[ql][i] = nk;
    atomicMax(&st.ctl->max_nn, n);
    if (n > P.cap) {
      atomicMax(&st.ctl->overflow_nn, n);
      atomicCAS(&st.ctl->error, 0, -4);
    }
  }
}

template <int FORM>
__device__ __forceinline__ void remap_body(const DevState& st, const DevParams& P, bool force) {
  if (skip(st.ctl, force)) return;
  using S = typename Traits<FORM>::S;
  const int pb = st.ctl->pb, qb = pb ^ 1;
  const int nl = st.ctl->nl, ql = nl ^ 1;
  const int64_t N = st.N;
  const Quad<S>* hold = (const Quad<S>*)st.hist[nl];
  Quad<S>* hnew = (Quad<S>*)st.hist[ql];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = st.order[i];
    const uint32_t omask = force ? 0u : st.cmask[nl][o];
    uint32_t nmask = 0;
    if (omask) {
      const int onn = st.nn[nl][o];
      const int nn = st.nn[ql][i];
      // the partners' caller indices of both lists (independent loads, issued together)
      int32_t ou[kMaxCap], nu[kMaxCap];
      bool sorted = true;
      for (int kk = 0; kk < onn; ++kk) ou[kk] = st.uid[pb][nbr_index(st.nbr[nl][(int64_t)kk * N + o])];
      for (int k = 0; k < nn; ++k) nu[k] = st.uid[qb][nbr_index(st.nbr[ql][(int64_t)k * N + i])];
      for (int kk = 1; kk < onn; ++kk) sorted = sorted && ou[kk - 1] < ou[kk];
      int kk = 0;
      for (int k = 0; k < nn; ++k) {
        const int32_t uj = nu[k];
        int hit = -1;
        if (sorted) {
          // lists built here hold their partners in caller-index order: one merge walk
          while (kk < onn && ou[kk] < uj) ++kk;
          if (kk < onn && ou[kk] == uj) hit = kk;
        } else {
          // lists of another order (an imported checkpoint): search
          for (int q = 0; q < onn; ++q)
            if (ou[q] == uj) {
              hit = q;
              break;
            }
        }
        if (hit >= 0 && ((omask >> hit) & 1u)) {
          stq(hnew + (int64_t)k * N + i, ldq(hold + (int64_t)hit * N + o));
          nmask |= 1u << k;
        }
      }
    }
    st.cmask[ql][i] = nmask;
  }
}

__device__ __forceinline__ void flip_body(const DevState& st, bool force) {
  if (skip(st.ctl, force)) return;
  Ctl* c = st.ctl;
  c->st ^= 1;
  c->pb ^= 1;
  c->nl ^= 1;
  c->disp_max_bits = 0u;
  c->need_rebuild = 0;
  c->rebuilds += 1;
}

// Pair list of the lists just built (before the flip): every particle appends, in
// slot order, its pairs with partners of higher index (a warp's particles
// contiguously, one atomic per warp), each stored from the particle that comes first
// in it (list bit) with the pair's slot in both lists; both slots record the pair id.  The order of the pairs in the
// list depends on scheduling; nothing computed from a pair does.
// The pairs a particle appends to the pair list: those with a partner of higher
// storage index, so each particle's pairs sit next to those of its neighbours in the
// (cell-sorted) order.  Their count per particle (pair_count), scanned into each
// particle's first pair, then the pairs themselves (pair_fill): the list is in
// storage order of the appending particle, the same for every run.
__device__ __forceinline__ uint32_t own_pairs(const int32_t* nbr, int ni, int64_t i, int64_t N) {
  uint32_t own = 0;
  for (int k = 0; k < ni; ++k)
    if (nbr_index(nbr[(int64_t)k * N + i]) > (int32_t)i) own |= 1u << k;
  return own;
}

__device__ __forceinline__ void pair_count_body(const DevState& st, bool force, bool current) {
  if (skip(st.ctl, force)) return;
  const int ql = current ? st.ctl->nl : st.ctl->nl ^ 1;  // the new lists, or the current ones
  const int64_t N = st.N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    st.pstart[i] = __popc(own_pairs(st.nbr[ql], st.nn[ql][i], i, N));
}

__device__ __forceinline__ void pair_fill_body(const DevState& st, bool force, bool current) {
  if (skip(st.ctl, force)) return;
  const int ql = current ? st.ctl->nl : st.ctl->nl ^ 1;
  const int64_t N = st.N;
  const int32_t* nbr = st.nbr[ql];
  const int32_t* nn = st.nn[ql];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // every listed pair once; more than the arrays hold is an internal error
    const int64_t total = st.pstart[N];
    if (total > st.pcap) atomicCAS(&st.ctl->error, 0, -9);
    st.ctl->npair = (uint32_t)(total < st.pcap ? total : st.pcap);
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int ni = nn[i];
    uint32_t own = own_pairs(nbr, ni, i, N), first = 0;
    for (int k = 0; k < ni; ++k)
      if (nbr_first(nbr[(int64_t)k * N + i])) first |= 1u << k;
    int64_t m = st.pstart[i];
    while (own) {
      const int k = __ffs(own) - 1;
      own &= own - 1;
      const int32_t j = nbr_index(nbr[(int64_t)k * N + i]);
      int k2 = -1;
      const int nj = nn[j];
      for (int kk = 0; kk < nj; ++kk)
        if (nbr_index(nbr[(int64_t)kk * N + j]) == (int32_t)i) {
          k2 = kk;
          break;
        }
      if (k2 < 0) {
        // lists are symmetric by construction; an unmatched pair is an internal error
        atomicCAS(&st.ctl->error, 0, -9);
        k2 = 0;
      }
      if (m >= st.pcap) break;  // reported above
      // the pair from the particle that comes first in it; each slot's pair id
      const bool i_first = (first >> k) & 1u;
      st.pairs[m] = i_first ? make_int4((int)i, k, j, k2) : make_int4(j, k2, (int)i, k);
      st.pid[(int64_t)k * N + i] = (int32_t)(m | (i_first ? kFirstBit : 0u));
      st.pid[(int64_t)k2 * N + j] = (int32_t)(m | (i_first ? 0u : kFirstBit));
      ++m;
    }
  }
}

__global__ void k_advance(Ctl* ctl, int n) { ctl->st = (ctl->st + n) & 1; }

// ---------------------------------------------------------------- kernels
// Single-bed kernels take the bed's views by value; the _e kernels of an ensemble
// take blockIdx.y as the bed and return at once for a bed without a rebuild.

__global__ void k_zero_bins(DevState st, int64_t nbins, bool force) { zero_bins_body(st, nbins, force); }
template <int FORM>
__global__ void k_bin_count(DevState st, DevParams P, int sub_off, bool force) {
  bin_count_body<FORM>(st, P, sub_off, force);
}
__global__ void k_scan1(DevState st, int64_t nbins, bool force) { scan1_body(st, nbins, force); }
__global__ void k_scan2(DevState st, int64_t nblk, int64_t nbins, bool force) {
  scan2_body(st, nblk, nbins, force);
}
__global__ void k_scan3(DevState st, int64_t nbins, bool force) { scan3_body(st, nbins, force); }
__global__ void k_scatter(DevState st, bool force) { scatter_body(st, force); }
__global__ void k_sort_bins(DevState st, int64_t nbins, bool force) { sort_bins_body(st, nbins, force); }
template <int FORM>
__global__ void k_gather(DevState st, int sub_off, bool force) { gather_body<FORM>(st, sub_off, force); }
template <int FORM>
__global__ void k_build(DevState st, DevParams P, int sub_off, bool force) {
  build_body<FORM>(st, P, sub_off, force);
}
template <int FORM>
__global__ void k_remap(DevState st, DevParams P, bool force) { remap_body<FORM>(st, P, force); }
__global__ void k_flip(DevState st, bool force) { flip_body(st, force); }
__global__ void k_pair_count(DevState st, bool force, bool current) { pair_count_body(st, force, current); }
__global__ void k_pscan1(DevState st, bool force) {
  if (!skip(st.ctl, force)) scan1_of(st.pstart, st.pstart, st.pscan_blk, st.N);
}
__global__ void k_pscan2(DevState st, int64_t nblk, bool force) {
  if (!skip(st.ctl, force)) scan2_of(st.pscan_blk, nblk, st.pstart, st.N);
}
__global__ void k_pscan3(DevState st, bool force) {
  if (!skip(st.ctl, force)) scan3_of(st.pstart, st.pscan_blk, st.N);
}
__global__ void k_pair_fill(DevState st, bool force, bool current) {
  pair_fill_body(st, force, current);
}


// Pair mode keeps a pair's spring in the first particle's slot only; this copies it
// to the partner's slot, as the per-particle loop keeps it (before the lists are
// read slot by slot: another launch variant, a checkpoint, the contact export).
template <int FORM>
__global__ void k_spring_sync(DevState st) {
  using S = typename Traits<FORM>::S;
  const int nl = st.ctl->nl;
  const int64_t N = st.N;
  const int64_t M = (int64_t)st.ctl->npair < st.pcap ? (int64_t)st.ctl->npair : st.pcap;
  Quad<S>* hist = (Quad<S>*)st.hist[nl];
  const uint32_t* cmask = st.cmask[nl];
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M;
       m += (int64_t)gridDim.x * blockDim.x) {
    const int4 pr = st.pairs[m];
    if ((cmask[pr.x] >> pr.y) & 1u)
      stq(hist + (int64_t)pr.w * N + pr.z, ldq(hist + (int64_t)pr.y * N + pr.x));
  }
}

// true when this block's bed has no rebuild pending (the whole block returns)
__device__ __forceinline__ bool ens_idle(const BedView* v) {
  return !v[blockIdx.y].st.ctl->need_rebuild;
}

__global__ void k_zero_bins_e(const BedView* v) {
  if (ens_idle(v)) return;
  const BedView& b = bed_view(v);
  zero_bins_body(b.st, b.P.nbins, false);
}
template <int FORM>
__global__ void k_bin_count_e(const BedView* v, int sub_off) {
  if (ens_idle(v)) return;
  const BedView& b = bed_view(v);
  bin_count_body<FORM>(b.st, b.P, sub_off, false);
}
__global__ void k_scan1_e(const BedView* v) {
  if (ens_idle(v)) return;
  const BedView& b = bed_view(v);
  if ((int64_t)blockIdx.x * kScanTile >= b.P.nbins) return;
  scan1_body(b.st, b.P.nbins, false);
}
__global__ void k_scan2_e(const BedView* v) {
  if (ens_idle(v)) return;
  const BedView& b = bed_view(v);
  scan2_body(b.st, (b.P.nbins + kScanTile - 1) / kScanTile, b.P.nbins, false);
}
__global__ void k_scan3_e(const BedView* v) {
  if (ens_idle(v)) return;
  const BedView& b = bed_view(v);
  if ((int64_t)blockIdx.x * kScanTile >= b.P.nbins) return;
  scan3_body(b.st, b.P.nbins, false);
}
__global__ void k_scatter_e(const BedView* v) {
  if (ens_idle(v)) return;
  const BedView& b = bed_view(v);
  scatter_body(b.st, false);
}
__global__ void k_sort_bins_e(const BedView* v) {
  if (ens_idle(v)) return;
  const BedView& b = bed_view(v);
  sort_bins_body(b.st, b.P.nbins, false);
}
template <int FORM>
__global__ void k_gather_e(const BedView* v, int sub_off) {
  if (ens_idle(v)) return;
  const BedView& b = bed_view(v);
  gather_body<FORM>(b.st, sub_off, false);
}
template <int FORM>
__global__ void k_build_e(const BedView* v, int sub_off) {
  if (ens_idle(v)) return;
  const BedView& b = bed_view(v);
  build_body<FORM>(b.st, b.P, sub_off, false);
}
template <int FORM>
__global__ void k_remap_e(const BedView* v) {
  if (ens_idle(v)) return;
  const BedView& b = bed_view(v);
  remap_body<FORM>(b.st, b.P, false);
}
// one thread per bed
__global__ void k_flip_e(const BedView* v, int B) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x)
    flip_body(v[b].st, false);
}

// Rebuild flags of every bed from its displacement; graph condition = any.
__global__ void k_check_e(const BedView* v, int B, cudaGraphConditionalHandle h, int use_cond) {
  int any = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    Ctl* c = v[b].st.ctl;
    const float hs = v[b].P.half_skin_f;
    const float m = __uint_as_float(c->disp_max_bits);
    const int need = (m > hs * hs) ? 1 : 0;
    c->need_rebuild = need;
    any |= need;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0 && use_cond) cudaGraphSetConditional(h, any ? 1u : 0u);
}

// Copy every bed's control block into one array (one read-back for all beds).
__global__ void k_ctl_gather_e(const BedView* v, int B, Ctl* out) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) out[b] = *v[b].st.ctl;
}

// every bed: rebuild at the next rebuild launch; and each bed's rebuild counter set
// (from / to a host-side table, so that the autotuner's rebuilds are not counted)
__global__ void k_force_need_e(const BedView* v, int B) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x)
    v[b].st.ctl->need_rebuild = 1;
}
__global__ void k_set_rebuilds_e(const BedView* v, int B, const int64_t* rebuilds) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x)
    v[b].st.ctl->rebuilds = rebuilds[b];
}

__global__ void k_advance_e(const BedView* v, int B, int n) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    Ctl* c = v[b].st.ctl;
    c->st = (c->st + n) & 1;
  }
}


inline unsigned grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 152 * 64) g = 152 * 64;
  return (unsigned)g;
}

// The pair list of the new lists (current = false: in a rebuild, before the flip) or
// of the current ones: counts, their scan, the pairs.
static void launch_pair_fill(const DevState& st, bool force, bool current, cudaStream_t s) {
  const int B = 256;
  const int64_t nblk = (st.N + kScanTile - 1) / kScanTile;
  k_pair_count<<<grid_for(st.N, B), B, 0, s>>>(st, force, current);
  k_pscan1<<<(unsigned)nblk, kScanThreads, 0, s>>>(st, force);
  k_pscan2<<<1, 1024, 0, s>>>(st, nblk, force);
  k_pscan3<<<(unsigned)nblk, kScanThreads, 0, s>>>(st, force);
  k_pair_fill<<<grid_for(st.N, B), B, 0, s>>>(st, force, current);
}

template <int FORM>
void rebuild_impl(const DevState& st, const DevParams& P, int sub_off, bool force, cudaStream_t s) {
  const int B = 256;
  const int64_t nblk = (P.nbins + kScanTile - 1) / kScanTile;
  if (force) k_force_need<<<1, 1, 0, s>>>(st.ctl);
  k_zero_bins<<<grid_for(P.nbins, B), B, 0, s>>>(st, P.nbins, false);
  k_bin_count<FORM><<<grid_for(st.N, B), B, 0, s>>>(st, P, sub_off, false);
  k_scan1<<<(unsigned)nblk, kScanThreads, 0, s>>>(st, P.nbins, false);
  k_scan2<<<1, 1024, 0, s>>>(st, nblk, P.nbins, false);
  k_scan3<<<(unsigned)nblk, kScanThreads, 0, s>>>(st, P.nbins, false);
  k_scatter<<<grid_for(st.N, B), B, 0, s>>>(st, false);
  k_sort_bins<<<grid_for(P.nbins, B), B, 0, s>>>(st, P.nbins, false);
  k_gather<FORM><<<grid_for(st.N, B), B, 0, s>>>(st, sub_off, false);
  k_build<FORM><<<grid_for(st.N, 128), 128, 0, s>>>(st, P, sub_off, false);
  k_remap<FORM><<<grid_for(st.N, B), B, 0, s>>>(st, P, force);
  if (st.pairs) launch_pair_fill(st, false, false, s);
  k_flip<<<1, 1, 0, s>>>(st, false);
}

template <int FORM>
void rebuild_ens_impl(const EnsLaunch& e, int sub_off, cudaStream_t s) {
  const int B = 256;
  const unsigned gy = (unsigned)e.B;
  auto per_bed = [](int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 64) g = 64;  // grid-stride loops cover larger beds
    return (unsigned)g;
  };
  const unsigned gn = per_bed(e.max_n, B), gb = per_bed(e.max_bins, B);
  const unsigned tiles = (unsigned)((e.max_bins + kScanTile - 1) / kScanTile);
  k_zero_bins_e<<<dim3(gb, gy), B, 0, s>>>(e.views);
  k_bin_count_e<FORM><<<dim3(gn, gy), B, 0, s>>>(e.views, sub_off);
  k_scan1_e<<<dim3(tiles, gy), kScanThreads, 0, s>>>(e.views);
  k_scan2_e<<<dim3(1, gy), 1024, 0, s>>>(e.views);
  k_scan3_e<<<dim3(tiles, gy), kScanThreads, 0, s>>>(e.views);
  k_scatter_e<<<dim3(gn, gy), B, 0, s>>>(e.views);
  k_sort_bins_e<<<dim3(gb, gy), B, 0, s>>>(e.views);
  k_gather_e<FORM><<<dim3(gn, gy), B, 0, s>>>(e.views, sub_off);
  k_build_e<FORM><<<dim3(per_bed(e.max_n, 128), gy), 128, 0, s>>>(e.views, sub_off);
  k_remap_e<FORM><<<dim3(gn, gy), B, 0, s>>>(e.views);
  k_flip_e<<<(e.B + 255) / 256, 256, 0, s>>>(e.views, e.B);
}

}  // namespace

void launch_rebuild(int form, const DevState& st, const DevParams& P, int sub_off, bool force,
                    cudaStream_t s) {
  switch (form) {
    case FORM_SPLIT: rebuild_impl<FORM_SPLIT>(st, P, sub_off, force, s); break;
    case FORM_PLAIN: rebuild_impl<FORM_PLAIN>(st, P, sub_off, force, s); break;
    default: rebuild_impl<FORM_FP64>(st, P, sub_off, force, s); break;
  }
}

void launch_rebuild_now(int form, const DevState& st, const DevParams& P, cudaStream_t s) {
  k_force_need<<<1, 1, 0, s>>>(st.ctl);
  launch_rebuild(form, st, P, 0, false, s);
}

void launch_pair_list(const DevState& st, const DevParams& P, cudaStream_t s) {
  if (st.pairs) launch_pair_fill(st, true, true, s);
}

void launch_spring_sync(int form, const DevState& st, cudaStream_t s) {
  if (!st.pairs) return;
  const unsigned g = grid_for(st.pcap, 256);
  if (form == FORM_SPLIT) k_spring_sync<FORM_SPLIT><<<g, 256, 0, s>>>(st);
  else if (form == FORM_PLAIN) k_spring_sync<FORM_PLAIN><<<g, 256, 0, s>>>(st);
}

void launch_check(const DevState& st, const DevParams& P, unsigned long long cond_handle,
                  int use_cond, cudaStream_t s) {
  float hs = P.half_skin_f;
  k_check<<<1, 1, 0, s>>>(st.ctl, hs * hs, (cudaGraphConditionalHandle)cond_handle, use_cond);
}

void launch_advance_parity(const DevState& st, int n, cudaStream_t s) {
  if (n & 1) k_advance<<<1, 1, 0, s>>>(st.ctl, n);
}

void launch_check_ens(const EnsLaunch& e, unsigned long long cond_handle, int use_cond,
                      cudaStream_t s) {
  k_check_e<<<1, 1024, 0, s>>>(e.views, e.B, (cudaGraphConditionalHandle)cond_handle, use_cond);
}

void launch_rebuild_ens(int form, const EnsLaunch& e, int sub_off, cudaStream_t s) {
  switch (form) {
    case FORM_SPLIT: rebuild_ens_impl<FORM_SPLIT>(e, sub_off, s); break;
    case FORM_PLAIN: rebuild_ens_impl<FORM_PLAIN>(e, sub_off, s); break;
    default: rebuild_ens_impl<FORM_FP64>(e, sub_off, s); break;
  }
}

void launch_ctl_gather_ens(const EnsLaunch& e, Ctl* out, cudaStream_t s) {
  k_ctl_gather_e<<<(e.B + 127) / 128, 128, 0, s>>>(e.views, e.B, out);
}

void launch_force_need_ens(const EnsLaunch& e, cudaStream_t s) {
  k_force_need_e<<<(e.B + 127) / 128, 128, 0, s>>>(e.views, e.B);
}

void launch_set_rebuilds_ens(const EnsLaunch& e, const int64_t* rebuilds, cudaStream_t s) {
  k_set_rebuilds_e<<<(e.B + 127) / 128, 128, 0, s>>>(e.views, e.B, rebuilds);
}

void launch_advance_ens(const EnsLaunch& e, int n, cudaStream_t s) {
  if (n & 1) k_advance_e<<<(e.B + 255) / 256, 256, 0, s>>>(e.views, e.B, n);
}


// ---------------------------------------------------------------- import/export

namespace {

template <class S>
__device__ __forceinline__ S s_from_double(double x);
template <>
__device__ __forceinline__ float s_from_double<float>(double x) {
  return __double2float_rn(x);
}
template <>
__device__ __forceinline__ double s_from_double<double>(double x) {
  return x;
}
template <>
__device__ __forceinline__ dd s_from_double<dd>(double x) {
  return dd_from_double(x);
}

template <int FORM>
__global__ void k_import(DevState st, const double* x, const double* v, const double* w,
                         const double* d, const double* rho, double pi6, double vc) {
  using S = typename Traits<FORM>::S;
  using F = typename Traits<FORM>::F;
  const int sb = st.ctl->st, pb = st.ctl->pb;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < st.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double di = d[i];
    const double r = 0.5 * di;
    const double Vp = __dmul_rn(__dmul_rn(__dmul_rn(pi6, di), di), di);
    const double m = __dmul_rn(rho[i], Vp);
    Quad<S> p{s_from_double<S>(x[3 * i]), s_from_double<S>(x[3 * i + 1]),
              s_from_double<S>(x[3 * i + 2]), s_from_double<S>(r)};
    stq((Quad<S>*)st.pos[sb] + i, p);
    stq((Quad<S>*)st.vel[sb] + i,
        Quad<S>{s_from_double<S>(v ? v[3 * i] : 0.0), s_from_double<S>(v ? v[3 * i + 1] : 0.0),
                s_from_double<S>(v ? v[3 * i + 2] : 0.0), s_from_double<S>(m)});
    stq((Quad<S>*)st.omg[sb] + i,
        Quad<S>{s_from_double<S>(w ? w[3 * i] : 0.0), s_from_double<S>(w ? w[3 * i + 1] : 0.0),
                s_from_double<S>(w ? w[3 * i + 2] : 0.0), S{}});
    stq((Quad<F>*)st.acc[pb] + i, Quad<F>{F(0), F(0), F(0), F(0)});
    st.uid[pb][i] = (int32_t)i;
    st.r64[pb][i] = r;
    st.vfrac[pb][i] = __ddiv_rn(Vp, vc);
    st.wmask[pb][i] = 0u;
    st.xb[pb][i] = make_float4((float)x[3 * i], (float)x[3 * i + 1], (float)x[3 * i + 2], 0.0f);
  }
}

// what: 0 x, 1 v, 2 omega, 3 a_prev
template <int FORM>
__global__ void k_export(DevState st, int what, double* out) {
  using S = typename Traits<FORM>::S;
  using F = typename Traits<FORM>::F;
  const int sb = st.ctl->st, pb = st.ctl->pb;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < st.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = st.uid[pb][i];
    double a, b, c;
    if (what == 3) {
      Quad<F> q = ldq((const Quad<F>*)st.acc[pb] + i);
      a = (double)q.a; b = (double)q.b; c = (double)q.c;
    } else {
      const void* base = what == 0 ? st.pos[sb] : (what == 1 ? st.vel[sb] : st.omg[sb]);
      Quad<S> q = ldq((const Quad<S>*)base + i);
      a = Num<S>::d(q.a); b = Num<S>::d(q.b); c = Num<S>::d(q.c);
    }
    out[3 * u] = a;
    out[3 * u + 1] = b;
    out[3 * u + 2] = c;
  }
}

__global__ void k_nbr_counts(DevState st, int64_t* counts) {
  const int pb = st.ctl->pb, nl = st.ctl->nl;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < st.N;
       i += (int64_t)gridDim.x * blockDim.x)
    counts[st.uid[pb][i]] = st.nn[nl][i];
}

__global__ void k_nbr_fill(DevState st, const int64_t* offsets, int64_t* out) {
  const int pb = st.ctl->pb, nl = st.ctl->nl;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < st.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = st.uid[pb][i];
    int64_t* o = out + offsets[u];
    const int n = st.nn[nl][i];
    for (int k = 0; k < n; ++k) {
      int64_t v = st.uid[pb][nbr_index(st.nbr[nl][(int64_t)k * st.N + i])];
      int c = k - 1;
      while (c >= 0 && o[c] > v) {
        o[c + 1] = o[c];
        --c;
      }
      o[c + 1] = v;
    }
  }
}

template <int FORM>
__global__ void k_contacts(DevState st, DevParams P, unsigned long long* count, int64_t cap,
                           int64_t* ij, double* xi) {
  using S = typename Traits<FORM>::S;
  const int pb = st.ctl->pb, nl = st.ctl->nl;
  const Quad<S>* hist = (const Quad<S>*)st.hist[nl];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < st.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t m = st.cmask[nl][i];
    if (!m) continue;
    const int32_t ui = st.uid[pb][i];
    const int n = st.nn[nl][i];
    for (int k = 0; k < n; ++k) {
      if (!((m >> k) & 1u)) continue;
      const int32_t uj = st.uid[pb][nbr_index(st.nbr[nl][(int64_t)k * st.N + i])];
      if (uj < ui) continue;
      unsigned long long slot = atomicAdd(count, 1ull);
      if ((int64_t)slot >= cap) continue;
      ij[2 * slot] = ui;
      ij[2 * slot + 1] = uj;
      const Quad<S> h = ldq(hist + (int64_t)k * st.N + i);
      xi[3 * slot + 0] = Num<S>::d(h.a);
      xi[3 * slot + 1] = Num<S>::d(h.b);
      xi[3 * slot + 2] = Num<S>::d(h.c);
    }
  }
}

// Springs of the pairs (ij[2k] < ij[2k+1], caller indices, sorted) set as the current
// history: every listed slot whose pair is in the table takes its spring (both
// particles' slots hold the same vector, as the pair evaluation keeps them); the
// other slots have none.
template <int FORM>
__global__ void k_springs_in(DevState st, int64_t m, const int64_t* ij, const double* xi) {
  using S = typename Traits<FORM>::S;
  const int pb = st.ctl->pb, nl = st.ctl->nl;
  Quad<S>* hist = (Quad<S>*)st.hist[nl];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < st.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ui = st.uid[pb][i];
    const int n = st.nn[nl][i];
    uint32_t mask = 0;
    for (int k = 0; k < n; ++k) {
      const int64_t uj = st.uid[pb][nbr_index(st.nbr[nl][(int64_t)k * st.N + i])];
      const int64_t a = ui < uj ? ui : uj, b = ui < uj ? uj : ui;
      int64_t lo = 0, hi = m;  // first entry >= (a, b)
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int64_t ma = ij[2 * mid], mb = ij[2 * mid + 1];
        if (ma < a || (ma == a && mb < b)) lo = mid + 1;
        else hi = mid;
      }
      if (lo < m && ij[2 * lo] == a && ij[2 * lo + 1] == b) {
        stq(hist + (int64_t)k * st.N + i,
            Quad<S>{s_from_double<S>(xi[3 * lo]), s_from_double<S>(xi[3 * lo + 1]),
                    s_from_double<S>(xi[3 * lo + 2]), S{}});
        mask |= 1u << k;
      }
    }
    st.cmask[nl][i] = mask;
  }
}

// Lagged accelerations (caller order, n x 3).
template <int FORM>
__global__ void k_accel_in(DevState st, const double* a) {
  using F = typename Traits<FORM>::F;
  const int pb = st.ctl->pb;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < st.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = st.uid[pb][i];
    stq((Quad<F>*)st.acc[pb] + i, Quad<F>{(F)a[3 * u], (F)a[3 * u + 1], (F)a[3 * u + 2], F(0)});
  }
}

// Wall springs, caller order [n][6 walls][3]; a wall whose spring is zero has none.
template <int FORM>
__global__ void k_wall_springs(DevState st, double* out, const double* in) {
  using S = typename Traits<FORM>::S;
  const int pb = st.ctl->pb;
  S* wh = (S*)st.whist[pb];
  const int64_t N = st.N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = st.uid[pb][i];
    if (out) {
      const uint32_t m = st.wmask[pb][i];
      for (int w = 0; w < 6; ++w)
        for (int c = 0; c < 3; ++c)
          out[18 * u + 3 * w + c] = ((m >> w) & 1u) ? Num<S>::d(wh[((int64_t)w * 3 + c) * N + i]) : 0.0;
    } else {
      uint32_t m = 0;
      for (int w = 0; w < 6; ++w) {
        bool any = false;
        for (int c = 0; c < 3; ++c) {
          const double v = in[18 * u + 3 * w + c];
          wh[((int64_t)w * 3 + c) * N + i] = s_from_double<S>(v);
          any |= v != 0.0;
        }
        if (any) m |= 1u << w;
      }
      st.wmask[pb][i] = m;
    }
  }
}

}  // namespace

void launch_springs_in(int form, const DevState& st, int64_t m, const int64_t* ij, const double* xi,
                       cudaStream_t s) {
  unsigned g = grid_for(st.N, 256);
  switch (form) {
    case FORM_SPLIT: k_springs_in<FORM_SPLIT><<<g, 256, 0, s>>>(st, m, ij, xi); break;
    case FORM_PLAIN: k_springs_in<FORM_PLAIN><<<g, 256, 0, s>>>(st, m, ij, xi); break;
    default: k_springs_in<FORM_FP64><<<g, 256, 0, s>>>(st, m, ij, xi); break;
  }
}

void launch_accel_in(int form, const DevState& st, const double* a, cudaStream_t s) {
  unsigned g = grid_for(st.N, 256);
  switch (form) {
    case FORM_SPLIT: k_accel_in<FORM_SPLIT><<<g, 256, 0, s>>>(st, a); break;
    case FORM_PLAIN: k_accel_in<FORM_PLAIN><<<g, 256, 0, s>>>(st, a); break;
    default: k_accel_in<FORM_FP64><<<g, 256, 0, s>>>(st, a); break;
  }
}

void launch_wall_springs(int form, const DevState& st, double* out, const double* in, cudaStream_t s) {
  unsigned g = grid_for(st.N, 256);
  switch (form) {
    case FORM_SPLIT: k_wall_springs<FORM_SPLIT><<<g, 256, 0, s>>>(st, out, in); break;
    case FORM_PLAIN: k_wall_springs<FORM_PLAIN><<<g, 256, 0, s>>>(st, out, in); break;
    default: k_wall_springs<FORM_FP64><<<g, 256, 0, s>>>(st, out, in); break;
  }
}

void launch_import(int form, const DevState& st, const double* x, const double* v, const double* w,
                   const double* d, const double* rho, const DevParams& P, cudaStream_t s) {
  const double pi6 = 3.14159265358979323846 / 6.0;
  unsigned g = grid_for(st.N, 256);
  // a graded mesh keeps V_p itself (the deposition divides by the cell's volume)
  const double vc = P.graded ? 1.0 : P.vc;
  switch (form) {
    case FORM_SPLIT: k_import<FORM_SPLIT><<<g, 256, 0, s>>>(st, x, v, w, d, rho, pi6, vc); break;
    case FORM_PLAIN: k_import<FORM_PLAIN><<<g, 256, 0, s>>>(st, x, v, w, d, rho, pi6, vc); break;
    default: k_import<FORM_FP64><<<g, 256, 0, s>>>(st, x, v, w, d, rho, pi6, vc); break;
  }
}

void launch_export(int form, const DevState& st, int what, double* out, cudaStream_t s) {
  unsigned g = grid_for(st.N, 256);
  switch (form) {
    case FORM_SPLIT: k_export<FORM_SPLIT><<<g, 256, 0, s>>>(st, what, out); break;
    case FORM_PLAIN: k_export<FORM_PLAIN><<<g, 256, 0, s>>>(st, what, out); break;
    default: k_export<FORM_FP64><<<g, 256, 0, s>>>(st, what, out); break;
  }
}

void launch_neighbors_export(const DevState& st, int64_t* counts, cudaStream_t s) {
  k_nbr_counts<<<grid_for(st.N, 256), 256, 0, s>>>(st, counts);
}

void launch_neighbors_fill(const DevState& st, const int64_t* offsets, int64_t* out,
                           cudaStream_t s) {
  k_nbr_fill<<<grid_for(st.N, 256), 256, 0, s>>>(st, offsets, out);
}

void launch_contacts_export(int form, const DevState& st, const DevParams& P,
                            unsigned long long* count, int64_t cap, int64_t* ij, double* xi,
                            cudaStream_t s) {
  unsigned g = grid_for(st.N, 256);
  switch (form) {
    case FORM_SPLIT: k_contacts<FORM_SPLIT><<<g, 256, 0, s>>>(st, P, count, cap, ij, xi); break;
    case FORM_PLAIN: k_contacts<FORM_PLAIN><<<g, 256, 0, s>>>(st, P, count, cap, ij, xi); break;
    default: k_contacts<FORM_FP64><<<g, 256, 0, s>>>(st, P, count, cap, ij, xi); break;
  }
}

}  // namespace sedi
