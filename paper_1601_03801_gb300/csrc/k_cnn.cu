// Learned warm start of the smoothing solve: a 3-layer 3x3x3 convolutional network
// 4 -> 32 -> 32 -> 4 (ReLU after the first two) on the averaging mesh, trained on
// the GPU by these kernels.  Weights and activations are stored in bfloat16,
// products accumulate in FP32.  Fields are channels-last [voxel][channel]; a tap
// outside the mesh wraps on periodic axes and reads zero otherwise.
//
// Parameter order (shared with the FP64 reference network of the tests):
//   w1[32][4][27] b1[32] w2[32][32][27] b2[32] w3[4][32][27] b3[4],
//   tap t = (kz*3 + ky)*3 + kx at offset (kx-1, ky-1, kz-1).
// Backward: data gradients are the same convolutions with mirrored taps and
// transposed weights; weight gradients are per-tap voxel sums (per-block partials
// reduced in a fixed order); loss = mean (y - target)^2; Adam on FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace sedi {

namespace {

struct Grid3 {
  int nx, ny, nz;
  int per[3];
  int64_t n;
};

__device__ __forceinline__ int64_t nb_of(const Grid3& g, int x, int y, int z, int dx, int dy, int dz) {
  int c[3] = {x + dx, y + dy, z + dz};
  const int n[3] = {g.nx, g.ny, g.nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (c[a] < 0) {
      if (!g.per[a]) return -1;
      c[a] += n[a];
    } else if (c[a] >= n[a]) {
      if (!g.per[a]) return -1;
      c[a] -= n[a];
    }
  }
  return ((int64_t)c[2] * g.ny + c[1]) * g.nx + c[0];
}

template <class T>
__device__ __forceinline__ float ld_in(const T* p);
template <>
__device__ __forceinline__ float ld_in<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <>
__device__ __forceinline__ float ld_in<float>(const float* p) {
  return *p;
}

// out[v][co] = b[co] + sum_t sum_ci w[t][ci][co] in[v + s*off(t)][ci]   (s = +1, or -1
// for the data gradient).  Optional ReLU, optional multiplication by the mask
// (mask[v][co] > 0) of a forward activation, output in bf16 or FP32.
template <int CIN, int COUT, class TIN, bool RELU, bool OUT_BF16>
__global__ void __launch_bounds__(128) k_conv(const TIN* in, const float* wt, const float* bias,
                                               void* out, const __nv_bfloat16* mask, Grid3 g,
                                               int sign) {
  extern __shared__ float sw[];  // [27][CIN][COUT] then bias[COUT]
  const int nw = 27 * CIN * COUT;
  for (int k = threadIdx.x; k < nw + COUT; k += blockDim.x) sw[k] = k < nw ? wt[k] : (bias ? bias[k - nw] : 0.0f);
  __syncthreads();
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.n) return;
  const int x = (int)(v % g.nx);
  const int y = (int)((v / g.nx) % g.ny);
  const int z = (int)(v / ((int64_t)g.nx * g.ny));
  float acc[COUT];
#pragma unroll
  for (int co = 0; co < COUT; ++co) acc[co] = sw[nw + co];
  for (int t = 0; t < 27; ++t) {
    const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
    const int64_t q = nb_of(g, x, y, z, sign * dx, sign * dy, sign * dz);
    if (q < 0) continue;
    const TIN* src = in + q * CIN;
    const float* wtap = sw + t * CIN * COUT;
#pragma unroll 4
    for (int ci = 0; ci < CIN; ++ci) {
      const float xv = ld_in<TIN>(src + ci);
#pragma unroll
      for (int co = 0; co < COUT; ++co) acc[co] = fmaf(wtap[ci * COUT + co], xv, acc[co]);
    }
  }
#pragma unroll
  for (int co = 0; co < COUT; ++co) {
    float r = acc[co];
    if (RELU) r = r > 0.0f ? r : 0.0f;
    if (mask && !(__bfloat162float(mask[v * COUT + co]) > 0.0f)) r = 0.0f;
    if (OUT_BF16) ((__nv_bfloat16*)out)[v * COUT + co] = __float2bfloat16_rn(r);
    else ((float*)out)[v * COUT + co] = r;
  }
}

// Weight gradient of one layer.  Grid (kWgBlocks, 27): block (b, t) sums over its
// share of the voxels, staged 128 at a time in shared memory, with each thread
// holding a few (co, ci) entries in registers; per-block partials go to
// part[b][t][co*CIN + ci] (and part_b[b][co] for the bias) and are summed in a fixed
// order by k_wgrad_reduce, so the gradient is deterministic.
//   dw[co][ci][t] = sum_v dout[v][co] in[v + off(t)][ci],  db[co] = sum_v dout[v][co]
constexpr int kWgBlocks = 64;

template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_wgrad(const __nv_bfloat16* in, const float* dout,
                                                float* part, float* part_b, Grid3 g) {
  constexpr int V = 128;
  constexpr int E = COUT * CIN;
  constexpr int PER = (E + 255) / 256;
  __shared__ float sd[V][COUT];
  __shared__ float si[V][CIN + 1];
  const int t = blockIdx.y;
  const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
  const int64_t per_block = (g.n + gridDim.x - 1) / gridDim.x;
  const int64_t vbeg = (int64_t)blockIdx.x * per_block;
  const int64_t vend = vbeg + per_block < g.n ? vbeg + per_block : g.n;
  float acc[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) acc[k] = 0.0f;
  float bacc = 0.0f;
  for (int64_t v0 = vbeg; v0 < vend; v0 += V) {
    __syncthreads();
    for (int k = threadIdx.x; k < V * COUT; k += blockDim.x) {
      const int64_t v = v0 + k / COUT;
      sd[k / COUT][k % COUT] = v < vend ? dout[v * COUT + k % COUT] : 0.0f;
    }
    for (int k = threadIdx.x; k < V * CIN; k += blockDim.x) {
      const int64_t v = v0 + k / CIN;
      float val = 0.0f;
      if (v < vend) {
        const int x = (int)(v % g.nx), y = (int)((v / g.nx) % g.ny), z = (int)(v / ((int64_t)g.nx * g.ny));
        const int64_t q = nb_of(g, x, y, z, dx, dy, dz);
        if (q >= 0) val = __bfloat162float(in[q * CIN + k % CIN]);
      }
      si[k / CIN][k % CIN] = val;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = threadIdx.x + k * 256;
      if (e < E) {
        const int co = e / CIN, ci = e % CIN;
        float s = acc[k];
        for (int v = 0; v < V; ++v) s = fmaf(sd[v][co], si[v][ci], s);
        acc[k] = s;
      }
    }
    if (t == 0 && threadIdx.x < COUT)
      for (int v = 0; v < V; ++v) bacc += sd[v][threadIdx.x];
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int e = threadIdx.x + k * 256;
    if (e < E) part[((int64_t)blockIdx.x * 27 + t) * E + e] = acc[k];
  }
  if (t == 0 && threadIdx.x < COUT) part_b[blockIdx.x * COUT + threadIdx.x] = bacc;
}

template <int CIN, int COUT>
__global__ void k_wgrad_reduce(const float* part, const float* part_b, float* dw, float* db) {
  constexpr int E = COUT * CIN;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 27 * E + COUT; k += gridDim.x * blockDim.x) {
    float s = 0.0f;
    if (k < 27 * E) {
      const int t = k / E, e = k % E;
      for (int b = 0; b < kWgBlocks; ++b) s += part[((int64_t)b * 27 + t) * E + e];
      const int co = e / CIN, ci = e % CIN;
      dw[((int64_t)co * CIN + ci) * 27 + t] = s;
    } else {
      const int co = k - 27 * E;
      for (int b = 0; b < kWgBlocks; ++b) s += part_b[b * COUT + co];
      db[co] = s;
    }
  }
}

// [O][I][27] (master layout) -> [27][I][O] forward taps, or [27][O][I] for the
// data gradient, each value rounded to bfloat16.
__global__ void k_pack(const float* w, float* fwd, float* bwd, int O, int I) {
  const int n = O * I * 27;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int o = k / (I * 27), i = (k / 27) % I, t = k % 27;
    const float r = __bfloat162float(__float2bfloat16_rn(w[k]));
    fwd[((int64_t)t * I + i) * O + o] = r;
    bwd[((int64_t)t * O + o) * I + i] = r;
  }
}

__global__ void k_round_bias(const float* b, float* out, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    out[k] = __bfloat162float(__float2bfloat16_rn(b[k]));
}

// y [v][4] FP32 vs target [v][4]: gradient 2 (y - t) / (4 N) and per-block loss sums
__global__ void k_mse(const float* y, const float* tgt, float* g, double* loss, int64_t n4) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n4; k += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[k] - tgt[k];
    g[k] = 2.0f * d / (float)n4;
    s += (double)d * (double)d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / (double)n4);
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.0f - b1) * gk;
    const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  }
}

// [C][4] channels-first FP64 field rows -> [v][4] bf16 network input, x / scale
__global__ void k_to_input(const double* f0, const double* f1, const double* f2, const double* f3,
                           float s0, float s1, float s2, float s3, __nv_bfloat16* x, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    x[4 * v + 0] = __float2bfloat16_rn((float)f0[v] / s0);
    x[4 * v + 1] = __float2bfloat16_rn((float)f1[v] / s1);
    x[4 * v + 2] = __float2bfloat16_rn((float)f2[v] / s2);
    x[4 * v + 3] = __float2bfloat16_rn((float)f3[v] / s3);
  }
}

int64_t blocks(int64_t n, int b) { return (n + b - 1) / b; }

}  // namespace

// Offsets of the packed parameter vector.
constexpr int kW1 = 0, kB1 = 32 * 4 * 27, kW2 = kB1 + 32, kB2 = kW2 + 32 * 32 * 27,
              kW3 = kB2 + 32, kB3 = kW3 + 4 * 32 * 27, kNP = kB3 + 4;

size_t cnn_param_count() { return kNP; }

size_t cnn_work_bytes(int64_t n) {
  // x(bf16x4) a1,a2(bf16x32) y(f32x4) g_y(f32x4) g2,g1(f32x32) + packed weights
  return (size_t)n * (8 + 64 + 64 + 16 + 16 + 128 + 128) + 8 * kNP * sizeof(float) + 1024 +
         27 * 32 * 32 * 2 + (size_t)kWgBlocks * (27 * 1024 + 32) * 4 + 1024;
}

struct CnnBufs {
  __nv_bfloat16 *x, *a1, *a2;
  float *y, *gy, *g2, *g1;
  float *wf1, *wb1, *wf2, *wb2, *wf3, *wb3, *bias_r;
  __nv_bfloat16* w2mma;  // [27][32][32] layer-2 weights for the tensor-core kernel
  float* wpart;          // [kWgBlocks][27][1024] weight-gradient partials
  float* bpart;          // [kWgBlocks][32] bias-gradient partials
};

static CnnBufs carve(void* work, int64_t n) {
  char* p = (char*)work;
  CnnBufs b;
  b.x = (__nv_bfloat16*)p; p += n * 8;
  b.a1 = (__nv_bfloat16*)p; p += n * 64;
  b.a2 = (__nv_bfloat16*)p; p += n * 64;
  b.y = (float*)p; p += n * 16;
  b.gy = (float*)p; p += n * 16;
  b.g2 = (float*)p; p += n * 128;
  b.g1 = (float*)p; p += n * 128;
  b.wf1 = (float*)p; p += 32 * 4 * 27 * 4;
  b.wb1 = (float*)p; p += 32 * 4 * 27 * 4;
  b.wf2 = (float*)p; p += 32 * 32 * 27 * 4;
  b.wb2 = (float*)p; p += 32 * 32 * 27 * 4;
  b.wf3 = (float*)p; p += 4 * 32 * 27 * 4;
  b.wb3 = (float*)p; p += 4 * 32 * 27 * 4;
  b.bias_r = (float*)p; p += 128 * 4;
  b.w2mma = (__nv_bfloat16*)p; p += 27 * 32 * 32 * 2;
  b.wpart = (float*)p; p += (size_t)kWgBlocks * 27 * 1024 * 4;
  b.bpart = (float*)p;
  return b;
}

static Grid3 grid_of(const DevParams& P) {
  Grid3 g;
  g.nx = P.nc[0];
  g.ny = P.nc[1];
  g.nz = P.nc[2];
  for (int a = 0; a < 3; ++a) g.per[a] = P.periodic[a];
  g.n = P.C;
  return g;
}

template <int CIN, int COUT, class TIN, bool RELU, bool OUT_BF16>
static void conv(const TIN* in, const float* w, const float* b, void* out,
                 const __nv_bfloat16* mask, const Grid3& g, int sign, cudaStream_t s) {
  const size_t smem = (27 * CIN * COUT + COUT) * sizeof(float);
  cudaFuncSetAttribute(k_conv<CIN, COUT, TIN, RELU, OUT_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  k_conv<CIN, COUT, TIN, RELU, OUT_BF16><<<(unsigned)blocks(g.n, 128), 128, smem, s>>>(
      in, w, b, out, mask, g, sign);
}

// Pack the bf16-rounded compute copies of the master weights.
static void pack(const float* master, CnnBufs& b, cudaStream_t s) {
  k_pack<<<64, 256, 0, s>>>(master + kW1, b.wf1, b.wb1, 32, 4);
  k_pack<<<256, 256, 0, s>>>(master + kW2, b.wf2, b.wb2, 32, 32);
  k_pack<<<64, 256, 0, s>>>(master + kW3, b.wf3, b.wb3, 4, 32);
  k_round_bias<<<1, 64, 0, s>>>(master + kB1, b.bias_r, 32);
  k_round_bias<<<1, 64, 0, s>>>(master + kB2, b.bias_r + 32, 32);
  k_round_bias<<<1, 64, 0, s>>>(master + kB3, b.bias_r + 64, 4);
}

void conv2_tensor(const float* master_w2, __nv_bfloat16* wbuf, const __nv_bfloat16* in,
                  const float* bias, __nv_bfloat16* out, int nx, int ny, int nz, const int* per,
                  int64_t n, cudaStream_t s);

static void forward(CnnBufs& b, const Grid3& g, const float* master, cudaStream_t s) {
  conv<4, 32, __nv_bfloat16, true, true>(b.x, b.wf1, b.bias_r, b.a1, nullptr, g, 1, s);
  conv2_tensor(master + kW2, b.w2mma, b.a1, b.bias_r + 32, b.a2, g.nx, g.ny, g.nz, g.per, g.n, s);
  conv<32, 4, __nv_bfloat16, false, false>(b.a2, b.wf3, b.bias_r + 64, b.y, nullptr, g, 1, s);
}

void cnn_input(const DevParams& P, const double* const f[4], const float scale[4], void* work,
               cudaStream_t s) {
  CnnBufs b = carve(work, P.C);
  k_to_input<<<(unsigned)std::min<int64_t>(blocks(P.C, 256), 4096), 256, 0, s>>>(
      f[0], f[1], f[2], f[3], scale[0], scale[1], scale[2], scale[3], b.x, P.C);
}

void cnn_forward(const DevParams& P, const float* master, void* work, float** y_out,
                 cudaStream_t s) {
  CnnBufs b = carve(work, P.C);
  const Grid3 g = grid_of(P);
  pack(master, b, s);
  forward(b, g, master, s);
  *y_out = b.y;
}

void cnn_loss_grad(const DevParams& P, const float* master, const float* target, float* grad,
                   double* loss, void* work, cudaStream_t s) {
  CnnBufs b = carve(work, P.C);
  const Grid3 g = grid_of(P);
  pack(master, b, s);
  forward(b, g, master, s);
  cudaMemsetAsync(grad, 0, kNP * sizeof(float), s);
  cudaMemsetAsync(loss, 0, sizeof(double), s);
  k_mse<<<(unsigned)std::min<int64_t>(blocks(4 * P.C, 256), 1024), 256, 0, s>>>(b.y, target, b.gy, loss, 4 * P.C);
  const dim3 wg(kWgBlocks, 27);
  // layer 3
  k_wgrad<32, 4><<<wg, 256, 0, s>>>(b.a2, b.gy, b.wpart, b.bpart, g);
  k_wgrad_reduce<32, 4><<<16, 256, 0, s>>>(b.wpart, b.bpart, grad + kW3, grad + kB3);
  conv<4, 32, float, false, false>(b.gy, b.wb3, nullptr, b.g2, b.a2, g, -1, s);
  // layer 2
  k_wgrad<32, 32><<<wg, 256, 0, s>>>(b.a1, b.g2, b.wpart, b.bpart, g);
  k_wgrad_reduce<32, 32><<<128, 256, 0, s>>>(b.wpart, b.bpart, grad + kW2, grad + kB2);
  conv<32, 32, float, false, false>(b.g2, b.wb2, nullptr, b.g1, b.a1, g, -1, s);
  // layer 1
  k_wgrad<4, 32><<<wg, 256, 0, s>>>(b.x, b.g1, b.wpart, b.bpart, g);
  k_wgrad_reduce<4, 32><<<16, 256, 0, s>>>(b.wpart, b.bpart, grad + kW1, grad + kB1);
}

void cnn_adam(float* master, const float* grad, float* m, float* v, int64_t t, float lr,
              cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  k_adam<<<64, 256, 0, s>>>(master, grad, m, v, kNP, lr, b1, b2, 1e-8f, c1, c2);
}

}  // namespace sedi

namespace sedi {

namespace {

__global__ void k_chan_first_to_vec(const double* in, float* out, int64_t n, int nc) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < nc; ++c) out[v * nc + c] = (float)in[c * n + v];
}

__global__ void k_vec_to_chan_first(const float* in, double* out, int64_t n, int nc) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < nc; ++c) out[c * n + v] = (double)in[v * nc + c];
}

template <class T>
__device__ __forceinline__ T t_add_f(T a, float b);
template <>
__device__ __forceinline__ double t_add_f<double>(double a, float b) { return a + (double)b; }
template <>
__device__ __forceinline__ float t_add_f<float>(float a, float b) { return a + b; }
template <>
__device__ __forceinline__ dd t_add_f<dd>(dd a, float b) { return dd_add_f(a, b); }

template <class T>
__device__ __forceinline__ float t_f(T a);
template <>
__device__ __forceinline__ float t_f<double>(double a) { return (float)a; }
template <>
__device__ __forceinline__ float t_f<float>(float a) { return a; }
template <>
__device__ __forceinline__ float t_f<dd>(dd a) { return a.hi; }

template <class T>
__device__ __forceinline__ T t_scale(T a, float s);
template <>
__device__ __forceinline__ double t_scale<double>(double a, float s) { return a * (double)s; }
template <>
__device__ __forceinline__ float t_scale<float>(float a, float s) { return a * s; }
template <>
__device__ __forceinline__ dd t_scale<dd>(dd a, float s) { return dd_mul_f(a, s); }

// guess = phi + scale_c * y_c on (eps, F_x, F_y, F_z) = fields (0, 4, 5, 6); the
// momentum fields eps*U (1, 2, 3) follow the predicted change of eps at fixed
// particle velocity: (eps U)^guess = (eps U)^m * eps^guess / eps^m.
template <class T>
__global__ void k_guess(const T* phi, const float* y, float s0, float s1, float s2, float s3,
                        T* guess, int64_t C) {
  const float sc[4] = {s0, s1, s2, s3};
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < C; v += (int64_t)gridDim.x * blockDim.x) {
    const T e = phi[v];
    const T eg = t_add_f<T>(e, sc[0] * y[v * 4]);
    guess[v] = eg;
    const float ef = t_f<T>(e);
    const float ratio = ef > 1e-9f ? t_f<T>(eg) / ef : 1.0f;
    for (int f = 1; f < 4; ++f) guess[f * C + v] = t_scale<T>(phi[f * C + v], ratio);
    for (int f = 4; f < 7; ++f) guess[f * C + v] = t_add_f<T>(phi[f * C + v], sc[f - 3] * y[v * 4 + f - 3]);
  }
}

}  // namespace

void cnn_chan_first_to_vec(const double* in, float* out, int64_t n, int nc, cudaStream_t s) {
  k_chan_first_to_vec<<<(unsigned)std::min<int64_t>(blocks(n, 256), 4096), 256, 0, s>>>(in, out, n, nc);
}

void cnn_vec_to_chan_first(const float* in, double* out, int64_t n, int nc, cudaStream_t s) {
  k_vec_to_chan_first<<<(unsigned)std::min<int64_t>(blocks(n, 256), 4096), 256, 0, s>>>(in, out, n, nc);
}

void cnn_guess(int form, const void* phi, const float* y, const float scale[4], void* guess,
               int64_t C, cudaStream_t s) {
  const unsigned g = (unsigned)std::min<int64_t>(blocks(C, 256), 4096);
  if (form == FORM_SPLIT)
    k_guess<dd><<<g, 256, 0, s>>>((const dd*)phi, y, scale[0], scale[1], scale[2], scale[3], (dd*)guess, C);
  else if (form == FORM_PLAIN)
    k_guess<float><<<g, 256, 0, s>>>((const float*)phi, y, scale[0], scale[1], scale[2], scale[3], (float*)guess, C);
  else
    k_guess<double><<<g, 256, 0, s>>>((const double*)phi, y, scale[0], scale[1], scale[2], scale[3], (double*)guess, C);
}

}  // namespace sedi

// ---------------------------------------------------------------- tensor-core layer 2
// The 32 -> 32 convolution holds 80% of the network's work.  Implicit GEMM on the
// tensor cores with mma.sync m16n8k16 (bf16 in, FP32 accumulate): each warp owns 16
// voxels (M) x 32 output channels (N, four n8 tiles); K = 27 taps x 32 channels in
// k16 steps.  A fragments are gathered straight from the channels-last bf16
// activations of each tap's neighbour voxel (one 32-bit word = two channels);
// weights sit in shared memory as [tap][n][k] so a B fragment is one 32-bit word.
namespace sedi {

namespace {

__device__ __forceinline__ void mma_bf16_16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// [O=32][I=32][27] FP32 master -> [27][n=32][k=32] bf16
__global__ void k_pack_mma(const float* w, __nv_bfloat16* out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 32 * 32 * 27; k += gridDim.x * blockDim.x) {
    const int o = k / (32 * 27), i = (k / 27) % 32, t = k % 27;
    out[(t * 32 + o) * 32 + i] = __float2bfloat16_rn(w[k]);
  }
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__global__ void __launch_bounds__(128) k_conv2_mma(const __nv_bfloat16* in, const __nv_bfloat16* wt,
                                                    const float* bias, __nv_bfloat16* out, Grid3 g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* sw = reinterpret_cast<__nv_bfloat16*>(smem_raw);  // [27][32][32]
  {
    const uint4* src = reinterpret_cast<const uint4*>(wt);
    uint4* dst = reinterpret_cast<uint4*>(sw);
    for (int k = threadIdx.x; k < 27 * 32 * 32 / 8; k += blockDim.x) dst[k] = src[k];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = lane >> 2, tig = lane & 3;
  const int64_t v0 = ((int64_t)blockIdx.x * 4 + warp) * 16;
  if (v0 >= g.n) return;
  const int64_t r0 = v0 + gid, r1 = v0 + gid + 8;
  const bool ok0 = r0 < g.n, ok1 = r1 < g.n;
  int c0[3], c1[3];
  c0[0] = (int)(r0 % g.nx); c0[1] = (int)((r0 / g.nx) % g.ny); c0[2] = (int)(r0 / ((int64_t)g.nx * g.ny));
  c1[0] = (int)(r1 % g.nx); c1[1] = (int)((r1 / g.nx) % g.ny); c1[2] = (int)(r1 / ((int64_t)g.nx * g.ny));
  float acc[4][4];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[nt][e] = 0.0f;
  for (int t = 0; t < 27; ++t) {
    const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
    const int64_t q0 = ok0 ? nb_of(g, c0[0], c0[1], c0[2], dx, dy, dz) : -1;
    const int64_t q1 = ok1 ? nb_of(g, c1[0], c1[1], c1[2], dx, dy, dz) : -1;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const int kb = ks * 16 + 2 * tig;
      uint32_t a[4];
      a[0] = q0 >= 0 ? ld_pair(in + q0 * 32 + kb) : 0u;
      a[1] = q1 >= 0 ? ld_pair(in + q1 * 32 + kb) : 0u;
      a[2] = q0 >= 0 ? ld_pair(in + q0 * 32 + kb + 8) : 0u;
      a[3] = q1 >= 0 ? ld_pair(in + q1 * 32 + kb + 8) : 0u;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const __nv_bfloat16* wrow = sw + (t * 32 + nt * 8 + gid) * 32 + kb;
        uint32_t b[2] = {ld_pair(wrow), ld_pair(wrow + 8)};
        mma_bf16_16816(acc[nt], a, b);
      }
    }
  }
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int col = nt * 8 + 2 * tig;
    const float b0 = bias[col], b1 = bias[col + 1];
    if (ok0) {
      __nv_bfloat162 o;
      o.x = __float2bfloat16_rn(fmaxf(acc[nt][0] + b0, 0.0f));
      o.y = __float2bfloat16_rn(fmaxf(acc[nt][1] + b1, 0.0f));
      *reinterpret_cast<__nv_bfloat162*>(out + r0 * 32 + col) = o;
    }
    if (ok1) {
      __nv_bfloat162 o;
      o.x = __float2bfloat16_rn(fmaxf(acc[nt][2] + b0, 0.0f));
      o.y = __float2bfloat16_rn(fmaxf(acc[nt][3] + b1, 0.0f));
      *reinterpret_cast<__nv_bfloat162*>(out + r1 * 32 + col) = o;
    }
  }
}

}  // namespace

}  // namespace sedi

namespace sedi {
void conv2_tensor(const float* master_w2, __nv_bfloat16* wbuf, const __nv_bfloat16* in,
                  const float* bias, __nv_bfloat16* out, int nx, int ny, int nz, const int* per,
                  int64_t n, cudaStream_t s) {
  Grid3 g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.per[0] = per[0]; g.per[1] = per[1]; g.per[2] = per[2];
  g.n = n;
  k_pack_mma<<<64, 256, 0, s>>>(master_w2, wbuf);
  const int smem = 27 * 32 * 32 * 2;
  cudaFuncSetAttribute(k_conv2_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int64_t warps = (n + 15) / 16;
  k_conv2_mma<<<(unsigned)((warps + 3) / 4), 128, smem, s>>>(in, wbuf, bias, out, g);
}
}  // namespace sedi
