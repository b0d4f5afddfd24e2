/*
 * Oracle (test infrastructure only): the small 3-D convolutional network that
 * supplies the initial guess of the smoothing solve (the learned warm start),
 * written as plain FP64 direct convolutions.
 *
 * Network: three 3x3x3 convolutions 4 -> 32 -> 32 -> 4 with bias, ReLU after the
 * first two.  Fields are channels-first [c][z][y][x] on the averaging mesh; a tap
 * reaching outside the mesh wraps on periodic axes and reads zero otherwise.
 *   out[o][v] = b[o] + sum_i sum_t w[o][i][t] in[i][v + off(t)],
 *   t = (kz*3 + ky)*3 + kx, off(t) = (kx-1, ky-1, kz-1).
 * Backward: the chain rule written out per layer (data gradient by the same taps
 * mirrored, weight gradient summed over voxels), MSE loss L = mean (y - target)^2.
 * Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *       w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
 * Optional rounding of every stored value to bfloat16 (round to nearest even)
 * emulates the storage precision of the tensor-core kernels.
 */
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct Grid {
  int nx, ny, nz;
  int per[3];
  int64_t n() const { return (int64_t)nx * ny * nz; }
};

/* index of the neighbour of voxel (x, y, z) at offset (dx, dy, dz), or -1 */
int64_t nb_index(const Grid& g, int x, int y, int z, int dx, int dy, int dz) {
  int c[3] = {x + dx, y + dy, z + dz};
  int n[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < 3; ++a) {
    if (c[a] < 0 || c[a] >= n[a]) {
      if (!g.per[a]) return -1;
      c[a] = (c[a] + n[a]) % n[a];
    }
  }
  return ((int64_t)c[2] * g.ny + c[1]) * g.nx + c[0];
}

double bf16(double v) {
  float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return v;  // inf / nan untouched
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  u &= 0xffff0000u;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

void conv(const Grid& g, int cin, int cout, const double* in, const double* w, const double* b,
          double* out) {
  const int64_t N = g.n();
  for (int o = 0; o < cout; ++o)
    for (int z = 0; z < g.nz; ++z)
      for (int y = 0; y < g.ny; ++y)
        for (int x = 0; x < g.nx; ++x) {
          double acc = b[o];
          for (int i = 0; i < cin; ++i)
            for (int kz = 0; kz < 3; ++kz)
              for (int ky = 0; ky < 3; ++ky)
                for (int kx = 0; kx < 3; ++kx) {
                  int64_t q = nb_index(g, x, y, z, kx - 1, ky - 1, kz - 1);
                  if (q < 0) continue;
                  int t = (kz * 3 + ky) * 3 + kx;
                  acc += w[((int64_t)o * cin + i) * 27 + t] * in[(int64_t)i * N + q];
                }
          out[(int64_t)o * N + ((int64_t)z * g.ny + y) * g.nx + x] = acc;
        }
}

/* gradients of one convolution: din (may be null), dw, db accumulated */
void conv_bwd(const Grid& g, int cin, int cout, const double* in, const double* w,
              const double* dout, double* din, double* dw, double* db) {
  const int64_t N = g.n();
  if (din) std::memset(din, 0, sizeof(double) * cin * N);
  for (int o = 0; o < cout; ++o)
    for (int z = 0; z < g.nz; ++z)
      for (int y = 0; y < g.ny; ++y)
        for (int x = 0; x < g.nx; ++x) {
          const int64_t v = ((int64_t)z * g.ny + y) * g.nx + x;
          const double go = dout[(int64_t)o * N + v];
          db[o] += go;
          for (int i = 0; i < cin; ++i)
            for (int kz = 0; kz < 3; ++kz)
              for (int ky = 0; ky < 3; ++ky)
                for (int kx = 0; kx < 3; ++kx) {
                  int64_t q = nb_index(g, x, y, z, kx - 1, ky - 1, kz - 1);
                  if (q < 0) continue;
                  int t = (kz * 3 + ky) * 3 + kx;
                  dw[((int64_t)o * cin + i) * 27 + t] += go * in[(int64_t)i * N + q];
                  if (din) din[(int64_t)i * N + q] += go * w[((int64_t)o * cin + i) * 27 + t];
                }
        }
}

}  // namespace

extern "C" {

/* Layer sizes: 4 -> 32 -> 32 -> 4.  Parameters packed as
   w1[32][4][27] b1[32] w2[32][32][27] b2[32] w3[4][32][27] b3[4]. */
int64_t orc_cnn_num_params() { return 32 * 4 * 27 + 32 + 32 * 32 * 27 + 32 + 4 * 32 * 27 + 4; }

/* Forward: in [4][N] -> out [4][N]; a1, a2 ([32][N] each, may be null) receive the
   post-ReLU activations.  round_bf16: round inputs, weights and stored activations
   to bfloat16 like the tensor-core kernels. */
int orc_cnn_forward(int nx, int ny, int nz, const int32_t* per, const double* params,
                    const double* in, double* out, double* a1, double* a2, int32_t round_bf16) {
  Grid g{nx, ny, nz, {per[0], per[1], per[2]}};
  const int64_t N = g.n();
  std::vector<double> p(params, params + orc_cnn_num_params());
  std::vector<double> x(in, in + 4 * N);
  if (round_bf16) {
    for (auto& v : p) v = bf16(v);
    for (auto& v : x) v = bf16(v);
  }
  const double* w1 = p.data();
  const double* b1 = w1 + 32 * 4 * 27;
  const double* w2 = b1 + 32;
  const double* b2 = w2 + 32 * 32 * 27;
  const double* w3 = b2 + 32;
  const double* b3 = w3 + 4 * 32 * 27;
  std::vector<double> h1(32 * N), h2(32 * N);
  conv(g, 4, 32, x.data(), w1, b1, h1.data());
  for (auto& v : h1) v = v > 0 ? v : 0.0;
  if (round_bf16)
    for (auto& v : h1) v = bf16(v);
  conv(g, 32, 32, h1.data(), w2, b2, h2.data());
  for (auto& v : h2) v = v > 0 ? v : 0.0;
  if (round_bf16)
    for (auto& v : h2) v = bf16(v);
  conv(g, 32, 4, h2.data(), w3, b3, out);
  if (a1) std::memcpy(a1, h1.data(), sizeof(double) * 32 * N);
  if (a2) std::memcpy(a2, h2.data(), sizeof(double) * 32 * N);
  return 0;
}

/* Loss L = mean over [4][N] of (out - target)^2 and its gradient w.r.t. params. */
double orc_cnn_loss_grad(int nx, int ny, int nz, const int32_t* per, const double* params,
                         const double* in, const double* target, double* grad) {
  Grid g{nx, ny, nz, {per[0], per[1], per[2]}};
  const int64_t N = g.n();
  std::vector<double> out(4 * N), h1(32 * N), h2(32 * N);
  orc_cnn_forward(nx, ny, nz, per, params, in, out.data(), h1.data(), h2.data(), 0);
  const double* w1 = params;
  const double* w2 = w1 + 32 * 4 * 27 + 32;
  const double* w3 = w2 + 32 * 32 * 27 + 32;
  std::memset(grad, 0, sizeof(double) * orc_cnn_num_params());
  double* gw1 = grad;
  double* gb1 = gw1 + 32 * 4 * 27;
  double* gw2 = gb1 + 32;
  double* gb2 = gw2 + 32 * 32 * 27;
  double* gw3 = gb2 + 32;
  double* gb3 = gw3 + 4 * 32 * 27;
  double loss = 0.0;
  std::vector<double> dout(4 * N);
  for (int64_t k = 0; k < 4 * N; ++k) {
    double d = out[k] - target[k];
    loss += d * d;
    dout[k] = 2.0 * d / (4.0 * N);
  }
  loss /= 4.0 * N;
  std::vector<double> d2(32 * N), d1(32 * N);
  conv_bwd(g, 32, 4, h2.data(), w3, dout.data(), d2.data(), gw3, gb3);
  for (int64_t k = 0; k < 32 * N; ++k)
    if (!(h2[k] > 0)) d2[k] = 0.0;
  conv_bwd(g, 32, 32, h1.data(), w2, d2.data(), d1.data(), gw2, gb2);
  for (int64_t k = 0; k < 32 * N; ++k)
    if (!(h1[k] > 0)) d1[k] = 0.0;
  conv_bwd(g, 4, 32, in, w1, d1.data(), nullptr, gw1, gb1);
  return loss;
}

/* One Adam step (step counter t >= 1) on params with moments m, v. */
void orc_adam(int64_t n, double* params, const double* grad, double* m, double* v, int64_t t,
              double lr, double beta1, double beta2, double eps) {
  const double c1 = 1.0 - std::pow(beta1, (double)t);
  const double c2 = 1.0 - std::pow(beta2, (double)t);
  for (int64_t k = 0; k < n; ++k) {
    m[k] = beta1 * m[k] + (1.0 - beta1) * grad[k];
    v[k] = beta2 * v[k] + (1.0 - beta2) * grad[k] * grad[k];
    params[k] -= lr * (m[k] / c1) / (std::sqrt(v[k] / c2) + eps);
  }
}

}  // extern "C"
