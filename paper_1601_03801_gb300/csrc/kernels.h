// Host-side launchers of the sm_103a kernels (one translation unit per phase).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace sedi {

// Launch variants of the substep kernel: threads per block and minimum resident
// blocks per SM (128/6, 64/12, 256/3 cap registers at 80 a thread, 128/8 at 64,
// 128/5 at 96).  The split and plain forms have all five; the FP64 parity form
// runs 128/6.
enum SubstepVariant {
  SUBSTEP_B128 = 0,
  SUBSTEP_B64 = 1,
  SUBSTEP_B256 = 2,
  SUBSTEP_B128_OCC8 = 3,
  SUBSTEP_B128_OCC5 = 4
};
constexpr int kSubstepVariants = 5;
inline int substep_block(int variant) { return variant == SUBSTEP_B64 ? 64 : variant == SUBSTEP_B256 ? 256 : 128; }

// k_force.cu: one fused substep (integrate = true) or forces only into st.fdbg.
// The last block of an integrating launch sets ctl->need_rebuild and, when
// use_cond, the graph condition next_cond of the following rebuild node.
void launch_substep(int form, const DevState& st, const DevMesh& mesh, const DevParams& P,
                    int sub_off, bool integrate, int variant, unsigned long long next_cond,
                    int use_cond, cudaStream_t s);

// k_bin.cu: rebuild = bin, sort by (bin, caller index), gather into the other
// buffers, build lists, carry springs over.  `conditional` kernels return at once
// unless ctl->need_rebuild is set.  sub_off: substep offset of the state buffer.
void launch_rebuild(int form, const DevState& st, const DevParams& P, int sub_off, bool force,
                    cudaStream_t s);
// Set ctl->need_rebuild from the displacement; optionally a graph conditional.
void launch_check(const DevState& st, const DevParams& P, unsigned long long cond_handle,
                  int use_cond, cudaStream_t s);
// ctl->st = (ctl->st + n) & 1 after n substeps.
void launch_advance_parity(const DevState& st, int n, cudaStream_t s);

// Scatter/gather between the sorted device state and caller order.
void launch_export(int form, const DevState& st, int what, double* out, cudaStream_t s);
void launch_import(int form, const DevState& st, const double* x, const double* v,
                   const double* w, const double* d, const double* rho, const DevParams& P,
                   cudaStream_t s);
void launch_neighbors_export(const DevState& st, int64_t* counts, cudaStream_t s);
void launch_neighbors_fill(const DevState& st, const int64_t* offsets, int64_t* out,
                           cudaStream_t s);
void launch_contacts_export(int form, const DevState& st, const DevParams& P,
                            unsigned long long* count, int64_t cap, int64_t* ij, double* xi,
                            cudaStream_t s);

// k_avg.cu: deposition, field conversion, persistent CG smoother, outputs.
void launch_deposit(int form, const DevState& st, const DevMesh& mesh, const DevParams& P,
                    void* qfields, cudaStream_t s);
void launch_fields_from_fixed(int form, const void* q, const DevParams& P, void* phi,
                              int nf, cudaStream_t s);
// Smooth nf fields [nf][C] in place (type by form).  guess may be null.
int launch_smooth(int form, const DevParams& P, void* phi, const void* guess, int nf,
                  void* work, const DevState& st, int* iters_dev, double rtol, int max_iter,
                  int n_tau, const double coef[3], cudaStream_t s);
size_t smooth_work_bytes(int form, int64_t C, int nf);
void launch_average_out(int form, const void* phi, const DevParams& P, void* ufe, double* eps,
                        double* Us, double* F, cudaStream_t s);
void launch_phi_convert(int form, const void* phi, double* out, int64_t n, int to_double,
                        cudaStream_t s);
void launch_phi_from_double(int form, const double* in, void* phi, int64_t n, cudaStream_t s);

// k_cnn.cu: learned warm start (3x3x3 CNN 4 -> 32 -> 32 -> 4, bf16 storage).
size_t cnn_param_count();
size_t cnn_work_bytes(int64_t n);
// network input from four channel rows (FP64 device arrays) divided by scale
void cnn_input(const DevParams& P, const double* const f[4], const float scale[4], void* work,
               cudaStream_t s);
// forward with the bf16-rounded copy of the FP32 master weights; *y_out: [v][4] FP32
void cnn_forward(const DevParams& P, const float* master, void* work, float** y_out,
                 cudaStream_t s);
// loss = mean (y - target)^2 ([v][4] FP32 target) and its gradient (FP32, packed order)
void cnn_loss_grad(const DevParams& P, const float* master, const float* target, float* grad,
                   double* loss, void* work, cudaStream_t s);
void cnn_adam(float* master, const float* grad, float* m, float* v, int64_t t, float lr,
              cudaStream_t s);
void cnn_chan_first_to_vec(const double* in, float* out, int64_t n, int nc, cudaStream_t s);
void cnn_vec_to_chan_first(const float* in, double* out, int64_t n, int nc, cudaStream_t s);
// guess = phi (+ scale * y on eps and F), in the smoothing word of the form
void cnn_guess(int form, const void* phi, const float* y, const float scale[4], void* guess,
               int64_t C, cudaStream_t s);

}  // namespace sedi
