// The network object of the learned preconditioner (learned.cu).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "unet.h"

// Sets the thread's fl_last_error_string() text (defined in plan.cu).
void fl_set_error_string(const char* msg);

namespace fl {

constexpr int kNetLayers = 11;
constexpr int kNetTensors = 12;  // input, ten hidden activations, output
constexpr int kNetInputs = 3;    // r / s_r, z0 / s_z, alpha
constexpr int kLossBlocks = 256;

struct NetState {
  int H = 0, W = 0;
  int c[3] = {16, 32, 64};
  cudaStream_t stream = nullptr;
  long long nparams = 0;
  long long woff[kNetLayers] = {}, boff[kNetLayers] = {};
  int cin_[kNetLayers] = {}, cout_[kNetLayers] = {};
  float* w = nullptr;          // FP32 master parameters (weights and biases, flat)
  __nv_bfloat16* wb = nullptr; // BF16 copy read by the convolutions
  float* g = nullptr;          // gradients
  float* m = nullptr;          // Adam moments
  float* v = nullptr;
  float* act[kNetTensors] = {};
  float* grad[kNetTensors] = {};
  float* gz = nullptr;
  float* gx = nullptr;
  float* part = nullptr;
  float* bpart = nullptr;
  double* lpart = nullptr;
  int step = 0;
  int use_tc = 1;              // 3 x 3 convolutions on tcgen05 (BF16 operands)
  // alpha gate (fl_net_set_alpha_gate): empty = the network serves every
  // alpha; else alpha in [gate_lo, gate_hi) split into gate.size() equal
  // bands, the network serving the enabled ones only
  double gate_lo = 0.0, gate_hi = 0.0;
  std::vector<uint8_t> gate;
  bool alpha_enabled(double alpha) const;
  int* err = nullptr;          // device flag of the bounded tensor-core waits
  std::vector<void*> allocs;

  int channels(int t) const;
  int level(int t) const;
  cudaError_t init(int h, int w, uint64_t seed, cudaStream_t s);
  ConvArgs conv_args(int l, bool input_grad) const;
  cudaError_t forward(const float* x, float* y);
  cudaError_t backward();
  cudaError_t loss_grad(const float* xs, const float* ts, int batch, double* loss);
  cudaError_t train_step(const float* xs, const float* ts, int batch, float lr, double* loss);
  ~NetState();
};

}  // namespace fl

namespace fl {
struct PcgState;
// Training pairs: z0 = r / k0, and the pair's features and target from r, z0,
// u*, x (2 * 256 partials in part).
cudaError_t launch_div_scalar(const double* r, double k0, double* z0, long long N, cudaStream_t s);
cudaError_t launch_training_pair(const double* r, const double* z0, const double* u_star, const double* x,
                                 double alpha, float* feat, float* target, long long N, double* part,
                                 cudaStream_t s);
cudaError_t launch_features(const float* r, const float* z0, const double* rr_part, int rr_count,
                            const double* zz_part, int zz_count, float alpha, float* x, long long N,
                            const PcgState* st, cudaStream_t s);
cudaError_t launch_combine(const float* r, const float* z0, const float* y, float* z, const double* zz_part,
                           int zz_count, double* rz_part, double* rzo_part, long long N, const PcgState* st,
                           int* count, cudaStream_t s);
cudaError_t launch_scale(const float* src, float* dst, float scale, long long N, const PcgState* st,
                         cudaStream_t s);
cudaError_t launch_fpcg_scalar(PcgState* st, const double* rr_part, int rr_count, const double* rz_part,
                               const double* rzo_part, int rz_count, cudaStream_t s);
}  // namespace fl

struct fl_net;
fl::NetState* fl_net_state(fl_net* n);
