// Interfaces of the U-Net kernels (unet.cu) used by the network driver
// (learned.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace fl {

enum { SRC_DIRECT = 0, SRC_POOL = 1, SRC_UP = 2 };

// One input source of a convolution: nc channels read from p, directly
// (same resolution), as the 2 x 2 average of a twice finer tensor, or as
// the nearest value of a twice coarser tensor.
struct ConvSrc {
  const float* p;
  int nc;
  int mode;
};

struct ConvArgs {
  ConvSrc src[2];
  int cin, cout;     // channels read / written by this launch
  int H, W;          // output resolution (multiples of 16)
  int k;             // 3 or 1
  const __nv_bfloat16* w;  // layer weights [cout_f][cin_f][k][k]
  int transposed;    // 1: input-gradient pass (weights read transposed and flipped)
  const float* bias; // nullable
  float* out;        // [cout][H][W]
  int relu;
  int tensor_cores;  // 1: 3 x 3 layers with cout % 16 == 0 run on tcgen05 (BF16 operands)
  int* err;          // device flag set when a bounded tensor-core wait gives up
};

cudaError_t launch_conv(const ConvArgs& a, cudaStream_t s);
cudaError_t configure_unet_kernels();
size_t conv_wgrad_partials(const ConvArgs& a);
cudaError_t launch_conv_wgrad(const ConvArgs& a, const float* gz, float* part, float* bpart, float* dw,
                              float* db, int accumulate, cudaStream_t s);
cudaError_t launch_relu_mask(const float* g, const float* act, float* gz, long long n, cudaStream_t s);
cudaError_t launch_scatter(const float* gx, int c_off, int nc, int mode, int H, int W, float* gsrc,
                           cudaStream_t s);
cudaError_t launch_mse(const float* y, const float* t, float* gy, long long n, float scale,
                       double* part, int nblocks, cudaStream_t s);
cudaError_t launch_adam(float* w, __nv_bfloat16* wb, const float* g, float* m, float* v, long long n,
                        float lr, int step, cudaStream_t s);
cudaError_t launch_to_bf16(const float* w, __nv_bfloat16* wb, long long n, cudaStream_t s);

}  // namespace fl
