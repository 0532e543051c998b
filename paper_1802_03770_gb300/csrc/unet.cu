// U-Net of the learned preconditioner: forward, backward and Adam kernels.
//
// The network (3-level U-Net, channels 16/32/64, 3 x 3 convolutions with
// zero padding and bias, ReLU, 2 x 2 average pooling, 2 x 2 nearest
// upsampling, skip concatenation, 1 x 1 head) maps the features
// [r / s_r, z0 / s_z, alpha] of a residual r to a correction of the base
// preconditioner z0 = B r.  Weights are kept as an FP32 master copy for
// Adam and a BF16 copy that the convolutions read; products are
// accumulated in FP32.  Activations are FP32, layout [channel][y][x].
//
// Pooling, upsampling and concatenation are not materialised: a
// convolution reads its input through up to two sources, each either
// direct, a 2 x 2 average of a twice finer tensor, or the nearest value of a
// twice coarser one.  The backward pass reuses the forward kernel with the
// weights read transposed and flipped (input gradient), a tiled weight
// gradient with per-tile partials reduced in a fixed order (deterministic),
// and a scatter that routes the input gradient back through the sources.
#include <cuda_bf16.h>

#include "chain.cuh"
#include "unet.h"

namespace fl {

namespace {

constexpr int TILE = 16;   // output pixels per CTA side
constexpr int CO = 16;     // output channels per CTA
constexpr int CI = 8;      // input channels per shared-memory chunk

// Value of input channel c (of the virtual concatenated input) at (y, x)
// of the output resolution H x W; zero outside the image.
__device__ __forceinline__ float src_value(const ConvArgs& a, int c, int y, int x) {
  if (y < 0 || y >= a.H || x < 0 || x >= a.W) return 0.f;
  const ConvSrc& s = (c < a.src[0].nc) ? a.src[0] : a.src[1];
  const int cc = (c < a.src[0].nc) ? c : c - a.src[0].nc;
  if (s.mode == SRC_DIRECT) return s.p[((size_t)cc * a.H + y) * a.W + x];
  if (s.mode == SRC_POOL) {
    const int W2 = 2 * a.W;
    const float* q = s.p + ((size_t)cc * 2 * a.H + 2 * y) * W2 + 2 * x;
    return 0.25f * (q[0] + q[1] + q[W2] + q[W2 + 1]);
  }
  // SRC_UP: twice coarser source
  return s.p[((size_t)cc * (a.H / 2) + (y >> 1)) * (a.W / 2) + (x >> 1)];
}

// Weight (output channel o, input channel i, tap t) of the layer as this
// launch reads it: w[o][i][t], or for the input-gradient pass of a layer
// w_f[cout_f][cin_f][k][k], w[i][o][k*k-1-t] (transposed and flipped).
__device__ __forceinline__ float weight(const ConvArgs& a, int o, int i, int t) {
  const int kk = a.k * a.k;
  if (!a.transposed) return __bfloat162float(a.w[((size_t)o * a.cin + i) * kk + t]);
  return __bfloat162float(a.w[((size_t)i * a.cout + o) * kk + (kk - 1 - t)]);
}

template <int K>
__global__ void __launch_bounds__(TILE * TILE) k_conv(ConvArgs a) {
  constexpr int R = K / 2;
  constexpr int S = TILE + 2 * R;
  __shared__ float tile[CI][S][S];
  __shared__ float ws[CO][CI][K * K];
  const int tx = threadIdx.x % TILE, ty = threadIdx.x / TILE;
  const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE;
  const int co0 = blockIdx.z * CO;
  float acc[CO];
#pragma unroll
  for (int o = 0; o < CO; ++o) acc[o] = 0.f;
  for (int c0 = 0; c0 < a.cin; c0 += CI) {
    for (int e = threadIdx.x; e < CI * S * S; e += TILE * TILE) {
      const int c = e / (S * S), rem = e - c * S * S;
      const int yy = rem / S, xx = rem - yy * S;
      tile[c][yy][xx] = (c0 + c < a.cin) ? src_value(a, c0 + c, y0 + yy - R, x0 + xx - R) : 0.f;
    }
    for (int e = threadIdx.x; e < CO * CI * K * K; e += TILE * TILE) {
      const int o = e / (CI * K * K), rem = e - o * CI * K * K;
      const int i = rem / (K * K), t = rem - i * K * K;
      ws[o][i][t] = (co0 + o < a.cout && c0 + i < a.cin) ? weight(a, co0 + o, c0 + i, t) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < CI; ++i) {
#pragma unroll
      for (int t = 0; t < K * K; ++t) {
        const float v = tile[i][ty + t / K][tx + t % K];
#pragma unroll
        for (int o = 0; o < CO; ++o) acc[o] = fmaf(v, ws[o][i][t], acc[o]);
      }
    }
    __syncthreads();
  }
  const int y = y0 + ty, x = x0 + tx;
#pragma unroll
  for (int o = 0; o < CO; ++o) {
    const int co = co0 + o;
    if (co < a.cout) {
      float z = acc[o] + (a.bias ? a.bias[co] : 0.f);
      if (a.relu) z = fmaxf(z, 0.f);
      a.out[((size_t)co * a.H + y) * a.W + x] = z;
    }
  }
}

// Weight and bias gradient partials of one 16 x 16 tile for 16 output and 8
// input channels: part[tile][co][ci][t] = sum_p gz[co][p] in[ci][p + t],
// bpart[tile][co] = sum_p gz[co][p] (written by the ci-chunk-0 CTAs).
template <int K>
__global__ void __launch_bounds__(TILE * TILE) k_conv_wgrad(ConvArgs a, const float* __restrict__ gz,
                                                           float* __restrict__ part,
                                                           float* __restrict__ bpart) {
  constexpr int R = K / 2;
  constexpr int S = TILE + 2 * R;
  __shared__ float tile[CI][S][S];
  __shared__ float g[CO][TILE * TILE];
  const int ntx = a.W / TILE;
  const int tile_id = blockIdx.y * ntx + blockIdx.x;
  const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE;
  const int nci = (a.cin + CI - 1) / CI;
  const int co0 = (blockIdx.z / nci) * CO;
  const int c0 = (blockIdx.z % nci) * CI;
  for (int e = threadIdx.x; e < CI * S * S; e += TILE * TILE) {
    const int c = e / (S * S), rem = e - c * S * S;
    const int yy = rem / S, xx = rem - yy * S;
    tile[c][yy][xx] = (c0 + c < a.cin) ? src_value(a, c0 + c, y0 + yy - R, x0 + xx - R) : 0.f;
  }
  for (int e = threadIdx.x; e < CO * TILE * TILE; e += TILE * TILE) {
    const int o = e / (TILE * TILE), p = e - o * TILE * TILE;
    const int yy = p / TILE, xx = p - yy * TILE;
    g[o][p] = (co0 + o < a.cout) ? gz[((size_t)(co0 + o) * a.H + y0 + yy) * a.W + x0 + xx] : 0.f;
  }
  __syncthreads();
  const size_t wsz = (size_t)a.cout * a.cin * K * K;
  for (int e = threadIdx.x; e < CO * CI * K * K; e += TILE * TILE) {
    const int o = e / (CI * K * K), rem = e - o * CI * K * K;
    const int i = rem / (K * K), t = rem - i * K * K;
    const int dy = t / K, dx = t % K;
    float s = 0.f;
    for (int p = 0; p < TILE * TILE; ++p) {
      const int yy = p / TILE, xx = p - yy * TILE;
      s = fmaf(g[o][p], tile[i][yy + dy][xx + dx], s);
    }
    if (co0 + o < a.cout && c0 + i < a.cin)
      part[(size_t)tile_id * wsz + ((size_t)(co0 + o) * a.cin + c0 + i) * K * K + t] = s;
  }
  if (c0 == 0) {
    for (int o = threadIdx.x; o < CO; o += TILE * TILE) {
      float s = 0.f;
      for (int p = 0; p < TILE * TILE; ++p) s += g[o][p];
      if (co0 + o < a.cout) bpart[(size_t)tile_id * a.cout + co0 + o] = s;
    }
  }
}

// out[i] (+)= sum over tiles of part[tile][i] (fixed order).
__global__ void k_reduce_tiles(const float* __restrict__ part, int ntiles, long long n,
                               float* __restrict__ out, int accumulate) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int t = 0; t < ntiles; ++t) s += part[(size_t)t * n + i];
  out[i] = accumulate ? out[i] + s : s;
}

// gz = g where the layer's ReLU output is positive, else 0.
__global__ void k_relu_mask(const float* __restrict__ g, const float* __restrict__ act,
                            float* __restrict__ gz, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) gz[i] = act[i] > 0.f ? g[i] : 0.f;
}

// Route the input gradient gx[cin][H][W] of a convolution to its sources
// (accumulating): direct +=, pooled source (2H x 2W) gets 0.25 gx in each
// of its 2 x 2 cells, upsampled source (H/2 x W/2) the sum of a 2 x 2 block.
__global__ void k_scatter(const float* __restrict__ gx, int c_off, int nc, int mode, int H, int W,
                          float* __restrict__ gsrc) {
  const long long n = (long long)nc * (mode == SRC_POOL ? 4 * H * W : (mode == SRC_UP ? H * W / 4 : H * W));
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (mode == SRC_DIRECT) {
    gsrc[i] += gx[(size_t)c_off * H * W + i];
  } else if (mode == SRC_POOL) {
    const int W2 = 2 * W;
    const long long c = i / (4LL * H * W), rem = i - c * 4LL * H * W;
    const int y = (int)(rem / W2), x = (int)(rem % W2);
    gsrc[i] += 0.25f * gx[((size_t)(c_off + c) * H + y / 2) * W + x / 2];
  } else {
    const int Wh = W / 2, Hh = H / 2;
    const long long c = i / ((long long)Hh * Wh), rem = i - c * Hh * Wh;
    const int y = (int)(rem / Wh), x = (int)(rem % Wh);
    const float* q = gx + ((size_t)(c_off + c) * H + 2 * y) * W + 2 * x;
    gsrc[i] += q[0] + q[1] + q[W] + q[W + 1];
  }
}

// MSE loss: gy = 2 (y - t) / (npix * batch), per-CTA partials of (y - t)^2.
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ gy,
                      long long n, float scale, double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float r = y[i] - t[i];
    gy[i] = 2.f * r * scale;
    s += (double)r * r;
  }
  const double v = cta_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// Adam (Kingma & Ba) on the FP32 master weights; refreshes the BF16 copy.
__global__ void k_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, long long n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  if (wb) wb[i] = __float2bfloat16(wi);
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) wb[i] = __float2bfloat16(w[i]);
}

}  // namespace

// --- 3 x 3 convolution on the tensor cores (tcgen05, kind::f16) ----------------
//
// Implicit GEMM: D[128 pixels][N = cout] += A[128][K] B[N][K]^T with
// K = 9 cin (k = 9 ci + 3 dy + dx) in chunks of 64.  The CTA first stages
// the input halo of its 8 x 16 output pixels (10 x 18 pixels of every input
// channel, through the sources' direct / pooled / upsampled reads) in
// shared memory as BF16, once; each K-chunk's A (im2col rows of the tile)
// is then gathered from that halo and B (the weights) from global memory,
// both stored K-major in the canonical no-swizzle layout (core matrices of
// 8 rows x 8 elements, 128 contiguous bytes; adjacent along K: 128 B,
// adjacent along rows: 1024 B) with 16-byte stores.  A and B have two
// stages: one thread issues the four 128 x N x 16 MMAs of chunk c into a
// TMEM accumulator and commits them to the stage's mbarrier while the CTA
// gathers chunk c + 1 into the other stage; a stage is refilled only after
// the commit of the MMAs that read it (bounded waits).  The epilogue reads
// TMEM lane p (= pixel p) with tcgen05.ld, adds the bias and applies the
// ReLU.  Operands are the same BF16 values in the same order as a gather
// straight from global memory, so the result is too.
namespace {

constexpr int TC_M = 128, TC_KC = 64, TC_NMAX = 96;
// threads per CTA: two per pixel row of the tile for the gathers; in the
// epilogue warps w and w + 4 read the same TMEM lane quadrant, halves of
// the columns
constexpr int TC_THREADS = 256;
constexpr int TC_CIN_MAX = 96;                  // input channels the halo holds
constexpr int TC_HALO_H = 10, TC_HALO_W = 18;   // 8 x 16 tile + 1-pixel border
constexpr int TC_HALO_PIX = TC_HALO_H * TC_HALO_W;
constexpr int TC_STAGE_A = TC_M * TC_KC;   // BF16 elements of one A stage
// halo bytes of cin channels, rounded up to 16 (the mbarriers follow it)
__host__ __device__ constexpr int tc_halo_bytes(int cin) { return (cin * TC_HALO_PIX * 2 + 15) & ~15; }
// dynamic shared memory of a launch with cout = n, cin input channels: the
// A stages (32 KB), the B stages (256 n bytes: 16-byte multiples for n a
// multiple of 16), the halo of cin padded to 8 channels, two mbarriers and
// the TMEM address slot
__host__ __device__ constexpr int tc_smem_bytes(int n, int cin) {
  return 2 * TC_STAGE_A * 2 + 2 * n * TC_KC * 2 + tc_halo_bytes((cin + 7) & ~7) + 32;
}
constexpr int TC_SMEM = tc_smem_bytes(TC_NMAX, TC_CIN_MAX);   // the largest launch
constexpr int kWaitLimit = 1 << 24;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start, leading (K) and stride (row-group)
// byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// canonical K-major offset of element (row, k) for a 64-wide K chunk
__device__ __forceinline__ int canon64(int row, int k) {
  return (((row >> 3) * 8 + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (int it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(mbar), "r"(phase) : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__global__ void __launch_bounds__(TC_THREADS) k_conv_tc(ConvArgs a, int tmem_cols) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  const int N = a.cout;
  // input channels padded to a multiple of 8 (zero channels), so that the
  // 8-wide K groups of the tap-major order k = cinp t + ci stay in one tap
  const int cinp = (a.cin + 7) & ~7;
  // shared memory sized for this layer (tc_smem_bytes): two stages of A,
  // two of B (N rows), the channel-last halo [10][18][cinp], two
  // mbarriers, the TMEM slot
  __nv_bfloat16* sa0 = reinterpret_cast<__nv_bfloat16*>(tc_smem);
  __nv_bfloat16* sb0 = sa0 + 2 * TC_STAGE_A;
  const int stage_b = N * TC_KC;
  __nv_bfloat16* halo = sb0 + 2 * stage_b;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(
      reinterpret_cast<unsigned char*>(halo) + tc_halo_bytes(cinp));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int x0 = blockIdx.x * 16, y0 = blockIdx.y * 8;
  const int K = cinp * 9;
  const int nchunks = (K + TC_KC - 1) / TC_KC;
  const uint32_t mb0 = smem_addr(mbar), mb1 = smem_addr(mbar + 1);
  auto mbs = [=](int s) { return s ? mb1 : mb0; };   // mbarrier of stage s
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb1));
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_addr(tmem_slot)), "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // input halo, BF16, channel-last: item i = (pixel r, group of 8
  // channels) is read from the sources (consecutive threads: consecutive
  // pixels of the same channels), packed and stored with one 16-byte store;
  // two items (sixteen reads) in flight per thread; padded channels are
  // zero.  Group cg of pixel r sits at 16-byte slot cg ^ (r & hmask) of the
  // pixel (hmask + 1: the largest power of two dividing cinp / 8), so that
  // reads of one group at consecutive pixels spread over the banks.
  const int ncg = cinp >> 3;
  const int hmask = (ncg & -ncg) - 1;
  {
    const int items = (cinp >> 3) * TC_HALO_PIX;
    for (int i0 = tid; i0 < items; i0 += 2 * TC_THREADS) {
      float v[2][8];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = i0 + h * TC_THREADS;
        const int cg = i / TC_HALO_PIX, r = i - cg * TC_HALO_PIX;
        const int hy = r / TC_HALO_W, hx = r - hy * TC_HALO_W;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int ci = 8 * cg + k;
          v[h][k] = (i < items && ci < a.cin) ? src_value(a, ci, y0 + hy - 1, x0 + hx - 1) : 0.f;
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = i0 + h * TC_THREADS;
        if (i >= items) continue;
        const int cg = i / TC_HALO_PIX, r = i - cg * TC_HALO_PIX;
        uint4 q;
        q.x = pack_bf16(__float2bfloat16(v[h][0]), __float2bfloat16(v[h][1]));
        q.y = pack_bf16(__float2bfloat16(v[h][2]), __float2bfloat16(v[h][3]));
        q.z = pack_bf16(__float2bfloat16(v[h][4]), __float2bfloat16(v[h][5]));
        q.w = pack_bf16(__float2bfloat16(v[h][6]), __float2bfloat16(v[h][7]));
        *reinterpret_cast<uint4*>(halo + r * cinp + 8 * (cg ^ (r & hmask))) = q;
      }
    }
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                         ((uint32_t)(TC_M >> 4) << 24);
  // this thread's 8-wide K group g of every chunk and its tile rows
  // 8 (oct0 + 4 j) + (tid & 7), j = 0 .. 3: the eight threads of a
  // quarter warp store eight consecutive rows of one group (16 bytes apart
  // in the canonical layout: no bank conflicts)
  const int g = (tid >> 3) & 7;
  const int oct0 = tid >> 6, rlo = tid & 7;
  bool ok = true;
  int issued = 0;   // chunks whose MMAs were issued (and committed)
  for (int ch = 0; ch < nchunks; ++ch) {
    const int s = ch & 1;
    if (ch >= 2) {
      // the MMAs of chunk ch - 2 read stage s: wait for their commit.  A
      // wait that gives up (in any thread) ends the loop for the whole CTA:
      // no more refills, no more MMAs.
      const bool got = mbar_wait(mbs(s), (uint32_t)(((ch - 2) >> 1) & 1));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (__syncthreads_or(!got)) {
        ok = false;
        break;
      }
    }
    __nv_bfloat16* sa = sa0 + s * TC_STAGE_A;
    __nv_bfloat16* sb = sb0 + s * stage_b;
    // the group's 8 k: tap t, channels ci0 .. ci0 + 7
    const int kg = ch * TC_KC + 8 * g;
    const bool kvalid = kg < K;
    const int t = kg / cinp, ci0 = kg - t * cinp;
    // A: the thread's four tile rows, one 16-byte halo read each
    {
      const int dy = t / 3, dx = t - 3 * dy;
      const int cg = ci0 >> 3;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int p = ((oct0 + 4 * j) << 3) + rlo;
        const int q = ((p >> 4) + dy) * TC_HALO_W + (p & 15) + dx;   // halo pixel
        uint4 v4 = make_uint4(0u, 0u, 0u, 0u);
        if (kvalid) v4 = *reinterpret_cast<const uint4*>(halo + q * cinp + 8 * (cg ^ (q & hmask)));
        *reinterpret_cast<uint4*>(sa + canon64(p, 8 * g)) = v4;
      }
    }
    // B: the weights of the group's 8 k for the thread's output channels
    // o = 8 (oct0 + 4 j) + (tid & 7) < N (all its loads issued together)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int o = ((oct0 + 4 * j) << 3) + rlo;
      if (o >= N) break;
      __nv_bfloat16 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int ci = ci0 + u;
        v[u] = __float2bfloat16(kvalid && ci < a.cin ? weight(a, o, ci, t) : 0.f);
      }
      uint4 q;
      q.x = pack_bf16(v[0], v[1]);
      q.y = pack_bf16(v[2], v[3]);
      q.z = pack_bf16(v[4], v[5]);
      q.w = pack_bf16(v[6], v[7]);
      *reinterpret_cast<uint4*>(sb + canon64(o, 8 * g)) = q;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < TC_KC / 16; ++kk) {
        const uint64_t ad = umma_desc(smem_addr(sa) + kk * 256, 128, 1024);
        const uint64_t bd = umma_desc(smem_addr(sb) + kk * 256, 128, 1024);
        const uint32_t acc = (ch > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
            :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(mbs(s)) : "memory");
    }
    issued = ch + 1;
  }
  // the last commit covers every MMA issued before it
  if (issued > 0) {
    const int last = issued - 1;
    const bool got = mbar_wait(mbs(last & 1), (uint32_t)((last >> 1) & 1));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_or(!got)) ok = false;
    if (!ok && tid == 0) {
      // one more bounded wait for the MMAs in flight before TMEM is released
      mbar_wait(mbs(last & 1), (uint32_t)((last >> 1) & 1));
      if (a.err) atomicExch(a.err, 1);
    }
    __syncthreads();
  }
  // epilogue: lane p of TMEM holds pixel p; warp w reads lanes 32 (w mod 4)
  // .. + 31 (its quadrant) and the 16-column groups 16 (w / 4), + 32, ...
  const int quad = warp & 3;
  const int p = quad * 32 + (tid & 31);
  const int y = y0 + (p >> 4), x = x0 + (p & 15);
  for (int c0 = 16 * (warp >> 2); c0 < N; c0 += 16 * (TC_THREADS / TC_M)) {
    if (!ok) {   // outputs of a tile whose MMAs did not complete are zeroed
      for (int j = 0; j < 16; ++j) a.out[((size_t)(c0 + j) * a.H + y) * a.W + x] = 0.f;
      continue;
    }
    uint32_t v[16];
    const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int co = c0 + j;
      float z = __uint_as_float(v[j]) + (a.bias ? a.bias[co] : 0.f);
      if (a.relu) z = fmaxf(z, 0.f);
      a.out[((size_t)co * a.H + y) * a.W + x] = z;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(tmem_cols));
}

}  // namespace

cudaError_t configure_unet_kernels() {
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_conv_tc),
                              cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
}

cudaError_t launch_conv(const ConvArgs& a, cudaStream_t s) {
  if (a.tensor_cores && a.k == 3 && a.cout % 16 == 0 && a.cout <= TC_NMAX && a.cin <= TC_CIN_MAX &&
      a.H % 8 == 0 && a.W % 16 == 0) {
    const int cols = a.cout <= 32 ? 32 : (a.cout <= 64 ? 64 : 128);
    dim3 grid(a.W / 16, a.H / 8);
    FL_KERNEL("unet_conv3_tc", s,
              k_conv_tc<<<grid, TC_THREADS, tc_smem_bytes(a.cout, a.cin), s>>>(a, cols));
    return cudaGetLastError();
  }
  dim3 grid(a.W / TILE, a.H / TILE, (a.cout + CO - 1) / CO);
  if (a.k == 3)
    FL_KERNEL("unet_conv3", s, k_conv<3><<<grid, TILE * TILE, 0, s>>>(a));
  else
    FL_KERNEL("unet_conv1", s, k_conv<1><<<grid, TILE * TILE, 0, s>>>(a));
  return cudaGetLastError();
}

size_t conv_wgrad_partials(const ConvArgs& a) {
  return (size_t)(a.W / TILE) * (a.H / TILE) * a.cout * a.cin * a.k * a.k;
}

cudaError_t launch_conv_wgrad(const ConvArgs& a, const float* gz, float* part, float* bpart,
                              float* dw, float* db, int accumulate, cudaStream_t s) {
  const int nci = (a.cin + CI - 1) / CI, nco = (a.cout + CO - 1) / CO;
  dim3 grid(a.W / TILE, a.H / TILE, nci * nco);
  if (a.k == 3)
    FL_KERNEL("unet_wgrad3", s, k_conv_wgrad<3><<<grid, TILE * TILE, 0, s>>>(a, gz, part, bpart));
  else
    FL_KERNEL("unet_wgrad1", s, k_conv_wgrad<1><<<grid, TILE * TILE, 0, s>>>(a, gz, part, bpart));
  const int ntiles = (a.W / TILE) * (a.H / TILE);
  const long long nw = (long long)a.cout * a.cin * a.k * a.k;
  FL_KERNEL("unet_reduce", s,
            k_reduce_tiles<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(part, ntiles, nw, dw, accumulate));
  FL_KERNEL("unet_reduce", s,
            k_reduce_tiles<<<(unsigned)((a.cout + 255) / 256), 256, 0, s>>>(bpart, ntiles, a.cout, db,
                                                                            accumulate));
  return cudaGetLastError();
}

cudaError_t launch_relu_mask(const float* g, const float* act, float* gz, long long n, cudaStream_t s) {
  FL_KERNEL("unet_mask", s, k_relu_mask<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, act, gz, n));
  return cudaGetLastError();
}

cudaError_t launch_scatter(const float* gx, int c_off, int nc, int mode, int H, int W, float* gsrc,
                           cudaStream_t s) {
  const long long n = (long long)nc * (mode == SRC_POOL ? 4LL * H * W : (mode == SRC_UP ? (long long)H * W / 4 : (long long)H * W));
  FL_KERNEL("unet_scatter", s,
            k_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(gx, c_off, nc, mode, H, W, gsrc));
  return cudaGetLastError();
}

cudaError_t launch_mse(const float* y, const float* t, float* gy, long long n, float scale,
                       double* part, int nblocks, cudaStream_t s) {
  FL_KERNEL("unet_mse", s, k_mse<<<nblocks, 256, 0, s>>>(y, t, gy, n, scale, part));
  return cudaGetLastError();
}

cudaError_t launch_adam(float* w, __nv_bfloat16* wb, const float* g, float* m, float* v, long long n,
                        float lr, int step, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  FL_KERNEL("unet_adam", s,
            k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, wb, g, m, v, n, lr, b1, b2, 1e-8f,
                                                                c1, c2));
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* w, __nv_bfloat16* wb, long long n, cudaStream_t s) {
  FL_KERNEL("unet_to_bf16", s, k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, wb, n));
  return cudaGetLastError();
}

}  // namespace fl
