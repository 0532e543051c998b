// The network object of the learned preconditioner: parameters (FP32
// master, BF16 copy, Adam moments), activations and gradients, forward,
// backward, training step, checkpoint files.  The architecture is described
// in unet.cu.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fraclap.h"
#include "chain.cuh"
#include "learned.h"
#include "unet.h"

namespace fl {

namespace {

// layer table: name, input sources (tensor id, mode), cout, k, level
enum { T_X = 0, T_E0A, T_E0B, T_E1A, T_E1B, T_BA, T_BB, T_D1A, T_D1B, T_D0A, T_D0B, T_Y, T_COUNT };

struct LayerSpec {
  int out;          // output tensor id
  int src[2];       // source tensor ids (-1 unused)
  int mode[2];
  int k;
  int relu;
};

const LayerSpec kLayers[kNetLayers] = {
    {T_E0A, {T_X, -1}, {SRC_DIRECT, 0}, 3, 1},
    {T_E0B, {T_E0A, -1}, {SRC_DIRECT, 0}, 3, 1},
    {T_E1A, {T_E0B, -1}, {SRC_POOL, 0}, 3, 1},
    {T_E1B, {T_E1A, -1}, {SRC_DIRECT, 0}, 3, 1},
    {T_BA, {T_E1B, -1}, {SRC_POOL, 0}, 3, 1},
    {T_BB, {T_BA, -1}, {SRC_DIRECT, 0}, 3, 1},
    {T_D1A, {T_BB, T_E1B}, {SRC_UP, SRC_DIRECT}, 3, 1},
    {T_D1B, {T_D1A, -1}, {SRC_DIRECT, 0}, 3, 1},
    {T_D0A, {T_D1B, T_E0B}, {SRC_UP, SRC_DIRECT}, 3, 1},
    {T_D0B, {T_D0A, -1}, {SRC_DIRECT, 0}, 3, 1},
    {T_Y, {T_D0B, -1}, {SRC_DIRECT, 0}, 1, 0},
};

// 64-bit mixer (splitmix64) and Box-Muller, for the He-normal initialisation.
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
double uniform01(uint64_t& s) { return ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

}  // namespace

int NetState::channels(int t) const {
  switch (t) {
    case T_X: return kNetInputs;
    case T_E0A: case T_E0B: case T_D0A: case T_D0B: return c[0];
    case T_E1A: case T_E1B: case T_D1A: case T_D1B: return c[1];
    case T_BA: case T_BB: return c[2];
    default: return 1;
  }
}

int NetState::level(int t) const {
  switch (t) {
    case T_E1A: case T_E1B: case T_D1A: case T_D1B: return 1;
    case T_BA: case T_BB: return 2;
    default: return 0;
  }
}

cudaError_t NetState::init(int h, int wd, uint64_t seed, cudaStream_t s) {
  H = h;
  W = wd;
  stream = s;
  nparams = 0;
  for (int l = 0; l < kNetLayers; ++l) {
    const LayerSpec& L = kLayers[l];
    int cin = 0;
    for (int j = 0; j < 2; ++j)
      if (L.src[j] >= 0) cin += channels(L.src[j]);
    cin_[l] = cin;
    cout_[l] = channels(L.out);
    woff[l] = nparams;
    nparams += (long long)cout_[l] * cin * L.k * L.k;
    boff[l] = nparams;
    nparams += cout_[l];
  }
  // He-normal weights, zero biases
  std::vector<float> host(nparams, 0.f);
  uint64_t st = seed;
  for (int l = 0; l < kNetLayers; ++l) {
    const int k = kLayers[l].k;
    const double stdv = std::sqrt(2.0 / (cin_[l] * k * k));
    for (long long i = woff[l]; i < boff[l]; ++i) {
      const double u1 = uniform01(st), u2 = uniform01(st);
      host[i] = (float)(stdv * std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2));
    }
  }
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) allocs.push_back(*p);
  };
  al((void**)&w, nparams * sizeof(float));
  al((void**)&wb, nparams * sizeof(__nv_bfloat16));
  al((void**)&g, nparams * sizeof(float));
  al((void**)&m, nparams * sizeof(float));
  al((void**)&v, nparams * sizeof(float));
  size_t maxg = 0, maxgx = 0, maxpart = 0;
  for (int t = 0; t < T_COUNT; ++t) {
    const size_t n = (size_t)channels(t) * (H >> level(t)) * (W >> level(t));
    al((void**)&act[t], n * sizeof(float));
    al((void**)&grad[t], n * sizeof(float));
    maxg = std::max(maxg, n);
  }
  for (int l = 0; l < kNetLayers; ++l) {
    const int lev = level(kLayers[l].out);
    maxgx = std::max(maxgx, (size_t)cin_[l] * (H >> lev) * (W >> lev));
    ConvArgs a = conv_args(l, false);
    maxpart = std::max(maxpart, conv_wgrad_partials(a));
  }
  al((void**)&gz, maxg * sizeof(float));
  al((void**)&gx, maxgx * sizeof(float));
  al((void**)&part, maxpart * sizeof(float));
  al((void**)&bpart, (size_t)(H / 16) * (W / 16) * 64 * sizeof(float));
  al((void**)&lpart, kLossBlocks * sizeof(double));
  al((void**)&err, sizeof(int));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(w, host.data(), nparams * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m, 0, nparams * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, nparams * sizeof(float), s);
  if (e == cudaSuccess) e = launch_to_bf16(w, wb, nparams, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = configure_unet_kernels();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  step = 0;
  return e;
}

NetState::~NetState() {
  for (void* p : allocs) cudaFree(p);
}

ConvArgs NetState::conv_args(int l, bool input_grad) const {
  const LayerSpec& L = kLayers[l];
  const int lev = level(L.out);
  ConvArgs a;
  memset(&a, 0, sizeof(a));
  a.H = H >> lev;
  a.W = W >> lev;
  a.k = L.k;
  a.w = wb + woff[l];
  a.tensor_cores = use_tc;
  a.err = err;
  if (!input_grad) {
    for (int j = 0; j < 2; ++j) {
      a.src[j].p = L.src[j] >= 0 ? act[L.src[j]] : nullptr;
      a.src[j].nc = L.src[j] >= 0 ? channels(L.src[j]) : 0;
      a.src[j].mode = L.mode[j];
    }
    a.cin = cin_[l];
    a.cout = cout_[l];
    a.bias = w + boff[l];
    a.out = act[L.out];
    a.relu = L.relu;
    a.transposed = 0;
  } else {
    a.src[0].p = gz;
    a.src[0].nc = cout_[l];
    a.src[0].mode = SRC_DIRECT;
    a.src[1].nc = 0;
    a.cin = cout_[l];
    a.cout = cin_[l];
    a.bias = nullptr;
    a.out = gx;
    a.relu = 0;
    a.transposed = 1;
  }
  return a;
}

cudaError_t NetState::forward(const float* x, float* y) {
  cudaError_t e = cudaMemcpyAsync(act[T_X], x, (size_t)kNetInputs * H * W * sizeof(float),
                                  cudaMemcpyDeviceToDevice, stream);
  for (int l = 0; l < kNetLayers && e == cudaSuccess; ++l) e = launch_conv(conv_args(l, false), stream);
  if (e == cudaSuccess && y)
    e = cudaMemcpyAsync(y, act[T_Y], (size_t)H * W * sizeof(float), cudaMemcpyDeviceToDevice, stream);
  return e;
}

// Accumulates the parameter gradients of one sample into g, given the
// gradient of the loss with respect to the output, already in grad[T_Y].
cudaError_t NetState::backward() {
  cudaError_t e = cudaSuccess;
  for (int t = 0; t < T_COUNT - 1 && e == cudaSuccess; ++t) {
    const size_t n = (size_t)channels(t) * (H >> level(t)) * (W >> level(t));
    e = cudaMemsetAsync(grad[t], 0, n * sizeof(float), stream);
  }
  for (int l = kNetLayers - 1; l >= 0 && e == cudaSuccess; --l) {
    const LayerSpec& L = kLayers[l];
    const int lev = level(L.out);
    const int h = H >> lev, wd = W >> lev;
    const long long n = (long long)cout_[l] * h * wd;
    if (L.relu) e = launch_relu_mask(grad[L.out], act[L.out], gz, n, stream);
    else e = cudaMemcpyAsync(gz, grad[L.out], n * sizeof(float), cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) break;
    e = launch_conv_wgrad(conv_args(l, false), gz, part, bpart, g + woff[l], g + boff[l], 1, stream);
    if (e != cudaSuccess || l == 0) continue;   // the input features need no gradient
    e = launch_conv(conv_args(l, true), stream);
    int c_off = 0;
    for (int j = 0; j < 2 && e == cudaSuccess; ++j) {
      if (L.src[j] < 0) continue;
      const int nc = channels(L.src[j]);
      e = launch_scatter(gx, c_off, nc, L.mode[j], h, wd, grad[L.src[j]], stream);
      c_off += nc;
    }
  }
  return e;
}

cudaError_t NetState::loss_grad(const float* xs, const float* ts, int batch, double* loss) {
  cudaError_t e = cudaMemsetAsync(g, 0, nparams * sizeof(float), stream);
  const long long npix = (long long)H * W;
  double total = 0.0;
  std::vector<double> lp(kLossBlocks);
  for (int b = 0; b < batch && e == cudaSuccess; ++b) {
    e = forward(xs + (size_t)b * kNetInputs * npix, nullptr);
    if (e == cudaSuccess)
      e = launch_mse(act[T_Y], ts + (size_t)b * npix, grad[T_Y], npix, 1.f / (float)(npix * batch),
                     lpart, kLossBlocks, stream);
    if (e == cudaSuccess) e = backward();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(lp.data(), lpart, kLossBlocks * sizeof(double), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    for (double x : lp) total += x;
  }
  if (loss) *loss = total / ((double)npix * batch);
  return e;
}

cudaError_t NetState::train_step(const float* xs, const float* ts, int batch, float lr, double* loss) {
  cudaError_t e = loss_grad(xs, ts, batch, loss);
  if (e == cudaSuccess) e = launch_adam(w, wb, g, m, v, nparams, lr, ++step, stream);
  return e;
}

}  // namespace fl

// --- C ABI ---------------------------------------------------------------------

struct fl_net : public fl::NetState {};

namespace {
thread_local std::string g_net_err;
fl_status net_fail(fl_status s, const std::string& m) {
  g_net_err = m;
  fl_set_error_string(m.c_str());
  return s;
}
fl_status net_cuda(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return FL_OK;
  return net_fail(e == cudaErrorMemoryAllocation ? FL_OOM : FL_CUDA_ERROR,
                  std::string(where) + ": " + cudaGetErrorString(e));
}
const uint32_t kMagic = 0x464c4e54;  // "FLNT"
uint64_t fnv1a(const void* p, size_t n) {
  const unsigned char* c = (const unsigned char*)p;
  uint64_t h = 1469598103934665603ULL;
  for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ULL;
  return h;
}
}  // namespace

extern "C" {

fl_status fl_net_create(int H, int W, uint64_t seed, void* stream, fl_net** out) {
  if (!out) return net_fail(FL_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (H < 64 || W < 64 || H % 64 || W % 64 || H > 4096 || W > 4096)
    return net_fail(FL_INVALID_ARG, "H and W must be multiples of 64 in [64, 4096]");
  fl_net* n = new fl_net();
  cudaError_t e = n->init(H, W, seed, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    delete n;
    return net_cuda(e, "fl_net_create");
  }
  *out = n;
  return FL_OK;
}

fl_status fl_net_destroy(fl_net* n) {
  if (n) {
    cudaStreamSynchronize(n->stream);
    delete n;
  }
  return FL_OK;
}

long long fl_net_num_params(const fl_net* n) { return n ? n->nparams : 0; }

fl_status fl_net_get_params(fl_net* n, float* host, float* grads_host) {
  if (!n || (!host && !grads_host)) return net_fail(FL_INVALID_ARG, "NULL argument");
  if (host) {
    fl_status s = net_cuda(cudaMemcpyAsync(host, n->w, n->nparams * sizeof(float),
                                           cudaMemcpyDeviceToHost, n->stream), "get params");
    if (s != FL_OK) return s;
  }
  if (grads_host) {
    fl_status s = net_cuda(cudaMemcpyAsync(grads_host, n->g, n->nparams * sizeof(float),
                                           cudaMemcpyDeviceToHost, n->stream), "get grads");
    if (s != FL_OK) return s;
  }
  return net_cuda(cudaStreamSynchronize(n->stream), "sync");
}

fl_status fl_net_set_params(fl_net* n, const float* host) {
  if (!n || !host) return net_fail(FL_INVALID_ARG, "NULL argument");
  cudaError_t e = cudaMemcpyAsync(n->w, host, n->nparams * sizeof(float), cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess) e = fl::launch_to_bf16(n->w, n->wb, n->nparams, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, n->nparams * sizeof(float), n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, n->nparams * sizeof(float), n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  n->step = 0;
  return net_cuda(e, "fl_net_set_params");
}

fl_status fl_net_forward(fl_net* n, const float* x_dev, float* y_dev) {
  if (!n || !x_dev || !y_dev) return net_fail(FL_INVALID_ARG, "NULL argument");
  return net_cuda(n->forward(x_dev, y_dev), "fl_net_forward");
}

fl_status fl_net_loss_grad(fl_net* n, const float* xs_dev, const float* ts_dev, int batch,
                           double* loss) {
  if (!n || !xs_dev || !ts_dev || batch < 1) return net_fail(FL_INVALID_ARG, "bad argument");
  return net_cuda(n->loss_grad(xs_dev, ts_dev, batch, loss), "fl_net_loss_grad");
}

fl_status fl_net_train_step(fl_net* n, const float* xs_dev, const float* ts_dev, int batch, float lr,
                            double* loss) {
  if (!n || !xs_dev || !ts_dev || batch < 1 || !(lr > 0.f)) return net_fail(FL_INVALID_ARG, "bad argument");
  return net_cuda(n->train_step(xs_dev, ts_dev, batch, lr, loss), "fl_net_train_step");
}

fl_status fl_net_save(fl_net* n, const char* path) {
  if (!n || !path) return net_fail(FL_INVALID_ARG, "NULL argument");
  std::vector<float> host(n->nparams);
  fl_status s = fl_net_get_params(n, host.data(), nullptr);
  if (s != FL_OK) return s;
  FILE* f = fopen(path, "wb");
  if (!f) return net_fail(FL_INVALID_ARG, std::string("cannot open ") + path);
  const uint32_t hdr[4] = {kMagic, 1u, (uint32_t)n->nparams, (uint32_t)n->step};
  const uint64_t sum = fnv1a(host.data(), host.size() * sizeof(float));
  bool ok = fwrite(hdr, sizeof(hdr), 1, f) == 1 && fwrite(&sum, sizeof(sum), 1, f) == 1 &&
            fwrite(host.data(), sizeof(float), host.size(), f) == host.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? FL_OK : net_fail(FL_INVALID_ARG, "write failed");
}

fl_status fl_net_load(fl_net* n, const char* path) {
  if (!n || !path) return net_fail(FL_INVALID_ARG, "NULL argument");
  FILE* f = fopen(path, "rb");
  if (!f) return net_fail(FL_INVALID_ARG, std::string("cannot open ") + path);
  uint32_t hdr[4];
  uint64_t sum = 0;
  std::vector<float> host(n->nparams);
  bool ok = fread(hdr, sizeof(hdr), 1, f) == 1 && fread(&sum, sizeof(sum), 1, f) == 1;
  ok = ok && hdr[0] == kMagic && hdr[1] == 1u && hdr[2] == (uint32_t)n->nparams;
  ok = ok && fread(host.data(), sizeof(float), host.size(), f) == host.size();
  fclose(f);
  if (!ok) return net_fail(FL_INVALID_ARG, "not a network file of this architecture");
  if (fnv1a(host.data(), host.size() * sizeof(float)) != sum)
    return net_fail(FL_INVALID_ARG, "network file checksum mismatch");
  fl_status s = fl_net_set_params(n, host.data());
  if (s == FL_OK) n->step = (int)hdr[3];
  return s;
}

}  // extern "C"

// --- kernels of the learned flexible CG ------------------------------------------

namespace fl {

namespace {

// Features of the network: x[0] = r / s_r, x[1] = z0 / s_z, x[2] = alpha,
// with s = root mean square from the partial sums of squares.
__global__ void __launch_bounds__(256) k_features(const float* __restrict__ r, const float* __restrict__ z0,
                                                   const double* __restrict__ rr_part, int rr_count,
                                                   const double* __restrict__ zz_part, int zz_count,
                                                   float alpha, float* __restrict__ x, long long N,
                                                   const PcgState* st) {
  __shared__ double red[32];
  if (st && st->done) return;
  const double rr = cta_sum_partials(rr_part, rr_count, red);
  const double zz = cta_sum_partials(zz_part, zz_count, red);
  const float ir = rr > 0 ? (float)rsqrt(rr / (double)N) : 0.f;
  const float iz = zz > 0 ? (float)rsqrt(zz / (double)N) : 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    x[i] = r[i] * ir;
    x[N + i] = z0[i] * iz;
    x[2 * N + i] = alpha;
  }
}

// z_new = z0 + s_z y; partials of r . z_new and r . z_old (z_old = z before
// the overwrite).
__global__ void __launch_bounds__(256) k_combine(const float* __restrict__ r, const float* __restrict__ z0,
                                                  const float* __restrict__ y, float* __restrict__ z,
                                                  const double* __restrict__ zz_part, int zz_count,
                                                  double* __restrict__ rz_part, double* __restrict__ rzo_part,
                                                  long long N, const PcgState* st) {
  __shared__ double red[32];
  if (st && st->done) return;
  const double zz = cta_sum_partials(zz_part, zz_count, red);
  const float sz = (float)sqrt(zz / (double)N);
  DotAcc<float> a, b;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const float zo = z[i];
    const float zn = z0[i] + sz * y[i];
    z[i] = zn;
    a.add(r[i] * zn);
    b.add(r[i] * zo);
  }
  const double sa = a.cta_total(red);
  const double sb = b.cta_total(red);
  if (threadIdx.x == 0) {
    rz_part[blockIdx.x] = sa;
    if (rzo_part) rzo_part[blockIdx.x] = sb;
  }
}

// dst = scale * src
__global__ void k_scale(const float* __restrict__ src, float* __restrict__ dst, float scale, long long N,
                        const PcgState* st) {
  if (st && st->done) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = scale * src[i];
}

// Flexible CG scalars: beta = (r.z_new - r.z_old) / rz (Polak-Ribiere),
// convergence on ||r||, breakdown when r.z_new <= 0 (then the caller falls
// back to the fixed preconditioner).
__global__ void k_fpcg_scalar(PcgState* st, const double* rr_part, int rr_count, const double* rz_part,
                              const double* rzo_part, int rz_count) {
  __shared__ double red[32];
  if (st->done) return;
  const double rr = cta_sum_partials(rr_part, rr_count, red);
  const double rz = cta_sum_partials(rz_part, rz_count, red);
  const double rzo = cta_sum_partials(rzo_part, rz_count, red);
  if (threadIdx.x == 0) {
    st->it += 1;
    st->rr = rr;
    if (!(st->pq > 0.0) || rr != rr || rz != rz) {
      st->done = 1;
      st->status = 3;
    } else if (rr <= st->tol2) {
      st->done = 1;
      st->status = 0;
    } else if (st->it >= st->maxit) {
      st->done = 1;
      st->status = 2;
    } else if (!(rz > 0.0)) {
      st->done = 1;
      st->status = 4;   // learned direction not a descent direction: fall back
    } else {
      st->beta = (rz - rzo) / st->rz;
      st->rz = rz;
    }
  }
}

constexpr int kFBlocks = 608;

// Training pairs (fl_net_training_pair).  z0 = r / k0: the diagonal base
// preconditioner of orders alpha < 1.
__global__ void __launch_bounds__(256) k_div_scalar(const double* __restrict__ r, double k0,
                                                     double* __restrict__ z0, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    z0[i] = r[i] / k0;
}

// Per-CTA partial sums of r^2 (part[b]) and z0^2 (part[G + b]).
__global__ void __launch_bounds__(256) k_pair_sums(const double* __restrict__ r,
                                                    const double* __restrict__ z0, long long N,
                                                    double* __restrict__ part) {
  __shared__ double red[32];
  double a = 0.0, b = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    a += r[i] * r[i];
    b += z0[i] * z0[i];
  }
  a = cta_sum(a, red);
  __syncthreads();
  b = cta_sum(b, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = a;
    part[gridDim.x + blockIdx.x] = b;
  }
}

// Features [r / s_r, z0 / s_z, alpha] and target (u* - x - z0) / s_z, in
// FP32, with s = max(root mean square, 1e-300) from the partials (summed in
// a fixed order by every CTA).
__global__ void __launch_bounds__(256) k_pair_write(const double* __restrict__ r,
                                                     const double* __restrict__ z0,
                                                     const double* __restrict__ u_star,
                                                     const double* __restrict__ x,
                                                     const double* __restrict__ part, int G,
                                                     double alpha, float* __restrict__ feat,
                                                     float* __restrict__ target, long long N) {
  __shared__ double red[32];
  const double rr = cta_sum_partials(part, G, red);
  const double zz = cta_sum_partials(part + G, G, red);
  const double sr = fmax(sqrt(rr / (double)N), 1e-300);
  const double sz = fmax(sqrt(zz / (double)N), 1e-300);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    feat[i] = (float)(r[i] / sr);
    feat[N + i] = (float)(z0[i] / sz);
    feat[2 * N + i] = (float)alpha;
    target[i] = (float)(((u_star[i] - x[i]) - z0[i]) / sz);
  }
}

constexpr int kPairBlocks = 256;

}  // namespace

cudaError_t launch_div_scalar(const double* r, double k0, double* z0, long long N, cudaStream_t s) {
  FL_KERNEL("div_scalar", s, k_div_scalar<<<kFBlocks, 256, 0, s>>>(r, k0, z0, N));
  return cudaGetLastError();
}

cudaError_t launch_training_pair(const double* r, const double* z0, const double* u_star, const double* x,
                                 double alpha, float* feat, float* target, long long N, double* part,
                                 cudaStream_t s) {
  FL_KERNEL("pair_sums", s, k_pair_sums<<<kPairBlocks, 256, 0, s>>>(r, z0, N, part));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  FL_KERNEL("pair_write", s,
            k_pair_write<<<kFBlocks, 256, 0, s>>>(r, z0, u_star, x, part, kPairBlocks, alpha, feat,
                                                  target, N));
  return cudaGetLastError();
}

cudaError_t launch_features(const float* r, const float* z0, const double* rr_part, int rr_count,
                            const double* zz_part, int zz_count, float alpha, float* x, long long N,
                            const PcgState* st, cudaStream_t s) {
  FL_KERNEL("features", s,
            k_features<<<kFBlocks, 256, 0, s>>>(r, z0, rr_part, rr_count, zz_part, zz_count, alpha, x, N, st));
  return cudaGetLastError();
}

cudaError_t launch_combine(const float* r, const float* z0, const float* y, float* z, const double* zz_part,
                           int zz_count, double* rz_part, double* rzo_part, long long N, const PcgState* st,
                           int* count, cudaStream_t s) {
  FL_KERNEL("combine", s,
            k_combine<<<kFBlocks, 256, 0, s>>>(r, z0, y, z, zz_part, zz_count, rz_part, rzo_part, N, st));
  *count = kFBlocks;
  return cudaGetLastError();
}

cudaError_t launch_scale(const float* src, float* dst, float scale, long long N, const PcgState* st,
                         cudaStream_t s) {
  FL_KERNEL("scale", s, k_scale<<<kFBlocks, 256, 0, s>>>(src, dst, scale, N, st));
  return cudaGetLastError();
}

cudaError_t launch_fpcg_scalar(PcgState* st, const double* rr_part, int rr_count, const double* rz_part,
                               const double* rzo_part, int rz_count, cudaStream_t s) {
  FL_KERNEL("fpcg_scalar", s, k_fpcg_scalar<<<1, 256, 0, s>>>(st, rr_part, rr_count, rz_part, rzo_part,
                                                               rz_count));
  return cudaGetLastError();
}

}  // namespace fl

fl::NetState* fl_net_state(fl_net* n) { return n; }

extern "C" {

bool fl::NetState::alpha_enabled(double alpha) const {
  if (gate.empty()) return true;
  if (!(alpha >= gate_lo && alpha < gate_hi)) return false;
  const int b = std::min((int)gate.size() - 1,
                         (int)((alpha - gate_lo) / (gate_hi - gate_lo) * (double)gate.size()));
  return gate[b] != 0;
}

fl_status fl_net_set_alpha_gate(fl_net* n, double lo, double hi, int bands, const uint8_t* enabled) {
  if (!n) return net_fail(FL_INVALID_ARG, "NULL net");
  if (bands == 0) {
    n->gate.clear();
    return FL_OK;
  }
  if (bands < 0 || bands > 4096 || !enabled || !std::isfinite(lo) || !std::isfinite(hi) || !(lo < hi))
    return net_fail(FL_INVALID_ARG, "alpha gate: need lo < hi (finite), 0 < bands <= 4096, enabled != NULL");
  n->gate_lo = lo;
  n->gate_hi = hi;
  n->gate.assign(enabled, enabled + bands);
  return FL_OK;
}

fl_status fl_net_set_tensor_cores(fl_net* n, int enable) {
  if (!n) return net_fail(FL_INVALID_ARG, "NULL net");
  n->use_tc = enable ? 1 : 0;
  return FL_OK;
}

fl_status fl_net_get_tensor(fl_net* n, int kind, int index, float* host, long long count) {
  if (!n || !host) return net_fail(FL_INVALID_ARG, "NULL argument");
  if ((kind != 0 && kind != 1) || index < 0 || index >= fl::kNetTensors)
    return net_fail(FL_INVALID_ARG, "kind must be 0 or 1 and index in [0, 12)");
  const long long size = (long long)n->channels(index) * (n->H >> n->level(index)) * (n->W >> n->level(index));
  if (count != size) return net_fail(FL_INVALID_ARG, "count differs from the tensor's size");
  const float* src = kind == 0 ? n->act[index] : n->grad[index];
  fl_status s = net_cuda(cudaMemcpyAsync(host, src, size * sizeof(float), cudaMemcpyDeviceToHost, n->stream),
                         "fl_net_get_tensor");
  if (s == FL_OK) s = net_cuda(cudaStreamSynchronize(n->stream), "fl_net_get_tensor");
  return s;
}

fl_status fl_net_check(fl_net* n) {
  if (!n) return net_fail(FL_INVALID_ARG, "NULL net");
  int flag = 0;
  fl_status s = net_cuda(cudaMemcpyAsync(&flag, n->err, sizeof(int), cudaMemcpyDeviceToHost, n->stream),
                         "fl_net_check");
  if (s == FL_OK) s = net_cuda(cudaStreamSynchronize(n->stream), "fl_net_check");
  if (s == FL_OK && flag) return net_fail(FL_DEVICE_TIMEOUT, "a tensor-core wait gave up");
  return s;
}

}  // extern "C"
