// Kernel launchers: the operator apply chain, the preconditioner chain, CG
// vector and scalar kernels, and the plan-time symbol build.
//
// The file is compiled twice (in parallel): FL_OPS_PART=1 holds the FP32
// instantiations and the precision-free kernels, FL_OPS_PART=2 the FP64
// instantiations and the plan-time symbol build.
#include <algorithm>

#ifndef FL_OPS_PART
#define FL_OPS_PART 1
#endif

#include "chain.cuh"

namespace fl {

// Launch the pass kernel template KERNEL<T, THREADS, VPT, LGLO> with the
// shape row_threads<T>(L) (ROWS) or col_threads<T>(L) (COLS): the Cfg shape,
// or the wide instantiations that hold one line of 2x or 4x its values.
#define FL_SHAPED_LAUNCH(KERNEL, T, BASE, V, L, grid, smem, s, arg)                          \
  do {                                                                                      \
    constexpr int b0_ = (BASE), v0_ = (V);                                                  \
    if ((L) <= b0_ * v0_) {                                                                 \
      pdl_launch(KERNEL<T, b0_, v0_>, grid, b0_, smem, s, arg);                             \
    } else if ((L) == 2 * b0_ * v0_) {                                                      \
      if constexpr (2 * b0_ * v0_ <= kMaxLen)                                               \
        pdl_launch(KERNEL<T, 2 * b0_, v0_, clog2(2 * b0_ * v0_)>, grid, 2 * b0_, smem, s, arg); \
    } else {                                                                                \
      if constexpr (4 * b0_ * v0_ <= kMaxLen)                                               \
        pdl_launch(KERNEL<T, 4 * b0_, v0_, clog2(4 * b0_ * v0_)>, grid, 4 * b0_, smem, s, arg); \
    }                                                                                       \
  } while (0)
#define FL_ROWS_LAUNCH(KERNEL, T, L, grid, smem, s, arg) \
  FL_SHAPED_LAUNCH(KERNEL, T, Cfg<T>::RT, Cfg<T>::RV, L, grid, smem, s, arg)
#define FL_COLS_LAUNCH(KERNEL, T, L, grid, smem, s, arg) \
  FL_SHAPED_LAUNCH(KERNEL, T, Cfg<T>::CT, Cfg<T>::CV, L, grid, smem, s, arg)

// ---------------------------------------------------------------------------
// CG vector kernels (grid-stride, kVecBlocks CTAs, one partial per CTA).

// CG update without preconditioner (z = r): x += alpha p, r -= alpha q with
// alpha = st->alpha (set by the apply's last CTA), partials of ||r||^2;
// with `step` the last CTA takes the CG scalar step (r.z = ||r||^2).
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_noprec_update(PcgState* st, T* x, T* r, const T* p,
                                                              const T* q, double* rr_part, int step,
                                                              long long N) {
  __shared__ double red[32];
  pdl_wait();
  if (st->done) return;
  const T al = (T)st->alpha;
  DotAcc<T> rr;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    x[i] += al * p[i];
    const T rn = r[i] - al * q[i];
    r[i] = rn;
    rr.add(rn * rn);
  }
  const double s = rr.cta_total(red);
  if (threadIdx.x == 0) rr_part[blockIdx.x] = s;
  if (step && arrive_last(&st->arrive, gridDim.x)) {
    const double rrv = cta_sum_partials(rr_part, gridDim.x, red);
    if (threadIdx.x == 0) pcg_step(st, rrv, rrv);
  }
}

template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_dot(const T* a, const T* b, double* part,
                                                    long long N) {
  __shared__ double red[32];
  DotAcc<T> v;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    v.add(a[i] * b[i]);
  const double s = v.cta_total(red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename T>
__global__ void k_copy_cast(const double* src, T* dst, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (T)src[i];
}

template <typename T>
__global__ void k_axpby(double a, const T* x, double b, T* y, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (T)(a * (double)x[i] + b * (double)y[i]);
}

// dst = mask ? src : 0 (dst nullable), per-CTA partials of sum (masked src)^2.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_mask_copy_dot(const T* src, const uint8_t* mask, T* dst,
                                                              double* part, long long N) {
  __shared__ double red[32];
  DotAcc<T> v;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const T x = (mask && !mask[i]) ? (T)0 : src[i];
    if (dst) dst[i] = x;
    v.add(x * x);
  }
  const double s = v.cta_total(red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

#if FL_OPS_PART == 1
// Scalar bookkeeping of CG (one CTA).
__global__ void k_pcg_init(PcgState* st, const double* bb_part, int bb_count, const double* rr_part,
                           int rr_count, const double* rz_part, int rz_count, double tol, int maxit) {
  __shared__ double red[32];
  const double bb = cta_sum_partials(bb_part, bb_count, red);
  const double rr = cta_sum_partials(rr_part, rr_count, red);
  const double rz = cta_sum_partials(rz_part, rz_count, red);
  if (threadIdx.x == 0) {
    st->bb = bb;
    st->rr = rr;
    st->rz = rz;
    st->tol2 = tol * tol * bb;
    st->beta = 0.0;
    st->alpha = 0.0;
    st->pq = 0.0;
    st->it = 0;
    st->maxit = maxit;
    st->status = 0;
    st->arrive = 0u;
    st->done = (bb == 0.0 || rr <= st->tol2) ? 1 : 0;
    if (!(rz > 0.0) && !st->done) { st->done = 1; st->status = 3; }
  }
}

__global__ void __launch_bounds__(kVecThreads) k_residual_from(const double* b, const double* u,
                                                                const double* mx, const uint8_t* mask,
                                                                double shift, double scale, float* r32,
                                                                double* part, long long N) {
  __shared__ double red[32];
  double v = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const double r = (mask && !mask[i]) ? 0.0 : b[i] - shift * u[i] - scale * mx[i];
    r32[i] = (float)r;
    v += r * r;
  }
  const double s = cta_sum(v, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_axmy(const double* u, double c, const double* mx, double* y, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = u[i] - c * mx[i];
}

// The splitmix64 finaliser (Steele, Lea, Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014): a bijective 64-bit mixer.
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// Sum over i of mix64(bits(u_i) ^ mix64(i)) mod 2^64: independent of the
// summation order; any change of the values changes their terms
// pseudo-randomly (a uniform change, such as scaling the whole array by a
// power of two, does not cancel out as it would with linear weights).
__global__ void k_hash(const double* u, unsigned long long* h, long long N) {
  unsigned long long acc = 0ull;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    acc += mix64((unsigned long long)__double_as_longlong(u[i]) ^ mix64((unsigned long long)i));
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(h, acc);
}

// v_i = prod_a sin(pi k_a (i_a + 1) / (n_a + 1)) with k_a = 1 (lowest mode)
// or k_a = n_a (highest), 0 off Omega: the separable DST-I eigenvectors of
// the FD Laplacian with the smallest and the largest eigenvalue.
__global__ void k_sine_mode(double* v, const uint8_t* mask, int d, int n0, int n1, int n2, int hi,
                            long long N) {
  const int ns[3] = {n0, n1, n2};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    long long rem = i;
    double val = 1.0;
    for (int ax = d - 1; ax >= 0; --ax) {
      const long long j = rem % ns[ax];
      rem /= ns[ax];
      const long long k = hi ? ns[ax] : 1;
      val *= sinpi((double)(k * (j + 1)) / (double)(ns[ax] + 1));
    }
    v[i] = (mask && !mask[i]) ? 0.0 : val;
  }
}

__global__ void k_sum(const double* part, int count, double* out) {
  __shared__ double red[32];
  const double s = cta_sum_partials(part, count, red);
  if (threadIdx.x == 0) *out = s;
}

#endif  // FL_OPS_PART == 1

#if FL_OPS_PART == 2
// ---------------------------------------------------------------------------
// Plan-time symbol: fill the circular embedding of k(m) (FP64, complex),
// FFT along every axis, keep the real part on [0, L_i/2]^d / prod L.

// Circular embedding of the kernel (grid units, c = C h^{-alpha}):
// k(0) = c (Z - 2d a), k(m) = c (-|m|^{-expo} + a [|m|_1 = 1]) for
// 0 < |m_i| <= n_i - 1, zero elsewhere (including the index L_i / 2);
// expo = d + alpha.
__global__ void k_fill_kernel(double2* buf, int d, int L0, int L1, int L2, int n0, int n1, int n2,
                               double c, double Z, double a, double expo, int dphys,
                               long long total) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int Ls[3] = {L0, L1, L2};
  const int ns[3] = {n0, n1, n2};
  long long rem = i;
  int m[3] = {0, 0, 0};
  for (int ax = d - 1; ax >= 0; --ax) {
    const int idx = (int)(rem % Ls[ax]);
    rem /= Ls[ax];
    m[ax] = idx <= Ls[ax] / 2 ? idx : idx - Ls[ax];
  }
  bool inside = true;
  double r2 = 0.0;
  int l1 = 0;
  for (int ax = 0; ax < d; ++ax) {
    if (abs(m[ax]) > ns[ax] - 1) inside = false;
    r2 += (double)m[ax] * m[ax];
    l1 += abs(m[ax]);
  }
  double v = 0.0;
  if (inside) {
    if (l1 == 0) v = c * (Z - 2.0 * dphys * a);
    else v = c * (-pow(r2, -0.5 * expo) + (l1 == 1 ? a : 0.0));
  }
  buf[i] = make_double2(v, 0.0);
}

template <int THREADS, int VPT>
__global__ void __launch_bounds__(THREADS) k_rows_c2c(double2* buf, int rows, int lg, int lgmax,
                                                     const double2* tw) {
  constexpr int LGC = clog2(THREADS * VPT);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SBuf<double2> sb{reinterpret_cast<double2*>(smem_raw)};
  const int L = 1 << lg, ls = L;
  const int NL = (VPT * THREADS) / L;
  const int r0 = blockIdx.x * NL;
  const int nl = min(NL, rows - r0);
  for (int e = threadIdx.x; e < nl * L; e += THREADS) {
    const int q = e / L, j = e - q * L;
    sb[q * ls + j] = buf[(size_t)(r0 + q) * L + j];
  }
  __syncthreads();
  fft_smem<VPT, false, LGC>(sb, lg, ls, 0, nl, tw, lgmax, false);
  for (int e = threadIdx.x; e < nl * L; e += THREADS) {
    const int q = e / L, j = e - q * L;
    buf[(size_t)(r0 + q) * L + j] = sb[q * ls + j];
  }
}

__global__ void k_extract_symbol(const double2* buf, int d, int L0, int L1, int L2, double inv,
                                 double* sig64, float* sig32, long long total) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int Ls[3] = {L0, L1, L2};
  long long rem = i, src = 0, mul = 1;
  for (int ax = d - 1; ax >= 0; --ax) {
    const int h = Ls[ax] / 2 + 1;
    const int k = (int)(rem % h);
    rem /= h;
    src += (long long)k * mul;
    mul *= Ls[ax];
  }
  const double v = buf[src].x * inv;
  sig64[i] = v;
  sig32[i] = (float)v;
}

// ---------------------------------------------------------------------------

#endif  // FL_OPS_PART == 2

// Large dynamic shared memory and the whole L1/shared carveout as shared
// memory, so that as many FFT tiles as fit are resident per SM.
static cudaError_t set_smem(const void* f) {
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  return e;
}

#if FL_OPS_PART == 1
cudaError_t configure_kernels_f64();

cudaError_t configure_kernels() {
  cudaError_t e = configure_kernels_f64();
  if (e == cudaSuccess) e = configure_rows_w8();
#define FL_SET(...)                                                         \
  if (e == cudaSuccess) e = set_smem(reinterpret_cast<const void*>(&__VA_ARGS__));
  FL_SET(k_rows_fwd<float, Cfg<float>::RT, Cfg<float>::RV>);
  FL_SET(k_rows_inv<float, Cfg<float>::RT, Cfg<float>::RV>);
  FL_SET(k_cols<float, Cfg<float>::CT, Cfg<float>::CV>);
  FL_SET(k_dst_rows<float, Cfg<float>::RT, Cfg<float>::RV>);
  FL_SET(k_dst_cols<float, Cfg<float>::CT, Cfg<float>::CV>);
  // the wide instantiations of the longest lines
  FL_SET(k_rows_fwd<float, 256, 16, 12>);
  FL_SET(k_rows_fwd<float, 512, 16, 13>);
  FL_SET(k_rows_inv<float, 256, 16, 12>);
  FL_SET(k_rows_inv<float, 512, 16, 13>);
  FL_SET(k_dst_rows<float, 256, 16, 12>);
  FL_SET(k_dst_rows<float, 512, 16, 13>);
#undef FL_SET
  return e;
}
#else
cudaError_t configure_kernels_f64() {
  cudaError_t e = cudaSuccess;
#define FL_SET(...)                                                         \
  if (e == cudaSuccess) e = set_smem(reinterpret_cast<const void*>(&__VA_ARGS__));
  FL_SET(k_rows_fwd<double, Cfg<double>::RT, Cfg<double>::RV>);
  FL_SET(k_rows_inv<double, Cfg<double>::RT, Cfg<double>::RV>);
  FL_SET(k_cols<double, Cfg<double>::CT, Cfg<double>::CV>);
  FL_SET(k_dst_rows<double, Cfg<double>::RT, Cfg<double>::RV>);
  FL_SET(k_dst_cols<double, Cfg<double>::CT, Cfg<double>::CV>);
  FL_SET(k_rows_c2c<Cfg<double>::RT, Cfg<double>::RV>);
  FL_SET(k_rows_fwd<double, 512, 16, 13>);
  FL_SET(k_rows_inv<double, 512, 16, 13>);
  FL_SET(k_dst_rows<double, 512, 16, 13>);
  FL_SET(k_cols<double, 512, 16, 13>);
  FL_SET(k_dst_cols<double, 512, 16, 13>);
  FL_SET(k_rows_c2c<2 * Cfg<double>::RT, Cfg<double>::RV>);
#undef FL_SET
  return e;
}
#endif

#if FL_OPS_PART == 1
bool pdl_enabled() {
  static const bool on = [] {
    const char* v = getenv("FRACLAP_PDL");
    return !(v && v[0] == '0');
  }();
  return on;
}

namespace {
thread_local cudaError_t t_launch_err = cudaSuccess;
}
void note_launch_error(cudaError_t e) {
  if (e != cudaSuccess && t_launch_err == cudaSuccess) t_launch_err = e;
}
cudaError_t take_launch_error() {
  const cudaError_t e = t_launch_err;
  t_launch_err = cudaSuccess;
  return e;
}

size_t partial_capacity(const Geo& g) {
  long long rows = g.N / g.n[g.d - 1];
  size_t c = (size_t)kVecBlocks;
  // row kernels of both precisions: one partial per CTA
  const int L = g.L[g.d - 1];
  c = std::max(c, (size_t)((rows + 1) / 2 + 1));
  c = std::max(c, (size_t)(rows / std::max(1, row_lines<double>(L)) + 2));
  c = std::max(c, (size_t)(rows / std::max(1, row_lines<float>(L)) + 2));
  return c;
}

#endif  // FL_OPS_PART == 1

template <typename T>
int apply_partials(const Geo& g) {
  const long long rows = g.N / g.n[g.d - 1];
  const int NL = row_lines<T>(g.L[g.d - 1]);
  return (int)(((rows + 1) / 2 + NL - 1) / NL);
}

template <typename T>
int precond_partials(const Geo& g) {
  const long long rows = g.N / g.n[g.d - 1];
  const int NL = row_lines<T>(g.L[g.d - 1]);
  return (int)((rows + NL - 1) / NL);
}

template <typename T>
ApplyChain<T> build_apply(const Geo& g, const Tables<T>& tb, const ApplyIO<T>& io) {
  ApplyChain<T> ch;
  const int d = g.d;
  const int Lx = g.L[d - 1];
  const long long rows = g.N / g.n[d - 1];
  const int NL = row_lines_at<T>(Lx, io.row_threads);
  ch.row_blocks = (int)(((rows + 1) / 2 + NL - 1) / NL);
  ch.row_smem = smem_bytes<T>(NL, Lx);
  const int rpp = d == 3 ? g.n[1] : (int)rows;
  const int pstride = d == 3 ? g.L[1] : 0;
  {
    RowsFwdArgs<T>& a = ch.fwd;
    a.u = io.u; a.p = io.p; a.acc = io.acc; a.x32 = io.x32; a.mask = io.mask;
    a.S = tb.S; a.tw = tb.tw; a.st = io.st;
    a.rows = (int)rows; a.n = g.n[d - 1]; a.H = g.H; a.lg = g.lg[d - 1]; a.lgmax = g.lgmax;
    a.rows_per_plane = rpp; a.plane_stride = pstride; a.pre = io.pre;
  }
  ch.ncols = 0;
  auto cols = [&](int axis, int mode, int rows_in, int rows_out, long long lstride,
                  long long ostride, int nouter, long long sig_line, long long sig_outer, int Lo) {
    ColsArgs<T>& a = ch.cols[ch.ncols];
    a.S = tb.S; a.tw = tb.tw; a.sig = tb.sig; a.st = io.st;
    a.H = g.H; a.lg = g.lg[axis]; a.lgmax = g.lgmax;
    a.rows_in = rows_in; a.rows_out = rows_out; a.lstride = lstride; a.ostride = ostride;
    a.nouter = nouter; a.mode = mode; a.sig_line = sig_line; a.sig_outer = sig_outer; a.Lo = Lo;
    const int L = g.L[axis];
    const int tx = tile_at<T>(plan_tx<T>(tb, axis, L), L, io.col_threads);
    a.ltx = ilog2i(tx);
    ch.cols_grid[ch.ncols] = dim3((g.H + tx - 1) / tx, nouter);
    ch.cols_smem[ch.ncols] = mode == COLS_CONV ? conv_tile_bytes<T>(tx, L) : cols_bytes<T>(tx, L);
    ch.ncols++;
  };
  if (d == 2) {
    cols(0, COLS_CONV, g.n[0], g.n[0], g.H, 0, 1, g.H, 0, 0);
  } else {
    const long long H = g.H, L1 = g.L[1];
    cols(1, COLS_FWD, g.n[1], g.L[1], H, L1 * H, g.n[0], 0, 0, 0);
    cols(0, COLS_CONV, g.n[0], g.n[0], L1 * H, H, g.L[1], (L1 / 2 + 1) * H, H, g.L[1]);
    cols(1, COLS_INV, g.L[1], g.n[1], H, L1 * H, g.n[0], 0, 0, 0);
  }
  {
    RowsInvArgs<T>& a = ch.inv;
    a.S = tb.S; a.tw = tb.tw; a.mask = io.mask; a.st = io.st;
    a.out = io.out; a.out32 = io.out32;
    // the epilogue's x is the apply input (after any pre-op)
    a.x = io.x; a.b = io.b; a.dotw = io.dotw; a.partials = io.partials;
    a.cm = io.cm; a.cx = io.cx; a.cb = io.cb;
    a.rows = (int)rows; a.n = g.n[d - 1]; a.H = g.H; a.lg = g.lg[d - 1]; a.lgmax = g.lgmax;
    a.rows_per_plane = rpp; a.plane_stride = pstride; a.dot_self = io.dot_self;
    a.fin = (io.partials && io.st) ? io.fin : FIN_NONE;
    a.nparts = ch.row_blocks; a.fst = io.st;
    a.outm = io.outm;
  }
  return ch;
}

template <typename T>
cudaError_t launch_apply(const Geo& g, const Tables<T>& tb, cudaStream_t s, const ApplyIO<T>& io) {
  const ApplyChain<T> ch = build_apply<T>(g, tb, io);
  const int Lx = g.L[g.d - 1];
  FL_KERNEL((sizeof(T) == 4 ? "rows_fwd" "<f32>" : "rows_fwd" "<f64>"), s,
            if constexpr (sizeof(T) == 4) {
              if (rows_w8(tb, Lx)) launch_rows_fwd_w8(ch.fwd, ch.row_blocks, ch.row_smem, s);
              else FL_ROWS_LAUNCH(k_rows_fwd, T, Lx, ch.row_blocks, ch.row_smem, s, ch.fwd);
            } else {
              FL_ROWS_LAUNCH(k_rows_fwd, T, Lx, ch.row_blocks, ch.row_smem, s, ch.fwd);
            });
  static const char* const kn[2][4] = {{"cols_fwd<f64>", "cols_conv<f64>", "cols_inv<f64>", "cols_full<f64>"},
                                       {"cols_fwd<f32>", "cols_conv<f32>", "cols_inv<f32>", "cols_full<f32>"}};
  for (int j = 0; j < ch.ncols; ++j)
    FL_KERNEL(kn[sizeof(T) == 4][ch.cols[j].mode], s,
              FL_COLS_LAUNCH(k_cols, T, 1 << ch.cols[j].lg, ch.cols_grid[j], ch.cols_smem[j], s,
                             ch.cols[j]));
  FL_KERNEL((sizeof(T) == 4 ? "rows_inv" "<f32>" : "rows_inv" "<f64>"), s,
            if constexpr (sizeof(T) == 4) {
              if (rows_w8(tb, Lx)) launch_rows_inv_w8(ch.inv, ch.row_blocks, ch.row_smem, s);
              else FL_ROWS_LAUNCH(k_rows_inv, T, Lx, ch.row_blocks, ch.row_smem, s, ch.inv);
            } else {
              FL_ROWS_LAUNCH(k_rows_inv, T, Lx, ch.row_blocks, ch.row_smem, s, ch.inv);
            });
  return launch_status();
}

template <typename T>
PrecChain<T> build_precond(const Geo& g, const Tables<T>& tb, const PrecIO<T>& io) {
  PrecChain<T> ch;
  const int d = g.d;
  const int nx = g.n[d - 1], Lx = g.L[d - 1];
  const long long rows = g.N / nx;
  const int NL = row_lines_at<T>(Lx, io.row_threads);
  ch.row_blocks = (int)((rows + NL - 1) / NL);
  ch.row_smem = smem_bytes<T>(NL, Lx);
  // DST normalisation of every axis but 0 (solved by the tridiagonal pass)
  double post = 1.0;
  for (int i = 1; i < d; ++i) post *= 2.0 / (g.n[i] + 1.0);
  {
    DstRowsArgs<T>& a = ch.first;
    a.in = io.in; a.out = tb.t; a.tw = tb.tw; a.chirp = tb.chirp[d - 1]; a.bhat = tb.bhat[d - 1];
    a.st = io.st; a.x = io.x; a.r = io.r; a.p = io.p; a.q = io.q;
    a.rr_part = io.rr_part;
    a.dotw = nullptr; a.dot_part = nullptr; a.post = 1.0;
    a.rows = (int)rows; a.n = nx; a.lg = g.lg[d - 1]; a.lgmax = g.lgmax; a.pre = io.pre;
    a.fin = FIN_NONE; a.nparts = ch.row_blocks; a.rr_in = nullptr; a.rr_count = 0;
    a.mask_in = io.input_unmasked ? nullptr : io.mask; a.mask_out = nullptr; a.add = nullptr;
  }
  ch.ncols = 0;
  auto cols = [&](int axis, long long lstride, long long ostride, int nouter) {
    DstColsArgs<T>& a = ch.cols[ch.ncols];
    a.v = tb.t; a.tw = tb.tw; a.chirp = tb.chirp[axis]; a.bhat = tb.bhat[axis]; a.st = io.st;
    a.post = 1.0;
    a.n = g.n[axis]; a.ncols = nx; a.lg = g.lg[axis]; a.lgmax = g.lgmax;
    a.ostride = ostride; a.lstride = lstride;
    const int L = g.L[axis];
    const int tx = tile_at<T>(plan_tx<T>(tb, axis, L), L, io.col_threads);
    a.ltx = ilog2i(tx);
    ch.cols_grid[ch.ncols] = dim3((nx + tx - 1) / tx, nouter);
    ch.cols_smem[ch.ncols] = cols_bytes<T>(tx, L);
    ch.ncols++;
  };
  {
    TriArgs<T>& a = ch.tri;
    a.v = tb.t; a.st = io.st; a.tab = tb.tri_tab;
    a.inv_sc = 1.0 / (io.scale * g.cA);
    a.diag = g.dphys == 1 ? 1 : 0;
    a.n = g.n[0];
    a.ncols = (int)(g.N / g.n[0]);
    a.m = (g.n[0] + kTriSeg - 1) / kTriSeg;
    const int tc = io.tri_cols > 0 ? io.tri_cols : kTriCols;
    ch.tri_blocks = (a.ncols + tc - 1) / tc;
  }
  if (d == 2) {
    ch.tri_after = 0;
  } else {
    const long long n1 = g.n[1], n2 = g.n[2];
    cols(1, n2, n1 * n2, g.n[0]);
    ch.tri_after = 1;
    cols(1, n2, n1 * n2, g.n[0]);
  }
  {
    DstRowsArgs<T>& a = ch.last;
    a.in = tb.t; a.out = io.out; a.tw = tb.tw; a.chirp = tb.chirp[d - 1]; a.bhat = tb.bhat[d - 1];
    a.st = io.st; a.x = nullptr; a.r = nullptr; a.p = nullptr; a.q = nullptr;
    a.rr_part = nullptr;
    a.dotw = io.dotw; a.dot_part = io.dot_part; a.post = post;
    a.rows = (int)rows; a.n = nx; a.lg = g.lg[d - 1]; a.lgmax = g.lgmax; a.pre = DPRE_NONE;
    // the CG step needs r.z partials (dotw), the update pass's ||r||^2
    // partials and a state
    const bool step = io.fin == FIN_STEP && io.dotw && io.dot_part && io.rr_part && io.st;
    a.fin = step ? FIN_STEP : FIN_NONE;
    a.nparts = ch.row_blocks; a.rr_in = io.rr_part; a.rr_count = ch.row_blocks;
    a.mask_in = nullptr; a.mask_out = io.keep_outside ? nullptr : io.mask; a.add = io.add;
  }
  return ch;
}

template <typename T>
cudaError_t prepare_precond(const Geo& g, Tables<T>& tb, double shift, double scale, cudaStream_t s) {
  if (tb.tri_shift == shift && tb.tri_scale == scale) return cudaSuccess;
  const int ncols = (int)(g.N / g.n[0]);
  const int m = (g.n[0] + kTriSeg - 1) / kTriSeg;
  FL_KERNEL((sizeof(T) == 4 ? "tri_table" "<f32>" : "tri_table" "<f64>"), s,
            k_tri_table<T><<<(ncols + 255) / 256, 256, 0, s>>>(
                tb.tri_tab, tb.mu[g.d - 1], g.d == 3 ? tb.mu[1] : nullptr, ncols, g.n[g.d - 1],
                shift, scale, g.cA, g.n[0], m, g.dphys == 1 ? 1 : 0));
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    tb.tri_shift = shift;
    tb.tri_scale = scale;
  }
  return e;
}

template <typename T>
cudaError_t launch_precond(const Geo& g, const Tables<T>& tb, cudaStream_t s, const PrecIO<T>& io) {
  // the tridiagonal pass's table must hold this shift and scale
  if (tb.tri_shift != io.shift || tb.tri_scale != io.scale) return cudaErrorInvalidValue;
  const PrecChain<T> ch = build_precond<T>(g, tb, io);
  const int Lx = g.L[g.d - 1];
  FL_KERNEL((sizeof(T) == 4 ? "dst_rows" "<f32>" : "dst_rows" "<f64>"), s,
            if constexpr (sizeof(T) == 4) {
              if (rows_w8(tb, Lx)) launch_dst_rows_w8(ch.first, ch.row_blocks, ch.row_smem, s);
              else FL_ROWS_LAUNCH(k_dst_rows, T, Lx, ch.row_blocks, ch.row_smem, s, ch.first);
            } else {
              FL_ROWS_LAUNCH(k_dst_rows, T, Lx, ch.row_blocks, ch.row_smem, s, ch.first);
            });
  for (int j = 0; j <= ch.ncols; ++j) {
    if (j == ch.tri_after)
      FL_KERNEL((sizeof(T) == 4 ? "tri_cols" "<f32>" : "tri_cols" "<f64>"), s,
                pdl_launch(k_tri_cols<T>, ch.tri_blocks, kTriCols * kTriSeg, 0, s, ch.tri));
    if (j < ch.ncols)
      FL_KERNEL((sizeof(T) == 4 ? "dst_cols" "<f32>" : "dst_cols" "<f64>"), s,
                FL_COLS_LAUNCH(k_dst_cols, T, 1 << ch.cols[j].lg, ch.cols_grid[j], ch.cols_smem[j], s,
                               ch.cols[j]));
  }
  FL_KERNEL((sizeof(T) == 4 ? "dst_rows" "<f32>" : "dst_rows" "<f64>"), s,
            if constexpr (sizeof(T) == 4) {
              if (rows_w8(tb, Lx)) launch_dst_rows_w8(ch.last, ch.row_blocks, ch.row_smem, s);
              else FL_ROWS_LAUNCH(k_dst_rows, T, Lx, ch.row_blocks, ch.row_smem, s, ch.last);
            } else {
              FL_ROWS_LAUNCH(k_dst_rows, T, Lx, ch.row_blocks, ch.row_smem, s, ch.last);
            });
  return launch_status();
}

template <typename T>
cudaError_t launch_noprec_update(long long N, cudaStream_t s, PcgState* st, T* x, T* r, const T* p,
                                 const T* q, double* rr_part, int step, int* count) {
  FL_KERNEL((sizeof(T) == 4 ? "noprec_update" "<f32>" : "noprec_update" "<f64>"), s,
            pdl_launch(k_noprec_update<T>, kVecBlocks, kVecThreads, 0, s, st, x, r, p, q, rr_part, step, N));
  *count = kVecBlocks;
  return launch_status();
}

template <typename T>
cudaError_t launch_dot(long long N, cudaStream_t s, const T* a, const T* b, double* part, int* count) {
  FL_KERNEL((sizeof(T) == 4 ? "dot" "<f32>" : "dot" "<f64>"), s,
            k_dot<T><<<kVecBlocks, kVecThreads, 0, s>>>(a, b, part, N));
  *count = kVecBlocks;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_copy_cast(long long N, cudaStream_t s, const double* src, T* dst) {
  FL_KERNEL((sizeof(T) == 4 ? "copy_cast" "<f32>" : "copy_cast" "<f64>"), s,
            k_copy_cast<T><<<kVecBlocks, kVecThreads, 0, s>>>(src, dst, N));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axpby(long long N, cudaStream_t s, double a, const T* x, double b, T* y) {
  FL_KERNEL((sizeof(T) == 4 ? "axpby" "<f32>" : "axpby" "<f64>"), s,
            k_axpby<T><<<kVecBlocks, kVecThreads, 0, s>>>(a, x, b, y, N));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mask_copy_dot(long long N, cudaStream_t s, const T* src, const uint8_t* mask, T* dst,
                                 double* part, int* count) {
  FL_KERNEL((sizeof(T) == 4 ? "mask_copy_dot" "<f32>" : "mask_copy_dot" "<f64>"), s,
            k_mask_copy_dot<T><<<kVecBlocks, kVecThreads, 0, s>>>(src, mask, dst, part, N));
  *count = kVecBlocks;
  return cudaGetLastError();
}
#if FL_OPS_PART == 1
template cudaError_t launch_mask_copy_dot<float>(long long, cudaStream_t, const float*, const uint8_t*, float*, double*, int*);
#else
template cudaError_t launch_mask_copy_dot<double>(long long, cudaStream_t, const double*, const uint8_t*, double*, double*, int*);
#endif

#if FL_OPS_PART == 1
cudaError_t launch_pcg_init(cudaStream_t s, PcgState* st, const double* bb_part, int bb_count,
                            const double* rr_part, int rr_count, const double* rz_part, int rz_count,
                            double tol, int maxit) {
  FL_KERNEL("pcg_init", s,
            k_pcg_init<<<1, 256, 0, s>>>(st, bb_part, bb_count, rr_part, rr_count, rz_part, rz_count, tol, maxit));
  return cudaGetLastError();
}

cudaError_t launch_residual_from(long long N, cudaStream_t s, const double* b, const double* u,
                                 const double* mx, const uint8_t* mask, double shift, double scale,
                                 float* r32, double* part, int* count) {
  FL_KERNEL("residual_from", s,
            k_residual_from<<<kVecBlocks, kVecThreads, 0, s>>>(b, u, mx, mask, shift, scale, r32, part, N));
  *count = kVecBlocks;
  return cudaGetLastError();
}

cudaError_t launch_axmy(long long N, cudaStream_t s, const double* u, double c, const double* mx,
                        double* y) {
  FL_KERNEL("axmy", s, k_axmy<<<kVecBlocks, kVecThreads, 0, s>>>(u, c, mx, y, N));
  return cudaGetLastError();
}

cudaError_t launch_hash(long long N, cudaStream_t s, const double* u, unsigned long long* h) {
  FL_KERNEL("hash", s, k_hash<<<kVecBlocks, kVecThreads, 0, s>>>(u, h, N));
  return cudaGetLastError();
}

cudaError_t launch_sine_mode(const Geo& g, cudaStream_t s, double* v, const uint8_t* mask, int hi) {
  FL_KERNEL("sine_mode", s,
            k_sine_mode<<<kVecBlocks, kVecThreads, 0, s>>>(v, mask, g.d, g.n[0], g.n[1], g.n[2], hi, g.N));
  return cudaGetLastError();
}

cudaError_t launch_sum(cudaStream_t s, const double* part, int count, double* out) {
  FL_KERNEL("sum", s,
            k_sum<<<1, 256, 0, s>>>(part, count, out));
  return cudaGetLastError();
}

#endif  // FL_OPS_PART == 1

#if FL_OPS_PART == 2
cudaError_t build_symbol(const Geo& g, double c, double Z, double a, double expo, cudaStream_t s,
                         double* sig64, float* sig32, const double2* tw64) {
  typedef Cfg<double> K;
  const int d = g.d;
  long long total = 1, half = 1;
  int Ls[3] = {1, 1, 1}, ns[3] = {1, 1, 1};
  for (int i = 0; i < d; ++i) {
    total *= g.L[i];
    half *= g.L[i] / 2 + 1;
    Ls[i] = g.L[i];
    ns[i] = g.n[i];
  }
  double2* buf = nullptr;
  cudaError_t e = cudaMallocAsync(&buf, total * sizeof(double2), s);
  if (e != cudaSuccess) return e;
  const int bt = 256;
  FL_KERNEL("fill_kernel", s,
            k_fill_kernel<<<(unsigned)((total + bt - 1) / bt), bt, 0, s>>>(buf, d, Ls[0], Ls[1], Ls[2], ns[0],
                                                                 ns[1], ns[2], c, Z, a, expo, g.dphys, total));
  // last axis: contiguous lines
  {
    const int L = g.L[d - 1];
    const long long rows = total / L;
    const int NL = row_lines<double>(L);
    const unsigned blocks = (unsigned)((rows + NL - 1) / NL);
    if (L <= K::RT * K::RV)
      FL_KERNEL("rows_c2c", s,
                k_rows_c2c<K::RT, K::RV><<<blocks, K::RT, smem_bytes<double>(NL, L), s>>>(
                    buf, (int)rows, g.lg[d - 1], g.lgmax, tw64));
    else
      FL_KERNEL("rows_c2c", s,
                k_rows_c2c<2 * K::RT, K::RV><<<blocks, 2 * K::RT, smem_bytes<double>(NL, L), s>>>(
                    buf, (int)rows, g.lg[d - 1], g.lgmax, tw64));
  }
  // slower axes: strided lines, full length in and out
  for (int axis = d - 2; axis >= 0; --axis) {
    ColsArgs<double> ca;
    ca.S = buf; ca.tw = tw64; ca.sig = nullptr; ca.st = nullptr;
    ca.H = Ls[d - 1]; ca.lg = g.lg[axis]; ca.lgmax = g.lgmax;
    ca.rows_in = Ls[axis]; ca.rows_out = Ls[axis]; ca.mode = COLS_FULL;
    ca.sig_line = 0; ca.sig_outer = 0; ca.Lo = 0;
    if (d == 2) { ca.lstride = Ls[1]; ca.ostride = 0; ca.nouter = 1; }
    else if (axis == 1) { ca.lstride = Ls[2]; ca.ostride = (long long)Ls[1] * Ls[2]; ca.nouter = Ls[0]; }
    else { ca.lstride = (long long)Ls[1] * Ls[2]; ca.ostride = Ls[2]; ca.nouter = Ls[1]; }
    const int tx = col_tx<double>(Ls[axis]);
    ca.ltx = ilog2i(tx);
    dim3 grid((ca.H + tx - 1) / tx, ca.nouter);
    FL_KERNEL("cols_symbol", s,
              FL_COLS_LAUNCH(k_cols, double, Ls[axis], grid, tile_bytes<double>(tx, Ls[axis]), s, ca));
  }
  double inv = 1.0;
  for (int i = 0; i < d; ++i) inv /= (double)g.L[i];
  FL_KERNEL("extract_symbol", s,
            k_extract_symbol<<<(unsigned)((half + bt - 1) / bt), bt, 0, s>>>(buf, d, Ls[0], Ls[1], Ls[2], inv,
                                                                  sig64, sig32, half));
  e = cudaGetLastError();
  cudaError_t e2 = cudaFreeAsync(buf, s);
  return e != cudaSuccess ? e : e2;
}

#endif  // FL_OPS_PART == 2

// explicit instantiations
#if FL_OPS_PART == 1
template cudaError_t launch_apply<float>(const Geo&, const Tables<float>&, cudaStream_t, const ApplyIO<float>&);
template ApplyChain<float> build_apply<float>(const Geo&, const Tables<float>&, const ApplyIO<float>&);
template PrecChain<float> build_precond<float>(const Geo&, const Tables<float>&, const PrecIO<float>&);
template int apply_partials<float>(const Geo&);
template int precond_partials<float>(const Geo&);
template cudaError_t prepare_precond<float>(const Geo&, Tables<float>&, double, double, cudaStream_t);
template cudaError_t launch_precond<float>(const Geo&, const Tables<float>&, cudaStream_t, const PrecIO<float>&);
template cudaError_t launch_noprec_update<float>(long long, cudaStream_t, PcgState*, float*, float*, const float*, const float*, double*, int, int*);
template cudaError_t launch_dot<float>(long long, cudaStream_t, const float*, const float*, double*, int*);
template cudaError_t launch_copy_cast<float>(long long, cudaStream_t, const double*, float*);
template cudaError_t launch_axpby<float>(long long, cudaStream_t, double, const float*, double, float*);
#else
template cudaError_t launch_apply<double>(const Geo&, const Tables<double>&, cudaStream_t, const ApplyIO<double>&);
template ApplyChain<double> build_apply<double>(const Geo&, const Tables<double>&, const ApplyIO<double>&);
template PrecChain<double> build_precond<double>(const Geo&, const Tables<double>&, const PrecIO<double>&);
template int apply_partials<double>(const Geo&);
template int precond_partials<double>(const Geo&);
template cudaError_t prepare_precond<double>(const Geo&, Tables<double>&, double, double, cudaStream_t);
template cudaError_t launch_precond<double>(const Geo&, const Tables<double>&, cudaStream_t, const PrecIO<double>&);
template cudaError_t launch_noprec_update<double>(long long, cudaStream_t, PcgState*, double*, double*, const double*, const double*, double*, int, int*);
template cudaError_t launch_dot<double>(long long, cudaStream_t, const double*, const double*, double*, int*);
template cudaError_t launch_copy_cast<double>(long long, cudaStream_t, const double*, double*);
template cudaError_t launch_axpby<double>(long long, cudaStream_t, double, const double*, double, double*);
#endif

}  // namespace fl
