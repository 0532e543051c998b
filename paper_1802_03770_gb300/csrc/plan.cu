// Host side of the C ABI: plan creation (constants, tables, symbol,
// workspaces), the apply / preconditioner entry points and the CG drivers
// (plain FP64 CG, FP32 CG inside FP64 iterative refinement, theta steps).
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fraclap.h"
#include "internal.h"
#include "chain.cuh"
#include "learned.h"
#include "persist.h"
#include "domain.h"

using namespace fl;

namespace {

thread_local std::string g_err;

fl_status fail(fl_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

fl_status cuda_fail(cudaError_t e, const char* where) {
  return fail(e == cudaErrorMemoryAllocation ? FL_OOM : FL_CUDA_ERROR,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define FL_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

template <typename T>
struct Vecs {
  T *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
};

}  // namespace

struct Profiler {
  struct Pending { const char* name; cudaEvent_t e0, e1; };
  struct Stat { std::string name; long long launches = 0; double ms = 0.0; };
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  std::vector<Stat> stats;
  cudaEvent_t take() {
    if (pool.empty()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  void resolve() {
    for (auto& pe : pending) {
      float ms = 0.f;
      cudaEventSynchronize(pe.e1);
      cudaEventElapsedTime(&ms, pe.e0, pe.e1);
      Stat* st = nullptr;
      for (auto& x : stats)
        if (x.name == pe.name) st = &x;
      if (!st) {
        stats.push_back(Stat());
        st = &stats.back();
        st->name = pe.name;
      }
      st->launches += 1;
      st->ms += ms;
      pool.push_back(pe.e0);
      pool.push_back(pe.e1);
    }
    pending.clear();
  }
  ~Profiler() {
    resolve();
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// A captured chunk of CG iterations of one precision, valid for one
// (preconditioner, shift, scale) configuration.
struct GraphCache {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool use_prec = false, domain = false;
  double shift = 0.0, scale = 0.0, pshift = 0.0, pscale = 0.0;
  long long kernels = 0;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
};

struct fl_plan {
  Geo g;
  int device = 0;          // CUDA device current at fl_plan_create
  double h, alpha, rho;
  double C, Z, a, c;
  double inner_tol;
  int max_outer;
  cudaStream_t stream;
  bool has_mask;
  uint8_t* mask = nullptr;
  Tables<float> t32;
  Tables<double> t64;
  Vecs<float> v32;
  Vecs<double> v64;
  double* part[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* dscalar = nullptr;
  double* u_e2e = nullptr;        // solution buffer of the host-array entry point
  PcgState* st = nullptr;
  PcgState* st_host = nullptr;  // pinned
  double* scalar_host = nullptr;  // pinned
  std::vector<void*> allocs;
  int64_t bytes = 0;
  struct Profiler* prof = nullptr;   // non-null while profiling is enabled
  GraphCache gcache[2];              // [0] FP64, [1] FP32 CG iteration graphs
  // learned preconditioner (fl_plan_attach_net)
  fl::NetState* net = nullptr;
  float* z0 = nullptr;     // base preconditioned residual
  float* feat = nullptr;   // network input, 3 x N
  double* lpart[3] = {nullptr, nullptr, nullptr};  // ||z0||^2, r.z, r.z_old partials
  // M u of the last time step's result (fl_time_step): mu_cache holds
  // M u_next of the previous step, valid for the array mu_of while its
  // contents still hash to mu_hash
  double* mu_cache = nullptr;
  const double* mu_of = nullptr;
  unsigned long long mu_hash = 0ull;
  bool mu_valid = false;
  unsigned long long* hash_dev = nullptr;
  unsigned long long* hash_host = nullptr;  // pinned
  // Rayleigh quotients of M on the lowest and highest sine modes
  // (FL_PRECOND_SHIFTED), computed on first use
  double mq_lo = 0.0, mq_hi = 0.0;
  bool mq_valid = false;
  // occluded domain: the hole's boundary Gamma and the capacitance factor of
  // the FD operator on Omega (domain.cu) for dom_shift, dom_scale
  fl::DomainData dom;
  int dom_points = 0;            // |Gamma| (may exceed kMaxGamma: no factor then)
  double dom_shift = -1.0, dom_scale = -1.0;
  float* dw32 = nullptr;         // w = B^{-1} r~ of the last application (N)
  float* dus32 = nullptr;        // E s, zero off Gamma (N)
  double* dw64 = nullptr;
  double* dus64 = nullptr;
};

namespace {
std::atomic<long long> g_launches{0};
thread_local Profiler* t_prof = nullptr;

// Makes the plan's profiler the active one for the duration of an API call.
struct ProfScope {
  Profiler* saved;
  explicit ProfScope(fl_plan* p);
  ~ProfScope() { t_prof = saved; }
};
}  // namespace

ProfScope::ProfScope(fl_plan* p) : saved(t_prof) { t_prof = p ? p->prof : nullptr; }

namespace {

enum { P_PQ = 0, P_RR = 1, P_RZ = 2, P_BB = 3, P_RES = 4, P_AUX = 5 };

constexpr int kGraphIters = 4;

// FRACLAP_GRAPHS=0 in the environment launches CG iterations one by one.
bool graphs_enabled() {
  static const bool on = [] {
    const char* v = getenv("FRACLAP_GRAPHS");
    return !(v && v[0] == '0');
  }();
  return on;
}

template <typename P>
cudaError_t dalloc(fl_plan* p, P** ptr, size_t bytes) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, bytes);
  if (e == cudaSuccess) {
    p->allocs.push_back(v);
    p->bytes += (int64_t)bytes;
    *ptr = reinterpret_cast<P*>(v);
  }
  return e;
}

void free_plan(fl_plan* p) {
  if (!p) return;
  for (auto& gc : p->gcache) gc.release();
  if (p->prof) {
    cudaStreamSynchronize(p->stream);
    delete p->prof;
  }
  for (void* v : p->allocs) cudaFree(v);
  if (p->st_host) cudaFreeHost(p->st_host);
  if (p->scalar_host) cudaFreeHost(p->scalar_host);
  if (p->hash_host) cudaFreeHost(p->hash_host);
  delete p;
}

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// twiddles exp(-2 pi i k / Lmax), chirps and chirp-kernel spectra for the
// DST-I of each axis (see kernels.cuh), in long double.
fl_status build_tables(fl_plan* p) {
  const Geo& g = p->g;
  const int Lmax = 1 << g.lgmax;
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<double2> tw64(Lmax);
  std::vector<float2> tw32(Lmax);
  for (int k = 0; k < Lmax; ++k) {
    const long double ang = -2.0L * pi * (long double)k / (long double)Lmax;
    tw64[k] = make_double2((double)cosl(ang), (double)sinl(ang));
    tw32[k] = make_float2((float)cosl(ang), (float)sinl(ang));
  }
  FL_CUDA(dalloc(p, &p->t64.tw, Lmax * sizeof(double2)));
  FL_CUDA(dalloc(p, &p->t32.tw, Lmax * sizeof(float2)));
  FL_CUDA(cudaMemcpy(p->t64.tw, tw64.data(), Lmax * sizeof(double2), cudaMemcpyHostToDevice));
  FL_CUDA(cudaMemcpy(p->t32.tw, tw32.data(), Lmax * sizeof(float2), cudaMemcpyHostToDevice));
  for (int ax = 0; ax < g.d; ++ax) {
    const int n = g.n[ax], L = g.L[ax];
    const long long N1 = n + 1;
    // c_m = exp(i pi m^2 / (2 N1)), with m^2 reduced mod 4 N1
    auto chirp = [&](long long m) {
      const long long m2 = (m * m) % (4 * N1);
      const long double ang = pi * (long double)m2 / (2.0L * (long double)N1);
      return std::complex<long double>(cosl(ang), sinl(ang));
    };
    std::vector<double2> c64(n);
    std::vector<float2> c32(n);
    for (int j = 0; j < n; ++j) {
      const auto c = chirp(j + 1);
      c64[j] = make_double2((double)c.real(), (double)c.imag());
      c32[j] = make_float2((float)c.real(), (float)c.imag());
    }
    std::vector<std::complex<long double>> b(L, 0.0L);
    for (int m = -(n - 1); m <= n - 1; ++m) b[(m + L) % L] = std::conj(chirp(m));
    host_fft(b);
    std::vector<double2> b64(L);
    std::vector<float2> b32(L);
    for (int k = 0; k < L; ++k) {
      const auto v = b[k] / (long double)L;
      b64[k] = make_double2((double)v.real(), (double)v.imag());
      b32[k] = make_float2((float)v.real(), (float)v.imag());
    }
    FL_CUDA(dalloc(p, &p->t64.chirp[ax], n * sizeof(double2)));
    FL_CUDA(dalloc(p, &p->t32.chirp[ax], n * sizeof(float2)));
    FL_CUDA(dalloc(p, &p->t64.bhat[ax], L * sizeof(double2)));
    FL_CUDA(dalloc(p, &p->t32.bhat[ax], L * sizeof(float2)));
    FL_CUDA(cudaMemcpy(p->t64.chirp[ax], c64.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
    FL_CUDA(cudaMemcpy(p->t32.chirp[ax], c32.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
    FL_CUDA(cudaMemcpy(p->t64.bhat[ax], b64.data(), L * sizeof(double2), cudaMemcpyHostToDevice));
    FL_CUDA(cudaMemcpy(p->t32.bhat[ax], b32.data(), L * sizeof(float2), cudaMemcpyHostToDevice));
    // eigenvalues of C h^d L along this axis: c (-a) 4 sin^2(pi k / (2 (n+1)))
    std::vector<double> mu(n);
    for (int k = 0; k < n; ++k) {
      const long double s = sinl(pi * (long double)(k + 1) / (2.0L * (long double)N1));
      mu[k] = (double)((long double)p->c * (long double)(-p->a) * 4.0L * s * s);
    }
    std::vector<float> mu32(mu.begin(), mu.end());
    FL_CUDA(dalloc(p, &p->t64.mu[ax], n * sizeof(double)));
    FL_CUDA(dalloc(p, &p->t32.mu[ax], n * sizeof(float)));
    FL_CUDA(cudaMemcpy(p->t64.mu[ax], mu.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    FL_CUDA(cudaMemcpy(p->t32.mu[ax], mu32.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  }
  return FL_OK;
}

template <typename T>
fl_status alloc_vecs(fl_plan* p, Vecs<T>& v) {
  const size_t b = (size_t)p->g.N * sizeof(T);
  FL_CUDA(dalloc(p, &v.b, b));
  FL_CUDA(dalloc(p, &v.x, b));
  FL_CUDA(dalloc(p, &v.r, b));
  FL_CUDA(dalloc(p, &v.z, b));
  FL_CUDA(dalloc(p, &v.p, b));
  FL_CUDA(dalloc(p, &v.q, b));
  return FL_OK;
}

template <typename T> Tables<T>& tables(fl_plan* p);
template <> Tables<float>& tables<float>(fl_plan* p) { return p->t32; }
template <> Tables<double>& tables<double>(fl_plan* p) { return p->t64; }
template <typename T> Vecs<T>& vecs(fl_plan* p);
template <> Vecs<float>& vecs<float>(fl_plan* p) { return p->v32; }
template <> Vecs<double>& vecs<double>(fl_plan* p) { return p->v64; }

// Read the device CG state (waits for the stream).
fl_status read_state(fl_plan* p) {
  FL_CUDA(cudaMemcpyAsync(p->st_host, p->st, sizeof(PcgState), cudaMemcpyDeviceToHost, p->stream));
  FL_CUDA(cudaStreamSynchronize(p->stream));
  return FL_OK;
}

fl_status read_sum(fl_plan* p, const double* part, int count, double* out) {
  FL_CUDA(launch_sum(p->stream, part, count, p->dscalar));
  FL_CUDA(cudaMemcpyAsync(p->scalar_host, p->dscalar, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  FL_CUDA(cudaStreamSynchronize(p->stream));
  *out = *p->scalar_host;
  return FL_OK;
}

// The preconditioner of a solve: z = (shift I + scale C h^d L)^{-1} r on the
// box (restricted to Omega), or none.
struct PrecChoice {
  bool use = false;
  double shift = 0.0, scale = 0.0;
  bool domain = false;   // occluded domain: the FD operator on Omega (capacitance solve)
};

fl_status precond_params_raw(fl_plan* p, int prec_mode, double shift, double scale, PrecChoice* pc);

// Rayleigh quotients v^T M v / v^T v of the lowest and the highest sine
// modes restricted to Omega, by FP64 applies (the CG direction buffers of
// the FP64 workspace serve as scratch); once per plan.
fl_status extreme_quotients(fl_plan* p) {
  if (p->mq_valid) return FL_OK;
  const Geo& g = p->g;
  double* v = p->v64.p;
  double q[2] = {0.0, 0.0};
  for (int hi = 0; hi < 2; ++hi) {
    FL_CUDA(launch_sine_mode(g, p->stream, v, p->mask, hi));
    ApplyIO<double> io;
    io.u = v; io.mask = p->mask; io.out = p->v64.q; io.x = v; io.cm = 1.0;
    io.dotw = v; io.partials = p->part[P_AUX];
    FL_CUDA(launch_apply<double>(g, p->t64, p->stream, io));
    double vmv = 0.0, vv = 0.0;
    fl_status st = read_sum(p, p->part[P_AUX], apply_partials<double>(g), &vmv);
    if (st != FL_OK) return st;
    int c = 0;
    FL_CUDA(launch_dot<double>(g.N, p->stream, v, v, p->part[P_RES], &c));
    st = read_sum(p, p->part[P_RES], c, &vv);
    if (st != FL_OK) return st;
    if (!(vv > 0.0)) return fail(FL_INVALID_ARG, "a sine mode vanishes on Omega");
    q[hi] = vmv / vv;
  }
  p->mq_lo = q[0];
  p->mq_hi = q[1];
  p->mq_valid = true;
  return FL_OK;
}

// Eigenvalue of C h^d L = cA (2d I - S) on the lowest (hi = 0) or highest
// sine mode: cA sum_i 4 sin^2(pi k_i / (2 (n_i + 1))) over the problem's axes.
double fd_mode_eigenvalue(const Geo& g, int hi) {
  double lam = 0.0;
  for (int i = g.d - g.dphys; i < g.d; ++i) {
    const double k = hi ? g.n[i] : 1.0;
    const double sn = std::sin(3.14159265358979323846 * k / (2.0 * (g.n[i] + 1.0)));
    lam += 4.0 * sn * sn;
  }
  return g.cA * lam;
}

// The FD solve's tridiagonal pass along axis 0 holds a column of at most
// 1024 values (32 segments of 32); 1D plans (n_0 = 1) solve per mode.
bool precond_fits(const fl_plan* p) { return p->g.n[0] <= 1024; }
const char* const kPrecondLimit = "the FD preconditioner needs n_0 <= 1024 (use FL_PRECOND_NONE)";

// The preconditioner of `prec_mode` for the operator shift I + scale M.
fl_status precond_params(fl_plan* p, int prec_mode, double shift, double scale, PrecChoice* pc) {
  const fl_status st = precond_params_raw(p, prec_mode, shift, scale, pc);
  if (st != FL_OK || !pc->use) return st;
  if (!precond_fits(p)) return fail(FL_INVALID_ARG, kPrecondLimit);
  // on an occluded domain every member of the FD family is solved on Omega
  // itself (the paper's choice, Sec. 4.4), except the restricted box solve
  pc->domain = p->has_mask && prec_mode != FL_PRECOND_BOX;
  if (pc->domain && p->dom_points > kMaxGamma)
    return fail(FL_INVALID_ARG, "the hole's boundary has more than 2048 points: use FL_PRECOND_BOX");
  return FL_OK;
}

fl_status precond_params_raw(fl_plan* p, int prec_mode, double shift, double scale, PrecChoice* pc) {
  pc->use = true;
  pc->shift = shift;
  pc->scale = scale;
  switch (prec_mode) {
    case FL_PRECOND_FD:
    case FL_PRECOND_BOX:
      return FL_OK;
    case FL_PRECOND_AUTO:
      if (p->alpha >= 1.0) return FL_OK;
      *pc = PrecChoice();
      return FL_OK;
    case FL_PRECOND_NONE:
      *pc = PrecChoice();
      return FL_OK;
    case FL_PRECOND_STENCIL:
      // shift I + scale M~: M~ has c (Z - 2d a) on the diagonal and c (a - 1)
      // on the stencil's neighbours, = c (Z - 2d) I + ((1 - a) / -a) cA (2d I - S)
      pc->shift = shift + scale * p->c * (p->Z - 2.0 * p->g.dphys);
      pc->scale = scale * (1.0 - p->a) / (-p->a);
      return FL_OK;
    case FL_PRECOND_SHIFTED: {
      const fl_status st = extreme_quotients(p);
      if (st != FL_OK) return st;
      const double lam_lo = fd_mode_eigenvalue(p->g, 0), lam_hi = fd_mode_eigenvalue(p->g, 1);
      const double A = shift + scale * p->mq_lo, B = shift + scale * p->mq_hi;
      const double x = B > A ? scale * (A * lam_hi - B * lam_lo) / (B - A) : shift;
      pc->shift = x > 0.0 ? x : 0.0;
      return FL_OK;
    }
    default:
      return fail(FL_INVALID_ARG, "unknown preconditioner mode");
  }
}

template <typename T> T* dom_w(fl_plan* p);
template <> float* dom_w<float>(fl_plan* p) { return p->dw32; }
template <> double* dom_w<double>(fl_plan* p) { return p->dw64; }
template <typename T> T* dom_us(fl_plan* p);
template <> float* dom_us<float>(fl_plan* p) { return p->dus32; }
template <> double* dom_us<double>(fl_plan* p) { return p->dus64; }

// Makes the plan's preconditioner of `pc` ready in precision T: the
// tridiagonal table of the box solve and, on an occluded domain, the
// capacitance factor of the FD operator on Omega (FP64 box solves; the CG
// direction buffers of the FP64 workspace serve as scratch).
template <typename T>
fl_status prepare_prec(fl_plan* p, const PrecChoice& pc) {
  if (pc.domain && (p->dom_shift != pc.shift || p->dom_scale != pc.scale)) {
    p->dom_shift = p->dom_scale = -1.0;
    if (p->dom.m > 0) {
      FL_CUDA(prepare_precond<double>(p->g, p->t64, pc.shift, pc.scale, p->stream));
      FL_CUDA(dom_build_capacitance(p->g, p->t64, p->dom, pc.shift, pc.scale, p->v64.p, p->v64.q,
                                    p->stream));
    }
    p->dom_shift = pc.shift;
    p->dom_scale = pc.scale;
  }
  FL_CUDA(prepare_precond<T>(p->g, tables<T>(p), pc.shift, pc.scale, p->stream));
  return FL_OK;
}

// One application of the preconditioner of `pc` as io describes it (its
// fused CG update, dot products and CG step included).  On an occluded
// domain: w = B^{-1} r (the box solve, with the update), the interface solve
// us = E s, then z = R (w + B^{-1} us) with io's dot products and step.
template <typename T>
cudaError_t apply_prec(fl_plan* p, const PrecChoice& pc, const PrecIO<T>& io, cudaStream_t s) {
  const Geo& g = p->g;
  Tables<T>& tb = tables<T>(p);
  if (!pc.domain) return launch_precond<T>(g, tb, s, io);
  PrecIO<T> a = io;
  a.out = dom_w<T>(p);
  a.dotw = nullptr; a.dot_part = nullptr; a.fin = FIN_NONE; a.keep_outside = true;
  cudaError_t e = launch_precond<T>(g, tb, s, a);
  if (e == cudaSuccess && p->dom.m > 0) e = dom_interface_solve<T>(p->dom, dom_w<T>(p), dom_us<T>(p), io.st, s);
  if (e != cudaSuccess) return e;
  PrecIO<T> b = io;
  b.pre = DPRE_NONE; b.in = dom_us<T>(p); b.input_unmasked = true; b.add = dom_w<T>(p);
  b.x = nullptr; b.r = nullptr; b.p = nullptr; b.q = nullptr;
  return launch_precond<T>(g, tb, s, b);
}

// Preconditioned CG for (shift I + scale M) x = b in precision T, all
// vectors in the plan's workspace of that precision (b = v.b, x = v.x),
// preconditioned by (pc.shift I + pc.scale C h^d L)^{-1} unless !pc.use.
// Stops when ||r|| <= tol ||b||.  Returns the status of the solve.
template <typename T>
fl_status run_pcg(fl_plan* p, bool x0_nonzero, double shift, double scale, const PrecChoice& pc,
                  double tol, int maxit, int* iters) {
  const bool use_prec = pc.use;
  const Geo& g = p->g;
  Vecs<T>& v = vecs<T>(p);
  Tables<T>& tb = tables<T>(p);
  cudaStream_t s = p->stream;
  int bb_count = 0, rz_count = 0;
  // r = b - A x  (or r = b masked)
  if (x0_nonzero) {
    ApplyIO<T> io;
    io.u = v.x; io.mask = p->mask; io.out = v.r; io.x = v.x; io.b = v.b;
    io.cm = -scale; io.cx = -shift; io.cb = 1.0;
    FL_CUDA(launch_apply<T>(g, tb, s, io));
    FL_CUDA(launch_mask_copy_dot<T>(g.N, s, v.b, p->mask, (T*)nullptr, p->part[P_BB], &bb_count));
  } else {
    FL_CUDA(cudaMemsetAsync(v.x, 0, g.N * sizeof(T), s));
    FL_CUDA(launch_mask_copy_dot<T>(g.N, s, v.b, p->mask, v.r, p->part[P_BB], &bb_count));
  }
  FL_CUDA(cudaMemsetAsync(v.p, 0, g.N * sizeof(T), s));
  T* z = use_prec ? v.z : v.r;
  if (use_prec) {
    const fl_status ps = prepare_prec<T>(p, pc);
    if (ps != FL_OK) return ps;
    PrecIO<T> io;
    io.in = v.r; io.out = v.z; io.shift = pc.shift; io.scale = pc.scale;
    io.dotw = v.r; io.dot_part = p->part[P_RZ]; io.mask = p->mask;
    FL_CUDA(apply_prec<T>(p, pc, io, s));
    rz_count = precond_partials<T>(g);
  } else {
    FL_CUDA(launch_dot<T>(g.N, s, v.r, v.r, p->part[P_RZ], &rz_count));
  }
  // ||r0||^2 for the initial convergence test (r0 = b when x0 = 0)
  const double* rr0_part = p->part[P_BB];
  int rr0_count = bb_count;
  if (x0_nonzero) {
    FL_CUDA(launch_dot<T>(g.N, s, v.r, v.r, p->part[P_AUX], &rr0_count));
    rr0_part = p->part[P_AUX];
  }
  FL_CUDA(launch_pcg_init(s, p->st, p->part[P_BB], bb_count, rr0_part, rr0_count, p->part[P_RZ],
                          rz_count, tol, maxit));
  // One CG iteration: q = A p (p = z + beta p fused; the apply's last CTA
  // forms pq and alpha), the x/r update fused into the first preconditioner
  // pass (or the plain update), and the scalar step in the last CTA of the
  // last pass.
  auto enqueue = [&](cudaStream_t qs) -> cudaError_t {
    ApplyIO<T> io;
    io.pre = PRE_PUPDATE; io.u = z; io.p = v.p; io.mask = p->mask; io.st = p->st;
    io.out = v.q; io.x = v.p; io.cm = scale; io.cx = shift;
    io.dotw = v.p; io.partials = p->part[P_PQ]; io.fin = FIN_PQ;
    cudaError_t e = launch_apply<T>(g, tb, qs, io);
    if (e != cudaSuccess) return e;
    int cnt = 0;
    if (use_prec) {
      PrecIO<T> pi;
      pi.pre = DPRE_UPDATE; pi.out = v.z; pi.shift = pc.shift; pi.scale = pc.scale;
      pi.x = v.x; pi.r = v.r; pi.p = v.p; pi.q = v.q; pi.rr_part = p->part[P_RR];
      pi.dotw = v.r; pi.dot_part = p->part[P_RZ]; pi.st = p->st; pi.fin = FIN_STEP;
      pi.mask = p->mask;
      return apply_prec<T>(p, pc, pi, qs);
    }
    return launch_noprec_update<T>(g.N, qs, p->st, v.x, v.r, v.p, v.q, p->part[P_RR], 1, &cnt);
  };
  // Iterations run in chunks of 4, 8, 16, 32 between reads of the device
  // state; a chunk is replays of a captured 4-iteration CUDA graph (not
  // while the per-kernel profiler is on).
  GraphCache& gc = p->gcache[sizeof(T) == 4 ? 1 : 0];
  const bool use_graph = p->prof == nullptr && graphs_enabled();
  if (use_graph && !(gc.exec && gc.use_prec == use_prec && gc.shift == shift && gc.scale == scale &&
                     gc.pshift == pc.shift && gc.pscale == pc.scale && gc.domain == pc.domain)) {
    gc.release();
    cudaStream_t cs = nullptr;
    FL_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const long long before = g_launches.load();
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    for (int k = 0; k < kGraphIters && e == cudaSuccess; ++k) e = enqueue(cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &gc.graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "CG iteration capture");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    FL_CUDA(cudaGraphInstantiate(&gc.exec, gc.graph, 0));
    gc.kernels = g_launches.load() - before;
    g_launches.fetch_sub(gc.kernels);   // counted when the graph runs
    gc.use_prec = use_prec;
    gc.shift = shift;
    gc.scale = scale;
    gc.pshift = pc.shift;
    gc.pscale = pc.scale;
    gc.domain = pc.domain;
  }
  // The next chunk covers the iterations the last chunk's convergence rate
  // predicts are left (+1), in multiples of the graph's 4, between 4 and 32;
  // iterations after convergence exit at entry but still cost a launch.
  int chunk = 4;
  double rr_last = -1.0;
  int it_last = 0;
  for (;;) {
    if (use_graph) {
      for (int c = 0; c < chunk / kGraphIters; ++c) {
        FL_CUDA(cudaGraphLaunch(gc.exec, s));
        g_launches.fetch_add(gc.kernels);
      }
    } else {
      for (int k = 0; k < chunk; ++k) FL_CUDA(enqueue(s));
    }
    fl_status st = read_state(p);
    if (st != FL_OK) return st;
    if (p->st_host->done) break;
    const double rr = p->st_host->rr;
    const int it = p->st_host->it;
    int next = chunk < 32 ? chunk * 2 : 32;
    if (rr_last > 0.0 && rr > 0.0 && rr < rr_last && it > it_last) {
      const double per_it = std::log(rr / rr_last) / (it - it_last);
      const double rem = std::log(p->st_host->tol2 / rr) / per_it;
      if (rem >= 0.0 && rem < 1e6) {
        const int want = (int)std::ceil(rem) + 1;
        next = std::min(32, std::max(kGraphIters, (want + kGraphIters - 1) / kGraphIters * kGraphIters));
      }
    }
    rr_last = rr;
    it_last = it;
    chunk = next;
  }
  *iters = p->st_host->it;
  switch (p->st_host->status) {
    case 0: return FL_OK;
    case 2: return fail(FL_NOT_CONVERGED, "CG reached the iteration cap");
    default: return fail(FL_BREAKDOWN, "CG breakdown (p^T A p <= 0 or NaN)");
  }
}

// True FP64 relative residual ||b - (shift I + scale M) u|| / ||b|| with b = v64.b.
fl_status true_residual(fl_plan* p, const double* u, double shift, double scale, double* rel) {
  const Geo& g = p->g;
  int c = 0;
  FL_CUDA(launch_mask_copy_dot<double>(g.N, p->stream, p->v64.b, p->mask, (double*)nullptr,
                                       p->part[P_AUX], &c));
  double bb = 0.0;
  fl_status st = read_sum(p, p->part[P_AUX], c, &bb);
  if (st != FL_OK) return st;
  ApplyIO<double> io;
  io.u = u; io.mask = p->mask; io.x = u; io.b = p->v64.b;
  io.cm = -scale; io.cx = -shift; io.cb = 1.0;
  io.partials = p->part[P_RES]; io.dot_self = 1;
  FL_CUDA(launch_apply<double>(g, p->t64, p->stream, io));
  double rr = 0.0;
  st = read_sum(p, p->part[P_RES], apply_partials<double>(g), &rr);
  if (st != FL_OK) return st;
  *rel = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  return FL_OK;
}

// Target relative reduction of the next FP32 inner solve of the FP64
// refinement.  need = tol / rel is the reduction still missing.  Within FP32
// reach (need >= 1e-6) the step aims at half of it, so that it can be the
// last one; otherwise at inner_tol.  floor is the true reduction the previous
// step achieved when that fell short of its target by more than 3x: the
// FP32 round-off of the operator limits what an inner solve can do to the
// true residual, and asking for more than that only spends iterations.
struct InnerTarget {
  double floor = 0.0, eta = 0.0, rel = 0.0;
  double next(double rel_now, double tol, double inner_tol) {
    if (eta > 0.0 && rel > 0.0) {
      const double ratio = rel_now / rel;
      floor = ratio > 3.0 * eta ? ratio : 0.0;
    }
    const double need = rel_now > 0.0 ? tol / rel_now : 1.0;
    eta = std::max(need >= 1e-6 ? 0.5 * need : inner_tol, floor);
    rel = rel_now;
    return eta;
  }
};

// Solve (shift I + scale M) u = b, b already in v64.b; u in/out (device).
bool trace_enabled();

// Flexible CG in FP32 for (shift I + scale M) x = b (b = v32.b, x0 = 0)
// with the learned preconditioner z = z0 + s_z N(r / s_r, z0 / s_z, alpha),
// z0 = the base preconditioner applied to r (FD-Laplacian solve for
// alpha >= 1, a diagonal scaling 1 / M_ii below).  beta is the
// Polak-Ribiere (flexible) one.  Returns FL_BREAKDOWN with *fallback = 1
// when r . z <= 0, so that the caller reruns the fixed preconditioner.
fl_status run_fpcg_learned(fl_plan* p, double shift, double scale, double tol, int maxit, int* iters,
                           int* fallback) {
  const Geo& g = p->g;
  Vecs<float>& v = p->v32;
  cudaStream_t s = p->stream;
  *fallback = 0;
  const bool fd = p->alpha >= 1.0;
  if (fd && !precond_fits(p)) return fail(FL_INVALID_ARG, kPrecondLimit);
  const float jac = (float)(1.0 / (shift + scale * p->c * (p->Z - 2.0 * g.d * p->a)));
  int bb_count = 0, zz_count = 0, rz_count = 0, rr_count = 0;
  if (fd) FL_CUDA(prepare_precond<float>(g, p->t32, shift, scale, s));
  auto base = [&](const PcgState* st) -> cudaError_t {
    cudaError_t e;
    if (fd) {
      PrecIO<float> io;
      io.in = v.r; io.out = p->z0; io.shift = shift; io.scale = scale;
      io.st = const_cast<PcgState*>(st); io.mask = p->mask;
      e = launch_precond<float>(g, p->t32, s, io);
    } else {
      e = launch_scale(v.r, p->z0, jac, g.N, st, s);
    }
    if (e == cudaSuccess) e = launch_dot<float>(g.N, s, p->z0, p->z0, p->lpart[0], &zz_count);
    return e;
  };
  auto learned = [&](const double* rr_part, int rr_cnt, const PcgState* st, double* rzo) -> cudaError_t {
    cudaError_t e = launch_features(v.r, p->z0, rr_part, rr_cnt, p->lpart[0], zz_count,
                                    (float)p->alpha, p->feat, g.N, st, s);
    if (e == cudaSuccess) e = p->net->forward(p->feat, nullptr);
    if (e == cudaSuccess)
      e = launch_combine(v.r, p->z0, p->net->act[kNetTensors - 1], v.z, p->lpart[0], zz_count,
                         p->lpart[1], rzo, g.N, st, &rz_count, s);
    return e;
  };
  FL_CUDA(cudaMemsetAsync(v.x, 0, g.N * sizeof(float), s));
  FL_CUDA(cudaMemsetAsync(v.p, 0, g.N * sizeof(float), s));
  FL_CUDA(cudaMemsetAsync(v.z, 0, g.N * sizeof(float), s));
  FL_CUDA(launch_mask_copy_dot<float>(g.N, s, v.b, p->mask, v.r, p->part[P_BB], &bb_count));
  FL_CUDA(base(nullptr));
  FL_CUDA(learned(p->part[P_BB], bb_count, nullptr, nullptr));
  FL_CUDA(launch_pcg_init(s, p->st, p->part[P_BB], bb_count, p->part[P_BB], bb_count, p->lpart[1],
                          rz_count, tol, maxit));
  for (;;) {
    for (int k = 0; k < 2; ++k) {
      ApplyIO<float> io;
      io.pre = PRE_PUPDATE; io.u = v.z; io.p = v.p; io.mask = p->mask; io.st = p->st;
      io.out = v.q; io.x = v.p; io.cm = scale; io.cx = shift;
      io.dotw = v.p; io.partials = p->part[P_PQ]; io.fin = FIN_PQ;
      FL_CUDA(launch_apply<float>(g, p->t32, s, io));
      FL_CUDA(launch_noprec_update<float>(g.N, s, p->st, v.x, v.r, v.p, v.q, p->part[P_RR], 0,
                                          &rr_count));
      FL_CUDA(base(p->st));
      FL_CUDA(learned(p->part[P_RR], rr_count, p->st, p->lpart[2]));
      FL_CUDA(launch_fpcg_scalar(p->st, p->part[P_RR], rr_count, p->lpart[1], p->lpart[2], rz_count, s));
    }
    fl_status st = read_state(p);
    if (st != FL_OK) return st;
    if (p->st_host->done) break;
  }
  *iters = p->st_host->it;
  switch (p->st_host->status) {
    case 0: return FL_OK;
    case 2: return fail(FL_NOT_CONVERGED, "flexible CG reached the iteration cap");
    case 4: *fallback = 1; return fail(FL_BREAKDOWN, "learned preconditioner gave r.z <= 0");
    // any other breakdown of the learned iteration (e.g. a non-finite network
    // output) also hands the correction to the fixed preconditioner
    default: *fallback = 1; return fail(FL_BREAKDOWN, "flexible CG breakdown");
  }
}

// Order-independent 64-bit hash of the N values of u (device), read back.
fl_status hash_of(fl_plan* p, const double* u, unsigned long long* h) {
  FL_CUDA(cudaMemsetAsync(p->hash_dev, 0, sizeof(unsigned long long), p->stream));
  FL_CUDA(launch_hash(p->g.N, p->stream, u, p->hash_dev));
  FL_CUDA(cudaMemcpyAsync(p->hash_host, p->hash_dev, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                          p->stream));
  FL_CUDA(cudaStreamSynchronize(p->stream));
  *h = *p->hash_host;
  return FL_OK;
}

// mx0 (nullable, with x0_nonzero): M u of the initial u, so that the first
// FP64 residual needs no apply; mx_out (nullable): every FP64 residual apply
// of the refinement also stores M u there.
fl_status solve_system(fl_plan* p, double* u, bool x0_nonzero, double shift, double scale,
                       double tol, int maxit, int mode, fl_solve_info* info,
                       const double* mx0 = nullptr, double* mx_out = nullptr) {
  const Geo& g = p->g;
  cudaStream_t s = p->stream;
  const int prec_mode = mode & 0xF0;
  const int precision = mode & 0x0F;
  if (!(tol > 0.0) || maxit < 1) return fail(FL_INVALID_ARG, "tol must be > 0 and maxit >= 1");
  if (precision == FL_MODE_LEARNED && (!p->net || p->has_mask))
    return fail(FL_INVALID_ARG, "FL_MODE_LEARNED needs a network attached to a plan without mask");
  PrecChoice pc;
  {
    const fl_status ps = precond_params(p, prec_mode, shift, scale, &pc);
    if (ps != FL_OK) return ps;
  }
  fl_solve_info loc;
  memset(&loc, 0, sizeof(loc));
  fl_status result = FL_OK;
  if (precision == FL_MODE_F64) {
    if (x0_nonzero) FL_CUDA(cudaMemcpyAsync(p->v64.x, u, g.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    int its = 0;
    result = run_pcg<double>(p, x0_nonzero, shift, scale, pc, tol, maxit, &its);
    if (result != FL_OK && result != FL_NOT_CONVERGED && result != FL_BREAKDOWN) return result;
    FL_CUDA(cudaMemcpyAsync(u, p->v64.x, g.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    loc.iterations = its;
  } else if (precision == FL_MODE_MIXED || precision == FL_MODE_LEARNED) {
    // FP64 iterative refinement: r = b - A u (FP64), A d = r by FP32 CG to
    // inner_tol, u += d.
    int c = 0;
    FL_CUDA(launch_mask_copy_dot<double>(g.N, s, p->v64.b, p->mask, (double*)nullptr, p->part[P_AUX], &c));
    double bb = 0.0;
    fl_status st = read_sum(p, p->part[P_AUX], c, &bb);
    if (st != FL_OK) return st;
    if (!x0_nonzero) FL_CUDA(cudaMemsetAsync(u, 0, g.N * sizeof(double), s));
    if (bb == 0.0) {
      FL_CUDA(cudaMemsetAsync(u, 0, g.N * sizeof(double), s));
      loc.converged = 1;
    } else {
      int total = 0;
      result = FL_NOT_CONVERGED;
      InnerTarget target;
      for (int outer = 0;; ++outer) {
        double rr = 0.0;
        if (outer == 0 && !x0_nonzero && !p->has_mask) {
          FL_CUDA(launch_copy_cast<float>(g.N, s, p->v64.b, p->v32.b));
          rr = bb;
        } else if (outer == 0 && x0_nonzero && mx0) {
          int cnt = 0;
          FL_CUDA(launch_residual_from(g.N, s, p->v64.b, u, mx0, p->mask, shift, scale, p->v32.b,
                                       p->part[P_RES], &cnt));
          st = read_sum(p, p->part[P_RES], cnt, &rr);
          if (st != FL_OK) return st;
        } else {
          ApplyIO<double> io;
          io.pre = outer > 0 ? PRE_ACCUM : PRE_NONE;
          io.u = u; io.acc = u; io.x32 = p->v32.x; io.mask = p->mask;
          io.out32 = p->v32.b; io.x = u; io.b = p->v64.b; io.outm = mx_out;
          io.cm = -scale; io.cx = -shift; io.cb = 1.0;
          io.partials = p->part[P_RES]; io.dot_self = 1;
          FL_CUDA(launch_apply<double>(g, p->t64, s, io));
          st = read_sum(p, p->part[P_RES], apply_partials<double>(g), &rr);
          if (st != FL_OK) return st;
        }
        loc.rel_residual = std::sqrt(rr / bb);
        loc.outer_iterations = outer;
        if (loc.rel_residual <= tol) { result = FL_OK; break; }
        if (!(rr == rr)) { result = fail(FL_BREAKDOWN, "NaN in the FP64 residual"); break; }
        if (outer >= p->max_outer) { result = fail(FL_NOT_CONVERGED, "refinement step cap reached"); break; }
        const double eta = target.next(loc.rel_residual, tol, p->inner_tol);
        int its = 0;
        fl_status in;
        if (precision == FL_MODE_LEARNED && p->net->alpha_enabled(p->alpha)) {
          int fallback = 0;
          in = run_fpcg_learned(p, shift, scale, eta, maxit, &its, &fallback);
          if (fallback) {   // plain preconditioned CG takes over this correction
            int its2 = 0;
            in = run_pcg<float>(p, false, shift, scale, pc, eta, maxit, &its2);
            its += its2;
          }
        } else {
          in = run_pcg<float>(p, false, shift, scale, pc, eta, maxit, &its);
        }
        total += its;
        if (trace_enabled())
          fprintf(stderr, "fraclap: refinement %d: rel %.3e -> inner eta %.2e, %d its, status %d\n",
                  outer, loc.rel_residual, eta, its, (int)in);
        if (in != FL_OK && in != FL_NOT_CONVERGED) { result = in; break; }
      }
      loc.iterations = total;
    }
  } else {
    return fail(FL_INVALID_ARG, "unknown precision mode");
  }
  // Final FP64 residual.  A converged refinement loop has just computed it
  // for the final u (the last FP64 apply accumulated the last correction
  // into u and formed f - A u from it); otherwise it is formed here.
  double rel = loc.rel_residual;
  const bool have_true = precision != FL_MODE_F64 && result == FL_OK;
  if (!have_true) {
    fl_status st = true_residual(p, u, shift, scale, &rel);
    if (st != FL_OK) return st;
  }
  loc.rel_residual = rel;
  loc.converged = rel <= tol * 1.0000001 ? 1 : 0;
  if (result == FL_OK && !loc.converged && precision == FL_MODE_F64 && rel <= 10 * tol) {
    // recursive and true residual differ by rounding; report, keep OK
  }
  loc.status = result;
  if (info) *info = loc;
  return result;
}

bool check_plan(const fl_plan* p) { return p != nullptr; }

// Axes with a strided pass: 2D the convolution along axis 0; 3D also the
// middle axis (forward/inverse FFT of the apply, DST of the preconditioner).
int strided_axes(const Geo& g, int* axes) {
  axes[0] = 0;
  if (g.d == 3) {
    axes[1] = 1;
    return 2;
  }
  return 1;
}

// Column-tile widths of one precision by timing: per axis with a strided
// pass (the others kept), every power of two from the widest tile down to
// 16 bytes of line element; a trial is kReps FP32/FP64 applies each
// followed by an FD preconditioner solve, on zero data, after one untimed
// trial run.  Keeps the fastest width per axis.
template <typename T>
fl_status autotune_precision(fl_plan* p) {
  constexpr int kReps = 5;
  const Geo& g = p->g;
  Tables<T>& tb = tables<T>(p);
  Vecs<T>& v = vecs<T>(p);
  cudaStream_t s = p->stream;
  FL_CUDA(cudaMemsetAsync(v.p, 0, g.N * sizeof(T), s));
  const bool with_prec = precond_fits(p);
  if (with_prec) FL_CUDA(prepare_precond<T>(g, tb, 0.0, 1.0, s));
  auto trial = [&]() -> cudaError_t {
    ApplyIO<T> io;
    io.u = v.p; io.mask = p->mask; io.out = v.q;
    cudaError_t e = launch_apply<T>(g, tb, s, io);
    if (e != cudaSuccess || !with_prec) return e;
    PrecIO<T> pi;
    pi.in = v.q; pi.out = v.z; pi.shift = 0.0; pi.scale = 1.0; pi.mask = p->mask;
    return launch_precond<T>(g, tb, s, pi);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FL_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce, "cudaEventCreate");
  }
  int axes[2];
  const int na = strided_axes(g, axes);
  for (int ia = 0; ia < na && ce == cudaSuccess; ++ia) {
    const int ax = axes[ia];
    const int widest = col_tx<T>(g.L[ax]);
    int best_tx = widest;
    float best_ms = -1.0f;
    for (int tx = widest; tx >= min_tx<T>() && ce == cudaSuccess; tx /= 2) {
      tb.tx[ax] = tx;
      ce = trial();
      if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
      for (int r = 0; r < kReps && ce == cudaSuccess; ++r) ce = trial();
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce == cudaSuccess && (best_ms < 0.0f || ms < best_ms)) {
        best_ms = ms;
        best_tx = tx;
      }
    }
    tb.tx[ax] = best_tx;
  }
  // FP32 row passes: the 128 x 16 and the 256 x 8 CTA shape (rows_w8.cu)
  if constexpr (sizeof(T) == 4) {
    const int Lx = g.L[g.d - 1];
    if (Lx >= 256 && Lx <= 2048) {
      int best_rs = 0;
      float best_ms = -1.0f;
      for (int rs = 0; rs < 2 && ce == cudaSuccess; ++rs) {
        tb.rshape = rs;
        ce = trial();
        if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
        for (int r = 0; r < kReps && ce == cudaSuccess; ++r) ce = trial();
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce == cudaSuccess && (best_ms < 0.0f || ms < best_ms)) {
          best_ms = ms;
          best_rs = rs;
        }
      }
      tb.rshape = best_rs;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ce != cudaSuccess) return cuda_fail(ce, "tile autotuning");
  return FL_OK;
}

// FRACLAP_TRACE=1 in the environment prints one line per refinement step.
bool trace_enabled() {
  static const bool on = [] {
    const char* v = getenv("FRACLAP_TRACE");
    return v && v[0] == '1';
  }();
  return on;
}

}  // namespace

// --- launch accounting and the per-kernel profiler -----------------------------


namespace fl {
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
bool prof_active() { return t_prof != nullptr; }
cudaEvent_t prof_begin(cudaStream_t s) {
  cudaEvent_t e = t_prof->take();
  cudaEventRecord(e, s);
  return e;
}
void prof_end(const char* name, cudaEvent_t e0, cudaStream_t s) {
  cudaEvent_t e1 = t_prof->take();
  cudaEventRecord(e1, s);
  t_prof->pending.push_back({name, e0, e1});
}
}  // namespace fl


extern "C" {

const char* fl_last_error_string(void) { return g_err.c_str(); }

}  // extern "C"

void fl_set_error_string(const char* msg) { g_err = msg ? msg : ""; }

namespace {
fl_status static_spec_lookup(int dev);
}  // namespace

extern "C" {

fl_status fl_plan_create(int d, const int64_t* n, double h, double alpha, const uint8_t* mask,
                         const fl_opts* opts, fl_plan** out) {
  if (!out) return fail(FL_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (d < 1 || d > 3) return fail(FL_INVALID_ARG, "d must be 1, 2 or 3");
  if (!n) return fail(FL_INVALID_ARG, "n is NULL");
  if (!(h > 0.0) || !std::isfinite(h)) return fail(FL_INVALID_ARG, "h must be > 0");
  if (!(alpha > 0.0 && alpha < 2.0)) return fail(FL_INVALID_ARG, "alpha must be in (0, 2)");
  fl_plan* p = new fl_plan();
  Geo& g = p->g;
  memset(&g, 0, sizeof(g));
  // a 1D problem is laid out as the single row of a 2D grid (1 x n)
  g.dphys = d;
  g.d = d == 1 ? 2 : d;
  int64_t nl[3] = {1, 1, 1};
  for (int i = 0; i < d; ++i) nl[g.d - d + i] = n[i];
  g.N = 1;
  g.lgmax = 0;
  for (int i = 0; i < 3; ++i) { g.n[i] = 1; g.L[i] = 1; g.lg[i] = 0; }
  const int64_t nmax = d == 3 ? 1024 : 4096;
  for (int i = 0; i < g.d; ++i) {
    if (nl[i] < 1 || nl[i] > nmax) {
      delete p;
      return fail(FL_INVALID_ARG, d == 3 ? "each n_i must be in [1, 1024] (d = 3)"
                                         : "each n_i must be in [1, 4096] (d = 1, 2)");
    }
    g.n[i] = (int)nl[i];
    g.lg[i] = std::max(4, ilog2(2 * g.n[i] - 1));  // L_i >= 2 n_i - 1, at least 16
    g.L[i] = 1 << g.lg[i];
    g.lgmax = std::max(g.lgmax, g.lg[i]);
    g.N *= g.n[i];
  }
  g.H = g.L[g.d - 1] / 2 + 1;
  g.spec = (g.d == 2) ? (long long)g.n[0] * g.H : (long long)g.n[0] * g.L[1] * g.H;
  p->h = h;
  p->alpha = alpha;
  p->rho = (opts && opts->rho > 0) ? opts->rho : 20.0;
  p->inner_tol = (opts && opts->inner_tol > 0) ? opts->inner_tol : 1e-4;
  p->max_outer = (opts && opts->max_outer > 0) ? opts->max_outer : 20;
  p->stream = opts ? (cudaStream_t)opts->stream : (cudaStream_t)0;
  p->C = c_alpha_d(alpha, d);
  p->Z = lattice_zeta(d, alpha);
  p->a = window_corr(d, alpha, p->rho);
  p->c = p->C * std::pow(h, -alpha);
  g.cA = p->c * (-p->a);
  fl_status st = FL_OK;
  cudaError_t e = configure_kernels();
  if (e != cudaSuccess) { free_plan(p); return cuda_fail(e, "configure_kernels"); }
  e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) { free_plan(p); return cuda_fail(e, "cudaGetDevice"); }
  // set-up of fl_apply_f32_static on this device: the module holding its
  // scratch array is loaded and the array's address looked up now, not at
  // the first call
  st = static_spec_lookup(p->device);
  if (st != FL_OK) { free_plan(p); return st; }
#define FL_TRY(x)                                   \
  do {                                              \
    cudaError_t e__ = (x);                          \
    if (e__ != cudaSuccess) { free_plan(p); return cuda_fail(e__, #x); } \
  } while (0)
  p->has_mask = false;
  if (mask) {
    for (long long i = 0; i < g.N; ++i)
      if (!mask[i]) { p->has_mask = true; break; }
  }
  if (p->has_mask) {
    FL_TRY(dalloc(p, &p->mask, g.N));
    FL_TRY(cudaMemcpy(p->mask, mask, g.N, cudaMemcpyHostToDevice));
    // Gamma: the points outside Omega with a grid neighbour in Omega (the
    // support of the capacitance correction of the FD solve on Omega)
    std::vector<int> gam;
    long long strides[3] = {1, 1, 1};   // row-major, last axis fastest
    for (int ax = g.d - 2; ax >= 0; --ax) strides[ax] = strides[ax + 1] * g.n[ax + 1];
    for (long long i = 0; i < g.N; ++i) {
      if (mask[i]) continue;
      int c[3] = {0, 0, 0};
      for (int ax = 0; ax < g.d; ++ax) c[ax] = (int)((i / strides[ax]) % g.n[ax]);
      bool near = false;
      for (int ax = 0; ax < g.d && !near; ++ax)
        for (int sg = -1; sg <= 1 && !near; sg += 2) {
          const int v = c[ax] + sg;
          if (v >= 0 && v < g.n[ax] && mask[i + sg * strides[ax]]) near = true;
        }
      if (near) gam.push_back((int)i);
    }
    p->dom_points = (int)gam.size();
    if (p->dom_points > 0 && p->dom_points <= kMaxGamma) {
      p->dom.m = p->dom_points;
      FL_TRY(dalloc(p, &p->dom.idx, gam.size() * sizeof(int)));
      FL_TRY(cudaMemcpy(p->dom.idx, gam.data(), gam.size() * sizeof(int), cudaMemcpyHostToDevice));
      FL_TRY(dalloc(p, &p->dom.LD, (size_t)p->dom.m * p->dom.m * sizeof(double)));
    }
    FL_TRY(dalloc(p, &p->dw32, g.N * sizeof(float)));
    FL_TRY(dalloc(p, &p->dus32, g.N * sizeof(float)));
    FL_TRY(dalloc(p, &p->dw64, g.N * sizeof(double)));
    FL_TRY(dalloc(p, &p->dus64, g.N * sizeof(double)));
    FL_TRY(cudaMemset(p->dus32, 0, g.N * sizeof(float)));
    FL_TRY(cudaMemset(p->dus64, 0, g.N * sizeof(double)));
    FL_TRY(configure_domain_kernels());
  }
  st = build_tables(p);
  if (st != FL_OK) { free_plan(p); return st; }
  long long half = 1;
  for (int i = 0; i < g.d; ++i) half *= g.L[i] / 2 + 1;
  FL_TRY(dalloc(p, &p->t64.sig, half * sizeof(double)));
  FL_TRY(dalloc(p, &p->t32.sig, half * sizeof(float)));
  FL_TRY(build_symbol(g, p->c, p->Z, p->a, d + alpha, p->stream, p->t64.sig, p->t32.sig, p->t64.tw));
  FL_TRY(cudaStreamSynchronize(p->stream));
  FL_TRY(dalloc(p, &p->t64.S, g.spec * sizeof(double2)));
  FL_TRY(dalloc(p, &p->t32.S, g.spec * sizeof(float2)));
  FL_TRY(dalloc(p, &p->t64.t, g.N * sizeof(double)));
  FL_TRY(dalloc(p, &p->t32.t, g.N * sizeof(float)));
  FL_TRY(dalloc(p, &p->t64.tri_tab, (size_t)kTriTab * (g.N / g.n[0]) * sizeof(double)));
  FL_TRY(dalloc(p, &p->t32.tri_tab, (size_t)kTriTab * (g.N / g.n[0]) * sizeof(float)));
  st = alloc_vecs(p, p->v32);
  if (st == FL_OK) st = alloc_vecs(p, p->v64);
  if (st != FL_OK) { free_plan(p); return st; }
  const size_t pc = partial_capacity(g);
  for (int i = 0; i < 6; ++i) FL_TRY(dalloc(p, &p->part[i], pc * sizeof(double)));
  FL_TRY(dalloc(p, &p->dscalar, sizeof(double)));
  FL_TRY(dalloc(p, &p->u_e2e, g.N * sizeof(double)));
  FL_TRY(dalloc(p, &p->st, sizeof(PcgState)));
  FL_TRY(cudaMallocHost(&p->st_host, sizeof(PcgState)));
  FL_TRY(cudaMallocHost(&p->scalar_host, sizeof(double)));
#undef FL_TRY
  *out = p;
  return FL_OK;
}

fl_status fl_plan_destroy(fl_plan* plan) {
  if (!plan) return FL_OK;
  cudaStreamSynchronize(plan->stream);
  free_plan(plan);
  return FL_OK;
}

fl_status fl_plan_describe(const fl_plan* p, fl_plan_desc* desc) {
  if (!check_plan(p) || !desc) return fail(FL_INVALID_ARG, "NULL plan or desc");
  memset(desc, 0, sizeof(*desc));
  desc->d = p->g.dphys;
  for (int i = 0; i < p->g.dphys; ++i) {
    desc->n[i] = p->g.n[p->g.d - p->g.dphys + i];
    desc->fft_len[i] = p->g.L[p->g.d - p->g.dphys + i];
  }
  desc->h = p->h;
  desc->alpha = p->alpha;
  desc->rho = p->rho;
  desc->c_alpha_d = p->C;
  desc->lattice_zeta = p->Z;
  desc->window_corr = p->a;
  desc->kernel0 = p->c * (p->Z - 2.0 * p->g.dphys * p->a);
  desc->workspace_bytes = p->bytes;
  return FL_OK;
}

fl_status fl_plan_set_tiles(fl_plan* p, const int tx[6]) {
  if (!check_plan(p) || !tx) return fail(FL_INVALID_ARG, "NULL argument");
  int axes[2];
  const int na = strided_axes(p->g, axes);
  for (int prec = 0; prec < 2; ++prec) {
    for (int ia = 0; ia < na; ++ia) {
      const int ax = axes[ia];
      const int v = tx[3 * prec + ax];
      const int widest = prec == 0 ? col_tx<float>(p->g.L[ax]) : col_tx<double>(p->g.L[ax]);
      const int narrowest = prec == 0 ? min_tx<float>() : min_tx<double>();
      if (v != 0 && (v < narrowest || v > widest || (v & (v - 1)) != 0))
        return fail(FL_INVALID_ARG, "tile width out of range or not a power of two");
    }
  }
  for (int ia = 0; ia < na; ++ia) {
    p->t32.tx[axes[ia]] = tx[axes[ia]];
    p->t64.tx[axes[ia]] = tx[3 + axes[ia]];
  }
  p->gcache[0].release();
  p->gcache[1].release();
  return FL_OK;
}

fl_status fl_plan_set_row_shape(fl_plan* p, int shape) {
  if (!check_plan(p)) return fail(FL_INVALID_ARG, "NULL plan");
  const int Lx = p->g.L[p->g.d - 1];
  if (shape != 0 && shape != 1) return fail(FL_INVALID_ARG, "row shape must be 0 or 1");
  if (shape == 1 && !(Lx >= 256 && Lx <= 2048))
    return fail(FL_INVALID_ARG, "row shape 1 needs padded rows of 256 .. 2048 points");
  p->t32.rshape = shape;
  p->gcache[0].release();
  p->gcache[1].release();
  return FL_OK;
}

int fl_plan_row_shape(const fl_plan* p) { return p ? p->t32.rshape : -1; }

fl_status fl_plan_autotune(fl_plan* p, int tx_out[6]) {
  ProfScope prof_scope(nullptr);
  if (!check_plan(p)) return fail(FL_INVALID_ARG, "NULL plan");
  p->gcache[0].release();
  p->gcache[1].release();
  fl_status st = autotune_precision<float>(p);
  if (st == FL_OK) st = autotune_precision<double>(p);
  if (st != FL_OK) return st;
  if (tx_out) {
    for (int i = 0; i < 6; ++i) tx_out[i] = 0;
    int axes[2];
    const int na = strided_axes(p->g, axes);
    for (int ia = 0; ia < na; ++ia) {
      const int ax = axes[ia];
      tx_out[ax] = plan_tx<float>(p->t32, ax, p->g.L[ax]);
      tx_out[3 + ax] = plan_tx<double>(p->t64, ax, p->g.L[ax]);
    }
  }
  return FL_OK;
}

fl_status fl_apply(fl_plan* p, const double* u, double* y) {
  ProfScope prof_scope(p);
  if (!check_plan(p) || !u || !y) return fail(FL_INVALID_ARG, "NULL argument");
  if (u == y) return fail(FL_INVALID_ARG, "u and y may not alias");
  ApplyIO<double> io;
  io.u = u; io.mask = p->mask; io.out = y;
  FL_CUDA(launch_apply<double>(p->g, p->t64, p->stream, io));
  return FL_OK;
}

fl_status fl_apply_f32(fl_plan* p, const float* u, float* y) {
  ProfScope prof_scope(p);
  if (!check_plan(p) || !u || !y) return fail(FL_INVALID_ARG, "NULL argument");
  if (u == y) return fail(FL_INVALID_ARG, "u and y may not alias");
  ApplyIO<float> io;
  io.u = u; io.mask = p->mask; io.out = y;
  FL_CUDA(launch_apply<float>(p->g, p->t32, p->stream, io));
  return FL_OK;
}

fl_status fl_precond(fl_plan* p, double shift, double scale, const double* r, double* z) {
  ProfScope prof_scope(p);
  if (!check_plan(p) || !r || !z) return fail(FL_INVALID_ARG, "NULL argument");
  if (r == z) return fail(FL_INVALID_ARG, "r and z may not alias");
  if (!(scale > 0.0) || !(shift >= 0.0) || !std::isfinite(scale) || !std::isfinite(shift))
    return fail(FL_INVALID_ARG, "the preconditioner needs shift >= 0 and scale > 0");
  if (!precond_fits(p)) return fail(FL_INVALID_ARG, kPrecondLimit);
  PrecChoice pc;
  {
    const fl_status ps = precond_params(p, FL_PRECOND_FD, shift, scale, &pc);
    if (ps != FL_OK) return ps;
    const fl_status pp = prepare_prec<double>(p, pc);
    if (pp != FL_OK) return pp;
  }
  PrecIO<double> io;
  io.in = r; io.out = z; io.shift = shift; io.scale = scale; io.mask = p->mask;
  FL_CUDA(apply_prec<double>(p, pc, io, p->stream));
  return FL_OK;
}

fl_status fl_precond_f32(fl_plan* p, double shift, double scale, const float* r, float* z) {
  ProfScope prof_scope(p);
  if (!check_plan(p) || !r || !z) return fail(FL_INVALID_ARG, "NULL argument");
  if (r == z) return fail(FL_INVALID_ARG, "r and z may not alias");
  if (!(scale > 0.0) || !(shift >= 0.0) || !std::isfinite(scale) || !std::isfinite(shift))
    return fail(FL_INVALID_ARG, "the preconditioner needs shift >= 0 and scale > 0");
  if (!precond_fits(p)) return fail(FL_INVALID_ARG, kPrecondLimit);
  PrecChoice pc;
  {
    const fl_status ps = precond_params(p, FL_PRECOND_FD, shift, scale, &pc);
    if (ps != FL_OK) return ps;
    const fl_status pp = prepare_prec<float>(p, pc);
    if (pp != FL_OK) return pp;
  }
  PrecIO<float> io;
  io.in = r; io.out = z; io.shift = shift; io.scale = scale; io.mask = p->mask;
  FL_CUDA(apply_prec<float>(p, pc, io, p->stream));
  return FL_OK;
}

fl_status fl_precond_params(fl_plan* p, int mode, double shift, double scale, double* pshift,
                            double* pscale) {
  ProfScope prof_scope(p);
  if (!check_plan(p) || !pshift || !pscale) return fail(FL_INVALID_ARG, "NULL argument");
  if (!(scale > 0.0) || !(shift >= 0.0) || !std::isfinite(scale) || !std::isfinite(shift))
    return fail(FL_INVALID_ARG, "the operator needs shift >= 0 and scale > 0");
  PrecChoice pc;
  const fl_status st = precond_params(p, mode & 0xF0, shift, scale, &pc);
  if (st != FL_OK) return st;
  *pshift = pc.use ? pc.shift : 0.0;
  *pscale = pc.use ? pc.scale : 0.0;
  return FL_OK;
}

fl_status fl_solve_elliptic(fl_plan* p, const double* f, double* u, int x0_nonzero, double tol,
                            int maxit, int mode, fl_solve_info* info) {
  ProfScope prof_scope(p);
  if (!check_plan(p) || !f || !u) return fail(FL_INVALID_ARG, "NULL argument");
  FL_CUDA(cudaMemcpyAsync(p->v64.b, f, p->g.N * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
  return solve_system(p, u, x0_nonzero != 0, 0.0, 1.0, tol, maxit, mode, info);
}

fl_status fl_solve_elliptic_host(fl_plan* p, const double* f_host, double* u_host, double tol,
                                 int maxit, int mode, fl_solve_info* info) {
  ProfScope prof_scope(p);
  if (!check_plan(p) || !f_host || !u_host) return fail(FL_INVALID_ARG, "NULL argument");
  const size_t bytes = p->g.N * sizeof(double);
  FL_CUDA(cudaMemcpyAsync(p->v64.b, f_host, bytes, cudaMemcpyHostToDevice, p->stream));
  double* u = p->u_e2e;
  fl_status st = solve_system(p, u, false, 0.0, 1.0, tol, maxit, mode, info);
  if (st != FL_OK && st != FL_NOT_CONVERGED) return st;
  FL_CUDA(cudaMemcpyAsync(u_host, u, bytes, cudaMemcpyDeviceToHost, p->stream));
  FL_CUDA(cudaStreamSynchronize(p->stream));
  return st;
}

fl_status fl_time_step(fl_plan* p, double dt, double theta, const double* u_prev,
                       const double* f_prev, const double* f_next, double* u_next, double tol,
                       int maxit, int mode, fl_solve_info* info) {
  ProfScope prof_scope(p);
  if (!check_plan(p) || !u_prev || !u_next) return fail(FL_INVALID_ARG, "NULL argument");
  if (!(dt > 0.0) || !(theta > 0.0 && theta <= 1.0))
    return fail(FL_INVALID_ARG, "dt must be > 0 and theta in (0, 1]");
  const Geo& g = p->g;
  cudaStream_t s = p->stream;
  double* b = p->v64.b;
  const int precision = mode & 0x0F;
  const bool refine = precision == FL_MODE_MIXED || precision == FL_MODE_LEARNED;
  // M u_prev from the previous step (its last FP64 residual apply) when
  // u_prev is that step's result, unchanged since (same array, same hash)
  bool cached = false;
  if (refine) {
    if (!p->mu_cache) FL_CUDA(dalloc(p, &p->mu_cache, g.N * sizeof(double)));
    if (!p->hash_dev) FL_CUDA(dalloc(p, &p->hash_dev, sizeof(unsigned long long)));
    if (!p->hash_host) FL_CUDA(cudaMallocHost((void**)&p->hash_host, sizeof(unsigned long long)));
    if (p->mu_valid && p->mu_of == u_prev) {
      unsigned long long h = 0ull;
      fl_status st = hash_of(p, u_prev, &h);
      if (st != FL_OK) return st;
      cached = h == p->mu_hash;
    }
  }
  p->mu_valid = false;
  // b = (I - (1-theta) dt M) u_prev + dt (theta f_next + (1-theta) f_prev)
  if (theta < 1.0) {
    if (cached) {
      FL_CUDA(launch_axmy(g.N, s, u_prev, (1.0 - theta) * dt, p->mu_cache, b));
    } else {
      ApplyIO<double> io;
      io.u = u_prev; io.mask = p->mask; io.out = b; io.x = u_prev;
      io.cm = -(1.0 - theta) * dt; io.cx = 1.0;
      FL_CUDA(launch_apply<double>(g, p->t64, s, io));
    }
  } else {
    FL_CUDA(cudaMemcpyAsync(b, u_prev, g.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (f_next) FL_CUDA(launch_axpby<double>(g.N, s, theta * dt, f_next, 1.0, b));
  if (f_prev && theta < 1.0) FL_CUDA(launch_axpby<double>(g.N, s, (1.0 - theta) * dt, f_prev, 1.0, b));
  if (u_next != u_prev)
    FL_CUDA(cudaMemcpyAsync(u_next, u_prev, g.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  const fl_status res = solve_system(p, u_next, true, 1.0, theta * dt, tol, maxit, mode, info,
                                     cached ? p->mu_cache : nullptr, refine ? p->mu_cache : nullptr);
  if (refine && (res == FL_OK || res == FL_NOT_CONVERGED)) {
    // the refinement's last FP64 residual apply stored M u_next
    unsigned long long h = 0ull;
    fl_status st = hash_of(p, u_next, &h);
    if (st != FL_OK) return st;
    p->mu_of = u_next;
    p->mu_hash = h;
    p->mu_valid = true;
  }
  return res;
}

long long fl_launch_count(void) { return g_launches.load(); }

fl_status fl_check_grid_barrier(int missing) {
  if (missing < 0 || missing > 1024) return fail(FL_INVALID_ARG, "missing must be in [0, 1024]");
  int gave_up = 0;
  FL_CUDA(persist_barrier_check(missing, &gave_up));
  if (gave_up) return fail(FL_DEVICE_TIMEOUT, "grid barrier: the CTAs gave up waiting");
  return FL_OK;
}

fl_status fl_profile_enable(fl_plan* p, int enable) {
  if (!check_plan(p)) return fail(FL_INVALID_ARG, "NULL plan");
  if (enable && !p->prof) p->prof = new Profiler();
  if (!enable && p->prof) {
    FL_CUDA(cudaStreamSynchronize(p->stream));
    delete p->prof;
    p->prof = nullptr;
  }
  return FL_OK;
}

int fl_profile_read(fl_plan* p, fl_kernel_stat* stats, int max_stats) {
  if (!check_plan(p) || !p->prof) return 0;
  cudaStreamSynchronize(p->stream);
  p->prof->resolve();
  const int n = (int)p->prof->stats.size();
  for (int i = 0; i < n && i < max_stats && stats; ++i) {
    const auto& st = p->prof->stats[i];
    memset(&stats[i], 0, sizeof(fl_kernel_stat));
    strncpy(stats[i].name, st.name.c_str(), sizeof(stats[i].name) - 1);
    stats[i].launches = st.launches;
    stats[i].total_ms = st.ms;
  }
  return n;
}

}  // extern "C"

// --- allocation-free FP32 apply ----------------------------------------------
// The half-spectrum workspace of fl_apply_f32_static.  In host code the name
// g_static_spec is only a stand-in: the kernels get the device address that
// cudaGetSymbolAddress returns with the plan's device current, looked up by
// fl_plan_create (set-up time) and kept per device.
namespace {
constexpr long long kStaticSpecElems = 1LL << 21;  // complex floats, 16 MiB
constexpr int kMaxDevices = 256;
static __device__ __align__(256) float2 g_static_spec[kStaticSpecElems];
std::mutex g_static_mu;
float2* g_static_addr[kMaxDevices] = {nullptr};

// Looks up (once) the device address of g_static_spec on device `dev`,
// which must be the current device.
fl_status static_spec_lookup(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return fail(FL_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* ptr = nullptr;
    FL_CUDA(cudaGetSymbolAddress(&ptr, g_static_spec));
    g_static_addr[dev] = reinterpret_cast<float2*>(ptr);
  }
  return FL_OK;
}
}  // namespace

extern "C" {

fl_status fl_apply_f32_static(fl_plan* p, const float* u, float* y) {
  ProfScope prof_scope(p);
  if (!check_plan(p) || !u || !y) return fail(FL_INVALID_ARG, "NULL argument");
  if (u == y) return fail(FL_INVALID_ARG, "u and y may not alias");
  if (p->g.spec > kStaticSpecElems)
    return fail(FL_INVALID_ARG, "plan too large for the static scratch (2^21 complex floats)");
  int dev = -1;
  FL_CUDA(cudaGetDevice(&dev));
  if (dev != p->device)
    return fail(FL_INVALID_ARG, "fl_apply_f32_static: the plan's device must be current");
  float2* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    scratch = g_static_addr[p->device];
  }
  if (!scratch) return fail(FL_INVALID_ARG, "static scratch not set up for the plan's device");
  Tables<float> tb = p->t32;
  tb.S = scratch;
  ApplyIO<float> io;
  io.u = u; io.mask = p->mask; io.out = y;
  FL_CUDA(launch_apply<float>(p->g, tb, p->stream, io));
  return FL_OK;
}

fl_status fl_sync(fl_plan* p) {
  if (!check_plan(p)) return fail(FL_INVALID_ARG, "NULL plan");
  FL_CUDA(cudaStreamSynchronize(p->stream));
  return FL_OK;
}

}  // extern "C"

// --- batched solves ------------------------------------------------------------
// Many independent elliptic problems (different sizes and orders) advance in
// lockstep: every pass of the FP64 residual, of the FP32 CG start-up and of a
// CG iteration is ONE launch over all problems (batch.cu).  The CG iteration
// chunk is captured once into a CUDA graph and replayed until every
// problem's device state reports done; problems that are done leave at the
// entry of each kernel.
namespace {

struct DevArena {
  std::vector<void*> ptrs;
  cudaError_t err = cudaSuccess;
  ~DevArena() {
    for (void* q : ptrs) cudaFree(q);
  }
  template <typename X>
  X* upload(const std::vector<X>& v) {
    if (v.empty() || err != cudaSuccess) return nullptr;
    void* d = nullptr;
    err = cudaMalloc(&d, v.size() * sizeof(X));
    if (err != cudaSuccess) return nullptr;
    ptrs.push_back(d);
    err = cudaMemcpy(d, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice);
    return reinterpret_cast<X*>(d);
  }
  template <typename X>
  X* alloc(size_t n) {
    if (err != cudaSuccess) return nullptr;
    void* d = nullptr;
    err = cudaMalloc(&d, n * sizeof(X));
    if (err == cudaSuccess) ptrs.push_back(d);
    return reinterpret_cast<X*>(d);
  }
};

template <typename A>
struct PassSet {
  std::vector<A> args;
  std::vector<int> off{0};
  std::vector<int> gx;
  size_t smem = 0;
  void add(const A& a, int blocks, int gxv, size_t sm) {
    args.push_back(a);
    off.push_back(off.back() + blocks);
    gx.push_back(gxv);
    smem = std::max(smem, sm);
  }
  BatchPass upload(DevArena& ar, int kind) {
    BatchPass bp;
    bp.kind = kind;
    bp.nprob = (int)args.size();
    bp.blocks = off.back();
    bp.smem = smem;
    bp.args = ar.upload(args);
    bp.off = ar.upload(off);
    bp.gx = ar.upload(gx);
    return bp;
  }
};

inline int vec_blocks(long long N) {
  return (int)std::min<long long>(kVecBlocks, std::max<long long>(1, (N + 1023) / 1024));
}

template <typename T>
struct ChainSets {
  PassSet<RowsFwdArgs<T>> fwd;
  PassSet<ColsArgs<T>> cols[3];
  PassSet<RowsInvArgs<T>> inv;
  void add(const ApplyChain<T>& ch) {
    fwd.add(ch.fwd, ch.row_blocks, ch.row_blocks, ch.row_smem);
    for (int j = 0; j < ch.ncols; ++j)
      cols[j].add(ch.cols[j], (int)(ch.cols_grid[j].x * ch.cols_grid[j].y), (int)ch.cols_grid[j].x,
                  ch.cols_smem[j]);
    inv.add(ch.inv, ch.row_blocks, ch.row_blocks, ch.row_smem);
  }
};

template <typename T>
struct PrecSets {
  PassSet<DstRowsArgs<T>> first;
  PassSet<DstColsArgs<T>> cols[3];
  PassSet<TriArgs<T>> tri;
  PassSet<DstRowsArgs<T>> last;
  int ncols = 0, tri_after = 0;
  void add(const PrecChain<T>& ch) {
    first.add(ch.first, ch.row_blocks, ch.row_blocks, ch.row_smem);
    for (int j = 0; j < ch.ncols; ++j)
      cols[j].add(ch.cols[j], (int)(ch.cols_grid[j].x * ch.cols_grid[j].y), (int)ch.cols_grid[j].x,
                  ch.cols_smem[j]);
    tri.add(ch.tri, ch.tri_blocks, ch.tri_blocks, 0);
    last.add(ch.last, ch.row_blocks, ch.row_blocks, ch.row_smem);
    ncols = ch.ncols;          // the same for every problem of one dimension
    tri_after = ch.tri_after;
  }
};

template <typename T>
struct ChainPasses {
  BatchPass fwd, cols[3], inv;
  int ncols = 0;
  void upload(DevArena& ar, ChainSets<T>& cs, int ncols_) {
    ncols = ncols_;
    fwd = cs.fwd.upload(ar, BK_ROWS_FWD);
    for (int j = 0; j < ncols; ++j) cols[j] = cs.cols[j].upload(ar, BK_COLS);
    inv = cs.inv.upload(ar, BK_ROWS_INV);
  }
  cudaError_t launch(cudaStream_t s) const {
    cudaError_t e = launch_batched<T>(fwd, s);
    for (int j = 0; j < ncols && e == cudaSuccess; ++j) e = launch_batched<T>(cols[j], s);
    if (e == cudaSuccess) e = launch_batched<T>(inv, s);
    return e;
  }
};

template <typename T>
struct PrecPasses {
  BatchPass first, cols[3], tri, last;
  int ncols = 0, tri_after = 0;
  void upload(DevArena& ar, PrecSets<T>& ps) {
    ncols = ps.ncols;
    tri_after = ps.tri_after;
    first = ps.first.upload(ar, BK_DST_ROWS);
    for (int j = 0; j < ncols; ++j) cols[j] = ps.cols[j].upload(ar, BK_DST_COLS);
    tri = ps.tri.upload(ar, BK_TRI_COLS);
    last = ps.last.upload(ar, BK_DST_ROWS);
  }
  cudaError_t launch(cudaStream_t s) const {
    cudaError_t e = launch_batched<T>(first, s);
    for (int j = 0; j <= ncols && e == cudaSuccess; ++j) {
      if (j == tri_after) e = launch_batched<T>(tri, s);
      if (j < ncols && e == cudaSuccess) e = launch_batched<T>(cols[j], s);
    }
    if (e == cudaSuccess) e = launch_batched<T>(last, s);
    return e;
  }
};

fl_status solve_batched_mixed(fl_plan* const* plans, int count, const double* const* f,
                              double* const* u, double tol, int maxit, int prec_mode, bool persist,
                              fl_solve_info* infos) {
  const int d = plans[0]->g.d;
  const int ncols = d == 2 ? 1 : 3;
  DevArena ar;
  PcgState* gates = ar.alloc<PcgState>(count);
  double* tol_dev = ar.alloc<double>(count);
  double* sums = ar.alloc<double>(count);
  if (ar.err != cudaSuccess) return cuda_fail(ar.err, "batched workspace");
  std::vector<int> prec(count);
  ChainSets<double> res64;
  PassSet<BVecArgs<double>> cast;
  std::vector<float*> out32(count);
  std::vector<BScalarArgs> sum_cast(count), sum_res(count), init(count);
  PassSet<BVecArgs<float>> start, noprec;
  PrecSets<float> pinit, pstep;
  ChainSets<float> apply32;
  for (int i = 0; i < count; ++i) {
    fl_plan* p = plans[i];
    const Geo& g = p->g;
    const int vb = vec_blocks(g.N);
    PrecChoice pc;
    {
      const fl_status ps = precond_params(p, prec_mode, 0.0, 1.0, &pc);
      if (ps != FL_OK) return ps;
    }
    prec[i] = pc.use;
    PcgState* st = p->st;
    const PcgState* gate = gates + i;
    // FP64: right-hand side of the zero guess, then residuals with u += x32
    BVecArgs<double> c = {};
    c.b = f[i]; c.x = u[i]; c.mask = p->mask; c.part = p->part[P_RES]; c.N = g.N;
    cast.add(c, vb, vb, 0);
    out32[i] = p->v32.b;
    sum_cast[i] = BScalarArgs{nullptr, gate, nullptr, 0, p->part[P_RES], vb, nullptr, 0, nullptr, 0};
    ApplyIO<double> io64;
    io64.pre = PRE_ACCUM; io64.u = u[i]; io64.acc = u[i]; io64.x32 = p->v32.x; io64.mask = p->mask;
    io64.st = const_cast<PcgState*>(gate); io64.out32 = p->v32.b; io64.x = u[i]; io64.b = f[i];
    io64.cm = -1.0; io64.cx = 0.0; io64.cb = 1.0; io64.partials = p->part[P_RES]; io64.dot_self = 1;
    res64.add(build_apply<double>(g, p->t64, io64));
    sum_res[i] = BScalarArgs{nullptr, gate, nullptr, 0, p->part[P_RES], apply_partials<double>(g),
                             nullptr, 0, nullptr, 0};
    // FP32 CG start-up (x0 = 0)
    BVecArgs<float> sa = {};
    sa.gate = gate; sa.st = st; sa.b = p->v32.b; sa.x = p->v32.x; sa.r = p->v32.r; sa.p = p->v32.p;
    sa.mask = p->mask; sa.part = p->part[P_BB]; sa.N = g.N;
    start.add(sa, vb, vb, 0);
    const int pcount = precond_partials<float>(g);
    if (prec[i]) {
      // on the plan's stream, before the batched stream waits for it
      FL_CUDA(prepare_precond<float>(g, p->t32, pc.shift, pc.scale, p->stream));
      PrecIO<float> pi;
      pi.shift = pc.shift; pi.scale = pc.scale;
      pi.in = p->v32.r; pi.out = p->v32.z; pi.dotw = p->v32.r; pi.dot_part = p->part[P_RZ];
      pi.mask = p->mask;
      pi.st = const_cast<PcgState*>(gate);
      pinit.add(build_precond<float>(g, p->t32, pi));
    }
    init[i] = BScalarArgs{st, gate, p->part[P_BB], vb, nullptr, 0,
                          prec[i] ? p->part[P_RZ] : p->part[P_BB], prec[i] ? pcount : vb,
                          tol_dev + i, maxit};
    // one CG iteration
    ApplyIO<float> ioa;
    ioa.pre = PRE_PUPDATE; ioa.u = prec[i] ? p->v32.z : p->v32.r; ioa.p = p->v32.p;
    ioa.mask = p->mask; ioa.st = st; ioa.out = p->v32.q; ioa.x = p->v32.p; ioa.cm = 1.0;
    ioa.dotw = p->v32.p; ioa.partials = p->part[P_PQ]; ioa.fin = FIN_PQ;
    ioa.row_threads = ioa.col_threads = persist ? kPersistThreads : 0;
    apply32.add(build_apply<float>(g, p->t32, ioa));
    // the x/r update and the CG scalar step (in the last CTA of the last pass)
    if (prec[i]) {
      PrecIO<float> pu;
      pu.shift = pc.shift; pu.scale = pc.scale;
      pu.pre = DPRE_UPDATE; pu.out = p->v32.z; pu.x = p->v32.x; pu.r = p->v32.r; pu.p = p->v32.p;
      pu.q = p->v32.q; pu.rr_part = p->part[P_RR]; pu.dotw = p->v32.r; pu.dot_part = p->part[P_RZ];
      pu.st = st; pu.fin = FIN_STEP; pu.mask = p->mask;
      pu.row_threads = pu.col_threads = persist ? kPersistThreads : 0;
      pu.tri_cols = persist ? kPersistTriCols : 0;
      pstep.add(build_precond<float>(g, p->t32, pu));
    } else {
      BVecArgs<float> nu = {};
      nu.st = st; nu.x = p->v32.x; nu.r = p->v32.r; nu.p = p->v32.p; nu.q = p->v32.q;
      nu.mask = p->mask; nu.part = p->part[P_RR]; nu.N = g.N;
      noprec.add(nu, vb, vb, 0);
    }
  }
  // upload every argument array once
  ChainPasses<double> R64;
  R64.upload(ar, res64, ncols);
  BatchPass CAST = cast.upload(ar, BK_CAST);
  float* const* out32_dev = ar.upload(out32);
  BScalarArgs* SUMC = ar.upload(sum_cast);
  BScalarArgs* SUMR = ar.upload(sum_res);
  BScalarArgs* INIT = ar.upload(init);
  BatchPass START = start.upload(ar, BK_CG_START);
  BatchPass NOPREC = noprec.upload(ar, BK_NOPREC);
  PrecPasses<float> PI, PS;
  PI.upload(ar, pinit);
  PS.upload(ar, pstep);
  ChainPasses<float> A32;
  A32.upload(ar, apply32, ncols);
  // the lockstep FP32 row passes take the 256 x 8 shape when every plan's
  // tuned (or set) row shape is that one (fl_plan_set_row_shape)
  if (!persist) {
    bool w8 = true;
    for (int i = 0; i < count && w8; ++i) w8 = rows_w8(plans[i]->t32, plans[i]->g.L[plans[i]->g.d - 1]);
    if (w8) {
      for (BatchPass* bp : {&A32.fwd, &A32.inv, &PI.first, &PI.last, &PS.first, &PS.last}) bp->w8 = 1;
    }
  }
  // the persistent launch: the CG iteration's passes as phases (the update
  // pass of the preconditioned problems and the plain update of the others
  // side by side), the problems' CG states and the barrier
  std::vector<PPhase> phases;
  size_t psmem = 0;
  bool map_overflow = false;
  if (persist) {
    // per logical block of a pass: its problem and its block within the
    // problem, packed (one load in the kernel instead of a search)
    auto item = [&](const BatchPass& bp, const std::vector<int>& off) {
      PItem it;
      it.kind = bp.kind; it.nprob = bp.nprob; it.blocks = bp.blocks;
      it.args = bp.args; it.off = bp.off; it.gx = bp.gx;
      std::vector<int> map(bp.blocks);
      for (int i = 0; i < bp.nprob; ++i) {
        if (off[i + 1] - off[i] >= (1 << 20)) map_overflow = true;
        for (int l = off[i]; l < off[i + 1]; ++l) map[l] = (i << 20) | (l - off[i]);
      }
      it.map = ar.upload(map);
      return it;
    };
    auto phase = [&](const BatchPass& a, const std::vector<int>& aoff, const BatchPass* b,
                     const std::vector<int>* boff) {
      PPhase ph;
      const std::pair<const BatchPass*, const std::vector<int>*> xs[2] = {{&a, &aoff}, {b, boff}};
      for (const auto& xo : xs) {
        const BatchPass* x = xo.first;
        if (!x || x->nprob == 0 || x->blocks == 0) continue;
        ph.item[ph.nitems++] = item(*x, *xo.second);
        ph.blocks += x->blocks;
        psmem = std::max(psmem, x->smem);
      }
      if (ph.nitems) phases.push_back(ph);
    };
    phase(A32.fwd, apply32.fwd.off, nullptr, nullptr);
    for (int j = 0; j < A32.ncols; ++j) phase(A32.cols[j], apply32.cols[j].off, nullptr, nullptr);
    phase(A32.inv, apply32.inv.off, nullptr, nullptr);
    phase(PS.first, pstep.first.off, &NOPREC, &noprec.off);
    for (int j = 0; j <= PS.ncols; ++j) {
      if (j == PS.tri_after) phase(PS.tri, pstep.tri.off, nullptr, nullptr);
      if (j < PS.ncols) phase(PS.cols[j], pstep.cols[j].off, nullptr, nullptr);
    }
    phase(PS.last, pstep.last.off, nullptr, nullptr);
  }
  PPhase* phases_dev = ar.upload(phases);
  std::vector<PcgState*> states(count);
  for (int i = 0; i < count; ++i) states[i] = plans[i]->st;
  PcgState* const* states_dev = persist ? ar.upload(states) : nullptr;
  PBarrier* pbar = persist ? ar.alloc<PBarrier>(1) : nullptr;
  if (ar.err != cudaSuccess) return cuda_fail(ar.err, "batched argument upload");
  int pgrid = 0;
  if (map_overflow)
    return fail(FL_INVALID_ARG, "FL_BATCH_PERSISTENT: a pass of one problem has 2^20 or more blocks");
  if (persist) {
    FL_CUDA(persist_configure(psmem, &pgrid));
    if (pgrid < 1) return fail(FL_CUDA_ERROR, "the device cannot run the persistent batched launch");
  }

  // a private stream (capturable), ordered after and before the plans' streams
  cudaStream_t bs = nullptr;
  cudaEvent_t ev = nullptr;
  FL_CUDA(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s;
    cudaEvent_t e;
    ~StreamGuard() {
      if (e) cudaEventDestroy(e);
      if (s) cudaStreamDestroy(s);
    }
  } guard{bs, nullptr};
  FL_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  guard.e = ev;
  for (int i = 0; i < count; ++i) {
    FL_CUDA(cudaEventRecord(ev, plans[i]->stream));
    FL_CUDA(cudaStreamWaitEvent(bs, ev, 0));
  }
  std::vector<PcgState> gh(count), sh(count);
  std::vector<double> rr(count), bb(count), tolh(count);
  std::vector<int> its(count, 0), outers(count, 0), conv(count, 0);
  std::vector<InnerTarget> targets(count);
  memset(gh.data(), 0, count * sizeof(PcgState));
  FL_CUDA(cudaMemcpyAsync(gates, gh.data(), count * sizeof(PcgState), cudaMemcpyHostToDevice, bs));
  auto read_sums = [&](std::vector<double>& out) -> fl_status {
    FL_CUDA(cudaMemcpyAsync(out.data(), sums, count * sizeof(double), cudaMemcpyDeviceToHost, bs));
    FL_CUDA(cudaStreamSynchronize(bs));
    return FL_OK;
  };
  // outer 0: the residual of u = 0 is f
  FL_CUDA(launch_cast_rhs(CAST, out32_dev, bs));
  FL_CUDA(launch_batched_scalar(2, SUMC, sums, count, bs));
  fl_status st = read_sums(bb);
  if (st != FL_OK) return st;
  rr = bb;
  // graph of a chunk of CG iterations, captured on first use
  const int kChunk = 8;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  struct GraphGuard {
    cudaGraph_t* g;
    cudaGraphExec_t* x;
    ~GraphGuard() {
      if (*x) cudaGraphExecDestroy(*x);
      if (*g) cudaGraphDestroy(*g);
    }
  } gguard{&graph, &exec};
  long long kernels_per_chunk = 0;
  bool persist_direct = false;
  if (persist) FL_CUDA(cudaMemsetAsync(pbar, 0, sizeof(PBarrier), bs));
  fl_status result = FL_OK;
  fl_plan* p0 = plans[0];
  for (int outer = 0;; ++outer) {
    bool all = true;
    for (int i = 0; i < count; ++i) {
      const double rel = bb[i] > 0 ? std::sqrt(rr[i] / bb[i]) : 0.0;
      conv[i] = rel <= tol;
      all = all && conv[i];
      if (!conv[i]) tolh[i] = targets[i].next(rel, tol, plans[i]->inner_tol);
      gh[i].done = conv[i];
      if (!conv[i]) outers[i] = outer;
    }
    if (all) break;
    if (outer >= p0->max_outer) {
      result = fail(FL_NOT_CONVERGED, "refinement step cap reached");
      break;
    }
    FL_CUDA(cudaMemcpyAsync(gates, gh.data(), count * sizeof(PcgState), cudaMemcpyHostToDevice, bs));
    FL_CUDA(cudaMemcpyAsync(tol_dev, tolh.data(), count * sizeof(double), cudaMemcpyHostToDevice, bs));
    // inner FP32 CG start-up
    FL_CUDA(launch_batched<float>(START, bs));
    FL_CUDA(PI.launch(bs));
    FL_CUDA(launch_batched_scalar(0, INIT, nullptr, count, bs));
    if (persist) {
      // every CG iteration of every problem in one cooperative launch,
      // captured once into a graph (direct launches if the capture fails)
      const int max_iters = maxit + 1;
      if (!exec && !persist_direct) {
        ProfScope off(nullptr);
        FL_CUDA(cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal));
        const cudaError_t ce = launch_persist_cg(phases_dev, (int)phases.size(), states_dev, count,
                                                 max_iters, pbar, pgrid, psmem, bs);
        const cudaError_t ee = cudaStreamEndCapture(bs, &graph);
        cudaError_t ie = cudaErrorUnknown;
        if (ce == cudaSuccess && ee == cudaSuccess) ie = cudaGraphInstantiate(&exec, graph, 0);
        if (ie != cudaSuccess) {
          cudaGetLastError();
          if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
          if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
          persist_direct = true;
        }
        g_launches.fetch_sub(1);   // counted when the graph runs
      }
      if (exec) {
        FL_CUDA(cudaGraphLaunch(exec, bs));
        g_launches.fetch_add(1);
      } else {
        FL_CUDA(launch_persist_cg(phases_dev, (int)phases.size(), states_dev, count, max_iters, pbar,
                                  pgrid, psmem, bs));
      }
      PBarrier bh = {};
      for (int i = 0; i < count; ++i)
        FL_CUDA(cudaMemcpyAsync(&sh[i], plans[i]->st, sizeof(PcgState), cudaMemcpyDeviceToHost, bs));
      FL_CUDA(cudaMemcpyAsync(&bh, pbar, sizeof(PBarrier), cudaMemcpyDeviceToHost, bs));
      FL_CUDA(cudaStreamSynchronize(bs));
      if (bh.err) {
        cudaMemsetAsync(pbar, 0, sizeof(PBarrier), bs);
        cudaStreamSynchronize(bs);
        return fail(FL_DEVICE_TIMEOUT, "persistent batched launch: a CTA gave up at a grid barrier");
      }
    }
    if (!persist && !exec) {
      const long long before = fl_launch_count();
      ProfScope off(nullptr);
      FL_CUDA(cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal));
      cudaError_t ce = cudaSuccess;
      for (int k = 0; k < kChunk && ce == cudaSuccess; ++k) {
        ce = A32.launch(bs);
        if (ce == cudaSuccess) ce = PS.launch(bs);
        if (ce == cudaSuccess) ce = launch_batched<float>(NOPREC, bs);
      }
      cudaError_t ee = cudaStreamEndCapture(bs, &graph);
      if (ce != cudaSuccess) return cuda_fail(ce, "batched CG capture");
      if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture");
      FL_CUDA(cudaGraphInstantiate(&exec, graph, 0));
      kernels_per_chunk = fl_launch_count() - before;
      g_launches.fetch_sub(kernels_per_chunk);   // counted when the graph runs
    }
    for (; !persist;) {
      FL_CUDA(cudaGraphLaunch(exec, bs));
      g_launches.fetch_add(kernels_per_chunk);
      bool alldone = true;
      for (int i = 0; i < count; ++i) {
        FL_CUDA(cudaMemcpyAsync(&sh[i], plans[i]->st, sizeof(PcgState), cudaMemcpyDeviceToHost, bs));
      }
      FL_CUDA(cudaStreamSynchronize(bs));
      for (int i = 0; i < count; ++i) alldone = alldone && sh[i].done;
      if (alldone) break;
    }
    for (int i = 0; i < count; ++i)
      if (!conv[i]) its[i] += sh[i].it;
    // FP64 residual with u += x32 (skips converged problems)
    FL_CUDA(R64.launch(bs));
    FL_CUDA(launch_batched_scalar(2, SUMR, sums, count, bs));
    std::vector<double> fresh(count);
    st = read_sums(fresh);
    if (st != FL_OK) return st;
    for (int i = 0; i < count; ++i)
      if (!conv[i]) rr[i] = fresh[i];
  }
  FL_CUDA(cudaEventRecord(ev, bs));
  for (int i = 0; i < count; ++i) FL_CUDA(cudaStreamWaitEvent(plans[i]->stream, ev, 0));
  FL_CUDA(cudaStreamSynchronize(bs));
  if (infos) {
    for (int i = 0; i < count; ++i) {
      fl_solve_info& in = infos[i];
      memset(&in, 0, sizeof(in));
      in.iterations = its[i];
      in.outer_iterations = outers[i] + (conv[i] && its[i] > 0 ? 1 : 0);
      in.rel_residual = bb[i] > 0 ? std::sqrt(rr[i] / bb[i]) : 0.0;
      in.converged = conv[i];
      in.status = conv[i] ? FL_OK : FL_NOT_CONVERGED;
    }
  }
  return result;
}

}  // namespace

extern "C" {

fl_status fl_solve_elliptic_batched(fl_plan* const* plans, int count, const double* const* f_dev,
                                    double* const* u_dev, double tol, int maxit, int mode,
                                    fl_solve_info* infos) {
  if (!plans || !f_dev || !u_dev || count < 1) return fail(FL_INVALID_ARG, "NULL argument or count < 1");
  for (int i = 0; i < count; ++i) {
    if (!plans[i] || !f_dev[i] || !u_dev[i]) return fail(FL_INVALID_ARG, "NULL plan or array");
    if (plans[i]->g.dphys != plans[0]->g.dphys)
      return fail(FL_INVALID_ARG, "all plans must have the same d");
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return fail(FL_INVALID_ARG, "a plan appears twice in the batch");
  }
  if (!(tol > 0.0) || maxit < 1) return fail(FL_INVALID_ARG, "tol must be > 0 and maxit >= 1");
  const int precision = mode & 0x0F, prec_mode = mode & 0xF0;
  if (prec_mode != FL_PRECOND_FD && prec_mode != FL_PRECOND_NONE && prec_mode != FL_PRECOND_AUTO &&
      prec_mode != FL_PRECOND_SHIFTED && prec_mode != FL_PRECOND_STENCIL && prec_mode != FL_PRECOND_BOX)
    return fail(FL_INVALID_ARG, "unknown preconditioner mode");
  if (precision == FL_MODE_F64) {
    // plain FP64 CG: the problems one after another
    fl_status worst = FL_OK;
    for (int i = 0; i < count; ++i) {
      fl_status s = fl_solve_elliptic(plans[i], f_dev[i], u_dev[i], 0, tol, maxit, mode,
                                      infos ? infos + i : nullptr);
      if (s != FL_OK && s != FL_NOT_CONVERGED) return s;
      if (s != FL_OK) worst = s;
    }
    return worst;
  }
  if (precision != FL_MODE_MIXED) return fail(FL_INVALID_ARG, "unknown precision mode");
  for (int i = 0; i < count; ++i)
    if (plans[i]->has_mask && prec_mode != FL_PRECOND_NONE && prec_mode != FL_PRECOND_BOX &&
        !(prec_mode == FL_PRECOND_AUTO && plans[i]->alpha < 1.0))
      return fail(FL_INVALID_ARG, "batched mixed solves of masked plans take FL_PRECOND_BOX or none");
  for (int i = 0; i < count; ++i)
    for (int ax = 0; ax < plans[i]->g.d; ++ax)
      if (plans[i]->g.L[ax] > 2048)
        return fail(FL_INVALID_ARG, "batched mixed solves need padded lengths <= 2048 (n_i <= 1024)");
  cudaError_t e = configure_batched_kernels();
  if (e != cudaSuccess) return cuda_fail(e, "configure_batched_kernels");
  // the persistent launch packs the problem index into 11 bits
  const bool persist = (mode & FL_BATCH_PERSISTENT) != 0 && count < 2048;
  return solve_batched_mixed(plans, count, f_dev, u_dev, tol, maxit, prec_mode, persist, infos);
}

}  // extern "C"

extern "C" {

fl_status fl_net_training_pair(fl_plan* p, const double* f, const double* u_star, const double* x,
                               float* feat, float* target) {
  ProfScope prof_scope(p);
  if (!check_plan(p) || !f || !u_star || !x || !feat || !target)
    return fail(FL_INVALID_ARG, "NULL argument");
  if (p->has_mask) return fail(FL_INVALID_ARG, "training pairs are formed on box plans");
  const Geo& g = p->g;
  cudaStream_t s = p->stream;
  double* r = p->v64.r;
  double* z0 = p->v64.z;
  // r = f - M x (FP64 apply, the epilogue forms the residual)
  ApplyIO<double> io;
  io.u = x; io.out = r; io.x = x; io.b = f; io.cm = -1.0; io.cx = 0.0; io.cb = 1.0;
  FL_CUDA(launch_apply<double>(g, p->t64, s, io));
  // z0 = B r: the FD-Laplacian solve for alpha >= 1, r / M_ii below
  if (p->alpha >= 1.0) {
    if (!precond_fits(p)) return fail(FL_INVALID_ARG, kPrecondLimit);
    PrecChoice pc;
    const fl_status ps = precond_params(p, FL_PRECOND_FD, 0.0, 1.0, &pc);
    if (ps != FL_OK) return ps;
    const fl_status pp = prepare_prec<double>(p, pc);
    if (pp != FL_OK) return pp;
    PrecIO<double> pi;
    pi.in = r; pi.out = z0; pi.shift = 0.0; pi.scale = 1.0;
    FL_CUDA(apply_prec<double>(p, pc, pi, s));
  } else {
    const double k0 = p->c * (p->Z - 2.0 * g.dphys * p->a);
    FL_CUDA(launch_div_scalar(r, k0, z0, g.N, s));
  }
  FL_CUDA(launch_training_pair(r, z0, u_star, x, p->alpha, feat, target, g.N, p->part[P_AUX], s));
  return FL_OK;
}

fl_status fl_plan_attach_net(fl_plan* p, fl_net* net) {
  if (!check_plan(p)) return fail(FL_INVALID_ARG, "NULL plan");
  if (!net) {
    p->net = nullptr;
    return FL_OK;
  }
  fl::NetState* ns = fl_net_state(net);
  if (p->g.dphys != 2 || ns->H != p->g.n[0] || ns->W != p->g.n[1])
    return fail(FL_INVALID_ARG, "the network's H x W must equal the 2D plan's n_0 x n_1");
  if (!p->z0) {
    FL_CUDA(dalloc(p, &p->z0, p->g.N * sizeof(float)));
    FL_CUDA(dalloc(p, &p->feat, 3 * p->g.N * sizeof(float)));
    for (int i = 0; i < 3; ++i) FL_CUDA(dalloc(p, &p->lpart[i], kVecBlocks * sizeof(double)));
  }
  p->net = ns;
  return FL_OK;
}

}  // extern "C"
