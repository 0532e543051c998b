// Internal interfaces between the host plan code (plan.cu), the kernel
// launchers (ops.cu) and the host constants (consts.cpp).
#pragma once

#include <complex>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace fl {

// --- consts.cpp ------------------------------------------------------------
double c_alpha_d(double alpha, int d);
double upper_gamma(double a, double x);
double lattice_zeta(int d, double alpha);
double window_corr(int d, double alpha, double rho);
void host_fft(std::vector<std::complex<long double>>& a);

// --- geometry of a plan ------------------------------------------------------
struct Geo {
  int d;          // layout dimension (2 or 3); a 1D problem is one row of a 2D layout
  int dphys;      // dimension of the problem: 1, 2 or 3
  int n[3];
  int L[3];
  int lg[3];
  int lgmax;
  int H;          // L[d-1]/2 + 1
  long long N;    // prod n
  long long spec; // complex entries of the operator spectrum workspace
  double cA;      // c (-a): weight of the finite-difference stencil in C h^d L
};

struct PcgState;

// Device tables and workspaces of one precision.
template <typename T>
struct Tables {
  typedef typename std::conditional<sizeof(T) == 4, float2, double2>::type C;
  C* tw = nullptr;            // exp(-2 pi i k / Lmax)
  T* sig = nullptr;           // kernel symbol / prod L
  C* chirp[3] = {nullptr, nullptr, nullptr};
  C* bhat[3] = {nullptr, nullptr, nullptr};
  C* S = nullptr;             // operator spectrum workspace
  T* t = nullptr;             // preconditioner workspace (N)
  T* mu[3] = {nullptr, nullptr, nullptr};  // eigenvalues of C h^d L per axis
  T* tri_tab = nullptr;       // per-column constants of the axis-0 tridiagonal solve
  double tri_shift = -1.0, tri_scale = -1.0;  // the shift and scale tri_tab holds
  int tx[3] = {0, 0, 0};      // column-tile width of the strided passes per axis (0: default)
  int rshape = 0;             // FP32 row passes: 0 = 128 threads x 16 values per line,
                              // 1 = 256 x 8 (lines of 256 .. 2048 points; rows_w8.cu)
};

// Inputs and outputs of one operator apply.
template <typename T>
struct ApplyIO {
  int pre = 0;                // PRE_NONE / PRE_PUPDATE / PRE_ACCUM
  const T* u = nullptr;       // PRE_NONE: input; PRE_PUPDATE: z
  T* p = nullptr;             // PRE_PUPDATE
  double* acc = nullptr;      // PRE_ACCUM
  const float* x32 = nullptr; // PRE_ACCUM
  const uint8_t* mask = nullptr;
  PcgState* st = nullptr;
  // epilogue: out = cm M x + cx x + cb b
  T* out = nullptr;
  float* out32 = nullptr;
  const T* x = nullptr;
  const T* b = nullptr;
  double cm = 1.0, cx = 0.0, cb = 0.0;
  const T* dotw = nullptr;
  double* partials = nullptr;
  int dot_self = 0;
  int fin = 0;                // FIN_PQ: the last CTA sets st->pq and st->alpha
  T* outm = nullptr;          // nullable: M x (the apply itself) as well
  int row_threads = 0;        // threads of a row-pass CTA; 0: the default shape
  int col_threads = 0;        // threads of a strided-pass CTA; 0: the default shape
};

// Inputs and outputs of one preconditioner solve.
template <typename T>
struct PrecIO {
  int pre = 0;                // DPRE_NONE / DPRE_UPDATE
  const T* in = nullptr;
  T* out = nullptr;
  double shift = 0.0, scale = 1.0;
  T* x = nullptr; T* r = nullptr; const T* p = nullptr; const T* q = nullptr;
  double* rr_part = nullptr;
  const T* dotw = nullptr; double* dot_part = nullptr;
  PcgState* st = nullptr;
  int fin = 0;                // FIN_STEP: the last pass ends with the CG scalar step
  const uint8_t* mask = nullptr;  // occluded domain: restrict input and output to Omega
  bool input_unmasked = false;    // keep the input outside Omega (mask applies to the output only)
  bool keep_outside = false;      // keep the output outside Omega (mask applies to the input only)
  const T* add = nullptr;         // nullable: out = mask ? (B^{-1} in + add) : 0
  int row_threads = 0;            // threads of a row-pass CTA; 0: the default shape
  int col_threads = 0;            // threads of a strided-pass CTA; 0: the default shape
  int tri_cols = 0;               // columns per tridiagonal-pass CTA; 0: kTriCols
};

// --- ops.cu: launchers (return the first CUDA error) --------------------------
template <typename T>
cudaError_t launch_apply(const Geo& g, const Tables<T>& tb, cudaStream_t s, const ApplyIO<T>& io);
template <typename T>
int apply_partials(const Geo& g);  // partials written by the apply epilogue
template <typename T>
cudaError_t launch_precond(const Geo& g, const Tables<T>& tb, cudaStream_t s, const PrecIO<T>& io);
template <typename T>
int precond_partials(const Geo& g);  // partials of the first / last DST pass
// Fill tb.tri_tab for (shift, scale) unless it already holds them.
template <typename T>
cudaError_t prepare_precond(const Geo& g, Tables<T>& tb, double shift, double scale, cudaStream_t s);
template <typename T>
cudaError_t launch_noprec_update(long long N, cudaStream_t s, PcgState* st, T* x, T* r,
                                 const T* p, const T* q, double* rr_part, int step, int* count);
template <typename T>
cudaError_t launch_dot(long long N, cudaStream_t s, const T* a, const T* b, double* part,
                       int* count);
template <typename T>
cudaError_t launch_copy_cast(long long N, cudaStream_t s, const double* src, T* dst);
template <typename T>
cudaError_t launch_axpby(long long N, cudaStream_t s, double a, const T* x, double b, T* y);
template <typename T>
cudaError_t launch_mask_copy_dot(long long N, cudaStream_t s, const T* src, const uint8_t* mask, T* dst,
                                 double* part, int* count);
cudaError_t launch_pcg_init(cudaStream_t s, PcgState* st, const double* bb_part, int bb_count,
                            const double* rr_part, int rr_count, const double* rz_part, int rz_count,
                            double tol, int maxit);
cudaError_t launch_sum(cudaStream_t s, const double* part, int count, double* out);
// v = the lowest (hi = 0) or highest (hi = 1) separable DST-I mode, 0 off the mask
cudaError_t launch_sine_mode(const Geo& g, cudaStream_t s, double* v, const uint8_t* mask, int hi);
// r = b - shift u - scale mx (masked) from a known mx = M u: FP64 r is not
// kept; r32 = (float) r and per-CTA partials of ||r||^2 are written.
cudaError_t launch_residual_from(long long N, cudaStream_t s, const double* b, const double* u,
                                 const double* mx, const uint8_t* mask, double shift, double scale,
                                 float* r32, double* part, int* count);
// y = u - c mx (b of a theta step from a known mx = M u)
cudaError_t launch_axmy(long long N, cudaStream_t s, const double* u, double c, const double* mx,
                        double* y);
// order-independent 64-bit hash of the bits of N doubles, added into *h (zero it first)
cudaError_t launch_hash(long long N, cudaStream_t s, const double* u, unsigned long long* h);
cudaError_t build_symbol(const Geo& g, double c, double Z, double a, double expo, cudaStream_t s,
                         double* sig64, float* sig32, const double2* tw64);
size_t partial_capacity(const Geo& g);

// --- launch accounting (plan.cu) ----------------------------------------------
// Every kernel launch of the library goes through FL_KERNEL: it counts the
// launch and, while a profiler is active on this thread, brackets it with
// CUDA events on its stream.
void note_launch();
bool prof_active();
cudaEvent_t prof_begin(cudaStream_t s);
void prof_end(const char* name, cudaEvent_t e0, cudaStream_t s);

#define FL_KERNEL(name, stream, ...)                                  \
  do {                                                                \
    ::fl::note_launch();                                              \
    cudaEvent_t fl_e0_ = ::fl::prof_active() ? ::fl::prof_begin(stream) : nullptr; \
    __VA_ARGS__;                                                      \
    if (fl_e0_) ::fl::prof_end(name, fl_e0_, stream);                 \
  } while (0)
cudaError_t configure_kernels();

}  // namespace fl
