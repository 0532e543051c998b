// Launch shapes and argument chains shared by the single-problem launchers
// (ops.cu), the batched launchers (batch.cu) and the host drivers (plan.cu).
#pragma once

#include <algorithm>
#include <cstdlib>
#include <utility>

#include "internal.h"
#include "kernels.cuh"

namespace fl {

// Launches the pass kernel k with the programmatic stream-serialization
// attribute (see pdl_wait_then_release), unless FRACLAP_PDL=0 is set in the
// environment.  A launch error is kept and returned by take_launch_error().
bool pdl_enabled();
void note_launch_error(cudaError_t e);
cudaError_t take_launch_error();

template <typename... KArgs, typename... Args>
inline void pdl_launch(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  note_launch_error(cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...));
}

// The first error of this thread's launches since the last call, and of
// the runtime's own last-error slot.
inline cudaError_t launch_status() {
  const cudaError_t e = cudaGetLastError();
  const cudaError_t p = take_launch_error();
  return e != cudaSuccess ? e : p;
}

// Launch shapes.  A CTA keeps VPT * THREADS complex values in shared memory:
// row passes one or two lines of L = 2048 (many small CTAs, up to eight per
// SM, so that a 1024-line pass fills all 152 SMs several times over);
// strided passes a tile of 4 (FP32) or 2 (FP64) columns of L = 2048, i.e. at
// least 32 contiguous bytes per line element.
template <typename T> struct Cfg;
template <> struct Cfg<float> {
  static constexpr int RT = 128, RV = 16;   // rows: threads, values per thread
  static constexpr int CT = 512, CV = 16;   // strided passes
};
template <> struct Cfg<double> {
  static constexpr int RT = 256, RV = 16;
  static constexpr int CT = 256, CV = 16;
};

constexpr int kVecBlocks = 608;   // 4 x 152 SMs, fixed for deterministic partials
constexpr int kVecThreads = 256;
constexpr int kMaxTx = 1 << kMaxLtx;
constexpr int kSmemLimit = 200 * 1024;
constexpr int kMaxLen = 8192;     // longest padded FFT line

// Threads of a row (column) pass on lines of length L: the Cfg shape while a
// CTA of that shape holds at least one line (tile), else one line of L
// values per CTA (FP32 rows: 4096 on 256 and 8192 on 512 threads; FP64 rows
// and columns: 8192 on 512 threads).
template <typename T> inline int row_threads(int L) {
  return L <= Cfg<T>::RT * Cfg<T>::RV ? Cfg<T>::RT : L / Cfg<T>::RV;
}
template <typename T> inline int col_threads(int L) {
  return L <= Cfg<T>::CT * Cfg<T>::CV ? Cfg<T>::CT : L / Cfg<T>::CV;
}
template <typename T> inline int row_lines(int L) { return (row_threads<T>(L) * Cfg<T>::RV) / L; }
// lines per CTA of a row pass whose CTAs have rt threads (rt = 0: the Cfg
// shape) while such a CTA holds at least one line
template <typename T> inline int row_lines_at(int L, int rt) {
  if (rt <= 0) return row_lines<T>(L);
  const int th = L <= rt * Cfg<T>::RV ? rt : L / Cfg<T>::RV;
  return (th * Cfg<T>::RV) / L;
}
template <typename T> inline int col_tx(int L) {
  return std::min(kMaxTx, (col_threads<T>(L) * Cfg<T>::CV) / L);
}
// the narrowest tile the tuner tries: 16 contiguous bytes per line element
template <typename T> inline int min_tx() {
  return std::max(1, 16 / (int)sizeof(typename Cplx<T>::type));
}
// column-tile width of a strided pass along `axis`: the plan's tuned width
// if set, else the widest tile that fits the CTA
template <typename T> inline int plan_tx(const Tables<T>& tb, int axis, int L) {
  return tb.tx[axis] > 0 ? tb.tx[axis] : col_tx<T>(L);
}
// a column-tile width tx narrowed to what a CTA of ct threads holds (ct = 0:
// tx unchanged)
template <typename T> inline int tile_at(int tx, int L, int ct) {
  if (ct <= 0) return tx;
  return std::max(1, std::min(tx, std::min(kMaxTx, (ct * Cfg<T>::CV) / L)));
}
// shared-memory bytes of `lines` lines of L complex values (padded, SBuf)
template <typename T> inline size_t smem_bytes(int lines, int L) {
  return (size_t)sbuf_elems((long long)lines * L) * sizeof(typename Cplx<T>::type);
}
// interleaved tile of tx columns of length L (padded, SBuf)
template <typename T> inline size_t tile_bytes(int tx, int L) {
  return (size_t)sbuf_elems((long long)tx * L) * sizeof(typename Cplx<T>::type);
}
// shared-memory bytes of a strided pass: the FFT tile, then (FP32) the
// line length's twiddle table
template <typename T> inline size_t cols_bytes(int tx, int L) {
  return tile_bytes<T>(tx, L) + (sizeof(T) == 4 ? (size_t)L * sizeof(typename Cplx<T>::type) : 0);
}
// ... and for a convolution pass, then the symbol's rows 0..L/2 for the
// tile's columns
template <typename T> inline size_t conv_tile_bytes(int tx, int L) {
  return cols_bytes<T>(tx, L) + (size_t)(L / 2 + 1) * tx * sizeof(T);
}
inline int ilog2i(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// One operator apply: the row pass, one (2D) or three (3D) strided passes
// and the last row pass, with their launch shapes.
template <typename T>
struct ApplyChain {
  RowsFwdArgs<T> fwd;
  ColsArgs<T> cols[3];
  dim3 cols_grid[3];
  size_t cols_smem[3];
  int ncols;
  RowsInvArgs<T> inv;
  int row_blocks;
  size_t row_smem;
};

// One preconditioner solve: DST rows; in 3D a strided DST pass along the
// middle axis; the tridiagonal solve along axis 0; in 3D the middle-axis DST
// again; DST rows.  The tridiagonal pass runs after the first `tri_after`
// strided passes.
template <typename T>
struct PrecChain {
  DstRowsArgs<T> first;
  DstColsArgs<T> cols[3];
  dim3 cols_grid[3];
  size_t cols_smem[3];
  int ncols;
  TriArgs<T> tri;
  int tri_after;
  int tri_blocks;
  DstRowsArgs<T> last;
  int row_blocks;
  size_t row_smem;
};

// --- batched passes (batch.cu) ----------------------------------------------

// Per-problem arguments of the batched CG vector kernels.
template <typename T>
struct BVecArgs {
  const PcgState* gate;      // nullable: skip the problem when gate->done
  PcgState* st;              // inner CG state
  const T* b;
  T* x;
  T* r;
  T* p;
  const T* q;
  const uint8_t* mask;
  double* part;              // per-CTA partials written by the kernel
  long long N;
};

// CG update without preconditioner (z aliases r): x += alpha p, r -= alpha q
// with alpha from the state (set by the apply's last CTA), partials of
// ||r||^2; the last CTA of the problem takes the CG scalar step.  bx of gx
// CTAs of the problem.
template <typename T>
__device__ __forceinline__ void body_b_noprec(const BVecArgs<T>& a, int bx, int gx) {
  __shared__ double red[32];
  if (a.st->done) return;
  const T al = (T)a.st->alpha;
  DotAcc<T> rr;
  for (long long k = (long long)bx * blockDim.x + threadIdx.x; k < a.N;
       k += (long long)gx * blockDim.x) {
    a.x[k] += al * a.p[k];
    const T rn = a.r[k] - al * a.q[k];
    a.r[k] = rn;
    rr.add(rn * rn);
  }
  const double s = rr.cta_total(red);
  if (threadIdx.x == 0) a.part[bx] = s;
  if (arrive_last(&a.st->arrive, gx)) {
    const double rrv = cta_sum_partials(a.part, gx, red);
    if (threadIdx.x == 0) pcg_step(a.st, rrv, rrv);
  }
}

// Per-problem arguments of the batched scalar kernels (one CTA each).
struct BScalarArgs {
  PcgState* st;
  const PcgState* gate;
  const double* bb_part;
  int bb_count;
  const double* rr_part;
  int rr_count;
  const double* rz_part;
  int rz_count;
  const double* tol;         // device pointer to the problem's tolerance
  int maxit;
};

enum { BK_ROWS_FWD = 0, BK_COLS, BK_ROWS_INV, BK_DST_ROWS, BK_DST_COLS, BK_CG_START, BK_NOPREC,
       BK_CAST, BK_TRI_COLS };

// One batched launch: device arrays of per-problem arguments and of block
// offsets (nprob + 1 entries) and grid x-extents.
struct BatchPass {
  int kind = 0;
  const void* args = nullptr;
  const int* off = nullptr;
  const int* gx = nullptr;
  int nprob = 0;
  int blocks = 0;
  size_t smem = 0;
  int w8 = 0;                // FP32 row passes: the 256 x 8 shape (same grid and memory)
};

template <typename T>
cudaError_t launch_batched(const BatchPass& bp, cudaStream_t s);

cudaError_t launch_cast_rhs(const BatchPass& bp, float* const* out32, cudaStream_t s);
// which: 0 = CG start-up scalars, 2 = sums into out
cudaError_t launch_batched_scalar(int which, const BScalarArgs* args, double* out, int nprob,
                                  cudaStream_t s);
cudaError_t configure_batched_kernels();

// FP32 row passes in the 256 x 8 shape (rows_w8.cu): the same grid and
// shared memory as the Cfg shape
constexpr int kRowsW8Threads = 256;
void launch_rows_fwd_w8(const RowsFwdArgs<float>& a, int grid, size_t smem, cudaStream_t s);
void launch_rows_inv_w8(const RowsInvArgs<float>& a, int grid, size_t smem, cudaStream_t s);
void launch_dst_rows_w8(const DstRowsArgs<float>& a, int grid, size_t smem, cudaStream_t s);
cudaError_t configure_rows_w8();
// whether a plan's FP32 row passes on lines of L points take the 256 x 8 shape
template <typename T> inline bool rows_w8(const Tables<T>& tb, int L) {
  return sizeof(T) == 4 && tb.rshape == 1 && L >= 256 && L <= 2048;
}

template <typename T>
ApplyChain<T> build_apply(const Geo& g, const Tables<T>& tb, const ApplyIO<T>& io);
template <typename T>
PrecChain<T> build_precond(const Geo& g, const Tables<T>& tb, const PrecIO<T>& io);

}  // namespace fl
