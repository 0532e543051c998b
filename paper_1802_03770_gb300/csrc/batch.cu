// Batched launches: one grid runs one pass for many independent problems of
// different sizes.  CTA b belongs to problem i with off[i] <= b < off[i+1];
// its local index l = b - off[i] is split as (l mod gx[i], l div gx[i]) into
// the (x, y) block index the single-problem kernel would have had.  The
// per-problem argument structs live in device memory and are the same the
// single-problem launchers build, so a batched pass computes exactly what
// the single launches compute.
#include "chain.cuh"

namespace fl {

__device__ __forceinline__ int batch_problem(const int* __restrict__ off, int nprob) {
  __shared__ int s_i;
  if (threadIdx.x == 0) {
    int lo = 0, hi = nprob - 1;
    const int b = blockIdx.x;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= b) lo = mid;
      else hi = mid - 1;
    }
    s_i = lo;
  }
  __syncthreads();
  return s_i;
}

#define FL_BATCHED_KERNEL(NAME, ARGS)                                                          \
  template <typename T, int THREADS, int VPT>                                                  \
  __global__ void __launch_bounds__(THREADS, min_ctas(THREADS))                               \
      kb_##NAME(const ARGS<T>* __restrict__ args, const int* __restrict__ off,                 \
                const int* __restrict__ gx, int nprob) {                                       \
    pdl_wait();                                                                                \
    const int i = batch_problem(off, nprob);                                                   \
    const ARGS<T> a = args[i];                                                                 \
    const int l = blockIdx.x - off[i];                                                         \
    body_##NAME<T, THREADS, VPT>(a, l % gx[i], l / gx[i]);                                     \
    pdl_release();                                                                             \
  }

FL_BATCHED_KERNEL(rows_fwd, RowsFwdArgs)
FL_BATCHED_KERNEL(cols, ColsArgs)
FL_BATCHED_KERNEL(rows_inv, RowsInvArgs)
FL_BATCHED_KERNEL(dst_rows, DstRowsArgs)
FL_BATCHED_KERNEL(dst_cols, DstColsArgs)

#undef FL_BATCHED_KERNEL

template <typename T>
__global__ void __launch_bounds__(kTriCols * kTriSeg)
    kb_tri_cols(const TriArgs<T>* __restrict__ args, const int* __restrict__ off, int nprob) {
  pdl_wait();
  const int i = batch_problem(off, nprob);
  const TriArgs<T> a = args[i];
  body_tri_cols<T>(a, blockIdx.x - off[i]);
  pdl_release();
}

// --- batched CG vector and scalar kernels -------------------------------------

// Start of an inner CG solve with x0 = 0: x = 0, p = 0, r = b (masked), and
// per-CTA partials of ||b||^2; inactive problems (st->done) do nothing.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) kb_cg_start(const BVecArgs<T>* __restrict__ args,
                                                          const int* __restrict__ off, int nprob) {
  __shared__ double red[32];
  pdl_wait();
  const int i = batch_problem(off, nprob);
  const BVecArgs<T> a = args[i];
  const int bx = blockIdx.x - off[i];
  const int gx = off[i + 1] - off[i];
  if (a.gate && a.gate->done) return;
  DotAcc<T> v;
  for (long long k = (long long)bx * blockDim.x + threadIdx.x; k < a.N;
       k += (long long)gx * blockDim.x) {
    const T bv = (a.mask && !a.mask[k]) ? (T)0 : a.b[k];
    a.r[k] = bv;
    a.x[k] = (T)0;
    a.p[k] = (T)0;
    v.add(bv * bv);
  }
  const double s = v.cta_total(red);
  if (threadIdx.x == 0) a.part[bx] = s;
}

template <typename T>
__global__ void __launch_bounds__(kVecThreads) kb_noprec_update(const BVecArgs<T>* __restrict__ args,
                                                               const int* __restrict__ off, int nprob) {
  pdl_wait();
  const int i = batch_problem(off, nprob);
  body_b_noprec<T>(args[i], blockIdx.x - off[i], off[i + 1] - off[i]);
}

// This file is compiled in two halves (FL_BATCH_PART 1: the FP32 passes and
// the precision-free kernels, 2: the FP64 passes) so that its template
// instantiations compile in parallel; without FL_BATCH_PART it holds both.
#if !defined(FL_BATCH_PART) || FL_BATCH_PART == 1
// FP64 right-hand side to the FP32 inner right-hand side (masked), with
// partials of ||b||^2 -- the residual of the zero initial guess.
__global__ void __launch_bounds__(kVecThreads) kb_cast_rhs(const BVecArgs<double>* __restrict__ args,
                                                          float* const* __restrict__ out32,
                                                          const int* __restrict__ off, int nprob) {
  __shared__ double red[32];
  const int i = batch_problem(off, nprob);
  const BVecArgs<double> a = args[i];
  float* o = out32[i];
  const int bx = blockIdx.x - off[i];
  const int gx = off[i + 1] - off[i];
  double v = 0.0;
  for (long long k = (long long)bx * blockDim.x + threadIdx.x; k < a.N;
       k += (long long)gx * blockDim.x) {
    const double bv = (a.mask && !a.mask[k]) ? 0.0 : a.b[k];
    o[k] = (float)bv;
    a.x[k] = 0.0;
    v += bv * bv;
  }
  const double s = cta_sum(v, red);
  if (threadIdx.x == 0) a.part[bx] = s;
}

// One CTA per problem: CG start-up scalars (as k_pcg_init).  Problems whose
// gate is done start done.
__global__ void kb_pcg_init(const BScalarArgs* __restrict__ args, int nprob) {
  __shared__ double red[32];
  const BScalarArgs a = args[blockIdx.x];
  const double bb = cta_sum_partials(a.bb_part, a.bb_count, red);
  const double rz = cta_sum_partials(a.rz_part, a.rz_count, red);
  if (threadIdx.x == 0) {
    PcgState* st = a.st;
    st->bb = bb;
    st->rr = bb;
    st->rz = rz;
    st->tol2 = a.tol[0] * a.tol[0] * bb;
    st->beta = 0.0;
    st->alpha = 0.0;
    st->pq = 0.0;
    st->it = 0;
    st->maxit = a.maxit;
    st->status = 0;
    st->arrive = 0u;
    st->done = (bb == 0.0 || (a.gate && a.gate->done)) ? 1 : 0;
    if (!(rz > 0.0) && !st->done) { st->done = 1; st->status = 3; }
  }
}

// One CTA per problem: sum of partials into out[i] (skips done gates).
__global__ void kb_sum(const BScalarArgs* __restrict__ args, double* out, int nprob) {
  __shared__ double red[32];
  const BScalarArgs a = args[blockIdx.x];
  if (a.gate && a.gate->done) return;
  const double s = cta_sum_partials(a.rr_part, a.rr_count, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

#endif

// --- launchers --------------------------------------------------------------

template <typename T>
cudaError_t launch_batched(const BatchPass& bp, cudaStream_t s) {
  typedef Cfg<T> K;
  if (bp.nprob == 0 || bp.blocks == 0) return cudaSuccess;
  switch (bp.kind) {
    case BK_ROWS_FWD:
      if constexpr (sizeof(T) == 4) {
        if (bp.w8) {
          FL_KERNEL("b_rows_fwd<f32>", s,
                    pdl_launch(kb_rows_fwd<T, kRowsW8Threads, 8>, bp.blocks, kRowsW8Threads, bp.smem, s,
                               (const RowsFwdArgs<T>*)bp.args, bp.off, bp.gx, bp.nprob));
          break;
        }
      }
      FL_KERNEL(sizeof(T) == 4 ? "b_rows_fwd<f32>" : "b_rows_fwd<f64>", s,
                pdl_launch(kb_rows_fwd<T, K::RT, K::RV>, bp.blocks, K::RT, bp.smem, s,
                           (const RowsFwdArgs<T>*)bp.args, bp.off, bp.gx, bp.nprob));
      break;
    case BK_COLS:
      FL_KERNEL(sizeof(T) == 4 ? "b_cols<f32>" : "b_cols<f64>", s,
                pdl_launch(kb_cols<T, K::CT, K::CV>, bp.blocks, K::CT, bp.smem, s,
                           (const ColsArgs<T>*)bp.args, bp.off, bp.gx, bp.nprob));
      break;
    case BK_ROWS_INV:
      if constexpr (sizeof(T) == 4) {
        if (bp.w8) {
          FL_KERNEL("b_rows_inv<f32>", s,
                    pdl_launch(kb_rows_inv<T, kRowsW8Threads, 8>, bp.blocks, kRowsW8Threads, bp.smem, s,
                               (const RowsInvArgs<T>*)bp.args, bp.off, bp.gx, bp.nprob));
          break;
        }
      }
      FL_KERNEL(sizeof(T) == 4 ? "b_rows_inv<f32>" : "b_rows_inv<f64>", s,
                pdl_launch(kb_rows_inv<T, K::RT, K::RV>, bp.blocks, K::RT, bp.smem, s,
                           (const RowsInvArgs<T>*)bp.args, bp.off, bp.gx, bp.nprob));
      break;
    case BK_DST_ROWS:
      if constexpr (sizeof(T) == 4) {
        if (bp.w8) {
          FL_KERNEL("b_dst_rows<f32>", s,
                    pdl_launch(kb_dst_rows<T, kRowsW8Threads, 8>, bp.blocks, kRowsW8Threads, bp.smem, s,
                               (const DstRowsArgs<T>*)bp.args, bp.off, bp.gx, bp.nprob));
          break;
        }
      }
      FL_KERNEL(sizeof(T) == 4 ? "b_dst_rows<f32>" : "b_dst_rows<f64>", s,
                pdl_launch(kb_dst_rows<T, K::RT, K::RV>, bp.blocks, K::RT, bp.smem, s,
                           (const DstRowsArgs<T>*)bp.args, bp.off, bp.gx, bp.nprob));
      break;
    case BK_DST_COLS:
      FL_KERNEL(sizeof(T) == 4 ? "b_dst_cols<f32>" : "b_dst_cols<f64>", s,
                pdl_launch(kb_dst_cols<T, K::CT, K::CV>, bp.blocks, K::CT, bp.smem, s,
                           (const DstColsArgs<T>*)bp.args, bp.off, bp.gx, bp.nprob));
      break;
    case BK_TRI_COLS:
      FL_KERNEL(sizeof(T) == 4 ? "b_tri_cols<f32>" : "b_tri_cols<f64>", s,
                pdl_launch(kb_tri_cols<T>, bp.blocks, kTriCols * kTriSeg, 0, s,
                           (const TriArgs<T>*)bp.args, bp.off, bp.nprob));
      break;
    case BK_CG_START:
      FL_KERNEL(sizeof(T) == 4 ? "b_cg_start<f32>" : "b_cg_start<f64>", s,
                pdl_launch(kb_cg_start<T>, bp.blocks, kVecThreads, 0, s,
                           (const BVecArgs<T>*)bp.args, bp.off,
                           bp.nprob));
      break;
    case BK_NOPREC:
      FL_KERNEL(sizeof(T) == 4 ? "b_noprec_update<f32>" : "b_noprec_update<f64>", s,
                pdl_launch(kb_noprec_update<T>, bp.blocks, kVecThreads, 0, s,
                           (const BVecArgs<T>*)bp.args, bp.off,
                           bp.nprob));
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return launch_status();
}

#if !defined(FL_BATCH_PART) || FL_BATCH_PART == 1
cudaError_t launch_cast_rhs(const BatchPass& bp, float* const* out32, cudaStream_t s) {
  if (bp.nprob == 0) return cudaSuccess;
  FL_KERNEL("b_cast_rhs", s,
            kb_cast_rhs<<<bp.blocks, kVecThreads, 0, s>>>((const BVecArgs<double>*)bp.args, out32,
                                                           bp.off, bp.nprob));
  return cudaGetLastError();
}

cudaError_t launch_batched_scalar(int which, const BScalarArgs* args, double* out, int nprob,
                                  cudaStream_t s) {
  if (nprob == 0) return cudaSuccess;
  if (which == 0)
    FL_KERNEL("b_pcg_init", s, kb_pcg_init<<<nprob, 256, 0, s>>>(args, nprob));
  else
    FL_KERNEL("b_sum", s, kb_sum<<<nprob, 256, 0, s>>>(args, out, nprob));
  return cudaGetLastError();
}

#endif

static cudaError_t set_batched_smem(const void* f) {
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  return e;
}

cudaError_t configure_batched_kernels_f64();

#if !defined(FL_BATCH_PART) || FL_BATCH_PART == 1
cudaError_t configure_batched_kernels() {
  cudaError_t e = configure_batched_kernels_f64();
  for (const void* f : {reinterpret_cast<const void*>(&kb_rows_fwd<float, Cfg<float>::RT, Cfg<float>::RV>),
                        reinterpret_cast<const void*>(&kb_rows_inv<float, Cfg<float>::RT, Cfg<float>::RV>),
                        reinterpret_cast<const void*>(&kb_cols<float, Cfg<float>::CT, Cfg<float>::CV>),
                        reinterpret_cast<const void*>(&kb_dst_rows<float, Cfg<float>::RT, Cfg<float>::RV>),
                        reinterpret_cast<const void*>(&kb_dst_cols<float, Cfg<float>::CT, Cfg<float>::CV>),
                        reinterpret_cast<const void*>(&kb_rows_fwd<float, kRowsW8Threads, 8>),
                        reinterpret_cast<const void*>(&kb_rows_inv<float, kRowsW8Threads, 8>),
                        reinterpret_cast<const void*>(&kb_dst_rows<float, kRowsW8Threads, 8>)})
    if (e == cudaSuccess) e = set_batched_smem(f);
  return e;
}

template cudaError_t launch_batched<float>(const BatchPass&, cudaStream_t);
#endif

#if !defined(FL_BATCH_PART) || FL_BATCH_PART == 2
cudaError_t configure_batched_kernels_f64() {
  cudaError_t e = cudaSuccess;
  for (const void* f : {reinterpret_cast<const void*>(&kb_rows_fwd<double, Cfg<double>::RT, Cfg<double>::RV>),
                        reinterpret_cast<const void*>(&kb_rows_inv<double, Cfg<double>::RT, Cfg<double>::RV>),
                        reinterpret_cast<const void*>(&kb_cols<double, Cfg<double>::CT, Cfg<double>::CV>)})
    if (e == cudaSuccess) e = set_batched_smem(f);
  return e;
}

template cudaError_t launch_batched<double>(const BatchPass&, cudaStream_t);
#endif

}  // namespace fl
