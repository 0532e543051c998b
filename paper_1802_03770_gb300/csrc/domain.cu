// The paper's preconditioner on an occluded domain Omega (Sec. 4.4): the
// finite-difference operator B_Omega = shift I + scale C h^d L restricted to
// the points of Omega, with Dirichlet conditions on every point of the box
// outside it.  The paper factorises B_Omega by sparse Cholesky; here it is
// applied exactly through the box operator B (the fast DST/tridiagonal solve
// of the full box) and a small dense system on the hole's boundary
// (capacitance matrix method, Buzbee, Dorr, George & Golub, SIAM J. Numer.
// Anal. 8, 1971):
//
//   Gamma = the points outside Omega with a grid neighbour in Omega,
//   E     = injection of Gamma into the box, C = E^T B^{-1} E (SPD),
//   w     = B^{-1} r~ (r~ = r on Omega, 0 elsewhere),
//   s     = -C^{-1} E^T w,
//   z     = R (w + B^{-1} E s).
//
// z~ = w + B^{-1} E s satisfies B z~ = r~ + E s and vanishes on Gamma; on
// the rest of the hole it solves the homogeneous equation with zero data on
// Gamma and the box boundary, so it vanishes there too.  On Omega,
// B z~ = r~ with z~ = 0 at every neighbour outside Omega: B_Omega z = r.
//
// C is formed once per (shift, scale) from |Gamma| FP64 box solves of unit
// vectors, factorised as L D L^T (right-looking, one launch per pivot), and
// each application solves with the factor in one CTA (FP64, for either
// precision of the box solves).
#include "chain.cuh"
#include "domain.h"

namespace fl {

namespace {

constexpr int kDomThreads = 1024;

// e = unit vector at Gamma point `cur` (and the previous one cleared).
__global__ void k_dom_unit(double* e, const int* __restrict__ idx, int prev, int cur) {
  if (threadIdx.x == 0) {
    if (prev >= 0) e[idx[prev]] = 0.0;
    e[idx[cur]] = 1.0;
  }
}

// Column `col` of C: C[b][col] = z[Gamma_b].
__global__ void k_dom_gather(const double* __restrict__ z, const int* __restrict__ idx, int m,
                             double* __restrict__ C, int col) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < m) C[(size_t)b * m + col] = z[idx[b]];
}

// C = (C + C^T) / 2 (the box solves are symmetric up to rounding).
__global__ void k_dom_symmetrize(double* C, int m) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m && j < i) {
    const double v = 0.5 * (C[(size_t)i * m + j] + C[(size_t)j * m + i]);
    C[(size_t)i * m + j] = v;
    C[(size_t)j * m + i] = v;
  }
}

// Pivot k of the right-looking L D L^T factorisation (lower triangle):
// A_ij -= A_ik A_jk / A_kk for k < j <= i.
__global__ void k_dom_ldl_step(double* C, int m, int k) {
  const int i = k + 1 + blockIdx.y * blockDim.y + threadIdx.y;
  const int j = k + 1 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m && j <= i) {
    const double piv = C[(size_t)k * m + k];
    C[(size_t)i * m + j] -= C[(size_t)i * m + k] * C[(size_t)j * m + k] / piv;
  }
}

// After the last pivot: L'_ik = A_ik / A_kk below the diagonal (unit lower
// factor), D_k = A_kk on it.
__global__ void k_dom_ldl_scale(double* C, int m) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m && k < i) C[(size_t)i * m + k] /= C[(size_t)k * m + k];
}

// s = -C^{-1} w_Gamma with C = L' D L'^T, scattered to us at Gamma (us is
// zero elsewhere and stays so).  One CTA; the triangular solves run in
// blocks of 32 unknowns: warp 0 solves the block (shuffles), then every
// thread updates the unknowns after (forward) or before (backward) it.
template <typename T>
__global__ void __launch_bounds__(kDomThreads) k_dom_solve(const T* __restrict__ w,
                                                           const int* __restrict__ idx,
                                                           const double* __restrict__ LD, int m,
                                                           T* __restrict__ us, const PcgState* st) {
  extern __shared__ double b[];   // m values
  if (st && st->done) return;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int a = tid; a < m; a += kDomThreads) b[a] = -(double)w[idx[a]];
  __syncthreads();
  // forward: L' y = b
  for (int kb = 0; kb < m; kb += 32) {
    const int nb = min(32, m - kb);
    if (tid < 32) {
      double v = lane < nb ? b[kb + lane] : 0.0;
      for (int t = 0; t < nb; ++t) {
        const double y = __shfl_sync(0xffffffffu, v, t);
        if (lane > t && lane < nb) v -= LD[(size_t)(kb + lane) * m + kb + t] * y;
      }
      if (lane < nb) b[kb + lane] = v;
    }
    __syncthreads();
    for (int i = kb + nb + tid; i < m; i += kDomThreads) {
      const double* row = LD + (size_t)i * m + kb;
      double acc = 0.0;
      for (int t = 0; t < nb; ++t) acc += row[t] * b[kb + t];
      b[i] -= acc;
    }
    __syncthreads();
  }
  for (int a = tid; a < m; a += kDomThreads) b[a] /= LD[(size_t)a * m + a];
  __syncthreads();
  // backward: L'^T x = y
  for (int kb = ((m - 1) / 32) * 32; kb >= 0; kb -= 32) {
    const int nb = min(32, m - kb);
    if (tid < 32) {
      double v = lane < nb ? b[kb + lane] : 0.0;
      for (int t = nb - 1; t >= 0; --t) {
        const double x = __shfl_sync(0xffffffffu, v, t);
        if (lane < t) v -= LD[(size_t)(kb + t) * m + kb + lane] * x;
      }
      if (lane < nb) b[kb + lane] = v;
    }
    __syncthreads();
    for (int i = tid; i < kb; i += kDomThreads) {
      double acc = 0.0;
      for (int t = 0; t < nb; ++t) acc += LD[(size_t)(kb + t) * m + i] * b[kb + t];
      b[i] -= acc;
    }
    __syncthreads();
  }
  for (int a = tid; a < m; a += kDomThreads) us[idx[a]] = (T)b[a];
}

}  // namespace

cudaError_t dom_build_capacitance(const Geo& g, const Tables<double>& tb, const DomainData& dd,
                                  double shift, double scale, double* e, double* z, cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(e, 0, g.N * sizeof(double), s);
  for (int a = 0; a < dd.m && err == cudaSuccess; ++a) {
    FL_KERNEL("dom_unit", s, k_dom_unit<<<1, 32, 0, s>>>(e, dd.idx, a - 1, a));
    PrecIO<double> io;
    io.in = e; io.out = z; io.shift = shift; io.scale = scale;   // the box operator: no mask
    err = launch_precond<double>(g, tb, s, io);
    if (err == cudaSuccess) {
      FL_KERNEL("dom_gather", s, k_dom_gather<<<(dd.m + 255) / 256, 256, 0, s>>>(z, dd.idx, dd.m, dd.LD, a));
      err = cudaGetLastError();
    }
  }
  if (err != cudaSuccess) return err;
  const dim3 blk(16, 16);
  const dim3 grid((dd.m + 15) / 16, (dd.m + 15) / 16);
  FL_KERNEL("dom_symmetrize", s, k_dom_symmetrize<<<grid, blk, 0, s>>>(dd.LD, dd.m));
  for (int k = 0; k + 1 < dd.m; ++k) {
    const int r = dd.m - k - 1;
    const dim3 gk((r + 15) / 16, (r + 15) / 16);
    FL_KERNEL("dom_ldl_step", s, k_dom_ldl_step<<<gk, blk, 0, s>>>(dd.LD, dd.m, k));
  }
  FL_KERNEL("dom_ldl_scale", s, k_dom_ldl_scale<<<grid, blk, 0, s>>>(dd.LD, dd.m));
  return cudaGetLastError();
}

template <typename T>
cudaError_t dom_interface_solve(const DomainData& dd, const T* w, T* us, const PcgState* st,
                                cudaStream_t s) {
  FL_KERNEL(sizeof(T) == 4 ? "dom_solve<f32>" : "dom_solve<f64>", s,
            k_dom_solve<T><<<1, kDomThreads, dd.m * sizeof(double), s>>>(w, dd.idx, dd.LD, dd.m, us, st));
  return cudaGetLastError();
}

cudaError_t configure_domain_kernels() {
  cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_dom_solve<float>),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kMaxGamma * (int)sizeof(double));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_dom_solve<double>),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxGamma * (int)sizeof(double));
  return e;
}

template cudaError_t dom_interface_solve<float>(const DomainData&, const float*, float*, const PcgState*,
                                                cudaStream_t);
template cudaError_t dom_interface_solve<double>(const DomainData&, const double*, double*,
                                                 const PcgState*, cudaStream_t);

}  // namespace fl
