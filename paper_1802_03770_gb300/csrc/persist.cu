// One launch for all inner CG iterations of a batch of independent problems
// (FP32 PCG of Sec. 3.1 inside the FP64 refinement, many grids at once).
//
// The lockstep batched solve (batch.cu) launches every pass of a CG
// iteration once over all problems.  Here one cooperative grid of
// kPersistThreads-thread CTAs, all resident on the GPU at once, runs those
// passes one after another: in each phase CTA c takes the logical blocks
// c, c + G, c + 2G, ... (G CTAs), each the block that a launch of the
// same shape would have run, then waits at a grid-wide barrier.  After the
// last phase of an iteration every CTA reads the problems' CG states; the
// kernel ends once all of them are done (converged, failed, or at their
// iteration cap), or after max_iters iterations.
//
// Memory ordering: a pass reads what the previous pass of the same launch
// wrote, so the pass bodies are compiled here without __restrict__ (no
// input may be cached as read-only for the whole launch), and each barrier
// is a release (fence, then arrive) and an acquire (fence after the wait)
// at GPU scope.  The bodies' own cross-CTA reads (partial sums, the CG
// state after arrive_last) already bypass L1.
//
// Every wait is bounded: a CTA that has waited kBarrierNs at a barrier sets
// bar->err and returns, and every other CTA returns at its next barrier, so
// the launch always ends; the host reads bar->err and reports a timeout.
#define FL_RESTRICT
#include "persist.h"

namespace fl {

// One logical block of one pass kind (persist_body.cu, compiled separately).
__device__ void persist_rows_fwd(const PItem& it, int i, int l);
__device__ void persist_cols(const PItem& it, int i, int l);
__device__ void persist_rows_inv(const PItem& it, int i, int l);
__device__ void persist_dst_rows(const PItem& it, int i, int l);
__device__ void persist_dst_cols(const PItem& it, int i, int l);
__device__ void persist_tri_cols(const PItem& it, int i, int l);
__device__ void persist_noprec(const PItem& it, int i, int l);

namespace {

constexpr int kPT = kPersistThreads;
constexpr unsigned long long kBarrierNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier (sense by generation): thread 0 reads the generation,
// arrives on the counter; the last arrival resets the counter and advances
// the generation, the others wait for it to change (bounded).  Returns
// false, to every thread of the CTA, when this CTA gave up or another CTA
// has recorded a failure.
__device__ bool grid_barrier(PBarrier* bar, unsigned int nctas) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int g = ld_acquire_u32(&bar->gen);
    __threadfence();
    if (atomicAdd(&bar->count, 1u) == nctas - 1u) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_u32(&bar->gen) == g) {
        if (*(volatile int*)&bar->err) { ok = 0; break; }
        if (global_ns() - t0 > kBarrierNs) {
          atomicExch(&bar->err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (ok && *(volatile int*)&bar->err) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ void run_block(const PItem& it, int b) {
  const int m = it.map[b];
  const int i = m >> 20, l = m & ((1 << 20) - 1);
  switch (it.kind) {
    case BK_ROWS_FWD: persist_rows_fwd(it, i, l); break;
    case BK_COLS: persist_cols(it, i, l); break;
    case BK_ROWS_INV: persist_rows_inv(it, i, l); break;
    case BK_DST_ROWS: persist_dst_rows(it, i, l); break;
    case BK_DST_COLS: persist_dst_cols(it, i, l); break;
    case BK_TRI_COLS: persist_tri_cols(it, i, l); break;
    case BK_NOPREC: persist_noprec(it, i, l); break;
    default: break;
  }
}

__global__ void __launch_bounds__(kPT, 1)
    k_persist_cg(const PPhase* __restrict__ phases, int nphases, PcgState* const* __restrict__ states,
                 int nprob, int max_iters, PBarrier* bar) {
  __shared__ int s_more;
  const unsigned int G = gridDim.x;
  for (int iter = 0; iter < max_iters; ++iter) {
    for (int ph = 0; ph < nphases; ++ph) {
      const PPhase& P = phases[ph];
      const int total = P.blocks;
      if (total == 0) continue;
      for (int b = blockIdx.x; b < total; b += (int)G) {
        __syncthreads();   // the previous block's shared-memory reads are done
        int k = 0, bb = b;
        while (k + 1 < P.nitems && bb >= P.item[k].blocks) {
          bb -= P.item[k].blocks;
          ++k;
        }
        run_block(P.item[k], bb);
      }
      if (!grid_barrier(bar, G)) return;
    }
    // Between this barrier and the next iteration's pass that can finish a
    // problem (the apply's last pass) no CTA writes a state's done flag, so
    // every CTA takes the same decision.
    if (threadIdx.x == 0) {
      int more = 0;
      for (int i = 0; i < nprob && !more; ++i) more = __ldcg(&states[i]->done) == 0;
      s_more = more;
    }
    __syncthreads();
    if (!s_more) break;
  }
}

// Diagnostic: every CTA of the grid arrives at one grid barrier that waits
// for gridDim.x + extra arrivals.
__global__ void k_barrier_check(PBarrier* bar, unsigned int extra) {
  grid_barrier(bar, gridDim.x + extra);
}

}  // namespace

cudaError_t persist_barrier_check(int missing, int* gave_up) {
  *gave_up = 0;
  int dev = 0, sms = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e != cudaSuccess) return e;
  if (!coop) return cudaErrorNotSupported;
  PBarrier* bar = nullptr;
  e = cudaMalloc(&bar, sizeof(PBarrier));
  if (e != cudaSuccess) return e;
  e = cudaMemset(bar, 0, sizeof(PBarrier));
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sms);
    cfg.blockDim = dim3(kPT);
    cfg.stream = nullptr;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    FL_KERNEL("barrier_check", nullptr,
              e = cudaLaunchKernelEx(&cfg, k_barrier_check, bar, (unsigned int)missing));
  }
  PBarrier h = {};
  if (e == cudaSuccess) e = cudaMemcpy(&h, bar, sizeof(PBarrier), cudaMemcpyDeviceToHost);
  cudaFree(bar);
  if (e == cudaSuccess) *gave_up = h.err;
  return e;
}

cudaError_t persist_configure(size_t smem, int* grid) {
  *grid = 0;
  int dev = 0, coop = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_persist_cg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_persist_cg, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist_cg, kPT, smem);
  if (e == cudaSuccess && coop) *grid = per_sm * sms;
  return e;
}

cudaError_t launch_persist_cg(const PPhase* phases, int nphases, PcgState* const* states, int nprob,
                              int max_iters, PBarrier* bar, int grid, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kPT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaSuccess;
  FL_KERNEL("persist_cg<f32>", s,
            e = cudaLaunchKernelEx(&cfg, k_persist_cg, phases, nphases, states, nprob, max_iters, bar));
  return e;
}

}  // namespace fl
