// FP32 row passes in a second CTA shape: 256 threads x 8 values per line
// instead of 128 x 16 (the same lines per CTA, so the same grids, shared
// memory and partial-sum counts), radix-8 stages instead of radix-16.  Half
// the values per thread shortens each CTA's dependent chain, which pays on
// grids of few rows (a pass over 64 rows of 2048 points: 14.5 -> 12.3 us)
// and costs on many (1024 rows: 18.9 -> 27.4 us); fl_plan_autotune times
// both shapes per plan and keeps the faster.  Compiled apart from ops.cu so
// that the two build in parallel.
#include "chain.cuh"

namespace fl {

void launch_rows_fwd_w8(const RowsFwdArgs<float>& a, int grid, size_t smem, cudaStream_t s) {
  pdl_launch(k_rows_fwd<float, kRowsW8Threads, 8>, grid, kRowsW8Threads, smem, s, a);
}

void launch_rows_inv_w8(const RowsInvArgs<float>& a, int grid, size_t smem, cudaStream_t s) {
  pdl_launch(k_rows_inv<float, kRowsW8Threads, 8>, grid, kRowsW8Threads, smem, s, a);
}

void launch_dst_rows_w8(const DstRowsArgs<float>& a, int grid, size_t smem, cudaStream_t s) {
  pdl_launch(k_dst_rows<float, kRowsW8Threads, 8>, grid, kRowsW8Threads, smem, s, a);
}

cudaError_t configure_rows_w8() {
  cudaError_t e = cudaSuccess;
  for (const void* f : {reinterpret_cast<const void*>(&k_rows_fwd<float, kRowsW8Threads, 8>),
                        reinterpret_cast<const void*>(&k_rows_inv<float, kRowsW8Threads, 8>),
                        reinterpret_cast<const void*>(&k_dst_rows<float, kRowsW8Threads, 8>)}) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
  }
  return e;
}

}  // namespace fl
