// Declarations of the persistent batched CG launch (persist.cu,
// persist_body.cu), used by the batched driver (plan.cu).
#pragma once

#include "chain.cuh"

namespace fl {

// --- one persistent launch for the CG iterations of a batch (persist.cu) -----
//
// A phase is one pass of a CG iteration over the batch: one or two items,
// each a set of per-problem argument structs (as in a BatchPass) that the
// phase runs side by side (they touch different problems).  Logical block b
// of a phase belongs to item k when it falls in that item's block range.
struct PItem {
  int kind = 0;              // BK_* (the FP32 CG iteration's passes)
  int nprob = 0;
  int blocks = 0;
  const void* args = nullptr;
  const int* off = nullptr;  // nprob + 1 block offsets
  const int* gx = nullptr;   // per-problem grid x-extent (2D block index)
  const int* map = nullptr;  // per logical block: problem << 20 | block within it
};
constexpr int kPItems = 2;
struct PPhase {
  int nitems = 0;
  int blocks = 0;            // sum of the items' blocks
  PItem item[kPItems];
};
// Grid barrier state (zeroed before the first launch and after a failure).
struct PBarrier {
  unsigned int count;
  unsigned int gen;
  int err;                   // 1: a CTA gave up waiting at a barrier
  int pad;
};
// The persistent kernel's CTA shape: the row passes hold
// row_lines_at(L, kPersistThreads) lines per CTA, the strided passes tiles
// of at most tile_at(., L, kPersistThreads) columns and the tridiagonal
// pass kPersistTriCols columns.
constexpr int kPersistThreads = 256;
constexpr int kPersistTriCols = kPersistThreads / kTriSeg;
// padded lengths the persistent kernel takes: every plan's (2^4 .. 2^11)
constexpr int kPersistLgMin = 4, kPersistLgMax = 11;
// Sets the kernel's shared-memory attributes for `smem` dynamic bytes and
// returns in *grid the co-resident CTA count (blocks per SM x SMs of the
// current device); 0 when the device cannot launch it cooperatively.
cudaError_t persist_configure(size_t smem, int* grid);
// Runs up to max_iters CG iterations (every phase in order, a grid barrier
// after each), stopping after the first iteration at whose end every state
// in states[0..nprob) is done.  Cooperative launch of `grid` CTAs.
cudaError_t launch_persist_cg(const PPhase* phases, int nphases, PcgState* const* states, int nprob,
                              int max_iters, PBarrier* bar, int grid, size_t smem, cudaStream_t s);
// One cooperative launch (one CTA per SM) whose CTAs all arrive at one grid
// barrier that waits for `missing` arrivals more than the grid has;
// *gave_up = 1 when the CTAs gave up waiting (always, for missing > 0,
// after the bounded wait).  Synchronous; on the current device.
cudaError_t persist_barrier_check(int missing, int* gave_up);

}  // namespace fl
