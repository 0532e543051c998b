// Pass bodies of the persistent batched CG launch (persist.cu): one logical
// block of one pass kind each, with the same per-problem argument structs
// as the lockstep batched launches (batch.cu).
//
// Compiled as relocatable device code, apart from the kernel that calls
// them: each function is register-allocated on its own (at most 80
// registers: three 256-thread CTAs per SM), which keeps the FFT values in
// registers; compiled into the kernel's own module the same bodies spilled
// kilobytes per thread and took minutes to compile.
#define FL_RESTRICT
#include "persist.h"

namespace fl {

namespace {

constexpr int kPT = kPersistThreads;
constexpr int kPV = Cfg<float>::CV;
// batched plans have padded lengths 2^4 .. 2^11
constexpr int kPLo = kPersistLgMin, kPHi = kPersistLgMax;
static_assert(kPersistTriCols * kTriSeg == kPT, "tridiagonal CTAs of kPT threads");

}  // namespace

// The line length is dispatched to compile-time constants (the bodies'
// index arithmetic folds; the same values as the lockstep kernels' fixed
// shapes).
#define FL_PERSIST_LG_SWITCH(LGV, CALL) \
  switch (LGV) {                        \
    case 4: { constexpr int LG = 4; CALL; } break;   \
    case 5: { constexpr int LG = 5; CALL; } break;   \
    case 6: { constexpr int LG = 6; CALL; } break;   \
    case 7: { constexpr int LG = 7; CALL; } break;   \
    case 8: { constexpr int LG = 8; CALL; } break;   \
    case 9: { constexpr int LG = 9; CALL; } break;   \
    case 10: { constexpr int LG = 10; CALL; } break; \
    case 11: { constexpr int LG = 11; CALL; } break; \
    default: break;                     \
  }
static_assert(kPersistLgMin == 4 && kPHi == 11, "the switch covers 2^4 .. 2^11");

__device__ void persist_rows_fwd(const PItem& it, int i, int l) {
  const RowsFwdArgs<float> a = static_cast<const RowsFwdArgs<float>*>(it.args)[i];
  const int gx = it.gx[i];
  FL_PERSIST_LG_SWITCH(a.lg, (body_rows_fwd_at<float, kPT, kPV, kPLo, kPHi>(a, l % gx, l / gx, LG)))
}
__device__ void persist_cols(const PItem& it, int i, int l) {
  const ColsArgs<float> a = static_cast<const ColsArgs<float>*>(it.args)[i];
  const int gx = it.gx[i];
  const int bx = l % gx, by = l / gx;
  const int w = block_ltx(a.ltx, bx, a.H);
  FL_PERSIST_LG_SWITCH(a.lg, (body_cols_at<float, kPT, kPV, kPLo, kPHi>(a, bx << a.ltx, by, LG, w)))
}
__device__ void persist_rows_inv(const PItem& it, int i, int l) {
  const RowsInvArgs<float> a = static_cast<const RowsInvArgs<float>*>(it.args)[i];
  const int gx = it.gx[i];
  FL_PERSIST_LG_SWITCH(a.lg, (body_rows_inv_at<float, kPT, kPV, kPLo, kPHi>(a, l % gx, l / gx, LG)))
}
__device__ void persist_dst_rows(const PItem& it, int i, int l) {
  const DstRowsArgs<float> a = static_cast<const DstRowsArgs<float>*>(it.args)[i];
  const int gx = it.gx[i];
  FL_PERSIST_LG_SWITCH(a.lg, (body_dst_rows_at<float, kPT, kPV, kPLo, kPHi>(a, l % gx, l / gx, LG)))
}
__device__ void persist_dst_cols(const PItem& it, int i, int l) {
  const DstColsArgs<float> a = static_cast<const DstColsArgs<float>*>(it.args)[i];
  const int gx = it.gx[i];
  const int bx = l % gx, by = l / gx;
  const int w = block_ltx(a.ltx, bx, a.ncols);
  FL_PERSIST_LG_SWITCH(a.lg, (body_dst_cols_at<float, kPT, kPV, kPLo, kPHi>(a, bx << a.ltx, by, LG, w)))
}
__device__ void persist_tri_cols(const PItem& it, int i, int l) {
  const TriArgs<float> a = static_cast<const TriArgs<float>*>(it.args)[i];
  body_tri_cols<float, kPersistTriCols>(a, l);
}
__device__ void persist_noprec(const PItem& it, int i, int l) {
  const BVecArgs<float> a = static_cast<const BVecArgs<float>*>(it.args)[i];
  body_b_noprec<float>(a, l, it.off[i + 1] - it.off[i]);
}

#undef FL_PERSIST_LG_SWITCH

}  // namespace fl
