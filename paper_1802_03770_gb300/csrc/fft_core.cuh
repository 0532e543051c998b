// Shared-memory FFT building blocks for sm_103a.
//
// A CTA transforms a batch of complex lines that live in shared memory, each
// of power-of-two length L.  The transform is a Stockham autosort FFT: stage
// s with radix R reads butterfly j's legs at j + r L/R, multiplies leg r by
// the twiddle w^(r k), k = j mod Ns, with w = exp(-+ 2 pi i / (Ns R)), does a
// radix-R DFT in registers and writes leg r to (j / Ns) Ns R + k + r Ns
// (Govindaraju et al., SC'08).  After the last stage the line is in natural
// order.  Stages are radix 16 (when a thread may hold 16 values), then radix
// 8, with one radix-4 or radix-2 stage for the remainder of log2 L (see
// FftPlan).
//
// Every stage is in place: each thread loads all legs of the butterflies it
// owns into registers, the CTA synchronises, then every thread writes.  The
// number of values a thread holds is VPT = lines * L / blockDim.x, a
// compile-time bound chosen by the launcher.
//
// Twiddles: FP64 stages load every power w^r from a table
// tw[k] = exp(-2 pi i k / Lmax) computed on the host in long double; FP32
// stages compute w with sincospif and the even powers by squaring; the
// other powers are complex products (see twiddles()).
//
// Two storage layouts: lines of stride ls (element j of line q at
// q * ls + j, ls a multiple of 16), and 2^ltx interleaved lines (element j
// of line c at j * 2^ltx + c, the natural layout of a tile of consecutive
// columns).  Indices are logical (see SBuf).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// Qualifier of the pass bodies' pointers: __restrict__ by default.  A kernel
// that runs several passes in one launch (a pass reading what an earlier
// pass of the same launch wrote) defines it empty before including this
// file, so that no input is taken as read-only for the whole launch.
#ifndef FL_RESTRICT
#define FL_RESTRICT __restrict__
#endif

namespace fl {

template <typename T> struct Cplx;
template <> struct Cplx<float> { typedef float2 type; };
template <> struct Cplx<double> { typedef double2 type; };

// Complex buffer in shared memory with one pad element after every 16: the
// logical index i is stored at i + i/16.  The first Stockham stage writes the
// R legs of a butterfly to R consecutive logical places (a stride of R
// complex values across threads), which without the pad puts every thread of
// a warp on the same banks.
template <typename C>
struct SBuf {
  C* p;
  __device__ __forceinline__ C& operator[](int i) const { return p[i + (i >> 4)]; }
  // view starting at logical offset `off` (a multiple of 16)
  __device__ __forceinline__ SBuf at(int off) const { return SBuf{p + off + (off >> 4)}; }
};
// complex elements to allocate for `logical` logical ones
inline constexpr long long sbuf_elems(long long logical) { return logical + logical / 16 + 1; }

template <typename C> __device__ __forceinline__ C cmake(decltype(C().x) a, decltype(C().x) b) {
  C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
#if defined(__CUDA_ARCH__) && !defined(FL_SCALAR_CADD)
// FP32: both halves in one paired add (sm_100 family), same rounding as two
// scalar adds.
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
#endif
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmake<C>(a.x, -a.y); }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return cmake<C>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename C> __device__ __forceinline__ C mul_mi(C a, bool inv) {
  return inv ? cmake<C>(-a.y, a.x) : cmake<C>(a.y, -a.x);
}
// multiply by exp(-+ i theta) given (cos theta, sin theta)
template <typename C, typename T> __device__ __forceinline__ C mul_rot(C a, T c, T s, bool inv) {
  const T sg = inv ? s : -s;
  return cmake<C>(a.x * c - a.y * sg, a.x * sg + a.y * c);
}

template <typename C> __device__ __forceinline__ void dft2(C* v) {
  C a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <typename C> __device__ __forceinline__ void dft4(C* v, bool inv) {
  C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  C t2 = cadd(v[1], v[3]), t3 = mul_mi(csub(v[1], v[3]), inv);
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}

template <typename C> __device__ __forceinline__ void dft8(C* v, bool inv) {
  typedef decltype(C().x) T;
  const T s = (T)0.70710678118654752440084436210484903928;
  C e[4] = {v[0], v[2], v[4], v[6]};
  C o[4] = {v[1], v[3], v[5], v[7]};
  dft4(e, inv);
  dft4(o, inv);
  // o[k] *= w8^k, w8 = (1 -+ i)/sqrt(2)
  o[1] = mul_rot(o[1], s, s, inv);
  o[2] = mul_mi(o[2], inv);
  o[3] = mul_rot(o[3], -s, s, inv);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = cadd(e[k], o[k]);
    v[k + 4] = csub(e[k], o[k]);
  }
}

// 16-point DFT as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2,
// X[k] = sum_n2 w16^(n2 k1) w4^(n2 k2) sum_n1 x[4 n1 + n2] w4^(n1 k1).
// HALF: x[8..15] are zero (the zero-padded half of a line), so the inner
// 4-point DFTs have two zero inputs.
template <bool HALF = false, typename C> __device__ __forceinline__ void dft16(C* v, bool inv) {
  typedef decltype(C().x) T;
  const T c1 = (T)0.92387953251128675612818318939678828682;  // cos(pi/8)
  const T s1 = (T)0.38268343236508977172845998403039886676;  // sin(pi/8)
  const T h = (T)0.70710678118654752440084436210484903928;
  C a[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    if (HALF) {
      const C x0 = v[n2], x1 = v[4 + n2];
      const C t = mul_mi(x1, inv);
      a[n2][0] = cadd(x0, x1);
      a[n2][1] = cadd(x0, t);
      a[n2][2] = csub(x0, x1);
      a[n2][3] = csub(x0, t);
    } else {
      a[n2][0] = v[n2];
      a[n2][1] = v[4 + n2];
      a[n2][2] = v[8 + n2];
      a[n2][3] = v[12 + n2];
      dft4(a[n2], inv);
    }
  }
  // twiddles w16^(n2 k1): (1,1)=1, (1,2)=2, (1,3)=3, (2,1)=2, (2,2)=4, (2,3)=6, (3,1)=3, (3,2)=6, (3,3)=9
  a[1][1] = mul_rot(a[1][1], c1, s1, inv);
  a[1][2] = mul_rot(a[1][2], h, h, inv);
  a[1][3] = mul_rot(a[1][3], s1, c1, inv);
  a[2][1] = mul_rot(a[2][1], h, h, inv);
  a[2][2] = mul_mi(a[2][2], inv);
  a[2][3] = mul_rot(a[2][3], -h, h, inv);
  a[3][1] = mul_rot(a[3][1], s1, c1, inv);
  a[3][2] = mul_rot(a[3][2], -h, h, inv);
  a[3][3] = mul_rot(a[3][3], -c1, -s1, inv);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C b[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
    dft4(b, inv);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
  }
}

template <int R, typename C> __device__ __forceinline__ void dftR(C* v, bool inv) {
  if (R == 2) dft2(v);
  else if (R == 4) dft4(v, inv);
  else if (R == 8) dft8(v, inv);
  else dft16(v, inv);
}

template <int R> struct LogR;
template <> struct LogR<2> { static constexpr int v = 1; };
template <> struct LogR<4> { static constexpr int v = 2; };
template <> struct LogR<8> { static constexpr int v = 3; };
template <> struct LogR<16> { static constexpr int v = 4; };

// w[r] = w1^r, r = 0..R-1, for w1 = exp(-2 pi i step / Lmax) (conjugated
// for the inverse).  FP64, and FP32 with TWT (tw then points to a copy of
// the table in shared memory): every power is loaded from the long-double
// table tw (GB300's FP64 rate makes the loads cheaper than products).  FP32: w1 = sincospif(-2 step / Lmax) (the
// argument is exact), w2, w4, w8 by squaring, the rest by products -- no
// table load on the stage's critical path (measured 3 % faster solves on
// the 1024^2 workload than the table, at unchanged iteration counts).
template <int R, bool TWT = false, typename C>
__device__ __forceinline__ void twiddles(const C* FL_RESTRICT tw, int step, bool inv, C* w, int lgmax) {
  auto ld = [&](int i) {
    C t;
    if constexpr (sizeof(t.x) == 4 && !TWT) {
      float sn, cs;
      sincospif(-(float)i * ldexpf(1.0f, 1 - lgmax), &sn, &cs);
      t.x = cs;
      t.y = sn;
    } else {
      t = tw[i];
    }
    if (inv) t.y = -t.y;
    return t;
  };
  w[0] = cmake<C>(1, 0);
  if constexpr (sizeof(w[0].x) == 8 || TWT) {
    // FP64, and FP32 with a table (TWT): every power straight from the table
    // (loads instead of products; r * step < Lmax)
#pragma unroll
    for (int r = 1; r < R; ++r) w[r] = ld(r * step);
    return;
  }
  if (R >= 2) w[1] = ld(step);
  if (R >= 4) {
    w[2] = sizeof(w[0].x) == 4 ? cmul(w[1], w[1]) : ld(2 * step);
    w[3] = cmul(w[1], w[2]);
  }
  if (R >= 8) {
    w[4] = sizeof(w[0].x) == 4 ? cmul(w[2], w[2]) : ld(4 * step);
    w[5] = cmul(w[4], w[1]);
    w[6] = cmul(w[4], w[2]);
    w[7] = cmul(w[4], w[3]);
  }
  if (R >= 16) {
    w[8] = sizeof(w[0].x) == 4 ? cmul(w[4], w[4]) : ld(8 * step);
#pragma unroll
    for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
  }
}

// One Stockham stage with a compile-time shape: radix R, length 2^LG,
// NS = product of the radices of the earlier stages.  MODE selects where the
// legs come from and where the outputs go:
//   STAGE_FIRST: legs from load(line, index) (NS = 1, no twiddles), outputs
//                to shared memory; a barrier between the two when sync_io
//                (the loader reads the buffer);
//   STAGE_MID:   shared memory to shared memory (two barriers);
//   STAGE_LAST:  legs from shared memory, outputs (natural order) to
//                epi(line, index, value); a barrier before the epilogue when
//                sync_io (the epilogue writes the buffer), none after.
// STAGE_FIRST and STAGE_MID end with a barrier.  With the shape known at
// compile time, leg r of a butterfly sits at a fixed physical offset from
// leg 0 (the SBuf pad is one element per 16, and the leg stride is a
// multiple of 16), so only the first leg's address is padded.
enum { STAGE_FIRST = 0, STAGE_MID = 1, STAGE_LAST = 2 };

__device__ __forceinline__ int sbuf_phys(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int clog2(int x) { return x <= 1 ? 0 : 1 + clog2(x / 2); }

template <int R, int VPT, bool IL, int LG, int NS, int MODE, bool HALF, bool TWT, typename C,
          typename Load, typename Epi>
__device__ __forceinline__ void stage_ct(SBuf<C> buf, int ls, int ltx, int nlines,
                                         const C* FL_RESTRICT tw, int lgmax, bool inv, Load& load,
                                         Epi& epi, bool sync_io) {
  constexpr int NB = VPT / R;
  constexpr int LGLR = LG - LogR<R>::v;
  constexpr int LR = 1 << LGLR;
  const int total = IL ? (LR << ltx) : (nlines << LGLR);
  // physical leg strides (valid when the logical stride is a multiple of 16)
  const int rd_stride = IL ? sbuf_phys(LR << ltx) : sbuf_phys(LR);
  const int wr_stride = IL ? sbuf_phys(NS << ltx) : sbuf_phys(NS);
  C v[NB][R];
  int line_of[NB], out0[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int g = threadIdx.x + b * blockDim.x;
    out0[b] = -1;
    line_of[b] = 0;
    if (g < total) {
      const int line = IL ? (g & ((1 << ltx) - 1)) : (g >> LGLR);
      const int j = IL ? (g >> ltx) : (g & (LR - 1));
      const int k = j & (NS - 1);
      if constexpr (MODE == STAGE_FIRST) {
        // HALF: legs R/2.. lie in the zero upper half of the line
#pragma unroll
        for (int r = 0; r < R; ++r)
          v[b][r] = (HALF && 2 * r >= R) ? cmake<C>(0, 0) : load(line, j + r * LR);
      } else {
        const int l0 = IL ? ((j << ltx) + line) : (line * ls + j);
        if ((IL ? ((LR << ltx) & 15) : (LR & 15)) == 0) {
          const C* p0 = buf.p + sbuf_phys(l0);
#pragma unroll
          for (int r = 0; r < R; ++r) v[b][r] = p0[r * rd_stride];
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) v[b][r] = buf[l0 + (IL ? ((r * LR) << ltx) : r * LR)];
        }
        if (NS > 1 && k != 0) {
          // twiddle w^(r k) = tw[r * k * Lmax / (NS R)]
          C w[R];
          twiddles<R, TWT>(tw, k << (lgmax - clog2(NS * R)), inv, w, lgmax);
#pragma unroll
          for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], w[r]);
        }
      }
      if constexpr (HALF && R == 16 && MODE == STAGE_FIRST) dft16<true>(v[b], inv);
      else dftR<R>(v[b], inv);
      line_of[b] = line;
      out0[b] = (j - k) * R + k;
    }
  }
  if (MODE == STAGE_MID || sync_io) __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if (out0[b] >= 0) {
      if constexpr (MODE == STAGE_LAST) {
#pragma unroll
        for (int r = 0; r < R; ++r) epi(line_of[b], out0[b] + r * NS, v[b][r]);
      } else {
        const int d0 = IL ? ((out0[b] << ltx) + line_of[b]) : (line_of[b] * ls + out0[b]);
        // NS a multiple of 16: fixed physical stride; NS = 1: the R legs are
        // R consecutive logical places inside one 16-element group (R | 16)
        if (!IL && NS == 1) {
          C* p0 = buf.p + sbuf_phys(d0);
#pragma unroll
          for (int r = 0; r < R; ++r) p0[r] = v[b][r];
        } else if ((IL ? ((NS << ltx) & 15) : (NS & 15)) == 0) {
          C* p0 = buf.p + sbuf_phys(d0);
#pragma unroll
          for (int r = 0; r < R; ++r) p0[r * wr_stride] = v[b][r];
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) buf[d0 + (IL ? ((r * NS) << ltx) : r * NS)] = v[b][r];
        }
      }
    }
  }
  if constexpr (MODE != STAGE_LAST) __syncthreads();
}

// Stage plan of a length-2^LG transform with VPT values per thread: radix 16
// while at least four factors of two remain (if VPT allows), then radix 8,
// then one radix-4 or radix-2 stage (n16, n8, tail).  A radix-2 remainder
// (LG = 1 mod 4) is avoided by taking 8 x 4 for the last 16 x 2: a radix-2
// stage gives every thread VPT/2 butterflies, each with its own twiddle.
template <int LG, int VPT>
struct FftPlan {
  static constexpr int n16 = VPT >= 16 ? (LG % 4 == 1 && LG >= 5 ? LG / 4 - 1 : LG / 4) : 0;
  static constexpr int n8 = (LG - 4 * n16) / 3;
  static constexpr int tail = LG - 4 * n16 - 3 * n8;
  static constexpr int S = n16 + n8 + (tail > 0 ? 1 : 0);
  __host__ __device__ static constexpr int radix(int s) {
    return s < n16 ? 16 : (s < n16 + n8 ? 8 : (1 << tail));
  }
  __host__ __device__ static constexpr int ns(int s) { return s == 0 ? 1 : ns(s - 1) * radix(s - 1); }
};

template <int LG, int VPT, bool IL, bool HALF, bool TWT, int ST, typename C, typename Load, typename Epi>
__device__ __forceinline__ void fft_io_stage(SBuf<C> buf, int ls, int ltx, int nlines,
                                             const C* FL_RESTRICT tw, int lgmax, bool inv, Load load,
                                             bool sync_load, Epi epi, bool sync_epi) {
  typedef FftPlan<LG, VPT> P;
  constexpr int R = P::radix(ST);
  constexpr int Ns = P::ns(ST);
  constexpr int MODE = ST == 0 ? STAGE_FIRST : (ST == P::S - 1 ? STAGE_LAST : STAGE_MID);
  stage_ct<R, VPT, IL, LG, Ns, MODE, HALF, TWT>(buf, ls, ltx, nlines, tw, lgmax, inv, load, epi,
                                          MODE == STAGE_FIRST ? sync_load : sync_epi);
  if constexpr (ST + 1 < P::S)
    fft_io_stage<LG, VPT, IL, HALF, TWT, ST + 1>(buf, ls, ltx, nlines, tw, lgmax, inv, load, sync_load,
                                               epi, sync_epi);
}

// A full transform of `nlines` lines (IL: 2^ltx interleaved lines) of length
// 2^LG: legs of the first stage from load(line, index), outputs to
// epi(line, index, value) in natural order.  sync_load: the loader reads the
// shared buffer (a barrier separates its reads from the first stage's
// writes); sync_epi: the epilogue writes the shared buffer.  The buffer is
// free again after a barrier that follows the call.
template <int LG, int VPT, bool IL, bool HALF, bool TWT, typename C, typename Load, typename Epi>
__device__ __forceinline__ void fft_io_ct(SBuf<C> buf, int ls, int ltx, int nlines,
                                          const C* FL_RESTRICT tw, int lgmax, bool inv, Load load,
                                          bool sync_load, Epi epi, bool sync_epi) {
  if constexpr (FftPlan<LG, VPT>::S >= 2) {
    fft_io_stage<LG, VPT, IL, HALF, TWT, 0>(buf, ls, ltx, nlines, tw, lgmax, inv, load, sync_load, epi,
                                          sync_epi);
  } else {
    // one stage: natural order in shared memory afterwards; each thread
    // hands on elements it reads (an epilogue writing the buffer rewrites
    // the element it was given)
    stage_ct<FftPlan<LG, VPT>::radix(0), VPT, IL, LG, 1, STAGE_FIRST, HALF, TWT>(
        buf, ls, ltx, nlines, tw, lgmax, inv, load, epi, sync_load);
    constexpr int L = 1 << LG;
    const int total = IL ? (L << ltx) : nlines * L;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int line = IL ? (e & ((1 << ltx) - 1)) : e / L;
      const int j = IL ? (e >> ltx) : e % L;
      epi(line, j, IL ? buf[e] : buf[line * ls + j]);
    }
  }
}

// Runtime length: dispatch to the compile-time plan of the lengths
// 2^LGLO .. 2^LGHI a kernel instantiation can hold (at most 2^4 .. 2^13);
// other lengths are never passed by the launchers.  HALF: the upper half of
// every input line is zero (a zero-padded line); the loader is then not
// called for it.
#define FL_FFT_LEN(LGV)                                                                     \
  if constexpr (LGV >= LGLO && LGV <= LGHI) {                                               \
    if (lg == LGV) {                                                                        \
      fft_io_ct<LGV, VPT, IL, HALF, TWT>(buf, ls, ltx, nlines, tw, lgmax, inv, load, sync_load, \
                                         epi, sync_epi);                                    \
      return;                                                                               \
    }                                                                                       \
  }
template <int VPT, bool IL, bool HALF = false, int LGHI = 11, int LGLO = 4, bool TWT = false, typename C,
          typename Load, typename Epi>
__device__ __forceinline__ void fft_io(SBuf<C> buf, int lg, int ls, int ltx, int nlines,
                                       const C* FL_RESTRICT tw, int lgmax, bool inv, Load load,
                                       bool sync_load, Epi epi, bool sync_epi) {
  FL_FFT_LEN(13)
  FL_FFT_LEN(12)
  FL_FFT_LEN(11)
  FL_FFT_LEN(10)
  FL_FFT_LEN(9)
  FL_FFT_LEN(8)
  FL_FFT_LEN(7)
  FL_FFT_LEN(6)
  FL_FFT_LEN(5)
  FL_FFT_LEN(4)
}
#undef FL_FFT_LEN

// In-place transform of lines in shared memory (natural order in and out)
// with the compile-time stage plan; ends with a barrier.
template <int VPT, bool IL, int LGHI = 11, int LGLO = 4, bool TWT = false, typename C>
__device__ __forceinline__ void fft_smem(SBuf<C> buf, int lg, int ls, int ltx, int nlines,
                                         const C* FL_RESTRICT tw, int lgmax, bool inv) {
  auto ld = [=](int q, int k) -> C { return IL ? buf[(k << ltx) + q] : buf[q * ls + k]; };
  auto st = [=](int q, int k, C v) {
    if (IL) buf[(k << ltx) + q] = v;
    else buf[q * ls + k] = v;
  };
  fft_io<VPT, IL, false, LGHI, LGLO, TWT>(buf, lg, ls, ltx, nlines, tw, lgmax, inv, ld, true, st, true);
  __syncthreads();
}

}  // namespace fl
