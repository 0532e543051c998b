// Shared-memory FFT building blocks for sm_103a.
//
// A CTA transforms a batch of complex lines that live in shared memory.
// Each line has power-of-two length L and the lines are spaced `ls`
// complex elements apart.  The transform is a Stockham autosort FFT: stage s
// with radix R reads butterfly j's legs at j + r L/R, multiplies leg r by the
// twiddle w^(r k), k = j mod Ns, with w = exp(-+ 2 pi i / (Ns R)), does a
// radix-R DFT in registers and writes leg r to (j / Ns) Ns R + k + r Ns
// (Govindaraju et al., SC'08).  After the last stage the line is in natural
// order.  Stages are radix 8 with one radix-4 or radix-2 stage when log2 L
// is not a multiple of 3.
//
// Every stage is in place: each thread loads all legs of the butterflies it
// owns into registers, the CTA synchronises, then every thread writes.  The
// number of values a thread holds is VPT = lines * L / blockDim.x, a
// compile-time bound chosen by the launcher.
//
// Twiddles come from a table tw[k] = exp(-2 pi i k / Lmax) computed on the
// host in long double; a line of length L uses stride Lmax / L.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fl {

template <typename T> struct Cplx;
template <> struct Cplx<float> { typedef float2 type; };
template <> struct Cplx<double> { typedef double2 type; };

template <typename C> __device__ __forceinline__ C cmake(decltype(C().x) a, decltype(C().x) b) {
  C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmake<C>(a.x, -a.y); }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return cmake<C>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename C> __device__ __forceinline__ C mul_mi(C a, bool inv) {
  return inv ? cmake<C>(-a.y, a.x) : cmake<C>(a.y, -a.x);
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
  o[1] = inv ? cmake<C>((o[1].x - o[1].y) * s, (o[1].x + o[1].y) * s)
             : cmake<C>((o[1].x + o[1].y) * s, (o[1].y - o[1].x) * s);
  o[2] = mul_mi(o[2], inv);
  o[3] = inv ? cmake<C>((-o[3].x - o[3].y) * s, (o[3].x - o[3].y) * s)
             : cmake<C>((o[3].y - o[3].x) * s, (-o[3].x - o[3].y) * s);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = cadd(e[k], o[k]);
    v[k + 4] = csub(e[k], o[k]);
  }
}

template <int R, typename C> __device__ __forceinline__ void dftR(C* v, bool inv) {
  if (R == 2) dft2(v);
  else if (R == 4) dft4(v, inv);
  else dft8(v, inv);
}

// One Stockham stage of radix R over `nlines` lines of length L = 2^lg.
// VPT: values per thread (upper bound, compile time).  Contains two
// __syncthreads(); every thread of the CTA must call it.
template <int R, int VPT, typename C>
__device__ __forceinline__ void stockham_stage(C* buf, int lg, int ls, int nlines, int Ns,
                                               const C* __restrict__ tw, int lgmax, bool inv) {
  constexpr int NB = VPT / R;  // butterflies per thread
  constexpr int LGR = R == 8 ? 3 : (R == 4 ? 2 : 1);
  const int lglr = lg - LGR;
  const int LR = 1 << lglr;
  const int total = nlines << lglr;
  C v[NB][R];
  int dst[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int g = threadIdx.x + b * blockDim.x;
    dst[b] = -1;
    if (g < total) {
      const int line = g >> lglr;
      const int j = g & (LR - 1);
      const int k = j & (Ns - 1);
      C* base = buf + (size_t)line * ls;
      // twiddle index for leg r: r * k * (Lmax / (Ns * R))
      const int step = k << (lgmax - __ffs(Ns * R) + 1);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x = base[j + r * LR];
        if (r > 0 && k != 0) {
          C w = tw[r * step];
          if (inv) w.y = -w.y;
          x = cmul(x, w);
        }
        v[b][r] = x;
      }
      dftR<R>(v[b], inv);
      dst[b] = line * ls + (j - k) * R + k;
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if (dst[b] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) buf[dst[b] + r * Ns] = v[b][r];
    }
  }
  __syncthreads();
}

// The same stage for 2^ltx lines stored interleaved: element j of line c is
// buf[j * tx + c] (the natural layout of a tile of tx consecutive columns).
// Consecutive threads take consecutive lines, so the leg reads are
// contiguous.
template <int R, int VPT, typename C>
__device__ __forceinline__ void stockham_stage_il(C* buf, int lg, int ltx, int Ns,
                                                  const C* __restrict__ tw, int lgmax, bool inv) {
  constexpr int NB = VPT / R;
  const int L = 1 << lg;
  const int LR = L / R;
  const int tx = 1 << ltx;
  const int total = LR << ltx;
  C v[NB][R];
  int dst[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int g = threadIdx.x + b * blockDim.x;
    dst[b] = -1;
    if (g < total) {
      const int c = g & (tx - 1);
      const int j = g >> ltx;
      const int k = j & (Ns - 1);
      const int step = k << (lgmax - __ffs(Ns * R) + 1);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x = buf[((j + r * LR) << ltx) + c];
        if (r > 0 && k != 0) {
          C w = tw[r * step];
          if (inv) w.y = -w.y;
          x = cmul(x, w);
        }
        v[b][r] = x;
      }
      dftR<R>(v[b], inv);
      dst[b] = (((j - k) * R + k) << ltx) + c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if (dst[b] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) buf[dst[b] + ((r * Ns) << ltx)] = v[b][r];
    }
  }
  __syncthreads();
}

template <int VPT, typename C>
__device__ __forceinline__ void fft_lines_il(C* buf, int lg, int ltx, const C* __restrict__ tw,
                                             int lgmax, bool inv) {
  int Ns = 1;
  int rem = lg;
  while (rem >= 3) {
    stockham_stage_il<8, VPT>(buf, lg, ltx, Ns, tw, lgmax, inv);
    Ns <<= 3;
    rem -= 3;
  }
  if (rem == 2) stockham_stage_il<4, VPT>(buf, lg, ltx, Ns, tw, lgmax, inv);
  else if (rem == 1) stockham_stage_il<2, VPT>(buf, lg, ltx, Ns, tw, lgmax, inv);
}

// Full FFT (unnormalised) of `nlines` lines of length 2^lg in shared memory.
// Forward: X_k = sum_j x_j exp(-2 pi i jk / L); inverse uses +.
// The caller must __syncthreads() before (data ready); on return the data is
// visible to all threads.
template <int VPT, typename C>
__device__ __forceinline__ void fft_lines(C* buf, int lg, int ls, int nlines, const C* __restrict__ tw, int lgmax,
                          bool inv) {
  int Ns = 1;
  int rem = lg;
  while (rem >= 3) {
    stockham_stage<8, VPT>(buf, lg, ls, nlines, Ns, tw, lgmax, inv);
    Ns <<= 3;
    rem -= 3;
  }
  if (rem == 2) stockham_stage<4, VPT>(buf, lg, ls, nlines, Ns, tw, lgmax, inv);
  else if (rem == 1) stockham_stage<2, VPT>(buf, lg, ls, nlines, Ns, tw, lgmax, inv);
}

}  // namespace fl
