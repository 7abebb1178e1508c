// Shared-memory Stockham FFTs of power-of-two length, radix 8 with one
// radix-4 or radix-2 tail pass.  Every participating thread owns eight points
// per pass, so a length-L transform of one column takes L/8 threads.  Many
// columns can be transformed together: element r of column c lives at
// buf[r * stride + c]; the caller maps threads to (column, butterfly).
//
// Direction SIGN = -1 computes X_m = sum_p x_p e^{-2 pi i m p / L},
// SIGN = +1 the same with e^{+...}; no normalisation.  Twiddles come from a
// table tw[m] = e^{-2 pi i m / L}, m < L (FP64-rounded), read through the
// read-only cache; SIGN = +1 conjugates them.
#pragma once

#include "common.cuh"

namespace isam {

template <int SIGN, typename C>
__device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a; a = cadd(t, b); b = csub(t, b);
}

template <int SIGN, typename C>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C t0 = cadd(a0, a2), t1 = csub(a0, a2);
  C t2 = cadd(a1, a3), t3 = cmul_i<SIGN>(csub(a1, a3));
  a0 = cadd(t0, t2); a2 = csub(t0, t2);
  a1 = cadd(t1, t3); a3 = csub(t1, t3);
}

template <int SIGN, typename T>
__device__ __forceinline__ void dft8(cplx<T>* a) {
  using C = cplx<T>;
  dft4<SIGN>(a[0], a[2], a[4], a[6]);
  dft4<SIGN>(a[1], a[3], a[5], a[7]);
  const T h = T(0.70710678118654752440);
  // odd half times W8^k, W8 = e^{SIGN 2 pi i / 8}
  C o1 = a[3], o2 = a[5], o3 = a[7];
  a[3] = mk<T>(h * (o1.x - SIGN * o1.y), h * (o1.y + SIGN * o1.x));
  a[5] = cmul_i<SIGN>(o2);
  a[7] = mk<T>(h * (-o3.x - SIGN * o3.y), h * (-o3.y + SIGN * o3.x));
  // combine: y_k = E_k + W^k O_k, y_{k+4} = E_k - W^k O_k
  C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  C p0 = a[1], p1 = a[3], p2 = a[5], p3 = a[7];
  a[0] = cadd(e0, p0); a[4] = csub(e0, p0);
  a[1] = cadd(e1, p1); a[5] = csub(e1, p1);
  a[2] = cadd(e2, p2); a[6] = csub(e2, p2);
  a[3] = cadd(e3, p3); a[7] = csub(e3, p3);
}

template <int SIGN, typename T>
__device__ __forceinline__ cplx<T> twiddle(const cplx<T>* __restrict__ tw, int m) {
  cplx<T> w = __ldg(tw + m);
  if (SIGN > 0) w.y = -w.y;
  return w;
}

// One Stockham pass of radix R on column `col` (element r at buf[r*stride+col]);
// this thread does 8/R butterflies j = b + u * (L/8).  Reads all its inputs,
// block barrier, writes.  Must be reached by every thread of the block.
template <int SIGN, int R, typename T>
__device__ __forceinline__ void stockham_pass(cplx<T>* buf, int stride, int col, int b, int L,
                                              int Ns, const cplx<T>* __restrict__ tw,
                                              bool active) {
  using C = cplx<T>;
  constexpr int NB = 8 / R;          // butterflies per thread
  const int LR = L / R;
  const int L8 = L >> 3;
  C v[8];
  if (active) {
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int j = b + u * L8;
#pragma unroll
      for (int r = 0; r < R; ++r) v[u * R + r] = buf[(j + r * LR) * stride + col];
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int j = b + u * L8;
      const int k = j & (Ns - 1);
      C* a = v + u * R;
      if (Ns > 1) {
        const int step = (L / (Ns * R)) * k;   // twiddle index for r = 1
#pragma unroll
        for (int r = 1; r < R; ++r) a[r] = cmul(a[r], twiddle<SIGN, T>(tw, r * step));
      }
      if (R == 8) dft8<SIGN, T>(a);
      else if (R == 4) dft4<SIGN>(a[0], a[1], a[2], a[3]);
      else dft2<SIGN>(a[0], a[1]);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[(base + r * Ns) * stride + col] = a[r];
    }
  }
  __syncthreads();
}

// Length-L transform (L = 2^logL, 1 <= L <= 8192) of column `col`.  For
// L >= 8 the active threads own butterfly b < L/8; for L < 8 the thread with
// b == 0 transforms the column directly.  Every thread of the block must call
// it (it contains barriers); it ends with a barrier.
template <int SIGN, typename T>
__device__ __forceinline__ void fft_smem(cplx<T>* buf, int stride, int col, int b, int L,
                                         int logL, const cplx<T>* __restrict__ tw,
                                         bool active) {
  using C = cplx<T>;
  if (L >= 8) {
    int Ns = 1;
    const int n8 = logL / 3;
    for (int p = 0; p < n8; ++p) {
      stockham_pass<SIGN, 8, T>(buf, stride, col, b, L, Ns, tw, active);
      Ns *= 8;
    }
    const int rem = logL - 3 * n8;
    if (rem == 2) stockham_pass<SIGN, 4, T>(buf, stride, col, b, L, Ns, tw, active);
    else if (rem == 1) stockham_pass<SIGN, 2, T>(buf, stride, col, b, L, Ns, tw, active);
  } else {
    __syncthreads();
    if (active && b == 0 && L > 1) {
      C a0 = buf[col], a1 = buf[stride + col];
      if (L == 2) {
        dft2<SIGN>(a0, a1);
      } else {
        C a2 = buf[2 * stride + col], a3 = buf[3 * stride + col];
        dft4<SIGN>(a0, a1, a2, a3);
        buf[2 * stride + col] = a2; buf[3 * stride + col] = a3;
      }
      buf[col] = a0; buf[stride + col] = a1;
    }
    __syncthreads();
  }
}

}  // namespace isam
