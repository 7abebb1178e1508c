// Column-split radix-16 transforms of the axial kernels' column pair, for
// FP32 and K = 2^LOGK, LOGK = 11 or 12 (K = 16 * 16 * 8 or 16 * 16 * 16).
//
// The pair's FFT buffer holds rows of two complex columns (cpair).  Here each
// of the K/8 threads owns one column of one radix-16 butterfly per pass
// (thread t: column c = t & 1, butterfly j = t >> 1, 16 complex points, the
// same 32 floats of data a radix-8 thread holds as 8 pairs), so a K-point
// transform takes three shared-memory passes instead of four with no change
// in threads or registers.  Lanes alternate columns, so a warp's 8-byte
// accesses to 16 consecutive rows cover 256 contiguous bytes.
//
// Two row layouts share the buffer: P8 (one padding row after every 8 rows,
// the layout of the interpolation and the adjoint scatter) and P16 (one after
// every 16 rows, under which the span-1 pass's writes to rows 16 j + r of
// consecutive j fall in distinct 16-byte bank groups).  Every pass reads all
// its inputs before a barrier and then writes, so a pass may read one layout
// and write the other: the forward transform ends in P8 for the
// interpolation, the inverse starts from P8 after the scatter.
#pragma once

#include "fft_smem.cuh"

namespace isam {
namespace c16 {

enum { P8 = 8, P16 = 16 };

// float2 index of (row, column c) in layout PAD, W float2 columns per row
// (2 for the axial column pair, 2 TP for a lateral tile of TP column pairs)
template <int PAD, int W = 2> __device__ __forceinline__ int el(int row, int c) {
  return W * (PAD == P8 ? row + (row >> 3) : row + (row >> 4)) + c;
}

// multiply by W16^1 = e^{SIGN 2 pi i / 16} and W16^3
template <int SIGN> __device__ __forceinline__ float2 w16_1(float2 o) {
  const float c = 0.92387953251128675613f, s = 0.38268343236508977173f;
  return make_float2(o.x * c - SIGN * o.y * s, o.y * c + SIGN * o.x * s);
}
template <int SIGN> __device__ __forceinline__ float2 w16_3(float2 o) {
  const float c = 0.38268343236508977173f, s = 0.92387953251128675613f;
  return make_float2(o.x * c - SIGN * o.y * s, o.y * c + SIGN * o.x * s);
}

// 16-point DFT in place, natural order in and out, as 4 x 4:
// X[k1 + 4 k2] = sum_{n2} W4^{n2 k2} W16^{n2 k1} sum_{n1} x[n2 + 4 n1] W4^{n1 k1}.
// HALF_ZERO: inputs 4..11 are zero (the span-1 pass of the twice zero-padded
// forward transform).
template <int SIGN, bool HALF_ZERO>
__device__ __forceinline__ void dft16(float2* a) {
  float2 b[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    if (HALF_ZERO) {
      const float2 x0 = a[n2], x3 = a[n2 + 12];
      b[n2][0] = cadd(x0, x3);
      b[n2][1] = sub_rot<SIGN>(x0, x3);
      b[n2][2] = csub(x0, x3);
      b[n2][3] = add_rot<SIGN>(x0, x3);
    } else {
      float2 x0 = a[n2], x1 = a[n2 + 4], x2 = a[n2 + 8], x3 = a[n2 + 12];
      dft4<SIGN>(x0, x1, x2, x3);
      b[n2][0] = x0; b[n2][1] = x1; b[n2][2] = x2; b[n2][3] = x3;
    }
  }
  b[1][1] = w16_1<SIGN>(b[1][1]);
  b[1][2] = ew8_1<SIGN>(b[1][2]);
  b[1][3] = w16_3<SIGN>(b[1][3]);
  b[2][1] = ew8_1<SIGN>(b[2][1]);
  b[2][2] = cmul_i<SIGN>(b[2][2]);
  b[2][3] = ew8_3<SIGN>(b[2][3]);
  b[3][1] = w16_3<SIGN>(b[3][1]);
  b[3][2] = ew8_3<SIGN>(b[3][2]);
  {
    const float2 t = w16_1<SIGN>(b[3][3]);                 // W16^9 = -W16^1
    b[3][3] = make_float2(-t.x, -t.y);
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 y0 = b[0][k1], y1 = b[1][k1], y2 = b[2][k1], y3 = b[3][k1];
    dft4<SIGN>(y0, y1, y2, y3);
    a[k1] = y0; a[k1 + 4] = y1; a[k1 + 8] = y2; a[k1 + 12] = y3;
  }
}

template <int SIGN, int R> __device__ __forceinline__ void dft_r(float2* a) {
  if constexpr (R == 16) dft16<SIGN, false>(a);
  else if constexpr (R == 8) dft8<SIGN>(a);
  else if constexpr (R == 4) dft4<SIGN>(a[0], a[1], a[2], a[3]);
  else dft2<SIGN>(a[0], a[1]);
}

// Twiddle table: per pass with span NS > 1 (radix R), entry k < NS holds
// (w, w^4), w = e^{-2 pi i k / (NS R)}: the span-16 segment (16 entries), then
// the span-256 one (256 entries).
template <int LOGK> struct Passes {
  static constexpr int K = 1 << LOGK;
  static constexpr int R3 = LOGK == 12 ? 16 : 8;   // radix of the span-256 pass
  static constexpr int entries = 16 + 256;
};

__host__ __device__ constexpr size_t twiddle_bytes() { return size_t(16 + 256) * sizeof(float4); }

template <int LOGK> __device__ __forceinline__ void build_twiddles(float4* tw) {
  for (int e = threadIdx.x; e < Passes<LOGK>::entries; e += blockDim.x) {
    const int ns = e < 16 ? 16 : 256, k = e < 16 ? e : e - 16;
    const int R = e < 16 ? 16 : Passes<LOGK>::R3;
    float s1, c1, s4, c4;
    sincospif(float(2 * k) / float(ns * R), &s1, &c1);
    sincospif(float(8 * k) / float(ns * R), &s4, &c4);
    tw[e] = make_float4(c1, -s1, c4, -s4);
  }
  __syncthreads();
}

// a[r] *= w^r, r = 1 .. R-1 (R = 2, 4, 8 or 16), from (w, w^4) (conjugated
// for SIGN > 0)
template <int SIGN, int R> __device__ __forceinline__ void twiddle(float2* a, float4 t) {
  float2 w1 = make_float2(t.x, t.y), w4 = make_float2(t.z, t.w);
  if (SIGN > 0) { w1.y = -w1.y; w4.y = -w4.y; }
  a[1] = cmul(a[1], w1);
  if constexpr (R == 2) return;
  const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
  a[2] = cmul(a[2], w2);
  a[3] = cmul(a[3], w3);
  if constexpr (R == 4) return;
  a[4] = cmul(a[4], w4);
  a[5] = cmul(a[5], cmul(w4, w1));
  a[6] = cmul(a[6], cmul(w4, w2));
  a[7] = cmul(a[7], cmul(w4, w3));
  if constexpr (R == 16) {
    const float2 w8 = cmul(w4, w4), w12 = cmul(w8, w4);
    a[8] = cmul(a[8], w8);
    a[9] = cmul(a[9], cmul(w8, w1));
    a[10] = cmul(a[10], cmul(w8, w2));
    a[11] = cmul(a[11], cmul(w8, w3));
    a[12] = cmul(a[12], w12);
    a[13] = cmul(a[13], cmul(w12, w1));
    a[14] = cmul(a[14], cmul(w12, w2));
    a[15] = cmul(a[15], cmul(w12, w3));
  }
}

// One Stockham pass of radix R and span NS over the column c of a length-L
// buffer of W columns: this thread's 16 / R butterflies j = b + u L/16 read
// rows j + r L/R (layout IN), barrier, write rows (j - k) R + k + r NS (layout
// OUT), barrier.  tw: this pass's segment (unused for NS = 1).
template <int SIGN, int R, int L, int NS, int IN, int OUT, int W = 2>
__device__ __forceinline__ void pass(float2* Y, int b, int c, const float4* tw) {
  constexpr int NB = 16 / R, LR = L / R, L16 = L / 16;
  float2 v[16];
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int j = b + u * L16;
#pragma unroll
    for (int r = 0; r < R; ++r) v[u * R + r] = Y[el<IN, W>(j + r * LR, c)];
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int j = b + u * L16;
    const int k = j & (NS - 1);
    float2* a = v + u * R;
    if (NS > 1) twiddle<SIGN, R>(a, tw[k]);
    dft_r<SIGN, R>(a);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) Y[el<OUT, W>(base + r * NS, c)] = a[r];
  }
  __syncthreads();
}

// Forward transform of the pair: scaled column samples (s(n - nz/2) x_n / sqrt(nz)
// at row (n - nz/2) mod K), zero-padded to K, e^{+} DFT; the result in layout P8.
// The span-1 pass runs on the loaded samples: butterfly j reads rows
// j + r K/16; rows [K/4, 3K/4) are zero and row j + r K/16 holds sample
// n = j + i K/16 with i = r - 12 (r >= 12) or r + 4 (r < 4).  x: this thread's
// column (NULL: a zero column).  Ends with a barrier.
template <int LOGK>
__device__ __forceinline__ void forward(float2* Y, const float2* x, const float* scale,
                                        const float4* tw) {
  constexpr int K = 1 << LOGK, K16 = K / 16;
  const int c = threadIdx.x & 1, j = threadIdx.x >> 1;
  float2 a[16];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int n = j + i * K16;
    a[i < 4 ? i + 12 : i - 4] = x ? cscale(x[n], __ldg(scale + n)) : make_float2(0.0f, 0.0f);
  }
  dft16<+1, true>(a);
#pragma unroll
  for (int r = 0; r < 16; ++r) Y[el<P16>(16 * j + r, c)] = a[r];
  __syncthreads();
  pass<+1, 16, K, 16, P16, P16>(Y, j, c, tw);
  pass<+1, Passes<LOGK>::R3, K, 256, P16, P8>(Y, j, c, tw + 16);
}

// Inverse transform of the pair from layout P8 (e^{-} DFT): two passes in
// shared memory, the last in registers, handing output row j + i K/16 of this
// thread's column to emit(i, value), i < 16.
template <int LOGK, typename Emit>
__device__ __forceinline__ void inverse(float2* Y, const float4* tw, Emit emit) {
  constexpr int K = 1 << LOGK, K16 = K / 16, R = Passes<LOGK>::R3, NB = 16 / R, LR = K / R;
  const int c = threadIdx.x & 1, j = threadIdx.x >> 1;
  pass<-1, 16, K, 1, P8, P16>(Y, j, c, tw);
  pass<-1, 16, K, 16, P16, P16>(Y, j, c, tw);
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int jj = j + u * K16;          // jj < 256 = NS: k = jj, output rows jj + 256 r
    float2 a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = Y[el<P16>(jj + r * LR, c)];
    twiddle<-1, R>(a, tw[16 + jj]);
    dft_r<-1, R>(a);
#pragma unroll
    for (int r = 0; r < R; ++r) emit(u + r * NB, a[r]);   // row jj + 256 r = j + (u + r NB) K/16
  }
}

// ---------------------------------------------------------------------------
// Lateral transforms of a tile of W = 2 TP columns (k_lat's compile-time
// instances), L = 1024 = 16 * 4 * 16 or 256 = 16 * 16: thread t owns column
// c = t mod W of butterfly j = t / W, the tile's rows in layout P8 before and
// after the transform, P16 between its passes.
// ---------------------------------------------------------------------------
// (span, radix) of the passes and the twiddle segments (span > 1, in pass
// order): L = 1024: (1, 16) (16, 4) (64, 16), segments of 16 and 64 entries;
// the radix-4 pass sits at span 16, where a thread's four butterflies
// j = b + 64 u share k = j mod 16 and so one twiddle entry.  L = 256: (1, 16)
// (16, 16), one segment of 16.
template <int LOGL> struct LatPasses;
template <> struct LatPasses<10> {
  static constexpr int entries = 16 + 64;
};
template <> struct LatPasses<8> {
  static constexpr int entries = 16;
};

template <int LOGL> __device__ __forceinline__ void build_lat_twiddles(float4* tw) {
  for (int e = threadIdx.x; e < LatPasses<LOGL>::entries; e += blockDim.x) {
    const int ns = e < 16 ? 16 : 64, k = e < 16 ? e : e - 16;
    const int R = e < 16 ? (LOGL == 10 ? 4 : 16) : 16;
    float s1, c1, s4, c4;
    sincospif(float(2 * k) / float(ns * R), &s1, &c1);
    sincospif(float(8 * k) / float(ns * R), &s4, &c4);
    tw[e] = make_float4(c1, -s1, c4, -s4);
  }
  __syncthreads();
}

// In-place unnormalised transform (SIGN -1: e^{-}) of the tile's W columns,
// rows in layout P8 before and after.  Every thread of the block calls it;
// it ends with a barrier.
template <int SIGN, int LOGL, int W>
__device__ __forceinline__ void lat_transform(float2* Y, const float4* tw) {
  constexpr int L = 1 << LOGL;
  const int c = threadIdx.x & (W - 1), j = threadIdx.x / W;
  if constexpr (LOGL == 10) {
    pass<SIGN, 16, L, 1, P8, P16, W>(Y, j, c, tw);
    pass<SIGN, 4, L, 16, P16, P16, W>(Y, j, c, tw);
    pass<SIGN, 16, L, 64, P16, P8, W>(Y, j, c, tw + 16);
  } else {
    pass<SIGN, 16, L, 1, P8, P16, W>(Y, j, c, tw);
    pass<SIGN, 16, L, 16, P16, P8, W>(Y, j, c, tw);
  }
}

}  // namespace c16
}  // namespace isam
