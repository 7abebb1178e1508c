// Shared-memory Stockham FFTs of length L = 2^p or 3 * 2^p (p >= 3): radix-8
// passes, one radix-4 or radix-2 pass for the rest of 2^p, and for L = 3 * 2^p
// a final radix-3 pass.  Every participating thread owns eight points per
// power-of-two pass, so a length-L transform of one column takes L/8 threads
// (each takes two or three of the L/3 radix-3 butterflies).  Many
// columns can be transformed together: element r of column c lives at
// buf[r * stride + c]; the caller maps threads to (column, butterfly).
//
// The element type E is a complex number (float2 / double2) or a pair of
// complex numbers (cpair<T>: two columns transformed in lock step with one
// 16- or 32-byte shared-memory access per point).
//
// Direction SIGN = -1 computes X_m = sum_p x_p e^{-2 pi i m p / L},
// SIGN = +1 the same with e^{+...}; no normalisation.  Twiddles come from a
// per-block shared-memory table (build_twiddles).
#pragma once

#include "common.cuh"

namespace isam {

template <typename T> struct alignas(2 * sizeof(cplx<T>)) cpair { cplx<T> a, b; };

// arithmetic on complex numbers and complex pairs
template <typename C> __device__ __forceinline__ C eadd(C a, C b) { return cadd(a, b); }
template <typename C> __device__ __forceinline__ C esub(C a, C b) { return csub(a, b); }
template <typename T> __device__ __forceinline__ cpair<T> eadd(cpair<T> a, cpair<T> b) {
  return {cadd(a.a, b.a), cadd(a.b, b.b)};
}
template <typename T> __device__ __forceinline__ cpair<T> esub(cpair<T> a, cpair<T> b) {
  return {csub(a.a, b.a), csub(a.b, b.b)};
}
template <int SIGN, typename C> __device__ __forceinline__ C emul_i(C a) { return cmul_i<SIGN>(a); }
template <int SIGN, typename T> __device__ __forceinline__ cpair<T> emul_i(cpair<T> a) {
  return {cmul_i<SIGN>(a.a), cmul_i<SIGN>(a.b)};
}
template <typename C> __device__ __forceinline__ C emul(C a, C w) { return cmul(a, w); }
template <typename T> __device__ __forceinline__ cpair<T> emul(cpair<T> a, cplx<T> w) {
  return {cmul(a.a, w), cmul(a.b, w)};
}
template <typename C, typename T> __device__ __forceinline__ C escale(C a, T s) { return cscale(a, s); }
template <typename T> __device__ __forceinline__ cpair<T> escale(cpair<T> a, T s) {
  return {cscale(a.a, s), cscale(a.b, s)};
}
// multiply by h (1 + SIGN i) and by h (-1 + SIGN i), h = 1/sqrt(2)
template <int SIGN, typename C> __device__ __forceinline__ C ew8_1(C o) {
  using T = decltype(o.x);
  const T h = T(0.70710678118654752440);
  C r; r.x = h * (o.x - SIGN * o.y); r.y = h * (o.y + SIGN * o.x); return r;
}
template <int SIGN, typename C> __device__ __forceinline__ C ew8_3(C o) {
  using T = decltype(o.x);
  const T h = T(0.70710678118654752440);
  C r; r.x = h * (-o.x - SIGN * o.y); r.y = h * (-o.y + SIGN * o.x); return r;
}
template <int SIGN, typename T> __device__ __forceinline__ cpair<T> ew8_1(cpair<T> o) {
  return {ew8_1<SIGN>(o.a), ew8_1<SIGN>(o.b)};
}
template <int SIGN, typename T> __device__ __forceinline__ cpair<T> ew8_3(cpair<T> o) {
  return {ew8_3<SIGN>(o.a), ew8_3<SIGN>(o.b)};
}

// t + SIGN i s and t - SIGN i s, lane by lane (no operand swap for the
// packed two-lane adds of the FP32 forms)
template <int SIGN, typename C> __device__ __forceinline__ C add_rot(C t, C s) {
  C r; r.x = t.x - SIGN * s.y; r.y = t.y + SIGN * s.x; return r;
}
template <int SIGN, typename C> __device__ __forceinline__ C sub_rot(C t, C s) {
  C r; r.x = t.x + SIGN * s.y; r.y = t.y - SIGN * s.x; return r;
}
template <int SIGN, typename T> __device__ __forceinline__ cpair<T> add_rot(cpair<T> t, cpair<T> s) {
  return {add_rot<SIGN>(t.a, s.a), add_rot<SIGN>(t.b, s.b)};
}
template <int SIGN, typename T> __device__ __forceinline__ cpair<T> sub_rot(cpair<T> t, cpair<T> s) {
  return {sub_rot<SIGN>(t.a, s.a), sub_rot<SIGN>(t.b, s.b)};
}

template <int SIGN, typename E>
__device__ __forceinline__ void dft2(E& a, E& b) {
  E t = a; a = eadd(t, b); b = esub(t, b);
}

template <int SIGN, typename E>
__device__ __forceinline__ void dft4(E& a0, E& a1, E& a2, E& a3) {
  E t0 = eadd(a0, a2), t1 = esub(a0, a2);
  E t2 = eadd(a1, a3), t3 = esub(a1, a3);
  a0 = eadd(t0, t2); a2 = esub(t0, t2);
  a1 = add_rot<SIGN>(t1, t3); a3 = sub_rot<SIGN>(t1, t3);
}

template <int SIGN, bool HALF_ZERO = false, typename E>
__device__ __forceinline__ void dft8(E* a) {
  if (HALF_ZERO) {
    // a[2..5] == 0: even part (a0, 0, 0, a6), odd part (a1, 0, 0, a7)
    const E e0 = eadd(a[0], a[6]), e2 = esub(a[0], a[6]);
    const E e1 = sub_rot<SIGN>(a[0], a[6]), e3 = add_rot<SIGN>(a[0], a[6]);
    const E o0 = eadd(a[1], a[7]), o2 = esub(a[1], a[7]);
    const E o1 = ew8_1<SIGN>(sub_rot<SIGN>(a[1], a[7]));
    const E o3 = ew8_3<SIGN>(add_rot<SIGN>(a[1], a[7]));
    a[0] = eadd(e0, o0); a[4] = esub(e0, o0);
    a[1] = eadd(e1, o1); a[5] = esub(e1, o1);
    a[2] = add_rot<SIGN>(e2, o2); a[6] = sub_rot<SIGN>(e2, o2);
    a[3] = eadd(e3, o3); a[7] = esub(e3, o3);
    return;
  }
  dft4<SIGN>(a[0], a[2], a[4], a[6]);
  dft4<SIGN>(a[1], a[3], a[5], a[7]);
  // odd half times W8^k, W8 = e^{SIGN 2 pi i / 8}
  a[3] = ew8_1<SIGN>(a[3]);
  a[7] = ew8_3<SIGN>(a[7]);
  // combine: y_k = E_k + W^k O_k, y_{k+4} = E_k - W^k O_k (W^2 = SIGN i)
  E e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  E p0 = a[1], p1 = a[3], p2 = a[5], p3 = a[7];
  a[0] = eadd(e0, p0); a[4] = esub(e0, p0);
  a[1] = eadd(e1, p1); a[5] = esub(e1, p1);
  a[2] = add_rot<SIGN>(e2, p2); a[6] = sub_rot<SIGN>(e2, p2);
  a[3] = eadd(e3, p3); a[7] = esub(e3, p3);
}

// Shared-memory row of logical row r: one padding row after every 8 rows,
// which makes the strided Stockham writes of 8- and 16-byte elements free of
// bank conflicts.  A column of L rows occupies padded_rows(L) rows.
__host__ __device__ __forceinline__ int prow(int r) { return r + (r >> 3); }
__host__ __device__ __forceinline__ int padded_rows(int L) { return L + (L >> 3); }

__device__ __forceinline__ void sincospi_(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_(double x, double* s, double* c) { sincospi(x, s, c); }

// Twiddle table of an L-point transform, in shared memory: for every pass
// with span Ns > 1 and radix R, entry k of that pass's segment holds
// w_k = e^{-2 pi i k / (Ns R)}, k < Ns.  A butterfly raises w_k to the powers
// r = 2 .. R-1 itself by repeated complex multiplication, so each pass reads
// one table entry per butterfly instead of R - 1.
__host__ __device__ __forceinline__ int twiddle_entries(int L, int logL, int r3 = 0) {
  if (L < 8) return 0;
  int n = 0, Ns = 1;
  const int n8 = logL / 3;
  for (int p = 0; p < n8; ++p) {
    if (Ns > 1) n += Ns;
    Ns *= 8;
  }
  const int rem = logL - 3 * n8;
  if (rem && Ns > 1) n += Ns;
  if (rem) Ns <<= rem;
  if (r3) n += Ns;
  return n;
}

// All threads of the block fill the table (ends with a barrier).  logL is
// log2 of the power-of-two factor; r3 = 1 for L = 3 * 2^logL.
template <typename T>
__device__ __forceinline__ void build_twiddles(cplx<T>* tab, int L, int logL, int r3 = 0) {
  if (L >= 8) {
    const int n8 = logL / 3, rem = logL - 3 * n8;
    const int npass = n8 + (rem ? 1 : 0) + r3;
    int off = 0, Ns = 1;
    for (int p = 0; p < npass; ++p) {
      const int R = p < n8 ? 8 : (p == n8 && rem ? (rem == 2 ? 4 : 2) : 3);
      if (Ns > 1) {
        for (int k = threadIdx.x; k < Ns; k += blockDim.x) {
          T s, c;
          sincospi_(T(2 * k) / T(Ns * R), &s, &c);
          tab[off + k] = mk<T>(c, -s);
        }
        off += Ns;
      }
      Ns *= R;
    }
  }
  __syncthreads();
}

// One Stockham pass of radix R on column `col` (logical row r at
// buf[prow(r)*stride+col]); this thread does 8/R butterflies j = b + u * (L/8).
// tw is this pass's twiddle segment.  HALF_ZERO: input rows in [L/4, 3L/4)
// are known zero and not read (first pass of a twice zero-padded transform).
// Reads all its inputs, block barrier, writes.  Every thread must reach it.
template <int SIGN, int R, bool HALF_ZERO, typename T, typename E>
__device__ __forceinline__ void stockham_pass(E* buf, int stride, int col, int b, int L,
                                              int Ns, const cplx<T>* tw, bool active) {
  constexpr int NB = 8 / R;          // butterflies per thread
  const int LR = L / R;
  const int L8 = L >> 3;
  E v[8];
  if (active) {
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int j = b + u * L8;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (HALF_ZERO && R == 8 && r >= 2 && r <= 5) {
          v[u * R + r] = E{};
        } else {
          v[u * R + r] = buf[prow(j + r * LR) * stride + col];
        }
      }
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int j = b + u * L8;
      const int k = j & (Ns - 1);
      E* a = v + u * R;
      if (Ns > 1) {
        cplx<T> w1 = tw[k];
        if (SIGN > 0) w1.y = -w1.y;
        cplx<T> w = w1;
        a[1] = emul(a[1], w);
#pragma unroll
        for (int r = 2; r < R; ++r) {
          w = cmul(w, w1);
          a[r] = emul(a[r], w);
        }
      }
      if (R == 8) dft8<SIGN, HALF_ZERO>(a);
      else if (R == 4) dft4<SIGN>(a[0], a[1], a[2], a[3]);
      else dft2<SIGN>(a[0], a[1]);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[prow(base + r * Ns) * stride + col] = a[r];
    }
  }
  __syncthreads();
}

// Final radix-3 pass of an L = 3 Ns transform (Ns = 2^p, the span reached by
// the power-of-two passes): butterfly j < Ns reads rows j, j + Ns, j + 2 Ns,
// multiplies by w^r (w = e^{SIGN 2 pi i j / (3 Ns)}), takes the 3-point DFT
// and writes rows j, j + Ns, j + 2 Ns.  Thread b takes j = b + u L/8, u < 3.
// Reads all its inputs, block barrier, writes.  Every thread must reach it.
template <int SIGN, typename T, typename E>
__device__ __forceinline__ void stockham_pass3(E* buf, int stride, int col, int b, int L, int Ns,
                                               const cplx<T>* tw, bool active) {
  const int L8 = L >> 3;
  E v[9];
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int j = b + u * L8;
    if (active && j < Ns) {
#pragma unroll
      for (int r = 0; r < 3; ++r) v[3 * u + r] = buf[prow(j + r * Ns) * stride + col];
    }
  }
  __syncthreads();
  const T h = T(0.86602540378443864676);   // sqrt(3)/2
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int j = b + u * L8;
    if (active && j < Ns) {
      cplx<T> w1 = tw[j];
      if (SIGN > 0) w1.y = -w1.y;
      E* a = v + 3 * u;
      a[1] = emul(a[1], w1);
      a[2] = emul(a[2], cmul(w1, w1));
      const E t1 = eadd(a[1], a[2]);
      const E t2 = esub(a[0], escale(t1, T(0.5)));
      const E t3 = escale(emul_i<SIGN>(esub(a[1], a[2])), h);
      buf[prow(j) * stride + col] = eadd(a[0], t1);
      buf[prow(j + Ns) * stride + col] = eadd(t2, t3);
      buf[prow(j + 2 * Ns) * stride + col] = esub(t2, t3);
    }
  }
  __syncthreads();
}

// Length-L transform (L = 2^logL, or 3 * 2^logL when r3, L <= 8192) of column
// `col`, using the twiddle table built by build_twiddles.  For L >= 8 the
// active threads own butterfly b < L/8; for L < 8 the thread with b == 0
// transforms the column directly.  HALF_ZERO: rows [L/4, 3L/4) of the input
// are zero (and need not be stored; powers of two only).  Every thread of the
// block must call it; it ends with a barrier.
template <int SIGN, bool HALF_ZERO, typename T, typename E>
__device__ __forceinline__ void fft_smem(E* buf, int stride, int col, int b, int L, int logL,
                                         const cplx<T>* tw, bool active, int r3 = 0) {
  if (L >= 8) {
    int Ns = 1;
    const int n8 = logL / 3;
    for (int p = 0; p < n8; ++p) {
      if (p == 0 && HALF_ZERO)
        stockham_pass<SIGN, 8, true, T>(buf, stride, col, b, L, Ns, tw, active);
      else
        stockham_pass<SIGN, 8, false, T>(buf, stride, col, b, L, Ns, tw, active);
      if (Ns > 1) tw += Ns;
      Ns *= 8;
    }
    const int rem = logL - 3 * n8;
    if (rem == 2) stockham_pass<SIGN, 4, false, T>(buf, stride, col, b, L, Ns, tw, active);
    else if (rem == 1) stockham_pass<SIGN, 2, false, T>(buf, stride, col, b, L, Ns, tw, active);
    if (rem) {
      if (Ns > 1) tw += Ns;
      Ns <<= rem;
    }
    if (r3) stockham_pass3<SIGN, T>(buf, stride, col, b, L, Ns, tw, active);
  } else {
    __syncthreads();
    if (active && b == 0 && L > 1) {
      E a0 = buf[col], a1 = buf[stride + col];
      if (L == 2) {
        dft2<SIGN>(a0, a1);
      } else {
        E a2 = buf[2 * stride + col], a3 = buf[3 * stride + col];
        dft4<SIGN>(a0, a1, a2, a3);
        buf[2 * stride + col] = a2; buf[3 * stride + col] = a3;
      }
      buf[col] = a0; buf[stride + col] = a1;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Compile-time-length Stockham transforms of column `col` at a compile-time
// stride (element of logical row r at buf[prow(r) * STRIDE + col]), thread b
// < L/8 active on every call.  With L, the stride and the pass span Ns
// constant, the rows a thread reads (j + r L/R) and writes (base + r Ns) lie
// at constant distances in the padded layout whenever the distance is a
// multiple of 8 rows, so each pass computes one padded base row for its reads
// and one for its writes and every access is a fixed offset from them.  Same
// arithmetic, in the same order, as stockham_pass / fft_smem.
// ---------------------------------------------------------------------------

// padded row of logical row r0 + r * STEP, given p0 = prow(r0): with STEP a
// compile-time multiple of 8 it is a fixed offset from p0
template <int STEP>
__device__ __forceinline__ int prow_at(int r0, int p0, int r) {
  if constexpr (STEP % 8 == 0) return p0 + r * (STEP + STEP / 8);
  else return prow(r0 + r * STEP);
}

template <int SIGN, int R, typename T, typename E>
__device__ __forceinline__ void twiddle_powers(E* a, cplx<T> w1) {
  if (SIGN > 0) w1.y = -w1.y;
  cplx<T> w = w1;
  a[1] = emul(a[1], w);
#pragma unroll
  for (int r = 2; r < R; ++r) {
    w = cmul(w, w1);
    a[r] = emul(a[r], w);
  }
}

template <int SIGN, int R, int L, int NS, bool HALF_ZERO, int STRIDE, typename T, typename E>
__device__ __forceinline__ void stockham_pass_ct(E* buf, int col, int b, const cplx<T>* tw) {
  constexpr int NB = 8 / R;          // butterflies per thread
  constexpr int LR = L / R;
  constexpr int L8 = L / 8;
  E v[8];
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int j = b + u * L8;
    const int p0 = prow(j);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (HALF_ZERO && R == 8 && r >= 2 && r <= 5) v[u * R + r] = E{};
      else v[u * R + r] = buf[prow_at<LR>(j, p0, r) * STRIDE + col];
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int j = b + u * L8;
    const int k = j & (NS - 1);
    E* a = v + u * R;
    if (NS > 1) twiddle_powers<SIGN, R, T>(a, tw[k]);
    if (R == 8) dft8<SIGN, HALF_ZERO>(a);
    else if (R == 4) dft4<SIGN>(a[0], a[1], a[2], a[3]);
    else dft2<SIGN>(a[0], a[1]);
    const int base = (j - k) * R + k;
    const int q0 = prow(base);
#pragma unroll
    for (int r = 0; r < R; ++r) buf[prow_at<NS>(base, q0, r) * STRIDE + col] = a[r];
  }
  __syncthreads();
}

// The passes of span NS and up (tw: the segment of span NS).  SKIP_LAST:
// stop before the last pass (last_pass_regs_ct takes it).
template <int SIGN, bool HALF_ZERO, int L, int NS, int STRIDE, typename T, bool SKIP_LAST = false,
          typename E>
__device__ __forceinline__ void fft_passes_ct(E* buf, int col, int b, const cplx<T>* tw) {
  if constexpr (NS * 8 <= L) {
    constexpr bool last = NS * 8 == L;
    if constexpr (!(last && SKIP_LAST))
      stockham_pass_ct<SIGN, 8, L, NS, HALF_ZERO && NS == 1, STRIDE, T>(buf, col, b, tw);
    fft_passes_ct<SIGN, HALF_ZERO, L, NS * 8, STRIDE, T, SKIP_LAST>(buf, col, b,
                                                                    tw + (NS > 1 ? NS : 0));
  } else if constexpr (NS * 4 == L && !SKIP_LAST) {
    stockham_pass_ct<SIGN, 4, L, NS, false, STRIDE, T>(buf, col, b, tw);
  } else if constexpr (NS * 2 == L && !SKIP_LAST) {
    stockham_pass_ct<SIGN, 2, L, NS, false, STRIDE, T>(buf, col, b, tw);
  }
}

// Offset in the twiddle table of the segment of the pass with span ns (a
// power of 8): the segments of the spans 8, 64, ... below it come first.
__host__ __device__ constexpr int tw_offset(int ns) {
  int o = 0;
  for (int s = 8; s < ns; s *= 8) o += s;
  return o;
}

// Register end of a compile-time transform.  Thread b owns the rows
// b + i L/8, i < 8, of its column: in the last pass (span L/R) its butterflies
// j = b + u L/8 read and write rows j + r L/R = b + (u + r 8/R) L/8, so the
// last pass can hand its outputs to global stores without a shared-memory
// round trip.
//
// last_pass_regs_ct: butterfly by butterfly, reads the last pass's inputs
// (the previous pass must have ended with a barrier), computes them and hands
// output row b + i L/8 to emit(i, value); writes no shared memory.
template <int SIGN, int LOGL, int STRIDE, typename T, typename E, typename Emit>
__device__ __forceinline__ void last_pass_regs_ct(const E* buf, int col, int b,
                                                  const cplx<T>* tw_table, Emit emit) {
  constexpr int L = 1 << LOGL, n8 = LOGL / 3, rem = LOGL - 3 * (LOGL / 3);
  constexpr int R = rem == 0 ? 8 : (1 << rem);
  constexpr int NS = L / R, NB = 8 / R, L8 = L / 8;
  const cplx<T>* tw = tw_table + tw_offset(rem == 0 ? (1 << (3 * (n8 - 1))) : (1 << (3 * n8)));
  const int p0 = prow(b);
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    E a[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = buf[prow_at<L8>(b, p0, u + r * NB) * STRIDE + col];
    if (NS > 1) twiddle_powers<SIGN, R, T>(a, tw[(b + u * L8) & (NS - 1)]);
    if (R == 8) dft8<SIGN>(a);
    else if (R == 4) dft4<SIGN>(a[0], a[1], a[2], a[3]);
    else dft2<SIGN>(a[0], a[1]);
#pragma unroll
    for (int r = 0; r < R; ++r) emit(u + r * NB, a[r]);
  }
}

// fft_smem for L = 2^LOGL (LOGL >= 3) and the stride known at compile time;
// thread b < L/8 transforms column col.  Ends with a barrier.
template <int SIGN, bool HALF_ZERO, int LOGL, int STRIDE, typename T, typename E>
__device__ __forceinline__ void fft_cols_ct(E* buf, int col, int b, const cplx<T>* tw) {
  static_assert(LOGL >= 3, "compile-time transforms start at L = 8");
  fft_passes_ct<SIGN, HALF_ZERO, (1 << LOGL), 1, STRIDE, T>(buf, col, b, tw);
}

// one column at stride 1 (the axial kernels: every thread of a block of L/8)
template <int SIGN, bool HALF_ZERO, int LOGL, typename T, typename E>
__device__ __forceinline__ void fft_smem_ct(E* buf, int b, const cplx<T>* tw) {
  fft_cols_ct<SIGN, HALF_ZERO, LOGL, 1, T>(buf, 0, b, tw);
}

}  // namespace isam
