// Axial Stolt-mapped NUFFT kernels.  One thread block per pair of lateral-
// frequency columns (q, -q): both share the Stolt map beta(|q|, k), so the
// positions, phases and interpolation coefficients are computed once and
// applied to two columns whose FFTs run in lock step (16- or 32-byte
// shared-memory elements).
//
//   k_ax_fwd  (§3.2, Eq. 3, 13, 16; min-max NUFFT of Fessler & Sutton):
//     S(q, k_j) = e^{j phi(k_j)} e^{j (2 k_j + beta) z0}
//                 sum_l c_l(f_j) Y[(m0_j + l) mod K],
//     Y = K-point e^{+} DFT of the scaled, zero-padded column
//         s(n - nz/2) eta_hat(q, z_n) / sqrt(nz) placed at (n - nz/2) mod K.
//   k_ax_adj  (Eq. 17, the exact adjoint of k_ax_fwd): every sample adds
//     c_l(f_j) conj(phase_j) R_hat(q, k_j) to bins m0_j + l, race-free without
//     atomics (see scatter_samples), then the K-point e^{-} DFT, truncation
//     and scaling.
//   k_ax_fused  both, with the data residual formed in between.
//
// Stolt positions are evaluated per sample from per-plan constants in
// float-float arithmetic (FP32 path) or double (FP64 path): the grid
// coordinate reaches ~5e4 bins while its fractional part must be right to
// ~1e-7.  Interpolation coefficients are evaluated from their even/odd
// polynomial form (see Poly), held in kernel parameters.
#pragma once

#include <limits.h>

#include "fft_col16.cuh"
#include "fft_smem.cuh"
#include "internal.cuh"

namespace isam {

__device__ __forceinline__ int signed_freq(int i, int n) { return i <= (n - 1) / 2 ? i : i - n; }
static inline int ilog2_dev(int v) { int r = 0; while ((1 << r) < v) ++r; return r; }

template <typename T> struct StoltPos;

// p_j = sqrt(4 kappa_j^2 - a), a = (q/dk)^2, in float-float; the unwrapped
// grid index is p_j - B with B = 2 kappa_0 - c0 (a multiple of K).
template <> struct StoltPos<float> {
  ff a;
  __device__ StoltPos(const StoltConst& c, int mx, int my) {
    a = ff_add(ff_mul_f({c.qx_hi, c.qx_lo}, float(mx * mx)),
               ff_mul_f({c.qy_hi, c.qy_lo}, float(my * my)));
  }
  __device__ __forceinline__ bool at(const StoltConst& c, int j, int& mfl, float& frac,
                                     float& turn) const {
    ff kap = ff_two_sum(c.kap_hi, float(j));            // j is an exact integer
    kap = ff_quick(kap.hi, kap.lo + c.kap_lo);
    ff k2 = ff_mul(kap, kap);
    k2.hi *= 4.0f; k2.lo *= 4.0f;                       // exact
    const ff x = ff_sub(k2, a);
    if (!(x.hi > 0.0f)) return false;
    const ff p = ff_sqrt_fast(x);
    ff t = ff_two_sum(p.hi, -c.B);
    t.lo += p.lo;
    float fl = floorf(t.hi);
    float fr = __fadd_rn(__fsub_rn(t.hi, fl), t.lo);
    if (fr < 0.0f) { fr += 1.0f; fl -= 1.0f; }
    else if (fr >= 1.0f) { fr -= 1.0f; fl += 1.0f; }
    mfl = int(fl);
    frac = fr;
    turn = 0.0f;
    if (c.focus) {                                      // (2 kappa - p) zeta, in turns
      const ff d = ff_sub({2.0f * kap.hi, 2.0f * kap.lo}, p);
      const ff r = ff_mul(d, {c.zeta_hi, c.zeta_lo});
      const float n = rintf(r.hi);
      turn = __fadd_rn(__fsub_rn(r.hi, n), r.lo);
    }
    return true;
  }
};

template <> struct StoltPos<double> {
  double a;
  __device__ StoltPos(const StoltConst& c, int mx, int my) {
    a = c.Qx * double(mx) * double(mx) + c.Qy * double(my) * double(my);
  }
  __device__ __forceinline__ bool at(const StoltConst& c, int j, int& mfl, double& frac,
                                     double& turn) const {
    const double kap = c.kap + double(j);
    const double x = 4.0 * kap * kap - a;
    if (!(x > 0.0)) return false;
    const double p = sqrt(x);
    const double d = a / (2.0 * kap + p);               // 2 kappa - p without cancellation
    const double t = (c.c0d + 2.0 * double(j)) - d;     // = p - B
    const double fl = floor(t);
    frac = t - fl;                                      // exact, in [0, 1)
    mfl = int(fl);
    turn = 0.0;
    if (c.focus) {
      const double r = d * c.zeta;
      turn = r - rint(r);
    }
    return true;
  }
};

__device__ __forceinline__ void sincos_turn(float t, float* s, float* c) { sincospif(2.0f * t, s, c); }
__device__ __forceinline__ void sincos_turn(double t, double* s, double* c) { sincospi(2.0 * t, s, c); }

template <typename T>
__device__ __forceinline__ cplx<T> spectral_phase(const StoltConst& sc, const cplx<T>* disp, int j,
                                                  T turn) {
  cplx<T> ph = __ldg(disp + j);
  if (sc.focus) {
    T s, c;
    sincos_turn(turn, &s, &c);
    ph = cmul(ph, mk<T>(c, s));
  }
  return ph;
}

// Row of the Stolt table (and of the filter table) for lateral frequency
// (mx, my): rows by |mx|, |my|.
__device__ __forceinline__ int stolt_class(const StoltConst& sc, int mx, int my) {
  return abs(my) * (sc.nx / 2 + 1) + abs(mx);
}

// Stolt position and spectral phase of sample j of one column pair, from the
// plan's table when present, else evaluated (float-float / double).
template <typename T> struct Positions {
  StoltPos<T> sp;
  const StoltEntry<T>* row;
  const cplx<T>* frow;       // filter B of this column's |q| class (evaluated path)
  __device__ Positions(const AxArgs<T>& A, int mx, int my) : sp(A.sc, mx, my) {
    const size_t cls = size_t(stolt_class(A.sc, mx, my)) * A.sc.nk;
    row = A.tab.stab ? A.tab.stab + cls : nullptr;
    frow = A.tab.filt ? A.tab.filt + cls : nullptr;
  }
  __device__ __forceinline__ bool at(const AxArgs<T>& A, int j, int& mfl, T& frac,
                                     cplx<T>& ph) const {
    if (row) {
      const StoltEntry<T> e = row[j];
      mfl = e.mfl;
      frac = e.frac;
      ph = e.ph;
      return e.mfl != INT_MIN;
    }
    T turn;
    if (!sp.at(A.sc, j, mfl, frac, turn)) return false;
    ph = spectral_phase<T>(A.sc, A.tab.disp, j, turn);
    if (frow) ph = cmul(ph, __ldg(frow + j));
    return true;
  }
};

// all J coefficients c_l(f)
template <typename T, int J>
__device__ __forceinline__ void coefficients(const Poly<T>& P, T frac, T* c) {
  constexpr int DE = PolyDeg<T>::DE, DO = PolyDeg<T>::DO;
  const T x = frac - T(0.5);
  const T y = T(4) * x * x;
#pragma unroll
  for (int p = 0; p < J / 2; ++p) {
    T e = P.e[p][DE];
#pragma unroll
    for (int k = DE - 1; k >= 0; --k) e = fma(e, y, P.e[p][k]);
    T o = P.o[p][DO];
#pragma unroll
    for (int k = DO - 1; k >= 0; --k) o = fma(o, y, P.o[p][k]);
    c[p] = fma(x, o, e);
    c[J - 1 - p] = fma(-x, o, e);
  }
}

template <typename T>
__device__ __forceinline__ void pair_columns(const AxArgs<T>& A, int& c1, int& c2, int& mx,
                                             int& my) {
  const int2 pr = A.pairs[blockIdx.x];
  c1 = pr.x;
  c2 = pr.y;
  mx = signed_freq(c1 % A.sc.nx, A.sc.nx);
  my = signed_freq(c1 / A.sc.nx, A.sc.ny);
}

// Shared memory of the axial kernels: the FFT buffer Y (padded rows of
// column pairs) followed by the K-point twiddle table.
template <typename T>
__device__ __forceinline__ cplx<T>* twiddle_table(unsigned char* raw, int K) {
  return reinterpret_cast<cplx<T>*>(raw + size_t(padded_rows(K)) * sizeof(cpair<T>));
}

// The forward K-point transform of the block's column pair: the
// compile-time-length Stockham form when LOGK > 0 (K = 2^LOGK, the sizes the
// kernels are instantiated for), else the runtime-length one.  Ends with a
// barrier.  (The inverse is in inverse_and_store.)
template <int LOGK, typename T>
__device__ __forceinline__ void axial_fft_fwd(cpair<T>* Y, int K, int logK, const cplx<T>* tw) {
  if constexpr (LOGK > 0) fft_smem_ct<+1, true, LOGK, T>(Y, threadIdx.x, tw);
  else fft_smem<+1, true, T>(Y, 1, 0, threadIdx.x, K, logK, tw, true);
}

// K and the block size K/8, as compile-time constants when LOGK > 0
template <int LOGK> __device__ __forceinline__ int axial_K(const StoltConst& sc) {
  return LOGK > 0 ? (1 << LOGK) : sc.K;
}
template <int LOGK> __device__ __forceinline__ int axial_threads() {
  return LOGK > 0 ? (1 << LOGK) / 8 : int(blockDim.x);
}

// Y (padded rows) = scaled columns c1 (a) and c2 (b), zero-padded to K, then
// the K-point e^{+} DFT.  The padding rows [nz/2, K - nz/2) are never stored:
// the first FFT pass knows them to be zero.  Ends with a barrier.
template <typename T, int LOGK>
__device__ __forceinline__ void load_and_fft(const AxArgs<T>& A, cpair<T>* Y, const cplx<T>* tw,
                                             int c1, int c2, bool two) {
  using C = cplx<T>;
  using V = cpair<T>;
  const StoltConst& sc = A.sc;
  const int K = axial_K<LOGK>(sc), nz = K / 2;
  const int tid = threadIdx.x, nt = axial_threads<LOGK>();
  const C* x1 = A.in + size_t(c1) * nz;
  const C* x2 = A.in + size_t(c2) * nz;
  // nz = 4 * blockDim: four samples per thread, loads issued before use
  V v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int n = tid + i * nt;
    v[i].a = x1[n];
    v[i].b = two ? x2[n] : mk<T>(0, 0);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int n = tid + i * nt;
    int p = n - nz / 2;
    if (p < 0) p += K;
    Y[prow(p)] = escale(v[i], __ldg(A.tab.scale + n));
  }
  __syncthreads();
  axial_fft_fwd<LOGK, T>(Y, K, sc.logK, tw);
}

// forward interpolation of both columns at sample j (before the phase)
template <typename T, int J>
__device__ __forceinline__ void interp_pair(const cpair<T>* Y, int K, int mfl, const T* c,
                                            cplx<T>& a1, cplx<T>& a2) {
  const int m0 = mfl - J / 2 + 1;
  a1 = mk<T>(0, 0);
  a2 = mk<T>(0, 0);
#pragma unroll
  for (int l = 0; l < J; ++l) {
    const cpair<T> y = Y[prow((m0 + l) & (K - 1))];
    a1 = cfma_r(c[l], y.a, a1);
    a2 = cfma_r(c[l], y.b, a2);
  }
}

// Adjoint interpolation in scatter form.  Thread t owns samples
// j = NRES t + rho (rho < NRES; nk <= K/2 = NRES * blockDim).  Stolt
// positions rise by at least two bins per sample (dp/dj = 4 kappa / p >= 2),
// so samples of one residue class rho lie >= 2 NRES >= J bins apart and
// their J-bin neighbourhoods are disjoint: in phase rho every thread adds
// its sample's J contributions to Y without atomics.  Phases are further
// split into chunks of K/2 unwrapped bins (chunk = floor(mfl / (K/2))) so
// that the wrap mod K never folds two neighbourhoods of one phase together.
// Each bin receives at most ceil(J/2) + 1 contributions per chunk, summed in
// a fixed order with fused multiply-adds.
constexpr int NRES = 4;

template <typename T> struct Sample {
  cpair<T> val;   // conj(phase) R of both columns
  T frac;         // fractional Stolt offset
  int mfl;        // unwrapped floor of the Stolt position
  int chunk;      // INT_MIN: evanescent (no contribution)
};

// Zero Y, find the block's range of Stolt positions (shared atomics on
// *lo, *hi, initialised by the caller before an earlier barrier) and assign
// every sample to a chunk of width K - J of unwrapped positions: within a
// chunk the J-bin neighbourhoods span fewer than K bins, so they never meet
// again after the wrap mod K.  Returns the number of chunks.
//
// warp_tail: there are two chunks and every chunk-1 sample belongs to the
// block's last warp.  Stolt positions rise with j (samples below the
// evanescent cut-off come first) and warp w owns samples
// [32 NRES w, 32 NRES (w + 1)), so this holds when the last sample of the
// warp before it, j* = NRES (nt - 32) - 1 (thread nt - 33), exists (j* < nk)
// and is in chunk 0 or evanescent.  Its position goes through *tail
// (INT_MAX: j* >= nk, INT_MIN: evanescent).
template <typename T, int J>
__device__ __forceinline__ int prepare_scatter(cpair<T>* Y, int K, int nt, int nk, Sample<T>* sm,
                                               int* lo, int* hi, int* tail, bool& warp_tail) {
  const cpair<T> zero = {mk<T>(0, 0), mk<T>(0, 0)};
  for (int i = threadIdx.x; i < K; i += nt) Y[prow(i)] = zero;
  int l = INT_MAX, h = INT_MIN;
#pragma unroll
  for (int rho = 0; rho < NRES; ++rho)
    if (sm[rho].chunk != INT_MIN) {
      l = min(l, sm[rho].mfl);
      h = max(h, sm[rho].mfl);
    }
  if (l != INT_MAX) {
    atomicMin(lo, l);
    atomicMax(hi, h);
  }
  if (int(threadIdx.x) == nt - 33)
    *tail = NRES * (nt - 32) - 1 >= nk ? INT_MAX
            : (sm[NRES - 1].chunk != INT_MIN ? sm[NRES - 1].mfl : INT_MIN);
  __syncthreads();
  const int base = *lo, width = K - J;
  warp_tail = false;
  if (base == INT_MAX) return 0;
#pragma unroll
  for (int rho = 0; rho < NRES; ++rho)
    if (sm[rho].chunk != INT_MIN) {
      int c = 0, d = sm[rho].mfl - base;
      while (d >= width) { d -= width; ++c; }
      sm[rho].chunk = c;
    }
  int n = 1;
  for (int d = *hi - base; d >= width; d -= width) ++n;
  const int t = *tail;
  warp_tail = n == 2 && nt >= 64 && t != INT_MAX && (t == INT_MIN || t - base < width);
  return n;
}

// the J contributions of one sample
template <typename T, int J>
__device__ __forceinline__ void add_sample(const AxArgs<T>& A, cpair<T>* Y, int K,
                                           const Sample<T>& sm) {
  using V = cpair<T>;
  T c[J];
  coefficients<T, J>(A.poly, sm.frac, c);
  const int m0 = sm.mfl - J / 2 + 1;
  const V v = sm.val;
#pragma unroll
  for (int l = 0; l < J; ++l) {
    const int bi = prow((m0 + l) & (K - 1));
    V y = Y[bi];
    y.a = cfma_r(c[l], v.a, y.a);
    y.b = cfma_r(c[l], v.b, y.b);
    Y[bi] = y;
  }
}

// Y must be zero; every thread adds its samples' J contributions, residue
// class by residue class and chunk by chunk (see the comment above NRES),
// each phase closed by a block barrier.  With warp_tail the last chunk's
// phases involve the last warp only and are closed by warp barriers, then one
// block barrier: the same phases in the same order, so the same sums.
template <typename T, int J>
__device__ __forceinline__ void scatter_samples(const AxArgs<T>& A, cpair<T>* Y, int K, int nt,
                                                const Sample<T>* sm, int nchunks, bool warp_tail) {
  const int block_chunks = warp_tail ? 1 : nchunks;
  for (int ch = 0; ch < block_chunks; ++ch) {
#pragma unroll
    for (int rho = 0; rho < NRES; ++rho) {
      if (sm[rho].chunk == ch) add_sample<T, J>(A, Y, K, sm[rho]);
      __syncthreads();
    }
  }
  if (warp_tail) {
    if ((int(threadIdx.x) >> 5) == (nt >> 5) - 1) {
#pragma unroll
      for (int rho = 0; rho < NRES; ++rho) {
        if (sm[rho].chunk == 1) add_sample<T, J>(A, Y, K, sm[rho]);
        __syncwarp();
      }
    }
    __syncthreads();
  }
}

// Sample n of both output columns: G = s y, or, when the kernel writes the
// lateral spectrum of u = eta^k - g/L, u_hat = eta_hat - G/L with eta_hat the
// kernel's own input (A.in, re-read here: the same samples the block loaded).
template <typename T>
__device__ __forceinline__ void put_output(const AxArgs<T>& A, cplx<T>* o1, cplx<T>* o2, int n,
                                           const cpair<T>& y, T s, int c1, int c2, bool two) {
  const int nz = A.sc.nz;
  if (A.u_hat_scale != T(0)) {
    const T f = s * A.u_hat_scale;
    o1[n] = csub(A.in[size_t(c1) * nz + n], cscale(y.a, f));
    if (two) o2[n] = csub(A.in[size_t(c2) * nz + n], cscale(y.b, f));
  } else {
    o1[n] = cscale(y.a, s);
    if (two) o2[n] = cscale(y.b, s);
  }
}

// Sample n of one output column (column index col of the plan's layout): the
// single-column form of put_output.
template <typename T>
__device__ __forceinline__ void put_output1(const AxArgs<T>& A, cplx<T>* o, int col, int n,
                                            const cplx<T>& y, T s) {
  if (A.u_hat_scale != T(0))
    o[n] = csub(A.in[size_t(col) * A.sc.nz + n], cscale(y, s * A.u_hat_scale));
  else
    o[n] = cscale(y, s);
}

// Y (after the e^{-} DFT): truncate to the nz samples, scale, store columns.
template <typename T, int LOGK>
__device__ __forceinline__ void store_columns(const AxArgs<T>& A, const cpair<T>* Y, int c1,
                                              int c2, bool two) {
  using C = cplx<T>;
  const int K = axial_K<LOGK>(A.sc), nz = K / 2, nt = axial_threads<LOGK>();
  C* o1 = A.out + size_t(c1) * nz;
  C* o2 = A.out + size_t(c2) * nz;
  for (int n = threadIdx.x; n < nz; n += nt) {
    int p = n - nz / 2;
    if (p < 0) p += K;
    const T s = __ldg(A.tab.scale + n);
    const cpair<T> y = Y[prow(p)];
    put_output(A, o1, o2, n, y, s, c1, c2, two);
  }
}

// The inverse transform of Y and store_columns.  Compile-time K: the last
// pass runs in registers and writes the kept rows straight to the columns
// (the rows thread b's last-pass butterfly produces, b + i K/8, are rows it
// stores: natural row p goes to sample n = p + nz/2 for p < nz/2 and
// p - (K - nz/2) for p >= K - nz/2, nz = K/2; the others are dropped).
template <typename T, int LOGK>
__device__ __forceinline__ void inverse_and_store(const AxArgs<T>& A, cpair<T>* Y,
                                                  const cplx<T>* tw, int c1, int c2, bool two) {
  if constexpr (LOGK > 0) {
    using C = cplx<T>;
    constexpr int K = 1 << LOGK, nz = K / 2, K8 = K / 8;
    const int b = threadIdx.x;
    fft_passes_ct<-1, false, K, 1, 1, T, true>(Y, 0, b, tw);
    C* o1 = A.out + size_t(c1) * nz;
    C* o2 = A.out + size_t(c2) * nz;
    last_pass_regs_ct<-1, LOGK, 1, T>(Y, 0, b, tw, [&](int i, const cpair<T>& y) {
      const int p = b + i * K8;
      if (i * K8 >= K / 4 && (i + 1) * K8 <= 3 * K / 4) return;   // rows [K/4, 3K/4)
      const int n = p < K / 4 ? p + nz / 2 : p - (K - nz / 2);
      put_output(A, o1, o2, n, y, __ldg(A.tab.scale + n), c1, c2, two);
    });
  } else {
    fft_smem<-1, false, T>(Y, 1, 0, threadIdx.x, A.sc.K, A.sc.logK, tw, true);
    store_columns<T, LOGK>(A, Y, c1, c2, two);
  }
}

// FP32 plans at K = 2048 and 4096 can take the column-split radix-16
// transforms (fft_col16.cuh): three shared-memory passes per transform instead
// of four, the same threads and registers; the forward ends, and the inverse
// starts, in the layout of the interpolation and the scatter.  C16 selects
// them (the plan's choice, AxArgs::radix16); other instances ignore it.
template <typename T, int LOGK> __host__ __device__ constexpr bool ax_col16_exists() {
  return std::is_same<T, float>::value && LOGK >= 11;
}
template <typename T, int LOGK, bool C16> __host__ __device__ constexpr bool ax_col16() {
  return C16 && ax_col16_exists<T, LOGK>();
}

template <typename T, int LOGK, bool C16>
__device__ __forceinline__ void ax_twiddles(cplx<T>* tw, const StoltConst& sc) {
  if constexpr (ax_col16<T, LOGK, C16>()) c16::build_twiddles<LOGK>(reinterpret_cast<float4*>(tw));
  else build_twiddles<T>(tw, axial_K<LOGK>(sc), sc.logK);
}

// Y = the K-point e^{+} DFT of the pair's scaled, zero-padded columns
template <typename T, int LOGK, bool C16>
__device__ __forceinline__ void ax_forward(const AxArgs<T>& A, cpair<T>* Y, const cplx<T>* tw,
                                           int c1, int c2, bool two) {
  if constexpr (ax_col16<T, LOGK, C16>()) {
    constexpr int nz = (1 << LOGK) / 2;
    const int c = threadIdx.x & 1;
    const cplx<T>* x = c == 0 ? A.in + size_t(c1) * nz : (two ? A.in + size_t(c2) * nz : nullptr);
    c16::forward<LOGK>(reinterpret_cast<float2*>(Y), reinterpret_cast<const float2*>(x),
                       reinterpret_cast<const float*>(A.tab.scale),
                       reinterpret_cast<const float4*>(tw));
  } else {
    load_and_fft<T, LOGK>(A, Y, tw, c1, c2, two);
  }
}

// The e^{-} DFT of Y, truncation to the nz kept rows, scaling, the columns'
// output (G, or u_hat = eta_hat - G/L)
template <typename T, int LOGK, bool C16>
__device__ __forceinline__ void ax_inverse(const AxArgs<T>& A, cpair<T>* Y, const cplx<T>* tw,
                                           int c1, int c2, bool two) {
  if constexpr (ax_col16<T, LOGK, C16>()) {
    // rows j + i K/16 of this thread's column; rows [K/4, 3K/4) are dropped
    constexpr int K = 1 << LOGK, nz = K / 2, K16 = K / 16;
    const int c = threadIdx.x & 1, jb = threadIdx.x >> 1;
    const int col = c ? c2 : c1;
    cplx<T>* o = A.out + size_t(col) * nz;
    const bool keep = c == 0 || two;
    c16::inverse<LOGK>(reinterpret_cast<float2*>(Y), reinterpret_cast<const float4*>(tw),
                       [&](int i, const float2& y) {
                         if (!keep || (i >= 4 && i < 12)) return;
                         const int p = jb + i * K16;
                         const int n = i < 4 ? p + nz / 2 : p - (K - nz / 2);
                         put_output1(A, o, col, n, reinterpret_cast<const cplx<T>&>(y),
                                     __ldg(A.tab.scale + n));
                       });
  } else {
    inverse_and_store<T, LOGK>(A, Y, tw, c1, c2, two);
  }
}

template <typename T, int J, int LOGK, bool C16>
__global__ void __launch_bounds__(512) k_ax_fwd(const __grid_constant__ AxArgs<T> A) {
  using C = cplx<T>;
  using V = cpair<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const StoltConst& sc = A.sc;
  const int K = axial_K<LOGK>(sc), nk = sc.nk;
  V* Y = reinterpret_cast<V*>(smem_raw);
  cplx<T>* tw = twiddle_table<T>(smem_raw, K);
  int c1, c2, mx, my;
  pair_columns(A, c1, c2, mx, my);
  const bool two = c2 != c1;
  // programmatic dependent launch (as k_ax_fused): twiddles before the wait
  cudaTriggerProgrammaticLaunchCompletion();
  ax_twiddles<T, LOGK, C16>(tw, sc);
  cudaGridDependencySynchronize();
  ax_forward<T, LOGK, C16>(A, Y, tw, c1, c2, two);

  const Positions<T> pos(A, mx, my);
  C* o1 = A.out + size_t(c1) * nk;
  C* o2 = A.out + size_t(c2) * nk;
  for (int j = threadIdx.x; j < nk; j += axial_threads<LOGK>()) {
    int mfl;
    T frac;
    C ph;
    C a1 = mk<T>(0, 0), a2 = mk<T>(0, 0);
    if (pos.at(A, j, mfl, frac, ph)) {
      T c[J];
      coefficients<T, J>(A.poly, frac, c);
      interp_pair<T, J>(Y, K, mfl, c, a1, a2);
      a1 = cmul(a1, ph);
      a2 = cmul(a2, ph);
    }
    o1[j] = a1;
    if (two) o2[j] = a2;
  }
}

template <typename T, int J, int LOGK, bool C16>
__global__ void __launch_bounds__(512, 2) k_ax_adj(const __grid_constant__ AxArgs<T> A) {
  using C = cplx<T>;
  using V = cpair<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const StoltConst& sc = A.sc;
  const int K = axial_K<LOGK>(sc), nk = sc.nk;
  V* Y = reinterpret_cast<V*>(smem_raw);
  cplx<T>* tw = twiddle_table<T>(smem_raw, K);
  __shared__ int ch_lo, ch_hi, ch_tail;
  const int tid = threadIdx.x, nt = axial_threads<LOGK>();
  int c1, c2, mx, my;
  pair_columns(A, c1, c2, mx, my);
  const bool two = c2 != c1;
  if (tid == 0) { ch_lo = INT_MAX; ch_hi = INT_MIN; }
  // programmatic dependent launch (as k_ax_fused): twiddles before the wait
  cudaTriggerProgrammaticLaunchCompletion();
  ax_twiddles<T, LOGK, C16>(tw, sc);
  cudaGridDependencySynchronize();
  const Positions<T> pos(A, mx, my);
  const C* r1 = A.in + size_t(c1) * nk;
  const C* r2 = A.in + size_t(c2) * nk;
  Sample<T> sm[NRES];
#pragma unroll
  for (int rho = 0; rho < NRES; ++rho) {
    const int j = NRES * tid + rho;
    sm[rho].chunk = INT_MIN;
    int mfl;
    T frac;
    C ph;
    if (j < nk && pos.at(A, j, mfl, frac, ph)) {
      sm[rho].val.a = cmulc(r1[j], ph);
      sm[rho].val.b = two ? cmulc(r2[j], ph) : mk<T>(0, 0);
      sm[rho].frac = frac;
      sm[rho].mfl = mfl;
      sm[rho].chunk = 0;
    }
  }
  bool warp_tail;
  const int nch = prepare_scatter<T, J>(Y, K, nt, nk, sm, &ch_lo, &ch_hi, &ch_tail, warp_tail);
  scatter_samples<T, J>(A, Y, K, nt, sm, nch, warp_tail);
  ax_inverse<T, LOGK, C16>(A, Y, tw, c1, c2, two);
}

// Forward model, data residual and adjoint of one column pair in one pass
// (Alg. 1 gradient):  S = phase . N(eta_hat);  the lateral spectrum of the
// real residual Re(F^{-1} S) - s_d is, column by column,
//   R(q) = (S(q) + conj(S(-q))) / 2 - F s_d (q),
// because F(Re v)(q) = (F v(q) + conj(F v(-q))) / 2 and q, -q are the two
// columns of the pair; then G = N'(conj(phase) R), written as is or, when
// u_hat_scale = 1/L, as u_hat = eta_hat - G/L (put_output).  F s_d is
// Hermitian, so only its c1 column is read.
// WS: also write the model spectra S to A.s_out.
template <typename T, int J, int LOGK, bool WS, bool C16>
__global__ void __launch_bounds__(512, 2) k_ax_fused(const __grid_constant__ AxArgs<T> A) {
  using C = cplx<T>;
  using V = cpair<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const StoltConst& sc = A.sc;
  const int K = axial_K<LOGK>(sc), nk = sc.nk;
  V* Y = reinterpret_cast<V*>(smem_raw);
  cplx<T>* tw = twiddle_table<T>(smem_raw, K);
  __shared__ int ch_lo, ch_hi, ch_tail;
  const int tid = threadIdx.x, nt = axial_threads<LOGK>();
  int c1, c2, mx, my;
  pair_columns(A, c1, c2, mx, my);
  const bool two = c2 != c1;
  if (tid == 0) { ch_lo = INT_MAX; ch_hi = INT_MIN; }
  constexpr bool COL16 = ax_col16<T, LOGK, C16>();
  // Programmatic dependent launch: the next kernel in the stream may start its
  // own prologue on SMs this grid leaves idle; this grid builds its twiddles,
  // then waits for the previous kernel before touching global data.
  cudaTriggerProgrammaticLaunchCompletion();
  ax_twiddles<T, LOGK, C16>(tw, sc);
  cudaGridDependencySynchronize();
  // the solve's stop flag (written by an earlier kernel, so visible after the
  // wait): loaded here, tested after the forward transform (before the first
  // global write), so its latency overlaps the transform
  const bool stopped = A.stop != nullptr && __ldcg(A.stop) != 0;
  // F s_d at this pair's samples, fetched before the transforms need them (the
  // column-split transforms take them after the forward transform: their
  // registers are needed there)
  const C* d1 = A.sdh + size_t(c1) * nk;
  C dqv[NRES];
  if constexpr (!COL16) {
#pragma unroll
    for (int rho = 0; rho < NRES; ++rho) {
      const int j = NRES * tid + rho;
      dqv[rho] = j < nk ? d1[j] : mk<T>(0, 0);
    }
  }
  ax_forward<T, LOGK, C16>(A, Y, tw, c1, c2, two);
  if (stopped) return;   // an earlier check stopped the solve: write nothing
  if constexpr (COL16) {
#pragma unroll
    for (int rho = 0; rho < NRES; ++rho) {
      const int j = NRES * tid + rho;
      dqv[rho] = j < nk ? d1[j] : mk<T>(0, 0);
    }
  }

  const Positions<T> pos(A, mx, my);
  Sample<T> sm[NRES];
#pragma unroll
  for (int rho = 0; rho < NRES; ++rho) {
    const int j = NRES * tid + rho;
    sm[rho].chunk = INT_MIN;
    if (j >= nk) continue;
    const C dq = dqv[rho];
    int mfl;
    T frac;
    C s1 = mk<T>(0, 0), s2 = mk<T>(0, 0), ph = mk<T>(0, 0);
    const bool prop = pos.at(A, j, mfl, frac, ph);
    if (prop) {
      T c[J];
      coefficients<T, J>(A.poly, frac, c);
      interp_pair<T, J>(Y, K, mfl, c, s1, s2);
      s1 = cmul(s1, ph);
      s2 = two ? cmul(s2, ph) : s1;
    }
    if (WS) {
      A.s_out[size_t(c1) * nk + j] = s1;
      if (two) A.s_out[size_t(c2) * nk + j] = s2;
    }
    const C R1 = csub(cscale(cadd(s1, cconj(s2)), T(0.5)), dq);
    const C R2 = csub(cscale(cadd(s2, cconj(s1)), T(0.5)), cconj(dq));   // F s_d(-q)
    if (prop) {
      sm[rho].val.a = cmulc(R1, ph);
      sm[rho].val.b = two ? cmulc(R2, ph) : mk<T>(0, 0);
      sm[rho].frac = frac;
      sm[rho].mfl = mfl;
      sm[rho].chunk = 0;
    }
  }
  __syncthreads();                       // all reads of Y are done
  bool warp_tail;
  const int nch = prepare_scatter<T, J>(Y, K, nt, nk, sm, &ch_lo, &ch_hi, &ch_tail, warp_tail);
  scatter_samples<T, J>(A, Y, K, nt, sm, nch, warp_tail);
  ax_inverse<T, LOGK, C16>(A, Y, tw, c1, c2, two);
}

// One thread per (|q| class, k_j): the same evaluation the kernels do on the fly.
template <typename T>
__global__ void k_stolt_table(const __grid_constant__ AxArgs<T> A, StoltEntry<T>* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int cls = blockIdx.y;
  if (j >= A.sc.nk) return;
  const int ncx = A.sc.nx / 2 + 1;
  const int mx = cls % ncx, my = cls / ncx;
  const StoltPos<T> sp(A.sc, mx, my);
  StoltEntry<T> e{};
  T turn;
  if (sp.at(A.sc, j, e.mfl, e.frac, turn)) {
    e.ph = spectral_phase<T>(A.sc, A.tab.disp, j, turn);
    if (A.tab.filt) e.ph = cmul(e.ph, A.tab.filt[size_t(cls) * A.sc.nk + j]);
  } else {
    e.mfl = INT_MIN;
    e.frac = T(0);
    e.ph = mk<T>(0, 0);
  }
  out[size_t(cls) * A.sc.nk + j] = e;
}

template <typename T> cudaError_t launch_stolt_table(const AxArgs<T>& a, StoltEntry<T>* out,
                                                     cudaStream_t s) {
  const int rows = (a.sc.ny / 2 + 1) * (a.sc.nx / 2 + 1);
  dim3 grid((a.sc.nk + 255) / 256, rows);
  AxArgs<T> b = a;
  b.tab.stab = nullptr;
  k_stolt_table<T><<<grid, 256, 0, s>>>(b, out);
  return cudaGetLastError();
}

template <typename T> size_t ax_smem_bytes(int K, int nk, bool adj) {
  (void)nk;
  (void)adj;
  return size_t(padded_rows(K)) * sizeof(cpair<T>) +
         size_t(twiddle_entries(K, ilog2_dev(K))) * sizeof(cplx<T>);
}

enum { AX_FWD = 0, AX_ADJ = 1, AX_FUSED = 2 };

template <typename T, int J, int LOGK, bool C16>
static cudaError_t launch_ax_JKC(const AxArgs<T>& a, int npairs, cudaStream_t s, int kind) {
  const int K = a.sc.K;
  const int threads = K / 8;
  const size_t sm = ax_smem_bytes<T>(K, a.sc.nk, kind != AX_FWD);
  void (*kern)(AxArgs<T>);
  if (kind == AX_ADJ) kern = k_ax_adj<T, J, LOGK, C16>;
  else if (kind == AX_FWD) kern = k_ax_fwd<T, J, LOGK, C16>;
  else kern = a.s_out ? k_ax_fused<T, J, LOGK, true, C16> : k_ax_fused<T, J, LOGK, false, C16>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  // programmatic dependent launch: each axial kernel builds its twiddles while
  // the previous kernel finishes, then waits for it (cudaGridDependencySynchronize)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(npairs);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

// the plan's radix choice (a.radix16) where both forms exist
template <typename T, int J, int LOGK>
static cudaError_t launch_ax_JK(const AxArgs<T>& a, int npairs, cudaStream_t s, int kind) {
  if constexpr (ax_col16_exists<T, LOGK>()) {
    if (a.radix16) return launch_ax_JKC<T, J, LOGK, true>(a, npairs, s, kind);
  }
  return launch_ax_JKC<T, J, LOGK, false>(a, npairs, s, kind);
}

// K = 4096 and 2048 (nz = 2048, 1024) run the compile-time-length instances
template <typename T, int J>
static cudaError_t launch_ax_J(const AxArgs<T>& a, int npairs, cudaStream_t s, int kind) {
  switch (a.sc.K) {
    case 4096: return launch_ax_JK<T, J, 12>(a, npairs, s, kind);
    case 2048: return launch_ax_JK<T, J, 11>(a, npairs, s, kind);
  }
  return launch_ax_JK<T, J, 0>(a, npairs, s, kind);
}

template <typename T>
static cudaError_t launch_ax(const AxArgs<T>& a, int npairs, cudaStream_t s, int kind) {
  switch (a.sc.J) {
    case 4: return launch_ax_J<T, 4>(a, npairs, s, kind);
    case 6: return launch_ax_J<T, 6>(a, npairs, s, kind);
    case 8: return launch_ax_J<T, 8>(a, npairs, s, kind);
  }
  return cudaErrorInvalidValue;
}

template <typename T> cudaError_t launch_ax_fwd(const AxArgs<T>& a, int npairs, cudaStream_t s) {
  return launch_ax<T>(a, npairs, s, AX_FWD);
}
template <typename T> cudaError_t launch_ax_adj(const AxArgs<T>& a, int npairs, cudaStream_t s) {
  return launch_ax<T>(a, npairs, s, AX_ADJ);
}
template <typename T> cudaError_t launch_ax_fused(const AxArgs<T>& a, int npairs,
                                                  cudaStream_t s) {
  return launch_ax<T>(a, npairs, s, AX_FUSED);
}

}  // namespace isam
