// Axial Stolt-mapped NUFFT kernels: one thread block per lateral-frequency
// column (q_x, q_y).
//
//   k_ax_fwd  (§3.2, Eq. 3, 13, 16; min-max NUFFT of Fessler & Sutton):
//     S(q, k_j) = e^{j phi(k_j)} e^{j (2 k_j + beta) z0}
//                 sum_l c_l(f_j) Y[(m0_j + l) mod K],
//     Y = K-point e^{+} DFT of the scaled, zero-padded column
//         s(n - nz/2) eta_hat(q, z_n) / sqrt(nz) placed at (n - nz/2) mod K.
//   k_ax_adj  (Eq. 17, the exact adjoint of k_ax_fwd): gathers
//     conj(phase_j) R_hat(q, k_j) c_l(f_j) into bins m0_j + l with compensated
//     (TwoSum) accumulation, K-point e^{-} DFT, truncation to the nz samples,
//     scaling.  The scatter is made race-free without atomics: Stolt positions
//     rise by at least two grid bins per k sample (dp/dj = 4 kappa / p >= 2),
//     so samples j with the same residue mod J/2 touch disjoint bins; samples
//     are processed residue class by residue class, in chunks of K/2 bins so
//     that the wrap mod K never folds two contributions onto one bin.
//
// Stolt positions are computed per sample from per-plan constants in
// float-float arithmetic (FP32 path) or double (FP64 path): the grid
// coordinate reaches ~5e4 bins while its fractional part must be right to
// ~1e-7, beyond single precision.
#include "fft_smem.cuh"
#include "internal.cuh"

namespace isam {

__device__ __forceinline__ int signed_freq(int i, int n) { return i <= (n - 1) / 2 ? i : i - n; }

template <typename T> struct StoltPos;

template <> struct StoltPos<float> {
  ff a;   // (q / dk)^2
  __device__ StoltPos(const StoltConst& c, int mx, int my) {
    a = ff_add(ff_mul_f({c.qx_hi, c.qx_lo}, float(mx * mx)),
               ff_mul_f({c.qy_hi, c.qy_lo}, float(my * my)));
  }
  // position of sample j: floor (unwrapped, integer) and fraction; focus turn
  __device__ __forceinline__ bool at(const StoltConst& c, int j, int& mfl, float& frac,
                                     float& turn) const {
    ff kap = ff_add({c.kap_hi, c.kap_lo}, {float(j), 0.0f});
    ff x = ff_sub(ff_mul_f(ff_mul(kap, kap), 4.0f), a);
    if (!(x.hi > 0.0f)) return false;
    ff p = ff_sqrt(x);
    ff D = ff_add(ff_mul_f(kap, 2.0f), p);
    ff d = ff_div(a, D);
    ff t = ff_sub({c.f0, 0.0f}, d);
    float fl = floorf(t.hi);
    float fr = __fadd_rn(__fsub_rn(t.hi, fl), t.lo);
    if (fr < 0.0f) { fr += 1.0f; fl -= 1.0f; }
    else if (fr >= 1.0f) { fr -= 1.0f; fl += 1.0f; }
    mfl = c.I0 + 2 * j + int(fl);
    frac = fr;
    turn = 0.0f;
    if (c.focus) {
      ff r = ff_mul(d, {c.zeta_hi, c.zeta_lo});
      float n = rintf(r.hi);
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
    double kap = c.kap + double(j);
    double x = 4.0 * kap * kap - a;
    if (!(x > 0.0)) return false;
    double p = sqrt(x);
    double d = a / (2.0 * kap + p);
    double t = (c.c0d - double(c.I0)) - d;
    double fl = floor(t);
    frac = t - fl;
    if (frac >= 1.0) { frac -= 1.0; fl += 1.0; }
    mfl = c.I0 + 2 * j + int(fl);
    turn = 0.0;
    if (c.focus) {
      double r = d * c.zeta;
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

// interpolation coefficients c_l(f) by linear interpolation of the table
template <typename T, int J>
__device__ __forceinline__ void coefficients(const T* __restrict__ tab, T frac, T* c) {
  T x = frac * T(TABLE_D);
  int i = min(int(x), TABLE_D - 1);
  T w = x - T(i);
  const T* row = tab + i * (2 * J);
#pragma unroll
  for (int l = 0; l < J; ++l) c[l] = fma(w, row[J + l], row[l]);
}

template <typename T, int J>
__global__ void __launch_bounds__(512) k_ax_fwd(AxArgs<T> A) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const StoltConst& sc = A.sc;
  const int K = sc.K, nz = sc.nz, nk = sc.nk;
  C* Y = reinterpret_cast<C*>(smem_raw);
  T* tab = reinterpret_cast<T*>(Y + K);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int col = blockIdx.x;

  for (int i = tid; i < (TABLE_D + 1) * 2 * J; i += nt) tab[i] = __ldg(A.tab.coef + i);
  // zero the padding: bins nz/2 .. K - nz/2 - 1
  for (int i = nz / 2 + tid; i < K - nz / 2; i += nt) Y[i] = mk<T>(0, 0);
  const C* x = A.in + size_t(col) * nz;
  for (int n = tid; n < nz; n += nt) {
    int p = n - nz / 2;
    if (p < 0) p += K;
    Y[p] = cscale(x[n], __ldg(A.tab.scale + n));
  }
  __syncthreads();
  fft_smem<+1, T>(Y, 1, 0, tid, K, sc.logK, A.tab.tw_K, true);

  const int ix = col % sc.nx, iy = col / sc.nx;
  StoltPos<T> sp(sc, signed_freq(ix, sc.nx), signed_freq(iy, sc.ny));
  C* out = A.out + size_t(col) * nk;
  for (int j = tid; j < nk; j += nt) {
    int mfl;
    T frac, turn;
    C acc = mk<T>(0, 0);
    if (sp.at(sc, j, mfl, frac, turn)) {
      T c[J];
      coefficients<T, J>(tab, frac, c);
      const int m0 = mfl - J / 2 + 1;
#pragma unroll
      for (int l = 0; l < J; ++l) {
        C y = Y[(m0 + l) & (K - 1)];
        acc.x = fma(c[l], y.x, acc.x);
        acc.y = fma(c[l], y.y, acc.y);
      }
      acc = cmul(acc, spectral_phase<T>(sc, A.tab.disp, j, turn));
    }
    out[j] = acc;
  }
}

// TwoSum-compensated add of v into (sum, comp)
template <typename T>
__device__ __forceinline__ void comp_add(T& sum, T& comp, T v) {
  T s = sum + v;
  T bb = s - sum;
  T err = (sum - (s - bb)) + (v - bb);
  sum = s;
  comp += err;
}

constexpr int MAXU = 4;   // nk / (K/8) <= 4 because nz >= nk

template <typename T, int J>
__global__ void __launch_bounds__(512) k_ax_adj(AxArgs<T> A) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const StoltConst& sc = A.sc;
  const int K = sc.K, nz = sc.nz, nk = sc.nk;
  C* Y = reinterpret_cast<C*>(smem_raw);
  C* Cc = Y + K;                                  // compensation terms
  T* tab = reinterpret_cast<T*>(Cc + K);
  __shared__ int chunk_lo, chunk_hi;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int col = blockIdx.x;

  if (tid == 0) { chunk_lo = INT_MAX; chunk_hi = INT_MIN; }
  for (int i = tid; i < (TABLE_D + 1) * 2 * J; i += nt) tab[i] = __ldg(A.tab.coef + i);
  for (int i = tid; i < K; i += nt) { Y[i] = mk<T>(0, 0); Cc[i] = mk<T>(0, 0); }
  __syncthreads();

  const int ix = col % sc.nx, iy = col / sc.nx;
  StoltPos<T> sp(sc, signed_freq(ix, sc.nx), signed_freq(iy, sc.ny));
  const C* rin = A.in + size_t(col) * nk;
  const int half = K / 2;
  int m0s[MAXU], chunk[MAXU];
  T cs[MAXU][J];
  C val[MAXU];
#pragma unroll
  for (int u = 0; u < MAXU; ++u) {
    const int j = tid + u * nt;
    chunk[u] = INT_MIN;
    if (j < nk) {
      int mfl;
      T frac, turn;
      if (sp.at(sc, j, mfl, frac, turn)) {
        coefficients<T, J>(tab, frac, cs[u]);
        m0s[u] = mfl - J / 2 + 1;
        val[u] = cmulc(__ldg(rin + j), spectral_phase<T>(sc, A.tab.disp, j, turn));
        // chunks of K/2 unwrapped bins (floor division)
        chunk[u] = (mfl >= 0) ? mfl / half : -((-mfl + half - 1) / half);
        atomicMin(&chunk_lo, chunk[u]);
        atomicMax(&chunk_hi, chunk[u]);
      }
    }
  }
  __syncthreads();
  const int clo = chunk_lo, chi = chunk_hi;
  constexpr int NR = J / 2;
  for (int ch = clo; ch <= chi; ++ch) {
    for (int rsd = 0; rsd < NR; ++rsd) {
#pragma unroll
      for (int u = 0; u < MAXU; ++u) {
        const int j = tid + u * nt;
        if (chunk[u] == ch && (j % NR) == rsd) {
#pragma unroll
          for (int l = 0; l < J; ++l) {
            const int bin = (m0s[u] + l) & (K - 1);
            C s = Y[bin], e = Cc[bin];
            comp_add(s.x, e.x, cs[u][l] * val[u].x);
            comp_add(s.y, e.y, cs[u][l] * val[u].y);
            Y[bin] = s;
            Cc[bin] = e;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < K; i += nt) Y[i] = cadd(Y[i], Cc[i]);
  __syncthreads();
  fft_smem<-1, T>(Y, 1, 0, tid, K, sc.logK, A.tab.tw_K, true);
  C* out = A.out + size_t(col) * nz;
  for (int n = tid; n < nz; n += nt) {
    int p = n - nz / 2;
    if (p < 0) p += K;
    out[n] = cscale(Y[p], __ldg(A.tab.scale + n));
  }
}

template <typename T>
static size_t ax_smem(int K, int J, bool adj) {
  return size_t(K) * sizeof(cplx<T>) * (adj ? 2 : 1) + size_t(TABLE_D + 1) * 2 * J * sizeof(T);
}

template <typename T, int J>
static cudaError_t launch_ax_J(const AxArgs<T>& a, int ncols, cudaStream_t s, bool adj) {
  const int K = a.sc.K;
  const int threads = K / 8;
  const size_t sm = ax_smem<T>(K, J, adj);
  if (adj) {
    cudaFuncSetAttribute(k_ax_adj<T, J>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    k_ax_adj<T, J><<<ncols, threads, sm, s>>>(a);
  } else {
    cudaFuncSetAttribute(k_ax_fwd<T, J>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    k_ax_fwd<T, J><<<ncols, threads, sm, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_ax(const AxArgs<T>& a, int ncols, cudaStream_t s, bool adj) {
  switch (a.sc.J) {
    case 4: return launch_ax_J<T, 4>(a, ncols, s, adj);
    case 6: return launch_ax_J<T, 6>(a, ncols, s, adj);
    case 8: return launch_ax_J<T, 8>(a, ncols, s, adj);
  }
  return cudaErrorInvalidValue;
}

template <typename T> cudaError_t launch_ax_fwd(const AxArgs<T>& a, int ncols, cudaStream_t s) {
  return launch_ax<T>(a, ncols, s, false);
}
template <typename T> cudaError_t launch_ax_adj(const AxArgs<T>& a, int ncols, cudaStream_t s) {
  return launch_ax<T>(a, ncols, s, true);
}

template cudaError_t launch_ax_fwd<float>(const AxArgs<float>&, int, cudaStream_t);
template cudaError_t launch_ax_fwd<double>(const AxArgs<double>&, int, cudaStream_t);
template cudaError_t launch_ax_adj<float>(const AxArgs<float>&, int, cudaStream_t);
template cudaError_t launch_ax_adj<double>(const AxArgs<double>&, int, cudaStream_t);

}  // namespace isam
