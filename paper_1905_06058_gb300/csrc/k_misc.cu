// Plan-time FP64 min-max NUFFT table, reductions and small elementwise kernels.
//
// Min-max interpolation (Fessler & Sutton, cited in §3.2).  For fractional
// grid offset f the J real coefficients c(f) minimise
//   sum_{n'} | s(n') sum_l c_l e^{i g lam_l n'} - e^{i g (f - 1/2) n'} |^2,
//   g = 2 pi / K, lam_l = l - (J-1)/2, n' = -nz/2..nz/2,
// whose normal equations are G c = r(f) with the real symmetric Toeplitz
//   G_{l,l'} = sum_{n'} s(n')^2 cos(g (l' - l) n'),
//   r_l(f)   = sum_{n'} s(n') cos(g (f - 1/2 - lam_l) n'),
// s(n') = psi_hat(0) / psi_hat(n'/K), psi_hat the Kaiser-Bessel transform
// with alpha = 2.34 J.  These sums and the J x J Cholesky solves run in FP64
// on the device (cond(G) < 1e5 for J <= 8), one block per offset.
#include <math.h>

#include "internal.cuh"

namespace isam {

__device__ __forceinline__ double kb_scale_dev(int n, int K, int J) {
  const double alpha = 2.34 * J;
  const double v = double(n) / double(K);
  const double r = sqrt(alpha * alpha - (M_PI * J * v) * (M_PI * J * v));
  return (sinh(alpha) / alpha) / (sinh(r) / r);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;   // valid in thread 0
}

// one block of 256 threads per offset f[i]; out64[i*J + l] = c_l(f[i])
__global__ void __launch_bounds__(256) k_minmax_nodes(int nz, int K, int J, const double* fs,
                                                      double* out64) {
  __shared__ double red[8];
  __shared__ double gsum[8], rsum[8];
  const double g = 2.0 * M_PI / K;
  const double f = fs[blockIdx.x];
  double pg[8], pr[8];
  for (int d = 0; d < 8; ++d) { pg[d] = 0.0; pr[d] = 0.0; }
  for (int n = -nz / 2 + int(threadIdx.x); n <= nz / 2; n += blockDim.x) {
    const double s = kb_scale_dev(n, K, J);
    for (int d = 0; d < J; ++d) {
      pg[d] += s * s * cos(g * d * n);
      const double lam = d - 0.5 * (J - 1);
      pr[d] += s * cos(g * (f - 0.5 - lam) * n);
    }
  }
  for (int d = 0; d < J; ++d) {
    double t = block_sum(pg[d], red);
    if (threadIdx.x == 0) gsum[d] = t;
    t = block_sum(pr[d], red);
    if (threadIdx.x == 0) rsum[d] = t;
  }
  if (threadIdx.x == 0) {
    // Cholesky of the Toeplitz G (G[i][j] = gsum[|i-j|]) and two triangular solves
    double Lc[8][8];
    for (int i = 0; i < J; ++i)
      for (int j = 0; j <= i; ++j) {
        double acc = gsum[i - j];
        for (int k = 0; k < j; ++k) acc -= Lc[i][k] * Lc[j][k];
        Lc[i][j] = (i == j) ? sqrt(acc) : acc / Lc[j][j];
      }
    double y[8];
    for (int i = 0; i < J; ++i) {
      double acc = rsum[i];
      for (int k = 0; k < i; ++k) acc -= Lc[i][k] * y[k];
      y[i] = acc / Lc[i][i];
    }
    for (int i = J - 1; i >= 0; --i) {
      double acc = y[i];
      for (int k = i + 1; k < J; ++k) acc -= Lc[k][i] * y[k];
      y[i] = acc / Lc[i][i];
    }
    for (int l = 0; l < J; ++l) out64[blockIdx.x * J + l] = y[l];
  }
}

cudaError_t minmax_nodes(int nz, int K, int J, const double* f, int n, double* out,
                         cudaStream_t s) {
  k_minmax_nodes<<<n, 256, 0, s>>>(nz, K, J, f, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Reductions: stage 1 writes one partial per block, stage 2 combines them in a
// fixed order (deterministic).  The max lets a NaN through: a NaN anywhere in
// the input makes the result NaN, so lambda = c ||A^H s||_inf taken from
// corrupted data is visibly non-finite instead of the max of the rest.
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T nan_max(T a, T b) {
  return (b > a || b != b) ? b : a;
}
template <typename T, bool MAX>
__global__ void __launch_bounds__(256) k_reduce1(const cplx<T>* x, size_t n, double* partial) {
  __shared__ double red[8];
  // |x_i|^2 in the data's precision; the max in it too, sums in double
  T vm = T(0);
  double v = 0.0;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    const cplx<T> a = x[i];
    const T m = a.x * a.x + a.y * a.y;
    if (MAX) vm = nan_max(vm, m);
    else v += double(m);
  }
  if (MAX) v = double(vm);
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(0xffffffffu, v, o);
    v = MAX ? nan_max(v, t) : v + t;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = red[0];
    for (int w = 1; w < int(blockDim.x >> 5); ++w) t = MAX ? nan_max(t, red[w]) : t + red[w];
    partial[blockIdx.x] = t;
  }
}

// One block of 256 threads combines values in a fixed order: every thread its
// strided share, then a shuffle tree within each warp and across the eight
// warps' results (the same order on every run; no serial chain of 256 adds).
template <bool MAX> __device__ __forceinline__ double combine(double a, double b) {
  return MAX ? nan_max(a, b) : a + b;
}
template <bool MAX> __device__ __forceinline__ double block256_combine(double v, double* red8) {
  for (int o = 16; o > 0; o >>= 1) v = combine<MAX>(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red8[threadIdx.x >> 5] = v;
  __syncthreads();
  v = threadIdx.x < 8 ? red8[threadIdx.x] : 0.0;
  if (threadIdx.x < 32)
    for (int o = 4; o > 0; o >>= 1) v = combine<MAX>(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;   // the block's result in thread 0
}

// single block: out = sqrt(max or sum of partial)
template <bool MAX>
__global__ void __launch_bounds__(256) k_reduce2(const double* partial, int n, double* out) {
  __shared__ double red[8];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v = combine<MAX>(v, partial[i]);
  v = block256_combine<MAX>(v, red);
  if (threadIdx.x == 0) *out = sqrt(v);
}

template <typename T> cudaError_t launch_max_abs(const cplx<T>* x, size_t n, double* partial,
                                                  int nblocks, double* out, cudaStream_t s) {
  k_reduce1<T, true><<<nblocks, 256, 0, s>>>(x, n, partial);
  k_reduce2<true><<<1, 256, 0, s>>>(partial, nblocks, out);
  return cudaGetLastError();
}
template <typename T> cudaError_t launch_norm2(const cplx<T>* x, size_t n, double* partial,
                                                int nblocks, double* out, cudaStream_t s) {
  k_reduce1<T, false><<<nblocks, 256, 0, s>>>(x, n, partial);
  k_reduce2<false><<<1, 256, 0, s>>>(partial, nblocks, out);
  return cudaGetLastError();
}
template cudaError_t launch_max_abs<float>(const float2*, size_t, double*, int, double*, cudaStream_t);
template cudaError_t launch_max_abs<double>(const double2*, size_t, double*, int, double*, cudaStream_t);
template cudaError_t launch_norm2<float>(const float2*, size_t, double*, int, double*, cudaStream_t);
template cudaError_t launch_norm2<double>(const double2*, size_t, double*, int, double*, cudaStream_t);

// sum_i w[i mod nz] |x_i| (w null: 1), the l1 term of Eq. 12: per-block FP64
// partials, then one block sums them in a fixed order into *out
template <typename T>
__global__ void __launch_bounds__(256) k_wl1(const cplx<T>* x, size_t n, const T* w, int nz,
                                             double* partial) {
  __shared__ double red[8];
  double v = 0.0;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    const cplx<T> a = x[i];
    const double m = sqrt(double(a.x) * a.x + double(a.y) * a.y);
    v += w ? double(w[i & size_t(nz - 1)]) * m : m;
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = red[0];
    for (int k = 1; k < int(blockDim.x >> 5); ++k) t += red[k];
    partial[blockIdx.x] = t;
  }
}
__global__ void __launch_bounds__(256) k_sum1(const double* partial, int n, double* out) {
  __shared__ double red[8];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += partial[i];
  v = block256_combine<false>(v, red);
  if (threadIdx.x == 0) *out = v;
}
template <typename T> cudaError_t launch_wl1(const cplx<T>* x, size_t n, const T* w, int nz,
                                             double* partial, int nblocks, double* out,
                                             cudaStream_t s) {
  k_wl1<T><<<nblocks, 256, 0, s>>>(x, n, w, nz, partial);
  k_sum1<<<1, 256, 0, s>>>(partial, nblocks, out);
  return cudaGetLastError();
}
template cudaError_t launch_wl1<float>(const float2*, size_t, const float*, int, double*, int,
                                       double*, cudaStream_t);
template cudaError_t launch_wl1<double>(const double2*, size_t, const double*, int, double*, int,
                                        double*, cudaStream_t);

// out[0..2] = column sums of partial[n][3]
__global__ void __launch_bounds__(256) k_sum3(const double* partial, int n, double* out,
                                              const StopRule sr) {
  __shared__ double red[3][8];
  // an earlier check stopped the solve: this iteration's kernels returned
  // without writing the partials
  if (sr.stop && *reinterpret_cast<const volatile int*>(sr.stop)) return;
  double v[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    for (int c = 0; c < 3; ++c) v[c] += partial[3 * i + c];
  for (int c = 0; c < 3; ++c) v[c] = block256_combine<false>(v[c], red[c]);
  if (threadIdx.x == 0) {
    for (int c = 0; c < 3; ++c) out[c] = v[c];
    if (sr.stop) {
      // Eq. 15 as the host evaluates it (the larger of the two norms, NaN kept)
      const double a = sqrt(v[0]), g = sqrt(v[1]), b = sqrt(v[2]);
      const double rr = a / ((g < b ? b : g) + sr.eps);
      *sr.rr = rr;
      if (rr < sr.tol) {
        sr.stop[1] = sr.iter;
        sr.stop[0] = 1;
      }
    }
  }
}
cudaError_t launch_sum3(const double* partial, int n, double* out, const StopRule& sr,
                        cudaStream_t s) {
  k_sum3<<<1, 256, 0, s>>>(partial, n, out, sr);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_select_iterate(const cplx<T>* a, const cplx<T>* b, cplx<T>* out, size_t n,
                                 const int* stop, int last) {
  const cplx<T>* src = stop[0] != 0 && ((last - stop[1]) & 1) ? b : a;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    out[i] = src[i];
}
template <typename T> cudaError_t launch_select_iterate(const cplx<T>* a, const cplx<T>* b,
                                                         cplx<T>* out, size_t n, const int* stop,
                                                         int last, cudaStream_t s) {
  k_select_iterate<T><<<1024, 256, 0, s>>>(a, b, out, n, stop, last);
  return cudaGetLastError();
}
template cudaError_t launch_select_iterate<float>(const float2*, const float2*, float2*, size_t,
                                                  const int*, int, cudaStream_t);
template cudaError_t launch_select_iterate<double>(const double2*, const double2*, double2*,
                                                   size_t, const int*, int, cudaStream_t);

template <typename T>
__global__ void k_scale(cplx<T>* x, size_t n, const double* denom) {
  const double d = *denom;
  const T f = d > 0.0 ? T(1.0 / d) : T(0);
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    x[i] = cscale(x[i], f);
}
template <typename T> cudaError_t launch_scale(cplx<T>* x, size_t n, const double* denom,
                                                cudaStream_t s) {
  k_scale<T><<<1024, 256, 0, s>>>(x, n, denom);
  return cudaGetLastError();
}
template cudaError_t launch_scale<float>(float2*, size_t, const double*, cudaStream_t);
template cudaError_t launch_scale<double>(double2*, size_t, const double*, cudaStream_t);

template <typename T>
__global__ void k_extrapolate(const cplx<T>* z1, const cplx<T>* z2, T mu, cplx<T>* out, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    const cplx<T> a = z1[i], b = z2[i];
    out[i] = cadd(a, cscale(csub(a, b), mu));
  }
}
template <typename T> cudaError_t launch_extrapolate(const cplx<T>* z1, const cplx<T>* z2, T mu,
                                                     cplx<T>* out, size_t n, cudaStream_t s) {
  k_extrapolate<T><<<1024, 256, 0, s>>>(z1, z2, mu, out, n);
  return cudaGetLastError();
}
template cudaError_t launch_extrapolate<float>(const float2*, const float2*, float, float2*, size_t, cudaStream_t);
template cudaError_t launch_extrapolate<double>(const double2*, const double2*, double, double2*, size_t, cudaStream_t);

template <typename A, typename B>
__global__ void k_convert(const cplx<A>* x, cplx<B>* y, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    y[i] = mk<B>(B(x[i].x), B(x[i].y));
}
template <typename Tsrc, typename Tdst> cudaError_t launch_convert(const cplx<Tsrc>* x,
                                                                   cplx<Tdst>* y, size_t n,
                                                                   cudaStream_t s) {
  k_convert<Tsrc, Tdst><<<1024, 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}
template cudaError_t launch_convert<float, double>(const float2*, double2*, size_t, cudaStream_t);
template cudaError_t launch_convert<double, float>(const double2*, float2*, size_t, cudaStream_t);

// deterministic start vector: splitmix64 of the index, uniform in [-0.5, 0.5)
__device__ __forceinline__ double hash01(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return double(x >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}
template <typename T>
__global__ void k_fill_start(cplx<T>* x, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    x[i] = mk<T>(T(hash01(2 * i)), T(hash01(2 * i + 1)));
}
template <typename T> cudaError_t launch_fill_start(cplx<T>* x, size_t n, cudaStream_t s) {
  k_fill_start<T><<<1024, 256, 0, s>>>(x, n);
  return cudaGetLastError();
}
template cudaError_t launch_fill_start<float>(float2*, size_t, cudaStream_t);
template cudaError_t launch_fill_start<double>(double2*, size_t, cudaStream_t);

}  // namespace isam

namespace isam {

// y = a - b (real arrays)
template <typename T>
__global__ void k_rsub(const T* a, const T* b, T* y, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    y[i] = a[i] - b[i];
}
template <typename T> cudaError_t launch_rsub(const T* a, const T* b, T* y, size_t n,
                                               cudaStream_t s) {
  k_rsub<T><<<1024, 256, 0, s>>>(a, b, y, n);
  return cudaGetLastError();
}
template cudaError_t launch_rsub<float>(const float*, const float*, float*, size_t, cudaStream_t);
template cudaError_t launch_rsub<double>(const double*, const double*, double*, size_t, cudaStream_t);

// y = x + alpha * v (complex arrays)
template <typename T>
__global__ void k_caxpy(const cplx<T>* x, const cplx<T>* v, T alpha, cplx<T>* y, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    y[i] = cadd(x[i], cscale(v[i], alpha));
}
template <typename T> cudaError_t launch_caxpy(const cplx<T>* x, const cplx<T>* v, T alpha,
                                                cplx<T>* y, size_t n, cudaStream_t s) {
  k_caxpy<T><<<1024, 256, 0, s>>>(x, v, alpha, y, n);
  return cudaGetLastError();
}
template cudaError_t launch_caxpy<float>(const float2*, const float2*, float, float2*, size_t, cudaStream_t);
template cudaError_t launch_caxpy<double>(const double2*, const double2*, double, double2*, size_t, cudaStream_t);

}  // namespace isam
