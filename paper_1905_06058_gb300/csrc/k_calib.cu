// Kernels for calibrating the dispersion coefficients a_1..a_4 (Eq. 7) and
// the focal depth z0 by gradient descent through the model.
//
// A depends on theta = (a_1..a_4, z0) only through the spectral phase
// P(q, k) = e^{j phi(k)} e^{j (2k + beta) z0}, so with S_x = P . N(F x) (the
// lateral spectrum of K_hat x before the real part) and F y the unitary
// lateral FFT of real spectra y,
//   <dA/dtheta x, y> = sum_{q,k} D_theta(q, k) Re( j conj(F y) S_x ),
//   D_{a_i} = (k - k0)^i,   D_{z0} = 2k + beta = a / (2 kappa + p) dk,
// in plan grid units (kappa = k/dk, a = (q/dk)^2, p = sqrt(4 kappa^2 - a)).
//
// k_param_reduce forms these sums per column pair (q, -q).  Where the "data"
// spectrum is itself the real part of a model spectrum E, F y = (E(q) +
// conj E(-q))/2 is formed pointwise from the pair, exactly as the fused
// gradient kernel forms the residual.  Sums are FP64: the polynomial moments
// m_i = sum t^i v with t = j - (nk-1)/2 (then a_i gradient = dk^i m_i) and
// m_z = sum (a / (2 kappa + p)) v (then z0 gradient = dk m_z).
#include <math.h>

#include <type_traits>

#include "internal.cuh"

namespace isam {

template <typename T>
__device__ __forceinline__ T im_part(cplx<T> F, cplx<T> S) {   // Re(j conj(F) S)
  return F.y * S.x - F.x * S.y;
}

template <typename T>
__device__ __forceinline__ cplx<T> real_part_spectrum(cplx<T> a, cplx<T> b) {
  return cscale(cadd(a, cconj(b)), T(0.5));   // F(Re v)(q) from F v(q), F v(-q)
}

template <typename T>
__global__ void __launch_bounds__(256) k_param_reduce(const __grid_constant__ ParamArgs<T> A) {
  using C = cplx<T>;
  const int2 pr = A.pairs[blockIdx.x];
  const int c1 = pr.x, c2 = pr.y;
  const bool two = c1 != c2;
  const int nk = A.sc.nk, nx = A.sc.nx;
  const int mx = c1 % nx <= (nx - 1) / 2 ? c1 % nx : c1 % nx - nx;
  const int ny = A.sc.ny, iy = c1 / nx;
  const int my = iy <= (ny - 1) / 2 ? iy : iy - ny;
  const double a = A.sc.Qx * double(mx) * mx + A.sc.Qy * double(my) * my;
  const double tc = 0.5 * double(nk - 1);
  C* s1 = A.su + size_t(c1) * nk;
  C* s2 = A.su + size_t(c2) * nk;
  const C* e1 = A.se ? A.se + size_t(c1) * nk : nullptr;
  const C* e2 = A.se ? A.se + size_t(c2) * nk : nullptr;
  const C* f1 = A.fd ? A.fd + size_t(c1) * nk : nullptr;
  const C* f2 = A.fd ? A.fd + size_t(c2) * nk : nullptr;
  double m[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  float mf[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  for (int j = threadIdx.x; j < nk; j += blockDim.x) {
    const C S1 = s1[j], S2 = s2[j];
    const C z = mk<T>(0, 0);
    const C E1 = e1 ? e1[j] : z, E2 = e2 ? e2[j] : z;
    C F1 = e1 ? real_part_spectrum<T>(E1, E2) : z;
    C F2 = e1 ? real_part_spectrum<T>(E2, E1) : z;
    if (f1) {
      F1 = cadd(F1, cscale(f1[j], A.fd_sign));
      F2 = cadd(F2, cscale(f2[j], A.fd_sign));
    }
    const C Fa1 = real_part_spectrum<T>(S1, S2), Fa2 = real_part_spectrum<T>(S2, S1);
    T v = im_part<T>(F1, S1);
    if (two) v += im_part<T>(F2, S2);
    if (e1) {
      v += im_part<T>(Fa1, E1);
      if (two) v += im_part<T>(Fa2, E2);
    }
    if (A.write_fa) {
      s1[j] = Fa1;
      if (two) s2[j] = Fa2;
    }
    if constexpr (std::is_same<T, float>::value) {
      // FP32 plans: weights (k_j - k0)^i in float (t = j - (nk-1)/2 is exact)
      // and the z0 weight a / (2 kappa + sqrt(4 kappa^2 - a)) with only the
      // cancelling 4 kappa^2 - a in double; a thread's few terms summed in
      // float (mf), the block's threads in double below
      const float t = float(j) - float(tc);
      float tp = t;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        mf[i] = fmaf(tp, v, mf[i]);
        tp *= t;
      }
      const double kap = A.sc.kap + double(j);
      const double x = fma(4.0 * kap, kap, -a);
      if (x > 0.0) {
        const float d = float(a) / (2.0f * float(kap) + sqrtf(float(x)));
        mf[4] = fmaf(d, v, mf[4]);
      }
    } else {
      const double dv = double(v);
      const double t = double(j) - tc;
      double tp = t;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        m[i] = fma(tp, dv, m[i]);
        tp *= t;
      }
      const double kap = A.sc.kap + double(j);
      const double x = 4.0 * kap * kap - a;
      if (x > 0.0) m[4] = fma(a / (2.0 * kap + sqrt(x)), dv, m[4]);
    }
  }
  if constexpr (std::is_same<T, float>::value) {
#pragma unroll
    for (int i = 0; i < 5; ++i) m[i] = double(mf[i]);
  }
  __shared__ double red[8][5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    double s = m[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][i] = s;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int w = 0; w < (blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
    A.partial[size_t(blockIdx.x) * 5 + threadIdx.x] += s;
  }
}

template <typename T> cudaError_t launch_param_reduce(const ParamArgs<T>& a, int npairs,
                                                      cudaStream_t s) {
  k_param_reduce<T><<<npairs, 256, 0, s>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_param_reduce<float>(const ParamArgs<float>&, int, cudaStream_t);
template cudaError_t launch_param_reduce<double>(const ParamArgs<double>&, int, cudaStream_t);

// ubar = J_T(u)^T zbar for z = T_tau(u) (Eq. 14), tau = lambda w_n / L:
// where the threshold passes u (the same test as the forward update),
// ubar = zbar - tau (zbar/|u| - u Re(conj(u) zbar)/|u|^3); else 0.
__device__ __forceinline__ float2 st_vjp(float2 u, float2 zb, float tau) {
  const float m2 = fmaf(u.x, u.x, u.y * u.y);
  const float inv = m2 > 0.0f ? rsqrtf(m2) : 0.0f;
  if (!(1.0f - tau * inv > 0.0f)) return make_float2(0.0f, 0.0f);
  const float rz = fmaf(u.x, zb.x, u.y * zb.y) * inv * inv * inv;
  return make_float2(zb.x - tau * (zb.x * inv - u.x * rz), zb.y - tau * (zb.y * inv - u.y * rz));
}
__device__ __forceinline__ double2 st_vjp(double2 u, double2 zb, double tau) {
  const double m2 = fma(u.x, u.x, u.y * u.y);
  const double am = sqrt(m2);
  if (!(m2 > 0.0) || !(1.0 - tau / am > 0.0)) return make_double2(0.0, 0.0);
  const double inv = 1.0 / am;
  const double rz = fma(u.x, zb.x, u.y * zb.y) * inv * inv * inv;
  return make_double2(zb.x - tau * (zb.x * inv - u.x * rz), zb.y - tau * (zb.y * inv - u.y * rz));
}

template <typename T>
__global__ void k_st_vjp(const cplx<T>* u, const cplx<T>* zbar, const T* w, T lam_over_L, int nz,
                         cplx<T>* out, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    const T tau = w ? lam_over_L * w[i & size_t(nz - 1)] : lam_over_L;
    out[i] = st_vjp(u[i], zbar[i], tau);
  }
}
template <typename T> cudaError_t launch_st_vjp(const cplx<T>* u, const cplx<T>* zbar, const T* w,
                                                T lam_over_L, int nz, cplx<T>* out, size_t n,
                                                cudaStream_t s) {
  k_st_vjp<T><<<1024, 256, 0, s>>>(u, zbar, w, lam_over_L, nz, out, n);
  return cudaGetLastError();
}
template cudaError_t launch_st_vjp<float>(const float2*, const float2*, const float*, float, int,
                                          float2*, size_t, cudaStream_t);
template cudaError_t launch_st_vjp<double>(const double2*, const double2*, const double*, double,
                                           int, double2*, size_t, cudaStream_t);

// etabar = ubar - b / L;  zb1 += (1 + mu) etabar;  zb2 -= mu etabar  (either may be null)
template <typename T>
__global__ void k_bwd_combine(const cplx<T>* ubar, const cplx<T>* b, T inv_L, T mu, cplx<T>* zb1,
                              cplx<T>* zb2, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    const cplx<T> e = csub(ubar[i], cscale(b[i], inv_L));
    if (zb1) zb1[i] = cadd(zb1[i], cscale(e, T(1) + mu));
    if (zb2) zb2[i] = csub(zb2[i], cscale(e, mu));
  }
}
template <typename T> cudaError_t launch_bwd_combine(const cplx<T>* ubar, const cplx<T>* b,
                                                     T inv_L, T mu, cplx<T>* zb1, cplx<T>* zb2,
                                                     size_t n, cudaStream_t s) {
  k_bwd_combine<T><<<1024, 256, 0, s>>>(ubar, b, inv_L, mu, zb1, zb2, n);
  return cudaGetLastError();
}
template cudaError_t launch_bwd_combine<float>(const float2*, const float2*, float, float, float2*,
                                               float2*, size_t, cudaStream_t);
template cudaError_t launch_bwd_combine<double>(const double2*, const double2*, double, double,
                                                double2*, double2*, size_t, cudaStream_t);

}  // namespace isam
