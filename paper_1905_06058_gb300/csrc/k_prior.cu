// Total-variation prior (§3.1 names TV among the convex priors Eq. 12 extends
// to): isotropic TV over (x, z) of each B-scan slice of the image
// [ny][nx][nz], with forward differences that are zero at the far edge.  Its
// prox z = argmin 1/2 ||z - u||^2 + tau TV(z) is found on the dual,
// z = u - tau grad^H p with |p| <= 1 per pixel, by fast gradient projection
// (Beck & Teboulle): steps of 1/(8 tau) (||grad||^2 <= 8), projection, and
// momentum beta_k from the host.  Each kernel writes only its own pixel.
#include <math.h>

#include "internal.cuh"

namespace isam {

template <typename T>
__device__ __forceinline__ T tv_tau(T tau, const double* lam_dev, double lam_scale) {
  return lam_dev ? T(lam_scale * *lam_dev) : tau;
}

// w = u - tau grad^H r,  (grad^H r)(x, z) = r_x(x-1, z) - r_x(x, z) + r_z(x, z-1) - r_z(x, z)
// with r_x(x, .) = 0 for x = -1 or x = nx - 1 and r_z(., z) = 0 for z = -1 or z = nz - 1
template <typename T>
__global__ void k_tv_primal(const cplx<T>* u, const cplx<T>* rx, const cplx<T>* rz, T tau0,
                            const double* lam_dev, double lam_scale, cplx<T>* w, int nx, int nz,
                            size_t n) {
  const T tau = tv_tau(tau0, lam_dev, lam_scale);
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    const int z = int(i & size_t(nz - 1));
    const int x = int((i / size_t(nz)) % size_t(nx));
    cplx<T> a = mk<T>(0, 0);
    if (x < nx - 1) a = csub(a, rx[i]);
    if (x > 0) a = cadd(a, rx[i - nz]);
    if (z < nz - 1) a = csub(a, rz[i]);
    if (z > 0) a = cadd(a, rz[i - 1]);
    w[i] = tau > T(0) ? csub(u[i], cscale(a, tau)) : u[i];
  }
}

// q = r + grad(w) / (8 tau), p_new = q / max(1, |q|), r = p_new + beta (p_new - p), p = p_new
template <typename T>
__global__ void k_tv_dual(const cplx<T>* w, cplx<T>* px, cplx<T>* pz, cplx<T>* rx, cplx<T>* rz,
                          T tau0, const double* lam_dev, double lam_scale, T beta, int nx, int nz,
                          size_t n) {
  const T tau = tv_tau(tau0, lam_dev, lam_scale);
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    if (!(tau > T(0))) {                       // tau = 0: z = u
      px[i] = pz[i] = rx[i] = rz[i] = mk<T>(0, 0);
      continue;
    }
    const int z = int(i & size_t(nz - 1));
    const int x = int((i / size_t(nz)) % size_t(nx));
    const cplx<T> wi = w[i];
    const cplx<T> gx = x < nx - 1 ? csub(w[i + nz], wi) : mk<T>(0, 0);
    const cplx<T> gz = z < nz - 1 ? csub(w[i + 1], wi) : mk<T>(0, 0);
    const T s = T(1) / (T(8) * tau);
    const cplx<T> qx = cadd(rx[i], cscale(gx, s));
    const cplx<T> qz = cadd(rz[i], cscale(gz, s));
    const T m2 = qx.x * qx.x + qx.y * qx.y + qz.x * qz.x + qz.y * qz.y;
    const T f = m2 > T(1) ? T(1) / sqrt(m2) : T(1);
    const cplx<T> nxv = cscale(qx, f), nzv = cscale(qz, f);
    rx[i] = cadd(nxv, cscale(csub(nxv, px[i]), beta));
    rz[i] = cadd(nzv, cscale(csub(nzv, pz[i]), beta));
    px[i] = nxv;
    pz[i] = nzv;
  }
}

template <typename T> cudaError_t launch_tv_primal(const cplx<T>* u, const cplx<T>* rx,
                                                   const cplx<T>* rz, T tau, const double* lam_dev,
                                                   double lam_scale, cplx<T>* w, int nx, int nz,
                                                   size_t n, cudaStream_t s) {
  k_tv_primal<T><<<1024, 256, 0, s>>>(u, rx, rz, tau, lam_dev, lam_scale, w, nx, nz, n);
  return cudaGetLastError();
}
template <typename T> cudaError_t launch_tv_dual(const cplx<T>* w, cplx<T>* px, cplx<T>* pz,
                                                 cplx<T>* rx, cplx<T>* rz, T tau,
                                                 const double* lam_dev, double lam_scale, T beta,
                                                 int nx, int nz, size_t n, cudaStream_t s) {
  k_tv_dual<T><<<1024, 256, 0, s>>>(w, px, pz, rx, rz, tau, lam_dev, lam_scale, beta, nx, nz, n);
  return cudaGetLastError();
}
template cudaError_t launch_tv_primal<float>(const float2*, const float2*, const float2*, float,
                                             const double*, double, float2*, int, int, size_t,
                                             cudaStream_t);
template cudaError_t launch_tv_primal<double>(const double2*, const double2*, const double2*,
                                              double, const double*, double, double2*, int, int,
                                              size_t, cudaStream_t);
template cudaError_t launch_tv_dual<float>(const float2*, float2*, float2*, float2*, float2*, float,
                                           const double*, double, float, int, int, size_t,
                                           cudaStream_t);
template cudaError_t launch_tv_dual<double>(const double2*, double2*, double2*, double2*, double2*,
                                            double, const double*, double, double, int, int, size_t,
                                            cudaStream_t);

}  // namespace isam
