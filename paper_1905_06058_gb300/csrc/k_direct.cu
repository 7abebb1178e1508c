// Dispersion-compensated inverse FFT of every A-scan (Eq. 9): the direct,
// non-iterative reconstruction on the full-range depth grid,
//   out(x, n) = (1/sqrt(nz)) sum_j s(x, k_j) e^{-j phi(k_j)} e^{-j 2 k_j z_n}.
// With k_j = k_min + j dk and z_n = (n - nz/2) dz, dz = pi/(nz dk):
//   2 k_j z_n = 2 pi (kappa_0 + j)(n - nz/2)/nz,  kappa_0 = k_min/dk, so
//   out(x, n) = post_n sum_j [(-1)^j s_j e^{-j phi_j}] e^{-2 pi i j n / nz},
//   post_n = e^{-2 pi i kappa_0 (n - nz/2)/nz} / sqrt(nz)   (tabulated in FP64),
// an nz-point DFT of the zero-padded, modulated samples (nk <= nz).
#include "fft_smem.cuh"
#include "internal.cuh"

namespace isam {

template <typename T>
__global__ void k_dc_ifft(const T* s, cplx<T>* out, const cplx<T>* disp, const cplx<T>* post,
                          int nk, int nz, int lognz) {
  extern __shared__ __align__(16) unsigned char raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(raw);
  cplx<T>* tw = buf + padded_rows(nz);
  const size_t a = blockIdx.x;
  const T* x = s + a * nk;
  build_twiddles<T>(tw, nz, lognz);
  for (int j = threadIdx.x; j < nz; j += blockDim.x) {
    cplx<T> v = mk<T>(0, 0);
    if (j < nk) {
      const T sj = (j & 1) ? -x[j] : x[j];
      const cplx<T> d = __ldg(disp + j);
      v = mk<T>(sj * d.x, -sj * d.y);
    }
    buf[prow(j)] = v;
  }
  __syncthreads();
  const int nb = nz >= 8 ? nz / 8 : 1;
  fft_smem<-1, false, T>(buf, 1, 0, threadIdx.x, nz, lognz, tw, threadIdx.x < nb);
  cplx<T>* o = out + a * nz;
  for (int n = threadIdx.x; n < nz; n += blockDim.x) o[n] = cmul(buf[prow(n)], __ldg(post + n));
}

template <typename T> cudaError_t launch_dc_ifft(const T* s, cplx<T>* out, const cplx<T>* disp,
                                                 const cplx<T>* post, int nk, int nz, int lognz,
                                                 int n_ascans, cudaStream_t st) {
  const int threads = nz / 8 > 32 ? nz / 8 : 32;
  const size_t sm = size_t(padded_rows(nz) + twiddle_entries(nz, lognz)) * sizeof(cplx<T>);
  cudaFuncSetAttribute(k_dc_ifft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  k_dc_ifft<T><<<n_ascans, threads, sm, st>>>(s, out, disp, post, nk, nz, lognz);
  return cudaGetLastError();
}
template cudaError_t launch_dc_ifft<float>(const float*, float2*, const float2*, const float2*,
                                           int, int, int, int, cudaStream_t);
template cudaError_t launch_dc_ifft<double>(const double*, double2*, const double2*,
                                            const double2*, int, int, int, int, cudaStream_t);

}  // namespace isam
