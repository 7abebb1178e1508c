// Lateral passes: batched shared-memory FFTs along the lateral axis (x, or y
// for volumes) of data viewed as [B][L][M], a block owning TZ consecutive
// columns m of one batch b (rows of TZ contiguous elements, coalesced).
// Unitary transforms (each axis scaled by 1/sqrt(L)), §2, Eq. 16-17.
//
// Fused variants remove whole round trips through HBM:
//   LAT_MID     R = F( Re(F^{-1} S) - s_d ): forward-model output, data residual
//               and the start of the adjoint in one pass (Alg. 1, gradient step);
//   LAT_UPDATE  g = F^{-1} G, then in image space the FISTA step of Alg. 1:
//               eta^k = z^{k-1} + mu_{k-1}(z^{k-1} - z^{k-2}),
//               z^k = T_{lambda w / L}(eta^k - g/L)            (Eq. 14),
//               eta^{k+1} = z^k + mu_k (z^k - z^{k-1}),
//               partial norms for the relative residual      (Eq. 15),
//               then eta_hat^{k+1} = F eta^{k+1}.
#include <math.h>

#include "fft_smem.cuh"
#include "internal.cuh"

namespace isam {

int lat_tile(int L, int M) {
  int tz = L >= 8 ? 8192 / L : 16;
  if (tz > 16) tz = 16;
  if (tz > M) tz = M;
  if (tz < 1) tz = 1;
  return tz;
}

template <typename T>
__device__ __forceinline__ cplx<T> soft_threshold(cplx<T> u, T tau) {
  // T_tau(u) = u max(|u|-tau,0) / (max(|u|-tau,0) + tau); 0 where 0/0  (Eq. 14)
  T mag = sqrt(u.x * u.x + u.y * u.y);
  T m = mag - tau;
  m = m > T(0) ? m : T(0);
  T den = m + tau;
  T f = den > T(0) ? m / den : T(0);
  return cscale(u, f);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(1024) k_lat(LatArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int TZ = a.TZ, L = a.L, logTZ = a.logTZ;
  const int col = tid & (TZ - 1), b = tid >> logTZ;
  const size_t M = size_t(a.M);
  const size_t base = size_t(blockIdx.y) * size_t(L) * M + size_t(blockIdx.x) * TZ;
  const int n_el = L * TZ;

  // load the tile
  if (MODE == LAT_R2C_FWD) {
    const T* in = static_cast<const T*>(a.in);
    for (int e = tid; e < n_el; e += nt) {
      const size_t gi = base + size_t(e >> logTZ) * M + (e & (TZ - 1));
      buf[e] = mk<T>(in[gi], T(0));
    }
  } else {
    const C* in = static_cast<const C*>(a.in);
    for (int e = tid; e < n_el; e += nt) {
      const size_t gi = base + size_t(e >> logTZ) * M + (e & (TZ - 1));
      buf[e] = in[gi];
    }
  }
  __syncthreads();

  if (MODE == LAT_C2C_FWD || MODE == LAT_R2C_FWD)
    fft_smem<-1, T>(buf, TZ, col, b, L, a.logL, a.tw, true);
  else
    fft_smem<+1, T>(buf, TZ, col, b, L, a.logL, a.tw, true);

  const T nrm = a.norm;
  if (MODE == LAT_C2C_FWD || MODE == LAT_C2C_INV || MODE == LAT_R2C_FWD) {
    C* out = static_cast<C*>(a.out);
    for (int e = tid; e < n_el; e += nt) {
      const size_t gi = base + size_t(e >> logTZ) * M + (e & (TZ - 1));
      out[gi] = cscale(buf[e], nrm);
    }
    return;
  }
  if (MODE == LAT_INV_REAL) {
    T* out = static_cast<T*>(a.out);
    for (int e = tid; e < n_el; e += nt) {
      const size_t gi = base + size_t(e >> logTZ) * M + (e & (TZ - 1));
      out[gi] = buf[e].x * nrm;
    }
    return;
  }
  if (MODE == LAT_MID) {
    for (int e = tid; e < n_el; e += nt) {
      const size_t gi = base + size_t(e >> logTZ) * M + (e & (TZ - 1));
      buf[e] = mk<T>(buf[e].x * nrm - a.s_d[gi], T(0));
    }
  }
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
  if (MODE == LAT_UPDATE) {
    bool bad = false;
    for (int e = tid; e < n_el; e += nt) {
      const size_t gi = base + size_t(e >> logTZ) * M + (e & (TZ - 1));
      const int n = int((size_t(blockIdx.x) * TZ + (e & (TZ - 1))) & size_t(a.nz - 1));
      const C gl = cscale(buf[e], nrm * a.inv_L);          // g^k = (1/L) A^H(A eta - s)
      const C z1 = a.z1[gi];
      const C z2 = a.z2[gi];
      const C eta = cadd(z1, cscale(csub(z1, z2), a.mu_prev));
      const T tau = a.w ? a.lam_over_L * a.w[n] : a.lam_over_L;
      const C z = soft_threshold<T>(csub(eta, gl), tau);
      a.zout[gi] = z;
      buf[e] = cadd(z, cscale(csub(z, z1), a.mu));
      const C d = csub(z, eta);
      const C dg = cadd(d, gl);
      acc0 += double(d.x) * d.x + double(d.y) * d.y;
      acc1 += double(gl.x) * gl.x + double(gl.y) * gl.y;
      acc2 += double(dg.x) * dg.x + double(dg.y) * dg.y;
      bad |= !(isfinite(z.x) && isfinite(z.y));
    }
    if (bad) atomicOr(a.flag, 1);
  }
  __syncthreads();
  fft_smem<-1, T>(buf, TZ, col, b, L, a.logL, a.tw, true);
  C* out = static_cast<C*>(a.out);
  for (int e = tid; e < n_el; e += nt) {
    const size_t gi = base + size_t(e >> logTZ) * M + (e & (TZ - 1));
    out[gi] = cscale(buf[e], nrm);
  }
  if (MODE == LAT_UPDATE && a.partial != nullptr) {
    __shared__ double red[3][32];
    acc0 = warp_sum(acc0); acc1 = warp_sum(acc1); acc2 = warp_sum(acc2);
    const int wid = tid >> 5, lane = tid & 31;
    if (lane == 0) { red[0][wid] = acc0; red[1][wid] = acc1; red[2][wid] = acc2; }
    __syncthreads();
    if (wid == 0) {
      const int nw = (nt + 31) >> 5;
      double v0 = lane < nw ? red[0][lane] : 0.0;
      double v1 = lane < nw ? red[1][lane] : 0.0;
      double v2 = lane < nw ? red[2][lane] : 0.0;
      v0 = warp_sum(v0); v1 = warp_sum(v1); v2 = warp_sum(v2);
      if (lane == 0) {
        const size_t blk = size_t(blockIdx.y) * gridDim.x + blockIdx.x;
        a.partial[3 * blk + 0] = v0;
        a.partial[3 * blk + 1] = v1;
        a.partial[3 * blk + 2] = v2;
      }
    }
  }
}

template <typename T, int MODE>
static cudaError_t launch_lat_mode(const LatArgs<T>& a, cudaStream_t s) {
  const int threads = (a.L >= 8 ? a.L / 8 : 1) * a.TZ;
  const size_t sm = size_t(a.L) * a.TZ * sizeof(cplx<T>);
  cudaFuncSetAttribute(k_lat<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  dim3 grid(a.M / a.TZ, a.B);
  k_lat<T, MODE><<<grid, threads, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_lat(int mode, const LatArgs<T>& a, cudaStream_t s) {
  switch (mode) {
    case LAT_C2C_FWD: return launch_lat_mode<T, LAT_C2C_FWD>(a, s);
    case LAT_C2C_INV: return launch_lat_mode<T, LAT_C2C_INV>(a, s);
    case LAT_R2C_FWD: return launch_lat_mode<T, LAT_R2C_FWD>(a, s);
    case LAT_INV_REAL: return launch_lat_mode<T, LAT_INV_REAL>(a, s);
    case LAT_MID: return launch_lat_mode<T, LAT_MID>(a, s);
    case LAT_UPDATE: return launch_lat_mode<T, LAT_UPDATE>(a, s);
  }
  return cudaErrorInvalidValue;
}

template cudaError_t launch_lat<float>(int, const LatArgs<float>&, cudaStream_t);
template cudaError_t launch_lat<double>(int, const LatArgs<double>&, cudaStream_t);

}  // namespace isam
