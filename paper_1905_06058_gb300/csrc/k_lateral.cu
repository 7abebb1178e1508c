// Lateral passes: batched shared-memory FFTs along the lateral axis (x, or y
// for volumes) of data viewed as [B][L][M], a block owning 2*TP consecutive
// columns m of one batch b.  Each shared-memory element holds two adjacent
// columns (16- or 32-byte accesses, one padding row per 8 rows), global rows
// are read and written as 2*TP*8 contiguous bytes.  Unitary transforms (each
// axis scaled by 1/sqrt(L)), §2, Eq. 16-17.
//
// LAT_UPDATE fuses the FISTA step of Alg. 1 between an inverse and a forward
// lateral transform:  g = F^{-1} G (the gradient A^H(A eta - s_d)),
//   eta^k = z^{k-1} + mu_{k-1}(z^{k-1} - z^{k-2}),
//   z^k = T_{lambda w / L}(eta^k - g/L)                            (Eq. 14),
//   eta^{k+1} = z^k + mu_k (z^k - z^{k-1}),  eta_hat^{k+1} = F eta^{k+1},
// with partial norms for the relative residual (Eq. 15).  LAT_UPDATE_U takes
// u_hat = eta_hat^k - G/L instead of G (the lateral transform is linear):
// u = F^{-1} u_hat, and z^{k-2} is not read.
#include <math.h>

#include <type_traits>

#include "fft_col16.cuh"
#include "fft_smem.cuh"
#include "internal.cuh"

namespace isam {

int lat_tile(int L, int M) {   // pair-columns per block (a power of two)
  int tp = L >= 8 ? 4096 / L : 8;
  if (tp > 8) tp = 8;
  if (tp > M / 2) tp = M / 2;
  if (tp < 1) tp = 1;
  while (tp & (tp - 1)) tp &= tp - 1;
  return tp;
}

bool fft_length(int L, int* log2, int* r3) {
  if (L < 1) return false;
  int t = 0, m = L;
  if (m % 3 == 0) { m /= 3; t = 1; }
  if (m & (m - 1)) return false;
  int p = 0;
  while ((1 << p) < m) ++p;
  if (t && p < 3) return false;
  *log2 = p;
  *r3 = t;
  return true;
}

// T_tau(u) = u max(|u| - tau, 0) / (max(|u| - tau, 0) + tau)  (Eq. 14),
// evaluated as u max(1 - tau / |u|, 0); 0 where |u| = 0.
__device__ __forceinline__ float2 soft_threshold(float2 u, float tau) {
  const float m2 = fmaf(u.x, u.x, u.y * u.y);
  const float f = m2 > 0.0f ? fmaxf(1.0f - tau * rsqrtf(m2), 0.0f) : 0.0f;
  return cscale(u, f);
}
__device__ __forceinline__ double2 soft_threshold(double2 u, double tau) {
  const double m2 = fma(u.x, u.x, u.y * u.y);
  const double f = m2 > 0.0 ? fmax(1.0 - tau / sqrt(m2), 0.0) : 0.0;
  return cscale(u, f);
}

// Sum of v over the threads of one warp that exist: a block of nt threads
// (any count, e.g. 8, 24 or 48 for short or 3 * 2^p lateral lengths) has a
// last warp of n = nt - 32 w lanes, and a shuffle may only name lanes that
// exist, so the mask holds lanes [0, n) and a lane adds a partner's value only
// when that partner exists.  The sum lands in lane 0.
__device__ __forceinline__ double warp_sum_lanes(double v, int n) {
  const unsigned mask = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_down_sync(mask, v, o);
    if (lane + o < n) v += t;
  }
  return v;
}

template <typename T> struct rpair_t;
template <> struct rpair_t<float> { using type = float2; };
template <> struct rpair_t<double> { using type = double2; };

// LOGL > 0: the transforms are the compile-time-length ones for L = 2^LOGL at
// the stride 2^LOGTP = TP (no radix-3 pass), with constant row offsets;
// LOGL = 0: runtime-length transforms.  The tile indexing is the same.
template <typename T, int MODE, int LOGL, int LOGTP, bool C16>
__global__ void __launch_bounds__(512, 2) k_lat(const __grid_constant__ LatArgs<T> a) {
  using C = cplx<T>;
  using V = cpair<T>;
  using RP = typename rpair_t<T>::type;   // two adjacent reals
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  const int tid = threadIdx.x, nt = blockDim.x;
  constexpr bool CT = LOGL > 0;
  const int TP = a.TZ, L = CT ? (1 << LOGL) : a.L, logTP = a.logTZ;
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(buf + size_t(padded_rows(L)) * TP);
  // FP32 at L = 1024 and 256: column-split radix-16 transforms (fft_col16.cuh)
  // when the plan chose them (C16)
  constexpr bool COL16 = C16 && CT && std::is_same<T, float>::value && (LOGL == 10 || LOGL == 8);
  // programmatic dependent launch: let the next kernel start its prologue,
  // build the twiddles, then wait for the previous kernel's results
  cudaTriggerProgrammaticLaunchCompletion();
  if constexpr (COL16) c16::build_lat_twiddles<LOGL>(reinterpret_cast<float4*>(tw));
  else build_twiddles<T>(tw, L, CT ? LOGL : a.logL, CT ? 0 : a.r3);
  cudaGridDependencySynchronize();
  // the solve's stop flag (written by an earlier kernel, so visible after the
  // wait): loaded here, tested before the first global write (after the first
  // transform), so its latency overlaps the tile's loads
  const bool stopped = a.stop != nullptr && __ldcg(a.stop) != 0;
  const int col = tid & (TP - 1), b = tid >> logTP;
  const size_t M = size_t(a.M);
  const size_t m_first = size_t(blockIdx.x) * (2 * TP);
  const size_t base = size_t(blockIdx.y) * size_t(L) * M + m_first;
  const int n_el = L * TP;

  // Every thread owns ept = n_el / blockDim elements (8 for L >= 8):
  // element i of a thread is e = tid + i * nt (row e / TP, pair-column e % TP).
  const int ept = n_el / nt;
  auto gidx = [&](int e) { return base + size_t(e >> logTP) * M + 2 * (e & (TP - 1)); };
  auto sidx = [&](int e) { return prow(e >> logTP) * TP + (e & (TP - 1)); };
  auto lat_fft = [&](auto sign) {
    constexpr int SIGN = decltype(sign)::value;
    if constexpr (COL16)
      c16::lat_transform<SIGN, LOGL, 2 * (1 << LOGTP)>(reinterpret_cast<float2*>(buf),
                                                        reinterpret_cast<const float4*>(tw));
    else if constexpr (CT) fft_cols_ct<SIGN, false, LOGL, (1 << LOGTP), T>(buf, col, b, tw);
    else fft_smem<SIGN, false, T>(buf, TP, col, b, L, a.logL, tw, true, a.r3);
  };
  using FWD = std::integral_constant<int, -1>;
  using INV = std::integral_constant<int, +1>;

  // load the tile: all global loads first, then the shared-memory stores
  {
    V v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i >= ept) break;
      const size_t gi = gidx(tid + i * nt);
      if (MODE == LAT_R2C_FWD) {
        const RP r = *reinterpret_cast<const RP*>(static_cast<const T*>(a.in) + gi);
        v[i].a = mk<T>(r.x, T(0));
        v[i].b = mk<T>(r.y, T(0));
      } else if (MODE == LAT_EXTRAP_FWD) {
        const V z1 = *reinterpret_cast<const V*>(a.z1 + gi);
        const V z2 = *reinterpret_cast<const V*>(a.z2 + gi);
        v[i] = eadd(z1, escale(esub(z1, z2), a.mu));
      } else {
        v[i] = *reinterpret_cast<const V*>(static_cast<const C*>(a.in) + gi);
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i >= ept) break;
      buf[sidx(tid + i * nt)] = v[i];
    }
  }
  __syncthreads();

  if (MODE == LAT_C2C_FWD || MODE == LAT_R2C_FWD || MODE == LAT_EXTRAP_FWD) lat_fft(FWD{});
  else lat_fft(INV{});
  if (stopped) return;   // an earlier check stopped the solve: write nothing

  const T nrm = a.norm;
  if (MODE == LAT_C2C_FWD || MODE == LAT_C2C_INV || MODE == LAT_R2C_FWD ||
      MODE == LAT_EXTRAP_FWD) {
    C* out = static_cast<C*>(a.out);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i >= ept) break;
      const int e = tid + i * nt;
      *reinterpret_cast<V*>(out + gidx(e)) = escale(buf[sidx(e)], nrm);
    }
    return;
  }
  if (MODE == LAT_INV_REAL) {
    T* out = static_cast<T*>(a.out);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i >= ept) break;
      const int e = tid + i * nt;
      const V v = buf[sidx(e)];
      RP r;
      r.x = v.a.x * nrm;
      r.y = v.b.x * nrm;
      *reinterpret_cast<RP*>(out + gidx(e)) = r;
    }
    return;
  }
  if (MODE == LAT_GRAD_STEP) {
    // u = eta^k - g/L with eta^k = z1 + mu_prev (z1 - z2), written to out
    const T sg = nrm * a.inv_L;
    C* out = static_cast<C*>(a.out);
    bool bad = false;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i >= ept) break;
      const int e = tid + i * nt;
      const size_t gi = gidx(e);
      const V z1 = *reinterpret_cast<const V*>(a.z1 + gi);
      const V z2 = *reinterpret_cast<const V*>(a.z2 + gi);
      const V eta = eadd(z1, escale(esub(z1, z2), a.mu_prev));
      const V u = esub(eta, escale(buf[sidx(e)], sg));
      *reinterpret_cast<V*>(out + gi) = u;
      bad |= !(isfinite(u.a.x) && isfinite(u.a.y) && isfinite(u.b.x) && isfinite(u.b.y));
    }
    if (bad) atomicOr(a.flag, 1);
    return;
  }
  // LAT_UPDATE / LAT_UPDATE_U, in two batches of four elements: loads of the
  // iterates first.  LAT_UPDATE forms u = eta^k - g/L from the gradient with
  // eta^k = z1 + mu_prev (z1 - z2); LAT_UPDATE_U transformed u itself.
  constexpr bool FROM_U = MODE == LAT_UPDATE_U;
  // norm partials: a thread's 8 elements (at most 32 squares per norm) summed
  // in the plan's precision, the block's threads in double
  T acc0 = T(0), acc1 = T(0), acc2 = T(0);
  bool bad = false;
  const T sg = nrm * a.inv_L;
  const T lam_over_L = a.lam_dev ? T(a.lam_scale * *a.lam_dev) : a.lam_over_L;
#pragma unroll
  for (int h = 0; h < 8; h += 4) {
    V z1v[4], z2v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (h + i >= ept) break;
      const size_t gi = gidx(tid + (h + i) * nt);
      z1v[i] = *reinterpret_cast<const V*>(a.z1 + gi);
      if (!FROM_U) z2v[i] = *reinterpret_cast<const V*>(a.z2 + gi);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (h + i >= ept) break;
      const int e = tid + (h + i) * nt;
      const size_t gi = gidx(e);
      const int n0 = int((m_first + 2 * (e & (TP - 1))) & size_t(a.nz - 1));
      const V z1 = z1v[i];
      V g, eta, u;
      if (FROM_U) {
        u = escale(buf[sidx(e)], nrm);
      } else {
        g = escale(buf[sidx(e)], sg);                       // g^k = (1/L) A^H(A eta - s)
        eta = eadd(z1, escale(esub(z1, z2v[i]), a.mu_prev));
        u = esub(eta, g);
      }
      const T tau0 = a.w ? lam_over_L * a.w[n0] : lam_over_L;
      const T tau1 = a.w ? lam_over_L * a.w[n0 + 1] : lam_over_L;
      if (a.uout) *reinterpret_cast<V*>(a.uout + gi) = u;
      V z;
      z.a = soft_threshold(u.a, tau0);
      z.b = soft_threshold(u.b, tau1);
      *reinterpret_cast<V*>(a.zout + gi) = z;
      buf[sidx(e)] = eadd(z, escale(esub(z, z1), a.mu));
      if (!FROM_U && a.partial) {
        const V d = esub(z, eta);
        const V dg = eadd(d, g);
        acc0 += d.a.x * d.a.x + d.a.y * d.a.y + d.b.x * d.b.x + d.b.y * d.b.y;
        acc1 += g.a.x * g.a.x + g.a.y * g.a.y + g.b.x * g.b.x + g.b.y * g.b.y;
        acc2 += dg.a.x * dg.a.x + dg.a.y * dg.a.y + dg.b.x * dg.b.x + dg.b.y * dg.b.y;
      }
      bad |= !(isfinite(z.a.x) && isfinite(z.a.y) && isfinite(z.b.x) && isfinite(z.b.y));
    }
  }
  if (bad) atomicOr(a.flag, 1);
  __syncthreads();
  lat_fft(FWD{});
  C* out = static_cast<C*>(a.out);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (i >= ept) break;
    const int e = tid + i * nt;
    *reinterpret_cast<V*>(out + gidx(e)) = escale(buf[sidx(e)], nrm);
  }
  if (a.partial != nullptr) {
    __shared__ double red[3][32];
    const int wid = tid >> 5, lane = tid & 31;
    const int nw = (nt + 31) >> 5;
    const int lanes = min(32, nt - 32 * wid);          // lanes of this warp that exist
    const double w0 = warp_sum_lanes(double(acc0), lanes);
    const double w1 = warp_sum_lanes(double(acc1), lanes);
    const double w2 = warp_sum_lanes(double(acc2), lanes);
    if (lane == 0) { red[0][wid] = w0; red[1][wid] = w1; red[2][wid] = w2; }
    __syncthreads();
    if (wid == 0) {
      double v0 = lane < nw ? red[0][lane] : 0.0;
      double v1 = lane < nw ? red[1][lane] : 0.0;
      double v2 = lane < nw ? red[2][lane] : 0.0;
      v0 = warp_sum_lanes(v0, lanes); v1 = warp_sum_lanes(v1, lanes);
      v2 = warp_sum_lanes(v2, lanes);
      if (lane == 0) {
        const size_t blk = size_t(blockIdx.y) * gridDim.x + blockIdx.x;
        a.partial[3 * blk + 0] = v0;
        a.partial[3 * blk + 1] = v1;
        a.partial[3 * blk + 2] = v2;
      }
    }
  }
}

// prox of tau ||details(W u)||_1 per A-scan (nz contiguous samples), W the
// orthonormal Haar transform along depth: in-place lifting levels with
// stride h = 1, 2, .., nz/2 (pair (i, i + h), i a multiple of 2h, becomes
// ((x_i + x_{i+h})/sqrt 2, (x_i - x_{i+h})/sqrt 2)), the complex soft
// threshold on every coefficient but the approximation (index 0), and the
// same butterflies in reverse order, which invert them.
template <typename T>
__global__ void k_haar_prox(const cplx<T>* u, cplx<T>* z, int nz, T tau, const double* lam_dev,
                            double lam_scale) {
  extern __shared__ __align__(16) unsigned char raw[];
  cplx<T>* x = reinterpret_cast<cplx<T>*>(raw);
  const size_t col = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < nz; i += nt) x[i] = u[col * nz + i];
  __syncthreads();
  const T r = T(0.70710678118654752440);
  for (int h = 1; h < nz; h <<= 1) {
    for (int p = tid; p < nz / (2 * h); p += nt) {
      const int i = p * 2 * h;
      const cplx<T> a0 = x[i], a1 = x[i + h];
      x[i] = cscale(cadd(a0, a1), r);
      x[i + h] = cscale(csub(a0, a1), r);
    }
    __syncthreads();
  }
  const T t = lam_dev ? T(lam_scale * *lam_dev) : tau;
  for (int i = tid; i < nz; i += nt)
    if (i) x[i] = soft_threshold(x[i], t);
  __syncthreads();
  for (int h = nz >> 1; h >= 1; h >>= 1) {
    for (int p = tid; p < nz / (2 * h); p += nt) {
      const int i = p * 2 * h;
      const cplx<T> a0 = x[i], a1 = x[i + h];
      x[i] = cscale(cadd(a0, a1), r);
      x[i + h] = cscale(csub(a0, a1), r);
    }
    __syncthreads();
  }
  for (int i = tid; i < nz; i += nt) z[col * nz + i] = x[i];
}

template <typename T> cudaError_t launch_haar_prox(const cplx<T>* u, cplx<T>* z, int nz,
                                                   size_t n_ascans, T tau, const double* lam_dev,
                                                   double lam_scale, cudaStream_t s) {
  const int threads = nz / 2 >= 256 ? 256 : (nz / 2 >= 32 ? nz / 2 : 32);
  const size_t sm = size_t(nz) * sizeof(cplx<T>);
  cudaFuncSetAttribute(k_haar_prox<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  k_haar_prox<T><<<unsigned(n_ascans), threads, sm, s>>>(u, z, nz, tau, lam_dev, lam_scale);
  return cudaGetLastError();
}
template cudaError_t launch_haar_prox<float>(const float2*, float2*, int, size_t, float,
                                             const double*, double, cudaStream_t);
template cudaError_t launch_haar_prox<double>(const double2*, double2*, int, size_t, double,
                                              const double*, double, cudaStream_t);

template <typename T> size_t lat_smem_bytes(int L, int TP) {
  int lg = 0, r3 = 0;
  fft_length(L, &lg, &r3);
  return size_t(padded_rows(L)) * TP * sizeof(cpair<T>) +
         size_t(twiddle_entries(L, lg, r3)) * sizeof(cplx<T>);
}

template <typename T, int MODE, int LOGL, int LOGTP, bool C16 = false>
static cudaError_t launch_lat_tile(const LatArgs<T>& a, cudaStream_t s) {
  const int threads = (a.L >= 8 ? a.L / 8 : 1) * a.TZ;
  const size_t sm = lat_smem_bytes<T>(a.L, a.TZ);
  auto* kern = k_lat<T, MODE, LOGL, LOGTP, C16>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  dim3 grid(a.M / (2 * a.TZ), a.B);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
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

// The FP32 solve passes at the tiles of the 1024-wide B-scans (L = 1024, 4
// pair-columns), the 512-wide ones and the 256 x 256 volumes (L = 512 or 256, 8
// pair-columns) run compile-time-length transforms, at L = 1024 and 256 in the
// column-split radix-16 form when the plan chose it (a.radix16); every other
// case the runtime-length ones.
template <typename T, int MODE>
static cudaError_t launch_lat_mode(const LatArgs<T>& a, cudaStream_t s) {
  constexpr bool hot = std::is_same<T, float>::value &&
                       (MODE == LAT_UPDATE || MODE == LAT_UPDATE_U || MODE == LAT_C2C_FWD ||
                        MODE == LAT_C2C_INV);
  if constexpr (hot) {
    if (!a.r3 && a.L == 1024 && a.TZ == 4)
      return a.radix16 ? launch_lat_tile<T, MODE, 10, 2, true>(a, s)
                       : launch_lat_tile<T, MODE, 10, 2>(a, s);
    if (!a.r3 && a.L == 512 && a.TZ == 8) return launch_lat_tile<T, MODE, 9, 3>(a, s);
    if (!a.r3 && a.L == 256 && a.TZ == 8)
      return a.radix16 ? launch_lat_tile<T, MODE, 8, 3, true>(a, s)
                       : launch_lat_tile<T, MODE, 8, 3>(a, s);
  }
  return launch_lat_tile<T, MODE, 0, 0>(a, s);
}

template <typename T> cudaError_t launch_lat(int mode, const LatArgs<T>& a, cudaStream_t s) {
  switch (mode) {
    case LAT_C2C_FWD: return launch_lat_mode<T, LAT_C2C_FWD>(a, s);
    case LAT_C2C_INV: return launch_lat_mode<T, LAT_C2C_INV>(a, s);
    case LAT_R2C_FWD: return launch_lat_mode<T, LAT_R2C_FWD>(a, s);
    case LAT_INV_REAL: return launch_lat_mode<T, LAT_INV_REAL>(a, s);
    case LAT_UPDATE: return launch_lat_mode<T, LAT_UPDATE>(a, s);
    case LAT_GRAD_STEP: return launch_lat_mode<T, LAT_GRAD_STEP>(a, s);
    case LAT_EXTRAP_FWD: return launch_lat_mode<T, LAT_EXTRAP_FWD>(a, s);
    case LAT_UPDATE_U: return launch_lat_mode<T, LAT_UPDATE_U>(a, s);
  }
  return cudaErrorInvalidValue;
}

template cudaError_t launch_lat<float>(int, const LatArgs<float>&, cudaStream_t);
template cudaError_t launch_lat<double>(int, const LatArgs<double>&, cudaStream_t);

}  // namespace isam
