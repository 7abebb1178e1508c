// Internal structures shared by the kernel translation units and the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace isam {

// Per-plan constants of the Stolt map in oversampled-grid units (K = 2 nz,
// grid unit = dk):  p_j = sqrt(4 kappa_j^2 - a) with kappa_j = k_j / dk and
// a = (q / dk)^2 = Qx mx^2 + Qy my^2.  Written as p_j = c0 + 2 j - d_j with
// c0 = 2 kappa_0 mod K (I0 + f0) and d_j = a / (2 kappa_j + p_j) >= 0.  The
// focus phase is e^{j 2 pi d_j zeta}, zeta = dk z0 / (2 pi).
struct StoltConst {
  // float-float copies for the FP32 path
  float kap_hi, kap_lo;
  float qx_hi, qx_lo, qy_hi, qy_lo;
  float zeta_hi, zeta_lo;
  float f0;
  float B;        // 2 kappa_0 - c0, an integer multiple of K (exact in float)
  // double copies for the FP64 path
  double kap, Qx, Qy, zeta, c0d;
  int I0;
  int K, logK, nx, ny, nk, nz, J;
  int focus;      // z0 != 0
};

// Stolt position and spectral phase of one (|q|, k_j) sample (mfl == INT_MIN:
// evanescent).  Tabulated per plan when the table is small (B-scans).
template <typename T> struct StoltEntry;
template <> struct alignas(16) StoltEntry<float> { int mfl; float frac; float2 ph; };
template <> struct alignas(16) StoltEntry<double> { int mfl; int pad; double frac; double2 ph; };

template <typename T> struct Tables {
  T* scale = nullptr;        // [nz]  s(n - nz/2) / sqrt(nz)
  cplx<T>* disp = nullptr;   // [nk]  e^{j phi(k_j)}
  StoltEntry<T>* stab = nullptr;  // [(ny/2+1)(nx/2+1)][nk] or null (computed on the fly)
  cplx<T>* filt = nullptr;   // [(ny/2+1)(nx/2+1)][nk] filter B of Eq. 3, or null (B = 1);
                             // folded into stab's phases when stab exists
};

// Min-max coefficients as polynomials in the fractional offset f.  With
// x = f - 1/2 and y = 4 x^2 the symmetric design gives, for tap pairs
// (p, J-1-p):  c_p = E_p(y) + x Q_p(y),  c_{J-1-p} = E_p(y) - x Q_p(y),
// E_p of degree DE and Q_p of degree DO, fitted in FP64 to exact min-max
// solutions at Chebyshev nodes (fit error 7.6e-9 relative in FP32 form,
// 1.4e-14 in FP64 form for J <= 8).
template <typename T> struct PolyDeg;
template <> struct PolyDeg<float> { static constexpr int DE = 4, DO = 3; };
template <> struct PolyDeg<double> { static constexpr int DE = 6, DO = 5; };
constexpr int POLY_MAXP = 4;
template <typename T> struct Poly {
  T e[POLY_MAXP][7];
  T o[POLY_MAXP][6];
};

// Lateral pass modes.
enum LatMode : int {
  LAT_C2C_FWD = 0,   // X = F x
  LAT_C2C_INV = 1,   // X = F^-1 x
  LAT_R2C_FWD = 2,   // real input, X = F x
  LAT_INV_REAL = 3,  // real output, Re(F^-1 x)
  LAT_UPDATE = 5,    // FISTA step in image space between F^-1 and F
  LAT_GRAD_STEP = 6, // u = eta^k - g/L after F^-1 (no threshold, no F): other priors
  LAT_EXTRAP_FWD = 7,// X = F(z1 + mu (z1 - z2)): the momentum step, then F
  LAT_UPDATE_U = 8,  // as LAT_UPDATE from u_hat = eta_hat^k - G/L: u = F^-1 u_hat (no z2,
                     // no norm partials)
};

template <typename T> struct LatArgs {
  const void* in;        // complex (or real for R2C)
  void* out;             // complex (or real for INV_REAL)
  int B, L, logL, M;     // data viewed as [B][L][M], transform along L
  int r3;                // L = 3 * 2^logL (else L = 2^logL)
  int TZ, logTZ;         // pair-columns (2 columns each) per block
  T norm;                // 1/sqrt(L)
  // LAT_UPDATE
  const cplx<T>* z1;     // z^{k-1}
  const cplx<T>* z2;     // z^{k-2}
  cplx<T>* zout;         // z^k (may alias z2)
  const T* w;            // [nz] weights or null
  int nz;
  T inv_L, lam_over_L, mu_prev, mu;
  double* partial;       // [gridDim.x*gridDim.y][3] norm partials, or null
  int* flag;             // non-finite flag
  cplx<T>* uout;         // optional: u^k = eta^k - g^k before the threshold
  const double* lam_dev; // optional: lambda / L = lam_scale * (*lam_dev), read on the device
  double lam_scale;
  // FP32 compile-time tiles at L = 1024 and 256: 1 runs the column-split
  // radix-16 transforms, 0 the radix-8 column-pair ones; ignored elsewhere
  int radix16;
  // solve with the device-side stop rule (see StopRule): a nonzero *stop, read
  // after the wait for the previous kernel, makes the launch return at once;
  // null elsewhere
  const int* stop;
};

// Columns q and -q share the Stolt map; the axial kernels process them as a
// pair (pairs[i] = (c1, c2), c2 == c1 for self-paired columns).
template <typename T> struct AxArgs {
  const cplx<T>* in;
  cplx<T>* out;
  StoltConst sc;
  Tables<T> tab;
  Poly<T> poly;
  const int2* pairs;
  // fused kernel only: lateral spectrum of the data, F s_d ([ny][nx][nk]; the
  // first column of each pair is read)
  const cplx<T>* sdh;
  // fused kernel: 0 writes G; else writes u_hat = in - u_hat_scale * G (the
  // lateral spectrum of eta^k - g/L, u_hat_scale = 1/L)
  T u_hat_scale;
  // fused kernel, optional: the model spectra S = phase . N(eta_hat)
  // ([ny][nx][nk], as k_ax_fwd writes them)
  cplx<T>* s_out;
  // FP32, K = 2048 or 4096: 1 runs the column-split radix-16 transforms, 0 the
  // radix-8 column-pair ones (the plan's tuned choice); ignored elsewhere
  int radix16;
  // fused kernel in a solve with the device-side stop rule: as LatArgs::stop
  const int* stop;
};

// launchers (return cudaGetLastError())
template <typename T> cudaError_t launch_lat(int mode, const LatArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_ax_fwd(const AxArgs<T>& a, int npairs, cudaStream_t s);
template <typename T> cudaError_t launch_ax_adj(const AxArgs<T>& a, int npairs, cudaStream_t s);
template <typename T> cudaError_t launch_ax_fused(const AxArgs<T>& a, int npairs, cudaStream_t s);
template <typename T> size_t ax_smem_bytes(int K, int nk, bool adj);

// Stolt table: entry [(|my| (nx/2+1) + |mx|) nk + j] for every |q| class
template <typename T> cudaError_t launch_stolt_table(const AxArgs<T>& a, StoltEntry<T>* out,
                                                     cudaStream_t s);

// FP64 exact min-max coefficients at offsets f[0..n) (device), out[i*J + l]
cudaError_t minmax_nodes(int nz, int K, int J, const double* f, int n, double* out,
                         cudaStream_t s);

// reductions / elementwise
template <typename T> cudaError_t launch_max_abs(const cplx<T>* x, size_t n, double* partial,
                                                  int nblocks, double* out, cudaStream_t s);
template <typename T> cudaError_t launch_norm2(const cplx<T>* x, size_t n, double* partial,
                                                int nblocks, double* out, cudaStream_t s);
// The stop rule of Eq. 15 evaluated on the device by the reduction of a
// check iteration: r_r = ||z - eta|| / (max(||g/L||, ||z - eta + g/L||) + eps)
// from the three sums, written to *rr; when r_r < tol, stop[0] = 1 and
// stop[1] = iter.  Once stop[0] is set, later checks (whose partials were not
// written) leave everything as it is.  stop null: the plain sums only.
struct StopRule {
  int* stop;       // [2] device: stopped flag, iteration of the stop
  double* rr;      // device: r_r of the latest evaluated check
  double tol, eps;
  int iter;
};
cudaError_t launch_sum3(const double* partial, int n, double* out, const StopRule& sr,
                        cudaStream_t s);
// out = the iterate of the stopping check: the two iterate buffers alternate,
// so z^{stop[1]} is in a (z^last) when last - stop[1] is even, else in b; a
// solve that did not stop (stop[0] == 0) returns a
template <typename T> cudaError_t launch_select_iterate(const cplx<T>* a, const cplx<T>* b,
                                                         cplx<T>* out, size_t n, const int* stop,
                                                         int last, cudaStream_t s);
template <typename T> cudaError_t launch_wl1(const cplx<T>* x, size_t n, const T* w, int nz,
                                             double* partial, int nblocks, double* out,
                                             cudaStream_t s);
template <typename T> cudaError_t launch_scale(cplx<T>* x, size_t n, const double* denom,
                                                cudaStream_t s);
template <typename T> cudaError_t launch_extrapolate(const cplx<T>* z1, const cplx<T>* z2, T mu,
                                                     cplx<T>* out, size_t n, cudaStream_t s);
template <typename Tsrc, typename Tdst> cudaError_t launch_convert(const cplx<Tsrc>* x,
                                                                   cplx<Tdst>* y, size_t n,
                                                                   cudaStream_t s);
template <typename T> cudaError_t launch_fill_start(cplx<T>* x, size_t n, cudaStream_t s);

template <typename T> cudaError_t launch_rsub(const T* a, const T* b, T* y, size_t n,
                                               cudaStream_t s);
template <typename T> cudaError_t launch_caxpy(const cplx<T>* x, const cplx<T>* v, T alpha,
                                                cplx<T>* y, size_t n, cudaStream_t s);

// calibration (k_calib.cu): <dA/dtheta x, y> partial sums per column pair
template <typename T> struct ParamArgs {
  cplx<T>* su;           // S_x [ny][nx][nk]; overwritten by (S(q) + conj S(-q))/2 if write_fa
  const cplx<T>* se;     // S_eta of a second model spectrum, or null
  const cplx<T>* fd;     // lateral spectrum of data (all columns), or null
  T fd_sign;             // data term: F1 = Re-spectrum(se) + fd_sign * fd
  const int2* pairs;
  StoltConst sc;
  double* partial;       // [npairs][5], accumulated
  int write_fa;
};
template <typename T> cudaError_t launch_param_reduce(const ParamArgs<T>& a, int npairs,
                                                      cudaStream_t s);
template <typename T> cudaError_t launch_st_vjp(const cplx<T>* u, const cplx<T>* zbar, const T* w,
                                                T lam_over_L, int nz, cplx<T>* out, size_t n,
                                                cudaStream_t s);
template <typename T> cudaError_t launch_bwd_combine(const cplx<T>* ubar, const cplx<T>* b,
                                                     T inv_L, T mu, cplx<T>* zb1, cplx<T>* zb2,
                                                     size_t n, cudaStream_t s);

// prox of tau ||details(W u)||_1, W the orthonormal Haar transform along depth
// of each A-scan (k_lateral.cu); tau = lam_scale * (*lam_dev) when lam_dev
template <typename T> cudaError_t launch_haar_prox(const cplx<T>* u, cplx<T>* z, int nz,
                                                   size_t n_ascans, T tau, const double* lam_dev,
                                                   double lam_scale, cudaStream_t s);

// total-variation prox pieces (k_prior.cu); tau = lam_scale * (*lam_dev) when lam_dev
template <typename T> cudaError_t launch_tv_primal(const cplx<T>* u, const cplx<T>* rx,
                                                   const cplx<T>* rz, T tau, const double* lam_dev,
                                                   double lam_scale, cplx<T>* w, int nx, int nz,
                                                   size_t n, cudaStream_t s);
template <typename T> cudaError_t launch_tv_dual(const cplx<T>* w, cplx<T>* px, cplx<T>* pz,
                                                 cplx<T>* rx, cplx<T>* rz, T tau,
                                                 const double* lam_dev, double lam_scale, T beta,
                                                 int nx, int nz, size_t n, cudaStream_t s);

// Eq. 9 direct reconstruction (k_direct.cu)
template <typename T> cudaError_t launch_dc_ifft(const T* s, cplx<T>* out, const cplx<T>* disp,
                                                 const cplx<T>* post, int nk, int nz, int lognz,
                                                 int n_ascans, cudaStream_t st);

int lat_tile(int L, int M);   // pair-columns per block of a lateral pass
template <typename T> size_t lat_smem_bytes(int L, int TP);
// L = 2^log2 or 3 * 2^log2 (log2 >= 3): *log2, *r3; false for other lengths
bool fft_length(int L, int* log2, int* r3);

}  // namespace isam
