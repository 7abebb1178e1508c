// C ABI of the library: plans, forward/adjoint operators and the MBIR solve.
//
// Per application of A (B-scan, ny = 1) three kernels run:
//   lateral FFT (x) -> k_ax_fwd (Stolt NUFFT + phases) -> lateral IFFT + Re;
// per application of A^H:
//   lateral FFT of the real spectra -> k_ax_adj -> lateral IFFT;
// per FISTA iteration (Alg. 1) two:
//   k_ax_fused (forward NUFFT, residual in the lateral-frequency domain,
//   adjoint NUFFT) -> LAT_UPDATE (lateral IFFT, FISTA step, lateral FFT).
// Volumes (ny > 1) add separate x passes around the y-axis update pass.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>

#include <algorithm>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "isam.h"
#include "internal.cuh"

using namespace isam;

namespace {

template <typename T> struct Impl {
  Tables<T> tab{};
  cplx<T>* eta_hat = nullptr;   // [ny][nx][nz]  lateral spectrum of the image
  cplx<T>* spec = nullptr;      // [ny][nx][nk]  complex spectra (S, then R_hat)
  cplx<T>* grad = nullptr;      // [ny][nx][nz]  G_hat / image temporaries
  cplx<T>* sdh = nullptr;       // [ny][nx][nk]  F s_d of the current solve
  cplx<T>* zA = nullptr;        // solver iterates
  cplx<T>* zB = nullptr;
  T* s_tmp = nullptr;           // [ny][nx][nk]  real spectra temporary
  T* s_host_stage = nullptr;    // device copy of host s_d for isam_solve_host
  cplx<T>* out_stage = nullptr; // device image for isam_solve_host
  // calibration: second complex spectrum, segment storage of the unrolled
  // gradient (u^k and eta_hat^k of up to seg_cap iterations), adjoint images
  cplx<T>* spec2 = nullptr;
  cplx<T>* seg = nullptr;
  int seg_cap = 0;
  cplx<T>* cal = nullptr;       // [5][n_img]: zbar x 3, ubar, b
  cplx<T>* dc_post = nullptr;   // [nz] output phase of the Eq. 9 reconstruction
  cplx<T>* tv = nullptr;        // [5][n_img]: TV dual p_x, p_z, momentum r_x, r_z, primal w
  bool ready = false;
};

}  // namespace

struct isam_plan {
  isam_params p{};
  int nx = 0, ny = 0, nk = 0, nz = 0, K = 0, J = 6;
  int device = 0;
  cudaStream_t stream = nullptr;
  StoltConst sc{};
  Impl<float> f32;
  Impl<double> f64;
  Poly<float> poly32{};
  Poly<double> poly64{};
  int2* pairs = nullptr;        // (q, -q) column pairs of the axial kernels
  int npairs = 0;
  double* partial = nullptr;    // reduction partials
  int n_partial = 0;
  double* dscal = nullptr;      // device scalars [8]
  double* hscal = nullptr;      // pinned host mirror [8]
  int* flag = nullptr;          // device non-finite flag
  // device-side stop rule of the solve: [stopped, iteration] on the device,
  // pinned mirrors of the pending check's outcome [0, 2) and of the final one
  // [2, 4), and an event after the pending check's copy
  int* dstop = nullptr;
  int* hstop = nullptr;
  cudaEvent_t ev_check = nullptr;
  double L_cache = 0.0;
  // autotuned choices (0: the built-in heuristics): lateral update tile width
  // and whether the fused kernel reads the Stolt table (1) or evaluates (2)
  int tune_tp = 0;
  int tune_table = 0;
  // FFT radix of the FP32 axial transforms at K = 2048 / 4096 and of the
  // compile-time lateral tiles at L = 1024 / 256: 16 (column-split radix-16
  // passes, the default) or 8 (radix-8 column-pair passes)
  int tune_radix_ax = 16;
  int tune_radix_lat = 16;
  int batch_refs = 0;           // batches whose graph records this plan's kernels
  // filter B of Eq. 3 per |q| class, interleaved (re, im); empty: B = 1
  std::vector<double> filt_host;
  double* cpartial = nullptr;   // [npairs][5] calibration partial sums
  int64_t launches = 0;
  size_t n_img = 0, n_spec = 0;
  // opt-in per-kernel-class timing with CUDA events on the plan's stream
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<cudaEvent_t> ev_pending;   // start, stop pairs
  std::vector<int> ev_class;
  double prof_ms[ISAM_KCLASS_COUNT] = {0};
  int64_t prof_n[ISAM_KCLASS_COUNT] = {0};
};

namespace {

constexpr int RED_BLOCKS = 1024;
// Stolt position/phase tables are kept when at most this large or at most
// one image array of the plan (16 B per (|q| class, k) sample against 8 or 16
// B per image sample: every B-scan and the 256^2 x 2048 volume); larger
// geometries evaluate positions in the kernels.
constexpr size_t kStoltTableMaxBytes = size_t(64) << 20;
// power iteration used when the caller gives no L: the top eigenvalues of
// A^H A lie close together, so convergence takes hundreds of steps
constexpr int kPowerIters = 1000;
constexpr double kPowerRtol = 1e-11;

isam_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return ISAM_OK;
  if (e == cudaErrorMemoryAllocation) return ISAM_ERR_OOM;
  return ISAM_ERR_CUDA;
}

cudaEvent_t take_event(isam_plan* P) {
  cudaEvent_t e = nullptr;
  if (!P->ev_pool.empty()) {
    e = P->ev_pool.back();
    P->ev_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    e = nullptr;
  }
  return e;
}

// Accumulate the elapsed times of recorded launches (call after a stream sync).
void harvest_events(isam_plan* P) {
  for (size_t i = 0; i + 1 < P->ev_pending.size(); i += 2) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, P->ev_pending[i], P->ev_pending[i + 1]) == cudaSuccess) {
      P->prof_ms[P->ev_class[i / 2]] += ms;
      P->prof_n[P->ev_class[i / 2]] += 1;
    }
    P->ev_pool.push_back(P->ev_pending[i]);
    P->ev_pool.push_back(P->ev_pending[i + 1]);
  }
  P->ev_pending.clear();
  P->ev_class.clear();
}

// Count (and, when profiling, time) one kernel launch of class `cls`.
template <typename F> isam_status launch(isam_plan* P, int cls, F&& f) {
  P->launches += 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (P->prof) {
    e0 = take_event(P);
    e1 = take_event(P);
    if (e0 && e1) cudaEventRecord(e0, P->stream);
  }
  cudaError_t err = f();
  if (P->prof && e0 && e1) {
    cudaEventRecord(e1, P->stream);
    P->ev_pending.push_back(e0);
    P->ev_pending.push_back(e1);
    P->ev_class.push_back(cls);
  }
  return from_cuda(err);
}

#define ISAM_TRY(expr)                              \
  do {                                              \
    isam_status _st = (expr);                       \
    if (_st != ISAM_OK) return _st;                 \
  } while (0)
#define CUDA_TRY(expr) ISAM_TRY(from_cuda(expr))

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) { int r = 0; while ((1 << r) < v) ++r; return r; }

// Device memory of plans: cudaMalloc, or the allocator installed with
// isam_set_allocator.  Every block from an installed allocator is recorded
// with the free function that owns it, so it is returned to that allocator
// even after another one has been installed.
struct AllocHook {
  isam_alloc_fn alloc = nullptr;
  isam_free_fn free = nullptr;
  void* ctx = nullptr;
};
std::mutex g_alloc_mu;
AllocHook g_alloc;
std::unordered_map<void*, AllocHook>& alloc_owners() {
  static std::unordered_map<void*, AllocHook> m;
  return m;
}

isam_status dalloc_bytes(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return ISAM_OK;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  if (g_alloc.alloc) {
    *p = g_alloc.alloc(bytes, g_alloc.ctx);
    if (!*p) return ISAM_ERR_OOM;
    alloc_owners()[*p] = g_alloc;
    return ISAM_OK;
  }
  return from_cuda(cudaMalloc(p, bytes));
}

void dfree(void* p) {
  if (!p) return;
  AllocHook h;
  bool hooked = false;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    auto it = alloc_owners().find(p);
    if (it != alloc_owners().end()) {
      h = it->second;
      hooked = true;
      alloc_owners().erase(it);
    }
  }
  if (hooked) h.free(p, h.ctx);
  else cudaFree(p);
}

template <typename T> isam_status dalloc(T** p, size_t n) {
  void* v = nullptr;
  const isam_status st = dalloc_bytes(&v, n * sizeof(T));
  *p = static_cast<T*>(v);
  return st;
}

template <typename T> void impl_free(Impl<T>& im) {
  dfree(im.tab.scale); dfree(im.tab.disp); dfree(im.tab.stab); dfree(im.tab.filt);
  dfree(im.eta_hat); dfree(im.spec); dfree(im.grad); dfree(im.sdh);
  dfree(im.zA); dfree(im.zB); dfree(im.s_tmp);
  dfree(im.s_host_stage); dfree(im.out_stage);
  dfree(im.spec2); dfree(im.seg); dfree(im.cal); dfree(im.dc_post); dfree(im.tv);
  im = Impl<T>();
}

double host_kb_scale(int n, int K, int J) {
  const double alpha = 2.34 * J;
  const double v = double(n) / double(K);
  const double r = sqrt(alpha * alpha - (M_PI * J * v) * (M_PI * J * v));
  return (sinh(alpha) / alpha) / (sinh(r) / r);
}

template <typename T> bool precision_fits(const isam_plan* P) {
  return ax_smem_bytes<T>(P->K, P->nk, true) <= 227u * 1024u &&
         ax_smem_bytes<T>(P->K, P->nk, false) <= 227u * 1024u;
}

// Tables that depend on the dispersion coefficients and the focal depth:
// e^{j phi(k_j)} (Eq. 7) and, when kept, the Stolt position/phase table.
// Asynchronous on the plan's stream (the host vector is copied synchronously).
template <typename T> isam_status phase_tables(isam_plan* P, Impl<T>& im) {
  const isam_params& p = P->p;
  const size_t rows = size_t(P->ny / 2 + 1) * (P->nx / 2 + 1);
  // filter B (before the Stolt table, which folds it into its phases)
  if (P->filt_host.empty()) {
    dfree(im.tab.filt);
    im.tab.filt = nullptr;
  } else {
    std::vector<cplx<T>> h(rows * P->nk);
    for (size_t i = 0; i < h.size(); ++i)
      h[i] = mk<T>(T(P->filt_host[2 * i]), T(P->filt_host[2 * i + 1]));
    if (!im.tab.filt) ISAM_TRY(dalloc(&im.tab.filt, h.size()));
    CUDA_TRY(cudaMemcpy(im.tab.filt, h.data(), sizeof(cplx<T>) * h.size(), cudaMemcpyHostToDevice));
  }
  {
    std::vector<cplx<T>> h(P->nk);
    const double dk = (p.k_max - p.k_min) / (P->nk - 1);
    const double k0 = 0.5 * (p.k_min + p.k_max);
    for (int j = 0; j < P->nk; ++j) {
      const double d = (p.k_min + dk * j) - k0;
      double phi = 0.0, pw = 1.0;
      for (int i = 0; i < p.n_disp; ++i) { pw *= d; phi += p.disp[i] * pw; }
      h[j] = mk<T>(T(cos(phi)), T(sin(phi)));
    }
    if (!im.tab.disp) ISAM_TRY(dalloc(&im.tab.disp, P->nk));
    CUDA_TRY(cudaMemcpy(im.tab.disp, h.data(), sizeof(cplx<T>) * P->nk, cudaMemcpyHostToDevice));
  }
  {
    const size_t bytes = rows * P->nk * sizeof(StoltEntry<T>);
    const size_t cap = std::max(kStoltTableMaxBytes, P->n_img * sizeof(cplx<T>));
    if (bytes <= cap && !(p.flags & ISAM_FLAG_NO_STOLT_TABLE)) {
      if (!im.tab.stab) ISAM_TRY(dalloc(&im.tab.stab, rows * P->nk));
      AxArgs<T> a{};
      a.sc = P->sc;
      a.tab = im.tab;
      CUDA_TRY(launch_stolt_table<T>(a, im.tab.stab, P->stream));
    }
  }
  return ISAM_OK;
}

template <typename T> isam_status impl_init(isam_plan* P, Impl<T>& im) {
  if (im.ready) return ISAM_OK;
  if (!precision_fits<T>(P)) return ISAM_ERR_UNSUPPORTED;
  // scaling s(n - nz/2) / sqrt(nz)
  {
    std::vector<T> h(P->nz);
    for (int n = 0; n < P->nz; ++n)
      h[n] = T(host_kb_scale(n - P->nz / 2, P->K, P->J) / sqrt(double(P->nz)));
    ISAM_TRY(dalloc(&im.tab.scale, P->nz));
    CUDA_TRY(cudaMemcpy(im.tab.scale, h.data(), sizeof(T) * P->nz, cudaMemcpyHostToDevice));
  }
  ISAM_TRY(phase_tables<T>(P, im));
  ISAM_TRY(dalloc(&im.eta_hat, P->n_img));
  ISAM_TRY(dalloc(&im.spec, P->n_spec));
  ISAM_TRY(dalloc(&im.grad, P->n_img));
  CUDA_TRY(cudaStreamSynchronize(P->stream));
  harvest_events(P);
  im.ready = true;
  return ISAM_OK;
}

template <typename T> Impl<T>& impl_of(isam_plan* P);
template <> Impl<float>& impl_of<float>(isam_plan* P) { return P->f32; }
template <> Impl<double>& impl_of<double>(isam_plan* P) { return P->f64; }

// ----------------------------------------------------------------------------
// launch helpers
// ----------------------------------------------------------------------------
template <typename T>
LatArgs<T> lat_args(int B, int L, int M, const void* in, void* out) {
  LatArgs<T> a{};
  a.in = in; a.out = out;
  a.B = B; a.L = L; a.M = M;
  fft_length(L, &a.logL, &a.r3);
  a.TZ = lat_tile(L, M); a.logTZ = ilog2(a.TZ);
  a.norm = T(1.0 / sqrt(double(L)));
  return a;
}

template <typename T> isam_status lat(isam_plan* P, int mode, const LatArgs<T>& a) {
  const int cls = mode == LAT_UPDATE || mode == LAT_UPDATE_U ? ISAM_KCLASS_LAT_UPDATE
                                                             : ISAM_KCLASS_LAT_FFT;
  LatArgs<T> b = a;
  b.radix16 = P->tune_radix_lat == 16 ? 1 : 0;
  return launch(P, cls, [&] { return launch_lat<T>(mode, b, P->stream); });
}

template <typename T> const Poly<T>& poly_of(const isam_plan* P);
template <> const Poly<float>& poly_of<float>(const isam_plan* P) { return P->poly32; }
template <> const Poly<double>& poly_of<double>(const isam_plan* P) { return P->poly64; }

template <typename T> AxArgs<T> ax_args(isam_plan* P, const Impl<T>& im, const cplx<T>* in,
                                       cplx<T>* out) {
  AxArgs<T> a{};
  a.in = in; a.out = out; a.sc = P->sc; a.tab = im.tab;
  a.poly = poly_of<T>(P);
  a.pairs = P->pairs;
  if (P->tune_table == 2) a.tab.stab = nullptr;
  a.radix16 = P->tune_radix_ax == 16 ? 1 : 0;
  return a;
}

// F_lat x (image or spectra layout with inner width W), possibly real input
template <typename T> isam_status lat_forward(isam_plan* P, Impl<T>& im, const void* in,
                                              cplx<T>* out, int W, bool real_in) {
  const int m0 = real_in ? LAT_R2C_FWD : LAT_C2C_FWD;
  (void)im;
  if (P->ny == 1) return lat<T>(P, m0, lat_args<T>(1, P->nx, W, in, out));
  ISAM_TRY(lat<T>(P, m0, lat_args<T>(P->ny, P->nx, W, in, out)));
  return lat<T>(P, LAT_C2C_FWD, lat_args<T>(1, P->ny, P->nx * W, out, out));
}

// F_lat^{-1} x, complex or real (Re) output; `in` is overwritten for volumes
template <typename T> isam_status lat_inverse(isam_plan* P, Impl<T>& im, cplx<T>* in, void* out,
                                              int W, bool real_out) {
  const int m1 = real_out ? LAT_INV_REAL : LAT_C2C_INV;
  (void)im;
  if (P->ny == 1) return lat<T>(P, m1, lat_args<T>(1, P->nx, W, in, out));
  ISAM_TRY(lat<T>(P, LAT_C2C_INV, lat_args<T>(1, P->ny, P->nx * W, in, in)));
  return lat<T>(P, m1, lat_args<T>(P->ny, P->nx, W, in, out));
}

template <typename T> isam_status op_forward(isam_plan* P, const void* eta, void* s) {
  Impl<T>& im = impl_of<T>(P);
  ISAM_TRY(lat_forward<T>(P, im, eta, im.eta_hat, P->nz, false));
  ISAM_TRY(launch(P, ISAM_KCLASS_AX_FWD, [&] {
    return launch_ax_fwd<T>(ax_args<T>(P, im, im.eta_hat, im.spec), P->npairs, P->stream);
  }));
  return lat_inverse<T>(P, im, im.spec, s, P->nk, true);
}

template <typename T> isam_status op_adjoint(isam_plan* P, const void* s, void* eta) {
  Impl<T>& im = impl_of<T>(P);
  ISAM_TRY(lat_forward<T>(P, im, s, im.spec, P->nk, true));
  ISAM_TRY(launch(P, ISAM_KCLASS_AX_ADJ, [&] {
    return launch_ax_adj<T>(ax_args<T>(P, im, im.spec, im.grad), P->npairs, P->stream);
  }));
  return lat_inverse<T>(P, im, im.grad, eta, P->nz, false);
}

template <typename T> isam_status max_abs_dev(isam_plan* P, const cplx<T>* x, double* out_host) {
  P->launches += 1;   // two kernels
  ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
    return launch_max_abs<T>(x, P->n_img, P->partial, RED_BLOCKS, P->dscal, P->stream);
  }));
  CUDA_TRY(cudaMemcpyAsync(P->hscal, P->dscal, sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  CUDA_TRY(cudaStreamSynchronize(P->stream));
  harvest_events(P);
  *out_host = P->hscal[0];
  return ISAM_OK;
}

// 1/2 ||A eta - s_d||^2 (the data term of Eq. 12) and the residual spectra
// A eta - s_d, in r_out or in the plan's spectra temporary
template <typename T> isam_status fidelity_impl(isam_plan* P, const void* eta, const T* s_d,
                                                T* r_out, double* value) {
  Impl<T>& im = impl_of<T>(P);
  T* r = r_out;
  if (!r) {
    if (!im.s_tmp) ISAM_TRY(dalloc(&im.s_tmp, P->n_spec));
    r = im.s_tmp;
  }
  ISAM_TRY(op_forward<T>(P, eta, r));
  ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] { return launch_rsub<T>(r, s_d, r, P->n_spec, P->stream); }));
  P->launches += 1;   // two kernels
  ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
    return launch_norm2<T>(reinterpret_cast<const cplx<T>*>(r), P->n_spec / 2, P->partial,
                           RED_BLOCKS, P->dscal + 5, P->stream);
  }));
  CUDA_TRY(cudaMemcpyAsync(P->hscal + 5, P->dscal + 5, sizeof(double), cudaMemcpyDeviceToHost,
                           P->stream));
  CUDA_TRY(cudaStreamSynchronize(P->stream));
  harvest_events(P);
  *value = 0.5 * P->hscal[5] * P->hscal[5];
  return ISAM_OK;
}

// power iteration for ||A^H A|| in precision T
template <typename T> isam_status power_iteration(isam_plan* P, int iters, double rtol,
                                                  const void* v0, int v0_double, double* L_out) {
  Impl<T>& im = impl_of<T>(P);
  ISAM_TRY(impl_init<T>(P, im));
  if (!im.zA) ISAM_TRY(dalloc(&im.zA, P->n_img));
  if (!im.zB) ISAM_TRY(dalloc(&im.zB, P->n_img));
  if (!im.s_tmp) ISAM_TRY(dalloc(&im.s_tmp, P->n_spec));
  cudaStream_t s = P->stream;
  if (v0) {
    const bool same = (sizeof(T) == 8) == (v0_double != 0);
    if (same) {
      CUDA_TRY(cudaMemcpyAsync(im.zA, v0, sizeof(cplx<T>) * P->n_img, cudaMemcpyDeviceToDevice, s));
    } else if (sizeof(T) == 8) {
      CUDA_TRY((launch_convert<float, double>(static_cast<const float2*>(v0),
                                              reinterpret_cast<double2*>(im.zA), P->n_img, s)));
    } else {
      CUDA_TRY((launch_convert<double, float>(static_cast<const double2*>(v0),
                                              reinterpret_cast<float2*>(im.zA), P->n_img, s)));
    }
  } else {
    CUDA_TRY(launch_fill_start<T>(im.zA, P->n_img, s));
  }
  P->launches += 4;
  CUDA_TRY(launch_norm2<T>(im.zA, P->n_img, P->partial, RED_BLOCKS, P->dscal, s));
  CUDA_TRY(launch_scale<T>(im.zA, P->n_img, P->dscal, s));
  double L = 0.0, L_prev = 0.0;
  for (int it = 0; it < iters; ++it) {
    ISAM_TRY(op_forward<T>(P, im.zA, im.s_tmp));
    ISAM_TRY(op_adjoint<T>(P, im.s_tmp, im.zB));
    P->launches += 3;
    CUDA_TRY(launch_norm2<T>(im.zB, P->n_img, P->partial, RED_BLOCKS, P->dscal, s));
    CUDA_TRY(launch_scale<T>(im.zB, P->n_img, P->dscal, s));
    CUDA_TRY(cudaMemcpyAsync(P->hscal, P->dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    harvest_events(P);
    L = P->hscal[0];
    std::swap(im.zA, im.zB);
    if (L == 0.0) break;
    if (fabs(L - L_prev) <= rtol * L) break;
    L_prev = L;
  }
  *L_out = L;
  return ISAM_OK;
}

// ----------------------------------------------------------------------------
// FISTA (Alg. 1)
// ----------------------------------------------------------------------------
// One iteration of Alg. 1: the fused gradient kernel on eta_hat^k (ehat_in,
// default the plan's buffer), then the lateral update, which writes z^k to
// zout, eta_hat^{k+1} to ehat_out (default the plan's buffer) and, when
// u_out is given, u^k = eta^k - g^k (before the threshold).
template <typename T> isam_status fista_iteration(isam_plan* P, Impl<T>& im,
                                                  const cplx<T>* z1, const cplx<T>* z2,
                                                  cplx<T>* zout, const T* w, double lam,
                                                  double L, double mu_prev, double mu,
                                                  bool norms, const cplx<T>* ehat_in = nullptr,
                                                  cplx<T>* ehat_out = nullptr,
                                                  cplx<T>* u_out = nullptr,
                                                  const double* lam_dev = nullptr,
                                                  double lam_scale = 0.0,
                                                  int prior = ISAM_PRIOR_L1,
                                                  int prior_iters = 0,
                                                  cplx<T>* s_out = nullptr,
                                                  const int* stop = nullptr,
                                                  const StopRule* stop_rule = nullptr) {
  cudaStream_t s = P->stream;
  if (!ehat_in) ehat_in = im.eta_hat;
  if (!ehat_out) ehat_out = im.eta_hat;
  // device-side stop rule (l1 prior): with stop set, every kernel of the
  // iteration writes nothing when an earlier check has stopped the solve;
  // stop_rule: the check iteration's reduction evaluates Eq. 15 (StopRule)
  AxArgs<T> ax = ax_args<T>(P, im, ehat_in, im.grad);
  ax.sdh = im.sdh;
  ax.s_out = s_out;
  ax.stop = stop;
  // l1 iterations without the residual check: the fused kernel writes the
  // lateral spectrum of u = eta^k - g/L (u_hat = eta_hat^k - G/L, linear in
  // both), so the update needs z^{k-1} only, not z^{k-2} to rebuild eta^k.
  // The check (Eq. 15) needs g and eta^k apart and takes the G path.
  const bool from_u = prior == ISAM_PRIOR_L1 && !norms;
  if (from_u) ax.u_hat_scale = T(1.0 / L);
  ISAM_TRY(launch(P, ISAM_KCLASS_AX_FUSED, [&] { return launch_ax_fused<T>(ax, P->npairs, s); }));
  if (prior == ISAM_PRIOR_HAAR_DEPTH || prior == ISAM_PRIOR_TV) {
    // u^k = eta^k - g/L in image space (in place over G_hat), the Haar prox to
    // z^k, then eta_hat^{k+1} = F(z^k + mu_k (z^k - z^{k-1}))
    LatArgs<T> g;
    if (P->ny == 1) {
      g = lat_args<T>(1, P->nx, P->nz, im.grad, im.grad);
    } else {
      ISAM_TRY(lat<T>(P, LAT_C2C_INV, lat_args<T>(P->ny, P->nx, P->nz, im.grad, im.grad)));
      g = lat_args<T>(1, P->ny, P->nx * P->nz, im.grad, im.grad);
    }
    g.z1 = z1; g.z2 = z2; g.inv_L = T(1.0 / L); g.mu_prev = T(mu_prev); g.flag = P->flag;
    ISAM_TRY(lat<T>(P, LAT_GRAD_STEP, g));
    if (prior == ISAM_PRIOR_HAAR_DEPTH) {
      ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
        return launch_haar_prox<T>(im.grad, zout, P->nz, size_t(P->nx) * P->ny, T(lam / L),
                                   lam_dev, lam_scale, s);
      }));
    } else {
      // TV prox of u = im.grad: the dual (p) carries over from the previous
      // iteration; r starts at p; fast gradient projection; z = u - tau grad^H p
      const size_t n = P->n_img;
      cplx<T>* px = im.tv;
      cplx<T>* pz = im.tv + n;
      cplx<T>* rx = im.tv + 2 * n;
      cplx<T>* rz = im.tv + 3 * n;
      cplx<T>* w = im.tv + 4 * n;
      const T tau = T(lam / L);
      CUDA_TRY(cudaMemcpyAsync(rx, px, 2 * n * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, s));
      double t = 1.0;
      const int iters = prior_iters > 0 ? prior_iters : 20;
      for (int i = 0; i < iters; ++i) {
        const double t_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        const T beta = T((t - 1.0) / t_next);
        t = t_next;
        ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
          return launch_tv_primal<T>(im.grad, rx, rz, tau, lam_dev, lam_scale, w, P->nx, P->nz, n,
                                     s);
        }));
        ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
          return launch_tv_dual<T>(w, px, pz, rx, rz, tau, lam_dev, lam_scale, beta, P->nx, P->nz,
                                   n, s);
        }));
      }
      ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
        return launch_tv_primal<T>(im.grad, px, pz, tau, lam_dev, lam_scale, zout, P->nx, P->nz,
                                   n, s);
      }));
    }
    LatArgs<T> e = lat_args<T>(P->ny, P->nx, P->nz, nullptr, ehat_out);
    e.z1 = zout; e.z2 = z1; e.mu = T(mu);
    ISAM_TRY(lat<T>(P, LAT_EXTRAP_FWD, e));
    if (P->ny > 1)
      ISAM_TRY(lat<T>(P, LAT_C2C_FWD, lat_args<T>(1, P->ny, P->nx * P->nz, ehat_out, ehat_out)));
    return ISAM_OK;
  }
  LatArgs<T> u;
  if (P->ny == 1) {
    u = lat_args<T>(1, P->nx, P->nz, im.grad, ehat_out);
  } else {
    LatArgs<T> x = lat_args<T>(P->ny, P->nx, P->nz, im.grad, im.grad);
    x.stop = stop;
    ISAM_TRY(lat<T>(P, LAT_C2C_INV, x));
    u = lat_args<T>(1, P->ny, P->nx * P->nz, im.grad, ehat_out);
  }
  u.stop = stop;
  if (P->tune_tp) {
    u.TZ = P->tune_tp;
    u.logTZ = ilog2(P->tune_tp);
  }
  u.z1 = z1; u.z2 = from_u ? nullptr : z2; u.zout = zout; u.w = w; u.nz = P->nz; u.uout = u_out;
  u.lam_dev = lam_dev; u.lam_scale = lam_scale;
  u.inv_L = T(1.0 / L); u.lam_over_L = T(lam / L); u.mu_prev = T(mu_prev); u.mu = T(mu);
  u.partial = norms ? P->partial : nullptr;
  u.flag = P->flag;
  ISAM_TRY(lat<T>(P, from_u ? LAT_UPDATE_U : LAT_UPDATE, u));
  if (norms) {
    const int nblk = (u.M / (2 * u.TZ)) * u.B;
    const StopRule sr = stop_rule ? *stop_rule : StopRule{};
    ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
      return launch_sum3(P->partial, nblk, P->dscal + 1, sr, s);
    }));
  }
  if (P->ny > 1) {
    LatArgs<T> x = lat_args<T>(P->ny, P->nx, P->nz, ehat_out, ehat_out);
    x.stop = stop;
    ISAM_TRY(lat<T>(P, LAT_C2C_FWD, x));
  }
  return ISAM_OK;
}

// t^1 = 1, t^{k+1} = (1 + sqrt(1 + 4 (t^k)^2))/2; mu_k = (t^k - 1)/t^{k+1}
void momentum(int kmax, std::vector<double>& mu) {
  std::vector<double> t(kmax + 2);
  t[1] = 1.0;
  for (int k = 1; k <= kmax; ++k) t[k + 1] = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t[k] * t[k]));
  mu.assign(kmax + 1, 0.0);
  for (int k = 1; k <= kmax; ++k) mu[k] = (t[k] - 1.0) / t[k + 1];
}

template <typename T> isam_status solve_impl(isam_plan* P, const T* s_d, const isam_solve_opts* o,
                                             cplx<T>* eta_out, isam_solve_state* state,
                                             isam_solve_info* info) {
  Impl<T>& im = impl_of<T>(P);
  cudaStream_t s = P->stream;
  if (!im.zA) ISAM_TRY(dalloc(&im.zA, P->n_img));
  if (!im.zB) ISAM_TRY(dalloc(&im.zB, P->n_img));
  int64_t launches0 = P->launches;
  const bool resume = state && state->k > 0;
  // lambda = c ||A^H s_d||_inf unless given
  double lam = o->lambda_abs;
  if (resume && state->lambda > 0) lam = state->lambda;
  if (!(lam > 0)) {
    ISAM_TRY(op_adjoint<T>(P, s_d, im.zA));
    double m = 0.0;
    ISAM_TRY(max_abs_dev<T>(P, im.zA, &m));
    lam = o->lambda_rel * m;
  }
  double L = o->L;
  if (resume && state->L > 0) L = state->L;
  if (!(L > 0)) {
    if (!(P->L_cache > 0)) {
      double Lc = 0.0;
      if (precision_fits<double>(P))
        ISAM_TRY(power_iteration<double>(P, kPowerIters, kPowerRtol, nullptr, 0, &Lc));
      else
        ISAM_TRY(power_iteration<T>(P, kPowerIters, kPowerRtol, nullptr, 0, &Lc));
      P->L_cache = Lc;
    }
    L = P->L_cache;
  }
  if (!(L > 0)) return ISAM_ERR_INVALID;
  const int k0 = resume ? state->k : 0;
  std::vector<double> mu;
  momentum(k0 + o->max_iter + 1, mu);
  cplx<T>* zP = im.zA;   // holds z^{k-1}
  cplx<T>* zQ = im.zB;   // holds z^{k-2}, receives z^k
  CUDA_TRY(cudaMemsetAsync(P->flag, 0, sizeof(int), s));
  if (resume) {
    CUDA_TRY(cudaMemcpyAsync(zP, state->z1, sizeof(cplx<T>) * P->n_img, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(zQ, state->z2, sizeof(cplx<T>) * P->n_img, cudaMemcpyDeviceToDevice, s));
    ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
      return launch_extrapolate<T>(zP, zQ, T(mu[k0]), im.grad, P->n_img, s);
    }));
    ISAM_TRY(lat_forward<T>(P, im, im.grad, im.eta_hat, P->nz, false));
  } else {
    CUDA_TRY(cudaMemsetAsync(zP, 0, sizeof(cplx<T>) * P->n_img, s));
    CUDA_TRY(cudaMemsetAsync(zQ, 0, sizeof(cplx<T>) * P->n_img, s));
    CUDA_TRY(cudaMemsetAsync(im.eta_hat, 0, sizeof(cplx<T>) * P->n_img, s));
  }
  if (o->prior == ISAM_PRIOR_TV) {                 // TV dual starts at 0 for every solve
    if (!im.tv) ISAM_TRY(dalloc(&im.tv, 5 * P->n_img));
    CUDA_TRY(cudaMemsetAsync(im.tv, 0, 2 * sizeof(cplx<T>) * P->n_img, s));
  }
  // lateral spectrum of the data, used by every iteration's residual
  if (!im.sdh) ISAM_TRY(dalloc(&im.sdh, P->n_spec));
  ISAM_TRY(lat_forward<T>(P, im, s_d, im.sdh, P->nk, true));
  const bool check = o->tol > 0;
  const int every = std::max(1, o->check_every);
  const double eps = o->eps > 0 ? o->eps : 1e-30;
  double rr = -1.0;
  int done = 0;
  // The stop rule runs on the device (StopRule; only the l1 prior takes
  // tol > 0).  The host reads a check's outcome kStopLag iterations after
  // queuing it, so a check never drains the GPU; only the iterations queued
  // while an outcome is unread carry the stop flag (their kernels write nothing
  // once it is set), and the result is the iterate of the stopping check.
  constexpr int kStopLag = 2;
  const bool dev_stop = check;
  if (dev_stop) CUDA_TRY(cudaMemsetAsync(P->dstop, 0, 2 * sizeof(int), s));
  bool pending = false;   // a check whose outcome the host has not read
  int since = 0;          // iterations queued after it
  for (int it = 1; it <= o->max_iter; ++it) {
    const int k = k0 + it;
    const bool norms = check && (it % every == 0 || it == o->max_iter);
    StopRule sr{};
    if (dev_stop) {
      sr.stop = P->dstop;
      sr.rr = P->dscal + 7;
      sr.tol = o->tol;
      sr.eps = eps;
      sr.iter = it;
    }
    ISAM_TRY(fista_iteration<T>(P, im, zP, zQ, zQ, static_cast<const T*>(o->w_dev), lam, L,
                                mu[k - 1], mu[k], norms, nullptr, nullptr, nullptr, nullptr, 0.0,
                                o->prior, o->prior_iters, nullptr, pending ? P->dstop : nullptr,
                                dev_stop && norms ? &sr : nullptr));
    std::swap(zP, zQ);   // zP = z^k, zQ = z^{k-1}
    done = it;
    if (dev_stop) {
      // read the pending check once kStopLag iterations keep the GPU busy, or
      // before this check's outcome takes the pinned slot
      if (pending && (++since >= kStopLag || norms)) {
        CUDA_TRY(cudaEventSynchronize(P->ev_check));
        pending = false;
        if (P->hstop[0]) break;
      }
      if (norms) {
        CUDA_TRY(cudaMemcpyAsync(P->hstop, P->dstop, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaEventRecord(P->ev_check, s));
        pending = true;
        since = 0;
      }
    }
  }
  if (dev_stop) {
    // where the device stopped (if it did) and r_r of that check, else of the last
    CUDA_TRY(cudaMemcpyAsync(P->hstop + 2, P->dstop, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(P->hscal + 7, P->dscal + 7, sizeof(double), cudaMemcpyDeviceToHost,
                             s));
    CUDA_TRY(cudaStreamSynchronize(s));
    rr = P->hscal[7];
    if (P->hstop[2]) {
      const int stop_it = P->hstop[3];
      if ((done - stop_it) & 1) std::swap(zP, zQ);   // z^{stop_it} and z^{stop_it - 1}
      done = stop_it;
    }
  }
  // objective of Eq. 12 at z^K
  double objective = -1.0;
  if (o->objective && o->prior == ISAM_PRIOR_L1) {
    if (!im.s_tmp) ISAM_TRY(dalloc(&im.s_tmp, P->n_spec));
    ISAM_TRY(op_forward<T>(P, zP, im.s_tmp));
    ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
      return launch_rsub<T>(im.s_tmp, s_d, im.s_tmp, P->n_spec, s);
    }));
    P->launches += 2;
    ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
      return launch_norm2<T>(reinterpret_cast<const cplx<T>*>(im.s_tmp), P->n_spec / 2,
                             P->partial, RED_BLOCKS, P->dscal + 5, s);
    }));
    ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
      return launch_wl1<T>(zP, P->n_img, static_cast<const T*>(o->w_dev), P->nz, P->partial,
                           RED_BLOCKS, P->dscal + 6, s);
    }));
    CUDA_TRY(cudaMemcpyAsync(P->hscal + 5, P->dscal + 5, 2 * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    harvest_events(P);
    objective = 0.5 * P->hscal[5] * P->hscal[5] + lam * P->hscal[6];
  }
  // result: z^K, optionally with the residual added back (Alg. 1, last step)
  if (o->residual_addback) {
    if (!im.s_tmp) ISAM_TRY(dalloc(&im.s_tmp, P->n_spec));
    ISAM_TRY(op_forward<T>(P, zP, im.s_tmp));
    ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
      return launch_rsub<T>(s_d, im.s_tmp, im.s_tmp, P->n_spec, s);
    }));
    ISAM_TRY(op_adjoint<T>(P, im.s_tmp, im.grad));
    ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
      return launch_caxpy<T>(zP, im.grad, T(1.0 / L), eta_out, P->n_img, s);
    }));
  } else if (zP != eta_out) {
    CUDA_TRY(cudaMemcpyAsync(eta_out, zP, sizeof(cplx<T>) * P->n_img, cudaMemcpyDeviceToDevice, s));
  }
  if (state) {
    CUDA_TRY(cudaMemcpyAsync(state->z1, zP, sizeof(cplx<T>) * P->n_img, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(state->z2, zQ, sizeof(cplx<T>) * P->n_img, cudaMemcpyDeviceToDevice, s));
    state->k = k0 + done;
    state->lambda = lam;
    state->L = L;
  }
  int hflag = 0;
  CUDA_TRY(cudaMemcpyAsync(P->hscal + 4, P->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  harvest_events(P);
  memcpy(&hflag, P->hscal + 4, sizeof(int));
  isam_status st = hflag ? ISAM_ERR_NONFINITE : ISAM_OK;
  if (info) {
    info->iterations = done;
    info->rr = rr;
    info->lambda = lam;
    info->L = L;
    info->status = st;
    info->objective = objective;
  }
  (void)launches0;
  return st;
}

isam_status validate(const isam_params* p) {
  if (!p) return ISAM_ERR_INVALID;
  const int nz = p->nz ? p->nz : p->nk;
  int lg = 0, r3 = 0;
  if (!fft_length(p->nx, &lg, &r3) || !fft_length(p->ny, &lg, &r3)) return ISAM_ERR_INVALID;
  if (!pow2(p->nk) || !pow2(nz)) return ISAM_ERR_INVALID;
  if (p->nx > 4096 || p->ny > 4096) return ISAM_ERR_UNSUPPORTED;
  if (p->nk < 16 || nz < 16) return ISAM_ERR_UNSUPPORTED;
  if (nz < p->nk || nz > 2048) return ISAM_ERR_UNSUPPORTED;
  if (!(p->k_min > 0) || !(p->k_max > p->k_min)) return ISAM_ERR_INVALID;
  if (p->nx > 1 && !(p->dx > 0)) return ISAM_ERR_INVALID;
  if (p->ny > 1 && !(p->dy > 0)) return ISAM_ERR_INVALID;
  if (p->n_disp < 0 || p->n_disp > 4) return ISAM_ERR_INVALID;
  if (p->precision != ISAM_FP32 && p->precision != ISAM_FP64) return ISAM_ERR_INVALID;
  const int J = p->nufft_J ? p->nufft_J : 6;
  if (J != 4 && J != 6 && J != 8) return ISAM_ERR_UNSUPPORTED;
  const int os = p->nufft_os ? p->nufft_os : 2;
  if (os != 2) return ISAM_ERR_UNSUPPORTED;
  if (!isfinite(p->z0)) return ISAM_ERR_INVALID;
  if (p->flags & ~(ISAM_FLAG_NO_STOLT_TABLE | ISAM_FLAG_AXIAL_MODEL)) return ISAM_ERR_INVALID;
  for (int i = 0; i < 4; ++i)
    if (!isfinite(p->disp[i])) return ISAM_ERR_INVALID;
  return ISAM_OK;
}

void split_ff(double v, float* hi, float* lo) {
  *hi = float(v);
  *lo = float(v - double(*hi));
}

void make_stolt(isam_plan* P) {
  const isam_params& p = P->p;
  StoltConst& c = P->sc;
  const double dk = (p.k_max - p.k_min) / (P->nk - 1);
  c.kap = p.k_min / dk;
  // the 1-D model puts every column on the q = 0 map (no lateral coupling)
  const bool axial = (p.flags & ISAM_FLAG_AXIAL_MODEL) != 0;
  c.Qx = P->nx > 1 && !axial ? pow(2.0 * M_PI / (P->nx * p.dx * dk), 2.0) : 0.0;
  c.Qy = P->ny > 1 && !axial ? pow(2.0 * M_PI / (P->ny * p.dy * dk), 2.0) : 0.0;
  c.zeta = axial ? 0.0 : dk * p.z0 / (2.0 * M_PI);
  c.c0d = fmod(2.0 * c.kap, double(P->K));
  c.I0 = int(floor(c.c0d));
  c.f0 = float(c.c0d - double(c.I0));
  c.B = float(2.0 * c.kap - c.c0d);
  split_ff(c.kap, &c.kap_hi, &c.kap_lo);
  split_ff(c.Qx, &c.qx_hi, &c.qx_lo);
  split_ff(c.Qy, &c.qy_hi, &c.qy_lo);
  split_ff(c.zeta, &c.zeta_hi, &c.zeta_lo);
  c.K = P->K; c.logK = ilog2(P->K);
  c.nx = P->nx; c.ny = P->ny; c.nk = P->nk; c.nz = P->nz; c.J = P->J;
  c.focus = c.zeta != 0.0;
}

// Least squares min ||V a - v|| for the Vandermonde V_ik = y_i^k (k <= deg),
// by Householder QR in double.
void ls_poly(const std::vector<double>& y, const std::vector<double>& v, int deg, double* a) {
  const int m = int(y.size()), n = deg + 1;
  std::vector<double> A(size_t(m) * n), b(v);
  for (int i = 0; i < m; ++i) {
    double pw = 1.0;
    for (int k = 0; k < n; ++k) { A[size_t(i) * n + k] = pw; pw *= y[i]; }
  }
  for (int k = 0; k < n; ++k) {
    double nrm = 0.0;
    for (int i = k; i < m; ++i) nrm += A[size_t(i) * n + k] * A[size_t(i) * n + k];
    nrm = sqrt(nrm);
    const double akk = A[size_t(k) * n + k];
    const double alpha = akk > 0 ? -nrm : nrm;
    std::vector<double> u(m, 0.0);
    for (int i = k; i < m; ++i) u[i] = A[size_t(i) * n + k];
    u[k] -= alpha;
    double un = 0.0;
    for (int i = k; i < m; ++i) un += u[i] * u[i];
    if (un == 0.0) continue;
    for (int c = k; c < n; ++c) {
      double d = 0.0;
      for (int i = k; i < m; ++i) d += u[i] * A[size_t(i) * n + c];
      d = 2.0 * d / un;
      for (int i = k; i < m; ++i) A[size_t(i) * n + c] -= d * u[i];
    }
    double d = 0.0;
    for (int i = k; i < m; ++i) d += u[i] * b[i];
    d = 2.0 * d / un;
    for (int i = k; i < m; ++i) b[i] -= d * u[i];
  }
  for (int k = n - 1; k >= 0; --k) {
    double acc = b[k];
    for (int c = k + 1; c < n; ++c) acc -= A[size_t(k) * n + c] * a[c];
    a[k] = acc / A[size_t(k) * n + k];
  }
}

// Exact min-max coefficients at Chebyshev nodes of y = 4 (f - 1/2)^2 (FP64,
// on the device), then the even/odd polynomial fits of both precisions.
isam_status build_poly(isam_plan* P) {
  constexpr int M = 48;
  const int J = P->J;
  std::vector<double> y(M), x(M), f(M);
  for (int i = 0; i < M; ++i) {
    y[i] = 0.5 * (cos(M_PI * (i + 0.5) / M) + 1.0);
    x[i] = 0.5 * sqrt(y[i]);
    f[i] = 0.5 + x[i];
  }
  double *df = nullptr, *dc = nullptr;
  ISAM_TRY(dalloc(&df, M));
  isam_status st = dalloc(&dc, size_t(M) * J);
  std::vector<double> c(size_t(M) * J);
  if (st == ISAM_OK) st = from_cuda(cudaMemcpy(df, f.data(), sizeof(double) * M, cudaMemcpyHostToDevice));
  if (st == ISAM_OK) st = from_cuda(minmax_nodes(P->nz, P->K, J, df, M, dc, P->stream));
  if (st == ISAM_OK) st = from_cuda(cudaStreamSynchronize(P->stream));
  if (st == ISAM_OK)
    st = from_cuda(cudaMemcpy(c.data(), dc, sizeof(double) * M * J, cudaMemcpyDeviceToHost));
  dfree(df);
  dfree(dc);
  if (st != ISAM_OK) return st;
  for (int p = 0; p < J / 2; ++p) {
    std::vector<double> e(M), o(M);
    for (int i = 0; i < M; ++i) {
      const double cp = c[size_t(i) * J + p], cm = c[size_t(i) * J + (J - 1 - p)];
      e[i] = 0.5 * (cp + cm);
      o[i] = 0.5 * (cp - cm) / x[i];
    }
    double ae[7] = {0}, ao[6] = {0};
    ls_poly(y, e, PolyDeg<double>::DE, ae);
    ls_poly(y, o, PolyDeg<double>::DO, ao);
    for (int k = 0; k <= PolyDeg<double>::DE; ++k) P->poly64.e[p][k] = ae[k];
    for (int k = 0; k <= PolyDeg<double>::DO; ++k) P->poly64.o[p][k] = ao[k];
    ls_poly(y, e, PolyDeg<float>::DE, ae);
    ls_poly(y, o, PolyDeg<float>::DO, ao);
    for (int k = 0; k <= PolyDeg<float>::DE; ++k) P->poly32.e[p][k] = float(ae[k]);
    for (int k = 0; k <= PolyDeg<float>::DO; ++k) P->poly32.o[p][k] = float(ao[k]);
  }
  return ISAM_OK;
}

// Columns (ix, iy) and (-ix, -iy) mod (nx, ny) share |q|; list each pair once.
isam_status build_pairs(isam_plan* P) {
  std::vector<int2> pr;
  for (int iy = 0; iy < P->ny; ++iy)
    for (int ix = 0; ix < P->nx; ++ix) {
      const int c = iy * P->nx + ix;
      const int d = ((P->ny - iy) % P->ny) * P->nx + (P->nx - ix) % P->nx;
      if (c <= d) pr.push_back(make_int2(c, d));
    }
  P->npairs = int(pr.size());
  ISAM_TRY(dalloc(&P->pairs, pr.size()));
  return from_cuda(cudaMemcpy(P->pairs, pr.data(), sizeof(int2) * pr.size(),
                              cudaMemcpyHostToDevice));
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

}  // namespace

extern "C" {

isam_status isam_set_allocator(isam_alloc_fn alloc, isam_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return ISAM_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc.alloc = alloc;
  g_alloc.free = free_fn;
  g_alloc.ctx = ctx;
  return ISAM_OK;
}

const char* isam_status_string(isam_status s) {
  switch (s) {
    case ISAM_OK: return "ok";
    case ISAM_ERR_INVALID: return "invalid argument";
    case ISAM_ERR_OOM: return "out of device memory";
    case ISAM_ERR_CUDA: return "CUDA error";
    case ISAM_ERR_NONFINITE: return "non-finite value in the solve";
    case ISAM_ERR_UNSUPPORTED: return "unsupported size or option";
  }
  return "unknown status";
}

isam_status isam_plan_create(const isam_params* p, void* stream, isam_plan** out) {
  if (!out) return ISAM_ERR_INVALID;
  *out = nullptr;
  ISAM_TRY(validate(p));
  isam_plan* P = new (std::nothrow) isam_plan();
  if (!P) return ISAM_ERR_OOM;
  P->p = *p;
  P->nx = p->nx; P->ny = p->ny; P->nk = p->nk; P->nz = p->nz ? p->nz : p->nk;
  P->p.nz = P->nz;
  P->K = 2 * P->nz;
  P->J = p->nufft_J ? p->nufft_J : 6;
  P->stream = static_cast<cudaStream_t>(stream);
  P->n_img = size_t(P->nx) * P->ny * P->nz;
  P->n_spec = size_t(P->nx) * P->ny * P->nk;
  cudaGetDevice(&P->device);
  make_stolt(P);
  isam_status st = ISAM_OK;
  {
    // partial sums: reductions use RED_BLOCKS, the FISTA update one per block
    const int M = P->ny == 1 ? P->nz : P->nx * P->nz;
    const int npairs_max = P->nx * P->ny / 2 + 4;
    P->n_partial = std::max(std::max(RED_BLOCKS, M / 2), npairs_max);   // any update tile
  }
  if (st == ISAM_OK) st = dalloc(&P->partial, size_t(P->n_partial) * 3);
  if (st == ISAM_OK) st = dalloc(&P->dscal, 8);
  if (st == ISAM_OK) st = dalloc(&P->flag, 1);
  if (st == ISAM_OK) st = from_cuda(cudaMallocHost(reinterpret_cast<void**>(&P->hscal), 8 * sizeof(double)));
  if (st == ISAM_OK) st = dalloc(&P->dstop, 2);
  if (st == ISAM_OK) st = from_cuda(cudaMallocHost(reinterpret_cast<void**>(&P->hstop), 4 * sizeof(int)));
  if (st == ISAM_OK) st = from_cuda(cudaEventCreateWithFlags(&P->ev_check, cudaEventDisableTiming));
  if (st == ISAM_OK) st = build_pairs(P);
  if (st == ISAM_OK) st = build_poly(P);
  if (st == ISAM_OK) {
    if (p->precision == ISAM_FP64) st = impl_init<double>(P, P->f64);
    else st = impl_init<float>(P, P->f32);
  }
  if (st != ISAM_OK) {
    isam_plan_destroy(P);
    return st;
  }
  *out = P;
  return ISAM_OK;
}

void isam_plan_destroy(isam_plan* P) {
  if (!P) return;
  DeviceGuard g(P->device);
  if (P->stream) cudaStreamSynchronize(P->stream);
  else cudaDeviceSynchronize();
  impl_free(P->f32);
  impl_free(P->f64);
  dfree(P->partial);
  dfree(P->cpartial);
  dfree(P->pairs);
  dfree(P->dscal);
  dfree(P->flag);
  dfree(P->dstop);
  if (P->hscal) cudaFreeHost(P->hscal);
  if (P->hstop) cudaFreeHost(P->hstop);
  if (P->ev_check) cudaEventDestroy(P->ev_check);
  harvest_events(P);
  for (cudaEvent_t e : P->ev_pool) cudaEventDestroy(e);
  delete P;
}

isam_status isam_set_stream(isam_plan* P, void* stream) {
  if (!P) return ISAM_ERR_INVALID;
  P->stream = static_cast<cudaStream_t>(stream);
  return ISAM_OK;
}

isam_status isam_forward(isam_plan* P, const void* eta, void* s) {
  if (!P || !eta || !s) return ISAM_ERR_INVALID;
  DeviceGuard g(P->device);
  P->launches = 0;
  if (P->p.precision == ISAM_FP64) return op_forward<double>(P, eta, s);
  return op_forward<float>(P, eta, s);
}

isam_status isam_adjoint(isam_plan* P, const void* s, void* eta) {
  if (!P || !eta || !s) return ISAM_ERR_INVALID;
  DeviceGuard g(P->device);
  P->launches = 0;
  if (P->p.precision == ISAM_FP64) return op_adjoint<double>(P, s, eta);
  return op_adjoint<float>(P, s, eta);
}

static isam_status check_opts(const isam_plan* P, const isam_solve_opts* o) {
  if (!o) return ISAM_ERR_INVALID;
  if (o->max_iter < 1) return ISAM_ERR_INVALID;
  if (!(o->lambda_abs > 0) && !(o->lambda_rel >= 0)) return ISAM_ERR_INVALID;
  if (o->tol < 0 || !isfinite(o->tol)) return ISAM_ERR_INVALID;
  if (o->prior != ISAM_PRIOR_L1 && o->prior != ISAM_PRIOR_HAAR_DEPTH && o->prior != ISAM_PRIOR_TV)
    return ISAM_ERR_INVALID;
  if (o->prior_iters < 0) return ISAM_ERR_INVALID;
  if (o->prior != ISAM_PRIOR_L1 && (o->w_dev || o->tol > 0)) return ISAM_ERR_UNSUPPORTED;
  (void)P;
  return ISAM_OK;
}

isam_status isam_solve(isam_plan* P, const void* s_d, const isam_solve_opts* o, void* eta_out,
                       isam_solve_state* state, isam_solve_info* info) {
  if (!P || !s_d || !eta_out) return ISAM_ERR_INVALID;
  ISAM_TRY(check_opts(P, o));
  if (state && (!state->z1 || !state->z2 || state->k < 0)) return ISAM_ERR_INVALID;
  if (state && state->k > 0 && o->prior == ISAM_PRIOR_TV) return ISAM_ERR_UNSUPPORTED;
  DeviceGuard g(P->device);
  P->launches = 0;
  if (P->p.precision == ISAM_FP64)
    return solve_impl<double>(P, static_cast<const double*>(s_d), o, static_cast<double2*>(eta_out),
                              state, info);
  return solve_impl<float>(P, static_cast<const float*>(s_d), o, static_cast<float2*>(eta_out),
                           state, info);
}

}  // extern "C"

template <typename T>
static isam_status solve_host_impl(isam_plan* P, const void* s_h, const isam_solve_opts* o,
                                   void* eta_h, isam_solve_info* info) {
  Impl<T>& im = impl_of<T>(P);
  if (!im.s_host_stage) ISAM_TRY(dalloc(&im.s_host_stage, P->n_spec));
  if (!im.out_stage) ISAM_TRY(dalloc(&im.out_stage, P->n_img));
  CUDA_TRY(cudaMemcpyAsync(im.s_host_stage, s_h, sizeof(T) * P->n_spec, cudaMemcpyHostToDevice,
                           P->stream));
  ISAM_TRY(solve_impl<T>(P, im.s_host_stage, o, im.out_stage, nullptr, info));
  CUDA_TRY(cudaMemcpyAsync(eta_h, im.out_stage, sizeof(cplx<T>) * P->n_img,
                           cudaMemcpyDeviceToHost, P->stream));
  return from_cuda(cudaStreamSynchronize(P->stream));
}

extern "C" {

isam_status isam_solve_host(isam_plan* P, const void* s_h, const isam_solve_opts* o, void* eta_h,
                            isam_solve_info* info) {
  if (!P || !s_h || !eta_h) return ISAM_ERR_INVALID;
  ISAM_TRY(check_opts(P, o));
  DeviceGuard g(P->device);
  P->launches = 0;
  if (P->p.precision == ISAM_FP64) return solve_host_impl<double>(P, s_h, o, eta_h, info);
  return solve_host_impl<float>(P, s_h, o, eta_h, info);
}

isam_status isam_lipschitz(isam_plan* P, int32_t iters, double rtol, const void* v0,
                           double* L_out) {
  if (!P || !L_out || iters < 0 || !(rtol >= 0)) return ISAM_ERR_INVALID;
  if (iters == 0) {
    iters = kPowerIters;
    rtol = kPowerRtol;
  }
  DeviceGuard g(P->device);
  P->launches = 0;
  const int v0_double = P->p.precision == ISAM_FP64;
  double L = 0.0;
  if (precision_fits<double>(P))
    ISAM_TRY(power_iteration<double>(P, iters, rtol, v0, v0_double, &L));
  else if (P->p.precision == ISAM_FP64)
    return ISAM_ERR_UNSUPPORTED;
  else
    ISAM_TRY(power_iteration<float>(P, iters, rtol, v0, v0_double, &L));
  P->L_cache = L;
  *L_out = L;
  return ISAM_OK;
}

isam_status isam_data_fidelity(isam_plan* P, const void* eta, const void* s_d, void* r_out,
                               double* value) {
  if (!P || !eta || !s_d || !value) return ISAM_ERR_INVALID;
  DeviceGuard g(P->device);
  P->launches = 0;
  if (P->p.precision == ISAM_FP64)
    return fidelity_impl<double>(P, eta, static_cast<const double*>(s_d),
                                 static_cast<double*>(r_out), value);
  return fidelity_impl<float>(P, eta, static_cast<const float*>(s_d), static_cast<float*>(r_out),
                              value);
}

isam_status isam_max_abs(isam_plan* P, const void* eta, double* out) {
  if (!P || !eta || !out) return ISAM_ERR_INVALID;
  DeviceGuard g(P->device);
  if (P->p.precision == ISAM_FP64) return max_abs_dev<double>(P, static_cast<const double2*>(eta), out);
  return max_abs_dev<float>(P, static_cast<const float2*>(eta), out);
}

int64_t isam_last_launch_count(const isam_plan* P) { return P ? P->launches : -1; }

isam_status isam_profile_enable(isam_plan* P, int32_t on) {
  if (!P) return ISAM_ERR_INVALID;
  DeviceGuard g(P->device);
  CUDA_TRY(cudaStreamSynchronize(P->stream));
  harvest_events(P);
  P->prof = on != 0;
  return ISAM_OK;
}

isam_status isam_profile_read(isam_plan* P, double* ms, int64_t* counts, int32_t reset) {
  if (!P || !ms || !counts) return ISAM_ERR_INVALID;
  DeviceGuard g(P->device);
  CUDA_TRY(cudaStreamSynchronize(P->stream));
  harvest_events(P);
  for (int c = 0; c < ISAM_KCLASS_COUNT; ++c) {
    ms[c] = P->prof_ms[c];
    counts[c] = P->prof_n[c];
    if (reset) { P->prof_ms[c] = 0.0; P->prof_n[c] = 0; }
  }
  return ISAM_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// Calibration of theta = (a_1..a_4, z0): parameter derivatives of A and the
// gradient through unrolled FISTA iterations (lambda and L held fixed).
// ----------------------------------------------------------------------------
namespace {

template <typename T> isam_status calib_buffers(isam_plan* P, Impl<T>& im, int seg_cap) {
  if (!im.spec2) ISAM_TRY(dalloc(&im.spec2, P->n_spec));
  if (!im.cal) ISAM_TRY(dalloc(&im.cal, 5 * P->n_img));
  if (!P->cpartial) ISAM_TRY(dalloc(&P->cpartial, size_t(P->npairs) * 5));
  if (seg_cap > im.seg_cap) {
    dfree(im.seg);
    im.seg = nullptr;
    im.seg_cap = 0;
    // [seg_cap] u^k, [seg_cap + 1] eta_hat^k, [seg_cap] model spectra S^k
    ISAM_TRY(dalloc(&im.seg, size_t(2 * seg_cap + 1) * P->n_img + size_t(seg_cap) * P->n_spec));
    im.seg_cap = seg_cap;
  }
  if (!im.zA) ISAM_TRY(dalloc(&im.zA, P->n_img));
  if (!im.zB) ISAM_TRY(dalloc(&im.zB, P->n_img));
  if (!im.sdh) ISAM_TRY(dalloc(&im.sdh, P->n_spec));
  if (!im.s_tmp) ISAM_TRY(dalloc(&im.s_tmp, P->n_spec));
  return ISAM_OK;
}

// Sum the [npairs][5] partials in a fixed order and convert the moments to
// derivatives: d/da_i = dk^i m_i, d/dz0 = dk m_z, times `factor`.
isam_status read_param_partials(isam_plan* P, double factor, double* grad) {
  std::vector<double> h(size_t(P->npairs) * 5);
  CUDA_TRY(cudaMemcpyAsync(h.data(), P->cpartial, h.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, P->stream));
  CUDA_TRY(cudaStreamSynchronize(P->stream));
  harvest_events(P);
  double m[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < P->npairs; ++b)
    for (int i = 0; i < 5; ++i) m[i] += h[size_t(b) * 5 + i];
  const double dk = (P->p.k_max - P->p.k_min) / (P->nk - 1);
  double pw = 1.0;
  for (int i = 0; i < 4; ++i) {
    pw *= dk;
    grad[i] = factor * pw * m[i];
  }
  grad[4] = factor * dk * m[4];
  return ISAM_OK;
}

template <typename T> ParamArgs<T> param_args(isam_plan* P, cplx<T>* su, const cplx<T>* se,
                                              const cplx<T>* fd, T fd_sign, bool write_fa) {
  ParamArgs<T> a{};
  a.su = su; a.se = se; a.fd = fd; a.fd_sign = fd_sign;
  a.pairs = P->pairs; a.sc = P->sc; a.partial = P->cpartial; a.write_fa = write_fa ? 1 : 0;
  return a;
}

// <dA/dtheta x, y>: S_x = phase . N(F x), F y, then the weighted sums.
template <typename T> isam_status param_grad_impl(isam_plan* P, const void* x, const void* y,
                                                  double* grad) {
  Impl<T>& im = impl_of<T>(P);
  ISAM_TRY(calib_buffers<T>(P, im, 0));
  cudaStream_t s = P->stream;
  CUDA_TRY(cudaMemsetAsync(P->cpartial, 0, sizeof(double) * 5 * P->npairs, s));
  ISAM_TRY(lat_forward<T>(P, im, x, im.eta_hat, P->nz, false));
  ISAM_TRY(launch(P, ISAM_KCLASS_AX_FWD, [&] {
    return launch_ax_fwd<T>(ax_args<T>(P, im, im.eta_hat, im.spec), P->npairs, s);
  }));
  ISAM_TRY(lat_forward<T>(P, im, y, im.spec2, P->nk, true));
  ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
    return launch_param_reduce<T>(param_args<T>(P, im.spec, nullptr, im.spec2, T(1), false),
                                  P->npairs, s);
  }));
  return read_param_partials(P, 1.0, grad);
}

isam_status check_unrolled_opts(const isam_plan* P, const isam_solve_opts* o, int every) {
  if (!o || o->max_iter < 1 || every < 1) return ISAM_ERR_INVALID;
  if (!(o->lambda_abs > 0) || !(o->L > 0) || !isfinite(o->lambda_abs) || !isfinite(o->L))
    return ISAM_ERR_INVALID;
  if (o->residual_addback) return ISAM_ERR_INVALID;
  if (o->prior != ISAM_PRIOR_L1) return ISAM_ERR_UNSUPPORTED;
  (void)P;
  return ISAM_OK;
}

// z^K of K = o->max_iter iterations from z^0 = 0; before iteration c*every+1
// the pair (z^{c every}, z^{c every - 1}) is copied to ckpt images 2c, 2c+1.
template <typename T> isam_status unrolled_impl(isam_plan* P, const T* s_d,
                                                const isam_solve_opts* o, int every,
                                                cplx<T>* ckpt, cplx<T>* z_out) {
  Impl<T>& im = impl_of<T>(P);
  ISAM_TRY(calib_buffers<T>(P, im, 0));
  cudaStream_t s = P->stream;
  const size_t bytes = sizeof(cplx<T>) * P->n_img;
  const int K = o->max_iter;
  std::vector<double> mu;
  momentum(K + 1, mu);
  cplx<T>* zP = im.zA;
  cplx<T>* zQ = im.zB;
  CUDA_TRY(cudaMemsetAsync(P->flag, 0, sizeof(int), s));
  CUDA_TRY(cudaMemsetAsync(zP, 0, bytes, s));
  CUDA_TRY(cudaMemsetAsync(zQ, 0, bytes, s));
  CUDA_TRY(cudaMemsetAsync(im.eta_hat, 0, bytes, s));
  ISAM_TRY(lat_forward<T>(P, im, s_d, im.sdh, P->nk, true));
  const T* w = static_cast<const T*>(o->w_dev);
  for (int k = 1; k <= K; ++k) {
    if ((k - 1) % every == 0 && ckpt) {
      const size_t c = size_t((k - 1) / every);
      CUDA_TRY(cudaMemcpyAsync(ckpt + 2 * c * P->n_img, zP, bytes, cudaMemcpyDeviceToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(ckpt + (2 * c + 1) * P->n_img, zQ, bytes, cudaMemcpyDeviceToDevice, s));
    }
    ISAM_TRY(fista_iteration<T>(P, im, zP, zQ, zQ, w, o->lambda_abs, o->L, mu[k - 1], mu[k], false));
    std::swap(zP, zQ);
  }
  CUDA_TRY(cudaMemcpyAsync(z_out, zP, bytes, cudaMemcpyDeviceToDevice, s));
  int flag = 0;
  CUDA_TRY(cudaMemcpyAsync(&flag, P->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  harvest_events(P);
  return flag ? ISAM_ERR_NONFINITE : ISAM_OK;
}

// Gradient of <z_bar, z^K> with respect to theta (and s_d when s_bar is
// given).  Segment by segment from the last: recompute its iterations from
// the checkpoint, keeping u^k and eta_hat^k, then run the reverse recursion
//   ubar = J_T(u^k)^T zbar^k,  etabar = ubar - (1/L) A^H A ubar,
//   theta_bar -= (1/L)(<dA ubar, A eta^k - s_d> + <A ubar, dA eta^k>),
//   s_bar += (1/L) A ubar,  zbar^{k-1} += (1 + mu_{k-1}) etabar,
//   zbar^{k-2} -= mu_{k-1} etabar.
template <typename T> isam_status unrolled_vjp_impl(isam_plan* P, const T* s_d,
                                                    const isam_solve_opts* o, int every,
                                                    const cplx<T>* ckpt, const cplx<T>* z_bar,
                                                    T* s_bar, double* grad) {
  Impl<T>& im = impl_of<T>(P);
  const int K = o->max_iter;
  const int C = std::min(every, K);
  ISAM_TRY(calib_buffers<T>(P, im, C));
  cudaStream_t s = P->stream;
  const size_t n = P->n_img, bytes = sizeof(cplx<T>) * n;
  const double L = o->L, lam = o->lambda_abs;
  const T* w = static_cast<const T*>(o->w_dev);
  std::vector<double> mu;
  momentum(K + 1, mu);
  cplx<T>* seg_u = im.seg;              // [C] images u^k
  cplx<T>* seg_eh = im.seg + C * n;     // [C + 1] images eta_hat^k
  cplx<T>* seg_S = im.seg + size_t(2 * im.seg_cap + 1) * n;   // [C] spectra K eta_hat^k
  const size_t ns = P->n_spec;
  cplx<T>* zb[3] = {im.cal, im.cal + n, im.cal + 2 * n};
  cplx<T>* ubar = im.cal + 3 * n;
  cplx<T>* bimg = im.cal + 4 * n;
  CUDA_TRY(cudaMemsetAsync(P->flag, 0, sizeof(int), s));
  CUDA_TRY(cudaMemsetAsync(P->cpartial, 0, sizeof(double) * 5 * P->npairs, s));
  CUDA_TRY(cudaMemcpyAsync(zb[0], z_bar, bytes, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemsetAsync(zb[1], 0, 2 * bytes, s));
  if (s_bar) CUDA_TRY(cudaMemsetAsync(s_bar, 0, sizeof(T) * P->n_spec, s));
  ISAM_TRY(lat_forward<T>(P, im, s_d, im.sdh, P->nk, true));
  int cur = 0;                          // zb[cur] = zbar^k, then zbar^{k-1}, zbar^{k-2}
  const int nseg = (K + C - 1) / C;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int k0 = sg * C, k1 = std::min(K, k0 + C);
    // recompute iterations k0+1 .. k1 from (z^{k0}, z^{k0-1})
    CUDA_TRY(cudaMemcpyAsync(im.zA, ckpt + 2 * size_t(sg) * n, bytes, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(im.zB, ckpt + (2 * size_t(sg) + 1) * n, bytes,
                             cudaMemcpyDeviceToDevice, s));
    ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
      return launch_extrapolate<T>(im.zA, im.zB, T(mu[k0]), im.grad, n, s);
    }));
    ISAM_TRY(lat_forward<T>(P, im, im.grad, seg_eh, P->nz, false));
    cplx<T>* zP = im.zA;
    cplx<T>* zQ = im.zB;
    for (int k = k0 + 1; k <= k1; ++k) {
      const int i = k - k0 - 1;
      ISAM_TRY(fista_iteration<T>(P, im, zP, zQ, zQ, w, lam, L, mu[k - 1], mu[k], false,
                                  seg_eh + i * n, seg_eh + (i + 1) * n, seg_u + i * n, nullptr,
                                  0.0, ISAM_PRIOR_L1, 0, seg_S + i * ns));
      std::swap(zP, zQ);
    }
    // reverse through the segment
    for (int k = k1; k > k0; --k) {
      const int i = k - k0 - 1;
      cplx<T>* zcur = zb[cur];
      cplx<T>* zm1 = zb[(cur + 1) % 3];
      cplx<T>* zm2 = zb[(cur + 2) % 3];
      ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
        return launch_st_vjp<T>(seg_u + i * n, zcur, w, T(lam / L), P->nz, ubar, n, s);
      }));
      // S_ubar and S_eta (lateral spectra of K_hat before the real part)
      ISAM_TRY(lat_forward<T>(P, im, ubar, im.eta_hat, P->nz, false));
      ISAM_TRY(launch(P, ISAM_KCLASS_AX_FWD, [&] {
        return launch_ax_fwd<T>(ax_args<T>(P, im, im.eta_hat, im.spec), P->npairs, s);
      }));
      // theta partials (S of eta_hat^k: kept by the recompute's fused kernel);
      // im.spec becomes F(A ubar)
      ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
        return launch_param_reduce<T>(param_args<T>(P, im.spec, seg_S + i * ns, im.sdh, T(-1), true),
                                      P->npairs, s);
      }));
      // b = A^H A ubar
      ISAM_TRY(launch(P, ISAM_KCLASS_AX_ADJ, [&] {
        return launch_ax_adj<T>(ax_args<T>(P, im, im.spec, im.grad), P->npairs, s);
      }));
      if (s_bar) {
        ISAM_TRY(lat_inverse<T>(P, im, im.spec, im.s_tmp, P->nk, true));
        ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
          return launch_caxpy<T>(reinterpret_cast<const cplx<T>*>(s_bar),
                                 reinterpret_cast<const cplx<T>*>(im.s_tmp), T(1.0 / L),
                                 reinterpret_cast<cplx<T>*>(s_bar), P->n_spec / 2, s);
        }));
      }
      ISAM_TRY(lat_inverse<T>(P, im, im.grad, bimg, P->nz, false));
      ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
        return launch_bwd_combine<T>(ubar, bimg, T(1.0 / L), T(mu[k - 1]), k - 1 >= 1 ? zm1 : nullptr,
                                     k - 2 >= 1 ? zm2 : nullptr, n, s);
      }));
      CUDA_TRY(cudaMemsetAsync(zcur, 0, bytes, s));   // becomes zbar^{k-3}
      cur = (cur + 1) % 3;
    }
  }
  int flag = 0;
  CUDA_TRY(cudaMemcpyAsync(&flag, P->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  ISAM_TRY(read_param_partials(P, -1.0 / L, grad));
  return flag ? ISAM_ERR_NONFINITE : ISAM_OK;
}

}  // namespace

extern "C" {

isam_status isam_set_model(isam_plan* P, int32_t n_disp, const double* disp, double z0) {
  if (!P || n_disp < 0 || n_disp > 4 || (n_disp > 0 && !disp) || !isfinite(z0))
    return ISAM_ERR_INVALID;
  if (P->batch_refs) return ISAM_ERR_INVALID;       // a batch graph records the plan
  for (int i = 0; i < n_disp; ++i)
    if (!isfinite(disp[i])) return ISAM_ERR_INVALID;
  DeviceGuard g(P->device);
  CUDA_TRY(cudaStreamSynchronize(P->stream));
  P->p.n_disp = n_disp;
  for (int i = 0; i < 4; ++i) P->p.disp[i] = i < n_disp ? disp[i] : 0.0;
  P->p.z0 = z0;
  make_stolt(P);
  if (P->f32.ready) ISAM_TRY(phase_tables<float>(P, P->f32));
  if (P->f64.ready) ISAM_TRY(phase_tables<double>(P, P->f64));
  P->L_cache = 0.0;
  return from_cuda(cudaStreamSynchronize(P->stream));
}

isam_status isam_set_filter(isam_plan* P, const double* b) {
  if (!P) return ISAM_ERR_INVALID;
  if (P->batch_refs) return ISAM_ERR_INVALID;       // a batch graph records the plan
  const size_t n = 2 * size_t(P->ny / 2 + 1) * (P->nx / 2 + 1) * P->nk;
  if (b)
    for (size_t i = 0; i < n; ++i)
      if (!isfinite(b[i])) return ISAM_ERR_INVALID;
  DeviceGuard g(P->device);
  CUDA_TRY(cudaStreamSynchronize(P->stream));
  if (b) P->filt_host.assign(b, b + n);
  else P->filt_host.clear();
  if (P->f32.ready) ISAM_TRY(phase_tables<float>(P, P->f32));
  if (P->f64.ready) ISAM_TRY(phase_tables<double>(P, P->f64));
  P->L_cache = 0.0;
  return from_cuda(cudaStreamSynchronize(P->stream));
}

isam_status isam_param_grad(isam_plan* P, const void* x, const void* y, double* grad) {
  if (!P || !x || !y || !grad) return ISAM_ERR_INVALID;
  DeviceGuard g(P->device);
  P->launches = 0;
  if (P->p.precision == ISAM_FP64) return param_grad_impl<double>(P, x, y, grad);
  return param_grad_impl<float>(P, x, y, grad);
}

int32_t isam_unrolled_checkpoint_images(int32_t K, int32_t every) {
  if (K < 1 || every < 1) return -1;
  return 2 * ((K + every - 1) / every);
}

isam_status isam_fista_unrolled(isam_plan* P, const void* s_d, const isam_solve_opts* o,
                                int32_t every, void* ckpt, void* z_out) {
  if (!P || !s_d || !z_out) return ISAM_ERR_INVALID;
  ISAM_TRY(check_unrolled_opts(P, o, every));
  DeviceGuard g(P->device);
  P->launches = 0;
  if (P->p.precision == ISAM_FP64)
    return unrolled_impl<double>(P, static_cast<const double*>(s_d), o, every,
                                 static_cast<double2*>(ckpt), static_cast<double2*>(z_out));
  return unrolled_impl<float>(P, static_cast<const float*>(s_d), o, every,
                              static_cast<float2*>(ckpt), static_cast<float2*>(z_out));
}

isam_status isam_fista_unrolled_vjp(isam_plan* P, const void* s_d, const isam_solve_opts* o,
                                    int32_t every, const void* ckpt, const void* z_bar,
                                    void* s_bar, double* grad) {
  if (!P || !s_d || !ckpt || !z_bar || !grad) return ISAM_ERR_INVALID;
  ISAM_TRY(check_unrolled_opts(P, o, every));
  DeviceGuard g(P->device);
  P->launches = 0;
  if (P->p.precision == ISAM_FP64)
    return unrolled_vjp_impl<double>(P, static_cast<const double*>(s_d), o, every,
                                     static_cast<const double2*>(ckpt),
                                     static_cast<const double2*>(z_bar),
                                     static_cast<double*>(s_bar), grad);
  return unrolled_vjp_impl<float>(P, static_cast<const float*>(s_d), o, every,
                                  static_cast<const float2*>(ckpt),
                                  static_cast<const float2*>(z_bar), static_cast<float*>(s_bar),
                                  grad);
}

}  // extern "C"

namespace {

template <typename T> isam_status dc_ifft_impl(isam_plan* P, const T* s, cplx<T>* out) {
  Impl<T>& im = impl_of<T>(P);
  if (!im.dc_post) {
    // post_n = e^{-2 pi i kappa_0 (n - nz/2) / nz} / sqrt(nz), the phase reduced in FP64
    std::vector<cplx<T>> h(P->nz);
    const double dk = (P->p.k_max - P->p.k_min) / (P->nk - 1);
    const double kap0 = P->p.k_min / dk;
    const double kf = kap0 - floor(kap0);
    const double kint = floor(kap0);
    for (int n = 0; n < P->nz; ++n) {
      const int m = n - P->nz / 2;
      // kappa_0 m / nz = (kint m mod nz)/nz + kf m / nz, both reduced to turns
      const double t1 = fmod(fmod(kint, double(P->nz)) * m, double(P->nz)) / P->nz;
      const double turn = t1 + kf * m / P->nz;
      const double ang = -2.0 * M_PI * (turn - floor(turn));
      h[n] = mk<T>(T(cos(ang) / sqrt(double(P->nz))), T(sin(ang) / sqrt(double(P->nz))));
    }
    ISAM_TRY(dalloc(&im.dc_post, P->nz));
    CUDA_TRY(cudaMemcpy(im.dc_post, h.data(), sizeof(cplx<T>) * P->nz, cudaMemcpyHostToDevice));
  }
  return launch(P, ISAM_KCLASS_MISC, [&] {
    return launch_dc_ifft<T>(s, out, im.tab.disp, im.dc_post, P->nk, P->nz, ilog2(P->nz),
                             P->nx * P->ny, P->stream);
  });
}

}  // namespace

extern "C" {

isam_status isam_dispersion_compensated_ifft(isam_plan* P, const void* s_d, void* eta) {
  if (!P || !s_d || !eta) return ISAM_ERR_INVALID;
  DeviceGuard g(P->device);
  P->launches = 0;
  if (P->p.precision == ISAM_FP64)
    return dc_ifft_impl<double>(P, static_cast<const double*>(s_d), static_cast<double2*>(eta));
  return dc_ifft_impl<float>(P, static_cast<const float*>(s_d), static_cast<float2*>(eta));
}

}  // extern "C"


// ----------------------------------------------------------------------------
// Batched solves recorded as one CUDA graph
// ----------------------------------------------------------------------------
struct isam_batch {
  int n = 0;
  int device = 0;
  std::vector<isam_plan*> plans;
  std::vector<isam_solve_opts> opts;
  std::vector<double> L;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  // timing: recorded as event nodes of the graph, at its start and at the end
  // of every entry's solve
  cudaEvent_t t_start = nullptr;
  std::vector<cudaEvent_t> t_done;
  bool ran = false;
  cudaEvent_t fork = nullptr;
  cudaStream_t origin = nullptr;
  bool own_origin = false;      // created here (capture cannot use the legacy stream)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;   // kernel launches recorded in the graph
};

namespace {

// Everything a recorded solve needs that cannot happen during capture:
// workspace allocation and the Lipschitz constant (cached per plan).
template <typename T> isam_status batch_prepare(isam_plan* P, const isam_solve_opts* o,
                                                double* L_out) {
  Impl<T>& im = impl_of<T>(P);
  if (!im.zA) ISAM_TRY(dalloc(&im.zA, P->n_img));
  if (!im.zB) ISAM_TRY(dalloc(&im.zB, P->n_img));
  if (!im.sdh) ISAM_TRY(dalloc(&im.sdh, P->n_spec));
  if (!im.s_tmp) ISAM_TRY(dalloc(&im.s_tmp, P->n_spec));
  if (o->prior == ISAM_PRIOR_TV && !im.tv) ISAM_TRY(dalloc(&im.tv, 5 * P->n_img));
  double L = o->L;
  if (!(L > 0)) {
    if (!(P->L_cache > 0)) {
      double Lc = 0.0;
      if (precision_fits<double>(P))
        ISAM_TRY(power_iteration<double>(P, kPowerIters, kPowerRtol, nullptr, 0, &Lc));
      else
        ISAM_TRY(power_iteration<T>(P, kPowerIters, kPowerRtol, nullptr, 0, &Lc));
      P->L_cache = Lc;
    }
    L = P->L_cache;
  }
  if (!(L > 0)) return ISAM_ERR_INVALID;
  *L_out = L;
  return ISAM_OK;
}

// One whole solve on the plan's stream with no host synchronisation: the
// relative lambda = c ||A^H s_d||_inf stays on the device (the update kernel
// reads it), so a recorded graph stays correct when s_d's contents change.
// With tol > 0 the stop rule runs on the device (StopRule): every iteration
// after the first check carries the stop flag, and the output is the iterate
// of the stopping check (launch_select_iterate).
template <typename T> isam_status batch_enqueue(isam_plan* P, const T* s_d,
                                                const isam_solve_opts* o, double L,
                                                cplx<T>* eta_out) {
  Impl<T>& im = impl_of<T>(P);
  cudaStream_t s = P->stream;
  const size_t bytes = sizeof(cplx<T>) * P->n_img;
  CUDA_TRY(cudaMemsetAsync(P->flag, 0, sizeof(int), s));
  ISAM_TRY(lat_forward<T>(P, im, s_d, im.sdh, P->nk, true));
  const double lam = o->lambda_abs;
  const double* lam_dev = nullptr;
  double lam_scale = 0.0;
  if (!(lam > 0)) {
    ISAM_TRY(op_adjoint<T>(P, s_d, im.zA));
    ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
      return launch_max_abs<T>(im.zA, P->n_img, P->partial, RED_BLOCKS, P->dscal, s);
    }));
    lam_dev = P->dscal;
    lam_scale = o->lambda_rel / L;
  }
  CUDA_TRY(cudaMemsetAsync(im.zA, 0, bytes, s));
  CUDA_TRY(cudaMemsetAsync(im.zB, 0, bytes, s));
  CUDA_TRY(cudaMemsetAsync(im.eta_hat, 0, bytes, s));
  if (o->prior == ISAM_PRIOR_TV) CUDA_TRY(cudaMemsetAsync(im.tv, 0, 2 * bytes, s));
  std::vector<double> mu;
  momentum(o->max_iter + 1, mu);
  cplx<T>* zP = im.zA;
  cplx<T>* zQ = im.zB;
  const T* w = static_cast<const T*>(o->w_dev);
  const bool check = o->tol > 0;
  const int every = std::max(1, o->check_every);
  const int first_check = std::min(every, o->max_iter);
  if (check) CUDA_TRY(cudaMemsetAsync(P->dstop, 0, 2 * sizeof(int), s));
  for (int k = 1; k <= o->max_iter; ++k) {
    const bool norms = check && (k % every == 0 || k == o->max_iter);
    StopRule sr{};
    sr.stop = P->dstop;
    sr.rr = P->dscal + 7;
    sr.tol = o->tol;
    sr.eps = o->eps > 0 ? o->eps : 1e-30;
    sr.iter = k;
    ISAM_TRY(fista_iteration<T>(P, im, zP, zQ, zQ, w, lam, L, mu[k - 1], mu[k], norms, nullptr,
                                nullptr, nullptr, lam_dev, lam_scale, o->prior, o->prior_iters,
                                nullptr, check && k > first_check ? P->dstop : nullptr,
                                norms ? &sr : nullptr));
    std::swap(zP, zQ);
  }
  cplx<T>* z = zP;
  if (check) {
    // z^{k_stop} (the last iterate when the rule did not fire) into eta_out;
    // the add-back below reads it there and updates it in place
    z = eta_out;
    ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
      return launch_select_iterate<T>(zP, zQ, z, P->n_img, P->dstop, o->max_iter, s);
    }));
  }
  if (o->residual_addback) {
    ISAM_TRY(op_forward<T>(P, z, im.s_tmp));
    ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
      return launch_rsub<T>(s_d, im.s_tmp, im.s_tmp, P->n_spec, s);
    }));
    ISAM_TRY(op_adjoint<T>(P, im.s_tmp, im.grad));
    ISAM_TRY(launch(P, ISAM_KCLASS_MISC, [&] {
      return launch_caxpy<T>(z, im.grad, T(1.0 / L), eta_out, P->n_img, s);
    }));
  } else if (!check) {
    CUDA_TRY(cudaMemcpyAsync(eta_out, zP, bytes, cudaMemcpyDeviceToDevice, s));
  }
  return ISAM_OK;
}

void batch_free(isam_batch* B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  for (cudaStream_t st : B->streams) cudaStreamDestroy(st);
  for (cudaEvent_t e : B->joins) cudaEventDestroy(e);
  for (cudaEvent_t e : B->t_done) cudaEventDestroy(e);
  if (B->t_start) cudaEventDestroy(B->t_start);
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->own_origin && B->origin) cudaStreamDestroy(B->origin);
  delete B;
}

}  // namespace

extern "C" {

isam_status isam_batch_create(isam_plan* const* plans, int32_t n, const void* const* s_d,
                              const isam_solve_opts* opts, void* const* eta_out, void* stream,
                              isam_batch** out) {
  if (!out) return ISAM_ERR_INVALID;
  *out = nullptr;
  if (!plans || n < 1 || !s_d || !opts || !eta_out) return ISAM_ERR_INVALID;
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !s_d[i] || !eta_out[i]) return ISAM_ERR_INVALID;
    ISAM_TRY(check_opts(plans[i], &opts[i]));
    if (plans[i]->prof || plans[i]->device != plans[0]->device) return ISAM_ERR_INVALID;
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return ISAM_ERR_INVALID;
  }
  DeviceGuard g(plans[0]->device);
  isam_batch* B = new isam_batch();
  B->n = n;
  B->device = plans[0]->device;
  B->origin = static_cast<cudaStream_t>(stream);
  B->plans.assign(plans, plans + n);
  B->opts.assign(opts, opts + n);
  B->L.assign(n, 0.0);
  isam_status st = ISAM_OK;
  for (int i = 0; i < n && st == ISAM_OK; ++i) {
    isam_plan* P = plans[i];
    st = P->p.precision == ISAM_FP64 ? batch_prepare<double>(P, &opts[i], &B->L[i])
                                     : batch_prepare<float>(P, &opts[i], &B->L[i]);
    if (st == ISAM_OK) st = from_cuda(cudaStreamSynchronize(P->stream));
  }
  if (st == ISAM_OK && !B->origin) {
    st = from_cuda(cudaStreamCreateWithFlags(&B->origin, cudaStreamNonBlocking));
    B->own_origin = st == ISAM_OK;
  }
  if (st == ISAM_OK) st = from_cuda(cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming));
  if (st == ISAM_OK) st = from_cuda(cudaEventCreate(&B->t_start));
  for (int i = 0; i < n && st == ISAM_OK; ++i) {
    cudaStream_t sx = nullptr;
    cudaEvent_t ev = nullptr, td = nullptr;
    st = from_cuda(cudaStreamCreateWithFlags(&sx, cudaStreamNonBlocking));
    if (st == ISAM_OK) B->streams.push_back(sx);
    if (st == ISAM_OK) st = from_cuda(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    if (st == ISAM_OK) B->joins.push_back(ev);
    if (st == ISAM_OK) st = from_cuda(cudaEventCreate(&td));
    if (st == ISAM_OK) B->t_done.push_back(td);
  }
  if (st != ISAM_OK) {
    batch_free(B);
    return st;
  }
  // record: fork every entry onto its own stream, join them back
  st = from_cuda(cudaStreamBeginCapture(B->origin, cudaStreamCaptureModeRelaxed));
  if (st == ISAM_OK)
    st = from_cuda(cudaEventRecordWithFlags(B->t_start, B->origin, cudaEventRecordExternal));
  if (st == ISAM_OK) st = from_cuda(cudaEventRecord(B->fork, B->origin));
  for (int i = 0; i < n && st == ISAM_OK; ++i) {
    isam_plan* P = plans[i];
    cudaStream_t saved = P->stream;
    const int64_t l0 = P->launches;
    P->stream = B->streams[i];
    st = from_cuda(cudaStreamWaitEvent(P->stream, B->fork, 0));
    if (st == ISAM_OK)
      st = P->p.precision == ISAM_FP64
               ? batch_enqueue<double>(P, static_cast<const double*>(s_d[i]), &opts[i], B->L[i],
                                       static_cast<double2*>(eta_out[i]))
               : batch_enqueue<float>(P, static_cast<const float*>(s_d[i]), &opts[i], B->L[i],
                                      static_cast<float2*>(eta_out[i]));
    if (st == ISAM_OK)
      st = from_cuda(cudaEventRecordWithFlags(B->t_done[i], P->stream, cudaEventRecordExternal));
    if (st == ISAM_OK) st = from_cuda(cudaEventRecord(B->joins[i], P->stream));
    if (st == ISAM_OK) st = from_cuda(cudaStreamWaitEvent(B->origin, B->joins[i], 0));
    B->kernels += P->launches - l0;
    P->stream = saved;
  }
  cudaGraph_t graph = nullptr;
  const isam_status end = from_cuda(cudaStreamEndCapture(B->origin, &graph));
  B->graph = graph;
  if (st == ISAM_OK) st = end;
  if (st == ISAM_OK) st = from_cuda(cudaGraphInstantiate(&B->exec, B->graph, 0));
  if (st != ISAM_OK) {
    cudaGetLastError();
    batch_free(B);
    return st;
  }
  for (isam_plan* P : B->plans) ++P->batch_refs;
  *out = B;
  return ISAM_OK;
}

isam_status isam_batch_run(isam_batch* B, isam_solve_info* info) {
  if (!B) return ISAM_ERR_INVALID;
  DeviceGuard g(B->device);
  CUDA_TRY(cudaGraphLaunch(B->exec, B->origin));
  CUDA_TRY(cudaStreamSynchronize(B->origin));
  B->ran = true;
  isam_status first = ISAM_OK;
  for (int i = 0; i < B->n; ++i) {
    isam_plan* P = B->plans[i];
    int flag = 0;
    double m = 0.0;
    CUDA_TRY(cudaMemcpy(&flag, P->flag, sizeof(int), cudaMemcpyDeviceToHost));
    const isam_solve_opts& o = B->opts[i];
    double lam = o.lambda_abs;
    if (!(lam > 0)) {
      CUDA_TRY(cudaMemcpy(&m, P->dscal, sizeof(double), cudaMemcpyDeviceToHost));
      lam = o.lambda_rel * m;
    }
    // the device-side stop rule's outcome: [stopped, iteration] and r_r
    int stop[2] = {0, 0};
    double rr = -1.0;
    if (o.tol > 0) {
      CUDA_TRY(cudaMemcpy(stop, P->dstop, 2 * sizeof(int), cudaMemcpyDeviceToHost));
      CUDA_TRY(cudaMemcpy(&rr, P->dscal + 7, sizeof(double), cudaMemcpyDeviceToHost));
    }
    const isam_status st = flag ? ISAM_ERR_NONFINITE : ISAM_OK;
    if (st != ISAM_OK && first == ISAM_OK) first = st;
    if (info) {
      info[i].iterations = stop[0] ? stop[1] : o.max_iter;
      info[i].rr = rr;
      info[i].lambda = lam;
      info[i].L = B->L[i];
      info[i].status = st;
      info[i].objective = -1.0;
    }
  }
  return first;
}

int64_t isam_batch_kernel_count(const isam_batch* B) { return B ? B->kernels : -1; }

isam_status isam_batch_entry_ms(const isam_batch* B, double* ms) {
  if (!B || !ms) return ISAM_ERR_INVALID;
  if (!B->ran) return ISAM_ERR_INVALID;
  DeviceGuard g(B->device);
  for (int i = 0; i < B->n; ++i) {
    float t = 0.0f;
    CUDA_TRY(cudaEventElapsedTime(&t, B->t_start, B->t_done[i]));
    ms[i] = double(t);
  }
  return ISAM_OK;
}

void isam_batch_destroy(isam_batch* B) {
  if (!B) return;
  DeviceGuard g(B->device);
  cudaStreamSynchronize(B->origin);
  for (isam_plan* P : B->plans) --P->batch_refs;
  batch_free(B);
}

}  // extern "C"

// ----------------------------------------------------------------------------
// Autotuning of launch shapes on the plan's own workload
// ----------------------------------------------------------------------------
namespace {

// Device time of `reps` FISTA iterations (after 2 untimed ones) on zero data:
// the kernels' work does not depend on the values.
template <typename T> isam_status time_iterations(isam_plan* P, int reps, float* ms) {
  Impl<T>& im = impl_of<T>(P);
  cudaStream_t s = P->stream;
  const size_t bytes = sizeof(cplx<T>) * P->n_img;
  CUDA_TRY(cudaMemsetAsync(im.zA, 0, bytes, s));
  CUDA_TRY(cudaMemsetAsync(im.zB, 0, bytes, s));
  CUDA_TRY(cudaMemsetAsync(im.eta_hat, 0, bytes, s));
  CUDA_TRY(cudaMemsetAsync(im.sdh, 0, sizeof(cplx<T>) * P->n_spec, s));
  cudaEvent_t a = nullptr, b = nullptr;
  CUDA_TRY(cudaEventCreate(&a));
  CUDA_TRY(cudaEventCreate(&b));
  isam_status st = ISAM_OK;
  for (int i = 0; i < reps + 2 && st == ISAM_OK; ++i) {
    if (i == 2) cudaEventRecord(a, s);
    st = fista_iteration<T>(P, im, im.zA, im.zB, im.zB, nullptr, 1.0, 1.0, 0.5, 0.5, false);
  }
  cudaEventRecord(b, s);
  if (st == ISAM_OK) st = from_cuda(cudaEventSynchronize(b));
  if (st == ISAM_OK) st = from_cuda(cudaEventElapsedTime(ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  harvest_events(P);
  return st;
}

// Key of a plan's launch-shape choice in the autotune cache file: the device
// and everything the timed kernels' shapes depend on.
std::string tune_key(const isam_plan* P, bool has_table) {
  cudaDeviceProp prop{};
  std::string dev = "gpu";
  if (cudaGetDeviceProperties(&prop, P->device) == cudaSuccess) dev = prop.name;
  for (char& c : dev)
    if (c == ' ') c = '_';
  char buf[256];
  snprintf(buf, sizeof(buf), "%s nx=%d ny=%d nk=%d nz=%d prec=%d J=%d table=%d", dev.c_str(),
           P->nx, P->ny, P->nk, P->nz, P->p.precision, P->J, has_table ? 1 : 0);
  return buf;
}

// One tuning of a plan: lateral tile (0: built-in), Stolt-table mode (0: the
// plan's default, 1: table, 2: evaluated), FFT radices (8 or 16).
struct Tuning {
  int tp = 0, tab = 0, rax = 16, rlat = 16;
};

// Cached choice for `key` from the file named by ISAM_AUTOTUNE_CACHE: lines
// "<key> -> tile=<t> stolt=<m> radix=<axial>/<lateral>" (lines without the
// radices, from earlier builds, mean 16/16); the last matching line wins.
bool tune_cache_lookup(const std::string& key, Tuning* out) {
  const char* path = getenv("ISAM_AUTOTUNE_CACHE");
  if (!path || !*path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  const std::string head = key + " -> ";
  while (fgets(line, sizeof(line), f)) {
    if (strncmp(line, head.c_str(), head.size()) != 0) continue;
    Tuning t;
    int consumed = 0;
    if (sscanf(line + head.size(), "tile=%d stolt=%d%n", &t.tp, &t.tab, &consumed) == 2) {
      int ra = 16, rl = 16;
      if (sscanf(line + head.size() + consumed, " radix=%d/%d", &ra, &rl) == 2) {
        t.rax = ra;
        t.rlat = rl;
      }
      *out = t;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void tune_cache_store(const std::string& key, const Tuning& t) {
  const char* path = getenv("ISAM_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s -> tile=%d stolt=%d radix=%d/%d\n", key.c_str(), t.tp, t.tab, t.rax, t.rlat);
  fclose(f);
}

// lateral extent and columns of the update pass (y for volumes)
void update_geometry(const isam_plan* P, int* L, int* M) {
  *L = P->ny == 1 ? P->nx : P->ny;
  *M = P->ny == 1 ? P->nz : P->nx * P->nz;
}

template <typename T> bool tuning_feasible(const isam_plan* P, const Tuning& t) {
  const Impl<T>& im = impl_of<T>(const_cast<isam_plan*>(P));
  int L, M;
  update_geometry(P, &L, &M);
  const bool tile_ok = t.tp == 0 || ((t.tp == 1 || t.tp == 2 || t.tp == 4 || t.tp == 8) &&
                                     t.tp <= M / 2 && (L >= 8 ? L / 8 : 1) * t.tp <= 512);
  const bool tab_ok = t.tab == 0 || ((t.tab == 1 || t.tab == 2) && im.tab.stab);
  const bool radix_ok = (t.rax == 8 || t.rax == 16) && (t.rlat == 8 || t.rlat == 16);
  return tile_ok && tab_ok && radix_ok;
}

void apply_tuning(isam_plan* P, const Tuning& t) {
  P->tune_tp = t.tp;
  P->tune_table = t.tab;
  P->tune_radix_ax = t.rax;
  P->tune_radix_lat = t.rlat;
}

template <typename T> void report_tuning(const isam_plan* P, isam_tuning* out) {
  const Impl<T>& im = impl_of<T>(const_cast<isam_plan*>(P));
  int L, M;
  update_geometry(P, &L, &M);
  out->lateral_tile = P->tune_tp ? P->tune_tp : lat_tile(L, M);
  out->stolt_table = P->tune_table == 2 ? 0 : (im.tab.stab ? 1 : 0);
  out->axial_radix = P->tune_radix_ax;
  out->lateral_radix = P->tune_radix_lat;
}

template <typename T> isam_status autotune_impl(isam_plan* P, isam_tuning* out) {
  Impl<T>& im = impl_of<T>(P);
  const std::string key = tune_key(P, im.tab.stab != nullptr);
  {
    // a cached choice that is still feasible for this plan is used as is
    Tuning t;
    if (tune_cache_lookup(key, &t) && tuning_feasible<T>(P, t)) {
      apply_tuning(P, t);
      if (out) report_tuning<T>(P, out);
      return ISAM_OK;
    }
  }
  if (!im.zA) ISAM_TRY(dalloc(&im.zA, P->n_img));
  if (!im.zB) ISAM_TRY(dalloc(&im.zB, P->n_img));
  if (!im.sdh) ISAM_TRY(dalloc(&im.sdh, P->n_spec));
  int L, M;
  update_geometry(P, &L, &M);
  const int threads_per_tp = L >= 8 ? L / 8 : 1;
  const bool fp32 = P->p.precision == ISAM_FP32;
  // radix-16 forms exist for FP32 axial transforms at K = 2048, 4096 and FP32
  // lateral tiles (L, tile) = (1024, 4) and (256, 8) of lengths 2^p
  const bool ax_both = fp32 && (P->K == 2048 || P->K == 4096);
  const bool prof = P->prof;
  P->prof = false;
  const int reps = 10;
  float best = 0.0f;
  Tuning best_t;
  bool have = false;
  const int tabs[2] = {1, 2};
  const int ntab = im.tab.stab ? 2 : 1;
  isam_status st = ISAM_OK;
  for (int it = 0; it < ntab && st == ISAM_OK; ++it) {
    for (int tp = 1; tp <= 8 && st == ISAM_OK; tp *= 2) {
      if (tp > M / 2 || threads_per_tp * tp > 512) continue;
      const bool lat_both = fp32 && ((L == 1024 && tp == 4) || (L == 256 && tp == 8));
      for (int ra = ax_both ? 8 : 16; ra <= 16 && st == ISAM_OK; ra += 8) {
        for (int rl = lat_both ? 8 : 16; rl <= 16 && st == ISAM_OK; rl += 8) {
          Tuning t;
          t.tp = tp;
          t.tab = im.tab.stab ? tabs[it] : 0;
          t.rax = ra;
          t.rlat = rl;
          apply_tuning(P, t);
          float ms = 0.0f;
          st = time_iterations<T>(P, reps, &ms);
          if (st == ISAM_OK && (!have || ms < best)) {
            best = ms;
            best_t = t;
            have = true;
          }
        }
      }
    }
  }
  P->prof = prof;
  apply_tuning(P, st == ISAM_OK ? best_t : Tuning());
  if (st == ISAM_OK) tune_cache_store(key, best_t);
  if (out) report_tuning<T>(P, out);
  return st;
}

}  // namespace

extern "C" {

isam_status isam_autotune_ex(isam_plan* P, isam_tuning* out) {
  if (!P) return ISAM_ERR_INVALID;
  if (P->batch_refs) return ISAM_ERR_INVALID;       // a batch graph records the plan
  DeviceGuard g(P->device);
  P->launches = 0;
  if (P->p.precision == ISAM_FP64) return autotune_impl<double>(P, out);
  return autotune_impl<float>(P, out);
}

isam_status isam_autotune(isam_plan* P, int32_t* tile, int32_t* stolt_table) {
  isam_tuning t{};
  const isam_status st = isam_autotune_ex(P, &t);
  if (tile) *tile = t.lateral_tile;
  if (stolt_table) *stolt_table = t.stolt_table;
  return st;
}

isam_status isam_get_tuning(const isam_plan* P, isam_tuning* out) {
  if (!P || !out) return ISAM_ERR_INVALID;
  if (P->p.precision == ISAM_FP64) report_tuning<double>(P, out);
  else report_tuning<float>(P, out);
  return ISAM_OK;
}

isam_status isam_set_tuning(isam_plan* P, const isam_tuning* in) {
  if (!P || !in) return ISAM_ERR_INVALID;
  if (P->batch_refs) return ISAM_ERR_INVALID;
  const bool has_table = P->p.precision == ISAM_FP64 ? P->f64.tab.stab != nullptr
                                                      : P->f32.tab.stab != nullptr;
  if (in->stolt_table != 0 && in->stolt_table != 1) return ISAM_ERR_INVALID;
  if (in->stolt_table == 1 && !has_table) return ISAM_ERR_UNSUPPORTED;
  Tuning t;
  t.tp = in->lateral_tile;
  t.tab = in->stolt_table == 1 ? 1 : (has_table ? 2 : 0);
  t.rax = in->axial_radix;
  t.rlat = in->lateral_radix;
  const bool ok = P->p.precision == ISAM_FP64 ? tuning_feasible<double>(P, t)
                                              : tuning_feasible<float>(P, t);
  if (!ok) return ISAM_ERR_INVALID;
  apply_tuning(P, t);
  return ISAM_OK;
}

}  // extern "C"

