"""FP64 CPU oracle for full-range dispersion-encoded ISAM (arXiv 1905.06058).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports, links or runs this
file; only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it, to check and to time the CUDA path.  It shares no code,
table or constant generator with the CUDA path: it recomputes every grid,
phase, Stolt position and NUFFT coefficient itself, in float64, the plain way.

What it computes (paper section / equation in brackets):

* forward model  s = Re(K_hat eta),  K_hat = diag(e^{j phi}) K   [§3, Eq. 12-13]
  with the ISAM operator K realised as lateral FFT, Stolt-mapped axial
  transform, lateral inverse FFT [§2, Eq. 1-5; §3.2, Eq. 16, b = 1]
  - mode "exact": the axial transform as the plain nonuniform DFT, i.e. the
    definition of H(q, beta) sampled at beta = -sqrt(4k^2 - q^2) [Eq. 3];
  - mode "nufft": the min-max-optimal NUFFT of Fessler & Sutton (cited in
    §3.2): scaling, zero-padded oversampled FFT, J-neighbour interpolation
    with coefficients that minimise the worst-case error, solved per point;
* adjoint  A^H y = K_hat^H y under the real inner product  [Eq. 17];
* weighted complex soft threshold [Eq. 14], relative residual [Eq. 15],
  the prox of an l1 prior on orthonormal Haar detail coefficients along depth
  and of an isotropic total-variation prior (fast dual gradient projection)
  (the other convex priors §3.1 names),
  FISTA [Alg. 1], residual add-back [Alg. 1, optional last step];
* Lipschitz constant of the gradient by power iteration;
* the optional filter B(q, k) of Eq. 3 (b of Eq. 16), as a table over |q|;
* the 1-D per-A-scan model of the DEFR objective (Eq. 10) and the
  dispersion-compensated IFFT (Eq. 9);
* derivatives for calibrating the dispersion coefficients a_1..a_4 (Eq. 7)
  and the focal depth z0 by gradient descent: <dA/dtheta x, y>, the
  Jacobian-transpose of the soft threshold (Eq. 14), and the gradient of
  <z_bar, z^K> through K unrolled FISTA iterations (Alg. 1) with lambda and
  L held fixed.

Readings of points the paper leaves open (they are the same on the CUDA
side, implemented independently):

* grids: k_j = k_min + j dk (j < nk, dk = (k_max-k_min)/(nk-1)), k0 the band
  centre; dz = pi/(nz dk); z_n = (n - nz/2) dz; q = 2 pi fftfreq(n, d);
* unitary lateral FFTs; axial transform scaled by 1/sqrt(nz);
* focus depth z0 enters as the phase e^{j(2k+beta)z0} (1 at q = 0);
* evanescent samples (4k^2 <= q^2) are zero in A and ignored in A^H;
* NUFFT: oversampling K = 2 nz, J even (default 6), Kaiser-Bessel-shaped
  scaling s(n') = psi_hat(0)/psi_hat(n'/K) with alpha = 2.34 J, min-max
  design over the symmetric index set n' = -nz/2 .. nz/2 (so coefficients
  are real); neighbours floor(p)-J/2+1 .. floor(p)+J/2 of position p;
* step 1/L and threshold lambda w / L in place of the paper's 1/N
  (Alg. 1, Eq. 14), L = ||A||^2;
* t^1 = 1, eta^1 = z^0 = 0; the returned image is z^k; the add-back is
  z^k + (1/L) A^H (s_d - A z^k).

Parity status: every public function here is pinned by a test in
tests/test_oracle_*.py against a closed form, a library routine, a
brute-force construction or an invariant (see each docstring).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np

# ----------------------------------------------------------------------------
# Grids and phases  (§2; conventions listed in the module docstring)
# ----------------------------------------------------------------------------


@dataclass
class Grid:
    nx: int
    ny: int
    nk: int
    nz: int
    k: np.ndarray       # [nk] wavenumbers, rad/m
    k0: float           # band centre (Eq. 7)
    dk: float
    dz: float
    z: np.ndarray       # [nz] depths, m (zero delay at index nz/2)
    q2: np.ndarray      # [ny, nx] squared lateral frequency qx^2 + qy^2


def make_grid(g) -> Grid:
    """Spectral, depth and lateral-frequency grids of a geometry ``g``."""
    nz = g.nz or g.nk
    dk = (g.k_max - g.k_min) / (g.nk - 1)
    k = g.k_min + dk * np.arange(g.nk)
    dz = math.pi / (nz * dk)
    z = (np.arange(nz) - nz // 2) * dz
    qx = 2 * math.pi * np.fft.fftfreq(g.nx, d=g.dx)
    qy = 2 * math.pi * np.fft.fftfreq(g.ny, d=g.dy) if g.ny > 1 else np.zeros(1)
    q2 = qy[:, None] ** 2 + qx[None, :] ** 2
    return Grid(g.nx, g.ny, g.nk, nz, k, 0.5 * (g.k_min + g.k_max), dk, dz, z, q2)


def dispersion_phase(g, grid: Grid) -> np.ndarray:
    """phi(k) = sum_i a_i (k - k0)^i  [§2, Eq. 7]."""
    dk = grid.k - grid.k0
    phi = np.zeros_like(grid.k)
    for i, a in enumerate(g.disp, start=1):
        phi += a * dk ** i
    return phi


def stolt_beta(q2: np.ndarray, k: np.ndarray):
    """beta = -sqrt(4k^2 - q^2) and the propagating mask 4k^2 > q^2  [Eq. 3]."""
    arg = 4.0 * k ** 2 - q2
    prop = arg > 0
    beta = -np.sqrt(np.where(prop, arg, 0.0))
    return beta, prop


def spectral_phase(g, grid: Grid) -> np.ndarray:
    """e^{j phi(k)} e^{j (2k + beta) z0} on propagating samples, 0 elsewhere.

    Shape [ny, nx, nk].  The first factor is the dispersion encoding
    [Eq. 7, Eq. 13]; the second places the Stolt map's origin at the focus.
    """
    beta, prop = stolt_beta(grid.q2[..., None], grid.k[None, None, :])
    ph = np.exp(1j * dispersion_phase(g, grid))[None, None, :] * \
        np.exp(1j * (2 * grid.k[None, None, :] + beta) * g.z0)
    return np.where(prop, ph, 0.0)


# ----------------------------------------------------------------------------
# Lateral transforms  F<->, F<->^{-1}  (§2, unitary)
# ----------------------------------------------------------------------------


def lateral_fft(a: np.ndarray) -> np.ndarray:
    return np.fft.fft2(a, axes=(0, 1), norm="ortho")


def lateral_ifft(a: np.ndarray) -> np.ndarray:
    return np.fft.ifft2(a, axes=(0, 1), norm="ortho")


# ----------------------------------------------------------------------------
# Min-max NUFFT (Fessler & Sutton, cited in §3.2)
# ----------------------------------------------------------------------------


def kb_scaling(nz: int, K: int, J: int) -> tuple[np.ndarray, np.ndarray]:
    """Design index set n' = -nz/2..nz/2 and scaling s(n') = psi_hat(0)/psi_hat(n'/K).

    psi_hat is the Fourier transform of a Kaiser-Bessel window of width J,
    sinh(sqrt(a^2 - (pi J v)^2)) / sqrt(a^2 - (pi J v)^2), a = 2.34 J.
    """
    alpha = 2.34 * J
    n = np.arange(-(nz // 2), nz // 2 + 1)

    def psi_hat(v):
        r = np.sqrt(alpha ** 2 - (math.pi * J * v) ** 2)
        return np.sinh(r) / r

    return n, psi_hat(0.0) / psi_hat(n / K)


class MinMaxInterpolator:
    """Min-max interpolation coefficients of one (nz, K, J) design.

    For a target position p (in oversampled-grid units) with fractional part
    f, the J real coefficients c minimise the worst case over unit-norm
    signals of the interpolation error, which is the least-squares problem

        min_c  sum_{n'} | s(n') sum_l c_l e^{j g (l-(J-1)/2) n'} - e^{j g (f-1/2) n'} |^2,

    g = 2 pi / K, over the symmetric design set n'.  It is solved in float64
    with a pseudo-inverse of the (nz+1) x J design matrix, per point.
    """

    def __init__(self, nz: int, K: int, J: int):
        if J % 2:
            raise ValueError("J must be even")
        self.nz, self.K, self.J = nz, K, J
        self.n, self.s = kb_scaling(nz, K, J)
        g = 2 * math.pi / K
        lam = np.arange(J) - (J - 1) / 2
        self.B = self.s[:, None] * np.exp(1j * g * np.outer(self.n, lam))
        self.P = np.linalg.pinv(self.B)

    def coefficients(self, f: np.ndarray, chunk: int = 4096) -> np.ndarray:
        """Real coefficients [len(f), J] for fractional offsets f in [0, 1)."""
        f = np.asarray(f, np.float64).ravel()
        g = 2 * math.pi / self.K
        out = np.empty((f.size, self.J))
        for a in range(0, f.size, chunk):
            V = np.exp(1j * g * np.outer(self.n, f[a:a + chunk] - 0.5))
            C = self.P @ V
            out[a:a + chunk] = C.real.T
        return out

    def worst_case_error(self, f: np.ndarray) -> np.ndarray:
        """max over ||x||=1 of the interpolation error = LS residual norm."""
        c = self.coefficients(f)
        g = 2 * math.pi / self.K
        V = np.exp(1j * g * np.outer(self.n, np.asarray(f) - 0.5))
        return np.linalg.norm(self.B @ c.T - V, axis=0)

    def scaling_of_samples(self) -> np.ndarray:
        """s(n') for the nz data samples n' = n - nz/2, n = 0..nz-1."""
        return self.s[:-1]


def grid_position(beta: np.ndarray, dz: float, K: int) -> np.ndarray:
    """Oversampled-grid coordinate p = omega / (2 pi / K), omega = -beta dz."""
    return -beta * dz * K / (2 * math.pi)


def nufft_forward_column(x: np.ndarray, p: np.ndarray, interp: MinMaxInterpolator,
                         c: Optional[np.ndarray] = None) -> np.ndarray:
    """X(p_j) ~= sum_n x_n e^{j 2 pi p_j (n - nz/2) / K}, min-max NUFFT.

    Steps: scale by s, zero-pad to K with sample n at n - nz/2 mod K,
    K-point DFT with e^{+j}, J-neighbour interpolation.  ``c`` optionally
    passes the coefficients of these positions, computed earlier by
    ``interp.coefficients`` (a memo; the arithmetic is the same).
    """
    nz, K, J = interp.nz, interp.K, interp.J
    v = np.zeros(K, np.complex128)
    idx = (np.arange(nz) - nz // 2) % K
    v[idx] = interp.scaling_of_samples() * x
    Y = np.fft.ifft(v) * K                      # sum_p v_p e^{+j 2 pi m p / K}
    fl = np.floor(p)
    f = p - fl
    m0 = fl.astype(np.int64) - J // 2 + 1
    if c is None:
        c = interp.coefficients(f)
    out = np.zeros(p.shape, np.complex128)
    for l in range(J):
        out += c[:, l] * Y[(m0 + l) % K]
    return out


def nufft_adjoint_column(y: np.ndarray, p: np.ndarray, interp: MinMaxInterpolator,
                         c: Optional[np.ndarray] = None) -> np.ndarray:
    """Exact adjoint of ``nufft_forward_column`` (ISAM back-projection, Eq. 17)."""
    nz, K, J = interp.nz, interp.K, interp.J
    fl = np.floor(p)
    f = p - fl
    m0 = fl.astype(np.int64) - J // 2 + 1
    if c is None:
        c = interp.coefficients(f)
    Yg = np.zeros(K, np.complex128)
    for l in range(J):
        np.add.at(Yg, (m0 + l) % K, c[:, l] * y)
    w = np.fft.fft(Yg)                           # sum_m Yg_m e^{-j 2 pi m p / K}
    idx = (np.arange(nz) - nz // 2) % K
    return interp.scaling_of_samples() * w[idx]


# ----------------------------------------------------------------------------
# The ISAM operator and its adjoint
# ----------------------------------------------------------------------------


def expand_filter(g, table: np.ndarray) -> np.ndarray:
    """The filter B(q, k) of Eq. 3 on every lateral-frequency column, [ny, nx, nk],
    from a table over |q| classes, [ny//2 + 1, nx//2 + 1, nk]: column (iy, ix)
    takes row (|my|, |mx|) with m the signed FFT index (B symmetric in q)."""
    ny, nx = g.ny, g.nx
    my = np.abs(np.fft.fftfreq(ny, 1.0 / ny).astype(int)) if ny > 1 else np.zeros(1, int)
    mx = np.abs(np.fft.fftfreq(nx, 1.0 / nx).astype(int))
    return table[my[:, None], mx[None, :], :]


class IsamOracle:
    """A = Re o diag(e^{j phi}) o K and A^H for one geometry  [Eq. 12-13, 16-17].

    ``filt`` (optional): the filter B of Eq. 3 as a table over |q| classes
    (see expand_filter); S = B . e^{j phi} e^{j(2k+beta)z0} . H (b of Eq. 16)."""

    def __init__(self, g, mode: str = "nufft", J: int = 6, filt: Optional[np.ndarray] = None):
        if mode not in ("exact", "nufft"):
            raise ValueError(mode)
        self.g, self.mode, self.J = g, mode, J
        self.grid = make_grid(g)
        gr = self.grid
        self.phase = spectral_phase(g, gr)                         # [ny,nx,nk]
        if filt is not None:
            self.phase = self.phase * expand_filter(g, filt)
        self.beta, self.prop = stolt_beta(gr.q2[..., None], gr.k[None, None, :])
        self.K = 2 * gr.nz
        self.interp = MinMaxInterpolator(gr.nz, self.K, J) if mode == "nufft" else None
        self.p = grid_position(self.beta, gr.dz, self.K)            # [ny,nx,nk]

    @property
    def image_shape(self):
        return (self.grid.ny, self.grid.nx, self.grid.nz)

    @property
    def spec_shape(self):
        return (self.grid.ny, self.grid.nx, self.grid.nk)

    # -- axial (per lateral-frequency column) --------------------------------
    def _nudft_matrix(self, iy, ix):
        """e^{-j beta_j z_n} of one column (kept when the whole set is small)."""
        key = (iy, ix)
        cache = self.__dict__.setdefault("_E", {})
        if key in cache:
            return cache[key]
        E = np.exp(-1j * np.outer(self.beta[iy, ix], self.grid.z))
        if self.grid.nx * self.grid.ny * E.size <= 4_000_000:
            cache[key] = E
        return E

    def _coef(self, iy, ix):
        """Min-max coefficients of one column's Stolt positions (memoised)."""
        cache = self.__dict__.setdefault("_C", {})
        if (iy, ix) in cache:
            return cache[(iy, ix)]
        p = self.p[iy, ix]
        c = self.interp.coefficients(p - np.floor(p))
        if self.grid.nx * self.grid.ny * c.size <= 50_000_000:
            cache[(iy, ix)] = c
        return c

    def _axial_exact_col(self, x, iy, ix):
        return self._nudft_matrix(iy, ix) @ x / math.sqrt(self.grid.nz)

    def _axial_exact_adj_col(self, y, iy, ix):
        return self._nudft_matrix(iy, ix).conj().T @ y / math.sqrt(self.grid.nz)

    def axial_forward(self, eta_hat: np.ndarray, cols=None) -> np.ndarray:
        """H(q, beta_j)/sqrt(nz) for every column, before the spectral phase."""
        gr = self.grid
        out = np.zeros(self.spec_shape, np.complex128)
        for iy in range(gr.ny):
            for ix in range(gr.nx):
                if cols is not None and (iy, ix) not in cols:
                    continue
                x = eta_hat[iy, ix]
                if self.mode == "exact":
                    out[iy, ix] = self._axial_exact_col(x, iy, ix)
                else:
                    out[iy, ix] = nufft_forward_column(x / math.sqrt(gr.nz), self.p[iy, ix],
                                                       self.interp, self._coef(iy, ix))
        return out * self.prop

    def axial_adjoint(self, y_hat: np.ndarray) -> np.ndarray:
        gr = self.grid
        out = np.zeros(self.image_shape, np.complex128)
        y_hat = y_hat * self.prop
        for iy in range(gr.ny):
            for ix in range(gr.nx):
                y = y_hat[iy, ix]
                if self.mode == "exact":
                    out[iy, ix] = self._axial_exact_adj_col(y, iy, ix)
                else:
                    out[iy, ix] = nufft_adjoint_column(y, self.p[iy, ix], self.interp,
                                                       self._coef(iy, ix)) / math.sqrt(gr.nz)
        return out

    # -- full operators -------------------------------------------------------
    def K_hat(self, eta: np.ndarray) -> np.ndarray:
        """Complex spectra diag(e^{j phi}) K eta, [ny, nx, nk]  [Eq. 13, 16]."""
        S = self.phase * self.axial_forward(lateral_fft(eta))
        return lateral_ifft(S)

    def forward(self, eta: np.ndarray) -> np.ndarray:
        """s = Re(K_hat eta)  [Eq. 5, 12]."""
        return self.K_hat(eta).real

    def adjoint(self, y: np.ndarray) -> np.ndarray:
        """A^H y = F^{-1}[ N'( conj(phase) F y ) ] for real y  [Eq. 17]."""
        R = lateral_fft(y.astype(np.complex128))
        return lateral_ifft(self.axial_adjoint(np.conj(self.phase) * R))


# ----------------------------------------------------------------------------
# Solver pieces  (§3, Alg. 1; §3.1)
# ----------------------------------------------------------------------------


def soft_threshold(u: np.ndarray, tau) -> np.ndarray:
    """T_tau(u) = u max(|u|-tau, 0) / (max(|u|-tau, 0) + tau), 0 where 0/0  [Eq. 14]."""
    m = np.maximum(np.abs(u) - tau, 0.0)
    den = m + tau
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(den > 0, u * m / np.where(den > 0, den, 1.0), 0.0)
    return r


def haar_forward(x: np.ndarray) -> np.ndarray:
    """Orthonormal Haar transform along the last axis (length 2^m, all levels).

    Level by level on the current approximation a (length n): a' = (a[0::2] +
    a[1::2])/sqrt 2, d = (a[0::2] - a[1::2])/sqrt 2; the output is
    [a_final, d_coarsest, ..., d_finest] (Mallat order)."""
    a = np.asarray(x, dtype=np.complex128)
    details = []
    while a.shape[-1] > 1:
        e, o = a[..., 0::2], a[..., 1::2]
        details.append((e - o) / math.sqrt(2))
        a = (e + o) / math.sqrt(2)
    return np.concatenate([a] + details[::-1], axis=-1)


def haar_inverse(c: np.ndarray) -> np.ndarray:
    """Inverse of haar_forward."""
    c = np.asarray(c, dtype=np.complex128)
    n = c.shape[-1]
    a = c[..., :1]
    pos = 1
    while pos < n:
        d = c[..., pos:2 * pos]
        out = np.empty(c.shape[:-1] + (2 * pos,), np.complex128)
        out[..., 0::2] = (a + d) / math.sqrt(2)
        out[..., 1::2] = (a - d) / math.sqrt(2)
        a = out
        pos *= 2
    return a


def haar_prox(u: np.ndarray, tau) -> np.ndarray:
    """prox of tau * (l1 norm of the Haar detail coefficients along depth):
    W^H T_tau(W u) with the approximation coefficient kept (W orthonormal)."""
    c = haar_forward(u)
    c[..., 1:] = soft_threshold(c[..., 1:], tau)
    return haar_inverse(c)


def tv_grad(x: np.ndarray):
    """Forward differences along x (axis -2) and z (axis -1), zero at the far
    edge: (dx, dz) with dx[..., i, :] = x[..., i+1, :] - x[..., i, :]."""
    dx = np.zeros_like(x)
    dz = np.zeros_like(x)
    dx[..., :-1, :] = x[..., 1:, :] - x[..., :-1, :]
    dz[..., :, :-1] = x[..., :, 1:] - x[..., :, :-1]
    return dx, dz


def tv_grad_adjoint(px: np.ndarray, pz: np.ndarray) -> np.ndarray:
    """Adjoint of tv_grad: <tv_grad(x), (px, pz)> = <x, tv_grad_adjoint(px, pz)>."""
    out = np.zeros_like(px)
    out[..., :-1, :] -= px[..., :-1, :]
    out[..., 1:, :] += px[..., :-1, :]
    out[..., :, :-1] -= pz[..., :, :-1]
    out[..., :, 1:] += pz[..., :, :-1]
    return out


def total_variation(x: np.ndarray) -> float:
    """Isotropic TV over (x, z) of every B-scan slice: sum sqrt(|dx|^2 + |dz|^2)."""
    dx, dz = tv_grad(x)
    return float(np.sum(np.sqrt(np.abs(dx) ** 2 + np.abs(dz) ** 2)))


class TVProx:
    """prox of tau TV (a total-variation prior, §3.1) by the fast gradient
    projection on the dual (Beck & Teboulle): z = u - tau grad^H p with
    |p| <= 1 per pixel; `iters` dual steps of size 1/(8 tau) per call, warm
    started from the previous call's p (the dual state of a FISTA solve)."""

    def __init__(self, iters: int = 20):
        self.iters = iters
        self.px = None
        self.pz = None

    def __call__(self, u: np.ndarray, tau: float) -> np.ndarray:
        if self.px is None or tau <= 0:
            self.px = np.zeros_like(u, dtype=np.complex128)
            self.pz = np.zeros_like(u, dtype=np.complex128)
        if tau <= 0:
            return np.array(u, dtype=np.complex128)
        px, pz = self.px, self.pz
        rx, rz = px.copy(), pz.copy()
        t = 1.0
        for _ in range(self.iters):
            w = u - tau * tv_grad_adjoint(rx, rz)
            gx, gz = tv_grad(w)
            qx = rx + gx / (8 * tau)
            qz = rz + gz / (8 * tau)
            m = np.maximum(1.0, np.sqrt(np.abs(qx) ** 2 + np.abs(qz) ** 2))
            nx_, nz_ = qx / m, qz / m
            t_next = (1 + math.sqrt(1 + 4 * t * t)) / 2
            beta = (t - 1) / t_next
            rx = nx_ + beta * (nx_ - px)
            rz = nz_ + beta * (nz_ - pz)
            px, pz, t = nx_, nz_, t_next
        self.px, self.pz = px, pz
        return u - tau * tv_grad_adjoint(px, pz)


def relative_residual(z, eta, g, eps=1e-12) -> float:
    """r_r = ||z - eta|| / (max(||g||, ||z - eta + g||) + eps)  [Eq. 15]."""
    d = z - eta
    return float(np.linalg.norm(d) / (max(np.linalg.norm(g), np.linalg.norm(d + g)) + eps))


def fista_t_sequence(n: int) -> np.ndarray:
    """t^1 = 1, t^{k+1} = (1 + sqrt(1 + 4 (t^k)^2)) / 2  [Alg. 1]."""
    t = np.empty(n + 1)
    t[0] = 1.0
    for i in range(n):
        t[i + 1] = (1 + math.sqrt(1 + 4 * t[i] ** 2)) / 2
    return t


def power_iteration(A: Callable, AH: Callable, v0: np.ndarray, iters: int = 50,
                    rtol: float = 1e-10) -> float:
    """L = ||A^H A|| by power iteration from the given unit start vector."""
    v = v0 / np.linalg.norm(v0)
    L_prev = 0.0
    L = 0.0
    for _ in range(iters):
        w = AH(A(v))
        L = float(np.linalg.norm(w))
        if L == 0:
            return 0.0
        v = w / L
        if abs(L - L_prev) <= rtol * L:
            break
        L_prev = L
    return L


def objective(A, eta, s_d, lam, w) -> float:
    """1/2 ||A eta - s_d||^2 + lambda w^T |eta|  [Eq. 12]."""
    r = A(eta) - s_d
    return float(0.5 * np.sum(r * r) + lam * np.sum(w * np.abs(eta)))


@dataclass
class FistaResult:
    eta: np.ndarray
    iterations: int
    rr: float
    lam: float
    L: float


def fista(A: Callable, AH: Callable, s_d: np.ndarray, lam: float, L: float, w=1.0,
          max_iter: int = 100, tol: float = 0.0, eps: float = 1e-12,
          addback: bool = False, shape=None, prox: Optional[Callable] = None) -> FistaResult:
    """MBIR full-range ISAM, Alg. 1, with step 1/L and threshold lambda w / L.

    Each iteration: g = (1/L) A^H(A eta - s_d); z = T(eta - g); stop when the
    relative residual (Eq. 15) drops below ``tol``; momentum update.  ``prox``
    (optional) replaces T for another convex prior (§3.1): z = prox(eta - g,
    lambda / L).
    """
    eta = np.zeros(shape, np.complex128)
    z_prev = np.zeros(shape, np.complex128)
    t = 1.0
    rr = float("inf")
    k = 0
    z = z_prev
    for k in range(1, max_iter + 1):
        g = AH(A(eta) - s_d) / L
        z = soft_threshold(eta - g, lam * w / L) if prox is None else prox(eta - g, lam / L)
        rr = relative_residual(z, eta, g, eps)
        if rr < tol:
            break
        t_next = (1 + math.sqrt(1 + 4 * t * t)) / 2
        eta = z + ((t - 1) / t_next) * (z - z_prev)
        z_prev = z
        t = t_next
    out = z
    if addback:
        out = z + AH(s_d - A(z)) / L
    return FistaResult(out, k, rr, lam, L)


def lambda_from_data(AH: Callable, s_d: np.ndarray, lambda_rel: float) -> float:
    """lambda = lambda_rel * ||A^H s_d||_inf."""
    return float(lambda_rel * np.abs(AH(s_d)).max())


# ----------------------------------------------------------------------------
# Brute force for tiny problems
# ----------------------------------------------------------------------------


def dense_real_matrix(op: IsamOracle) -> np.ndarray:
    """Real matrix M with s = M [Re eta; Im eta], built column by column."""
    n = int(np.prod(op.image_shape))
    m = int(np.prod(op.spec_shape))
    M = np.zeros((m, 2 * n))
    for i in range(n):
        e = np.zeros(n, np.complex128)
        e[i] = 1.0
        M[:, i] = op.forward(e.reshape(op.image_shape)).ravel()
        e[i] = 1j
        M[:, n + i] = op.forward(e.reshape(op.image_shape)).ravel()
    return M


class AxialModelOracle:
    """The 1-D dispersion-encoded model of each A-scan on its own (the model of
    the DEFR objective, Eq. 10, with our scaling): every lateral position is an
    independent nx = ny = 1 problem, s(x, k) = Re(e^{j phi(k)} N(eta(x, .))(k)),
    no lateral coupling and no focus term (2k + beta = 0 at q = 0)."""

    def __init__(self, g, mode: str = "nufft", J: int = 6):
        import dataclasses
        self.g = g
        self.col = IsamOracle(dataclasses.replace(g, nx=1, ny=1, dy=0.0), mode, J)
        nz = g.nz or g.nk
        self.image_shape = (g.ny, g.nx, nz)
        self.spec_shape = (g.ny, g.nx, g.nk)

    def forward(self, eta: np.ndarray) -> np.ndarray:
        out = np.zeros(self.spec_shape)
        for iy in range(self.g.ny):
            for ix in range(self.g.nx):
                out[iy, ix] = self.col.forward(eta[iy, ix][None, None, :])[0, 0]
        return out

    def adjoint(self, y: np.ndarray) -> np.ndarray:
        out = np.zeros(self.image_shape, np.complex128)
        for iy in range(self.g.ny):
            for ix in range(self.g.nx):
                out[iy, ix] = self.col.adjoint(y[iy, ix][None, None, :])[0, 0]
        return out


def dispersion_compensated_ifft(g, s_d: np.ndarray) -> np.ndarray:
    """F_vert^{-1}(s_d e^{-j phi}) per A-scan on the depth grid z_n  [Eq. 9].

    Direct sum (1/sqrt(nz)) sum_j s_d(k_j) e^{-j phi(k_j)} e^{-j 2 k_j z_n}.
    """
    gr = make_grid(g)
    phi = dispersion_phase(g, gr)
    E = np.exp(-1j * (np.outer(gr.z, 2 * gr.k)))          # [nz, nk]
    a = s_d * np.exp(-1j * phi)
    return np.einsum("zk,...k->...z", E, a) / math.sqrt(gr.nz)


# ----------------------------------------------------------------------------
# Calibration derivatives: theta = (a1, a2, a3, a4, z0)
# ----------------------------------------------------------------------------
# A depends on theta only through the spectral phase P(q, k) = e^{j phi(k)}
# e^{j (2k + beta) z0} [Eq. 7, Eq. 13 and the focus reading], so
#   dA/dtheta x = Re F^{-1}( j D_theta . P . N(F x) ),
#   D_{a_i} = (k - k0)^i,   D_{z0} = 2k + beta   (0 on evanescent samples).

PARAM_NAMES = ("a1", "a2", "a3", "a4", "z0")


def phase_log_derivatives(g, grid: Grid) -> np.ndarray:
    """D_theta(q, k), [5, ny, nx, nk]: dP/dtheta = j D_theta P  [Eq. 7, 13]."""
    beta, prop = stolt_beta(grid.q2[..., None], grid.k[None, None, :])
    shape = beta.shape
    D = np.zeros((5,) + shape)
    d = grid.k - grid.k0
    for i in range(4):
        D[i] = np.broadcast_to(d ** (i + 1), shape)
    D[4] = np.where(prop, 2 * grid.k[None, None, :] + beta, 0.0)
    return D


def forward_param_derivative(op: IsamOracle, x: np.ndarray, i: int) -> np.ndarray:
    """dA/dtheta_i x: the forward model with j D_i inserted after the phase."""
    D = phase_log_derivatives(op.g, op.grid)[i]
    S = 1j * D * op.phase * op.axial_forward(lateral_fft(x))
    return lateral_ifft(S).real


def param_grad(op: IsamOracle, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """<dA/dtheta x, y> for the five parameters (real inner product on spectra)."""
    return np.array([float(np.sum(forward_param_derivative(op, x, i) * y)) for i in range(5)])


def soft_threshold_vjp(u: np.ndarray, tau, zbar: np.ndarray) -> np.ndarray:
    """J^T zbar for z = T_tau(u) of Eq. 14, u complex (a map on R^2 per element).

    Where |u| > tau, T(u) = u - tau u/|u| and its (symmetric) Jacobian applied
    to v is v - tau (v/|u| - u Re(conj(u) v)/|u|^3); where |u| <= tau, T = 0.
    """
    a = np.abs(u)
    live = a > tau
    tau = np.broadcast_to(tau, u.shape)
    with np.errstate(invalid="ignore", divide="ignore"):
        inv = np.where(live, 1.0 / np.where(live, a, 1.0), 0.0)
        v = zbar - tau * (zbar * inv - u * np.real(np.conj(u) * zbar) * inv ** 3)
    return np.where(live, v, 0.0)


@dataclass
class UnrolledGrad:
    z: np.ndarray            # z^K
    theta_bar: np.ndarray    # d<z_bar, z^K>/dtheta, [5]
    s_bar: np.ndarray        # d<z_bar, z^K>/ds_d


def fista_unrolled_vjp(op: IsamOracle, s_d: np.ndarray, lam: float, L: float, K: int,
                       z_bar: np.ndarray, w=1.0) -> UnrolledGrad:
    """Gradient of <z_bar, z^K> (real inner product) through K FISTA iterations.

    Forward (Alg. 1 with step 1/L, threshold lambda w / L, t^1 = 1):
      eta^k = z^{k-1} + mu_{k-1} (z^{k-1} - z^{k-2}),  mu_{k-1} = (t^{k-1}-1)/t^k,
      u^k = eta^k - (1/L) A^H (A eta^k - s_d),  z^k = T(u^k),  z^0 = z^{-1} = 0.
    Reverse, k = K .. 1 (every iterate kept; lambda and L are constants):
      ubar = J_T(u^k)^T zbar^k,  etabar = ubar - (1/L) A^H A ubar,
      theta_bar -= (1/L) (<dA ubar, A eta^k - s_d> + <A ubar, dA eta^k>),
      s_bar += (1/L) A ubar,
      zbar^{k-1} += (1 + mu_{k-1}) etabar,  zbar^{k-2} -= mu_{k-1} etabar.
    """
    shape = op.image_shape
    zero = np.zeros(shape, np.complex128)
    tau = lam * w / L
    t = fista_t_sequence(K + 1)           # t[k-1] = t^k
    mu = np.zeros(K + 1)                  # mu[k] = (t^k - 1)/t^{k+1}, mu[0] = 0
    for k in range(1, K + 1):
        mu[k] = (t[k - 1] - 1) / t[k]
    z_prev2, z_prev = zero, zero
    etas, us = [None], [None]
    for k in range(1, K + 1):
        eta = z_prev + mu[k - 1] * (z_prev - z_prev2)
        u = eta - op.adjoint(op.forward(eta) - s_d) / L
        etas.append(eta)
        us.append(u)
        z_prev2, z_prev = z_prev, soft_threshold(u, tau)
    zK = z_prev
    zbar = [zero.copy() for _ in range(K + 1)]
    zbar[K] = z_bar.astype(np.complex128)
    theta_bar = np.zeros(5)
    s_bar = np.zeros(op.spec_shape)
    for k in range(K, 0, -1):
        ubar = soft_threshold_vjp(us[k], tau, zbar[k])
        Au = op.forward(ubar)
        etabar = ubar - op.adjoint(Au) / L
        r = op.forward(etas[k]) - s_d
        theta_bar -= (param_grad(op, ubar, r) + param_grad(op, etas[k], Au)) / L
        s_bar += Au / L
        if k - 1 >= 1:
            zbar[k - 1] += (1 + mu[k - 1]) * etabar
        if k - 2 >= 1:
            zbar[k - 2] -= mu[k - 1] * etabar
    return UnrolledGrad(zK, theta_bar, s_bar)

