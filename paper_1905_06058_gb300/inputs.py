"""Seeded synthetic inputs for full-range dispersion-encoded ISAM.

This module only draws the problem: the acquisition geometry (spectral band,
lateral pitch, focus, dispersion coefficients), the complex susceptibility
``eta`` of a synthetic specimen, the measurement noise and the spectrometer's
count model.  It contains none of the reconstruction arithmetic (no lateral
FFT, Stolt map, NUFFT or solver): the interference term that the count model
and the noise act on is always passed in by the caller, who computes it with
whichever forward operator it trusts.

The specimen families follow the paper's workloads: isolated complex point
scatterers at both positive and negative optical delay (§1, sparsity
premise), layered tissue-like interfaces with sparse complex speckle (§4.1
samples) and SD-OCT spectra of 2048 samples per A-scan with background
subtraction by the mean over A-scans (§4.1).

Every draw is seeded; ``SEED_BASE + config_id`` seeds the named workloads.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

SEED_BASE = 1905_06058


@dataclasses.dataclass
class Geometry:
    """Acquisition parameters, as the paper states the problem (§2, §4.1).

    Units: wavenumbers in rad/m, lengths in m, dispersion coefficient a_i in
    rad*m^i about k0 = (k_min + k_max)/2 (Eq. 7).  ``nz`` is the number of
    depth samples of the reconstructed full-range image; 0 means ``nk``.
    """

    nx: int
    ny: int
    nk: int
    nz: int
    k_min: float
    k_max: float
    dx: float
    dy: float
    na: float
    z0: float
    disp: tuple = (0.0, 0.0, 0.0, 0.0)

    def __post_init__(self):
        if self.nz == 0:
            self.nz = self.nk
        self.disp = tuple(float(a) for a in self.disp) + (0.0,) * (4 - len(self.disp))

    @property
    def n_image(self) -> int:
        return self.ny * self.nx * self.nz

    @property
    def n_spec(self) -> int:
        return self.ny * self.nx * self.nk

    def as_dict(self) -> dict:
        return dataclasses.asdict(self)


@dataclasses.dataclass
class Workload:
    name: str
    geom: Geometry
    eta: np.ndarray            # complex [ny][nx][nz], ground truth
    seed: int
    snr_db: Optional[float]    # additive Gaussian noise level on the spectra
    lambda_rel: float          # lambda = lambda_rel * ||A^H s_d||_inf
    iters: int                 # FISTA iterations of the stated workload
    counts: bool = False       # 12-bit detector model + background subtraction


# ----------------------------------------------------------------------------
# Geometry helpers (physical set-up, not the operator)
# ----------------------------------------------------------------------------

def band_from_wavelength(lambda0: float, bandwidth: float) -> tuple[float, float]:
    """Linear-in-k band covering lambda0 +- bandwidth/2."""
    return 2 * math.pi / (lambda0 + bandwidth / 2), 2 * math.pi / (lambda0 - bandwidth / 2)


def lateral_pitch(lambda0: float, na: float) -> float:
    """Nyquist-like A-scan pitch: half the Gaussian waist w0 = lambda0/(pi NA)."""
    return 0.5 * lambda0 / (math.pi * na)


def depth_range(k_min: float, k_max: float, nk: int) -> float:
    """Full complex depth range pi/dk of spectra sampled at nk points."""
    return math.pi / ((k_max - k_min) / (nk - 1))


def draw_dispersion(rng: np.random.Generator, k_min: float, k_max: float) -> tuple:
    """Quadratic + cubic dispersion (Eq. 7, N_p = 3, a1 = 0).

    Magnitudes are drawn in radians at the band edge: a2*(B/2)^2 in U[10, 30]
    and a3*(B/2)^3 in U[3, 10], random signs (B = k_max - k_min).
    """
    half = 0.5 * (k_max - k_min)
    a2 = rng.choice([-1.0, 1.0]) * rng.uniform(10.0, 30.0) / half ** 2
    a3 = rng.choice([-1.0, 1.0]) * rng.uniform(3.0, 10.0) / half ** 3
    return (0.0, a2, a3, 0.0)


# ----------------------------------------------------------------------------
# Specimens
# ----------------------------------------------------------------------------

def point_scatterers(rng, shape, count, amp=(0.2, 1.0), exclude_row0=False, min_sep=0):
    """Complex point scatterers on grid pixels, uniform over all x(,y) and +-z.

    |a| ~ U[amp], arg(a) ~ U[0, 2pi).  ``min_sep`` keeps scatterers at least
    that many pixels apart (Chebyshev distance) for isolation tests.
    """
    eta = np.zeros(shape, np.complex128)
    ny, nx, nz = shape
    placed = []
    lo_z = 1 if exclude_row0 else 0
    tries = 0
    while len(placed) < count:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place isolated scatterers")
        p = (int(rng.integers(ny)), int(rng.integers(nx)), int(rng.integers(lo_z, nz)))
        if min_sep and any(max(abs(p[0] - q[0]), abs(p[1] - q[1]), abs(p[2] - q[2])) < min_sep
                           for q in placed):
            continue
        if eta[p] != 0:
            continue
        placed.append(p)
        eta[p] = rng.uniform(*amp) * np.exp(2j * math.pi * rng.uniform())
    return eta


def layered_specimen(rng, shape, n_layers, speckle_frac, n_points, dtype=np.complex128):
    """Tissue-like specimen: smooth random interfaces, sparse speckle, points.

    Interfaces are depth profiles z(x, y) made of a few random low spatial
    frequencies, spread over both delay halves; each pixel on an interface
    has amplitude U[0.3, 1] times a random phase.  Speckle is complex
    Gaussian (sigma 0.15) on ``speckle_frac`` of all pixels.
    """
    ny, nx, nz = shape
    eta = np.zeros(shape, dtype)
    yy, xx = np.meshgrid(np.arange(ny) / max(ny, 1), np.arange(nx) / nx, indexing="ij")
    for _ in range(n_layers):
        centre = rng.uniform(0.1, 0.9) * nz
        prof = np.full((ny, nx), centre)
        for _h in range(3):
            fx, fy = rng.integers(1, 4), (rng.integers(1, 4) if ny > 1 else 0)
            prof += rng.uniform(0.01, 0.04) * nz * np.sin(
                2 * math.pi * (fx * xx + fy * yy) + rng.uniform(0, 2 * math.pi))
        rows = np.clip(np.rint(prof).astype(np.int64), 0, nz - 1)
        amp = rng.uniform(0.3, 1.0, (ny, nx)) * np.exp(2j * math.pi * rng.uniform(size=(ny, nx)))
        iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        eta[iy, ix, rows] += amp.astype(dtype)
    n_spk = int(round(speckle_frac * eta.size))
    flat = rng.choice(eta.size, size=n_spk, replace=False)
    spk = 0.15 * (rng.standard_normal(n_spk) + 1j * rng.standard_normal(n_spk)) / math.sqrt(2)
    eta.reshape(-1)[flat] += spk.astype(dtype)
    flat = rng.choice(eta.size, size=n_points, replace=False)
    pts = rng.uniform(0.2, 1.0, n_points) * np.exp(2j * math.pi * rng.uniform(size=n_points))
    eta.reshape(-1)[flat] += pts.astype(dtype)
    return eta


# ----------------------------------------------------------------------------
# Measurement model pieces that act on a given interference term
# ----------------------------------------------------------------------------

def add_noise(s_clean: np.ndarray, snr_db: float, rng: np.random.Generator) -> np.ndarray:
    """Additive white Gaussian noise at SNR = 10 log10(|s|^2 / |noise|^2)."""
    noise = rng.standard_normal(s_clean.shape)
    scale = np.linalg.norm(s_clean) / (np.linalg.norm(noise) * 10 ** (snr_db / 20))
    return s_clean + scale * noise


def detector_counts(interference: np.ndarray, k: np.ndarray, rng: np.random.Generator,
                    full_scale: int = 4095) -> np.ndarray:
    """12-bit spectrometer model followed by background subtraction (§4.1).

    counts = round(DC(k) + g * interference + shot-like noise), clipped to
    [0, 4095], as float32; then the background (mean over A-scans at each k)
    is subtracted.  DC(k) is a Gaussian spectral envelope peaking at ~55% of
    full scale and g puts the interference peak at ~35% of full scale.
    """
    kc = 0.5 * (k[0] + k[-1])
    width = 0.45 * (k[-1] - k[0])
    env = 0.55 * full_scale * np.exp(-((k - kc) / width) ** 2)
    g = 0.35 * full_scale / max(np.abs(interference).max(), 1e-30)
    raw = env + g * interference + rng.standard_normal(interference.shape) * 2.0
    counts = np.clip(np.rint(raw), 0, full_scale).astype(np.float32)
    lat_axes = tuple(range(counts.ndim - 1))
    return (counts - counts.mean(axis=lat_axes, keepdims=True)).astype(np.float32)


def start_vector(shape, seed: int) -> np.ndarray:
    """Seeded complex start vector for the power iteration (unit norm)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return v / np.linalg.norm(v)


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

LAMBDA0 = 1300e-9
BANDWIDTH = 100e-9


def _geometry(nx, ny, nk, nz, na, focus_frac, rng, lambda0=LAMBDA0, bandwidth=BANDWIDTH):
    k_min, k_max = band_from_wavelength(lambda0, bandwidth)
    dx = lateral_pitch(lambda0, na)
    rng_z = depth_range(k_min, k_max, nk)
    z0 = (focus_frac - 0.5) * rng_z       # focus measured from the top of the image
    return Geometry(nx=nx, ny=ny, nk=nk, nz=nz, k_min=k_min, k_max=k_max, dx=dx,
                    dy=dx if ny > 1 else 0.0, na=na, z0=z0,
                    disp=draw_dispersion(rng, k_min, k_max))


def config1() -> Workload:
    """128 x 256 spectra -> 128 x 512 full-range image, 40 point scatterers, FP64."""
    seed = SEED_BASE + 1
    rng = np.random.default_rng(seed)
    g = _geometry(128, 1, 256, 512, 0.1, 0.3, rng)
    eta = point_scatterers(rng, (1, 128, 512), 40)
    return Workload("bscan_128x256_to_128x512_fp64", g, eta, seed, 30.0, 0.01, 100)


def config2(dtype=np.complex128) -> Workload:
    """1024 A-scans x 2048 spectral samples, layered specimen, 12-bit counts."""
    seed = SEED_BASE + 2
    rng = np.random.default_rng(seed)
    g = _geometry(1024, 1, 2048, 2048, 0.15, 0.3, rng)
    eta = layered_specimen(rng, (1, 1024, 2048), 6, 0.02, 200, dtype)
    return Workload("bscan_1024x2048_fp32", g, eta, seed, None, 0.01, 200, counts=True)


def config3(dtype=np.complex64, nx=256, nk=2048, n_points=5000) -> Workload:
    """256 x 256 x 2048 volume, 3 curved layers, 1% speckle, 25 dB."""
    seed = SEED_BASE + 3
    rng = np.random.default_rng(seed)
    g = _geometry(nx, nx, nk, nk, 0.15, 0.3, rng)
    eta = layered_specimen(rng, (nx, nx, nk), 3, 0.01, n_points, dtype)
    return Workload(f"volume_{nx}x{nx}x{nk}_fp32", g, eta, seed, 25.0, 0.02, 150)


@dataclasses.dataclass
class CalibWorkload:
    """B-scans of one geometry made with a hidden dispersion and focal depth."""

    name: str
    geom: Geometry           # the hidden truth: geom.disp, geom.z0
    etas: list               # specimens, [1, nx, nz] each
    start: np.ndarray        # theta = (a1..a4, z0) where the fit starts
    snr_db: float
    lambda_rel: float
    K: int
    every: int


def config5(n_bscans: int = 16, nx: int = 512, nk: int = 2048) -> CalibWorkload:
    """16 B-scans of 512 x 2048 with hidden (a2, a3, z0); the fit starts with
    a2 off by 0.6 rad and a3 by -0.4 rad at the band edge and z0 off by 1% of
    the depth range.  K = 20 unrolled iterations, checkpoints every 5."""
    seed = SEED_BASE + 5
    rng = np.random.default_rng(seed)
    g = _geometry(nx, 1, nk, nk, 0.1, 0.3, rng)
    etas = [layered_specimen(np.random.default_rng(seed + 10 + b), (1, nx, nk), 3, 0.01, 100,
                             np.complex64) for b in range(n_bscans)]
    half = 0.5 * (g.k_max - g.k_min)
    start = np.array(list(g.disp) + [g.z0], dtype=np.float64)
    start[1] += 0.6 / half ** 2
    start[2] -= 0.4 / half ** 3
    start[4] += 0.01 * depth_range(g.k_min, g.k_max, nk)
    return CalibWorkload(f"calib_{n_bscans}x{nx}x{nk}", g, etas, start, 30.0, 0.01, 20, 5)


@dataclasses.dataclass
class BatchEntry:
    """One B-scan of an uneven batch: its geometry and how its specimen is drawn."""

    geom: Geometry
    seed: int
    sparsity: float          # fraction of speckle pixels
    lambda_rel: float


def config4(n: int = 96) -> list:
    """96 B-scans of uneven size for one batched launch: Nx from {256, 384,
    512, 768, 1024}, Nk = nz from {1024, 2048}, NA U[0.08, 0.2], focus at
    U[0.2, 0.8] of the range, own dispersion (as draw_dispersion), speckle
    sparsity U[1%, 3%] plus 2 interfaces and 50 points, lambda_rel
    U[0.005, 0.02], 30 dB noise; 200 iterations each."""
    seed = SEED_BASE + 4
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nx = int(rng.choice([256, 384, 512, 768, 1024]))
        nk = int(rng.choice([1024, 2048]))
        g = _geometry(nx, 1, nk, nk, float(rng.uniform(0.08, 0.2)), float(rng.uniform(0.2, 0.8)),
                      rng)
        out.append(BatchEntry(g, seed + 100 + i, float(rng.uniform(0.01, 0.03)),
                              float(rng.uniform(0.005, 0.02))))
    return out


def batch_specimen(e: BatchEntry, dtype=np.complex64) -> np.ndarray:
    rng = np.random.default_rng(e.seed)
    return layered_specimen(rng, (1, e.geom.nx, e.geom.nz), 2, e.sparsity, 50, dtype)


def small_bscan(nx=32, nk=64, nz=0, na=0.1, focus_frac=0.3, n_points=6, seed=7,
                dispersion=True, dx_scale=1.0, min_sep=0, ny=1) -> Workload:
    """Small seeded case for parity tests (several tiles and a ragged tail)."""
    rng = np.random.default_rng(SEED_BASE + 1000 + seed)
    g = _geometry(nx, ny, nk, nz or nk, na, focus_frac, rng)
    g.dx *= dx_scale
    if ny > 1:
        g.dy = g.dx
    if not dispersion:
        g.disp = (0.0, 0.0, 0.0, 0.0)
    eta = point_scatterers(rng, (ny, nx, g.nz), n_points, min_sep=min_sep)
    return Workload(f"small_{ny}x{nx}x{nk}", g, eta, SEED_BASE + 1000 + seed, 30.0, 0.01, 50)


def random_image(shape, seed) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def random_spectra(shape, seed) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape)


def depth_weights(nz: int, lo: float = 0.5, hi: float = 1.0) -> np.ndarray:
    """MBIR+ weights, linear in image row from ``lo`` (top) to ``hi`` (§3.1)."""
    return np.linspace(lo, hi, nz)
