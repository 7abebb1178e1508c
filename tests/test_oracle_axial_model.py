"""Pins of the oracle's 1-D per-A-scan model (Eq. 10) and Eq. 9.

Each A-scan of a B-scan or volume is checked against the numpy FFT route of
the dispersed DFT (forward) and against the direct dispersion-compensated
IFFT sum (adjoint, exact mode); the pair passes the dot-product test."""
import math

import numpy as np
import pytest

from oracle import isam_oracle as O
from paper_1905_06058_gb300 import inputs as I


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def numpy_forward(g, eta_col, gr):
    a = eta_col * np.exp(2j * g.k_min * gr.z)
    dft = np.fft.ifft(a) * gr.nz
    j = np.arange(gr.nk)
    S = dft[: gr.nk] * np.exp(-1j * math.pi * j) / math.sqrt(gr.nz)
    return (np.exp(1j * O.dispersion_phase(g, gr)) * S).real


@pytest.mark.parametrize("ny,nx,nk,nz", [(1, 6, 32, 32), (1, 4, 32, 64), (3, 2, 16, 16)])
@pytest.mark.parametrize("mode,tol", [("exact", 1e-12), ("nufft", 2e-5)])
def test_axial_model_columns(ny, nx, nk, nz, mode, tol):
    g = I.small_bscan(nx=nx, ny=ny, nk=nk, nz=nz, seed=3).geom
    op = O.AxialModelOracle(g, mode)
    gr = O.make_grid(g)
    eta = I.random_image(op.image_shape, 4)
    s = op.forward(eta)
    y = I.random_spectra(op.spec_shape, 5)
    a = op.adjoint(y)
    for iy in range(ny):
        for ix in range(nx):
            assert rel(s[iy, ix], numpy_forward(g, eta[iy, ix], gr)) < tol
            assert rel(a[iy, ix], O.dispersion_compensated_ifft(g, y[iy, ix])) < tol
    lhs = np.sum(s * y)
    rhs = np.real(np.vdot(eta, a))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(s) * np.linalg.norm(y)


def test_axial_model_ignores_focus_and_lateral_pitch():
    g = I.small_bscan(nx=4, nk=32, nz=32, seed=6).geom
    import dataclasses
    g2 = dataclasses.replace(g, z0=3 * g.z0 + 1e-4, dx=0.5 * g.dx)
    eta = I.random_image((1, 4, 32), 7)
    assert np.array_equal(O.AxialModelOracle(g, "exact").forward(eta),
                          O.AxialModelOracle(g2, "exact").forward(eta))
