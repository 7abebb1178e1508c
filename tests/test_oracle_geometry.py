"""Pins of the oracle's geometric building blocks against what the paper and the
physics fix, independently of how the oracle writes them:

* the Stolt map of Eq. 3 (beta = -sqrt(4k^2 - q^2)): at q = 0 it is the 1-D
  OCT round trip beta = -2k; samples with |q| >= 2k are evanescent; the
  map lies on the circle beta^2 + q^2 = (2k)^2; d beta / dk <= -2 (the
  adjoint scatter's residue classes rely on it);
* the grid position of a sample in the K = 2 nz oversampled grid: at q = 0
  consecutive samples sit exactly two bins apart (dz = pi / (nz dk));
* the spectral phase: unit modulus on propagating samples, zero on
  evanescent ones, and at q = 0 the focus factor drops out (e^{j phi(k)}
  alone, §2);
* the dispersion polynomial of Eq. 7 at hand-evaluated points;
* the lateral transforms: unitary and mutually inverse.
"""
import math

import numpy as np
import pytest

from oracle import isam_oracle as O
from paper_1905_06058_gb300 import inputs as I


def test_stolt_map_round_trip_and_cutoff():
    k = np.linspace(4.6e6, 5.1e6, 257)
    beta, prop = O.stolt_beta(np.zeros_like(k), k)
    assert prop.all()
    np.testing.assert_allclose(beta, -2.0 * k, rtol=1e-15)
    # lateral frequencies below, at and above the cutoff 2k
    k0 = 5.0e6
    q = np.array([0.0, 1.0e6, 9.99e6, 2.0 * k0, 1.2e7])
    beta, prop = O.stolt_beta(q ** 2, np.full(q.shape, k0))
    assert prop.tolist() == [True, True, True, False, False]
    assert (beta[~prop] == 0).all() and (beta[prop] < 0).all()
    np.testing.assert_allclose(beta[prop] ** 2 + q[prop] ** 2, 4 * k0 ** 2, rtol=1e-12)


def test_stolt_map_slope_at_least_two():
    rng = np.random.default_rng(3)
    k = np.linspace(4.6e6, 5.1e6, 2001)
    for q in rng.uniform(0, 9.0e6, 8):
        beta, prop = O.stolt_beta(np.full(k.shape, q * q), k)
        assert prop.all()
        slope = np.diff(beta) / np.diff(k)
        assert (slope <= -2.0 + 1e-9).all()


def test_grid_positions_two_bins_per_sample_at_q0():
    wl = I.small_bscan(nx=8, nk=64, nz=64, seed=3)
    gr = O.make_grid(wl.geom)
    beta, _ = O.stolt_beta(np.zeros(gr.nk), gr.k)
    p = O.grid_position(beta, gr.dz, 2 * gr.nz)
    np.testing.assert_allclose(np.diff(p), 2.0, rtol=0, atol=1e-9)
    # and the first sample sits at 2 k_min / dk bins
    assert p[0] == pytest.approx(2 * gr.k[0] / gr.dk, rel=1e-12)


def test_spectral_phase_modulus_support_and_q0():
    wl = I.small_bscan(nx=32, nk=64, nz=64, seed=4, dx_scale=0.1)   # some evanescent columns
    g = wl.geom
    assert g.z0 != 0
    gr = O.make_grid(g)
    ph = O.spectral_phase(g, gr)
    _, prop = O.stolt_beta(gr.q2[..., None], gr.k[None, None, :])
    assert (~prop).any() and prop.any()
    np.testing.assert_allclose(np.abs(ph[prop]), 1.0, rtol=1e-14)
    assert (ph[~prop] == 0).all()
    # q = 0 (column 0 in FFT order): the focus phase e^{j (2k + beta) z0} is 1
    np.testing.assert_allclose(ph[0, 0], np.exp(1j * O.dispersion_phase(g, gr)), rtol=1e-13)


def test_dispersion_polynomial_hand_values():
    g = I.small_bscan(nx=8, nk=64, nz=64, seed=5).geom
    gr = O.make_grid(g)
    g.disp = (0.0, 1.0e-10, 0.0, 0.0)                # a2 only
    k0 = gr.k0
    gr.k = np.array([k0, k0 + 1.0e5, k0 - 2.0e5])
    np.testing.assert_allclose(O.dispersion_phase(g, gr), [0.0, 1.0, 4.0], atol=1e-12)
    g.disp = (2.0e-6, 0.0, 3.0e-16, 0.0)             # a1 (a delay) and a3
    np.testing.assert_allclose(O.dispersion_phase(g, gr),
                               [0.0, 0.2 + 0.3, -0.4 - 2.4], atol=1e-12)


def test_lateral_transforms_unitary_and_inverse():
    rng = np.random.default_rng(6)
    a = rng.standard_normal((4, 12, 5)) + 1j * rng.standard_normal((4, 12, 5))
    f = O.lateral_fft(a)
    assert np.linalg.norm(f) == pytest.approx(np.linalg.norm(a), rel=1e-13)
    np.testing.assert_allclose(O.lateral_ifft(f), a, atol=1e-13)
    # a single lateral frequency: the plane wave e^{j 2 pi m x / nx} maps to one bin
    x = np.arange(12)
    w = np.exp(2j * math.pi * 3 * x / 12)[None, :, None] * np.ones((1, 1, 2))
    F = O.lateral_fft(w)
    assert np.abs(F[0, 3]).min() == pytest.approx(math.sqrt(12), rel=1e-12)
    assert np.abs(np.delete(F[0], 3, axis=0)).max() < 1e-12
