"""Pins of the oracle's ISAM operator A and adjoint A^H (§2-§3, Eq. 3-17).

Each check ties the oracle to something other than itself: numpy's FFT at
q = 0 (where the Stolt map is the identity and A is the DEFR 1-D model,
Eq. 10, and A^H the dispersion-compensated IFFT, Eq. 9), the adjoint
identity, the mirror ambiguity at zero dispersion (Eq. 6), the focal-plane
property of ISAM (a scatterer in focus is not blurred laterally) and the
paraxial (Fresnel) limit of the Stolt map.
"""
import math

import numpy as np
import pytest

from oracle import isam_oracle as O
from paper_1905_06058_gb300 import inputs as I


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def small_geom(nx=8, ny=1, nk=16, nz=0, disp=True, z0_frac=0.3, seed=1, dx_scale=1.0):
    return I.small_bscan(nx=nx, ny=ny, nk=nk, nz=nz, dispersion=disp, focus_frac=z0_frac,
                         seed=seed, dx_scale=dx_scale).geom


@pytest.mark.parametrize("nz_factor", [1, 2])
@pytest.mark.parametrize("mode,tol", [("exact", 1e-12), ("nufft", 2e-5)])
def test_q0_forward_is_dispersed_dft(nz_factor, mode, tol):
    """nx = 1: A eta = Re(e^{j phi} (1/sqrt nz) sum_n eta_n e^{j 2 k z_n})  (Eq. 10)."""
    g = small_geom(nx=1, nk=32, nz=32 * nz_factor)
    op = O.IsamOracle(g, mode)
    gr = op.grid
    eta = I.random_image((1, 1, gr.nz), 5)
    s = op.forward(eta)[0, 0]
    # numpy route: 2 k_j z_n = 2 k_min z_n + 2 pi j (n - nz/2) / nz
    a = eta[0, 0] * np.exp(2j * g.k_min * gr.z)
    dft = np.fft.ifft(a) * gr.nz                         # sum_n a_n e^{+j 2 pi j n / nz}
    j = np.arange(gr.nk)
    S = dft[: gr.nk] * np.exp(-1j * math.pi * j) / math.sqrt(gr.nz)
    phi = O.dispersion_phase(g, gr)
    ref = (np.exp(1j * phi) * S).real
    assert rel(s, ref) < tol


@pytest.mark.parametrize("mode,tol", [("exact", 1e-12), ("nufft", 2e-5)])
def test_q0_adjoint_is_dispersion_compensated_ifft(mode, tol):
    """nx = 1: A^H y = F^{-1}(y e^{-j phi}) on the depth grid  (Eq. 9)."""
    g = small_geom(nx=1, nk=32)
    op = O.IsamOracle(g, mode)
    gr = op.grid
    y = I.random_spectra((1, 1, gr.nk), 9)
    got = op.adjoint(y)[0, 0]
    phi = O.dispersion_phase(g, gr)
    b = y[0, 0] * np.exp(-1j * phi) * np.exp(1j * math.pi * np.arange(gr.nk))
    ref = np.fft.fft(b, gr.nz) * np.exp(-2j * g.k_min * gr.z) / math.sqrt(gr.nz)
    assert rel(got, ref) < tol
    # and the oracle's direct Eq. 9 routine agrees with the same numpy route
    assert rel(O.dispersion_compensated_ifft(g, y[0, 0]), ref) < 1e-12


@pytest.mark.parametrize("mode", ["exact", "nufft"])
@pytest.mark.parametrize("ny,nx,nk,nz", [(1, 8, 16, 16), (1, 6, 12, 24), (4, 4, 8, 8)])
def test_adjoint_dot_product(mode, ny, nx, nk, nz):
    """<A eta, y>_R = Re <eta, A^H y> to 1e-12 (real inner product)."""
    g = small_geom(nx=nx, ny=ny, nk=nk, nz=nz)
    op = O.IsamOracle(g, mode)
    eta = I.random_image(op.image_shape, 11)
    y = I.random_spectra(op.spec_shape, 12)
    lhs = np.sum(op.forward(eta) * y)
    rhs = np.real(np.vdot(eta, op.adjoint(y)))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(eta) * np.linalg.norm(y) * 10


@pytest.mark.parametrize("J,tol", [(6, 1e-5), (8, 1e-7)])
def test_nufft_mode_tracks_exact_mode(J, tol):
    g = small_geom(nx=16, nk=64, nz=64)
    ex = O.IsamOracle(g, "exact")
    nu = O.IsamOracle(g, "nufft", J=J)
    eta = I.random_image(ex.image_shape, 2)
    y = I.random_spectra(ex.spec_shape, 3)
    assert rel(nu.forward(eta), ex.forward(eta)) < tol
    assert rel(nu.adjoint(y), ex.adjoint(y)) < tol


def test_mirror_ambiguity_without_dispersion():
    """a = 0, z0 = 0: A eta = A conj(eta(x, -z)) (Eq. 6); a != 0 breaks it (Eq. 8)."""
    g = small_geom(nx=8, nk=32, disp=False, z0_frac=0.5)
    assert g.z0 == 0.0
    op = O.IsamOracle(g, "exact")
    eta = I.random_image(op.image_shape, 4)
    eta[..., 0] = 0                                       # z_0 has no mirror on the grid
    nz = op.grid.nz
    mirror = np.conj(eta[..., (nz - np.arange(nz)) % nz])
    assert rel(op.forward(mirror), op.forward(eta)) < 1e-12
    g2 = small_geom(nx=8, nk=32, disp=True, z0_frac=0.5)
    op2 = O.IsamOracle(g2, "exact")
    assert rel(op2.forward(mirror), op2.forward(eta)) > 0.2


def test_focal_plane_scatterer_is_not_blurred():
    """A point at the focus depth only reaches its own A-scan (ISAM premise, §1-2);
    a point away from focus spreads over neighbouring A-scans."""
    g = small_geom(nx=16, nk=32, disp=True)
    gr = O.make_grid(g)
    n0 = 9
    g.z0 = float(gr.z[n0])                               # focus on a grid row
    op = O.IsamOracle(g, "exact")
    eta = np.zeros(op.image_shape, complex)
    eta[0, 5, n0] = 0.7 * np.exp(0.4j)
    s = op.forward(eta)[0]
    off = np.delete(s, 5, axis=0)
    assert np.abs(off).max() < 1e-12 * np.abs(s).max()
    # the lone A-scan is the dispersed carrier of a reflector at z0 (Eq. 8)
    phi = O.dispersion_phase(g, gr)
    ref = (0.7 * np.exp(0.4j) * np.exp(1j * (phi + 2 * gr.k * g.z0))).real / math.sqrt(gr.nz)
    np.testing.assert_allclose(s[5], ref, atol=1e-12)
    eta2 = np.zeros_like(eta)
    eta2[0, 5, n0 + 12] = 1.0
    s2 = op.forward(eta2)[0]
    assert np.abs(np.delete(s2, 5, axis=0)).max() > 1e-3 * np.abs(s2).max()


def test_defocus_matches_fresnel_limit():
    """For q << 2k the Stolt map gives the paraxial defocus phase:
    S(q,k)/S(0,k) -> exp(-j q^2 (z_s - z0) / (4k)) exp(-j q x_s)."""
    g = small_geom(nx=64, nk=32, disp=True, dx_scale=40.0)   # coarse pitch: small q
    op = O.IsamOracle(g, "exact")
    gr = op.grid
    xs, ns = 3, 20
    eta = np.zeros(op.image_shape, complex)
    eta[0, xs, ns] = 1.0
    S = O.lateral_fft(op.K_hat(eta))[0]                  # back to (q, k)
    qx = 2 * math.pi * np.fft.fftfreq(g.nx, d=g.dx)
    dz_s = gr.z[ns] - g.z0
    ratio = S / S[0][None, :]
    fres = np.exp(-1j * np.outer(qx ** 2, 1 / (4 * gr.k)) * dz_s) * \
        np.exp(-1j * np.outer(qx * xs * g.dx, np.ones(gr.nk)))
    # paraxial error ~ q^4 |dz| / (64 k^3)
    bound = (qx.max() ** 4 * abs(dz_s) / (64 * gr.k.min() ** 3)) * 2 + 1e-12
    assert np.abs(ratio - fres).max() < bound
    assert bound < 0.05                                  # the test is not vacuous


def test_lipschitz_is_one_at_q0_and_matches_svd():
    # nx = 1, nz = nk and nz = 2 nk: rows of K are orthonormal, so ||A||^2 = 1
    for nzf in (1, 2):
        g = small_geom(nx=1, nk=16, nz=16 * nzf)
        op = O.IsamOracle(g, "exact")
        v0 = I.start_vector(op.image_shape, 1)
        L = O.power_iteration(op.forward, op.adjoint, v0, iters=500, rtol=1e-13)
        assert L == pytest.approx(1.0, abs=1e-9)
    g = small_geom(nx=4, nk=8, nz=8)
    op = O.IsamOracle(g, "exact")
    M = O.dense_real_matrix(op)
    smax = np.linalg.svd(M, compute_uv=False)[0]
    v0 = I.start_vector(op.image_shape, 2)
    L = O.power_iteration(op.forward, op.adjoint, v0, iters=2000, rtol=1e-14)
    assert L == pytest.approx(smax ** 2, rel=1e-8)


def test_dense_matrix_reproduces_forward():
    g = small_geom(nx=4, nk=8, nz=8)
    op = O.IsamOracle(g, "exact")
    M = O.dense_real_matrix(op)
    eta = I.random_image(op.image_shape, 8)
    v = np.concatenate([eta.real.ravel(), eta.imag.ravel()])
    np.testing.assert_allclose(M @ v, op.forward(eta).ravel(), atol=1e-12)
    # and its transpose is the adjoint under the real inner product
    y = I.random_spectra(op.spec_shape, 9)
    ah = op.adjoint(y).ravel()
    np.testing.assert_allclose(M.T @ y.ravel(), np.concatenate([ah.real, ah.imag]), atol=1e-12)


def test_evanescent_columns_are_dropped():
    g = small_geom(nx=16, nk=16, dx_scale=0.05)           # pitch far below lambda/2
    op = O.IsamOracle(g, "nufft")
    assert (~op.prop).any() and op.prop.any()
    eta_hat = np.zeros(op.image_shape, complex)
    iy, ix = np.argwhere(~op.prop.any(axis=-1))[0]
    eta_hat[iy, ix] = 1.0
    S = op.axial_forward(eta_hat)
    assert np.abs(S).max() == 0.0
    eta = I.random_image(op.image_shape, 1)
    y = I.random_spectra(op.spec_shape, 2)
    lhs = np.sum(op.forward(eta) * y)
    rhs = np.real(np.vdot(eta, op.adjoint(y)))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_grid_conventions():
    g = small_geom(nx=8, nk=16, nz=32)
    gr = O.make_grid(g)
    assert gr.k[0] == g.k_min and gr.k[-1] == pytest.approx(g.k_max, rel=1e-15)
    assert gr.z[gr.nz // 2] == 0.0
    # full complex depth range pi / dk regardless of nz
    assert gr.nz * gr.dz == pytest.approx(math.pi / gr.dk, rel=1e-14)
