"""Pins of the oracle's filter B(q, k) (Eq. 3; b of Eq. 16).

A real filter that depends on k only scales every spectral sample (Re and
the lateral transforms commute with a real per-k factor); a pure phase
e^{j psi(k)} with psi a polynomial in (k - k0) equals extra dispersion terms
(Eq. 7); B = 1 is the unfiltered model; the filtered pair passes the
dot-product test; the class table is symmetric in q by construction."""
import dataclasses

import numpy as np
import pytest

from oracle import isam_oracle as O
from paper_1905_06058_gb300 import inputs as I


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def geom(nx=8, ny=1, nk=32, nz=32, seed=3):
    return I.small_bscan(nx=nx, ny=ny, nk=nk, nz=nz, seed=seed).geom


def table_shape(g):
    return ((g.ny // 2 + 1) if g.ny > 1 else 1, g.nx // 2 + 1, g.nk)


@pytest.mark.parametrize("mode", ["exact", "nufft"])
def test_real_k_only_filter_scales_spectra(mode):
    g = geom()
    c = np.random.default_rng(1).uniform(0.2, 1.5, g.nk)
    tab = np.broadcast_to(c, table_shape(g)).astype(complex)
    eta = I.random_image((1, g.nx, g.nz), 2)
    s_f = O.IsamOracle(g, mode, filt=tab).forward(eta)
    s = O.IsamOracle(g, mode).forward(eta)
    assert rel(s_f, s * c) < 1e-13


@pytest.mark.parametrize("mode", ["exact", "nufft"])
def test_phase_filter_equals_extra_dispersion(mode):
    g = geom(nx=6, nk=32, nz=64)
    gr = O.make_grid(g)
    extra = (3e-5, -2e-10, 0.0, 0.0)
    d = gr.k - gr.k0
    psi = sum(a * d ** (i + 1) for i, a in enumerate(extra))
    tab = np.broadcast_to(np.exp(1j * psi), table_shape(g)).astype(complex)
    g2 = dataclasses.replace(g, disp=tuple(a + b for a, b in zip(g.disp, extra)))
    eta = I.random_image((1, g.nx, gr.nz), 3)
    y = I.random_spectra((1, g.nx, g.nk), 4)
    op_f, op2 = O.IsamOracle(g, mode, filt=tab), O.IsamOracle(g2, mode)
    assert rel(op_f.forward(eta), op2.forward(eta)) < 1e-12
    assert rel(op_f.adjoint(y), op2.adjoint(y)) < 1e-12


@pytest.mark.parametrize("ny,nx", [(1, 8), (4, 4)])
def test_filtered_pair_dot_product_and_unit_filter(ny, nx):
    g = geom(nx=nx, ny=ny, nk=16, nz=16)
    rng = np.random.default_rng(5)
    shp = table_shape(g)
    tab = rng.uniform(0.3, 1.2, shp) * np.exp(1j * rng.uniform(-1, 1, shp))
    op = O.IsamOracle(g, "exact", filt=tab)
    eta = I.random_image(op.image_shape, 6)
    y = I.random_spectra(op.spec_shape, 7)
    lhs = np.sum(op.forward(eta) * y)
    rhs = np.real(np.vdot(eta, op.adjoint(y)))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(op.forward(eta)) * np.linalg.norm(y)
    one = O.IsamOracle(g, "exact", filt=np.ones(shp, complex))
    assert np.array_equal(one.forward(eta), O.IsamOracle(g, "exact").forward(eta))
    B = O.expand_filter(g, tab)
    # column -q takes the same row as q
    assert np.array_equal(B[:, 1], B[:, nx - 1])
    if ny > 1:
        assert np.array_equal(B[1, 2], B[ny - 1, nx - 2])
