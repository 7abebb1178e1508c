"""Pins of the oracle's calibration derivatives (theta = a1..a4, z0).

Every derivative is checked against central finite differences of the
oracle's own forward model or FISTA (which use none of the derivative
formulas), and against special cases the model fixes: the focal-depth
derivative vanishes on the q = 0 column (2k + beta = 0 there), and the
unrolled iterate equals the oracle's FISTA."""
import dataclasses

import numpy as np
import pytest

from oracle import isam_oracle as O
from paper_1905_06058_gb300 import inputs as I


def geom(nx=8, nk=32, nz=32, seed=3, ny=1):
    return I.small_bscan(nx=nx, nk=nk, nz=nz, seed=seed, ny=ny).geom


def perturbed(g, i, h):
    if i < 4:
        d = list(g.disp) + [0.0] * (4 - len(g.disp))
        d[i] += h
        return dataclasses.replace(g, disp=tuple(d))
    return dataclasses.replace(g, z0=g.z0 + h)


def steps(g):
    """Finite-difference steps: a phase change of ~1e-5 rad at the band edge."""
    gr = O.make_grid(g)
    dmax = np.abs(gr.k - gr.k0).max()
    return [1e-5 / dmax ** (i + 1) for i in range(4)] + [1e-5 / (2 * gr.k.max())]


@pytest.mark.parametrize("mode", ["exact", "nufft"])
@pytest.mark.parametrize("ny", [1, 2])
def test_param_grad_matches_central_differences(mode, ny):
    g = geom(ny=ny, nx=8 if ny == 1 else 4, nk=32, nz=32)
    op = O.IsamOracle(g, mode)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(op.image_shape) + 1j * rng.standard_normal(op.image_shape)
    y = rng.standard_normal(op.spec_shape)
    grad = O.param_grad(op, x, y)
    for i, h in enumerate(steps(g)):
        fp = np.sum(O.IsamOracle(perturbed(g, i, h), mode).forward(x) * y)
        fm = np.sum(O.IsamOracle(perturbed(g, i, -h), mode).forward(x) * y)
        fd = (fp - fm) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(grad).max()), O.PARAM_NAMES[i]


def test_focus_derivative_vanishes_on_q0_column():
    """At q = 0, beta = -2k: the focus phase is 1 for every z0 (nx = 1)."""
    g = geom(nx=1, nk=32, nz=64)
    op = O.IsamOracle(g, "exact")
    rng = np.random.default_rng(2)
    x = rng.standard_normal(op.image_shape) + 1j * rng.standard_normal(op.image_shape)
    y = rng.standard_normal(op.spec_shape)
    grad = O.param_grad(op, x, y)
    assert grad[4] == 0.0
    assert np.all(np.abs(grad[:4]) > 0)


def test_phase_log_derivatives_closed_form():
    g = geom(nx=4, nk=16, nz=16)
    gr = O.make_grid(g)
    D = O.phase_log_derivatives(g, gr)
    assert np.array_equal(D[1, 0, 2], (gr.k - gr.k0) ** 2)
    q2 = gr.q2[0, 1]
    assert np.allclose(D[4, 0, 1], q2 / (2 * gr.k + np.sqrt(4 * gr.k ** 2 - q2)), rtol=1e-12)
    assert np.all(D[4, 0, 0] == 0)


def test_soft_threshold_vjp_matches_finite_differences():
    rng = np.random.default_rng(4)
    n = 200
    u = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 2
    tau = rng.uniform(0.1, 1.5, n)
    zbar = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    v = O.soft_threshold_vjp(u, tau, zbar)
    h = 1e-6
    for part in (1.0, 1j):
        fd = (np.real(np.conj(zbar) * (O.soft_threshold(u + h * part, tau) -
                                        O.soft_threshold(u - h * part, tau)))) / (2 * h)
        got = np.real(np.conj(v) * part)
        keep = np.abs(np.abs(u) - tau) > 1e-3          # away from the kink
        assert np.allclose(got[keep], fd[keep], rtol=1e-6, atol=1e-8)
    assert np.all(v[np.abs(u) <= tau] == 0)


def _unrolled_problem(seed=5, K=8):
    g = geom(nx=8, nk=32, nz=32, seed=seed)
    op = O.IsamOracle(g, "exact")
    wl = I.small_bscan(nx=8, nk=32, nz=32, seed=seed)
    s = I.add_noise(op.forward(wl.eta), 30.0, np.random.default_rng(seed))
    L = O.power_iteration(op.forward, op.adjoint, I.start_vector(op.image_shape, seed), 300, 1e-13)
    lam = O.lambda_from_data(op.adjoint, s, 0.05)
    rng = np.random.default_rng(seed + 1)
    zbar = rng.standard_normal(op.image_shape) + 1j * rng.standard_normal(op.image_shape)
    return g, op, s, L, lam, zbar, K


def test_unrolled_iterate_equals_fista():
    g, op, s, L, lam, zbar, K = _unrolled_problem()
    res = O.fista_unrolled_vjp(op, s, lam, L, K, zbar)
    ref = O.fista(op.forward, op.adjoint, s, lam, L, max_iter=K, shape=op.image_shape)
    assert np.allclose(res.z, ref.eta, rtol=0, atol=1e-14 * np.abs(ref.eta).max())


def test_unrolled_theta_grad_matches_central_differences():
    g, op, s, L, lam, zbar, K = _unrolled_problem()
    w = I.depth_weights(op.grid.nz)[None, None, :]
    res = O.fista_unrolled_vjp(op, s, lam, L, K, zbar, w=w)

    def J(gg):
        o = O.IsamOracle(gg, "exact")
        z = O.fista(o.forward, o.adjoint, s, lam, L, w=w, max_iter=K, shape=o.image_shape).eta
        return float(np.real(np.vdot(zbar, z)))

    for i, h in enumerate(steps(g)):
        fd = (J(perturbed(g, i, h)) - J(perturbed(g, i, -h))) / (2 * h)
        assert res.theta_bar[i] == pytest.approx(fd, rel=1e-5), O.PARAM_NAMES[i]


def test_unrolled_data_grad_matches_central_differences():
    g, op, s, L, lam, zbar, K = _unrolled_problem(seed=6)
    res = O.fista_unrolled_vjp(op, s, lam, L, K, zbar)
    d = np.random.default_rng(9).standard_normal(op.spec_shape)
    h = 1e-6 * np.abs(s).max()

    def J(ss):
        z = O.fista(op.forward, op.adjoint, ss, lam, L, max_iter=K, shape=op.image_shape).eta
        return float(np.real(np.vdot(zbar, z)))

    fd = (J(s + h * d) - J(s - h * d)) / (2 * h)
    assert float(np.sum(res.s_bar * d)) == pytest.approx(fd, rel=1e-5)
