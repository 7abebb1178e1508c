"""Pins of the oracle's MBIR solver (§3, Eq. 12, 14, 15; Alg. 1).

Hand-worked closed forms (tests/golden/), the first-order optimality (KKT)
certificate of the weighted-l1 problem, agreement with plain ISTA run to
convergence, the lambda above which the minimiser is zero, and recovery of
isolated point scatterers (the paper's sparsity premise).
"""
import os

import numpy as np
import pytest

from oracle import isam_oracle as O
from paper_1905_06058_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#", ndmin=2)


def test_soft_threshold_hand_values():
    for ur, ui, tau, er, ei in load("soft_threshold.txt"):
        got = O.soft_threshold(np.array([ur + 1j * ui]), tau)[0]
        assert got == pytest.approx(er + 1j * ei, abs=1e-15)


def test_soft_threshold_is_prox_of_weighted_l1():
    """T_tau(u) minimises 1/2|v-u|^2 + tau|v| (checked by brute force on a grid)."""
    rng = np.random.default_rng(0)
    for _ in range(5):
        u = complex(*rng.normal(size=2))
        tau = rng.uniform(0, 1.5)
        t = O.soft_threshold(np.array([u]), tau)[0]
        xs = np.linspace(-3, 3, 601)
        V = xs[:, None] + 1j * xs[None, :]
        f = 0.5 * np.abs(V - u) ** 2 + tau * np.abs(V)
        best = V.ravel()[np.argmin(f)]
        assert abs(best - t) < 0.015


def test_fista_momentum_hand_values():
    t = O.fista_t_sequence(5)
    for k, tk in load("fista_momentum.txt"):
        assert t[int(k) - 1] == pytest.approx(tk, rel=1e-15)
    assert np.all(t >= (np.arange(1, 7) + 1) / 2)        # t^k >= (k+1)/2


def test_relative_residual_hand_values():
    for d0, d1, g0, g1, e in load("relative_residual.txt"):
        eta = np.zeros(2)
        z = np.array([d0, d1])
        g = np.array([g0, g1])
        assert O.relative_residual(z, eta, g, eps=0.0) == pytest.approx(e, rel=1e-15)


def test_objective_hand_values():
    """Eq. 12 on the hand case of tests/golden/objective.txt: a dropped 1/2, a
    weight applied twice or to the data term, |eta|^2 for |eta| or a sign error
    in the residual each change every row."""
    def A(eta):
        return np.array([eta[0].real + eta[1].real, eta[0].imag, eta[1].real - eta[0].imag])

    eta = np.array([3 + 4j, -1 + 0j])
    s_d = np.array([1.0, 2.0, -1.0])
    for lam, w0, w1, e in load("objective.txt"):
        got = O.objective(A, eta, s_d, lam, np.array([w0, w1]))
        assert got == pytest.approx(e, rel=1e-15)


def test_objective_with_the_isam_operator():
    """With the real operator: at eta = 0 only 1/2 ||s_d||^2 remains, and with
    s_d = A eta only the weighted l1 term (to rounding of A eta - s_d)."""
    wl = I.small_bscan(nx=8, nk=16, nz=16, n_points=4, seed=5)
    op = O.IsamOracle(wl.geom, "exact")
    s = op.forward(wl.eta)
    w = I.depth_weights(op.grid.nz)[None, None, :]
    zero = np.zeros(op.image_shape, complex)
    assert O.objective(op.forward, zero, s, 0.3, w) == pytest.approx(0.5 * np.sum(s * s),
                                                                       rel=1e-14)
    l1 = float(np.sum(w * np.abs(wl.eta)))
    assert l1 > 0
    assert O.objective(op.forward, wl.eta, s, 0.3, w) == pytest.approx(0.3 * l1, rel=1e-12)


def tiny_problem(mode="exact", seed=3, nx=4, nk=8, nz=8, n_points=3):
    wl = I.small_bscan(nx=nx, nk=nk, nz=nz, n_points=n_points, seed=seed)
    op = O.IsamOracle(wl.geom, mode)
    s = op.forward(wl.eta)
    return wl, op, s


def kkt_violation(op, eta, s, lam, w):
    g = op.adjoint(op.forward(eta) - s)
    on = np.abs(eta) > 1e-9
    viol_on = np.abs(g[on] + lam * w[on] * eta[on] / np.abs(eta[on]))
    viol_off = np.maximum(np.abs(g[~on]) - lam * w[~on], 0)
    return max(viol_on.max(initial=0), viol_off.max(initial=0)) / lam


def test_fista_reaches_kkt_point_and_matches_ista():
    wl, op, s = tiny_problem()
    L = O.power_iteration(op.forward, op.adjoint, I.start_vector(op.image_shape, 1), 500, 1e-14)
    lam = 0.05 * np.abs(op.adjoint(s)).max()
    w = np.broadcast_to(I.depth_weights(op.grid.nz), op.image_shape)
    res = O.fista(op.forward, op.adjoint, s, lam, L, w=w, max_iter=4000, shape=op.image_shape)
    assert kkt_violation(op, res.eta, s, lam, w) < 1e-6
    # plain ISTA (no momentum) run long on the dense matrix reaches the same objective
    M = O.dense_real_matrix(op)
    n = res.eta.size
    x = np.zeros(2 * n)
    for _ in range(60000):
        v = x - M.T @ (M @ x - s.ravel()) / L
        c = O.soft_threshold(v[:n] + 1j * v[n:], lam * w.ravel() / L)
        x = np.concatenate([c.real, c.imag])
    eta_ista = (x[:n] + 1j * x[n:]).reshape(op.image_shape)
    f_fista = O.objective(op.forward, res.eta, s, lam, w)
    f_ista = O.objective(op.forward, eta_ista, s, lam, w)
    assert abs(f_fista - f_ista) <= 1e-8 * f_ista


def test_zero_solution_above_lambda_max_and_addback():
    """lambda >= max|A^H s| / w  =>  minimiser 0; add-back then returns A^H s / L."""
    wl, op, s = tiny_problem()
    L = O.power_iteration(op.forward, op.adjoint, I.start_vector(op.image_shape, 1), 300)
    ahs = op.adjoint(s)
    lam = O.lambda_from_data(op.adjoint, s, 1.0)
    assert lam == pytest.approx(np.abs(ahs).max())
    res = O.fista(op.forward, op.adjoint, s, lam * 1.0001, L, max_iter=20,
                  shape=op.image_shape, addback=True)
    np.testing.assert_allclose(res.eta, ahs / L, atol=1e-14)
    res2 = O.fista(op.forward, op.adjoint, s, lam * 1.0001, L, max_iter=20, shape=op.image_shape)
    assert np.abs(res2.eta).max() == 0.0


def test_stop_rule_breaks_early():
    wl, op, s = tiny_problem()
    L = O.power_iteration(op.forward, op.adjoint, I.start_vector(op.image_shape, 1), 300)
    lam = 0.05 * np.abs(op.adjoint(s)).max()
    res = O.fista(op.forward, op.adjoint, s, lam, L, max_iter=5000, tol=1e-3,
                  shape=op.image_shape)
    assert res.iterations < 5000 and res.rr < 1e-3


def test_recovers_isolated_point_scatterers():
    """Noiseless spectra of a few isolated on-grid scatterers at both delays:
    l1-MBIR (Alg. 1) recovers their support and amplitudes up to shrinkage,
    the mirror terms are suppressed by the dispersion encoding (§2, Eq. 8)."""
    wl = I.small_bscan(nx=16, nk=64, nz=64, n_points=4, seed=21, min_sep=6)
    op = O.IsamOracle(wl.geom, "exact")
    s = op.forward(wl.eta)
    L = O.power_iteration(op.forward, op.adjoint, I.start_vector(op.image_shape, 1), 200)
    lam = 0.02 * np.abs(op.adjoint(s)).max()
    res = O.fista(op.forward, op.adjoint, s, lam, L, max_iter=3000, shape=op.image_shape)
    truth = np.abs(wl.eta) > 0
    top = np.argsort(np.abs(res.eta).ravel())[::-1][: truth.sum()]
    assert set(top) == set(np.flatnonzero(truth.ravel()))
    err = np.abs(res.eta[truth] - wl.eta[truth])
    assert err.max() < 0.1 * np.abs(wl.eta[truth]).min()
    # nothing but the scatterers survives above 5% of the weakest one
    rest = np.abs(res.eta[~truth])
    assert rest.max() < 0.05 * np.abs(wl.eta[truth]).min()
