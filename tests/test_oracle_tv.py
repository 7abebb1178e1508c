"""Pins of the oracle's total-variation prior (§3.1).

grad^H is the adjoint of grad (dot-product test); TV of a constant image is
0 and the prox leaves it unchanged; the duality gap of the FGP prox,
computed from the definitions (primal 1/2||z - u||^2 + tau TV(z) against the
dual -1/2||u - tau grad^H p||^2 + 1/2||u||^2 for the feasible p), closes
with the iteration count; on a tiny real 1-D case the prox matches a brute
force minimisation of the (exact, nonsmooth) objective."""
import numpy as np

from oracle import isam_oracle as O


def test_grad_adjoint_dot_product():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 5, 7)) + 1j * rng.standard_normal((2, 5, 7))
    px = rng.standard_normal((2, 5, 7)) + 1j * rng.standard_normal((2, 5, 7))
    pz = rng.standard_normal((2, 5, 7)) + 1j * rng.standard_normal((2, 5, 7))
    gx, gz = O.tv_grad(x)
    lhs = np.vdot(px, gx) + np.vdot(pz, gz)
    rhs = np.vdot(O.tv_grad_adjoint(px, pz), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_constant_image_is_fixed():
    u = np.full((1, 6, 8), 0.3 - 0.7j)
    assert O.total_variation(u) == 0.0
    assert np.allclose(O.TVProx(30)(u, 0.5), u, atol=1e-15)


def gap(u, tau, prox):
    z = prox(u, tau)
    primal = 0.5 * np.sum(np.abs(z - u) ** 2) + tau * O.total_variation(z)
    m = np.sqrt(np.abs(prox.px) ** 2 + np.abs(prox.pz) ** 2)
    assert m.max() <= 1 + 1e-12                           # dual feasible
    v = u - tau * O.tv_grad_adjoint(prox.px, prox.pz)
    dual = -0.5 * np.sum(np.abs(v) ** 2) + 0.5 * np.sum(np.abs(u) ** 2)
    return primal - dual, primal


def test_duality_gap_closes():
    rng = np.random.default_rng(2)
    u = rng.standard_normal((1, 12, 16)) + 1j * rng.standard_normal((1, 12, 16))
    gaps = []
    for iters in (5, 50, 2000):
        g, primal = gap(u, 0.3, O.TVProx(iters))
        assert g >= -1e-9
        gaps.append(g / primal)
    assert gaps[2] < 1e-4 and gaps[2] < gaps[1] < gaps[0]


def test_prox_matches_brute_force_1d():
    from scipy.optimize import minimize
    rng = np.random.default_rng(3)
    u = rng.standard_normal((1, 1, 6))
    tau = 0.4
    z = O.TVProx(5000)(u.astype(complex), tau).real

    def f(v):
        return 0.5 * np.sum((v - u[0, 0]) ** 2) + tau * np.sum(np.abs(np.diff(v)))
    best = min((minimize(f, x0, method="Nelder-Mead", options=dict(xatol=1e-10, fatol=1e-14,
                                                                     maxiter=40000))
                for x0 in (u[0, 0], z[0, 0], np.zeros(6))), key=lambda r: r.fun)
    assert f(z[0, 0]) <= best.fun + 1e-8
    assert np.allclose(z[0, 0], best.x, atol=1e-3)
