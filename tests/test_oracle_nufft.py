"""Pins of the oracle's min-max NUFFT (Fessler & Sutton, cited in §3.2).

The NUFFT is an approximation, so it is pinned against the plain definition
it approximates (the direct nonuniform DFT), against the worst-case bound the
min-max design itself promises, and by the adjoint identity.
"""
import math

import numpy as np
import pytest

from oracle import isam_oracle as O


def nudft(x, p, K):
    nz = x.size
    n = np.arange(nz) - nz // 2
    return np.exp(2j * math.pi * np.outer(p, n) / K) @ x


@pytest.mark.parametrize("nz", [16, 64, 256])
@pytest.mark.parametrize("J", [4, 6, 8])
def test_nufft_matches_direct_nudft_within_minmax_bound(nz, J):
    rng = np.random.default_rng(nz * 10 + J)
    K = 2 * nz
    interp = O.MinMaxInterpolator(nz, K, J)
    x = rng.standard_normal(nz) + 1j * rng.standard_normal(nz)
    # positions anywhere on the periodic grid, including exact grid nodes and wrap
    p = np.concatenate([rng.uniform(0, K, 200), np.arange(0, K, 7.0), [K - 1e-9, 0.5]])
    got = O.nufft_forward_column(x, p, interp)
    ref = nudft(x, p, K)
    err = np.abs(got - ref)
    # min-max design: |error(p)| <= worst_case(p) * ||x||  (Cauchy-Schwarz bound,
    # the design set contains the data support)
    bound = interp.worst_case_error(p - np.floor(p)) * np.linalg.norm(x)
    assert np.all(err <= bound * (1 + 1e-9) + 1e-12)
    rel = np.linalg.norm(err) / np.linalg.norm(ref)
    assert rel < {4: 2e-3, 6: 2e-5, 8: 3e-7}[J]


def test_nufft_error_falls_with_J():
    nz, K = 128, 256
    f = np.linspace(0, 1, 41)[:-1]
    w = [O.MinMaxInterpolator(nz, K, J).worst_case_error(f).max() / math.sqrt(nz + 1)
         for J in (4, 6, 8)]
    assert w[0] > 20 * w[1] > 400 * w[2]
    # published order of magnitude for J = 6, K = 2N with KB-shaped scaling
    assert 1e-7 < w[1] < 2e-5


def test_worst_case_is_attained():
    """The bound is tight: the conjugate error profile attains it."""
    nz, K, J = 32, 64, 6
    interp = O.MinMaxInterpolator(nz, K, J)
    p = np.array([17.3])
    f = p - np.floor(p)
    c = interp.coefficients(f)[0]
    g = 2 * math.pi / K
    lam = np.arange(J) - (J - 1) / 2
    n = interp.n
    # error profile over the design set, then worst-case signal on the data support
    e = interp.s * (np.exp(1j * g * np.outer(n, lam)) @ c) - np.exp(1j * g * (f[0] - 0.5) * n)
    x = np.conj(e[:-1]) / np.linalg.norm(e[:-1])
    # undo the common phase of the neighbour frame: the error on data x is
    m0 = int(np.floor(p[0])) - J // 2 + 1
    x = x * np.exp(-1j * g * (m0 + (J - 1) / 2) * n[:-1])
    err = abs(O.nufft_forward_column(x, p, interp)[0] - nudft(x, p, K)[0])
    assert err == pytest.approx(np.linalg.norm(e[:-1]), rel=1e-9)
    assert err <= interp.worst_case_error(f)[0] * (1 + 1e-12)


def test_coefficients_are_real_and_symmetric():
    interp = O.MinMaxInterpolator(64, 128, 6)
    f = np.array([0.1, 0.37, 0.5])
    c = interp.coefficients(f)
    # mirror symmetry of the symmetric design: c_l(f) = c_{J-1-l}(1-f)
    c2 = interp.coefficients(1 - f)
    np.testing.assert_allclose(c, c2[:, ::-1], rtol=1e-9, atol=1e-12)
    # interpolation of a constant signal (x = delta at n' = 0 gives Y = s(0) = 1)
    np.testing.assert_allclose(c.sum(axis=1), 1.0, atol=1e-4)


@pytest.mark.parametrize("J", [6, 8])
def test_nufft_adjoint_identity(J):
    rng = np.random.default_rng(3)
    nz, K = 64, 128
    interp = O.MinMaxInterpolator(nz, K, J)
    p = np.sort(rng.uniform(10, 300, 50))
    x = rng.standard_normal(nz) + 1j * rng.standard_normal(nz)
    y = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    lhs = np.vdot(y, O.nufft_forward_column(x, p, interp))
    rhs = np.vdot(O.nufft_adjoint_column(y, p, interp), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_kb_scaling_shape():
    n, s = O.kb_scaling(64, 128, 6)
    assert n[0] == -32 and n[-1] == 32 and s.size == 65
    assert s[32] == pytest.approx(1.0)
    np.testing.assert_allclose(s, s[::-1])
    assert np.all(np.diff(s[32:]) > 0)          # 1/psi_hat grows towards the band edge
