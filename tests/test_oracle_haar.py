"""Pins of the oracle's Haar prior (a wavelet-sparsity prior, §3.1).

The transform equals the explicit orthonormal Haar matrix built from its
basis functions (brute force for n <= 16), is orthonormal and inverted by
haar_inverse; the prox satisfies the optimality conditions of
min 1/2 ||z - u||^2 + tau ||details(W z)||_1 coefficient by coefficient and
beats random perturbations of itself."""
import math

import numpy as np
import pytest

from oracle import isam_oracle as O


def haar_matrix(n):
    """Rows: the constant 1/sqrt(n), then for each scale s (coarse to fine) and
    shift k the function +1 on the first half and -1 on the second half of the
    k-th block of length n/2^s, normalised."""
    rows = [np.full(n, 1 / math.sqrt(n))]
    s = 0
    while (1 << s) < n:
        blk = n >> s
        for k in range(1 << s):
            r = np.zeros(n)
            r[k * blk: k * blk + blk // 2] = 1
            r[k * blk + blk // 2: (k + 1) * blk] = -1
            rows.append(r / math.sqrt(blk))
        s += 1
    return np.array(rows)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16])
def test_haar_equals_explicit_matrix(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    H = haar_matrix(n)
    assert np.allclose(H @ H.T, np.eye(n), atol=1e-14)
    assert np.allclose(O.haar_forward(x), x @ H.T, atol=1e-13)
    assert np.allclose(O.haar_inverse(O.haar_forward(x)), x, atol=1e-13)


def test_haar_prox_optimality():
    rng = np.random.default_rng(7)
    n, tau = 32, 0.4
    u = rng.standard_normal((5, n)) + 1j * rng.standard_normal((5, n))
    z = O.haar_prox(u, tau)
    cz, cu = O.haar_forward(z), O.haar_forward(u)
    # approximation coefficient untouched; details: c_u - c_z = tau c_z/|c_z| or |c_u| <= tau
    assert np.allclose(cz[:, 0], cu[:, 0], atol=1e-13)
    d = cu[:, 1:] - cz[:, 1:]
    nz = np.abs(cz[:, 1:]) > 1e-12        # exact zeros come back as ~1e-17
    assert np.allclose(d[nz], tau * cz[:, 1:][nz] / np.abs(cz[:, 1:][nz]), atol=1e-12)
    assert np.all(np.abs(cu[:, 1:][~nz]) <= tau + 1e-12)

    def obj(zz):
        c = O.haar_forward(zz)
        return 0.5 * np.sum(np.abs(zz - u) ** 2) + tau * np.sum(np.abs(c[:, 1:]))
    f0 = obj(z)
    for k in range(20):
        p = rng.standard_normal(z.shape) + 1j * rng.standard_normal(z.shape)
        assert obj(z + 1e-3 * p) >= f0 - 1e-12
