"""GPU parity of A and A^H (C ABI) against the FP64 oracle, element by element.

Tolerances: FP32 path <= 1e-5 relative L2 per application (and the adjoint
dot-product test <= 1e-5); FP64 path <= 1e-10 (its min-max coefficients are
fitted polynomials good to ~1e-14, its Stolt positions are double)."""
import math

import numpy as np
import pytest

from oracle import isam_oracle as O
from paper_1905_06058_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-10}


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    return T


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def plan_for(geom, prec="fp32", J=6, table=True):
    from paper_1905_06058_gb300.isam import Plan
    return Plan(geom, precision=prec, J=J, stolt_table=table)


def to_dev(torch, a, prec, cplx):
    if cplx:
        dt = np.complex128 if prec == "fp64" else np.complex64
    else:
        dt = np.float64 if prec == "fp64" else np.float32
    return torch.from_numpy(np.ascontiguousarray(a.astype(dt))).cuda()


CASES = [
    # (name, kwargs of small_bscan)
    ("bscan_32x64", dict(nx=32, nk=64, nz=64)),
    ("bscan_64x128_nz256", dict(nx=64, nk=128, nz=256)),
    ("bscan_128x256_nz512", dict(nx=128, nk=256, nz=512)),
    ("bscan_16x512", dict(nx=16, nk=512, nz=512)),
    ("ascan_q0", dict(nx=1, nk=64, nz=64)),
    ("volume_4x8x32", dict(nx=8, ny=4, nk=32, nz=32)),
    ("volume_8x8x64_nz128", dict(nx=8, ny=8, nk=64, nz=128)),
    ("evanescent_edge", dict(nx=32, nk=64, nz=64, dx_scale=0.08)),
    ("no_focus_no_disp", dict(nx=32, nk=64, nz=64, dispersion=False, focus_frac=0.5)),
    # nz = 2048 (K = 4096, 512 threads per column pair): the benchmarked size
    ("bscan_8x2048", dict(nx=8, nk=2048, nz=2048)),
    ("ascan_q0_2048", dict(nx=1, nk=2048, nz=2048)),
    ("volume_4x2x2048", dict(nx=4, ny=2, nk=2048, nz=2048)),
    ("bscan_4x1024_nz2048", dict(nx=4, nk=1024, nz=2048)),
    # lateral sizes 3 * 2^p: radix-8/4/2 passes then one radix-3 pass
    ("bscan_384x64_radix3", dict(nx=384, nk=64, nz=64)),
    ("bscan_768x32_radix3", dict(nx=768, nk=32, nz=64)),
    ("volume_24x24x32_radix3", dict(nx=24, ny=24, nk=32, nz=32)),
]


@pytest.mark.parametrize("table", [True, False], ids=["stolt_table", "stolt_evaluated"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("name,kw", CASES)
def test_forward_adjoint_match_oracle(torch, prec, name, kw, table):
    wl = I.small_bscan(seed=5, n_points=8, **kw)
    g = wl.geom
    ref = O.IsamOracle(g, "nufft")
    plan = plan_for(g, prec, table=table)
    eta = I.random_image(ref.image_shape, 1) * 0.5 + wl.eta
    s = plan.forward(to_dev(torch, eta, prec, True)).cpu().numpy()
    s_ref = ref.forward(eta)
    assert rel(s, s_ref) < TOL[prec], "forward"
    y = I.random_spectra(ref.spec_shape, 2)
    a = plan.adjoint(to_dev(torch, y, prec, False)).cpu().numpy()
    a_ref = ref.adjoint(y)
    assert rel(a, a_ref) < TOL[prec], "adjoint"
    plan.close()


@pytest.mark.parametrize("J", [4, 6, 8])
def test_k4096_matches_oracle_for_every_J(torch, J):
    """nz = 2048 (K = 4096) at 16 lateral columns, FP32, against the oracle."""
    wl = I.small_bscan(nx=16, nk=2048, nz=2048, seed=11)
    ref = O.IsamOracle(wl.geom, "nufft", J=J)
    eta = I.random_image(ref.image_shape, 12)
    y = I.random_spectra(ref.spec_shape, 13)
    plan = plan_for(wl.geom, "fp32", J=J)
    s = plan.forward(to_dev(torch, eta, "fp32", True)).cpu().numpy()
    a = plan.adjoint(to_dev(torch, y, "fp32", False)).cpu().numpy()
    plan.close()
    assert rel(s, ref.forward(eta)) < 1e-5
    assert rel(a, ref.adjoint(y)) < 1e-5


@pytest.mark.parametrize("J", [4, 8])
def test_other_neighbour_counts(torch, J):
    wl = I.small_bscan(nx=32, nk=128, nz=128, seed=9)
    ref = O.IsamOracle(wl.geom, "nufft", J=J)
    plan = plan_for(wl.geom, "fp32", J=J)
    eta = I.random_image(ref.image_shape, 3)
    s = plan.forward(to_dev(torch, eta, "fp32", True)).cpu().numpy()
    assert rel(s, ref.forward(eta)) < 1e-5
    y = I.random_spectra(ref.spec_shape, 4)
    a = plan.adjoint(to_dev(torch, y, "fp32", False)).cpu().numpy()
    assert rel(a, ref.adjoint(y)) < 1e-5
    plan.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-12)])
def test_adjoint_dot_product_on_gpu(torch, prec, tol):
    """<A eta, y> = Re<eta, A^H y> of the GPU operator pair itself."""
    wl = I.small_bscan(nx=64, nk=256, nz=256, seed=4)
    plan = plan_for(wl.geom, prec)
    eta = I.random_image(plan.image_shape, 5)
    y = I.random_spectra(plan.spec_shape, 6)
    Ae = plan.forward(to_dev(torch, eta, prec, True)).cpu().numpy().astype(np.float64)
    AHy = plan.adjoint(to_dev(torch, y, prec, False)).cpu().numpy().astype(np.complex128)
    lhs = np.sum(Ae * y)
    rhs = np.real(np.vdot(eta, AHy))
    assert abs(lhs - rhs) <= tol * np.linalg.norm(Ae) * np.linalg.norm(y)
    plan.close()


def test_nufft_tracks_exact_definition_on_gpu(torch):
    """GPU A against the plain nonuniform-DFT definition: within the J = 6 min-max bound."""
    wl = I.small_bscan(nx=32, nk=128, nz=128, seed=6)
    ex = O.IsamOracle(wl.geom, "exact")
    plan = plan_for(wl.geom, "fp64")
    eta = I.random_image(ex.image_shape, 7)
    s = plan.forward(to_dev(torch, eta, "fp64", True)).cpu().numpy()
    assert rel(s, ex.forward(eta)) < 1e-5


def test_launch_count_and_determinism(torch):
    wl = I.small_bscan(nx=64, nk=128, nz=128, seed=2)
    plan = plan_for(wl.geom)
    eta = to_dev(torch, I.random_image(plan.image_shape, 1), "fp32", True)
    s1 = plan.forward(eta)
    assert plan.last_launch_count() == 3
    s2 = plan.forward(eta)
    assert torch.equal(s1, s2)
    a1 = plan.adjoint(s1)
    assert plan.last_launch_count() == 3
    assert torch.equal(a1, plan.adjoint(s2))


# --------------------------------------------------------------------------
# Full-size B-scan (1024 A-scans x 2048 samples, the benchmarked launch
# configuration): sampled outputs that the oracle computes one by one.
# --------------------------------------------------------------------------

def test_full_bscan_forward_sampled_columns(torch):
    wl = I.config2(dtype=np.complex64)
    g = wl.geom
    plan = plan_for(g)
    eta = wl.eta.astype(np.complex64)
    s = plan.forward(to_dev(torch, eta, "fp32", True)).cpu().numpy()[0]
    # oracle: S(q, k) at a few k for every q column, then the lateral inverse FFT
    ref = O.IsamOracle(g, "nufft")
    gr = ref.grid
    ks = np.array([0, 1, 777, 1024, 2046, 2047])
    eta_hat = O.lateral_fft(eta.astype(np.complex128))[0]
    S = np.zeros((g.nx, ks.size), complex)
    for ix in range(g.nx):
        p = ref.p[0, ix, ks]
        S[ix] = O.nufft_forward_column(eta_hat[ix] / math.sqrt(gr.nz), p, ref.interp)
    S *= ref.phase[0][:, ks] * ref.prop[0][:, ks]
    s_ref = np.fft.ifft(S, axis=0, norm="ortho").real
    assert rel(s[:, ks], s_ref) < 1e-5


def test_full_bscan_adjoint_sampled_rows(torch):
    wl = I.config2(dtype=np.complex64)
    g = wl.geom
    plan = plan_for(g)
    y = I.random_spectra((1, g.nx, g.nk), 3).astype(np.float32)
    a = plan.adjoint(to_dev(torch, y, "fp32", False)).cpu().numpy()[0]
    ref = O.IsamOracle(g, "exact")
    gr = ref.grid
    rows = np.array([0, 5, 1023, 1024, 1500, 2047])
    R = O.lateral_fft(y.astype(np.float64).astype(complex))[0] * np.conj(ref.phase[0]) * ref.prop[0]
    G = np.zeros((g.nx, rows.size), complex)
    for ix in range(g.nx):
        E = np.exp(1j * np.outer(gr.z[rows], ref.beta[0, ix]))     # e^{+j beta z}
        G[ix] = E @ R[ix] / math.sqrt(gr.nz)
    a_ref = np.fft.ifft(G, axis=0, norm="ortho")
    # exact-definition reference: NUFFT (J = 6) approximation plus FP32 rounding
    assert rel(a[:, rows], a_ref) < 3e-5


# --------------------------------------------------------------------------
# Full-size volume (256 x 256 A-scans x 2048 samples, 2-D lateral transform,
# the benchmarked volume launch): sampled k planes of A eta and sampled depth
# planes of A^H y, each computed by the oracle one plane at a time.
# --------------------------------------------------------------------------

@pytest.mark.slow
def test_full_volume_forward_adjoint_sampled(torch):
    wl = I.config3(dtype=np.complex64)
    g = wl.geom
    ref = O.IsamOracle(g, "nufft")
    gr = ref.grid
    plan = plan_for(g)
    # forward: S(q, k) at six k for every (qy, qx) column, then the 2-D lateral IFFT
    s = plan.forward(to_dev(torch, wl.eta, "fp32", True))
    ks = np.array([0, 1, 777, 1024, 2046, 2047])
    s = s[:, :, torch.from_numpy(ks).cuda()].cpu().numpy()
    eta_hat = O.lateral_fft(wl.eta.astype(np.complex128))
    S = np.zeros((g.ny, g.nx, ks.size), complex)
    for iy in range(g.ny):
        for ix in range(g.nx):
            S[iy, ix] = O.nufft_forward_column(eta_hat[iy, ix] / math.sqrt(gr.nz),
                                               ref.p[iy, ix, ks], ref.interp)
    del eta_hat
    S *= ref.phase[:, :, ks] * ref.prop[:, :, ks]
    assert rel(s, O.lateral_ifft(S).real) < 1e-5
    # adjoint: the exact sum over k of R(q, k) e^{+j beta z} at six depths
    y = I.random_spectra(ref.spec_shape, 4).astype(np.float32)
    a = plan.adjoint(to_dev(torch, y, "fp32", False))
    rows = np.array([0, 5, 1023, 1024, 1500, 2047])
    a = a[:, :, torch.from_numpy(rows).cuda()].cpu().numpy()
    plan.close()
    R = O.lateral_fft(y.astype(np.float64).astype(complex)) * np.conj(ref.phase) * ref.prop
    G = np.zeros((g.ny, g.nx, rows.size), complex)
    for i, r in enumerate(rows):
        for iy in range(0, g.ny, 32):
            E = np.exp(1j * gr.z[r] * ref.beta[iy:iy + 32])
            G[iy:iy + 32, :, i] = np.einsum("yxk,yxk->yx", R[iy:iy + 32], E)
    G /= math.sqrt(gr.nz)
    # exact-definition reference: NUFFT (J = 6) approximation plus FP32 rounding
    assert rel(a, O.lateral_ifft(G)) < 3e-5
