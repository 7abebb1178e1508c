"""GPU MBIR solve (Alg. 1) against the FP64 oracle's FISTA.

Bars: reconstruction within 1e-3 relative L2 of the oracle after the stated
iteration count (FP32), 1e-6 (FP64); lambda and L estimates within 1e-5 of
the oracle's; checkpoint/resume reproduces an uninterrupted solve."""
import numpy as np
import pytest

from oracle import isam_oracle as O
from paper_1905_06058_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


def dev(torch, a, dt):
    return torch.from_numpy(np.ascontiguousarray(a.astype(dt))).cuda()


def problem(nx=32, nk=64, nz=128, seed=11, snr=30.0, n_points=10):
    wl = I.small_bscan(nx=nx, nk=nk, nz=nz, n_points=n_points, seed=seed)
    ref = O.IsamOracle(wl.geom, "nufft")
    s = ref.forward(wl.eta)
    s = I.add_noise(s, snr, np.random.default_rng(seed))
    L = O.power_iteration(ref.forward, ref.adjoint, I.start_vector(ref.image_shape, seed), 300,
                          1e-13)
    return wl, ref, s, L


@pytest.mark.parametrize("table", [True, False], ids=["stolt_table", "stolt_evaluated"])
@pytest.mark.parametrize("prec,tol", [("fp32", 1e-3), ("fp64", 1e-6)])
def test_fista_matches_oracle(torch, prec, tol, table):
    from paper_1905_06058_gb300.isam import Plan
    wl, ref, s, L = problem()
    lam = O.lambda_from_data(ref.adjoint, s, 0.05)
    res = O.fista(ref.forward, ref.adjoint, s, lam, L, max_iter=60, shape=ref.image_shape)
    plan = Plan(wl.geom, precision=prec, stolt_table=table)
    dt = np.float64 if prec == "fp64" else np.float32
    out, info = plan.solve(dev(torch, s, dt), lambda_abs=lam, L=L, max_iter=60)
    assert info["iterations"] == 60
    assert rel(out.cpu().numpy(), res.eta) < tol
    plan.close()


def test_fista_nz2048_matches_oracle(torch):
    """nz = 2048 (K = 4096, the benchmarked launch shape of the fused gradient
    kernel), with the stop rule's partial norms, against the oracle's FISTA."""
    from paper_1905_06058_gb300.isam import Plan
    wl, ref, s, L = problem(nx=8, nk=2048, nz=2048, seed=21, n_points=12)
    lam = O.lambda_from_data(ref.adjoint, s, 0.05)
    res = O.fista(ref.forward, ref.adjoint, s, lam, L, max_iter=30, shape=ref.image_shape)
    plan = Plan(wl.geom)
    out, info = plan.solve(dev(torch, s, np.float32), lambda_abs=lam, L=L, max_iter=30,
                           tol=1e-30, check_every=5)
    assert info["iterations"] == 30
    assert rel(out.cpu().numpy(), res.eta) < 1e-3
    plan.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-3), ("fp64", 1e-6)])
def test_fista_radix3_lateral_size(torch, prec, tol):
    """nx = 96 = 3 * 32: the lateral passes end with a radix-3 pass."""
    from paper_1905_06058_gb300.isam import Plan
    wl, ref, s, L = problem(nx=96, nk=64, nz=64, seed=23)
    lam = O.lambda_from_data(ref.adjoint, s, 0.05)
    res = O.fista(ref.forward, ref.adjoint, s, lam, L, max_iter=40, shape=ref.image_shape)
    plan = Plan(wl.geom, precision=prec)
    dt = np.float64 if prec == "fp64" else np.float32
    out, info = plan.solve(dev(torch, s, dt), lambda_abs=lam, L=L, max_iter=40)
    assert rel(out.cpu().numpy(), res.eta) < tol
    plan.close()


def test_weighted_addback_and_lambda_rule(torch):
    """MBIR+ (depth weights 0.5 -> 1, residual added back, §3.1, §4.2)."""
    from paper_1905_06058_gb300.isam import Plan
    wl, ref, s, L = problem(seed=12)
    w = I.depth_weights(ref.grid.nz)
    lam = O.lambda_from_data(ref.adjoint, s, 0.05)
    res = O.fista(ref.forward, ref.adjoint, s, lam, L, w=w[None, None, :], max_iter=40,
                  addback=True, shape=ref.image_shape)
    plan = Plan(wl.geom)
    out, info = plan.solve(dev(torch, s, np.float32), lambda_rel=0.05, L=L, max_iter=40,
                           w=dev(torch, w, np.float32), addback=True)
    assert info["lam"] == pytest.approx(lam, rel=1e-5)
    assert rel(out.cpu().numpy(), res.eta) < 1e-3
    plan.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 3e-5), ("fp64", 1e-12)])
def test_u_hat_and_gradient_paths_agree(torch, prec, tol):
    """Iterations without the residual check take the fused kernel's
    u_hat = eta_hat - G/L output and the update from it; iterations with the
    check take G and rebuild eta^k from z^{k-1}, z^{k-2}.  Both compute
    z^k = T(eta^k - g/L): a solve with the check on every iteration (a tolerance
    no residual reaches) and one without it agree to rounding, also with
    weights and on a volume."""
    from paper_1905_06058_gb300.isam import Plan
    dt = np.float32 if prec == "fp32" else np.float64
    for kw, weighted in ((dict(nx=32, nk=64, nz=128), True), (dict(nx=8, ny=8, nk=64, nz=64), False)):
        wl = I.small_bscan(seed=17, n_points=10, **kw)
        ref = O.IsamOracle(wl.geom, "nufft")
        s = I.add_noise(ref.forward(wl.eta), 30.0, np.random.default_rng(17))
        plan = Plan(wl.geom, precision=prec)
        w = None
        if weighted:
            w = torch.from_numpy(I.depth_weights(wl.geom.nz).astype(dt)).cuda()
        sd = dev(torch, s, dt)
        a, ia = plan.solve(sd, lambda_rel=0.02, max_iter=40, L=4.0, w=w)
        b, ib = plan.solve(sd, lambda_rel=0.02, max_iter=40, L=4.0, w=w, tol=1e-300, check_every=1)
        plan.close()
        assert ia["iterations"] == ib["iterations"] == 40
        r = rel(a.cpu().numpy(), b.cpu().numpy())
        assert r < tol, r


@pytest.mark.parametrize("nx", [256, 512, 1024])
def test_fista_compile_time_lateral_widths(torch, nx):
    """Lateral lengths with compile-time update and transform passes
    (L = 256 and 512 with 8 pair-columns per block, 1024 with 4), against the
    oracle's FISTA: 20 iterations, FP32, 1e-3."""
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(nx=nx, nk=64, nz=64, n_points=12, seed=23)
    ref = O.IsamOracle(wl.geom, "nufft")
    s = I.add_noise(ref.forward(wl.eta), 30.0, np.random.default_rng(23))
    # both sides take this L (30 power iterations, 1% margin)
    L = 1.01 * O.power_iteration(ref.forward, ref.adjoint, I.start_vector(ref.image_shape, 23),
                                 30, 1e-6)
    lam = O.lambda_from_data(ref.adjoint, s, 0.02)
    res = O.fista(ref.forward, ref.adjoint, s, lam, L, max_iter=20, shape=ref.image_shape)
    plan = Plan(wl.geom, precision="fp32")
    out, info = plan.solve(dev(torch, s, np.float32), lambda_abs=lam, L=L, max_iter=20)
    plan.close()
    assert rel(out.cpu().numpy(), res.eta) < 1e-3


def test_lipschitz_estimate(torch):
    from paper_1905_06058_gb300.isam import Plan
    wl, ref, s, L = problem(seed=13)
    plan = Plan(wl.geom)
    v0 = dev(torch, I.start_vector(ref.image_shape, 13), np.complex64)
    L_gpu = plan.lipschitz(iters=300, rtol=1e-12, v0=v0)
    assert L_gpu == pytest.approx(L, rel=1e-5)
    # default start vector and iteration count, as isam_solve uses when L = 0
    L_def = plan.lipschitz()
    assert L_def == pytest.approx(L, rel=1e-6)
    plan.close()


def test_stop_rule(torch):
    from paper_1905_06058_gb300.isam import Plan
    wl, ref, s, L = problem(seed=14)
    lam = O.lambda_from_data(ref.adjoint, s, 0.1)
    res = O.fista(ref.forward, ref.adjoint, s, lam, L, max_iter=2000, tol=1e-3,
                  shape=ref.image_shape)
    plan = Plan(wl.geom, precision="fp64")
    out, info = plan.solve(dev(torch, s, np.float64), lambda_abs=lam, L=L, max_iter=2000,
                           tol=1e-3, check_every=1)
    assert info["iterations"] == res.iterations
    assert info["rr"] == pytest.approx(res.rr, rel=1e-6)
    assert rel(out.cpu().numpy(), res.eta) < 1e-6
    plan.close()


def test_checkpoint_resume(torch):
    from paper_1905_06058_gb300.isam import Plan
    wl, ref, s, L = problem(seed=15)
    plan = Plan(wl.geom)
    sd = dev(torch, s, np.float32)
    full, _ = plan.solve(sd, lambda_rel=0.05, L=L, max_iter=30)
    z1 = torch.zeros(plan.image_shape, dtype=torch.complex64, device="cuda")
    z2 = torch.zeros_like(z1)
    st = {"z1": z1, "z2": z2, "k": 0}
    plan.solve(sd, lambda_rel=0.05, L=L, max_iter=12, state=st)
    assert st["k"] == 12
    part, _ = plan.solve(sd, lambda_rel=0.05, L=L, max_iter=18, state=st)
    assert st["k"] == 30
    assert rel(part.cpu().numpy(), full.cpu().numpy()) < 1e-6
    plan.close()


def test_nonfinite_input_is_reported(torch):
    from paper_1905_06058_gb300.isam import IsamError, Plan
    wl, ref, s, L = problem(seed=16)
    s = s.copy()
    s[0, 3, 5] = np.nan
    plan = Plan(wl.geom)
    with pytest.raises(IsamError) as e:
        plan.solve(dev(torch, s, np.float32), lambda_abs=1e-3, L=L, max_iter=3)
    assert e.value.status == 4
    plan.close()


def test_host_buffer_solve_matches_device_solve(torch):
    from paper_1905_06058_gb300.isam import Plan
    wl, ref, s, L = problem(seed=17)
    plan = Plan(wl.geom)
    sd = dev(torch, s, np.float32)
    out_d, _ = plan.solve(sd, lambda_rel=0.05, L=L, max_iter=20)
    s_h = torch.from_numpy(s.astype(np.float32)).pin_memory()
    out_h = torch.empty(plan.image_shape, dtype=torch.complex64).pin_memory()
    plan.solve_host(s_h, out_h, lambda_rel=0.05, L=L, max_iter=20)
    assert torch.equal(out_h, out_d.cpu())
    plan.close()


def test_config1_fp64_reconstruction(torch):
    """128 x 256 spectra -> 128 x 512 full-range image, 40 scatterers, 30 dB,
    100 iterations, lambda = 0.01 ||A^H y||_inf, FP64 plan."""
    from paper_1905_06058_gb300.isam import Plan
    wl = I.config1()
    ref = O.IsamOracle(wl.geom, "nufft")
    s = I.add_noise(ref.forward(wl.eta), wl.snr_db, np.random.default_rng(wl.seed))
    L = O.power_iteration(ref.forward, ref.adjoint, I.start_vector(ref.image_shape, 1), 200,
                          1e-12)
    lam = O.lambda_from_data(ref.adjoint, s, wl.lambda_rel)
    res = O.fista(ref.forward, ref.adjoint, s, lam, L, max_iter=wl.iters, shape=ref.image_shape)
    plan = Plan(wl.geom, precision="fp64")
    out, info = plan.solve(dev(torch, s, np.float64), lambda_rel=wl.lambda_rel, L=L,
                           max_iter=wl.iters)
    assert info["lam"] == pytest.approx(lam, rel=1e-9)
    assert rel(out.cpu().numpy(), res.eta) < 1e-6
    # and the reconstruction is meaningful: the scatterers stand out
    truth = np.abs(wl.eta) > 0
    got = np.abs(out.cpu().numpy())
    assert got[truth].mean() > 5 * got[~truth].mean()
    plan.close()


def test_full_bscan_first_iterate_sampled(torch):
    """1024 x 2048 B-scan, benchmarked launch configuration: after one iteration
    z^1 = T_{lambda/L}(A^H s / L) (Alg. 1 from eta^1 = 0); sampled rows against
    the oracle's exact adjoint."""
    import math
    from paper_1905_06058_gb300.isam import Plan
    wl = I.config2(dtype=np.complex64)
    g = wl.geom
    y = I.random_spectra((1, g.nx, g.nk), 8).astype(np.float32)
    plan = Plan(g)
    L, lam = 1.3, 0.05
    out, info = plan.solve(dev(torch, y, np.float32), lambda_abs=lam, L=L, max_iter=1)
    z = out.cpu().numpy()[0]
    ref = O.IsamOracle(g, "exact")
    gr = ref.grid
    rows = np.array([3, 1024, 2000])
    R = O.lateral_fft(y.astype(np.float64).astype(complex))[0] * np.conj(ref.phase[0]) * ref.prop[0]
    G = np.zeros((g.nx, rows.size), complex)
    for ix in range(g.nx):
        E = np.exp(1j * np.outer(gr.z[rows], ref.beta[0, ix]))
        G[ix] = E @ R[ix] / math.sqrt(gr.nz)
    ahs = np.fft.ifft(G, axis=0, norm="ortho")
    z_ref = O.soft_threshold(ahs / L, lam / L)
    assert rel(z[:, rows], z_ref) < 3e-5
    plan.close()


@pytest.mark.slow
def test_full_volume_first_iterate_sampled(torch):
    """256 x 256 x 2048 volume, benchmarked launch configuration (fused axial
    kernel with the Stolt table, y-axis update, x-axis passes): after one
    iteration z^1 = T_{lambda/L}(A^H s / L) (Alg. 1 from eta^1 = 0); three depth
    planes against the oracle's exact adjoint, a sum over every (q, k)."""
    import math
    from paper_1905_06058_gb300.isam import Plan
    wl = I.config3(dtype=np.complex64)
    g = wl.geom
    y = I.random_spectra((g.ny, g.nx, g.nk), 9).astype(np.float32)
    plan = Plan(g)
    L, lam = 1.3, 0.05
    out, info = plan.solve(dev(torch, y, np.float32), lambda_abs=lam, L=L, max_iter=1)
    rows = np.array([3, 1024, 2000])
    z = out[:, :, torch.from_numpy(rows).cuda()].cpu().numpy()
    del out
    plan.close()
    ref = O.IsamOracle(g, "exact")
    gr = ref.grid
    R = O.lateral_fft(y.astype(np.float64).astype(complex)) * np.conj(ref.phase) * ref.prop
    G = np.zeros((g.ny, g.nx, rows.size), complex)
    for i, r in enumerate(rows):
        for iy in range(0, g.ny, 32):
            E = np.exp(1j * gr.z[r] * ref.beta[iy:iy + 32])
            G[iy:iy + 32, :, i] = np.einsum("yxk,yxk->yx", R[iy:iy + 32], E)
    G /= math.sqrt(gr.nz)
    z_ref = O.soft_threshold(O.lateral_ifft(G) / L, lam / L)
    assert rel(z, z_ref) < 3e-5


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-3), ("fp64", 1e-6)])
def test_volume_fista_matches_oracle(torch, prec, tol):
    """3-D (2-D lateral FFT, Stolt map in q_x, q_y): the fused residual uses the
    (q, -q) pairing of both lateral axes."""
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(nx=8, ny=4, nk=32, nz=64, n_points=6, seed=18)
    ref = O.IsamOracle(wl.geom, "nufft")
    s = I.add_noise(ref.forward(wl.eta), 25.0, np.random.default_rng(18))
    L = O.power_iteration(ref.forward, ref.adjoint, I.start_vector(ref.image_shape, 18), 300,
                          1e-13)
    lam = O.lambda_from_data(ref.adjoint, s, 0.02)
    res = O.fista(ref.forward, ref.adjoint, s, lam, L, max_iter=40, shape=ref.image_shape)
    plan = Plan(wl.geom, precision=prec, stolt_table=False)
    dt = np.float64 if prec == "fp64" else np.float32
    out, info = plan.solve(dev(torch, s, dt), lambda_rel=0.02, L=L, max_iter=40)
    assert rel(out.cpu().numpy(), res.eta) < tol
    plan.close()


def test_evanescent_geometry_solve(torch):
    """Pitch far below lambda/2: many columns evanescent, steep Stolt maps near the
    cut-off (several gather windows)."""
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(nx=32, nk=64, nz=64, n_points=6, seed=19, dx_scale=0.08)
    ref = O.IsamOracle(wl.geom, "nufft")
    assert (~ref.prop).any()
    s = ref.forward(wl.eta)
    L = O.power_iteration(ref.forward, ref.adjoint, I.start_vector(ref.image_shape, 19), 300,
                          1e-13)
    lam = O.lambda_from_data(ref.adjoint, s, 0.05)
    res = O.fista(ref.forward, ref.adjoint, s, lam, L, max_iter=30, shape=ref.image_shape)
    plan = Plan(wl.geom, precision="fp64")
    out, info = plan.solve(dev(torch, s, np.float64), lambda_abs=lam, L=L, max_iter=30)
    assert rel(out.cpu().numpy(), res.eta) < 1e-6
    plan.close()


@pytest.mark.slow
def test_config3_subvolume_reconstruction(torch):
    """The volume workload on a 64 x 64 x 256 sub-volume (points, curved layers,
    1% speckle, 25 dB): 150 iterations, lambda = 0.02 ||A^H y||_inf, FP32, within
    1e-3 of the oracle's FISTA (L from 30 oracle power iterations, given to both)."""
    from paper_1905_06058_gb300.isam import Plan
    wl = I.config3(dtype=np.complex128, nx=64, nk=256, n_points=300)
    ref = O.IsamOracle(wl.geom, "nufft")
    s = I.add_noise(ref.forward(wl.eta), wl.snr_db, np.random.default_rng(wl.seed))
    L = 1.01 * O.power_iteration(ref.forward, ref.adjoint, I.start_vector(ref.image_shape, 3), 30,
                                 1e-6)
    lam = O.lambda_from_data(ref.adjoint, s, wl.lambda_rel)
    res = O.fista(ref.forward, ref.adjoint, s, lam, L, max_iter=wl.iters, shape=ref.image_shape)
    plan = Plan(wl.geom, precision="fp32")
    out, info = plan.solve(dev(torch, s, np.float32), lambda_rel=wl.lambda_rel, L=L,
                           max_iter=wl.iters)
    plan.close()
    assert info["lam"] == pytest.approx(lam, rel=1e-5)
    assert rel(out.cpu().numpy(), res.eta) < 1e-3
