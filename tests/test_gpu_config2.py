"""The benchmarked B-scan solved in full and compared with the oracle.

The 1024 A-scan x 2048-sample layered specimen, its spectra through the
12-bit count model with background removal (§4.1), lambda = 0.01 ||A^H s_d||_inf,
200 iterations of Alg. 1 with the relative residual of Eq. 15 evaluated every
20 iterations (a tolerance no residual reaches, as the bench runs it), on three
paths that take the same L: the oracle's FISTA (FP64, NumPy), the FP64 plan and
the FP32 plan.  Bars: FP32 within 1e-3 relative L2 of the oracle, FP64 within
1e-6; lambda within 1e-5 (FP32) / 1e-9 (FP64) of the oracle's.  The oracle's
part takes several minutes (its min-max coefficients for 2M samples, then 200
iterations of about one second), hence the slow mark.
"""
import time

import numpy as np
import pytest

from oracle import isam_oracle as O
from paper_1905_06058_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_config2_full_size_reconstruction():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1905_06058_gb300.isam import Plan

    t0 = time.perf_counter()
    wl = I.config2()
    geo = wl.geom
    ref = O.IsamOracle(geo, "nufft")
    k = geo.k_min + (geo.k_max - geo.k_min) / (geo.nk - 1) * np.arange(geo.nk)
    s32 = I.detector_counts(ref.forward(wl.eta), k, np.random.default_rng(wl.seed))
    s = s32.astype(np.float64)
    # one L for every side: 20 oracle power iterations with a 2% margin
    L = 1.02 * O.power_iteration(ref.forward, ref.adjoint, I.start_vector(ref.image_shape, 2), 20,
                                 1e-8)
    lam = O.lambda_from_data(ref.adjoint, s, wl.lambda_rel)
    res = O.fista(ref.forward, ref.adjoint, s, lam, L, max_iter=wl.iters, shape=ref.image_shape)
    t_oracle = time.perf_counter() - t0
    assert res.iterations == wl.iters

    errs = {}
    for prec, dt, bar, lam_tol in (("fp32", np.float32, 1e-3, 1e-5),
                                   ("fp64", np.float64, 1e-6, 1e-9)):
        plan = Plan(geo, precision=prec)
        sd = torch.from_numpy(np.ascontiguousarray(s32.astype(dt))).cuda()
        out, info = plan.solve(sd, lambda_rel=wl.lambda_rel, L=L, max_iter=wl.iters, tol=1e-12,
                               check_every=20)
        plan.close()
        assert info["iterations"] == wl.iters
        assert info["lam"] == pytest.approx(lam, rel=lam_tol)
        errs[prec] = rel(out.cpu().numpy(), res.eta)
        assert errs[prec] < bar, (prec, errs[prec])
    print(f"config 2, 200 iterations: FP32 vs oracle {errs['fp32']:.3e}, FP64 vs oracle "
          f"{errs['fp64']:.3e} (oracle {t_oracle:.0f} s, L = {L:.6f}, lambda = {lam:.6e})")
