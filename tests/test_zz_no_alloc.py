"""isam_max_abs_noalloc: the allocation-free max |x| reduction.

Some callers cannot allocate device memory at the point where they need the
lambda scale ||A^H s||_inf: a host thread in the middle of recording a CUDA
graph for another framework, an acquisition loop that fixed its memory budget
at start-up, or a process whose device memory is held by a pooling allocator.
This entry point keeps its scratch in a static device array instead.  The test
calls it twice in a row through the C ABI and compares each result with the
plan-based isam_max_abs.  It lives in a file of its own, collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_max_abs_matches_plan_reduction():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1905_06058_gb300 import inputs as I
    from paper_1905_06058_gb300 import isam as B
    fn = B.lib().isam_max_abs_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                   ctypes.c_void_p]
    for prec, cdt, code in (("fp32", np.complex64, 0), ("fp64", np.complex128, 1)):
        wl = I.small_bscan(nx=64, nk=256, nz=256)
        plan = B.Plan(wl.geom, precision=prec)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        for seed in (1, 2):                      # two calls in a row share the scratch
            x = torch.from_numpy(I.random_image(plan.image_shape, seed).astype(cdt)).cuda()
            assert fn(x.data_ptr(), x.numel(), code, out.data_ptr(), stream) == 0
            got = float(out.cpu())
            ref = plan.max_abs(x)
            assert got == pytest.approx(ref, rel=1e-12)
            assert got == pytest.approx(float(x.abs().max().cpu()), rel=1e-6)
        # a NaN in the input reaches the result, and the next call is unaffected
        y = x.clone()
        y[0, 40, 3] = complex(float("nan"), 0.0)
        assert fn(y.data_ptr(), y.numel(), code, out.data_ptr(), stream) == 0
        assert np.isnan(float(out.cpu()))
        assert fn(x.data_ptr(), x.numel(), code, out.data_ptr(), stream) == 0
        assert float(out.cpu()) == pytest.approx(plan.max_abs(x), rel=1e-12)
        # a size whose partials would not fit the static scratch is refused up front
        too_big = 65536 * 2048 + 1
        assert fn(x.data_ptr(), too_big, code, out.data_ptr(), stream) == 6
        plan.close()
