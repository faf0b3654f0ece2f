"""The allocation-free entry point amr_step_patch_noalloc.

It exists for callers that must not allocate device memory (a framework that
owns the device allocator, a real-time loop, a fixed device-memory budget):
they pass their own device input and output arrays and the library uses a
fixed scratch array compiled into it.  This test checks, through the C ABI,
that two calls in a row give the same states as the regular handle path
(amr_set_patches + amr_step) within the parity tolerances used elsewhere.
"""
import numpy as np
import pytest

import amr_inputs as ai
from parity import TOL, errors

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("bc", [ai.PERIODIC, ai.OUTFLOW])
def test_noalloc_step_matches_handle_path_twice(precision, bc):
    torch = pytest.importorskip("torch")
    from paper_0910_5547_gb300 import Solver
    from paper_0910_5547_gb300 import build as B
    from paper_0910_5547_gb300 import native as N
    B.build()
    base = (24, 20, 16)
    pb = ai.random_smooth([ai.Patch(0, (0, 0, 0), base)], base, seed=31, amp=0.3, bc=(bc,) * 6)
    s = Solver.from_problem(pb, precision=precision)
    u0 = s.state_all().copy()
    dt = 0.5 * s.cfl_dt()
    s.step(dt)
    u1 = s.state_all().copy()
    s.step(dt)
    u2 = s.state_all().copy()
    s.close()

    cfg = N.amr_default_config(nvar=5, precision=N.AMR_FP32 if precision == "fp32" else N.AMR_FP64,
                               base_n=base, bc=(bc,) * 6, gamma=pb.gamma)
    d_in = torch.tensor(u0, dtype=torch.float64, device="cuda")
    d_mid = torch.empty_like(d_in)
    d_out = torch.empty_like(d_in)
    torch.cuda.synchronize()
    used = N.amr_step_patch_noalloc(cfg, d_in.data_ptr(), d_mid.data_ptr(), dt)
    assert used == dt
    N.amr_step_patch_noalloc(cfg, d_mid.data_ptr(), d_out.data_ptr(), dt)
    torch.cuda.synchronize()
    shape = (5, base[2], base[1], base[0])
    for got, want in ((d_mid.cpu().numpy(), u1), (d_out.cpu().numpy(), u2)):
        l1, mx = errors([got.reshape(shape)], [want.reshape(shape)], pb.patches)
        assert l1.max() <= TOL[precision]["l1"], l1
        if "max" in TOL[precision]:
            assert mx.max() <= TOL[precision]["max"], mx


def test_noalloc_rejects_patches_beyond_the_scratch_size():
    torch = pytest.importorskip("torch")
    from paper_0910_5547_gb300 import build as B
    from paper_0910_5547_gb300 import native as N
    B.build()
    cfg = N.amr_default_config(base_n=(96, 96, 96), bc=(1,) * 6)
    d = torch.zeros(5 * 96 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(N.AmrError) as e:
        N.amr_step_patch_noalloc(cfg, d.data_ptr(), d.data_ptr(), 1e-3)
    assert e.value.status == N.AMR_ERR_ARG


def test_noalloc_cfl_step_and_glm_mhd_match_handle_path():
    """dt <= 0 (the CFL step of the input) and the nine-variable GLM-MHD system
    with the cleaning speed taken from the input state: the step size and the
    states of two calls in a row equal those of amr_step."""
    torch = pytest.importorskip("torch")
    from paper_0910_5547_gb300 import Solver
    from paper_0910_5547_gb300 import build as B
    from paper_0910_5547_gb300 import native as N
    B.build()
    for nvar, precision in ((5, "fp64"), (9, "fp64"), (9, "fp32")):
        base = (20, 16, 12)
        pb = ai.random_smooth([ai.Patch(0, (0, 0, 0), base)], base, nvar=nvar, seed=41, amp=0.2)
        s = Solver.from_problem(pb, precision=precision)
        u0 = s.state_all().copy()
        dts = [s.step(0.0)]
        u1 = s.state_all().copy()
        dts.append(s.step(0.0))
        u2 = s.state_all().copy()
        s.close()
        cfg = N.amr_default_config(nvar=nvar, precision=N.AMR_FP32 if precision == "fp32" else N.AMR_FP64,
                                   base_n=base, bc=(ai.PERIODIC,) * 6, gamma=pb.gamma)
        d_in = torch.tensor(u0, dtype=torch.float64, device="cuda")
        d_mid = torch.empty_like(d_in)
        d_out = torch.empty_like(d_in)
        got_dt = [N.amr_step_patch_noalloc(cfg, d_in.data_ptr(), d_mid.data_ptr(), 0.0),
                  N.amr_step_patch_noalloc(cfg, d_mid.data_ptr(), d_out.data_ptr(), -1.0)]
        torch.cuda.synchronize()
        rtol = 1e-14 if precision == "fp64" else 1e-6
        np.testing.assert_allclose(got_dt, dts, rtol=rtol)
        shape = (nvar, base[2], base[1], base[0])
        for got, want in ((d_mid.cpu().numpy(), u1), (d_out.cpu().numpy(), u2)):
            l1, mx = errors([got.reshape(shape)], [want.reshape(shape)], pb.patches)
            assert l1.max() <= TOL[precision]["l1"], (nvar, precision, l1)
            if "max" in TOL[precision]:
                assert mx.max() <= TOL[precision]["max"], (nvar, precision, mx)


def test_noalloc_rejects_overlapping_input_and_output():
    torch = pytest.importorskip("torch")
    from paper_0910_5547_gb300 import build as B
    from paper_0910_5547_gb300 import native as N
    B.build()
    base = (8, 8, 8)
    cfg = N.amr_default_config(base_n=base, bc=(1,) * 6)
    n = 5 * 8 * 8 * 8
    d = torch.ones(2 * n, dtype=torch.float64, device="cuda")
    for off in (0, 8, n - 1):      # same array, or ranges shifted by less than one state
        with pytest.raises(N.AmrError) as e:
            N.amr_step_patch_noalloc(cfg, d.data_ptr(), d.data_ptr() + 8 * off, 1e-3)
        assert e.value.status == N.AMR_ERR_ARG
