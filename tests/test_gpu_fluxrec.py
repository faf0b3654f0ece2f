"""GPU parity of the direct flux reconstruction variant (riemann = AMR_FLUXREC,
Euler) against the FP64 oracle with the same reading (tests/test_oracle_fluxrec.py
pins it): Sod to t = 0.2, a tiled Kelvin-Helmholtz box, a three-level periodic
hierarchy (with conservation), batched vs plain bitwise, the allocation-free
entry point, and the rejection of GLM-MHD.  Tolerances of tests/parity.py."""
import numpy as np
import pytest

import amr_inputs as ai
import oracle as orc
from parity import TOL, assert_parity, errors
from test_oracle_amr_mhd import three_level_seeded

pytestmark = pytest.mark.gpu

from paper_0910_5547_gb300 import Solver  # noqa: E402
from paper_0910_5547_gb300 import build as B  # noqa: E402
from paper_0910_5547_gb300 import native as N  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    N.load()
    yield


def _pair(pb, precision, steps=None, t_end=None, **kw):
    o = orc.Oracle(pb, nthreads=8, riemann=orc.FLUXREC)
    s = Solver.from_problem(pb, precision=precision, riemann="fluxrec", **kw)
    if t_end is not None:
        assert o.run_to(t_end) == s.run_to(t_end)
    else:
        for _ in range(steps):
            o.step(0.0)
            s.step(0.0)
    s.check()
    return o, s


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sod_to_t02(precision):
    pb = ai.sod(n=32)
    o, s = _pair(pb, precision, t_end=0.2)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "sod-fluxrec")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_kelvin_helmholtz_tiled(precision):
    pb = ai.kelvin_helmholtz(N=64, tile=16)
    o, s = _pair(pb, precision, steps=5)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "kh64-fluxrec")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_three_level_periodic_hierarchy(precision):
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, seed=9, amp=0.3)
    o, s = _pair(pb, precision, steps=2)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "amr-fluxrec")
    if precision == "fp64":
        t0 = Solver.from_problem(pb, precision="fp64", riemann="fluxrec").totals()
        t1 = s.totals()
        assert np.allclose(t1, t0, rtol=0.0, atol=2e-14 * np.abs(t0).max())


def test_batched_and_plain_are_bitwise_equal():
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, seed=4, amp=0.3)
    a = Solver.from_problem(pb, precision="fp32", riemann="fluxrec", batched=True)
    b = Solver.from_problem(pb, precision="fp32", riemann="fluxrec", batched=False, use_graph=False)
    for _ in range(2):
        a.step(0.0)
        b.step(0.0)
    for x, y in zip(a.all_cons(), b.all_cons()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_entry_point(precision):
    torch = pytest.importorskip("torch")
    base = (24, 20, 16)
    pb = ai.random_smooth([ai.Patch(0, (0, 0, 0), base)], base, seed=31, amp=0.3, bc=(ai.OUTFLOW,) * 6)
    s = Solver.from_problem(pb, precision=precision, riemann="fluxrec")
    u0 = s.state_all().copy()
    dt = 0.5 * s.cfl_dt()
    s.step(dt)
    u1 = s.state_all().copy()
    s.close()
    cfg = N.amr_default_config(nvar=5, precision=N.AMR_FP32 if precision == "fp32" else N.AMR_FP64,
                               base_n=base, bc=(ai.OUTFLOW,) * 6, gamma=pb.gamma, riemann=N.AMR_FLUXREC)
    d_in = torch.tensor(u0, dtype=torch.float64, device="cuda")
    d_out = torch.empty_like(d_in)
    torch.cuda.synchronize()
    N.amr_step_patch_noalloc(cfg, d_in.data_ptr(), d_out.data_ptr(), dt)
    torch.cuda.synchronize()
    shape = (5, base[2], base[1], base[0])
    l1, _ = errors([d_out.cpu().numpy().reshape(shape)], [u1.reshape(shape)], pb.patches)
    assert l1.max() <= TOL[precision]["l1"], l1


def test_mhd_is_rejected():
    pb = ai.orszag_tang(N=16, tile=8)
    with pytest.raises(N.AmrError) as e:
        Solver.from_problem(pb, precision="fp32", riemann="fluxrec")
    assert e.value.status == N.AMR_ERR_ARG
