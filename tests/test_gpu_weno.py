"""GPU parity of the third-order WENO face states (recon = AMR_WENO3) against
the FP64 oracle with the same reading (tests/test_oracle_weno.py pins it): Sod
to t = 0.2 (HLL and LLF), a tiled Kelvin-Helmholtz box, three-level periodic
hierarchies for Euler and GLM-MHD (with conservation), Orszag-Tang; batched vs
plain bitwise; the WENO3 build under a 128-column tiling; the rejections
(WENO3 with flux reconstruction, the allocation-free path).  Tolerances of
tests/parity.py."""
import numpy as np
import pytest

import amr_inputs as ai
import oracle as orc
from parity import assert_parity
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


def _pair(pb, precision, steps=None, t_end=None, riemann="hll", **kw):
    o = orc.Oracle(pb, nthreads=8, recon=orc.WENO3, riemann={"hll": orc.HLL, "llf": orc.LLF}[riemann])
    s = Solver.from_problem(pb, precision=precision, recon="weno3", riemann=riemann, **kw)
    if t_end is not None:
        assert o.run_to(t_end) == s.run_to(t_end)
    else:
        for _ in range(steps):
            o.step(0.0)
            s.step(0.0)
    s.check()
    return o, s


@pytest.mark.parametrize("riemann", ["hll", "llf"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sod_to_t02(precision, riemann):
    pb = ai.sod(n=32)
    o, s = _pair(pb, precision, t_end=0.2, riemann=riemann)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, f"sod-weno3-{riemann}")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_kelvin_helmholtz_tiled(precision):
    pb = ai.kelvin_helmholtz(N=64, tile=16)
    o, s = _pair(pb, precision, steps=5)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "kh64-weno3")


@pytest.mark.parametrize("nvar", [5, 9])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_three_level_periodic_hierarchy(precision, nvar):
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, nvar=nvar, seed=12, amp=0.25)
    t0 = Solver.from_problem(pb, precision="fp64", recon="weno3").totals()
    o, s = _pair(pb, precision, steps=2)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, f"amr3-weno3-{nvar}")
    if precision == "fp64":
        t1 = s.totals()
        keep = slice(0, 5) if nvar == 5 else slice(0, 8)   # psi is not conserved under cleaning
        assert np.allclose(t1[keep], t0[keep], rtol=0.0, atol=2e-14 * np.abs(t0).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_orszag_tang(precision):
    pb = ai.orszag_tang(N=32, tile=16)
    o, s = _pair(pb, precision, steps=4)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "ot32-weno3")


def test_batched_and_plain_are_bitwise_equal():
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, seed=13, amp=0.3)
    a = Solver.from_problem(pb, precision="fp32", recon="weno3", batched=True)
    b = Solver.from_problem(pb, precision="fp32", recon="weno3", batched=False, use_graph=False)
    for _ in range(2):
        a.step(0.0)
        b.step(0.0)
    for x, y in zip(a.all_cons(), b.all_cons()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("nvar", [5, 9])
def test_128_column_tiling_runs_the_weno3_build(nvar):
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, nvar=nvar, seed=14, amp=0.2)
    o = orc.Oracle(pb, nthreads=8, recon=orc.WENO3)
    s = Solver.from_problem(pb, precision="fp32", recon="weno3")
    s.set_tiling(max_wx=5, max_cols=128, zchunk=7, ctas_per_sm=0)
    for _ in range(2):
        o.step(0.0)
        s.step(0.0)
    s.check()
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, "fp32", f"weno3-128cols-{nvar}")


def test_rejections():
    pb = ai.sod(n=16)
    with pytest.raises(N.AmrError) as e:
        Solver.from_problem(pb, precision="fp32", recon="weno3", riemann="fluxrec")
    assert e.value.status == N.AMR_ERR_ARG
    torch = pytest.importorskip("torch")
    base = (16, 16, 16)
    cfg = N.amr_default_config(nvar=5, precision=N.AMR_FP32, base_n=base, recon=N.AMR_WENO3)
    d_in = torch.ones(5 * 16 ** 3, dtype=torch.float64, device="cuda")
    d_out = torch.empty_like(d_in)
    with pytest.raises(N.AmrError) as e:
        N.amr_step_patch_noalloc(cfg, d_in.data_ptr(), d_out.data_ptr(), 1e-3)
    assert e.value.status == N.AMR_ERR_ARG
