"""The second stream of a batched multi-level step (stage-2 parent gather and
prolongation beside stage 1, flux-register kernels beside the stages and the
finer levels) against one stream: the same states bit for bit, with graph
replay and eager launches, Euler and GLM-MHD, FP32 and FP64, periodic and
outflow, WENO3 face states, spanning blocks, and through regrids inside the
coarse step; also on the full static 4-level Sedov hierarchy."""
import numpy as np
import pytest

import amr_inputs as ai
from test_oracle_amr_mhd import three_level_seeded

pytestmark = pytest.mark.gpu

from paper_0910_5547_gb300 import Solver  # noqa: E402
from paper_0910_5547_gb300 import build as B  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    yield


def run(pb, steps, overlap, schedule=None, regrid_first=False, **kw):
    s = Solver.from_problem(pb, **kw)
    s.set_overlap(overlap)
    if regrid_first:
        s.step()
        s.regrid(threshold=0.1)
    if schedule is not None:
        s.set_regrid_schedule(schedule, threshold=0.1)
    for _ in range(steps):
        s.step()
    s.check()
    out = s.state_all().copy()
    patches = [(p.level, tuple(p.lo), tuple(p.n)) for p in s.patches]
    s.close()
    return patches, out


def same(a, b):
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1])


@pytest.mark.parametrize("nvar,precision", [(5, "fp32"), (5, "fp64"), (9, "fp32"), (9, "fp64")])
@pytest.mark.parametrize("bc", [ai.PERIODIC, ai.OUTFLOW])
def test_three_levels_side_stream_equals_one_stream(nvar, precision, bc):
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, nvar=nvar, seed=5, amp=0.2, bc=(bc,) * 6)
    same(run(pb, 3, True, precision=precision), run(pb, 3, False, precision=precision))
    same(run(pb, 2, True, precision=precision, use_graph=False),
         run(pb, 2, False, precision=precision, use_graph=False))


def test_weno3_and_patch_blocks():
    pb = ai.random_smooth(three_level_seeded(7), (32,) * 3, seed=9, amp=0.3)
    same(run(pb, 3, True, precision="fp32", recon="weno3"), run(pb, 3, False, precision="fp32", recon="weno3"))
    same(run(pb, 3, True, precision="fp32", item_span="patch"), run(pb, 3, False, precision="fp32", item_span="patch"))


@pytest.mark.parametrize("bc", [ai.PERIODIC, ai.OUTFLOW])
def test_scheduled_regrids_inside_the_step(bc):
    patches = ai.uniform_patches((32,) * 3, (16,) * 3)
    pb = ai.random_smooth(patches, (32,) * 3, seed=12, amp=0.6, bc=(bc,) * 6)
    a = run(pb, 2, True, schedule=1, regrid_first=True, precision="fp64", max_level=3)
    b = run(pb, 2, False, schedule=1, regrid_first=True, precision="fp64", max_level=3)
    same(a, b)
    assert max(p[0] for p in a[0]) >= 2


def test_sedov_four_levels():
    pb = ai.sedov_amr()
    same(run(pb, 2, True, precision="fp32"), run(pb, 2, False, precision="fp32"))
