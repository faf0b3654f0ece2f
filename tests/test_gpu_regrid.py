"""GPU regridding against the oracle's independent regrid: identical patch lists
(integer work, exact) and FP64 states within the parity tolerance, across
regrid -> step -> regrid cycles; FP32 regrid conserves totals."""
import numpy as np
import pytest

import amr_inputs as ai
import oracle as orc
from oracle import regrid as rg
from parity import assert_parity

pytestmark = pytest.mark.gpu

from paper_0910_5547_gb300 import Solver  # noqa: E402
from paper_0910_5547_gb300 import build as B  # noqa: E402
from paper_0910_5547_gb300 import native as N  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    yield


def clumpy(seed, bc):
    patches = ai.uniform_patches((32,) * 3, (16,) * 3)
    return ai.random_smooth(patches, (32,) * 3, seed=seed, amp=0.6, bc=(bc,) * 6)


@pytest.mark.parametrize("bc", [ai.PERIODIC, ai.OUTFLOW])
def test_regrid_cycles_match_the_oracle_fp64(bc):
    pb = clumpy(3, bc)
    o = orc.Oracle(pb, max_level=2, nthreads=8)
    s = Solver.from_problem(pb, precision="fp64", max_level=2)
    for cycle in range(3):
        for _ in range(2):
            o.step()
            s.step()
        o = rg.regrid(o, threshold=0.1, buffer=2, block=4, max_patch=32)
        s.regrid(threshold=0.1, buffer=2, block=4, max_patch=32)
        assert [(p.level, tuple(p.lo), tuple(p.n)) for p in s.patches] == \
               [(p.level, tuple(p.lo), tuple(p.n)) for p in o.patches], f"cycle {cycle}"
        assert_parity(s.all_cons(), o.all_cons(), o.patches, "fp64", f"regrid cycle {cycle}")
    assert max(p.level for p in s.patches) == 2
    o.step()
    s.step()
    s.check()
    assert_parity(s.all_cons(), o.all_cons(), o.patches, "fp64", "after regrid")


def test_regrid_fp32_conserves_totals_and_nests():
    pb = clumpy(5, ai.PERIODIC)
    s = Solver.from_problem(pb, precision="fp32", max_level=3)
    for _ in range(3):
        s.step()
        t0 = s.totals()
        n = s.regrid(threshold=0.1)
        t1 = s.totals()
        assert n == len(s.patches)
        assert np.all(np.abs(t1 - t0) <= 2e-6 * np.abs(t0).max()), (t0, t1)
    c = N.amr_default_config(base_n=(32,) * 3, max_level=3, bc=(ai.PERIODIC,) * 6)
    assert N.amr_validate_patches(c, s.patches)[0] == N.AMR_OK
    s.step()
    s.check()


def test_regrid_rejects_bad_parameters():
    pb = clumpy(5, ai.PERIODIC)
    s = Solver.from_problem(pb, precision="fp32", max_level=1)
    with pytest.raises(N.AmrError) as e:
        s.regrid(block=3)
    assert e.value.status == N.AMR_ERR_ARG


@pytest.mark.parametrize("bc", [ai.PERIODIC, ai.OUTFLOW])
def test_scheduled_midstep_regrid_matches_the_oracle_fp64(bc):
    """Finer levels rebuilt after every step of levels <= 1 inside each coarse step
    (Sec. 3 recursion): after every coarse step the GPU hierarchy equals the oracle's
    (exact) and the state matches within the FP64 parity tolerance."""
    pb = clumpy(12, bc)
    o = orc.Oracle(pb, max_level=3, nthreads=8)
    s = Solver.from_problem(pb, precision="fp64", max_level=3)
    o.step()
    s.step()
    o = rg.regrid(o, threshold=0.1)
    s.regrid(threshold=0.1)
    rg.set_regrid_schedule(o, 1, threshold=0.1)
    s.set_regrid_schedule(1, threshold=0.1)
    for k in range(2):
        o.step()
        s.step()
        assert [(p.level, tuple(p.lo), tuple(p.n)) for p in s.patches] == \
               [(p.level, tuple(p.lo), tuple(p.n)) for p in o.patches], f"coarse step {k}"
        assert_parity(s.all_cons(), o.all_cons(), o.patches, "fp64", f"scheduled regrid, coarse step {k}")
    assert len(o.regrid_log) == 6
    assert max(p.level for p in s.patches) >= 2
    ph = N.amr_get_regrid_timing(s.h)
    assert ph["cluster"] > 0.0 and ph["plan"] > 0.0
    s.check()


def test_scheduled_regrid_fp32_conserves_and_nests():
    pb = clumpy(14, ai.PERIODIC)
    s = Solver.from_problem(pb, precision="fp32", max_level=3)
    s.step()
    s.regrid(threshold=0.1)
    s.set_regrid_schedule(1, threshold=0.1)
    t0 = s.totals()
    for _ in range(2):
        s.step()
        c = N.amr_default_config(base_n=(32,) * 3, max_level=3, bc=(ai.PERIODIC,) * 6)
        assert N.amr_validate_patches(c, s.patches)[0] == N.AMR_OK
    t1 = s.totals()
    assert np.all(np.abs(t1 - t0) <= 2e-6 * np.abs(t0).max()), (t0, t1)
    s.set_regrid_schedule(-1)
    s.step()
    s.check()


def test_regrid_schedule_rejects_bad_parameters():
    s = Solver.from_problem(clumpy(3, ai.PERIODIC), precision="fp32", max_level=2)
    with pytest.raises(N.AmrError):
        s.set_regrid_schedule(1, block=3)
    with pytest.raises(N.AmrError):
        s.set_regrid_schedule(1, threshold=0.0)
    s.set_regrid_schedule(-1)
    s.step()
    s.check()


@pytest.mark.parametrize("bc", [ai.PERIODIC, ai.OUTFLOW])
def test_block_tags_on_gpu_and_byte_flags_agree(bc):
    """The regrid tags blocks on the GPU when every flagged level's block grid fits
    a 2^28-bit map, else downloads one byte per cell and tags on the host.  With
    max_level 12 the deep levels' grids exceed that (host path); with max_level 3
    they do not (GPU path).  The same flags then give the same new hierarchy and
    the same filled state, and both agree with the oracle."""
    pb = clumpy(7, bc)
    runs = []
    for ml in (3, 12):
        s = Solver.from_problem(pb, precision="fp64", max_level=ml)
        s.step(0.002)
        s.regrid(threshold=0.1, buffer=2, block=2, max_patch=16, min_level=0)
        s.check()
        runs.append(([(p.level, tuple(p.lo), tuple(p.n)) for p in s.patches], s.all_cons()))
    assert runs[0][0] == runs[1][0]
    assert max(p[0] for p in runs[0][0]) == 1
    for a, b in zip(runs[0][1], runs[1][1]):
        assert np.array_equal(a, b)
    o = orc.Oracle(pb, max_level=3, nthreads=8)
    o.step(0.002)
    o = rg.regrid(o, threshold=0.1, buffer=2, block=2, max_patch=16)
    assert runs[0][0] == [(p.level, tuple(p.lo), tuple(p.n)) for p in o.patches]


@pytest.mark.parametrize("bc", [ai.PERIODIC, ai.OUTFLOW])
@pytest.mark.parametrize("block,buffer", [(2, 0), (2, 2), (8, 0), (8, 8)])
def test_block_and_buffer_sizes_match_the_oracle(bc, block, buffer):
    """The GPU's block tags, parent rings and refinable sets for other block and
    buffer sizes: the same three-level hierarchy as the oracle's clustering, and
    the refilled state within the FP64 parity tolerance."""
    pb = clumpy(21, bc)
    o = orc.Oracle(pb, max_level=2, nthreads=8)
    s = Solver.from_problem(pb, precision="fp64", max_level=2)
    kw = dict(threshold=0.1, buffer=buffer, block=block, max_patch=4 * block)
    for cycle in range(2):
        o.step()
        s.step()
        o = rg.regrid(o, **kw)
        s.regrid(**kw)
        assert [(p.level, tuple(p.lo), tuple(p.n)) for p in s.patches] == \
               [(p.level, tuple(p.lo), tuple(p.n)) for p in o.patches], f"cycle {cycle}"
        assert_parity(s.all_cons(), o.all_cons(), o.patches, "fp64", f"regrid block {block} buffer {buffer}")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mhd_regrid_matches_the_oracle_with_div_b(precision):
    """GLM-MHD on a regridded hierarchy: the same patches as the oracle's regrid,
    the refilled and stepped state within the parity tolerance, and the div B
    norms of the new hierarchy alike."""
    patches = ai.uniform_patches((32,) * 3, (16,) * 3)
    pb = ai.random_smooth(patches, (32,) * 3, nvar=9, gamma=5.0 / 3.0, seed=13, amp=0.6)
    o = orc.Oracle(pb, max_level=2, nthreads=8, ch=1.5)
    s = Solver.from_problem(pb, precision=precision, max_level=2, ch=1.5)
    kw = dict(threshold=0.1, buffer=2, block=4, max_patch=32)
    for cycle in range(2):
        o.step(0.002)
        s.step(0.002)
        o = rg.regrid(o, **kw)
        s.regrid(**kw)
        assert [(p.level, tuple(p.lo), tuple(p.n)) for p in s.patches] == \
               [(p.level, tuple(p.lo), tuple(p.n)) for p in o.patches], f"cycle {cycle}"
    o.step(0.002)
    s.step(0.002)
    s.check()
    assert max(p.level for p in s.patches) >= 1
    assert_parity(s.all_cons(), o.all_cons(), o.patches, precision, "mhd regrid")
    want, got = o.divb_norms(), s.divb_norms()
    if precision == "fp64":
        assert np.allclose(got, want, rtol=1e-10, atol=1e-12 * want[2])
    else:
        assert abs(got[0] - want[0]) <= 2e-5 * want[2] and np.allclose(got[2:], want[2:], rtol=2e-6)


def test_flux_reconstruction_regrid_matches_the_oracle():
    pb = clumpy(17, ai.PERIODIC)
    o = orc.Oracle(pb, max_level=2, nthreads=8, riemann=orc.FLUXREC)
    s = Solver.from_problem(pb, precision="fp64", max_level=2, riemann="fluxrec")
    kw = dict(threshold=0.1, buffer=2, block=4, max_patch=32)
    for cycle in range(2):
        o.step()
        s.step()
        o = rg.regrid(o, **kw)
        s.regrid(**kw)
        assert [(p.level, tuple(p.lo), tuple(p.n)) for p in s.patches] == \
               [(p.level, tuple(p.lo), tuple(p.n)) for p in o.patches], f"cycle {cycle}"
        assert_parity(s.all_cons(), o.all_cons(), o.patches, "fp64", f"fluxrec regrid {cycle}")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_weno3_scheduled_midstep_regrid_matches_the_oracle(precision):
    """Third-order WENO face states through the mid-step rebuilds of a regrid
    schedule (finer levels rebuilt after every step of levels <= 1): the same
    hierarchies as the oracle's, and the states within the parity tolerance."""
    pb = clumpy(21, ai.PERIODIC)
    o = orc.Oracle(pb, max_level=3, nthreads=8, recon=orc.WENO3)
    s = Solver.from_problem(pb, precision=precision, max_level=3, recon="weno3")
    o.step()
    s.step()
    o = rg.regrid(o, threshold=0.1)
    s.regrid(threshold=0.1)
    rg.set_regrid_schedule(o, 1, threshold=0.1)
    s.set_regrid_schedule(1, threshold=0.1)
    for k in range(2):
        dt = o.step()
        s.step(dt)
        assert [(p.level, tuple(p.lo), tuple(p.n)) for p in s.patches] == \
               [(p.level, tuple(p.lo), tuple(p.n)) for p in o.patches], f"coarse step {k}"
        assert_parity(s.all_cons(), o.all_cons(), o.patches, precision, f"weno3 scheduled regrid {k}")
    assert max(p.level for p in s.patches) >= 2
    s.check()
