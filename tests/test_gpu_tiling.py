"""Every compiled build of the stage kernel (threads per CTA x register budget),
selected with amr_set_tiling, against the FP64 oracle: a three-level periodic
hierarchy and a single ragged outflow box whose x/y extents leave partial
tiles.  The 128-thread builds run with the largest tiles their shared-memory
strides allow (wx = 5, wy = 25: the widest plane, 9 x 29 cells, and x-state
array, 7 x 25).  Builds a precision/physics does not have, and bad shapes, are
rejected and leave the previous tiling in place.  Tolerances of tests/parity.py."""
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

# (columns per CTA, resident CTAs per SM) of every compiled build
BUILDS = {
    ("fp32", 5): [(256, 2), (256, 3), (128, 4)],
    ("fp32", 9): [(256, 1), (256, 2), (128, 2), (128, 3)],
    ("fp64", 5): [(256, 1), (256, 2), (128, 2)],
    ("fp64", 9): [(256, 1), (128, 2)],
}
CASES = sorted(BUILDS)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    N.load()
    yield


def _problems(nvar):
    amr = ai.random_smooth(three_level_seeded(), (32,) * 3, nvar=nvar, seed=21, amp=0.2)
    box = (37, 25, 11)   # 128 columns, max_wx 5: tiles of 5 x 25 (and 4 x 25)
    ragged = ai.random_smooth([ai.Patch(0, (0, 0, 0), box)], box, nvar=nvar, seed=22, amp=0.3,
                              bc=(ai.OUTFLOW,) * 6)
    return [("amr3", amr, 2), ("ragged", ragged, 3)]


def _reference(pb, steps):
    o = orc.Oracle(pb, nthreads=8)
    for _ in range(steps):
        o.step(0.0)
    return o


@pytest.mark.parametrize("precision,nvar", CASES)
def test_every_build_matches_the_oracle(precision, nvar):
    for label, pb, steps in _problems(nvar):
        o = _reference(pb, steps)
        want = o.all_cons()
        for cols, ctas in BUILDS[(precision, nvar)]:
            shapes = [(0, 0)] + ([(5, 7)] if cols == 128 else [(13, 5)])   # (max_wx, zchunk)
            for max_wx, zchunk in shapes:
                s = Solver.from_problem(pb, precision=precision)
                s.set_tiling(max_wx=max_wx, max_cols=cols, zchunk=zchunk, ctas_per_sm=ctas)
                for _ in range(steps):
                    s.step(0.0)
                s.check()
                assert_parity(s.all_cons(), want, pb.patches, precision,
                              f"{label} cols={cols} ctas={ctas} wx<={max_wx} z={zchunk}")
                s.close()


@pytest.mark.parametrize("precision,nvar", CASES)
def test_missing_builds_and_bad_shapes_are_rejected(precision, nvar):
    have = set(BUILDS[(precision, nvar)])
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, nvar=nvar, seed=23, amp=0.2)
    s = Solver.from_problem(pb, precision=precision)
    ref = Solver.from_problem(pb, precision=precision)
    cols0, ctas0 = BUILDS[(precision, nvar)][-1]
    s.set_tiling(max_wx=8, max_cols=cols0, zchunk=4, ctas_per_sm=ctas0)
    ref.set_tiling(max_wx=8, max_cols=cols0, zchunk=4, ctas_per_sm=ctas0)
    bad = [dict(max_cols=c, ctas_per_sm=k) for c in (256, 128) for k in range(1, 6) if (c, k) not in have]
    bad += [dict(max_wx=33), dict(max_wx=-1), dict(max_cols=200), dict(max_cols=64), dict(zchunk=-1),
            dict(ctas_per_sm=-1)]
    for kw in bad:
        with pytest.raises(N.AmrError) as e:
            s.set_tiling(**kw)
        assert e.value.status == N.AMR_ERR_ARG, kw
    for _ in range(2):   # the rejected calls changed nothing: same result as the untouched solver
        s.step(0.0)
        ref.step(0.0)
    for a, b in zip(s.all_cons(), ref.all_cons()):
        assert np.array_equal(a, b)
    s.close()
    ref.close()


def test_tiling_set_before_the_hierarchy_applies_to_it():
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, nvar=9, seed=24, amp=0.2)
    cfg = N.amr_default_config(nvar=9, precision=N.AMR_FP32, base_n=pb.base_n, bc=pb.bc, gamma=pb.gamma,
                               max_level=pb.max_level)
    h = N.amr_create(cfg)
    N.amr_set_tiling(h, 5, 128, 7, 3)
    N.amr_set_patches(h, pb.patches, pb.prim)
    o = _reference(pb, 2)
    for _ in range(2):
        N.amr_step(h, 0.0)
    got = [N.amr_get_state(h, i, (9, p.n[2], p.n[1], p.n[0])) for i, p in enumerate(pb.patches)]
    assert_parity(got, o.all_cons(), pb.patches, "fp32", "tiling-before-patches")
    N.amr_destroy(h)
