"""Pins of the oracle's regridding (no GPU): conservation, idempotence,
exact prolongation of a uniform state, flagged cells covered, proper nesting."""
import numpy as np
import pytest

import amr_inputs as ai
import oracle as orc
from oracle import regrid as rg


def _clumpy(n=32, seed=3, bc=ai.PERIODIC):
    patches = ai.uniform_patches((n,) * 3, (16,) * 3)
    pb = ai.random_smooth(patches, (n,) * 3, seed=seed, amp=0.6, bc=(bc,) * 6)
    return pb


def test_regrid_conserves_totals_and_covers_flags():
    pb = _clumpy()
    o = orc.Oracle(pb, max_level=2)
    o.step()
    t0 = o.totals()
    fl = rg.flags(o, 0.1)
    assert 0 < sum(int(f.sum()) for f in fl) < sum(f.size for f in fl)
    o2 = rg.regrid(o, threshold=0.1)
    assert any(p.level == 1 for p in o2.patches)
    assert np.all(np.abs(o2.totals() - t0) <= 1e-13 * np.abs(t0).max())
    # every flagged level-0 cell lies under a level-1 patch
    for p, f in zip(o.patches, fl):
        for (k, j, i) in zip(*np.nonzero(f)):
            g = (2 * (p.lo[0] + i), 2 * (p.lo[1] + j), 2 * (p.lo[2] + k))
            assert any(q.level == 1 and all(q.lo[d] <= g[d] < q.lo[d] + q.n[d] for d in range(3))
                       for q in o2.patches)
    # a second regrid adds level 2 and keeps the totals
    o2.step()
    t1 = o2.totals()
    o3 = rg.regrid(o2, threshold=0.1)
    assert max(p.level for p in o3.patches) == 2
    assert np.all(np.abs(o3.totals() - t1) <= 1e-13 * np.abs(t1).max())


def test_regrid_of_a_uniform_state_is_exact_and_unrefined():
    pb = ai.uniform(ai.uniform_patches((16,) * 3, (8,) * 3), (16,) * 3)
    o = orc.Oracle(pb, max_level=2)
    o2 = rg.regrid(o)
    assert [p.level for p in o2.patches] == [0] * 8          # no gradient, no refinement
    for a, b in zip(o.all_cons(), o2.all_cons()):
        assert np.array_equal(a, b)


def test_new_fine_cells_of_a_uniform_parent_are_uniform():
    # refinement forced by a density step in x; far from it the new cells equal the parent exactly
    pb = ai.sod(n=32)
    o = orc.Oracle(pb, max_level=1)
    o2 = rg.regrid(o)
    fine = [i for i, p in enumerate(o2.patches) if p.level == 1]
    assert fine
    for i in fine:
        u = o2.cons(i)
        p = o2.patches[i]
        x = (np.arange(p.n[0]) + p.lo[0] + 0.5) / 64
        far = np.abs(x - 0.5) > 2.5 / 32
        left = far & (x < 0.5)
        assert np.all(u[0][:, :, left] == 1.0)


def test_regrid_is_idempotent_on_an_unchanged_state():
    pb = _clumpy(seed=8)
    o = orc.Oracle(pb, max_level=1)
    o.step()
    o2 = rg.regrid(o, threshold=0.1)
    o3 = rg.regrid(o2, threshold=0.1)
    assert o3.patches == o2.patches
    for a, b in zip(o2.all_cons(), o3.all_cons()):
        assert np.array_equal(a, b)


def test_regridded_hierarchies_are_properly_nested():
    pb = _clumpy(seed=11, bc=ai.OUTFLOW)
    o = orc.Oracle(pb, max_level=3)
    for _ in range(3):
        o.step()
        o = rg.regrid(o, threshold=0.1)
    from paper_0910_5547_gb300 import build as B
    from paper_0910_5547_gb300 import native as N
    B.build()
    c = N.amr_default_config(base_n=(32,) * 3, max_level=3, bc=(ai.OUTFLOW,) * 6)
    st, msg = N.amr_validate_patches(c, o.patches)
    assert st == N.AMR_OK, msg
    assert max(p.level for p in o.patches) >= 2


def _validate(patches, bc, n=32, max_level=3):
    from paper_0910_5547_gb300 import build as B
    from paper_0910_5547_gb300 import native as N
    B.build()
    c = N.amr_default_config(base_n=(n,) * 3, max_level=max_level, bc=(bc,) * 6)
    return N.amr_validate_patches(c, patches)


@pytest.mark.parametrize("bc", [ai.PERIODIC, ai.OUTFLOW])
def test_midstep_regrid_conserves_and_nests(bc):
    """Sec. 3 recursion with the finer levels rebuilt after every step of levels
    <= 1: the rebuilds happen after each level-1 step (twice per coarse step) and
    each level-0 step, the totals hold to round-off (periodic) and every
    hierarchy met along the way is properly nested."""
    pb = _clumpy(seed=12, bc=bc)
    o = orc.Oracle(pb, max_level=3)
    o.step()
    o = rg.regrid(o, threshold=0.1)
    t0 = o.totals()
    rg.set_regrid_schedule(o, 1, threshold=0.1)
    for _ in range(2):
        o.step()
    assert [lv for lv, _ in o.regrid_log] == [1, 1, 0, 1, 1, 0]
    if bc == ai.PERIODIC:
        assert np.all(np.abs(o.totals() - t0) <= 1e-13 * np.abs(t0).max())
    for _, pl in o.regrid_log:
        st, msg = _validate(pl, bc)
        assert st == 0, msg
    assert max(p.level for p in o.patches) >= 2


def test_midstep_regrid_of_a_uniform_state_changes_nothing():
    pb = ai.uniform(ai.uniform_patches((16,) * 3, (8,) * 3), (16,) * 3)
    o = orc.Oracle(pb, max_level=2)
    u0 = o.all_cons()
    rg.set_regrid_schedule(o, 1)
    o.step(0.01)
    assert [p.level for p in o.patches] == [0] * 8
    for a, b in zip(u0, o.all_cons()):
        assert np.array_equal(a, b)


def test_removed_schedule_is_a_plain_step():
    pb = _clumpy(seed=13)
    runs = []
    for sched in (False, True):
        o = orc.Oracle(pb, max_level=2)
        o.step()
        o = rg.regrid(o, threshold=0.1)
        if sched:
            rg.set_regrid_schedule(o, 1, threshold=0.1)
            rg.set_regrid_schedule(o, -1)
        o.step()
        runs.append(o.all_cons())
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
