"""Batched stage blocks that span the patches of a z-layer (item_span = layers,
the default: the patches of a level with one z range that tile a rectangle are
cut into column blocks as one region) against blocks that stay inside one
patch (item_span = patch): the same states bit for bit, with seeded 8-32
patches on nested levels, both physics and precisions, WENO3 face states,
periodic and outflow boxes, persistent launches, tilings of 128 and 256
columns, and through mid-step rebuilds."""
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


def run(pb, steps, tiling=None, persistent=None, **kw):
    out = []
    for mode in ("layers", "patch"):
        s = Solver.from_problem(pb, item_span=mode, **kw)
        if tiling:
            s.set_tiling(*tiling)
        if persistent is not None:
            s.set_persistent(persistent)
        for _ in range(steps):
            s.step(0.0)
        s.check()
        out.append(s.state_all().copy())
        s.close()
    assert np.array_equal(out[0], out[1]), np.abs(out[0] - out[1]).max()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("bc", [ai.PERIODIC, ai.OUTFLOW])
def test_nested_seeded_patches_euler(precision, bc):
    pb = ai.random_smooth(ai.nested_cubes(48, (48, 48), seed=7), (48,) * 3, seed=3, amp=0.2, bc=(bc,) * 6)
    run(pb, 2, precision=precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_glm_mhd_and_weno3(precision):
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, nvar=9, seed=8, amp=0.2)
    run(pb, 2, precision=precision)
    pe = ai.random_smooth(ai.nested_cubes(48, (48,), seed=9), (48,) * 3, seed=4, amp=0.2)
    run(pe, 2, precision=precision, recon="weno3")


@pytest.mark.parametrize("tiling,persistent", [((32, 256, 32, 0), 1), ((16, 128, 16, 0), 0), ((8, 256, 5, 0), 0)])
def test_tilings_and_launch_forms(tiling, persistent):
    pb = ai.sedov_amr(base=48, sides=(48, 48), seed=5)
    run(pb, 2, tiling=tiling, persistent=persistent, precision="fp32")


def test_mid_step_rebuilds():
    pb = ai.blast_clumps(base=32, levels=3, side=32, seed=6)
    out = []
    for mode in ("layers", "patch"):
        s = Solver.from_problem(pb, precision="fp32", item_span=mode)
        s.set_regrid_schedule(pb.max_level - 2, threshold=0.3, buffer=2, block=4, max_patch=16)
        for _ in range(2):
            s.step(0.0)
        s.check()
        out.append(s.state_all().copy())
        s.close()
    assert np.array_equal(out[0], out[1])
