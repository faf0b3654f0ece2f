"""Stages that read same-level ghost layers straight from the neighbouring patch
(ghost_fill = direct, the default) against stages that read ghost cells copied
into every patch first (ghost_fill = copy): the same states bit for bit, on
hierarchies that mix sibling faces, periodic self-images, outflow faces,
coarse-fine faces and faces the flux registers read, for both physics, both
precisions, both reconstructions, batched and plain launches, tilings whose
z chunks end inside a patch, and through mid-step rebuilds."""
import numpy as np
import pytest

import amr_inputs as ai
from test_oracle_amr_mhd import three_level_seeded, two_level

pytestmark = pytest.mark.gpu

from paper_0910_5547_gb300 import Solver  # noqa: E402
from paper_0910_5547_gb300 import build as B  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    yield


def run(pb, steps, tiling=None, **kw):
    out = []
    for mode in ("direct", "copy"):
        s = Solver.from_problem(pb, ghost_fill=mode, **kw)
        if tiling:
            s.set_tiling(*tiling)
        for _ in range(steps):
            s.step(0.0)
        s.check()
        out.append(s.state_all().copy())
        s.close()
    return out


def same(a, b):
    assert a.shape == b.shape
    assert np.array_equal(a, b), np.abs(a - b).max()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("bc", [ai.PERIODIC, ai.OUTFLOW])
def test_three_level_euler(precision, bc):
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, seed=5, amp=0.2, bc=(bc,) * 6)
    same(*run(pb, 2, precision=precision))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_three_level_glm_mhd_and_plain_launches(precision):
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, nvar=9, seed=8, amp=0.2)
    same(*run(pb, 2, precision=precision))
    same(*run(pb, 1, precision=precision, batched=False, use_graph=False))


@pytest.mark.parametrize("tiling", [(32, 256, 32, 0), (16, 128, 5, 0), (8, 256, 3, 0)])
def test_single_periodic_patch_and_tilings(tiling):
    pb = ai.kelvin_helmholtz(N=48, tile=None)
    same(*run(pb, 3, tiling=tiling, precision="fp32"))


def test_mixed_boundaries_and_weno3():
    pb = ai.random_smooth(two_level(), (16,) * 3, seed=9, amp=0.2, bc=(ai.PERIODIC, ai.PERIODIC, ai.OUTFLOW,
                                                                         ai.OUTFLOW, ai.PERIODIC, ai.PERIODIC))
    same(*run(pb, 2, precision="fp64"))
    same(*run(pb, 2, precision="fp32", recon="weno3"))


def test_sedov_hierarchy_ragged_patches():
    pb = ai.sedov_amr(base=32, sides=(32, 32), seed=3)
    same(*run(pb, 2, precision="fp32"))


def test_mid_step_rebuilds():
    pb = ai.blast_clumps(base=16, levels=3, side=16, seed=4)
    out = []
    for mode in ("direct", "copy"):
        s = Solver.from_problem(pb, precision="fp32", ghost_fill=mode)
        s.set_regrid_schedule(pb.max_level - 2, threshold=0.3, buffer=2, block=4, max_patch=16)
        for _ in range(2):
            s.step(0.0)
        s.check()
        out.append((s.state_all().copy(), [(p.level, tuple(p.lo), tuple(p.n)) for p in s.patches]))
        s.close()
    assert out[0][1] == out[1][1]
    same(out[0][0], out[1][0])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_coarse_fine_faces_on_coarse_patch_boundaries(precision):
    """A fine block whose footprint is exactly one coarse patch: every coarse-fine
    face lies on a face of a neighbouring coarse patch, so the coarse-side flux
    register stencils reach into those patches' ghost cells (those faces must
    keep copied ghost cells)."""
    patches = ai.uniform_patches((16, 16, 16), (8, 8, 8))
    patches += [ai.Patch(1, (x, y, z), (8, 8, 8)) for z in (16, 24) for y in (16, 24) for x in (16, 24)]
    pb = ai.random_smooth(patches, (16,) * 3, seed=12, amp=0.2)
    same(*run(pb, 3, precision=precision))
    pb9 = ai.random_smooth(patches, (16,) * 3, nvar=9, seed=13, amp=0.2)
    same(*run(pb9, 2, precision=precision))
