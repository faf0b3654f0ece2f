"""GPU parity against the FP64 oracle on the edge cases of the patch geometry:
a periodic slab two cells thick (a patch is its own periodic image), the
largest patch edge (1024 cells), ragged level-0 patches of 2-6 cells, an
anisotropic box (different dx per axis), and fine patches on both sides of a
periodic boundary and against an outflow face.  Tolerances of tests/parity.py."""
import dataclasses

import numpy as np
import pytest

import amr_inputs as ai
import oracle as orc
from parity import assert_parity

pytestmark = pytest.mark.gpu

from paper_0910_5547_gb300 import Solver  # noqa: E402
from paper_0910_5547_gb300 import build as B  # noqa: E402
from paper_0910_5547_gb300 import native as N  # noqa: E402

P, O = ai.PERIODIC, ai.OUTFLOW


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    N.load()
    yield


def _run(pb, precision, steps=3, **kw):
    o = orc.Oracle(pb, nthreads=8, **kw)
    s = Solver.from_problem(pb, precision=precision, **kw)
    for _ in range(steps):
        o.step(0.0)
        s.step(0.0)
    s.check()
    return o, s


def _ragged(n, sizes):
    cuts = [0]
    i = 0
    while cuts[-1] < n:
        cuts.append(min(n, cuts[-1] + sizes[i % len(sizes)]))
        i += 1
    out = []
    for z0, z1 in zip(cuts[:-1], cuts[1:]):
        for y0, y1 in zip(cuts[:-1], cuts[1:]):
            for x0, x1 in zip(cuts[:-1], cuts[1:]):
                out.append(ai.Patch(0, (x0, y0, z0), (x1 - x0, y1 - y0, z1 - z0)))
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_two_cell_thick_periodic_slab(precision):
    pb = ai.random_smooth(ai.uniform_patches((64, 2, 2), (16, 2, 2)), (64, 2, 2), seed=3)
    o, s = _run(pb, precision)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "slab 64x2x2")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_largest_patch_edge(precision):
    pb = ai.random_smooth([ai.Patch(0, (0, 0, 0), (1024, 8, 8))], (1024, 8, 8), seed=4)
    o, s = _run(pb, precision)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "1024x8x8 patch")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("bc", [P, O])
def test_ragged_patches_of_two_to_six_cells(precision, bc):
    pb = ai.random_smooth(_ragged(16, [2, 3, 5, 6]), (16, 16, 16), seed=5, bc=(bc,) * 6)
    o, s = _run(pb, precision)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "2-6 cell patches")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_anisotropic_box(precision):
    """base (24, 16, 12) on [0,3] x [0,1] x [0,0.75]: dx = (1/8, 1/16, 1/16)."""
    pb = ai.random_smooth(ai.uniform_patches((24, 16, 12), (10, 6, 5)), (24, 16, 12), seed=6, bc=(O,) * 6)
    pb = dataclasses.replace(pb, domain_lo=(0.0, 0.0, 0.0), domain_hi=(3.0, 1.0, 0.75))
    o = orc.Oracle(pb, nthreads=8)
    s = Solver.from_problem(pb, precision=precision)
    for _ in range(4):
        o.step(0.0)
        s.step(0.0)
    s.check()
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "anisotropic box")


def _edge_fine_patches(bc):
    """Level 0: 16^3 in 8^3 tiles.  Level 1 (32^3 index space): slabs x in [0, 8) and
    [24, 32), y and z in [8, 24) -- on a periodic box the two slabs are neighbours
    across the boundary; on an outflow box each touches an outflow face."""
    patches = ai.uniform_patches((16,) * 3, (8,) * 3)
    for x0 in (0, 24):
        for y0 in (8, 16):
            for z0 in (8, 16):
                patches.append(ai.Patch(1, (x0, y0, z0), (8, 8, 8)))
    return ai.random_smooth(patches, (16,) * 3, seed=8, bc=(bc,) * 6)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("bc", [P, O])
def test_fine_patches_at_the_domain_boundary(precision, bc):
    pb = _edge_fine_patches(bc)
    o, s = _run(pb, precision, steps=2)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, f"fine at boundary bc={bc}")
    if bc == P:   # conservation across the periodic coarse-fine boundaries
        so = Solver.from_problem(pb, precision="fp64")
        t0 = so.totals()
        for _ in range(2):
            so.step(0.0)
        t1 = so.totals()
        assert np.allclose(t1, t0, rtol=0.0, atol=1e-13 * np.max(np.abs(t0)))
