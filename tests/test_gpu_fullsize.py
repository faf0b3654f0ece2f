"""Parity at the benchmark's full size (Kelvin-Helmholtz 256^3 periodic, 512
patches of 32^3, the launch configuration the benchmark times): one RK2 step on
the GPU, then sampled cells recomputed one by one by the oracle.  A cell after
one step depends only on the cells within four cells of it along the axes, so
the oracle advances a 9^3 neighbourhood (taken with periodic wrap) and its
centre is exact.  Conservation of every total is checked at full size too."""
import numpy as np
import pytest

import amr_inputs as ai
import oracle as orc
from parity import TOL

pytestmark = pytest.mark.gpu

from paper_0910_5547_gb300 import Solver  # noqa: E402
from paper_0910_5547_gb300 import build as B  # noqa: E402

N = 256
DT = 2.0e-4          # below the CFL limit 0.4 / (3 * 256 * (|v| + c)) ~ 2.2e-4
RNG = np.random.default_rng(99)


@pytest.fixture(scope="module")
def kh():
    B.build()
    pb = ai.kelvin_helmholtz(N=N, tile=32)
    W = np.empty((5, N, N, N))
    for p, w in zip(pb.patches, pb.prim):
        W[:, p.lo[2]:p.lo[2] + 32, p.lo[1]:p.lo[1] + 32, p.lo[0]:p.lo[0] + 32] = w
    return pb, W


def samples():
    pts = [(0, 0, 0), (31, 32, 33), (255, 128, 64), (64, 63, 64), (16, 191, 200), (100, 192, 31)]
    pts += [tuple(int(x) for x in RNG.integers(0, N, 3)) for _ in range(26)]
    return pts


def oracle_cell(W, x, y, z):
    idx = [np.arange(c - 4, c + 5) % N for c in (x, y, z)]
    sub = W[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]
    o = orc.Oracle(patches=[ai.Patch(0, (0, 0, 0), (9, 9, 9))], prim=[np.ascontiguousarray(sub)],
                   base_n=(9, 9, 9), domain_hi=(9.0 / N,) * 3, bc=(ai.OUTFLOW,) * 6, nvar=5, gamma=1.4)
    o.step(DT)
    return o.cons(0)[:, 4, 4, 4]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_kh256_one_step_sampled_cells(kh, precision):
    pb, W = kh
    s = Solver.from_problem(pb, precision=precision)
    t0 = s.totals()
    s.step(DT)
    s.check()
    flat = s.state_all()
    t1 = s.totals()
    per = 5 * 32 ** 3
    ref_scale = np.array([2.0, 0.5, 0.02, 0.02, 7.0])
    worst = 0.0
    for (x, y, z) in samples():
        pi = (z // 32) * 64 + (y // 32) * 8 + (x // 32)
        p = pb.patches[pi]
        assert p.lo == (x // 32 * 32, y // 32 * 32, z // 32 * 32)
        u = flat[pi * per:(pi + 1) * per].reshape(5, 32, 32, 32)[:, z % 32, y % 32, x % 32]
        want = oracle_cell(W, x, y, z)
        err = np.abs(u - want) / np.maximum(np.abs(want), ref_scale)
        worst = max(worst, err.max())
    tol = 1e-12 if precision == "fp64" else 5 * TOL["fp32"]["l1"]
    assert worst <= tol, worst
    scale = np.abs(t0).max()
    assert np.all(np.abs(t1 - t0) <= (1e-13 if precision == "fp64" else 2e-6) * scale), t1 - t0
