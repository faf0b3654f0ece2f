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


# ---------------------------------------------------------------------------
# GLM-MHD Orszag-Tang 192^3 (one patch), fixed cleaning speed
# ---------------------------------------------------------------------------

def test_orszag_tang_192_one_step_sampled_cells():
    n = 192
    dt, ch = 2.0e-4, 2.0
    pb = ai.orszag_tang(N=n, tile=None)
    W = pb.prim[0]
    s = Solver.from_problem(pb, precision="fp64", ch=ch)
    t0 = s.totals()
    s.step(dt)
    s.check()
    u = s.cons(0)
    t1 = s.totals()
    rng = np.random.default_rng(5)
    pts = [(0, 0, 0), (191, 95, 7)] + [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(10)]
    scale = np.array([0.25, 0.3, 0.3, 0.3, 0.5, 0.3, 0.3, 0.3, 0.3])
    worst = 0.0
    for (x, y, z) in pts:
        idx = [np.arange(c - 4, c + 5) % n for c in (x, y, z)]
        sub = W[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]
        o = orc.Oracle(patches=[ai.Patch(0, (0, 0, 0), (9, 9, 9))], prim=[np.ascontiguousarray(sub)],
                       base_n=(9, 9, 9), domain_hi=(9.0 / n,) * 3, bc=(ai.OUTFLOW,) * 6, nvar=9,
                       gamma=pb.gamma, ch=ch)
        o.step(dt)
        want = o.cons(0)[:, 4, 4, 4]
        worst = max(worst, (np.abs(u[:, z, y, x] - want) / np.maximum(np.abs(want), scale)).max())
    assert worst <= 1e-12, worst
    assert np.all(np.abs(t1 - t0) <= 1e-12 * np.abs(t0).max()), t1 - t0


# ---------------------------------------------------------------------------
# Static 4-level Sedov hierarchy (base 128^3, ~4300 patches): one coarse step
# ---------------------------------------------------------------------------

SEDOV_DT = 2.0e-7    # below the CFL step of the finest level times 8


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sedov_4level_one_coarse_step_sampled_cells(precision):
    pb = ai.sedov_amr()
    L = pb.max_level
    base = pb.base_n[0]
    s = Solver.from_problem(pb, precision=precision)
    t0 = s.totals()
    s.step(SEDOV_DT)
    s.check()
    cons = s.all_cons()
    t1 = s.totals()
    # mass and energy: no flux through the outflow walls in one step (ambient gas at rest)
    rt = 1e-12 if precision == "fp64" else 2e-6
    assert abs(t1[0] - t0[0]) <= rt * t0[0] and abs(t1[4] - t0[4]) <= rt * t0[4], (t0, t1)
    tol = 1e-10 if precision == "fp64" else 5e-5

    def locate(level, g):
        for i, p in enumerate(pb.patches):
            if p.level == level and all(p.lo[d] <= g[d] < p.lo[d] + p.n[d] for d in range(3)):
                return i, p
        raise AssertionError("cell not found")

    # (a) finest-level cells more than 32 cells inside the finest region: eight substeps of
    #     dt/8 depend only on finest-level data within 32 cells (4 per substep)
    side = pb.meta["sides"][-1]
    Nl = base << L
    lo_l, hi_l = (Nl - side) // 2, (Nl + side) // 2
    rng = np.random.default_rng(7)
    centre = Nl // 2
    finest = [(centre, centre, centre), (centre - 1, centre, centre + 2)]
    finest += [tuple(int(v) for v in rng.integers(lo_l + 33, hi_l - 33, 3)) for _ in range(2)]
    for g in finest:
        i, p = locate(L, g)
        box_lo = tuple(c - 32 for c in g)
        prim, _, _ = ai.sedov_prim([ai.Patch(L, box_lo, (65, 65, 65))], base, L)
        dxl = 1.0 / Nl
        o = orc.Oracle(patches=[ai.Patch(0, (0, 0, 0), (65, 65, 65))], prim=prim, base_n=(65, 65, 65),
                       domain_lo=tuple(c * dxl for c in box_lo), domain_hi=tuple((c + 65) * dxl for c in box_lo),
                       bc=(ai.OUTFLOW,) * 6, nvar=5, gamma=pb.gamma, nthreads=8)
        for _ in range(1 << L):
            o.step(SEDOV_DT / (1 << L))
        want = o.cons(0)[:, 32, 32, 32]
        got = cons[i][:, g[2] - p.lo[2], g[1] - p.lo[1], g[0] - p.lo[0]]
        err = np.abs(got - want) / np.maximum(np.abs(want), np.array([1.0, 1e-3, 1e-3, 1e-3, 1e-3]))
        assert err.max() <= tol, (g, got, want)
    # (b) level-0 cells more than 4 cells away from every level-1 footprint: one step of dt
    l1_side = pb.meta["sides"][0]
    f_lo, f_hi = ((base << 1) - l1_side) // 4, ((base << 1) + l1_side) // 4
    coarse = [(2, 3, 5), (127, 64, 0), (0, 0, 127), (64, 3, 120), (f_lo - 5, f_lo - 5, 60)]
    for g in coarse:
        assert any(c < f_lo - 4 or c >= f_hi + 4 for c in g)
        i, p = locate(0, g)
        blo = tuple(max(0, c - 4) for c in g)
        bhi = tuple(min(base, c + 5) for c in g)
        n = tuple(b - a for a, b in zip(blo, bhi))
        prim, _, _ = ai.sedov_prim([ai.Patch(0, blo, n)], base, L)
        dx0 = 1.0 / base
        o = orc.Oracle(patches=[ai.Patch(0, (0, 0, 0), n)], prim=prim, base_n=n,
                       domain_lo=tuple(c * dx0 for c in blo), domain_hi=tuple(c * dx0 for c in bhi),
                       bc=(ai.OUTFLOW,) * 6, nvar=5, gamma=pb.gamma)
        o.step(SEDOV_DT)
        c = tuple(gg - b for gg, b in zip(g, blo))
        want = o.cons(0)[:, c[2], c[1], c[0]]
        got = cons[i][:, g[2] - p.lo[2], g[1] - p.lo[1], g[0] - p.lo[0]]
        err = np.abs(got - want) / np.maximum(np.abs(want), np.array([1.0, 1e-3, 1e-3, 1e-3, 1e-3]))
        assert err.max() <= tol, (g, got, want)


# ---------------------------------------------------------------------------
# Adaptive blast in clumps (base 64^3 + 5 levels): one coarse step with the
# workload's regrid cadence (15 rebuilds inside the step)
# ---------------------------------------------------------------------------

def test_adaptive_full_size_one_coarse_step_invariants():
    """The gas at the outflow walls is at rest at the ambient pressure for the
    first coarse step, so mass and energy are conserved and the momentum fluxes
    of opposite walls cancel; every rebuilt hierarchy stays properly nested and
    every state physical."""
    from paper_0910_5547_gb300 import native as N
    pb = ai.blast_clumps()
    rkw = dict(threshold=0.3, buffer=4, block=4, max_patch=32)
    s = Solver.from_problem(pb, precision="fp32")
    s.step(0.0)
    s.regrid(**rkw)
    t0 = s.totals()
    c0 = N.amr_get_regrid_counts(s.h)
    s.set_regrid_schedule(pb.max_level - 2, **rkw)
    s.step(0.0)
    s.check()
    t1 = s.totals()
    c1 = N.amr_get_regrid_counts(s.h)
    assert (c1[0] + c1[1]) - (c0[0] + c0[1]) == 1 + 2 + 4 + 8     # after each step of levels 0..3
    assert abs(t1[0] - t0[0]) <= 2e-6 * t0[0] and abs(t1[4] - t0[4]) <= 2e-6 * t0[4], (t0, t1)
    pscale = np.sqrt(2.0 * t0[0] * t0[4])
    assert np.all(np.abs(t1[1:4] - t0[1:4]) <= 2e-6 * pscale), (t0, t1)
    cfg = N.amr_default_config(base_n=pb.base_n, max_level=pb.max_level, bc=pb.bc)
    assert N.amr_validate_patches(cfg, s.patches)[0] == N.AMR_OK
    assert max(p.level for p in s.patches) == pb.max_level
