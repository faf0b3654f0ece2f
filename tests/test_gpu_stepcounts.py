"""Parity at full size and at the workloads' step counts, every cell compared.

* static 4-level Sedov hierarchy (Sec. 6.2 blast, base 128^3, seeded 8-32
  patches, about 4300 patches and 31.6M cells): 10 coarse steps;
* GLM-MHD Orszag-Tang vortex extended in z (Sec. 7), uniform 192^3 as the one
  patch the benchmark times: 50 steps.

The oracle takes its CFL step every step and the GPU solvers (FP64 and FP32,
batched launches with graph replay, as timed) take the same dt sequence.  The
oracle runs the 192^3 box as 216 patches of 32^3 cut from the same initial
arrays (the oracle's result does not depend on the tiling of a uniform
periodic grid; its threads work over patches).  FP64: L1 rel <= 1e-10 and max
rel <= 1e-8 on both metrics; FP32: vector-metric L1 rel <= 2e-5 (the
per-variable FP32 figures are recorded and printed with the session summary).
The Kelvin-Helmholtz 256^3 workload (100 steps) is compared in the benchmark,
on the solver the benchmark times.
"""
import numpy as np
import pytest

import amr_inputs as ai
import oracle as orc
from parity import assert_parity

pytestmark = pytest.mark.gpu

from paper_0910_5547_gb300 import Solver  # noqa: E402
from paper_0910_5547_gb300 import build as B  # noqa: E402


def split_uniform(pb, tile):
    """The single-patch problem pb as tile^3 patches holding the same initial values."""
    n = pb.patches[0].n
    w = pb.prim[0]
    patches = ai.uniform_patches(n, (tile,) * 3)
    prim = [np.ascontiguousarray(w[:, p.lo[2]:p.lo[2] + p.n[2], p.lo[1]:p.lo[1] + p.n[1], p.lo[0]:p.lo[0] + p.n[0]])
            for p in patches]
    return ai.Problem(pb.name, pb.nvar, pb.gamma, pb.base_n, pb.bc, patches, prim, pb.domain_lo, pb.domain_hi,
                      pb.max_level)


def join_uniform(patches, cons, n, nvar):
    out = np.empty((nvar, n[2], n[1], n[0]))
    for p, u in zip(patches, cons):
        out[:, p.lo[2]:p.lo[2] + p.n[2], p.lo[1]:p.lo[1] + p.n[1], p.lo[0]:p.lo[0] + p.n[0]] = u
    return out


def lockstep(o, solvers, steps):
    for _ in range(steps):
        dt = o.step()
        for s in solvers.values():
            s.step(dt, sync=False)
    for s in solvers.values():
        s.check()


def test_sedov_4level_10_coarse_steps_every_cell():
    B.build()
    pb = ai.sedov_amr()
    o = orc.Oracle(pb, nthreads=0)
    solvers = {p: Solver.from_problem(pb, precision=p) for p in ("fp64", "fp32")}
    t0 = o.totals()
    lockstep(o, solvers, 10)
    ref = o.all_cons()
    for prec, s in solvers.items():
        assert_parity(s.all_cons(), ref, pb.patches, prec, f"fullsize sedov-4level 10 coarse steps {prec}")
        t1 = s.totals()
        # outflow walls, ambient gas at rest: mass and energy stay
        rt = 1e-12 if prec == "fp64" else 2e-6
        assert abs(t1[0] - t0[0]) <= rt * t0[0] and abs(t1[4] - t0[4]) <= rt * t0[4], (prec, t0, t1)
        s.close()


def test_orszag_tang_192_50_steps_every_cell():
    B.build()
    pb = ai.orszag_tang(N=192, tile=None)
    po = split_uniform(pb, 32)
    o = orc.Oracle(po, nthreads=0)
    solvers = {p: Solver.from_problem(pb, precision=p) for p in ("fp64", "fp32")}
    lockstep(o, solvers, 50)
    ref = [join_uniform(po.patches, o.all_cons(), pb.patches[0].n, 9)]
    for prec, s in solvers.items():
        assert_parity(s.all_cons(), ref, pb.patches, prec, f"fullsize orszag-tang-192 50 steps {prec}")
        s.close()
