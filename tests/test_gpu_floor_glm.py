"""GPU parity of the optional pressure floor and GLM damping source against the
FP64 oracle (same tolerances as the other parity tests), the floor counter,
and the exact decay of psi under damping."""
import math

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


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    N.load()
    yield


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("p_floor", [0.0, 1e-5])
def test_floor_parity_on_double_rarefaction(precision, p_floor):
    """Receding streams at ambient p = 1e-6; a floor of 1e-5 acts in every cell."""
    pb = ai.double_rarefaction(32, 8, tile=16, p=1e-6)
    o = orc.Oracle(pb, nthreads=8, p_floor=p_floor)
    s = Solver.from_problem(pb, precision=precision, p_floor=p_floor)
    for _ in range(8):
        o.step(0.0)
        s.step(0.0)
    s.check()
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, f"rarefaction floor={p_floor}")
    hits = s.floor_count()
    cells = sum(p.n[0] * p.n[1] * p.n[2] for p in pb.patches)
    if p_floor > 0.0:
        assert hits > cells          # every cell, both stages, several steps
        assert hits <= 2 * 8 * cells
    else:
        assert hits == 0
    assert s.floor_count() == 0      # read and reset


def test_fp64_sod_never_needs_the_floor():
    """FP64 configurations never rely on the floor: with a tiny floor the Sod run
    records no activation and matches the floor-free oracle."""
    pb = ai.sod(n=32)
    o = orc.Oracle(pb, nthreads=8)
    s = Solver.from_problem(pb, precision="fp64", p_floor=1e-12)
    n_o = o.run_to(0.2)
    n_s = s.run_to(0.2)
    assert n_o == n_s
    assert s.floor_count() == 0
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, "fp64", "sod-floor")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_glm_damping_exact_decay(precision):
    n, alpha, ch, dt, steps = 16, 0.5, 2.0, 0.01, 6
    pb = ai.uniform(ai.uniform_patches((n,) * 3, (8,) * 3), (n,) * 3, nvar=9, gamma=5.0 / 3.0,
                    state=(1.1, 0.3, -0.2, 0.1, 0.8, 0.5, 0.2, -0.1, 0.7))
    s = Solver.from_problem(pb, precision=precision, ch=ch, glm_alpha=alpha)
    u0 = s.all_cons()
    for _ in range(steps):
        s.step(dt)
    s.check()
    expect = 0.7 * math.exp(-alpha * ch * steps * dt * n)
    tol = 1e-12 if precision == "fp64" else 2e-6
    for a, b in zip(s.all_cons(), u0):
        assert np.allclose(a[8], expect, rtol=tol, atol=0.0)
        assert np.array_equal(a[:8], b[:8]) if precision == "fp64" else np.allclose(a[:8], b[:8], rtol=1e-6)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_glm_damping_parity_on_amr(precision):
    """Three-level periodic MHD hierarchy with a smooth field, fixed c_h and damping."""
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, nvar=9, gamma=5.0 / 3.0, seed=5)
    o = orc.Oracle(pb, nthreads=8, ch=1.5, glm_alpha=0.8)
    s = Solver.from_problem(pb, precision=precision, ch=1.5, glm_alpha=0.8)
    for _ in range(2):
        o.step(0.002)
        s.step(0.002)
    s.check()
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "mhd-amr-glm")
