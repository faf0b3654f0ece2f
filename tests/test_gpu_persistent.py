"""Persistent stage launches (one wave of resident CTAs taking work items from a
device counter) against one CTA per work item: the same states bit for bit over
several steps (every launch must leave the counter at zero for the next), with
graph replay and eager launches, both physics and precisions, WENO3 face states
and every tiling shape the autotuner tries; and the autotuner's report lists
both launch forms."""
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


def states(pb, steps, mode, tiling=None, **kw):
    s = Solver.from_problem(pb, **kw)
    if tiling:
        s.set_tiling(*tiling)
    s.set_persistent(mode)
    for _ in range(steps):
        s.step(0.0)
    s.check()
    out = s.state_all().copy()
    s.close()
    return out


@pytest.mark.parametrize("nvar,precision", [(5, "fp32"), (5, "fp64"), (9, "fp32"), (9, "fp64")])
def test_three_level_persistent_equals_per_item(nvar, precision):
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, nvar=nvar, seed=5, amp=0.2)
    a = states(pb, 3, 0, precision=precision)
    b = states(pb, 3, 1, precision=precision)
    assert np.array_equal(a, b)
    c = states(pb, 2, 1, precision=precision, use_graph=False)
    d = states(pb, 2, 0, precision=precision, use_graph=False)
    assert np.array_equal(c, d)


@pytest.mark.parametrize("tiling", [(32, 256, 32, 0), (16, 256, 16, 0), (16, 128, 8, 0), (32, 256, 64, 0)])
def test_tilings_and_weno3(tiling):
    pb = ai.kelvin_helmholtz(N=64, tile=16)
    assert np.array_equal(states(pb, 2, 0, tiling, precision="fp32"), states(pb, 2, 1, tiling, precision="fp32"))
    assert np.array_equal(states(pb, 2, 0, tiling, precision="fp32", recon="weno3"),
                          states(pb, 2, 1, tiling, precision="fp32", recon="weno3"))


def test_autotuner_times_both_forms():
    pb = ai.kelvin_helmholtz(N=64, tile=32)
    s = Solver.from_problem(pb, precision="fp32")
    rep = s.autotune()
    assert "persistent" in rep and rep.count("\n") >= 15
    s.set_persistent(0)
    assert "persistent" not in s.autotune()
    s.close()
