"""Stream-ordered state copies through the C ABI (amr_set_state_async,
amr_get_state_all_async, amr_wait_state): a pipelined loop whose uploads and
downloads overlap the steps gives bitwise the states of the synchronous loop,
with a different input every step (so the three staging slots per direction
cannot be confused), with two or three host input buffers in rotation (the
loop waits for the download of step k - depth before reusing a buffer); the
slots follow a regrid; unknown tickets are rejected."""
import numpy as np
import pytest

import amr_inputs as ai

pytestmark = pytest.mark.gpu

from paper_0910_5547_gb300 import Solver  # noqa: E402
from paper_0910_5547_gb300 import build as B  # noqa: E402
from paper_0910_5547_gb300 import native as N  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    N.load()
    yield


def _pinned(n):
    torch = pytest.importorskip("torch")
    return torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()


@pytest.mark.parametrize("depth", [2, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pipelined_loop_equals_synchronous_loop(precision, depth):
    pb = ai.kelvin_helmholtz(N=32, tile=16)
    s = Solver.from_problem(pb, precision=precision)
    base = s.state_all().copy()
    n = base.size
    ins = [base * (1.0 + 0.01 * k) for k in range(7)]   # scaled conserved states: same v and e
    dt = 0.5 * s.cfl_dt()
    want = []
    for x in ins:
        N.amr_set_state(s.h, x, N.AMR_STATE_CONSERVED)
        s.step(dt)
        out = np.empty(n)
        N.amr_get_state_all(s.h, out)
        want.append(out)
    h_in = [_pinned(n) for _ in range(depth)]
    h_out = [_pinned(n) for _ in range(len(ins))]
    tickets = []
    for k, x in enumerate(ins):
        if k >= depth:
            N.amr_wait_state(s.h, tickets[k - depth])   # the input buffer of step k - depth is free again
        h_in[k % depth][:] = x
        N.amr_set_state_async(s.h, h_in[k % depth])
        s.step(dt, sync=False)
        tickets.append(N.amr_get_state_all_async(s.h, h_out[k]))
    for t in tickets:
        N.amr_wait_state(s.h, t)
    s.check()
    for got, exp in zip(h_out, want):
        assert np.array_equal(got, exp)
    s.close()


def test_async_slots_follow_a_regrid_and_bad_tickets_fail():
    patches = ai.uniform_patches((32,) * 3, (16,) * 3)
    pb = ai.random_smooth(patches, (32,) * 3, seed=3, amp=0.6)
    s = Solver.from_problem(pb, precision="fp64", max_level=2)
    out = _pinned(int(N.amr_state_size(s.h)))
    N.amr_wait_state(s.h, N.amr_get_state_all_async(s.h, out))
    assert np.array_equal(out, s.state_all())
    s.step()
    s.regrid(threshold=0.1)
    m = int(N.amr_state_size(s.h))
    assert m != out.size
    out2 = _pinned(m)
    t = N.amr_get_state_all_async(s.h, out2)
    N.amr_wait_state(s.h, t)
    assert np.array_equal(out2, s.state_all())
    with pytest.raises(N.AmrError) as e:
        N.amr_wait_state(s.h, t + 5)
    assert e.value.status == N.AMR_ERR_ARG
    s.close()
