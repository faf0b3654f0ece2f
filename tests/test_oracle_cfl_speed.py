"""Pins of the oracle's CFL step size, GLM-MHD fast magnetosonic speed and
cleaning speed c_h against closed forms.  No GPU needed.

CFL (the paper gives none; reading: dt0 = C / max over all cells of all levels
of sum_d (|v_d| + c_d) / dx0_d, level l stepping dt0 / 2^l): uniform states
with known v and c on an anisotropic grid, and a two-level hierarchy whose
fastest cells lie on the fine level only.  A max over d instead of the sum,
the fine level's dx instead of dx0, or a rate that skips fine levels each
changes dt by a factor of 1.5 or more.

Fast magnetosonic speed (Sec. 7.1, Heaviside units since the energy holds
B^2 / 2; a^2 = gamma p / rho, b = B / sqrt(rho)):
  B parallel to d:       c_f,d = max(a, |b_d|)
  B perpendicular to d:  c_f,d = sqrt(a^2 + b^2)
(the two textbook limits of c_f^2 = (a^2 + b^2 + sqrt((a^2 + b^2)^2 - 4 a^2 b_d^2)) / 2).
B^2 in place of B_d^2 under the inner root, or a missing 1/rho, fails one of them.

Cleaning speed (c_h <= 0 in the configuration): the largest |v_d| + c_f,d over
all cells and axes at the start of the coarse step.
"""
import math

import numpy as np
import pytest

import amr_inputs as ai
import oracle as orc

P, O = ai.PERIODIC, ai.OUTFLOW


def _const_problem(patches, base_n, nvar, gamma, state_of, dom_hi=(1.0, 1.0, 1.0), bc=P):
    prim = []
    for p in patches:
        w = np.zeros((nvar, p.n[2], p.n[1], p.n[0]))
        s = state_of(p)
        for v in range(nvar):
            w[v] = s[v]
        prim.append(w)
    return ai.Problem("const", nvar, gamma, tuple(base_n), (bc,) * 6, patches, prim,
                      domain_hi=tuple(dom_hi), max_level=max(p.level for p in patches))


def _rate(state, dx, gamma, cf):
    """sum_d (|v_d| + c_d) / dx_d with per-axis signal speeds cf[d]."""
    return sum((abs(state[1 + d]) + cf[d]) / dx[d] for d in range(3))


def test_cfl_uniform_state_anisotropic_grid_sums_the_axes():
    gamma, cfl = 1.4, 0.4
    base = (16, 8, 12)
    dom_hi = (1.0, 0.5, 2.0)
    dx = [dom_hi[d] / base[d] for d in range(3)]         # 1/16, 1/16, 1/6: all different rates
    st = (1.3, 0.7, -0.45, 0.2, 0.9)
    a = math.sqrt(gamma * st[4] / st[0])
    pb = _const_problem(ai.uniform_patches(base, (8, 8, 6)), base, 5, gamma, lambda p: st, dom_hi)
    o = orc.Oracle(pb, cfl=cfl)
    want = cfl / _rate(st, dx, gamma, (a, a, a))
    assert o.cfl_dt() == pytest.approx(want, rel=1e-14)
    # a max over the axes instead of the sum would give at least 1.5x this step
    max_form = cfl / max((abs(st[1 + d]) + a) / dx[d] for d in range(3))
    assert max_form > 1.5 * want
    # the step taken with dt <= 0 is that step
    assert o.step(0.0) == pytest.approx(want, rel=1e-14)


def test_cfl_two_level_takes_the_fine_cells_at_the_coarse_spacing():
    """Fine cells hold a faster state than every coarse cell (covered ones
    included); dt0 = C / rate_fine(dx0): the Courant number of level l is
    dt0 / 2^l * rate / (dx0 / 2^l), the same on every level."""
    gamma, cfl = 1.4, 0.4
    base = (16, 16, 16)
    patches = ai.uniform_patches(base, (8, 8, 8)) + [ai.Patch(1, (8, 8, 8), (16, 16, 16))]
    slow = (1.0, 0.1, 0.0, 0.0, 1.0)
    fast = (1.0, 2.5, -1.0, 0.5, 3.0)
    pb = _const_problem(patches, base, 5, gamma, lambda p: fast if p.level == 1 else slow, bc=O)
    o = orc.Oracle(pb, cfl=cfl)
    dx0 = [1.0 / 16] * 3
    a_fast = math.sqrt(gamma * fast[4] / fast[0])
    a_slow = math.sqrt(gamma * slow[4] / slow[0])
    want = cfl / _rate(fast, dx0, gamma, (a_fast,) * 3)
    assert o.cfl_dt() == pytest.approx(want, rel=1e-14)
    assert cfl / _rate(slow, dx0, gamma, (a_slow,) * 3) > 1.5 * want    # skipping level 1 would differ
    assert want > 1.5 * cfl / _rate(fast, [d / 2 for d in dx0], gamma, (a_fast,) * 3)  # so would dx1


def _mhd_state(rho, v, p, B, psi=0.0):
    return (rho, v[0], v[1], v[2], p, B[0], B[1], B[2], psi)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("strong", [False, True])
def test_fast_speed_parallel_and_perpendicular_limits(axis, strong):
    """B along one axis: on that axis c_f = max(a, |b|), on the other two
    c_f = sqrt(a^2 + b^2).  The weak field has |b| < a, the strong one |b| > a,
    so both branches of the max are taken."""
    gamma, cfl = 5.0 / 3.0, 0.4
    rho, p = 1.7, 0.6
    a = math.sqrt(gamma * p / rho)
    Bmag = (0.5 if not strong else 3.0) * a * math.sqrt(rho)
    B = [0.0, 0.0, 0.0]
    B[axis] = -Bmag
    v = (0.11, -0.23, 0.07)
    st = _mhd_state(rho, v, p, B)
    b = Bmag / math.sqrt(rho)
    cf = [math.sqrt(a * a + b * b)] * 3
    cf[axis] = max(a, b)
    base = (8, 8, 8)
    pb = _const_problem(ai.uniform_patches(base, base), base, 9, gamma, lambda q: st)
    o = orc.Oracle(pb, cfl=cfl)
    dx = [1.0 / 8] * 3
    assert o.cfl_dt() == pytest.approx(cfl / _rate(st, dx, gamma, cf), rel=1e-13)
    o.step(1e-4)
    assert o.last_ch() == pytest.approx(max(abs(v[d]) + cf[d] for d in range(3)), rel=1e-13)


def test_fast_speed_oblique_field_and_cleaning_speed_over_two_patches():
    """An oblique field: the full formula c_f,d^2 = (s + sqrt(s^2 - 4 a^2 b_d^2)) / 2,
    s = a^2 + b^2, here written through the other root, the slow speed c_s,d:
    c_f^2 + c_s^2 = s and c_f^2 c_s^2 = a^2 b_d^2 (Vieta).  Two patches with
    different states: dt and c_h take the maxima over both."""
    gamma, cfl = 5.0 / 3.0, 0.3
    A = _mhd_state(1.2, (0.3, -0.1, 0.2), 0.8, (0.6, -0.9, 0.4))
    Bst = _mhd_state(0.7, (-0.6, 0.4, 0.1), 0.3, (-0.2, 0.5, 1.1))
    base = (16, 8, 8)
    patches = [ai.Patch(0, (0, 0, 0), (8, 8, 8)), ai.Patch(0, (8, 0, 0), (8, 8, 8))]
    pb = _const_problem(patches, base, 9, gamma, lambda q: A if q.lo[0] == 0 else Bst)
    dx = (1.0 / 16, 1.0 / 8, 1.0 / 8)

    def speeds(st):
        rho, p = st[0], st[4]
        a2 = gamma * p / rho
        b2 = [st[5 + d] ** 2 / rho for d in range(3)]
        s = a2 + sum(b2)
        out = []
        for d in range(3):
            # c_f^2 and c_s^2 are the roots of x^2 - s x + a^2 b_d^2 = 0
            cs2 = 2.0 * a2 * b2[d] / (s + math.sqrt(s * s - 4.0 * a2 * b2[d]))
            cf2 = s - cs2
            assert cf2 * cs2 == pytest.approx(a2 * b2[d], rel=1e-12)
            out.append(math.sqrt(cf2))
        return out

    cfA, cfB = speeds(A), speeds(Bst)
    o = orc.Oracle(pb, cfl=cfl)
    rate = max(_rate(A, dx, gamma, cfA), _rate(Bst, dx, gamma, cfB))
    assert o.cfl_dt() == pytest.approx(cfl / rate, rel=1e-13)
    o.step(1e-4)
    ch = max(max(abs(st[1 + d]) + cf[d] for d in range(3)) for st, cf in ((A, cfA), (Bst, cfB)))
    assert o.last_ch() == pytest.approx(ch, rel=1e-13)


def test_fixed_cleaning_speed_is_kept():
    st = _mhd_state(1.0, (0.1, 0.0, 0.0), 1.0, (0.5, 0.0, 0.0))
    base = (8, 8, 8)
    pb = _const_problem(ai.uniform_patches(base, base), base, 9, 5.0 / 3.0, lambda q: st)
    o = orc.Oracle(pb, ch=2.75)
    o.step(1e-4)
    assert o.last_ch() == 2.75


def test_hydro_fast_speed_reduces_to_sound_speed():
    """B = 0 in the MHD system: every axis has c_f = a, so the MHD and Euler CFL steps agree."""
    gamma = 1.4
    st9 = _mhd_state(1.3, (0.2, -0.1, 0.3), 0.9, (0.0, 0.0, 0.0))
    base = (8, 8, 8)
    o9 = orc.Oracle(_const_problem(ai.uniform_patches(base, base), base, 9, gamma, lambda q: st9))
    o5 = orc.Oracle(_const_problem(ai.uniform_patches(base, base), base, 5, gamma, lambda q: st9[:5]))
    assert o9.cfl_dt() == pytest.approx(o5.cfl_dt(), rel=1e-15)
