"""Pins of two optional terms of the oracle: the positivity floor of the
reconstructed pressure (p_floor) and the GLM damping source of psi
(glm_alpha, the damping rate controlled by c_h in Sec. 7.1).  No GPU needed."""
import math

import numpy as np

import amr_inputs as ai
import oracle as orc


def test_floor_raises_only_states_below_it():
    """The reconstructed pressure is max(p, p_floor): a state below the floor reads
    p_floor, a state above it reads exactly the same value as without a floor."""
    lo = orc.prim_to_cons(np.array([0.7, 0.3, -0.2, 0.1, 1e-9]))
    hi = orc.prim_to_cons(np.array([0.7, 0.3, -0.2, 0.1, 0.5]))
    w_lo = orc.cons_to_prim(lo, p_floor=1e-4)
    assert math.isclose(w_lo[4], 1e-4, rel_tol=1e-13)
    assert math.isclose(orc.cons_to_prim(lo)[4], 1e-9, rel_tol=1e-6)
    assert np.array_equal(w_lo[:4], orc.cons_to_prim(lo)[:4])
    assert np.array_equal(orc.cons_to_prim(hi, p_floor=1e-4), orc.cons_to_prim(hi))


def test_floor_keeps_the_update_conservative():
    """With the floor above the ambient pressure it acts in every cell, changes the
    solution, and the totals still hold to round-off: the floor enters only the
    reconstruction, never the conserved state."""
    pb = ai.double_rarefaction(32, 4, p=1e-6)
    runs = {}
    for pf in (0.0, 1e-5):
        o = orc.Oracle(pb, p_floor=pf)
        t0 = o.totals()
        for _ in range(8):
            o.step(0.0)
        t1 = o.totals()
        scale = np.array([abs(t0[0]), 2.0 * abs(t0[0]), 1.0, 1.0, abs(t0[4])])  # |momentum| <= rho u
        assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (pf, t1 - t0)
        runs[pf] = np.concatenate([u.ravel() for u in o.all_cons()])
    assert np.max(np.abs(runs[1e-5] - runs[0.0])) > 1e-8


def _uniform_mhd(psi0=0.7, n=8):
    return ai.uniform(ai.uniform_patches((n,) * 3, (n,) * 3), (n,) * 3, nvar=9, gamma=5.0 / 3.0,
                      state=(1.1, 0.3, -0.2, 0.1, 0.8, 0.5, 0.2, -0.1, psi0))


def test_glm_damping_of_uniform_state_is_the_exact_decay():
    """A uniform state has no flux divergence, so psi obeys d psi/dt = -(alpha c_h / dx) psi
    alone: psi(t) = psi0 exp(-alpha c_h t / dx); every other variable stays bitwise."""
    n, alpha, ch, dt, steps = 8, 0.5, 2.0, 0.01, 6
    pb = _uniform_mhd(n=n)
    o = orc.Oracle(pb, ch=ch, glm_alpha=alpha)
    u0 = o.all_cons()[0]
    for _ in range(steps):
        o.step(dt)
    u1 = o.all_cons()[0]
    expect = 0.7 * math.exp(-alpha * ch * steps * dt / (1.0 / n))
    assert np.allclose(u1[8], expect, rtol=1e-13, atol=0.0)
    assert np.array_equal(u1[:8], u0[:8])


def test_glm_damping_off_is_pure_hyperbolic_cleaning():
    """glm_alpha = 0 leaves a uniform psi unchanged, bitwise."""
    pb = _uniform_mhd()
    o = orc.Oracle(pb, ch=2.0)
    u0 = o.all_cons()[0]
    for _ in range(3):
        o.step(0.01)
    assert np.array_equal(o.all_cons()[0], u0)


def test_glm_damping_reduces_psi_on_a_smooth_field():
    """On a smooth periodic MHD field the damped run ends with a smaller psi norm than
    the undamped one, and the mass, momentum, energy and B totals are unchanged by it."""
    pb = ai.random_smooth(ai.uniform_patches((16,) * 3, (8,) * 3), (16,) * 3, nvar=9, gamma=5.0 / 3.0, seed=5)
    res = {}
    for alpha in (0.0, 0.8):
        o = orc.Oracle(pb, ch=1.5, glm_alpha=alpha)
        t0 = o.totals()
        for _ in range(4):
            o.step(0.004)
        t1 = o.totals()
        assert np.allclose(t1[:8], t0[:8], rtol=0.0, atol=1e-13 * np.max(np.abs(t0[:8])))
        res[alpha] = sum(float(np.sum(u[8] ** 2)) for u in o.all_cons())
    assert res[0.8] < res[0.0]
