"""Pins of the oracle's direct flux reconstruction (Euler; Sec. 4 names it as the
second class of schemes the framework applies to).  Reading: Lax-Friedrichs
splitting F+- = (F(U) +- alpha U) / 2 with alpha the largest |v_d| + c of the
four stencil cells, F+ reconstructed from the left, F- from the right, each by
the Sec. 4 PLM face value.

* consistency: a uniform stencil gives the physical flux F(U);
* a stencil whose split fluxes are linear (constant velocity and pressure,
  linear density: F and U linear, alpha fixed) gives the mean of the two cells'
  fluxes exactly, which fixes the half slope and the sum F+ + F- (a full slope
  leaves alpha (U2 - U1) / 2 behind);
* which side each split flux is taken from is fixed by the Sod run (the
  downwind choice is unstable);
* the exact Sod solution, second-order convergence on a smooth wave, bitwise
  uniform-state preservation, conservation on a periodic box, mirror symmetry;
* GLM-MHD is rejected (Euler only).
"""
import math

import numpy as np
import pytest

import amr_inputs as ai
import oracle as orc
import riemann_exact as rex

RNG = np.random.default_rng(77)
SOD = (1.0, 0.0, 1.0, 0.125, 0.0, 0.1)


def _cons(w, gamma=1.4):
    rho, vx, vy, vz, p = w
    return np.array([rho, rho * vx, rho * vy, rho * vz, p / (gamma - 1) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)])


@pytest.mark.parametrize("d", [0, 1, 2])
def test_uniform_stencil_gives_the_physical_flux(d):
    for _ in range(20):
        w = np.array([RNG.uniform(0.2, 3), *RNG.uniform(-2, 2, 3), RNG.uniform(0.1, 4)])
        f = orc.fluxrec_face(np.tile(_cons(w), (4, 1)), d)
        assert np.allclose(f, orc.phys_flux(w, d), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("theta", [1.0, 1.5, 2.0])
def test_linear_split_fluxes_give_the_mean_of_the_two_cells(d, theta):
    v = RNG.uniform(-1.5, 1.5, 3)
    p = 0.8
    rho = 1.0 + 0.1 * np.arange(4)                 # linear density, constant v and p
    u4 = np.array([_cons((r, *v, p)) for r in rho])
    f = orc.fluxrec_face(u4, d, theta=theta)
    want = 0.5 * (orc.phys_flux(np.array([rho[1], *v, p]), d) + orc.phys_flux(np.array([rho[2], *v, p]), d))
    assert np.allclose(f, want, rtol=1e-13, atol=1e-13)
    # the reversed stencil (the same two cells, density now falling) gives the mean as well
    g = orc.fluxrec_face(u4[::-1].copy(), d, theta=theta)
    assert np.allclose(g, 0.5 * (orc.phys_flux(np.array([rho[2], *v, p]), d) +
                                 orc.phys_flux(np.array([rho[1], *v, p]), d)), rtol=1e-13, atol=1e-13)


def _sod_l1(n, t_end, **kw):
    pb = ai.sod(n=n, ny=1, t_end=t_end)
    o = orc.Oracle(pb, **kw)
    o.run_to(t_end)
    rho = o.cons(0)[0, 0, 0, :]
    x = np.arange(n) / n
    er, _, _ = rex.cell_average(x, x + 1.0 / n, t_end, 0.5, SOD)
    return np.abs(rho - er).mean()


def test_sod_matches_the_exact_solution_and_converges():
    e100 = _sod_l1(100, 0.14, riemann=orc.FLUXREC)
    e400 = _sod_l1(400, 0.14, riemann=orc.FLUXREC)
    assert e100 < 1e-2
    assert e400 < 0.35 * e100
    # Lax-Friedrichs splitting is more diffusive than the two-wave HLL flux
    assert _sod_l1(100, 0.14) < e100


def test_advected_wave_is_second_order():
    errs = []
    for n in (32, 64, 128):
        pb = ai.advected_wave(n=n)
        o = orc.Oracle(pb, riemann=orc.FLUXREC)
        o.run_to(1.0)
        x = (np.arange(n) + 0.5) / n
        errs.append(np.abs(o.cons(0)[0, 0, 0] - (1 + 0.2 * np.sin(2 * np.pi * x))).mean())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= 1.8, (errs, orders)


def test_uniform_state_bitwise_and_periodic_conservation():
    patches = ai.uniform_patches((16, 16, 16), (8, 8, 8))
    o = orc.Oracle(ai.uniform(patches, (16, 16, 16)), riemann=orc.FLUXREC)
    u0 = o.all_cons()
    for _ in range(3):
        o.step(0.01)
    for a, b in zip(u0, o.all_cons()):
        assert np.array_equal(a, b)
    o = orc.Oracle(ai.random_smooth(patches, (16, 16, 16), seed=3), riemann=orc.FLUXREC)
    t0 = o.totals()
    for _ in range(4):
        o.step()
    assert np.all(np.abs(o.totals() - t0) <= 1e-13 * np.abs(t0).max())


def test_mirror_symmetry():
    pb = ai.sod(n=64, ny=1)
    pm = ai.sod(n=64, ny=1)
    pm.prim[0] = pm.prim[0][:, :, :, ::-1].copy()
    o, om = orc.Oracle(pb, riemann=orc.FLUXREC), orc.Oracle(pm, riemann=orc.FLUXREC)
    for _ in range(30):
        o.step(0.002)
        om.step(0.002)
    u, um = o.cons(0), om.cons(0)
    np.testing.assert_allclose(u[0], um[0][:, :, ::-1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(u[1], -um[1][:, :, ::-1], rtol=0, atol=1e-12)


def test_mhd_is_rejected():
    pb = ai.orszag_tang(N=16, tile=8)
    with pytest.raises(ValueError):
        orc.Oracle(pb, riemann=orc.FLUXREC)
