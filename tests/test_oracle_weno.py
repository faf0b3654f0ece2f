"""Pins of the oracle's third-order WENO face states (recon = WENO3; the
abstract's "higher order shock capturing schemes", read as the Jiang-Shu r = 2
scheme on the same three-cell stencils as the Sec. 4 PLM):

* linear data: both candidates are exact, so the face values are the linear
  function at the face;
* a symmetric extremum (a = c: equal smoothness indicators, so the linear
  weights 1/3, 2/3 apply) gives the value at the face of the quadratic whose
  cell averages are (a, b, c), found here by solving the 3 x 3 moment system;
* a step picks the smooth candidate (no new extremum, up to the eps weight);
* face values of cell averages of a sine converge at third order (PLM at
  second) and are more accurate than PLM from 256 cells on;
* runs: Sod against the exact solution, uniform state bitwise, periodic
  conservation, mirror symmetry, a smooth wave converging at third order
  (PLM: second) and more accurate than PLM at 512 cells, the
  GLM-MHD system, and WENO3 with direct flux reconstruction rejected.
"""
import math

import numpy as np
import pytest

import amr_inputs as ai
import oracle as orc
import riemann_exact as rex

RNG = np.random.default_rng(2024)
SOD = (1.0, 0.0, 1.0, 0.125, 0.0, 0.1)


def test_linear_data_is_reconstructed_exactly():
    for _ in range(50):
        a, b = RNG.uniform(-3, 3, 2)
        u4 = [a + b * k for k in range(4)]          # cell averages of a + b x, cells centred at 0..3
        ul, ur = orc.weno3_face(u4)
        face = a + b * 1.5                          # the face between cells 1 and 2
        assert abs(ul - face) <= 1e-12 * (1 + abs(face))
        assert abs(ur - face) <= 1e-12 * (1 + abs(face))


def _quadratic_face(a, b, c):
    """Value at x = 1/2 of the quadratic whose averages over [k - 1/2, k + 1/2], k = -1, 0, 1, are a, b, c."""
    m = np.array([[1.0, k, k * k + 1.0 / 12.0] for k in (-1, 0, 1)])
    al, be, ga = np.linalg.solve(m, [a, b, c])
    return al + be * 0.5 + ga * 0.25


def test_symmetric_extremum_uses_the_linear_weights():
    for _ in range(50):
        a, b = RNG.uniform(-2, 2, 2)
        d = RNG.uniform(-2, 2)
        # left state of the face between cells 1 and 2 from (u0, u1, u2) = (a, b, a)
        ul, _ = orc.weno3_face([a, b, a, d])
        assert abs(ul - _quadratic_face(a, b, a)) <= 1e-12 * (1 + abs(ul))
        # right state from (u3, u2, u1) = (a, b, a), mirrored
        _, ur = orc.weno3_face([d, a, b, a])
        assert abs(ur - _quadratic_face(a, b, a)) <= 1e-12 * (1 + abs(ur))


def test_a_step_takes_the_smooth_candidate():
    ul, ur = orc.weno3_face([0.0, 0.0, 1.0, 1.0])
    assert abs(ul) < 1e-9 and abs(ur - 1.0) < 1e-9
    for _ in range(20):
        lo, hi = sorted(RNG.uniform(-5, 5, 2))
        ul, ur = orc.weno3_face([lo, lo, hi, hi])
        assert lo - 1e-9 <= ul <= hi + 1e-9 and lo - 1e-9 <= ur <= hi + 1e-9
        assert abs(ul - lo) < 1e-6 * (hi - lo) + 1e-12 and abs(ur - hi) < 1e-6 * (hi - lo) + 1e-12


def _face_errors(n, face):
    h = 1.0 / n
    x = np.arange(n) * h
    avg = (np.cos(2 * np.pi * x) - np.cos(2 * np.pi * (x + h))) / (2 * np.pi * h)
    err = 0.0
    for i in range(n):
        ul, ur = face([avg[(i - 2) % n], avg[(i - 1) % n], avg[i], avg[(i + 1) % n]])
        exact = math.sin(2 * np.pi * i * h)
        err += abs(ul - exact) + abs(ur - exact)
    return err / n


def test_face_values_converge_at_third_order():
    e = {n: _face_errors(n, orc.weno3_face) for n in (128, 256, 512)}
    assert math.log2(e[128] / e[256]) >= 2.8, e
    assert math.log2(e[256] / e[512]) >= 2.8, e
    p256, p512 = (_face_errors(n, orc.plm_face) for n in (256, 512))
    assert math.log2(p256 / p512) < 2.3            # PLM: second order
    assert e[256] < p256 and e[512] < 0.5 * p512


def _sod_l1(n, t_end, **kw):
    pb = ai.sod(n=n, ny=1, t_end=t_end)
    o = orc.Oracle(pb, **kw)
    o.run_to(t_end)
    rho = o.cons(0)[0, 0, 0, :]
    x = np.arange(n) / n
    er, _, _ = rex.cell_average(x, x + 1.0 / n, t_end, 0.5, SOD)
    return np.abs(rho - er).mean()


def test_sod_matches_the_exact_solution():
    e100 = _sod_l1(100, 0.14, recon=orc.WENO3)
    e400 = _sod_l1(400, 0.14, recon=orc.WENO3)
    assert e100 < 1e-2 and e400 < 0.4 * e100


def test_uniform_state_conservation_and_mirror_symmetry():
    patches = ai.uniform_patches((16, 16, 16), (8, 8, 8))
    o = orc.Oracle(ai.uniform(patches, (16, 16, 16)), recon=orc.WENO3)
    u0 = o.all_cons()
    for _ in range(3):
        o.step(0.01)
    for a, b in zip(u0, o.all_cons()):
        assert np.array_equal(a, b)
    o = orc.Oracle(ai.random_smooth(patches, (16, 16, 16), seed=5), recon=orc.WENO3)
    t0 = o.totals()
    for _ in range(4):
        o.step()
    assert np.all(np.abs(o.totals() - t0) <= 1e-13 * np.abs(t0).max())
    pb, pm = ai.sod(n=64, ny=1), ai.sod(n=64, ny=1)
    pm.prim[0] = pm.prim[0][:, :, :, ::-1].copy()
    a, b = orc.Oracle(pb, recon=orc.WENO3), orc.Oracle(pm, recon=orc.WENO3)
    for _ in range(30):
        a.step(0.002)
        b.step(0.002)
    ua, ub = a.cons(0), b.cons(0)
    np.testing.assert_allclose(ua[0], ub[0][:, :, ::-1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(ua[1], -ub[1][:, :, ::-1], rtol=0, atol=1e-12)


def test_smooth_wave_converges_faster_than_plm():
    err = {}
    for n in (256, 512):
        pb = ai.advected_wave(n=n)
        x = (np.arange(n) + 0.5) / n
        for name, kw in (("plm", {}), ("weno3", {"recon": orc.WENO3})):
            o = orc.Oracle(pb, **kw)
            o.run_to(1.0)
            err[name, n] = np.abs(o.cons(0)[0, 0, 0] - (1 + 0.2 * np.sin(2 * np.pi * x))).mean()
    assert math.log2(err["weno3", 256] / err["weno3", 512]) >= 2.5, err
    assert math.log2(err["plm", 256] / err["plm", 512]) < 2.3, err
    assert err["weno3", 512] < 0.5 * err["plm", 512], err


def test_glm_mhd_runs_and_conserves():
    pb = ai.orszag_tang(N=16, tile=8)
    o = orc.Oracle(pb, recon=orc.WENO3)
    t0 = o.totals()
    for _ in range(3):
        o.step()
    assert np.all(np.isfinite(o.totals()))
    assert np.all(np.abs(o.totals() - t0)[:8] <= 1e-12 * np.abs(t0).max())


def test_weno3_with_flux_reconstruction_is_rejected():
    with pytest.raises((ValueError, RuntimeError)):
        orc.Oracle(ai.sod(n=16, ny=1), recon=orc.WENO3, riemann=orc.FLUXREC)
