"""Pins of the FP64 oracle against facts fixed outside it (no GPU needed).

Each test checks the oracle against something it does not compute itself:
printed textbook values, closed forms, exact solutions, invariants, or
special cases that reduce to a simpler known answer.  A plausible mistake in
the oracle (a dropped term, a wrong sign, a swapped index) fails at least one.
"""
import json
import math
import os

import numpy as np
import pytest

import amr_inputs as ai
import oracle as orc
import riemann_exact as rex

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
RNG = np.random.default_rng(1234)


# ---------------------------------------------------------------------------
# the exact Riemann solver used as a pin is itself pinned to printed values
# ---------------------------------------------------------------------------

def test_exact_riemann_matches_printed_star_values():
    g = json.load(open(os.path.join(GOLD, "sod_star_toro.json")))
    ps, us, rl, rr = rex.star_state(*g["left"], *g["right"], g=g["gamma"])
    assert abs(ps - g["p_star"]) <= 5e-6
    assert abs(us - g["u_star"]) <= 5e-6
    assert abs(rl - g["rho_star_L"]) <= 5e-6
    assert abs(rr - g["rho_star_R"]) <= 5e-6


# ---------------------------------------------------------------------------
# limiter and reconstruction (Sec. 4)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("a,b,c,want", [
    (1.0, 2.0, 3.0, 1.0), (3.0, 2.0, 1.0, 1.0), (-1.0, -2.0, -3.0, -1.0), (-3.0, -0.5, -2.0, -0.5),
    (1.0, -2.0, 3.0, 0.0), (-1.0, 2.0, 3.0, 0.0), (1.0, 2.0, -3.0, 0.0),
    (0.0, 2.0, 3.0, 0.0), (2.0, 0.0, 3.0, 0.0), (2.0, 3.0, 0.0, 0.0), (0.0, 0.0, 0.0, 0.0),
])
def test_minmod3_truth_table(a, b, c, want):
    assert orc.minmod3(a, b, c) == want


def test_minmod2_truth_table():
    assert orc.minmod2(1.0, 2.0) == 1.0
    assert orc.minmod2(-3.0, -2.0) == -2.0
    assert orc.minmod2(1.0, -1.0) == 0.0
    assert orc.minmod2(0.0, 5.0) == 0.0


@pytest.mark.parametrize("theta", [1.0, 1.5, 2.0])
def test_plm_reconstructs_linear_data_exactly(theta):
    a, b = 0.7, -0.3
    u4 = [a + b * k for k in range(4)]          # cells i-2 .. i+1
    face = a + b * 1.5                          # value at x_{i-1/2}
    ul, ur = orc.plm_face(u4, theta=theta)
    assert ul == pytest.approx(face, abs=1e-15)
    assert ur == pytest.approx(face, abs=1e-15)


def test_plm_is_first_order_at_extrema_and_literal_flag_doubles_offset():
    ul, ur = orc.plm_face([0.0, 1.0, 0.0, -1.0], theta=1.5)
    assert ul == 1.0                            # local maximum: zero slope
    assert ur == 0.5                            # cell i: half of min(1.5, 1.5, 1) added
    ul2, ur2 = orc.plm_face([0.0, 1.0, 0.0, -1.0], theta=1.5, plm_literal=True)
    assert (ul2, ur2) == (1.0, 1.0)


# ---------------------------------------------------------------------------
# fluxes, EOS, Riemann solvers
# ---------------------------------------------------------------------------

def _random_state(nvar, rng=RNG):
    w = np.empty(nvar)
    w[0] = rng.uniform(0.2, 3.0)
    w[1:4] = rng.uniform(-1.5, 1.5, 3)
    w[4] = rng.uniform(0.1, 4.0)
    if nvar == 9:
        w[5:8] = rng.uniform(-1.0, 1.0, 3)
        w[8] = rng.uniform(-0.2, 0.2)
    return w


@pytest.mark.parametrize("nvar", [5, 9])
def test_prim_cons_roundtrip_and_energy_definition(nvar):
    for _ in range(20):
        w = _random_state(nvar)
        u = orc.prim_to_cons(w, nvar=nvar, gamma=1.4)
        # rho E = p/(gamma-1) + rho v^2/2 (+ B^2/2): Sec. 4 E = v^2/2 + e, p = (gamma-1) rho e
        E = w[4] / 0.4 + 0.5 * w[0] * np.dot(w[1:4], w[1:4])
        if nvar == 9:
            E += 0.5 * np.dot(w[5:8], w[5:8])
        assert u[4] == pytest.approx(E, rel=1e-14)
        np.testing.assert_allclose(orc.cons_to_prim(u, nvar=nvar, gamma=1.4), w, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("nvar", [5, 9])
@pytest.mark.parametrize("kind", [orc.HLL, orc.LLF])
def test_riemann_consistency(nvar, kind):
    """F(w, w) equals the physical flux F(w) for both solvers, all directions."""
    for _ in range(10):
        w = _random_state(nvar)
        for d in range(3):
            f = orc.riemann(w, w, d, nvar=nvar, kind=kind, ch=2.0)
            np.testing.assert_allclose(f, orc.phys_flux(w, d, nvar=nvar, ch=2.0), rtol=1e-13, atol=1e-13)


def _perm_state(w, perm):
    """Relabel axes: new axis k is old axis perm[k] (vectors permuted)."""
    out = w.copy()
    out[1:4] = w[1 + np.array(perm)]
    if len(w) == 9:
        out[5:8] = w[5 + np.array(perm)]
    return out


@pytest.mark.parametrize("nvar", [5, 9])
def test_flux_rotational_invariance(nvar):
    """The y and z fluxes are the x flux of the axis-relabelled state (index pins)."""
    for _ in range(10):
        w = _random_state(nvar)
        wr = _random_state(nvar)
        for d, perm in ((1, (1, 2, 0)), (2, (2, 0, 1))):
            f_d = orc.riemann(w, wr, d, nvar=nvar, ch=1.7)
            f_x = orc.riemann(_perm_state(w, perm), _perm_state(wr, perm), 0, nvar=nvar, ch=1.7)
            np.testing.assert_allclose(_perm_state(f_d, perm), f_x, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("M", [1.5, 2.5, 6.0])
def test_rankine_hugoniot_stationary_shock(M):
    """Across a stationary normal shock (normal-shock relations) the physical x flux is
    continuous in every component, with an arbitrary tangential velocity."""
    g = 1.4
    r1, p1 = 1.0, 1.0
    u1 = M * math.sqrt(g * p1 / r1)
    r2 = r1 * (g + 1) * M * M / ((g - 1) * M * M + 2)
    p2 = p1 * (1 + 2 * g / (g + 1) * (M * M - 1))
    u2 = r1 * u1 / r2
    w1 = np.array([r1, u1, 0.3, -0.2, p1])
    w2 = np.array([r2, u2, 0.3, -0.2, p2])
    np.testing.assert_allclose(orc.phys_flux(w1, 0), orc.phys_flux(w2, 0), rtol=1e-12)
    # and the upwind solvers return that flux for the shock itself
    np.testing.assert_allclose(orc.riemann(w1, w1, 0), orc.phys_flux(w1, 0), rtol=1e-13)


def test_hll_upwinds_supersonic_states():
    wl = np.array([1.0, 3.0, 0.1, 0.0, 0.5])     # supersonic to the right on both sides
    wr = np.array([0.8, 2.9, 0.0, 0.2, 0.4])
    np.testing.assert_allclose(orc.riemann(wl, wr, 0), orc.phys_flux(wl, 0), rtol=1e-14)
    wl2, wr2 = wl.copy(), wr.copy()
    wl2[1], wr2[1] = -3.0, -2.9
    np.testing.assert_allclose(orc.riemann(wl2, wr2, 0), orc.phys_flux(wr2, 0), rtol=1e-14)


def test_mhd_with_zero_field_is_hydro():
    for _ in range(10):
        w5 = _random_state(5)
        v5 = _random_state(5)
        w9 = np.concatenate([w5, np.zeros(4)])
        v9 = np.concatenate([v5, np.zeros(4)])
        for d in range(3):
            f9 = orc.riemann(w9, v9, d, nvar=9, ch=1.3)
            f5 = orc.riemann(w5, v5, d, nvar=5)
            np.testing.assert_allclose(f9[:5], f5, rtol=1e-14, atol=1e-15)
            assert np.all(f9[5:] == 0.0)


def test_mhd_induction_flux_is_antisymmetric_and_psi_pair():
    """F^d_{B_k} = v_d B_k - v_k B_d: zero for k = d replaced by psi, F^d_psi = ch^2 B_d,
    and sum over the electric-field structure: F^x_{B_y} = -F^y_{B_x}."""
    w = _random_state(9)
    ch = 1.9
    fx, fy, fz = (orc.phys_flux(w, d, nvar=9, ch=ch) for d in range(3))
    assert fx[5] == w[8] and fy[6] == w[8] and fz[7] == w[8]
    assert fx[8] == pytest.approx(ch * ch * w[5])
    assert fx[6] == pytest.approx(-fy[5], rel=1e-14)
    assert fx[7] == pytest.approx(-fz[5], rel=1e-14)
    assert fy[7] == pytest.approx(-fz[6], rel=1e-14)


# ---------------------------------------------------------------------------
# uniform-grid integration (Sec. 4 MOL + Sec. 5.1 RK2)
# ---------------------------------------------------------------------------

SOD = (1.0, 0.0, 1.0, 0.125, 0.0, 0.1)


def _sod_l1(n, t_end, **kw):
    pb = ai.sod(n=n, ny=1, t_end=t_end)
    o = orc.Oracle(pb, **kw)
    steps = o.run_to(t_end)
    rho = o.cons(0)[0, 0, 0, :]
    x = np.arange(n) / n
    er, _, _ = rex.cell_average(x, x + 1.0 / n, t_end, 0.5, SOD)
    return np.abs(rho - er).mean(), steps


def test_sod_1d_matches_exact_solution_and_converges():
    e100, _ = _sod_l1(100, 0.14)       # the paper's Sec. 6.1 resolution and output time
    e400, _ = _sod_l1(400, 0.14)
    assert e100 < 8e-3
    assert e400 < 0.5 * e100


def test_sod_1d_llf_also_converges_but_is_more_diffusive():
    e_hll, _ = _sod_l1(200, 0.14)
    e_llf, _ = _sod_l1(200, 0.14, riemann=orc.LLF)
    assert e_llf < 1e-2
    assert e_hll <= e_llf


def test_sod_3d_single_patch_config():
    """32^3 single patch, outflow, CFL 0.4, to t = 0.2: every (y, z) column equals the
    others bit-for-bit and matches the exact solution."""
    pb = ai.sod(n=32)
    o = orc.Oracle(pb)
    steps = o.run_to(0.2)
    u = o.cons(0)
    assert np.all(u == u[:, :1, :1, :])
    x = np.arange(32) / 32
    er, eu, ep = rex.cell_average(x, x + 1 / 32, 0.2, 0.5, SOD)
    assert np.abs(u[0, 0, 0] - er).mean() < 0.02
    assert 20 <= steps <= 80


def test_sod_axis_permutation_is_bitwise():
    prof = []
    for axis in range(3):
        pb = ai.sod(n=32, axis=axis, ny=4)
        o = orc.Oracle(pb)
        for _ in range(10):
            o.step(0.004)
        u = o.cons(0)
        rho = np.moveaxis(u[0], 2 - axis, 2)[0, 0]
        mom = np.moveaxis(u[1 + axis], 2 - axis, 2)[0, 0]
        prof.append((rho, mom))
    for k in (1, 2):
        assert np.array_equal(prof[k][0], prof[0][0])
        assert np.array_equal(prof[k][1], prof[0][1])


def test_sod_mirror_symmetry():
    pb = ai.sod(n=64, ny=1)
    pm = ai.sod(n=64, ny=1)
    pm.prim[0] = pm.prim[0][:, :, :, ::-1].copy()
    o, om = orc.Oracle(pb), orc.Oracle(pm)
    for _ in range(30):
        o.step(0.002)
        om.step(0.002)
    u, um = o.cons(0), om.cons(0)
    np.testing.assert_allclose(u[0], um[0][:, :, ::-1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(u[1], -um[1][:, :, ::-1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(u[4], um[4][:, :, ::-1], rtol=0, atol=1e-12)


def test_advected_wave_is_second_order():
    errs = []
    for n in (32, 64, 128):
        pb = ai.advected_wave(n=n)
        o = orc.Oracle(pb)
        o.run_to(1.0)
        x = (np.arange(n) + 0.5) / n
        errs.append(np.abs(o.cons(0)[0, 0, 0] - (1 + 0.2 * np.sin(2 * np.pi * x))).mean())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= 1.8, (errs, orders)


def test_literal_full_slope_plm_is_not_second_order():
    """The printed PLM (full limited difference added at the face) is not a
    second-order scheme: on the same smooth problem its error does not shrink."""
    errs = []
    for n in (32, 64):
        pb = ai.advected_wave(n=n)
        o = orc.Oracle(pb, plm_literal=True)
        o.run_to(0.5)
        x = (np.arange(n) + 0.5) / n
        err = np.abs(o.cons(0)[0, 0, 0] - (1 + 0.2 * np.sin(2 * np.pi * (x - 0.5)))).mean()
        errs.append(err if np.isfinite(err) else np.inf)
    assert not (errs[1] < errs[0] / 3.0)


def test_uniform_state_is_preserved_bitwise_on_a_uniform_grid():
    patches = ai.uniform_patches((16, 16, 16), (8, 8, 8))
    pb = ai.uniform(patches, (16, 16, 16))
    o = orc.Oracle(pb)
    u0 = o.all_cons()
    for _ in range(3):
        o.step(0.01)
    for a, b in zip(u0, o.all_cons()):
        assert np.array_equal(a, b)


def test_periodic_conservation_uniform_grid():
    patches = ai.uniform_patches((16, 16, 16), (8, 8, 8))
    pb = ai.random_smooth(patches, (16, 16, 16), seed=3)
    o = orc.Oracle(pb)
    t0 = o.totals()
    for _ in range(4):
        o.step()
    t1 = o.totals()
    scale = np.abs(t0).max()
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0)
