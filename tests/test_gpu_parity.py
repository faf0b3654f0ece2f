"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs, at sizes the oracle finishes in seconds that still span
several tiles and ragged patches.  FP64: L1 rel <= 1e-10 and max rel <= 1e-8;
FP32: L1 rel <= 2e-5."""
import numpy as np
import pytest

import amr_inputs as ai
import oracle as orc
from parity import assert_parity, errors
from test_oracle_amr_mhd import three_level_seeded, two_level

pytestmark = pytest.mark.gpu

from paper_0910_5547_gb300 import Solver  # noqa: E402
from paper_0910_5547_gb300 import build as B  # noqa: E402
from paper_0910_5547_gb300 import native as N  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    N.load()
    yield


def run_pair(pb, precision, steps=None, dt=None, t_end=None, **kw):
    """Advance the oracle and the GPU solver side by side; each takes its own CFL step
    unless dt is given."""
    o = orc.Oracle(pb, nthreads=8, **{k: v for k, v in kw.items() if k in ("riemann", "theta", "ch", "cfl")})
    skw = {k: v for k, v in kw.items() if k in ("theta", "ch", "cfl", "batched", "use_graph")}
    if "riemann" in kw:
        skw["riemann"] = "llf" if kw["riemann"] == orc.LLF else "hll"
    s = Solver.from_problem(pb, precision=precision, **skw)
    if t_end is not None:
        n_o = o.run_to(t_end)
        n_s = s.run_to(t_end)
        assert n_o == n_s, (n_o, n_s)
    else:
        for _ in range(steps):
            o.step(dt or 0.0)
            s.step(dt or 0.0)
    s.check()
    return o, s


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sod_single_patch_to_t02(precision):
    pb = ai.sod(n=32)
    o, s = run_pair(pb, precision, t_end=0.2)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "sod32")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sod_llf_variant(precision):
    pb = ai.sod(n=32, axis=1)
    o, s = run_pair(pb, precision, steps=10, dt=0.004, riemann=orc.LLF)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "sod-llf")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_kelvin_helmholtz_tiled(precision):
    pb = ai.kelvin_helmholtz(N=64, tile=16)
    o, s = run_pair(pb, precision, steps=5)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "kh64")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ragged_patches_mixed_boundaries(precision):
    base = (40, 24, 20)
    patches = ai.uniform_patches(base, (16, 16, 16))
    pb = ai.random_smooth(patches, base, seed=17, bc=(1, 1, 0, 0, 1, 1), amp=0.3)
    o, s = run_pair(pb, precision, steps=4)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "ragged")


@pytest.mark.parametrize("theta", [1.0, 2.0])
def test_theta_values(theta):
    base = (24, 24, 24)
    patches = ai.uniform_patches(base, (12, 12, 12))
    pb = ai.random_smooth(patches, base, seed=23, amp=0.4)
    o, s = run_pair(pb, "fp64", steps=3, theta=theta)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, "fp64", f"theta{theta}")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("bc", [ai.PERIODIC, ai.OUTFLOW])
def test_two_level_amr(precision, bc):
    pb = ai.random_smooth(two_level(), (16,) * 3, seed=9, amp=0.2, bc=(bc,) * 6)
    o, s = run_pair(pb, precision, steps=3)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "amr2")
    np.testing.assert_allclose(s.totals(), o.totals(), rtol=1e-12 if precision == "fp64" else 1e-5, atol=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_three_level_amr_parity_and_conservation(precision):
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, seed=5, amp=0.2)
    t0 = Solver.from_problem(pb, precision=precision).totals()
    # the GPU's initial totals (its own primitive -> conserved conversion) against the oracle's;
    # the oracle adds the cells one after another (error bound (N-1) u, 3.6e-12 relative for
    # 32^3 cells), the GPU in a fixed tree
    t0_o = orc.Oracle(pb).totals()
    np.testing.assert_allclose(t0, t0_o, rtol=0, atol=(4e-12 if precision == "fp64" else 1e-7) * np.abs(t0_o).max())
    o, s = run_pair(pb, precision, steps=2)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "amr3")
    t1 = s.totals()
    scale = np.abs(t0).max()
    rt = 2e-14 if precision == "fp64" else 2e-6
    assert np.all(np.abs(t1 - t0) <= rt * scale), (t1 - t0)
    np.testing.assert_allclose(t1, o.totals(), rtol=0, atol=(1e-12 if precision == "fp64" else 1e-5) * scale)


def test_sedov_small_hierarchy_outflow():
    pb = ai.sedov_amr(base=32, sides=(32, 32), seed=3)
    o, s = run_pair(pb, "fp64", steps=2)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, "fp64", "sedov-small")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_orszag_tang_mhd(precision):
    pb = ai.orszag_tang(N=32, tile=16)
    t0 = Solver.from_problem(pb, precision=precision).totals()
    t0_o = orc.Oracle(pb).totals()   # summation orders differ, as above
    np.testing.assert_allclose(t0, t0_o, rtol=0, atol=(4e-12 if precision == "fp64" else 1e-7) * np.abs(t0_o).max())
    o, s = run_pair(pb, precision, steps=4)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "ot32")
    scale = np.abs(t0).max()
    np.testing.assert_allclose(s.totals(), t0, rtol=0, atol=(2e-14 if precision == "fp64" else 1e-6) * scale)
    np.testing.assert_allclose(s.totals(), o.totals(), rtol=0, atol=(1e-12 if precision == "fp64" else 1e-5) * scale)


def test_mhd_amr_fp64():
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, nvar=9, seed=8, amp=0.2)
    o, s = run_pair(pb, "fp64", steps=2)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, "fp64", "mhd-amr3")


def test_brio_wu_quasi_1d():
    pb = ai.brio_wu(n=128, ny=2)
    o, s = run_pair(pb, "fp64", t_end=0.05)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, "fp64", "brio-wu")
    u = s.cons(0)
    assert np.all(u[5] == 0.75) and np.all(u[8] == 0.0)


def test_uniform_state_exact_on_amr_fp32():
    pb = ai.uniform(two_level(), (16,) * 3, bc=(ai.PERIODIC,) * 6)
    s = Solver.from_problem(pb, precision="fp32")
    u0 = s.state_all()
    for _ in range(3):
        s.step(0.01)
    assert np.array_equal(s.state_all(), u0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_plain_and_batched_and_graph_are_bitwise_equal(precision):
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, seed=12, amp=0.2)
    outs = []
    for batched, graph in ((True, True), (True, False), (False, False)):
        s = Solver.from_problem(pb, precision=precision, batched=batched, use_graph=graph)
        for _ in range(2):
            s.step()
        outs.append(s.state_all())
        s.close()
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])


def test_checkpoint_roundtrip_is_bitwise():
    pb = ai.random_smooth(two_level(), (16,) * 3, seed=4, amp=0.2)
    s = Solver.from_problem(pb, precision="fp64")
    s.step()
    snap = s.state_all().copy()
    s.step()
    after = s.state_all().copy()
    s2 = Solver.from_problem(pb, precision="fp64")
    s2.set_state(snap)
    assert np.array_equal(s2.state_all(), snap)
    s2.step()
    assert np.array_equal(s2.state_all(), after)


def test_nonphysical_input_is_rejected():
    pb = ai.sod(n=16)
    pb.prim[0][4, 3, 3, 3] = -1.0
    with pytest.raises(N.AmrError) as e:
        Solver.from_problem(pb)
    assert e.value.status == N.AMR_ERR_NONPHYSICAL
    pb.prim[0][4, 3, 3, 3] = np.nan
    with pytest.raises(N.AmrError) as e:
        Solver.from_problem(pb)
    assert e.value.status == N.AMR_ERR_NONPHYSICAL


def test_nonphysical_state_during_step_is_reported():
    """A host-injected state with negative internal energy is flagged by the kernels
    (no device fault: the flag is a status word read after the step)."""
    pb = ai.sod(n=16)
    s = Solver.from_problem(pb)
    flat = s.state_all()
    flat[4 * 16 ** 3 + 100] = 0.0          # rho E = 0 with rho > 0: e = 0 -> non-physical
    s.set_state(flat, kind=N.AMR_STATE_CONSERVED)
    with pytest.raises(N.AmrError) as e:
        s.check()
    assert e.value.status == N.AMR_ERR_NONPHYSICAL


def test_state_calls_before_set_patches_fail_cleanly():
    c = N.amr_default_config()
    h = N.amr_create(c)
    try:
        with pytest.raises(N.AmrError) as e:
            N.amr_step(h, 0.1)
        assert e.value.status == N.AMR_ERR_STATE
        for call in (lambda: N.amr_divb_norms(h), lambda: N.amr_set_state_async(h, np.zeros(8)),
                     lambda: N.amr_get_state_all_async(h, np.zeros(8)), lambda: N.amr_conserved_totals(h, 5)):
            with pytest.raises(N.AmrError) as e:
                call()
            assert e.value.status == N.AMR_ERR_STATE
        with pytest.raises(N.AmrError) as e:
            N.amr_wait_state(h, 0)                 # no download was issued
        assert e.value.status == N.AMR_ERR_ARG
    finally:
        N.amr_destroy(h)


def test_kernel_launch_counter_counts_graph_nodes():
    pb = ai.kelvin_helmholtz(N=32, tile=16)
    s = Solver.from_problem(pb, precision="fp32")
    n0 = s.launches()
    s.step(0.001, sync=False)
    s.step(0.001, sync=False)
    s.check()
    per = (s.launches() - n0) / 2
    assert per >= 5            # set_dt + 2 x (ghost copy + stage)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_autotune_keeps_results_and_reports_candidates(precision):
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, seed=14, amp=0.2)
    s = Solver.from_problem(pb, precision=precision)
    u0 = s.state_all().copy()
    rep = s.autotune()
    assert np.array_equal(s.state_all(), u0)            # tuning does not touch the state
    lines = [l for l in rep.splitlines() if l.startswith("tile")]
    assert len(lines) >= 4 and "chosen" in rep
    o = orc.Oracle(pb, nthreads=8)
    for _ in range(2):
        o.step()
        s.step()
    s.check()
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "autotuned")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mhd_turbulence_parity(precision):
    """Sec. 7 decaying MHD turbulence (Mach 10, gamma 1.001, beta 0.1) at 32^3 in 16^3
    patches, three CFL steps."""
    pb = ai.mhd_turbulence(N=32, tile=16)
    o, s = run_pair(pb, precision, steps=3)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "mhd-turbulence")


def test_mhd_turbulence_decays_in_one_crossing_time():
    """Sec. 7: a significant fraction of the turbulent kinetic energy decays within one
    dynamical (flow crossing) time L / v_rms = 0.1; FP32 batched at 32^3."""
    pb = ai.mhd_turbulence(N=32, tile=16)
    s = Solver.from_problem(pb, precision="fp32")

    def kinetic():
        return sum(float(np.sum(0.5 * (u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / u[0])) for u in s.all_cons())

    k0 = kinetic()
    n = s.run_to(0.1)
    s.check()
    assert n > 50
    assert kinetic() < 0.6 * k0


def test_torch_allocator_path_is_bitwise_and_accounted():
    """Device memory taken from PyTorch's caching allocator (amr_config.dev_alloc /
    dev_free): the same bits as the library's own stream-ordered allocations, the
    arena shows up in torch's accounting, and is returned by close() and by a regrid."""
    import torch
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, seed=4)
    base = torch.cuda.memory_allocated()
    s_t = Solver.from_problem(pb, precision="fp32", allocator="torch")
    held = torch.cuda.memory_allocated() - base
    cells = sum(p.n[0] * p.n[1] * p.n[2] for p in pb.patches)
    assert held > 2 * 5 * 4 * cells          # at least U and U1
    s_d = Solver.from_problem(pb, precision="fp32")
    for _ in range(2):
        s_t.step(0.0)
        s_d.step(0.0)
    for a, b in zip(s_t.all_cons(), s_d.all_cons()):
        assert np.array_equal(a, b)
    s_t.regrid(threshold=0.05, buffer=2, block=4, max_patch=16)
    s_t.step(0.0)
    s_t.check()
    s_t.close()
    s_d.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


@pytest.mark.parametrize("graph", [True, False])
def test_cell_update_counter(graph):
    """amr_cell_updates: each coarse step adds sum_l cells_l 2^l, with graph replay and eagerly."""
    pb = ai.random_smooth(three_level_seeded(), (32,) * 3, seed=4)
    s = Solver.from_problem(pb, precision="fp32", use_graph=graph)
    per_step = sum((p.n[0] * p.n[1] * p.n[2]) << p.level for p in pb.patches)
    c0 = N.amr_cell_updates(s.h)
    for _ in range(3):
        s.step(0.0, sync=False)
    s.check()
    assert N.amr_cell_updates(s.h) - c0 == 3 * per_step


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_concave_fine_region_and_one_cell_gap(precision):
    """Coarse cells with several flux registers: an L-shaped fine region (the
    coarse cells in its inner corner border fine patches along x and along y)
    and two fine patches one coarse cell apart (that cell borders both along x).
    Their refluxes apply in (axis, side) order; parity with the oracle and
    conservation on the periodic box."""
    patches = ai.uniform_patches((16, 16, 16), (8, 8, 8))
    patches += [ai.Patch(1, (8, 8, 8), (8, 8, 8)), ai.Patch(1, (16, 8, 8), (8, 8, 8)),
                ai.Patch(1, (8, 16, 8), (8, 8, 8)),
                ai.Patch(1, (0, 0, 24), (8, 8, 4)), ai.Patch(1, (10, 0, 24), (8, 8, 4))]
    pb = ai.random_smooth(patches, (16,) * 3, seed=14, amp=0.25)
    t0 = Solver.from_problem(pb, precision=precision).totals()
    o, s = run_pair(pb, precision, steps=3)
    assert_parity(s.all_cons(), o.all_cons(), pb.patches, precision, "concave+gap")
    t1 = s.totals()
    scale = np.abs(t0).max()
    assert np.all(np.abs(t1 - t0) <= (2e-14 if precision == "fp64" else 2e-6) * scale), (t1 - t0)
