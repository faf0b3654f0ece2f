#!/usr/bin/env python
"""Benchmark of the AMR finite-volume update on GB300.

Workload: 3D Euler, Kelvin-Helmholtz shear layer in a periodic 256^3 box tiled
by 512 patches of 32^3 (rho 2 / 1, vx +-0.5, p 2.5, seeded v_y noise), gamma
1.4, PLM (theta 1.5) + HLL + TVD-RK2, CFL 0.4 recomputed on the GPU every step.

One "step" = one full RK2 coarse step of every cell (16.8M cell-updates).
Headline `value`: batched FP32 path (one launch per kernel, CUDA-graph replay)
in cell-updates/s, device-timed with CUDA events on the solver's stream.
Also measured in the same run: the plain per-patch FP64 path and the batched
FP64 path (same metric), the per-class kernel times (CUDA events around every
launch) that give the stage kernel's HBM roofline fraction, the end-to-end
rate through the C ABI with host buffers, and the FP64 CPU oracle on the host
cores (`cpu_baseline`).

`--impl reference` times the oracle alone (the reference arm of this
benchmark), each step being one RK2 step of a 128^3 periodic sub-box of the
same workload.  Under torchrun every rank advances its own replica on its own
GPU (weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "cell-updates/s and % HBM roofline, batched FP32 vs plain FP64, 1 GB300"
UNIT = "cell-updates/s"
N = 256
TILE = 32


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(elapsed: float, units_per_rank: float, dist=None, device=None):
    """Whole-job throughput of independent replicas: every rank processed
    `units_per_rank` units; the job time is the slowest rank's time (max over
    ranks, all-reduced).  Returns (value, max_elapsed)."""
    ws = 1
    if dist is not None and dist.is_available() and dist.is_initialized():
        import torch
        ws = dist.get_world_size()
        t = torch.tensor([elapsed], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    return ws * units_per_rank / elapsed, elapsed


def stage_source_sha() -> str:
    """Hash of the stage kernel's source: kernels.cuh (all of it), physics.cuh and amr_types.h."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_0910_5547_gb300", "csrc")
    src = "".join(open(os.path.join(csrc, f)).read() for f in ("kernels.cuh", "physics.cuh", "amr_types.h"))
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def stage_profile():
    """From the committed ncu summary of the FP32 stage kernel on this workload, used only
    while the kernel source is the one that was profiled: DRAM bytes per stage-kernel launch
    (mean of stage 1 and stage 2) and warp instructions per cell-update (both stages)."""
    import re
    sha = stage_source_sha()
    out = {"traffic_per_launch": None, "warp_inst_per_cell_update": None}
    try:
        txt = open(os.path.join(ROOT, "profiles", "stage_kernel_fp32_kh256.md")).read()
    except OSError:
        return out
    m = re.search(r"source_sha=(\w+) traffic_per_launch=(\d+)", txt)
    if m and m.group(1) == sha:
        out["traffic_per_launch"] = int(m.group(2))
        k = re.search(r"warp_inst_per_cell_update=([0-9.]+)", txt)
        if k:
            out["warp_inst_per_cell_update"] = float(k.group(1))
    return out


def stage_traffic():
    return stage_profile()["traffic_per_launch"]


def turbulence_diagnostics(packed, n, gamma):
    """Mean Mach number |v| / c_s, magnetic energy sum B^2/2 dV and kinetic energy of a
    single-patch 9-variable state (unit box)."""
    import numpy as np
    u = packed.reshape(9, n, n, n)
    rho = u[0]
    v2 = (u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / rho ** 2
    b2 = u[5] ** 2 + u[6] ** 2 + u[7] ** 2
    p = (gamma - 1.0) * (u[4] - 0.5 * rho * v2 - 0.5 * b2)
    mach = float(np.mean(np.sqrt(v2 / (gamma * p / rho))))
    dv = 1.0 / n ** 3
    return mach, float(0.5 * b2.sum() * dv), float(0.5 * (rho * v2).sum() * dv)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for k, nm in enumerate(names):
                    if r[3 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(mx)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(sm)
        return out


def make_solver(pb, precision, batched, graph, stream, **kw):
    from paper_0910_5547_gb300 import Solver
    return Solver.from_problem(pb, precision=precision, batched=batched, use_graph=graph,
                               stream=stream.cuda_stream, **kw)


def timed_steps(torch, s, stream, steps, dt=0.0):
    """Device time of `steps` coarse steps with CUDA events on the solver's stream."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        s.step(dt, sync=False)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def parity_errors(got, ref):
    """Errors of single-level states against the oracle's, per variable over all
    cells: the vector-normalised L1 (momentum components against the momentum
    norm, as the parity tests assert for FP32) and the per-variable L1 and max
    (each variable against its own norm; a field that is zero in the problem
    against the density's)."""
    import numpy as np
    nv = ref[0].shape[0]
    num = np.zeros(nv)
    den = np.zeros(nv)
    mx = np.zeros(nv)
    rmx = np.zeros(nv)
    for g, r in zip(got, ref):
        d = np.abs(g - r).reshape(nv, -1)
        a = np.abs(r).reshape(nv, -1)
        num += d.sum(axis=1)
        den += a.sum(axis=1)
        mx = np.maximum(mx, d.max(axis=1))
        rmx = np.maximum(rmx, a.max(axis=1))
    ref_norm = den.copy()
    vden = den.copy()
    vden[1:4] = den[1:4].sum()
    den[den < 1e-12 * den[0]] = den[0]
    rmx[rmx < 1e-12 * rmx[0]] = rmx[0]
    return {"l1_vector_metric": float((num / vden).max()), "l1_per_variable": [float(x) for x in num / den],
            "max_per_variable": [float(x) for x in mx / rmx],
            "reference_l1_norm_per_variable": [float(x) for x in ref_norm]}


def chosen_tiling(report: str):
    """(max_wx, max_cols, zchunk, ctas_per_sm, persistent) of the candidate the autotuner kept."""
    import re
    lines = [l for l in report.splitlines() if l.startswith("tile ")]
    m = re.search(r"chosen: candidate (\d+)", report)
    if not m:
        return None
    line = lines[int(m.group(1))]
    t = re.match(r"tile wx<=(\d+) cols<=(\d+) z=(\d+) ctas/SM=(\d+)", line)
    return tuple(int(x) for x in t.groups()) + (1 if " persistent" in line else 0,) if t else None


def cpu_model():
    """CPU model string of the host (x86 'model name', else the Arm implementer/part codes)."""
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                fields.setdefault(k.strip(), v.strip())
    except OSError:
        return "unknown"
    if "model name" in fields:
        return fields["model name"]
    if "CPU part" in fields:
        return f"Arm implementer {fields.get('CPU implementer', '?')} part {fields['CPU part']}"
    return "unknown"


def cpu_baseline(steps, parity_steps, stream, tiling):
    """The FP64 oracle as it stands, all host cores, on a bounded sample: the first
    `steps` RK2 steps of the full 256^3 / 32^3-patch workload are timed.  The oracle
    then continues to `parity_steps` steps, and the same dt sequence (the oracle's
    CFL steps) runs through the library in FP32 and FP64, on the single 256^3 patch
    with the headline's tiling (the configuration `value` times) and on the 512
    patches of 32^3; every cell of their final states is compared with the oracle's."""
    import numpy as np

    import amr_inputs as ai
    import oracle as orc
    cores = len(os.sched_getaffinity(0))
    pb = ai.kelvin_helmholtz(N=N, tile=TILE)
    single = ai.kelvin_helmholtz(N=N, tile=None)
    assert all(np.array_equal(w, single.prim[0][:, p.lo[2]:p.lo[2] + p.n[2], p.lo[1]:p.lo[1] + p.n[1],
                                                 p.lo[0]:p.lo[0] + p.n[0]]) for p, w in zip(pb.patches, pb.prim))
    o = orc.Oracle(pb, nthreads=cores)
    t = time.perf_counter()
    dts = [o.step() for _ in range(steps)]
    dt = time.perf_counter() - t
    out = {"value": N ** 3 * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{steps} RK2 steps (CFL dt) of the full 256^3 periodic workload, 512 patches of 32^3, "
                     f"FP64, OpenMP over patches; {dt:.1f} s wall"}
    t = time.perf_counter()
    dts += [o.step() for _ in range(max(0, parity_steps - steps))]
    t_rest = time.perf_counter() - t
    ref = o.all_cons()
    del o
    parity = {"steps": len(dts), "dt": "the oracle's CFL steps (0.4), replayed by the GPU solvers",
              "oracle_s": round(dt + t_rest, 1)}
    for prec in ("fp32", "fp64"):
        for name, prob in (("single_256", single), ("tiled_512", pb)):
            s = make_solver(prob, prec, True, True, stream)
            if name == "single_256" and tiling and prec == "fp32":
                s.set_tiling(*tiling[:4])
                s.set_persistent(tiling[4])
            for d in dts:
                s.step(d, sync=False)
            s.check()
            got = s.all_cons()
            s.close()
            if name == "single_256":
                full = np.empty((5, N, N, N))
                for p, u in zip(pb.patches, ref):
                    full[:, p.lo[2]:p.lo[2] + p.n[2], p.lo[1]:p.lo[1] + p.n[1], p.lo[0]:p.lo[0] + p.n[0]] = u
                parity[f"{prec}_{name}"] = parity_errors(got, [full])
                del full
            else:
                parity[f"{prec}_{name}"] = parity_errors(got, ref)
            del got
    parity["tiling_single_256_fp32"] = list(tiling) if tiling else None
    out["parity"] = parity
    del ref
    # single thread: one RK2 step of a 128^3 sub-box of the same workload (same patches)
    sub = ai.kelvin_helmholtz(N=128, tile=TILE)
    o1 = orc.Oracle(sub, nthreads=1)
    t = time.perf_counter()
    o1.step()
    dt1 = time.perf_counter() - t
    del o1
    out["single_thread"] = {"value": 128 ** 3 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"1 RK2 step of a 128^3 periodic sub-box, 64 patches of 32^3; {dt1:.1f} s wall"}
    out["cpu_model"] = cpu_model()
    # the other workloads, one (coarse) step each, all cores
    per = {}
    for name, mk, dt, what in (
            ("sedov_4level", ai.sedov_amr, 2.0e-7, "one coarse step (15 level steps) of the static 4-level "
                                                   "Sedov hierarchy, dt 2e-7"),
            ("adaptive_initial", ai.blast_clumps, 0.0, "one coarse step of the adaptive workload's initial "
                                                      "6-level hierarchy (no regrid), CFL dt"),
            ("orszag_tang_192", lambda: ai.orszag_tang(N=192, tile=32), 0.0, "one RK2 step of GLM-MHD "
                                                                              "Orszag-Tang 192^3, CFL dt")):
        pbx = mk()
        ox = orc.Oracle(pbx, nthreads=cores)
        t = time.perf_counter()
        ox.step(dt)
        dtx = time.perf_counter() - t
        per[name] = {"value": pbx.cell_updates_per_coarse_step() / dtx, "unit": UNIT,
                     "sample": f"{what}; {dtx:.1f} s wall"}
        del ox, pbx
    out["per_config"] = per
    return out


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import amr_inputs as ai
    import oracle as orc
    oracle_cores = len(os.sched_getaffinity(0))
    # the sample box shrinks with the step count so that the run stays within minutes
    n = 128 if args.steps <= 300 else (96 if args.steps <= 1000 else 64)
    pb = ai.kelvin_helmholtz(N=n, tile=TILE)
    o = orc.Oracle(pb, nthreads=oracle_cores)
    for _ in range(args.warmup):
        o.step()
    t = time.perf_counter()
    for _ in range(args.steps):
        o.step()
    wall = time.perf_counter() - t
    value = n ** 3 * args.steps / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "kelvin_helmholtz_periodic_32^3_patches", "sample_box": f"{n}^3",
                   "full_box": f"{N}^3", "dt": "CFL 0.4 every step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_cores, "kind": "oracle",
                         "sample": f"each step = one RK2 step of a {n}^3 periodic sub-box of the 256^3 "
                                   f"Kelvin-Helmholtz workload (same 32^3 patches), FP64 oracle, OpenMP",
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--cpu-steps", type=int, default=8)
    ap.add_argument("--tiling", default="",
                    help="max_wx,max_cols,zchunk,ctas_per_sm,persistent for the headline solver instead of the "
                         "autotuner's choice (reproducible profiles)")
    ap.add_argument("--parity-steps", type=int, default=100,
                    help="RK2 steps of the full-size comparison with the oracle (the oracle's first --cpu-steps "
                         "steps are the timed CPU baseline)")
    ap.add_argument("--only", default="",
                    help="comma list of phases: fp32,tiled,fp64,fluxrec,weno3,plain,e2e,amr,amr32,mhd,adaptive (default: "
                         "all but amr32)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)

    from paper_0910_5547_gb300 import build as B
    from paper_0910_5547_gb300 import native as NV
    if rank == 0:
        B.build()
    if ws > 1:
        dist.barrier()

    import amr_inputs as ai
    phases = set(args.only.split(",")) if args.only else {"fp32", "tiled", "fp64", "plain", "e2e", "amr", "mhd",
                                                          "fluxrec", "weno3",
                                                          "adaptive"}
    single = ai.kelvin_helmholtz(N=N, tile=None)          # one 256^3 patch
    tiled = ai.kelvin_helmholtz(N=N, tile=TILE) if phases & {"tiled", "plain"} else None
    cells = N ** 3
    stream = torch.cuda.Stream()

    def barrier():
        if ws > 1:
            dist.barrier()

    def max_over_ranks(x):
        return aggregate(x, 1.0, dist if ws > 1 else None, device="cuda")[1]

    def rate(pb, precision, batched, graph, steps):
        so = make_solver(pb, precision, batched, graph, stream)
        if batched:
            so.autotune()
        for _ in range(2):
            so.step(0.0, sync=False)
        t = timed_steps(torch, so, stream, steps)
        so.check()
        so.close()
        return ws * cells * steps / max_over_ranks(t)

    # ---- headline: single-patch batched FP32, graph replay, CFL every step ----
    s = make_solver(single, "fp32", True, True, stream)
    if args.tiling:
        fixed = [int(x) for x in args.tiling.split(",")]
        s.set_tiling(*fixed[:4])
        s.set_persistent(fixed[4] if len(fixed) > 4 else 0)
        tune_report = ("tile wx<=%d cols<=%d z=%d ctas/SM=%d%s: fixed\nchosen: candidate 0\n"
                       % (*fixed[:4], " persistent" if len(fixed) > 4 and fixed[4] else ""))
    else:
        tune_report = s.autotune()
    for _ in range(args.warmup):
        s.step(0.0, sync=False)
    torch.cuda.synchronize()
    s.check()
    n0 = s.launches()
    tot0 = s.totals()
    barrier()
    with ClockSampler(local) as clk:
        elapsed = timed_steps(torch, s, stream, args.steps)
    barrier()
    launches = s.launches() - n0
    s.check()
    tot1 = s.totals()
    # median of single-step device times (graph replay, CUDA events per step), beside the mean
    per_step = [timed_steps(torch, s, stream, 1) * 1e3 for _ in range(max(5, min(args.steps, 30)))]
    # periodic box: mass, momentum and energy are conserved; drift of the FP32 state
    # over the timed steps, measured by the FP64 totals (momentum against its norm)
    scale = [abs(tot0[0]), max(abs(tot0[1]), abs(tot0[2]), abs(tot0[3]), abs(tot0[0])), 0, 0, abs(tot0[4])]
    drift = {k: float(abs(tot1[i] - tot0[i]) / scale[i]) for i, k in ((0, "mass"), (1, "x_momentum"), (4, "energy"))}
    value, elapsed = aggregate(elapsed, cells * args.steps, dist if ws > 1 else None, device="cuda")

    # ---- per-kernel event timing (eager launches, same solver and state) ----
    ksteps = max(3, min(args.steps, 20))
    NV.amr_set_timing(s.h, True)
    for _ in range(ksteps):
        s.step(0.0, sync=False)
    tm = NV.amr_get_timing(s.h)
    NV.amr_set_timing(s.h, False)
    V, W = 5, 4
    t1, c1 = tm["stage1"]
    t2, c2 = tm["stage2"]
    stage_bytes = (2 + 3) * V * W * cells            # stage 1: read U, write U1; stage 2: read U1, U, write U
    achieved = stage_bytes / ((t1 + t2) / ksteps / 1e3) / 1e9
    peak, peak_kind = peaks()
    step_kernel_ms = {k: round(v[0] / ksteps, 4) for k, v in tm.items() if v[1]}
    # issue ceiling: the profiled warp instructions per cell-update issued at one per cycle
    # by each of the 4 schedulers of every SM, at the median SM clock of the timed region
    prof = stage_profile()
    clocks = clk.summary()
    issue = None
    if prof["warp_inst_per_cell_update"] and clocks.get("sm_mhz"):
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        t_issue = prof["warp_inst_per_cell_update"] * cells / (sms * 4 * clocks["sm_mhz"] * 1e6)
        t_stage = (t1 + t2) / ksteps / 1e3
        issue = {"warp_inst_per_cell_update": prof["warp_inst_per_cell_update"], "sms": sms,
                 "sm_mhz": clocks["sm_mhz"], "min_stage_ms_per_step": t_issue * 1e3,
                 "frac": t_issue / t_stage,
                 "note": "stage 1 + stage 2 time at one warp instruction per cycle per scheduler "
                         "(instruction count from the committed ncu capture) over the measured time"}
    alu = NV.amr_peak_fma_rates()
    s.close()

    sub = min(args.steps, 200)   # step counts of the other workloads follow this, not the headline's
    e2e = None
    if "e2e" in phases:
        # end to end through the C ABI: every step uploads its input state (FP64, pinned)
        # and downloads its result; the uploads and downloads run on the library's copy
        # streams beside the steps (three steps in flight, three host buffers per
        # direction).  Measured before the other workloads build and free tens of GB of
        # host arrays: pinned buffers allocated after that moved data markedly slower on
        # the same box.
        s = make_solver(single, "fp32", True, True, stream)
        nstate = NV.amr_state_size(s.h)
        depth = 3
        h_in = [torch.empty(nstate, dtype=torch.float64, pin_memory=True).numpy() for _ in range(depth)]
        h_out = [torch.empty(nstate, dtype=torch.float64, pin_memory=True).numpy() for _ in range(depth)]
        h_in[0][:] = s.state_all()
        for b in h_in[1:]:
            b[:] = h_in[0]
        ke = max(3, min(args.steps, 20))

        def e2e_steps(n):
            tickets = []
            for k in range(n):
                if k >= depth:
                    NV.amr_wait_state(s.h, tickets[k - depth])   # buffers k % depth are free again
                NV.amr_set_state_async(s.h, h_in[k % depth], NV.AMR_STATE_CONSERVED)
                s.step(0.0, sync=False)
                tickets.append(NV.amr_get_state_all_async(s.h, h_out[k % depth]))
            for t in tickets[-depth:]:
                NV.amr_wait_state(s.h, t)

        e2e_steps(3)
        barrier()
        t = time.perf_counter()
        e2e_steps(ke)
        e2e_t = max_over_ranks(time.perf_counter() - t)
        s.check()
        s.close()
        e2e = {"value": ws * cells * ke / e2e_t, "unit": UNIT, "h2d_bytes_per_step": nstate * 8,
               "d2h_bytes_per_step": nstate * 8, "steps": ke,
               "note": "per step: packed FP64 conserved state host->device (pinned), one RK2 step (CFL), "
                       "state device->host, through amr_set_state_async / amr_step / amr_get_state_all_async; "
                       "copies of neighbouring steps overlap on the library's copy streams"}

    extra = {}
    k64 = max(3, sub // 10)
    if "tiled" in phases:
        extra["fp32_tiled_512"] = {"value": rate(tiled, "fp32", True, True, sub), "unit": UNIT,
                                   "workload": "same box as 512 patches of 32^3, batched launches + graph"}
    if "fp64" in phases:
        extra["fp64_batched"] = {"value": rate(single, "fp64", True, True, k64), "unit": UNIT, "steps": k64,
                                 "workload": "single 256^3 patch, batched + graph"}
    if "weno3" in phases:
        # third-order WENO face states (recon = weno3) on the same single 256^3 patch
        so = make_solver(single, "fp32", True, True, stream, recon="weno3")
        so.autotune()
        for _ in range(2):
            so.step(0.0, sync=False)
        kw3 = max(3, sub)
        with ClockSampler(local) as clk3:
            tw3 = timed_steps(torch, so, stream, kw3)
        NV.amr_set_timing(so.h, True)
        for _ in range(ksteps):
            so.step(0.0, sync=False)
        tmw = NV.amr_get_timing(so.h)
        NV.amr_set_timing(so.h, False)
        so.check()
        so.close()
        tsw = (tmw["stage1"][0] + tmw["stage2"][0]) / ksteps
        extra["weno3_fp32"] = {
            "value": ws * cells * kw3 / max_over_ranks(tw3), "unit": UNIT, "steps": kw3,
            "stage_ms": {"stage1": round(tmw["stage1"][0] / ksteps, 4), "stage2": round(tmw["stage2"][0] / ksteps, 4)},
            "stage_hbm_frac": stage_bytes / (tsw / 1e3) / 1e9 / peak, "clocks": clk3.summary(),
            "workload": "Kelvin-Helmholtz 256^3 single patch, FP32, HLL on third-order WENO face states "
                        "(recon=weno3), batched + graph"}

    if "fluxrec" in phases:
        # the direct flux reconstruction variant (Sec. 4's second class of schemes) on the
        # same single 256^3 patch: rate with graph replay, stage-kernel event times
        so = make_solver(single, "fp32", True, True, stream, riemann="fluxrec")
        so.autotune()
        for _ in range(2):
            so.step(0.0, sync=False)
        kf = max(3, sub // 4)
        tf = timed_steps(torch, so, stream, kf)
        NV.amr_set_timing(so.h, True)
        for _ in range(ksteps):
            so.step(0.0, sync=False)
        tmf = NV.amr_get_timing(so.h)
        NV.amr_set_timing(so.h, False)
        so.check()
        so.close()
        tsf = (tmf["stage1"][0] + tmf["stage2"][0]) / ksteps
        extra["fluxrec_fp32"] = {
            "value": ws * cells * kf / max_over_ranks(tf), "unit": UNIT, "steps": kf,
            "stage_ms": {"stage1": round(tmf["stage1"][0] / ksteps, 4), "stage2": round(tmf["stage2"][0] / ksteps, 4)},
            "stage_hbm_frac": stage_bytes / (tsf / 1e3) / 1e9 / peak,
            "workload": "Kelvin-Helmholtz 256^3 single patch, FP32, riemann=fluxrec (Lax-Friedrichs split fluxes "
                        "reconstructed by PLM), batched + graph"}
    if "plain" in phases:
        plain = "512 patches of 32^3, one stage-kernel and ghost-copy launch per patch, no graph"
        extra["fp64_plain"] = {"value": rate(tiled, "fp64", False, False, k64), "unit": UNIT, "steps": k64,
                               "workload": plain}
        extra["fp32_plain"] = {"value": rate(tiled, "fp32", False, False, k64), "unit": UNIT, "steps": k64,
                               "workload": plain}
        extra["fp64_batched_tiled_512"] = {"value": rate(tiled, "fp64", True, True, k64), "unit": UNIT,
                                           "steps": k64, "workload": "512 patches of 32^3, batched + graph"}
        if "fp32_tiled_512" in extra:
            b32, p32 = extra["fp32_tiled_512"]["value"], extra["fp32_plain"]["value"]
            b64, p64 = extra["fp64_batched_tiled_512"]["value"], extra["fp64_plain"]["value"]
            extra["batched_fp32_over_plain_fp64"] = b32 / p64
            extra["speedup_decomposition_kh512"] = {
                "batched_fp32_over_plain_fp64": b32 / p64,
                "batching_at_fp32": b32 / p32, "batching_at_fp64": b64 / p64,
                "precision_batched": b32 / b64, "precision_plain": p32 / p64,
                "note": "batched FP32 / plain FP64 = batching x precision, taken in either order"}

    def amr_rates(pb, label, fp64_plain_steps=1):
        """Cell-updates/s (sum over levels of cells_l 2^l per coarse step) of the batched FP32
        path and the plain per-patch FP64 path on a multi-level hierarchy, plus kernel-class times."""
        cu = pb.cell_updates_per_coarse_step()
        so = make_solver(pb, "fp32", True, True, stream)
        chosen = chosen_tiling(so.autotune())
        for _ in range(2):
            so.step(0.0, sync=False)
        ka = max(3, sub // 20)
        t = timed_steps(torch, so, stream, ka)
        NV.amr_set_timing(so.h, True)
        for _ in range(2):
            so.step(0.0, sync=False)
        tmk = NV.amr_get_timing(so.h)
        NV.amr_set_timing(so.h, False)
        so.check()
        so.close()
        value = ws * cu * ka / max_over_ranks(t)
        bpc = 5 * pb.nvar * 4              # algorithmic bytes per cell-update, FP32
        out = {"value": value, "unit": UNIT, "steps": ka, "patches": len(pb.patches),
               "levels": pb.nlevels, "cell_updates_per_coarse_step": cu,
               "class_ms_per_coarse_step": {k: round(v[0] / 2, 3) for k, v in tmk.items() if v[1]},
               "roofline": {"bound": "hbm", "achieved": value / ws * bpc / 1e9, "peak": peak, "unit": "GB/s",
                            "frac": value / ws * bpc / 1e9 / peak, "peak_kind": peak_kind,
                            "algorithmic_bytes_per_cell_update": bpc,
                            "note": "whole coarse step (every kernel class) against the interior cell-updates' "
                                    "algorithmic bytes"},
               "workload": label}
        if chosen:
            # the other stage launch form (persistent CTAs or one CTA per work item), same tiling
            so = make_solver(pb, "fp32", True, True, stream)
            so.set_tiling(*chosen[:4])
            so.set_persistent(1 - chosen[4])
            for _ in range(2):
                so.step(0.0, sync=False)
            t_other = timed_steps(torch, so, stream, ka)
            so.check()
            so.close()
            out["launch_form"] = {"chosen": "persistent" if chosen[4] else "one CTA per item",
                                  "tiling": list(chosen[:4]),
                                  "other_form_value": ws * cu * ka / max_over_ranks(t_other)}
            # the same step on one stream (no second stream for the stage-2 parent fill and the registers)
            so = make_solver(pb, "fp32", True, True, stream)
            so.set_tiling(*chosen[:4])
            so.set_persistent(chosen[4])
            so.set_overlap(False)
            for _ in range(2):
                so.step(0.0, sync=False)
            t_one = timed_steps(torch, so, stream, ka)
            so.check()
            so.close()
            out["one_stream_value"] = ws * cu * ka / max_over_ranks(t_one)
        if fp64_plain_steps:
            def one(precision, batched, steps):
                sp = make_solver(pb, precision, batched, batched, stream)
                sp.step(0.0, sync=False)
                tp = timed_steps(torch, sp, stream, steps)
                sp.check()
                sp.close()
                return ws * cu * steps / max_over_ranks(tp)
            out["fp64_plain"] = one("fp64", False, fp64_plain_steps)
            out["fp32_plain"] = one("fp32", False, 1)
            out["fp64_batched"] = one("fp64", True, 2)
            out["batched_fp32_over_plain_fp64"] = value / out["fp64_plain"]
            out["speedup_decomposition"] = {
                "batching_at_fp32": value / out["fp32_plain"], "batching_at_fp64": out["fp64_batched"] / out["fp64_plain"],
                "precision_batched": value / out["fp64_batched"], "precision_plain": out["fp32_plain"] / out["fp64_plain"]}
        return out

    if "amr" in phases or "amr32" in phases:
        extra["amr_static_sedov"] = amr_rates(
            ai.sedov_amr(), "static 4-level Sedov hierarchy, base 128^3, seeded 8-32 patches, outflow",
            fp64_plain_steps=1 if "amr" in phases else 0)
    if "adaptive" in phases:
        pb = ai.blast_clumps()
        rkw = dict(threshold=0.3, buffer=4, block=4, max_patch=32)
        lmax = pb.max_level

        def adaptive_start():
            so = make_solver(pb, "fp32", True, True, stream)
            so.autotune()
            so.step(0.0)
            so.regrid(**rkw)
            NV.amr_get_regrid_timing(so.h)        # reset the phase sums
            return so

        # (1) the workload's cadence: after every step of a level <= L_max - 2 (every 4 finest
        # steps) the finer levels are rebuilt inside the coarse step
        so = adaptive_start()
        so.set_regrid_schedule(lmax - 2, **rkw)
        c0 = NV.amr_cell_updates(so.h)
        t_sched = timed_steps(torch, so, stream, 4)
        cu_sched = NV.amr_cell_updates(so.h) - c0
        ph_sched = NV.amr_get_regrid_timing(so.h)
        counts_sched = NV.amr_get_regrid_counts(so.h)
        sched_shape = [len(so.patches), 1 + max(p.level for p in so.patches)]
        so.check()
        so.close()
        # (2) regrid between coarse steps only (graph replay inside each step)
        so = adaptive_start()
        tot_cu, t_steps, t_regrid, counts = 0, 0.0, 0.0, []
        phases_s = {k: 0.0 for k in NV.REGRID_PHASES}
        for _ in range(4):
            c0 = NV.amr_cell_updates(so.h)
            t_steps += timed_steps(torch, so, stream, 1)
            tot_cu += NV.amr_cell_updates(so.h) - c0
            t0 = time.perf_counter()
            so.regrid(**rkw)
            t_regrid += time.perf_counter() - t0
            for k, v in NV.amr_get_regrid_timing(so.h).items():
                phases_s[k] += v
            counts.append([len(so.patches), 1 + max(p.level for p in so.patches)])
        # kernel classes of one eager coarse step on the final (11k-patch) hierarchy
        NV.amr_set_timing(so.h, True)
        so.step(0.0, sync=False)
        tm_ad = NV.amr_get_timing(so.h)
        NV.amr_set_timing(so.h, False)
        so.check()
        so.close()
        rg_s = sum(ph_sched.values())
        extra["adaptive_blast_clumps"] = {
            "value_with_regrid": ws * cu_sched / max_over_ranks(t_sched),
            "value": ws * cu_sched / max_over_ranks(max(t_sched - rg_s, 1e-9)), "unit": UNIT,
            "coarse_steps": 4, "cell_updates": cu_sched, "regrid_s": rg_s,
            "regrid_phases_s": {k: round(v, 4) for k, v in ph_sched.items()},
            "regrids_new_unchanged_memo": list(counts_sched),
            "patches_levels_at_end": sched_shape,
            "regrid_between_coarse_steps": {
                "value": ws * tot_cu / max_over_ranks(t_steps),
                "value_with_regrid": ws * tot_cu / max_over_ranks(t_steps + t_regrid), "cell_updates": tot_cu,
                "regrid_s": t_regrid, "regrid_phases_s": {k: round(v, 4) for k, v in phases_s.items()},
                "class_ms_one_coarse_step_final_hierarchy": {k: round(v[0], 3) for k, v in tm_ad.items() if v[1]},
                "patches_levels_after_each_regrid": counts},
            "workload": f"blast in a log-normal clump field (sigma 1), base 64^3 + {lmax} levels, FP32 batched, "
                        f"density-gradient regrid (threshold 0.3) of the levels above l after every step of "
                        f"a level l <= {lmax - 2} (every 4 finest steps); 'value' excludes the host regrid time"}
    if "mhd" in phases:
        ot = ai.orszag_tang(N=192, tile=None)
        mhd = {"fp32_uniform_192": rate(ot, "fp32", True, True, max(3, sub // 4)) * (192 ** 3) / cells}
        del ot
        mhd["fp32_over_hydro_fp32_per_cell"] = mhd["fp32_uniform_192"] / value
        # Sec. 7 decaying turbulence: 128^3, Mach 10, gamma 1.001, beta 0.1, with the
        # paper's two diagnostics (mean Mach number, magnetic energy) around the timed steps
        turb = ai.mhd_turbulence(N=128)
        so = make_solver(turb, "fp32", True, True, stream)
        so.autotune()
        d0 = turbulence_diagnostics(so.state_all(), 128, turb.gamma)
        b0 = so.divb_norms()
        for _ in range(2):
            so.step(0.0, sync=False)
        kt = max(3, sub // 4)
        tt = timed_steps(torch, so, stream, kt)
        so.check()
        d1 = turbulence_diagnostics(so.state_all(), 128, turb.gamma)
        b1 = so.divb_norms()
        so.close()
        mhd["turbulence_128"] = {"value": ws * 128 ** 3 * kt / max_over_ranks(tt), "unit": UNIT, "steps": kt,
                                 "mean_mach": [d0[0], d1[0]], "magnetic_energy": [d0[1], d1[1]],
                                 "kinetic_energy": [d0[2], d1[2]],
                                 "divb_l1_over_b_l1": [b0[0] / b0[2], b1[0] / b1[2]],
                                 "divb_max_over_b_max": [b0[1] / b0[3], b1[1] / b1[3]],
                                 "workload": "decaying MHD turbulence 128^3, Mach 10, gamma 1.001, beta 0.1, "
                                             "P(k) ~ k^-2 (seeded); diagnostics before and after the "
                                             f"{kt + 2} steps"}
        del turb
        mhd["amr_3level"] = amr_rates(ai.orszag_tang(amr_sides=(96, 96), amr_base=96),
                                      "GLM-MHD Orszag-Tang, 3 levels, base 96^3", fp64_plain_steps=0)
        mhd["unit"] = UNIT
        extra["mhd_orszag_tang"] = mhd

    if rank != 0:
        return
    cpu = None if args.no_cpu else cpu_baseline(args.cpu_steps, max(args.parity_steps, args.cpu_steps), stream,
                                                chosen_tiling(tune_report))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "kelvin_helmholtz_256^3_periodic", "cells": cells, "patches": 1,
                   "path": "batched FP32, CUDA graph per coarse step",
                   "dt": "CFL 0.4 recomputed on the GPU every step",
                   "l2": "working set (U + U1, 0.7 GB FP32) exceeds the 129 MB L2; no flush",
                   "parallelism": f"replicas x{ws}"},
        **extra,
        "roofline": {"bound": "hbm", "kernel": "stage_kernel (stage 1 + stage 2)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": stage_traffic(),
                     "algorithmic_per_launch": stage_bytes // 2,
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_cell_update": (2 + 3) * V * W,
                     "note": "achieved = algorithmic bytes of the stage-1 and stage-2 launches over their summed "
                             "CUDA-event durations; traffic = mean DRAM bytes per launch from the committed ncu "
                             "capture (null if the kernel source changed since)",
                     "timed_steps": ksteps,
                     "frac_of_nominal_7900": achieved / 7900.0,
                     "traffic_bytes_per_cell_update": (None if stage_traffic() is None
                                                       else 2 * stage_traffic() / cells),
                     "issue_ceiling": issue,
                     "alu_peaks_tflops": {"fp32_fma": alu["fp32_flops"] / 1e12,
                                          "fp64_fma": alu["fp64_flops"] / 1e12}},
        "step_ms_median": statistics.median(per_step),
        "step_kernel_ms": step_kernel_ms,
        "autotune": [l for l in tune_report.splitlines() if l],
        "cell_update_roofline_frac": value / ws * (2 + 3) * V * W / (peak * 1e9),
        "conservation_drift": {**drift, "steps": args.steps, "note": "relative change of the FP64 totals of "
                               "the FP32 state over the timed steps (periodic box)"},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "parity": None if cpu is None else cpu.pop("parity"),
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
