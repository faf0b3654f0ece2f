"""ctypes binding of the C ABI in include/amr.h (argument marshalling only).

Every function has the name of the C entry point it wraps.  Non-OK statuses
raise ``AmrError`` (carrying ``.status`` and the library's message).  The
shared library must have been built (``paper_0910_5547_gb300.build.build()``);
there is no fallback of any kind when it is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, List, Sequence

import numpy as np

from . import build as _build

AMR_OK = 0
AMR_ERR_ARG = -1
AMR_ERR_NESTING = -2
AMR_ERR_CUDA = -3
AMR_ERR_NONPHYSICAL = -4
AMR_ERR_TIMEOUT = -5
AMR_ERR_STATE = -6
AMR_FP64, AMR_FP32 = 0, 1
AMR_HLL, AMR_LLF, AMR_FLUXREC = 0, 1, 2
AMR_PLM, AMR_WENO3 = 0, 1
AMR_BC_OUTFLOW, AMR_BC_PERIODIC = 0, 1
AMR_STATE_CONSERVED, AMR_STATE_PRIMITIVE = 0, 1
AMR_GHOST_DIRECT, AMR_GHOST_COPY = 0, 1
AMR_SPAN_LAYERS, AMR_SPAN_PATCH = 0, 1

STATUS_NAMES = {0: "AMR_OK", -1: "AMR_ERR_ARG", -2: "AMR_ERR_NESTING", -3: "AMR_ERR_CUDA",
                -4: "AMR_ERR_NONPHYSICAL", -5: "AMR_ERR_TIMEOUT", -6: "AMR_ERR_STATE"}

# every entry point declared in include/amr.h
EXPORTS = ["amr_default_config", "amr_create", "amr_validate_patches", "amr_set_patches", "amr_set_state",
           "amr_state_size", "amr_step", "amr_cfl_dt", "amr_get_state", "amr_get_state_all",
           "amr_conserved_totals", "amr_check", "amr_kernel_launches", "amr_last_error", "amr_global_error",
           "amr_destroy", "amr_set_timing", "amr_get_timing", "amr_step_patch_noalloc", "amr_regrid",
           "amr_get_patches", "amr_autotune", "amr_set_tiling", "amr_get_regrid_timing", "amr_floor_count",
           "amr_set_regrid_schedule", "amr_cell_updates", "amr_divb_norms", "amr_set_state_async",
           "amr_get_state_all_async", "amr_wait_state", "amr_partition_patches", "amr_get_regrid_counts",
           "amr_peak_fma_rates", "amr_set_persistent", "amr_set_overlap"]
REGRID_PHASES = ["flag", "cluster", "plan", "fill_tables", "install", "fill"]
TIMING_CLASSES = ["stage1", "stage2", "ghost", "parent", "registers", "sync", "speed"]


class AmrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
        self.msg = msg


# Device allocator callbacks of amr_config (dev_alloc / dev_free).
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class amr_config(ctypes.Structure):
    _fields_ = [
        ("nvar", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("riemann", ctypes.c_int),
        ("gamma", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("base_n", ctypes.c_int * 3),
        ("domain_lo", ctypes.c_double * 3),
        ("domain_hi", ctypes.c_double * 3),
        ("bc", ctypes.c_int * 6),
        ("max_level", ctypes.c_int),
        ("ref_ratio", ctypes.c_int),
        ("ch", ctypes.c_double),
        ("p_floor", ctypes.c_double),
        ("glm_alpha", ctypes.c_double),
        ("batched", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("cuda_stream", ctypes.c_void_p),
        ("dev_alloc", ALLOC_FN),
        ("dev_free", FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
        ("recon", ctypes.c_int),
        ("ghost_fill", ctypes.c_int),
        ("item_span", ctypes.c_int),
    ]


class amr_patch(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("lo", ctypes.c_int * 3), ("n", ctypes.c_int * 3)]


class amr_regrid_params(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_double), ("buffer", ctypes.c_int), ("block", ctypes.c_int),
                ("max_patch", ctypes.c_int), ("min_level", ctypes.c_int)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libamr_gb300.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"native library {path} is missing: run paper_0910_5547_gb300.build.build() "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    H = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    L.amr_default_config.argtypes = [ctypes.POINTER(amr_config)]
    L.amr_default_config.restype = None
    L.amr_create.argtypes = [ctypes.POINTER(amr_config), ctypes.POINTER(H)]
    L.amr_validate_patches.argtypes = [ctypes.POINTER(amr_config), ctypes.c_int, ctypes.POINTER(amr_patch),
                                       ctypes.c_char_p, ctypes.c_int]
    L.amr_set_patches.argtypes = [H, ctypes.c_int, ctypes.POINTER(amr_patch), ctypes.POINTER(dp), ctypes.c_int]
    L.amr_set_state.argtypes = [H, dp, ctypes.c_int]
    L.amr_state_size.argtypes = [H]
    L.amr_state_size.restype = ctypes.c_longlong
    L.amr_step.argtypes = [H, ctypes.c_double, dp]
    L.amr_cfl_dt.argtypes = [H, dp]
    L.amr_get_state.argtypes = [H, ctypes.c_int, dp]
    L.amr_get_state_all.argtypes = [H, dp]
    L.amr_conserved_totals.argtypes = [H, dp]
    L.amr_check.argtypes = [H]
    L.amr_kernel_launches.argtypes = [H]
    L.amr_kernel_launches.restype = ctypes.c_longlong
    L.amr_last_error.argtypes = [H]
    L.amr_last_error.restype = ctypes.c_char_p
    L.amr_global_error.argtypes = []
    L.amr_global_error.restype = ctypes.c_char_p
    L.amr_destroy.argtypes = [H]
    L.amr_destroy.restype = None
    L.amr_step_patch_noalloc.argtypes = [ctypes.POINTER(amr_config), ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_double, dp]
    L.amr_step_patch_noalloc.restype = ctypes.c_int
    L.amr_set_persistent.argtypes = [H, ctypes.c_int]
    L.amr_set_persistent.restype = ctypes.c_int
    L.amr_set_overlap.argtypes = [H, ctypes.c_int]
    L.amr_set_overlap.restype = ctypes.c_int
    L.amr_peak_fma_rates.argtypes = [dp]
    L.amr_peak_fma_rates.restype = ctypes.c_int
    L.amr_regrid.argtypes = [H, ctypes.POINTER(amr_regrid_params), ctypes.POINTER(ctypes.c_int)]
    L.amr_regrid.restype = ctypes.c_int
    L.amr_set_regrid_schedule.argtypes = [H, ctypes.POINTER(amr_regrid_params), ctypes.c_int]
    L.amr_set_regrid_schedule.restype = ctypes.c_int
    L.amr_cell_updates.argtypes = [H]
    L.amr_cell_updates.restype = ctypes.c_longlong
    L.amr_get_patches.argtypes = [H, ctypes.POINTER(amr_patch), ctypes.c_int]
    L.amr_autotune.argtypes = [H, ctypes.c_char_p, ctypes.c_int]
    L.amr_autotune.restype = ctypes.c_int
    L.amr_set_tiling.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.amr_set_tiling.restype = ctypes.c_int
    L.amr_get_regrid_timing.argtypes = [H, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    L.amr_get_regrid_timing.restype = ctypes.c_int
    L.amr_floor_count.argtypes = [H, ctypes.POINTER(ctypes.c_longlong)]
    L.amr_floor_count.restype = ctypes.c_int
    L.amr_divb_norms.argtypes = [H, dp]
    L.amr_divb_norms.restype = ctypes.c_int
    L.amr_set_state_async.argtypes = [H, dp, ctypes.c_int]
    L.amr_set_state_async.restype = ctypes.c_int
    L.amr_get_state_all_async.argtypes = [H, dp, ctypes.POINTER(ctypes.c_longlong)]
    L.amr_get_state_all_async.restype = ctypes.c_int
    L.amr_wait_state.argtypes = [H, ctypes.c_longlong]
    L.amr_wait_state.restype = ctypes.c_int
    L.amr_get_patches.restype = ctypes.c_int
    L.amr_set_timing.argtypes = [H, ctypes.c_int]
    L.amr_get_timing.argtypes = [H, dp, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]
    for name in ("amr_create", "amr_validate_patches", "amr_set_patches", "amr_set_state", "amr_step",
                 "amr_cfl_dt", "amr_get_state", "amr_get_state_all", "amr_conserved_totals", "amr_check",
                 "amr_set_timing", "amr_get_timing"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(h, st: int):
    if st != AMR_OK:
        L = load()
        msg = (L.amr_last_error(h) if h else L.amr_global_error()) or b""
        raise AmrError(st, msg.decode())


def amr_default_config(**overrides) -> amr_config:
    c = amr_config()
    load().amr_default_config(ctypes.byref(c))
    for k, v in overrides.items():
        if isinstance(getattr(c, k), ctypes.Array):
            getattr(c, k)[:] = list(v)
        else:
            setattr(c, k, v)
    return c


def torch_allocator():
    """(dev_alloc, dev_free) callbacks that take the handle's device memory from
    PyTorch's caching allocator on the handle's stream.  Keep the returned pair alive
    as long as the handle."""
    import torch

    def _alloc(nbytes, stream, ctx):
        s = torch.cuda.ExternalStream(stream) if stream else None
        return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=s))

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    return ALLOC_FN(_alloc), FREE_FN(_free)


def make_patches(patches: Sequence) -> ctypes.Array:
    arr = (amr_patch * len(patches))()
    for i, p in enumerate(patches):
        arr[i].level = int(p.level)
        arr[i].lo[:] = [int(x) for x in p.lo]
        arr[i].n[:] = [int(x) for x in p.n]
    return arr


def amr_create(cfg: amr_config) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(None, load().amr_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def amr_partition_patches(cfg: amr_config, patches: Sequence, nranks: int) -> np.ndarray:
    """Owner rank per patch (Morton ranges of equal cell counts per level); host only."""
    arr = make_patches(patches)
    out = np.zeros(len(patches), dtype=np.int32)
    L = load()
    L.amr_partition_patches.argtypes = [ctypes.POINTER(amr_config), ctypes.c_int, ctypes.POINTER(amr_patch),
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.amr_partition_patches.restype = ctypes.c_int
    st = L.amr_partition_patches(ctypes.byref(cfg), len(patches), arr, nranks,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if st != AMR_OK:
        raise AmrError(st, "amr_partition_patches")
    return out


def amr_validate_patches(cfg: amr_config, patches: Sequence):
    """Returns (status, message); host only, needs no GPU."""
    arr = make_patches(patches)
    buf = ctypes.create_string_buffer(512)
    st = load().amr_validate_patches(ctypes.byref(cfg), len(patches), arr, buf, 512)
    return st, buf.value.decode()


def amr_set_patches(h, patches: Sequence, states: Sequence[np.ndarray], kind: int = AMR_STATE_PRIMITIVE):
    arr = make_patches(patches)
    keep = [np.ascontiguousarray(s, dtype=np.float64) for s in states]
    ptrs = (ctypes.POINTER(ctypes.c_double) * len(keep))(*[_dp(a) for a in keep])
    _check(h, load().amr_set_patches(h, len(patches), arr, ptrs, kind))


def amr_set_state(h, packed: np.ndarray, kind: int = AMR_STATE_CONSERVED):
    assert packed.dtype == np.float64 and packed.flags.c_contiguous
    _check(h, load().amr_set_state(h, _dp(packed), kind))


def amr_state_size(h) -> int:
    return int(load().amr_state_size(h))


def amr_step(h, dt: float = 0.0, sync: bool = True) -> float:
    """One coarse step; returns the dt taken when sync (else nan)."""
    if sync:
        used = ctypes.c_double(0.0)
        _check(h, load().amr_step(h, dt, ctypes.byref(used)))
        return used.value
    _check(h, load().amr_step(h, dt, None))
    return float("nan")


def amr_cfl_dt(h) -> float:
    dt = ctypes.c_double(0.0)
    _check(h, load().amr_cfl_dt(h, ctypes.byref(dt)))
    return dt.value


def amr_get_state(h, patch: int, shape) -> np.ndarray:
    out = np.empty(shape, dtype=np.float64)
    _check(h, load().amr_get_state(h, patch, _dp(out)))
    return out


def amr_get_state_all(h, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        out = np.empty(amr_state_size(h), dtype=np.float64)
    assert out.dtype == np.float64 and out.flags.c_contiguous
    _check(h, load().amr_get_state_all(h, _dp(out)))
    return out


def amr_conserved_totals(h, nvar: int) -> np.ndarray:
    out = np.zeros(nvar, dtype=np.float64)
    _check(h, load().amr_conserved_totals(h, _dp(out)))
    return out


def amr_get_regrid_counts(h) -> tuple:
    """(regrids that installed a new hierarchy, regrids that found it unchanged,
    regrids that reused the previous clustering of their min_level)."""
    c = (ctypes.c_longlong * 3)()
    L = load()
    L.amr_get_regrid_counts.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]
    L.amr_get_regrid_counts.restype = ctypes.c_int
    _check(h, L.amr_get_regrid_counts(h, c))
    return int(c[0]), int(c[1]), int(c[2])


def amr_set_state_async(h, packed: np.ndarray, kind: int = AMR_STATE_CONSERVED) -> None:
    """Enqueue the upload of a packed FP64 state; keep `packed` unchanged until a
    later amr_wait_state has returned."""
    assert packed.dtype == np.float64 and packed.flags.c_contiguous
    _check(h, load().amr_set_state_async(h, _dp(packed), kind))


def amr_get_state_all_async(h, out: np.ndarray) -> int:
    """Enqueue the download of the state into `out`; returns the ticket to wait for."""
    assert out.dtype == np.float64 and out.flags.c_contiguous
    t = ctypes.c_longlong(-1)
    _check(h, load().amr_get_state_all_async(h, _dp(out), ctypes.byref(t)))
    return t.value


def amr_wait_state(h, ticket: int) -> None:
    _check(h, load().amr_wait_state(h, ticket))


def amr_divb_norms(h) -> np.ndarray:
    """[sum |div B| dV, max |div B|, sum |B|/dx_min dV, max |B|/dx_min] over leaf cells."""
    out = np.zeros(4, dtype=np.float64)
    _check(h, load().amr_divb_norms(h, _dp(out)))
    return out


def amr_check(h):
    _check(h, load().amr_check(h))


def amr_kernel_launches(h) -> int:
    return int(load().amr_kernel_launches(h))


def amr_last_error(h) -> str:
    return (load().amr_last_error(h) or b"").decode()


def amr_set_timing(h, on: bool):
    _check(h, load().amr_set_timing(h, int(on)))


def amr_get_timing(h) -> dict:
    """{class: (total_ms, launches)} since timing was switched on (then reset)."""
    n = len(TIMING_CLASSES)
    ms = np.zeros(n)
    cnt = (ctypes.c_longlong * n)()
    _check(h, load().amr_get_timing(h, _dp(ms), cnt, n))
    return {c: (float(ms[i]), int(cnt[i])) for i, c in enumerate(TIMING_CLASSES)}


def amr_step_patch_noalloc(cfg: amr_config, state_in_ptr: int, state_out_ptr: int, dt: float = 0.0,
                           sync: bool = True) -> float:
    """One RK2 step of one uniform patch with no device allocation; the pointers are
    caller-owned DEVICE arrays (FP64 conserved, [nvar][nz][ny][nx])."""
    L = load()
    if sync:
        used = ctypes.c_double(0.0)
        st = L.amr_step_patch_noalloc(ctypes.byref(cfg), ctypes.c_void_p(state_in_ptr),
                                      ctypes.c_void_p(state_out_ptr), dt, ctypes.byref(used))
        if st != AMR_OK:
            raise AmrError(st, "amr_step_patch_noalloc failed")
        return used.value
    st = L.amr_step_patch_noalloc(ctypes.byref(cfg), ctypes.c_void_p(state_in_ptr), ctypes.c_void_p(state_out_ptr),
                                  dt, None)
    if st != AMR_OK:
        raise AmrError(st, "amr_step_patch_noalloc failed")
    return float("nan")


def amr_set_persistent(h, mode: int) -> None:
    """Stage launch form: 0 one CTA per work item, 1 persistent CTAs, -1 the autotuner decides."""
    _check(h, load().amr_set_persistent(h, int(mode)))


def amr_set_overlap(h, on: bool) -> None:
    """Second stream of a multi-level batched step (stage-2 parent fill and registers beside the stages)."""
    _check(h, load().amr_set_overlap(h, 1 if on else 0))


def amr_peak_fma_rates() -> dict:
    """FP32 and FP64 FMA rates of the current device's CUDA cores, FLOP/s."""
    out = (ctypes.c_double * 2)()
    st = load().amr_peak_fma_rates(out)
    if st != AMR_OK:
        raise AmrError(st, "amr_peak_fma_rates failed")
    return {"fp32_flops": out[0], "fp64_flops": out[1]}


class PatchRecord:
    def __init__(self, level, lo, n):
        self.level, self.lo, self.n = level, tuple(lo), tuple(n)

    def __repr__(self):
        return f"Patch(level={self.level}, lo={self.lo}, n={self.n})"


def amr_regrid(h, threshold=0.3, buffer=2, block=4, max_patch=32, min_level=0) -> int:
    prm = amr_regrid_params(threshold, buffer, block, max_patch, min_level)
    n = ctypes.c_int(0)
    _check(h, load().amr_regrid(h, ctypes.byref(prm), ctypes.byref(n)))
    return n.value


def amr_set_regrid_schedule(h, max_level: int, threshold=0.3, buffer=2, block=4, max_patch=32):
    """Rebuild the levels finer than l after every step of a level l <= max_level
    (max_level < 0: no schedule)."""
    prm = amr_regrid_params(threshold, buffer, block, max_patch, 0)
    _check(h, load().amr_set_regrid_schedule(h, ctypes.byref(prm), int(max_level)))


def amr_cell_updates(h) -> int:
    """Interior cell-updates performed by amr_step so far (sum over level steps)."""
    return int(load().amr_cell_updates(h))


def amr_set_tiling(h, max_wx: int = 0, max_cols: int = 0, zchunk: int = 0, ctas_per_sm: int = 0) -> None:
    """Fix the stage-kernel work items (x width cap, columns per CTA, z chunk) and build (CTAs per SM)."""
    _check(h, load().amr_set_tiling(h, max_wx, max_cols, zchunk, ctas_per_sm))


def amr_autotune(h) -> str:
    """Pick the fastest stage-kernel tiling for the installed hierarchy; returns the report."""
    buf = ctypes.create_string_buffer(4096)
    _check(h, load().amr_autotune(h, buf, 4096))
    return buf.value.decode()


def amr_floor_count(h) -> int:
    """Interior primitive recoveries raised by the pressure floor since the last call."""
    n = ctypes.c_longlong(0)
    _check(h, load().amr_floor_count(h, ctypes.byref(n)))
    return int(n.value)


def amr_get_regrid_timing(h) -> dict:
    """Host seconds of the phases of the last amr_regrid (REGRID_PHASES)."""
    buf = (ctypes.c_double * len(REGRID_PHASES))()
    _check(h, load().amr_get_regrid_timing(h, buf, len(REGRID_PHASES)))
    return {k: buf[i] for i, k in enumerate(REGRID_PHASES)}


def amr_get_patches(h) -> list:
    L = load()
    n = L.amr_get_patches(h, None, 0)
    if n < 0:
        raise AmrError(AMR_ERR_STATE, "no patches installed")
    arr = (amr_patch * max(n, 1))()
    L.amr_get_patches(h, arr, n)
    return [PatchRecord(arr[i].level, arr[i].lo[:], arr[i].n[:]) for i in range(n)]


def amr_destroy(h):
    if h:
        load().amr_destroy(h)
