"""FP64 CPU oracle for the AMR finite-volume update -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (``paper_0910_5547_gb300``)
never does: it runs on its own CUDA kernels and fails loudly without them.

The numerics live in ``amr_oracle.c`` (plain unfused C, -ffp-contract=off);
this module compiles it with gcc and wraps it with ctypes.

Parity status of each oracle function (pins live in tests/test_oracle_*.py):
  minmod3 / PLM          -- truth table, linear data, second-order convergence
  HLL / LLF flux         -- consistency F(U,U) = F(U), exact Sod solution
  RK2 three-line form    -- algebraic identity with the Shu-Osher form
  ghost fill, prolong,   -- uniform state exact, linear data exact, conservation
  restrict, reflux          to round-off on periodic AMR boxes, AMR vs uniform fine
  GLM-MHD                -- B = 0 reduces to hydro, Brio-Wu invariants, conservation
The Kelvin-Helmholtz, Orszag-Tang and Sedov-AMR solutions at finite step
counts have no closed form: the oracle is pinned there only through the
invariants above (parity unpinned for those exact values).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

HLL, LLF, FLUXREC = 0, 1, 2
PLM, WENO3 = 0, 1
OUTFLOW, PERIODIC = 0, 1


class OrcConfig(ctypes.Structure):
    _fields_ = [
        ("nvar", ctypes.c_int),
        ("riemann", ctypes.c_int),
        ("plm_literal", ctypes.c_int),
        ("gamma", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("base_n", ctypes.c_int * 3),
        ("domain_lo", ctypes.c_double * 3),
        ("domain_hi", ctypes.c_double * 3),
        ("bc", ctypes.c_int * 6),
        ("max_level", ctypes.c_int),
        ("ch", ctypes.c_double),
        ("p_floor", ctypes.c_double),
        ("glm_alpha", ctypes.c_double),
        ("nthreads", ctypes.c_int),
        ("recon", ctypes.c_int),
    ]


class OrcPatch(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("lo", ctypes.c_int * 3), ("n", ctypes.c_int * 3)]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2 -ffp-contract=off, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                    os.path.getmtime(os.path.join(_HERE, "amr_oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            cp = ctypes.POINTER(OrcConfig)
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [cp, ctypes.c_int, ctypes.POINTER(OrcPatch)]
            L.orc_error.restype = ctypes.c_char_p
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            for fn in (L.orc_set_prim, L.orc_set_cons, L.orc_get_cons):
                fn.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
                fn.restype = ctypes.c_int
            L.orc_cfl_dt.argtypes = [ctypes.c_void_p]
            L.orc_cfl_dt.restype = ctypes.c_double
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_double, dp]
            L.orc_step.restype = ctypes.c_int
            L.orc_totals.argtypes = [ctypes.c_void_p, dp]
            L.orc_divb.argtypes = [ctypes.c_void_p, dp]
            L.orc_divb.restype = ctypes.c_int
            L.orc_last_ch.argtypes = [ctypes.c_void_p]
            L.orc_last_ch.restype = ctypes.c_double
            L.orc_fill_ghosts.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double]
            L.orc_fill_ghosts.restype = ctypes.c_int
            L.orc_get_ghosted.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, dp]
            L.orc_get_ghosted.restype = ctypes.c_int
            L.orc_save_old.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_save_old.restype = ctypes.c_int
            L.orc_minmod3.argtypes = [ctypes.c_double] * 3
            L.orc_minmod3.restype = ctypes.c_double
            L.orc_minmod2.argtypes = [ctypes.c_double] * 2
            L.orc_minmod2.restype = ctypes.c_double
            L.orc_plm_face.argtypes = [cp, dp, dp, dp]
            L.orc_weno3_face.argtypes = [dp, dp, dp]
            L.orc_phys_flux.argtypes = [cp, dp, ctypes.c_int, ctypes.c_double, dp]
            L.orc_prim_to_cons.argtypes = [cp, dp, dp]
            L.orc_cons_to_prim.argtypes = [cp, dp, dp]
            L.orc_riemann.argtypes = [cp, dp, dp, ctypes.c_int, ctypes.c_double, dp]
            L.orc_fluxrec_face.argtypes = [cp, dp, ctypes.c_int, dp]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_config(nvar=5, gamma=1.4, theta=1.5, cfl=0.4, base_n=(32, 32, 32), bc=(OUTFLOW,) * 6,
                riemann=HLL, plm_literal=False, max_level=0, ch=0.0, domain_lo=(0.0, 0.0, 0.0),
                domain_hi=(1.0, 1.0, 1.0), nthreads=0, p_floor=0.0, glm_alpha=0.0, recon=PLM) -> OrcConfig:
    c = OrcConfig()
    c.nvar, c.riemann, c.plm_literal = nvar, riemann, int(plm_literal)
    c.gamma, c.theta, c.cfl = gamma, theta, cfl
    c.base_n[:] = list(base_n)
    c.domain_lo[:] = list(domain_lo)
    c.domain_hi[:] = list(domain_hi)
    c.bc[:] = list(bc)
    c.max_level, c.ch, c.nthreads = max_level, ch, nthreads
    c.p_floor, c.glm_alpha = p_floor, glm_alpha
    c.recon = recon
    return c


class Oracle:
    """A running oracle simulation (patch ids are positions in the given list)."""

    def __init__(self, problem=None, *, patches=None, prim=None, cons=None, nthreads=0, **cfg):
        if problem is not None:
            cfg.setdefault("nvar", problem.nvar)
            cfg.setdefault("gamma", problem.gamma)
            cfg.setdefault("base_n", problem.base_n)
            cfg.setdefault("bc", problem.bc)
            cfg.setdefault("max_level", problem.max_level)
            cfg.setdefault("domain_lo", problem.domain_lo)
            cfg.setdefault("domain_hi", problem.domain_hi)
            patches = problem.patches if patches is None else patches
            if prim is None and cons is None:
                prim = problem.prim
        self.cfg = make_config(nthreads=nthreads, **cfg)
        self.nvar = self.cfg.nvar
        self.patches = list(patches)
        arr = (OrcPatch * len(self.patches))()
        for i, p in enumerate(self.patches):
            arr[i].level = p.level
            arr[i].lo[:] = list(p.lo)
            arr[i].n[:] = list(p.n)
        L = lib()
        self._h = L.orc_create(ctypes.byref(self.cfg), len(self.patches), arr)
        if not self._h:
            raise ValueError("oracle: " + L.orc_error().decode())
        src = prim if prim is not None else cons
        fn = L.orc_set_prim if prim is not None else L.orc_set_cons
        for i, a in enumerate(src):
            a = np.ascontiguousarray(a, dtype=np.float64)
            fn(self._h, i, _dp(a))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def cfl_dt(self) -> float:
        return lib().orc_cfl_dt(self._h)

    def step(self, dt: float = 0.0) -> float:
        used = ctypes.c_double(0.0)
        rc = lib().orc_step(self._h, dt, ctypes.byref(used))
        if rc != 0:
            raise RuntimeError("oracle step failed: " + lib().orc_error().decode())
        return used.value

    def run_to(self, t_end: float, max_steps: int = 100000) -> int:
        """CFL steps, the last one clipped to land on t_end; returns the step count."""
        t, k = 0.0, 0
        while t < t_end * (1 - 1e-14) and k < max_steps:
            dt = min(self.cfl_dt(), t_end - t)
            self.step(dt)
            t += dt
            k += 1
        return k

    def cons(self, i: int) -> np.ndarray:
        p = self.patches[i]
        out = np.empty((self.nvar, p.n[2], p.n[1], p.n[0]), dtype=np.float64)
        lib().orc_get_cons(self._h, i, _dp(out))
        return out

    def all_cons(self) -> List[np.ndarray]:
        return [self.cons(i) for i in range(len(self.patches))]

    def prim(self, i: int) -> np.ndarray:
        u = self.cons(i)
        flat = u.reshape(self.nvar, -1)
        out = np.empty_like(flat)
        ui = np.empty(self.nvar)
        wi = np.empty(self.nvar)
        L = lib()
        for c in range(flat.shape[1]):
            ui[:] = flat[:, c]
            L.orc_cons_to_prim(ctypes.byref(self.cfg), _dp(ui), _dp(wi))
            out[:, c] = wi
        return out.reshape(u.shape)

    def totals(self) -> np.ndarray:
        out = np.zeros(self.nvar)
        lib().orc_totals(self._h, _dp(out))
        return out

    def divb_norms(self) -> np.ndarray:
        """[sum |div B| dV, max |div B|, sum |B|/dx_min dV, max |B|/dx_min] over
        leaf cells after a ghost refill at the current time (GLM-MHD only)."""
        out = np.zeros(4)
        if lib().orc_divb(self._h, _dp(out)) != 0:
            raise RuntimeError("oracle div B needs nvar = 9 and a valid ghost fill")
        return out

    def last_ch(self) -> float:
        return lib().orc_last_ch(self._h)

    def save_old(self, level: int) -> None:
        lib().orc_save_old(self._h, level)

    def fill_ghosts(self, level: int, which: int = 0, alpha: float = 0.0) -> None:
        if lib().orc_fill_ghosts(self._h, level, which, alpha) != 0:
            raise RuntimeError("oracle ghost fill failed: " + lib().orc_error().decode())

    def ghosted(self, i: int, which: int = 0) -> np.ndarray:
        """Full ghosted array (nvar, nz+4, ny+4, nx+4); never-filled edge/corner ghosts are NaN."""
        p = self.patches[i]
        out = np.empty((self.nvar, p.n[2] + 4, p.n[1] + 4, p.n[0] + 4), dtype=np.float64)
        lib().orc_get_ghosted(self._h, i, which, _dp(out))
        return out


# ---- point functions ------------------------------------------------------

def minmod3(a, b, c) -> float:
    return lib().orc_minmod3(a, b, c)


def minmod2(a, b) -> float:
    return lib().orc_minmod2(a, b)


def plm_face(u4: Sequence[float], theta=1.5, plm_literal=False):
    cfg = make_config(theta=theta, plm_literal=plm_literal)
    u = np.ascontiguousarray(u4, dtype=np.float64)
    ul, ur = np.zeros(1), np.zeros(1)
    lib().orc_plm_face(ctypes.byref(cfg), _dp(u), _dp(ul), _dp(ur))
    return float(ul[0]), float(ur[0])


def weno3_face(u4: Sequence[float]):
    """Third-order WENO states (left, right) of the face between u4[1] and u4[2]."""
    u = np.ascontiguousarray(u4, dtype=np.float64)
    ul, ur = np.zeros(1), np.zeros(1)
    lib().orc_weno3_face(_dp(u), _dp(ul), _dp(ur))
    return float(ul[0]), float(ur[0])


def prim_to_cons(w, nvar=5, gamma=1.4) -> np.ndarray:
    cfg = make_config(nvar=nvar, gamma=gamma)
    w = np.ascontiguousarray(w, dtype=np.float64)
    u = np.zeros(nvar)
    lib().orc_prim_to_cons(ctypes.byref(cfg), _dp(w), _dp(u))
    return u


def cons_to_prim(u, nvar=5, gamma=1.4, p_floor=0.0) -> np.ndarray:
    cfg = make_config(nvar=nvar, gamma=gamma, p_floor=p_floor)
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.zeros(nvar)
    lib().orc_cons_to_prim(ctypes.byref(cfg), _dp(u), _dp(w))
    return w


def phys_flux(w, d, nvar=5, gamma=1.4, ch=1.0) -> np.ndarray:
    cfg = make_config(nvar=nvar, gamma=gamma)
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.zeros(nvar)
    lib().orc_phys_flux(ctypes.byref(cfg), _dp(w), d, ch, _dp(f))
    return f


def fluxrec_face(u4, d, gamma=1.4, theta=1.5) -> np.ndarray:
    """Direct flux reconstruction (Euler) at the face between rows 1 and 2 of
    four conserved states u4[4][5] along axis d."""
    cfg = make_config(nvar=5, gamma=gamma, theta=theta, riemann=FLUXREC)
    u4 = np.ascontiguousarray(u4, dtype=np.float64)
    f = np.zeros(5)
    lib().orc_fluxrec_face(ctypes.byref(cfg), _dp(u4), d, _dp(f))
    return f


def riemann(wl, wr, d, nvar=5, gamma=1.4, ch=1.0, kind=HLL) -> np.ndarray:
    cfg = make_config(nvar=nvar, gamma=gamma, riemann=kind)
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    f = np.zeros(nvar)
    lib().orc_riemann(ctypes.byref(cfg), _dp(wl), _dp(wr), d, ch, _dp(f))
    return f
