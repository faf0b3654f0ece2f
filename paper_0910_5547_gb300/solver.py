"""Convenience wrapper around the C ABI: one ``Solver`` owns one amr_handle.

Argument marshalling only -- every step of the method runs in the native
library's CUDA kernels.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np

from . import native as N


class Solver:
    """A patch hierarchy resident on the GPU.

    ``patches`` are objects with ``level``, ``lo`` and ``n``; ``state`` is a list
    of float64 arrays (nvar, nz, ny, nx), primitive (default) or conserved.
    """

    def __init__(self, patches: Sequence, state: Sequence[np.ndarray], *, nvar=5, precision="fp64",
                 gamma=1.4, theta=1.5, cfl=0.4, base_n=(32, 32, 32), bc=(0,) * 6, max_level=None,
                 riemann="hll", ch=0.0, batched=True, use_graph=True, domain_lo=(0.0, 0.0, 0.0),
                 domain_hi=(1.0, 1.0, 1.0), kind=N.AMR_STATE_PRIMITIVE, stream=None, p_floor=0.0,
                 glm_alpha=0.0, allocator=None, recon="plm", ghost_fill="direct", item_span="layers"):
        self.patches = list(patches)
        self.nvar = nvar
        if max_level is None:
            max_level = max(p.level for p in self.patches)
        self.cfg = N.amr_default_config(
            nvar=nvar, precision=N.AMR_FP32 if precision == "fp32" else N.AMR_FP64,
            riemann={"hll": N.AMR_HLL, "llf": N.AMR_LLF, "fluxrec": N.AMR_FLUXREC}[riemann], gamma=gamma,
            theta=theta, cfl=cfl,
            base_n=base_n, bc=bc, max_level=max_level, ch=ch, p_floor=p_floor, glm_alpha=glm_alpha,
            batched=int(batched), use_graph=int(use_graph),
            recon={"plm": N.AMR_PLM, "weno3": N.AMR_WENO3}[recon],
            ghost_fill={"direct": N.AMR_GHOST_DIRECT, "copy": N.AMR_GHOST_COPY}[ghost_fill],
            item_span={"layers": N.AMR_SPAN_LAYERS, "patch": N.AMR_SPAN_PATCH}[item_span],
            domain_lo=domain_lo, domain_hi=domain_hi, cuda_stream=stream)
        # allocator="torch": device memory from PyTorch's caching allocator (callbacks kept alive here)
        self._alloc_fns = N.torch_allocator() if allocator == "torch" else None
        if self._alloc_fns is not None:
            self.cfg.dev_alloc, self.cfg.dev_free = self._alloc_fns
        self.h = N.amr_create(self.cfg)
        N.amr_set_patches(self.h, self.patches, state, kind)
        self.offsets = np.cumsum([0] + [nvar * p.n[0] * p.n[1] * p.n[2] for p in self.patches])

    @classmethod
    def from_problem(cls, pb, **kw):
        kw.setdefault("nvar", pb.nvar)
        kw.setdefault("gamma", pb.gamma)
        kw.setdefault("base_n", pb.base_n)
        kw.setdefault("bc", pb.bc)
        kw.setdefault("max_level", pb.max_level)
        kw.setdefault("domain_lo", pb.domain_lo)
        kw.setdefault("domain_hi", pb.domain_hi)
        return cls(pb.patches, pb.prim, **kw)

    def close(self):
        if getattr(self, "h", None):
            N.amr_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


    def floor_count(self) -> int:
        """Interior cells (per stage) in which the pressure floor acted since the last call."""
        return N.amr_floor_count(self.h)

    def cfl_dt(self) -> float:
        return N.amr_cfl_dt(self.h)

    def run_to(self, t_end: float, max_steps: int = 100000) -> int:
        t, k = 0.0, 0
        while t < t_end * (1 - 1e-14) and k < max_steps:
            dt = min(self.cfl_dt(), t_end - t)
            self.step(dt)
            t += dt
            k += 1
        return k

    def state_all(self) -> np.ndarray:
        return N.amr_get_state_all(self.h)

    def cons(self, i: int) -> np.ndarray:
        p = self.patches[i]
        return N.amr_get_state(self.h, i, (self.nvar, p.n[2], p.n[1], p.n[0]))

    def all_cons(self) -> List[np.ndarray]:
        flat = self.state_all()
        out = []
        for i, p in enumerate(self.patches):
            out.append(flat[self.offsets[i]:self.offsets[i + 1]].reshape(self.nvar, p.n[2], p.n[1], p.n[0]))
        return out

    def set_state(self, packed: np.ndarray, kind=N.AMR_STATE_CONSERVED):
        N.amr_set_state(self.h, packed, kind)

    def totals(self) -> np.ndarray:
        return N.amr_conserved_totals(self.h, self.nvar)

    def divb_norms(self) -> np.ndarray:
        """GLM-MHD: [sum |div B| dV, max |div B|, sum |B|/dx_min dV, max |B|/dx_min]
        over leaf cells (centred differences after a ghost refill)."""
        return N.amr_divb_norms(self.h)

    def check(self):
        N.amr_check(self.h)

    def launches(self) -> int:
        return N.amr_kernel_launches(self.h)

    def set_tiling(self, max_wx: int = 0, max_cols: int = 0, zchunk: int = 0, ctas_per_sm: int = 0) -> None:
        """Fix the stage-kernel work items and build instead of autotuning (0 = default)."""
        N.amr_set_tiling(self.h, max_wx, max_cols, zchunk, ctas_per_sm)

    def set_persistent(self, mode: int) -> None:
        """Stage launch form: 0 one CTA per work item, 1 persistent CTAs, -1 the autotuner decides."""
        N.amr_set_persistent(self.h, mode)

    def set_overlap(self, on: bool) -> None:
        """Run the stage-2 parent fill and the register kernels on a second stream (default) or not."""
        N.amr_set_overlap(self.h, on)

    def autotune(self) -> str:
        """Time the stage kernel's candidate tilings on this hierarchy and keep the fastest."""
        return N.amr_autotune(self.h)

    def set_regrid_schedule(self, max_level: int, **kw):
        """Rebuild the finer levels after every step of a level <= max_level during step()."""
        N.amr_set_regrid_schedule(self.h, max_level, **kw)
        self._scheduled = max_level >= 0

    def step(self, dt: float = 0.0, sync: bool = True) -> float:
        used = N.amr_step(self.h, dt, sync)
        if getattr(self, "_scheduled", False):
            self._refresh_patches()
        return used

    def _refresh_patches(self):
        self.patches = N.amr_get_patches(self.h)
        self.offsets = np.cumsum([0] + [self.nvar * p.n[0] * p.n[1] * p.n[2] for p in self.patches])

    def regrid(self, **kw) -> int:
        """Rebuild the refined levels from density-gradient flags (see amr_regrid)."""
        n = N.amr_regrid(self.h, **kw)
        self.patches = N.amr_get_patches(self.h)
        self.offsets = np.cumsum([0] + [self.nvar * p.n[0] * p.n[1] * p.n[2] for p in self.patches])
        return n
