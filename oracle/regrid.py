"""Reference regridding for the oracle (TEST INFRASTRUCTURE ONLY).

Written independently of the CUDA library from this description of the
refinement procedure (the paper leaves hierarchy creation to the host, Sec. 3):

1. A cell of level l (min_level <= l < max_level) is flagged where
   max_d |rho(i+e_d) - rho(i-e_d)| / (2 rho(i)) > threshold (oracle.c, FP64).
2. Every flagged cell, grown by `buffer` cells, tags the blocks of `block`
   cells (of its level) it touches.
3. A tagged block of level l tags on level l-1 its parent block and the 26
   blocks around that parent (so the finer refinement stays nested).
4. Top-down from min_level: a tagged block is refined if each of its 26
   neighbours is covered by the (new) level l or lies beyond an outflow face;
   refined blocks are merged in (z, y, x) order into boxes, each grown along x,
   then y, then z, up to max_patch / (2 block) blocks per axis; a box of blocks
   of level l becomes a level-(l+1) patch of 2*block cells per block, clipped to
   the domain; the blocks of level l+1 these patches cover feed the next level.
"""
from __future__ import annotations

import ctypes
import math
from typing import List

import numpy as np

from . import Oracle, OrcPatch, lib

PERIODIC = 1


class P:
    def __init__(self, level, lo, n):
        self.level, self.lo, self.n = level, tuple(int(x) for x in lo), tuple(int(x) for x in n)

    def __eq__(self, o):
        return (self.level, self.lo, self.n) == (o.level, tuple(o.lo), tuple(o.n))

    def __repr__(self):
        return f"P({self.level}, {self.lo}, {self.n})"

    @property
    def ncell(self):
        return self.n[0] * self.n[1] * self.n[2]


def flags(o: Oracle, threshold: float) -> List[np.ndarray]:
    """Per-patch uint8 flag arrays (nz, ny, nx) from the oracle state."""
    total = sum(p.n[0] * p.n[1] * p.n[2] for p in o.patches)
    out = np.zeros(total, dtype=np.uint8)
    L = lib()
    L.orc_flags.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_ubyte)]
    L.orc_flags.restype = ctypes.c_int
    if L.orc_flags(o._h, threshold, out.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))) != 0:
        raise RuntimeError("oracle flags failed")
    res, k = [], 0
    for p in o.patches:
        n = p.n[0] * p.n[1] * p.n[2]
        res.append(out[k:k + n].reshape(p.n[2], p.n[1], p.n[0]))
        k += n
    return res


def cluster(patches, flag_arrays, base_n, bc, max_level, threshold=0.3, buffer=2, block=4, max_patch=32,
            min_level=0) -> List[P]:
    B = block
    per = [bc[2 * d] == PERIODIC for d in range(3)]

    def N(l, d):
        return base_n[d] << l

    def nb(l, d):
        return (N(l, d) + B - 1) // B

    tags = [set() for _ in range(max_level + 1)]
    for p, f in zip(patches, flag_arrays):
        l = p.level
        if l < min_level or l >= max_level or f is None:
            continue
        for (k, j, i) in zip(*np.nonzero(f)):
            c = (p.lo[0] + i, p.lo[1] + j, p.lo[2] + k)
            rng = []
            for d in range(3):
                lo, hi = c[d] - buffer, c[d] + buffer
                if not per[d]:
                    lo, hi = max(lo, 0), min(hi, N(l, d) - 1)
                rng.append(range(math.floor(lo / B), math.floor(hi / B) + 1))
            for z in rng[2]:
                for y in rng[1]:
                    for x in rng[0]:
                        q = [x, y, z]
                        for d in range(3):
                            if per[d]:
                                q[d] %= nb(l, d)
                        tags[l].add(tuple(q))
    for l in range(max_level - 1, min_level, -1):
        for b in list(tags[l]):
            pb = [b[0] // 2, b[1] // 2, b[2] // 2]
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        q = [pb[0] + dx, pb[1] + dy, pb[2] + dz]
                        ok = True
                        for d in range(3):
                            n = nb(l - 1, d)
                            if q[d] < 0 or q[d] >= n:
                                if per[d]:
                                    q[d] %= n
                                else:
                                    ok = False
                        if ok:
                            tags[l - 1].add(tuple(q))
    out = [P(p.level, p.lo, p.n) for p in patches if p.level <= min_level]
    cover = set()
    for p in patches:
        if p.level != min_level:
            continue
        a0, a1 = [], []
        for d in range(3):
            a0.append(-(-p.lo[d] // B))
            e = (p.lo[d] + p.n[d]) // B
            if p.lo[d] + p.n[d] == N(min_level, d) and N(min_level, d) % B:
                e += 1
            a1.append(e)
        for z in range(a0[2], a1[2]):
            for y in range(a0[1], a1[1]):
                for x in range(a0[0], a1[0]):
                    cover.add((x, y, z))
    maxb = max_patch // (2 * B)
    for l in range(min_level, max_level):
        refine = set()
        for b in tags[l]:
            ok = True
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        q = [b[0] + dx, b[1] + dy, b[2] + dz]
                        outside = False
                        for d in range(3):
                            n = nb(l, d)
                            if q[d] < 0 or q[d] >= n:
                                if per[d]:
                                    q[d] %= n
                                else:
                                    outside = True
                        if not outside and tuple(q) not in cover:
                            ok = False
            if ok:
                refine.add(b)
        if not refine:
            break
        done = set()
        new_cover = set()
        for b in sorted(refine, key=lambda t: (t[2], t[1], t[0])):
            if b in done:
                continue

            def free(x, y, z):
                return (x, y, z) in refine and (x, y, z) not in done

            nx = ny = nz = 1
            while nx < maxb and free(b[0] + nx, b[1], b[2]):
                nx += 1
            while ny < maxb and all(free(b[0] + i, b[1] + ny, b[2]) for i in range(nx)):
                ny += 1
            while nz < maxb and all(free(b[0] + i, b[1] + j, b[2] + nz) for i in range(nx) for j in range(ny)):
                nz += 1
            for z in range(nz):
                for y in range(ny):
                    for x in range(nx):
                        done.add((b[0] + x, b[1] + y, b[2] + z))
            lo = [2 * B * b[d] for d in range(3)]
            n = [min(2 * B * (nx, ny, nz)[d], N(l + 1, d) - lo[d]) for d in range(3)]
            out.append(P(l + 1, lo, n))
            for z in range(lo[2] // B, (lo[2] + n[2] + B - 1) // B):
                for y in range(lo[1] // B, (lo[1] + n[1] + B - 1) // B):
                    for x in range(lo[0] // B, (lo[0] + n[0] + B - 1) // B):
                        new_cover.add((x, y, z))
        cover = new_cover
    return out


def regrid(o: Oracle, threshold=0.3, buffer=2, block=4, max_patch=32, min_level=0) -> Oracle:
    """Flag, cluster and fill: a new Oracle on the new hierarchy."""
    fl = flags(o, threshold)
    cfg = o.cfg
    newp = cluster(o.patches, fl, tuple(cfg.base_n), tuple(cfg.bc), cfg.max_level, threshold, buffer, block,
                   max_patch, min_level)
    arr = (OrcPatch * len(newp))()
    for i, p in enumerate(newp):
        arr[i].level = p.level
        arr[i].lo[:] = list(p.lo)
        arr[i].n[:] = list(p.n)
    L = lib()
    L.orc_regrid_fill.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(OrcPatch), ctypes.c_int]
    L.orc_regrid_fill.restype = ctypes.c_void_p
    h = L.orc_regrid_fill(o._h, len(newp), arr, min_level)
    if not h:
        raise RuntimeError("oracle regrid failed: " + L.orc_error().decode())
    new = Oracle.__new__(Oracle)
    new.cfg = cfg
    new.nvar = o.nvar
    new.patches = newp
    new._h = h
    return new


def flags_at(o: Oracle, threshold: float, level: int, alpha: float) -> List[np.ndarray]:
    """Flags in the middle of a coarse step, after a step of `level` (see orc_flags_at)."""
    total = sum(p.n[0] * p.n[1] * p.n[2] for p in o.patches)
    out = np.zeros(total, dtype=np.uint8)
    L = lib()
    L.orc_flags_at.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                               ctypes.POINTER(ctypes.c_ubyte)]
    L.orc_flags_at.restype = ctypes.c_int
    if L.orc_flags_at(o._h, threshold, level, alpha, out.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))) != 0:
        raise RuntimeError("oracle flags failed")
    res, k = [], 0
    for p in o.patches:
        n = p.n[0] * p.n[1] * p.n[2]
        res.append(out[k:k + n].reshape(p.n[2], p.n[1], p.n[0]))
        k += n
    return res


_HOOK = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_double)


def set_regrid_schedule(o: Oracle, max_level: int, threshold=0.3, buffer=2, block=4, max_patch=32):
    """From now on every orc_step rebuilds the levels finer than l after each step of a
    level l <= max_level (flag, cluster, fill in place); o.patches follows the hierarchy
    and o.regrid_log records (level, new patch list) of every rebuild.
    max_level < 0 removes the schedule."""
    L = lib()
    L.orc_set_regrid_hook.argtypes = [ctypes.c_void_p, ctypes.c_int, _HOOK, ctypes.c_void_p]
    L.orc_set_regrid_hook.restype = None
    L.orc_regrid_inplace.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(OrcPatch), ctypes.c_int]
    L.orc_regrid_inplace.restype = ctypes.c_int
    if max_level < 0:
        L.orc_set_regrid_hook(o._h, -1, _HOOK(), None)
        o._regrid_hook = None
        return
    cfg = o.cfg
    o.regrid_log = []

    def hook(ctx, level, alpha):
        try:
            fl = flags_at(o, threshold, level, alpha)
            newp = cluster(o.patches, fl, tuple(cfg.base_n), tuple(cfg.bc), cfg.max_level, threshold, buffer,
                           block, max_patch, level)
            arr = (OrcPatch * len(newp))()
            for i, p in enumerate(newp):
                arr[i].level = p.level
                arr[i].lo[:] = list(p.lo)
                arr[i].n[:] = list(p.n)
            if L.orc_regrid_inplace(o._h, len(newp), arr, level) != 0:
                return -1
            o.patches = newp
            o.regrid_log.append((level, list(newp)))
            return 0
        except Exception:            # noqa: BLE001 -- reported to the C caller as a failed step
            import traceback
            traceback.print_exc()
            return -1

    o._regrid_hook = _HOOK(hook)
    L.orc_set_regrid_hook(o._h, max_level, o._regrid_hook, None)
