"""Seeded synthetic workloads for the AMR finite-volume update.

This module is the one piece shared by the CPU oracle and the CUDA path: it
only lays out patches and writes PRIMITIVE initial fields
(rho, vx, vy, vz, p [, Bx, By, Bz, psi]).  It holds none of the method's
arithmetic -- each side converts primitives to conserved variables with its
own equation of state.

Every generator returns a ``Problem``: solver settings (gamma, boundary
conditions, domain), the patch list ``(level, lo, n)`` sorted by level, and
one float64 array of shape ``(nvar, nz, ny, nx)`` per patch (interior cells,
x fastest).  Random numbers come from ``numpy.random.Generator(PCG64(seed))``.

Workloads (the paper's test problems, restated):
  * sod            -- Sod shock tube (Sec. 6.1): (rho, p) = (1, 1 | 0.125, 0.1), u = 0
  * kelvin_helmholtz -- periodic shear layer with seeded v_y noise
  * sedov_amr      -- static nested AMR hierarchy around a Sedov-Taylor blast
                      (Sec. 6.2: p = 3 (gamma-1) E / (4 pi r0^3) inside r0)
  * orszag_tang    -- GLM-MHD vortex extended in z (Sec. 7 workload shape)
  * brio_wu        -- MHD shock tube (Sec. 7.2)
  * advected_wave  -- smooth density wave advected through a periodic box
  * uniform        -- a constant state on any hierarchy
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

OUTFLOW, PERIODIC = 0, 1


@dataclass
class Patch:
    level: int
    lo: Tuple[int, int, int]
    n: Tuple[int, int, int]

    @property
    def ncell(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]


@dataclass
class Problem:
    name: str
    nvar: int
    gamma: float
    base_n: Tuple[int, int, int]
    bc: Tuple[int, int, int, int, int, int]
    patches: List[Patch]
    prim: List[np.ndarray]
    domain_lo: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    domain_hi: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    max_level: int = 0
    t_end: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def nlevels(self) -> int:
        return 1 + max(p.level for p in self.patches)

    def cell_updates_per_coarse_step(self) -> int:
        """Sum over levels of cells_l * 2^l (each level subcycles 2^l times)."""
        return sum(p.ncell << p.level for p in self.patches)


def _centres(p: Patch, base_n, dom_lo, dom_hi):
    """Cell-centre coordinates (z, y, x) broadcastable arrays of patch p."""
    out = []
    for d in (2, 1, 0):
        dx = (dom_hi[d] - dom_lo[d]) / (base_n[d] << p.level)
        c = dom_lo[d] + (np.arange(p.n[d]) + p.lo[d] + 0.5) * dx
        shape = [1, 1, 1]
        shape[2 - d] = p.n[d]
        out.append(c.reshape(shape))
    return out  # z, y, x


def partition_axis(length: int, rng: np.random.Generator, lo: int = 8, hi: int = 32) -> List[int]:
    """Split an even length into even pieces in [lo, hi] drawn from rng."""
    assert length % 2 == 0 and length >= lo
    out = []
    rem = length
    while rem > 0:
        if rem <= hi and (rem == hi or rng.random() < 0.35 or rem < 2 * lo):
            out.append(rem)
            break
        choices = [c for c in range(lo, hi + 1, 2) if (rem - c == 0) or (rem - c >= lo)]
        c = int(rng.choice(choices))
        out.append(c)
        rem -= c
    assert sum(out) == length and all(lo <= c <= hi and c % 2 == 0 for c in out)
    return out


def box_patches(level: int, lo: Sequence[int], hi: Sequence[int], rng: np.random.Generator,
                pmin: int = 8, pmax: int = 32) -> List[Patch]:
    """Tile the box [lo, hi) of one level by a tensor product of seeded even lengths."""
    cuts = []
    for d in range(3):
        lens = partition_axis(hi[d] - lo[d], rng, pmin, pmax)
        starts = lo[d] + np.concatenate([[0], np.cumsum(lens)[:-1]])
        cuts.append(list(zip(starts.tolist(), lens)))
    out = []
    for (z0, nz) in cuts[2]:
        for (y0, ny) in cuts[1]:
            for (x0, nx) in cuts[0]:
                out.append(Patch(level, (int(x0), int(y0), int(z0)), (int(nx), int(ny), int(nz))))
    return out


def uniform_patches(N: Sequence[int], tile: Sequence[int]) -> List[Patch]:
    """Level-0 tiling of an N[0] x N[1] x N[2] box by tiles (last ones ragged)."""
    out = []
    for z0 in range(0, N[2], tile[2]):
        for y0 in range(0, N[1], tile[1]):
            for x0 in range(0, N[0], tile[0]):
                out.append(Patch(0, (x0, y0, z0), (min(tile[0], N[0] - x0), min(tile[1], N[1] - y0),
                                                    min(tile[2], N[2] - z0))))
    return out


def _fill(problem_patches, base_n, nvar, fn, dom_lo=(0.0, 0.0, 0.0), dom_hi=(1.0, 1.0, 1.0)):
    prim = []
    for p in problem_patches:
        z, y, x = _centres(p, base_n, dom_lo, dom_hi)
        w = np.zeros((nvar, p.n[2], p.n[1], p.n[0]), dtype=np.float64)
        fn(p, w, x, y, z)
        prim.append(w)
    return prim


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def sod(n: int = 32, axis: int = 0, ny: int | None = None, tile: int | None = None,
        gamma: float = 1.4, t_end: float = 0.2) -> Problem:
    """Sod tube along `axis`: left (rho, p) = (1, 1), right (0.125, 0.1), u = 0, x0 = 0.5, outflow."""
    N = [ny or n, ny or n, ny or n]
    N[axis] = n
    t = tile or max(N)
    patches = uniform_patches(N, (min(t, N[0]), min(t, N[1]), min(t, N[2])))

    def fn(p, w, x, y, z):
        c = (x, y, z)[axis]
        left = np.broadcast_to(c < 0.5, w.shape[1:])
        w[0] = np.where(left, 1.0, 0.125)
        w[4] = np.where(left, 1.0, 0.1)

    return Problem("sod", 5, gamma, tuple(N), (OUTFLOW,) * 6, patches, _fill(patches, N, 5, fn),
                   t_end=t_end, meta={"axis": axis})


def double_rarefaction(n: int = 32, ny: int = 8, tile: int | None = None, u: float = 2.0, p: float = 1e-6,
                       gamma: float = 1.4) -> Problem:
    """Two periodic pairs of receding streams along x (rho = 1, vx = -u for x < 0.5 and +u
    beyond, pressure p): strong rarefactions at x = 0.5 and x = 0 drive the middle towards
    vacuum, the workload of the positivity floor."""
    N = [n, ny, ny]
    t = tile or max(N)
    patches = uniform_patches(N, (min(t, N[0]), min(t, N[1]), min(t, N[2])))

    def fn(pt, w, x, y, z):
        left = np.broadcast_to(x < 0.5, w.shape[1:])
        w[0] = 1.0
        w[1] = np.where(left, -u, u)
        w[4] = p

    return Problem("double_rarefaction", 5, gamma, tuple(N), (PERIODIC,) * 6, patches, _fill(patches, N, 5, fn))


def kelvin_helmholtz(N: int = 256, tile: int | None = 32, seed: int = 20091, amp: float = 0.01,
                     gamma: float = 1.4) -> Problem:
    """Periodic shear layer: rho = 2, vx = +0.5 inside |y - 0.5| < 0.25, rho = 1, vx = -0.5
    outside, p = 2.5, v_y uniform in (-amp, amp) per cell (seeded), v_z = 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.uniform(-amp, amp, size=(N, N, N))  # [z][y][x] over the whole box
    t = tile or N
    patches = uniform_patches((N, N, N), (t, t, t))

    def fn(p, w, x, y, z):
        inside = np.broadcast_to(np.abs(y - 0.5) < 0.25, w.shape[1:])
        w[0] = np.where(inside, 2.0, 1.0)
        w[1] = np.where(inside, 0.5, -0.5)
        w[2] = noise[p.lo[2]:p.lo[2] + p.n[2], p.lo[1]:p.lo[1] + p.n[1], p.lo[0]:p.lo[0] + p.n[0]]
        w[4] = 2.5

    return Problem("kelvin_helmholtz", 5, gamma, (N, N, N), (PERIODIC,) * 6, patches,
                   _fill(patches, (N, N, N), 5, fn), meta={"seed": seed})


def mhd_turbulence(N: int = 128, tile: int | None = None, mach: float = 10.0, gamma: float = 1.001,
                   beta: float = 0.1, slope: float = -2.0, seed: int = 20096) -> Problem:
    """Decaying MHD turbulence (Sec. 7): uniform density rho = 1 and sound speed 1
    (p = 1 / gamma), an isotropic random velocity field with the Burgers-like energy
    spectrum E(k) ~ k^slope (slope -2; E summed over shells |k| = k, i.e. mode power
    |v_k|^2 ~ k^(slope - 2)) for 1 <= |k| <= N/2 with seeded random phases, each
    component drawn independently, scaled to an rms Mach number `mach`; a uniform
    field B = (B0, 0, 0) with plasma beta 2 p / B0^2 = beta (Heaviside units, energy
    B^2/2), psi = 0; periodic, nvar = 9."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = np.fft.fftfreq(N) * N
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(kk)
    band = (kk >= 1.0) & (kk <= N / 2)
    amp[band] = kk[band] ** ((slope - 2.0) / 2.0)
    vel = []
    for _ in range(3):
        coef = amp * (rng.standard_normal(kk.shape) + 1j * rng.standard_normal(kk.shape))
        vel.append(np.real(np.fft.ifftn(coef)))      # [z][y][x]
    vel = np.array(vel)
    p0 = 1.0 / gamma
    vel *= mach / np.sqrt(np.mean(np.sum(vel * vel, axis=0)))
    b0 = np.sqrt(2.0 * p0 / beta)
    t = tile or N
    patches = uniform_patches((N, N, N), (t, t, t))

    def fn(p, w, x, y, z):
        sl = (slice(p.lo[2], p.lo[2] + p.n[2]), slice(p.lo[1], p.lo[1] + p.n[1]), slice(p.lo[0], p.lo[0] + p.n[0]))
        w[0] = 1.0
        for d in range(3):
            w[1 + d] = vel[d][sl]
        w[4] = p0
        w[5] = b0

    return Problem("mhd_turbulence", 9, gamma, (N, N, N), (PERIODIC,) * 6, patches, _fill(patches, (N, N, N), 9, fn),
                   meta={"seed": seed, "mach": mach, "beta": beta})


def nested_cubes(base: int, sides: Sequence[int], seed: int, pmin=8, pmax=32) -> List[Patch]:
    """Level 0 = whole box tiled by seeded 8..32 patches; level l >= 1 = a centred cube of
    `sides[l-1]` level-l cells, tiled the same way."""
    rng = np.random.Generator(np.random.PCG64(seed))
    patches = box_patches(0, (0, 0, 0), (base, base, base), rng, pmin, pmax)
    for l, side in enumerate(sides, start=1):
        Nl = base << l
        lo = (Nl - side) // 2
        assert lo % 2 == 0 and side % 2 == 0
        patches += box_patches(l, (lo,) * 3, (lo + side,) * 3, rng, pmin, pmax)
    return patches


def sedov_prim(patches: List[Patch], base: int, levels: int, gamma: float = 1.4, E: float = 1.0,
               r0_cells: float = 2.0, rho: float = 1.0, p_amb: float = 1e-5):
    """Primitive Sedov-Taylor initial data (Sec. 6.2) on any patches of a hierarchy with
    `levels` refinements over a base^3 unit box: p_in = 3 (gamma-1) E / (4 pi r0^3) in cells
    whose centre lies within r0 = r0_cells finest cells of the box centre."""
    r0 = r0_cells / (base << levels)
    p_in = 3.0 * (gamma - 1.0) * E / (4.0 * np.pi * r0 ** 3)

    def fn(p, w, x, y, z):
        r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
        w[0] = rho
        w[4] = np.where(np.broadcast_to(r2 <= r0 * r0, w.shape[1:]), p_in, p_amb)

    return _fill(patches, (base,) * 3, 5, fn), p_in, r0


def sedov_amr(base: int = 128, sides=(192, 224, 224), seed: int = 20092, gamma: float = 1.4,
              E: float = 1.0, r0_cells: float = 2.0, rho: float = 1.0, p_amb: float = 1e-5) -> Problem:
    """Static nested hierarchy around a Sedov-Taylor blast (Sec. 6.2 set-up): E deposited in
    cells whose centre lies within r0 = r0_cells finest cells of the box centre,
    p_in = 3 (gamma-1) E / (4 pi r0^3); ambient rho and p elsewhere; outflow."""
    patches = nested_cubes(base, sides, seed)
    L = len(sides)
    prim, p_in, r0 = sedov_prim(patches, base, L, gamma, E, r0_cells, rho, p_amb)
    return Problem("sedov_amr", 5, gamma, (base,) * 3, (OUTFLOW,) * 6, patches, prim, max_level=L,
                   meta={"seed": seed, "p_in": p_in, "r0": r0, "sides": tuple(sides)})


def orszag_tang(N: int = 192, tile: int | None = 32, seed: int = 20095, gamma: float = 5.0 / 3.0,
                amr_sides: Sequence[int] | None = None, amr_base: int = 96) -> Problem:
    """GLM-MHD Orszag-Tang vortex, independent of z, plus seeded v_z noise U(-1e-3, 1e-3):
    rho = 25/(36 pi), p = 5/(12 pi), v = (-sin 2pi y, sin 2pi x, 0),
    B = B0 (-sin 2pi y, sin 4pi x, 0), B0 = 1/sqrt(4 pi), psi = 0; periodic."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if amr_sides:
        patches = nested_cubes(amr_base, amr_sides, seed)
        base = amr_base
    else:
        t = tile or N
        patches = uniform_patches((N, N, N), (t, t, t))
        base = N
    noise = [rng.uniform(-1e-3, 1e-3, size=(p.n[2], p.n[1], p.n[0])) for p in patches]
    B0 = 1.0 / np.sqrt(4.0 * np.pi)

    def fn(p, w, x, y, z):
        shp = w.shape[1:]
        w[0] = 25.0 / (36.0 * np.pi)
        w[1] = np.broadcast_to(-np.sin(2 * np.pi * y), shp)
        w[2] = np.broadcast_to(np.sin(2 * np.pi * x), shp)
        w[4] = 5.0 / (12.0 * np.pi)
        w[5] = np.broadcast_to(-B0 * np.sin(2 * np.pi * y), shp)
        w[6] = np.broadcast_to(B0 * np.sin(4 * np.pi * x), shp)

    prim = _fill(patches, (base,) * 3, 9, fn)
    for w, nz in zip(prim, noise):
        w[3] = nz
    return Problem("orszag_tang", 9, gamma, (base,) * 3, (PERIODIC,) * 6, patches, prim,
                   max_level=len(amr_sides or ()), meta={"seed": seed})


def brio_wu(n: int = 200, ny: int = 1, gamma: float = 2.0, t_end: float = 0.1) -> Problem:
    """MHD shock tube along x: left (rho, p, vx, vy, Bx, By) = (1, 1, 0, 0, 0.75, 1), right
    (0.125, 0.1, 0, 0, 0.75, -1), v_z = B_z = psi = 0; outflow in x, periodic in y, z."""
    N = (n, ny, ny)
    patches = [Patch(0, (0, 0, 0), N)]

    def fn(p, w, x, y, z):
        left = np.broadcast_to(x < 0.5, w.shape[1:])
        w[0] = np.where(left, 1.0, 0.125)
        w[4] = np.where(left, 1.0, 0.1)
        w[5] = 0.75
        w[6] = np.where(left, 1.0, -1.0)

    return Problem("brio_wu", 9, gamma, N, (OUTFLOW, OUTFLOW, PERIODIC, PERIODIC, PERIODIC, PERIODIC),
                   patches, _fill(patches, N, 9, fn), t_end=t_end)


def advected_wave(n: int = 64, ny: int = 1, amp: float = 0.2, vel=(1.0, 0.0, 0.0), axis: int = 0,
                  gamma: float = 1.4, tile: int | None = None) -> Problem:
    """rho = 1 + amp sin(2 pi x_axis), v = vel, p = 1 in a periodic box: the exact solution is
    the initial density translated by vel * t."""
    N = [ny, ny, ny]
    N[axis] = n
    t = tile or max(N)
    patches = uniform_patches(N, (min(t, N[0]), min(t, N[1]), min(t, N[2])))

    def fn(p, w, x, y, z):
        c = (x, y, z)[axis]
        w[0] = np.broadcast_to(1.0 + amp * np.sin(2 * np.pi * c), w.shape[1:])
        w[1], w[2], w[3] = vel
        w[4] = 1.0

    return Problem("advected_wave", 5, gamma, tuple(N), (PERIODIC,) * 6, patches,
                   _fill(patches, N, 5, fn), meta={"amp": amp, "vel": vel, "axis": axis})


def uniform(patches: List[Patch], base_n, nvar: int = 5, gamma: float = 1.4, bc=(PERIODIC,) * 6,
            state=(1.3, 0.2, -0.1, 0.3, 0.9, 0.2, -0.3, 0.1, 0.0)) -> Problem:
    """A constant primitive state on any patch set."""

    def fn(p, w, x, y, z):
        for v in range(nvar):
            w[v] = state[v]

    return Problem("uniform", nvar, gamma, tuple(base_n), tuple(bc), patches,
                   _fill(patches, base_n, nvar, fn), max_level=max(p.level for p in patches))


def random_smooth(patches: List[Patch], base_n, nvar: int = 5, seed: int = 7, gamma: float = 1.4,
                  bc=(PERIODIC,) * 6, amp: float = 0.1) -> Problem:
    """Smooth periodic fields made of a few seeded Fourier modes (positive rho and p)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    modes = rng.integers(1, 3, size=(nvar, 3, 3))
    phases = rng.uniform(0, 2 * np.pi, size=(nvar, 3))
    base_state = np.array([1.0, 0.3, -0.2, 0.1, 1.0, 0.3, 0.2, -0.1, 0.0])[:nvar]

    def fn(p, w, x, y, z):
        for v in range(nvar):
            f = np.zeros(w.shape[1:])
            for m in range(3):
                kx, ky, kz = modes[v, m]
                f = f + np.sin(2 * np.pi * (kx * x + ky * y + kz * z) + phases[v, m])
            w[v] = base_state[v] + amp * f / 3.0

    return Problem("random_smooth", nvar, gamma, tuple(base_n), tuple(bc), patches,
                   _fill(patches, base_n, nvar, fn), max_level=max(p.level for p in patches),
                   meta={"seed": seed})


def cp_alfven(n: int = 32, amp: float = 0.1, rho: float = 1.0, p: float = 0.1, Bx: float = 1.0,
              gamma: float = 5.0 / 3.0) -> Problem:
    """Circularly polarised Alfven wave along x (an exact nonlinear ideal-MHD solution):
    v_perp = amp (0, sin 2pi x, cos 2pi x), B_perp = -sqrt(rho) v_perp, uniform rho, p, Bx;
    it travels at Bx / sqrt(rho) in +x.  Periodic, quasi-1D (n x 1 x 1)."""
    N = (n, 1, 1)
    patches = [Patch(0, (0, 0, 0), N)]

    def fn(pt, w, x, y, z):
        shp = w.shape[1:]
        s, c = np.broadcast_to(np.sin(2 * np.pi * x), shp), np.broadcast_to(np.cos(2 * np.pi * x), shp)
        w[0] = rho
        w[2] = amp * s
        w[3] = amp * c
        w[4] = p
        w[5] = Bx
        w[6] = -np.sqrt(rho) * amp * s
        w[7] = -np.sqrt(rho) * amp * c

    return Problem("cp_alfven", 9, gamma, N, (PERIODIC,) * 6, patches, _fill(patches, N, 9, fn),
                   meta={"amp": amp, "speed": Bx / np.sqrt(rho)})


def _trilinear_periodic(field: np.ndarray, x, y, z):
    """Periodic trilinear interpolation of a cell-centred unit-box field [z][y][x] at points."""
    n = field.shape[0]
    gx, gy, gz = x * n - 0.5, y * n - 0.5, z * n - 0.5
    i0, j0, k0 = np.floor(gx).astype(int), np.floor(gy).astype(int), np.floor(gz).astype(int)
    fx, fy, fz = gx - i0, gy - j0, gz - k0
    out = 0.0
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                w = (fx if di else 1 - fx) * (fy if dj else 1 - fy) * (fz if dk else 1 - fz)
                out = out + w * field[(k0 + dk) % n, (j0 + dj) % n, (i0 + di) % n]
    return out


def blast_clumps(base: int = 64, levels: int = 5, side: int = 64, seed: int = 20093, sigma: float = 1.0,
                 smooth: float = 2.0, gamma: float = 1.4, E: float = 1.0, r0_cells: float = 2.0,
                 p_amb: float = 1e-5) -> Problem:
    """Adaptive-AMR workload: a spherical blast (Sec. 6.2 deposit in r <= r0_cells finest cells)
    in a seeded log-normal clump field rho = exp(sigma g - sigma^2 / 2), g unit-variance Gaussian
    white noise on the base grid smoothed by a Gaussian of `smooth` base cells (periodic FFT) and
    sampled trilinearly at every level; pressure p_amb outside the blast; outflow.  The initial
    hierarchy is `levels` nested centred cubes of `side` cells around the blast (seeded 8-32
    patches); later hierarchies come from regridding."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal((base,) * 3)
    k = np.fft.fftfreq(base) * base
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    filt = np.exp(-0.5 * (2 * np.pi * smooth / base) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    g = np.real(np.fft.ifftn(np.fft.fftn(g) * filt))
    g = (g - g.mean()) / g.std()
    patches = nested_cubes(base, (side,) * levels, seed)
    r0 = r0_cells / (base << levels)
    p_in = 3.0 * (gamma - 1.0) * E / (4.0 * np.pi * r0 ** 3)

    def fn(p, w, x, y, z):
        shp = w.shape[1:]
        X, Y, Z = np.broadcast_arrays(x, y, z)
        w[0] = np.exp(sigma * _trilinear_periodic(g, X, Y, Z) - 0.5 * sigma ** 2).reshape(shp)
        r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2
        w[4] = np.where(r2 <= r0 * r0, p_in, p_amb)

    return Problem("blast_clumps", 5, gamma, (base,) * 3, (OUTFLOW,) * 6, patches,
                   _fill(patches, (base,) * 3, 5, fn), max_level=levels,
                   meta={"seed": seed, "p_in": p_in, "r0": r0})

