"""Error metrics used by the GPU parity tests.

Two metrics, both per conserved variable v and weighted by cell volume:

* ``errors_per_variable`` (the plain per-variable metric, over LEAF cells, i.e.
  cells no finer patch covers):
      L1 rel  = sum |U_v - U_ref,v| dV / sum |U_ref,v| dV
      max rel = max |U_v - U_ref,v| / max |U_ref,v|
  A variable whose reference norm is below 1e-12 of the density's (a field
  that is zero in the problem) is normalised by the density's norm instead.

* ``errors`` (the vector-normalised metric, over all cells of all patches):
  the same sums, but a component of a vector (momentum, magnetic field) is
  divided by the norm of the whole vector (sum over its three components) and
  psi by the magnetic-field norm, so a component that is nearly zero in a given
  problem is measured against the vector it belongs to, independent of the axes.

``assert_parity`` asserts the tolerances on both metrics for FP64 and on the
vector metric for FP32, records every result, and the test session prints the
worst of each (``tests/conftest.py``), so the FP32 per-variable figure is always
reported next to the asserted one.
"""
import numpy as np

TOL = {
    "fp64": {"l1": 1e-10, "max": 1e-8},
    "fp32": {"l1": 2e-5},
}

# (label, precision, vector L1 (max over vars), per-variable L1 array, per-variable max array)
RECORDS = []


def errors(got, ref, patches):
    nv = ref[0].shape[0]
    num = np.zeros(nv)
    den = np.zeros(nv)
    mx = np.zeros(nv)
    ref_mx = np.zeros(nv)
    for g, r, p in zip(got, ref, patches):
        vol = 8.0 ** (-p.level)
        d = np.abs(g - r).reshape(nv, -1)
        num += d.sum(axis=1) * vol
        den += np.abs(r).reshape(nv, -1).sum(axis=1) * vol
        mx = np.maximum(mx, d.max(axis=1))
        ref_mx = np.maximum(ref_mx, np.abs(r).reshape(nv, -1).max(axis=1))
    S = den.copy()
    M = ref_mx.copy()
    S[1:4] = den[1:4].sum()
    M[1:4] = ref_mx[1:4].max()
    if nv == 9:
        S[5:9] = den[5:8].sum()
        M[5:9] = ref_mx[5:8].max()
    S[S < 1e-12 * S[0]] = S[0]
    M[M < 1e-12 * M[0]] = M[0]
    return num / S, mx / M


def leaf_masks(patches):
    """Per patch, a boolean (nz, ny, nx) array: True where no patch of the next
    level covers the cell (a level-(l+1) patch covers the level-l cells
    [lo // 2, (lo + n) // 2) on every axis)."""
    masks = []
    by_level = {}
    for q in patches:
        by_level.setdefault(q.level, []).append(q)
    arrs = {}
    for lev, qs in by_level.items():
        lo = np.array([q.lo for q in qs]) // 2
        hi = (np.array([q.lo for q in qs]) + np.array([q.n for q in qs])) // 2
        arrs[lev] = (lo, hi)
    for p in patches:
        m = np.ones((p.n[2], p.n[1], p.n[0]), dtype=bool)
        if p.level + 1 in arrs:
            lo, hi = arrs[p.level + 1]
            plo = np.array(p.lo)
            phi = plo + np.array(p.n)
            a = np.maximum(lo, plo)
            b = np.minimum(hi, phi)
            hit = np.all(b > a, axis=1)
            for ai_, bi_ in zip(a[hit], b[hit]):
                s = ai_ - plo
                e = bi_ - plo
                m[s[2]:e[2], s[1]:e[1], s[0]:e[0]] = False
        masks.append(m)
    return masks


def errors_per_variable(got, ref, patches, masks=None):
    """L1 and max relative error of every variable over leaf cells (the
    per-variable metric; see the module docstring)."""
    nv = ref[0].shape[0]
    if masks is None:
        masks = leaf_masks(patches)
    num = np.zeros(nv)
    den = np.zeros(nv)
    mx = np.zeros(nv)
    ref_mx = np.zeros(nv)
    for g, r, p, m in zip(got, ref, patches, masks):
        if not m.any():
            continue
        vol = 8.0 ** (-p.level)
        d = np.abs(g - r)[:, m]
        a = np.abs(r)[:, m]
        num += d.sum(axis=1) * vol
        den += a.sum(axis=1) * vol
        mx = np.maximum(mx, d.max(axis=1))
        ref_mx = np.maximum(ref_mx, a.max(axis=1))
    den[den < 1e-12 * den[0]] = den[0]
    ref_mx[ref_mx < 1e-12 * ref_mx[0]] = ref_mx[0]
    return num / den, mx / ref_mx


def assert_parity(got, ref, patches, precision, label=""):
    l1, mx = errors(got, ref, patches)
    pl1, pmx = errors_per_variable(got, ref, patches)
    RECORDS.append((label, precision, float(l1.max()), pl1, pmx))
    tol = TOL[precision]
    assert np.all(np.isfinite(l1)), (label, l1)
    assert l1.max() <= tol["l1"], f"{label} {precision} L1 rel {l1}"
    if "max" in tol:
        assert mx.max() <= tol["max"], f"{label} {precision} max rel {mx}"
    if precision == "fp64":
        assert pl1.max() <= tol["l1"], f"{label} fp64 per-variable L1 rel {pl1}"
        assert pmx.max() <= tol["max"], f"{label} fp64 per-variable max rel {pmx}"
    return l1.max(), mx.max()


VAR_NAMES = {5: ("rho", "mx", "my", "mz", "E"),
             9: ("rho", "mx", "my", "mz", "E", "Bx", "By", "Bz", "psi")}


def summary_lines():
    """Worst recorded errors per precision: vector metric and per-variable metric."""
    out = []
    for prec in ("fp64", "fp32"):
        rs = [r for r in RECORDS if r[1] == prec]
        if not rs:
            continue
        vec = max(rs, key=lambda r: r[2])
        pv = max(rs, key=lambda r: float(r[3].max()))
        pm = max(rs, key=lambda r: float(r[4].max()))
        name = lambda a: VAR_NAMES[len(a)][int(np.argmax(a))] if len(a) in VAR_NAMES else "?"
        out.append(f"parity {prec}: {len(rs)} checks; worst vector-metric L1 {vec[2]:.2e} ({vec[0]}); "
                   f"worst per-variable L1 {pv[3].max():.2e} ({pv[0]}, {name(pv[3])}), "
                   f"max {pm[4].max():.2e} ({pm[0]}, {name(pm[4])})")
    for r in RECORDS:
        if r[0].startswith("fullsize"):
            out.append(f"{r[0]}: vector-metric L1 {r[2]:.2e}; per-variable L1 "
                       + " ".join(f"{x:.1e}" for x in r[3]) + "; max " + " ".join(f"{x:.1e}" for x in r[4]))
    return out
