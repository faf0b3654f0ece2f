"""Error metrics used by the GPU parity tests.

Per conserved variable v, over all cells of all patches weighted by cell
volume:  L1 rel = sum |U - U_ref| dV / sum |U_ref| dV, where a variable whose
reference norm is below 1e-12 of the density norm is normalised by the density
norm instead;  max rel = max |U - U_ref| / max |U_ref| (same fallback).
"""
import numpy as np

TOL = {
    "fp64": {"l1": 1e-10, "max": 1e-8},
    "fp32": {"l1": 2e-5},
}


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
    small = den < 1e-12 * den[0]
    den[small] = den[0]
    ref_mx[ref_mx < 1e-12 * ref_mx[0]] = ref_mx[0]
    return num / den, mx / ref_mx


def assert_parity(got, ref, patches, precision, label=""):
    l1, mx = errors(got, ref, patches)
    tol = TOL[precision]
    assert np.all(np.isfinite(l1)), (label, l1)
    assert l1.max() <= tol["l1"], f"{label} {precision} L1 rel {l1}"
    if "max" in tol:
        assert mx.max() <= tol["max"], f"{label} {precision} max rel {mx}"
    return l1.max(), mx.max()
