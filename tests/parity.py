"""Error metrics used by the GPU parity tests.

Per conserved variable v, over all cells of all patches weighted by cell
volume:  L1 rel = sum |U - U_ref| dV / S_v,  max rel = max |U - U_ref| / M_v.
S_v (M_v) is the L1 norm (max) of the variable itself for rho and rho E; for a
component of a vector (momentum, magnetic field) it is the norm of the whole
vector (sum over its three components), so that a component that is nearly
zero in a given problem (e.g. z-momentum of a flow without z-motion) is
measured against the vector it belongs to, independent of the axes; psi is
measured against the magnetic-field norm.
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


def assert_parity(got, ref, patches, precision, label=""):
    l1, mx = errors(got, ref, patches)
    tol = TOL[precision]
    assert np.all(np.isfinite(l1)), (label, l1)
    assert l1.max() <= tol["l1"], f"{label} {precision} L1 rel {l1}"
    if "max" in tol:
        assert mx.max() <= tol["max"], f"{label} {precision} max rel {mx}"
    return l1.max(), mx.max()
