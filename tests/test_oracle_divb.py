"""Pins of the oracle's div B diagnostic (GLM-MHD, Sec. 7.1: psi exists to keep
div B small; the norms are the plain centred difference over leaf cells).

* A periodic product-free trigonometric field: the centred difference of
  sin(k x + phi) over two cells is cos(k x + phi) sin(k h) / h exactly (sum-to-
  product identity), so the discrete divergence has a closed form on any
  anisotropic grid and any patch decomposition.
* A linear field on a two-level outflow hierarchy: each B_d is independent of
  x_d except for alpha x in B_x, so D = alpha in every interior leaf cell and
  alpha / 2 in the leaf cells of the two x faces (outflow ghosts copy the edge
  cell); covered cells are excluded, fine cells weigh their own volume.
* A constant field: D = 0, and the |B| / dx_min normalisation is a sum of leaf
  volumes over the level's cell size.
"""
import math

import numpy as np
import pytest

import amr_inputs as ai
import oracle as orc

P, O = ai.PERIODIC, ai.OUTFLOW


def _problem(patches, base_n, bfn, bc, dom_hi=(1.0, 1.0, 1.0)):
    def fn(p, w, x, y, z):
        w[0] = 1.0
        w[4] = 1.0
        bx, by, bz = bfn(x, y, z)
        w[5] = bx
        w[6] = by
        w[7] = bz

    return ai.Problem("divb", 9, 5.0 / 3.0, tuple(base_n), tuple(bc), patches,
                      ai._fill(patches, base_n, 9, fn, (0.0, 0.0, 0.0), dom_hi),
                      domain_hi=dom_hi, max_level=max(p.level for p in patches))


def test_trig_field_closed_form_anisotropic_patches():
    base, L = (16, 12, 8), (1.0, 2.0, 0.5)
    h = [L[d] / base[d] for d in range(3)]
    A, k, ph = (0.7, -1.3, 0.4), (1, 2, 1), (0.3, 1.1, -0.6)
    kap = [2 * math.pi * k[d] / L[d] for d in range(3)]

    def bfn(x, y, z):
        s = [A[d] * np.sin(kap[d] * c + ph[d]) for d, c in enumerate((x, y, z))]
        shp = np.broadcast_shapes(x.shape, y.shape, z.shape)
        return [np.broadcast_to(v, shp) for v in s]

    pb = _problem(ai.uniform_patches(base, (8, 6, 4)), base, bfn, (P,) * 6, L)
    got = orc.Oracle(pb, nthreads=4).divb_norms()
    # closed form at the cell centres of the whole box
    c = [(np.arange(base[d]) + 0.5) * h[d] for d in range(3)]
    X, Y, Zc = np.meshgrid(c[0], c[1], c[2], indexing="ij")
    D = sum(A[d] * np.cos(kap[d] * q + ph[d]) * math.sin(kap[d] * h[d]) / h[d]
            for d, q in enumerate((X, Y, Zc)))
    Bm = np.sqrt(sum((A[d] * np.sin(kap[d] * q + ph[d])) ** 2 for d, q in enumerate((X, Y, Zc)))) / min(h)
    vol = h[0] * h[1] * h[2]
    want = [np.abs(D).sum() * vol, np.abs(D).max(), Bm.sum() * vol, Bm.max()]
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * want[2])


def _two_level():
    patches = ai.uniform_patches((16,) * 3, (8,) * 3)
    patches.append(ai.Patch(1, (8, 8, 8), (16, 16, 16)))   # coarse cells 4..11, away from every face
    return patches


def test_linear_field_on_two_levels_outflow():
    alpha = 0.37

    def bfn(x, y, z):
        return [alpha * x + 0.5 * y - 0.2 * z, 0.3 * z + 0.8 * x, -0.6 * x + 0.25 * y]

    pb = _problem(_two_level(), (16,) * 3, bfn, (O,) * 6)
    got = orc.Oracle(pb, nthreads=4).divb_norms()
    h0 = 1.0 / 16
    assert got[0] == pytest.approx(alpha * (1.0 - h0), rel=1e-12)
    assert got[1] == pytest.approx(alpha, rel=1e-12)


def test_constant_field_normalisation_on_two_levels():
    B = np.array([0.4, -0.9, 0.2])
    pb = _problem(_two_level(), (16,) * 3, lambda x, y, z: [np.full(np.broadcast_shapes(x.shape, y.shape, z.shape),
                                                                   b) for b in B], (O,) * 6)
    got = orc.Oracle(pb, nthreads=4).divb_norms()
    h0, h1 = 1.0 / 16, 1.0 / 32
    v_fine = 0.5 ** 3                       # the level-1 patch covers half of each axis
    bmag = float(np.linalg.norm(B))
    assert got[0] == 0.0 and got[1] == 0.0
    assert got[2] == pytest.approx(bmag * ((1.0 - v_fine) / h0 + v_fine / h1), rel=1e-13)
    assert got[3] == pytest.approx(bmag / h1, rel=1e-13)


def test_divb_needs_mhd():
    pb = ai.uniform(ai.uniform_patches((8,) * 3, (8,) * 3), (8,) * 3)
    with pytest.raises(RuntimeError):
        orc.Oracle(pb, nthreads=1).divb_norms()
