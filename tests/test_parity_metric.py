"""Host-side checks of the parity metrics (no GPU): leaf masks of a nested
hierarchy, the per-variable normalisation and its zero-field fallback."""
import numpy as np

import amr_inputs as ai
from parity import errors, errors_per_variable, leaf_masks


def test_leaf_masks_of_two_levels():
    base = ai.uniform_patches((16, 16, 16), (8, 8, 8))
    fine = [ai.Patch(1, (8, 8, 8), (8, 16, 16)), ai.Patch(1, (16, 8, 8), (8, 16, 16))]
    m = leaf_masks(base + fine)
    covered = sum(int((~x).sum()) for x in m[:len(base)])
    assert covered == 8 * 8 * 8                       # the fine box [8, 24)^3 covers [4, 12)^3 coarse
    assert all(x.all() for x in m[len(base):])         # the finest level is all leaf
    # patch (0,0,0) covers coarse [0,8)^3: its covered part is [4,8)^3
    assert int((~m[0]).sum()) == 4 ** 3 and not m[0][4:, 4:, 4:].any()


def test_per_variable_metric_and_fallback():
    p = [ai.Patch(0, (0, 0, 0), (4, 4, 4))]
    ref = np.zeros((5, 4, 4, 4))
    ref[0] = 2.0
    ref[1] = 1.0
    ref[3] = 1e-3           # small but nonzero: normalised by itself
    ref[4] = 5.0            # ref[2] stays zero: normalised by rho
    got = ref.copy()
    got[1] += 1e-6
    got[2] += 1e-6
    got[3] += 1e-6
    l1, mx = errors_per_variable([got], [ref], p)
    np.testing.assert_allclose(l1, [0, 1e-6, 5e-7, 1e-3, 0], rtol=1e-9, atol=1e-20)
    np.testing.assert_allclose(mx, [0, 1e-6, 5e-7, 1e-3, 0], rtol=1e-9, atol=1e-20)
    # the vector metric divides m_z's error by the whole momentum norm (1 + 1e-3)
    v1, _ = errors([got], [ref], p)
    assert abs(v1[3] - 1e-6 / (1.0 + 1e-3)) < 1e-15
