"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every entry point declared in include/amr.h, and the host-only patch
validation returns the documented status codes."""
import os
import re

import pytest

import amr_inputs as ai
from paper_0910_5547_gb300 import build as B
from paper_0910_5547_gb300 import native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    yield


def declared_entry_points():
    txt = open(os.path.join(ROOT, "include", "amr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(amr_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    import ctypes
    lib = ctypes.CDLL(B.LIB)
    names = declared_entry_points()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(N.EXPORTS) == names


def test_tiling_on_a_null_handle_is_rejected():
    assert N.load().amr_set_tiling(None, 0, 0, 0, 0) == N.AMR_ERR_ARG


def cfg(**kw):
    return N.amr_default_config(**kw)


def P(level, lo, n):
    return ai.Patch(level, tuple(lo), tuple(n))


def test_valid_uniform_and_amr_sets():
    assert N.amr_validate_patches(cfg(base_n=(32, 32, 32)), [P(0, (0, 0, 0), (32, 32, 32))])[0] == N.AMR_OK
    two = ai.uniform_patches((16, 16, 16), (8, 8, 8)) + [P(1, (8, 8, 8), (16, 16, 16))]
    assert N.amr_validate_patches(cfg(base_n=(16, 16, 16), max_level=1), two)[0] == N.AMR_OK


def test_full_size_static_hierarchy_validates():
    pb = ai.sedov_amr()
    c = cfg(base_n=pb.base_n, max_level=pb.max_level)
    st, msg = N.amr_validate_patches(c, pb.patches)
    assert st == N.AMR_OK, msg
    assert 3500 < len(pb.patches) < 4500


@pytest.mark.parametrize("patches,base,maxl,want", [
    ([P(0, (0, 0, 0), (16, 16, 8)), P(0, (0, 0, 4), (16, 16, 8))], (16, 16, 16), 0, N.AMR_ERR_NESTING),  # overlap
    ([P(0, (0, 0, 0), (16, 16, 8))], (16, 16, 16), 0, N.AMR_ERR_NESTING),                               # gap
    ([P(0, (0, 0, 0), (16, 16, 16)), P(1, (9, 8, 8), (8, 8, 8))], (16, 16, 16), 1, N.AMR_ERR_NESTING),  # odd lo
    ([P(0, (0, 0, 0), (16, 16, 16)), P(1, (8, 8, 8), (7, 8, 8))], (16, 16, 16), 1, N.AMR_ERR_NESTING),  # odd n
    ([P(0, (0, 0, 0), (16, 16, 16)), P(1, (0, 8, 8), (8, 8, 8))], (16, 16, 16), 1, N.AMR_OK),           # at outflow face
    ([P(0, (0, 0, 0), (16, 16, 16)), P(1, (2, 8, 8), (8, 8, 8)), P(2, (4, 16, 16), (8, 8, 8))], (16, 16, 16), 2,
     N.AMR_ERR_NESTING),                                                                                    # not nested
    ([P(0, (0, 0, 0), (1, 16, 16)), P(0, (1, 0, 0), (15, 16, 16))], (16, 16, 16), 0, N.AMR_ERR_ARG),     # size 1
    ([P(0, (0, 0, 0), (16, 16, 16)), P(1, (8, 8, 8), (8, 8, 8))], (16, 16, 16), 0, N.AMR_ERR_ARG),       # level > max
    ([P(1, (8, 8, 8), (8, 8, 8)), P(0, (0, 0, 0), (16, 16, 16))], (16, 16, 16), 1, N.AMR_ERR_ARG),       # unsorted
    ([P(0, (0, 0, 0), (16, 16, 16)), P(1, (28, 8, 8), (4, 8, 8))], (16, 16, 16), 1, N.AMR_OK),           # at outflow face
])
def test_validation_status_codes(patches, base, maxl, want):
    st, msg = N.amr_validate_patches(cfg(base_n=base, max_level=maxl), patches)
    assert st == want, msg


def test_empty_patch_set_is_rejected():
    st, msg = N.amr_validate_patches(cfg(), [])
    assert st == N.AMR_ERR_ARG, msg


def test_periodic_nesting_wraps_around_the_domain():
    base = (16, 16, 16)
    pats = [P(0, (0, 0, 0), (16, 16, 16)), P(1, (0, 8, 8), (8, 8, 8))]
    assert N.amr_validate_patches(cfg(base_n=base, max_level=1, bc=(1,) * 6), pats)[0] == N.AMR_OK
    # level 2 patch near the periodic x face needs level-1 coverage across the wrap
    pats2 = pats + [P(2, (0, 20, 20), (8, 8, 8))]
    st, _ = N.amr_validate_patches(cfg(base_n=base, max_level=2, bc=(1,) * 6), pats2)
    assert st == N.AMR_ERR_NESTING


@pytest.mark.parametrize("field,value", [("nvar", 7), ("precision", 3), ("gamma", 1.0), ("theta", 2.5),
                                         ("cfl", 0.0), ("ref_ratio", 4), ("max_level", 13), ("recon", 2)])
def test_bad_config_is_rejected(field, value):
    c = cfg(**{field: value})
    st, msg = N.amr_validate_patches(c, [P(0, (0, 0, 0), (32, 32, 32))])
    assert st == N.AMR_ERR_ARG, msg


def test_flux_reconstruction_is_euler_only():
    one = [P(0, (0, 0, 0), (32, 32, 32))]
    assert N.amr_validate_patches(cfg(riemann=N.AMR_FLUXREC), one)[0] == N.AMR_OK
    st, msg = N.amr_validate_patches(cfg(riemann=N.AMR_FLUXREC, nvar=9), one)
    assert st == N.AMR_ERR_ARG and "FLUXREC" in msg
    assert N.amr_validate_patches(cfg(riemann=3), one)[0] == N.AMR_ERR_ARG


def test_weno3_needs_a_riemann_solve():
    one = [P(0, (0, 0, 0), (32, 32, 32))]
    for nvar in (5, 9):
        for r in (N.AMR_HLL, N.AMR_LLF):
            assert N.amr_validate_patches(cfg(recon=N.AMR_WENO3, riemann=r, nvar=nvar), one)[0] == N.AMR_OK
    st, msg = N.amr_validate_patches(cfg(recon=N.AMR_WENO3, riemann=N.AMR_FLUXREC), one)
    assert st == N.AMR_ERR_ARG and "WENO3" in msg


def test_unpaired_periodic_faces_rejected():
    st, msg = N.amr_validate_patches(cfg(bc=(1, 0, 0, 0, 0, 0)), [P(0, (0, 0, 0), (32, 32, 32))])
    assert st == N.AMR_ERR_ARG and "periodic" in msg


def test_config_struct_layout_matches_the_header(tmp_path):
    """The ctypes amr_config has the size and field offsets of the C struct in
    include/amr.h (compiled here with the host C compiler)."""
    import ctypes
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in N.amr_config._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"amr.h\"\nint main(void) {\n"
                   "  printf(\"%zu\\n\", sizeof(amr_config));\n"
                   + "".join(f"  printf(\"%zu\\n\", offsetof(amr_config, {f}));\n" for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got[0] == ctypes.sizeof(N.amr_config)
    assert got[1:] == [getattr(N.amr_config, f).offset for f in fields]
