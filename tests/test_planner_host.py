"""Host planner checks that need no GPU, with the planner source compiled with a
small C++ driver (`planner_check.cpp`):
* the regrid fill of a new hierarchy fills every cell of every rebuilt patch
  exactly once, from the old patches of its level (copy segments that keep each
  cell in place) or by prolongation (fresh boxes);
* the ghost tables cover each of the two ghost layers of every patch face
  exactly once (same-level copies of the right level cell, periodic images,
  outflow boundary cells, or prolongation boxes) and nothing else;
* the flux-register rectangles hold exactly the coarse cells next to each fine
  patch face that the fine level does not cover (Sec. 3's correction), each
  once, and a rectangle reflowed in any order shares no cell with another;
* the stage work items, per patch and batched (blocks over z-layers of patches
  that tile a rectangle included), cover every interior cell exactly once;
* the parent-tile gathers hold, once each, every parent cell the prolongation
  reads, taken from the right coarse cell;
* every coarse cell under a finer patch is restricted once, from the patch that
  holds its children, and the leaf-coverage boxes mark exactly those cells;
* a face whose ghost layers the stage kernel reads in place maps each ghost
  cell to the interior cell at that level position (periodic image) or to the
  patch's own boundary cell (outflow);
* the flattened lists the batched kernels walk address the same cells as the
  boxes they come from (prolongation by parent cell, ghost copies);
* the host clustering of flagged cells into new patches gives the oracle's
  hierarchy (oracle.regrid.cluster, an independent implementation)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import amr_inputs as ai

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_0910_5547_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not found")
    out = str(tmp_path_factory.mktemp("planner") / "planner_check")
    cmd = ["g++", "-O1", "-std=c++17", "-pthread", "-I", CSRC, os.path.join(HERE, "planner_check.cpp"),
           os.path.join(CSRC, "hierarchy.cpp"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def listing(patches):
    lines = [str(len(patches))]
    lines += [" ".join(map(str, (p.level, *p.lo, *p.n))) for p in patches]
    return "\n".join(lines)


def run(checker, base, max_level, old, new):
    text = f"fill {base} {base} {base} {max_level}\n{listing(old)}\n{listing(new)}\n"
    r = subprocess.run([checker], input=text, capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    return [int(x) for x in r.stdout.split()[1:]]


def test_fill_covers_every_rebuilt_cell_once(checker):
    # the same nested cubes tiled by two seeded partitions: partial overlaps everywhere
    old = ai.nested_cubes(32, (32, 32), 11, pmin=8, pmax=16)
    new = ai.nested_cubes(32, (32, 32), 12, pmin=8, pmax=16)
    segs, fresh = run(checker, 32, 2, old, new)
    assert segs > 0 and fresh == 0   # same covered region: everything is copied


def test_fill_prolongs_the_cells_no_old_patch_held(checker):
    # larger refined cubes than before: the new cells outside the old cubes are prolonged
    old = ai.nested_cubes(32, (24, 24), 21, pmin=8, pmax=16)
    new = ai.nested_cubes(32, (40, 48), 22, pmin=8, pmax=24)
    segs, fresh = run(checker, 32, 2, old, new)
    assert segs > 0 and fresh > 0


def test_fill_with_shifted_and_shrunk_levels(checker):
    rng = np.random.Generator(np.random.PCG64(5))
    old = ai.nested_cubes(32, (32, 40), 31, pmin=8, pmax=16)
    new = [p for p in ai.nested_cubes(32, (16, 24), 32, pmin=8, pmax=16)]
    # drop a few refined patches of the new hierarchy (holes are allowed for the fill)
    keep = [p for p in new if p.level == 0 or rng.random() > 0.2]
    run(checker, 32, 2, old, keep)


def ghost(checker, base, max_level, bc, patches, mode="ghost"):
    text = f"{mode} {base} {base} {base} {max_level} {' '.join(map(str, bc))}\n{listing(patches)}\n"
    r = subprocess.run([checker], input=text, capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    return [int(x) for x in r.stdout.split()[1:]]


@pytest.mark.parametrize("bc", [(ai.PERIODIC,) * 6, (ai.OUTFLOW,) * 6,
                                (ai.PERIODIC, ai.PERIODIC, ai.OUTFLOW, ai.OUTFLOW, ai.PERIODIC, ai.PERIODIC)])
def test_ghost_layers_covered_once(checker, bc):
    segs, boxes = ghost(checker, 32, 2, bc, ai.nested_cubes(32, (32, 32), 11, pmin=8, pmax=16))
    assert segs > 0 and boxes > 0


def test_ghost_layers_of_the_sedov_hierarchy(checker):
    pb = ai.sedov_amr()
    segs, boxes = ghost(checker, pb.base_n[0], pb.max_level, pb.bc, pb.patches)
    assert segs > 0 and boxes > 0


@pytest.mark.parametrize("bc", [(ai.PERIODIC,) * 6, (ai.OUTFLOW,) * 6,
                                (ai.PERIODIC, ai.PERIODIC, ai.OUTFLOW, ai.OUTFLOW, ai.PERIODIC, ai.PERIODIC)])
def test_register_cells(checker, bc):
    (n,) = ghost(checker, 32, 2, bc, ai.nested_cubes(32, (32, 32), 11, pmin=8, pmax=16), mode="registers")
    assert n > 0


def test_register_cells_of_a_refined_region_touching_the_domain_boundary(checker):
    # the level-1 cube spans the whole domain along x: periodic registers wrap, outflow ones stop
    base = 16
    patches = ai.box_patches(0, (0, 0, 0), (base,) * 3, np.random.Generator(np.random.PCG64(3)), 4, 8)
    patches += ai.box_patches(1, (0, 8, 8), (32, 24, 24), np.random.Generator(np.random.PCG64(4)), 4, 8)
    for bc in ((ai.PERIODIC,) * 6, (ai.OUTFLOW,) * 6):
        (n,) = ghost(checker, base, 1, bc, patches, mode="registers")
        assert n > 0


def test_register_cells_on_partly_covered_faces(checker):
    # a refined slab attached to one face of a refined cube: the cube's patch faces
    # there border the fine level over most of their area, but not all of it
    base = 32
    rng = np.random.Generator(np.random.PCG64(7))
    patches = ai.box_patches(0, (0, 0, 0), (base,) * 3, rng, 8, 16)
    patches += ai.box_patches(1, (16, 16, 16), (40, 40, 40), rng, 8, 16)
    patches += ai.box_patches(1, (40, 16, 16), (48, 40, 36), rng, 8, 12)
    for bc in ((ai.PERIODIC,) * 6, (ai.OUTFLOW,) * 6):
        (n,) = ghost(checker, base, 1, bc, patches, mode="registers")
        assert n > 0
        segs, boxes = ghost(checker, base, 1, bc, patches)
        assert boxes > 0


@pytest.mark.parametrize("tiling", [(32, 256, 32), (16, 256, 16), (16, 128, 8), (32, 256, 64)])
def test_stage_items_cover_every_cell_once(checker, tiling):
    pb = ai.sedov_amr()
    text = (f"items {pb.base_n[0]} {pb.base_n[1]} {pb.base_n[2]} {pb.max_level} {' '.join(map(str, pb.bc))}\n"
            f"{listing(pb.patches)}\n{' '.join(map(str, tiling))}\n")
    r = subprocess.run([checker], input=text, capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    nitems, nspan = [int(x) for x in r.stdout.split()[1:]]
    assert nspan > 0   # the nested cubes' z-layers tile rectangles: blocks span patches


@pytest.mark.parametrize("bc", [(ai.PERIODIC,) * 6, (ai.OUTFLOW,) * 6])
def test_gathers_hold_every_parent_cell_the_prolongation_reads(checker, bc):
    (n,) = ghost(checker, 32, 2, bc, ai.nested_cubes(32, (32, 32), 11, pmin=8, pmax=16), mode="gathers")
    assert n > 0
    base = 16   # a refined region across the whole domain along x: wrapped or clamped parents
    patches = ai.box_patches(0, (0, 0, 0), (base,) * 3, np.random.Generator(np.random.PCG64(3)), 4, 8)
    patches += ai.box_patches(1, (0, 8, 8), (32, 24, 24), np.random.Generator(np.random.PCG64(4)), 4, 8)
    (n,) = ghost(checker, base, 1, bc, patches, mode="gathers")
    assert n > 0


def test_restriction_and_coverage(checker):
    (n,) = ghost(checker, 32, 2, (ai.PERIODIC,) * 6, ai.nested_cubes(32, (32, 32), 11, pmin=8, pmax=16),
                 mode="restrict")
    assert n == 16 ** 3 + 16 ** 3   # the two refined cubes of 32^3 fine cells cover 16^3 cells each below
    base = 32
    rng = np.random.Generator(np.random.PCG64(7))
    patches = ai.box_patches(0, (0, 0, 0), (base,) * 3, rng, 8, 16)
    patches += ai.box_patches(1, (16, 16, 16), (40, 40, 40), rng, 8, 16)
    patches += ai.box_patches(1, (40, 16, 16), (48, 40, 36), rng, 8, 12)
    (n,) = ghost(checker, base, 1, (ai.OUTFLOW,) * 6, patches, mode="restrict")
    assert n == 12 ** 3 + 4 * 12 * 10


@pytest.mark.parametrize("bc", [(ai.PERIODIC,) * 6, (ai.OUTFLOW,) * 6,
                                (ai.PERIODIC, ai.PERIODIC, ai.OUTFLOW, ai.OUTFLOW, ai.PERIODIC, ai.PERIODIC)])
def test_faces_read_in_place_map_to_the_right_cells(checker, bc):
    (n,) = ghost(checker, 32, 2, bc, ai.nested_cubes(32, (32, 32), 11, pmin=8, pmax=16), mode="faces")
    assert n > 0
    pb = ai.sedov_amr()
    (n,) = ghost(checker, pb.base_n[0], pb.max_level, bc, pb.patches, mode="faces")
    assert n > 0


@pytest.mark.parametrize("bc", [(ai.PERIODIC,) * 6, (ai.OUTFLOW,) * 6])
def test_flattened_lists_address_the_same_cells(checker, bc):
    (n,) = ghost(checker, 32, 2, bc, ai.nested_cubes(32, (32, 32), 11, pmin=8, pmax=16), mode="flat")
    assert n > 0
    base = 32   # prolongation boxes on odd rectangles of a partly covered face
    rng = np.random.Generator(np.random.PCG64(7))
    patches = ai.box_patches(0, (0, 0, 0), (base,) * 3, rng, 8, 16)
    patches += ai.box_patches(1, (16, 16, 16), (40, 40, 40), rng, 8, 16)
    patches += ai.box_patches(1, (40, 16, 16), (48, 40, 36), rng, 8, 12)
    (n,) = ghost(checker, base, 1, bc, patches, mode="flat")
    assert n > 0


def host_cluster(checker, base, max_level, bc, patches, flags, buffer, block, max_patch, min_level):
    lines = [f"cluster {base} {base} {base} {max_level} {' '.join(map(str, bc))} {buffer} {block} {max_patch} "
             f"{min_level}", listing(patches)]
    for f in flags:
        lines.append("0" if f is None else "1 " + " ".join(map(str, f.astype(np.uint8).ravel())))
    r = subprocess.run([checker], input="\n".join(lines) + "\n", capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    rows = r.stdout.split("\n")[1:]
    return [tuple(map(int, x.split())) for x in rows if x.strip()]


@pytest.mark.parametrize("bc", [(ai.PERIODIC,) * 6, (ai.OUTFLOW,) * 6])
@pytest.mark.parametrize("buffer,block,max_patch,min_level", [(2, 4, 32, 0), (1, 2, 16, 0), (4, 8, 32, 1)])
def test_host_clustering_matches_the_oracle(checker, bc, buffer, block, max_patch, min_level):
    from oracle import regrid as rg
    patches = ai.nested_cubes(16, (16, 16), 41, pmin=8, pmax=16)
    rng = np.random.Generator(np.random.PCG64(97 + buffer + block))
    flags = []
    for p in patches:
        if p.level < min_level or p.level >= 2:
            flags.append(None)
            continue
        f = np.zeros((p.n[2], p.n[1], p.n[0]), dtype=bool)
        # a few seeded blobs of flagged cells
        for _ in range(2):
            c = [int(rng.integers(0, p.n[d])) for d in range(3)]
            r = int(rng.integers(1, 4))
            f[max(0, c[2] - r):c[2] + r, max(0, c[1] - r):c[1] + r, max(0, c[0] - r):c[0] + r] = True
        flags.append(f)
    ours = host_cluster(checker, 16, 2, bc, patches, flags, buffer, block, max_patch, min_level)
    ref = rg.cluster(patches, flags, (16,) * 3, bc, 2, buffer=buffer, block=block, max_patch=max_patch,
                     min_level=min_level)
    assert ours == [(q.level, *q.lo, *q.n) for q in ref]
    assert any(q[0] >= 1 for q in ours)
