"""Host-side partition of a hierarchy over ranks (the split a multi-GPU run
would use; runs here have one GPU): every patch gets one owner, each level's
patches form one contiguous Morton range per rank, the cell counts per rank are
balanced to within one patch, and two gloo ranks computing it independently
own disjoint sets that cover the hierarchy."""
import os
import sys

import numpy as np
import pytest

import amr_inputs as ai
from paper_0910_5547_gb300 import native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _morton(p, L):
    c = [((2 * p.lo[d] + p.n[d]) << (L - p.level)) >> 1 for d in range(3)]
    key = 0
    for b in range(21):
        for d in range(3):
            key |= ((c[d] >> b) & 1) << (3 * b + d)
    return key


@pytest.mark.parametrize("nranks", [1, 2, 3, 8])
def test_partition_is_contiguous_and_balanced_per_level(nranks):
    pb = ai.sedov_amr(base=32, sides=(48, 56, 56))
    cfg = N.amr_default_config(base_n=pb.base_n, max_level=pb.max_level, bc=pb.bc)
    own = N.amr_partition_patches(cfg, pb.patches, nranks)
    assert own.shape == (len(pb.patches),) and own.min() >= 0 and own.max() < nranks
    L = max(p.level for p in pb.patches)
    for l in range(L + 1):
        idx = [i for i, p in enumerate(pb.patches) if p.level == l]
        order = sorted(idx, key=lambda i: _morton(pb.patches[i], L))
        seq = [int(own[i]) for i in order]
        assert seq == sorted(seq)                    # one contiguous range per rank
        w = np.array([pb.patches[i].ncell for i in idx])
        per = np.bincount([own[i] for i in idx], weights=[pb.patches[i].ncell for i in idx], minlength=nranks)
        assert per.max() <= w.sum() / nranks + w.max()
    if nranks == 1:
        assert not own.any()


def test_partition_rejects_bad_arguments():
    cfg = N.amr_default_config()
    with pytest.raises(N.AmrError):
        N.amr_partition_patches(cfg, [ai.Patch(0, (0, 0, 0), (32, 32, 32))], 0)


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import amr_inputs as ai2
    from paper_0910_5547_gb300 import native as N2
    pb = ai2.sedov_amr(base=32, sides=(48, 56, 56))
    cfg = N2.amr_default_config(base_n=pb.base_n, max_level=pb.max_level, bc=pb.bc)
    own = N2.amr_partition_patches(cfg, pb.patches, world)
    mine = torch.tensor((own == rank).astype(np.int64))
    gathered = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(gathered, mine)
    bound = sum(max(p.ncell for p in pb.patches if p.level == l) for l in range(1 + max(p.level for p in pb.patches)))
    q.put((rank, torch.stack(gathered).sum(0).tolist(), int(sum(p.ncell for p, o in zip(pb.patches, own) if o == rank)),
           bound))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_own_disjoint_sets_covering_the_hierarchy():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29800 + os.getpid() % 150
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert all(c == 1 for c in res[0][1])            # every patch owned exactly once
    cells = [r[2] for r in res]
    # each level is balanced to within one of its patches, so the totals to within
    # the sum over levels of the largest patch
    assert abs(cells[0] - cells[1]) <= res[0][3]
