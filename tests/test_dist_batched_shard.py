"""The batched form's multi-GPU split (abft_batched_partition + host gather of
the per-matrix statuses) as two gloo ranks on the CPU.  Each rank takes the
share the partition gives it and produces the status rows of its matrices
(here from the oracle, standing in for the GPU launch); rank 0 gathers them.
Checked: every matrix lands on exactly one rank, the shares are balanced,
and the gathered table equals a single-process run over all matrices."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COUNT = 48


def _batch():
    sys.path.insert(0, ROOT)
    from paper_2301_03166_b300 import workloads as W
    sizes = W.batched_sizes(COUNT, 8, 72, seed=77)
    faults = {}
    r = W.rng(78)
    for q in range(0, COUNT, 8):
        i = q + int(r.integers(0, 8))
        n = int(sizes[i])
        if n > 16:
            row, col = int(r.integers(16, n)), int(r.integers(16, n))
            if col // 16 > row // 16:
                row, col = col, row
            faults[i] = (0, 0, row, col, 1e3)
    return sizes, faults


def _status_rows(ids, sizes, faults):
    """(info, detected, corrected, uncorrectable, ev_step, ev_kind, ev_row,
    ev_col) per matrix, as the batched kernel reports them."""
    import oracle
    from paper_2301_03166_b300 import workloads as W
    rows = []
    for i in ids:
        A = W.spd_mmt(int(sizes[i]), seed=100000 + int(i))
        fl = [faults[i]] if i in faults else []
        _, info, rep = oracle.potrf(A, 16, oracle.FULL, fl)
        e = rep["loc"][0] if rep["loc"] else (-1, -1, -1, -1, 0.0)
        rows.append([info, rep["detected"], rep["corrected"], rep["uncorrectable"],
                     e[0], e[1], e[2], e[3]])
    return np.array(rows, dtype=np.int32).reshape(len(ids), 8)


def _rank_main(rank, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": "2", "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2301_03166_b300 import shard
    dist.init_process_group("gloo")
    sizes, faults = _batch()
    owner, load = shard.partition(sizes, 2)
    mine = shard.shard_ids(owner, rank)
    full = shard.gather_statuses(mine, _status_rows(mine, sizes, faults), COUNT)
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), full)
    np.save(os.path.join(out_dir, f"ids{rank}.npy"), mine)
    dist.destroy_process_group()


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_properties():
    sys.path.insert(0, ROOT)
    from paper_2301_03166_b300 import shard
    from paper_2301_03166_b300 import workloads as W
    sizes = W.batched_sizes(4096, 32, 512, seed=1005)
    work = sizes.astype(np.float64) ** 3 / 3
    for G in (1, 2, 3, 4, 8):
        owner, load = shard.partition(sizes, G)
        assert owner.min() >= 0 and owner.max() < G
        assert np.allclose([work[owner == g].sum() for g in range(G)], load, rtol=1e-12)
        # greedy LPT: no share exceeds another by more than one matrix's work
        assert load.max() - load.min() <= work.max()
        assert load.max() / load.min() < 1.001
        assert np.array_equal(owner, shard.partition(sizes, G)[0])   # deterministic
    # by hand: orders 3 3 2 2 2 have works 9 9 8/3 8/3 8/3; largest first, each
    # to the lighter GPU, ties to GPU 0: 9 | 9, then 0, 1, 0
    owner, load = shard.partition(np.array([3, 3, 2, 2, 2]), 2)
    assert list(owner) == [0, 1, 0, 1, 0] and list(load) == [9 + 16 / 3, 9 + 8 / 3]


@pytest.mark.timeout(300)
def test_two_rank_shard_gather_gloo(tmp_path):
    mp.spawn(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=2, join=True)
    ids = [np.load(tmp_path / f"ids{r}.npy") for r in range(2)]
    allids = np.sort(np.concatenate(ids))
    assert np.array_equal(allids, np.arange(COUNT))          # every matrix exactly once
    assert len(ids[0]) > 0 and len(ids[1]) > 0
    sizes, faults = _batch()
    gathered = np.load(tmp_path / "gathered.npy")
    single = _status_rows(np.arange(COUNT), sizes, faults)
    assert np.array_equal(gathered, single)
    assert gathered[:, 2].sum() == len(faults) and np.all(gathered[:, 0] == 0)
