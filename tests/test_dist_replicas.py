"""The N > 1 path of bench.py on CPU: two ranks over gloo (127.0.0.1).  A
single factorization is not sharded ("replicas only"), so the multi-rank
logic is the host side: rank setup from the torchrun environment, the
barrier, the maximum of the per-rank time over the ranks, and a single JSON
line from rank 0 (the reference arm, on a small oracle sample)."""
import importlib.util
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load_bench():
    saved = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec = importlib.util.spec_from_file_location("bench_rank", os.path.join(ROOT, "bench.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
    finally:
        sys.argv = saved
    return mod


def _rank_main(rank, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": "2", "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    bench = _load_bench()
    ws, r, local = bench.dist_setup()
    bench.barrier(ws)
    m = bench.max_over_ranks(10.0 * (rank + 1), ws, "cpu")
    bench.CPU_SAMPLE_N = 96   # a small oracle sample: the check is the rank logic
    saved = sys.argv
    sys.argv = ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    try:
        args = bench.parse()
    finally:
        sys.argv = saved
    out_path = os.path.join(out_dir, f"rank{rank}.txt")
    with open(out_path, "w") as f:
        old = sys.stdout
        sys.stdout = f
        try:
            bench.run_reference(args, ws, r)
        finally:
            sys.stdout = old
    with open(os.path.join(out_dir, f"meta{rank}.json"), "w") as f:
        json.dump({"ws": ws, "rank": r, "local": local, "max": m}, f)
    import torch.distributed as dist
    dist.destroy_process_group()


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.timeout(300)
def test_two_rank_replicas_gloo(tmp_path):
    mp.spawn(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=2, join=True)
    metas = [json.load(open(tmp_path / f"meta{r}.json")) for r in range(2)]
    assert [(m["ws"], m["rank"], m["local"]) for m in metas] == [(2, 0, 0), (2, 1, 1)]
    assert all(m["max"] == 20.0 for m in metas)          # max over ranks, on every rank
    out0 = (tmp_path / "rank0.txt").read_text().strip().splitlines()
    out1 = (tmp_path / "rank1.txt").read_text().strip()
    assert out1 == ""                                   # only rank 0 prints
    line = json.loads(out0[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
