"""Batched ABFT Cholesky (abft_potrf_batched, one persistent launch): every
sampled matrix equals the single-matrix oracle with the same block size, the
injected faults (one per 64 matrices) are located and corrected, FP32
matches the FP64 factor to FP32 accuracy, and the CUDA-graph replay gives
the same results as the eager launch."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import tune
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def make_batch(count, dtype, seed0=100000, lo=32, hi=512, nb=64, fault_every=64, fseed=5):
    sizes = W.batched_sizes(count, lo, hi, seed=1005 + count)
    mats = [W.spd_mmt(int(n), seed0 + i) for i, n in enumerate(sizes)]
    offs = np.concatenate([[0], np.cumsum(sizes.astype(np.int64) ** 2)[:-1]])
    flat = np.concatenate([m.reshape(-1) for m in mats])
    buf = torch.from_numpy(flat).to(DEV).to(dtype)
    r = W.rng(fseed)
    faults = {}
    for q in range(0, count, fault_every):
        i = q + int(r.integers(0, min(fault_every, count - q)))
        n = int(sizes[i])
        b = nb(n) if callable(nb) else nb
        if n <= b:
            continue
        row = int(r.integers(b, n)); col = int(r.integers(b, n))
        if col // b > row // b:
            row, col = col, row
        faults[i] = (0, abft.F_MEMORY, row, col, 1e3)
    return abft.Batch(buf, sizes, offs, nb, faults), mats, faults


@pytest.mark.parametrize("nb", [32, 64])
def test_batched_f64_vs_oracle(nb):
    batch, mats, faults = make_batch(256, torch.float64, nb=nb, fault_every=16)
    abft.potrf_batched(batch)
    torch.cuda.synchronize()
    st = batch.statuses()
    for i in list(range(0, 256, 9)) + list(faults):
        L = batch.matrix(i).cpu().numpy()
        Lo, info, rep = oracle.potrf(mats[i], nb, oracle.FULL,
                                     [(f[0], f[1], f[2], f[3], f[4]) for f in [faults[i]]] if i in faults else [])
        assert st[i]["info"] == 0 and info == 0
        assert np.abs(np.tril(L) - np.tril(Lo)).max() <= 1e-12 * max(1.0, np.abs(Lo).max())
        assert np.array_equal(np.triu(L, 1), np.triu(mats[i], 1))      # upper triangle untouched
        assert st[i]["corrected"] == rep["corrected"] and st[i]["detected"] == rep["detected"]
        if i in faults:
            f = faults[i]
            assert (st[i]["ev_step"], st[i]["ev_kind"], st[i]["ev_row"], st[i]["ev_col"]) == (0, 0, f[2], f[3])


def test_batched_f32():
    batch, mats, faults = make_batch(200, torch.float32, nb=64, fault_every=20)
    abft.potrf_batched(batch)
    torch.cuda.synchronize()
    st = batch.statuses()
    for i in range(200):
        assert st[i]["info"] == 0
        if i in faults:
            assert st[i]["corrected"] == 1 and (st[i]["ev_row"], st[i]["ev_col"]) == faults[i][2:4]
        else:
            assert st[i]["detected"] == 0
    for i in range(0, 200, 13):
        L = np.tril(batch.matrix(i).cpu().numpy().astype(np.float64))
        Lf = np.linalg.cholesky(mats[i])
        assert np.abs(L - Lf).max() <= 64 * 2.0 ** -24 * np.abs(Lf).max()


def test_batched_graph_replay_and_tuner(tmp_path):
    table = tune.tune(torch.float64, DEV, per_bucket=32, cache=str(tmp_path / "tune.json"))
    assert set(table) == {0, 1, 2} and all(v in (32, 64) for v in table.values())
    nbf = tune.chooser(table)
    batch, mats, faults = make_batch(300, torch.float64, nb=nbf, fault_every=64)
    buf0 = batch.buf.clone()
    abft.potrf_batched(batch)
    ref = batch.buf.clone()
    for _ in range(2):
        batch.buf.copy_(buf0)
        abft.potrf_batched(batch, use_graph=True)
        torch.cuda.synchronize()
        assert torch.equal(batch.buf, ref)
    abft.lib().abft_batched_graph_reset()


def test_batched_ctas_per_sm_tuner(tmp_path):
    """The launch-level knob: the tuner picks a CTA count in range, and the
    factors and statuses do not depend on it (one CTA per matrix), eager or
    replayed from a graph keyed by the grid."""
    cache = str(tmp_path / "tune.json")
    for dt in (torch.float64, torch.float32):
        c = tune.tune_launch(dt, DEV, table={0: 64, 1: 64, 2: 64}, count=160, cache=cache, reps=1)
        assert 1 <= c <= tune.MAX_CTAS_PER_SM["f64" if dt == torch.float64 else "f32"]
        assert tune.tune_launch(dt, DEV, count=160, cache=cache) == c          # cached
    batch, mats, faults = make_batch(200, torch.float32, nb=64, fault_every=20)
    buf0 = batch.buf.clone()
    abft.potrf_batched(batch)
    ref, ref_st = batch.buf.clone(), batch.status.clone()
    try:
        for c in (1, 3):
            assert abft.set_batched_ctas_per_sm(c) in (0, 1)
            for graph in (False, True):
                batch.buf.copy_(buf0)
                batch.status.zero_()
                abft.potrf_batched(batch, use_graph=graph)
                torch.cuda.synchronize()
                assert torch.equal(batch.buf, ref) and torch.equal(batch.status, ref_st)
    finally:
        abft.set_batched_ctas_per_sm(0)
        abft.lib().abft_batched_graph_reset()


def test_batched_config_4096():
    """The batched configuration: 4096 matrices, n uniform in [32, 512], one
    fault per 64 matrices, FP64, one persistent launch."""
    batch, mats, faults = make_batch(4096, torch.float64, nb=64, fault_every=64)
    abft.potrf_batched(batch, use_graph=True)
    torch.cuda.synchronize()
    st = batch.statuses()
    assert all(s["info"] == 0 for s in st)
    for i, f in faults.items():
        assert st[i]["corrected"] == 1 and (st[i]["ev_row"], st[i]["ev_col"]) == (f[2], f[3])
    assert sum(s["detected"] for s in st) == len(faults)
    for i in range(0, 4096, 257):
        Lo, _, _ = oracle.potrf(mats[i], 64, oracle.FULL)
        assert np.abs(np.tril(batch.matrix(i).cpu().numpy()) - np.tril(Lo)).max() <= 1e-12
    abft.lib().abft_batched_graph_reset()


def test_batched_graph_key_holds_tau_scale():
    """A replayed graph must use the threshold of the call that replays it: the
    same buffers with a threshold scale large enough to hide the injected
    fault report nothing, and the original scale finds it again."""
    batch, mats, faults = make_batch(64, torch.float64, nb=64, fault_every=16)
    assert faults
    buf0 = batch.buf.clone()
    ws = abft.Workspace()
    abft.potrf_batched(batch, use_graph=True, workspace=ws)
    torch.cuda.synchronize()
    assert sum(s["detected"] for s in batch.statuses()) == len(faults)
    for scale, expect in ((1e30, 0), (1.0, len(faults))):
        batch.buf.copy_(buf0)
        batch.status.zero_()
        abft.potrf_batched(batch, tau_scale=scale, use_graph=True, workspace=ws)
        torch.cuda.synchronize()
        assert sum(s["detected"] for s in batch.statuses()) == expect
    abft.lib().abft_batched_graph_reset()


def test_sharded_batch_equals_one_launch():
    """The multi-GPU split run shard after shard on one GPU: each share of
    abft_batched_partition factored by its own launch gives the same factors
    and, gathered by matrix index, the same statuses as one launch over all."""
    from paper_2301_03166_b300 import shard
    count, G = 300, 3
    batch, mats, faults = make_batch(count, torch.float64, nb=64, fault_every=20)
    abft.potrf_batched(batch)
    torch.cuda.synchronize()
    ref = batch.status.cpu().numpy()
    owner, load = shard.partition(batch.sizes, G)
    assert load.max() / load.min() < 1.05
    parts_ids, parts_st = [], []
    for g in range(G):
        ids = shard.shard_ids(owner, g)
        sz = [batch.sizes[i] for i in ids]
        offs = np.concatenate([[0], np.cumsum(np.asarray(sz, dtype=np.int64) ** 2)[:-1]])
        buf = torch.cat([torch.from_numpy(mats[i].reshape(-1)) for i in ids]).to(DEV)
        loc = {int(i): k for k, i in enumerate(ids)}
        sb = abft.Batch(buf, sz, offs, 64, {loc[i]: f for i, f in faults.items() if i in loc})
        abft.potrf_batched(sb)
        torch.cuda.synchronize()
        for k, i in enumerate(ids):
            assert torch.equal(sb.matrix(k), batch.matrix(int(i)))
        parts_ids.append(ids)
        parts_st.append(sb.status.cpu().numpy())
    full = shard.gather_statuses(np.concatenate(parts_ids), np.concatenate(parts_st), count)
    assert np.array_equal(full, ref)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nb", [32, 64])
@pytest.mark.parametrize("mode", [abft.NONE, abft.FULL])
def test_batched_edge_orders_and_failure(dtype, nb, mode):
    """Orders below, at and just past the block sizes (single-column PD
    phases, odd last blocks, ragged edge tiles), FP64 against the oracle and
    FP32 against LAPACK, and one indefinite matrix in the middle of the batch:
    its info is the 1-based column of the first non-positive pivot and the
    matrices around it are unaffected."""
    sizes = np.array([1, 2, 3, 7, 31, 32, 33, 63, 64, 65, 97, 127, 129, 200])
    bad = 9                                   # n = 65: pivot 40 made negative
    mats = [W.spd_mmt(int(n), 7000 + i) for i, n in enumerate(sizes)]
    mats[bad] = mats[bad].copy()
    mats[bad][39, 39] = -10.0
    offs = np.concatenate([[0], np.cumsum(sizes.astype(np.int64) ** 2)[:-1]])
    buf = torch.from_numpy(np.concatenate([m.reshape(-1) for m in mats])).to(DEV).to(dtype)
    batch = abft.Batch(buf, sizes, offs, nb)
    abft.potrf_batched(batch, mode=mode)
    torch.cuda.synchronize()
    st = batch.statuses()
    for i, n in enumerate(sizes):
        if i == bad:
            assert st[i]["info"] == 40
            continue
        assert st[i]["info"] == 0 and st[i]["detected"] == 0, (i, st[i])
        L = np.tril(batch.matrix(i).cpu().numpy().astype(np.float64))
        if dtype == torch.float64:
            Lo, info, _ = oracle.potrf(mats[i], nb, oracle.FULL if mode == abft.FULL else oracle.NONE)
            assert info == 0
            assert np.abs(L - np.tril(Lo)).max() <= 1e-12 * max(1.0, np.abs(Lo).max())
        else:
            Lf = np.linalg.cholesky(mats[i])
            assert np.abs(L - Lf).max() <= 64 * 2.0 ** -24 * np.abs(Lf).max()
        # the strict upper triangle is left as it was
        U = np.triu(batch.matrix(i).cpu().numpy().astype(np.float64), 1)
        assert np.array_equal(U, np.triu(mats[i].astype(np.float32 if dtype == torch.float32 else np.float64).astype(np.float64), 1))
