"""Autotuner for the batched ABFT Cholesky.  Two knobs, both timed on the
persistent kernel with synthetic SPD matrices and cached in a JSON file keyed
by the GPU name:
  * tune(): the block size (32 or 64) per size bucket and dtype, a
    per-matrix choice (item.nb);
  * tune_launch(): the persistent CTAs per SM of the launch (1 up to the most
    that fit: FP64 2, FP32 4), timed on the whole size mix with the tuned
    block sizes, a per-launch choice (abft_batched_set_ctas_per_sm).
The kernel's threads per CTA (256) and its one CTA per matrix are fixed by its
design.  (Host-side orchestration only; the timed work runs in libabft.)"""
import json
import os

import numpy as np
import torch

from . import abft

BUCKETS = ((32, 127), (128, 255), (256, 512))
CANDIDATES = (32, 64)


def _bucket(n):
    for i, (lo, hi) in enumerate(BUCKETS):
        if lo <= n <= hi:
            return i
    return len(BUCKETS) - 1


def _sample(lo, hi, count, dtype, device, seed):
    r = np.random.Generator(np.random.PCG64(seed))
    return _spd_batch(r.integers(lo, hi + 1, count), dtype, device, seed)


def _spd_batch(sizes, dtype, device, seed):
    offs = np.concatenate([[0], np.cumsum(sizes.astype(np.int64) ** 2)[:-1]])
    buf = torch.empty(int((sizes.astype(np.int64) ** 2).sum()), dtype=dtype, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    for i, n in enumerate(sizes):
        M = torch.randn(int(n), int(n), generator=g, dtype=torch.float64, device=device)
        A = M @ M.T / n + torch.eye(int(n), dtype=torch.float64, device=device)
        buf[offs[i]:offs[i] + n * n] = A.reshape(-1).to(dtype)
    return buf, sizes, offs


def tune(dtype=torch.float64, device="cuda", per_bucket=None, cache=None, reps=3):
    """Returns {bucket_index: nb} for `dtype`; reads / updates `cache` (a JSON path)."""
    name = torch.cuda.get_device_name(device)
    key = "f64" if dtype == torch.float64 else "f32"
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as fh:
            table = json.load(fh)
    if name in table and key in table[name]:
        return {int(k): v for k, v in table[name][key].items()}
    per_bucket = per_bucket or 2 * torch.cuda.get_device_properties(device).multi_processor_count
    best = {}
    ws = abft.Workspace()
    for b, (lo, hi) in enumerate(BUCKETS):
        buf0, sizes, offs = _sample(lo, hi, per_bucket, dtype, device, seed=77 + b)
        times = {}
        for nb in CANDIDATES:
            buf = buf0.clone()
            batch = abft.Batch(buf, sizes, offs, nb)
            abft.potrf_batched(batch, workspace=ws)
            torch.cuda.synchronize(device)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                buf.copy_(buf0)
                abft.potrf_batched(batch, workspace=ws)
            e1.record()
            torch.cuda.synchronize(device)
            times[nb] = e0.elapsed_time(e1)
        best[b] = min(times, key=times.get)
    if cache:
        table.setdefault(name, {})[key] = {str(k): v for k, v in best.items()}
        with open(cache, "w") as fh:
            json.dump(table, fh, indent=1)
    return best


def chooser(table):
    """nb for a matrix of order n from a tuned {bucket: nb} table."""
    return lambda n: table[_bucket(n)]


MAX_CTAS_PER_SM = {"f64": 2, "f32": 4}


def tune_launch(dtype=torch.float64, device="cuda", table=None, sizes=None, count=4096, cache=None,
                reps=3, lo=32, hi=512):
    """Returns the persistent CTAs per SM (1 .. MAX_CTAS_PER_SM) that factor a
    batch fastest, block sizes from `table` ({bucket: nb}, tune() when None).
    The batch is the size mix to be run: `sizes` (the orders of its
    matrices), else `count` orders uniform in [lo, hi].  The choice depends
    on how many matrices each CTA gets (with about one each, fewer CTAs per SM
    finish the largest sooner), so tune with the batch's own count.  Reads /
    updates `cache` (keyed by the GPU and the batch's count); the library's
    setting is restored afterwards."""
    name = torch.cuda.get_device_name(device)
    if sizes is not None:
        count = len(sizes)
    key = ("f64" if dtype == torch.float64 else "f32") + "_ctas_per_sm_" + str(count)
    stored = {}
    if cache and os.path.exists(cache):
        with open(cache) as fh:
            stored = json.load(fh)
    if name in stored and key in stored[name]:
        return int(stored[name][key])
    table = table or tune(dtype, device, cache=cache, reps=reps)
    nbf = chooser(table)
    if sizes is None:
        buf0, sizes, offs = _sample(lo, hi, count, dtype, device, seed=91)
    else:
        sizes = np.asarray(sizes)
        buf0, _, offs = _spd_batch(sizes, dtype, device, seed=91)
    ws = abft.Workspace()
    times = {}
    prev = abft.set_batched_ctas_per_sm(0)
    try:
        for c in range(1, MAX_CTAS_PER_SM[key[:3]] + 1):
            abft.set_batched_ctas_per_sm(c)
            buf = buf0.clone()
            batch = abft.Batch(buf, sizes, offs, nbf)
            abft.potrf_batched(batch, workspace=ws)
            torch.cuda.synchronize(device)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                buf.copy_(buf0)
                abft.potrf_batched(batch, workspace=ws)
            e1.record()
            torch.cuda.synchronize(device)
            times[c] = e0.elapsed_time(e1)
    finally:
        abft.set_batched_ctas_per_sm(prev)
    best = min(times, key=times.get)
    if cache:
        stored = {}
        if os.path.exists(cache):
            with open(cache) as fh:
                stored = json.load(fh)
        stored.setdefault(name, {})[key] = best
        with open(cache, "w") as fh:
            json.dump(stored, fh, indent=1)
    return best
