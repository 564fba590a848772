"""Autotuner for the batched ABFT Cholesky: picks the block size (32 or 64)
per size bucket and dtype by timing the persistent kernel on synthetic
matrices of that bucket, and caches the choice in a JSON file keyed by the
GPU name.  (Host-side orchestration only; the timed work runs in libabft.)"""
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
    sizes = r.integers(lo, hi + 1, count)
    offs = np.concatenate([[0], np.cumsum(sizes.astype(np.int64) ** 2)[:-1]])
    buf = torch.empty(int((sizes.astype(np.int64) ** 2).sum()), dtype=dtype, device=device)
    for i, n in enumerate(sizes):
        M = torch.randn(int(n), int(n), dtype=torch.float64, device=device)
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
