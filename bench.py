#!/usr/bin/env python
"""Benchmark: ABFT Cholesky on one B300 (per rank), one JSON line on stdout.

A step is one FP64 ABFT-protected blocked Cholesky factorization
(full checksums, faults injected at 1 per 10 steps) of the n = 16384,
block 256 matrix A = M M^T / n + I (M iid N(0, 1), seeded), resident in HBM:
the working copy is reset from a pristine copy and factored; the report
(events, counters) is read back.  The matrix (2.1 GB) is larger than L2, so
no separate L2 flush is needed between steps.

Besides the contract's keys, the line reports the context figures:
- `energy`: board joules per factorization, from NVML's energy counter
  (read only);
- `cpu_lapack`: LAPACK dpotrf on all host cores on the same matrix,
  without checksums, a stronger CPU baseline than the oracle;
- sections for the FP64-accurate and 16-bit forms, the look-ahead, LU / QR
  and the batched factorization.

--impl reference times the CPU oracle (plain C, one core) on a bounded
sample of the same workload instead (rank 0 only).
"""
import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

WORKLOAD = "FP64 ABFT Cholesky (full checksums, faults 1 per 10 steps), n=16384, block 256"
METRIC = "ABFT Cholesky TFLOP/s & % peak at n=16384: FP64 vs BF16+IR at 1e-12 residual"
CPU_SAMPLE_N = 4096   # oracle sample: one full ABFT Cholesky at this order, block 256 (~13 s)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--nb", type=int, default=256)
    p.add_argument("--no-overhead", action="store_true", help="skip the NONE-mode overhead run")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-mixed", action="store_true", help="skip the BF16/FP16 + IR solve")
    p.add_argument("--no-adjoint", action="store_true",
                   help="skip the GP forward + backward timings (n = 4096, 16384)")
    p.add_argument("--no-lu-qr", action="store_true", help="skip the LU and QR timings")
    p.add_argument("--no-batched", action="store_true", help="skip the batched timings")
    p.add_argument("--no-lookahead", action="store_true",
                   help="skip the look-ahead section (BF16 factorization with and without "
                        "look-ahead, per-iteration time prediction as a self-check)")
    p.add_argument("--no-emulated", action="store_true",
                   help="skip the FP64-accurate factorization with the BF16 tensor-core update")
    p.add_argument("--no-conditioned", action="store_true",
                   help="skip the conditioned solves: A = Q diag(sigma) Q^T with kappa 1e2, 1e6, "
                        "1e10, n = --cond-n, block 512, 16 right-hand sides; GMRES-IR on the "
                        "BF16 / FP16 factor and refinement on the FP64-accurate factor, against "
                        "the FP64 form")
    p.add_argument("--cond-n", type=int, default=32768)
    p.add_argument("--campaign", action="store_true",
                   help="add the fault campaign: share of correct factorizations and time per "
                        "factorization for no / single-side / full / adaptive checksums")
    p.add_argument("--campaign-trials", type=int, default=60)
    p.add_argument("--profile-case", default=None,
                   choices=["fp64", "fp64-emu", "mixed-bf16", "mixed-f16", "potrs-f32", "lu",
                            "lu-emu", "qr", "qr-emu", "batched-f64", "batched-f32", "fp64-pipes",
                            "adjoint", "adjoint-emu"],
                   help="run one case once after one warm-up, print nothing (for ncu): the FP64 "
                        "ABFT Cholesky of the benchmark, a BF16 / FP16 solve with iterative "
                        "refinement, an FP32 two-sweep solve with the FP64 factor, or the ABFT "
                        "LU (FP64 / FP64-accurate update) or QR of the uniform matrix, or the GP "
                        "loss forward and backward (FP64 / FP64-accurate); at --n, --nb")
    return p.parse_args()


def chol_flops(n):
    return n ** 3 / 3.0


def tmu_flops(n, nb):
    """Algorithmic flops of the symmetric trailing updates of one factorization:
    step k updates the lower triangle of an m_k x m_k block with a rank-kb
    product, m_k (m_k + 1) kb flops (border and diagonal-block extras excluded)."""
    tot = 0.0
    for K0 in range(0, n, nb):
        kb = min(nb, n - K0)
        m = n - K0 - kb
        tot += m * (m + 1) * kb
    return tot


# ------------------------------------------------------------- energy
class BoardEnergy:
    """NVML's total-energy counter of the board this process runs on, read
    only (mJ since the driver loaded), for the context figure "board energy
    per factorization".  NVML is reached through pynvml or, where that module
    is missing, through the driver's libnvidia-ml by ctypes (the documented C
    entry points); the board is found by the CUDA device's PCI address, else
    its UUID.  Reads return None where NVML or the counter is unavailable."""

    def __init__(self, dev):
        self.h = None
        self.c = None
        try:
            p = torch.cuda.get_device_properties(dev)
            bus = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0".encode()
            uuid = f"GPU-{p.uuid}".encode()
        except Exception:
            return
        try:
            import pynvml
            self.nv = pynvml
            pynvml.nvmlInit()
            try:
                self.h = pynvml.nvmlDeviceGetHandleByPciBusId(bus)
            except Exception:
                self.h = pynvml.nvmlDeviceGetHandleByUUID(uuid)
            pynvml.nvmlDeviceGetTotalEnergyConsumption(self.h)
            return
        except Exception:
            self.h = None
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(h)) != 0:
                if lib.nvmlDeviceGetHandleByUUID(ctypes.c_char_p(uuid), ctypes.byref(h)) != 0:
                    return
            e = ctypes.c_ulonglong()
            if lib.nvmlDeviceGetTotalEnergyConsumption(h, ctypes.byref(e)) == 0:
                self.c = (lib, h)
        except Exception:
            self.c = None

    def read(self):
        try:
            if self.h is not None:
                return float(self.nv.nvmlDeviceGetTotalEnergyConsumption(self.h))
            if self.c is not None:
                e = ctypes.c_ulonglong()
                if self.c[0].nvmlDeviceGetTotalEnergyConsumption(self.c[1], ctypes.byref(e)) == 0:
                    return float(e.value)
        except Exception:
            pass
        return None

    @staticmethod
    def joules(e0, e1, calls):
        if e0 is None or e1 is None or e1 <= e0 or calls <= 0:
            return None
        return (e1 - e0) * 1e-3 / calls


# ------------------------------------------------------------- clocks
def board_id(dev):
    """The board behind CUDA device `dev` as nvidia-smi names it: its PCI bus
    id (nvidia-smi ignores CUDA_VISIBLE_DEVICES, so a CUDA index can name
    another board), else its UUID, else the CUDA index."""
    try:
        p = torch.cuda.get_device_properties(dev)
        return f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
    except Exception:
        pass
    try:
        return f"GPU-{torch.cuda.get_device_properties(dev).uuid}"
    except Exception:
        return str(dev)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons, watts = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            try:
                watts.append(float(parts[3]))
            except ValueError:
                pass
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_mean": statistics.mean(watts) if watts else None}


# ------------------------------------------------------------- helpers
def dgemm_peak(dev):
    """Measured FP64 peak: cuBLAS DGEMM (torch.matmul float64, 4096^3), best of 3."""
    a = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    b = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    torch.cuda.synchronize(dev)
    best = 1e30
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize(dev)
        best = min(best, e0.elapsed_time(e1))
    del a, b
    return 2 * 4096 ** 3 / (best * 1e-3) / 1e12


def kernel_source_hash():
    p = os.path.join(ROOT, "paper_2301_03166_b300", "csrc", "k_gemm_f64.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


# ncu-measured DRAM traffic of the FP64 TMU kernel in bytes per updated C
# element (dram__bytes_read.sum + dram__bytes_write.sum of the step-0 TMU at
# n = 4096 divided by its 7.86 M updated elements), valid only for the kernel
# source it was measured on; scaled to the benchmark's launches by the number
# of updated elements.
TMU_TRAFFIC = {"4155d564486da839": 83.312640e6 / 7864320}


def cpu_baseline(steps=1, warm=0):
    """The oracle as it stands (plain C, single thread) on one bounded sample:
    a full FP64 ABFT Cholesky at n = CPU_SAMPLE_N, block 256."""
    import oracle
    from paper_2301_03166_b300 import workloads as W
    n = CPU_SAMPLE_N
    A = W.spd_mmt(n, seed=1000 + n)
    faults = W.fault_schedule(n, 256, "cholesky", seed=2000 + n)
    times = []
    for i in range(warm + steps):
        t0 = time.perf_counter()
        oracle.potrf(A, 256, oracle.FULL, faults)
        t = time.perf_counter() - t0
        if i >= warm:
            times.append(t)
    return times, n


def lapack_baseline(A_host):
    """The stronger CPU baseline: LAPACK dpotrf (scipy's OpenBLAS, all host
    cores, no checksums) on the benchmark's matrix, once.  Returns
    (seconds, BLAS threads used, BLAS name)."""
    import scipy.linalg
    threads, name = os.cpu_count(), "LAPACK dpotrf"
    try:
        from threadpoolctl import threadpool_info
        info = [d for d in threadpool_info() if d.get("user_api") == "blas"]
        if info:
            threads = info[0].get("num_threads", threads)
            name = f"LAPACK dpotrf ({info[0].get('internal_api', 'blas')})"
    except Exception:
        pass
    a = np.array(A_host, order="F", copy=True)   # column-major: no copy inside LAPACK
    t0 = time.perf_counter()
    scipy.linalg.cholesky(a, lower=True, overwrite_a=True, check_finite=False)
    return time.perf_counter() - t0, threads, name


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws, dev):
    if ws == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------- arms
def run_reference(args, ws, rank):
    if rank != 0:
        return
    times, n = cpu_baseline(steps=args.steps, warm=args.warmup)
    t = sum(times) / len(times)
    v = chol_flops(n) / t / 1e12
    sample = (f"one full FP64 ABFT Cholesky (full checksums, faults 1 per 10 steps) at n={n}, "
              f"block 256, per step; TFLOP/s counted as n^3/3")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": args.n, "nb": args.nb, "mode": "full",
                   "cpu_sample_n": n},
        "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args, ws, rank, local):
    from paper_2301_03166_b300 import abft
    from paper_2301_03166_b300 import workloads as W
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n, nb = args.n, args.nb
    peak = dgemm_peak(dev)
    A0 = W.spd_mmt_torch(n, seed=1000 + n, device=dev)
    A = torch.empty_like(A0)
    faults = W.fault_schedule(n, nb, "cholesky", seed=2000 + n)
    wsp = abft.Workspace()
    expected = sorted((f[0], 0, f[2], f[3]) for f in faults)

    def step(mode=abft.FULL, fl=faults):
        A.copy_(A0)
        rc, rep = abft.potrf(A, nb, mode, faults=fl, workspace=wsp)
        return rc, rep

    for _ in range(args.warmup):
        rc, rep = step()
    assert rc == 0, f"potrf returned {rc}"
    events_ok = [(e[0], e[1], e[2], e[3]) for e in rep["loc"]] == expected

    energy = BoardEnergy(dev)
    clocks = ClockSampler(board_id(local))
    clocks.start()
    abft.timing_enable(True)
    launches0 = abft.launch_count()
    barrier(ws)
    torch.cuda.synchronize(dev)
    en0 = energy.read()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        rc, rep = step()
    e1.record()
    torch.cuda.synchronize(dev)
    en1 = energy.read()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    launches = abft.launch_count() - launches0
    phases = abft.timing_read()
    abft.timing_enable(False)
    clk = clocks.stop()
    ms = max_over_ranks(ms, ws, dev)
    ms_step = ms / args.steps
    j_fact = BoardEnergy.joules(en0, en1, args.steps)
    src = ("NVML total-energy counter of this rank's board over the timed region, divided "
           "by the steps (read only; context)")
    if j_fact is None and clk.get("power_w_mean"):
        # no energy counter: the mean of the board power samples taken during
        # the timed region, times the time per factorization
        j_fact = clk["power_w_mean"] * ms_step * 1e-3
        src = ("mean board power (nvidia-smi power.draw, 200 ms samples over the timed "
               "region) x time per factorization (read only; context)")
    energy_line = {"board_joules_per_factorization": j_fact,
                   "board_watts_avg": (j_fact / (ms_step * 1e-3)) if j_fact else None,
                   "source": src}
    value = ws * chol_flops(n) / (ms_step * 1e-3) / 1e12

    # roofline of the dominant kernel (the FP64 trailing update)
    tmu_ms, tmu_launches = phases["tmu"]
    tmu_achieved = tmu_flops(n, nb) * args.steps / (tmu_ms * 1e-3) / 1e12 if tmu_ms > 0 else None
    bpe = TMU_TRAFFIC.get(kernel_source_hash())
    elems = 0
    for K0 in range(0, n, nb):
        q = (n - K0 - min(nb, n - K0) + nb - 1) // nb
        elems += q * (q + 1) // 2 * nb * nb
    traffic = bpe * elems if bpe else None
    roofline = {"bound": "alu", "kernel": "k_gemm_f64 (FP64 DFMA trailing update)",
                "achieved": tmu_achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (tmu_achieved / peak) if tmu_achieved else None,
                "peak_source": "measured cuBLAS DGEMM 4096^3 in this run (B300 has no FP64 tensor path; "
                               "DFMA microbenchmark 1.13 TFLOP/s)",
                "traffic": (traffic * args.steps / tmu_launches) if traffic else None,
                "traffic_note": "bytes per launch, scaled from an ncu capture at n=4096 by updated C elements",
                "tmu_share_of_step": tmu_ms / ms if ms > 0 else None,
                # event pairs of the timed steps; with look-ahead the PD and panel
                # solve run on the caller's stream beside the rest of the update
                # on a side stream, so these intervals overlap (their sum can
                # exceed the step) and PD / PU include waiting for SMs
                "phase_stream_ms_per_step_overlapping": {k: v[0] / args.steps
                                                         for k, v in phases.items()}}
    # a truthful breakdown: one more step with look-ahead off (every phase on
    # the caller's stream, one after another), its phases and its wall time
    prev_la = abft.set_lookahead(False)
    abft.timing_enable(True)
    torch.cuda.synchronize(dev)
    e0.record()
    step()
    e1.record()
    torch.cuda.synchronize(dev)
    seq = abft.timing_read()
    abft.timing_enable(False)
    abft.set_lookahead(prev_la)
    roofline["phase_ms_sequential_step"] = {k: v[0] for k, v in seq.items()}
    roofline["sequential_step_ms"] = e0.elapsed_time(e1)
    roofline["tmu_share_of_sequential_step"] = seq["tmu"][0] / e0.elapsed_time(e1)

    overhead = None
    if not args.no_overhead:
        step(abft.NONE, ())
        torch.cuda.synchronize(dev)
        e0.record()
        for _ in range(args.steps):
            step(abft.NONE, ())
        e1.record()
        torch.cuda.synchronize(dev)
        ms_none = e0.elapsed_time(e1) / args.steps
        overhead = {"ms_full": ms_step, "ms_none": ms_none,
                    "abft_overhead_pct": 100.0 * (ms_step / ms_none - 1.0)}

    last_joules = [None]   # board energy per call of the last timed() (NVML, context)

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize(dev)
        j0 = energy.read()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        out = None
        for _ in range(steps):
            out = fn()
        t1.record()
        torch.cuda.synchronize(dev)
        last_joules[0] = BoardEnergy.joules(j0, energy.read(), steps)
        return t0.elapsed_time(t1) / steps, out

    emulated = None
    if not args.no_emulated:
        # FP64-accurate factorization with the trailing update on the BF16 tensor
        # cores (ABFT_F64_EMU): same matrix, faults and checksums as the step;
        # accuracy against the FP64 factor above and by a probe backward error
        # ||(L L^T - A) v|| / (||A|| ||v||) with a seeded random v (FP64 on the GPU).
        Lref = torch.tril(A).clone()
        def emu_step():
            A.copy_(A0)
            return abft.potrf(A, nb, abft.FULL, dtype=abft.F64_EMU, faults=faults, workspace=wsp)
        for _ in range(max(1, args.warmup)):
            rc_e, rep_e = emu_step()
        abft.timing_enable(True)
        torch.cuda.synchronize(dev)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(args.steps):
            rc_e, rep_e = emu_step()
        t1.record()
        torch.cuda.synchronize(dev)
        ph_e = abft.timing_read()
        abft.timing_enable(False)
        ms_e = t0.elapsed_time(t1) / args.steps
        Le = torch.tril(A)
        gv = torch.Generator(device=dev)
        gv.manual_seed(4242)
        v = torch.randn(n, 1, generator=gv, dtype=torch.float64, device=dev)
        Av = A0 @ v
        def probe(Lx):
            return float(torch.linalg.norm(Lx @ (Lx.T @ v) - Av) /
                         (torch.linalg.norm(A0, ord=float("inf")) * torch.linalg.norm(v)))
        emulated = {"ms": ms_e, "tflops": chol_flops(n) / (ms_e * 1e-3) / 1e12,
                    "pct_of_fp64_peak": 100 * chol_flops(n) / (ms_e * 1e-3) / 1e12 / peak,
                    "speedup_vs_fp64": ms_step / ms_e, "rc": rc_e,
                    "events_match_injected": [(e[0], e[1], e[2], e[3]) for e in rep_e["loc"]] == expected,
                    "probe_backward_err": probe(Le), "probe_backward_err_fp64": probe(Lref),
                    "max_rel_diff_vs_fp64_factor": float((Le - Lref).abs().max() / Lref.abs().max()),
                    # overlapping stream intervals (look-ahead on), as in the roofline
                    "phase_stream_ms_per_step_overlapping": {k: vv[0] / args.steps
                                                             for k, vv in ph_e.items()},
                    "tmu_tensor_tflops_equiv": tmu_flops(n, nb) / (ph_e["tmu"][0] / args.steps * 1e-3) / 1e12}
        del Lref, Le, v, Av

    mixed = None
    if not args.no_mixed:
        # time to solution of A X = B (16 right-hand sides) at a 1e-12 backward
        # error: FP64 form = FP64 ABFT potrf + FP64 potrs; mixed = BF16 / FP16
        # ABFT potrf + iterative refinement (posv_ir), same matrix and faults.
        B = torch.from_numpy(W.rhs(n, 16, seed=1003)).to(dev)
        Xb = torch.empty_like(B)
        Lbuf = torch.empty_like(A0)
        def fp64_solve():
            A.copy_(A0)
            abft.potrf(A, nb, abft.FULL, faults=faults, workspace=wsp)
            Xb.copy_(B)
            abft.potrs(A, Xb, nb, abft.F64)
            return None
        ms_fp64, _ = timed(fp64_solve, 1, 1)
        mixed = {"fp64_ms_to_solution": ms_fp64, "fp64_board_joules": last_joules[0]}
        amax_diag = float(A0.diagonal().max().item())
        small = [(f[0], f[1], f[2], f[3], 1e-2) for f in faults]   # the same places, delta 1e-2
        for name, dt in (("bf16", abft.MIXED_BF16), ("f16", abft.MIXED_F16)):
            def mixed_solve():
                return abft.posv_ir(A0, B, nb, dt, abft.FULL, tol=1e-12, maxit=100, faults=faults,
                                    L=Lbuf, X=Xb, workspace=wsp)
            ms_mix, res = timed(mixed_solve, max(1, args.steps), 1)
            rc_m, _, _, rep_m = res
            mixed[name] = {"ms_to_solution": ms_mix, "speedup_vs_fp64": ms_fp64 / ms_mix,
                           "tflops_equiv": chol_flops(n) / (ms_mix * 1e-3) / 1e12,
                           "ir_iters": rep_m["ir_iters"], "backward_err": rep_m["backward_err"],
                           "rc": rc_m, "faults_corrected": rep_m["corrected"],
                           "board_joules": last_joules[0],
                           # the trailing-tile detector: per-column thresholds
                           # tau_j = 4 gamma_g(2^-24) |c|_j + tau64 from the
                           # abs-checksums; an error above tau_max (1 + max_ratio)
                           # is flagged at every step and column
                           "detector": {
                               "max_ratio_clean": rep_m["max_ratio"], "tau_max": rep_m["tau"],
                               "smallest_detectable_delta": rep_m["tau"] * (1 + rep_m["max_ratio"]),
                               "scalar_fp32_tau_it_replaces": 8 * 2.0 ** -24 * n * nb * amax_diag}}
            # the same factorization with errors of 1e-2 (below the scalar bound it
            # replaces) at the same places: each located and corrected
            Lbuf.copy_(A0)
            rc_s, rep_s = abft.potrf(Lbuf, nb, abft.FULL, dtype=dt, faults=small, workspace=wsp)
            mixed[name]["detector"]["small_faults"] = {
                "delta": 1e-2, "injected": len(small), "corrected": rep_s["corrected"],
                "located_at_injected": [(e[0], e[2], e[3]) for e in rep_s["loc"]] ==
                sorted((f[0], f[2], f[3]) for f in small)}
        del Lbuf, Xb, B

    lookahead = None
    if not args.no_lookahead:
        # Look-ahead (Sec. 2.1, Fig. example-lu (b), on one GPU): the BF16 ABFT
        # factorization of the benchmark matrix with and without it, and, as a
        # self-check of the per-step costs it trades, the per-iteration time
        # prediction of Sec. 3.2.1 (last four iterations weighted 1/2, 1/4, 1/8,
        # 1/8, scaled by the operations' work ratios) against the measured
        # per-iteration times of PD, PU, TMU and verification.
        def bf16_factor():
            A.copy_(A0)
            return abft.potrf(A, nb, abft.FULL, dtype=abft.MIXED_BF16, faults=faults, workspace=wsp)
        lookahead = {}
        for on in (False, True):
            abft.set_lookahead(on)
            ms_la, _ = timed(bf16_factor, max(1, args.steps), 1)
            lookahead["ms_on" if on else "ms_off"] = ms_la
        lookahead["speedup"] = lookahead["ms_off"] / lookahead["ms_on"]
        abft.timing_enable(True)
        bf16_factor()
        torch.cuda.synchronize(dev)
        marks = abft.timing_marks()
        abft.timing_enable(False)
        nsteps = (n + nb - 1) // nb
        pred_err = {}
        for op in ("pd", "pu", "tmu", "verify"):
            T = np.zeros(nsteps)
            for ph, k, ms in marks:
                if ph == op and 0 <= k < nsteps:
                    T[k] += ms
            Wk = np.array([abft.chol_step_work(n, nb, op, k) for k in range(nsteps)])
            pr = abft.predict_step_times(T, Wk)
            sel = [k for k in range(4, nsteps) if Wk[k] > 0 and T[k] > 0 and np.isfinite(pr[k])]
            rel = np.abs(pr[sel] - T[sel]) / T[sel]
            pred_err[op] = {"mean_rel_err": float(rel.mean()), "max_rel_err": float(rel.max()),
                            "steps": len(sel)}
        lookahead["prediction"] = pred_err

    conditioned = None
    if not args.no_conditioned:
        # Conditioned solves: A = Q diag(sigma) Q^T, sigma_i = kappa^(-i/(n-1)),
        # 16 N(0,1) right-hand sides, target backward error 1e-12, block 512.
        # At n = 32768 Q is a product of random butterfly networks (the QR of a
        # Gaussian matrix would take minutes on the FP64 pipe; same spectrum).
        # Time to solution of the FP64 form (FP64 ABFT potrf + potrs), of
        # GMRES-IR preconditioned by the BF16 / FP16 ABFT factor (automatic
        # shift), and of refinement on the FP64-accurate factor (ABFT_F64_EMU,
        # block 256: the slice update takes at most 256 columns), each with its
        # backward error and its error against the FP64 form's solution.
        nc, nbc = args.cond_n, 512
        Bc = torch.from_numpy(W.rhs(nc, 16, seed=1003)).to(dev)
        Xc = torch.empty_like(Bc)
        conditioned = {"n": nc, "nb": nbc, "tol": 1e-12, "nrhs": 16,
                       "matrix": ("Q diag(sigma) Q^T, Q = 2 random butterfly networks"
                                  if nc & (nc - 1) == 0 else "Q diag(sigma) Q^T, Q from QR(N(0,1))")}
        for kappa in (1e2, 1e6, 1e10):
            if nc & (nc - 1) == 0:
                Ac = W.spd_kappa_butterfly_torch(nc, kappa, seed=1002, device=dev)
            else:
                Ac = W.spd_kappa_torch(nc, kappa, seed=1002, device=dev)
            Lc = torch.empty_like(Ac)
            anorm = float(Ac.abs().sum(1).amax())
            def eta_of(X):
                R = Bc - Ac @ X
                return float((R.abs().amax(0) / (anorm * X.abs().amax(0) + Bc.abs().amax(0))).max())
            def fp64_form():
                Lc.copy_(Ac)
                abft.potrf(Lc, nbc, abft.FULL, workspace=wsp)
                Xc.copy_(Bc)
                abft.potrs(Lc, Xc, nbc, abft.F64)
            ms64, _ = timed(fp64_form, 1, 0)   # one run (about 12 s at n = 32768)
            X64 = Xc.clone()
            entry = {"fp64_ms_to_solution": ms64, "fp64_backward_err": eta_of(X64)}
            runs = [("bf16", abft.MIXED_BF16, nbc, True), ("f16", abft.MIXED_F16, nbc, True),
                    ("fp64_emulated_ir", abft.F64_EMU, 256, False)]
            for name, dt, nbr, gmres in runs:
                if gmres:
                    maxit = 3 if kappa >= 1e10 else 20
                    def run():
                        return abft.posv_gmres_ir(Ac, Bc, nbr, dt, abft.FULL, tol=1e-12,
                                                  maxit=maxit, m=60, inner_tol=1e-6, L=Lc, X=Xc,
                                                  workspace=wsp)
                else:
                    def run():
                        return abft.posv_ir(Ac, Bc, nbr, dt, abft.FULL, tol=1e-12, maxit=10,
                                            L=Lc, X=Xc, workspace=wsp)
                ms_g, res = timed(run, 1, 1)
                rc_g, _, _, rep_g = res
                err = float((Xc - X64).abs().max() / X64.abs().max())
                e = {"ms_to_solution": ms_g, "speedup_vs_fp64": ms64 / ms_g, "nb": nbr,
                     "rc": rc_g, "backward_err": rep_g["backward_err"],
                     "reached_tol": rep_g["backward_err"] <= 1e-12,
                     "ir_iters": rep_g["ir_iters"], "rel_err_vs_fp64_form": err}
                if gmres:
                    e.update({"gmres_iters": rep_g["gmres_iters"], "attempts": rep_g["attempts"],
                              "shift": rep_g["shift"]})
                entry[name] = e
            emu_ms = entry["fp64_emulated_ir"]["ms_to_solution"]
            for name in ("bf16", "f16"):
                entry[name]["speedup_vs_fp64_emulated_ir"] = emu_ms / entry[name]["ms_to_solution"]
            conditioned[f"{kappa:.0e}"] = entry
            del Ac, Lc, X64
        del Bc, Xc

    campaign = None
    if args.campaign:
        # Fault campaign (Sec. 3.1.2 / E5 of the paper, with error rates as
        # inputs instead of overclocking): errors arrive as Poisson processes
        # per second of the factorization, with rates that rise through it --
        # none in steps 0-4, 0D errors in steps 5-9, 0D and 1D errors in steps
        # 10-14 (expected counts 0.8, then 0.5 + 0.3) -- and strike uniformly
        # over the trailing block triangle of their step.  Each trial factors
        # the same matrix under each policy; it is correct when no error is left
        # in the factor (max |L - L_clean| <= 1e-10 max |L_clean|).
        ncp, nbp = 4096, 256
        Np = ncp // nbp
        Ap = W.spd_mmt_torch(ncp, seed=1000 + ncp, device=dev)
        Wp = torch.empty_like(Ap)
        def fact(modes, flist=()):
            Wp.copy_(Ap)
            return abft.potrf_sched(Wp, nbp, modes, faults=flist, workspace=wsp, check=False)
        fact([abft.NONE] * Np)
        Lclean = torch.tril(Wp).clone()
        lmax = float(Lclean.abs().max())
        # per-step time, predicted from the step's share of the update flops
        t_all, _ = timed(lambda: fact([abft.NONE] * Np), 3, 1)
        flk = np.array([(ncp - (k + 1) * nbp) ** 2 * nbp + nbp ** 3 for k in range(Np)],
                       dtype=np.float64)
        Tk = (t_all * 1e-3) * flk / flk.sum()
        segments = [(0, 5, 0.0, 0.0), (5, 10, 0.8, 0.0), (10, 15, 0.5, 0.3)]
        lam_k = np.zeros((Np, 3))
        modes_ad = [abft.NONE] * Np
        cov_ad = [1.0] * Np
        for k0, k1, mu0, mu1 in segments:
            ts = float(Tk[k0:k1].sum())
            lam = (mu0 / ts, mu1 / ts, 0.0)
            lam_k[k0:k1] = lam
            m_seg, c_seg = abft.adaptive_modes(ncp, nbp, lam, 0.999999, Tk.tolist())
            modes_ad[k0:k1] = m_seg[k0:k1]
            cov_ad[k0:k1] = c_seg[k0:k1]
        policies = {"none": [abft.NONE] * Np, "single": [abft.SINGLE] * Np,
                    "full": [abft.FULL] * Np, "adaptive": modes_ad}
        r = W.rng(7000)
        trials = []
        for t in range(args.campaign_trials):
            fl_t = []
            for k in range(Np - 1):
                T0 = (k + 1) * nbp
                for mu, kinds in ((lam_k[k, 0] * Tk[k], (abft.F_MEMORY,)),
                                  (lam_k[k, 1] * Tk[k], (abft.F_ROW1D, abft.F_COL1D))):
                    for _ in range(int(r.poisson(mu))):
                        row = int(r.integers(T0, ncp))
                        col = int(r.integers(T0, min(ncp, (row // nbp + 1) * nbp)))
                        kind = kinds[int(r.integers(0, len(kinds)))]
                        fl_t.append((k, kind, row, col, float(r.choice([-1.0, 1.0]) * 1e2)))
            trials.append(fl_t)
        campaign = {"n": ncp, "nb": nbp, "trials": len(trials),
                    "expected_errors": {"steps_0_4": 0.0, "steps_5_9_0d": 0.8,
                                        "steps_10_14_0d": 0.5, "steps_10_14_1d": 0.3},
                    "fc_desired": 0.999999, "adaptive_modes": modes_ad,
                    "adaptive_min_coverage": float(min(cov_ad)),
                    "errors_per_trial": float(np.mean([len(x) for x in trials]))}
        for name, modes in policies.items():
            ok = 0
            for fl_t in trials:
                rc_t, _ = fact(modes, fl_t)
                good = rc_t == 0 and float((torch.tril(Wp) - Lclean).abs().max()) <= 1e-10 * lmax
                ok += int(good)
            ms_p, _ = timed(lambda: fact(modes), 3, 1)
            campaign[name] = {"correct_pct": 100.0 * ok / len(trials), "ms_clean": ms_p}
        for name in ("single", "full", "adaptive"):
            campaign[name]["overhead_pct_vs_none"] = 100.0 * (
                campaign[name]["ms_clean"] / campaign["none"]["ms_clean"] - 1.0)
        del Ap, Wp, Lclean

    lu_qr = None
    if not args.no_lu_qr:
        lu_qr = {}
        U0 = W.uniform_torch(n, seed=1001 + n, device=dev)
        lu_f = W.fault_schedule(n, nb, "lu", seed=3000 + n)
        qr_f = W.fault_schedule(n, nb, "qr", seed=4000 + n)
        def lu_step():
            A.copy_(U0)
            return abft.getrf(A, nb, abft.FULL, faults=lu_f, workspace=wsp)
        def lu_emu_step():   # the trailing update FP64-accurate on the BF16 tensor cores
            A.copy_(U0)
            return abft.getrf(A, nb, abft.FULL, dtype=abft.F64_EMU, faults=lu_f, workspace=wsp)
        def qr_step():
            A.copy_(U0)
            return abft.geqrf(A, nb, abft.FULL, faults=qr_f, workspace=wsp)
        def qr_emu_step():   # V^T [C, r] and C -= V X FP64-accurate on the BF16 tensor cores
            A.copy_(U0)
            return abft.geqrf(A, nb, abft.FULL, dtype=abft.F64_EMU, faults=qr_f, workspace=wsp)
        for name, fn, fl, flops in (("lu", lu_step, lu_f, 2 * n ** 3 / 3),
                                    ("lu_fp64_emulated", lu_emu_step, lu_f, 2 * n ** 3 / 3),
                                    ("qr", qr_step, qr_f, 4 * n ** 3 / 3),
                                    ("qr_fp64_emulated", qr_emu_step, qr_f, 4 * n ** 3 / 3)):
            ms_x, res = timed(fn, 1, 1)
            rep_x = res[-1]
            lu_qr[name] = {"ms": ms_x, "tflops": flops / (ms_x * 1e-3) / 1e12,
                           "pct_of_fp64_peak": 100 * flops / (ms_x * 1e-3) / 1e12 / peak,
                           "faults_located": [(e[0], e[2], e[3]) for e in rep_x["loc"]]
                           == sorted((f[0], f[2], f[3]) for f in fl)}
        del U0

    batched = None
    if not args.no_batched:
        # 4096 SPD matrices, n uniform in [32, 512], one fault per 64 matrices,
        # one persistent launch replayed from a CUDA graph; FP64 and FP32.
        # With N ranks the matrices are split by abft_batched_partition (longest
        # processing time first on n^3/3): each GPU factors its share, the time
        # is the maximum over the ranks, and the statuses are gathered on rank
        # 0 over the host group (nothing is exchanged on the data path).
        from paper_2301_03166_b300 import shard
        from paper_2301_03166_b300 import tune
        sizes = W.batched_sizes(4096, 32, 512, seed=1005)
        owner, load = shard.partition(sizes, ws)
        mine = shard.shard_ids(owner, rank)
        msz = sizes[mine]
        offs = np.concatenate([[0], np.cumsum(msz.astype(np.int64) ** 2)[:-1]])
        tot = int((msz.astype(np.int64) ** 2).sum())
        g = torch.Generator(device=dev)
        base = torch.empty(max(1, tot), dtype=torch.float64, device=dev)
        for li, gi in enumerate(mine):   # matrix gi from its own seed, whatever the split
            nn = int(sizes[gi])
            g.manual_seed(100000 + int(gi))
            M = torch.randn(nn, nn, generator=g, dtype=torch.float64, device=dev)
            Ai = M @ M.T / nn
            Ai.diagonal().add_(1.0)
            base[offs[li]:offs[li] + nn * nn] = Ai.reshape(-1)
        r = W.rng(6000)
        fpos = {q + int(r.integers(0, 64)): q for q in range(0, 4096, 64)}   # one per 64
        bflops = float(sum(int(nn) ** 3 / 3.0 for nn in sizes))
        batched = {"count": 4096, "flops_per_batch": bflops, "gpus": ws,
                   "split": "LPT on n^3/3 (abft_batched_partition), statuses gathered on host",
                   "work_max_over_min": float(load.max() / max(load.min(), 1.0))}
        hgroup = None
        if ws > 1:
            import torch.distributed as dist
            hgroup = dist.new_group(backend="gloo")
        for name, tdt in (("f64", torch.float64), ("f32", torch.float32)):
            table = tune.tune(tdt, dev, per_bucket=64)
            nbf = tune.chooser(table)
            cps = tune.tune_launch(tdt, dev, table=table, sizes=msz)
            abft.set_batched_ctas_per_sm(cps)
            bfaults, gfaults = {}, {}
            fr = W.rng(6001)
            for gi in sorted(fpos):
                nn, b = int(sizes[gi]), nbf(int(sizes[gi]))
                row, col = int(fr.integers(b, max(b + 1, nn))), int(fr.integers(b, max(b + 1, nn)))
                if nn > b:
                    if col // b > row // b:
                        row, col = col, row
                    gfaults[gi] = (0, abft.F_MEMORY, row, col, 1e3)
            local = {int(gi): li for li, gi in enumerate(mine)}
            for gi, f in gfaults.items():
                if gi in local:
                    bfaults[local[gi]] = f
            buf0 = base.to(tdt)
            buf = buf0.clone()
            bt = abft.Batch(buf, msz, offs, nbf, bfaults)
            bws = abft.Workspace()
            def bstep():
                buf.copy_(buf0)
                abft.potrf_batched(bt, use_graph=True, workspace=bws)
            barrier(ws)
            ms_b, _ = timed(bstep, max(1, args.steps), 2)
            ms_copy, _ = timed(lambda: buf.copy_(buf0), max(1, args.steps), 1)
            ms_f = max_over_ranks(ms_b - ms_copy, ws, dev)
            st = shard.gather_statuses(mine, bt.status.cpu().numpy(), 4096, hgroup)
            entry = {"ms_per_batch": ms_f, "matrices_per_s": 4096 / (ms_f * 1e-3),
                     "tflops": bflops / (ms_f * 1e-3) / 1e12, "nb_by_bucket": table,
                     "ctas_per_sm": cps, "bfaults": len(gfaults)}
            if st is not None:   # rank 0: every matrix once, every fault located and corrected
                F = {f: i for i, f in enumerate(abft._STATUS_FIELDS)}
                entry["all_located_and_corrected"] = bool(
                    np.all(st[:, F["info"]] == 0) and
                    int(st[:, F["detected"]].sum()) == len(gfaults) and
                    all(st[gi, F["corrected"]] == 1 and
                        (st[gi, F["ev_row"]], st[gi, F["ev_col"]]) == f[2:4]
                        for gi, f in gfaults.items()))
            batched[name] = entry
            del buf0, buf, bt
        abft.set_batched_ctas_per_sm(0)
        abft.lib().abft_batched_graph_reset()
        del base

    adjoint = None
    if not args.no_adjoint:
        # GP configuration: X n x 8 iid N(0,1), K = exp(-|xi - xj|^2 / 2) + 1e-2 I,
        # y iid N(0,1), loss = y^T K^{-1} y / 2 + logdet K / 2; forward (ABFT
        # Cholesky, solve, logdet) and backward (the hand-written adjoints)
        # through torch.autograd, timed with CUDA events.  Gradient error: against
        # the FP64 closed form (K^{-1} - alpha alpha^T)/2 on the host (n = 4096),
        # and d loss / d lengthscale against central differences (n = 16384).
        from paper_2301_03166_b300 import autograd as ag
        adjoint = {}
        for na in (4096, 16384):
            Xn, yn = W.gp_inputs(na, 8, seed=1004)
            Xg = torch.from_numpy(Xn).to(dev)
            yg = torch.from_numpy(yn).to(dev)
            def kernel(ell):
                sq = (Xg * Xg).sum(1)
                D = torch.clamp(sq[:, None] + sq[None, :] - 2.0 * Xg @ Xg.T, min=0.0)
                return torch.exp(-D / (2.0 * ell ** 2)) + 1e-2 * torch.eye(na, dtype=torch.float64,
                                                                          device=dev)
            K0 = kernel(1.0)
            entry = {}
            for tag, dt in (("fp64", abft.F64), ("fp64_emulated", abft.F64_EMU)):
                Kr = K0.clone().requires_grad_(True)
                def fwd():
                    return ag.gp_negative_log_likelihood_terms(Kr, yg, 256, dtype=dt)
                def fwd_bwd():
                    Kr.grad = None
                    loss = fwd()
                    loss.backward()
                    return loss
                ms_f, _ = timed(lambda: fwd().detach(), 1, 1)
                ms_fb, loss = timed(fwd_bwd, 1, 1)
                e = {"ms_forward": ms_f, "ms_forward_backward": ms_fb, "ms_backward": ms_fb - ms_f,
                     "loss": float(loss.item())}
                if na == 4096:
                    Kh = K0.cpu().numpy()
                    Kinv = np.linalg.inv(Kh)
                    al = Kinv @ yn
                    Gc = 0.5 * (Kinv - np.outer(al, al))
                    e["grad_rel_err_vs_closed_form"] = float(
                        np.linalg.norm(Kr.grad.cpu().numpy() - Gc) / np.linalg.norm(Gc))
                else:
                    ell = torch.tensor(1.0, dtype=torch.float64, device=dev, requires_grad=True)
                    ag.gp_negative_log_likelihood_terms(kernel(ell), yg, 256, dtype=dt).backward()
                    h = 1e-6
                    with torch.no_grad():
                        lp = ag.gp_negative_log_likelihood_terms(kernel(1.0 + h), yg, 256, dtype=dt)
                        lm = ag.gp_negative_log_likelihood_terms(kernel(1.0 - h), yg, 256, dtype=dt)
                    fd = (lp.item() - lm.item()) / (2 * h)
                    e["dloss_dlengthscale_rel_err_vs_fd"] = abs(ell.grad.item() - fd) / max(1.0, abs(fd))
                entry[tag] = e
                del Kr
            adjoint[f"n{na}"] = entry
            del K0, Xg, yg

    e2e = None
    if not args.no_e2e:
        A0h = A0.cpu().pin_memory()
        Lh = torch.empty_like(A0h).pin_memory()
        def e2e_step():
            A.copy_(A0h, non_blocking=True)
            rc, rep = abft.potrf(A, nb, abft.FULL, faults=faults, workspace=wsp)
            Lh.copy_(A, non_blocking=True)
            torch.cuda.synchronize(dev)
            return rc
        e2e_step()
        barrier(ws)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        t = (time.perf_counter() - t0) / args.steps
        t = max_over_ranks(t, ws, dev)
        e2e = {"value": ws * chol_flops(n) / t / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": n * n * 8, "d2h_bytes_per_step": n * n * 8 + ctypes.sizeof(abft.Report),
               "ms_per_step": t * 1e3}
        del A0h, Lh

    cpu = None
    cpu_lapack = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        times, ns = cpu_baseline()
        cpu = {"value": chol_flops(ns) / times[0] / 1e12, "unit": "TFLOP/s", "cores": 1,
               "kind": "oracle",
               "sample": f"one full FP64 ABFT Cholesky (full checksums, faults 1 per 10 steps) "
                         f"at n={ns}, block 256, {times[0]:.1f} s; TFLOP/s counted as n^3/3"}
        try:
            t_l, thr, lname = lapack_baseline(A0.cpu().numpy())
            cpu_lapack = {"value": chol_flops(n) / t_l / 1e12, "unit": "TFLOP/s", "cores": thr,
                          "kind": lname,
                          "sample": f"one Cholesky of the benchmark matrix (n={n}, no "
                                    f"checksums) on the host, {t_l:.1f} s"}
        except Exception as e:   # context only: never fail the bench line for it
            cpu_lapack = {"value": None, "unavailable": repr(e)[:200]}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "nb": nb, "mode": "full",
                       "faults_per_step": len(faults), "l2": "inputs larger than L2 (2.1 GB matrix)",
                       "parallelism": f"replicas x{ws}"},
            "pct_of_fp64_peak": 100.0 * value / ws / peak,
            "abft": {"detected": rep["detected"], "corrected": rep["corrected"],
                     "uncorrectable": rep["uncorrectable"], "events_match_injected": events_ok,
                     "max_ratio": rep["max_ratio"], **(overhead or {})},
            "fp64_emulated": emulated,
            "mixed_precision_ir": mixed, "lookahead": lookahead, "conditioned": conditioned,
            "adjoint": adjoint,
            "campaign": campaign,
            "lu_qr": lu_qr,
            "batched": batched,
            "roofline": roofline, "cpu_baseline": cpu, "cpu_lapack": cpu_lapack, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk,
            "energy": energy_line,
        }), flush=True)


def profile_case(args):
    """One case, warm-up then once, for a profiler; the same inputs as the
    benchmark's."""
    from paper_2301_03166_b300 import abft
    from paper_2301_03166_b300 import workloads as W
    dev = torch.device("cuda:0")
    if args.profile_case == "fp64-pipes":
        # the FP64 FMA against the FP64 tensor-core MMA, with the SM clock seen
        clocks = ClockSampler(board_id(0))
        clocks.start()
        r = {"dfma_tflops": abft.fp64_pipe_probe(0, 200000),
             "dmma_m8n8k4_tflops": abft.fp64_pipe_probe(1, 200000)}
        r["clocks"] = clocks.stop()
        print(json.dumps(r), flush=True)
        return
    n, nb = args.n, args.nb
    A0 = W.spd_mmt_torch(n, seed=1000 + n, device=dev)
    A = torch.empty_like(A0)
    faults = W.fault_schedule(n, nb, "cholesky", seed=2000 + n)
    wsp = abft.Workspace()
    B = torch.from_numpy(W.rhs(n, 16, seed=1003)).to(dev)
    X = torch.empty_like(B)
    if args.profile_case in ("batched-f64", "batched-f32"):
        # 1024 matrices of the batched configuration's size mix (n in [32, 512]),
        # block 64, one fault per 64 matrices: 0.77 GB in FP64, above L2
        sizes = W.batched_sizes(1024, 32, 512, seed=1005)
        offs = np.concatenate([[0], np.cumsum(sizes.astype(np.int64) ** 2)[:-1]])
        tdt = torch.float64 if args.profile_case == "batched-f64" else torch.float32
        buf0 = torch.cat([torch.from_numpy(W.spd_mmt(int(m), seed=100000 + i).reshape(-1))
                          for i, m in enumerate(sizes)]).to(dev).to(tdt)
        buf = buf0.clone()
        r = W.rng(6000)
        bf = {}
        for q in range(0, 1024, 64):
            i = q + int(r.integers(0, 64))
            m = int(sizes[i])
            if m > 64:
                row, col = int(r.integers(64, m)), int(r.integers(64, m))
                bf[i] = (0, abft.F_MEMORY, max(row, col), min(row, col), 1e3)
        bt = abft.Batch(buf, sizes, offs, 64, bf)
        for _ in range(2):
            buf.copy_(buf0)
            abft.potrf_batched(bt, workspace=wsp)
        torch.cuda.synchronize(dev)
        return
    if args.profile_case in ("lu", "lu-emu", "qr", "qr-emu"):
        U0 = W.uniform_torch(n, seed=1001 + n, device=dev)
        for _ in range(2):
            A.copy_(U0)
            if args.profile_case in ("qr", "qr-emu"):
                dt = abft.F64 if args.profile_case == "qr" else abft.F64_EMU
                abft.geqrf(A, nb, abft.FULL, dtype=dt,
                           faults=W.fault_schedule(n, nb, "qr", seed=4000 + n), workspace=wsp)
            else:
                dt = abft.F64 if args.profile_case == "lu" else abft.F64_EMU
                abft.getrf(A, nb, abft.FULL, dtype=dt,
                           faults=W.fault_schedule(n, nb, "lu", seed=3000 + n), workspace=wsp)
        torch.cuda.synchronize(dev)
        return
    if args.profile_case in ("adjoint", "adjoint-emu"):
        # the GP loss of the adjoint configuration (X n x 8, K = exp(-|xi - xj|^2 / 2)
        # + 1e-2 I), forward and backward through torch.autograd, twice
        from paper_2301_03166_b300 import autograd as ag
        Xn, yn = W.gp_inputs(n, 8, seed=1004)
        Xg = torch.from_numpy(Xn).to(dev)
        yg = torch.from_numpy(yn).to(dev)
        sq = (Xg * Xg).sum(1)
        D = torch.clamp(sq[:, None] + sq[None, :] - 2.0 * Xg @ Xg.T, min=0.0)
        K0 = torch.exp(-D / 2.0) + 1e-2 * torch.eye(n, dtype=torch.float64, device=dev)
        dt = abft.F64 if args.profile_case == "adjoint" else abft.F64_EMU
        for _ in range(2):
            Kr = K0.clone().requires_grad_(True)
            ag.gp_negative_log_likelihood_terms(Kr, yg, nb, dtype=dt).backward()
        torch.cuda.synchronize(dev)
        return
    if args.profile_case == "potrs-f32":
        A.copy_(A0)
        abft.potrf(A, nb, abft.FULL, workspace=wsp)
    for _ in range(2):
        if args.profile_case in ("fp64", "fp64-emu"):
            A.copy_(A0)
            dt = abft.F64 if args.profile_case == "fp64" else abft.F64_EMU
            abft.potrf(A, nb, abft.FULL, dtype=dt, faults=faults, workspace=wsp)
        elif args.profile_case == "potrs-f32":
            X.copy_(B)
            abft.potrs(A, X, nb, abft.F32)
        else:
            dt = abft.MIXED_BF16 if args.profile_case == "mixed-bf16" else abft.MIXED_F16
            abft.posv_ir(A0, B, nb, dt, abft.FULL, tol=1e-12, maxit=100, faults=faults, L=A,
                         X=X, workspace=wsp)
    torch.cuda.synchronize(dev)


def main():
    args = parse()
    if args.profile_case:
        profile_case(args)
        return
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
