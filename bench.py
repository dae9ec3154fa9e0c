#!/usr/bin/env python
"""Benchmark of the PICO noise-map hot path on GB300 (one JSON line on rank 0).

One step = one pass of the whole hot path over one batch of synthetic input:
a PICO variance map from K random-phase probes (probe draw, K batched CG-SENSE
solves of 30 iterations with the fused SENSE normal operator, accumulation)
plus a PMR map from K replicas (k-space noise draw, adjoint, the same batched
CG, accumulation) on the 320x320, 15-coil, R=2 + 24-line knee-shaped
Cartesian workload.  ``value`` is CG solves (probes + replicas) per second
over all ranks, inputs resident in HBM; ``e2e`` is the same metric through the
C ABI from host buffers (operator upload, maps read back) per step.

``--impl reference`` times the CPU oracle on the host cores instead (a bounded
sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1%-error noise map, PICO vs PMR on one GB300; probe-solves/s; p99 latency"
UNIT = "probe-solves/s"
SEED_PICO, SEED_PMR = 20260521, 7700417
FP32_LANES_PER_SM, N_SM, SM_MAX_MHZ = 128, 152, 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="knee320_r2")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def workload(name):
    import synth
    w = synth.WORKLOADS[name]
    return w, w.inputs()


def flops_per_probe(w):
    """Algorithmic FLOPs of one normal-operator application to one image:
    per coil and readout column an FFT and an inverse FFT of length ny
    (5 N log2 N each) and the sensitivity multiply / conjugate combine-add
    (6 + 8 flops per sample) plus the mask (2 per sample)."""
    N = w.ny
    return w.nc * w.nx * (2 * 5 * N * math.log2(N) + 16 * N)


def bytes_per_probe_normal(w):
    """HBM bytes of one fused CG normal-operator launch per image: reads r and
    p_old, writes p and q (complex64)."""
    return 4 * w.ny * w.nx * 8


def cores_in_use():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline leg)
# ---------------------------------------------------------------------------
def oracle_sample(w, inp, nprobe=1, nrep=1):
    from oracle import ops as O
    from oracle import pico as OP
    op = O.Operator(inp["smaps"], inp["noise_cov"], mask=inp["mask"])
    t0 = time.perf_counter()
    OP.pico(op, SEED_PICO, 0, nprobe, 0.0, w.max_iter, 0.0)
    OP.pmr(op, SEED_PMR, 0, nrep, w.sigma, 0.0, w.max_iter, 0.0)
    dt = time.perf_counter() - t0
    return (nprobe + nrep) / dt, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, inp = workload(args.workload)
    for _ in range(args.warmup):
        oracle_sample(w, inp)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_sample(w, inp)
        times.append(dt)
    total = sum(times)
    value = 2 * args.steps / total
    sample = f"1 PICO probe + 1 PMR replica per step ({w.max_iter} CG iterations each), FP64 NumPy"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": args.workload, "ny": w.ny, "nx": w.nx, "coils": w.nc, "R": w.R, "acs": w.acs,
                   "cg_iters": w.max_iter, "probes_per_step": 1, "replicas_per_step": 1},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev, self.proc, self.lines = dev, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thr.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2605_09590_gb300 as pico
    from paper_2605_09590_gb300 import build as pico_build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        pico_build.build()
    if world > 1:
        dist.barrier()
    pico.load_library()

    w, inp = workload(args.workload)
    K = w.probes
    n = w.ny * w.nx
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    op = pico.Operator(inp["smaps"], mask=inp["mask"], noise_cov=inp["noise_cov"], max_batch=K,
                       power_iters=15, stream=stream.cuda_stream)
    s = torch.zeros((w.ny, w.nx), dtype=torch.float64, device=dev)
    ss, ps, pss = torch.zeros_like(s), torch.zeros_like(s), torch.zeros_like(s)
    red = torch.zeros((2, w.ny, w.nx), dtype=torch.float64, device=dev)

    def step(i):
        begin = (i * world + rank) * K
        pico.pico_variance_map(op.ctx, SEED_PICO, begin, K, pico.PICO_PROBE_PHASE, w.max_iter, 0.0, s, ss, True)
        pico.pico_pmr(op.ctx, SEED_PMR, begin, K, w.sigma, w.max_iter, 0.0, ps, pss, True)
        if world > 1:   # combine the partial maps of all ranks (one exchange per map)
            red[0].copy_(s)
            red[1].copy_(ps)
            dist.all_reduce(red)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    pico.pico_launch_count(op.ctx, reset=True)
    pico.pico_profile(op.ctx, True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev[0].record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    launches = pico.pico_launch_count(op.ctx)
    norm_ms, norm_n = pico.pico_profile_read(op.ctx, 0)
    upd_ms, upd_n = pico.pico_profile_read(op.ctx, 1)
    pmr_ms, pmr_n = pico.pico_profile_read(op.ctx, 2)
    acc_ms, acc_n = pico.pico_profile_read(op.ctx, 3)
    pico.pico_profile(op.ctx, False)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    solves = 2 * K * args.steps * world
    value = solves / (total_ms / 1e3)

    # roofline of the dominant kernel (the fused CG normal operator)
    avg_norm_s = norm_ms / max(norm_n, 1) / 1e3
    flops_launch = K * flops_per_probe(w)
    achieved = flops_launch / avg_norm_s / 1e12
    peak = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": "k_col_normal<20,16,CG>",
            "avg_launch_ms": avg_norm_s * 1e3, "launches": norm_n,
            "hbm_GBps_algorithmic": K * bytes_per_probe_normal(w) / avg_norm_s / 1e9,
            "peak_note": "FP32 FMA peak 152 SM x 128 lanes x 2 x 2070 MHz (nominal max clock)"}
    share = {"normal_op_ms": norm_ms, "cg_vector_ms": upd_ms, "pmr_adjoint_ms": pmr_ms, "accumulate_ms": acc_ms}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64", "data": "synthetic",
        "config": {"workload": args.workload, "ny": w.ny, "nx": w.nx, "coils": w.nc, "R": w.R, "acs": w.acs,
                   "noise_cov": "15x15 correlated", "cg_iters": w.max_iter, "probes_per_step": K,
                   "replicas_per_step": K, "l2": f"working set {4 * K * n * 8 / 1e9:.2f} GB of CG vectors > 129 MB L2",
                   "parallelism": f"probe shards x{world}"},
        "roofline": roof, "kernel_ms_in_timed_region": share,
        "gpu_launches": launches,
        "clocks": clk,
        "latency_ms": {"p50": statistics.median(per_step), "p99": max(per_step) if len(per_step) < 100 else
                       sorted(per_step)[int(0.99 * len(per_step))]},
    }

    # end to end through the C ABI from host buffers
    if not args.no_e2e:
        S_h = np.ascontiguousarray(inp["smaps"])
        m_h, C_h = inp["mask"], inp["noise_cov"]
        out_h = np.empty((2, w.ny, w.nx), dtype=np.float64)
        e2e_steps = max(2, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            op2 = pico.Operator(S_h, mask=m_h, noise_cov=C_h, max_batch=K, power_iters=15,
                                stream=stream.cuda_stream)
            a, _ = op2.variance_sums(SEED_PICO, K, w.max_iter, 0.0, probe_begin=(i * world + rank) * K)
            b, _ = op2.pmr_sums(SEED_PMR, K, w.sigma, w.max_iter, 0.0, rep_begin=(i * world + rank) * K)
            out_h[0] = a.cpu().numpy()
            out_h[1] = b.cpu().numpy()
            op2.close()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([dt], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        line["e2e"] = {"value": 2 * K * e2e_steps * world / dt, "unit": UNIT,
                       "h2d_bytes_per_step": int(S_h.nbytes + m_h.nbytes + (C_h.nbytes if C_h is not None else 0)),
                       "d2h_bytes_per_step": int(out_h.nbytes), "steps": e2e_steps,
                       "includes": "pico_init (upload, whitening, power method, workspace) + maps + read-back"}

    if rank == 0 and world == 1 and not args.no_cpu:
        v, dt = oracle_sample(w, inp)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"1 PICO probe + 1 PMR replica of the same workload, {dt:.1f} s, "
                                          f"NumPy FP64 (single-threaded pocketfft; {cores_in_use()} cores visible)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    op.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
