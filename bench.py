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

With one GPU the same line also carries, under their own keys, the spiral
240x240 R=2 workload (throughput and time to a 1 %-error map under both
solver rules), the nonlinear CS workload and the serving mix (p50 / p99
request latency); ``--no-extra`` leaves them out.

``--gpus N`` runs N ranks (one per GPU): started by torch.distributed.run, or
re-launched through it when the environment has no WORLD_SIZE.  Each rank
takes its own probe range and the partial running sums are combined with one
all-reduce per step.

``--impl reference`` times the CPU oracle on the host cores instead (a bounded
sample of the same workload per step, one single-threaded oracle process per
core).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1%-error noise map, PICO vs PMR on one GB300; probe-solves/s; p99 latency"
UNIT = "probe-solves/s"
SEED_PICO, SEED_PMR = 20260521, 7700417
FP32_LANES_PER_SM, N_SM, SM_MAX_MHZ = 128, 152, 2070.0
CSRC = os.path.join(ROOT, "paper_2605_09590_gb300", "csrc")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="knee320_r2")
    ap.add_argument("--solver", default="global", choices=["global", "columns"],
                    help="CG of the primary workload: whole image (default) or per readout column")
    ap.add_argument("--probes", type=int, default=0, help="probes (and replicas) per step; 0 = the workload's")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-t1pct", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="leave out the spiral, CS and serving keys of the default one-GPU line")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes instead of pico_autotune's choice")
    ap.add_argument("--serving", type=int, default=200, help="requests of the serving mix (0: none)")
    ap.add_argument("--serving-load", type=float, default=0.8, help="offered load of the serving mix")
    ap.add_argument("--t1pct-spiral", action="store_true",
                    help="with --workload spiral240_rN: time to 1%% against the full exact diagonal (minutes)")
    ap.add_argument("--t1pct-cs", type=int, default=0, metavar="NREF",
                    help="time to 1%% on the CS workload against method-specific references of NREF samples")
    return ap.parse_args()


def maybe_relaunch(args):
    """``--gpus N`` without a launcher: re-exec this script under
    torch.distributed.run with N ranks; a mismatch with WORLD_SIZE is an error."""
    env = os.environ.get("WORLD_SIZE")
    if args.gpus > 1 and env is None:
        import socket
        s = socket.socket()
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
        s.close()
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr", "127.0.0.1", f"--master-port={port}", os.path.abspath(__file__)] + sys.argv[1:]
        os.execv(sys.executable, cmd)
    if env is not None and int(env) != args.gpus:
        sys.exit(f"bench.py: --gpus {args.gpus} does not match WORLD_SIZE={env}")


def workload(name, probes=0):
    import dataclasses
    import synth
    w = synth.WORKLOADS[name]
    if probes:
        w = dataclasses.replace(w, probes=probes)
    return w, w.inputs()


def flops_per_probe(w):
    """Algorithmic FLOPs of one normal-operator application to one image.

    Cartesian (column-decoupled): per coil and readout column an FFT and an
    inverse FFT of length ny (5 N log2 N each) plus the sensitivity multiply,
    conjugate combine-add and mask (16 flops per sample).
    Spiral (Toeplitz, grid L = 2n): per coil n row FFTs, L column FFT pairs and
    n row IFFTs of length L (5 L log2 L each), plus 16 flops per image sample
    and 2 per grid sample for the kernel multiply."""
    if w.kind == "cartesian":
        N = w.ny
        return w.nc * w.nx * (2 * 5 * N * math.log2(N) + 16 * N)
    n, L = w.ny, 2 * w.ny
    fft = 5 * L * math.log2(L)
    return w.nc * ((2 * n + 2 * L) * fft + 16 * n * n + 2 * L * L)


def alg_bytes_normal(w, K):
    """Algorithmic HBM bytes of one normal-operator launch over K images inside
    CG: every image reads r and p_old and writes p and q (4 images of 8 bytes
    per voxel), plus one pass over the operator's own data -- the whitened
    sensitivities S (Cartesian) or S and the real Toeplitz kernel T^ on the
    2n x 2n grid (spiral).  Spiral images also move their coil half-grids
    through HBM between the three Toeplitz passes (4 x nc x n x 2n complex64
    per image)."""
    V = w.ny * w.nx * 8
    S = w.nc * V
    per = 4 * V
    if w.kind == "spiral":
        # the streaming Toeplitz passes write and read every coil's n x 2n
        # half-grid twice (the passes are separate launches)
        S += (2 * w.ny) ** 2 * 4
        per += 4 * w.nc * w.ny * 2 * w.ny * 8
    return K * per + S


def flops_2d_normal(w):
    """Algorithmic FLOPs of one 2-D-mask Cartesian normal operator on one image:
    per coil a 2-D FFT and inverse 2-D FFT of n x n (4 n line FFTs of length n,
    5 n log2 n each) plus 16 flops per image sample (S multiply, conj(S)
    combine-add) and 2 per k-space sample (mask)."""
    n = w.ny
    return w.nc * (4 * n * 5 * n * math.log2(n) + 18 * n * n)


def kernel_digest(*names):
    """Short hash of the kernel sources a measured counter belongs to."""
    h = hashlib.sha256()
    for nm in names:
        with open(os.path.join(CSRC, nm), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant
# kernel from one ncu capture (the summaries in the profiles folder; two
# full-size launches averaged, a one-pass metric set), keyed by (workload,
# images per launch, kernel, digest of the kernel sources at capture time): a
# changed kernel no longer matches and its traffic is reported as null.
GRAM_FILES = ("gram.cu", "tc_util.cuh", "kernels.cuh", "f16_split.cuh")
PERSIST_FILES = ("colcg_persist.cu", "tc_util.cuh", "kernels.cuh", "f16_split.cuh")
TRAFFIC = {
    ("knee320_r2", 256, "gram", "580cead29cb443a1"): (713.137664e6 + 378.007808e6 + 711.760128e6 + 374.798592e6) / 2,
    ("knee320_r2", 256, "persist", "b7cf5961e2e5f7f1"): (473.558528e6 + 375.167488e6 + 473.355264e6 + 371.994624e6) / 2,
    # one spiral normal operator = k_toep_rows_fwd + k_toep_cols_w + k_toep_rows_inv (two of each averaged)
    ("spiral240_r2", 256, "fft", "40fe3b9a9e3fec65"): ((4720.102912e6 + 4661.500160e6 + 4719.623168e6 + 4658.126080e6)
                                                       + (5086.091520e6 + 133.305856e6 + 5086.246656e6 + 133.519616e6)
                                                       + (474.891264e6 + 4772.518912e6 + 474.142464e6 + 4772.286208e6)) / 2,
}


def measured_peaks():
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        return json.load(f)


def traffic_of(w, K, kernel, kernel_files):
    dig = kernel_digest(*kernel_files)
    return TRAFFIC.get((w.name, K, kernel, dig)), dig


def gram_roofline(w, K, avg_s, launches):
    """Roofline of the tensor-core normal operator (k_gram_normal), HBM-bound.

    achieved = algorithmic bytes per launch (alg_bytes_normal: r, p_old read,
    p, q written per image, one pass over S) / the launch's average CUDA-event
    time, against the measured copy bandwidth.  The split G planes the kernel
    streams instead of S are not algorithmic bytes; they show up in `traffic`.
    The tensor view is kept as a secondary key: nx dense complex
    (ny x ny) x (ny x K) products, 8 ny^2 nx flops per image, issued as three
    FP16 products (dense-equivalent work, not the method's own flop count)."""
    mp = measured_peaks()
    alg = alg_bytes_normal(w, K)
    achieved = alg / avg_s / 1e9
    traffic, dig = traffic_of(w, K, "gram", GRAM_FILES)
    cplx = 8.0 * w.ny * w.ny * w.nx * K
    return {"bound": "hbm", "achieved": achieved, "peak": mp["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / mp["hbm_gbs"], "traffic": traffic,
            "traffic_over_algorithmic": traffic / alg if traffic else None,
            "kernel": "k_gram_normal<16,0,0,1> (tcgen05 kind::f16, FP16 head + remainder of scaled operands, "
                      "fused CG direction update, TMA epilogue)",
            "kernel_digest": dig, "avg_launch_ms": avg_s * 1e3, "launches": launches,
            "algorithmic_bytes_per_launch": alg,
            "peak_note": "measured copy bandwidth (of measured)",
            "tensor_dense_equivalent": {"achieved_TFLOPs": 3.0 * cplx / avg_s / 1e12, "peak_TFLOPs": mp["bf16_tflops"],
                                        "frac": 3.0 * cplx / avg_s / 1e12 / mp["bf16_tflops"],
                                        "note": "3 FP16 products per complex term of the dense per-column "
                                                "Gram contraction; peak = measured bf16 burst (the FP16 dense "
                                                "rate is the same)"}}


def fft_roofline(w, K, avg_s, launches):
    """Roofline of an FFT-based normal operator (column FFTs or the three
    Toeplitz passes), bound by FP32 issue; the HBM view of the same launch
    (alg_bytes_normal) is a secondary key."""
    mp = measured_peaks()
    flops = K * flops_per_probe(w)
    achieved = flops / avg_s / 1e12
    peak = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    files = ("cart_impl.cuh", "kernels.cuh") if w.kind == "cartesian" else ("spiral_impl.cuh", "kernels.cuh")
    traffic, dig = traffic_of(w, K, "fft", files)
    alg = alg_bytes_normal(w, K)
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_over_algorithmic": traffic / alg if traffic else None, "kernel_digest": dig,
            "kernel": "k_col_normal (fused CG prologue)" if w.kind == "cartesian" else
                      "k_toep_rows_fwd + k_toep_cols_w + k_toep_rows_inv (one normal operator)",
            "avg_launch_ms": avg_s * 1e3, "launches": launches,
            "peak_note": "FP32 FMA peak 152 SM x 128 lanes x 2 x 2070 MHz (nominal max clock)",
            "hbm": {"achieved_GBps": alg / avg_s / 1e9, "peak_GBps": mp["hbm_gbs"],
                    "frac": alg / avg_s / 1e9 / mp["hbm_gbs"], "algorithmic_bytes_per_launch": alg}}


def onchip_roofline(w, K, avg_s, launches, solver):
    """Roofline of the on-chip CG solve of small phase-encode images (one launch
    per solve of K images): FP32 work of the dense per-column products,
    8 ny^2 nx flops per image and update, max_iter updates, against the FP32
    FMA peak; the HBM view (the right-hand sides in, the solutions out, G_j
    once) is secondary -- the workload fits in L2 and is latency-bound."""
    mp = measured_peaks()
    flops = 8.0 * w.ny * w.ny * w.nx * K * w.max_iter
    peak = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    V = w.ny * w.nx * 8
    byts = 2 * K * V + w.nx * w.ny * w.ny * 8
    return {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": flops / avg_s / 1e12 / peak, "traffic": None,
            "kernel": ("k_colcg_small<NY,T,GLOBAL> (whole CG solve on chip, one cooperative launch per solve, "
                       "column sums exchanged within each image group)" if solver == "global" else
                       "k_colcg_small<NY,T> (whole per-column CG solve on chip, one launch per solve)"),
            "avg_launch_ms": avg_s * 1e3, "launches": launches,
            "peak_note": "FP32 FMA peak 152 SM x 128 lanes x 2 x 2070 MHz (nominal max clock)",
            "hbm": {"achieved_GBps": byts / avg_s / 1e9, "peak_GBps": mp["hbm_gbs"],
                    "frac": byts / avg_s / 1e9 / mp["hbm_gbs"]}}


def normal_ops_per_probe(w):
    """Normal-operator applications per probe: one CG solve (lam = 0) or two
    solves and one A^H A (lam > 0)."""
    return w.max_iter if w.lam == 0 else 2 * w.max_iter + 1


def cores_in_use():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline leg)
# ---------------------------------------------------------------------------
def oracle_sample(w, inp, nprobe=1, nrep=1):
    """Time the oracle on a bounded sample in this process (one core);
    returns (probe-solves/s, seconds, description)."""
    import numpy as np
    from oracle import ops as O
    from oracle import pico as OP
    if w.kind == "cartesian":
        op = O.Operator(inp["smaps"], inp["noise_cov"], mask=inp["mask"])
        t0 = time.perf_counter()
        OP.pico(op, SEED_PICO, 0, nprobe, 0.0, w.max_iter, 0.0)
        OP.pmr(op, SEED_PMR, 0, nrep, w.sigma, 0.0, w.max_iter, 0.0)
        dt = time.perf_counter() - t0
        return (nprobe + nrep) / dt, dt, (f"{nprobe} PICO probe + {nrep} PMR replica of the same workload "
                                          f"({w.max_iter} CG iterations each)")
    if w.kind == "cs":
        from oracle import cs as OCS
        op = O.Operator(inp["smaps"], inp["noise_cov"], mask=inp["mask"])
        b = op.forward(inp["phantom"].astype(np.complex128))
        h, g = OCS.wavelet_filters(4)
        lam = w.extra["lam_l1_rel"] * np.abs(OCS.dwt2(op.adjoint(b), w.extra["levels"], h, g)).max()
        t0 = time.perf_counter()
        f = OCS.Fista(op, b, lam, w.max_iter, levels=w.extra["levels"])
        t1 = time.perf_counter()
        OCS.pico_cs(f, SEED_PICO, 0, nprobe)
        sigma = cs_sigma(w, np.sqrt(np.mean(np.abs(b[:, inp["mask"].astype(bool)]) ** 2)))
        OCS.pmr_cs(f, SEED_PMR, 0, nrep, sigma)
        t2 = time.perf_counter()
        per_pair = (t2 - t1)
        value = 2.0 * w.probes / ((t1 - t0) + w.probes * per_pair)
        return value, t2 - t0, (f"FISTA reconstruction ({t1 - t0:.1f} s) + {nprobe} Jacobian probe + {nrep} "
                                f"PMR replica ({per_pair:.1f} s), scaled to a step of {w.probes} + {w.probes}")
    op = O.Operator(inp["smaps"], inp["noise_cov"], traj=inp["traj"])
    x = np.ones((w.ny, w.nx), dtype=np.complex128)
    t0 = time.perf_counter()
    op.normal(x, 0.1)
    dt = time.perf_counter() - t0
    per_probe = normal_ops_per_probe(w) * dt
    per_rep = w.max_iter * dt
    return 2.0 / (per_probe + per_rep), dt, (f"one exact-NUDFT A^H A application ({dt:.1f} s), scaled to "
                                             f"{normal_ops_per_probe(w)} per probe and {w.max_iter} per replica")


_OW = {}   # per-process state of the oracle pool workers


def _oracle_worker_init(name):
    from oracle import ops as O
    w, inp = workload(name)
    _OW["w"] = w
    _OW["op"] = O.Operator(inp["smaps"], inp["noise_cov"], mask=inp["mask"])


def _oracle_task(task):
    from oracle import pico as OP
    kind, i = task
    w, op = _OW["w"], _OW["op"]
    if kind == "ready":
        time.sleep(0.2)
        return os.getpid()
    if kind == "pico":
        OP.pico(op, SEED_PICO, i, 1, 0.0, w.max_iter, 0.0)
    else:
        OP.pmr(op, SEED_PMR, i, 1, w.sigma, 0.0, w.max_iter, 0.0)
    return os.getpid()


class OraclePool:
    """One single-threaded oracle process per host core (spawned, so that no
    process is forked after the first GPU call).  A step solves one PICO probe
    and one PMR replica per core; the value is solves per wall-clock second."""

    def __init__(self, name):
        import multiprocessing as mp
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        self.cores = cores_in_use()
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init, initargs=(name,))
        self.pool.map(_oracle_task, [("ready", i) for i in range(self.cores)], chunksize=1)
        self.next = 0

    def step(self):
        tasks = [(k, self.next + i) for i in range(self.cores) for k in ("pico", "pmr")]
        self.next += self.cores
        t0 = time.perf_counter()
        pids = self.pool.map(_oracle_task, tasks, chunksize=1)
        dt = time.perf_counter() - t0
        return len(tasks) / dt, dt, len(set(pids))

    def close(self):
        self.pool.close()
        self.pool.join()


def arm_config(w, world=1):
    """The workload description both arms print (``--impl ours`` adds the
    values it computes on the device, such as the CS weight and noise level)."""
    K = w.probes
    n = w.ny * w.nx
    if w.kind == "cs":
        return {"workload": w.name, "ny": w.ny, "nx": w.nx, "coils": w.nc, "R": w.R,
                "mask": f"Poisson-disc, {w.acs}x{w.acs} calibration", "noise_cov": "correlated",
                "recon": f"L1-wavelet FISTA (db4, {w.extra['levels']} levels), {w.max_iter} iterations, "
                         f"lambda = {w.extra['lam_l1_rel']} max|W A^H b|",
                "probes_per_step": K, "replicas_per_step": K,
                "unit_note": "one solve = one Jacobian-probe product J(J^T v) or one FISTA replica",
                "l2": f"working set {6 * K * n * 8 / 1e9:.2f} GB of images + "
                      f"{w.max_iter * n * 8 / 1e6:.0f} MB trajectory > 129 MB L2",
                "parallelism": f"probe shards x{world}"}
    return {"workload": w.name, "ny": w.ny, "nx": w.nx, "coils": w.nc, "R": w.R, "acs": w.acs,
            "noise_cov": "correlated" if w.noise_corr else "white", "lambda_rel": w.lam,
            "cg_iters": w.max_iter, "probes_per_step": K, "replicas_per_step": K,
            "l2": (f"working set {4 * K * n * 8 / 1e9:.2f} GB of CG vectors > 129 MB L2 (no flush needed)"
                   if 4 * K * n * 8 > 129e6 else
                   f"working set {4 * K * n * 8 / 1e6:.1f} MB fits in L2: steps run back to back without a "
                   f"flush (a latency-bound workload)"),
            "parallelism": f"probe shards x{world}"}


def cs_sigma(w, data_rms):
    """PMR noise level of the CS workload: ``pmr_snr_db`` below the data rms."""
    return float(data_rms) * 10.0 ** (-w.extra["pmr_snr_db"] / 20.0)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, inp = workload(args.workload)
    if w.kind == "cartesian":
        pool = OraclePool(w.name)
        for _ in range(args.warmup):
            pool.step()
        times, vals, procs = [], [], 0
        for _ in range(args.steps):
            v, dt, procs = pool.step()
            times.append(dt)
            vals.append(v)
        pool.close()
        cores = pool.cores
        sample = (f"one PICO probe + one PMR replica ({w.max_iter} CG iterations each) per core in "
                  f"{cores} single-threaded FP64 NumPy oracle processes ({procs} took work), per step")
    else:
        for _ in range(args.warmup):
            oracle_sample(w, inp)
        times, vals = [], []
        for _ in range(args.steps):
            v, dt, sample = oracle_sample(w, inp)
            times.append(dt)
            vals.append(v)
        cores = 1
        sample = sample + ", FP64 NumPy on one core, per step"
    total = sum(times)
    value = sum(v * t for v, t in zip(vals, times)) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": arm_config(w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
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
# time to a 1 %-error noise map (Sec. 3.2.2 protocol: N in steps of 10)
# ---------------------------------------------------------------------------
def exact_variance_cartesian(op, w, torch):
    """Exact diag(Sigma) of a phase-encode Cartesian operator on the GPU.

    A^H A is block diagonal over readout columns, so the probe e_y (x) 1 (row y
    set to one) returns column y of every column block at once: ny converged
    solves give the whole diagonal."""
    ny, nx = w.ny, w.nx
    diag = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    B = 64
    for y0 in range(0, ny, B):
        nb = min(B, ny - y0)
        rhs = torch.zeros((nb, ny, nx), dtype=torch.complex64, device="cuda")
        rhs[torch.arange(nb), torch.arange(y0, y0 + nb)] = 1.0
        x = op.cg(rhs, 100, 1e-6)
        diag[y0:y0 + nb] = x[torch.arange(nb), torch.arange(y0, y0 + nb)].real.double()
    return diag.flatten(), None


def exact_variance_unit_probes(op, w, torch, voxels=None, batch=256):
    """Exact diag(Sigma) by unit-vector probing on the GPU:
    Sigma_kk = x_k^H M x_k with x_k = (M + lam)^-1 e_k (one converged solve and
    one normal-operator application per voxel, batched).  With ``voxels`` only
    those (flat) voxel indices are computed."""
    n = w.ny * w.nx
    idx = torch.arange(n, device="cuda") if voxels is None else voxels
    lam = op.info["lambda_phys"]
    diag = torch.empty(idx.numel(), dtype=torch.float64, device="cuda")
    for k0 in range(0, idx.numel(), batch):
        nb = min(batch, idx.numel() - k0)
        rhs = torch.zeros((nb, n), dtype=torch.complex64, device="cuda")
        rhs[torch.arange(nb), idx[k0:k0 + nb]] = 1.0
        x = op.cg(rhs.view(nb, w.ny, w.nx), 100, 1e-6)
        y = op.apply_normal(x)                       # (M + lam) x
        xy = (x.conj() * y).real.double().flatten(1).sum(1)
        xx = (x.abs() ** 2).double().flatten(1).sum(1)
        diag[k0:k0 + nb] = xy - lam * xx
    return diag, voxels


_EXACT = {}   # exact reference diagonals, computed once per workload


def measure_time_to_1pct(op, w, torch, pico, max_n=20000, step=10, cg=None, arms=None, subset=0):
    """cg = (max_iter, rtol) of the estimators' solves; default the workload's
    fixed iteration count (the reference is always the converged diagonal).
    With ``subset`` > 0 the reference and the NRMSE cover that many seeded
    random voxels (unit-vector probing of the whole image takes minutes)."""
    max_iter, rtol = cg if cg else (w.max_iter, 0.0)
    key = (w.name, subset)
    if key in _EXACT:
        ref, vox, how = _EXACT[key]
    elif w.kind == "cartesian" and not subset:
        ref, vox = exact_variance_cartesian(op, w, torch)
        how = f"exact diag(Sigma) from {w.ny} structured converged CG solves"
    elif subset:
        import numpy as np
        g = np.random.default_rng(0x5EB)
        vox = torch.from_numpy(np.sort(g.choice(w.ny * w.nx, subset, replace=False))).cuda()
        ref, vox = exact_variance_unit_probes(op, w, torch, vox)
        how = (f"exact diag(Sigma) by unit-vector probing of {subset} seeded random voxels; NRMSE over "
               f"those voxels")
    else:
        ref, vox = exact_variance_unit_probes(op, w, torch)
        how = f"exact diag(Sigma) by unit-vector probing ({w.ny * w.nx} converged solves)"
    _EXACT[key] = (ref, vox, how)
    ref_std = ref.clamp_min(0).sqrt()
    nref = torch.linalg.vector_norm(ref_std)
    out = {"reference": how, "step": step, "cg": {"max_iter": max_iter, "rtol": rtol},
           "threshold": 0.01, "nrmse_on": "std maps",
           "reference_range": [float(ref.min()), float(ref.max())]}
    if arms is None:
        # the three probe families of the ablation (Sec. 3.2.2; Eqs. 18-20) and PMR
        arms = (("pico", pico.PICO_PROBE_PHASE), ("pico_rademacher", pico.PICO_PROBE_RADEMACHER),
                ("pico_gauss", pico.PICO_PROBE_GAUSS), ("pmr", None))
    for name, kind in arms:
        s = torch.zeros((w.ny, w.nx), dtype=torch.float64, device="cuda")
        ss = torch.zeros_like(s)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        elapsed, n, hit = 0.0, 0, None
        curve = []
        while n < max_n:
            ev0.record()
            if kind is not None:
                pico.pico_variance_map(op.ctx, SEED_PICO + 1, n, step, kind, max_iter, rtol, s, ss, True)
            else:
                pico.pico_pmr(op.ctx, SEED_PMR + 1, n, step, w.sigma, max_iter, rtol, s, ss, True)
            ev1.record()
            torch.cuda.synchronize()
            elapsed += ev0.elapsed_time(ev1) / 1e3
            n += step
            est = (s.flatten() if vox is None else s.flatten()[vox]) / n
            err = float(torch.linalg.vector_norm(est.clamp_min(0).sqrt() - ref_std) / nref)
            if n in (10, 50, 100, 200, 500, 1000, 2000, 5000, 10000):
                curve.append((n, round(err, 5)))
            if err <= 0.01:
                hit = (n, elapsed, err)
                break
        out[name] = ({"N": hit[0], "seconds_in_steps": hit[1], "nrmse": hit[2], "curve": curve}
                     if hit else {"N": None, "nrmse_at_max": err, "max_n": max_n, "curve": curve})
    return out


# ---------------------------------------------------------------------------
# serving mix: Poisson arrivals of uneven requests (p50 / p99 latency, maps/s)
# ---------------------------------------------------------------------------
def serving_mix(nreq, seed=0):
    import numpy as np
    import synth
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(nreq):
        u = rng.random()
        K = int(rng.choice([32, 64, 128, 256]))
        if u < 0.5:      # Cartesian, 5-smooth even matrix in [192, 384], 8-32 coils
            n = int(rng.choice([192, 240, 256, 320, 384]))
            nc = int(rng.choice([8, 16, 24, 32]))
            # correlation 0.1 at 15 coils, scaled down for more coils to stay well conditioned
            rho = 0.1 * min(1.0, (15.0 / nc) ** 0.5)
            reqs.append(dict(smaps=synth.coil_maps(n, n, nc, i), mask=synth.mask_pe(n, 2, 24),
                             noise_cov=synth.noise_cov(nc, i, rho=rho), seed=i, nprobes=K, max_iter=30,
                             kind=f"cart{n}x{nc}"))
        elif u < 0.8:    # spiral 240^2, 20 coils, R in {2, 3, 4}
            R = int(rng.choice([2, 3, 4]))
            reqs.append(dict(smaps=synth.coil_maps(240, 240, 20, i), traj=synth.spiral_traj(240, 16, 4096, R),
                             lam=0.1, seed=i, nprobes=K, max_iter=30, kind=f"spiral_r{R}"))
        else:            # nonlinear CS 320^2, 15 coils, Poisson-disc R=2 (Jacobian PICO of FISTA)
            reqs.append(dict(cs=True, seed=i, nprobes=K, kind="cs320"))
    return reqs


def cs_request_inputs(pico, torch, seed, mask, n=320, nc=15, iters=100, levels=4):
    """Data of a CS serving request: whitened k-space of a seeded phantom through a
    seeded coil set (computed with the library's forward operator), and the L1
    weight 1e-2 max|W A^H b|."""
    import numpy as np
    import synth
    S = synth.coil_maps(n, n, nc, seed)
    cov = synth.noise_cov(nc, seed)
    op = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=15, max_batch=1)
    x0 = torch.from_numpy(synth.phantom(n, seed).astype(np.complex64)).cuda().reshape(1, n, n)
    b = op.forward(x0)
    coef = torch.empty_like(x0)
    pico.pico_wavelet(op.ctx, op.adjoint(b), coef, levels)
    lam = 1e-2 * float(coef.abs().max())
    op.close()
    return dict(smaps=S, mask=mask, noise_cov=cov, cs_data=b[0].cpu().numpy(), cs_lambda=lam, cs_iters=iters,
                cs_levels=levels)


def run_serving(pico, nreq=200, loads=(0.8,), max_active=4, ncap=60):
    """Capacity from a closed loop over the first ``ncap`` requests of the mix
    (all submitted at once), then an open loop of ``nreq`` Poisson arrivals at
    each offered load (a fraction of that capacity): p50 / p99 of the request
    latency (done - arrival) and maps/s."""
    import numpy as np
    import torch
    import synth
    reqs = serving_mix(nreq)
    if any(r.get("cs") for r in reqs):
        mask = synth.poisson_disc_mask(320, 320, 2.0, 24, 0)     # one sampling pattern for all CS requests
        for r in reqs:
            if r.pop("cs", False):
                r.update(cs_request_inputs(pico, torch, r["seed"], mask))
    strip = lambda r: {k: v for k, v in r.items() if k != "kind"}
    ncap = min(ncap, nreq)
    sv = pico.Server(max_active=max_active, chunk=64)
    t0 = time.perf_counter()
    ids = [sv.submit(**strip(r)) for r in reqs[:ncap]]
    for i in ids:
        sv.wait(i)
    cap = ncap / (time.perf_counter() - t0)
    sv.close()
    kinds = {}
    for r in reqs:
        k = r["kind"].split("x")[0] if r["kind"].startswith("cart") else r["kind"]
        kinds[k] = kinds.get(k, 0) + 1
    out = {"requests": nreq, "request_kinds": kinds,
           "mix": "50% Cartesian 192-384 / 8-32 coils, 30% spiral 240 R=2-4 (30 CG iterations), 20% "
                  "nonlinear CS 320x320 15 coils Poisson-disc R=2 (FISTA 100 iterations, Jacobian PICO); "
                  "K in {32,64,128,256}",
           "capacity_maps_per_s": cap, "capacity_from_requests": ncap, "max_active": max_active, "loads": []}
    rng = np.random.default_rng(1)
    for rho in loads:
        rate = rho * cap
        gaps = rng.exponential(1.0 / rate, size=nreq)
        sv = pico.Server(max_active=max_active, chunk=64)
        t0 = time.perf_counter()
        ids = []
        for r, g in zip(reqs, gaps):
            time.sleep(g)
            ids.append(sv.submit(**strip(r)))
        infos = [sv.wait(i)[2] for i in ids]
        wall = time.perf_counter() - t0
        sv.close()
        lat = np.array([i["t_done"] - i["t_arrival"] for i in infos])
        out["loads"].append({"offered": rho, "p50_s": float(np.percentile(lat, 50)),
                             "p99_s": float(np.percentile(lat, 99)), "max_s": float(lat.max()),
                             "maps_per_s": nreq / wall, "latency_samples": int(lat.size)})
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def timed_steps(step, steps, warmup, torch, dist, world, stream, dev_index, ctxs, pico):
    """Warm up, then time `steps` calls of step(i) with CUDA events on the
    launching stream, bracketed by a barrier and a synchronisation on both
    sides; clocks are sampled meanwhile.  Returns (total_ms, per-step ms,
    clocks, launches, per-class (ms, launches) of the first context)."""
    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(dev_index)
    clocks.start()
    time.sleep(0.3)
    for c in ctxs:
        pico.pico_launch_count(c, reset=True)
        pico.pico_profile(c, True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev[0].record(stream)
    for i in range(steps):
        step(warmup + i)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    launches = sum(pico.pico_launch_count(c) for c in ctxs)
    prof = [pico.pico_profile_read(ctxs[0], k) for k in range(4)]
    for c in ctxs:
        pico.pico_profile(c, False)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, per_step, clk, launches, prof


def colcg_roofline(w, K, avg_s, launches):
    """Roofline of the fused per-column CG update (k_gram_normal with the
    column-CG epilogue), HBM-bound: per image it reads r and p_old (the
    contraction operand), writes p, reads and writes x and writes r (6 images
    of 8 bytes per voxel), plus one pass over S; no separate vector kernel
    runs.  Against the measured copy bandwidth."""
    mp = measured_peaks()
    V = w.ny * w.nx * 8
    alg = 6 * K * V + w.nc * V
    achieved = alg / avg_s / 1e9
    traffic, dig = traffic_of(w, K, "colcg", GRAM_FILES)
    return {"bound": "hbm", "achieved": achieved, "peak": mp["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / mp["hbm_gbs"], "traffic": traffic,
            "traffic_over_algorithmic": traffic / alg if traffic else None,
            "kernel": "k_gram_normal<16,0,1,1> (tcgen05 kind::f16 column-CG update: operator, step, x / r update "
                      "and next beta in one launch, 2-CTA clusters)",
            "kernel_digest": dig, "avg_launch_ms": avg_s * 1e3, "launches": launches,
            "algorithmic_bytes_per_launch": alg, "peak_note": "measured copy bandwidth (of measured)"}


def persist_rows(ny):
    """Rows per CTA of the whole-solve per-column kernel (0: not used)."""
    if ny % 16:
        return 0
    for nt in (80, 64, 48, 32):
        if ny % nt == 0 and 2 <= ny // nt <= 8:
            return nt
    return 0


def persist_roofline(w, K, avg_s, launches):
    """Roofline of the per-column CG with the whole solve in one launch
    (k_colcg_persist: a cluster owns a column and 128 images, x, r, p stay on
    chip).  Tensor-bound: every update issues 12 FP16 MMAs of M 128 x N NT x
    K 16 per 16-row chunk (the FP16 head + remainder split of the complex
    product, dense-equivalent work) for every (column, image tile, row block),
    max_iter updates per launch, against the measured sustained dense bf16
    peak (the kernel runs for milliseconds inside a long step; FP16 runs at the
    bf16 rate).  The HBM view: the right-hand sides in and the solutions out
    (2 images of 8 bytes per voxel) and G once."""
    mp = measured_peaks()
    nt = persist_rows(w.ny)
    tiles = -(-K // 128)
    flops = float(w.max_iter) * w.nx * tiles * (w.ny // nt) * (w.ny // 16) * 12 * 2 * 128 * nt * 16
    achieved = flops / avg_s / 1e12
    V = w.ny * w.nx * 8
    byts = 2 * K * V + 8 * w.nx * w.ny * w.ny
    peak = mp["bf16_tflops_sustained"]
    traffic, dig = traffic_of(w, K, "persist", PERSIST_FILES)
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "kernel_digest": dig,
            "traffic_over_hbm_bytes": traffic / byts if traffic else None,
            "kernel": "k_colcg_persist<%d> (whole per-column CG solve per launch: clusters of %d CTAs own a column "
                      "and 128 images, x / p / accumulator in tensor memory, r in shared memory, tcgen05 "
                      "kind::f16)" % (nt, w.ny // nt),
            "avg_launch_ms": avg_s * 1e3, "launches": launches, "mma_flops_per_launch": flops,
            "peak_note": "measured sustained dense bf16 GEMM peak (of measured); FP16 MMAs run at the bf16 rate",
            "hbm": {"achieved_GBps": byts / avg_s / 1e9, "peak_GBps": mp["hbm_gbs"],
                    "frac": byts / avg_s / 1e9 / mp["hbm_gbs"], "bytes_per_launch": byts}}


def bench_linear(args, w, inp, pico, torch, dist, world, rank, local, steps, warmup, primary, tune_cache,
                 solver="global"):
    """One step = PICO map of K probes + PMR map of K replicas on a linear
    (CG-SENSE) workload; returns (sub-line, operator).  solver = "columns"
    runs CG per readout column (phase-encode Cartesian)."""
    import numpy as np
    K = w.probes
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    op = pico.Operator(inp["smaps"], mask=inp.get("mask"), traj=inp.get("traj"), noise_cov=inp["noise_cov"],
                       lam=w.lam, max_batch=K, power_iters=15, stream=stream.cuda_stream)
    tuning = None if args.no_autotune else op.autotune(cache=tune_cache)
    if solver != "global":
        op.set_solver(solver)
    maps = [torch.zeros((w.ny, w.nx), dtype=torch.float64, device=dev) for _ in range(4)]
    s, ss, ps, pss = maps

    def step(i):
        begin = (i * world + rank) * K
        pico.pico_variance_map(op.ctx, SEED_PICO, begin, K, pico.PICO_PROBE_PHASE, w.max_iter, 0.0, s, ss, False)
        pico.pico_pmr(op.ctx, SEED_PMR, begin, K, w.sigma, w.max_iter, 0.0, ps, pss, False)
        if world > 1:   # this step's maps over all ranks' probes: the one exchange per step
            pico.reduce_running_sums(maps)

    total_ms, per_step, clk, launches, prof = timed_steps(step, steps, warmup, torch, dist, world, stream, local,
                                                          [op.ctx], pico)
    op.sync()
    solves = 2 * K * steps * world
    value = solves / (total_ms / 1e3)
    (norm_ms, norm_n), (upd_ms, _), (pmr_ms, _), (acc_ms, _) = prof
    avg_norm_s = norm_ms / max(norm_n, 1) / 1e3
    gram_on = op.info["normal_op"] == 1 and K >= op.tuning["gram_min_batch"]
    if solver == "columns" and op.info["normal_op"] == 1:
        persist = persist_rows(w.ny) > 0 and os.environ.get("PICO_COLCG_PERSIST", "1") != "0" and \
            os.environ.get("PICO_GRAM_TF32", "0") == "0"
        roof = persist_roofline(w, K, avg_norm_s, norm_n) if persist else colcg_roofline(w, K, avg_norm_s, norm_n)
    elif op.info["normal_op"] == 3:
        roof = onchip_roofline(w, K, avg_norm_s, norm_n, solver)
    else:
        roof = gram_roofline(w, K, avg_norm_s, norm_n) if gram_on else fft_roofline(w, K, avg_norm_s, norm_n)
    nsamp = K * world
    line = {
        "value": value, "unit": UNIT, "steps": steps, "warmup": warmup, "ms_per_step": total_ms / steps,
        "config": dict(arm_config(w, world), cg_solver=solver), "roofline": roof,
        "kernel_ms_in_timed_region": {"normal_op_ms": norm_ms, "cg_vector_ms": upd_ms, "pmr_adjoint_ms": pmr_ms,
                                      "accumulate_ms": acc_ms},
        "gpu_launches": launches,
        "tuning": {"applied": op.tuning, "autotuned": tuning is not None,
                   "us_per_image_iteration": getattr(op, "autotune_table", None)},
        "clocks": clk,
        "step_ms": {"p50": statistics.median(per_step), "max": max(per_step)},
        "last_step_maps": {"pico_mean_variance": float(s.mean() / nsamp), "pmr_mean_variance":
                           float(ps.mean() / nsamp), "samples_per_map": nsamp},
    }
    if primary and not args.no_e2e:
        S_h = np.ascontiguousarray(inp["smaps"])
        m_h = inp["mask"] if w.kind == "cartesian" else inp["traj"]
        C_h = inp["noise_cov"]
        out_h = np.empty((2, w.ny, w.nx), dtype=np.float64)
        e2e_steps = max(2, min(steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            kw = {"mask": m_h} if w.kind == "cartesian" else {"traj": m_h}
            op2 = pico.Operator(S_h, noise_cov=C_h, lam=w.lam, max_batch=K, power_iters=15,
                                stream=stream.cuda_stream, **kw)
            if tuning is not None:
                op2.autotune(cache=tune_cache)   # a cache hit: the tuning measured above
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
                       "includes": "pico_init (upload, whitening, power method, workspace) + tuning from the "
                                   "JSON cache + maps + read-back"}
    return line, op


def t1pct_linear(op, w, torch, pico, spiral_subset, arms=None):
    """Time to a 1 %-NRMSE standard-deviation map.  Cartesian: the ablation's
    three probe families and PMR against the exact diagonal (arms="pico_pmr":
    PICO and PMR only).  Spiral: PICO and PMR with 30 fixed CG iterations and
    with the paper's solver rule (at most 100 iterations, relative residual
    1e-2, Sec. 3.2.2)."""
    K = w.probes
    if w.kind == "cartesian":
        sel = (("pico", pico.PICO_PROBE_PHASE), ("pmr", None)) if arms == "pico_pmr" else None
        t1 = measure_time_to_1pct(op, w, torch, pico, step=10, arms=sel)
        names = ("pico", "pmr")
    else:
        arms = (("pico", pico.PICO_PROBE_PHASE), ("pmr", None))
        t1 = measure_time_to_1pct(op, w, torch, pico, step=50, arms=arms, subset=spiral_subset)
        t1["paper_cg_rule"] = measure_time_to_1pct(op, w, torch, pico, step=50, cg=(100, 1e-2), arms=arms,
                                                   subset=spiral_subset)
        names = ("pico", "pmr")
    # device seconds per probe and per replica at the bench's batch size, timed separately
    s = torch.zeros((w.ny, w.nx), dtype=torch.float64, device="cuda")
    ss, ps, pss = torch.zeros_like(s), torch.zeros_like(s), torch.zeros_like(s)
    stream = torch.cuda.current_stream()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    pico.pico_variance_map(op.ctx, SEED_PICO, 0, K, pico.PICO_PROBE_PHASE, w.max_iter, 0.0, s, ss, True)
    e1.record(stream)
    pico.pico_pmr(op.ctx, SEED_PMR, 0, K, w.sigma, w.max_iter, 0.0, ps, pss, True)
    e2.record(stream)
    torch.cuda.synchronize()
    per = {"pico": e0.elapsed_time(e1) / 1e3 / K, "pmr": e1.elapsed_time(e2) / 1e3 / K}
    for name in names:
        t1[name]["seconds_per_sample_batched"] = per[name]
        if t1[name].get("N"):
            t1[name]["seconds_at_batched_rate"] = t1[name]["N"] * per[name]
    return t1


def measure_time_to_1pct_cs(op, w, torch, pico, sigma, nref, step=10, max_n=20000):
    """Time to a 1 %-NRMSE standard-deviation map for the nonlinear CS
    reconstruction (Sec. 3.2.3 protocol): PICO and PMR converge to slightly
    different limits, so each is compared with its own high-count reference
    (nref samples under another seed).  The reference's own sampling error
    is estimated from its running sums (delta method, Var(sqrt(m)) ~ Var(m) /
    4m) and reported; `N_corrected` is the first N whose squared NRMSE minus
    that floor is <= 1e-4."""
    ny, nx = w.ny, w.nx
    K = w.probes
    out = {"protocol": f"method-specific references of {nref} samples, N in steps of {step}",
           "threshold": 0.01, "nrmse_on": "std maps over the reference's support (std >= 10% of max)"}

    def run(name, seed, begin, n, s, ss):
        if name == "pico":
            pico.pico_cs_variance_map(op.ctx, seed, begin, n, pico.PICO_PROBE_PHASE, s, ss, True)
        else:
            pico.pico_cs_pmr(op.ctx, seed, begin, n, sigma, s, ss, True)

    for name in ("pico", "pmr"):
        rs = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
        rss = torch.zeros_like(rs)
        t0 = time.perf_counter()
        for b in range(0, nref, K):
            run(name, SEED_PICO + 101 if name == "pico" else SEED_PMR + 101, b, min(K, nref - b), rs, rss)
        torch.cuda.synchronize()
        t_ref = time.perf_counter() - t0
        m = (rs / nref).clamp_min(0)
        var_m = ((rss / nref - m * m).clamp_min(0) / (nref - 1))
        ref_std = m.sqrt()
        sup = ref_std >= 0.1 * ref_std.max()
        nref_norm = torch.linalg.vector_norm(ref_std[sup])
        floor2 = float((var_m[sup] / (4 * m[sup])).sum() / (nref_norm ** 2))
        s = torch.zeros_like(rs)
        ss = torch.zeros_like(rs)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        elapsed, n, hit, hitc, curve = 0.0, 0, None, None, []
        while n < max_n:
            ev0.record()
            run(name, SEED_PICO + 1 if name == "pico" else SEED_PMR + 1, n, step, s, ss)
            ev1.record()
            torch.cuda.synchronize()
            elapsed += ev0.elapsed_time(ev1) / 1e3
            n += step
            err = float(torch.linalg.vector_norm(((s / n).clamp_min(0).sqrt() - ref_std)[sup]) / nref_norm)
            if n in (10, 50, 100, 200, 500, 1000, 2000, 5000, 10000):
                curve.append((n, round(err, 5)))
            if hitc is None and err * err - floor2 <= 1e-4:
                hitc = (n, elapsed, err)
            if err <= 0.01:
                hit = (n, elapsed, err)
                break
        out[name] = {"reference_seconds": t_ref, "reference_self_nrmse": floor2 ** 0.5, "curve": curve,
                     "support_fraction": float(sup.double().mean())}
        if hit:
            out[name].update({"N": hit[0], "seconds": hit[1], "nrmse": hit[2]})
        else:
            out[name].update({"N": None, "nrmse_at_max": err, "max_n": max_n})
        if hitc:
            out[name].update({"N_corrected": hitc[0], "seconds_corrected": hitc[1]})
    return out


def bench_cs(args, w, inp, pico, torch, dist, world, rank, local, steps, warmup, primary):
    """Nonlinear CS workload: one step = the L1-wavelet FISTA reconstruction
    (the linearisation point), K Jacobian-probe products J(J^T v) accumulated
    into the PICO map (Sec. 2.2.5) and K PMR replicas (FISTA reruns on b + n_i,
    Sec. 3.2.3).  ``value`` counts probes + replicas per second."""
    import numpy as np
    K = w.probes
    levels, iters = w.extra["levels"], w.max_iter
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    op = pico.Operator(inp["smaps"], mask=inp["mask"], noise_cov=inp["noise_cov"], max_batch=K, power_iters=15,
                       stream=stream.cuda_stream)
    # data b = A x0 (whitened), weight and PMR noise level (set-up, outside the timed region)
    x0 = torch.from_numpy(np.ascontiguousarray(inp["phantom"], dtype=np.complex64)).to(dev)
    b = op.forward(x0.reshape(1, w.ny, w.nx))[0].contiguous()
    ahb = op.adjoint(b.reshape((1,) + tuple(b.shape)))
    coef = torch.empty_like(ahb)
    pico.pico_wavelet(op.ctx, ahb, coef, levels)
    lam = w.extra["lam_l1_rel"] * float(coef.abs().max())
    m = torch.from_numpy(inp["mask"].astype(bool)).to(dev)
    sigma = cs_sigma(w, float((b.abs() ** 2)[:, m].mean().sqrt()))
    x = torch.empty((w.ny, w.nx), dtype=torch.complex64, device=dev)
    maps = [torch.zeros((w.ny, w.nx), dtype=torch.float64, device=dev) for _ in range(4)]
    s, ss, ps, pss = maps

    def step(i):
        begin = (i * world + rank) * K
        pico.pico_cs_recon(op.ctx, b, lam, iters, levels, x)
        pico.pico_cs_variance_map(op.ctx, SEED_PICO, begin, K, pico.PICO_PROBE_PHASE, s, ss, False)
        pico.pico_cs_pmr(op.ctx, SEED_PMR, begin, K, sigma, ps, pss, False)
        if world > 1:
            pico.reduce_running_sums(maps)

    total_ms, per_step, clk, launches, prof = timed_steps(step, steps, warmup, torch, dist, world, stream, local,
                                                          [op.ctx], pico)
    op.sync()
    value = 2 * K * steps * world / (total_ms / 1e3)
    norm_ms, norm_n = prof[0]
    # images through the normal operator per step: the reconstruction runs on
    # one image (iters launches); Jacobian PICO (VJP + M g + JVP) and CS PMR
    # (FISTA) run on K images (3 iters + 1 launches)
    images = steps * (iters + (3 * iters + 1) * K)
    avg_norm_s = norm_ms / max(norm_n, 1) / 1e3
    achieved = images * flops_2d_normal(w) / (norm_ms / 1e3) / 1e12
    peak = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    img = w.ny * w.nx * 8
    mp = measured_peaks()
    hbm = images * (2 * img + 4 * w.nc * img) / (norm_ms / 1e3) / 1e9
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None,
            "kernel": "k_toep_rows_fwd + k_toep_cols + k_toep_rows_inv (2-D-mask normal operator, no padding)",
            "avg_launch_ms": avg_norm_s * 1e3, "launches": norm_n, "images": images,
            "peak_note": "FP32 FMA peak 152 SM x 128 lanes x 2 x 2070 MHz (nominal max clock); achieved = "
                         "algorithmic flops of every image through the operator / its total time",
            "hbm": {"achieved_GBps_incl_coil_grids": hbm, "peak_GBps": mp["hbm_gbs"], "frac": hbm / mp["hbm_gbs"]}}
    line = {
        "value": value, "unit": UNIT, "steps": steps, "warmup": warmup, "ms_per_step": total_ms / steps,
        "config": dict(arm_config(w, world), lambda_l1=lam, pmr_sigma=sigma),
        "roofline": roof,
        "kernel_ms_in_timed_region": {"normal_op_ms": norm_ms, "cg_vector_ms": prof[1][0],
                                      "noise_adjoint_ms": prof[2][0], "elementwise_and_dwt_ms": prof[3][0]},
        "gpu_launches": launches, "clocks": clk,
        "step_ms": {"p50": statistics.median(per_step), "max": max(per_step)},
    }
    if primary and not args.no_e2e:
        S_h, m_h, C_h = np.ascontiguousarray(inp["smaps"]), inp["mask"], inp["noise_cov"]
        b_h = b.cpu().pin_memory()
        out_h = np.empty((2, w.ny, w.nx), dtype=np.float64)
        e2e_steps = max(2, min(steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            op2 = pico.Operator(S_h, mask=m_h, noise_cov=C_h, max_batch=K, power_iters=15, stream=stream.cuda_stream)
            bd = b_h.to(dev, non_blocking=True)
            xd = torch.empty((w.ny, w.nx), dtype=torch.complex64, device=dev)
            a = torch.empty((w.ny, w.nx), dtype=torch.float64, device=dev)
            c = torch.empty_like(a)
            begin = (i * world + rank) * K
            pico.pico_cs_recon(op2.ctx, bd, lam, iters, levels, xd)
            pico.pico_cs_variance_map(op2.ctx, SEED_PICO, begin, K, pico.PICO_PROBE_PHASE, a)
            pico.pico_cs_pmr(op2.ctx, SEED_PMR, begin, K, sigma, c)
            out_h[0] = a.cpu().numpy()
            out_h[1] = c.cpu().numpy()
            op2.close()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([dt], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        line["e2e"] = {"value": 2 * K * e2e_steps * world / dt, "unit": UNIT,
                       "h2d_bytes_per_step": int(S_h.nbytes + m_h.nbytes + C_h.nbytes + b_h.numel() * 8),
                       "d2h_bytes_per_step": int(out_h.nbytes), "steps": e2e_steps,
                       "includes": "pico_init (upload, whitening, power method) + data upload + reconstruction "
                                   "+ both maps + read-back"}
    if primary and rank == 0 and world == 1 and args.t1pct_cs > 0:
        line["time_to_1pct"] = measure_time_to_1pct_cs(op, w, torch, pico, sigma, args.t1pct_cs)
    op.close()
    return line


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    maybe_relaunch(args)
    import numpy as np  # noqa: F401
    import torch
    import torch.distributed as dist

    import paper_2605_09590_gb300 as pico
    from paper_2605_09590_gb300 import build as pico_build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.device_count() < (local + 1):
        sys.exit(f"bench.py: rank {rank} needs GPU {local}, {torch.cuda.device_count()} visible")
    # the CPU baseline's process pool is spawned before the first GPU call
    cpu_pool = None
    w, inp = workload(args.workload, args.probes)
    if rank == 0 and world == 1 and not args.no_cpu and w.kind == "cartesian":
        cpu_pool = OraclePool(w.name)
    torch.cuda.set_device(local)
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        pico_build.build()
    if world > 1:
        dist.barrier()
    pico.load_library()

    tune_cache = os.environ.get("PICO_TUNE_CACHE") or os.path.join(
        tempfile.gettempdir(), "pico_tune_%d_%d.json" % (os.getpid(), rank))
    if not os.environ.get("PICO_TUNE_CACHE"):
        import atexit
        atexit.register(lambda: os.path.exists(tune_cache) and os.remove(tune_cache))

    if w.kind == "cs":
        sub = bench_cs(args, w, inp, pico, torch, dist, world, rank, local, args.steps, args.warmup, True)
        op = None
    else:
        sub, op = bench_linear(args, w, inp, pico, torch, dist, world, rank, local, args.steps, args.warmup,
                               True, tune_cache, solver=args.solver)
    line = {"metric": METRIC, "n_gpus": world, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64", "data": "synthetic"}
    line.update(sub)
    line["config"] = sub["config"]

    if op is not None and rank == 0 and world == 1 and not args.no_t1pct and (
            w.kind == "cartesian" or args.t1pct_spiral):
        line["time_to_1pct"] = t1pct_linear(op, w, torch, pico, spiral_subset=0)
    colcg_ok = op is not None and w.kind == "cartesian" and args.solver == "global" and (
        op.info["normal_op"] == 1 or w.ny in (32, 64, 96))
    if op is not None:
        op.close()
    if colcg_ok and not args.no_extra:
        # the same step with CG run per readout column (same fixed point, other iterates)
        col, cop = bench_linear(args, w, inp, pico, torch, dist, world, rank, local, args.steps, args.warmup,
                                False, tune_cache, solver="columns")
        if rank == 0 and world == 1 and not args.no_t1pct:
            col["time_to_1pct"] = t1pct_linear(cop, w, torch, pico, spiral_subset=0, arms="pico_pmr")
        cop.close()
        line["column_cg"] = col

    if rank == 0 and world == 1 and not args.no_extra and args.workload == "knee320_r2":
        ws, inps = workload("spiral240_r2")
        spi, sop = bench_linear(args, ws, inps, pico, torch, dist, 1, 0, local, 3, 2, False, tune_cache)
        if not args.no_t1pct:
            spi["time_to_1pct"] = t1pct_linear(sop, ws, torch, pico, spiral_subset=2304)
        sop.close()
        line["spiral240_r2"] = spi
        wc, inpc = workload("cs320_r2")
        line["cs320_r2"] = bench_cs(args, wc, inpc, pico, torch, dist, 1, 0, local, 3, 1, False)
        if args.serving > 0:
            line["serving"] = run_serving(pico, args.serving, loads=(args.serving_load,))

    if cpu_pool is not None:
        vals = []
        for _ in range(2):
            v, dt, procs = cpu_pool.step()
            vals.append((v, dt, procs))
        cpu_pool.close()
        v = sum(a * b for a, b, _ in vals) / sum(b for _, b, _ in vals)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cpu_pool.cores, "kind": "oracle",
                                "sample": f"2 rounds of one PICO probe + one PMR replica ({w.max_iter} CG iterations "
                                          f"each) per core, {cpu_pool.cores} single-threaded FP64 NumPy oracle "
                                          f"processes ({vals[-1][2]} took work), {sum(b for _, b, _ in vals):.1f} s"}
    elif rank == 0 and world == 1 and not args.no_cpu:
        v, dt, desc = oracle_sample(w, inp)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{desc}, {dt:.1f} s, FP64 NumPy on one core"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
