"""The benchmark's roofline arithmetic, on the CPU.

The bench line reports the dominant kernel's algorithmic bytes (or flops) per
launch over its CUDA-event time against a measured peak.  These tests pin the
per-unit figures to their definitions written out by hand: four images of
8-byte voxels per image and launch (r and p_old read, p and q written) plus
one pass over the operator's data, the Toeplitz passes' coil half-grids, and
the FFT flop counts 5 L log2 L per transform.
"""
import math

import pytest

import bench
import synth


def test_cartesian_normal_operator_bytes():
    w = synth.WORKLOADS["knee320_r2"]
    image = 320 * 320 * 8
    assert image == 819_200
    # 256 images x (read r, p_old; write p, q) + the 15 whitened coil maps once
    assert bench.alg_bytes_normal(w, 256) == 256 * 4 * image + 15 * image == 851_148_800


def test_spiral_normal_operator_bytes():
    w = synth.WORKLOADS["spiral240_r2"]
    image = 240 * 240 * 8
    half_grid = 240 * 480 * 8             # one coil's n x 2n complex64 grid between the passes
    that = 480 * 480 * 4                  # the real Toeplitz kernel, float32
    per_image = 4 * image + 4 * 20 * half_grid
    assert bench.alg_bytes_normal(w, 256) == 256 * per_image + 20 * image + that == 19_356_364_800


def test_fft_flop_counts():
    knee = synth.WORKLOADS["knee320_r2"]
    # per coil and readout column a forward and an inverse 320-point FFT plus 16 flops per sample
    expect = 15 * 320 * (2 * 5 * 320 * math.log2(320) + 16 * 320)
    assert bench.flops_per_probe(knee) == pytest.approx(expect, rel=1e-12)
    assert 152.0e6 < expect < 152.6e6
    sp = synth.WORKLOADS["spiral240_r2"]
    n, L = 240, 480
    # per coil: n row FFTs, 2L column FFTs (forward and inverse), n inverse row FFTs of length L
    expect = 20 * ((n + 2 * L + n) * 5 * L * math.log2(L) + 16 * n * n + 2 * L * L)
    assert bench.flops_per_probe(sp) == pytest.approx(expect, rel=1e-12)
    assert 643.0e6 < expect < 643.6e6


def test_measured_traffic_is_keyed_by_the_kernel_sources(monkeypatch):
    w = synth.WORKLOADS["knee320_r2"]
    traffic, dig = bench.traffic_of(w, 256, "gram", bench.GRAM_FILES)
    assert len(dig) == 16
    if traffic is not None:
        # the capture moved the algorithmic bytes plus the FP16 G planes (262 MB), no re-reads
        ratio = traffic / bench.alg_bytes_normal(w, 256)
        assert 1.2 < ratio < 1.35
    # a source digest without a capture reports no traffic
    monkeypatch.setattr(bench, "kernel_digest", lambda *names: "0" * 16)
    assert bench.traffic_of(w, 256, "gram", bench.GRAM_FILES) == (None, "0" * 16)


def test_gram_roofline_fraction(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 6784.5, "bf16_tflops": 1908.5,
                                                           "bf16_tflops_sustained": 1705.9})
    w = synth.WORKLOADS["knee320_r2"]
    r = bench.gram_roofline(w, 256, 275e-6, 300)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(851_148_800 / 275e-6 / 1e9, rel=1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / 6784.5, rel=1e-12)
    # dense-equivalent tensor view: nx products of (ny x ny) by (ny x K), 8 flops per complex MAC, 3 FP16 terms
    cplx = 8.0 * 320 * 320 * 320 * 256
    assert r["tensor_dense_equivalent"]["achieved_TFLOPs"] == pytest.approx(3 * cplx / 275e-6 / 1e12, rel=1e-12)
