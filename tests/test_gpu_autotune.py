"""GPU tests of the run-time tuning (pico_get_tuning / pico_set_tuning / pico_autotune).

Tuning changes launch shapes only: the operator, CG and maps must keep
agreeing with the FP64 oracle and with the untuned context, the autotuner's
choices must be consistent with its own measurements, and the JSON cache must
reproduce a tuning without measuring again.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import ops as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_09590_gb300 as pico  # noqa: E402
from paper_2605_09590_gb300 import build as pico_build  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    pico_build.build()
    pico.load_library()


def cart(ny=160, nx=32, nc=4, seed=3, max_batch=128):
    S = synth.coil_maps(ny, nx, nc, seed)
    cov = synth.noise_cov(nc, seed)
    mask = synth.mask_pe(ny, 2, 8)
    return S, cov, mask, pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=max_batch)


def test_set_tuning_validates_and_round_trips():
    _, _, _, op = cart()
    t0 = op.tuning
    assert t0["gram_kc"] == 16 and t0["gram_a_tmem"] == 0 and t0["probe_batch"] == 0
    for bad in ({"gram_kc": 12}, {"gram_a_tmem": 2}, {"probe_batch": 129}, {"probe_batch": -1},
                {"gram_min_batch": -3}):
        with pytest.raises(pico.PicoError) as e:
            op.set_tuning(**bad)
        assert e.value.status == pico.PICO_E_INVALID
        assert op.tuning == t0
    op.set_tuning(gram_min_batch=32, probe_batch=48)
    assert op.tuning["gram_min_batch"] == 32 and op.tuning["probe_batch"] == 48


def test_gram_chunk_change_rebuilds_the_operator():
    S, cov, mask, op = cart()
    oop = O.Operator(S, cov, mask=mask)
    g = np.random.default_rng(0)
    x = (g.standard_normal((70, 160, 32)) + 1j * g.standard_normal((70, 160, 32))).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    y16 = op.apply_normal(xd).cpu().numpy()
    op.set_tuning(gram_kc=8)
    y8 = op.apply_normal(xd).cpu().numpy()
    for b in (0, 69):
        want = oop.normal(x[b].astype(np.complex128))
        for y in (y16, y8):
            assert np.linalg.norm(y[b] - want) / np.linalg.norm(want) < 1e-5
    # kc = 16 runs the FP16 head + remainder split, kc = 8 the TF32 split: the same
    # ~22 significant bits per product, rounded differently
    assert np.abs(y8 - y16).max() / np.abs(y16).max() < 1e-5


def test_autotune_choices_follow_its_measurements():
    _, _, _, op = cart()
    tuning, table = pico.pico_autotune(op.ctx, 3)
    assert set(table) == {"fft", "gram16", "gram16_tmem", "gram8"}
    batches = sorted(table["fft"])
    assert batches == [16, 32, 64, 128]
    assert all(v > 0 for row in table.values() for v in row.values())
    top = batches[-1]
    best = min(("gram16", "gram16_tmem", "gram8"), key=lambda k: table[k][top])
    assert (tuning["gram_kc"], tuning["gram_a_tmem"]) == {"gram16": (16, 0), "gram16_tmem": (16, 1),
                                                          "gram8": (8, 0)}[best]
    gmin = tuning["gram_min_batch"]
    for b in batches:
        if b >= gmin:
            assert table[best][b] <= table["fft"][b]
    assert tuning["probe_batch"] == 0 or tuning["probe_batch"] in batches
    assert op.tuning == tuning
    assert pico.pico_sync(op.ctx) is None


def test_tuned_maps_agree_with_untuned_maps():
    S, cov, mask, op = cart(max_batch=128)
    ref_s, _ = op.variance_sums(11, 96, 30, 0.0)
    ref_p, _ = op.pmr_sums(12, 40, 1e-2, 30)
    op.autotune(iters=3)
    for t in (op.tuning, dict(op.tuning, probe_batch=32, gram_min_batch=64)):
        op.set_tuning(**t)
        s, _ = op.variance_sums(11, 96, 30, 0.0)
        p, _ = op.pmr_sums(12, 40, 1e-2, 30)
        assert ((s - ref_s).abs().max() / ref_s.abs().max()).item() < 1e-5
        assert ((p - ref_p).abs().max() / ref_p.abs().max()).item() < 1e-5


def test_json_cache_reuses_a_tuning(tmp_path):
    path = str(tmp_path / "tune.json")
    _, _, _, op = cart(max_batch=64)
    t1 = op.autotune(cache=path, iters=2)
    db = json.load(open(path))
    assert len(db) == 1
    (entry,) = db.values()
    assert entry["tuning"] == t1
    # a second context of the same operator takes the stored tuning as is
    _, _, _, op2 = cart(max_batch=64)
    op2.set_tuning(probe_batch=16)
    t2 = op2.autotune(cache=path)
    assert t2 == t1 and op2.tuning == t1
    assert os.path.getsize(path) > 0


def test_autotune_spiral_context_picks_a_batch():
    n, nc = 64, 6
    S = synth.coil_maps(n, n, nc, 3)
    traj = synth.spiral_traj(n, 16, 512, 2)
    op = pico.Operator(S, traj=traj, lam=0.1, power_iters=0, max_batch=64)
    tuning, table = pico.pico_autotune(op.ctx, 2)
    assert set(table) == {"fft"} and sorted(table["fft"]) == [16, 32, 64]
    assert tuning["probe_batch"] in (0, 16, 32)
    s_tuned, _ = op.variance_sums(5, 40, 10, 0.0)
    op.set_tuning(probe_batch=0)
    s_full, _ = op.variance_sums(5, 40, 10, 0.0)
    # the Toeplitz operator treats every image alike, whatever the batch
    assert torch.equal(s_tuned, s_full)
