"""Serving runtime: requests of uneven size admitted as they arrive; each
result is bit-identical to the same request computed alone."""
import threading

import numpy as np
import pytest

import synth

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


def requests():
    out = []
    S = synth.coil_maps(64, 64, 8, 1)
    out.append(dict(smaps=S, mask=synth.mask_pe(64, 2, 0), seed=11, nprobes=40, max_iter=20))
    S = synth.coil_maps(96, 80, 6, 2)
    out.append(dict(smaps=S, mask=synth.mask_pe(96, 2, 8), noise_cov=synth.noise_cov(6, 2), seed=12, nprobes=24,
                    max_iter=25, pmr_reps=12, pmr_sigma=0.5))
    S = synth.coil_maps(64, 64, 5, 3)
    out.append(dict(smaps=S, traj=synth.spiral_traj(64, 16, 256, 2), lam=0.1, seed=13, nprobes=10, max_iter=15,
                    pmr_reps=6, pmr_sigma=1e-2))
    S = synth.coil_maps(320, 320, 15, 4)
    out.append(dict(smaps=S, mask=synth.mask_pe(320, 2, 24), noise_cov=synth.noise_cov(15, 4), seed=14,
                    nprobes=64, max_iter=30))
    S = synth.coil_maps(64, 64, 8, 1)
    out.append(dict(smaps=S, mask=synth.mask_pe(64, 2, 0), seed=15, nprobes=33, max_iter=20, probe_kind=2))
    return out


def alone(r):
    kw = {k: r[k] for k in ("mask", "traj", "noise_cov") if k in r}
    op = pico.Operator(r["smaps"], lam=r.get("lam", 0.0), power_iters=15, max_batch=64, **kw)
    s, _ = op.variance_sums(r["seed"], r["nprobes"], r["max_iter"], 0.0, kind=r.get("probe_kind", 0))
    var = s.cpu().numpy() / r["nprobes"]
    pmr = None
    if r.get("pmr_reps"):
        p, _ = op.pmr_sums(r["seed"], r["pmr_reps"], r["pmr_sigma"], r["max_iter"])
        pmr = p.cpu().numpy() / r["pmr_reps"]
    op.close()
    return var, pmr


def test_mix_equals_alone_bitwise():
    # the server launches `chunk` probes at a time, as the context built alone
    # does with max_batch = chunk: batches of 64+ images of the 320x320 request
    # run on the tensor-core Gram operator, the others on the column-FFT kernel
    reqs = requests()
    sv = pico.Server(max_active=3, chunk=64)
    ids = [None] * len(reqs)

    def submit(i):
        ids[i] = sv.submit(**reqs[i])

    threads = [threading.Thread(target=submit, args=(i,)) for i in range(len(reqs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    got = [sv.wait(i) for i in ids]
    sv.close()
    for r, (var, pmr, info) in zip(reqs, got):
        assert info["status"] == 0 and info["t_done"] >= info["t_admit"] >= info["t_arrival"]
        v0, p0 = alone(r)
        assert np.array_equal(var, v0)
        if p0 is not None:
            assert np.array_equal(pmr, p0)


def test_admission_respects_memory_budget():
    reqs = [r for r in requests() if r["smaps"].shape[1] == 64 and "mask" in r]
    fp = [pico.pico_footprint(r["smaps"], mask=r["mask"], max_batch=64) + 3 * 64 * 64 * 8 for r in reqs]
    budget = int(max(fp) * 1.5)           # one request at a time fits, two do not
    sv = pico.Server(hbm_budget=budget, max_active=4, chunk=8)
    ids = [sv.submit(**r) for r in reqs]
    infos = [sv.wait(i)[2] for i in ids]
    sv.close()
    # admitted in arrival order, each only after the previous one finished
    for a, b in zip(infos, infos[1:]):
        assert b["t_admit"] >= a["t_done"] - 1e-6
    with pytest.raises(pico.PicoError):
        pico.Server(hbm_budget=1000).submit(**reqs[0])


def _cs_request(n=64, nc=8, seed=21):
    """A nonlinear-CS request: Poisson-disc mask, phantom data, weight 1e-2 max|W A^H b|."""
    S = synth.coil_maps(n, n, nc, seed)
    mask = synth.poisson_disc_mask(n, n, 2.0, 12, seed)
    op = pico.Operator(S, mask=mask, power_iters=15, max_batch=8)
    x0 = torch.from_numpy(synth.phantom(n, seed).astype(np.complex64)).cuda().reshape(1, n, n)
    b = op.forward(x0)
    coef = torch.empty_like(x0)
    pico.pico_wavelet(op.ctx, op.adjoint(b), coef, 4)
    lam = 1e-2 * float(coef.abs().max())
    op.close()
    return dict(smaps=S, mask=mask, seed=seed, nprobes=12, pmr_reps=10, pmr_sigma=1e-3,
                cs_data=b[0].cpu().numpy(), cs_lambda=lam, cs_iters=30, cs_levels=4)


def _cs_alone(r, chunk):
    n = r["smaps"].shape[1]
    op = pico.Operator(r["smaps"], mask=r["mask"], power_iters=15, max_batch=chunk)
    x = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    pico.pico_cs_recon(op.ctx, torch.from_numpy(r["cs_data"]).cuda(), r["cs_lambda"], r["cs_iters"], r["cs_levels"],
                       x)
    s = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    ss = torch.zeros_like(s)
    p = torch.zeros_like(s)
    for b in range(0, r["nprobes"], chunk):
        pico.pico_cs_variance_map(op.ctx, r["seed"], b, min(chunk, r["nprobes"] - b), 0, s, ss, b > 0)
    for b in range(0, r["pmr_reps"], chunk):
        pico.pico_cs_pmr(op.ctx, r["seed"], b, min(chunk, r["pmr_reps"] - b), r["pmr_sigma"], p, None, b > 0)
    out = s.cpu().numpy() / r["nprobes"], p.cpu().numpy() / r["pmr_reps"]
    op.close()
    return out


def test_cs_requests_in_the_mix_equal_alone_bitwise():
    cs = _cs_request()
    reqs = [cs, requests()[0], requests()[1]]
    sv = pico.Server(max_active=3, chunk=8)
    ids = [sv.submit(**r) for r in reqs]
    got = [sv.wait(i) for i in ids]
    sv.close()
    var, pmr, info = got[0]
    assert info["status"] == 0
    v0, p0 = _cs_alone(cs, 8)
    assert np.array_equal(var, v0) and np.array_equal(pmr, p0)
    # a 12-probe Jacobian PICO map may dip below zero voxelwise; its mean may not
    assert var.mean() > 0 and np.all(pmr >= 0)
