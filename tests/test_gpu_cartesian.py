"""GPU parity of the Cartesian hot path against the CPU oracle (through the C ABI).

Tolerances.  The CUDA path keeps vectors in complex64 and accumulates inner
products in FP64; the oracle is FP64 throughout.  Single operator
applications agree to float32 rounding of an FFT pair per coil (<= 2e-6
relative in norm).  After 30 CG iterations the per-voxel difference of the
variance estimate, relative to the exact diagonal Sigma_kk, must stay below
1e-4 (the stated parity bound for identical probe seeds).
"""
import numpy as np
import pytest

import synth
from oracle import ops as O
from oracle import pico as OP
from oracle import rng as ORNG
from oracle import solvers as OS

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


@pytest.fixture(autouse=True)
def _column_fft_path(monkeypatch):
    # this module covers the column-FFT normal operator; the tensor-core Gram
    # operator (the default for ny >= 128) has its own module
    monkeypatch.setenv("PICO_NORMAL_OP", "fft")


def case(ny, nx, nc, R=2, acs=0, corr=False, seed=0):
    S = synth.coil_maps(ny, nx, nc, seed)
    cov = synth.noise_cov(nc, seed) if corr else None
    mask = synth.mask_pe(ny, R, acs)
    return S, cov, mask


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def rand_imgs(nb, ny, nx, seed):
    g = np.random.default_rng(seed)
    return (g.standard_normal((nb, ny, nx)) + 1j * g.standard_normal((nb, ny, nx))).astype(np.complex64)


# (ny, nx): several column tiles and a ragged last tile; several FFT splits
SHAPES = [(64, 64), (80, 40), (96, 72), (120, 33), (128, 20), (320, 48)]


@pytest.mark.parametrize("ny,nx", SHAPES)
@pytest.mark.parametrize("lam", [0.0, 0.05])
def test_apply_normal_matches_oracle(ny, nx, lam):
    S, cov, mask = case(ny, nx, 5, R=2, acs=4, corr=True, seed=ny + nx)
    op = pico.Operator(S, mask=mask, noise_cov=cov, lam=lam, power_iters=0, max_batch=4)
    oop = O.Operator(S, cov, mask=mask)
    x = rand_imgs(3, ny, nx, 1)
    y = op.apply_normal(to_dev(x)).cpu().numpy()
    for b in range(3):
        want = oop.normal(x[b].astype(np.complex128), lam)
        err = np.linalg.norm(y[b] - want) / np.linalg.norm(want)
        assert err < 2e-6, err


def test_apply_normal_is_hermitian_psd():
    S, cov, mask = case(96, 64, 6, R=3, acs=8, corr=True, seed=3)
    op = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0)
    x, z = rand_imgs(1, 96, 64, 2), rand_imgs(1, 96, 64, 3)
    Mx = op.apply_normal(to_dev(x)).cpu().numpy().astype(np.complex128)
    Mz = op.apply_normal(to_dev(z)).cpu().numpy().astype(np.complex128)
    a, b = np.vdot(z, Mx), np.vdot(Mz, x)
    assert abs(a - b) / abs(a) < 1e-5
    assert np.vdot(x, Mx).real > 0


@pytest.mark.parametrize("ny,nx,nc,acs,corr,lam", [(64, 64, 8, 0, False, 0.0), (96, 56, 6, 8, True, 0.0),
                                                   (80, 48, 4, 4, True, 0.1)])
def test_cg_fixed_iterations_matches_oracle(ny, nx, nc, acs, corr, lam):
    S, cov, mask = case(ny, nx, nc, acs=acs, corr=corr, seed=7)
    op = pico.Operator(S, mask=mask, noise_cov=cov, lam=lam, power_iters=0, max_batch=4)
    oop = O.Operator(S, cov, mask=mask)
    rhs = rand_imgs(5, ny, nx, 11)                 # 5 systems: two batches of 4 + ragged
    x, iters, relres = op.cg(to_dev(rhs), 30, 0.0, stats=True)
    x = x.cpu().numpy()
    assert np.all(iters == 30)
    for b in range(5):
        want, it, rr = OS.cg(lambda z: oop.normal(z, lam), rhs[b].astype(np.complex128), 30, 0.0)
        err = np.linalg.norm(x[b] - want) / np.linalg.norm(want)
        assert err < 1e-4, err
        assert abs(relres[b] - rr) <= 1e-3 * rr + 1e-6


def test_cg_stopping_rule_matches_oracle():
    S, cov, mask = case(64, 48, 6, acs=4, corr=True, seed=9)
    op = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=8)
    oop = O.Operator(S, cov, mask=mask)
    rhs = rand_imgs(3, 64, 48, 5)
    _, iters, relres = op.cg(to_dev(rhs), 100, 1e-3, stats=True)
    for b in range(3):
        _, it, rr = OS.cg(lambda z: oop.normal(z), rhs[b].astype(np.complex128), 100, 1e-3)
        assert abs(int(iters[b]) - it) <= 1, (iters[b], it)
        assert relres[b] <= 1e-3


def test_cg_stopping_rule_after_other_solves_on_the_same_context():
    # earlier fixed-iteration solves leave large r^H r partials in the context's
    # per-iteration tables; a later tolerance-stopped solve must not read them
    S, cov, mask = case(64, 48, 6, acs=4, corr=True, seed=10)
    op = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=8)
    oop = O.Operator(S, cov, mask=mask)
    op.cg(to_dev(rand_imgs(8, 64, 48, 1) * 1e3), 60, 0.0)
    rhs = np.zeros((3, 64, 48), dtype=np.complex64)
    for b in range(3):
        rhs[b, 5 + 7 * b, :] = 1.0                      # structured right-hand sides, converge fast
    x, iters, relres = op.cg(to_dev(rhs), 100, 1e-6, stats=True)
    x = x.cpu().numpy()
    for b in range(3):
        want, it, _ = OS.cg(lambda z: oop.normal(z), rhs[b].astype(np.complex128), 100, 1e-6)
        assert np.linalg.norm(x[b] - want) / np.linalg.norm(want) < 1e-4
        assert abs(int(iters[b]) - it) <= 1 and relres[b] <= 1e-6


def _pico_sums(op, seed, K, it, kind=pico.PICO_PROBE_PHASE, begin=0):
    s, ss = op.variance_sums(seed, K, it, 0.0, probe_begin=begin, kind=kind)
    return s.cpu().numpy(), ss.cpu().numpy()


@pytest.mark.parametrize("kind", [ORNG.PROBE_PHASE, ORNG.PROBE_RADEMACHER, ORNG.PROBE_GAUSS])
def test_variance_map_same_seed_parity_sense64(kind):
    # 64x64, 8 coils, uniform R=2, no calibration lines, K=32, 30 CG iterations
    S, cov, mask = case(64, 64, 8, R=2, acs=0, seed=0)
    op = pico.Operator(S, mask=mask, power_iters=0, max_batch=32)
    oop = O.Operator(S, None, mask=mask)
    K = 32 if kind == ORNG.PROBE_PHASE else 8
    s, ss = _pico_sums(op, 1234, K, 30, kind)
    so, sso = OP.pico(oop, 1234, 0, K, 0.0, 30, 0.0, kind=kind)
    d, _, _ = OP.column_exact(oop)
    rel = np.abs(s / K - so / K) / d
    assert rel.max() < 1e-4, rel.max()


def test_variance_map_band_and_closed_form_sense64():
    S, _, mask = case(64, 64, 8, R=2, acs=0, seed=0)
    op = pico.Operator(S, mask=mask, power_iters=15, max_batch=64)
    oop = O.Operator(S, None, mask=mask)
    K = 256
    s, _ = _pico_sums(op, 99, K, 60)
    var_cf, _, g_cf = OP.sense_closed_form(oop.S, 2)
    _, _, half = OP.column_exact(oop)
    z = (s / K - var_cf) / np.sqrt(half / K + 1e-30)
    assert np.all(np.abs(z) < 6), np.abs(z).max()
    assert np.mean(np.abs(z) > 3) < 0.01
    info = op.info
    lmax = OS.power_method(lambda x: oop.normal(x), (64, 64), 15)
    assert abs(info["lambda_max"] - lmax) / lmax < 1e-5


def test_probe_split_and_resume_are_bitwise_identical():
    S, cov, mask = case(80, 40, 5, acs=4, corr=True, seed=4)
    op = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=8)
    full_s, full_ss = op.variance_sums(5, 20, 20, 0.0)
    s, ss = op.variance_sums(5, 7, 20, 0.0, probe_begin=0)
    op.variance_sums(5, 13, 20, 0.0, probe_begin=7, sum_=s, sumsq=ss)
    assert torch.equal(full_s, s) and torch.equal(full_ss, ss)
    # a different batch size (how probes are grouped on the device) gives the same bits
    op2 = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=3)
    s2, ss2 = op2.variance_sums(5, 20, 20, 0.0)
    assert torch.equal(full_s, s2)


def test_pmr_same_seed_parity():
    S, cov, mask = case(64, 48, 6, R=2, acs=4, corr=True, seed=2)
    op = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=8)
    oop = O.Operator(S, cov, mask=mask)
    N, sigma = 10, 1e-2
    s, _ = op.pmr_sums(21, N, sigma, 30)
    s = s.cpu().numpy()
    so, _ = OP.pmr(oop, 21, 0, N, sigma, 0.0, 30, 0.0)
    d, _, _ = OP.column_exact(oop)
    rel = np.abs(s / N - so / N) / d
    assert rel.max() < 1e-4, rel.max()


def test_pmr_band_against_exact_diagonal():
    S, cov, mask = case(64, 64, 8, R=2, acs=0, seed=0)
    op = pico.Operator(S, mask=mask, power_iters=0, max_batch=64)
    oop = O.Operator(S, None, mask=mask)
    N = 256
    s, _ = op.pmr_sums(3, N, 1.0, 60)
    d, _, _ = OP.column_exact(oop)
    z = (s.cpu().numpy() / N - d) / np.sqrt(d ** 2 / N)
    assert np.all(np.abs(z) < 6)
    assert np.mean(np.abs(z) > 3) < 0.01


def test_full_sampling_one_probe_is_exact():
    S, _, _ = case(64, 64, 8, seed=1)
    mask = np.ones(64, dtype=np.uint8)
    op = pico.Operator(S, mask=mask, power_iters=0)
    s, _ = _pico_sums(op, 3, 1, 10)
    assert np.abs(s - 1.0).max() < 1e-5            # sum |S|^2 = 1 => Sigma = I


def test_finalize_and_gfactor():
    S, _, mask = case(64, 64, 8, R=2, seed=0)
    op = pico.Operator(S, mask=mask, power_iters=0)
    K = 64
    s, ss = op.variance_sums(8, K, 40, 0.0)
    var, se = op.finalize(s, ss, K)
    sn, ssn = s.cpu().numpy(), ss.cpu().numpy()
    assert np.allclose(var.cpu().numpy(), sn / K, rtol=1e-6)
    want_se = np.sqrt(np.maximum(ssn / K - (sn / K) ** 2, 0) / (K - 1))
    assert np.allclose(se.cpu().numpy(), want_se, rtol=1e-5, atol=1e-9)
    ref = torch.full_like(var, 0.5)
    g = torch.empty_like(var)
    pico.pico_gfactor(op.ctx, var, ref, 2.0, g)
    assert np.allclose(g.cpu().numpy(), np.sqrt(var.cpu().numpy() / (2 * 0.5)), rtol=1e-6)


def test_errors_are_reported_not_raised_on_device():
    S, _, mask = case(64, 64, 4)
    with pytest.raises(pico.PicoError) as e:
        pico.Operator(S, mask=mask, hbm_budget=1024)
    assert e.value.status == pico.PICO_E_OOM
    with pytest.raises(pico.PicoError) as e:
        pico.Operator(synth.coil_maps(70, 64, 2, 0), mask=synth.mask_pe(70, 2))
    assert e.value.status == pico.PICO_E_UNSUPPORTED
    op = pico.Operator(S, mask=mask, power_iters=0, max_iter_cap=16)
    s = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(pico.PicoError) as e:
        pico.pico_variance_map(op.ctx, 0, 0, 4, 0, 17, 0.0, s)
    assert e.value.status == pico.PICO_E_INVALID
    with pytest.raises(pico.PicoError):
        pico.pico_variance_map(op.ctx, 0, 0, 4, 7, 10, 0.0, s)


# ---------------------------------------------------------------------------
# full size: 320x320, 15 correlated coils, R=2 + 24 calibration lines, K=256
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def knee():
    w = synth.WORKLOADS["knee320_r2"]
    inp = w.inputs()
    oop = O.Operator(inp["smaps"], inp["noise_cov"], mask=inp["mask"])
    return w, inp, oop


def test_full_size_cg_batch_sampled_parity(knee):
    w, inp, oop = knee
    op = pico.Operator(inp["smaps"], mask=inp["mask"], noise_cov=inp["noise_cov"], power_iters=0,
                       max_batch=w.probes)
    n = w.ny * w.nx
    # the bench's launch shape: one batch of 256 right-hand sides (probe images)
    rhs = np.stack([ORNG.probe(77, i, n).reshape(w.ny, w.nx) for i in range(w.probes)]).astype(np.complex64)
    x = op.cg(to_dev(rhs), w.max_iter, 0.0).cpu().numpy()
    for i in (0, 131, 255):
        want, _, _ = OS.cg(lambda z: oop.normal(z), rhs[i].astype(np.complex128), w.max_iter, 0.0)
        err = np.linalg.norm(x[i] - want) / np.linalg.norm(want)
        assert err < 1e-4, (i, err)


def test_full_size_variance_map_band(knee):
    w, inp, oop = knee
    op = pico.Operator(inp["smaps"], mask=inp["mask"], noise_cov=inp["noise_cov"], max_batch=w.probes)
    s, _ = op.variance_sums(2026, w.probes, w.max_iter, 0.0)
    d, _, half = OP.column_exact(oop)
    K = w.probes
    z = (s.cpu().numpy() / K - d) / np.sqrt(half / K)
    # 30 CG iterations are not fully converged; allow the truncation bias on top of the band
    assert np.mean(np.abs(z) > 4) < 0.01, np.mean(np.abs(z) > 4)
    assert np.abs(s.cpu().numpy() / K - d).max() / d.max() < 0.2


def test_adaptive_stopping_matches_plain_run():
    S, cov, mask = case(64, 64, 8, R=2, acs=4, corr=True, seed=12)
    op = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=16)
    s = torch.empty((64, 64), dtype=torch.float64, device="cuda")
    ss = torch.empty_like(s)
    used, rel = pico.pico_variance_map_adaptive(op.ctx, 9, pico.PICO_PROBE_PHASE, 8, 400, 30, 0.0, 0.02, s, ss)
    assert 8 <= used <= 400 and used % 8 == 0 and rel <= 0.02
    s2, ss2 = op.variance_sums(9, used, 30, 0.0)
    assert torch.equal(s, s2) and torch.equal(ss, ss2)       # same probes, same order, same bits
    sn, ssn = s2.cpu().numpy(), ss2.cpu().numpy()
    m = sn / used
    se = np.sqrt(np.maximum(ssn / used - m * m, 0) / (used - 1))
    assert abs(np.linalg.norm(se) / np.linalg.norm(m) - rel) < 1e-9
    # one chunk fewer would not have met the target
    if used > 8:
        s3, ss3 = op.variance_sums(9, used - 8, 30, 0.0)
        n3 = used - 8
        m3 = s3.cpu().numpy() / n3
        se3 = np.sqrt(np.maximum(ss3.cpu().numpy() / n3 - m3 * m3, 0) / (n3 - 1))
        assert np.linalg.norm(se3) / np.linalg.norm(m3) > 0.02
