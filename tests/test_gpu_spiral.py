"""GPU parity of the spiral (non-Cartesian) path against the CPU oracle.

The oracle applies the exact NUDFT; the GPU normal operator is the Toeplitz
embedding of that exact NUDFT (so they agree to float32 rounding), while the
PMR adjoint on the GPU uses Kaiser-Bessel gridding (W = 6, oversampling 2),
whose approximation error is checked separately against the exact adjoint.
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


def small(n=64, nc=6, R=2, nsamp=512, seed=3, corr=False):
    S = synth.coil_maps(n, n, nc, seed)
    traj = synth.spiral_traj(n, 16, nsamp, R)
    cov = synth.noise_cov(nc, seed) if corr else None
    return S, traj, cov


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def rand_imgs(nb, n, seed):
    g = np.random.default_rng(seed)
    return (g.standard_normal((nb, n, n)) + 1j * g.standard_normal((nb, n, n))).astype(np.complex64)


@pytest.mark.parametrize("n,lam", [(64, 0.0), (64, 0.1), (80, 0.1), (96, 0.0)])
def test_toeplitz_normal_matches_exact_nudft(n, lam):
    S, traj, cov = small(n, 5, 2, 384, seed=n, corr=True)
    op = pico.Operator(S, traj=traj, noise_cov=cov, lam=lam, power_iters=0, max_batch=3)
    oop = O.Operator(S, cov, traj=traj)
    x = rand_imgs(3, n, 1)
    y = op.apply_normal(to_dev(x)).cpu().numpy()
    for b in range(3):
        want = oop.normal(x[b].astype(np.complex128), lam)
        err = np.linalg.norm(y[b] - want) / np.linalg.norm(want)
        assert err < 2e-5, err


def test_power_method_and_lambda():
    S, traj, _ = small()
    op = pico.Operator(S, traj=traj, lam=0.1, power_iters=15)
    oop = O.Operator(S, None, traj=traj)
    lp, lmax = OP.lambda_phys(oop, 0.1, 15, 1.01)
    assert abs(op.info["lambda_max"] - lmax) / lmax < 1e-5
    assert abs(op.info["lambda_phys"] - lp) / lp < 1e-5


def test_spiral_cg_and_variance_map_same_seed():
    S, traj, _ = small(64, 6, 2, 512, seed=4)
    op = pico.Operator(S, traj=traj, lam=0.1, power_iters=15, max_batch=8)
    oop = O.Operator(S, None, traj=traj)
    lam = op.info["lambda_phys"]
    rhs = rand_imgs(2, 64, 9)
    x = op.cg(to_dev(rhs), 30, 0.0).cpu().numpy()
    for b in range(2):
        want, _, _ = OS.cg(lambda z: oop.normal(z, lam), rhs[b].astype(np.complex128), 30, 0.0)
        assert np.linalg.norm(x[b] - want) / np.linalg.norm(want) < 1e-4
    K = 8
    s, _ = op.variance_sums(11, K, 30, 0.0)
    so, _ = OP.pico(oop, 11, 0, K, lam, 30, 0.0)
    Sig = OP.dense_cov(OP.dense_normal(oop), lam)
    d = np.real(np.diag(Sig)).reshape(64, 64)
    rel = np.abs(s.cpu().numpy() / K - so / K) / d
    assert rel.max() < 1e-4, rel.max()


def test_spiral_variance_map_band():
    S, traj, _ = small(64, 6, 2, 512, seed=5)
    op = pico.Operator(S, traj=traj, lam=0.1, power_iters=15, max_batch=64)
    oop = O.Operator(S, None, traj=traj)
    lam = op.info["lambda_phys"]
    Sig = OP.dense_cov(OP.dense_normal(oop), lam)
    d = np.real(np.diag(Sig)).reshape(64, 64)
    var = OP.per_sample_variance(Sig, "phase").reshape(64, 64)
    K = 128
    s, _ = op.variance_sums(12, K, 60, 0.0)
    z = (s.cpu().numpy() / K - d) / np.sqrt(var / K)
    assert np.all(np.abs(z) < 6), np.abs(z).max()
    assert np.mean(np.abs(z) > 3) < 0.01


def test_spiral_pmr_same_seed_within_gridding_error():
    S, traj, _ = small(64, 6, 2, 512, seed=6)
    op = pico.Operator(S, traj=traj, lam=0.1, power_iters=15, max_batch=8)
    oop = O.Operator(S, None, traj=traj)
    lam = op.info["lambda_phys"]
    N, sigma = 6, 1e-2
    s, _ = op.pmr_sums(31, N, sigma, 30)
    so, _ = OP.pmr(oop, 31, 0, N, sigma, lam, 30, 0.0)
    Sig = OP.dense_cov(OP.dense_normal(oop), lam)
    d = np.real(np.diag(Sig)).reshape(64, 64)
    rel = np.abs(s.cpu().numpy() / N - so / N) / d
    # Kaiser-Bessel W = 6, oversampling 2: the gridded adjoint is accurate to ~1e-5 relative
    assert rel.max() < 1e-3, rel.max()
    assert np.median(rel) < 1e-4, np.median(rel)


# ---------------------------------------------------------------------------
# full size: 240x240, 20 coils, 16 x 4096 variable-density spiral, R = 2
# ---------------------------------------------------------------------------
def test_full_size_toeplitz_on_sampled_outputs():
    w = synth.WORKLOADS["spiral240_r2"]
    inp = w.inputs()
    S, traj = inp["smaps"], inp["traj"]
    n = w.ny
    op = pico.Operator(S, traj=traj, lam=0.0, power_iters=0, max_batch=w.probes)
    # the bench's launch shape: one batch of 256 images; image b is a unit impulse at r_b
    rng = np.random.default_rng(0)
    pos = rng.integers(0, n, size=(w.probes, 2))
    x = np.zeros((w.probes, n, n), dtype=np.complex64)
    x[np.arange(w.probes), pos[:, 0], pos[:, 1]] = 1.0
    y = op.apply_normal(to_dev(x)).cpu().numpy()
    # exact: (A^H A d_r0)[r] = sum_c conj(S_c[r]) S_c[r0] h(r - r0),
    # h(d) = (1/n^2) sum_m exp(+2 pi i k_m . d / n)
    k = traj.astype(np.float64)
    S64 = S.astype(np.complex128)
    for b in (0, 77, 255):
        y0, x0 = pos[b]
        outs = rng.integers(0, n, size=(6, 2))
        outs[0] = (y0, x0)
        for (yy, xx) in outs:
            dy, dx = yy - y0, xx - x0
            h = np.exp(2j * np.pi * (k[:, 0] * dx + k[:, 1] * dy) / n).sum() / n ** 2
            want = np.sum(np.conj(S64[:, yy, xx]) * S64[:, y0, x0]) * h
            got = y[b, yy, xx]
            assert abs(got - want) <= 1e-5 * abs(y[b, y0, x0]) + 1e-4 * abs(want), (b, yy, xx, got, want)


def test_full_size_gridding_adjoint_against_exact_nudft():
    """pico_adjoint (Kaiser-Bessel W = 6, oversampling 2, gather gridding on the
    480 x 480 grid) on one random whitened k-space vector of the full workload
    (20 coils x 32768 samples) against the exact NUDFT adjoint."""
    w = synth.WORKLOADS["spiral240_r2"]
    inp = w.inputs()
    S, traj = inp["smaps"], inp["traj"]
    n, M = w.ny, traj.shape[0]
    op = pico.Operator(S, traj=traj, lam=0.0, power_iters=0, max_batch=2)
    g = np.random.default_rng(21)
    y = (g.standard_normal((1, w.nc, M)) + 1j * g.standard_normal((1, w.nc, M))).astype(np.complex64)
    x = op.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()[0]
    oop = O.Operator(S, None, traj=traj)
    want = oop.adjoint(y[0].astype(np.complex128))
    err = np.abs(x - want) / np.abs(want).max()
    # the gridding approximation (W = 6, os = 2): about 1e-4 of the peak, far below at most voxels
    assert err.max() < 1e-3, err.max()
    assert np.median(err) < 1e-4, np.median(err)
    op.close()


def test_full_size_pico_probes_same_seed_at_the_bench_launch_shape():
    """Probes 0 and 255 of one 256-probe batch (lam = 0.1: solve, A^H A, solve;
    30 CG updates each) against the oracle's same-seed products with the exact
    Toeplitz-form operator.  The GPU's per-probe product is the difference of
    two running-sum maps (every image of a batch is processed on its own, so
    the products do not depend on the batch); per voxel
    |d_gpu - d_oracle| <= 1e-4 max(|u_k|, 0.1 median |u|), u = Sigma v."""
    w = synth.WORKLOADS["spiral240_r2"]
    inp = w.inputs()
    S, traj = inp["smaps"], inp["traj"]
    n, K, seed = w.ny, w.probes, 3131
    op = pico.Operator(S, traj=traj, lam=w.lam, power_iters=15, max_batch=K)
    lam = op.info["lambda_phys"]
    s_all, _ = op.variance_sums(seed, K, w.max_iter, 0.0)                  # the bench's launch shape
    s_wo_last, _ = op.variance_sums(seed, K - 1, w.max_iter, 0.0)
    s_wo_first, _ = op.variance_sums(seed, K - 1, w.max_iter, 0.0, probe_begin=1)
    op.sync()
    d_gpu = {K - 1: (s_all - s_wo_last).cpu().numpy(), 0: (s_all - s_wo_first).cpu().numpy()}
    op.close()
    T = O.ToeplitzNormal(S, traj)
    lmax = OS.power_method(lambda x: T.apply(x), (n, n), 15)
    assert abs(lam - w.lam * 1.01 * lmax) <= 1e-5 * lam
    for i in (0, K - 1):
        v = ORNG.probe(seed, i, n * n).reshape(n, n)
        x1, _, _ = OS.cg(lambda z: T.apply(z, lam), v, w.max_iter)
        u, _, _ = OS.cg(lambda z: T.apply(z, lam), T.apply(x1), w.max_iter)
        d_o = np.real(np.conj(v) * u)
        scale = np.maximum(np.abs(u), 0.1 * np.median(np.abs(u)))
        err = np.abs(d_gpu[i] - d_o) / scale
        assert err.max() < 1e-4, (i, err.max())
