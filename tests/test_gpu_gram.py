"""GPU parity of the tensor-core (dense per-column Gram) Cartesian normal operator.

Cartesian contexts with a phase-encode mask and ny a multiple of 16, ny >= 128,
apply A^H A inside CG as nx dense ny x ny products on the tcgen05 tensor cores
with a 3-term TF32 split.  These tests compare that path with the FP64 oracle
(operator, CG, PICO, PMR), with the column-FFT path of the same library
(PICO_NORMAL_OP=fft), and check its determinism across batch sizes.
PICO_GRAM_MIN_BATCH=1 makes every batch use the Gram operator here (contexts
keep batches below 64 images on the column-FFT kernel by default).

Tolerances: one operator application agrees with the oracle to 1e-5 relative
in norm (the split keeps about 21 mantissa bits per product; the tensor-memory
FP32 accumulation over 6 ny products dominates, about 6e-6 at ny = 384);
after 30 CG iterations the same 1e-4 bounds as the FFT path.
"""
import os

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
def _gram_for_every_batch(monkeypatch):
    # contexts use the Gram operator for batches of 64+ images by default;
    # these small cases exercise it at every batch size
    monkeypatch.setenv("PICO_GRAM_MIN_BATCH", "1")


def case(ny, nx, nc, R=2, acs=8, corr=True, seed=0):
    S = synth.coil_maps(ny, nx, nc, seed)
    cov = synth.noise_cov(nc, seed) if corr else None
    return S, cov, synth.mask_pe(ny, R, acs)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def rand_imgs(nb, ny, nx, seed):
    g = np.random.default_rng(seed)
    return (g.standard_normal((nb, ny, nx)) + 1j * g.standard_normal((nb, ny, nx))).astype(np.complex64)


def fft_path_operator(*args, **kw):
    old = os.environ.get("PICO_NORMAL_OP")
    os.environ["PICO_NORMAL_OP"] = "fft"
    try:
        return pico.Operator(*args, **kw)
    finally:
        if old is None:
            del os.environ["PICO_NORMAL_OP"]
        else:
            os.environ["PICO_NORMAL_OP"] = old


def operator_with_env(var, val, *args, **kw):
    old = os.environ.get(var)
    os.environ[var] = val
    try:
        return pico.Operator(*args, **kw)
    finally:
        if old is None:
            del os.environ[var]
        else:
            os.environ[var] = old


# With PICO_GRAM_ATMEM=1 the split direction is staged in tensor memory for
# tiles of up to 192 output rows (ny 128, 160, 320, 384 here; 240 and 256 stay
# in shared memory); the default stages it in shared memory.  Both feed the
# same products to the same FP32 accumulation, so the two agree to rounding.
@pytest.mark.parametrize("ny,nx", [(128, 9), (160, 7), (320, 5), (384, 4)])
def test_tensor_memory_operand_matches_shared_memory_operand(ny, nx):
    S, cov, mask = case(ny, nx, 4, acs=6, seed=ny)
    x = to_dev(rand_imgs(130, ny, nx, 3))
    # both with the TF32 split (the FP16 operands are staged in shared memory only)
    os.environ["PICO_GRAM_TF32"] = "1"
    try:
        ops = [operator_with_env("PICO_GRAM_ATMEM", v, S, mask=mask, noise_cov=cov, lam=0.02, power_iters=0,
                                 max_batch=130) for v in ("1", "0")]
    finally:
        del os.environ["PICO_GRAM_TF32"]
    ya, yb = (o.apply_normal(x) for o in ops)
    assert ((ya - yb).abs().max() / yb.abs().max()).item() < 1e-6
    xa, ia, ra = ops[0].cg(x, 12, 0.0, stats=True)
    xb, ib, rb = ops[1].cg(x, 12, 0.0, stats=True)
    assert ((xa - xb).abs().max() / xb.abs().max()).item() < 1e-5
    assert np.allclose(ra, rb, rtol=1e-3, atol=1e-7)
    for o in ops:
        assert pico.pico_sync(o.ctx) is None


def test_path_selection():
    S, cov, mask = case(320, 24, 4)
    assert pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0).info["normal_op"] == 1
    assert fft_path_operator(S, mask=mask, noise_cov=cov, power_iters=0).info["normal_op"] == 0
    S, cov, mask = case(64, 64, 4)
    # ny = 64: the solves run on chip (dense G_j in shared memory); PICO_NORMAL_OP=fft keeps the column FFTs
    assert pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0).info["normal_op"] == 3
    assert fft_path_operator(S, mask=mask, noise_cov=cov, power_iters=0).info["normal_op"] == 0


# (ny, nx): one and two output-row tiles, ragged column counts, several tile widths
@pytest.mark.parametrize("ny,nx", [(128, 20), (160, 33), (192, 8), (240, 17), (256, 12), (320, 21), (384, 10)])
@pytest.mark.parametrize("lam", [0.0, 0.05])
def test_apply_normal_matches_oracle(ny, nx, lam):
    S, cov, mask = case(ny, nx, 5, acs=6, seed=ny + nx)
    op = pico.Operator(S, mask=mask, noise_cov=cov, lam=lam, power_iters=0, max_batch=4)
    assert op.info["normal_op"] == 1
    oop = O.Operator(S, cov, mask=mask)
    x = rand_imgs(5, ny, nx, 1)                       # two batches of 4 + 1
    y = op.apply_normal(to_dev(x)).cpu().numpy()
    for b in range(5):
        want = oop.normal(x[b].astype(np.complex128), lam)
        err = np.linalg.norm(y[b] - want) / np.linalg.norm(want)
        assert err < 1e-5, (b, err)
    assert pico.pico_sync(op.ctx) is None


def test_apply_normal_across_image_tiles():
    # 130 images: a full 128-image tile and a ragged second one
    ny, nx = 160, 6
    S, cov, mask = case(ny, nx, 4, seed=5)
    op = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=130)
    oop = O.Operator(S, cov, mask=mask)
    x = rand_imgs(130, ny, nx, 2)
    y = op.apply_normal(to_dev(x)).cpu().numpy()
    for b in (0, 63, 127, 128, 129):
        want = oop.normal(x[b].astype(np.complex128))
        assert np.linalg.norm(y[b] - want) / np.linalg.norm(want) < 1e-5, b
    # each image's result does not depend on where it sits in the batch
    y1 = op.apply_normal(to_dev(x[129:130])).cpu().numpy()
    assert np.array_equal(y1[0], y[129])


@pytest.mark.parametrize("ny,nx,nc,lam", [(128, 24, 6, 0.0), (160, 18, 5, 0.1)])
def test_cg_fixed_iterations_matches_oracle(ny, nx, nc, lam):
    S, cov, mask = case(ny, nx, nc, seed=7)
    op = pico.Operator(S, mask=mask, noise_cov=cov, lam=lam, power_iters=0, max_batch=4)
    oop = O.Operator(S, cov, mask=mask)
    rhs = rand_imgs(5, ny, nx, 11)
    x, iters, relres = op.cg(to_dev(rhs), 30, 0.0, stats=True)
    x = x.cpu().numpy()
    assert np.all(iters == 30)
    for b in range(5):
        want, it, rr = OS.cg(lambda z: oop.normal(z, lam), rhs[b].astype(np.complex128), 30, 0.0)
        err = np.linalg.norm(x[b] - want) / np.linalg.norm(want)
        assert err < 1e-4, err
        assert abs(relres[b] - rr) <= 1e-3 * rr + 1e-6


@pytest.mark.parametrize("iters,rtol", [(30, 0.0), (7, 0.0), (30, 1e-3), (9, 1e-6)])
def test_x_advanced_per_pair_of_iterations_gives_the_same_bits(iters, rtol):
    """On the tensor-core path x is advanced once per two iterations (the two
    FMAs of a value in the same order, one pass over x saved); with
    PICO_CG_PAIR_X=0 it is advanced every iteration.  Solutions, update counts
    and residuals are the same bits, for even and odd iteration counts, with
    and without the stopping rule (which runs the iterations in chunks)."""
    S, cov, mask = case(160, 18, 5, seed=13)
    rhs = to_dev(rand_imgs(6, 160, 18, 17))
    out = []
    for v in ("1", "0"):
        op = operator_with_env("PICO_CG_PAIR_X", v, S, mask=mask, noise_cov=cov, lam=0.05, power_iters=0, max_batch=8)
        x, it, rel = op.cg(rhs, iters, rtol, stats=True)
        op.sync()
        out.append((x.cpu(), np.array(it), np.array(rel)))
        op.close()
    assert torch.equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


def test_cg_stopping_rule_matches_oracle():
    S, cov, mask = case(128, 16, 6, seed=9)
    op = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=8)
    oop = O.Operator(S, cov, mask=mask)
    rhs = rand_imgs(3, 128, 16, 5)
    x, iters, relres = op.cg(to_dev(rhs), 100, 1e-3, stats=True)
    for b in range(3):
        _, it, rr = OS.cg(lambda z: oop.normal(z), rhs[b].astype(np.complex128), 100, 1e-3)
        assert abs(int(iters[b]) - it) <= 1, (iters[b], it)
        assert relres[b] <= 1e-3


def test_variance_map_same_seed_parity_and_fft_path_agreement():
    ny, nx = 128, 16
    S, cov, mask = case(ny, nx, 6, seed=3)
    oop = O.Operator(S, cov, mask=mask)
    d, _, _ = OP.column_exact(oop)
    K = 12
    op = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=8)
    s, _ = op.variance_sums(31, K, 30, 0.0)
    so, _ = OP.pico(oop, 31, 0, K, 0.0, 30, 0.0)
    assert (np.abs(s.cpu().numpy() - so) / K / d).max() < 1e-4
    opf = fft_path_operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=8)
    sf, _ = opf.variance_sums(31, K, 30, 0.0)
    assert (np.abs(s.cpu().numpy() - sf.cpu().numpy()) / K / d).max() < 1e-4


def test_pmr_same_seed_parity():
    ny, nx = 160, 32                      # the PMR adjoint needs an x-FFT length of this build
    S, cov, mask = case(ny, nx, 6, seed=2)
    op = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=8)
    oop = O.Operator(S, cov, mask=mask)
    N, sigma = 10, 1e-2
    s, _ = op.pmr_sums(21, N, sigma, 30)
    so, _ = OP.pmr(oop, 21, 0, N, sigma, 0.0, 30, 0.0)
    d, _, _ = OP.column_exact(oop)
    assert (np.abs(s.cpu().numpy() - so) / N / d).max() < 1e-4


def test_batch_grouping_and_resume_are_bitwise_identical():
    ny, nx = 128, 10
    S, cov, mask = case(ny, nx, 5, seed=4)
    op = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=8)
    full_s, full_ss = op.variance_sums(5, 20, 20, 0.0)
    s, ss = op.variance_sums(5, 7, 20, 0.0, probe_begin=0)
    op.variance_sums(5, 13, 20, 0.0, probe_begin=7, sum_=s, sumsq=ss)
    assert torch.equal(full_s, s) and torch.equal(full_ss, ss)
    op2 = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=3)
    s2, _ = op2.variance_sums(5, 20, 20, 0.0)
    assert torch.equal(full_s, s2)


def test_lambda_positive_composition_matches_oracle():
    # Sigma v = (M + lam)^-1 M (M + lam)^-1 v: solve, A^H A on the solution, solve
    ny, nx, lam = 128, 12, 0.1
    S, cov, mask = case(ny, nx, 5, seed=8)
    op = pico.Operator(S, mask=mask, noise_cov=cov, lam=lam, power_iters=0, max_batch=4)
    oop = O.Operator(S, cov, mask=mask)
    K = 6
    s, _ = op.variance_sums(13, K, 30, 0.0)
    so, _ = OP.pico(oop, 13, 0, K, lam, 30, 0.0)
    d, _, _ = OP.column_exact(oop, lam)
    assert (np.abs(s.cpu().numpy() - so) / K / d).max() < 1e-4


# ---------------------------------------------------------------------------
# full size: 320x320, 15 correlated coils, R=2 + 24 calibration lines, K=256
# (the benchmark's launch shape)
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
    assert op.info["normal_op"] == 1
    n = w.ny * w.nx
    rhs = np.stack([ORNG.probe(77, i, n).reshape(w.ny, w.nx) for i in range(w.probes)]).astype(np.complex64)
    x = op.cg(to_dev(rhs), w.max_iter, 0.0).cpu().numpy()
    for i in (0, 127, 128, 255):
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
    assert np.mean(np.abs(z) > 4) < 0.01, np.mean(np.abs(z) > 4)
    assert np.abs(s.cpu().numpy() / K - d).max() / d.max() < 0.2
    assert pico.pico_sync(op.ctx) is None


# The default operands are FP16 head + remainder pairs (kind::f16) after
# power-of-two scaling: G_j by a per-column scale from the bound
# P[0] max_y sum_c |S_c[y, j]|^2, the direction by a per-image scale from the
# bound sqrt(r^H r) + beta |p_prev| (CG) or max |x| (an application).
# PICO_GRAM_TF32=1 selects the TF32 split.  Both keep about 22 significant
# bits per product; the scales make the FP16 range irrelevant, checked here
# with sensitivities 1e4 and 1e-4 times the unit-energy maps (G_j entries
# near 1e8 and 1e-8).
@pytest.mark.parametrize("scale", [1.0, 1e4, 1e-4])
def test_fp16_operands_match_the_oracle_and_tf32(scale):
    ny, nx = 320, 6
    S, cov, mask = case(ny, nx, 5, acs=6, seed=31)
    S = (S * scale).astype(np.complex64)
    kw = dict(mask=mask, noise_cov=cov, lam=0.0, power_iters=0, max_batch=70)
    f16 = pico.Operator(S, **kw)
    tf32 = operator_with_env("PICO_GRAM_TF32", "1", S, **kw)
    oop = O.Operator(S, cov, mask=mask)
    x = rand_imgs(70, ny, nx, 4)
    y16, y32 = (o.apply_normal(to_dev(x)).cpu().numpy() for o in (f16, tf32))
    for b in (0, 69):
        want = oop.normal(x[b].astype(np.complex128))
        assert np.linalg.norm(y16[b] - want) / np.linalg.norm(want) < 1e-5
        assert np.linalg.norm(y32[b] - want) / np.linalg.norm(want) < 1e-5
    # 30 CG updates: the FP16 and TF32 solves agree with the FP64 CG to the usual 1e-4
    xs = to_dev(x)
    for o in (f16, tf32):
        xc = o.cg(xs, 30, 0.0).cpu().numpy()
        for b in (0, 69):
            xo, _, _ = OS.cg(lambda z: oop.normal(z), x[b].astype(np.complex128), 30)
            assert np.abs(xc[b] - xo).max() / np.abs(xo).max() < 1e-4, (scale, b)
        assert pico.pico_sync(o.ctx) is None
    # the per-column CG on FP16 operands as well
    f16.set_solver("columns")
    xc = f16.cg(xs, 30, 0.0).cpu().numpy()
    xo, _, _ = OS.cg_columns(oop, x[[0, 69]].astype(np.complex128), 0.0, 30)
    for i, b in enumerate((0, 69)):
        assert np.abs(xc[b] - xo[i]).max() / np.abs(xo[i]).max() < 1e-4, (scale, b)
