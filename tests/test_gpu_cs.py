"""Nonlinear CS path on the GPU: 2-D-mask operators, L1-wavelet FISTA, its
Jacobian (JVP / VJP) and the Jacobian PICO estimator against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import cs as OCS
from oracle import ops as O
from oracle import pico as OP

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def case64():
    n, nc = 64, 8
    S = synth.coil_maps(n, n, nc, 5)
    mask = synth.poisson_disc_mask(n, n, 2.0, 12, 5)
    op = pico.Operator(S, mask=mask, power_iters=15, max_batch=8)
    oop = O.Operator(S, None, mask=mask)
    x0 = synth.phantom(n, 5).astype(np.complex128)
    b = oop.forward(x0)
    h, g = OCS.wavelet_filters(4)
    lam = 1e-2 * np.abs(OCS.dwt2(oop.adjoint(b), 4, h, g)).max()
    return n, nc, S, mask, op, oop, b, lam


def test_2d_mask_operators_match_oracle(case64):
    n, nc, S, mask, op, oop, b, lam = case64
    g = np.random.default_rng(1)
    x = (g.standard_normal((2, n, n)) + 1j * g.standard_normal((2, n, n))).astype(np.complex64)
    y = op.apply_normal(dev(x)).cpu().numpy()
    k = op.forward(dev(x)).cpu().numpy()
    xa = op.adjoint(dev(k)).cpu().numpy()
    for i in range(2):
        assert rel(y[i], oop.normal(x[i].astype(np.complex128))) < 2e-6
        assert rel(k[i], oop.forward(x[i].astype(np.complex128))) < 2e-6
        assert rel(xa[i], oop.adjoint(k[i].astype(np.complex128))) < 2e-6


def test_fista_reconstruction_matches_oracle(case64):
    n, nc, S, mask, op, oop, b, lam = case64
    f = OCS.Fista(oop, b, lam, 30, levels=4)
    x = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    pico.pico_cs_recon(op.ctx, dev(b), lam, 30, 4, x)
    assert rel(x.cpu().numpy(), f.x) < 1e-4


def test_jvp_vjp_match_oracle_and_finite_differences(case64):
    n, nc, S, mask, op, oop, b, lam = case64
    f = OCS.Fista(oop, b, lam, 30, levels=4)
    x = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    pico.pico_cs_recon(op.ctx, dev(b), lam, 30, 4, x)
    g = np.random.default_rng(2)
    m = O.mask2d(mask, n)[None]
    db = ((g.standard_normal((2, nc, n, n)) + 1j * g.standard_normal((2, nc, n, n))) * m).astype(np.complex64)
    dx = torch.empty((2, n, n), dtype=torch.complex64, device="cuda")
    pico.pico_cs_jvp(op.ctx, dev(db), dx)
    # FP64 central differences of the oracle reconstruction (the Jacobian it approximates)
    eps = 1e-6 * np.linalg.norm(b) / np.linalg.norm(db[0])
    fd = (OCS.Fista(oop, b + eps * db[0], lam, 30, levels=4).x
          - OCS.Fista(oop, b - eps * db[0], lam, 30, levels=4).x) / (2 * eps)
    assert rel(dx[0].cpu().numpy(), fd) < 1e-3
    assert rel(dx[1].cpu().numpy(), f.jvp(db[1].astype(np.complex128))) < 1e-3
    xb = (g.standard_normal((2, n, n)) + 1j * g.standard_normal((2, n, n))).astype(np.complex64)
    bb = torch.empty((2, nc, n, n), dtype=torch.complex64, device="cuda")
    pico.pico_cs_vjp(op.ctx, dev(xb), bb)
    assert rel(bb[0].cpu().numpy(), f.vjp(xb[0].astype(np.complex128))) < 1e-3
    # adjoint identity of the GPU pair itself
    lhs = float(np.vdot(xb.astype(np.complex128), dx.cpu().numpy().astype(np.complex128)).real)
    rhs = float(np.vdot(bb.cpu().numpy().astype(np.complex128), db.astype(np.complex128)).real)
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)


def test_jacobian_pico_same_seed(case64):
    n, nc, S, mask, op, oop, b, lam = case64
    f = OCS.Fista(oop, b, lam, 30, levels=4)
    x = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    pico.pico_cs_recon(op.ctx, dev(b), lam, 30, 4, x)
    K = 6
    s = torch.empty((n, n), dtype=torch.float64, device="cuda")
    pico.pico_cs_variance_map(op.ctx, 17, 0, K, 0, s)
    so, _ = OCS.pico_cs(f, 17, 0, K)
    assert rel(s.cpu().numpy() / K, so / K) < 1e-3
    # every voxel within 1e-5 of the map's largest value (measured against the exact
    # Jacobian diagonal: below 7e-6 of it at every voxel)
    err = np.abs(s.cpu().numpy() - so).max() / np.abs(so).max()
    assert err < 1e-5, err


def test_linear_case_jacobian_equals_reconstruction(case64):
    n, nc, S, mask, op, oop, b, lam = case64
    x = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    pico.pico_cs_recon(op.ctx, dev(b), 0.0, 40, 4, x)       # lambda = 0: f is linear, J = f
    g = np.random.default_rng(3)
    db = ((g.standard_normal((1, nc, n, n)) + 1j * g.standard_normal((1, nc, n, n))) * O.mask2d(mask, n)[None]
          ).astype(np.complex64)
    dx = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
    pico.pico_cs_jvp(op.ctx, dev(db), dx)
    xl = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    pico.pico_cs_recon(op.ctx, dev(db[0]), 0.0, 40, 4, xl)
    assert rel(dx[0].cpu().numpy(), xl.cpu().numpy()) < 1e-5


def test_autograd_function_backward_is_the_vjp(case64):
    n, nc, S, mask, op, oop, b, lam = case64
    F = pico.cs_function()
    bt = dev(b).requires_grad_(True)
    x = F.apply(op, bt, lam, 30, 4)
    g = torch.from_numpy((np.random.default_rng(4).standard_normal((n, n)) + 0.5j).astype(np.complex64)).cuda()
    (gb,) = torch.autograd.grad((g.conj() * x).real.sum(), bt)
    bb = torch.empty((1, nc, n, n), dtype=torch.complex64, device="cuda")
    pico.pico_cs_vjp(op.ctx, g.reshape(1, n, n), bb)
    assert torch.allclose(gb, bb[0], rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("levels", [1, 4])
def test_wavelet_operator_matches_oracle(case64, levels):
    n, nc, S, mask, op, oop, b, lam = case64
    h, g = OCS.wavelet_filters(4)
    r = np.random.default_rng(5)
    x = (r.standard_normal((3, n, n)) + 1j * r.standard_normal((3, n, n))).astype(np.complex64)
    c = torch.empty((3, n, n), dtype=torch.complex64, device="cuda")
    pico.pico_wavelet(op.ctx, dev(x), c, levels)
    xi = dev(x)
    pico.pico_wavelet(op.ctx, xi, xi, levels, inverse=True)          # in place
    for i in range(3):
        assert rel(c[i].cpu().numpy(), OCS.dwt2(x[i].astype(np.complex128), levels, h, g)) < 2e-6
        assert rel(xi[i].cpu().numpy(), OCS.idwt2(x[i].astype(np.complex128), levels, h, g)) < 2e-6


def test_cs_pmr_same_seed_matches_oracle(case64):
    n, nc, S, mask, op, oop, b, lam = case64
    f = OCS.Fista(oop, b, lam, 30, levels=4)
    x = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    pico.pico_cs_recon(op.ctx, dev(b), lam, 30, 4, x)
    sigma = 0.1 * float(np.sqrt(np.mean(np.abs(b[:, mask.astype(bool)]) ** 2)))
    K = 5                                               # max_batch 8: one chunk; then 3 more accumulated
    s = torch.empty((n, n), dtype=torch.float64, device="cuda")
    ss = torch.empty_like(s)
    pico.pico_cs_pmr(op.ctx, 23, 0, K, sigma, s, ss)
    pico.pico_cs_pmr(op.ctx, 23, K, 3, sigma, s, ss, accumulate=True)
    so, sso = OCS.pmr_cs(f, 23, 0, K + 3, sigma)
    assert rel(s.cpu().numpy(), so) < 2e-3
    assert rel(ss.cpu().numpy(), sso) < 4e-3
    # every voxel within 3e-4 of the map's largest value: each replica reruns 30 FP32
    # FISTA iterations on noisy data (measured against the exact Jacobian
    # diagonal: a few 1e-5 of it at most voxels, 1.1e-4 at the worst)
    err = np.abs(s.cpu().numpy() - so).max() / so.max()
    assert err < 3e-4, err
    # the reconstruction itself is unchanged by the replica runs
    xs = x.clone()
    pico.pico_cs_recon(op.ctx, dev(b), lam, 30, 4, x)
    assert torch.equal(x, xs)


def test_cs_on_a_phase_encode_context_after_tensor_core_batches(monkeypatch):
    # a 1-D-mask context whose CG batches ran on the tensor-core Gram operator
    # (column-planar CG vectors) still reconstructs in the natural layout
    monkeypatch.setenv("PICO_GRAM_MIN_BATCH", "1")
    n, nc = 128, 4
    S = synth.coil_maps(n, n, nc, 9)
    mask = synth.mask_pe(n, 2, 8)
    op = pico.Operator(S, mask=mask, power_iters=15, max_batch=8)
    assert op.info["normal_op"] == 1
    op.variance_sums(3, 8, 10, 0.0)
    oop = O.Operator(S, None, mask=mask)
    b = oop.forward(synth.phantom(n, 9).astype(np.complex128))
    h, g = OCS.wavelet_filters(4)
    lam = 1e-2 * np.abs(OCS.dwt2(oop.adjoint(b), 4, h, g)).max()
    f = OCS.Fista(oop, b, lam, 20, levels=4)
    x = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    pico.pico_cs_recon(op.ctx, dev(b), lam, 20, 4, x)
    assert rel(x.cpu().numpy(), f.x) < 1e-4


# ---------------------------------------------------------------------------
# full size: 320x320, 15 correlated coils, Poisson-disc R=2, 100 FISTA
# iterations, the benchmark's launch shape (64 probes per launch)
# ---------------------------------------------------------------------------
def test_full_size_cs_sampled_parity():
    w = synth.WORKLOADS["cs320_r2"]
    inp = w.inputs()
    levels, iters = w.extra["levels"], w.max_iter
    oop = O.Operator(inp["smaps"], inp["noise_cov"], mask=inp["mask"])
    b = oop.forward(inp["phantom"].astype(np.complex128))
    h, g = OCS.wavelet_filters(4)
    lam = w.extra["lam_l1_rel"] * np.abs(OCS.dwt2(oop.adjoint(b), levels, h, g)).max()
    f = OCS.Fista(oop, b, lam, iters, levels=levels)
    op = pico.Operator(inp["smaps"], mask=inp["mask"], noise_cov=inp["noise_cov"], power_iters=15,
                       max_batch=w.probes)
    x = torch.empty((w.ny, w.nx), dtype=torch.complex64, device="cuda")
    pico.pico_cs_recon(op.ctx, dev(b), lam, iters, levels, x)
    assert rel(x.cpu().numpy(), f.x) < 2e-4            # 100 FP32 iterations
    K, i0 = w.probes, 5
    s64 = torch.zeros((w.ny, w.nx), dtype=torch.float64, device="cuda")
    pico.pico_cs_variance_map(op.ctx, 77, 0, K, 0, s64)           # one launch of 64 probes
    parts = torch.zeros_like(s64)
    one = torch.zeros_like(s64)
    for i in range(K):                                             # the same probes one at a time
        pico.pico_cs_variance_map(op.ctx, 77, i, 1, 0, one)
        parts += one
        if i == i0:
            probe5 = one.cpu().numpy().copy()
    assert torch.allclose(s64, parts, rtol=1e-9, atol=0)           # batching does not change a probe
    so, _ = OCS.pico_cs(f, 77, i0, 1)                              # one probe through the oracle
    assert rel(probe5, so) < 1e-3
    sigma = 0.1 * float(np.sqrt(np.mean(np.abs(b[:, inp["mask"].astype(bool)]) ** 2)))
    pm = torch.zeros_like(s64)
    pico.pico_cs_pmr(op.ctx, 78, 3, 1, sigma, pm)
    po, _ = OCS.pmr_cs(f, 78, 3, 1, sigma)
    assert rel(pm.cpu().numpy(), po) < 2e-3
