"""Pins that hold the CPU oracle to the mathematics (no GPU needed).

Each test checks an oracle function against something other than itself: a
published test vector, a hand-derived example, a textbook closed form, an
explicitly built matrix, a Krylov-subspace optimality property, or a
distributional identity of the paper (Eqs. 15-17, A1).
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import ops, pico, rng, solvers

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


# --------------------------------------------------------------------------
# counter-based generator
# --------------------------------------------------------------------------
def test_splitmix64_published_vectors():
    for seed, i, val in _rows("splitmix64.txt"):
        got = int(rng.splitmix64(np.uint64(int(seed)), np.uint64(int(i))))
        assert got == int(val, 16)


def test_probe_families_moments():
    n = 200_000
    v = rng.probe(7, 3, n, rng.PROBE_PHASE)
    assert np.allclose(np.abs(v), 1.0, atol=1e-15)               # kappa = 1 exactly
    assert abs(v.mean()) < 5 / math.sqrt(n)
    th = np.angle(v) % (2 * np.pi)
    hist, _ = np.histogram(th, bins=32, range=(0, 2 * np.pi))
    chi2 = ((hist - n / 32) ** 2 / (n / 32)).sum()
    assert chi2 < 80                                              # 31 dof
    r = rng.probe(7, 3, n, rng.PROBE_RADEMACHER)
    assert set(np.unique(r.real)) == {-1.0, 1.0} and np.all(r.imag == 0)
    assert abs(r.real.mean()) < 5 / math.sqrt(n)
    g = rng.probe(7, 3, n, rng.PROBE_GAUSS)
    assert abs(np.mean(np.abs(g) ** 2) - 1) < 0.02               # E|v|^2 = 1
    assert abs(np.mean(np.abs(g) ** 4) - 2) < 0.08               # kappa = 2
    # distinct probes are uncorrelated: E[v_i conj(v_j)] = 0 (Eq. 15)
    w = rng.probe(7, 4, n, rng.PROBE_PHASE)
    assert abs(np.vdot(v, w)) / n < 5 / math.sqrt(n)


# --------------------------------------------------------------------------
# operators
# --------------------------------------------------------------------------
def _small_cart(ny=12, nx=10, nc=3, R=2, acs=2, corr=True, seed=1):
    S = synth.coil_maps(ny, nx, nc, seed)
    cov = synth.noise_cov(nc, seed) if corr else None
    mask = synth.mask_pe(ny, R, acs)
    return ops.Operator(S, cov, mask=mask), S, cov, mask


def test_whitening_makes_noise_white():
    nc = 6
    cov = synth.noise_cov(nc, 3)
    S = synth.coil_maps(4, 4, nc, 3)
    Sw = ops.whiten(S, cov)
    # whitened operator = L^-1 applied across coils: L^-1 Sigma_n L^-H = I
    L = np.linalg.cholesky(cov)
    Li = np.linalg.inv(L)
    assert np.allclose(Li @ cov @ Li.conj().T, np.eye(nc), atol=1e-12)
    assert np.allclose(Sw, np.einsum("cd,dyx->cyx", Li, S.astype(np.complex128)))


def test_fft_operator_equals_explicit_dft_matrix():
    op, *_ = _small_cart()
    A = op.matrix()                                # from the DFT definition
    x = (np.random.default_rng(0).standard_normal((op.ny, op.nx))
         + 1j * np.random.default_rng(1).standard_normal((op.ny, op.nx)))
    m = ops.mask2d(op.mask, op.nx).reshape(-1) > 0
    fwd = op.forward(x)
    got = np.concatenate([fwd[c].reshape(-1)[m] for c in range(op.nc)])
    assert np.allclose(got, A @ x.reshape(-1), atol=1e-12)
    assert np.allclose(op.normal(x).reshape(-1), A.conj().T @ (A @ x.reshape(-1)), atol=1e-12)


def test_adjoint_dot_product():
    op, *_ = _small_cart(16, 14, 4)
    g = np.random.default_rng(5)
    x = g.standard_normal((op.ny, op.nx)) + 1j * g.standard_normal((op.ny, op.nx))
    y = g.standard_normal((op.nc, op.ny, op.nx)) + 1j * g.standard_normal((op.nc, op.ny, op.nx))
    y = y * ops.mask2d(op.mask, op.nx)[None]
    assert abs(np.vdot(op.forward(x), y) - np.vdot(x, op.adjoint(y))) < 1e-10


def test_column_decoupling_matches_dense():
    op, *_ = _small_cart(12, 6, 3)
    M = pico.dense_normal(op)
    ny, nx = op.ny, op.nx
    for col in range(nx):
        idx = np.arange(ny) * nx + col
        assert np.allclose(M[np.ix_(idx, idx)], ops.cart_column_normal(op.S, op.mask, col), atol=1e-12)
    # and nothing couples different columns
    Mc = M.copy()
    for col in range(nx):
        idx = np.arange(ny) * nx + col
        Mc[np.ix_(idx, idx)] = 0
    assert np.abs(Mc).max() < 1e-12


def test_grid_aligned_nudft_equals_fft():
    n = 8
    ky, kx = np.meshgrid(np.arange(-n // 2, n // 2), np.arange(-n // 2, n // 2), indexing="ij")
    traj = np.stack([kx.reshape(-1), ky.reshape(-1)], axis=1).astype(np.float32)
    E = ops.Nudft(traj, n)
    z = np.random.default_rng(2).standard_normal((n, n)) + 1j * np.random.default_rng(3).standard_normal((n, n))
    F = np.fft.fft2(z, norm="ortho")
    want = F[ky.reshape(-1) % n, kx.reshape(-1) % n]
    assert np.allclose(E.forward(z), want, atol=1e-12)
    w = np.random.default_rng(4).standard_normal(n * n) + 0j
    assert abs(np.vdot(E.forward(z), w) - np.vdot(z, E.adjoint(w))) < 1e-10


def test_spiral_dense_normal_from_psf_matches_explicit_matrix():
    n, nc = 8, 3
    S = synth.coil_maps(n, n, nc, 5)
    traj = synth.spiral_traj(n, n_interleaves=4, nsamp=50, R=1)
    op = ops.Operator(S, synth.noise_cov(nc, 5), traj=traj)
    A = op.matrix()
    assert np.allclose(pico.dense_normal(op), A.conj().T @ A, atol=1e-12)


def test_spiral_operator_matches_explicit_matrix():
    n, nc = 8, 3
    S = synth.coil_maps(n, n, nc, 4)
    traj = synth.spiral_traj(n, n_interleaves=4, nsamp=40, R=1)
    op = ops.Operator(S, None, traj=traj)
    A = op.matrix()
    x = np.random.default_rng(6).standard_normal((n, n)) + 0.5j
    assert np.allclose(op.normal(x).reshape(-1), A.conj().T @ (A @ x.reshape(-1)), atol=1e-10)


# --------------------------------------------------------------------------
# exact covariance: closed forms
# --------------------------------------------------------------------------
def test_hand_derived_sense_example():
    S = np.array([[[1.0], [0.5]], [[0.0], [1.0]]], dtype=np.complex64)     # [nc=2][ny=2][nx=1]
    op = ops.Operator(S, None, mask=np.array([1, 0], dtype=np.uint8))
    Sig = pico.dense_cov(pico.dense_normal(op))
    full = ops.Operator(S, None, mask=np.array([1, 1], dtype=np.uint8))
    Sig_ref = pico.dense_cov(pico.dense_normal(full))
    g = pico.gfactor(np.real(np.diag(Sig)), np.real(np.diag(Sig_ref)), 2)
    vs = pico.per_sample_variance(Sig, "phase")
    for (y, va, vr, gg, vp) in _rows("sense_2x1_r2.txt"):
        y = int(y)
        assert abs(Sig[y, y].real - float(va)) < 1e-12
        assert abs(Sig_ref[y, y].real - float(vr)) < 1e-12
        assert abs(g[y] - float(gg)) < 1e-12
        assert abs(vs[y] - float(vp)) < 1e-12


@pytest.mark.parametrize("n,nc,R", [(16, 4, 2), (24, 6, 3), (32, 8, 2)])
def test_dense_inverse_matches_closed_form_sense(n, nc, R):
    S = synth.coil_maps(n, n, nc, 11)
    op = ops.Operator(S, None, mask=synth.mask_pe(n, R, 0))
    Sig = pico.dense_cov(pico.dense_normal(op))
    var, var_ref, g = pico.sense_closed_form(op.S, R)
    assert np.allclose(np.real(np.diag(Sig)).reshape(n, n), var, rtol=1e-10, atol=0)
    assert np.allclose(var_ref, 1.0, atol=1e-6)                # sum |S|^2 = 1
    assert np.all(g >= 1 - 1e-9)                               # unregularised SENSE: g >= 1


def test_uniform_mask_offset_leaves_variance_unchanged():
    n, nc, R = 16, 4, 2
    S = synth.coil_maps(n, n, nc, 12)
    a = ops.Operator(S, None, mask=synth.mask_pe(n, R, 0, offset=0))
    b = ops.Operator(S, None, mask=synth.mask_pe(n, R, 0, offset=1))
    da = np.real(np.diag(pico.dense_cov(pico.dense_normal(a))))
    db = np.real(np.diag(pico.dense_cov(pico.dense_normal(b))))
    assert np.allclose(da, db, rtol=1e-10)


def test_column_exact_matches_dense_with_acs_and_correlated_noise():
    op, *_ = _small_cart(16, 8, 4, R=2, acs=4, corr=True)
    for lam in (0.0, 0.3):
        Sig = pico.dense_cov(pico.dense_normal(op), lam)
        d, rowe, half = pico.column_exact(op, lam)
        assert np.allclose(np.real(np.diag(Sig)).reshape(op.ny, op.nx), d, rtol=1e-10)
        assert np.allclose(np.sum(np.abs(Sig) ** 2, axis=1).reshape(op.ny, op.nx), rowe, rtol=1e-10)
        assert np.allclose(pico.per_sample_variance(Sig, "phase").reshape(op.ny, op.nx), half,
                           rtol=1e-9, atol=1e-14)


def test_full_sampling_gives_inverse_coil_energy():
    n, nc = 12, 4
    S = synth.coil_maps(n, n, nc, 13, normalize=False)
    op = ops.Operator(S, None, mask=np.ones(n, dtype=np.uint8))
    d, _, half = pico.column_exact(op)
    assert np.allclose(d, 1.0 / np.sum(np.abs(S.astype(np.complex128)) ** 2, axis=0), rtol=1e-10)
    assert np.abs(half).max() < 1e-20                                   # Sigma is diagonal


def test_tikhonov_shrinkage():
    op, *_ = _small_cart(16, 6, 4, R=2, acs=2)
    d0, *_ = pico.column_exact(op, 0.0)
    for lam in (1e-3, 0.1, 1.0):
        dl, *_ = pico.column_exact(op, lam)
        assert np.all(dl < d0)                                          # App. D, Proposition


# --------------------------------------------------------------------------
# solvers
# --------------------------------------------------------------------------
def test_cg_iterate_is_krylov_energy_minimiser():
    op, *_ = _small_cart(10, 6, 3)
    M = pico.dense_normal(op)
    lam = 0.05
    Ml = M + lam * np.eye(M.shape[0])
    b = rng.probe(3, 0, M.shape[0])
    xs = np.linalg.solve(Ml, b)
    for k in (1, 3, 6):
        x, it, _ = solvers.cg(lambda z: Ml @ z, b, k)
        assert it == k
        K = np.stack([np.linalg.matrix_power(Ml, j) @ b for j in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        y = np.linalg.solve(Q.conj().T @ Ml @ Q, Q.conj().T @ b)        # Galerkin = A-norm minimiser
        assert np.allclose(x, Q @ y, rtol=1e-8, atol=1e-10)
        assert np.linalg.norm(x - xs) <= np.linalg.norm(xs)
    x, it, rel = solvers.cg(lambda z: Ml @ z, b, 500, 1e-12)
    assert rel <= 1e-12 and np.allclose(x, xs, rtol=1e-9)


def test_cg_stopping_rule():
    A = np.diag(np.arange(1.0, 51.0)) + 0j
    b = np.ones(50) + 0j
    x, it, rel = solvers.cg(lambda z: A @ z, b, 1000, 1e-3)
    r = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert rel <= 1e-3 and abs(r - rel) < 1e-8
    _, it2, rel2 = solvers.cg(lambda z: A @ z, b, it - 1, 1e-3)
    assert rel2 > 1e-3                                                  # one fewer step is not enough


def test_power_method_matches_eigvalsh():
    op, *_ = _small_cart(12, 8, 3)
    M = pico.dense_normal(op)
    top = np.linalg.eigvalsh(M)[-1]
    lam = solvers.power_method(lambda x: op.normal(x), (op.ny, op.nx), 400)
    assert abs(lam - top) / top < 1e-6
    x0 = rng.probe(solvers.POWER_SEED, 0, op.ny * op.nx) / np.sqrt(op.ny * op.nx)
    assert abs(solvers.power_method(lambda x: op.normal(x), (op.ny, op.nx), 1)
               - np.linalg.norm(M @ x0)) < 1e-12


# --------------------------------------------------------------------------
# the estimator: unbiasedness (Eqs. 15-17) and per-sample variance (Eq. A1)
# --------------------------------------------------------------------------
def _dense_case():
    op, *_ = _small_cart(12, 8, 3, R=2, acs=2, corr=True, seed=21)
    Sig = pico.dense_cov(pico.dense_normal(op), 0.0)
    return op, Sig


@pytest.mark.parametrize("kind,name", [(rng.PROBE_PHASE, "phase"), (rng.PROBE_RADEMACHER, "rademacher"),
                                       (rng.PROBE_GAUSS, "gauss")])
def test_per_sample_variance_formula(kind, name):
    op, Sig = _dense_case()
    n = Sig.shape[0]
    K = 6000
    D = np.empty((K, n))
    for i in range(K):
        v = rng.probe(99, i, n, kind)
        D[i] = np.real(np.conj(v) * (Sig @ v))
    emp_mean, emp_var = D.mean(axis=0), D.var(axis=0)
    want_var = pico.per_sample_variance(Sig, name)
    diag = np.real(np.diag(Sig))
    # unbiased: mean within 6 standard errors at every voxel
    assert np.all(np.abs(emp_mean - diag) <= 6 * np.sqrt(want_var / K) + 1e-12)
    # variance matches Eq. A1 (real part) to sampling accuracy
    assert np.allclose(emp_var, want_var, rtol=0.12, atol=1e-12)


def test_random_phase_beats_gaussian():
    _, Sig = _dense_case()
    assert np.all(pico.per_sample_variance(Sig, "phase") < pico.per_sample_variance(Sig, "gauss"))


def test_pico_with_cg_band_against_exact_diagonal():
    op, *_ = _small_cart(16, 10, 4, R=2, acs=2, corr=True, seed=5)
    d, _, half = pico.column_exact(op)
    K = 64
    s, _ = pico.pico(op, 2024, 0, K, 0.0, max_iter=200, rtol=1e-12)
    z = (s / K - d) / np.sqrt(half / K)
    assert np.all(np.abs(z) < 6)
    assert np.mean(np.abs(z) > 3) < 0.02


def test_pico_one_probe_exact_for_diagonal_covariance():
    n, nc = 12, 4
    S = synth.coil_maps(n, n, nc, 8)                   # sum |S|^2 = 1
    op = ops.Operator(S, None, mask=np.ones(n, dtype=np.uint8))
    s, _ = pico.pico(op, 5, 0, 1, 0.0, max_iter=50, rtol=1e-13)
    assert np.allclose(s, 1.0, atol=1e-10)


def test_pmr_band_against_exact_diagonal():
    op, *_ = _small_cart(12, 8, 3, R=2, acs=2, corr=True, seed=6)
    d, _, _ = pico.column_exact(op)
    N = 400
    s, _ = pico.pmr(op, 77, 0, N, 1e-2, 0.0, max_iter=200, rtol=1e-12)
    z = (s / N - d) / np.sqrt(d ** 2 / N)            # |x|^2 ~ Exp(Sigma_kk)
    assert np.all(np.abs(z) < 6)
    assert np.mean(np.abs(z) > 3) < 0.03


def test_pmr_noise_is_white_and_masked():
    op, *_ = _small_cart(16, 16, 2, R=2, acs=0, corr=False)
    n = pico.pmr_noise(op, 3, 0, 0.5)
    m = ops.mask2d(op.mask, op.nx)[None].repeat(op.nc, 0) > 0
    assert np.all(n[~m] == 0)
    assert abs(np.mean(np.abs(n[m]) ** 2) - 0.25) < 0.03


def test_lambda_phys_uses_power_estimate():
    op, *_ = _small_cart(12, 8, 3)
    lp, lmax = pico.lambda_phys(op, 0.1, 15, 1.01)
    assert abs(lp - 0.1 * 1.01 * lmax) < 1e-15
    top = np.linalg.eigvalsh(pico.dense_normal(op))[-1]
    assert lmax <= top * (1 + 1e-12) and lmax > 0.5 * top


def test_nrmse_hand_computed():
    # est - ref = (3, -1, 0): ||.|| = sqrt(10); ||ref|| = sqrt(0 + 25 + 4) = sqrt(29)
    est = np.array([3.0, 4.0, 2.0])
    ref = np.array([0.0, 5.0, 2.0])
    assert pico.nrmse(est, ref) == pytest.approx(np.sqrt(10.0 / 29.0), rel=1e-15)
    # over a support: only the last two voxels, (-1, 0) against (5, 2)
    sup = np.array([False, True, True])
    assert pico.nrmse(est, ref, sup) == pytest.approx(1.0 / np.sqrt(29.0), rel=1e-15)
    # a 2-D map and its flattening give the same value; scaling both maps leaves it unchanged
    assert pico.nrmse(est.reshape(3, 1), ref.reshape(3, 1)) == pytest.approx(pico.nrmse(est, ref), rel=1e-15)
    assert pico.nrmse(7 * est, 7 * ref) == pytest.approx(pico.nrmse(est, ref), rel=1e-14)


# --------------------------------------------------------------------------
# per-column CG (phase-encode Cartesian: A^H A block diagonal over columns)
# --------------------------------------------------------------------------
def test_cg_batched_follows_cg_on_every_system():
    g = np.random.default_rng(4)
    n, B = 12, 5
    Z = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    A = Z.conj().T @ Z + 0.3 * np.eye(n)
    rhs = g.standard_normal((n, B)) + 1j * g.standard_normal((n, B))
    rhs[:, 3] = 0.0                                                     # a zero system takes no update
    for max_iter, rtol in ((4, 0.0), (50, 1e-6), (7, 1e-2)):
        X, it, rel = solvers.cg_batched(lambda P: A @ P, rhs, max_iter, rtol)
        for b in range(B):
            x, i1, r1 = solvers.cg(lambda z: A @ z, rhs[:, b], max_iter, rtol)
            assert it[b] == i1
            assert np.allclose(X[:, b], x, rtol=1e-9, atol=1e-12)   # BLAS order only
            if rtol == 1e-6:       # converged: both residuals are rounding-level, below the tolerance
                assert rel[b] <= 1e-6 and r1 <= 1e-6
            else:
                assert abs(rel[b] - r1) <= 1e-9 * r1
    assert it[3] == 0 and np.all(X[:, 3] == 0)


def test_cg_columns_is_global_cg_on_a_single_column():
    S = synth.coil_maps(16, 1, 3, 2)
    op = ops.Operator(S, None, mask=synth.mask_pe(16, 2, 2))
    v = rng.probe(9, 0, 16).reshape(16, 1)
    for k in (1, 4, 9):
        xc, itc, relc = solvers.cg_columns(op, v, 0.02, k)
        xg, itg, relg = solvers.cg(lambda z: op.normal(z, 0.02), v, k)
        assert itc == itg == k
        assert np.allclose(xc, xg, rtol=1e-11, atol=1e-13)
        assert abs(relc - relg) < 1e-11


def test_cg_columns_iterate_is_the_per_column_krylov_minimiser_and_converges():
    op, *_ = _small_cart(12, 5, 3, R=2, acs=2)
    P = ops.pe_projector(op.mask)
    lam = 0.03
    v = rng.probe(5, 1, 12 * 5).reshape(12, 5)
    for k in (1, 3, 5):
        x, it, _ = solvers.cg_columns(op, v, lam, k)
        for col in range(5):
            G = ops.cart_column_normal(op.S, op.mask, col, P) + lam * np.eye(12)
            b = v[:, col]
            K = np.stack([np.linalg.matrix_power(G, j) @ b for j in range(k)], axis=1)
            Q, _ = np.linalg.qr(K)
            y = np.linalg.solve(Q.conj().T @ G @ Q, Q.conj().T @ b)    # Galerkin = G-norm minimiser
            assert np.allclose(x[:, col], Q @ y, rtol=1e-8, atol=1e-10)
    # converged: the exact solve of the whole normal equations (dense M)
    M = pico.dense_normal(op) + lam * np.eye(60)
    xs = np.linalg.solve(M, v.reshape(-1)).reshape(12, 5)
    x, it, rel = solvers.cg_columns(op, v, lam, 200, 1e-13)
    assert rel <= 1e-12 and np.allclose(x, xs, rtol=1e-10, atol=1e-12)


def test_cg_columns_stops_each_column_on_its_own_residual():
    op, *_ = _small_cart(16, 6, 3, R=2, acs=2)
    P = ops.pe_projector(op.mask)
    v = rng.probe(6, 2, 16 * 6).reshape(16, 6)
    v[:, 2] = 0.0
    x, it, rel = solvers.cg_columns(op, v, 0.0, 100, 1e-4)
    assert np.all(x[:, 2] == 0)
    for col in (0, 1, 3, 4, 5):
        G = ops.cart_column_normal(op.S, op.mask, col, P)
        r = np.linalg.norm(v[:, col] - G @ x[:, col]) / np.linalg.norm(v[:, col])
        assert r <= 1e-4
    assert rel <= 1e-4
    # batch of images = images one by one
    vb = np.stack([v, 2 * v + 1j])
    xb, itb, relb = solvers.cg_columns(op, vb, 0.1, 7)
    for i in range(2):
        xi, iti, reli = solvers.cg_columns(op, vb[i], 0.1, 7)
        assert np.allclose(xb[i], xi, rtol=1e-13, atol=1e-15) and itb[i] == iti and abs(relb[i] - reli) < 1e-13


def test_pico_with_column_cg_band_against_exact_diagonal():
    op, *_ = _small_cart(16, 8, 4, R=2, acs=2)
    d, rowe, half = pico.column_exact(op, 0.0)
    K = 400
    s, _ = pico.pico(op, 11, 0, K, 0.0, 60, 0.0, solver="columns")
    z = (s / K - d) / np.sqrt(half / K)
    assert np.all(np.abs(z) < 6) and np.mean(np.abs(z) > 3) < 0.02
    # converged per-column solves and converged global solves give the same per-probe products
    s1, _ = pico.pico(op, 11, 0, 3, 0.0, 200, 1e-12, solver="columns")
    s2, _ = pico.pico(op, 11, 0, 3, 0.0, 200, 1e-12)
    assert np.allclose(s1, s2, rtol=1e-9, atol=1e-12)


def test_spiral_toeplitz_normal_equals_exact_nudft_normal():
    n = 24
    S = synth.coil_maps(n, n, 3, 7)
    traj = synth.spiral_traj(n, 4, 160, 1)
    T = ops.ToeplitzNormal(S, traj)
    op = ops.Operator(S, None, traj=traj)
    g = np.random.default_rng(8)
    for lam in (0.0, 0.3):
        x = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
        want = op.normal(x, lam)
        assert np.allclose(T.apply(x, lam), want, rtol=1e-11, atol=1e-12 * np.abs(want).max())
