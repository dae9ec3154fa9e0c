"""Pins of the nonlinear-CS oracle (L1-wavelet FISTA and its Jacobian)."""
import os

import numpy as np
import pytest

import synth
from oracle import cs, ops, pico, rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_db4_filter_matches_published_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "db4_scaling_filter.txt"))
            if l.strip() and not l.startswith("#")]
    want = np.array([float(v) for _, v in rows])
    assert np.allclose(cs.daubechies_filter(4), want, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_daubechies_filters_are_orthonormal_with_vanishing_moments(p):
    h, g = cs.wavelet_filters(p)
    L = len(h)
    assert abs(h.sum() - np.sqrt(2)) < 1e-12
    for m in range(0, L, 2):          # double-shift orthonormality
        assert abs(np.dot(h[: L - m], h[m:]) - (1.0 if m == 0 else 0.0)) < 1e-12
    k = np.arange(L)
    for q in range(p):                # p vanishing moments of the wavelet
        assert abs(np.sum(g * k ** q)) < 1e-8 * max(1, L ** q)


def test_haar_one_level_by_hand():
    h, g = cs.wavelet_filters(1)
    x = np.array([[1.0, 3.0], [5.0, 11.0]])
    c = cs.dwt2(x, 1, h, g)
    # rows: a = (x0 + x1)/sqrt2, d = (x1 - x0)/sqrt2 (g = [-1/sqrt2... sign by g[m] = (-1)^m h[1-m])
    r = np.array([[(1 + 3), (1 * g[0] + 3 * g[1]) * np.sqrt(2)], [(5 + 11), (5 * g[0] + 11 * g[1]) * np.sqrt(2)]]) / np.sqrt(2)
    want = np.array([[r[0, 0] + r[1, 0], r[0, 1] + r[1, 1]],
                     [r[0, 0] * g[0] + r[1, 0] * g[1], r[0, 1] * g[0] + r[1, 1] * g[1]]]) / np.array([[np.sqrt(2)], [1]])
    assert np.allclose(c[0, 0], (1 + 3 + 5 + 11) / 2)
    assert np.allclose(c, want)


@pytest.mark.parametrize("n,levels", [(16, 2), (40, 3), (64, 4)])
def test_dwt_is_orthogonal_and_invertible(n, levels):
    h, g = cs.wavelet_filters(4)
    g_ = np.random.default_rng(0)
    x = g_.standard_normal((n, n)) + 1j * g_.standard_normal((n, n))
    c = cs.dwt2(x, levels, h, g)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-10 * np.linalg.norm(x)
    assert np.allclose(cs.idwt2(c, levels, h, g), x, atol=1e-12)
    y = g_.standard_normal((n, n)) + 0j
    assert abs(np.vdot(cs.dwt2(y, levels, h, g), c) - np.vdot(y, x)) < 1e-9


def test_soft_threshold_tangent_by_finite_differences():
    g_ = np.random.default_rng(1)
    c = g_.standard_normal(200) + 1j * g_.standard_normal(200)
    tau = 0.8
    c = c[np.abs(np.abs(c) - tau) > 1e-3]
    dc = g_.standard_normal(c.shape) + 1j * g_.standard_normal(c.shape)
    eps = 1e-7
    fd = (cs.soft(c + eps * dc, tau) - cs.soft(c - eps * dc, tau)) / (2 * eps)
    assert np.allclose(cs.soft_tangent(c, tau, dc), fd, atol=1e-7)
    # symmetric for Re<.,.>
    e = g_.standard_normal(c.shape) + 1j * g_.standard_normal(c.shape)
    assert abs(np.vdot(e, cs.soft_tangent(c, tau, dc)).real - np.vdot(cs.soft_tangent(c, tau, e), dc).real) < 1e-10


def _cs_case(n=32, nc=4, iters=30, lam_rel=1e-2, seed=3):
    S = synth.coil_maps(n, n, nc, seed)
    mask = synth.poisson_disc_mask(n, n, 2.0, 8, seed)
    op = ops.Operator(S, None, mask=mask)
    x0 = synth.phantom(n, seed).astype(np.complex128)
    b = op.forward(x0)
    h, g = cs.wavelet_filters(4)
    lam = lam_rel * np.abs(cs.dwt2(op.adjoint(b), 3, h, g)).max()
    return op, b, cs.Fista(op, b, lam, iters, levels=3)


def test_fista_converges_to_the_lasso_minimiser():
    op, b, f = _cs_case(iters=400)
    x = f.x
    # optimality: W x is a fixed point of the proximal gradient step
    y = x - (op.normal(x) - op.adjoint(b)) / f.Lc
    fixed = f.WH(cs.soft(f.W(y), f.tau))
    assert np.linalg.norm(fixed - x) <= 1e-5 * np.linalg.norm(x)


def test_jvp_matches_central_differences():
    op, b, f = _cs_case()
    g_ = np.random.default_rng(2)
    db = (g_.standard_normal(b.shape) + 1j * g_.standard_normal(b.shape)) * ops.mask2d(op.mask, op.nx)[None]
    eps = 1e-6 * np.linalg.norm(b) / np.linalg.norm(db)
    fp = cs.Fista(op, b + eps * db, f.lam, f.iters, levels=3).x
    fm = cs.Fista(op, b - eps * db, f.lam, f.iters, levels=3).x
    fd = (fp - fm) / (2 * eps)
    jv = f.jvp(db)
    assert np.linalg.norm(jv - fd) <= 1e-5 * np.linalg.norm(fd)


def test_vjp_is_the_real_adjoint_of_jvp():
    op, b, f = _cs_case(iters=20)
    g_ = np.random.default_rng(3)
    db = (g_.standard_normal(b.shape) + 1j * g_.standard_normal(b.shape)) * ops.mask2d(op.mask, op.nx)[None]
    xb = g_.standard_normal((op.ny, op.nx)) + 1j * g_.standard_normal((op.ny, op.nx))
    lhs = np.vdot(xb, f.jvp(db)).real
    rhs = np.vdot(f.vjp(xb), db).real
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_linear_case_jacobian_is_the_reconstruction_and_sigma():
    # lam = 0: FISTA is linear in b, so J db = f(db); converged, J J^H = M^-1 (Eq. 21)
    S = synth.coil_maps(16, 16, 8, 7)                 # 8 coils: cond(A^H A) ~ 4.5
    op = ops.Operator(S, None, mask=synth.mask_pe(16, 2, 4))
    b = op.forward(synth.phantom(16, 7).astype(np.complex128))
    f = cs.Fista(op, b, 0.0, 300, levels=2)
    g_ = np.random.default_rng(4)
    db = (g_.standard_normal(b.shape) + 1j * g_.standard_normal(b.shape)) * ops.mask2d(op.mask, op.nx)[None]
    lin = cs.Fista(op, db, 0.0, 300, levels=2).x
    assert np.allclose(f.jvp(db), lin, atol=1e-10 * np.abs(lin).max())
    Sig = pico.dense_cov(pico.dense_normal(op))
    v = rng.probe(5, 0, 256).reshape(16, 16)
    u, w = f.jvp(f.vjp(v)).reshape(-1), Sig @ v.reshape(-1)
    assert np.linalg.norm(u - w) <= 1e-10 * np.linalg.norm(w)


def _linear_case(n=16, iters=300):
    S = synth.coil_maps(n, n, 8, 7)
    op = ops.Operator(S, None, mask=synth.mask_pe(n, 2, n // 4))
    b = op.forward(synth.phantom(n, 7).astype(np.complex128))
    return op, b, cs.Fista(op, b, 0.0, iters, levels=2)


def test_jacobian_diag_is_the_covariance_diagonal_in_the_linear_case():
    # lam = 0, converged: J = M^-1 A^H is C-linear, E|J n|^2 = diag(M^-1) (Eqs. 8-10)
    op, b, f = _linear_case(n=8, iters=200)
    want = np.real(np.diag(pico.dense_cov(pico.dense_normal(op)))).reshape(op.ny, op.nx)
    assert np.allclose(cs.jacobian_diag(f), want, rtol=1e-7)


def test_cs_pmr_linear_case_is_the_reconstruction_of_the_noise():
    # lam = 0: f(b + n) - f(b) = f(n) = J n exactly, so each sample is |J n_i|^2 / sigma^2
    op, b, f = _linear_case(iters=60)
    sigma = 0.3
    s, ss = cs.pmr_cs(f, 11, 2, 3, sigma)
    ws, wss = np.zeros_like(s), np.zeros_like(s)
    for i in range(2, 5):
        d = np.abs(f.jvp(pico.pmr_noise(op, 11, i, sigma))) ** 2 / sigma ** 2
        ws += d
        wss += d * d
    assert np.allclose(s, ws, rtol=1e-9) and np.allclose(ss, wss, rtol=1e-9)


def test_cs_pmr_small_noise_limit_is_the_tangent():
    # nonlinear f: (f(b + sigma n) - f(b)) / sigma -> J n as sigma -> 0 (first order in sigma)
    op, b, f = _cs_case(n=16, nc=4, iters=20)
    n1 = pico.pmr_noise(op, 5, 0, 1.0)
    jn = f.jvp(n1)
    for sigma, bound in [(1e-4, 1e-3), (1e-6, 1e-5)]:
        s, _ = cs.pmr_cs(f, 5, 0, 1, sigma)
        assert np.linalg.norm(np.sqrt(s) - np.abs(jn)) <= bound * np.linalg.norm(jn)


def test_jacobian_pico_and_cs_pmr_are_unbiased_for_the_jacobian_diagonal():
    # Sec. 2.2.5: both estimate E|J n|^2; band from each estimator's own sample variance
    op, b, f = _cs_case(n=16, nc=4, iters=12)
    exact = cs.jacobian_diag(f)
    K = 300
    for s, ss in (cs.pico_cs(f, 21, 0, K), cs.pmr_cs(f, 22, 0, K, 1e-6)):
        mean = s / K
        var = (ss / K - mean ** 2) * K / (K - 1)
        z = (mean - exact) / np.sqrt(var / K)
        assert np.abs(z).max() <= 6.0
        assert np.mean(np.abs(z) > 3.0) <= 0.02
