"""Nonlinear compressed-sensing reconstruction and its Jacobian (oracle, FP64).

Sec. 2.2.5 linearises a nonlinear reconstruction ``f: b_w -> x`` at the
noise-free data ``k0 = A x`` and probes ``Sigma ~ J_f J_f^H``.  The
reconstruction here is L1-wavelet FISTA (Beck & Teboulle 2009; the paper's
FISTA of Sec. 3.2.3 with a Daubechies-4 wavelet penalty in place of TV):

    min_x  1/2 ||A x - b||^2 + lam ||W x||_1 ,   W orthonormal periodised 2-D DWT.

FISTA from ``x_0 = z_0 = 0``, ``t_0 = 1``, step ``1/Lc`` with
``Lc = 1.01 lambda_max(A^H A)`` (Sec. 3.3):

    y_k     = z_k - (A^H A z_k - A^H b) / Lc
    x_{k+1} = W^H S_tau(W y_k),            tau = lam / Lc
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
    z_{k+1} = x_{k+1} + c_k (x_{k+1} - x_k),  c_k = (t_k - 1) / t_{k+1}

with the complex soft threshold ``S_tau(c) = c max(0, 1 - tau/|c|)``.  The
map is R-linear in the tangent (not C-linear): the derivative of ``S_tau`` at
``c`` with ``|c| > tau`` and ``u = c/|c|`` is
``dS[dc] = (1 - tau/|c|) dc + (tau/|c|) u Re(conj(u) dc)`` (zero for
``|c| <= tau``), a symmetric map for the real inner product ``Re<a, b>``.

``jvp`` propagates a k-space tangent through the stored iterations;
``vjp`` is its adjoint for ``Re<.,.>`` (reverse sweep).  PICO for the
nonlinear reconstruction accumulates ``Re(conj(v) J J^T v)`` (Alg. 1 with the
covariance product replaced by Jacobian products, Sec. 2.2.5).
"""
from __future__ import annotations

import math

import numpy as np

from . import ops, pico, rng, solvers


# ----------------------------------------------------------------------------
# Daubechies filters by spectral factorisation (Daubechies 1988)
# ----------------------------------------------------------------------------
def daubechies_filter(p: int) -> np.ndarray:
    """Scaling filter (2p taps, sum sqrt(2)) of the orthonormal wavelet with p vanishing moments.

    ``|m0(w)|^2 = cos^{2p}(w/2) P(sin^2(w/2))`` with ``P(y) = sum_{k<p} C(p-1+k, k) y^k``.
    With ``z = e^{iw}``, ``sin^2(w/2) = (2 - z - 1/z)/4``; the roots of
    ``z^{p-1} P(.)`` come in pairs ``(r, 1/r)``; keeping those inside the unit
    circle gives the minimum-phase factor, multiplied by ``((1 + z)/2)^p``.
    """
    # polynomial in z (ascending powers) of z^{p-1} * P((2 - z - 1/z)/4)
    q = np.polynomial.polynomial
    acc = np.zeros(2 * p - 1)
    base = np.array([-1.0, 2.0, -1.0]) / 4.0          # (-1 + 2z - z^2)/4 = z * (2 - z - 1/z)/4
    for k in range(p):
        term = np.array([math.comb(p - 1 + k, k)], dtype=float)
        for _ in range(k):
            term = q.polymul(term, base)
        term = q.polymul(term, np.eye(1, p - k, p - 1 - k)[0])   # times z^{p-1-k}
        acc[: len(term)] += term
    roots = q.polyroots(acc)
    inside = roots[np.abs(roots) < 1.0]
    h = np.real(np.poly(inside))                      # descending powers == coefficients of z^-n
    for _ in range(p):
        h = np.convolve(h, [1.0, 1.0])
    h = h / h.sum() * math.sqrt(2.0)
    return h


def wavelet_filters(p: int = 4):
    """(scaling h, wavelet g) with ``g[m] = (-1)^m h[L-1-m]``."""
    h = daubechies_filter(p)
    L = len(h)
    g = np.array([(-1) ** m * h[L - 1 - m] for m in range(L)])
    return h, g


# ----------------------------------------------------------------------------
# Periodised orthonormal 2-D DWT
# ----------------------------------------------------------------------------
def _analysis_1d(x: np.ndarray, h, g, axis: int) -> np.ndarray:
    """``a[k] = sum_m h[m] x[(2k+m) mod n]``, ``d[k] = sum_m g[m] x[(2k+m) mod n]`` -> [a | d]."""
    x = np.moveaxis(x, axis, -1)
    n = x.shape[-1]
    a = np.zeros(x.shape[:-1] + (n // 2,), dtype=complex)
    d = np.zeros_like(a)
    k = np.arange(n // 2)
    for m in range(len(h)):
        xm = x[..., (2 * k + m) % n]
        a += h[m] * xm
        d += g[m] * xm
    return np.moveaxis(np.concatenate([a, d], axis=-1), -1, axis)


def _synthesis_1d(c: np.ndarray, h, g, axis: int) -> np.ndarray:
    """Transpose of ``_analysis_1d`` (its inverse for an orthonormal filter pair)."""
    c = np.moveaxis(c, axis, -1)
    n = c.shape[-1]
    a, d = c[..., : n // 2], c[..., n // 2:]
    x = np.zeros(c.shape, dtype=complex)
    k = np.arange(n // 2)
    for m in range(len(h)):
        np.add.at(x, (..., (2 * k + m) % n), h[m] * a + g[m] * d)
    return np.moveaxis(x, -1, axis)


def dwt2(x: np.ndarray, levels: int, h, g) -> np.ndarray:
    """J-level 2-D DWT; coefficients in place (the approximation band top-left)."""
    c = np.array(x, dtype=complex)
    ny, nx = c.shape
    for _ in range(levels):
        sub = c[:ny, :nx]
        sub = _analysis_1d(sub, h, g, axis=1)
        sub = _analysis_1d(sub, h, g, axis=0)
        c[:ny, :nx] = sub
        ny, nx = ny // 2, nx // 2
    return c


def idwt2(c: np.ndarray, levels: int, h, g) -> np.ndarray:
    x = np.array(c, dtype=complex)
    shapes = []
    ny, nx = x.shape
    for _ in range(levels):
        shapes.append((ny, nx))
        ny, nx = ny // 2, nx // 2
    for ny, nx in reversed(shapes):
        sub = x[:ny, :nx]
        sub = _synthesis_1d(sub, h, g, axis=0)
        sub = _synthesis_1d(sub, h, g, axis=1)
        x[:ny, :nx] = sub
    return x


# ----------------------------------------------------------------------------
# soft threshold and its tangent
# ----------------------------------------------------------------------------
def soft(c: np.ndarray, tau: float) -> np.ndarray:
    a = np.abs(c)
    return np.where(a > tau, c * (1.0 - tau / np.where(a > 0, a, 1.0)), 0.0)


def soft_tangent(c: np.ndarray, tau: float, dc: np.ndarray) -> np.ndarray:
    """Derivative of ``soft`` at ``c`` applied to ``dc`` (R-linear, symmetric)."""
    a = np.abs(c)
    act = a > tau
    aa = np.where(act, a, 1.0)
    u = c / aa
    out = (1.0 - tau / aa) * dc + (tau / aa) * u * np.real(np.conj(u) * dc)
    return np.where(act, out, 0.0)


# ----------------------------------------------------------------------------
# FISTA and its Jacobian
# ----------------------------------------------------------------------------
class Fista:
    """L1-wavelet FISTA on a whitened operator; keeps the trajectory for J."""

    def __init__(self, op: ops.Operator, b: np.ndarray, lam: float, iters: int, levels: int = 4,
                 power_iters: int = 15, margin: float = 1.01, p: int = 4):
        self.op, self.b, self.lam, self.iters, self.levels = op, np.asarray(b, dtype=complex), lam, iters, levels
        self.h, self.g = wavelet_filters(p)
        lmax = solvers.power_method(lambda x: op.normal(x), (op.ny, op.nx), power_iters)
        self.Lc = margin * lmax
        self.tau = lam / self.Lc
        t = [1.0]
        for _ in range(iters):
            t.append((1.0 + math.sqrt(1.0 + 4.0 * t[-1] ** 2)) / 2.0)
        self.c = [(t[k] - 1.0) / t[k + 1] for k in range(iters)]
        self.Ahb = op.adjoint(self.b)
        self.Wy = []          # W y_k for k = 0..iters-1 (the points where S is differentiated)
        self.x = self._run()

    def W(self, x):
        return dwt2(x, self.levels, self.h, self.g)

    def WH(self, c):
        return idwt2(c, self.levels, self.h, self.g)

    def _run(self, Ahb=None, keep=True):
        """The FISTA iterations for the data term ``A^H b`` (the stored one by default)."""
        op = self.op
        Ahb = self.Ahb if Ahb is None else Ahb
        x = np.zeros((op.ny, op.nx), dtype=complex)
        z = x.copy()
        for k in range(self.iters):
            y = z - (op.normal(z) - Ahb) / self.Lc
            wy = self.W(y)
            if keep:
                self.Wy.append(wy)
            xn = self.WH(soft(wy, self.tau))
            z = xn + self.c[k] * (xn - x)
            x = xn
        return x

    def recon(self, b: np.ndarray) -> np.ndarray:
        """``f(b)`` with this reconstruction's weight, step and iteration count."""
        return self._run(self.op.adjoint(np.asarray(b, dtype=complex)), keep=False)

    def jvp(self, db: np.ndarray) -> np.ndarray:
        """``J db``: tangent of the reconstruction for a k-space tangent ``db``."""
        op = self.op
        Ahdb = op.adjoint(np.asarray(db, dtype=complex))
        dx = np.zeros((op.ny, op.nx), dtype=complex)
        dz = dx.copy()
        for k in range(self.iters):
            dy = dz - (op.normal(dz) - Ahdb) / self.Lc
            dxn = self.WH(soft_tangent(self.Wy[k], self.tau, self.W(dy)))
            dz = dxn + self.c[k] * (dxn - dx)
            dx = dxn
        return dx

    def vjp(self, xbar: np.ndarray) -> np.ndarray:
        """``J^T xbar`` for the real inner product ``Re<.,.>`` (reverse sweep)."""
        op = self.op
        K = self.iters
        xb = [None] * (K + 1)
        xb[K] = np.asarray(xbar, dtype=complex).copy()
        zb = np.zeros((op.ny, op.nx), dtype=complex)       # cotangent of z_{k+1}
        ybsum = np.zeros((op.ny, op.nx), dtype=complex)
        for k in range(K - 1, -1, -1):
            xk1 = xb[k + 1] + (1.0 + self.c[k]) * zb
            xb[k] = -self.c[k] * zb
            yb = self.WH(soft_tangent(self.Wy[k], self.tau, self.W(xk1)))
            zb = yb - op.normal(yb) / self.Lc
            ybsum += yb
        return op.forward(ybsum / self.Lc)


def pico_cs(fista: Fista, seed: int, probe_begin: int, nprobes: int, kind: int = rng.PROBE_PHASE):
    """Running sums of Alg. 1 with ``Sigma v`` replaced by ``J (J^T v)`` (Sec. 2.2.5)."""
    ny, nx = fista.op.ny, fista.op.nx
    s = np.zeros((ny, nx))
    ss = np.zeros((ny, nx))
    for i in range(probe_begin, probe_begin + nprobes):
        v = rng.probe(seed, i, ny * nx, kind).reshape(ny, nx)
        u = fista.jvp(fista.vjp(v))
        d = np.real(np.conj(v) * u)
        s += d
        ss += d * d
    return s, ss


def pmr_cs(fista: Fista, seed: int, rep_begin: int, nreps: int, sigma: float):
    """PMR for the nonlinear reconstruction (Sec. 3.2.3): running sums of
    ``d_i = |f(b + n_i) - f(b)|^2 / sigma^2`` with ``n_i`` the whitened k-space
    noise of replica ``i`` (the same draw as the linear PMR), ``f(b)`` the
    stored reconstruction."""
    ny, nx = fista.op.ny, fista.op.nx
    s = np.zeros((ny, nx))
    ss = np.zeros((ny, nx))
    for i in range(rep_begin, rep_begin + nreps):
        n = pico.pmr_noise(fista.op, seed, i, sigma)
        d = np.abs(fista.recon(fista.b + n) - fista.x) ** 2 / sigma ** 2
        s += d
        ss += d * d
    return s, ss


def jacobian_diag(fista: Fista) -> np.ndarray:
    """Exact target of Jacobian PICO and of small-noise PMR (Sec. 2.2.5):
    ``E|J n|_k^2`` for ``n ~ CN(0, I)``, which for the R-linear ``J`` is
    ``1/2 (||J^T e_k||^2 + ||J^T (i e_k)||^2)`` with ``J^T`` the adjoint for
    ``Re<.,.>``; one VJP per real and per imaginary unit image."""
    ny, nx = fista.op.ny, fista.op.nx
    out = np.zeros(ny * nx)
    for k in range(ny * nx):
        e = np.zeros(ny * nx, dtype=complex)
        e[k] = 1.0
        r = fista.vjp(e.reshape(ny, nx))
        e[k] = 1j
        i = fista.vjp(e.reshape(ny, nx))
        out[k] = 0.5 * (np.vdot(r, r).real + np.vdot(i, i).real)
    return out.reshape(ny, nx)
