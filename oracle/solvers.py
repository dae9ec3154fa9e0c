"""Solvers (oracle side, FP64).

* Conjugate gradients on the normal equations ``(A^H A + lam I) x = rhs``
  (Sec. 2.1.3, Eq. 6; CG-SENSE).  Textbook Hestenes-Stiefel form with
  ``x0 = 0``; the stopping rule is checked after every update:
  stop once ``||r|| <= rtol * ||rhs||`` or after ``max_iter`` updates.
* The same CG run on many independent systems at once (``cg_batched``: one
  step length and one stopping test per system), and per readout column of a
  Cartesian phase-encode operator (``cg_columns``): with a mask on ``ky``
  only, ``A^H A`` is block diagonal over the columns (Sec. 2.1.3 with
  ``F^H M F = (F_y^H M_y F_y) (x) I``), so the normal equations split into
  ``nx`` independent ``ny x ny`` systems, each solved by its own CG.  Its
  iterates differ from CG on the whole image; its fixed point is the same.
* Power method for ``lambda_max(A^H A)`` used for spectral normalisation
  (Sec. 3.2.1 and Sec. 3.3: 15 steps, 1.01 margin).
"""
from __future__ import annotations

import numpy as np

from . import ops, rng

#: seed of the hash-drawn start vector of the power method (a fixed constant of
#: this implementation; the paper does not give a start vector).
POWER_SEED = 0x50574D


def cg(apply, rhs: np.ndarray, max_iter: int, rtol: float = 0.0):
    """Solve ``apply(x) = rhs`` by CG from ``x0 = 0``.

    Returns ``(x, iters, relres)`` where ``relres = ||r|| / ||rhs||``.
    """
    b = np.asarray(rhs, dtype=np.complex128)
    x = np.zeros_like(b)
    r = b.copy()
    rr = float(np.vdot(r, r).real)
    rr0 = rr
    if rr0 == 0.0:
        return x, 0, 0.0
    p = np.zeros_like(b)
    beta = 0.0
    it = 0
    while it < max_iter:
        if rr <= (rtol * rtol) * rr0:
            break
        p = r + beta * p
        q = apply(p)
        pq = float(np.vdot(p, q).real)
        alpha = rr / pq
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(np.vdot(r, r).real)
        beta = rr_new / rr
        rr = rr_new
        it += 1
    return x, it, float(np.sqrt(rr / rr0))


def power_method(apply, shape, iters: int, seed: int = POWER_SEED):
    """Largest eigenvalue of a Hermitian PSD operator by ``iters`` power steps.

    Start: the random-phase probe of index 0 under ``seed``, scaled to unit
    norm.  Each step ``y = apply(x); lam = ||y||; x = y / lam``; the estimate
    is ``lam`` of the last step.
    """
    n = int(np.prod(shape))
    x = rng.probe(seed, 0, n).reshape(shape) / np.sqrt(n)
    lam = 0.0
    for _ in range(iters):
        y = apply(x)
        lam = float(np.linalg.norm(y))
        x = y / lam
    return lam


def cg_batched(apply, rhs: np.ndarray, max_iter: int, rtol: float = 0.0):
    """CG from ``x0 = 0`` on the independent systems ``apply(X)[:, b] = rhs[:, b]``.

    ``rhs`` is ``[n][B]``; ``apply`` maps an ``[n][B]`` block column by column.
    Every system has its own step ``alpha_b = r_b^H r_b / p_b^H q_b`` and
    ``beta_b``, and stops on its own (``||r_b|| <= rtol ||rhs_b||`` or after
    ``max_iter`` updates): each column follows exactly the steps of ``cg``.
    Returns ``(X, iters[B], relres[B])``.
    """
    b = np.asarray(rhs, dtype=np.complex128)
    x = np.zeros_like(b)
    r = b.copy()
    rr = np.real(np.sum(np.conj(r) * r, axis=0))
    rr0 = rr.copy()
    p = np.zeros_like(b)
    beta = np.zeros(b.shape[1])
    iters = np.zeros(b.shape[1], dtype=np.int64)
    for _ in range(max_iter):
        live = rr > (rtol * rtol) * rr0          # systems that take this update
        if not np.any(live):
            break
        p = np.where(live[None, :], r + beta[None, :] * p, p)
        q = apply(p)
        pq = np.real(np.sum(np.conj(p) * q, axis=0))
        alpha = np.where(live, rr / np.where(live, pq, 1.0), 0.0)
        x = x + alpha[None, :] * p
        r = r - alpha[None, :] * q
        rr_new = np.real(np.sum(np.conj(r) * r, axis=0))
        beta = np.where(live, rr_new / np.where(live, rr, 1.0), beta)
        rr = np.where(live, rr_new, rr)
        iters += live
    with np.errstate(invalid="ignore", divide="ignore"):
        relres = np.where(rr0 > 0, np.sqrt(rr / np.where(rr0 > 0, rr0, 1.0)), 0.0)
    return x, iters, relres


def cg_columns(op, rhs: np.ndarray, lam: float, max_iter: int, rtol: float = 0.0, P=None):
    """Per-readout-column CG for a Cartesian phase-encode operator.

    Column ``j`` of every right-hand side is solved against that column's block
    ``G_j + lam I`` with ``G_j = ops.cart_column_normal(...)`` by CG from 0
    (``cg_batched`` over the batch), stopping per column on
    ``||r_j|| <= rtol ||rhs_j||``.  ``rhs``: ``[ny][nx]`` or ``[B][ny][nx]``.
    Returns ``(x, iters, relres)``: ``x`` shaped like ``rhs``; ``iters[B]`` the
    largest number of updates any column of an image took; ``relres[B]`` =
    ``||r|| / ||rhs||`` over the whole image.
    """
    assert op.mask is not None and np.asarray(op.mask).ndim == 1, "phase-encode Cartesian operators only"
    b = np.asarray(rhs, dtype=np.complex128)
    single = b.ndim == 2
    if single:
        b = b[None]
    B, ny, nx = b.shape
    if P is None:
        P = ops.pe_projector(op.mask)
    x = np.zeros_like(b)
    iters = np.zeros(B, dtype=np.int64)
    r2 = np.zeros(B)
    for col in range(nx):
        G = ops.cart_column_normal(op.S, op.mask, col, P) + lam * np.eye(ny)
        xc, it, rel = cg_batched(lambda Z: G @ Z, b[:, :, col].T, max_iter, rtol)
        x[:, :, col] = xc.T
        iters = np.maximum(iters, it)
        # ||r_j||^2 of every image from the column's relative residual
        r2 += (rel ** 2) * np.real(np.sum(np.abs(b[:, :, col]) ** 2, axis=1))
    b2 = np.real(np.sum(np.abs(b) ** 2, axis=(1, 2)))
    relres = np.where(b2 > 0, np.sqrt(r2 / np.where(b2 > 0, b2, 1.0)), 0.0)
    if single:
        return x[0], int(iters[0]), float(relres[0])
    return x, iters, relres
