"""Solvers (oracle side, FP64).

* Conjugate gradients on the normal equations ``(A^H A + lam I) x = rhs``
  (Sec. 2.1.3, Eq. 6; CG-SENSE).  Textbook Hestenes-Stiefel form with
  ``x0 = 0``; the stopping rule is checked after every update:
  stop once ``||r|| <= rtol * ||rhs||`` or after ``max_iter`` updates.
* Power method for ``lambda_max(A^H A)`` used for spectral normalisation
  (Sec. 3.2.1 and Sec. 3.3: 15 steps, 1.01 margin).
"""
from __future__ import annotations

import numpy as np

from . import rng

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
