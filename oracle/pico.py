"""PICO, PMR and exact covariance diagonals (oracle side, FP64).

* Image-domain noise covariance of the Tikhonov CG-SENSE reconstruction
  ``Sigma = (M + lam I)^-1 M (M + lam I)^-1``, ``M = A^H A`` (Sec. 2.1.4,
  Eq. 8; ``Sigma = M^-1`` for ``lam = 0``, Eq. 9); variance map
  ``diag(Sigma)`` (Eq. 10); g-factor (Eq. 11).
* PICO estimate ``(1/N) sum_i Re(conj(v_i) * (Sigma v_i))`` (Eqs. 12-14,
  Alg. 1), where ``Sigma v`` is applied implicitly: one CG solve when
  ``lam = 0``; solve, ``A^H A``, solve when ``lam > 0`` (Sec. 2.2.3).
* PMR (Sec. 1 "Pseudo Multiple Replica"; Sec. 3.2.2): replica ``i`` draws
  whitened k-space noise ``n_i ~ CN(0, sigma^2 I)`` on the sampled positions,
  reconstructs ``x_i = (M + lam I)^-1 A^H n_i`` (the linear recon of ``b + n``
  minus that of ``b``), and averages ``|x_i|^2 / sigma^2``.
* Per-sample variances of ``Re delta_k`` for each probe family (App. B,
  Eq. A1 restated for the real part that Alg. 1 keeps).
"""
from __future__ import annotations

import numpy as np

from . import ops, rng, solvers


def lambda_phys(op: ops.Operator, lam_rel: float, power_iters: int = 15,
                margin: float = 1.01) -> tuple[float, float]:
    """Tikhonov weight in physical units, ``lam_rel * margin * lambda_max``.

    Reading: the paper normalises every forward operator by a 15-step power
    estimate of ``lambda_max`` times 1.01 (Sec. 3.3) and quotes ``lam = 0.1``
    (Sec. 3.2.2) for that normalised operator; maps are reported for ``A``
    itself.  Returns ``(lam_phys, lambda_max)``; ``power_iters = 0`` takes
    ``lam_rel`` as physical.
    """
    if power_iters <= 0:
        return float(lam_rel), 0.0
    lmax = solvers.power_method(lambda x: op.normal(x), (op.ny, op.nx), power_iters)
    return float(lam_rel) * margin * lmax, lmax


# ----------------------------------------------------------------------------
# Exact covariance (dense, tiny images) -- Eqs. 8-10
# ----------------------------------------------------------------------------
def dense_normal(op: ops.Operator) -> np.ndarray:
    """Dense ``M = A^H A``.  Cartesian: from the explicit encoding matrix.
    Spiral: ``M[r, r'] = sum_c conj(S_c[r]) S_c[r'] h(r - r')`` with the NUDFT
    point-spread function ``h(d) = (1/n^2) sum_m exp(+2 pi i k_m . d / n)``
    (the entries of ``E^H E`` written out), which avoids forming ``A``."""
    if op.kind != "spiral":
        A = op.matrix()
        return A.conj().T @ A
    n = op.ny
    k = np.asarray(op.traj, dtype=np.float64)
    d = np.arange(-(n - 1), n, dtype=np.float64)
    ex = np.exp(2j * np.pi * np.outer(k[:, 0], d) / n)          # [M][dx]
    ey = np.exp(2j * np.pi * np.outer(k[:, 1], d) / n)          # [M][dy]
    h = (ey.T @ ex) / n ** 2                                     # h[dy + n-1, dx + n-1]
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ry, rx = yy.reshape(-1), xx.reshape(-1)
    H = h[(ry[:, None] - ry[None, :]) + n - 1, (rx[:, None] - rx[None, :]) + n - 1]
    Sf = op.S.reshape(op.nc, -1)
    G = np.einsum("cr,cs->rs", np.conj(Sf), Sf)
    return G * H


def dense_cov(M: np.ndarray, lam: float = 0.0) -> np.ndarray:
    """``Sigma = (M + lam I)^-1 M (M + lam I)^-1`` (Eq. 8; Eq. 9 at lam = 0)."""
    n = M.shape[0]
    if lam == 0.0:
        return np.linalg.inv(M)
    Ri = np.linalg.inv(M + lam * np.eye(n))
    return Ri @ M @ Ri


def column_exact(op: ops.Operator, lam: float = 0.0):
    """Exact ``diag(Sigma)`` and row energies ``sum_l |Sigma_kl|^2`` per voxel for a
    Cartesian phase-encode mask, by one dense ``ny x ny`` inverse per readout column
    (``A^H A`` is block diagonal over columns, see ``ops.cart_column_normal``).

    Returns ``(diag, rowenergy, offdiag_half)`` as ``[ny][nx]`` float64 arrays,
    where ``offdiag_half = 1/2 sum_{l != k} |Sigma_kl|^2`` is the random-phase
    per-sample variance of ``Re delta_k``.
    """
    assert op.mask is not None and op.mask.ndim == 1
    ny, nx = op.ny, op.nx
    diag = np.zeros((ny, nx))
    rowe = np.zeros((ny, nx))
    P = ops.pe_projector(op.mask)
    for col in range(nx):
        M = ops.cart_column_normal(op.S, op.mask, col, P)
        Sig = dense_cov(M, lam)
        d = np.real(np.diag(Sig))
        diag[:, col] = d
        rowe[:, col] = np.sum(np.abs(Sig) ** 2, axis=1)
    return diag, rowe, 0.5 * (rowe - diag ** 2)


def sense_closed_form(smaps: np.ndarray, R: int):
    """Closed-form SENSE variance and g-factor for uniform ``R``-fold phase-encode
    undersampling keeping ``ky = 0 (mod R)`` and no calibration lines
    (Pruessmann et al. 1999, the paper's analytic reference, Sec. 3.2.1).

    With orthonormal DFTs, ``F_y^H M_y F_y`` averages the ``R`` voxels of an alias
    set ``{y + j ny/R}``; hence on each alias set ``A^H A = (1/R) S_set^H S_set``
    (``S_set``: ``nc x R``) and ``sigma^2 = R [(S^H S)^-1]_rr``; the fully sampled
    reference has ``sigma_ref^2 = 1 / sum_c |S_c|^2`` and
    ``g = sqrt([(S^H S)^-1]_rr [S^H S]_rr)`` (Eq. 11).

    Returns ``(var_acc, var_ref, g)``, each ``[ny][nx]``.
    """
    S = np.asarray(smaps, dtype=np.complex128)
    nc, ny, nx = S.shape
    assert ny % R == 0
    step = ny // R
    var = np.zeros((ny, nx))
    g = np.zeros((ny, nx))
    for x in range(nx):
        for y0 in range(step):
            ys = [y0 + j * step for j in range(R)]
            Ss = S[:, ys, x]                       # nc x R
            G = Ss.conj().T @ Ss
            Gi = np.linalg.inv(G)
            for j, y in enumerate(ys):
                var[y, x] = R * Gi[j, j].real
                g[y, x] = np.sqrt(Gi[j, j].real * G[j, j].real)
    var_ref = 1.0 / np.sum(np.abs(S) ** 2, axis=0)
    return var, var_ref, g


# ----------------------------------------------------------------------------
# Implicit covariance application (Sec. 2.2.3) and PICO (Alg. 1)
# ----------------------------------------------------------------------------
def solve(op: ops.Operator, rhs: np.ndarray, lam: float, max_iter: int, rtol: float = 0.0,
          solver: str = "global") -> np.ndarray:
    """``(M + lam I)^-1 rhs`` by CG from 0 (Eq. 6): ``solver = "global"`` runs
    CG on the whole image (``solvers.cg``), ``"columns"`` runs it on every
    readout column's block of a phase-encode Cartesian operator
    (``solvers.cg_columns``: same fixed point, other iterates)."""
    if solver == "columns":
        return solvers.cg_columns(op, rhs, lam, max_iter, rtol)[0]
    assert solver == "global", solver
    return solvers.cg(lambda z: op.normal(z, lam), rhs, max_iter, rtol)[0]


def apply_sigma(op: ops.Operator, v: np.ndarray, lam: float, max_iter: int, rtol: float = 0.0,
                solver: str = "global"):
    """``u = Sigma v`` via CG on the normal equations.

    ``lam = 0``: ``u = M^-1 v`` (one solve).  ``lam > 0``:
    ``u = (M + lam)^-1 M (M + lam)^-1 v`` (solve, apply ``M``, solve).
    """
    x1 = solve(op, v, lam, max_iter, rtol, solver)
    if lam == 0.0:
        return x1
    w = op.normal(x1, 0.0)
    return solve(op, w, lam, max_iter, rtol, solver)


def pico(op: ops.Operator, seed: int, probe_begin: int, nprobes: int, lam: float,
         max_iter: int, rtol: float = 0.0, kind: int = rng.PROBE_PHASE, sigma_apply=None,
         solver: str = "global"):
    """Running sums of Alg. 1 over probes ``probe_begin .. probe_begin+nprobes-1``.

    Returns ``(s, ss)`` with ``s = sum_i Re(conj(v_i) u_i)`` and
    ``ss = sum_i Re(conj(v_i) u_i)^2`` (both ``[ny][nx]`` float64);
    the variance map is ``s / nprobes`` (Alg. 1 output, real part kept).
    ``sigma_apply`` replaces the CG application (e.g. a dense ``Sigma``);
    ``solver`` picks the CG of ``solve``.
    """
    ny, nx = op.ny, op.nx
    s = np.zeros((ny, nx))
    ss = np.zeros((ny, nx))
    for i in range(probe_begin, probe_begin + nprobes):
        v = rng.probe(seed, i, ny * nx, kind).reshape(ny, nx)
        if sigma_apply is None:
            u = apply_sigma(op, v, lam, max_iter, rtol, solver)
        else:
            u = sigma_apply(v)
        d = np.real(np.conj(v) * u)
        s += d
        ss += d * d
    return s, ss


def pmr_noise(op: ops.Operator, seed: int, rep: int, sigma: float) -> np.ndarray:
    """Whitened k-space noise of replica ``rep`` (zero at unsampled Cartesian positions)."""
    idx = op.kspace_index()
    n = rng.cnoise(seed, rep, idx.reshape(-1), sigma).reshape(idx.shape)
    if op.kind == "cartesian":
        n = n * ops.mask2d(op.mask, op.nx)[None]
    return n


def pmr(op: ops.Operator, seed: int, rep_begin: int, nreps: int, sigma: float, lam: float,
        max_iter: int, rtol: float = 0.0, solver: str = "global"):
    """Running sums of PMR: ``s = sum_i |x_i|^2 / sigma^2``, ``ss = sum_i (|x_i|^2/sigma^2)^2``."""
    ny, nx = op.ny, op.nx
    s = np.zeros((ny, nx))
    ss = np.zeros((ny, nx))
    for i in range(rep_begin, rep_begin + nreps):
        n = pmr_noise(op, seed, i, sigma)
        b = op.adjoint(n)
        x = solve(op, b, lam, max_iter, rtol, solver)
        d = np.abs(x) ** 2 / sigma ** 2
        s += d
        ss += d * d
    return s, ss


# ----------------------------------------------------------------------------
# Per-sample variances of Re(delta_k) (App. B, Eq. A1, real part)
# ----------------------------------------------------------------------------
def per_sample_variance(Sig: np.ndarray, kind: str) -> np.ndarray:
    """Exact variance of one sample ``Re(conj(v_k) (Sigma v)_k)`` at every voxel.

    random phase:   1/2 sum_{l!=k} |S_kl|^2
    real Rademacher:    sum_{l!=k} (Re S_kl)^2
    complex Gaussian: S_kk^2 + 1/2 sum_{l!=k} |S_kl|^2
    PMR (|x_k|^2, x ~ CN(0, Sigma)): S_kk^2
    """
    d = np.real(np.diag(Sig))
    off = np.abs(Sig) ** 2
    np.fill_diagonal(off, 0.0)
    half_off = 0.5 * off.sum(axis=1)
    if kind == "phase":
        return half_off
    if kind == "rademacher":
        re = np.real(Sig) ** 2
        np.fill_diagonal(re, 0.0)
        return re.sum(axis=1)
    if kind == "gauss":
        return d ** 2 + half_off
    if kind == "pmr":
        return d ** 2
    raise ValueError(kind)


def nrmse(est: np.ndarray, ref: np.ndarray, support=None) -> float:
    """``||est - ref||_2 / ||ref||_2`` over ``support`` (all voxels by default)."""
    e, r = np.asarray(est, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    if support is not None:
        e, r = e[support], r[support]
    return float(np.linalg.norm(e - r) / np.linalg.norm(r))


def gfactor(var_acc: np.ndarray, var_ref: np.ndarray, R: float) -> np.ndarray:
    """``g = sigma_acc / (sqrt(R) sigma_ref)`` (Eq. 11)."""
    return np.sqrt(np.asarray(var_acc) / (R * np.asarray(var_ref)))
