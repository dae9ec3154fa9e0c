"""Encoding operators (oracle side, FP64).

Forward model ``b = A x + n`` (Sec. 2.1.1, Eq. 1) after pre-whitening
(Sec. 2.1.2, Eq. 3): ``A = L^-1 A~`` with ``L L^H = Sigma_n``.  Because the
sampling pattern is the same for every coil, ``L^-1`` (which mixes coils at
each k-space sample) folds into the sensitivities:
``S'_c = sum_c' (L^-1)_{c c'} S_c'``.

Readings fixed here (the paper leaves them open):
* Fourier transforms are orthonormal (unit-norm DFT rows); the NUDFT carries
  ``1/sqrt(ny nx)`` so a grid-aligned trajectory reproduces the FFT
  (Sec. 3.3, "Cartesian operators used the same NUFFT framework with
  grid-aligned trajectories").
* No density compensation inside ``A``: the least-squares problem of Eq. 4 is
  unweighted so that whitened noise stays white.
* Cartesian masks index the natural-order DFT frequency ``ky``; a
  phase-encode mask samples every ``kx`` of a kept ``ky`` line.
* Spiral voxel coordinates are ``x, y = 0..n-1``; trajectories are in cycles
  per field of view.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# Pre-whitening, Sec. 2.1.2 (Eq. 3) and App. D remark (i)
# ----------------------------------------------------------------------------
def whiten(smaps: np.ndarray, noise_cov: np.ndarray | None) -> np.ndarray:
    """Whitened sensitivities ``S' = L^-1 S`` with ``L`` the Cholesky factor of Sigma_n."""
    S = np.asarray(smaps, dtype=np.complex128)
    if noise_cov is None:
        return S.copy()
    L = np.linalg.cholesky(np.asarray(noise_cov, dtype=np.complex128))
    Linv = np.linalg.inv(L)
    return np.einsum("cd,dyx->cyx", Linv, S)


# ----------------------------------------------------------------------------
# Cartesian SENSE encoding (Sec. 2.1.1; Sec. 3.2.1 phase-encode undersampling)
# ----------------------------------------------------------------------------
def mask2d(mask: np.ndarray, nx: int) -> np.ndarray:
    m = np.asarray(mask)
    if m.ndim == 1:
        m = np.repeat(m[:, None], nx, axis=1)
    return m.astype(np.float64)


def cart_forward(x: np.ndarray, S: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """``A x``: coil images, orthonormal 2-D DFT, sampling mask -> ``[nc][ny][nx]``."""
    m = mask2d(mask, S.shape[2])
    return np.fft.fft2(S * x[None], norm="ortho") * m[None]


def cart_adjoint(y: np.ndarray, S: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """``A^H y``: mask, orthonormal inverse DFT, conjugate coil combine."""
    m = mask2d(mask, S.shape[2])
    return np.sum(np.conj(S) * np.fft.ifft2(y * m[None], norm="ortho"), axis=0)


def cart_normal(x: np.ndarray, S: np.ndarray, mask: np.ndarray, lam: float = 0.0) -> np.ndarray:
    """``(A^H A + lam I) x`` (Eq. 6 left-hand side)."""
    return cart_adjoint(cart_forward(x, S, mask), S, mask) + lam * x


def dft_matrix(n: int) -> np.ndarray:
    """Orthonormal DFT matrix from its definition ``F[k, j] = exp(-2 pi i k j / n) / sqrt(n)``."""
    k = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(k, k) / n) / np.sqrt(n)


def cart_matrix(S: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """Explicit encoding matrix ``A`` (rows = sampled (c, ky, kx), cols = voxels y*nx+x).

    Built from the DFT definition, not an FFT; only for tiny images.
    """
    nc, ny, nx = S.shape
    Fy, Fx = dft_matrix(ny), dft_matrix(nx)
    F2 = np.kron(Fy, Fx)                       # rows (ky, kx), cols (y, x)
    m = mask2d(mask, nx).reshape(-1) > 0
    rows = []
    for c in range(nc):
        rows.append(F2[m] * S[c].reshape(-1)[None, :])
    return np.concatenate(rows, axis=0)


def pe_projector(mask_1d: np.ndarray) -> np.ndarray:
    """``P = F_y^H diag(mask) F_y`` from the DFT definition (dense ``ny x ny``)."""
    Fy = dft_matrix(len(mask_1d))
    return Fy.conj().T @ (np.asarray(mask_1d, dtype=np.float64)[:, None] * Fy)


def cart_column_normal(S: np.ndarray, mask_1d: np.ndarray, col: int, P: np.ndarray | None = None) -> np.ndarray:
    """Dense ``A^H A`` restricted to readout column ``col`` for a phase-encode mask.

    With a mask on ``ky`` only, ``F^H M F = (F_y^H M_y F_y) (x) I_x``, so
    ``A^H A`` acts on each column independently as
    ``sum_c diag(S_c[:, col])^H P diag(S_c[:, col])``, ``P = F_y^H M_y F_y``.
    """
    ny = S.shape[1]
    if P is None:
        P = pe_projector(mask_1d)
    M = np.zeros((ny, ny), dtype=np.complex128)
    for c in range(S.shape[0]):
        s = S[c, :, col]
        M += np.conj(s)[:, None] * P * s[None, :]
    return M


# ----------------------------------------------------------------------------
# Non-Cartesian (spiral) encoding: exact NUDFT (Sec. 3.2.2; readings above)
# ----------------------------------------------------------------------------
class Nudft:
    """Exact NUDFT ``E[m, (y, x)] = exp(-2 pi i (kx_m x + ky_m y) / n) / n`` for an n x n image."""

    def __init__(self, traj: np.ndarray, n: int):
        t = np.asarray(traj, dtype=np.float64)
        self.n = n
        r = np.arange(n, dtype=np.float64)
        self.ex = np.exp(-2j * np.pi * np.outer(t[:, 0], r) / n) / np.sqrt(n)   # [M][x]
        self.ey = np.exp(-2j * np.pi * np.outer(t[:, 1], r) / n) / np.sqrt(n)   # [M][y]

    def forward(self, z: np.ndarray) -> np.ndarray:
        """``(E z)[m] = sum_{y,x} ey[m,y] ex[m,x] z[y,x]``."""
        t = z @ self.ex.T                      # [y][m]
        return np.einsum("my,ym->m", self.ey, t)

    def adjoint(self, w: np.ndarray) -> np.ndarray:
        """``(E^H w)[y,x] = sum_m conj(ey[m,y]) conj(ex[m,x]) w[m]``."""
        return (np.conj(self.ey).T * w[None, :]) @ np.conj(self.ex)


def spiral_forward(x, S, E: Nudft):
    return np.stack([E.forward(S[c] * x) for c in range(S.shape[0])])


def spiral_adjoint(y, S, E: Nudft):
    return np.sum(np.stack([np.conj(S[c]) * E.adjoint(y[c]) for c in range(S.shape[0])]), axis=0)


def spiral_normal(x, S, E: Nudft, lam: float = 0.0):
    return spiral_adjoint(spiral_forward(x, S, E), S, E) + lam * x


def spiral_matrix(S: np.ndarray, traj: np.ndarray) -> np.ndarray:
    """Explicit spiral encoding matrix for tiny images (rows (c, m), cols y*n+x)."""
    nc, n, _ = S.shape
    t = np.asarray(traj, dtype=np.float64)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ph = np.outer(t[:, 0], xx.reshape(-1)) + np.outer(t[:, 1], yy.reshape(-1))
    E = np.exp(-2j * np.pi * ph / n) / n
    return np.concatenate([E * S[c].reshape(-1)[None, :] for c in range(nc)], axis=0)


class ToeplitzNormal:
    """``A^H A`` of the exact-NUDFT spiral encoding applied through its
    point-spread function (for full-size images, where the NUDFT itself costs
    minutes per application).

    ``(E^H E z)[r] = sum_r' h(r - r') z[r']`` with
    ``h(d) = (1/n^2) sum_m exp(+2 pi i k_m . d / n)`` (the entries of
    ``E^H E`` written out, as in ``pico.dense_normal``); the lags span
    ``[-(n-1), n-1]^2``, so the sum is a linear convolution that a circular
    one on the ``2n x 2n`` grid reproduces exactly (convolution theorem, FFT
    pair of NumPy).  ``apply`` adds the coil sensitivities and ``lam``.
    """

    def __init__(self, S: np.ndarray, traj: np.ndarray):
        self.S = np.asarray(S, dtype=np.complex128)
        n = self.S.shape[1]
        self.n = n
        k = np.asarray(traj, dtype=np.float64)
        d = np.arange(-(n - 1), n, dtype=np.float64)
        ex = np.exp(2j * np.pi * np.outer(k[:, 0], d) / n)        # [M][dx]
        ey = np.exp(2j * np.pi * np.outer(k[:, 1], d) / n)        # [M][dy]
        h = (ey.T @ ex) / n ** 2                                   # h[dy + n-1, dx + n-1]
        L = 2 * n
        C = np.zeros((L, L), dtype=np.complex128)
        C[np.ix_(np.arange(-(n - 1), n) % L, np.arange(-(n - 1), n) % L)] = h
        self.T = np.fft.fft2(C)

    def apply(self, x: np.ndarray, lam: float = 0.0) -> np.ndarray:
        n, L = self.n, 2 * self.n
        out = lam * np.asarray(x, dtype=np.complex128)
        for c in range(self.S.shape[0]):
            z = np.zeros((L, L), dtype=np.complex128)
            z[:n, :n] = self.S[c] * x
            w = np.fft.ifft2(self.T * np.fft.fft2(z))[:n, :n]
            out = out + np.conj(self.S[c]) * w
        return out


class Operator:
    """Whitened encoding operator of one acquisition (Cartesian or spiral)."""

    def __init__(self, smaps, noise_cov=None, mask=None, traj=None):
        self.S = whiten(smaps, noise_cov)
        self.nc, self.ny, self.nx = self.S.shape
        self.mask = None if mask is None else np.asarray(mask)
        self.traj = None if traj is None else np.asarray(traj)
        self.E = Nudft(self.traj, self.ny) if self.traj is not None else None

    @property
    def kind(self):
        return "spiral" if self.E is not None else "cartesian"

    def forward(self, x):
        return spiral_forward(x, self.S, self.E) if self.E is not None else cart_forward(x, self.S, self.mask)

    def adjoint(self, y):
        return spiral_adjoint(y, self.S, self.E) if self.E is not None else cart_adjoint(y, self.S, self.mask)

    def normal(self, x, lam=0.0):
        return self.adjoint(self.forward(x)) + lam * x

    def matrix(self):
        if self.E is not None:
            return spiral_matrix(self.S, self.traj)
        return cart_matrix(self.S, self.mask)

    def kspace_shape(self):
        if self.E is not None:
            return (self.nc, self.traj.shape[0])
        return (self.nc, self.ny, self.nx)

    def kspace_index(self):
        """Flat element index of every k-space sample used by PMR noise draws.

        Cartesian: ``(c * ny + ky) * nx + kx`` over the full grid (unsampled
        positions are masked out after drawing); spiral: ``c * M + m``.
        """
        return np.arange(int(np.prod(self.kspace_shape())), dtype=np.int64).reshape(self.kspace_shape())
