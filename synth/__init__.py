"""Seeded synthetic inputs for the PICO noise-map workloads.

This module only *draws inputs*: coil sensitivities, coil-noise covariances,
Cartesian phase-encode masks and variable-density spiral trajectories.  It
contains none of the estimator's arithmetic (no Fourier transforms, no solves,
no probes), so both the CUDA path and the CPU oracle may consume its arrays.

The paper's datasets (Stanford knee, a spiral brain-phantom scan, fastMRI knee;
Sec. 3.1) are not available; these generators stand in for them with the
matrix sizes, coil counts and sampling patterns the paper describes
(320x320 with 15 coils, Sec. 3.1 "fastMRI knee"; spiral at R = 2, 3, 4,
Sec. 3.2.2).

Conventions shared by every consumer:

* images are row-major ``[ny][nx]`` complex64, voxel ``(y, x)`` with
  ``y, x`` counted from 0;
* Cartesian masks are indexed by the DFT frequency ``ky`` in natural
  (unshifted) order, ``ky = 0`` is DC;
* spiral trajectories are ``[nsamp][2]`` float32 ``(kx, ky)`` in cycles per
  field of view, so a Nyquist step is 1.0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "coil_maps",
    "noise_cov",
    "mask_pe",
    "spiral_traj",
    "poisson_disc_mask",
    "phantom",
    "Workload",
    "WORKLOADS",
]


def coil_maps(ny: int, nx: int, nc: int, seed: int, radius: float = 0.6,
              width: float = 0.35, normalize: bool = True) -> np.ndarray:
    """Smooth complex Gaussian-bump coil sensitivities, complex64 ``[nc][ny][nx]``.

    Coil ``c`` sits on a circle of ``radius`` field-of-view units around the
    image centre (angle ``2 pi c / nc`` plus a seeded jitter); its magnitude is
    a Gaussian of standard deviation ``width`` FOV and its phase is a seeded
    linear ramp ``alpha x + beta y + gamma``.  With ``normalize`` the maps are
    scaled voxelwise so that ``sum_c |S_c|^2 = 1``.
    """
    rng = np.random.default_rng(np.random.SeedSequence([0xC011, seed, ny, nx, nc]))
    yy = (np.arange(ny, dtype=np.float64) - ny / 2) / ny
    xx = (np.arange(nx, dtype=np.float64) - nx / 2) / nx
    Y, X = np.meshgrid(yy, xx, indexing="ij")
    maps = np.empty((nc, ny, nx), dtype=np.complex128)
    jitter = rng.uniform(-0.25, 0.25, size=nc) * (2 * math.pi / max(nc, 1))
    alpha = rng.uniform(-math.pi, math.pi, size=nc)
    beta = rng.uniform(-math.pi, math.pi, size=nc)
    gamma = rng.uniform(0.0, 2 * math.pi, size=nc)
    for c in range(nc):
        phi = 2 * math.pi * c / nc + jitter[c]
        cy, cx = radius * math.sin(phi), radius * math.cos(phi)
        mag = np.exp(-((Y - cy) ** 2 + (X - cx) ** 2) / (2 * width ** 2))
        maps[c] = mag * np.exp(1j * (alpha[c] * X * 2 * math.pi
                                     + beta[c] * Y * 2 * math.pi + gamma[c]))
    if normalize:
        maps /= np.sqrt(np.sum(np.abs(maps) ** 2, axis=0, keepdims=True))
    return maps.astype(np.complex64)


def noise_cov(nc: int, seed: int, rho: float = 0.1, min_eig: float = 0.2) -> np.ndarray:
    """Hermitian positive-definite coil-noise covariance, complex128 ``[nc][nc]``.

    ``Sigma_n = D^(1/2) C D^(1/2)`` with ``C = I + rho * H``, ``H`` Hermitian
    with zero diagonal and unit-modulus random-phase off-diagonal entries
    (redrawn until ``lambda_min(C) > min_eig``) and ``D`` diagonal, uniform in
    ``[0.8, 1.2]``.
    """
    rng = np.random.default_rng(np.random.SeedSequence([0x5161, seed, nc]))
    for _ in range(1000):
        ph = rng.uniform(0.0, 2 * math.pi, size=(nc, nc))
        H = np.triu(np.exp(1j * ph), 1)
        H = H + H.conj().T
        C = np.eye(nc) + rho * H
        if np.linalg.eigvalsh(C).min() > min_eig:
            break
    else:  # pragma: no cover - rho this small always succeeds
        raise RuntimeError("could not draw a well-conditioned coil covariance")
    d = np.sqrt(rng.uniform(0.8, 1.2, size=nc))
    return (d[:, None] * C * d[None, :]).astype(np.complex128)


def mask_pe(ny: int, R: int, acs: int = 0, offset: int = 0) -> np.ndarray:
    """Phase-encode sampling mask, uint8 ``[ny]`` in natural DFT order.

    Keeps ``ky = offset (mod R)`` plus ``acs`` fully sampled central lines
    ``ky in [-acs/2, acs/2)`` (taken modulo ``ny``).
    """
    m = np.zeros(ny, dtype=np.uint8)
    m[offset % R::R] = 1
    for k in range(-(acs // 2), acs - acs // 2):
        m[k % ny] = 1
    return m


def spiral_traj(n: int, n_interleaves: int = 16, nsamp: int = 4096, R: int = 1,
                kmax: float | None = None, density_power: float = 1.5) -> np.ndarray:
    """Variable-density spiral, float32 ``[n_kept * nsamp][2]`` in cycles/FOV.

    Interleaf ``l`` follows ``k(t) = kmax * t^p * exp(j (2 pi Nt t + 2 pi l / L))``
    for ``t`` in ``[0, 1]`` with ``p = density_power``; ``Nt`` (turns) is the
    smallest integer for which the spacing between neighbouring interleaves at
    the edge, ``p * kmax / (L * Nt)``, is at most one Nyquist step.
    Shot subsampling keeps the interleaves ``l = 0 (mod R)``.
    """
    if kmax is None:
        kmax = n / 2.0
    L = n_interleaves
    turns = math.ceil(density_power * kmax / L)
    t = np.arange(nsamp, dtype=np.float64) / (nsamp - 1)
    out = []
    for l in range(0, L, R):
        k = kmax * t ** density_power * np.exp(1j * (2 * math.pi * turns * t + 2 * math.pi * l / L))
        out.append(np.stack([k.real, k.imag], axis=1))
    traj = np.concatenate(out, axis=0)
    # keep the half-open box [-n/2, n/2): the point exactly at +n/2 is moved
    # to its periodic image.
    traj = np.where(traj >= n / 2, traj - n, traj)
    return traj.astype(np.float32)


@dataclass(frozen=True)
class Workload:
    """A named synthetic workload (sizes follow the paper's experiments)."""
    name: str
    kind: str            # "cartesian", "spiral" or "cs" (2-D Poisson-disc mask, L1-wavelet FISTA)
    ny: int
    nx: int
    nc: int
    R: int
    acs: int = 0
    noise_corr: bool = False
    probes: int = 32
    max_iter: int = 30
    lam: float = 0.0
    sigma: float = 1.0
    n_interleaves: int = 16
    nsamp: int = 4096
    reps: int = 0
    seed: int = 0
    extra: dict = field(default_factory=dict)

    def inputs(self, seed: int | None = None) -> dict:
        s = self.seed if seed is None else seed
        out = {"smaps": coil_maps(self.ny, self.nx, self.nc, s)}
        out["noise_cov"] = noise_cov(self.nc, s) if self.noise_corr else None
        if self.kind == "cartesian":
            out["mask"] = mask_pe(self.ny, self.R, self.acs)
        elif self.kind == "cs":
            out["mask"] = poisson_disc_mask(self.ny, self.nx, float(self.R), self.acs, s)
            out["phantom"] = phantom(self.ny, s)
        else:
            out["traj"] = spiral_traj(self.ny, self.n_interleaves, self.nsamp, self.R)
        return out


WORKLOADS = {
    # 64x64, 8 coils, uniform R=2 without calibration lines, K=32, 30 CG iterations.
    "sense64_r2": Workload("sense64_r2", "cartesian", 64, 64, 8, 2, acs=0,
                           probes=32, max_iter=30),
    # knee-shaped 320x320, 15 correlated coils, R=2 plus 24 central lines.
    "knee320_r2": Workload("knee320_r2", "cartesian", 320, 320, 15, 2, acs=24,
                           noise_corr=True, probes=256, max_iter=30),
    # 240x240 spiral, 20 coils, 16 interleaves x 4096 samples, Tikhonov 0.1.
    "spiral240_r2": Workload("spiral240_r2", "spiral", 240, 240, 20, 2, probes=256,
                             max_iter=30, lam=0.1, sigma=1e-2, reps=500),
    "spiral240_r3": Workload("spiral240_r3", "spiral", 240, 240, 20, 3, probes=256,
                             max_iter=30, lam=0.1, sigma=1e-2, reps=500),
    "spiral240_r4": Workload("spiral240_r4", "spiral", 240, 240, 20, 4, probes=256,
                             max_iter=30, lam=0.1, sigma=1e-2, reps=500),
    # 320x320, 15 correlated coils, variable-density Poisson-disc R=2 with a 24x24
    # calibration block; L1-wavelet (db4, 4 levels) FISTA, 100 iterations, weight
    # 1e-2 max|W A^H b|; K=64 Jacobian probes; PMR noise 45 dB below the data rms.
    "cs320_r2": Workload("cs320_r2", "cs", 320, 320, 15, 2, acs=24, noise_corr=True,
                         probes=64, max_iter=100,
                         extra={"levels": 4, "lam_l1_rel": 1e-2, "pmr_snr_db": 45.0}),
}


def poisson_disc_mask(ny: int, nx: int, R: float, calib: int = 24, seed: int = 0,
                      density_power: float = 1.0) -> np.ndarray:
    """Variable-density Poisson-disc sampling mask, uint8 ``[ny][nx]`` in natural DFT order.

    Dart throwing in the centred ``(ky, kx)`` plane: a candidate is accepted if no
    accepted point lies within ``r(k) = r0 (1 + density_power * |k| / k_max)``
    of it (Bridson-style rejection with a growing radius), the central
    ``calib x calib`` block is fully sampled, and ``r0`` is bisected until the
    acceleration ``ny nx / #samples`` is within 2 % of ``R``.
    """
    rng = np.random.default_rng(np.random.SeedSequence([0x9D15C, seed, ny, nx]))
    ky = np.arange(ny) - ny // 2
    kx = np.arange(nx) - nx // 2
    KY, KX = np.meshgrid(ky, kx, indexing="ij")
    kn = np.sqrt((KY / (ny / 2)) ** 2 + (KX / (nx / 2)) ** 2) / math.sqrt(2)
    order = rng.permutation(ny * nx)
    calib_blk = (KY >= -(calib // 2)) & (KY < calib - calib // 2) & (KX >= -(calib // 2)) & (KX < calib - calib // 2)

    def draw(r0):
        m = calib_blk.copy()
        cell = max(r0, 0.5)
        grid = {}
        for idx in order:
            y, x = divmod(int(idx), nx)
            if m[y, x]:
                continue
            r = r0 * (1.0 + density_power * kn[y, x])
            gy, gx = int(y // cell), int(x // cell)
            reach = int(math.ceil(r * (1.0 + density_power) / cell)) + 1
            ok = True
            for dy in range(-reach, reach + 1):
                for dx in range(-reach, reach + 1):
                    for (py, px) in grid.get((gy + dy, gx + dx), ()):
                        rr = r0 * (1.0 + density_power * 0.5 * (kn[y, x] + kn[py, px]))
                        if (py - y) ** 2 + (px - x) ** 2 < rr * rr:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                m[y, x] = True
                grid.setdefault((gy, gx), []).append((y, x))
        return m

    lo, hi = 0.5, 4.0
    best = None
    for _ in range(20):
        r0 = 0.5 * (lo + hi)
        m = draw(r0)
        acc = ny * nx / m.sum()
        best = m
        if abs(acc - R) / R < 0.02:
            break
        if acc < R:
            lo = r0
        else:
            hi = r0
    # centred -> natural DFT order
    return np.fft.ifftshift(best).astype(np.uint8)


def phantom(n: int, seed: int = 0, n_ellipses: int = 10) -> np.ndarray:
    """Seeded piecewise-constant ellipse phantom, complex64 ``[n][n]`` (smooth phase)."""
    rng = np.random.default_rng(np.random.SeedSequence([0xE111, seed, n]))
    yy = (np.arange(n) - n / 2) / (n / 2)
    Y, X = np.meshgrid(yy, yy, indexing="ij")
    img = np.zeros((n, n))
    img[(X / 0.75) ** 2 + (Y / 0.9) ** 2 <= 1] = 1.0
    for _ in range(n_ellipses - 1):
        cx, cy = rng.uniform(-0.5, 0.5, 2)
        ax, ay = rng.uniform(0.05, 0.3, 2)
        th = rng.uniform(0, math.pi)
        Xr = (X - cx) * math.cos(th) + (Y - cy) * math.sin(th)
        Yr = -(X - cx) * math.sin(th) + (Y - cy) * math.cos(th)
        img[(Xr / ax) ** 2 + (Yr / ay) ** 2 <= 1] += rng.uniform(-0.4, 0.4)
    phase = np.exp(1j * math.pi * 0.3 * (X + 0.5 * Y))
    return (img * phase).astype(np.complex64)
