"""Counter-based random draws for probes and PMR noise (oracle side).

The paper draws probe phases ``theta ~ U[0, 2 pi)`` (Sec. 2.2.4, Eq. 20;
Alg. 1) and PMR k-space noise ``n ~ CN(0, sigma^2 I)`` (Sec. 1, PMR) but fixes
no generator.  To compare runs with identical seeds, both the CUDA path and
this oracle implement the same counter-based generator from its published
definition: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) with the 64-bit output finaliser
``mix64``.  The two implementations are written separately.

Definition used by both sides
-----------------------------
``splitmix64(s, i)`` is output ``i`` (counting from 0) of SplitMix64 seeded
with state ``s``:  ``mix64(s + GAMMA * (i + 1))`` modulo ``2**64``.

* stream key of probe (or replica) ``p`` under ``seed``:
  ``key = splitmix64(seed, p)``
* word ``j`` of that stream: ``h_j = splitmix64(key, j)``
* uniform in [0, 1):  ``u(h) = (h >> 40) * 2**-24``  (24 bits, exact in float32)
* uniform in (0, 1]:  ``u1(h) = ((h >> 40) + 1) * 2**-24``

Element ``e`` (a voxel index ``y * nx + x``, or a k-space index) uses the
words ``h_{2e}`` and ``h_{2e+1}``:

* random phase (Eq. 20):        ``v = exp(2 pi i u(h_{2e}))``
* real Rademacher (Eq. 19):     ``v = +1`` if bit 63 of ``h_{2e}`` is 0 else ``-1``
* complex Gaussian (Eq. 18):    ``v = sqrt(-ln u1(h_{2e})) exp(2 pi i u(h_{2e+1}))``
  (Box-Muller in polar form; ``E|v|^2 = 1``)
* PMR noise:                    ``sigma`` times the complex Gaussian draw.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB

PROBE_PHASE = 0
PROBE_RADEMACHER = 1
PROBE_GAUSS = 2


def mix64(z):
    """SplitMix64 output finaliser on uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64(state, i):
    """Output ``i`` (0-based) of SplitMix64 seeded with ``state``."""
    state = np.asarray(state, dtype=np.uint64)
    i = np.asarray(i, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(state + np.uint64(GAMMA) * (i + np.uint64(1)))


def stream_key(seed: int, index: int) -> np.uint64:
    """Key of probe / replica ``index`` under ``seed``."""
    return splitmix64(np.uint64(seed & MASK64), np.uint64(index))


def words(key, j):
    return splitmix64(key, j)


def unif(h):
    """Uniform in [0, 1) from the top 24 bits (float64, exact)."""
    return (np.asarray(h, dtype=np.uint64) >> np.uint64(40)).astype(np.float64) * 2.0 ** -24


def unif_open0(h):
    """Uniform in (0, 1] from the top 24 bits (float64, exact)."""
    return ((np.asarray(h, dtype=np.uint64) >> np.uint64(40)).astype(np.float64) + 1.0) * 2.0 ** -24


def probe(seed: int, index: int, n: int, kind: int = PROBE_PHASE) -> np.ndarray:
    """Probe image ``v`` of ``n`` voxels (complex128), Sec. 2.2.4 / Alg. 1 step (1)."""
    key = stream_key(seed, index)
    e = np.arange(n, dtype=np.uint64)
    h0 = words(key, np.uint64(2) * e)
    if kind == PROBE_PHASE:
        th = 2.0 * np.pi * unif(h0)
        return np.cos(th) + 1j * np.sin(th)
    if kind == PROBE_RADEMACHER:
        sgn = (h0 >> np.uint64(63)).astype(np.float64)
        return (1.0 - 2.0 * sgn).astype(np.complex128)
    if kind == PROBE_GAUSS:
        h1 = words(key, np.uint64(2) * e + np.uint64(1))
        r = np.sqrt(-np.log(unif_open0(h0)))
        th = 2.0 * np.pi * unif(h1)
        return r * (np.cos(th) + 1j * np.sin(th))
    raise ValueError(f"unknown probe kind {kind}")


def cnoise(seed: int, index: int, elems: np.ndarray, sigma: float) -> np.ndarray:
    """``CN(0, sigma^2)`` draws at element indices ``elems`` of replica ``index``."""
    key = stream_key(seed, index)
    e = np.asarray(elems, dtype=np.uint64)
    h0 = words(key, np.uint64(2) * e)
    h1 = words(key, np.uint64(2) * e + np.uint64(1))
    r = np.sqrt(-np.log(unif_open0(h0)))
    th = 2.0 * np.pi * unif(h1)
    return sigma * r * (np.cos(th) + 1j * np.sin(th))
