"""Forward / adjoint encoding operators (pico_forward, pico_adjoint) against the oracle."""
import numpy as np
import pytest

import synth
from oracle import ops as O

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


def rnd(shape, seed):
    g = np.random.default_rng(seed)
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)).astype(np.complex64)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("ny,nx", [(64, 64), (96, 80), (320, 320)])
def test_cartesian_forward_adjoint(ny, nx):
    nc = 5
    S = synth.coil_maps(ny, nx, nc, 1)
    cov = synth.noise_cov(nc, 1)
    mask = synth.mask_pe(ny, 2, 8)
    op = pico.Operator(S, mask=mask, noise_cov=cov, power_iters=0, max_batch=2)
    oop = O.Operator(S, cov, mask=mask)
    x = rnd((3, ny, nx), 2)
    y = op.forward(dev(x)).cpu().numpy()
    for b in range(3):
        assert rel(y[b], oop.forward(x[b].astype(np.complex128))) < 2e-6
    k = rnd((3, nc, ny, nx), 3) * O.mask2d(mask, nx)[None, None]
    xa = op.adjoint(dev(k)).cpu().numpy()
    for b in range(3):
        assert rel(xa[b], oop.adjoint(k[b].astype(np.complex128))) < 2e-6


def test_spiral_forward_adjoint_against_exact_nudft():
    n, nc = 64, 4
    S = synth.coil_maps(n, n, nc, 2)
    traj = synth.spiral_traj(n, 16, 512, 2)
    op = pico.Operator(S, traj=traj, power_iters=0, max_batch=2)
    oop = O.Operator(S, None, traj=traj)
    x = rnd((3, n, n), 4)
    y = op.forward(dev(x)).cpu().numpy()
    for b in range(3):
        assert rel(y[b], oop.forward(x[b].astype(np.complex128))) < 1e-4   # Kaiser-Bessel W=6, os=2
    k = rnd((3, nc, traj.shape[0]), 5)
    xa = op.adjoint(dev(k)).cpu().numpy()
    for b in range(3):
        assert rel(xa[b], oop.adjoint(k[b].astype(np.complex128))) < 1e-4
    # the gridding pair is an exact adjoint pair (same kernel both ways)
    lhs = np.vdot(y.astype(np.complex128), k.astype(np.complex128))
    rhs = np.vdot(x.astype(np.complex128), xa.astype(np.complex128))
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_cg_sense_reconstruction_full_sampling_recovers_image():
    n, nc = 64, 6
    S = synth.coil_maps(n, n, nc, 3)                  # sum |S|^2 = 1 => A^H A = I
    op = pico.Operator(S, mask=np.ones(n, dtype=np.uint8), power_iters=0)
    x = dev(rnd((2, n, n), 6))
    b = op.forward(x)
    xr = op.cg(op.adjoint(b), 10, 0.0)
    assert torch.allclose(xr, x, atol=1e-4, rtol=1e-4)
