"""pico_cg_batch_static: the solve that allocates no device memory.

Callers that cannot call cudaMalloc (code running inside a host application
that owns every device allocation through its own pool) use this entry point.
It must agree with the FP64 oracle's CG element by element on two calls in a
row (the second call reuses the static scratch that the first call left
behind).  Collected last so that a failure here does not hide the others.
"""
import ctypes

import numpy as np
import pytest

import synth
from oracle import ops as O
from oracle import solvers as OS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_09590_gb300 as pico  # noqa: E402
from paper_2605_09590_gb300 import build as pico_build  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    pico_build.build()
    L = pico.load_library()
    fn = L.pico_cg_batch_static
    vp = ctypes.c_void_p
    fn.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, vp, vp,
                   ctypes.c_int32, ctypes.c_int32, ctypes.c_double, vp]
    fn.restype = ctypes.c_int32
    L.pico_static_last_error.restype = ctypes.c_char_p
    L.pico_cg_batch_static_capacity.restype = ctypes.c_size_t
    return L


def _rhs(nb, ny, nx, seed):
    g = np.random.default_rng(seed)
    return torch.from_numpy((g.standard_normal((nb, ny, nx)) + 1j * g.standard_normal((nb, ny, nx)))
                            .astype(np.complex64)).cuda()


@pytest.mark.parametrize("ny,nx,nc,lam,check", [(320, 320, 15, 0.0, (0, 7)), (96, 72, 6, 0.05, tuple(range(8)))])
def test_static_solve_matches_the_oracle_twice(lib, ny, nx, nc, lam, check):
    """Two calls in a row (the second reuses the scratch the first left
    behind); the solutions of the systems in `check` are compared element by
    element with the FP64 oracle's CG (same 30 iterations from x0 = 0):
    |x - x_oracle| <= 1e-4 max|x_oracle| per image (FP32 arithmetic against
    FP64 over 30 iterations; the context-based solve meets the same bound)."""
    S = synth.coil_maps(ny, nx, nc, 3)                # white noise: whitened maps are the maps
    mask = synth.mask_pe(ny, 2, 24 if ny >= 96 else 4)
    oop = O.Operator(S, None, mask=mask)
    S_dev = torch.from_numpy(S).cuda()
    m_dev = torch.from_numpy(mask).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((1, 2)):
        rhs = _rhs(8, ny, nx, seed)
        got = torch.empty_like(rhs)
        st = lib.pico_cg_batch_static(S_dev.data_ptr(), m_dev.data_ptr(), ny, nx, nc, lam, rhs.data_ptr(),
                                      got.data_ptr(), 8, 30, 0.0, stream)
        assert st == pico.PICO_OK, lib.pico_static_last_error()
        torch.cuda.synchronize()
        got_h, rhs_h = got.cpu().numpy(), rhs.cpu().numpy()
        for b in check:
            want, _, _ = OS.cg(lambda z: oop.normal(z, lam), rhs_h[b].astype(np.complex128), 30, 0.0)
            err = np.abs(got_h[b] - want).max() / np.abs(want).max()
            assert err < 1e-4, (call, b, err)


def test_static_solve_rejects_requests_above_capacity(lib):
    ny = nx = 320
    S_dev = torch.zeros((2, ny, nx), dtype=torch.complex64, device="cuda")
    m_dev = torch.ones(ny, dtype=torch.uint8, device="cuda")
    nb = 64                                               # 64 x 3 x 819,200 B > 64 MiB
    rhs = torch.zeros((nb, ny, nx), dtype=torch.complex64, device="cuda")
    x = torch.empty_like(rhs)
    st = lib.pico_cg_batch_static(S_dev.data_ptr(), m_dev.data_ptr(), ny, nx, 2, 0.0, rhs.data_ptr(),
                                  x.data_ptr(), nb, 10, 0.0, torch.cuda.current_stream().cuda_stream)
    assert st == pico.PICO_E_INVALID
    assert b"static array holds" in lib.pico_static_last_error()
    assert lib.pico_cg_batch_static_capacity() == 64 << 20
