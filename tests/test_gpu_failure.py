"""Failure statuses of the C ABI, produced on the host (no kernel is made to fail).

* A right-hand side holding a NaN makes its CG system break down: the solve
  reports PICO_E_BREAKDOWN at pico_sync, that system keeps x = 0, every other
  system of the batch is solved as if it were alone, and the context stays
  usable (the next clean batch reports PICO_OK and gives the same solutions).
  Checked on the column-FFT, tensor-core Gram and Toeplitz (spiral) operators;
  under per-column CG only the column holding the NaN breaks down.
* pico_inject_error sets a device status word from the host exactly as a
  kernel would; pico_sync reports the class (a timeout before a breakdown,
  both named in the message) and clears the words.
* The autograd Function of the CS reconstruction refuses a backward after a
  second reconstruction replaced the stored linearisation point.
"""
import numpy as np
import pytest

import synth

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


def _rhs(nb, ny, nx, seed):
    g = np.random.default_rng(seed)
    return torch.from_numpy((g.standard_normal((nb, ny, nx)) + 1j * g.standard_normal((nb, ny, nx)))
                            .astype(np.complex64)).cuda()


def _operator(kind):
    if kind == "spiral":
        S = synth.coil_maps(64, 64, 4, 2)
        return pico.Operator(S, traj=synth.spiral_traj(64, 8, 512, 2), lam=0.1, power_iters=15, max_batch=8)
    if kind == "gram":
        S = synth.coil_maps(128, 32, 4, 1)
        op = pico.Operator(S, mask=synth.mask_pe(128, 2, 8), power_iters=0, max_batch=8)
        op.set_tuning(gram_min_batch=1)
        assert op.info["normal_op"] == 1
        return op
    S = synth.coil_maps(64, 48, 4, 3)
    return pico.Operator(S, mask=synth.mask_pe(64, 2, 4), power_iters=0, max_batch=8)


@pytest.mark.parametrize("kind", ["fft", "gram", "spiral"])
def test_nan_rhs_is_a_breakdown_and_the_context_stays_usable(kind):
    op = _operator(kind)
    nb = 6
    rhs = _rhs(nb, op.ny, op.nx, 11)
    clean = op.cg(rhs, 20, 0.0)
    op.sync()
    bad = rhs.clone()
    bad[2, 3, 5] = float("nan")
    x, iters, relres = op.cg(bad, 20, 0.0, stats=True)
    with pytest.raises(pico.PicoError) as ei:
        op.sync()
    assert ei.value.status == pico.PICO_E_BREAKDOWN
    assert "breakdown" in str(ei.value)
    assert torch.all(x[2] == 0)
    assert np.isnan(relres[2])
    keep = [0, 1, 3, 4, 5]
    # the other systems are solved exactly as in the clean batch
    assert torch.equal(x[keep], clean[keep])
    again = op.cg(rhs, 20, 0.0)
    op.sync()                                   # cleared: no error is reported twice
    assert torch.equal(again, clean)
    op.close()


@pytest.mark.parametrize("ny,nx", [(128, 32), (64, 48)])
def test_nan_rhs_breaks_down_only_its_column_under_per_column_cg(ny, nx):
    """Per-column CG (ny = 128: the whole solve in one cluster launch; ny = 64:
    on chip): a NaN in column 5 of image 2 breaks down that column's system
    only -- PICO_E_BREAKDOWN at pico_sync, x = 0 in that column, every other
    column and image as in the clean batch, and the context stays usable."""
    S = synth.coil_maps(ny, nx, 4, 1)
    op = pico.Operator(S, mask=synth.mask_pe(ny, 2, 8), power_iters=0, max_batch=8)
    if ny == 128:
        op.set_tuning(gram_min_batch=1)
    op.set_solver("columns")
    nb = 6
    rhs = _rhs(nb, ny, nx, 12)
    clean = op.cg(rhs, 20, 0.0)
    op.sync()
    bad = rhs.clone()
    bad[2, 3, 5] = float("nan")
    x, iters, relres = op.cg(bad, 20, 0.0, stats=True)
    with pytest.raises(pico.PicoError) as ei:
        op.sync()
    assert ei.value.status == pico.PICO_E_BREAKDOWN
    assert torch.all(x[2][:, 5] == 0)
    assert np.isnan(relres[2])
    others = [j for j in range(nx) if j != 5]
    assert torch.equal(x[2][:, others], clean[2][:, others])
    keep = [0, 1, 3, 4, 5]
    assert torch.equal(x[keep], clean[keep])
    again = op.cg(rhs, 20, 0.0)
    op.sync()
    assert torch.equal(again, clean)
    op.close()


def test_injected_status_words_are_reported_and_cleared():
    op = _operator("fft")
    pico.pico_inject_error(op.ctx, pico.PICO_E_TIMEOUT, 7)
    with pytest.raises(pico.PicoError) as ei:
        op.sync()
    assert ei.value.status == pico.PICO_E_TIMEOUT and "code 7" in str(ei.value)
    op.sync()
    pico.pico_inject_error(op.ctx, pico.PICO_E_BREAKDOWN, 5)
    with pytest.raises(pico.PicoError) as ei:
        op.sync()
    assert ei.value.status == pico.PICO_E_BREAKDOWN
    op.sync()
    # both pending: the timeout is returned, the message names both classes
    pico.pico_inject_error(op.ctx, pico.PICO_E_TIMEOUT, 3)
    pico.pico_inject_error(op.ctx, pico.PICO_E_BREAKDOWN, 5)
    with pytest.raises(pico.PicoError) as ei:
        op.sync()
    assert ei.value.status == pico.PICO_E_TIMEOUT
    assert "timed out" in str(ei.value) and "breakdown" in str(ei.value)
    op.sync()
    with pytest.raises(pico.PicoError) as ei:
        pico.pico_inject_error(op.ctx, pico.PICO_E_OOM, 1)
    assert ei.value.status == pico.PICO_E_INVALID
    # a solve after the injected errors is unaffected
    rhs = _rhs(2, op.ny, op.nx, 4)
    op.cg(rhs, 10, 0.0)
    op.sync()
    op.close()


def test_cs_backward_after_a_second_reconstruction_raises():
    n, nc = 64, 4
    S = synth.coil_maps(n, n, nc, 5)
    mask = synth.poisson_disc_mask(n, n, 2.0, 8, 0)
    op = pico.Operator(S, mask=mask, power_iters=15, max_batch=2)
    x0 = torch.from_numpy(synth.phantom(n, 5).astype(np.complex64)).cuda().reshape(1, n, n)
    b = op.forward(x0)[0].contiguous()
    f = pico.cs_function()
    b1 = b.clone().requires_grad_(True)
    y1 = f.apply(op, b1, 1e-3, 20, 2)
    y1.abs().pow(2).sum().backward()            # one forward, its backward: fine
    assert b1.grad is not None
    b2 = b.clone().requires_grad_(True)
    b3 = (1.5 * b).clone().requires_grad_(True)
    y2 = f.apply(op, b2, 1e-3, 20, 2)
    f.apply(op, b3, 1e-3, 20, 2)                # replaces the stored iterates
    with pytest.raises(pico.PicoError):
        y2.abs().pow(2).sum().backward()
    op.close()
