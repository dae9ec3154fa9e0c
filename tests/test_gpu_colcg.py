"""GPU parity of CG run per readout column (pico_set_solver(PICO_SOLVER_COLUMNS)).

With a phase-encode mask A^H A is block diagonal over the readout columns, so
the normal equations split into nx independent ny x ny systems; the context
then runs CG on every column with its own step lengths and stopping test:
for ny >= 128 the whole solve in one launch (a thread-block cluster owns a
column and 128 images; x, r, p on chip for every update), or one fused
tensor-core launch per update (PICO_COLCG_PERSIST=0: x and r updated in the
operator's epilogue, the column's sums added across the row tiles of a
cluster); for ny = 32, 64, 96 the whole solve on chip in shared memory.  The oracle is ``oracle.solvers.cg_columns`` (the same CG on every
column's dense block, FP64), pinned in tests/test_oracle_pins.py.

Tolerances: the solutions after 30 updates agree per element to
1e-4 max|x| (FP32 against FP64, the same bound as the whole-image CG); PICO
maps per voxel to 1e-4 of the exact diagonal Sigma_kk (the parity bar for
identical probe seeds).  Cases cover clusters of 2, 4 and 6 CTAs (ny = 128,
320, 384; 256 in the comparison with the per-update kernel), ragged image
tiles (batches that are not multiples of 128, warps with finished and
unused lanes) and the bench's full launch shape (320 x 320, 15 coils, 256
probes).
"""
import numpy as np
import pytest

import synth
from oracle import ops as O
from oracle import pico as OP
from oracle import rng as ORNG
from oracle import solvers as OS

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


def rand_imgs(nb, ny, nx, seed):
    g = np.random.default_rng(seed)
    return (g.standard_normal((nb, ny, nx)) + 1j * g.standard_normal((nb, ny, nx))).astype(np.complex64)


def column_operator(ny, nx, nc, R=2, acs=8, corr=True, seed=0, lam=0.0, max_batch=64):
    S = synth.coil_maps(ny, nx, nc, seed)
    cov = synth.noise_cov(nc, seed) if corr else None
    mask = synth.mask_pe(ny, R, acs)
    op = pico.Operator(S, mask=mask, noise_cov=cov, lam=lam, power_iters=0, max_batch=max_batch)
    op.set_solver("columns")
    return op, O.Operator(S, cov, mask=mask)


@pytest.mark.parametrize("ny,nx,nc,nb,lam", [(128, 24, 4, 5, 0.0), (320, 16, 6, 7, 0.0), (320, 12, 4, 130, 0.02),
                                             (384, 8, 4, 3, 0.0)])
def test_column_cg_solutions_match_the_oracle(ny, nx, nc, nb, lam):
    op, oop = column_operator(ny, nx, nc, lam=lam, max_batch=max(nb, 8))
    rhs = rand_imgs(nb, ny, nx, 3)
    x = op.cg(torch.from_numpy(rhs).cuda(), 30, 0.0).cpu().numpy()
    op.sync()
    check = sorted({0, nb // 2, nb - 1})
    xo, _, _ = OS.cg_columns(oop, rhs[check].astype(np.complex128), lam, 30)
    for i, b in enumerate(check):
        err = np.abs(x[b] - xo[i]).max() / np.abs(xo[i]).max()
        assert err < 1e-4, (b, err)
    op.close()


@pytest.mark.parametrize("ny,nx,nc,nb,lam", [(320, 12, 6, 130, 0.01), (256, 10, 4, 5, 0.0), (128, 16, 4, 9, 0.0)])
def test_whole_solve_launch_matches_per_update_launches(ny, nx, nc, nb, lam, monkeypatch):
    """ny = 320, 256, 128 (clusters of 4, 4 and 2 CTAs): the per-column solve
    runs as one launch per batch with x, r and p on chip for every iteration;
    PICO_COLCG_PERSIST=0 selects one fused launch per update instead.  The same
    CG on the same FP16 operands, summed in other orders (the one-launch
    kernel takes each CTA's own rows of the contraction first): after 30
    updates the two agree to 1e-4 of max|x|, the bar both meet against the
    oracle, which the one-launch solve is checked against per element."""
    S = synth.coil_maps(ny, nx, nc, 11)
    cov = synth.noise_cov(nc, 11)
    mask = synth.mask_pe(ny, 2, 8)
    rhs = rand_imgs(nb, ny, nx, 12)
    xs, counts = [], []
    for v in ("1", "0"):
        monkeypatch.setenv("PICO_COLCG_PERSIST", v)
        op = pico.Operator(S, mask=mask, noise_cov=cov, lam=lam, power_iters=0, max_batch=nb)
        op.set_solver("columns")
        d = torch.from_numpy(rhs).cuda()
        op.cg(d, 30, 0.0)
        op.sync()
        pico.pico_launch_count(op.ctx, reset=True)
        x = op.cg(d, 30, 0.0)
        op.sync()
        counts.append(pico.pico_launch_count(op.ctx))
        xs.append(x.cpu().numpy())
        op.close()
    assert np.abs(xs[0] - xs[1]).max() / np.abs(xs[1]).max() < 1e-4
    assert counts[0] + 25 <= counts[1]              # one launch per solve instead of one per update
    oop = O.Operator(S, cov, mask=mask)
    check = sorted({0, nb - 1})
    xo, _, _ = OS.cg_columns(oop, rhs[check].astype(np.complex128), lam, 30)
    for i, b in enumerate(check):
        assert np.abs(xs[0][b] - xo[i]).max() / np.abs(xo[i]).max() < 1e-4, b


@pytest.mark.parametrize("ny,solver", [(64, "global"), (64, "columns"), (320, "columns")])
def test_solves_are_bitwise_repeatable(ny, solver):
    """The one-launch solves (on-chip small images, the whole-image exchange
    between blocks, the cluster kernel of larger images) repeated 10 times on
    the same right-hand sides: identical bits and no breakdown every time, also
    far below float precision (40 updates on an exactly solvable R = 2
    operator drive the residual to 1e-20), where a race between a block's
    threads had made solves break down or skip."""
    nx = 64 if ny == 64 else 24
    S = synth.coil_maps(ny, nx, 8, 3)
    op = pico.Operator(S, mask=synth.mask_pe(ny, 2, 0), power_iters=0, max_batch=256)
    if solver == "columns":
        op.set_solver("columns")
    rhs = torch.from_numpy(rand_imgs(256, ny, nx, 21)).cuda()
    first = None
    for _ in range(10):
        x = op.cg(rhs, 40, 0.0)
        op.sync()                                   # raises on any breakdown or timeout
        if first is None:
            first = x.clone()
        assert torch.equal(x, first)
    op.close()


def test_column_cg_stopping_rule_and_report():
    op, oop = column_operator(320, 16, 6)
    rhs = rand_imgs(4, 320, 16, 5)
    x, iters, relres = op.cg(torch.from_numpy(rhs).cuda(), 60, 1e-3, stats=True)
    op.sync()
    x = x.cpu().numpy()
    xo, ito, relo = OS.cg_columns(oop, rhs.astype(np.complex128), 0.0, 60, 1e-3)
    for b in range(4):
        assert relres[b] <= 1e-3 * (1 + 1e-3)
        assert abs(int(iters[b]) - int(ito[b])) <= 1      # FP32 vs FP64 residual at the threshold
        r = rhs[b].astype(np.complex128) - np.stack(
            [O.cart_column_normal(oop.S, oop.mask, j) @ x[b][:, j] for j in range(16)], axis=1)
        assert np.linalg.norm(r) / np.linalg.norm(rhs[b]) < 2e-3
        assert np.abs(x[b] - xo[b]).max() / np.abs(xo[b]).max() < 2e-3
    op.close()


def test_column_cg_is_deterministic_across_batches():
    op, _ = column_operator(320, 16, 6, max_batch=160)
    rhs = torch.from_numpy(rand_imgs(150, 320, 16, 8)).cuda()
    whole = op.cg(rhs, 20, 0.0)
    part = torch.cat([op.cg(rhs[:70].contiguous(), 20, 0.0), op.cg(rhs[70:].contiguous(), 20, 0.0)])
    op.sync()
    assert torch.equal(whole, part)                  # every (image, column) is solved on its own
    op.close()


def test_global_solver_is_restored():
    op, oop = column_operator(128, 16, 4)
    assert op.solver == pico.PICO_SOLVER_COLUMNS
    op.set_solver("global")
    assert op.solver == pico.PICO_SOLVER_GLOBAL
    rhs = rand_imgs(2, 128, 16, 9)
    x = op.cg(torch.from_numpy(rhs).cuda(), 30, 0.0).cpu().numpy()
    xo, _, _ = OS.cg(lambda z: oop.normal(z), rhs[1].astype(np.complex128), 30)
    assert np.abs(x[1] - xo).max() / np.abs(xo).max() < 1e-4
    op.close()


def test_column_solver_is_refused_where_unsupported():
    S = synth.coil_maps(48, 40, 4, 0)
    # ny = 48: neither a tensor-core context (ny < 128) nor an on-chip size (32, 64, 96)
    op = pico.Operator(S, mask=synth.mask_pe(48, 2, 4), power_iters=0, max_batch=8)
    with pytest.raises(pico.PicoError) as ei:
        op.set_solver("columns")
    assert ei.value.status == pico.PICO_E_UNSUPPORTED
    assert op.solver == pico.PICO_SOLVER_GLOBAL
    op.close()


def _dense_columns(oop):
    P = O.pe_projector(oop.mask)
    return np.stack([O.cart_column_normal(oop.S, oop.mask, j, P) for j in range(oop.nx)])   # [nx][ny][ny]


def _oracle_map(oop, seed, K, iters, solver):
    """Same-seed PICO sums over probes 0..K-1 (lam = 0): probes from the oracle's
    generator, K solves as one batch (each system follows its own CG steps)."""
    ny, nx = oop.ny, oop.nx
    V = np.stack([ORNG.probe(seed, i, ny * nx) for i in range(K)]).reshape(K, ny, nx)
    if solver == "columns":
        X, _, _ = OS.cg_columns(oop, V, 0.0, iters)
    else:
        G = _dense_columns(oop)

        def apply(P):            # [ny*nx][K] -> the dense per-column normal operator on every image
            Z = P.reshape(ny, nx, K).transpose(1, 0, 2)          # [nx][ny][K]
            return np.matmul(G, Z).transpose(1, 0, 2).reshape(ny * nx, K)

        Xf, _, _ = OS.cg_batched(apply, V.reshape(K, ny * nx).T, iters)
        X = Xf.T.reshape(K, ny, nx)
    d = np.real(np.conj(V) * X)
    return d.sum(axis=0)


@pytest.mark.parametrize("solver", ["global", "columns"])
def test_full_size_pico_map_per_voxel_same_seed(solver):
    """The bench's launch shape: 320 x 320, 15 correlated coils, R = 2 + 24
    lines, one batch of 256 probes, 30 updates; every voxel of the GPU map
    within 1e-4 Sigma_kk of the oracle's same-seed map."""
    w = synth.WORKLOADS["knee320_r2"]
    inp = w.inputs()
    K, seed = 256, 4242
    op = pico.Operator(inp["smaps"], mask=inp["mask"], noise_cov=inp["noise_cov"], power_iters=0, max_batch=K)
    assert op.info["normal_op"] == 1
    if solver == "columns":
        op.set_solver("columns")
    s, _ = op.variance_sums(seed, K, w.max_iter, 0.0)
    op.sync()
    s = s.cpu().numpy()
    op.close()
    oop = O.Operator(inp["smaps"], inp["noise_cov"], mask=inp["mask"])
    so = _oracle_map(oop, seed, K, w.max_iter, solver)
    d, _, _ = OP.column_exact(oop)
    err = np.abs(s - so) / K / d
    assert err.max() < 1e-4, (solver, err.max())


@pytest.mark.parametrize("ny,nx,nc,nb,lam", [(64, 64, 8, 32, 0.0), (32, 20, 4, 40, 0.05), (96, 16, 6, 17, 0.0)])
def test_small_images_whole_solve_on_chip_matches_the_oracle(ny, nx, nc, nb, lam):
    """ny = 32, 64, 96 (no tensor-core operator): the whole per-column solve in one launch."""
    S = synth.coil_maps(ny, nx, nc, 2)
    mask = synth.mask_pe(ny, 2, 0 if ny == 64 else 4)
    op = pico.Operator(S, mask=mask, lam=lam, power_iters=0, max_batch=nb)
    assert op.info["normal_op"] == 3
    op.set_solver("columns")
    rhs = rand_imgs(nb, ny, nx, 6)
    x, iters, relres = op.cg(torch.from_numpy(rhs).cuda(), 30, 0.0, stats=True)
    op.sync()
    x = x.cpu().numpy()
    oop = O.Operator(S, None, mask=mask)
    check = sorted({0, nb // 2, nb - 1})
    xo, ito, relo = OS.cg_columns(oop, rhs[check].astype(np.complex128), lam, 30)
    for i, b in enumerate(check):
        assert np.abs(x[b] - xo[i]).max() / np.abs(xo[i]).max() < 1e-4, b
        assert iters[b] == ito[i]
    op.close()


def test_small_images_pico_and_pmr_maps_same_seed():
    """sense64_r2 shape (64 x 64, 8 coils, R = 2, 32 probes): PICO and PMR maps
    per voxel within 1e-4 Sigma_kk of the oracle with per-column CG."""
    w = synth.WORKLOADS["sense64_r2"]
    inp = w.inputs()
    K = w.probes
    op = pico.Operator(inp["smaps"], mask=inp["mask"], noise_cov=inp["noise_cov"], power_iters=15, max_batch=K)
    op.set_solver("columns")
    s, _ = op.variance_sums(77, K, w.max_iter, 0.0)
    pm, _ = op.pmr_sums(78, K, 1.0, w.max_iter, 0.0)
    op.sync()
    oop = O.Operator(inp["smaps"], inp["noise_cov"], mask=inp["mask"])
    so, _ = OP.pico(oop, 77, 0, K, 0.0, w.max_iter, 0.0, solver="columns")
    po, _ = OP.pmr(oop, 78, 0, K, 1.0, 0.0, w.max_iter, 0.0, solver="columns")
    d, _, _ = OP.column_exact(oop)
    assert (np.abs(s.cpu().numpy() - so) / K / d).max() < 1e-4
    assert (np.abs(pm.cpu().numpy() - po) / K / d).max() < 1e-4
    op.close()


@pytest.mark.parametrize("ny,nx,nc,nb,lam", [(64, 64, 8, 32, 0.0), (32, 24, 4, 70, 0.05), (96, 20, 6, 9, 0.0)])
def test_small_images_whole_image_cg_on_chip_matches_the_oracle(ny, nx, nc, nb, lam):
    """The default (whole-image) CG of small phase-encode images on chip: one
    cooperative launch per solve, per-column partial sums exchanged between
    the blocks of an image group (release / acquire flags); the same CG as the
    oracle's solvers.cg."""
    S = synth.coil_maps(ny, nx, nc, 5)
    mask = synth.mask_pe(ny, 2, 4)
    op = pico.Operator(S, mask=mask, lam=lam, power_iters=0, max_batch=nb)
    assert op.info["normal_op"] == 3 and op.solver == pico.PICO_SOLVER_GLOBAL
    oop = O.Operator(S, None, mask=mask)
    rhs = rand_imgs(nb, ny, nx, 8)
    x, iters, relres = op.cg(torch.from_numpy(rhs).cuda(), 30, 0.0, stats=True)
    op.sync()
    x = x.cpu().numpy()
    for b in sorted({0, nb // 2, nb - 1}):
        xo, ito, relo = OS.cg(lambda z: oop.normal(z, lam), rhs[b].astype(np.complex128), 30, 0.0)
        assert np.abs(x[b] - xo).max() / np.abs(xo).max() < 1e-4, b
        assert iters[b] == ito and abs(relres[b] - relo) <= 1e-3 * relo + 1e-6
    # stopping rule: every image of the batch on its own
    x2, it2, rel2 = op.cg(torch.from_numpy(rhs).cuda(), 100, 1e-3, stats=True)
    op.sync()
    for b in (0, nb - 1):
        _, ito, _ = OS.cg(lambda z: oop.normal(z, lam), rhs[b].astype(np.complex128), 100, 1e-3)
        assert abs(int(it2[b]) - ito) <= 1 and rel2[b] <= 1e-3
    op.close()
