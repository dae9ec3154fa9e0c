"""g-factor maps end to end (Eq. 11): accelerated and reference PICO maps on
the GPU, combined by pico_gfactor, against the oracle.

* Cartesian 64 x 64, 8 coils with sum_c |S_c|^2 = 1, uniform R = 2 without
  calibration lines (the paper's analytic SENSE reference, Sec. 3.2.1):
  - same seed: the GPU maps equal the oracle's same-seed PICO maps to 1e-4,
    and so do the g maps computed from them;
  - against the closed form: the accelerated variance estimate lies in its
    sampling band around Pruessmann's R [(S^H S)^-1]_rr (|z| <= 6, at most 1 %
    beyond 3 sigma, the exact per-sample variance 1/2 |Sigma_kl|^2 of the 2 x 2
    alias blocks), the fully sampled reference map is exact (one probe,
    diagonal covariance), and the GPU g map agrees with the closed-form g to
    the delta-method bound of that band.
* Spiral 64 x 64 (the reference reading for lam > 0: all interleaves, the same
  coils and the same physical Tikhonov weight -- without it the reference is
  singular, the spiral leaves the k-space corners unsampled; R = interleaves /
  kept interleaves): the GPU maps equal the oracle's same-seed maps to 1e-4 of
  the largest exact variance at every voxel, the g maps agree to the bound that
  follows from it, and the 256-probe g map is within sampling error of the g of
  the exact dense covariances.
"""
import numpy as np
import pytest

import synth
from oracle import ops as O
from oracle import pico as OP

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


def _map(op, seed, K, iters=30):
    s, _ = op.variance_sums(seed, K, iters, 0.0)
    var, _ = op.finalize(s, torch.zeros_like(s), K)
    op.sync()
    return var, s.cpu().numpy()


def _g(op, var_acc, var_ref, R):
    g = torch.empty_like(var_acc)
    pico.pico_gfactor(op.ctx, var_acc, var_ref, R, g)
    op.sync()
    return g.cpu().numpy()


def test_cartesian_gfactor_same_seed_and_closed_form():
    n, nc, R = 64, 8, 2
    S = synth.coil_maps(n, n, nc, 3)
    mask_acc = synth.mask_pe(n, R, 0)
    mask_ref = np.ones(n, dtype=np.uint8)
    K, seed = 1024, 515
    acc = pico.Operator(S, mask=mask_acc, power_iters=0, max_batch=256)
    ref = pico.Operator(S, mask=mask_ref, power_iters=0, max_batch=8)
    va, sa = _map(acc, seed, K, 40)
    vr, sr = _map(ref, seed + 1, 1, 10)                 # one probe is exact for a diagonal covariance
    g = _g(acc, va, vr, R)
    # same seed: the oracle's maps from the same probes (a subset of probes keeps the oracle fast)
    oa, _ = OP.pico(O.Operator(S, None, mask=mask_acc), seed, 0, 32, 0.0, 40, 0.0)
    orf, _ = OP.pico(O.Operator(S, None, mask=mask_ref), seed + 1, 0, 1, 0.0, 10, 0.0)
    va32, sa32 = _map(acc, seed, 32, 40)
    g32 = _g(acc, va32, vr, R)
    d, _, per = OP.column_exact(O.Operator(S, None, mask=mask_acc))   # exact diag and 1/2 sum_{l!=k} |Sigma_kl|^2
    assert (np.abs(sa32 - oa) / 32 / d).max() < 1e-4                  # same-seed maps, per voxel
    g_o = OP.gfactor(oa / 32, orf, R)
    assert (np.abs(g32 - g_o) / g_o).max() < 1e-4
    # closed form (Pruessmann): exact reference, band for the accelerated map, g within its delta-method bound
    var_cf, vref_cf, g_cf = OP.sense_closed_form(S, R)
    assert np.abs(vr.cpu().numpy() - vref_cf).max() < 1e-5
    assert np.abs(d - var_cf).max() < 1e-9
    z = (va.cpu().numpy() - var_cf) / np.sqrt(per / K)
    assert np.all(np.abs(z) <= 6) and np.mean(np.abs(z) > 3) <= 0.01
    # g = sqrt(var / (R var_ref)): sd(g) = sd(var) / (2 g R var_ref)
    sd_g = np.sqrt(per / K) / (2 * g_cf * R * vref_cf)
    assert np.all(np.abs(g - g_cf) <= 6 * sd_g + 1e-6)
    acc.close()
    ref.close()


def test_spiral_gfactor_with_fully_sampled_reference():
    n, nc, L, ns = 64, 6, 16, 512
    S = synth.coil_maps(n, n, nc, 4)
    R = 2
    traj_acc = synth.spiral_traj(n, L, ns, R)
    traj_ref = synth.spiral_traj(n, L, ns, 1)
    oacc = O.Operator(S, None, traj=traj_acc)
    oref = O.Operator(S, None, traj=traj_ref)
    lam_a, _ = OP.lambda_phys(oacc, 0.1)                # one physical weight for both reconstructions
    K, seed = 256, 909
    acc = pico.Operator(S, traj=traj_acc, lam=lam_a, power_iters=0, max_batch=K)
    ref = pico.Operator(S, traj=traj_ref, lam=lam_a, power_iters=0, max_batch=K)
    va, sa = _map(acc, seed, K, 60)
    vr, sr = _map(ref, seed + 1, K, 60)
    g = _g(acc, va, vr, float(L) / (L // R))
    # same seed against the oracle's CG maps (a few probes)
    Ka = 8
    va8, sa8 = _map(acc, seed, Ka, 60)
    vr8, sr8 = _map(ref, seed + 1, Ka, 60)
    oa, _ = OP.pico(oacc, seed, 0, Ka, lam_a, 60, 0.0)
    orf, _ = OP.pico(oref, seed + 1, 0, Ka, lam_a, 60, 0.0)
    g8 = _g(acc, va8, vr8, float(L) / (L // R))
    Sa = OP.dense_cov(OP.dense_normal(oacc), lam_a)
    Sr = OP.dense_cov(OP.dense_normal(oref), lam_a)
    da, dr = np.real(np.diag(Sa)).reshape(n, n), np.real(np.diag(Sr)).reshape(n, n)
    assert np.abs(sa8 - oa).max() / Ka < 1e-4 * da.max()
    assert np.abs(sr8 - orf).max() / Ka < 1e-4 * dr.max()
    # g from the same-seed maps: the maps agree to ea = 1e-4 max(da) and er = 1e-4
    # max(dr) at every voxel, so g (a square root of their ratio) agrees to
    # 1/2 (ea / a + er / r) relative -- checked (with a factor 2) wherever both
    # errors are below 10 % of the 8-probe values
    a, r = oa / Ka, orf / Ka
    ea, er = 1e-4 * da.max(), 1e-4 * dr.max()
    ok = (a > 10 * ea) & (r > 10 * er)
    g_o = OP.gfactor(np.where(ok, a, 1.0), np.where(ok, r, 1.0), float(L) / (L // R))
    bound = 0.5 * (ea / np.where(ok, a, 1.0) + er / np.where(ok, r, 1.0))
    assert ok.mean() > 0.3
    assert np.all((np.abs(g8 - g_o) <= 2 * bound * g_o)[ok])
    # the 256-probe g map against the g of the exact covariances (sampling error only)
    g_ex = OP.gfactor(da, dr, float(L) / (L // R))
    assert np.median(np.abs(g - g_ex) / g_ex) < 0.05
    acc.close()
    ref.close()
