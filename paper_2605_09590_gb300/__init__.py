"""GB300-native PICO noise-map hot path: thin Python binding of ``libpico``.

``libpico.so`` (built from ``csrc/`` for sm_103a, see ``build.py``) exposes the
C ABI declared in ``include/pico.h``.  This module only marshals arguments:
every step of the path -- probe draws, the SENSE normal operator, batched CG,
accumulation, PMR noise and its adjoint -- runs in the library's CUDA
kernels.  PyTorch supplies device memory and the CUDA stream.  There is no CPU
fallback: if the library is missing the calls raise.

The functions carry the ABI's names (``pico_init``, ``pico_apply_normal``,
``pico_cg_batch``, ``pico_variance_map``, ``pico_pmr``, ...); ``Operator`` is a
small owner object over one context.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpico.so")

PICO_OK, PICO_E_INVALID, PICO_E_OOM, PICO_E_CUDA, PICO_E_TIMEOUT, PICO_E_BREAKDOWN, PICO_E_UNSUPPORTED = range(7)
PICO_CARTESIAN, PICO_SPIRAL = 0, 1
PICO_PROBE_PHASE, PICO_PROBE_RADEMACHER, PICO_PROBE_GAUSS = 0, 1, 2
PICO_SOLVER_GLOBAL, PICO_SOLVER_COLUMNS = 0, 1
STATUS_NAMES = ["PICO_OK", "PICO_E_INVALID", "PICO_E_OOM", "PICO_E_CUDA", "PICO_E_TIMEOUT",
                "PICO_E_BREAKDOWN", "PICO_E_UNSUPPORTED"]


class PicoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


class pico_operator_desc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("ny", ctypes.c_int32), ("nx", ctypes.c_int32), ("ncoils", ctypes.c_int32),
        ("smaps", ctypes.c_void_p), ("noise_cov", ctypes.c_void_p), ("mask", ctypes.c_void_p),
        ("mask_2d", ctypes.c_int32), ("traj", ctypes.c_void_p), ("nsamp", ctypes.c_int64),
        ("oversamp", ctypes.c_float), ("kb_width", ctypes.c_int32), ("lambda_", ctypes.c_double),
        ("power_iters", ctypes.c_int32), ("power_margin", ctypes.c_double), ("max_batch", ctypes.c_int32),
        ("max_iter_cap", ctypes.c_int32),
    ]


class pico_info(ctypes.Structure):
    _fields_ = [
        ("lambda_max", ctypes.c_double), ("lambda_phys", ctypes.c_double), ("kind", ctypes.c_int32),
        ("ny", ctypes.c_int32), ("nx", ctypes.c_int32), ("ncoils", ctypes.c_int32), ("max_batch", ctypes.c_int32),
        ("max_iter_cap", ctypes.c_int32), ("nsamp", ctypes.c_int64), ("device_bytes", ctypes.c_uint64),
        ("normal_op", ctypes.c_int32),
    ]


class pico_tuning(ctypes.Structure):
    _fields_ = [
        ("gram_min_batch", ctypes.c_int32), ("gram_kc", ctypes.c_int32), ("gram_a_tmem", ctypes.c_int32),
        ("probe_batch", ctypes.c_int32),
    ]


class pico_request(ctypes.Structure):
    _fields_ = [
        ("op", pico_operator_desc), ("seed", ctypes.c_uint64), ("nprobes", ctypes.c_int32),
        ("probe_kind", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("rtol", ctypes.c_double),
        ("pmr_reps", ctypes.c_int32), ("pmr_sigma", ctypes.c_double),
        ("cs_data", ctypes.c_void_p), ("cs_lambda", ctypes.c_double), ("cs_iters", ctypes.c_int32),
        ("cs_levels", ctypes.c_int32),
    ]


class pico_request_info(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_int64), ("status", ctypes.c_int32), ("t_arrival", ctypes.c_double),
        ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("footprint_bytes", ctypes.c_int64),
    ]


_lib: Optional[ctypes.CDLL] = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load ``libpico.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpico is not built ({path} missing); run paper_2605_09590_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sigs = {
        "pico_init": ([ctypes.POINTER(pico_operator_desc), vp, ctypes.c_size_t, ctypes.POINTER(vp)], i32),
        "pico_get_info": ([vp, ctypes.POINTER(pico_info)], i32),
        "pico_apply_normal": ([vp, vp, vp, i32], i32),
        "pico_cg_batch": ([vp, vp, vp, i32, i32, f64, vp, vp], i32),
        "pico_forward": ([vp, vp, vp, i32], i32),
        "pico_adjoint": ([vp, vp, vp, i32], i32),
        "pico_variance_map": ([vp, u64, i64, i32, i32, i32, f64, vp, vp, i32], i32),
        "pico_pmr": ([vp, u64, i64, i32, f64, i32, f64, vp, vp, i32], i32),
        "pico_variance_map_adaptive": ([vp, u64, i32, i32, i64, i32, f64, f64, vp, vp,
                                        ctypes.POINTER(i64), ctypes.POINTER(f64)], i32),
        "pico_finalize": ([vp, vp, vp, i64, vp, vp], i32),
        "pico_cs_recon": ([vp, vp, f64, i32, i32, vp], i32),
        "pico_cs_jvp": ([vp, vp, vp, i32], i32),
        "pico_cs_vjp": ([vp, vp, vp, i32], i32),
        "pico_cs_variance_map": ([vp, u64, i64, i32, i32, vp, vp, i32], i32),
        "pico_cs_pmr": ([vp, u64, i64, i32, f64, vp, vp, i32], i32),
        "pico_wavelet": ([vp, vp, vp, i32, i32, i32], i32),
        "pico_gfactor": ([vp, vp, vp, f64, vp], i32),
        "pico_profile": ([vp, i32], i32),
        "pico_profile_read": ([vp, i32, ctypes.POINTER(f64), ctypes.POINTER(i64)], i32),
        "pico_launch_count": ([vp, ctypes.POINTER(i64), i32], i32),
        "pico_get_tuning": ([vp, ctypes.POINTER(pico_tuning)], i32),
        "pico_set_tuning": ([vp, ctypes.POINTER(pico_tuning)], i32),
        "pico_autotune": ([vp, i32, ctypes.POINTER(pico_tuning), ctypes.POINTER(f64), i32], i32),
        "pico_tune_select": ([ctypes.POINTER(f64), i32, i32, ctypes.POINTER(pico_tuning)], i32),
        "pico_inject_error": ([vp, i32, i32], i32),
        "pico_set_solver": ([vp, i32], i32),
        "pico_get_solver": ([vp, ctypes.POINTER(i32)], i32),
        "pico_cs_generation": ([vp, ctypes.POINTER(i64)], i32),
        "pico_footprint": ([ctypes.POINTER(pico_operator_desc), i32, ctypes.POINTER(ctypes.c_size_t)], i32),
        "pico_server_create": ([ctypes.c_size_t, i32, i32, ctypes.POINTER(vp)], i32),
        "pico_server_submit": ([vp, ctypes.POINTER(pico_request), ctypes.POINTER(i64)], i32),
        "pico_server_wait": ([vp, i64, vp, vp, ctypes.POINTER(pico_request_info)], i32),
        "pico_server_destroy": ([vp], i32),
        "pico_sync": ([vp], i32),
        "pico_last_error": ([vp], ctypes.c_char_p),
        "pico_destroy": ([vp], None),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(ctx, st: int):
    if st != PICO_OK:
        msg = load_library().pico_last_error(ctx).decode() if ctx else ""
        raise PicoError(st, msg)


def _dev_ptr(t, dtype, what: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t.data_ptr()


# ----------------------------------------------------------------------------
# functions with the ABI's names
# ----------------------------------------------------------------------------
def pico_init(smaps: np.ndarray, mask: Optional[np.ndarray] = None, noise_cov: Optional[np.ndarray] = None,
              traj: Optional[np.ndarray] = None, lam: float = 0.0, power_iters: int = 15,
              power_margin: float = 1.01, max_batch: int = 64, max_iter_cap: int = 128,
              oversamp: float = 2.0, kb_width: int = 6, stream=None, hbm_budget: int = 0) -> int:
    """Create a context (returns the opaque handle)."""
    lib = load_library()
    d, keep = make_desc(smaps, mask, noise_cov, traj, lam, power_iters, power_margin, max_batch, max_iter_cap,
                        oversamp, kb_width)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    h = ctypes.c_void_p()
    st = lib.pico_init(ctypes.byref(d), ctypes.c_void_p(stream), hbm_budget, ctypes.byref(h))
    if st != PICO_OK:
        msg = lib.pico_last_error(h).decode() if h.value else ""
        if h.value:
            lib.pico_destroy(h)
        raise PicoError(st, msg)
    return h.value


def make_desc(smaps, mask=None, noise_cov=None, traj=None, lam=0.0, power_iters=15, power_margin=1.01,
              max_batch=64, max_iter_cap=128, oversamp=2.0, kb_width=6):
    """``pico_operator_desc`` plus the arrays it points to (keep them alive)."""
    S = np.ascontiguousarray(smaps, dtype=np.complex64)
    nc, ny, nx = S.shape
    d = pico_operator_desc()
    d.kind = PICO_SPIRAL if traj is not None else PICO_CARTESIAN
    d.ny, d.nx, d.ncoils = ny, nx, nc
    keep = [S]
    d.smaps = S.ctypes.data
    if noise_cov is not None:
        C = np.ascontiguousarray(noise_cov, dtype=np.complex128)
        keep.append(C)
        d.noise_cov = C.ctypes.data
    if mask is not None:
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        keep.append(m)
        d.mask = m.ctypes.data
        d.mask_2d = 1 if m.ndim == 2 else 0
    if traj is not None:
        tr = np.ascontiguousarray(traj, dtype=np.float32)
        keep.append(tr)
        d.traj = tr.ctypes.data
        d.nsamp = tr.shape[0]
    d.oversamp, d.kb_width = oversamp, kb_width
    d.lambda_ = lam
    d.power_iters, d.power_margin = power_iters, power_margin
    d.max_batch, d.max_iter_cap = max_batch, max_iter_cap
    return d, keep


def pico_get_info(ctx) -> dict:
    info = pico_info()
    _check(ctx, load_library().pico_get_info(ctx, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in pico_info._fields_}


def pico_apply_normal(ctx, x, y) -> None:
    import torch
    _check(ctx, load_library().pico_apply_normal(ctx, _dev_ptr(x, torch.complex64, "x"),
                                                 _dev_ptr(y, torch.complex64, "y"), x.shape[0]))


def pico_forward(ctx, x, y) -> None:
    import torch
    _check(ctx, load_library().pico_forward(ctx, _dev_ptr(x, torch.complex64, "x"),
                                            _dev_ptr(y, torch.complex64, "y"), x.shape[0]))


def pico_adjoint(ctx, y, x) -> None:
    import torch
    _check(ctx, load_library().pico_adjoint(ctx, _dev_ptr(y, torch.complex64, "y"),
                                            _dev_ptr(x, torch.complex64, "x"), x.shape[0]))


def pico_cg_batch(ctx, rhs, x, max_iter: int, rtol: float = 0.0, stats: bool = False):
    import torch
    nb = rhs.shape[0]
    it = np.zeros(nb, dtype=np.int32) if stats else None
    rr = np.zeros(nb, dtype=np.float64) if stats else None
    _check(ctx, load_library().pico_cg_batch(
        ctx, _dev_ptr(rhs, torch.complex64, "rhs"), _dev_ptr(x, torch.complex64, "x"), nb, max_iter, rtol,
        it.ctypes.data if stats else None, rr.ctypes.data if stats else None))
    return (it, rr) if stats else None


def pico_variance_map(ctx, seed: int, probe_begin: int, nprobes: int, probe_kind: int, max_iter: int,
                      rtol: float, sum_, sumsq=None, accumulate: bool = False) -> None:
    import torch
    _check(ctx, load_library().pico_variance_map(
        ctx, seed & (2 ** 64 - 1), probe_begin, nprobes, probe_kind, max_iter, rtol,
        _dev_ptr(sum_, torch.float64, "sum"), None if sumsq is None else _dev_ptr(sumsq, torch.float64, "sumsq"),
        1 if accumulate else 0))


def pico_variance_map_adaptive(ctx, seed: int, probe_kind: int, chunk: int, max_probes: int, max_iter: int,
                               rtol: float, target: float, sum_, sumsq) -> tuple[int, float]:
    import torch
    used, rel = ctypes.c_int64(), ctypes.c_double()
    _check(ctx, load_library().pico_variance_map_adaptive(
        ctx, seed & (2 ** 64 - 1), probe_kind, chunk, max_probes, max_iter, rtol, target,
        _dev_ptr(sum_, torch.float64, "sum"), _dev_ptr(sumsq, torch.float64, "sumsq"),
        ctypes.byref(used), ctypes.byref(rel)))
    return used.value, rel.value


def pico_pmr(ctx, seed: int, rep_begin: int, nreps: int, sigma: float, max_iter: int, rtol: float, sum_,
             sumsq=None, accumulate: bool = False) -> None:
    import torch
    _check(ctx, load_library().pico_pmr(
        ctx, seed & (2 ** 64 - 1), rep_begin, nreps, sigma, max_iter, rtol, _dev_ptr(sum_, torch.float64, "sum"),
        None if sumsq is None else _dev_ptr(sumsq, torch.float64, "sumsq"), 1 if accumulate else 0))


def pico_cs_recon(ctx, b, lambda_l1: float, iters: int, levels: int, x) -> None:
    import torch
    _check(ctx, load_library().pico_cs_recon(ctx, _dev_ptr(b, torch.complex64, "b"), lambda_l1, iters, levels,
                                             _dev_ptr(x, torch.complex64, "x")))


def pico_cs_jvp(ctx, db, dx) -> None:
    import torch
    _check(ctx, load_library().pico_cs_jvp(ctx, _dev_ptr(db, torch.complex64, "db"),
                                           _dev_ptr(dx, torch.complex64, "dx"), dx.shape[0]))


def pico_cs_vjp(ctx, xbar, bbar) -> None:
    import torch
    _check(ctx, load_library().pico_cs_vjp(ctx, _dev_ptr(xbar, torch.complex64, "xbar"),
                                           _dev_ptr(bbar, torch.complex64, "bbar"), xbar.shape[0]))


def pico_cs_variance_map(ctx, seed: int, probe_begin: int, nprobes: int, probe_kind: int, sum_, sumsq=None,
                         accumulate: bool = False) -> None:
    import torch
    _check(ctx, load_library().pico_cs_variance_map(
        ctx, seed & (2 ** 64 - 1), probe_begin, nprobes, probe_kind, _dev_ptr(sum_, torch.float64, "sum"),
        None if sumsq is None else _dev_ptr(sumsq, torch.float64, "sumsq"), 1 if accumulate else 0))


def pico_cs_pmr(ctx, seed: int, rep_begin: int, nreps: int, sigma: float, sum_, sumsq=None,
                accumulate: bool = False) -> None:
    import torch
    _check(ctx, load_library().pico_cs_pmr(
        ctx, seed & (2 ** 64 - 1), rep_begin, nreps, sigma, _dev_ptr(sum_, torch.float64, "sum"),
        None if sumsq is None else _dev_ptr(sumsq, torch.float64, "sumsq"), 1 if accumulate else 0))


def pico_wavelet(ctx, x, out, levels: int, inverse: bool = False) -> None:
    import torch
    _check(ctx, load_library().pico_wavelet(ctx, _dev_ptr(x, torch.complex64, "x"),
                                            _dev_ptr(out, torch.complex64, "out"), x.shape[0], levels,
                                            1 if inverse else 0))


def pico_finalize(ctx, sum_, sumsq, count: int, var=None, stderr=None) -> None:
    import torch
    _check(ctx, load_library().pico_finalize(
        ctx, _dev_ptr(sum_, torch.float64, "sum"), None if sumsq is None else _dev_ptr(sumsq, torch.float64, "sumsq"),
        count, None if var is None else _dev_ptr(var, torch.float32, "var"),
        None if stderr is None else _dev_ptr(stderr, torch.float32, "stderr")))


def pico_gfactor(ctx, var_acc, var_ref, R: float, g) -> None:
    import torch
    _check(ctx, load_library().pico_gfactor(ctx, _dev_ptr(var_acc, torch.float32, "var_acc"),
                                            _dev_ptr(var_ref, torch.float32, "var_ref"), R,
                                            _dev_ptr(g, torch.float32, "g")))


def pico_profile(ctx, enable: bool) -> None:
    _check(ctx, load_library().pico_profile(ctx, 1 if enable else 0))


def pico_profile_read(ctx, kernel_class: int) -> tuple[float, int]:
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(ctx, load_library().pico_profile_read(ctx, kernel_class, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def pico_launch_count(ctx, reset: bool = False) -> int:
    n = ctypes.c_int64()
    _check(ctx, load_library().pico_launch_count(ctx, ctypes.byref(n), 1 if reset else 0))
    return n.value


def pico_get_tuning(ctx) -> dict:
    t = pico_tuning()
    _check(ctx, load_library().pico_get_tuning(ctx, ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in pico_tuning._fields_}


def pico_set_tuning(ctx, tuning: dict) -> None:
    t = pico_tuning(**{f: int(tuning[f]) for f, _ in pico_tuning._fields_})
    _check(ctx, load_library().pico_set_tuning(ctx, ctypes.byref(t)))


AUTOTUNE_CANDIDATES = ("fft", "gram16", "gram16_tmem", "gram8")


def pico_autotune(ctx, iters: int = 0) -> tuple[dict, dict]:
    """Measure and apply the fastest tuning; returns (tuning, {candidate: {batch: us per image-iteration}})."""
    t = pico_tuning()
    times = (ctypes.c_double * 24)()
    _check(ctx, load_library().pico_autotune(ctx, iters, ctypes.byref(t), times, 24))
    mb = pico_get_info(ctx)["max_batch"]
    batches = (16, 32, 64, 128, 256, mb)
    table = {}
    for k, name in enumerate(AUTOTUNE_CANDIDATES):
        row = {b: times[k * 6 + i] for i, b in enumerate(batches) if times[k * 6 + i] == times[k * 6 + i]}
        if row:
            table[name] = row
    return {f: getattr(t, f) for f, _ in pico_tuning._fields_}, table


def pico_tune_select(table: dict, max_batch: int, gram: bool = True) -> dict:
    """The autotuner's choice for a table {candidate: {batch: us per image-iteration}} (host only)."""
    batches = (16, 32, 64, 128, 256, max_batch)
    times = (ctypes.c_double * 24)(*([float("nan")] * 24))
    for k, name in enumerate(AUTOTUNE_CANDIDATES):
        for i, b in enumerate(batches):
            if b in table.get(name, {}):
                times[k * 6 + i] = table[name][b]
    t = pico_tuning()
    _check(None, load_library().pico_tune_select(times, max_batch, 1 if gram else 0, ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in pico_tuning._fields_}


def pico_sync(ctx) -> None:
    _check(ctx, load_library().pico_sync(ctx))


def pico_set_solver(ctx, solver: int) -> None:
    """PICO_SOLVER_GLOBAL (CG on the whole image) or PICO_SOLVER_COLUMNS (CG per
    readout column of a phase-encode Cartesian operator)."""
    _check(ctx, load_library().pico_set_solver(ctx, solver))


def pico_get_solver(ctx) -> int:
    v = ctypes.c_int32()
    _check(ctx, load_library().pico_get_solver(ctx, ctypes.byref(v)))
    return v.value


def pico_inject_error(ctx, status: int, code: int = 1) -> None:
    """Host-side fault injection: the next ``pico_sync`` reports ``status``
    (PICO_E_TIMEOUT or PICO_E_BREAKDOWN) exactly as if a kernel had set it."""
    _check(ctx, load_library().pico_inject_error(ctx, status, code))


def pico_cs_generation(ctx) -> int:
    g = ctypes.c_int64()
    _check(ctx, load_library().pico_cs_generation(ctx, ctypes.byref(g)))
    return g.value


def pico_last_error(ctx) -> str:
    return load_library().pico_last_error(ctx).decode()


def pico_destroy(ctx) -> None:
    if ctx:
        load_library().pico_destroy(ctx)


# ----------------------------------------------------------------------------
# owner object
# ----------------------------------------------------------------------------
class Operator:
    """One acquisition's whitened encoding operator and its GPU workspace."""

    def __init__(self, smaps, mask=None, noise_cov=None, traj=None, **kw):
        import torch
        self.torch = torch
        self.ctx = pico_init(smaps, mask=mask, noise_cov=noise_cov, traj=traj, **kw)
        self.info = pico_get_info(self.ctx)
        self.ny, self.nx = self.info["ny"], self.info["nx"]
        import hashlib
        h = hashlib.sha1()
        for a in (mask, traj):
            if a is not None:
                h.update(np.ascontiguousarray(np.asarray(a)).tobytes())
        self._shape_key = "k{kind}_{ny}x{nx}_c{ncoils}_b{max_batch}_op{normal_op}".format(**self.info) + \
            "_" + h.hexdigest()[:16]

    @property
    def tuning(self) -> dict:
        return pico_get_tuning(self.ctx)

    @property
    def solver(self) -> int:
        return pico_get_solver(self.ctx)

    def set_solver(self, solver) -> None:
        """``"global"`` / ``"columns"`` (or the PICO_SOLVER_* values)."""
        if isinstance(solver, str):
            solver = {"global": PICO_SOLVER_GLOBAL, "columns": PICO_SOLVER_COLUMNS}[solver]
        pico_set_solver(self.ctx, solver)

    def set_tuning(self, **fields) -> None:
        t = self.tuning
        t.update(fields)
        pico_set_tuning(self.ctx, t)

    def autotune(self, cache: Optional[str] = None, iters: int = 0) -> dict:
        """Pick the launch shapes for this operator on this GPU (pico_autotune).

        With ``cache`` (a JSON file path) a tuning measured earlier for the same
        operator shape, mask / trajectory, batch capacity and device is reused,
        and a new measurement is stored there."""
        import json
        key = self._shape_key + "_" + self.torch.cuda.get_device_name().replace(" ", "-")
        db = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                db = json.load(f)
            if key in db:
                pico_set_tuning(self.ctx, db[key]["tuning"])
                self.autotune_table = db[key].get("us_per_image_iteration", {})
                return self.tuning
        tuning, table = pico_autotune(self.ctx, iters)
        self.autotune_table = table
        if cache:
            db[key] = {"tuning": tuning,
                       "us_per_image_iteration": {k: {str(b): v for b, v in r.items()} for k, r in table.items()}}
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(db, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return tuning

    def close(self):
        if self.ctx:
            pico_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _img(self, nb, dtype=None):
        t = self.torch
        return t.empty((nb, self.ny, self.nx), dtype=dtype or t.complex64, device="cuda")

    def apply_normal(self, x):
        y = self.torch.empty_like(x)
        pico_apply_normal(self.ctx, x, y)
        return y

    def kspace_shape(self, nb):
        nc = self.info["ncoils"]
        if self.info["kind"] == PICO_CARTESIAN:
            return (nb, nc, self.ny, self.nx)
        return (nb, nc, self.info["nsamp"])

    def forward(self, x):
        y = self.torch.empty(self.kspace_shape(x.shape[0]), dtype=self.torch.complex64, device=x.device)
        pico_forward(self.ctx, x, y)
        return y

    def adjoint(self, y):
        x = self.torch.empty((y.shape[0], self.ny, self.nx), dtype=self.torch.complex64, device=y.device)
        pico_adjoint(self.ctx, y, x)
        return x

    def cg(self, rhs, max_iter, rtol=0.0, stats=False):
        x = self.torch.empty_like(rhs)
        st = pico_cg_batch(self.ctx, rhs, x, max_iter, rtol, stats)
        return (x, *st) if stats else x

    def variance_sums(self, seed, nprobes, max_iter, rtol=0.0, probe_begin=0, kind=PICO_PROBE_PHASE,
                      sum_=None, sumsq=None):
        t = self.torch
        acc = sum_ is not None
        if sum_ is None:
            sum_ = t.empty((self.ny, self.nx), dtype=t.float64, device="cuda")
            sumsq = t.empty_like(sum_)
        pico_variance_map(self.ctx, seed, probe_begin, nprobes, kind, max_iter, rtol, sum_, sumsq, acc)
        return sum_, sumsq

    def pmr_sums(self, seed, nreps, sigma, max_iter, rtol=0.0, rep_begin=0, sum_=None, sumsq=None):
        t = self.torch
        acc = sum_ is not None
        if sum_ is None:
            sum_ = t.empty((self.ny, self.nx), dtype=t.float64, device="cuda")
            sumsq = t.empty_like(sum_)
        pico_pmr(self.ctx, seed, rep_begin, nreps, sigma, max_iter, rtol, sum_, sumsq, acc)
        return sum_, sumsq

    def finalize(self, sum_, sumsq, count):
        t = self.torch
        var = t.empty((self.ny, self.nx), dtype=t.float32, device="cuda")
        se = t.empty_like(var)
        pico_finalize(self.ctx, sum_, sumsq, count, var, se)
        return var, se

    def sync(self):
        pico_sync(self.ctx)


# ----------------------------------------------------------------------------
# nonlinear CS reconstruction as a differentiable function
# ----------------------------------------------------------------------------
def cs_function():
    """``torch.autograd.Function`` of the L1-wavelet FISTA reconstruction ``x = f(b)``.

    ``apply(op, b, lambda_l1, iters, levels)`` reconstructs one acquisition
    (``b``: whitened k-space of ``op``'s layout).  Backward returns
    ``J^T grad_x`` (``pico_cs_vjp``; the real-inner-product adjoint, which is
    PyTorch's convention for complex gradients), forward-mode AD ``J db``
    (``pico_cs_jvp``).  The context keeps the iterates of its most recent
    reconstruction only, so backward and jvp raise ``PicoError`` if another
    reconstruction has run on the same operator since this output's forward.
    """
    import torch

    class CSRecon(torch.autograd.Function):
        @staticmethod
        def forward(ctx, op, b, lambda_l1, iters, levels):
            x = torch.empty((op.ny, op.nx), dtype=torch.complex64, device=b.device)
            pico_cs_recon(op.ctx, b.detach().contiguous(), lambda_l1, iters, levels, x)
            ctx.op = op
            ctx.kshape = tuple(b.shape)
            ctx.generation = pico_cs_generation(op.ctx)
            return x

        @staticmethod
        def _check_point(ctx):
            if pico_cs_generation(ctx.op.ctx) != ctx.generation:
                raise PicoError(PICO_E_INVALID, "the operator ran another CS reconstruction after this output's "
                                                "forward; its Jacobian is no longer stored")

        @staticmethod
        def backward(ctx, grad_x):
            CSRecon._check_point(ctx)
            op = ctx.op
            bbar = torch.empty((1,) + ctx.kshape, dtype=torch.complex64, device=grad_x.device)
            pico_cs_vjp(op.ctx, grad_x.contiguous().reshape(1, op.ny, op.nx), bbar)
            return None, bbar.reshape(ctx.kshape), None, None, None

        @staticmethod
        def jvp(ctx, _op, db, *_):
            CSRecon._check_point(ctx)
            op = ctx.op
            dx = torch.empty((1, op.ny, op.nx), dtype=torch.complex64, device=db.device)
            pico_cs_jvp(op.ctx, db.contiguous().reshape((1,) + ctx.kshape), dx)
            return dx.reshape(op.ny, op.nx)

    return CSRecon


# ----------------------------------------------------------------------------
# serving runtime
# ----------------------------------------------------------------------------
class Server:
    """Noise-map request server (``pico_server_*``): submit from any thread, wait for results."""

    def __init__(self, hbm_budget: int = 0, max_active: int = 4, chunk: int = 64):
        self.lib = load_library()
        h = ctypes.c_void_p()
        st = self.lib.pico_server_create(hbm_budget, max_active, chunk, ctypes.byref(h))
        if st != PICO_OK:
            raise PicoError(st, "pico_server_create")
        self.h = h.value
        self.shapes = {}

    def submit(self, smaps, mask=None, traj=None, noise_cov=None, lam=0.0, seed=0, nprobes=32,
               probe_kind=PICO_PROBE_PHASE, max_iter=30, rtol=0.0, pmr_reps=0, pmr_sigma=1.0,
               power_iters=15, max_batch=64, cs_data=None, cs_lambda=0.0, cs_iters=100, cs_levels=4) -> int:
        """Queue one request; with ``cs_data`` (whitened k-space, complex64,
        layout of ``Operator.forward``) the maps are those of the L1-wavelet
        CS reconstruction (Jacobian PICO and CS PMR)."""
        d, keep = make_desc(smaps, mask, noise_cov, traj, lam, power_iters, 1.01, max_batch, 128)
        r = pico_request()
        r.op = d
        r.seed, r.nprobes, r.probe_kind, r.max_iter, r.rtol = seed & (2 ** 64 - 1), nprobes, probe_kind, max_iter, rtol
        r.pmr_reps, r.pmr_sigma = pmr_reps, pmr_sigma
        if cs_data is not None:
            cs = np.ascontiguousarray(cs_data, dtype=np.complex64)
            keep.append(cs)
            r.cs_data, r.cs_lambda, r.cs_iters, r.cs_levels = cs.ctypes.data, cs_lambda, cs_iters, cs_levels
        rid = ctypes.c_int64()
        st = self.lib.pico_server_submit(self.h, ctypes.byref(r), ctypes.byref(rid))
        if st != PICO_OK:
            raise PicoError(st, "pico_server_submit")
        self.shapes[rid.value] = (d.ny, d.nx, pmr_reps > 0)
        return rid.value

    def wait(self, rid: int):
        ny, nx, has_pmr = self.shapes.pop(rid)
        var = np.zeros((ny, nx), dtype=np.float64)
        pmr = np.zeros((ny, nx), dtype=np.float64) if has_pmr else None
        info = pico_request_info()
        st = self.lib.pico_server_wait(self.h, rid, var.ctypes.data, None if pmr is None else pmr.ctypes.data,
                                       ctypes.byref(info))
        if st != PICO_OK:
            raise PicoError(st, f"request {rid}")
        return var, pmr, {f: getattr(info, f) for f, _ in pico_request_info._fields_}

    def close(self):
        if self.h:
            self.lib.pico_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pico_footprint(smaps, mask=None, traj=None, with_kspace=False, **kw) -> int:
    d, keep = make_desc(smaps, mask, kw.pop("noise_cov", None), traj, **kw)
    out = ctypes.c_size_t()
    _check(None, load_library().pico_footprint(ctypes.byref(d), 1 if with_kspace else 0, ctypes.byref(out)))
    return out.value


# ----------------------------------------------------------------------------
# host-side sharding of probes across ranks (one process per GPU)
# ----------------------------------------------------------------------------
def shard_range(total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous probe range ``(begin, count)`` of ``rank`` out of ``world``."""
    base, extra = divmod(total, world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def reduce_running_sums(sums, group=None) -> None:
    """Combine the running sums of all ranks in place: the one exchange of a
    sharded map.  Probes (and PMR replicas) are independent (Alg. 1), so the
    sums over all probes are the sums of the ranks' partial sums.

    ``sums``: equally shaped float64 tensors on this rank's device (e.g. the
    PICO ``sum``/``sumsq`` and PMR ``sum``/``sumsq`` maps); they are packed
    into one buffer, summed over the process group with one all-reduce, and
    written back, so every rank ends with the totals.  Summation order across
    ranks is the collective's; within a rank the probe order is kept."""
    import torch
    import torch.distributed as dist
    if not sums:
        return
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return
    flat = torch.cat([t.reshape(-1) for t in sums])
    dist.all_reduce(flat, group=group)
    off = 0
    for t in sums:
        n = t.numel()
        t.copy_(flat[off:off + n].view_as(t))
        off += n
