"""ctypes binding of libystat (include/ystat.h): argument marshalling only.

Every step of the estimator runs in the library's CUDA kernels.  This module turns
torch CUDA tensors (or numpy arrays, for the host entry point) into the C structs
and back; it computes nothing itself.  If libystat.so has not been built, loading
fails with an ImportError-style RuntimeError -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libystat.so")
HEADER = os.path.join(HERE, "..", "include", "ystat.h")

YS_OK, YS_ERR_ARG, YS_ERR_OOM, YS_ERR_CUDA, YS_ERR_TIMEOUT, YS_ERR_UNSUPPORTED, YS_ERR_STATE = range(7)
ASSIGN = {"ngp": 1, "cic": 2, "tsc": 3}


class YsConfig(ctypes.Structure):
    _fields_ = [
        ("n_mesh", ctypes.c_int32),
        ("box_min", ctypes.c_double * 3),
        ("box_len", ctypes.c_double),
        ("observer", ctypes.c_double * 3),
        ("assign", ctypes.c_int32),
        ("interlace", ctypes.c_int32),
        ("compensate", ctypes.c_int32),
        ("ell_max", ctypes.c_int32),
        ("k_min", ctypes.c_double),
        ("dk", ctypes.c_double),
        ("n_bins", ctypes.c_int32),
        ("alpha", ctypes.c_double),
        ("max_particles", ctypes.c_int64),
        ("stream", ctypes.c_void_p),
    ]


class YsCatalog(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_void_p),
        ("y", ctypes.c_void_p),
        ("z", ctypes.c_void_p),
        ("w", ctypes.c_void_p),
        ("nbar", ctypes.c_void_p),
        ("n", ctypes.c_int64),
    ]


class YsResult(ctypes.Structure):
    _fields_ = [
        ("k_mean", ctypes.c_void_p),
        ("n_modes", ctypes.c_void_p),
        ("p0", ctypes.c_void_p),
        ("p2", ctypes.c_void_p),
        ("p4", ctypes.c_void_p),
        ("alpha", ctypes.c_double),
        ("norm_I", ctypes.c_double),
        ("shot_noise", ctypes.c_double),
        ("p6", ctypes.c_void_p),
    ]


NUM_KERNEL_CLASSES = 8
KERNEL_CLASSES = ["particle_count", "tile_scan", "particle_bin", "tile_deposit", "yz_stage", "unused",
                  "x_combine", "finalize"]


class YsStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * NUM_KERNEL_CLASSES), ("ms", ctypes.c_double * NUM_KERNEL_CLASSES)]


class YsTuning(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32 * 3), ("yz_grid", ctypes.c_int32), ("ring_lead", ctypes.c_int32),
                ("assign_ms", ctypes.c_double),
                ("measure_ms", ctypes.c_double), ("x_pencils", ctypes.c_int32)]


class YstatError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib().ys_status_string(status).decode()
        if status == YS_ERR_CUDA:
            msg += ": " + _lib().ys_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} (status {status})")


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libystat.so is not built ({LIB_PATH}); run "
                               "python -m paper_1505_05341_gb300.build")
        lib = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        lib.ys_plan_create.argtypes = [ctypes.POINTER(YsConfig), ctypes.POINTER(P)]
        lib.ys_plan_device_bytes.argtypes = [P]
        lib.ys_plan_device_bytes.restype = ctypes.c_size_t
        lib.ys_assign.argtypes = [P, ctypes.POINTER(YsCatalog), ctypes.POINTER(YsCatalog)]
        lib.ys_measure_multipoles_async.argtypes = [P, P]
        lib.ys_measure_multipoles.argtypes = [P, ctypes.POINTER(YsResult)]
        lib.ys_estimate_host.argtypes = [P, ctypes.POINTER(YsCatalog), ctypes.POINTER(YsCatalog),
                                         ctypes.POINTER(YsResult)]
        lib.ys_plan_destroy.argtypes = [P]
        lib.ys_assign_noalloc.argtypes = [P, ctypes.POINTER(YsCatalog), ctypes.POINTER(YsCatalog)]
        lib.ys_randoms_cache.argtypes = [P, ctypes.POINTER(YsCatalog)]
        lib.ys_assign_cached.argtypes = [P, ctypes.POINTER(YsCatalog)]
        lib.ys_plan_set_profiling.argtypes = [P, ctypes.c_int]
        lib.ys_plan_set_fault_injection.argtypes = [P, ctypes.c_int64, ctypes.c_int32]
        lib.ys_plan_set_direct_assign.argtypes = [P, ctypes.c_int]
        lib.ys_plan_copy_mesh.argtypes = [P, P, ctypes.c_int64]
        lib.ys_plan_get_stats.argtypes = [P, ctypes.POINTER(YsStats), ctypes.c_int]
        lib.ys_plan_autotune.argtypes = [P, ctypes.POINTER(YsCatalog), ctypes.POINTER(YsCatalog), ctypes.c_int32,
                                         ctypes.POINTER(YsTuning)]
        lib.ys_batch_create.argtypes = [ctypes.POINTER(YsConfig), ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(P)]
        lib.ys_batch_result_stride.argtypes = [P]
        lib.ys_batch_result_stride.restype = ctypes.c_int64
        lib.ys_batch_autotune.argtypes = [P, ctypes.POINTER(YsCatalog), ctypes.POINTER(YsCatalog), ctypes.c_int32]
        lib.ys_batch_run.argtypes = [P, ctypes.POINTER(YsCatalog), ctypes.POINTER(YsCatalog), P, P]
        lib.ys_batch_destroy.argtypes = [P]
        F, D, I64 = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double), ctypes.c_int64
        lib.ys_mlp_create.argtypes = [F, ctypes.POINTER(P)]
        lib.ys_mlp_get_state.argtypes = [P, F, F, F, ctypes.POINTER(I64)]
        lib.ys_mlp_set_state.argtypes = [P, F, F, F, I64]
        lib.ys_mlp_forward.argtypes = [P, P, I64, P, P]
        lib.ys_mlp_gradient.argtypes = [P, P, P, I64, P, P, P]
        lib.ys_mlp_train_step.argtypes = [P, P, P, I64, ctypes.c_float, P, P]
        lib.ys_mlp_features.argtypes = [P, P, ctypes.c_int32, I64, ctypes.c_int32, ctypes.c_double, P, P, P, P, P]
        lib.ys_mlp_correct.argtypes = [P, P, ctypes.c_int32, I64, ctypes.c_int32, ctypes.c_double, P, P]
        lib.ys_mlp_destroy.argtypes = [P]
        lib.ys_wedges.argtypes = [P, ctypes.c_int32, I64, ctypes.c_int32, P, P]
        lib.ys_sum_gal.argtypes = [ctypes.POINTER(YsConfig), ctypes.POINTER(YsCatalog), ctypes.POINTER(YsCatalog),
                                   P, P]
        lib.ys_sum_grid.argtypes = [P, P, P]
        lib.ys_status_string.argtypes = [ctypes.c_int]
        lib.ys_status_string.restype = ctypes.c_char_p
        lib.ys_last_cuda_error.restype = ctypes.c_char_p
        for name in ("ys_plan_create", "ys_assign", "ys_measure_multipoles_async",
                     "ys_measure_multipoles", "ys_estimate_host", "ys_plan_destroy",
                     "ys_plan_set_profiling", "ys_plan_get_stats", "ys_assign_noalloc", "ys_plan_autotune",
                     "ys_plan_set_fault_injection", "ys_randoms_cache", "ys_assign_cached",
                     "ys_plan_set_direct_assign",
                     "ys_batch_create", "ys_batch_autotune", "ys_batch_run", "ys_batch_destroy",
                     "ys_mlp_create", "ys_mlp_get_state", "ys_mlp_set_state", "ys_mlp_forward",
                     "ys_mlp_gradient", "ys_mlp_train_step", "ys_mlp_features", "ys_mlp_correct",
                     "ys_mlp_destroy", "ys_wedges", "ys_sum_gal", "ys_sum_grid"):
            getattr(lib, name).restype = ctypes.c_int
        _LIB = lib
    return _LIB


def load_library():
    """Load libystat.so (raises if it is missing)."""
    return _lib()


def header_functions():
    """Names of the functions include/ystat.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ys_[a-z_]+)\s*\(", txt)))


@dataclasses.dataclass
class Result:
    k: np.ndarray
    n_modes: np.ndarray
    p0: np.ndarray
    p2: np.ndarray
    p4: np.ndarray
    alpha: float
    norm_I: float
    shot_noise: float
    status: int = YS_OK
    p6: np.ndarray | None = None   # l_max = 6 plans only


def _check(status, where, allow=()):
    if status != YS_OK and status not in allow:
        raise YstatError(status, where)
    return status


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def make_config(n_mesh, box_min, box_len, observer=(0.0, 0.0, 0.0), assign="cic", interlace=False,
                compensate=True, ell_max=4, k_min=0.0, dk=0.01, n_bins=None, k_max=None, alpha=-1.0,
                max_particles=0, stream=None):
    """A filled ys_config (shells of width dk from k_min up to k_max, default Nyquist)."""
    if n_bins is None:
        kmax = k_max if k_max is not None else np.pi * n_mesh / box_len
        n_bins = int(np.ceil((kmax - k_min) / dk - 1e-9))
    cfg = YsConfig()
    cfg.n_mesh = n_mesh
    cfg.box_min = (ctypes.c_double * 3)(*box_min)
    cfg.box_len = box_len
    cfg.observer = (ctypes.c_double * 3)(*observer)
    cfg.assign = ASSIGN[assign] if isinstance(assign, str) else int(assign)
    cfg.interlace = int(bool(interlace))
    cfg.compensate = int(bool(compensate))
    cfg.ell_max = ell_max
    cfg.k_min = k_min
    cfg.dk = dk
    cfg.n_bins = n_bins
    cfg.alpha = alpha
    cfg.max_particles = int(max_particles)
    cfg.stream = stream
    return cfg


def row_len(n_bins, ell_max=4):
    """Doubles in a result row: 5 n_bins + 5, plus n_bins of P_6 for l_max = 6."""
    return 5 * n_bins + 5 + (n_bins if ell_max >= 6 else 0)


def parse_row(row, n_bins, ell_max=4):
    """Split one result row [k | n_modes | p0 | p2 | p4 | alpha, I, S/I, n_out, timeout (| p6)]."""
    row = np.asarray(row, dtype=np.float64)
    nb = n_bins
    p6 = row[5 * nb + 5:6 * nb + 5].copy() if ell_max >= 6 else None
    return Result(row[:nb], row[nb:2 * nb], row[2 * nb:3 * nb], row[3 * nb:4 * nb], row[4 * nb:5 * nb],
                  float(row[5 * nb]), float(row[5 * nb + 1]), float(row[5 * nb + 2]),
                  YS_ERR_TIMEOUT if row[5 * nb + 4] != 0 else (YS_ERR_ARG if row[5 * nb + 3] > 0 else YS_OK), p6)


class Plan:
    """One estimator configuration on the current CUDA device (ys_plan)."""

    def __init__(self, n_mesh, box_min, box_len, observer=(0.0, 0.0, 0.0), assign="cic",
                 interlace=False, compensate=True, ell_max=4, k_min=0.0, dk=0.01, n_bins=None,
                 k_max=None, alpha=-1.0, max_particles=0, stream=None):
        lib = _lib()
        cfg = make_config(n_mesh, box_min, box_len, observer, assign, interlace, compensate, ell_max, k_min,
                          dk, n_bins, k_max, alpha, max_particles, stream)
        n_bins = cfg.n_bins
        self.cfg = cfg
        self.n_bins = n_bins
        self.ell_max = ell_max
        self.row_len = row_len(n_bins, ell_max)
        h = ctypes.c_void_p()
        _check(lib.ys_plan_create(ctypes.byref(cfg), ctypes.byref(h)), "ys_plan_create")
        self._h = h
        self._keep = None

    @property
    def device_bytes(self):
        return _lib().ys_plan_device_bytes(self._h)

    @staticmethod
    def _cat(x, y, z, w=None, nbar=None):
        c = YsCatalog()
        c.x, c.y, c.z, c.w, c.nbar = _ptr(x), _ptr(y), _ptr(z), _ptr(w), _ptr(nbar)
        c.n = int(x.shape[0])
        return c

    def assign(self, gal, ran):
        """gal, ran: dicts or tuples of device float32 tensors (x, y, z, w, nbar)."""
        g = self._cat(*gal)
        r = self._cat(*ran)
        self._keep = (gal, ran)
        _check(_lib().ys_assign(self._h, ctypes.byref(g), ctypes.byref(r)), "ys_assign")

    def cache_randoms(self, ran):
        """ys_randoms_cache: deposit these randoms once (device tensors x, y, z, w, nbar)."""
        r = self._cat(*ran)
        self._keep_ran = ran
        _check(_lib().ys_randoms_cache(self._h, ctypes.byref(r)), "ys_randoms_cache")

    def assign_cached(self, gal):
        """ys_assign_cached: the galaxies against the kept randoms."""
        g = self._cat(*gal)
        self._keep = (gal, None)
        _check(_lib().ys_assign_cached(self._h, ctypes.byref(g)), "ys_assign_cached")

    def measure_async(self, d_out=None):
        _check(_lib().ys_measure_multipoles_async(self._h, _ptr(d_out)), "ys_measure_multipoles_async")

    def _result_struct(self):
        nb = self.n_bins
        arrs = [np.empty(nb, dtype=np.float64) for _ in range(6)]
        res = YsResult()
        res.k_mean, res.n_modes, res.p0, res.p2, res.p4, res.p6 = [a.ctypes.data for a in arrs]
        return res, arrs

    def _result(self, res, arrs, st):
        return Result(*arrs[:5], res.alpha, res.norm_I, res.shot_noise, st,
                      arrs[5] if self.ell_max >= 6 else None)

    def measure(self, allow_outside=False):
        res, arrs = self._result_struct()
        st = _check(_lib().ys_measure_multipoles(self._h, ctypes.byref(res)), "ys_measure_multipoles",
                    allow=(YS_ERR_ARG,) if allow_outside else ())
        return self._result(res, arrs, st)

    def estimate_host(self, gal, ran):
        """End to end from host numpy float32 arrays (x, y, z, w, nbar)."""
        gal = [None if a is None else np.ascontiguousarray(a, dtype=np.float32) for a in gal]
        ran = [None if a is None else np.ascontiguousarray(a, dtype=np.float32) for a in ran]
        g = self._cat(*gal)
        r = self._cat(*ran)
        res, arrs = self._result_struct()
        st = _check(_lib().ys_estimate_host(self._h, ctypes.byref(g), ctypes.byref(r), ctypes.byref(res)),
                    "ys_estimate_host")
        return self._result(res, arrs, st)

    def autotune(self, gal, ran, reps=3):
        """ys_plan_autotune on device catalogues; returns the chosen YsTuning."""
        g, r, t = self._cat(*gal), self._cat(*ran), YsTuning()
        self._keep = (gal, ran)
        _check(_lib().ys_plan_autotune(self._h, ctypes.byref(g), ctypes.byref(r), reps, ctypes.byref(t)),
               "ys_plan_autotune")
        return t

    def sum_grid(self, wedges=False):
        """ys_sum_grid: the direct sum over this plan's assigned mesh nodes.  Returns the
        Result, and (P_perp, P_para) of the wedges' definition when ``wedges``."""
        import torch
        row = torch.empty(self.row_len, dtype=torch.float64, device="cuda")
        wd = torch.empty(2 * self.n_bins, dtype=torch.float64, device="cuda") if wedges else None
        _check(_lib().ys_sum_grid(self._h, _ptr(row), _ptr(wd)), "ys_sum_grid")
        res = parse_row(row.cpu().numpy(), self.n_bins, self.ell_max)
        if not wedges:
            return res
        w = wd.cpu().numpy()
        return res, (w[:self.n_bins], w[self.n_bins:])

    def mesh(self):
        """ys_plan_copy_mesh: the assigned mesh(es) as a host float32 array (m, n, n, n),
        x-major with z fastest; m = 2 when interlaced."""
        n = self.cfg.n_mesh
        m = 2 if self.cfg.interlace else 1
        out = np.empty((m, n, n, n), dtype=np.float32)
        _check(_lib().ys_plan_copy_mesh(self._h, out.ctypes.data, out.size), "ys_plan_copy_mesh")
        return out

    def set_fault_injection(self, wait_limit_ns=0, skip_plane=-1):
        """ys_plan_set_fault_injection: bound of the y,z-stage waits, and the plane whose
        completion is withheld (-1: none)."""
        _check(_lib().ys_plan_set_fault_injection(self._h, int(wait_limit_ns), int(skip_plane)),
               "ys_plan_set_fault_injection")

    def set_direct_assign(self, enable: bool):
        """ys_plan_set_direct_assign: reductions into an L2-resident mesh (True) or the
        tile-sorted assignment (False)."""
        _check(_lib().ys_plan_set_direct_assign(self._h, int(bool(enable))), "ys_plan_set_direct_assign")

    def set_profiling(self, enable: bool):
        _check(_lib().ys_plan_set_profiling(self._h, int(bool(enable))), "ys_plan_set_profiling")

    def stats(self, reset=False):
        """{kernel class: (launches, summed device ms)} since the last reset."""
        st = YsStats()
        _check(_lib().ys_plan_get_stats(self._h, ctypes.byref(st), int(bool(reset))), "ys_plan_get_stats")
        return {name: (int(st.launches[i]), float(st.ms[i])) for i, name in enumerate(KERNEL_CLASSES)}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().ys_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """ys_batch: many catalogues (mixed configurations) in one graph launch, measured in
    waves of up to `lanes` catalogues per configuration."""

    def __init__(self, configs, lanes=8):
        lib = _lib()
        n = len(configs)
        arr = (YsConfig * n)(*configs)
        h = ctypes.c_void_p()
        _check(lib.ys_batch_create(arr, n, lanes, ctypes.byref(h)), "ys_batch_create")
        self._h = h
        self.n = n
        self.n_bins = [c.n_bins for c in configs]
        self.ell_max = [c.ell_max for c in configs]
        self.stride = int(lib.ys_batch_result_stride(h))
        self._keep = None

    @staticmethod
    def _cats(cats):
        arr = (YsCatalog * len(cats))()
        for i, c in enumerate(cats):
            arr[i] = Plan._cat(*c)
        return arr

    def autotune(self, gals, rans, reps=2):
        _check(_lib().ys_batch_autotune(self._h, self._cats(gals), self._cats(rans), reps), "ys_batch_autotune")

    def run(self, gals, rans, d_results, stream=None):
        """gals, rans: lists of device tensor tuples; d_results: device float64 (n, stride)."""
        self._keep = (gals, rans, d_results)
        self._g, self._r = self._cats(gals), self._cats(rans)
        _check(_lib().ys_batch_run(self._h, self._g, self._r, _ptr(d_results), stream), "ys_batch_run")

    def results(self, d_results):
        host = d_results.cpu().numpy() if hasattr(d_results, "cpu") else np.asarray(d_results)
        return [parse_row(host[i], self.n_bins[i], self.ell_max[i]) for i in range(self.n)]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().ys_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


MLP_PARAMS = 8899


def _fptr(a):
    return ctypes.cast(a.ctypes.data, ctypes.POINTER(ctypes.c_float)) if a is not None else None


class Mlp:
    """ys_mlp: the learned aliasing/window correction network (device-resident).

    Device arrays are torch CUDA tensors (or anything with ``data_ptr``); feature rows
    are float32 (rows, 5), targets/outputs float32 (rows, 3), result rows float64."""

    def __init__(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != MLP_PARAMS:
            raise ValueError(f"expected {MLP_PARAMS} parameters, got {p.size}")
        h = ctypes.c_void_p()
        _check(_lib().ys_mlp_create(_fptr(p), ctypes.byref(h)), "ys_mlp_create")
        self._h = h

    def state(self):
        """(params, m, v, step) on the host."""
        w, m, v = (np.empty(MLP_PARAMS, np.float32) for _ in range(3))
        t = ctypes.c_int64()
        _check(_lib().ys_mlp_get_state(self._h, _fptr(w), _fptr(m), _fptr(v), ctypes.byref(t)), "ys_mlp_get_state")
        return w, m, v, int(t.value)

    def params(self):
        return self.state()[0]

    def set_state(self, params, m=None, v=None, step=0):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float32) for a in (params, m, v)]
        _check(_lib().ys_mlp_set_state(self._h, *(_fptr(a) for a in arrs), int(step)), "ys_mlp_set_state")

    def forward(self, d_x, d_y, rows=None, stream=None):
        rows = d_x.shape[0] if rows is None else rows
        _check(_lib().ys_mlp_forward(self._h, _ptr(d_x), rows, _ptr(d_y), stream), "ys_mlp_forward")

    def gradient(self, d_x, d_t, d_grad=None, d_sse=None, rows=None, stream=None):
        rows = d_x.shape[0] if rows is None else rows
        _check(_lib().ys_mlp_gradient(self._h, _ptr(d_x), _ptr(d_t), rows, _ptr(d_grad), _ptr(d_sse), stream),
               "ys_mlp_gradient")

    def train_step(self, d_x, d_t, lr, d_sse=None, rows=None, stream=None):
        rows = d_x.shape[0] if rows is None else rows
        _check(_lib().ys_mlp_train_step(self._h, _ptr(d_x), _ptr(d_t), rows, float(lr), _ptr(d_sse), stream),
               "ys_mlp_train_step")

    @staticmethod
    def features(d_rows, n_bins, k_nyq, d_x, d_src, d_count, d_fine_rows=None, d_t=None, stream=None):
        n_cat, stride = d_rows.shape
        _check(_lib().ys_mlp_features(_ptr(d_rows), _ptr(d_fine_rows), n_cat, stride, n_bins, float(k_nyq),
                                      _ptr(d_x), _ptr(d_t), _ptr(d_src), _ptr(d_count), stream), "ys_mlp_features")

    def correct(self, d_rows, n_bins, k_nyq, d_out, stream=None):
        n_cat, stride = d_rows.shape
        _check(_lib().ys_mlp_correct(self._h, _ptr(d_rows), n_cat, stride, n_bins, float(k_nyq), _ptr(d_out),
                                     stream), "ys_mlp_correct")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().ys_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def wedges(d_rows, n_bins, d_out, stream=None):
    """ys_wedges: (P_perp, P_para) of Eqs. 16-17 for the result rows d_rows (device
    float64 (n_cat, stride)) into d_out (device float64 (n_cat, 2, n_bins))."""
    n_cat, stride = d_rows.shape
    _check(_lib().ys_wedges(_ptr(d_rows), n_cat, stride, n_bins, _ptr(d_out), stream), "ys_wedges")


def sum_gal(n_mesh, box_min, box_len, gal, ran, observer=(0.0, 0.0, 0.0), ell_max=4, k_min=0.0, dk=0.01,
            n_bins=None, k_max=None, alpha=-1.0, wedges=False, stream=None):
    """ys_sum_gal: the galaxy direct sum at the half-grid modes of an n_mesh^3 lattice.
    gal, ran: tuples of device float32 tensors (x, y, z, w, nbar).  Returns the Result,
    and (P_perp, P_para) of the wedges' definition when ``wedges``."""
    import torch
    cfg = make_config(n_mesh, box_min, box_len, observer, "cic", False, False, ell_max, k_min, dk, n_bins,
                      k_max, alpha, 0, stream)
    nb = cfg.n_bins
    row = torch.empty(row_len(nb, ell_max), dtype=torch.float64, device="cuda")
    wd = torch.empty(2 * nb, dtype=torch.float64, device="cuda") if wedges else None
    g, r = Plan._cat(*gal), Plan._cat(*ran)
    _check(_lib().ys_sum_gal(ctypes.byref(cfg), ctypes.byref(g), ctypes.byref(r), _ptr(row), _ptr(wd)),
           "ys_sum_gal")
    res = parse_row(row.cpu().numpy(), nb, ell_max)
    if not wedges:
        return res
    w = wd.cpu().numpy()
    return res, (w[:nb], w[nb:])
