"""The C ABI: the library loads, exports every function include/ystat.h declares,
and validates arguments on the host (no GPU needed for any of this)."""
import ctypes

import pytest

import paper_1505_05341_gb300 as ys
from paper_1505_05341_gb300 import ystat


def test_library_exports_every_header_function():
    lib = ys.load_library()
    names = ys.header_functions()
    assert {"ys_plan_create", "ys_assign", "ys_measure_multipoles", "ys_plan_destroy"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings():
    lib = ys.load_library()
    for s in range(7):
        assert lib.ys_status_string(s)
    assert lib.ys_status_string(99) == b"unknown status"


def _cfg(**kw):
    c = ystat.YsConfig()
    c.n_mesh = kw.get("n_mesh", 32)
    c.box_min = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    c.box_len = kw.get("box_len", 100.0)
    c.observer = (ctypes.c_double * 3)(-10.0, 0.0, 0.0)
    c.assign = kw.get("assign", 2)
    c.interlace = kw.get("interlace", 0)
    c.compensate = 1
    c.ell_max = kw.get("ell_max", 4)
    c.k_min = 0.0
    c.dk = kw.get("dk", 0.01)
    c.n_bins = kw.get("n_bins", 10)
    c.alpha = -1.0
    c.max_particles = 0
    c.stream = None
    return c


@pytest.mark.parametrize("kw,status", [
    (dict(n_mesh=100), ystat.YS_ERR_UNSUPPORTED),
    (dict(n_mesh=48), ystat.YS_ERR_UNSUPPORTED),
    (dict(box_len=-1.0), ystat.YS_ERR_ARG),
    (dict(assign=4), ystat.YS_ERR_ARG),
    (dict(ell_max=3), ystat.YS_ERR_ARG),
    (dict(n_bins=0), ystat.YS_ERR_ARG),
    (dict(dk=0.0), ystat.YS_ERR_ARG),
    (dict(interlace=2), ystat.YS_ERR_ARG),
])
def test_invalid_config_rejected_on_host(kw, status):
    lib = ys.load_library()
    h = ctypes.c_void_p()
    assert lib.ys_plan_create(ctypes.byref(_cfg(**kw)), ctypes.byref(h)) == status
    assert not h.value


def test_null_arguments():
    lib = ys.load_library()
    assert lib.ys_plan_create(None, None) == ystat.YS_ERR_ARG
    assert lib.ys_assign(None, None, None) == ystat.YS_ERR_ARG
    assert lib.ys_measure_multipoles(None, None) == ystat.YS_ERR_ARG
    assert lib.ys_plan_destroy(None) == ystat.YS_OK
    assert lib.ys_plan_device_bytes(None) == 0


def test_no_gpu_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = ys.load_library()
    h = ctypes.c_void_p()
    assert lib.ys_plan_create(ctypes.byref(_cfg()), ctypes.byref(h)) == ystat.YS_ERR_CUDA
    with pytest.raises(ys.YstatError):
        ys.Plan(32, (0.0, 0.0, 0.0), 100.0)
