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
    assert lib.ys_plan_copy_mesh(None, None, 0) == ystat.YS_ERR_ARG
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


# C types of the header's struct members and the ctypes types the binding must use
_CTYPES = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double}


def _header_structs():
    """{name: [(member, ctypes type)]} for every typedef struct of include/ystat.h."""
    import os
    import re
    path = os.path.join(os.path.dirname(ys.__file__), "..", "include", "ystat.h")
    text = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(\w+)\s+(\d+)", text)}
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+);", text, flags=re.S):
        members = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            m = re.fullmatch(r"(?:const\s+)?(\w+)\s*(\*?)\s*(\w+)(?:\[(\w+)\])?", decl)
            assert m, decl
            ctype, star, member, dim = m.groups()
            t = ctypes.c_void_p if star else _CTYPES[ctype]
            if dim:
                t = t * (int(dim) if dim.isdigit() else consts[dim])
            members.append((member, t))
        out[name] = members
    return out


@pytest.mark.parametrize("cname,pyname", [("ys_config", "YsConfig"), ("ys_catalog", "YsCatalog"),
                                          ("ys_result", "YsResult"), ("ys_stats", "YsStats"),
                                          ("ys_tuning", "YsTuning")])
def test_binding_structs_match_header(cname, pyname):
    """Every ctypes structure of the binding has the header's members, in order, with
    the same C types (so sizes and offsets agree)."""
    want = _header_structs()[cname]
    got = getattr(ystat, pyname)._fields_
    assert [n for n, _ in got] == [n for n, _ in want]
    for (n, t_got), (_, t_want) in zip(got, want):
        assert ctypes.sizeof(t_got) == ctypes.sizeof(t_want), n
        base = lambda t: getattr(t, "_type_", t)
        assert base(t_got) == base(t_want) or (t_got is ctypes.c_void_p and t_want is ctypes.c_void_p), n


def test_every_header_function_is_documented():
    """Each entry point of include/ystat.h is preceded by its own comment block (only
    #define and typedef lines may sit between them), of some substance."""
    import os
    import re
    path = os.path.join(os.path.dirname(ys.__file__), "..", "include", "ystat.h")
    text = open(path).read()
    names = ys.header_functions()
    assert names
    for name in names:
        m = re.search(r"^[\w\s\*]*?\b" + name + r"\s*\(", text, flags=re.M)
        assert m, name
        before = text[:m.start()].rstrip()
        lines = before.split("\n")
        while lines and lines[-1].lstrip().startswith(("#define", "typedef")):
            lines.pop()
        before = "\n".join(lines).rstrip()
        assert before.endswith("*/"), name
        comment = before[before.rfind("/*"):]
        assert len(comment) >= 40, (name, comment)
