"""The C ABI on the host (no GPU needed): the libraries build and load, every
function declared in include/*.h is exported, and the ctypes mirrors of the
argument structs have the C layout."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(sdp_\w+)\s*\(", re.M)


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        src = re.sub(r"typedef\s+struct[^;]*?\}\s*\w+\s*;", "", src, flags=re.S)
        names |= set(DECL.findall(src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_05179_gb300 import api
    return ctypes.CDLL(api.lib_path())


def test_header_declares_the_operators():
    d = declared()
    for must in ("sdp_split_eval", "sdp_split_backward", "sdp_reinsert_eval",
                 "sdp_split_plan_create", "sdp_plan_run", "sdp_plan_autotune",
                 "sdp_split_count_arcs", "sdp_device_status", "sdp_saa_search_create",
                 "sdp_saa_search_run", "sdp_saa_search_state", "sdp_saa_search_destroy"):
        assert must in d


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts(lib):
    from paper_2602_05179_gb300 import api
    lib.sdp_split_args_size.restype = ctypes.c_size_t
    lib.sdp_reinsert_args_size.restype = ctypes.c_size_t
    assert lib.sdp_split_args_size() == ctypes.sizeof(api.SplitArgs)
    assert lib.sdp_reinsert_args_size() == ctypes.sizeof(api.ReinsertArgs)
    lib.sdp_saa_search_desc_size.restype = ctypes.c_size_t
    assert lib.sdp_saa_search_desc_size() == ctypes.sizeof(api.SaaSearchDesc)
    lib.sdp_version.restype = ctypes.c_int
    assert lib.sdp_version() == 1


def test_search_argument_checks_on_the_host(lib):
    """sdp_saa_search_create rejects bad descriptors before touching a
    device; host pointers are not device pointers."""
    from paper_2602_05179_gb300 import api
    lib.sdp_saa_search_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.sdp_saa_search_create.restype = ctypes.c_int
    h = ctypes.c_void_p()
    assert lib.sdp_saa_search_create(None, ctypes.byref(h)) == -1
    buf = (ctypes.c_int32 * 64)()

    def desc(**kw):
        d = api.SaaSearchDesc()
        d.n, d.Q, d.S, d.B, d.moves, d.seed = 10, 30, 4, 8, 7, 1
        d.coords = d.demands = d.tour0 = ctypes.addressof(buf)
        for k, v in kw.items():
            setattr(d, k, v)
        return d
    for kw, code in ((dict(n=1), -5), (dict(n=4096), -5), (dict(B=0), -1), (dict(S=0), -1),
                     (dict(moves=0), -1), (dict(moves=8), -1), ({}, -1)):
        assert lib.sdp_saa_search_create(ctypes.byref(desc(**kw)), ctypes.byref(h)) == code, kw
        assert not h.value
    lib.sdp_saa_search_run.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
    lib.sdp_saa_search_run.restype = ctypes.c_int
    assert lib.sdp_saa_search_run(None, 1, None, None, None) == -1
    lib.sdp_saa_search_destroy.argtypes = [ctypes.c_void_p]
    lib.sdp_saa_search_destroy(None)


def test_workspace_query_is_host_only(lib):
    from paper_2602_05179_gb300 import api
    a = api.SplitArgs()
    a.n, a.Q, a.S, a.algo = 500, 200, 1000, 2
    lib.sdp_split_workspace_bytes.restype = ctypes.c_size_t
    lib.sdp_split_workspace_bytes.argtypes = [ctypes.c_void_p]
    w = lib.sdp_split_workspace_bytes(ctypes.byref(a))
    # tour records + fallback list + fallback scratch, all bounded
    assert 500 * 16 + 1000 * 4 < w < 64 << 20


def test_generator_library_exports(lib):
    g = ctypes.CDLL(os.path.join(ROOT, "paper_2602_05179_gb300", "libsdpgen.so"))
    assert hasattr(g, "sdpgen_uniform_int") and hasattr(g, "sdpgen_poisson_clip")


def test_product_path_has_no_oracle_import():
    """The CUDA path and the oracle share no code and neither imports the
    other."""
    pkg = os.path.join(ROOT, "paper_2602_05179_gb300")
    files = [f for f in glob.glob(os.path.join(pkg, "**", "*"), recursive=True)
             if f.endswith((".py", ".cu", ".cuh")) and "_build" not in f]
    for f in files:
        src = open(f).read()
        assert "import oracle" not in src and "from oracle" not in src, f
        assert "sdp_oracle" not in src, f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if f.endswith((".py", ".c")):
            src = open(f).read()
            assert "import paper_2602_05179_gb300" not in src, f
            assert "from paper_2602_05179_gb300" not in src, f
            assert "sdp.h" not in src and "StepRec" not in src, f


def test_product_path_raises_without_its_library(monkeypatch, tmp_path):
    """No CPU path: with libsdp.so absent every operator call raises before
    computing anything."""
    import torch
    from paper_2602_05179_gb300 import api
    monkeypatch.setattr(api, "_LIB_PATH", str(tmp_path / "libsdp.so"))
    monkeypatch.setattr(api, "_lib", None)
    tour = torch.arange(1, 6, dtype=torch.int32)
    q = torch.ones((4, 5), dtype=torch.int32)
    xy = torch.zeros((6, 2), dtype=torch.float32)
    with pytest.raises(RuntimeError, match="missing"):
        api.split_eval(tour, 10, q, coords=xy)
    with pytest.raises(RuntimeError, match="missing"):
        api.reinsert_eval(3, 10, 5, 1.0, 2.0, 0.0, torch.ones(3), torch.ones((4, 3),
                          dtype=torch.int32))
    with pytest.raises(RuntimeError, match="missing"):
        api.status()


def test_product_path_refuses_host_tensors(lib):
    """With the library loaded, tensors in ordinary host memory are refused
    (only device memory, or pinned host demands read by the kernels, is
    accepted): nothing falls back to a CPU computation."""
    import torch
    from paper_2602_05179_gb300 import api
    tour = torch.arange(1, 6, dtype=torch.int32)
    q = torch.ones((4, 5), dtype=torch.int32)
    xy = torch.zeros((6, 2), dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA tensor"):
        api.split_eval(tour, 10, q, coords=xy)
    with pytest.raises(ValueError, match="CUDA tensor"):
        api.reinsert_eval(3, 10, 5, 1.0, 2.0, 0.0, torch.ones(3), torch.ones((4, 3),
                          dtype=torch.int32))
