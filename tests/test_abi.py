"""The C-ABI library builds, loads and exports every declared symbol; host-side argument checks
return error codes without touching a GPU."""
import ctypes
import glob
import os

import numpy as np
import pytest

import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def atos():
    import paper_2112_00132_gb300 as pkg
    pkg.build()
    return pkg


def test_exports_every_declared_symbol(atos):
    lib = atos.lib()
    headers = glob.glob(os.path.join(ROOT, "include", "*.h"))
    assert headers
    names = set()
    for h in headers:
        names |= set(atos.header_functions(h))
    assert {"atos_bfs", "atos_pagerank", "atos_color", "atos_graph_create", "atos_queue_config"} <= names
    for name in sorted(names):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_status_strings(atos):
    assert atos.status_string(0) == "ok"
    for code in range(-9, 0):
        assert atos.status_string(code) not in ("", "unknown status")
    assert atos.status_string(-99) == "unknown status"
    assert "sm_103a" in atos.version()


def test_queue_config_presets(atos):
    d = atos.queue_config()
    assert (d.worker_size, d.fetch_size, d.strategy) == (256, 256, atos.PERSISTENT)
    w = atos.queue_config("persist-warp")
    assert (w.worker_size, w.fetch_size) == (32, 1)
    assert atos.queue_config("discrete-cta").strategy == atos.DISCRETE
    assert atos.queue_config("bsp").strategy == atos.BSP
    t = atos.queue_config("autotune")
    assert t.flags & atos.abi.FLAG_USE_TUNED and t.worker_size == d.worker_size
    with pytest.raises(atos.AtosError):
        atos.queue_config("no-such-preset")
    assert atos.lib().atos_queue_config(None, None) == atos.abi.ERR_INVALID_ARG


def test_csr_validate(atos):
    g = gg.rmat(8, seed=1)
    assert atos.csr_validate(g.row_ptr, g.col) == 0
    assert atos.csr_validate(g.row_ptr, g.col, check_symmetric=True) == 0
    bad = g.col.copy(); bad[3] = g.n
    assert atos.csr_validate(g.row_ptr, bad) == atos.abi.ERR_BAD_CSR
    bad = g.col.copy(); bad[3] = -1
    assert atos.csr_validate(g.row_ptr, bad) == atos.abi.ERR_BAD_CSR
    rp = g.row_ptr.copy(); rp[5], rp[6] = rp[6], rp[5] - 1
    assert atos.csr_validate(rp, g.col) == atos.abi.ERR_BAD_CSR
    rp = g.row_ptr.copy(); rp[-1] -= 1
    assert atos.csr_validate(rp, g.col) == atos.abi.ERR_BAD_CSR
    # a directed edge without its mirror
    assert atos.csr_validate(np.array([0, 1, 1]), np.array([1]), check_symmetric=True) == atos.abi.ERR_BAD_CSR
    assert atos.csr_validate(np.array([0, 1, 1]), np.array([1])) == 0
    assert atos.csr_validate(np.array([0]), np.array([], dtype=np.int32)) == 0  # empty graph


def test_null_and_range_arguments(atos):
    L = atos.lib()
    out = ctypes.c_void_p()
    assert L.atos_graph_create(None, None, 4, 0, 0, None, ctypes.byref(out)) == atos.abi.ERR_INVALID_ARG
    rp = np.array([0, 1, 2], dtype=np.int32)
    col = np.array([1, 0], dtype=np.int32)
    assert L.atos_graph_create(rp.ctypes.data, col.ctypes.data, 2, 2, 0, None, None) == atos.abi.ERR_INVALID_ARG
    assert L.atos_graph_create(rp.ctypes.data, col.ctypes.data, -1, 2, 0, None,
                               ctypes.byref(out)) == atos.abi.ERR_INVALID_ARG
    assert L.atos_graph_create(rp.ctypes.data, col.ctypes.data, 2, 2**31, 0, None,
                               ctypes.byref(out)) == atos.abi.ERR_INVALID_ARG
    # borrow without device pointers is rejected before any CUDA call
    assert L.atos_graph_create(rp.ctypes.data, col.ctypes.data, 2, 2, 2, None,
                               ctypes.byref(out)) == atos.abi.ERR_INVALID_ARG
    bad = np.array([0, 1, 3], dtype=np.int32)  # row_ptr[n] != nnz
    assert L.atos_graph_create(bad.ctypes.data, col.ctypes.data, 2, 2, 0, None,
                               ctypes.byref(out)) == atos.abi.ERR_BAD_CSR
    assert L.atos_bfs(None, None, 1, None, None, None, None) == atos.abi.ERR_INVALID_ARG
    assert L.atos_pagerank(None, 0.85, 1e-9, None, None, None, None) == atos.abi.ERR_INVALID_ARG
    assert L.atos_color(None, None, None, None, None, None) == atos.abi.ERR_INVALID_ARG
    assert L.atos_graph_destroy(None) == 0


def test_product_path_does_not_import_the_oracle():
    import subprocess
    import sys
    code = ("import sys, paper_2112_00132_gb300 as p; p.lib(); "
            "assert 'oracle' not in sys.modules, 'the product imported the oracle'")
    subprocess.check_call([sys.executable, "-c", code], cwd=ROOT)
    src = "\n".join(open(f).read() for f in glob.glob(os.path.join(ROOT, "paper_2112_00132_gb300", "**", "*.*"),
                                                       recursive=True) if f.endswith((".py", ".cu", ".cuh")))
    assert "import oracle" not in src and "oracle." not in src


def test_checked_library_exports_the_same_symbols(atos):
    """The bounds-checked variant (built with ATOS_CHECKED) exports every function the header
    declares, like the normal library (no GPU needed to load it)."""
    from paper_2112_00132_gb300.compile_lib import build
    lib = ctypes.CDLL(build(checked=True))
    for name in atos.header_functions():
        assert hasattr(lib, name), name
    lib.atos_status_string.restype = ctypes.c_char_p
    assert b"bounds" in lib.atos_status_string(-9)
