"""The C-ABI library builds, loads and exports every symbol include/truss.h
declares.  No compute call: these run without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "truss.h")


@pytest.fixture(scope="module")
def pkt():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1707_02000_gb300 as pkt

    return pkt


def declared_functions():
    names = []
    for path in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if path.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", path)).read()
            names += re.findall(r"^TRUSS_API\s+[\w\s\*]+?\b(truss_\w+)\s*\(", txt, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("truss_build_csr", "truss_support", "truss_decompose", "truss_free", "truss_edge_list"):
        assert must in names


def test_library_exports_every_declared_symbol(pkt):
    lib = ctypes.CDLL(pkt.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(pkt.EXPORTS) == set(declared_functions())


def test_strerror_and_defaults_without_gpu(pkt):
    assert pkt.strerror(0) == "ok"
    assert "vertex id" in pkt.strerror(pkt.EBADGRAPH)
    assert pkt.strerror(12345) == "unknown status"
    o = pkt.default_opts()
    assert o.loop == pkt.LOOP_PERSISTENT and o.variant == pkt.VAR_AUTO and o.level_jump == 1
    assert ctypes.sizeof(pkt.Opts) == 80 and ctypes.sizeof(pkt.Stats) == 96


def test_null_arguments_are_rejected_without_gpu(pkt):
    lib = pkt.library()
    assert lib.truss_build_csr(None, None, 0, 0, 0, None, None) == pkt.EINVAL
    out = ctypes.c_void_p()
    assert lib.truss_build_csr(None, None, 5, 3, 0, None, ctypes.byref(out)) == pkt.EINVAL
    assert lib.truss_build_csr(None, None, -1, 3, 0, None, ctypes.byref(out)) == pkt.EINVAL
    m = ctypes.c_int64()
    assert lib.truss_num_edges(None, ctypes.byref(m)) == pkt.EINVAL
    assert lib.truss_decompose(None, None, None, None, None) == pkt.EINVAL
    assert lib.truss_support(None, None, None) == pkt.EINVAL


def test_no_oracle_in_product_path():
    """The package never imports the oracle and has no CPU fallback."""
    pkg = os.path.join(ROOT, "paper_1707_02000_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "truss_oracle" not in txt, f
