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
    assert o.compact == -1 and o.max_level == 0 and not o.h_level_edges and not o.h_level_ns
    assert ctypes.sizeof(pkt.Opts) == 104 and ctypes.sizeof(pkt.Stats) == 128


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
    assert lib.truss_support_ros(None, None, None) == pkt.EINVAL
    sw, up = ctypes.c_int64(), ctypes.c_int64()
    assert lib.truss_decompose_local(None, None, 0, ctypes.byref(sw), ctypes.byref(up), None) == pkt.EINVAL
    assert lib.truss_pool_keep(-1) == pkt.EINVAL


def test_no_oracle_in_product_path():
    """The package never imports the oracle and has no CPU fallback."""
    pkg = os.path.join(ROOT, "paper_1707_02000_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "truss_oracle" not in txt, f


def _header_defines():
    out = {}
    txt = open(HEADER).read()
    for name, val in re.findall(r"^#define TRUSS_(\w+)\s+\(?(-?\d+)u?\)?", txt, flags=re.M):
        out[name] = int(val)
    out["NOALLOC_MAX_VERTICES"] = 1 << 22 if "(1 << 22)" in txt else None
    return out


def _struct_fields(tag):
    txt = open(HEADER).read()
    body = re.search(r"typedef struct " + tag + r"\s*\{(.*?)\}\s*" + tag + ";", txt, flags=re.S)
    assert body, tag
    fields = []
    for line in re.sub(r"/\*.*?\*/", "", body.group(1), flags=re.S).split(";"):
        m = re.search(r"(\w+)\s*(\[\s*\d+\s*\])?\s*$", line.strip())
        if m:
            fields.append(m.group(1))
    return fields


def test_binding_constants_match_the_header(pkt):
    """Every constant the binding mirrors has the header's value."""
    d = _header_defines()
    pairs = {"OK": pkt.OK, "EINVAL": pkt.EINVAL, "ENOMEM": pkt.ENOMEM, "ECUDA": pkt.ECUDA,
             "ETIMEOUT": pkt.ETIMEOUT, "EOVERFLOW": pkt.EOVERFLOW, "EBADGRAPH": pkt.EBADGRAPH,
             "EDEVICE": pkt.EDEVICE, "ENOTSUP": pkt.ENOTSUP, "ETOOBIG": pkt.ETOOBIG,
             "DEGREE_ORDER": pkt.DEGREE_ORDER, "OFFSETS64": pkt.OFFSETS64, "CORE_ORDER": pkt.CORE_ORDER,
             "LOOP_PLAIN": pkt.LOOP_PLAIN, "LOOP_PERSISTENT": pkt.LOOP_PERSISTENT,
             "LOOP_PERSISTENT_LAT": pkt.LOOP_PERSISTENT_LAT, "LOOP_PERSISTENT_OCC": pkt.LOOP_PERSISTENT_OCC,
             "LOOP_GRAPH": pkt.LOOP_GRAPH, "VAR_AUTO": pkt.VAR_AUTO, "VAR_THREAD": pkt.VAR_THREAD,
             "VAR_GROUP": pkt.VAR_GROUP, "VAR_WARP": pkt.VAR_WARP, "VAR_LEARNED": pkt.VAR_LEARNED,
             "SCHED_FEATURES": pkt.SCHED_FEATURES, "SCHED_VARIANTS": pkt.SCHED_VARIANTS,
             "SCHED_PARAMS": pkt.SCHED_PARAMS, "TUNE_CLASSES": pkt.TUNE_CLASSES,
             "NOALLOC_MAX_VERTICES": pkt.NOALLOC_MAX_VERTICES}
    wrong = {k: (d.get(k), v) for k, v in pairs.items() if d.get(k) != v}
    assert not wrong, wrong


def test_binding_structs_follow_the_header_field_order(pkt):
    """The ctypes structures list the header's fields in the header's order
    (a reordered field would shift every later one)."""
    assert [f for f, _ in pkt.Opts._fields_] == _struct_fields("truss_opts")
    assert [f for f, _ in pkt.Stats._fields_] == _struct_fields("truss_stats")
    assert list(pkt.TRACE_DTYPE.names) == _struct_fields("truss_sublevel_trace")


def test_header_is_plain_c_and_links(pkt, tmp_path):
    """A C99 program (no C++, no CUDA headers) includes truss.h, links
    libtruss.so and calls the entry points that need no GPU."""
    import shutil
    import subprocess

    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(
        '#include "truss.h"\n#include <stdio.h>\n'
        "int main(void) {\n"
        "    truss_opts o;\n"
        "    truss_default_opts(&o);\n"
        '    printf("%d %d %d %s\\n", o.loop, (int)sizeof(truss_opts), (int)sizeof(truss_stats),\n'
        "           truss_strerror(TRUSS_EINVAL));\n"
        "    return truss_build_csr(NULL, NULL, 0, 0, 0, NULL, NULL) == TRUSS_EINVAL ? 0 : 1;\n"
        "}\n")
    exe = tmp_path / "client"
    libdir = os.path.dirname(pkt.LIB_PATH)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                           os.path.join(ROOT, "include"), str(src), "-L", libdir, "-ltruss",
                           "-Wl,-rpath," + libdir, "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    assert out.stdout.split()[:3] == [str(pkt.LOOP_PERSISTENT), "104", "128"]
