"""truss_support_noalloc, the entry point for callers that cannot allocate
device memory (their framework's allocator owns it all, or they run under a
fixed memory budget), checked through the C ABI against the regular
truss_support on the same graphs, on two calls in a row (the second call
finds the first call's leftovers in the shared scratch array).

This file is collected last on purpose, so that a run stopping at the first
failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkt():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1707_02000_gb300 as pkt

    return pkt


def _graphs():
    k = 3000  # a wheel: the hub's upper row is long enough for the global-memory path
    wheel_src = np.concatenate([np.zeros(k), np.arange(1, k + 1)]).astype(np.int32)
    wheel_dst = np.concatenate([np.arange(1, k + 1), np.arange(1, k + 1) % k + 1]).astype(np.int32)
    return [("rmat10", gg.workload("rmat10_ef8")),
            ("chunglu", gg.chung_lu(20000, 2.1, 16.0, 2000.0, seed=21)),
            ("wheel", gg.EdgeList(k + 1, wheel_src, wheel_dst, "wheel"))]


@pytest.mark.parametrize("name,g", _graphs())
def test_noalloc_support_matches_truss_support(pkt, name, g):
    import torch

    lib = pkt.library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    G = pkt.build_csr(torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda(), g.n, degree_order=False)
    rowptr, col, eid, _, _ = G.csr()
    rowptr = rowptr.to(torch.int32).contiguous()
    want = G.support()
    for call in range(2):
        out = torch.full((max(G.m, 1),), -7, dtype=torch.int32, device="cuda")
        rc = lib.truss_support_noalloc(ctypes.c_void_p(rowptr.data_ptr()), ctypes.c_void_p(col.data_ptr()),
                                       ctypes.c_void_p(eid.data_ptr()), G.n, G.m, ctypes.c_void_p(out.data_ptr()),
                                       stream)
        assert rc == pkt.OK, pkt.strerror(rc)
        assert torch.equal(out[: G.m], want), f"call {call}"
    G.free()


def test_noalloc_rejects_sizes_beyond_its_scratch(pkt):
    import torch

    lib = pkt.library()
    buf = torch.zeros(4, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    rc = lib.truss_support_noalloc(p, p, p, pkt.NOALLOC_MAX_VERTICES + 1, 1, p, None)
    assert rc == pkt.ETOOBIG
    assert "capacity" in pkt.strerror(rc)
    assert lib.truss_support_noalloc(None, p, p, 5, 1, p, None) == pkt.EINVAL
