"""truss_support_noalloc, the entry point for callers that cannot allocate
device memory (their framework's allocator owns it all, or they run under a
fixed memory budget), checked through the C ABI against the CPU oracle's
support on the same graphs (and the regular truss_support beside it), on two
calls in a row (the second call finds the first call's leftovers in the
shared scratch array and must leave the free device memory unchanged).

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

    import oracle

    lib = pkt.library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # without relabelling the library's edge ids are the canonical ones
    G = pkt.build_csr(torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda(), g.n, degree_order=False)
    rowptr, col, eid, _, _ = G.csr()
    rowptr = rowptr.to(torch.int32).contiguous()
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    want = torch.from_numpy(oracle.support(g.n, eu, ev)).cuda()
    assert torch.equal(G.support(), want)  # the regular entry point agrees with the oracle
    outs = [torch.full((max(G.m, 1),), -7, dtype=torch.int32, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    for call, out in enumerate(outs):
        free_before = torch.cuda.mem_get_info()[0]
        rc = lib.truss_support_noalloc(ctypes.c_void_p(rowptr.data_ptr()), ctypes.c_void_p(col.data_ptr()),
                                       ctypes.c_void_p(eid.data_ptr()), G.n, G.m, ctypes.c_void_p(out.data_ptr()),
                                       stream)
        assert rc == pkt.OK, pkt.strerror(rc)
        torch.cuda.synchronize()
        if call == 1:
            # the first call may load the library's device code (and with it
            # the static scratch array); the second must take no memory
            assert torch.cuda.mem_get_info()[0] == free_before
        assert torch.equal(out[: G.m], want), f"call {call}"
    G.free()


def test_noalloc_rejects_bad_row_offsets_before_reading_through_them(pkt):
    import torch

    lib = pkt.library()
    n, m = 4, 3  # a path 0-1-2-3: rows {1}, {0,2}, {1,3}, {2}
    good = [0, 1, 3, 5, 6]
    col = torch.tensor([1, 0, 2, 1, 3, 2], dtype=torch.int32, device="cuda")
    eid = torch.tensor([0, 0, 1, 1, 2, 2], dtype=torch.int32, device="cuda")
    out = torch.zeros(m, dtype=torch.int32, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    for rows, want in ((good, pkt.OK), ([1, 1, 3, 5, 6], pkt.EBADGRAPH), ([0, 3, 1, 5, 6], pkt.EBADGRAPH),
                       ([0, 1, 3, 5, 7], pkt.EBADGRAPH), ([0, 1, 3, 5, 1 << 30], pkt.EBADGRAPH)):
        rp = torch.tensor(rows, dtype=torch.int32, device="cuda")
        out.fill_(-7)
        assert lib.truss_support_noalloc(P(rp), P(col), P(eid), n, m, P(out), None) == want, rows
        if want == pkt.OK:
            assert out.tolist() == [0, 0, 0]
        else:
            assert out.tolist() == [-7, -7, -7]  # nothing was written


def test_noalloc_rejects_sizes_beyond_its_scratch(pkt):
    import torch

    lib = pkt.library()
    buf = torch.zeros(4, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    rc = lib.truss_support_noalloc(p, p, p, pkt.NOALLOC_MAX_VERTICES + 1, 1, p, None)
    assert rc == pkt.ETOOBIG
    assert "capacity" in pkt.strerror(rc)
    assert lib.truss_support_noalloc(None, p, p, 5, 1, p, None) == pkt.EINVAL
    # 2m must fit the int32 row offsets
    assert lib.truss_support_noalloc(p, p, p, 4, 1 << 30, p, None) == pkt.EOVERFLOW
    # a call with no vertices and no edges does only the one-time set-up
    assert lib.truss_support_noalloc(p, p, p, 0, 0, p, None) == pkt.OK
    assert lib.truss_support_noalloc(p, p, p, 0, 1, p, None) == pkt.EBADGRAPH
