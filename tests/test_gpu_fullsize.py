"""Device results at the workloads' full sizes, in the launch configuration
bench.py times (degree-ordered CSR, persistent loop, default variants).

The exact oracle is too slow to run at these sizes inside a test, so each
result is checked by properties that hold at any size: the certificate of
oracle.certify (lower bound by the k-truss property, upper bound by the
returned peeling order; together they fix the trussness exactly), the
support against the oracle's own per-edge count, and the triangle count."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkt():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1707_02000_gb300 as pkt

    return pkt


def _run(pkt, g, loop):
    import torch

    src = torch.from_numpy(g.src).cuda()
    dst = torch.from_numpy(g.dst).cuda()
    G = pkt.build_csr(src, dst, g.n)
    step = torch.empty(G.m, dtype=torch.int32, device="cuda")
    tau, st = G.decompose(loop=loop, peel_step=step, stats=True)
    S = G.support()
    u, v = G.edge_list()
    out = (u.cpu().numpy(), v.cpu().numpy(), tau.cpu().numpy(), step.cpu().numpy(), S.cpu().numpy(), st)
    G.free()
    return out


@pytest.mark.parametrize("name", ["chunglu_n2^20_d20", "rgg2d_n2^21_d32"])
def test_full_size_certified(pkt, name):
    g = gg.workload(name)
    u, v, tau, step, S, st = _run(pkt, g, pkt.LOOP_PERSISTENT)
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    assert np.array_equal(u, eu) and np.array_equal(v, ev)
    bad, first = oracle.certify(g.n, eu, ev, tau, step)
    assert bad == 0, f"{bad} edges violate the certificate (first: {first})"
    assert np.all(tau <= S + 2)
    assert st["triangles"] * 3 == int(S.astype(np.int64).sum())


def test_rmat10_exact_in_every_form(pkt):
    g = gg.workload("rmat10_ef8")
    eu, ev, want = oracle.truss_of_edges(g.n, g.src, g.dst)
    for loop in (pkt.LOOP_PLAIN, pkt.LOOP_PERSISTENT):
        u, v, tau, step, S, st = _run(pkt, g, loop)
        assert np.array_equal(tau, want)
