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


def test_batch_4096_graphs_exact(pkt):
    """The ragged batch at full size: 4096 Chung-Lu graphs (seeds 1000..5095,
    log-uniform sizes and mean degrees) in one decomposition, every graph
    bit-exact against the oracle (Algorithm 1 per graph on host threads)."""
    gs = gg.chung_lu_batch(4096, seed0=1000)
    got, st = pkt.decompose_batch(gs, stats=True)
    want = oracle.truss_batch(gs)
    assert st["m"] == sum(len(w) for w in want)
    flat_got = np.concatenate([t.cpu().numpy() for t in got])
    flat_want = np.concatenate(want)
    assert np.array_equal(flat_got, flat_want)


def test_rmat24_sampled_certificate(pkt):
    """R-MAT scale 24, edge factor 16 (2^28 samples, int64 row offsets):
    the edge list is compared in full with the oracle's canonicalisation,
    the peeling order is checked over all edges, and the per-edge certificate
    conditions for 20,000 uniformly sampled edges plus the 500 edges of
    highest trussness and a sample of the last sub-level."""
    import torch

    g = gg.workload("rmat24_ef16")
    src = torch.from_numpy(g.src).cuda()
    dst = torch.from_numpy(g.dst).cuda()
    G = pkt.build_csr(src, dst, g.n, offsets64=True)
    del src, dst
    step = torch.empty(G.m, dtype=torch.int32, device="cuda")
    tau, st = G.decompose(loop=pkt.LOOP_PERSISTENT, peel_step=step, stats=True)
    # the walk holds over 2^34 shorter-row entries: the 6-blocks-per-SM form
    assert st["dmin_sum"] >= 1 << 34 and st["blocks_per_sm"] == 6
    tau = tau.cpu().numpy()
    step = step.cpu().numpy()
    u, v = G.edge_list()
    u, v = u.cpu().numpy(), v.cpu().numpy()
    G.free()
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    assert np.array_equal(u, eu) and np.array_equal(v, ev)
    rng = np.random.default_rng(24)
    top = np.argsort(tau)[-500:]
    last = np.nonzero(step == step.max())[0]
    sample = np.unique(np.concatenate([rng.choice(eu.size, 20000, replace=False), top,
                                       rng.choice(last, min(200, last.size), replace=False)]))
    bad, first = oracle.certify_sample(g.n, eu, ev, tau, step, sample)
    assert bad == 0, f"{bad} violations (first edge {first})"
