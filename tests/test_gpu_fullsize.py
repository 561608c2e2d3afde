"""Device results at the workloads' full sizes, in the launch configuration
bench.py times (degree-ordered CSR, persistent loop, default variants).

The exact oracle is too slow to run at these sizes inside a test, so each
result is checked by properties that hold at any size: the certificate of
oracle.certify (lower bound by the k-truss property, upper bound by the
returned peeling order; together they fix the trussness exactly), the
support against the oracle's own per-edge count, and the triangle count.
The R-MAT scale-24 result is checked by the edge list over every edge, the
certificate's order condition over every edge and its per-edge conditions
on a sample; where tests/golden/ holds digests of the oracle's own result
(a run of several hours on one core), it is compared over every edge."""
import hashlib
import os

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


def _run(pkt, g, loop, locality=False):
    import torch

    src = torch.from_numpy(g.src).cuda()
    dst = torch.from_numpy(g.dst).cuda()
    G = pkt.build_csr(src, dst, g.n, locality_order=locality)
    step = torch.empty(G.m, dtype=torch.int32, device="cuda")
    tau, st = G.decompose(loop=loop, peel_step=step, stats=True)
    S = G.support()
    u, v = G.edge_list()
    out = (u.cpu().numpy(), v.cpu().numpy(), tau.cpu().numpy(), step.cpu().numpy(), S.cpu().numpy(), st)
    G.free()
    return out


@pytest.mark.parametrize("name,locality", [("chunglu_n2^20_d20", False), ("rgg2d_n2^21_d32", False),
                                           ("rgg2d_n2^21_d32", True)])
def test_full_size_certified(pkt, name, locality):
    """Certified over every edge in the timed launch configuration, and for
    the geometric workload also in the reverse Cuthill-McKee order."""
    g = gg.workload(name)
    u, v, tau, step, S, st = _run(pkt, g, pkt.LOOP_PERSISTENT, locality)
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


def _golden_rmat24():
    path = os.path.join(os.path.dirname(__file__), "golden", "rmat24_ef16_truss.txt")
    if not os.path.exists(path):
        pytest.skip("tests/golden/rmat24_ef16_truss.txt is missing: run tests/golden/make_rmat24_digest.py")
    rec, hist = {}, {}
    for ln in open(path):
        f = ln.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "hist":
            hist[int(f[1])] = int(f[2])
        else:
            rec[f[0]] = f[1]
    return rec, hist


def _sha256_i32(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    return h.hexdigest()


def test_rmat24_sampled_certificate(pkt):
    """R-MAT scale 24, edge factor 16 (int64 row offsets), persistent loop as
    timed: the canonical edge list equals the oracle's over every edge; the
    trussness, with the peeling order the device reports, passes
    oracle.certify_sample -- the claims never decrease along the (sub-level,
    id) order over all edges, and each sampled edge of claimed trussness k
    lies in at least k - 2 triangles of edges claiming >= k and in at most
    k - 2 triangles of edges peeled after it.  The sample: 16,000 uniform
    edges and up to 8 edges of every trussness present, so that the deep
    levels of the dense core are covered too."""
    import torch

    g = gg.workload("rmat24_ef16")
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    src = torch.from_numpy(g.src).cuda()
    dst = torch.from_numpy(g.dst).cuda()
    G = pkt.build_csr(src, dst, g.n, offsets64=True)
    del src, dst
    assert G.m == eu.size
    u, v = G.edge_list()
    assert np.array_equal(u.cpu().numpy(), eu) and np.array_equal(v.cpu().numpy(), ev)
    del u, v
    step = torch.empty(G.m, dtype=torch.int32, device="cuda")
    tau, st = G.decompose(peel_step=step, stats=True)
    tau, step = tau.cpu().numpy(), step.cpu().numpy()
    G.free()
    assert st["compactions"] > 0 and int(tau.max()) == st["t_max"]
    rng = np.random.default_rng(24)
    picks = [rng.choice(eu.size, 16000, replace=False)]
    order = np.argsort(tau, kind="stable")
    levels, first = np.unique(tau[order], return_index=True)
    for i, k in enumerate(levels):
        end = first[i + 1] if i + 1 < levels.size else order.size
        ids = order[first[i]:end]
        picks.append(ids[rng.choice(ids.size, min(8, ids.size), replace=False)])
    sample = np.unique(np.concatenate(picks)).astype(np.int64)
    bad, first_bad = oracle.certify_sample(g.n, eu, ev, tau, step, sample)
    assert bad == 0, first_bad


def test_rmat24_matches_the_oracle_everywhere(pkt):
    """R-MAT scale 24, edge factor 16 (2^28 samples, int64 row offsets), in
    the persistent and the plain loop: the canonical edge list and the
    trussness of every one of its 260,381,693 edges hash to the digests of
    the oracle's own result (Algorithm 1, run once by
    tests/golden/make_rmat24_digest.py), and the per-level distribution
    equals the oracle's trussness histogram."""
    import torch

    rec, hist = _golden_rmat24()
    g = gg.workload("rmat24_ef16")
    src = torch.from_numpy(g.src).cuda()
    dst = torch.from_numpy(g.dst).cuda()
    G = pkt.build_csr(src, dst, g.n, offsets64=True)
    del src, dst
    assert G.m == int(rec["m"])
    u, v = G.edge_list()
    assert _sha256_i32(u.cpu().numpy(), v.cpu().numpy()) == rec["edges_sha256"]
    del u, v
    want_hist = np.zeros(max(hist) - 1, np.int64)
    for k, c in hist.items():
        want_hist[k - 2] = c
    for loop in (pkt.LOOP_PERSISTENT, pkt.LOOP_PLAIN):
        tau, (edges, ns), st = G.decompose(loop=loop, level_hist=True, stats=True)
        assert _sha256_i32(tau.cpu().numpy()) == rec["truss_sha256"], loop
        assert st["t_max"] == int(rec["truss_max"])
        assert np.array_equal(edges, want_hist)
        # the rows were compacted and the walk shrank accordingly
        assert st["compactions"] > 0 and st["walked"] < st["dmin_sum"]
        del tau
    G.free()
