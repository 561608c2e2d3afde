"""Row compaction and the per-level distribution, CUDA path vs the CPU oracle.

Compaction drops the entries of processed edges from the rows between
levels (Algorithm 5 never uses a triangle with a processed edge), so the
trussness, the frontier of every sub-level and the sub-level each edge is
peeled in must be exactly the serial run's.  What changes is the walk: each
live edge's walk length becomes min(live d(u), live d(v)) at the last
compaction, which the trace reports and these tests recompute from the
oracle's own peeling order."""
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


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def host(t):
    return t.cpu().numpy()


def graphs():
    return [("rmat10", gg.workload("rmat10_ef8")),
            ("chunglu", gg.chung_lu(4000, 2.1, 16.0, 400.0, seed=11)),
            ("rgg", gg.rgg2d(4000, 24.0, seed=12)),
            # hubs of degree > 1024: their longer rows stay in the bitmaps
            ("chunglu_hubs", gg.chung_lu(20000, 2.1, 20.0, 5000.0, seed=13)),
            ("gnp", gg.small_random(60, 0.4, seed=14))]


LOOPS = ["plain", "persistent_lat", "persistent_occ"]


def _loop(pkt, name):
    return {"plain": pkt.LOOP_PLAIN, "persistent_lat": pkt.LOOP_PERSISTENT_LAT,
            "persistent_occ": pkt.LOOP_PERSISTENT_OCC, "graph": pkt.LOOP_GRAPH}[name]


def live_pct(held):
    """The library's trigger: compact once the live edges are at most this
    share (%) of the held ones."""
    return 80 if held >= 1 << 25 else 50


def expected_walks(n, eu, ev, step, olv, osz, min_held=0):
    """Per sub-level: (sum and max of the walk lengths, light edges) and the
    number of compactions and slots visited, when compaction runs before the
    Scan of a level once 100 (m - processed) <= live_pct(held) held (and
    held >= min_held).  Level 0 walks nothing (its edges lie in no triangle),
    so it adds nothing to the walked total."""
    m = eu.size
    deg = np.bincount(np.concatenate([eu, ev]), minlength=n)
    walk = np.minimum(deg[eu], deg[ev]).astype(np.int64)
    held, processed, count, slots = m, 0, 0, 0
    out = []
    for k in range(len(osz)):
        if k == 0 or olv[k] != olv[k - 1]:  # a Scan opens this level
            if processed > 0 and held >= min_held and 100 * (m - processed) <= live_pct(held) * held:
                live = step >= k
                ld = np.bincount(np.concatenate([eu[live], ev[live]]), minlength=n)
                walk = np.where(live, np.minimum(ld[eu], ld[ev]), walk)
                count += 1
                slots += 2 * held
                held = m - processed
        sel = step == k
        out.append((int(walk[sel].sum()), int(walk[sel].max()), int((walk[sel] <= 32).sum())))
        processed += int(osz[k])
    return out, count, slots


@pytest.mark.parametrize("loop", LOOPS)
@pytest.mark.parametrize("off64", [False, True])
@pytest.mark.parametrize("name,g", graphs())
def test_compaction_is_exact_and_walks_live_rows(pkt, name, g, loop, off64):
    import torch

    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n, offsets64=off64)
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    want, olv, osz, ostep = oracle.pkt_serial(g.n, eu, ev, return_steps=True)
    step = torch.empty(max(G.m, 1), dtype=torch.int32, device="cuda")
    tau, (lv, sz), tr, st = G.decompose(loop=_loop(pkt, loop), compact=1, record=True, trace=True, stats=True,
                                        peel_step=step)
    assert np.array_equal(host(tau), want)
    assert np.array_equal(host(step)[: G.m], ostep)
    assert np.array_equal(lv, olv) and np.array_equal(sz, osz)
    walks, count, slots = expected_walks(g.n, eu, ev, ostep, olv, osz)
    assert st["compactions"] == count and st["compacted_slots"] == slots
    if name != "gnp":  # sparse graphs peel most edges early: compaction runs
        assert count > 0
    assert [int(x) for x in tr["dsum"]] == [w[0] for w in walks]
    assert [int(x) for x in tr["dmax"]] == [w[1] for w in walks]
    assert [int(x) for x in tr["n_light"]] == [w[2] for w in walks]
    walked = sum(w[0] for w, l in zip(walks, olv) if l > 0)
    assert st["walked"] == walked <= st["dmin_sum"]
    if count > 0:
        assert st["walked"] < st["dmin_sum"]
    # the certificate accepts the result with its peeling order
    assert oracle.certify(g.n, eu, ev, host(tau), host(step)[: G.m])[0] == 0
    # compaction off: the static walk lengths, the same result
    tau0, st0 = G.decompose(loop=_loop(pkt, loop), compact=0, stats=True)
    assert np.array_equal(host(tau0), want)
    static_walk = sum(w[0] for w, l in zip(expected_walks(g.n, eu, ev, ostep, olv, osz, min_held=1 << 62)[0], olv)
                      if l > 0)
    assert st0["compactions"] == 0 and st0["walked"] == static_walk
    G.free()


@pytest.fixture(scope="module")
def big_sparse():
    """2^23 vertices, 3.4e7 random pairs plus 3000 dense communities of 12
    to 47 vertices: more than 2^25 edges (so a compaction tests the row
    slots against one live bit per edge instead of reading the support /
    stamp pairs), most of them peeled at level 0, the communities up to
    trussness 14.  Its int32 support counters (139 MB) would take more than
    half of L2 and 16-bit ones fit, so the support packs two counters a
    word."""
    rng = np.random.default_rng(5)
    n, k = 1 << 23, 34_000_000
    src = [rng.integers(0, n, k, dtype=np.int32)]
    dst = [rng.integers(0, n, k, dtype=np.int32)]
    for _ in range(3000):
        size = int(rng.integers(12, 48))
        verts = rng.choice(n, size, replace=False).astype(np.int32)
        iu, ju = np.triu_indices(size, 1)
        keep = rng.random(iu.size) < 0.6
        src.append(verts[iu[keep]])
        dst.append(verts[ju[keep]])
    src, dst = np.concatenate(src), np.concatenate(dst)
    eu, ev = oracle.canonical(n, src, dst)
    assert eu.size >= 1 << 25
    return n, src, dst, oracle.truss(n, eu, ev), oracle.support(n, eu, ev)


@pytest.mark.parametrize("loop", ["plain", "persistent_occ"])
@pytest.mark.parametrize("off64", [False, True])
def test_compaction_of_a_graph_beyond_2_25_edges(pkt, big_sparse, loop, off64):
    n, src, dst, want, S = big_sparse
    G = pkt.build_csr(dev(src), dev(dst), n, offsets64=off64)
    assert np.array_equal(host(G.support()), S)
    tau, st = G.decompose(loop=_loop(pkt, loop), stats=True)
    assert np.array_equal(host(tau), want)
    assert st["compactions"] > 0 and st["walked"] < st["dmin_sum"]
    tau0, st0 = G.decompose(loop=_loop(pkt, loop), compact=0, stats=True)
    assert np.array_equal(host(tau0), want) and st0["compactions"] == 0
    G.free()


@pytest.mark.parametrize("loop", LOOPS)
def test_repeated_runs_after_compaction(pkt, loop):
    """Compaction writes only its own buffers: later runs on the same graph,
    with or without it and in other loop forms, are exact."""
    g = gg.chung_lu(20000, 2.1, 20.0, 5000.0, seed=13)
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
    want = oracle.truss_of_edges(g.n, g.src, g.dst)[2]
    for k, c in enumerate((1, 1, 0, 1, -1)):
        tau = G.decompose(loop=_loop(pkt, loop) if k % 2 == 0 else pkt.LOOP_GRAPH, compact=c)
        assert np.array_equal(host(tau), want), (k, c)
    assert np.array_equal(host(G.support()), oracle.support(g.n, *oracle.canonical(g.n, g.src, g.dst)))
    G.free()


def test_automatic_compaction_threshold(pkt):
    """Automatic mode compacts graphs of at least TRUSS_COMPACT_MIN_EDGES
    edges, and only while the rows hold that many; smaller graphs never."""
    small = gg.workload("rmat10_ef8")
    G = pkt.build_csr(dev(small.src), dev(small.dst), small.n)
    _, st = G.decompose(stats=True)
    assert st["compactions"] == 0 and st["walked"] <= st["dmin_sum"]
    g = gg.chung_lu(60000, 2.1, 20.0, 3000.0, seed=15)
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
    assert G.m >= 65536
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    want, olv, osz, ostep = oracle.pkt_serial(g.n, eu, ev, return_steps=True)
    for loop in (pkt.LOOP_PLAIN, pkt.LOOP_PERSISTENT):
        tau, tr, st = G.decompose(loop=loop, trace=True, stats=True)
        assert np.array_equal(host(tau), want)
        walks, count, slots = expected_walks(g.n, eu, ev, ostep, olv, osz, min_held=65536)
        assert st["compactions"] == count > 0 and st["compacted_slots"] == slots
        assert [int(x) for x in tr["dsum"]] == [w[0] for w in walks]
    # the graph-driven loop does not compact
    tau, st = G.decompose(loop=pkt.LOOP_GRAPH, stats=True)
    assert np.array_equal(host(tau), want) and st["compactions"] == 0
    G.free()


@pytest.mark.parametrize("loop", ["plain", "persistent_lat", "persistent_occ", "graph"])
def test_level_distribution(pkt, loop):
    """Fig. 6: edges peeled per support level equal the oracle's trussness
    histogram (trussness l + 2 at level l); every level that peels edges has
    device time, the others none."""
    for name, g in graphs()[:4]:
        G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
        tau, (edges, ns), st = G.decompose(loop=_loop(pkt, loop), level_hist=True, stats=True)
        want = oracle.truss_of_edges(g.n, g.src, g.dst)[2]
        assert np.array_equal(host(tau), want)
        hist = np.bincount(want - 2)
        assert np.array_equal(edges, hist), name
        assert np.all(ns[hist > 0] > 0) and np.all(ns[hist == 0] == 0), name
        assert len(edges) == st["t_max"] - 1
        # a short capacity keeps the first levels only
        _, (e2, _) = G.decompose(loop=_loop(pkt, loop), level_hist=True, max_level=3)
        assert np.array_equal(e2, hist[:3])
        G.free()


def test_bad_options_are_rejected(pkt):
    g = gg.workload("rmat10_ef8")
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
    for kw in (dict(compact=2), dict(compact=-2)):
        with pytest.raises(pkt.TrussError) as ex:
            G.decompose(**kw)
        assert ex.value.status == pkt.EINVAL
    G.free()
