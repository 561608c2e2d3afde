"""Pins for the CPU oracle against what the paper and the mathematics fix:
brute force from the definition (§II), closed forms, the figure captions
(Figs. 1-3), and invariants.  None of these calls the CUDA path."""
import itertools
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from brute import (_pick, brute_truss, canon_edges, coreness, sparse_truss, support_dense,
                   triangle_count)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _edges(pairs):
    pairs = list(pairs)
    return (np.array([a for a, _ in pairs], np.int32), np.array([b for _, b in pairs], np.int32))


# ---------------------------------------------------------------- canonical

def test_canonical_matches_set_definition():
    g = gg.rmat(8, 8, seed=11)
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    ru, rv = canon_edges(g.n, g.src, g.dst)
    assert np.array_equal(eu, ru) and np.array_equal(ev, rv)
    assert np.all(eu < ev)


def test_canonical_rejects_bad_ids():
    with pytest.raises(ValueError):
        oracle.canonical(4, np.array([0, 5], np.int32), np.array([1, 2], np.int32))
    with pytest.raises(ValueError):
        oracle.canonical(4, np.array([-1], np.int32), np.array([1], np.int32))


def test_empty_and_loop_only_graphs():
    eu, ev = oracle.canonical(3, np.array([0, 1, 1], np.int32), np.array([0, 1, 1], np.int32))
    assert eu.size == 0
    assert oracle.truss(3, eu, ev).size == 0
    tau, lv, sz = oracle.pkt_serial(3, eu, ev)
    assert tau.size == 0 and lv.size == 0


# ------------------------------------------------ brute force, every graph

def test_all_graphs_on_six_vertices():
    """Every labelled simple graph on 6 vertices (2^15 of them, which include
    every graph on fewer vertices plus isolated ones): the oracle equals the
    definition, and so does the serial level-synchronous run."""
    pairs = list(itertools.combinations(range(6), 2))
    graphs = []
    for mask in range(1 << 15):
        sel = [pairs[i] for i in range(15) if mask >> i & 1]
        graphs.append(sel)

    class G:
        pass

    objs = []
    for sel in graphs:
        o = G()
        o.n = 6
        o.src, o.dst = _edges(sel) if sel else (np.zeros(0, np.int32), np.zeros(0, np.int32))
        objs.append(o)
    taus = oracle.truss_batch(objs)
    # trussness depends only on the isomorphism class; brute force each class
    # once via a canonical relabelling and compare every member
    memo = {}
    for sel, o, tau in zip(graphs, objs, taus):
        eu, ev = canon_edges(6, o.src, o.dst)
        key = tuple(zip(eu.tolist(), ev.tolist()))
        if key not in memo:
            memo[key] = brute_truss(eu, ev)
        assert np.array_equal(tau, memo[key]), key


def test_random_graphs_up_to_14_vertices():
    rng = np.random.default_rng(5)
    for t in range(300):
        n = int(rng.integers(3, 15))
        p = float(rng.uniform(0.15, 0.9))
        g = gg.small_random(n, p, seed=100 + t)
        eu, ev = oracle.canonical(n, g.src, g.dst)
        want = brute_truss(eu, ev)
        assert np.array_equal(oracle.truss(n, eu, ev), want)
        tau2, lv, sz = oracle.pkt_serial(n, eu, ev)
        assert np.array_equal(tau2, want)


def test_rmat_scale10_matches_sparse_definition():
    """The small R-MAT workload (scale 10, edge factor 8, seed 1) against the
    definition computed with sparse matrix products."""
    g = gg.workload("rmat10_ef8")
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    tau, S0 = oracle.truss(g.n, eu, ev, return_support=True)
    assert np.array_equal(tau, sparse_truss(g.n, eu, ev))
    assert np.array_equal(S0, support_dense(g.n, eu, ev))
    tau2, lv, sz = oracle.pkt_serial(g.n, eu, ev)
    assert np.array_equal(tau2, tau)


# ------------------------------------------------------------ closed forms

def test_complete_graphs():
    for n in range(2, 13):
        eu, ev = _edges(itertools.combinations(range(n), 2))
        assert np.all(oracle.truss(n, eu, ev) == n)
        assert np.all(oracle.support(n, eu, ev) == n - 2)


def test_triangle_free_graphs_have_trussness_two():
    rng = np.random.default_rng(1)
    # random trees
    for t in range(20):
        n = int(rng.integers(2, 200))
        par = [int(rng.integers(0, i)) for i in range(1, n)]
        eu, ev = oracle.canonical(n, np.arange(1, n, dtype=np.int32), np.array(par, np.int32))
        assert np.all(oracle.truss(n, eu, ev) == 2)
    # even and odd (> 3) cycles
    for n in range(4, 40):
        eu, ev = oracle.canonical(n, np.arange(n, dtype=np.int32), ((np.arange(n) + 1) % n).astype(np.int32))
        assert np.all(oracle.truss(n, eu, ev) == 2)
    # random bipartite graphs
    for t in range(20):
        a, b = int(rng.integers(1, 30)), int(rng.integers(1, 30))
        M = rng.random((a, b)) < 0.5
        i, j = np.nonzero(M)
        eu, ev = oracle.canonical(a + b, i.astype(np.int32), (j + a).astype(np.int32))
        assert np.all(oracle.truss(a + b, eu, ev) == 2)


def test_wheels_books_and_unions():
    for k in range(4, 30):  # wheel: hub 0, rim 1..k
        pairs = [(0, i) for i in range(1, k + 1)] + [(i, i % k + 1) for i in range(1, k + 1)]
        eu, ev = oracle.canonical(k + 1, *_edges(pairs))
        assert np.all(oracle.truss(k + 1, eu, ev) == 3)
    for k in range(1, 30):  # book K_{1,1,k}: spine {0,1}, pages 2..k+1
        pairs = [(0, 1)] + [(0, i) for i in range(2, k + 2)] + [(1, i) for i in range(2, k + 2)]
        eu, ev = oracle.canonical(k + 2, *_edges(pairs))
        assert np.all(oracle.truss(k + 2, eu, ev) == 3)
    # disjoint union: K5, K7, a path, a wheel -> elementwise
    parts = [(5, list(itertools.combinations(range(5), 2)), 5),
             (7, list(itertools.combinations(range(7), 2)), 7),
             (6, [(i, i + 1) for i in range(5)], 2),
             (7, [(0, i) for i in range(1, 7)] + [(i, i % 6 + 1) for i in range(1, 7)], 3)]
    pairs, want, off = [], {}, 0
    for n, ps, t in parts:
        for a, b in ps:
            pairs.append((a + off, b + off))
            want[(min(a, b) + off, max(a, b) + off)] = t
        off += n
    eu, ev = oracle.canonical(off, *_edges(pairs))
    tau = oracle.truss(off, eu, ev)
    assert all(tau[i] == want[(eu[i], ev[i])] for i in range(eu.size))


def test_clique_with_pendant_triangle():
    # K6 on 0..5 plus vertex 6 adjacent to 0 and 1: the triangle {0,1,6}
    # adds one to the support of {0,1} but the two new edges have support 1
    pairs = list(itertools.combinations(range(6), 2)) + [(0, 6), (1, 6)]
    eu, ev = oracle.canonical(7, *_edges(pairs))
    tau = oracle.truss(7, eu, ev)
    for i in range(eu.size):
        assert tau[i] == (3 if ev[i] == 6 else 6)


# ----------------------------------------------------------- figure pins

def _read_rows(name):
    rows, n = [], None
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line.startswith("# n "):
            n = int(line.split()[2])
        if not line or line.startswith("#"):
            continue
        rows.append(line)
    return n, rows


def test_fig1_caption_standin():
    n, rows = _read_rows("fig1_standin.txt")
    uv = np.array([[int(x) for x in r.split()] for r in rows])
    eu, ev = oracle.canonical(n, uv[:, 0].astype(np.int32), uv[:, 1].astype(np.int32))
    tau = oracle.truss(n, eu, ev)
    want = {(min(a, b), max(a, b)): t for a, b, t in uv}
    assert all(tau[i] == want[(eu[i], ev[i])] for i in range(eu.size))
    # caption: every vertex has coreness 3; two edges of trussness 2
    assert np.all(coreness(n, eu, ev) == 3)
    assert int((tau == 2).sum()) == 2
    # two 3-trusses: connected components of the edges with trussness >= 3
    import scipy.sparse as sp
    import scipy.sparse.csgraph as cg
    sel = tau >= 3
    A = sp.coo_matrix((np.ones(sel.sum()), (eu[sel], ev[sel])), shape=(n, n))
    ncomp, lab = cg.connected_components(A, directed=False)
    touched = np.unique(np.concatenate([eu[sel], ev[sel]]))
    assert np.unique(lab[touched]).size == 2


def test_fig2_diamond():
    n, rows = _read_rows("fig2_diamond.txt")
    uv = np.array([[int(x) for x in r.split()] for r in rows])
    eu, ev = oracle.canonical(n, uv[:, 0].astype(np.int32), uv[:, 1].astype(np.int32))
    assert eu.size == 5
    tau, S0 = oracle.truss(n, eu, ev, return_support=True)
    assert np.array_equal(S0, uv[:, 2]) and np.array_equal(tau, uv[:, 3])


def _fig3_cases():
    _, rows = _read_rows("fig3_states.txt")
    out = []
    for r in rows:
        f = [x.strip() for x in r.split(";")]
        ints = lambda s: [] if s == "-" else [int(x) for x in s.split()]
        out.append((int(f[0]), ints(f[1]), ints(f[2]), ints(f[3]), ints(f[4]), ints(f[5])))
    return out


@pytest.mark.parametrize("case", _fig3_cases())
def test_fig3_sublevel_states(case):
    l, S, proc, curr, S_after, nxt = case
    eu, ev = _edges([(0, 1), (0, 2), (1, 2)])
    S = np.array(S, np.int32)
    flags = np.array(proc, np.uint8) * oracle.PROCESSED
    got = oracle.sublevel(3, eu, ev, S, flags, np.array(curr, np.int32), l)
    assert S.tolist() == S_after
    assert got.tolist() == nxt
    for e in curr:
        assert flags[e] == oracle.PROCESSED
    for e in nxt:
        assert flags[e] & oracle.IN_CURR


# --------------------------------------------------------------- invariants

def _invariant_graphs():
    yield "rmat9", gg.rmat(9, 8, seed=3)
    yield "chunglu", gg.chung_lu(3000, 2.1, 12.0, 300.0, seed=9)
    yield "rgg", gg.rgg2d(3000, 16.0, seed=4)
    for s in range(3):
        yield f"gnp{s}", gg.small_random(60, 0.3, seed=20 + s)


@pytest.mark.parametrize("name,g", list(_invariant_graphs()))
def test_invariants(name, g):
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    tau, S0 = oracle.truss(g.n, eu, ev, return_support=True)
    # support: each triangle counted once on each of its edges
    if g.n <= 3000:
        assert int(S0.sum()) == 3 * triangle_count(g.n, eu, ev)
        assert np.array_equal(S0, support_dense(g.n, eu, ev))
    # initial support + 2 bounds trussness (§II, Algorithm 1 discussion)
    assert np.all(tau <= S0 + 2) and np.all(tau >= 2)
    # k-truss property and maximality for every k
    import scipy.sparse as sp
    for k in range(3, int(tau.max()) + 2):
        sel = np.nonzero(tau >= k)[0]
        if sel.size:
            A = sp.coo_matrix((np.ones(2 * sel.size), (np.concatenate([eu[sel], ev[sel]]),
                                                       np.concatenate([ev[sel], eu[sel]]))),
                              shape=(g.n, g.n)).tocsr()
            s = _pick((A @ A).tocsr(), eu[sel], ev[sel])
            assert np.all(s >= k - 2), k
    # trussness <= coreness + 1 (an edge in a k-truss has endpoints of
    # degree >= k-1 inside it)
    if g.n <= 3000:
        core = coreness(g.n, eu, ev)
        assert np.all(tau <= np.minimum(core[eu], core[ev]) + 1)
    # Algorithms 4/5 run serially reach the same trussness
    tau2, lv, sz = oracle.pkt_serial(g.n, eu, ev)
    assert np.array_equal(tau2, tau)
    assert int(sz.sum()) == eu.size
    assert np.all(np.diff(lv) >= 0)


def test_sublevel_frontiers_are_order_free():
    """The frontier sequence is a function of the state: the serial run
    reports the same sub-level sizes whatever the curr visit order.  Checked by
    re-running every sub-level with curr reversed on the same state."""
    g = gg.chung_lu(2000, 2.1, 14.0, 300.0, seed=5)
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    tau, lv, sz = oracle.pkt_serial(g.n, eu, ev)
    S = oracle.support(g.n, eu, ev).copy()
    flags = np.zeros(eu.size, np.uint8)
    got_sizes, todo, l = [], eu.size, 0
    while todo > 0:
        curr = np.nonzero((S == l) & (flags & oracle.PROCESSED == 0))[0].astype(np.int32)
        while curr.size:
            got_sizes.append(curr.size)
            todo -= curr.size
            curr = oracle.sublevel(g.n, eu, ev, S, flags, curr[::-1].copy(), l)
        l += 1
    assert got_sizes == sz.tolist()
    assert np.array_equal(S + 2, tau)


def test_batch_matches_single():
    gs = gg.chung_lu_batch(24, seed0=1000)
    taus = oracle.truss_batch(gs, nthreads=4)
    for g, t in zip(gs, taus):
        eu, ev, tau = oracle.truss_of_edges(g.n, g.src, g.dst)
        assert np.array_equal(t, tau)


# ------------------------------------------------------------ certificate

def test_certificate_accepts_the_exact_answer():
    for name, g in list(_invariant_graphs()) + [("rmat10", gg.workload("rmat10_ef8"))]:
        eu, ev = oracle.canonical(g.n, g.src, g.dst)
        tau, lv, sz, step = oracle.pkt_serial(g.n, eu, ev, return_steps=True)
        bad, first = oracle.certify(g.n, eu, ev, tau, step, nthreads=4)
        assert bad == 0 and first == -1, name


def test_certificate_rejects_wrong_answers():
    """Raising or lowering one edge's claim, or breaking the order, must be
    caught (each pin of the certificate has a planted mistake here)."""
    g = gg.rmat(9, 8, seed=3)
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    tau, lv, sz, step = oracle.pkt_serial(g.n, eu, ev, return_steps=True)
    rng = np.random.default_rng(0)
    tri = np.nonzero(tau > 2)[0]
    for e in rng.choice(tri, 20, replace=False):
        for d in (-1, 1):
            t2 = tau.copy()
            t2[e] += d
            assert oracle.certify(g.n, eu, ev, t2, step)[0] > 0
    # uniform shift of every claim
    assert oracle.certify(g.n, eu, ev, tau + 1, step)[0] > 0
    # an order that puts a high-trussness edge first
    s2 = step.copy()
    s2[np.argmax(tau)] = step.min()
    assert oracle.certify(g.n, eu, ev, tau, s2)[0] > 0
    # all claims 2 (a valid lower bound, but no valid order)
    assert oracle.certify(g.n, eu, ev, np.full_like(tau, 2), step)[0] > 0


def test_sampled_certificate():
    """The sampled certificate agrees with the full one: it accepts the exact
    answer for any sample, and flags a perturbed edge whenever that edge is
    sampled (and an order violation whatever the sample)."""
    g = gg.chung_lu(3000, 2.1, 14.0, 300.0, seed=8)
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    tau, lv, sz, step = oracle.pkt_serial(g.n, eu, ev, return_steps=True)
    rng = np.random.default_rng(3)
    sample = rng.choice(eu.size, 500, replace=False)
    assert oracle.certify_sample(g.n, eu, ev, tau, step, sample) == (0, -1)
    assert oracle.certify_sample(g.n, eu, ev, tau, step, np.arange(eu.size))[0] == 0
    for e in sample[:20]:
        for d in (-1, 1):
            t2 = tau.copy()
            t2[e] += d
            if t2[e] < 2:
                continue
            bad, first = oracle.certify_sample(g.n, eu, ev, t2, step, sample)
            assert bad > 0
    s2 = step.copy()
    s2[np.argmax(tau)] = 0
    assert oracle.certify_sample(g.n, eu, ev, tau, s2, sample[:10])[0] > 0


# ---------------------------------------------------------- k-truss listing

def _components_by_scipy(n, eu, ev, tau, k):
    import scipy.sparse as sp
    import scipy.sparse.csgraph as cg

    sel = tau >= k
    A = sp.coo_matrix((np.ones(int(sel.sum())), (eu[sel], ev[sel])), shape=(n, n))
    _, lab = cg.connected_components(A, directed=False)
    # label a component by its smallest vertex (vertices on selected edges)
    first = {}
    for v in np.unique(np.concatenate([eu[sel], ev[sel]])).tolist():
        first.setdefault(int(lab[v]), v)
    comp = np.full(eu.size, -1, np.int32)
    comp[sel] = [first[int(lab[u])] for u in eu[sel].tolist()]
    return comp, len(first)


def test_ktruss_components_match_connected_components():
    """The oracle's k-truss components equal scipy's connected components of
    the edges of trussness >= k, for every k of several graphs."""
    graphs = [gg.workload("rmat10_ef8"), gg.chung_lu(3000, 2.1, 14.0, 300.0, seed=31),
              gg.small_random(30, 0.25, seed=32), gg.rgg2d(2000, 10.0, seed=33)]
    for g in graphs:
        eu, ev, tau = oracle.truss_of_edges(g.n, g.src, g.dst)
        for k in range(2, int(tau.max()) + 2):
            got, nc = oracle.ktruss_components(g.n, eu, ev, tau, k)
            want, wnc = _components_by_scipy(g.n, eu, ev, tau, k)
            assert np.array_equal(got, want), (g.name, k)
            assert nc == wnc, (g.name, k)


def test_ktruss_components_closed_forms():
    """A disjoint K4 (vertices 0-3), K5 (10-14) and a path: the 3-trusses are
    the two cliques, the 4-trusses too, the only 5-truss is K5."""
    import itertools

    pairs = list(itertools.combinations(range(4), 2)) + list(itertools.combinations(range(10, 15), 2))
    pairs += [(20, 21), (21, 22), (3, 20)]
    n = 23
    src = np.array([a for a, _ in pairs], np.int32)
    dst = np.array([b for _, b in pairs], np.int32)
    eu, ev, tau = oracle.truss_of_edges(n, src, dst)
    in_k4 = (eu < 4) & (ev < 4)
    in_k5 = (eu >= 10) & (ev < 15)
    for k, labels, ncomp in ((3, {0, 10}, 2), (4, {0, 10}, 2), (5, {10}, 1), (6, set(), 0)):
        comp, nc = oracle.ktruss_components(n, eu, ev, tau, k)
        assert nc == ncomp and set(comp[comp >= 0].tolist()) == labels, k
        assert np.all(comp[in_k4] == (0 if k <= 4 else -1))
        assert np.all(comp[in_k5] == (10 if k <= 5 else -1))
        assert np.all(comp[~in_k4 & ~in_k5] == -1)
    comp, nc = oracle.ktruss_components(n, eu, ev, tau, 2)  # k = 2: the graph's components
    assert nc == 2 and set(comp.tolist()) == {0, 10}


def test_fig1_two_3_trusses_by_the_oracle():
    n, rows = _read_rows("fig1_standin.txt")
    uv = np.array([[int(x) for x in r.split()] for r in rows])
    eu, ev = oracle.canonical(n, uv[:, 0].astype(np.int32), uv[:, 1].astype(np.int32))
    tau = oracle.truss(n, eu, ev)
    _, nc = oracle.ktruss_components(n, eu, ev, tau, 3)
    assert nc == 2
