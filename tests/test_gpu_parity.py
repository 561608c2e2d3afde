"""CUDA path vs the CPU oracle, element by element (bit-exact: every output is
an integer).  All calls go through the C ABI (libtruss.so) via the binding."""
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


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


def small_graphs():
    out = [("rmat10", gg.workload("rmat10_ef8")),
           ("rmat8_s7", gg.rmat(8, 16, seed=7)),
           ("chunglu", gg.chung_lu(4000, 2.1, 16.0, 400.0, seed=11)),
           ("rgg", gg.rgg2d(4000, 24.0, seed=12))]
    for s in range(4):
        out.append((f"gnp{s}", gg.small_random(40 + 10 * s, 0.35, seed=300 + s)))
    return out


SMALL = small_graphs()


def _flags(relabel, off64):
    return dict(degree_order=relabel, offsets64=off64)


# ------------------------------------------------------------------ build

def test_fig2_csr_layout(pkt):
    """Fig. 2: the augmented CSR of the n = 4, m = 5 graph, built without
    relabelling, matches the layout derived by hand in the fixture."""
    lines = open(os.path.join(GOLD, "fig2_diamond.txt")).read().splitlines()
    want = {}
    for ln in lines:
        for key in ("Es", "N", "Eid"):
            if ln.startswith(f"#   {key} ") and "=" in ln:
                want[key] = [int(x) for x in ln.split("=")[1].replace("|", " ").split()]
        if ln.startswith("#   Eo"):
            want["Eo"] = [int(x) for x in ln.split("=")[1].split()]
    rows = [ln.split() for ln in lines if ln and not ln.startswith("#")]
    src = np.array([int(r[0]) for r in rows], np.int32)
    dst = np.array([int(r[1]) for r in rows], np.int32)
    G = pkt.build_csr(dev(src), dev(dst), 4, degree_order=False)
    rp, col, eid, eo, order = G.csr()
    assert host(rp).tolist() == want["Es"]
    assert host(col).tolist() == want["N"]
    assert host(eid).tolist() == want["Eid"]
    assert host(eo).tolist() == want["Eo"]
    assert host(order).tolist() == [0, 1, 2, 3]
    assert host(G.support()).tolist() == [int(r[2]) for r in rows]
    assert host(G.decompose()).tolist() == [int(r[3]) for r in rows]


@pytest.mark.parametrize("relabel,off64", [(True, False), (False, False), (True, True)])
@pytest.mark.parametrize("name,g", SMALL)
def test_edge_list_and_support(pkt, name, g, relabel, off64):
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n, **_flags(relabel, off64))
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    u, v = G.edge_list()
    assert G.m == eu.size
    assert np.array_equal(host(u), eu) and np.array_equal(host(v), ev)
    assert np.array_equal(host(G.support()), oracle.support(g.n, eu, ev))
    # the internal CSR is a valid sorted adjacency with consistent edge ids
    rp, col, eid, eo, order = (host(x) for x in G.csr())
    assert rp[0] == 0 and rp[-1] == 2 * eu.size
    lab = order  # internal vertex -> input label
    for x in range(0, g.n, max(1, g.n // 50)):
        row = col[rp[x]:rp[x + 1]]
        assert np.all(np.diff(row) > 0)
        assert eo[x] == rp[x] + np.searchsorted(row, x + 1)
        ids = eid[rp[x]:rp[x + 1]]
        a, b = lab[x], lab[row]
        assert np.array_equal(eu[ids], np.minimum(a, b)) and np.array_equal(ev[ids], np.maximum(a, b))


def _dense_core_graph(n, core, p, filler, seed):
    """A dense random core (``core`` vertices at random labels, pairs joined
    with probability ``p``) inside ``n`` vertices with ``filler`` random
    edges: core vertices get N+(u) longer than a warp's 256 entries."""
    rng = np.random.default_rng(seed)
    c = rng.choice(n, core, replace=False).astype(np.int32)
    iu, ju = np.triu_indices(core, 1)
    keep = rng.random(iu.size) < p
    src = np.concatenate([c[iu[keep]], rng.integers(0, n, filler, dtype=np.int32)])
    dst = np.concatenate([c[ju[keep]], rng.integers(0, n, filler, dtype=np.int32)])
    return src, dst


@pytest.fixture(scope="module")
def dense_core():
    n = 1 << 21
    src, dst = _dense_core_graph(n, 900, 0.6, 1 << 20, seed=77)
    eu, ev = oracle.canonical(n, src, dst)
    return n, src, dst, eu, ev, oracle.support(n, eu, ev), oracle.truss(n, eu, ev)


@pytest.mark.parametrize("relabel,off64", [(True, False), (False, False), (True, True)])
def test_support_block_kernel_instances(pkt, dense_core, relabel, off64):
    """Vertices with N+(u) longer than 256 entries go to the block-per-vertex
    support kernel: in degree order their label windows are short and N+(u)
    is probed in a shared-memory bitmap over the window; without relabelling
    the core sits at low labels of 2^21 (windows too wide for shared memory)
    and the kernel searches the staged N+(u).  Support and the triangle count
    against the oracle in both, and the support again once the peeling
    workspace (hub bitmaps, side switch) exists."""
    n, src, dst, eu, ev, S, T = dense_core
    G = pkt.build_csr(dev(src), dev(dst), n, **_flags(relabel, off64))
    assert int(np.bincount(np.concatenate([eu, ev]), minlength=n).max()) > 500
    assert np.array_equal(host(G.support()), S)
    assert G.triangle_count() == int(S.sum()) // 3
    tau = host(G.decompose())
    assert np.array_equal(host(G.support()), S)
    assert np.array_equal(tau, T)


# ------------------------------------------------------------ decomposition

# the persistent kernel in both register budgets (the automatic choice picks
# one of them per graph) and the graph-driven loop
LOOPS = ["plain", "persistent_lat", "persistent_occ", "graph"]
VARIANTS = ["auto", "thread", "group", "warp"]


def _loop(pkt, name):
    return {"plain": pkt.LOOP_PLAIN, "persistent": pkt.LOOP_PERSISTENT, "persistent_lat": pkt.LOOP_PERSISTENT_LAT,
            "persistent_occ": pkt.LOOP_PERSISTENT_OCC, "graph": pkt.LOOP_GRAPH}[name]


def _var(pkt, name):
    return {"auto": pkt.VAR_AUTO, "thread": pkt.VAR_THREAD, "group": pkt.VAR_GROUP, "warp": pkt.VAR_WARP}[name]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("loop", LOOPS)
@pytest.mark.parametrize("name,g", SMALL)
def test_decompose_matches_oracle(pkt, name, g, loop, variant):
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
    tau = G.decompose(loop=_loop(pkt, loop), variant=_var(pkt, variant))
    eu, ev, want = oracle.truss_of_edges(g.n, g.src, g.dst)
    assert np.array_equal(host(tau), want)


@pytest.mark.parametrize("loop", LOOPS)
@pytest.mark.parametrize("relabel,off64", [(True, False), (False, False), (False, True)])
def test_sublevel_frontiers_match_serial_run(pkt, loop, relabel, off64):
    """The frontier of every sub-level is a function of the state, so the
    device must produce exactly the serial run's (level, |curr|) sequence."""
    for name, g in SMALL[:4]:
        G = pkt.build_csr(dev(g.src), dev(g.dst), g.n, **_flags(relabel, off64))
        tau, (lv, sz) = G.decompose(loop=_loop(pkt, loop), record=True, level_jump=True)
        eu, ev = oracle.canonical(g.n, g.src, g.dst)
        want, olv, osz = oracle.pkt_serial(g.n, eu, ev)
        assert np.array_equal(host(tau), want), name
        assert np.array_equal(lv, olv) and np.array_equal(sz, osz), name


def test_level_jump_off_gives_same_result(pkt):
    g = gg.rgg2d(3000, 24.0, seed=5)
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
    a = host(G.decompose(level_jump=False, loop=pkt.LOOP_PLAIN))
    b = host(G.decompose(level_jump=True, loop=pkt.LOOP_PERSISTENT))
    c = host(G.decompose(level_jump=False, loop=pkt.LOOP_PERSISTENT))
    assert np.array_equal(a, b) and np.array_equal(a, c)
    assert np.array_equal(a, oracle.truss_of_edges(g.n, g.src, g.dst)[2])


def test_all_graphs_on_five_vertices(pkt):
    """Every labelled graph on 5 vertices through the device path."""
    import itertools

    pairs = list(itertools.combinations(range(5), 2))
    for mask in range(1 << 10):
        sel = [pairs[i] for i in range(10) if mask >> i & 1]
        if not sel:
            continue
        src = np.array([a for a, _ in sel], np.int32)
        dst = np.array([b for _, b in sel], np.int32)
        G = pkt.build_csr(dev(src), dev(dst), 5)
        tau = host(G.decompose(loop=pkt.LOOP_PERSISTENT if mask & 1 else pkt.LOOP_PLAIN))
        assert np.array_equal(tau, oracle.truss_of_edges(5, src, dst)[2]), sel
        G.free()


def test_random_small_graphs(pkt):
    rng = np.random.default_rng(17)
    for t in range(60):
        n = int(rng.integers(3, 15))
        g = gg.small_random(n, float(rng.uniform(0.2, 0.9)), seed=900 + t)
        if g.n_in == 0:
            continue
        G = pkt.build_csr(dev(g.src), dev(g.dst), n, degree_order=bool(t & 1))
        tau = host(G.decompose(variant=int(rng.integers(-1, 3))))
        assert np.array_equal(tau, oracle.truss_of_edges(n, g.src, g.dst)[2])


def test_closed_forms(pkt):
    import itertools

    for n in (3, 8, 33, 70):  # K_n: every edge has trussness n
        pr = np.array(list(itertools.combinations(range(n), 2)), np.int32)
        G = pkt.build_csr(dev(pr[:, 0]), dev(pr[:, 1]), n)
        assert np.all(host(G.decompose()) == n)
        assert np.all(host(G.support()) == n - 2)
    # a long path and a big star: no triangles
    n = 5000
    G = pkt.build_csr(dev(np.arange(n - 1)), dev(np.arange(1, n)), n)
    assert np.all(host(G.decompose()) == 2)
    G = pkt.build_csr(dev(np.zeros(n - 1)), dev(np.arange(1, n)), n)
    assert np.all(host(G.decompose()) == 2)
    # wheel with a 3000-vertex rim: hub rows long enough to be split
    k = 3000
    src = np.concatenate([np.zeros(k), np.arange(1, k + 1)])
    dst = np.concatenate([np.arange(1, k + 1), np.arange(1, k + 1) % k + 1])
    G = pkt.build_csr(dev(src), dev(dst), k + 1)
    for loop in (pkt.LOOP_PLAIN, pkt.LOOP_PERSISTENT):
        assert np.all(host(G.decompose(loop=loop)) == 3)


def _fig3_cases():
    rows = [ln for ln in open(os.path.join(GOLD, "fig3_states.txt")).read().splitlines()
            if ln.strip() and not ln.startswith("#")]
    out = []
    for r in rows:
        f = [x.strip() for x in r.split(";")]
        ints = lambda s: [] if s == "-" else [int(x) for x in s.split()]
        out.append((int(f[0]), ints(f[1]), ints(f[2]), ints(f[3]), ints(f[4]), ints(f[5])))
    return out


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("case", _fig3_cases())
def test_fig3_sublevel_states(pkt, case, variant):
    """Fig. 3: one ProcessSubLevel on hand-set states of one triangle."""
    import torch

    l, S, proc, curr, S_after, nxt = case
    G = pkt.build_csr(dev([0, 0, 1]), dev([1, 2, 2]), 3, degree_order=False)
    dS = dev(S)
    flags = torch.tensor(proc, dtype=torch.uint8, device="cuda") * pkt.PROCESSED
    got = G.peel_sublevel(dS, flags, dev(curr), l, variant=_var(pkt, variant))
    assert host(dS).tolist() == S_after
    assert sorted(host(got).tolist()) == nxt
    fl = host(flags)
    for e in curr:
        assert fl[e] == pkt.PROCESSED
    for e in nxt:
        assert fl[e] & pkt.IN_CURR


def test_sublevel_states_on_larger_graph(pkt):
    """Every sub-level of a real run, replayed one at a time through the
    state-level entry point with relabelling on, against the oracle's."""
    import torch

    g = gg.chung_lu(1500, 2.1, 14.0, 300.0, seed=31)
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n, degree_order=True)
    S = oracle.support(g.n, eu, ev).copy()
    flags = np.zeros(eu.size, np.uint8)
    dS = dev(S)
    dF = torch.zeros(eu.size, dtype=torch.uint8, device="cuda")
    todo, l, steps = eu.size, 0, 0
    while todo > 0:
        curr = np.nonzero((S == l) & (flags & oracle.PROCESSED == 0))[0].astype(np.int32)
        while curr.size:
            todo -= curr.size
            want_next = oracle.sublevel(g.n, eu, ev, S, flags, curr, l)
            dF[torch.from_numpy(curr).long().cuda()] |= pkt.IN_CURR
            got_next = G.peel_sublevel(dS, dF, dev(curr), l, variant=steps % 3 - 1)
            assert np.array_equal(np.sort(host(got_next)), want_next)
            assert np.array_equal(host(dS), S)
            assert np.array_equal(host(dF), flags)
            curr = want_next
            steps += 1
        l += 1


# ----------------------------------------------------------------- edge cases

def test_empty_and_degenerate_inputs(pkt):
    import torch

    e = torch.empty(0, dtype=torch.int32, device="cuda")
    for n in (0, 1, 10):
        G = pkt.build_csr(e, e, n)
        assert G.m == 0 and G.decompose().numel() == 0 and G.support().numel() == 0
    # only self-loops and repeats of one edge
    G = pkt.build_csr(dev([3, 3, 1, 2, 2, 1]), dev([3, 3, 2, 1, 1, 2]), 5)
    assert G.m == 1 and host(G.decompose()).tolist() == [2]
    # isolated vertices around a triangle, both orientations, repeats
    G = pkt.build_csr(dev([7, 9, 9, 8, 7]), dev([9, 8, 7, 7, 8]), 20)
    assert host(G.decompose()).tolist() == [3, 3, 3]
    u, v = G.edge_list()
    assert host(u).tolist() == [7, 7, 8] and host(v).tolist() == [8, 9, 9]


def test_bad_ids_are_rejected(pkt):
    with pytest.raises(pkt.TrussError) as ex:
        pkt.build_csr(dev([0, 1]), dev([1, 5]), 5)
    assert ex.value.status == pkt.EBADGRAPH
    with pytest.raises(pkt.TrussError) as ex:
        pkt.build_csr(dev([0, -1]), dev([1, 2]), 5)
    assert ex.value.status == pkt.EBADGRAPH


@pytest.mark.parametrize("relabel", [False, True])
def test_bad_frontier_ids_are_rejected(pkt, relabel):
    """A caller's frontier for one ProcessSubLevel is validated on the device
    before any kernel indexes with it: ids outside [0, m) and repeated ids
    give EBADGRAPH, more ids than edges EINVAL, and the state is left
    untouched."""
    import torch

    # K4: six edges, each in two triangles
    G = pkt.build_csr(dev([0, 0, 0, 1, 1, 2]), dev([1, 2, 3, 2, 3, 3]), 4, degree_order=relabel)
    m = G.m
    for curr, status in (([0, m], pkt.EBADGRAPH), ([-1], pkt.EBADGRAPH), ([2, 2], pkt.EBADGRAPH),
                         ([0, 1, 2, 3, 4, 5, 0], pkt.EINVAL)):
        dS = dev([2] * m)
        flags = torch.zeros(m, dtype=torch.uint8, device="cuda")
        with pytest.raises(pkt.TrussError) as ex:
            G.peel_sublevel(dS, flags, dev(curr), 2)
        assert ex.value.status == status, curr
        assert host(dS).tolist() == [2] * m and host(flags).tolist() == [0] * m
    # a valid frontier still runs after the rejections: all six edges at
    # level 2 are processed together, and no support changes
    dS = dev([2] * m)
    flags = torch.zeros(m, dtype=torch.uint8, device="cuda")
    nxt = G.peel_sublevel(dS, flags, dev(list(range(m))), 2)
    assert nxt.numel() == 0 and host(dS).tolist() == [2] * m
    assert host(flags).tolist() == [pkt.PROCESSED] * m


@pytest.mark.parametrize("loop", ["persistent_lat", "persistent_occ", "graph"])
def test_barrier_wait_limit_returns_status(pkt, loop):
    """A grid-barrier wait (persistent forms) or a phase (graph form) that
    runs past its limit ends the run with TRUSS_ETIMEOUT (here the limit is
    1 ns, so the first one runs out); the context stays usable and the next
    call is exact."""
    g = gg.workload("rmat10_ef8")
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
    with pytest.raises(pkt.TrussError) as ex:
        G.decompose(loop=_loop(pkt, loop), timeout_ns=1)
    assert ex.value.status == pkt.ETIMEOUT
    tau = G.decompose(loop=_loop(pkt, loop))
    assert np.array_equal(host(tau), oracle.truss_of_edges(g.n, g.src, g.dst)[2])


def test_host_buffer_pipeline(pkt):
    for name, g in SMALL[:3]:
        tau, st = pkt.decompose_host(g.src, g.dst, g.n)
        assert np.array_equal(tau, oracle.truss_of_edges(g.n, g.src, g.dst)[2])
        assert st["m"] == tau.size


def test_stats(pkt):
    g = gg.workload("rmat10_ef8")
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
    tau, st = G.decompose(stats=True)
    eu, ev, want = oracle.truss_of_edges(g.n, g.src, g.dst)
    S0 = oracle.support(g.n, eu, ev)
    assert st["triangles"] * 3 == int(S0.sum())
    assert st["t_max"] == int(want.max())
    assert st["m"] == eu.size
    _, lv, sz = oracle.pkt_serial(g.n, eu, ev)
    assert st["sublevels"] == sz.size and st["levels"] == np.unique(lv).size


def _scan_sequence(m, tau, step):
    """Levels of the Scans of Algorithm 4 with level jumps (an empty Scan
    jumps to the smallest live support), and the entries each visits: all m
    for the first, then the survivors of the one before -- edges of a higher
    level, plus edges of its own level that entered a later sub-level than
    the Scan's frontier."""
    L = tau.astype(np.int64) - 2
    levels = np.unique(L)
    first = {int(l): int(step[L == l].min()) for l in levels}
    seq, l, done = [], 0, 0
    while done < m:
        seq.append(l)
        if l in first:
            done += int((L == l).sum())
            l += 1
        else:
            l = int(levels[levels > l].min())
    surv = lambda l: int((L > l).sum()) + (int(((L == l) & (step != first[l])).sum()) if l in first else 0)
    visited = [m] + [surv(x) for x in seq[:-1]]
    return seq, visited


@pytest.mark.parametrize("loop", ["plain", "persistent_lat", "graph"])
def test_core_order_is_a_degeneracy_order_and_exact(pkt, loop):
    """With TRUSS_CORE_ORDER the internal labels follow the device k-core
    peel: every vertex has at most its coreness (brute-force minimum-degree
    removal) of neighbours with a higher label; trussness is unchanged."""
    from brute import coreness

    graphs = [gg.workload("rmat10_ef8"), gg.chung_lu(6000, 2.1, 12.0, 600.0, seed=21),
              gg.rgg2d(5000, 14.0, seed=22), gg.small_random(40, 0.3, seed=23)]
    for g in graphs:
        G = pkt.build_csr(dev(g.src), dev(g.dst), g.n, core_order=True)
        eu, ev, want = oracle.truss_of_edges(g.n, g.src, g.dst)
        assert np.array_equal(host(G.decompose(loop=_loop(pkt, loop))), want), g.name
        rp, col, eid, eo, order = (host(x) for x in G.csr())
        core = coreness(g.n, eu, ev)
        up = rp[1:] - eo  # neighbours after each internal vertex
        assert np.all(up <= core[order]), g.name
        G.free()


def _rcm_host(n, eu, ev):
    """Reverse Cuthill-McKee labels written out on the host: breadth-first
    search from the vertex of highest degree (lowest label among ties); each
    new level in order of (lowest rank among its neighbours in the level
    before, label); ranks reversed; unreached vertices first, in label
    order.  Returns the input label of each internal label."""
    adj = [[] for _ in range(n)]
    for a, b in zip(eu.tolist(), ev.tolist()):
        adj[a].append(b)
        adj[b].append(a)
    deg = np.array([len(r) for r in adj])
    rank = {}
    if deg.max(initial=0) > 0:
        s = int(np.flatnonzero(deg == deg.max())[0])
        rank[s] = 0
        level = [s]
        while level:
            par = {}
            for u in level:
                for w in adj[u]:
                    if w not in rank:
                        par[w] = min(par.get(w, n), rank[u])
            level = sorted(par, key=lambda w: (par[w], w))
            for w in level:
                rank[w] = len(rank)
    reached = len(rank)
    for v in range(n):
        if v not in rank:
            rank[v] = len(rank)
    order = np.empty(n, np.int64)
    for v, r in rank.items():
        order[n - 1 - r] = v
    return order, reached


@pytest.mark.parametrize("loop", ["plain", "persistent"])
def test_locality_order_is_rcm_and_exact(pkt, loop):
    """With TRUSS_LOCALITY_ORDER the internal labels are the reverse
    Cuthill-McKee order the host restatement gives, vertex for vertex
    (connected and disconnected graphs, isolated vertices); the edge list,
    the support and the trussness are the oracle's."""
    two = gg.small_random(50, 0.3, seed=41)
    union = gg.EdgeList(230, np.concatenate([two.src, two.src + 60, np.array([120, 121, 122], np.int32)]),
                        np.concatenate([two.dst, two.dst + 60, np.array([121, 122, 120], np.int32)]), "union")
    graphs = [gg.workload("rmat10_ef8"), gg.chung_lu(6000, 2.1, 12.0, 600.0, seed=21),
              gg.rgg2d(5000, 14.0, seed=22), union]
    for g in graphs:
        G = pkt.build_csr(dev(g.src), dev(g.dst), g.n, locality_order=True)
        eu, ev, want = oracle.truss_of_edges(g.n, g.src, g.dst)
        u, v = G.edge_list()
        assert np.array_equal(host(u), eu) and np.array_equal(host(v), ev), g.name
        assert np.array_equal(host(G.support()), oracle.support(g.n, eu, ev)), g.name
        assert np.array_equal(host(G.decompose(loop=_loop(pkt, loop))), want), g.name
        rp, col, eid, eo, order = (host(x) for x in G.csr())
        want_order, reached = _rcm_host(g.n, eu, ev)
        assert np.array_equal(order, want_order), g.name
        assert 0 < reached <= g.n
        G.free()


def _want_bps(st):
    per_level = st["dmin_sum"] // (st["max_support"] + 1)
    return 6 if per_level >= 1 << 24 or st["dmin_sum"] >= 1 << 34 else 4


def test_persistent_form_choice(pkt):
    """The automatic persistent form takes 6 blocks per SM when the
    shorter-row entries of the walk (W = sum of min(d(u), d(v))) reach 2^24
    per support level or 2^34 in all, and 4 otherwise; forced forms are
    honoured and every form gives the oracle's trussness."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for g in (gg.rgg2d(30000, 20.0, seed=5), gg.chung_lu(30000, 2.1, 12.0, 3000.0, seed=6)):
        G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
        eu, ev, want = oracle.truss_of_edges(g.n, g.src, g.dst)
        S = oracle.support(g.n, eu, ev)
        for loop in (pkt.LOOP_PERSISTENT, pkt.LOOP_PERSISTENT_LAT, pkt.LOOP_PERSISTENT_OCC):
            tau, st = G.decompose(loop=loop, stats=True)
            assert np.array_equal(host(tau), want)
            assert st["max_support"] == int(S.max())
            bps = {pkt.LOOP_PERSISTENT: _want_bps(st), pkt.LOOP_PERSISTENT_LAT: 4, pkt.LOOP_PERSISTENT_OCC: 6}[loop]
            assert st["blocks_per_sm"] == bps and st["grid_blocks"] == bps * sms
        _, st = G.decompose(loop=pkt.LOOP_PLAIN, stats=True)
        assert st["grid_blocks"] == 0 and st["blocks_per_sm"] == 0
    # a level of the geometric workload holds about 3e7 entries: 6 blocks
    g = gg.workload("rgg2d_n2^21_d32")
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
    _, st = G.decompose(loop=pkt.LOOP_PERSISTENT, stats=True)
    assert _want_bps(st) == 6 and st["blocks_per_sm"] == 6
    G.free()


@pytest.mark.parametrize("loop", LOOPS)
def test_scan_counts_match_the_live_list(pkt, loop):
    """Scans and scanned entries reported by the library equal the counts
    the serial run implies: each Scan after the first visits exactly the
    edges the previous one kept."""
    for g in (gg.workload("rmat10_ef8"), gg.chung_lu(3000, 2.1, 14.0, 300.0, seed=8)):
        G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
        _, st = G.decompose(loop=_loop(pkt, loop), stats=True)
        eu, ev = oracle.canonical(g.n, g.src, g.dst)
        want, _, _, ostep = oracle.pkt_serial(g.n, eu, ev, return_steps=True)
        seq, visited = _scan_sequence(eu.size, want, ostep)
        assert st["scans"] == len(seq)
        assert st["scanned"] == sum(visited), (st["scanned"], sum(visited))


@pytest.mark.parametrize("loop", LOOPS)
def test_peel_steps_match_serial_run_and_certify(pkt, loop):
    """The sub-level each edge was peeled in equals the serial run's, and
    the (trussness, peel step) pair passes the certificate."""
    import torch

    for name, g in SMALL:
        G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
        step = torch.empty(G.m, dtype=torch.int32, device="cuda")
        tau = host(G.decompose(loop=_loop(pkt, loop), peel_step=step))
        eu, ev = oracle.canonical(g.n, g.src, g.dst)
        want, _, _, ostep = oracle.pkt_serial(g.n, eu, ev, return_steps=True)
        assert np.array_equal(tau, want), name
        assert np.array_equal(host(step), ostep), name
        assert oracle.certify(g.n, eu, ev, tau, host(step))[0] == 0


@pytest.mark.parametrize("loop", LOOPS)
def test_sublevel_trace(pkt, loop):
    """The per-sub-level trace agrees with the recorded frontier sequence and
    with the graph: sizes sum to m, todo counts down, lane groups are valid,
    dsum/dmax match the frontier's shorter-row lengths."""
    g = gg.chung_lu(4000, 2.1, 16.0, 400.0, seed=11)
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
    tau, (lv, sz), tr = G.decompose(loop=_loop(pkt, loop), record=True, trace=True)
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    want, olv, osz, step = oracle.pkt_serial(g.n, eu, ev, return_steps=True)
    assert np.array_equal(host(tau), want)
    assert np.array_equal(tr["level"], olv) and np.array_equal(tr["n_light"] + tr["n_heavy"], osz)
    assert np.array_equal(tr["todo"], eu.size - np.concatenate([[0], np.cumsum(osz)[:-1]]))
    assert set(np.unique(tr["group"])) <= {1, 16, 32}
    assert np.all(tr["t_ns"] > 0) and tr["scan_ns"][0] > 0 and np.all(tr["scan_ns"] >= 0)
    deg = np.bincount(np.concatenate([eu, ev]), minlength=g.n)
    dmin = np.minimum(deg[eu], deg[ev])
    for k in range(len(tr)):
        sel = step == k
        assert tr["dsum"][k] == int(dmin[sel].sum()) and tr["dmax"][k] == int(dmin[sel].max())
        assert tr["n_light"][k] == int((dmin[sel] <= 32).sum())


@pytest.mark.parametrize("loop", LOOPS)
def test_batch_matches_oracle(pkt, loop):
    """Many independent graphs of uneven size in one run (their disjoint
    union), including an empty graph and a triangle-free one."""
    gs = gg.chung_lu_batch(48, seed0=1000)
    gs.insert(5, gg.EdgeList(7, np.zeros(0, np.int32), np.zeros(0, np.int32), "empty"))
    gs.insert(9, gg.EdgeList(6, np.arange(5, dtype=np.int32), np.arange(1, 6, dtype=np.int32), "path"))
    got = pkt.decompose_batch(gs, loop=_loop(pkt, loop))
    want = oracle.truss_batch(gs, nthreads=4)
    assert len(got) == len(gs)
    for g, t, w in zip(gs, got, want):
        assert np.array_equal(host(t), w), g.name


def test_batch_rejects_ids_outside_their_graph(pkt):
    a = gg.EdgeList(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    b = gg.EdgeList(3, np.array([0, 1], np.int32), np.array([1, 3], np.int32))  # 3 is outside graph b
    with pytest.raises(pkt.TrussError) as ex:
        pkt.decompose_batch([a, b])
    assert ex.value.status == pkt.EBADGRAPH


# ---------------------------------------------------------- k-truss listing

@pytest.mark.parametrize("order", ["degree", "core", "input"])
def test_ktruss_components_match_oracle(pkt, order):
    """Every k-truss (component of the edges of trussness >= k, labelled by
    its smallest input vertex) equals the oracle's, for every k, in every
    internal vertex order."""
    import itertools

    pairs = list(itertools.combinations(range(4), 2)) + list(itertools.combinations(range(10, 15), 2))
    pairs += [(20, 21), (21, 22), (3, 20)]
    cliques = gg.EdgeList(23, np.array([a for a, _ in pairs], np.int32), np.array([b for _, b in pairs], np.int32),
                          "cliques")
    graphs = [cliques, gg.workload("rmat10_ef8"), gg.chung_lu(6000, 2.1, 12.0, 600.0, seed=41),
              gg.rgg2d(5000, 14.0, seed=42), gg.small_random(40, 0.3, seed=43)]
    for g in graphs:
        G = pkt.build_csr(dev(g.src), dev(g.dst), g.n, degree_order=order == "degree", core_order=order == "core")
        eu, ev, want_tau = oracle.truss_of_edges(g.n, g.src, g.dst)
        tau = G.decompose()
        assert np.array_equal(host(tau), want_tau)
        for k in sorted({2, 3, int(want_tau.max()), int(want_tau.max()) + 1} | set(range(2, 8))):
            comp, nc = G.ktruss_components(tau, k)
            want, wnc = oracle.ktruss_components(g.n, eu, ev, want_tau, k)
            assert np.array_equal(host(comp), want), (g.name, k)
            assert nc == wnc, (g.name, k)
        G.free()


def test_ktruss_components_full_size(pkt):
    """The bench workload: the k-trusses for k = 3, 20 and the top level,
    from the device trussness, equal the oracle's components of the same
    trussness."""
    g = gg.workload("chunglu_n2^20_d20")
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
    tau = G.decompose()
    th = host(tau)
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    for k in (3, 20, int(th.max())):
        comp, nc = G.ktruss_components(tau, k)
        want, wnc = oracle.ktruss_components(g.n, eu, ev, th, k)
        assert np.array_equal(host(comp), want) and nc == wnc, k
    G.free()


def test_triangle_count(pkt):
    """The triangle-count mode of the support kernels gives T = (sum of the
    oracle's supports) / 3, with int32 and int64 row offsets, and the
    decomposition's own count on the bench workload."""
    for g in (gg.workload("rmat10_ef8"), gg.chung_lu(6000, 2.1, 12.0, 600.0, seed=51), gg.rgg2d(5000, 14.0, seed=52),
              gg.small_random(40, 0.3, seed=53)):
        eu, ev = oracle.canonical(g.n, g.src, g.dst)
        T = int(oracle.support(g.n, eu, ev).astype(np.int64).sum()) // 3
        for off64 in (False, True):
            G = pkt.build_csr(dev(g.src), dev(g.dst), g.n, offsets64=off64)
            assert G.triangle_count() == T, (g.name, off64)
            G.free()
    g = gg.workload("chunglu_n2^20_d20")
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
    _, st = G.decompose(stats=True)
    assert G.triangle_count() == st["triangles"]
    G.free()


@pytest.mark.parametrize("relabel,off64", [(True, False), (False, False), (True, True)])
def test_edge_centric_support_matches_oracle(pkt, relabel, off64):
    """Algorithm 2's edge-centric support (every edge counts its common
    neighbours on its own) equals the oracle's S(e) element by element, on
    graphs with short rows, hub rows (bitmap probes), a wheel whose hub row
    spans many rounds of a warp, and the empty graph."""
    k = 3000
    wheel = gg.EdgeList(k + 1, np.concatenate([np.zeros(k), np.arange(1, k + 1)]).astype(np.int32),
                        np.concatenate([np.arange(1, k + 1), np.arange(1, k + 1) % k + 1]).astype(np.int32), "wheel")
    hubs = gg.chung_lu(20000, 2.1, 20.0, 5000.0, seed=13)
    for name, g in SMALL + [("wheel", wheel), ("hubs", hubs)]:
        G = pkt.build_csr(dev(g.src), dev(g.dst), g.n, **_flags(relabel, off64))
        eu, ev = oracle.canonical(g.n, g.src, g.dst)
        want = oracle.support(g.n, eu, ev)
        assert np.array_equal(host(G.support_ros()), want), name
        # unchanged by a decomposition (and its compactions) before it
        G.decompose(compact=1)
        assert np.array_equal(host(G.support_ros()), want), name
        G.free()
    e = dev(np.zeros(0, np.int32))
    G = pkt.build_csr(e, e, 4)
    assert G.support_ros().numel() == 0


@pytest.mark.parametrize("relabel,off64", [(True, False), (False, False), (True, True)])
def test_support_switches_to_hub_bitmaps(pkt, relabel, off64):
    """Graphs with hub vertices (degree >= 1024): for pairs u < v whose v is
    a hub and whose N+(v) is longer than u's entries above v, the support
    kernels walk those entries and probe v's bitmap.  The support equals the
    oracle's, the probes happen, and they replace more N+(v) entries than
    they cost (the switch is taken when it saves at least a tenth of W+)."""
    k = 3000
    wheel = gg.EdgeList(k + 1, np.concatenate([np.zeros(k), np.arange(1, k + 1)]).astype(np.int32),
                        np.concatenate([np.arange(1, k + 1), np.arange(1, k + 1) % k + 1]).astype(np.int32), "wheel")
    probes = 0
    for g in (gg.chung_lu(20000, 2.1, 20.0, 5000.0, seed=13), gg.chung_lu(30000, 1.9, 40.0, 20000.0, seed=17),
              gg.rmat(14, 32, seed=9), wheel):
        G = pkt.build_csr(dev(g.src), dev(g.dst), g.n, **_flags(relabel, off64))
        eu, ev = oracle.canonical(g.n, g.src, g.dst)
        S = oracle.support(g.n, eu, ev)
        assert np.array_equal(host(G.support()), S), g.name
        tau, st = G.decompose(stats=True)
        assert np.array_equal(host(tau), oracle.truss(g.n, eu, ev)), g.name
        assert st["support_walked"] + st["support_hub_probes"] <= st["wedges_up"], g.name
        if st["support_hub_probes"] > 0:
            # a switch that ran saved at least a tenth of W+: the N+(v)
            # entries it skipped less the probes it made instead
            saved = st["wedges_up"] - st["support_walked"] - st["support_hub_probes"]
            assert 10 * saved >= st["wedges_up"], g.name
        probes += st["support_hub_probes"]
        G.free()
    if relabel:
        assert probes > 0


def test_pool_keep_setting(pkt):
    """The pool retention setting changes nothing but memory reuse: builds
    and decompositions around each setting stay exact."""
    g = gg.chung_lu(20000, 2.1, 20.0, 5000.0, seed=13)
    want = oracle.truss_of_edges(g.n, g.src, g.dst)[2]
    for keep in (0, 1 << 34, 16 << 30):
        pkt.pool_keep(keep)
        G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
        assert np.array_equal(host(G.decompose()), want), keep
        G.free()
        tau, _ = pkt.decompose_host(g.src, g.dst, g.n)
        assert np.array_equal(tau, want), keep
