"""The asynchronous local (h-index) truss iteration, CUDA path vs the CPU
oracle: element by element on small graphs and the R-MAT scale-10 workload,
on cliques whose h-index needs the counting fallback above the histogram,
and at the full size of the power-law and geometric workloads by the
oracle's certificate (the witness order is the peel's, the values checked
are the local iteration's own)."""
import itertools

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


def small():
    k = 3000
    wheel = gg.EdgeList(k + 1, np.concatenate([np.zeros(k), np.arange(1, k + 1)]).astype(np.int32),
                        np.concatenate([np.arange(1, k + 1), np.arange(1, k + 1) % k + 1]).astype(np.int32), "wheel")
    return [("rmat10", gg.workload("rmat10_ef8")), ("rmat8_s7", gg.rmat(8, 16, seed=7)),
            ("chunglu", gg.chung_lu(4000, 2.1, 16.0, 400.0, seed=11)), ("rgg", gg.rgg2d(4000, 24.0, seed=12)),
            ("hubs", gg.chung_lu(20000, 2.1, 20.0, 5000.0, seed=13)), ("wheel", wheel)] + [
        (f"gnp{s}", gg.small_random(40 + 10 * s, 0.35, seed=300 + s)) for s in range(4)]


@pytest.mark.parametrize("relabel,off64", [(True, False), (False, False), (True, True)])
def test_local_iteration_matches_oracle(pkt, relabel, off64):
    for name, g in small():
        G = pkt.build_csr(dev(g.src), dev(g.dst), g.n, degree_order=relabel, offsets64=off64)
        tau, st = G.decompose_local(stats=True)
        want = oracle.truss_of_edges(g.n, g.src, g.dst)[2]
        assert np.array_equal(host(tau), want), name
        if want.size and want.max() > 2:
            assert st["sweeps"] >= 2 and st["updates"] > 0
        G.free()


def test_cliques_and_the_counting_fallback(pkt):
    """K_n: every edge has trussness n.  Above 513 the h-index is found by
    the counting search past the histogram's top bucket; a clique joined to
    a pendant triangle and a path keeps their values."""
    for n in (4, 60, 513, 514, 700):
        pr = np.array(list(itertools.combinations(range(n), 2)), np.int32)
        src = np.concatenate([pr[:, 0], [n, n, n + 1, n + 2]]).astype(np.int32)
        dst = np.concatenate([pr[:, 1], [n + 1, n + 2, n + 2, n + 3]]).astype(np.int32)
        G = pkt.build_csr(dev(src), dev(dst), n + 4)
        tau = host(G.decompose_local())
        want = oracle.truss_of_edges(n + 4, src, dst)[2]
        assert np.array_equal(tau, want), n
        assert np.all(tau[: pr.shape[0]] == n)
        G.free()


def test_empty_and_sweep_limit(pkt):
    e = dev(np.zeros(0, np.int32))
    G = pkt.build_csr(e, e, 5)
    assert G.decompose_local().numel() == 0
    g = gg.chung_lu(4000, 2.1, 16.0, 400.0, seed=11)
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
    with pytest.raises(pkt.TrussError) as ex:
        G.decompose_local(max_sweeps=1)
    assert ex.value.status == pkt.ETIMEOUT
    # the graph stays usable
    assert np.array_equal(host(G.decompose_local()), oracle.truss_of_edges(g.n, g.src, g.dst)[2])


@pytest.mark.parametrize("name", ["chunglu_n2^20_d20", "rgg2d_n2^21_d32"])
def test_local_iteration_full_size_certified(pkt, name):
    import torch

    g = gg.workload(name)
    G = pkt.build_csr(dev(g.src), dev(g.dst), g.n)
    tau, st = G.decompose_local(stats=True)
    step = torch.empty(G.m, dtype=torch.int32, device="cuda")
    G.decompose(peel_step=step)
    eu, ev = oracle.canonical(g.n, g.src, g.dst)
    bad, first = oracle.certify(g.n, eu, ev, host(tau), host(step))
    assert bad == 0, f"{bad} edges violate the certificate (first: {first})"
    G.free()
