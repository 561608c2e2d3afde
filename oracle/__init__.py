"""CPU oracle for truss decomposition -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (the CUDA library and its
binding) never calls it and never falls back to it.

The arithmetic lives in ``truss_oracle.c`` (plain serial C, compiled with gcc
on first use); this module only marshals numpy arrays.  Every function
follows the paper's definitions and algorithms as cited in that file:
§II (support, k-truss, trussness), Algorithm 1 (serial bottom-up peel),
Algorithms 4 and 5 (level-synchronous Scan / ProcessSubLevel, run serially).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "truss_oracle.c")
_LIB = os.path.join(_HERE, "libtruss_oracle.so")
_lib = None

PROCESSED = 1
IN_CURR = 2


def build(force: bool = False) -> str:
    """Compile ``libtruss_oracle.so`` next to its source (gcc)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
    os.replace(tmp, _LIB)
    return _LIB


def bind(path: str):
    """Load an oracle library at ``path`` and declare its signatures."""
    lib = ctypes.CDLL(path)
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    I32, I64 = ctypes.c_int32, ctypes.c_int64
    lib.or_canonical.argtypes = [i32p, i32p, I64, I32, i32p, i32p]
    lib.or_canonical.restype = I64
    lib.or_support.argtypes = [I32, I64, i32p, i32p, i32p]
    lib.or_support.restype = ctypes.c_int
    lib.or_truss_wc.argtypes = [I32, I64, i32p, i32p, i32p, i32p]
    lib.or_truss_wc.restype = ctypes.c_int
    lib.or_pkt_serial.argtypes = [I32, I64, i32p, i32p, i32p, i32p, i64p, I64, i32p]
    lib.or_pkt_serial.restype = I64
    lib.or_sublevel.argtypes = [I32, I64, i32p, i32p, i32p, u8p, i32p, I64, I32, i32p]
    lib.or_sublevel.restype = I64
    lib.or_truss_batch.argtypes = [I64, i32p, i64p, i32p, i32p, i64p, i32p, ctypes.c_int]
    lib.or_truss_batch.restype = ctypes.c_int
    lib.or_certify.argtypes = [I32, I64, i32p, i32p, i32p, i32p, ctypes.c_int, i64p]
    lib.or_certify.restype = I64
    lib.or_certify_sample.argtypes = [I32, I64, i32p, i32p, i32p, i32p, i64p, I64, i64p]
    lib.or_certify_sample.restype = I64
    lib.or_ktruss_components.argtypes = [I32, I64, i32p, i32p, i32p, I32, i32p]
    lib.or_ktruss_components.restype = I64
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = bind(build())
    return _lib


def use_library(lib) -> None:
    """Route this module's functions to another bound library (tests that
    check the pins against deliberately broken copies of the oracle use
    this); ``use_library(None)`` restores the real one."""
    global _lib
    _lib = lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _check(rc, what):
    if rc == -1:
        raise ValueError(f"oracle {what}: bad argument")
    if rc == -2:
        raise MemoryError(f"oracle {what}: out of memory")
    if rc < 0:
        raise RuntimeError(f"oracle {what}: error {rc}")


def canonical(n: int, src, dst):
    """Undirected canonical edge list (u < v, lexicographic, no self-loops or
    repeats).  Returns ``(eu, ev)``; the position is the edge id."""
    lib = _load()
    s, sp = _i32(src)
    d, dp = _i32(dst)
    eu = np.empty(max(s.shape[0], 1), np.int32)
    ev = np.empty(max(s.shape[0], 1), np.int32)
    m = lib.or_canonical(sp, dp, s.shape[0], n, _i32(eu)[1], _i32(ev)[1])
    _check(m, "canonical")
    return eu[:m].copy(), ev[:m].copy()


def support(n: int, eu, ev) -> np.ndarray:
    """Per-edge triangle count S(e) = |N(u) ∩ N(v)| (§II)."""
    lib = _load()
    eu, up = _i32(eu)
    ev, vp = _i32(ev)
    S = np.empty(max(eu.shape[0], 1), np.int32)
    _check(lib.or_support(n, eu.shape[0], up, vp, _i32(S)[1]), "support")
    return S[: eu.shape[0]]


def truss(n: int, eu, ev, return_support: bool = False):
    """Trussness per canonical edge by the serial peel of Algorithm 1."""
    lib = _load()
    eu, up = _i32(eu)
    ev, vp = _i32(ev)
    m = eu.shape[0]
    tau = np.empty(max(m, 1), np.int32)
    S0 = np.empty(max(m, 1), np.int32)
    _check(lib.or_truss_wc(n, m, up, vp, _i32(tau)[1], _i32(S0)[1]), "truss")
    if return_support:
        return tau[:m], S0[:m]
    return tau[:m]


def truss_of_edges(n: int, src, dst):
    """Canonicalise a raw edge list, then decompose it.  Returns (eu, ev, tau)."""
    eu, ev = canonical(n, src, dst)
    return eu, ev, truss(n, eu, ev)


def pkt_serial(n: int, eu, ev, max_sub: int = 1 << 20, return_steps: bool = False):
    """Algorithm 4 with Algorithm 5, one edge at a time.  Returns
    ``(tau, sub_levels, sub_sizes)``: trussness and, per non-empty sub-level,
    its level l and frontier size |curr|; with ``return_steps`` also the
    sub-level number each edge was peeled in."""
    lib = _load()
    eu, up = _i32(eu)
    ev, vp = _i32(ev)
    m = eu.shape[0]
    tau = np.empty(max(m, 1), np.int32)
    step = np.empty(max(m, 1), np.int32)
    lv = np.empty(max_sub, np.int32)
    sz = np.empty(max_sub, np.int64)
    ns = lib.or_pkt_serial(n, m, up, vp, _i32(tau)[1], _i32(lv)[1],
                           sz.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), max_sub, _i32(step)[1])
    _check(ns, "pkt_serial")
    if ns > max_sub:
        raise ValueError("more sub-levels than max_sub")
    if return_steps:
        return tau[:m], lv[:ns].copy(), sz[:ns].copy(), step[:m].copy()
    return tau[:m], lv[:ns].copy(), sz[:ns].copy()


def certify(n: int, eu, ev, tau, step, nthreads: int | None = None):
    """Check a claimed trussness with its claimed peeling order against the
    definition (see or_certify).  Returns ``(violations, first_bad_edge)``;
    zero violations proves the claim exact."""
    lib = _load()
    eu, up = _i32(eu)
    ev, vp = _i32(ev)
    tau, tp = _i32(tau)
    step, sp = _i32(step)
    fb = ctypes.c_int64()
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    r = lib.or_certify(n, eu.shape[0], up, vp, tp, sp, nthreads, ctypes.byref(fb))
    _check(r, "certify")
    return int(r), int(fb.value)


def sublevel(n: int, eu, ev, S, flags, curr, l: int):
    """One ProcessSubLevel (Algorithm 5) on the given state.  ``S`` (int32)
    and ``flags`` (uint8; bit 0 processed, bit 1 inCurr) are updated in place
    as the algorithm leaves them (curr processed, next marked in-curr).
    Returns ``next`` in ascending edge id order."""
    lib = _load()
    eu, up = _i32(eu)
    ev, vp = _i32(ev)
    assert S.dtype == np.int32 and S.flags.c_contiguous
    assert flags.dtype == np.uint8 and flags.flags.c_contiguous
    curr, cp = _i32(curr)
    nxt = np.empty(max(eu.shape[0], 1), np.int32)
    k = lib.or_sublevel(n, eu.shape[0], up, vp, S.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                        flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), cp, curr.shape[0], l,
                        _i32(nxt)[1])
    _check(k, "sublevel")
    return nxt[:k].copy()


def truss_batch(graphs, nthreads: int | None = None):
    """Decompose many independent raw edge lists (objects with ``n``, ``src``,
    ``dst``) on host threads.  Returns a list of per-graph trussness arrays
    (canonical order of each graph)."""
    lib = _load()
    G = len(graphs)
    nverts = np.array([g.n for g in graphs], np.int32)
    eoff = np.zeros(G + 1, np.int64)
    eoff[1:] = np.cumsum([g.src.shape[0] for g in graphs])
    src = np.concatenate([g.src for g in graphs]).astype(np.int32) if G else np.zeros(1, np.int32)
    dst = np.concatenate([g.dst for g in graphs]).astype(np.int32) if G else np.zeros(1, np.int32)
    mo = np.zeros(max(G, 1), np.int64)
    tau = np.empty(max(int(eoff[-1]), 1), np.int32)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    rc = lib.or_truss_batch(G, _i32(nverts)[1], eoff.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            _i32(src)[1], _i32(dst)[1], mo.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            _i32(tau)[1], nthreads)
    _check(rc, "truss_batch")
    return [tau[eoff[i]: eoff[i] + mo[i]].copy() for i in range(G)]


def certify_sample(n: int, eu, ev, tau, step, sample):
    """or_certify's per-edge conditions for the edge ids in ``sample`` and
    its order check over all edges.  Returns ``(violations, first_bad)``."""
    lib = _load()
    eu, up = _i32(eu)
    ev, vp = _i32(ev)
    tau, tp = _i32(tau)
    step, sp = _i32(step)
    sample = np.ascontiguousarray(sample, np.int64)
    fb = ctypes.c_int64()
    r = lib.or_certify_sample(n, eu.shape[0], up, vp, tp, sp, sample.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                              sample.shape[0], ctypes.byref(fb))
    _check(r, "certify_sample")
    return int(r), int(fb.value)


def ktruss_components(n: int, eu, ev, tau, k: int):
    """The k-trusses as components (§II): per edge, the smallest vertex label
    of its component among the edges of trussness >= k, or -1; and the
    number of components."""
    lib = _load()
    eu, pu = _i32(eu)
    ev, pv = _i32(ev)
    tau, pt = _i32(tau)
    comp = np.empty(max(eu.size, 1), np.int32)
    nc = lib.or_ktruss_components(n, eu.size, pu, pv, pt, k, comp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    _check(nc, "ktruss_components")
    return comp[: eu.size].copy(), int(nc)
