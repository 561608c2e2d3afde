"""Seeded synthetic graph inputs for the truss decomposition tests and bench.

This module only draws inputs: raw undirected edge lists (int32 ``src``,
``dst`` arrays, possibly holding self-loops and repeated pairs) with the
shapes of the paper's workload classes (social-network-like power-law graphs
and mesh-like geometric graphs, §IV-A).  It holds none of the method's
arithmetic; both the CUDA path and the CPU oracle canonicalise the lists on
their own.  The generators are written in C (``graphgen.c``) with
counter-based randomness, so every array is a pure function of its seed.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libgraphgen.so`` next to its source (gcc, a second or two)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread",
                           _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, i32p, i32p]
        lib.gg_rmat.restype = ctypes.c_int
        lib.gg_chung_lu.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_uint64, ctypes.c_int64, i32p, i32p]
        lib.gg_chung_lu.restype = ctypes.c_int
        lib.gg_chung_lu_weights.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
        lib.gg_chung_lu_weights.restype = ctypes.c_int
        lib.gg_rgg2d.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, i32p, i32p]
        lib.gg_rgg2d.restype = ctypes.c_int64
        lib.gg_batch_params.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_double)]
        lib.gg_batch_params.restype = None
        lib.gg_rand64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.gg_rand64.restype = ctypes.c_uint64
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


@dataclass
class EdgeList:
    """A raw undirected edge list on ``n`` vertices."""
    n: int
    src: np.ndarray  # int32
    dst: np.ndarray  # int32
    name: str = ""

    @property
    def n_in(self) -> int:
        return int(self.src.shape[0])


def rmat(scale: int, edge_factor: int, a=0.57, b=0.19, c=0.19, seed: int = 1) -> EdgeList:
    """R-MAT: ``edge_factor * 2^scale`` recursive-quadrant samples."""
    lib = _load()
    ns = edge_factor << scale
    src = np.empty(ns, np.int32)
    dst = np.empty(ns, np.int32)
    if lib.gg_rmat(scale, ns, a, b, c, seed, _p(src), _p(dst)) != 0:
        raise ValueError("bad R-MAT parameters")
    return EdgeList(1 << scale, src, dst, f"rmat{scale}_ef{edge_factor}_s{seed}")


def chung_lu_weights(n: int, gamma: float, mean_deg: float, max_deg: float) -> np.ndarray:
    w = np.empty(n, np.float64)
    _load().gg_chung_lu_weights(n, gamma, mean_deg, max_deg, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return w


def chung_lu(n: int, gamma: float, mean_deg: float, max_deg: float, seed: int) -> EdgeList:
    """Chung-Lu: ``round(n * mean_deg / 2)`` endpoint pairs drawn in proportion
    to power-law expected degrees ``(i+1)^(-1/(gamma-1))`` scaled to
    ``mean_deg`` and clipped at ``max_deg``."""
    lib = _load()
    ns = int(round(n * mean_deg / 2.0))
    src = np.empty(ns, np.int32)
    dst = np.empty(ns, np.int32)
    if lib.gg_chung_lu(n, gamma, mean_deg, max_deg, seed, ns, _p(src), _p(dst)) != 0:
        raise ValueError("bad Chung-Lu parameters")
    return EdgeList(n, src, dst, f"chunglu_n{n}_g{gamma}_d{mean_deg:g}_s{seed}")


def rgg2d(n: int, mean_deg: float, seed: int) -> EdgeList:
    """2-D random geometric graph on the unit square (no wrap-around)."""
    lib = _load()
    cnt = lib.gg_rgg2d(n, mean_deg, seed, None, None)
    if cnt < 0:
        raise ValueError("bad RGG parameters")
    src = np.empty(cnt, np.int32)
    dst = np.empty(cnt, np.int32)
    got = lib.gg_rgg2d(n, mean_deg, seed, _p(src), _p(dst))
    assert got == cnt
    return EdgeList(n, src, dst, f"rgg2d_n{n}_d{mean_deg:g}_s{seed}")


def batch_params(seed: int, n_lo=64, n_hi=8192, d_lo=8.0, d_hi=64.0):
    n = ctypes.c_int32()
    d = ctypes.c_double()
    _load().gg_batch_params(seed, n_lo, n_hi, d_lo, d_hi, ctypes.byref(n), ctypes.byref(d))
    return int(n.value), float(d.value)


def chung_lu_batch(num_graphs: int, seed0: int = 1000, gamma: float = 2.3,
                   n_lo=64, n_hi=8192, d_lo=8.0, d_hi=64.0) -> list[EdgeList]:
    """The ragged batch: graph ``i`` uses seed ``seed0 + i``, a log-uniform
    vertex count and mean degree, and weights clipped at ``n_i - 1``."""
    out = []
    for i in range(num_graphs):
        s = seed0 + i
        n, d = batch_params(s, n_lo, n_hi, d_lo, d_hi)
        out.append(chung_lu(n, gamma, d, float(n - 1), s))
    return out


def rand64(seed: int, stream: int, i: int) -> int:
    return int(_load().gg_rand64(seed, stream, i))


# The named workloads (sizes as the paper-class stand-ins use them).  Each
# entry is (generator of a seed, the workload's own seed); another seed gives
# a graph of the same family and size (calibration inputs).
WORKLOADS = {
    "rmat10_ef8": (lambda s: rmat(10, 8, seed=s), 1),
    "chunglu_n2^20_d20": (lambda s: chung_lu(1 << 20, 2.1, 20.0, float(1 << 14), s), 2),
    "rgg2d_n2^21_d32": (lambda s: rgg2d(1 << 21, 32.0, s), 3),
    "rmat24_ef16": (lambda s: rmat(24, 16, seed=s), 4),
    # the R-MAT scale-24 generator at 1/8 of its size: a case small enough
    # for a full profiler capture of the same kernels
    "rmat21_ef16": (lambda s: rmat(21, 16, seed=s), 4),
}
BATCH_WORKLOAD = "chunglu_batch4096"


def workload(name: str, seed: int | None = None) -> EdgeList:
    """The named workload; ``seed`` replaces its own seed."""
    fn, s0 = WORKLOADS[name]
    g = fn(s0 if seed is None else seed)
    g.name = name if seed is None or seed == s0 else f"{name}_s{seed}"
    return g


def small_random(n: int, p: float, seed: int) -> EdgeList:
    """Erdos-Renyi G(n, p) drawn from the counter-based stream (small tests)."""
    lib = _load()
    iu, ju = np.triu_indices(n, 1)
    k = np.arange(iu.shape[0], dtype=np.uint64)
    draws = np.array([lib.gg_rand64(seed, 7, int(x)) for x in k], dtype=np.uint64) if k.size < 4096 else None
    if draws is None:
        raise ValueError("small_random is for small graphs")
    u = (draws >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    sel = u < p
    return EdgeList(n, iu[sel].astype(np.int32), ju[sel].astype(np.int32), f"gnp{n}_{p}_s{seed}")


def _mean_degree_note(g: EdgeList) -> float:
    return 2.0 * g.n_in / max(g.n, 1) if g.n else math.nan
