"""Python binding of libtruss.so: GB300 truss decomposition (PKT).

Argument marshalling only.  Every step of the computation runs in the CUDA
kernels behind the C ABI declared in ``include/truss.h``; PyTorch provides
device memory and streams.  There is no CPU fallback: importing this module
without a built ``libtruss.so`` raises, and every call needs a CUDA device.

Typical use::

    import torch, paper_1707_02000_gb300 as pkt
    g = pkt.build_csr(src_cuda_int32, dst_cuda_int32, n)
    tau = g.decompose()            # int32[m] on the GPU, canonical edge order
    u, v = g.edge_list()           # the canonical edges, input labels
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtruss.so")

OK = 0
EINVAL, ENOMEM, ECUDA, ETIMEOUT, EOVERFLOW, EBADGRAPH, EDEVICE, ENOTSUP, ETOOBIG = -1, -2, -3, -4, -5, -6, -7, -8, -9
NOALLOC_MAX_VERTICES = 1 << 22
DEGREE_ORDER = 1
OFFSETS64 = 2
CORE_ORDER = 4
LOCALITY_ORDER = 8
LOOP_PLAIN, LOOP_PERSISTENT, LOOP_PERSISTENT_LAT, LOOP_PERSISTENT_OCC, LOOP_GRAPH = 0, 1, 2, 3, 4
VAR_AUTO, VAR_THREAD, VAR_GROUP, VAR_WARP, VAR_LEARNED = -1, 0, 1, 2, 3
SCHED_FEATURES, SCHED_VARIANTS, SCHED_PARAMS, TUNE_CLASSES = 5, 3, 1357, 128
PROCESSED, IN_CURR = 1, 2

# Every symbol include/truss.h declares (checked by the tests).
EXPORTS = (
    "truss_strerror", "truss_build_csr", "truss_free", "truss_num_edges", "truss_num_vertices",
    "truss_edge_list", "truss_csr_copy", "truss_support", "truss_default_opts", "truss_decompose",
    "truss_peel_sublevel", "truss_decompose_host", "truss_sync", "truss_support_noalloc",
    "truss_decompose_batch", "truss_sched_features", "truss_sched_init", "truss_sched_grad",
    "truss_sched_train", "truss_sched_predict", "truss_autotune", "truss_ktruss_components",
    "truss_triangle_count", "truss_support_ros", "truss_decompose_local", "truss_pool_keep",
)


class TrussError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})")


class Opts(ctypes.Structure):
    _fields_ = [("loop", ctypes.c_int32), ("variant", ctypes.c_int32), ("sync", ctypes.c_int32),
                ("level_jump", ctypes.c_int32), ("timeout_ns", ctypes.c_int64),
                ("h_sub_level", ctypes.POINTER(ctypes.c_int32)), ("h_sub_size", ctypes.POINTER(ctypes.c_int64)),
                ("max_sub", ctypes.c_int64), ("d_peel_step", ctypes.c_void_p),
                ("h_trace", ctypes.c_void_p), ("sched_params", ctypes.c_void_p),
                ("tune_table", ctypes.c_void_p), ("compact", ctypes.c_int32), ("max_level", ctypes.c_int32),
                ("h_level_edges", ctypes.c_void_p), ("h_level_ns", ctypes.c_void_p)]


# truss_sublevel_trace, one record per sub-level
TRACE_DTYPE = np.dtype([("level", "<i4"), ("group", "<i4"), ("n_light", "<i4"), ("n_heavy", "<i4"),
                        ("n_chunks", "<u4"), ("dmax", "<i4"), ("dsum", "<i8"), ("todo", "<i8"), ("t_ns", "<i8"),
                        ("scan_ns", "<i8")])


class Stats(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("sublevels", ctypes.c_int64), ("scans", ctypes.c_int64),
                ("triangles", ctypes.c_int64), ("t_max", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("ms_support", ctypes.c_float), ("ms_peel", ctypes.c_float), ("launches", ctypes.c_int64),
                ("wedges_up", ctypes.c_int64), ("dmin_sum", ctypes.c_int64), ("scanned", ctypes.c_int64),
                ("grid_blocks", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("max_support", ctypes.c_int32), ("compactions", ctypes.c_int32), ("walked", ctypes.c_int64),
                ("compacted_slots", ctypes.c_int64), ("support_walked", ctypes.c_int64),
                ("support_hub_probes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _declare(lib):
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    pp = ctypes.POINTER(ctypes.c_void_p)
    lib.truss_strerror.argtypes = [ctypes.c_int]
    lib.truss_strerror.restype = ctypes.c_char_p
    lib.truss_build_csr.argtypes = [vp, vp, i64, i32, u32, vp, pp]
    lib.truss_free.argtypes = [vp]
    lib.truss_free.restype = None
    lib.truss_num_edges.argtypes = [vp, ctypes.POINTER(i64)]
    lib.truss_num_vertices.argtypes = [vp, ctypes.POINTER(i32)]
    lib.truss_edge_list.argtypes = [vp, vp, vp, vp]
    lib.truss_csr_copy.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.truss_support.argtypes = [vp, vp, vp]
    lib.truss_support_ros.argtypes = [vp, vp, vp]
    lib.truss_pool_keep.argtypes = [i64]
    lib.truss_decompose_local.argtypes = [vp, vp, i64, ctypes.POINTER(i64), ctypes.POINTER(i64), vp]
    lib.truss_ktruss_components.argtypes = [vp, vp, i32, vp, vp, vp]
    lib.truss_triangle_count.argtypes = [vp, vp, vp]
    lib.truss_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.truss_default_opts.restype = None
    lib.truss_decompose.argtypes = [vp, vp, ctypes.POINTER(Opts), ctypes.POINTER(Stats), vp]
    lib.truss_peel_sublevel.argtypes = [vp, vp, vp, vp, i64, i32, vp, ctypes.POINTER(i64), i32, vp]
    lib.truss_decompose_host.argtypes = [vp, vp, i64, i32, u32, vp, i64, ctypes.POINTER(i64),
                                         ctypes.POINTER(Opts), ctypes.POINTER(Stats), vp]
    lib.truss_sync.argtypes = [vp, vp]
    lib.truss_support_noalloc.argtypes = [vp, vp, vp, i32, i64, vp, vp]
    lib.truss_decompose_batch.argtypes = [vp, vp, vp, vp, i32, u32, vp, i64, vp, ctypes.POINTER(Opts),
                                          ctypes.POINTER(Stats), vp]
    lib.truss_sched_features.argtypes = [vp, i64, vp]
    lib.truss_sched_features.restype = None
    lib.truss_sched_init.argtypes = [vp, ctypes.c_uint64, vp]
    lib.truss_sched_grad.argtypes = [vp, vp, vp, i64, vp, ctypes.POINTER(ctypes.c_float), vp]
    lib.truss_sched_train.argtypes = [vp, vp, vp, i64, i32, ctypes.c_float, ctypes.POINTER(ctypes.c_float), vp]
    lib.truss_sched_predict.argtypes = [vp, vp, i64, vp, vp]
    lib.truss_autotune.argtypes = [vp, vp, i32, vp]
    for name in EXPORTS:
        if name not in ("truss_strerror", "truss_free", "truss_default_opts", "truss_sched_features"):
            getattr(lib, name).restype = ctypes.c_int
    return lib


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
                      " (there is no CPU fallback)")
_lib = _declare(ctypes.CDLL(LIB_PATH))


def library():
    """The loaded ctypes library (for tests of the raw C ABI)."""
    return _lib


def strerror(status: int) -> str:
    return _lib.truss_strerror(status).decode()


def _check(rc: int, what: str):
    if rc != OK:
        raise TrussError(rc, what)


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    assert t.is_cuda and t.is_contiguous(), "expects a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


def default_opts(**kw) -> Opts:
    o = Opts()
    _lib.truss_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _policy(o: Opts, sched_params, tune_table):
    """Sets the learned model (device float32[SCHED_PARAMS]) and the tuned
    table (int8[TUNE_CLASSES]) on ``o``; returns the table array, which the
    caller keeps alive for the call."""
    if sched_params is not None:
        assert sched_params.numel() == SCHED_PARAMS and str(sched_params.dtype) == "torch.float32"
        assert sched_params.is_cuda and sched_params.is_contiguous()
        o.sched_params = sched_params.data_ptr()
    if tune_table is not None:
        tune_table = np.ascontiguousarray(tune_table, np.int8)
        assert tune_table.shape == (TUNE_CLASSES,)
        o.tune_table = tune_table.ctypes.data
    return tune_table


class Graph:
    """A device-resident graph handle (owns its device memory)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        m = ctypes.c_int64()
        n = ctypes.c_int32()
        _check(_lib.truss_num_edges(self._h, ctypes.byref(m)), "truss_num_edges")
        _check(_lib.truss_num_vertices(self._h, ctypes.byref(n)), "truss_num_vertices")
        self.m = int(m.value)
        self.n = int(n.value)

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            _lib.truss_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def _empty(self, k):
        torch = _torch()
        return torch.empty(max(k, 1), dtype=torch.int32, device="cuda")[:k]

    def edge_list(self, stream=None):
        u, v = self._empty(self.m), self._empty(self.m)
        _check(_lib.truss_edge_list(self._h, _dptr(u) if self.m else None, _dptr(v) if self.m else None,
                                    _stream(stream)), "truss_edge_list")
        return u, v

    def csr(self, stream=None):
        torch = _torch()
        rp = torch.empty(self.n + 1, dtype=torch.int64, device="cuda")
        eo = torch.empty(max(self.n, 1), dtype=torch.int64, device="cuda")
        col, eid = self._empty(2 * self.m), self._empty(2 * self.m)
        order = self._empty(self.n)
        _check(_lib.truss_csr_copy(self._h, _dptr(rp), _dptr(col) if self.m else None,
                                   _dptr(eid) if self.m else None, _dptr(eo), _dptr(order) if self.n else None,
                                   _stream(stream)), "truss_csr_copy")
        return rp, col, eid, eo[: self.n], order

    def support(self, out=None, stream=None):
        out = self._empty(self.m) if out is None else out
        _check(_lib.truss_support(self._h, _dptr(out) if self.m else None, _stream(stream)), "truss_support")
        return out

    def decompose(self, out=None, loop=LOOP_PERSISTENT, variant=VAR_AUTO, sync=True, level_jump=True,
                  timeout_ns=10_000_000_000, record=False, max_sub=1 << 20, stream=None, stats=False,
                  peel_step=None, trace=False, sched_params=None, tune_table=None, compact=-1,
                  level_hist=False, max_level=1 << 16):
        """Trussness (int32[m], canonical order).  With ``record`` also
        returns the (level, |curr|) of every sub-level; with ``trace`` a
        structured array (TRACE_DTYPE) with one record per sub-level; with
        ``level_hist`` a pair of int64 arrays (edges peeled, device ns) per
        support level 0..t_max-2; with ``stats`` a dict of run statistics;
        ``peel_step`` (a CUDA int32[m] tensor) receives the sub-level each
        edge was peeled in; ``compact`` selects row compaction (-1 automatic,
        0 off, 1 on)."""
        out = self._empty(self.m) if out is None else out
        o = default_opts(loop=loop, variant=variant, sync=int(bool(sync or record or trace or level_hist)),
                         level_jump=int(bool(level_jump)), timeout_ns=timeout_ns, compact=compact)
        hl = hn = None
        if level_hist:
            hl = np.zeros(max_level, np.int64)
            hn = np.zeros(max_level, np.int64)
            o.h_level_edges = hl.ctypes.data
            o.h_level_ns = hn.ctypes.data
            o.max_level = max_level
        tune_table = _policy(o, sched_params, tune_table)
        tr = None
        if trace:
            tr = np.zeros(max_sub, TRACE_DTYPE)
            o.h_trace = tr.ctypes.data
            o.max_sub = max_sub
        if peel_step is not None and self.m:
            o.d_peel_step = peel_step.data_ptr()
        rl = rs = None
        if record:
            rl = np.zeros(max_sub, np.int32)
            rs = np.zeros(max_sub, np.int64)
            o.h_sub_level = rl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            o.h_sub_size = rs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
            o.max_sub = max_sub
        st = Stats()
        _check(_lib.truss_decompose(self._h, _dptr(out) if self.m else None, ctypes.byref(o),
                                    ctypes.byref(st), _stream(stream)), "truss_decompose")
        res = [out]
        if record:
            k = min(int(st.sublevels), max_sub)
            res.append((rl[:k].copy(), rs[:k].copy()))
        if trace:
            res.append(tr[: min(int(st.sublevels), max_sub)].copy())
        if level_hist:
            k = min(max(int(st.t_max) - 1, 0), max_level)
            res.append((hl[:k].copy(), hn[:k].copy()))
        if stats:
            res.append(st.as_dict())
        return res[0] if len(res) == 1 else tuple(res)

    def peel_sublevel(self, S, flags, curr, l, variant=VAR_AUTO, stream=None):
        """One ProcessSubLevel on a caller-set state (device tensors, canonical
        order); S and flags are updated in place.  Returns next (device)."""
        nxt = self._empty(self.m)
        k = ctypes.c_int64()
        _check(_lib.truss_peel_sublevel(self._h, _dptr(S) if self.m else None, _dptr(flags) if self.m else None,
                                        _dptr(curr) if curr.numel() else None, curr.numel(), l,
                                        _dptr(nxt) if self.m else None, ctypes.byref(k), variant,
                                        _stream(stream)), "truss_peel_sublevel")
        return nxt[: k.value]

    def support_ros(self, out=None, stream=None):
        """S(e) by the edge-centric scheme of Algorithm 2 (canonical order)."""
        out = self._empty(self.m) if out is None else out
        _check(_lib.truss_support_ros(self._h, _dptr(out) if self.m else None, _stream(stream)), "truss_support_ros")
        return out

    def decompose_local(self, out=None, max_sweeps: int = 0, stats: bool = False, stream=None):
        """Trussness by the asynchronous local h-index iteration (canonical
        order); with ``stats`` also {"sweeps", "updates"}."""
        out = self._empty(self.m) if out is None else out
        sw, up = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.truss_decompose_local(self._h, _dptr(out) if self.m else None, max_sweeps, ctypes.byref(sw),
                                          ctypes.byref(up), _stream(stream)), "truss_decompose_local")
        return (out, {"sweeps": int(sw.value), "updates": int(up.value)}) if stats else out

    def triangle_count(self, stream=None) -> int:
        """Number of triangles (each counted once)."""
        t = ctypes.c_int64()
        _check(_lib.truss_triangle_count(self._h, ctypes.byref(t), _stream(stream)), "truss_triangle_count")
        return int(t.value)

    def ktruss_components(self, tau, k: int, stream=None):
        """The k-trusses: per edge (canonical order, CUDA int32 tensor) the
        smallest input vertex label of its component among the edges of
        trussness >= k, or -1; and the number of components."""
        comp = self._empty(self.m)
        nc = ctypes.c_int64()
        _check(_lib.truss_ktruss_components(self._h, _dptr(tau) if self.m else None, k,
                                            _dptr(comp) if self.m else None, ctypes.byref(nc), _stream(stream)),
               "truss_ktruss_components")
        return comp, int(nc.value)

    def autotune(self, repeats: int = 1, stream=None):
        """Autotuned variant table (int8[TUNE_CLASSES]) for this graph."""
        t = np.full(TUNE_CLASSES, -1, np.int8)
        _check(_lib.truss_autotune(self._h, t.ctypes.data_as(ctypes.c_void_p), repeats, _stream(stream)),
               "truss_autotune")
        return t

    def sync(self, stream=None):
        _check(_lib.truss_sync(self._h, _stream(stream)), "truss_sync")


def build_csr(src, dst, n: int, degree_order: bool = True, offsets64: bool = False, core_order: bool = False,
              locality_order: bool = False, stream=None) -> Graph:
    """Device graph from CUDA int32 tensors ``src``, ``dst`` (raw pairs);
    ``core_order`` relabels in a degeneracy (k-core) order instead of by
    degree, ``locality_order`` in a reverse Cuthill-McKee order (for
    mesh-like graphs)."""
    assert src.dtype == dst.dtype and str(src.dtype) == "torch.int32" and src.numel() == dst.numel()
    flags = ((DEGREE_ORDER if degree_order else 0) | (OFFSETS64 if offsets64 else 0)
             | (CORE_ORDER if core_order else 0) | (LOCALITY_ORDER if locality_order else 0))
    h = ctypes.c_void_p()
    k = src.numel()
    _check(_lib.truss_build_csr(_dptr(src) if k else None, _dptr(dst) if k else None, k, n, flags,
                                _stream(stream), ctypes.byref(h)), "truss_build_csr")
    return Graph(h)


def pool_keep(nbytes: int):
    """Bytes of freed device memory the library's stream-ordered pool keeps
    for reuse on the current device (truss_pool_keep)."""
    _check(_lib.truss_pool_keep(int(nbytes)), "truss_pool_keep")


def decompose_host(src: np.ndarray, dst: np.ndarray, n: int, degree_order: bool = True, offsets64: bool = False,
                   out: np.ndarray | None = None, loop=LOOP_PERSISTENT, variant=VAR_AUTO, stream=None,
                   sched_params=None, tune_table=None, compact=-1):
    """Host arrays in, host trussness out (canonical order): the C ABI's
    truss_decompose_host.  ``src``/``dst`` should be pinned for speed."""
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    cap = src.shape[0] if out is None else out.shape[0]
    out = np.empty(max(cap, 1), np.int32) if out is None else out
    flags = (DEGREE_ORDER if degree_order else 0) | (OFFSETS64 if offsets64 else 0)
    m = ctypes.c_int64()
    o = default_opts(loop=loop, variant=variant, sync=1, compact=compact)
    tune_table = _policy(o, sched_params, tune_table)
    st = Stats()
    _check(_lib.truss_decompose_host(src.ctypes.data_as(ctypes.c_void_p), dst.ctypes.data_as(ctypes.c_void_p),
                                     src.shape[0], n, flags, out.ctypes.data_as(ctypes.c_void_p), cap,
                                     ctypes.byref(m), ctypes.byref(o), ctypes.byref(st), _stream(stream)),
           "truss_decompose_host")
    return out[: m.value], st.as_dict()


def decompose_batch(graphs, degree_order: bool = True, loop=LOOP_PERSISTENT, variant=VAR_AUTO, stream=None,
                    stats: bool = False, sched_params=None, tune_table=None, compact=-1):
    """Decompose many independent graphs (objects with ``n``, ``src``,
    ``dst``; ids local to each graph) in one run on the device.  Returns the
    list of per-graph trussness arrays (CUDA tensors, canonical order of
    each graph)."""
    torch = _torch()
    G = len(graphs)
    eoff = np.zeros(G + 1, np.int64)
    eoff[1:] = np.cumsum([int(g.src.shape[0]) for g in graphs])
    nverts = np.array([g.n for g in graphs], np.int32)
    src = torch.from_numpy(np.concatenate([g.src for g in graphs]).astype(np.int32) if G else np.zeros(0, np.int32))
    dst = torch.from_numpy(np.concatenate([g.dst for g in graphs]).astype(np.int32) if G else np.zeros(0, np.int32))
    src, dst = src.cuda(), dst.cuda()
    cap = int(eoff[-1])
    out = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
    moff = np.zeros(G + 1, np.int64)
    o = default_opts(loop=loop, variant=variant, sync=1, compact=compact)
    tune_table = _policy(o, sched_params, tune_table)
    st = Stats()
    _check(_lib.truss_decompose_batch(_dptr(src) if cap else None, _dptr(dst) if cap else None,
                                      eoff.ctypes.data_as(ctypes.c_void_p), nverts.ctypes.data_as(ctypes.c_void_p),
                                      G, (DEGREE_ORDER if degree_order else 0), _dptr(out), cap,
                                      moff.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o), ctypes.byref(st),
                                      _stream(stream)), "truss_decompose_batch")
    res = [out[moff[i]: moff[i + 1]] for i in range(G)]
    return (res, st.as_dict()) if stats else res


# ------------------------------------------------------- learned scheduler

def sched_features(trace_records) -> np.ndarray:
    """Features (float32[n][5]) of trace records (TRACE_DTYPE)."""
    tr = np.ascontiguousarray(trace_records, TRACE_DTYPE)
    x = np.zeros((tr.shape[0], SCHED_FEATURES), np.float32)
    _lib.truss_sched_features(tr.ctypes.data_as(ctypes.c_void_p), tr.shape[0], x.ctypes.data_as(ctypes.c_void_p))
    return x


def sched_init(seed: int = 0, stream=None):
    torch = _torch()
    p = torch.empty(SCHED_PARAMS, dtype=torch.float32, device="cuda")
    _check(_lib.truss_sched_init(_dptr(p), seed, _stream(stream)), "truss_sched_init")
    return p


def sched_grad(params, x, y, stream=None):
    """(loss, gradient) of the scheduler's MSE on device tensors x [n,5], y [n,3]."""
    torch = _torch()
    g = torch.empty(SCHED_PARAMS, dtype=torch.float32, device="cuda")
    loss = ctypes.c_float()
    _check(_lib.truss_sched_grad(_dptr(params), _dptr(x), _dptr(y), x.shape[0], _dptr(g), ctypes.byref(loss),
                                 _stream(stream)), "truss_sched_grad")
    return float(loss.value), g


def sched_train(params, x, y, epochs: int = 2000, lr: float = 3e-3, stream=None) -> float:
    loss = ctypes.c_float()
    _check(_lib.truss_sched_train(_dptr(params), _dptr(x), _dptr(y), x.shape[0], epochs, lr, ctypes.byref(loss),
                                  _stream(stream)), "truss_sched_train")
    return float(loss.value)


def sched_predict(params, x, stream=None):
    torch = _torch()
    out = torch.empty((x.shape[0], SCHED_VARIANTS), dtype=torch.float32, device="cuda")
    _check(_lib.truss_sched_predict(_dptr(params), _dptr(x), x.shape[0], _dptr(out), _stream(stream)),
           "truss_sched_predict")
    return out


def sched_dataset(graph: "Graph", repeats: int = 1):
    """Training data the method generates itself: decompose ``graph`` under
    each light-edge variant with tracing; every sub-level gives one sample
    (features, log2 time of each variant).  Only sub-levels with light edges
    (where the variant acts) are kept.  Returns (x [n,5], y [n,3]) numpy."""
    traces = []
    for v in (VAR_THREAD, VAR_GROUP, VAR_WARP):
        runs = []
        for _ in range(repeats):
            _, tr = graph.decompose(loop=LOOP_PERSISTENT, variant=v, trace=True)
            runs.append(tr)
        t = np.stack([r["t_ns"] for r in runs]).mean(0)
        traces.append((runs[0], t))
    base = traces[-1][0]
    keep = base["n_light"] > 0
    x = sched_features(base[keep])
    y = np.log2(np.stack([t[keep] for _, t in traces], 1).astype(np.float64) + 1.0).astype(np.float32)
    return x, y
