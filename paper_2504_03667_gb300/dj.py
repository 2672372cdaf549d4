"""Python binding of include/dj.h: same names, argument marshalling only.

Every computation happens in libdj.so's CUDA kernels; this module converts
Python / numpy / torch arguments to the C types and raises DjError on a
negative status.  There is no fallback: if libdj.so is missing or cannot be
loaded, importing the binding raises.

Device buffers are passed as torch CUDA tensors (or raw integer device
addresses); streams as torch.cuda.Stream, an integer cudaStream_t, or None
for torch's current stream.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libdj.so")

DJ_OK = 0
DJ_EINVAL = -1
DJ_ENOMEM = -2
DJ_EOVERFLOW = -3
DJ_ECUDA = -4
DJ_ETIMEOUT = -5
DJ_EBUSY = -6
DJ_EUNSUPPORTED = -7
DJ_INF = 2**31 - 1

DJ_MODE_AUTO, DJ_MODE_PHASE, DJ_MODE_PLAIN = 0, 1, 2
DJ_ENGINE_AUTO, DJ_ENGINE_GRID, DJ_ENGINE_CLUSTER = 0, 1, 2
DJ_SETTLE_AUTO, DJ_SETTLE_OUT, DJ_SETTLE_OUT_IN, DJ_SETTLE_OUT_DYN_IN, DJ_SETTLE_DYN = 0, 1, 2, 3, 4
DJ_FORMAT_DENSE, DJ_FORMAT_CSR = 0, 1
DJ_COPIES_AUTO, DJ_COPIES_NARROW, DJ_COPIES_WIDE = 0, 1, 2
DJ_BATCH_ENGINE_AUTO, DJ_BATCH_ENGINE_CLUSTER, DJ_BATCH_ENGINE_LOCKSTEP = 0, 1, 2


class DjError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class dj_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("pitch", ctypes.c_int32), ("directed", ctypes.c_int32),
                ("min_weight", ctypes.c_int32), ("max_weight", ctypes.c_int32), ("device", ctypes.c_int32),
                ("matrix", ctypes.c_void_p), ("minout", ctypes.c_void_p), ("minin", ctypes.c_void_p),
                ("bytes", ctypes.c_uint64), ("entries", ctypes.c_uint64), ("format", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class dj_solve_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("engine", ctypes.c_int32), ("cluster_size", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("unroll", ctypes.c_int32),
                ("timeout_ns", ctypes.c_int64), ("debug_skip_cta", ctypes.c_int32),
                ("trace_cap", ctypes.c_int32), ("trace", ctypes.c_void_p), ("settle", ctypes.c_int32),
                ("live", ctypes.c_int32), ("rowsplit", ctypes.c_int32), ("rowpush", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class dj_batch_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("cluster_size", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("clusters", ctypes.c_int32), ("settle", ctypes.c_int32), ("copies", ctypes.c_int32),
                ("engine", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class dj_serve_opts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("max_slots", ctypes.c_int32), ("cluster_size", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("clusters", ctypes.c_int32), ("idle_timeout_ns", ctypes.c_int64),
                ("reserved", ctypes.c_int32 * 8)]


class dj_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("p50_us", ctypes.c_double), ("p90_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("mean_us", ctypes.c_double), ("solves_per_s", ctypes.c_double),
                ("resident_bytes", ctypes.c_uint64), ("kernel_launches", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 7)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_INT = ctypes.c_int

# name -> (restype, argtypes); mirrors include/dj.h
SIGNATURES = {
    "dj_last_error": (ctypes.c_char_p, []),
    "dj_status_string": (ctypes.c_char_p, [_INT]),
    "dj_version": (_INT, []),
    "dj_load_edges": (_INT, [_I32, _I64, _P, _P, _P, _INT, _U64, ctypes.POINTER(_P)]),
    "dj_load_edges_csr": (_INT, [_I32, _I64, _P, _P, _P, _INT, _U64, ctypes.POINTER(_P)]),
    "dj_load_dense": (_INT, [_I32, _P, _I64, _INT, _U64, ctypes.POINTER(_P)]),
    "dj_graph_upload": (_INT, [_P, _P, _I64, _U64]),
    "dj_graph_download": (_INT, [_P, _P, _I64, _U64]),
    "dj_graph_get_info": (_INT, [_P, ctypes.POINTER(dj_graph_info)]),
    "dj_graph_free": (_INT, [_P]),
    "dj_solve_opts_init": (None, [ctypes.POINTER(dj_solve_opts)]),
    "dj_sssp": (_INT, [_P, _I32, _P, _P, _U64]),
    "dj_sssp_ex": (_INT, [_P, _I32, _P, _P, ctypes.POINTER(dj_solve_opts), _U64]),
    "dj_sssp_host": (_INT, [_P, _I32, _P, _P, _U64]),
    "dj_sssp_noalloc": (_INT, [_P, _I32, _P, _P, _U64]),
    "dj_sssp_lc": (_INT, [_P, _I32, _P, _P, _U64]),
    "dj_sync": (_INT, [_U64]),
    "dj_last_phases": (_INT, []),
    "dj_sssp_batch": (_INT, [_P, _P, _I32, _P, _P, _U64]),
    "dj_batch_opts_init": (None, [ctypes.POINTER(dj_batch_opts)]),
    "dj_batch_create": (_INT, [_P, _P, _I32, _P, _P, ctypes.POINTER(dj_batch_opts), ctypes.POINTER(_P)]),
    "dj_batch_launch": (_INT, [_P, _U64]),
    "dj_batch_free": (_INT, [_P]),
    "dj_batch_autotune": (_INT, [_P, _U64, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                 ctypes.POINTER(ctypes.c_float)]),
    "dj_batch_get_engine": (_INT, [_P, ctypes.POINTER(_I32)]),
    "dj_tune_load": (_INT, [ctypes.c_char_p]),
    "dj_tune_save": (_INT, [ctypes.c_char_p]),
    "dj_tune_lookup": (_INT, [_I32, _U64, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "dj_serve_opts_init": (None, [ctypes.POINTER(dj_serve_opts)]),
    "dj_serve_create": (_INT, [ctypes.POINTER(dj_serve_opts), ctypes.POINTER(_P)]),
    "dj_serve_add_graph": (_INT, [_P, _P, ctypes.POINTER(_I32)]),
    "dj_serve_submit": (_INT, [_P, _I32, _I32, _P, _P, ctypes.POINTER(_U64)]),
    "dj_serve_poll": (_INT, [_P, _U64, ctypes.POINTER(_INT)]),
    "dj_serve_wait": (_INT, [_P, _U64, _I64]),
    "dj_serve_result": (_INT, [_P, _U64, _P, _P]),
    "dj_serve_stats_get": (_INT, [_P, ctypes.POINTER(dj_serve_stats)]),
    "dj_serve_destroy": (_INT, [_P]),
    "dj_serve": (_INT, [_P, _I32, _I64, _P, _P, _P, _P, _P, ctypes.POINTER(dj_serve_opts),
                        ctypes.POINTER(dj_serve_stats)]),
}

_lib = None


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load libdj.so (raises OSError if it is missing: no fallback exists)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"libdj.so not built at {p}; run __graft_entry__.build() (nvcc for sm_103a)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(rc: int) -> int:
    if rc != DJ_OK:
        msg = load_library().dj_last_error()
        raise DjError(rc, (msg or b"").decode() or load_library().dj_status_string(rc).decode())
    return rc


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _dptr(x) -> int:
    """Device address of a torch CUDA tensor (int32, contiguous) or a raw integer."""
    if isinstance(x, int):
        return x
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError("expected a CUDA tensor or a device address")
    if x.dtype != torch.int32 or not x.is_contiguous():
        raise TypeError("device buffers must be contiguous int32")
    return int(x.data_ptr())


def _host_i32(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a


class Graph:
    """Owner of a dj_graph* (device matrix); freed by free() or garbage collection."""

    def __init__(self, handle: int):
        self.handle = handle

    @property
    def info(self) -> dict:
        return dj_graph_get_info(self)

    @property
    def n(self) -> int:
        return self.info["n"]

    def free(self):
        if self.handle:
            load_library().dj_graph_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _gh(g) -> int:
    return g.handle if isinstance(g, Graph) else int(g)


# ---------------------------------------------------------------------- graphs

def dj_version() -> int:
    return load_library().dj_version()


def dj_load_edges(n: int, src, dst, w, directed: bool, stream=None) -> Graph:
    s, d, ww = _host_i32(src), _host_i32(dst), _host_i32(w)
    if not (s.shape == d.shape == ww.shape) or s.ndim != 1:
        raise ValueError("src, dst, w must be 1-D arrays of equal length")
    out = _P()
    _check(load_library().dj_load_edges(int(n), int(s.shape[0]), s.ctypes.data, d.ctypes.data, ww.ctypes.data,
                                        int(bool(directed)), _stream(stream), ctypes.byref(out)))
    return Graph(out.value)


def dj_load_edges_csr(n: int, src, dst, w, directed: bool, stream=None) -> Graph:
    """The same graph in compressed-row form only (no n x n matrix); dj_sssp solves it."""
    s, d, ww = _host_i32(src), _host_i32(dst), _host_i32(w)
    if not (s.shape == d.shape == ww.shape) or s.ndim != 1:
        raise ValueError("src, dst, w must be 1-D arrays of equal length")
    out = _P()
    _check(load_library().dj_load_edges_csr(int(n), int(s.shape[0]), s.ctypes.data, d.ctypes.data,
                                            ww.ctypes.data, int(bool(directed)), _stream(stream), ctypes.byref(out)))
    return Graph(out.value)


def dj_load_dense(W, stream=None) -> Graph:
    """W: an n x n int32 numpy array (host) or torch CUDA tensor (device)."""
    try:
        import torch
        is_dev = isinstance(W, torch.Tensor) and W.is_cuda
    except ImportError:  # pragma: no cover
        is_dev = False
    out = _P()
    if is_dev:
        n, ld = W.shape[0], W.stride(0)
        _check(load_library().dj_load_dense(int(n), _dptr(W), int(ld), 1, _stream(stream), ctypes.byref(out)))
    else:
        A = _host_i32(W)
        n, ld = A.shape[0], A.shape[1]
        _check(load_library().dj_load_dense(int(n), A.ctypes.data, int(ld), 0, _stream(stream), ctypes.byref(out)))
    return Graph(out.value)


def dj_graph_upload(g, W, stream=None):
    """Copy host matrix W (n x ld int32, ideally pinned: numpy or a pinned CPU tensor) into g."""
    if hasattr(W, "data_ptr"):
        ptr, ld = int(W.data_ptr()), int(W.stride(0))
    else:
        ptr, ld = int(W.ctypes.data), int(W.strides[0] // 4)
    _check(load_library().dj_graph_upload(_gh(g), ptr, ld, _stream(stream)))


def dj_graph_download(g, stream=None) -> np.ndarray:
    n = dj_graph_get_info(g)["n"]
    W = np.empty((n, n), dtype=np.int32)
    _check(load_library().dj_graph_download(_gh(g), W.ctypes.data, n, _stream(stream)))
    return W


def dj_graph_get_info(g) -> dict:
    info = dj_graph_info()
    _check(load_library().dj_graph_get_info(_gh(g), ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in info._fields_}


def dj_graph_free(g):
    if isinstance(g, Graph):
        g.free()
    else:
        _check(load_library().dj_graph_free(int(g)))


# ---------------------------------------------------------------------- solves

def make_solve_opts(mode=DJ_MODE_AUTO, engine=DJ_ENGINE_AUTO, cluster_size=0, threads=0, ctas_per_sm=0,
                    unroll=0, timeout_ns=0, debug_skip_cta=-1, trace=None, settle=0, live=0,
                    rowsplit=0, rowpush=0) -> dj_solve_opts:
    """trace: optional int64 CUDA tensor receiving the per-phase timeline.
    live: grid engine column filter (0 auto, -1 off, > 0 gather threshold in 4-column groups).
    rowsplit: grid engine row-split phases (0 auto, -1 off, > 0 minimum settled candidates).
    rowpush: grid engine row-push phases (0 auto on sparse graphs, -1 off, > 0 minimum candidates)."""
    o = dj_solve_opts()
    load_library().dj_solve_opts_init(ctypes.byref(o))
    o.mode, o.engine, o.cluster_size, o.threads = mode, engine, cluster_size, threads
    o.ctas_per_sm, o.unroll, o.timeout_ns, o.debug_skip_cta = ctas_per_sm, unroll, timeout_ns, debug_skip_cta
    if trace is not None:
        o.trace, o.trace_cap = int(trace.data_ptr()), int(trace.numel())
    o.settle = settle
    o.live = live
    o.rowsplit = rowsplit
    o.rowpush = rowpush
    return o


def dj_sssp(g, source: int, dist, pred, stream=None):
    _check(load_library().dj_sssp(_gh(g), int(source), _dptr(dist), _dptr(pred), _stream(stream)))


def dj_sssp_ex(g, source: int, dist, pred, opts: Optional[dj_solve_opts] = None, stream=None):
    o = opts if opts is not None else make_solve_opts()
    _check(load_library().dj_sssp_ex(_gh(g), int(source), _dptr(dist), _dptr(pred), ctypes.byref(o),
                                     _stream(stream)))


def dj_sssp_host(g, source: int, dist_host=None, pred_host=None, stream=None):
    """Solve with HOST result buffers (numpy int32 or pinned CPU tensors); returns (dist, pred)."""
    n = dj_graph_get_info(g)["n"]
    if dist_host is None:
        dist_host = np.empty(n, dtype=np.int32)
    if pred_host is None:
        pred_host = np.empty(n, dtype=np.int32)

    def hp(a):
        return int(a.data_ptr()) if hasattr(a, "data_ptr") else int(a.ctypes.data)

    _check(load_library().dj_sssp_host(_gh(g), int(source), hp(dist_host), hp(pred_host), _stream(stream)))
    return dist_host, pred_host


def dj_sssp_noalloc(g, source: int, dist, pred, stream=None):
    """Solve without allocating device memory (fixed scratch array in the library)."""
    _check(load_library().dj_sssp_noalloc(_gh(g), int(source), _dptr(dist), _dptr(pred), _stream(stream)))


def dj_sssp_lc(g, source: int, dist, pred, stream=None):
    """Label-correcting solve (the paper's CUDA variant): exact dist, pred a shortest-path tree."""
    _check(load_library().dj_sssp_lc(_gh(g), int(source), _dptr(dist), _dptr(pred), _stream(stream)))


def dj_sync(stream=None):
    _check(load_library().dj_sync(_stream(stream)))


def dj_last_phases() -> int:
    return load_library().dj_last_phases()


def _ptr_array(items) -> ctypes.Array:
    arr = (_P * max(len(items), 1))()
    for i, x in enumerate(items):
        arr[i] = x
    return arr


def dj_sssp_batch(graphs: Sequence, sources, dists: Sequence, preds: Sequence, stream=None):
    k = len(graphs)
    g = _ptr_array([_gh(x) for x in graphs])
    s = _host_i32(sources)
    d = _ptr_array([_dptr(x) for x in dists])
    p = _ptr_array([_dptr(x) for x in preds])
    _check(load_library().dj_sssp_batch(ctypes.addressof(g), s.ctypes.data, k, ctypes.addressof(d),
                                        ctypes.addressof(p), _stream(stream)))


class Batch:
    def __init__(self, handle: int):
        self.handle = handle

    def free(self):
        if self.handle:
            load_library().dj_batch_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def dj_batch_create(graphs: Sequence, sources, dists: Sequence, preds: Sequence, mode=DJ_MODE_AUTO,
                    cluster_size=0, clusters=0, settle=DJ_SETTLE_AUTO, copies=0, engine=DJ_BATCH_ENGINE_AUTO) -> Batch:
    """copies: DJ_COPIES_AUTO (0), DJ_COPIES_NARROW (1) or DJ_COPIES_WIDE (2) ring copies.
    engine: DJ_BATCH_ENGINE_AUTO (0), _CLUSTER (1) or _LOCKSTEP (2)."""
    o = dj_batch_opts()
    load_library().dj_batch_opts_init(ctypes.byref(o))
    o.mode, o.cluster_size, o.clusters, o.settle, o.copies = mode, cluster_size, clusters, settle, copies
    o.engine = engine
    k = len(graphs)
    g = _ptr_array([_gh(x) for x in graphs])
    s = _host_i32(sources)
    d = _ptr_array([_dptr(x) for x in dists])
    p = _ptr_array([_dptr(x) for x in preds])
    out = _P()
    _check(load_library().dj_batch_create(ctypes.addressof(g), s.ctypes.data, k, ctypes.addressof(d),
                                          ctypes.addressof(p), ctypes.byref(o), ctypes.byref(out)))
    return Batch(out.value)


def dj_batch_launch(b: Batch, stream=None):
    _check(load_library().dj_batch_launch(b.handle, _stream(stream)))


def dj_batch_free(b: Batch):
    b.free()


def dj_batch_autotune(b: Batch, stream=None) -> dict:
    c, t, ms = _I32(), _I32(), ctypes.c_float()
    _check(load_library().dj_batch_autotune(b.handle, _stream(stream), ctypes.byref(c), ctypes.byref(t),
                                            ctypes.byref(ms)))
    return {"cluster_size": c.value, "threads": t.value, "ms": ms.value, "engine": dj_batch_get_engine(b)}


def dj_batch_get_engine(b: Batch) -> str:
    e = _I32()
    _check(load_library().dj_batch_get_engine(b.handle, ctypes.byref(e)))
    return "lockstep" if e.value == DJ_BATCH_ENGINE_LOCKSTEP else "cluster"


def dj_tune_load(path: str):
    _check(load_library().dj_tune_load(os.fsencode(path)))


def dj_tune_save(path: str):
    _check(load_library().dj_tune_save(os.fsencode(path)))


def dj_tune_lookup(n: int, entries: int, num_sms: int) -> Optional[dict]:
    """The autotuner's entry for (n, finite entries, SM count), or None."""
    e, c = _I32(), _I32()
    rc = load_library().dj_tune_lookup(int(n), int(entries), int(num_sms), ctypes.byref(e), ctypes.byref(c))
    if rc == DJ_EINVAL:
        return None
    _check(rc)
    return {"engine": "lockstep" if e.value == DJ_BATCH_ENGINE_LOCKSTEP else "cluster", "cluster_size": c.value}


# ---------------------------------------------------------------------- serving

def make_serve_opts(hbm_budget=0, max_slots=0, cluster_size=0, threads=0, clusters=0,
                    idle_timeout_ns=0) -> dj_serve_opts:
    o = dj_serve_opts()
    load_library().dj_serve_opts_init(ctypes.byref(o))
    o.hbm_budget, o.max_slots, o.cluster_size = hbm_budget, max_slots, cluster_size
    o.threads, o.clusters, o.idle_timeout_ns = threads, clusters, idle_timeout_ns
    return o


class Server:
    def __init__(self, handle: int):
        self.handle = handle

    def destroy(self):
        if self.handle:
            load_library().dj_serve_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def dj_serve_create(opts: Optional[dj_serve_opts] = None) -> Server:
    o = opts if opts is not None else make_serve_opts()
    out = _P()
    _check(load_library().dj_serve_create(ctypes.byref(o), ctypes.byref(out)))
    return Server(out.value)


def dj_serve_add_graph(s: Server, g) -> int:
    gid = _I32()
    _check(load_library().dj_serve_add_graph(s.handle, _gh(g), ctypes.byref(gid)))
    return gid.value


def dj_serve_submit(s: Server, graph_id: int, source: int, dist=None, pred=None) -> Optional[int]:
    """Returns the ticket, or None if the server is busy (DJ_EBUSY)."""
    t = _U64()
    rc = load_library().dj_serve_submit(s.handle, int(graph_id), int(source), _dptr(dist) if dist is not None else None,
                                        _dptr(pred) if pred is not None else None, ctypes.byref(t))
    if rc == DJ_EBUSY:
        return None
    _check(rc)
    return t.value


def dj_serve_poll(s: Server, ticket: int) -> bool:
    d = _INT()
    _check(load_library().dj_serve_poll(s.handle, int(ticket), ctypes.byref(d)))
    return bool(d.value)


def dj_serve_wait(s: Server, ticket: int, timeout_ns: int = 10_000_000_000):
    _check(load_library().dj_serve_wait(s.handle, int(ticket), int(timeout_ns)))


def dj_serve_result(s: Server, ticket: int, n: int):
    d = np.empty(n, dtype=np.int32)
    p = np.empty(n, dtype=np.int32)
    _check(load_library().dj_serve_result(s.handle, int(ticket), d.ctypes.data, p.ctypes.data))
    return d, p


def dj_serve_stats_get(s: Server) -> dict:
    st = dj_serve_stats()
    _check(load_library().dj_serve_stats_get(s.handle, ctypes.byref(st)))
    return st.as_dict()


def dj_serve_destroy(s: Server):
    s.destroy()


def dj_serve(graphs: Sequence, req_graph, req_source, arrival_s, out_dist=None, out_pred=None,
             opts: Optional[dj_serve_opts] = None) -> dict:
    o = opts if opts is not None else make_serve_opts()
    G = _ptr_array([_gh(x) for x in graphs])
    rg = _host_i32(req_graph)
    rs = _host_i32(req_source)
    at = np.ascontiguousarray(arrival_s, dtype=np.float64)
    R = rg.shape[0]
    od = _ptr_array([_dptr(x) if x is not None else 0 for x in out_dist]) if out_dist is not None else None
    op = _ptr_array([_dptr(x) if x is not None else 0 for x in out_pred]) if out_pred is not None else None
    st = dj_serve_stats()
    _check(load_library().dj_serve(ctypes.addressof(G), len(graphs), R, rg.ctypes.data, rs.ctypes.data, at.ctypes.data,
                                   ctypes.addressof(od) if od is not None else None,
                                   ctypes.addressof(op) if op is not None else None, ctypes.byref(o),
                                   ctypes.byref(st)))
    return st.as_dict()
