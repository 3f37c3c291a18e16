"""Python binding of libmce_gb300 (argument marshalling only).

Every step of the computation runs in the CUDA library; this module converts
arguments (torch CUDA tensors for device buffers, numpy arrays for host
buffers) and mirrors the C structs of include/mce.h.  There is no CPU
fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

MCE_OK, MCE_EINVAL, MCE_ENOMEM, MCE_EOVERFLOW, MCE_EBUDGET, MCE_ETIMEOUT, MCE_ECUDA, MCE_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
RANK_DEGREE, RANK_DEGEN, RANK_TRIANGLE, RANK_LEARNED, RANK_USER = 0, 1, 2, 3, 4
RANKS = {"degree": RANK_DEGREE, "degen": RANK_DEGEN, "triangle": RANK_TRIANGLE, "learned": RANK_LEARNED,
         "user": RANK_USER}
HIST_CAP = 1024

_lock = threading.Lock()
_lib = None


class MceError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [
        ("rank_kind", ctypes.c_int32),
        ("user_rank", ctypes.c_void_p),
        ("model", ctypes.c_void_p),
        ("node_budget", ctypes.c_uint64),
        ("hash_seed", ctypes.c_uint64),
        ("stream", ctypes.c_void_p),
        ("list_off", ctypes.c_void_p),
        ("list_vtx", ctypes.c_void_p),
        ("list_max_cliques", ctypes.c_int64),
        ("list_max_words", ctypes.c_int64),
        ("pv_count", ctypes.c_void_p),
        ("pv_hash", ctypes.c_void_p),
        ("pv_nodes", ctypes.c_void_p),
        ("split", ctypes.c_int32),
        ("split_nodes", ctypes.c_uint32),
        ("order_by_model", ctypes.c_int32),
        ("warps_per_block", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("shared_words", ctypes.c_int32),
        ("time_limit_ms", ctypes.c_uint32),
        ("subset", ctypes.c_void_p),
        ("subset_len", ctypes.c_int64),
        ("subset_on_host", ctypes.c_int32),
        ("subproblem_budget", ctypes.c_uint64),
        ("queue_capacity", ctypes.c_int32),
        ("warp_small_search", ctypes.c_int32),
        ("whole_graph", ctypes.c_int32),
        ("sm_limit", ctypes.c_int32),
        ("lane_search_words", ctypes.c_int32),
        ("split_model", ctypes.c_void_p),
        ("heavy_nodes", ctypes.c_uint32),
        ("heavy_split_nodes", ctypes.c_uint32),
        ("lane_hold_waiting", ctypes.c_uint32),
    ]


class ResultC(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_uint64),
        ("hash", ctypes.c_uint64),
        ("tree_nodes", ctypes.c_uint64),
        ("hist_len", ctypes.c_int32),
        ("complete", ctypes.c_int32),
        ("hist", ctypes.c_uint64 * HIST_CAP),
        ("list_cliques", ctypes.c_int64),
        ("list_words", ctypes.c_int64),
        ("tasks_split", ctypes.c_uint64),
        ("subproblems", ctypes.c_int32),
        ("ms_rank", ctypes.c_float),
        ("ms_enum", ctypes.c_float),
        ("ms_search", ctypes.c_float),
        ("word_ops", ctypes.c_uint64),
        ("incomplete", ctypes.c_int64),
        ("stats", ctypes.c_uint64 * 8),
    ]


class DeltaC(ctypes.Structure):
    _fields_ = [
        ("applied", ctypes.c_int64),
        ("dropped", ctypes.c_int64),
        ("new_count", ctypes.c_uint64),
        ("new_hash", ctypes.c_uint64),
        ("sub_count", ctypes.c_uint64),
        ("sub_hash", ctypes.c_uint64),
        ("new_hist_len", ctypes.c_int32),
        ("sub_hist_len", ctypes.c_int32),
        ("new_hist", ctypes.c_uint64 * HIST_CAP),
        ("sub_hist", ctypes.c_uint64 * HIST_CAP),
        ("alive", ctypes.c_uint64),
        ("ms", ctypes.c_float),
    ]


EXEC_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_int64, ctypes.POINTER(DeltaC))


class ServerOpts(ctypes.Structure):
    _fields_ = [
        ("slots", ctypes.c_int32),
        ("mem_budget", ctypes.c_uint64),
        ("mem_fixed", ctypes.c_uint64),
        ("execute", EXEC_FN),
        ("execute_ctx", ctypes.c_void_p),
    ]


class RequestInfoC(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_int64),
        ("tenant", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("edges", ctypes.c_int64),
        ("arrival_ms", ctypes.c_double),
        ("admit_ms", ctypes.c_double),
        ("done_ms", ctypes.c_double),
        ("reserved", ctypes.c_uint64),
        ("delta", DeltaC),
    ]


class ServerStatsC(ctypes.Structure):
    _fields_ = [
        ("completed", ctypes.c_int64),
        ("failed", ctypes.c_int64),
        ("edges", ctypes.c_int64),
        ("applied", ctypes.c_int64),
        ("new_cliques", ctypes.c_uint64),
        ("subsumed_cliques", ctypes.c_uint64),
        ("p50_ms", ctypes.c_double),
        ("p99_ms", ctypes.c_double),
        ("max_ms", ctypes.c_double),
        ("wait_p50_ms", ctypes.c_double),
        ("wait_p99_ms", ctypes.c_double),
        ("span_ms", ctypes.c_double),
        ("edges_per_s", ctypes.c_double),
        ("max_in_flight", ctypes.c_int32),
        ("peak_reserved", ctypes.c_uint64),
        ("mem_budget", ctypes.c_uint64),
    ]


# (name, argtypes, restype) of every exported symbol of include/mce.h
_vp, _i32, _i64, _u64, _f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float
_P = ctypes.POINTER
SIGNATURES = {
    "mce_strerror": ([_i32], ctypes.c_char_p),
    "mce_last_error": ([], ctypes.c_char_p),
    "mce_opts_init": ([_P(Opts)], None),
    "mce_kernel_launches": ([], _u64),
    "mce_debug_fail_alloc": ([_i64], None),
    "mce_graph_create": ([_vp, _vp, _i64, _i32, _i32, _vp, _P(_vp)], _i32),
    "mce_graph_from_csr": ([_vp, _vp, _i32, _i64, _i32, _vp, _P(_vp)], _i32),
    "mce_graph_csr": ([_vp, _P(_i32), _P(_i64), _P(_vp), _P(_vp)], _i32),
    "mce_graph_copy_csr": ([_vp, _vp, _vp, _i32, _vp], _i32),
    "mce_graph_free": ([_vp], None),
    "mce_vertex_key": ([_vp, _i32, _vp, _vp], _i32),
    "mce_rank": ([_vp, _P(Opts), _vp], _i32),
    "mce_enumerate": ([_vp, _P(Opts), _P(ResultC)], _i32),
    "mce_features": ([_vp, _vp, _vp], _i32),
    "mce_features_kind": ([_vp, _i32, _vp, _vp], _i32),
    "mce_model_set_features": ([_vp, _i32], _i32),
    "mce_model_create": ([_i32, _u64, _P(_vp)], _i32),
    "mce_model_free": ([_vp], None),
    "mce_model_num_params": ([_vp], _i64),
    "mce_model_get": ([_vp, _vp], _i32),
    "mce_model_set": ([_vp, _vp], _i32),
    "mce_model_loss_grad": ([_vp, _vp, _vp, _i32, _vp, _P(_f32), _vp], _i32),
    "mce_model_train": ([_vp, _vp, _vp, _i32, _i32, _i32, _f32, _u64, _vp, _P(_f32)], _i32),
    "mce_model_predict": ([_vp, _vp, _i32, _i32, _vp, _vp], _i32),
    "mce_enumerate_batched": ([_vp, _vp, _i32, _P(Opts), _vp, _vp, _vp, _P(ResultC)], _i32),
    "mce_batched_create": ([_vp, _vp, _i32, _P(Opts), _P(_vp)], _i32),
    "mce_batched_run": ([_vp, _vp], _i32),
    "mce_batched_read": ([_vp, _vp, _vp, _vp, _vp, _P(ResultC)], _i32),
    "mce_batched_tune": ([_vp, _vp, _u64, _i32, _P(_i32), _P(ctypes.c_uint32), _P(_i32)], _i32),
    "mce_batched_free": ([_vp], None),
    "imce_open": ([_vp, _P(Opts), _P(_vp)], _i32),
    "imce_server_opts_init": ([_P(ServerOpts)], None),
    "imce_server_create": ([_P(ServerOpts), _P(_vp)], _i32),
    "imce_server_add_tenant": ([_vp, _vp, _P(Opts), _P(_i32)], _i32),
    "imce_server_submit": ([_vp, _i32, _vp, _vp, _i64, ctypes.c_double, _P(_i64)], _i32),
    "imce_server_wait": ([_vp, _i64, _P(RequestInfoC)], _i32),
    "imce_server_drain": ([_vp], _i32),
    "imce_server_reset_clock": ([_vp], _i32),
    "imce_server_stats_get": ([_vp, _P(ServerStatsC)], _i32),
    "imce_server_tenant": ([_vp, _i32], _vp),
    "imce_server_free": ([_vp], None),
    "imce_add_edges": ([_vp, _vp, _vp, _i64, _i32, _P(DeltaC)], _i32),
    "imce_remove_edges": ([_vp, _vp, _vp, _i64, _i32, _P(DeltaC)], _i32),
    "imce_graph": ([_vp], _vp),
    "imce_cliques": ([_vp, _vp, _vp, _i64, _i64, _P(_i64), _P(_i64)], _i32),
    "imce_close": ([_vp], None),
    "mce_enumerate_stream": ([_vp, _P(Opts), _i64, _vp, _vp, _P(ResultC)], _i32),
    "mce_enumerate_noalloc": ([_vp, _vp, _i32, _i64, _vp, _u64, _vp, _P(ResultC)], _i32),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise OSError(f"{path} missing: run __graft_entry__.build()")
                _build.build()
            lib = ctypes.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _check(st, what):
    if st == MCE_OK:
        return st
    lib = load()
    raise MceError(st, f"{what}: {lib.mce_strerror(st).decode()} ({lib.mce_last_error().decode()})")


def kernel_launches() -> int:
    return int(load().mce_kernel_launches())


def debug_fail_alloc(after: int):
    """Make the library's device allocation after `after` more successful ones
    fail (MCE_ENOMEM); negative disarms."""
    load().mce_debug_fail_alloc(int(after))


def _ptr(t):
    """Device or host address of a torch tensor / numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


@dataclass
class Result:
    count: int
    hash: int
    tree_nodes: int
    hist: np.ndarray
    complete: bool
    list_cliques: int
    list_words: int
    tasks_split: int
    subproblems: int
    ms_rank: float
    ms_enum: float
    ms_search: float = 0.0
    word_ops: int = 0
    status: int = 0
    stats: tuple = ()
    incomplete: int = 0


def _result(r: ResultC, status: int) -> Result:
    hist = np.array(r.hist[: r.hist_len], dtype=np.uint64)
    return Result(int(r.count), int(r.hash), int(r.tree_nodes), hist, bool(r.complete), int(r.list_cliques),
                  int(r.list_words), int(r.tasks_split), int(r.subproblems), float(r.ms_rank), float(r.ms_enum),
                  float(r.ms_search), int(r.word_ops), status, tuple(int(x) for x in r.stats), int(r.incomplete))


class Graph:
    """A device-resident CSR built by mce_graph_create."""

    def __init__(self, n: int, u, v, stream=None):
        lib = load()
        import torch
        on_dev = isinstance(u, torch.Tensor) and u.is_cuda
        if isinstance(u, torch.Tensor):
            u, v = u.contiguous(), v.contiguous()
            assert u.dtype == torch.int32 and v.dtype == torch.int32
        else:
            u = np.ascontiguousarray(u, dtype=np.int32)
            v = np.ascontiguousarray(v, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(lib.mce_graph_create(_ptr(u), _ptr(v), len(u), int(n), int(on_dev), _stream_ptr(stream),
                                    ctypes.byref(h)), "mce_graph_create")
        self._h, self.n = h, int(n)
        self._owned = True

    @classmethod
    def from_csr(cls, row_ptr, col, stream=None):
        """mce_graph_from_csr: a validated copy of a simple undirected CSR."""
        import torch
        on_dev = isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda
        if isinstance(row_ptr, torch.Tensor):
            row_ptr, col = row_ptr.contiguous(), col.contiguous()
            assert row_ptr.dtype == torch.int32 and col.dtype == torch.int32
        else:
            row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
            col = np.ascontiguousarray(col, dtype=np.int32)
        n = len(row_ptr) - 1
        h = ctypes.c_void_p()
        _check(load().mce_graph_from_csr(_ptr(row_ptr), _ptr(col) if len(col) else None, n, len(col), int(on_dev),
                                         _stream_ptr(stream), ctypes.byref(h)), "mce_graph_from_csr")
        g = cls.__new__(cls)
        g._h, g.n, g._owned = h, n, True
        return g

    @classmethod
    def _borrow(cls, handle, n):
        g = cls.__new__(cls)
        g._h, g.n, g._owned = ctypes.c_void_p(handle), n, False
        return g

    def close(self):
        if getattr(self, "_h", None) and self._owned:
            load().mce_graph_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def csr(self):
        """(row_ptr, col) copied to host numpy arrays (mce_graph_copy_csr)."""
        n, nnz = ctypes.c_int32(), ctypes.c_int64()
        _check(load().mce_graph_csr(self._h, ctypes.byref(n), ctypes.byref(nnz), None, None), "mce_graph_csr")
        row = np.zeros(n.value + 1, dtype=np.int32)
        col = np.zeros(max(nnz.value, 1), dtype=np.int32)
        _check(load().mce_graph_copy_csr(self._h, row.ctypes.data, col.ctypes.data, 1, _stream_ptr(None)),
               "mce_graph_copy_csr")
        return row, col[: nnz.value]

    @property
    def nnz(self) -> int:
        nnz = ctypes.c_int64()
        _check(load().mce_graph_csr(self._h, None, ctypes.byref(nnz), None, None), "mce_graph_csr")
        return int(nnz.value)


def make_opts(rank="degen", user_rank=None, model=None, node_budget=0, seed=0, stream=None, list_buf=None,
              per_vertex=None, split=True, order_by_model=False, warps_per_block=0, blocks_per_sm=0,
              time_limit_ms=0, subset=None, subproblem_budget=0, shared_words=0, split_nodes=0,
              queue_capacity=0, warp_small_search=False, whole_graph=False, sm_limit=0,
              lane_search_words=0, split_model=None, heavy_nodes=0, heavy_split_nodes=0,
              lane_hold_waiting=0) -> Opts:
    o = Opts()
    load().mce_opts_init(ctypes.byref(o))
    o.rank_kind = RANKS[rank] if isinstance(rank, str) else int(rank)
    o.user_rank = _ptr(user_rank)
    o.model = model._h if model is not None else None
    o.node_budget = node_budget
    o.hash_seed = seed
    o.stream = _stream_ptr(stream)
    if list_buf is not None:
        off, vtx = list_buf
        o.list_off, o.list_vtx = _ptr(off), _ptr(vtx)
        o.list_max_cliques, o.list_max_words = off.numel(), vtx.numel()
    if per_vertex is not None:
        o.pv_count, o.pv_hash, o.pv_nodes = (_ptr(t) for t in per_vertex)
    o.split = int(split)
    o.split_nodes = split_nodes
    o.order_by_model = int(order_by_model)
    o.warps_per_block = warps_per_block
    o.blocks_per_sm = blocks_per_sm
    o.shared_words = shared_words
    o.time_limit_ms = time_limit_ms
    if subset is not None:
        o.subset, o.subset_len = _ptr(subset), int(subset.numel() if hasattr(subset, "numel") else len(subset))
        o.subset_on_host = int(isinstance(subset, np.ndarray) or not subset.is_cuda)
    o.subproblem_budget = subproblem_budget
    o.queue_capacity = queue_capacity
    o.warp_small_search = int(warp_small_search)
    o.whole_graph = int(whole_graph)
    o.sm_limit = sm_limit
    o.lane_search_words = lane_search_words
    o.split_model = split_model._h if split_model is not None else None
    o.heavy_nodes = heavy_nodes
    o.heavy_split_nodes = heavy_split_nodes
    o.lane_hold_waiting = lane_hold_waiting
    return o


def enumerate_cliques(g: Graph, allow=(MCE_OK,), **kw) -> Result:
    """mce_enumerate.  Keyword arguments as make_opts."""
    lib = load()
    o = make_opts(**kw)
    r = ResultC()
    st = lib.mce_enumerate(g._h, ctypes.byref(o), ctypes.byref(r))
    if st not in allow:
        _check(st, "mce_enumerate")
    return _result(r, st)


SINK = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                        ctypes.c_int64, ctypes.c_int64)


def enumerate_stream(g: Graph, on_chunk, buf_words: int = 1 << 24, allow=(MCE_OK,), **kw) -> Result:
    """mce_enumerate_stream: on_chunk(off, vtx) gets each chunk's clique list
    as numpy arrays (copies), clique i at vtx[off[i]] (size, then ids)."""
    lib = load()
    o = make_opts(**kw)

    def tramp(_ctx, off, vtx, nc, nw):
        on_chunk(np.ctypeslib.as_array(off, shape=(nc,)).copy() if nc else np.zeros(0, np.int64),
                 np.ctypeslib.as_array(vtx, shape=(nw,)).copy() if nw else np.zeros(0, np.int32))

    cb = SINK(tramp)
    r = ResultC()
    st = lib.mce_enumerate_stream(g._h, ctypes.byref(o), int(buf_words), ctypes.cast(cb, ctypes.c_void_p), None,
                                  ctypes.byref(r))
    if st not in allow:
        _check(st, "mce_enumerate_stream")
    return _result(r, st)


def enumerate_noalloc(g: Graph, rank_dev, seed: int = 0, stream=None) -> Result:
    """mce_enumerate_noalloc on the CSR held by `g` with a device rank."""
    lib = load()
    n, nnz, rp, cl = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib.mce_graph_csr(g._h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(rp), ctypes.byref(cl)),
           "mce_graph_csr")
    r = ResultC()
    st = lib.mce_enumerate_noalloc(rp, cl, n.value, nnz.value, _ptr(rank_dev), seed, _stream_ptr(stream),
                                   ctypes.byref(r))
    _check(st, "mce_enumerate_noalloc")
    return _result(r, st)


def enumerate_noalloc_csr(row_ptr, col, n: int, rank_dev, seed: int = 0, stream=None) -> Result:
    """mce_enumerate_noalloc on caller device arrays (row_ptr int32[n+1], col
    int32[nnz], rank int32[n]); the library checks them before use."""
    lib = load()
    r = ResultC()
    st = lib.mce_enumerate_noalloc(_ptr(row_ptr), _ptr(col), int(n), int(col.numel()), _ptr(rank_dev), seed,
                                   _stream_ptr(stream), ctypes.byref(r))
    _check(st, "mce_enumerate_noalloc")
    return _result(r, st)


def vertex_key(g: Graph, kind, stream=None):
    import torch
    key = torch.empty(max(g.n, 1), dtype=torch.int64, device="cuda")
    _check(load().mce_vertex_key(g._h, RANKS[kind] if isinstance(kind, str) else kind, _stream_ptr(stream),
                                 _ptr(key)), "mce_vertex_key")
    return key[: g.n]


def rank(g: Graph, **kw):
    import torch
    out = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")
    o = make_opts(**kw)
    _check(load().mce_rank(g._h, ctypes.byref(o), _ptr(out)), "mce_rank")
    return out[: g.n]


FEATURES = {"full": 0, "light": 1}


def features(g: Graph, stream=None, kind="full"):
    import torch
    f = torch.empty((max(g.n, 1), 8), dtype=torch.float32, device="cuda")
    _check(load().mce_features_kind(g._h, FEATURES[kind], _stream_ptr(stream), _ptr(f)), "mce_features_kind")
    return f[: g.n]


def decode_list(off, vtx, n_cliques):
    """Host copy of a clique list -> sorted list of sorted tuples."""
    off = off[:n_cliques].cpu().numpy() if hasattr(off, "cpu") else np.asarray(off[:n_cliques])
    vtx = vtx.cpu().numpy() if hasattr(vtx, "cpu") else np.asarray(vtx)
    out = []
    for p in off.tolist():
        k = int(vtx[p])
        out.append(tuple(sorted(int(x) for x in vtx[p + 1: p + 1 + k])))
    return sorted(out)


class Model:
    """MLP cost model (mce_model_*)."""

    def __init__(self, hidden: int = 64, seed: int = 0, features: str = "full"):
        h = ctypes.c_void_p()
        _check(load().mce_model_create(hidden, seed, ctypes.byref(h)), "mce_model_create")
        self._h, self.hidden = h, hidden
        _check(load().mce_model_set_features(h, FEATURES[features]), "mce_model_set_features")
        self.features = features

    def close(self):
        if getattr(self, "_h", None):
            load().mce_model_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self) -> int:
        return int(load().mce_model_num_params(self._h))

    def get(self) -> np.ndarray:
        a = np.zeros(self.num_params, dtype=np.float32)
        _check(load().mce_model_get(self._h, a.ctypes.data), "mce_model_get")
        return a

    def set(self, params: np.ndarray):
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert len(a) == self.num_params
        _check(load().mce_model_set(self._h, a.ctypes.data), "mce_model_set")

    def loss_grad(self, feat, label, stream=None):
        g = np.zeros(self.num_params, dtype=np.float32)
        loss = ctypes.c_float()
        _check(load().mce_model_loss_grad(self._h, _ptr(feat), _ptr(label), feat.shape[0], _stream_ptr(stream),
                                          ctypes.byref(loss), g.ctypes.data), "mce_model_loss_grad")
        return float(loss.value), g

    def train(self, feat, label, epochs=5, batch=4096, lr=1e-3, seed=0, stream=None) -> float:
        loss = ctypes.c_float()
        _check(load().mce_model_train(self._h, _ptr(feat), _ptr(label), feat.shape[0], epochs, batch, lr, seed,
                                      _stream_ptr(stream), ctypes.byref(loss)), "mce_model_train")
        return float(loss.value)

    def predict(self, feat, bf16=True, stream=None):
        import torch
        out = torch.empty(max(feat.shape[0], 1), dtype=torch.float32, device="cuda")
        _check(load().mce_model_predict(self._h, _ptr(feat), feat.shape[0], int(bf16), _stream_ptr(stream),
                                        _ptr(out)), "mce_model_predict")
        return out[: feat.shape[0]]


def enumerate_batched(g: Graph, graph_ptr, allow=(MCE_OK, MCE_EBUDGET), **kw):
    """mce_enumerate_batched: per-graph (counts, hashes, status) and the total."""
    import torch
    lib = load()
    k = len(graph_ptr) - 1
    gp = np.ascontiguousarray(graph_ptr, dtype=np.int32)
    counts = torch.zeros(max(k, 1), dtype=torch.int64, device="cuda")
    hashes = torch.zeros(max(k, 1), dtype=torch.int64, device="cuda")
    status = torch.zeros(max(k, 1), dtype=torch.int32, device="cuda")
    o = make_opts(**kw)
    r = ResultC()
    st = lib.mce_enumerate_batched(g._h, gp.ctypes.data, k, ctypes.byref(o), _ptr(counts), _ptr(hashes),
                                   _ptr(status), ctypes.byref(r))
    if st not in allow:
        _check(st, "mce_enumerate_batched")
    u64 = lambda t: t[:k].cpu().numpy().view(np.uint64)  # noqa: E731
    return u64(counts), u64(hashes), status[:k].cpu().numpy(), _result(r, st)


class BatchedPlan:
    """mce_batched_*: prepared once, each run captured into / replayed from a CUDA graph."""

    def __init__(self, g: Graph, graph_ptr, **kw):
        self.k = len(graph_ptr) - 1
        self._gptr = np.ascontiguousarray(graph_ptr, dtype=np.int32)
        self._g = g                               # the plan points into g
        o = make_opts(**kw)
        h = ctypes.c_void_p()
        _check(load().mce_batched_create(g._h, self._gptr.ctypes.data, self.k, ctypes.byref(o), ctypes.byref(h)),
               "mce_batched_create")
        self._h = h
        self._stream = kw.get("stream")

    def close(self):
        if getattr(self, "_h", None):
            load().mce_batched_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self):
        _check(load().mce_batched_run(self._h, _stream_ptr(self._stream)), "mce_batched_run")

    def read(self):
        counts = np.zeros(self.k, np.uint64)
        hashes = np.zeros(self.k, np.uint64)
        status = np.zeros(self.k, np.int32)
        r = ResultC()
        st = load().mce_batched_read(self._h, _stream_ptr(self._stream), counts.ctypes.data, hashes.ctypes.data,
                                     status.ctypes.data, ctypes.byref(r))
        if st not in (MCE_OK, MCE_EBUDGET):
            _check(st, "mce_batched_read")
        return counts, hashes, status, _result(r, st)

    def tune(self, tune_budget=0, repeats=1):
        """Returns (blocks per SM, hand-over interval, whole-warp small search)."""
        bps, sp, ws = ctypes.c_int32(), ctypes.c_uint32(), ctypes.c_int32()
        _check(load().mce_batched_tune(self._h, _stream_ptr(self._stream), tune_budget, repeats, ctypes.byref(bps),
                                       ctypes.byref(sp), ctypes.byref(ws)), "mce_batched_tune")
        return int(bps.value), int(sp.value), bool(ws.value)


@dataclass
class Delta:
    applied: int
    dropped: int
    new_count: int
    new_hash: int
    sub_count: int
    sub_hash: int
    new_hist: np.ndarray
    sub_hist: np.ndarray
    alive: int
    ms: float


def _delta(d: DeltaC) -> Delta:
    return Delta(int(d.applied), int(d.dropped), int(d.new_count), int(d.new_hash), int(d.sub_count),
                 int(d.sub_hash), np.array(d.new_hist[: d.new_hist_len], dtype=np.uint64),
                 np.array(d.sub_hist[: d.sub_hist_len], dtype=np.uint64), int(d.alive), float(d.ms))


class Imce:
    """Incremental maximal cliques (imce_open / imce_add_edges)."""

    def __init__(self, g: Graph, seed: int = 0, stream=None, rank="degen"):
        h = ctypes.c_void_p()
        o = make_opts(rank=rank, seed=seed, stream=stream)
        _check(load().imce_open(g._h, ctypes.byref(o), ctypes.byref(h)), "imce_open")
        self._h, self.n = h, g.n

    def close(self):
        if getattr(self, "_h", None):
            load().imce_close(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_edges(self, u, v) -> Delta:
        import torch
        on_dev = isinstance(u, torch.Tensor) and u.is_cuda
        if not isinstance(u, torch.Tensor):
            u = np.ascontiguousarray(u, dtype=np.int32)
            v = np.ascontiguousarray(v, dtype=np.int32)
        d = DeltaC()
        _check(load().imce_add_edges(self._h, _ptr(u), _ptr(v), len(u), int(on_dev), ctypes.byref(d)),
               "imce_add_edges")
        return _delta(d)

    def remove_edges(self, u, v) -> Delta:
        """imce_remove_edges: delta.new_* = created cliques, delta.sub_* = removed ones."""
        import torch
        on_dev = isinstance(u, torch.Tensor) and u.is_cuda
        if not isinstance(u, torch.Tensor):
            u = np.ascontiguousarray(u, dtype=np.int32)
            v = np.ascontiguousarray(v, dtype=np.int32)
        d = DeltaC()
        _check(load().imce_remove_edges(self._h, _ptr(u), _ptr(v), len(u), int(on_dev), ctypes.byref(d)),
               "imce_remove_edges")
        return _delta(d)

    def graph(self) -> Graph:
        return Graph._borrow(load().imce_graph(self._h), self.n)

    def cliques(self, max_cliques: int, max_words: int):
        import torch
        off = torch.empty(max(max_cliques, 1), dtype=torch.int64, device="cuda")
        vtx = torch.empty(max(max_words, 1), dtype=torch.int32, device="cuda")
        nc, nw = ctypes.c_int64(), ctypes.c_int64()
        _check(load().imce_cliques(self._h, _ptr(off), _ptr(vtx), max_cliques, max_words, ctypes.byref(nc),
                                   ctypes.byref(nw)), "imce_cliques")
        return decode_list(off, vtx, nc.value)


@dataclass
class RequestInfo:
    id: int
    tenant: int
    status: int
    edges: int
    arrival_ms: float
    admit_ms: float
    done_ms: float
    reserved: int
    delta: Delta


class Server:
    """imce_server_*: continuous batching of edge batches over tenants.

    `execute` (tests only) replaces imce_add_edges by a Python callable
    f(tenant, u, v) -> Delta-like tuple, so the scheduler runs without a GPU."""

    def __init__(self, slots=4, mem_budget=0, mem_fixed=0, execute=None):
        lib = load()
        o = ServerOpts()
        lib.imce_server_opts_init(ctypes.byref(o))
        o.slots, o.mem_budget, o.mem_fixed = slots, mem_budget, mem_fixed
        self._cb = None
        if execute is not None:
            def tramp(_ctx, tenant, u, v, k, out):
                try:
                    ua = np.ctypeslib.as_array(ctypes.cast(u, ctypes.POINTER(ctypes.c_int32)), (k,)).copy() if k else \
                        np.zeros(0, np.int32)
                    va = np.ctypeslib.as_array(ctypes.cast(v, ctypes.POINTER(ctypes.c_int32)), (k,)).copy() if k else \
                        np.zeros(0, np.int32)
                    st, applied, new_count = execute(tenant, ua, va)
                    out.contents.applied = applied
                    out.contents.dropped = k - applied
                    out.contents.new_count = new_count
                    return st
                except Exception:                 # noqa: BLE001 - reported as a failed batch
                    return MCE_ESTATE
            self._cb = EXEC_FN(tramp)
            o.execute = self._cb
        h = ctypes.c_void_p()
        _check(lib.imce_server_create(ctypes.byref(o), ctypes.byref(h)), "imce_server_create")
        self._h = h
        self._n = []

    def close(self):
        if getattr(self, "_h", None):
            load().imce_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_tenant(self, g: Graph | None = None, seed: int = 0, rank="degen") -> int:
        t = ctypes.c_int32()
        o = make_opts(rank=rank, seed=seed) if g is not None else None
        _check(load().imce_server_add_tenant(self._h, g._h if g is not None else None,
                                             ctypes.byref(o) if o is not None else None, ctypes.byref(t)),
               "imce_server_add_tenant")
        self._n.append(g.n if g is not None else 0)
        return int(t.value)

    def submit(self, tenant: int, u, v, arrival_ms: float = -1.0) -> int:
        u = np.ascontiguousarray(u, dtype=np.int32)
        v = np.ascontiguousarray(v, dtype=np.int32)
        rid = ctypes.c_int64()
        _check(load().imce_server_submit(self._h, tenant, u.ctypes.data, v.ctypes.data, len(u), float(arrival_ms),
                                         ctypes.byref(rid)), "imce_server_submit")
        return int(rid.value)

    def wait(self, rid: int) -> RequestInfo:
        info = RequestInfoC()
        st = load().imce_server_wait(self._h, rid, ctypes.byref(info))
        if st == MCE_EINVAL and info.id != rid:
            _check(st, "imce_server_wait")
        return RequestInfo(int(info.id), int(info.tenant), int(info.status), int(info.edges), info.arrival_ms,
                           info.admit_ms, info.done_ms, int(info.reserved), _delta(info.delta))

    def drain(self):
        _check(load().imce_server_drain(self._h), "imce_server_drain")

    def reset_clock(self):
        _check(load().imce_server_reset_clock(self._h), "imce_server_reset_clock")

    def stats(self) -> dict:
        st = ServerStatsC()
        _check(load().imce_server_stats_get(self._h, ctypes.byref(st)), "imce_server_stats_get")
        return {name: getattr(st, name) for name, _ in ServerStatsC._fields_}

    def cliques(self, tenant: int, max_cliques: int, max_words: int):
        """Alive cliques of an idle tenant (imce_cliques on its state)."""
        import torch
        h = load().imce_server_tenant(self._h, tenant)
        if not h:
            raise MceError(MCE_EINVAL, "imce_server_tenant: no device state")
        off = torch.empty(max(max_cliques, 1), dtype=torch.int64, device="cuda")
        vtx = torch.empty(max(max_words, 1), dtype=torch.int32, device="cuda")
        nc, nw = ctypes.c_int64(), ctypes.c_int64()
        _check(load().imce_cliques(h, _ptr(off), _ptr(vtx), max_cliques, max_words, ctypes.byref(nc),
                                   ctypes.byref(nw)), "imce_cliques")
        return decode_list(off, vtx, nc.value)
