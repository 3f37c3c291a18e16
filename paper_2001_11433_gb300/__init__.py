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


# (name, argtypes, restype) of every exported symbol of include/mce.h
_vp, _i32, _i64, _u64, _f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float
_P = ctypes.POINTER
SIGNATURES = {
    "mce_strerror": ([_i32], ctypes.c_char_p),
    "mce_last_error": ([], ctypes.c_char_p),
    "mce_opts_init": ([_P(Opts)], None),
    "mce_kernel_launches": ([], _u64),
    "mce_graph_create": ([_vp, _vp, _i64, _i32, _i32, _vp, _P(_vp)], _i32),
    "mce_graph_csr": ([_vp, _P(_i32), _P(_i64), _P(_vp), _P(_vp)], _i32),
    "mce_graph_copy_csr": ([_vp, _vp, _vp, _i32, _vp], _i32),
    "mce_graph_free": ([_vp], None),
    "mce_vertex_key": ([_vp, _i32, _vp, _vp], _i32),
    "mce_rank": ([_vp, _P(Opts), _vp], _i32),
    "mce_enumerate": ([_vp, _P(Opts), _P(ResultC)], _i32),
    "mce_features": ([_vp, _vp, _vp], _i32),
    "mce_model_create": ([_i32, _u64, _P(_vp)], _i32),
    "mce_model_free": ([_vp], None),
    "mce_model_num_params": ([_vp], _i64),
    "mce_model_get": ([_vp, _vp], _i32),
    "mce_model_set": ([_vp, _vp], _i32),
    "mce_model_loss_grad": ([_vp, _vp, _vp, _i32, _vp, _P(_f32), _vp], _i32),
    "mce_model_train": ([_vp, _vp, _vp, _i32, _i32, _i32, _f32, _u64, _vp, _P(_f32)], _i32),
    "mce_model_predict": ([_vp, _vp, _i32, _i32, _vp, _vp], _i32),
    "mce_enumerate_batched": ([_vp, _vp, _i32, _P(Opts), _vp, _vp, _vp, _P(ResultC)], _i32),
    "imce_open": ([_vp, _P(Opts), _P(_vp)], _i32),
    "imce_add_edges": ([_vp, _vp, _vp, _i64, _i32, _P(DeltaC)], _i32),
    "imce_graph": ([_vp], _vp),
    "imce_cliques": ([_vp, _vp, _vp, _i64, _i64, _P(_i64), _P(_i64)], _i32),
    "imce_close": ([_vp], None),
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
              time_limit_ms=0, subset=None, subproblem_budget=0, shared_words=0, split_nodes=0) -> Opts:
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


def features(g: Graph, stream=None):
    import torch
    f = torch.empty((max(g.n, 1), 8), dtype=torch.float32, device="cuda")
    _check(load().mce_features(g._h, _stream_ptr(stream), _ptr(f)), "mce_features")
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

    def __init__(self, hidden: int = 64, seed: int = 0):
        h = ctypes.c_void_p()
        _check(load().mce_model_create(hidden, seed, ctypes.byref(h)), "mce_model_create")
        self._h, self.hidden = h, hidden

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
        return Delta(int(d.applied), int(d.dropped), int(d.new_count), int(d.new_hash), int(d.sub_count),
                     int(d.sub_hash), np.array(d.new_hist[: d.new_hist_len], dtype=np.uint64),
                     np.array(d.sub_hist[: d.sub_hist_len], dtype=np.uint64), int(d.alive), float(d.ms))

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
