"""CPU oracle for maximal clique enumeration — test infrastructure only.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_2001_11433_gb300``) and neither imports the other; both consume the
seeded inputs of ``graphgen``.

The arithmetic lives in ``oracle.c`` (plain sequential C: Algorithm 1 TTT,
Algorithm 5 per-vertex decomposition, Algorithms 6 + 9 for new cliques,
Algorithm 8 for subsumed cliques, and the plain set-difference definitions
of Section 5).  This module only marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            sig = {
                "or_graph_from_pairs": ([i32, vp, vp, i64], vp),
                "or_graph_free": ([vp], None),
                "or_graph_nnz": ([vp], i64),
                "or_graph_n": ([vp], i32),
                "or_graph_export": ([vp, vp, vp], None),
                "or_graph_plus": ([vp, vp, vp, i64], vp),
                "or_graph_minus": ([vp, vp, vp, i64], vp),
                "or_canonical_deletion": ([vp, vp, vp, i64, vp, vp], i64),
                "or_dmce_alg": ([vp, vp, vp, i64, vp, vp], None),
                "or_dmce_diff": ([vp, vp, vp, i64, vp, vp], None),
                "or_imce_remove": ([vp, vp, vp, i64, vp, vp], i64),
                "or_out_new": ([ctypes.c_int, u64], vp),
                "or_out_free": ([vp], None),
                "or_out_count": ([vp], u64),
                "or_out_hash": ([vp], u64),
                "or_out_nodes": ([vp], u64),
                "or_out_overflow": ([vp], i32),
                "or_out_hist_len": ([vp], i32),
                "or_out_hist": ([vp, vp], None),
                "or_out_list_len": ([vp], i64),
                "or_out_list_nnz": ([vp], i64),
                "or_out_list_copy": ([vp, vp, vp], None),
                "or_degree": ([vp, vp], None),
                "or_core_numbers": ([vp, vp], None),
                "or_triangles": ([vp, vp], None),
                "or_rank_from_key": ([i32, vp, vp], None),
                "or_ttt_whole": ([vp, vp], None),
                "or_parmce": ([vp, vp, vp, i64, i32, vp, vp, vp, vp, u64, vp], i32),
                "or_canonical_batch": ([vp, vp, vp, i64, vp, vp], i64),
                "or_imce_alg": ([vp, vp, vp, i64, vp, vp], None),
                "or_imce_diff": ([vp, vp, vp, i64, vp, vp], None),
                "or_imce_open": ([vp, u64, i32], vp),
                "or_imce_close": ([vp], None),
                "or_imce_graph": ([vp], vp),
                "or_imce_alive": ([vp], i64),
                "or_imce_add": ([vp, vp, vp, i64, vp, vp], i64),
                "or_imce_cliques": ([vp, vp], None),
                "or_clique_hash": ([vp, i32, u64], u64),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


@dataclass
class Result:
    """Summary of a set of maximal cliques (and the cliques, if requested)."""
    count: int
    hash: int
    nodes: int
    hist: np.ndarray
    cliques: list | None = None          # sorted list of sorted tuples
    per_vertex: dict = field(default_factory=dict)


def _result(out, want_list: bool) -> Result:
    lib = _L()
    if lib.or_out_overflow(out):
        raise RuntimeError("oracle: clique larger than its histogram")
    hl = lib.or_out_hist_len(out)
    hist = np.zeros(hl, dtype=np.uint64)
    if hl:
        lib.or_out_hist(out, hist.ctypes.data)
    cl = None
    if want_list:
        nc, nnz = lib.or_out_list_len(out), lib.or_out_list_nnz(out)
        off = np.zeros(nc + 1, dtype=np.int64)
        vtx = np.zeros(max(nnz, 1), dtype=np.int32)
        lib.or_out_list_copy(out, off.ctypes.data, vtx.ctypes.data)
        cl = sorted(tuple(int(x) for x in vtx[off[i]:off[i + 1]]) for i in range(nc))
    return Result(int(lib.or_out_count(out)), int(lib.or_out_hash(out)), int(lib.or_out_nodes(out)), hist, cl)


class Graph:
    """Simple undirected graph built from raw pairs (self loops and repeats dropped)."""

    def __init__(self, n: int, u, v):
        u, v = _i32(u), _i32(v)
        assert len(u) == len(v)
        self._h = _L().or_graph_from_pairs(int(n), u.ctypes.data, v.ctypes.data, len(u))
        if not self._h:
            raise ValueError("vertex id outside [0, n)")
        self.n = int(n)

    @classmethod
    def _wrap(cls, h, n):
        g = cls.__new__(cls)
        g._h, g.n = h, n
        return g

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and getattr(self, "_owned", True):
            _L().or_graph_free(h)
            self._h = None

    @property
    def nnz(self) -> int:
        return int(_L().or_graph_nnz(self._h))

    def csr(self):
        rp = np.zeros(self.n + 1, dtype=np.int64)
        col = np.zeros(max(self.nnz, 1), dtype=np.int32)
        _L().or_graph_export(self._h, rp.ctypes.data, col.ctypes.data)
        return rp, col[: self.nnz]

    def plus(self, hu, hv) -> "Graph":
        hu, hv = _i32(hu), _i32(hv)
        return Graph._wrap(_L().or_graph_plus(self._h, hu.ctypes.data, hv.ctypes.data, len(hu)), self.n)

    def minus(self, hu, hv) -> "Graph":
        hu, hv = _i32(hu), _i32(hv)
        return Graph._wrap(_L().or_graph_minus(self._h, hu.ctypes.data, hv.ctypes.data, len(hu)), self.n)


def degree(g: Graph) -> np.ndarray:
    out = np.zeros(g.n, dtype=np.int64)
    _L().or_degree(g._h, out.ctypes.data)
    return out


def core_numbers(g: Graph) -> np.ndarray:
    out = np.zeros(g.n, dtype=np.int32)
    _L().or_core_numbers(g._h, out.ctypes.data)
    return out


def triangles(g: Graph) -> np.ndarray:
    out = np.zeros(g.n, dtype=np.int64)
    _L().or_triangles(g._h, out.ctypes.data)
    return out


def rank_from_key(key) -> np.ndarray:
    """rank[v] = position of (key[v], v) in ascending lexicographic order."""
    key = np.ascontiguousarray(key, dtype=np.float64)
    rank = np.zeros(len(key), dtype=np.int32)
    _L().or_rank_from_key(len(key), key.ctypes.data, rank.ctypes.data)
    return rank


def rank(g: Graph, kind: str) -> np.ndarray:
    """Section 4.2 ranks: 'degree', 'degen' (core number), 'triangle'."""
    if kind == "degree":
        key = degree(g)
    elif kind == "degen":
        key = core_numbers(g)
    elif kind == "triangle":
        key = triangles(g)
    else:
        raise ValueError(kind)
    return rank_from_key(key)


def ttt_whole(g: Graph, want_list: bool = False, seed: int = 0) -> Result:
    lib = _L()
    out = lib.or_out_new(int(want_list), seed)
    try:
        lib.or_ttt_whole(g._h, out)
        return _result(out, want_list)
    finally:
        lib.or_out_free(out)


def parmce(g: Graph, rank_arr, subset=None, threads: int = 1, want_list: bool = False,
           per_vertex: bool = False, seed: int = 0, node_cap: int = 0) -> Result:
    """Algorithm 5 run one subproblem at a time (on `threads` host threads).

    With `subset`, only those vertices' subproblems run; per-vertex arrays
    are indexed like `subset` (or by vertex id when subset is None).  With
    `node_cap`, a subproblem whose search tree has more than node_cap nodes
    is given up, left out of the result and flagged in per_vertex["over"]."""
    lib = _L()
    rank_arr = _i32(rank_arr)
    sub = None if subset is None else _i32(subset)
    ns = g.n if sub is None else len(sub)
    pv = [np.zeros(ns, dtype=np.uint64) for _ in range(3)] if per_vertex else None
    over = np.zeros(max(ns, 1), dtype=np.uint8) if node_cap else None
    out = lib.or_out_new(int(want_list), seed)
    try:
        used = lib.or_parmce(g._h, rank_arr.ctypes.data, None if sub is None else sub.ctypes.data, ns,
                             threads, out,
                             *(p.ctypes.data for p in pv) if pv else (None, None, None),
                             int(node_cap), None if over is None else over.ctypes.data)
        r = _result(out, want_list)
        r.per_vertex["threads"] = int(used)
        if pv:
            r.per_vertex.update(count=pv[0], hash=pv[1], nodes=pv[2])
        if over is not None:
            r.per_vertex["over"] = over[:ns].astype(bool)
        return r
    finally:
        lib.or_out_free(out)


def canonical_batch(g: Graph, u, v):
    u, v = _i32(u), _i32(v)
    hu = np.zeros(max(len(u), 1), dtype=np.int32)
    hv = np.zeros(max(len(u), 1), dtype=np.int32)
    k = _L().or_canonical_batch(g._h, u.ctypes.data, v.ctypes.data, len(u), hu.ctypes.data, hv.ctypes.data)
    if k < 0:
        raise ValueError("vertex id outside [0, n)")
    return hu[:k].copy(), hv[:k].copy()


def canonical_deletion(g: Graph, u, v):
    """Deletion batch in arrival order: pairs that are edges of g, each once."""
    u, v = _i32(u), _i32(v)
    hu = np.zeros(max(len(u), 1), dtype=np.int32)
    hv = np.zeros(max(len(u), 1), dtype=np.int32)
    k = _L().or_canonical_deletion(g._h, u.ctypes.data, v.ctypes.data, len(u), hu.ctypes.data, hv.ctypes.data)
    if k < 0:
        raise ValueError("vertex id outside [0, n)")
    return hu[:k].copy(), hv[:k].copy()


def _imce2(fn, g, hu, hv, seed):
    lib = _L()
    hu, hv = _i32(hu), _i32(hv)
    a, b = lib.or_out_new(1, seed), lib.or_out_new(1, seed)
    try:
        fn(g._h, hu.ctypes.data, hv.ctypes.data, len(hu), a, b)
        return _result(a, True), _result(b, True)
    finally:
        lib.or_out_free(a)
        lib.or_out_free(b)


def imce_alg(g: Graph, hu, hv, seed: int = 0):
    """(Λnew, Λdel) by Algorithms 6 + 9 and 8; hu/hv a canonical batch."""
    return _imce2(_L().or_imce_alg, g, hu, hv, seed)


def imce_diff(g: Graph, hu, hv, seed: int = 0):
    """(Λnew, Λdel) by the plain set differences; hu/hv a canonical batch."""
    return _imce2(_L().or_imce_diff, g, hu, hv, seed)


def dmce_alg(g: Graph, hu, hv, seed: int = 0):
    """(removed, created) cliques of deleting a canonical batch from g, by the
    reduction to the incremental case (Algorithms 6 + 9 on g, then Algorithm
    8's splits kept when maximal in g - H)."""
    return _imce2(_L().or_dmce_alg, g, hu, hv, seed)


def dmce_diff(g: Graph, hu, hv, seed: int = 0):
    """(C(g) \\ C(g - H), C(g - H) \\ C(g)) by the plain set differences."""
    return _imce2(_L().or_dmce_diff, g, hu, hv, seed)


class Imce:
    """Graph plus its maximal cliques, updated batch by batch (mode B)."""

    def __init__(self, g: Graph, seed: int = 0, threads: int = 1):
        self._h = _L().or_imce_open(g._h, seed, threads)
        self.n, self.seed = g.n, seed

    def close(self):
        if getattr(self, "_h", None):
            _L().or_imce_close(self._h)
            self._h = None

    __del__ = close

    def add(self, u, v, want_list: bool = True):
        lib = _L()
        u, v = _i32(u), _i32(v)
        a, b = lib.or_out_new(int(want_list), self.seed), lib.or_out_new(int(want_list), self.seed)
        try:
            rho = lib.or_imce_add(self._h, u.ctypes.data, v.ctypes.data, len(u), a, b)
            if rho < 0:
                raise ValueError("vertex id outside [0, n)")
            return int(rho), _result(a, want_list), _result(b, want_list)
        finally:
            lib.or_out_free(a)
            lib.or_out_free(b)

    def remove(self, u, v, want_list: bool = True):
        """Delete a batch of edges: (deleted ρ, removed cliques, created cliques)."""
        lib = _L()
        u, v = _i32(u), _i32(v)
        a, b = lib.or_out_new(int(want_list), self.seed), lib.or_out_new(int(want_list), self.seed)
        try:
            rho = lib.or_imce_remove(self._h, u.ctypes.data, v.ctypes.data, len(u), a, b)
            if rho < 0:
                raise ValueError("vertex id outside [0, n)")
            return int(rho), _result(a, want_list), _result(b, want_list)
        finally:
            lib.or_out_free(a)
            lib.or_out_free(b)

    @property
    def alive(self) -> int:
        return int(_L().or_imce_alive(self._h))

    def cliques(self, want_list: bool = True) -> Result:
        lib = _L()
        out = lib.or_out_new(int(want_list), self.seed)
        try:
            lib.or_imce_cliques(self._h, out)
            return _result(out, want_list)
        finally:
            lib.or_out_free(out)

    def graph_csr(self):
        g = Graph._wrap(_L().or_imce_graph(self._h), self.n)
        g._owned = False
        return g.csr()


def clique_hash(k, seed: int = 0) -> int:
    k = _i32(k)
    return int(_L().or_clique_hash(k.ctypes.data, len(k), seed))
