"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package draws raw edge samples only.  It contains none of the
enumeration arithmetic: samples may hold self-loops and repeated pairs, and
each consumer normalises them into a simple undirected graph itself
(Section 3: simple undirected graphs; Section 6.1: self loops, parallel edges
and directions are dropped).

The C library (gen.c) is compiled on first use with gcc into this directory.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_SO = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

BASE_SEED = 20010433


def build(force: bool = False) -> str:
    """Compile gen.c into libgraphgen.so (plain C, no architecture flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P32 = ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))
            i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            lib.gg_er.argtypes = [i32, dbl, u64, P32, P32]
            lib.gg_er.restype = i64
            lib.gg_rmat.argtypes = [i32, i64, dbl, dbl, dbl, u64, P32, P32]
            lib.gg_rmat.restype = i64
            lib.gg_chung_lu.argtypes = [i32, dbl, dbl, dbl, u64, P32, P32,
                                        ctypes.POINTER(ctypes.POINTER(ctypes.c_double))]
            lib.gg_chung_lu.restype = i64
            lib.gg_chung_lu_i0.argtypes = [i32, dbl, dbl, dbl]
            lib.gg_chung_lu_i0.restype = dbl
            lib.gg_planted_cliques.argtypes = [i32, i32, i32, i32, u64, P32, P32]
            lib.gg_planted_cliques.restype = i64
            lib.gg_batched_er.argtypes = [i32, i32, i32, dbl, dbl, u64,
                                          ctypes.c_void_p, ctypes.c_void_p, P32, P32]
            lib.gg_batched_er.restype = i64
            lib.gg_edge_stream.argtypes = [i32, ctypes.c_void_p, ctypes.c_void_p, i64, i64, u64, P32, P32]
            lib.gg_edge_stream.restype = i64
            lib.gg_batch_schedule.argtypes = [i64, dbl, dbl, u64,
                                              ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)),
                                              ctypes.POINTER(ctypes.POINTER(ctypes.c_double))]
            lib.gg_batch_schedule.restype = i64
            lib.gg_substream_seed.argtypes = [u64, u64]
            lib.gg_substream_seed.restype = u64
            lib.gg_free.argtypes = [ctypes.c_void_p]
            lib.gg_free.restype = None
            _lib = lib
    return _lib


def _take(ptr, m, dtype):
    lib = _L()
    if m < 0:
        raise MemoryError("generator allocation failed")
    if m == 0:
        if ptr:
            lib.gg_free(ptr)
        return np.zeros(0, dtype=dtype)
    arr = np.ctypeslib.as_array(ptr, shape=(m,)).copy()
    lib.gg_free(ptr)
    return arr.astype(dtype, copy=False)


def _pair_call(fn, *args):
    pu = ctypes.POINTER(ctypes.c_int32)()
    pv = ctypes.POINTER(ctypes.c_int32)()
    m = fn(*args, ctypes.byref(pu), ctypes.byref(pv))
    return _take(pu, m, np.int32), _take(pv, m, np.int32)


def substream_seed(base: int, k: int) -> int:
    return int(_L().gg_substream_seed(base, k))


def er(n: int, p: float, seed: int):
    """G(n, p): one draw per pair (i<j) in lexicographic order."""
    return _pair_call(_L().gg_er, n, p, seed)


def rmat(scale: int, samples: int, a: float, b: float, c: float, seed: int):
    """R-MAT samples (may include self-loops and repeats)."""
    return _pair_call(_L().gg_rmat, scale, samples, a, b, c, seed)


def chung_lu(n: int, gamma: float, wmax: float, m_target: float, seed: int):
    """Chung-Lu graph; returns (u, v, weights)."""
    lib = _L()
    pu = ctypes.POINTER(ctypes.c_int32)()
    pv = ctypes.POINTER(ctypes.c_int32)()
    pw = ctypes.POINTER(ctypes.c_double)()
    m = lib.gg_chung_lu(n, gamma, wmax, m_target, seed, ctypes.byref(pu), ctypes.byref(pv), ctypes.byref(pw))
    u, v = _take(pu, m, np.int32), _take(pv, m, np.int32)
    w = np.ctypeslib.as_array(pw, shape=(n,)).copy()
    lib.gg_free(pw)
    return u, v, w


def planted_cliques(n: int, count: int, kmin: int, kmax: int, seed: int):
    return _pair_call(_L().gg_planted_cliques, n, count, kmin, kmax, seed)


def batched_er(k: int, nmin: int, nmax: int, pmin: float, pmax: float, seed: int):
    """k disjoint G(n_g, p_g); returns (u, v, graph_ptr[k+1], p[k])."""
    gptr = np.zeros(k + 1, dtype=np.int32)
    probs = np.zeros(k, dtype=np.float64)
    u, v = _pair_call(_L().gg_batched_er, k, nmin, nmax, pmin, pmax, seed,
                      gptr.ctypes.data, probs.ctypes.data)
    return u, v, gptr, probs


def edge_stream(n: int, w: np.ndarray, base_keys_sorted: np.ndarray, count: int, seed: int):
    """`count` new edges, endpoints proportional to w, avoiding base edges and repeats."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    keys = np.ascontiguousarray(base_keys_sorted, dtype=np.uint64)
    return _pair_call(_L().gg_edge_stream, n, w.ctypes.data, keys.ctypes.data, len(keys), count, seed)


def batch_schedule(total: int, lo: float, hi: float, seed: int):
    lib = _L()
    ps = ctypes.POINTER(ctypes.c_int64)()
    pg = ctypes.POINTER(ctypes.c_double)()
    nb = lib.gg_batch_schedule(total, lo, hi, seed, ctypes.byref(ps), ctypes.byref(pg))
    sizes = _take(ps, nb, np.int64)
    gaps = np.ctypeslib.as_array(pg, shape=(nb,)).copy() if nb > 0 else np.zeros(0)
    if nb > 0:
        lib.gg_free(pg)
    return sizes, gaps


def canonical_keys(u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Sorted unique keys a<<32|b (a<b) of the simple graph behind raw samples.

    Used only to tell the edge-stream generator which pairs already exist; it
    is input bookkeeping, not part of either implementation under test."""
    u = u.astype(np.int64)
    v = v.astype(np.int64)
    keep = u != v
    a = np.minimum(u, v)[keep]
    b = np.maximum(u, v)[keep]
    return np.unique((a << 32) | b).astype(np.uint64)


# ---------------------------------------------------------------------------
# The five workloads (raw samples).  Seeds: BASE_SEED + workload index.
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    n: int
    u: np.ndarray
    v: np.ndarray
    extra: dict = field(default_factory=dict)


def er_2000(seed: int = BASE_SEED + 1) -> Workload:
    """Erdos-Renyi G(2000, 0.01)."""
    u, v = er(2000, 0.01, seed)
    return Workload("er_n2000_p0.01", 2000, u, v)


def rmat_18(seed: int = BASE_SEED + 2, scale: int = 18, edge_factor: int = 16) -> Workload:
    """R-MAT scale 18, 16*n samples, (a,b,c,d) = (0.57, 0.19, 0.19, 0.05)."""
    n = 1 << scale
    u, v = rmat(scale, edge_factor * n, 0.57, 0.19, 0.19, seed)
    return Workload(f"rmat_s{scale}_ef{edge_factor}", n, u, v)


def chung_lu_planted(seed: int = BASE_SEED + 3, n: int = 1_700_000, gamma: float = 2.2,
                     wmax: float = 35_000.0, m_target: float = 11_000_000.0,
                     n_cliques: int = 200, kmin: int = 20, kmax: int = 60) -> Workload:
    """Chung-Lu power-law graph plus planted cliques of uniform size [kmin, kmax]."""
    u1, v1, w = chung_lu(n, gamma, wmax, m_target, substream_seed(seed, 0))
    u2, v2 = planted_cliques(n, n_cliques, kmin, kmax, substream_seed(seed, 1))
    name = f"chunglu_n{n}_g{gamma}_wmax{int(wmax)}_planted{n_cliques}"
    return Workload(name, n, np.concatenate([u1, u2]), np.concatenate([v1, v2]), {"w": w})


def batched_er_4096(seed: int = BASE_SEED + 4, k: int = 4096, nmin: int = 32, nmax: int = 2048,
                    pmin: float = 0.1, pmax: float = 0.6) -> Workload:
    """k independent G(n_g, p_g), n_g log-uniform in [nmin, nmax], p_g ~ U[pmin, pmax]."""
    u, v, gptr, probs = batched_er(k, nmin, nmax, pmin, pmax, seed)
    return Workload(f"batched_er_k{k}", int(gptr[-1]), u, v, {"graph_ptr": gptr, "p": probs})


def chung_lu_stream(seed: int = BASE_SEED + 5, n: int = 500_000, gamma: float = 2.3,
                    wmax: float = 2000.0, m_target: float = 2_000_000.0,
                    stream_edges: int = 1_000_000, batch_lo: float = 1e3, batch_hi: float = 1e5) -> Workload:
    """Base Chung-Lu graph plus a stream of new edges cut into log-uniform batches."""
    u, v, w = chung_lu(n, gamma, wmax, m_target, substream_seed(seed, 0))
    keys = canonical_keys(u, v)
    su, sv = edge_stream(n, w, keys, stream_edges, substream_seed(seed, 1))
    sizes, gaps = batch_schedule(stream_edges, batch_lo, batch_hi, substream_seed(seed, 2))
    return Workload(f"chunglu_n{n}_g{gamma}_stream{stream_edges}", n, u, v,
                    {"w": w, "stream_u": su, "stream_v": sv, "batch_sizes": sizes, "gaps": gaps})
