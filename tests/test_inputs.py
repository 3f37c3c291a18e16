"""The seeded synthetic inputs follow their stated recipes (host only)."""
import math

import numpy as np
import pytest

import graphgen


def test_seeded_and_deterministic():
    a = graphgen.er(400, 0.05, 11)
    b = graphgen.er(400, 0.05, 11)
    c = graphgen.er(400, 0.05, 12)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not (len(a[0]) == len(c[0]) and np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]))
    r1 = graphgen.rmat(10, 16 << 10, 0.57, 0.19, 0.19, 3)
    r2 = graphgen.rmat(10, 16 << 10, 0.57, 0.19, 0.19, 3)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])


def test_er_edge_count_and_simplicity():
    n, p = 2000, 0.01
    u, v = graphgen.er(n, p, 20010434)
    pairs = n * (n - 1) // 2
    mean, sd = pairs * p, math.sqrt(pairs * p * (1 - p))
    assert abs(len(u) - mean) < 5 * sd
    assert (u < v).all() and (u >= 0).all() and (v < n).all()       # one draw per pair i < j
    assert len(np.unique(u.astype(np.int64) * n + v)) == len(u)


def test_rmat_quadrant_probabilities():
    scale, a, b, c = 14, 0.57, 0.19, 0.19
    u, v = graphgen.rmat(scale, 16 << scale, a, b, c, 7)
    n = 1 << scale
    assert len(u) == 16 << scale and (u >= 0).all() and (u < n).all() and (v >= 0).all() and (v < n).all()
    m = len(u)
    for bit in (scale - 1, scale // 2, 0):       # every recursion level draws the same quadrant law
        top_u = (u >> bit) & 1
        top_v = (v >> bit) & 1
        sd = math.sqrt(m * 0.25)
        assert abs((top_u == 0).sum() - m * (a + b)) < 6 * sd
        assert abs((top_v == 0).sum() - m * (a + c)) < 6 * sd
        assert abs(((top_u == 1) & (top_v == 1)).sum() - m * (1 - a - b - c)) < 6 * sd


def test_chung_lu_weights_and_edges():
    n, gamma, wmax, m_target = 20000, 2.2, 300.0, 80000.0
    u, v, w = graphgen.chung_lu(n, gamma, wmax, m_target, 5)
    assert w.max() == pytest.approx(wmax, rel=1e-6)
    assert w.sum() == pytest.approx(2 * m_target, rel=1e-3)                 # Σw = 2m by bisection
    assert np.all(np.diff(w) <= 0)                                          # decreasing power law
    # w_i ∝ (i + i0)^(-1/(γ-1)): far from the head the log-log slope is -1/(γ-1)
    slope = math.log(w[10000] / w[1000]) / math.log(10001.0 / 1001.0)
    assert -1 / (gamma - 1) - 0.03 < slope < -1 / (gamma - 1) + 0.05
    assert abs(len(u) - m_target) < 0.05 * m_target
    assert (u != v).all()
    keys = np.minimum(u, v).astype(np.int64) * n + np.maximum(u, v)
    assert len(np.unique(keys)) == len(keys)


def test_planted_cliques_sizes():
    u, v = graphgen.planted_cliques(100000, 20, 20, 60, 9)
    # 20 cliques of size k in [20, 60] contribute k(k-1)/2 pairs each
    assert 20 * 190 <= len(u) <= 20 * 1770


def test_batched_graphs_are_disjoint_and_log_uniform():
    u, v, gptr, probs = graphgen.batched_er(256, 32, 2048, 0.1, 0.6, 13)
    sizes = np.diff(gptr)
    assert gptr[0] == 0 and (sizes >= 32).all() and (sizes <= 2048).all()
    assert ((probs >= 0.1) & (probs <= 0.6)).all()
    g_of = np.searchsorted(gptr, u, side="right") - 1
    assert np.array_equal(g_of, np.searchsorted(gptr, v, side="right") - 1)   # no edge between graphs
    lg = np.log(sizes)
    assert abs(lg.mean() - (math.log(32) + math.log(2048)) / 2) < 0.4          # log-uniform sizes


def test_edge_stream_rules():
    w = graphgen.chung_lu_stream(n=20000, m_target=80000, wmax=280.0, stream_edges=6000, batch_lo=300,
                                 batch_hi=3000)
    su, sv = w.extra["stream_u"], w.extra["stream_v"]
    n = w.n
    assert len(su) == 6000 and (su != sv).all()
    base = set((np.minimum(w.u, w.v).astype(np.int64) * n + np.maximum(w.u, w.v)).tolist())
    new = np.minimum(su, sv).astype(np.int64) * n + np.maximum(su, sv)
    assert len(np.unique(new)) == len(new)                                    # no repeats
    assert not any(k in base for k in new.tolist())                           # no base edges
    sizes = w.extra["batch_sizes"]
    assert sizes.sum() == 6000
    assert ((sizes[:-1] >= 300) & (sizes[:-1] <= 3000)).all() and 1 <= sizes[-1] <= 3000
    assert len(w.extra["gaps"]) == len(sizes) and (w.extra["gaps"] > 0).all()
