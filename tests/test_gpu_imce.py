"""GPU parity of incremental MCE (Section 5) against the CPU oracle."""
import itertools
import json
import os
import random

import numpy as np
import pytest

import graphgen
import oracle as O

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def hist_of(cliques):
    if not cliques:
        return []
    h = [0] * (max(len(c) for c in cliques) + 1)
    for c in cliques:
        h[len(c)] += 1
    return h


def set_hash(cliques, seed=0):
    return sum(O.clique_hash(list(c), seed) for c in cliques) % (1 << 64)


def check_delta(d, new_cl, del_cl, seed=0):
    assert d.new_count == len(new_cl) and d.sub_count == len(del_cl)
    assert d.new_hash == set_hash(new_cl, seed) and d.sub_hash == set_hash(del_cl, seed)
    assert list(d.new_hist) == hist_of(new_cl) and list(d.sub_hist) == hist_of(del_cl)


@pytest.mark.parametrize("fixture", ["fig3_worked_example.json", "removed_figure_example.json"])
def test_worked_examples(gpu_lib, fixture):
    mce = gpu_lib
    with open(os.path.join(GOLDEN, fixture)) as f:
        ex = json.load(f)
    idx = {str(v): i for i, v in enumerate(ex["vertices"])}
    n = len(idx)
    u = np.array([idx[str(a)] for a, b in ex["edges"]], np.int32)
    v = np.array([idx[str(b)] for a, b in ex["edges"]], np.int32)
    st = mce.Imce(mce.Graph(n, u, v))
    as_ids = lambda cl: sorted(tuple(sorted(idx[str(x)] for x in c)) for c in cl)  # noqa: E731
    assert st.cliques(64, 1024) == as_ids(ex["initial_cliques"])
    alive = set(as_ids(ex["initial_cliques"]))
    for b in ex["batches"]:
        bu = np.array([idx[str(a)] for a, c in b["add"]], np.int32)
        bv = np.array([idx[str(c)] for a, c in b["add"]], np.int32)
        d = st.add_edges(bu, bv)
        assert d.applied == len(b["add"]) and d.dropped == 0
        check_delta(d, as_ids(b["new"]), as_ids(b["subsumed"]))
        alive = (alive - set(as_ids(b["subsumed"]))) | set(as_ids(b["new"]))
        assert st.cliques(64, 1024) == sorted(alive)
        assert d.alive == len(alive)


@pytest.mark.parametrize("n", [4, 20, 70])
def test_complete_minus_edge(gpu_lib, n):
    mce = gpu_lib
    pairs = [p for p in itertools.combinations(range(n), 2) if p != (0, 1)]
    u = np.array([a for a, b in pairs], np.int32)
    v = np.array([b for a, b in pairs], np.int32)
    st = mce.Imce(mce.Graph(n, u, v))
    d = st.add_edges(np.array([1], np.int32), np.array([0], np.int32))
    assert d.new_count == 1 and d.sub_count == 2
    assert list(d.new_hist) == [0] * n + [1]
    assert st.cliques(8, 4096) == [tuple(range(n))]


@pytest.mark.parametrize("k", [3, 5, 7])
def test_moon_moser_plus_edge(gpu_lib, k):
    mce = gpu_lib
    parts = [list(range(3 * i, 3 * i + 3)) for i in range(k)]
    pairs = [(a, b) for i in range(k) for j in range(i + 1, k) for a in parts[i] for b in parts[j]]
    n = 3 * k
    st = mce.Imce(mce.Graph(n, np.array([a for a, b in pairs], np.int32), np.array([b for a, b in pairs], np.int32)))
    d = st.add_edges(np.array([0], np.int32), np.array([1], np.int32))
    assert d.new_count == 3 ** (k - 1) and d.sub_count == 2 * 3 ** (k - 1)
    assert d.alive == 2 * 3 ** (k - 1)


@pytest.mark.parametrize("seed", range(6))
def test_random_batches_match_oracle(gpu_lib, seed):
    mce = gpu_lib
    rng = random.Random(900 + seed)
    n = rng.randint(10, 120)
    p = rng.choice([0.05, 0.15, 0.3])
    u, v = graphgen.er(n, p, 900 + seed)
    og = O.Graph(n, u, v)
    ost = O.Imce(og, seed=seed)
    st = mce.Imce(mce.Graph(n, _t(u), _t(v)), seed=seed)
    for b in range(5):
        k = rng.randint(1, 60)
        bu = np.array([rng.randrange(n) for _ in range(k)], np.int32)
        bv = np.array([rng.randrange(n) for _ in range(k)], np.int32)
        rho, onew, odel = ost.add(bu, bv)
        d = st.add_edges(_t(bu), _t(bv)) if b % 2 else st.add_edges(bu, bv)
        assert d.applied == rho and d.dropped == k - rho
        check_delta(d, onew.cliques, odel.cliques, seed)
        assert st.cliques(1 << 16, 1 << 20) == ost.cliques().cliques


def test_invalid_batch_leaves_state(gpu_lib):
    mce = gpu_lib
    u, v = graphgen.er(50, 0.2, 4)
    st = mce.Imce(mce.Graph(50, u, v))
    before = st.cliques(4096, 65536)
    with pytest.raises(mce.MceError) as e:
        st.add_edges(np.array([1, 2], np.int32), np.array([3, 50], np.int32))
    assert e.value.status == mce.MCE_EINVAL
    assert st.cliques(4096, 65536) == before


def test_empty_and_all_dropped_batches(gpu_lib):
    mce = gpu_lib
    u, v = graphgen.er(40, 0.2, 5)
    st = mce.Imce(mce.Graph(40, u, v))
    d = st.add_edges(np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert d.applied == 0 and d.new_count == 0
    d = st.add_edges(np.array([3, u[0], v[0]], np.int32), np.array([3, v[0], u[0]], np.int32))
    assert d.applied == 0 and d.dropped == 3 and d.sub_count == 0


def test_chung_lu_stream_prefix(gpu_lib):
    """A scaled-down dynamic workload: Chung-Lu base graph plus stream batches."""
    mce = gpu_lib
    w = graphgen.chung_lu_stream(n=20000, m_target=80000, wmax=280.0, stream_edges=6000, batch_lo=300, batch_hi=3000)
    og = O.Graph(w.n, w.u, w.v)
    ost = O.Imce(og, threads=4)
    st = mce.Imce(mce.Graph(w.n, _t(w.u), _t(w.v)))
    su, sv = w.extra["stream_u"], w.extra["stream_v"]
    pos = 0
    for size in w.extra["batch_sizes"]:
        bu, bv = su[pos:pos + size], sv[pos:pos + size]
        pos += size
        rho, onew, odel = ost.add(bu, bv)
        d = st.add_edges(_t(bu), _t(bv))
        assert d.applied == rho
        check_delta(d, onew.cliques, odel.cliques)
    assert d.alive == ost.alive


# ---------------------------------------------------------------- Algorithm 8 beyond the warp's buffers

def _imce_vs_oracle(mce, n, pairs, add):
    u = np.array([a for a, b in pairs], np.int32)
    v = np.array([b for a, b in pairs], np.int32)
    st = mce.Imce(mce.Graph(n, _t(u), _t(v)))
    ost = O.Imce(O.Graph(n, u, v))
    au = np.array([a for a, b in add], np.int32)
    av = np.array([b for a, b in add], np.int32)
    rho, onew, odel = ost.add(au, av)
    d = st.add_edges(au, av)
    assert d.applied == rho
    check_delta(d, onew.cliques, odel.cliques)
    assert st.cliques(1 << 16, 1 << 20) == ost.cliques().cliques
    return d


def test_new_clique_over_256_vertices(gpu_lib):
    """K_300 minus (0, 1), then (0, 1) added: one new clique of 300 vertices
    subsumes K_300 - 0 and K_300 - 1 (the masks of Algorithm 8 run over the
    two endpoints only)."""
    n = 300
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n) if (i, j) != (0, 1)]
    d = _imce_vs_oracle(gpu_lib, n, pairs, [(0, 1)])
    assert (d.new_count, d.sub_count) == (1, 2)


def test_split_set_beyond_the_warp_buffer(gpu_lib):
    """Moon-Moser graph K_{3,...,3} with 8 parts plus every edge inside the
    parts: the graph becomes complete, and the one new clique subsumes all
    3^8 = 6,561 old cliques, more than Algorithm 8's split set holds in a
    warp's buffer (4,096), so the enumerating fallback finds them."""
    k = 8
    parts = [list(range(3 * i, 3 * i + 3)) for i in range(k)]
    pairs = [(a, b) for i in range(k) for j in range(i + 1, k) for a in parts[i] for b in parts[j]]
    add = [(p[0], p[1]) for p in parts] + [(p[0], p[2]) for p in parts] + [(p[1], p[2]) for p in parts]
    d = _imce_vs_oracle(gpu_lib, 3 * k, pairs, add)
    assert (d.new_count, d.sub_count) == (1, 3 ** k)


def test_more_than_512_new_edges_in_one_clique(gpu_lib):
    """40 isolated vertices, then all 780 edges among them: K_40 is new and
    subsumes the 40 singletons."""
    n = 40
    d = _imce_vs_oracle(gpu_lib, n, [], [(i, j) for i in range(n) for j in range(i + 1, n)])
    assert (d.new_count, d.sub_count) == (1, 40)
