"""GPU edge deletions (imce_remove_edges) against the CPU oracle.

Deletions reduce to additions (Section 5: G = (G - H) + H): the removed
cliques are the new cliques of adding H to G - H and the created cliques are
Algorithm 8's splits of the removed ones that are maximal in G - H.  The
oracle implements the same reduction and the plain set differences."""
import itertools
import random

import numpy as np
import pytest

import graphgen
import oracle as O

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _pairs_graph(mce, n, pairs):
    u = np.array([a for a, b in pairs], np.int32)
    v = np.array([b for a, b in pairs], np.int32)
    return mce.Graph(n, _t(u), _t(v)), O.Graph(n, u, v)


def _key(d):
    return (d.applied, d.dropped, d.new_count, d.new_hash, list(d.new_hist), d.sub_count, d.sub_hash,
            list(d.sub_hist), d.alive)


def _okey(k, rho, rem, cre, alive):
    return (rho, k - rho, cre.count, cre.hash, list(cre.hist), rem.count, rem.hash, list(rem.hist), alive)


@pytest.mark.parametrize("n", [3, 4, 9, 40])
def test_complete_graph_minus_an_edge(gpu_lib, n):
    """K_n minus (0, 2): K_n is removed, K_n - 0 and K_n - 2 are created."""
    mce = gpu_lib
    g, _ = _pairs_graph(mce, n, list(itertools.combinations(range(n), 2)))
    st = mce.Imce(g)
    d = st.remove_edges(np.array([2], np.int32), np.array([0], np.int32))
    assert d.applied == 1 and d.sub_count == 1 and d.new_count == 2
    assert list(d.sub_hist) == [0] * n + [1] and list(d.new_hist) == [0] * (n - 1) + [2]
    assert st.cliques(16, 1024) == sorted([tuple(x for x in range(n) if x != 0), tuple(x for x in range(n) if x != 2)])
    assert d.alive == 2


@pytest.mark.parametrize("k", [3, 5])
def test_moon_moser_minus_an_edge_between_parts(gpu_lib, k):
    """Deleting an edge between two parts of K_{3,...,3} removes the 3^(k-2)
    cliques through it and creates none."""
    mce = gpu_lib
    parts = [list(range(3 * i, 3 * i + 3)) for i in range(k)]
    pairs = [(a, b) for i in range(k) for j in range(i + 1, k) for a in parts[i] for b in parts[j]]
    g, _ = _pairs_graph(mce, 3 * k, pairs)
    st = mce.Imce(g)
    d = st.remove_edges(np.array([0], np.int32), np.array([3], np.int32))
    assert (d.sub_count, d.new_count, d.alive) == (3 ** (k - 2), 0, 3 ** k - 3 ** (k - 2))


def test_deleting_a_whole_star_leaves_singletons(gpu_lib):
    mce = gpu_lib
    n = 7
    g, _ = _pairs_graph(mce, n, [(0, i) for i in range(1, n)])
    st = mce.Imce(g)
    d = st.remove_edges(np.zeros(n - 1, np.int32), np.arange(1, n, dtype=np.int32))
    assert (d.applied, d.sub_count, d.new_count) == (n - 1, n - 1, n)
    assert st.cliques(64, 256) == [(i,) for i in range(n)]


@pytest.mark.parametrize("seed", range(6))
def test_random_add_and_delete_sequences(gpu_lib, seed):
    """Mixed batches of additions and deletions (with self loops, repeats,
    pairs that are not edges, and reversed pairs) against the oracle's state
    machine, batch by batch: summaries and the full clique list."""
    mce = gpu_lib
    rng = random.Random(9000 + seed)
    n = rng.choice([30, 60, 120])
    u, v = graphgen.er(n, rng.choice([0.1, 0.25, 0.4]), 70 + seed)
    g = mce.Graph(n, _t(u), _t(v))
    og = O.Graph(n, u, v)
    st, ost = mce.Imce(g), O.Imce(og)
    for b in range(8):
        k = rng.randint(1, 3 * n)
        bu = np.array([rng.randrange(n) for _ in range(k)], np.int32)
        bv = np.array([rng.randrange(n) for _ in range(k)], np.int32)
        if b % 2:
            # deletions: mostly edges of the current graph, both orders
            row, col = ost.graph_csr()
            src = np.repeat(np.arange(n), np.diff(row))
            if len(col):
                pick = np.array([rng.randrange(len(col)) for _ in range(k)])
                bu[: k // 2], bv[: k // 2] = col[pick[: k // 2]], src[pick[: k // 2]]
            rho, rem, cre = ost.remove(bu, bv)
            d = st.remove_edges(_t(bu), _t(bv)) if b % 4 == 1 else st.remove_edges(bu, bv)
            assert _key(d) == _okey(k, rho, rem, cre, ost.alive), b
        else:
            rho, new, sub = ost.add(bu, bv)
            d = st.add_edges(bu, bv)
            assert (d.applied, d.new_count, d.new_hash, d.sub_count, d.sub_hash, d.alive) == \
                (rho, new.count, new.hash, sub.count, sub.hash, ost.alive), b
        assert st.cliques(1 << 16, 1 << 20) == ost.cliques().cliques, b
        row_o, col_o = ost.graph_csr()
        row_g, col_g = st.graph().csr()
        assert np.array_equal(np.asarray(row_g), row_o) and np.array_equal(np.asarray(col_g), col_o), b


def test_delete_then_add_back(gpu_lib):
    """Deleting H and adding it back returns to the original clique set; the
    addition's new cliques are the deletion's removed ones."""
    mce = gpu_lib
    rng = random.Random(5)
    n = 80
    u, v = graphgen.er(n, 0.3, 8)
    g = mce.Graph(n, _t(u), _t(v))
    st = mce.Imce(g)
    start = st.cliques(1 << 16, 1 << 20)
    row, col = st.graph().csr()
    src = np.repeat(np.arange(n), np.diff(np.asarray(row)))
    pick = rng.sample(range(len(col)), 40)
    hu, hv = np.asarray(src)[pick].astype(np.int32), np.asarray(col)[pick].astype(np.int32)
    d1 = st.remove_edges(hu, hv)
    d2 = st.add_edges(hu, hv)
    assert (d2.new_count, d2.new_hash) == (d1.sub_count, d1.sub_hash)
    assert (d2.sub_count, d2.sub_hash) == (d1.new_count, d1.new_hash)
    assert st.cliques(1 << 16, 1 << 20) == start


def test_chung_lu_stream_deleted_again(gpu_lib):
    """A scaled dynamic workload: Chung-Lu base plus stream batches added,
    then the same batches deleted in reverse order, each step against the
    oracle; the graph ends where it started."""
    mce = gpu_lib
    w = graphgen.chung_lu_stream(n=20000, m_target=80000, wmax=280.0, stream_edges=6000, batch_lo=300,
                                 batch_hi=3000)
    og = O.Graph(w.n, w.u, w.v)
    ost = O.Imce(og, threads=4)
    st = mce.Imce(mce.Graph(w.n, _t(w.u), _t(w.v)))
    start = st.cliques(1 << 20, 1 << 22)
    su, sv = w.extra["stream_u"], w.extra["stream_v"]
    offs = np.concatenate([[0], np.cumsum(w.extra["batch_sizes"])])
    for i in range(len(offs) - 1):
        ost.add(su[offs[i]:offs[i + 1]], sv[offs[i]:offs[i + 1]], want_list=False)
        st.add_edges(_t(su[offs[i]:offs[i + 1]]), _t(sv[offs[i]:offs[i + 1]]))
    for i in reversed(range(len(offs) - 1)):
        bu, bv = su[offs[i]:offs[i + 1]], sv[offs[i]:offs[i + 1]]
        rho, rem, cre = ost.remove(bu, bv, want_list=False)
        d = st.remove_edges(_t(bu), _t(bv))
        assert _key(d) == _okey(len(bu), rho, rem, cre, ost.alive), i
    assert st.cliques(1 << 20, 1 << 22) == start


def test_invalid_or_failed_deletion_leaves_state(gpu_lib):
    mce = gpu_lib
    u, v = graphgen.er(60, 0.2, 4)
    st = mce.Imce(mce.Graph(60, _t(u), _t(v)))
    before = st.cliques(4096, 65536)
    with pytest.raises(mce.MceError) as e:
        st.remove_edges(np.array([u[0], 2], np.int32), np.array([v[0], 60], np.int32))
    assert e.value.status == mce.MCE_EINVAL
    assert st.cliques(4096, 65536) == before
    # every device allocation of the call made to fail in turn
    fails = 0
    try:
        for after in range(300):
            mce.debug_fail_alloc(after)
            try:
                st.remove_edges(u[:20], v[:20])
            except mce.MceError as err:
                assert err.status == mce.MCE_ENOMEM
                mce.debug_fail_alloc(-1)
                assert st.cliques(4096, 65536) == before
                fails += 1
                continue
            break
    finally:
        mce.debug_fail_alloc(-1)
    assert fails >= 10
    og = O.Graph(60, u, v)
    ost = O.Imce(og)
    ost.remove(u[:20], v[:20])
    assert st.cliques(4096, 65536) == ost.cliques().cliques


# ---------------------------------------------------------------- created cliques beyond the warp's buffers

def _remove_vs_oracle(mce, n, pairs, rem):
    u = np.array([a for a, b in pairs], np.int32)
    v = np.array([b for a, b in pairs], np.int32)
    st = mce.Imce(mce.Graph(n, _t(u), _t(v)))
    ost = O.Imce(O.Graph(n, u, v))
    ru = np.array([a for a, b in rem], np.int32)
    rv = np.array([b for a, b in rem], np.int32)
    rho, orem, ocre = ost.remove(ru, rv)
    d = st.remove_edges(ru, rv)
    assert _key(d) == _okey(len(ru), rho, orem, ocre, ost.alive)
    assert st.cliques(1 << 16, 1 << 20) == ost.cliques().cliques
    return d


def test_removed_clique_over_256_vertices(gpu_lib):
    """K_300 minus (0, 1): the removed clique has 300 vertices; Algorithm 8's
    masks run over the two endpoints only, so it splits into K_300 - 0 and
    K_300 - 1."""
    n = 300
    d = _remove_vs_oracle(gpu_lib, n, list(itertools.combinations(range(n), 2)), [(0, 1)])
    assert (d.sub_count, d.new_count, d.alive) == (1, 2, 2)


def test_created_set_beyond_the_warp_buffer(gpu_lib):
    """K_24 minus the 24 edges inside 8 parts of 3: the removed K_24 splits
    into the 3^8 = 6,561 maximal cliques of the Moon-Moser graph, more than
    the split set holds in a warp's buffer (4,096), so the enumerating
    fallback produces them."""
    k = 8
    parts = [list(range(3 * i, 3 * i + 3)) for i in range(k)]
    rem = [(p[0], p[1]) for p in parts] + [(p[0], p[2]) for p in parts] + [(p[1], p[2]) for p in parts]
    d = _remove_vs_oracle(gpu_lib, 3 * k, list(itertools.combinations(range(3 * k), 2)), rem)
    assert (d.sub_count, d.new_count) == (1, 3 ** k)
    assert list(d.new_hist) == [0] * k + [3 ** k]


def test_more_than_512_deleted_edges_in_one_clique(gpu_lib):
    """K_40 with all 780 edges deleted: K_40 is removed and the 40 singletons
    are created (the enumerating fallback takes cliques with more than 512
    deleted edges inside)."""
    n = 40
    pairs = list(itertools.combinations(range(n), 2))
    d = _remove_vs_oracle(gpu_lib, n, pairs, pairs)
    assert (d.sub_count, d.new_count, d.alive) == (1, n, n)


def test_cocktail_party_from_complete_graph(gpu_lib):
    """K_30 minus a perfect matching of 15 edges: the removed K_30 splits
    into the 2^15 = 32,768 maximal cliques of the cocktail-party graph, each
    of size 15 (enumerating fallback, record space grown on the way)."""
    n = 30
    rem = [(2 * i, 2 * i + 1) for i in range(n // 2)]
    d = _remove_vs_oracle(gpu_lib, n, list(itertools.combinations(range(n), 2)), rem)
    assert (d.sub_count, d.new_count, d.alive) == (1, 2 ** 15, 2 ** 15)


def test_more_than_256_endpoints_in_one_clique_is_refused(gpu_lib):
    """K_300 minus a perfect matching (300 endpoints of deleted edges inside
    the one removed clique) is beyond Algorithm 8's masks: MCE_ESTATE, and the
    graph and the clique set are unchanged."""
    mce = gpu_lib
    n = 300
    pairs = list(itertools.combinations(range(n), 2))
    g, _ = _pairs_graph(mce, n, pairs)
    st = mce.Imce(g)
    before = st.cliques(16, 1024)
    row0, col0 = st.graph().csr()
    with pytest.raises(mce.MceError) as e:
        st.remove_edges(np.arange(0, n, 2, dtype=np.int32), np.arange(1, n, 2, dtype=np.int32))
    assert e.value.status == mce.MCE_ESTATE
    assert st.cliques(16, 1024) == before
    row1, col1 = st.graph().csr()
    assert np.array_equal(np.asarray(row0), np.asarray(row1)) and np.array_equal(np.asarray(col0), np.asarray(col1))
