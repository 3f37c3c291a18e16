"""Pins for the oracle's edge-deletion maintenance (the reduction of a
deletion batch to the incremental step of Section 5).  CPU only."""
import itertools
import random

import numpy as np
import pytest

import oracle as O
from test_oracle import brute_force_maximal_cliques, complete_multipartite, edges_of, graph, random_pairs


def test_canonical_deletion_keeps_existing_edges_once():
    g = graph(5, [(0, 1), (1, 2), (2, 3)])
    hu, hv = O.canonical_deletion(g, [1, 2, 0, 4, 1, 3], [0, 1, 1, 4, 2, 4])
    # (1,0) kept as (0,1); (2,1) kept as (1,2); repeat (0,1), self loop, repeat (1,2), non-edge dropped
    assert list(zip(hu.tolist(), hv.tolist())) == [(0, 1), (1, 2)]
    with pytest.raises(ValueError):
        O.canonical_deletion(g, [0], [5])


@pytest.mark.parametrize("n", [3, 4, 7, 12])
def test_complete_graph_minus_an_edge(n):
    """Deleting (a, b) from K_n removes K_n and creates K_n - a and K_n - b."""
    g = graph(n, list(itertools.combinations(range(n), 2)))
    hu, hv = O.canonical_deletion(g, [2], [0])
    for fn in (O.dmce_alg, O.dmce_diff):
        rem, cre = fn(g, hu, hv)
        assert rem.cliques == [tuple(range(n))]
        assert cre.cliques == sorted([tuple(x for x in range(n) if x != 0), tuple(x for x in range(n) if x != 2)])


@pytest.mark.parametrize("k", [3, 4, 5])
def test_moon_moser_minus_an_edge_between_parts(k):
    """Moon–Moser graph K_{3,...,3}: its 3^k maximal cliques take one vertex
    per part.  Deleting an edge (a, b) between two parts removes the 3^(k-2)
    cliques through a and b and creates none: K - a is extended by any other
    vertex of a's part."""
    n, pairs, _ = complete_multipartite([3] * k)
    g = graph(n, pairs)
    hu, hv = O.canonical_deletion(g, [0], [3])
    rem, cre = O.dmce_alg(g, hu, hv)
    assert rem.count == 3 ** (k - 2) and cre.count == 0
    assert all(0 in c and 3 in c for c in rem.cliques)
    assert O.ttt_whole(g.minus(hu, hv)).count == 3 ** k - 3 ** (k - 2)


def test_deleting_every_edge_of_a_star_leaves_singletons():
    n = 6
    g = graph(n, [(0, i) for i in range(1, n)])
    hu, hv = O.canonical_deletion(g, [0] * (n - 1), list(range(1, n)))
    rem, cre = O.dmce_alg(g, hu, hv)
    assert rem.cliques == [(0, i) for i in range(1, n)]
    assert cre.cliques == [(i,) for i in range(n)]


@pytest.mark.parametrize("seed", range(12))
def test_small_random_against_brute_force(seed):
    """Both modes against exhaustive enumeration of C(G) and C(G - H)."""
    rng = random.Random(4400 + seed)
    n = rng.randint(4, 13)
    pairs = random_pairs(n, rng.choice([0.3, 0.5, 0.75]), rng)
    if not pairs:
        pairs = [(0, 1)]
    g = graph(n, pairs)
    batch = rng.sample(pairs, rng.randint(1, len(pairs)))
    hu, hv = O.canonical_deletion(g, [a for a, b in batch], [b for a, b in batch])
    left = sorted(set(pairs) - set(zip(hu.tolist(), hv.tolist())))
    before = set(brute_force_maximal_cliques(n, pairs))
    after = set(brute_force_maximal_cliques(n, left))
    for fn in (O.dmce_alg, O.dmce_diff):
        rem, cre = fn(g, hu, hv)
        assert rem.cliques == sorted(before - after)
        assert cre.cliques == sorted(after - before)


@pytest.mark.parametrize("seed", range(6))
def test_created_cliques_are_splits_of_removed_ones(seed):
    rng = random.Random(800 + seed)
    n = 40
    pairs = random_pairs(n, 0.3, rng)
    g = graph(n, pairs)
    batch = rng.sample(pairs, 15)
    hu, hv = O.canonical_deletion(g, [a for a, b in batch], [b for a, b in batch])
    rem, cre = O.dmce_alg(g, hu, hv)
    deleted = set(zip(hu.tolist(), hv.tolist()))
    for c in rem.cliques:
        assert any((a, b) in deleted for a, b in itertools.combinations(c, 2))
    for c in cre.cliques:
        assert not any((a, b) in deleted for a, b in itertools.combinations(c, 2))
        assert any(set(c) < set(r) for r in rem.cliques)
    r2, c2 = O.dmce_diff(g, hu, hv)
    assert (rem.count, rem.hash, cre.count, cre.hash) == (r2.count, r2.hash, c2.count, c2.hash)


def test_delete_then_add_back_swaps_the_roles():
    """Deleting H and adding it back: the addition's new cliques are the
    deletion's removed ones and its subsumed cliques the created ones."""
    rng = random.Random(31)
    n = 60
    pairs = random_pairs(n, 0.2, rng)
    g = graph(n, pairs)
    st = O.Imce(g)
    batch = rng.sample(pairs, 25)
    bu, bv = edges_of(batch)
    total = st.alive
    rho, rem, cre = st.remove(bu, bv)
    assert rho == 25
    assert st.alive == total - rem.count + cre.count
    rho2, new, sub = st.add(bu, bv)
    assert rho2 == 25
    assert new.cliques == rem.cliques and sub.cliques == cre.cliques
    assert st.alive == total


@pytest.mark.parametrize("seed", range(4))
def test_mixed_batches_keep_the_invariant(seed):
    """Alternating additions and deletions on one state: the cliques kept
    always equal a recomputation on the current graph."""
    rng = random.Random(9000 + seed)
    n = 50
    pairs = set(random_pairs(n, 0.15, rng))
    st = O.Imce(graph(n, sorted(pairs)))
    for step in range(6):
        if step % 2:
            cand = sorted(pairs)
            batch = rng.sample(cand, min(len(cand), rng.randint(1, 20)))
            bu, bv = edges_of(batch)
            rho, _, _ = st.remove(np.concatenate([bu, [3]]), np.concatenate([bv, [3]]))   # + a self loop
            assert rho == len(batch)
            pairs -= set(batch)
        else:
            batch = [tuple(sorted(rng.sample(range(n), 2))) for _ in range(rng.randint(1, 20))]
            bu, bv = edges_of(batch)
            st.add(bu, bv)
            pairs |= set(batch)
        expect = O.ttt_whole(graph(n, sorted(pairs)), want_list=True)
        assert st.cliques().cliques == expect.cliques
        assert st.alive == expect.count
