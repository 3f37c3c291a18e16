"""Serving loop on the GPU: a tenant's results are the same whether its
batches are served alone or mixed with other tenants' batches, and they
equal the oracle's incremental results."""
import random

import numpy as np
import pytest

import graphgen
import oracle as O

pytestmark = pytest.mark.gpu


def hist_of(cliques):
    if not cliques:
        return []
    h = [0] * (max(len(c) for c in cliques) + 1)
    for c in cliques:
        h[len(c)] += 1
    return h


def set_hash(cliques):
    return sum(O.clique_hash(list(c)) for c in cliques) % (1 << 64)


def tenant_stream(seed, n, p, batches):
    rng = random.Random(seed)
    u, v = graphgen.er(n, p, seed)
    bs = []
    for _ in range(batches):
        k = rng.randint(1, 80)
        bs.append((np.array([rng.randrange(n) for _ in range(k)], np.int32),
                   np.array([rng.randrange(n) for _ in range(k)], np.int32)))
    return n, u, v, bs


def summary(d):
    return (d.applied, d.dropped, d.new_count, d.new_hash, d.sub_count, d.sub_hash, list(d.new_hist),
            list(d.sub_hist), d.alive)


def serve(mce, streams, slots, mem_budget=0, interleave=True):
    srv = mce.Server(slots=slots, mem_budget=mem_budget)
    ts = [srv.add_tenant(mce.Graph(n, u, v)) for n, u, v, _ in streams]
    ids = {t: [] for t in ts}
    order = [(t, j) for j in range(max(len(s[3]) for s in streams)) for t in ts] if interleave else \
        [(t, j) for t in ts for j in range(len(streams[t][3]))]
    for t, j in order:
        if j < len(streams[t][3]):
            ids[t].append(srv.submit(t, *streams[t][3][j]))
    out = {t: [srv.wait(i) for i in ids[t]] for t in ts}
    srv.drain()
    final = {t: srv.cliques(t, 1 << 16, 1 << 20) for t in ts}
    st = srv.stats()
    srv.close()
    return out, final, st


@pytest.fixture(scope="module")
def streams():
    return [tenant_stream(600 + i, n, p, 6) for i, (n, p) in enumerate([(90, 0.2), (140, 0.1), (60, 0.35)])]


def test_alone_and_mixed_are_identical_and_match_oracle(gpu_lib, streams):
    mce = gpu_lib
    alone, alone_final, _ = serve(mce, streams[:1], slots=1)
    mixed, mixed_final, st = serve(mce, streams, slots=4)
    assert [summary(i.delta) for i in alone[0]] == [summary(i.delta) for i in mixed[0]]
    assert alone_final[0] == mixed_final[0]
    assert st["completed"] == sum(len(s[3]) for s in streams) and st["failed"] == 0
    assert st["p50_ms"] <= st["p99_ms"]
    for t, (n, u, v, bs) in enumerate(streams):
        ost = O.Imce(O.Graph(n, u, v))
        for info, (bu, bv) in zip(mixed[t], bs):
            rho, onew, odel = ost.add(bu, bv)
            d = info.delta
            assert info.status == 0 and d.applied == rho
            assert (d.new_count, d.new_hash, list(d.new_hist)) == (len(onew.cliques), set_hash(onew.cliques),
                                                                   hist_of(onew.cliques))
            assert (d.sub_count, d.sub_hash, list(d.sub_hist)) == (len(odel.cliques), set_hash(odel.cliques),
                                                                   hist_of(odel.cliques))
        assert mixed_final[t] == ost.cliques().cliques


def test_tight_memory_budget_serialises_without_changing_results(gpu_lib, streams):
    mce = gpu_lib
    free_run, _, _ = serve(mce, streams, slots=4)
    tight, _, st = serve(mce, streams, slots=4, mem_budget=1)
    assert st["max_in_flight"] == 1
    for t in free_run:
        assert [summary(i.delta) for i in free_run[t]] == [summary(i.delta) for i in tight[t]]
