"""Scheduler of the serving loop (imce_server_*) on the host: the batch runner
is replaced by a Python hook, so ordering, admission and the latency
statistics are checked without a GPU."""
import threading
import time

import numpy as np
import pytest

mce = pytest.importorskip("paper_2001_11433_gb300")


class Recorder:
    """Hook that sleeps, records the execution order and the concurrency."""

    def __init__(self, sleep_s=0.02, fail=()):
        self.lock = threading.Lock()
        self.order, self.active, self.max_active = [], set(), 0
        self.peak_same_tenant = 0
        self.sleep_s, self.fail = sleep_s, set(fail)

    def __call__(self, tenant, u, v):
        tag = int(u[0]) if len(u) else -1
        with self.lock:
            self.peak_same_tenant = max(self.peak_same_tenant, sum(1 for t, _ in self.active if t == tenant) + 1)
            self.active.add((tenant, tag))
            self.max_active = max(self.max_active, len(self.active))
            self.order.append((tenant, tag))
        time.sleep(self.sleep_s)
        with self.lock:
            self.active.discard((tenant, tag))
        if tag in self.fail:
            return mce.MCE_ESTATE, 0, 0
        return mce.MCE_OK, len(u), 1


@pytest.fixture
def lib():
    try:
        mce.load()
    except Exception as e:  # noqa: BLE001
        pytest.skip(f"library not built: {e}")
    return mce


def batch(tag, k=4):
    return np.full(k, tag, np.int32), np.full(k, tag + 1, np.int32)


def test_tenant_order_and_cross_tenant_concurrency(lib):
    rec = Recorder(sleep_s=0.1)
    srv = lib.Server(slots=4, execute=rec)
    ts = [srv.add_tenant() for _ in range(4)]
    ids = []
    for j in range(5):
        for t in ts:
            ids.append(srv.submit(t, *batch(100 * t + j)))
    srv.drain()
    for t in ts:
        assert [tag for tt, tag in rec.order if tt == t] == [100 * t + j for j in range(5)]
    assert rec.peak_same_tenant == 1          # a tenant never runs two batches at once
    assert rec.max_active > 1                 # different tenants do
    st = srv.stats()
    assert st["completed"] == 20 and st["failed"] == 0 and st["edges"] == 80
    assert st["max_in_flight"] == rec.max_active
    srv.close()


def test_memory_admission(lib):
    # execute mode: tenants have n = nnz = 0, so a batch of k pairs projects
    # mem_fixed + 16 + 112 k bytes
    rec = Recorder(sleep_s=0.1)
    srv = lib.Server(slots=4, execute=rec, mem_fixed=1000, mem_budget=1600)
    ts = [srv.add_tenant() for _ in range(4)]
    for t in ts:
        srv.submit(t, *batch(10 * t, k=2))        # 1240 bytes each: one at a time
    srv.drain()
    assert rec.max_active == 1 and srv.stats()["max_in_flight"] == 1
    srv.close()
    rec = Recorder(sleep_s=0.1)
    srv = lib.Server(slots=4, execute=rec, mem_fixed=1000, mem_budget=2600)
    ts = [srv.add_tenant() for _ in range(4)]
    for t in ts:
        srv.submit(t, *batch(10 * t, k=2))
    srv.drain()
    assert rec.max_active == 2
    assert srv.stats()["peak_reserved"] == 2 * 1240
    srv.close()


def test_oversized_batch_runs_alone_and_holds_later_ones(lib):
    rec = Recorder(sleep_s=0.2)
    srv = lib.Server(slots=4, execute=rec, mem_fixed=100, mem_budget=300)
    a, b, c = (srv.add_tenant() for _ in range(3))
    ra = srv.submit(a, *batch(1, k=1))            # 228 bytes, in flight first
    time.sleep(0.01)
    rb = srv.submit(b, *batch(2, k=10))           # 1236 bytes > budget: waits until alone
    rc = srv.submit(c, *batch(3, k=0))            # 116 bytes: fits, but held behind b
    ia, ib, ic = srv.wait(ra), srv.wait(rb), srv.wait(rc)
    assert ib.admit_ms >= ia.done_ms - 1e-6       # b admitted only when nothing else was in flight
    assert ic.admit_ms >= ib.admit_ms             # c not admitted ahead of the older b
    srv.close()


def test_arrival_times_and_percentiles(lib):
    rec = Recorder(sleep_s=0.005)
    srv = lib.Server(slots=2, execute=rec)
    t = srv.add_tenant()
    srv.reset_clock()
    arrivals = [0.0, 5.0, 40.0, 45.0, 80.0, 120.0, 121.0, 122.0]
    ids = [srv.submit(t, *batch(j), arrival_ms=a) for j, a in enumerate(arrivals)]
    infos = [srv.wait(i) for i in ids]
    for inf, a in zip(infos, arrivals):
        assert inf.arrival_ms == pytest.approx(a, abs=0.5) or inf.arrival_ms >= a
        assert inf.admit_ms >= a - 1e-6
        assert inf.done_ms >= inf.admit_ms + 4.0
    for x, y in zip(infos, infos[1:]):
        assert y.admit_ms >= x.done_ms - 1e-6     # one tenant: strictly serial
    lat = np.sort([i.done_ms - i.arrival_ms for i in infos])
    st = srv.stats()
    nearest = lambda q: lat[max(int(np.ceil(q * len(lat))), 1) - 1]  # noqa: E731
    assert st["p50_ms"] == pytest.approx(nearest(0.5), abs=1e-6)
    assert st["p99_ms"] == pytest.approx(nearest(0.99), abs=1e-6)
    assert st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    srv.close()


def test_failed_batch_is_reported_and_later_batches_run(lib):
    rec = Recorder(sleep_s=0.001, fail={7})
    srv = lib.Server(slots=2, execute=rec)
    t = srv.add_tenant()
    ids = [srv.submit(t, *batch(j)) for j in (5, 7, 9)]
    infos = [srv.wait(i) for i in ids]
    assert [i.status for i in infos] == [0, mce.MCE_ESTATE, 0]
    st = srv.stats()
    assert st["completed"] == 2 and st["failed"] == 1
    srv.close()


def test_bad_arguments(lib):
    srv = lib.Server(slots=1, execute=Recorder())
    with pytest.raises(mce.MceError):
        srv.submit(3, *batch(1))                  # unknown tenant
    with pytest.raises(mce.MceError):
        srv.wait(99)
    srv.close()
    with pytest.raises(mce.MceError):
        lib.Server(slots=0, execute=Recorder())
