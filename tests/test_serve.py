"""Host logic of the continuous-batching service (`serve.py`) with a fake
backend: results reach the right request whether it runs alone or in a mix,
requests join the open group of their key (while it builds, and while its
solve session runs), cache misses of different keys are built in one batch,
the accounted device bytes never exceed the budget, idle entries are evicted
least recently used first, and failures reach the caller."""
import threading
import time

import numpy as np
import pytest

from paper_2111_11058_gb300 import serve as S


class FakeBackend:
    def __init__(self, build_s=0.03, solve_s=0.01, fail_names=(), s=8):
        self.s = s                                   # generating waves per cell (bounds L_m)
        self.build_s, self.solve_s = build_s, solve_s
        self.fail = set(fail_names)
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        self.building = 0
        self.max_building = 0
        self.builds = []
        self.freed = []
        self.build_many_calls = []
        self.sessions = []

    def make_stream(self):
        return object()

    def _enter(self):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)

    def _leave(self):
        with self.lock:
            self.active -= 1

    def build(self, sc, freq, st):
        self._enter()
        with self.lock:
            self.building += 1
            self.max_building = max(self.max_building, self.building)
        try:
            time.sleep(self.build_s)
            if sc.name in self.fail:
                raise RuntimeError("build failed: " + sc.name)
            self.builds.append((sc.name, freq))
            return (sc.name, freq), S.estimate_n(sc, self.s)   # the estimate is an upper bound
        finally:
            with self.lock:
                self.building -= 1
            self._leave()

    def build_many(self, items, st):
        self.build_many_calls.append([(sc.name, f) for sc, f in items])
        return [self.build(sc, f, st) for sc, f in items]

    def open_session(self, handle, exc, st):
        s = FakeSession(self, handle, exc)
        self.sessions.append(s)
        return s

    def solve(self, handle, exc, st):
        self._enter()
        try:
            time.sleep(self.solve_s)
            return expected(handle, exc), np.full(exc.shape[0], 3, np.int32)
        finally:
            self._leave()

    def free(self, handle):
        self.freed.append(handle)


class FakeSession:
    """A solve that takes joins at 'block boundaries' (every tenth of the solve time) until it finishes."""

    def __init__(self, be, handle, exc):
        self.be, self.handle = be, handle
        self.exc = [exc]
        self.n = exc.shape[0]
        self.queue = []
        self.closed = False
        self.joined = 0
        self.lock = threading.Lock()

    def join(self, exc):
        with self.lock:
            if self.closed or self.n + exc.shape[0] > S.MAX_BLOCK_RHS:
                return None
            slot, self.n = self.n, self.n + exc.shape[0]
            self.queue.append(exc)
            self.joined += 1
            return slot

    def run(self):
        self.be._enter()
        try:
            t_end = time.perf_counter() + self.be.solve_s
            while True:
                time.sleep(self.be.solve_s / 10)
                with self.lock:
                    if self.queue:
                        self.exc += self.queue
                        self.queue = []
                        t_end = max(t_end, time.perf_counter() + self.be.solve_s / 2)
                    elif time.perf_counter() >= t_end:
                        self.closed = True
                        break
            allx = np.concatenate(self.exc, axis=0)
            return expected(self.handle, allx), np.full(allx.shape[0], 3, np.int32)
        finally:
            self.be._leave()

    def free(self):
        pass


def expected(handle, exc):
    name, freq = handle
    h = sum(map(ord, name))
    return np.stack([freq * exc[:, 0] + h, exc[:, 1] * exc[:, 2] + freq], axis=1)


def scat(name, nt=40, ncell=4):
    return S.Scatterer(name, np.zeros((nt // 2 + 2, 3)), np.zeros((nt, 3), np.int32), 2.0, ncell)


def req(sc, freq, nrhs, seed):
    rng = np.random.default_rng(seed)
    return S.Request(sc, freq, rng.uniform(0, 3, size=(nrhs, 3)))


def one_key_bytes(sc, nrhs=128, s=8):
    n = S.estimate_n(sc, s)
    return (S.entry_bytes(sc.nt, sc.ne, n, sc.ncell) + S.build_transient_bytes(sc.nt, sc.ne, n)
            + S.solve_bytes(n, nrhs, sc.ne))


def test_results_route_alone_and_in_mix():
    scs = [scat("a"), scat("b"), scat("c")]
    reqs = [req(scs[i % 3], 1.0 + 0.1 * (i % 2), 1 + i % 7, i) for i in range(30)]
    be = FakeBackend()
    srv = S.Server(be, hbm_budget=10**12, n_streams=3)
    futs = [srv.submit(r) for r in reqs]
    res = [f.result(timeout=30) for f in futs]
    srv.close()
    for r, out in zip(reqs, res):
        np.testing.assert_array_equal(out.rcs, expected(r.key, r.exc))   # same as alone
        assert out.rcs.shape == (r.nrhs, 2) and out.rid == r.rid
    assert be.max_active >= 2                     # batches ran concurrently
    assert len(set(be.builds)) == len(be.builds)  # each (scatterer, frequency) built once
    assert srv.hits + srv.misses == sum(len(b["keys"]) for b in srv.log)   # one count per key group


def test_requests_join_the_group_being_built():
    sc = scat("a")
    be = FakeBackend(build_s=0.2)
    srv = S.Server(be, hbm_budget=10**12, n_streams=1)
    first = srv.submit(req(sc, 1.0, 4, 0))           # occupies the only worker (build)
    time.sleep(0.05)
    rest = [srv.submit(req(sc, 1.0, 40, k)) for k in range(1, 6)]   # 200 RHS arrive during the build
    res = [f.result(timeout=30) for f in [first] + rest]
    srv.close()
    for k, r in enumerate(res):
        np.testing.assert_array_equal(r.rcs, expected((sc.name, 1.0), req(sc, 1.0, 4 if k == 0 else 40, k).exc))
    assert len({r.batch_id for r in res[:4]}) == 1 and res[0].batch_rhs == 124   # 3 joined, cut at 128 RHS
    assert {r.batch_rhs for r in res[4:]} == {80} and res[4].batch_id == res[5].batch_id
    assert all(r.cache_hit for r in res[4:]) and not res[0].cache_hit
    assert srv.log[0]["joined"] == 3 and srv.log[0]["requests"] == 4


def test_request_joins_a_running_solve():
    sc = scat("a")
    be = FakeBackend(build_s=0.01, solve_s=0.4)
    srv = S.Server(be, hbm_budget=10**12, n_streams=1)
    a = srv.submit(req(sc, 1.0, 8, 0))
    time.sleep(0.15)                                  # built; its session runs
    b = srv.submit(req(sc, 1.0, 8, 1))
    ra, rb = a.result(timeout=30), b.result(timeout=30)
    srv.close()
    np.testing.assert_array_equal(rb.rcs, expected((sc.name, 1.0), req(sc, 1.0, 8, 1).exc))
    np.testing.assert_array_equal(ra.rcs, expected((sc.name, 1.0), req(sc, 1.0, 8, 0).exc))
    assert ra.batch_id == rb.batch_id and rb.batch_rhs == 16
    assert be.sessions[0].joined == 1 and len(srv.log) == 1 and srv.log[0]["joined"] == 1


def test_cache_misses_of_other_keys_build_together():
    scs = [scat("a"), scat("b"), scat("c"), scat("d")]
    be = FakeBackend(build_s=0.1)
    srv = S.Server(be, hbm_budget=10**12, n_streams=1)
    futs = [srv.submit(req(scs[i], 1.0, 4, i)) for i in range(4)]   # a starts alone; b, c and d wait
    futs.append(srv.submit(req(scs[0], 1.0, 2, 9)))                 # joins the open group of a
    res = [f.result(timeout=30) for f in futs]
    srv.close()
    for i, r in enumerate(res[:4]):
        np.testing.assert_array_equal(r.rcs, expected((scs[i].name, 1.0), req(scs[i], 1.0, 4, i).exc))
    np.testing.assert_array_equal(res[4].rcs, expected(("a", 1.0), req(scs[0], 1.0, 2, 9).exc))
    assert be.build_many_calls == [[("b", 1.0), ("c", 1.0), ("d", 1.0)]]
    assert [len(b["keys"]) for b in srv.log] == [1, 3] and srv.log[1]["requests"] == 3
    assert srv.log[0]["joined"] == 1 and res[4].batch_id == res[0].batch_id


def test_budget_admission_and_lru_eviction():
    scs = [scat("a", nt=4000), scat("b", nt=4000), scat("c", nt=4000)]   # GB-sized entries
    n = S.estimate_n(scs[0], 1000)
    # room for one build (entry, transient, solve) plus half an entry: one resident entry at a time
    budget = one_key_bytes(scs[0], s=1000) + S.entry_bytes(scs[0].nt, scs[0].ne, n, scs[0].ncell) // 2
    be = FakeBackend(s=1000)
    srv = S.Server(be, hbm_budget=budget, n_streams=3)
    order = [0, 1, 0, 2, 1, 0]
    futs = []
    for k, i in enumerate(order):
        futs.append(srv.submit(req(scs[i], 1.0, 8, k)))
    res = [f.result(timeout=60) for f in futs]
    srv.close()
    for k, i in enumerate(order):
        np.testing.assert_array_equal(res[k].rcs, expected((scs[i].name, 1.0), req(scs[i], 1.0, 8, k).exc))
    assert srv.peak_bytes <= budget
    assert srv.evictions >= 2
    assert be.max_building == 1                      # the budget serialised the builds
    assert len(be.freed) >= srv.evictions


def test_oversize_and_too_many_rhs_rejected():
    sc = scat("a")
    be = FakeBackend()
    srv = S.Server(be, hbm_budget=one_key_bytes(sc, nrhs=4) // 2, n_streams=2)
    with pytest.raises(MemoryError):
        srv.submit(req(sc, 1.0, 4, 0)).result(timeout=10)
    with pytest.raises(ValueError):
        srv.submit(req(sc, 1.0, S.MAX_BLOCK_RHS + 1, 1)).result(timeout=10)
    srv.close()


def test_failed_build_reaches_caller_and_is_not_cached():
    bad, good = scat("bad"), scat("good")
    be = FakeBackend(fail_names={"bad"})
    srv = S.Server(be, hbm_budget=10**12, n_streams=2)
    f1 = srv.submit(req(bad, 1.0, 3, 0))
    f2 = srv.submit(req(good, 1.0, 3, 1))
    with pytest.raises(RuntimeError):
        f1.result(timeout=10)
    assert f2.result(timeout=10).rcs.shape == (3, 2)
    assert ("bad", 1.0) not in srv.cache
    be.fail.clear()
    assert srv.submit(req(bad, 1.0, 2, 2)).result(timeout=10).rcs.shape == (2, 2)   # rebuilt
    srv.close()


def test_summary_statistics():
    assert S.overlap_ms([(0, 2), (1, 3), (5, 6)]) == pytest.approx(1.0)
    assert S.overlap_ms([(0, 1), (1, 2)]) == 0.0
    off = S.poisson_arrivals(100.0, 2000, seed=1)
    assert np.all(np.diff(off) > 0) and abs(off[-1] / 2000 - 0.01) < 0.002
