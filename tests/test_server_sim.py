"""CPU tests of the serving scheduler (continuous batching, admission by
memory, back-pressure, bounded waits) through the C ABI, with the library's
simulated backend: the same scheduler, no GPU, chunks "take" a set time per
(token, row) item.  Failures are made on the host only."""
import threading
import time

import pytest

from paper_2505_07329_b300 import build, phe


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    phe.lib()


def _server(**kw):
    cfg = dict(mem_budget_bytes=1 << 20, chunk_tokens=4, max_active=16, max_jobs_per_iteration=16,
               max_queue=64, wait_timeout_ms=5000, simulate=True, sim_ns_per_item=2000.0)
    cfg.update(kw)
    return phe.phe_server_create(None, **cfg)


def test_all_requests_complete_with_latencies():
    srv = _server()
    try:
        ids = [phe.phe_server_submit(srv, None, 0, T, sim_rows=rows) for T, rows in [(10, 8), (3, 2), (17, 5), (0, 4)]]
        lats = [phe.phe_server_wait(srv, i, 10000) for i in ids]
        st = phe.phe_server_stats(srv)
        assert st["completed"] == 4 and st["failed"] == 0
        assert st["tokens_completed"] == 30
        assert lats[3] == 0.0  # T = 0 completes at submission
        assert 0 <= st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        assert st["reserved_bytes"] == 0
    finally:
        phe.phe_server_destroy(srv)


def test_admission_never_exceeds_the_memory_budget():
    # simulated chunk bytes: tn*L*N*8 + tn*rows*N*4 + tn*rows*4 with N = L = 1
    rows, chunk = 10, 4
    one_chunk = chunk * 8 + chunk * rows * 4 + chunk * rows * 4
    srv = _server(mem_budget_bytes=2 * one_chunk, chunk_tokens=chunk)
    try:
        ids = [phe.phe_server_submit(srv, None, 0, 12, sim_rows=rows) for _ in range(6)]
        for i in ids:
            phe.phe_server_wait(srv, i, 20000)
        st = phe.phe_server_stats(srv)
        assert st["peak_reserved_bytes"] <= 2 * one_chunk
        assert st["peak_reserved_bytes"] >= one_chunk
        # 6 requests x 3 chunks, at most 2 chunks per iteration
        assert st["iterations"] >= 9
    finally:
        phe.phe_server_destroy(srv)


def test_request_larger_than_the_budget_is_refused():
    srv = _server(mem_budget_bytes=100)
    try:
        with pytest.raises(phe.PheError) as ei:
            phe.phe_server_submit(srv, None, 0, 64, sim_rows=1000)
        assert ei.value.status == phe.PHE_ENOMEM
    finally:
        phe.phe_server_destroy(srv)


def test_late_short_request_overtakes_a_long_one():
    # continuous batching: a request that arrives while a long one runs joins
    # at the next iteration instead of waiting for the long one to finish
    srv = _server(chunk_tokens=1, sim_ns_per_item=1e6)  # 1 ms per (token,row)
    try:
        long_id = phe.phe_server_submit(srv, None, 0, 200, sim_rows=1)  # ~200 ms
        time.sleep(0.03)
        short_id = phe.phe_server_submit(srv, None, 0, 2, sim_rows=1)
        phe.phe_server_wait(srv, short_id, 10000)
        done, _ = phe.phe_server_poll(srv, long_id)
        assert done == 0, "the short request should finish while the long one is still running"
        phe.phe_server_wait(srv, long_id, 10000)
    finally:
        phe.phe_server_destroy(srv)


def test_queue_full_gives_back_pressure():
    srv = _server(max_active=1, max_queue=2, chunk_tokens=1, sim_ns_per_item=2e5)
    try:
        ids = [phe.phe_server_submit(srv, None, 0, 1000, sim_rows=1)]  # ~200 ms
        time.sleep(0.02)  # the first becomes active
        ids += [phe.phe_server_submit(srv, None, 0, 5, sim_rows=1) for _ in range(2)]
        with pytest.raises(phe.PheError) as ei:
            phe.phe_server_submit(srv, None, 0, 5, sim_rows=1)
        assert ei.value.status == phe.PHE_EBUSY
        for i in ids:
            phe.phe_server_wait(srv, i, 20000)
    finally:
        phe.phe_server_destroy(srv)


def test_wait_is_bounded():
    srv = _server(chunk_tokens=1, sim_ns_per_item=1e6)
    try:
        rid = phe.phe_server_submit(srv, None, 0, 300, sim_rows=1)
        t0 = time.monotonic()
        with pytest.raises(phe.PheError) as ei:
            phe.phe_server_wait(srv, rid, 20)
        assert ei.value.status == phe.PHE_ETIMEOUT
        assert time.monotonic() - t0 < 2.0
    finally:
        phe.phe_server_destroy(srv)


def test_stalled_iteration_fails_the_server_after_its_bound():
    # an iteration that would take 2 s against a 50 ms bound on every host wait
    srv = _server(chunk_tokens=100, wait_timeout_ms=50, sim_ns_per_item=2e7)
    try:
        rid = phe.phe_server_submit(srv, None, 0, 100, sim_rows=1)
        with pytest.raises(phe.PheError):
            phe.phe_server_wait(srv, rid, 10000)
        done, _ = phe.phe_server_poll(srv, rid)
        assert done == -1
        with pytest.raises(phe.PheError) as ei:
            phe.phe_server_submit(srv, None, 0, 1, sim_rows=1)
        assert ei.value.status == phe.PHE_ETIMEOUT
        assert phe.phe_server_stats(srv)["failed"] == 1
    finally:
        phe.phe_server_destroy(srv)


def test_concurrent_submitters():
    srv = _server(sim_ns_per_item=100.0)
    ids, lock = [], threading.Lock()

    def client(k):
        for j in range(20):
            rid = phe.phe_server_submit(srv, None, 0, 1 + (k * 7 + j) % 9, sim_rows=3)
            with lock:
                ids.append(rid)
    try:
        threads = [threading.Thread(target=client, args=(k,)) for k in range(8)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for i in ids:
            phe.phe_server_wait(srv, i, 20000)
        st = phe.phe_server_stats(srv)
        assert st["completed"] == 160 and len(set(ids)) == 160
    finally:
        phe.phe_server_destroy(srv)


def test_destroy_drains_pending_work():
    srv = _server(chunk_tokens=2, sim_ns_per_item=1e4)
    ids = [phe.phe_server_submit(srv, None, 0, 9, sim_rows=4) for _ in range(5)]
    phe.phe_server_destroy(srv)  # returns after the work is done
    assert len(ids) == 5


def test_failed_request_is_reported_only_after_its_work_drains():
    # the iteration in flight "runs" for 1.5 s; the 50 ms bound fails the
    # server at once, but the request may still be read and written until
    # the iteration finishes, so it is failing, not failed, until then
    srv = _server(chunk_tokens=100, wait_timeout_ms=50, sim_ns_per_item=1.5e7)
    try:
        t0 = time.monotonic()
        rid = phe.phe_server_submit(srv, None, 0, 100, sim_rows=1)
        time.sleep(0.4)
        done, _ = phe.phe_server_poll(srv, rid)
        assert done == 0 and time.monotonic() - t0 < 1.3
        assert phe.phe_server_stats(srv)["failed"] == 0
        with pytest.raises(phe.PheError) as ei:
            phe.phe_server_wait(srv, rid, 100)
        assert ei.value.status == phe.PHE_ETIMEOUT
        with pytest.raises(phe.PheError):
            phe.phe_server_wait(srv, rid, 10000)
        assert time.monotonic() - t0 >= 1.45
        done, _ = phe.phe_server_poll(srv, rid)
        assert done == -1
        assert phe.phe_server_stats(srv)["failed"] == 1
    finally:
        phe.phe_server_destroy(srv)


def test_work_that_never_drains_leaves_requests_pending():
    # an iteration far longer than the drain bound (3 s): the request is
    # never reported failed, its waits time out, and destroy still returns
    srv = _server(chunk_tokens=100, wait_timeout_ms=50, sim_ns_per_item=6e8)
    try:
        rid = phe.phe_server_submit(srv, None, 0, 100, sim_rows=1)
        time.sleep(0.5)
        done, _ = phe.phe_server_poll(srv, rid)
        assert done == 0
        with pytest.raises(phe.PheError) as ei:
            phe.phe_server_wait(srv, rid, 100)
        assert ei.value.status == phe.PHE_ETIMEOUT
        with pytest.raises(phe.PheError):
            phe.phe_server_submit(srv, None, 0, 1, sim_rows=1)
    finally:
        t0 = time.monotonic()
        phe.phe_server_destroy(srv)
        assert time.monotonic() - t0 < 2.0


def test_large_request_is_not_starved_by_small_ones():
    # 100 ms large chunks need 80 kB of a 100 kB budget; 1 ms small chunks
    # (880 B) arrive at 2.5x the served rate.  Without aging, small chunks
    # in flight keep the budget above 20 kB and the large request waits for
    # the whole small backlog (about 3.5 s); with it, it runs within a few
    # iterations of reaching the head of the queue.
    srv = _server(mem_budget_bytes=100_000, chunk_tokens=10, max_active=4096, max_jobs_per_iteration=64,
                  max_queue=100_000, sim_ns_per_item=1e4)
    stop = threading.Event()
    small = []

    def feeder():
        while not stop.is_set():
            small.append(phe.phe_server_submit(srv, None, 0, 50, sim_rows=10))
            time.sleep(0.002)
    try:
        th = threading.Thread(target=feeder)
        th.start()
        time.sleep(0.3)
        t_large = time.monotonic()
        big = phe.phe_server_submit(srv, None, 0, 10, sim_rows=1000)
        phe.phe_server_wait(srv, big, 20000)
        waited = time.monotonic() - t_large
        stop.set()
        th.join()
        assert waited < 2.0, f"large request waited {waited:.2f} s"
        for i in small:
            phe.phe_server_wait(srv, i, 60000)
    finally:
        stop.set()
        phe.phe_server_destroy(srv)
