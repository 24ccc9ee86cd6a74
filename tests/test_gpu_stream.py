"""Continuous batching in one resident engine (dt_stream_*): jobs of mixed
sizes join the running engine at round boundaries, and each job's result
equals the oracle's DT of its points alone (integer output: bit-exact)."""
import threading
import time

import numpy as np
import pytest

import oracle
import pointsets

pytestmark = pytest.mark.gpu


def _drain(stream, ids, timeout_s=120.0):
    t0 = time.time()
    while time.time() - t0 < timeout_s:
        stream.run(4)
        if all(stream.status(j)[0] not in (0, 1) for j in ids):
            return
    raise AssertionError("jobs did not finish")


@pytest.mark.parametrize("dim", [2, 3])
def test_stream_jobs_match_oracle(dim):
    from paper_1902_07554_gb300 import Stream, Triangulator
    sizes = [7, 40, 900, 5000, 23_000, 120, 61_000, 300, 2_500, 15_000]
    jobs = []
    for i, m in enumerate(sizes):
        if dim == 3 and i % 2:
            jobs.append(pointsets.clustered(m, 100 + i))
        else:
            jobs.append(pointsets.uniform(m, dim, 100 + i))
    with Triangulator(0) as tri:
        st = Stream(tri, dim, 200_000, 16)
        ids = [st.submit(P) for P in jobs]
        _drain(st, ids)
        for j, P in zip(ids, jobs):
            assert st.status(j)[0] == 2
            assert np.array_equal(st.fetch(j).astype(np.int64), oracle.delaunay(P)), len(P)
            st.release(j)
        info = st.info()
        assert info["running"] == 0 and info["queued"] == 0 and info["free_points"] == info["capacity"]
        st.close()


def test_stream_reuses_capacity_and_slots():
    """More points and jobs over time than the stream holds at once: freed
    ranges and instance slots are reused, results stay exact."""
    from paper_1902_07554_gb300 import Stream, Triangulator
    jobs = [pointsets.uniform(int(m), 3, 300 + i) for i, m in enumerate(np.linspace(2000, 30_000, 12))]
    with Triangulator(0) as tri:
        st = Stream(tri, 3, 70_000, 3)
        ids = [st.submit(P) for P in jobs]
        _drain(st, ids)
        for j, P in zip(ids, jobs):
            assert np.array_equal(st.fetch(j).astype(np.int64), oracle.delaunay(P))
        assert st.info()["quanta"] >= 4
        st.close()


def test_stream_admits_arrivals_while_running():
    """A large job runs; small jobs submitted from another thread while it
    runs are admitted at round boundaries and run beside it (they are seen
    running before it finishes), and every result is exact."""
    from paper_1902_07554_gb300 import Stream, Triangulator
    big = pointsets.clustered(400_000, 9)
    small = [pointsets.uniform(2000 + 100 * i, 3, 500 + i) for i in range(6)]
    done_at, running_at = {}, {}
    with Triangulator(0) as tri:
        st = Stream(tri, 3, 600_000, 16)
        big_id = st.submit(big)
        ids = []

        def feed():
            time.sleep(0.02)
            for P in small:
                ids.append(st.submit(P))
                time.sleep(0.005)

        th = threading.Thread(target=feed)
        th.start()
        t0 = time.time()
        while time.time() - t0 < 120:
            st.run(1)
            for j in [big_id] + list(ids):
                s, _ = st.status(j)
                if s == 1 and j not in running_at:
                    running_at[j] = time.time()
                if s == 2 and j not in done_at:
                    done_at[j] = time.time()
            if len(done_at) == 1 + len(small) and not th.is_alive():
                break
        th.join()
        assert len(done_at) == 1 + len(small)
        assert sum(1 for j in ids if running_at.get(j, 1e30) < done_at[big_id]) >= 2
        assert np.array_equal(st.fetch(big_id).astype(np.int64), oracle.delaunay(big))
        for j, P in zip(ids, small):
            assert np.array_equal(st.fetch(j).astype(np.int64), oracle.delaunay(P))
        st.close()


def test_stream_bad_jobs_fail_alone():
    from paper_1902_07554_gb300 import Stream, Triangulator
    good = pointsets.uniform(3000, 3, 1)
    dup = pointsets.uniform(500, 3, 2)
    dup[100] = dup[7]
    tiny = pointsets.uniform(3, 3, 3)
    flat = np.concatenate([pointsets.uniform(200, 2, 4), np.zeros((200, 1))], axis=1)
    with Triangulator(0) as tri:
        st = Stream(tri, 3, 50_000, 8)
        ids = [st.submit(P) for P in (good, dup, tiny, flat)]
        _drain(st, ids)
        codes = [st.status(j)[0] for j in ids]
        assert codes == [2, -2, -1, -3]
        assert np.array_equal(st.fetch(ids[0]).astype(np.int64), oracle.delaunay(good))
        st.close()


def test_stream_recovers_after_a_device_limit():
    """A walk limit run out on purpose fails the running jobs with
    DT_E_TIMEOUT; the same stream then serves new jobs exactly."""
    from paper_1902_07554_gb300 import DTError, Stream, Triangulator
    P = pointsets.uniform(20_000, 3, 77)
    with Triangulator(0, walk_limit=1) as tri:
        st = Stream(tri, 3, 100_000, 8)
        j = st.submit(P)
        with pytest.raises(DTError) as e:
            for _ in range(200):
                st.run(4)
        assert e.value.code == -5 and st.status(j)[0] == -5
        tri.configure(walk_limit=0)
        j2 = st.submit(P)
        _drain(st, [j2])
        assert np.array_equal(st.fetch(j2).astype(np.int64), oracle.delaunay(P))
        st.close()
