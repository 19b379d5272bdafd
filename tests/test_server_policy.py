"""The serving scheduler's policy on the CPU: the library's own scheduler thread
driven through nufft_server_create_with_executor with a fake executor whose
plan entries are bookkeeping records and whose work completes when the test
(or a timer) says so.

Checked: FIFO admission, the slot limit, entry reuse and resident points,
capacity classes, the memory budget with least-recently-used eviction,
waiting for running work, rejection of requests larger than the budget, the
per-request time limit, shutdown, and a randomised stress run whose
invariants (slots, budget, one request per entry at a time, every ticket
answered once) are checked on every launch.
"""
import ctypes
import random
import threading
import time

import pytest

S = pytest.importorskip("paper_1808_06736_gb300.serve")


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1808_06736_gb300 import build
    build.build()
    S._L()


def key(r):
    return (r.kind, r.dim, tuple(r.nmodes), r.isign, r.prec, r.eps)


class Fake:
    """Entries cost 1000 bytes per mode plus 10 per point of capacity."""

    def __init__(self, budget, max_inflight=2, timeout_s=0.0, auto=None):
        self.lock = threading.Lock()
        self.created, self.destroyed, self.launches = [], [], []
        self.live = {}          # entry id -> (key, mcap, bytes)
        self.busy = set()
        self.inflight = {}      # ticket -> entry id
        self.max_seen = 0
        self.errors = []
        self.next_id = 1
        self.auto = auto        # None: the test completes; float: complete after that many seconds
        self.budget = budget
        self.max_inflight = max_inflight
        self._cb = (S.ESTIMATE_FN(self._estimate), S.CREATE_FN(self._create), S.LAUNCH_FN(self._launch),
                    S.DESTROY_FN(self._destroy))
        ex = S.nufft_executor(None, *self._cb)
        self.ex = ex
        st, self.h = S.nufft_server_create_with_executor(ex, budget, max_inflight, timeout_s)
        assert st == 0

    @staticmethod
    def cost(r, mcap):
        n = r.nmodes[0] * (r.nmodes[1] if r.dim > 1 else 1) * (r.nmodes[2] if r.dim > 2 else 1)
        return 1000 * n + 10 * mcap

    def _estimate(self, ctx, r, mcap, out):
        out[0] = self.cost(r.contents, mcap)
        return 0

    def _create(self, ctx, r, mcap, entry, nbytes):
        with self.lock:
            eid = self.next_id
            self.next_id += 1
            b = self.cost(r.contents, mcap)
            self.live[eid] = (key(r.contents), mcap, b)
            self.created.append((eid, key(r.contents), mcap))
            if sum(v[2] for v in self.live.values()) > self.budget:
                self.errors.append("budget exceeded at create %d" % eid)
        entry[0] = eid
        nbytes[0] = b
        return 0

    def _launch(self, ctx, entry, r, slot, skip, ticket):
        eid = entry
        with self.lock:
            if eid in self.busy:
                self.errors.append("entry %d launched while busy" % eid)
            if self.live[eid][1] < r.contents.M:
                self.errors.append("entry %d too small" % eid)
            self.busy.add(eid)
            self.inflight[ticket] = eid
            self.max_seen = max(self.max_seen, len(self.inflight))
            if len(self.inflight) > self.max_inflight:
                self.errors.append("more than %d in flight" % self.max_inflight)
            self.launches.append((ticket, eid, slot, skip, r.contents.tag))
        if self.auto is not None:
            threading.Timer(self.auto * random.random(), self.complete, args=(ticket,)).start()
        return 0

    def _destroy(self, ctx, entry):
        with self.lock:
            if entry in self.busy:
                self.errors.append("entry %d destroyed while busy" % entry)
            self.destroyed.append(entry)
            self.live.pop(entry, None)

    def complete(self, ticket, status=0):
        with self.lock:
            eid = self.inflight.pop(ticket)
            self.busy.discard(eid)
        S.nufft_server_complete(self.h, ticket, status)

    def submit(self, M=1000, n=(8, 8), kind=1, points_key=0, tag=0, eps=1e-5):
        r = S.make_request(kind, len(n), n, 1, 1, eps, M, tag=tag, points_key=points_key)
        r.x = r.y = r.z = 1
        r.in_ = r.out = 1
        st, t = S.nufft_server_submit(self.h, r)
        assert st == 0
        return t

    def wait_launches(self, k, timeout=5.0):
        t0 = time.time()
        while time.time() - t0 < timeout:
            with self.lock:
                if len(self.launches) >= k:
                    return True
            time.sleep(0.002)
        return False

    def poll_all(self, k, timeout=5.0):
        got = []
        t0 = time.time()
        while len(got) < k and time.time() - t0 < timeout:
            got += S.nufft_server_poll(self.h, 64, 0.05)[1]
        return got

    def close(self):
        S.nufft_server_destroy(self.h)


def test_fifo_and_slot_limit():
    f = Fake(budget=10 ** 9, max_inflight=2)
    ts = [f.submit(M=1000 + i, tag=i) for i in range(5)]
    assert f.wait_launches(2)
    time.sleep(0.05)
    assert len(f.launches) == 2
    f.complete(ts[0])
    assert f.wait_launches(3)
    f.complete(ts[1])
    f.complete(ts[2])
    assert f.wait_launches(5)
    f.complete(ts[3])
    f.complete(ts[4])
    done = f.poll_all(5)
    assert [c.status for c in done] == [0] * 5
    assert [l[0] for l in f.launches] == ts  # admitted in arrival order
    assert f.max_seen <= 2 and not f.errors
    assert S.nufft_server_drain(f.h, 1.0) == 0
    f.close()


def test_reuse_resident_points_and_capacity():
    f = Fake(budget=10 ** 9, max_inflight=1)
    t1 = f.submit(M=5000, points_key=7)
    assert f.wait_launches(1)
    f.complete(t1)
    t2 = f.submit(M=5000, points_key=7)       # same key, same points: binning skipped
    assert f.wait_launches(2)
    f.complete(t2)
    t3 = f.submit(M=6000, points_key=7)       # other M: reuse, rebin
    assert f.wait_launches(3)
    f.complete(t3)
    t4 = f.submit(M=10000)                    # beyond capacity 8192: a new entry of capacity 16384
    assert f.wait_launches(4)
    f.complete(t4)
    done = {c.ticket: c for c in f.poll_all(4)}
    assert [done[t].reused for t in (t1, t2, t3, t4)] == [0, 2, 1, 0]
    assert [l[3] for l in f.launches] == [0, 1, 0, 0]
    assert [c[2] for c in f.created] == [8192, 16384]
    st = S.nufft_server_stats_get(f.h)
    assert st["entries_created"] == 2 and st["binning_skipped"] == 1 and st["entries_reused"] == 2
    f.close()
    assert not f.errors


def test_lru_eviction_within_budget():
    # each entry: 1000 * 64 + 10 * 4096 = 104960 bytes; the budget holds two
    f = Fake(budget=2 * 104960 + 100, max_inflight=1)
    ta = f.submit(n=(8, 8), kind=1)
    assert f.wait_launches(1)
    f.complete(ta)
    tb = f.submit(n=(8, 8), kind=2)
    assert f.wait_launches(2)
    f.complete(tb)
    ta2 = f.submit(n=(8, 8), kind=1)  # reuse A: now B is the least recently used
    assert f.wait_launches(3)
    f.complete(ta2)
    tc = f.submit(n=(4, 16), kind=1)
    assert f.wait_launches(4)
    f.complete(tc)
    f.poll_all(4)
    assert len(f.created) == 3
    assert f.destroyed == [f.created[1][0]]  # B went, A stayed
    st = S.nufft_server_stats_get(f.h)
    assert st["entries_evicted"] == 1 and st["peak_bytes"] <= f.budget
    f.close()
    assert not f.errors


def test_waits_for_memory_then_runs():
    f = Fake(budget=104960 + 100, max_inflight=4)  # one entry at a time
    ta = f.submit(kind=1)
    tb = f.submit(kind=2)
    assert f.wait_launches(1)
    time.sleep(0.05)
    assert len(f.launches) == 1  # B waits for A's memory although slots are free
    f.complete(ta)
    assert f.wait_launches(2)
    f.complete(tb)
    done = f.poll_all(2)
    assert sorted(c.status for c in done) == [0, 0]
    assert len(f.destroyed) == 1
    f.close()
    assert not f.errors


def test_rejects_requests_larger_than_budget():
    f = Fake(budget=50000, max_inflight=2)
    t_big = f.submit(n=(64, 64))
    done = f.poll_all(1)
    assert done[0].ticket == t_big and done[0].status == S.NUFFT_ERR_REJECTED
    f2 = f.submit(n=(2, 2), M=10)
    assert f.wait_launches(1)
    f.complete(f2)
    assert f.poll_all(1)[0].status == 0
    assert S.nufft_server_stats_get(f.h)["rejected"] == 1
    f.close()


def test_time_limit_reports_and_holds_the_slot():
    f = Fake(budget=10 ** 9, max_inflight=1, timeout_s=0.05)
    t1 = f.submit()
    t2 = f.submit()
    t0 = time.time()
    done = f.poll_all(1, timeout=2.0)
    # an early report: the work still runs, so the caller's buffers are not yet free
    assert done[0].ticket == t1 and done[0].status == S.NUFFT_ERR_TIMEOUT and done[0].pending == 1
    assert 0.04 <= time.time() - t0 < 1.5
    time.sleep(0.05)
    assert len(f.launches) == 1  # the slot is still held by the unfinished work
    assert S.nufft_server_drain(f.h, 0.05) == S.NUFFT_ERR_TIMEOUT
    assert S.nufft_server_poll(f.h, 8, 0.05)[1] == []  # no final completion while the work runs
    f.complete(t1)               # the late finish frees it and sends t1's final completion
    done = f.poll_all(1)
    assert done[0].ticket == t1 and done[0].status == 0 and done[0].pending == 0
    assert done[0].t_done >= done[0].t_admit + 0.05  # the final report is the late finish, after the limit
    assert f.wait_launches(2)    # only then does the slot take the next request
    f.complete(t2)
    done = f.poll_all(1)
    assert done[0].ticket == t2 and done[0].status == 0 and done[0].pending == 0
    assert S.nufft_server_poll(f.h, 8, 0.05)[1] == []
    st = S.nufft_server_stats_get(f.h)
    assert st["timeouts"] == 1 and st["completed"] == 2
    f.close()


def test_final_completion_comes_after_the_work_ends():
    # the executor finishes every request after the time limit: each ticket gets an early
    # TIMEOUT report first and its final completion only once the executor has reported it
    f = Fake(budget=10 ** 9, max_inflight=2, timeout_s=0.02)
    tickets = [f.submit(tag=i) for i in range(4)]
    finished_at = {}
    seen = []
    t_end = time.time() + 10
    while len(finished_at) < 4 and time.time() < t_end:
        time.sleep(0.05)  # well past the limit
        with f.lock:
            running = list(f.inflight)
        for t in running:
            finished_at[t] = S.nufft_server_clock()
            f.complete(t)
        seen += S.nufft_server_poll(f.h, 64, 0.0)[1]
    seen += f.poll_all(8 - len(seen), timeout=2.0)
    assert sorted(finished_at) == tickets
    for t in tickets:
        cs = [c for c in seen if c.ticket == t]
        assert [c.pending for c in cs] == [1, 0], cs
        assert cs[0].status == S.NUFFT_ERR_TIMEOUT and cs[1].status == 0
        assert cs[1].t_done >= finished_at[t] - 0.01  # final only after the executor reported the work done
    assert not f.errors
    f.close()


def test_shutdown_leaks_entries_the_executor_never_finished():
    # destroy waits (here 0.2 s) for running work; the entry of a request the executor never
    # reports may still be in use on the device, so it is not destroyed; idle entries are
    f = Fake(budget=10 ** 9, max_inflight=2)
    assert S.nufft_server_set_shutdown_wait(f.h, 0.2) == 0
    assert S.nufft_server_set_shutdown_wait(f.h, 0.0) == -1
    ta = f.submit(n=(8, 8), tag=1)
    tb = f.submit(n=(16, 16), tag=2)
    assert f.wait_launches(2)
    f.complete(tb)
    assert f.poll_all(1)[0].ticket == tb
    with f.lock:
        stuck = f.inflight[ta]
    t0 = time.time()
    f.close()  # ta never completes
    assert 0.15 <= time.time() - t0 < 5.0
    assert not f.errors                     # nothing was destroyed while busy
    assert stuck not in f.destroyed         # the stuck entry was leaked
    assert len(f.destroyed) == len(f.created) - 1


def test_invalid_requests_are_refused_at_submit():
    f = Fake(budget=10 ** 9)
    r = S.make_request(4, 2, (8, 8), 1, 1, 1e-5, 10)
    r.x = r.y = r.in_ = r.out = 1
    assert S.nufft_server_submit(f.h, r)[0] == -1
    r = S.make_request(1, 2, (8, 8), 1, 1, 1e-5, 10)
    r.x = r.in_ = r.out = 1                 # y missing for d = 2
    assert S.nufft_server_submit(f.h, r)[0] == -1
    r = S.make_request(3, 1, (8,), 1, 1, 1e-5, 10)
    r.x = r.in_ = r.out = r.out3 = 1        # LSQ without targets / grad_x
    assert S.nufft_server_submit(f.h, r)[0] == -1
    assert S.nufft_server_stats_get(f.h)["submitted"] == 0
    f.close()


def test_shutdown_with_queued_and_running_work():
    f = Fake(budget=10 ** 9, max_inflight=1, auto=0.05)
    for i in range(4):
        f.submit(tag=i)
    assert f.wait_launches(1)
    f.close()  # returns after the running request finished; queued ones are failed
    assert not f.errors
    assert len(f.destroyed) == len(f.created)


def test_randomised_stress_invariants():
    random.seed(3)
    shapes = [(8, 8), (16, 16), (4, 4, 4), (32,)]
    budget = 3 * (1000 * 256 + 10 * 65536)
    f = Fake(budget=budget, max_inflight=3, auto=0.004)
    tickets = []
    for i in range(300):
        n = random.choice(shapes)
        M = int(10 ** random.uniform(2, 4.7))
        tickets.append(f.submit(M=M, n=n, kind=random.choice([1, 2]), points_key=random.choice([0, 1, 2]), tag=i))
        if i % 25 == 0:
            time.sleep(0.003)
    done = f.poll_all(300, timeout=30.0)
    assert sorted(c.ticket for c in done) == tickets
    assert all(c.status == 0 for c in done)
    assert all(c.t_submit <= c.t_admit <= c.t_done for c in done)
    st = S.nufft_server_stats_get(f.h)
    assert st["peak_inflight"] <= 3 and st["peak_bytes"] <= budget and st["completed"] == 300
    assert S.nufft_server_drain(f.h, 5.0) == 0
    f.close()
    assert not f.errors, f.errors[:5]
    assert len(f.destroyed) == len(f.created)


def test_request_bytes_estimate_counts_grid_and_points():
    # host-only: 3D N = 64^3 complex64 at eps 1e-5 -> fine grid 128^3 (w = 6)
    r = S.make_request(2, 3, (64, 64, 64), -1, 1, 1e-5, 100000, upsampfac=2.0)
    st, b = S.nufft_request_bytes(r, 131072)
    assert st == 0
    grid = 128 ** 3 * 8
    assert b >= 2 * grid + 131072 * 16          # grid + cuFFT area bound + point records
    assert b <= 2 * grid + 131072 * 16 + 8 * 2 ** 20
    st, b2 = S.nufft_request_bytes(r, 262144)
    assert b2 - b >= 131072 * 16
    r3 = S.make_request(3, 3, (64, 64, 64), -1, 1, 1e-5, 100000, upsampfac=2.0)
    st, b3 = S.nufft_request_bytes(r3, 131072)
    assert b3 - b == ((2 + 3) * 131072 + 64 ** 3) * 8  # gradient scratch
    assert S.nufft_request_bytes(r, 10)[0] == -1  # capacity below M


def test_upsampling_choice_per_request():
    """upsampfac 0: 5/4 when the fine-grid work saved outweighs the wider kernel's extra
    stencil cells (few points on a big grid), 2 otherwise, and never 5/4 when eps would need
    w > 16 there; explicit values pass through; requests with different factors do not share
    plan entries, and the estimate follows the smaller grid."""
    pick = lambda M, eps=1e-3, n=(256, 256, 256), sig=0.0, prec=1: S.upsampfac_for(1, n, eps, M, prec, upsampfac=sig)
    assert pick(10 ** 5) == 1.25 and pick(10 ** 6) == 1.25
    assert pick(10 ** 8) == 2.0
    # complex64 3D at 1e-5: the correction would amplify rounding past eps (Eq. (rmax)); complex128 is fine
    assert pick(10 ** 5, eps=1e-5) == 2.0 and pick(10 ** 5, eps=1e-5, prec=2) == 1.25
    assert pick(10 ** 5, eps=1e-11, prec=2) == 2.0
    assert pick(10 ** 8, sig=1.25) == 1.25 and pick(10 ** 5, sig=2.0) == 2.0
    r = S.make_request(1, 3, (256, 256, 256), 1, 1, 1e-5, 10 ** 5, upsampfac=1.5)
    assert S.nufft_request_upsampfac(r) == 0.0
    st2, b2 = S.nufft_request_bytes(S.make_request(1, 3, (256,) * 3, 1, 1, 1e-3, 10 ** 5, upsampfac=2.0), 2 ** 17)
    st5, b5 = S.nufft_request_bytes(S.make_request(1, 3, (256,) * 3, 1, 1, 1e-3, 10 ** 5), 2 ** 17)
    assert st2 == 0 and st5 == 0 and b5 < b2 / 3
    f = Fake(budget=10 ** 12, max_inflight=1)
    t1 = f.submit(M=1000, n=(512, 512), eps=1e-3)  # same shape, two factors: two entries
    assert f.wait_launches(1)
    f.complete(t1)
    r = S.make_request(1, 2, (512, 512), 1, 1, 1e-3, 1000, upsampfac=2.0)
    r.x = r.y = r.z = r.in_ = r.out = 1
    st, t2 = S.nufft_server_submit(f.h, r)
    assert st == 0 and f.wait_launches(2)
    f.complete(t2)
    f.poll_all(2)
    keys = [c[1] for c in f.created]
    f.close()
    assert len(f.created) == 2 and keys[0][:5] == keys[1][:5], keys
    assert not f.errors
