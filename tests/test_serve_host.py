"""Scheduler of the serving loop on the host, with a fake device: admission
by free memory, grouping, FIFO order, lanes, completion and latency stats."""
import numpy as np

from paper_2203_11484_gb300 import serve as S
from paper_2203_11484_gb300 import workloads as W


class FakeBackend(S.Backend):
    """A group finishes `service` seconds after launch (simulated clock)."""

    def __init__(self, free, service_per_request=1.0):
        self.free = free
        self.t = 0.0
        self.service = service_per_request
        self.launched = []

    def free_bytes(self):
        return self.free

    def launch(self, group, lane):
        self.launched.append((self.t, lane, [r.rid for r in group]))
        return self.t + self.service * len(group) ** 0.5   # batching amortises

    def done(self, handle):
        return self.t >= handle


def _req(rid, scene="a", w=64, h=64, m=100, arrival=0.0):
    cam = W.Camera((0, 0, 0), (0, 0, 1), (0, 1, 0), 60.0, w, h)
    gen = W.GenParams(d_close=1.0, m_close=m // 2, m_far=m - m // 2)
    return S.Request(rid, scene, W.View(cam, gen, W.GatherParams(1e-4, 1e-5)), arrival)


def _drive(server, backend, reqs, dt=0.05, limit=10000):
    reqs = sorted(reqs, key=lambda r: r.arrival)
    i = 0
    for _ in range(limit):
        while i < len(reqs) and reqs[i].arrival <= backend.t:
            server.submit(reqs[i])
            i += 1
        server.tick(backend.t)
        if i == len(reqs) and not server.queue and not server.running:
            return
        backend.t += dt
    raise AssertionError("did not finish")


def test_admission_respects_memory_and_groups():
    n_tris = {"a": 1000, "b": 1000}
    reqs = [_req(k, "a" if k < 6 else "b", arrival=0.01 * k) for k in range(10)]
    one = S.estimate_bytes(reqs[0].view, 1000)
    be = FakeBackend(free=int(3.5 * one) + (1 << 20))
    srv = S.Server(be, n_tris, lanes=4, max_group=8, reserve_bytes=1 << 20)
    _drive(srv, be, reqs)
    assert len(srv.finished) == 10
    assert srv.max_in_flight_bytes <= 3.5 * one          # never over budget
    for t, lane, ids in be.launched:
        scenes = {"a" if i < 6 else "b" for i in ids}
        assert len(scenes) == 1 and 1 <= len(ids) <= 3
    order = [i for _, _, ids in be.launched for i in ids]
    assert order == sorted(order)                         # FIFO admission
    assert all(r.t_done >= r.t_admit >= r.arrival for r in srv.finished)


def test_single_lane_single_request_is_a_plain_queue():
    reqs = [_req(k, arrival=0.0) for k in range(5)]
    be = FakeBackend(free=1 << 40)
    srv = S.Server(be, {"a": 10}, lanes=1, max_group=1, reserve_bytes=0)
    _drive(srv, be, reqs)
    assert [ids for _, _, ids in be.launched] == [[0], [1], [2], [3], [4]]
    assert srv.max_concurrent_groups == 1
    st = S.summarize(srv.finished)
    assert st["requests"] == 5 and st["p99_ms"] >= st["p50_ms"] > 0


def test_continuous_batching_admits_late_arrivals_while_busy():
    reqs = [_req(0, arrival=0.0), _req(1, arrival=0.0), _req(2, arrival=0.3), _req(3, arrival=0.35)]
    be = FakeBackend(free=1 << 40, service_per_request=1.0)
    srv = S.Server(be, {"a": 10}, lanes=2, max_group=4, reserve_bytes=0)
    _drive(srv, be, reqs)
    # the first two go together; the late ones start on the second lane while
    # the first group is still running
    assert be.launched[0][2] == [0, 1]
    assert be.launched[1][2] == [2] and be.launched[1][0] < 1.0
    assert srv.max_concurrent_groups == 2


def test_memory_full_waits_instead_of_overcommitting():
    reqs = [_req(k, w=512, h=512, m=5000) for k in range(4)]
    one = S.estimate_bytes(reqs[0].view, 10)
    be = FakeBackend(free=one + 10)
    srv = S.Server(be, {"a": 10}, lanes=4, max_group=4, reserve_bytes=0)
    _drive(srv, be, reqs)
    assert srv.max_concurrent_groups == 1 and len(srv.finished) == 4


def test_poisson_arrivals_rate():
    rng = np.random.default_rng(0)
    t = S.poisson_arrivals(rng, 5.0, 20000)
    assert abs(len(t) / t[-1] - 5.0) < 0.1
