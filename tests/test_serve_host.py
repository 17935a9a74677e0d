"""The serving loop's host logic (admission by HBM budget before and after
allocation, sessions joining and leaving while the loop runs, Poisson
arrivals, one frame in flight per slot, FIFO dispatch per session,
saturation) with a fake slot: no device involved."""

import time
from dataclasses import dataclass

import pytest

from paper_1712_03084_gb300 import serve


@dataclass
class _Frame:
    n_points: int


class _FakeSlot:
    """Takes 0.5 ms per frame; records what the loop asks of it."""

    def __init__(self, sess, nbytes, log):
        self.sid = sess.sid
        self.nbytes = nbytes
        self.busy = False
        self.tag = None
        self.t_done = 0.0
        self.log = log
        self.closed = False

    def device_bytes(self):
        return self.nbytes

    def submit(self, frame, tag=None):
        assert not self.busy, "one frame in flight per slot"
        self.busy = True
        self.tag = tag
        self.t_done = time.perf_counter() + 0.0005
        if tag is not None:
            self.log.append((self.sid, tag[-1]))

    def ready(self):
        return time.perf_counter() >= self.t_done

    def finish(self):
        assert self.busy
        self.busy = False
        return 100, 200

    def mesh(self):
        return ("mesh", self.sid, self.tag[-1])

    def close(self):
        self.closed = True


def _server(budget, nbytes, log, made=None, estimate=None):
    def factory(sess):
        sl = _FakeSlot(sess, nbytes, log)
        if made is not None:
            made.append(sl)
        return sl
    return serve.Server(budget, slot_factory=factory, sync=lambda: None,
                        estimate=estimate or (lambda sess: nbytes * sess.n_slots))


def _sessions(n, rate):
    return [serve.Session(sid, (64, 64, 64), (-1, -1, -1, 1, 1, 1), [_Frame(10), _Frame(12)], rate_hz=rate)
            for sid in range(n)]


def test_admission_respects_the_budget():
    srv = _server(25, 10, [])
    sess = _sessions(3, 30.0)
    assert [srv.admit(s) for s in sess] == [True, True, False]
    assert srv.used == 20 and srv.rejected == [2]
    srv.close()
    assert all(s.slot is None or s.slot.closed for s in sess)


def test_every_arrival_is_served_in_order():
    log = []
    srv = _server(1 << 30, 10, log)
    for s in _sessions(3, 200.0):
        srv.admit(s)
    st = srv.run(duration_s=0.2, seed=7, keep_meshes={(1, 0), (2, 3)})
    # the same seed gives the same arrivals: count them the way the loop draws them
    import numpy as np
    rng = np.random.default_rng(7)
    expect = 0
    for _ in range(3):
        t = 0.0
        while True:
            t += rng.exponential(1.0 / 200.0)
            if t > 0.2:
                break
            expect += 1
    assert st["frames"] == expect == len(log)
    for sid in range(3):
        ks = [k for s, k in log if s == sid]
        assert ks == sorted(ks) == list(range(len(ks)))       # FIFO, nothing skipped
    assert st["p99_ms"] >= st["p50_ms"] > 0 and st["frames_per_s"] > 0
    assert st["meshes"][(1, 0)] == ("mesh", 1, 0) and st["meshes"][(2, 3)] == ("mesh", 2, 3)
    srv.close()


def test_saturation_makes_every_frame_available_at_once():
    log = []
    srv = _server(1 << 30, 10, log)
    for s in _sessions(2, 50.0):
        srv.admit(s)
    st = srv.run(duration_s=0.4, saturate=True)
    assert st["frames"] == 2 * 20 == len(log)
    srv.close()


def test_the_default_slot_needs_a_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    srv = serve.Server(1 << 30)
    with pytest.raises(Exception):
        srv.admit(_sessions(1, 30.0)[0])


def test_a_session_over_the_estimate_allocates_nothing():
    made = []
    srv = _server(25, 10, [], made=made, estimate=lambda sess: 30)
    assert not srv.admit(_sessions(1, 30.0)[0])
    assert made == [] and srv.rejected == [0] and srv.used == 0


def test_the_real_size_after_warm_up_is_checked_again():
    """The estimate fits but the slots' size after running the session's
    frames does not: the slots are closed again and nothing is charged."""
    made = []
    srv = _server(25, 30, [], made=made, estimate=lambda sess: 10)
    assert not srv.admit(_sessions(1, 30.0)[0])
    assert len(made) == 1 and made[0].closed and srv.used == 0


def test_a_rejected_session_gets_in_after_another_leaves():
    """Budget for one session: the second joins at 0.05 s, waits, and is
    admitted when the first leaves at 0.1 s; its later frames are served."""
    log = []
    srv = _server(15, 10, log)
    a, b = _sessions(2, 400.0)
    a.stop_s = 0.1
    b.start_s = 0.05
    assert srv.admit(a)
    st = srv.run(duration_s=0.3, seed=3, late=[b])
    kinds = [(e[0], e[1], e[3] if e[0] == "join" else None) for e in st["events"]]
    assert ("join", 1, False) in kinds and ("leave", 0, None) in kinds and ("join", 1, True) in kinds
    assert kinds.index(("leave", 0, None)) < kinds.index(("join", 1, True))
    served_b = [k for s_, k in log if s_ == 1]
    assert len(served_b) > 10 and served_b == sorted(served_b)
    assert all(k > 0 for k in served_b[:1]) or st["not_served"] > 0
    assert srv.used == 10 and [s.sid for s in srv.sessions] == [1]
    srv.close()


def test_two_slots_per_session_run_two_frames_at_once():
    log = []
    made = []
    srv = _server(1 << 30, 10, log, made=made)
    s = _sessions(1, 50.0)[0]
    s.n_slots = 2
    assert srv.admit(s) and len(made) == 2
    st = srv.run(duration_s=0.2, saturate=True)
    assert st["frames"] == 10
    ks = [k for _, k in log]
    assert ks == list(range(10))          # dispatched in arrival order over both slots
    assert st["per_grid"][64]["frames"] == 10
    srv.close()
