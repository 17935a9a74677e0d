"""The serving loop's host logic (admission by HBM budget, Poisson arrivals,
one frame in flight per slot, FIFO order per session, saturation) with a
fake slot: no device involved."""

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
            self.log.append((self.sid, tag[1]))

    def ready(self):
        return time.perf_counter() >= self.t_done

    def finish(self):
        assert self.busy
        self.busy = False
        return 100, 200

    def mesh(self):
        return ("mesh", self.sid, self.tag[1])

    def close(self):
        self.closed = True


def _server(budget, nbytes, log):
    return serve.Server(budget, slot_factory=lambda sess: _FakeSlot(sess, nbytes, log), sync=lambda: None)


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
