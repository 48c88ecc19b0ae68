"""Host logic of the serving loop (admission, ticks, faults), against a stand-in
engine that computes each pair with the oracle.  No GPU."""
import collections

import numpy as np
import pytest
import torch

import oracle
import scenes
from paper_1612_08825_gb300 import RESULT_DTYPE
from paper_1612_08825_gb300.serve import Frame, Server, replay, saturate

LEVELS = 2


def _pair(E0, E1):
    """Oracle records of one pair in the library's record layout."""
    ref = oracle.ttc_pair(E0, E1, levels=LEVELS, mode=1)
    out = np.zeros(LEVELS, dtype=RESULT_DTYPE)
    for name in RESULT_DTYPE.names:
        out[name] = ref[name]
    return out


class FakeEngine:
    """Engine protocol on the CPU: a tick completes after `delay` polls."""

    dtype = torch.uint8

    def __init__(self, delay=1, max_H=64, max_W=96):
        self.delay = delay
        self.max_H, self.max_W = max_H, max_W
        self.opened, self.closed = 0, 0
        self.outstanding = 0
        self.max_outstanding = 0
        self.batches = []

    def fixed_bytes(self):
        return 1000

    def fits(self, H, W):
        return H <= self.max_H and W <= self.max_W

    def stream_bytes(self, H, W):
        return 3 * H * W

    def open(self, H, W):
        self.opened += 1
        return {"prev": None, "alive": True}

    def close(self, h):
        assert h["alive"]
        h["alive"] = False
        self.closed += 1

    def has_prev(self, h):
        return h["prev"] is not None

    def launch(self, items):
        recs, npairs = [], 0
        for h, f in items:
            assert h["alive"]
            cur = f.data.numpy()
            if h["prev"] is not None:
                recs.append(_pair(h["prev"], cur))
                npairs += 1
            else:
                recs.append(None)
            h["prev"] = cur
        self.batches.append(npairs)
        self.outstanding += 1
        self.max_outstanding = max(self.max_outstanding, self.outstanding)
        return {"polls": 0, "recs": recs}

    def done(self, t):
        t["polls"] += 1
        return t["polls"] > self.delay

    def wait(self, t):
        t["polls"] = self.delay + 1

    def results(self, t):
        self.outstanding -= 1
        return t["recs"]


def _frames(H, W, n, seed):
    sc = scenes.tilted_plane_scene(H, W, seed=seed, Z0=15.0, speed=0.05)
    return scenes.render_sequence(sc, n)


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3
        return self.t


def test_admission_under_budget_and_release():
    eng = FakeEngine()
    srv = Server(eng, hbm_budget_bytes=1000 + 3 * (32 * 48) * 3, max_batch=4, clock=FakeClock())
    assert srv.admit(0, 32, 48) and srv.admit(1, 32, 48) and srv.admit(2, 32, 48)
    assert not srv.admit(3, 32, 48)                    # budget exhausted
    assert not srv.admit(4, 128, 48)                   # larger than the engine allows
    assert srv.stats["rejected_streams"] == 2
    with pytest.raises(ValueError):
        srv.admit(0, 32, 48)
    srv.remove(1)
    assert eng.closed == 1 and srv.used == 1000 + 2 * 3 * 32 * 48
    assert srv.admit(3, 32, 48)                        # room again


def test_results_match_oracle_and_first_frame_has_none():
    eng = FakeEngine(delay=2)
    srv = Server(eng, 10**9, max_batch=8, clock=FakeClock())
    seqs = {0: _frames(32, 48, 4, 1), 1: _frames(40, 64, 4, 2)}
    for sid, f in seqs.items():
        assert srv.admit(sid, f.shape[1], f.shape[2])
    done = []
    for k in range(4):
        for sid, f in seqs.items():
            assert srv.offer(Frame(sid, k, float(k), f[k]))
        done += srv.step()
    done += srv.drain()
    by = collections.defaultdict(dict)
    for c in done:
        by[c.stream][c.seq] = c
    for sid, f in seqs.items():
        assert sorted(by[sid]) == [0, 1, 2, 3]
        assert by[sid][0].records is None and by[sid][0].level == -1
        for k in range(1, 4):
            ref = oracle.ttc_pair(f[k - 1].numpy(), f[k].numpy(), levels=LEVELS, mode=1)
            assert np.array_equal(by[sid][k].records, _pair(f[k - 1].numpy(), f[k].numpy()))
            assert by[sid][k].level == oracle.select_level(ref, 0)
    assert eng.max_outstanding <= 2


def test_one_frame_per_stream_per_tick_and_batch_limit():
    eng = FakeEngine(delay=0)
    srv = Server(eng, 10**9, max_batch=2, max_in_flight=1, clock=FakeClock())
    fr = {s: _frames(24, 32, 3, 10 + s) for s in range(3)}
    for s in range(3):
        srv.admit(s, 24, 32)
        for k in range(3):
            srv.offer(Frame(s, k, float(k) + 0.1 * s, fr[s][k]))
    done = srv.drain()
    # first tick: three first frames (no pairs); then at most two pairs per tick,
    # oldest arrival first
    assert eng.batches[0] == 0
    assert all(b <= 2 for b in eng.batches)
    assert sum(eng.batches) == 6
    order = [(c.stream, c.seq) for c in done if c.records is not None]
    assert order.index((0, 1)) < order.index((0, 2))
    assert order[:2] == [(0, 1), (1, 1)]


def test_malformed_frames_rejected():
    eng = FakeEngine()
    srv = Server(eng, 10**9, max_batch=4, clock=FakeClock())
    srv.admit(0, 24, 32)
    good = _frames(24, 32, 1, 3)[0]
    assert not srv.offer(Frame(0, 0, 0.0, good[:, :30]))                 # wrong width
    assert not srv.offer(Frame(0, 0, 0.0, good.float()))                  # wrong dtype
    assert not srv.offer(Frame(0, 0, 0.0, good.numpy()))                  # not a tensor
    assert not srv.offer(Frame(5, 0, 0.0, good))                          # unknown stream
    assert srv.stats["rejected_frames"] == 4
    assert srv.offer(Frame(0, 0, 0.0, good))
    assert srv.pending_frames() == 1


def test_queue_overflow_drops_oldest():
    eng = FakeEngine()
    srv = Server(eng, 10**9, max_batch=4, max_pending=2, clock=FakeClock())
    srv.admit(0, 24, 32)
    fr = _frames(24, 32, 4, 4)
    for k in range(4):
        srv.offer(Frame(0, k, float(k), fr[k]))
    assert srv.stats["dropped_frames"] == 2
    done = srv.drain()
    assert [c.seq for c in done] == [2, 3]
    assert np.array_equal(done[1].records, _pair(fr[2].numpy(), fr[3].numpy()))


def test_stream_removed_mid_flight():
    eng = FakeEngine(delay=3)
    srv = Server(eng, 10**9, max_batch=4, clock=FakeClock())
    fr = {s: _frames(24, 32, 3, 20 + s) for s in range(2)}
    for s in range(2):
        srv.admit(s, 24, 32)
        srv.offer(Frame(s, 0, 0.0, fr[s][0]))
    done = srv.step()                                     # tick with both first frames
    for s in range(2):
        srv.offer(Frame(s, 1, 1.0, fr[s][1]))
    srv.remove(1)                                         # goes away with a frame in flight
    assert eng.closed == 0 and 1 in srv.streams           # buffers still in use
    assert srv.stats["dropped_frames"] == 1
    assert not srv.offer(Frame(1, 2, 2.0, fr[1][2]))
    done += srv.drain()
    assert eng.closed == 1 and 1 not in srv.streams
    assert all(c.stream == 0 for c in done)
    assert srv.stats["discarded_results"] == 1
    assert [c.seq for c in done] == [0, 1]
    # re-admitted: starts cold
    assert srv.admit(1, 24, 32)
    srv.offer(Frame(1, 0, 3.0, fr[1][2]))
    done = srv.drain()
    assert done[0].records is None


def test_stalled_producer_does_not_hold_others():
    eng = FakeEngine(delay=0)
    srv = Server(eng, 10**9, max_batch=4, max_in_flight=1, clock=FakeClock())
    fr = {s: _frames(24, 32, 4, 30 + s) for s in range(2)}
    for s in range(2):
        srv.admit(s, 24, 32)
    srv.offer(Frame(1, 0, 0.0, fr[1][0]))                 # stream 1 stalls after one frame
    for k in range(4):
        srv.offer(Frame(0, k, float(k), fr[0][k]))
        srv.step(block=True)
    srv.drain()
    assert srv.stats["results"] == 3 and srv.stats["first_frames"] == 2


def test_replay_and_saturate_drivers():
    eng = FakeEngine(delay=1)
    srv = Server(eng, 10**9, max_batch=8)
    fr = {s: _frames(24, 32, 3, 40 + s) for s in range(3)}
    for s in range(3):
        srv.admit(s, 24, 32)
    arr = [(0.0005 * k, s, k) for k in range(3) for s in range(3)]
    done = replay(srv, arr, lambda s, q: fr[s][q])
    assert srv.stats["results"] == 6 and all(c.latency >= 0 for c in done)
    done = saturate(srv, lambda s, q: fr[s][q % 3], ticks=4)
    assert srv.stats["ticks"] >= 4 + 3 and len(done) >= 9
