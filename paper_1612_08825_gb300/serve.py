"""Serving loop: many camera streams, continuous batching into the batch API.

The paper computes time to contact for one camera (Sec. V); a server sees many.
Every camera stream keeps its previous frame and that frame's pyramid (levels 1..L-1
of the 2x2 block-sum pyramid, Sec. V-B) resident on the device, so each arriving
frame is uploaded once and its pyramid is built once.  Frames that have arrived are
gathered into ticks (at most one frame per stream per tick, oldest first); a tick is
one ``ttc_batch_prepare`` + ``ttc_batch_run`` over all its pairs (Sec. V-A per pair
and level), then the per-level records come back to the host, where the multi-scale
rule picks a level (Sec. V-B).  Up to two ticks are in flight: the uploads and host
work of one overlap the kernels of the other.

Admission: a stream is admitted only while the device bytes of all admitted streams
plus the engine's fixed workspace stay within the HBM budget.  Faults are handled on
the host: malformed frames are rejected, a removed stream's pending frames are
dropped and its buffers are freed once no tick in flight still reads them, a stream
whose producer stalls simply has no frame in the ticks meanwhile, and a full
per-stream queue drops its oldest frame.  A stream's first frame (and the first
frame after it is re-admitted) yields no result: it only becomes the resident
previous frame.

The engines own the device side; ``Server`` is pure host logic, so that it can be
tested against a stand-in engine without a GPU.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Dict, List, Optional

import numpy as np
import torch

from . import (MODE_FOE, RESULT_DTYPE, TtcContext, _frame_args, pyramid_layout, results_to_numpy,
               select_level)

__all__ = ["Frame", "Completed", "Server", "NativeServer", "CudaBatchEngine", "PerFrameEngine", "latency_summary",
           "replay", "saturate"]


@dataclasses.dataclass
class Frame:
    stream: int
    seq: int
    t_arrival: float
    data: torch.Tensor          # (H, W) host tensor (pinned for asynchronous uploads)


@dataclasses.dataclass
class Completed:
    stream: int
    seq: int
    t_arrival: float
    t_done: float
    records: Optional[np.ndarray]    # per-level records, None for a stream's first frame
    level: int                       # level chosen by the multi-scale rule, -1 if none

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class _Stream:
    def __init__(self, sid: int, H: int, W: int, handle, nbytes: int, max_pending: int):
        self.sid, self.H, self.W = sid, H, W
        self.handle = handle
        self.nbytes = nbytes
        self.pending: collections.deque = collections.deque(maxlen=max_pending)
        self.in_flight = 0            # frames of this stream in ticks not yet collected
        self.closed = False


class Server:
    """Continuous batching of camera streams over an engine (see module docstring)."""

    def __init__(self, engine, hbm_budget_bytes: int, max_batch: int, rule: int = 0, max_pending: int = 4,
                 max_in_flight: int = 2, clock=time.perf_counter):
        if max_in_flight < 1 or max_in_flight > 2:
            raise ValueError("max_in_flight is 1 or 2 (three frame slots per stream)")
        self.engine = engine
        self.budget = int(hbm_budget_bytes)
        self.max_batch = int(max_batch)
        self.rule = rule
        self.max_pending = max_pending
        self.max_in_flight = max_in_flight
        self.clock = clock
        self.streams: Dict[int, _Stream] = {}
        self.used = engine.fixed_bytes()
        self.ticks: collections.deque = collections.deque()     # (ticket, items)
        self.stats = collections.Counter()

    # -- admission -----------------------------------------------------------------
    def admit(self, sid: int, H: int, W: int) -> bool:
        """Admit stream `sid` of H x W frames if the HBM budget allows it."""
        if sid in self.streams:
            raise ValueError(f"stream {sid} is already admitted")
        if not self.engine.fits(H, W):
            self.stats["rejected_streams"] += 1
            return False
        need = self.engine.stream_bytes(H, W)
        if self.used + need > self.budget:
            self.stats["rejected_streams"] += 1
            return False
        self.streams[sid] = _Stream(sid, H, W, self.engine.open(H, W), need, self.max_pending)
        self.used += need
        self.stats["admitted_streams"] += 1
        return True

    def remove(self, sid: int):
        """The stream goes away: pending frames are dropped; buffers are freed when no
        tick in flight still uses them."""
        st = self.streams.get(sid)
        if st is None or st.closed:
            return
        st.closed = True
        self.stats["dropped_frames"] += len(st.pending)
        st.pending.clear()
        self._release_if_idle(st)

    def _release_if_idle(self, st: _Stream):
        if st.closed and st.in_flight == 0 and self.streams.get(st.sid) is st:
            self.engine.close(st.handle)
            self.used -= st.nbytes
            del self.streams[st.sid]

    # -- frames --------------------------------------------------------------------
    def offer(self, frame: Frame) -> bool:
        """A frame arrives.  Rejected (False) if its stream is unknown or closed, or if
        its shape or dtype do not match the stream's."""
        st = self.streams.get(frame.stream)
        if st is None or st.closed:
            self.stats["rejected_frames"] += 1
            return False
        d = frame.data
        if (not isinstance(d, torch.Tensor) or d.dim() != 2 or tuple(d.shape) != (st.H, st.W)
                or d.dtype != self.engine.dtype or d.is_cuda):
            self.stats["rejected_frames"] += 1
            return False
        if len(st.pending) == st.pending.maxlen:
            self.stats["dropped_frames"] += 1         # the oldest goes
        st.pending.append(frame)
        self.stats["offered_frames"] += 1
        return True

    def pending_frames(self) -> int:
        return sum(len(s.pending) for s in self.streams.values())

    # -- ticks ---------------------------------------------------------------------
    def _gather(self) -> list:
        # one frame per stream, oldest arrival first, at most max_batch pairs; first
        # frames of streams (no pair) ride along without counting against the batch
        cands = [s for s in self.streams.values() if s.pending and not s.closed]
        cands.sort(key=lambda s: s.pending[0].t_arrival)
        items, npairs = [], 0
        for s in cands:
            has_prev = self.engine.has_prev(s.handle)
            if has_prev and npairs >= self.max_batch:
                continue
            items.append((s, s.pending.popleft()))
            npairs += has_prev
        return items

    def step(self, block: bool = False) -> List[Completed]:
        """Launch a tick if frames are pending and a slot is free, and collect every
        finished tick (waiting for the oldest one if `block` or if no launch was
        possible while ticks are in flight)."""
        done = self._collect(block=False)
        if len(self.ticks) < self.max_in_flight:
            items = self._gather()
            if items:
                ticket = self.engine.launch([(s.handle, f) for s, f in items])
                for s, _ in items:
                    s.in_flight += 1
                self.ticks.append((ticket, items))
                self.stats["ticks"] += 1
        if block and self.ticks:
            done += self._collect(block=True)
        return done

    def _collect(self, block: bool) -> List[Completed]:
        out = []
        while self.ticks:
            ticket, items = self.ticks[0]
            if not self.engine.done(ticket):
                if not block:
                    break
                self.engine.wait(ticket)
            t_done = self.clock()
            self.ticks.popleft()
            recs = self.engine.results(ticket)
            for (s, f), r in zip(items, recs):
                s.in_flight -= 1
                if s.closed:
                    self.stats["discarded_results"] += 1
                    self._release_if_idle(s)
                    continue
                lvl = select_level(r, self.rule) if r is not None else -1
                out.append(Completed(s.sid, f.seq, f.t_arrival, t_done, r, lvl))
                self.stats["results" if r is not None else "first_frames"] += 1
            block = False
        return out

    def drain(self) -> List[Completed]:
        """Run ticks until nothing is pending or in flight."""
        out = []
        while self.ticks or self.pending_frames():
            out += self.step(block=True)
        return out


# ---------------------------------------------------------------------------------
# engines
# ---------------------------------------------------------------------------------

class _DevStream:
    """Device state of one stream: three frame slots and two pyramid blocks."""

    def __init__(self, H, W, dtype, levels, device):
        self.H, self.W = H, W
        self.frames = torch.empty((3, H, W), dtype=dtype, device=device)
        lay = pyramid_layout(H, W, levels, dtype)
        self.pyr_bytes = lay["bytes"]
        self.pyr = torch.empty((2, max(self.pyr_bytes, 256)), dtype=torch.uint8, device=device)
        self.cur = -1          # slot of the resident previous frame, -1: none yet
        self.pyr_cur = 0       # block holding the resident frame's pyramid
        self.pyr_valid = False


def _dev_stream_bytes(H, W, dtype, levels) -> int:
    es = torch.tensor([], dtype=dtype).element_size()
    return 3 * H * W * es + 2 * max(pyramid_layout(H, W, levels, dtype)["bytes"], 256)


class CudaBatchEngine:
    """Ticks as batches: uploads on a copy stream, one prepare + run per tick on the
    compute stream, per-level records copied to pinned host memory."""

    def __init__(self, max_H: int, max_W: int, levels: int, max_batch: int, dtype=torch.uint8, mode: int = MODE_FOE,
                 rows_per_tile: Optional[list] = None, device=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.levels, self.max_batch, self.dtype, self.mode = levels, max_batch, dtype, mode
        self.max_H, self.max_W = max_H, max_W
        _frame_args(torch.empty(0, dtype=dtype))          # uint8 or float32 only
        self.ctx = TtcContext(max_H, max_W, max_levels=levels, max_pairs=max_batch, device=self.device)
        # a fixed tile plan makes each pair's result independent of the rest of its tick
        self.ctx.batch_set_plan(rows_per_tile or [64] * levels)
        self.compute = torch.cuda.Stream(self.device)
        self.copy = torch.cuda.Stream(self.device)
        n = max_batch * levels
        self.dev_out = [self.ctx.new_results(n) for _ in range(2)]
        self.host_out = [torch.empty(n * RESULT_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
                         for _ in range(2)]
        self.k = 0
        self.launches = 0

    def fixed_bytes(self) -> int:
        return self.ctx.workspace_bytes + 2 * self.dev_out[0].numel()

    def fits(self, H, W) -> bool:
        return H <= self.max_H and W <= self.max_W and (H >> (self.levels - 1)) >= 2 and (W >> (self.levels - 1)) >= 2

    def stream_bytes(self, H, W) -> int:
        return _dev_stream_bytes(H, W, self.dtype, self.levels)

    def open(self, H, W):
        return _DevStream(H, W, self.dtype, self.levels, self.device)

    def close(self, h):
        h.frames = None
        h.pyr = None

    def has_prev(self, h) -> bool:
        return h.cur >= 0

    def set_plan(self, rows_per_tile):
        self.ctx.batch_set_plan(rows_per_tile)

    def autotune(self, host_pairs, reps: int = 3) -> list:
        """Time 64- and 16-row tiles per level on a representative batch of host frame
        pairs [(prev, cur)] and keep the faster plan (fixed from then on)."""
        with torch.cuda.stream(self.compute):
            dev = [(a.to(self.device, non_blocking=True), b.to(self.device, non_blocking=True)) for a, b in host_pairs]
            self.ctx.batch_prepare(dev, self.levels)
            rows = self.ctx.batch_autotune(self.mode, reps=reps, out=self.dev_out[0])
        self.compute.synchronize()
        self.ctx.batch_set_plan(rows)
        return rows

    def launch(self, items):
        up = torch.cuda.Event()
        pairs, index, slots = [], [], []
        with torch.cuda.stream(self.copy):
            for h, f in items:
                slot = (h.cur + 1) % 3
                h.frames[slot].copy_(f.data, non_blocking=True)
                slots.append(slot)
            up.record(self.copy)
        for (h, _), slot in zip(items, slots):
            if h.cur >= 0:
                nxt = 1 - h.pyr_cur
                prev_pyr = h.pyr[h.pyr_cur] if h.pyr_valid else None
                index.append(len(pairs))
                pairs.append((h.frames[h.cur], h.frames[slot], prev_pyr, h.pyr[nxt]))
                h.pyr_cur, h.pyr_valid = nxt, True
            else:
                index.append(None)
            h.cur = slot
        k = self.k % 2
        self.k += 1
        n = len(pairs)
        with torch.cuda.stream(self.compute):
            self.compute.wait_event(up)
            if n:
                self.ctx.batch_prepare(pairs, self.levels)
                self.ctx.batch_run(self.mode, out=self.dev_out[k])
                self.launches += self.ctx.last_launch_count
                nb = n * self.levels * RESULT_DTYPE.itemsize
                self.host_out[k][:nb].copy_(self.dev_out[k][:nb], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.compute)
        return ev, k, index, n, pairs

    def done(self, ticket) -> bool:
        return ticket[0].query()

    def wait(self, ticket):
        ticket[0].synchronize()

    def results(self, ticket):
        _, k, index, n, _ = ticket
        L = self.levels
        recs = results_to_numpy(self.host_out[k][:n * L * RESULT_DTYPE.itemsize]) if n else None
        return [recs[i * L:(i + 1) * L].copy() if i is not None else None for i in index]


class PerFrameEngine:
    """The plain per-frame path: each frame is uploaded and solved with one
    ``ttc_solve`` call against the stream's resident previous frame (pyramids are
    rebuilt in the context each time), one pair after another."""

    def __init__(self, max_H: int, max_W: int, levels: int, dtype=torch.uint8, mode: int = MODE_FOE, device=None,
                 max_items: int = 64):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.levels, self.dtype, self.mode = levels, dtype, mode
        self.max_H, self.max_W = max_H, max_W
        self.ctx = TtcContext(max_H, max_W, max_levels=levels, max_pairs=1, device=self.device)
        self.compute = torch.cuda.Stream(self.device)
        self.dev_out = self.ctx.new_results(levels)
        # pinned host records, a ring as deep as a tick can be (two ticks in flight)
        self.host_ring = torch.empty((2 * max_items, levels * RESULT_DTYPE.itemsize), dtype=torch.uint8,
                                     pin_memory=True)
        self.ring_pos = 0
        self.launches = 0

    def fixed_bytes(self) -> int:
        return self.ctx.workspace_bytes + self.dev_out.numel()

    def fits(self, H, W) -> bool:
        return H <= self.max_H and W <= self.max_W and (H >> (self.levels - 1)) >= 2 and (W >> (self.levels - 1)) >= 2

    def stream_bytes(self, H, W) -> int:
        es = torch.tensor([], dtype=self.dtype).element_size()
        return 2 * H * W * es

    def open(self, H, W):
        h = _DevStream.__new__(_DevStream)
        h.H, h.W = H, W
        h.frames = torch.empty((2, H, W), dtype=self.dtype, device=self.device)
        h.cur = -1
        return h

    def close(self, h):
        h.frames = None

    def has_prev(self, h) -> bool:
        return h.cur >= 0

    def launch(self, items):
        recs = []
        with torch.cuda.stream(self.compute):
            for h, f in items:
                slot = (h.cur + 1) % 2
                h.frames[slot].copy_(f.data, non_blocking=True)
                if h.cur >= 0:
                    self.ctx.solve(h.frames[h.cur], h.frames[slot], self.levels, self.mode, out=self.dev_out)
                    self.launches += self.ctx.last_launch_count
                    host = self.host_ring[self.ring_pos % self.host_ring.shape[0]]
                    self.ring_pos += 1
                    host.copy_(self.dev_out, non_blocking=True)
                    recs.append(host)
                else:
                    recs.append(None)
                h.cur = slot
            ev = torch.cuda.Event()
            ev.record(self.compute)
        return ev, recs

    def done(self, ticket) -> bool:
        return ticket[0].query()

    def wait(self, ticket):
        ticket[0].synchronize()

    def results(self, ticket):
        return [results_to_numpy(r).copy() if r is not None else None for r in ticket[1]]


def latency_summary(done: List[Completed]) -> dict:
    lat = np.array([c.latency for c in done if c.records is not None], dtype=np.float64) * 1e3
    if lat.size == 0:
        return {"n": 0}
    return {"n": int(lat.size), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "mean_ms": float(lat.mean())}


def replay(server: Server, arrivals, frame_fn, clock=time.perf_counter) -> List[Completed]:
    """Real-time replay: arrivals [(t_seconds, stream, seq)] are offered when the clock
    reaches them (stamped with their scheduled time, so that a late offer counts as
    latency), and ticks run whenever frames are pending and a tick slot is free."""
    done: List[Completed] = []
    t0 = clock()
    i, n = 0, len(arrivals)
    while i < n or server.ticks or server.pending_frames():
        now = clock() - t0
        while i < n and arrivals[i][0] <= now:
            t, sid, seq = arrivals[i]
            server.offer(Frame(sid, seq, t0 + t, frame_fn(sid, seq)))
            i += 1
        done += server.step(block=False)
        if i < n and not server.ticks and not server.pending_frames():
            wait = arrivals[i][0] - (clock() - t0)
            if wait > 2e-4:
                time.sleep(wait - 1e-4)
    return done


def saturate(server: Server, frame_fn, ticks: int, clock=time.perf_counter) -> List[Completed]:
    """As fast as possible: every open stream always has its next frame waiting."""
    done: List[Completed] = []
    seq = collections.Counter()
    launched = server.stats["ticks"] + ticks
    while server.stats["ticks"] < launched or server.ticks:
        if server.stats["ticks"] < launched:
            for sid, st in list(server.streams.items()):
                if not st.pending and not st.closed:
                    server.offer(Frame(sid, seq[sid], clock(), frame_fn(sid, seq[sid])))
                    seq[sid] += 1
        done += server.step(block=len(server.ticks) >= server.max_in_flight)
    # frames still waiting when the target was reached went into further ticks: the loop
    # ends only when nothing is in flight, and a step launches whatever waits
    return done


class _NativeStream:
    def __init__(self, srv, nid, H, W):
        self._srv, self.nid, self.H, self.W = srv, nid, H, W
        self.closed = False

    @property
    def pending(self):
        # waiting frames (not yet in a tick), as the drivers expect
        return self._srv._L.ttc_server_waiting(self._srv._h, self.nid)


class NativeServer:
    """The serving runtime of the library (ttc_server_*): the same admission, ticks and
    fault handling as Server, run natively (uploads, batch, records, level choice), with
    the interface the replay / saturate drivers use."""

    def __init__(self, max_H: int, max_W: int, levels: int, hbm_budget_bytes: int, max_batch: int,
                 mode: int = MODE_FOE, rule: int = 0, dtype=torch.uint8, max_streams: int = 256,
                 max_pending: int = 4, rows_per_tile: Optional[list] = None, clock=time.perf_counter):
        import ctypes
        from . import SERVED_DTYPE, load, _check, _vp
        self._ct = ctypes
        self._L = load()
        self._SERVED = SERVED_DTYPE
        self.levels, self.rule, self.dtype = levels, rule, dtype
        self.max_in_flight = 2
        self.clock = clock
        rows = (ctypes.c_int * levels)(*(rows_per_tile or [64] * levels))
        h = _vp()
        _check(self._L.ttc_server_create(ctypes.byref(h), max_H, max_W, levels, mode, rule,
                                         0 if dtype == torch.uint8 else 1, max_batch, max_streams, max_pending,
                                         int(hbm_budget_bytes), rows), "ttc_server_create")
        self._h = h
        self._check = _check
        self.streams: Dict[int, _NativeStream] = {}
        self._keep: Dict[tuple, Frame] = {}
        self._buf = np.zeros(256, dtype=SERVED_DTYPE)
        self.stats = collections.Counter()

    @property
    def used(self) -> int:
        return int(self._L.ttc_server_bytes_in_use(self._h))

    @property
    def ticks(self):
        return [None] * int(self._L.ttc_server_in_flight(self._h))

    def pending_frames(self) -> int:
        return int(self._L.ttc_server_waiting(self._h, -1))

    def admit(self, sid: int, H: int, W: int) -> bool:
        if sid in self.streams:
            raise ValueError(f"stream {sid} is already admitted")
        nid = self._ct.c_int(-1)
        st = self._L.ttc_server_admit(self._h, H, W, self._ct.byref(nid))
        if st == 4:
            self.stats["rejected_streams"] += 1
            return False
        self._check(st, "ttc_server_admit")
        self.streams[sid] = _NativeStream(self, nid.value, H, W)
        self._sid = getattr(self, "_sid", {})
        self._sid[nid.value] = sid
        self.stats["admitted_streams"] += 1
        return True

    def remove(self, sid: int):
        st = self.streams.pop(sid, None)
        if st is None:
            return
        st.closed = True
        self._check(self._L.ttc_server_remove(self._h, st.nid), "ttc_server_remove")

    def offer(self, frame: Frame) -> bool:
        st = self.streams.get(frame.stream)
        d = frame.data
        if (st is None or not isinstance(d, torch.Tensor) or d.dim() != 2 or d.is_cuda or d.dtype != self.dtype
                or tuple(d.shape) != (st.H, st.W) or d.stride(1) != 1):
            self.stats["rejected_frames"] += 1
            return False
        r = self._L.ttc_server_submit(self._h, st.nid, d.data_ptr(), d.stride(0) * d.element_size(),
                                      int(frame.seq), float(frame.t_arrival))
        if r != 0:
            self.stats["rejected_frames"] += 1
            return False
        self._keep[(st.nid, int(frame.seq))] = frame      # alive until reported
        self.stats["offered_frames"] += 1
        return True

    def step(self, block: bool = False) -> List[Completed]:
        n = self._ct.c_int(0)
        self._check(self._L.ttc_server_step(self._h, 1 if block else 0, self._buf.ctypes.data, len(self._buf),
                                            self._ct.byref(n)), "ttc_server_step")
        t_done = self.clock()
        out = []
        for r in self._buf[:n.value]:
            nid, seq, status = int(r["stream"]), int(r["seq"]), int(r["status"])
            self._keep.pop((nid, seq), None)
            sid = self._sid.get(nid, nid)
            if status == 1:
                out.append(Completed(sid, seq, float(r["t_arrival"]), t_done, r["records"][:self.levels].copy(),
                                     int(r["level"])))
                self.stats["results"] += 1
            elif status == 0:
                out.append(Completed(sid, seq, float(r["t_arrival"]), t_done, None, -1))
                self.stats["first_frames"] += 1
            elif status == -1:
                self.stats["dropped_frames"] += 1
            else:
                self.stats["discarded_results"] += 1
        self.stats["ticks"] = int(self._L.ttc_server_ticks(self._h))
        return out

    def drain(self) -> List[Completed]:
        out = []
        while self.ticks or self.pending_frames():
            out += self.step(block=True)
        return out

    def drive(self, frames: Dict[int, list], pairs: int) -> dict:
        """The library's load generator (ttc_server_drive): every stream in `frames`
        (sid -> list of host frames of its size, cycled) always has a frame waiting; the
        server is stepped natively, two ticks in flight, until `pairs` results are back,
        and the ticks still in flight then complete too (so "pairs" may exceed the
        request; the server is idle on return).  Returns seconds, pairs served and
        p50 / p99 latency (ms, submission to report)."""
        ct = self._ct
        sids = list(frames)
        nf = len(frames[sids[0]])
        if any(len(frames[s]) != nf for s in sids):
            raise ValueError("every stream gives the same number of frames")
        ids = (ct.c_int * len(sids))(*[self.streams[s].nid for s in sids])
        ptrs = (ct.c_void_p * (len(sids) * nf))(*[f.data_ptr() for s in sids for f in frames[s]])
        pitches = (ct.c_int64 * len(sids))(*[frames[s][0].stride(0) * frames[s][0].element_size() for s in sids])
        sec, got = ct.c_double(0), ct.c_int64(0)
        p50, p99 = ct.c_double(0), ct.c_double(0)
        self._check(self._L.ttc_server_drive(self._h, ids, len(sids), ptrs, pitches, nf, int(pairs), ct.byref(sec),
                                             ct.byref(got), ct.byref(p50), ct.byref(p99)), "ttc_server_drive")
        self.stats["ticks"] = int(self._L.ttc_server_ticks(self._h))
        return {"seconds": sec.value, "pairs": int(got.value), "p50_ms": p50.value, "p99_ms": p99.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.ttc_server_destroy(self._h)
            self._h = self._ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
