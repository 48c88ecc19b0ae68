"""Serving path on the GPU: caller-owned per-frame pyramids in the batch API, and the
serving loop over the batch engine (results vs the oracle, identical alone and in a
mix of streams, host-side faults)."""
import collections

import numpy as np
import pytest
import torch

import oracle
import paper_1612_08825_gb300 as ft
import scenes
from _tol import check_record
from paper_1612_08825_gb300.serve import CudaBatchEngine, Frame, PerFrameEngine, Server, replay, saturate

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
LEVELS = 4
PLAN = [64, 64, 16, 16]


def _video(H, W, n, seed):
    sc = scenes.tilted_plane_scene(H=H, W=W, seed=seed, Z0=18.0, speed=0.06, m=16, pmin=3.0, pmax=40.0)
    return scenes.render_sequence(sc, n, device=DEV).cpu()


SIZES = [(120, 160), (243, 337), (480, 640), (1080, 1920), (35, 71)]


def _pyr_level(block, lay, l, H, W):
    off, pitch = lay["offsets"][l], lay["pitches"][l]
    h, w = H >> l, W >> l
    raw = block[off:off + pitch * h].view(h, pitch)[:, :2 * w].contiguous()
    return raw.view(torch.int16).to(torch.int32).cpu().numpy() & 0xFFFF


def test_pyramid_layout_and_plan_errors():
    lay = ft.pyramid_layout(1080, 1920, 4)
    assert lay["pitches"][1:] == [1920, 960, 480]
    assert lay["bytes"] == sum(((lay["pitches"][l] * (1080 >> l) + 255) // 256) * 256 for l in (1, 2, 3))
    with pytest.raises(ft.FtError):
        ft.pyramid_layout(12, 12, 4)                       # level 3 would be 1 x 1
    ctx = ft.TtcContext(64, 64, 3, 2)
    with pytest.raises(ft.FtError):
        ctx.batch_set_plan([64, 32, 16])
    ctx.batch_set_plan([64, 16, 16])
    ctx.batch_set_plan(None)
    ctx.close()


def test_caller_pyramids_same_as_context_pyramids():
    """Pairs (f0, f1) then (f1, f2) with the pyramids in caller blocks (f1's built
    once, by the first pair, and read by the second) give bitwise the records of the
    same pairs with context pyramids; the stored levels are the exact block sums."""
    vids = [_video(H, W, 3, 50 + i) for i, (H, W) in enumerate(SIZES)]
    dev = [v.to(DEV) for v in vids]
    n = len(SIZES)
    ctx = ft.TtcContext(1080, 1920, LEVELS, 2 * n)
    ctx.batch_set_plan(PLAN)
    ctx.batch_prepare([(d[0], d[1]) for d in dev] + [(d[1], d[2]) for d in dev], levels=LEVELS)
    ref = ft.results_to_numpy(ctx.batch_run(mode=1)).reshape(2, n, LEVELS)
    lays = [ft.pyramid_layout(H, W, LEVELS) for H, W in SIZES]
    blocks = [torch.full((2, max(l["bytes"], 256)), 0xAB, dtype=torch.uint8, device=DEV) for l in lays]
    ctx.batch_prepare([(d[0], d[1], None, b[0]) for d, b in zip(dev, blocks)], levels=LEVELS)
    first = ft.results_to_numpy(ctx.batch_run(mode=1)).reshape(n, LEVELS)
    ctx.batch_prepare([(d[1], d[2], b[0], b[1]) for d, b in zip(dev, blocks)], levels=LEVELS)
    second = ft.results_to_numpy(ctx.batch_run(mode=1)).reshape(n, LEVELS)
    torch.cuda.synchronize()
    assert first.tobytes() == ref[0].tobytes()
    assert second.tobytes() == ref[1].tobytes()
    for i, (H, W) in enumerate(SIZES):
        for k, frame in ((0, vids[i][1]), (1, vids[i][2])):
            img = frame.numpy().astype(np.float64)
            for l in range(1, LEVELS):
                img = oracle.downsample(img)
                got = _pyr_level(blocks[i][k], lays[i], l, H, W)
                assert np.array_equal(got, (img * 4 ** l).astype(np.int64)), (H, W, k, l)
        if (H, W) == (1080, 1920):
            continue
        for p in range(2):
            r = oracle.ttc_pair(vids[i][p].numpy(), vids[i][p + 1].numpy(), levels=LEVELS, mode=1)
            for l in range(LEVELS):
                check_record((first, second)[p][i, l], r[l], 1, l)
    ctx.close()


def test_misaligned_pyramid_rejected():
    v = _video(64, 96, 2, 7).to(DEV)
    ctx = ft.TtcContext(64, 96, 3, 1)
    blk = torch.zeros(4096, dtype=torch.uint8, device=DEV)
    with pytest.raises(ft.FtError):
        ctx.batch_prepare([(v[0], v[1], None, blk[8:])], levels=3)
    with pytest.raises(ft.FtError):
        ctx.batch_prepare([(v[0], v[1], blk, blk)], levels=3)
    ctx.close()


STREAMS = [(0, 120, 160), (1, 480, 640), (2, 243, 337), (3, 1080, 1920), (4, 240, 320), (5, 35, 71)]
NFR = 5


def _serve(streams, frames, engine_kind="batch", remove_at=None):
    if engine_kind == "batch":
        eng = CudaBatchEngine(1080, 1920, LEVELS, max_batch=8, rows_per_tile=PLAN)
    else:
        eng = PerFrameEngine(1080, 1920, LEVELS)
    srv = Server(eng, 40 << 30, max_batch=8)
    for sid, H, W in streams:
        assert srv.admit(sid, H, W)
    done = []
    for k in range(NFR):
        for sid, _, _ in streams:
            if remove_at is not None and (sid, k) == remove_at:
                srv.remove(sid)
            srv.offer(Frame(sid, k, float(k), frames[sid][k]))
        done += srv.step()
    done += srv.drain()
    return done, srv


def test_server_results_oracle_and_mix_invariance():
    frames = {sid: _video(H, W, NFR, 200 + sid).pin_memory() for sid, H, W in STREAMS}
    mix, srv = _serve(STREAMS, frames)
    assert srv.stats["results"] == len(STREAMS) * (NFR - 1) and srv.stats["first_frames"] == len(STREAMS)
    by = {(c.stream, c.seq): c for c in mix}
    for sid, H, W in STREAMS:
        alone, _ = _serve([(sid, H, W)], frames)
        for c in alone:
            m = by[(sid, c.seq)]
            if c.records is None:
                assert m.records is None
                continue
            assert m.records.tobytes() == c.records.tobytes(), (sid, c.seq)
            assert m.level == c.level
        if H * W > 500_000:
            continue
        for k in range(1, NFR):
            r = oracle.ttc_pair(frames[sid][k - 1].numpy(), frames[sid][k].numpy(), levels=LEVELS, mode=1)
            for l in range(LEVELS):
                check_record(by[(sid, k)].records[l], r[l], 1, l)


def test_server_stream_removed_mid_flight_others_unchanged():
    frames = {sid: _video(H, W, NFR, 400 + sid).pin_memory() for sid, H, W in STREAMS}
    full, _ = _serve(STREAMS, frames)
    cut, srv = _serve(STREAMS, frames, remove_at=(3, 2))
    assert all(c.stream != 3 or c.seq < 2 for c in cut)
    assert 3 not in srv.streams
    ref = {(c.stream, c.seq): c.records for c in full}
    for c in cut:
        if c.records is not None:
            assert c.records.tobytes() == ref[(c.stream, c.seq)].tobytes()


def test_per_frame_engine_matches_batch_engine():
    frames = {sid: _video(H, W, NFR, 600 + sid).pin_memory() for sid, H, W in STREAMS[:3]}
    a, _ = _serve(STREAMS[:3], frames)
    b, _ = _serve(STREAMS[:3], frames, engine_kind="per_frame")
    ra = {(c.stream, c.seq): c.records for c in a if c.records is not None}
    for c in b:
        if c.records is None:
            continue
        r = oracle.ttc_pair(frames[c.stream][c.seq - 1].numpy(), frames[c.stream][c.seq].numpy(),
                            levels=LEVELS, mode=1)
        for l in range(LEVELS):
            check_record(c.records[l], r[l], 1, l)
            check_record(ra[(c.stream, c.seq)][l], r[l], 1, l)


def test_replay_and_saturate_on_gpu():
    frames = {sid: _video(H, W, 3, 800 + sid).pin_memory() for sid, H, W in STREAMS}
    eng = CudaBatchEngine(1080, 1920, LEVELS, max_batch=8, rows_per_tile=PLAN)
    srv = Server(eng, 40 << 30, max_batch=8)
    for sid, H, W in STREAMS:
        srv.admit(sid, H, W)
    arr = scenes.poisson_arrivals(len(STREAMS), 200.0, 0.05, seed=3)
    done = replay(srv, arr, lambda s, q: frames[s][q % 3])
    assert len(done) == len(arr) - srv.stats["dropped_frames"]
    assert all(c.latency >= 0 for c in done)
    n0 = srv.stats["results"]
    saturate(srv, lambda s, q: frames[s][q % 3], ticks=6)
    assert srv.stats["results"] - n0 >= 5 * len(STREAMS)
    assert eng.launches > 0


from paper_1612_08825_gb300.serve import NativeServer  # noqa: E402


def _serve_native(streams, frames, remove_at=None, max_pending=4):
    srv = NativeServer(1080, 1920, LEVELS, 40 << 30, max_batch=8, rows_per_tile=PLAN, max_pending=max_pending)
    for sid, H, W in streams:
        assert srv.admit(sid, H, W)
    done = []
    for k in range(NFR):
        for sid, _, _ in streams:
            if remove_at is not None and (sid, k) == remove_at:
                srv.remove(sid)
            srv.offer(Frame(sid, k, float(k), frames[sid][k]))
        done += srv.step()
    done += srv.drain()
    return done, srv


def test_native_server_matches_python_server_bitwise():
    """The native serving runtime and the Python server over the same batch API give
    bitwise the same records and level choices for every frame."""
    frames = {sid: _video(H, W, NFR, 900 + sid).pin_memory() for sid, H, W in STREAMS}
    py, _ = _serve(STREAMS, frames)
    nat, srv = _serve_native(STREAMS, frames)
    assert srv.stats["results"] == len(STREAMS) * (NFR - 1) and srv.stats["first_frames"] == len(STREAMS)
    a = {(c.stream, c.seq): c for c in py}
    b = {(c.stream, c.seq): c for c in nat}
    assert a.keys() == b.keys()
    for key, c in a.items():
        if c.records is None:
            assert b[key].records is None
        else:
            assert b[key].records.tobytes() == c.records.tobytes(), key
            assert b[key].level == c.level
    srv.close()


def test_native_server_faults():
    frames = {sid: _video(H, W, NFR, 950 + sid).pin_memory() for sid, H, W in STREAMS}
    cut, srv = _serve_native(STREAMS, frames, remove_at=(3, 2))
    assert all(c.stream != 3 or c.seq < 2 for c in cut)
    full = {(c.stream, c.seq): c.records for c in _serve_native(STREAMS, frames)[0]}
    for c in cut:
        if c.records is not None:
            assert c.records.tobytes() == full[(c.stream, c.seq)].tobytes()
    srv.close()
    # queue overflow: five frames offered before any step with room for two
    srv = NativeServer(480, 640, LEVELS, 40 << 30, max_batch=8, rows_per_tile=PLAN, max_pending=2)
    assert srv.admit(0, 480, 640)
    f = _video(480, 640, 5, 77).pin_memory()
    for k in range(5):
        assert srv.offer(Frame(0, k, float(k), f[k]))
    done = srv.drain()
    assert srv.stats["dropped_frames"] == 3 and [c.seq for c in done] == [3, 4]
    # malformed and oversized requests
    assert not srv.offer(Frame(0, 9, 0.0, f[0][:, :100]))
    assert not srv.admit(1, 1080, 1920)                        # larger than the server's frames
    srv.close()
    with pytest.raises(ft.FtError):
        NativeServer(480, 640, LEVELS, 1024, max_batch=8)     # the budget cannot hold the workspace


def test_native_server_replay_and_saturate():
    frames = {sid: _video(H, W, 3, 990 + sid).pin_memory() for sid, H, W in STREAMS}
    srv = NativeServer(1080, 1920, LEVELS, 40 << 30, max_batch=8, rows_per_tile=PLAN)
    for sid, H, W in STREAMS:
        srv.admit(sid, H, W)
    arr = scenes.poisson_arrivals(len(STREAMS), 200.0, 0.05, seed=3)
    done = replay(srv, arr, lambda s, q: frames[s][q % 3])
    assert len(done) == len(arr) - srv.stats["dropped_frames"]
    n0 = srv.stats["results"]
    saturate(srv, lambda s, q: frames[s][q % 3], ticks=6)
    assert srv.stats["results"] - n0 >= 5 * len(STREAMS)
    srv.close()


def test_native_load_generator():
    """ttc_server_drive keeps every stream supplied and returns at least the pairs asked
    for, with latencies; the server then still serves frames offered the ordinary way."""
    frames = {sid: _video(H, W, 3, 1200 + sid).pin_memory() for sid, H, W in STREAMS}
    srv = NativeServer(1080, 1920, LEVELS, 40 << 30, max_batch=8, rows_per_tile=PLAN)
    for sid, H, W in STREAMS:
        assert srv.admit(sid, H, W)
    r = srv.drive({sid: list(frames[sid]) for sid, *_ in STREAMS}, pairs=10 * len(STREAMS))
    assert r["pairs"] >= 10 * len(STREAMS) and r["seconds"] > 0
    assert 0 < r["p50_ms"] <= r["p99_ms"]
    for sid, H, W in STREAMS:
        assert srv.offer(Frame(sid, 10 ** 6, 0.0, frames[sid][0]))
    res = [c for c in srv.drain() if c.records is not None]
    assert sorted(c.stream for c in res) == sorted(sid for sid, *_ in STREAMS)
    for c in res:
        assert c.records.shape[0] == LEVELS and np.all(c.records["flags"] & ft.FLAG_TIMEOUT == 0)
    srv.close()


def _serve_native_records(streams, frames, dtype):
    srv = NativeServer(1080, 1920, LEVELS, 40 << 30, max_batch=8, rows_per_tile=PLAN, dtype=dtype)
    for sid, H, W in streams:
        assert srv.admit(sid, H, W)
    done = []
    for k in range(NFR):
        for sid, _, _ in streams:
            assert srv.offer(Frame(sid, k, float(k), frames[sid][k]))
        done += srv.step()
    done += srv.drain()
    n = srv.stats["results"]
    srv.close()
    return {(c.stream, c.seq): (c.records.tobytes(), c.level) for c in done if c.records is not None}, n


def test_native_server_upload_paths_bitwise():
    """A frame reaches its device slot by the gather kernel (under 1 MB, in page-locked
    memory, rows and pitch whole 16-byte words) or by the copy engine (pageable memory,
    large frames, other pitches); contiguous or pitched, the records are bitwise the same."""
    streams = [(0, 120, 160), (1, 240, 320), (2, 480, 640), (3, 720, 1280), (4, 100, 200), (5, 1080, 1920)]
    for dtype in (torch.uint8, torch.float32):
        ss = streams if dtype == torch.uint8 else streams[:3]
        base = {sid: _video(H, W, NFR, 1300 + sid) for sid, H, W in ss}
        if dtype != torch.uint8:
            base = {sid: v.float() for sid, v in base.items()}
        es = base[0].element_size()

        def pitched(v, pin, extra):
            n, H, W = v.shape
            buf = torch.zeros((n, H, W + extra), dtype=v.dtype)
            if pin:
                buf = buf.pin_memory()
            buf[:, :, :W] = v
            return buf[:, :, :W]

        def pad16(W):
            # elements that take the row to the next multiple of 16 bytes, plus 16 bytes
            return (-(W * es) % 16) // es + 16 // es

        variants = {
            "page-locked": {sid: v.pin_memory() for sid, v in base.items()},
            "pageable": {sid: v.clone() for sid, v in base.items()},
            "page-locked pitched": {sid: pitched(v, True, pad16(v.shape[2])) for sid, v in base.items()},
            "pageable pitched": {sid: pitched(v, False, pad16(v.shape[2])) for sid, v in base.items()},
            "page-locked, pitch not a 16-byte multiple": {sid: pitched(v, True, 3) for sid, v in base.items()},
        }
        ref = None
        for name, frames in variants.items():
            got, n = _serve_native_records(ss, frames, dtype)
            assert n == len(ss) * (NFR - 1), name
            if ref is None:
                ref = got
            else:
                assert got.keys() == ref.keys(), name
                for key in ref:
                    assert got[key] == ref[key], (dtype, name, key)
