// Serving runtime: many camera streams, continuous batching over the batch entry
// points (no counterpart in the paper, which processes one camera; Sec. V-B's estimate
// is produced at every frame of every stream).
//
// Every admitted stream owns three device frame slots and two pyramid blocks (levels
// 1..L-1 of its last two frames).  A tick takes at most one waiting frame per stream
// (oldest arrival first, at most max_batch pairs), uploads the frames (one copy-engine copy
// each on a copy stream; small frames in page-locked memory by a gather kernel on a third
// stream, which reads the caller's host memory directly), and runs one ttc_batch_prepare +
// ttc_batch_run on the compute stream: the pair (previous frame, new frame) reads the
// previous frame's pyramid from one block and writes the new frame's to the other, so
// every frame is uploaded once and its pyramid built once.  The records come back to
// page-locked host memory; the multi-scale rule picks a level on the host.  At most two
// ticks are in flight, so the uploads and host work of one overlap the kernels of the
// other; with three frame slots per stream, the slot a tick uploads into was last read
// by a tick that has completed.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include "common.cuh"

namespace {

struct Frame {
    const void *host;
    int64_t pitch, seq;
    double t;
};

struct Stream {
    int H = 0, W = 0;
    bool open = false, closing = false;
    unsigned char *mem = nullptr;          // 3 frame slots, then 2 pyramid blocks
    size_t slot_bytes = 0, pyr_bytes = 0, nbytes = 0;
    int cur = -1;                          // slot of the resident previous frame
    int pyr_cur = 0;                       // block holding its pyramid
    bool pyr_valid = false;
    int in_flight = 0;                     // frames of this stream in ticks not yet collected
    std::deque<Frame> pending;
};

struct Item {
    int stream;
    Frame f;
    int pair;                              // index in the tick's batch, -1 for a first frame
};

struct Tick {
    cudaEvent_t ev;
    int buf;
    std::vector<Item> items;
};

}  // namespace

struct ttc_server {
    int max_H, max_W, levels, mode, rule, dtype, es, max_batch, max_streams, max_pending;
    int64_t budget, used;
    ttc_ctx *ctx = nullptr;
    cudaStream_t compute = nullptr, copy = nullptr, gather = nullptr;
    cudaEvent_t up_ev = nullptr, gather_ev = nullptr;
    ttc_level_result *dev_out[2] = {nullptr, nullptr};
    ttc_level_result *host_out[2] = {nullptr, nullptr};
    std::vector<Stream> streams;
    std::deque<Tick> ticks;
    std::vector<cudaEvent_t> spare_events;
    std::deque<ttc_served> reports;        // ready for the caller
    std::vector<ttc_pair_desc> descs;
    int next_buf = 0;
    int64_t launched = 0;                  // ticks launched so far
};

namespace {

ft_status cuda_fail(cudaError_t e)
{
    ft::set_cuda_error(e);
    return FT_ERR_CUDA;
}

void report(ttc_server *s, int stream, const Frame &f, int status)
{
    ttc_served r;
    std::memset(&r, 0, sizeof(r));
    r.stream = stream;
    r.seq = f.seq;
    r.t_arrival = f.t;
    r.status = status;
    r.level = -1;
    s->reports.push_back(r);
}

void release(ttc_server *s, int id)
{
    Stream &st = s->streams[(size_t)id];
    if (!st.closing || st.in_flight > 0 || !st.mem) return;
    cudaFree(st.mem);                      // no tick in flight reads it
    st.mem = nullptr;
    s->used -= (int64_t)st.nbytes;
    st.open = false;
}

// collect completed ticks (the oldest one waited for when `wait`)
ft_status collect(ttc_server *s, bool wait)
{
    while (!s->ticks.empty()) {
        Tick &t = s->ticks.front();
        cudaError_t e = wait ? cudaEventSynchronize(t.ev) : cudaEventQuery(t.ev);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) return cuda_fail(e);
        wait = false;
        for (const Item &it : t.items) {
            Stream &st = s->streams[(size_t)it.stream];
            --st.in_flight;
            if (st.closing) {
                report(s, it.stream, it.f, FT_SERVED_DISCARDED);
                release(s, it.stream);
                continue;
            }
            if (it.pair < 0) {
                report(s, it.stream, it.f, FT_SERVED_FIRST_FRAME);
                continue;
            }
            report(s, it.stream, it.f, FT_SERVED_RESULT);
            ttc_served &r = s->reports.back();
            std::memcpy(r.records, s->host_out[t.buf] + (size_t)it.pair * s->levels,
                        (size_t)s->levels * sizeof(ttc_level_result));
            r.level = ttc_select_level(r.records, s->levels, s->rule);
        }
        s->spare_events.push_back(t.ev);
        s->ticks.pop_front();
    }
    return FT_OK;
}

// Small frames go to the device by a kernel that reads the caller's page-locked host
// memory directly: the copy engine spends a fixed time on every copy (about 2 us, against
// 0.4 us of transfer for a 320 x 240 uint8 frame), while one launch moves many frames at
// once, beside the copy engine's copies of the large frames.
// Frames below 1 MB: on 64 streams of 320x240 .. 1920x1080 uint8 frames, a tick took
// 0.316 ms with this limit, 0.335 ms with 512 KB, and 0.41 ms with every frame gathered
// (the kernel then competes with the previous tick's kernels for the SMs).
constexpr size_t GATHER_BYTES = 1024 * 1024;
constexpr int GATHER_MAX = 48;                // frames per launch (kernel parameter space)
constexpr int GATHER_THREADS = 256;
constexpr int GATHER_UNROLL = 8;              // 16-byte words per thread in flight
constexpr int GATHER_WORDS = GATHER_THREADS * GATHER_UNROLL;   // per CTA

struct GatherFrame {
    const int4 *src;                          // device address of the first row
    int4 *dst;                                // contiguous destination (the frame slot)
    int pitch16, row16, rows;                 // source pitch and row length in 16-byte words
    int first_block;                          // first CTA of the frame
};

struct GatherList {
    GatherFrame f[GATHER_MAX];
    int n;
};

__global__ void __launch_bounds__(GATHER_THREADS) gather_frames_kernel(const GatherList L)
{
    // the frame of this CTA: the last one whose first CTA is at or before it
    int lo = 0, hi = L.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.f[mid].first_block <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const GatherFrame g = L.f[lo];
    const int words = g.rows * g.row16;
    const int w0 = ((int)blockIdx.x - g.first_block) * GATHER_WORDS + (int)threadIdx.x;
    int4 v[GATHER_UNROLL];
#pragma unroll
    for (int k = 0; k < GATHER_UNROLL; ++k) {
        const int w = w0 + k * GATHER_THREADS;
        if (w < words) {
            const int r = w / g.row16;
            v[k] = g.src[(int64_t)r * g.pitch16 + (w - r * g.row16)];
        }
    }
#pragma unroll
    for (int k = 0; k < GATHER_UNROLL; ++k) {
        const int w = w0 + k * GATHER_THREADS;
        if (w < words) g.dst[w] = v[k];
    }
}

// The device address of page-locked host memory [p, p + extent), 16-byte aligned, with
// both ends in page-locked memory; null otherwise (pageable memory goes to the copy engine).
const void *pinned_device_address(const void *p, size_t extent)
{
    cudaPointerAttributes a{}, b{};
    const unsigned char *last = static_cast<const unsigned char *>(p) + extent - 1;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
        return nullptr;
    const unsigned char *da = static_cast<const unsigned char *>(a.devicePointer);
    const unsigned char *db = static_cast<const unsigned char *>(b.devicePointer);
    if (db - da != (std::ptrdiff_t)(extent - 1) || (reinterpret_cast<uintptr_t>(da) & 15) != 0) return nullptr;
    return da;
}

// launches the gather kernel over the listed frames on the gather stream
cudaError_t launch_gather(ttc_server *s, GatherList &L, int blocks)
{
    if (L.n == 0) return cudaSuccess;
    gather_frames_kernel<<<blocks, GATHER_THREADS, 0, s->gather>>>(L);
    L.n = 0;
    return cudaGetLastError();
}

ft_status launch_tick(ttc_server *s)
{
    std::vector<int> cand;
    for (int i = 0; i < (int)s->streams.size(); ++i) {
        const Stream &st = s->streams[(size_t)i];
        if (st.open && !st.closing && !st.pending.empty()) cand.push_back(i);
    }
    if (cand.empty()) return FT_OK;
    std::stable_sort(cand.begin(), cand.end(), [s](int a, int b) {
        return s->streams[(size_t)a].pending.front().t < s->streams[(size_t)b].pending.front().t;
    });
    Tick t;
    t.buf = s->next_buf;
    int npairs = 0;
    for (int id : cand) {
        Stream &st = s->streams[(size_t)id];
        const bool pair = st.cur >= 0;
        if (pair && npairs >= s->max_batch) continue;
        t.items.push_back({id, st.pending.front(), pair ? npairs : -1});
        st.pending.pop_front();
        npairs += pair;
    }
    // uploads: each frame into the slot after the resident one (that slot was last read by
    // the tick before the previous one, which has completed: at most two are in flight)
    cudaError_t e = cudaSuccess;
    s->descs.clear();
    GatherList gl;
    gl.n = 0;
    int gblocks = 0;
    bool gathered_any = false;
    for (Item &it : t.items) {
        Stream &st = s->streams[(size_t)it.stream];
        const int slot = (st.cur + 1) % 3;
        unsigned char *dst = st.mem + (size_t)slot * st.slot_bytes;
        const size_t row = (size_t)st.W * (size_t)s->es;
        const size_t bytes = row * (size_t)st.H;
        const void *dsrc = nullptr;
        if (bytes < GATHER_BYTES && row % 16 == 0 && it.f.pitch % 16 == 0 && it.f.pitch < ((int64_t)1 << 34))
            dsrc = pinned_device_address(it.f.host, (size_t)it.f.pitch * (size_t)(st.H - 1) + row);
        if (dsrc) {
            // a small page-locked frame: one entry of the gather kernel's list
            GatherFrame &g = gl.f[gl.n++];
            g.src = static_cast<const int4 *>(dsrc);
            g.dst = reinterpret_cast<int4 *>(dst);
            g.pitch16 = (int)(it.f.pitch / 16);
            g.row16 = (int)(row / 16);
            g.rows = st.H;
            g.first_block = gblocks;
            gblocks += (int)((bytes / 16 + GATHER_WORDS - 1) / GATHER_WORDS);
            gathered_any = true;
            if (gl.n == GATHER_MAX) {
                if ((e = launch_gather(s, gl, gblocks)) != cudaSuccess) return cuda_fail(e);
                gblocks = 0;
            }
        } else if ((size_t)it.f.pitch == row) {
            // contiguous rows: one linear copy (a 2-D copy of many short rows runs well below
            // the link's rate); otherwise a 2-D copy
            e = cudaMemcpyAsync(dst, it.f.host, bytes, cudaMemcpyHostToDevice, s->copy);
        } else {
            e = cudaMemcpy2DAsync(dst, row, it.f.host, (size_t)it.f.pitch, row, (size_t)st.H,
                                  cudaMemcpyHostToDevice, s->copy);
        }
        if (e != cudaSuccess) return cuda_fail(e);
        if (st.cur >= 0) {
            unsigned char *pyr = st.mem + 3 * st.slot_bytes;
            const int nxt = 1 - st.pyr_cur;
            ttc_pair_desc d;
            d.prev = st.mem + (size_t)st.cur * st.slot_bytes;
            d.cur = dst;
            d.H = st.H;
            d.W = st.W;
            d.pitch_bytes = (int64_t)row;
            d.prev_pyramid = st.pyr_valid ? pyr + (size_t)st.pyr_cur * st.pyr_bytes : nullptr;
            d.cur_pyramid = pyr + (size_t)nxt * st.pyr_bytes;
            s->descs.push_back(d);
            st.pyr_cur = nxt;
            st.pyr_valid = true;
        }
        st.cur = slot;
        ++st.in_flight;
    }
    if ((e = launch_gather(s, gl, gblocks)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaEventRecord(s->up_ev, s->copy)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaStreamWaitEvent(s->compute, s->up_ev, 0)) != cudaSuccess) return cuda_fail(e);
    if (gathered_any) {
        if ((e = cudaEventRecord(s->gather_ev, s->gather)) != cudaSuccess) return cuda_fail(e);
        if ((e = cudaStreamWaitEvent(s->compute, s->gather_ev, 0)) != cudaSuccess) return cuda_fail(e);
    }
    if (npairs > 0) {
        ft_status st = ttc_batch_prepare(s->ctx, s->descs.data(), npairs, s->dtype, s->levels, s->compute);
        if (st == FT_OK) st = ttc_batch_run(s->ctx, s->mode, s->dev_out[t.buf], s->compute);
        if (st != FT_OK) return st;
        e = cudaMemcpyAsync(s->host_out[t.buf], s->dev_out[t.buf],
                            (size_t)npairs * s->levels * sizeof(ttc_level_result), cudaMemcpyDeviceToHost,
                            s->compute);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (s->spare_events.empty()) {
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e);
        s->spare_events.push_back(ev);
    }
    t.ev = s->spare_events.back();
    s->spare_events.pop_back();
    if ((e = cudaEventRecord(t.ev, s->compute)) != cudaSuccess) return cuda_fail(e);
    s->ticks.push_back(std::move(t));
    s->next_buf ^= 1;
    ++s->launched;
    return FT_OK;
}

}  // namespace

extern "C" ft_status ttc_server_create(ttc_server **out, int max_H, int max_W, int levels, int mode, int rule,
                                       int dtype, int max_batch, int max_streams, int max_pending,
                                       int64_t hbm_budget_bytes, const int *rows_per_tile)
{
    FT_API_RANGE;
    if (!out) return FT_ERR_INVALID_ARG;
    *out = nullptr;
    if ((dtype != FT_U8 && dtype != FT_F32) || (mode != FT_MODE_TTC && mode != FT_MODE_FOE) ||
        (rule != 0 && rule != 1) || max_batch < 1 || max_streams < 1 || max_pending < 1)
        return FT_ERR_INVALID_ARG;
    if (levels < 1) return FT_ERR_INVALID_ARG;
    if (levels > FT_MAX_LEVELS) return FT_ERR_UNSUPPORTED;
    ttc_server *s = new (std::nothrow) ttc_server();
    if (!s) return FT_ERR_WORKSPACE;
    s->max_H = max_H;
    s->max_W = max_W;
    s->levels = levels;
    s->mode = mode;
    s->rule = rule;
    s->dtype = dtype;
    s->es = dtype == FT_U8 ? 1 : 4;
    s->max_batch = max_batch;
    s->max_streams = max_streams;
    s->max_pending = max_pending;
    s->budget = hbm_budget_bytes;
    ft_status st = ttc_ctx_create(&s->ctx, max_H, max_W, levels, max_batch);
    if (st == FT_OK) {
        int rows[FT_MAX_LEVELS];
        for (int l = 0; l < levels; ++l) rows[l] = rows_per_tile ? rows_per_tile[l] : 64;
        st = ttc_batch_set_plan(s->ctx, rows, levels);
    }
    cudaError_t e = cudaSuccess;
    const size_t rec = (size_t)max_batch * levels * sizeof(ttc_level_result);
    if (st == FT_OK) {
        e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->up_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->gather, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->gather_ev, cudaEventDisableTiming);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaMalloc(&s->dev_out[b], rec);
            if (e == cudaSuccess) e = cudaMallocHost(&s->host_out[b], rec);
        }
        if (e != cudaSuccess) st = cuda_fail(e);
    }
    if (st != FT_OK) {
        ttc_server_destroy(s);
        return st;
    }
    s->used = (int64_t)ttc_ctx_workspace_bytes(s->ctx) + 2 * (int64_t)rec;
    if (s->used > s->budget) {
        ttc_server_destroy(s);
        return FT_ERR_WORKSPACE;
    }
    *out = s;
    return FT_OK;
}

extern "C" void ttc_server_destroy(ttc_server *s)
{
    if (!s) return;
    if (s->compute) cudaStreamSynchronize(s->compute);
    if (s->copy) cudaStreamSynchronize(s->copy);
    if (s->gather) cudaStreamSynchronize(s->gather);
    for (Stream &st : s->streams) cudaFree(st.mem);
    for (Tick &t : s->ticks) cudaEventDestroy(t.ev);
    for (cudaEvent_t ev : s->spare_events) cudaEventDestroy(ev);
    for (int b = 0; b < 2; ++b) {
        cudaFree(s->dev_out[b]);
        if (s->host_out[b]) cudaFreeHost(s->host_out[b]);
    }
    if (s->up_ev) cudaEventDestroy(s->up_ev);
    if (s->gather_ev) cudaEventDestroy(s->gather_ev);
    if (s->gather) cudaStreamDestroy(s->gather);
    if (s->compute) cudaStreamDestroy(s->compute);
    if (s->copy) cudaStreamDestroy(s->copy);
    ttc_ctx_destroy(s->ctx);
    delete s;
}

extern "C" ft_status ttc_server_stream_bytes(const ttc_server *s, int H, int W, int64_t *bytes)
{
    if (!s || !bytes) return FT_ERR_INVALID_ARG;
    int64_t pyr = 0;
    const ft_status st = ttc_pyramid_layout(H, W, s->levels, s->dtype, nullptr, nullptr, &pyr);
    if (st != FT_OK) return st;
    const int64_t slot = ((int64_t)H * W * s->es + 255) / 256 * 256;
    *bytes = 3 * slot + 2 * ((std::max<int64_t>(pyr, 256) + 255) / 256 * 256);
    return FT_OK;
}

extern "C" ft_status ttc_server_admit(ttc_server *s, int H, int W, int *stream_id)
{
    FT_API_RANGE;
    if (!s || !stream_id) return FT_ERR_INVALID_ARG;
    if (H > s->max_H || W > s->max_W) return FT_ERR_WORKSPACE;
    int64_t need = 0;
    ft_status st = ttc_server_stream_bytes(s, H, W, &need);
    if (st != FT_OK) return st;
    int open = 0;
    for (const Stream &x : s->streams) open += x.open;
    if (open >= s->max_streams || s->used + need > s->budget) return FT_ERR_WORKSPACE;
    Stream x;
    x.H = H;
    x.W = W;
    x.slot_bytes = (size_t)(((int64_t)H * W * s->es + 255) / 256 * 256);
    int64_t pyr = 0;
    ttc_pyramid_layout(H, W, s->levels, s->dtype, nullptr, nullptr, &pyr);
    x.pyr_bytes = (size_t)((std::max<int64_t>(pyr, 256) + 255) / 256 * 256);
    x.nbytes = (size_t)need;
    cudaError_t e = cudaMalloc(&x.mem, x.nbytes);
    if (e != cudaSuccess) return cuda_fail(e);
    x.open = true;
    s->streams.push_back(std::move(x));
    s->used += need;
    *stream_id = (int)s->streams.size() - 1;
    return FT_OK;
}

extern "C" ft_status ttc_server_remove(ttc_server *s, int id)
{
    if (!s || id < 0 || id >= (int)s->streams.size()) return FT_ERR_INVALID_ARG;
    Stream &st = s->streams[(size_t)id];
    if (!st.open || st.closing) return FT_ERR_INVALID_ARG;
    st.closing = true;
    for (const Frame &f : st.pending) report(s, id, f, FT_SERVED_DROPPED);
    st.pending.clear();
    release(s, id);
    return FT_OK;
}

extern "C" ft_status ttc_server_submit(ttc_server *s, int id, const void *frame, int64_t pitch_bytes, int64_t seq,
                                       double t_arrival)
{
    if (!s || !frame || id < 0 || id >= (int)s->streams.size()) return FT_ERR_INVALID_ARG;
    Stream &st = s->streams[(size_t)id];
    if (!st.open || st.closing) return FT_ERR_INVALID_ARG;
    if (pitch_bytes < (int64_t)st.W * s->es) return FT_ERR_SHAPE;
    st.pending.push_back({frame, pitch_bytes, seq, t_arrival});
    if ((int)st.pending.size() > s->max_pending) {
        report(s, id, st.pending.front(), FT_SERVED_DROPPED);     // the oldest goes
        st.pending.pop_front();
    }
    return FT_OK;
}

extern "C" ft_status ttc_server_step(ttc_server *s, int wait, ttc_served *done, int max_done, int *n_done)
{
    FT_API_RANGE;
    if (!s || !n_done || (max_done > 0 && !done) || max_done < 0) return FT_ERR_INVALID_ARG;
    *n_done = 0;
    ft_status st = collect(s, false);
    if (st == FT_OK && s->ticks.size() < 2) st = launch_tick(s);
    if (st == FT_OK && wait && !s->ticks.empty() && s->reports.empty()) st = collect(s, true);
    if (st != FT_OK) return st;
    int n = 0;
    while (n < max_done && !s->reports.empty()) {
        done[n++] = s->reports.front();
        s->reports.pop_front();
    }
    *n_done = n;
    return FT_OK;
}

extern "C" int ttc_server_in_flight(const ttc_server *s) { return s ? (int)s->ticks.size() : 0; }

extern "C" int64_t ttc_server_ticks(const ttc_server *s) { return s ? s->launched : 0; }

extern "C" int ttc_server_waiting(const ttc_server *s, int id)
{
    if (!s) return 0;
    if (id >= 0) return id < (int)s->streams.size() ? (int)s->streams[(size_t)id].pending.size() : 0;
    int n = (int)s->reports.size();
    for (const Stream &st : s->streams) n += (int)st.pending.size();
    return n;
}

extern "C" int64_t ttc_server_bytes_in_use(const ttc_server *s) { return s ? s->used : 0; }

extern "C" int ttc_server_launches(const ttc_server *s) { return s && s->ctx ? ttc_ctx_last_launch_count(s->ctx) : 0; }

// Load generator (measurement of the runtime, no counterpart in the paper): every listed
// stream always has a frame waiting, taken in turn from its nframes host frames, and the
// server is stepped until `pairs` results have come back.  Each tick therefore carries one
// pair per stream, and the rate is that of the runtime and the device, not of the caller.
extern "C" ft_status ttc_server_drive(ttc_server *s, const int *ids, int nstreams, const void *const *frames,
                                      const int64_t *pitches, int nframes, int64_t pairs, double *seconds,
                                      int64_t *served, double *p50_ms, double *p99_ms)
{
    FT_API_RANGE;
    if (!s || !ids || !frames || !pitches || nstreams < 1 || nframes < 1 || pairs < 1) return FT_ERR_INVALID_ARG;
    for (int i = 0; i < nstreams; ++i)
        if (ids[i] < 0 || ids[i] >= (int)s->streams.size() || !s->streams[(size_t)ids[i]].open)
            return FT_ERR_INVALID_ARG;
    using clk = std::chrono::steady_clock;
    const clk::time_point t0 = clk::now();
    auto now = [&] { return std::chrono::duration<double>(clk::now() - t0).count(); };
    std::vector<int64_t> next((size_t)nstreams, 0);
    std::vector<double> lat;
    lat.reserve((size_t)pairs);
    std::vector<ttc_served> done((size_t)std::max(64, 2 * nstreams));
    int64_t got = 0;
    auto step = [&](int wait) {
        int n = 0;
        const ft_status st = ttc_server_step(s, wait, done.data(), (int)done.size(), &n);
        const double t = now();
        for (int k = 0; k < n; ++k)
            if (done[(size_t)k].status == FT_SERVED_RESULT) {
                lat.push_back(1e3 * (t - done[(size_t)k].t_arrival));
                ++got;
            }
        return st;
    };
    while (got < pairs) {
        for (int i = 0; i < nstreams; ++i) {
            if (ttc_server_waiting(s, ids[i]) > 0) continue;
            const int64_t q = next[(size_t)i]++;
            const ft_status st = ttc_server_submit(s, ids[i], frames[(size_t)i * nframes + (size_t)(q % nframes)],
                                                   pitches[i], q, now());
            if (st != FT_OK) return st;
        }
        // wait only when a tick is already in flight: this step launches a second one first,
        // so the next tick's host work and uploads overlap the kernels of the one waited for
        const ft_status st = step(ttc_server_in_flight(s) >= 1 ? 1 : 0);
        if (st != FT_OK) return st;
    }
    // the ticks still in flight complete (their pairs count) before the call returns, so
    // the server is idle again
    for (;;) {
        bool waiting = false;
        for (int i = 0; i < nstreams; ++i) waiting = waiting || ttc_server_waiting(s, ids[i]) > 0;
        if (!waiting && ttc_server_in_flight(s) == 0) break;
        const ft_status st = step(1);
        if (st != FT_OK) return st;
    }
    if (seconds) *seconds = now();
    if (served) *served = got;
    auto pct = [&](double q) {
        std::vector<double> v(lat);
        const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
        std::nth_element(v.begin(), v.begin() + (std::ptrdiff_t)k, v.end());
        return v[k];
    };
    if (p50_ms) *p50_ms = lat.empty() ? 0.0 : pct(0.5);
    if (p99_ms) *p99_ms = lat.empty() ? 0.0 : pct(0.99);
    return FT_OK;
}

