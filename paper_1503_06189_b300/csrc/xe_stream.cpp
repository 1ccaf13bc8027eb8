// xe_stream.cpp -- A7: the streaming serving loop, host runtime around the libxe kernels.
//
// Paper correspondences (Sec. II): packets of each F-engine stream are handled separately until
// after correlation; buffer objects (here: device packet regions and frame slots) connect the
// stages; memory is allocated only at start-up and freed at shutdown; a "Data Ready" event gates the
// device work of a frame and a host callback marks its output full (Sec. II-B).
//
// Data path of one frame k of stream s:
//   submit   the host reads each packet's header (seq -> frame k) and copies runs of packets of one
//            frame straight into region (s, k mod ring_frames) in device memory (H2D on the stream's
//            copy stream); no host-side payload copy.
//   close    when more than reorder_window packets of later frames have arrived on stream s, frame
//            k is closed: an event marks its last H2D copy and it joins the ready queue.
//   admit    the scheduler thread takes up to max_batch ready frames for which frame slots are free
//            (continuous batching: frames that become ready while earlier rounds are on the GPU join
//            the next round as slots free up), and enqueues on one of n_cuda_streams streams:
//            each frame's index (which packet holds each slot; the payloads stay where they
//            landed), ONE batched persistent correlation launch reading the samples of all of them
//            straight from their packet regions, a normalisation per frame, and a host callback.
//            A region is reusable once that correlation has read it.
//   complete the callback timestamps the frames (latency = close -> complete) and queues them for
//            xe_stream_poll; xe_stream_release returns the slot.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "xe_internal.h"

namespace xe {
namespace serve {

using Clock = std::chrono::steady_clock;

struct Region {                  // device packet region of one frame of one stream
    uint8_t *dev = nullptr;
    int64_t frame = -1;          // frame using the region, -1 = never used
    uint32_t count = 0;          // packets copied in
    bool closed = false;
    bool issued = false;         // correlation enqueued; `consumed` marks when it has read the packets
    cudaEvent_t copied = nullptr;
    cudaEvent_t consumed = nullptr;
};

struct PerStream {
    std::mutex mu;
    std::vector<Region> regions;
    int64_t next_close = 0;      // oldest frame not yet closed
    int64_t max_frame = -1;      // newest frame seen
    cudaStream_t copy = nullptr;
};

struct Slot {
    uint8_t *filled;
    uint32_t *lost, *stats, *n, *owner;   // owner: the frame's index, [F_s / 8][T / 4]
    int32_t *vis;
    float *out;
};

struct Ready {
    int32_t stream;
    int64_t frame;
    Clock::time_point t_close;
};

struct Done {
    int32_t stream, slot;
    int64_t frame;
    uint32_t packets, batch;
    uint64_t latency_ns;
};

struct BatchRec {
    xe_stream *rt;
    uint32_t id;
    std::vector<Ready> frames;
    std::vector<int> slots;
    std::vector<uint32_t> packets;
};

}  // namespace serve
}  // namespace xe

struct xe_stream {
    xe_stream_cfg cfg{};
    int device = 0;
    int Q = 0, Fs = 0;
    int64_t P = 0;
    uint32_t cap = 0;                       // packets per region
    size_t ws_c_bytes = 0, total_bytes = 0;
    void *pool = nullptr;
    std::vector<std::unique_ptr<xe::serve::PerStream>> streams;
    std::vector<xe::serve::Slot> slot_mem;
    std::vector<cudaStream_t> cs;
    std::vector<void *> ws_c;

    std::mutex mu;                          // everything below
    std::condition_variable cv_sched, cv_done;
    std::deque<xe::serve::Ready> ready;
    std::vector<int> free_slots;
    std::deque<xe::serve::Done> done;
    std::vector<uint64_t> latencies;
    uint64_t packets_submitted = 0, packets_late = 0, frames_closed = 0, frames_done = 0, frames_released = 0;
    uint64_t batches = 0, max_batch_seen = 0;
    int error = XE_OK;
    bool stop = false;
    std::thread sched;
};

namespace xe {
namespace serve {

static inline uint64_t seq_of(const uint8_t *rec) {
    uint64_t s;
    std::memcpy(&s, rec + 8, 8);
    return s;
}

// Closes frame k of stream `sid` (caller holds ps.mu and k == ps.next_close).
static void close_frame(xe_stream *rt, int sid, PerStream &ps, int64_t k) {
    const int R = rt->cfg.ring_frames;
    Region &r = ps.regions[k % R];
    if (r.frame == k) {
        cudaEventRecord(r.copied, ps.copy);
        r.closed = true;
    }
    ps.next_close = k + 1;
    {
        std::lock_guard<std::mutex> lk(rt->mu);
        rt->ready.push_back(Ready{sid, k, Clock::now()});
        rt->frames_closed++;
    }
    rt->cv_sched.notify_one();
}

// Packets of frames newer than k already in the regions of stream ps.
static uint64_t newer_packets(const xe_stream *rt, const PerStream &ps, int64_t k) {
    uint64_t n = 0;
    for (const Region &r : ps.regions)
        if (r.frame > k) n += r.count;
    (void)rt;
    return n;
}

// Releases the device resources xe_stream_create acquired; any of them may be missing (a create
// that failed part-way). Used on create's failure paths and by xe_stream_destroy.
static void free_runtime(xe_stream *rt) {
    for (cudaStream_t st : rt->cs) cudaStreamDestroy(st);
    for (auto &ps : rt->streams) {
        if (ps->copy) cudaStreamDestroy(ps->copy);
        for (Region &r : ps->regions) {
            if (r.copied) cudaEventDestroy(r.copied);
            if (r.consumed) cudaEventDestroy(r.consumed);
        }
    }
    if (rt->pool) cudaFree(rt->pool);
    rt->cs.clear();
    rt->ws_c.clear();
    rt->streams.clear();
    rt->pool = nullptr;
}

static void on_batch_done(void *p) {
    BatchRec *rec = static_cast<BatchRec *>(p);
    xe_stream *rt = rec->rt;
    const auto now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(rt->mu);
        for (size_t i = 0; i < rec->frames.size(); ++i) {
            const uint64_t ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(now - rec->frames[i].t_close).count();
            rt->done.push_back(Done{rec->frames[i].stream, rec->slots[i], rec->frames[i].frame, rec->packets[i], rec->id, ns});
            rt->latencies.push_back(ns);
            rt->frames_done++;
        }
    }
    rt->cv_done.notify_all();
    delete rec;
}

static void scheduler(xe_stream *rt) {
    cudaSetDevice(rt->device);
    const xe_stream_cfg &c = rt->cfg;
    const xe_shape shape{c.n_inputs, rt->Fs, c.n_time};
    uint32_t batch_id = 0;
    for (;;) {
        std::vector<Ready> frames;
        std::vector<int> slots;
        {
            std::unique_lock<std::mutex> lk(rt->mu);
            rt->cv_sched.wait(lk, [&] { return rt->stop || (!rt->ready.empty() && !rt->free_slots.empty()); });
            if (rt->stop) return;
            if (c.batch_wait_us > 0) {   // gather window: let more frames join this round
                const size_t want = std::min<size_t>((size_t)c.max_batch, rt->free_slots.size());
                rt->cv_sched.wait_for(lk, std::chrono::microseconds(c.batch_wait_us),
                                      [&] { return rt->stop || rt->ready.size() >= want; });
                if (rt->stop) return;
            }
            const size_t n = std::min({(size_t)c.max_batch, rt->ready.size(), rt->free_slots.size()});
            for (size_t i = 0; i < n; ++i) {
                frames.push_back(rt->ready.front());
                rt->ready.pop_front();
                slots.push_back(rt->free_slots.back());
                rt->free_slots.pop_back();
            }
            rt->batches++;
            rt->max_batch_seen = std::max<uint64_t>(rt->max_batch_seen, n);
        }
        const uint32_t bid = batch_id++;
        cudaStream_t st = rt->cs[bid % rt->cs.size()];
        void *ws = rt->ws_c[bid % rt->cs.size()];
        BatchRec *rec = new BatchRec{rt, bid, frames, slots, {}};
        std::vector<xe_job> jobs;
        std::vector<packet_src> srcs;
        std::vector<Region *> regs;
        int err = XE_OK;
        for (size_t i = 0; i < frames.size(); ++i) {
            const Ready &f = frames[i];
            const Slot &sl = rt->slot_mem[slots[i]];
            PerStream &ps = *rt->streams[f.stream];
            const uint8_t *pk = nullptr;
            uint32_t count = 0;
            Region *reg = nullptr;
            {
                std::lock_guard<std::mutex> lk(ps.mu);
                Region &r = ps.regions[f.frame % c.ring_frames];
                if (r.frame == f.frame) {
                    reg = &r;
                    pk = r.dev;
                    count = r.count;
                    cudaStreamWaitEvent(st, r.copied, 0);      // the frame's "Data Ready"
                }
            }
            rec->packets.push_back(count);
            cudaMemsetAsync(sl.lost, 0, (size_t)rt->Fs * 4, st);
            cudaMemsetAsync(sl.stats, 0, 5 * 4, st);
            int e = index_streams(pk, count, c.pkt_stride, (uint64_t)f.frame * rt->Q, c.groups_per_stream,
                                  (uint32_t)f.stream, shape, sl.filled, sl.lost, sl.stats, sl.owner, st);
            if (e) err = e;
            regs.push_back(reg);
            jobs.push_back(xe_job{nullptr, sl.vis, shape, 0, 0});
            // a frame whose region was lost has no packets: the index sends every read to zeros
            srcs.push_back(packet_src{pk ? pk : reinterpret_cast<const uint8_t *>(sl.owner), sl.owner, c.pkt_stride});
        }
        int e = correlate_packets_batched(jobs.data(), srcs.data(), (int)jobs.size(), ws, rt->ws_c_bytes, st);
        if (e) err = e;
        for (size_t i = 0; i < frames.size(); ++i) {
            if (!regs[i]) continue;
            PerStream &ps = *rt->streams[frames[i].stream];
            std::lock_guard<std::mutex> lk(ps.mu);
            cudaEventRecord(regs[i]->consumed, st);           // the correlation has read the packets
            regs[i]->issued = true;
        }
        for (size_t i = 0; i < frames.size(); ++i) {
            const Slot &sl = rt->slot_mem[slots[i]];
            e = xe_normalize(sl.vis, shape, (uint32_t)c.n_time, sl.lost, nullptr, nullptr, sl.out, sl.n, st);
            if (e) err = e;
        }
        if (cudaLaunchHostFunc(st, on_batch_done, rec) != cudaSuccess) {
            err = XE_ECUDA;
            delete rec;
        }
        if (err) {
            std::lock_guard<std::mutex> lk(rt->mu);
            rt->error = err;
        }
    }
}

}  // namespace serve
}  // namespace xe

using namespace xe;
using namespace xe::serve;

extern "C" {

int xe_stream_create(const xe_stream_cfg *cfg, xe_stream **out) {
    if (!cfg || !out) return XE_EINVAL;
    const xe_stream_cfg c = *cfg;
    if (c.n_streams < 1 || c.groups_per_stream < 1 || c.n_inputs < 16 || c.n_inputs % 16 || c.n_time < 4 ||
        c.n_time % 4 || c.n_time > XE_MAX_TIME || c.reorder_window < 1 || c.ring_frames < 2 || c.max_batch < 1 ||
        c.max_batch > XE_MAX_JOBS || c.n_cuda_streams < 1 || c.slots < 0 || c.batch_wait_us < 0 || c.pkt_stride % 16 ||
        c.pkt_stride < 16u + 32u * (uint32_t)c.n_inputs)
        return XE_EINVAL;
    auto rt = std::make_unique<xe_stream>();
    rt->cfg = c;
    XE_TRY_CUDA(cudaGetDevice(&rt->device));
    rt->Q = c.n_time / 4;
    rt->Fs = 8 * c.groups_per_stream;
    rt->P = npairs(c.n_inputs);
    const uint64_t pkts_per_frame = (uint64_t)rt->Q * c.groups_per_stream;
    rt->cap = (uint32_t)(pkts_per_frame + pkts_per_frame / 4 + 64);   // room for duplicates
    const xe_shape shape{c.n_inputs, rt->Fs, c.n_time};
    const size_t owner_bytes = (size_t)rt->Q * (rt->Fs / 8) * 4;
    xe_job probe{nullptr, nullptr, shape, 0, 0};
    rt->ws_c_bytes = round_up(xe_correlate_batched_workspace_size(&probe, 1, nullptr), 1024);
    if (!rt->ws_c_bytes) return XE_EINVAL;

    auto al = [](size_t b) { return (size_t)round_up((int64_t)b, 1024); };
    const size_t region_bytes = al((size_t)rt->cap * c.pkt_stride);
    const size_t slot_bytes = al((size_t)rt->Q * (rt->Fs / 8)) + al((size_t)rt->Fs * 4) + al(32) +
                              2 * al((size_t)rt->Fs * rt->P * 8) + al((size_t)rt->Fs * rt->P * 4) + al(owner_bytes);
    const size_t fixed = (size_t)c.n_streams * c.ring_frames * region_bytes + (size_t)c.n_cuda_streams * al(rt->ws_c_bytes);
    int slots = c.slots;
    if (slots == 0) {
        if (c.hbm_budget == 0) slots = 2 * c.max_batch;
        else if (c.hbm_budget > fixed) slots = (int)std::min<uint64_t>((c.hbm_budget - fixed) / slot_bytes, 4096);
    }
    if (slots < 1) return XE_ENOMEM;
    rt->total_bytes = fixed + (size_t)slots * slot_bytes;
    if (c.hbm_budget && rt->total_bytes > c.hbm_budget) return XE_ENOMEM;
    if (cudaMalloc(&rt->pool, rt->total_bytes) != cudaSuccess) {
        cudaGetLastError();
        return XE_ENOMEM;
    }
    uint8_t *p = static_cast<uint8_t *>(rt->pool);
    auto take = [&](size_t b) { uint8_t *q = p; p += al(b); return q; };
    // events and streams; each is registered in rt before it is created, so that a failure part-way
    // releases everything created so far
    auto create_handles = [&]() -> int {
        for (int s = 0; s < c.n_streams; ++s) {
            rt->streams.push_back(std::make_unique<PerStream>());
            PerStream &ps = *rt->streams.back();
            ps.regions.resize(c.ring_frames);
            for (Region &r : ps.regions) {
                r.dev = take((size_t)rt->cap * c.pkt_stride);
                XE_TRY_CUDA(cudaEventCreateWithFlags(&r.copied, cudaEventDisableTiming));
                XE_TRY_CUDA(cudaEventCreateWithFlags(&r.consumed, cudaEventDisableTiming));
            }
            XE_TRY_CUDA(cudaStreamCreateWithFlags(&ps.copy, cudaStreamNonBlocking));
        }
        for (int i = 0; i < c.n_cuda_streams; ++i) {
            cudaStream_t st;
            XE_TRY_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            rt->cs.push_back(st);
            rt->ws_c.push_back(take(rt->ws_c_bytes));
        }
        return XE_OK;
    };
    if (int e = create_handles()) {
        free_runtime(rt.get());
        return e;
    }
    for (int i = 0; i < slots; ++i) {
        Slot sl;
        sl.filled = take((size_t)rt->Q * (rt->Fs / 8));
        sl.lost = reinterpret_cast<uint32_t *>(take((size_t)rt->Fs * 4));
        sl.stats = reinterpret_cast<uint32_t *>(take(32));
        sl.vis = reinterpret_cast<int32_t *>(take((size_t)rt->Fs * rt->P * 8));
        sl.out = reinterpret_cast<float *>(take((size_t)rt->Fs * rt->P * 8));
        sl.n = reinterpret_cast<uint32_t *>(take((size_t)rt->Fs * rt->P * 4));
        sl.owner = reinterpret_cast<uint32_t *>(take(owner_bytes));
        rt->slot_mem.push_back(sl);
        rt->free_slots.push_back(slots - 1 - i);
    }
    rt->sched = std::thread(scheduler, rt.get());
    *out = rt.release();
    return XE_OK;
}

int xe_stream_submit(xe_stream *rt, int32_t sid, const void *host_pkts, uint32_t n) {
    if (!rt || sid < 0 || sid >= rt->cfg.n_streams || (n && !host_pkts)) return XE_EINVAL;
    if (n == 0) return XE_OK;
    const xe_stream_cfg &c = rt->cfg;
    const int R = c.ring_frames;
    const uint8_t *h = static_cast<const uint8_t *>(host_pkts);
    PerStream &ps = *rt->streams[sid];
    std::lock_guard<std::mutex> lk(ps.mu);
    // pass 1: every packet's region must be usable, else nothing is consumed
    bool again = false;
    for (uint32_t i = 0; i < n; ++i) {
        const int64_t k = (int64_t)(seq_of(h + (size_t)i * c.pkt_stride) / (uint64_t)rt->Q);
        if (k < ps.next_close) continue;
        // a frame R or more behind k cannot stay open: its region is needed
        while (ps.next_close <= k - R) close_frame(rt, sid, ps, ps.next_close);
        Region &r = ps.regions[k % R];
        if (r.frame == k || r.frame < 0) continue;
        if (r.frame < k && r.closed && r.issued && cudaEventQuery(r.consumed) == cudaSuccess) continue;
        again = true;
    }
    if (again) return XE_EAGAIN;
    // pass 2: copy runs of packets of one frame into that frame's region
    uint64_t late = 0;
    for (uint32_t i = 0; i < n;) {
        const int64_t k = (int64_t)(seq_of(h + (size_t)i * c.pkt_stride) / (uint64_t)rt->Q);
        uint32_t j = i + 1;
        while (j < n && (int64_t)(seq_of(h + (size_t)j * c.pkt_stride) / (uint64_t)rt->Q) == k) ++j;
        if (k < ps.next_close) {
            late += j - i;
            i = j;
            continue;
        }
        Region &r = ps.regions[k % R];
        if (r.frame != k) {
            r.frame = k;
            r.count = 0;
            r.closed = false;
            r.issued = false;
        }
        const uint32_t take = std::min<uint32_t>(j - i, rt->cap - r.count);
        if (take) {
            XE_TRY_CUDA(cudaMemcpyAsync(r.dev + (size_t)r.count * c.pkt_stride, h + (size_t)i * c.pkt_stride,
                                        (size_t)take * c.pkt_stride, cudaMemcpyHostToDevice, ps.copy));
            r.count += take;
        }
        late += (j - i) - take;
        ps.max_frame = std::max(ps.max_frame, k);
        i = j;
    }
    // close every frame that more than reorder_window packets of later frames have overtaken
    while (ps.next_close <= ps.max_frame && newer_packets(rt, ps, ps.next_close) > (uint64_t)c.reorder_window)
        close_frame(rt, sid, ps, ps.next_close);
    std::lock_guard<std::mutex> g(rt->mu);
    rt->packets_submitted += n;
    rt->packets_late += late;
    return rt->error;
}

int xe_stream_flush(xe_stream *rt) {
    if (!rt) return XE_EINVAL;
    for (int s = 0; s < rt->cfg.n_streams; ++s) {
        PerStream &ps = *rt->streams[s];
        std::lock_guard<std::mutex> lk(ps.mu);
        while (ps.next_close <= ps.max_frame) close_frame(rt, s, ps, ps.next_close);
    }
    return XE_OK;
}

int xe_stream_poll(xe_stream *rt, xe_result *out, int32_t timeout_ms) {
    if (!rt || !out) return XE_EINVAL;
    std::unique_lock<std::mutex> lk(rt->mu);
    if (!rt->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)), [&] { return !rt->done.empty(); }))
        return rt->error ? rt->error : XE_ETIMEOUT;
    const Done d = rt->done.front();
    rt->done.pop_front();
    const Slot &sl = rt->slot_mem[d.slot];
    out->stream_id = d.stream;
    out->slot = d.slot;
    out->frame = d.frame;
    out->out = sl.out;
    out->vis = sl.vis;
    out->n = sl.n;
    out->lost = sl.lost;
    out->stats = sl.stats;
    out->packets = d.packets;
    out->batch = d.batch;
    out->latency_ns = d.latency_ns;
    return XE_OK;
}

int xe_stream_release(xe_stream *rt, const xe_result *r) {
    if (!rt || !r || r->slot < 0 || r->slot >= (int)rt->slot_mem.size()) return XE_EINVAL;
    {
        std::lock_guard<std::mutex> lk(rt->mu);
        if (std::find(rt->free_slots.begin(), rt->free_slots.end(), r->slot) != rt->free_slots.end()) return XE_EINVAL;
        rt->free_slots.push_back(r->slot);
        rt->frames_released++;
    }
    rt->cv_sched.notify_one();
    return XE_OK;
}

int xe_stream_stats(xe_stream *rt, xe_stream_stats_t *o) {
    if (!rt || !o) return XE_EINVAL;
    std::lock_guard<std::mutex> lk(rt->mu);
    std::memset(o, 0, sizeof(*o));
    o->packets_submitted = rt->packets_submitted;
    o->packets_late = rt->packets_late;
    o->frames_closed = rt->frames_closed;
    o->frames_done = rt->frames_done;
    o->frames_released = rt->frames_released;
    o->batches = rt->batches;
    o->max_batch_seen = rt->max_batch_seen;
    o->device_bytes = rt->total_bytes;
    o->slots = (int32_t)rt->slot_mem.size();
    if (!rt->latencies.empty()) {
        std::vector<uint64_t> v = rt->latencies;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))] / 1e3; };
        o->latency_p50_us = pct(0.50);
        o->latency_p99_us = pct(0.99);
        o->latency_max_us = v.back() / 1e3;
    }
    return rt->error;
}

int xe_stream_destroy(xe_stream *rt) {
    if (!rt) return XE_EINVAL;
    {
        std::lock_guard<std::mutex> lk(rt->mu);
        rt->stop = true;
    }
    rt->cv_sched.notify_all();
    if (rt->sched.joinable()) rt->sched.join();
    int status = XE_OK;
    // every kernel has bounded waits, so the queues drain; poll them with an overall limit
    const auto t0 = Clock::now();
    std::vector<cudaStream_t> all = rt->cs;
    for (auto &ps : rt->streams) all.push_back(ps->copy);
    for (cudaStream_t st : all) {
        while (cudaStreamQuery(st) == cudaErrorNotReady) {
            if (Clock::now() - t0 > std::chrono::seconds(30)) { status = XE_ETIMEOUT; break; }
            std::this_thread::sleep_for(std::chrono::microseconds(200));
        }
    }
    if (status == XE_OK) {
        free_runtime(rt);
        delete rt;
    }
    return status;
}

}  // extern "C"
