// xe_stream.cpp -- A7: the streaming serving loop, host runtime around the libxe kernels.
//
// Paper correspondences (Sec. II): packets of each F-engine stream are handled separately until
// after correlation; buffer objects (here: device packet regions and frame slots) connect the
// stages; memory is allocated only at start-up and freed at shutdown; a "Data Ready" event gates the
// device work of a frame and a host callback marks its output full (Sec. II-B).
//
// Data path of one frame k of stream s:
//   submit   the host reads each packet's header (seq -> frame k) and copies runs of packets of one
//            frame straight into region (s, k mod ring_frames) in device memory (H2D from host
//            packets, or D2D from packets already in device memory, on the stream's copy stream);
//            no host-side payload copy.
//   close    when more than reorder_window packets of later frames have arrived on stream s, frame
//            k is closed: an event marks its last copy and it joins the ready queue.
//   admit    the scheduler thread takes up to max_batch ready frames for which frame slots are free
//            (continuous batching: frames that become ready while earlier rounds are on the GPU join
//            the next round as slots free up), and enqueues on one of n_cuda_streams streams:
//            each frame's index (which packet holds each slot; the payloads stay where they
//            landed), ONE batched persistent correlation launch reading the samples of all of them
//            straight from their packet regions, a normalisation per frame, and a host callback.
//            A region is reusable once that correlation has read it.
//   complete the callback timestamps the frames and queues them for xe_stream_poll;
//            xe_stream_release returns the slot. Two latencies per frame: from its close, and from
//            the submission of its last packet (the latter includes the reorder-window wait).
//
// Everything the loop needs after start-up is allocated by xe_stream_create: the ready and done
// queues are fixed rings, the per-round records come from a pool with one record per slot (a round
// holds at least one slot until its frames are released), the scheduler's per-round arrays are
// sized max_batch, and latencies go into fixed log-linear histograms. Submitting, scheduling and
// completing frames allocate no host memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <cmath>
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
    Clock::time_point t_last{};  // submission of the last packet copied in
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
    Clock::time_point t_close, t_last;
};

struct Done {
    int32_t stream, slot;
    int64_t frame;
    uint32_t packets, batch;
    uint64_t latency_ns, latency_submit_ns;
};

// Fixed-capacity FIFO; the storage is allocated once (reset) and never grows.
template <typename T>
struct Ring {
    std::vector<T> buf;
    size_t head = 0, n = 0;
    void reset(size_t cap) { buf.assign(std::max<size_t>(cap, 1), T{}); head = n = 0; }
    bool full() const { return n == buf.size(); }
    bool empty() const { return n == 0; }
    size_t size() const { return n; }
    bool push(const T &v) {
        if (full()) return false;
        buf[(head + n) % buf.size()] = v;
        ++n;
        return true;
    }
    T &front() { return buf[head]; }
    void pop() { head = (head + 1) % buf.size(); --n; }
};

// Log-linear latency histogram (64 sub-buckets per power of two: about 1.6 % resolution).
struct LatencyHist {
    static constexpr int kSub = 64, kBuckets = 59 * kSub;
    uint64_t counts[kBuckets] = {};
    uint64_t total = 0, max = 0;
    static int bucket(uint64_t ns) {
        if (ns < (uint64_t)kSub) return (int)ns;
        const int e = 63 - __builtin_clzll(ns);   // >= 6
        return (e - 5) * kSub + (int)((ns >> (e - 6)) & (kSub - 1));
    }
    static double mid(int b) {
        if (b < kSub) return b;
        const int e = b / kSub + 5, sub = b % kSub;
        const double lo = std::ldexp((double)(kSub + sub), e - 6);
        return lo + std::ldexp(0.5, e - 6);
    }
    void add(uint64_t ns) {
        counts[bucket(ns)]++;
        total++;
        max = std::max(max, ns);
    }
    // value of rank round(q (total - 1)) in sorted order, to the bucket's resolution
    double pct(double q) const {
        if (!total) return 0.0;
        const uint64_t rank = (uint64_t)(q * (double)(total - 1) + 0.5);
        uint64_t cum = 0;
        for (int b = 0; b < kBuckets; ++b) {
            cum += counts[b];
            if (cum > rank) return std::min(mid(b), (double)max);
        }
        return (double)max;
    }
};

struct BatchRec {
    xe_stream *rt = nullptr;
    uint32_t id = 0;
    int n = 0;
    std::vector<Ready> frames;     // sized max_batch at start-up
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
    // scheduler scratch, sized max_batch at start-up (only the scheduler thread touches it)
    std::vector<xe_job> jobs;
    std::vector<xe::packet_src> srcs;
    std::vector<xe::serve::Region *> regs;

    std::mutex mu;                          // everything below
    std::condition_variable cv_sched, cv_done;
    xe::serve::Ring<xe::serve::Ready> ready;
    xe::serve::Ring<int> free_slots;
    xe::serve::Ring<xe::serve::Done> done;
    std::vector<xe::serve::BatchRec> recs;  // one per slot
    xe::serve::Ring<xe::serve::BatchRec *> free_recs;
    std::vector<uint8_t> slot_free;         // 1 while the slot is in free_slots
    xe::serve::LatencyHist lat_close, lat_submit;
    uint64_t packets_submitted = 0, packets_late = 0, frames_closed = 0, frames_done = 0, frames_released = 0;
    uint64_t batches = 0, max_batch_seen = 0;
    int error = XE_OK;
    bool stop = false;
    std::thread sched;
};

namespace xe {
namespace serve {

static inline uint64_t seq_of(const uint8_t *hdr) {
    uint64_t s;
    std::memcpy(&s, hdr + 8, 8);
    return s;
}

// Closes frame k of stream `sid` (caller holds ps.mu and k == ps.next_close). Returns false, having
// changed nothing, when the ready queue is full.
static bool close_frame(xe_stream *rt, int sid, PerStream &ps, int64_t k) {
    const int R = rt->cfg.ring_frames;
    Region &r = ps.regions[k % R];
    const bool has = r.frame == k;
    const auto now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(rt->mu);
        if (!rt->ready.push(Ready{sid, k, now, has ? r.t_last : now})) return false;
        rt->frames_closed++;
    }
    if (has) {
        cudaEventRecord(r.copied, ps.copy);
        r.closed = true;
    }
    ps.next_close = k + 1;
    rt->cv_sched.notify_one();
    return true;
}

// Packets of frames newer than k already in the regions of stream ps.
static uint64_t newer_packets(const PerStream &ps, int64_t k) {
    uint64_t n = 0;
    for (const Region &r : ps.regions)
        if (r.frame > k) n += r.count;
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
        for (int i = 0; i < rec->n; ++i) {
            const Ready &f = rec->frames[i];
            const uint64_t ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(now - f.t_close).count();
            const uint64_t ns_sub =
                (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(now - f.t_last).count();
            rt->done.push(Done{f.stream, rec->slots[i], f.frame, rec->packets[i], rec->id, ns, ns_sub});
            rt->lat_close.add(ns);
            rt->lat_submit.add(ns_sub);
            rt->frames_done++;
        }
        rt->free_recs.push(rec);
    }
    rt->cv_done.notify_all();
}

static void scheduler(xe_stream *rt) {
    cudaSetDevice(rt->device);
    const xe_stream_cfg &c = rt->cfg;
    const xe_shape shape{c.n_inputs, rt->Fs, c.n_time};
    uint32_t batch_id = 0;
    for (;;) {
        BatchRec *rec = nullptr;
        {
            std::unique_lock<std::mutex> lk(rt->mu);
            auto admissible = [&] { return !rt->ready.empty() && !rt->free_slots.empty() && !rt->free_recs.empty(); };
            rt->cv_sched.wait(lk, [&] { return rt->stop || admissible(); });
            if (rt->stop) return;
            if (c.batch_wait_us > 0) {   // gather window: let more frames join this round
                const size_t want = std::min<size_t>((size_t)c.max_batch, rt->free_slots.size());
                rt->cv_sched.wait_for(lk, std::chrono::microseconds(c.batch_wait_us),
                                      [&] { return rt->stop || rt->ready.size() >= want; });
                if (rt->stop) return;
            }
            rec = rt->free_recs.front();
            rt->free_recs.pop();
            const size_t n = std::min({(size_t)c.max_batch, rt->ready.size(), rt->free_slots.size()});
            rec->n = (int)n;
            for (size_t i = 0; i < n; ++i) {
                rec->frames[i] = rt->ready.front();
                rt->ready.pop();
                rec->slots[i] = rt->free_slots.front();
                rt->free_slots.pop();
                rt->slot_free[rec->slots[i]] = 0;
            }
            rt->batches++;
            rt->max_batch_seen = std::max<uint64_t>(rt->max_batch_seen, n);
        }
        const uint32_t bid = batch_id++;
        rec->id = bid;
        cudaStream_t st = rt->cs[bid % rt->cs.size()];
        void *ws = rt->ws_c[bid % rt->cs.size()];
        int err = XE_OK;
        for (int i = 0; i < rec->n; ++i) {
            const Ready &f = rec->frames[i];
            const Slot &sl = rt->slot_mem[rec->slots[i]];
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
            rec->packets[i] = count;
            cudaMemsetAsync(sl.lost, 0, (size_t)rt->Fs * 4, st);
            cudaMemsetAsync(sl.stats, 0, 5 * 4, st);
            int e = index_streams(pk, count, c.pkt_stride, (uint64_t)f.frame * rt->Q, c.groups_per_stream,
                                  (uint32_t)f.stream, shape, sl.filled, sl.lost, sl.stats, sl.owner, st);
            if (e) err = e;
            rt->regs[i] = reg;
            rt->jobs[i] = xe_job{nullptr, sl.vis, shape, 0, 0};
            // a frame whose region was lost has no packets: the index sends every read to zeros
            rt->srcs[i] = packet_src{pk ? pk : reinterpret_cast<const uint8_t *>(sl.owner), sl.owner, c.pkt_stride};
        }
        int e = correlate_packets_batched(rt->jobs.data(), rt->srcs.data(), rec->n, ws, rt->ws_c_bytes, st);
        if (e) err = e;
        for (int i = 0; i < rec->n; ++i) {
            if (!rt->regs[i]) continue;
            PerStream &ps = *rt->streams[rec->frames[i].stream];
            std::lock_guard<std::mutex> lk(ps.mu);
            cudaEventRecord(rt->regs[i]->consumed, st);       // the correlation has read the packets
            rt->regs[i]->issued = true;
        }
        for (int i = 0; i < rec->n; ++i) {
            const Slot &sl = rt->slot_mem[rec->slots[i]];
            e = xe_normalize(sl.vis, shape, (uint32_t)c.n_time, sl.lost, nullptr, nullptr, sl.out, sl.n, st);
            if (e) err = e;
        }
        if (cudaLaunchHostFunc(st, on_batch_done, rec) != cudaSuccess) {
            err = XE_ECUDA;
            std::lock_guard<std::mutex> lk(rt->mu);
            rt->free_recs.push(rec);
        }
        if (err) {
            std::lock_guard<std::mutex> lk(rt->mu);
            rt->error = err;
        }
    }
}

// Packets of one submission: their headers are read on the host, their records copied from host
// (H2D) or device (D2D) memory.
struct Source {
    const uint8_t *recs;      // n records of pkt_stride bytes
    const uint8_t *hdrs;      // host, header i at hdrs + i * hdr_stride
    size_t hdr_stride;
    cudaMemcpyKind kind;
};

static int submit(xe_stream *rt, int32_t sid, const Source &src, uint32_t n) {
    const xe_stream_cfg &c = rt->cfg;
    const int R = c.ring_frames;
    PerStream &ps = *rt->streams[sid];
    auto frame_of = [&](uint32_t i) { return (int64_t)(seq_of(src.hdrs + (size_t)i * src.hdr_stride) / (uint64_t)rt->Q); };
    std::lock_guard<std::mutex> lk(ps.mu);
    // pass 1: every packet's region must be usable, else nothing is consumed
    bool again = false;
    for (uint32_t i = 0; i < n; ++i) {
        const int64_t k = frame_of(i);
        if (k < ps.next_close) continue;
        // a frame R or more behind k cannot stay open: its region is needed
        while (ps.next_close <= k - R)
            if (!close_frame(rt, sid, ps, ps.next_close)) return XE_EAGAIN;   // ready queue full
        Region &r = ps.regions[k % R];
        if (r.frame == k || r.frame < 0) continue;
        if (r.frame < k && r.closed && r.issued && cudaEventQuery(r.consumed) == cudaSuccess) continue;
        again = true;
    }
    if (again) return XE_EAGAIN;
    // pass 2: copy runs of packets of one frame into that frame's region
    uint64_t late = 0;
    const auto now = Clock::now();
    for (uint32_t i = 0; i < n;) {
        const int64_t k = frame_of(i);
        uint32_t j = i + 1;
        while (j < n && frame_of(j) == k) ++j;
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
            XE_TRY_CUDA(cudaMemcpyAsync(r.dev + (size_t)r.count * c.pkt_stride, src.recs + (size_t)i * c.pkt_stride,
                                        (size_t)take * c.pkt_stride, src.kind, ps.copy));
            r.count += take;
            r.t_last = now;
        }
        late += (j - i) - take;
        ps.max_frame = std::max(ps.max_frame, k);
        i = j;
    }
    // close every frame that more than reorder_window packets of later frames have overtaken (a full
    // ready queue leaves it open until a later submission or flush)
    while (ps.next_close <= ps.max_frame && newer_packets(ps, ps.next_close) > (uint64_t)c.reorder_window)
        if (!close_frame(rt, sid, ps, ps.next_close)) break;
    std::lock_guard<std::mutex> g(rt->mu);
    rt->packets_submitted += n;
    rt->packets_late += late;
    return rt->error;
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
    // host-side state of the loop, all sized here: queues, round records, scheduler scratch
    rt->ready.reset((size_t)c.n_streams * (4 * (size_t)c.ring_frames + 4) + (size_t)slots);
    rt->free_slots.reset((size_t)slots);
    rt->done.reset((size_t)slots);
    rt->slot_free.assign((size_t)slots, 1);
    rt->recs.resize((size_t)slots);
    rt->free_recs.reset((size_t)slots);
    for (BatchRec &r : rt->recs) {
        r.rt = rt.get();
        r.frames.resize((size_t)c.max_batch);
        r.slots.resize((size_t)c.max_batch);
        r.packets.resize((size_t)c.max_batch);
        rt->free_recs.push(&r);
    }
    rt->jobs.resize((size_t)c.max_batch);
    rt->srcs.resize((size_t)c.max_batch);
    rt->regs.resize((size_t)c.max_batch);
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
        rt->free_slots.push(slots - 1 - i);
    }
    rt->sched = std::thread(scheduler, rt.get());
    *out = rt.release();
    return XE_OK;
}

int xe_stream_submit(xe_stream *rt, int32_t sid, const void *host_pkts, uint32_t n) {
    if (!rt || sid < 0 || sid >= rt->cfg.n_streams || (n && !host_pkts)) return XE_EINVAL;
    if (n == 0) return XE_OK;
    const uint8_t *h = static_cast<const uint8_t *>(host_pkts);
    return submit(rt, sid, Source{h, h, rt->cfg.pkt_stride, cudaMemcpyHostToDevice}, n);
}

int xe_stream_submit_device(xe_stream *rt, int32_t sid, const void *dev_pkts, const void *host_headers,
                            uint32_t n) {
    if (!rt || sid < 0 || sid >= rt->cfg.n_streams || (n && (!dev_pkts || !host_headers))) return XE_EINVAL;
    if (n == 0) return XE_OK;
    return submit(rt, sid,
                  Source{static_cast<const uint8_t *>(dev_pkts), static_cast<const uint8_t *>(host_headers), 16,
                         cudaMemcpyDeviceToDevice},
                  n);
}

int xe_stream_flush(xe_stream *rt) {
    if (!rt) return XE_EINVAL;
    int status = XE_OK;
    for (int s = 0; s < rt->cfg.n_streams; ++s) {
        PerStream &ps = *rt->streams[s];
        std::lock_guard<std::mutex> lk(ps.mu);
        while (ps.next_close <= ps.max_frame)
            if (!close_frame(rt, s, ps, ps.next_close)) {
                status = XE_EAGAIN;
                break;
            }
    }
    return status;
}

int xe_stream_poll(xe_stream *rt, xe_result *out, int32_t timeout_ms) {
    if (!rt || !out) return XE_EINVAL;
    std::unique_lock<std::mutex> lk(rt->mu);
    if (!rt->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)), [&] { return !rt->done.empty(); }))
        return rt->error ? rt->error : XE_ETIMEOUT;
    const Done d = rt->done.front();
    rt->done.pop();
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
    out->latency_submit_ns = d.latency_submit_ns;
    return XE_OK;
}

int xe_stream_release(xe_stream *rt, const xe_result *r) {
    if (!rt || !r || r->slot < 0 || r->slot >= (int)rt->slot_mem.size()) return XE_EINVAL;
    {
        std::lock_guard<std::mutex> lk(rt->mu);
        if (rt->slot_free[r->slot]) return XE_EINVAL;
        rt->slot_free[r->slot] = 1;
        rt->free_slots.push(r->slot);
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
    o->latency_p50_us = rt->lat_close.pct(0.50) / 1e3;
    o->latency_p99_us = rt->lat_close.pct(0.99) / 1e3;
    o->latency_max_us = rt->lat_close.max / 1e3;
    o->latency_submit_p50_us = rt->lat_submit.pct(0.50) / 1e3;
    o->latency_submit_p99_us = rt->lat_submit.pct(0.99) / 1e3;
    o->latency_submit_max_us = rt->lat_submit.max / 1e3;
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
