/*
 * xe.h -- C ABI of libxe, a B300 (sm_103a) X-engine for 4+4-bit complex radio-correlator data.
 *
 * The operations follow Recnik et al., "An Efficient Real-time Data Pipeline for the CHIME
 * Pathfinder Radio Telescope X-Engine": packet-to-frame assembly (Sec. II-A), cross-correlation
 * and integration of all input pairs per frequency channel (Sec. I, Sec. II-B), and the
 * normalisation of the integrated matrix by per-visibility sample counts (Sec. II-C).
 *
 * Conventions shared by every call
 *   - Samples are one byte: high nibble = real, low nibble = imaginary, 4-bit two's complement
 *     in [-8, 7]. A frame is uint8 [T][F][N] (time, channel, input), N a multiple of 16.
 *   - Visibilities V_f[i,j] = sum_t x_i(t) conj(x_j(t)) for i <= j are stored as int32 [F][P][2]
 *     with P = N(N+1)/2, packed row-major upper triangle including the diagonal, {re, im}.
 *     Position of (i, j): p = i*N - i*(i-1)/2 + (j - i).
 *   - Every pointer argument is a DEVICE pointer owned by the caller unless stated otherwise; the
 *     library allocates no device memory on any of these calls. Scratch space ("workspace") is
 *     sized by the matching *_workspace_size() call and passed in by the caller.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls only enqueue work on
 *     it and return; they never synchronise, except where stated.
 *   - Every call returns a status: XE_OK or a negative XE_E* code; on error nothing is enqueued.
 *     Device-side bounded waits that expire record XE_ETIMEOUT in a device status word read by
 *     xe_device_status().
 */
#ifndef XE_H
#define XE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XE_OK 0
#define XE_EINVAL (-1)      /* bad shape, pointer, alignment or argument */
#define XE_EOVERFLOW (-2)   /* T (or an integration length) beyond the int32 bound 2^24 - 1 */
#define XE_ENOMEM (-3)      /* workspace too small, or over the configured device-memory budget */
#define XE_ECUDA (-4)       /* a CUDA runtime/driver call failed; see xe_last_cuda_error() */
#define XE_ETIMEOUT (-5)    /* a bounded device or host wait expired */
#define XE_EAGAIN (-6)      /* no free slot right now (admission); retry later */

/* Largest time-sample count whose int32 sums cannot overflow: |re V| <= 128 per sample, so
 * 128 * (2^24 - 1) = 2^31 - 128 is the largest reachable value. */
#define XE_MAX_TIME 16777215
/* Largest input count N of a correlation (N is a multiple of 16 from 16 up). */
#define XE_MAX_INPUTS 4096

typedef struct {
    int32_t n_inputs;   /* N: inputs (antenna feeds x polarisations), multiple of 16 */
    int32_t n_chan;     /* F: frequency channels */
    int32_t n_time;     /* T: time samples */
} xe_shape;

/* ---------------------------------------------------------------- library */

/* Human-readable text of a status code. Never NULL. */
const char *xe_strerror(int status);
/* cudaError_t of the last failing CUDA call in this thread (0 if none). */
int xe_last_cuda_error(void);
/* ABI version: major * 10000 + minor * 100 + patch. */
int xe_version(void);
/* Reads and clears the device status word on the current device (XE_OK or XE_ETIMEOUT).
 * Synchronises `stream`. */
int xe_device_status(int *status_out, void *stream);
/* Failure-detection self test: enqueues one kernel that waits on a flag nothing ever sets, with
 * a limit of `timeout_ns` nanoseconds, then records XE_ETIMEOUT in the device status word and
 * returns. The context stays usable. */
int xe_selftest_timeout(uint64_t timeout_ns, void *stream);

/* ---------------------------------------------------------------- A1: assembly (Sec. II-A) */

/*
 * Frame assembly from UDP packets (Sec. II-A.2): each packet's data section is placed at the slot
 * its sequence number gives, lost packets leave zeros, out-of-order packets land by sequence
 * number, duplicates are ignored. Channel groups of all streams are placed at their global
 * channel index, which combines the streams of a server (Sec. II, Sec. II-C).
 *
 *   pkts        device, n_pkts records of pkt_stride bytes, in arrival order. Record layout:
 *               16-byte little-endian header {u16 stream_id; u16 chan_group; u32 reserved;
 *               u64 seq} then the payload [4 t][8 f][N n] bytes. pkt_stride % 16 == 0 and
 *               pkt_stride >= 16 + 32 N.
 *   seq0        sequence number of the frame's first slot; the frame covers slots seq0 ..
 *               seq0 + T/4 - 1 (seq counts packets = 4 time samples).
 *   groups_per_stream  channel groups (8 channels each) per stream; the global group of a packet
 *               is stream_id * groups_per_stream + chan_group, channels [8G, 8G + 8).
 *   s           frame shape; T % 4 == 0, F % 8 == 0, (F/8) % groups_per_stream == 0.
 *   frame       out, uint8 [T][F][N]; every byte is written (payload or zero).
 *   filled      out, uint8 [T/4][F/8]; 1 where the slot's packet arrived.
 *   lost        in/out, uint32 [F]; += 4 for every missing packet of the channel's group
 *               (lost samples per channel, summed over an integration by the caller).
 *   stats       in/out, uint32 [5]; += {ok, duplicate, late (seq < seq0), early (seq >= end),
 *               invalid (stream or group outside the frame)}.
 *   ws          workspace of xe_assemble_workspace_size(s) bytes (any contents).
 * The first arrival of a slot wins; results do not depend on thread timing.
 */
size_t xe_assemble_workspace_size(xe_shape s);
int xe_assemble(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0,
                int32_t groups_per_stream, xe_shape s, uint8_t *frame, uint8_t *filled,
                uint32_t *lost, uint32_t *stats, void *ws, size_t ws_bytes, void *stream);

/*
 * Allocation-free variant of xe_assemble. The paper has no counterpart to this call: it exists for
 * callers that cannot allocate device memory where they assemble frames -- real-time receive loops
 * that must not block (cudaMalloc can synchronise the device and stall for milliseconds), or
 * plug-ins whose host application owns every device allocation and hands out no scratch space.
 *
 * Arguments and results are those of xe_assemble, without the workspace: the owner table lives in
 * a static array inside libxe of XE_ASSEMBLE_NOALLOC_MAX_SLOTS entries (1 MiB per device that loads
 * the library, held until the process exits). A frame may use at most that many (slot, group)
 * pairs, (T/4) * (F/8) <= XE_ASSEMBLE_NOALLOC_MAX_SLOTS; larger frames return XE_ENOMEM.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current); so does the first call after the device's context has been reset, since the
 * array then lives at a new address. Make that first call before any stream capture; a call with
 * n_pkts = 0 on a small shape serves. The call allocates nothing. All calls share the one array
 * and each call resets the part it uses, so calls whose kernels may overlap on the GPU (for
 * example on different streams) race and must be serialised by the caller.
 */
#define XE_ASSEMBLE_NOALLOC_MAX_SLOTS (1 << 18)
int xe_assemble_noalloc(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0,
                        int32_t groups_per_stream, xe_shape s, uint8_t *frame, uint8_t *filled,
                        uint32_t *lost, uint32_t *stats, void *stream);

/* ---------------------------------------------------------------- A2: unpack */

/*
 * Unpack a frame into the tensor-core operand of the correlation (Sec. II-B: the packed 4-bit
 * data cross the host link unpromoted; the promotion happens here, on the device). For channel f
 * and sample t, row t of y holds 2N FP8 E5M2 codes in groups of four inputs, (16 Re x_{4g..4g+3},
 * Im x_{4g..4g+3}) for g = 0..N/4-1 (the integers are exact in E5M2; the factor 16 is a power of
 * two removed again when the correlation is drained), then zeros up to R.
 *   y      out, uint8 [F][ldy][R] with R = round_up(2N, 128); rows T..ldy-1 are zero.
 *          ldy % 128 == 0 and ldy >= T.
 */
int xe_unpack(const uint8_t *frame, xe_shape s, uint8_t *y, int64_t ldy, void *stream);

/* ---------------------------------------------------------------- time shift (Fig. 4) */

/*
 * Integer time shift of every input, the "time shifting" stage Fig. 4's caption names among the
 * optional GPU stages between a frame's transfer and its correlation (the paper defines it no
 * further). Reading used: input n of every channel is delayed by delays[n] samples,
 *   out[t][f][n] = in[t - delays[n]][f][n] for t >= delays[n], 0 (no data) for t < delays[n];
 * a common signal that reaches input n tau_n samples late is re-aligned by delays[n] = D - tau_n.
 * Lost samples of the input frame are zeros and stay zeros. Run it on an assembled frame before
 * xe_correlate.
 *   in, out     device, uint8 [T][F][N], distinct buffers, 16-byte aligned
 *   delays      HOST, int32 [N], 0 <= delays[n] <= T (read during the call)
 * When the delays of every 128 consecutive inputs lie within 256 samples of each other, tiles of
 * 128 rows x 128 inputs are shifted through shared memory (bounded device waits: XE_ETIMEOUT in
 * xe_device_status); wider spreads take a kernel that reads each sample from global memory.
 * Errors: XE_EINVAL (shape, pointers, overlap, alignment, a delay out of range), XE_ECUDA.
 */
int xe_time_shift(const uint8_t *in, xe_shape s, const int32_t *delays, uint8_t *out, void *stream);

/*
 * The shift's samples without data, as the per-input counters xe_normalize takes (Sec. II-C):
 *   flag_count[f][n] += delays[n]                   (input n has no data in its first delays[n] samples)
 *   flag_pairs[f][p(i,j)] += min(delays[i], delays[j])  (samples missing for both inputs)
 * for every channel f. With these (added to any F-engine flag counts), xe_normalize divides each
 * visibility by the number of samples in which both inputs had data.
 *   delays      HOST, int32 [N], as for xe_time_shift
 *   flag_count  device, uint32 [F][N], in/out;  flag_pairs  device, uint32 [F][P], in/out
 * Errors: XE_EINVAL, XE_ECUDA.
 */
int xe_time_shift_counts(const int32_t *delays, xe_shape s, uint32_t *flag_count, uint32_t *flag_pairs,
                         void *stream);

/* ---------------------------------------------------------------- A3/A4: correlation */

/* Engines of the correlation. */
#define XE_ENGINE_AUTO 0        /* the tuned default (XE_ENGINE_FUSED_PAIR) */
#define XE_ENGINE_UNPACKED 1    /* A2 unpack to HBM (MN-major), then the tcgen05 GEMM reads it */
#define XE_ENGINE_FUSED 2       /* the GEMM loads packed bytes and expands them in shared memory */
#define XE_ENGINE_UNPACKED_K 3  /* A2 unpack to HBM transposed (K-major), then the GEMM */
#define XE_ENGINE_FUSED_PAIR 4  /* as FUSED, on CTA pairs: 256x256 blocks with M = 256 pair MMAs */
#define XE_ENGINE_LEGACY_S4 5   /* baseline, no tcgen05: warp-level mma.sync m16n8k64 with 4-bit signed
                                   operands straight on the packed samples (three MMAs per tile:
                                   Re V = A B^T, Im V = 2 A' B'^T - A B'^T with B' nibble-swapped and
                                   A' the Im nibbles); max_strip, k_flush and n_ctas are ignored */
#define XE_ENGINE_LEGACY_S8 6   /* baseline, no tcgen05: as LEGACY_S4 with mma.sync m16n8k32 on int8 (re, im)
                                   pairs unpacked in shared memory */

typedef struct {
    int32_t engine;      /* XE_ENGINE_* */
    int32_t max_strip;   /* single-CTA engines: 1..4 tiles of 128x128 per work item along a row;
                            <= 2 double-buffers the tensor-memory accumulator (default 4). The
                            pair engine always computes 256x256 blocks. */
    int32_t k_flush;     /* time samples accumulated in TMEM before draining to int32; multiple
                            of 128, at most 32768 (keeps every FP32 partial sum below 2^22,
                            where it is exact); 0 = default (32768) */
    int32_t n_ctas;      /* persistent CTAs; 0 = one per SM */
} xe_tune;

/*
 * Cross-correlation of all input pairs for every channel of one frame (Sec. I: the X-engine
 * correlates all inputs against one another within each band; Sec. II-B: kernels do the
 * cross-correlation and integration, adding to the previous output).
 *   frame       device, uint8 [T][F][N]
 *   vis         in/out, int32 [F][P][2]; written when accumulate == 0, added to otherwise
 *               (integration over frames, Sec. II-B). The caller keeps the integrated sample
 *               count <= XE_MAX_TIME.
 *   ws          workspace of xe_correlate_workspace_size(s) bytes.
 * Results are bit-exact integers. Errors: XE_EINVAL (shape: N % 16, N < 16, F < 1, T < 0, or
 * N > 4096), XE_EOVERFLOW (T > XE_MAX_TIME), XE_ENOMEM (ws too small).
 */
size_t xe_correlate_workspace_size(xe_shape s);
int xe_correlate(const uint8_t *frame, xe_shape s, int32_t *vis, int accumulate, void *ws,
                 size_t ws_bytes, void *stream);

/*
 * Rate probe of the legacy warp-level integer tensor path (the baseline XE_ENGINE_LEGACY_S4 runs
 * on): `blocks` CTAs of 256 threads, each warp issuing iters x 8 independent mma.sync with
 * register operands. kind 0: m16n8k64 s4 x s4 -> s32 (16,384 int ops per instruction); kind 1:
 * m16n8k32 s8 x s8 -> s32 (8,192); kind 2: the CUDA-core dp4a (four int8 products added to an
 * int32; 256 int ops per warp instruction), for comparison. The caller times the launch on `stream`.
 *   sink   device, int32 [blocks * 256]: written (keeps the results live), values meaningless.
 * Errors: XE_EINVAL (kind, blocks < 1, iters < 1, sink NULL), XE_ECUDA.
 */
int xe_probe_mma_legacy(int32_t kind, int32_t blocks, int32_t iters, int32_t *sink, void *stream);

/* ---------------------------------------------------------------- tuning table (A6) */

/* Item layouts of the CTA-pair engine. Packet mode (xe_correlate_packets, the serving loop) runs a
 * kernel with 128-sample stages that reads samples in 4-sample slots, with layouts 0-4. Frame mode
 * (xe_correlate, xe_correlate_batched) runs either that kernel (T % 4 == 0 only) or a kernel with
 * 256-sample stages and every Gram block its own item (XE_LAYOUT_FRAME_BLOCKS). Without a table
 * entry a frame launch takes the 128-sample kernel with the fold layout when its largest job has
 * 129 to 256 inputs, and the 256-sample kernel otherwise. */
#define XE_LAYOUT_AUTO 0       /* fold for N > 128; below, Gram blocks with twins from T >= 16384 */
#define XE_LAYOUT_GRAM 1       /* Gram blocks: doubles and singles, twins from T >= 16384, wide singles below */
#define XE_LAYOUT_GRAM_TWIN 2  /* Gram blocks, twins at any T */
#define XE_LAYOUT_GRAM_WIDE 3  /* Gram blocks, wide singles at any T */
#define XE_LAYOUT_FOLD 4       /* one fold item per whole 256-input super-block (N > 128; else GRAM); see
                                  XE_LAYOUT_FOLD_SPLIT for launches whose last round would be ragged */
#define XE_LAYOUT_FRAME_BLOCKS 5   /* frame mode: every Gram block its own item, 256-sample stages */
#define XE_LAYOUT_FOLD_SPLIT 6     /* fold, and a one-job launch of 129-256 inputs splits its channels' samples
                                      evenly over the CTA pairs (pieces add through L2); AUTO and FOLD do so
                                      when whole channels would leave over a tenth of the last round idle */

/*
 * One entry of the library's tuning table: the choices of the CTA-pair engine for jobs with N inputs
 * and t_bucket / 2 < T <= t_bucket (t_bucket a power of two >= 128) in one mode (packets or
 * frames). The table is filled by an
 * autotuner that measures the candidates on the device (paper_1503_06189_b300/autotune.py) and is
 * consulted by every pair-engine launch: a batched launch takes each job's layout from its own
 * entry, and the launch-wide choices (pairs, odd_pairs, k_flush, and in frame mode the kernel:
 * XE_LAYOUT_FRAME_BLOCKS or not) from the entry of its largest job.
 * A non-zero field of an explicit xe_tune argument overrides the table.
 */
#define XE_TUNE_PACKETS 0      /* entry for packet-mode launches (xe_correlate_packets, serving loop) */
#define XE_TUNE_FRAMES 1       /* entry for frame-mode launches (xe_correlate, xe_correlate_batched) */

typedef struct {
    int32_t n_inputs;   /* N of the entry */
    int32_t t_bucket;   /* T bucket: power of two >= 128 */
    int32_t mode;       /* XE_TUNE_PACKETS or XE_TUNE_FRAMES */
    int32_t layout;     /* XE_LAYOUT_* (XE_LAYOUT_FRAME_BLOCKS: frame mode only) */
    int32_t pairs;      /* CTA pairs per launch, 0 = as many as can be resident; a count that would
                           add a round of work items at a launch's item count (the tuner measures
                           at its own probe size) gives way to the fewest pairs that keep the
                           rounds of a launch on all resident pairs */
    int32_t odd_pairs;  /* 1: an odd pair count, 0: as counted, -1: the layout's default (odd for Gram) */
    int32_t k_flush;    /* drain interval in samples, multiple of 128 up to 32768; 0 = default */
} xe_tune_entry;

#define XE_TUNE_MAX_ENTRIES 256

/* Replaces the tuning table (n = 0 clears it; then every job takes the built-in choices).
 * Host memory, read during the call. Errors: XE_EINVAL (n < 0 or > XE_TUNE_MAX_ENTRIES, an entry
 * with a field out of range, or two entries for one (N, t_bucket)). */
int xe_tune_table_set(const xe_tune_entry *entries, int32_t n);
/* Copies up to cap entries of the table into out (host memory); returns the number of entries. */
int xe_tune_table_get(xe_tune_entry *out, int32_t cap);

/* ---------------------------------------------------------------- A6: batched persistent */

#define XE_MAX_JOBS 64

typedef struct {
    const uint8_t *frame;  /* device, uint8 [T][F][N] */
    int32_t *vis;          /* device, int32 [F][P][2] */
    xe_shape s;
    int32_t accumulate;    /* 0: write, 1: add */
    int32_t max_strip;     /* 1..4: tile width of this job's work items; 0 = the call's tune */
} xe_job;

/*
 * All channels of up to XE_MAX_JOBS frames, of possibly different N, F and T, in one persistent
 * launch (Sec. II-B: chains of operations are preloaded to hide launch latency). `jobs` is a HOST
 * array, read during the call. `tune` may be NULL (tuned defaults). The launch is capturable in a
 * CUDA graph. Same per-job rules and errors as xe_correlate.
 */
size_t xe_correlate_batched_workspace_size(const xe_job *jobs, int32_t n_jobs, const xe_tune *tune);
int xe_correlate_batched(const xe_job *jobs, int32_t n_jobs, const xe_tune *tune, void *ws,
                         size_t ws_bytes, void *stream);

/*
 * Zero-copy assembly and correlation of one frame (A1 + A2..A4 without the assembled frame;
 * Sec. II-A.2 for the placement rules, Sec. II-B for the correlation). The result is exactly that of
 * xe_assemble followed by xe_correlate on the assembled frame: the same vis, filled, lost and stats.
 * The payloads are never copied into a frame: the call builds the frame's index (which packet, if
 * any, supplies each 4-sample slot of each 8-channel group; first arrival wins, as in
 * xe_assemble) and the correlator reads every sample straight from its packet through that index,
 * reading lost slots as zeros. This saves the frame's write and re-read in device memory (2 bytes
 * of traffic per packed sample).
 *
 *   pkts, n_pkts, pkt_stride, seq0, groups_per_stream, s, filled, lost, stats: as xe_assemble
 *               (T % 4 == 0, F % 8 == 0; lost and stats accumulate).
 *   vis         as xe_correlate (accumulate != 0 adds to it).
 *   ws          workspace of xe_correlate_packets_workspace_size(s) bytes (any contents).
 * Runs the tuned pair engine. The packet buffer must stay unchanged until the call's work on
 * `stream` has finished. Errors: those of xe_assemble and xe_correlate.
 */
size_t xe_correlate_packets_workspace_size(xe_shape s);
int xe_correlate_packets(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0,
                         int32_t groups_per_stream, xe_shape s, int32_t *vis, int accumulate,
                         uint8_t *filled, uint32_t *lost, uint32_t *stats, void *ws, size_t ws_bytes,
                         void *stream);

/*
 * xe_correlate_packets with the time shift of Fig. 4's caption applied while the samples are read
 * (no shifted frame is written, no extra pass over the data). The result is exactly that of
 * xe_assemble, then xe_time_shift with `delays`, then xe_correlate: input n of every channel is
 * read delays[n] samples late, and the first delays[n] samples of the frame read as zeros (no
 * data). The shift is applied per block of 16 inputs, the unit one converter thread reads: the 16
 * inputs 16b .. 16b + 15 must share one delay (inputs fed through one cable or digitiser board).
 *   delays      HOST, int32 [N], 0 <= delays[n] <= T, delays[16b + k] == delays[16b] (read during
 *               the call; the values go into the launch's parameters, so a captured graph keeps them)
 *   others      as xe_correlate_packets (same workspace size).
 * Add the samples without data to the normalisation's counters with xe_time_shift_counts.
 * Errors: those of xe_correlate_packets; XE_EINVAL for a delay out of range or differing within a
 * block of 16 inputs.
 */
int xe_correlate_packets_shifted(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0,
                                 int32_t groups_per_stream, xe_shape s, const int32_t *delays, int32_t *vis,
                                 int accumulate, uint8_t *filled, uint32_t *lost, uint32_t *stats, void *ws,
                                 size_t ws_bytes, void *stream);

/*
 * F-engine flags of one frame (Sec. II-C: the F-engine flags samples of individual inputs,
 * frequencies and times, sends the flags as bit fields with the data and zeroes the flagged samples;
 * the X-engine counts them per input and, per sample, the inputs flagged together). Footer reading
 * used: at byte 16 + 32N of each packet record, [4 t][8 f][N/8] bytes, bit n % 8 of byte n / 8 set
 * when input n is flagged (records of at least 16 + 36N bytes; 9,232 B at N = 256). Packets are
 * placed as xe_assemble places them (first arrival of a slot wins; late, early, invalid and
 * duplicate packets are ignored); a missing packet flags nothing (its samples are lost instead).
 *
 *   pkts, n_pkts, pkt_stride, seq0, groups_per_stream, s: as xe_assemble.
 *   flag_count  in/out, uint32 [F][N]; += flagged samples of input n in channel f.
 *   flag_pairs  in/out, uint32 [F][P]; += samples in which inputs i <= j are both flagged.
 *   ws          workspace of xe_flag_counts_workspace_size(s) bytes (any contents).
 * Feed both to xe_normalize. Cost grows with E^2 for E inputs flagged in one sample.
 * Errors: XE_EINVAL (geometry, records without a footer, alignment), XE_ENOMEM, XE_ECUDA.
 */
size_t xe_flag_counts_workspace_size(xe_shape s);
int xe_flag_counts(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0,
                   int32_t groups_per_stream, xe_shape s, uint32_t *flag_count, uint32_t *flag_pairs,
                   void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------- A5: normalisation (Sec. II-C) */

/*
 * Normalisation by the per-visibility sample count (Sec. II-C): packet loss is one counter per
 * channel applied to every point of the matrix; F-engine flags are counted per input and channel;
 * inputs flagged in the same sample are counted back once per pair.
 *   n_ij = t_int - lost[f] - c[f][i] - c[f][j] + x[f][p(i,j)]   (i != j)
 *   n_ii = t_int - lost[f] - c[f][i]
 *   out  = (float)V / (float)n_ij with IEEE division, 0 where n_ij <= 0.
 *   vis         device, int32 [F][P][2] (integrated visibilities)
 *   lost        device, uint32 [F]: lost samples per channel over the integration
 *   flag_count  device, uint32 [F][N] or NULL; flag_pairs device, uint32 [F][P] or NULL (both
 *               or neither)
 *   out         out, float [F][P][2];  n_out  out, uint32 [F][P] or NULL
 * Errors: XE_EINVAL, XE_EOVERFLOW (t_int > XE_MAX_TIME).
 */
int xe_normalize(const int32_t *vis, xe_shape s, uint32_t t_int, const uint32_t *lost,
                 const uint32_t *flag_count, const uint32_t *flag_pairs, float *out,
                 uint32_t *n_out, void *stream);

/* ---------------------------------------------------------------- A7: serving loop (Sec. II) */

/*
 * A streaming X-engine that keeps packet buffers, frames and visibilities resident on the device
 * (Sec. II: buffer objects and ring buffers between threads; all memory allocated at start-up and
 * freed at shutdown, Sec. II; per-stream processing until after correlation, then combined, Sec. II
 * and II-C; "Data Ready" events and host callbacks, Sec. II-B).
 *
 * Producers submit packets of their F-engine stream as they arrive (any order within the reorder
 * window). The host reads only the 16-byte headers: each run of packets of one frame is copied
 * directly into that frame's device packet region. A frame closes when more than reorder_window
 * packets of later frames have arrived on its stream (or at xe_stream_flush); closed frames are
 * admitted into free device slots, indexed (the assembly's placement rules without moving the
 * payloads, as in xe_correlate_packets), correlated together in one batched persistent launch per
 * admission round that reads every sample from its packet region, and normalised by their sample
 * counts (xe_normalize). A packet region is reused once that launch has read it. Rounds run on a
 * pool of CUDA streams and overlap on the device; a host callback marks each frame complete.
 * Results stay on the device until released.
 *
 * Frame k of a stream covers seq [k*T/4, (k+1)*T/4). All device memory is allocated by
 * xe_stream_create (within hbm_budget when it is non-zero) and freed by xe_stream_destroy.
 */
typedef struct {
    int32_t n_streams;          /* F-engine streams (stream_id 0..n_streams-1) */
    int32_t groups_per_stream;  /* channel groups of 8 per stream: F_s = 8 * groups_per_stream */
    int32_t n_inputs;           /* N, multiple of 16 */
    int32_t n_time;             /* T per frame, multiple of 4 */
    uint32_t pkt_stride;        /* bytes per packet record, multiple of 16, >= 16 + 32 N */
    int32_t reorder_window;     /* packets of later frames after which a frame closes (>= 1) */
    int32_t ring_frames;        /* device packet regions per stream (frames buffered), >= 2 */
    int32_t slots;              /* device frame slots (frames in flight or unreleased); 0 = by budget */
    int32_t max_batch;          /* frames correlated per launch, 1..XE_MAX_JOBS */
    int32_t n_cuda_streams;     /* CUDA streams rounds are spread over, >= 1 */
    uint64_t hbm_budget;        /* bytes the runtime may allocate; 0 = no limit */
    int32_t batch_wait_us;      /* after the first ready frame, wait up to this long for more frames
                                   to join the round (0 = admit at once) */
} xe_stream_cfg;

typedef struct xe_stream xe_stream;

typedef struct {
    int32_t stream_id;
    int32_t slot;               /* pass back to xe_stream_release */
    int64_t frame;              /* frame index k */
    const float *out;           /* device, float [F_s][P][2]: V / n, valid until released */
    const int32_t *vis;         /* device, int32 [F_s][P][2]: integrated visibilities */
    const uint32_t *n;          /* device, uint32 [F_s][P]: samples per visibility */
    const uint32_t *lost;       /* device, uint32 [F_s]: lost samples per channel */
    const uint32_t *stats;      /* device, uint32 [5]: ok, duplicate, late, early, invalid */
    uint32_t packets;           /* packets submitted into this frame's region */
    uint32_t batch;             /* admission round that carried the frame */
    uint64_t latency_ns;        /* frame closed -> its results complete on the device */
    uint64_t latency_submit_ns; /* submission of the frame's last packet -> results complete (includes
                                   the wait for the reorder window to close the frame) */
} xe_result;

typedef struct {
    uint64_t packets_submitted, packets_late, frames_closed, frames_done, frames_released;
    uint64_t batches, max_batch_seen;
    double latency_p50_us, latency_p99_us, latency_max_us;              /* close -> complete */
    uint64_t device_bytes;
    int32_t slots;
    double latency_submit_p50_us, latency_submit_p99_us, latency_submit_max_us;   /* last packet -> complete */
} xe_stream_stats_t;

/* Creates the runtime on the current device. Errors: XE_EINVAL, XE_ENOMEM (budget too small for
 * two slots and the packet regions), XE_ECUDA. */
int xe_stream_create(const xe_stream_cfg *cfg, xe_stream **out);
/* Submits n_pkts packets (host memory, arrival order) of one stream. Packets of closed frames count
 * as late and are dropped. Returns XE_EAGAIN, having consumed nothing, when a packet belongs to a
 * frame whose packet region is still in use, or when frames must close and the queue of closed
 * frames is full (the device or the consumer is behind): poll, release and retry. Pinned host
 * memory is copied asynchronously: keep it unchanged until the frames it holds have completed. */
int xe_stream_submit(xe_stream *s, int32_t stream_id, const void *host_pkts, uint32_t n_pkts);
/* As xe_stream_submit for packets already in device memory (for example written there by a NIC,
 * with the headers also delivered to the host, or replayed from a device ring): dev_pkts holds
 * n_pkts records of pkt_stride bytes on the runtime's device, host_headers the same packets' 16-byte
 * headers back to back in host memory (read during the call, to route each packet to its frame).
 * The records are copied device to device into the frames' packet regions; keep dev_pkts unchanged
 * until the frames it holds have completed. */
int xe_stream_submit_device(xe_stream *s, int32_t stream_id, const void *dev_pkts, const void *host_headers,
                            uint32_t n_pkts);
/* Closes every open frame (end of data). XE_EAGAIN if the queue of closed frames filled up first:
 * poll, release and call it again. */
int xe_stream_flush(xe_stream *s);
/* Waits up to timeout_ms for the next completed frame (completion order). XE_ETIMEOUT if none. */
int xe_stream_poll(xe_stream *s, xe_result *out, int32_t timeout_ms);
/* Returns a completed frame's slot to the pool. */
int xe_stream_release(xe_stream *s, const xe_result *r);
int xe_stream_stats(xe_stream *s, xe_stream_stats_t *out);
/* Waits (bounded) for outstanding device work, then frees everything. */
int xe_stream_destroy(xe_stream *s);

#ifdef __cplusplus
}
#endif

#endif /* XE_H */
