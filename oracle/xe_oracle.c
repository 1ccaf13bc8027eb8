/*
 * xe_oracle.c -- plain, slow, obviously correct CPU oracle of the X-engine hot path.
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the package smoke check and the CPU-baseline leg of the
 * benchmark call it; the product library never links, loads or calls anything in this directory,
 * and this file includes nothing from the product. Paper: Recnik et al., "An Efficient Real-time
 * Data Pipeline for the CHIME Pathfinder Radio Telescope X-Engine" (cited by section below).
 *
 * Conventions (readings of the paper where it is silent; each is listed in the design notes):
 *   - a sample is one byte, high nibble = real part, low nibble = imaginary part, both 4-bit
 *     two's complement in [-8, 7]                                      (Sec. I "4+4-bit complex")
 *   - V_f[i,j] = sum_t x_{f,t}[i] * conj(x_{f,t}[j]) for i <= j             (Sec. I, Sec. II-B)
 *   - visibilities are stored as the packed upper triangle incl. the diagonal, row-major,
 *     [F][P][2] with P = N(N+1)/2 and {re, im} interleaved          (Table I output size)
 *   - frames are [T][F][N] bytes; packets carry [4 t][8 f][N n] after a 16-byte header
 *     {u16 stream_id, u16 chan_group, u32 reserved, u64 seq}           (Sec. II-A)
 *
 * All sums are in int64 with plain loops in the order the definitions are written. OpenMP only
 * splits independent (channel, row) pairs across threads; it reorders no arithmetic.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define XO_OK 0
#define XO_EINVAL (-1)
#define XO_EOVERFLOW (-2)

/* One 4+4-bit sample -> (re, im). Sec. I: the data are reduced to 4+4-bit complex numbers. */
void xo_sample(uint8_t b, int *re, int *im) {
    int hi = (b >> 4) & 0xF;
    int lo = b & 0xF;
    *re = hi >= 8 ? hi - 16 : hi;
    *im = lo >= 8 ? lo - 16 : lo;
}

/* Number of packed visibilities per channel: the upper triangle including the diagonal. */
int64_t xo_npairs(int n) { return (int64_t)n * (n + 1) / 2; }

/* Position of (i, j), i <= j, in the row-major packed upper triangle. Rows 0..i-1 hold
 * N + (N-1) + ... + (N-i+1) = i*N - i*(i-1)/2 entries; (i, j) is entry j-i of row i. */
int64_t xo_pidx(int i, int j, int n) {
    return (int64_t)i * n - (int64_t)i * (i - 1) / 2 + (j - i);
}

/*
 * Correlation of channels [f0, f0+nf) of a frame [T][F][N] (Sec. I: the X-engine "correlates all
 * of the inputs against one another within each frequency band"; Sec. II-B: kernels do the
 * cross-correlation and integration).
 *   re V[i,j] = sum_t (a_i a_j + b_i b_j),  im V[i,j] = sum_t (b_i a_j - a_i b_j),  x = a + i b.
 * vis: int64 [nf][P][2]. Returns XO_EOVERFLOW if any component does not fit in int32 (the
 * visibility format), XO_OK otherwise; vis holds the exact int64 sums in both cases.
 */
int xo_correlate(const uint8_t *frame, int N, int F, int T, int f0, int nf, int64_t *vis) {
    if (!frame || !vis || N <= 0 || F <= 0 || T < 0 || f0 < 0 || nf < 0 || f0 + nf > F) return XO_EINVAL;
    const int64_t P = xo_npairs(N);
    int overflow = 0;
    for (int fc = 0; fc < nf; ++fc) {
        const int f = f0 + fc;
        /* the channel's samples, unpacked: a[n][t], b[n][t] */
        int *a = (int *)malloc(sizeof(int) * (size_t)N * (size_t)(T > 0 ? T : 1));
        int *b = (int *)malloc(sizeof(int) * (size_t)N * (size_t)(T > 0 ? T : 1));
        if (!a || !b) { free(a); free(b); return XO_EINVAL; }
        for (int t = 0; t < T; ++t)
            for (int n = 0; n < N; ++n)
                xo_sample(frame[((size_t)t * F + f) * N + n], &a[(size_t)n * T + t], &b[(size_t)n * T + t]);
        int ovf = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : ovf)
        for (int i = 0; i < N; ++i) {
            const int *ai = a + (size_t)i * T, *bi = b + (size_t)i * T;
            for (int j = i; j < N; ++j) {
                const int *aj = a + (size_t)j * T, *bj = b + (size_t)j * T;
                int64_t sr = 0, si = 0;
                for (int t = 0; t < T; ++t) {
                    sr += (int64_t)ai[t] * aj[t] + (int64_t)bi[t] * bj[t];
                    si += (int64_t)bi[t] * aj[t] - (int64_t)ai[t] * bj[t];
                }
                int64_t *v = vis + ((size_t)fc * P + xo_pidx(i, j, N)) * 2;
                v[0] = sr;
                v[1] = si;
                if (sr > INT32_MAX || sr < INT32_MIN || si > INT32_MAX || si < INT32_MIN) ovf = 1;
            }
        }
        overflow |= ovf;
        free(a);
        free(b);
    }
    return overflow ? XO_EOVERFLOW : XO_OK;
}

/*
 * Selected visibilities of one channel f, straight from the definition (for sampled checks of
 * frames too large to correlate in full on the CPU). pairs: int32 [n][2] with i <= j; vis: int64
 * [n][2].
 */
int xo_correlate_pairs(const uint8_t *frame, int N, int F, int T, int f, const int32_t *pairs, int n,
                       int64_t *vis) {
    if (!frame || !pairs || !vis || N <= 0 || F <= 0 || T < 0 || f < 0 || f >= F || n < 0) return XO_EINVAL;
    for (int q = 0; q < n; ++q)
        if (pairs[2 * q] < 0 || pairs[2 * q] > pairs[2 * q + 1] || pairs[2 * q + 1] >= N) return XO_EINVAL;
#pragma omp parallel for schedule(dynamic, 4)
    for (int q = 0; q < n; ++q) {
        const int i = pairs[2 * q], j = pairs[2 * q + 1];
        int64_t sr = 0, si = 0;
        for (int t = 0; t < T; ++t) {
            int ai, bi, aj, bj;
            xo_sample(frame[((size_t)t * F + f) * N + i], &ai, &bi);
            xo_sample(frame[((size_t)t * F + f) * N + j], &aj, &bj);
            sr += (int64_t)ai * aj + (int64_t)bi * bj;
            si += (int64_t)bi * aj - (int64_t)ai * bj;
        }
        vis[2 * q] = sr;
        vis[2 * q + 1] = si;
    }
    return XO_OK;
}

/*
 * Frame assembly from UDP packets (Sec. II-A.2: loss zero-fill, reorder by sequence number,
 * duplicates ignored), replayed packet by packet in arrival order.
 *   pkts      n_pkts records of pkt_stride bytes: 16-byte header then [4][8][N] payload
 *   seq0      sequence number of the frame's first packet slot; the frame spans T/4 slots
 *   gps       channel groups (of 8 channels) per stream; global group G = stream_id*gps + chan_group
 * Outputs: frame [T][F][N]; filled [T/4][F/8] (1 = the slot's packet arrived); lost [F] += lost
 * samples per channel (4 per missing packet); stats[5] += {ok, duplicate, late, early, invalid}.
 * A packet is "late" when seq < seq0, "early" when seq >= seq0 + T/4, "invalid" when its stream or
 * group is outside the frame. The first arrival of a slot wins; later arrivals are duplicates.
 */
int xo_assemble(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0, int gps,
                int N, int F, int T, uint8_t *frame, uint8_t *filled, uint32_t *lost, uint32_t *stats) {
    if (N <= 0 || F <= 0 || T <= 0 || (T % 4) || (F % 8) || gps <= 0 || ((F / 8) % gps)) return XO_EINVAL;
    const uint32_t payload = 4u * 8u * (uint32_t)N;
    if (pkt_stride < 16 + payload) return XO_EINVAL;
    const int Q = T / 4, G = F / 8, S = G / gps;
    memset(filled, 0, (size_t)Q * G);
    for (uint32_t k = 0; k < n_pkts; ++k) {
        const uint8_t *p = pkts + (size_t)k * pkt_stride;
        uint16_t sid, grp;
        uint64_t seq;
        memcpy(&sid, p + 0, 2);
        memcpy(&grp, p + 2, 2);
        memcpy(&seq, p + 8, 8);
        if (sid >= S || grp >= gps) { stats[4]++; continue; }
        if (seq < seq0) { stats[2]++; continue; }
        if (seq - seq0 >= (uint64_t)Q) { stats[3]++; continue; }
        const int slot = (int)(seq - seq0);
        const int g = sid * gps + grp;
        if (filled[(size_t)slot * G + g]) { stats[1]++; continue; }
        filled[(size_t)slot * G + g] = 1;
        stats[0]++;
        for (int tt = 0; tt < 4; ++tt)
            for (int ff = 0; ff < 8; ++ff)
                for (int n = 0; n < N; ++n)
                    frame[((size_t)(4 * slot + tt) * F + (8 * g + ff)) * N + n] =
                        p[16 + ((size_t)tt * 8 + ff) * N + n];
    }
    /* Sec. II-A.2: where a packet is missing, zeros are written in its place. */
    for (int slot = 0; slot < Q; ++slot)
        for (int g = 0; g < G; ++g) {
            if (filled[(size_t)slot * G + g]) continue;
            for (int tt = 0; tt < 4; ++tt)
                for (int ff = 0; ff < 8; ++ff) {
                    memset(frame + ((size_t)(4 * slot + tt) * F + (8 * g + ff)) * N, 0, (size_t)N);
                }
            for (int ff = 0; ff < 8; ++ff) lost[8 * g + ff] += 4;
        }
    return XO_OK;
}

/*
 * F-engine flags of one frame (Sec. II-C: flags for each input, frequency and time sample arrive in
 * the packets' footers; flagged samples are already zero in the data). Footer reading used here:
 * at byte 16 + 32N of a packet, [4 t][8 f][N/8] bytes, bit n % 8 of byte n / 8 set when input n is
 * flagged. Packets are replayed in arrival order with the assembly's rules (first arrival of a
 * slot wins; late, early, invalid and duplicate packets are ignored); a missing packet flags
 * nothing (its samples are lost, not flagged).
 * Outputs (accumulated): flag_count [F][N] += flagged samples of input n in channel f;
 * flag_pairs [F][P] += samples in which inputs i and j (i <= j) are both flagged.
 */
int xo_flag_counts(const uint8_t *pkts, uint32_t n_pkts, uint32_t pkt_stride, uint64_t seq0, int gps,
                   int N, int F, int T, uint32_t *flag_count, uint32_t *flag_pairs) {
    if (N <= 0 || N % 8 || F <= 0 || T <= 0 || (T % 4) || (F % 8) || gps <= 0 || ((F / 8) % gps))
        return XO_EINVAL;
    const uint32_t footer = 16u + 32u * (uint32_t)N;
    if (pkt_stride < footer + 4u * (uint32_t)N) return XO_EINVAL;
    const int Q = T / 4, G = F / 8, S = G / gps;
    const int64_t P = xo_npairs(N);
    uint8_t *seen = calloc((size_t)Q * G, 1);
    if (!seen) return XO_EINVAL;
    for (uint32_t k = 0; k < n_pkts; ++k) {
        const uint8_t *p = pkts + (size_t)k * pkt_stride;
        uint16_t sid, grp;
        uint64_t seq;
        memcpy(&sid, p + 0, 2);
        memcpy(&grp, p + 2, 2);
        memcpy(&seq, p + 8, 8);
        if (sid >= S || grp >= gps || seq < seq0 || seq - seq0 >= (uint64_t)Q) continue;
        const int slot = (int)(seq - seq0), g = sid * gps + grp;
        if (seen[(size_t)slot * G + g]) continue;
        seen[(size_t)slot * G + g] = 1;
        for (int tt = 0; tt < 4; ++tt)
            for (int ff = 0; ff < 8; ++ff) {
                const uint8_t *bits = p + footer + ((size_t)tt * 8 + ff) * (N / 8);
                const int f = 8 * g + ff;
                for (int i = 0; i < N; ++i) {
                    if (!((bits[i / 8] >> (i % 8)) & 1)) continue;
                    flag_count[(size_t)f * N + i] += 1;
                    for (int j = i; j < N; ++j)
                        if ((bits[j / 8] >> (j % 8)) & 1) flag_pairs[(size_t)f * P + xo_pidx(i, j, N)] += 1;
                }
            }
    }
    free(seen);
    return XO_OK;
}

/*
 * Per-visibility sample counts by brute force: n_ij = sum_t [valid_i(t) and valid_j(t)].
 * valid: [T][F][N] bytes, nonzero = the sample entered the correlation (Sec. II-C: lost or
 * flagged samples are zeroed before correlation). n: uint32 [F][P].
 */
int xo_counts_from_mask(const uint8_t *valid, int N, int F, int T, uint32_t *n) {
    if (!valid || !n || N <= 0 || F <= 0 || T < 0) return XO_EINVAL;
    const int64_t P = xo_npairs(N);
    for (int f = 0; f < F; ++f)
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = 0; i < N; ++i)
            for (int j = i; j < N; ++j) {
                uint32_t c = 0;
                for (int t = 0; t < T; ++t)
                    c += (valid[((size_t)t * F + f) * N + i] && valid[((size_t)t * F + f) * N + j]) ? 1u : 0u;
                n[(size_t)f * P + xo_pidx(i, j, N)] = c;
            }
    return XO_OK;
}

/*
 * Per-visibility sample counts by the paper's counter scheme (Sec. II-C):
 *   - packet loss is one counter per channel, applied to every matrix point: -lost[f]
 *   - F-engine flags are counted per input and frequency:                       -c[f][i] - c[f][j]
 *   - pairs flagged in the same sample were subtracted twice, so they are added back: +x[f][p(i,j)]
 *   n_ij = t_int - lost[f] - c[f][i] - c[f][j] + x[f][p]   (c[f][i] counted as x[f][p(i,i)] on the diagonal)
 * flag_count (uint32 [F][N]) and flag_pairs (uint32 [F][P]) may both be NULL (no flags).
 */
int xo_counts_from_counters(uint32_t t_int, const uint32_t *lost, const uint32_t *flag_count,
                            const uint32_t *flag_pairs, int N, int F, uint32_t *n) {
    if (!lost || !n || N <= 0 || F <= 0 || (!flag_count) != (!flag_pairs)) return XO_EINVAL;
    const int64_t P = xo_npairs(N);
    for (int f = 0; f < F; ++f)
        for (int i = 0; i < N; ++i)
            for (int j = i; j < N; ++j) {
                const int64_t p = xo_pidx(i, j, N);
                int64_t c = (int64_t)t_int - lost[f];
                if (flag_count) {
                    if (i == j) c -= flag_count[(size_t)f * N + i];
                    else c -= (int64_t)flag_count[(size_t)f * N + i] + flag_count[(size_t)f * N + j]
                              - flag_pairs[(size_t)f * P + p];
                }
                n[(size_t)f * P + p] = c < 0 ? 0u : (uint32_t)c;
            }
    return XO_OK;
}

/*
 * Normalisation (Sec. II-C: "the fraction of lost data given by the normalization matrix is then
 * applied to the correlation matrix"): out = V / n_ij, rounded once from double to float; 0 when
 * n_ij = 0. vis: int64 [F][P][2], n: uint32 [F][P], out: float [F][P][2].
 */
int xo_normalize(const int64_t *vis, const uint32_t *n, int N, int F, float *out) {
    if (!vis || !n || !out || N <= 0 || F <= 0) return XO_EINVAL;
    const int64_t P = xo_npairs(N);
    for (int64_t q = 0; q < (int64_t)F * P; ++q) {
        if (n[q] == 0) { out[2 * q] = 0.0f; out[2 * q + 1] = 0.0f; continue; }
        out[2 * q] = (float)((double)vis[2 * q] / (double)n[q]);
        out[2 * q + 1] = (float)((double)vis[2 * q + 1] / (double)n[q]);
    }
    return XO_OK;
}

/*
 * Time shifting. Fig. 4's caption names "time shifting" among the optional GPU stages between the
 * frame's transfer and the correlation, and the paper defines it no further. Reading used: every
 * input n of every channel is delayed by an integer number of samples d[n], 0 <= d[n] <= T:
 *   out[t][f][n] = in[t - d[n]][f][n]  for t >= d[n],
 *   out[t][f][n] = 0 (no data)          for t <  d[n].
 * in, out: uint8 [T][F][N] (distinct buffers); delays: int32 [N].
 */
int xo_time_shift(const uint8_t *in, int N, int F, int T, const int32_t *delays, uint8_t *out) {
    if (!in || !out || !delays || N <= 0 || F <= 0 || T < 0) return XO_EINVAL;
    for (int n = 0; n < N; ++n)
        if (delays[n] < 0 || delays[n] > T) return XO_EINVAL;
    for (int t = 0; t < T; ++t)
        for (int f = 0; f < F; ++f)
            for (int n = 0; n < N; ++n) {
                const int src = t - delays[n];
                out[((size_t)t * F + f) * N + n] = src >= 0 ? in[((size_t)src * F + f) * N + n] : 0;
            }
    return XO_OK;
}

/*
 * The shift's samples without data, in the form of the per-input counters of Sec. II-C (added to
 * flag_count and flag_pairs, which xo_counts_from_counters takes): input n of every channel has
 * its first d[n] samples without data, c[f][n] += d[n]; inputs i and j both lack their first
 * min(d[i], d[j]) samples, x[f][p(i,j)] += min(d[i], d[j]).
 * flag_count: uint32 [F][N], flag_pairs: uint32 [F][P].
 */
int xo_time_shift_counts(const int32_t *delays, int N, int F, uint32_t *flag_count, uint32_t *flag_pairs) {
    if (!delays || !flag_count || !flag_pairs || N <= 0 || F <= 0) return XO_EINVAL;
    const int64_t P = xo_npairs(N);
    for (int f = 0; f < F; ++f)
        for (int i = 0; i < N; ++i) {
            flag_count[(size_t)f * N + i] += (uint32_t)delays[i];
            for (int j = i; j < N; ++j) {
                const int m = delays[i] < delays[j] ? delays[i] : delays[j];
                flag_pairs[(size_t)f * P + xo_pidx(i, j, N)] += (uint32_t)m;
            }
        }
    return XO_OK;
}

/* Threads the OpenMP runtime will use (reported beside the CPU baseline). */
int xo_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
