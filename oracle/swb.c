/*
 * Plain C volume oracle for RANLUX++ outputs: the RANLUX subtract-with-borrow
 * recurrence itself (Sec. 1 and Sec. 2 of Hahnfeld & Moneta, arXiv 2106.02504; base
 * b = 2^24, lags r = 24 and s = 10, with a borrow bit), run p steps per delivered block
 * of 24 numbers at luxury level p.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU baseline
 * leg of bench.py load this library.  It shares no code with the CUDA library; it never
 * touches the LCG form that the CUDA path computes with, which makes it an independent
 * check of that path: the LCG advance X <- a^p X mod m must reproduce exactly these
 * numbers (the equivalence the paper relies on, Sec. 1).
 *
 * Every function is single-threaded and reentrant; callers parallelise over streams.
 *
 * Window convention: w[0..23] are the 24 live numbers, w[0] the oldest; c is the
 * borrow.  Read position pos counts 24-bit words already consumed from the current
 * block (0..24).  Draw rule (a reading, the paper does not spell it out): a u24 draw
 * needs one unread word, a double needs two (value w[pos] + 2^24 w[pos+1], times
 * 2^-48, Sec. 2.3); when the block has too few unread words the generator first moves
 * to the next block (p more steps) and the position restarts at 0.
 */
#include <stdint.h>
#include <string.h>

#define SWB_R 24
#define SWB_S 10
#define SWB_MASK 0xFFFFFFu

/* p recurrence steps: x_n = x_{n-s} - x_{n-r} - c_{n-1} mod 2^24, new borrow = 1 iff
 * the difference was negative.  Afterwards w[] holds the newest 24 numbers, oldest
 * first. */
void swb_block(uint32_t w[SWB_R], uint32_t *carry, int32_t p)
{
    uint32_t ring[SWB_R];
    memcpy(ring, w, sizeof ring);
    uint32_t c = *carry;
    int oldest = 0; /* ring[oldest] = x_{n-24}, ring[(oldest + 14) % 24] = x_{n-10} */
    for (int32_t step = 0; step < p; ++step) {
        int lag_s = oldest + (SWB_R - SWB_S);
        if (lag_s >= SWB_R)
            lag_s -= SWB_R;
        /* Both numbers are below 2^24, so the difference is negative exactly when
         * bit 31 of its 32-bit wrap-around is set, and its low 24 bits are the
         * difference mod 2^24 (2^32 is a multiple of 2^24). */
        uint32_t diff = ring[lag_s] - ring[oldest] - c;
        c = diff >> 31;
        ring[oldest] = diff & SWB_MASK; /* x_n replaces x_{n-24} */
        oldest = oldest + 1 == SWB_R ? 0 : oldest + 1;
    }
    for (int i = 0; i < SWB_R; ++i) {
        int k = oldest + i;
        if (k >= SWB_R)
            k -= SWB_R;
        w[i] = ring[k];
    }
    *carry = c;
}

/* n 24-bit integers; returns the number of blocks advanced. */
int64_t swb_draw_u24(uint32_t w[SWB_R], uint32_t *carry, int32_t *pos, int32_t p,
                     int64_t n, uint32_t *out)
{
    int64_t blocks = 0;
    for (int64_t k = 0; k < n; ++k) {
        if (*pos + 1 > SWB_R) {
            swb_block(w, carry, p);
            *pos = 0;
            ++blocks;
        }
        out[k] = w[*pos] & SWB_MASK;
        *pos += 1;
    }
    return blocks;
}

/* n 48-bit integers v = w[pos] + 2^24 w[pos+1]; returns the number of blocks. */
int64_t swb_draw_bits48(uint32_t w[SWB_R], uint32_t *carry, int32_t *pos, int32_t p,
                        int64_t n, uint64_t *out)
{
    int64_t blocks = 0;
    for (int64_t k = 0; k < n; ++k) {
        if (*pos + 2 > SWB_R) {
            swb_block(w, carry, p);
            *pos = 0;
            ++blocks;
        }
        out[k] = (uint64_t)w[*pos] | ((uint64_t)w[*pos + 1] << 24);
        *pos += 2;
    }
    return blocks;
}

/* n doubles in [0, 1): the 48-bit integer converted to double (exact, it is below
 * 2^53) and scaled by 2^-48 (exact, a power of two). */
int64_t swb_draw_f64(uint32_t w[SWB_R], uint32_t *carry, int32_t *pos, int32_t p,
                     int64_t n, double *out)
{
    int64_t blocks = 0;
    const double scale = 1.0 / 281474976710656.0; /* 2^-48 */
    for (int64_t k = 0; k < n; ++k) {
        if (*pos + 2 > SWB_R) {
            swb_block(w, carry, p);
            *pos = 0;
            ++blocks;
        }
        uint64_t v = (uint64_t)w[*pos] | ((uint64_t)w[*pos + 1] << 24);
        out[k] = (double)v * scale;
        *pos += 2;
    }
    return blocks;
}

/* n single-precision floats w 2^-24 in [0, 1), one number each (exact). */
int64_t swb_draw_f32(uint32_t w[SWB_R], uint32_t *carry, int32_t *pos, int32_t p,
                     int64_t n, float *out)
{
    int64_t blocks = 0;
    const float scale = 1.0f / 16777216.0f; /* 2^-24 */
    for (int64_t k = 0; k < n; ++k) {
        if (*pos + 1 > SWB_R) {
            swb_block(w, carry, p);
            *pos = 0;
            ++blocks;
        }
        out[k] = (float)w[*pos] * scale;
        *pos += 1;
    }
    return blocks;
}

/* Fused consumer: exact sum of n 48-bit integers and a 256-bin histogram of their top
 * 8 bits (hist is accumulated, not cleared). */
int64_t swb_sum_hist48(uint32_t w[SWB_R], uint32_t *carry, int32_t *pos, int32_t p,
                       int64_t n, uint64_t *sum, uint64_t hist[256])
{
    int64_t blocks = 0;
    uint64_t s = 0;
    for (int64_t k = 0; k < n; ++k) {
        if (*pos + 2 > SWB_R) {
            swb_block(w, carry, p);
            *pos = 0;
            ++blocks;
        }
        uint64_t v = (uint64_t)w[*pos] | ((uint64_t)w[*pos + 1] << 24);
        s += v;
        hist[v >> 40] += 1;
        *pos += 2;
    }
    *sum = s;
    return blocks;
}

/* Many streams, each described by its own window/borrow/position, one after another.
 * w: n_streams x 24 words, carry/pos: n_streams each; draws `count` values per stream;
 * out: n_streams x count values, stream-major.  kind: 0 = u24 (uint32 out),
 * 1 = f64 (double out), 2 = bits48 (uint64 out), 3 = f32 (float out). */
void swb_draw_many(int64_t n_streams, uint32_t *w, uint32_t *carry, int32_t *pos,
                   int32_t p, int64_t count, int32_t kind, void *out)
{
    for (int64_t i = 0; i < n_streams; ++i) {
        uint32_t *wi = w + i * SWB_R;
        if (kind == 0)
            swb_draw_u24(wi, carry + i, pos + i, p, count, (uint32_t *)out + i * count);
        else if (kind == 1)
            swb_draw_f64(wi, carry + i, pos + i, p, count, (double *)out + i * count);
        else if (kind == 3)
            swb_draw_f32(wi, carry + i, pos + i, p, count, (float *)out + i * count);
        else
            swb_draw_bits48(wi, carry + i, pos + i, p, count, (uint64_t *)out + i * count);
    }
}

/* Fused consumer over many streams: per-stream exact sums, one shared histogram. */
void swb_sum_hist_many(int64_t n_streams, uint32_t *w, uint32_t *carry, int32_t *pos,
                       int32_t p, int64_t count, uint64_t *sums, uint64_t hist[256])
{
    for (int64_t i = 0; i < n_streams; ++i)
        swb_sum_hist48(w + i * SWB_R, carry + i, pos + i, p, count, sums + i, hist);
}
