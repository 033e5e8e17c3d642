/*
 * rlxpp — RANLUX++ random number streams on one NVIDIA GB300 (sm_103a).
 *
 * C ABI of librlxpp.so.  The method is the one of Hahnfeld & Moneta, "A Portable
 * Implementation of RANLUX++" (arXiv 2106.02504): the RANLUX subtract-with-borrow
 * generator (base 2^24, lags 24 and 10, with a borrow bit) run as a linear
 * congruential generator X <- A X mod m with m = 2^576 - 2^240 + 1 (Sec. 1, Sec. 2.2)
 * and A = a^p, a = 2^-24 mod m, for luxury level p.  Each stream keeps the paper's
 * state (Sec. 2): 24 RANLUX numbers packed in 576 bits, the borrow bit, the read
 * position.  A refill converts the numbers to the LCG state, multiplies by A
 * (multiply9x9, Sec. 2.1), reduces mod m (mod_m, Sec. 2.2) and converts back
 * (Sec. 2.3).
 *
 * Conventions shared by every entry point
 *  - Calls are asynchronous on the CUDA stream passed as `cuda_stream` (a
 *    cudaStream_t; NULL = the legacy default stream).  Argument errors are detected on
 *    the host and returned at once; errors found by kernels are sticky and reported by
 *    rlxpp_sync().
 *  - Pointers to per-stream arrays and outputs may point to device memory or to host
 *    memory (pinned or pageable).  Host arrays are staged through device buffers that
 *    the library owns; the call then returns only after the host data has been read
 *    (inputs) or written (outputs).
 *  - The caller owns every buffer it passes; the library owns the generator state.
 *  - A handle is not thread-safe: calls on one handle must not overlap in time.
 *  - Every call returns RLXPP_OK or an error code; rlxpp_last_error() gives a message
 *    for the calling thread's last failure.  The environment variable RLXPP_LOG, read
 *    once, turns on host logging to stderr: 1 logs every failure with its message, 2
 *    also each create, destroy, draw, skip and seed call.
 *  - Draw order (a reading; the paper does not fix it): the 24 numbers of a block are
 *    delivered oldest first.  A u24 draw returns the next number; a double takes the
 *    next two numbers w_k, w_{k+1} (both from the current block; otherwise the stream
 *    refills first and a lone leftover number is skipped) and returns
 *    (w_k + 2^24 w_{k+1}) * 2^-48, exactly (Sec. 2.3: 48 bits per double).
 *  - Seeding (Sec. 2.4, exponentiation by squaring; the 2^96 spacing is the one in
 *    Sec. 2.5): seed s, 1 <= s < 2^64, starts at the LCG state A^(2^96 s), read
 *    position 0.
 */
#ifndef RLXPP_H
#define RLXPP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlxpp_gen rlxpp_gen;

typedef enum rlxpp_status {
  RLXPP_OK = 0,
  RLXPP_ERR_INVALID = 1,     /* bad argument or state record                        */
  RLXPP_ERR_NOMEM = 2,       /* device or pinned host allocation failed             */
  RLXPP_ERR_CUDA = 3,        /* a CUDA runtime call failed                          */
  RLXPP_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up                  */
  RLXPP_ERR_UNSUPPORTED = 5  /* valid request the library does not implement        */
} rlxpp_status;

/* Exported state of one stream (88 bytes), the paper's generator state (Sec. 2):
 *  d[9]   the 24 RANLUX numbers, number k at bits 24k..24k+23 of the little-endian
 *         576-bit value (k = 0 the oldest);
 *  carry  the borrow bit, 0 or 1;
 *  pos    numbers already read from the current block, 0..24;
 *  p      luxury level (must be one of the handle's levels on import);
 *  reserved must be 0. */
typedef struct rlxpp_state {
  uint64_t d[9];
  uint32_t carry;
  uint32_t pos;
  uint32_t p;
  uint32_t reserved;
} rlxpp_state;

/* Largest number of distinct luxury levels one handle can hold. */
#define RLXPP_MAX_LEVELS 16

/* Create a handle for n_streams streams and seed them.
 *  levels[n_levels]   host array of luxury levels p >= 1 (Sec. 4.2 uses p = 2048);
 *                     1 <= n_levels <= RLXPP_MAX_LEVELS.  For each level the library
 *                     computes A = a^p and a table of A^(j 16^w) (w < 40, j < 16) on
 *                     the device (Sec. 2.4).
 *  level_of_stream    NULL (every stream uses levels[0]) or n_streams bytes, each
 *                     < n_levels, host or device.
 *  seeds              n_streams uint64 seeds >= 1, host or device; stream i starts at
 *                     A^(2^96 seeds[i]).
 *  out                receives the handle; *out is NULL on failure.
 * n_streams may be 0.  Fails with RLXPP_ERR_INVALID on a bad level, level index or
 * seed: a zero in a host seed array fails the call; level indices and device seeds are
 * checked on the device and reported by rlxpp_sync() (such a stream then holds the
 * LCG state 1 at level 0). */
rlxpp_status rlxpp_create(uint64_t n_streams, const uint32_t* levels, uint32_t n_levels,
                          const uint8_t* level_of_stream, const uint64_t* seeds,
                          void* cuda_stream, rlxpp_gen** out);

/* Re-seed every stream in place (levels unchanged): stream i restarts at
 * A^(2^96 seeds[i]) with read position 0.  seeds: n_streams uint64 >= 1, host or
 * device; a zero in a host array fails the call with RLXPP_ERR_INVALID, a zero in a
 * device array leaves that stream unchanged and is reported by rlxpp_sync(). */
rlxpp_status rlxpp_seed(rlxpp_gen* gen, const uint64_t* seeds, void* cuda_stream);

/* Skip ahead (Sec. 2.4): stream i applies n_i LCG advances, X <- A^(n_i) X, without
 * producing output; its read position is unchanged.  n128: n_streams pairs of uint64
 * (low word first), host or device; n_i < 2^128.  Computed by square-and-multiply over
 * the 4-bit-window power table (at most 32 modular products per stream). */
rlxpp_status rlxpp_skip(rlxpp_gen* gen, const uint64_t* n128, void* cuda_stream);

/* Draw 24-bit integers (Sec. 2.4, IntRndm) into uint32 out.
 *  counts == NULL: every stream draws count_each values; stream i writes
 *                  out[i * count_each + k], k < count_each (offsets ignored).
 *  counts != NULL: stream i draws counts[i] >= 0 values to out[offsets[i] + k];
 *                  counts and offsets are n_streams int64 each, host or device, and
 *                  the output ranges must not overlap.
 * out: host or device. */
rlxpp_status rlxpp_draw_u24(rlxpp_gen* gen, const int64_t* counts, const int64_t* offsets,
                            int64_t count_each, uint32_t* out, void* cuda_stream);

/* Draw doubles in [0, 1) with 48 random bits each (Sec. 2.3, Rndm); same layout rules
 * as rlxpp_draw_u24. */
rlxpp_status rlxpp_draw_f64(rlxpp_gen* gen, const int64_t* counts, const int64_t* offsets,
                            int64_t count_each, double* out, void* cuda_stream);

/* Asynchronous draws into page-locked host memory (the values of rlxpp_draw_u24 and
 * rlxpp_draw_f64 with one count for all streams: row i of out holds stream i's
 * count_each values).  The values are computed on cuda_stream into a device staging
 * buffer that the handle owns and copied to out on the handle's internal copy stream;
 * the call returns once the work is queued.  The streams advance in cuda_stream's
 * order, so later calls on that stream (device draws, skips) run without waiting for
 * the copies.  out is complete once a stream made to wait by rlxpp_host_wait has
 * reached that point; until then out must stay allocated and untouched.  A later
 * asynchronous draw reuses the staging buffer after the earlier copies (in stream
 * order, no host wait).  RLXPP_ERR_INVALID when out is not page-locked host memory. */
rlxpp_status rlxpp_draw_u24_host_async(rlxpp_gen* gen, int64_t count_each, uint32_t* out,
                                       void* cuda_stream);
rlxpp_status rlxpp_draw_f64_host_async(rlxpp_gen* gen, int64_t count_each, double* out,
                                       void* cuda_stream);

/* Makes cuda_stream wait (on the device, without blocking the host) until the copies of
 * every asynchronous host draw issued so far on this handle have completed. */
rlxpp_status rlxpp_host_wait(rlxpp_gen* gen, void* cuda_stream);

/* Draw single-precision floats in [0, 1): one RANLUX number w each, w 2^-24 (exact in
 * binary32; the 24-bit output RANLUX itself delivers, Sec. 1); float out, same layout
 * rules as rlxpp_draw_u24. */
rlxpp_status rlxpp_draw_f32(rlxpp_gen* gen, const int64_t* counts, const int64_t* offsets,
                            int64_t count_each, float* out, void* cuda_stream);

/* Draw standard Gaussian doubles (the distributions ROOT builds on Rndm, Sec. 2.4), by
 * the Box-Muller transform (Box and Muller, Ann. Math. Statist. 29, 1958) on
 * consecutive pairs (d_a, d_b) of the stream's doubles (the rlxpp_draw_f64 sequence):
 * u1 = 1 - d_a in (0, 1], r = sqrt(-2 ln u1), then r cos(2 pi d_b) and r sin(2 pi d_b).
 * n values take 2 ceil(n / 2) doubles (an odd count drops its last sine), so afterwards
 * the stream stands where rlxpp_draw_f64 of 2 ceil(n / 2) values would leave it.  ln,
 * sqrt, sin and cos are the library's own fixed-point routines on the 48-bit integers
 * (table-driven log, Taylor series, Newton's iteration for 1/sqrt): each value is within
 * half a unit in the last place plus 2^-56 r of the exact transform of its pair.
 * double out, same layout rules as rlxpp_draw_u24 (count = normals per stream). */
rlxpp_status rlxpp_draw_normal_f64(rlxpp_gen* gen, const int64_t* counts, const int64_t* offsets,
                                   int64_t count_each, double* out, void* cuda_stream);

/* Draw exponential doubles with rate 1 (another of the distributions ROOT builds on
 * Rndm, Sec. 2.4) by inversion: x = -ln(1 - d) for each double d of the stream (the
 * rlxpp_draw_f64 sequence; 1 - d in (0, 1], d = 0 gives +0).  ln is the library's own
 * fixed-point table-driven logarithm of the 48-bit integer 2^48 - v: each value is
 * within half a unit in the last place plus 2^-60 x of the exact one.  double out, same
 * layout rules as rlxpp_draw_u24; the stream moves as rlxpp_draw_f64 of the same count
 * would move it. */
rlxpp_status rlxpp_draw_exp_f64(rlxpp_gen* gen, const int64_t* counts, const int64_t* offsets,
                                int64_t count_each, double* out, void* cuda_stream);

/* Draw raw LCG doubles, for comparison only (Sec. 2.3 names this form, Sibidanov's,
 * only to replace it by the RANLUX numbers: its top bits lean towards 0 because the
 * state is below m).  Each refill gives 11 values v_k 2^-52 with
 * v_k = (X >> 52 k) mod 2^52, k = 0 .. 10, of the new LCG state X, low bits first (the
 * top 4 bits of X are not used).  A stream's draw of n values starts with a refill
 * (the unread part of its current block is skipped), takes ceil(n / 11) refills, drops
 * the values of the last one past n and leaves the stream at the end of that block
 * (read position 24); n = 0 leaves it unchanged.  Runs on the integer pipe on every
 * path.  double out, same layout rules as rlxpp_draw_u24. */
rlxpp_status rlxpp_draw_raw_f64(rlxpp_gen* gen, const int64_t* counts, const int64_t* offsets,
                                int64_t count_each, double* out, void* cuda_stream);

/* Skip random numbers without generating them (Sec. 2.4), counted in values of one
 * kind: stream i moves exactly as if it had drawn n_values[i] values of `kind`
 * (RLXPP_KIND_U24, RLXPP_KIND_F64 or RLXPP_KIND_F32) and discarded them: the rest of
 * its current block, then whole blocks by X <- A^blocks X over the power table.
 * n_values: n_streams uint64, host or device. */
rlxpp_status rlxpp_skip_values(rlxpp_gen* gen, const uint64_t* n_values, uint32_t kind,
                               void* cuda_stream);

/* Fused consumer (the GPU benchmark of Sec. 4.2 sums every number a thread draws):
 * every stream draws count_each doubles without storing them.  sums (NULL or
 * n_streams uint64, device) receives, per stream, the exact sum of the 48-bit
 * integers v behind its doubles (double = v 2^-48); hist (device, 256 uint64) is
 * incremented at bin v >> 40 for every value.  hist is accumulated, not cleared. */
rlxpp_status rlxpp_draw_f64_sum_hist(rlxpp_gen* gen, int64_t count_each, uint64_t* sums,
                                     uint64_t* hist, void* cuda_stream);

/* ---- batched requests (uneven counts, mixed levels and kinds, sequence splitting) ----
 * A request draws `count` values of one kind from one stream, starting `skip` LCG
 * advances after the stream's current state, at read position `pos` of that block
 * (pos = the stream's own position with skip = 0 continues it exactly; rlxpp_get_state
 * reports positions).  Requests are independent: several may name the same stream
 * (each reads its own part of the sequence) and none needs another to finish first.
 *
 * The library splits every request into chunks of at most L refills and starts each
 * chunk from its own block by jump-ahead (X <- A^b X over the power table, Sec. 2.4),
 * so a long request runs on many threads; chunks are ordered longest first and taken
 * from a device work queue by one persistent kernel for all luxury levels together.
 * L, the product kernel, the threads per stream and the grid are chosen by the
 * handle's tuner (rlxpp_autotune_requests) or by defaults. */
#define RLXPP_KIND_U24 0u
#define RLXPP_KIND_F64 1u
#define RLXPP_KIND_F32 2u /* rlxpp_skip_values only; requests take u24 and f64 */
#define RLXPP_REQ_ADVANCE 1u /* flag: move each stream to the end of its request (at most
                                one request per stream); otherwise states are unchanged */

typedef struct rlxpp_request {
  uint64_t stream; /* stream index < n_streams                                       */
  uint64_t skip;   /* LCG advances (blocks) between the current state and the start  */
  uint32_t pos;    /* numbers of the start block already consumed, 0..24             */
  uint32_t kind;   /* RLXPP_KIND_U24 (uint32 out) or RLXPP_KIND_F64 (double out)       */
  int64_t count;   /* values to draw, >= 0                                           */
  uint64_t offset; /* index of the first value in out_u24 or out_f64 (by kind)       */
} rlxpp_request;   /* 40 bytes */

typedef struct rlxpp_tuning {
  uint32_t chunk_blocks;  /* L: refills per chunk, >= 2                                  */
  uint32_t blocks_per_sm; /* persistent grid = blocks_per_sm x SMs blocks, 1..8        */
  uint32_t path;          /* which kernel runs the chunks (paths defined below):
                             RLXPP_PATH_IMAD: one thread per chunk, integer pipe;
                             RLXPP_PATH_TENSOR: one thread per chunk, 128-chunk tiles
                             on the tensor cores (4 CTAs per SM at most); a request of
                             at least 32 L blocks is cut into warps of 32 strided
                             chunks (lane t of a warp draws every 32nd block from its
                             own, by products with A^32), whose blocks leave as one
                             contiguous run per warp and refill;
                             RLXPP_PATH_WARP: 32 threads per chunk (one warp, one limb
                             per lane), for few long chunks.  The path also fixes the
                             limb width of the product: 32-bit limbs on the integer
                             pipe (IMAD, WARP), 8-bit limbs in the tensor product     */
  uint32_t threads_per_block; /* block shape: threads per CTA, 0 = the path's default
                             (128); IMAD and WARP take 64, 128 or 256, TENSOR only 128
                             (one 128-row tile per CTA); blocks_per_sm x
                             threads_per_block <= 2048                                  */
} rlxpp_tuning;

typedef struct rlxpp_plan rlxpp_plan;

/* Plan requests (host array reqs[n_reqs]): validates them (stream < n_streams,
 * pos <= 24, kind, count >= 0, skip + refills < 2^64, no stream twice with
 * RLXPP_REQ_ADVANCE), splits them into chunks and uploads the work list to device
 * memory owned by the plan.  tuning: NULL = the handle's tuned choice for requests of
 * this shape, else the defaults (the handle's path).  Synchronous; the plan belongs
 * to `gen`. */
rlxpp_status rlxpp_plan_requests(rlxpp_gen* gen, const rlxpp_request* reqs, uint64_t n_reqs,
                                 uint32_t flags, const rlxpp_tuning* tuning, rlxpp_plan** out);

/* Run a plan: out_u24 / out_f64 are device arrays large enough for every request's
 * offset + count of its kind (NULL allowed when no request has that kind).  Issues
 * one kernel launch on cuda_stream (two with RLXPP_REQ_ADVANCE: a snapshot of the
 * requested streams' states first), no allocation and no host synchronisation, so it
 * can be captured in a CUDA graph and replayed; every run recomputes the same values
 * unless RLXPP_REQ_ADVANCE moved the streams.  The plan's work counters are reset by
 * the kernel itself at its end, so runs of one plan must not overlap on the device
 * (run them on one stream, or wait between them). */
rlxpp_status rlxpp_run_plan(rlxpp_gen* gen, const rlxpp_plan* plan, uint32_t* out_u24,
                            double* out_f64, void* cuda_stream);

/* Work items (chunks) of a plan, and its tuning. */
uint64_t rlxpp_plan_items(const rlxpp_plan* plan);
rlxpp_tuning rlxpp_plan_tuning(const rlxpp_plan* plan);

void rlxpp_destroy_plan(rlxpp_plan* plan);

/* plan + run + destroy in one call; the work list is allocated, uploaded and freed in
 * order on cuda_stream (no device-wide synchronisation), and the host request array may
 * be reused when the call returns. */
rlxpp_status rlxpp_draw_requests(rlxpp_gen* gen, const rlxpp_request* reqs, uint64_t n_reqs,
                                 uint32_t* out_u24, double* out_f64, uint32_t flags,
                                 void* cuda_stream);

/* Tuner: times candidate (kernel, chunk length, block shape, grid) choices on these
 * requests (the integer-pipe kernel with one thread or one warp per chunk, and the
 * tensor-core kernel, i.e. threads per stream, limb width and product; 64, 128 or 256
 * threads per CTA where the kernel allows it; without RLXPP_REQ_ADVANCE, so the
 * streams do not move; the outputs are overwritten) and keeps the fastest for requests of the same shape (log2 buckets of the request count
 * and of the total refills).  The choice is kept in the handle and, when the
 * environment variable RLXPP_TUNE_CACHE names a file, appended there and read back
 * by later handles on the same device model.  best may be NULL. */
rlxpp_status rlxpp_autotune_requests(rlxpp_gen* gen, const rlxpp_request* reqs, uint64_t n_reqs,
                                     uint32_t* out_u24, double* out_f64, void* cuda_stream,
                                     rlxpp_tuning* best);

/* Export / import the state of every stream (Sec. 4.2: the state is plain memory that
 * can move between host and device and continue the same sequence).  dst/src:
 * n_streams records, host or device.  Import checks each record on the device:
 * carry <= 1, pos <= 24, p one of the handle's levels, reserved == 0, and (d, carry)
 * must be the RANLUX form of an LCG state X with 0 < X < m, i.e. converting
 * X = d - floor(d / 2^336) + carry back gives the same record (every state the
 * recurrence reaches after 24 steps, and every exported state, has this form).  A bad
 * record leaves its stream unchanged and sets a sticky RLXPP_ERR_INVALID reported by
 * rlxpp_sync(). */
rlxpp_status rlxpp_get_state(const rlxpp_gen* gen, rlxpp_state* dst, void* cuda_stream);
rlxpp_status rlxpp_set_state(rlxpp_gen* gen, const rlxpp_state* src, void* cuda_stream);

/* Wait for the handle's work on cuda_stream and return (and clear) the sticky device
 * status: RLXPP_OK, RLXPP_ERR_INVALID or RLXPP_ERR_TIMEOUT. */
rlxpp_status rlxpp_sync(rlxpp_gen* gen, void* cuda_stream);

/* ---- refill path -------------------------------------------------------------------
 * RLXPP_PATH_IMAD: the product on the integer pipe, one thread per stream.
 * RLXPP_PATH_TENSOR (the default): the product A X mod m as an exact-integer fp16
 * matrix product on
 * the tensor cores (tcgen05.mma, fp32 accumulation in tensor memory): with
 * R_j = A 2^(8j) mod m, A X = sum_j x_j R_j = sum_k S_k 2^(8k) (mod m) where x_j are
 * the 72 bytes of X and S_k = sum_j x_j byte_k(R_j) < 2^23, so a tile of 128 streams is
 * one 128 x 80 x 80 product per refill (Sec. 2.1-2.2 computed differently, same
 * result).  It serves the plain draws of single-level handles (a tile's streams share
 * one multiplier; plain draws of multi-level handles use the integer kernel) and the
 * batched requests of the handle (chunks are grouped by level into tiles).
 * RLXPP_PATH_WARP: the plain draws (u24, f32, f64, fused sum/histogram) with one warp
 * per stream, lane l holding limb l, every multi-limb sum's carries resolved across the
 * warp at once: for few streams, where the latency of one refill counts (a single
 * stream read in order); Gaussian and exponential draws of such a handle use the
 * integer kernels, and its batched requests (without a tuning) one warp per chunk.  All
 * paths give bit-identical results.  Synchronises the device. */
#define RLXPP_PATH_IMAD 0u
#define RLXPP_PATH_TENSOR 1u
#define RLXPP_PATH_WARP 2u
rlxpp_status rlxpp_set_path(rlxpp_gen* gen, uint32_t path);
uint32_t rlxpp_get_path(const rlxpp_gen* gen);

/* Number of streams of the handle. */
uint64_t rlxpp_num_streams(const rlxpp_gen* gen);

/* Message for the calling thread's last failed call ("" if none). */
const char* rlxpp_last_error(void);

/* Release the handle and its device memory (synchronises the device first). */
void rlxpp_destroy(rlxpp_gen* gen);

/* ---- seeding without device allocation --------------------------------------------
 * The paper has no counterpart of this entry point.  It serves callers that must not
 * allocate device memory themselves or through this library: code that runs inside a
 * host application which owns the whole device-memory budget (a fixed pool carved out
 * at start-up), code on a latency-critical path where cudaMalloc/cudaFree would stall
 * on an implicit device synchronisation, and code that may not create a handle
 * (rlxpp_create allocates the resident state and the tables).
 *
 * It writes the seeded state of n_streams streams — exactly the records rlxpp_create
 * followed by rlxpp_get_state would give — into caller-owned records, which the caller
 * can keep, copy or import with rlxpp_set_state.
 *  levels[n_levels]  host array of luxury levels p >= 1, 1 <= n_levels <=
 *                    RLXPP_NOALLOC_MAX_LEVELS; more levels are rejected with
 *                    RLXPP_ERR_INVALID.
 *  level_of_stream   NULL (all streams at levels[0]) or n_streams bytes, device memory;
 *                    a stream whose index is >= n_levels gets an all-zero record
 *                    (p = 0 marks it invalid).
 *  seeds             n_streams uint64, device memory; a zero seed (seeds start at 1)
 *                    also gets an all-zero record.
 *  out               n_streams records, device memory.
 * Host pointers are rejected (staging them would allocate).
 *
 * Scratch: the multiplier and the power table of each level are computed on the
 * device, at every call, into one fixed array of the library (184,608 bytes, room for
 * RLXPP_NOALLOC_MAX_LEVELS levels) that every GPU loading the library holds until the
 * process exits.  The call allocates nothing (no cudaMalloc, cudaFree or allocating
 * library routine).  Every call looks up the array's device address in the current
 * device's context (cudaGetSymbolAddress, a host query), so a context reset between
 * calls is harmless; the first lookup in a context may load the library's device
 * code, which a stream capture does not allow, so make one call outside any capture
 * first (after a cudaDeviceReset too).  Device memory of another GPU is rejected with
 * RLXPP_ERR_INVALID.  All calls share the array and it keeps the last call's contents:
 * calls that overlap on the GPU (on different streams or from different threads) race
 * and must be serialised by the caller.  Each call costs the table set-up of its
 * levels (a few short kernels per level) plus one seeding kernel. */
#define RLXPP_NOALLOC_MAX_LEVELS 4
rlxpp_status rlxpp_seed_states_noalloc(const uint32_t* levels, uint32_t n_levels,
                                       const uint8_t* level_of_stream, const uint64_t* seeds,
                                       uint64_t n_streams, rlxpp_state* out, void* cuda_stream);

/* ---- unit-test entry points (device arithmetic on n independent items) ----------
 * Numbers are little-endian arrays of uint64 limbs, item-major; all pointers are
 * device pointers and n may be 0.
 *  rlxpp_test_multiply9x9  x[9], y[9] -> out[18] = x * y              (Sec. 2.1)
 *  rlxpp_test_mod_m        in[18]     -> out[9]  = in mod m, in [0, m) (Sec. 2.2)
 *  rlxpp_test_mul_mod      x[9], y[9] -> out[9]  = x y mod m; x, y < 2^576
 *  rlxpp_test_to_ranlux    x[9] (< m) -> d[9] = floor(2^576 x / m), carry[1] (Sec. 2.3)
 *  rlxpp_test_to_lcg       d[9], carry[1] -> x[9] = d - floor(d / 2^336) + carry
 *  rlxpp_test_f64_from48   v[1] (< 2^48) -> out[1] = bit pattern of v 2^-48
 * The same two steps as the warp-cooperative refill computes them (one warp per item,
 * one 32-bit limb per lane), same layouts:
 *  rlxpp_test_warp_mod_m     in[18] -> out[9] = in mod m, in [0, m)      (Sec. 2.2)
 *  rlxpp_test_warp_to_ranlux x[9] (< m) -> d[9], carry[1]                 (Sec. 2.3)
 * The integer-pipe elementary functions under the distribution draws (Sec. 2.4); each
 * output is a double's bit pattern, a quiet NaN for an input out of range:
 *  rlxpp_test_neg_ln48       w[1] in [1, 2^48] -> out[1] = -ln(w 2^-48)
 *  rlxpp_test_cos_sin_2pi48  v[1] (< 2^48)     -> out[2] = cos, sin of 2 pi v 2^-48
 *  rlxpp_test_box_muller48   v[2] (< 2^48)     -> out[2] = r cos 2 pi d_b, r sin 2 pi d_b with
 *                            r = sqrt(-2 ln(1 - d_a)), d = v 2^-48 */
rlxpp_status rlxpp_test_multiply9x9(const uint64_t* x, const uint64_t* y, uint64_t* out,
                                    uint64_t n, void* cuda_stream);
rlxpp_status rlxpp_test_mod_m(const uint64_t* in, uint64_t* out, uint64_t n, void* cuda_stream);
rlxpp_status rlxpp_test_mul_mod(const uint64_t* x, const uint64_t* y, uint64_t* out,
                                uint64_t n, void* cuda_stream);
rlxpp_status rlxpp_test_to_ranlux(const uint64_t* x, uint64_t* d, uint32_t* carry,
                                  uint64_t n, void* cuda_stream);
rlxpp_status rlxpp_test_to_lcg(const uint64_t* d, const uint32_t* carry, uint64_t* x,
                               uint64_t n, void* cuda_stream);
rlxpp_status rlxpp_test_f64_from48(const uint64_t* v, uint64_t* out, uint64_t n,
                                   void* cuda_stream);
rlxpp_status rlxpp_test_warp_mod_m(const uint64_t* in, uint64_t* out, uint64_t n, void* cuda_stream);
rlxpp_status rlxpp_test_warp_to_ranlux(const uint64_t* x, uint64_t* d, uint32_t* carry, uint64_t n,
                                       void* cuda_stream);
rlxpp_status rlxpp_test_neg_ln48(const uint64_t* w, uint64_t* out, uint64_t n, void* cuda_stream);
rlxpp_status rlxpp_test_cos_sin_2pi48(const uint64_t* v, uint64_t* out, uint64_t n,
                                      void* cuda_stream);
rlxpp_status rlxpp_test_box_muller48(const uint64_t* v, uint64_t* out, uint64_t n,
                                     void* cuda_stream);

/* One tensor-path product per item: out[9] = A x mod m for luxury p (x < m, device
 * arrays of 9 uint64 limbs per item); synchronous. */
rlxpp_status rlxpp_test_tc_mulmod(uint32_t p, const uint64_t* x, uint64_t* out, uint64_t n,
                                  void* cuda_stream);

/* Failure-path test: runs one tensor-path tile whose MMA is never issued, so its
 * bounded mbarrier wait (about 2^22 polls) must give up; returns RLXPP_ERR_TIMEOUT
 * when the kernel reported the timeout and left the context usable.  scratch: 9
 * uint64 of device memory (not written). */
rlxpp_status rlxpp_test_tc_timeout(uint64_t* scratch, void* cuda_stream);

/* ---- serving loop (host side, native) -------------------------------------------
 * A continuous-batching request loop over the streams of one generator.  Each
 * submitted request (count u24 or f64 values from one stream) is given the next
 * segment of its stream at once (start block and read position by the draw rule), so
 * requests run independently by jump-ahead; it is admitted when its output fits a
 * device arena of pool_bytes (first fit in 256-byte granules), launched with what else
 * is admitted (up to max_batch) as one rlxpp_draw_requests batch on one of
 * n_cuda_streams streams while earlier batches run, copied (RLXPP_SERVER_COPY_TO_HOST)
 * to a page-locked mirror of the arena, the batch's requests below small_bytes first,
 * and completed when its copy has finished.  With max_queued_bytes > 0 a request that
 * would push the bytes waiting for the arena past it, or one larger than the arena,
 * is rejected (accepted = 0) and takes no numbers from its stream.  A request not yet
 * launched can be cancelled; its segment of the stream is then skipped.  Times are
 * seconds from the server's creation (or from the start of rlxpp_server_run_trace).
 * The generator must outlive the server; a server is not thread-safe. */
typedef struct rlxpp_server rlxpp_server;
#define RLXPP_SERVER_COPY_TO_HOST 1u /* copy each result to the page-locked mirror       */
#define RLXPP_SERVER_KEEP_RESULTS 2u /* keep a copy of each result for rlxpp_server_result */
typedef struct rlxpp_served {        /* one completed request                          */
  uint64_t rid, stream, skip;        /* id; stream; start block (advances from the state) */
  uint32_t pos, kind;                /* read position in the start block; RLXPP_KIND_*  */
  int64_t count;                     /* values                                          */
  uint64_t offset, nbytes;           /* byte offset in the arena; bytes of output       */
  double arrival, launch, done;      /* seconds                                         */
} rlxpp_served;                      /* 80 bytes */
typedef struct rlxpp_server_state {
  uint64_t waiting, admitted, inflight_groups, arena_used, queued_bytes, done, rejected, cancelled;
  uint64_t max_launch_us;  /* longest host time of one batch launch, microseconds      */
  uint64_t slow_launches;  /* batch launches that took 1 ms or more on the host         */
  /* Device-side times of completed batches, from CUDA events recorded on the batch's
   * stream: "kernel" = from the batch's first operation to the end of its request
   * kernel, "copy" = from there to the end of its last device-to-host copy.  A latency
   * excursion whose batches show long copy times was spent on the link; one with
   * short device times was spent waiting on the host. */
  uint64_t batches_timed;                 /* completed batches with device times       */
  uint64_t kernel_us_sum, kernel_us_max;  /* microseconds                              */
  uint64_t copy_us_sum, copy_us_max;      /* microseconds                              */
} rlxpp_server_state;
rlxpp_status rlxpp_server_create(rlxpp_gen* gen, uint64_t pool_bytes, uint32_t n_cuda_streams,
                                 uint32_t max_batch, uint64_t small_bytes, uint64_t max_queued_bytes,
                                 uint32_t flags, rlxpp_server** out);
void rlxpp_server_destroy(rlxpp_server* server);
/* arrival < 0: now.  The id must not belong to a request that is pending or not yet
 * taken by rlxpp_server_take_done. */
rlxpp_status rlxpp_server_submit(rlxpp_server* server, uint64_t rid, uint64_t stream, uint32_t kind,
                                 int64_t count, double arrival, int* accepted);
rlxpp_status rlxpp_server_cancel(rlxpp_server* server, uint64_t rid, int* cancelled);
/* One round: retire finished copies, admit, launch (wait_for_one: first wait on the
 * host for the oldest batch's next copy group).  rlxpp_server_drain runs rounds until
 * nothing is waiting, admitted or in flight. */
rlxpp_status rlxpp_server_pump(rlxpp_server* server, int wait_for_one);
rlxpp_status rlxpp_server_drain(rlxpp_server* server);
rlxpp_status rlxpp_server_stats(const rlxpp_server* server, rlxpp_server_state* out);
/* Up to max completed requests in completion order (each once) into out; *n = count. */
rlxpp_status rlxpp_server_take_done(rlxpp_server* server, rlxpp_served* out, uint64_t max, uint64_t* n);
/* The kept result of a completed request (RLXPP_SERVER_KEEP_RESULTS): nbytes must be its
 * size; the copy is released. */
rlxpp_status rlxpp_server_result(rlxpp_server* server, uint64_t rid, void* dst, uint64_t nbytes);
/* Replays a trace on an idle server: request i (id i) of count[i] values (f64 if
 * is_f64[i], else u24) from stream[i] is submitted once arrival[i] seconds have passed;
 * latency[i] receives its completion minus its arrival in seconds, -1 if rejected.  The
 * launch and device times of rlxpp_server_stats start again from zero at each call. */
rlxpp_status rlxpp_server_run_trace(rlxpp_server* server, uint64_t n, const double* arrival,
                                    const uint64_t* stream, const int64_t* count, const uint8_t* is_f64,
                                    double* latency);

/* Failure-path test: the library's device allocation number `after` from now (0 = the
 * next one) reports out of memory without allocating, once; after < 0 switches this
 * off.  Process-wide (one countdown shared by all threads and handles).  Calls that hit
 * it return RLXPP_ERR_NOMEM and release what they had allocated; a handle whose call
 * failed keeps its previous state. */
rlxpp_status rlxpp_test_fail_alloc(int64_t after);

/* Luxury multiplier A = a^p mod m as 9 uint64 limbs written to host memory out9,
 * computed on the device (Sec. 1: RANLUX as an LCG with a large multiplier). */
rlxpp_status rlxpp_luxury_multiplier(uint32_t p, uint64_t* out9);

#ifdef __cplusplus
}
#endif

#endif /* RLXPP_H */
