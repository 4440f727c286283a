/*
 * sws.h -- C ABI of a GB300 (sm_103a) library for sliding window sums and the minimizer
 * pipeline built on them, after R. Snytsar and Y. Turakhia, "Parallel approach to sliding
 * window sums" (arXiv 1811.10074).
 *
 * General rules for every entry point:
 *   - Data pointers are DEVICE pointers owned by the caller unless stated otherwise; the
 *     library never frees or keeps them.  Outputs are preallocated by the caller.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls
 *     are asynchronous on it: inputs must stay valid and outputs untouched until the stream
 *     reaches the call.
 *   - Every call returns an sws_status.  Nothing aborts, exits or traps.  Argument errors are
 *     reported before any work is queued.  Faults found on the device (a bounded wait that ran
 *     out) are recorded in the context and reported by sws_sync().
 *   - A context owns the device workspace that some calls need (tile status words for ordered
 *     output).  One context may be used from one host thread at a time; calls that use the
 *     workspace must not overlap on the device (use one context per concurrent stream).
 *   - Lengths are element counts (bases for DNA).  DNA is 2-bit packed: A=0 C=1 G=2 T=3, base
 *     i in byte i>>2 at bits 2*(i&3); a sequence of n bases occupies ceil(n/4) bytes.
 */
#ifndef SWS_H
#define SWS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status ------------------------------------------------------------------------------ */
typedef int sws_status;
#define SWS_OK 0
#define SWS_ERR_INVALID 1     /* bad argument (message in sws_last_error)                   */
#define SWS_ERR_OOM 2         /* the context workspace could not be grown                  */
#define SWS_ERR_CAPACITY 3    /* more results than the caller's capacity (count still exact) */
#define SWS_ERR_CUDA 4        /* a CUDA runtime call failed                                 */
#define SWS_ERR_TIMEOUT 5     /* a bounded device-side wait ran out; results are invalid     */
#define SWS_ERR_UNSUPPORTED 6 /* valid but outside what this build implements               */

/* Thread-local description of the last error of this thread (never NULL). */
const char *sws_last_error(void);

/* ---- context ----------------------------------------------------------------------------- */
typedef struct sws_ctx sws_ctx;

/* Create a context on CUDA device `device` (made current on the calling thread). */
sws_status sws_create(sws_ctx **out, int device);
/* Destroy a context; waits for the device first.  NULL is accepted. */
sws_status sws_destroy(sws_ctx *ctx);
/* Grow the workspace to at least `bytes` now (so that later calls, e.g. under stream
 * capture, allocate nothing).  Returns SWS_ERR_OOM if it cannot. */
sws_status sws_reserve(sws_ctx *ctx, uint64_t bytes);
/* Wait for `stream`, then report (and clear) any device-side fault recorded by this
 * context's kernels: SWS_ERR_TIMEOUT if a bounded wait ran out. */
sws_status sws_sync(sws_ctx *ctx, void *stream);

/* ---- sliding window sum (Eq. 2, Sec. 2.2) ---------------------------------------------- */
/* Operators.  Element layouts:
 *   SWS_OP_ADD_I32    int32, addition mod 2^32
 *   SWS_OP_MIN_I32    int32, signed minimum
 *   SWS_OP_MAX_I32    int32, signed maximum
 *   SWS_OP_XOR_I32    int32, bitwise xor
 *   SWS_OP_AFFINE_U32 pair {uint32 a, uint32 b} (8 bytes) = map x -> a*x+b mod 2^32; the sum
 *                     x_p (+) x_{p+1} is the map "apply x_p, then x_{p+1}" (not commutative)
 *   SWS_OP_ADD_F32    float, addition (results are fp32; not bit-reproducible across variants) */
#define SWS_OP_ADD_I32 0
#define SWS_OP_MIN_I32 1
#define SWS_OP_MAX_I32 2
#define SWS_OP_XOR_I32 3
#define SWS_OP_AFFINE_U32 4
#define SWS_OP_ADD_F32 5

/* Algorithm variants. */
#define SWS_VARIANT_AUTO 0          /* the variant sws_tune_sliding_sum chose for (op, w), else the
                                       library's rule (block combine: in registers for w <= 8,
                                       warp-private or CTA streams on large inputs, one-shot tiles
                                       otherwise)                                                  */
#define SWS_VARIANT_BLOCK_COMBINE 1 /* blocks of w: in-block suffix + next-block prefix, O(1)/output;
                                       one-shot CTA tiles                                          */
#define SWS_VARIANT_DOUBLING 2      /* ceil(log2 w) doubling levels, O(log w)/output            */
#define SWS_VARIANT_PREFIX_DIFF 3   /* y_p = S_{p+w-1} - S_{p-1}; ADD_I32 and XOR_I32 only      */
#define SWS_VARIANT_BLOCK_COMBINE_STREAM 4 /* block combine in a persistent kernel fed by 2-D TMA
                                       copies; needs w = c*m with c = 16 (int32/fp32) or 8 (affine)
                                       and m in {1,2,4,8,16,32} or a multiple of 32 (w <= 4096 int32,
                                       <= 2048 affine), a 16-byte aligned input of at least 128
                                       bytes, else SWS_ERR_UNSUPPORTED.  A copy that never completes within
                                       about a second sets the context's error word (reported by
                                       sws_sync as SWS_ERR_TIMEOUT).                               */
#define SWS_VARIANT_BLOCK_COMBINE_WARP 5 /* block combine in warp-private streams (each warp walks its
                                       own run of 2 KB tiles fed by 2-D TMA copies; no CTA barrier,
                                       no halo); needs w = c*G with c = 16 (int32/fp32) or 8 (affine)
                                       and G in {1,2,4,8,16,32}, and the input as for _STREAM, else
                                       SWS_ERR_UNSUPPORTED.  Time-outs as for _STREAM.              */

/* Failure detection self-test (no counterpart in the paper).  Queues one warp that runs one of
 * the library's bounded device-side waits against a flag that nothing ever sets:
 *   which = 0 : the look-back poll (a predecessor tile whose status word stays zero);
 *   which = 1 : an mbarrier wait for 16 bytes of a TMA copy that is never issued.
 * The wait gives up after about a second, records the time-out in the context's error word and
 * returns; the next sws_sync on that stream returns SWS_ERR_TIMEOUT (and clears the word) and the
 * context stays usable.  Nothing faults, traps or hangs.  which outside {0, 1}: SWS_ERR_INVALID. */
sws_status sws_selftest_wait_timeout(sws_ctx *ctx, int which, void *stream);

/* Failure self-test of the ordered minimizer output (no counterpart in the paper).  Runs the
 * single-kernel (look-back) minimizer path -- the path sws_minimizers takes for small inputs and
 * sws_minimizers_noalloc always takes -- with k = 15, w = 10 over three tiles of a zeroed scratch
 * sequence in the context's workspace, its staging copies announced on the tiles' mbarriers but
 * never issued, so every tile's bounded copy wait runs out.  count_out (device uint64) is set to
 * all ones when the call is queued and must stay all ones: a tile whose input never arrived
 * publishes a failure in place of its count, every later tile then fails in turn, and no tile
 * writes the total.  The next sws_sync returns SWS_ERR_TIMEOUT and the context stays usable.
 * Takes about a second on the device; nothing faults, traps or hangs. */
sws_status sws_selftest_minimizer_timeout(sws_ctx *ctx, uint64_t *count_out, void *stream);

#define SWS_VARIANT_COUNT 6

/* Autotuner for the sliding sum: on a scratch input of n elements (a fixed pseudo-random pattern
 * in the context's workspace), after warming the GPU up with at least 10 ms of work, times the
 * library's fixed rule and every variant that applies to (op, w) -- the warp-private variant in
 * each of its run shapes -- (best of five launches on `stream`, CUDA events), and remembers for
 * (op, w) the fastest if it beats the rule by more than 2% (else the rule): later
 * SWS_VARIANT_AUTO calls with this op and w and at least n/8 elements use it.  Blocks until the
 * timing is done.  Timings taken under a profiler that serialises launches are not meaningful.
 *   variant_out : optional, the chosen SWS_VARIANT_* (SWS_VARIANT_AUTO: the rule stays).
 *   ms_out      : optional, SWS_VARIANT_COUNT floats: milliseconds per variant (index 0: the
 *                 rule), -1 where a variant does not apply.
 * Uses workspace (2 n elements).  w too large for this build: SWS_ERR_UNSUPPORTED. */
sws_status sws_tune_sliding_sum(sws_ctx *ctx, int op, int w, uint64_t n, int *variant_out, float *ms_out,
                                void *stream);

/* Eq. 2: out[p] = in[p] (+) in[p+1] (+) ... (+) in[p+w-1] for p = 0 .. n-w (n-w+1 outputs,
 * exactly w addends each, Sec. 2.2).
 *   in, out : device arrays of n and n-w+1 elements of the operator's type; must not overlap;
 *             aligned to the element size (16-byte alignment enables vector access).
 *   n < w   : writes nothing and returns SWS_OK.   w < 1 or an unknown op: SWS_ERR_INVALID.
 * Uses no workspace. */
sws_status sws_sliding_sum(sws_ctx *ctx, int op, int w, const void *in, void *out, uint64_t n, int variant,
                           void *stream);

/* ---- k-mers (Sec. 2.4: a k-mer is the sliding sum of k bases under concatenation) --------- */
#define SWS_KMER_FWD 0       /* r_i..r_{i+k-1} as a base-4 number, first base most significant  */
#define SWS_KMER_RC 1        /* reverse complement of the same k bases                            */
#define SWS_KMER_CANONICAL 2 /* min(FWD, RC)                                                      */
#define SWS_KMER_HASH 3      /* Wang's 64-bit integer mix of CANONICAL, truncated to 2k bits after
                                every step (a bijection on [0, 4^k))                              */

/* Values of the n-k+1 k-mers of a packed sequence.  1 <= k <= 32.  out holds uint32 values
 * when 2k <= 32, else uint64.  n < k writes nothing. */
sws_status sws_kmers(sws_ctx *ctx, const uint8_t *seq, uint64_t n, int k, int kind, void *out, void *stream);

/* ---- minimizers (Sec. 2.4) ---------------------------------------------------------------- */
/* Keys a window's minimum is taken over (ties go to the leftmost k-mer, i.e. keys are
 * ordered by (value, position)). */
#define SWS_MINI_HASH 0      /* SWS_KMER_HASH values (the default; "hashed k-mers", Sec. 4)  */
#define SWS_MINI_CANONICAL 1 /* canonical k-mers                                          */
#define SWS_MINI_FWD 2       /* forward k-mers: lexicographic seeds as in the Fig. 2 example */

/* Minimizers of one packed sequence of n bases (n < 2^32).
 * For every window position p (w consecutive k-mers starting at p, Sec. 2.4) the least key
 * and its position are found; consecutive windows with the same pick store it once.
 *   nblocks   : device int64 pairs [start, end) of bases that are N, sorted and disjoint (may be
 *               NULL when n_nblocks = 0).  A window touching an N base is dropped and each
 *               N-free stretch is an independent sequence (no deduplication across N-blocks).
 *   hash_out  : key values, uint32 when 2k <= 32 else uint64; pos_out: uint32 k-mer starts.
 *               Picks come in increasing position.  At most `capacity` are written.
 *   count_out : device uint64 receiving the exact number of picks (also when > capacity:
 *               then only the first `capacity` picks are stored).
 *   Limits: 1 <= k <= 32, 1 <= w <= 4000.  Uses workspace (8 bytes per 4032 windows). */
sws_status sws_minimizers(sws_ctx *ctx, const uint8_t *seq, uint64_t n, int k, int w, int mode,
                          const int64_t *nblocks, uint64_t n_nblocks, void *hash_out, uint32_t *pos_out,
                          uint64_t capacity, uint64_t *count_out, void *stream);

/* Capacity query for sws_minimizers (Sec. 2.4): the exact number of picks sws_minimizers would
 * store for the same arguments, written to count_out (device uint64), without writing any pick.
 * The same kernels run in a counting mode (no staging area), so the count is exact; a capacity of
 * *count_out then suffices for sws_minimizers.  Errors and limits as for sws_minimizers.  Uses
 * workspace (about 12 bytes per 4000 windows). */
sws_status sws_minimizers_count(sws_ctx *ctx, const uint8_t *seq, uint64_t n, int k, int w, int mode,
                                const int64_t *nblocks, uint64_t n_nblocks, uint64_t *count_out, void *stream);

/* The seed table of a packed sequence in one call (Sec. 2.4, Fig. 1): its minimizers (as
 * sws_minimizers with the same k, w, mode and N-blocks), then the position table and pointer
 * table built from the (key, position) hits as sws_kmer_table does with hash_bits = 2k.
 *   sorted_hash/sorted_pos : device outputs of `capacity` entries (sorted_hash uint32 when
 *                            2k <= 32, else uint64): the hits sorted by key, positions ascending
 *                            within a key.  They also hold the unsorted hits while the table is
 *                            built, so no second hit array is allocated.
 *   bucket_offsets         : device uint64 [2^bucket_bits + 1], 0 <= bucket_bits <= min(2k, 32).
 *   count                  : HOST uint64 receiving the number of hits m.
 * The call waits for the minimizers to finish (the sort is sized by m) and then queues the sort on
 * `stream`; it returns with the sort still running.  m > capacity: *count = m, SWS_ERR_CAPACITY,
 * outputs undefined.  A bounded device-side wait that ran out while finding the minimizers:
 * SWS_ERR_TIMEOUT.  Uses workspace (about 16 bytes per hit, 24 when 2k > 32). */
sws_status sws_build_table(sws_ctx *ctx, const uint8_t *seq, uint64_t n, int k, int w, int mode,
                           const int64_t *nblocks, uint64_t n_nblocks, int bucket_bits, void *sorted_hash,
                           uint32_t *sorted_pos, uint64_t capacity, uint64_t *bucket_offsets, uint64_t *count,
                           void *stream);

/* Paper-equivalent task of Sec. 4: deduplicated sliding minimum, with (value, position) keys,
 * over a precomputed array of m uint32 key values (e.g. hashed 15-mers).  Outputs as for
 * sws_minimizers (key_out uint32).  1 <= w <= 4000, m < 2^32. */
sws_status sws_minimizers_from_keys(sws_ctx *ctx, const uint32_t *keys, uint64_t m, int w, uint32_t *key_out,
                                    uint32_t *pos_out, uint64_t capacity, uint64_t *count_out, void *stream);

/* Batched minimizers: nreads reads stored back to back in one packed stream, read r being
 * bases [base_offsets[r], base_offsets[r+1]) (device int64 array of nreads+1 entries,
 * non-decreasing, base_offsets[0] = 0, base_offsets[nreads] = total_bases, which is also passed
 * by value; total_bases < 2^32).  Every read is an independent sequence (Sec. 2.4 applied per
 * read); all reads are processed by one launch whose tiles span read boundaries.
 *   hash_out/pos_out : picks of all reads, read by read; positions are read-local.
 *   pick_offsets     : device uint64 [nreads+1]; read r's picks are
 *                      [pick_offsets[r], pick_offsets[r+1]); pick_offsets[nreads] = total.
 *   count_out        : device uint64, the exact total (only `capacity` picks are stored).
 * Same limits as sws_minimizers.  Uses workspace. */
sws_status sws_minimizers_batch(sws_ctx *ctx, const uint8_t *seq, const int64_t *base_offsets, uint64_t nreads,
                                uint64_t total_bases, int k, int w, int mode, void *hash_out, uint32_t *pos_out,
                                uint64_t capacity, uint64_t *pick_offsets, uint64_t *count_out, void *stream);

/* ---- batched minimizers in one captured graph (Sec. 2.4 per read) ------------------------- */
/* A reusable pipeline for batches of up to max_reads reads and max_bases bases with fixed k, w
 * and key mode.  All buffers are allocated at creation; sws_batch_run replays one captured CUDA
 * graph (one persistent minimizer launch plus its scan, gather and fix-up kernels) whatever the
 * size of the batch, reading the sizes from a device descriptor.  Results are those of
 * sws_minimizers_batch on the same reads.
 *   options: SWS_BATCH_DEFAULT takes the single-pass kernel for hashed k-mers with k <= 16 and
 *            4 <= w <= 17 (one launch: picks placed in order from per-tile counts), otherwise the
 *            staged path (the staged kernel for 4 <= w <= 256 and k <= 32, otherwise the generic
 *            kernel writing per-tile slots, then a scan and a gather); SWS_BATCH_TUNE times every
 *            applicable path, the single-kernel look-back path included, on a synthetic batch of
 *            the largest size and keeps the fastest (see sws_batch_io.tuned_ms);
 *            SWS_BATCH_LOOKBACK forces the look-back path.
 * One run may be in flight per object: sws_batch_run waits for the previous run to finish before
 * it overwrites the descriptor.  Use one object per concurrent stream. */
typedef struct sws_batch sws_batch;
#define SWS_BATCH_DEFAULT 0
#define SWS_BATCH_TUNE 1
#define SWS_BATCH_LOOKBACK 2
typedef struct sws_batch_io {
  uint8_t *seq;            /* device input: packed bases of the reads back to back, >= max_bases */
  int64_t *offsets;        /* device input: read r = bases [offsets[r], offsets[r+1]), max_reads+1 */
  void *hash;              /* device output: pick keys (uint32 when 2k <= 32, else uint64)      */
  uint32_t *pos;           /* device output: read-local pick positions                          */
  uint64_t *pick_offsets;  /* device output: [max_reads+1], as in sws_minimizers_batch          */
  uint64_t *count;         /* device output: number of picks                                    */
  uint64_t capacity;       /* entries of hash/pos (= max_bases, never exceeded)                  */
  uint64_t max_reads, max_bases;
  int path;                /* 0: staged kernel, 1: look-back kernel, 2: single-pass kernel       */
  float tuned_ms[3];       /* measured ms per largest batch for each path (-1: not timed)        */
} sws_batch_io;
sws_status sws_batch_create(sws_ctx *ctx, uint64_t max_reads, uint64_t max_bases, int k, int w, int mode,
                            int options, sws_batch **out);
sws_status sws_batch_destroy(sws_batch *b);
/* The batch's device buffers (owned by the batch; valid until sws_batch_destroy). */
sws_status sws_batch_io_get(sws_batch *b, sws_batch_io *io);
/* Process the first nreads reads (total_bases bases) already in io.seq / io.offsets, on stream. */
sws_status sws_batch_run(sws_batch *b, uint64_t nreads, uint64_t total_bases, void *stream);
/* Wait for the last run and report a device-side fault (SWS_ERR_TIMEOUT) if one occurred. */
sws_status sws_batch_sync(sws_batch *b);

/* ---- serving: a request loop with continuous batching ------------------------------------ */
/* A server answers minimizer requests (one packed host sequence each; Sec. 2.4 per request)
 * with continuous batching: a worker thread forms batches from the queued requests in arrival
 * order and runs each on a free slot (a batch graph, a stream and pinned staging of its own), so
 * several batches are on the device at once and requests arriving meanwhile join the next batch
 * as soon as a slot is free.  A request is admitted while the device bytes it needs fit
 * hbm_budget_bytes next to those in flight.  Results are those of sws_minimizers on the request
 * alone (uint32 keys, so k <= 16; positions from 0).  Latency is measured from submission to the
 * moment the worker sees the result on the host.  Submitted bases are copied once, into pinned
 * memory; answers stay in pinned memory until released (sws_server_collect / _release) or copied
 * out (sws_server_result). */
typedef struct sws_server sws_server;
typedef struct sws_server_config {
  int k, w, mode;                  /* as for sws_minimizers (k <= 16)                          */
  uint32_t slots;                  /* batches in flight at once (>= 1)                          */
  uint64_t max_requests_per_batch; /* requests one batch may hold                               */
  uint64_t max_bases_per_batch;    /* bases one batch may hold; also the longest request        */
  uint64_t hbm_budget_bytes;       /* admission budget (0: half the free device memory)         */
} sws_server_config;
typedef struct sws_server_statistics {
  uint64_t completed, batches, bases, pending;
  double p50_s, p99_s, max_s, mean_s; /* latencies of completed requests                        */
  double span_s;                      /* first submission to last completion                   */
} sws_server_statistics;
sws_status sws_server_create(sws_ctx *ctx, const sws_server_config *cfg, sws_server **out);
/* Queue a request (the bases are copied; the caller's buffer may be reused at once).
 * SWS_ERR_CAPACITY if nbases > max_bases_per_batch. */
sws_status sws_server_submit(sws_server *s, const uint8_t *packed, uint64_t nbases, uint64_t *request_id);
/* Queue `count` requests in one call: packed[i] holds nbases[i] bases (copied); their ids go to
 * request_ids[i].  One lock and one wake-up for the lot; if any argument is wrong (a NULL
 * sequence, a request longer than max_bases_per_batch: SWS_ERR_INVALID / SWS_ERR_CAPACITY)
 * nothing is queued. */
sws_status sws_server_submit_batch(sws_server *s, const uint8_t *const *packed, const uint64_t *nbases, uint64_t count,
                                   uint64_t *request_ids);
/* Wait up to timeout_s seconds (0: just look) for a request; *done = 1 once it is answered. */
sws_status sws_server_wait(sws_server *s, uint64_t request_id, double timeout_s, int *done);
/* Copy an answered request's picks to host buffers and forget the request (whether or not it was
 * collected).  SWS_ERR_CAPACITY (with *count set) if capacity is too small; the request stays. */
sws_status sws_server_result(sws_server *s, uint64_t request_id, uint32_t *hash, uint32_t *pos, uint64_t capacity,
                             uint64_t *count, double *latency_s);
/* Collect up to max_n answered requests not collected before, in the order they were answered,
 * waiting up to timeout_s seconds (0: just look) for the first.  For each: its id, pick count,
 * pointers to its keys and positions IN THE SERVER'S PINNED RESULT MEMORY (read them in place; no
 * copy is made), and its latency (latency_s may be NULL).  *n_out = the number collected.  The
 * pointers stay valid until the request is released; a server holds 2 * slots + 2 result blocks
 * (one per batch), and a batch whose block is still held by unreleased answers waits, so release
 * promptly. */
sws_status sws_server_collect(sws_server *s, uint64_t max_n, double timeout_s, uint64_t *ids, uint64_t *counts,
                              const uint32_t **hash, const uint32_t **pos, double *latency_s, uint64_t *n_out);
/* Forget n answered requests (collected or not) and give their result memory back.  An id that is
 * unknown or not yet answered: SWS_ERR_INVALID (the others are still released). */
sws_status sws_server_release(sws_server *s, const uint64_t *ids, uint64_t n);
sws_status sws_server_stats(sws_server *s, sws_server_statistics *out);
sws_status sws_server_reset_stats(sws_server *s);
/* Finish running and queued requests (queued ones only while a result block is free for them),
 * stop the worker and free everything, answers not yet released included. */
sws_status sws_server_destroy(sws_server *s);

/* ---- minimizers without allocation ------------------------------------------------------ */
/* The paper has no counterpart to this entry point; it exists for callers that cannot allocate
 * device memory: code running inside a device-memory allocator's hooks (allocating there would
 * re-enter the allocator), programs whose device memory is all handed out in advance by a
 * framework that owns it, and latency-critical paths that must not pay for, or risk the failure
 * of, an allocation.  It computes exactly what sws_minimizers computes (same arguments, same
 * outputs, no N-block or key-mode difference), on the calling thread's current device, without a
 * context and without calling cudaMalloc, cudaFree or any allocating routine.
 *   Scratch: a fixed 4 MiB array in device global memory that the library declares, held by every
 *     device that loads the library until the process exits.  It bounds the input: at most
 *     262,128 tiles of (4096 - w) / 64 * 64 windows each (about 1.05e9 bases at w = 10); longer
 *     inputs are rejected with SWS_ERR_INVALID before any work is queued.
 *   Set-up: the first call on each device looks up the array's device address (with that device
 *     current); make that first call before any stream capture.
 *   Sharing: every call uses the same array, so calls that overlap on the GPU (for example on two
 *     streams at once) race and give wrong results; serialize them.
 *   Faults: count_out is set to all ones when the call is queued; if a bounded device-side wait
 *     runs out, the ordered output is not completed and count_out stays all ones. */
sws_status sws_minimizers_noalloc(const uint8_t *seq, uint64_t n, int k, int w, int mode, const int64_t *nblocks,
                                  uint64_t n_nblocks, void *hash_out, uint32_t *pos_out, uint64_t capacity,
                                  uint64_t *count_out, void *stream);

/* ---- seed table (Sec. 2.4, Fig. 1) -------------------------------------------------------- */
/* Build the seed table from m (hash, position) hits: a position table listing the hits sorted by
 * hash, and a pointer table with, for every bucket b of hash values (bucket of h =
 * h >> (hash_bits - bucket_bits)), the index of its first hit.
 *   hash, pos          : device input; hash is uint32 when hash_bits <= 32, else uint64.  Hits
 *                        should come in increasing position (as sws_minimizers writes them): the
 *                        sort is stable, so each hash's hits then stay in position order.
 *   sorted_hash/pos    : device outputs of m entries (same types); must not overlap the inputs.
 *   bucket_offsets     : device uint64 [2^bucket_bits + 1]; hits of bucket b are
 *                        [bucket_offsets[b], bucket_offsets[b+1]); the last entry is m.
 *   Limits: 1 <= hash_bits <= 64, 0 <= bucket_bits <= min(hash_bits, 32), m < 2^32.
 * Uses workspace (about 16 bytes per hit, 24 when hash_bits > 32). */
sws_status sws_kmer_table(sws_ctx *ctx, const void *hash, const uint32_t *pos, uint64_t m, int hash_bits,
                          int bucket_bits, void *sorted_hash, uint32_t *sorted_pos, uint64_t *bucket_offsets,
                          void *stream);

/* Strand of each minimizer pick (Sec. 2.4 over canonical k-mers, which pick the smaller of the
 * forward k-mer and its reverse complement): 0 when the forward k-mer at the pick is the smaller
 * or they are equal (a palindrome, possible for even k), 1 when the reverse complement is.
 *   seq, n, k  : the 2-bit packed sequence (or read batch) the picks came from, 1 <= k <= 32.
 *   base_offsets, pick_offsets, nreads : NULL/NULL/0 for picks of one sequence (pos = base
 *                index); for a batch, the read offsets (nreads + 1) and the pick offsets from
 *                sws_minimizers_batch (pos read-local).
 *   pos, m     : device, the picks' positions.  strand_out : device uint8 [m]; a pick whose k-mer
 *                does not lie inside the sequence gets 255.
 * Uses no workspace. */
sws_status sws_minimizer_strands(sws_ctx *ctx, const uint8_t *seq, uint64_t n, int k, const int64_t *base_offsets,
                                 const uint64_t *pick_offsets, uint64_t nreads, const uint32_t *pos, uint64_t m,
                                 uint8_t *strand_out, void *stream);

/* ---- seeding (Sec. 2.3) with the seed table (Sec. 2.4, Fig. 1) ------------------------------ */

/* Seed lookup: for each of nq query seeds, the run of its hits in a position table built by
 * sws_kmer_table (same hash_bits and bucket_bits): the pointer table gives the bucket's range and
 * two binary searches the run of equal hashes.
 *   sorted_hash, bucket_offsets : the table (device; sorted_hash uint32 when hash_bits <= 32,
 *                                 else uint64; m entries; offsets 2^bucket_bits + 1).
 *   query_hash : device, nq seeds of the same type.  A hash outside [0, 2^hash_bits) has no hits.
 *   first, count : device outputs, nq each: query i's hits are sorted_pos[first[i] ..
 *                  first[i] + count[i]) of the table (positions ascending within the run).
 * Limits as sws_kmer_table.  Uses no workspace. */
sws_status sws_seed_lookup(sws_ctx *ctx, const void *sorted_hash, uint64_t m, int hash_bits, int bucket_bits,
                           const uint64_t *bucket_offsets, const void *query_hash, uint64_t nq, uint64_t *first,
                           uint32_t *count, void *stream);

/* Seed hits: expand the runs found by sws_seed_lookup into (query index, reference position)
 * pairs, in query order and, per query, position order.  A seed with more than max_occ hits is
 * skipped (the usual repeat filter; max_occ = 0: no limit).
 *   first, count : device, from sws_seed_lookup;  sorted_pos : device, the table's positions.
 *   hit_query, hit_pos : device outputs; at most `capacity` pairs are written.
 *   hit_count : device uint64 receiving the exact number of kept pairs (also when > capacity).
 * nq < 2^32.  Uses workspace (8 bytes per 1024 queries). */
sws_status sws_seed_hits(sws_ctx *ctx, const uint64_t *first, const uint32_t *count, uint64_t nq, uint32_t max_occ,
                         const uint32_t *sorted_pos, uint32_t *hit_query, uint32_t *hit_pos, uint64_t capacity,
                         uint64_t *hit_count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SWS_H */
