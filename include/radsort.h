/*
 * radsort.h -- C ABI of the GB300 (sm_103a) Radsort library.
 *
 * Radsort ("Parallel O(sqrt n) Overhead LSD Radix Sort", Clausecker and
 * Schintke) is a stable LSD radix sort. Instead of an n-element output
 * buffer it uses a constant number of scratch blocks plus O(n/b)
 * bookkeeping.
 *
 * Problem statement (Sec. 1): sort n elements whose keys are n_t-tuples over
 * an alphabet of sigma symbols into lexicographic order, stably.  Here a key is
 * an unsigned integer of key_bytes (4 or 8) read as n_t = ceil(8*key_bytes /
 * digit_bits) digits of digit_bits bits each (sigma = 2^digit_bits), digit 0
 * the most significant; the result is ascending unsigned order, stable, with
 * the optional 32-bit values moved together with their keys.
 *
 * Conventions for every call below:
 *  - keys / values / workspace are DEVICE pointers owned by the caller unless
 *    stated; they must be 16-byte aligned (cudaMalloc and torch allocations
 *    are); values may be NULL (keys only).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued on it asynchronously; the calls never synchronise it.
 *  - Argument errors are returned synchronously and nothing is enqueued.
 *    Errors detected on the device (a bounded wait that ran out, a violated
 *    invariant) are recorded in a sticky library status word that
 *    radsort_device_status() reads; the device never traps.
 *  - n = 0 and n = 1 are no-ops that return RADSORT_OK.
 */
#ifndef RADSORT_H
#define RADSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RADSORT_OK = 0,
    RADSORT_EINVAL = 1,    /* bad argument (size, width, alignment, plan) */
    RADSORT_ENOMEM = 2,    /* device allocation failed / workspace too small */
    RADSORT_ECUDA = 3,     /* a CUDA runtime call failed */
    RADSORT_ETIMEOUT = 4,  /* a bounded device-side wait ran out */
    RADSORT_EINTERNAL = 5  /* a device-side invariant check failed */
} radsort_status;

/* flags for radsort_sort_ex */
#define RADSORT_KEY_FLOAT32 0x1u /* 4-byte keys are IEEE float32; sorted by the
                                    total order (-NaN < -inf < ... < -0 < +0 <
                                    ... < +inf < +NaN) via an order-preserving
                                    bit transform applied before and undone
                                    after the sort. */

/*
 * Block layouts (radsort_plan.layout).
 *  RADSORT_LAYOUT_CHUNKS: the paper's parallel variant (Sec. 4.3).  The array
 *    is split into p chunks, each with its own head start of sigma blocks and
 *    its own chain of blocks per bucket; T holds 2*sigma*p blocks.
 *  RADSORT_LAYOUT_GRID: one free list and one chain per bucket for the whole
 *    array, as in the sequential algorithm (Sec. 2), laid on the block grid of
 *    each round's output (blocks that hold the start of a bucket are shared
 *    by the buckets in them).  All SMs work on it through a decoupled
 *    look-back; T holds 4*sigma + 1 blocks whatever the parallelism, and
 *    after the last round every block but the tail is full.  Needs n < 2^31.
 *  RADSORT_LAYOUT_MSD: the MSD split of Sec. 4.3 (last paragraph): the first
 *    round sorts by the most significant digit in the chunk layout with
 *    p = sigma chunks, its sigma buckets become the chunks, and every chunk
 *    then runs the remaining rounds from its least significant digit on its
 *    own (each CTA's working set is one bucket).  8-bit digits only (T holds
 *    2*sigma^2 blocks); num_chunks must be 0; block_size 0 picks the largest
 *    of 64 .. 1024 within 2% of the array (else 64).  With radsort_sort_rounds,
 *    round 1 is the split and round r > 1 the digit at bits [(r-2)*8, (r-1)*8).
 *  RADSORT_LAYOUT_SCRATCH: short arrays are sorted out of place (Alg. 1) with
 *    the alternate arrays inside the workspace, the paper's suggestion for
 *    arrays below Radsort's crossover (Sec. 5: use T as A').  The automatic
 *    plan takes it for n <= RADSORT_SCRATCH_MAX_N; radsort_sort_rounds never
 *    uses it.
 */
#define RADSORT_LAYOUT_AUTO 0u
#define RADSORT_LAYOUT_CHUNKS 1u
#define RADSORT_LAYOUT_GRID 2u
#define RADSORT_LAYOUT_SCRATCH 3u
#define RADSORT_LAYOUT_MSD 4u
#define RADSORT_SCRATCH_MAX_N ((size_t)1 << 18)

/* Tuning plan.  Zero fields mean "choose automatically": the scratch layout
 * up to RADSORT_SCRATCH_MAX_N elements, the grid layout below 2^31 (largest
 * block size within 2% of the array's bytes), the chunk layout beyond. */
typedef struct {
    uint32_t block_size; /* b: elements per block, power of two in [64, 4096] */
    uint32_t num_chunks; /* p (chunk layout): chunks sorted in parallel, each
                            with its own head start of sigma blocks (Sec. 4.3);
                            nonzero with layout AUTO selects the chunk layout */
    uint32_t layout;     /* RADSORT_LAYOUT_* */
    uint32_t shape;      /* grid layout, tile shape of the round kernel:
                            0 or 1, one CTA of 16 consumer warps per SM on the
                            largest tiles; 2 (8-bit digits), two groups of 8
                            warps on smaller tiles (4096 or 8192 elements),
                            for arrays of few tiles per SM */
    uint32_t reserved[4];
} radsort_plan;

/* Human-readable name of a status code (static storage). */
const char *radsort_status_str(radsort_status s);

/* Fills *plan with the automatic choice for these sizes. */
radsort_status radsort_plan_default(size_t n, int key_bytes, int value_bytes, int digit_bits,
                                    radsort_plan *plan);

/*
 * Autotuner (no counterpart in the paper): times, on `stream`, sorts of a copy
 * of keys[0..n) (and values, if not NULL) under every plan of the automatic
 * plan's layout whose workspace fits the same budget (2% of the arrays, or
 * 1.25x the least workspace of any block size), and returns the fastest in
 * *plan.  Grid layout: block sizes 256 .. 4096 that a tile holds whole, with
 * both tile shapes (radsort_plan.shape 0 and 2) for 8-bit digits; chunk
 * layout: the automatic chunk count with block sizes 256 .. 2048.  Arrays up
 * to RADSORT_SCRATCH_MAX_N get the out-of-place plan without timing.
 * keys and values are read, never written (each timed sort starts from a
 * fresh device copy); while tuning, the call allocates that copy and the
 * largest candidate workspace (stream-ordered) and waits for the stream.
 * Results are cached per (device, ceil(log2 n), key_bytes, value bytes,
 * digit_bits):
 * a cached entry whose plan is valid for this n returns without touching the
 * GPU (otherwise the call tunes again and replaces it).  EINVAL on a bad width,
 * a NULL plan or an unaligned array; a failed timed sort returns its status.
 */
radsort_status radsort_autotune(const void *keys, const uint32_t *values, size_t n, int key_bytes,
                                int digit_bits, void *stream, radsort_plan *plan);

/*
 * radsort_autotune for both digit widths: tunes (or takes from the cache)
 * the plan for 8-bit and for 11-bit digits and returns the faster width in
 * *digit_bits with its plan (8 when the arrays are small enough that neither
 * is timed).  Pass both to radsort_sort_ex.  Same arguments, allocation,
 * synchronisation and errors as radsort_autotune.
 */
radsort_status radsort_autotune_digits(const void *keys, const uint32_t *values, size_t n, int key_bytes,
                                       void *stream, int *digit_bits, radsort_plan *plan);

/*
 * Bytes of device workspace radsort_sort_ex needs: the scratch array T
 * (2*sigma*p blocks in the chunk layout, Sec. 2.1 and 4.3; 4*sigma + 1 in the
 * grid layout), the block permutation pi and its successor, the usage array
 * U (Alg. 5-6, chunk layout), the partial-block list P, the per-chunk
 * counters or (grid layout) the digit histograms and the look-back words of
 * one round.  This is the sort's whole extra device memory beyond the
 * caller's arrays.  value_bytes is 0 or 4.
 */
radsort_status radsort_workspace_size(size_t n, int key_bytes, int value_bytes, int digit_bits,
                                      const radsort_plan *plan, size_t *bytes);

/*
 * Alg. 2 (radSort): setup (Alg. 4), n_t rounds of sortPhase (Alg. 5) and
 * fixupPhase (Alg. 6), then Finalize (Alg. 7), in place on keys[0..n) and
 * values[0..n).  key_bytes: 4 or 8.  digit_bits: 8 (sigma = 256) or 11
 * (sigma = 2048).  Allocates its workspace with cudaMallocAsync on `stream`
 * and frees it the same way.
 */
radsort_status radsort_sort(void *keys, uint32_t *values, size_t n, int key_bytes, int digit_bits,
                            void *stream);

/*
 * As radsort_sort, with flags (RADSORT_KEY_FLOAT32), an explicit plan
 * (NULL = automatic) and a caller-provided workspace of at least
 * radsort_workspace_size() bytes (NULL = allocate as radsort_sort does).
 * The workspace must stay untouched until the sort has completed on `stream`.
 */
radsort_status radsort_sort_ex(void *keys, uint32_t *values, size_t n, int key_bytes,
                               int digit_bits, uint32_t flags, const radsort_plan *plan,
                               void *workspace, size_t workspace_bytes, void *stream);

/*
 * The permuted representation without Finalize (Sec. 4.1, "Avoiding
 * Finalisation"): runs setup and the first `rounds` rounds (0 <= rounds <= n_t)
 * on keys/values in place, then writes the logical sequence -- the used
 * elements of logical blocks sigma*p .. f-1 in order, each block's length
 * given by sizeOfNextBlock (Alg. 3) -- to out_keys/out_values (n entries;
 * out_values may be NULL).  keys/values are left in the block layout (their
 * contents are unspecified afterwards).  After `rounds` rounds the sequence is
 * the stable sort by the `rounds` least significant digits.
 */
radsort_status radsort_sort_rounds(void *keys, uint32_t *values, size_t n, int key_bytes,
                                   int digit_bits, int rounds, const radsort_plan *plan,
                                   void *out_keys, uint32_t *out_values, void *stream);

/*
 * The permuted representation kept between calls (Sec. 4.1, "Avoiding
 * Finalisation"; truncation is Alg. 8).  A handle holds a Radsort state on
 * the caller's keys/values and workspace in the grid layout: the block map
 * pi, whose logical blocks hold the current sequence, every block full but
 * the last.  Rounds can be run on it, its blocks listed in logical order for
 * consumers that only iterate (no data moves), the sequence cut to a prefix
 * without disturbing the state, the data modified in place through the
 * listed blocks and sorted again, and Finalize applied when the caller wants
 * the sequence contiguous in keys/values.
 *
 * radsort_perm_workspace_size: device bytes the handle needs besides the
 *   arrays (as radsort_workspace_size for the grid layout with block size
 *   block_size, 0 = automatic).  EINVAL if the grid layout cannot take n
 *   (n >= 2^31) or the block size is not one it takes.
 * radsort_perm_open: setup (Alg. 4) on keys[0..n) / values (NULL = keys
 *   only); the host handle is allocated with malloc and returned in *out.
 *   keys, values and workspace stay in use until radsort_perm_close; their
 *   contents are the state, not a sequence, until radsort_perm_finalize.
 * radsort_perm_rounds: rounds first .. first+count-1 of Alg. 2's loop
 *   (round r: sortPhase on digit n_t-1-r, i.e. bits [r*d, (r+1)*d) of the
 *   key, then fixupPhase), 0 <= first, first + count <= n_t.  Rounds 0 ..
 *   n_t-1 sort the current sequence completely; a later call may start over
 *   at round 0 (after the keys were changed, or after a truncation).  The
 *   digit histograms are taken from the current sequence when it changed
 *   size since they were last taken; a caller who changed keys in place calls
 *   radsort_perm_keys_changed first.
 * radsort_perm_size: the current element count and the number of list
 *   entries (floor(n/b) + 1; the last entry may have length 0).
 * radsort_perm_blocks: writes the list to out_dev (device memory, at least
 *   that many entries, else EINVAL): entry q is logical block q of the
 *   sequence, with the device addresses of its first key and value and its
 *   used length; the sequence is entry 0's elements, then entry 1's, ...
 *   Valid until the next rounds / truncate / finalize call.
 * radsort_perm_gather: copies the sequence into out_keys / out_values (n
 *   entries each; out_values NULL = keys only).
 * radsort_perm_truncate: keeps the first m <= n elements (Alg. 8); the
 *   blocks past the new end become free blocks of the state.
 * radsort_perm_finalize: Finalize (Alg. 7): keys[0..n) / values[0..n) then
 *   hold the sequence; the handle accepts only radsort_perm_close after it.
 * radsort_perm_close: frees the host handle (no device work, no wait).
 * All calls but size and close are stream-ordered on `stream`.
 */
typedef struct radsort_perm radsort_perm;
typedef struct {
    uint64_t keys;     /* device address of the block's first key */
    uint64_t values;   /* device address of its first value (0 without values) */
    uint32_t len;      /* used elements, the block's keys[0 .. len) */
    uint32_t reserved;
} radsort_block;

radsort_status radsort_perm_workspace_size(size_t n, int key_bytes, int value_bytes, int digit_bits,
                                           uint32_t block_size, size_t *bytes);
radsort_status radsort_perm_open(void *keys, uint32_t *values, size_t n, int key_bytes, int digit_bits,
                                 uint32_t block_size, void *workspace, size_t workspace_bytes,
                                 void *stream, radsort_perm **out);
radsort_status radsort_perm_rounds(radsort_perm *h, int first, int count, void *stream);
radsort_status radsort_perm_keys_changed(radsort_perm *h);
radsort_status radsort_perm_size(const radsort_perm *h, size_t *n, size_t *entries);
radsort_status radsort_perm_blocks(radsort_perm *h, radsort_block *out_dev, size_t cap, void *stream);
radsort_status radsort_perm_gather(radsort_perm *h, void *out_keys, uint32_t *out_values, void *stream);
radsort_status radsort_perm_truncate(radsort_perm *h, size_t m, void *stream);
radsort_status radsort_perm_finalize(radsort_perm *h, void *stream);
radsort_status radsort_perm_close(radsort_perm *h);

/*
 * Comparison baseline: a conventional out-of-place LSD radix sort, Alg. 1
 * applied for t = n_t-1 .. 0, with one upfront pass that histograms all
 * digits and a decoupled look-back scan per round.  keys_alt / values_alt are
 * caller-provided n-element scratch arrays (the n*(key+value) bytes of extra
 * memory that Radsort avoids); the result ends in keys / values.
 */
radsort_status radsort_lsd_oop_sort(void *keys, uint32_t *values, void *keys_alt,
                                    uint32_t *values_alt, size_t n, int key_bytes, int digit_bits,
                                    void *stream);

/*
 * Device scratch that radsort_lsd_oop_sort allocates (stream-ordered) and
 * frees within the call, besides the caller's alternate arrays: the digit
 * histograms and bucket offsets of every round, and the look-back ring.
 * value_bytes: 0 (keys only) or 4.  Host-only; EINVAL on a bad width.
 */
radsort_status radsort_lsd_oop_scratch_size(size_t n, int key_bytes, int value_bytes,
                                            int digit_bits, size_t *bytes);

/*
 * Batched segmented sort: each segment [offsets[s], offsets[s+1]) of keys (and
 * values) is sorted stably and independently (n = offsets[num_segments]).
 * offsets_dev is the device copy of the num_segments+1 offsets (read by the
 * kernels); offsets_host the same values on the host (used to plan the long
 * segments).  Segments up to 4096 elements (2048 for 11-bit digits) are sorted
 * in shared memory.  Segments up to 2^18 elements are sorted out of place in
 * per-CTA scratch as long as the longest of them (at most 2 CTAs per SM, held
 * to 6% of the arrays' bytes), the paper's suggestion of reusing T as the A'
 * of Alg. 1 for short arrays (Sec. 5).
 * Both classes are handled by one persistent launch each.  Longer segments
 * run the full Radsort (Alg. 2), or Alg. 1 with alternate buffers in the
 * workspace when their start is not 16-byte aligned; they are spread, longest
 * first, over up to 4 library-owned streams (created on the first call that
 * has long segments on a device) that start after the work already on
 * `stream` and that `stream` waits for, each with its own part of the
 * workspace.  workspace: at least radsort_segmented_workspace_size() bytes,
 * or NULL to allocate stream-ordered.  With 8-bit digits a smaller caller
 * workspace, down to radsort_segmented_workspace_size_min() bytes, selects
 * the fastest of two low-memory plans that fits: (1) the medium segments
 * longer than 16448 elements are sorted in place by Radsort itself on one
 * CTA each (Alg. 4-7 on blocks of 32 elements, with 2 sigma + 2 scratch
 * blocks per CTA, two CTAs per SM, one per SM on 7/8 of the SMs beside long
 * segments), the shorter ones out of place in those
 * scratch blocks; (2) as (1), and a long segment whose start is not 16-byte
 * aligned has its first (at most 3) elements set aside, the rest sorted by
 * Radsort and those elements merged back, instead of the alternate buffers.
 * On 20,000 lognormal arrays (2^29 keys + values) the plans hold 9%, 3.4%
 * and 0.95% of the arrays' bytes; (1) and (2) run about 30% slower than the
 * fastest plan.  With a caller workspace the call
 * issues only kernel launches, memsets and event records / waits, so it can
 * be captured in a CUDA graph (make a first call with long segments before
 * capturing, so that the streams exist).  Calls from several host threads
 * on one device take turns while they enqueue.
 */
radsort_status radsort_segmented_workspace_size(const uint64_t *offsets_host, size_t num_segments,
                                                int key_bytes, int value_bytes, int digit_bits,
                                                size_t *bytes);
radsort_status radsort_segmented_workspace_size_min(const uint64_t *offsets_host, size_t num_segments,
                                                    int key_bytes, int value_bytes, int digit_bits,
                                                    size_t *bytes);
radsort_status radsort_sort_segmented(void *keys, uint32_t *values, const uint64_t *offsets_dev,
                                      const uint64_t *offsets_host, size_t num_segments,
                                      int key_bytes, int digit_bits, void *workspace,
                                      size_t workspace_bytes, void *stream);

/*
 * Autotuner of the batched sort (no counterpart in the paper): times
 * radsort_sort_segmented on a device copy of keys / values (not modified)
 * with 8- and 11-bit digits, twice each, and returns the faster width in
 * *digit_bits.  Allocates the copy and the larger workspace stream-ordered
 * and waits for `stream`.  EINVAL on a bad width, NULL pointers or
 * unaligned arrays; a failed timed sort returns its status.
 */
radsort_status radsort_segmented_autotune(const void *keys, const uint32_t *values, const uint64_t *offsets_dev,
                                         const uint64_t *offsets_host, size_t num_segments, int key_bytes,
                                         void *stream, int *digit_bits);

/*
 * Comparison baseline for the batched sort: the same segments, the same
 * shared-memory and per-CTA passes for the short ones, and the long ones
 * sorted out of place (Alg. 1, radsort_lsd_oop_sort) into keys_alt /
 * values_alt, n-element caller arrays (the memory Radsort avoids), on the
 * same internal streams.  The result ends in keys / values.  workspace: at
 * least radsort_lsd_oop_segmented_workspace_size() bytes, or NULL.
 */
radsort_status radsort_lsd_oop_segmented_workspace_size(const uint64_t *offsets_host, size_t num_segments,
                                                        int key_bytes, int value_bytes, int digit_bits,
                                                        size_t *bytes);
radsort_status radsort_lsd_oop_sort_segmented(void *keys, uint32_t *values, void *keys_alt,
                                              uint32_t *values_alt, const uint64_t *offsets_dev,
                                              const uint64_t *offsets_host, size_t num_segments,
                                              int key_bytes, int digit_bits, void *workspace,
                                              size_t workspace_bytes, void *stream);

/*
 * radsort_sort_noalloc: radsort_sort without any device allocation.  The
 * paper has no counterpart; this entry point exists for callers that cannot
 * allocate device memory at the point of the call -- code running inside a
 * framework that owns all device memory through its own pool, loops whose
 * latency cannot absorb the implicit synchronisation and fragmentation of
 * cudaMalloc, or error paths that run when memory is already exhausted.
 *
 * The workspace is a fixed array of RADSORT_NOALLOC_SCRATCH_BYTES compiled into
 * the library (every GPU that loads the library holds it until the process
 * exits).  The plan is the automatic one (grid layout) when its workspace
 * fits, else the chunk layout with block size 256 and as many chunks (up to
 * one per SM) as fit; an n whose workspace does not fit even with one chunk
 * returns RADSORT_ENOMEM and enqueues nothing.  With 8-bit digits the grid
 * layout fits up to 2^31 - 1 elements with 4-byte keys (with or without
 * values) and with 8-byte keys alone, up to 2^30 with 8-byte keys and values;
 * with 11-bit digits up to 2^30 4-byte keys alone and 2^29 with values or with
 * 8-byte keys, 2^28 with 8-byte keys and values.
 * Every call looks up the array's device address on the current device with
 * cudaGetSymbolAddress (which allocates nothing), so the address stays right
 * after a context reset; the first call on a device may also load the
 * library's device code there, so make that first call before any stream
 * capture.  No call allocates or frees memory.  All calls share the one
 * array: calls that overlap on the GPU (other streams, other host threads)
 * race and corrupt each other; serialise them.  Each call rebuilds every
 * part of the workspace it reads, so a previous call's leftovers do no harm.
 */
#define RADSORT_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
radsort_status radsort_sort_noalloc(void *keys, uint32_t *values, size_t n, int key_bytes,
                                    int digit_bits, void *stream);

/* Order-preserving bit transform for float32 keys, in place on the device:
 * inverse = 0 maps IEEE bits to unsigned-orderable bits, inverse = 1 back. */
radsort_status radsort_float_keys(uint32_t *keys, size_t n, int inverse, void *stream);

/*
 * Synchronises `stream`, returns the sticky device status accumulated by all
 * sorts since the last call (RADSORT_OK if none failed), and clears it.
 */
radsort_status radsort_device_status(void *stream);

/*
 * Failure-path probe (no counterpart in the paper; for tests).  Launches one
 * thread on `stream` that waits for the device word *flag to become non-zero
 * the way every wait of the library does: at most `iterations` polls, each
 * followed by a sleep of at least 64 ns (1 <= iterations <= 2^26, the
 * library's own limit).  If the flag stays 0 the wait runs out, and the next
 * radsort_device_status returns RADSORT_ETIMEOUT; the context stays usable.
 * EINVAL (synchronously) on a null flag or an iteration count out of range.
 */
radsort_status radsort_debug_wait_probe(const uint32_t *flag, unsigned iterations, void *stream);

/*
 * Tracing (no counterpart in the paper; measurement support).  While enabled,
 * every sort records a CUDA event pair on its own stream around each phase:
 * setup (Alg. 4), each round's sortPhase kernel (Alg. 5), each fixupPhase
 * (Alg. 6) and Finalize (Alg. 7).  radsort_trace_read waits for the recorded
 * events, copies up to `cap` records in launch order into `out`, stores the
 * number recorded in *count, and clears the list.  Records: phase 0 = setup,
 * 1 = sortPhase, 2 = fixupPhase, 3 = Finalize, 4 = key transform; `round` is
 * the digit round (or -1); `ms` the event-measured duration.
 * radsort_launch_count returns the number of kernels this library has
 * launched since it was loaded.
 */
typedef struct {
    int32_t phase;
    int32_t round;
    float ms;
} radsort_trace_rec;

radsort_status radsort_trace_enable(int on);
radsort_status radsort_trace_read(radsort_trace_rec *out, int cap, int *count);
radsort_status radsort_launch_count(uint64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* RADSORT_H */
