/*
 * fpparse.h -- C ABI of the GB300 bulk decimal-text -> binary64 parser.
 *
 * The library converts delimited ASCII decimal numbers to the nearest
 * IEEE-754 binary64, rounding ties to even, bit for bit (the problem of
 * Section 1 of Lemire, "Number Parsing at a Gigabyte per Second").  Every
 * step runs in CUDA kernels on the device: field indexing, significand and
 * exponent parsing (Section 4), the truncated power-of-five product of
 * Algorithm 1 (Section 5, justified in Sections 6-10), the 19-digit truncation check for long
 * significands (Section 11) and an exact big-number fallback for the rare
 * cases those cannot settle.  There is no CPU fallback.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers.  Unless stated otherwise, text, output and count pointers are
 * DEVICE memory owned by the caller.  The library never frees them and
 * never keeps them after the work queued by the call has finished.
 *
 * Streams.  `stream` is a cudaStream_t (NULL = the legacy default stream).
 * Calls are asynchronous: they return once the work is queued on `stream`;
 * outputs, counts and device-side errors are valid after the stream has
 * reached that point.  Calls on the same stream are ordered.  Calls on
 * different streams may run concurrently; each stream gets its own scratch.
 * A parse call's kernels are programmatic dependent launches and release
 * the kernel queued after them early: a caller's kernel launched with
 * programmatic stream serialization right after a call may start before
 * the call has finished, so it must wait (cudaGridDependencySynchronize)
 * before it reads the call's results, as that launch mode requires; any
 * other operation queued after a call starts once the call is complete.
 *
 * Host threads.  Every entry point may be called from any host thread; the
 * library's shared state (the per-stream scratch table, the configuration,
 * device properties) is guarded by one lock, held while a call queues its
 * work.  A stream's scratch is reused by its next call, so calls on the SAME
 * stream must not overlap in time across threads (fp_parse_f64_host keeps
 * that stream's staging buffers while it copies); threads that each use
 * their own stream need no coordination.  fp_set_config applies to calls
 * that start after it returns.  A request server has its own scheduler
 * thread and streams; its submit / wait calls may come from any thread.
 *
 * Fields.  A field is a maximal run of bytes between separators, the
 * separators being '\n' and `delim` (pass '\n' for newline-only).  Field i of
 * the buffer is written to out_f64[i] / out_status[i].  A buffer ending in a
 * separator has no trailing empty field; an empty field elsewhere is
 * INVALID.  A buffer of len bytes holds at most fp_max_fields(len) fields;
 * the output arrays must hold that many entries.
 *
 * Grammar of a field (Section 4; the library's reading):
 *     [ \t\r]*  [+-]?  ( d+ ( '.' d* )? | '.' d+ )  ( [eE] [+-]? d+ )?  [ \t\r]*
 * Digits may be arbitrarily many (Section 11: up to 768 significant digits
 * can matter; all of them are honoured).  An explicit exponent of magnitude
 * above 10^15 saturates, which is exact for fields shorter than ~10^15 bytes.
 *
 * Results.  out_f64[i] is the nearest binary64 to the field's exact decimal
 * value, ties to even; the sign is applied last, so "-0" gives -0.0 and
 * "-1e999" gives -inf (Algorithm 1 flips the sign bit).  out_status[i] is
 * one of FP_STATUS_*; an INVALID field gets the quiet NaN 0x7FF8000000000000.
 * Results do not depend on which internal path produced them.
 *
 * Reading of text bytes.  The kernels only use bytes inside [text, text+len).
 * Staging copies move whole aligned 16-byte granules, so they may read up
 * to 15 bytes on either side of the range within the same granule (never
 * another page); those bytes are never used.
 *
 * Errors.  Argument errors are returned before anything is queued.  CUDA
 * launch or allocation failures return FP_ERR_CUDA.  Conditions found on the
 * device (a bounded wait that ran out, an internal limit) are recorded in
 * the per-stream error word, read with fp_get_error().
 */
#ifndef FPPARSE_H
#define FPPARSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st; /* cudaStream_t is `struct CUstream_st *` */

#if defined(__GNUC__)
#define FP_API __attribute__((visibility("default")))
#else
#define FP_API
#endif

typedef enum {
    FP_OK = 0,
    FP_ERR_ARG = 1,      /* a bad pointer, size or flag                       */
    FP_ERR_CAPACITY = 2, /* an output or internal capacity would be exceeded   */
    FP_ERR_CUDA = 3,     /* a CUDA call failed (launch, copy, allocation)      */
    FP_ERR_BUDGET = 4,   /* a device-memory budget would be exceeded           */
    FP_ERR_TIMEOUT = 5,  /* a bounded device-side wait ran out                 */
    FP_ERR_INTERNAL = 6  /* an internal invariant failed on the device        */
} fp_err_t;

/* Per-field status byte (device). */
enum {
    FP_STATUS_OK = 0,        /* finite, or an exact zero                      */
    FP_STATUS_INVALID = 1,   /* not a number under the grammar; value is NaN  */
    FP_STATUS_OVERFLOW = 2,  /* finite text whose value rounds to +-infinity  */
    FP_STATUS_UNDERFLOW = 3, /* nonzero text whose value rounds to +-0        */
    FP_STATUS_BAD_SHAPE = 4  /* fp_parse_ex column-major: wrong terminator    */
};

/* Path counters, accumulated over calls on one stream (fp_get_stats).      */
typedef struct {
    uint64_t calls;           /* parse calls queued on this stream              */
    uint64_t fields;          /* fields parsed                                   */
    uint64_t bytes;           /* text bytes parsed                               */
    uint64_t one_multiply;    /* fast-path Algorithm 1 runs with one 64x64 product */
    uint64_t two_multiplies;  /* Algorithm 1 runs that needed the second product   */
    uint64_t long_fields;     /* more than 19 significant digits (Section 11)    */
    uint64_t long_settled;    /* ... settled by the w / w+1 check                */
    uint64_t fallback;        /* fields resolved by the exact fallback kernel    */
    uint64_t fallback_bignum; /* ... that needed a big-number comparison         */
    uint64_t queue_overflow;  /* fallback fields found by scanning (queue full)  */
    uint64_t general_tokenizer; /* fields that needed the general tokenizer       */
} fp_stats_t;

/*
 * fp_max_fields -- capacity rule for output arrays.
 *   Returns the largest number of fields a len-byte buffer can hold: len
 *   (every byte a separator, each closing an empty field), 0 for len == 0.
 *   Output arrays of this many entries are always sufficient.
 */
FP_API size_t fp_max_fields(size_t len);

/*
 * fp_parse_f64 -- parse every field of one buffer (Sections 4-11).
 *   text        device pointer to len bytes (any alignment; may be NULL iff len == 0)
 *   len         bytes in the buffer (< 2^40)
 *   delim       the second separator besides '\n'
 *   out_f64     device array, fp_max_fields(len) doubles; field i -> out_f64[i]
 *   out_status  device array, fp_max_fields(len) bytes; field i -> out_status[i]
 *   out_count   device pointer to one uint64_t: the number of fields
 *   stream      CUDA stream the work is queued on
 * Entries of out_f64/out_status beyond the field count are left unchanged.
 * The first call on a stream (and a call needing more scratch than any
 * before it) allocates the stream's scratch with cudaMalloc; make such a
 * call before capturing the stream into a CUDA graph.
 * Returns FP_OK once queued; FP_ERR_ARG for NULL pointers with len > 0.
 */
FP_API fp_err_t fp_parse_f64(const char *text, size_t len, char delim, double *out_f64,
                      uint8_t *out_status, uint64_t *out_count, struct CUstream_st *stream);

/*
 * fp_parse_f32 -- fp_parse_f64 with binary32 results: the nearest float,
 *   ties to even (Section 2's 32-bit format; Algorithm 1's 32-bit case,
 *   Section 5: 26 provably exact bits after one product, ties only for
 *   q in [-17, 10]; the same 19-digit check and exact fallback, Section 11).
 *   out_f32     device array, fp_max_fields(len) floats; field i -> out_f32[i]
 *   Other arguments, statuses and asynchrony as fp_parse_f64; INVALID
 *   fields get the quiet NaN 0x7FC00000.  The first call on a stream needing
 *   more room than any before it also allocates 8 bytes per possible field
 *   of scratch (where unsettled fields keep their text location until the
 *   fallback kernel decides them).
 */
FP_API fp_err_t fp_parse_f32(const char *text, size_t len, char delim, float *out_f32,
                             uint8_t *out_status, uint64_t *out_count,
                             struct CUstream_st *stream);

/*
 * fp_parse_ex -- one buffer with options beyond the decimal-to-binary64
 *   default: the binary32 format, the hexadecimal-float or JSON grammar, and
 *   column-major results for CSV blocks.  (The paper's Algorithm 1 covers
 *   both formats, Section 5; hexadecimal floats are Appendix C's exact form;
 *   Section 4 names JSON's stricter number grammar among the format
 *   variants; the columnar layout has no counterpart in the paper.)
 *   opt->delim     the second separator besides '\n'
 *   opt->format    FP_FORMAT_F64 (out_values: doubles) or FP_FORMAT_F32 (floats)
 *   opt->grammar   FP_GRAMMAR_DECIMAL: the decimal grammar above;
 *                  FP_GRAMMAR_HEX: that, or a hexadecimal float
 *                    [+-]? 0[xX] (h+ (. h*)? | . h+) ([pP] [+-]? d+)?
 *                    (binary exponent optional; rounded exactly, ties to even);
 *                  FP_GRAMMAR_JSON: the JSON number grammar
 *                    -? (0 | [1-9] d*) (. d+)? ([eE] [+-]? d+)?
 *                    ('+', leading zeros, "5." and ".5" are INVALID)
 *   opt->columns   0: field i -> out_values[i] (fp_max_fields(len) entries);
 *                  K >= 2 (< 2^24): field i -> column i mod K, row i div K,
 *                    entry (i mod K) * rows_cap + (i div K); K * rows_cap
 *                    entries; fields whose row is >= rows_cap are not stored
 *                    (the count still counts them).  A field whose terminator
 *                    disagrees with its column -- the last column must end at
 *                    '\n' or at the end of the text, the others at delim --
 *                    gets status FP_STATUS_BAD_SHAPE (its value is stored).
 *   opt->rows_cap  entries per column (columns >= 2)
 * The JSON and column-major modes run with 8 KiB chunks when the configured
 * chunk size is 4 or 8 KiB and with 16 KiB chunks otherwise.  Binary32 and
 * column-major calls use the same per-stream location scratch as
 * fp_parse_f32.  FP_ERR_ARG for unknown options or columns == 1.
 */
#define FP_FORMAT_F64 0
#define FP_FORMAT_F32 1
#define FP_GRAMMAR_DECIMAL 0
#define FP_GRAMMAR_HEX 1
#define FP_GRAMMAR_JSON 2
typedef struct {
  char delim;
  uint8_t format;
  uint8_t grammar;
  uint8_t reserved;
  uint32_t columns;
  uint64_t rows_cap;
} fp_options_t;
FP_API fp_err_t fp_parse_ex(const char *text, size_t len, const fp_options_t *opt,
                            void *out_values, uint8_t *out_status, uint64_t *out_count,
                            struct CUstream_st *stream);

/*
 * fp_parse_f64_batch -- parse many independent buffers in one persistent
 * launch (work is split by chunk across all buffers, not by buffer).
 *   texts        HOST array of nbuf device pointers (NULL allowed iff lens[b] == 0)
 *   lens         HOST array of nbuf lengths (each < 2^40)
 *   nbuf         number of buffers (1 .. 2^24)
 *   delim        as for fp_parse_f64
 *   out_f64      device array; buffer b's field i -> out_f64[out_offsets[b] + i]
 *   out_status   device array, same indexing
 *   out_offsets  HOST array of nbuf+1 non-decreasing offsets: buffer b owns
 *                entries [out_offsets[b], out_offsets[b+1]) of both arrays.
 *                Fields beyond that capacity are counted but not stored, so
 *                a region of fp_max_fields(lens[b]) entries is always enough.
 *   out_counts   device array of nbuf uint64_t: fields per buffer (the true
 *                count, which may exceed the region's capacity)
 *   stream       CUDA stream
 * The descriptors are staged and copied to the device inside the call, so
 * the host arrays may be reused as soon as the call returns.  Scratch is
 * allocated as for fp_parse_f64.
 */
FP_API fp_err_t fp_parse_f64_batch(const char *const *texts, const size_t *lens, uint32_t nbuf,
                            char delim, double *out_f64, uint8_t *out_status,
                            const uint64_t *out_offsets, uint64_t *out_counts,
                            struct CUstream_st *stream);

/*
 * Batch plans: the descriptors of a fixed set of buffers uploaded once, with
 * their own scratch, so that one call launches the whole batch with no host
 * work beyond two memsets and two kernel launches -- a sequence that can be
 * captured into a CUDA graph and replayed.  (Same results as
 * fp_parse_f64_batch with the same arguments.)
 *
 * fp_batch_plan_create -- arguments as for fp_parse_f64_batch, minus the
 *   stream, plus `flags`; the buffers and output arrays must stay valid for
 *   the plan's life.  Synchronous; allocates device memory; the chunk size
 *   and blocks per SM are those of fp_get_config at this call.  With
 *   FP_PLAN_GRAPH in `flags` the launch sequence is captured once into a
 *   CUDA graph here, and each fp_batch_plan_launch replays it with one
 *   cudaGraphLaunch.  *plan receives the plan.
 * fp_batch_plan_launch -- queue the parse of every buffer of the plan on
 *   `stream`.  Launches of one plan must not overlap on the GPU.  Plan
 *   launches add nothing to fp_get_stats or fp_timing_read.
 * fp_batch_plan_destroy -- synchronise and free the plan (NULL is ignored).
 */
typedef struct fp_batch_plan fp_batch_plan;
#define FP_PLAN_GRAPH 1u
FP_API fp_err_t fp_batch_plan_create(const char *const *texts, const size_t *lens, uint32_t nbuf,
                                     char delim, double *out_f64, uint8_t *out_status,
                                     const uint64_t *out_offsets, uint64_t *out_counts,
                                     uint32_t flags, fp_batch_plan **plan);
FP_API fp_err_t fp_batch_plan_launch(fp_batch_plan *plan, struct CUstream_st *stream);
FP_API fp_err_t fp_batch_plan_destroy(fp_batch_plan *plan);

/*
 * fp_batch_plan_gather -- pack the results of the plan's last launch in
 *   buffer order, for one copy back: the k_b = min(out_counts[b],
 *   out_offsets[b + 1] - out_offsets[b]) values and statuses buffer b holds
 *   go to dst_f64 / dst_status from the sum of the earlier buffers' k_b on,
 *   and that sum over all buffers (the total) to *dst_total.
 *   dst_f64 (8-byte aligned), dst_status and dst_total are addresses the
 *   device can write (device memory, or pinned host memory through its
 *   device address), with room for the total (at most out_offsets[nbuf] -
 *   out_offsets[0] entries); they must not overlap the plan's outputs.
 *   Queued on `stream` after the launch (two kernels: a scan of the counts,
 *   then a copy in pieces of 8192 fields); no host synchronisation.  Returns FP_ERR_ARG
 *   for a null plan, or null arrays when the plan has outputs.
 */
FP_API fp_err_t fp_batch_plan_gather(fp_batch_plan *plan, double *dst_f64, uint8_t *dst_status,
                                     uint64_t *dst_total, struct CUstream_st *stream);

/*
 * Request server: continuous batching of parse requests held in HOST memory.
 *   (The paper has no counterpart: it measures one buffer at a time.  This is
 *   the serving form of the same parse.)
 * One scheduler thread per server owns one device-memory arena of
 * `device_budget` bytes, cut into a text region (1 B per unit), a value
 * region (8 B per unit) and a status region (1 B per unit); a request of
 * `len` bytes holds len + 16 units, rounded up to 256, from admission to
 * completion.  Requests are admitted first-come first-served as arena space
 * frees up (a request that does not fit waits, and so do those behind it).
 * Whenever one of `max_inflight` launch slots is free, the admitted
 * requests not yet launched, in order, up to `launch_bytes` of text (at
 * least one, at most `max_batch`) go into one launch
 * sequence on that slot's stream: a gather kernel copies the texts from
 * host memory into the arena, the persistent batched parse and its
 * fallback run, and a scatter kernel writes each request's first
 * min(fields, out_cap) values and statuses straight into the caller's
 * host arrays; then the request's units are released.  The kernels reach
 * host memory directly when it is pinned (page-locked); requests of 1 MB
 * or more, and texts and arrays in pageable memory, are moved by copy
 * calls instead (results after their counts are back).  A request below
 * 8 MB launched alone with pinned arrays is copied in and parsed straight
 * into its host arrays (no gather or scatter).  A request of 32 MB or more
 * launched alone with pinned text and arrays is cut at separators into
 * segments (as fp_parse_f64_host cuts such a text) whose copies in, parses
 * and copies out overlap, each segment one parse launch.  Different
 * slots' sequences overlap on the device.  Results equal those of
 * fp_parse_f64 on the same text, alone or in any mix.
 * Besides the arena, each slot's stream holds the parse scratch of up to
 * one budget's worth of chunks (24 B per 4 KiB of budget/10, plus the
 * fallback queue), and pinned piece tables for its copy kernels (about
 * 0.2% of budget/10).
 *
 * fp_server_create -- start a server on the current device.  cfg fields:
 *   device_budget  bytes for the arena (>= 4 KiB; allocated here at once)
 *   max_batch      most requests in one launch, 1..65536
 *   max_inflight   launches in flight at once, 1..8
 *   delim          field separator besides '\n'
 *   launch_bytes   text bytes one launch takes at most (at least one
 *                  request); 0 means 32 MB
 * fp_server_submit -- queue one request and return at once.
 *   host_text    len bytes of host memory (pinned copies fastest)
 *   host_f64     host array of out_cap doubles
 *   host_status  host array of out_cap bytes
 *   out_cap      entries the two arrays hold: the first min(fields, out_cap)
 *                results are written (fp_max_fields(len) always suffices)
 *   request_id   receives the request's id
 *   All three arrays must stay valid and untouched until the request is
 *   waited for.  FP_ERR_BUDGET if len units exceed the whole arena.
 * fp_server_wait -- wait up to timeout_ns (< 0: no limit, 0: poll) for a
 *   request; on completion fills *info, forgets the request and returns
 *   the request's own error (FP_OK when parsed); FP_ERR_TIMEOUT if it is
 *   not done yet (the request stays); FP_ERR_ARG for an unknown id.
 * fp_server_get_stats -- totals since creation.
 * fp_server_destroy -- wait for every submitted request, stop the thread,
 *   free everything (NULL is ignored).
 * Times are CLOCK_MONOTONIC nanoseconds.
 */
typedef struct fp_server fp_server;
typedef struct {
  uint64_t device_budget;
  uint32_t max_batch;
  uint32_t max_inflight;
  char delim;
  uint64_t launch_bytes; /* text bytes per launch at most (0: 32 MB) */
} fp_server_config_t;
typedef struct {
  uint64_t count;      /* fields in the text (min(count, out_cap) written) */
  int32_t error;       /* fp_err_t of this request */
  uint32_t batch_size; /* requests in the launch that parsed it */
  int64_t submit_ns, admit_ns, launch_ns, done_ns;
} fp_request_info_t;
typedef struct {
  /* launches: parse launches (a segmented request counts one per segment) */
  uint64_t submitted, completed, launches, bytes, fields;
  uint64_t peak_units;     /* most arena units held at once */
  uint64_t peak_requests;  /* most requests admitted at once */
  uint64_t max_batch_seen; /* largest launch */
} fp_server_stats_t;
FP_API fp_err_t fp_server_create(const fp_server_config_t *cfg, fp_server **server);
FP_API fp_err_t fp_server_submit(fp_server *server, const char *host_text, size_t len,
                                 double *host_f64, uint8_t *host_status, size_t out_cap,
                                 uint64_t *request_id);
FP_API fp_err_t fp_server_wait(fp_server *server, uint64_t request_id, int64_t timeout_ns,
                               fp_request_info_t *info);
FP_API fp_err_t fp_server_get_stats(fp_server *server, fp_server_stats_t *out);
FP_API fp_err_t fp_server_destroy(fp_server *server);

/*
 * fp_get_stats -- copy the path counters of `stream` into *host_out
 * (host memory).  Synchronises `stream`.  If reset != 0 the counters are
 * zeroed afterwards.
 */
FP_API fp_err_t fp_get_stats(fp_stats_t *host_out, int reset, struct CUstream_st *stream);

/*
 * fp_get_error -- synchronise `stream` and return the first device-side
 * error recorded by calls on it since the last fp_get_error (FP_OK if none);
 * clears it.
 */
FP_API fp_err_t fp_get_error(struct CUstream_st *stream);

/*
 * fp_set_config / fp_get_config -- launch parameters used by later calls
 * (all streams).  chunk_bytes: text bytes per work tile (4096, 8192, 12288
 * or 16384; at the default 16384, fp_parse_f64 / fp_parse_f32 calls on
 * texts below 4 MB use 4096, so that more blocks share a small text);
 * ctas_per_sm: resident blocks per SM for the persistent grid (1..8, or 0
 * for as many as fit, the default; a value above what fits is capped);
 * fallback_queue: entries of the per-stream fallback queue (1024 .. 2^28).
 * Returns FP_ERR_ARG for values outside those sets.
 */
typedef struct {
    uint32_t chunk_bytes;
    uint32_t ctas_per_sm;
    uint32_t fallback_queue;
} fp_config_t;
FP_API fp_err_t fp_set_config(const fp_config_t *cfg);
FP_API fp_err_t fp_get_config(fp_config_t *cfg);

/*
 * fp_autotune -- time the candidate configurations on a device buffer
 * supplied by the caller (text/len as for fp_parse_f64; it should be
 * representative of the workload), pick the fastest, make it current and,
 * if cache_path is not NULL, record it in that file.  The candidates: chunk
 * sizes 4096, 8192, 12288 and 16384 x blocks per SM 1, 2, 3, 4 or all that
 * fit; then, for the fastest of those, fallback queue depths 2^16, 2^18,
 * 2^20 and 2^22 (the smallest within 2% of the fastest is kept).  The
 * mapping of threads to numbers is fixed by field class and not tuned: one
 * thread per field of up to 30 bytes, one warp per field in the fallback.
 * The cache holds one JSON object per line, keyed by the GPU's name and the
 * workload's class: the text's size (below 4 MB, below 64 MB, larger) and
 * the share of its fields that reach the fallback kernel (below 0.1%,
 * below 10%, more), measured by one untimed call first.  If the file holds
 * an entry for the same GPU and class, it is loaded instead and nothing
 * else is timed.  Synchronous; allocates temporary output arrays with
 * cudaMalloc and frees them before returning.  While it times, the
 * candidates are the current configuration (fp_set_config), so calls from
 * other threads meanwhile may run under any of them; on an error the
 * configuration from before the call is restored.
 */
FP_API fp_err_t fp_autotune(const char *text, size_t len, char delim, const char *cache_path,
                     fp_config_t *chosen);

/*
 * fp_timing_enable -- when on > 0, every on-th later parse call on a stream
 * (counting that stream's calls; on = 1: every call) records CUDA events on
 * the stream around each kernel it launches, and the library adds up those
 * kernels' device time per stream without synchronising (events are
 * harvested as they complete).  on <= 0 turns it off (the default).  An
 * event between two kernels ends their programmatic overlap, so a timed
 * call takes a few microseconds longer than an untimed one; timing a sample
 * of the calls (on > 1) keeps that cost off the others.
 */
FP_API fp_err_t fp_timing_enable(int on);

/*
 * fp_timing_read -- wait for the timed calls queued on `stream`, return the
 * summed device time in milliseconds of their parse kernels (*parse_ms) and
 * fallback kernels (*fallback_ms) and the number of calls (*calls), then
 * reset the sums.  All three are host pointers.
 */
FP_API fp_err_t fp_timing_read(struct CUstream_st *stream, double *parse_ms,
                               double *fallback_ms, uint64_t *calls);

/*
 * fp_parse_f64_host -- end-to-end parse of a HOST buffer.
 *   host_text    host pointer to len bytes (pinned memory copies fastest)
 *   host_f64     host array of at least fp_max_fields(len) doubles
 *   host_status  host array of at least fp_max_fields(len) bytes
 *   host_count   host pointer: the number of fields
 * Copies the text to a per-stream device staging buffer and parses it
 * there.  When host_f64 and host_status are pinned and len < 8 MB, the
 * parse kernel writes the results (and the count) straight into them
 * through their device addresses; otherwise the library reads the field
 * count and copies back exactly that many results.  When all three host
 * arrays are pinned and len >= 32 MB, the text is cut at separators into
 * segments (at least four, of at most about 32 MB; on texts of 64 MB and
 * more the last three shrink to 16, 8 and 4 MB, so that little is left to
 * do after the last bytes arrive) whose copies in, parses and copies out
 * overlap, each segment's count written by its parse kernel into pinned
 * host memory (results identical).  Synchronous: returns after the
 * results are in host memory.  The staging buffers are allocated with
 * cudaMalloc on first use and grown as needed.
 */
FP_API fp_err_t fp_parse_f64_host(const char *host_text, size_t len, char delim,
                                  double *host_f64, uint8_t *host_status, uint64_t *host_count,
                                  struct CUstream_st *stream);

/*
 * fp_parse_f64_noalloc -- fp_parse_f64 for callers that must not allocate.
 *   (The paper has no counterpart: this is a deployment variant of the same
 *   parse.)  Same arguments, results and asynchrony as fp_parse_f64, but no
 *   call ever allocates memory: the scratch of the two kernels lives in one
 *   fixed 2 MiB + 256 B device array inside the library, which every GPU that
 *   loads the library holds until the process exits.  It is for callers that
 *   may not allocate once running -- fixed-memory or certified processes,
 *   plugins whose host owns all allocations, services that must not fail on
 *   an allocation mid-request.
 *   Limits: len < 2^40 (else FP_ERR_ARG), and at most 65,536 chunks of the
 *   current chunk size (len + (text % 16) <= 65,536 * chunk_bytes: 1 GiB at
 *   the default 16 KiB chunks; texts below 4 MB use 4 KiB chunks, as
 *   fp_parse_f64 does); beyond that it returns FP_ERR_CAPACITY.  Both checks
 *   come before any CUDA call, so a refused call queues nothing.  The first
 *   call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) and the launch shape.  Under CUDA's lazy module
 *   loading (CUDA_MODULE_LOADING=LAZY, the default) the library's device
 *   code, and with it the array, is loaded on a device only when first used,
 *   which can allocate device memory at that moment: a caller that must not
 *   allocate once running makes one call (len 0 is enough) on each device at
 *   start-up, or runs with CUDA_MODULE_LOADING=EAGER.  Later calls allocate
 *   nothing.
 *   Every call on every stream shares the one array and clears its control
 *   part on `stream` first: calls whose work overlaps on the GPU (different
 *   streams without ordering) race and give wrong results.  Order them, or
 *   use fp_parse_f64.  Device-side error conditions of these calls are not
 *   reported (fp_get_error does not see them); path counters are not kept.
 */
FP_API fp_err_t fp_parse_f64_noalloc(const char *text, size_t len, char delim, double *out_f64,
                                     uint8_t *out_status, uint64_t *out_count,
                                     struct CUstream_st *stream);

/* fp_shutdown -- synchronise and free every stream's scratch. */
FP_API fp_err_t fp_shutdown(void);

/* fp_strerror -- static text for an fp_err_t. */
FP_API const char *fp_strerror(fp_err_t err);

#ifdef __cplusplus
}
#endif
#endif /* FPPARSE_H */
