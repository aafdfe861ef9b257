/* lopc.h -- C ABI of the B300 (sm_103a) implementation of the hot path of the
 * Local-Order-Preserving Compressor (LOPC): error-bounded quantization, local-order
 * repair (subbins), lossless coding of bins and subbins, and decompression.
 *
 * The operations follow "Fast Topology-Aware Lossy Data Compression with Full
 * Preservation of Critical Points and Local Order":
 *   - problem statement, ABS and NOA bounds ..................... Sec. III-A
 *   - half-width quantizer, bins and subbins ..................... Sec. III-A
 *   - flags and subbin repair (Algorithms 1, 2) .................. Sec. III-B, III-D
 *   - termination, minimality, resolution ........................ Sec. III-E
 *   - lossless coding: bins as a Lorenzo or 1D-difference residual, NB-mapped, then
 *     BIT.RZE_1 (the paper's DIFFNB.BIT.RZE_1 is the 1D case); subbins BIT.RZE_w.RZE_1;
 *     independent 16 KiB chunks ................................... Sec. III-C, II-C
 *   - decoding (bin, subbin) to a value .......................... Sec. III-D, III-E
 *   - the repair schedule: tiles, or the paper's worklist ........... Sec. III-D
 *   - verification: local order, critical points, false positives /
 *     negatives / types, error bound, PSNR ......................... Sec. II, Table III
 * Where the paper leaves a choice open (neighbourhood, tie-break direction, exact
 * quantizer arithmetic, stream layout), the library fixes one reading; the stream
 * layout is described in the project's design notes.
 *
 * Conventions for every entry point:
 *   - Device pointers ("d_" prefix) point to memory of the current CUDA device;
 *     host pointers ("h_" prefix, or plain) to host memory.  The caller owns every
 *     buffer; the library never allocates device memory on these paths.  A
 *     synchronising single-field call reads its few result bytes back through a
 *     small pinned host buffer that the library allocates once per host thread
 *     (cudaMallocHost; on failure it uses the stack instead).
 *     lopc_decompress_noalloc never does.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Work is stream-ordered.  Calls documented as "synchronising" wait for the
 *     stream once before returning, to report a size or a status.
 *   - Fields are dense, C order (slowest dimension first): dims[0] x dims[1] for 2D,
 *     dims[0] x dims[1] x dims[2] for 3D, float32 or float64 values.  The number of
 *     points must be below 2^32.
 *   - Every function returns a status (LOPC_OK or a negative LOPC_ERR_*); no C++
 *     exception crosses the ABI.  After an error the contents of outputs are
 *     unspecified; the workspace may be reused.
 */
#ifndef LOPC_H
#define LOPC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LOPC_API __attribute__((visibility("default")))
#else
#define LOPC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Stream format written by this library.  Format 2 codes each chunk's bins with a
 * Lorenzo residual or a 1D difference (bit 30 of the chunk's size entry); format 1
 * (1D difference only) is still read. */
#define LOPC_VERSION 2

/* Status codes. */
#define LOPC_OK 0
#define LOPC_ERR_INVALID_ARG (-1)   /* bad descriptor, null pointer, eb <= 0 or not finite */
#define LOPC_ERR_NONFINITE (-2)     /* NaN or +-Inf in the field */
#define LOPC_ERR_RANGE (-3)         /* |x|/eps too large for the bin words (2^30 f32, 2^52 f64) */
#define LOPC_ERR_CAPACITY (-4)      /* output buffer too small */
#define LOPC_ERR_CORRUPT (-5)       /* stream fails validation */
#define LOPC_ERR_NOT_CONVERGED (-6) /* repair round cap reached (only with a lowered cap) */
#define LOPC_ERR_CUDA (-7)          /* a CUDA runtime call failed */
#define LOPC_ERR_WORKSPACE (-8)     /* workspace missing or smaller than required */
#define LOPC_ERR_BUSY (-9)          /* serving engine full: no result slot or rerun-list room */

/* Element type and error-bound mode (Sec. III-A). */
#define LOPC_F32 0
#define LOPC_F64 1
#define LOPC_ABS 0 /* |x - x_hat| <= eb */
#define LOPC_NOA 1 /* |x - x_hat| <= eb * (max(x) - min(x)) */

typedef struct {
  int32_t dtype;   /* LOPC_F32 or LOPC_F64 */
  int32_t ndim;    /* 2 or 3 */
  int64_t dims[3]; /* slowest first; a 2D field uses dims[0..1] and dims[2] = 0 */
  int32_t mode;    /* LOPC_ABS or LOPC_NOA */
  int32_t reserved;
  double eb;       /* error bound, > 0 and finite */
} lopc_field_desc;

/* Worst-case stream size in bytes for a field (0 for an invalid descriptor): the
 * 128-byte header, the size table of the bin and subbin records of every 16 KiB chunk
 * (Sec. II-C), and each record at its raw size (Sec. III-C stores a record raw when
 * coding would not shrink it), padded to 16 bytes. */
LOPC_API size_t lopc_compress_bound(const lopc_field_desc* desc);

/* Device scratch bytes that lopc_compress needs for this field (0 if invalid): the
 * per-point subbins and neighbour masks of the repair (Alg. 1-2, Sec. III-B), the
 * repair's per-tile rounds state (Sec. III-D), and one record slot per chunk for
 * the bin and subbin coders (Sec. III-C). */
LOPC_API size_t lopc_compress_workspace_size(const lopc_field_desc* desc);

/* Compresses a field (Sec. III): resolves eps (NOA: from the value range), quantizes
 * every value to a bin of width eps (Sec. III-A), raises subbins to the least values
 * that keep every neighbour pair's order (Alg. 1-2, Sec. III-E), and encodes bins
 * and subbins chunk by chunk (Sec. III-C).
 *   d_x      field values (dtype, dims from desc), device memory, read only
 *   d_out    stream output, device memory, out_cap bytes (lopc_compress_bound is
 *            always enough); receives *out_size bytes
 *   out_size host pointer, receives the stream length
 *   d_ws     device workspace of ws_size >= lopc_compress_workspace_size bytes
 * Synchronising (one wait, to read the size and the status).
 * Errors: INVALID_ARG, NONFINITE, RANGE, CAPACITY, WORKSPACE, NOT_CONVERGED, CUDA. */
LOPC_API int lopc_compress(const lopc_field_desc* desc, const void* d_x, void* d_out, size_t out_cap,
                  size_t* out_size, void* d_ws, size_t ws_size, void* stream);

/* Reads the descriptor from the first 128 bytes of a stream held in HOST memory: the
 * field's dtype, dimensions, bound mode and eb (the inputs of the problem statement,
 * Sec. III-A), which size the decompression's output and workspace.
 * Errors: INVALID_ARG (null), CORRUPT (bad header). */
LOPC_API int lopc_peek(const void* h_stream, size_t n, lopc_field_desc* desc);

/* Device scratch bytes that lopc_decompress needs for streams of this field: a status
 * word and the byte offsets of every chunk's two records (Sec. II-C, III-C). */
LOPC_API size_t lopc_decompress_workspace_size(const lopc_field_desc* desc);

/* Decompresses a stream (Sec. III-D/E): decodes each chunk's bins and subbins and
 * writes x_hat = the subbin-th representable value above the lowest value of the
 * bin.  d_in/in_size: the stream in device memory; d_x: output field, x_cap bytes.
 * Synchronising (reads the 128-byte header to the host, then waits for the status).
 * Errors: INVALID_ARG, CORRUPT, CAPACITY, WORKSPACE, CUDA. */
LOPC_API int lopc_decompress(const void* d_in, size_t in_size, void* d_x, size_t x_cap, void* d_ws, size_t ws_size,
                    void* stream);

/* ---- batches (many fields, one launch sequence).  The fields' tiles share one
 * launch per kernel and one device-driven repair loop (a CUDA graph whose while-node
 * runs repair rounds until no tile is dirty), so a batch costs no host round trip
 * per round; each field's stream is byte-identical to its single-field stream.
 * Host arrays hold n entries; d_out_size and d_status are DEVICE arrays of n that
 * receive each field's stream length and status.  Asynchronous: nothing waits for
 * the stream; read the results after synchronising.  The workspace must not be used
 * by another call until this one has finished on the GPU.  A compression batch holds
 * at most LOPC_MAX_BATCH_FIELDS fields (the field index is a grid dimension of several
 * kernels): a larger n returns LOPC_ERR_INVALID_ARG, and its workspace size is 0. */
#define LOPC_MAX_BATCH_FIELDS 65535
LOPC_API size_t lopc_batch_compress_workspace_size(int n, const lopc_field_desc* descs);

/* Launch plan of a batched compression (the paper compresses one field per call
 * and has no counterpart).  Four entries per array, one per field class: 0 float32
 * 2D, 1 float32 3D, 2 float64 2D, 3 float64 3D.  Output bytes never depend on it:
 * the repair reaches the same least fixpoint under every schedule (Sec. III-E).
 *   rerun_blocks_per_sm  persistent blocks per SM of the repair rounds, [1, 16];
 *   pass_budget16        frontier evaluations a tile of the tile pass may spend, in
 *                        sixteenths of its points, before it finishes in topological
 *                        order, [1, 4096];
 *   pass_dense16         same-bin neighbour pairs, in sixteenths of a full tile's
 *                        pairs, above which a tile goes to topological order at
 *                        once, [0, 17] (17 = never);
 *   pass_order           order of the tile pass: 0 decided per field from its tiles'
 *                        sampled bin spans, 1 tile index order, 2 ascending tile key.
 * Out-of-range values are clamped. */
typedef struct {
  int32_t rerun_blocks_per_sm[4];
  int32_t pass_budget16[4];
  int32_t pass_dense16[4];
  int32_t pass_order[4];
} lopc_plan;

/* The library's default plan, and this thread's current one (the lopc_tune_*
 * settings, which the autotuner writes). */
LOPC_API void lopc_plan_default(lopc_plan* plan);
LOPC_API void lopc_plan_get(lopc_plan* plan);

/* Compresses n fields (the per-field operation of lopc_compress, Sec. III) in one
 * launch sequence.  d_x, d_out, out_cap: n entries each (host arrays of device
 * pointers and capacities); d_out_size, d_status: DEVICE arrays of n.  plan: the
 * launch plan, or NULL for this thread's current plan (lopc_plan_get).
 * Errors (returned): INVALID_ARG, WORKSPACE, CUDA; per field (in d_status): OK,
 * NONFINITE, RANGE, CAPACITY, NOT_CONVERGED. */
LOPC_API int lopc_batch_compress(int n, const lopc_field_desc* descs, const void* const* d_x, void* const* d_out,
                                 const size_t* out_cap, uint64_t* d_out_size, int* d_status,
                                 const lopc_plan* plan, void* d_ws, size_t ws_size, void* stream);

/* Decompresses n streams (descs from lopc_peek of each header) into d_x[i]; each
 * stream's status goes to the DEVICE array d_status.  Asynchronous.  A stream whose
 * header does not match its descriptor (dtype, ndim, dims or chunk count) is reported
 * as CORRUPT and leaves d_x[i] unwritten. */
LOPC_API size_t lopc_batch_decompress_workspace_size(int n, const lopc_field_desc* descs);
LOPC_API int lopc_batch_decompress(int n, const lopc_field_desc* descs, const void* const* d_in,
                                   const size_t* in_size, void* const* d_x, int* d_status, void* d_ws,
                                   size_t ws_size, void* stream);

/* Decompression that allocates nothing and takes no workspace (the paper has no
 * counterpart; this is a library convenience).  It is meant for callers that cannot
 * call cudaMalloc: code running inside a memory allocator's callbacks, under a host
 * framework that reserves all device memory up front, or on paths that must not
 * take the driver's allocation locks.  Same arguments and result as
 * lopc_decompress minus the workspace.
 *   - Scratch lives in a fixed device array of the library (1 MiB + 256 bytes on
 *     every GPU that loads it, held until the process exits), so streams of at most
 *     lopc_noalloc_max_chunks() chunks (65536: 256 Mi float32 or 128 Mi float64
 *     points) are accepted; larger ones return LOPC_ERR_WORKSPACE before any work.
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress); the first call on a device also loads the library's
 *     device code there, so make that first call before any stream capture.
 *   - All calls share the array: calls whose work overlaps on the GPU (other streams,
 *     other host threads) race and must be serialised by the caller.  Every call,
 *     failed ones included, returns with its work on the array finished.
 * Synchronising.  Errors: INVALID_ARG, CORRUPT, CAPACITY, WORKSPACE, CUDA. */
LOPC_API int lopc_decompress_noalloc(const void* d_in, size_t in_size, void* d_x, size_t x_cap, void* stream);

/* Largest chunk count lopc_decompress_noalloc accepts. */
LOPC_API int64_t lopc_noalloc_max_chunks(void);

/* Runs the quantizer and the repair only and exports their results, for testing
 * each stage against a reference: d_bins[i] (int64) and d_subbins[i] (uint64), one
 * per point in C order.  Same workspace as lopc_compress.  Synchronising.
 * Errors: as lopc_compress (no CAPACITY). */
LOPC_API int lopc_quantize_repair(const lopc_field_desc* desc, const void* d_x, int64_t* d_bins, uint64_t* d_subbins,
                         void* d_ws, size_t ws_size, void* stream);

/* ---- verification.  What a reconstruction y keeps of the field x, in one pass over
 * both on the GPU:
 *   - the local order of Sec. II: neighbour pairs (Freudenthal neighbourhood, each
 *     pair once) whose order differs, ties broken by the lower index in each field;
 *   - critical points (Sec. II): every point of x and of y is a minimum (empty lower
 *     link), else a maximum (empty upper link), else regular (one lower and one upper
 *     link piece), else a saddle; link pieces are connected in the triangulation;
 *   - Table III's counts: false positives (regular in x, critical in y), false
 *     negatives (critical in x, regular in y), false types (critical in both with
 *     another class); link_mismatches: points whose pair (lower pieces, upper pieces)
 *     differs, which also catches a saddle of another multiplicity;
 *   - the error bound of Sec. III-A: max |x - y| and eps = eb (ABS) or
 *     eb * (max(x) - min(x)) (NOA), in binary64; and the PSNR,
 *     20 log10(max(x) - min(x)) - 10 log10(mse), +inf when mse = 0.
 * Integer counts and max_abs_err are exact; mse (and so psnr) is a sum in a fixed
 * order, deterministic on a given GPU; for float32 fields the squares are summed in
 * float32 over at most 16 points before binary64 (relative error below 2e-6). */
typedef struct {
  int64_t points;
  int64_t order_violations;
  int64_t cp_x[4];          /* minima, maxima, saddles, regular points of x */
  int64_t cp_y[4];          /* the same for y */
  int64_t false_positives;
  int64_t false_negatives;
  int64_t false_types;
  int64_t link_mismatches;
  int64_t nonfinite;        /* points where x or y is NaN or infinite */
  double x_min, x_max;
  double max_abs_err;       /* max |x - y| */
  double mse;               /* mean (x - y)^2 */
  double psnr;
  double eps;               /* the bound of desc (mode, eb) for x */
  int32_t bound_ok;         /* max_abs_err <= eps */
  int32_t reserved;
} lopc_verify_report;

/* Device scratch bytes that lopc_verify needs (0 for an invalid descriptor). */
LOPC_API size_t lopc_verify_workspace_size(const lopc_field_desc* desc);

/* Compares d_y (a reconstruction) with d_x, both fields described by desc (the
 * bound fields mode and eb give report.eps), and writes the report to h_report
 * (host).  d_types_x, if not NULL, receives one byte per point of x in C order:
 * the number of lower-link pieces | the number of upper-link pieces << 4 (Sec. II);
 * d_types_y the same for y (only together with d_types_x).  The workspace must be
 * 256-byte aligned.  Synchronising.
 * Errors: INVALID_ARG, WORKSPACE, CUDA; NONFINITE when x or y holds NaN or an
 * infinity (the report is filled, with the count in report.nonfinite). */
LOPC_API int lopc_verify(const lopc_field_desc* desc, const void* d_x, const void* d_y, uint8_t* d_types_x,
                         uint8_t* d_types_y, lopc_verify_report* h_report, void* d_ws, size_t ws_size,
                         void* stream);

/* Repair schedules of the single-field calls (lopc_compress, lopc_quantize_repair):
 *   LOPC_REPAIR_TILES (default): tile-local fixpoints in shared memory, then reruns of
 *     the tiles whose halo rose, in device-driven rounds;
 *   LOPC_REPAIR_WORKLIST: the paper's schedule (Sec. III-D, Alg. 2): from subbins 0,
 *     one thread per worklist point, atomicMax raises, the greater same-bin neighbours
 *     of a raised point on the next worklist (deduplicated by an iteration stamp).
 * Both reach the same least fixpoint, so streams are identical.  The worklist mode
 * needs 12 more workspace bytes per point: query lopc_compress_workspace_size after
 * setting the mode.  Batches and the serving engine always use tiles.  Per thread;
 * returns the previous mode, or INVALID_ARG for an unknown one. */
#define LOPC_REPAIR_TILES 0
#define LOPC_REPAIR_WORKLIST 1
LOPC_API int lopc_set_repair_mode(int mode);

/* Caps the number of repair rounds after the first (all-tile) round for later calls
 * on this thread (0 restores the default, which a valid field never reaches).  A
 * lowered cap makes lopc_compress return LOPC_ERR_NOT_CONVERGED.  Returns the
 * previous cap. */
LOPC_API int64_t lopc_set_round_cap(int64_t cap);

/* Statistics of the last lopc_compress on this thread: repair rounds and tile runs
 * (first pass plus reruns).  Either pointer may be NULL. */
LOPC_API void lopc_last_stats(int64_t* rounds, int64_t* tile_runs);

/* Statistics of the last compression on this thread: block-wide sweeps of the
 * tile-local fixpoint summed over all tile runs, and the largest count of one run. */
LOPC_API void lopc_last_fixpoint_stats(int64_t* sweeps_total, int64_t* sweeps_max);

/* Measurement aid: SM cycles of the last compression on this thread, summed over
 * blocks, per phase: 0 tile load + quantization, 1 flags, 2 tile fixpoint, 3 state
 * write-back, 4 bin record, 5 rerun load and check, 6 rerun fixpoint, 7 rerun load and check of
 * tiles whose constraints all held, 8 rerun write-back and marking.
 * Copies min(n, 9) values and returns 9. */
LOPC_API int lopc_last_phase_cycles(int64_t* cycles, int n);

/* Measurement aid: tiles listed for each repair round after the first (all-tile)
 * round, in the last compression on this thread that ran with per-kernel timing on
 * (the host-driven loop); the last entry is the empty list that ended the repair.
 * Copies min(n, rounds) values and returns the number of rounds. */
LOPC_API int lopc_last_round_tiles(int64_t* out, int n);

/* Measurement aid: work of the tile-local fixpoint in the last compression on this
 * thread: point evaluations and subbin raises in the tile pass, then the same in
 * the reruns, then the rerun tiles loaded and how many of them found every
 * constraint into the tile holding (check only), then 1 if the tile pass took the
 * tiles in tile-key order (lopc_tune_set_pass_order), else 0.  Copies min(n, 7)
 * values and returns 7. */
LOPC_API int lopc_last_fixpoint_work(int64_t* out, int n);

/* Measurement aid: while enabled, the decoder adds up SM cycles per phase over all
 * blocks of the current device: 0 bin record RZE, 1 bin planes + prefix sum, 2 bin
 * range and lowest-value cache, 3 subbin RZE_1, 4 subbin RZE_w, 5 planes + values.
 * lopc_decode_phase_read synchronises the device, copies min(n, 8) sums, resets them
 * and returns 8 (or a negative status). */
LOPC_API int lopc_decode_phase_enable(int on);
LOPC_API int lopc_decode_phase_read(int64_t* out, int n);

/* Per-kernel timing for measurement: while enabled, every kernel the library
 * launches is bracketed by CUDA events recorded on the launching stream, and the
 * elapsed times are added up per kernel when the call returns.  Off by default;
 * state is per thread.  lopc_profile_read copies up to `cap` entries (kernel name,
 * launches, total milliseconds) and returns the number of kernels seen. */
LOPC_API void lopc_profile_enable(int on);
LOPC_API void lopc_profile_reset(void);
LOPC_API int lopc_profile_read(const char** names, int64_t* launches, double* total_ms, int cap);
/* The times of every timed launch of one kernel (by the name lopc_profile_read
 * reports), in launch order: copies up to `cap` and returns how many there are. */
LOPC_API int lopc_profile_read_launches(const char* name, double* ms, int cap);

/* ---- serving engine (round-level continuous batching; the paper compresses one
 * field per call and has no counterpart).  Fields are submitted as they arrive and
 * join the repair between rounds: each lopc_engine_step runs `rounds` repair rounds
 * (compaction of the dirty tiles, then their reruns) over every field in repair on
 * the engine's rounds stream, while on its aux stream it runs the tile pass and the
 * first round of the fields submitted since the last step, and encodes and packs
 * the fields whose last compaction found no dirty tile.  A field's state stays in
 * its own workspace from submit to completion; its stream is byte-identical to
 * lopc_compress's.  One host thread drives an engine.
 *
 * Create: max_fields result slots and room for max_tiles tiles of fields in repair
 * (chunk tiles: 4096 float32 or 2048 float64 points each); allocates its tables and
 * two streams once.  Errors: INVALID_ARG, CUDA. */
typedef struct lopc_engine lopc_engine;
LOPC_API int lopc_engine_create(int max_fields, int64_t max_tiles, lopc_engine** out);

/* Waits for the engine's streams and frees it; fields still in flight are dropped. */
LOPC_API void lopc_engine_destroy(lopc_engine* e);

/* Device bytes of the per-field state that lopc_engine_submit needs (0 if invalid). */
LOPC_API size_t lopc_engine_field_workspace_size(const lopc_field_desc* desc);

/* Queues one field.  d_x, d_out (out_cap bytes) and d_ws (ws_size bytes, 256-byte
 * aligned) are device memory owned by the caller and must stay valid until
 * lopc_engine_poll reports `tag`.  The engine's work on the field waits for
 * everything enqueued so far on ready_stream (the stream that produced d_x).
 * Errors: INVALID_ARG, WORKSPACE, BUSY (no slot or list room: retry after a poll),
 * CUDA. */
LOPC_API int lopc_engine_submit(lopc_engine* e, const lopc_field_desc* desc, const void* d_x, void* d_out,
                                size_t out_cap, void* d_ws, size_t ws_size, uint64_t tag, void* ready_stream);

/* One engine step (see above).  Blocks only until the step's last compaction has
 * been read back; its rerun round is still running when it returns.  *active
 * (may be NULL) receives the number of fields submitted and not yet polled.
 * Errors: INVALID_ARG, CUDA. */
LOPC_API int lopc_engine_step(lopc_engine* e, int rounds, int* active);

/* Non-blocking: copies up to cap finished fields (tag, stream length, status: OK,
 * NONFINITE, RANGE, CAPACITY, NOT_CONVERGED) and returns how many; their buffers
 * are the caller's again.  Returns a negative status on error. */
LOPC_API int lopc_engine_poll(lopc_engine* e, uint64_t* tags, uint64_t* sizes, int* statuses, int cap);

/* Waits until all work enqueued by the engine has finished on the GPU. */
LOPC_API int lopc_engine_sync(lopc_engine* e);

/* ---- launch tuning.  Persistent rerun blocks per SM for each field class (0 f32
 * 2D, 1 f32 3D, 2 f64 2D, 3 f64 3D), used by later calls on this thread; values are
 * clamped to [1, 16].  Output bytes never depend on them.  lopc_tune_get copies
 * the current four values. */
LOPC_API void lopc_tune_set(const int* rerun_blocks_per_sm);
LOPC_API void lopc_tune_get(int* rerun_blocks_per_sm);

/* Launch tuning of the tile pass's fixpoint, per field class; later calls on this
 * thread use it and output bytes never depend on it.  A tile whose same-bin
 * neighbour pairs exceed dense/16 of a full tile's pairs is solved in topological
 * order at once (default 8; 17 = never; clamped to [0, 17]); any other tile runs
 * frontier sweeps until they have spent budget/16 evaluations per point (default 64;
 * clamped to [1, 4096]) and then finishes in topological order. */
LOPC_API void lopc_tune_set_budget(const int* sixteenths);
LOPC_API void lopc_tune_get_budget(int* sixteenths);
LOPC_API void lopc_tune_set_dense(const int* sixteenths);
LOPC_API void lopc_tune_get_dense(int* sixteenths);

/* Order in which the tile pass takes a field's tiles, per field class; later calls on
 * this thread use it and output bytes never depend on it.  0 (default): by the field,
 * as in 2 when the bins its tiles' samples span (each tile clamped at 256) average
 * below 48, else as in 1.  1: tile index order, each tile's fixpoint starting from
 * halo subbins 0.  2: ascending tile key (the rerun order), each tile's fixpoint
 * starting from the subbins its earlier neighbour tiles have written.  Clamped to
 * [0, 2]. */
LOPC_API void lopc_tune_set_pass_order(const int* modes);
LOPC_API void lopc_tune_get_pass_order(int* modes);

/* Human-readable text of a status code (static storage). */
LOPC_API const char* lopc_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* LOPC_H */
