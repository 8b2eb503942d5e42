/*
 * szx.h -- C ABI of the B300 (sm_103a) SZx block compressor / decompressor.
 *
 * The codec is the ultra-fast error-bounded lossy compressor of Yu et al.,
 * "SZx: an Ultra-fast Error-bounded Lossy Compressor for Scientific Datasets"
 * (arXiv 2201.13020).  The problem it solves is stated in Sec. III, Eq. 1:
 * given N values d_i and an absolute error bound e, produce a byte stream whose
 * decompression d'_i satisfies |d_i - d'_i| <= e for every i, as fast as
 * possible (compression and decompression throughput, Eq. 2 and Eq. 3, count
 * input bytes N * b per second).
 *
 * Method (Sec. IV, Algorithm 1): the array is cut into consecutive blocks of
 * `block` values (128 by default, Sec. V-A.2).  A block whose values all lie
 * within e of mu, the mean of its min and max, is "constant" and stores only
 * mu.  Other blocks are normalised by mu, each value keeps the bits Eq. 4
 * requires, right-shifted by Eq. 5 so they fill whole bytes, and only the bytes
 * that differ from the previous value ("mid-bytes") are stored, with a 2-bit
 * code per value counting the identical leading bytes.
 *
 * Conventions for every call below:
 *   - Pointers named d_* are CUDA device pointers on the current device and
 *     must be 16-byte aligned; the caller allocates and owns all of them.
 *     No compress or decompress call allocates memory: the compress calls
 *     keep their scratch in the tail of the caller's output buffer (see
 *     szx_compress_bound) or, for szx_compress_static_async, in a fixed array
 *     inside the library; the synchronous szx_decompress takes its status
 *     word from another fixed array inside the library.  (The batch planning
 *     calls and szx_server_create allocate host memory, and the server its
 *     own small status words, as documented there.)
 *   - `stream` is a cudaStream_t (0 = the legacy default stream).  All device
 *     work is enqueued on it in order.
 *   - Values are IEEE 754 binary32 (SZX_F32) or binary64 (SZX_F64), little
 *     endian, contiguous.
 *   - `block` is the block length b: a power of two in [32, 1024].
 *   - `eb` is the absolute error bound: finite and > 0.  For SZX_F32 the bound
 *     used is the largest float <= eb.  (A value-range relative bound REL of
 *     the paper, Sec. IV footnote, is REL * (max - min), computed by the caller.)
 *   - Every call returns a szx_status and never aborts the process.  On an
 *     error the contents of the output buffer are unspecified.
 *   - The compressed stream is deterministic: the same input, dtype, eb and
 *     block give the same bytes on every run and every launch configuration.
 */
#ifndef SZX_H
#define SZX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { SZX_F32 = 0, SZX_F64 = 1 } szx_dtype;

typedef enum {
    SZX_OK = 0,
    SZX_ERR_INVALID = 1,     /* bad argument (null, misaligned, eb, block, n) */
    SZX_ERR_TOO_SMALL = 2,   /* output capacity below what the call needs */
    SZX_ERR_CORRUPT = 3,     /* compressed input is malformed or truncated */
    SZX_ERR_NOMEM = 4,       /* a planning call could not allocate host memory */
    SZX_ERR_CUDA = 5,        /* a CUDA runtime call failed */
    SZX_ERR_TIMEOUT = 6      /* a bounded device-side wait ran out */
} szx_status;

/* Opaque CUDA stream handle (binary-compatible with cudaStream_t). */
typedef struct CUstream_st *szx_stream_t;

/* Parsed 64-byte stream header. */
typedef struct {
    uint32_t block;        /* b */
    uint32_t tile_blocks;  /* G: blocks per tile record */
    uint64_t n;            /* number of values */
    szx_dtype dtype;
    uint64_t e_bits;       /* bit pattern of the bound used (f32 in the low 32 bits) */
    uint64_t nonconst;     /* non-constant blocks, raw ones included */
    uint64_t raw;          /* blocks stored verbatim */
    uint64_t escalated;    /* blocks whose reqBits grew past Eq. 4 to meet e */
    uint64_t total_bytes;  /* stream size */
} szx_header;

/*
 * Bytes the output buffer of szx_compress / szx_compress_async must hold for n
 * values: the largest possible stream (every block stored verbatim plus the
 * per-block metadata) followed by the call's device scratch space (tile
 * tickets and the look-back status words of the offset scan).  Returns 0 for
 * invalid arguments.  Host-only; no CUDA call.
 * Paper: Algorithm 1 stores either mu_k alone (constant block) or a block's
 * lead codes and mid bytes, and the mid bytes of a value are at most its
 * whole width (Eq. 4 clamps R_k at the mantissa width); the bound is that
 * worst case, every block kept verbatim, plus the per-block metadata of the
 * stream layout.
 */
size_t szx_compress_bound(size_t n, szx_dtype dtype, uint32_t block);

/* Largest possible stream size alone (no scratch tail).  Host-only. */
size_t szx_stream_max_bytes(size_t n, szx_dtype dtype, uint32_t block);

/*
 * Compress n values at d_in into the stream at d_out (Algorithm 1 with the
 * Eq. 4 / Eq. 5 byte-aligned packing; Sec. V-B for the GPU design it
 * replaces).  out_capacity must be >= szx_compress_bound(n, dtype, block).
 * On SZX_OK, *out_bytes holds the stream size; the stream occupies
 * d_out[0 .. *out_bytes), and the bytes after it up to out_capacity are
 * scratch that the call overwrote.  Synchronous: returns after the stream
 * and its size are complete (one small device-to-host copy and a stream
 * synchronisation).  Errors: SZX_ERR_INVALID, SZX_ERR_TOO_SMALL, SZX_ERR_CUDA,
 * SZX_ERR_TIMEOUT.
 */
szx_status szx_compress(const void *d_in, size_t n, szx_dtype dtype, double eb,
                        uint32_t block, void *d_out, size_t out_capacity,
                        size_t *out_bytes, szx_stream_t stream);

/*
 * Asynchronous form of szx_compress: enqueues the work and returns without
 * synchronising.  When the work completes, d_result[0] holds the stream size
 * and d_result[1] a szx_status (SZX_OK or SZX_ERR_TIMEOUT); d_result is a
 * device (or mapped pinned) pointer to two uint64_t, or NULL.  The stream size
 * is also in the stream header (bytes 56..63).  Safe to capture in a CUDA
 * graph.  Host-side argument errors are returned immediately.
 */
szx_status szx_compress_async(const void *d_in, size_t n, szx_dtype dtype,
                              double eb, uint32_t block, void *d_out,
                              size_t out_capacity, uint64_t *d_result,
                              szx_stream_t stream);

/*
 * Size of the fixed device array that szx_compress_static_async uses as its
 * scratch, and the largest tile count it accepts: a 128-byte header plus one
 * 8-byte look-back word per tile.  Every tile holds at least 32 KiB of input,
 * so the limit admits any input of up to 131056 * 32 KiB (about 4 GiB).
 */
#define SZX_STATIC_SCRATCH_BYTES (1u << 20)
#define SZX_STATIC_MAX_TILES ((SZX_STATIC_SCRATCH_BYTES - 128u) / 8u)

/*
 * Compression that allocates nothing: the paper has no counterpart; it is
 * an interface variant of szx_compress_async for callers whose output buffer
 * is exactly szx_stream_max_bytes(n, dtype, block) long and who may not
 * allocate scratch space.  The stream it writes is byte-identical to
 * szx_compress_async's for the same arguments.
 *
 * d_in, n, dtype, eb, block, d_out, d_result, stream: as szx_compress_async.
 * out_capacity must be >= szx_stream_max_bytes(n, dtype, block); nothing past
 * the stream's own bytes is written.  The look-back scratch is one array of
 * SZX_STATIC_SCRATCH_BYTES inside the library, per device; no call allocates
 * device or host memory.
 *
 * Set-up: the first call made with a given device current looks up that
 * device's array address (cudaGetSymbolAddress, which may load the
 * library's device code) and keeps it; make that first call before any
 * stream capture.  A cudaDeviceReset (or any other destruction of the
 * device's primary context) between calls is not supported: the kept
 * address would be stale.  Each call clears the array prefix it uses on
 * `stream` before its kernel.
 *
 * Sharing: all calls on one device use the same array.  Calls that can
 * overlap in time (on different streams, or from different host threads
 * without ordering) race on it and produce undefined streams; order them.
 *
 * Errors (returned immediately): SZX_ERR_INVALID for the same argument errors
 * as szx_compress_async and for an input whose tile count exceeds
 * SZX_STATIC_MAX_TILES; SZX_ERR_TOO_SMALL if out_capacity is below
 * szx_stream_max_bytes; SZX_ERR_CUDA if a CUDA call fails.  Device-side
 * results arrive in d_result as for szx_compress_async.
 */
szx_status szx_compress_static_async(const void *d_in, size_t n,
                                     szx_dtype dtype, double eb,
                                     uint32_t block, void *d_out,
                                     size_t out_capacity, uint64_t *d_result,
                                     szx_stream_t stream);

/*
 * Read and check the 64-byte header of the stream at d_in (device pointer;
 * one 64-byte device-to-host copy, synchronous on `stream`).  Errors:
 * SZX_ERR_INVALID (null), SZX_ERR_CORRUPT (bad magic, version, dtype, block,
 * tile size, or total_bytes > in_bytes), SZX_ERR_CUDA.
 * Paper: the header carries what decompression needs besides the blocks
 * (Sec. III's problem: N, the value type and e; Sec. V-A.2's block size b);
 * the paper fixes no byte layout, so the fields and their order are this
 * library's (little endian: magic, version, dtype, b, blocks per tile, n, the
 * bits of e, counts of non-constant, raw and escalated blocks, total bytes).
 */
szx_status szx_header_read(const void *d_in, size_t in_bytes, szx_header *h,
                           szx_stream_t stream);

/*
 * Decompress the stream d_in[0 .. in_bytes) into d_out (n values of the
 * stream's dtype; out_capacity >= n * 4 or n * 8 bytes).  *n_out and
 * *dtype_out receive the header's values (either may be NULL).  Every read
 * of the stream is bounds-checked on the device; a malformed stream returns
 * SZX_ERR_CORRUPT.  Synchronous (one 64-byte header read, the status clear
 * and the kernel, one 4-byte status read).  Allocates nothing: its device status word is one of
 * 256 words of a fixed array inside the library, taken round-robin, so that
 * up to 256 calls in flight at once (from different host threads) get
 * distinct words.
 * Paper: the inverse of Algorithm 1 -- a constant block decodes to mu_k; a
 * non-constant block rebuilds each truncated word from its lead code (the
 * identical leading bytes come from the previous value) and its mid bytes,
 * undoes the Eq. 5 shift and adds mu_k (d'_i = RN((t_i << s) + mu_k)); Sec.
 * V-B describes the GPU decoder whose prefix scan the tile index replaces.
 */
szx_status szx_decompress(const void *d_in, size_t in_bytes, void *d_out,
                          size_t out_capacity, size_t *n_out,
                          szx_dtype *dtype_out, szx_stream_t stream);

/*
 * Asynchronous decompression of a stream whose header the caller already
 * holds (from szx_header_read, or from the compressing side).  The kernel
 * re-checks the stream's header against *h.  On completion *d_status (device
 * pointer, may be NULL) holds a szx_status; the call sets it to SZX_OK first.
 * Safe to capture in a CUDA graph.  Errors returned at once: SZX_ERR_INVALID
 * (null or misaligned pointers, a header with an invalid dtype, block, n or
 * tile size), SZX_ERR_CORRUPT (total_bytes outside [sections, in_bytes]),
 * SZX_ERR_TOO_SMALL (out_capacity), SZX_ERR_CUDA.
 * Paper: as szx_decompress (the inverse of Algorithm 1; Sec. V-B).
 */
szx_status szx_decompress_async(const void *d_in, size_t in_bytes,
                                const szx_header *h, void *d_out,
                                size_t out_capacity, uint32_t *d_status,
                                szx_stream_t stream);

/* ------------------------------------------------------------------------
 * Batches: many fields in few launches.  The paper has no batch interface; it
 * is a throughput form of szx_compress / szx_decompress for many independent
 * arrays (Sec. III's problem applied to each).  Streams and decoded values are
 * byte-identical to the single-field calls'.
 *
 * Life cycle: plan (host only) -> szx_batch_workspace_bytes -> szx_batch_upload
 * (writes the plan's descriptor tables into the caller's device workspace;
 * synchronous on `stream`) -> szx_batch_run any number of times (enqueues one
 * small kernel that clears the plan's counters and, for decompression, every
 * stream's status word, then one persistent kernel launch per (dtype, block)
 * group, no host synchronisation; the same sequence can be captured in a CUDA
 * graph) ->
 * szx_batch_destroy.  A plan remembers the workspace it was uploaded to;
 * running it with another one returns SZX_ERR_INVALID.  Buffers named in the
 * fields must stay valid while the plan is run; runs of one plan must not
 * overlap in time (they share the workspace).
 * ------------------------------------------------------------------------ */

/* One field to compress: as the arguments of szx_compress_async, except that
 * block may be 0: szx_batch_autotune then chooses b among 64, 128 and 256 for
 * the plan's block-0 fields of each dtype together (128 until it runs), and
 * out_capacity must hold the largest stream of the three. */
typedef struct {
    const void *d_in;    /* n values, 16-byte aligned */
    size_t n;
    szx_dtype dtype;
    double eb;           /* absolute bound, finite and > 0 */
    uint32_t block;      /* power of two in [32, 1024], or 0 (see above) */
    void *d_out;         /* the field's stream, 16-byte aligned */
    size_t out_capacity; /* >= szx_stream_max_bytes(n, dtype, block) */
} szx_field;

/* One stream to decompress. */
typedef struct {
    const void *d_in;    /* the stream, 16-byte aligned */
    size_t in_bytes;
    szx_header header;   /* its header (szx_header_read, or the compressing side) */
    void *d_out;         /* n values, 16-byte aligned */
    size_t out_capacity; /* >= n * 4 or n * 8 bytes */
    uint32_t *d_status;  /* device word for the stream's szx_status, or NULL */
} szx_stream_field;

typedef struct szx_batch_plan szx_batch_plan; /* opaque, host memory */

/* Plan the compression of `count` fields (host only; allocates host memory).
 * Errors: SZX_ERR_INVALID (a field's arguments, as for szx_compress_async),
 * SZX_ERR_TOO_SMALL (a field's out_capacity), SZX_ERR_NOMEM. */
szx_status szx_batch_compress_plan(const szx_field *fields, int count,
                                   szx_batch_plan **plan);

/* Plan the decompression of `count` streams (host only).  Errors:
 * SZX_ERR_INVALID, SZX_ERR_CORRUPT (header inconsistent with in_bytes),
 * SZX_ERR_TOO_SMALL, SZX_ERR_NOMEM.  Every stream is still checked on the
 * device; its status word receives SZX_ERR_CORRUPT if it is malformed. */
szx_status szx_batch_decompress_plan(const szx_stream_field *streams, int count,
                                     szx_batch_plan **plan);

/* Device workspace bytes the plan needs (0 for a NULL plan). */
size_t szx_batch_workspace_bytes(const szx_batch_plan *plan);

/* Write the plan's tables into d_ws (device, 256-byte aligned, at least
 * szx_batch_workspace_bytes).  d_results (compression plans): device array of
 * 2 * count uint64_t receiving {stream bytes, szx_status} per field, in the
 * caller's field order, after each run; may be NULL (the sizes are also in
 * each stream's header).  Synchronous on `stream`. */
szx_status szx_batch_upload(szx_batch_plan *plan, void *d_ws, size_t ws_bytes,
                            uint64_t *d_results, szx_stream_t stream);

/* Enqueue one run of the plan on `stream`. */
szx_status szx_batch_run(const szx_batch_plan *plan, void *d_ws,
                         szx_stream_t stream);

/* Autotuner.  Per group, time runs of that group alone on `stream` in every
 * shape the kernels have and keep the fastest in the plan:
 *   - consumer (decoding) warps per CTA: 8, or 4 where a block still covers
 *     whole lanes (f32 with b >= 64, f64 with b <= 512); with 4 warps each lane
 *     holds twice the values and each warp twice the blocks (threads per CTA
 *     = 32 * warps + 64; a tile is always 32 KiB of values, 64 KiB for f64
 *     with b = 1024, so the stream does not change);
 *   - CTAs per SM: 2 or 1;
 *   - for a compression group of block-0 fields, the block length b among 64,
 *     128 and 256 (this changes the stream): among the lengths whose fastest
 *     time is within 2% of the fastest overall, the one whose streams are the
 *     smallest (the best compression ratio, Sec. V-A.2's trade-off).
 * Runs the plan's own work, so it overwrites the outputs (with the bytes of
 * the chosen shape), and re-uploads the tables if b changes.  Synchronous.
 * The paper has no counterpart (it fixes b = 128 by its Fig. 7 study). */
szx_status szx_batch_autotune(szx_batch_plan *plan, void *d_ws,
                              szx_stream_t stream);

/* Number of groups; writes up to `capacity` CTAs-per-SM choices (0 = as many
 * as fit) into ctas_per_sm (which may be NULL when capacity is 0). */
int szx_batch_groups(const szx_batch_plan *plan, int *ctas_per_sm, int capacity);

/* A group's shape. */
typedef struct {
    szx_dtype dtype;
    uint32_t block;            /* b (the tuner's choice for block-0 fields) */
    int auto_block;            /* 1: its fields were given block 0 */
    uint32_t fields;
    uint64_t tiles;
    int ctas_per_sm;           /* 0 = as many as fit */
    int warps_per_cta;         /* consumer (decoding) warps: 8 or 4 */
    uint32_t threads_per_cta;  /* 32 * warps_per_cta + 64 */
    uint32_t values_per_lane;  /* 32 or 64 (f32), 16 or 32 (f64) */
    uint32_t blocks_per_warp;  /* 32 * values_per_lane / b */
    float tuned_ms;            /* the tuner's time for the group, 0 if not tuned */
} szx_batch_group;

/* The shape of group `group` (0 .. szx_batch_groups - 1).  Errors:
 * SZX_ERR_INVALID. */
szx_status szx_batch_group_info(const szx_batch_plan *plan, int group, szx_batch_group *info);

/* Set a group's shape by hand (ctas_per_sm 0, 1 or 2; warps_per_cta 8 or 4
 * where the kernels have it).  Errors: SZX_ERR_INVALID. */
szx_status szx_batch_set_group(szx_batch_plan *plan, int group, int ctas_per_sm, int warps_per_cta);

void szx_batch_destroy(szx_batch_plan *plan);

/* ------------------------------------------------------------------------
 * Serving: requests that arrive over time, compressed streams resident in a
 * device memory pool (the paper has no serving interface; it is a request
 * form of szx_compress_async / szx_decompress_async).  A request is admitted,
 * oldest first, as soon as one of the server's slots (CUDA streams) and room
 * in the pool are free, so requests arriving while others run join them and
 * overlap on the device.  The loop never synchronises the device; results and
 * streams are byte-identical to the single calls'.
 * ------------------------------------------------------------------------ */

typedef struct szx_server szx_server; /* opaque, host memory */

#define SZX_REQ_COMPRESS 0
#define SZX_REQ_DECOMPRESS 1

typedef struct {
    int kind;           /* SZX_REQ_COMPRESS or SZX_REQ_DECOMPRESS */
    double arrival_s;   /* arrival, seconds after the run starts */
    /* compression: as szx_compress_async's arguments */
    const void *d_in;
    size_t n;
    szx_dtype dtype;
    double eb;
    uint32_t block;
    /* decompression: index (in the same run) of an earlier compression whose
     * resident stream it decodes; keep_output: leave the decoded values
     * allocated in the pool (at `offset`, `bytes` long) for the caller to read
     * and release, else they are freed on completion */
    int source;
    int keep_output;
    /* filled in by szx_server_run */
    int status;         /* szx_status of the request (-1 if it never ran) */
    double admit_s;     /* admission, seconds after the start */
    double done_s;      /* first observation of completion */
    uint64_t offset;    /* pool offset: compression's resident stream, or kept output */
    uint64_t bytes;     /* stream bytes (compression) or output bytes */
} szx_request;

/* Create a server over the caller's device pool (256-byte aligned,
 * pool_bytes long; the caller keeps ownership) with `slots` CUDA streams
 * (1..64), on the current device.  Allocates its own small pinned and device
 * status words.  Errors: SZX_ERR_INVALID, SZX_ERR_NOMEM, SZX_ERR_CUDA. */
szx_status szx_server_create(void *d_pool, size_t pool_bytes, int slots,
                             szx_server **server);

/* The pool's base address, and its free bytes (not counting fragmentation). */
void *szx_server_pool(const szx_server *server);
size_t szx_server_free_bytes(const szx_server *server);

/* Run `count` requests to completion (arrivals are timed from the call).
 * Per-request outcomes are written into reqs; *max_in_flight (may be NULL)
 * receives the largest number of requests that ran at once.  Returns
 * SZX_ERR_NOMEM if a request could never fit in the pool (that request's
 * status says so; the others still ran), else SZX_OK.  Resident streams of
 * the run stay allocated until szx_server_release. */
szx_status szx_server_run(szx_server *server, szx_request *reqs, int count,
                          int *max_in_flight);

/* Give back a pool range returned in a request (offset, bytes). */
szx_status szx_server_release(szx_server *server, uint64_t offset,
                              uint64_t bytes);

/* Wait for the server's streams and free its resources (not the pool). */
void szx_server_destroy(szx_server *server);

/*
 * Random access: decompress only blocks [first_block, first_block + nblocks)
 * of the stream whose header is *h.  Every block is coded from its own values
 * alone (Algorithm 1), and the tile index gives each tile record's offset, so
 * only the tiles holding those blocks are read.  d_out receives
 * min(n, (first_block + nblocks) * b) - first_block * b values, the same
 * bits a full decompression puts at that position.  Errors as for
 * szx_decompress_async, plus SZX_ERR_INVALID for an empty or out-of-range
 * block range.  Asynchronous.
 */
szx_status szx_decompress_range_async(const void *d_in, size_t in_bytes,
                                      const szx_header *h, size_t first_block,
                                      size_t nblocks, void *d_out,
                                      size_t out_capacity, uint32_t *d_status,
                                      szx_stream_t stream);

/* Human-readable name of a status code. */
const char *szx_status_string(szx_status s);

/* Library version string. */
const char *szx_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SZX_H */
