/*
 * hi.h -- C ABI of the GB300 interpolation predictor / error-bounded
 * quantizer (the lossy decomposition stage of cuSZ-Hi, arXiv 2507.11165).
 *
 * Model of the data (Sec. 3.2, Sec. 5.1.1):
 *   A float32 field x[n0][n1][n2] (row-major, n2 fastest; a 1D or 2D field
 *   uses leading dims of 1; a dim of size 1 is inactive) is cut into blocks
 *   of (A+1) points per active dim that share their faces.  Points whose
 *   coordinates are all multiples of the anchor stride A form the anchor
 *   grid and are stored verbatim.  Every other point is predicted level by
 *   level (stride 2^l, l = log2(A)-1 .. 0) by 1D linear or cubic spline
 *   interpolation along a per-level dimension sequence, from values that are
 *   already reconstructed, and its prediction error is quantized linearly
 *   into a one-byte code (Sec. 5.2.1): code = q + 128 with q in [-127,127];
 *   code 0 marks an outlier, stored separately as (index, value).
 *   Reconstruction repeats the traversal (Eq. 1: |x - x'| <= eps).
 *
 * Conventions:
 *   - Every pointer named d_* is device memory owned by the caller; h_* is
 *     host memory.  The library never allocates or frees memory.
 *   - All work is enqueued on the given stream and is asynchronous; results
 *     that are device-resident (the header, the outlier count, the status
 *     word) are read after synchronising, e.g. with hi_header_read().
 *   - Functions validate their host arguments synchronously and return
 *     HI_EINVAL (nothing is enqueued) on a bad argument.  Conditions found
 *     on the device (outlier capacity exceeded, a corrupt record, a bounded
 *     wait that ran out) are recorded in the status word of the header
 *     (first error wins) and never fault or hang the GPU.
 *   - Re-entrant: independent calls on different streams may overlap as long
 *     as they use distinct buffers and workspaces.
 *   - Index type: outlier indices are uint32, so a field holds fewer than
 *     2^32 points (HI_EINVAL otherwise).
 */
#ifndef HI_H
#define HI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cudaStream_t;

#if defined(__GNUC__)
#define HI_API __attribute__((visibility("default")))
#else
#define HI_API
#endif

typedef enum {
    HI_OK = 0,
    HI_EINVAL = 1,    /* bad argument (checked on the host, nothing enqueued)   */
    HI_ENOMEM = 2,    /* workspace too small                                    */
    HI_ECAPACITY = 3, /* more outliers than the caller's capacity (device)      */
    HI_ECUDA = 4,     /* a CUDA launch or runtime call failed                   */
    HI_ETIMEOUT = 5,  /* a bounded device-side wait ran out (device)            */
    HI_ECORRUPT = 6   /* decompress input is inconsistent (device)              */
} hi_status;

enum { HI_EB_ABS = 0, HI_EB_REL = 1 };
/* Interpolation of a level: 1D splines along the level's dimension sequence
 * (Sec. 5.1.2, Fig. 4a), or the multi-dimensional scheme (Sec. 5.1.2,
 * Fig. 4b: points with 1, 2, 3 odd coordinates in turn, the mean of the
 * highest-order 1D interpolations along their odd dims; the order field is
 * then unused but must still be a permutation). */
enum { HI_LINEAR = 0, HI_CUBIC = 1, HI_MD_LINEAR = 2, HI_MD_CUBIC = 3 };

#define HI_MAX_LEVELS 8
#define HI_MAGIC 0x48693235u /* "Hi25" */
#define HI_VERSION 1u

/* Interpolation configuration of one level (Sec. 5.1.2, Sec. 5.1.3):
 * the spline and the sequence of dimensions of its 1D passes.  order[] is a
 * permutation of {0,1,2}; passes along inactive dims are empty. */
typedef struct {
    uint8_t interp;   /* HI_LINEAR, HI_CUBIC, HI_MD_LINEAR or HI_MD_CUBIC */
    uint8_t order[3]; /* dimension sequence, 0 = slowest */
} hi_level;

/* Compression parameters (host memory). */
typedef struct {
    uint64_t dims[3];       /* n0, n1, n2: slowest -> fastest, each >= 1          */
    double eb;              /* error bound: absolute, or relative to max - min    */
    uint32_t eb_mode;       /* HI_EB_ABS or HI_EB_REL (Sec. 6.1.4)                */
    uint32_t anchor_stride; /* A: 2, 4, 8, 16 or 32 (Sec. 5.1.1 uses 16)          */
    uint32_t autotune;      /* 1: choose level[] on the device among the 1D       */
                            /* sequences (Sec. 5.1.3); 2: also the multi-        */
                            /* dimensional scheme; 0: use level[] as given        */
    uint32_t tuning;        /* launch shape, 0 = library default; else bits 0-1:  */
                            /* threads per CTA (1: 64, 2: 128), bits 2-3: tile    */
                            /* buffers (1: one, 2: two, prefetching)              */
    hi_level level[HI_MAX_LEVELS]; /* level[l]: stride 2^l; used when !autotune  */
} hi_params;

/* Self-describing record of one compressed field (device memory, written by
 * hi_compress, read by hi_decompress).  It fixes everything needed to
 * reconstruct: geometry, the resolved per-level configuration and the
 * float32 quantizer constants. */
typedef struct {
    uint32_t magic;         /* HI_MAGIC                                             */
    uint32_t version;       /* HI_VERSION                                           */
    uint64_t dims[3];
    uint32_t anchor_stride;
    uint32_t eb_mode;
    double eb;              /* as requested                                         */
    double eps;             /* resolved absolute bound: eb or eb * (vmax - vmin)    */
    float eb_f;             /* largest float <= eps: |x - x'| < eb_f is enforced    */
    float ebx2_f;           /* fl(2 eps): x' = p + q * ebx2_f                       */
    float r_f;              /* fl(1 / (2 eps)): q = rint((x - p) * r_f)             */
    float vmin, vmax;       /* range over finite values (REL mode; 0 otherwise)     */
    uint32_t status;        /* hi_status of device-side conditions, 0 = OK          */
    uint64_t n_outliers;    /* outliers found (may exceed out_cap)                  */
    uint64_t out_cap;       /* capacity of the outlier arrays at compression        */
    uint64_t n_anchors;
    hi_level level[HI_MAX_LEVELS];
    uint32_t n_levels;
    uint32_t reserved[7];
} hi_header;

/* Sizes of a compression of p (host call, no GPU work).
 *   n_points  = n0 n1 n2 = entries of the code array (uint8) and of a field;
 *   n_anchors = prod_d ((n_d - 1) / A + 1) = entries of the anchor grid;
 *   n_blocks  = prod over active dims of ceil((n_d - 1) / A);
 *   ws_bytes  = device workspace hi_compress needs (range partials and the
 *               auto-tuner's per-sample error sums).
 * Any output pointer may be NULL. */
HI_API hi_status hi_query(const hi_params* p, uint64_t* n_points, uint64_t* n_anchors, uint64_t* n_blocks,
                   size_t* ws_bytes);

/* Compress (Sec. 3.2, Sec. 5.1, Sec. 5.2.1).  Enqueues, in order: header
 * set-up; for HI_EB_REL the value range of d_x and eps = eb * (max - min)
 * (eps = eb if the range is 0); for autotune the per-level choice of spline
 * and dimension sequence on 0.2% of the blocks (in one launch with the
 * range when both are asked for: neither needs the other); then the fused
 * predict-quantize pass.
 *   d_x        [n_points] float32 input, 4-byte aligned (16 for the fast path)
 *   d_codes    [n_points] uint8 codes in the layout of d_x (anchors get 128)
 *   d_anchors  [n_anchors] float32 anchor grid, row-major
 *   d_out_idx, d_out_val [out_cap] outliers (linear index, value) in an
 *              unspecified order; the count goes to d_header->n_outliers and
 *              a count above out_cap sets HI_ECAPACITY (the codes stay valid;
 *              call again with a larger capacity)
 *   d_hist     [256] uint32 histogram of the codes of non-anchor points, or NULL
 *   d_recon    [n_points] float32 reconstructed field x', or NULL
 *   d_header   one hi_header
 *   d_ws       workspace of at least hi_query's ws_bytes (8-byte aligned) */
HI_API hi_status hi_compress(const hi_params* p, const float* d_x, uint8_t* d_codes, float* d_anchors,
                      uint32_t* d_out_idx, float* d_out_val, uint64_t out_cap, uint32_t* d_hist,
                      float* d_recon, hi_header* d_header, void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* hi_compress with no caller workspace and no allocation.  The paper has no
 * counterpart; this is a convenience of this library.
 *
 * For callers that cannot hand the library a workspace buffer: code that
 * must not call cudaMalloc (it synchronises the device and can fail under a
 * fixed memory budget), or that runs inside a host which owns all device
 * memory and offers no allocator.  The arguments and results are those of
 * hi_compress without d_ws / ws_bytes; the workspace is instead a fixed
 * scratch array of HI_STATIC_WS_BYTES inside the library's own device image,
 * one per GPU.  Nothing is allocated or freed, by this call or on its behalf.
 *
 *   - Size limit: when hi_query's ws_bytes for p exceeds HI_STATIC_WS_BYTES
 *     the call returns HI_ENOMEM and enqueues nothing; use hi_compress with
 *     a workspace of your own then.  1 MiB holds every field of at most
 *     10^7 points at any A, and every 3D field at A = 16.
 *   - Set-up: the first call on each device (the device current at the
 *     call) looks up the scratch array's device address, which may load the
 *     library's device code; make that first call before any stream capture
 *     begins.  A failed look-up returns HI_ECUDA.  The address is kept per
 *     device and context: after a device reset (a new context) the next call
 *     looks it up again, so make that call before any capture too.
 *   - Zero state: nothing in the scratch has to start at zero; the call's
 *     first kernel resets the counters it uses.
 *   - Races: every call on a device shares that device's one scratch array.
 *     Two calls that may run at the same time (different streams, or
 *     different host threads without ordering) corrupt each other; order
 *     them on one stream or synchronise between them. */
#define HI_STATIC_WS_BYTES (1u << 20)
HI_API hi_status hi_compress_static_ws(const hi_params* p, const float* d_x, uint8_t* d_codes, float* d_anchors,
                                uint32_t* d_out_idx, float* d_out_val, uint64_t out_cap, uint32_t* d_hist,
                                float* d_recon, hi_header* d_header, cudaStream_t stream);

/* Decompress (Eq. 1; the same traversal as hi_compress): x' = p + (code -
 * 128) * ebx2_f, or the stored outlier value for code 0.  p supplies the
 * geometry for the launch (dims, anchor_stride) and must match d_header,
 * which also supplies the per-level configuration and constants.
 *   d_out_idx/d_out_val hold out_cap entries, of which
 *   min(d_header->n_outliers, out_cap) are used; an index outside the field
 *   or n_outliers > out_cap sets HI_ECORRUPT / HI_ECAPACITY in *d_status.
 *   d_out      [n_points] float32 output
 *   d_status   one uint32 (may be NULL): 0 on success, else a hi_status.
 *   d_ws       at least HI_DECOMPRESS_WS_BYTES of device workspace (8-byte
 *              aligned; hi_query's ws_bytes always suffices). */
#define HI_DECOMPRESS_WS_BYTES 256
HI_API hi_status hi_decompress(const hi_params* p, const hi_header* d_header, const uint8_t* d_codes,
                        const float* d_anchors, const uint32_t* d_out_idx, const float* d_out_val,
                        uint64_t out_cap, float* d_out, uint32_t* d_status, void* d_ws, size_t ws_bytes,
                        cudaStream_t stream);

/* Auto-tune only (Sec. 5.1.3): writes the chosen level[] and n_levels into
 * d_header (other fields untouched).  Uniformly sampled blocks (every
 * (n_blocks / m)-th, m = max(1, round(0.002 n_points / A^d))); per level and
 * per candidate (1D: cubic before linear, dimension sequences in
 * lexicographic order; then, for autotune = 2 and two or more active dims,
 * the multi-dimensional scheme, cubic before linear: up to 14) the sum of
 * |x - p| with predictions from the original values; the
 * smallest sum wins, ties to the first candidate.  Uses the same workspace
 * as hi_compress. */
HI_API hi_status hi_autotune(const hi_params* p, const float* d_x, hi_header* d_header, void* d_ws, size_t ws_bytes,
                      cudaStream_t stream);

/* Per-sample, per-level, per-candidate error sums of the last hi_autotune /
 * hi_compress(autotune) call on this workspace, for inspection: copies
 * m * L * ncfg doubles (sample-major, then level, then candidate) into
 * h_err (synchronises the stream).  *m, *L, *ncfg may be NULL. */
HI_API hi_status hi_autotune_errors(const hi_params* p, const void* d_ws, double* h_err, size_t h_err_len,
                             uint32_t* m, uint32_t* L, uint32_t* ncfg, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Batches: many independent fields of uneven shapes compressed together,
 * one launch per stage for the whole batch.  Each field's codes, anchors,
 * outliers (as a set), histogram, reconstruction and header are those
 * hi_compress gives for it alone.  The predict-quantize launch is
 * persistent: its CTAs take (field, tile) work items from one queue over the
 * concatenated tile lists, so small fields do not leave the GPU idle.
 * Not in the paper, which compresses one field per call.
 * ------------------------------------------------------------------------ */

/* One field of a batch: its parameters and buffers, as for hi_compress
 * (d_x may be NULL in a batch used only by hi_decompress_batch), and where
 * hi_decompress_batch writes its reconstruction (d_out).  Every field of a
 * batch has the same anchor_stride, 8 or 16. */
typedef struct {
    hi_params p;
    const float* d_x;
    uint8_t* d_codes;
    float* d_anchors;
    uint32_t* d_out_idx;
    float* d_out_val;
    uint64_t out_cap;
    uint32_t* d_hist;   /* or NULL */
    float* d_recon;     /* or NULL */
    hi_header* d_header;
    float* d_out;       /* reconstruction target of hi_decompress_batch, or NULL */
} hi_batch_field;

/* A prepared batch (host memory, written by hi_batch_prepare).  The
 * offsets describe the library's layout of the workspace; callers read
 * tuning and the totals and leave the rest alone. */
typedef struct {
    uint32_t n_fields;
    uint32_t anchor_stride;
    uint32_t tuning;        /* launch shape of predict-quantize (hi_params.tuning encoding) */
    uint32_t all_tma;       /* every field is staged by TMA (two buffers possible)           */
    uint64_t total_tiles;   /* work items of predict-quantize                                */
    uint64_t total_chunks;  /* work items of the value range (relative-bound fields)        */
    uint64_t total_samples; /* auto-tune samples over all auto-tuned fields                 */
    uint64_t ws_bytes;      /* workspace the batch uses                                      */
    uint64_t off_table, off_prefix, off_tickets, off_partials, off_err;
    uint64_t reserved[4];
} hi_batch_plan;

/* Workspace bytes a batch of n fields needs (host call, no GPU work);
 * HI_EINVAL for a field hi_compress would refuse, mixed or unsupported
 * anchor strides, or n == 0. */
HI_API hi_status hi_batch_query(uint32_t n, const hi_batch_field* h_fields, size_t* ws_bytes);

/* Validate the batch, write its field table into d_ws (at least
 * hi_batch_query's bytes, 256-byte aligned) and fill *h_plan.  The copy is
 * synchronous: the call returns when the table is on the device.  tuning:
 * the launch shape (hi_params.tuning encoding, 0 = 128 threads, one
 * buffer).  The buffers of every field must stay valid while the plan is
 * used; d_ws belongs to the plan until the caller is done with it. */
HI_API hi_status hi_batch_prepare(uint32_t n, const hi_batch_field* h_fields, uint32_t tuning, void* d_ws,
                                  size_t ws_bytes, hi_batch_plan* h_plan, cudaStream_t stream);

/* Compress every field of a prepared batch.  Enqueues four launches on
 * stream (header set-up; value range of every relative-bound field beside
 * the auto-tuner of every auto-tuned field; the tuner's choices into the
 * field records; predict-quantize of all tiles) and
 * nothing else: no host synchronisation, no memory copy.  The stage events
 * of hi_set_stage_events (0..4) are recorded as for hi_compress.  Calls that
 * share d_ws must not overlap. */
HI_API hi_status hi_compress_batch(const hi_batch_plan* h_plan, void* d_ws, cudaStream_t stream);

/* Reconstruct every field of a prepared batch from its record (codes,
 * anchors, outliers and header, as hi_compress or hi_compress_batch left
 * them) into its d_out (Eq. 1; the level-by-level reconstruction of
 * Sec. 3.2, as hi_decompress does for one field): two launches for the
 * whole batch (the outlier values of every field into its output, then one
 * persistent reconstruction over the (field, tile) work items of all
 * fields), no host synchronisation, no memory copy; capturable in a CUDA
 * graph.  Each field's output equals hi_decompress of it alone.  Every field
 * needs d_out (4-byte aligned, its point count of floats).  A field whose
 * header is not a valid record, reports an error or holds more outliers than
 * out_cap is left unwritten and sets HI_ECAPACITY (over capacity) or
 * HI_ECORRUPT in *d_status (device uint32, may be NULL; first error wins;
 * cleared by the call); an outlier index past a field's end sets
 * HI_ECORRUPT.  HI_EINVAL (nothing enqueued) for a plan without d_out on
 * every field.  Calls that share d_ws must not overlap (with each other or
 * with hi_compress_batch).  Not in the paper, which reconstructs one field
 * per call. */
HI_API hi_status hi_decompress_batch(const hi_batch_plan* h_plan, void* d_ws, uint32_t* d_status, cudaStream_t stream);

/* Launch-shape tuner of a prepared batch: times hi_compress_batch under
 * each candidate shape (128 then 64 threads per CTA, each with one buffer,
 * then two where every field is staged by TMA), reps timed runs each after
 * one warm-up, and stores the fastest in h_plan->tuning.  h_ms (may be
 * NULL) receives the mean ms per run of the four candidates in that order
 * (0 for one not tried).  Synchronises the stream; the outputs of the
 * fields are overwritten with the same values by every run. */
HI_API hi_status hi_batch_tune_launch(hi_batch_plan* h_plan, void* d_ws, uint32_t reps, float* h_ms,
                                      cudaStream_t stream);

/* Measurement hook: record CUDA events between the stages of later
 * hi_compress / hi_decompress calls made by the calling host thread.
 * events[0..7] (cudaEvent_t handles created by the caller):
 *   hi_compress:   0 before header set-up, 1 before the range pass, 2 before
 *                  the auto-tuner, 3 before predict-quantize, 4 after it
 *                  (with both a relative bound and auto-tune, range and
 *                  auto-tuner share one launch between events 1 and 2);
 *   hi_decompress: 5 before the outlier scatter, 6 before reconstruction,
 *                  7 after it.
 * A stage that does not run still records its event.  n must be 8; pass
 * events = NULL to switch recording off.  No GPU work of its own. */
HI_API hi_status hi_set_stage_events(void* const* events, uint32_t n);

/* Quantization-code reordering (Sec. 5.2.2, Eq. 3).  The code of the point
 * (x, y, z) of the field (x slowest) moves to position I(x, y, z) of a 1D
 * sequence in which the codes of each interpolation level lie together:
 * the anchors first (in row-major order of the anchor grid), then level
 * log2(A) - 1, ..., level 0, row-major within a level.  The level of a
 * point is the largest l <= log2 A with 2^l dividing all its coordinates.
 * The paper writes the within-level rank for level 0 on the global grid;
 * for coarser levels the library takes the same rank on the stride-2^l
 * subgrid (the reading under which Eq. 3's prefix(l) counts the coarser
 * points).  The codes are those of hi_compress; the reordering feeds a
 * lossless coder and is not needed by hi_decompress, which reads the
 * row-major array.
 *   hi_reorder_codes:   d_seq[I(x, y, z)] = d_codes[x][y][z]
 *   hi_unreorder_codes: d_codes[x][y][z] = d_seq[I(x, y, z)]
 * p: the field's parameters (only dims and anchor_stride matter, but p
 * must be valid for hi_compress).  d_codes and d_seq: n_points bytes each
 * of device memory owned by the caller; they must not overlap.  Enqueued
 * on stream, asynchronous, nothing allocated.  Returns HI_EINVAL for a
 * NULL pointer, invalid parameters or overlapping buffers (nothing
 * enqueued), HI_ECUDA if the launch fails. */
HI_API hi_status hi_reorder_codes(const hi_params* p, const uint8_t* d_codes, uint8_t* d_seq, cudaStream_t stream);
HI_API hi_status hi_unreorder_codes(const hi_params* p, const uint8_t* d_seq, uint8_t* d_codes,
                                    cudaStream_t stream);

/* hi_compress that also writes the codes in the reordered order of
 * hi_reorder_codes (Sec. 5.2.2, Eq. 3) to d_seq (n_points bytes, not
 * overlapping d_codes), the input of the lossless pipelines below.  All
 * other arguments and results are those of hi_compress, and d_codes is
 * written as there.  Where the field allows it the predict-quantize kernel
 * stores each tile's codes to their places in d_seq from shared memory,
 * one aligned store per run of consecutive places, instead of a separate
 * pass over the code array: A = 8 or 16, n2 a multiple of A, d_seq 16-byte
 * aligned, fewer than 2^32 points, and every run starting at a multiple of
 * its length (true when each dim is a multiple of 2A, e.g. 512^3 at
 * A = 16).  Otherwise hi_reorder_codes runs after the kernel on the same
 * stream.  HI_EINVAL for a NULL d_seq or overlapping code arrays.
 * hi_compress_seq_fused: 1 when a call with these parameters and pointers
 * takes the single-kernel form, else 0 (host only, no GPU work). */
HI_API hi_status hi_compress_seq(const hi_params* p, const float* d_x, uint8_t* d_codes, uint8_t* d_seq,
                                 float* d_anchors, uint32_t* d_out_idx, float* d_out_val, uint64_t out_cap,
                                 uint32_t* d_hist, float* d_recon, hi_header* d_header, void* d_ws,
                                 size_t ws_bytes, cudaStream_t stream);
HI_API int hi_compress_seq_fused(const hi_params* p, const uint8_t* d_codes, const uint8_t* d_seq);

/* The value range of the value-range-relative bound (Sec. 6.1.4) alone:
 * the min and the max over the finite values of d_x go to d_header->vmin /
 * vmax (0 and 0 when there is none), with the header's eps and float32
 * constants derived from them as hi_compress would.  For a field processed
 * in parts (out of core, or one part per GPU): the parts' ranges combine
 * into the field's, whose eps each part then takes as an absolute bound.
 * p: the part's parameters, eb_mode HI_EB_REL.  d_ws: at least
 * HI_DECOMPRESS_WS_BYTES + 8 KiB (hi_query's ws_bytes always suffices).
 * Two launches on stream, no sync; HI_EINVAL / HI_ENOMEM / HI_ECUDA as for
 * hi_compress. */
HI_API hi_status hi_value_range(const hi_params* p, const float* d_x, hi_header* d_header, void* d_ws,
                                size_t ws_bytes, cudaStream_t stream);

/* Throughput-mode lossless pipeline TCMS1-BIT1-RRE1 (Sec. 5.2.3): a byte
 * sequence (normally the output of hi_reorder_codes) into a self-describing
 * stream, and back.  Stages, per 16 KiB chunk: TCMS1 maps each byte, read as
 * a signed int8, to magnitude-sign form ((b << 1) ^ (b >> 7); the zero
 * residual 128 becomes 0xff); BIT1 transposes the chunk into 8 bit planes
 * (most significant first, zero-padded to a multiple of 64 elements); RRE1
 * keeps the bytes that differ from their predecessor plus a bitmap of them,
 * and compresses the bitmap the same way until it is at most 64 bytes.  The
 * paper names the stages only; the chunking, plane order, recursion depth
 * and container are this library's reading:
 *   stream = u64 n | u32 16384 | u32 nchunks | u32 size[nchunks] | zero
 *            padding to 16 bytes | payloads, each padded to 16 bytes;
 *   size[k] = padded payload bytes, bit 31 set when chunk k is stored raw
 *            (its encoding would not be shorter);
 *   payload = the top bitmap level, then the kept bytes of each level below
 *            it, top down.
 * hi_tp_query: *max_stream_bytes = the largest stream for n input bytes;
 *   *ws_bytes = the workspace both calls need (either pointer may be NULL).
 * hi_tp_encode: d_in (n bytes) -> d_out (16-byte aligned, out_cap >=
 *   max_stream_bytes, not overlapping d_in); the stream length is written to
 *   *d_len (device uint64).  d_ws: ws_bytes >= hi_tp_query's, 16-byte
 *   aligned.  Three launches on stream, no sync.
 * hi_tp_decode: d_in (a stream of in_len bytes, 16-byte aligned) -> d_out
 *   (n bytes, the length the stream was made from).  A stream that does not
 *   match n or whose table or payloads are inconsistent sets HI_ECORRUPT in
 *   *d_status (may be NULL) and leaves the affected chunks unwritten.  Two
 *   launches on stream, no sync.
 * All three return HI_EINVAL for NULL or misaligned pointers, short
 * buffers, a too-small workspace or n >= 2^44 (nothing enqueued), HI_ECUDA
 * if a launch fails. */
HI_API hi_status hi_tp_query(uint64_t n, uint64_t* max_stream_bytes, size_t* ws_bytes);
HI_API hi_status hi_tp_encode(const uint8_t* d_in, uint64_t n, uint8_t* d_out, uint64_t out_cap, uint64_t* d_len,
                              void* d_ws, size_t ws_bytes, cudaStream_t stream);
HI_API hi_status hi_tp_decode(const uint8_t* d_in, uint64_t in_len, uint8_t* d_out, uint64_t n, uint32_t* d_status,
                              void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Compression-ratio-mode lossless pipeline HF-RRE4-TCMS8-RZE1 (Sec. 5.2.3)
 * over a byte sequence (normally the reordered codes): Huffman coding of the
 * bytes, then per 16 KiB chunk of the Huffman bytes repeat elimination on
 * 4-byte words with a recursively reduced bitmap, the magnitude-sign
 * transform (w << 1) ^ (w >> 63) on 8-byte words, zero elimination on
 * bytes.  Code construction and container are this library's reading:
 *   Huffman lengths from the tree merging the two lowest (weight, creation
 *   index) nodes, leaves created first in symbol order; lengths above 16
 *   halve every nonzero weight (at least 1) and rebuild; canonical codes;
 *   blocks of 4096 symbols, MSB first, each padded to 32 bits.
 *   stream = u64 n | u32 4096 | u32 nblocks | u64 H | u32 16384 |
 *   u32 nchunks | u8 length[256] | u32 words[nblocks] | u16 sub[3 nblocks]
 *   | zero pad to 4 | (u32 size, u32 m1)[nchunks] | zero pad to 16 |
 *   payloads padded to 16 (size bit 31: raw); sub[3 b + j - 1] = the bit
 *   offset in block b of its symbol 1024 j (its bit count when shorter),
 *   where a decoder may start: four independent streams a block.
 * hi_cr_query: *max_stream_bytes = the largest stream for n input bytes,
 *   *ws_bytes = the workspace both calls need (either pointer may be NULL).
 * hi_cr_encode: d_in (n bytes, 16-byte aligned) -> d_out (16-byte aligned,
 *   out_cap >= max_stream_bytes, not overlapping d_in); the stream length
 *   goes to *d_len (device uint64).  Nine launches and a 1 KiB memset on
 *   stream, no sync.
 * hi_cr_decode: d_in (a stream of in_len bytes, 16-byte aligned) -> d_out
 *   (n bytes, 16-byte aligned).  A stream that does not match n or whose
 *   tables, payloads or codes are inconsistent sets HI_ECORRUPT in *d_status
 *   (may be NULL); the affected chunks or blocks are left unwritten.  Three
 *   launches on stream, no sync.
 * All three return HI_EINVAL for NULL or misaligned pointers, short buffers,
 * a too-small workspace or n >= 2^32 (symbol counts are 32-bit; nothing
 * enqueued), HI_ECUDA if a launch fails.  The caller owns every buffer; the
 * calls allocate nothing. */
HI_API hi_status hi_cr_query(uint64_t n, uint64_t* max_stream_bytes, size_t* ws_bytes);
HI_API hi_status hi_cr_encode(const uint8_t* d_in, uint64_t n, uint8_t* d_out, uint64_t out_cap, uint64_t* d_len,
                              void* d_ws, size_t ws_bytes, cudaStream_t stream);
HI_API hi_status hi_cr_decode(const uint8_t* d_in, uint64_t in_len, uint8_t* d_out, uint64_t n, uint32_t* d_status,
                              void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* The absolute bound and the float32 quantizer constants of Eq. 1 from a
 * value range, on the host, with the same IEEE double operations the device
 * uses in hi_compress (Sec. 6.1.4 read as eps = eb * (vmax - vmin); eps = eb
 * for a zero range or HI_EB_ABS; eb_f = the largest float <= eps, ebx2_f =
 * fl(2 eps), r_f = fl(1 / (2 eps))).  For a field processed in parts
 * (out of core, or one part per GPU): combine the parts' vmin / vmax
 * (hi_value_range), resolve eps here and compress each part at the absolute
 * bound eps.  Host only, no CUDA call.  HI_EINVAL for a NULL out, a bad mode
 * or eb, or constants that are not finite and positive. */
typedef struct {
    double eps;
    float eb_f, ebx2_f, r_f;
    float pad;
} hi_eps;
HI_API hi_status hi_resolve_eps(uint32_t eb_mode, double eb, float vmin, float vmax, hi_eps* out);

/* Entropy-estimated compressed size (the record a Huffman-type entropy coder,
 * Sec. 5.2.2, approaches): H = -sum p_k log2 p_k over the 256-bin code
 * histogram h_hist (bins in ascending order, IEEE double), est_bytes =
 * ceil(N_pred H / 8) + 8 n_outliers + 4 n_anchors + header_bytes with N_pred
 * the histogram total, cr = 4 n_points / est_bytes, bit_rate = 8 est_bytes /
 * n_points (bits per value).  Host only.  HI_EINVAL for NULL pointers or
 * n_points = 0. */
typedef struct {
    double entropy_bits;
    uint64_t est_bytes;
    double cr;
    double bit_rate;
} hi_cr_estimate;
HI_API hi_status hi_estimate_cr(const uint32_t* h_hist, uint64_t n_outliers, uint64_t n_anchors, uint64_t n_points,
                                uint64_t header_bytes, hi_cr_estimate* out);

/* The auto-tuner's per-level choice (Sec. 5.1.3) from per-sample error
 * sums, on the host: h_err holds m * L * ncfg doubles (sample-major, then
 * level, then candidate, as hi_autotune_errors returns them; m, L, ncfg as
 * hi_autotune_errors reports for p).  Per (level, candidate) the samples are
 * summed in the order the device sums them (sample k into partial k mod 32,
 * ascending k, then the 32 partials by the butterfly j + (j ^ 16), j + (j ^
 * 8), ..., j + (j ^ 1)); each level takes the smallest sum, ties to the first
 * candidate of hi_autotune's enumeration.  For a field compressed in parts:
 * the parts' rows of the whole field's sample blocks, gathered into one
 * array, give the choice the whole field would make.  Writes level[0 .. L)
 * of *out and leaves its other fields as they are.  Host only; HI_EINVAL for
 * bad arguments or a short h_err. */
HI_API hi_status hi_autotune_select(const hi_params* p, const double* h_err, size_t h_err_len, hi_params* out);

/* Copy the device header to the host (synchronises the stream). */
HI_API hi_status hi_header_read(const hi_header* d_header, hi_header* h_header, cudaStream_t stream);

/* Short text for a status code. */
HI_API const char* hi_status_str(int status);

/* Library version (HI_VERSION). */
HI_API uint32_t hi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HI_H */
