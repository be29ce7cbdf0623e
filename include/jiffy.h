/*
 * jiffy.h -- C ABI of the GB300 Jiffy LiDAR scan codec.
 *
 * Jiffy (Ford & Ford, "Lossless SIMD Compression of LiDAR Range and Attribute
 * Scan Sequences", arXiv 2209.08196) compresses sequences of LiDAR scans held
 * as H x W images of unsigned integers (rows = beams, columns = azimuth), one
 * image ("plane") per attribute: range, second-return range, signal,
 * reflectivity, ambient, ... (Sec. III-A, Sec. IV-B). Per attribute and scan
 * it quantizes to a precision (Sec. III-B), extracts and codes the zero
 * bitmask (Sec. III-C), removes the zero samples, forms intra-scan (I) or
 * predicted-scan (P) residuals (Sec. III-C, III-D) chosen by trial
 * compression (Sec. III-E), delta and ZigZag (Eq. 1) codes them and packs
 * them in frames of 128 integers with exceptions (PFOR, Sec. II).
 *
 * Every stage runs in this library's CUDA kernels on one GPU. All functions
 * take plain pointers and sizes. "device" pointers are CUDA device memory of
 * the stream's device; "host" pointers are ordinary CPU memory. A `cuda_stream`
 * argument is a cudaStream_t passed as void* (NULL = the legacy default
 * stream); work is enqueued on it in stream order.
 *
 * Byte layout (the paper leaves it open; this library's format, version 1,
 * little-endian, every section 4-byte aligned):
 *   stream header (before the first frame after create/reset), 16 + 8A bytes:
 *     "JFY1", u16 version = 1, u16 A, u32 H, u32 W,
 *     per attribute { u8 dtype_bytes, u8 zigzag variant (1 = Eq. 1, 0 =
 *                     none), u8 stage flags (bit 0: no zero mask, bit 1:
 *                     no delta), u8 0, u32 precision }
 *                     (Sec. III-A: precision is stored)
 *   frame, one per scan: header 8 + 12A bytes
 *     u32 frame_bytes, u32 scan_index (frames since create/reset),
 *     per attribute { u8 mode (0 = I, 1 = P), 3 x u8 0, u32 section_bytes,
 *                     u32 nnz }
 *   then per attribute a section: a row table of H x { u32 end, u32 carry }
 *     (end = byte end of the row's chunk counted from the first chunk; carry
 *     = the residual preceding the row's first residual in the scan's flat
 *     nonzero vector, 0 if none) and H row chunks:
 *     mask class words (2 bits per 32-sample mask word: 0 = all clear,
 *     1 = all valid bits set, 2 = literal follows), literal mask words,
 *     block headers {u8 b, u8 exceptions, u8 high bits, u8 0}, block bodies
 *     (low bits, exception positions, exception high bits).
 *   A stream created with stage switches (jiffy_options.stages) leaves out
 *   steps: without the mask stage row chunks have no mask part and every
 *   sample is coded (frame nnz = H * W), without the delta the residuals are
 *   packed directly (row carries are still recorded), without ZigZag the
 *   32-bit two's complement words are packed.
 *   With JIFFY_STAGE_ZSTD_MASK the row chunks have no mask part either; the
 *   section's mask follows its row table as one Zstandard frame (RFC 8878,
 *   the mask coding of Sec. III-C): u32 frame bytes F, u32 end of each of
 *   its ceil(H ceil(W/8) / 8192) blocks (from the frame's start), the F
 *   frame bytes, zero bytes up to a multiple of 4; the row ends count from
 *   the first chunk after it. The frame holds the coded mask bits (the XOR
 *   with the previous scan's for P), LSB first, each row in ceil(W/8) bytes
 *   with zero padding bits; any Zstandard decoder restores it. Its blocks,
 *   one per 8192 bytes, are RLE, Raw or Compressed (Huffman-coded literals,
 *   one stream up to 1023 bytes and four above, direct or FSE-coded
 *   weights, no sequences).
 *
 * Errors: every function returns a jiffy_status; nothing aborts. A failed
 * call leaves the stream's state (previous scan, frame counter) unchanged.
 * Thread safety: a jiffy_stream may be used by one host thread at a time;
 * different streams are independent.
 */
#ifndef JIFFY_H
#define JIFFY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  JIFFY_OK = 0,
  JIFFY_ERR_INVALID_ARG = 1, /* bad pointer, size, shape, dtype or option */
  JIFFY_ERR_CAPACITY = 2,    /* output buffer too small; required size reported */
  JIFFY_ERR_CORRUPT = 3,     /* malformed or mismatching input stream */
  JIFFY_ERR_STATE = 4,       /* call not valid in the stream's current state */
  JIFFY_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  JIFFY_ERR_CUDA = 6,        /* a CUDA runtime call failed */
  JIFFY_ERR_NOMEM = 7        /* device or host allocation failed */
} jiffy_status;

typedef enum { JIFFY_ENCODER = 0, JIFFY_DECODER = 1 } jiffy_role;

/* One attribute plane: sample size (1, 2 or 4 bytes, unsigned) and the
 * quantization precision P >= 1 (Sec. III-B). The encoder codes
 * q = min(floor((v + floor(P/2)) / P), floor(max/P)) and the decoder returns
 * q * P; |v - q*P| <= P/2 wherever the clamp does not act (Sec. IV-G). */
typedef struct {
  uint32_t dtype_bytes;
  uint32_t precision;
} jiffy_attr_desc;

/* Stage switches (jiffy_options.stages): each removes one step of the codec,
 * for the ablated codecs of Sec. IV-H (Table IV). With force_mode = 0 as
 * well, NO_MASK | NO_DELTA | NO_ZIGZAG is "SIMD-PFOR" alone, NO_MASK |
 * NO_ZIGZAG is "Delta -> SIMD-PFOR", NO_MASK is "Delta -> ZigZag ->
 * SIMD-PFOR" and 0 is "Mask -> Delta -> ZigZag -> SIMD-PFOR". */
#define JIFFY_STAGE_NO_MASK 1u   /* no zero mask: every sample is coded, zeros too */
#define JIFFY_STAGE_NO_DELTA 2u  /* residuals packed without the horizontal delta */
#define JIFFY_STAGE_NO_ZIGZAG 4u /* deltas packed as 32-bit two's complement words */
/* Not an ablation: the zero mask coded as Sec. III-C describes, packed into
 * bytes and compressed as one Zstandard frame per section, in place of the
 * per-row class words (the layout is above). Cannot be combined with
 * JIFFY_STAGE_NO_MASK. The allocation-free decode does not take it. */
#define JIFFY_STAGE_ZSTD_MASK 8u

/* test_lines: number of scanlines of the trial compression (Sec. III-E;
 * Sec. IV-E uses 4); rows floor((2k+1)H/(2L)), k < L, >= 1. test_lines >= H
 * makes every row a test row: the brute-force choice between I and P over
 * the data sections (mask excluded), at about the cost of coding each scan
 * a second time. force_mode: -1 picks I or P per attribute and scan by
 * trial, 0 forces I, 1 forces P (the first frame after create/reset is
 * always I). stages: JIFFY_STAGE_* bits, 0 = the full codec; recorded in the
 * stream header, and a decoder must be created with the same bits. */
typedef struct {
  uint32_t test_lines;
  int32_t force_mode;
  uint32_t stages;
} jiffy_options;

typedef struct jiffy_stream jiffy_stream;

/* Creates a codec stream on CUDA device `device`: the encoder or decoder of
 * one sensor's scan sequence with H x W planes and n_attr attributes.
 * 1 <= H <= 4096, 1 <= W <= 16384, 1 <= n_attr <= 64. opt may be NULL
 * (test_lines = 4, force_mode = -1, stages = 0). The stream owns its device state (the
 * previous scan of every attribute, Sec. III-D) and scratch; *out receives
 * the handle. Errors: INVALID_ARG, NOMEM, CUDA. */
jiffy_status jiffy_stream_create(jiffy_stream** out, jiffy_role role, uint32_t H, uint32_t W,
                                 uint32_t n_attr, const jiffy_attr_desc* attrs,
                                 const jiffy_options* opt, int device);

/* Releases the stream and its device memory (synchronizes its device). */
void jiffy_stream_destroy(jiffy_stream* s);

/* Forgets the previous scan: the next frame is an I frame preceded by a new
 * stream header (a resume point). */
jiffy_status jiffy_stream_reset(jiffy_stream* s);

/* Upper bound of the bytes n_scans frames (plus a stream header) can take. */
size_t jiffy_max_encoded_size(uint32_t H, uint32_t W, uint32_t n_attr, const jiffy_attr_desc* attrs,
                              uint32_t n_scans);

/* Encodes one scan. planes: host array of n_attr device pointers, each an
 * H x W row-major dense plane of dtype_bytes samples (borrowed for the call).
 * out: device buffer of out_capacity bytes, 16-byte aligned. On JIFFY_OK,
 * *out_len (host) = bytes written (the stream header is included before the
 * first frame). On JIFFY_ERR_CAPACITY, *out_len = bytes required and nothing
 * valid is written. Synchronizes cuda_stream before returning. */
jiffy_status jiffy_encode(jiffy_stream* s, const void* const* planes, void* out, size_t out_capacity,
                          size_t* out_len, void* cuda_stream);

/* Encodes n_scans consecutive scans of the stream in one pass (the P
 * prediction of scan t uses scan t-1's input, Sec. III-D, so all scans are
 * coded in parallel). planes: host array of n_scans * n_attr device pointers,
 * scan-major (planes[t * n_attr + a]). frame_offsets (host, nullable, n_scans
 * + 1 entries) receives the byte offset of each frame in out and the total
 * length last. Otherwise as jiffy_encode. */
jiffy_status jiffy_encode_seq(jiffy_stream* s, uint32_t n_scans, const void* const* planes, void* out,
                              size_t out_capacity, uint64_t* frame_offsets, size_t* out_len,
                              void* cuda_stream);

/* Decodes one frame (preceded by the stream header for the first frame after
 * create/reset) of in_len bytes at device pointer in (4-byte aligned) into
 * planes_out (host array of n_attr device pointers, H x W dense). Errors:
 * CORRUPT (malformed frame, shape/dtype/precision mismatch with the stream
 * header, wrong scan index), TIMEOUT, CUDA. Synchronizes cuda_stream. */
jiffy_status jiffy_decode(jiffy_stream* s, const void* in, size_t in_len, void* const* planes_out,
                          void* cuda_stream);

/* Decodes n_scans consecutive frames. frame_offsets (host, n_scans + 1
 * entries) gives each frame's byte offset in `in` and the end of the last
 * one, as returned by jiffy_encode_seq. planes_out: n_scans * n_attr device
 * pointers, scan-major. Scans are decoded in parallel; a P frame's rows wait
 * on the same rows of the previous frame. Synchronizes cuda_stream. */
jiffy_status jiffy_decode_seq(jiffy_stream* s, uint32_t n_scans, const void* in, size_t in_len,
                              const uint64_t* frame_offsets, void* const* planes_out, void* cuda_stream);

/* Enqueue-only forms of jiffy_encode_seq / jiffy_decode_seq, for a pipeline
 * that stays on the device: an encode followed by a decode on the same CUDA
 * stream needs no host round trip in between. Each returns once its work is
 * on cuda_stream, without waiting.
 *
 * jiffy_encode_seq_async: as jiffy_encode_seq, but the n_scans + 1 frame
 * offsets (the last one = the bytes written) go to frame_offsets_dev, a
 * device array of uint64 (8-byte aligned; nullable), and no length comes
 * back to the host. jiffy_decode_seq_async: as jiffy_decode_seq, but
 * frame_offsets_dev is a device array (as written by jiffy_encode_seq_async)
 * and in_capacity the bytes readable at `in`; the kernel checks every offset
 * (aligned, increasing by at least a frame header, inside in_capacity) before
 * reading, so a bad offset is CORRUPT, never an out-of-bounds read.
 *
 * The stream's state advances at once; a stream may take several
 * enqueue-only calls in a row. Argument errors are returned at once; errors
 * found on the device (CORRUPT, CAPACITY, TIMEOUT) are reported by the next
 * jiffy_stream_wait, after which a stream that failed holds no usable
 * previous scan and must be reset. The device buffers must stay valid until
 * the work is done; a synchronous call on the stream waits first. */
jiffy_status jiffy_encode_seq_async(jiffy_stream* s, uint32_t n_scans, const void* const* planes, void* out,
                                    size_t out_capacity, uint64_t* frame_offsets_dev, void* cuda_stream);
jiffy_status jiffy_decode_seq_async(jiffy_stream* s, uint32_t n_scans, const void* in, size_t in_capacity,
                                    const uint64_t* frame_offsets_dev, void* const* planes_out, void* cuda_stream);

/* Waits for the stream's enqueue-only calls and returns JIFFY_OK, or the
 * error the device reported for any of them (then reset the stream). */
jiffy_status jiffy_stream_wait(jiffy_stream* s);

/* ---- Many streams in one pass (serving many sensors). A batch context owns
 * the scratch of batched calls on one device. In one call every stream
 * codes its own consecutive scans; all rows of all streams run in the same
 * kernel launches, each stream keeping its own state, shape and attributes.
 * A stream may appear at most once per call and must live on the batch's
 * device. */
typedef struct jiffy_batch jiffy_batch;

jiffy_status jiffy_batch_create(jiffy_batch** out, int device);
void jiffy_batch_destroy(jiffy_batch* b);

/* Encodes, for i < n, n_scans[i] consecutive scans of encoder streams[i]:
 * planes[i] is a host array of n_scans[i] * n_attr device pointers
 * (scan-major), outs[i] a 16-byte aligned device buffer of caps[i] bytes.
 * frame_offsets (nullable host array of n host pointers, each nullable):
 * frame_offsets[i] receives n_scans[i] + 1 offsets as in jiffy_encode_seq.
 * out_lens[i] (host) = bytes written (or required, on JIFFY_ERR_CAPACITY);
 * statuses[i] (host) = that stream's status; a stream whose status is not
 * JIFFY_OK keeps its state. Returns JIFFY_OK if every stream succeeded, else
 * the first failing status. Synchronizes cuda_stream (Sec. III-D prediction
 * within each stream, as jiffy_encode_seq). */
jiffy_status jiffy_encode_batch(jiffy_batch* b, uint32_t n, jiffy_stream* const* streams, const uint32_t* n_scans,
                                const void* const* const* planes, void* const* outs, const size_t* caps,
                                uint64_t* const* frame_offsets, size_t* out_lens, jiffy_status* statuses,
                                void* cuda_stream);

/* Decodes, for i < n, n_frames[i] frames of decoder streams[i] from ins[i]
 * (in_lens[i] bytes, 4-byte aligned, device) with frame_offsets[i] (host,
 * n_frames[i] + 1 entries) into planes_out[i] (host array of
 * n_frames[i] * n_attr device pointers). statuses[i] as in
 * jiffy_encode_batch. Synchronizes cuda_stream. */
jiffy_status jiffy_decode_batch(jiffy_batch* b, uint32_t n, jiffy_stream* const* streams, const uint32_t* n_frames,
                                const void* const* ins, const size_t* in_lens, const uint64_t* const* frame_offsets,
                                void* const* const* planes_out, jiffy_status* statuses, void* cuda_stream);

/* Enqueue-only forms of the two calls above: they return once the work is
 * on cuda_stream, without waiting. The host arrays out_lens, frame_offsets
 * and statuses must stay valid until jiffy_batch_wait(b) fills them; the
 * streams count as advanced until then (jiffy_batch_wait rolls back those
 * that failed) and may not take part in another call before it. A batch has
 * at most one unfinished call (JIFFY_ERR_STATE otherwise). With two batch
 * contexts the host can prepare and enqueue one call while the other runs. */
jiffy_status jiffy_encode_batch_async(jiffy_batch* b, uint32_t n, jiffy_stream* const* streams,
                                      const uint32_t* n_scans, const void* const* const* planes,
                                      void* const* outs, const size_t* caps, uint64_t* const* frame_offsets,
                                      size_t* out_lens, jiffy_status* statuses, void* cuda_stream);
jiffy_status jiffy_decode_batch_async(jiffy_batch* b, uint32_t n, jiffy_stream* const* streams,
                                      const uint32_t* n_frames, const void* const* ins, const size_t* in_lens,
                                      const uint64_t* const* frame_offsets, void* const* const* planes_out,
                                      jiffy_status* statuses, void* cuda_stream);

/* Waits for the batch's unfinished call (if any) and reports its results as
 * the synchronous call would: JIFFY_OK, or the first failing status. */
jiffy_status jiffy_batch_wait(jiffy_batch* b);

/* enable != 0: the batch captures its call's launch sequence (table upload,
 * counter clearing, kernels, result download) in a CUDA graph and replays it
 * while the calls keep the same shape (streams' H, W, attribute counts and
 * scan counts, in order); the segment table, which holds the buffers and
 * frame indices, is re-uploaded by the graph each time. Off by default for
 * batches; single-stream calls (jiffy_encode(_seq), jiffy_decode(_seq))
 * always replay their sequence this way while their shape repeats. Kernel
 * timing (profiling) works with replays. */
jiffy_status jiffy_batch_set_graphs(jiffy_batch* b, int enable);

/* enable != 0: on the first call of each shape class (role, widest row,
 * log2 of the row count) the batch times the rows kernel under each
 * candidate launch configuration (warps per CTA, resident CTAs per SM, row
 * items per ticket), repeating the call's kernels on the same inputs, and
 * keeps the fastest for later calls of that class. Off by default.
 * If the environment variable JIFFY_TUNE_CACHE names a file, enabling loads
 * the configurations tuned earlier on this kind of device (SM count and
 * compute capability) from it, and each new tuning rewrites it (a text file,
 * one line per shape class, replaced atomically); an unreadable or foreign
 * file only means tuning anew. */
jiffy_status jiffy_batch_set_autotune(jiffy_batch* b, int enable);

/* Fixes the launch configuration of the role's rows kernel for the batch's
 * later calls, over the tuner's choice: warps per CTA (encode 1, 2, 4;
 * decode 1, 2, 4, 8), resident CTAs per SM, row items per ticket (decode
 * only, <= 64). 0 leaves a field automatic; a request that does not fit the
 * device falls back to the automatic choice. Every configuration codes the
 * same bytes. */
jiffy_status jiffy_batch_set_launch(jiffy_batch* b, jiffy_role role, uint32_t warps_per_cta,
                                    uint32_t ctas_per_sm, uint32_t items_per_ticket);

/* Counters and the last launch configuration, in this order: calls, graph
 * captures, graph replays, tuning runs, tuned shape classes, last rows
 * kernel's warps per CTA, CTAs per SM, items per ticket, grid. Writes
 * min(n, 9) values to info (host). */
jiffy_status jiffy_batch_info(const jiffy_batch* b, uint64_t* info, uint32_t n);

/* Per-kernel device timing of the batch's calls, as for streams below. */
jiffy_status jiffy_batch_set_profiling(jiffy_batch* b, int enable);
uint32_t jiffy_batch_kernel_times(const jiffy_batch* b, float* ms, uint32_t n);

/* Per-kernel device timing (CUDA events recorded around each kernel launch
 * on the call's cuda_stream). enable != 0 turns it on for later calls. */
jiffy_status jiffy_stream_set_profiling(jiffy_stream* s, int enable);

/* Device milliseconds of each kernel launched by the stream's last
 * successful call, in launch order (encode: trial, rows, placement; decode:
 * rows); after jiffy_stream_wait, the averages over the enqueue-only calls
 * since the previous wait. Writes min(n, count) values to ms (host) and
 * returns the count (0 if profiling is off or no call completed). */
uint32_t jiffy_stream_kernel_times(const jiffy_stream* s, float* ms, uint32_t n);

/* Allocation-free decode of one frame, for callers that may not allocate
 * device memory once they run: real-time stacks that fix their device
 * footprint at start-up, or hosts whose own allocator already holds the
 * device's memory. The paper has no counterpart; it exists for those callers.
 * Decodes the frame in `in` (in_len bytes, device, 4-byte aligned, preceded
 * by the stream header when scan_index == 0) into planes_out (host array of
 * n_attr device pointers, H x W). stages: the stream's stage switches
 * (jiffy_options.stages, 0 for the full codec; for scan 0 they must match the
 * stream header, else CORRUPT). prev_planes (host array of n_attr device
 * pointers, nullable) must hold the previous frame's decoded planes when the
 * frame has P attributes (JIFFY_ERR_STATE if it is NULL then); it may be
 * planes_out itself (in-place decode: every previous pixel is read before the
 * same pixel is written). No handle is needed and nothing is allocated:
 * scratch is a fixed device array in the library, shared by every call (calls
 * that overlap on the GPU race on it). The first call on each device looks up
 * that array's address; make it before any stream capture. Limits: n_attr <=
 * 16, n_attr * H <= 16384, W <= 16384; beyond them JIFFY_ERR_INVALID_ARG, and
 * so is JIFFY_STAGE_ZSTD_MASK (its frames need scratch of their own).
 * Synchronizes cuda_stream. */
jiffy_status jiffy_decode_frame_noalloc(const void* in, size_t in_len, uint32_t H, uint32_t W, uint32_t n_attr,
                                        const jiffy_attr_desc* attrs, uint32_t scan_index, uint32_t stages,
                                        const void* const* prev_planes, void* const* planes_out, void* cuda_stream);

/* Checkpoint / resume. A stream's whole state is its previous scan as
 * decoded (q * P, the P predictor of the next frame, Sec. III-D) and its
 * frame counter; I frames need none of it. jiffy_stream_save_state writes it
 * to host memory host_buf (jiffy_stream_state_size(s) bytes: a header with
 * "JFYS", version 1, H, W, the attribute count, stage switches, frame counter
 * and each attribute's sample bytes and precision, then the previous scan's
 * planes), waiting for the copy; jiffy_stream_load_state restores such a
 * state into a stream of the same H, W, attributes and stage switches (either
 * role: encoders and decoders hold the same state), whose next frame then
 * continues the saved stream, P frames included. Errors: a null handle or
 * buffer, or a state of another configuration -> JIFFY_ERR_INVALID_ARG; too
 * small a buffer -> JIFFY_ERR_CAPACITY; a stream with an unfinished call or
 * enqueue-only calls not yet waited for -> JIFFY_ERR_STATE; a buffer that is
 * not a saved state of that size -> JIFFY_ERR_CORRUPT. The state of a stream
 * that has coded no frame since create/reset loads as such (next frame I). */
size_t jiffy_stream_state_size(const jiffy_stream* s);
jiffy_status jiffy_stream_save_state(jiffy_stream* s, void* host_buf, size_t capacity);
jiffy_status jiffy_stream_load_state(jiffy_stream* s, const void* host_buf, size_t len);

/* Copies src's previous scan and frame counter into dst (same H, W,
 * attributes and stage switches, same device, any roles), so that dst continues src's stream.
 * Encoders and decoders hold the same state, the previous scan as decoded
 * (q * P, Sec. III-D), so a decoder can take over from an encoder (e.g. to
 * decode the frame the encoder codes next) and the other way round.
 * Neither stream may be in an unfinished call (JIFFY_ERR_STATE).
 * Stream-ordered on cuda_stream; does not wait. */
jiffy_status jiffy_stream_copy_state(jiffy_stream* dst, const jiffy_stream* src, void* cuda_stream);

/* Failure-detection test hook (the failure is made on the host; nothing
 * faults): in the stream's next call, row item `row_item` -- numbered
 * (a * n_scans + t) * H + r over the call's scans t, attributes a and rows r
 * -- does not publish its status: a decoder row its completion (waited on by
 * the same row of the next frame when that is a P row), an encoder row its
 * last residual (waited on by the next row when that row's previous-row tail
 * holds no nonzero sample). A row that waits on it gives up after the bounded
 * device wait (2 s); the call then returns JIFFY_ERR_TIMEOUT, the stream's
 * state stays unchanged and the device stays usable. Applies to one call.
 * Errors: INVALID_ARG. */
jiffy_status jiffy_stream_test_withhold_row(jiffy_stream* s, uint32_t row_item);

/* Device bytes the stream holds now (state, tables and its own scratch). */
size_t jiffy_stream_device_bytes(const jiffy_stream* s);

/* Frames coded since create/reset (the next frame's scan_index). */
uint32_t jiffy_stream_frame_index(const jiffy_stream* s);

/* Human-readable name of a status code (static string). */
const char* jiffy_status_string(jiffy_status st);

/* ---- Input standardization (Sec. III-A): points given as floating-point
 * Cartesian coordinates become the canonical H x W image the codec takes:
 * spherical coordinates, rows by altitude (nearest beam), columns by azimuth,
 * ranges and attributes quantized to unsigned integers, 0 where a pixel has
 * no valid point. The arithmetic is exact integer arithmetic (the paper fixes
 * none): coordinates round(x * units_per_m) (float32 product, ties to even),
 * range = nearest integer to the Euclidean norm, angles by a 30-step CORDIC
 * in 32-bit integers (binary angles of 2^32 per turn, within 6e-8 rad of the
 * exact angle); a pixel hit by several points keeps the nearest (then the
 * first). */
typedef struct {
  uint32_t H, W;                 /* rows (beams) and columns, as jiffy_stream_create */
  const double* beam_altitude;   /* host, H entries, radians within +-pi/2, strictly decreasing
                                  * (row 0 = top beam); copied at create */
  double azimuth0;               /* radians: where column 0 starts, counterclockwise from +x */
  int32_t clockwise;             /* nonzero: columns advance clockwise (y is negated) */
  float units_per_m;             /* range unit per metre, e.g. 1000 for millimetres (> 0) */
  uint32_t range_bytes;          /* range sample size: 2 or 4 */
  uint32_t min_range, max_range; /* valid ranges in range units; others give 0 */
} jiffy_sensor_desc;

/* One per-point attribute: values (device, n_points floats), quantized as
 * round(v * scale) clamped to the sample type (v * scale <= 0 or NaN -> 0)
 * into out (device, H x W samples of dtype_bytes = 1, 2 or 4). */
typedef struct {
  const float* values;
  void* out;
  float scale;
  uint32_t dtype_bytes;
} jiffy_point_attr;

typedef struct jiffy_standardizer jiffy_standardizer;

/* Creates a standardizer for one sensor on `device` (owns a pixel table of
 * H x W x 8 bytes per scan of its largest call, and the beam table). Points more than half a beam spacing
 * above the first or below the last beam are dropped (H > 1). Errors:
 * INVALID_ARG (shape, unit, range size, non-decreasing or non-finite beams),
 * NOMEM, CUDA. */
jiffy_status jiffy_standardizer_create(jiffy_standardizer** out, const jiffy_sensor_desc* sensor, int device);

/* Releases the standardizer (synchronizes its device). */
void jiffy_standardizer_destroy(jiffy_standardizer* s);

/* Standardizes one scan: xyz (device, 3 * n_points floats, x y z per point,
 * metres) -> range_out (device, H x W samples of range_bytes, row-major) and
 * n_attr <= 16 attribute images (attrs: host array). Stream-ordered on
 * cuda_stream, does not wait; calls on one standardizer must be ordered on
 * one stream. Errors: INVALID_ARG, CUDA. */
jiffy_status jiffy_standardize(jiffy_standardizer* s, const float* xyz, uint32_t n_points, void* range_out,
                               uint32_t n_attr, const jiffy_point_attr* attrs, void* cuda_stream);

/* Standardizes n_scans <= 256 scans in one pass (two kernel launches for
 * all of them). Scan t's points are [point_offsets[t], point_offsets[t+1])
 * of xyz (host array of n_scans + 1 non-decreasing point indices, fewer than
 * 2^32 points per scan); the attributes' values are indexed the same way.
 * range_out and every attribute's out hold n_scans consecutive H x W images.
 * The first call with more scans than any before it reallocates the pixel
 * table (n_scans x H x W x 8 bytes) after waiting for cuda_stream. Otherwise
 * as jiffy_standardize; NOMEM if the table cannot grow. */
jiffy_status jiffy_standardize_seq(jiffy_standardizer* s, uint32_t n_scans, const float* xyz,
                                   const uint64_t* point_offsets, void* range_out, uint32_t n_attr,
                                   const jiffy_point_attr* attrs, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* JIFFY_H */
