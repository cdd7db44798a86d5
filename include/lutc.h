/*
 * lutc -- detector LUT generation and LUT-based image correction on GB300
 * (sm_103a), behind a plain C ABI.
 *
 * The paper's framework (Sections I-II) lets a client name a processing task,
 * hand over an input data set with a comma-separated parameter list (matrix
 * dimensions, data type, polynomial orders) and name where the results go;
 * generating look-up tables and correcting images with them is one of the
 * tasks it names (Section I).  Each entry point below is one such task on device memory: the
 * caller passes the input, the parameters and the output, the library runs
 * its own CUDA kernels on the caller's stream.
 *
 * The paper prints no formula for the task; the library defines it as follows
 * (M = 2^bits - 1, all arithmetic exact on integers, so every output is
 * bit-exact):
 *   (L) D[c][x] = clamp(floor((A[c] x^2 + G[c] x + O[c] + 2^15) / 2^16), 0, M)
 *       per detector (column) c, Q16 quadratic A, gain G, offset O -- the
 *       polynomial detector model whose coefficients the paper's
 *       least-squares fit produces (Section III-B).
 *   (P) corrected pixel d = D[c][min(raw, M)].
 *   (H) h[v] = number of pixels of a band with corrected value v (2^bits bins).
 *   (S) N = sum h; lo / hi = least v with 100 cdf(v) >= 2N / >= 98N;
 *       S[v] = 0 if hi == lo, else clamp(trunc(((v-lo) 255 + trunc((hi-lo)/2)) / (hi-lo)), 0, 255).
 *   (C) C[c][x] = S[D[c][x]].
 *   (A) out8 = C[c][min(raw, M)].
 *
 * Conventions shared by every call:
 *   - Pointers to pixels, tables, histograms and workspaces are DEVICE
 *     pointers owned by the caller; the library never allocates, frees or
 *     keeps them.  Descriptor structs (lutc_raster, lutc_coeffs arrays) are
 *     HOST memory, read during the call only.
 *   - Rasters are planar and band-sequential: band b, row y starts at byte
 *     b * height * pitch_bytes + y * pitch_bytes of `data`; pixels are uint16.
 *     Outputs use the same layout with their own row pitch.
 *   - Tables are [band][column][2^bits] (or [column][2^bits] for one band).
 *   - bits is 8..16; bands is 1..LUTC_MAX_BANDS.
 *   - Calls are asynchronous on `stream` (NULL = legacy default stream) and
 *     return a status: LUTC_OK, or a negative code from argument checks
 *     (detected before anything is enqueued) or from a failed kernel launch
 *     (LUTC_ECUDA).  No call throws, exits or aborts the process.
 */
#ifndef LUTC_H_
#define LUTC_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LUTC_API __attribute__((visibility("default")))
#else
#define LUTC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/** A cudaStream_t; NULL means the legacy default stream. */
typedef struct CUstream_st* lutc_stream;

/** Status codes. */
enum {
    LUTC_OK = 0,
    LUTC_EINVAL = -1,       /**< an argument is out of range or a pointer is NULL */
    LUTC_EUNSUPPORTED = -2, /**< valid in principle, not supported by this library version */
    LUTC_ENOMEM = -3,       /**< a workspace is too small / device memory exhausted */
    LUTC_ECUDA = -4,        /**< a CUDA call or kernel launch failed */
    LUTC_ETIMEOUT = -5,     /**< a bounded wait expired */
    LUTC_EBUSY = -6,        /**< admission refused (resource budget) */
    LUTC_ESHUTDOWN = -7,    /**< the object is shutting down */
    LUTC_ECANCELED = -8     /**< a queued request was withdrawn (lutc_server_cancel) */
};

#define LUTC_MIN_BITS 8
#define LUTC_MAX_BITS 16
#define LUTC_MAX_BANDS 64

/** Flags of lutc_correct_image. */
#define LUTC_STRETCH 1 /**< full pipeline, uint8 output; without it: detector only, uint16 output */

/** Q16 coefficients of one band: A (quadratic), G (gain), O (offset), each int32[ncols], device memory. */
typedef struct {
    const int32_t* A;
    const int32_t* G;
    const int32_t* O;
    int32_t ncols;
} lutc_coeffs;

/** A planar uint16 raster in device memory (layout in the file comment). */
typedef struct {
    const uint16_t* data;
    int64_t pitch_bytes; /**< >= 2 * width; the fast path wants data and pitch 16-byte aligned */
    int32_t width;       /**< columns (detectors), >= 0 */
    int32_t height;      /**< rows (scan lines), >= 0 */
    int32_t bands;       /**< 1..LUTC_MAX_BANDS */
    int32_t bits;        /**< DN bit depth, 8..16 */
} lutc_raster;

/** Library version, major * 10000 + minor * 100 + patch. */
LUTC_API int lutc_version(void);

/** Static, human-readable text of a status code. */
LUTC_API const char* lutc_strerror(int status);

/**
 * Step (L), the LUT generation of Section I: lut[c][x] = D[c][x] for c < ncols,
 * x < 2^bits.  lut: device uint16[ncols][2^bits], written in full.
 */
LUTC_API int lutc_lutgen(const lutc_coeffs* coeffs, int bits, uint16_t* lut, lutc_stream stream);

/**
 * Step (P), the image correction of Section I with a materialised LUT:
 * out[b][y][c] = lut[b][c][min(in[b][y][c], M)].
 * lut: device uint16[bands][width][2^bits]; out: device uint16 rows of out_pitch_bytes (>= 2 * width).
 */
LUTC_API int lutc_apply_u16(const lutc_raster* in, const uint16_t* lut, uint16_t* out, int64_t out_pitch_bytes,
                   lutc_stream stream);

/**
 * Step (H) with D evaluated from the coefficients: hist[b][v] for every band.
 * per_band: host array of in->bands coefficient sets (ncols == width).
 * hist: device uint64[bands][2^bits]; it is zeroed by the call, then filled.
 */
LUTC_API int lutc_hist(const lutc_raster* in, const lutc_coeffs* per_band, uint64_t* hist, lutc_stream stream);

/**
 * Step (S) for `bands` histograms: S[b][v] (device uint8[bands][2^bits]) and
 * lohi[b] = {lo, hi} (device int32[bands][2]).  N is the histogram's own sum.
 */
LUTC_API int lutc_stretch(const uint64_t* hist, int bands, int bits, uint8_t* S, int32_t* lohi, lutc_stream stream);

/**
 * Step (C) for one band: clut[c][x] = S[min(lut[c][x], M)].
 * lut: device uint16[ncols][2^bits]; S: device uint8[2^bits]; clut: device uint8[ncols][2^bits].
 */
LUTC_API int lutc_compose(const uint16_t* lut, const uint8_t* S, int ncols, int bits, uint8_t* clut, lutc_stream stream);

/**
 * Step (A) with a materialised composed LUT: out[b][y][c] = clut[b][c][min(in[b][y][c], M)].
 * clut: device uint8[bands][width][2^bits]; out: device uint8 rows of out_pitch_bytes (>= width).
 */
LUTC_API int lutc_apply_u8(const lutc_raster* in, const uint8_t* clut, uint8_t* out, int64_t out_pitch_bytes,
                  lutc_stream stream);

/** Bytes of workspace lutc_correct_image needs for this raster (0 if the raster is invalid). */
LUTC_API size_t lutc_correct_image_workspace(const lutc_raster* in);

/**
 * Byte offsets, inside that workspace, of the per-band tables the fused call
 * leaves behind: hist (uint64[bands][2^bits]), S (uint8[bands][2^bits]) and
 * lohi (int32[bands][2]).  Any output pointer may be NULL.  Returns LUTC_OK or LUTC_EINVAL.
 */
LUTC_API int lutc_correct_image_tables(const lutc_raster* in, size_t* hist_offset, size_t* S_offset, size_t* lohi_offset);

/**
 * The whole correction of a raster without materialising any LUT: Section I's
 * LUT generation and image correction as one task.
 * With LUTC_STRETCH: pass 1 evaluates D on chip and builds every band's
 * histogram (H), a scan builds S and lo/hi (S), pass 2 re-reads the raw
 * raster and writes out8 = S[D[c][raw]] (= steps C and A fused); out is
 * uint8.  Without it: one pass writes the uint16 detector-corrected raster
 * (P); out is uint16.
 * per_band: host array of in->bands coefficient sets (ncols == width).
 * workspace: device memory of at least lutc_correct_image_workspace(in)
 * bytes, 256-byte aligned, owned by the caller; it must not be shared with
 * another call in flight.  out_pitch_bytes >= width * sizeof(output element).
 */
LUTC_API int lutc_correct_image(const lutc_raster* in, const lutc_coeffs* per_band, int flags, void* out,
                       int64_t out_pitch_bytes, void* workspace, size_t workspace_bytes, lutc_stream stream);

/**
 * Pass 2 of the fused correction on its own (steps C and A without a
 * composed table): out8[b][y][c] = S[b][D[b][c][min(raw, M)]], with D
 * evaluated from the coefficients.  For callers that build S themselves, e.g.
 * from histograms summed over several devices before the scan.
 * S: device uint8[bands][2^bits], 16-byte aligned; out rows of out_pitch_bytes (>= width).
 */
LUTC_API int lutc_apply_stretch(const lutc_raster* in, const lutc_coeffs* per_band, const uint8_t* S, uint8_t* out,
                                int64_t out_pitch_bytes, lutc_stream stream);

/**
 * Reads and clears the current device's status word: 0, or the first error a
 * kernel of this library recorded on the device (LUTC_ETIMEOUT when a bounded
 * wait inside a kernel expired; the kernel then returned early and its
 * output is not valid).  Synchronises `stream`.  Returns LUTC_OK or LUTC_ECUDA.
 */
LUTC_API int lutc_device_status(int* status, lutc_stream stream);

/**
 * Exercises the kernels' failure path: launches one block that waits on an
 * mbarrier nothing will complete, with a limit of `wait_cycles` SM clock
 * cycles (1 .. 2^31) instead of the kernels' ~2 s; the wait gives up, records
 * LUTC_ETIMEOUT in the status word (see lutc_device_status) and the block
 * returns.  The device stays usable.  Asynchronous on `stream`; LUTC_EINVAL
 * for a limit out of range.
 */
LUTC_API int lutc_selftest_wait_timeout(long long wait_cycles, lutc_stream stream);

/**
 * Device workspace bytes of lutc_correct_image_host for this raster and flags
 * (0 for an invalid raster or flags): the fused path's tables, a device copy
 * of the raster and a staging area for the output (rows padded to 16 bytes).
 */
LUTC_API size_t lutc_correct_image_host_workspace(const lutc_raster* in, int flags);

/**
 * lutc_correct_image for a raster and an output in HOST memory: the same
 * result, with the host-to-device copies, both passes and the device-to-host
 * copies pipelined in chunks of rows (copy engines in both directions overlap
 * each other and the kernels; Section II's client-server round trip, whose
 * transfer cost the paper's future work sets out to cut).
 *
 * in: raster whose `data` is host memory (page-locked memory lets the copies
 *     run asynchronously and overlap; pageable memory works but serialises).
 *     Any pitch; layout as for lutc_correct_image.
 * per_band: device coefficients, as for lutc_correct_image.
 * out: host memory, uint8 (LUTC_STRETCH) or uint16 rows, band b row y at
 *     byte offset (b * height + y) * out_pitch_bytes.
 * workspace: device, >= lutc_correct_image_host_workspace(in, flags) bytes,
 *     256-byte aligned; caller-owned.
 * Work runs on `stream` and on two library-owned copy streams per device;
 * `stream` is made to wait for all of it, so work enqueued on `stream`
 * afterwards (or a synchronisation of it) sees the finished output.  Returns
 * LUTC_EINVAL / LUTC_ENOMEM before anything is enqueued, LUTC_ECUDA if an
 * enqueue fails.
 */
LUTC_API int lutc_correct_image_host(const lutc_raster* in, const lutc_coeffs* per_band, int flags, void* out,
                                     int64_t out_pitch_bytes, void* workspace, size_t workspace_bytes,
                                     lutc_stream stream);

/** Device workspace bytes of lutc_correct_frames_host for `frames` frames of this shape (two halves when frames > 1). */
LUTC_API size_t lutc_correct_frames_host_workspace(const lutc_raster* in, int flags, int frames);

/**
 * lutc_correct_image_host over a sequence of n frames of one sensor: every
 * frame has in's shape, pitch and bits and the same coefficients; frame f is
 * read from host memory at frames[f] and written to host memory at outs[f]
 * (out_pitch_bytes as for lutc_correct_image_host).  Frames alternate two
 * halves of the workspace, so a frame's copies in overlap the previous
 * frame's pass 2 and copies out.  Same stream semantics and errors as
 * lutc_correct_image_host (LUTC_EINVAL for n < 0 or a null frame or output).
 */
LUTC_API int lutc_correct_frames_host(const lutc_raster* in, const void* const* frames, int n,
                                      const lutc_coeffs* per_band, int flags, void* const* outs,
                                      int64_t out_pitch_bytes, void* workspace, size_t workspace_bytes,
                                      lutc_stream stream);

/* ------------------------------------------------------------------------
 * The paper's task interface.  A client names a task with a flag, passes a
 * comma-separated parameter list of at most 200 bytes (sizes of the data
 * and its element type, among others) and the data, and names where the
 * result goes (Section II, Fig. 3).  lutc_submit is that call in process;
 * the data and result buffers are passed as pointer arrays.
 * ------------------------------------------------------------------------ */

/** Task flags of lutc_submit. */
enum {
    LUTC_TASK_LUTGEN = 1,        /**< in {A, G, O}; out {lut}; params width, bits */
    LUTC_TASK_HIST = 2,          /**< in {raster, A, G, O}; out {hist}; params width, height, bands, bits[, pitch] */
    LUTC_TASK_STRETCH = 3,       /**< in {hist}; out {S, lohi}; params bands, bits */
    LUTC_TASK_COMPOSE = 4,       /**< in {lut, S}; out {clut}; params width, bits */
    LUTC_TASK_APPLY = 5,         /**< in {raster, table}; out {out}; params width, height, bands, bits, table=u16|u8[, pitch, out_pitch] */
    LUTC_TASK_CORRECT_IMAGE = 6, /**< in {raster, A, G, O}; out {out}; params width, height, bands, bits[, stretch, pitch, out_pitch]; workspace */
    LUTC_TASK_DEVICE_INFO = 7,   /**< out {char buffer} (HOST); params capacity */
    LUTC_TASK_DEMOSAIC = 8,      /**< in {raster[, A, G, O]}; out {rgb}; params width, height, bits, pattern=rggb|bggr|grbg|gbrg[, pitch, out_pitch] */
    LUTC_TASK_FIT = 9            /**< in {x, y}; out {coef, status[, q16]}; params width (detectors), height (lines), order, targets=line|sample[, pitch] */
};

#define LUTC_PARAMS_MAX 200 /**< longest parameter string (the paper's 200-byte header field) */

/**
 * Runs task `task` with parameters `params` ("key=value,key=value", ASCII,
 * at most LUTC_PARAMS_MAX bytes, no spaces).  A, G, O are device int32 arrays
 * of [bands][width]; raster and outputs are device buffers with the layouts
 * of the matching lutc_* call (pitch and out_pitch in bytes default to
 * packed rows).  workspace is needed by LUTC_TASK_CORRECT_IMAGE with
 * stretch=1 (lutc_correct_image_workspace bytes); stretch defaults to 1.
 * Returns the task's status, or LUTC_EINVAL for an unknown task, a malformed,
 * unknown, missing or out-of-range parameter, or too few buffers; nothing is
 * enqueued then.
 */
LUTC_API int lutc_submit(int task, const char* params, const void* const* inputs, int n_inputs,
                         void* const* outputs, int n_outputs, void* workspace, size_t workspace_bytes,
                         lutc_stream stream);

/**
 * The paper's remote-GPU information utility (Section IV): writes an XML
 * document listing every visible GPU -- name, compute capability, warp size,
 * total constant memory, total global memory, shared memory per block, clock
 * rate, multiprocessor count, registers per block, maximum threads per block,
 * maximum grid size and maximum block dimensions -- into the HOST buffer xml
 * of `capacity` bytes (NUL-terminated).  *needed (may be NULL) receives the
 * bytes the document needs.  Returns LUTC_OK, LUTC_ENOMEM when capacity is
 * too small (nothing useful written), or LUTC_EINVAL.  With no GPU visible the
 * document lists none.
 */
LUTC_API int lutc_device_info(char* xml, size_t capacity, size_t* needed);

/**
 * Measurement aid beside the device listing: the listing states the clock and
 * the multiprocessor count, not the fp64 fused multiply-add rate that bounds
 * the least-squares fit (Section III-B).  Launches `blocks` (1 .. 2^20) blocks
 * of 256 threads on `stream`, each thread running `iters` (1 .. 2^24) rounds
 * of 8 independent fp64 FMA chains on registers and storing one double to
 * sink[block * 256 + thread] (device memory, blocks * 256 doubles, caller
 * owned).  *fmas (may be NULL) receives the FMAs the launch performs; timing
 * the launch with CUDA events on `stream` gives the device's FMA rate.
 * Asynchronous.  Returns LUTC_OK, LUTC_EINVAL or LUTC_ECUDA.
 */
LUTC_API int lutc_probe_fp64_fma(int blocks, long long iters, double* sink, long long* fmas, lutc_stream stream);

/* ------------------------------------------------------------------------
 * The paper's transport (Section II, Fig. 3): a TCP server in front of
 * lutc_submit.
 *
 * Request: the 260-byte header -- task name (29 bytes, NUL-padded: "lutgen",
 * "hist", "stretch", "compose", "apply", "correct_image", "device_info",
 * "demosaic", "fit"), the byte '+', the parameter list (200 bytes,
 * NUL-padded, as for lutc_submit) and the output name (30 bytes) -- then the
 * payload length (uint64, little endian) and the payload: the task's inputs
 * in lutc_submit's order, packed back to back, rasters and tables with packed
 * rows (demosaic: the three coefficient arrays are optional).  Reply: status
 * (int32, little endian), the output name echoed (30 bytes), the result
 * length (uint64) and the task's outputs packed back to back (device_info:
 * the XML text).  A malformed header, an unknown task or a payload whose
 * length does not match the parameters is answered with LUTC_EINVAL and an
 * empty result; the connection stays usable.
 * ------------------------------------------------------------------------ */

typedef struct lutc_net_server lutc_net_server;
#define LUTC_NET_HEADER_BYTES 260

/**
 * Listens on `address` (dotted IPv4, NULL = 127.0.0.1) and `port` (0 = any
 * free port, see lutc_net_server_port) and serves every connection on its own
 * thread and CUDA stream of GPU `device`.  Returns LUTC_EINVAL for bad
 * arguments, LUTC_EBUSY if the socket cannot be bound.
 */
LUTC_API int lutc_net_server_create(const char* address, int port, int device, lutc_net_server** out);
/** The bound TCP port. */
LUTC_API int lutc_net_server_port(const lutc_net_server* server);
/** Requests answered so far, and how many of them with a non-zero status. */
LUTC_API int lutc_net_server_stats(const lutc_net_server* server, uint64_t* requests, uint64_t* failures);
/** Stops listening, closes every connection (after the request in progress) and frees the server. */
LUTC_API int lutc_net_server_destroy(lutc_net_server* server);

/* ------------------------------------------------------------------------
 * Bilinear Bayer demosaicing (Section III.A, case study 1), optionally fused
 * with the detector correction.
 * ------------------------------------------------------------------------ */

/** Colour filter array patterns, named by the 2x2 cell read row by row from the raster's origin. */
enum { LUTC_BAYER_RGGB = 0, LUTC_BAYER_BGGR = 1, LUTC_BAYER_GRBG = 2, LUTC_BAYER_GBRG = 3 };

/**
 * out[k][y][x], k = R, G, B: a pixel keeps its own colour; each missing colour
 * is the average of the neighbours of that colour among its 8 direct
 * neighbours inside the image, rounded half up in integers,
 * (sum + count/2) / count (0 when no such neighbour exists, which happens only
 * in images one pixel wide or high).  With `coeffs` (one band, ncols == width)
 * every photosite is first replaced by its detector-corrected value
 * D[x][min(raw, 2^bits - 1)] (step L), so the interpolation sees corrected
 * values; without, the raw values are used as they are.
 *
 * in: one-band raster (bands == 1); any pitch and alignment, 16-byte aligned
 *     rows take vector loads.  pattern: LUTC_BAYER_*.
 * out: device uint16, three planes of in->height rows, plane k row y at byte
 *     offset (k * height + y) * out_pitch_bytes (>= 2 * width, even); 16-byte
 *     aligned rows take vector stores.
 * Returns LUTC_EINVAL for a bad raster, pattern, output or coefficient set
 * before any launch; an empty raster returns LUTC_OK with nothing launched.
 * LUTC_EUNSUPPORTED, before any launch, for a frame of more than 1 048 560
 * rows that the persistent TMA-fed kernel does not take (rows not 16-byte
 * aligned, fewer than 144 columns, or a raw frame of at most 4 M pixels).
 * Asynchronous on `stream`.
 */
LUTC_API int lutc_demosaic(const lutc_raster* in, const lutc_coeffs* coeffs, int pattern, uint16_t* out,
                           int64_t out_pitch_bytes, lutc_stream stream);

/* ------------------------------------------------------------------------
 * Per-detector least-squares polynomial fit (Section III.B, case study 2):
 * the calibration step that produces the coefficients the LUT is built from.
 * ------------------------------------------------------------------------ */

#define LUTC_FIT_MAX_ORDER 3
#define LUTC_FIT_MAX_LINES 65536 /**< the exact 64-bit power sums of x^3 hold up to 2^16 lines */

/**
 * For every column c < ncols, the polynomial f_c(x) = a_0 + a_1 x + ... +
 * a_m x^m of order m = `order` (1..3) that minimises
 * sum_{i<n} (y_i - f_c(x[i][c]))^2, by the normal equations the paper
 * derives (zero first derivatives of the squared error), solved in fp64.
 *
 * x: device uint16, n calibration lines of ncols samples, line i at byte
 *    offset i * x_pitch_bytes (>= 2 * ncols, even).
 * y: device doubles: with y_pitch_bytes == 0, one target per line (y[i]);
 *    otherwise one per sample, line i at byte offset i * y_pitch_bytes
 *    (>= 8 * ncols, multiple of 8).
 * coef: device double[ncols][order + 1], a_0 first.
 * status: device int32[ncols]: 0 fitted; 1 fewer than order + 1 distinct
 *    abscissae in the column (singular system; coefficients NaN, codes 0);
 *    2 a Q16 code out of range (codes 0).
 * q16: NULL, or (order <= 2) device int32[3][ncols]: the rows A, G, O of the
 *    Q16 coefficients of D(x) = A x^2 + G x + O that lutc_lutgen consumes,
 *    round(a_2 2^16), round(a_1 2^16), round(a_0 2^16) (half away from zero;
 *    A = 0 for order 1); a code of magnitude above 2^31 - 1 sets status 2.
 * Returns LUTC_EINVAL (order outside 1..3, n < order + 1 or above
 * LUTC_FIT_MAX_LINES, q16 with order 3,
 * null or misaligned buffers, bad pitches) before any launch; ncols == 0
 * returns LUTC_OK with nothing launched.  Asynchronous on `stream`.
 * Accuracy: the normal equations square the conditioning of the samples'
 * Vandermonde matrix; columns whose abscissae span a narrow range lose
 * digits accordingly (a property of the method, not of the kernel).
 */
LUTC_API int lutc_fit(const uint16_t* x, int64_t x_pitch_bytes, const double* y, int64_t y_pitch_bytes, int n,
                      int ncols, int order, double* coef, int32_t* status, int32_t* q16, lutc_stream stream);

/* ------------------------------------------------------------------------
 * Batches: many independent rasters corrected by one persistent launch per
 * phase.  The paper's server receives tasks from many clients (Sections I-II);
 * a batch is a set of such tasks of uneven size, bit depth and band count,
 * each with its own coefficients, run together so that the GPU stays full.
 * ------------------------------------------------------------------------ */

/** One image of a batch.  Pointers as in lutc_correct_image; per_band is a
 *  host array of in.bands coefficient sets that is read by lutc_batch_create
 *  only.  out is uint8 with LUTC_STRETCH, uint16 without. */
typedef struct {
    lutc_raster in;
    const lutc_coeffs* per_band;
    void* out;
    int64_t out_pitch_bytes;
    int32_t flags;
} lutc_job;

/** Launch configuration of a batch; every field 0 = choose automatically. */
typedef struct {
    int32_t column_threads; /**< 64, 128 or 256: strip width 8 * column_threads for every image */
    int32_t blocks_per_sm;  /**< cap of resident blocks per SM (0 = occupancy maximum) */
    int32_t use_graph;      /**< 1: the first lutc_batch_run captures the batch in a CUDA graph, later runs replay it */
} lutc_batch_config;

/** A prepared batch (host object; its device data lives in the caller's workspace). */
typedef struct lutc_batch_st* lutc_batch;

/** Workspace bytes a batch of these jobs needs (0 if a job is invalid). */
LUTC_API size_t lutc_batch_workspace(const lutc_job* jobs, int n);

/**
 * Validates the jobs, plans the launches and writes the device descriptors
 * (job table, tensor maps, coefficient pointers) into `workspace` with
 * copies enqueued on `stream`.  The jobs' rasters, coefficients and outputs
 * must stay valid until lutc_batch_destroy.  config may be NULL.  Images the
 * TMA kernels cannot take (unaligned rows, width < 256, 16-bit) are corrected
 * one by one inside the batch with lutc_correct_image.  Returns LUTC_OK,
 * LUTC_EINVAL (bad job, *out untouched), LUTC_ENOMEM (workspace too small)
 * or LUTC_ECUDA.
 */
LUTC_API int lutc_batch_create(const lutc_job* jobs, int n, const lutc_batch_config* config, void* workspace,
                               size_t workspace_bytes, lutc_stream stream, lutc_batch* out);

/**
 * Enqueues the whole batch on `stream`: one histogram pass, one scan and one
 * gather pass for all LUTC_STRETCH images, one pass for all detector-only
 * images, then the images corrected one by one.  With use_graph the first
 * call captures this sequence in a CUDA graph (on an internal stream; make
 * that first call before capturing `stream` yourself) and every call
 * launches the graph.  Results equal lutc_correct_image on each image.
 * The passes balance their blocks at run time (a block that finishes its
 * planned share takes half of the largest share left); every run starts
 * from the planned shares again.  Runs of one batch share its workspace
 * (histograms, tables, the blocks' shares): runs that overlap on the GPU
 * race, so enqueue them on one stream.
 */
LUTC_API int lutc_batch_run(lutc_batch batch, lutc_stream stream);

/** Device pointers of job `job`'s tables after a run (LUTC_STRETCH jobs): hist
 *  uint64[bands][2^bits], S uint8[bands][2^bits], lohi int32[bands][2]. */
LUTC_API int lutc_batch_tables(lutc_batch batch, int job, uint64_t** hist, uint8_t** S, int32_t** lohi);

/** Releases the host object and its graph; the workspace is the caller's. */
LUTC_API int lutc_batch_destroy(lutc_batch batch);

/**
 * The whole batch in one call: plans the jobs as lutc_batch_create does,
 * enqueues them once on `stream` (no graph) and releases the plan.  config
 * may be NULL (automatic configuration); a configuration returned by
 * lutc_batch_autotune for the same kind of batch may be passed instead (its
 * use_graph is ignored).  workspace: lutc_batch_workspace(jobs, n) bytes of
 * device memory, 256-byte aligned, in use until the enqueued work completes.
 * Returns what lutc_batch_create or lutc_batch_run returns.
 */
LUTC_API int lutc_batch_correct(const lutc_job* jobs, int n, const lutc_batch_config* config, void* workspace,
                                size_t workspace_bytes, lutc_stream stream);

/**
 * The batch autotuner: times every launch configuration (strip width x
 * blocks per SM) on these jobs -- `reps` runs each after one warm-up run, CUDA
 * events on `stream`, which it synchronises -- and writes the fastest to
 * *best (use_graph set) and its mean time in ms to *best_ms (may be NULL).
 * The outputs are written by every trial.
 */
LUTC_API int lutc_batch_autotune(const lutc_job* jobs, int n, void* workspace, size_t workspace_bytes,
                                 lutc_stream stream, int reps, lutc_batch_config* best, float* best_ms);

/* ------------------------------------------------------------------------
 * Serving: an in-process request loop that plays the paper's GPU server
 * (Sections I-II: clients submit a task, its data and parameters, and get
 * the result back).  Requests are queued, admitted against a device-memory
 * budget, grouped into batches of up to max_batch requests or max_wait_us,
 * and run as overlapping batches on up to `streams` CUDA streams while new
 * requests keep arriving (continuous batching).  A request that arrives while
 * no batch is on the device launches at once (waiting would only add
 * latency); requests that arrive while batches run accumulate until a batch
 * is full, the window ends, or the device goes idle.  Each sensor's
 * coefficients are uploaded to the device on its first request and cached.
 * ------------------------------------------------------------------------ */

/** Server configuration; zero fields take the defaults in brackets. */
typedef struct {
    size_t budget_bytes;  /**< device memory for request buffers and batch tables [40 GiB] */
    int32_t max_batch;    /**< requests per batch [32] */
    int32_t max_wait_us;  /**< longest a request waits for its batch to fill [2000]; 1 = launch at once */
    int32_t streams;      /**< batches in flight [3] */
    int32_t max_queue;    /**< pending requests before submit returns LUTC_EBUSY [4096] */
    int32_t fake_device;  /**< test facility: 1 = run no CUDA at all; a batch "completes" fake_latency_us after launch */
    int32_t fake_latency_us;
    int32_t fail_every;   /**< test facility: when > 0, every fail_every-th batch is failed on the host with LUTC_ECUDA */
    int32_t hold_when_idle; /**< 1: every batch waits out its window even on an idle device; 0 [default]: launch at once when idle */
} lutc_server_config;

/** Request flags. */
#define LUTC_REQ_HOST 2 /**< raster and output are HOST memory: the server copies them in and out */

/** Per-request outcome, filled by lutc_server_wait. */
typedef struct {
    int32_t status;      /**< LUTC_OK, LUTC_ECUDA (failed batch), LUTC_ESHUTDOWN (server closed first),
                              LUTC_ECANCELED (withdrawn by lutc_server_cancel) */
    int32_t batch_size;  /**< requests in the batch that carried it */
    double submit_s;     /**< host steady-clock seconds at submit */
    double start_s;      /**< ... when its batch was formed */
    double launched_s;   /**< ... when its batch's work had been enqueued */
    double done_s;       /**< ... when its batch was seen complete */
    int32_t cache_miss;  /**< 1 if this request uploaded its sensor's coefficients */
    int32_t pad;
} lutc_request_info;

typedef struct lutc_server_st* lutc_server;

/** Creates a server (config may be NULL) on the current device; starts its threads. */
LUTC_API int lutc_server_create(const lutc_server_config* config, lutc_server* out);

/**
 * Registers sensor `sensor_id` (0..65535): its raster geometry and host
 * coefficient arrays A, G, O of [bands][width] int32 (copied).  Nothing is
 * uploaded until its first request.  Returns LUTC_OK or LUTC_EINVAL.
 */
LUTC_API int lutc_server_register_sensor(lutc_server server, int sensor_id, int width, int bands, int bits,
                                         const int32_t* A, const int32_t* G, const int32_t* O);

/**
 * Queues one request: the sensor's raster of `height` rows (row pitch
 * pitch_bytes) is corrected with LUTC_STRETCH into out (row pitch
 * out_pitch_bytes, uint8).  With LUTC_REQ_HOST in flags both are host
 * memory; otherwise device memory.  Buffers must stay valid until the ticket
 * completes.  Returns LUTC_OK and a ticket, LUTC_EINVAL, LUTC_EBUSY (queue
 * full, or the request alone exceeds the budget) or LUTC_ESHUTDOWN.
 */
LUTC_API int lutc_server_submit(lutc_server server, int sensor_id, const uint16_t* raster, int height,
                                int64_t pitch_bytes, uint8_t* out, int64_t out_pitch_bytes, int flags,
                                uint64_t* ticket);

/**
 * Waits up to timeout_us (< 0: forever) for a ticket; on completion fills
 * *info (may be NULL) and forgets the ticket.  Returns LUTC_OK (see
 * info->status for the request's own outcome), LUTC_ETIMEOUT (still
 * running; the ticket stays valid) or LUTC_EINVAL (unknown ticket).
 */
LUTC_API int lutc_server_wait(lutc_server server, uint64_t ticket, int64_t timeout_us, lutc_request_info* info);

/**
 * Withdraws a request that is still queued (not yet taken into a batch): it
 * completes at once with status LUTC_ECANCELED and its buffers are not touched
 * again; lutc_server_wait returns it as usual.  Returns LUTC_OK, LUTC_EBUSY when
 * the request is already in a batch or done (it then completes normally), or
 * LUTC_EINVAL for an unknown ticket.
 */
LUTC_API int lutc_server_cancel(lutc_server server, uint64_t ticket);

/** One request of a replayed schedule (lutc_server_replay); the fields after at_s are lutc_server_submit's. */
typedef struct {
    double at_s;             /**< arrival, seconds after the replay starts (0 ..  3600, non-decreasing) */
    const uint16_t* raster;
    uint8_t* out;
    int64_t pitch_bytes;
    int64_t out_pitch_bytes;
    int32_t sensor_id;
    int32_t height;
    int32_t flags;
    int32_t pad;
} lutc_replay_request;

/**
 * Open-loop load generator: a native thread of the library submits
 * requests[i] when its arrival time is due (a request the queue refuses with
 * LUTC_EBUSY is retried every 20 us, for up to 120 s), while the calling
 * thread collects every ticket in order.  info[i] receives the request's
 * outcome (lutc_server_wait) and scheduled_s[i] (may be NULL) the
 * steady-clock second it was due, on the clock of info's timestamps:
 * latency = info[i].done_s - scheduled_s[i] counts any lateness of the
 * hand-over (info[i].submit_s - scheduled_s[i]) against the request.  All
 * arrival times 0 make a closed burst.  Blocks until every request has
 * completed.  Returns LUTC_OK; LUTC_EINVAL for bad arguments (nothing is
 * submitted); or the first submit or wait error, after which the remaining
 * requests are not submitted and their info[].status holds that error.
 */
LUTC_API int lutc_server_replay(lutc_server server, const lutc_replay_request* requests, int n,
                                lutc_request_info* info, double* scheduled_s);

/** Counters: requests completed, batches launched, bytes of the budget in use now, largest batch. */
LUTC_API int lutc_server_stats(lutc_server server, uint64_t* completed, uint64_t* batches, size_t* budget_in_use,
                               int32_t* largest_batch);

/** Stops the threads: pending requests complete with LUTC_ESHUTDOWN, batches in flight finish; frees everything. */
LUTC_API int lutc_server_destroy(lutc_server server);

/** Kernel families of the fused path (lutc_tuning.path). */
#define LUTC_PATH_AUTO 0  /**< TMA-staged kernels when the raster allows them, else strip kernels */
#define LUTC_PATH_TMA 1   /**< TMA-staged persistent kernels (needs 16-byte aligned rows, width >= 256) */
#define LUTC_PATH_STRIP 2 /**< plain strip kernels with 16-byte vector loads (any alignment) */

/**
 * Launch configuration of the fused path for one bit depth.  Every field 0
 * means "choose automatically".  column_threads (64, 128 or 256) sets the
 * strip width to 8 * column_threads detectors; blocks_per_sm caps the
 * persistent grid below the occupancy maximum.  Results never depend on
 * these settings, only speed does.
 */
typedef struct {
    int32_t path;
    int32_t column_threads;
    int32_t blocks_per_sm;
} lutc_tuning;

/**
 * Sets (tuning != NULL) or resets to automatic (NULL) the process-wide launch
 * configuration used for rasters of `bits` (8..16) by lutc_hist,
 * lutc_apply_stretch and lutc_correct_image; an autotuner calls this with the
 * fastest configuration it measured.  Takes effect for calls made after it
 * returns.  Returns LUTC_OK or LUTC_EINVAL.
 */
LUTC_API int lutc_set_tuning(int bits, const lutc_tuning* tuning);

/** Reads the configuration lutc_set_tuning stored for `bits` (all zero if automatic). */
LUTC_API int lutc_get_tuning(int bits, lutc_tuning* tuning);

/**
 * Which kernel family the calling host thread's most recent call with pixels
 * to process ran -- lutc_hist, lutc_apply_stretch or lutc_correct_image
 * (either mode), or the host-raster calls built on them: LUTC_PATH_TMA (the
 * TMA-staged persistent kernels) or LUTC_PATH_STRIP (the plain strip
 * kernels); LUTC_PATH_AUTO (0) before this thread has made such a call.  The
 * TMA family needs 16-byte aligned rows, width >= 256, bands * height < 2^31,
 * the driver's tensor-map encoder and a tuning that allows it; a call that
 * cannot have it runs the strip kernels with the same result, and this query
 * is how a caller (or a measurement) sees which one ran.  Calls rejected by
 * their argument checks, and empty rasters, leave it unchanged.  Per host
 * thread; no GPU work.  Returns LUTC_OK, or LUTC_EINVAL when path is NULL.
 */
LUTC_API int lutc_last_path(int* path);

/** Size of the fixed device scratch array behind lutc_correct_image_static (1 MiB per GPU). */
#define LUTC_STATIC_SCRATCH_BYTES (1u << 20)

/**
 * lutc_correct_image without a caller-provided workspace, for callers that
 * cannot allocate device memory: a plain C client with no device allocator
 * of its own, a latency-bound loop in which an allocation would stall the
 * device, or a framework whose memory manager owns every device allocation.
 * The paper has no counterpart: this is a convenience of this library, not a
 * step of the method.
 *
 * Same arguments and result as lutc_correct_image, minus the workspace; the
 * arguments are checked in the same order, so a malformed raster, a NULL
 * coefficient set, an unknown flag or a bad output gives LUTC_EINVAL whatever
 * the raster's size.  With LUTC_STRETCH the scratch (per-band histogram,
 * stretch table and lo/hi) comes from one file-scope device array of
 * LUTC_STATIC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits; the call allocates nothing.  A raster whose tables need
 * more than that is rejected with LUTC_ENOMEM before anything is enqueued:
 * the tables take 9 * 2^bits bytes per band (plus 256-byte rounding), so
 * 1 MiB holds at most 1 band at 16 bits, 3 at 15, 7 at 14, 14 at 13, 28 at
 * 12, 56 at 11 and every band count (LUTC_MAX_BANDS) at 10 bits or fewer;
 * lutc_correct_image_workspace(in) <= LUTC_STATIC_SCRATCH_BYTES is the exact
 * test.  Without LUTC_STRETCH no scratch is used and any raster is accepted.
 *
 * The first call with LUTC_STRETCH on a device looks up the array's device
 * address on the current device (cudaGetSymbolAddress) and caches it; make
 * that first call before any stream capture on that device.  Every call on a
 * device shares the one array, which keeps the previous call's tables (the
 * histogram is cleared at the start of each call): calls that overlap on the
 * GPU -- concurrent streams, or host threads without ordering -- race on it
 * and give wrong results.  Serialise them on one stream.
 */
LUTC_API int lutc_correct_image_static(const lutc_raster* in, const lutc_coeffs* per_band, int flags, void* out,
                                       int64_t out_pitch_bytes, lutc_stream stream);

/** Phases lutc_trace_read reports per traced call. */
#define LUTC_TRACE_PHASES 3 /**< pass 1 (histogram clear + histogram), scan, pass 2 */

/**
 * Tracing of lutc_correct_image (with LUTC_STRETCH) and of lutc_batch_run
 * without a graph: while enabled, each call records a CUDA event on its
 * stream before pass 1 and after each phase, for up to `capacity` calls (a
 * batch's last phase also covers its detector-only and one-by-one images).  capacity 0 disables tracing and releases the
 * events.  Process-wide; not for concurrent callers.  Returns LUTC_OK,
 * LUTC_EINVAL or LUTC_ECUDA.
 */
LUTC_API int lutc_trace_enable(int capacity);

/**
 * Waits for the recorded events and writes the phase durations in
 * milliseconds, ms[call * LUTC_TRACE_PHASES + phase], for at most max_calls
 * traced calls; then starts a new trace.  Returns the number of calls
 * written (>= 0) or a negative status.
 */
LUTC_API int lutc_trace_read(float* ms, int max_calls);

#ifdef __cplusplus
}
#endif

#endif /* LUTC_H_ */
