/*
 * decolor.h - C ABI of the GB300 colour-temperature decolorization library
 * (libdecolor.so, built for sm_103a).
 *
 * The library computes the luminance of Eq. 1-6 of Ambalathankandy, Ou and Ikebe,
 * "A color temperature-based high-speed decolorization: an empirical approach for
 * tone mapping applications" (arXiv 2108.13656), Sec. II-B, and fuses it with the
 * global tone curve of Sec. III-B-1 and the smoothed local-histogram-equalisation
 * tone mapping of Sec. III-B-2.  Every pass of a call is one persistent CUDA launch
 * over a (possibly ragged) batch of images of one input sample type.
 *
 * Conventions shared by every entry point
 *  - Images are interleaved RGB (R, G, B per pixel, no padding between pixels),
 *    row-major, with an arbitrary row stride in bytes.  Samples are 8-bit codes
 *    (DC_U8, read as code/255, no linearisation), IEEE binary16 (DC_F16) or
 *    binary32 (DC_F32) linear values.  Negative samples are read as 0.
 *  - 8-bit input is "LDR"; binary16/binary32 input is "HDR".  The tone-mapping
 *    statistics use L for LDR and ln(L + delta) for HDR (see each call).
 *  - Outputs are one channel of the same width and height: DC_U8 (the value y in
 *    [0,1] rounded to floor(255 y + 1/2), clamped), DC_F16 (round to nearest even)
 *    or DC_F32.
 *  - All pointers inside dc_image_in / dc_image_out, `stats` and `ws` are DEVICE
 *    pointers owned by the caller.  The descriptor arrays `in` and `out` and the
 *    parameter structs are HOST memory, read during the call only.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  They never allocate device memory and never synchronise.  Input must
 *    not overlap output.  Two calls that share a workspace must be ordered (same
 *    stream or an event between them).
 *  - Return value: DC_OK or a DC_ERR_* code.  A call is a short chain of passes
 *    (one persistent kernel each, chained with programmatic dependent launch on
 *    `stream`); no kernel ever waits for another CTA, so a call cannot hang on the
 *    device.  Argument errors (DC_ERR_INVALID_ARG, DC_ERR_UNSUPPORTED_DTYPE,
 *    DC_ERR_WORKSPACE, DC_ERR_TOO_MANY) are found before anything is enqueued.
 *    DC_ERR_CUDA from a failed memset or launch can come after earlier passes of
 *    the same call were enqueued: the outputs are then incomplete, and the next
 *    call on that workspace (registered or not) clears the counters those passes
 *    left before it starts.
 *  - Vector path: when an image's data pointers and row strides are 16-byte
 *    aligned, pixels move in 16-byte vectors; otherwise the image takes a scalar
 *    path with the same results.
 *  - Limits: width, height >= 1; width * height <= 2^28 per image; at most
 *    DC_MAX_BATCH images per call.
 */
#ifndef DECOLOR_H
#define DECOLOR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DC_API __attribute__((visibility("default")))
#else
#define DC_API
#endif

/* ---- status codes ---- */
#define DC_OK 0
#define DC_ERR_INVALID_ARG 1       /* a size, stride, pointer or parameter is out of range */
#define DC_ERR_UNSUPPORTED_DTYPE 2 /* a dtype is not DC_U8 / DC_F16 / DC_F32 */
#define DC_ERR_WORKSPACE 3         /* ws is NULL, misaligned (256 B) or smaller than needed */
#define DC_ERR_CUDA 4              /* a CUDA runtime call failed (launch, memset, attribute) */
#define DC_ERR_TIMEOUT 5           /* reserved: a device-side wait ran past its limit */
#define DC_ERR_TOO_MANY 6          /* more than DC_MAX_BATCH images */

/* ---- sample types ---- */
#define DC_U8 0
#define DC_F16 1
#define DC_F32 2

/* ---- operations (for dc_workspace_bytes and the tuning table) ---- */
#define DC_OP_DECOLORIZE 0
#define DC_OP_GLOBAL 1
#define DC_OP_LOCAL 2

/* ---- global curve modes ---- */
#define DC_SIGMOID 0 /* centred sigmoid (Sec. III-B-1) */
#define DC_HISTEQ 1  /* histogram equalisation (global analogue of Sec. III-B-2) */

#define DC_MAX_BATCH 4096
#define DC_MAX_BINS 32

typedef struct {
    const void* data;     /* device pointer to the first pixel of the first row */
    int32_t width;        /* pixels per row, >= 1 */
    int32_t height;       /* rows, >= 1 */
    int64_t stride_bytes; /* bytes between rows, >= 3 * width * sample size */
    int32_t dtype;        /* DC_U8, DC_F16 or DC_F32 */
    int32_t reserved;     /* must be 0 */
} dc_image_in;

typedef struct {
    void* data;           /* device pointer, width x height x channels samples of `dtype` */
    int64_t stride_bytes; /* bytes between rows, >= width * channels * sample size */
    int32_t dtype;        /* DC_U8, DC_F16 or DC_F32 */
    int32_t channels;     /* 0 or 1: the gray (tone-mapped) plane; 3: interleaved RGB colour
                             reconstruction of the tone-mapped image (tone-mapping calls only),
                             C_out = min(1, y (C_in / L)^color_s) per channel, a black pixel
                             (L = 0) giving y in every channel.  The paper shows colour
                             tone-mapped images (Fig. tmo_1, Fig. GTMO, Sec. II-D) without
                             stating how they are formed; this is the library's reading. */
} dc_image_out;

/* Luminance channel the tone mapping works on (Sec. III-B-1, Fig. GTMO, compares the
 * paper's channel with Y of YCbCr and V of HSV). */
#define DC_LUMA_OURS 0 /* Eq. 1-6 (Sec. II-B) */
#define DC_LUMA_Y 1    /* Gray = 0.2989 R + 0.5870 G + 0.1140 B (MATLAB rgb2gray, quoted in Sec. I) */
#define DC_LUMA_V 2    /* V of HSV = max(R, G, B) */
#define DC_LUMA_LSTAR 3 /* CIE L* of CIELAB / 100 (Sec. I, Fig. 2, Table 1): 116 f(Y) - 16 of the
                          Rec. 709 / sRGB luminance Y (D65 white), 8-bit codes decoded with
                          the sRGB transfer function first; not offered for 8-bit input with
                          an f32 output through the local operator (DC_ERR_UNSUPPORTED_DTYPE:
                          its binary32 cube root is too coarse for that output's tolerance) */

/* Eq. 3 and Eq. 6 weights; the paper uses beta_r = 0.55 and beta_k = 0.8
 * (Sec. II-B).  The paper states 0.5 < beta < 1; the library accepts [0, 1].
 * luma selects the channel (DC_LUMA_*; the betas are used by DC_LUMA_OURS only);
 * color_s in [0, 8] is the saturation exponent of colour outputs (1 keeps every
 * channel's ratio to the luminance, 0 gives gray; unused for gray outputs). */
typedef struct {
    float beta_r;
    float beta_k;
    int32_t luma;
    float color_s;
} dc_decolor_params;

/* Global curve (Sec. III-B-1 names it a centred sigmoid and prints no formula):
 *  DC_SIGMOID: y = 1 / (1 + exp(-gain_k * (ln(L + delta) - mu))), mu = mean of
 *              ln(L + delta) over the image, so y = 1/2 at the log-mean.
 *  DC_HISTEQ : LDR: y = (number of pixels with gray code <= q) / N, q = the 8-bit
 *              gray code floor(255 L + 1/2);
 *              HDR: u = (ln(L+delta) - lmin) / (lmax - lmin) (1/2 when lmax = lmin),
 *              256 bins over u, y = piecewise-linear cumulative histogram at u.
 *              The HDR u uses ln(L + delta) in 2^-24 fixed point (exact integer
 *              min, max and bin arithmetic, absolute error about 1e-7).
 * Defaults: gain_k = 1, delta = 1e-4.  gain_k >= 0; delta finite and at least
 * FLT_MIN (a normal binary32 number). */
typedef struct {
    int32_t mode;
    float gain_k;
    float delta;
    int32_t reserved; /* must be 0 */
} dc_global_params;

/* Local operator: smoothed local-histogram equalisation (Sec. III-B-2; the paper
 * cites Kass and Solomon's smoothed local histogram filters and gives no formula).
 * u = L (LDR) or the normalised log luminance as in DC_HISTEQ (HDR).  Each pixel
 * adds tent weights to the two nearest of `bins` bin centres (j + 1/2)/bins;
 * histograms are summed over block_s x block_s blocks and then over a
 * (2 radius_blocks + 1)^2 window of blocks, truncated at the image border; each
 * block's tone curve is its window's cumulative histogram with every bin's mass
 * spread uniformly over the bin; a pixel's value is the bilinear blend of the four
 * nearest block curves (nominal block centres, clamped at the border) evaluated at
 * its own u, then y = alpha * F + (1 - alpha) * u.
 * HDR u is computed from ln(L + delta) in 2^-24 fixed point as in DC_HISTEQ.
 * Defaults: block_s = 32, radius_blocks = 2, bins = 32, alpha = 1, delta = 1e-4.
 * Limits: 1 <= block_s <= 64, 0 <= radius_blocks <= 16, 2 <= bins <= DC_MAX_BINS,
 * alpha in [0, 1], delta finite and at least FLT_MIN. */
typedef struct {
    int32_t block_s;
    int32_t radius_blocks;
    int32_t bins;
    float alpha;
    float delta;
    int32_t reserved; /* must be 0 */
} dc_local_params;

/* Per-image statistics of the global pass (device memory, written by the call). */
typedef struct {
    float mu;             /* mean of ln(L + delta) */
    float logmin;         /* min of ln(L + delta) */
    float logmax;         /* max of ln(L + delta) */
    float reserved0;
    int64_t logsum_fixed; /* exact sum over pixels of ln(L + delta) in units of 2^-24:
                             DC_SIGMOID and 8-bit input round each 8-pixel (u8, f16) or
                             4-pixel (f32) group's sum once; HDR DC_HISTEQ sums every
                             pixel's fixed-point logarithm */
    int64_t npix;         /* width * height */
    uint32_t hist[256];   /* LDR: 8-bit gray-code histogram (always filled);
                             HDR: the DC_HISTEQ u-bin histogram (zeros in DC_SIGMOID) */
} dc_global_stats;

/* Kernel launch shape used for one (operation, input sample type): threads per CTA
 * (256), tile rows and columns (columns a multiple of 16, or 0 - the default - to
 * size tiles per call so that they split evenly over the CTAs; the local operator's
 * tile is block_s rows high and its columns a multiple of lcm(block_s, 16), with 0
 * picking the width whose tiles balance best over the resident CTAs) and resident
 * CTAs per SM (0 = as many as fit).  None of these change results: every reduction
 * in the library is exact integer arithmetic. */
typedef struct {
    int32_t threads;
    int32_t tile_rows;
    int32_t tile_cols;
    int32_t ctas_per_sm;
} dc_tuning;

/* Eq. 1-6 (Sec. II-B): out = L per pixel.  ws: see dc_workspace_bytes. */
DC_API int dc_decolorize(const dc_image_in* in, const dc_image_out* out, int32_t n,
                         const dc_decolor_params* params, void* ws, size_t ws_bytes, void* stream);

/* Eq. 1-6 then the global curve of Sec. III-B-1 (dc_global_params).  `stats` is
 * NULL or a device array of n dc_global_stats, written in input order. */
DC_API int dc_decolorize_tonemap_global(const dc_image_in* in, const dc_image_out* out, int32_t n,
                                        const dc_decolor_params* params,
                                        const dc_global_params* gparams, dc_global_stats* stats,
                                        void* ws, size_t ws_bytes, void* stream);

/* Eq. 1-6 then the local operator of Sec. III-B-2 (dc_local_params). */
DC_API int dc_decolorize_tonemap_local(const dc_image_in* in, const dc_image_out* out, int32_t n,
                                       const dc_decolor_params* params,
                                       const dc_local_params* lparams, void* ws, size_t ws_bytes,
                                       void* stream);

/* Frame sequences (the real-time use the paper motivates in Sec. I and
 * Sec. III-B-2; it names no temporal scheme).  Per video stream a device record
 * carries m, an estimate of the log-mean of ln(L + delta); a frame is tone-mapped
 * with the centred sigmoid of Sec. III-B-1 around the carried m instead of its own
 * log-mean, so one pass over the frame suffices, and the pass also sums the
 * frame's own log-mean mu_t, after which m <- (1 - lambda) m + lambda mu_t.
 * `state` is a device array of n records (one per image of the batch, each image
 * the next frame of its own stream), caller-owned and written by the call.
 * restart = 1 starts the streams afresh: each frame is centred on its own log-mean
 * (two passes, the global call's result) and m = mu.  Records must be restarted
 * before their first use.  lambda in (0, 1].
 * DC_HISTEQ: a frame of a running sequence is mapped through the previous frame's
 * cumulative histogram (8-bit: of gray codes; HDR: of u in the previous frame's log
 * range, its coordinate clamped to that range) and its own histogram, binned the same
 * way, and its own log range go to the next frame (lambda unused); again one pass.
 * The outputs of a restarted frame equal dc_decolorize_tonemap_global's.  Outputs
 * may be gray or colour (channels 3). */
typedef struct {
    float m;           /* carried log-mean estimate (DC_SIGMOID) */
    float mu_last;     /* log-mean of the last frame (DC_SIGMOID) */
    int64_t frames;    /* frames seen since the restart */
    int32_t vmin, vmax; /* DC_HISTEQ, HDR input: the last frame's range of round(ln(L + delta) 2^24) */
    int64_t npix;      /* DC_HISTEQ: pixels of the last frame */
    uint32_t hist[256]; /* DC_HISTEQ: the last frame's histogram */
} dc_video_state;

DC_API int dc_decolorize_tonemap_video(const dc_image_in* in, const dc_image_out* out, int32_t n,
                                       const dc_decolor_params* params, const dc_global_params* gparams,
                                       float lambda, int32_t restart, dc_video_state* state, void* ws,
                                       size_t ws_bytes, void* stream);

/* Local tone mapping of frame sequences (the real-time use of Sec. III-B-2 and
 * Fig. SLHE_TMO(a); the paper names no temporal scheme).  A frame of a running
 * sequence is mapped through the block tables of the previous frame of its stream
 * (Sec. III-B-2's operator, dc_local_params) and, for HDR input, takes its
 * coordinates in the previous frame's log range (clamped): so the frame is read once,
 * in one pass that also bins it into its own block histograms, and a second, small
 * pass builds the tables (and records the range) the next frame is mapped through.
 * A restarted frame (restart = 1, required for a record's first use) is the local
 * operator on its own (dc_decolorize_tonemap_local's result) and starts the record.
 * `state` is a caller-owned device buffer of dc_video_local_state_bytes() bytes
 * (256-byte aligned) holding one record per image of the batch in input order (a
 * 256-byte header and the image's tables); keep it, the images' sizes and lparams
 * unchanged between the frames of a sequence.  ws: as for DC_OP_LOCAL.  Outputs may be
 * gray or colour (channels 3: the colour reconstruction of each frame).  Errors: DC_ERR_INVALID_ARG for a NULL, misaligned or
 * too small state buffer, restart not 0 or 1, or the local call's argument errors. */
DC_API size_t dc_video_local_state_bytes(const dc_image_in* in, int32_t n, const dc_local_params* lparams);
DC_API int dc_decolorize_tonemap_local_video(const dc_image_in* in, const dc_image_out* out, int32_t n,
                                             const dc_decolor_params* params, const dc_local_params* lparams,
                                             int32_t restart, void* state, size_t state_bytes, void* ws,
                                             size_t ws_bytes, void* stream);

/* Parameter presets (host only).  DC_PRESET_PAPER: beta_r = 0.55, beta_k = 0.8
 * (Sec. II-B).  Fig. SLHE_TMO(c) shows the paper's luminance controlling the
 * background and the foreground separately through local tone mapping: TM1,
 * "background boost", and TM2, "background suppression", without their values.
 * Reading: beta_k trades the warm blend L_WARM against the cool blend L_COOL in
 * Eq. 6, so a lower beta_k lifts the cool (typically background) colours and a higher
 * one suppresses them: TM1 = (0.55, 0.55), TM2 = (0.55, 0.95), both within the
 * paper's 0.5 < beta < 1.  Every preset uses DC_LUMA_OURS, color_s = 1 and the
 * default local operator (block_s 32, radius 2, 32 bins, alpha 1, delta 1e-4).
 * `p` or `l` may be NULL.  Returns DC_ERR_INVALID_ARG for an unknown preset. */
#define DC_PRESET_PAPER 0
#define DC_PRESET_TM1 1
#define DC_PRESET_TM2 2
DC_API int dc_preset(int32_t preset, dc_decolor_params* p, dc_local_params* l);

/* Global tone mapping for callers that cannot allocate device memory (no
 * counterpart in the paper; it is a deployment convenience).  Same arguments and
 * results as dc_decolorize_tonemap_global, without a workspace: the scratch is a
 * fixed DC_NOALLOC_SCRATCH_BYTES array in the library's device memory, held by
 * every GPU that loads the library until the process exits.  The call allocates
 * nothing; it returns DC_ERR_WORKSPACE when the batch needs more scratch than
 * that (about 1.1 KiB per image).  The first call on a device looks up the
 * array's address with that device current; make that first call before any
 * stream capture.  Every call reuses the same array, so calls whose executions
 * overlap on the GPU (other streams, other threads) race: order them. */
#define DC_NOALLOC_SCRATCH_BYTES 65536
DC_API int dc_decolorize_tonemap_global_noalloc(const dc_image_in* in, const dc_image_out* out, int32_t n,
                                                const dc_decolor_params* params,
                                                const dc_global_params* gparams, dc_global_stats* stats,
                                                void* stream);

/* Workspace bytes a call of `op` (DC_OP_*) needs for these inputs; op_params is
 * NULL (DC_OP_DECOLORIZE, DC_OP_GLOBAL) or a dc_local_params* (DC_OP_LOCAL).
 * Returns 0 when the arguments are invalid.  The workspace must be 256-byte
 * aligned; its contents need no initialisation (each call resets what it uses).
 * For 8-bit input (global and local tone mapping, gray output) the size includes
 * an f32 luminance plane (4 bytes per pixel) that spares the later passes from
 * recomputing Eq. 1-6; a call given less (down to dc_workspace_min_bytes) runs
 * without it, with identical results. */
DC_API size_t dc_workspace_bytes(int32_t op, const dc_image_in* in, int32_t n,
                                 const void* op_params);

/* The least workspace a call of `op` accepts for these inputs (no optional plane);
 * same arguments and 0 on invalid arguments.  The paper has no counterpart. */
DC_API size_t dc_workspace_min_bytes(int32_t op, const dc_image_in* in, int32_t n,
                                     const void* op_params);

/* Registers a workspace kept for calls of this library only: zeroes its ws_bytes
 * (on `stream`, then synchronises it, once) and remembers the address.  Calls on a
 * registered workspace clear their control block at the end of their last pass, so
 * a call whose control block is no larger than the previous call's needs no
 * clearing memset before its first pass (one stream operation fewer per call).
 * Until dc_workspace_release the caller must neither write to that memory nor free
 * it, and only one call at a time may use it.  Returns DC_ERR_WORKSPACE for a NULL
 * or misaligned pointer or fewer than 256 bytes.  The paper has no counterpart. */
DC_API int dc_workspace_prepare(void* ws, size_t ws_bytes, void* stream);

/* Forgets a registered workspace (before its memory is freed or reused). */
DC_API int dc_workspace_release(void* ws);

/* Synchronises `stream`, then reads the device-side error word of workspace `ws`
 * (reserved for device-detected errors; the current kernels never wait on each
 * other and report DC_OK).  Returns DC_ERR_CUDA if the copy fails. */
DC_API int dc_query_status(const void* ws, void* stream);

/* Static English description of a status code. */
DC_API const char* dc_status_string(int status);

/* Launch-shape table used by later calls (per operation and input sample type);
 * used by the autotuner.  Returns DC_ERR_INVALID_ARG for values out of range. */
DC_API int dc_set_tuning(int32_t op, int32_t in_dtype, const dc_tuning* t);
DC_API int dc_get_tuning(int32_t op, int32_t in_dtype, dc_tuning* t);

/* Profiling switch for later calls (default 0).  When on, each launch records per
 * image and phase the earliest tile start and latest tile end (globaltimer ns) and,
 * summed over CTAs, the time spent waiting for earlier phases, for free stages, for
 * tiles and for stage data.  Adds a few atomics per tile. */
DC_API int dc_debug_profile(int32_t on);

/* Synchronises `stream` and copies the profile of the last launch that used `ws`
 * into out[]: 8 launch counters (dependency wait, stage wait, tile wait, data wait,
 * tiles, kernel start, kernel end, reserved) followed, for each of the first n_img
 * images of that launch, by 4 phase start and 4 phase end timestamps. */
DC_API int dc_debug_read_profile(const void* ws, int32_t n_img, uint64_t* out, void* stream);

/* Local tile width (pixels along a block row) that a dc_decolorize_tonemap_local
 * call on n images of heights[k] x widths[k] with this block_s would use on a GPU
 * with n_sm SMs, given the current tuning for in_dtype (0 width = automatic, see
 * dc_tuning).  The tiling of Sec. III-B-2's block grid into launch tiles changes no
 * result; the paper has no counterpart.  Host only, thread-safe; *cols receives the
 * width.  Errors: DC_ERR_INVALID_ARG for null pointers, n outside 1..DC_MAX_BATCH,
 * block_s outside 1..64, n_sm < 1, a non-positive size or an unknown in_dtype. */
DC_API int dc_local_tile_cols(int32_t block_s, const int32_t* heights, const int32_t* widths, int32_t n,
                              int32_t in_dtype, int32_t n_sm, int32_t* cols);

/* Number of kernels the last successful call on this thread enqueued. */
DC_API int dc_last_launch_count(void);

/* Test hook for the error paths (host side; the paper has no counterpart): for
 * k > 0 the k-th kernel launch of every later call (counted from 1 within the
 * call) is not issued and the call returns DC_ERR_CUDA after enqueueing the passes
 * before it; k = 0 turns it off.  The library starts with the value of the
 * environment variable DC_FAIL_LAUNCH, else 0.  Returns DC_ERR_INVALID_ARG for
 * k < 0.  No GPU fault is involved: the kernel is simply not launched. */
DC_API int dc_debug_fail_launch(int32_t k);

/* Bounds-checked build (compiled with -DDC_BOUNDS_CHECK): *checked = 1 and *flags =
 * the OR of the buffers some kernel tried to access outside (1 input, 2 output,
 * 4 plane, 8 workspace) since the last read, which clears them; such accesses were
 * skipped.  Other builds: *checked = 0, *flags = 0.  Synchronous (reads device
 * memory).  The paper has no counterpart. */
DC_API int dc_debug_bounds(uint32_t* flags, int32_t* checked);

/* ABI version (major * 100 + minor): 200 since the channel choice, colour outputs,
 * frame sequences and presets. */
DC_API int dc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DECOLOR_H */
