// Internal structures shared by the host side (dc_abi.cu) and the engine kernels.
//
// A call runs each image through a short chain of passes ("phases": statistics,
// histograms, tone curve ...).  Every pass is one persistent kernel launch over
// the tiles of that pass for all images of the batch; passes follow each other
// on the caller's stream, so a pass sees everything the previous one wrote and no
// kernel ever waits for another CTA.
#pragma once

#include <stdint.h>

#include "../../include/decolor.h"

namespace dc {

constexpr int kMaxPhases = 4;
constexpr int kCapSmall = 1;     // params capacity for single-image calls
constexpr int kCapMid = 16;
constexpr int kCapLarge = 256;   // largest batch per launch (kernel parameter space)
constexpr int kLogFixedShift = 24;  // logsum and fixed-point log unit is 2^-24

// Resident CTAs per SM the pass kernels are compiled for (launch bounds); the host
// sizes its automatic tiles for that many CTAs per SM.
#ifndef DC_MIN_CTAS
#define DC_MIN_CTAS 4
#endif

// phase kinds
enum PhaseKind : int32_t {
    PK_DECOLOR = 0,   // L -> out
    PK_STATS = 1,     // log statistics (+ 8-bit gray histogram) (+ L plane)
    PK_LOGHIST = 2,   // HDR histogram of u (DC_HISTEQ)
    PK_APPLY_G = 3,   // global curve -> out
    PK_BLOCKH = 4,    // local: block histograms
    PK_CDF = 5,       // local: window sums -> per-block cumulative tables
    PK_APPLY_L = 6,   // local: bilinear blend of block curves -> out
    PK_STATS_LOG = 7, // HDR histogram forms: exact fixed-point log statistics (+ plane)
    PK_VIDEO = 8,     // frame sequences: sigmoid around the carried log-mean + this frame's log-sum
    PK_VIDEO_L = 9,   // local frame sequences: block histograms of the frame and its mapping
                      // through the previous frame's tables, in one pass
    PK_VIDEO_H = 10,  // histogram-equalisation frame sequences: the previous frame's cumulative
                      // histogram + this frame's histogram, in one pass
};

// Per-image record of a local frame sequence (caller-owned state buffer): this header,
// then the block tables (f32, Hb x Wb x (bins + 1)) the next frame is mapped through.
struct DcVideoLocalHead {
    int32_t vmin, vmax;   // the last frame's range of round(ln(L + delta) 2^24) (HDR input)
    int64_t frames;       // frames since the restart
    uint32_t pad[60];
};
static_assert(sizeof(DcVideoLocalHead) == 256, "state header is 256 bytes");

// per-image flags
enum : uint32_t {
    IF_VEC = 1u,      // 16-byte aligned pointers and strides: vector path
    IF_LPLANE = 2u,   // the image keeps an f32 plane (`plane`) that holds L between phases
    IF_PLANE_LOG = 4u,  // ... and it holds round(ln(L + delta) 2^24) as int32 bits instead of L
    IF_COLOR = 8u,    // interleaved RGB output (colour reconstruction), 3 samples per pixel
    IF_UPRECISE = 16u,  // 8-bit input, local operator: the bin coordinate comes from the float-float
                        // luminance (f32 outputs); a plane, if kept, holds that coordinate as int32 bits
};

struct DcImage {                 // 104 bytes
    const uint8_t* in;
    uint8_t* out;
    int64_t in_stride;           // bytes between (logical) rows
    int64_t out_stride;
    uint8_t* plane;              // f32 plane kept between passes (the output, or workspace for 8-bit input)
    int64_t plane_stride;
    int32_t rows, cols;          // logical geometry of pixelwise phases
    int32_t prow, pcol;          // physical geometry (local operator)
    int32_t out_dt;
    uint32_t flags;
    int32_t tiles_x;             // tiles per tile row, pixelwise phases
    int32_t tiles_x_loc;         // tiles per block row, local phases
    int32_t Hb, Wb;              // local: blocks
    int64_t ws_hist;             // byte offsets into the workspace (local)
    uint8_t* lvs;                // local frame sequences: the image's state record, or NULL
};

// Per-image control block, cleared (memset) before the first pass of a call.  The
// statistics pass accumulates into it with integer atomics; a later pass, which
// starts only after the previous one has completed, derives what it needs (mu,
// lmin, lmax) from the integer accumulators itself, so no tile has to finalise a
// pass.  done[] is not used by the pass kernels.
struct DcImgCtrl {
    uint32_t done[kMaxPhases];
    unsigned long long logsum;   // two's complement, units of 2^-24
    uint32_t lmax_ord;           // ordered encoding of max ln(L+delta): of the float
                                 // (PK_STATS) or of the 2^-24 fixed-point value (PK_STATS_LOG)
    uint32_t lmin_nord;          // bitwise NOT of the ordered encoding of the min
    uint32_t pad[2];
    // profiling (only when enabled): per phase, NOT of the earliest tile start and
    // the latest tile end, in globaltimer nanoseconds
    unsigned long long t_start_not[kMaxPhases];
    unsigned long long t_end[kMaxPhases];
    uint32_t hist[256];
};

// Profile counters of one call (only when enabled), ns.  The pass kernels fill
// PROF_TILES, PROF_KSTART_NOT and PROF_KEND; the wait slots stay zero (no pass
// kernel waits on another CTA) and are kept for the layout of the read-back.
enum ProfSlot {
    PROF_DEP_WAIT = 0,
    PROF_EMPTY_WAIT = 1,
    PROF_TILE_WAIT = 2,
    PROF_DATA_WAIT = 3,
    PROF_TILES = 4,       // tiles processed
    PROF_KSTART_NOT = 5,  // NOT of the earliest CTA start
    PROF_KEND = 6,        // latest CTA end
    PROF_SLOTS = 8
};

// Per-launch control block, cleared by the host before the launch.
struct DcCtrl {
    uint32_t done_ctas;          // CTAs of the last pass that finished (self-clearing calls)
    uint32_t pad[15];
    unsigned long long prof[PROF_SLOTS];
    uint32_t pad2[32];
    // followed by DcImgCtrl[n]
};

// Call-level header at the start of the workspace: the device-side error word.
struct DcWsHeader {
    uint32_t error;
    uint32_t pad[63];
};

template <int CAP>
struct DcBatch {
    int32_t n_img, n_phase;
    int32_t phase_kind[kMaxPhases];
    int32_t tile_rows, tile_cols;      // pixelwise phases
    int32_t loc_tile_cols;             // local phases (tile height = block_s)
    int32_t cdf_cols;                  // block columns per window-CDF tile (<= kCdfMaxChunk)
    float beta_r, beta_k;
    int32_t ldr;                       // 8-bit input
    int32_t mode;                      // DC_SIGMOID / DC_HISTEQ
    float gain_k, delta;
    int32_t gain_is_one;
    int32_t need_gray_hist;            // LDR: gray histogram wanted (HISTEQ or stats)
    int32_t need_logsum;               // statistics pass: the log-sum is used (sigmoid, or a stats record)
    int32_t need_minmax;               // statistics pass: min/max of the log are used (histogram
                                       // coordinates of the HDR forms, or a stats record)
    int32_t luma;                      // DC_LUMA_*
    float color_s;                     // saturation exponent of colour outputs
    int32_t color_s_one;               // color_s == 1
    float lambda;                      // frame sequences: smoothing of the carried log-mean
    dc_video_state* vstate;            // frame sequences: per image (input order), or NULL
    int32_t block_s, radius, bins;
    uint32_t s_magic;                  // ceil(2^32 / block_s), 0 for block_s = 1: exact division of offsets < 2^16
    float alpha;
    uint32_t profile;                  // record phase timestamps
    int32_t reset_bytes;               // > 0: the last pass's last CTA clears this many bytes of the
                                       // control block (from ctrl), leaving it zero for the next call
    DcCtrl* ctrl;
    uint32_t* err;                     // call-level error word (workspace header)
    dc_global_stats* stats;            // nullable; indexed by img_stats_index
    uint8_t* ws;
    int64_t ws_bytes;                  // workspace size (bounds-checked build)
    uint8_t* lvs_buf;                  // local frame sequences: the caller's state buffer
    int64_t lvs_bytes;                 // ... and its size (bounds-checked build)
    int32_t stats_index[CAP];
    DcImage img[CAP];
    int32_t reverse[kMaxPhases];         // hand a pass's tiles out last-first (L2 reuse)
    int32_t seg_start[kMaxPhases][CAP + 1];  // first tile of each image, per pass
};

#ifdef __CUDACC__
__host__ __device__
#endif
inline int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// launcher entry points (one per input sample type), defined in dc_engine_*.cu
struct LaunchShape {
    int threads;
    int grid;
};

// opk: 0 decolorize, 1 global, 2 local; kind: PhaseKind; ph: index of the pass;
// pl: 1 = the pass reads the plane every image of the launch keeps (histogram and apply
// passes) or keeps only the reduction the call uses (statistics passes); 2 = colour output
// (apply passes)
int launch_engine_u8(const void* batch, int cap, int opk, int kind, int ph, int pl, LaunchShape ls, void* stream);
int launch_engine_f16(const void* batch, int cap, int opk, int kind, int ph, int pl, LaunchShape ls, void* stream);
int launch_engine_f32(const void* batch, int cap, int opk, int kind, int ph, int pl, LaunchShape ls, void* stream);
int occupancy_u8(int cap, int opk, int kind, int pl);
int occupancy_f16(int cap, int opk, int kind, int pl);
int occupancy_f32(int cap, int opk, int kind, int pl);
int bounds_u8(uint32_t* flags);   // bounds-check flags per translation unit (-1: not built with checks)
int bounds_f16(uint32_t* flags);
int bounds_f32(uint32_t* flags);

// Smallest workspace a call accepts (without the optional 8-bit plane); 0 on error.
size_t workspace_min_bytes(int32_t op, const dc_image_in* in, int32_t n, const void* op_params);

}  // namespace dc
