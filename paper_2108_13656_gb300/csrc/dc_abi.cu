// Host side of the C ABI declared in include/decolor.h: argument validation,
// workspace layout, the tile schedule (segment table) and the launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "dc_internal.h"

using namespace dc;

namespace {

constexpr int kOpkDecolor = 0, kOpkGlobal = 1, kOpkLocal = 2;
constexpr int64_t kHeaderBytes = 256;
constexpr int64_t kMaxPixels = int64_t(1) << 28;
constexpr int kMaxLocalSide = 1 << 16;
constexpr int kLocMaxBlocksX = 32;
constexpr int kLocMaxCols = 1024;
constexpr int kCdfMaxChunk = 64;  // block columns of a window-CDF tile, at most (shared-memory staging)

std::mutex g_mu;
// tile_cols 0: sized per launch so the pass's tiles split evenly over the CTAs
dc_tuning g_tune[3][3] = {
    {{256, 1, 0, 0}, {256, 1, 0, 0}, {256, 1, 0, 0}},
    {{256, 1, 0, 0}, {256, 1, 0, 0}, {256, 1, 0, 0}},
    {{256, 32, 0, 0}, {256, 32, 0, 0}, {256, 32, 0, 0}},
};
constexpr int kAutoCtasPerSm = DC_MIN_CTAS;  // resident CTAs of a pass kernel (launch bounds)

// Workspaces registered with dc_workspace_prepare.  A call's control block (header
// and per-launch / per-image records at the start of the workspace) must be zero
// when its first pass starts.  For each registered workspace the host tracks how
// many leading bytes are zero between calls: a call whose control block lies inside
// that prefix needs no clearing memset, and its last pass clears the block again.
// The bytes after a call's control block (histograms, curves, planes) are left
// dirty, so afterwards the clean prefix ends with the block; a profiled call leaves
// its counters for reading (prefix 0 until a later call clears it).
struct CleanWs {
    size_t bytes;  // registered size
    size_t clean;  // leading bytes known to be zero between calls
};
std::unordered_map<uintptr_t, CleanWs> g_clean;  // guarded by g_mu

// For a call whose control block ends at `need` bytes: whether it can skip the
// clearing memset and whether its last pass must clear the block (registered
// workspace).  Nothing is recorded yet: the block is dirty as soon as a pass runs,
// and clean again only once the last pass has been enqueued (finish_clear).
void plan_clear(const void* ws, size_t need, bool profiling, bool* skip_memset, bool* clear_at_end)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_clean.find(reinterpret_cast<uintptr_t>(ws));
    if (it == g_clean.end() || it->second.bytes < need) {
        *skip_memset = false;
        *clear_at_end = false;
        if (it != g_clean.end()) it->second.clean = 0;
        return;
    }
    *skip_memset = !profiling && it->second.clean >= need;
    *clear_at_end = !profiling;
    it->second.clean = 0;  // until every pass of the call is enqueued
}

// After the launches of a call's group: with every pass enqueued, the last one
// leaves the control block zero (`clear_at_end`); after a failed memset or launch
// the block holds partial counters, so the next call on the workspace clears it
// with a memset.
void finish_clear(const void* ws, size_t need, bool ok, bool clear_at_end)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_clean.find(reinterpret_cast<uintptr_t>(ws));
    if (it == g_clean.end()) return;
    it->second.clean = (ok && clear_at_end) ? need : 0;
}

// Launch failure injection for tests of the error paths (host side only): when
// k > 0, the k-th kernel launch of every later call returns DC_ERR_CUDA without
// being issued.  Set by dc_debug_fail_launch or, at load, by DC_FAIL_LAUNCH.
std::atomic<int> g_fail_launch{0};
struct FailLaunchInit {
    FailLaunchInit()
    {
        const char* e = std::getenv("DC_FAIL_LAUNCH");
        if (e) g_fail_launch.store(std::atoi(e));
    }
} g_fail_launch_init;
int g_profile = 0;
thread_local int g_last_launches = 0;
thread_local int g_call_launches = 0;

int esz(int dt) { return dt == DC_U8 ? 1 : (dt == DC_F16 ? 2 : 4); }
bool dt_ok(int dt) { return dt == DC_U8 || dt == DC_F16 || dt == DC_F32; }
bool finite_in(float v, float lo, float hi) { return std::isfinite(v) && v >= lo && v <= hi; }
bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

struct OpArgs {
    int opk;
    const dc_global_params* g;
    const dc_local_params* l;
    dc_global_stats* stats;
    dc_video_state* vstate = nullptr;  // frame sequences (global sigmoid only)
    bool restart = false;              // frame sequences: centre each frame on its own log-mean
    float lambda = 1.0f;
    uint8_t* lvs = nullptr;            // local frame sequences: the state buffer
    int64_t lvs_bytes = 0;
    const std::vector<int64_t>* lvs_off = nullptr;  // per input image: offset of its record
    bool video() const { return vstate != nullptr || lvs != nullptr; }
};

// Bytes of an image's local frame-sequence record: a 256-byte header and its block
// tables (f32, Hb x Wb x (bins + 1)), 256-byte aligned.
int64_t lvs_record_bytes(const dc_image_in& in, const dc_local_params& l)
{
    const int64_t Hb = (in.height + l.block_s - 1) / l.block_s, Wb = (in.width + l.block_s - 1) / l.block_s;
    return 256 + align_up(Hb * Wb * (l.bins + 1) * 4, 256);
}

int out_channels(const dc_image_out& o) { return o.channels == 3 ? 3 : 1; }

int validate_image(const dc_image_in& in, const dc_image_out* out, bool local, bool tonemap)
{
    if (!dt_ok(in.dtype)) return DC_ERR_UNSUPPORTED_DTYPE;
    if (in.reserved != 0 || in.width < 1 || in.height < 1) return DC_ERR_INVALID_ARG;
    if ((int64_t)in.width * in.height > kMaxPixels) return DC_ERR_INVALID_ARG;
    if (local && (in.width > kMaxLocalSide || in.height > kMaxLocalSide)) return DC_ERR_INVALID_ARG;
    const int ie = esz(in.dtype);
    if (in.data == nullptr || in.stride_bytes < (int64_t)3 * in.width * ie) return DC_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(in.data) % ie) != 0 || (in.stride_bytes % ie) != 0) return DC_ERR_INVALID_ARG;
    if (out) {
        if (!dt_ok(out->dtype)) return DC_ERR_UNSUPPORTED_DTYPE;
        if (out->data == nullptr || (out->channels != 0 && out->channels != 1 && out->channels != 3))
            return DC_ERR_INVALID_ARG;
        if (out->channels == 3 && !tonemap) return DC_ERR_INVALID_ARG;  // colour needs a tone-mapped y
        const int oe = esz(out->dtype) * out_channels(*out);
        if (out->stride_bytes < (int64_t)in.width * oe) return DC_ERR_INVALID_ARG;
        if ((reinterpret_cast<uintptr_t>(out->data) % esz(out->dtype)) != 0 || (out->stride_bytes % esz(out->dtype)) != 0)
            return DC_ERR_INVALID_ARG;
    }
    return DC_OK;
}

int validate_params(const dc_decolor_params* p, const OpArgs& op)
{
    if (!p || !finite_in(p->beta_r, 0.f, 1.f) || !finite_in(p->beta_k, 0.f, 1.f)) return DC_ERR_INVALID_ARG;
    if (p->luma < DC_LUMA_OURS || p->luma > DC_LUMA_LSTAR || !finite_in(p->color_s, 0.f, 8.f)) return DC_ERR_INVALID_ARG;
    if (op.vstate) {
        if (op.opk != kOpkGlobal || !finite_in(op.lambda, 0.f, 1.f) || !(op.lambda > 0.f)) return DC_ERR_INVALID_ARG;
    }
    if (op.lvs && op.opk != kOpkLocal) return DC_ERR_INVALID_ARG;
    if (op.opk == kOpkGlobal) {
        const dc_global_params* g = op.g;
        if (!g || (g->mode != DC_SIGMOID && g->mode != DC_HISTEQ) || g->reserved != 0) return DC_ERR_INVALID_ARG;
        if (!finite_in(g->gain_k, 0.f, 1e6f) || !std::isfinite(g->delta) || !(g->delta >= FLT_MIN)) return DC_ERR_INVALID_ARG;
    } else if (op.opk == kOpkLocal) {
        const dc_local_params* l = op.l;
        if (!l || l->reserved != 0) return DC_ERR_INVALID_ARG;
        if (l->block_s < 1 || l->block_s > 64 || l->radius_blocks < 0 || l->radius_blocks > 16) return DC_ERR_INVALID_ARG;
        if (l->bins < 2 || l->bins > DC_MAX_BINS || !finite_in(l->alpha, 0.f, 1.f)) return DC_ERR_INVALID_ARG;
        if (!std::isfinite(l->delta) || !(l->delta >= FLT_MIN)) return DC_ERR_INVALID_ARG;
    }
    return DC_OK;
}

int gcd_i(int a, int b) { return b == 0 ? a : gcd_i(b, a % b); }

// Local tile width: a multiple of lcm(block_s, 16) (at most 1024 for block_s <= 64),
// at most kLocMaxBlocksX blocks and 1024 pixels.
int local_tile_cols(int s, int want)
{
    const int l = s / gcd_i(s, 16) * 16;
    int m = std::max(1, want / l);
    while (m > 1 && ((l * m) / s > kLocMaxBlocksX || l * m > kLocMaxCols)) --m;
    return l * m;
}

// Block columns per window-CDF tile.  The pass is latency-bound: a tile waits for
// its L2 loads (the block histograms of 2R + 1 block rows) before its scans, and a
// CTA's tiles follow one another.  So the narrowest chunk whose tiles all fit the
// persistent grid at once wins (more tiles, shorter ones); when even the widest
// needs several rounds, the widest (the fewest rounds).
int cdf_cols_auto(const std::vector<std::pair<int, int>>& hbwb, int64_t slots)
{
    static const int cand[] = {16, 24, 32, 48, kCdfMaxChunk};
    for (int c : cand) {
        int64_t T = 0;
        for (const auto& d : hbwb) T += (int64_t)d.first * ((d.second + c - 1) / c);
        if (T <= slots) return c;
    }
    return kCdfMaxChunk;
}

// Local tile width when none is tuned: among the widths above, the one whose tiles
// spread most evenly over the persistent grid.  Model: CTA c takes tiles c,
// c + grid, ... and a tile costs its pixels plus 3/4 of a block for the curve
// staging and prologue; the widest width whose maximum CTA cost is within 6% of
// the smallest wins (narrow tiles stage more curves per pixel than the model
// counts).  (A CTA's time follows its own work: one left with a second tile runs
// mostly alone at the end.)  A single image is modelled tile by tile (cached per
// size); a batch, whose size mix rarely repeats, by its tile count alone (rounds of
// the grid times a full tile's cost), so that choosing stays a few microseconds.
// Batches whose 512-pixel tiling already gives many rounds keep 512 pixels.
int local_tile_cols_auto(int s, const std::vector<std::pair<int, int>>& hw, int nsm, int cps)
{
    const int l = s / gcd_i(s, 16) * 16;
    const int dflt = local_tile_cols(s, 512);
    nsm = std::max(1, nsm);
    const int64_t slots = (int64_t)nsm * std::max(1, cps);
    int64_t t_dflt = 0;
    for (const auto& d : hw) t_dflt += (int64_t)((d.first + s - 1) / s) * ((d.second + dflt - 1) / dflt);
    if (t_dflt > 4 * slots || hw.size() > 64) return dflt;
    const bool single = hw.size() == 1;
    uint64_t key = 0;
    static std::mutex mu;
    static std::unordered_map<uint64_t, int> cache;
    if (single) {
        key = ((uint64_t)(uint32_t)hw[0].first << 32 | (uint32_t)hw[0].second) * 1099511628211ull ^
              ((uint64_t)s << 48 | (uint64_t)(uint32_t)nsm << 8 | (uint64_t)(cps & 0xFF));
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    const int64_t ovh = std::max<int64_t>(256, (int64_t)s * s * 3 / 4);
    struct Cand {
        int w;
        int64_t mc;
    };
    std::vector<Cand> cands;
    std::vector<int64_t> cta;
    for (int m = 1;; ++m) {
        const int w = l * m;
        if (m > 1 && (w / s > kLocMaxBlocksX || w > kLocMaxCols)) break;
        int64_t T = 0;
        for (const auto& d : hw) T += (int64_t)((d.first + s - 1) / s) * ((d.second + w - 1) / w);
        const int64_t grid = std::min(T, slots);
        if (!single) {
            cands.push_back({w, (T + grid - 1) / grid * ((int64_t)s * w + ovh)});
        } else {
            cta.assign((size_t)grid, 0);
            const int H = hw[0].first, W = hw[0].second, tx = (W + w - 1) / w;
            int64_t t = 0;
            for (int r0 = 0; r0 < H; r0 += s)
                for (int c = 0; c < tx; ++c, ++t)
                    cta[(size_t)(t % grid)] += (int64_t)std::min(s, H - r0) * std::min(w, W - c * w) + ovh;
            cands.push_back({w, *std::max_element(cta.begin(), cta.end())});
        }
        if (w / s > kLocMaxBlocksX || w > kLocMaxCols) break;
    }
    int64_t min_mc = INT64_MAX;
    for (const Cand& c : cands) min_mc = std::min(min_mc, c.mc);
    int best = dflt;
    for (const Cand& c : cands)  // narrow to wide: the widest within the margin wins
        if (c.mc * 100 <= min_mc * 106) best = c.w;
    if (single) {
        std::lock_guard<std::mutex> lk(mu);
        if (cache.size() > 1024) cache.clear();
        cache[key] = best;
    }
    return best;
}

struct Geometry {
    DcImage im;
    int tiles[kMaxPhases];
    int64_t local_bytes;
    int64_t plane_bytes;  // workspace plane (8-bit input)
};

struct LaunchPlan {
    int in_dt;
    bool plane;            // every image keeps an f32 plane between passes
    bool color;            // every image has a colour (3-channel) output
    std::vector<int> idx;  // positions in the caller's arrays
};

// An image keeps its luminance (or its fixed-point log) in its f32 output between
// passes: HDR input, a tone-mapping operation, a gray f32 output.
bool keeps_plane(const OpArgs& op, int in_dt, const dc_image_out& o)
{
    return op.opk != kOpkDecolor && in_dt != DC_U8 && o.dtype == DC_F32 && out_channels(o) == 1;
}

// 8-bit input through the local operator with an f32 output (gray or colour): the bin
// coordinate comes from the float-float luminance (binary32 L is too coarse for the
// curve's slope at f32 precision).
bool precise_coord(const OpArgs& op, int in_dt, const dc_image_out& o)
{
    return op.opk == kOpkLocal && in_dt == DC_U8 && o.dtype == DC_F32;
}

// Passes that read the plane instead of recomputing L from RGB (an 8-bit local
// call writes its plane in the block-histogram pass, the first one).
bool reads_plane(int kind, int in_dt)
{
    return kind == PK_LOGHIST || kind == PK_APPLY_G || kind == PK_APPLY_L || (kind == PK_BLOCKH && in_dt != DC_U8);
}

// Phase chain of an operation for one input class.
int phase_list(const OpArgs& op, bool ldr, int32_t* kinds)
{
    if (op.opk == kOpkDecolor) {
        kinds[0] = PK_DECOLOR;
        return 1;
    }
    if (op.opk == kOpkGlobal) {
        if (op.vstate && !op.restart) {  // a frame of a running sequence: one pass
            kinds[0] = op.g->mode == DC_HISTEQ ? PK_VIDEO_H : PK_VIDEO;
            return 1;
        }
        kinds[0] = PK_STATS;
        if (op.g->mode == DC_HISTEQ && !ldr) {
            kinds[0] = PK_STATS_LOG;  // the histogram of u needs the exact log coordinate
            kinds[1] = PK_LOGHIST;
            kinds[2] = PK_APPLY_G;
            return 3;
        }
        kinds[1] = PK_APPLY_G;
        return 2;
    }
    int n = 0;
    if (op.lvs && !op.restart) {  // a frame of a running local sequence: fused pass, then its tables
        kinds[0] = PK_VIDEO_L;
        kinds[1] = PK_CDF;
        return 2;
    }
    if (!ldr) kinds[n++] = PK_STATS_LOG;
    kinds[n++] = PK_BLOCKH;
    kinds[n++] = PK_CDF;
    kinds[n++] = PK_APPLY_L;
    return n;
}

void make_geometry(const dc_image_in& in, const dc_image_out& out, const OpArgs& op, const dc_tuning& tu,
                   int n_phase, const int32_t* kinds, Geometry& g, int tile_rows, int tile_cols, int loc_cols,
                   int cdf_cols, bool u8_plane)
{
    DcImage& im = g.im;
    std::memset(&im, 0, sizeof(im));
    const int ie = esz(in.dtype), oe = esz(out.dtype);
    const int W = in.width, H = in.height;
    im.in = static_cast<const uint8_t*>(in.data);
    im.out = static_cast<uint8_t*>(out.data);
    im.out_dt = out.dtype;
    im.prow = H;
    im.pcol = W;
    const int och = out_channels(out);
    const bool dense = in.stride_bytes == (int64_t)3 * W * ie && out.stride_bytes == (int64_t)W * oe * och;
    if (op.opk != kOpkLocal && dense) {
        im.rows = 1;
        im.cols = W * H;
        im.in_stride = (int64_t)3 * W * H * ie;
        im.out_stride = (int64_t)W * H * oe * och;
    } else {
        im.rows = H;
        im.cols = W;
        im.in_stride = in.stride_bytes;
        im.out_stride = out.stride_bytes;
    }
    bool vec = al16(in.data) && al16(out.data);
    if (im.rows > 1) vec = vec && (in.stride_bytes % 16 == 0) && (out.stride_bytes % 16 == 0);
    im.flags = vec ? IF_VEC : 0u;
    if (och == 3) im.flags |= IF_COLOR;
    if (precise_coord(op, in.dtype, out)) im.flags |= IF_UPRECISE;
    g.plane_bytes = 0;
    if (keeps_plane(op, in.dtype, out)) {
        im.flags |= IF_LPLANE;
        im.plane = im.out;
        im.plane_stride = im.out_stride;
        // the local operator and HDR histogram equalisation only need ln(L + delta)
        if (op.opk == kOpkLocal || (op.opk == kOpkGlobal && op.g->mode == DC_HISTEQ)) im.flags |= IF_PLANE_LOG;
    } else if (u8_plane) {
        im.flags |= IF_LPLANE;  // `plane` is set by the caller, in the workspace
        im.plane_stride = align_up((int64_t)im.cols * 4, 16);
        g.plane_bytes = align_up(im.plane_stride * im.rows, 256);
    }
    im.tiles_x = (im.cols + tile_cols - 1) / tile_cols;
    const int tiles_y = (im.rows + tile_rows - 1) / tile_rows;
    g.local_bytes = 0;
    if (op.opk == kOpkLocal) {
        const int s = op.l->block_s, B = op.l->bins;
        im.Hb = (H + s - 1) / s;
        im.Wb = (W + s - 1) / s;
        im.tiles_x_loc = (W + loc_cols - 1) / loc_cols;
        const int64_t hist_bytes = align_up((int64_t)im.Hb * im.Wb * B * 8, 256);
        const int64_t cdf_bytes = align_up((int64_t)im.Hb * im.Wb * (B + 1) * 4, 256);
        g.local_bytes = hist_bytes + cdf_bytes;
    }
    (void)tu;
    for (int p = 0; p < n_phase; ++p) {
        if (op.opk == kOpkLocal)
            g.tiles[p] = kinds[p] == PK_CDF ? im.Hb * ((im.Wb + cdf_cols - 1) / cdf_cols) : im.Hb * im.tiles_x_loc;
        else
            g.tiles[p] = tiles_y * im.tiles_x;
    }
}

template <int CAP>
int build_and_launch(const dc_image_in* in, const dc_image_out* out, const std::vector<int>& idx, bool plane,
                     bool color, bool allow_u8_plane, const dc_decolor_params* p, const OpArgs& op, uint8_t* ws,
                     int64_t ws_bytes_total, bool first, int64_t* need, void* stream, bool launch)
{
    const int n = (int)idx.size();
    const int in_dt = in[idx[0]].dtype;
    const bool ldr = in_dt == DC_U8;
    bool u8_plane = false;
    // 8-bit input keeps an f32 luminance plane in the workspace, whatever the launch
    // group's size: the later passes are bound by instruction issue, so reading 4
    // bytes a pixel (from L2, or from DRAM once the plane outgrows L2) beats
    // recomputing Eq. 1-6 from the 3 RGB bytes.  (Not for colour outputs, whose apply
    // pass re-reads RGB anyway, nor for a frame of a running sequence, a single pass.)
    if (allow_u8_plane && ldr && op.opk != kOpkDecolor && !color && !(op.video() && !op.restart)) u8_plane = true;
    plane = plane || u8_plane;
    dc_tuning tu;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        tu = g_tune[op.opk][in_dt];
    }
    DcBatch<CAP>* b = new (std::nothrow) DcBatch<CAP>();
    if (!b) return DC_ERR_INVALID_ARG;
    std::memset(b, 0, sizeof(DcBatch<CAP>));
    b->n_phase = phase_list(op, ldr, b->phase_kind);
    b->tile_rows = std::max(1, tu.tile_rows);
    if (tu.tile_cols > 0) {
        b->tile_cols = std::max(16, (tu.tile_cols + 15) / 16 * 16);
    } else {
        // automatic: one tile per CTA for a single image, about four for a batch
        int64_t px = 0;
        for (int k = 0; k < n; ++k) px += (int64_t)in[idx[k]].width * in[idx[k]].height;
        int nsm = 152, dev = 0;
        if (launch && cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const int64_t ctas = (int64_t)nsm * (tu.ctas_per_sm > 0 ? tu.ctas_per_sm : kAutoCtasPerSm) * (n == 1 ? 1 : 4);
        const int64_t want = (px + ctas - 1) / ctas;
        b->tile_cols = (int)std::min<int64_t>(1 << 20, std::max<int64_t>(1024, (want + 15) / 16 * 16));
        b->tile_rows = 1;
    }
    if (op.opk == kOpkLocal) {
        if (tu.tile_cols > 0) {
            b->loc_tile_cols = local_tile_cols(op.l->block_s, tu.tile_cols);
        } else {
            std::vector<std::pair<int, int>> hw(n);
            for (int k = 0; k < n; ++k) hw[k] = {in[idx[k]].height, in[idx[k]].width};
            int nsm = 152, dev = 0;
            if (launch && cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            b->loc_tile_cols = local_tile_cols_auto(op.l->block_s, hw, nsm,
                                                    tu.ctas_per_sm > 0 ? tu.ctas_per_sm : kAutoCtasPerSm);
        }
        std::vector<std::pair<int, int>> hbwb(n);
        const int s = op.l->block_s;
        for (int k = 0; k < n; ++k)
            hbwb[k] = {(in[idx[k]].height + s - 1) / s, (in[idx[k]].width + s - 1) / s};
        int nsm = 152, dev = 0;
        if (launch && cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        b->cdf_cols = cdf_cols_auto(hbwb, (int64_t)nsm * (tu.ctas_per_sm > 0 ? tu.ctas_per_sm : kAutoCtasPerSm));
    }
    b->beta_r = p->beta_r;
    b->beta_k = p->beta_k;
    b->luma = p->luma;
    b->color_s = p->color_s;
    b->color_s_one = p->color_s == 1.0f;
    b->lambda = op.lambda;
    b->vstate = op.vstate;
    b->ldr = ldr ? 1 : 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        b->profile = g_profile ? 1u : 0u;
    }
    if (op.opk == kOpkGlobal) {
        b->mode = op.g->mode;
        b->gain_k = op.g->gain_k;
        b->delta = op.g->delta;
        b->gain_is_one = op.g->gain_k == 1.0f;
        b->need_gray_hist = ldr && (op.g->mode == DC_HISTEQ || op.stats != nullptr);
        b->stats = op.stats;
        // the sigmoid needs mu; HDR histogram equalisation the log range; a stats
        // record both
        b->need_logsum = op.g->mode == DC_SIGMOID || op.stats != nullptr;
        b->need_minmax = (op.g->mode == DC_HISTEQ && !ldr) || op.stats != nullptr;
    } else if (op.opk == kOpkLocal) {
        b->block_s = op.l->block_s;
        // ceil(2^32 / s) for s >= 2 (2^32 itself does not fit: s = 1 is flagged by 0)
        b->s_magic = op.l->block_s == 1 ? 0u
                     : (uint32_t)(((uint64_t(1) << 32) + (uint64_t)op.l->block_s - 1) / (uint64_t)op.l->block_s);
        b->radius = op.l->radius_blocks;
        b->bins = op.l->bins;
        b->alpha = op.l->alpha;
        b->delta = op.l->delta;
        b->need_logsum = 0;  // the local operator uses only the log range
        b->need_minmax = 1;
    }
    // workspace layout: header | ctrl | per-image local buffers
    const int64_t ctrl_bytes = align_up((int64_t)sizeof(DcCtrl) + (int64_t)n * sizeof(DcImgCtrl), 256);
    int64_t off = kHeaderBytes + ctrl_bytes;
    std::vector<Geometry> geo(n);
    for (int k = 0; k < n; ++k) {
        make_geometry(in[idx[k]], out[idx[k]], op, tu, b->n_phase, b->phase_kind, geo[k], b->tile_rows,
                      b->tile_cols, b->loc_tile_cols, b->cdf_cols, u8_plane);
        geo[k].im.ws_hist = off;
        off += geo[k].local_bytes;
        if (geo[k].plane_bytes > 0) {
            geo[k].im.plane = ws ? ws + off : nullptr;
            off += geo[k].plane_bytes;
        }
        if (op.lvs && ws) geo[k].im.lvs = op.lvs + (*op.lvs_off)[(size_t)idx[k]];
        b->img[k] = geo[k].im;
        b->stats_index[k] = idx[k];
    }
    *need = std::max(*need, off);
    // per pass: first tile of each image; passes that re-read what the previous
    // pixel pass read hand their tiles out last-first
    {
        bool dir = false;
        for (int ph = 0; ph < b->n_phase; ++ph) {
            if (b->phase_kind[ph] == PK_CDF) {
                b->reverse[ph] = 0;
            } else {
                b->reverse[ph] = dir ? 1 : 0;
                dir = !dir;
            }
            int64_t total = 0;
            for (int i = 0; i < n; ++i) {
                b->seg_start[ph][i] = (int32_t)total;
                total += geo[i].tiles[ph];
                if (total > INT32_MAX / 2) {
                    delete b;
                    return DC_ERR_INVALID_ARG;
                }
            }
            b->seg_start[ph][n] = (int32_t)total;
        }
    }
    b->n_img = n;
    if (!launch) {
        delete b;
        return DC_OK;
    }
    b->ws = ws;
    b->ws_bytes = ws_bytes_total;
    b->lvs_buf = op.lvs;
    b->lvs_bytes = op.lvs_bytes;
    b->err = reinterpret_cast<uint32_t*>(ws);
    b->ctrl = reinterpret_cast<DcCtrl*>(ws + kHeaderBytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bool skip_memset = false, clear_at_end = false;
    const size_t block_end = (size_t)(kHeaderBytes + ctrl_bytes);
    plan_clear(ws, block_end, b->profile != 0, &skip_memset, &clear_at_end);
    b->reset_bytes = clear_at_end ? (int32_t)ctrl_bytes : 0;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        finish_clear(ws, block_end, false, clear_at_end);
        delete b;
        return DC_ERR_CUDA;
    }
    if (!skip_memset) {
        const size_t clear_bytes = first ? block_end : (size_t)ctrl_bytes;
        uint8_t* clear_ptr = first ? ws : ws + kHeaderBytes;
        if (cudaMemsetAsync(clear_ptr, 0, clear_bytes, st) != cudaSuccess) {
            finish_clear(ws, block_end, false, clear_at_end);
            delete b;
            return DC_ERR_CUDA;
        }
    }
    const int fail_at = g_fail_launch.load(std::memory_order_relaxed);
    int rc = DC_OK;
    for (int ph = 0; ph < b->n_phase && rc == DC_OK; ++ph) {
        const int kind = b->phase_kind[ph];
        // the flag: reads the plane (histogram and apply passes), or keeps only the
        // reduction the call uses (statistics passes)
        const int pl = kind == PK_STATS       ? (b->need_minmax == 0 ? 1 : 0)
                       : kind == PK_STATS_LOG ? (b->need_logsum == 0 ? 1 : 0)
                       : (color && (kind == PK_APPLY_G || kind == PK_APPLY_L || kind == PK_VIDEO || kind == PK_VIDEO_L ||
                                   kind == PK_VIDEO_H)) ? 2
                                              : ((plane && reads_plane(kind, in_dt)) ? 1 : 0);
        int occ = in_dt == DC_U8 ? occupancy_u8(CAP, op.opk, kind, pl)
                                 : (in_dt == DC_F16 ? occupancy_f16(CAP, op.opk, kind, pl) : occupancy_f32(CAP, op.opk, kind, pl));
        if (occ <= 0) occ = 1;
        const int per_sm = tu.ctas_per_sm > 0 ? std::min(tu.ctas_per_sm, occ) : occ;
        LaunchShape ls;
        ls.threads = 256;
        ls.grid = (int)std::min<int64_t>(b->seg_start[ph][n], (int64_t)per_sm * nsm);
        if (fail_at > 0 && g_call_launches + 1 == fail_at)
            rc = DC_ERR_CUDA;  // injected failure: this pass is not issued
        else if (in_dt == DC_U8)
            rc = launch_engine_u8(b, CAP, op.opk, kind, ph, pl, ls, stream);
        else if (in_dt == DC_F16)
            rc = launch_engine_f16(b, CAP, op.opk, kind, ph, pl, ls, stream);
        else
            rc = launch_engine_f32(b, CAP, op.opk, kind, ph, pl, ls, stream);
        if (rc == DC_OK) ++g_call_launches;
    }
    finish_clear(ws, block_end, rc == DC_OK, clear_at_end);
    delete b;
    return rc;
}

int run(const dc_image_in* in, const dc_image_out* out, int32_t n, const dc_decolor_params* p, const OpArgs& op,
        void* ws, size_t ws_bytes, void* stream, size_t* query, bool min_query = false)
{
    if (!in || n < 1) return DC_ERR_INVALID_ARG;
    if (n > DC_MAX_BATCH) return DC_ERR_TOO_MANY;
    if (!query && !out) return DC_ERR_INVALID_ARG;
    int rc = validate_params(p, op);
    if (rc != DC_OK) return rc;
    for (int k = 0; k < n; ++k) {
        rc = validate_image(in[k], query ? nullptr : &out[k], op.opk == kOpkLocal, op.opk != kOpkDecolor);
        if (rc != DC_OK) return rc;
    }
    if (!query && p->luma == DC_LUMA_LSTAR && op.opk == kOpkLocal) {
        for (int k = 0; k < n; ++k)
            if (in[k].dtype == DC_U8 && out[k].dtype == DC_F32) return DC_ERR_UNSUPPORTED_DTYPE;
    }
    if (!query) {
        // input must not overlap output
        for (int k = 0; k < n; ++k) {
            const uint8_t* a0 = static_cast<const uint8_t*>(in[k].data);
            const uint8_t* a1 = a0 + (in[k].height - 1) * in[k].stride_bytes + (int64_t)3 * in[k].width * esz(in[k].dtype);
            const uint8_t* b0 = static_cast<const uint8_t*>(out[k].data);
            const uint8_t* b1 = b0 + (in[k].height - 1) * out[k].stride_bytes +
                                (int64_t)in[k].width * esz(out[k].dtype) * out_channels(out[k]);
            if (a0 < b1 && b0 < a1) return DC_ERR_INVALID_ARG;
        }
    }
    // a fake (valid) output descriptor for size queries
    std::vector<dc_image_out> fake;
    const dc_image_out* outs = out;
    if (query) {
        fake.resize(n);
        for (int k = 0; k < n; ++k) {
            fake[k].data = reinterpret_cast<void*>(uintptr_t(256));
            fake[k].stride_bytes = (int64_t)in[k].width * 4;
            fake[k].dtype = DC_F32;
            fake[k].channels = 0;
        }
        outs = fake.data();
    }
    // group by input sample type and plane use, keep caller order inside a group,
    // chunk by capacity (a size query groups by sample type only: its groups are
    // never smaller than the call's)
    std::vector<LaunchPlan> plans;
    for (int dt = DC_U8; dt <= DC_F32; ++dt) {
        for (int pl = 0; pl < 3; ++pl) {  // no plane, plane, colour output (never a plane)
            LaunchPlan cur;
            cur.in_dt = dt;
            cur.plane = pl == 1;
            cur.color = pl == 2;
            for (int k = 0; k < n; ++k) {
                if (in[k].dtype != dt || keeps_plane(op, dt, outs[k]) != cur.plane || (out_channels(outs[k]) == 3) != cur.color)
                    continue;
                cur.idx.push_back(k);
                if ((int)cur.idx.size() == kCapLarge) {
                    plans.push_back(cur);
                    cur.idx.clear();
                }
            }
            if (!cur.idx.empty()) plans.push_back(cur);
        }
    }
    // workspace: with the optional 8-bit planes (what dc_workspace_bytes reports) and
    // without them (the least a call accepts); a call keeps the planes when its
    // workspace holds them
    int64_t need[2] = {kHeaderBytes, kHeaderBytes};
    for (int with_plane = 0; with_plane < 2; ++with_plane) {
        for (const LaunchPlan& pl : plans) {
            const int cnt = (int)pl.idx.size();
            const bool a = with_plane != 0;
            int64_t* nd = &need[with_plane];
            int r2;
            if (cnt <= kCapSmall)
                r2 = build_and_launch<kCapSmall>(in, outs, pl.idx, pl.plane, pl.color, a, p, op, nullptr, 0, false, nd, nullptr, false);
            else if (cnt <= kCapMid)
                r2 = build_and_launch<kCapMid>(in, outs, pl.idx, pl.plane, pl.color, a, p, op, nullptr, 0, false, nd, nullptr, false);
            else
                r2 = build_and_launch<kCapLarge>(in, outs, pl.idx, pl.plane, pl.color, a, p, op, nullptr, 0, false, nd, nullptr, false);
            if (r2 != DC_OK) return r2;
        }
    }
    if (query) {
        *query = (size_t)(min_query ? need[0] : need[1]);
        return DC_OK;
    }
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < (size_t)need[0]) return DC_ERR_WORKSPACE;
    const bool use_planes = ws_bytes >= (size_t)need[1];
    g_call_launches = 0;
    bool first = true;
    for (const LaunchPlan& pl : plans) {
        const int cnt = (int)pl.idx.size();
        int64_t dummy = 0;
        uint8_t* w = static_cast<uint8_t*>(ws);
        int r2;
        if (cnt <= kCapSmall)
            r2 = build_and_launch<kCapSmall>(in, out, pl.idx, pl.plane, pl.color, use_planes, p, op, w, (int64_t)ws_bytes, first, &dummy, stream, true);
        else if (cnt <= kCapMid)
            r2 = build_and_launch<kCapMid>(in, out, pl.idx, pl.plane, pl.color, use_planes, p, op, w, (int64_t)ws_bytes, first, &dummy, stream, true);
        else
            r2 = build_and_launch<kCapLarge>(in, out, pl.idx, pl.plane, pl.color, use_planes, p, op, w, (int64_t)ws_bytes, first, &dummy, stream, true);
        if (r2 != DC_OK) return r2;
        first = false;
    }
    g_last_launches = g_call_launches;
    return DC_OK;
}

// Workspace a call needs: with the optional 8-bit planes (min_only false) or the
// least it accepts.  0 on invalid arguments.
size_t workspace_query(int32_t op, const dc_image_in* in, int32_t n, const void* op_params, bool min_only)
{
    static const dc_decolor_params kBeta = {0.55f, 0.8f, DC_LUMA_OURS, 1.0f};
    static const dc_global_params kGlobal = {DC_SIGMOID, 1.0f, 1e-4f, 0};
    OpArgs a{0, nullptr, nullptr, nullptr};
    if (op == DC_OP_DECOLORIZE) {
        a.opk = kOpkDecolor;
    } else if (op == DC_OP_GLOBAL) {
        a.opk = kOpkGlobal;
        a.g = &kGlobal;
    } else if (op == DC_OP_LOCAL) {
        a.opk = kOpkLocal;
        a.l = static_cast<const dc_local_params*>(op_params);
        if (!a.l) return 0;
    } else {
        return 0;
    }
    size_t need = 0;
    if (run(in, nullptr, n, &kBeta, a, nullptr, 0, nullptr, &need, min_only) != DC_OK) return 0;
    return need;
}

}  // namespace

extern "C" {

DC_API int dc_decolorize(const dc_image_in* in, const dc_image_out* out, int32_t n, const dc_decolor_params* params,
                         void* ws, size_t ws_bytes, void* stream)
{
    OpArgs op{kOpkDecolor, nullptr, nullptr, nullptr};
    return run(in, out, n, params, op, ws, ws_bytes, stream, nullptr);
}

DC_API int dc_decolorize_tonemap_global(const dc_image_in* in, const dc_image_out* out, int32_t n,
                                        const dc_decolor_params* params, const dc_global_params* gparams,
                                        dc_global_stats* stats, void* ws, size_t ws_bytes, void* stream)
{
    OpArgs op{kOpkGlobal, gparams, nullptr, stats};
    return run(in, out, n, params, op, ws, ws_bytes, stream, nullptr);
}

DC_API int dc_decolorize_tonemap_local(const dc_image_in* in, const dc_image_out* out, int32_t n,
                                       const dc_decolor_params* params, const dc_local_params* lparams, void* ws,
                                       size_t ws_bytes, void* stream)
{
    OpArgs op{kOpkLocal, nullptr, lparams, nullptr};
    return run(in, out, n, params, op, ws, ws_bytes, stream, nullptr);
}

DC_API int dc_decolorize_tonemap_video(const dc_image_in* in, const dc_image_out* out, int32_t n,
                                       const dc_decolor_params* params, const dc_global_params* gparams, float lambda,
                                       int32_t restart, dc_video_state* state, void* ws, size_t ws_bytes, void* stream)
{
    if (!state || (restart != 0 && restart != 1)) return DC_ERR_INVALID_ARG;
    OpArgs op{kOpkGlobal, gparams, nullptr, nullptr};
    op.vstate = state;
    op.restart = restart != 0;
    op.lambda = lambda;
    return run(in, out, n, params, op, ws, ws_bytes, stream, nullptr);
}

DC_API size_t dc_video_local_state_bytes(const dc_image_in* in, int32_t n, const dc_local_params* lparams)
{
    if (!in || !lparams || n < 1 || n > DC_MAX_BATCH || lparams->block_s < 1 || lparams->block_s > 64 ||
        lparams->bins < 2 || lparams->bins > DC_MAX_BINS)
        return 0;
    int64_t total = 0;
    for (int k = 0; k < n; ++k) {
        if (in[k].width < 1 || in[k].height < 1) return 0;
        total += lvs_record_bytes(in[k], *lparams);
    }
    return (size_t)total;
}

DC_API int dc_decolorize_tonemap_local_video(const dc_image_in* in, const dc_image_out* out, int32_t n,
                                             const dc_decolor_params* params, const dc_local_params* lparams,
                                             int32_t restart, void* state, size_t state_bytes, void* ws,
                                             size_t ws_bytes, void* stream)
{
    if (!in || n < 1) return DC_ERR_INVALID_ARG;
    if (n > DC_MAX_BATCH) return DC_ERR_TOO_MANY;
    if (!state || (reinterpret_cast<uintptr_t>(state) & 255u) != 0 || (restart != 0 && restart != 1))
        return DC_ERR_INVALID_ARG;
    const size_t need = dc_video_local_state_bytes(in, n, lparams);
    if (need == 0 || state_bytes < need) return DC_ERR_INVALID_ARG;
    std::vector<int64_t> off((size_t)n);
    int64_t o = 0;
    for (int k = 0; k < n; ++k) {
        off[(size_t)k] = o;
        o += lvs_record_bytes(in[k], *lparams);
    }
    OpArgs op{kOpkLocal, nullptr, lparams, nullptr};
    op.lvs = static_cast<uint8_t*>(state);
    op.lvs_bytes = (int64_t)state_bytes;
    op.lvs_off = &off;
    op.restart = restart != 0;
    return run(in, out, n, params, op, ws, ws_bytes, stream, nullptr);
}

DC_API int dc_preset(int32_t preset, dc_decolor_params* p, dc_local_params* l)
{
    float bk;
    switch (preset) {
    case DC_PRESET_PAPER: bk = 0.8f; break;   // Sec. II-B
    case DC_PRESET_TM1: bk = 0.55f; break;    // background boost: cool blend weighted up
    case DC_PRESET_TM2: bk = 0.95f; break;    // background suppression: warm blend dominates
    default: return DC_ERR_INVALID_ARG;
    }
    if (p) *p = dc_decolor_params{0.55f, bk, DC_LUMA_OURS, 1.0f};
    if (l) *l = dc_local_params{32, 2, 32, 1.0f, 1e-4f, 0};
    return DC_OK;
}

DC_API size_t dc_workspace_bytes(int32_t op, const dc_image_in* in, int32_t n, const void* op_params)
{
    return workspace_query(op, in, n, op_params, false);
}

DC_API size_t dc_workspace_min_bytes(int32_t op, const dc_image_in* in, int32_t n, const void* op_params)
{
    return workspace_query(op, in, n, op_params, true);
}

DC_API int dc_workspace_prepare(void* ws, size_t ws_bytes, void* stream)
{
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < (size_t)kHeaderBytes) return DC_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ws, 0, ws_bytes, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return DC_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    g_clean[reinterpret_cast<uintptr_t>(ws)] = CleanWs{ws_bytes, ws_bytes};
    return DC_OK;
}

DC_API int dc_workspace_release(void* ws)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_clean.erase(reinterpret_cast<uintptr_t>(ws));
    return DC_OK;
}

DC_API int dc_query_status(const void* ws, void* stream)
{
    if (!ws) return DC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return DC_ERR_CUDA;
    uint32_t err = 0;
    if (cudaMemcpy(&err, ws, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess) return DC_ERR_CUDA;
    return (int)err;
}

DC_API const char* dc_status_string(int status)
{
    switch (status) {
    case DC_OK: return "ok";
    case DC_ERR_INVALID_ARG: return "invalid argument";
    case DC_ERR_UNSUPPORTED_DTYPE: return "unsupported sample type";
    case DC_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case DC_ERR_CUDA: return "CUDA runtime error";
    case DC_ERR_TIMEOUT: return "device-side dependency wait timed out";
    case DC_ERR_TOO_MANY: return "too many images in one call";
    default: return "unknown status";
    }
}

DC_API int dc_set_tuning(int32_t op, int32_t in_dtype, const dc_tuning* t)
{
    if (op < DC_OP_DECOLORIZE || op > DC_OP_LOCAL || !dt_ok(in_dtype) || !t) return DC_ERR_INVALID_ARG;
    if (t->threads != 256) return DC_ERR_INVALID_ARG;
    if (t->tile_rows < 1 || t->tile_rows > 4096 || t->tile_cols < 0 || t->tile_cols > (1 << 20) || (t->tile_cols % 16) != 0)
        return DC_ERR_INVALID_ARG;
    if (t->ctas_per_sm < 0 || t->ctas_per_sm > 32) return DC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    g_tune[op][in_dtype] = *t;
    return DC_OK;
}

DC_API int dc_get_tuning(int32_t op, int32_t in_dtype, dc_tuning* t)
{
    if (op < DC_OP_DECOLORIZE || op > DC_OP_LOCAL || !dt_ok(in_dtype) || !t) return DC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    *t = g_tune[op][in_dtype];
    return DC_OK;
}

DC_API int dc_debug_profile(int32_t on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_profile = on ? 1 : 0;
    return DC_OK;
}

DC_API int dc_debug_read_profile(const void* ws, int32_t n_img, uint64_t* out, void* stream)
{
    if (!ws || !out || n_img < 0 || n_img > kCapLarge) return DC_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return DC_ERR_CUDA;
    const uint8_t* ctrl = static_cast<const uint8_t*>(ws) + kHeaderBytes;
    DcCtrl c;
    if (cudaMemcpy(&c, ctrl, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return DC_ERR_CUDA;
    for (int i = 0; i < PROF_SLOTS; ++i) out[i] = c.prof[i];
    out[PROF_KSTART_NOT] = ~out[PROF_KSTART_NOT];
    for (int i = 0; i < n_img; ++i) {
        DcImgCtrl ic;
        if (cudaMemcpy(&ic, ctrl + sizeof(DcCtrl) + (size_t)i * sizeof(DcImgCtrl), sizeof(ic),
                       cudaMemcpyDeviceToHost) != cudaSuccess)
            return DC_ERR_CUDA;
        for (int p = 0; p < kMaxPhases; ++p) {
            out[PROF_SLOTS + i * 2 * kMaxPhases + p] = ic.t_start_not[p] ? ~ic.t_start_not[p] : 0ull;
            out[PROF_SLOTS + i * 2 * kMaxPhases + kMaxPhases + p] = ic.t_end[p];
        }
    }
    return DC_OK;
}

DC_API int dc_local_tile_cols(int32_t block_s, const int32_t* heights, const int32_t* widths, int32_t n,
                              int32_t in_dtype, int32_t n_sm, int32_t* cols)
{
    if (!heights || !widths || !cols || n < 1 || n > DC_MAX_BATCH || block_s < 1 || block_s > 64 || n_sm < 1 ||
        !dt_ok(in_dtype))
        return DC_ERR_INVALID_ARG;
    dc_tuning tu;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        tu = g_tune[DC_OP_LOCAL][in_dtype];
    }
    std::vector<std::pair<int, int>> hw((size_t)n);
    for (int k = 0; k < n; ++k) {
        if (heights[k] < 1 || widths[k] < 1) return DC_ERR_INVALID_ARG;
        hw[(size_t)k] = {heights[k], widths[k]};
    }
    *cols = tu.tile_cols > 0 ? local_tile_cols(block_s, tu.tile_cols)
                             : local_tile_cols_auto(block_s, hw, n_sm, tu.ctas_per_sm > 0 ? tu.ctas_per_sm : kAutoCtasPerSm);
    return DC_OK;
}

DC_API int dc_last_launch_count(void) { return g_last_launches; }

DC_API int dc_debug_fail_launch(int32_t k)
{
    if (k < 0) return DC_ERR_INVALID_ARG;
    g_fail_launch.store(k);
    return DC_OK;
}

DC_API int dc_debug_bounds(uint32_t* flags, int32_t* checked)
{
    if (!flags || !checked) return DC_ERR_INVALID_ARG;
    uint32_t f[3] = {0u, 0u, 0u};
    const int r0 = bounds_u8(&f[0]), r1 = bounds_f16(&f[1]), r2 = bounds_f32(&f[2]);
    if (r0 == DC_ERR_CUDA || r1 == DC_ERR_CUDA || r2 == DC_ERR_CUDA) return DC_ERR_CUDA;
    *checked = r0 == DC_OK ? 1 : 0;
    *flags = f[0] | f[1] | f[2];
    return DC_OK;
}

DC_API int dc_version(void) { return 200; }

}  // extern "C"

namespace dc {
size_t workspace_min_bytes(int32_t op, const dc_image_in* in, int32_t n, const void* op_params)
{
    return workspace_query(op, in, n, op_params, true);
}
}  // namespace dc
