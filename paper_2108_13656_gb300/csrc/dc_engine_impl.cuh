// Pass kernels: one persistent kernel per pass kind, each covering that pass's
// tiles for every image of the batch.  Included by one translation unit per input
// sample type.
#pragma once

#include <type_traits>

#include "dc_engine.cuh"

namespace dc {

struct TileRect {
    int r0, r1, c0, c1;
};

// Values a tile derives from an image's finished statistics pass.  For the
// fixed-point log forms: vmin, vmax of v = round(ln(L + delta) 2^24), the range
// R = vmax - vmin shifted right by sh until it is below 2^30 (Rs), and the
// fixed-point reciprocals m_loc = floor(bins 2^56 / Rs), m_glob = floor(256 2^54 / Rs)
// that turn v into bin coordinates.  A constant image gets the range [v - 1, v + 1],
// which puts every pixel at u = 1/2.
struct Derived {
    float mu, exp_mu, lmin, lmax;
    int vmin, vmax, sh;
    uint32_t Rs;
    unsigned long long m_loc, m_glob;
};

// Coordinate shifts: 2^-24 of a bin for the local operator (bins <= 64), 2^-22 of
// a bin for the 256-bin global histogram, so that nb 2^S stays below 2^31.
constexpr int kLocTS = 24, kGlobTS = 22;

__device__ __forceinline__ void cta_sync() { __syncthreads(); }

// Precise 8-bit bin coordinates of a group (IF_UPRECISE), as int32 bits in q.
template <int IN_DT>
__device__ __forceinline__ void ucoord_group(const uint32_t (&w)[12], int n, const Beta& be, int bins,
                                             float (&q)[InT<IN_DT>::G])
{
#pragma unroll
    for (int k = 0; k < InT<IN_DT>::G; ++k)
        q[k] = k < n ? __uint_as_float(ucoord_u8(u8_at(w, 3 * k), u8_at(w, 3 * k + 1), u8_at(w, 3 * k + 2), be, bins))
                     : 0.0f;
}

// Groups a thread loads before computing any of them (memory-level parallelism):
// the light plane-reading phases keep 64 bytes in flight per thread, the f32 RGB
// phases two 48-byte groups; the 8-bit and f16 RGB phases (more arithmetic per
// byte) rely on the number of warps instead (measured: two groups there cost time
// or registers).
#ifndef DC_UNROLL_F32_RGB
#define DC_UNROLL_F32_RGB 2
#endif
template <int IN_DT, bool PLANE>
struct Unroll {
    static constexpr int value = PLANE ? (InT<IN_DT>::G == 4 ? 4 : 2) : (IN_DT == DC_F32 ? DC_UNROLL_F32_RGB : 1);
};

// ------------------------------------------------------------ tile geometry ---
template <int CAP>
__device__ __forceinline__ int cdf_cols_tiles(const DcBatch<CAP>& P, const DcImage& im)
{
    return (im.Wb + P.cdf_cols - 1) / P.cdf_cols;
}

template <int OPK, int CAP>
__device__ __forceinline__ int phase_tiles(const DcBatch<CAP>& P, const DcImage& im, int kind)
{
    if constexpr (OPK == OPK_LOCAL) {
        return kind == PK_CDF ? im.Hb * cdf_cols_tiles(P, im) : im.Hb * im.tiles_x_loc;
    } else {
        return ((im.rows + P.tile_rows - 1) / P.tile_rows) * im.tiles_x;
    }
}

// Rectangle of tile lt of a phase; for the local operator also its block row I
// (for the CDF phase, tr.c0..tr.c1 are block columns).
template <int OPK, int CAP>
__device__ __forceinline__ TileRect tile_rect(const DcBatch<CAP>& P, const DcImage& im, int kind, int lt, int& I)
{
    TileRect tr;
    I = 0;
    if constexpr (OPK == OPK_LOCAL) {
        if (kind != PK_CDF) {
            I = lt / im.tiles_x_loc;
            const int tx = lt - I * im.tiles_x_loc;
            tr.r0 = I * P.block_s;
            tr.r1 = min(tr.r0 + P.block_s, im.prow);
            tr.c0 = tx * P.loc_tile_cols;
            tr.c1 = min(tr.c0 + P.loc_tile_cols, im.pcol);
        } else {
            const int ncc = cdf_cols_tiles(P, im);
            I = lt / ncc;
            tr.r0 = tr.r1 = 0;
            tr.c0 = (lt - I * ncc) * P.cdf_cols;
            tr.c1 = min(tr.c0 + P.cdf_cols, im.Wb);
        }
    } else {
        const int ty = lt / im.tiles_x;
        const int tx = lt - ty * im.tiles_x;
        tr.r0 = ty * P.tile_rows;
        tr.r1 = min(tr.r0 + P.tile_rows, im.rows);
        tr.c0 = tx * P.tile_cols;
        tr.c1 = min(tr.c0 + P.tile_cols, im.cols);
    }
    return tr;
}


// The coordinate parameters of a fixed-point log range [vmin, vmax] (see Derived).
__device__ __forceinline__ void derive_range(Derived& d, int vmin, int vmax, bool local, int bins)
{
    constexpr float unit = 1.0f / (float)(1 << kLogFixedShift);
    d.sh = 0;
    d.Rs = 2u;
    d.m_loc = d.m_glob = 0ull;
    d.lmin = (float)vmin * unit;
    d.lmax = (float)vmax * unit;
    if (vmax > vmin) {
        d.vmin = vmin;
        d.vmax = vmax;
        uint32_t R = (uint32_t)vmax - (uint32_t)vmin;
        while (R >= (1u << 30)) {
            R >>= 1;
            ++d.sh;
        }
        d.Rs = R;
    } else {
        d.vmin = vmin - 1;
        d.vmax = vmin + 1;
    }
    static_assert(DC_MAX_BINS <= 32 && 32 + kLocTS + 5 <= 63 && 32 + kGlobTS + 8 <= 63, "reciprocals fit in 64 bits");
    if (local)
        d.m_loc = ((unsigned long long)(unsigned)max(bins, 1) << (32 + kLocTS)) / d.Rs;
    else
        d.m_glob = (256ull << (32 + kGlobTS)) / d.Rs;
}

// mu, lmin, lmax from the exact integer accumulators of a finished stats pass
// (fixed_log: the min and max are of the 2^-24 fixed-point logarithms), and the
// fixed-point reciprocal of the log range for the operator's histogram: the local
// operator's (bins) or the global one's (256 bins).  One thread of each CTA runs
// this while the others wait, so only what the pass uses is computed: mu when the
// log-sum was kept, the reciprocal by a 64-bit division (nb 2^(32+S) <= 2^62).
__device__ __forceinline__ Derived derive(const DcImgCtrl* ic, long long N, bool fixed_log, bool want_mu,
                                          bool local, int bins)
{
    Derived d;
    constexpr float unit = 1.0f / (float)(1 << kLogFixedShift);
    d.mu = 0.0f;
    d.exp_mu = 1.0f;
    if (want_mu) {
        const long long sum = (long long)ld_cg_u64(&ic->logsum);
        const long long q = sum / N, rem = sum - q * N;
        d.mu = (__ll2float_rn(q) + __ll2float_rn(rem) / __ll2float_rn(N)) * unit;
        d.exp_mu = expf(d.mu);
    }
    d.vmin = d.vmax = d.sh = 0;
    d.Rs = 2u;
    d.m_loc = d.m_glob = 0ull;
    if (fixed_log) {
        const int vmax = (int)(ld_cg_u32(&ic->lmax_ord) ^ 0x80000000u);
        const int vmin = (int)(~ld_cg_u32(&ic->lmin_nord) ^ 0x80000000u);
        derive_range(d, vmin, vmax, local, bins);
    } else {
        d.lmin = ord_dec(~ld_cg_u32(&ic->lmin_nord));
        d.lmax = ord_dec(ld_cg_u32(&ic->lmax_ord));
    }
    return d;
}

// Bin coordinate t = nb u = nb (v - vmin) / R of a fixed-point log value, in units
// of 2^-S (0 <= t <= nb): floor(dv m / 2^32) with dv = (v - vmin) >> sh <= Rs and
// the fixed-point reciprocal m = floor(nb 2^(32+S) / Rs), i.e. floor(t 2^S) or one
// unit below it (the reciprocal's truncation is below 2^-32 of it and dv < 2^30).
// The product is at most nb 2^S < 2^31, so with m = mh 2^32 + ml it is
// dv mh + floor(dv ml / 2^32) in 32-bit arithmetic, exactly.  v is always one of the
// image's own fixed-point logs, so vmin <= v <= vmax holds without a clamp (vmin and
// vmax are their exact minimum and maximum; a value a ragged group's unused lane
// carries gives an unused coordinate, computed in wrapping unsigned arithmetic).
template <int S>
__device__ __forceinline__ uint32_t bin_coord(int v, const Derived& d)
{
    const uint32_t dv = ((uint32_t)v - (uint32_t)d.vmin) >> d.sh;
    const unsigned long long m = S == kLocTS ? d.m_loc : d.m_glob;
    return dv * (uint32_t)(m >> 32) + __umulhi(dv, (uint32_t)m);
}

// Bin coordinate of a fixed-point log value in a carried range, clamped to it (a
// frame's own values may lie outside the previous frame's range).
template <int S>
__device__ __forceinline__ uint32_t bin_coord_clamped(int v, const Derived& d)
{
    return bin_coord<S>(min(max(v, d.vmin), d.vmax), d);
}

// Bin coordinate of a value a histogram pass sees: from the plane's fixed-point
// log (a histogram pass then keeps the coordinate in the plane for the apply
// pass), or from L recomputed from RGB.
template <int S>
__device__ __forceinline__ uint32_t coord_of(float val, bool is_log_plane, float delta, const Derived& d)
{
    return bin_coord<S>(is_log_plane ? __float_as_int(val) : ln_q24(val + delta), d);
}

// ------------------------------------------------------------- group walk ---
// Visit every group of a tile: f(r, c, n, vec, v) with the group's source values
// v (the luminance from RGB, or the plane values).  Groups start at columns that
// are multiples of G from the row start, whatever the tile shape.  Threads form a
// TXT x (256/TXT) grid, TXT the smallest power of two covering a row's groups, so
// the mapping needs no integer division; each thread issues the loads of U groups
// before computing any of them.
// RAW (RGB walks only): f also receives the group's raw sample words, which a
// ragged or unaligned group gathers sample by sample (lanes past n zero), so that
// every group then takes the same decode.
template <int IN_DT, bool PLANE, bool RAW = false, class F>
__device__ __forceinline__ void walk_group(const DcImage& im, const Beta& be, F&& f, int r, int c, int n, bool vec,
                                           const uint8_t* src, float (&v)[InT<IN_DT>::G],
                                           uint32_t (&w)[PLANE ? 1 : 12], bool load)
{
    static_assert(!(RAW && PLANE), "raw samples come from an RGB walk");
    if (load) {
        if constexpr (PLANE) {
            if (vec)
                GroupIO<IN_DT>::from_plane_at(im, reinterpret_cast<const float*>(src), v);
            else
                GroupIO<IN_DT>::from_plane(im, r, c, n, false, v);
        } else {
            if (vec)
                GroupIO<IN_DT>::load_raw_at(im, src, w);
            else if constexpr (RAW)
                GroupIO<IN_DT>::gather_raw(im, r, c, n, w);
            else
                GroupIO<IN_DT>::luminance(im, r, c, n, false, be, v);
        }
    } else {
        if constexpr (!PLANE) {
            if (vec || RAW) GroupIO<IN_DT>::decode(w, be, v);
        }
        if constexpr (RAW)
            f(r, c, n, vec, v, w);
        else
            f(r, c, n, vec, v);
    }
}

// Full groups are addressed from a pointer per thread: along a row the U groups of
// an iteration sit at constant offsets from it, down a column it advances by a
// fixed step, so no group recomputes its address from (r, c).
template <int IN_DT, bool PLANE, bool RAW = false, class F>
__device__ __forceinline__ void walk_tile(const DcImage& im, const TileRect& t, const Beta& be, F&& f)
{
    constexpr int G = InT<IN_DT>::G, U = Unroll<IN_DT, PLANE>::value;
    constexpr int GB = PLANE ? 4 * G : 3 * InT<IN_DT>::ESZ * G;  // source bytes of a group
    const int gpr = (t.c1 - t.c0 + G - 1) / G;
    const int lg = gpr >= kThreads ? 8 : 32 - __clz(gpr - 1);
    const int txt = 1 << lg;
    const int tx = threadIdx.x & (txt - 1);
    const int rpi = kThreads >> lg;
    const bool vec_img = (im.flags & IF_VEC) != 0;
    const uint8_t* const src0 = PLANE ? im.plane : im.in;
    const int64_t sstride = PLANE ? im.plane_stride : im.in_stride;
    int c[U], n[U], rr[U];
    bool vec[U];
    float v[U][G];
    uint32_t w[U][PLANE ? 1 : 12];
    if (gpr >= kThreads) {
        // long rows: the U groups of an iteration lie along the row
        for (int r = t.r0; r < t.r1; ++r) {
            const uint8_t* q = src0 + (int64_t)r * sstride + (int64_t)(t.c0 / G + tx) * GB;
            for (int g = tx; g < gpr; g += U * kThreads, q += (int64_t)U * kThreads * GB) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int gu = g + u * kThreads;
                    c[u] = t.c0 + gu * G;
                    n[u] = gu < gpr ? min(G, t.c1 - c[u]) : 0;
                    vec[u] = vec_img && n[u] == G;
                    if (n[u] > 0)
                        walk_group<IN_DT, PLANE, RAW>(im, be, f, r, c[u], n[u], vec[u], q + u * kThreads * GB, v[u], w[u],
                                                      true);
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (n[u] > 0) walk_group<IN_DT, PLANE, RAW>(im, be, f, r, c[u], n[u], vec[u], nullptr, v[u], w[u], false);
            }
        }
    } else {
        // short rows: one group per thread per row, the U groups lie in U rows
        const int cc = t.c0 + tx * G;
        const int nn = tx < gpr ? min(G, t.c1 - cc) : 0;
        const bool vv = vec_img && nn == G;
        const int r_first = t.r0 + (threadIdx.x >> lg);
        const int64_t step = (int64_t)rpi * sstride;
        const uint8_t* q = src0 + (int64_t)r_first * sstride + (int64_t)(t.c0 / G + tx) * GB;
        for (int r = r_first; r < t.r1; r += U * rpi, q += U * step) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                rr[u] = r + u * rpi;
                n[u] = rr[u] < t.r1 ? nn : 0;
                if (n[u] > 0) walk_group<IN_DT, PLANE, RAW>(im, be, f, rr[u], cc, n[u], vv, q + u * step, v[u], w[u], true);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (n[u] > 0) walk_group<IN_DT, PLANE, RAW>(im, be, f, rr[u], cc, n[u], vv, nullptr, v[u], w[u], false);
        }
    }
}

// Block-patch walk of a local-operator tile: each warp takes patches about one
// block wide (lx lanes of G pixels across, lx the largest power of two <= s/G, and
// 32/lx rows down), so that the lanes of a warp read the same block's tone curves -
// mostly the same or neighbouring bins of them - instead of several blocks' (fewer
// shared-memory bank conflicts).  Groups stay aligned to multiples of G.
template <int IN_DT, bool PLANE, bool RAW = false, class F>
__device__ __forceinline__ void walk_block_patches(const DcImage& im, const TileRect& t, int s, const Beta& be, F&& f)
{
    constexpr int G = InT<IN_DT>::G, U = Unroll<IN_DT, PLANE>::value;
    constexpr int W = kThreads / 32;
    const int lgx = min(5, 31 - __clz(max(1, s / G)));
    const int lx = 1 << lgx, ly = 32 >> lgx, pw = lx * G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gx = lane & (lx - 1), gy = lane >> lgx;
    const int npx = (t.c1 - t.c0 + pw - 1) / pw;
    const bool vec_img = (im.flags & IF_VEC) != 0;
    int c[U], n[U], rr[U];
    bool vec[U];
    float v[U][G];
    uint32_t w[U][PLANE ? 1 : 12];
    // warp w takes patch columns w, w + W, ... and walks each down the tile, U
    // patches at a time (no integer division)
    for (int px = warp; px < npx; px += W) {
        const int cc = t.c0 + px * pw + gx * G;
        const int nn = max(0, min(G, t.c1 - cc));
        const bool vv = vec_img && nn == G;
        for (int r0 = t.r0 + gy; r0 < t.r1; r0 += U * ly) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                rr[u] = r0 + u * ly;
                c[u] = cc;
                n[u] = rr[u] < t.r1 ? nn : 0;
                vec[u] = vv;
                if (n[u] > 0) {
                    const uint8_t* src = PLANE ? im.plane + (int64_t)rr[u] * im.plane_stride + (int64_t)c[u] * 4
                                               : im.in + (int64_t)rr[u] * im.in_stride + (int64_t)c[u] * 3 * InT<IN_DT>::ESZ;
                    walk_group<IN_DT, PLANE, RAW>(im, be, f, rr[u], c[u], n[u], vec[u], src, v[u], w[u], true);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (n[u] > 0) walk_group<IN_DT, PLANE, RAW>(im, be, f, rr[u], c[u], n[u], vec[u], nullptr, v[u], w[u], false);
        }
    }
}

// The same walk for a pass that reads the f32 plane and writes the output: f(r, c,
// v) turns the G plane values of a group into output values in place and the walk
// stores them in the output type OUT_DT.  A thread's groups share one column, so
// full groups of an aligned image move through two row pointers advanced by ly
// rows at a time; a ragged right edge takes the general group I/O.
template <int IN_DT, int OUT_DT, class F>
__device__ __forceinline__ void walk_block_patches_plane(const DcImage& im, const TileRect& t, int s, F&& f)
{
    constexpr int G = InT<IN_DT>::G, U = Unroll<IN_DT, true>::value;
    constexpr int OE = OUT_DT == DC_U8 ? 1 : (OUT_DT == DC_F16 ? 2 : 4);
    constexpr int W = kThreads / 32;
    const int lgx = min(5, 31 - __clz(max(1, s / G)));
    const int lx = 1 << lgx, ly = 32 >> lgx, pw = lx * G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gx = lane & (lx - 1), gy = lane >> lgx;
    const int npx = (t.c1 - t.c0 + pw - 1) / pw;
    const bool vec_img = (im.flags & IF_VEC) != 0;
    const int64_t pstep = im.plane_stride * ly, ostep = im.out_stride * ly;
    const int64_t pext = GroupIO<IN_DT>::plane_extent(im), oext = GroupIO<IN_DT>::out_extent(im);
    for (int px = warp; px < npx; px += W) {
        const int cc = t.c0 + px * pw + gx * G;
        const int nn = max(0, min(G, t.c1 - cc));
        if (vec_img && nn == G) {
            const uint8_t* pp = im.plane + (int64_t)(t.r0 + gy) * im.plane_stride + (int64_t)cc * 4;
            uint8_t* op = im.out + (int64_t)(t.r0 + gy) * im.out_stride + (int64_t)cc * OE;
            for (int r0 = t.r0 + gy; r0 < t.r1; r0 += U * ly) {
                float v[U][G];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float* q = reinterpret_cast<const float*>(pp + u * pstep);
                    const bool ok = r0 + u * ly < t.r1 && bc_ok(q, G * 4, im.plane, pext, BC_PLANE);
#pragma unroll
                    for (int k = 0; k < G; k += 4) {
                        const float4 x = ok ? ld_cg_f4(q + k) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        v[u][k] = x.x;
                        v[u][k + 1] = x.y;
                        v[u][k + 2] = x.z;
                        v[u][k + 3] = x.w;
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (r0 + u * ly < t.r1) {
                        f(r0 + u * ly, cc, v[u]);
                        uint8_t* o = op + u * ostep;
                        if (bc_ok(o, G * OE, im.out, oext, BC_OUT)) GroupIO<IN_DT>::template store_full<OUT_DT>(o, v[u]);
                    }
                }
                pp += U * pstep;
                op += U * ostep;
            }
        } else if (nn > 0) {
            for (int r = t.r0 + gy; r < t.r1; r += ly) {
                float v[G];
                GroupIO<IN_DT>::from_plane(im, r, cc, nn, false, v);
                f(r, cc, v);
                GroupIO<IN_DT>::store(im, r, cc, nn, false, v);
            }
        }
    }
}

// PLANE: the pass reads the f32 plane an earlier pass kept (every image of the
// launch has one), else it recomputes the luminance from RGB.
template <int IN_DT, bool PLANE, class F>
__device__ __forceinline__ void consume_tile(const DcImage& im, const TileRect& t, const Beta& be, F&& f)
{
    walk_tile<IN_DT, PLANE>(im, t, be, f);
}

// --------------------------------------------------------------- reductions --
__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Inclusive scan of one uint32 per consumer thread.
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t* scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) scratch[warp] = v;
    cta_sync();
    uint32_t off = 0;
    for (int w = 0; w < warp; ++w) off += scratch[w];
    cta_sync();
    return v + off;
}

// ------------------------------------------------------------- phase: stats --
// LOGQ = false (sigmoid curve, 8-bit input): ln(L + delta) from the hardware
// logarithm, each group's pairwise sum rounded once to 2^-24; min/max on the
// floats.  LOGQ = true (HDR histogram forms): the fixed-point logarithm of every
// pixel, summed exactly; min/max on the integers; the plane keeps the integers.
template <int IN_DT, bool LOGQ, bool LEAN, int CAP>
__device__ void tile_stats(const DcBatch<CAP>& P, const DcImage& im, DcImgCtrl* ic,
                           const TileRect& t, const Beta& be, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    SmemStats& S = *reinterpret_cast<SmemStats*>(smem);
    const bool want_hist = !LOGQ && P.need_gray_hist != 0;
    const bool plane_out = (im.flags & IF_LPLANE) != 0;
    const bool plane_log = (im.flags & IF_PLANE_LOG) != 0;
    if (want_hist) {
        for (int b = threadIdx.x; b < 256; b += kThreads) S.hist[b] = 0;
        cta_sync();
    }
    long long acc = 0;
    float vmin = INFINITY, vmax = -INFINITY;
    int qmin = INT_MAX, qmax = INT_MIN;
    const float delta = P.delta;
    // LEAN: only the reduction the call uses - the log-sum for the sigmoid (no min/max),
    // the log range for the HDR histogram forms (no log-sum); otherwise both, for the
    // stats record
    constexpr bool SUM = !(LOGQ && LEAN), MM = !(!LOGQ && LEAN);
    consume_tile<IN_DT, false>(im, t, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
        float v[G];
        if constexpr (LOGQ) {
            auto px = [&](int k) __attribute__((always_inline)) {
                const int q = ln_q24(Lv[k] + delta);
                if constexpr (SUM) acc += q;
                qmin = min(qmin, q);
                qmax = max(qmax, q);
                v[k] = __int_as_float(q);
            };
            if (n == G) {  // a full group (the common case) without a guard per pixel
#pragma unroll
                for (int k = 0; k < G; ++k) px(k);
            } else {
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    if (k < n) px(k);
                    else v[k] = 0.0f;
                }
            }
            if (plane_out) GroupIO<IN_DT>::store_plane(im, r, c, n, vec, plane_log ? v : Lv);
        } else {
            // base-2 logarithms: the group's sum is scaled to natural units once, and
            // min / max (monotone in the scaling) when the record is written
#pragma unroll
            for (int k = 0; k < G; ++k) {
                if (k < n) {
                    v[k] = lg2_ftz(Lv[k] + delta);
                    if constexpr (MM) {
                        vmin = fminf(vmin, v[k]);
                        vmax = fmaxf(vmax, v[k]);
                    }
                    if (want_hist) atomicAdd(&S.hist[quant_u8(Lv[k])], 1u);
                } else {
                    v[k] = 0.0f;
                }
            }
            if (plane_out) GroupIO<IN_DT>::store_plane(im, r, c, n, vec, Lv);
            acc += __float2ll_rn(pairwise_sum<G>(v) * kLn2Q24);
        }
    });
    acc = warp_sum_ll(acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (LOGQ) {
        qmin = __reduce_min_sync(0xffffffffu, qmin);
        qmax = __reduce_max_sync(0xffffffffu, qmax);
        if (lane == 0) {
            S.wsum[warp] = acc;
            S.wmin[warp] = __int_as_float(qmin);
            S.wmax[warp] = __int_as_float(qmax);
        }
    } else {
        vmin = warp_min(vmin) * 0.693147180559945309f;  // (the natural logarithm of each pixel's)
        vmax = warp_max(vmax) * 0.693147180559945309f;
        if (lane == 0) {
            S.wsum[warp] = acc;
            S.wmin[warp] = vmin;
            S.wmax[warp] = vmax;
        }
    }
    cta_sync();
    if (threadIdx.x == 0) {
        long long sum = 0;
        for (int w = 0; w < (kThreads / 32); ++w) sum += S.wsum[w];
        atomicAdd(&ic->logsum, (unsigned long long)sum);
        if constexpr (LOGQ) {
            int mn = INT_MAX, mx = INT_MIN;
            for (int w = 0; w < (kThreads / 32); ++w) {
                mn = min(mn, __float_as_int(S.wmin[w]));
                mx = max(mx, __float_as_int(S.wmax[w]));
            }
            if (mx >= mn) {  // ordered encoding of a signed integer: flip the sign bit
                atomicMax(&ic->lmax_ord, (uint32_t)mx ^ 0x80000000u);
                atomicMax(&ic->lmin_nord, ~((uint32_t)mn ^ 0x80000000u));
            }
        } else {
            float mn = INFINITY, mx = -INFINITY;
            for (int w = 0; w < (kThreads / 32); ++w) {
                mn = fminf(mn, S.wmin[w]);
                mx = fmaxf(mx, S.wmax[w]);
            }
            if (mx >= mn) {
                atomicMax(&ic->lmax_ord, ord_enc(mx));
                atomicMax(&ic->lmin_nord, ~ord_enc(mn));
            }
        }
    }
    if (want_hist) {
        for (int b = threadIdx.x; b < 256; b += kThreads)
            if (S.hist[b]) atomicAdd(&ic->hist[b], S.hist[b]);
    }
}

// ---------------------------------------------------------- phase: log hist --
template <int IN_DT, bool PLANE, int CAP>
__device__ void tile_loghist(const DcBatch<CAP>& P, const DcImage& im, DcImgCtrl* ic,
                             const TileRect& t, const Beta& be, const Derived& d, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    SmemStats& S = *reinterpret_cast<SmemStats*>(smem);
    for (int b = threadIdx.x; b < 256; b += kThreads) S.hist[b] = 0;
    constexpr bool plane = PLANE;
    const bool is_log = plane && (im.flags & IF_PLANE_LOG) != 0;
    const float delta = P.delta;
    cta_sync();
    consume_tile<IN_DT, PLANE>(im, t, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
        float tq[G] = {};
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const uint32_t q = k < n ? coord_of<kGlobTS>(Lv[k], is_log, delta, d) : 0u;
            tq[k] = __uint_as_float(q);
            if (k < n) atomicAdd(&S.hist[min(q >> kGlobTS, 255u)], 1u);
        }
        // the apply pass reads the coordinate instead of the logarithm
        if (is_log) GroupIO<IN_DT>::store_plane(im, r, c, n, vec, tq);
    });
    cta_sync();
    for (int b = threadIdx.x; b < 256; b += kThreads)
        if (S.hist[b]) atomicAdd(&ic->hist[b], S.hist[b]);
}

// Per-image statistics record, written once by the first tile of the last phase.
template <int CAP>
__device__ void write_stats(const DcBatch<CAP>& P, const DcImage& im, const DcImgCtrl* ic, int img,
                            const Derived& d)
{
    dc_global_stats* st = &P.stats[P.stats_index[img]];
    const bool has_hist = P.ldr || P.mode == DC_HISTEQ;
    st->hist[threadIdx.x] = has_hist ? ld_cg_u32(&ic->hist[threadIdx.x]) : 0u;
    if (threadIdx.x == 0) {
        st->mu = d.mu;
        st->logmin = d.lmin;
        st->logmax = d.lmax;
        st->reserved0 = 0.0f;
        st->logsum_fixed = (int64_t)ld_cg_u64(&ic->logsum);
        st->npix = (long long)im.prow * (long long)im.pcol;
    }
}

// ------------------------------------------------------- phase: global apply --
template <int IN_DT, bool PLANE, int CAP>
__device__ void tile_apply_global(const DcBatch<CAP>& P, const DcImage& im,
                                  DcImgCtrl* ic, const TileRect& t, const Beta& be, const Derived& d,
                                  unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    SmemApplyG& S = *reinterpret_cast<SmemApplyG*>(smem);
    constexpr bool plane = PLANE;
    const bool is_log = plane && (im.flags & IF_PLANE_LOG) != 0;
    const float delta = P.delta;
    if (P.mode == DC_SIGMOID) {
        const float mu = d.mu, exp_mu = d.exp_mu, k = P.gain_k;
        const bool one = P.gain_is_one != 0;
        consume_tile<IN_DT, PLANE>(im, t, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const float x = Lv[j] + delta;
                // y = 1 / (1 + exp(-k (ln x - mu)));  k = 1: y = x / (x + e^mu)
                Lv[j] = one ? __fdividef(x, x + exp_mu) : rcp_fast(1.0f + exp_fast(-k * (ln_fast(x) - mu)));
            }
            GroupIO<IN_DT>::store(im, r, c, n, vec, Lv);
        });
    } else {
        // cumulative table from the finished histogram (every tile builds its own copy)
        const long long N = (long long)im.prow * (long long)im.pcol;
        const uint32_t h = ld_cg_u32(&ic->hist[threadIdx.x]);
        SmemStats& T = *reinterpret_cast<SmemStats*>(smem + sizeof(SmemApplyG));
        const uint32_t cum = block_incl_scan(h, T.scan);
        const float invN = 1.0f / __ll2float_rn(N);
        if (P.ldr) {
            S.lut[threadIdx.x] = __uint2float_rn(cum) * invN;  // y for gray code q: count(<= q) / N
        } else {
            S.lut[threadIdx.x] = __uint2float_rn(cum - h) * invN;  // edge b: count(bins < b) / N
            if (threadIdx.x == 0) S.lut[256] = 1.0f;
        }
        cta_sync();
        const bool ldr = P.ldr != 0;
        consume_tile<IN_DT, PLANE>(im, t, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
#pragma unroll
            for (int j = 0; j < G; ++j) {
                if (ldr) {
                    Lv[j] = S.lut[quant_u8(Lv[j])];
                } else {
                    // bin coordinate: kept in the plane by the histogram pass, or
                    // computed from L recomputed from RGB
                    const uint32_t q = is_log ? __float_as_uint(Lv[j]) : coord_of<kGlobTS>(Lv[j], false, delta, d);
                    const uint32_t b = min(q >> kGlobTS, 255u);
                    const float frac = (float)(q - (b << kGlobTS)) * (1.0f / (float)(1u << kGlobTS));
                    const float e0 = S.lut[b], e1 = S.lut[b + 1];
                    Lv[j] = fmaf(frac, e1 - e0, e0);
                }
            }
            GroupIO<IN_DT>::store(im, r, c, n, vec, Lv);
        });
    }
}

// Global curve with colour output: L and the tone-mapped y from the recomputed
// luminance, then the colour reconstruction of every pixel (interleaved RGB out).
template <int IN_DT, int CAP>
__device__ void tile_apply_global_color(const DcBatch<CAP>& P, const DcImage& im, DcImgCtrl* ic, const TileRect& t,
                                        const Beta& be, const Derived& d, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    SmemApplyG& S = *reinterpret_cast<SmemApplyG*>(smem);
    const float delta = P.delta, cs = P.color_s;
    const bool s_one = P.color_s_one != 0, sigmoid = P.mode == DC_SIGMOID, ldr = P.ldr != 0;
    if (!sigmoid) {
        const long long N = (long long)im.prow * (long long)im.pcol;
        const uint32_t h = ld_cg_u32(&ic->hist[threadIdx.x]);
        SmemStats& T = *reinterpret_cast<SmemStats*>(smem + sizeof(SmemApplyG));
        const uint32_t cum = block_incl_scan(h, T.scan);
        const float invN = 1.0f / __ll2float_rn(N);
        if (ldr) {
            S.lut[threadIdx.x] = __uint2float_rn(cum) * invN;
        } else {
            S.lut[threadIdx.x] = __uint2float_rn(cum - h) * invN;
            if (threadIdx.x == 0) S.lut[256] = 1.0f;
        }
        cta_sync();
    }
    const float mu = d.mu, exp_mu = d.exp_mu, k = P.gain_k;
    const bool one = P.gain_is_one != 0;
    walk_tile<IN_DT, false, true>(im, t, be, [&](int r, int c, int n, bool vec, float (&Lv)[G], const uint32_t (&w)[12])
                                                 __attribute__((always_inline)) {
        float y[G], o[3 * G];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (sigmoid) {
                const float x = Lv[j] + delta;
                y[j] = one ? __fdividef(x, x + exp_mu) : rcp_fast(1.0f + exp_fast(-k * (ln_fast(x) - mu)));
            } else if (ldr) {
                y[j] = S.lut[quant_u8(Lv[j])];
            } else {
                const uint32_t q = coord_of<kGlobTS>(Lv[j], false, delta, d);
                const uint32_t b = min(q >> kGlobTS, 255u);
                const float frac = (float)(q - (b << kGlobTS)) * (1.0f / (float)(1u << kGlobTS));
                const float e0 = S.lut[b], e1 = S.lut[b + 1];
                y[j] = fmaf(frac, e1 - e0, e0);
            }
        }
        GroupIO<IN_DT>::color_values(w, Lv, y, be, cs, s_one, o);
        GroupIO<IN_DT>::store_rgb(im, r, c, n, vec, o);
    });
}

// ---------------------------------------------------------- phase: video --
// Frame sequences: the centred sigmoid around the carried log-mean m of the image's
// stream (one pass), and the frame's own log-sum for the next estimate, rounded per
// group to 2^-24 exactly as the statistics pass sums it.
// Histogram equalisation of a frame of a running sequence: the cumulative table of
// the previous frame's histogram (the stream's record) maps every pixel - 8-bit: its
// gray code; HDR: its u-bin in the previous frame's log range, clamped - and the
// frame's own histogram (binned the same way) and own log range are accumulated.
template <int IN_DT, bool COLOR, int CAP>
__device__ void tile_video_histeq(const DcBatch<CAP>& P, const DcImage& im, DcImgCtrl* ic, const dc_video_state* vs,
                                  const TileRect& t, const Beta& be, const Derived& d, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    constexpr bool ldr = IN_DT == DC_U8;
    SmemStats& S = *reinterpret_cast<SmemStats*>(smem);
    SmemApplyG& A = *reinterpret_cast<SmemApplyG*>(smem + sizeof(SmemStats));
    const uint32_t h = ld_cg_u32(&vs->hist[threadIdx.x]);
    const uint32_t cum = block_incl_scan(h, S.scan);
    const long long Np = max((long long)ld_cg_u64(reinterpret_cast<const unsigned long long*>(&vs->npix)), 1ll);
    const float invN = 1.0f / __ll2float_rn(Np);
    if (ldr) {
        A.lut[threadIdx.x] = __uint2float_rn(cum) * invN;  // code q: count(<= q) / N
    } else {
        A.lut[threadIdx.x] = __uint2float_rn(cum - h) * invN;  // edge b: count(bins < b) / N
        if (threadIdx.x == 0) A.lut[256] = 1.0f;
    }
    S.hist[threadIdx.x] = 0u;
    const float delta = P.delta;
    int qmin = INT_MAX, qmax = INT_MIN;
    cta_sync();
    auto curve = [&](int n, const float (&Lv)[G], float (&y)[G]) __attribute__((always_inline)) {
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (ldr) {
                const uint32_t q = quant_u8(Lv[j]);
                y[j] = A.lut[q];
                if (j < n) atomicAdd(&S.hist[q], 1u);
            } else {
                const int v = ln_q24(Lv[j] + delta);
                if (j < n) {
                    qmin = min(qmin, v);
                    qmax = max(qmax, v);
                }
                const uint32_t q = bin_coord_clamped<kGlobTS>(v, d);
                const uint32_t b = min(q >> kGlobTS, 255u);
                const float frac = (float)(q - (b << kGlobTS)) * (1.0f / (float)(1u << kGlobTS));
                const float e0 = A.lut[b], e1 = A.lut[b + 1];
                y[j] = fmaf(frac, e1 - e0, e0);
                if (j < n) atomicAdd(&S.hist[b], 1u);
            }
        }
    };
    if constexpr (COLOR) {
        const float cs = P.color_s;
        const bool s_one = P.color_s_one != 0;
        walk_tile<IN_DT, false, true>(im, t, be, [&](int r, int c, int n, bool vec, float (&Lv)[G], const uint32_t (&w)[12])
                                                     __attribute__((always_inline)) {
            float y[G], o[3 * G];
            curve(n, Lv, y);
            GroupIO<IN_DT>::color_values(w, Lv, y, be, cs, s_one, o);
            GroupIO<IN_DT>::store_rgb(im, r, c, n, vec, o);
        });
    } else {
        consume_tile<IN_DT, false>(im, t, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
            float y[G];
            curve(n, Lv, y);
            GroupIO<IN_DT>::store(im, r, c, n, vec, y);
        });
    }
    cta_sync();
    if (S.hist[threadIdx.x]) atomicAdd(&ic->hist[threadIdx.x], S.hist[threadIdx.x]);
    if constexpr (!ldr) {
        qmin = __reduce_min_sync(0xffffffffu, qmin);
        qmax = __reduce_max_sync(0xffffffffu, qmax);
        if ((threadIdx.x & 31) == 0) {
            S.wmin[threadIdx.x >> 5] = __int_as_float(qmin);
            S.wmax[threadIdx.x >> 5] = __int_as_float(qmax);
        }
        cta_sync();
        if (threadIdx.x == 0) {
            int mn = INT_MAX, mx = INT_MIN;
            for (int w = 0; w < kThreads / 32; ++w) {
                mn = min(mn, __float_as_int(S.wmin[w]));
                mx = max(mx, __float_as_int(S.wmax[w]));
            }
            if (mx >= mn) {
                atomicMax(&ic->lmax_ord, (uint32_t)mx ^ 0x80000000u);
                atomicMax(&ic->lmin_nord, ~((uint32_t)mn ^ 0x80000000u));
            }
        }
    }
}

// COLOR: interleaved RGB output (the colour reconstruction of each pixel).
template <int IN_DT, bool COLOR, int CAP>
__device__ void tile_video(const DcBatch<CAP>& P, const DcImage& im, DcImgCtrl* ic, const TileRect& t,
                           const Beta& be, const Derived& d, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    SmemStats& S = *reinterpret_cast<SmemStats*>(smem);
    const float delta = P.delta, mu = d.mu, exp_mu = d.exp_mu, k = P.gain_k;
    const bool one = P.gain_is_one != 0;
    long long acc = 0;
    // y of a group in place and its log-sum; Lv: the luminance
    auto curve = [&](int n, float (&Lv)[G], float (&y)[G]) __attribute__((always_inline)) {
        float v[G];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const float x = Lv[j] + delta;
            const float l2 = lg2_ftz(x);  // (summed as the statistics pass sums it)
            v[j] = j < n ? l2 : 0.0f;
            y[j] = one ? __fdividef(x, x + exp_mu)
                       : rcp_fast(1.0f + exp_fast(-k * (l2 * 0.693147180559945309f - mu)));
        }
        acc += __float2ll_rn(pairwise_sum<G>(v) * kLn2Q24);
    };
    if constexpr (COLOR) {
        const float cs = P.color_s;
        const bool s_one = P.color_s_one != 0;
        walk_tile<IN_DT, false, true>(im, t, be, [&](int r, int c, int n, bool vec, float (&Lv)[G], const uint32_t (&w)[12])
                                                     __attribute__((always_inline)) {
            float y[G], o[3 * G];
            curve(n, Lv, y);
            GroupIO<IN_DT>::color_values(w, Lv, y, be, cs, s_one, o);
            GroupIO<IN_DT>::store_rgb(im, r, c, n, vec, o);
        });
    } else {
        consume_tile<IN_DT, false>(im, t, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
            curve(n, Lv, Lv);
            GroupIO<IN_DT>::store(im, r, c, n, vec, Lv);
        });
    }
    acc = warp_sum_ll(acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) S.wsum[warp] = acc;
    cta_sync();
    if (threadIdx.x == 0) {
        long long sum = 0;
        for (int w = 0; w < (kThreads / 32); ++w) sum += S.wsum[w];
        atomicAdd(&ic->logsum, (unsigned long long)sum);
    }
}

// ---------------------------------------------------- phase: local histograms --
// Tent binning: x = B u - 1/2 in 2^-20 fixed point, clamped to [0, (B-1) 2^20];
// j = x >> 20 takes 1 - f, bin j+1 takes f.  Per block and bin the tile counts the
// pixels with lower bin j and sums their f (two native 32-bit shared atomics per
// run of equal keys; exact for blocks up to 64 x 64).  Bin j's mass is then
// count_j 2^20 - F_j + F_{j-1}, stored as a 64-bit integer in units of 2^-20.
template <int IN_DT, bool PLANE, int CAP>
__device__ void tile_blockh(const DcBatch<CAP>& P, const DcImage& im, const TileRect& t, int I,
                            const Beta& be, const Derived& d, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    SmemBlockH& S = *reinterpret_cast<SmemBlockH*>(smem);
    const int s = P.block_s, B = P.bins;
    const int nbx = (t.c1 - t.c0 + s - 1) / s;
    const int BS = blockh_stride(B);
    static_assert(blockh_stride(DC_MAX_BINS) <= DC_MAX_BINS + 8, "counter stride");
    for (int k = threadIdx.x; k < nbx * BS; k += kThreads) {
        S.cnt[k] = 0u;
        S.fs[k] = 0u;
    }
    constexpr bool plane = PLANE;
    const bool plane_out = !PLANE && (im.flags & IF_LPLANE) != 0;  // this pass writes the plane
    const bool is_log = plane && (im.flags & IF_PLANE_LOG) != 0;
    const bool ldr = P.ldr != 0;
    const float delta = P.delta, scale = (float)B * 1048576.0f;
    const int xmax = (B - 1) << 20;
    const uint32_t magic = P.s_magic;
    const bool group_in_block = magic != 0u && s % G == 0;  // a G-pixel group never straddles blocks
    // 8-bit input with the precise coordinate: from the raw codes of an RGB walk
    const bool precise = ldr && (im.flags & IF_UPRECISE) != 0;
    cta_sync();
    // wp: the group's raw words (RGB walk) or null (plane walk); PREC: the precise
    // 8-bit coordinate, a literal at each (inlined) call, so that each walk's loop
    // holds only its own path
    auto group_fn = [&](bool PREC, int r, int c, int n, bool vec, float (&Lv)[G], const uint32_t (*wp)[12])
                        __attribute__((always_inline)) {
        float qv[G];
        if (PREC) ucoord_group<IN_DT>(*wp, n, be, B, qv);
        const int blk0 = group_in_block ? (int)__umulhi((uint32_t)(c - t.c0), magic) : 0;
        int cur = -1;
        uint32_t rc = 0u, rf = 0u;
        auto px = [&](int k) __attribute__((always_inline)) {
            int x;
            if (PREC) {
                // t - 1/2 from 2^-24 to 2^-20 units, rounded (as for HDR input)
                x = min(max(((int)__float_as_uint(qv[k]) - (1 << (kLocTS - 1)) + 8) >> (kLocTS - 20), 0), xmax);
            } else if (ldr) {
                x = min(max(__float2int_rn(fmaf(fminf(fmaxf(Lv[k], 0.0f), 1.0f), scale, -524288.0f)), 0), xmax);
            } else {
                // t - 1/2 from 2^-24 to 2^-20 units, rounded
                const uint32_t q = coord_of<kLocTS>(Lv[k], is_log, delta, d);
                x = min(max(((int)q - (1 << (kLocTS - 1)) + 8) >> (kLocTS - 20), 0), xmax);
            }
            int blk = blk0;
            if (!group_in_block) {
                const uint32_t off = (uint32_t)(c + k - t.c0);
                blk = magic ? (int)__umulhi(off, magic) : (int)off;
            }
            const int key = blk * BS + (x >> 20);
            const uint32_t f = (uint32_t)x & 0xFFFFFu;
            if (key == cur) {
                ++rc;
                rf += f;
            } else {
                if (cur >= 0) {
                    atomicAdd(&S.cnt[cur], rc);
                    atomicAdd(&S.fs[cur], rf);
                }
                cur = key;
                rc = 1u;
                rf = f;
            }
        };
        // an RGB walk's full group (the common case) without a guard per pixel (for
        // the plane walk this measured slower)
        if (!PLANE && n == G) {
#pragma unroll
            for (int k = 0; k < G; ++k) px(k);
        } else {
#pragma unroll
            for (int k = 0; k < G; ++k)
                if (k < n) px(k);
        }
        if (cur >= 0) {
            atomicAdd(&S.cnt[cur], rc);
            atomicAdd(&S.fs[cur], rf);
        }
        // 8-bit input with a workspace plane: the apply pass reads the luminance
        // instead of recomputing it (an HDR plane keeps the fixed-point log, from
        // which the apply pass takes the same coordinate)
        if constexpr (!PLANE) {
            if (plane_out) GroupIO<IN_DT>::store_plane(im, r, c, n, vec, PREC ? qv : Lv);
        }
    };
    if constexpr (PLANE) {
        walk_tile<IN_DT, true>(im, t, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
            group_fn(false, r, c, n, vec, Lv, nullptr);
        });
    } else if (IN_DT == DC_U8 && precise) {  // the raw codes are needed
        walk_tile<IN_DT, false, true>(im, t, be,
                                      [&](int r, int c, int n, bool vec, float (&Lv)[G], const uint32_t (&w)[12])
                                          __attribute__((always_inline)) {
                                              group_fn(true, r, c, n, vec, Lv, &w);
                                          });
    } else {
        walk_tile<IN_DT, false>(im, t, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
            group_fn(false, r, c, n, vec, Lv, nullptr);
        });
    }
    cta_sync();
    unsigned long long* H = reinterpret_cast<unsigned long long*>(P.ws + im.ws_hist);
    const int J0 = t.c0 / s;
    for (int k = threadIdx.x; k < nbx * B; k += kThreads) {
        const int blk = k / B, j = k - blk * B;
        const int e = blk * BS + j;
        const unsigned long long fprev = j > 0 ? S.fs[e - 1] : 0u;
        const unsigned long long h = ((unsigned long long)S.cnt[e] << 20) - S.fs[e] + fprev;
        unsigned long long* q = &H[((size_t)I * im.Wb + (J0 + blk)) * B + j];
        if (bc_ok(q, 8, P.ws, P.ws_bytes, BC_WS)) *q = h;
    }
}

// ------------------------------------------------ phase: window sums and CDF --
// Tile: block row I, block columns [t.c0, t.c1).
// The block tables of an image: in its local frame-sequence record (after the
// 256-byte header) when it has one, else in the workspace after its block histograms.
template <int CAP>
__device__ __forceinline__ float* local_tables(const DcBatch<CAP>& P, const DcImage& im)
{
    if (im.lvs) return reinterpret_cast<float*>(im.lvs + sizeof(DcVideoLocalHead));
    return reinterpret_cast<float*>(P.ws + im.ws_hist + align_up((int64_t)im.Hb * im.Wb * P.bins * 8, 256));
}

// Bounds check of an access to an image's block tables (bounds-checked build).
template <int CAP>
__device__ __forceinline__ bool tables_ok(const DcBatch<CAP>& P, const DcImage& im, const void* p, int64_t bytes)
{
    return im.lvs ? bc_ok(p, bytes, P.lvs_buf, P.lvs_bytes, BC_WS) : bc_ok(p, bytes, P.ws, P.ws_bytes, BC_WS);
}

template <int CAP>
__device__ void tile_cdf(const DcBatch<CAP>& P, const DcImage& im, const DcImgCtrl* ic, int I, int lt,
                         const TileRect& t, unsigned char* smem)
{
    SmemCdf& S = *reinterpret_cast<SmemCdf*>(smem);
    const int B = P.bins, R = P.radius, Hb = im.Hb, Wb = im.Wb;
    const unsigned long long* H = reinterpret_cast<const unsigned long long*>(P.ws + im.ws_hist);
    float* E = local_tables(P, im);
    // a local frame sequence: the record carries this frame's own log range (its
    // statistics or fused pass accumulated it) and counts the frame
    if (im.lvs && lt == 0 && threadIdx.x == 0) {
        DcVideoLocalHead* h = reinterpret_cast<DcVideoLocalHead*>(im.lvs);
        if (!P.ldr) {
            h->vmax = (int)(ld_cg_u32(&ic->lmax_ord) ^ 0x80000000u);
            h->vmin = (int)(~ld_cg_u32(&ic->lmin_nord) ^ 0x80000000u);
        }
        h->frames = P.phase_kind[0] == PK_VIDEO_L ? h->frames + 1 : 1;
    }
    const int i0 = max(0, I - R), i1 = min(Hb - 1, I + R);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int J0 = t.c0;
    const int lo = max(0, J0 - R), hi = min(Wb, t.c1 + R);
    const int ncol = hi - lo;
    // column sums over the window's block rows: a warp per staged column and a lane
    // per bin (B <= 32), three columns per round so that their loads are in flight
    // together (the 16 + 2R columns of a default tile take one round); no integer
    // division
    {
        constexpr int NW = kThreads / 32, NC = 3;
        const size_t rs = (size_t)Wb * B;
        if (lane < B) {
            for (int c0 = warp; c0 < ncol; c0 += NC * NW) {
                // column c0 + h NW sits h NW B entries after column c0
                const unsigned long long* q = H + ((size_t)i0 * Wb + lo + c0) * B + lane;
                bool has[NC];
                unsigned long long v[NC];
#pragma unroll
                for (int h = 0; h < NC; ++h) {
                    has[h] = c0 + h * NW < ncol;
                    v[h] = 0ull;
                }
#pragma unroll 5
                for (int I2 = i0; I2 <= i1; ++I2, q += rs) {
#pragma unroll
                    for (int h = 0; h < NC; ++h) {
                        const unsigned long long* qh = q + h * NW * B;
                        v[h] += (has[h] && bc_ok(qh, 8, P.ws, P.ws_bytes, BC_WS)) ? ld_cg_u64(qh) : 0ull;
                    }
                }
#pragma unroll
                for (int h = 0; h < NC; ++h)
                    if (has[h]) S.v[(c0 + h * NW) * B + lane] = v[h];
            }
        }
    }
    cta_sync();
    const int nout = t.c1 - t.c0;
    for (int o = warp; o < nout; o += (kThreads / 32)) {
        const int J = J0 + o;
        unsigned long long w = 0ull;
        if (lane < B) {
            const int a = max(0, J - R), b = min(Wb - 1, J + R);
            for (int jj = a; jj <= b; ++jj) w += S.v[(jj - lo) * B + lane];
        }
        // inclusive scan over bins
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += u;
        }
        const unsigned long long total = __shfl_sync(0xffffffffu, w, 31);
        float* e = E + ((size_t)I * Wb + J) * (B + 1);
        if (!tables_ok(P, im, e, (int64_t)(B + 1) * 4)) continue;
        if (lane < B) e[lane + 1] = __ull2float_rn(w) / __ull2float_rn(total);
        if (lane == 0) e[0] = 0.0f;
    }
}

// ------------------------------------------------------- phase: local apply --
// The tile's block row and its neighbours' cumulative tables are staged as
// (F at the start of bin j, F(j+1) - F(j)) pairs, so each of the four block curves
// costs one 64-bit shared load and one FMA.  The bilinear geometry is tabulated
// once per tile: per column the table slot of its left block and its weight, per
// row the slot row of its upper block and its weight.
// PL: 0 recomputes L from RGB, 1 reads the plane, 2 recomputes L and writes the
// colour reconstruction (interleaved RGB output).
template <int IN_DT, int PL, int CAP>
__device__ void tile_apply_local(const DcBatch<CAP>& P, const DcImage& im, const TileRect& t, int I,
                                 const Beta& be, const Derived& d, unsigned char* smem)
{
    constexpr bool PLANE = PL == 1, COLOR = PL == 2;
    constexpr int G = InT<IN_DT>::G;
    constexpr int kColGroups = (kLocMaxCols + 16) / G;  // column-table stride between a group's entries
    static_assert((kLocMaxCols + 16) % G == 0, "column table splits into G rows");
    constexpr bool ldr = IN_DT == DC_U8;  // u = L; otherwise the fixed-point log coordinate
    SmemApplyL& S = *reinterpret_cast<SmemApplyL*>(smem);
    const int s = P.block_s, B = P.bins, Hb = im.Hb, Wb = im.Wb;
    const int nbx = (t.c1 - t.c0 + s - 1) / s;
    const int J0 = t.c0 / s;
    const int W2 = nbx + 2, B1 = B + 1;
    // slot stride 8 (mod 16) pairs: the same or a nearby bin of neighbouring blocks
    // lands 16 banks away (lanes of a warp read neighbouring blocks' curves at
    // similar bins)
    constexpr int SB = kTabSlot;
    const float* E = local_tables(P, im);
    {
        static_assert(DC_MAX_BINS <= 32, "one lane per bin");
        // one warp per slot column and lane j per bin, two columns per
        // round: the twelve L2 loads of a round are in flight together
        constexpr int NW = kThreads / 32;
        const int j = threadIdx.x & 31, w = threadIdx.x >> 5;
        int rowoff[3];
#pragma unroll
        for (int sr = 0; sr < 3; ++sr) rowoff[sr] = min(max(I - 1 + sr, 0), Hb - 1) * Wb;
        if (j < B) {
            for (int sc0 = w; sc0 < W2; sc0 += 2 * NW) {
                float e0[2][3], e1[2][3];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int sc = sc0 + h * NW;
                    const int J2 = min(max(J0 - 1 + sc, 0), Wb - 1);
#pragma unroll
                    for (int sr = 0; sr < 3; ++sr) {
                        const float* e = E + (size_t)(rowoff[sr] + J2) * B1 + j;
                        const bool ok = sc < W2 && tables_ok(P, im, e, 8);
                        e0[h][sr] = ok ? ld_cg_f(e) : 0.0f;
                        e1[h][sr] = ok ? ld_cg_f(e + 1) : 0.0f;
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int sc = sc0 + h * NW;
                    if (sc < W2) {
#pragma unroll
                        for (int sr = 0; sr < 3; ++sr)
                            S.tab[sr * kTabRow + sc * SB + j] = make_float2(e0[h][sr], e1[h][sr] - e0[h][sr]);
                    }
                }
            }
        }
    }
    // bilinear geometry: nominal block centres ((J + 1/2) s); a pixel at x + 1/2
    // lies between the centres of blocks floor(x/s - 1/2) and the next
    const float inv_s = 1.0f / (float)s;
    // (a ragged group's lanes past the tile read the last column's entry)
    for (int k = threadIdx.x; k < t.c1 - t.c0 + G; k += kThreads) {
        const float fx = fmaf((float)(min(t.c0 + k, t.c1 - 1)) + 0.5f, inv_s, -0.5f);
        const float flx = floorf(fx);
        S.col[(k % G) * kColGroups + k / G] = make_int2(((int)flx - (J0 - 1)) * SB, __float_as_int(fx - flx));
    }
    for (int k = threadIdx.x; k < t.r1 - t.r0; k += kThreads) {
        const float fy = fmaf((float)(t.r0 + k) + 0.5f, inv_s, -0.5f);
        const float fly = floorf(fy);
        S.row[k] = make_int2(((int)fly - (I - 1)) * kTabRow, __float_as_int(fy - fly));
    }
    const float delta = P.delta, Bf = (float)B, alpha = P.alpha;
    constexpr int WSB = kTabRow;
    const bool precise = ldr && (im.flags & IF_UPRECISE) != 0;
    cta_sync();
    // CM, how a pixel's value gives its bin coordinate: 0 u = L (8-bit input), 1 the
    // precise 8-bit coordinate as int32 bits, 2 the HDR fixed-point log (from the plane)
    // or L (recomputed from RGB)
    auto body = [&](auto alpha_one, auto out_dt, auto cm) {
        constexpr int CM = decltype(cm)::value;
        // output values of one group in place
        auto curve_fn = [&](int r, int c, float (&Lv)[G]) __attribute__((always_inline)) {
            const int2 ri = S.row[r - t.r0];
            const float2* rowp = S.tab + ri.x;
            const float wy = __int_as_float(ri.y);
            const int2* colp = S.col + (c - t.c0) / G;  // entry k of the group at colp[k * kColGroups]
#pragma unroll
            for (int k = 0; k < G; ++k) {
                // bin j and position tt in it: from u = L (8-bit input) or exactly from
                // a fixed-point coordinate (precise 8-bit, HDR)
                int j;
                float tt, u = 0.0f;
                if constexpr (CM == 0) {
                    u = fminf(fmaxf(Lv[k], 0.0f), 1.0f);
                    const float Bu = Bf * u;
                    const float jf = fminf(__fadd_rd(Bu, 8388608.0f), 8388608.0f + (float)(B - 1));  // 2^23 + floor
                    j = (int)(__float_as_uint(jf) - 0x4B000000u);
                    tt = Bu - (jf - 8388608.0f);
                } else {
                    // the bin coordinate of the histogram pass: the precise 8-bit one, the
                    // HDR one from the fixed-point log the plane keeps, or from L
                    uint32_t q;
                    if constexpr (CM == 1)
                        q = __float_as_uint(Lv[k]);
                    else
                        q = PLANE ? bin_coord<kLocTS>(__float_as_int(Lv[k]), d) : coord_of<kLocTS>(Lv[k], false, delta, d);
                    const uint32_t jq = min(q >> kLocTS, (uint32_t)(B - 1));
                    j = (int)jq;
                    // (q - j 2^24) / 2^24 in [0, 1] through the float bit pattern of 1 + x
                    tt = __uint_as_float(0x3F800000u + ((q - (jq << kLocTS)) >> (kLocTS - 23))) - 1.0f;
                    if constexpr (!decltype(alpha_one)::value) u = (float)q * (1.0f / (Bf * (float)(1u << kLocTS)));
                }
                const int2 ci = colp[k * kColGroups];
                const float wx = __int_as_float(ci.y);
                const float2* p = rowp + ci.x + j;
                const float2 a = p[0], b = p[SB], cc = p[WSB], dd = p[WSB + SB];
                const float f00 = fmaf(tt, a.y, a.x), f01 = fmaf(tt, b.y, b.x);
                const float f10 = fmaf(tt, cc.y, cc.x), f11 = fmaf(tt, dd.y, dd.x);
                const float top = fmaf(wx, f01 - f00, f00);
                const float bot = fmaf(wx, f11 - f10, f10);
                const float F = fmaf(wy, bot - top, top);
                if constexpr (decltype(alpha_one)::value) {
                    Lv[k] = F;
                } else {
                    Lv[k] = fmaf(alpha, F - u, u);
                }
            }
        };
        if constexpr (PLANE) {
            walk_block_patches_plane<IN_DT, decltype(out_dt)::value>(im, t, s, curve_fn);
        } else if constexpr (COLOR) {
            const float cs = P.color_s;
            const bool s_one = P.color_s_one != 0;
            walk_block_patches<IN_DT, false, true>(
                im, t, s, be, [&](int r, int c, int n, bool vec, float (&Lv)[G], const uint32_t (&w)[12])
                                  __attribute__((always_inline)) {
                    float y[G], o[3 * G];
                    if constexpr (CM == 1) {
                        ucoord_group<IN_DT>(w, n, be, B, y);
                    } else {
#pragma unroll
                        for (int k = 0; k < G; ++k) y[k] = Lv[k];
                    }
                    curve_fn(r, c, y);
                    GroupIO<IN_DT>::color_values(w, Lv, y, be, cs, s_one, o);
                    GroupIO<IN_DT>::store_rgb(im, r, c, n, vec, o);
                });
        } else if constexpr (CM == 1) {
            walk_block_patches<IN_DT, false, true>(
                im, t, s, be, [&](int r, int c, int n, bool vec, float (&Lv)[G], const uint32_t (&w)[12])
                                  __attribute__((always_inline)) {
                    ucoord_group<IN_DT>(w, n, be, B, Lv);
                    curve_fn(r, c, Lv);
                    GroupIO<IN_DT>::store(im, r, c, n, vec, Lv);
                });
        } else {
            walk_block_patches<IN_DT, false>(im, t, s, be,
                                             [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
                                                 curve_fn(r, c, Lv);
                                                 GroupIO<IN_DT>::store(im, r, c, n, vec, Lv);
                                             });
        }
    };
    // alpha = 1, the output type (plane-reading pass) and the coordinate mode as
    // compile-time constants of the pixel loop
    auto by_cm = [&](auto alpha_one, auto out_dt) {
        if constexpr (ldr) {
            if (precise)
                body(alpha_one, out_dt, std::integral_constant<int, 1>{});
            else
                body(alpha_one, out_dt, std::integral_constant<int, 0>{});
        } else {
            body(alpha_one, out_dt, std::integral_constant<int, 2>{});
        }
    };
    auto by_out = [&](auto alpha_one) {
        if constexpr (!PLANE) {
            by_cm(alpha_one, std::integral_constant<int, DC_F32>{});  // (the store dispatches itself)
        } else {
            if (im.out_dt == DC_U8)
                by_cm(alpha_one, std::integral_constant<int, DC_U8>{});
            else if (im.out_dt == DC_F16)
                by_cm(alpha_one, std::integral_constant<int, DC_F16>{});
            else
                by_cm(alpha_one, std::integral_constant<int, DC_F32>{});
        }
    };
    if (alpha == 1.0f)
        by_out(std::true_type{});
    else
        by_out(std::false_type{});
}

// ------------------------------------------------- phase: local frame sequence --
// Staging of the tables of block row I and its neighbours (value, slope pairs) and
// of the tile's bilinear geometry, as the apply pass does it.
template <int IN_DT, int CAP>
__device__ __forceinline__ void stage_curves(const DcBatch<CAP>& P, const DcImage& im, const TileRect& t, int I,
                                             SmemApplyL& S)
{
    constexpr int G = InT<IN_DT>::G;
    constexpr int kColGroups = (kLocMaxCols + 16) / G;
    constexpr int NW = kThreads / 32;
    const int s = P.block_s, B = P.bins, Hb = im.Hb, Wb = im.Wb;
    const int nbx = (t.c1 - t.c0 + s - 1) / s;
    const int J0 = t.c0 / s;
    const int W2 = nbx + 2, B1 = B + 1;
    const float* E = local_tables(P, im);
    const int j = threadIdx.x & 31, w = threadIdx.x >> 5;
    int rowoff[3];
#pragma unroll
    for (int sr = 0; sr < 3; ++sr) rowoff[sr] = min(max(I - 1 + sr, 0), Hb - 1) * Wb;
    if (j < B) {
        for (int sc = w; sc < W2; sc += NW) {
            const int J2 = min(max(J0 - 1 + sc, 0), Wb - 1);
#pragma unroll
            for (int sr = 0; sr < 3; ++sr) {
                const float* e = E + (size_t)(rowoff[sr] + J2) * B1 + j;
                const bool ok = tables_ok(P, im, e, 8);
                const float e0 = ok ? ld_cg_f(e) : 0.0f, e1 = ok ? ld_cg_f(e + 1) : 0.0f;
                S.tab[sr * kTabRow + sc * kTabSlot + j] = make_float2(e0, e1 - e0);
            }
        }
    }
    const float inv_s = 1.0f / (float)s;
    for (int k = threadIdx.x; k < t.c1 - t.c0 + G; k += kThreads) {
        const float fx = fmaf((float)(min(t.c0 + k, t.c1 - 1)) + 0.5f, inv_s, -0.5f);
        const float flx = floorf(fx);
        S.col[(k % G) * kColGroups + k / G] = make_int2(((int)flx - (J0 - 1)) * kTabSlot, __float_as_int(fx - flx));
    }
    for (int k = threadIdx.x; k < t.r1 - t.r0; k += kThreads) {
        const float fy = fmaf((float)(t.r0 + k) + 0.5f, inv_s, -0.5f);
        const float fly = floorf(fy);
        S.row[k] = make_int2(((int)fly - (I - 1)) * kTabRow, __float_as_int(fy - fly));
    }
}

// One pass per frame of a running local sequence: the tile stages the previous
// frame's tables of its block row and neighbours, then every pixel (RGB read once)
// goes into the tent histograms of its block (this frame's tables, built by the next
// pass) and through the bilinear blend of the staged curves (the output).  HDR
// coordinates are taken in the carried range, clamped; the frame's own range is
// accumulated for the next frame.
template <int IN_DT, bool COLOR, int CAP>
__device__ void tile_video_local(const DcBatch<CAP>& P, const DcImage& im, DcImgCtrl* ic, const TileRect& t, int I,
                                 const Beta& be, const Derived& d, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    constexpr int kColGroups = (kLocMaxCols + 16) / G;
    constexpr bool ldr = IN_DT == DC_U8;
    SmemApplyL& S = *reinterpret_cast<SmemApplyL*>(smem);
    SmemBlockH& Hs = *reinterpret_cast<SmemBlockH*>(smem + sizeof(SmemApplyL));
    const int s = P.block_s, B = P.bins;
    const int nbx = (t.c1 - t.c0 + s - 1) / s;
    const int BS = blockh_stride(B);
    stage_curves<IN_DT>(P, im, t, I, S);
    for (int k = threadIdx.x; k < nbx * BS; k += kThreads) {
        Hs.cnt[k] = 0u;
        Hs.fs[k] = 0u;
    }
    const float delta = P.delta, Bf = (float)B, alpha = P.alpha, scale = Bf * 1048576.0f;
    const bool alpha_one = alpha == 1.0f;
    const int xmax = (B - 1) << 20;
    const uint32_t magic = P.s_magic;
    const bool group_in_block = magic != 0u && s % G == 0;
    const bool precise = ldr && (im.flags & IF_UPRECISE) != 0;
    int qmin = INT_MAX, qmax = INT_MIN;
    cta_sync();
    // PREC: the precise 8-bit coordinate (a literal at each inlined call)
    auto group_fn = [&](bool PREC, int r, int c, int n, bool vec, float (&Lv)[G], const uint32_t (*wp)[12])
                        __attribute__((always_inline)) {
        uint32_t q[G];  // coordinate t = bins u in 2^-24 units (precise 8-bit, HDR)
        if (PREC) {
            float qf[G];
            ucoord_group<IN_DT>(*wp, n, be, B, qf);
#pragma unroll
            for (int k = 0; k < G; ++k) q[k] = __float_as_uint(qf[k]);
        } else if (!ldr) {
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const int v = ln_q24(Lv[k] + delta);
                if (k < n) {
                    qmin = min(qmin, v);
                    qmax = max(qmax, v);
                }
                q[k] = bin_coord_clamped<kLocTS>(v, d);
            }
        }
        // tent histograms (run-length merged shared atomics, as the histogram pass)
        const int blk0 = group_in_block ? (int)__umulhi((uint32_t)(c - t.c0), magic) : 0;
        int cur = -1;
        uint32_t rc = 0u, rf = 0u;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            if (k < n) {
                int x;
                if (ldr && !PREC)
                    x = min(max(__float2int_rn(fmaf(fminf(fmaxf(Lv[k], 0.0f), 1.0f), scale, -524288.0f)), 0), xmax);
                else
                    x = min(max(((int)q[k] - (1 << (kLocTS - 1)) + 8) >> (kLocTS - 20), 0), xmax);
                int blk = blk0;
                if (!group_in_block) {
                    const uint32_t off = (uint32_t)(c + k - t.c0);
                    blk = magic ? (int)__umulhi(off, magic) : (int)off;
                }
                const int key = blk * BS + (x >> 20);
                const uint32_t f = (uint32_t)x & 0xFFFFFu;
                if (key == cur) {
                    ++rc;
                    rf += f;
                } else {
                    if (cur >= 0) {
                        atomicAdd(&Hs.cnt[cur], rc);
                        atomicAdd(&Hs.fs[cur], rf);
                    }
                    cur = key;
                    rc = 1u;
                    rf = f;
                }
            }
        }
        if (cur >= 0) {
            atomicAdd(&Hs.cnt[cur], rc);
            atomicAdd(&Hs.fs[cur], rf);
        }
        // the previous frame's curves (bilinear blend, as the apply pass)
        float Lk[COLOR ? G : 1];  // colour output: the luminance, for the channel ratios
        if constexpr (COLOR) {
#pragma unroll
            for (int k = 0; k < G; ++k) Lk[k] = Lv[k];
        }
        const int2 ri = S.row[r - t.r0];
        const float2* rowp = S.tab + ri.x;
        const float wy = __int_as_float(ri.y);
        const int2* colp = S.col + (c - t.c0) / G;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            int j;
            float tt, u;
            if (ldr && !PREC) {
                u = fminf(fmaxf(Lv[k], 0.0f), 1.0f);
                const float Bu = Bf * u;
                const float jf = fminf(__fadd_rd(Bu, 8388608.0f), 8388608.0f + (float)(B - 1));
                j = (int)(__float_as_uint(jf) - 0x4B000000u);
                tt = Bu - (jf - 8388608.0f);
            } else {
                const uint32_t jq = min(q[k] >> kLocTS, (uint32_t)(B - 1));
                j = (int)jq;
                tt = __uint_as_float(0x3F800000u + ((q[k] - (jq << kLocTS)) >> (kLocTS - 23))) - 1.0f;
                u = (float)q[k] * (1.0f / (Bf * (float)(1u << kLocTS)));
            }
            const int2 ci = colp[k * kColGroups];
            const float wx = __int_as_float(ci.y);
            const float2* p = rowp + ci.x + j;
            const float2 a = p[0], b = p[kTabSlot], cc = p[kTabRow], dd = p[kTabRow + kTabSlot];
            const float f00 = fmaf(tt, a.y, a.x), f01 = fmaf(tt, b.y, b.x);
            const float f10 = fmaf(tt, cc.y, cc.x), f11 = fmaf(tt, dd.y, dd.x);
            const float top = fmaf(wx, f01 - f00, f00);
            const float bot = fmaf(wx, f11 - f10, f10);
            const float F = fmaf(wy, bot - top, top);
            Lv[k] = alpha_one ? F : fmaf(alpha, F - u, u);
        }
        if constexpr (COLOR) {
            float o[3 * G];
            GroupIO<IN_DT>::color_values(*wp, Lk, Lv, be, P.color_s, P.color_s_one != 0, o);
            GroupIO<IN_DT>::store_rgb(im, r, c, n, vec, o);
        } else {
            GroupIO<IN_DT>::store(im, r, c, n, vec, Lv);
        }
    };
    if (precise || COLOR) {  // the raw samples are needed
        walk_block_patches<IN_DT, false, true>(im, t, s, be,
                                               [&](int r, int c, int n, bool vec, float (&Lv)[G], const uint32_t (&w)[12])
                                                   __attribute__((always_inline)) {
                                                       if (precise)
                                                           group_fn(true, r, c, n, vec, Lv, &w);
                                                       else
                                                           group_fn(false, r, c, n, vec, Lv, &w);
                                                   });
    } else {
        walk_block_patches<IN_DT, false>(im, t, s, be, [&](int r, int c, int n, bool vec, float (&Lv)[G])
                                                            __attribute__((always_inline)) {
                                                                group_fn(false, r, c, n, vec, Lv, nullptr);
                                                            });
    }
    cta_sync();
    // this frame's block histograms (the next pass builds the tables from them)
    unsigned long long* H = reinterpret_cast<unsigned long long*>(P.ws + im.ws_hist);
    const int J0 = t.c0 / s;
    for (int k = threadIdx.x; k < nbx * B; k += kThreads) {
        const int blk = k / B, j = k - blk * B;
        const int e = blk * BS + j;
        const unsigned long long fprev = j > 0 ? Hs.fs[e - 1] : 0u;
        const unsigned long long h = ((unsigned long long)Hs.cnt[e] << 20) - Hs.fs[e] + fprev;
        unsigned long long* qh = &H[((size_t)I * im.Wb + (J0 + blk)) * B + j];
        if (bc_ok(qh, 8, P.ws, P.ws_bytes, BC_WS)) *qh = h;
    }
    // HDR: this frame's own range, for the next frame
    if constexpr (!ldr) {
        __shared__ int s_min[kThreads / 32], s_max[kThreads / 32];
        qmin = __reduce_min_sync(0xffffffffu, qmin);
        qmax = __reduce_max_sync(0xffffffffu, qmax);
        if ((threadIdx.x & 31) == 0) {
            s_min[threadIdx.x >> 5] = qmin;
            s_max[threadIdx.x >> 5] = qmax;
        }
        cta_sync();
        if (threadIdx.x == 0) {
            int mn = INT_MAX, mx = INT_MIN;
            for (int w = 0; w < kThreads / 32; ++w) {
                mn = min(mn, s_min[w]);
                mx = max(mx, s_max[w]);
            }
            if (mx >= mn) {
                atomicMax(&ic->lmax_ord, (uint32_t)mx ^ 0x80000000u);
                atomicMax(&ic->lmin_nord, ~((uint32_t)mn ^ 0x80000000u));
            }
        }
    }
}

// ------------------------------------------------------------ the engine -----
static_assert(kThreads == 256, "per-bin work uses one consumer thread per histogram bin");

template <int KIND>
struct PassSmem {
    static constexpr size_t value = KIND == PK_STATS || KIND == PK_STATS_LOG || KIND == PK_LOGHIST ? sizeof(SmemStats)
                                    : KIND == PK_VIDEO                     ? sizeof(SmemStats)
                                    : KIND == PK_VIDEO_H                   ? sizeof(SmemStats) + sizeof(SmemApplyG)
                                    : KIND == PK_APPLY_G                   ? sizeof(SmemApplyG) + sizeof(SmemStats)
                                    : KIND == PK_BLOCKH                    ? sizeof(SmemBlockH)
                                    : KIND == PK_CDF                       ? sizeof(SmemCdf)
                                    : KIND == PK_APPLY_L                   ? sizeof(SmemApplyL)
                                    : KIND == PK_VIDEO_L                   ? sizeof(SmemApplyL) + sizeof(SmemBlockH)
                                                                           : 16;
    // above the static limit the pass takes its shared memory dynamically
    static constexpr bool dynamic = value > 40 * 1024;
};

// Frame sequences, after the last tile of the pass: every image's stream estimate
// m <- m + lambda (mu_t - m), mu_t the frame's log-mean from its exact log-sum.
template <int CAP>
__device__ void video_update(const DcBatch<CAP>& P)
{
    constexpr float unit = 1.0f / (float)(1 << kLogFixedShift);
    if (P.mode == DC_HISTEQ) {  // the frame's histogram, pixel count and (HDR) own range
        static_assert(kThreads == 256, "a thread per histogram bin");
        for (int i = 0; i < P.n_img; ++i) {
            const DcImage& im = P.img[i];
            const DcImgCtrl* ic = img_ctrl(P.ctrl, i);
            dc_video_state* st = &P.vstate[P.stats_index[i]];
            st->hist[threadIdx.x] = ld_cg_u32(&ic->hist[threadIdx.x]);
            if (threadIdx.x == 0) {
                st->npix = (long long)im.prow * (long long)im.pcol;
                st->frames += 1;
                if (!P.ldr) {
                    st->vmax = (int)(ld_cg_u32(&ic->lmax_ord) ^ 0x80000000u);
                    st->vmin = (int)(~ld_cg_u32(&ic->lmin_nord) ^ 0x80000000u);
                }
            }
        }
        return;
    }
    for (int i = threadIdx.x; i < P.n_img; i += kThreads) {
        const DcImage& im = P.img[i];
        const long long N = (long long)im.prow * (long long)im.pcol;
        const long long sum = (long long)ld_cg_u64(&img_ctrl(P.ctrl, i)->logsum);
        const long long q = sum / N, rem = sum - q * N;
        const float mu = (__ll2float_rn(q) + __ll2float_rn(rem) / __ll2float_rn(N)) * unit;
        dc_video_state* st = &P.vstate[P.stats_index[i]];
        st->m = fmaf(P.lambda, mu - st->m, st->m);
        st->mu_last = mu;
        st->frames += 1;
    }
}

// One pass over all tiles of pass `ph` (kind KIND) of every image in the batch.
// CTAs take tiles round-robin (last-first when the pass re-reads what the previous
// pass just read, so the most recently touched data is still in L2).  PL: for the
// histogram and apply passes 1 = reads the plane, 2 = colour output (apply passes);
// for the statistics passes 1 = only the reduction the call uses.
template <int IN_DT, int OPK, int KIND, int CAP, int PL>
__global__ void __launch_bounds__(kThreads, DC_MIN_CTAS) pass_kernel(const __grid_constant__ DcBatch<CAP> P, int ph)
{
    __shared__ __align__(16) unsigned char smem_static[PassSmem<KIND>::dynamic ? 16 : PassSmem<KIND>::value];
    extern __shared__ __align__(16) unsigned char smem_dynamic[];
    unsigned char* const smem = PassSmem<KIND>::dynamic ? smem_dynamic : smem_static;
    __shared__ Derived s_d;
    const Beta be = {P.beta_r, 1.0f - P.beta_r, P.beta_k, 1.0f - P.beta_k, P.luma};
    const int total = P.seg_start[ph][P.n_img];
    const bool rev = P.reverse[ph] != 0;
    // derived values of the stats pass are needed by every later pass that
    // normalises log luminance or applies the sigmoid
    const bool fixed_log = P.phase_kind[0] == PK_STATS_LOG;
    const bool need_d = KIND != PK_STATS && KIND != PK_STATS_LOG && KIND != PK_CDF && KIND != PK_DECOLOR &&
                        (P.phase_kind[0] == PK_STATS || fixed_log);
    // programmatic dependent launch: let the next pass start launching its CTAs as
    // ours retire, and wait here until the previous pass has completed and its
    // memory is visible
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (P.profile && threadIdx.x == 0) atomicMax(&P.ctrl->prof[PROF_KSTART_NOT], ~globaltimer_ns());
    int cached = -1;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int tt = rev ? total - 1 - t : t;
        int lo = 0, hi = P.n_img - 1;  // image: last one whose first tile is <= tt
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.seg_start[ph][mid] <= tt) lo = mid; else hi = mid - 1;
        }
        const int img = lo, lt = tt - P.seg_start[ph][img];
        const DcImage& im = P.img[img];
        DcImgCtrl* ic = img_ctrl(P.ctrl, img);
        if (need_d && img != cached) {
            if (threadIdx.x == 0)
                s_d = derive(ic, (long long)im.prow * (long long)im.pcol, fixed_log, P.need_logsum != 0,
                             OPK == OPK_LOCAL, P.bins);
            cta_sync();
            cached = img;
        }
        if constexpr (KIND == PK_VIDEO_L) {
            if (img != cached) {  // HDR: coordinates in the range the previous frame left in the record
                if (threadIdx.x == 0 && !P.ldr) {
                    const DcVideoLocalHead* h = reinterpret_cast<const DcVideoLocalHead*>(im.lvs);
                    derive_range(s_d, ld_cg_u32(reinterpret_cast<const uint32_t*>(&h->vmin)),
                                 ld_cg_u32(reinterpret_cast<const uint32_t*>(&h->vmax)), true, P.bins);
                }
                cta_sync();
                cached = img;
            }
        }
        if constexpr (KIND == PK_VIDEO || KIND == PK_VIDEO_H) {
            if (img != cached) {  // the stream's carried estimate (updated only after the pass)
                if (threadIdx.x == 0) {
                    const dc_video_state* vs = &P.vstate[P.stats_index[img]];
                    s_d.mu = ld_cg_f(&vs->m);
                    s_d.exp_mu = expf(s_d.mu);
                    if (P.mode == DC_HISTEQ && !P.ldr)  // coordinates in the previous frame's range
                        derive_range(s_d, (int)ld_cg_u32(reinterpret_cast<const uint32_t*>(&vs->vmin)),
                                     (int)ld_cg_u32(reinterpret_cast<const uint32_t*>(&vs->vmax)), false, 256);
                }
                cta_sync();
                cached = img;
            }
        }
        if (P.profile && threadIdx.x == 0) atomicMax(&ic->t_start_not[ph], ~globaltimer_ns());
        int I;
        const TileRect tr = tile_rect<OPK>(P, im, KIND, lt, I);
        if constexpr (KIND == PK_DECOLOR) {
            constexpr int G = InT<IN_DT>::G;
            consume_tile<IN_DT, false>(im, tr, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) {
                GroupIO<IN_DT>::store(im, r, c, n, vec, Lv);
            });
        } else if constexpr (KIND == PK_STATS) {
            tile_stats<IN_DT, false, PL != 0>(P, im, ic, tr, be, smem);  // (PL: only the log-sum)
        } else if constexpr (KIND == PK_STATS_LOG) {
            tile_stats<IN_DT, true, PL != 0>(P, im, ic, tr, be, smem);  // (PL: only the log range)
        } else if constexpr (KIND == PK_LOGHIST) {
            tile_loghist<IN_DT, PL == 1>(P, im, ic, tr, be, s_d, smem);
        } else if constexpr (KIND == PK_APPLY_G) {
            if (P.stats && lt == 0) write_stats(P, im, ic, img, s_d);
            if (P.vstate && lt == 0) {  // a restarted stream: this frame's statistics start the record
                dc_video_state* st = &P.vstate[P.stats_index[img]];
                if (P.mode == DC_HISTEQ) st->hist[threadIdx.x] = ld_cg_u32(&ic->hist[threadIdx.x]);
                if (threadIdx.x == 0) {
                    st->m = s_d.mu;
                    st->mu_last = s_d.mu;
                    st->frames = 1;
                    st->npix = (long long)im.prow * (long long)im.pcol;
                    st->vmax = (int)(ld_cg_u32(&ic->lmax_ord) ^ 0x80000000u);
                    st->vmin = (int)(~ld_cg_u32(&ic->lmin_nord) ^ 0x80000000u);
                }
            }
            if constexpr (PL == 2)
                tile_apply_global_color<IN_DT>(P, im, ic, tr, be, s_d, smem);
            else
                tile_apply_global<IN_DT, PL == 1>(P, im, ic, tr, be, s_d, smem);
        } else if constexpr (KIND == PK_BLOCKH) {
            tile_blockh<IN_DT, PL == 1>(P, im, tr, I, be, s_d, smem);
        } else if constexpr (KIND == PK_CDF) {
            tile_cdf(P, im, ic, I, lt, tr, smem);
        } else if constexpr (KIND == PK_VIDEO) {
            tile_video<IN_DT, PL == 2>(P, im, ic, tr, be, s_d, smem);
        } else if constexpr (KIND == PK_VIDEO_H) {
            tile_video_histeq<IN_DT, PL == 2>(P, im, ic, &P.vstate[P.stats_index[img]], tr, be, s_d, smem);
        } else if constexpr (KIND == PK_VIDEO_L) {
            tile_video_local<IN_DT, PL == 2>(P, im, ic, tr, I, be, s_d, smem);
        } else {
            tile_apply_local<IN_DT, PL>(P, im, tr, I, be, s_d, smem);
        }
        cta_sync();  // shared memory is reused by the next tile
        if (P.profile && threadIdx.x == 0) {
            atomicMax(&ic->t_end[ph], globaltimer_ns());
            atomicAdd(&P.ctrl->prof[PROF_TILES], 1ull);
        }
    }
    if (P.profile && threadIdx.x == 0) atomicMax(&P.ctrl->prof[PROF_KEND], globaltimer_ns());
    // Self-clearing call: after the last pass the control block is zero again for the
    // next call on this workspace.  Every CTA fences its work on the block and counts
    // itself; the one that counts last clears the block, counter included.  No CTA
    // waits for another.
    // A frame-sequence pass's last CTA also updates every stream's estimate first.
    if ((P.reset_bytes > 0 || KIND == PK_VIDEO || KIND == PK_VIDEO_H) && ph == P.n_phase - 1) {
        __shared__ uint32_t s_last;
        cta_sync();
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = atomicAdd(&P.ctrl->done_ctas, 1u) == gridDim.x - 1 ? 1u : 0u;
        }
        cta_sync();
        if (s_last) {
            __threadfence();
            if constexpr (KIND == PK_VIDEO || KIND == PK_VIDEO_H) {
                video_update(P);
                cta_sync();
            }
            if (P.reset_bytes > 0) {
                uint4* c = reinterpret_cast<uint4*>(P.ctrl);
                for (int i = threadIdx.x; i < P.reset_bytes / 16; i += kThreads) c[i] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
    }
}

template <int IN_DT, int OPK, int KIND, int CAP, int PL>
int launch_one(const void* batch, int ph, LaunchShape ls, void* stream)
{
    const DcBatch<CAP>& b = *reinterpret_cast<const DcBatch<CAP>*>(batch);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ls.grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    if constexpr (PassSmem<KIND>::dynamic) {
        // (once per kernel: allow its dynamic shared memory)
        static const cudaError_t attr_rc = cudaFuncSetAttribute(
            pass_kernel<IN_DT, OPK, KIND, CAP, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassSmem<KIND>::value);
        if (attr_rc != cudaSuccess) return DC_ERR_CUDA;
        cfg.dynamicSmemBytes = PassSmem<KIND>::value;
    }
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = ph > 0 ? 1 : 0;  // the first pass follows the memset
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, pass_kernel<IN_DT, OPK, KIND, CAP, PL>, b, ph) != cudaSuccess) return DC_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? DC_OK : DC_ERR_CUDA;
}

template <int IN_DT, int OPK, int KIND, int CAP, int PL>
int occupancy_one()
{
    int nb = 0;
    if constexpr (PassSmem<KIND>::dynamic) {
        static const cudaError_t attr_rc = cudaFuncSetAttribute(
            pass_kernel<IN_DT, OPK, KIND, CAP, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassSmem<KIND>::value);
        if (attr_rc != cudaSuccess) return 0;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass_kernel<IN_DT, OPK, KIND, CAP, PL>, kThreads,
                                                      PassSmem<KIND>::dynamic ? PassSmem<KIND>::value : 0) != cudaSuccess)
        return 0;
    return nb;
}

// Valid (operation, pass kind, variant) triples, expanded for every batch capacity.
// The variant is 1 = "reads the plane" for the histogram and apply passes (8-bit
// input: only the apply passes) and "lean reduction" for the statistics passes
// (8-bit input has no STATS_LOG pass), 2 = colour output for the apply passes.
#define DC_FOR_EACH_PASS(X)                                                                           \
    X(OPK_DECOLOR, PK_DECOLOR, 0) X(OPK_GLOBAL, PK_STATS, 0) X(OPK_GLOBAL, PK_STATS, 1)              \
        X(OPK_GLOBAL, PK_STATS_LOG, 0) X(OPK_GLOBAL, PK_STATS_LOG, 1) X(OPK_GLOBAL, PK_LOGHIST, 0)    \
        X(OPK_GLOBAL, PK_LOGHIST, 1) X(OPK_GLOBAL, PK_APPLY_G, 0) X(OPK_GLOBAL, PK_APPLY_G, 1)        \
        X(OPK_GLOBAL, PK_APPLY_G, 2) X(OPK_GLOBAL, PK_VIDEO, 0) X(OPK_GLOBAL, PK_VIDEO, 2)            \
        X(OPK_GLOBAL, PK_VIDEO_H, 0) X(OPK_GLOBAL, PK_VIDEO_H, 2)                                     \
        X(OPK_LOCAL, PK_STATS_LOG, 0)                                                                 \
        X(OPK_LOCAL, PK_STATS_LOG, 1) X(OPK_LOCAL, PK_BLOCKH, 0) X(OPK_LOCAL, PK_BLOCKH, 1)           \
        X(OPK_LOCAL, PK_CDF, 0) X(OPK_LOCAL, PK_APPLY_L, 0) X(OPK_LOCAL, PK_APPLY_L, 1)               \
        X(OPK_LOCAL, PK_APPLY_L, 2) X(OPK_LOCAL, PK_VIDEO_L, 0) X(OPK_LOCAL, PK_VIDEO_L, 2)

template <int IN_DT>
int launch_dispatch(const void* batch, int cap, int opk, int kind, int ph, int pl, LaunchShape ls, void* stream)
{
#define DC_CASE(OP, K, PL)                                                                               \
    if constexpr (!PL || IN_DT != DC_U8 || K == PK_APPLY_G || K == PK_APPLY_L || K == PK_STATS || K == PK_VIDEO || \
                  K == PK_VIDEO_L || K == PK_VIDEO_H) {       \
        if (opk == OP && kind == K && pl == PL) {                                                       \
            if (cap == kCapSmall) return launch_one<IN_DT, OP, K, kCapSmall, PL>(batch, ph, ls, stream); \
            if (cap == kCapMid) return launch_one<IN_DT, OP, K, kCapMid, PL>(batch, ph, ls, stream);     \
            if (cap == kCapLarge) return launch_one<IN_DT, OP, K, kCapLarge, PL>(batch, ph, ls, stream); \
        }                                                                                               \
    }
    DC_FOR_EACH_PASS(DC_CASE)
#undef DC_CASE
    return DC_ERR_INVALID_ARG;
}

template <int IN_DT>
int occupancy_dispatch(int cap, int opk, int kind, int pl)
{
#define DC_CASE(OP, K, PL)                                                                 \
    if constexpr (!PL || IN_DT != DC_U8 || K == PK_APPLY_G || K == PK_APPLY_L || K == PK_STATS || K == PK_VIDEO || \
                  K == PK_VIDEO_L || K == PK_VIDEO_H) { \
        if (opk == OP && kind == K && pl == PL) {                                         \
            if (cap == kCapSmall) return occupancy_one<IN_DT, OP, K, kCapSmall, PL>(); \
            if (cap == kCapMid) return occupancy_one<IN_DT, OP, K, kCapMid, PL>();     \
            if (cap == kCapLarge) return occupancy_one<IN_DT, OP, K, kCapLarge, PL>(); \
        }                                                                                 \
    }
    DC_FOR_EACH_PASS(DC_CASE)
#undef DC_CASE
    return 0;
}

// Bounds-check flags of this translation unit's kernels (read and cleared); -1 when
// the library was built without checks.
template <int IN_DT>
int bounds_take(uint32_t* flags)
{
#ifdef DC_BOUNDS_CHECK
    unsigned int v = 0u, z = 0u;
    if (cudaMemcpyFromSymbol(&v, g_bounds_flags, sizeof(v)) != cudaSuccess ||
        cudaMemcpyToSymbol(g_bounds_flags, &z, sizeof(z)) != cudaSuccess)
        return DC_ERR_CUDA;
    *flags = v;
    return DC_OK;
#else
    *flags = 0u;
    return -1;
#endif
}

// The batch descriptor travels in kernel parameter space (limit 32764 bytes).
static_assert(sizeof(DcBatch<kCapLarge>) <= 32764, "batch descriptor exceeds kernel parameter space");

}  // namespace dc
