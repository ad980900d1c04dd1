// Engine kernel body: tile queue, producer warp (TMA streaming), consumer warps
// (per-phase tile work).  Included by one translation unit per input sample type.
#pragma once

#include "dc_pipe.cuh"

namespace dc {

struct TileRect {
    int r0, r1, c0, c1;
};

// ------------------------------------------------------------ tile geometry ---
template <int OPK, int CAP>
__device__ __forceinline__ int cdf_cols_tiles(const DcImage& im)
{
    return (im.Wb + kCdfChunk - 1) / kCdfChunk;
}

template <int OPK, int CAP>
__device__ __forceinline__ int phase_tiles(const DcBatch<CAP>& P, const DcImage& im, int kind)
{
    if constexpr (OPK == OPK_LOCAL) {
        return kind == PK_CDF ? im.Hb * cdf_cols_tiles<OPK, CAP>(im) : im.Hb * im.tiles_x_loc;
    } else {
        return ((im.rows + P.tile_rows - 1) / P.tile_rows) * im.tiles_x;
    }
}

// Rectangle of tile lt of a phase; for the local operator also its block row I
// (and, for the CDF phase, its first block column J0 in tr.c0).
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
            const int ncc = cdf_cols_tiles<OPK, CAP>(im);
            I = lt / ncc;
            tr.r0 = tr.r1 = 0;
            tr.c0 = (lt - I * ncc) * kCdfChunk;
            tr.c1 = min(tr.c0 + kCdfChunk, im.Wb);
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

// Phases after the first read the f32 plane when the image keeps one.
__device__ __forceinline__ bool from_plane(const DcImage& im, int kind)
{
    return (im.flags & IF_LPLANE) != 0 && kind != PK_STATS && kind != PK_DECOLOR;
}

// ----------------------------------------------------------------- producer ---
// Streams the tile's full groups into the stage ring, in the chunk order the
// consumers use.  Returns false when a wait ran out.
template <int IN_DT, int CAP>
__device__ bool produce_tile(const DcBatch<CAP>& P, PipeSmem<IN_DT>& ps, Ring& data, const DcImage& im,
                             const TileRect& t, bool plane)
{
    using PS = PipeSmem<IN_DT>;
    constexpr int G = InT<IN_DT>::G, ESZ = InT<IN_DT>::ESZ, SG = PS::kGroups;
    const ChunkGeo g = chunk_geo<SG>(t.r0, t.r1, t.c0, t.c1, G, (im.flags & IF_VEC) != 0);
    if (g.nchunks == 0) return true;
    const int bpp = plane ? 4 : 3 * ESZ;
    const int bpg = G * bpp;
    const uint8_t* base = (plane ? im.out : im.in) + (int64_t)t.c0 * bpp;
    const int64_t stride = plane ? im.out_stride : im.in_stride;
    if (plane) fence_proxy_async_global();
    ChunkCursor<SG> cur;
    cur.start(g, t.r0);
    for (int k = 0; k < g.nchunks; ++k) {
        if (!mbar_test_wait(&ps.empty[data.idx], data.parity ^ 1u)) {
            const unsigned long long t0 = P.profile ? globaltimer_ns() : 0ull;
            if (!mbar_wait_slow(&ps.empty[data.idx], data.parity ^ 1u, P.err, P.timeout_ns)) return false;
            if (P.profile) atomicAdd(&P.ctrl->prof[PROF_EMPTY_WAIT], globaltimer_ns() - t0);
        }
        unsigned char* dst = ps.stage[data.idx];
        unsigned long long* full = &ps.full[data.idx];
        if (g.ngv <= SG) {
            const int rows = min(g.rpc, t.r1 - cur.row);
            const uint32_t row_bytes = (uint32_t)(g.ngv * bpg);
            mbar_arrive_expect_tx(full, row_bytes * (uint32_t)rows);
            const uint8_t* src = base + (int64_t)cur.row * stride;
            for (int j = 0; j < rows; ++j, src += stride) tma_load_1d(dst + ((j << g.lg) * bpg), src, row_bytes, full);
        } else {
            const int ng = min(SG, g.ngv - cur.g0);
            const uint32_t bytes = (uint32_t)(ng * bpg);
            mbar_arrive_expect_tx(full, bytes);
            tma_load_1d(dst, base + (int64_t)cur.row * stride + (int64_t)cur.g0 * bpg, bytes, full);
        }
        cur.next(g);
        data.advance(PS::kStages);
    }
    return true;
}

// mu, lmin, lmax from the exact integer accumulators of a finished stats pass.
__device__ __forceinline__ Derived derive(const DcImgCtrl* ic, long long N)
{
    Derived d;
    const long long sum = (long long)ld_cg_u64(&ic->logsum);
    const long long q = sum / N, rem = sum - q * N;
    d.mu = (__ll2float_rn(q) + __ll2float_rn(rem) / __ll2float_rn(N)) * (1.0f / (float)(1 << kLogFixedShift));
    d.exp_mu = expf(d.mu);
    d.lmin = ord_dec(~ld_cg_u32(&ic->lmin_nord));
    d.lmax = ord_dec(ld_cg_u32(&ic->lmax_ord));
    d.inv_range = d.lmax > d.lmin ? 1.0f / (d.lmax - d.lmin) : 0.0f;
    return d;
}

// One lane of the producer warp: pulls tiles from the queue (one ahead), waits
// for the phases a tile depends on, hands the tile to the consumers and streams
// its pixels.
template <int IN_DT, int OPK, int CAP>
__device__ void producer_loop(const DcBatch<CAP>& P, PipeSmem<IN_DT>& ps)
{
    Ring data{0u, 0u}, tring{0u, 0u};
    int next = (int)atomicAdd(&P.ctrl->next_tile, 1u);
    int sg_i = 0;
    // image whose phases [0, ready_p) are known complete, with its derived values
    int ready_img = -1, ready_p = 0;
    Derived ready_d = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    for (;;) {
        TileMsg m;
        m.tile = -1;
        int kind = PK_CDF;
        const int tile = next;
        if (tile < P.total_tiles && ld_relaxed_u32(P.err) == 0) {
            next = (int)atomicAdd(&P.ctrl->next_tile, 1u);  // overlaps this tile
            while (sg_i + 1 < P.n_seg && P.seg[sg_i + 1].start <= tile) ++sg_i;
            const DcSegment sg = P.seg[sg_i];
            const int nt = (sg_i + 1 < P.n_seg ? P.seg[sg_i + 1].start : P.total_tiles) - sg.start;
            int lt = tile - sg.start;
            if (sg.reverse) lt = nt - 1 - lt;
            const int img = sg.img, p = sg.phase;
            const DcImage& im = P.img[img];
            DcImgCtrl* ic = img_ctrl(P.ctrl, img);
            bool ok = true;
            const int known = img == ready_img ? ready_p : 0;
            if (p > known) {
                // every earlier phase of this image must have published all its tiles
                const unsigned long long t0 = P.profile ? globaltimer_ns() : 0ull;
                for (int q = p - 1; q >= known && ok; --q)
                    ok = wait_count(&ic->done[q], (uint32_t)phase_tiles<OPK>(P, im, P.phase_kind[q]), P.err,
                                    P.timeout_ns) == 0;
                if (P.profile) atomicAdd(&P.ctrl->prof[PROF_DEP_WAIT], globaltimer_ns() - t0);
                if (ok) {
                    if (img != ready_img && P.phase_kind[0] == PK_STATS)
                        ready_d = derive(ic, (long long)im.prow * (long long)im.pcol);
                    ready_img = img;
                    ready_p = p;
                }
            }
            if (ok) {
                m.tile = tile;
                m.lt = lt;
                m.img = img;
                m.p = p;
                m.d = ready_d;
                kind = P.phase_kind[p];
            }
        }
        if (!mbar_wait(&ps.tempty[tring.idx], tring.parity ^ 1u, P.err, P.timeout_ns)) return;
        ps.msg[tring.idx] = m;
        mbar_arrive(&ps.tfull[tring.idx]);
        tring.advance(kTileRing);
        if (m.tile < 0) return;
        if (kind != PK_CDF) {
            const DcImage& im = P.img[m.img];
            int I;
            const TileRect tr = tile_rect<OPK>(P, im, kind, m.lt, I);
            if (!produce_tile<IN_DT>(P, ps, data, im, tr, from_plane(im, kind))) return;
        }
    }
}

// ---------------------------------------------------------------- consumers ---
// Visit every group of a tile: full groups from the stage ring, then the scalar
// remainder (ragged row ends, or every group of an unaligned image) from global
// memory.  f(r, c, n, vec, v) gets the group's source values v: the luminance
// (from RGB) or the plane values.
template <int IN_DT, int CAP, class F>
__device__ __forceinline__ void consume_tile(const DcBatch<CAP>& P, PipeSmem<IN_DT>& ps, Ring& data,
                                             const DcImage& im, const TileRect& t, bool plane, const Beta& be, F&& f)
{
    using PS = PipeSmem<IN_DT>;
    constexpr int G = InT<IN_DT>::G, SG = PS::kGroups, GPT = PS::kGPT;
    const bool vec_img = (im.flags & IF_VEC) != 0;
    const ChunkGeo g = chunk_geo<SG>(t.r0, t.r1, t.c0, t.c1, G, vec_img);
    const int tid = threadIdx.x;
    ChunkCursor<SG> cur;
    cur.start(g, t.r0);
    for (int k = 0; k < g.nchunks; ++k) {
        bool ok = mbar_test_wait(&ps.full[data.idx], data.parity);
        if (!ok) {
            const unsigned long long t0 = (P.profile && tid == 0) ? globaltimer_ns() : 0ull;
            ok = mbar_wait_slow(&ps.full[data.idx], data.parity, P.err, P.timeout_ns);
            if (P.profile && tid == 0) atomicAdd(&P.ctrl->prof[PROF_DATA_WAIT], globaltimer_ns() - t0);
        }
        int r[GPT], c[GPT];
        bool valid[GPT];
        float v[GPT][G];
        uint32_t w[GPT][12];
#pragma unroll
        for (int i = 0; i < GPT; ++i) {
            const int sidx = tid + i * kThreads;
            valid[i] = cur.slot(g, t.r1, t.c0, G, sidx, r[i], c[i]) && ok;
            if (valid[i]) {
                if (plane) {
                    const float4* q = reinterpret_cast<const float4*>(ps.stage[data.idx] + sidx * (4 * G));
#pragma unroll
                    for (int j = 0; j < G / 4; ++j) {
                        const float4 x = q[j];
                        v[i][4 * j] = x.x;
                        v[i][4 * j + 1] = x.y;
                        v[i][4 * j + 2] = x.z;
                        v[i][4 * j + 3] = x.w;
                    }
                } else {
                    const uint4* q = reinterpret_cast<const uint4*>(ps.stage[data.idx] + sidx * 48);
                    const uint4 a = q[0], b = q[1], d = q[2];
                    w[i][0] = a.x; w[i][1] = a.y; w[i][2] = a.z; w[i][3] = a.w;
                    w[i][4] = b.x; w[i][5] = b.y; w[i][6] = b.z; w[i][7] = b.w;
                    w[i][8] = d.x; w[i][9] = d.y; w[i][10] = d.z; w[i][11] = d.w;
                }
            }
        }
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&ps.empty[data.idx]);
        data.advance(PS::kStages);
        cur.next(g);
#pragma unroll
        for (int i = 0; i < GPT; ++i) {
            if (valid[i]) {
                if (!plane) GroupIO<IN_DT>::decode(w[i], be, v[i]);
                f(r[i], c[i], G, true, v[i]);
            }
        }
    }
    const int c_rem = t.c0 + g.ngv * G;
    if (c_rem < t.c1) {
        // scalar remainder, rows spread over threads, groups at multiples of G
        const int gpr = (t.c1 - c_rem + G - 1) / G;
        const int nslots = (t.r1 - t.r0) * gpr;
        for (int s = tid; s < nslots; s += kThreads) {
            const int rr = s / gpr;
            const int r = t.r0 + rr;
            const int c = c_rem + (s - rr * gpr) * G;
            const int n = min(G, t.c1 - c);
            float v[G];
            if (plane)
                GroupIO<IN_DT>::from_plane(im, r, c, n, false, v);
            else
                GroupIO<IN_DT>::luminance(im, r, c, n, false, be, v);
            f(r, c, n, false, v);
        }
    }
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
    consumer_sync();
    uint32_t off = 0;
    for (int w = 0; w < warp; ++w) off += scratch[w];
    consumer_sync();
    return v + off;
}

// ------------------------------------------------------------- phase: stats --
template <int IN_DT, int CAP>
__device__ void tile_stats(const DcBatch<CAP>& P, PipeSmem<IN_DT>& ps, Ring& data, const DcImage& im, DcImgCtrl* ic,
                           const TileRect& t, const Beta& be, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    SmemStats& S = *reinterpret_cast<SmemStats*>(smem);
    const bool want_hist = P.need_gray_hist != 0;
    const bool plane_out = (im.flags & IF_LPLANE) != 0;
    const bool plane_log = (im.flags & IF_PLANE_LOG) != 0;
    if (want_hist) {
        for (int b = threadIdx.x; b < 256; b += kThreads) S.hist[b] = 0;
        consumer_sync();
    }
    long long acc = 0;
    float vmin = INFINITY, vmax = -INFINITY;
    const float delta = P.delta;
    consume_tile<IN_DT>(P, ps, data, im, t, false, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
        float v[G];
#pragma unroll
        for (int k = 0; k < G; ++k) {
            if (k < n) {
                v[k] = ln_fast(Lv[k] + delta);
                vmin = fminf(vmin, v[k]);
                vmax = fmaxf(vmax, v[k]);
                if (want_hist) atomicAdd(&S.hist[quant_u8(Lv[k])], 1u);
            } else {
                v[k] = 0.0f;
            }
        }
        if (plane_out) GroupIO<IN_DT>::store(im, r, c, n, vec, plane_log ? v : Lv);
        acc += __float2ll_rn(pairwise_sum<G>(v) * (float)(1 << kLogFixedShift));
    });
    acc = warp_sum_ll(acc);
    vmin = warp_min(vmin);
    vmax = warp_max(vmax);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        S.wsum[warp] = acc;
        S.wmin[warp] = vmin;
        S.wmax[warp] = vmax;
    }
    consumer_sync();
    if (threadIdx.x == 0) {
        long long s = 0;
        float mn = INFINITY, mx = -INFINITY;
        for (int w = 0; w < kConsumerWarps; ++w) {
            s += S.wsum[w];
            mn = fminf(mn, S.wmin[w]);
            mx = fmaxf(mx, S.wmax[w]);
        }
        atomicAdd(&ic->logsum, (unsigned long long)s);
        if (mx >= mn) {
            atomicMax(&ic->lmax_ord, ord_enc(mx));
            atomicMax(&ic->lmin_nord, ~ord_enc(mn));
        }
    }
    if (want_hist) {
        for (int b = threadIdx.x; b < 256; b += kThreads)
            if (S.hist[b]) atomicAdd(&ic->hist[b], S.hist[b]);
    }
}

// ---------------------------------------------------------- phase: log hist --
template <int IN_DT, int CAP>
__device__ void tile_loghist(const DcBatch<CAP>& P, PipeSmem<IN_DT>& ps, Ring& data, const DcImage& im, DcImgCtrl* ic,
                             const TileRect& t, const Beta& be, const Derived& d, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    SmemStats& S = *reinterpret_cast<SmemStats*>(smem);
    for (int b = threadIdx.x; b < 256; b += kThreads) S.hist[b] = 0;
    const bool plane = from_plane(im, PK_LOGHIST);
    const bool is_log = (im.flags & IF_PLANE_LOG) != 0;
    const float delta = P.delta;
    consumer_sync();
    consume_tile<IN_DT>(P, ps, data, im, t, plane, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
#pragma unroll
        for (int k = 0; k < G; ++k)
            if (k < n) {
                const float u = log_u(Lv[k], plane && is_log, delta, d.lmin, d.inv_range);
                atomicAdd(&S.hist[min((int)(256.0f * u), 255)], 1u);
            }
    });
    consumer_sync();
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
template <int IN_DT, int CAP>
__device__ void tile_apply_global(const DcBatch<CAP>& P, PipeSmem<IN_DT>& ps, Ring& data, const DcImage& im,
                                  DcImgCtrl* ic, const TileRect& t, const Beta& be, const Derived& d,
                                  unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    SmemApplyG& S = *reinterpret_cast<SmemApplyG*>(smem);
    const bool plane = from_plane(im, PK_APPLY_G);
    const bool is_log = plane && (im.flags & IF_PLANE_LOG) != 0;
    const float delta = P.delta;
    if (P.mode == DC_SIGMOID) {
        const float mu = d.mu, exp_mu = d.exp_mu, k = P.gain_k;
        const bool one = P.gain_is_one != 0;
        consume_tile<IN_DT>(P, ps, data, im, t, plane, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
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
        consumer_sync();
        const bool ldr = P.ldr != 0;
        consume_tile<IN_DT>(P, ps, data, im, t, plane, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
#pragma unroll
            for (int j = 0; j < G; ++j) {
                if (ldr) {
                    Lv[j] = S.lut[quant_u8(Lv[j])];
                } else {
                    const float u = 256.0f * log_u(Lv[j], is_log, delta, d.lmin, d.inv_range);
                    const int b = min((int)u, 255);
                    const float e0 = S.lut[b], e1 = S.lut[b + 1];
                    Lv[j] = fmaf(u - (float)b, e1 - e0, e0);
                }
            }
            GroupIO<IN_DT>::store(im, r, c, n, vec, Lv);
        });
    }
}

// ---------------------------------------------------- phase: local histograms --
template <int IN_DT, int CAP>
__device__ void tile_blockh(const DcBatch<CAP>& P, PipeSmem<IN_DT>& ps, Ring& data, const DcImage& im,
                            const TileRect& t, int I, const Beta& be, const Derived& d, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    constexpr int kCountShift = 42;
    SmemBlockH& S = *reinterpret_cast<SmemBlockH*>(smem);
    const int s = P.block_s, B = P.bins;
    const int nbx = (t.c1 - t.c0 + s - 1) / s;
    for (int k = threadIdx.x; k < nbx * B; k += kThreads) S.h[k] = 0ull;
    const bool plane = from_plane(im, PK_BLOCKH);
    const bool is_log = plane && (im.flags & IF_PLANE_LOG) != 0;
    const bool ldr = P.ldr != 0;
    const float delta = P.delta, Bf = (float)B;
    const uint32_t magic = P.s_magic;
    consumer_sync();
    consume_tile<IN_DT>(P, ps, data, im, t, plane, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
        int cur = -1;
        unsigned long long acc = 0ull;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            if (k < n) {
                const float u = ldr ? fminf(fmaxf(Lv[k], 0.0f), 1.0f) : log_u(Lv[k], is_log, delta, d.lmin, d.inv_range);
                // tent binning onto bin centres (j + 1/2)/B
                const float x = fmaf(Bf, u, -0.5f);
                int j;
                float f;
                if (x <= 0.0f) {
                    j = 0;
                    f = 0.0f;
                } else if (x >= Bf - 1.0f) {
                    j = B - 1;
                    f = 0.0f;
                } else {
                    j = (int)x;
                    f = x - (float)j;
                }
                const uint32_t off = (uint32_t)(c + k - t.c0);
                const int blk = magic ? (int)__umulhi(off, magic) : (int)off;
                const int key = blk * B + j;
                const unsigned long long val = (1ull << kCountShift) | (unsigned long long)__float2uint_rn(f * 16777216.0f);
                if (key == cur) {
                    acc += val;
                } else {
                    if (cur >= 0) atomicAdd(&S.h[cur], acc);
                    cur = key;
                    acc = val;
                }
            }
        }
        if (cur >= 0) atomicAdd(&S.h[cur], acc);
    });
    consumer_sync();
    // unpack: bin j holds count_j * 2^24 - F_j + F_{j-1}
    const unsigned long long mask = (1ull << kCountShift) - 1ull;
    unsigned long long* H = reinterpret_cast<unsigned long long*>(P.ws + im.ws_hist);
    const int J0 = t.c0 / s;
    for (int k = threadIdx.x; k < nbx * B; k += kThreads) {
        const int blk = k / B, j = k - blk * B;
        const unsigned long long v = S.h[k];
        const unsigned long long Fprev = j > 0 ? (S.h[k - 1] & mask) : 0ull;
        const unsigned long long h = ((v >> kCountShift) << 24) - (v & mask) + Fprev;
        H[((size_t)I * im.Wb + (J0 + blk)) * B + j] = h;
    }
}

// ------------------------------------------------ phase: window sums and CDF --
// Tile: block row I, block columns [t.c0, t.c1).
template <int CAP>
__device__ void tile_cdf(const DcBatch<CAP>& P, const DcImage& im, int I, const TileRect& t, unsigned char* smem)
{
    SmemCdf& S = *reinterpret_cast<SmemCdf*>(smem);
    const int B = P.bins, R = P.radius, Hb = im.Hb, Wb = im.Wb;
    const unsigned long long* H = reinterpret_cast<const unsigned long long*>(P.ws + im.ws_hist);
    float* E = reinterpret_cast<float*>(P.ws + im.ws_hist + align_up((int64_t)Hb * Wb * B * 8, 256));
    const int i0 = max(0, I - R), i1 = min(Hb - 1, I + R);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int J0 = t.c0;
    const int lo = max(0, J0 - R), hi = min(Wb, t.c1 + R);
    const int ncol = hi - lo;
    for (int k = threadIdx.x; k < ncol * B; k += kThreads) {
        const int jj = lo + k / B, j = k % B;
        unsigned long long v = 0ull;
        for (int I2 = i0; I2 <= i1; ++I2) v += ld_cg_u64(&H[((size_t)I2 * Wb + jj) * B + j]);
        S.v[k] = v;
    }
    consumer_sync();
    const int nout = t.c1 - t.c0;
    for (int o = warp; o < nout; o += kConsumerWarps) {
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
        if (lane < B) e[lane + 1] = __ull2float_rn(w) / __ull2float_rn(total);
        if (lane == 0) e[0] = 0.0f;
    }
}

// ------------------------------------------------------- phase: local apply --
template <int IN_DT, int CAP>
__device__ void tile_apply_local(const DcBatch<CAP>& P, PipeSmem<IN_DT>& ps, Ring& data, const DcImage& im,
                                 const TileRect& t, int I, const Beta& be, const Derived& d, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    SmemApplyL& S = *reinterpret_cast<SmemApplyL*>(smem);
    const int s = P.block_s, B = P.bins, Hb = im.Hb, Wb = im.Wb;
    const int nbx = (t.c1 - t.c0 + s - 1) / s;
    const int J0 = t.c0 / s;
    const int W2 = nbx + 2, B1 = B + 1;
    const float* E = reinterpret_cast<const float*>(P.ws + im.ws_hist + align_up((int64_t)Hb * Wb * B * 8, 256));
    for (int k = threadIdx.x; k < 3 * W2 * B1; k += kThreads) {
        const int sr = k / (W2 * B1);
        const int rem = k - sr * W2 * B1;
        const int sc = rem / B1, j = rem - sc * B1;
        const int I2 = min(max(I - 1 + sr, 0), Hb - 1);
        const int J2 = min(max(J0 - 1 + sc, 0), Wb - 1);
        S.tab[k] = ld_cg_f(&E[((size_t)I2 * Wb + J2) * B1 + j]);
    }
    const bool plane = from_plane(im, PK_APPLY_L);
    const bool is_log = plane && (im.flags & IF_PLANE_LOG) != 0;
    const bool ldr = P.ldr != 0;
    const float delta = P.delta, Bf = (float)B, inv_s = 1.0f / (float)s, alpha = P.alpha;
    consumer_sync();
    consume_tile<IN_DT>(P, ps, data, im, t, plane, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
        const float fy = fmaf((float)r + 0.5f, inv_s, -0.5f);
        const float fly = floorf(fy);
        const float wy = fy - fly;
        const int sr0 = (int)fly - (I - 1);
        const float* row0 = S.tab + sr0 * W2 * B1;
        const float* row1 = row0 + W2 * B1;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const float u = ldr ? fminf(fmaxf(Lv[k], 0.0f), 1.0f) : log_u(Lv[k], is_log, delta, d.lmin, d.inv_range);
            const float fx = fmaf((float)(c + k) + 0.5f, inv_s, -0.5f);
            const float flx = floorf(fx);
            const float wx = fx - flx;
            const int sc0 = (int)flx - (J0 - 1);
            const float Bu = Bf * u;
            const int j = min((int)Bu, B - 1);
            const float tt = Bu - (float)j;
            const float* a0 = row0 + sc0 * B1 + j;
            const float* a1 = row1 + sc0 * B1 + j;
            const float f00 = fmaf(tt, a0[1] - a0[0], a0[0]);
            const float f01 = fmaf(tt, a0[B1 + 1] - a0[B1], a0[B1]);
            const float f10 = fmaf(tt, a1[1] - a1[0], a1[0]);
            const float f11 = fmaf(tt, a1[B1 + 1] - a1[B1], a1[B1]);
            const float top = fmaf(wx, f01 - f00, f00);
            const float bot = fmaf(wx, f11 - f10, f10);
            const float F = fmaf(wy, bot - top, top);
            Lv[k] = fmaf(alpha, F - u, u);
        }
        GroupIO<IN_DT>::store(im, r, c, n, vec, Lv);
    });
}

// ------------------------------------------------------------ the engine -----
static_assert(kThreads == 256, "per-bin work uses one consumer thread per histogram bin");

template <int OPK>
struct PhaseSmem {
    static constexpr size_t value = OPK == OPK_GLOBAL ? sizeof(SmemApplyG) + sizeof(SmemStats) : SmemBytes<OPK>::value;
};

template <int IN_DT, int OPK>
constexpr size_t engine_smem_bytes()
{
    return sizeof(PipeSmem<IN_DT>) + PhaseSmem<OPK>::value + 64;
}

template <int IN_DT, int OPK, int CAP>
__device__ void consumer_loop(const DcBatch<CAP>& P, PipeSmem<IN_DT>& ps, unsigned char* smem, int* s_abort)
{
    const Beta be = {P.beta_r, 1.0f - P.beta_r, P.beta_k, 1.0f - P.beta_k};
    Ring data{0u, 0u}, tring{0u, 0u};
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long t0 = P.profile ? globaltimer_ns() : 0ull;
            *s_abort = mbar_wait(&ps.tfull[tring.idx], tring.parity, P.err, P.timeout_ns) ? 0 : 1;
            if (P.profile) atomicAdd(&P.ctrl->prof[PROF_TILE_WAIT], globaltimer_ns() - t0);
        }
        consumer_sync();
        if (*s_abort) return;
        const TileMsg m = ps.msg[tring.idx];
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(&ps.tempty[tring.idx]);
        tring.advance(kTileRing);
        if (m.tile < 0) return;
        const int img = m.img, p = m.p, kind = P.phase_kind[p];
        const DcImage im = P.img[img];  // one copy per tile, not per group
        DcImgCtrl* ic = img_ctrl(P.ctrl, img);
        int I;
        const TileRect tr = tile_rect<OPK>(P, im, kind, m.lt, I);
        if (P.profile && threadIdx.x == 0) atomicMax(&ic->t_start_not[p], ~globaltimer_ns());
        if constexpr (OPK == OPK_DECOLOR) {
            constexpr int G = InT<IN_DT>::G;
            consume_tile<IN_DT>(P, ps, data, im, tr, false, be, [&](int r, int c, int n, bool vec, float (&Lv)[G]) __attribute__((always_inline)) {
                GroupIO<IN_DT>::store(im, r, c, n, vec, Lv);
            });
        } else if constexpr (OPK == OPK_GLOBAL) {
            if (kind == PK_STATS) {
                tile_stats<IN_DT>(P, ps, data, im, ic, tr, be, smem);
            } else if (kind == PK_LOGHIST) {
                tile_loghist<IN_DT>(P, ps, data, im, ic, tr, be, m.d, smem);
            } else {
                if (P.stats && m.lt == 0) write_stats(P, im, ic, img, m.d);
                tile_apply_global<IN_DT>(P, ps, data, im, ic, tr, be, m.d, smem);
            }
        } else {
            if (kind == PK_STATS)
                tile_stats<IN_DT>(P, ps, data, im, ic, tr, be, smem);
            else if (kind == PK_BLOCKH)
                tile_blockh<IN_DT>(P, ps, data, im, tr, I, be, m.d, smem);
            else if (kind == PK_CDF)
                tile_cdf(P, im, I, tr, smem);
            else
                tile_apply_local<IN_DT>(P, ps, data, im, tr, I, be, m.d, smem);
        }
        consumer_sync();
        if (threadIdx.x == 0) {
            if (P.profile) {
                atomicMax(&ic->t_end[p], globaltimer_ns());
                atomicAdd(&P.ctrl->prof[PROF_TILES], 1ull);
            }
            if (!(P.withhold_ready && p == 0)) red_release_add(&ic->done[p], 1u);
        }
    }
}

template <int IN_DT, int OPK, int CAP>
#ifndef DC_MIN_CTAS
#define DC_MIN_CTAS 2
#endif
__global__ void __launch_bounds__(kBlockThreads, DC_MIN_CTAS) engine_kernel(const __grid_constant__ DcBatch<CAP> P)
{
    extern __shared__ __align__(128) unsigned char dsmem[];
    PipeSmem<IN_DT>& ps = *reinterpret_cast<PipeSmem<IN_DT>*>(dsmem);
    unsigned char* phase_smem = dsmem + sizeof(PipeSmem<IN_DT>);
    int* s_abort = reinterpret_cast<int*>(phase_smem + PhaseSmem<OPK>::value);
    if (threadIdx.x == 0) {
        for (int i = 0; i < PipeSmem<IN_DT>::kStages; ++i) {
            mbar_init(&ps.full[i], 1);
            mbar_init(&ps.empty[i], kConsumerWarps);
        }
        for (int i = 0; i < kTileRing; ++i) {
            mbar_init(&ps.tfull[i], 1);
            mbar_init(&ps.tempty[i], kConsumerWarps);
        }
        fence_mbarrier_init();
    }
    if (P.profile && threadIdx.x == 0) atomicMax(&P.ctrl->prof[PROF_KSTART_NOT], ~globaltimer_ns());
    __syncthreads();
    if (threadIdx.x >= kThreads) {
        if (threadIdx.x == kThreads) producer_loop<IN_DT, OPK>(P, ps);
        return;
    }
    consumer_loop<IN_DT, OPK>(P, ps, phase_smem, s_abort);
    if (P.profile && threadIdx.x == 0) atomicMax(&P.ctrl->prof[PROF_KEND], globaltimer_ns());
}

template <int IN_DT, int OPK, int CAP>
int launch_one(const void* batch, LaunchShape ls, void* stream)
{
    static unsigned long long attr_set = 0ull;  // one bit per device
    constexpr size_t smem = engine_smem_bytes<IN_DT, OPK>();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DC_ERR_CUDA;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(__atomic_load_n(&attr_set, __ATOMIC_ACQUIRE) & bit)) {
        if (cudaFuncSetAttribute(engine_kernel<IN_DT, OPK, CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return DC_ERR_CUDA;
        __atomic_fetch_or(&attr_set, bit, __ATOMIC_RELEASE);
    }
    const DcBatch<CAP>& b = *reinterpret_cast<const DcBatch<CAP>*>(batch);
    engine_kernel<IN_DT, OPK, CAP><<<ls.grid, kBlockThreads, smem, (cudaStream_t)stream>>>(b);
    return cudaGetLastError() == cudaSuccess ? DC_OK : DC_ERR_CUDA;
}

template <int IN_DT, int OPK, int CAP>
int occupancy_one()
{
    constexpr size_t smem = engine_smem_bytes<IN_DT, OPK>();
    if (cudaFuncSetAttribute(engine_kernel<IN_DT, OPK, CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, engine_kernel<IN_DT, OPK, CAP>, kBlockThreads, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

template <int IN_DT>
int launch_dispatch(const void* batch, int cap, int opk, LaunchShape ls, void* stream)
{
#define DC_CASE(OP, C) \
    if (opk == OP && cap == C) return launch_one<IN_DT, OP, C>(batch, ls, stream);
    DC_CASE(OPK_DECOLOR, kCapSmall)
    DC_CASE(OPK_DECOLOR, kCapMid)
    DC_CASE(OPK_DECOLOR, kCapLarge)
    DC_CASE(OPK_GLOBAL, kCapSmall)
    DC_CASE(OPK_GLOBAL, kCapMid)
    DC_CASE(OPK_GLOBAL, kCapLarge)
    DC_CASE(OPK_LOCAL, kCapSmall)
    DC_CASE(OPK_LOCAL, kCapMid)
    DC_CASE(OPK_LOCAL, kCapLarge)
#undef DC_CASE
    return DC_ERR_INVALID_ARG;
}

template <int IN_DT>
int occupancy_dispatch(int cap, int opk)
{
#define DC_CASE(OP, C) \
    if (opk == OP && cap == C) return occupancy_one<IN_DT, OP, C>();
    DC_CASE(OPK_DECOLOR, kCapSmall)
    DC_CASE(OPK_DECOLOR, kCapMid)
    DC_CASE(OPK_DECOLOR, kCapLarge)
    DC_CASE(OPK_GLOBAL, kCapSmall)
    DC_CASE(OPK_GLOBAL, kCapMid)
    DC_CASE(OPK_GLOBAL, kCapLarge)
    DC_CASE(OPK_LOCAL, kCapSmall)
    DC_CASE(OPK_LOCAL, kCapMid)
    DC_CASE(OPK_LOCAL, kCapLarge)
#undef DC_CASE
    return 0;
}

// The batch descriptor travels in kernel parameter space (limit 32764 bytes).
static_assert(sizeof(DcBatch<kCapLarge>) <= 32764, "batch descriptor exceeds kernel parameter space");

}  // namespace dc
