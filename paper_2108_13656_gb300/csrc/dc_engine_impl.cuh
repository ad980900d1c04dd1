// Engine kernel body: tile queue, phase dispatch, per-phase tile work and the
// end-of-phase finalisation.  Included by one translation unit per input type.
#pragma once

#include "dc_engine.cuh"

namespace dc {

struct TileRect {
    int r0, r1, c0, c1;
};

// Iterate the G-pixel groups of a tile: f(r, c, n, vec).  Groups start at
// columns that are multiples of G from the row start, whatever the tile shape.
template <int IN_DT, class F>
__device__ __forceinline__ void for_each_group(const DcImage& im, const TileRect& t, F&& f)
{
    constexpr int G = InT<IN_DT>::G;
    const int gpr = (t.c1 - t.c0 + G - 1) / G;
    const int nslots = (t.r1 - t.r0) * gpr;
    const bool vec_img = (im.flags & IF_VEC) != 0;
    for (int s = threadIdx.x; s < nslots; s += kThreads) {
        const int rr = s / gpr;
        const int r = t.r0 + rr;
        const int c = t.c0 + (s - rr * gpr) * G;
        const int n = min(G, t.c1 - c);
        f(r, c, n, vec_img && n == G);
    }
}

template <int IN_DT>
__device__ __forceinline__ void load_L(const DcImage& im, int r, int c, int n, bool vec, bool plane,
                                       const Beta& be, float (&Lv)[InT<IN_DT>::G])
{
    if (plane)
        GroupIO<IN_DT>::from_plane(im, r, c, n, vec, Lv);
    else
        GroupIO<IN_DT>::luminance(im, r, c, n, vec, be, Lv);
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

// Block-wide inclusive scan of one uint32 per thread (kThreads values).
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t* scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) scratch[warp] = v;
    __syncthreads();
    uint32_t off = 0;
    for (int w = 0; w < warp; ++w) off += scratch[w];
    __syncthreads();
    return v + off;
}

// ------------------------------------------------------------- phase: stats --
template <int IN_DT, int CAP>
__device__ void tile_stats(const DcBatch<CAP>& P, const DcImage& im, DcImgCtrl* ic, const TileRect& t,
                           const Beta& be, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    SmemStats& S = *reinterpret_cast<SmemStats*>(smem);
    const bool want_hist = P.need_gray_hist != 0;
    const bool plane_out = (im.flags & IF_LPLANE) != 0;
    if (want_hist) {
        for (int b = threadIdx.x; b < 256; b += kThreads) S.hist[b] = 0;
        __syncthreads();
    }
    long long acc = 0;
    float vmin = INFINITY, vmax = -INFINITY;
    const float delta = P.delta;
    for_each_group<IN_DT>(im, t, [&](int r, int c, int n, bool vec) {
        float Lv[G];
        GroupIO<IN_DT>::luminance(im, r, c, n, vec, be, Lv);
        if (plane_out) GroupIO<IN_DT>::store(im, r, c, n, vec, Lv);
        float v[G];
#pragma unroll
        for (int k = 0; k < G; ++k) {
            if (k < n) {
                v[k] = logf(Lv[k] + delta);
                vmin = fminf(vmin, v[k]);
                vmax = fmaxf(vmax, v[k]);
                if (want_hist) atomicAdd(&S.hist[quant_u8(Lv[k])], 1u);
            } else {
                v[k] = 0.0f;
            }
        }
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
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        float mn = INFINITY, mx = -INFINITY;
        for (int w = 0; w < kThreads / 32; ++w) {
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

template <int CAP>
__device__ void finalize_stats(const DcBatch<CAP>& P, const DcImage& im, DcImgCtrl* ic, int img,
                               unsigned char* smem)
{
    SmemStats& S = *reinterpret_cast<SmemStats*>(smem);
    const long long N = (long long)im.prow * (long long)im.pcol;
    __shared__ float s_mu, s_lmin, s_lmax;
    if (threadIdx.x == 0) {
        const long long sum = (long long)ld_cg_u64(&ic->logsum);
        const long long q = sum / N, rem = sum - q * N;
        const float mu = (__ll2float_rn(q) + __ll2float_rn(rem) / __ll2float_rn(N)) * (1.0f / (float)(1 << kLogFixedShift));
        const float lmin = ord_dec(~ld_cg_u32(&ic->lmin_nord));
        const float lmax = ord_dec(ld_cg_u32(&ic->lmax_ord));
        ic->mu = mu;
        ic->lmin = lmin;
        ic->lmax = lmax;
        ic->exp_mu = expf(mu);
        ic->inv_range = lmax > lmin ? 1.0f / (lmax - lmin) : 0.0f;
        s_mu = mu;
        s_lmin = lmin;
        s_lmax = lmax;
    }
    __syncthreads();
    const bool ldr_histeq = P.ldr && P.mode == DC_HISTEQ && P.block_s == 0;
    if (ldr_histeq || (P.stats && P.ldr)) {
        const uint32_t h = ld_cg_u32(&ic->hist[threadIdx.x]);
        const uint32_t cum = block_incl_scan(h, S.scan);
        if (ldr_histeq) ic->lut[threadIdx.x] = __uint2float_rn(cum) / __ll2float_rn(N);
        if (P.stats) P.stats[P.stats_index[img]].hist[threadIdx.x] = h;
    } else if (P.stats) {
        P.stats[P.stats_index[img]].hist[threadIdx.x] = 0u;
    }
    if (P.stats && threadIdx.x == 0) {
        dc_global_stats* st = &P.stats[P.stats_index[img]];
        st->mu = s_mu;
        st->logmin = s_lmin;
        st->logmax = s_lmax;
        st->reserved0 = 0.0f;
        st->logsum_fixed = (int64_t)ld_cg_u64(&ic->logsum);
        st->npix = N;
    }
}

// ---------------------------------------------------------- phase: log hist --
template <int IN_DT, int CAP>
__device__ void tile_loghist(const DcBatch<CAP>& P, const DcImage& im, DcImgCtrl* ic, const TileRect& t,
                             const Beta& be, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    SmemStats& S = *reinterpret_cast<SmemStats*>(smem);
    for (int b = threadIdx.x; b < 256; b += kThreads) S.hist[b] = 0;
    const float lmin = ld_cg_f(&ic->lmin), inv_range = ld_cg_f(&ic->inv_range), delta = P.delta;
    const bool plane = (im.flags & IF_LPLANE) != 0;
    __syncthreads();
    for_each_group<IN_DT>(im, t, [&](int r, int c, int n, bool vec) {
        float Lv[G];
        load_L<IN_DT>(im, r, c, n, vec, plane, be, Lv);
#pragma unroll
        for (int k = 0; k < G; ++k)
            if (k < n) {
                const float u = log_u(Lv[k], delta, lmin, inv_range);
                atomicAdd(&S.hist[min((int)(256.0f * u), 255)], 1u);
            }
    });
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += kThreads)
        if (S.hist[b]) atomicAdd(&ic->hist[b], S.hist[b]);
}

template <int CAP>
__device__ void finalize_loghist(const DcBatch<CAP>& P, const DcImage& im, DcImgCtrl* ic, int img,
                                 unsigned char* smem)
{
    SmemStats& S = *reinterpret_cast<SmemStats*>(smem);
    const long long N = (long long)im.prow * (long long)im.pcol;
    const uint32_t h = ld_cg_u32(&ic->hist[threadIdx.x]);
    const uint32_t cum = block_incl_scan(h, S.scan);
    // edge[b] = (pixels in bins < b) / N
    ic->lut[threadIdx.x] = __uint2float_rn(cum - h) / __ll2float_rn(N);
    if (threadIdx.x == kThreads - 1) ic->lut[256] = 1.0f;
    if (P.stats) P.stats[P.stats_index[img]].hist[threadIdx.x] = h;
}

// ------------------------------------------------------- phase: global apply --
template <int IN_DT, int CAP>
__device__ void tile_apply_global(const DcBatch<CAP>& P, const DcImage& im, DcImgCtrl* ic,
                                  const TileRect& t, const Beta& be, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    SmemApplyG& S = *reinterpret_cast<SmemApplyG*>(smem);
    const bool plane = (im.flags & IF_LPLANE) != 0;
    const float delta = P.delta;
    if (P.mode == DC_SIGMOID) {
        const float mu = ld_cg_f(&ic->mu), exp_mu = ld_cg_f(&ic->exp_mu), k = P.gain_k;
        const bool one = P.gain_is_one != 0;
        for_each_group<IN_DT>(im, t, [&](int r, int c, int n, bool vec) {
            float Lv[G];
            load_L<IN_DT>(im, r, c, n, vec, plane, be, Lv);
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const float x = Lv[j] + delta;
                // y = 1 / (1 + exp(-k (ln x - mu)));  k = 1: y = x / (x + e^mu)
                Lv[j] = one ? x / (x + exp_mu) : 1.0f / (1.0f + expf(-k * (logf(x) - mu)));
            }
            GroupIO<IN_DT>::store(im, r, c, n, vec, Lv);
        });
    } else {
        const int nlut = P.ldr ? 256 : 257;
        for (int b = threadIdx.x; b < nlut; b += kThreads) S.lut[b] = ld_cg_f(&ic->lut[b]);
        const float lmin = ld_cg_f(&ic->lmin), inv_range = ld_cg_f(&ic->inv_range);
        __syncthreads();
        const bool ldr = P.ldr != 0;
        for_each_group<IN_DT>(im, t, [&](int r, int c, int n, bool vec) {
            float Lv[G];
            load_L<IN_DT>(im, r, c, n, vec, plane, be, Lv);
#pragma unroll
            for (int j = 0; j < G; ++j) {
                if (ldr) {
                    Lv[j] = S.lut[quant_u8(Lv[j])];
                } else {
                    const float u = 256.0f * log_u(Lv[j], delta, lmin, inv_range);
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
__device__ void tile_blockh(const DcBatch<CAP>& P, const DcImage& im, DcImgCtrl* ic, const TileRect& t,
                            int I, const Beta& be, unsigned char* smem)
{
    constexpr int G = InT<IN_DT>::G;
    constexpr int kCountShift = 42;
    SmemBlockH& S = *reinterpret_cast<SmemBlockH*>(smem);
    const int s = P.block_s, B = P.bins;
    const int nbx = (t.c1 - t.c0 + s - 1) / s;
    for (int k = threadIdx.x; k < nbx * B; k += kThreads) S.h[k] = 0ull;
    const bool plane = (im.flags & IF_LPLANE) != 0;
    const bool ldr = P.ldr != 0;
    float lmin = 0.0f, inv_range = 0.0f;
    if (!ldr) {
        lmin = ld_cg_f(&ic->lmin);
        inv_range = ld_cg_f(&ic->inv_range);
    }
    const float delta = P.delta, Bf = (float)B;
    __syncthreads();
    for_each_group<IN_DT>(im, t, [&](int r, int c, int n, bool vec) {
        float Lv[G];
        load_L<IN_DT>(im, r, c, n, vec, plane, be, Lv);
        int cur = -1;
        unsigned long long acc = 0ull;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            if (k < n) {
                const float u = ldr ? fminf(fmaxf(Lv[k], 0.0f), 1.0f) : log_u(Lv[k], delta, lmin, inv_range);
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
                const int key = ((c + k - t.c0) / s) * B + j;
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
    __syncthreads();
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
template <int CAP>
__device__ void tile_cdf(const DcBatch<CAP>& P, const DcImage& im, int I, unsigned char* smem)
{
    SmemCdf& S = *reinterpret_cast<SmemCdf*>(smem);
    const int B = P.bins, R = P.radius, Hb = im.Hb, Wb = im.Wb;
    const unsigned long long* H = reinterpret_cast<const unsigned long long*>(P.ws + im.ws_hist);
    float* E = reinterpret_cast<float*>(P.ws + im.ws_hist + align_up((int64_t)Hb * Wb * B * 8, 256));
    const int i0 = max(0, I - R), i1 = min(Hb - 1, I + R);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int J0 = 0; J0 < Wb; J0 += kCdfChunk) {
        const int lo = max(0, J0 - R), hi = min(Wb, J0 + kCdfChunk + R);
        const int ncol = hi - lo;
        for (int k = threadIdx.x; k < ncol * B; k += kThreads) {
            const int jj = lo + k / B, j = k % B;
            unsigned long long v = 0ull;
            for (int I2 = i0; I2 <= i1; ++I2) v += ld_cg_u64(&H[((size_t)I2 * Wb + jj) * B + j]);
            S.v[k] = v;
        }
        __syncthreads();
        const int nout = min(kCdfChunk, Wb - J0);
        for (int o = warp; o < nout; o += kThreads / 32) {
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
        __syncthreads();
    }
}

// ------------------------------------------------------- phase: local apply --
template <int IN_DT, int CAP>
__device__ void tile_apply_local(const DcBatch<CAP>& P, const DcImage& im, DcImgCtrl* ic,
                                 const TileRect& t, int I, const Beta& be, unsigned char* smem)
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
    const bool plane = (im.flags & IF_LPLANE) != 0;
    const bool ldr = P.ldr != 0;
    float lmin = 0.0f, inv_range = 0.0f;
    if (!ldr) {
        lmin = ld_cg_f(&ic->lmin);
        inv_range = ld_cg_f(&ic->inv_range);
    }
    const float delta = P.delta, Bf = (float)B, inv_s = 1.0f / (float)s, alpha = P.alpha;
    __syncthreads();
    for_each_group<IN_DT>(im, t, [&](int r, int c, int n, bool vec) {
        float Lv[G];
        load_L<IN_DT>(im, r, c, n, vec, plane, be, Lv);
        const float fy = fmaf((float)r + 0.5f, inv_s, -0.5f);
        const float fly = floorf(fy);
        const float wy = fy - fly;
        const int sr0 = (int)fly - (I - 1);
        const float* row0 = S.tab + sr0 * W2 * B1;
        const float* row1 = row0 + W2 * B1;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const float u = ldr ? fminf(fmaxf(Lv[k], 0.0f), 1.0f) : log_u(Lv[k], delta, lmin, inv_range);
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
static_assert(kThreads == 256, "per-bin finalisation uses one thread per histogram bin");

template <int IN_DT, int OPK, int CAP>
__global__ void __launch_bounds__(kThreads) engine_kernel(const __grid_constant__ DcBatch<CAP> P)
{
    __shared__ __align__(16) unsigned char smem[SmemBytes<OPK>::value];
    __shared__ int s_tile, s_flag;
    const Beta be = {P.beta_r, 1.0f - P.beta_r, P.beta_k, 1.0f - P.beta_k};
    for (;;) {
        if (threadIdx.x == 0) {
            int tt = -1;
            if (ld_relaxed_u32(P.err) == 0) tt = (int)atomicAdd(&P.ctrl->next_tile, 1u);
            s_tile = tt;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0 || tile >= P.total_tiles) break;
        // segment holding this tile: largest sg with seg[sg].start <= tile
        int lo = 0, hi = P.n_seg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.seg[mid].start <= tile) lo = mid; else hi = mid - 1;
        }
        const DcSegment sg = P.seg[lo];
        const int nt = (lo + 1 < P.n_seg ? P.seg[lo + 1].start : P.total_tiles) - sg.start;
        int lt = tile - sg.start;
        if (sg.reverse) lt = nt - 1 - lt;
        const int img = sg.img, p = sg.phase, kind = P.phase_kind[p];
        const DcImage& im = P.img[img];
        DcImgCtrl* ic = img_ctrl(P.ctrl, img);
        if (p > 0) {
            if (threadIdx.x == 0) {
                s_flag = wait_ready(&ic->ready[p - 1], P.err, P.timeout_ns);
                __threadfence();
            }
            __syncthreads();
            const int abort_tile = s_flag;
            __syncthreads();
            if (abort_tile) continue;
        }
        // tile rectangle
        TileRect tr;
        int I = 0;
        if constexpr (OPK == OPK_LOCAL) {
            if (kind != PK_CDF) {
                I = lt / im.tiles_x_loc;
                const int tx = lt - I * im.tiles_x_loc;
                tr.r0 = I * P.block_s;
                tr.r1 = min(tr.r0 + P.block_s, im.prow);
                tr.c0 = tx * P.loc_tile_cols;
                tr.c1 = min(tr.c0 + P.loc_tile_cols, im.pcol);
            } else {
                I = lt;
            }
        } else {
            const int ty = lt / im.tiles_x;
            const int tx = lt - ty * im.tiles_x;
            tr.r0 = ty * P.tile_rows;
            tr.r1 = min(tr.r0 + P.tile_rows, im.rows);
            tr.c0 = tx * P.tile_cols;
            tr.c1 = min(tr.c0 + P.tile_cols, im.cols);
        }
        switch (kind) {
        case PK_DECOLOR:
            if constexpr (OPK == OPK_DECOLOR) {
                for_each_group<IN_DT>(im, tr, [&](int r, int c, int n, bool vec) {
                    float Lv[InT<IN_DT>::G];
                    GroupIO<IN_DT>::luminance(im, r, c, n, vec, be, Lv);
                    GroupIO<IN_DT>::store(im, r, c, n, vec, Lv);
                });
            }
            break;
        case PK_STATS:
            if constexpr (OPK != OPK_DECOLOR) tile_stats<IN_DT>(P, im, ic, tr, be, smem);
            break;
        case PK_LOGHIST:
            if constexpr (OPK == OPK_GLOBAL) tile_loghist<IN_DT>(P, im, ic, tr, be, smem);
            break;
        case PK_APPLY_G:
            if constexpr (OPK == OPK_GLOBAL) tile_apply_global<IN_DT>(P, im, ic, tr, be, smem);
            break;
        case PK_BLOCKH:
            if constexpr (OPK == OPK_LOCAL) tile_blockh<IN_DT>(P, im, ic, tr, I, be, smem);
            break;
        case PK_CDF:
            if constexpr (OPK == OPK_LOCAL) tile_cdf(P, im, I, smem);
            break;
        case PK_APPLY_L:
            if constexpr (OPK == OPK_LOCAL) tile_apply_local<IN_DT>(P, im, ic, tr, I, be, smem);
            break;
        default:
            break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const uint32_t old = atomicAdd(&ic->done[p], 1u);
            s_flag = (old == (uint32_t)nt - 1u);
        }
        __syncthreads();
        if (s_flag) {
            __threadfence();
            if constexpr (OPK != OPK_DECOLOR) {
                if (kind == PK_STATS) finalize_stats(P, im, ic, img, smem);
                if constexpr (OPK == OPK_GLOBAL) {
                    if (kind == PK_LOGHIST) finalize_loghist(P, im, ic, img, smem);
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                if (!(P.withhold_ready && p == 0)) st_release_u32(&ic->ready[p], 1u);
            }
        }
        __syncthreads();
    }
}

template <int IN_DT, int OPK, int CAP>
int launch_one(const void* batch, LaunchShape ls, void* stream)
{
    const DcBatch<CAP>& b = *reinterpret_cast<const DcBatch<CAP>*>(batch);
    engine_kernel<IN_DT, OPK, CAP><<<ls.grid, kThreads, 0, (cudaStream_t)stream>>>(b);
    return cudaGetLastError() == cudaSuccess ? DC_OK : DC_ERR_CUDA;
}

template <int IN_DT, int OPK, int CAP>
int occupancy_one()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, engine_kernel<IN_DT, OPK, CAP>, kThreads, 0) !=
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

}  // namespace dc

namespace dc {
// The batch descriptor travels in kernel parameter space (limit 32764 bytes).
static_assert(sizeof(DcBatch<kCapLarge>) <= 32764, "batch descriptor exceeds kernel parameter space");
}  // namespace dc
