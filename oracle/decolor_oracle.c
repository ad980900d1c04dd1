/*
 * FP64 CPU oracle: colour-temperature decolorization (Eq. 1-6) and the global
 * and local tone-mapping passes the paper applies to the resulting luminance
 * (Sec. III-B-1 and Sec. III-B-2).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header or
 * constant with the CUDA library and it is deliberately plain: one pixel at a
 * time, sequential sums, IEEE double arithmetic, no blocking or reordering
 * beyond what the definitions state.  Build: gcc -O2 -ffp-contract=off -fPIC
 * -shared (no fast-math), so that every operation is a correctly rounded
 * double operation.
 *
 * Readings of points the paper leaves open (each is also pinned in tests):
 *  - black pixel: Eq. 4 and Eq. 5 divide by R+G+B; at R=G=B=0 the luminance is
 *    taken as 0, the continuous extension (0 <= L <= max(R,G,B)).
 *  - decode: 8-bit codes are used as v/255 with no linearisation; binary16 and
 *    binary32 samples are linear radiance used as they are; negative samples
 *    are treated as 0.
 *  - global curve (the "centered sigmoid" of Sec. III-B-1):
 *      y = 1 / (1 + exp(-k (ln(L + delta) - mu))),  mu = mean ln(L + delta).
 *  - global histogram equalisation: 8-bit input bins the 8-bit gray code
 *    q = floor(255 L + 1/2) and maps y = sum_{j<=q} h_j / N (textbook HE);
 *    HDR input bins u = (ln(L+delta) - lmin)/(lmax - lmin) into 256 bins and
 *    maps through the piecewise-linear cumulative histogram.
 *  - local operator (smoothed local-histogram equalisation, Sec. III-B-2, in
 *    the family of Kass and Solomon's smoothed local histogram filters): tent
 *    (linear) binning of u into `bins` bins with centres (j+1/2)/bins, block
 *    histograms over s x s blocks, a (2R+1)^2-block box window truncated at
 *    the image border, per-block cumulative histograms with each bin's mass
 *    spread uniformly over its bin, and bilinear interpolation between the
 *    four nearest nominal block centres ((I+1/2)s, (J+1/2)s), clamped at the
 *    border.  Output alpha*F + (1-alpha)*u.
 *  - comparison channels (Sec. I, Fig. GTMO): MATLAB's rgb2gray weights as the
 *    paper quotes them, and V of HSV = max(R, G, B), on the same decoded samples;
 *    CIE L* / 100 from Rec. 709 relative luminance (D65 white), 8-bit codes decoded
 *    with the sRGB transfer function first (CIELAB is defined on linear light).
 *  - colour reconstruction (colour outputs of Fig. tmo_1 and Fig. GTMO, no formula):
 *    C_out = min(1, y (C_in / L)^s), a black pixel taken as achromatic.
 *  - frame sequences (real-time use, Sec. I; no scheme given): frame t is centred
 *    on the log-mean estimate carried from the frames before it,
 *    m_t = (1 - lambda) m_{t-1} + lambda mu_t, the first frame on its own mu_0.
 *    For the local operator, frame t is mapped through frame t-1's block tables and,
 *    for HDR input, takes its coordinates in frame t-1's log range (both one frame
 *    behind); its own tables, from those coordinates, and its own range go to frame
 *    t+1.  The first frame is the local operator on its own.
 * Parity of the tone-mapping parameters (k, delta, s, R, bins, alpha) is
 * unpinned by the paper, which prints none of them; the operators are pinned
 * by closed forms and invariants in the tests instead.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_U8 = 0, OR_F16 = 1, OR_F32 = 2 };

/* IEEE 754 binary16 -> double, straight from the format definition. */
static double or_half_to_double(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int e = (h >> 10) & 31;
    int m = h & 1023;
    double v;
    if (e == 0)
        v = ldexp((double)m, -24);            /* subnormal: m * 2^-24 */
    else if (e == 31)
        v = m ? NAN : INFINITY;
    else
        v = ldexp((double)(m + 1024), e - 25); /* (1 + m/1024) * 2^(e-15) */
    return sign ? -v : v;
}

static double or_sample(const unsigned char* px, int dtype, int c)
{
    double v;
    if (dtype == OR_U8) {
        v = (double)px[c] / 255.0;
    } else if (dtype == OR_F16) {
        uint16_t h;
        memcpy(&h, px + 2 * c, 2);
        v = or_half_to_double(h);
    } else {
        float f;
        memcpy(&f, px + 4 * c, 4);
        v = (double)f;
    }
    if (!(v > 0.0))
        v = 0.0; /* negative (and NaN) samples are treated as black */
    return v;
}

/* Eq. 1-6 for one pixel. */
double oracle_luminance(double R, double G, double B, double beta_R, double beta_k)
{
    double S = R + G + B;
    if (S == 0.0)
        return 0.0;
    double L_WHITE = sqrt((R * R + G * G + B * B) / 3.0);                 /* Eq. 1 */
    double L_B = B;                                                       /* Eq. 2 */
    double L_GR = sqrt(beta_R * R * R + (1.0 - beta_R) * G * G);          /* Eq. 3 */
    double L_WARM = (R / S) * L_GR + (1.0 - R / S) * L_WHITE;             /* Eq. 4 */
    double L_COOL = (1.0 - B / S) * L_B + (B / S) * L_WHITE;              /* Eq. 5 */
    return sqrt(beta_k * L_WARM * L_WARM + (1.0 - beta_k) * L_COOL * L_COOL); /* Eq. 6 */
}

/* Decolorize an interleaved RGB image into a row-major H x W double plane. */
int oracle_decolorize(const void* data, int32_t W, int32_t H, int64_t stride_bytes,
                      int32_t dtype, double beta_R, double beta_k, double* L)
{
    if (W < 0 || H < 0 || dtype < OR_U8 || dtype > OR_F32)
        return 1;
    int esz = dtype == OR_U8 ? 1 : (dtype == OR_F16 ? 2 : 4);
    const unsigned char* base = (const unsigned char*)data;
    for (int32_t y = 0; y < H; ++y) {
        const unsigned char* row = base + (int64_t)y * stride_bytes;
        for (int32_t x = 0; x < W; ++x) {
            const unsigned char* px = row + (int64_t)x * 3 * esz;
            double R = or_sample(px, dtype, 0);
            double G = or_sample(px, dtype, 1);
            double B = or_sample(px, dtype, 2);
            L[(int64_t)y * W + x] = oracle_luminance(R, G, B, beta_R, beta_k);
        }
    }
    return 0;
}

/* Image-wide log statistics: mu = mean ln(L+delta), and its min and max. */
void oracle_log_stats(const double* L, int64_t n, double delta, double* mu, double* lmin,
                      double* lmax)
{
    double sum = 0.0, lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        double v = log(L[i] + delta);
        sum += v;
        if (v < lo) lo = v;
        if (v > hi) hi = v;
    }
    *mu = n > 0 ? sum / (double)n : 0.0;
    *lmin = n > 0 ? lo : 0.0;
    *lmax = n > 0 ? hi : 0.0;
}

/* 8-bit gray code of a luminance in [0, 1]. */
static int or_gray_code(double L)
{
    double q = floor(255.0 * L + 0.5);
    if (q < 0.0) q = 0.0;
    if (q > 255.0) q = 255.0;
    return (int)q;
}

/* Normalised log luminance used by the HDR histogram forms. */
static double or_log_u(double L, double delta, double lmin, double lmax)
{
    if (!(lmax > lmin))
        return 0.5;
    double u = (log(L + delta) - lmin) / (lmax - lmin);
    if (u < 0.0) u = 0.0;
    if (u > 1.0) u = 1.0;
    return u;
}

static int or_u_bin256(double u)
{
    int b = (int)floor(256.0 * u);
    if (b < 0) b = 0;
    if (b > 255) b = 255;
    return b;
}

void oracle_gray_hist(const double* L, int64_t n, uint32_t* hist)
{
    for (int j = 0; j < 256; ++j) hist[j] = 0;
    for (int64_t i = 0; i < n; ++i) hist[or_gray_code(L[i])] += 1;
}

void oracle_log_hist(const double* L, int64_t n, double delta, double lmin, double lmax,
                     uint32_t* hist)
{
    for (int j = 0; j < 256; ++j) hist[j] = 0;
    for (int64_t i = 0; i < n; ++i) hist[or_u_bin256(or_log_u(L[i], delta, lmin, lmax))] += 1;
}

/* Centred sigmoid: y = 1/2 exactly where ln(L+delta) = mu. */
void oracle_tone_sigmoid(const double* L, int64_t n, double k, double delta, double mu, double* y)
{
    for (int64_t i = 0; i < n; ++i)
        y[i] = 1.0 / (1.0 + exp(-k * (log(L[i] + delta) - mu)));
}

/* Textbook 8-bit histogram equalisation on the gray codes. */
void oracle_tone_histeq_ldr(const double* L, int64_t n, const uint32_t* hist, double* y)
{
    double cdf[256];
    double acc = 0.0;
    for (int j = 0; j < 256; ++j) {
        acc += (double)hist[j];
        cdf[j] = acc;
    }
    for (int64_t i = 0; i < n; ++i) y[i] = cdf[or_gray_code(L[i])] / (double)n;
}

/* Piecewise-linear cumulative histogram of the normalised log luminance. */
void oracle_tone_histeq_hdr(const double* L, int64_t n, double delta, double lmin, double lmax,
                            const uint32_t* hist, double* y)
{
    double below[257];
    below[0] = 0.0;
    for (int j = 0; j < 256; ++j) below[j + 1] = below[j] + (double)hist[j];
    for (int64_t i = 0; i < n; ++i) {
        double u = or_log_u(L[i], delta, lmin, lmax);
        int b = or_u_bin256(u);
        double f = 256.0 * u - (double)b;
        y[i] = (below[b] + f * (double)hist[b]) / (double)n;
    }
}

/* Tent binning of u in [0,1] into `bins` bins centred at (j+1/2)/bins. */
static void or_tent(double u, int bins, int* j0, double* w0, int* j1, double* w1)
{
    double x = bins * u - 0.5;
    if (x <= 0.0) {
        *j0 = 0; *w0 = 1.0; *j1 = 0; *w1 = 0.0;
    } else if (x >= bins - 1) {
        *j0 = bins - 1; *w0 = 1.0; *j1 = bins - 1; *w1 = 0.0;
    } else {
        int j = (int)floor(x);
        double f = x - j;
        *j0 = j; *w0 = 1.0 - f; *j1 = j + 1; *w1 = f;
    }
}

/* Cumulative histogram with each bin's mass spread uniformly over its bin. */
static double or_cdf_eval(const double* edge, int bins, double u)
{
    double x = bins * u;
    if (x <= 0.0) return edge[0];
    if (x >= bins) return edge[bins];
    int j = (int)floor(x);
    return edge[j] + (edge[j + 1] - edge[j]) * (x - j);
}

/*
 * Smoothed local-histogram equalisation of a luminance plane.
 * ldr != 0: u = L; otherwise u is the normalised log luminance (lmin, lmax).
 * Returns 0 on success, 1 on bad arguments, 2 on allocation failure.
 */
int oracle_tone_local(const double* L, int32_t W, int32_t H, int32_t ldr, int32_t s,
                      int32_t Rb, int32_t bins, double alpha, double delta, double lmin,
                      double lmax, double* y)
{
    if (W <= 0 || H <= 0 || s <= 0 || Rb < 0 || bins < 1)
        return 1;
    int32_t Hb = (H + s - 1) / s, Wb = (W + s - 1) / s;
    size_t nb = (size_t)Hb * Wb * bins;
    double* h = (double*)calloc(nb, sizeof(double));
    double* edge = (double*)calloc((size_t)Hb * Wb * (bins + 1), sizeof(double));
    double* u = (double*)malloc((size_t)W * H * sizeof(double));
    if (!h || !edge || !u) {
        free(h); free(edge); free(u);
        return 2;
    }
    for (int64_t i = 0; i < (int64_t)W * H; ++i) {
        double v = ldr ? L[i] : or_log_u(L[i], delta, lmin, lmax);
        if (v < 0.0) v = 0.0;
        if (v > 1.0) v = 1.0;
        u[i] = v;
    }
    /* block histograms */
    for (int32_t py = 0; py < H; ++py)
        for (int32_t px = 0; px < W; ++px) {
            int j0, j1;
            double w0, w1;
            or_tent(u[(int64_t)py * W + px], bins, &j0, &w0, &j1, &w1);
            double* hb = h + ((size_t)(py / s) * Wb + (px / s)) * bins;
            hb[j0] += w0;
            hb[j1] += w1;
        }
    /* window sums and per-block cumulative histograms */
    double* win = (double*)malloc(sizeof(double) * bins);
    if (!win) {
        free(h); free(edge); free(u);
        return 2;
    }
    for (int32_t I = 0; I < Hb; ++I)
        for (int32_t J = 0; J < Wb; ++J) {
            for (int j = 0; j < bins; ++j) win[j] = 0.0;
            for (int32_t I2 = I - Rb; I2 <= I + Rb; ++I2) {
                if (I2 < 0 || I2 >= Hb) continue;
                for (int32_t J2 = J - Rb; J2 <= J + Rb; ++J2) {
                    if (J2 < 0 || J2 >= Wb) continue;
                    const double* hb = h + ((size_t)I2 * Wb + J2) * bins;
                    for (int j = 0; j < bins; ++j) win[j] += hb[j];
                }
            }
            double total = 0.0;
            for (int j = 0; j < bins; ++j) total += win[j];
            double* e = edge + ((size_t)I * Wb + J) * (bins + 1);
            double acc = 0.0;
            e[0] = 0.0;
            for (int j = 0; j < bins; ++j) {
                acc += win[j];
                e[j + 1] = acc / total;
            }
        }
    /* bilinear blend of the four nearest block tone curves */
    for (int32_t py = 0; py < H; ++py) {
        double fy = (py + 0.5) / s - 0.5;
        int32_t I0 = (int32_t)floor(fy);
        double wy = fy - I0;
        int32_t I1 = I0 + 1;
        if (I0 < 0) I0 = 0;
        if (I1 < 0) I1 = 0;
        if (I0 > Hb - 1) I0 = Hb - 1;
        if (I1 > Hb - 1) I1 = Hb - 1;
        for (int32_t px = 0; px < W; ++px) {
            double fx = (px + 0.5) / s - 0.5;
            int32_t J0 = (int32_t)floor(fx);
            double wx = fx - J0;
            int32_t J1 = J0 + 1;
            if (J0 < 0) J0 = 0;
            if (J1 < 0) J1 = 0;
            if (J0 > Wb - 1) J0 = Wb - 1;
            if (J1 > Wb - 1) J1 = Wb - 1;
            double up = u[(int64_t)py * W + px];
            double f00 = or_cdf_eval(edge + ((size_t)I0 * Wb + J0) * (bins + 1), bins, up);
            double f01 = or_cdf_eval(edge + ((size_t)I0 * Wb + J1) * (bins + 1), bins, up);
            double f10 = or_cdf_eval(edge + ((size_t)I1 * Wb + J0) * (bins + 1), bins, up);
            double f11 = or_cdf_eval(edge + ((size_t)I1 * Wb + J1) * (bins + 1), bins, up);
            double F = (1.0 - wy) * ((1.0 - wx) * f00 + wx * f01) + wy * ((1.0 - wx) * f10 + wx * f11);
            y[(int64_t)py * W + px] = alpha * F + (1.0 - alpha) * up;
        }
    }
    free(win);
    free(h);
    free(edge);
    free(u);
    return 0;
}

/*
 * Comparison luminance channels of Sec. I and Fig. GTMO / Sec. III-B-1, which the
 * paper tone-maps beside its own:
 *   luma 0: the colour-temperature luminance of Eq. 1-6;
 *   luma 1: MATLAB's rgb2gray weighted sum quoted in Sec. I,
 *           Gray = 0.2989 R + 0.5870 G + 0.1140 B;
 *   luma 2: V of HSV, the largest channel;
 *   luma 3: CIE L* of CIELAB / 100 (Sec. I, Fig. 2, Table 1), of linear samples
 *           (oracle_decolorize_luma decodes 8-bit sRGB codes to linear first).
 * Returns NAN for an unknown luma code.
 */
/* CIE 1976 lightness of linear RGB (Rec. 709 / sRGB primaries, D65 white, Yn = 1),
 * divided by 100: L* = 116 f(Y) - 16, f(t) = cbrt(t) above (6/29)^3, else
 * t / (3 (6/29)^2) + 4/29, with Y = 0.2126 R + 0.7152 G + 0.0722 B. */
static double or_lstar(double R, double G, double B)
{
    double Y = 0.2126 * R + 0.7152 * G + 0.0722 * B;
    double d = 6.0 / 29.0;
    double f = Y > d * d * d ? cbrt(Y) : Y / (3.0 * d * d) + 4.0 / 29.0;
    return (116.0 * f - 16.0) / 100.0;
}

/* sRGB-encoded value in [0, 1] to linear light (the sRGB transfer function). */
static double or_srgb_linear(double c)
{
    return c <= 0.04045 ? c / 12.92 : pow((c + 0.055) / 1.055, 2.4);
}

double oracle_luma(double R, double G, double B, int32_t luma, double beta_R, double beta_k)
{
    if (luma == 0)
        return oracle_luminance(R, G, B, beta_R, beta_k);
    if (luma == 3)
        return or_lstar(R, G, B);  /* linear samples */
    if (luma == 1)
        return 0.2989 * R + 0.5870 * G + 0.1140 * B;
    if (luma == 2) {
        double m = R;
        if (G > m) m = G;
        if (B > m) m = B;
        return m;
    }
    return NAN;
}

/* oracle_decolorize with a choice of luminance channel. */
int oracle_decolorize_luma(const void* data, int32_t W, int32_t H, int64_t stride_bytes, int32_t dtype,
                           int32_t luma, double beta_R, double beta_k, double* L)
{
    if (W < 0 || H < 0 || dtype < OR_U8 || dtype > OR_F32 || luma < 0 || luma > 3)
        return 1;
    int esz = dtype == OR_U8 ? 1 : (dtype == OR_F16 ? 2 : 4);
    const unsigned char* base = (const unsigned char*)data;
    for (int32_t y = 0; y < H; ++y) {
        const unsigned char* row = base + (int64_t)y * stride_bytes;
        for (int32_t x = 0; x < W; ++x) {
            const unsigned char* px = row + (int64_t)x * 3 * esz;
            double R = or_sample(px, dtype, 0);
            double G = or_sample(px, dtype, 1);
            double B = or_sample(px, dtype, 2);
            if (luma == 3 && dtype == OR_U8) {  /* CIELAB is defined on linear light */
                R = or_srgb_linear(R);
                G = or_srgb_linear(G);
                B = or_srgb_linear(B);
            }
            L[(int64_t)y * W + x] = oracle_luma(R, G, B, luma, beta_R, beta_k);
        }
    }
    return 0;
}

/*
 * Colour reconstruction of a tone-mapped luminance (the colour outputs of
 * Fig. tmo_1, Fig. GTMO and Sec. II-D; the paper does not state the method).
 * Reading: every channel keeps its ratio to the luminance it was decolorized to,
 * raised to a saturation exponent s, and is scaled to the tone-mapped value:
 *   C_out = min(1, y (C_in / L)^s),
 * with 0^0 = 1 (a black channel is y when s = 0, 0 when s > 0) and a black pixel
 * (L = 0) taken as achromatic: every channel is y.  `L` and `y` are W x H planes;
 * `out` is W x H x 3, interleaved.
 */
int oracle_color_reconstruct(const void* data, int32_t W, int32_t H, int64_t stride_bytes, int32_t dtype,
                             const double* L, const double* y, double s, double* out)
{
    if (W < 0 || H < 0 || dtype < OR_U8 || dtype > OR_F32 || !(s >= 0.0))
        return 1;
    int esz = dtype == OR_U8 ? 1 : (dtype == OR_F16 ? 2 : 4);
    const unsigned char* base = (const unsigned char*)data;
    for (int32_t py = 0; py < H; ++py) {
        const unsigned char* row = base + (int64_t)py * stride_bytes;
        for (int32_t px = 0; px < W; ++px) {
            int64_t i = (int64_t)py * W + px;
            for (int c = 0; c < 3; ++c) {
                double C = or_sample(row + (int64_t)px * 3 * esz, dtype, c);
                double v;
                if (L[i] == 0.0)
                    v = y[i];
                else if (C == 0.0)
                    v = s == 0.0 ? y[i] : 0.0;
                else
                    v = y[i] * pow(C / L[i], s);
                out[3 * i + c] = v < 1.0 ? v : 1.0;
            }
        }
    }
    return 0;
}

/*
 * Frame sequences (the real-time use of Sec. I and Sec. III-B; the paper names no
 * temporal scheme).  Reading: frame t is tone-mapped with the centred sigmoid
 * around the log-mean estimate m_{t-1} carried from the frames before it, so one
 * pass over the frame suffices, and the estimate then follows the frame's own
 * log-mean mu_t by exponential smoothing:
 *   m_t = (1 - lambda) m_{t-1} + lambda mu_t,   0 < lambda <= 1.
 * The first frame has no estimate: it is centred on its own mu_0, and m_0 = mu_0.
 * This function is that update (one step), written out for the test of the state.
 */
double oracle_video_mu_update(double m_prev, double mu_frame, double lambda)
{
    return (1.0 - lambda) * m_prev + lambda * mu_frame;
}

/*
 * The two halves of the local operator of Sec. III-B-2 on a coordinate plane u
 * (already in [0, 1]), for frame sequences: the per-block cumulative tables of the
 * (2Rb+1)^2-block window of tent-binned block histograms, and the bilinear blend of
 * the four nearest block tables at each pixel's own u.  oracle_tone_local is the two
 * in sequence on one image; a frame of a running sequence (Sec. I, III-B-2 real-time
 * use; no scheme in the paper) applies the previous frame's tables to its own u and
 * then builds its own tables for the next frame.  `edge` is Hb x Wb x (bins + 1).
 * Returns 0, 1 on bad arguments, 2 on allocation failure.
 */
int oracle_local_tables(const double* u, int32_t W, int32_t H, int32_t s, int32_t Rb, int32_t bins, double* edge)
{
    if (W <= 0 || H <= 0 || s <= 0 || Rb < 0 || bins < 1)
        return 1;
    int32_t Hb = (H + s - 1) / s, Wb = (W + s - 1) / s;
    double* h = (double*)calloc((size_t)Hb * Wb * bins, sizeof(double));
    double* win = (double*)malloc(sizeof(double) * bins);
    if (!h || !win) {
        free(h); free(win);
        return 2;
    }
    for (int32_t py = 0; py < H; ++py)
        for (int32_t px = 0; px < W; ++px) {
            int j0, j1;
            double w0, w1;
            or_tent(u[(int64_t)py * W + px], bins, &j0, &w0, &j1, &w1);
            double* hb = h + ((size_t)(py / s) * Wb + (px / s)) * bins;
            hb[j0] += w0;
            hb[j1] += w1;
        }
    for (int32_t I = 0; I < Hb; ++I)
        for (int32_t J = 0; J < Wb; ++J) {
            for (int j = 0; j < bins; ++j) win[j] = 0.0;
            for (int32_t I2 = I - Rb; I2 <= I + Rb; ++I2) {
                if (I2 < 0 || I2 >= Hb) continue;
                for (int32_t J2 = J - Rb; J2 <= J + Rb; ++J2) {
                    if (J2 < 0 || J2 >= Wb) continue;
                    const double* hb = h + ((size_t)I2 * Wb + J2) * bins;
                    for (int j = 0; j < bins; ++j) win[j] += hb[j];
                }
            }
            double total = 0.0;
            for (int j = 0; j < bins; ++j) total += win[j];
            double* e = edge + ((size_t)I * Wb + J) * (bins + 1);
            double acc = 0.0;
            e[0] = 0.0;
            for (int j = 0; j < bins; ++j) {
                acc += win[j];
                e[j + 1] = acc / total;
            }
        }
    free(win);
    free(h);
    return 0;
}

int oracle_local_apply(const double* u, const double* edge, int32_t W, int32_t H, int32_t s, int32_t bins,
                       double alpha, double* y)
{
    if (W <= 0 || H <= 0 || s <= 0 || bins < 1)
        return 1;
    int32_t Hb = (H + s - 1) / s, Wb = (W + s - 1) / s;
    for (int32_t py = 0; py < H; ++py) {
        double fy = (py + 0.5) / s - 0.5;
        int32_t I0 = (int32_t)floor(fy);
        double wy = fy - I0;
        int32_t I1 = I0 + 1;
        if (I0 < 0) I0 = 0;
        if (I1 < 0) I1 = 0;
        if (I0 > Hb - 1) I0 = Hb - 1;
        if (I1 > Hb - 1) I1 = Hb - 1;
        for (int32_t px = 0; px < W; ++px) {
            double fx = (px + 0.5) / s - 0.5;
            int32_t J0 = (int32_t)floor(fx);
            double wx = fx - J0;
            int32_t J1 = J0 + 1;
            if (J0 < 0) J0 = 0;
            if (J1 < 0) J1 = 0;
            if (J0 > Wb - 1) J0 = Wb - 1;
            if (J1 > Wb - 1) J1 = Wb - 1;
            double up = u[(int64_t)py * W + px];
            double f00 = or_cdf_eval(edge + ((size_t)I0 * Wb + J0) * (bins + 1), bins, up);
            double f01 = or_cdf_eval(edge + ((size_t)I0 * Wb + J1) * (bins + 1), bins, up);
            double f10 = or_cdf_eval(edge + ((size_t)I1 * Wb + J0) * (bins + 1), bins, up);
            double f11 = or_cdf_eval(edge + ((size_t)I1 * Wb + J1) * (bins + 1), bins, up);
            double F = (1.0 - wy) * ((1.0 - wx) * f00 + wx * f01) + wy * ((1.0 - wx) * f10 + wx * f11);
            y[(int64_t)py * W + px] = alpha * F + (1.0 - alpha) * up;
        }
    }
    return 0;
}

/* The coordinate plane of the local operator: u = L clamped to [0, 1] (8-bit input)
 * or the normalised log luminance in the range (lmin, lmax), clamped (HDR input). */
void oracle_local_coord(const double* L, int64_t n, int32_t ldr, double delta, double lmin, double lmax, double* u)
{
    for (int64_t i = 0; i < n; ++i) {
        double v = ldr ? L[i] : or_log_u(L[i], delta, lmin, lmax);
        if (v < 0.0) v = 0.0;
        if (v > 1.0) v = 1.0;
        u[i] = v;
    }
}
