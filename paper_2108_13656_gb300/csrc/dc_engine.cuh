// Pass kernels: decolorization (Eq. 1-6, Sec. II-B) fused with the global
// (Sec. III-B-1) and local (Sec. III-B-2) tone-mapping passes.
//
// Layout and schedule (see dc_internal.h): a batch of images, each a chain of
// passes, each pass cut into tiles; one persistent launch per pass takes the
// tiles of every image in a fixed round-robin order (tile t goes to CTA
// t mod grid).  Pixels are read in groups (8 u8 pixels = 24 bytes, 8 f16 or
// 4 f32 pixels = 48 bytes) with 8- or 16-byte vector loads when the image is
// 16-byte aligned; everything else (ragged row tails, unaligned images) takes a
// per-pixel path with identical arithmetic.  All arithmetic is binary32; every
// cross-thread reduction is exact integer arithmetic (the log-sum in 2^-24 fixed
// point, min/max on ordered bit patterns, histograms as counts), so results do
// not depend on the launch shape.
#pragma once

#include <climits>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dc_internal.h"

namespace dc {

constexpr int kThreads = 256;
constexpr int kLocMaxBlocksX = 32;    // max blocks per local tile row
constexpr int kCdfMaxChunk = 64;      // block columns per CDF tile, at most
constexpr int kMaxRadius = 16;

template <int IN_DT> struct InT;
template <> struct InT<DC_U8> { static constexpr int G = 8; static constexpr int ESZ = 1; };
template <> struct InT<DC_F16> { static constexpr int G = 8; static constexpr int ESZ = 2; };
template <> struct InT<DC_F32> { static constexpr int G = 4; static constexpr int ESZ = 4; };

enum OpKind { OPK_DECOLOR = 0, OPK_GLOBAL = 1, OPK_LOCAL = 2 };

// ---------------------------------------------------- bounds-checked build ---
// Built with -DDC_BOUNDS_CHECK, every global access of the pass kernels is checked
// against the extent of the buffer it targets (input, output, plane, workspace); an
// access outside is skipped (a load gives 0) and a bit is set in a per-library flag
// word that dc_debug_bounds reads.  It stands in for a memory checker: tests run the
// odd shapes, strides and batches through such a build and expect no flag.
enum : uint32_t { BC_IN = 1u, BC_OUT = 2u, BC_PLANE = 4u, BC_WS = 8u };
#ifdef DC_BOUNDS_CHECK
static __device__ unsigned int g_bounds_flags;
__device__ __forceinline__ bool bc_ok(const void* p, int64_t bytes, const void* base, int64_t extent, uint32_t bit)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(p), b0 = reinterpret_cast<uintptr_t>(base);
    const bool ok = a >= b0 && bytes >= 0 && a + (uintptr_t)bytes <= b0 + (uintptr_t)extent;
    if (!ok) atomicOr(&g_bounds_flags, bit);
    return ok;
}
#else
__device__ __forceinline__ bool bc_ok(const void*, int64_t, const void*, int64_t, uint32_t) { return true; }
#endif

// ------------------------------------------------------------ memory access ---
// Input pixels: read-only for the whole launch, so the loads may be scheduled
// freely (not volatile).  A thread's group is 24 or 48 contiguous bytes, so the lanes
// of a warp read at a 24- or 48-byte stride and the two or three loads of a group
// touch the same cache lines: the lines are allocated in L1 (first-evicted), so that
// the later loads of a group hit what the first one brought in instead of fetching
// the same sectors from L2 again.
__device__ __forceinline__ uint4 ld_stream16(const void* p)
{
    uint4 v;
    asm("ld.global.nc.L1::evict_first.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

// L2 eviction-priority policies (createpolicy): input that is read once can leave
// L2 first, so that a plane written for the next pass stays resident.
__device__ __forceinline__ unsigned long long policy_evict_first()
{
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ unsigned long long policy_evict_last()
{
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint4 ld_stream16_hint(const void* p, unsigned long long pol)
{
    uint4 v;
    asm("ld.global.nc.L1::evict_first.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ void st_f4_hint(float* p, float4 v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ uint2 ld_stream8(const void* p)
{
    uint2 v;
    asm("ld.global.nc.L1::evict_first.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

// Data other CTAs of the same launch wrote (the L plane, histograms, tables):
// L2 only, never a stale L1 line.  Ordinary loads to the compiler, so independent
// ones are issued back to back.
__device__ __forceinline__ float4 ld_cg_f4(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float ld_cg_f(const float* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ld_cg_u64(const unsigned long long* p) { return __ldcg(p); }
__device__ __forceinline__ uint32_t ld_cg_u32(const uint32_t* p) { return __ldcg(p); }

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------- fast binary32 math --
// Hardware approximations (PTX sqrt.approx / rcp.approx, and the lg2/ex2 based
// intrinsics); their errors are a few ulp, far inside the 2e-6 parity tolerance.
__device__ __forceinline__ float sqrt_fast(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_fast(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// Hardware base-2 logarithm without subnormal handling (every caller's argument is
// at least FLT_MIN).
__device__ __forceinline__ float lg2_ftz(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// ln x = log2(x) ln 2, for x >= FLT_MIN.
__device__ __forceinline__ float ln_fast(float x) { return lg2_ftz(x) * 0.693147180559945309f; }
// ln 2 in units of 2^-24: a group's sum of base-2 logarithms times this is its sum of
// natural logarithms in the 2^-24 fixed point of the log-sum.
constexpr float kLn2Q24 = 0.693147180559945309f * 16777216.0f;
__device__ __forceinline__ float exp_fast(float x) { return __expf(x); }

// ------------------------------------------------------------- Eq. 1-6 -------
struct Beta {
    float bR, one_m_bR, bk, one_m_bk;
    int luma;  // DC_LUMA_OURS (Eq. 1-6), DC_LUMA_Y or DC_LUMA_V
};

// CIE 1976 lightness / 100 of linear samples (Rec. 709 luminance, D65 white, Yn = 1):
// 116 f(Y) - 16 with f the cube root above (6/29)^3 and the linear segment below.
__device__ __forceinline__ float lstar_linear(float R, float G, float B)
{
    const float Y = fmaf(0.0722f, B, fmaf(0.7152f, G, 0.2126f * R));
    const float f = Y > 0.008856451679f ? cbrtf(Y) : fmaf(Y, 841.0f / 108.0f, 4.0f / 29.0f);
    return fmaf(116.0f, f, -16.0f) * 0.01f;
}
// An sRGB-encoded value in [0, 1] to linear light.
__device__ __forceinline__ float srgb_to_linear(float c)
{
    return c <= 0.04045f ? c * (1.0f / 12.92f) : powf((c + 0.055f) * (1.0f / 1.055f), 2.4f);
}

// The comparison channels of Sec. I / Fig. GTMO on non-negative samples: MATLAB's
// rgb2gray weights, V of HSV, or CIE L* (linear samples).
__device__ __forceinline__ float luma_other(float R, float G, float B, int luma)
{
    if (luma == DC_LUMA_LSTAR) return lstar_linear(R, G, B);
    return luma == DC_LUMA_Y ? fmaf(0.1140f, B, fmaf(0.5870f, G, 0.2989f * R)) : fmaxf(R, fmaxf(G, B));
}

// ------------------------------------------------- paired binary32 (f32x2) ---
// Blackwell executes add/sub/mul/fma on a pair of binary32 values as one
// instruction; each lane rounds exactly like the scalar instruction, so a pixel
// gives the same bits through the paired and the scalar form below.
struct F2 {
    unsigned long long v;
};
__device__ __forceinline__ F2 f2(float a, float b)
{
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ F2 f2s(float a) { return f2(a, a); }
__device__ __forceinline__ void f2split(F2 x, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v)); }
__device__ __forceinline__ F2 operator+(F2 a, F2 b)
{
    F2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    F2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b)
{
    F2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 f2fma(F2 a, F2 b, F2 c)
{
    F2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}

// Eq. 1-6 in binary32 for one pixel.  R+G+B = 0 gives 0 (continuous extension).
// The operation order is that of luminance_x2, lane by lane.
__device__ __forceinline__ float luminance_f32(float R, float G, float B, const Beta& be)
{
    const float S = (R + G) + B;
    const float R2 = R * R, G2 = G * G;
    const float L_WHITE = sqrt_fast(fmaf(B, B, R2 + G2) * (1.0f / 3.0f));  // Eq. 1
    const float L_B = B;                                                     // Eq. 2
    const float L_GR = sqrt_fast(fmaf(be.bR, R2, be.one_m_bR * G2));         // Eq. 3
    const float inv = rcp_fast(S);
    const float r = R * inv, b = B * inv;
    const float L_WARM = fmaf(r, L_GR - L_WHITE, L_WHITE);                    // Eq. 4
    const float L_COOL = fmaf(b, L_WHITE - L_B, L_B);                         // Eq. 5
    const float L = sqrt_fast(fmaf(be.bk, L_WARM * L_WARM, (be.one_m_bk * L_COOL) * L_COOL));  // Eq. 6
    return S > 0.0f ? L : 0.0f;
}

// Eq. 1-6 for two pixels: the additions and products in f32x2, the square roots
// and the reciprocal per lane.  U8: samples are 8-bit codes, so S = R+G+B is 0 or at
// least 1; the reciprocal of max(S, 1/2) then gives every term of a black pixel as 0
// (and the other pixels the same bits), with no select.
template <bool U8 = false>
__device__ __forceinline__ void luminance_x2(F2 R, F2 G, F2 B, const Beta& be, float& L0, float& L1, float& s0,
                                             float& s1)
{
    const F2 S = (R + G) + B;
    const F2 R2 = R * R, G2 = G * G;
    float a0, a1, c0, c1;
    f2split(f2fma(B, B, R2 + G2) * f2s(1.0f / 3.0f), a0, a1);
    const F2 L_WHITE = f2(sqrt_fast(a0), sqrt_fast(a1));                      // Eq. 1
    f2split(f2fma(f2s(be.bR), R2, f2s(be.one_m_bR) * G2), c0, c1);
    const F2 L_GR = f2(sqrt_fast(c0), sqrt_fast(c1));                         // Eq. 3
    f2split(S, s0, s1);
    const F2 inv = U8 ? f2(rcp_fast(fmaxf(s0, 0.5f)), rcp_fast(fmaxf(s1, 0.5f))) : f2(rcp_fast(s0), rcp_fast(s1));
    const F2 r = R * inv, b = B * inv;
    const F2 L_WARM = f2fma(r, L_GR - L_WHITE, L_WHITE);                      // Eq. 4
    const F2 L_COOL = f2fma(b, L_WHITE - B, B);                               // Eq. 5 (L_B = B)
    f2split(f2fma(f2s(be.bk), L_WARM * L_WARM, (f2s(be.one_m_bk) * L_COOL) * L_COOL), a0, a1);
    if (U8) {
        L0 = sqrt_fast(a0);                                                   // Eq. 6
        L1 = sqrt_fast(a1);
    } else {
        L0 = s0 > 0.0f ? sqrt_fast(a0) : 0.0f;
        L1 = s1 > 0.0f ? sqrt_fast(a1) : 0.0f;
    }
}

template <bool U8 = false>
__device__ __forceinline__ void luminance_x2(F2 R, F2 G, F2 B, const Beta& be, float& L0, float& L1)
{
    float s0, s1;
    luminance_x2<U8>(R, G, B, be, L0, L1, s0, s1);
}

// Linear samples of arbitrary magnitude: Eq. 1-6 are 1-homogeneous, so a pixel
// whose squares leave the binary32 range is scaled by a power of two first (exact)
// and the result scaled back.
static __device__ __noinline__ float luminance_rescaled(float R, float G, float B, const Beta& be)
{
    const float m = fmaxf(R, fmaxf(G, B));
    int e;
    frexpf(m, &e);
    const float s = ldexpf(1.0f, -e);
    return ldexpf(luminance_f32(R * s, G * s, B * s, be), e);
}

__device__ __forceinline__ float luminance_hdr(float R, float G, float B, const Beta& be)
{
    R = fmaxf(R, 0.0f);
    G = fmaxf(G, 0.0f);
    B = fmaxf(B, 0.0f);
    const float L = luminance_f32(R, G, B, be);
    // samples beyond about 2^63 overflow the squares (inf or NaN); samples below
    // about 2^-63 flush them (0 for a non-black pixel): both take the scaled path
    if (!(L <= 3.0e38f) || (L == 0.0f && R + G + B > 0.0f)) return luminance_rescaled(R, G, B, be);
    return L;
}

// ------------------------------------------------------ fixed-point log ------
// ln x in units of 2^-24, for x >= FLT_MIN: x = 2^e m with m in (1/sqrt 2, sqrt 2],
// ln x = e ln 2 + ln m, the first term from ln 2 in 2^-32 units (error below 2^-30
// for any e) rounded to 2^-24, ln m (|ln m| < 0.35) from the hardware base-2
// logarithm (absolute error about 2^-22 on [1/2, 2]) rounded to 2^-24.  Absolute
// error about 2e-7 whatever the magnitude of ln x, where a binary32 ln x near 7 is
// only good to 5e-7 and its normalisation by the log range adds as much again: the
// histogram forms need the absolute error.
constexpr long long kLn2Q32 = 2977044472LL;  // round(ln 2 * 2^32)
constexpr int kLn2Q32Hi = 11629079, kLn2Q32Lo = 248;  // kLn2Q32 = 256 Hi + Lo
static_assert(256LL * kLn2Q32Hi + kLn2Q32Lo == kLn2Q32, "split of ln 2");
__device__ __forceinline__ int ln_q24(float x)
{
    // e = floor((bits(x) - bits(m0)) / 2^23) with m0 the first binary32 above
    // 1/sqrt 2; then bits(m) = bits(x) - e 2^23 lies in [bits(m0), bits(m0) + 2^23),
    // i.e. m in (1/sqrt 2, sqrt 2] and x = 2^e m
    const int bits = __float_as_int(x);
    const int e = (bits - 0x3F3504F4) >> 23;
    const float m = __int_as_float(bits - (e << 23));
    // ln m in 2^-24 units (ln 2 2^24 is ln 2 scaled by a power of two: one rounding)
    const float lm = lg2_ftz(m) * (0.693147180559945309f * 16777216.0f);
    // e ln 2 in 2^-24 units rounded half up, (e kLn2Q32 + 128) >> 8, in 32-bit
    // pieces (|e| <= 150): e Hi + floor((e Lo + 128) / 256)
    const int ep = e * kLn2Q32Hi + ((e * kLn2Q32Lo + 128) >> 8);
    return ep + __float2int_rn(lm);
}

// Two linear pixels: negatives (and NaN) to 0, the paired Eq. 1-6, and the scaled
// path for a pixel whose squares leave the binary32 range.
__device__ __forceinline__ void luminance_hdr_x2(float R0, float G0, float B0, float R1, float G1, float B1,
                                                 const Beta& be, float& L0, float& L1)
{
    R0 = fmaxf(R0, 0.0f);
    G0 = fmaxf(G0, 0.0f);
    B0 = fmaxf(B0, 0.0f);
    R1 = fmaxf(R1, 0.0f);
    G1 = fmaxf(G1, 0.0f);
    B1 = fmaxf(B1, 0.0f);
    float s0, s1;  // (R + G) + B of each pixel
    luminance_x2(f2(R0, R1), f2(G0, G1), f2(B0, B1), be, L0, L1, s0, s1);
    if (!(L0 <= 3.0e38f) || (L0 == 0.0f && s0 > 0.0f)) L0 = luminance_rescaled(R0, G0, B0, be);
    if (!(L1 <= 3.0e38f) || (L1 == 0.0f && s1 > 0.0f)) L1 = luminance_rescaled(R1, G1, B1, be);
}

// ----------------------------------------------- float-float (hi + lo) ------
// Unevaluated sums of two binary32 numbers (Dekker; Knuth's two-sum; the FMA
// product error), about 44 significant bits.  Used where binary32 alone is too
// coarse: the 8-bit local operator's bin coordinate, whose curve slope reaches the
// bin count (a binary32 L, good to about 1e-7, would move its output by up to 3e-6).
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b), bp = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp))};
}
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b)  // |a| >= |b| or a = 0
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ FF ff_add(FF x, FF y)
{
    const FF s = ff_two_sum(x.hi, y.hi);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ FF ff_neg(FF x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ FF ff_mul(FF x, FF y)
{
    const FF p = ff_prod(x.hi, y.hi);
    return ff_fast_two_sum(p.hi, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo)));
}
__device__ __forceinline__ FF ff_mulf(FF x, float f)
{
    const FF p = ff_prod(x.hi, f);
    return ff_fast_two_sum(p.hi, fmaf(x.lo, f, p.lo));
}
// a / b for binary32 a, b (b > 0): the rounded quotient and the exact remainder's share.
__device__ __forceinline__ FF ff_divf(float a, float b)
{
    const float q = __fdiv_rn(a, b);
    return ff_fast_two_sum(q, __fdiv_rn(fmaf(-q, b, a), b));
}
// x / b for a float-float x and binary32 b > 0.
__device__ __forceinline__ FF ff_div_by(FF x, float b)
{
    const float q = __fdiv_rn(x.hi, b);
    return ff_fast_two_sum(q, __fdiv_rn(__fadd_rn(fmaf(-q, b, x.hi), x.lo), b));
}
// Square root: the rounded root s of hi and one Newton correction (x - s^2) / 2s.
__device__ __forceinline__ FF ff_sqrt(FF x)
{
    if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
    const float s = __fsqrt_rn(x.hi);
    const float r = __fadd_rn(fmaf(-s, s, x.hi), x.lo);
    return ff_fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.0f, s)));
}

// Eq. 1-6 in float-float for 8-bit codes R, G, B (0..255, exact in binary32), in
// code units; the betas are the binary32 parameters themselves (1 - beta exactly).
__device__ __forceinline__ FF luminance_ff(float R, float G, float B, const Beta& be)
{
    const float S = (R + G) + B;  // exact
    if (S == 0.0f) return {0.0f, 0.0f};
    const float R2 = R * R, G2 = G * G;                     // exact (< 2^16)
    const float n1 = fmaf(B, B, R2 + G2);                   // exact (< 2^18)
    const FF L_WHITE = ff_sqrt(ff_divf(n1, 3.0f));          // Eq. 1
    const FF omR = ff_two_sum(1.0f, -be.bR);
    const FF L_GR = ff_sqrt(ff_add(ff_prod(be.bR, R2), ff_mulf(omR, G2)));  // Eq. 3
    const FF r = ff_divf(R, S), b = ff_divf(B, S);
    const FF L_WARM = ff_add(L_WHITE, ff_mul(r, ff_add(L_GR, ff_neg(L_WHITE))));   // Eq. 4
    const FF L_COOL = ff_add({B, 0.0f}, ff_mul(b, ff_add(L_WHITE, {-B, 0.0f})));   // Eq. 5, L_B = B
    const FF omk = ff_two_sum(1.0f, -be.bk);
    const FF Q = ff_add(ff_mulf(ff_mul(L_WARM, L_WARM), be.bk), ff_mul(omk, ff_mul(L_COOL, L_COOL)));
    return ff_sqrt(Q);                                      // Eq. 6
}

// The chosen channel of 8-bit codes in float-float (code units).
__device__ __forceinline__ FF luma_ff(float R, float G, float B, const Beta& be)
{
    if (be.luma == DC_LUMA_OURS) return luminance_ff(R, G, B, be);
    if (be.luma == DC_LUMA_Y) return ff_add(ff_add(ff_prod(0.2989f, R), ff_prod(0.5870f, G)), ff_prod(0.1140f, B));
    if (be.luma == DC_LUMA_LSTAR)  // (binary32 only; the host does not route L* here)
        return {255.0f * lstar_linear(srgb_to_linear(R * (1.0f / 255.0f)), srgb_to_linear(G * (1.0f / 255.0f)),
                                      srgb_to_linear(B * (1.0f / 255.0f))),
                0.0f};
    return {fmaxf(R, fmaxf(G, B)), 0.0f};
}

// Bin coordinate t = bins * L / 255 of an 8-bit pixel in units of 2^-24 (rounded),
// from the float-float luminance: 0 <= t 2^24 <= bins 2^24 <= 2^29.
__device__ __forceinline__ uint32_t ucoord_u8(float R, float G, float B, const Beta& be, int bins)
{
    const FF L = luma_ff(R, G, B, be);
    const FF t = ff_div_by(ff_mulf(L, (float)bins), 255.0f);
    const float hs = t.hi * 16777216.0f, ls = t.lo * 16777216.0f;  // exact scalings
    const int qh = __float2int_rn(hs);
    const int q = qh + __float2int_rn(__fadd_rn(__fsub_rn(hs, (float)qh), ls));
    return (uint32_t)min(max(q, 0), bins << 24);
}

// 8-bit code of y in [0,1]: floor(255 y + 1/2), clamped.
__device__ __forceinline__ uint32_t quant_u8(float y)
{
    float t = fmaxf(fminf(fmaf(y, 255.0f, 0.5f), 255.0f), 0.0f);
    return __float_as_uint(__fadd_rd(t, 8388608.0f)) & 0xFFu;
}

// u8 sample -> float via the exponent-bias trick (2^23 + v, minus 2^23): exact.
__device__ __forceinline__ float u8_biased(const uint32_t (&w)[12], int idx)
{
    return __uint_as_float(__byte_perm(w[idx >> 2], 0x4B00u, 0x5440u | (uint32_t)(idx & 3)));
}
__device__ __forceinline__ float u8_at(const uint32_t (&w)[12], int idx) { return u8_biased(w, idx) - 8388608.0f; }
// The same for the samples idx and idx + 3 (one channel of two neighbouring pixels).
__device__ __forceinline__ F2 u8_pair(const uint32_t (&w)[12], int idx)
{
    return f2(u8_biased(w, idx), u8_biased(w, idx + 3)) - f2s(8388608.0f);
}

// ordered-uint encoding of floats (monotone), for exact atomic min/max
__device__ __forceinline__ uint32_t ord_enc(float f)
{
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord_dec(uint32_t o)
{
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}

// ------------------------------------------------------------ group I/O ------
template <int IN_DT>
struct GroupIO {
    static constexpr int G = InT<IN_DT>::G;
    static constexpr int ESZ = InT<IN_DT>::ESZ;

    // Luminance in [0,1] units (8-bit codes / 255; linear values as they are) of a
    // full group given as its 48 raw bytes (twelve 32-bit words).
    __device__ static __forceinline__ void decode(const uint32_t (&w)[12], const Beta& be, float (&Lv)[G])
    {
        if (be.luma != DC_LUMA_OURS) {
            decode_other(w, be.luma, Lv);
            return;
        }
        if constexpr (IN_DT == DC_U8) {
#pragma unroll
            for (int k = 0; k < G; k += 2) {
                float L0, L1;
                luminance_x2<true>(u8_pair(w, 3 * k), u8_pair(w, 3 * k + 1), u8_pair(w, 3 * k + 2), be, L0, L1);
                f2split(f2(L0, L1) * f2s(1.0f / 255.0f), Lv[k], Lv[k + 1]);
            }
        } else if constexpr (IN_DT == DC_F16) {
            float f[24];
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                __half2 h;
                memcpy(&h, &w[k], 4);
                float2 v = __half22float2(h);
                f[2 * k] = v.x;
                f[2 * k + 1] = v.y;
            }
#pragma unroll
            for (int k = 0; k < G; k += 2)
                luminance_hdr_x2(f[3 * k], f[3 * k + 1], f[3 * k + 2], f[3 * k + 3], f[3 * k + 4], f[3 * k + 5], be,
                                 Lv[k], Lv[k + 1]);
        } else {
#pragma unroll
            for (int k = 0; k < G; k += 2)
                luminance_hdr_x2(__uint_as_float(w[3 * k]), __uint_as_float(w[3 * k + 1]), __uint_as_float(w[3 * k + 2]),
                                 __uint_as_float(w[3 * k + 3]), __uint_as_float(w[3 * k + 4]),
                                 __uint_as_float(w[3 * k + 5]), be, Lv[k], Lv[k + 1]);
        }
    }

    // Sample i (0 .. 3G-1) of a group's raw words as a linear value: 8-bit codes as
    // code values (0..255, not yet divided by 255); HDR samples with negatives and
    // NaN read as 0.
    __device__ static __forceinline__ float sample(const uint32_t (&w)[12], int i)
    {
        if constexpr (IN_DT == DC_U8) {
            return u8_at(w, i);
        } else if constexpr (IN_DT == DC_F16) {
            __half2 h;
            memcpy(&h, &w[i >> 1], 4);
            const float2 v = __half22float2(h);
            return fmaxf((i & 1) ? v.y : v.x, 0.0f);
        } else {
            return fmaxf(__uint_as_float(w[i]), 0.0f);
        }
    }

    // The comparison channels (DC_LUMA_Y, DC_LUMA_V) of a group, in [0,1] units.
    __device__ static __forceinline__ void decode_other(const uint32_t (&w)[12], int luma, float (&Lv)[G])
    {
#pragma unroll
        for (int k = 0; k < G; ++k) {
            float R = sample(w, 3 * k), Gc = sample(w, 3 * k + 1), B = sample(w, 3 * k + 2);
            if (IN_DT == DC_U8 && luma == DC_LUMA_LSTAR) {  // CIELAB is defined on linear light
                R = srgb_to_linear(R * (1.0f / 255.0f));
                Gc = srgb_to_linear(Gc * (1.0f / 255.0f));
                B = srgb_to_linear(B * (1.0f / 255.0f));
                Lv[k] = lstar_linear(R, Gc, B);
            } else {
                const float v = luma_other(R, Gc, B, luma);
                Lv[k] = IN_DT == DC_U8 ? v * (1.0f / 255.0f) : v;
            }
        }
    }

    // Bytes each buffer of an image spans (for the bounds-checked build).
    __device__ static __forceinline__ int64_t in_extent(const DcImage& im)
    {
        return (int64_t)(im.rows - 1) * im.in_stride + (int64_t)im.cols * 3 * ESZ;
    }
    __device__ static __forceinline__ int64_t plane_extent(const DcImage& im)
    {
        return (int64_t)(im.rows - 1) * im.plane_stride + (int64_t)im.cols * 4;
    }
    __device__ static __forceinline__ int64_t out_extent(const DcImage& im)
    {
        const int oe = im.out_dt == DC_U8 ? 1 : (im.out_dt == DC_F16 ? 2 : 4);
        return (int64_t)(im.rows - 1) * im.out_stride + (int64_t)im.cols * oe * ((im.flags & IF_COLOR) ? 3 : 1);
    }

    // The n (< G, or unaligned) pixels at (r, c) packed like a full group's raw words,
    // the lanes past n zero: the same decode then applies.
    __device__ static void gather_raw(const DcImage& im, int r, int c, int n, uint32_t (&w)[12])
    {
#pragma unroll
        for (int k = 0; k < 12; ++k) w[k] = 0u;
        const uint8_t* p = im.in + (int64_t)r * im.in_stride + (int64_t)c * 3 * ESZ;
        if (!bc_ok(p, (int64_t)n * 3 * ESZ, im.in, in_extent(im), BC_IN)) return;
        for (int i = 0; i < 3 * n; ++i) {
            if constexpr (ESZ == 1) {
                w[i >> 2] |= (uint32_t)__ldg(p + i) << (8 * (i & 3));
            } else if constexpr (ESZ == 2) {
                w[i >> 1] |= (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p) + i) << (16 * (i & 1));
            } else {
                w[i] = __ldg(reinterpret_cast<const uint32_t*>(p) + i);
            }
        }
    }

    // Colour reconstruction of one group (DC_LUMA_* luminance Lv in [0,1] units, tone-
    // mapped values y): o[3k + i] = min(1, y (C_i / L)^s), a black pixel giving y.
    // The ratio C_i / L is taken in code units for 8-bit input; a pixel whose L lies
    // outside [2^-60, 2^60] is scaled by a power of two first (exact), its luminance
    // recomputed, so that the ratio keeps full precision.
    __device__ static __forceinline__ void color_values(const uint32_t (&w)[12], const float (&Lv)[G],
                                                        const float (&y)[G], const Beta& be, float s, bool s_one,
                                                        float (&o)[3 * G])
    {
#pragma unroll
        for (int k = 0; k < G; ++k) {
            float C[3] = {sample(w, 3 * k), sample(w, 3 * k + 1), sample(w, 3 * k + 2)};
            float L = IN_DT == DC_U8 ? Lv[k] * 255.0f : Lv[k];
            if (!(L > 0.0f)) {
                o[3 * k] = o[3 * k + 1] = o[3 * k + 2] = y[k];
                continue;
            }
            if (L < 0x1p-60f || L > 0x1p60f) rescale_pixel(C, be, L);
            if (s_one) {
                const float q = y[k] * rcp_fast(L);
#pragma unroll
                for (int i = 0; i < 3; ++i) o[3 * k + i] = fminf(C[i] * q, 1.0f);
            } else {
                const float lL = lg2_ftz(L);
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    o[3 * k + i] = C[i] > 0.0f ? fminf(y[k] * exp2f(s * (lg2_ftz(C[i]) - lL)), 1.0f)
                                               : (s == 0.0f ? y[k] : 0.0f);
            }
        }
    }

    // A pixel with a tiny or huge luminance: samples scaled by 2^-e (e the exponent of
    // the largest) and its luminance recomputed from them (every channel is
    // 1-homogeneous, so the ratios are unchanged).
    __device__ static __forceinline__ void rescale_pixel(float (&C)[3], const Beta& be, float& L)
    {
        int e;
        frexpf(fmaxf(C[0], fmaxf(C[1], C[2])), &e);
        const float sc = ldexpf(1.0f, -e);
        C[0] *= sc;
        C[1] *= sc;
        C[2] *= sc;
        L = be.luma == DC_LUMA_OURS ? luminance_f32(C[0], C[1], C[2], be) : luma_other(C[0], C[1], C[2], be.luma);
    }

    // Store the 3n colour values of n pixels at (r, c) (interleaved RGB output).
    __device__ static void store_rgb(const DcImage& im, int r, int c, int n, bool vec, const float (&o)[3 * G])
    {
        const int oe = im.out_dt == DC_U8 ? 1 : (im.out_dt == DC_F16 ? 2 : 4);
        uint8_t* p = im.out + (int64_t)r * im.out_stride + (int64_t)c * 3 * oe;
        if (!bc_ok(p, (int64_t)(vec ? G : n) * 3 * oe, im.out, out_extent(im), BC_OUT)) return;
        if (im.out_dt == DC_U8) {
            if (vec) {  // 3G bytes at a multiple of 3G: 8-byte pieces (G = 8) or 4-byte ones (G = 4)
                uint32_t wv[3 * G / 4];
#pragma unroll
                for (int k = 0; k < 3 * G / 4; ++k) wv[k] = 0u;
#pragma unroll
                for (int k = 0; k < 3 * G; ++k) wv[k >> 2] |= quant_u8(o[k]) << (8 * (k & 3));
                if constexpr (G == 8) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) reinterpret_cast<uint2*>(p)[k] = make_uint2(wv[2 * k], wv[2 * k + 1]);
                } else {
#pragma unroll
                    for (int k = 0; k < 3; ++k) reinterpret_cast<uint32_t*>(p)[k] = wv[k];
                }
            } else {
                for (int k = 0; k < 3 * n; ++k) p[k] = (uint8_t)quant_u8(o[k]);
            }
        } else if (im.out_dt == DC_F16) {
            if (vec) {  // 6G bytes at a multiple of 6G: 16-byte pieces (G = 8) or 8-byte ones (G = 4)
                uint32_t wv[3 * G / 2];
#pragma unroll
                for (int k = 0; k < 3 * G / 2; ++k) {
                    __half2 h = __floats2half2_rn(o[2 * k], o[2 * k + 1]);
                    memcpy(&wv[k], &h, 4);
                }
                if constexpr (G == 8) {
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        reinterpret_cast<uint4*>(p)[k] = make_uint4(wv[4 * k], wv[4 * k + 1], wv[4 * k + 2], wv[4 * k + 3]);
                } else {
#pragma unroll
                    for (int k = 0; k < 3; ++k) reinterpret_cast<uint2*>(p)[k] = make_uint2(wv[2 * k], wv[2 * k + 1]);
                }
            } else {
                for (int k = 0; k < 3 * n; ++k) reinterpret_cast<__half*>(p)[k] = __float2half_rn(o[k]);
            }
        } else {
            if (vec) {  // 12G bytes: 16-byte pieces
#pragma unroll
                for (int k = 0; k < 3 * G / 4; ++k)
                    reinterpret_cast<float4*>(p)[k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
            } else {
                for (int k = 0; k < 3 * n; ++k) reinterpret_cast<float*>(p)[k] = o[k];
            }
        }
    }

    // The raw bytes of a full, aligned group: 24 (u8, three 8-byte loads) or 48
    // (f16, f32, three 16-byte loads).
    // With a plane kept for later passes (f16/f32 input), the input is read only
    // once, so it is loaded with an evict-first L2 policy.
    __device__ static __forceinline__ void load_raw(const DcImage& im, int r, int c, uint32_t (&w)[12])
    {
        load_raw_at(im, im.in + (int64_t)r * im.in_stride + (int64_t)c * 3 * ESZ, w);
    }
    // The same from the group's address p.
    __device__ static __forceinline__ void load_raw_at(const DcImage& im, const uint8_t* p, uint32_t (&w)[12])
    {
        if (!bc_ok(p, 3 * G * ESZ, im.in, in_extent(im), BC_IN)) {
#pragma unroll
            for (int k = 0; k < 12; ++k) w[k] = 0u;
            return;
        }
        if constexpr (IN_DT == DC_U8) {
            const uint2 a = ld_stream8(p), b = ld_stream8(p + 8), d = ld_stream8(p + 16);
            w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y; w[4] = d.x; w[5] = d.y;
        } else if (im.flags & IF_LPLANE) {
            const unsigned long long pol = policy_evict_first();
            const uint4 a = ld_stream16_hint(p, pol), b = ld_stream16_hint(p + 16, pol), d = ld_stream16_hint(p + 32, pol);
            w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
            w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
            w[8] = d.x; w[9] = d.y; w[10] = d.z; w[11] = d.w;
        } else {
            const uint4 a = ld_stream16(p), b = ld_stream16(p + 16), d = ld_stream16(p + 32);
            w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
            w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
            w[8] = d.x; w[9] = d.y; w[10] = d.z; w[11] = d.w;
        }
    }

    // Luminance of the n pixels starting at (r, c) read straight from global memory.
    // vec: full 16-byte aligned group.
    __device__ static void luminance(const DcImage& im, int r, int c, int n, bool vec,
                                     const Beta& be, float (&Lv)[G])
    {
        const uint8_t* p = im.in + (int64_t)r * im.in_stride + (int64_t)c * 3 * ESZ;
        if (vec) {
            uint32_t w[12];
            load_raw(im, r, c, w);
            decode(w, be, Lv);
        } else {
            const bool ok = bc_ok(p, (int64_t)n * 3 * ESZ, im.in, in_extent(im), BC_IN);
#pragma unroll
            for (int k = 0; k < G; ++k) Lv[k] = (ok && k < n) ? scalar_luminance(p + k * 3 * ESZ, be) : 0.0f;
        }
    }

    // One pixel through the scalar path (ragged tails and unaligned images).
    __device__ static __noinline__ float scalar_luminance(const uint8_t* q, const Beta& be)
    {
        if (be.luma != DC_LUMA_OURS) {
            float c[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if constexpr (IN_DT == DC_U8) {
                    c[i] = (float)__ldg(q + i);
                } else if constexpr (IN_DT == DC_F16) {
                    c[i] = fmaxf(__half2float(reinterpret_cast<const __half*>(q)[i]), 0.0f);
                } else {
                    c[i] = fmaxf(__ldg(reinterpret_cast<const float*>(q) + i), 0.0f);
                }
            }
            if (IN_DT == DC_U8 && be.luma == DC_LUMA_LSTAR)
                return lstar_linear(srgb_to_linear(c[0] * (1.0f / 255.0f)), srgb_to_linear(c[1] * (1.0f / 255.0f)),
                                    srgb_to_linear(c[2] * (1.0f / 255.0f)));
            const float v = luma_other(c[0], c[1], c[2], be.luma);
            return IN_DT == DC_U8 ? v * (1.0f / 255.0f) : v;
        }
        if constexpr (IN_DT == DC_U8) {
            return luminance_f32((float)__ldg(q), (float)__ldg(q + 1), (float)__ldg(q + 2), be) * (1.0f / 255.0f);
        } else if constexpr (IN_DT == DC_F16) {
            const __half* h = reinterpret_cast<const __half*>(q);
            return luminance_hdr(__half2float(h[0]), __half2float(h[1]), __half2float(h[2]), be);
        } else {
            const float* f = reinterpret_cast<const float*>(q);
            return luminance_hdr(__ldg(f), __ldg(f + 1), __ldg(f + 2), be);
        }
    }

    // Luminance (or its fixed-point log or bin coordinate) from the f32 plane an
    // earlier phase wrote.
    // A full, aligned group of the plane at p.
    __device__ static __forceinline__ void from_plane_at(const DcImage& im, const float* p, float (&Lv)[G])
    {
        const bool ok = bc_ok(p, G * 4, im.plane, plane_extent(im), BC_PLANE);
#pragma unroll
        for (int k = 0; k < G; k += 4) {
            const float4 v = ok ? ld_cg_f4(p + k) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            Lv[k] = v.x;
            Lv[k + 1] = v.y;
            Lv[k + 2] = v.z;
            Lv[k + 3] = v.w;
        }
    }

    __device__ static void from_plane(const DcImage& im, int r, int c, int n, bool vec, float (&Lv)[G])
    {
        const float* p = reinterpret_cast<const float*>(im.plane + (int64_t)r * im.plane_stride) + c;
        if (!bc_ok(p, (int64_t)(vec ? G : n) * 4, im.plane, plane_extent(im), BC_PLANE)) {
#pragma unroll
            for (int k = 0; k < G; ++k) Lv[k] = 0.0f;
            return;
        }
        if (vec) {
#pragma unroll
            for (int k = 0; k < G; k += 4) {
                float4 v = ld_cg_f4(p + k);
                Lv[k] = v.x;
                Lv[k + 1] = v.y;
                Lv[k + 2] = v.z;
                Lv[k + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < G; ++k) Lv[k] = (k < n) ? ld_cg_f(p + k) : 0.0f;
        }
    }

    // The f32 plane a stats pass keeps for the next passes (evict-last in L2).
    __device__ static __forceinline__ void store_plane(const DcImage& im, int r, int c, int n, bool vec,
                                                       const float (&y)[G])
    {
        float* p = reinterpret_cast<float*>(im.plane + (int64_t)r * im.plane_stride) + c;
        if (!bc_ok(p, (int64_t)(vec ? G : n) * 4, im.plane, plane_extent(im), BC_PLANE)) return;
        if (vec) {
            const unsigned long long pol = policy_evict_last();
#pragma unroll
            for (int k = 0; k < G; k += 4) st_f4_hint(p + k, make_float4(y[k], y[k + 1], y[k + 2], y[k + 3]), pol);
        } else {
#pragma unroll
            for (int k = 0; k < G; ++k)
                if (k < n) p[k] = y[k];
        }
    }

    // A full, aligned group of G values at p in the output sample type OUT_DT.
    template <int OUT_DT>
    __device__ static __forceinline__ void store_full(uint8_t* p, const float (&y)[G])
    {
        if constexpr (OUT_DT == DC_U8) {
            uint32_t w[(G + 3) / 4];
#pragma unroll
            for (int k = 0; k < (G + 3) / 4; ++k) w[k] = 0;
#pragma unroll
            for (int k = 0; k < G; ++k) w[k >> 2] |= quant_u8(y[k]) << (8 * (k & 3));
            if constexpr (G == 8) {
                *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
            } else {
                *reinterpret_cast<uint32_t*>(p) = w[0];
            }
        } else if constexpr (OUT_DT == DC_F16) {
            uint32_t w[G / 2];
#pragma unroll
            for (int k = 0; k < G / 2; ++k) {
                __half2 h = __floats2half2_rn(y[2 * k], y[2 * k + 1]);
                memcpy(&w[k], &h, 4);
            }
            if constexpr (G == 8) {
                *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
            } else {
                *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < G; k += 4)
                *reinterpret_cast<float4*>(p + 4 * k) = make_float4(y[k], y[k + 1], y[k + 2], y[k + 3]);
        }
    }

    // Store n values (in [0,1] units) at (r, c) in the output sample type.
    __device__ static void store(const DcImage& im, int r, int c, int n, bool vec, const float (&y)[G])
    {
        uint8_t* base = im.out + (int64_t)r * im.out_stride;
        {
            const int oe = im.out_dt == DC_U8 ? 1 : (im.out_dt == DC_F16 ? 2 : 4);
            if (!bc_ok(base + (int64_t)c * oe, (int64_t)(vec ? G : n) * oe, im.out, out_extent(im), BC_OUT)) return;
        }
        if (im.out_dt == DC_U8) {
            uint8_t* p = base + c;
            if (vec) {
                uint32_t w[(G + 3) / 4];
#pragma unroll
                for (int k = 0; k < (G + 3) / 4; ++k) w[k] = 0;
#pragma unroll
                for (int k = 0; k < G; ++k) w[k >> 2] |= quant_u8(y[k]) << (8 * (k & 3));
                if constexpr (G == 16) {
                    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
                } else if constexpr (G == 8) {
                    *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
                } else {
                    *reinterpret_cast<uint32_t*>(p) = w[0];
                }
            } else {
#pragma unroll
                for (int k = 0; k < G; ++k)
                    if (k < n) p[k] = (uint8_t)quant_u8(y[k]);
            }
        } else if (im.out_dt == DC_F16) {
            __half* p = reinterpret_cast<__half*>(base) + c;
            if (vec) {
                uint32_t w[G / 2];
#pragma unroll
                for (int k = 0; k < G / 2; ++k) {
                    __half2 h = __floats2half2_rn(y[2 * k], y[2 * k + 1]);
                    memcpy(&w[k], &h, 4);
                }
                if constexpr (G == 16) {
                    reinterpret_cast<uint4*>(p)[0] = make_uint4(w[0], w[1], w[2], w[3]);
                    reinterpret_cast<uint4*>(p)[1] = make_uint4(w[4], w[5], w[6], w[7]);
                } else if constexpr (G == 8) {
                    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
                } else {
                    *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
                }
            } else {
#pragma unroll
                for (int k = 0; k < G; ++k)
                    if (k < n) p[k] = __float2half_rn(y[k]);
            }
        } else {
            float* p = reinterpret_cast<float*>(base) + c;
            if (vec) {
#pragma unroll
                for (int k = 0; k < G; k += 4)
                    *reinterpret_cast<float4*>(p + k) = make_float4(y[k], y[k + 1], y[k + 2], y[k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < G; ++k)
                    if (k < n) p[k] = y[k];
            }
        }
    }
};

// Pairwise sum of a compile-time-length array (fixed order).
template <int N>
__device__ __forceinline__ float pairwise_sum(const float* v)
{
    if constexpr (N == 1) {
        return v[0];
    } else {
        return pairwise_sum<N / 2>(v) + pairwise_sum<N - N / 2>(v + N / 2);
    }
}

// ------------------------------------------------------------ shared memory ---
struct SmemStats {
    uint32_t hist[256];
    long long wsum[kThreads / 32];
    float wmin[kThreads / 32], wmax[kThreads / 32];
    uint32_t scan[kThreads];
};
struct SmemApplyG {
    float lut[260];
};
// Per-block stride of the block-histogram pass's shared counters: at least B and 8
// (mod 32), so that equal bins of neighbouring blocks (a warp covers several blocks
// of a row) fall 8 banks apart; at most DC_MAX_BINS + 8.
__host__ __device__ constexpr int blockh_stride(int bins) { return bins + ((8 - bins % 32) + 32) % 32; }
struct SmemBlockH {
    uint32_t cnt[kLocMaxBlocksX * (DC_MAX_BINS + 8)];  // pixels whose lower tent bin is j
    uint32_t fs[kLocMaxBlocksX * (DC_MAX_BINS + 8)];   // their upper-bin fractions, units of 2^-20
};
struct SmemCdf {
    unsigned long long v[(kCdfMaxChunk + 2 * kMaxRadius) * DC_MAX_BINS];
};
constexpr int kLocMaxCols = 1024;    // widest local tile
// Geometry of the apply pass's curve table, fixed at compile time so that the four
// curve reads of a pixel are one address plus immediate offsets: slots of
// kTabSlot (value, slope) pairs - at least DC_MAX_BINS and 8 (mod 16), i.e. 16 banks
// between neighbouring slots - and block rows of kLocMaxBlocksX + 2 slots.
constexpr int kTabSlot = DC_MAX_BINS + ((24 - DC_MAX_BINS % 16) % 16);
constexpr int kTabRow = (kLocMaxBlocksX + 2) * kTabSlot;
static_assert(kTabSlot % 16 == 8, "neighbouring slots 16 banks apart");
constexpr int kLocMaxRows = 64;      // tallest local tile (block_s)
struct SmemApplyL {
    float2 tab[3 * kTabRow];  // per block and bin: (F at bin start, slope)
    // per tile column x: table slot offset of the left block and the weight bits, at
    // (x mod G) * (kLocMaxCols + 16) / G + x / G for groups of G pixels, so that the
    // lanes of a warp, one group each, read neighbouring entries
    int2 col[kLocMaxCols + 16];
    int2 row[kLocMaxRows];  // per tile row: table slot offset of the upper block row, weight bits
};

template <int OPK>
struct SmemBytes {
    static constexpr size_t a = sizeof(SmemStats) > sizeof(SmemApplyG) ? sizeof(SmemStats) : sizeof(SmemApplyG);
    static constexpr size_t b = sizeof(SmemBlockH) > sizeof(SmemCdf) ? sizeof(SmemBlockH) : sizeof(SmemCdf);
    static constexpr size_t c = b > sizeof(SmemApplyL) ? b : sizeof(SmemApplyL);
    static constexpr size_t value = OPK == OPK_LOCAL ? (a > c ? a : c) : a;
};

__device__ __forceinline__ DcImgCtrl* img_ctrl(DcCtrl* c, int i)
{
    return reinterpret_cast<DcImgCtrl*>(reinterpret_cast<uint8_t*>(c) + sizeof(DcCtrl)) + i;
}



}  // namespace dc
