// Streaming pipeline of the engine: one producer warp moves pixel data into a ring
// of shared-memory stages with 1-D TMA bulk copies (cp.async.bulk, completion on
// an mbarrier) while eight consumer warps compute.  A "chunk" is up to 256 pixel
// groups (one per consumer thread) of one tile; short tile rows are packed several
// to a chunk at power-of-two strides so that consumer thread t always finds its
// group at stage + t * bytes_per_group.  Every wait is bounded by the launch's
// timeout and records DC_ERR_TIMEOUT when it runs out.
#pragma once

#include "dc_engine.cuh"

namespace dc {

constexpr int kTileRing = 2;
constexpr int kConsumerWarps = kThreads / 32;
constexpr int kBlockThreads = kThreads + 32;     // consumers + one producer warp

// Groups per consumer thread per stage and stage count, per input sample type: a
// 48-byte group holds 16 u8, 8 f16 or 4 f32 pixels.
template <int IN_DT> struct PipeCfg;
#ifndef DC_GPT_HDR
#define DC_GPT_HDR 1
#endif
#ifndef DC_STAGES_HDR
#define DC_STAGES_HDR 4
#endif
template <> struct PipeCfg<DC_U8> { static constexpr int GPT = 1, STAGES = 4; };
template <> struct PipeCfg<DC_F16> { static constexpr int GPT = DC_GPT_HDR, STAGES = DC_STAGES_HDR; };
template <> struct PipeCfg<DC_F32> { static constexpr int GPT = DC_GPT_HDR, STAGES = DC_STAGES_HDR; };

// Values a tile derives from an image's finished statistics pass.
struct Derived {
    float mu, exp_mu, lmin, lmax, inv_range;
};

// Producer -> consumer message: the next tile (tile < 0: no more work).
struct TileMsg {
    int tile, lt, img, p;
    Derived d;
};

template <int IN_DT>
struct __align__(128) PipeSmem {
    static constexpr int kGPT = PipeCfg<IN_DT>::GPT;
    static constexpr int kStages = PipeCfg<IN_DT>::STAGES;
    static constexpr int kGroups = kThreads * kGPT;  // groups per stage
    static constexpr int kBytes = kGroups * 48;
    unsigned char stage[kStages][kBytes];
    unsigned long long full[kStages];
    unsigned long long empty[kStages];
    unsigned long long tfull[kTileRing];
    unsigned long long tempty[kTileRing];
    TileMsg msg[kTileRing];
};

struct Ring {
    uint32_t idx, parity;
    __device__ __forceinline__ void advance(int n)
    {
        if (++idx == (uint32_t)n) {
            idx = 0;
            parity ^= 1u;
        }
    }
};

// ------------------------------------------------------------ PTX wrappers ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(b))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* b, uint32_t tx)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_addr(b)),
                 "r"(tx)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking probe of the phase with the given parity.
__device__ __forceinline__ bool mbar_test_wait(unsigned long long* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false (and DC_ERR_TIMEOUT
// recorded) when it did not complete within timeout_ns.
static __device__ __noinline__ bool mbar_wait_slow(unsigned long long* b, uint32_t parity, uint32_t* err,
                                                   unsigned long long timeout_ns)
{
    const unsigned long long t0 = globaltimer_ns();
    const unsigned long long max_iter = timeout_ns / 8ull + 65536ull;
    for (unsigned long long it = 0;; ++it) {
        if (mbar_try_wait(b, parity)) return true;
        if (globaltimer_ns() - t0 > timeout_ns || it > max_iter) {
            atomicCAS(err, 0u, (uint32_t)DC_ERR_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ bool mbar_wait(unsigned long long* b, uint32_t parity, uint32_t* err,
                                          unsigned long long timeout_ns)
{
    if (mbar_try_wait(b, parity)) return true;
    return mbar_wait_slow(b, parity, err, timeout_ns);
}

__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, unsigned long long* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_mbarrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Order this thread's earlier generic-proxy view of global memory (data other CTAs
// published, acquired through a phase counter) before later TMA reads of it.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Barrier over the 256 consumer threads only (the producer warp never joins it).
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory"); }

// --------------------------------------------------------- chunk geometry ----
// Full vector groups of a tile row segment are streamed, SG groups per chunk;
// ngv = 0 means the tile goes through the scalar path entirely.  Short rows are
// packed 2^lg groups apart, so group slot s of a chunk sits at stage + s * bpg.
struct ChunkGeo {
    int ngv;      // full groups per row
    int lg;       // log2 of the packed row stride in groups (ngv <= SG)
    int rpc;      // rows per chunk (ngv <= SG)
    int nchunks;
};

template <int SG>
__device__ __forceinline__ ChunkGeo chunk_geo(int r0, int r1, int c0, int c1, int G, bool vec)
{
    ChunkGeo g;
    g.ngv = vec ? (c1 - c0) / G : 0;
    const int nrows = r1 - r0;
    if (g.ngv == 0) {
        g.lg = 0;
        g.rpc = 1;
        g.nchunks = 0;
    } else if (g.ngv <= SG) {
        g.lg = 32 - __clz(g.ngv - 1);
        g.rpc = SG >> g.lg;
        g.nchunks = (nrows + g.rpc - 1) / g.rpc;
    } else {
        g.lg = 0;
        g.rpc = 1;
        g.nchunks = nrows * ((g.ngv + SG - 1) / SG);
    }
    return g;
}

// Walks the chunks of a tile in order without divisions: for short rows the first
// row of the chunk, for long rows the row and its first group.
template <int SG>
struct ChunkCursor {
    int row, g0;
    __device__ __forceinline__ void start(const ChunkGeo& g, int r0)
    {
        row = r0;
        g0 = 0;
    }
    __device__ __forceinline__ void next(const ChunkGeo& g)
    {
        if (g.ngv <= SG) {
            row += g.rpc;
        } else {
            g0 += SG;
            if (g0 >= g.ngv) {
                g0 = 0;
                ++row;
            }
        }
    }
    // slot s of the current chunk: its row and first column; false when empty
    __device__ __forceinline__ bool slot(const ChunkGeo& g, int r1, int c0, int G, int s, int& r, int& c) const
    {
        if (g.ngv <= SG) {
            const int j = s >> g.lg, gi = s & ((1 << g.lg) - 1);
            r = row + j;
            c = c0 + gi * G;
            return r < r1 && gi < g.ngv;
        }
        r = row;
        c = c0 + (g0 + s) * G;
        return g0 + s < g.ngv;
    }
};

}  // namespace dc
