// gemm_dev.cuh -- the device side of the BF16 projection GEMM on the
// sm_100-family tensor cores (tcgen05.mma, accumulator in tensor memory,
// operands staged by TMA), as tile functions shared by the one-tile-per-CTA
// kernel (gemm_tc.cu) and the persistent decoder (persist.cu).
//
// Y[token][feature] = sum_k X[token][k] Wt[feature][k].  The projection is
// the MMA's A operand (M = 128 output features per tile) and the tokens are
// its B operand (N = 64 or 32 tokens per tile), so a decoder step with a few dozen
// tokens fills one tile and the weights stream through once.  Weights are
// consumed in 64-element K chunks (one 128-byte swizzle atom) through a
// TMA ring as deep as the shared-memory budget allows (all chunks of a
// 384-wide projection).  The token operand either streams through the same ring
// (compact bf16 rows) or is built by the CTA in shared memory: RMSNorm of the
// FP32 residual stream rows (the pre-norm of every projection, Sec. 3.1) or
// the channel-scaled latents (the latent embedding).  One thread issues the
// MMAs, every K step in ascending order into one accumulator (the dual
// form's up projection has a second issuer and accumulator); 256 threads run
// the epilogue from TMEM (warps w and w + 4 read the same 32 feature rows,
// half of the token columns each) with the destination rows of the tile's
// tokens resolved once into shared memory.  The tensor core computes an
// output element identically whatever the MMA's N and whichever operand
// holds the tokens, so with the accumulation order fixed every output
// element is the same function of its row and column whatever the tile, the
// launch or the kernel it falls in.
//
// Two forms change only the resources, not the arithmetic: lean tiles (a
// 96 KB ring and four-row token builds, two CTAs per SM, for launches with
// more tiles than SMs) and 32-token tiles (TN = 32, for launches whose
// 64-token grid leaves SMs idle).
//
// A tile runs in two parts.  gemm_tile_pre resolves the tile's token table
// and issues the weight copies of its first ring stages; it reads nothing a
// previous kernel or phase writes, so callers run it before waiting for
// their inputs.  gemm_tile_main loads or builds the token operand, runs the
// MMAs and the epilogue.  The barrier parities (GemmPipe) carry over from tile to
// tile, so one CTA can run any sequence of tiles of any shapes and ring
// depths.
//
// E4M3 projections (F8) take the same tile: weights are E4M3 bytes with a
// dequantisation scale per feature row (one power of two per source tensor),
// the token operand is always built in shared memory as E4M3 with a
// power-of-two scale per token computed from that token's own row, the MMA is
// kind::f8f6f4 (K = 32 per instruction) over 128-element chunks (the same 128
// bytes per row as a bf16 chunk), and the epilogue multiplies the FP32
// accumulator by the two scales, both powers of two, so dequantisation is
// exact and a token's result still depends on nothing but its own row.
//
// Every mbarrier wait is bounded (~2 s of globaltimer); on expiry the CTA
// raises its abort flag, waits (bounded) for its own copies and MMAs and
// skips the epilogue; the caller reports ST_TIMEOUT.
#pragma once

#include "internal.h"
#include "device_common.cuh"

#include <cuda.h>
#include <cuda_fp8.h>

namespace psw {
namespace tc {

constexpr int TM = 128;        // output features per tile (MMA M)
constexpr int NT = 64;         // tokens per tile (MMA N)
constexpr int KC = 64;         // K elements per stage (128 bytes of bf16)
constexpr int KC8 = 128;       // K elements per stage of an E4M3 projection (128 bytes)
constexpr int MAXS = 8;        // ring stages at most (barrier pairs)
constexpr int RING_BUDGET = 216 * 1024;   // dynamic shared memory of the ring and the resident operand
constexpr int RING_BUDGET_LEAN = 96 * 1024;   // the same for two CTAs per SM (lean tiles)
constexpr int A_BYTES = TM * KC * 2;
constexpr int B_BYTES = NT * KC * 2;
constexpr int KRES_MAX = 512;  // largest K of a token operand built in shared memory
constexpr uint64_t WAIT_NS = 2000000000ull;
constexpr int NTHREADS = 256;  // 8 warps: warps w and w + 4 share TMEM lanes 32 (w % 4) .. + 31
constexpr int NARRIVE = 2;     // commits that release a ring stage or finish a tile (two per tile: the dual
                               // form's two issuers commit once each, the single issuer twice)
constexpr int NPROD = 4;       // copy producers: lane 0 of warps 0, 5, 6 and 7
// tensor-memory columns of a tile: one accumulator of tn columns (two, gate
// and up, for the dual form)
__host__ __device__ constexpr uint32_t tile_tcols(bool dual, int tn = NT) { return (dual ? 2 : 1) * tn; }
// Bytes of one 128-byte-wide K chunk of a tn-token operand.
__host__ __device__ constexpr int tok_chunk_bytes(int tn) { return tn * 128; }

__host__ __device__ constexpr int kchunk(bool f8) { return f8 ? KC8 : KC; }

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on a phase of an mbarrier; false after ~2 s.  The test of an
// already completed phase is inline; the polling loop is out of line.
static __device__ __noinline__ bool mbar_wait_slow(uint64_t *b, uint32_t parity)
{
    uint64_t t0 = gtime();
    while (!mbar_try(b, parity))
        if (gtime() - t0 > WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity)
{
    if (mbar_try(b, parity)) return true;
    return mbar_wait_slow(b, parity);
}

__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *tm, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(su32(dst)), "l"(tm), "r"(su32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Orders this thread's view of global memory (including what other threads
// released to it) before its later tensor-copy reads, and its own generic
// writes before later async-proxy accesses.
__device__ __forceinline__ void fence_proxy_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row atoms 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
    d |= (uint64_t)1 << 46;                          // version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: F32 accumulate, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t dt, uint64_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dt), "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

// Instruction descriptor, kind::f8f6f4: F32 accumulate, E4M3 A and B
// (format 0), both K-major.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma8(uint32_t dt, uint64_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dt), "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t tmem, uint32_t cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
}

__device__ __forceinline__ void tmem_ld8_async(uint32_t addr, uint32_t *r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 8 / 16 consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_get8(uint32_t addr, float *v)
{
    uint32_t r[8];
    tmem_ld8_async(addr, r);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_get16(uint32_t addr, float *v)
{
    uint32_t r[16];
    tmem_ld8_async(addr, r);
    tmem_ld8_async(addr + 8, r + 8);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// Eight columns at addr and eight at addr2 under one wait.
__device__ __forceinline__ void tmem_get8x2(uint32_t addr, uint32_t addr2, float *v, float *v2)
{
    uint32_t r[8], r2[8];
    tmem_ld8_async(addr, r);
    tmem_ld8_async(addr2, r2);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 8; i++) { v[i] = __uint_as_float(r[i]); v2[i] = __uint_as_float(r2[i]); }
}

// Byte offset of element (row r, column k) of a K-major bf16 operand laid
// out in 128-byte-swizzled atoms of 64 columns x NT rows.
template <int TN = NT>
__device__ __forceinline__ uint32_t swz(int r, int k)
{
    int kc = k >> 6, col = k & 63;
    uint32_t byte = (uint32_t)col * 2;
    return (uint32_t)kc * tok_chunk_bytes(TN) + (uint32_t)r * 128 + ((((byte >> 4) ^ (uint32_t)(r & 7))) << 4) +
           (byte & 15);
}

// The same for an 8-bit operand: atoms of 128 columns.
template <int TN = NT>
__device__ __forceinline__ uint32_t swz8(int r, int k)
{
    int kc = k >> 7;
    uint32_t byte = (uint32_t)(k & 127);
    return (uint32_t)kc * tok_chunk_bytes(TN) + (uint32_t)r * 128 + ((((byte >> 4) ^ (uint32_t)(r & 7))) << 4) +
           (byte & 15);
}

__device__ __forceinline__ uint2 pack4(float a, float b, float c, float d)
{
    __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    return make_uint2(*reinterpret_cast<uint32_t *>(&lo), *reinterpret_cast<uint32_t *>(&hi));
}

// Four E4M3 values (round to nearest even, saturating), a in the low byte.
__device__ __forceinline__ uint32_t e4m3x4(float a, float b, float c, float d)
{
    uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
}

// Power-of-two scaling of a row for E4M3: with max |x| in [2^e, 2^(e+1)),
// x * 2^(7-e) has magnitude below 256 (E4M3 reaches 448).  Sets *qmul =
// 2^(7-e) and returns the dequantisation scale 2^(e-7); e is clamped at
// -100 so both stay normal FP32 numbers (an all-zero row gets 2^-107).
__device__ __forceinline__ float row_scale_e4m3(float amax, float *qmul)
{
    int e = (int)((__float_as_uint(amax) >> 23) & 255) - 127;
    e = e < -100 ? -100 : e;
    *qmul = __uint_as_float((uint32_t)(127 + 7 - e) << 23);
    return __uint_as_float((uint32_t)(127 - 7 + e) << 23);
}

// Per-CTA shared state of the engine.
struct GemmShared {
    uint64_t full[MAXS], empty[MAXS], done;
    uint32_t tmem_slot;
    volatile int abort;
    float stab[NSCALES];
    float xs[NT];              // E4M3 projections: dequantisation scale of each token of the tile
    const int16_t *yrow[NT];
    uintptr_t tab[4][NT];
};

// Ring state carried from tile to tile.  Each ring stage has its own
// full/empty barrier pair, and the thread that waits on a barrier keeps the
// parity of the next completion it needs, so tiles of different ring depths
// can follow one another (the ring is idle between tiles).
// Every thread keeps the same copy, updated at the end of each tile, so
// that any thread can issue any stage's copies: chunk j of a tile with ring
// depth nst fills stage j % nst for its (j / nst)-th time in the tile.
struct GemmPipe {
    uint32_t fills = 0;        // parity of the fills of each stage before this tile (bit s)
    uint32_t empties = 0;      // parity of the releases (empty completions) of each stage before this tile
    uint32_t ntile = 0;        // tiles completed (phase of the done barrier)
};

// Parity of the u-th fill of stage s in the current tile (its full
// barrier's completion).  A stage is released (its empty barrier completes)
// only when the tile fills it again, so the ring needs no release between
// tiles: the done barrier already means every MMA has read its operands.
__device__ __forceinline__ uint32_t fill_parity(const GemmPipe &pp, int s, int u)
{
    return ((pp.fills >> s) & 1) ^ (uint32_t)(u & 1);
}

// Parity of the release the u-th (u >= 1) fill of stage s waits for.
__device__ __forceinline__ uint32_t release_parity(const GemmPipe &pp, int s, int u)
{
    return ((pp.empties >> s) & 1) ^ (uint32_t)((u - 1) & 1);
}

// Account for a finished tile of nk chunks over nst stages.
__device__ __forceinline__ void pipe_advance(GemmPipe &pp, int nk, int nst)
{
    for (int s = 0; s < nst; s++) {
        int uses = (nk - s + nst - 1) / nst;
        pp.fills ^= (uint32_t)(uses & 1) << s;
        pp.empties ^= (uint32_t)((uses - 1) & 1) << s;
    }
}

// Ring stage bytes: the weight chunk(s) and, for a streamed token operand,
// its chunk.
__host__ __device__ constexpr int stage_bytes(bool dual, bool resident, int tn = NT)
{
    return (dual ? 2 : 1) * A_BYTES + (resident ? 0 : tok_chunk_bytes(tn));
}

// K chunks of a projection.
__host__ __device__ constexpr int kchunks(int K, bool f8) { return (K + kchunk(f8) - 1) / kchunk(f8); }

// Ring depth of a projection: as many stages as its K chunks, the barrier
// pairs and the shared-memory budget (after the resident operand) allow.
// Lean tiles (single accumulator, two CTAs per SM) have the smaller budget.
__host__ __device__ constexpr int ring_stages(bool dual, bool resident, int K, bool f8 = false, bool lean = false,
                                             int tn = NT)
{
    int nk = kchunks(K, f8), res = resident ? nk * tok_chunk_bytes(tn) : 0;
    int st = ((lean ? RING_BUDGET_LEAN : RING_BUDGET) - res) / stage_bytes(dual, resident, tn);
    st = st < MAXS ? st : MAXS;
    st = st < nk ? st : nk;
    return st < 1 ? 1 : st;
}

// Dynamic shared memory of a tile (ring, then the resident token operand),
// without the 1024-byte alignment slack.
__host__ __device__ constexpr int tile_smem(bool dual, bool resident, int K, bool f8 = false, bool lean = false,
                                           int tn = NT)
{
    return ring_stages(dual, resident, K, f8, lean, tn) * stage_bytes(dual, resident, tn) +
           (resident ? kchunks(K, f8) * tok_chunk_bytes(tn) : 0);
}

// Initialise the barriers (thread 0; the caller synchronises).
__device__ __forceinline__ void gemm_shared_init(GemmShared &S)
{
    for (int s = 0; s < MAXS; s++) { mbar_init(&S.full[s], 1); mbar_init(&S.empty[s], NARRIVE); }
    mbar_init(&S.done, NARRIVE);
    S.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The gains of lane l's elements 4l + 128c .. +3 (c < CH), loaded once per
// build (they sit at any float offset), and the reciprocal 1/K the mean of
// squares uses.
template <int CH>
__device__ __forceinline__ void load_gain(const float *__restrict__ gain, int K, float4 *gh)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < CH; c++) {
        int e = lane * 4 + c * 128;
        gh[c] = e < K ? make_float4(gain[e], gain[e + 1], gain[e + 2], gain[e + 3]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// 1 / RMS of a row from its sum of squares (approximate reciprocal square
// root; the same instruction sequence for every token, so encoder and decoder
// agree bit for bit).
__device__ __forceinline__ float inv_rms(float ss, float invK) { return rsqrtf(fmaf(ss, invK, 1e-6f)); }

// RMSNorm of RB rows r0 .. r0+RB-1 of the tile by one warp, every load of
// the rows issued before the first reduction; lane l holds elements
// 4l + 128c .. +3 of a row (c < CH).
template <int RB, int CH, int TN = NT>
__device__ __forceinline__ void norm_rows(const float *__restrict__ xrows, const float *__restrict__ gain, int K,
                                          int M, int m0, int r0, uint8_t *res)
{
    const int lane = threadIdx.x & 31;
    float4 v[RB][CH], gh[CH];
    float ss[RB];
    load_gain<CH>(gain, K, gh);
    const float invK = 1.0f / (float)K;
#pragma unroll
    for (int b = 0; b < RB; b++) {
        int m = m0 + r0 + b;
        const float *x = m < M ? xrows + (long)m * K : nullptr;
#pragma unroll
        for (int c = 0; c < CH; c++) {
            int e = lane * 4 + c * 128;
            v[b][c] = (x && e < K) ? *(const float4 *)(x + e) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
#pragma unroll
    for (int b = 0; b < RB; b++) {
        ss[b] = 0.0f;
#pragma unroll
        for (int c = 0; c < CH; c++) {
            ss[b] = fmaf(v[b][c].x, v[b][c].x, ss[b]); ss[b] = fmaf(v[b][c].y, v[b][c].y, ss[b]);
            ss[b] = fmaf(v[b][c].z, v[b][c].z, ss[b]); ss[b] = fmaf(v[b][c].w, v[b][c].w, ss[b]);
        }
        ss[b] = warp_sum(ss[b]);
    }
#pragma unroll
    for (int b = 0; b < RB; b++) {
        int r = r0 + b;
        float inv = m0 + r < M ? inv_rms(ss[b], invK) : 0.0f;
#pragma unroll
        for (int c = 0; c < CH; c++) {
            int e = lane * 4 + c * 128;
            if (e >= K) continue;
            *(uint2 *)(res + swz<TN>(r, e)) = pack4(v[b][c].x * inv * gh[c].x, v[b][c].y * inv * gh[c].y,
                                                v[b][c].z * inv * gh[c].z, v[b][c].w * inv * gh[c].w);
        }
    }
}

// RMSNorm of one FP32 row times the gain into a compact bf16 row dst[0..K)
// in global memory, the row's elements already in registers (v: lane l's
// elements 4l + 128c .. +3, zero past K; gh: the same lanes' gains,
// load_gain): the arithmetic of norm_rows for one row (the same fused
// multiply-add chain and butterfly sum), so the row equals, bit for bit,
// the operand a tile builds in shared memory.  Used where a projection's
// tiles stream the normalised rows with TMA instead of each feature tile
// normalising them again.
template <int CH>
__device__ __forceinline__ void norm_row_store(const float4 *v, const float4 *gh, float invK, int K,
                                               __nv_bfloat16 *__restrict__ dst)
{
    const int lane = threadIdx.x & 31;
    float ss = 0.0f;
#pragma unroll
    for (int c = 0; c < CH; c++) {
        ss = fmaf(v[c].x, v[c].x, ss); ss = fmaf(v[c].y, v[c].y, ss);
        ss = fmaf(v[c].z, v[c].z, ss); ss = fmaf(v[c].w, v[c].w, ss);
    }
    ss = warp_sum(ss);
    const float inv = inv_rms(ss, invK);
#pragma unroll
    for (int c = 0; c < CH; c++) {
        int e = lane * 4 + c * 128;
        if (e >= K) continue;
        *(uint2 *)(dst + e) = pack4(v[c].x * inv * gh[c].x, v[c].y * inv * gh[c].y, v[c].z * inv * gh[c].z,
                                    v[c].w * inv * gh[c].w);
    }
}

// norm_row_store of the FP32 row x[0..K), loaded here.
template <int CH>
__device__ __forceinline__ void norm_row_global(const float *__restrict__ x, const float4 *gh, float invK, int K,
                                                __nv_bfloat16 *__restrict__ dst)
{
    const int lane = threadIdx.x & 31;
    float4 v[CH];
#pragma unroll
    for (int c = 0; c < CH; c++) {
        int e = lane * 4 + c * 128;
        v[c] = e < K ? *(const float4 *)(x + e) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    norm_row_store<CH>(v, gh, invK, K, dst);
}

// The E4M3 operand rows of norm_rows8 and quant_rows8 for one row in global
// memory: the same lane layout and operations (sum of squares, reciprocal
// square root, gain, absolute maximum, power-of-two scale, conversion), so a
// row streamed by the wide projection kernel equals, byte for byte, the row
// a tile builds in shared memory; *xs receives its dequantisation scale.
// The _store forms take the row already in registers (v: lane l's elements
// 4l + 128c .. +3, zero past K, overwritten; q: lane l's elements
// 8l + 256c .. +7 as bf16, zero past K), the _global forms load it first.
template <int CH>
__device__ __forceinline__ void norm_row8_store(float4 *v, const float4 *gh, float invK, int K,
                                                uint8_t *__restrict__ dst, float *xs)
{
    const int lane = threadIdx.x & 31;
    float ss = 0.0f;
#pragma unroll
    for (int c = 0; c < CH; c++) {
        ss = fmaf(v[c].x, v[c].x, ss); ss = fmaf(v[c].y, v[c].y, ss);
        ss = fmaf(v[c].z, v[c].z, ss); ss = fmaf(v[c].w, v[c].w, ss);
    }
    ss = warp_sum(ss);
    const float inv = inv_rms(ss, invK);
    float amax = 0.0f;
#pragma unroll
    for (int c = 0; c < CH; c++) {
        int e = lane * 4 + c * 128;
        if (e >= K) continue;
        v[c] = make_float4(v[c].x * inv * gh[c].x, v[c].y * inv * gh[c].y, v[c].z * inv * gh[c].z,
                           v[c].w * inv * gh[c].w);
        amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v[c].x), fabsf(v[c].y)), fmaxf(fabsf(v[c].z), fabsf(v[c].w))));
    }
    float qm, sc = row_scale_e4m3(warp_max(amax), &qm);
#pragma unroll
    for (int c = 0; c < CH; c++) {
        int e = lane * 4 + c * 128;
        if (e >= K) continue;
        *(uint32_t *)(dst + e) = e4m3x4(v[c].x * qm, v[c].y * qm, v[c].z * qm, v[c].w * qm);
    }
    if (lane == 0) *xs = sc;
}

template <int CH>
__device__ __forceinline__ void norm_row8_global(const float *__restrict__ x, const float4 *gh, float invK, int K,
                                                 uint8_t *__restrict__ dst, float *xs)
{
    const int lane = threadIdx.x & 31;
    float4 v[CH];
#pragma unroll
    for (int c = 0; c < CH; c++) {
        int e = lane * 4 + c * 128;
        v[c] = e < K ? *(const float4 *)(x + e) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    norm_row8_store<CH>(v, gh, invK, K, dst, xs);
}

template <int CH>
__device__ __forceinline__ void quant_row8_store(const uint4 *q, int K, uint8_t *__restrict__ dst, float *xs)
{
    const int lane = threadIdx.x & 31;
    float amax = 0.0f;
#pragma unroll
    for (int c = 0; c < CH; c++) {
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&q[c]);
#pragma unroll
        for (int i = 0; i < 4; i++) {
            float2 f = __bfloat1622float2(h[i]);
            amax = fmaxf(amax, fmaxf(fabsf(f.x), fabsf(f.y)));
        }
    }
    float qm, sc = row_scale_e4m3(warp_max(amax), &qm);
#pragma unroll
    for (int c = 0; c < CH; c++) {
        int e = lane * 8 + c * 256;
        if (e >= K) continue;
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&q[c]);
        float2 f0 = __bfloat1622float2(h[0]), f1 = __bfloat1622float2(h[1]);
        float2 f2 = __bfloat1622float2(h[2]), f3 = __bfloat1622float2(h[3]);
        *(uint2 *)(dst + e) = make_uint2(e4m3x4(f0.x * qm, f0.y * qm, f1.x * qm, f1.y * qm),
                                         e4m3x4(f2.x * qm, f2.y * qm, f3.x * qm, f3.y * qm));
    }
    if (lane == 0) *xs = sc;
}

template <int CH>
__device__ __forceinline__ void quant_row8_global(const __nv_bfloat16 *__restrict__ row, int K,
                                                  uint8_t *__restrict__ dst, float *xs)
{
    const int lane = threadIdx.x & 31;
    uint4 q[CH];
#pragma unroll
    for (int c = 0; c < CH; c++) {
        int e = lane * 8 + c * 256;
        q[c] = e < K ? *(const uint4 *)(row + e) : make_uint4(0, 0, 0, 0);
    }
    quant_row8_store<CH>(q, K, dst, xs);
}

// Build the token operand of rows m0 .. m0+63 in shared memory; rows past M
// are zero.  Warp w builds rows 8w .. 8w+7.  A_NORM: RMSNorm of the FP32 rows
// xrows[m] times the gain; A_EMBED / A_ZHAT: the channel-scaled latents of
// the token, or the z-hat of its hyperlatent (row pointers resolved
// beforehand into yrow).  All of a warp's loads are in
// flight together (K <= 384: the eight rows at once; lean tiles, with half
// the registers, four at a time).  One out-of-line copy serves every
// projection mode (keeps the instruction footprint small).
template <int RB, int TN = NT>
__device__ __forceinline__ void embed_rows(const float *__restrict__ gain, int K, int r0, uint8_t *res,
                                           const int16_t *const *yrow)
{
    constexpr int CH = KRES_MAX / 128;
    const int lane = threadIdx.x & 31;
    short4 q[RB][CH];
#pragma unroll
    for (int b = 0; b < RB; b++) {
        const int16_t *y = yrow[r0 + b];
#pragma unroll
        for (int c = 0; c < CH; c++) {
            int e = lane * 4 + c * 128;
            q[b][c] = (y && e < K) ? *(const short4 *)(y + e) : make_short4(0, 0, 0, 0);   // rows 8-byte aligned
        }
    }
#pragma unroll
    for (int b = 0; b < RB; b++) {
#pragma unroll
        for (int c = 0; c < CH; c++) {
            int e = lane * 4 + c * 128;
            if (e >= K) continue;
            const float *gm = gain + e;
            *(uint2 *)(res + swz<TN>(r0 + b, e)) = pack4(gm[0] * (float)q[b][c].x, gm[1] * (float)q[b][c].y,
                                                     gm[2] * (float)q[b][c].z, gm[3] * (float)q[b][c].w);
        }
    }
}

template <bool LEAN, int TN = NT>
static __device__ __noinline__ void build_tokens(const GemmArgs &g, int m0, uint8_t *res, const int16_t *const *yrow)
{
    const int warp = threadIdx.x >> 5;
    const int K = g.K, M = g.M, r0 = warp * (TN / 8);
    const float *gain = g.a_gain;
    if constexpr (TN == 32) {                          // four rows per warp
        if (g.asrc == A_NORM) {
            if (K <= 384) norm_rows<4, 3, TN>(g.xrows, gain, K, M, m0, r0, res);
            else norm_rows<4, 4, TN>(g.xrows, gain, K, M, m0, r0, res);
        } else {
            embed_rows<4, TN>(gain, K, r0, res, yrow);
        }
        return;
    }
    if (g.asrc == A_NORM) {
        const float *xrows = g.xrows;
        if (K <= 384 && !LEAN) {
            norm_rows<8, 3>(xrows, gain, K, M, m0, r0, res);
        } else if (K <= 384) {
            norm_rows<4, 3>(xrows, gain, K, M, m0, r0, res);
            norm_rows<4, 3>(xrows, gain, K, M, m0, r0 + 4, res);
        } else {
            norm_rows<4, 4>(xrows, gain, K, M, m0, r0, res);
            norm_rows<4, 4>(xrows, gain, K, M, m0, r0 + 4, res);
        }
        return;
    }
    if (!LEAN) {
        embed_rows<8>(gain, K, r0, res, yrow);
    } else {
        embed_rows<4>(gain, K, r0, res, yrow);
        embed_rows<4>(gain, K, r0 + 4, res, yrow);
    }
}

// E4M3 token operand: RMSNorm rows as norm_rows, then each row quantised
// with its own power-of-two scale (xs[r]); lane l holds elements 4l + 128c.
template <int RB, int CH, int TN = NT>
__device__ __forceinline__ void norm_rows8(const float *__restrict__ xrows, const float *__restrict__ gain, int K,
                                           int M, int m0, int r0, uint8_t *res, float *xs)
{
    const int lane = threadIdx.x & 31;
    float4 v[RB][CH], gh[CH];
    float ss[RB];
    load_gain<CH>(gain, K, gh);
    const float invK = 1.0f / (float)K;
#pragma unroll
    for (int b = 0; b < RB; b++) {
        int m = m0 + r0 + b;
        const float *x = m < M ? xrows + (long)m * K : nullptr;
#pragma unroll
        for (int c = 0; c < CH; c++) {
            int e = lane * 4 + c * 128;
            v[b][c] = (x && e < K) ? *(const float4 *)(x + e) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
#pragma unroll
    for (int b = 0; b < RB; b++) {
        ss[b] = 0.0f;
#pragma unroll
        for (int c = 0; c < CH; c++) {
            ss[b] = fmaf(v[b][c].x, v[b][c].x, ss[b]); ss[b] = fmaf(v[b][c].y, v[b][c].y, ss[b]);
            ss[b] = fmaf(v[b][c].z, v[b][c].z, ss[b]); ss[b] = fmaf(v[b][c].w, v[b][c].w, ss[b]);
        }
        ss[b] = warp_sum(ss[b]);
    }
#pragma unroll
    for (int b = 0; b < RB; b++) {
        int r = r0 + b;
        float inv = m0 + r < M ? inv_rms(ss[b], invK) : 0.0f;
        float amax = 0.0f;
#pragma unroll
        for (int c = 0; c < CH; c++) {
            int e = lane * 4 + c * 128;
            if (e >= K) continue;
            v[b][c] = make_float4(v[b][c].x * inv * gh[c].x, v[b][c].y * inv * gh[c].y, v[b][c].z * inv * gh[c].z,
                                  v[b][c].w * inv * gh[c].w);
            amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v[b][c].x), fabsf(v[b][c].y)), fmaxf(fabsf(v[b][c].z), fabsf(v[b][c].w))));
        }
        float qm, sc = row_scale_e4m3(warp_max(amax), &qm);
#pragma unroll
        for (int c = 0; c < CH; c++) {
            int e = lane * 4 + c * 128;
            if (e >= K) continue;
            *(uint32_t *)(res + swz8<TN>(r, e)) = e4m3x4(v[b][c].x * qm, v[b][c].y * qm, v[b][c].z * qm, v[b][c].w * qm);
        }
        if (lane == 0) xs[r] = sc;
    }
}

// E4M3 token operand from compact bf16 rows A[m][lda] (K <= 256 CH): lane l
// holds elements 8l + 256c of RB rows.
template <int RB, int CH, int TN = NT>
__device__ __forceinline__ void quant_rows8(const __nv_bfloat16 *__restrict__ A, int lda, int K, int M, int m0,
                                            int r0, uint8_t *res, float *xs)
{
    const int lane = threadIdx.x & 31;
    uint4 q[RB][CH];
#pragma unroll
    for (int b = 0; b < RB; b++) {
        int m = m0 + r0 + b;
        const __nv_bfloat16 *row = m < M ? A + (long)m * lda : nullptr;
#pragma unroll
        for (int c = 0; c < CH; c++) {
            int e = lane * 8 + c * 256;
            q[b][c] = (row && e < K) ? *(const uint4 *)(row + e) : make_uint4(0, 0, 0, 0);
        }
    }
#pragma unroll
    for (int b = 0; b < RB; b++) {
        float amax = 0.0f;
#pragma unroll
        for (int c = 0; c < CH; c++) {
            const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&q[b][c]);
#pragma unroll
            for (int i = 0; i < 4; i++) {
                float2 f = __bfloat1622float2(h[i]);
                amax = fmaxf(amax, fmaxf(fabsf(f.x), fabsf(f.y)));
            }
        }
        float qm, sc = row_scale_e4m3(warp_max(amax), &qm);
        const int r = r0 + b;
#pragma unroll
        for (int c = 0; c < CH; c++) {
            int e = lane * 8 + c * 256;
            if (e >= K) continue;
            const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&q[b][c]);
            float2 f0 = __bfloat1622float2(h[0]), f1 = __bfloat1622float2(h[1]);
            float2 f2 = __bfloat1622float2(h[2]), f3 = __bfloat1622float2(h[3]);
            *(uint2 *)(res + swz8<TN>(r, e)) = make_uint2(e4m3x4(f0.x * qm, f0.y * qm, f1.x * qm, f1.y * qm),
                                                      e4m3x4(f2.x * qm, f2.y * qm, f3.x * qm, f3.y * qm));
        }
        if (lane == 0) xs[r] = sc;
    }
}

// Build the E4M3 token operand of rows m0 .. m0+63 (warp w: rows 8w ..
// 8w+7): A_NORM (K <= 512) or compact bf16 rows (A_DIRECT, K <= 1024).
// Lean tiles take four rows at a time.
template <bool LEAN, int TN = NT>
static __device__ __noinline__ void build_tokens8(const GemmArgs &g, int m0, uint8_t *res, float *xs)
{
    const int r0 = (threadIdx.x >> 5) * (TN / 8);
    if constexpr (TN == 32) {                          // four rows per warp
        if (g.asrc == A_NORM) {
            if (g.K <= 384) norm_rows8<4, 3, TN>(g.xrows, g.a_gain, g.K, g.M, m0, r0, res, xs);
            else norm_rows8<4, 4, TN>(g.xrows, g.a_gain, g.K, g.M, m0, r0, res, xs);
        } else {
            const __nv_bfloat16 *A = (const __nv_bfloat16 *)g.A;
            if (g.K <= 512) quant_rows8<4, 2, TN>(A, g.lda, g.K, g.M, m0, r0, res, xs);
            else quant_rows8<4, 4, TN>(A, g.lda, g.K, g.M, m0, r0, res, xs);
        }
        return;
    }
    if (g.asrc == A_NORM) {
        if (g.K <= 384 && !LEAN) {
            norm_rows8<8, 3>(g.xrows, g.a_gain, g.K, g.M, m0, r0, res, xs);
        } else if (g.K <= 384) {
            norm_rows8<4, 3>(g.xrows, g.a_gain, g.K, g.M, m0, r0, res, xs);
            norm_rows8<4, 3>(g.xrows, g.a_gain, g.K, g.M, m0, r0 + 4, res, xs);
        } else {
            norm_rows8<4, 4>(g.xrows, g.a_gain, g.K, g.M, m0, r0, res, xs);
            norm_rows8<4, 4>(g.xrows, g.a_gain, g.K, g.M, m0, r0 + 4, res, xs);
        }
        return;
    }
    const __nv_bfloat16 *A = (const __nv_bfloat16 *)g.A;
    if (LEAN) {
        if (g.K <= 512) {
            quant_rows8<4, 2>(A, g.lda, g.K, g.M, m0, r0, res, xs);
            quant_rows8<4, 2>(A, g.lda, g.K, g.M, m0, r0 + 4, res, xs);
        } else {
            for (int b = 0; b < 8; b += 2) quant_rows8<2, 4>(A, g.lda, g.K, g.M, m0, r0 + b, res, xs);
        }
    } else if (g.K <= 512) {
        quant_rows8<8, 2>(A, g.lda, g.K, g.M, m0, r0, res, xs);                 // every load in flight at once
    } else {
        quant_rows8<8, 4>(A, g.lda, g.K, g.M, m0, r0, res, xs);
    }
}

// Per-token addresses a mode needs, resolved once per tile by threads 0..63:
// cache rows (EPI_STORE into a cache, EPI_QKV), the hyperprior row
// (EPI_RESID_BASE, EPI_SET_BIAS with eh_out), the head outputs (EPI_HEADS),
// the latents (A_EMBED) or z-hat (A_ZHAT).  Entry r of a tile's token table
// (row m0 + r): tab[k][r * ts] for k < 4 (ts: the table's row stride) and,
// for A_EMBED / A_ZHAT, the operand's source row.
template <int MODE>
__device__ __forceinline__ void table_row(const GemmArgs &g, int m0, int r, uintptr_t *tab, int ts,
                                          const int16_t **yrow)
{
    int m = m0 + r;
    tab[r] = tab[ts + r] = tab[2 * ts + r] = tab[3 * ts + r] = 0;
    if (yrow) yrow[r] = nullptr;
    const Epi &e = g.epi;
    if (m >= g.M || !e.tok) return;
    int tk = e.tok[m];
    const Slot &s = e.slots[tok_slot(tk)];
    int p = tok_pos(tk);
    if (yrow && g.asrc == A_EMBED) yrow[r] = s.y + (long)p * g.K;
    if (yrow && g.asrc == A_ZHAT) {
        const int i = p / s.W, j = p - i * s.W, Wh = (s.W + e.hr - 1) / e.hr;
        yrow[r] = s.zhat + ((long)(i / e.hr) * Wh + j / e.hr) * g.K;
    }
    if (MODE == EPI_STORE && e.st_sel != CS_NONE) {
        tab[r] = (uintptr_t)cache_row<__nv_bfloat16>(s, e.st_sel, e.st_layer, p, e.d);
    } else if (MODE == EPI_QKV) {
        int layer = e.ring ? e.kv_layer * e.Tf + s.ring[s.nfr - 1] : e.kv_layer;
        tab[r] = (uintptr_t)cache_row<__nv_bfloat16>(s, e.kc_sel, layer, p, e.d);
        tab[ts + r] = (uintptr_t)cache_row<__nv_bfloat16>(s, e.vc_sel, layer, p, e.d);
    } else if (MODE == EPI_RESID_BASE || (MODE == EPI_SET_BIAS && e.eh_out)) {
        tab[ts + r] = (uintptr_t)(s.eh + (long)p * g.N);
    } else if (MODE == EPI_HEADS) {
        const long o = (long)p * e.C + e.c0;
        tab[r] = (uintptr_t)(s.mu + o);
        tab[ts + r] = (uintptr_t)(s.sigma + o);
        tab[2 * ts + r] = (uintptr_t)(s.idx + o);
        tab[3 * ts + r] = (uintptr_t)(s.m + o);
    }
}

template <int MODE, int TN = NT>
__device__ __forceinline__ void build_table(const GemmArgs &g, int m0, GemmShared &S)
{
    int r = threadIdx.x;
    if (r < TN) table_row<MODE>(g, m0, r, &S.tab[0][0], NT, S.yrow);
}

// The value of output (feature f, token) from its accumulator y (and the
// up projection's y2 for the dual form), as the epilogue mode defines it
// (bf / ga, gb: the feature's bias, or the heads' channel-wise scale and
// offset); *oi: the heads' scale index or rounded mean.  Every epilogue of
// every kernel goes through this one definition.
template <int MODE, bool DUAL>
__device__ __forceinline__ float epi_value(float y, float y2, int f, float bf, float ga, float gb,
                                           const float *stab, int *oi)
{
    *oi = 0;
    if (MODE == EPI_HEADS) {
        if (f & 1) {
            float sg = expf(fminf(fmaxf(ga * y + gb, LN_SIG_LO), LN_SIG_HI));
            *oi = scale_index(stab, sg);
            return sg;
        }
        float mu = ga * y + gb;
        *oi = (int)rintf(fminf(fmaxf(mu, -32768.0f), 32767.0f));
        return mu;
    }
    if (MODE == EPI_SET_BIAS) return y + bf;
    if (MODE == EPI_BIAS_SILU) return silu_fast(y + bf);
    if (MODE == EPI_SWIGLU) return DUAL ? silu_fast(y) * y2 : y;
    return y;
}

// A warp's 32 features (f0w + lane) x 8 tokens (rows m0 + c0 .. + 7) of a
// bf16-output mode, o[j] = the lane's value for token c0 + j: staged in
// shared memory (stg: 512 bytes of this warp) so that each lane stores 8
// consecutive features of one token in one 16-byte write.  tab, ts: the
// tile's token table (cache rows).
template <int MODE>
__device__ __forceinline__ void store_bf16_8(const Epi &e, int M, int N, int m0, int c0, int f0w,
                                             const float *o, uint16_t *stg, const uintptr_t *tab, int ts)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        __nv_bfloat16 b = __float2bfloat16_rn(o[j]);
        stg[j * 32 + lane] = *reinterpret_cast<uint16_t *>(&b);
    }
    __syncwarp();
    const int jr = lane >> 2, fc = (lane & 3) * 8;
    const uint4 val = *reinterpret_cast<const uint4 *>(stg + jr * 32 + fc);
    __syncwarp();
    const int r = c0 + jr, m = m0 + r, fb = f0w + fc;
    if (m < M && fb < N) {
        __nv_bfloat16 *dst;
        if (MODE == EPI_STORE)
            dst = e.st_sel == CS_NONE ? (__nv_bfloat16 *)e.out + (long)m * e.ld_out + fb
                                      : (__nv_bfloat16 *)tab[r] + fb;
        else if (MODE == EPI_QKV)
            dst = fb < e.q_cols ? (__nv_bfloat16 *)e.out + (long)m * e.ld_out + fb
                  : fb < e.q_cols + e.d ? (__nv_bfloat16 *)tab[r] + (fb - e.q_cols)
                                        : (__nv_bfloat16 *)tab[ts + r] + (fb - e.q_cols - e.d);
        else
            dst = (__nv_bfloat16 *)e.out + (long)m * e.ld_out + fb;
        if (fb + 8 <= N) {
            *reinterpret_cast<uint4 *>(dst) = val;
        } else {
            const __nv_bfloat16 *pv = reinterpret_cast<const __nv_bfloat16 *>(&val);
            for (int i = 0; i < N - fb; i++) dst[i] = pv[i];
        }
    }
}

// The epilogue of a tile: wait for the MMAs, read the accumulator from TMEM
// and write the mode's outputs.  Thread t holds feature row f0 + 32 (w % 4)
// + lane (w = its warp) and token columns 32 (w / 4) .. + 31.  Residual
// modes read the rows they update while the MMAs still run.  Other modes
// walk their columns 8 at a time in a rolled loop and, per group, compute
// every value before storing any (the output pointers are generic, so each
// store could alias later loads).  Out of line: one copy per mode, small
// enough to stay in the instruction cache.
template <bool DUAL, int MODE, bool F8, bool LEAN, int TN>
static __device__ __noinline__ void gemm_epilogue(GemmShared &S, uint8_t *ring, uint32_t tmem, const GemmArgs &g,
                                                  int f0, int m0, GemmPipe &pp)
{
    constexpr bool RESID = MODE == EPI_RESID || MODE == EPI_RESID_BASE;
    constexpr int PRE = LEAN ? TN / 4 : TN / 2;                    // residual values read before the MMAs end
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int M = g.M, N = g.N;
    const Epi e = g.epi;
    const int f = f0 + (warp & 3) * 32 + lane;
    const bool fok = f < N;
    const int cb = (warp >> 2) * (TN / 2);
    float old[RESID ? TN / 2 : 1];
    if constexpr (RESID) {
#pragma unroll
        for (int j = 0; j < PRE; j++) {
            const int r = cb + j, m = m0 + r;
            const float *src = MODE == EPI_RESID ? e.rows + (long)m * N : (const float *)S.tab[1][r];
            old[j] = (fok && m < M) ? src[f] : 0.0f;
        }
    }
    bool ok = mbar_wait(&S.done, pp.ntile & 1);
    if (!ok) S.abort = 1;
    fence_after();
    __syncthreads();
    pp.ntile++;
    if (S.abort) {
        fence_before();
        __syncthreads();
        return;
    }
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    // E4M3: dequantisation scales of the feature row (both products below
    // are of powers of two, hence exact)
    float wf = 1.0f, wf2 = 1.0f;
    if constexpr (F8) {
        if (fok) { wf = g.wsc[f]; if (DUAL) wf2 = g.wsc2[f]; }
    }
    if constexpr (RESID) {
#pragma unroll
        for (int h = 0; h < TN / 32; h++) {
            if (h * 16 >= PRE) {
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int r = cb + 16 * h + j, m = m0 + r;
                    const float *src = MODE == EPI_RESID ? e.rows + (long)m * N : (const float *)S.tab[1][r];
                    old[16 * h + j] = (fok && m < M) ? src[f] : 0.0f;
                }
            }
            float v[16];
            tmem_get16(trow + cb + 16 * h, v);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                if constexpr (F8) v[j] *= wf * S.xs[cb + 16 * h + j];
                const int m = m0 + cb + 16 * h + j;
                if (fok && m < M) e.rows[(long)m * N + f] = old[16 * h + j] + v[j];
            }
        }
    } else {
        // per-feature constants; heads: even feature rows give mu of channel
        // f / 2, odd rows its sigma
        float bf = 0.0f, ga = 0.0f, gb = 0.0f;
        if ((MODE == EPI_SET_BIAS || MODE == EPI_BIAS_SILU) && fok) bf = e.bias[f];
        if (MODE == EPI_HEADS && fok) {
            ga = (f & 1) ? e.gsg[f >> 1] : e.gmu[f >> 1];
            gb = (f & 1) ? e.bsg[f >> 1] : e.bmu[f >> 1];
        }
#pragma unroll 1
        for (int c0 = cb; c0 < cb + TN / 2; c0 += 8) {
            float v[8], v2[8], o[8];
            int oi[8];
            if (DUAL) tmem_get8x2(trow + c0, trow + TN + c0, v, v2);
            else tmem_get8(trow + c0, v);
            if constexpr (F8) {
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const float t = S.xs[c0 + j];
                    v[j] *= wf * t;
                    if (DUAL) v2[j] *= wf2 * t;
                }
            }
#pragma unroll
            for (int j = 0; j < 8; j++) o[j] = epi_value<MODE, DUAL>(v[j], DUAL ? v2[j] : 0.0f, f, bf, ga, gb, S.stab, &oi[j]);
            if constexpr (MODE == EPI_HEADS || MODE == EPI_SET_BIAS) {
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const int r = c0 + j, m = m0 + r;
                    if (!(fok && m < M)) continue;
                    const float y = o[j];
                    if (MODE == EPI_HEADS) {
                        const int c = f >> 1;
                        if (f & 1) {
                            ((float *)S.tab[1][r])[c] = y;
                            ((uint8_t *)S.tab[2][r])[c] = (uint8_t)oi[j];
                        } else {
                            ((float *)S.tab[0][r])[c] = y;
                            ((int32_t *)S.tab[3][r])[c] = oi[j];
                        }
                    } else if (e.eh_out) {
                        ((float *)S.tab[1][r])[f] = y;
                    } else {
                        e.rows[(long)m * N + f] = y;
                    }
                }
            } else {
                // bf16 rows through shared memory (the ring, idle now)
                store_bf16_8<MODE>(e, M, N, m0, c0, f0 + (warp & 3) * 32, o, (uint16_t *)(ring + warp * 512),
                                   &S.tab[0][0], NT);
            }
        }
    }
    // the ring is written by tensor copies again after this
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
}

// Everything of a tile that does not depend on data written by earlier work:
// the token table (threads 0..63), the scale table, and the weight copies of
// the ring's stages (stage s issued by lane 0 of warp s: one thread issues a
// tensor copy only every ~150 ns).  Returns the number of stages filled.  The
// caller synchronises the CTA before gemm_tile_main.
template <bool DUAL, int MODE, bool F8 = false, bool LEAN = false, int TN = NT>
__device__ __forceinline__ int gemm_tile_pre(GemmShared &S, uint8_t *ring, const CUtensorMap *tmW,
                                             const CUtensorMap *tmW2, const GemmArgs &g, int f0, int m0,
                                             GemmPipe &pp)
{
    constexpr int KCH = kchunk(F8);
    if (MODE == EPI_HEADS && threadIdx.x < NSCALES) S.stab[threadIdx.x] = g.epi.scale[threadIdx.x];
    build_table<MODE, TN>(g, m0, S);
    const bool resident = F8 || g.asrc != A_DIRECT;
    const int stage = stage_bytes(DUAL, resident, TN);
    const int nst = ring_stages(DUAL, resident, g.K, F8, LEAN, TN);
    const int s = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0 && s < nst) {
        // the ring is idle between tiles (the previous tile's MMAs are done)
        uint8_t *st = ring + s * stage;
        mbar_expect_tx(&S.full[s], stage);
        tma_load(st, tmW, &S.full[s], s * KCH, f0);
        if (DUAL) tma_load(st + A_BYTES, tmW2, &S.full[s], s * KCH, f0);
    }
    return nst;
}

// The rest of a tile, after the caller's wait for its inputs and a CTA
// barrier: token operand, MMAs, epilogue.  `first` is gemm_tile_pre's
// result.  Roles: lane 0 of warp 1 issues the MMAs into the accumulator (the
// gate accumulator of the dual form, whose up accumulator lane 0 of warp 2
// feeds); lane 0 of warps 0, 5, 6 and 7 issue the copies of the chunks past
// the first ring fill, each the refills of its own stages.
template <bool DUAL, int MODE, bool F8 = false, bool LEAN = false, int TN = NT>
__device__ __forceinline__ void gemm_tile_main(GemmShared &S, uint8_t *ring, uint32_t tmem, const CUtensorMap *tmW,
                                               const CUtensorMap *tmW2, const CUtensorMap *tmX, const GemmArgs &g,
                                               int f0, int m0, int first, GemmPipe &pp)
{
    constexpr int NACC = DUAL ? 2 : 1;
    constexpr int KCH = kchunk(F8);
    const bool resident = F8 || g.asrc != A_DIRECT;
    const int stage = stage_bytes(DUAL, resident, TN);
    const int nk = kchunks(g.K, F8), nst = ring_stages(DUAL, resident, g.K, F8, LEAN, TN);
    uint8_t *res = ring + nst * stage;                             // resident token operand
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const bool producer = lane == 0 && (warp == 0 || warp > 4);
    const int p = warp == 0 ? 0 : warp - 4;                        // producer index
    if (!resident && producer) {
        // the first fill's token chunks, spread over the producers (the MMA
        // issuers go straight to their loops)
        fence_proxy_global();
        for (int s = p; s < first; s += NPROD)
            tma_load(ring + s * stage + NACC * A_BYTES, tmX, &S.full[s], s * KC, m0);
    }
    if (resident) {
        if (F8) build_tokens8<LEAN, TN>(g, m0, res, S.xs);
        else build_tokens<LEAN, TN>(g, m0, res, S.yrow);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }

    if (producer) {
        // producers: every refill of stage s comes from producer s % NPROD,
        // in chunk order, so a producer waits for a stage's release only
        // after issuing (or seeing issued) the fill before it: the release it
        // waits for is never more than one phase ahead of the barrier
        int jend = first;
        for (int j = first; j < nk; j++) {
            int s = j % nst, u = j / nst;
            if (s % NPROD != p) continue;
            if (S.abort) break;
            if (!mbar_wait(&S.empty[s], release_parity(pp, s, u))) { S.abort = 1; break; }
            uint8_t *st = ring + s * stage;
            mbar_expect_tx(&S.full[s], stage);
            tma_load(st, tmW, &S.full[s], j * KCH, f0);
            if (DUAL) tma_load(st + A_BYTES, tmW2, &S.full[s], j * KCH, f0);
            if (!resident) tma_load(st + NACC * A_BYTES, tmX, &S.full[s], j * KC, m0);
            jend = j + 1;
        }
        if (S.abort) {
            // let this producer's copies land before the CTA can go on or exit
            for (int j = first; j < jend; j++)
                if ((j % nst) % NPROD == p) mbar_wait(&S.full[j % nst], fill_parity(pp, j % nst, j / nst));
        }
    } else if (lane == 0 && (warp == 1 || (DUAL && warp == 2))) {
        // MMA issuers: every K step of every chunk, in ascending K, into one
        // accumulator (the output element's only summation order, whatever
        // the tile shape, the launch or the kernel).  The dual form's up
        // projection has its own issuer; a single issuer commits twice, so
        // a stage that is filled again in this tile is released, and the
        // tile finished, after two commits either way.
        const uint32_t id = F8 ? idesc_e4m3(TM, TN) : idesc_bf16(TM, TN);
        const uint32_t acc = tmem + (warp == 2 ? (uint32_t)TN : 0u);
        const uint32_t aoff = warp == 2 ? (uint32_t)A_BYTES : 0u;
        for (int j = 0; j < nk; j++) {
            int s = j % nst, u = j / nst;
            if (S.abort) break;
            if (!mbar_wait(&S.full[s], fill_parity(pp, s, u))) { S.abort = 1; break; }
            fence_after();
            uint32_t base = su32(ring + s * stage) + aoff;
            uint32_t bb = resident ? su32(res) + j * tok_chunk_bytes(TN) : su32(ring + s * stage) + NACC * A_BYTES;
            // four K steps of 32 bytes along the 128-byte rows (16 bf16 or 32 E4M3 each)
#pragma unroll
            for (int q = 0; q < 4; q++) {
                if (F8) mma8(acc, sdesc(base + q * 32), sdesc(bb + q * 32), id, (j | q) != 0);
                else mma(acc, sdesc(base + q * 32), sdesc(bb + q * 32), id, (j | q) != 0);
            }
            if (j + nst < nk) {                                        // the stage is filled again in this tile
                mma_commit(&S.empty[s]);
                if (!DUAL) mma_commit(&S.empty[s]);
            }
        }
        mma_commit(&S.done);
        if (!DUAL) mma_commit(&S.done);
    }
    __syncwarp();
    gemm_epilogue<DUAL, MODE, F8, LEAN, TN>(S, ring, tmem, g, f0, m0, pp);
    pipe_advance(pp, nk, nst);
}

}  // namespace tc

// A tensor map of the 2D bf16 array [rows][ld] (K used columns), box of
// box_rows x 64 elements (x 128 bytes for an E4M3 array, f8), 128-byte
// swizzle, rows and columns past the end read as zero (cached per argument
// tuple; host).
bool gemm_tensor_map(const void *ptr, int rows, int K, int ld, int box_rows, CUtensorMap *out, bool f8 = false);

}  // namespace psw
