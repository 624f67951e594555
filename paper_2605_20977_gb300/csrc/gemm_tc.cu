// gemm_tc.cu -- BF16 projection GEMM on the sm_100-family tensor cores
// (tcgen05.mma, accumulator in tensor memory, weights staged by TMA).
//
// Y[token][feature] = sum_k X[token][k] Wt[feature][k].  The projection is
// the MMA's A operand (M = 128 output features per CTA) and the tokens are
// its B operand (N = 64 tokens per CTA), so a decoder step with a few dozen
// tokens fills one tile and the weights stream through once.  Weights are
// consumed in 64-element K chunks (one 128-byte swizzle atom) through a
// 4-stage TMA ring.  The token operand either streams through the same ring
// (compact bf16 rows) or is built once per CTA in shared memory by the CTA
// itself: RMSNorm of the FP32 residual stream rows (the pre-norm of every
// projection, Sec. 3.1) or the channel-scaled latents (the latent
// embedding).  One thread issues the MMAs; 128 threads run the epilogue from
// TMEM (thread t holds feature row t of the tile) with the destination rows
// of the tile's tokens resolved once into shared memory.  Accumulation order
// is fixed (ascending K chunks), so every output element is the same function
// of its row and column whatever the tile or launch it falls in.
//
// Every mbarrier wait is bounded (~2 s of globaltimer); on expiry the CTA
// records ST_TIMEOUT, waits (bounded) for its own copies and MMAs, frees its
// tensor memory and returns.
#include "internal.h"
#include "device_common.cuh"

#include <cuda.h>

#include <map>
#include <mutex>
#include <tuple>

namespace psw {

namespace {

constexpr int TM = 128;        // output features per CTA (MMA M)
constexpr int NT = 64;         // tokens per CTA (MMA N)
constexpr int KC = 64;         // K elements per stage (128 bytes of bf16)
constexpr int STAGES = 4;
constexpr int A_BYTES = TM * KC * 2;
constexpr int B_BYTES = NT * KC * 2;
constexpr int KRES_MAX = 512;  // largest K of a token operand built in shared memory
constexpr int TAB_BYTES = 4 * NT * 8;
constexpr uint64_t WAIT_NS = 2000000000ull;

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

// Bounded wait on a phase of an mbarrier; false after ~2 s.
__device__ __noinline__ bool mbar_wait(uint64_t *b, uint32_t parity)
{
    if (mbar_try(b, parity)) return true;
    uint64_t t0 = gtime();
    while (!mbar_try(b, parity))
        if (gtime() - t0 > WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *tm, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(su32(dst)), "l"(tm), "r"(su32(bar)), "r"(x), "r"(y)
        : "memory");
}

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

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t addr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row r, column k) of a K-major bf16 operand laid
// out in 128-byte-swizzled atoms of 64 columns x NT rows.
__device__ __forceinline__ uint32_t swz(int r, int k)
{
    int kc = k >> 6, col = k & 63;
    uint32_t byte = (uint32_t)col * 2;
    return (uint32_t)kc * B_BYTES + (uint32_t)r * 128 + ((((byte >> 4) ^ (uint32_t)(r & 7))) << 4) + (byte & 15);
}

__device__ __forceinline__ uint2 pack4(float a, float b, float c, float d)
{
    __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    return make_uint2(*reinterpret_cast<uint32_t *>(&lo), *reinterpret_cast<uint32_t *>(&hi));
}

constexpr int NTHREADS = 256;  // 8 warps: warps w and w + 4 share TMEM lanes 32 (w % 4) .. + 31

// Build the token operand of rows m0 .. m0+63 in shared memory; rows past M
// are zero.  A_NORM: RMSNorm of the FP32 rows xrows[m] times the gain (warp w
// normalises rows 8w .. 8w+7, four at a time with all their loads issued
// first); A_EMBED: the channel-scaled latents of the token (row pointers
// resolved beforehand into yrow).
__device__ void build_tokens(const GemmArgs &g, int m0, uint8_t *res, const int16_t *const *yrow)
{
    constexpr int RB = 4;                              // rows in flight per warp
    constexpr int CH = KRES_MAX / 128;                 // float4 chunks per lane and row, at most
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nch = (g.K + 127) / 128;
    for (int r0 = warp * (NT / 8); r0 < (warp + 1) * (NT / 8); r0 += RB) {
        if (g.asrc == A_NORM) {
            float4 v[RB][CH];
            float ss[RB];
#pragma unroll
            for (int b = 0; b < RB; b++) {
                int m = m0 + r0 + b;
                const float *x = m < g.M ? g.xrows + (long)m * g.K : nullptr;
                ss[b] = 0.0f;
#pragma unroll
                for (int c = 0; c < CH; c++) {
                    int e = lane * 4 + c * 128;
                    v[b][c] = (x && c < nch && e < g.K) ? *(const float4 *)(x + e) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int b = 0; b < RB; b++) {
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
                float inv = m0 + r < g.M ? 1.0f / sqrtf(ss[b] / (float)g.K + 1e-6f) : 0.0f;
#pragma unroll
                for (int c = 0; c < CH; c++) {
                    int e = lane * 4 + c * 128;
                    if (c >= nch || e >= g.K) continue;
                    const float *gn = g.a_gain + e;            // gains sit at any float offset
                    *(uint2 *)(res + swz(r, e)) = pack4(v[b][c].x * inv * gn[0], v[b][c].y * inv * gn[1],
                                                        v[b][c].z * inv * gn[2], v[b][c].w * inv * gn[3]);
                }
            }
        } else {
#pragma unroll
            for (int b = 0; b < RB; b++) {
                int r = r0 + b;
                const int16_t *y = yrow[r];
                for (int e = lane * 4; e < g.K; e += 128) {
                    short4 q = y ? *(const short4 *)(y + e) : make_short4(0, 0, 0, 0);   // rows 8-byte aligned
                    const float *gm = g.a_gain + e;
                    *(uint2 *)(res + swz(r, e)) = pack4(gm[0] * (float)q.x, gm[1] * (float)q.y, gm[2] * (float)q.z,
                                                        gm[3] * (float)q.w);
                }
            }
        }
    }
}

// Per-token addresses a mode needs, resolved once per CTA by threads 0..63:
// cache rows (EPI_STORE into a cache, EPI_QKV), the hyperprior row
// (EPI_RESID_BASE), the head outputs (EPI_HEADS), the latents (A_EMBED).
template <int MODE>
__device__ void build_table(const GemmArgs &g, int m0, uintptr_t (*tab)[NT], const int16_t **yrow)
{
    int r = threadIdx.x;
    if (r >= NT) return;
    int m = m0 + r;
    tab[0][r] = tab[1][r] = tab[2][r] = tab[3][r] = 0;
    yrow[r] = nullptr;
    const Epi &e = g.epi;
    if (m >= g.M || !e.tok) return;
    int tk = e.tok[m];
    const Slot &s = e.slots[tok_slot(tk)];
    int p = tok_pos(tk);
    if (g.asrc == A_EMBED) yrow[r] = s.y + (long)p * g.K;
    if (MODE == EPI_STORE && e.st_sel != CS_NONE) {
        tab[0][r] = (uintptr_t)cache_row<__nv_bfloat16>(s, e.st_sel, e.st_layer, p, e.d);
    } else if (MODE == EPI_QKV) {
        int layer = e.ring ? e.kv_layer * e.Tf + s.ring[s.nfr - 1] : e.kv_layer;
        tab[0][r] = (uintptr_t)cache_row<__nv_bfloat16>(s, e.kc_sel, layer, p, e.d);
        tab[1][r] = (uintptr_t)cache_row<__nv_bfloat16>(s, e.vc_sel, layer, p, e.d);
    } else if (MODE == EPI_RESID_BASE) {
        tab[1][r] = (uintptr_t)(s.eh + (long)p * g.N);
    } else if (MODE == EPI_HEADS) {
        tab[0][r] = (uintptr_t)(s.mu + (long)p * e.C);
        tab[1][r] = (uintptr_t)(s.sigma + (long)p * e.C);
        tab[2][r] = (uintptr_t)(s.idx + (long)p * e.C);
        tab[3][r] = (uintptr_t)(s.m + (long)p * e.C);
    }
}

template <bool DUAL, int MODE>
__global__ void __launch_bounds__(NTHREADS, 1)
k_gemm_tc(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmW2,
          const __grid_constant__ CUtensorMap tmX, GemmArgs g, int *status)
{
    constexpr int NACC = DUAL ? 2 : 1;
    constexpr uint32_t TCOLS = DUAL ? 2 * NT : NT;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    __shared__ float stab[NSCALES];
    __shared__ const int16_t *yrow[NT];

    const bool resident = g.asrc != A_DIRECT;
    const int stage = NACC * A_BYTES + (resident ? 0 : B_BYTES);
    const int nk = g.K / KC;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *res = smem + STAGES * stage;                          // resident token operand
    uintptr_t(*tab)[NT] = (uintptr_t(*)[NT])(res + (resident ? nk * B_BYTES : 0));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int f0 = blockIdx.x * TM, m0 = blockIdx.y * NT;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    pdl_trigger();
    // token lists, the slot table and the scale table are fixed for the
    // whole decode: read them before waiting for the previous kernel
    if (MODE == EPI_HEADS && threadIdx.x < NSCALES) stab[threadIdx.x] = g.epi.scale[threadIdx.x];
    build_table<MODE>(g, m0, tab, yrow);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;

    // the first stages' weight copies start before the previous kernel ends
    const int first = nk < STAGES ? nk : STAGES;
    if (threadIdx.x == 0) {
        for (int kc = 0; kc < first; kc++) {
            uint8_t *st = smem + kc * stage;
            mbar_expect_tx(&full[kc], stage);
            tma_load(st, &tmW, &full[kc], kc * KC, f0);
            if (DUAL) tma_load(st + A_BYTES, &tmW2, &full[kc], kc * KC, f0);
        }
    }
    pdl_wait();                                        // activations are ready from here on
    if (threadIdx.x == 0 && !resident)
        for (int kc = 0; kc < first; kc++) tma_load(smem + kc * stage + NACC * A_BYTES, &tmX, &full[kc], kc * KC, m0);
    if (resident) {
        build_tokens(g, m0, res, yrow);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }

    if (warp == 0 && lane == 0) {
        // producer: remaining stages of the TMA ring
        int issued = first;
        for (int kc = first; kc < nk; kc++) {
            int s = kc % STAGES, it = kc / STAGES;
            if (abort_flag) break;
            if (!mbar_wait(&empty[s], (it - 1) & 1)) { abort_flag = 1; break; }
            uint8_t *st = smem + s * stage;
            mbar_expect_tx(&full[s], stage);
            tma_load(st, &tmW, &full[s], kc * KC, f0);
            if (DUAL) tma_load(st + A_BYTES, &tmW2, &full[s], kc * KC, f0);
            if (!resident) tma_load(st + NACC * A_BYTES, &tmX, &full[s], kc * KC, m0);
            issued = kc + 1;
        }
        if (abort_flag) {
            // let this CTA's copies land before it can exit
            for (int kc = (issued > STAGES ? issued - STAGES : 0); kc < issued; kc++)
                mbar_wait(&full[kc % STAGES], (kc / STAGES) & 1);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t id = idesc_bf16(TM, NT);
        for (int kc = 0; kc < nk; kc++) {
            int s = kc % STAGES, it = kc / STAGES;
            if (abort_flag) break;
            if (!mbar_wait(&full[s], it & 1)) { abort_flag = 1; break; }
            fence_after();
            uint32_t base = su32(smem + s * stage);
            uint32_t bb = resident ? su32(res) + kc * B_BYTES : base + NACC * A_BYTES;
#pragma unroll
            for (int k = 0; k < KC / 16; k++) {
                uint32_t acc = (kc | k) != 0;
                mma(tmem, sdesc(base + k * 32), sdesc(bb + k * 32), id, acc);
                if (DUAL) mma(tmem + NT, sdesc(base + A_BYTES + k * 32), sdesc(bb + k * 32), id, acc);
            }
            mma_commit(&empty[s]);
        }
        mma_commit(&done);
    }
    __syncwarp();
    bool ok = mbar_wait(&done, 0);
    if (!ok) abort_flag = 1;
    fence_after();
    __syncthreads();
    if (abort_flag) {
        if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
    } else {
        const Epi &e = g.epi;
        const int f = f0 + (warp & 3) * 32 + lane;
        const bool fok = f < g.N;
        const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        for (int c0 = (warp >> 2) * (NT / 2); c0 < (warp >> 2) * (NT / 2) + NT / 2; c0 += 16) {
            float v[16], v2[16];
            tmem_ld16(trow + c0, v);
            if (DUAL) tmem_ld16(trow + NT + c0, v2);
            if (MODE == EPI_RESID || MODE == EPI_RESID_BASE) {
                // every read first, then the stores: independent round trips
                float old[16];
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int r = c0 + j, m = m0 + r;
                    const bool okm = fok && m < g.M;
                    const float *src = MODE == EPI_RESID ? e.rows + (long)m * g.N : (const float *)tab[1][r];
                    old[j] = okm ? src[f] : 0.0f;
                }
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int m = m0 + c0 + j;
                    if (fok && m < g.M) e.rows[(long)m * g.N + f] = old[j] + v[j];
                }
                continue;
            }
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int r = c0 + j, m = m0 + r;
                const bool okm = fok && m < g.M;
                const float y = v[j];
                if (MODE == EPI_HEADS) {
                    float part = __shfl_xor_sync(0xffffffffu, y, 1);
                    if (okm && !(f & 1)) {
                        int c = f >> 1;
                        float mu = e.gmu[c] * y + e.bmu[c];
                        float sg = expf(fminf(fmaxf(e.gsg[c] * part + e.bsg[c], LN_SIG_LO), LN_SIG_HI));
                        ((float *)tab[0][r])[c] = mu;
                        ((float *)tab[1][r])[c] = sg;
                        int l = NSCALES - 1;
                        for (int t = 0; t < NSCALES; t++)
                            if (stab[t] >= sg) { l = t; break; }
                        ((uint8_t *)tab[2][r])[c] = (uint8_t)l;
                        ((int32_t *)tab[3][r])[c] = (int32_t)rintf(fminf(fmaxf(mu, -32768.0f), 32767.0f));
                    }
                } else if (!okm) {
                    continue;
                } else if (MODE == EPI_STORE) {
                    if (e.st_sel == CS_NONE) ((__nv_bfloat16 *)e.out)[(long)m * e.ld_out + f] = __float2bfloat16_rn(y);
                    else ((__nv_bfloat16 *)tab[0][r])[f] = __float2bfloat16_rn(y);
                } else if (MODE == EPI_QKV) {
                    if (f < e.q_cols) ((__nv_bfloat16 *)e.out)[(long)m * e.ld_out + f] = __float2bfloat16_rn(y);
                    else if (f < e.q_cols + e.d) ((__nv_bfloat16 *)tab[0][r])[f - e.q_cols] = __float2bfloat16_rn(y);
                    else ((__nv_bfloat16 *)tab[1][r])[f - e.q_cols - e.d] = __float2bfloat16_rn(y);
                } else if (MODE == EPI_SET_BIAS) {
                    e.rows[(long)m * g.N + f] = y + e.bias[f];
                } else if (MODE == EPI_BIAS_SILU) {
                    ((__nv_bfloat16 *)e.out)[(long)m * e.ld_out + f] = __float2bfloat16_rn(silu_f(y + e.bias[f]));
                } else if (MODE == EPI_SWIGLU) {
                    if (DUAL) ((__nv_bfloat16 *)e.out)[(long)m * e.ld_out + f] = __float2bfloat16_rn(silu_f(y) * v2[j]);
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_mu;
EncodeTiledFn g_encode = nullptr;
std::map<std::tuple<const void *, int, int, int, int>, CUtensorMap> g_maps;

EncodeTiledFn encoder()
{
    if (!g_encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (EncodeTiledFn)fn;
    }
    return g_encode;
}

// 2D bf16 [rows][ld] (K used columns) with a box of box_rows x 64, 128-byte
// swizzle; rows past the end read as zero.
bool tensor_map(const void *ptr, int rows, int K, int ld, int box_rows, CUtensorMap *out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_tuple(ptr, rows, K, ld, box_rows);
    auto it = g_maps.find(key);
    if (it != g_maps.end()) { *out = it->second; return true; }
    EncodeTiledFn enc = encoder();
    if (!enc) return false;
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    if (g_maps.size() > 65536) g_maps.clear();
    g_maps[key] = m;
    *out = m;
    return true;
}

size_t smem_bytes(bool dual, bool resident, int K)
{
    int nacc = dual ? 2 : 1;
    size_t stage = (size_t)nacc * A_BYTES + (resident ? 0 : B_BYTES);
    return STAGES * stage + (resident ? (size_t)(K / KC) * B_BYTES : 0) + TAB_BYTES + 1024;
}

}  // namespace

bool gemm_tc_supported(int prec, int N, int K, int asrc)
{
    return prec == P_BF16 && K % KC == 0 && K >= KC && N >= 1 && (asrc == A_DIRECT || K <= KRES_MAX);
}

template <bool DUAL, int MODE>
bool set_attr(size_t bytes)
{
    return cudaFuncSetAttribute(k_gemm_tc<DUAL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
           cudaSuccess;
}

// Checks for the tensor-map entry point and raises the kernels' dynamic
// shared-memory limit (done before any stream capture).
bool gemm_tc_available()
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!encoder()) return false;
    size_t m2 = std::max(smem_bytes(true, true, KRES_MAX), smem_bytes(true, false, 0));
    size_t m1 = std::max(smem_bytes(false, true, KRES_MAX), smem_bytes(false, false, 0));
    return set_attr<true, EPI_SWIGLU>(m2) && set_attr<false, EPI_STORE>(m1) && set_attr<false, EPI_QKV>(m1) &&
           set_attr<false, EPI_RESID>(m1) && set_attr<false, EPI_RESID_BASE>(m1) &&
           set_attr<false, EPI_BIAS_SILU>(m1) && set_attr<false, EPI_SET_BIAS>(m1) && set_attr<false, EPI_HEADS>(m1);
}

bool gemm_tc(const GemmArgs &g, cudaStream_t s)
{
    CUtensorMap tw, tw2, tx;
    bool dual = g.epi.mode == EPI_SWIGLU;
    bool resident = g.asrc != A_DIRECT;
    if (!tensor_map(g.Wt, g.N, g.K, g.K, TM, &tw)) return false;
    if (dual && !tensor_map(g.Wt2, g.N, g.K, g.K, TM, &tw2)) return false;
    if (!dual) tw2 = tw;
    if (!resident) {
        if (!tensor_map(g.A, g.M, g.K, g.lda, NT, &tx)) return false;
    } else {
        tx = tw;
    }
    dim3 grid((g.N + TM - 1) / TM, (g.M + NT - 1) / NT);
    size_t smem = smem_bytes(dual, resident, g.K);
    int *st = g.status;
    dim3 block(NTHREADS);
    cudaError_t e;
    switch (g.epi.mode) {
    case EPI_SWIGLU: e = launch_pdl(k_gemm_tc<true, EPI_SWIGLU>, grid, block, smem, s, tw, tw2, tx, g, st); break;
    case EPI_STORE: e = launch_pdl(k_gemm_tc<false, EPI_STORE>, grid, block, smem, s, tw, tw2, tx, g, st); break;
    case EPI_QKV: e = launch_pdl(k_gemm_tc<false, EPI_QKV>, grid, block, smem, s, tw, tw2, tx, g, st); break;
    case EPI_RESID: e = launch_pdl(k_gemm_tc<false, EPI_RESID>, grid, block, smem, s, tw, tw2, tx, g, st); break;
    case EPI_RESID_BASE:
        e = launch_pdl(k_gemm_tc<false, EPI_RESID_BASE>, grid, block, smem, s, tw, tw2, tx, g, st);
        break;
    case EPI_BIAS_SILU:
        e = launch_pdl(k_gemm_tc<false, EPI_BIAS_SILU>, grid, block, smem, s, tw, tw2, tx, g, st);
        break;
    case EPI_SET_BIAS: e = launch_pdl(k_gemm_tc<false, EPI_SET_BIAS>, grid, block, smem, s, tw, tw2, tx, g, st); break;
    case EPI_HEADS: e = launch_pdl(k_gemm_tc<false, EPI_HEADS>, grid, block, smem, s, tw, tw2, tx, g, st); break;
    default: return false;
    }
    return e == cudaSuccess;
}

}  // namespace psw
