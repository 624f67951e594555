// gemm_ws.cu -- projections of launches with many tokens (a wide decoder
// batch, the encoder's masked pass): one persistent, warp-specialised tcgen05
// kernel per projection.
//
// A tile is 128 tokens x TNF output features (TNF = 64, 128 or 256, chosen
// per launch; the dual SwiGLU form keeps a gate and an up accumulator of TNF
// each, TNF <= 128): the tokens are the MMA's A operand (M = 128, one token
// per tensor-memory lane), the projection its B operand (N = TNF), so each
// epilogue thread owns one token's row piece (the warp's 32 rows go out
// through a small shared staging buffer as row-contiguous stores).
// The tiles, feature tile major, are split into equal contiguous ranges,
// one per CTA (one CTA per SM), so a CTA's tiles mostly share one feature
// tile; when a feature tile's weights fit (<= 96 KB) they are copied once
// and stay resident in shared memory (copied again only where a range
// crosses into the next feature tile), so only token chunks stream through
// the ring -- half the L2 traffic of a tile that re-reads its weights.
// Roles:
//   warp 0, lane 0     copies (the first resident weights before waiting for
//                      the previous kernel, then the 64-wide K chunks of
//                      every tile through a 4..8-stage ring);
//   warp 1 (2), lane 0 issues the MMAs, every K step in ascending order into
//                      one accumulator (the up projection's on warp 2), into
//                      one of two tensor-memory buffers, so a tile's MMAs run
//                      while the epilogue drains the previous tile;
//   warp 3             resolves each tile's token table (the cache, hyperprior
//                      or head rows its outputs go to) into one of two
//                      shared tables, ahead of the epilogue;
//   warps 4..11        the epilogue: warp w reads tensor-memory lanes
//                      32 (w % 4) .. + 31 (its tokens) and half of the
//                      buffer's columns (features), and writes the mode's
//                      outputs.
// The token operand is always compact bf16 rows (A_DIRECT; normalised
// inputs come from launch_norm_rows).  The accumulation order (one
// accumulator, K ascending) and the per-element epilogue (epi_value) are
// those of the one-tile-per-CTA kernel, and the tensor core computes an
// element the same whatever the MMA's shape and whichever operand holds the
// tokens, so a token's outputs are bit-identical whichever kernel its launch
// takes.
//
// Every wait is bounded (~2 s): on expiry the CTA raises its abort flag,
// every role leaves its loop, the copy producer and the MMA issuers wait
// (bounded) for their own copies and MMAs, and the launch reports
// ST_TIMEOUT.
#include "gemm_dev.cuh"

#include <algorithm>

namespace psw {

using namespace tc;

namespace {

constexpr int WS_THREADS = 384;                       // 12 warps
constexpr int WS_EPI0 = 4;                            // first epilogue warp
constexpr int WS_EPI_WARPS = 8;
constexpr int WS_TM = 128;                            // tokens per tile (MMA M)
constexpr int WS_TAB = WS_TM;                         // token-table rows
constexpr int WS_MAXST = 8;                           // ring stages at most
constexpr int WS_STG = 4096;                          // epilogue staging of one warp: 32 rows x 128 bytes
constexpr int WS_DYN = 176 * 1024;                    // resident weights + ring (+ staging and slack)
constexpr int WS_WRES_MAX = 96 * 1024;                // resident weights at most
constexpr int WS_XCHUNK = WS_TM * 128;                // one 64-wide K chunk of a token tile
constexpr uint32_t WS_TCOLS = 512;                    // two accumulator buffers

// Geometry of a launch, the same on host and device.
struct WsGeom {
    int tnf;                      // features per tile
    int nf, ntok, ntiles, grid;   // feature tiles, token tiles, tiles, CTAs
    int wres;                     // 1: the feature tile's weights stay resident
    int wchunk;                   // bytes of one K chunk of the tile's weights (both, dual form)
    int stage, nst;               // ring stage bytes and stages
};

__host__ __device__ inline WsGeom ws_geom(int tnf, bool dual, int M, int N, int K, int sms)
{
    WsGeom q{};
    q.tnf = tnf;
    q.nf = (N + tnf - 1) / tnf;
    q.ntok = (M + WS_TM - 1) / WS_TM;
    q.ntiles = q.nf * q.ntok;
    q.grid = q.ntiles < sms ? q.ntiles : sms;
    q.wchunk = (dual ? 2 : 1) * tnf * 128;
    const int nk = K / KC;
    q.wres = q.wchunk * nk <= WS_WRES_MAX;
    q.stage = WS_XCHUNK + (q.wres ? 0 : q.wchunk);
    int st = (WS_DYN - (q.wres ? q.wchunk * nk : 0)) / q.stage;
    q.nst = st < WS_MAXST ? st : WS_MAXST;
    return q;
}

__host__ __device__ inline int ws_smem_bytes(const WsGeom &q, int K)
{
    return (q.wres ? q.wchunk * (K / KC) : 0) + q.nst * q.stage + WS_EPI_WARPS * WS_STG + 1024;
}

struct WsShared {
    uint64_t full[WS_MAXST], empty[WS_MAXST];
    uint64_t tfull[2], tempty[2], fin, wbar, wempty;
    uint64_t tabfull[2], tabempty[2];
    uint32_t tmem_slot;
    volatile int abort;
    float stab[NSCALES];
    uintptr_t tab[2][4 * WS_TAB];
};

// Modes whose outputs go to rows the token table names.
__host__ __device__ constexpr bool ws_needs_table(int mode)
{
    return mode == EPI_QKV || mode == EPI_STORE || mode == EPI_RESID_BASE || mode == EPI_HEADS;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

// 32 consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr));
}

__device__ __forceinline__ uint32_t bf16x2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Epilogue of one tile for this thread: token row r (tensor-memory lane) of
// the tile (m0: the tile's first token), features fh .. fh + TNF / 2 of the
// output (accumulator columns fh - f0 ..), once the tile's MMAs are complete
// (the full barrier at parity par; false if that wait expired).  Each lane
// holds its own token's row piece; the warp's 32 rows go through its
// staging buffer stg (row pieces stored with their 16-byte chunks
// XOR-swizzled by the row, conflict-free both ways) so that global loads and
// stores are row-contiguous runs of 64 or 128 bytes.  Residual modes read the
// rows they update (cooperatively, coalesced) while the MMAs still run.
template <bool DUAL, int MODE, int TNF>
__device__ __forceinline__ bool ws_epilogue(const GemmArgs &g, WsShared &S, const uintptr_t *tab, uint64_t *full,
                                            uint32_t par, uint32_t tacc, int r, int m0, int f0, int fh,
                                            uint8_t *stg)
{
    constexpr bool RESID = MODE == EPI_RESID || MODE == EPI_RESID_BASE;
    constexpr int NC = TNF / 2;                               // features of this thread
    const int lane = threadIdx.x & 31;
    const int M = g.M, N = g.N;
    const Epi &e = g.epi;
    const int rw = r - lane;                                  // the warp's first row in the tile
    const uint32_t tcol = tacc + (uint32_t)(fh - f0);
    if constexpr (RESID) {
        static_assert(NC <= 64, "residual tiles keep their old values in registers");
        // lane l, pass k: row rw + (l >> 3) + 4k, 16-byte chunk l & 7 of each
        // 32-feature group (128 bytes of a row per eight lanes)
        float4 old[NC / 32][8];
        const int cr = lane >> 3, cc = lane & 7;
#pragma unroll
        for (int gI = 0; gI < NC / 32; gI++)
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int rr = rw + cr + 4 * k, m = m0 + rr, f = fh + 32 * gI + 4 * cc;
                const float *src = MODE == EPI_RESID ? e.rows + (long)m * N : (const float *)tab[WS_TAB + rr];
                old[gI][k] = (m < M && f < N) ? *reinterpret_cast<const float4 *>(src + f)
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        if (S.abort || !mbar_wait(full, par)) return false;
        fence_after();
#pragma unroll
        for (int gI = 0; gI < NC / 32; gI++) {
            uint32_t v[32];
            tmem_ld32(tcol + 32 * gI, v);
            tmem_wait_ld();
            // old values to the staging rows, this lane's row back, sum, out
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int rr = cr + 4 * k;
                *reinterpret_cast<float4 *>(stg + rr * 128 + ((cc ^ (rr & 7)) << 4)) = old[gI][k];
            }
            __syncwarp();
#pragma unroll
            for (int c = 0; c < 8; c++) {
                float4 *p = reinterpret_cast<float4 *>(stg + lane * 128 + ((c ^ (lane & 7)) << 4));
                const float4 a = *p;
                *p = make_float4(a.x + __uint_as_float(v[4 * c]), a.y + __uint_as_float(v[4 * c + 1]),
                                 a.z + __uint_as_float(v[4 * c + 2]), a.w + __uint_as_float(v[4 * c + 3]));
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int rr = cr + 4 * k, m = m0 + rw + rr, f = fh + 32 * gI + 4 * cc;
                const float4 val = *reinterpret_cast<const float4 *>(stg + rr * 128 + ((cc ^ (rr & 7)) << 4));
                if (m < M && f < N) *reinterpret_cast<float4 *>(e.rows + (long)m * N + f) = val;
            }
            __syncwarp();
        }
        return true;
    } else {
        if (S.abort || !mbar_wait(full, par)) return false;
        fence_after();
        const int m = m0 + r;
        const bool mok = m < M;
#pragma unroll 1
        for (int c = 0; c < NC; c += 32) {
            const int f = fh + c;                             // first feature of the group
            uint32_t v[32], v2[DUAL ? 32 : 1];
            tmem_ld32(tcol + c, v);
            if constexpr (DUAL) tmem_ld32(tcol + TNF + c, v2);
            tmem_wait_ld();
            if (f >= N) continue;                             // the same for the whole warp
            float o[32];
            int oi[32];
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const int fj = f + j;
                float bf = 0.0f, ga = 0.0f, gb = 0.0f;
                if (MODE == EPI_SET_BIAS || MODE == EPI_BIAS_SILU) bf = e.bias[fj];
                if (MODE == EPI_HEADS) {
                    ga = (fj & 1) ? e.gsg[fj >> 1] : e.gmu[fj >> 1];
                    gb = (fj & 1) ? e.bsg[fj >> 1] : e.bmu[fj >> 1];
                }
                o[j] = epi_value<MODE, DUAL>(__uint_as_float(v[j]), DUAL ? __uint_as_float(v2[j % (DUAL ? 32 : 1)]) : 0.0f,
                                             fj, bf, ga, gb, S.stab, &oi[j]);
            }
            if constexpr (MODE == EPI_HEADS) {
                // features 2c / 2c + 1 are mu / sigma of channel c: 16 channels
                if (!mok) continue;
                const int c0 = f >> 1;
                float *mu = (float *)tab[r] + c0, *sg = (float *)tab[WS_TAB + r] + c0;
                uint8_t *ix = (uint8_t *)tab[2 * WS_TAB + r] + c0;
                int32_t *mm = (int32_t *)tab[3 * WS_TAB + r] + c0;
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    reinterpret_cast<float4 *>(mu)[i] = make_float4(o[8 * i], o[8 * i + 2], o[8 * i + 4], o[8 * i + 6]);
                    reinterpret_cast<float4 *>(sg)[i] = make_float4(o[8 * i + 1], o[8 * i + 3], o[8 * i + 5], o[8 * i + 7]);
                    reinterpret_cast<int4 *>(mm)[i] = make_int4(oi[8 * i], oi[8 * i + 2], oi[8 * i + 4], oi[8 * i + 6]);
                }
                uint32_t w[4];
#pragma unroll
                for (int i = 0; i < 4; i++)
                    w[i] = (uint32_t)(oi[8 * i + 1] & 255) | ((uint32_t)(oi[8 * i + 3] & 255) << 8) |
                           ((uint32_t)(oi[8 * i + 5] & 255) << 16) | ((uint32_t)(oi[8 * i + 7] & 255) << 24);
                *reinterpret_cast<uint4 *>(ix) = make_uint4(w[0], w[1], w[2], w[3]);
            } else {
                // this lane's 64-byte row piece (four chunks) to the staging
                // rows, then lane l stores chunk l & 3 of rows (l >> 2) + 8k
#pragma unroll
                for (int i = 0; i < 4; i++)
                    *reinterpret_cast<uint4 *>(stg + lane * 64 + ((i ^ ((lane >> 1) & 3)) << 4)) =
                        make_uint4(bf16x2(o[8 * i], o[8 * i + 1]), bf16x2(o[8 * i + 2], o[8 * i + 3]),
                                   bf16x2(o[8 * i + 4], o[8 * i + 5]), bf16x2(o[8 * i + 6], o[8 * i + 7]));
                __syncwarp();
                const int cc = lane & 3;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int rr = (lane >> 2) + 8 * k, row = rw + rr, mm = m0 + row, ff = f + 8 * cc;
                    const uint4 val = *reinterpret_cast<const uint4 *>(stg + rr * 64 + ((cc ^ ((rr >> 1) & 3)) << 4));
                    if (mm < M) {
                        __nv_bfloat16 *dst;
                        if (MODE == EPI_STORE)
                            dst = e.st_sel == CS_NONE ? (__nv_bfloat16 *)e.out + (long)mm * e.ld_out + ff
                                                      : (__nv_bfloat16 *)tab[row] + ff;
                        else if (MODE == EPI_QKV)
                            dst = f < e.q_cols ? (__nv_bfloat16 *)e.out + (long)mm * e.ld_out + ff
                                  : f < e.q_cols + e.d ? (__nv_bfloat16 *)tab[row] + (ff - e.q_cols)
                                                       : (__nv_bfloat16 *)tab[WS_TAB + row] + (ff - e.q_cols - e.d);
                        else
                            dst = (__nv_bfloat16 *)e.out + (long)mm * e.ld_out + ff;
                        *reinterpret_cast<uint4 *>(dst) = val;
                    }
                }
                __syncwarp();
            }
        }
        return true;
    }
}

template <bool DUAL, int MODE, int TNF>
__global__ void __launch_bounds__(WS_THREADS, 1)
k_gemm_ws(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmW2,
          const __grid_constant__ CUtensorMap tmX, const __grid_constant__ GemmArgs g, int sms, int *status)
{
    constexpr int NACC = DUAL ? 2 : 1;
    extern __shared__ uint8_t smem_raw[];
    __shared__ WsShared S;
    const WsGeom q = ws_geom(TNF, DUAL, g.M, g.N, g.K, sms);
    const int nk = g.K / KC;
    uint8_t *wbuf = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *ring = wbuf + (q.wres ? q.wchunk * nk : 0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this CTA's tiles tb .. te - 1: tile t is feature tile t / ntok, token tile t % ntok
    const int tb = (int)((long)blockIdx.x * q.ntiles / q.grid), te = (int)((long)(blockIdx.x + 1) * q.ntiles / q.grid);
    if (threadIdx.x == 0) {
        for (int s = 0; s < q.nst; s++) { mbar_init(&S.full[s], 1); mbar_init(&S.empty[s], NACC); }
        for (int b = 0; b < 2; b++) {
            mbar_init(&S.tfull[b], NACC);
            mbar_init(&S.tempty[b], WS_EPI_WARPS);
            mbar_init(&S.tabfull[b], 32);
            mbar_init(&S.tabempty[b], WS_EPI_WARPS);
        }
        mbar_init(&S.fin, NACC);
        mbar_init(&S.wbar, 1);
        mbar_init(&S.wempty, NACC);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&S.tmem_slot, WS_TCOLS);
    if (MODE == EPI_HEADS && threadIdx.x < NSCALES) S.stab[threadIdx.x] = g.epi.scale[threadIdx.x];
    fence_before();
    __syncthreads();
    fence_after();
    pdl_trigger();
    const uint32_t tmem = S.tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // resident weights of feature tile fi (the nload-th copy)
            auto load_weights = [&](int fi) {
                mbar_expect_tx(&S.wbar, (uint32_t)(q.wchunk * nk));
                for (int j = 0; j < nk; j++) {
                    tma_load(wbuf + j * q.wchunk, &tmW, &S.wbar, j * KC, fi * TNF);
                    if (DUAL) tma_load(wbuf + j * q.wchunk + TNF * 128, &tmW2, &S.wbar, j * KC, fi * TNF);
                }
            };
            int cur_f = -1, nload = 0;
            if (q.wres && tb < te) {
                // the projection's weights do not change: the first copy goes
                // out before the wait for the previous kernel
                cur_f = tb / q.ntok;
                load_weights(cur_f);
                nload = 1;
            }
            pdl_wait();                                    // the token rows are the previous kernel's output
            fence_proxy_global();
            // chunk `it` of the CTA's sequence fills stage it % nst for the
            // (it / nst)-th time, after the MMAs released its previous use
            int it = 0;
            for (int t = tb; t < te && !S.abort; t++) {
                const int fi = t / q.ntok, f0 = fi * TNF, m0 = (t % q.ntok) * WS_TM;
                if (q.wres && fi != cur_f) {
                    // the previous feature tile's MMAs are done with its weights
                    if (!mbar_wait(&S.wempty, (nload - 1) & 1)) { S.abort = 1; break; }
                    load_weights(fi);
                    cur_f = fi;
                    nload++;
                }
                for (int j = 0; j < nk; j++, it++) {
                    const int s = it % q.nst, u = it / q.nst;
                    if (u > 0 && !mbar_wait(&S.empty[s], (u - 1) & 1)) { S.abort = 1; break; }
                    uint8_t *st = ring + s * q.stage;
                    mbar_expect_tx(&S.full[s], (uint32_t)q.stage);
                    tma_load(st, &tmX, &S.full[s], j * KC, m0);
                    if (!q.wres) {
                        tma_load(st + WS_XCHUNK, &tmW, &S.full[s], j * KC, f0);
                        if (DUAL) tma_load(st + WS_XCHUNK + TNF * 128, &tmW2, &S.full[s], j * KC, f0);
                    }
                }
            }
            // every copy this thread issued has landed before the CTA exits
            // (the last fill of each stage; earlier ones were consumed)
            for (int k = it > q.nst ? it - q.nst : 0; k < it; k++) mbar_wait(&S.full[k % q.nst], (k / q.nst) & 1);
            if (nload) mbar_wait(&S.wbar, (nload - 1) & 1);
        }
    } else if (warp == 1 || (DUAL && warp == 2)) {
        if (lane == 0) {
            const uint32_t id = idesc_bf16(WS_TM, TNF);
            const uint32_t woff = warp == 2 ? (uint32_t)(TNF * 128) : 0u;
            int it = 0, i = 0, cur_f = -1, nuse = 0;
            for (int t = tb; t < te && !S.abort; t++, i++) {
                const int b = i & 1, ub = i >> 1, fi = t / q.ntok;
                if (q.wres && fi != cur_f) {
                    // the earlier MMAs release the resident weights; wait for the new ones
                    if (cur_f >= 0) mma_commit(&S.wempty);
                    if (!mbar_wait(&S.wbar, nuse & 1)) { S.abort = 1; break; }
                    cur_f = fi;
                    nuse++;
                }
                if (ub > 0 && !mbar_wait(&S.tempty[b], (ub - 1) & 1)) { S.abort = 1; break; }
                fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * NACC * TNF) + (warp == 2 ? (uint32_t)TNF : 0u);
                for (int j = 0; j < nk; j++, it++) {
                    const int s = it % q.nst, u = it / q.nst;
                    if (S.abort) break;
                    if (!mbar_wait(&S.full[s], u & 1)) { S.abort = 1; break; }
                    fence_after();
                    const uint32_t xa = su32(ring + s * q.stage);
                    const uint32_t wb = (q.wres ? su32(wbuf + j * q.wchunk) : xa + WS_XCHUNK) + woff;
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        mma(acc, sdesc(xa + k * 32), sdesc(wb + k * 32), id, (j | k) != 0);
                    mma_commit(&S.empty[s]);
                }
                mma_commit(&S.tfull[b]);
            }
            // every MMA this thread issued is complete before the tensor
            // memory is freed
            mma_commit(&S.fin);
            mbar_wait(&S.fin, 0);
        }
    } else if (warp == 3) {
        if constexpr (ws_needs_table(MODE)) {
            // token tables (the token list and slot table are fixed for the
            // whole decode: no wait for the previous kernel)
            int i = 0;
            for (int t = tb; t < te && !S.abort; t++, i++) {
                const int b = i & 1, ub = i >> 1;
                if (ub > 0 && !mbar_wait(&S.tabempty[b], (ub - 1) & 1)) { S.abort = 1; break; }
                for (int r = lane; r < WS_TM; r += 32) table_row<MODE>(g, (t % q.ntok) * WS_TM, r, S.tab[b], WS_TAB, nullptr);
                mbar_arrive(&S.tabfull[b]);
            }
        }
    } else if (warp >= WS_EPI0) {
        pdl_wait();                                        // rows and caches of the previous kernel
        const int r = (warp & 3) * 32 + lane;              // token row of the tile (tensor-memory lane)
        const int half = (warp - WS_EPI0) >> 2;
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
        uint8_t *stg = ring + q.nst * q.stage + (warp - WS_EPI0) * WS_STG;
        int i = 0;
        for (int t = tb; t < te && !S.abort; t++, i++) {
            const int b = i & 1, ub = i >> 1;
            const int f0 = (t / q.ntok) * TNF, fh = f0 + half * (TNF / 2);
            bool ok = !ws_needs_table(MODE) || mbar_wait(&S.tabfull[b], ub & 1);
            ok = ok && ws_epilogue<DUAL, MODE, TNF>(g, S, S.tab[b], &S.tfull[b], ub & 1,
                                                    tmem + lanes + (uint32_t)(b * NACC * TNF), r,
                                                    (t % q.ntok) * WS_TM, f0, fh, stg);
            if (!ok) S.abort = 1;
            fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&S.tempty[b]);
                if (ws_needs_table(MODE)) mbar_arrive(&S.tabempty[b]);
            }
            if (!ok) break;
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x == 0 && S.abort) atomicOr(status, ST_TIMEOUT);
    if (warp == 1) tmem_free(tmem, WS_TCOLS);
}

// Widest tile of a form: 128 features for the dual form (two accumulators
// per buffer) and the residual modes (old values in registers), else 256.
__host__ __device__ constexpr int ws_max_tn(bool dual, int mode)
{
    return (dual || mode == EPI_RESID || mode == EPI_RESID_BASE) ? 128 : 256;
}

template <bool DUAL, int MODE, int TNF>
bool ws_attr()
{
    return cudaFuncSetAttribute(k_gemm_ws<DUAL, MODE, TNF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                WS_DYN + WS_EPI_WARPS * WS_STG + 1024) == cudaSuccess;
}

template <bool DUAL, int MODE>
bool ws_attr_all()
{
    return ws_attr<DUAL, MODE, 64>() && ws_attr<DUAL, MODE, 128>() && ws_attr<DUAL, MODE, ws_max_tn(DUAL, MODE)>();
}

int ws_sms()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <bool DUAL, int MODE, int TNF>
cudaError_t ws_launch(const CUtensorMap &tw, const CUtensorMap &tw2, const CUtensorMap &tx, const GemmArgs &g,
                      cudaStream_t s)
{
    const int sms = ws_sms();
    const WsGeom q = ws_geom(TNF, DUAL, g.M, g.N, g.K, sms);
    dim3 grid(q.grid), block(WS_THREADS);
    return launch_pdl(k_gemm_ws<DUAL, MODE, TNF>, grid, block, (size_t)ws_smem_bytes(q, g.K), s, tw, tw2, tx, g, sms,
                      g.status);
}

template <bool DUAL, int MODE>
cudaError_t ws_launch_tn(int tnf, const CUtensorMap &tw, const CUtensorMap &tw2, const CUtensorMap &tx,
                         const GemmArgs &g, cudaStream_t s)
{
    if (tnf == 64) return ws_launch<DUAL, MODE, 64>(tw, tw2, tx, g, s);
    if (tnf == 128) return ws_launch<DUAL, MODE, 128>(tw, tw2, tx, g, s);
    return ws_launch<DUAL, MODE, ws_max_tn(DUAL, MODE)>(tw, tw2, tx, g, s);
}

}  // namespace

bool gemm_ws_prepare()
{
    return ws_attr_all<false, EPI_STORE>() && ws_attr_all<false, EPI_QKV>() && ws_attr_all<false, EPI_RESID>() &&
           ws_attr_all<false, EPI_RESID_BASE>() && ws_attr_all<false, EPI_BIAS_SILU>() &&
           ws_attr_all<false, EPI_HEADS>() && ws_attr_all<true, EPI_SWIGLU>();
}

bool gemm_takes_ws(int prec, const GemmArgs &g)
{
    return prec == P_BF16 && g.M >= WIDE_M && gemm_ws_supported(g);
}

bool gemm_ws_supported(const GemmArgs &g)
{
    const int m = g.epi.mode;
    if (m == EPI_HEADS && (g.epi.C % 16 || g.N != 2 * g.epi.C)) return false;
    if (m == EPI_QKV && (g.epi.d % 32 || g.epi.q_cols % 32 || g.epi.ld_out % 8)) return false;
    if (m == EPI_STORE && g.epi.st_sel == CS_NONE && g.epi.ld_out % 8) return false;
    if ((m == EPI_STORE || m == EPI_QKV) && g.epi.d % 8) return false;
    if ((m == EPI_SWIGLU || m == EPI_BIAS_SILU) && g.epi.ld_out % 8) return false;
    return !g.f8 && g.asrc == A_DIRECT && g.K % KC == 0 && g.K >= KC && g.N >= 32 && g.N % 32 == 0 &&
           g.lda % 8 == 0 &&
           (m == EPI_STORE || m == EPI_QKV || m == EPI_RESID || m == EPI_RESID_BASE || m == EPI_BIAS_SILU ||
            m == EPI_HEADS || m == EPI_SWIGLU);
}

// Features per tile: the width with the least estimated time of the busiest
// CTA.  A tile's time is the slower of its MMA chain (one thread issues an
// MMA in ~84 cycles at N <= 128 and ~124 at N = 256, the tensor pipe's rate)
// and its copies (~110 GB/s per SM out of L2: the token chunks, plus the
// weight chunks unless they are resident); the epilogue overlaps the next
// tile.  Resident weights cost one copy per CTA.  Ties go to the wider tile.
int gemm_ws_tile_features(int N, int M, int K, bool dual, bool resid)
{
    const int sms = ws_sms();
    int best = 64;
    double best_cost = 1e30;
    for (int tnf = ws_max_tn(dual, resid ? EPI_RESID : EPI_STORE); tnf >= 64; tnf /= 2) {
        const WsGeom q = ws_geom(tnf, dual, M, N, K, sms);
        const int tiles = (q.ntiles + q.grid - 1) / q.grid;
        const double mma_us = (K / 16.0) * (tnf == 256 ? 124.0 : 84.0) * (dual ? 1.3 : 1.0) / 2000.0;
        const double bytes = (double)WS_XCHUNK * (K / KC) + (q.wres ? 0.0 : (double)q.wchunk * (K / KC));
        const double load_us = bytes / 110e3;
        const double cost = tiles * (mma_us > load_us ? mma_us : load_us) +
                            (q.wres ? (double)q.wchunk * (K / KC) / 110e3 : 0.0);
        if (cost < best_cost - 1e-9) { best_cost = cost; best = tnf; }
    }
    return best;
}

bool gemm_ws(const GemmArgs &g, cudaStream_t s)
{
    if (!gemm_ws_supported(g)) return false;
    const bool dual = g.epi.mode == EPI_SWIGLU;
    const int tnf = gemm_ws_tile_features(g.N, g.M, g.K, dual, g.epi.mode == EPI_RESID || g.epi.mode == EPI_RESID_BASE);
    CUtensorMap tw, tw2, tx;
    if (!gemm_tensor_map(g.Wt, g.N, g.K, g.K, tnf, &tw)) return false;
    if (dual && !gemm_tensor_map(g.Wt2, g.N, g.K, g.K, tnf, &tw2)) return false;
    if (!dual) tw2 = tw;
    if (!gemm_tensor_map(g.A, g.M, g.K, g.lda, WS_TM, &tx)) return false;
    cudaError_t e;
    switch (g.epi.mode) {
    case EPI_SWIGLU: e = ws_launch_tn<true, EPI_SWIGLU>(tnf, tw, tw2, tx, g, s); break;
    case EPI_STORE: e = ws_launch_tn<false, EPI_STORE>(tnf, tw, tw2, tx, g, s); break;
    case EPI_QKV: e = ws_launch_tn<false, EPI_QKV>(tnf, tw, tw2, tx, g, s); break;
    case EPI_RESID: e = ws_launch_tn<false, EPI_RESID>(tnf, tw, tw2, tx, g, s); break;
    case EPI_RESID_BASE: e = ws_launch_tn<false, EPI_RESID_BASE>(tnf, tw, tw2, tx, g, s); break;
    case EPI_BIAS_SILU: e = ws_launch_tn<false, EPI_BIAS_SILU>(tnf, tw, tw2, tx, g, s); break;
    case EPI_HEADS: e = ws_launch_tn<false, EPI_HEADS>(tnf, tw, tw2, tx, g, s); break;
    default: return false;
    }
    return e == cudaSuccess;
}

}  // namespace psw
