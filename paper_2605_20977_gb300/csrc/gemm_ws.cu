// gemm_ws.cu -- projections of launches with many tokens (a wide decoder
// batch, the encoder's masked pass): one persistent, warp-specialised tcgen05
// kernel per projection.
//
// A tile is 128 output features x TNB tokens (TNB = 64, 128 or 256, chosen
// per launch; at most 128 for the dual SwiGLU form, whose gate and up
// accumulators are both kept): the projection is
// the MMA's A operand (M = 128, one feature per tensor-memory lane), the
// tokens its B operand (N = TNB; a 256-token tile is issued as two N = 128
// halves by two threads).  One CTA per SM walks the tiles
// blockIdx.x, + grid, ... (feature tile fastest, so CTAs running together
// share token tiles in L2).  A resident-weight schedule (contiguous
// feature-major ranges per CTA, the feature tile's weights kept in shared
// memory) is built in but off (WS_RESIDENT): it measured slower at decode
// sizes, its first tile starting later.
// Roles:
//   warp 0, lane 0     copies (the first resident weights before waiting for
//                      the previous kernel, then the 64-wide K chunks of
//                      every tile through a 4..8-stage ring of ~192 KB);
//   warp 1 (2), lane 0 issues the MMAs, every K step in ascending order into
//                      one accumulator (the up projection's, or the second
//                      128 tokens' of a 256-token tile, on warp 2), into
//                      one of two tensor-memory buffers, so a tile's MMAs run
//                      while the epilogue drains the previous tile;
//   warp 3             resolves each tile's token table (the cache, hyperprior
//                      or head rows its outputs go to) into one of two
//                      shared tables, ahead of the epilogue;
//   warps 4..19        the epilogue: warp w reads the 32 feature rows
//                      32 (w % 4) .. + 31 of the buffer (lane = feature) and
//                      a quarter of its token columns, 16 at a time, and
//                      writes the mode's outputs (residual rows coalesced
//                      along the features, bf16 rows through a 512-byte
//                      staging buffer per warp as 16-byte stores); four
//                      epilogue warps per scheduler hide each other's
//                      tensor-memory and store latencies.
// The token operand is always compact bf16 rows (A_DIRECT; normalised
// inputs come from launch_norm_rows).  The accumulation order (one
// accumulator, K ascending) and the per-element epilogue (epi_value,
// store_bf16_8) are those of the one-tile-per-CTA kernel, and the tensor
// core computes an element the same whatever the MMA's shape, so a token's
// outputs are bit-identical whichever kernel its launch takes.
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

constexpr int WS_EPI0 = 4;                            // first epilogue warp
constexpr int WS_EPI_WARPS = 16;                      // four per scheduler: one per lane quarter and column group
constexpr int WS_CGROUPS = WS_EPI_WARPS / 4;          // column groups of a tile (a quarter of its tokens each)
constexpr int WS_THREADS = 32 * (WS_EPI0 + WS_EPI_WARPS);
constexpr int WS_TAB = 256;                           // token-table rows (tokens of a tile at most)
constexpr int WS_MAXST = 8;                           // ring stages at most
constexpr int WS_STG = 512;                           // epilogue staging of one warp: 32 features x 8 tokens
constexpr int WS_DYN = 192 * 1024;                    // resident weights + ring
constexpr int WS_WRES_MAX = 96 * 1024;                // resident weights at most
constexpr uint32_t WS_TCOLS = 512;                    // two accumulator buffers
constexpr bool WS_RESIDENT = false;                   // resident-weight schedule (measured slower at decode sizes)

// Geometry of a launch, the same on host and device.
struct WsGeom {
    int tnb;                      // tokens per tile
    int nf, ntok, ntiles, grid;   // feature tiles, token tiles, tiles, CTAs
    int wres;                     // 1: the feature tile's weights stay resident
    int wchunk, xchunk;           // bytes of one K chunk of a tile's weights (both, dual form) / tokens
    int stage, nst;               // ring stage bytes and stages
};

__host__ __device__ inline WsGeom ws_geom(int tnb, bool dual, int M, int N, int K, int sms)
{
    WsGeom q{};
    q.tnb = tnb;
    q.nf = (N + TM - 1) / TM;
    q.ntok = (M + tnb - 1) / tnb;
    q.ntiles = q.nf * q.ntok;
    q.grid = q.ntiles < sms ? q.ntiles : sms;
    q.wchunk = (dual ? 2 : 1) * A_BYTES;
    q.xchunk = tnb * 128;
    const int nk = K / KC;
    // resident weights pay when a CTA has at least three tiles (their copy
    // delays the first tile's token chunks); they need feature-major ranges
    q.wres = WS_RESIDENT && q.wchunk * nk <= WS_WRES_MAX && q.ntiles >= 3 * q.grid;
    q.stage = q.xchunk + (q.wres ? 0 : q.wchunk);
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

// Byte offset of cache `sel`'s base pointer in a slot record.
__device__ __forceinline__ int slot_cache_off(int sel)
{
    switch (sel) {
    case CS_K1: return (int)offsetof(Slot, K1);
    case CS_V1: return (int)offsetof(Slot, V1);
    case CS_K2: return (int)offsetof(Slot, K2);
    case CS_V2: return (int)offsetof(Slot, V2);
    case CS_KA: return (int)offsetof(Slot, Ka);
    case CS_VA: return (int)offsetof(Slot, Va);
    case CS_QA: return (int)offsetof(Slot, qa);
    case CS_CK: return (int)offsetof(Slot, CK);
    case CS_CV: return (int)offsetof(Slot, CV);
    case CS_XK: return (int)offsetof(Slot, XK);
    case CS_LK: return (int)offsetof(Slot, LK);
    case CS_LV: return (int)offsetof(Slot, LV);
    default: return (int)offsetof(Slot, XV);
    }
}

// The QKV token table rows lane + 32 j (j < PER) of the tile at m0: the
// key and value cache rows of each token (table_row's values), with the
// loads of all PER rows in flight together -- the token words, then the
// slots' stride, cache bases and ring position -- and no branch between
// them (rows past M read row M - 1 and are written as zero).
template <int PER>
__device__ __forceinline__ void qkv_table_rows(const GemmArgs &g, int m0, uintptr_t *tab, int ts)
{
    const Epi &e = g.epi;
    const int lane = threadIdx.x & 31;
    const int koff = slot_cache_off(e.kc_sel), voff = slot_cache_off(e.vc_sel);
    int tk[PER];
#pragma unroll
    for (int j = 0; j < PER; j++) tk[j] = e.tok[min(m0 + lane + 32 * j, g.M - 1)];
    const char *sl[PER];
    int stride[PER], nfr[PER];
    uintptr_t kb[PER], vb[PER];
#pragma unroll
    for (int j = 0; j < PER; j++) {
        sl[j] = (const char *)&e.slots[tok_slot(tk[j])];
        stride[j] = ((const Slot *)sl[j])->stride;
        nfr[j] = ((const Slot *)sl[j])->nfr;
        kb[j] = *(const uintptr_t *)(sl[j] + koff);
        vb[j] = *(const uintptr_t *)(sl[j] + voff);
    }
    int layer[PER];
#pragma unroll
    for (int j = 0; j < PER; j++)
        layer[j] = e.ring ? e.kv_layer * e.Tf + ((const Slot *)sl[j])->ring[nfr[j] - 1] : e.kv_layer;
#pragma unroll
    for (int j = 0; j < PER; j++) {
        const int r = lane + 32 * j;
        const bool ok = m0 + r < g.M;
        const long row = ((long)layer[j] * stride[j] + tok_pos(tk[j])) * e.d * (long)sizeof(__nv_bfloat16);
        tab[r] = ok ? kb[j] + (uintptr_t)row : 0;
        tab[ts + r] = ok ? vb[j] + (uintptr_t)row : 0;
        tab[2 * ts + r] = tab[3 * ts + r] = 0;
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

// 16 consecutive accumulator columns at addr (and at addr2 for the dual
// form) under one wait.
template <bool DUAL>
__device__ __forceinline__ void tmem_ld16x(uint32_t addr, uint32_t addr2, uint32_t *v, uint32_t *v2)
{
    tmem_ld8_async(addr, v);
    tmem_ld8_async(addr + 8, v + 8);
    if (DUAL) {
        tmem_ld8_async(addr2, v2);
        tmem_ld8_async(addr2 + 8, v2 + 8);
    }
    tmem_wait_ld();
}

// Epilogue of one tile for this warp: feature rows f0 + 32 quarter + lane,
// token columns cb .. cb + TNB / WS_CGROUPS of the accumulator at tacc (m0:
// the tile's first token), once the tile's MMAs are complete (the full
// barrier at parity par; false if that wait expired).  Residual modes read
// the rows they update while the MMAs still run (all of a thread's values in
// flight at once); every mode reads the accumulator 16 columns per wait.
template <bool DUAL, int MODE, int TNB, bool F8>
__device__ __forceinline__ bool ws_epilogue(const GemmArgs &g, WsShared &S, const uintptr_t *tab, uint64_t *full,
                                            uint32_t par, uint32_t tacc, int f0, int m0, int quarter, int cb,
                                            uint16_t *stg)
{
    constexpr bool RESID = MODE == EPI_RESID || MODE == EPI_RESID_BASE;
    constexpr int NC = TNB / WS_CGROUPS;                      // token columns of this warp
    const int lane = threadIdx.x & 31;
    const int M = g.M, N = g.N;
    const Epi &e = g.epi;
    const int f = f0 + quarter * 32 + lane;
    const bool fok = f < N;
    const uint32_t trow = tacc + (uint32_t)cb;
    // E4M3: the feature row's and each token's dequantisation scales (their
    // products are powers of two, exact), applied as the one-tile kernel does
    float wf = 1.0f, wf2 = 1.0f;
    if constexpr (F8) {
        if (fok) { wf = g.wsc[f]; if (DUAL) wf2 = g.wsc2[f]; }
    }
    if constexpr (RESID) {
        static_assert(NC <= 64, "residual tiles keep their old values in registers");
        // the rows' old values: the first 32 columns' read while the MMAs
        // run (16 for a 256-token tile, whose warps hold 64 columns), each
        // later 16-column chunk's ahead of its use
        constexpr int PRE = NC <= 32 ? NC : 16;
        constexpr int AHEAD = NC <= 32 ? 2 : 1;
        float old[NC];
        const int nv = fok ? min(NC, M - (m0 + cb)) : 0;         // this warp's rows m0 + cb + j, j < nv
        float *rowf = e.rows + (long)(m0 + cb) * N + f;          // row j at rowf[j * N]
        auto load_old = [&](int j) {
            const float *src = MODE == EPI_RESID ? rowf + j * N : (const float *)tab[WS_TAB + cb + j] + f;
            old[j] = j < nv ? *src : 0.0f;
        };
#pragma unroll
        for (int j = 0; j < PRE; j++) load_old(j);
        if (S.abort || !mbar_wait(full, par)) return false;
        fence_after();
#pragma unroll
        for (int h = 0; h < NC / 16; h++) {
            if (16 * (h + AHEAD) >= PRE && 16 * (h + AHEAD) < NC) {
#pragma unroll
                for (int j = 0; j < 16; j++) load_old(16 * (h + AHEAD) + j);
            }
            uint32_t v[16], v2[1];
            tmem_ld16x<false>(trow + 16 * h, 0, v, v2);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                float y = __uint_as_float(v[j]);
                if constexpr (F8) {
                    const int m = m0 + cb + 16 * h + j;
                    y *= wf * (m < M ? g.xs[m] : 0.0f);
                }
                if (16 * h + j < nv) rowf[(16 * h + j) * N] = old[16 * h + j] + y;
            }
        }
        return true;
    } else {
        if (S.abort || !mbar_wait(full, par)) return false;
        fence_after();
        float bf = 0.0f, ga = 0.0f, gb = 0.0f;
        if ((MODE == EPI_SET_BIAS || MODE == EPI_BIAS_SILU) && fok) bf = e.bias[f];
        if (MODE == EPI_HEADS && fok) {
            ga = (f & 1) ? e.gsg[f >> 1] : e.gmu[f >> 1];
            gb = (f & 1) ? e.bsg[f >> 1] : e.bmu[f >> 1];
        }
#pragma unroll 1
        for (int c16 = 0; c16 < NC; c16 += 16) {
            uint32_t v[16], v2[DUAL ? 16 : 1];
            tmem_ld16x<DUAL>(trow + c16, trow + TNB + c16, v, v2);
            if (m0 + cb + c16 >= M) continue;                   // the same for the whole warp
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int c0 = cb + c16 + 8 * q;                 // tile column of the group's first token
                float o[8];
                int oi[8];
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    float y = __uint_as_float(v[8 * q + j]);
                    float y2 = DUAL ? __uint_as_float(v2[(8 * q + j) % (DUAL ? 16 : 1)]) : 0.0f;
                    if constexpr (F8) {
                        const int m = m0 + c0 + j;
                        const float t = m < M ? g.xs[m] : 0.0f;
                        y *= wf * t;
                        if (DUAL) y2 *= wf2 * t;
                    }
                    o[j] = epi_value<MODE, DUAL>(y, y2, f, bf, ga, gb, S.stab, &oi[j]);
                }
                if constexpr (MODE == EPI_HEADS || MODE == EPI_SET_BIAS) {
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        const int rr = c0 + j, m = m0 + rr;
                        if (!(fok && m < M)) continue;
                        if (MODE == EPI_HEADS) {
                            const int c = f >> 1;
                            if (f & 1) {
                                ((float *)tab[WS_TAB + rr])[c] = o[j];
                                ((uint8_t *)tab[2 * WS_TAB + rr])[c] = (uint8_t)oi[j];
                            } else {
                                ((float *)tab[rr])[c] = o[j];
                                ((int32_t *)tab[3 * WS_TAB + rr])[c] = oi[j];
                            }
                        } else {
                            e.rows[(long)m * N + f] = o[j];
                        }
                    }
                } else {
                    store_bf16_8<MODE>(e, M, N, m0, c0, f0 + quarter * 32, o, stg, tab, WS_TAB);
                }
            }
        }
        return true;
    }
}

template <bool DUAL, int MODE, int TNB, bool F8>
__global__ void __launch_bounds__(WS_THREADS, 1)
k_gemm_ws(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmW2,
          const __grid_constant__ CUtensorMap tmX, const __grid_constant__ GemmArgs g, int sms, int *status)
{
    // issuers: the dual form's two (one accumulator each); a 256-token tile
    // of the single form is also issued by two threads, each into its own
    // 128 accumulator columns for its 128 tokens (the same weights chunk)
    constexpr bool SPLIT = !DUAL && TNB == 256;
    constexpr int NACC = (DUAL || SPLIT) ? 2 : 1;
    constexpr int BCOLS = DUAL ? 2 * TNB : TNB;             // tensor-memory columns of one buffer
    // a K chunk is one 128-byte swizzle row of both operands: 64 bf16 or 128 E4M3
    constexpr int KCH = F8 ? KC8 : KC;
    extern __shared__ uint8_t smem_raw[];
    __shared__ WsShared S;
    const WsGeom q = ws_geom(TNB, DUAL, g.M, g.N, F8 ? g.K / 2 : g.K, sms);   // the ring's geometry in bytes
    const int nk = g.K / KCH;
    uint8_t *wbuf = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *ring = wbuf + (q.wres ? q.wchunk * nk : 0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this CTA's tiles: with resident weights the contiguous range tb .. te - 1
    // (tile t: feature tile t / ntok, token tile t % ntok), otherwise
    // blockIdx.x, + grid, ... (tile t: feature tile t % nf, token tile t / nf,
    // so the CTAs running together share token tiles in L2)
    const int tb = q.wres ? (int)((long)blockIdx.x * q.ntiles / q.grid) : blockIdx.x;
    const int te = q.wres ? (int)((long)(blockIdx.x + 1) * q.ntiles / q.grid) : q.ntiles;
    const int ts = q.wres ? 1 : q.grid;
    auto tile_f = [&](int t) { return q.wres ? t / q.ntok : t % q.nf; };
    auto tile_m = [&](int t) { return q.wres ? t % q.ntok : t / q.nf; };
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
                    tma_load(wbuf + j * q.wchunk, &tmW, &S.wbar, j * KCH, fi * TM);
                    if (DUAL) tma_load(wbuf + j * q.wchunk + A_BYTES, &tmW2, &S.wbar, j * KCH, fi * TM);
                }
            };
            int cur_f = -1, nload = 0;
            if (q.wres && tb < te) {
                // the projection's weights do not change: the first copy goes
                // out before the wait for the previous kernel
                cur_f = tile_f(tb);
                load_weights(cur_f);
                nload = 1;
            }
            // streamed weights: the first tile's first ring fill of weight
            // chunks goes out before the wait too (their token chunks after it)
            const int pre = q.wres ? 0 : (nk < q.nst ? nk : q.nst);
            for (int j = 0; j < pre; j++) {
                uint8_t *st = ring + j * q.stage;
                mbar_expect_tx(&S.full[j], (uint32_t)q.stage);
                tma_load(st + q.xchunk, &tmW, &S.full[j], j * KCH, tile_f(tb) * TM);
                if (DUAL) tma_load(st + q.xchunk + A_BYTES, &tmW2, &S.full[j], j * KCH, tile_f(tb) * TM);
            }
            pdl_wait();                                    // the token rows are the previous kernel's output
            fence_proxy_global();
            // chunk `it` of the CTA's sequence fills stage it % nst for the
            // (it / nst)-th time, after the MMAs released its previous use
            int it = 0;
            for (int t = tb; t < te && !S.abort; t += ts) {
                const int fi = tile_f(t), f0 = fi * TM, m0 = tile_m(t) * TNB;
                if (q.wres && fi != cur_f) {
                    // the previous feature tile's MMAs are done with its weights
                    if (!mbar_wait(&S.wempty, (nload - 1) & 1)) { S.abort = 1; break; }
                    load_weights(fi);
                    cur_f = fi;
                    nload++;
                }
                for (int j = 0; j < nk; j++, it++) {
                    const int s = it % q.nst, u = it / q.nst;
                    uint8_t *st = ring + s * q.stage;
                    if (it < pre) {                          // its weights already on the way
                        tma_load(st, &tmX, &S.full[s], j * KCH, m0);
                        continue;
                    }
                    if (u > 0 && !mbar_wait(&S.empty[s], (u - 1) & 1)) { S.abort = 1; break; }
                    mbar_expect_tx(&S.full[s], (uint32_t)q.stage);
                    tma_load(st, &tmX, &S.full[s], j * KCH, m0);
                    if (!q.wres) {
                        tma_load(st + q.xchunk, &tmW, &S.full[s], j * KCH, f0);
                        if (DUAL) tma_load(st + q.xchunk + A_BYTES, &tmW2, &S.full[s], j * KCH, f0);
                    }
                }
            }
            // every copy this thread issued has landed before the CTA exits
            // (the last fill of each stage; earlier ones were consumed)
            for (int k = it > q.nst ? it - q.nst : 0; k < it; k++) mbar_wait(&S.full[k % q.nst], (k / q.nst) & 1);
            if (nload) mbar_wait(&S.wbar, (nload - 1) & 1);
        }
    } else if (warp == 1 || (NACC == 2 && warp == 2)) {
        if (lane == 0) {
            constexpr int NI = SPLIT ? TNB / 2 : TNB;             // the MMA's N
            const uint32_t id = F8 ? idesc_e4m3(TM, NI) : idesc_bf16(TM, NI);
            const uint32_t woff = DUAL && warp == 2 ? (uint32_t)A_BYTES : 0u;
            // the second issuer of a split tile: tokens NI.. (rows NI.. of the chunk)
            const uint32_t xoff = SPLIT && warp == 2 ? (uint32_t)(NI * 128) : 0u;
            int it = 0, i = 0, cur_f = -1, nuse = 0;
            for (int t = tb; t < te && !S.abort; t += ts, i++) {
                const int b = i & 1, ub = i >> 1, fi = tile_f(t);
                if (q.wres && fi != cur_f) {
                    // the earlier MMAs release the resident weights; wait for the new ones
                    if (cur_f >= 0) mma_commit(&S.wempty);
                    if (!mbar_wait(&S.wbar, nuse & 1)) { S.abort = 1; break; }
                    cur_f = fi;
                    nuse++;
                }
                if (ub > 0 && !mbar_wait(&S.tempty[b], (ub - 1) & 1)) { S.abort = 1; break; }
                fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * BCOLS) + (warp == 2 ? (uint32_t)(DUAL ? TNB : NI) : 0u);
                for (int j = 0; j < nk; j++, it++) {
                    const int s = it % q.nst, u = it / q.nst;
                    if (S.abort) break;
                    if (!mbar_wait(&S.full[s], u & 1)) { S.abort = 1; break; }
                    fence_after();
                    const uint32_t xs0 = su32(ring + s * q.stage), xb = xs0 + xoff;
                    const uint32_t wa = (q.wres ? su32(wbuf + j * q.wchunk) : xs0 + q.xchunk) + woff;
                    // four K steps of 32 bytes along the 128-byte rows (16 bf16 or 32 E4M3 each)
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        if constexpr (F8) mma8(acc, sdesc(wa + k * 32), sdesc(xb + k * 32), id, (j | k) != 0);
                        else mma(acc, sdesc(wa + k * 32), sdesc(xb + k * 32), id, (j | k) != 0);
                    }
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
            for (int t = tb; t < te && !S.abort; t += ts, i++) {
                const int b = i & 1, ub = i >> 1;
                if (ub > 0 && !mbar_wait(&S.tabempty[b], (ub - 1) & 1)) { S.abort = 1; break; }
                if (MODE == EPI_QKV && g.epi.tok)
                    qkv_table_rows<TNB / 32>(g, tile_m(t) * TNB, S.tab[b], WS_TAB);
                else
                    for (int r = lane; r < TNB; r += 32)
                        table_row<MODE>(g, tile_m(t) * TNB, r, S.tab[b], WS_TAB, nullptr);
                mbar_arrive(&S.tabfull[b]);
            }
        }
    } else if (warp >= WS_EPI0) {
        pdl_wait();                                        // rows and caches of the previous kernel
        const int quarter = warp & 3, cb = ((warp - WS_EPI0) >> 2) * (TNB / WS_CGROUPS);
        const uint32_t lanes = (uint32_t)(quarter * 32) << 16;
        uint16_t *stg = (uint16_t *)(ring + q.nst * q.stage + (warp - WS_EPI0) * WS_STG);
        int i = 0;
        for (int t = tb; t < te && !S.abort; t += ts, i++) {
            const int b = i & 1, ub = i >> 1;
            bool ok = !ws_needs_table(MODE) || mbar_wait(&S.tabfull[b], ub & 1);
            ok = ok && ws_epilogue<DUAL, MODE, TNB, F8>(g, S, S.tab[b], &S.tfull[b], ub & 1,
                                                    tmem + lanes + (uint32_t)(b * BCOLS), tile_f(t) * TM,
                                                    tile_m(t) * TNB, quarter, cb, stg);
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

// Widest tile of a form: 128 tokens for the dual form (two accumulators
// per buffer), else 256.
__host__ __device__ constexpr int ws_max_tn(bool dual, int mode)
{
    return dual ? 128 : 256;
}

template <bool DUAL, int MODE, int TNB, bool F8>
bool ws_attr()
{
    return cudaFuncSetAttribute(k_gemm_ws<DUAL, MODE, TNB, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                WS_DYN + WS_EPI_WARPS * WS_STG + 1024) == cudaSuccess;
}

template <bool DUAL, int MODE, bool F8 = false>
bool ws_attr_all()
{
    return ws_attr<DUAL, MODE, 64, F8>() && ws_attr<DUAL, MODE, 128, F8>() &&
           ws_attr<DUAL, MODE, ws_max_tn(DUAL, MODE), F8>();
}

// Modes whose E4M3 projections take the wide kernel (the transformer
// blocks' projections; the embedding and heads stay BF16).
__host__ __device__ constexpr bool ws_f8_mode(int mode)
{
    return mode == EPI_STORE || mode == EPI_QKV || mode == EPI_RESID || mode == EPI_RESID_BASE || mode == EPI_SWIGLU;
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

template <bool DUAL, int MODE, int TNB, bool F8>
cudaError_t ws_launch(const CUtensorMap &tw, const CUtensorMap &tw2, const CUtensorMap &tx, const GemmArgs &g,
                      cudaStream_t s)
{
    const int sms = ws_sms();
    const int kb = F8 ? g.K / 2 : g.K;                 // the bf16 width of the same bytes (ring geometry)
    const WsGeom q = ws_geom(TNB, DUAL, g.M, g.N, kb, sms);
    dim3 grid(q.grid), block(WS_THREADS);
    return launch_pdl(k_gemm_ws<DUAL, MODE, TNB, F8>, grid, block, (size_t)ws_smem_bytes(q, kb), s, tw, tw2, tx, g,
                      sms, g.status);
}

template <bool DUAL, int MODE, bool F8 = false>
cudaError_t ws_launch_tn(int tnb, const CUtensorMap &tw, const CUtensorMap &tw2, const CUtensorMap &tx,
                         const GemmArgs &g, cudaStream_t s)
{
    if (tnb == 64) return ws_launch<DUAL, MODE, 64, F8>(tw, tw2, tx, g, s);
    if (tnb == 128) return ws_launch<DUAL, MODE, 128, F8>(tw, tw2, tx, g, s);
    return ws_launch<DUAL, MODE, ws_max_tn(DUAL, MODE), F8>(tw, tw2, tx, g, s);
}

}  // namespace

bool gemm_ws_prepare()
{
    return ws_attr_all<false, EPI_STORE>() && ws_attr_all<false, EPI_QKV>() && ws_attr_all<false, EPI_RESID>() &&
           ws_attr_all<false, EPI_RESID_BASE>() && ws_attr_all<false, EPI_BIAS_SILU>() &&
           ws_attr_all<false, EPI_HEADS>() && ws_attr_all<true, EPI_SWIGLU>() && ws_attr_all<false, EPI_SET_BIAS>() &&
           ws_attr_all<false, EPI_STORE, true>() && ws_attr_all<false, EPI_QKV, true>() &&
           ws_attr_all<false, EPI_RESID, true>() && ws_attr_all<false, EPI_RESID_BASE, true>() &&
           ws_attr_all<true, EPI_SWIGLU, true>();
}

bool gemm_takes_ws(int prec, const GemmArgs &g)
{
    return prec == P_BF16 && g.M >= WIDE_M && gemm_ws_supported(g);
}

bool gemm_ws_supported(const GemmArgs &g)
{
    const int m = g.epi.mode;
    if (m == EPI_HEADS && (g.epi.C % 16 || g.epi.c0 % 16 || g.N % 32 || g.epi.c0 + g.N / 2 > g.epi.C)) return false;
    if (m == EPI_QKV && (g.epi.d % 32 || g.epi.q_cols % 32 || g.epi.ld_out % 8)) return false;
    if (m == EPI_STORE && g.epi.st_sel == CS_NONE && g.epi.ld_out % 8) return false;
    if ((m == EPI_STORE || m == EPI_QKV) && g.epi.d % 8) return false;
    if ((m == EPI_SWIGLU || m == EPI_BIAS_SILU) && g.epi.ld_out % 8) return false;
    if (g.f8 && (!ws_f8_mode(m) || !g.xs || !g.wsc || (m == EPI_SWIGLU && !g.wsc2) || g.K % KC8)) return false;
    if (m == EPI_SET_BIAS && (g.f8 || g.epi.eh_out)) return false;
    return g.asrc == A_DIRECT && g.K % KC == 0 && g.K >= KC && g.N >= 32 && g.N % 32 == 0 &&
           g.lda % 8 == 0 &&
           (m == EPI_STORE || m == EPI_QKV || m == EPI_RESID || m == EPI_RESID_BASE || m == EPI_BIAS_SILU ||
            m == EPI_HEADS || m == EPI_SWIGLU || m == EPI_SET_BIAS);
}

// Tokens per tile: the width with the least estimated time of the busiest
// CTA -- its tiles x the slower of a tile's MMAs and epilogue (they overlap
// across tiles), plus the faster of the two once.  One thread issues an MMA
// in about the same time for any N up to 128 (~185 cycles, above the tensor
// pipe's time for N = 128), so a tile's MMA time is its K chunks whatever
// its width up to 128; a 256-token tile has two issuers (~1.1x); the
// epilogue, ~0.86x a 128-token tile's MMA time at K = 384, grows with the
// tile's tokens (measured with cycle counters on the 1080p projections).
// Ties go to the wider tile (fewer weight re-reads).
int gemm_ws_tile_tokens(int N, int M, int K, bool dual, bool resid)
{
    const int sms = ws_sms();
    int best = 64;
    double best_cost = 1e30;
    for (int tnb = ws_max_tn(dual, resid ? EPI_RESID : EPI_STORE); tnb >= 64; tnb /= 2) {
        const WsGeom q = ws_geom(tnb, dual, M, N, K, sms);
        const int tiles = (q.ntiles + q.grid - 1) / q.grid;
        const double mma = (K / 384.0) * (tnb == 256 && !dual ? 1.1 : 1.0), epi = 0.86 * tnb / 128.0;
        const double cost = tiles * (mma > epi ? mma : epi) + (mma < epi ? mma : epi);
        if (cost < best_cost - 1e-9) { best_cost = cost; best = tnb; }
    }
    return best;
}

bool gemm_ws(const GemmArgs &g, cudaStream_t s)
{
    if (!gemm_ws_supported(g)) return false;
    const bool dual = g.epi.mode == EPI_SWIGLU, f8 = g.f8 != 0;
    // an E4M3 projection has half the MMAs of a BF16 one of the same K
    int tnb = gemm_ws_tile_tokens(g.N, g.M, f8 ? g.K / 2 : g.K, dual,
                                  g.epi.mode == EPI_RESID || g.epi.mode == EPI_RESID_BASE);
    if (g.tnb == 64 || g.tnb == 128 || g.tnb == 256) tnb = std::min(g.tnb, ws_max_tn(dual, g.epi.mode));
    CUtensorMap tw, tw2, tx;
    if (!gemm_tensor_map(g.Wt, g.N, g.K, g.K, TM, &tw, f8)) return false;
    if (dual && !gemm_tensor_map(g.Wt2, g.N, g.K, g.K, TM, &tw2, f8)) return false;
    if (!dual) tw2 = tw;
    if (!gemm_tensor_map(g.A, g.M, g.K, g.lda, tnb, &tx, f8)) return false;
    cudaError_t e;
    if (f8) {
        switch (g.epi.mode) {
        case EPI_SWIGLU: e = ws_launch_tn<true, EPI_SWIGLU, true>(tnb, tw, tw2, tx, g, s); break;
        case EPI_STORE: e = ws_launch_tn<false, EPI_STORE, true>(tnb, tw, tw2, tx, g, s); break;
        case EPI_QKV: e = ws_launch_tn<false, EPI_QKV, true>(tnb, tw, tw2, tx, g, s); break;
        case EPI_RESID: e = ws_launch_tn<false, EPI_RESID, true>(tnb, tw, tw2, tx, g, s); break;
        case EPI_RESID_BASE: e = ws_launch_tn<false, EPI_RESID_BASE, true>(tnb, tw, tw2, tx, g, s); break;
        default: return false;
        }
        return e == cudaSuccess;
    }
    switch (g.epi.mode) {
    case EPI_SWIGLU: e = ws_launch_tn<true, EPI_SWIGLU>(tnb, tw, tw2, tx, g, s); break;
    case EPI_STORE: e = ws_launch_tn<false, EPI_STORE>(tnb, tw, tw2, tx, g, s); break;
    case EPI_QKV: e = ws_launch_tn<false, EPI_QKV>(tnb, tw, tw2, tx, g, s); break;
    case EPI_RESID: e = ws_launch_tn<false, EPI_RESID>(tnb, tw, tw2, tx, g, s); break;
    case EPI_RESID_BASE: e = ws_launch_tn<false, EPI_RESID_BASE>(tnb, tw, tw2, tx, g, s); break;
    case EPI_BIAS_SILU: e = ws_launch_tn<false, EPI_BIAS_SILU>(tnb, tw, tw2, tx, g, s); break;
    case EPI_HEADS: e = ws_launch_tn<false, EPI_HEADS>(tnb, tw, tw2, tx, g, s); break;
    case EPI_SET_BIAS: e = ws_launch_tn<false, EPI_SET_BIAS>(tnb, tw, tw2, tx, g, s); break;
    default: return false;
    }
    return e == cudaSuccess;
}

}  // namespace psw
