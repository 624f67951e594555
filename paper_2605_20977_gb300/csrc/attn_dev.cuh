// attn_dev.cuh -- masked window attention of one (token, head) per warp
// (Sec. 3.2 masks, Fig. 2b), shared by the attention kernel and the
// persistent decoder.  The per-token arithmetic depends only on the token,
// its head and the cached keys and values, never on the launch it runs in.
#pragma once

#include "internal.h"
#include "device_common.cuh"

namespace psw {


__device__ __forceinline__ int label_of(int mask, int i, int j)
{
    return mask == 1 ? ((i & 3) + (j & 3)) & 3 : 2 * i + j;
}

// Sec. 3.2 / Fig. 2b visibility: kind 0 (accumulator): strictly smaller
// label; kind 1 (spatial self-attention): the position itself or a label
// not above its own; for the 2i+j label also a smaller raster index.
__device__ __forceinline__ bool visible(int mask, int kind, int W, int pi, int pj, int qi, int qj)
{
    if (kind < 0) return true;
    if (kind == 1 && qi == pi && qj == pj) return true;
    int lp = label_of(mask, pi, pj), lq = label_of(mask, qi, qj);
    bool ok = kind == 0 ? lq < lp : lq <= lp;
    if (mask == 0) ok = ok && (qi * W + qj < pi * W + pj);
    return ok;
}

// Raw storage of B bytes of one row slice (kept packed until use).
template <int B> struct RawT;
template <> struct RawT<2> { using type = unsigned short; };
template <> struct RawT<4> { using type = unsigned int; };
template <> struct RawT<8> { using type = uint2; };
template <> struct RawT<16> { using type = uint4; };

// The n floats packed in raw storage of T elements.
template <typename T, int N, typename R>
__device__ __forceinline__ void unpack(const R &r, float *o)
{
    if constexpr (sizeof(T) == 4) {
        const float *f = reinterpret_cast<const float *>(&r);
#pragma unroll
        for (int i = 0; i < N; i++) o[i] = f[i];
    } else if constexpr (N == 1) {
        o[0] = __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(&r));
    } else {
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&r);
#pragma unroll
        for (int i = 0; i < N / 2; i++) {
            float2 f = __bfloat1622float2(h[i]);
            o[2 * i] = f.x; o[2 * i + 1] = f.y;
        }
    }
}

// 16-byte asynchronous copy global -> shared (cached in L2 only), and the
// wait for all of a thread's outstanding copies.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// (c0, c1) = (a0 b0 + c0, a1 b1 + c1): two independent fused multiply-adds,
// each rounded to nearest even as fmaf, in one packed instruction.
__device__ __forceinline__ void fma2(float &c0, float &c1, float a0, float a1, float b0, float b1)
{
    asm("{\n\t.reg .b64 pa, pb, pc;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\tmov.b64 pc, {%0, %1};\n\t"
        "fma.rn.f32x2 pc, pa, pb, pc;\n\tmov.b64 {%0, %1}, pc;\n\t}"
        : "+f"(c0), "+f"(c1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// The two bf16 of a packed word as floats (exact: the bits move into place).
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// Shared staging of one attention warp: CK key rows (the 16-byte pieces of
// row r stored in the order piece ^ (r & SWM), so that 16-byte reads of the
// same piece by consecutive lanes hit distinct banks without padding) and CK
// value rows of one head, the query, and the list of visible keys (cache row
// and relative-bias index) for up to MAXC candidates.  Spatial windows use
// 24-key chunks (24 keys are visible at most at k = 7) and a 64-entry list
// (96 for 9 x 9 windows): under 7 KB per warp at 64-wide heads, so eight
// blocks of four warps fit on an SM; temporal windows (Tf * k * k <= 256,
// checked at context creation) 32-key chunks and the full list.
template <typename T, int DH, int CK_ = 32, int MAXC_ = 256>
struct __align__(16) AttnWarp {
    static constexpr int RB = DH * (int)sizeof(T);            // bytes of one head's row slice
    static constexpr int PR = RB / 16;                         // 16-byte pieces per row slice
    static constexpr int SWM = PR < 8 ? PR - 1 : 7;            // piece swizzle mask of the key rows
    static constexpr int CK = CK_;
    static constexpr int MAXC = MAXC_;
    unsigned char kbuf[CK * RB];
    unsigned char vbuf[CK * RB];
    unsigned char qraw[RB];                                    // the query as stored, copied with the first keys
    float qs[DH];
    int rows[MAXC];
    unsigned short bix[MAXC];
};

// One warp per (token, head).  The warp first lists the visible window
// positions (Sec. 3.2 masks; frames oldest first, raster order within a
// window) as cache rows.  Then, 32 listed keys at a time, the warp copies the
// head's slices of their key and value rows into shared memory (consecutive
// lanes take consecutive 16-byte pieces of a row, so the gathers coalesce;
// one memory round trip per chunk), lane c scores key c as
// q.k / sqrt(DH) + relative bias, and every lane accumulates its PER output
// dimensions over the chunk's values.  The softmax runs online over chunks
// (one chunk for spatial windows up to 7 x 7) with max and sum by
// butterflies; values accumulate in list order and the sum of the weights
// divides at the end.
template <typename T, int DH, bool PDL, int CK = 32, int MAXC = 256>
__device__ __forceinline__ void attn_item(const AttnArgs &a, int gw, AttnWarp<T, DH, CK, MAXC> &sm)
{
    constexpr int PER = DH / 32;
    constexpr int RB = AttnWarp<T, DH, CK, MAXC>::RB, SWM = AttnWarp<T, DH, CK, MAXC>::SWM;
    constexpr int PR = RB / 16;                                // 16-byte pieces per row slice
    constexpr int EPU = 16 / (int)sizeof(T);                   // elements per piece
    // 64-wide BF16 heads: each lane copies piece lane % 8 of rows lane / 8,
    // + 4, ...; a key's score sums its even and its odd dimensions in two
    // FP32 chains (packed pair FMAs) added at the end; values accumulate two
    // dimensions per lane with packed pair FMAs (the same roundings as two
    // fmaf)
    constexpr bool PAIR = sizeof(T) == 2 && DH == 64;
    using VRaw = typename RawT<PER * (int)sizeof(T)>::type;
    const int lane = threadIdx.x & 31;
    const int tokn = gw / a.nh, h = gw % a.nh;
    const int tk = a.tok[tokn];
    const Slot &s = a.slots[tok_slot(tk)];
    const int p = tok_pos(tk);
    const int H = s.H, W = s.W, stride = s.stride;
    const int pi = p / W, pj = p % W, w = (a.k - 1) >> 1, kk = a.k * a.k;
    const int nfr = a.temporal ? s.nfr : 1;
    const int ncand = nfr * kk;
    int cnt = 0;
    // candidate cidx = fr * kk + c, window row c / k, column c % k: the
    // quotients by multiplication with the reciprocals (exact here: cidx <
    // 256 and k <= 9 keep (x + 0.5) / d at least 0.5 / d away from an
    // integer, far above the float error)
    const float inv_kk = 1.0f / (float)kk, inv_k = 1.0f / (float)a.k;
    for (int c0 = 0; c0 < ncand; c0 += 32) {
        int cidx = c0 + lane, fr = (int)(((float)cidx + 0.5f) * inv_kk), c = cidx - fr * kk;
        int cr = (int)(((float)c + 0.5f) * inv_k), qi = pi + cr - w, qj = pj + (c - cr * a.k) - w;
        bool ok = cidx < ncand && qi >= 0 && qi < H && qj >= 0 && qj < W &&
                  visible(a.mask, a.kind, W, pi, pj, qi, qj);
        unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            int at = cnt + __popc(bal & ((1u << lane) - 1u));
            int layer = a.temporal ? a.layer * a.Tf + s.ring[fr] : a.layer;
            sm.rows[at] = layer * stride + qi * W + qj;
            sm.bix[at] = (unsigned short)((a.temporal ? nfr - 1 - fr : 0) * kk + c);
        }
        cnt += __popc(bal);
    }
    if (PDL) {
        pdl_trigger();
        pdl_wait();                                    // queries, keys and values are ready from here on
    }
    const T *q = a.q_sel == CS_NONE ? (const T *)a.Q + (long)tokn * a.d + h * DH
                                    : cache_row<const T>(s, a.q_sel, 0, p, a.d) + h * DH;
    // the query travels with the first chunk's keys and values: one memory
    // round trip for all three
    if (lane < PR) cp_async16(sm.qraw + lane * 16, (const char *)q + lane * 16);
    bool qready = false;
    const char *Kb = (const char *)(cache_row<const T>(s, a.k_sel, 0, 0, a.d) + h * DH);
    const char *Vb = (const char *)(cache_row<const T>(s, a.v_sel, 0, 0, a.d) + h * DH);
    const long rsb = (long)a.d * (long)sizeof(T);              // bytes between cache rows
    const float *bias = a.bias + (long)h * a.bias_h_stride;
    const float scale = rsqrtf((float)DH);
    unsigned char *kb = sm.kbuf, *vb = sm.vbuf;
    float mx = -INFINITY, z = 0.0f, o[PER];
#pragma unroll
    for (int i = 0; i < PER; i++) o[i] = 0.0f;
    for (int base = 0; base < cnt; base += CK) {
        const int nc = min(CK, cnt - base);
        if constexpr (PAIR) {
            static_assert(PR == 8 && CK % 4 == 0, "64-wide bf16 rows: 8 pieces, 4 rows per pass");
            const int u = lane & 7;
#pragma unroll
            for (int i = 0; i < CK / 4; i++) {
                const int r = (lane >> 3) + 4 * i;
                if (r < nc) {
                    const long off = (long)sm.rows[base + r] * rsb + u * 16;
                    cp_async16(kb + r * RB + ((u ^ (r & SWM)) << 4), Kb + off);
                    cp_async16(vb + r * RB + u * 16, Vb + off);
                }
            }
        } else {
            for (int x = lane; x < nc * PR; x += 32) {
                int r = x / PR, u = x - r * PR;
                long off = (long)sm.rows[base + r] * rsb + u * 16;
                cp_async16(kb + r * RB + ((u ^ (r & SWM)) << 4), Kb + off);
                cp_async16(vb + r * RB + u * 16, Vb + off);
            }
        }
        // key lane's relative bias, loaded while the copies are in flight
        const float bz = lane < nc ? bias[sm.bix[base + lane]] : 0.0f;
        cp_async_wait_all();
        __syncwarp();
        if (!qready) {
            for (int e = lane; e < DH; e += 32) sm.qs[e] = to_f<T>(reinterpret_cast<const T *>(sm.qraw)[e]);
            __syncwarp();
            qready = true;
        }
        float sc = -INFINITY;
        if (lane < nc) {
            const uint4 *kr = reinterpret_cast<const uint4 *>(kb + lane * RB);
            const int sw = lane & SWM;
            float acc = 0.0f;
            if constexpr (PAIR) {
                const float4 *q4 = reinterpret_cast<const float4 *>(sm.qs);
                float ae = 0.0f, ao = 0.0f;                    // even and odd dimensions
#pragma unroll
                for (int u = 0; u < PR; u++) {
                    const uint4 w = kr[u ^ sw];
                    const float4 qa = q4[2 * u], qb = q4[2 * u + 1];
                    fma2(ae, ao, qa.x, qa.y, bf_lo(w.x), bf_hi(w.x));
                    fma2(ae, ao, qa.z, qa.w, bf_lo(w.y), bf_hi(w.y));
                    fma2(ae, ao, qb.x, qb.y, bf_lo(w.z), bf_hi(w.z));
                    fma2(ae, ao, qb.z, qb.w, bf_lo(w.w), bf_hi(w.w));
                }
                acc = ae + ao;
            } else {
#pragma unroll
                for (int u = 0; u < PR; u++) {
                    float kv[EPU];
                    unpack<T, EPU>(kr[u ^ sw], kv);
#pragma unroll
                    for (int i = 0; i < EPU; i++) acc = fmaf(sm.qs[u * EPU + i], kv[i], acc);
                }
            }
            sc = acc * scale + bz;
        }
        const float mnew = fmaxf(mx, warp_max(sc));
        const float corr = expf(mx - mnew);
        const float e = lane < nc ? expf(sc - mnew) : 0.0f;
        z = z * corr + warp_sum(e);
#pragma unroll
        for (int i = 0; i < PER; i++) o[i] *= corr;
        const VRaw *vr = reinterpret_cast<const VRaw *>(vb) + lane;
        if constexpr (PAIR) {
#pragma unroll
            for (int u = 0; u < CK; u++) {
                if (u >= nc) break;                            // the same for the whole warp
                const float pu = __shfl_sync(0xffffffffu, e, u);
                const uint32_t wv = vr[u * 32];
                fma2(o[0], o[1], pu, pu, bf_lo(wv), bf_hi(wv));
            }
        } else {
            for (int u = 0; u < nc; u++) {
                float pu = __shfl_sync(0xffffffffu, e, u);
                float vv[PER];
                unpack<T, PER>(vr[u * 32], vv);
#pragma unroll
                for (int i = 0; i < PER; i++) o[i] = fmaf(pu, vv[i], o[i]);
            }
        }
        mx = mnew;
        __syncwarp();                                  // the next chunk reuses the buffers
    }
    if (!qready) cp_async_wait_all();                  // no keys: the query copy lands before the buffers are reused
    const float inv = z > 0.0f ? 1.0f / z : 0.0f;
    T *out = (T *)a.O + (long)tokn * a.d + h * DH + lane * PER;
#pragma unroll
    for (int u = 0; u < PER; u++) out[u] = from_f<T>(o[u] * inv);
}

}  // namespace psw
