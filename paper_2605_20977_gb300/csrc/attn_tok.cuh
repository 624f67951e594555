// attn_tok.cuh -- masked window attention of one token and a group of TK_HG
// heads per warp (Sec. 3.2 masks, Fig. 2b), on the tensor cores (mma.sync
// m16n8k16, BF16 operands, FP32 accumulation), shared by the attention
// kernel and the persistent decoder.  For 64-wide heads (d = 64 nh, nh a
// multiple of TK_HG, at most 8).
//
// The group's heads are the rows of block-diagonal operands: row h of the
// query operand holds q_h in head h's 64 columns of the group's width and
// zeros elsewhere, so S = Q K^T over that width gives row h = q_h . K_h for
// every key; for P V the operand row h holds P_h in head h's 16-key block of
// a k-step, so row h of the product is P_h V_h.  Rows TK_HG..15 stay zero.
// One candidate list per token (the window positions its mask shows,
// frames oldest first, raster order within a window); keys 16 at a time:
// the chunk's key and value rows (all heads) are copied into shared memory
// with cp.async, 16-byte pieces XOR-swizzled by the row so ldmatrix reads
// are conflict-free; online softmax across chunks in FP32 (scores scaled by
// 1/sqrt(64), plus the relative bias); the probabilities enter P V rounded to
// BF16 and the FP32 row sum divides at the end.  A token's arithmetic
// depends only on the token, its keys and values, never on the launch.
#pragma once

#include "internal.h"
#include "device_common.cuh"
#include "attn_dev.cuh"

namespace psw {

constexpr int TK_CK = 16;          // keys per chunk: two key tiles of 8, one P V k-step
constexpr int TK_MAXC = 256;       // candidate list (Tf * k * k <= 256)
constexpr int TK_HG = 2;           // heads per warp
constexpr int TK_DW = 64 * TK_HG;  // the group's width
constexpr int TK_PR = TK_DW / 8;   // 16-byte pieces of a staged row

// Shared staging of one warp: list, then the chunk's K rows and V rows of
// the head group ([TK_CK][TK_DW] bf16 each, swizzled pieces).
__host__ __device__ constexpr size_t attn_tok_bytes()
{
    return (size_t)TK_MAXC * 4 + (size_t)TK_MAXC * 2 + 2 * (size_t)TK_CK * TK_DW * 2;
}
// Whether the token form takes these attention arguments: 64-wide BF16
// heads, and windows that show more keys than the per-(token, head) form's
// single 24-key chunk (the cyclic mask, and the unmasked temporal and LRP
// windows); the 2i+j masks keep that form, which measured faster there.
// The choice depends only on the model and the layer, never on a launch.
__host__ __device__ inline bool attn_tok_ok(int prec, int d, int nh, int mask, int kind)
{
    return prec == P_BF16 && nh >= TK_HG && nh <= 8 && nh % TK_HG == 0 && d == 64 * nh && (mask == 1 || kind < 0);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mma_bf16(float *c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Byte offset of 16-byte piece u of row r in a staged [TK_CK][TK_DW] tile.
__device__ __forceinline__ uint32_t tk_off(int r, int u) { return (uint32_t)(r * TK_PR + (u ^ (r & 7))) * 16u; }

// Warp item gw of the launch: token gw / (nh / TK_HG), heads TK_HG (gw mod
// (nh / TK_HG)) ..; sm: this warp's staging (attn_tok_bytes()).
template <bool PDL>
__device__ __forceinline__ void attn_token(const AttnArgs &a, int gw, unsigned char *sm)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int ng = a.nh / TK_HG, tokn = gw / ng, h0 = (gw - tokn * ng) * TK_HG;
    int *rows = reinterpret_cast<int *>(sm);
    unsigned short *bix = reinterpret_cast<unsigned short *>(sm + TK_MAXC * 4);
    unsigned char *kb = sm + TK_MAXC * 6, *vb = kb + TK_CK * TK_DW * 2;
    const int tk = a.tok[tokn];
    const Slot &s = a.slots[tok_slot(tk)];
    const int p = tok_pos(tk);
    const int H = s.H, W = s.W, stride = s.stride;
    const int pi = p / W, pj = p % W, w = (a.k - 1) >> 1, kk = a.k * a.k;
    const int nfr = a.temporal ? s.nfr : 1;
    const int ncand = nfr * kk;
    int cnt = 0;
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
            rows[at] = layer * stride + qi * W + qj;
            bix[at] = (unsigned short)((a.temporal ? nfr - 1 - fr : 0) * kk + c);
        }
        cnt += __popc(bal);
    }
    if (PDL) {
        pdl_trigger();
        pdl_wait();                                    // queries, keys and values are ready from here on
    }
    const int d = a.d;
    const __nv_bfloat16 *q = a.q_sel == CS_NONE ? (const __nv_bfloat16 *)a.Q + (long)tokn * d
                                                : cache_row<const __nv_bfloat16>(s, a.q_sel, 0, p, d);
    // the query fragments of this lane's head row (g < TK_HG: head h0 + g):
    // dims 16j + 2t (+1) and 16j + 8 + 2t (+1) of the head, j = 0..3
    uint32_t qa[4], qb[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        qa[j] = qb[j] = 0u;
        if (g < TK_HG) {
            const uint32_t *qr = reinterpret_cast<const uint32_t *>(q + (h0 + g) * 64 + 16 * j + 2 * t);
            qa[j] = qr[0];
            qb[j] = qr[4];
        }
    }
    // the group's slices of the key and value rows
    const char *Kb = (const char *)(cache_row<const __nv_bfloat16>(s, a.k_sel, 0, 0, d) + h0 * 64);
    const char *Vb = (const char *)(cache_row<const __nv_bfloat16>(s, a.v_sel, 0, 0, d) + h0 * 64);
    const long rsb = (long)d * 2;
    const float scale = 0.125f;                        // 1 / sqrt(64)
    const float *bias = a.bias + (long)(h0 + (g < TK_HG ? g : 0)) * a.bias_h_stride;
    float mx = -INFINITY, z = 0.0f;
    float o[8][4];
#pragma unroll
    for (int i = 0; i < 8; i++) o[i][0] = o[i][1] = o[i][2] = o[i][3] = 0.0f;
    const uint32_t kb_s = smem_u32(kb), vb_s = smem_u32(vb);
    for (int base = 0; base < cnt; base += TK_CK) {
        const int nc = min(TK_CK, cnt - base);
        for (int x = lane; x < TK_CK * TK_PR; x += 32) {
            const int r = x / TK_PR, u = x - r * TK_PR;
            const uint32_t so = tk_off(r, u);
            if (r < nc) {
                const long off = (long)rows[base + r] * rsb + u * 16;
                cp_async16(kb + so, Kb + off);
                cp_async16(vb + so, Vb + off);
            } else {
                *reinterpret_cast<uint4 *>(kb + so) = make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4 *>(vb + so) = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        cp_async_wait_all();
        __syncwarp();
        // S = Q K^T: 2 key tiles of 8, 4 k-steps per head of the group
        float sc[2][4];
#pragma unroll
        for (int i = 0; i < 2; i++) sc[i][0] = sc[i][1] = sc[i][2] = sc[i][3] = 0.0f;
        {
            const int mi = lane >> 3, key = (mi >> 1) * 8 + (lane & 7), half = mi & 1;
#pragma unroll
            for (int hd = 0; hd < TK_HG; hd++) {
#pragma unroll
                for (int j = 0; j < 4; j++) {              // k-step 4 hd + j: dims hd*64 + 16 j .. + 15
                    uint32_t b0, b1, b2, b3;
                    ldsm_x4(kb_s + tk_off(key, 8 * hd + 2 * j + half), b0, b1, b2, b3);
                    const uint32_t a0 = g == hd ? qa[j] : 0u, a2 = g == hd ? qb[j] : 0u;
                    mma_bf16(sc[0], a0, 0u, a2, 0u, b0, b1);
                    mma_bf16(sc[1], a0, 0u, a2, 0u, b2, b3);
                }
            }
        }
        // scores of row g: keys 2t, 2t + 1 (tile 0) and 8 + 2t, 9 + 2t (tile 1)
        float sv[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int key = (e >> 1) * 8 + 2 * t + (e & 1);
            sv[e] = key < nc && g < TK_HG ? sc[e >> 1][e & 1] * scale + bias[bix[base + key]] : -INFINITY;
        }
        float cm = fmaxf(fmaxf(sv[0], sv[1]), fmaxf(sv[2], sv[3]));
        cm = fmaxf(cm, __shfl_xor_sync(0xffffffffu, cm, 1));
        cm = fmaxf(cm, __shfl_xor_sync(0xffffffffu, cm, 2));
        const float mnew = fmaxf(mx, cm);
        const float corr = mnew == -INFINITY ? 1.0f : expf(mx - mnew);
        float pv[4], ps = 0.0f;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            pv[e] = sv[e] == -INFINITY ? 0.0f : expf(sv[e] - mnew);
            ps += pv[e];
        }
        ps += __shfl_xor_sync(0xffffffffu, ps, 1);
        ps += __shfl_xor_sync(0xffffffffu, ps, 2);
        z = z * corr + ps;
        mx = mnew;
#pragma unroll
        for (int i = 0; i < 8; i++) { o[i][0] *= corr; o[i][1] *= corr; }
        const uint32_t pa0 = pack_bf16(pv[0], pv[1]), pa2 = pack_bf16(pv[2], pv[3]);
        // O += P V: one k-step (the chunk's 16 keys) per head of the group, 8 dim tiles
        {
            const int mi = lane >> 3, key = (mi & 1) * 8 + (lane & 7), dhalf = mi >> 1;
#pragma unroll
            for (int hd = 0; hd < TK_HG; hd++) {
                const uint32_t a0 = g == hd ? pa0 : 0u, a2 = g == hd ? pa2 : 0u;
#pragma unroll
                for (int i = 0; i < 4; i++) {          // dims hd*64 + 16 i .. + 15
                    uint32_t b0, b1, b2, b3;
                    ldsm_x4_t(vb_s + tk_off(key, hd * 8 + 2 * i + dhalf), b0, b1, b2, b3);
                    mma_bf16(o[2 * i], a0, 0u, a2, 0u, b0, b1);
                    mma_bf16(o[2 * i + 1], a0, 0u, a2, 0u, b2, b3);
                }
            }
        }
        __syncwarp();                                  // the next chunk reuses the buffers
    }
    if (g < TK_HG) {
        const float inv = z > 0.0f ? 1.0f / z : 0.0f;
        __nv_bfloat16 *out = (__nv_bfloat16 *)a.O + (long)tokn * d + (h0 + g) * 64 + 2 * t;
#pragma unroll
        for (int i = 0; i < 8; i++)
            *reinterpret_cast<uint32_t *>(out + 8 * i) = pack_bf16(o[i][0] * inv, o[i][1] * inv);
    }
}

}  // namespace psw
