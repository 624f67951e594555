// api.cu -- the C ABI (include/psw.h): context and sequence lifetime, the
// encoder's masked parallel pass, the batched wavefront / raster decoder
// (captured once per batch shape into a CUDA graph and replayed) and the
// coder entry points.  Host code only enqueues kernels; every step of the
// model runs on the GPU.
#include "internal.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <initializer_list>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

using namespace psw;

namespace {

thread_local std::string g_create_err;

// Offsets of every tensor in the flat FP32 weight vector (packing order
// documented with psw_weights_count).
struct BlockOff {
    long g_attn, Wq, Wk, Wv, Wo, bias;
    long g_x, Wxq, Wxk, Wxv, Wxo, xbias;
    long g_ffn, Wg, Wu, Wd;
};
// A down- or upsampling residual block of the convolutional hyperprior.
struct RbOff {
    long Wa, ba, Wb, bb, Ws, bs;
};
struct Layout {
    long gamma_in, W_in, b_in, gamma_z, W_hp, b_hp;
    long g_za = -1;                                   // convolutional hyperprior (-1: none)
    std::vector<RbOff> rbd, rbu;
    long fp_H1 = -1, fp_b1 = -1, fp_a1 = -1, fp_H2 = -1, fp_b2 = -1, fp_a2 = -1, fp_H3 = -1, fp_b3 = -1,
         fp_a3 = -1, fp_H4 = -1, fp_b4 = -1;
    long gamma_c, W_c, b_c, pad, g_ctx;
    std::vector<BlockOff> ctx, sm1, sm2;
    long acc_g_q, acc_g_kv, acc_Wq, acc_Wk, acc_Wv, acc_Wo, acc_bias, acc_g_ffn, acc_Wg, acc_Wu, acc_Wd;
    long g_head, W1m, b1m, W2m, W1s, b1s, W2s, gamma_mu, beta_mu, gamma_sig, beta_sig;
    long lrp_g_rep = -1, lrp_W_rep = -1, lrp_gamma_y = -1, lrp_W_y = -1, lrp_b_in = -1;   // LRP Transformer
    std::vector<BlockOff> lrp;
    long lrp_g_out = -1, lrp_W_eps = -1, lrp_b_eps = -1;
    long ct_g_in = -1, ct_W_in = -1, ct_b_in = -1, ct_gamma_y = -1, ct_E = -1;   // Channel Transformer
    std::vector<long> ct_g_mix, ct_M, ct_g_ffn, ct_Wg, ct_Wu, ct_Wd;
    long total;
};

struct Cursor {
    long at = 0;
    long take(long n) { long o = at; at += n; return o; }
};

BlockOff layout_block(Cursor &cu, const psw_model_desc &m, bool cross, bool tf_bias)
{
    BlockOff b;
    long dd = (long)m.d * m.d, kk = (long)m.k * m.k;
    b.g_attn = cu.take(m.d);
    b.Wq = cu.take(dd); b.Wk = cu.take(dd); b.Wv = cu.take(dd); b.Wo = cu.take(dd);
    b.bias = cu.take((long)m.nh * (tf_bias ? m.Tf : 1) * kk);
    if (cross) {
        b.g_x = cu.take(m.d);
        b.Wxq = cu.take(dd); b.Wxk = cu.take(dd); b.Wxv = cu.take(dd); b.Wxo = cu.take(dd);
        b.xbias = cu.take((long)m.nh * m.Tf * kk);
    } else {
        b.g_x = b.Wxq = b.Wxk = b.Wxv = b.Wxo = b.xbias = -1;
    }
    b.g_ffn = cu.take(m.d);
    b.Wg = cu.take((long)m.d * m.F); b.Wu = cu.take((long)m.d * m.F); b.Wd = cu.take((long)m.F * m.d);
    return b;
}

// Residual blocks per hyperprior transform: log2 r (0 if r is not a power
// of two in [2, 16]).
int hyper_blocks(const psw_model_desc &m)
{
    for (int b = 1; b <= 4; b++)
        if (m.r == (1 << b)) return b;
    return 0;
}

Layout make_layout(const psw_model_desc &m)
{
    Layout y;
    Cursor cu;
    long dd = (long)m.d * m.d, kk = (long)m.k * m.k;
    y.gamma_in = cu.take(m.C); y.W_in = cu.take((long)m.C * m.d); y.b_in = cu.take(m.d);
    y.gamma_z = cu.take(m.Ch);
    if (m.hp) {
        const int nb = hyper_blocks(m);
        const long Ch = m.Ch;
        y.W_hp = y.b_hp = -1;
        y.g_za = cu.take(m.d);
        for (int b = 0; b < nb; b++) {           // analysis: d -> Ch, then Ch -> Ch
            long Ci = b == 0 ? m.d : Ch, Co = Ch;
            RbOff r;
            r.Wa = cu.take(9 * Ci * Co); r.ba = cu.take(Co); r.Wb = cu.take(9 * Co * Co); r.bb = cu.take(Co);
            r.Ws = cu.take(Ci * Co); r.bs = cu.take(Co);
            y.rbd.push_back(r);
        }
        for (int b = 0; b < nb; b++) {           // synthesis: Ch -> Ch, last Ch -> d
            long Ci = Ch, Co = b == nb - 1 ? m.d : Ch;
            RbOff r;
            r.Wa = cu.take(9 * Ci * 4 * Co); r.ba = cu.take(4 * Co); r.Wb = cu.take(9 * Co * Co); r.bb = cu.take(Co);
            r.Ws = cu.take(9 * Ci * 4 * Co); r.bs = cu.take(4 * Co);
            y.rbu.push_back(r);
        }
        y.fp_H1 = cu.take(Ch * 3); y.fp_b1 = cu.take(Ch * 3); y.fp_a1 = cu.take(Ch * 3);
        y.fp_H2 = cu.take(Ch * 9); y.fp_b2 = cu.take(Ch * 3); y.fp_a2 = cu.take(Ch * 3);
        y.fp_H3 = cu.take(Ch * 9); y.fp_b3 = cu.take(Ch * 3); y.fp_a3 = cu.take(Ch * 3);
        y.fp_H4 = cu.take(Ch * 3); y.fp_b4 = cu.take(Ch);
    } else {
        y.W_hp = cu.take((long)m.r * m.r * m.Ch * m.d); y.b_hp = cu.take(m.d);
    }
    y.gamma_c = y.W_c = y.b_c = y.pad = y.g_ctx = -1;
    if (m.temporal) {
        y.gamma_c = cu.take(m.C); y.W_c = cu.take((long)m.C * m.d); y.b_c = cu.take(m.d); y.pad = cu.take(m.d);
        for (int l = 0; l < m.Lc; l++) y.ctx.push_back(layout_block(cu, m, false, true));
        y.g_ctx = cu.take(m.d);
    }
    for (int l = 0; l < m.L; l++) y.sm1.push_back(layout_block(cu, m, m.temporal != 0, false));
    y.acc_g_q = cu.take(m.d); y.acc_g_kv = cu.take(m.d);
    y.acc_Wq = cu.take(dd); y.acc_Wk = cu.take(dd); y.acc_Wv = cu.take(dd); y.acc_Wo = cu.take(dd);
    y.acc_bias = cu.take((long)m.nh * kk);
    y.acc_g_ffn = cu.take(m.d);
    y.acc_Wg = cu.take((long)m.d * m.F); y.acc_Wu = cu.take((long)m.d * m.F); y.acc_Wd = cu.take((long)m.F * m.d);
    for (int l = 0; l < m.L; l++) y.sm2.push_back(layout_block(cu, m, m.temporal != 0, false));
    if (m.Nc) {
        long dc = m.dc, dg = dc / m.Nc, Cg = m.C / m.Nc;
        y.ct_g_in = cu.take(m.d); y.ct_W_in = cu.take((long)m.d * dc); y.ct_b_in = cu.take(dc);
        y.ct_gamma_y = cu.take(m.C); y.ct_E = cu.take((long)(m.Nc - 1) * Cg * dg);
        for (int l = 0; l < m.Lct; l++) {
            y.ct_g_mix.push_back(cu.take(dc)); y.ct_M.push_back(cu.take(dc * dc)); y.ct_g_ffn.push_back(cu.take(dc));
            y.ct_Wg.push_back(cu.take((long)m.Nc * dg * m.Fc)); y.ct_Wu.push_back(cu.take((long)m.Nc * dg * m.Fc));
            y.ct_Wd.push_back(cu.take((long)m.Nc * m.Fc * dg));
        }
        // grouped heads
        y.g_head = cu.take(dc);
        y.W1m = cu.take(m.Nc * dg * dg); y.b1m = cu.take(dc); y.W2m = cu.take(m.Nc * dg * Cg);
        y.W1s = cu.take(m.Nc * dg * dg); y.b1s = cu.take(dc); y.W2s = cu.take(m.Nc * dg * Cg);
    } else {
        y.g_head = cu.take(m.d);
        y.W1m = cu.take(dd); y.b1m = cu.take(m.d); y.W2m = cu.take((long)m.d * m.C);
        y.W1s = cu.take(dd); y.b1s = cu.take(m.d); y.W2s = cu.take((long)m.d * m.C);
    }
    y.gamma_mu = cu.take(m.C); y.beta_mu = cu.take(m.C); y.gamma_sig = cu.take(m.C); y.beta_sig = cu.take(m.C);
    if (m.Llrp) {
        long dh = m.Nc ? m.dc : m.d;
        y.lrp_g_rep = cu.take(dh); y.lrp_W_rep = cu.take(dh * m.d); y.lrp_gamma_y = cu.take(m.C);
        y.lrp_W_y = cu.take((long)m.C * m.d); y.lrp_b_in = cu.take(m.d);
        for (int l = 0; l < m.Llrp; l++) y.lrp.push_back(layout_block(cu, m, false, m.temporal != 0));
        y.lrp_g_out = cu.take(m.d); y.lrp_W_eps = cu.take((long)m.d * m.C); y.lrp_b_eps = cu.take(m.C);
    }
    y.total = cu.at;
    return y;
}

bool desc_valid(const psw_model_desc *m, std::string &why)
{
    if (!m) { why = "null model descriptor"; return false; }
    if (m->C < 1 || m->C > 4096) { why = "C must be in [1, 4096]"; return false; }
    if (m->Ch < 1 || m->Ch > 4096 || m->r < 1 || m->r > 16) { why = "bad hyperprior shape"; return false; }
    if (m->d < 32 || m->d % 32 || m->d > 4096) { why = "d must be a multiple of 32 in [32, 4096]"; return false; }
    if (m->nh < 1 || m->d % m->nh) { why = "nh must divide d"; return false; }
    int dh = m->d / m->nh;
    if (dh != 32 && dh != 64 && dh != 128) { why = "head width d/nh must be 32, 64 or 128"; return false; }
    if (m->F < 32 || m->F % 32 || m->F > 16384) { why = "F must be a multiple of 32 in [32, 16384]"; return false; }
    if (m->L < 1 || m->L > 64) { why = "L must be in [1, 64]"; return false; }
    if (m->k < 1 || m->k % 2 == 0 || m->k * m->k > MAX_KK) { why = "k must be odd with k*k <= 81"; return false; }
    if (m->mask != 0 && m->mask != 1) { why = "mask must be 0 or 1"; return false; }
    if (m->Llrp < 0 || m->Llrp > 64) { why = "Llrp must be in [0, 64]"; return false; }
    if (m->hp != 0 && m->hp != 1) { why = "hp must be 0 or 1"; return false; }
    if (m->hp && (!hyper_blocks(*m) || m->Ch > 256 || m->Ch % 4 || m->d % 4)) {
        why = "convolutional hyperprior: r a power of two in [2, 16], Ch <= 256 and Ch, d multiples of 4";
        return false;
    }
    if (m->Nc == 0) {
        if (m->dc || m->Lct || m->Fc) { why = "dc, Lct and Fc must be 0 without channel groups"; return false; }
    } else {
        if (m->Nc < 1 || m->Nc > 16 || m->C % m->Nc || m->dc < 64 || m->dc % m->Nc) {
            why = "channel groups: 1 <= Nc <= 16 dividing C and dc"; return false;
        }
        int dg = m->dc / m->Nc;
        if (dg % 64 || dg > 512) { why = "dc / Nc must be a multiple of 64, at most 512"; return false; }
        if (m->Lct < 1 || m->Lct > 16) { why = "Lct must be in [1, 16]"; return false; }
        if (m->Fc < 64 || m->Fc % 64 || m->Fc > 16384) { why = "Fc must be a multiple of 64 in [64, 16384]"; return false; }
    }
    if (m->temporal == 1) {
        if (m->Lc < 1 || m->Lc > 64) { why = "Lc must be in [1, 64]"; return false; }
        if (m->Tf < 1 || m->Tf > MAX_TF || m->Tf * m->k * m->k > 256) { why = "need Tf <= 4 and Tf*k*k <= 256"; return false; }
    } else if (m->temporal != 0) {
        why = "temporal must be 0 or 1"; return false;
    }
    return true;
}

struct BlockDev {                      // transposed projections, compute type
    void *Wqkv = nullptr, *Wo = nullptr, *Wg = nullptr, *Wu = nullptr, *Wd = nullptr;
    void *Wxq = nullptr, *Wxkv = nullptr, *Wxo = nullptr;
};

size_t esize(int prec) { return prec == P_BF16 ? 2 : 4; }

// One captured decode: graph segments of at most SEG_STEPS global steps,
// their token lists and launch count.
constexpr int SEG_STEPS = 512;
// Graph cache key: workspace generation, batch size, engine flag, then one
// (sequence pointer, grid and schedule) pair per frame from KEY_SEQ0 on.
constexpr size_t KEY_SEQ0 = 3;
struct GraphRec {
    std::vector<cudaGraphExec_t> exec;
    int *d_tok = nullptr;
    int2 *d_kn = nullptr;
    int *d_step = nullptr;             // persistent decoder: step offsets [Tmax], counts [Tmax]
    int Tmax = 0;
    double ntok = 0, ntok_prev = 0;    // tokens over all steps; those that also run Spatial Module 1
    bool persist = false;              // exec holds the prologue only; the steps run persistently
    long launches = 0;
    long used = 0;                     // last use (least recently used graphs are dropped first)
};
constexpr size_t GRAPH_CAP = 16;       // recorded batch shapes kept per context

void graph_free(GraphRec &g)
{
    for (cudaGraphExec_t e : g.exec) cudaGraphExecDestroy(e);
    g.exec.clear();
    cudaFree(g.d_tok);
    cudaFree(g.d_kn);
    cudaFree(g.d_step);
    g.d_tok = nullptr;
    g.d_kn = nullptr;
    g.d_step = nullptr;
}

}  // namespace

struct psw_ctx {
    psw_model_desc md;
    int prec = 0;                      // storage / compute type of everything but E4M3 projections
    bool fp8 = false;                  // PSW_FP8: block projections on E4M3 weights
    std::unordered_map<const void *, const float *> f8sc;   // E4M3 operand -> its per-row dequantisation scales
    size_t budget = 0, bytes = 0, arena = 0;
    Layout lay;
    float *w = nullptr;                // flat FP32 weights on the device
    char *wmat = nullptr;              // arena of transposed projections
    std::vector<BlockDev> ctxb, sm1, sm2, lrpb;
    BlockDev acc;                      // Wqkv = [Wq]; Wxkv = [Wk; Wv]
    void *Wrep = nullptr, *Wy = nullptr, *Weps = nullptr;   // LRP input [d][dh], [d][C] and output [C][d] projections
    // Channel Transformer (index g of group g, l * Nc + g of block l): input
    // rows [dg][d] of W_in, the mixing operand [dg][(g + 1) dg] (input groups
    // 0..g of output group g), SwiGLU [Fc][dg] x 2 and [dg][Fc]; grouped
    // heads [2 dg][dg], interleaved [2 Cg][2 dg] and their first-layer bias
    std::vector<void *> ct_win, ct_mix, ct_wg, ct_wu, ct_wd, ct_wh1, ct_wh2;
    std::vector<float *> ct_bh1;
    // convolutional hyperprior: convolution operands [out][K] (K = taps x
    // input channels, tap-major) per block; an RB-up block's first
    // convolution and skip stacked [8 Co][9 Ch]; merged biases (RB-down:
    // bs + bb [Co]; RB-up: ba then bs + bb per sub-position [8 Co])
    std::vector<void *> hd_wa, hd_wb, hd_ws, hu_w, hu_wb;
    std::vector<float *> hd_bias, hu_bias;
    float *hg[3] = {nullptr, nullptr, nullptr};   // FP32 grids
    void *hcol = nullptr;                         // im2col operand rows (compute type)
    size_t hg_elems = 0, hcol_elems = 0, hz_cap = 0, h_bytes = 0;
    // z-hat coder: factorized-prior tables (host copy and device) and scratch
    std::vector<uint32_t> ptab;
    uint32_t *d_pcdf = nullptr;
    int *d_pmeta = nullptr;
    uint8_t *hz_idx = nullptr;
    int32_t *hz_m = nullptr;
    int *hz_order = nullptr, *hz_status = nullptr;
    uint32_t *hz_rstate = nullptr, *hz_rptr = nullptr, *hz_rend = nullptr, *hz_nw = nullptr;
    uint16_t *hz_scratch = nullptr;
    uint64_t *hz_total = nullptr;
    void *Win = nullptr;               // latent embedding [d][C]
    std::vector<void *> Whp_t;         // tensor-core hyperprior embedding: tap t's [d][Ch] (empty: CUDA-core kernel)
    void *Wh1 = nullptr;               // heads, first layers [W1m; W1s]: [2d][d]
    void *Wh2 = nullptr;               // heads, second layers interleaved: row 2c = mu_c, 2c+1 = sigma_c: [2C][2d]
    float *bh1 = nullptr;              // [b1m; b1s]
    CdfTables tabs{};
    uint32_t *d_cdf = nullptr;
    int *d_meta = nullptr;
    float *d_scale = nullptr;
    double *rate_buf = nullptr, *h_rate = nullptr;
    size_t rate_cap = 0;
    // shared per-launch workspace (compact token rows) and the slot table
    void *Xn = nullptr, *Q = nullptr, *O = nullptr, *Hid = nullptr;
    float *Xa = nullptr, *Xb = nullptr, *Xg = nullptr;   // FP32 residual rows: SM1 / accumulator+SM2 / context
    float *Xc = nullptr;               // Channel Transformer rows, group-major: group g at Xc + g * ws_rows * dg
    uint8_t *Xn8 = nullptr;            // FP8 contexts: E4M3 token rows streamed to the wide kernel [ws_rows][<= 1024]
    float *xs8 = nullptr;              // and their dequantisation scales [ws_rows]
    void *NM = nullptr;                // its normalised mixing inputs [Lct][ws_rows][dc] (compute type)
    size_t ws_rows = 0, ws_bytes = 0;
    int ws_gen = 0;
    Slot *d_slots = nullptr, *h_slots = nullptr;
    int *d_status = nullptr;           // timeouts of bounded device waits
    int *h_status = nullptr;           // pinned: [MAX_SLOTS + 1]
    int *d_bstatus = nullptr;          // a batched decode's per-frame status words [MAX_SLOTS]
    CopyJob *d_jobs = nullptr, *h_jobs = nullptr;   // a batched decode's output copies [4 MAX_SLOTS]
    int *d_tok = nullptr;              // direct-launch token lists
    int2 *d_kn = nullptr;
    size_t tok_cap = 0, kn_cap = 0;
    cudaStream_t cap_stream = nullptr;
    std::map<std::vector<long>, GraphRec> graphs;
    long graph_clock = 0;
    bool use_graphs = true;
    // persistent decoder: the program of one step (rebuilt when the
    // workspace moves), its kernel's shared memory and grid, barrier words
    int engine = PSW_ENGINE_AUTO;
    int tile_policy[PSW_TILE_CLASSES] = {0, 0, 0, 0};   // wide kernel tokens per tile per launch class (0: automatic)
    int last_engine = 0;               // engine of the last decode (0: direct launches)
    ProgramBuilder *prog = nullptr;
    int prog_gen = -1;
    bool prog_ok = false;
    const Op *p_ops = nullptr;
    int p_nops = 0;
    const void *p_maps = nullptr;
    int p_nmaps = 0;
    double p_flops_tok[2] = {0, 0};    // algorithmic FLOPs per token of the phases on this / the previous step's tokens
    double p_bytes_tok[2] = {0, 0};    // their attention bytes per token
    double p_wbytes = 0;               // weight bytes streamed per step
    int *d_step = nullptr;             // direct-launch step tables
    size_t step_cap = 0;
    size_t p_smem = 0;
    bool p_f8 = false;                 // the program has E4M3 projections
    int p_grid = 0;
    unsigned *d_pbar = nullptr;        // [0]: barrier counter, [1]: abort flag
    std::string err;
    std::vector<psw_seq *> seqs;
    // instrumentation
    long launches = 0;
    bool prof = false;
    struct Rec { int cls; cudaEvent_t a, b; double flops, bytes; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> evpool;
    size_t evnext = 0;
};

struct psw_seq {
    psw_ctx *ctx = nullptr;
    int maxH = 0, maxW = 0, maxHW = 0;
    size_t bytes = 0;
    std::vector<void *> allocs;
    float *eh = nullptr;                                 // hyperprior tokens, FP32 [HW][d]
    void *qa = nullptr;                                  // accumulator queries [HW][d]
    void *K1 = nullptr, *V1 = nullptr, *K2 = nullptr, *V2 = nullptr, *Ka = nullptr, *Va = nullptr;
    void *CK = nullptr, *CV = nullptr, *XK = nullptr, *XV = nullptr;   // temporal rings
    void *LK = nullptr, *LV = nullptr;                   // LRP keys / values [Llrp (x Tf)][HW][d]
    float *rep = nullptr;                                // LRP input: Spatial Module 2 stream, FP32 [HW][d]
    int coded_H = 0, coded_W = 0;                        // grid of the last coded frame
    int lrp_done = 0;                                    // frames whose LRP ran (temporal model)
    float *mu = nullptr, *sigma = nullptr;
    uint8_t *idx = nullptr;
    int32_t *m = nullptr;
    int16_t *y = nullptr, *yprev = nullptr;
    int frame = 0;
    uint32_t *rstate = nullptr, *rptr = nullptr, *rend = nullptr, *enc_nw = nullptr;
    uint16_t *enc_scratch = nullptr;
    uint64_t *enc_total = nullptr, *h_total = nullptr;
    int *d_status = nullptr;
    int *d_order = nullptr;
    int sH = -1, sW = -1, sKind = -1, T = 0;
    std::vector<int> h_order, h_start;
};

namespace {

psw_status fail(psw_ctx *ctx, psw_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf; else g_create_err = buf;
    return st;
}

#define CK_CUDA(ctx, call)                                                                                \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return fail(ctx, PSW_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

const float *W(const psw_ctx *c, long off) { return c->w + off; }

// ---------------------------------------------------------------- instrumentation

// Kernel classes reported by psw_profile_end.
enum KClass { K_GEMM_TC, K_GEMM_SIMT, K_ATTN, K_NORM, K_EMBED, K_HEADS, K_RANS, K_OTHER, K_PERSIST, K_NCLASS };
const char *const kclass_name[K_NCLASS] = {"gemm_tc", "gemm_simt", "attention", "rmsnorm",
                                          "embed", "heads", "rans", "other", "persistent"};

cudaEvent_t ev_get(psw_ctx *c)
{
    if (c->evnext == c->evpool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->evpool.push_back(e);
    }
    return c->evpool[c->evnext++];
}

// Counts one kernel launch; when profiling, brackets it with events.
struct Scope {
    psw_ctx *c;
    cudaStream_t s;
    psw_ctx::Rec r;
    Scope(psw_ctx *c_, cudaStream_t s_, int cls, double flops, double bytes) : c(c_), s(s_)
    {
        c->launches++;
        if (c->prof) {
            r = psw_ctx::Rec{cls, ev_get(c), ev_get(c), flops, bytes};
            cudaEventRecord(r.a, s);
        }
    }
    ~Scope()
    {
        if (c->prof) {
            cudaEventRecord(r.b, s);
            c->recs.push_back(r);
        }
    }
};

#define LAUNCH(P_, cls, flops, bytes, call)                 \
    do {                                                    \
        Scope sc_((P_).c, (P_).s, (cls), (flops), (bytes)); \
        call;                                               \
    } while (0)

// ---------------------------------------------------------------- weights

// Transposed ([out][in], K-major), compute-typed copies of every block
// projection, carved from one arena.  A dry run only sums the sizes.  In an
// FP8 context every block projection the E4M3 tile takes is stored as E4M3
// bytes, each source tensor (Wq, Wk, Wv, Wg, ... of each block) quantised
// with its own power-of-two scale, and followed by its vector of per-row
// dequantisation scales; the latent embedding and the heads stay BF16.
bool prepare_projections(psw_ctx *c, bool dry)
{
    const psw_model_desc &m = c->md;
    const Layout &lay = c->lay;
    int d = m.d, prec = c->prec;
    size_t es = esize(prec), used = 0;
    bool ok = true;
    bool no8 = false;                  // set: operands stay in the compute type even in an FP8 context
    float *stage = nullptr;            // one source tensor in FP32 [N][K] before E4M3 quantisation
    if (!dry && c->fp8 && cudaMalloc(&stage, (size_t)std::max(m.F, d) * std::max(m.F, d) * 4) != cudaSuccess)
        return false;
    auto carve_b = [&](size_t bytes) -> void * {
        size_t sz = ((bytes + 255) / 256) * 256;
        void *p = dry ? nullptr : (void *)(c->wmat + used);
        used += sz;
        return p;
    };
    auto carve = [&](size_t rows, size_t cols) -> void * { return carve_b(rows * cols * es); };
    auto tr = [&](long off, int K, int N, void *dst, int row_off) {
        if (!dry) launch_transpose_convert(prec, c->w + off, K, N, dst, row_off, 0);
    };
    // One projection operand [N][K] from source tensors [K][n_i] (flat
    // offsets) stacked at consecutive rows; asrc: how its tokens are built.
    auto operand = [&](int N, int K, int asrc, std::initializer_list<long> srcs) -> void * {
        bool f8 = c->fp8 && !no8 && gemm_tc8_supported(N, K, asrc);
        void *p = carve_b((size_t)N * K * (f8 ? 1 : es));
        float *sc = f8 ? (float *)carve_b((size_t)N * 4) : nullptr;
        int n = N / (int)srcs.size(), row = 0;
        for (long off : srcs) {
            if (dry) continue;
            if (!f8) {
                tr(off, K, n, p, row);
            } else {
                launch_transpose_convert(P_F32, c->w + off, K, n, stage, 0, 0);
                float s = quantize_e4m3(stage, (size_t)n * K, (uint8_t *)p + (size_t)row * K);
                std::vector<float> hs(n, s);
                if (s <= 0.0f || cudaMemcpy(sc + row, hs.data(), (size_t)n * 4, cudaMemcpyHostToDevice) != cudaSuccess)
                    ok = false;
            }
            row += n;
        }
        if (f8 && !dry) c->f8sc[p] = sc;
        return p;
    };
    auto mk_block = [&](const BlockOff &bo, bool cross) {
        BlockDev b;
        b.Wqkv = operand(3 * d, d, A_NORM, {bo.Wq, bo.Wk, bo.Wv});
        b.Wo = operand(d, d, A_DIRECT, {bo.Wo});
        b.Wg = operand(m.F, d, A_NORM, {bo.Wg});
        b.Wu = operand(m.F, d, A_NORM, {bo.Wu});
        b.Wd = operand(d, m.F, A_DIRECT, {bo.Wd});
        if (cross) {
            b.Wxq = operand(d, d, A_NORM, {bo.Wxq});
            b.Wxkv = operand(2 * d, d, A_NORM, {bo.Wxk, bo.Wxv});
            b.Wxo = operand(d, d, A_DIRECT, {bo.Wxo});
        }
        return b;
    };
    std::vector<BlockDev> ctxb, sm1, sm2;
    if (m.temporal)
        for (int l = 0; l < m.Lc; l++) ctxb.push_back(mk_block(lay.ctx[l], false));
    for (int l = 0; l < m.L; l++) sm1.push_back(mk_block(lay.sm1[l], m.temporal != 0));
    for (int l = 0; l < m.L; l++) sm2.push_back(mk_block(lay.sm2[l], m.temporal != 0));
    BlockDev ab;
    ab.Wqkv = operand(d, d, A_NORM, {lay.acc_Wq});
    ab.Wxkv = operand(2 * d, d, A_NORM, {lay.acc_Wk, lay.acc_Wv});
    ab.Wo = operand(d, d, A_DIRECT, {lay.acc_Wo});
    ab.Wg = operand(m.F, d, A_NORM, {lay.acc_Wg});
    ab.Wu = operand(m.F, d, A_NORM, {lay.acc_Wu});
    ab.Wd = operand(d, m.F, A_DIRECT, {lay.acc_Wd});
    // the LRP Transformer's projections stay in the compute type (BF16 in an
    // FP8 context)
    std::vector<BlockDev> lrpb;
    void *wrep = nullptr, *weps = nullptr, *wy = nullptr;
    no8 = true;
    for (int l = 0; l < m.Llrp; l++) lrpb.push_back(mk_block(lay.lrp[l], false));
    if (m.Llrp) {
        wrep = operand(d, m.Nc ? m.dc : d, A_NORM, {lay.lrp_W_rep});
        weps = operand(m.C, d, A_NORM, {lay.lrp_W_eps});
    }
    // the Channel Transformer's projections stay in the compute type as well
    std::vector<void *> ct_win, ct_mix, ct_wg, ct_wu, ct_wd, ct_wh1, ct_wh2;
    std::vector<float *> ct_bh1;
    const int G = m.Nc, dg = G ? m.dc / G : 0, Cg = G ? m.C / G : 0;
    if (G) {
        char *win = (char *)operand(m.dc, d, A_NORM, {lay.ct_W_in});
        for (int g = 0; g < G; g++) ct_win.push_back(dry ? nullptr : win + (size_t)g * dg * d * es);
        for (int l = 0; l < m.Lct; l++)
            for (int g = 0; g < G; g++) {
                ct_wg.push_back(operand(m.Fc, dg, A_NORM, {lay.ct_Wg[l] + (long)g * dg * m.Fc}));
                ct_wu.push_back(operand(m.Fc, dg, A_NORM, {lay.ct_Wu[l] + (long)g * dg * m.Fc}));
                ct_wd.push_back(operand(dg, m.Fc, A_DIRECT, {lay.ct_Wd[l] + (long)g * m.Fc * dg}));
                ct_mix.push_back(carve(dg, (size_t)(g + 1) * dg));      // assembled below
            }
        for (int g = 0; g < G; g++) {
            void *h1 = carve(2 * dg, dg);
            tr(lay.W1m + (long)g * dg * dg, dg, dg, h1, 0);
            tr(lay.W1s + (long)g * dg * dg, dg, dg, h1, dg);
            ct_wh1.push_back(h1);
            ct_wh2.push_back(carve(2 * (size_t)Cg, 2 * dg));             // assembled below
            ct_bh1.push_back((float *)carve(2 * dg, es == 2 ? 2 : 1));   // 2 dg floats
        }
    }
    std::vector<void *> hd_wa, hd_wb, hd_ws, hu_w, hu_wb;
    std::vector<float *> hd_bias, hu_bias;
    if (m.hp) {
        const int nb = hyper_blocks(m), Ch = m.Ch;
        for (int b = 0; b < nb; b++) {
            const int Ci = b == 0 ? d : Ch, Co = Ch;
            hd_wa.push_back(operand(Co, 9 * Ci, A_DIRECT, {lay.rbd[b].Wa}));
            hd_wb.push_back(operand(Co, 9 * Co, A_DIRECT, {lay.rbd[b].Wb}));
            hd_ws.push_back(operand(Co, Ci, A_DIRECT, {lay.rbd[b].Ws}));
            hd_bias.push_back((float *)carve_b((size_t)Co * 4));
        }
        for (int b = 0; b < nb; b++) {
            const int Ci = Ch, Co = b == nb - 1 ? d : Ch;
            hu_w.push_back(operand(8 * Co, 9 * Ci, A_DIRECT, {lay.rbu[b].Wa, lay.rbu[b].Ws}));
            hu_wb.push_back(operand(Co, 9 * Co, A_DIRECT, {lay.rbu[b].Wb}));
            hu_bias.push_back((float *)carve_b((size_t)8 * Co * 4));
        }
    }
    cudaFree(stage);
    if (!ok) return false;
    void *win = carve(d, m.C); tr(lay.W_in, m.C, d, win, 0);
    // the hyperprior token embedding as r * r projections (one per sub-pixel
    // tap) on the tensor cores, where their shape takes them
    std::vector<void *> whp_t;
    if (!m.hp && prec == P_BF16 && gemm_tc_supported(P_BF16, d, m.Ch, A_ZHAT))
        for (int t = 0; t < m.r * m.r; t++) {
            void *wt = carve(d, m.Ch);
            tr(lay.W_hp + (long)t * m.Ch * d, m.Ch, d, wt, 0);
            whp_t.push_back(wt);
        }
    if (m.Llrp) { wy = carve(d, m.C); tr(lay.lrp_W_y, m.C, d, wy, 0); }
    // the plain heads (the grouped heads of a Channel Transformer replace them)
    void *wh1 = nullptr, *wh2 = nullptr;
    float *bh1 = nullptr;
    if (!G) {
        wh1 = carve(2 * d, d); tr(lay.W1m, d, d, wh1, 0); tr(lay.W1s, d, d, wh1, d);
        wh2 = carve(2 * (size_t)m.C, 2 * d);
        bh1 = (float *)carve(2 * d, es == 2 ? 2 : 1);            // 2d floats
    }
    if (dry) { c->arena = used; return true; }
    if (used > c->arena) return false;
    // interleaved block-diagonal second layer, assembled in FP32 then converted
    if (!G) {
        std::vector<float> w2m((size_t)d * m.C), w2s((size_t)d * m.C), buf((size_t)2 * m.C * 2 * d, 0.0f);
        cudaMemcpy(w2m.data(), c->w + lay.W2m, w2m.size() * 4, cudaMemcpyDeviceToHost);
        cudaMemcpy(w2s.data(), c->w + lay.W2s, w2s.size() * 4, cudaMemcpyDeviceToHost);
        for (int ch = 0; ch < m.C; ch++)
            for (int e = 0; e < d; e++) {
                buf[(size_t)(2 * ch) * 2 * d + e] = w2m[(size_t)e * m.C + ch];
                buf[(size_t)(2 * ch + 1) * 2 * d + d + e] = w2s[(size_t)e * m.C + ch];
            }
        float *tmp = nullptr;
        if (cudaMalloc(&tmp, buf.size() * 4) != cudaSuccess) return false;
        cudaMemcpy(tmp, buf.data(), buf.size() * 4, cudaMemcpyHostToDevice);
        launch_convert(prec, tmp, buf.size(), wh2, 0);
        cudaDeviceSynchronize();
        cudaFree(tmp);
        cudaMemcpy(bh1, c->w + lay.b1m, d * 4, cudaMemcpyDeviceToDevice);
        cudaMemcpy(bh1 + d, c->w + lay.b1s, d * 4, cudaMemcpyDeviceToDevice);
    }
    if (G) {
        // mixing operands: output group g's columns of M over input groups
        // 0..g (the block-lower-triangular mask), [K = (g+1) dg][N = dg] in
        // FP32, then transposed and converted; grouped heads' second layers
        // interleaved as for the plain heads
        const int dc = m.dc;
        std::vector<float> M((size_t)dc * dc), buf;
        float *tmp = nullptr;
        if (cudaMalloc(&tmp, (size_t)dc * dc * 4) != cudaSuccess) return false;
        for (int l = 0; l < m.Lct; l++) {
            cudaMemcpy(M.data(), c->w + lay.ct_M[l], M.size() * 4, cudaMemcpyDeviceToHost);
            for (int g = 0; g < G; g++) {
                int K = (g + 1) * dg;
                buf.assign((size_t)K * dg, 0.0f);
                for (int i = 0; i < K; i++)
                    for (int o = 0; o < dg; o++) buf[(size_t)i * dg + o] = M[(size_t)i * dc + g * dg + o];
                cudaMemcpy(tmp, buf.data(), buf.size() * 4, cudaMemcpyHostToDevice);
                launch_transpose_convert(prec, tmp, K, dg, ct_mix[(size_t)l * G + g], 0, 0);
                cudaDeviceSynchronize();
            }
        }
        std::vector<float> w2m((size_t)dg * Cg), w2s((size_t)dg * Cg);
        for (int g = 0; g < G; g++) {
            cudaMemcpy(w2m.data(), c->w + lay.W2m + (long)g * dg * Cg, w2m.size() * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(w2s.data(), c->w + lay.W2s + (long)g * dg * Cg, w2s.size() * 4, cudaMemcpyDeviceToHost);
            buf.assign((size_t)2 * Cg * 2 * dg, 0.0f);
            for (int ch = 0; ch < Cg; ch++)
                for (int e = 0; e < dg; e++) {
                    buf[(size_t)(2 * ch) * 2 * dg + e] = w2m[(size_t)e * Cg + ch];
                    buf[(size_t)(2 * ch + 1) * 2 * dg + dg + e] = w2s[(size_t)e * Cg + ch];
                }
            cudaMemcpy(tmp, buf.data(), buf.size() * 4, cudaMemcpyHostToDevice);
            launch_convert(prec, tmp, buf.size(), ct_wh2[g], 0);
            cudaDeviceSynchronize();
            cudaMemcpy(ct_bh1[g], c->w + lay.b1m + (long)g * dg, dg * 4, cudaMemcpyDeviceToDevice);
            cudaMemcpy(ct_bh1[g] + dg, c->w + lay.b1s + (long)g * dg, dg * 4, cudaMemcpyDeviceToDevice);
        }
        cudaFree(tmp);
    }
    c->ctxb = ctxb; c->sm1 = sm1; c->sm2 = sm2; c->acc = ab;
    c->lrpb = lrpb; c->Wrep = wrep; c->Wy = wy; c->Weps = weps;
    if (m.hp) {
        // merged biases of the residual sums (host FP32 additions)
        const int nb = hyper_blocks(m), Ch = m.Ch;
        std::vector<float> a, b2, b3, buf;
        for (int b = 0; b < nb; b++) {
            a.resize(Ch); b2.resize(Ch);
            cudaMemcpy(a.data(), c->w + lay.rbd[b].bs, Ch * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(b2.data(), c->w + lay.rbd[b].bb, Ch * 4, cudaMemcpyDeviceToHost);
            for (int o = 0; o < Ch; o++) a[o] += b2[o];
            cudaMemcpy(hd_bias[b], a.data(), Ch * 4, cudaMemcpyHostToDevice);
        }
        for (int b = 0; b < nb; b++) {
            const int Co = b == nb - 1 ? d : Ch;
            a.resize(4 * Co); b2.resize(4 * Co); b3.resize(Co); buf.assign(8 * Co, 0.0f);
            cudaMemcpy(a.data(), c->w + lay.rbu[b].ba, 4 * Co * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(b2.data(), c->w + lay.rbu[b].bs, 4 * Co * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(b3.data(), c->w + lay.rbu[b].bb, Co * 4, cudaMemcpyDeviceToHost);
            for (int e = 0; e < 4 * Co; e++) buf[e] = a[e];
            for (int sub = 0; sub < 4; sub++)
                for (int o = 0; o < Co; o++) buf[4 * Co + sub * Co + o] = b2[sub * Co + o] + b3[o];
            cudaMemcpy(hu_bias[b], buf.data(), 8 * Co * 4, cudaMemcpyHostToDevice);
        }
    }
    c->ct_win = ct_win; c->ct_mix = ct_mix; c->ct_wg = ct_wg; c->ct_wu = ct_wu; c->ct_wd = ct_wd;
    c->ct_wh1 = ct_wh1; c->ct_wh2 = ct_wh2; c->ct_bh1 = ct_bh1;
    c->hd_wa = hd_wa; c->hd_wb = hd_wb; c->hd_ws = hd_ws; c->hu_w = hu_w; c->hu_wb = hu_wb;
    c->hd_bias = hd_bias; c->hu_bias = hu_bias;
    c->Win = win; c->Wh1 = wh1; c->Wh2 = wh2; c->bh1 = bh1;
    c->Whp_t = whp_t;
    return true;
}

// ---------------------------------------------------------------- factorized prior

// The factorized prior of z-hat (Fig. 1 right; the univariate density of
// Balle et al. 2018): per channel the cumulative
// c(x) = sigmoid(f4(f3(f2(f1(x))))) through widths 1 -> 3 -> 3 -> 3 -> 1,
// f_k(v) = g_k(softplus(H_k) v + b_k), g_k(t) = t + tanh(a_k) tanh(t) for
// k < 4, f_4 affine; double precision, sums over ascending inputs after the
// bias.  Host code: the tables are built once per context.
double prior_softplus(double x) { return x > 30.0 ? x : log1p(exp(x)); }

double prior_cdf(const Layout &L, const float *w, int ch, double x)
{
    auto W_ = [&](long off) { return (double)w[off]; };
    double v1[3], v2[3], v3[3];
    for (int i = 0; i < 3; i++) {
        double t = W_(L.fp_b1 + ch * 3 + i) + prior_softplus(W_(L.fp_H1 + ch * 3 + i)) * x;
        v1[i] = t + tanh(W_(L.fp_a1 + ch * 3 + i)) * tanh(t);
    }
    for (int i = 0; i < 3; i++) {
        double t = W_(L.fp_b2 + ch * 3 + i);
        for (int k = 0; k < 3; k++) t += prior_softplus(W_(L.fp_H2 + (ch * 3 + i) * 3 + k)) * v1[k];
        v2[i] = t + tanh(W_(L.fp_a2 + ch * 3 + i)) * tanh(t);
    }
    for (int i = 0; i < 3; i++) {
        double t = W_(L.fp_b3 + ch * 3 + i);
        for (int k = 0; k < 3; k++) t += prior_softplus(W_(L.fp_H3 + (ch * 3 + i) * 3 + k)) * v2[k];
        v3[i] = t + tanh(W_(L.fp_a3 + ch * 3 + i)) * tanh(t);
    }
    double t = W_(L.fp_b4 + ch);
    for (int k = 0; k < 3; k++) t += prior_softplus(W_(L.fp_H4 + ch * 3 + k)) * v3[k];
    return 1.0 / (1.0 + exp(-t));
}

constexpr int PRIOR_T = 31;                 // support half-width of every channel's table
constexpr int PRIOR_N = 2 * PRIOR_T + 2;    // slots: -T..T, escape

// Packed tables (cum | freq << 16, PRIOR_N slots per channel) with the
// scale tables' rule: freq = 1 + floor(pmf (2^16 - n)), escape = both tails,
// the remainder to symbol 0.
void build_prior_tables(const psw_model_desc &m, const Layout &L, const float *w, std::vector<uint32_t> &packed)
{
    packed.assign((size_t)m.Ch * PRIOR_N, 0);
    const int T = PRIOR_T, n = PRIOR_N;
    const double room = (double)((1u << CDF_PREC) - (uint32_t)n);
    uint32_t fr[PRIOR_N];
    for (int ch = 0; ch < m.Ch; ch++) {
        long sum = 0;
        for (int v = -T; v <= T; v++) {
            double pmf = prior_cdf(L, w, ch, v + 0.5) - prior_cdf(L, w, ch, v - 0.5);
            fr[v + T] = 1u + (uint32_t)floor(pmf * room);
            sum += fr[v + T];
        }
        double pesc = prior_cdf(L, w, ch, -T - 0.5) + (1.0 - prior_cdf(L, w, ch, T + 0.5));
        fr[2 * T + 1] = 1u + (uint32_t)floor(pesc * room);
        sum += fr[2 * T + 1];
        fr[T] = (uint32_t)((long)fr[T] + ((long)(1u << CDF_PREC) - sum));
        uint32_t cum = 0;
        for (int sl = 0; sl < n; sl++) {
            packed[(size_t)ch * n + sl] = cum | (fr[sl] << 16);
            cum += fr[sl];
        }
    }
}

// ---------------------------------------------------------------- schedules

// PSW_SCHED_WAVEFRONT: positions grouped by mask label in ascending label
// order (raster order inside a step); PSW_SCHED_RASTER: one position per
// step.  order: positions in schedule order; step t is order[start[t] ..
// start[t+1]).
void build_schedule(const psw_model_desc &m, int H, int W_, int kind, std::vector<int> &order,
                    std::vector<int> &start)
{
    int HW = H * W_;
    order.assign(HW, 0);
    start.clear();
    if (kind == PSW_SCHED_RASTER) {
        for (int p = 0; p <= HW; p++) start.push_back(p);
        for (int p = 0; p < HW; p++) order[p] = p;
        return;
    }
    auto lab = [&](int i, int j) { return m.mask == 1 ? ((i % 4) + (j % 4)) % 4 : 2 * i + j; };
    int maxl = 0;
    for (int i = 0; i < H; i++)
        for (int j = 0; j < W_; j++) maxl = std::max(maxl, lab(i, j));
    std::vector<int> cnt(maxl + 1, 0), fillp(maxl + 1, 0);
    for (int i = 0; i < H; i++)
        for (int j = 0; j < W_; j++) cnt[lab(i, j)]++;
    int at = 0;
    for (int t = 0; t <= maxl; t++) {
        fillp[t] = at;
        if (cnt[t] > 0) start.push_back(at);
        at += cnt[t];
    }
    start.push_back(HW);
    for (int i = 0; i < H; i++)
        for (int j = 0; j < W_; j++) order[fillp[lab(i, j)]++] = i * W_ + j;
}

psw_status seq_schedule(psw_seq *q, int H, int W_, int kind)
{
    if (q->sH == H && q->sW == W_ && q->sKind == kind) return PSW_OK;
    build_schedule(q->ctx->md, H, W_, kind, q->h_order, q->h_start);
    q->T = (int)q->h_start.size() - 1;
    CK_CUDA(q->ctx, cudaMemcpy(q->d_order, q->h_order.data(), sizeof(int) * H * W_, cudaMemcpyHostToDevice));
    q->sH = H; q->sW = W_; q->sKind = kind;
    return PSW_OK;
}

// The slot of a sequence's current frame (pointers to its caches).
// frame: the frame index the slot describes (default: the next to code).
Slot make_slot(const psw_seq *q, int H, int W_, int sched, int frame = -1)
{
    const psw_model_desc &m = q->ctx->md;
    Slot s;
    memset(&s, 0, sizeof(s));
    if (frame < 0) frame = q->frame;
    s.H = H; s.W = W_; s.stride = q->maxHW; s.frame = frame; s.sched = sched;
    s.nfr = 1;
    if (m.temporal) {
        int f = frame, f0 = std::max(0, f - m.Tf + 1);
        s.nfr = f - f0 + 1;
        for (int u = 0; u < s.nfr; u++) s.ring[u] = (f0 + u) % m.Tf;
    }
    s.eh = q->eh;
    s.qa = q->qa; s.K1 = q->K1; s.V1 = q->V1; s.K2 = q->K2; s.V2 = q->V2; s.Ka = q->Ka; s.Va = q->Va;
    s.CK = q->CK; s.CV = q->CV; s.XK = q->XK; s.XV = q->XV;
    s.LK = q->LK; s.LV = q->LV; s.rep = q->rep;
    s.mu = q->mu; s.sigma = q->sigma; s.idx = q->idx; s.m = q->m; s.y = q->y;
    s.yprev = q->yprev;
    s.rstate = q->rstate; s.rptr = q->rptr; s.rend = q->rend;
    s.order = q->d_order;
    s.status = q->d_status;
    return s;
}

// ---------------------------------------------------------------- workspace

// Workspace bytes for `rows` token rows: operand rows (queries, attention
// output, normalised or embedding operands: the widest token operand),
// hidden rows (SwiGLU, heads), the FP32 residual rows of Spatial Module 1,
// the accumulator / Spatial Module 2 and the Context Transformer, and the
// Channel Transformer's FP32 rows and normalised mixing inputs.
void ws_sizes(const psw_model_desc &m, int prec, size_t rows, size_t &bd, size_t &bf, size_t &bx, size_t &bg,
              size_t &bc, size_t &bn)
{
    size_t es = esize(prec);
    int wop = std::max({m.d, m.C, m.Nc ? m.dc : 0});
    int whid = std::max({m.F, 2 * m.d, m.Nc ? m.Fc : 0, m.Nc ? 2 * (m.dc / m.Nc) : 0});
    bd = rows * wop * es;
    bf = rows * whid * es;
    bx = rows * m.d * 4;
    bg = m.temporal ? bx : 16;
    bc = m.Nc ? rows * m.dc * 4 : 16;
    bn = m.Nc ? (size_t)m.Lct * rows * m.dc * es : 16;
}

psw_status ensure_workspace(psw_ctx *c, size_t rows)
{
    if (rows <= c->ws_rows) return PSW_OK;
    const psw_model_desc &m = c->md;
    size_t es = esize(c->prec);
    CK_CUDA(c, cudaDeviceSynchronize());
    cudaFree(c->Xn); cudaFree(c->Q); cudaFree(c->O); cudaFree(c->Hid);
    cudaFree(c->Xa); cudaFree(c->Xb); cudaFree(c->Xg); cudaFree(c->Xc); cudaFree(c->NM);
    cudaFree(c->Xn8); cudaFree(c->xs8);
    c->Xn = c->Q = c->O = c->Hid = c->NM = nullptr;
    c->Xa = c->Xb = c->Xg = c->Xc = nullptr;
    c->Xn8 = nullptr; c->xs8 = nullptr;
    c->bytes -= c->ws_bytes;
    c->ws_rows = 0; c->ws_bytes = 0;
    size_t bd, bf, bx, bg, bc, bn;
    ws_sizes(m, c->prec, rows, bd, bf, bx, bg, bc, bn);
    if (cudaMalloc(&c->Xn, bd) != cudaSuccess || cudaMalloc(&c->Q, bd) != cudaSuccess ||
        cudaMalloc(&c->O, bd) != cudaSuccess || cudaMalloc(&c->Hid, bf) != cudaSuccess ||
        cudaMalloc(&c->Xa, bx) != cudaSuccess || cudaMalloc(&c->Xb, bx) != cudaSuccess ||
        cudaMalloc(&c->Xg, bg) != cudaSuccess || cudaMalloc(&c->Xc, bc) != cudaSuccess ||
        cudaMalloc(&c->NM, bn) != cudaSuccess)
        return fail(c, PSW_ERR_OOM, "workspace of %zu rows", rows);
    const size_t b8 = c->fp8 ? rows * 1024 : 16, bs8 = c->fp8 ? rows * 4 : 16;
    if (cudaMalloc(&c->Xn8, b8) != cudaSuccess || cudaMalloc(&c->xs8, bs8) != cudaSuccess)
        return fail(c, PSW_ERR_OOM, "workspace of %zu rows", rows);
    c->ws_rows = rows;
    c->ws_bytes = 3 * bd + bf + 2 * bx + bg + bc + bn + b8 + bs8;
    c->bytes += c->ws_bytes;
    c->ws_gen++;
    for (auto &kv : c->graphs) graph_free(kv.second);
    c->graphs.clear();
    return PSW_OK;
}

// Hyperprior workspace for frames up to H x W: the largest FP32 grid and
// im2col operand over the analysis and synthesis blocks, and the z-hat
// coder's scratch for the ceil(H/r) x ceil(W/r) grid.
void hyper_sizes(const psw_model_desc &m, int H, int W_, size_t &grid, size_t &col, size_t &hz)
{
    const int nb = hyper_blocks(m), r = m.r, Ch = m.Ch, d = m.d;
    grid = (size_t)H * W_ * d;
    col = 0;
    int h = H, w = W_, Ci = d;
    for (int b = 0; b < nb; b++) {
        int ho = (h + 1) / 2, wo = (w + 1) / 2;
        size_t P = (size_t)ho * wo;
        grid = std::max(grid, P * Ch);
        col = std::max(col, std::max(P * 9 * Ci, P * 9 * Ch));
        h = ho; w = wo; Ci = Ch;
    }
    h = (H + r - 1) / r; w = (W_ + r - 1) / r;
    hz = (size_t)h * w;
    grid = std::max(grid, hz * Ch);
    for (int b = 0; b < nb; b++) {
        const int Co = b == nb - 1 ? d : Ch;
        size_t P = (size_t)h * w;
        grid = std::max(grid, std::max(P * 8 * Co, 4 * P * Co));
        col = std::max(col, std::max(P * 9 * Ch, 4 * P * 9 * Co));
        h *= 2; w *= 2;
    }
}

psw_status ensure_hyper(psw_ctx *c, int H, int W_)
{
    if (!c->md.hp) return PSW_OK;
    size_t grid, col, hz;
    hyper_sizes(c->md, H, W_, grid, col, hz);
    if (grid <= c->hg_elems && col <= c->hcol_elems && hz <= c->hz_cap) return PSW_OK;
    grid = std::max(grid, c->hg_elems); col = std::max(col, c->hcol_elems); hz = std::max(hz, c->hz_cap);
    CK_CUDA(c, cudaDeviceSynchronize());
    for (float *&g : c->hg) { cudaFree(g); g = nullptr; }
    cudaFree(c->hcol); cudaFree(c->hz_idx); cudaFree(c->hz_m); cudaFree(c->hz_order); cudaFree(c->hz_status);
    cudaFree(c->hz_rstate); cudaFree(c->hz_rptr); cudaFree(c->hz_rend); cudaFree(c->hz_nw); cudaFree(c->hz_scratch);
    cudaFree(c->hz_total);
    c->hcol = nullptr; c->hz_idx = nullptr; c->hz_m = nullptr; c->hz_order = c->hz_status = nullptr;
    c->hz_rstate = c->hz_rptr = c->hz_rend = c->hz_nw = nullptr; c->hz_scratch = nullptr; c->hz_total = nullptr;
    c->bytes -= c->h_bytes;
    c->h_bytes = 0; c->hg_elems = c->hcol_elems = c->hz_cap = 0;
    const size_t Ch = c->md.Ch, es = esize(c->prec);
    bool ok = true;
    size_t bytes = 0;
    auto al = [&](void **p, size_t b) {
        if (ok && cudaMalloc(p, b ? b : 16) != cudaSuccess) ok = false;
        bytes += b;
    };
    for (float *&g : c->hg) al((void **)&g, grid * 4);
    al(&c->hcol, col * es);
    al((void **)&c->hz_idx, hz * Ch);
    al((void **)&c->hz_m, hz * Ch * 4);
    al((void **)&c->hz_order, hz * 4);
    al((void **)&c->hz_status, 4);
    al((void **)&c->hz_rstate, Ch * 32 * 4);
    al((void **)&c->hz_rptr, Ch * 4);
    al((void **)&c->hz_rend, Ch * 4);
    al((void **)&c->hz_nw, (2 * Ch + 1) * 4);
    al((void **)&c->hz_scratch, Ch * (3 * hz + 64) * 2);
    al((void **)&c->hz_total, 8);
    if (!ok) return fail(c, PSW_ERR_OOM, "hyperprior workspace for %dx%d", H, W_);
    c->hg_elems = grid; c->hcol_elems = col; c->hz_cap = hz; c->h_bytes = bytes;
    c->bytes += bytes;
    launch_hyper_coder_tables((int)hz, (int)Ch, c->hz_idx, c->hz_m, c->hz_order, 0);
    CK_CUDA(c, cudaDeviceSynchronize());
    // recorded graphs name the old buffers
    c->ws_gen++;
    for (auto &kv : c->graphs) graph_free(kv.second);
    c->graphs.clear();
    return PSW_OK;
}

// ---------------------------------------------------------------- model passes

struct Pass {
    psw_ctx *c;
    cudaStream_t s;
    const Slot *S;                     // device slot table
    bool *failed;
    ProgramBuilder *rec = nullptr;     // set: record phases of the persistent decoder instead of launching
    int tokset = TS_CUR;               // which step's tokens recorded phases work on
    // the workspace Xn holds bf16(RMSNorm(xn_rows[m]) * xn_gain) for m < xn_m
    // (written by the last launch that produced or updated those rows)
    mutable const float *xn_rows = nullptr, *xn_gain = nullptr;
    mutable int xn_m = 0;
    // FP8: Xn8 / xs8 hold the E4M3 rows of RMSNorm(x8_rows[m]) * x8_gain for m < x8_m
    mutable const float *x8_rows = nullptr, *x8_gain = nullptr;
    mutable int x8_m = 0;
};

// One projection; asrc / a_stream / a_gain say where its token operand
// comes from (compact rows A, the RMSNorm of a residual stream, or the
// channel-scaled latents).
void gemm_any(const Pass &P, int asrc, const float *xrows, const float *a_gain, const void *A, int lda, const void *Wt,
              const void *Wt2, int M, int N, int K, const Epi &e)
{
    if (M <= 0) return;
    const bool writes_rows = e.mode == EPI_RESID || e.mode == EPI_RESID_BASE || e.mode == EPI_SET_BIAS;
    GemmArgs g{};
    g.A = A; g.lda = lda; g.asrc = asrc; g.xrows = xrows; g.a_gain = a_gain; g.prep = P.c->Xn;
    g.Wt = Wt; g.Wt2 = Wt2; g.M = M; g.N = N; g.K = K; g.epi = e;
    g.epi.slots = P.S;
    g.status = P.c->d_status;
    g.tnb = P.c->tile_policy[e.mode == EPI_QKV ? PSW_TILE_QKV
                             : (e.mode == EPI_RESID || e.mode == EPI_RESID_BASE) ? PSW_TILE_RESIDUAL
                             : e.mode == EPI_SWIGLU ? PSW_TILE_SWIGLU : PSW_TILE_OTHER];
    auto f8 = P.c->f8sc.find(Wt);
    if (f8 != P.c->f8sc.end()) {
        auto f82 = Wt2 ? P.c->f8sc.find(Wt2) : P.c->f8sc.end();
        g.f8 = 1; g.wsc = f8->second; g.wsc2 = f82 != P.c->f8sc.end() ? f82->second : nullptr;
    }
    if (P.rec) {
        if (!program_gemm(P.rec, g, P.tokset)) *P.failed = true;
        double nw = Wt2 ? 2.0 : 1.0;
        P.c->p_flops_tok[P.tokset] += 2.0 * nw * N * K;
        P.c->p_wbytes += nw * N * K * 2.0;
        return;
    }
    bool tc = g.f8 || gemm_tc_supported(P.c->prec, N, K, asrc);
    if (tc && !g.f8 && asrc == A_NORM && M >= WIDE_M && K <= 512) {
        // a wide launch: its token rows are normalised once (the same bf16
        // values every feature tile would build), by the residual launch
        // that last updated them or here, and streamed to the tiles
        if (!(P.xn_rows == xrows && P.xn_gain == a_gain && P.xn_m == M)) {
            LAUNCH(P, K_NORM, 0.0, (double)M * K * 6.0,
                   if (!launch_norm_rows(xrows, a_gain, M, K, P.c->Xn, P.s)) *P.failed = true);
            P.xn_rows = xrows; P.xn_gain = a_gain; P.xn_m = M;
        }
        g.asrc = asrc = A_DIRECT; g.A = P.c->Xn; g.lda = K;
    }
    if (tc && !g.f8 && asrc == A_EMBED && M >= WIDE_M && K <= 512 && e.tok) {
        // a wide latent embedding: its operand rows (the bf16 values a tile
        // would build) written once and streamed to the tiles
        GemmArgs t = g;
        t.asrc = A_DIRECT; t.A = P.c->Xn; t.lda = K;
        if (gemm_takes_ws(P.c->prec, t)) {
            LAUNCH(P, K_EMBED, 0.0, (double)M * K * 4.0,
                   if (!launch_embed_rows(P.S, e.tok, M, a_gain, K, P.c->Xn, P.s)) *P.failed = true);
            P.xn_rows = nullptr;                       // Xn holds these rows now
            g = t;
            asrc = A_DIRECT;
        }
    }
    if (g.f8 && M >= WIDE_M && K % 128 == 0 && (asrc == A_NORM ? K <= 512 : asrc == A_DIRECT ? K <= 1024 : false)) {
        // a wide E4M3 launch: its token rows are quantised once (the bytes
        // and scales an E4M3 tile would build) and streamed to the tiles
        GemmArgs t = g;
        t.asrc = A_DIRECT; t.A = P.c->Xn8; t.lda = K; t.xs = P.c->xs8;
        if (gemm_takes_ws(P.c->prec, t)) {
            if (asrc == A_NORM) {
                if (!(P.x8_rows == xrows && P.x8_gain == a_gain && P.x8_m == M)) {
                    LAUNCH(P, K_NORM, 0.0, (double)M * K * 5.0,
                           if (!launch_rows8(A_NORM, xrows, a_gain, nullptr, 0, M, K, P.c->Xn8, P.c->xs8, P.s))
                               *P.failed = true);
                    P.x8_rows = xrows; P.x8_gain = a_gain; P.x8_m = M;
                }
            } else {
                LAUNCH(P, K_NORM, 0.0, (double)M * K * 3.0,
                       if (!launch_rows8(A_DIRECT, nullptr, nullptr, A, lda, M, K, P.c->Xn8, P.c->xs8, P.s))
                           *P.failed = true);
                P.x8_rows = nullptr;
            }
            g = t;
            asrc = A_DIRECT;
        }
    }
    if (writes_rows) P.xn_rows = P.x8_rows = nullptr;  // the rows change: Xn / Xn8 no longer hold their norm
    if (!tc && asrc != A_DIRECT) P.c->launches++;      // the operand-preparation kernel
    double es = P.c->prec == P_BF16 ? 2.0 : 4.0, nw = Wt2 ? 2.0 : 1.0, wes = g.f8 ? 1.0 : es;
    double out_b = (e.mode == EPI_RESID || e.mode == EPI_RESID_BASE) ? 8.0 : es;
    Scope sc(P.c, P.s, tc ? K_GEMM_TC : K_GEMM_SIMT, 2.0 * nw * M * N * K,
             nw * N * K * wes + (double)M * K * es + (double)M * N * out_b);
    if (!gemm(P.c->prec, g, P.s)) *P.failed = true;
}

void gemm_call(const Pass &P, const void *A, int lda, const void *Wt, const void *Wt2, int M, int N, int K,
               const Epi &e)
{
    gemm_any(P, A_DIRECT, nullptr, nullptr, A, lda, Wt, Wt2, M, N, K, e);
}

// Projection of the RMSNorm (gain at gain_off) of the FP32 rows X [M][K].
void gemm_norm(const Pass &P, const float *X, long gain_off, const void *Wt, const void *Wt2, int M, int N, int K,
               const Epi &e)
{
    gemm_any(P, A_NORM, X, W(P.c, gain_off), nullptr, 0, Wt, Wt2, M, N, K, e);
}

Epi epi_qkv(const int *tok, int d, int q_cols, void *out, int kc, int vc, int layer, int ring = 0, int Tf = 1)
{
    Epi e{};
    e.mode = EPI_QKV; e.tok = tok; e.d = d; e.q_cols = q_cols; e.out = out; e.ld_out = d;
    e.kc_sel = kc; e.vc_sel = vc; e.kv_layer = layer; e.ring = ring; e.Tf = Tf; e.st_sel = CS_NONE;
    return e;
}
Epi epi_resid(const int *tok, float *rows, bool base = false)
{
    Epi e{};
    e.mode = base ? EPI_RESID_BASE : EPI_RESID; e.tok = tok; e.rows = rows; e.st_sel = CS_NONE;
    return e;
}
Epi epi_store(const int *tok, void *out, int ld, int cache = CS_NONE, int layer = 0, int d = 0)
{
    Epi e{};
    e.mode = EPI_STORE; e.tok = tok; e.out = out; e.ld_out = ld; e.st_sel = cache; e.st_layer = layer; e.d = d;
    return e;
}
Epi epi_swiglu(void *out, int ld)
{
    Epi e{};
    e.mode = EPI_SWIGLU; e.out = out; e.ld_out = ld; e.st_sel = CS_NONE;
    return e;
}
Epi epi_bias_silu(const int *tok, void *out, int ld, const float *bias)
{
    Epi e{};
    e.mode = EPI_BIAS_SILU; e.tok = tok; e.out = out; e.ld_out = ld; e.bias = bias; e.st_sel = CS_NONE;
    return e;
}
Epi epi_set_bias(const int *tok, float *rows, const float *bias)
{
    Epi e{};
    e.mode = EPI_SET_BIAS; e.tok = tok; e.rows = rows; e.bias = bias; e.st_sel = CS_NONE;
    return e;
}

double attn_flops(const psw_model_desc &m, int n, double nkeys) { return 4.0 * n * nkeys * m.d; }
// mean visible keys: about half the window under the causal masks, all of it unmasked
double attn_keys(const AttnArgs &a, int Tf)
{
    return a.kind < 0 ? (double)(a.temporal ? Tf : 1) * a.k * a.k : 0.5 * a.k * a.k;
}
double attn_bytes(const psw_model_desc &m, const AttnArgs &a)
{
    return a.n * (double)m.d * 2.0 * (2.0 * attn_keys(a, m.Tf) + 2.0);
}

AttnArgs attn_args(const Pass &P, const int *tok, int n, const void *Qp, int q_sel, int ksel, int vsel, int layer,
                   const float *bias, int bias_h_stride, int kind, int temporal)
{
    AttnArgs a{};
    const psw_model_desc &m = P.c->md;
    a.tok = tok; a.n = n; a.slots = P.S; a.Q = Qp; a.q_sel = q_sel;
    a.k_sel = ksel; a.v_sel = vsel; a.layer = layer; a.temporal = temporal; a.Tf = m.Tf;
    a.bias = bias; a.bias_h_stride = bias_h_stride;
    a.O = P.c->O; a.d = m.d; a.nh = m.nh; a.k = m.k; a.mask = m.mask; a.kind = kind;
    return a;
}

void attention(const Pass &P, const AttnArgs &a)
{
    const psw_model_desc &m = P.c->md;
    if (P.rec) {
        program_attn(P.rec, a, P.tokset);
        AttnArgs one = a;
        one.n = 1;
        P.c->p_flops_tok[P.tokset] += attn_flops(m, 1, attn_keys(a, m.Tf));
        P.c->p_bytes_tok[P.tokset] += attn_bytes(m, one);
        return;
    }
    LAUNCH(P, K_ATTN, attn_flops(m, a.n, attn_keys(a, m.Tf)), attn_bytes(m, a), launch_attention(P.c->prec, a, P.s));
}

// SwiGLU feed-forward with pre-norm and residual (Sec. 3.1).
void ffn(const Pass &P, const BlockDev &bd, long g_ffn, float *X, const int *tok, int n)
{
    psw_ctx *c = P.c;
    const psw_model_desc &m = c->md;
    Epi sw = epi_swiglu(c->Hid, m.F);
    sw.tok = tok;
    gemm_norm(P, X, g_ffn, bd.Wg, bd.Wu, n, m.F, m.d, sw);
    gemm_call(P, c->Hid, m.F, bd.Wd, nullptr, n, m.d, m.F, epi_resid(tok, X));
}

// One spatial block (Sec. 3.1: RMSNorm pre-norm, window self-attention over
// S(p), temporal cross-attention for the temporal model, SwiGLU) on the
// tokens tok[0..n).  X: their FP32 residual rows; kc/vc: this module's
// caches at layer l; bidx: the block's index in the temporal K/V ring
// (Spatial Module 1 blocks 0..L-1, Spatial Module 2 blocks L..2L-1).
void spatial_block(const Pass &P, const BlockOff &bo, const BlockDev &bd, int bidx, float *X, int kc, int vc,
                   int l, const int *tok, int n)
{
    psw_ctx *c = P.c;
    const psw_model_desc &m = c->md;
    int d = m.d, kk = m.k * m.k;
    gemm_norm(P, X, bo.g_attn, bd.Wqkv, nullptr, n, 3 * d, d, epi_qkv(tok, d, d, c->Q, kc, vc, l));
    attention(P, attn_args(P, tok, n, c->Q, CS_NONE, kc, vc, l, W(c, bo.bias), kk, 1, 0));
    gemm_call(P, c->O, d, bd.Wo, nullptr, n, d, d, epi_resid(tok, X));
    if (m.temporal) {
        gemm_norm(P, X, bo.g_x, bd.Wxq, nullptr, n, d, d, epi_store(tok, c->Q, d));
        attention(P, attn_args(P, tok, n, c->Q, CS_NONE, CS_XK, CS_XV, bidx, W(c, bo.xbias), m.Tf * kk, -1, 1));
        gemm_call(P, c->O, d, bd.Wxo, nullptr, n, d, d, epi_resid(tok, X));
    }
    ffn(P, bd, bo.g_ffn, X, tok, n);
}

// Hyperprior synthesis (Fig. 1 right, RB-up blocks): gamma_z * z-hat of
// the slot of tok[0] through the sub-pixel residual blocks; the last grid
// cropped into the slot's hyperprior tokens.  Per block, one projection
// computes the first convolution and the skip convolution of the same
// taps (stacked, biases ba and bs + bb); the skip half is shuffled into the
// output grid, the first half is the LeakyReLU'd, shuffled input of the
// second convolution, whose result is added.
void hyper_synthesis(const Pass &P, const int *tok, int H, int W_)
{
    psw_ctx *c = P.c;
    const psw_model_desc &m = c->md;
    const int nb = hyper_blocks(m), Ch = m.Ch, d = m.d;
    int h = (H + m.r - 1) / m.r, w = (W_ + m.r - 1) / m.r;
    float *x = c->hg[0], *U = c->hg[1], *o = c->hg[2];
    P.xn_rows = P.x8_rows = nullptr;
    LAUNCH(P, K_EMBED, 0.0, (double)h * w * Ch * 6.0,
           launch_zhat_grid(P.S, tok, h * w, W(c, c->lay.gamma_z), Ch, x, P.s));
    for (int b = 0; b < nb; b++) {
        const int Co = b == nb - 1 ? d : Ch, Pn = h * w;
        LAUNCH(P, K_EMBED, 0.0, (double)Pn * 9 * Ch * 6.0,
               launch_im2col(c->prec, x, h, w, Ch, 0, 0, 0, 3, 1, c->hcol, P.s));
        gemm_call(P, c->hcol, 9 * Ch, c->hu_w[b], nullptr, Pn, 8 * Co, 9 * Ch, epi_set_bias(nullptr, U, c->hu_bias[b]));
        LAUNCH(P, K_EMBED, 0.0, (double)Pn * 4 * Co * 8.0, launch_shuffle(U + 4 * Co, h, w, Co, 8 * Co, o, P.s));
        LAUNCH(P, K_EMBED, 0.0, (double)Pn * 4 * 9 * Co * 6.0,
               launch_im2col(c->prec, U, 2 * h, 2 * w, Co, 1, 8 * Co, 1, 3, 1, c->hcol, P.s));
        gemm_call(P, c->hcol, 9 * Co, c->hu_wb[b], nullptr, 4 * Pn, Co, 9 * Co, epi_resid(nullptr, o));
        h *= 2; w *= 2;
        float *t = x; x = o; o = U; U = t;               // the output is the next block's input
    }
    LAUNCH(P, K_EMBED, 0.0, (double)H * W_ * d * 8.0, launch_crop_eh(P.S, tok, x, w, H, W_, d, P.s));
}

// Hyperprior analysis (RB-down blocks) of the H x W frame whose Spatial
// Module 1 rows are in Xa (raster order): RMSNorm(x1) * g_za, per block the
// strided 3 x 3 convolution and LeakyReLU, the 3 x 3 convolution added to
// the strided 1 x 1 skip (biases bs + bb merged); z rounded into zhat.
void hyper_analysis(const Pass &P, int H, int W_, int16_t *zhat, float *z_out)
{
    psw_ctx *c = P.c;
    const psw_model_desc &m = c->md;
    const int nb = hyper_blocks(m), Ch = m.Ch, d = m.d;
    float *x = c->hg[0], *A = c->hg[1], *o = c->hg[2];
    LAUNCH(P, K_NORM, 0.0, (double)H * W_ * d * 8.0, launch_rmsnorm(P_F32, c->Xa, H * W_, W(c, c->lay.g_za), d, x, P.s));
    int h = H, w = W_, Ci = d;
    for (int b = 0; b < nb; b++) {
        const int ho = (h + 1) / 2, wo = (w + 1) / 2, Pn = ho * wo;
        LAUNCH(P, K_EMBED, 0.0, (double)Pn * 9 * Ci * 6.0,
               launch_im2col(c->prec, x, h, w, Ci, 0, 0, 0, 3, 2, c->hcol, P.s));
        gemm_call(P, c->hcol, 9 * Ci, c->hd_wa[b], nullptr, Pn, Ch, 9 * Ci,
                  epi_set_bias(nullptr, A, W(c, c->lay.rbd[b].ba)));
        LAUNCH(P, K_EMBED, 0.0, (double)Pn * Ci * 6.0, launch_im2col(c->prec, x, h, w, Ci, 0, 0, 0, 1, 2, c->hcol, P.s));
        gemm_call(P, c->hcol, Ci, c->hd_ws[b], nullptr, Pn, Ch, Ci, epi_set_bias(nullptr, o, c->hd_bias[b]));
        LAUNCH(P, K_EMBED, 0.0, (double)Pn * 9 * Ch * 6.0,
               launch_im2col(c->prec, A, ho, wo, Ch, 0, 0, 1, 3, 1, c->hcol, P.s));
        gemm_call(P, c->hcol, 9 * Ch, c->hd_wb[b], nullptr, Pn, Ch, 9 * Ch, epi_resid(nullptr, o));
        h = ho; w = wo; Ci = Ch;
        float *t = x; x = o; o = A; A = t;
    }
    LAUNCH(P, K_OTHER, 0.0, (double)h * w * Ch * 6.0, launch_round_z(x, (long)h * w * Ch, zhat, z_out, P.s));
}

void frame_context(const Pass &P, const int *tok, int n);

// Positions of the frame of slot `slot` (H x W, hyperprior r times coarser)
// grouped by sub-pixel tap t = (i mod r) r + (j mod r), raster order within
// a tap, appended to the segment of each tap.
void tap_tokens(int slot, int H, int W_, int r, std::vector<std::vector<int>> &seg)
{
    seg.resize((size_t)r * r);
    for (int i = 0; i < H; i++)
        for (int j = 0; j < W_; j++) seg[(size_t)(i % r) * r + j % r].push_back(tok_make(slot, i * W_ + j));
}

// The hyperprior tokens on the tensor cores (Sec. 3.1: the embedded
// hyperprior; Fig. 1 right): for each tap t, the positions tok[off[t] ..
// + n[t]) of every frame, eh[p] = W_hp[t]^T (gamma_z * z-hat of p's
// hyperlatent) + b_hp -- the sub-pixel embedding launch_embed_hyper
// computes on the CUDA cores, as one projection per tap.
void hyper_embed_tc(const Pass &P, const int *tok, const std::vector<int> &off, const std::vector<int> &n)
{
    psw_ctx *c = P.c;
    const psw_model_desc &m = c->md;
    for (size_t t = 0; t < c->Whp_t.size(); t++) {
        Epi e = epi_set_bias(tok + off[t], nullptr, W(c, c->lay.b_hp));
        e.eh_out = 1; e.hr = m.r;
        gemm_any(P, A_ZHAT, nullptr, W(c, c->lay.gamma_z), nullptr, 0, c->Whp_t[t], nullptr, n[t], m.d, m.Ch, e);
    }
}

// Per-frame preparation for the tokens tok[0..n) (all positions of one
// slot, in raster order; eh: that slot's hyperprior rows): hyperprior
// tokens and accumulator queries (they depend only on the hyperlatents,
// Sec. 3.1), and for the temporal model this frame's Context Transformer
// pass and every spatial block's cross-attention K/V.
void frame_prologue(const Pass &P, const int *tok, int H, int W_, const float *eh, bool embed = true,
                    bool context = true)
{
    const int n = H * W_;
    psw_ctx *c = P.c;
    const psw_model_desc &m = c->md;
    int d = m.d, kk = m.k * m.k;
    P.xn_rows = P.x8_rows = nullptr;                   // rows written outside gemm_any follow
    if (m.hp) {
        hyper_synthesis(P, tok, H, W_);
    } else if (embed && c->Whp_t.empty()) {
        LAUNCH(P, K_EMBED, 2.0 * n * m.Ch * d, n * (m.Ch * 2.0 + d * 4.0),
               launch_embed_hyper(P.S, tok, n, H, W_, m.Ch, m.r, W(c, c->lay.gamma_z), W(c, c->lay.W_hp),
                                  W(c, c->lay.b_hp), d, P.s));
    }
    gemm_norm(P, eh, c->lay.acc_g_q, c->acc.Wqkv, nullptr, n, d, d, epi_store(tok, nullptr, d, CS_QA, 0, d));
    if (!m.temporal || !context) return;
    frame_context(P, tok, n);
}

// Rows of one batched Context Transformer pass at most (the workspace grows
// to the pass's rows: ~9 KB per row at d = 384).
constexpr int CTX_ROWS_MAX = 262144;

// Frames b0 .. b1 - 1 of a decode plan whose prologue tokens are
// consecutive; groups of whole frames of at most CTX_ROWS_MAX rows (one
// frame alone if larger).
template <typename F>
void ctx_groups(const std::vector<int> &pro_n, F fn)
{
    int b0 = 0, rows = 0;
    for (int b = 0; b < (int)pro_n.size(); b++) {
        if (b > b0 && rows + pro_n[b] > CTX_ROWS_MAX) {
            fn(b0, b, rows);
            b0 = b; rows = 0;
        }
        rows += pro_n[b];
    }
    if (b0 < (int)pro_n.size()) fn(b0, (int)pro_n.size(), rows);
}

// The temporal model's per-frame context: the Context Transformer pass and
// every spatial block's cross-attention keys and values (Sec. 3.1).
void frame_context(const Pass &P, const int *tok, int n)
{
    psw_ctx *c = P.c;
    const psw_model_desc &m = c->md;
    int d = m.d, kk = m.k * m.k;
    // Context Transformer (Sec. 3.1): temporally shifted latents (learned
    // padding vector for frame 0), time-causal window attention over the
    // frames of the ring at each layer, final RMSNorm.
    LAUNCH(P, K_EMBED, 2.0 * n * m.C * d, n * (m.C * 2.0 + d * 4.0),
           launch_embed_context(P.S, tok, n, m.C, W(c, c->lay.gamma_c), W(c, c->lay.W_c), W(c, c->lay.b_c),
                                W(c, c->lay.pad), d, c->Xg, P.s));
    P.xn_rows = P.x8_rows = nullptr;
    for (int l = 0; l < m.Lc; l++) {
        const BlockOff &bo = c->lay.ctx[l];
        const BlockDev &bd = c->ctxb[l];
        gemm_norm(P, c->Xg, bo.g_attn, bd.Wqkv, nullptr, n, 3 * d, d, epi_qkv(tok, d, d, c->Q, CS_CK, CS_CV, l, 1, m.Tf));
        attention(P, attn_args(P, tok, n, c->Q, CS_NONE, CS_CK, CS_CV, l, W(c, bo.bias), m.Tf * kk, -1, 1));
        gemm_call(P, c->O, d, bd.Wo, nullptr, n, d, d, epi_resid(tok, c->Xg));
        ffn(P, bd, bo.g_ffn, c->Xg, tok, n);
    }
    for (int b = 0; b < 2 * m.L; b++) {
        const BlockDev &bd = b < m.L ? c->sm1[b] : c->sm2[b - m.L];
        gemm_norm(P, c->Xg, c->lay.g_ctx, bd.Wxkv, nullptr, n, 2 * d, d,
                  epi_qkv(tok, d, 0, nullptr, CS_XK, CS_XV, b, 1, m.Tf));
    }
}

// Spatial Module 1 on tokens whose latents are known, then the accumulator
// keys/values from its normalised output (Sec. 3.1).
void run_sm1(const Pass &P, const int *tok, int n)
{
    psw_ctx *c = P.c;
    const psw_model_desc &m = c->md;
    int d = m.d;
    if (n <= 0) return;
    gemm_any(P, A_EMBED, nullptr, W(c, c->lay.gamma_in), nullptr, 0, c->Win, nullptr, n, d, m.C,
             epi_set_bias(tok, c->Xa, W(c, c->lay.b_in)));
    for (int l = 0; l < m.L; l++) spatial_block(P, c->lay.sm1[l], c->sm1[l], l, c->Xa, CS_K1, CS_V1, l, tok, n);
    gemm_norm(P, c->Xa, c->lay.acc_g_kv, c->acc.Wxkv, nullptr, n, 2 * d, d, epi_qkv(tok, d, 0, nullptr, CS_KA, CS_VA, 0));
}

// Accumulator (hyperprior query and residual, keys/values over A(p)),
// Spatial Module 2 and heads on tokens tok[0..n) (Sec. 3.1, Fig. 2b).
void run_acc_sm2_heads(const Pass &P, const int *tok, int n)
{
    psw_ctx *c = P.c;
    const psw_model_desc &m = c->md;
    int d = m.d;
    if (n <= 0) return;
    attention(P, attn_args(P, tok, n, nullptr, CS_QA, CS_KA, CS_VA, 0, W(c, c->lay.acc_bias), m.k * m.k, 0, 0));
    gemm_call(P, c->O, d, c->acc.Wo, nullptr, n, d, d, epi_resid(tok, c->Xb, true));
    ffn(P, c->acc, c->lay.acc_g_ffn, c->Xb, tok, n);
    for (int l = 0; l < m.L; l++)
        spatial_block(P, c->lay.sm2[l], c->sm2[l], m.L + l, c->Xb, CS_K2, CS_V2, l, tok, n);
    if (m.Nc) return;                  // the Channel Transformer's groups follow (run_ct_group)
    if (m.Llrp) {
        // the final representation at these positions, kept for the LRP
        // Transformer (the persistent decoder has no phase for it)
        if (P.rec) *P.failed = true;
        else LAUNCH(P, K_OTHER, 0.0, (double)n * d * 8.0, launch_store_rows(P.S, tok, n, c->Xb, d, d, 0, P.s));
    }
    // prediction heads (Sec. 3.1): RMSNorm, both first layers as one
    // projection with bias and SiLU, then both second layers as one
    // interleaved projection whose epilogue applies the channel-wise output
    // scaling, sigma's exp and clamp, and the quantisation
    gemm_norm(P, c->Xb, c->lay.g_head, c->Wh1, nullptr, n, 2 * d, d, epi_bias_silu(tok, c->Hid, 2 * d, c->bh1));
    Epi eh{};
    eh.mode = EPI_HEADS; eh.tok = tok; eh.st_sel = CS_NONE; eh.C = m.C; eh.scale = c->d_scale;
    eh.gmu = W(c, c->lay.gamma_mu); eh.bmu = W(c, c->lay.beta_mu);
    eh.gsg = W(c, c->lay.gamma_sig); eh.bsg = W(c, c->lay.beta_sig);
    gemm_call(P, c->Hid, 2 * d, c->Wh2, nullptr, n, 2 * m.C, 2 * d, eh);
}

// Channel Transformer and grouped heads of channel group g (Sec. 3.1
// Channel Transformer paragraph; Sec. 3.2: N channel groups after the s
// spatial steps) on the tokens tok[0..n), whose Spatial Module 2 rows are in
// Xb.  The group's FP32 rows (its own block of Xc) start as the normalised
// Spatial Module 2 rows projected to the group plus, with the channel shift,
// the embedding of group g - 1's latents; each block writes the group's
// normalised rows into the block's mixing input NM (groups 0..g-1 were
// written by the earlier sub-steps on the same tokens), adds the masked
// mixing of input groups 0..g, then the group's SwiGLU; the grouped heads
// write the parameters of the group's channels.  Every launch is per token,
// so encoder and decoder (and any batch) compute the same bits.
void run_ct_group(const Pass &P, const int *tok, int n, int g)
{
    psw_ctx *c = P.c;
    const psw_model_desc &m = c->md;
    const Layout &y = c->lay;
    if (n <= 0) return;
    const int G = m.Nc, dc = m.dc, dg = dc / G, Cg = m.C / G, d = m.d;
    const size_t es = esize(c->prec);
    float *Xg = c->Xc + (size_t)g * c->ws_rows * dg;
    gemm_norm(P, c->Xb, y.ct_g_in, c->ct_win[g], nullptr, n, dg, d, epi_set_bias(tok, Xg, W(c, y.ct_b_in) + g * dg));
    if (g > 0) {
        P.xn_rows = P.x8_rows = nullptr;               // rows written outside gemm_any
        LAUNCH(P, K_EMBED, 2.0 * n * Cg * dg, n * (Cg * 2.0 + dg * 8.0),
               launch_ct_embed(P.S, tok, n, m.C, (g - 1) * Cg, Cg, W(c, y.ct_gamma_y) + (g - 1) * Cg,
                               W(c, y.ct_E) + (long)(g - 1) * Cg * dg, dg, Xg, P.s));
    }
    for (int l = 0; l < m.Lct; l++) {
        const int bi = l * G + g;
        char *nm = (char *)c->NM + (size_t)l * c->ws_rows * dc * es;
        const float *gm = W(c, y.ct_g_mix[l]) + g * dg;
        if (c->prec == P_BF16) {
            LAUNCH(P, K_NORM, 0.0, (double)n * dg * 6.0,
                   if (!launch_norm_rows(Xg, gm, n, dg, nm + (size_t)g * dg * es, P.s, dc)) *P.failed = true);
        } else {
            LAUNCH(P, K_NORM, 0.0, (double)n * dg * 8.0,
                   launch_rmsnorm(c->prec, Xg, n, gm, dg, nm + (size_t)g * dg * es, P.s, dc));
        }
        gemm_call(P, nm, dc, c->ct_mix[bi], nullptr, n, dg, (g + 1) * dg, epi_resid(tok, Xg));
        Epi sw = epi_swiglu(c->Hid, m.Fc);
        sw.tok = tok;
        gemm_norm(P, Xg, y.ct_g_ffn[l] + g * dg, c->ct_wg[bi], c->ct_wu[bi], n, m.Fc, dg, sw);
        gemm_call(P, c->Hid, m.Fc, c->ct_wd[bi], nullptr, n, dg, m.Fc, epi_resid(tok, Xg));
    }
    if (m.Llrp) LAUNCH(P, K_OTHER, 0.0, (double)n * dg * 8.0, launch_store_rows(P.S, tok, n, Xg, dg, dc, g * dg, P.s));
    gemm_norm(P, Xg, y.g_head + g * dg, c->ct_wh1[g], nullptr, n, 2 * dg, dg,
              epi_bias_silu(tok, c->Hid, 2 * dg, c->ct_bh1[g]));
    Epi eh{};
    eh.mode = EPI_HEADS; eh.tok = tok; eh.st_sel = CS_NONE; eh.C = m.C; eh.c0 = g * Cg; eh.scale = c->d_scale;
    eh.gmu = W(c, y.gamma_mu) + g * Cg; eh.bmu = W(c, y.beta_mu) + g * Cg;
    eh.gsg = W(c, y.gamma_sig) + g * Cg; eh.bsg = W(c, y.beta_sig) + g * Cg;
    gemm_call(P, c->Hid, 2 * dg, c->ct_wh2[g], nullptr, n, 2 * Cg, 2 * dg, eh);
}

// LRP Transformer over every position of one coded frame (Sec. 3.1 latent
// residual prediction; tokens tok[0..n) in raster order, so the slot's rep
// rows are the compact rows of the launch): the input token from the
// channel-scaled latents and the normalised representation, Llrp blocks of
// window self-attention without prediction mask (for the temporal model over
// the ring of the last Tf frames' keys and values of the same block) and
// SwiGLU, then eps = RMSNorm . W_eps + b_eps into eps [n][C] (skipped if eps
// is null).
void run_lrp(const Pass &P, const int *tok, int n, const float *rep, float *eps)
{
    psw_ctx *c = P.c;
    const psw_model_desc &m = c->md;
    const Layout &y = c->lay;
    int d = m.d, kk = m.k * m.k, tmp = m.temporal != 0;
    P.xn_rows = P.x8_rows = nullptr;
    gemm_any(P, A_EMBED, nullptr, W(c, y.lrp_gamma_y), nullptr, 0, c->Wy, nullptr, n, d, m.C,
             epi_set_bias(tok, c->Xa, W(c, y.lrp_b_in)));
    gemm_norm(P, rep, y.lrp_g_rep, c->Wrep, nullptr, n, d, m.Nc ? m.dc : d, epi_resid(tok, c->Xa));
    for (int l = 0; l < m.Llrp; l++) {
        const BlockOff &bo = y.lrp[l];
        const BlockDev &bd = c->lrpb[l];
        gemm_norm(P, c->Xa, bo.g_attn, bd.Wqkv, nullptr, n, 3 * d, d,
                  epi_qkv(tok, d, d, c->Q, CS_LK, CS_LV, l, tmp, m.Tf));
        attention(P, attn_args(P, tok, n, c->Q, CS_NONE, CS_LK, CS_LV, l, W(c, bo.bias), (tmp ? m.Tf : 1) * kk, -1,
                               tmp));
        gemm_call(P, c->O, d, bd.Wo, nullptr, n, d, d, epi_resid(tok, c->Xa));
        ffn(P, bd, bo.g_ffn, c->Xa, tok, n);
    }
    if (eps) gemm_norm(P, c->Xa, y.lrp_g_out, c->Weps, nullptr, n, m.C, d, epi_set_bias(tok, eps, W(c, y.lrp_b_eps)));
}

// The persistent decoder's program for the current workspace: the phases
// of one step, recorded from the same pass functions the graph path
// launches (so both run identical tiles).  Built once per workspace
// generation; false if the context cannot run it.
bool ensure_program(psw_ctx *c)
{
    if (c->prog_gen == c->ws_gen) return c->prog_ok;
    program_free(c->prog);
    c->prog = nullptr;
    c->prog_ok = false;
    c->prog_gen = c->ws_gen;
    if (c->prec != P_BF16 || c->ws_rows == 0 || c->md.Llrp || c->md.Nc) return false;
    c->prog = program_new((int)c->ws_rows);
    c->p_flops_tok[0] = c->p_flops_tok[1] = c->p_bytes_tok[0] = c->p_bytes_tok[1] = c->p_wbytes = 0;
    bool failed = false;
    Pass P{c, nullptr, c->d_slots, &failed};
    P.rec = c->prog;
    P.tokset = TS_PREV;
    run_sm1(P, nullptr, 1);
    P.tokset = TS_CUR;
    run_acc_sm2_heads(P, nullptr, 1);
    program_rans(c->prog);
    if (failed) return false;
    if (!program_upload(c->prog, &c->p_ops, &c->p_nops, &c->p_maps, &c->p_nmaps, &c->p_smem, &c->p_f8))
        return false;
    if (!persist_prepare(c->p_smem, c->p_f8, &c->p_grid)) return false;
    if (!c->d_pbar && cudaMalloc(&c->d_pbar, 2 * sizeof(unsigned)) != cudaSuccess) return false;
    c->prog_ok = true;
    return true;
}

CoderDev coder(const psw_ctx *c) { return CoderDev{c->d_cdf, c->d_meta}; }

psw_status check_frame(psw_ctx *c, psw_seq *q, const psw_frame_desc *fd)
{
    if (!c || !q || q->ctx != c) return fail(c, PSW_ERR_INVALID, "context/sequence mismatch");
    if (!fd) return fail(c, PSW_ERR_INVALID, "null frame descriptor");
    if (fd->H < 1 || fd->W < 1 || fd->H > q->maxH || fd->W > q->maxW)
        return fail(c, PSW_ERR_INVALID, "frame %dx%d outside the sequence maximum %dx%d", fd->H, fd->W, q->maxH, q->maxW);
    if (fd->schedule != PSW_SCHED_WAVEFRONT && fd->schedule != PSW_SCHED_RASTER)
        return fail(c, PSW_ERR_INVALID, "unknown schedule %d", fd->schedule);
    if (fd->schedule == PSW_SCHED_RASTER && c->md.mask == 1)
        return fail(c, PSW_ERR_INVALID, "raster order is not a valid schedule for the cyclic mask");
    return PSW_OK;
}

size_t seq_bytes_for(const psw_model_desc &m, int prec, int H, int W_)
{
    size_t HW = (size_t)H * W_, d = m.d, es = esize(prec);
    size_t b = 0;
    b += HW * d * 4;                                                // eh
    b += HW * d * es;                                               // qa
    b += (4 * (size_t)m.L + 2) * HW * d * es;                       // K1 V1 K2 V2 Ka Va
    if (m.temporal) b += 2 * ((size_t)m.Lc + 2 * (size_t)m.L) * m.Tf * HW * d * es;
    b += HW * m.C * (4 + 4 + 1 + 4 + 2 + 2);                        // mu sigma idx m y yprev
    b += (size_t)m.C * 32 * 4 + 2 * (size_t)m.C * 4 + (2 * (size_t)m.C + 1) * 4;
    b += (size_t)m.C * (3 * HW + 64) * 2;                           // encoder scratch
    b += HW * 4 + 64;
    if (m.Llrp) b += HW * (m.Nc ? m.dc : d) * 4 + 2 * (size_t)m.Llrp * (m.temporal ? m.Tf : 1) * HW * d * es;   // rep, LK, LV
    return b;
}

// Upload the slot table (n entries) and reset the status words.
psw_status upload_slots(psw_ctx *c, const std::vector<psw_seq *> &qs, int n, cudaStream_t s)
{
    CK_CUDA(c, cudaMemcpyAsync(c->d_slots, c->h_slots, sizeof(Slot) * n, cudaMemcpyHostToDevice, s));
    CK_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
    for (psw_seq *q : qs) CK_CUDA(c, cudaMemsetAsync(q->d_status, 0, sizeof(int), s));
    return PSW_OK;
}

// Read the status words back (context word OR-ed into each sequence's).
psw_status read_status(psw_ctx *c, const std::vector<psw_seq *> &qs, cudaStream_t s, std::vector<int> &out)
{
    CK_CUDA(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    for (size_t b = 0; b < qs.size(); b++)
        CK_CUDA(c, cudaMemcpyAsync(c->h_status + 1 + b, qs[b]->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK_CUDA(c, cudaStreamSynchronize(s));
    out.assign(qs.size(), 0);
    for (size_t b = 0; b < qs.size(); b++) out[b] = c->h_status[1 + b] | c->h_status[0];
    return PSW_OK;
}

psw_status status_code(psw_ctx *c, int st)
{
    if (st & ST_CORRUPT) return fail(c, PSW_ERR_CORRUPT, "bitstream failed validation");
    if (st & ST_TIMEOUT) return fail(c, PSW_ERR_TIMEOUT, "a bounded device wait timed out");
    if (st & ST_CAPACITY) return fail(c, PSW_ERR_CAPACITY, "container larger than its buffer");
    return PSW_OK;
}

psw_status grow_tokens(psw_ctx *c, size_t ntok, size_t nkn)
{
    if (ntok > c->tok_cap) {
        CK_CUDA(c, cudaDeviceSynchronize());
        cudaFree(c->d_tok);
        c->d_tok = nullptr; c->tok_cap = 0;
        CK_CUDA(c, cudaMalloc(&c->d_tok, ntok * sizeof(int)));
        c->tok_cap = ntok;
    }
    if (nkn > c->kn_cap) {
        CK_CUDA(c, cudaDeviceSynchronize());
        cudaFree(c->d_kn);
        c->d_kn = nullptr; c->kn_cap = 0;
        CK_CUDA(c, cudaMalloc(&c->d_kn, nkn * sizeof(int2)));
        c->kn_cap = nkn;
    }
    return PSW_OK;
}

// Token lists of a batched decode.  Layout of tok: for each slot its HW
// prologue tokens, then for each global step t the tokens of step t of every
// slot (slot-major); kn[t][b] = (first symbol, count) of slot b at step t.
struct DecodePlan {
    int n = 0, Tmax = 0;
    std::vector<const float *> eh;      // each slot's hyperprior rows
    std::vector<int> tok, pro_off, pro_n, pro_h, pro_w, step_off, step_n;
    std::vector<int> tap_off, tap_n;    // tensor-core hyperprior embedding: each tap's positions of every frame
    std::vector<int2> kn;
    size_t max_step = 0;
};

DecodePlan plan_decode(const std::vector<psw_seq *> &qs, const psw_frame_desc *fds, int r_taps)
{
    DecodePlan D;
    D.n = (int)qs.size();
    for (int b = 0; b < D.n; b++) {
        D.pro_off.push_back((int)D.tok.size());
        D.eh.push_back(qs[b]->eh);
        int HW = fds[b].H * fds[b].W;
        D.pro_n.push_back(HW);
        D.pro_h.push_back(fds[b].H);
        D.pro_w.push_back(fds[b].W);
        for (int p = 0; p < HW; p++) D.tok.push_back(tok_make(b, p));
        D.Tmax = std::max(D.Tmax, qs[b]->T);
    }
    if (r_taps > 0) {
        std::vector<std::vector<int>> seg;
        for (int b = 0; b < D.n; b++) tap_tokens(b, fds[b].H, fds[b].W, r_taps, seg);
        for (auto &v : seg) {
            D.tap_off.push_back((int)D.tok.size());
            D.tap_n.push_back((int)v.size());
            D.tok.insert(D.tok.end(), v.begin(), v.end());
        }
    }
    D.kn.assign((size_t)D.Tmax * D.n, make_int2(0, 0));
    for (int t = 0; t < D.Tmax; t++) {
        D.step_off.push_back((int)D.tok.size());
        for (int b = 0; b < D.n; b++) {
            const psw_seq *q = qs[b];
            if (t >= q->T) continue;
            int a0 = q->h_start[t], a1 = q->h_start[t + 1];
            D.kn[(size_t)t * D.n + b] = make_int2(a0, a1 - a0);
            for (int a = a0; a < a1; a++) D.tok.push_back(tok_make(b, q->h_order[a]));
        }
        D.step_n.push_back((int)D.tok.size() - D.step_off.back());
        D.max_step = std::max(D.max_step, (size_t)D.step_n.back());
    }
    return D;
}

// Enqueue global steps [t0, t1) of a planned decode; the first segment also
// runs the prologues and coder initialisation, the last the coder check.
void enqueue_decode(psw_ctx *c, const DecodePlan &D, const int *d_tok, const int2 *d_kn, cudaStream_t s, bool *failed,
                    int t0, int t1)
{
    Pass P{c, s, c->d_slots, failed};
    if (t0 == 0) {
        // the hyperprior tokens of every frame: per tap on the tensor cores,
        // else in one CUDA-core launch (the convolutional hyperprior's
        // synthesis stays per frame)
        const bool batch_embed = !c->md.hp && D.n > 1 && c->Whp_t.empty();
        if (!c->Whp_t.empty() && !c->md.hp) hyper_embed_tc(P, d_tok, D.tap_off, D.tap_n);
        if (batch_embed) {
            const int Hm = *std::max_element(D.pro_h.begin(), D.pro_h.end());
            const int Wm = *std::max_element(D.pro_w.begin(), D.pro_w.end());
            double npos = 0.0;
            for (int b = 0; b < D.n; b++) npos += D.pro_n[b];
            LAUNCH(P, K_EMBED, 2.0 * npos * c->md.Ch * c->md.d, npos * (c->md.Ch * 2.0 + c->md.d * 4.0),
                   launch_embed_hyper_batch(P.S, D.n, Hm, Wm, c->md.Ch, c->md.r, W(c, c->lay.gamma_z),
                                            W(c, c->lay.W_hp), W(c, c->lay.b_hp), c->md.d, P.s));
        }
        for (int b = 0; b < D.n; b++)
            frame_prologue(P, d_tok + D.pro_off[b], D.pro_h[b], D.pro_w[b], D.eh[b], !batch_embed, false);
        // the temporal model's Context Transformer over the positions of
        // groups of frames together (every launch is per token)
        if (c->md.temporal)
            ctx_groups(D.pro_n, [&](int b0, int, int rows) { frame_context(P, d_tok + D.pro_off[b0], rows); });
        Scope sc(c, s, K_RANS, 0.0, (double)D.n * c->md.C * 128.0);
        launch_rans_dec_init(c->d_slots, D.n, c->md.C, s);
    }
    for (int t = t0; t < t1; t++) {
        if (t > 0) run_sm1(P, d_tok + D.step_off[t - 1], D.step_n[t - 1]);
        run_acc_sm2_heads(P, d_tok + D.step_off[t], D.step_n[t]);
        const int G = std::max(c->md.Nc, 1), Cg = c->md.C / G;
        for (int g = 0; g < G; g++) {
            // with a Channel Transformer, group g's parameters, then its symbols
            if (c->md.Nc) run_ct_group(P, d_tok + D.step_off[t], D.step_n[t], g);
            Scope sc(c, s, K_RANS, 0.0, (double)D.step_n[t] * Cg * 9.0);
            launch_rans_dec_step(coder(c), c->d_slots, D.n, d_kn + (size_t)t * D.n, c->md.C, s, g * Cg, Cg);
        }
    }
    if (t1 == D.Tmax) {
        Scope sc(c, s, K_RANS, 0.0, (double)D.n * c->md.C * 128.0);
        launch_rans_dec_finish(c->d_slots, D.n, c->md.C, s);
    }
}

// Steps [0, Tmax) of a planned decode on the persistent decoder, then the
// coder's final check.  ntok / ntok_prev: tokens over all steps, and those
// that also pass Spatial Module 1 (the algorithmic FLOPs of the launch).
psw_status persist_run(psw_ctx *c, const int *d_tok, const int *d_step, const int2 *d_kn, int n, int Tmax,
                       double ntok, double ntok_prev, cudaStream_t s)
{
    CK_CUDA(c, cudaMemsetAsync(c->d_pbar, 0, 2 * sizeof(unsigned), s));
    PersistArgs pa{};
    pa.ops = c->p_ops; pa.nops = c->p_nops; pa.maps = c->p_maps; pa.nmaps = c->p_nmaps;
    pa.tok = d_tok; pa.step_off = d_step; pa.step_n = d_step + Tmax;
    pa.kn = d_kn; pa.nslots = n;
    pa.cd = coder(c); pa.slots = c->d_slots; pa.C = c->md.C;
    pa.t0 = 0; pa.t1 = Tmax;
    pa.bar = c->d_pbar; pa.abort_g = (int *)(c->d_pbar + 1); pa.status = c->d_status;
    double flops = c->p_flops_tok[TS_CUR] * ntok + c->p_flops_tok[TS_PREV] * ntok_prev;
    double bytes = c->p_wbytes * Tmax + c->p_bytes_tok[TS_CUR] * ntok + c->p_bytes_tok[TS_PREV] * ntok_prev;
    {
        Scope sc(c, s, K_PERSIST, flops, bytes);
        if (!persist_launch(pa, c->p_grid, c->p_smem, c->p_f8, s))
            return fail(c, PSW_ERR_CUDA, "persistent decoder launch: %s", cudaGetErrorString(cudaGetLastError()));
    }
    Scope sc(c, s, K_RANS, 0.0, (double)n * c->md.C * 128.0);
    launch_rans_dec_finish(c->d_slots, n, c->md.C, s);
    return PSW_OK;
}

// Decode n frames of n sequences together (the engine behind
// psw_decode_frame and psw_decode_batch).
psw_status decode_run(psw_ctx *c, int n, psw_seq *const *seqs, const psw_frame_desc *fds,
                      const uint8_t *const *bs, const size_t *lens, const int16_t *const *zhat,
                      int16_t *const *yout, float *const *mu_out, float *const *sg_out, int *status_out,
                      cudaStream_t s)
{
    if (n < 1 || n > MAX_SLOTS) return fail(c, PSW_ERR_INVALID, "batch of %d frames (1..%d)", n, MAX_SLOTS);
    std::vector<psw_seq *> qs(seqs, seqs + n);
    for (int b = 0; b < n; b++) {
        psw_status st = check_frame(c, qs[b], &fds[b]);
        if (st) return st;
        for (int a = 0; a < b; a++)
            if (qs[a] == qs[b]) return fail(c, PSW_ERR_INVALID, "a sequence appears twice in one batch");
        if (!bs[b] || !zhat[b] || !yout[b]) return fail(c, PSW_ERR_INVALID, "null pointer for frame %d", b);
        if ((uintptr_t)bs[b] & 3) return fail(c, PSW_ERR_INVALID, "bitstream %d must be 4-byte aligned", b);
        if ((st = seq_schedule(qs[b], fds[b].H, fds[b].W, fds[b].schedule))) return st;
    }
    for (int b = 0; b < n; b++) {
        Slot sl = make_slot(qs[b], fds[b].H, fds[b].W, fds[b].schedule);
        sl.bs = bs[b]; sl.len = lens[b]; sl.zhat = zhat[b];
        sl.status = c->d_bstatus + b;                  // the call's status words sit together
        c->h_slots[b] = sl;
    }
    // graph key: the workspace generation, the engine and the batch shape
    bool failed = false;
    // the persistent engine records no graphs: a call plans its token lists,
    // launches the per-frame prologues and one cooperative kernel, so batches
    // that change from call to call (a serving loop) cost no graph recording
    bool want = c->engine == PSW_ENGINE_PERSISTENT && c->prec == P_BF16;
    bool graph = c->use_graphs && !c->prof && !want;
    std::vector<long> key{0, (long)n, (long)want};
    static_assert(KEY_SEQ0 == 3, "key layout");
    for (int b = 0; b < n; b++) {
        key.push_back((long)(uintptr_t)qs[b]);
        key.push_back(((long)fds[b].H << 32) | ((long)fds[b].W << 2) | fds[b].schedule);
    }
    GraphRec *gr = nullptr;
    key[0] = c->ws_gen;
    if (graph) {
        auto it = c->graphs.find(key);
        if (it != c->graphs.end()) {
            gr = &it->second;
            gr->used = ++c->graph_clock;
        }
    }
    DecodePlan D;
    psw_status st;
    if (!gr) {
        D = plan_decode(qs, fds, c->Whp_t.empty() ? 0 : c->md.r);
        size_t rows = D.max_step;
        for (int b = 0; b < n; b++) rows = std::max(rows, (size_t)D.pro_n[b]);
        if (c->md.temporal) ctx_groups(D.pro_n, [&](int, int, int r) { rows = std::max(rows, (size_t)r); });
        if ((st = ensure_workspace(c, rows))) return st;
        key[0] = c->ws_gen;
    }
    bool persist = want && ensure_program(c);
    if (want && !persist && c->engine == PSW_ENGINE_PERSISTENT)
        return fail(c, PSW_ERR_CUDA, "the persistent decoder could not be set up for this context");
    // persistent decoder: per-step token offsets and counts, token totals
    std::vector<int> steps;
    double ntok = 0, ntok_prev = 0;
    if (!gr && persist) {
        steps.assign(2 * (size_t)std::max(D.Tmax, 1), 0);
        for (int t = 0; t < D.Tmax; t++) {
            steps[t] = D.step_off[t];
            steps[D.Tmax + t] = D.step_n[t];
            ntok += D.step_n[t];
            if (t + 1 < D.Tmax) ntok_prev += D.step_n[t];
        }
    }
    // slot table and status words: three transfers for the whole batch
    CK_CUDA(c, cudaMemcpyAsync(c->d_slots, c->h_slots, sizeof(Slot) * n, cudaMemcpyHostToDevice, s));
    CK_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
    CK_CUDA(c, cudaMemsetAsync(c->d_bstatus, 0, n * sizeof(int), s));
    if (graph) {
        if (!gr) {
            GraphRec g;
            g.persist = persist;
            g.Tmax = D.Tmax;
            g.ntok = ntok;
            g.ntok_prev = ntok_prev;
            CK_CUDA(c, cudaMalloc(&g.d_tok, D.tok.size() * sizeof(int)));
            CK_CUDA(c, cudaMalloc(&g.d_kn, std::max<size_t>(D.kn.size(), 1) * sizeof(int2)));
            CK_CUDA(c, cudaMemcpy(g.d_tok, D.tok.data(), D.tok.size() * sizeof(int), cudaMemcpyHostToDevice));
            if (!D.kn.empty())
                CK_CUDA(c, cudaMemcpy(g.d_kn, D.kn.data(), D.kn.size() * sizeof(int2), cudaMemcpyHostToDevice));
            if (persist) {
                CK_CUDA(c, cudaMalloc(&g.d_step, steps.size() * sizeof(int)));
                CK_CUDA(c, cudaMemcpy(g.d_step, steps.data(), steps.size() * sizeof(int), cudaMemcpyHostToDevice));
            }
            long l0 = c->launches;
            // persistent: one graph with the prologues and coder set-up;
            // otherwise every step, in segments of SEG_STEPS
            int span = persist ? 1 : std::max(D.Tmax, 1), seg = persist ? 1 : SEG_STEPS;
            for (int t0 = 0; t0 < span; t0 += seg) {
                int t1 = persist ? 0 : std::min(D.Tmax, t0 + SEG_STEPS);
                cudaGraph_t gph;
                cudaGraphExec_t ex = nullptr;
                cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    enqueue_decode(c, D, g.d_tok, g.d_kn, c->cap_stream, &failed, t0, t1);
                    e = cudaStreamEndCapture(c->cap_stream, &gph);
                }
                if (e == cudaSuccess && !failed) {
                    e = cudaGraphInstantiate(&ex, gph, 0);
                    cudaGraphDestroy(gph);
                }
                if (e != cudaSuccess || failed) {
                    c->launches = l0;
                    graph_free(g);
                    return fail(c, PSW_ERR_CUDA, "decode capture: %s",
                                failed ? "GEMM setup failed" : cudaGetErrorString(e));
                }
                g.exec.push_back(ex);
            }
            g.launches = c->launches - l0;
            c->launches = l0;
            if (c->graphs.size() >= GRAPH_CAP) {
                // every earlier decode has completed (each call synchronises
                // its stream before returning): drop the least recently used
                auto lru = c->graphs.begin();
                for (auto jt = c->graphs.begin(); jt != c->graphs.end(); ++jt)
                    if (jt->second.used < lru->second.used) lru = jt;
                graph_free(lru->second);
                c->graphs.erase(lru);
            }
            g.used = ++c->graph_clock;
            gr = &(c->graphs[key] = g);
        }
        for (cudaGraphExec_t ex : gr->exec) CK_CUDA(c, cudaGraphLaunch(ex, s));
        c->launches += gr->launches;
        if (gr->persist &&
            (st = persist_run(c, gr->d_tok, gr->d_step, gr->d_kn, n, gr->Tmax, gr->ntok, gr->ntok_prev, s)))
            return st;
        c->last_engine = gr->persist ? PSW_ENGINE_PERSISTENT : PSW_ENGINE_GRAPH;
    } else {
        if ((st = grow_tokens(c, D.tok.size(), std::max<size_t>(D.kn.size(), 1)))) return st;
        CK_CUDA(c, cudaMemcpyAsync(c->d_tok, D.tok.data(), D.tok.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        if (!D.kn.empty())
            CK_CUDA(c, cudaMemcpyAsync(c->d_kn, D.kn.data(), D.kn.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        if (persist) {
            if (steps.size() > c->step_cap) {
                CK_CUDA(c, cudaDeviceSynchronize());
                cudaFree(c->d_step);
                c->d_step = nullptr; c->step_cap = 0;
                CK_CUDA(c, cudaMalloc(&c->d_step, steps.size() * sizeof(int)));
                c->step_cap = steps.size();
            }
            CK_CUDA(c, cudaMemcpyAsync(c->d_step, steps.data(), steps.size() * sizeof(int), cudaMemcpyHostToDevice, s));
            enqueue_decode(c, D, c->d_tok, c->d_kn, s, &failed, 0, 0);
            if (!failed && (st = persist_run(c, c->d_tok, c->d_step, c->d_kn, n, D.Tmax, ntok, ntok_prev, s)))
                return st;
        } else {
            enqueue_decode(c, D, c->d_tok, c->d_kn, s, &failed, 0, D.Tmax);
        }
        CK_CUDA(c, cudaStreamSynchronize(s));   // host token lists are reused by the next call
        if (failed) return fail(c, PSW_ERR_CUDA, "a GEMM launch could not be prepared");
        c->last_engine = persist ? PSW_ENGINE_PERSISTENT : 0;
    }
    CK_CUDA(c, cudaGetLastError());
    // every frame's outputs and its sequence's previous latents in one copy
    // launch, then the status words back in two transfers
    int nj = 0;
    unsigned long long maxb = 0;
    auto job = [&](const void *src, void *dst, size_t bytes) {
        c->h_jobs[nj++] = CopyJob{src, dst, (unsigned long long)bytes};
        maxb = std::max<unsigned long long>(maxb, bytes);
    };
    for (int b = 0; b < n; b++) {
        psw_seq *q = qs[b];
        size_t nsym = (size_t)fds[b].H * fds[b].W * c->md.C;
        job(q->y, yout[b], nsym * 2);
        if (mu_out && mu_out[b]) job(q->mu, mu_out[b], nsym * 4);
        if (sg_out && sg_out[b]) job(q->sigma, sg_out[b], nsym * 4);
        job(q->y, q->yprev, nsym * 2);
    }
    CK_CUDA(c, cudaMemcpyAsync(c->d_jobs, c->h_jobs, nj * sizeof(CopyJob), cudaMemcpyHostToDevice, s));
    launch_copy_jobs(c->d_jobs, nj, maxb, s);
    CK_CUDA(c, cudaGetLastError());
    CK_CUDA(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK_CUDA(c, cudaMemcpyAsync(c->h_status + 1, c->d_bstatus, n * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK_CUDA(c, cudaStreamSynchronize(s));
    std::vector<int> sts(n);
    for (int b = 0; b < n; b++) sts[b] = c->h_status[1 + b] | c->h_status[0];
    psw_status first = PSW_OK;
    for (int b = 0; b < n; b++) {
        qs[b]->frame++;
        qs[b]->coded_H = fds[b].H; qs[b]->coded_W = fds[b].W;
        psw_status sb = status_code(c, sts[b]);
        if (status_out) status_out[b] = sb;
        if (sb && !first) first = sb;
    }
    return first;
}

// Encode the symbols of slot 0 (already in the slot table) into a container.
void encode_symbols(psw_ctx *c, psw_seq *q, const psw_frame_desc *fd, uint8_t *bs, size_t cap, cudaStream_t s)
{
    int HW = fd->H * fd->W, C = c->md.C;
    int cap_words = 3 * HW + 64;
    {
        Scope sc(c, s, K_RANS, 0.0, (double)HW * C * 7.0);
        launch_rans_encode(coder(c), c->d_slots, 0, HW, C, q->enc_scratch, cap_words, q->enc_nw, q->rstate, s);
    }
    {
        Scope sc(c, s, K_RANS, 0.0, (double)HW * C * 2.0);
        launch_rans_assemble(fd->H, fd->W, C, fd->schedule, q->enc_scratch, cap_words, q->enc_nw, q->rstate, bs, cap,
                             q->enc_total, q->d_status, s);
    }
    cudaMemcpyAsync(q->h_total, q->enc_total, 8, cudaMemcpyDeviceToHost, s);
}

}  // namespace

bool psw_coder_view(const psw_ctx *c, int *C, int *mask, const uint32_t **cdf, const int **meta)
{
    if (!c) return false;
    *C = c->md.C;
    *mask = c->md.mask;
    *cdf = c->d_cdf;
    *meta = c->d_meta;
    return true;
}

// ====================================================================== ABI

extern "C" {

size_t psw_weights_count(const psw_model_desc *desc)
{
    std::string why;
    if (!desc_valid(desc, why)) return 0;
    return (size_t)make_layout(*desc).total;
}

const char *psw_last_error(const psw_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

size_t psw_ctx_bytes(const psw_ctx *ctx) { return ctx ? ctx->bytes : 0; }

size_t psw_seq_bytes(const psw_ctx *ctx, int max_H, int max_W)
{
    if (!ctx || max_H < 1 || max_W < 1) return 0;
    return seq_bytes_for(ctx->md, ctx->prec, max_H, max_W);
}

psw_status psw_create(const psw_model_desc *desc, const float *weights_host, size_t n_weights, int precision,
                      size_t hbm_budget, psw_ctx **out)
{
    if (!out) return fail(nullptr, PSW_ERR_INVALID, "null output pointer");
    *out = nullptr;
    std::string why;
    if (!desc_valid(desc, why)) return fail(nullptr, PSW_ERR_INVALID, "%s", why.c_str());
    if (precision != PSW_FP32 && precision != PSW_BF16 && precision != PSW_FP8)
        return fail(nullptr, PSW_ERR_INVALID, "unknown precision %d", precision);
    Layout lay = make_layout(*desc);
    if (!weights_host || n_weights != (size_t)lay.total)
        return fail(nullptr, PSW_ERR_INVALID, "expected %ld weights, got %zu", lay.total, n_weights);
    if (precision != PSW_FP32 && !gemm_tc_available())
        return fail(nullptr, PSW_ERR_CUDA, "the driver offers no cuTensorMapEncodeTiled entry point");
    if (precision != PSW_FP32 && !gemm_ws_prepare())
        return fail(nullptr, PSW_ERR_CUDA, "wide projection kernel attributes");
    if (!attention_prepare()) return fail(nullptr, PSW_ERR_CUDA, "attention kernel attributes");
    psw_ctx *c = new psw_ctx();
    c->md = *desc; c->budget = hbm_budget; c->lay = lay;
    c->prec = precision == PSW_FP8 ? P_BF16 : precision;
    c->fp8 = precision == PSW_FP8;
    prepare_projections(c, /*dry=*/true);
    build_cdf_tables(c->tabs);
    c->bytes = (size_t)lay.total * 4 + c->arena + (size_t)c->tabs.total * 4 + 3 * 64 * 4 + 64 * 4 +
               MAX_SLOTS * sizeof(Slot);
    if (hbm_budget && c->bytes > hbm_budget) {
        size_t need = c->bytes;
        psw_destroy(c);
        return fail(nullptr, PSW_ERR_OOM, "weights and tables need %zu bytes, budget %zu", need, hbm_budget);
    }
    cudaError_t e = cudaMalloc(&c->w, (size_t)lay.total * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->wmat, c->arena);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_cdf, (size_t)c->tabs.total * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_meta, 3 * 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_scale, 64 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_slots, MAX_SLOTS * sizeof(Slot));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_bstatus, MAX_SLOTS * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_jobs, 4 * MAX_SLOTS * sizeof(CopyJob));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_jobs, 4 * MAX_SLOTS * sizeof(CopyJob));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_slots, MAX_SLOTS * sizeof(Slot));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_status, (MAX_SLOTS + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_rate, sizeof(double));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        psw_destroy(c);
        return fail(nullptr, PSW_ERR_OOM, "device allocation: %s", cudaGetErrorString(e));
    }
    int meta[3 * 64];
    for (int l = 0; l < 64; l++) { meta[l] = c->tabs.T[l]; meta[64 + l] = c->tabs.n[l]; meta[128 + l] = c->tabs.off[l]; }
    e = cudaMemcpy(c->w, weights_host, (size_t)lay.total * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_cdf, c->tabs.packed, (size_t)c->tabs.total * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_meta, meta, sizeof(meta), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_scale, c->tabs.scale, 64 * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !prepare_projections(c, /*dry=*/false)) e = cudaErrorInvalidValue;
    if (e == cudaSuccess && desc->hp) {
        build_prior_tables(*desc, lay, weights_host, c->ptab);
        std::vector<int> pm(3 * (size_t)desc->Ch);
        for (int ch = 0; ch < desc->Ch; ch++) {
            pm[ch] = PRIOR_T; pm[desc->Ch + ch] = PRIOR_N; pm[2 * desc->Ch + ch] = ch * PRIOR_N;
        }
        e = cudaMalloc(&c->d_pcdf, c->ptab.size() * 4);
        if (e == cudaSuccess) e = cudaMalloc(&c->d_pmeta, pm.size() * sizeof(int));
        if (e == cudaSuccess) e = cudaMemcpy(c->d_pcdf, c->ptab.data(), c->ptab.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->d_pmeta, pm.data(), pm.size() * sizeof(int), cudaMemcpyHostToDevice);
        c->bytes += c->ptab.size() * 4 + pm.size() * sizeof(int);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        psw_destroy(c);
        return fail(nullptr, PSW_ERR_CUDA, "weight upload / preparation: %s", cudaGetErrorString(e));
    }
    *out = c;
    return PSW_OK;
}

void psw_destroy(psw_ctx *c)
{
    if (!c) return;
    while (!c->seqs.empty()) psw_seq_destroy(c->seqs.back());
    for (auto &kv : c->graphs) graph_free(kv.second);
    program_free(c->prog);
    cudaFree(c->d_pbar);
    cudaFree(c->d_step);
    cudaFree(c->w); cudaFree(c->wmat); cudaFree(c->d_cdf); cudaFree(c->d_meta); cudaFree(c->d_scale);
    cudaFree(c->d_bstatus); cudaFree(c->d_jobs);
    if (c->h_jobs) cudaFreeHost(c->h_jobs);
    cudaFree(c->rate_buf); cudaFree(c->d_slots); cudaFree(c->d_status); cudaFree(c->d_tok); cudaFree(c->d_kn);
    cudaFree(c->Xn); cudaFree(c->Q); cudaFree(c->O); cudaFree(c->Hid);
    cudaFree(c->Xa); cudaFree(c->Xb); cudaFree(c->Xg); cudaFree(c->Xc); cudaFree(c->NM);
    cudaFree(c->Xn8); cudaFree(c->xs8);
    for (float *g : c->hg) cudaFree(g);
    cudaFree(c->hcol); cudaFree(c->hz_idx); cudaFree(c->hz_m); cudaFree(c->hz_order); cudaFree(c->hz_status);
    cudaFree(c->hz_rstate); cudaFree(c->hz_rptr); cudaFree(c->hz_rend); cudaFree(c->hz_nw); cudaFree(c->hz_scratch);
    cudaFree(c->hz_total); cudaFree(c->d_pcdf); cudaFree(c->d_pmeta);
    if (c->h_rate) cudaFreeHost(c->h_rate);
    if (c->h_slots) cudaFreeHost(c->h_slots);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
    free_cdf_tables(c->tabs);
    delete c;
}

psw_status psw_seq_create(psw_ctx *c, int max_H, int max_W, psw_seq **out)
{
    if (!c || !out) return fail(c, PSW_ERR_INVALID, "null argument");
    *out = nullptr;
    if (max_H < 1 || max_W < 1 || max_H > 4096 || max_W > 4096 || (long)max_H * max_W >= (1L << POS_BITS))
        return fail(c, PSW_ERR_INVALID, "bad maximum grid %dx%d", max_H, max_W);
    size_t need = seq_bytes_for(c->md, c->prec, max_H, max_W);
    size_t ws_more = 0, HW = (size_t)max_H * max_W;
    if (HW > c->ws_rows) {
        size_t bd, bf, bx, bg, bc, bn;
        ws_sizes(c->md, c->prec, HW, bd, bf, bx, bg, bc, bn);
        ws_more = 3 * bd + bf + 2 * bx + bg + bc + bn - c->ws_bytes;
    }
    size_t used = c->bytes;
    for (psw_seq *s : c->seqs) used += s->bytes;
    if (c->budget && used + need + ws_more > c->budget)
        return fail(c, PSW_ERR_OOM, "sequence needs %zu bytes; %zu of %zu in use", need + ws_more, used, c->budget);
    psw_status st = ensure_workspace(c, HW);
    if (st) return st;
    if ((st = ensure_hyper(c, max_H, max_W))) return st;
    psw_seq *q = new psw_seq();
    q->ctx = c; q->maxH = max_H; q->maxW = max_W; q->maxHW = (int)HW; q->bytes = need;
    const psw_model_desc &m = c->md;
    size_t d = m.d, es = esize(c->prec);
    bool okay = true;
    auto dal = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (!okay) return nullptr;
        if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) { okay = false; return nullptr; }
        q->allocs.push_back(p);
        return p;
    };
    q->eh = (float *)dal(HW * d * 4);
    q->qa = dal(HW * d * es);
    q->K1 = dal(m.L * HW * d * es); q->V1 = dal(m.L * HW * d * es);
    q->K2 = dal(m.L * HW * d * es); q->V2 = dal(m.L * HW * d * es);
    q->Ka = dal(HW * d * es); q->Va = dal(HW * d * es);
    if (m.temporal) {
        q->CK = dal((size_t)m.Lc * m.Tf * HW * d * es); q->CV = dal((size_t)m.Lc * m.Tf * HW * d * es);
        q->XK = dal(2 * (size_t)m.L * m.Tf * HW * d * es); q->XV = dal(2 * (size_t)m.L * m.Tf * HW * d * es);
    }
    if (m.Llrp) {
        size_t lb = (size_t)m.Llrp * (m.temporal ? m.Tf : 1) * HW * d * es;
        q->rep = (float *)dal(HW * (m.Nc ? m.dc : d) * 4);
        q->LK = dal(lb); q->LV = dal(lb);
    }
    q->mu = (float *)dal(HW * m.C * 4); q->sigma = (float *)dal(HW * m.C * 4);
    q->idx = (uint8_t *)dal(HW * m.C); q->m = (int32_t *)dal(HW * m.C * 4);
    q->y = (int16_t *)dal(HW * m.C * 2); q->yprev = (int16_t *)dal(HW * m.C * 2);
    q->rstate = (uint32_t *)dal((size_t)m.C * 32 * 4);
    q->rptr = (uint32_t *)dal((size_t)m.C * 4); q->rend = (uint32_t *)dal((size_t)m.C * 4);
    q->enc_nw = (uint32_t *)dal((2 * (size_t)m.C + 1) * 4);
    q->enc_scratch = (uint16_t *)dal((size_t)m.C * (3 * HW + 64) * 2);
    q->enc_total = (uint64_t *)dal(8);
    q->d_status = (int *)dal(4);
    q->d_order = (int *)dal(HW * 4);
    if (okay && cudaMallocHost(&q->h_total, 8) != cudaSuccess) okay = false;
    if (!okay) {
        psw_seq_destroy(q);
        return fail(c, PSW_ERR_OOM, "sequence allocation of %zu bytes failed", need);
    }
    c->seqs.push_back(q);
    *out = q;
    return PSW_OK;
}

psw_status psw_seq_reset(psw_seq *q)
{
    if (!q) return PSW_ERR_INVALID;
    q->frame = 0;
    q->coded_H = q->coded_W = 0;
    q->lrp_done = 0;
    return PSW_OK;
}

void psw_seq_destroy(psw_seq *q)
{
    if (!q) return;
    if (q->ctx) {
        psw_ctx *c = q->ctx;
        cudaDeviceSynchronize();
        // drop the graphs that name this sequence
        for (auto it = c->graphs.begin(); it != c->graphs.end();) {
            bool hit = false;
            for (size_t a = KEY_SEQ0; a < it->first.size(); a += 2)
                if (it->first[a] == (long)(uintptr_t)q) hit = true;
            if (hit) {
                graph_free(it->second);
                it = c->graphs.erase(it);
            } else {
                ++it;
            }
        }
        auto &v = c->seqs;
        for (size_t a = 0; a < v.size(); a++)
            if (v[a] == q) { v.erase(v.begin() + a); break; }
    }
    for (void *p : q->allocs) cudaFree(p);
    if (q->h_total) cudaFreeHost(q->h_total);
    delete q;
}

size_t psw_bitstream_capacity(const psw_ctx *c, const psw_frame_desc *fd)
{
    if (!c || !fd || fd->H < 1 || fd->W < 1) return 0;
    return container_capacity(fd->H, fd->W, c->md.C);
}

psw_status psw_encode_params(psw_ctx *c, psw_seq *q, const psw_frame_desc *fd, const int16_t *yhat_dev,
                             const int16_t *zhat_dev, float *mu_dev, float *sigma_dev, uint8_t *bitstream_dev,
                             size_t cap, size_t *len_out, void *stream)
{
    psw_status st = check_frame(c, q, fd);
    if (st) return st;
    if (!yhat_dev || !zhat_dev) return fail(c, PSW_ERR_INVALID, "null latent / hyperlatent pointer");
    if (bitstream_dev && !len_out) return fail(c, PSW_ERR_INVALID, "len_out required with a bitstream");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = seq_schedule(q, fd->H, fd->W, fd->schedule))) return st;
    int HW = fd->H * fd->W;
    size_t nsym = (size_t)HW * c->md.C;
    if ((st = ensure_workspace(c, HW))) return st;
    const bool tc_embed = !c->Whp_t.empty() && !c->md.hp;
    if ((st = grow_tokens(c, tc_embed ? 2 * (size_t)HW : HW, 1))) return st;
    Slot sl = make_slot(q, fd->H, fd->W, fd->schedule);
    sl.zhat = zhat_dev;
    c->h_slots[0] = sl;
    std::vector<psw_seq *> qs{q};
    if ((st = upload_slots(c, qs, 1, s))) return st;
    std::vector<int> tok(HW);
    for (int p = 0; p < HW; p++) tok[p] = tok_make(0, p);
    // the tensor-core hyperprior embedding's positions, tap by tap
    std::vector<int> tap_off, tap_n;
    if (tc_embed) {
        std::vector<std::vector<int>> seg;
        tap_tokens(0, fd->H, fd->W, c->md.r, seg);
        for (auto &v : seg) {
            tap_off.push_back((int)tok.size());
            tap_n.push_back((int)v.size());
            tok.insert(tok.end(), v.begin(), v.end());
        }
    }
    CK_CUDA(c, cudaMemcpyAsync(c->d_tok, tok.data(), tok.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CK_CUDA(c, cudaMemcpyAsync(q->y, yhat_dev, nsym * 2, cudaMemcpyDeviceToDevice, s));
    bool failed = false;
    Pass P{c, s, c->d_slots, &failed};
    // masked parallel pass over every position (Sec. 3.1, Sec. 3.2)
    if (tc_embed) hyper_embed_tc(P, c->d_tok, tap_off, tap_n);
    frame_prologue(P, c->d_tok, fd->H, fd->W, q->eh);
    run_sm1(P, c->d_tok, HW);
    run_acc_sm2_heads(P, c->d_tok, HW);
    for (int g = 0; g < c->md.Nc; g++) run_ct_group(P, c->d_tok, HW, g);
    if (mu_dev) CK_CUDA(c, cudaMemcpyAsync(mu_dev, q->mu, nsym * 4, cudaMemcpyDeviceToDevice, s));
    if (sigma_dev) CK_CUDA(c, cudaMemcpyAsync(sigma_dev, q->sigma, nsym * 4, cudaMemcpyDeviceToDevice, s));
    CK_CUDA(c, cudaGetLastError());
    if (len_out) *len_out = 0;
    if (bitstream_dev) encode_symbols(c, q, fd, bitstream_dev, cap, s);
    // the sequence advances even if the container did not fit
    CK_CUDA(c, cudaMemcpyAsync(q->yprev, q->y, nsym * 2, cudaMemcpyDeviceToDevice, s));
    std::vector<int> sts;
    if ((st = read_status(c, qs, s, sts))) return st;   // synchronises: the token list is free again
    q->frame++;
    q->coded_H = fd->H; q->coded_W = fd->W;
    if (bitstream_dev) *len_out = (size_t)*q->h_total;
    if (failed) return fail(c, PSW_ERR_CUDA, "a GEMM launch could not be prepared");
    if (sts[0] & ST_CAPACITY)
        return fail(c, PSW_ERR_CAPACITY, "container needs %zu bytes, capacity %zu", (size_t)*q->h_total, cap);
    return status_code(c, sts[0]);
}

psw_status psw_decode_frame(psw_ctx *c, psw_seq *q, const psw_frame_desc *fd, const uint8_t *bitstream_dev,
                            size_t len, const int16_t *zhat_dev, int16_t *yhat_out_dev, float *mu_dev,
                            float *sigma_dev, void *stream)
{
    if (!c) return PSW_ERR_INVALID;
    return decode_run(c, 1, &q, fd, &bitstream_dev, &len, &zhat_dev, &yhat_out_dev, &mu_dev, &sigma_dev, nullptr,
                      (cudaStream_t)stream);
}

psw_status psw_decode_batch(psw_ctx *c, int n, psw_seq *const *seqs, const psw_frame_desc *fds,
                            const uint8_t *const *bitstreams_dev, const size_t *lens, const int16_t *const *zhat_dev,
                            int16_t *const *yhat_out_dev, float *const *mu_dev, float *const *sigma_dev,
                            int *status_out, void *stream)
{
    if (!c) return PSW_ERR_INVALID;
    if (n < 1 || !seqs || !fds || !bitstreams_dev || !lens || !zhat_dev || !yhat_out_dev)
        return fail(c, PSW_ERR_INVALID, "bad batch arguments");
    return decode_run(c, n, seqs, fds, bitstreams_dev, lens, zhat_dev, yhat_out_dev, mu_dev, sigma_dev, status_out,
                      (cudaStream_t)stream);
}

psw_status psw_lrp_residual(psw_ctx *c, psw_seq *q, const psw_frame_desc *fd, float *eps_dev, void *stream)
{
    psw_status st = check_frame(c, q, fd);
    if (st) return st;
    const psw_model_desc &m = c->md;
    if (m.Llrp <= 0) return fail(c, PSW_ERR_INVALID, "the model has no LRP Transformer");
    if (q->frame < 1) return fail(c, PSW_ERR_INVALID, "no frame coded since the sequence was created or reset");
    if (fd->H != q->coded_H || fd->W != q->coded_W)
        return fail(c, PSW_ERR_INVALID, "frame %dx%d is not the last coded frame's grid %dx%d", fd->H, fd->W,
                    q->coded_H, q->coded_W);
    if (m.temporal && q->lrp_done < q->frame - 1)
        return fail(c, PSW_ERR_INVALID, "the LRP of frame %d was not run", q->lrp_done);
    if (m.temporal && q->lrp_done > q->frame - 1)
        return fail(c, PSW_ERR_INVALID, "the LRP of frame %d already ran", q->frame - 1);
    if (!eps_dev && !m.temporal) return fail(c, PSW_ERR_INVALID, "null eps pointer");
    cudaStream_t s = (cudaStream_t)stream;
    int HW = fd->H * fd->W;
    if ((st = ensure_workspace(c, HW))) return st;
    if ((st = grow_tokens(c, HW, 1))) return st;
    c->h_slots[0] = make_slot(q, fd->H, fd->W, fd->schedule, q->frame - 1);
    std::vector<psw_seq *> qs{q};
    if ((st = upload_slots(c, qs, 1, s))) return st;
    std::vector<int> tok(HW);
    for (int p = 0; p < HW; p++) tok[p] = tok_make(0, p);
    CK_CUDA(c, cudaMemcpyAsync(c->d_tok, tok.data(), HW * sizeof(int), cudaMemcpyHostToDevice, s));
    bool failed = false;
    Pass P{c, s, c->d_slots, &failed};
    run_lrp(P, c->d_tok, HW, q->rep, eps_dev);
    CK_CUDA(c, cudaGetLastError());
    std::vector<int> sts;
    if ((st = read_status(c, qs, s, sts))) return st;   // synchronises: the token list is free again
    if (failed) return fail(c, PSW_ERR_CUDA, "a GEMM launch could not be prepared");
    q->lrp_done = q->frame;
    return status_code(c, sts[0]);
}

psw_status psw_hyper_encode(psw_ctx *c, psw_seq *q, const psw_frame_desc *fd, const int16_t *yhat_dev,
                            int16_t *zhat_dev, float *z_dev, uint8_t *bitstream_dev, size_t cap, size_t *len_out,
                            void *stream)
{
    psw_status st = check_frame(c, q, fd);
    if (st) return st;
    const psw_model_desc &m = c->md;
    if (!m.hp) return fail(c, PSW_ERR_INVALID, "the model has no convolutional hyperprior");
    if (!yhat_dev || !zhat_dev) return fail(c, PSW_ERR_INVALID, "null latent / hyperlatent pointer");
    if (bitstream_dev && !len_out) return fail(c, PSW_ERR_INVALID, "len_out required with a bitstream");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = seq_schedule(q, fd->H, fd->W, fd->schedule))) return st;
    const int HW = fd->H * fd->W, Hh = (fd->H + m.r - 1) / m.r, Wh = (fd->W + m.r - 1) / m.r, HWz = Hh * Wh;
    if ((st = ensure_workspace(c, HW))) return st;
    if ((st = grow_tokens(c, HW, 1))) return st;
    if ((st = ensure_hyper(c, fd->H, fd->W))) return st;
    // slot 0: the frame (Spatial Module 1 and, for the temporal model, its
    // context); slot 1: the z-hat coder
    Slot sl = make_slot(q, fd->H, fd->W, fd->schedule);
    sl.zhat = zhat_dev;
    c->h_slots[0] = sl;
    Slot zs;
    memset(&zs, 0, sizeof(zs));
    zs.H = Hh; zs.W = Wh; zs.stride = HWz; zs.sched = PSW_SCHED_RASTER; zs.nfr = 1;
    zs.y = zhat_dev; zs.idx = c->hz_idx; zs.m = c->hz_m; zs.order = c->hz_order;
    zs.rstate = c->hz_rstate; zs.rptr = c->hz_rptr; zs.rend = c->hz_rend; zs.status = c->hz_status;
    c->h_slots[1] = zs;
    std::vector<psw_seq *> qs{q};
    if ((st = upload_slots(c, qs, 2, s))) return st;
    CK_CUDA(c, cudaMemsetAsync(c->hz_status, 0, sizeof(int), s));
    std::vector<int> tok(HW);
    for (int p = 0; p < HW; p++) tok[p] = tok_make(0, p);
    CK_CUDA(c, cudaMemcpyAsync(c->d_tok, tok.data(), HW * sizeof(int), cudaMemcpyHostToDevice, s));
    CK_CUDA(c, cudaMemcpyAsync(q->y, yhat_dev, (size_t)HW * m.C * 2, cudaMemcpyDeviceToDevice, s));
    bool failed = false;
    Pass P{c, s, c->d_slots, &failed};
    if (m.temporal) frame_context(P, c->d_tok, HW);
    run_sm1(P, c->d_tok, HW);
    hyper_analysis(P, fd->H, fd->W, zhat_dev, z_dev);
    if (len_out) *len_out = 0;
    if (bitstream_dev) {
        const int cap_words = 3 * HWz + 64;
        CoderDev cd{c->d_pcdf, c->d_pmeta, m.Ch};
        {
            Scope sc(c, s, K_RANS, 0.0, (double)HWz * m.Ch * 7.0);
            launch_rans_encode(cd, c->d_slots, 1, HWz, m.Ch, c->hz_scratch, cap_words, c->hz_nw, c->hz_rstate, s);
        }
        Scope sc(c, s, K_RANS, 0.0, (double)HWz * m.Ch * 2.0);
        launch_rans_assemble(Hh, Wh, m.Ch, PSW_SCHED_RASTER, c->hz_scratch, cap_words, c->hz_nw, c->hz_rstate,
                             bitstream_dev, cap, c->hz_total, c->hz_status, s);
    }
    CK_CUDA(c, cudaGetLastError());
    uint64_t total = 0;
    int zst = 0;
    if (bitstream_dev) CK_CUDA(c, cudaMemcpyAsync(&total, c->hz_total, 8, cudaMemcpyDeviceToHost, s));
    CK_CUDA(c, cudaMemcpyAsync(&zst, c->hz_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    std::vector<int> sts;
    if ((st = read_status(c, qs, s, sts))) return st;   // synchronises
    if (failed) return fail(c, PSW_ERR_CUDA, "a GEMM launch could not be prepared");
    if (bitstream_dev) *len_out = (size_t)total;
    if (zst & ST_CAPACITY) return fail(c, PSW_ERR_CAPACITY, "z-hat container needs %zu bytes, capacity %zu",
                                       (size_t)total, cap);
    return status_code(c, sts[0] | zst);
}

psw_status psw_hyper_decode(psw_ctx *c, const psw_frame_desc *fd, const uint8_t *bitstream_dev, size_t len,
                            int16_t *zhat_dev, void *stream)
{
    if (!c) return PSW_ERR_INVALID;
    const psw_model_desc &m = c->md;
    if (!m.hp) return fail(c, PSW_ERR_INVALID, "the model has no convolutional hyperprior");
    if (!fd || fd->H < 1 || fd->W < 1 || !bitstream_dev || !zhat_dev) return fail(c, PSW_ERR_INVALID, "bad argument");
    if ((uintptr_t)bitstream_dev & 3) return fail(c, PSW_ERR_INVALID, "bitstream must be 4-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const int Hh = (fd->H + m.r - 1) / m.r, Wh = (fd->W + m.r - 1) / m.r, HWz = Hh * Wh;
    psw_status st;
    if ((st = ensure_hyper(c, fd->H, fd->W))) return st;
    if ((st = grow_tokens(c, 1, 1))) return st;
    Slot zs;
    memset(&zs, 0, sizeof(zs));
    zs.H = Hh; zs.W = Wh; zs.stride = HWz; zs.sched = PSW_SCHED_RASTER; zs.nfr = 1;
    zs.y = zhat_dev; zs.idx = c->hz_idx; zs.m = c->hz_m; zs.order = c->hz_order;
    zs.rstate = c->hz_rstate; zs.rptr = c->hz_rptr; zs.rend = c->hz_rend; zs.status = c->hz_status;
    zs.bs = bitstream_dev; zs.len = len;
    c->h_slots[0] = zs;
    CK_CUDA(c, cudaMemcpyAsync(c->d_slots, c->h_slots, sizeof(Slot), cudaMemcpyHostToDevice, s));
    CK_CUDA(c, cudaMemsetAsync(c->hz_status, 0, sizeof(int), s));
    int2 kn = make_int2(0, HWz);
    CK_CUDA(c, cudaMemcpyAsync(c->d_kn, &kn, sizeof(int2), cudaMemcpyHostToDevice, s));
    CoderDev cd{c->d_pcdf, c->d_pmeta, m.Ch};
    launch_rans_dec_init(c->d_slots, 1, m.Ch, s);
    launch_rans_dec_step(cd, c->d_slots, 1, c->d_kn, m.Ch, s);
    launch_rans_dec_finish(c->d_slots, 1, m.Ch, s);
    c->launches += 3;
    CK_CUDA(c, cudaGetLastError());
    int zst = 0;
    CK_CUDA(c, cudaMemcpyAsync(&zst, c->hz_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK_CUDA(c, cudaStreamSynchronize(s));
    return status_code(c, zst);
}

psw_status psw_prior_table(const psw_ctx *c, int ch, uint32_t *freq_host, int cap, int *n_out)
{
    if (!c || !c->md.hp || ch < 0 || ch >= c->md.Ch) return PSW_ERR_INVALID;
    if (n_out) *n_out = PRIOR_N;
    if (!freq_host) return PSW_OK;
    if (cap < PRIOR_N) return PSW_ERR_CAPACITY;
    for (int a = 0; a < PRIOR_N; a++) freq_host[a] = c->ptab[(size_t)ch * PRIOR_N + a] >> 16;
    return PSW_OK;
}

psw_status psw_rate(psw_ctx *c, size_t n, const int16_t *yhat_dev, const float *mu_dev, const float *sigma_dev,
                    double *bits_out_host, void *stream)
{
    if (!c || !bits_out_host || (n && (!yhat_dev || !mu_dev || !sigma_dev)))
        return fail(c, PSW_ERR_INVALID, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    size_t need = (size_t)rate_partials(n) + 1;
    if (need > c->rate_cap) {
        CK_CUDA(c, cudaStreamSynchronize(s));
        cudaFree(c->rate_buf);
        c->rate_buf = nullptr;
        c->rate_cap = 0;
        CK_CUDA(c, cudaMalloc(&c->rate_buf, need * sizeof(double)));
        c->rate_cap = need;
    }
    launch_rate(n, yhat_dev, mu_dev, sigma_dev, c->rate_buf + 1, c->rate_buf, s);
    CK_CUDA(c, cudaMemcpyAsync(c->h_rate, c->rate_buf, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK_CUDA(c, cudaStreamSynchronize(s));
    *bits_out_host = *c->h_rate;
    return PSW_OK;
}

psw_status psw_quantize(psw_ctx *c, size_t n, const float *mu_dev, const float *sigma_dev, uint8_t *idx_dev,
                        int32_t *m_dev, void *stream)
{
    if (!c || (n && (!mu_dev || !sigma_dev || !idx_dev || !m_dev))) return fail(c, PSW_ERR_INVALID, "null argument");
    launch_quantize(n, mu_dev, sigma_dev, c->d_scale, idx_dev, m_dev, (cudaStream_t)stream);
    CK_CUDA(c, cudaGetLastError());
    return PSW_OK;
}

psw_status psw_scale_table(const psw_ctx *c, float *table_host)
{
    if (!c || !table_host) return PSW_ERR_INVALID;
    memcpy(table_host, c->tabs.scale, sizeof(c->tabs.scale));
    return PSW_OK;
}

psw_status psw_cdf_table(const psw_ctx *c, int l, uint32_t *freq_host, int cap, int *n_out, int *T_out)
{
    if (!c || l < 0 || l >= NSCALES) return PSW_ERR_INVALID;
    int n = c->tabs.n[l];
    if (n_out) *n_out = n;
    if (T_out) *T_out = c->tabs.T[l];
    if (!freq_host) return PSW_OK;
    if (cap < n) return PSW_ERR_CAPACITY;
    for (int a = 0; a < n; a++) freq_host[a] = c->tabs.packed[c->tabs.off[l] + a] >> 16;
    return PSW_OK;
}

psw_status psw_rans_encode(psw_ctx *c, psw_seq *q, const psw_frame_desc *fd, const int16_t *yhat_dev,
                           const uint8_t *idx_dev, const int32_t *m_dev, uint8_t *bitstream_dev, size_t cap,
                           size_t *len_out, void *stream)
{
    psw_status st = check_frame(c, q, fd);
    if (st) return st;
    if (!yhat_dev || !idx_dev || !m_dev || !bitstream_dev || !len_out) return fail(c, PSW_ERR_INVALID, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = seq_schedule(q, fd->H, fd->W, fd->schedule))) return st;
    Slot sl = make_slot(q, fd->H, fd->W, fd->schedule);
    sl.y = const_cast<int16_t *>(yhat_dev);
    sl.idx = const_cast<uint8_t *>(idx_dev);
    sl.m = const_cast<int32_t *>(m_dev);
    c->h_slots[0] = sl;
    std::vector<psw_seq *> qs{q};
    if ((st = upload_slots(c, qs, 1, s))) return st;
    encode_symbols(c, q, fd, bitstream_dev, cap, s);
    std::vector<int> sts;
    if ((st = read_status(c, qs, s, sts))) return st;
    *len_out = (size_t)*q->h_total;
    if (sts[0] & ST_CAPACITY) return fail(c, PSW_ERR_CAPACITY, "container needs %zu bytes, capacity %zu", *len_out, cap);
    return status_code(c, sts[0]);
}

psw_status psw_rans_decode(psw_ctx *c, psw_seq *q, const psw_frame_desc *fd, const uint8_t *bitstream_dev,
                           size_t len, const uint8_t *idx_dev, const int32_t *m_dev, int16_t *yhat_out_dev,
                           void *stream)
{
    psw_status st = check_frame(c, q, fd);
    if (st) return st;
    if (!bitstream_dev || !idx_dev || !m_dev || !yhat_out_dev) return fail(c, PSW_ERR_INVALID, "null argument");
    if ((uintptr_t)bitstream_dev & 3) return fail(c, PSW_ERR_INVALID, "bitstream must be 4-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = seq_schedule(q, fd->H, fd->W, fd->schedule))) return st;
    int C = c->md.C;
    Slot sl = make_slot(q, fd->H, fd->W, fd->schedule);
    sl.bs = bitstream_dev; sl.len = len;
    sl.idx = const_cast<uint8_t *>(idx_dev);
    sl.m = const_cast<int32_t *>(m_dev);
    sl.y = yhat_out_dev;
    c->h_slots[0] = sl;
    std::vector<psw_seq *> qs{q};
    if ((st = upload_slots(c, qs, 1, s))) return st;
    std::vector<int2> kn(q->T);
    for (int t = 0; t < q->T; t++) kn[t] = make_int2(q->h_start[t], q->h_start[t + 1] - q->h_start[t]);
    if ((st = grow_tokens(c, 1, q->T))) return st;
    CK_CUDA(c, cudaMemcpyAsync(c->d_kn, kn.data(), q->T * sizeof(int2), cudaMemcpyHostToDevice, s));
    launch_rans_dec_init(c->d_slots, 1, C, s);
    for (int t = 0; t < q->T; t++) launch_rans_dec_step(coder(c), c->d_slots, 1, c->d_kn + t, C, s);
    launch_rans_dec_finish(c->d_slots, 1, C, s);
    std::vector<int> sts;
    if ((st = read_status(c, qs, s, sts))) return st;
    return status_code(c, sts[0]);
}

long psw_launch_count(const psw_ctx *c) { return c ? c->launches : 0; }

psw_status psw_check_wait_timeout(psw_ctx *c, double seconds)
{
    if (!c) return fail(nullptr, PSW_ERR_INVALID, "null context");
    if (!(seconds > 0.0 && seconds <= 10.0)) return fail(c, PSW_ERR_INVALID, "limit must be in (0, 10] s");
    CK_CUDA(c, cudaMemset(c->d_status, 0, sizeof(int)));
    if (!wait_probe((uint64_t)(seconds * 1e9), c->d_status, 0)) return fail(c, PSW_ERR_CUDA, "wait probe launch");
    int st = 0;
    CK_CUDA(c, cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CK_CUDA(c, cudaMemset(c->d_status, 0, sizeof(int)));
    if (st & ST_TIMEOUT) return fail(c, PSW_ERR_TIMEOUT, "the bounded wait expired after %.3f s", seconds);
    return PSW_OK;
}

psw_status psw_quantize_e4m3(size_t n, const float *src, uint8_t *dst, float *scale_out)
{
    if (!scale_out || (n && (!src || !dst))) return fail(nullptr, PSW_ERR_INVALID, "null argument");
    if (((uintptr_t)src & 15) || ((uintptr_t)dst & 3)) return fail(nullptr, PSW_ERR_INVALID, "misaligned buffer");
    float s = quantize_e4m3(src, n, dst);
    if (s <= 0.0f) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(nullptr, PSW_ERR_CUDA, "E4M3 quantisation: %s", cudaGetErrorString(e));
        return fail(nullptr, PSW_ERR_INVALID, "NaN or Inf among the values");
    }
    *scale_out = s;
    return PSW_OK;
}

psw_status psw_set_engine(psw_ctx *c, int engine)
{
    if (!c) return fail(nullptr, PSW_ERR_INVALID, "null context");
    if (engine < PSW_ENGINE_AUTO || engine > PSW_ENGINE_PERSISTENT)
        return fail(c, PSW_ERR_INVALID, "unknown engine %d", engine);
    if (engine == PSW_ENGINE_PERSISTENT && c->prec != P_BF16)
        return fail(c, PSW_ERR_INVALID, "the persistent decoder runs BF16 and FP8 contexts only");
    if (engine == PSW_ENGINE_PERSISTENT && (c->md.Llrp || c->md.Nc))
        return fail(c, PSW_ERR_INVALID, "the persistent decoder does not run contexts with an LRP or a Channel Transformer");
    c->engine = engine;
    return PSW_OK;
}

int psw_last_engine(const psw_ctx *c) { return c ? c->last_engine : 0; }

psw_status psw_set_tile_policy(psw_ctx *c, int cls, int tokens)
{
    if (!c) return fail(nullptr, PSW_ERR_INVALID, "null context");
    if (cls < 0 || cls >= PSW_TILE_CLASSES) return fail(c, PSW_ERR_INVALID, "unknown launch class %d", cls);
    if (tokens != 0 && tokens != 64 && tokens != 128 && tokens != 256)
        return fail(c, PSW_ERR_INVALID, "tokens per tile must be 0, 64, 128 or 256");
    if (c->tile_policy[cls] == tokens) return PSW_OK;
    CK_CUDA(c, cudaDeviceSynchronize());
    c->tile_policy[cls] = tokens;
    // recorded graphs hold the old launches
    c->ws_gen++;
    for (auto &kv : c->graphs) graph_free(kv.second);
    c->graphs.clear();
    return PSW_OK;
}

int psw_tile_policy(const psw_ctx *c, int cls)
{
    return c && cls >= 0 && cls < PSW_TILE_CLASSES ? c->tile_policy[cls] : -1;
}

psw_status psw_profile_begin(psw_ctx *c)
{
    if (!c) return PSW_ERR_INVALID;
    c->recs.clear();
    c->evnext = 0;
    c->prof = true;
    return PSW_OK;
}

psw_status psw_profile_end(psw_ctx *c, psw_kernel_stat *out, int cap, int *n_out)
{
    if (!c) return PSW_ERR_INVALID;
    c->prof = false;
    CK_CUDA(c, cudaDeviceSynchronize());
    psw_kernel_stat tot[K_NCLASS];
    memset(tot, 0, sizeof(tot));
    for (int k = 0; k < K_NCLASS; k++) snprintf(tot[k].name, sizeof(tot[k].name), "%s", kclass_name[k]);
    for (const auto &r : c->recs) {
        float ms = 0.0f;
        CK_CUDA(c, cudaEventElapsedTime(&ms, r.a, r.b));
        tot[r.cls].launches++;
        tot[r.cls].ms += ms;
        tot[r.cls].flops += r.flops;
        tot[r.cls].bytes += r.bytes;
    }
    c->recs.clear();
    c->evnext = 0;
    int n = 0;
    for (int k = 0; k < K_NCLASS && n < cap; k++)
        if (tot[k].launches) out[n++] = tot[k];
    if (n_out) *n_out = n;
    return PSW_OK;
}

}  // extern "C"
