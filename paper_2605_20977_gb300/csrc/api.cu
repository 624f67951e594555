// api.cu -- the C ABI (include/psw.h): context and sequence lifetime, the
// encoder's masked parallel pass, the wavefront / raster decoder and the
// coder entry points.  Host code only enqueues kernels; every step of the
// model runs on the GPU.
#include "internal.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
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
struct Layout {
    long gamma_in, W_in, b_in, gamma_z, W_hp, b_hp;
    long gamma_c, W_c, b_c, pad, g_ctx;
    std::vector<BlockOff> ctx, sm1, sm2;
    long acc_g_q, acc_g_kv, acc_Wq, acc_Wk, acc_Wv, acc_Wo, acc_bias, acc_g_ffn, acc_Wg, acc_Wu, acc_Wd;
    long g_head, W1m, b1m, W2m, W1s, b1s, W2s, gamma_mu, beta_mu, gamma_sig, beta_sig;
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

Layout make_layout(const psw_model_desc &m)
{
    Layout y;
    Cursor cu;
    long dd = (long)m.d * m.d, kk = (long)m.k * m.k;
    y.gamma_in = cu.take(m.C); y.W_in = cu.take((long)m.C * m.d); y.b_in = cu.take(m.d);
    y.gamma_z = cu.take(m.Ch); y.W_hp = cu.take((long)m.r * m.r * m.Ch * m.d); y.b_hp = cu.take(m.d);
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
    y.g_head = cu.take(m.d);
    y.W1m = cu.take(dd); y.b1m = cu.take(m.d); y.W2m = cu.take((long)m.d * m.C);
    y.W1s = cu.take(dd); y.b1s = cu.take(m.d); y.W2s = cu.take((long)m.d * m.C);
    y.gamma_mu = cu.take(m.C); y.beta_mu = cu.take(m.C); y.gamma_sig = cu.take(m.C); y.beta_sig = cu.take(m.C);
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
    if (m->temporal) {
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

}  // namespace

struct psw_ctx {
    psw_model_desc md;
    int prec = 0;
    size_t budget = 0, bytes = 0, arena = 0;
    Layout lay;
    float *w = nullptr;                // flat FP32 weights on the device
    char *wmat = nullptr;              // arena of transposed projections
    std::vector<BlockDev> ctxb, sm1, sm2;
    BlockDev acc;                      // Wqkv = [Wq]; Wxkv = [Wk; Wv]
    CdfTables tabs{};
    uint32_t *d_cdf = nullptr;
    int *d_meta = nullptr;
    float *d_scale = nullptr;
    double *rate_buf = nullptr, *h_rate = nullptr;
    size_t rate_cap = 0;
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
    float *eh = nullptr, *x1 = nullptr, *x2 = nullptr, *g = nullptr;   // FP32 streams [HW][d]
    void *qa = nullptr;                                  // accumulator queries [HW][d]
    void *K1 = nullptr, *V1 = nullptr, *K2 = nullptr, *V2 = nullptr, *Ka = nullptr, *Va = nullptr;
    void *Xn = nullptr, *Q = nullptr, *O = nullptr, *Hid = nullptr;    // compact token buffers
    void *CK = nullptr, *CV = nullptr, *XK = nullptr, *XV = nullptr;   // temporal rings
    float *mu = nullptr, *sigma = nullptr;
    uint8_t *idx = nullptr;
    int32_t *m = nullptr;
    int16_t *y = nullptr, *yprev = nullptr;
    int frame = 0;
    uint32_t *rstate = nullptr, *rptr = nullptr, *rend = nullptr, *enc_nw = nullptr;
    uint16_t *enc_scratch = nullptr;
    uint64_t *enc_total = nullptr, *h_total = nullptr;
    int *d_status = nullptr, *h_status = nullptr;
    int *d_ident = nullptr, *d_order = nullptr;
    int sH = -1, sW = -1, sKind = -1, T = 0;
    std::vector<int> h_order, h_start;
    bool launch_failed = false;
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

// Kernel classes reported by psw_profile_end.
enum KClass { K_GEMM_TC, K_GEMM_SIMT, K_ATTN, K_NORM, K_EMBED, K_HEADS, K_RANS, K_OTHER, K_NCLASS };
const char *const kclass_name[K_NCLASS] = {"gemm_tc", "gemm_simt", "attention", "rmsnorm",
                                          "embed", "heads", "rans", "other"};

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

// Transposed ([out][in], K-major), compute-typed copies of every block
// projection, carved from one arena.  A dry run only sums the sizes.
bool prepare_projections(psw_ctx *c, bool dry)
{
    const psw_model_desc &m = c->md;
    const Layout &lay = c->lay;
    int d = m.d, prec = c->prec;
    size_t es = esize(prec), used = 0;
    auto carve = [&](size_t rows, size_t cols) -> void * {
        size_t sz = ((rows * cols * es + 255) / 256) * 256;
        void *p = dry ? nullptr : (void *)(c->wmat + used);
        used += sz;
        return p;
    };
    auto tr = [&](long off, int K, int N, void *dst, int row_off) {
        if (!dry) launch_transpose_convert(prec, c->w + off, K, N, dst, row_off, 0);
    };
    auto mk_block = [&](const BlockOff &bo, bool cross) {
        BlockDev b;
        b.Wqkv = carve(3 * d, d);
        tr(bo.Wq, d, d, b.Wqkv, 0); tr(bo.Wk, d, d, b.Wqkv, d); tr(bo.Wv, d, d, b.Wqkv, 2 * d);
        b.Wo = carve(d, d); tr(bo.Wo, d, d, b.Wo, 0);
        b.Wg = carve(m.F, d); tr(bo.Wg, d, m.F, b.Wg, 0);
        b.Wu = carve(m.F, d); tr(bo.Wu, d, m.F, b.Wu, 0);
        b.Wd = carve(d, m.F); tr(bo.Wd, m.F, d, b.Wd, 0);
        if (cross) {
            b.Wxq = carve(d, d); tr(bo.Wxq, d, d, b.Wxq, 0);
            b.Wxkv = carve(2 * d, d); tr(bo.Wxk, d, d, b.Wxkv, 0); tr(bo.Wxv, d, d, b.Wxkv, d);
            b.Wxo = carve(d, d); tr(bo.Wxo, d, d, b.Wxo, 0);
        }
        return b;
    };
    std::vector<BlockDev> ctxb, sm1, sm2;
    if (m.temporal)
        for (int l = 0; l < m.Lc; l++) ctxb.push_back(mk_block(lay.ctx[l], false));
    for (int l = 0; l < m.L; l++) sm1.push_back(mk_block(lay.sm1[l], m.temporal != 0));
    for (int l = 0; l < m.L; l++) sm2.push_back(mk_block(lay.sm2[l], m.temporal != 0));
    BlockDev ab;
    ab.Wqkv = carve(d, d); tr(lay.acc_Wq, d, d, ab.Wqkv, 0);
    ab.Wxkv = carve(2 * d, d); tr(lay.acc_Wk, d, d, ab.Wxkv, 0); tr(lay.acc_Wv, d, d, ab.Wxkv, d);
    ab.Wo = carve(d, d); tr(lay.acc_Wo, d, d, ab.Wo, 0);
    ab.Wg = carve(m.F, d); tr(lay.acc_Wg, d, m.F, ab.Wg, 0);
    ab.Wu = carve(m.F, d); tr(lay.acc_Wu, d, m.F, ab.Wu, 0);
    ab.Wd = carve(d, m.F); tr(lay.acc_Wd, m.F, d, ab.Wd, 0);
    if (dry) { c->arena = used; return true; }
    if (used > c->arena) return false;
    c->ctxb = ctxb; c->sm1 = sm1; c->sm2 = sm2; c->acc = ab;
    return true;
}

// Schedules: PSW_SCHED_WAVEFRONT = positions grouped by mask label in
// ascending label order (raster order inside a step), PSW_SCHED_RASTER =
// one position per step.  order: positions in schedule order; step t is
// order[start[t] .. start[t+1]).
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

// ---------------------------------------------------------------- model passes

struct Pass {
    psw_ctx *c;
    psw_seq *q;
    cudaStream_t s;
    int H, W;
    int HW() const { return H * W; }
};

size_t cache_stride(const Pass &P) { return (size_t)P.q->maxHW * P.c->md.d * esize(P.c->prec); }
void *cache_at(void *base, const Pass &P, long i) { return (char *)base + i * cache_stride(P); }

void gemm_call(const Pass &P, const void *A, int lda, const void *Wt, const void *Wt2, int M, int N, int K,
               const Epi &e)
{
    GemmArgs g{};
    g.A = A; g.lda = lda; g.Wt = Wt; g.Wt2 = Wt2; g.M = M; g.N = N; g.K = K; g.epi = e;
    g.status = P.q->d_status;
    if (M <= 0) return;
    bool tc = gemm_tc_supported(P.c->prec, N, K);
    double es = P.c->prec == P_BF16 ? 2.0 : 4.0, nw = Wt2 ? 2.0 : 1.0;
    double out_b = (e.mode == EPI_RESID || e.mode == EPI_RESID_BASE) ? 8.0 : es;
    Scope sc(P.c, P.s, tc ? K_GEMM_TC : K_GEMM_SIMT, 2.0 * nw * M * N * K,
             nw * N * K * es + (double)M * K * es + (double)M * N * out_b);
    if (!gemm(P.c->prec, g, P.s)) P.q->launch_failed = true;
}

Epi epi_qkv(const int *pos, int d, int q_cols, void *out, void *kc, void *vc)
{
    Epi e{};
    e.mode = EPI_QKV; e.pos = pos; e.d = d; e.q_cols = q_cols; e.out = out; e.ld_out = d; e.kc = kc; e.vc = vc;
    return e;
}
Epi epi_resid(const int *pos, float *x, const float *base = nullptr)
{
    Epi e{};
    e.mode = base ? EPI_RESID_BASE : EPI_RESID; e.pos = pos; e.resid = x; e.base = base;
    return e;
}
Epi epi_store(const int *pos, int scatter, void *out, int ld)
{
    Epi e{};
    e.mode = EPI_STORE; e.pos = pos; e.scatter = scatter; e.out = out; e.ld_out = ld;
    return e;
}
Epi epi_swiglu(void *out, int ld)
{
    Epi e{};
    e.mode = EPI_SWIGLU; e.out = out; e.ld_out = ld;
    return e;
}

#define LAUNCH(P_, cls, flops, bytes, call)                 \
    do {                                                    \
        Scope sc_((P_).c, (P_).s, (cls), (flops), (bytes)); \
        call;                                               \
    } while (0)

double attn_flops(const psw_model_desc &m, int n, double nkeys) { return 4.0 * n * nkeys * m.d; }
// mean visible keys: about half the window under the causal masks, all of it unmasked
double attn_keys(const AttnArgs &a) { return a.kind < 0 ? (double)a.nfr * a.k * a.k : 0.5 * a.k * a.k; }
double attn_bytes(const psw_model_desc &m, const AttnArgs &a)
{
    double es = 2.0;   // bf16 K/V rows; FP32 runs report the same algorithmic count
    return a.n * (double)m.d * es * (2.0 * attn_keys(a) + 2.0);
}

AttnArgs attn_args(const Pass &P, const int *pos, int n, const void *Qp, int q_full, const float *bias,
                   int bias_h_stride, int kind)
{
    AttnArgs a{};
    const psw_model_desc &m = P.c->md;
    a.pos = pos; a.n = n; a.Q = Qp; a.q_full = q_full;
    a.bias = bias; a.bias_h_stride = bias_h_stride;
    a.O = P.q->O; a.H = P.H; a.W = P.W; a.d = m.d; a.nh = m.nh; a.k = m.k; a.mask = m.mask; a.kind = kind;
    return a;
}

// SwiGLU feed-forward with pre-norm and residual (Sec. 3.1).
void ffn(const Pass &P, const BlockDev &bd, long g_ffn, float *x, const int *pos, int n)
{
    psw_ctx *c = P.c;
    psw_seq *q = P.q;
    const psw_model_desc &m = c->md;
    LAUNCH(P, K_NORM, 3.0 * n * m.d, n * m.d * 6.0, launch_rmsnorm(c->prec, pos, n, x, W(c, g_ffn), m.d, q->Xn, 0, P.s));
    gemm_call(P, q->Xn, m.d, bd.Wg, bd.Wu, n, m.F, m.d, epi_swiglu(q->Hid, m.F));
    gemm_call(P, q->Hid, m.F, bd.Wd, nullptr, n, m.d, m.F, epi_resid(pos, x));
}

// One spatial block (Sec. 3.1: RMSNorm pre-norm, window self-attention over
// S(p), temporal cross-attention for the temporal model, SwiGLU) on the
// positions pos[0..n).  x: residual stream [HW][d].  Kc/Vc: this block's
// window caches.  bidx: the block's index in the temporal K/V ring (SM1
// blocks 0..L-1, SM2 blocks L..2L-1).
void spatial_block(const Pass &P, const BlockOff &bo, const BlockDev &bd, int bidx, float *x, void *Kc,
                   void *Vc, const int *pos, int n)
{
    psw_ctx *c = P.c;
    psw_seq *q = P.q;
    const psw_model_desc &m = c->md;
    int d = m.d, kk = m.k * m.k;
    LAUNCH(P, K_NORM, 3.0 * n * d, n * d * 6.0, launch_rmsnorm(c->prec, pos, n, x, W(c, bo.g_attn), d, q->Xn, 0, P.s));
    gemm_call(P, q->Xn, d, bd.Wqkv, nullptr, n, 3 * d, d, epi_qkv(pos, d, d, q->Q, Kc, Vc));
    AttnArgs a = attn_args(P, pos, n, q->Q, 0, W(c, bo.bias), kk, 1);
    a.K[0] = Kc; a.V[0] = Vc; a.nfr = 1; a.age[0] = 0;
    LAUNCH(P, K_ATTN, attn_flops(m, a.n, attn_keys(a)), attn_bytes(m, a), launch_attention(c->prec, a, P.s));
    gemm_call(P, q->O, d, bd.Wo, nullptr, n, d, d, epi_resid(pos, x));
    if (m.temporal) {
        LAUNCH(P, K_NORM, 3.0 * n * d, n * d * 6.0, launch_rmsnorm(c->prec, pos, n, x, W(c, bo.g_x), d, q->Xn, 0, P.s));
        gemm_call(P, q->Xn, d, bd.Wxq, nullptr, n, d, d, epi_store(pos, 0, q->Q, d));
        AttnArgs xa = attn_args(P, pos, n, q->Q, 0, W(c, bo.xbias), m.Tf * kk, -1);
        int f = q->frame, f0 = std::max(0, f - m.Tf + 1);
        xa.nfr = f - f0 + 1;
        for (int ff = f0; ff <= f; ff++) {
            int u = ff - f0;
            xa.K[u] = cache_at(q->XK, P, (long)bidx * m.Tf + ff % m.Tf);
            xa.V[u] = cache_at(q->XV, P, (long)bidx * m.Tf + ff % m.Tf);
            xa.age[u] = f - ff;
        }
        LAUNCH(P, K_ATTN, attn_flops(m, xa.n, attn_keys(xa)), attn_bytes(m, xa), launch_attention(c->prec, xa, P.s));
        gemm_call(P, q->O, d, bd.Wxo, nullptr, n, d, d, epi_resid(pos, x));
    }
    ffn(P, bd, bo.g_ffn, x, pos, n);
}

// Per-frame preparation: hyperprior tokens and accumulator queries for
// every position (they depend only on the hyperlatents, Sec. 3.1), and for
// the temporal model the Context Transformer pass of this frame.
void frame_prologue(const Pass &P, const int16_t *zhat, const int16_t *yprev)
{
    psw_ctx *c = P.c;
    psw_seq *q = P.q;
    const psw_model_desc &m = c->md;
    int d = m.d, HW = P.HW(), Wh = (P.W + m.r - 1) / m.r, kk = m.k * m.k;
    LAUNCH(P, K_EMBED, 2.0 * HW * m.Ch * d, HW * (m.Ch * 2.0 + d * 4.0),
           launch_embed_hyper(zhat, P.H, P.W, Wh, m.Ch, m.r, W(c, c->lay.gamma_z), W(c, c->lay.W_hp),
                              W(c, c->lay.b_hp), d, q->eh, P.s));
    LAUNCH(P, K_NORM, 3.0 * HW * d, HW * d * 6.0, launch_rmsnorm(c->prec, nullptr, HW, q->eh, W(c, c->lay.acc_g_q), d, q->Xn, 0, P.s));
    gemm_call(P, q->Xn, d, c->acc.Wqkv, nullptr, HW, d, d, epi_store(nullptr, 0, q->qa, d));
    if (!m.temporal) return;
    // Context Transformer (Sec. 3.1): temporally shifted latents (learned
    // padding vector for frame 0), time-causal window attention over the
    // last Tf frames of each layer, final RMSNorm; then every spatial
    // block's cross-attention K/V of this frame.
    int f = q->frame, slot = f % m.Tf, f0 = std::max(0, f - m.Tf + 1);
    if (f == 0) LAUNCH(P, K_EMBED, 0.0, HW * d * 4.0, launch_fill_rows(W(c, c->lay.pad), HW, d, q->g, P.s));
    else LAUNCH(P, K_EMBED, 2.0 * HW * m.C * d, HW * (m.C * 2.0 + d * 4.0),
                launch_embed_latent(nullptr, HW, yprev, m.C, W(c, c->lay.gamma_c), W(c, c->lay.W_c),
                                    W(c, c->lay.b_c), d, q->g, P.s));
    for (int l = 0; l < m.Lc; l++) {
        const BlockOff &bo = c->lay.ctx[l];
        const BlockDev &bd = c->ctxb[l];
        LAUNCH(P, K_NORM, 3.0 * HW * d, HW * d * 6.0, launch_rmsnorm(c->prec, nullptr, HW, q->g, W(c, bo.g_attn), d, q->Xn, 0, P.s));
        gemm_call(P, q->Xn, d, bd.Wqkv, nullptr, HW, 3 * d, d,
                  epi_qkv(nullptr, d, d, q->Q, cache_at(q->CK, P, (long)l * m.Tf + slot),
                          cache_at(q->CV, P, (long)l * m.Tf + slot)));
        AttnArgs a = attn_args(P, nullptr, HW, q->Q, 0, W(c, bo.bias), m.Tf * kk, -1);
        a.nfr = f - f0 + 1;
        for (int ff = f0; ff <= f; ff++) {
            int u = ff - f0;
            a.K[u] = cache_at(q->CK, P, (long)l * m.Tf + ff % m.Tf);
            a.V[u] = cache_at(q->CV, P, (long)l * m.Tf + ff % m.Tf);
            a.age[u] = f - ff;
        }
        LAUNCH(P, K_ATTN, attn_flops(m, a.n, attn_keys(a)), attn_bytes(m, a), launch_attention(c->prec, a, P.s));
        gemm_call(P, q->O, d, bd.Wo, nullptr, HW, d, d, epi_resid(nullptr, q->g));
        ffn(P, bd, bo.g_ffn, q->g, nullptr, HW);
    }
    LAUNCH(P, K_NORM, 3.0 * HW * d, HW * d * 6.0, launch_rmsnorm(c->prec, nullptr, HW, q->g, W(c, c->lay.g_ctx), d, q->Xn, 0, P.s));
    for (int b = 0; b < 2 * m.L; b++) {
        const BlockDev &bd = b < m.L ? c->sm1[b] : c->sm2[b - m.L];
        gemm_call(P, q->Xn, d, bd.Wxkv, nullptr, HW, 2 * d, d,
                  epi_qkv(nullptr, d, 0, nullptr, cache_at(q->XK, P, (long)b * m.Tf + slot),
                          cache_at(q->XV, P, (long)b * m.Tf + slot)));
    }
}

// Spatial Module 1 on positions whose latents are known, then the
// accumulator keys/values from its normalised output (Sec. 3.1).
void run_sm1(const Pass &P, const int16_t *y, const int *pos, int n)
{
    psw_ctx *c = P.c;
    psw_seq *q = P.q;
    const psw_model_desc &m = c->md;
    int d = m.d;
    if (n <= 0) return;
    LAUNCH(P, K_EMBED, 2.0 * n * m.C * d, n * (m.C * 2.0 + d * 4.0),
           launch_embed_latent(pos, n, y, m.C, W(c, c->lay.gamma_in), W(c, c->lay.W_in), W(c, c->lay.b_in), d,
                               q->x1, P.s));
    for (int l = 0; l < m.L; l++)
        spatial_block(P, c->lay.sm1[l], c->sm1[l], l, q->x1, cache_at(q->K1, P, l), cache_at(q->V1, P, l), pos, n);
    LAUNCH(P, K_NORM, 3.0 * n * d, n * d * 6.0, launch_rmsnorm(c->prec, pos, n, q->x1, W(c, c->lay.acc_g_kv), d, q->Xn, 0, P.s));
    gemm_call(P, q->Xn, d, c->acc.Wxkv, nullptr, n, 2 * d, d, epi_qkv(pos, d, 0, nullptr, q->Ka, q->Va));
}

// Accumulator (hyperprior query and residual, keys/values over A(p)),
// Spatial Module 2 and heads on positions pos[0..n) (Sec. 3.1, Fig. 2b).
void run_acc_sm2_heads(const Pass &P, const int *pos, int n)
{
    psw_ctx *c = P.c;
    psw_seq *q = P.q;
    const psw_model_desc &m = c->md;
    int d = m.d;
    if (n <= 0) return;
    AttnArgs a = attn_args(P, pos, n, q->qa, 1, W(c, c->lay.acc_bias), m.k * m.k, 0);
    a.K[0] = q->Ka; a.V[0] = q->Va; a.nfr = 1; a.age[0] = 0;
    LAUNCH(P, K_ATTN, attn_flops(m, a.n, attn_keys(a)), attn_bytes(m, a), launch_attention(c->prec, a, P.s));
    gemm_call(P, q->O, d, c->acc.Wo, nullptr, n, d, d, epi_resid(pos, q->x2, q->eh));
    ffn(P, c->acc, c->lay.acc_g_ffn, q->x2, pos, n);
    for (int l = 0; l < m.L; l++)
        spatial_block(P, c->lay.sm2[l], c->sm2[l], m.L + l, q->x2, cache_at(q->K2, P, l), cache_at(q->V2, P, l), pos, n);
    HeadsArgs h{};
    h.pos = pos; h.n = n; h.x = q->x2; h.d = d; h.C = m.C;
    h.g = W(c, c->lay.g_head); h.W1m = W(c, c->lay.W1m); h.b1m = W(c, c->lay.b1m); h.W2m = W(c, c->lay.W2m);
    h.W1s = W(c, c->lay.W1s); h.b1s = W(c, c->lay.b1s); h.W2s = W(c, c->lay.W2s);
    h.gamma_mu = W(c, c->lay.gamma_mu); h.beta_mu = W(c, c->lay.beta_mu);
    h.gamma_sig = W(c, c->lay.gamma_sig); h.beta_sig = W(c, c->lay.beta_sig);
    h.scale = c->d_scale; h.mu = q->mu; h.sigma = q->sigma; h.idx = q->idx; h.m = q->m;
    LAUNCH(P, K_HEADS, 2.0 * n * (2.0 * d * d + 2.0 * d * m.C), n * (d * 4.0 + m.C * 13.0),
           launch_heads(h, P.s));
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

psw_status read_status(psw_ctx *c, psw_seq *q, cudaStream_t s, int *st_out)
{
    CK_CUDA(c, cudaMemcpyAsync(q->h_status, q->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK_CUDA(c, cudaStreamSynchronize(s));
    *st_out = *q->h_status;
    return PSW_OK;
}

size_t seq_bytes_for(const psw_model_desc &m, int prec, int H, int W_)
{
    size_t HW = (size_t)H * W_, d = m.d, es = esize(prec);
    size_t b = 0;
    b += 4 * HW * d * 4;                                            // eh, x1, x2, g
    b += HW * d * es;                                               // qa
    b += (4 * (size_t)m.L + 2) * HW * d * es;                       // K1 V1 K2 V2 Ka Va
    b += 3 * HW * d * es + HW * (size_t)m.F * es;                   // Xn Q O Hid
    if (m.temporal) b += 2 * ((size_t)m.Lc + 2 * (size_t)m.L) * m.Tf * HW * d * es;
    b += HW * m.C * (4 + 4 + 1 + 4 + 2 + 2);                        // mu sigma idx m y yprev
    b += (size_t)m.C * 32 * 4 + 2 * (size_t)m.C * 4 + (2 * (size_t)m.C + 1) * 4;
    b += (size_t)m.C * (3 * HW + 64) * 2;                           // encoder scratch
    b += 2 * HW * 4 + 64;
    return b;
}

// Encode the symbols y / idx / m ([HW][C], schedule order from the cached
// schedule) into a container; *len = its size.
psw_status encode_symbols(psw_ctx *c, psw_seq *q, const psw_frame_desc *fd, const int16_t *y, const uint8_t *idx,
                          const int32_t *m, uint8_t *bs, size_t cap, size_t *len, cudaStream_t s)
{
    int HW = fd->H * fd->W, C = c->md.C;
    int cap_words = 3 * HW + 64;
    {
        Scope sc(c, s, K_RANS, 0.0, (double)HW * C * 7.0);
        launch_rans_encode(coder(c), q->d_order, HW, C, y, idx, m, q->enc_scratch, cap_words, q->enc_nw, q->rstate, s);
    }
    Scope sc2(c, s, K_RANS, 0.0, (double)HW * C * 2.0);
    launch_rans_assemble(fd->H, fd->W, C, fd->schedule, q->enc_scratch, cap_words, q->enc_nw, q->rstate, bs, cap,
                         q->enc_total, q->d_status, s);
    CK_CUDA(c, cudaMemcpyAsync(q->h_total, q->enc_total, 8, cudaMemcpyDeviceToHost, s));
    CK_CUDA(c, cudaMemcpyAsync(q->h_status, q->d_status, 4, cudaMemcpyDeviceToHost, s));
    CK_CUDA(c, cudaStreamSynchronize(s));
    *len = (size_t)*q->h_total;
    if (*q->h_status & ST_CAPACITY) return fail(c, PSW_ERR_CAPACITY, "container needs %zu bytes, capacity %zu", *len, cap);
    return PSW_OK;
}

}  // namespace

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
    if (precision != PSW_FP32 && precision != PSW_BF16)
        return fail(nullptr, PSW_ERR_INVALID, "unknown precision %d", precision);
    Layout lay = make_layout(*desc);
    if (!weights_host || n_weights != (size_t)lay.total)
        return fail(nullptr, PSW_ERR_INVALID, "expected %ld weights, got %zu", lay.total, n_weights);
    if (precision == PSW_BF16 && !gemm_tc_available())
        return fail(nullptr, PSW_ERR_CUDA, "the driver offers no cuTensorMapEncodeTiled entry point");
    psw_ctx *c = new psw_ctx();
    c->md = *desc; c->prec = precision; c->budget = hbm_budget; c->lay = lay;
    prepare_projections(c, /*dry=*/true);
    build_cdf_tables(c->tabs);
    c->bytes = (size_t)lay.total * 4 + c->arena + (size_t)c->tabs.total * 4 + 3 * 64 * 4 + 64 * 4;
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
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_rate, sizeof(double));
    if (e != cudaSuccess) {
        psw_destroy(c);
        return fail(nullptr, PSW_ERR_OOM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
    int meta[3 * 64];
    for (int l = 0; l < 64; l++) { meta[l] = c->tabs.T[l]; meta[64 + l] = c->tabs.n[l]; meta[128 + l] = c->tabs.off[l]; }
    e = cudaMemcpy(c->w, weights_host, (size_t)lay.total * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_cdf, c->tabs.packed, (size_t)c->tabs.total * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_meta, meta, sizeof(meta), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_scale, c->tabs.scale, 64 * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !prepare_projections(c, /*dry=*/false)) e = cudaErrorInvalidValue;
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
    cudaFree(c->w); cudaFree(c->wmat); cudaFree(c->d_cdf); cudaFree(c->d_meta); cudaFree(c->d_scale);
    cudaFree(c->rate_buf);
    if (c->h_rate) cudaFreeHost(c->h_rate);
    for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
    free_cdf_tables(c->tabs);
    delete c;
}

psw_status psw_seq_create(psw_ctx *c, int max_H, int max_W, psw_seq **out)
{
    if (!c || !out) return fail(c, PSW_ERR_INVALID, "null argument");
    *out = nullptr;
    if (max_H < 1 || max_W < 1 || max_H > 4096 || max_W > 4096 || (long)max_H * max_W > (1L << 24))
        return fail(c, PSW_ERR_INVALID, "bad maximum grid %dx%d", max_H, max_W);
    size_t need = seq_bytes_for(c->md, c->prec, max_H, max_W);
    size_t used = c->bytes;
    for (psw_seq *s : c->seqs) used += s->bytes;
    if (c->budget && used + need > c->budget)
        return fail(c, PSW_ERR_OOM, "sequence needs %zu bytes; %zu of %zu in use", need, used, c->budget);
    psw_seq *q = new psw_seq();
    q->ctx = c; q->maxH = max_H; q->maxW = max_W; q->maxHW = max_H * max_W; q->bytes = need;
    const psw_model_desc &m = c->md;
    size_t HW = q->maxHW, d = m.d, es = esize(c->prec);
    bool okay = true;
    auto dal = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (!okay) return nullptr;
        if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) { okay = false; return nullptr; }
        q->allocs.push_back(p);
        return p;
    };
    q->eh = (float *)dal(HW * d * 4); q->x1 = (float *)dal(HW * d * 4); q->x2 = (float *)dal(HW * d * 4);
    q->g = (float *)dal(m.temporal ? HW * d * 4 : 16);
    q->qa = dal(HW * d * es);
    q->K1 = dal(m.L * HW * d * es); q->V1 = dal(m.L * HW * d * es);
    q->K2 = dal(m.L * HW * d * es); q->V2 = dal(m.L * HW * d * es);
    q->Ka = dal(HW * d * es); q->Va = dal(HW * d * es);
    q->Xn = dal(HW * d * es); q->Q = dal(HW * d * es); q->O = dal(HW * d * es); q->Hid = dal(HW * m.F * es);
    if (m.temporal) {
        q->CK = dal((size_t)m.Lc * m.Tf * HW * d * es); q->CV = dal((size_t)m.Lc * m.Tf * HW * d * es);
        q->XK = dal(2 * (size_t)m.L * m.Tf * HW * d * es); q->XV = dal(2 * (size_t)m.L * m.Tf * HW * d * es);
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
    q->d_ident = (int *)dal(HW * 4);
    if (okay && (cudaMallocHost(&q->h_total, 8) != cudaSuccess || cudaMallocHost(&q->h_status, 4) != cudaSuccess))
        okay = false;
    if (!okay) {
        psw_seq_destroy(q);
        return fail(c, PSW_ERR_OOM, "sequence allocation of %zu bytes failed", need);
    }
    std::vector<int> ident(HW);
    for (size_t p = 0; p < HW; p++) ident[p] = (int)p;
    cudaError_t e = cudaMemcpy(q->d_ident, ident.data(), HW * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(q->x1, 0, HW * d * 4);
    if (e == cudaSuccess) e = cudaMemset(q->x2, 0, HW * d * 4);
    if (e != cudaSuccess) {
        psw_seq_destroy(q);
        return fail(c, PSW_ERR_CUDA, "sequence initialisation: %s", cudaGetErrorString(e));
    }
    c->seqs.push_back(q);
    *out = q;
    return PSW_OK;
}

psw_status psw_seq_reset(psw_seq *q)
{
    if (!q) return PSW_ERR_INVALID;
    q->frame = 0;
    return PSW_OK;
}

void psw_seq_destroy(psw_seq *q)
{
    if (!q) return;
    for (void *p : q->allocs) cudaFree(p);
    if (q->h_total) cudaFreeHost(q->h_total);
    if (q->h_status) cudaFreeHost(q->h_status);
    if (q->ctx) {
        auto &v = q->ctx->seqs;
        for (size_t a = 0; a < v.size(); a++)
            if (v[a] == q) { v.erase(v.begin() + a); break; }
    }
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
    Pass P{c, q, s, fd->H, fd->W};
    CK_CUDA(c, cudaMemsetAsync(q->d_status, 0, 4, s));
    CK_CUDA(c, cudaMemcpyAsync(q->y, yhat_dev, nsym * 2, cudaMemcpyDeviceToDevice, s));
    frame_prologue(P, zhat_dev, q->yprev);
    // masked parallel pass over every position (Sec. 3.1, Sec. 3.2)
    run_sm1(P, q->y, q->d_ident, HW);
    run_acc_sm2_heads(P, q->d_ident, HW);
    if (mu_dev) CK_CUDA(c, cudaMemcpyAsync(mu_dev, q->mu, nsym * 4, cudaMemcpyDeviceToDevice, s));
    if (sigma_dev) CK_CUDA(c, cudaMemcpyAsync(sigma_dev, q->sigma, nsym * 4, cudaMemcpyDeviceToDevice, s));
    CK_CUDA(c, cudaGetLastError());
    if (len_out) *len_out = 0;
    if (bitstream_dev) st = encode_symbols(c, q, fd, q->y, q->idx, q->m, bitstream_dev, cap, len_out, s);
    // the sequence advances even if the container did not fit
    CK_CUDA(c, cudaMemcpyAsync(q->yprev, q->y, nsym * 2, cudaMemcpyDeviceToDevice, s));
    int dst = 0;
    psw_status st2 = read_status(c, q, s, &dst);
    q->frame++;
    if (st2) return st2;
    if (q->launch_failed) { q->launch_failed = false; return fail(c, PSW_ERR_CUDA, "a GEMM launch could not be prepared"); }
    if (dst & ST_TIMEOUT) return fail(c, PSW_ERR_TIMEOUT, "device wait timed out");
    return st;
}

psw_status psw_decode_frame(psw_ctx *c, psw_seq *q, const psw_frame_desc *fd, const uint8_t *bitstream_dev,
                            size_t len, const int16_t *zhat_dev, int16_t *yhat_out_dev, float *mu_dev,
                            float *sigma_dev, void *stream)
{
    psw_status st = check_frame(c, q, fd);
    if (st) return st;
    if (!bitstream_dev || !zhat_dev || !yhat_out_dev) return fail(c, PSW_ERR_INVALID, "null pointer argument");
    if ((uintptr_t)bitstream_dev & 3) return fail(c, PSW_ERR_INVALID, "bitstream must be 4-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = seq_schedule(q, fd->H, fd->W, fd->schedule))) return st;
    const psw_model_desc &m = c->md;
    int HW = fd->H * fd->W;
    size_t nsym = (size_t)HW * m.C;
    Pass P{c, q, s, fd->H, fd->W};
    CK_CUDA(c, cudaMemsetAsync(q->d_status, 0, 4, s));
    frame_prologue(P, zhat_dev, q->yprev);
    {
        Scope sc(c, s, K_RANS, 0.0, (double)m.C * 128.0);
        launch_rans_dec_init(bitstream_dev, len, fd->H, fd->W, m.C, fd->schedule, q->rstate, q->rptr, q->rend,
                             q->d_status, s);
    }
    const int *ord = q->d_order;
    for (int t = 0; t < q->T; t++) {
        int a0 = q->h_start[t], n = q->h_start[t + 1] - a0;
        if (t > 0) {
            int b0 = q->h_start[t - 1];
            run_sm1(P, q->y, ord + b0, a0 - b0);
        }
        run_acc_sm2_heads(P, ord + a0, n);
        Scope sc(c, s, K_RANS, 0.0, (double)n * m.C * 7.0 + (double)len * n / HW);
        launch_rans_dec_step(coder(c), ord, a0, n, m.C, q->idx, q->m, bitstream_dev, q->rstate, q->rptr, q->rend,
                             q->y, q->d_status, s);
    }
    {
        Scope sc(c, s, K_RANS, 0.0, (double)m.C * 128.0);
        launch_rans_dec_finish(bitstream_dev, m.C, q->rstate, q->rptr, q->rend, q->d_status, s);
    }
    CK_CUDA(c, cudaGetLastError());
    CK_CUDA(c, cudaMemcpyAsync(yhat_out_dev, q->y, nsym * 2, cudaMemcpyDeviceToDevice, s));
    if (mu_dev) CK_CUDA(c, cudaMemcpyAsync(mu_dev, q->mu, nsym * 4, cudaMemcpyDeviceToDevice, s));
    if (sigma_dev) CK_CUDA(c, cudaMemcpyAsync(sigma_dev, q->sigma, nsym * 4, cudaMemcpyDeviceToDevice, s));
    CK_CUDA(c, cudaMemcpyAsync(q->yprev, q->y, nsym * 2, cudaMemcpyDeviceToDevice, s));
    int dst = 0;
    if ((st = read_status(c, q, s, &dst))) return st;
    q->frame++;
    if (q->launch_failed) { q->launch_failed = false; return fail(c, PSW_ERR_CUDA, "a GEMM launch could not be prepared"); }
    if (dst & ST_CORRUPT) return fail(c, PSW_ERR_CORRUPT, "bitstream failed validation");
    if (dst & ST_TIMEOUT) return fail(c, PSW_ERR_TIMEOUT, "device wait timed out");
    return PSW_OK;
}

psw_status psw_decode_batch(psw_ctx *c, int n, psw_seq *const *seqs, const psw_frame_desc *fds,
                            const uint8_t *const *bitstreams_dev, const size_t *lens, const int16_t *const *zhat_dev,
                            int16_t *const *yhat_out_dev, int *status_out, void *stream)
{
    if (!c || n < 0 || (n > 0 && (!seqs || !fds || !bitstreams_dev || !lens || !zhat_dev || !yhat_out_dev)))
        return fail(c, PSW_ERR_INVALID, "bad batch arguments");
    psw_status first = PSW_OK;
    for (int a = 0; a < n; a++) {
        psw_status st = psw_decode_frame(c, seqs[a], &fds[a], bitstreams_dev[a], lens[a], zhat_dev[a],
                                         yhat_out_dev[a], nullptr, nullptr, stream);
        if (status_out) status_out[a] = st;
        if (st && !first) first = st;
    }
    return first;
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
    CK_CUDA(c, cudaMemsetAsync(q->d_status, 0, 4, s));
    return encode_symbols(c, q, fd, yhat_dev, idx_dev, m_dev, bitstream_dev, cap, len_out, s);
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
    CK_CUDA(c, cudaMemsetAsync(q->d_status, 0, 4, s));
    launch_rans_dec_init(bitstream_dev, len, fd->H, fd->W, C, fd->schedule, q->rstate, q->rptr, q->rend, q->d_status, s);
    for (int t = 0; t < q->T; t++) {
        int a0 = q->h_start[t], n = q->h_start[t + 1] - a0;
        launch_rans_dec_step(coder(c), q->d_order, a0, n, C, idx_dev, m_dev, bitstream_dev, q->rstate, q->rptr,
                             q->rend, yhat_out_dev, q->d_status, s);
    }
    launch_rans_dec_finish(bitstream_dev, C, q->rstate, q->rptr, q->rend, q->d_status, s);
    int dst = 0;
    if ((st = read_status(c, q, s, &dst))) return st;
    if (dst & ST_CORRUPT) return fail(c, PSW_ERR_CORRUPT, "bitstream failed validation");
    return PSW_OK;
}

long psw_launch_count(const psw_ctx *c) { return c ? c->launches : 0; }

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
