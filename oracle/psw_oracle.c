/*
 * psw_oracle.c -- plain FP64 CPU oracle for the P-SWA context model
 * ("Parallel Context Modeling for Sliding Window Attention in Neural Video
 * Coding", Kopte & Kaup).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Style: one position at a time, plain loops in a fixed order, double
 * precision, compiled with -ffp-contract=off.  Every position's arithmetic is
 * the same function of the same inputs whichever decoding schedule calls it,
 * so the masked parallel pass, the wavefront decode and the raster decode give
 * bit-identical parameters.
 *
 * Paper passages followed (section / figure of the paper):
 *   Sec. 3.1 (Overview, Fig. 1): Context Transformer with temporal shift and
 *     learned padding vector; Spatial Module 1 -> hyperprior -> accumulator
 *     (cross-attention, Q and residual from the hyperprior, K/V from Spatial
 *     Module 1 masked to strictly past positions) -> Spatial Module 2 ->
 *     prediction heads (two-layer MLPs for mu and sigma); SwiGLU + RMSNorm
 *     pre-norm blocks; channel-wise scaling at the input and outputs.
 *   Sec. 3.2 (Parallel decoding, Fig. 2): step labels; the accumulator sees
 *     labels strictly below its own, spatial self-attention also sees
 *     positions of the same step; 2D windows.
 *   Sec. 4.1: 7x7 spatial windows, T x 7 x 7 temporal windows.
 *   Fig. 1 (right): Q / AE / AD -- realised here as a Gaussian scale table,
 *     integer CDF tables and interleaved rANS (the paper names no coder);
 *     the convolutional hyperprior (down- and upsampling residual blocks,
 *     z-hat coded under a factorized prior).
 *   Sec. 3.1 (Channel Transformer paragraph), Sec. 3.2 (s spatial steps
 *     times N channel groups), Sec. 4.1 (N = 4, width 1024, 2 blocks).
 *   Sec. 3.1 (LRP paragraph), Sec. 4.3 (time-causal LRP Transformer).
 *
 * Readings of silent points (each is listed in the design notes):
 *   - step label l(i,j) = 2i+j with an extra raster clause rho(q) < rho(p) in
 *     both masks, so raster order is also a valid schedule; the cyclic
 *     s = 4 label ((i mod 4)+(j mod 4)) mod 4 (Fig. 2a) without that clause;
 *   - softmax over an empty key set is 0;
 *   - RMSNorm eps 1e-6; sigma = exp(clamp(s, ln 0.11, ln 256));
 *   - per-head relative position bias tables over the window;
 *   - out-of-frame positions are absent (clipped windows, no padding tokens).
 *
 * Parity pins (see tests/test_oracle_*.py): closed forms for RMSNorm, SiLU,
 * SwiGLU, attention special cases and the quantised-Gaussian likelihood;
 * the Fig. 2b receptive field transcribed by hand; brute-force causality;
 * schedule equivalence; rANS round trips and CDF invariants; E4M3 rounding
 * against hand values of the format and a library cast.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Configuration and weight layout                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int H, W, C;          /* latent grid and channels                       */
    int Hh, Wh, Ch, r;    /* hyperprior grid, channels, upsampling factor    */
    int d, nh, F, L, k;   /* width, heads, FFN width, blocks/module, window  */
    int temporal;         /* 1: Context Transformer + temporal cross-attn    */
    int Lc, Tf;           /* Context Transformer blocks, frames in window    */
    int mask;             /* 0: l = 2i+j (+ raster clause); 1: cyclic s = 4  */
    int Llrp;             /* LRP Transformer blocks (0: none)                */
    int Nc, dc, Lct, Fc;  /* Channel Transformer: groups (0: none), width,
                             blocks, SwiGLU width per group                */
    int hp;               /* 1: convolutional hyperprior (RB blocks) with a
                             factorized prior for z; 0: z given, embedded
                             by a transposed convolution                   */
} or_cfg;

typedef struct {
    long g_attn, Wq, Wk, Wv, Wo, bias;
    long g_x, Wxq, Wxk, Wxv, Wxo, xbias;   /* -1 when absent */
    long g_ffn, Wg, Wu, Wd;
} or_blk;

typedef struct {
    long g_q, g_kv, Wq, Wk, Wv, Wo, bias, g_ffn, Wg, Wu, Wd;
} or_accw;

#define OR_MAXL 64

/* A down- or upsampling residual block of the hyperprior (Fig. 1 right). */
typedef struct {
    long Wa, ba, Wb, bb, Ws, bs;
} or_rb;

#define OR_MAXRB 4

typedef struct {
    long gamma_in, W_in, b_in;
    long gamma_z, W_hp, b_hp;
    long g_za;                                   /* hyperprior analysis input gain */
    or_rb rbd[OR_MAXRB], rbu[OR_MAXRB];          /* analysis / synthesis blocks    */
    long fp_H1, fp_b1, fp_a1, fp_H2, fp_b2, fp_a2, fp_H3, fp_b3, fp_a3, fp_H4, fp_b4;   /* factorized prior */
    long gamma_c, W_c, b_c, pad, g_ctx;
    or_blk ctx[OR_MAXL], sm1[OR_MAXL], sm2[OR_MAXL];
    or_accw acc;
    long g_head, W1m, b1m, W2m, W1s, b1s, W2s;
    long gamma_mu, beta_mu, gamma_sig, beta_sig;
    long lrp_g_rep, lrp_W_rep, lrp_gamma_y, lrp_W_y, lrp_b_in;   /* LRP Transformer (-1: none) */
    or_blk lrp[OR_MAXL];
    long lrp_g_out, lrp_W_eps, lrp_b_eps;
    long ct_g_in, ct_W_in, ct_b_in, ct_gamma_y, ct_E;   /* Channel Transformer (-1: none) */
    long ct_g_mix[OR_MAXL], ct_M[OR_MAXL], ct_g_ffn[OR_MAXL], ct_Wg[OR_MAXL], ct_Wu[OR_MAXL], ct_Wd[OR_MAXL];
    long total;
} or_layout;

static long take(long *cur, long n) { long o = *cur; *cur += n; return o; }

/* Residual blocks per hyperprior transform: log2 r (each halves or
 * doubles the grid); -1 if r is not a power of two in [2, 16]. */
int or_hyper_blocks(const or_cfg *c)
{
    for (int b = 1; b <= OR_MAXRB; b++)
        if (c->r == (1 << b)) return b;
    return -1;
}

/* Packing order of the flat weight vector (all matrices are [in][out], used
 * as x . W).  The order is an interface, documented with the C-ABI. */
static void layout_block(long *cur, const or_cfg *c, or_blk *b, int cross, int tf_bias)
{
    long dd = (long)c->d * c->d, kk = (long)c->k * c->k;
    b->g_attn = take(cur, c->d);
    b->Wq = take(cur, dd); b->Wk = take(cur, dd); b->Wv = take(cur, dd); b->Wo = take(cur, dd);
    b->bias = take(cur, (long)c->nh * (tf_bias ? c->Tf : 1) * kk);
    if (cross) {
        b->g_x = take(cur, c->d);
        b->Wxq = take(cur, dd); b->Wxk = take(cur, dd); b->Wxv = take(cur, dd); b->Wxo = take(cur, dd);
        b->xbias = take(cur, (long)c->nh * c->Tf * kk);
    } else {
        b->g_x = b->Wxq = b->Wxk = b->Wxv = b->Wxo = b->xbias = -1;
    }
    b->g_ffn = take(cur, c->d);
    b->Wg = take(cur, (long)c->d * c->F); b->Wu = take(cur, (long)c->d * c->F);
    b->Wd = take(cur, (long)c->F * c->d);
}

static void make_layout(const or_cfg *c, or_layout *lay)
{
    long cur = 0, dd = (long)c->d * c->d, kk = (long)c->k * c->k;
    memset(lay, 0, sizeof(*lay));
    lay->gamma_in = take(&cur, c->C);
    lay->W_in = take(&cur, (long)c->C * c->d);
    lay->b_in = take(&cur, c->d);
    lay->gamma_z = take(&cur, c->Ch);
    if (c->hp) {
        int nb = or_hyper_blocks(c);
        long Ch = c->Ch;
        lay->W_hp = lay->b_hp = -1;
        lay->g_za = take(&cur, c->d);
        for (int b = 0; b < nb; b++) {          /* analysis: d -> Ch, then Ch -> Ch */
            long Ci = b == 0 ? c->d : Ch, Co = Ch;
            lay->rbd[b].Wa = take(&cur, 9 * Ci * Co); lay->rbd[b].ba = take(&cur, Co);
            lay->rbd[b].Wb = take(&cur, 9 * Co * Co); lay->rbd[b].bb = take(&cur, Co);
            lay->rbd[b].Ws = take(&cur, Ci * Co); lay->rbd[b].bs = take(&cur, Co);
        }
        for (int b = 0; b < nb; b++) {          /* synthesis: Ch -> Ch, last Ch -> d */
            long Ci = Ch, Co = b == nb - 1 ? c->d : Ch;
            lay->rbu[b].Wa = take(&cur, 9 * Ci * 4 * Co); lay->rbu[b].ba = take(&cur, 4 * Co);
            lay->rbu[b].Wb = take(&cur, 9 * Co * Co); lay->rbu[b].bb = take(&cur, Co);
            lay->rbu[b].Ws = take(&cur, 9 * Ci * 4 * Co); lay->rbu[b].bs = take(&cur, 4 * Co);
        }
        lay->fp_H1 = take(&cur, Ch * 3); lay->fp_b1 = take(&cur, Ch * 3); lay->fp_a1 = take(&cur, Ch * 3);
        lay->fp_H2 = take(&cur, Ch * 9); lay->fp_b2 = take(&cur, Ch * 3); lay->fp_a2 = take(&cur, Ch * 3);
        lay->fp_H3 = take(&cur, Ch * 9); lay->fp_b3 = take(&cur, Ch * 3); lay->fp_a3 = take(&cur, Ch * 3);
        lay->fp_H4 = take(&cur, Ch * 3); lay->fp_b4 = take(&cur, Ch);
    } else {
        lay->W_hp = take(&cur, (long)c->r * c->r * c->Ch * c->d);
        lay->b_hp = take(&cur, c->d);
        lay->g_za = -1;
    }
    if (c->temporal) {
        lay->gamma_c = take(&cur, c->C);
        lay->W_c = take(&cur, (long)c->C * c->d);
        lay->b_c = take(&cur, c->d);
        lay->pad = take(&cur, c->d);
        for (int l = 0; l < c->Lc; l++) layout_block(&cur, c, &lay->ctx[l], 0, 1);
        lay->g_ctx = take(&cur, c->d);
    } else {
        lay->gamma_c = lay->W_c = lay->b_c = lay->pad = lay->g_ctx = -1;
    }
    for (int l = 0; l < c->L; l++) layout_block(&cur, c, &lay->sm1[l], c->temporal, 0);
    lay->acc.g_q = take(&cur, c->d);
    lay->acc.g_kv = take(&cur, c->d);
    lay->acc.Wq = take(&cur, dd); lay->acc.Wk = take(&cur, dd);
    lay->acc.Wv = take(&cur, dd); lay->acc.Wo = take(&cur, dd);
    lay->acc.bias = take(&cur, (long)c->nh * kk);
    lay->acc.g_ffn = take(&cur, c->d);
    lay->acc.Wg = take(&cur, (long)c->d * c->F); lay->acc.Wu = take(&cur, (long)c->d * c->F);
    lay->acc.Wd = take(&cur, (long)c->F * c->d);
    for (int l = 0; l < c->L; l++) layout_block(&cur, c, &lay->sm2[l], c->temporal, 0);
    int dh = c->Nc > 0 ? c->dc : c->d;     /* width of the heads' input */
    if (c->Nc > 0) {
        long dg = c->dc / c->Nc, Cg = c->C / c->Nc, dc = c->dc;
        lay->ct_g_in = take(&cur, c->d);
        lay->ct_W_in = take(&cur, (long)c->d * dc);
        lay->ct_b_in = take(&cur, dc);
        lay->ct_gamma_y = take(&cur, c->C);
        lay->ct_E = take(&cur, (long)(c->Nc - 1) * Cg * dg);
        for (int l = 0; l < c->Lct; l++) {
            lay->ct_g_mix[l] = take(&cur, dc);
            lay->ct_M[l] = take(&cur, dc * dc);
            lay->ct_g_ffn[l] = take(&cur, dc);
            lay->ct_Wg[l] = take(&cur, (long)c->Nc * dg * c->Fc);
            lay->ct_Wu[l] = take(&cur, (long)c->Nc * dg * c->Fc);
            lay->ct_Wd[l] = take(&cur, (long)c->Nc * c->Fc * dg);
        }
        /* grouped heads: per group [dg][dg] and [dg][Cg] */
        lay->g_head = take(&cur, dc);
        lay->W1m = take(&cur, (long)c->Nc * dg * dg); lay->b1m = take(&cur, dc);
        lay->W2m = take(&cur, (long)c->Nc * dg * Cg);
        lay->W1s = take(&cur, (long)c->Nc * dg * dg); lay->b1s = take(&cur, dc);
        lay->W2s = take(&cur, (long)c->Nc * dg * Cg);
    } else {
        lay->ct_g_in = lay->ct_W_in = lay->ct_b_in = lay->ct_gamma_y = lay->ct_E = -1;
        lay->g_head = take(&cur, c->d);
        lay->W1m = take(&cur, dd); lay->b1m = take(&cur, c->d); lay->W2m = take(&cur, (long)c->d * c->C);
        lay->W1s = take(&cur, dd); lay->b1s = take(&cur, c->d); lay->W2s = take(&cur, (long)c->d * c->C);
    }
    lay->gamma_mu = take(&cur, c->C); lay->beta_mu = take(&cur, c->C);
    lay->gamma_sig = take(&cur, c->C); lay->beta_sig = take(&cur, c->C);
    if (c->Llrp > 0) {
        lay->lrp_g_rep = take(&cur, dh);
        lay->lrp_W_rep = take(&cur, (long)dh * c->d);
        lay->lrp_gamma_y = take(&cur, c->C);
        lay->lrp_W_y = take(&cur, (long)c->C * c->d);
        lay->lrp_b_in = take(&cur, c->d);
        for (int l = 0; l < c->Llrp; l++) layout_block(&cur, c, &lay->lrp[l], 0, c->temporal != 0);
        lay->lrp_g_out = take(&cur, c->d);
        lay->lrp_W_eps = take(&cur, (long)c->d * c->C);
        lay->lrp_b_eps = take(&cur, c->C);
    } else {
        lay->lrp_g_rep = lay->lrp_W_rep = lay->lrp_gamma_y = lay->lrp_W_y = lay->lrp_b_in = -1;
        lay->lrp_g_out = lay->lrp_W_eps = lay->lrp_b_eps = -1;
    }
    lay->total = cur;
}

long or_weights_count(const or_cfg *c)
{
    or_layout lay;
    if (c->L > OR_MAXL || c->Lc > OR_MAXL || c->Llrp > OR_MAXL || c->Lct > OR_MAXL) return -1;
    if (c->hp && or_hyper_blocks(c) < 0) return -1;
    make_layout(c, &lay);
    return lay.total;
}

/* ------------------------------------------------------------------------ */
/* Elementary operations (Sec. 3.1: RMSNorm pre-norm, SwiGLU, attention)      */
/* ------------------------------------------------------------------------ */

#define OR_EPS 1e-6

/* RMSNorm: y = x / sqrt(mean(x^2) + eps) * g. */
void or_rmsnorm(const double *x, const double *g, int d, double *y)
{
    double ss = 0.0;
    for (int i = 0; i < d; i++) ss += x[i] * x[i];
    double inv = 1.0 / sqrt(ss / (double)d + OR_EPS);
    for (int i = 0; i < d; i++) y[i] = x[i] * inv * g[i];
}

/* y[o] = sum_i x[i] W[i][o], summed in ascending i. */
void or_matvec(const double *x, const double *W, int n_in, int n_out, double *y)
{
    for (int o = 0; o < n_out; o++) y[o] = 0.0;
    for (int i = 0; i < n_in; i++) {
        const double xi = x[i];
        const double *row = W + (long)i * n_out;
        for (int o = 0; o < n_out; o++) y[o] += xi * row[o];
    }
}

double or_silu(double x) { return x / (1.0 + exp(-x)); }

/* SwiGLU feed-forward: out = (SiLU(x Wg) * (x Wu)) Wd.  x already normed. */
void or_swiglu(const double *x, const double *Wg, const double *Wu, const double *Wd,
               int d, int F, double *out)
{
    double *g = (double *)malloc(sizeof(double) * F);
    double *u = (double *)malloc(sizeof(double) * F);
    or_matvec(x, Wg, d, F, g);
    or_matvec(x, Wu, d, F, u);
    for (int f = 0; f < F; f++) g[f] = or_silu(g[f]) * u[f];
    or_matvec(g, Wd, F, d, out);
    free(g); free(u);
}

/* Multi-head attention of one query over an explicit key list.
 * q: [d]; K[j], V[j]: pointers to [d] rows; bias: [nkeys][nh].
 * Per head: s_j = q_h.K_jh / sqrt(dh) + bias_jh; p = softmax(s) (max
 * subtracted, sums in ascending j); out_h = sum_j p_j V_jh.
 * An empty key list gives 0 (softmax over the empty set taken as 0). */
void or_attend(const double *q, int nkeys, const double *const *K, const double *const *V,
               const double *bias, int nh, int d, double *out)
{
    int dh = d / nh;
    double scale = 1.0 / sqrt((double)dh);
    double *s = (double *)malloc(sizeof(double) * (nkeys > 0 ? nkeys : 1));
    for (int h = 0; h < nh; h++) {
        double *o = out + h * dh;
        for (int e = 0; e < dh; e++) o[e] = 0.0;
        if (nkeys == 0) continue;
        double mx = -INFINITY;
        for (int j = 0; j < nkeys; j++) {
            double acc = 0.0;
            const double *kj = K[j] + h * dh;
            for (int e = 0; e < dh; e++) acc += q[h * dh + e] * kj[e];
            s[j] = acc * scale + bias[(long)j * nh + h];
            if (s[j] > mx) mx = s[j];
        }
        double z = 0.0;
        for (int j = 0; j < nkeys; j++) { s[j] = exp(s[j] - mx); z += s[j]; }
        for (int j = 0; j < nkeys; j++) {
            double p = s[j] / z;
            const double *vj = V[j] + h * dh;
            for (int e = 0; e < dh; e++) o[e] += p * vj[e];
        }
    }
    free(s);
}

/* ------------------------------------------------------------------------ */
/* Step labels and masks (Sec. 3.2, Fig. 2)                                  */
/* ------------------------------------------------------------------------ */

int or_label(int mask, int i, int j)
{
    if (mask == 1) return ((i % 4) + (j % 4)) % 4;   /* Fig. 2a, minus 1 */
    return 2 * i + j;                               /* single diagonal wavefront */
}

/* Accumulator set A(p): window positions with a strictly smaller label (and,
 * for the 2i+j mask, a smaller raster index).  kind 0 = A, 1 = S (spatial
 * self-attention: p itself plus window positions with label <= l(p)). */
int or_visible(int mask, int kind, int W, int pi, int pj, int qi, int qj)
{
    if (kind == 1 && qi == pi && qj == pj) return 1;
    int lp = or_label(mask, pi, pj), lq = or_label(mask, qi, qj);
    int ok = (kind == 0) ? (lq < lp) : (lq <= lp);
    if (mask == 0) ok = ok && ((long)qi * W + qj < (long)pi * W + pj);
    return ok;
}

/* Keys of position p under mask kind, ascending raster order.  Returns the
 * count; idx receives raster indices, off receives window offsets
 * (di + w) * k + (dj + w). */
int or_window_keys(const or_cfg *c, int kind, int p, int *idx, int *off)
{
    int w = (c->k - 1) / 2, pi = p / c->W, pj = p % c->W, n = 0;
    for (int di = -w; di <= w; di++) {
        int qi = pi + di;
        if (qi < 0 || qi >= c->H) continue;
        for (int dj = -w; dj <= w; dj++) {
            int qj = pj + dj;
            if (qj < 0 || qj >= c->W) continue;
            if (kind >= 0 && !or_visible(c->mask, kind, c->W, pi, pj, qi, qj)) continue;
            idx[n] = qi * c->W + qj;
            off[n] = (di + w) * c->k + (dj + w);
            n++;
        }
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Model state                                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    const or_cfg *c;
    const double *w;
    or_layout lay;
    int HW;
    int frame;            /* index of the frame being coded                 */
    double *x1, *K1, *V1; /* SM1 residual stream, per-layer keys/values      */
    double *eh, *Ka, *Va; /* hyperprior tokens, accumulator keys/values      */
    double *x2, *K2, *V2; /* SM2 residual stream, per-layer keys/values      */
    double *q;            /* per-position query scratch                      */
    double *XK, *XV;      /* temporal cross K/V: [2L][Tf slots][HW][d]        */
    double *CK, *CV;      /* context transformer K/V: [Lc][Tf slots][HW][d]   */
    double *LK, *LV;      /* LRP Transformer K/V: [Llrp][Tf slots][HW][d]    */
    double *xc;           /* Channel Transformer output per position [HW][dc] */
    double *ctM[OR_MAXL]; /* its mixing matrices with the block mask applied */
    double *mu, *sigma;   /* [HW][C]                                        */
} or_state;

static double *zalloc(long n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

static int state_init(or_state *s, const or_cfg *c, const double *w)
{
    memset(s, 0, sizeof(*s));
    s->c = c; s->w = w; s->HW = c->H * c->W;
    make_layout(c, &s->lay);
    long hd = (long)s->HW * c->d;
    s->x1 = zalloc(hd); s->K1 = zalloc(hd * c->L); s->V1 = zalloc(hd * c->L);
    s->eh = zalloc(hd); s->Ka = zalloc(hd); s->Va = zalloc(hd);
    s->x2 = zalloc(hd); s->K2 = zalloc(hd * c->L); s->V2 = zalloc(hd * c->L);
    s->q = zalloc(hd);
    s->mu = zalloc((long)s->HW * c->C); s->sigma = zalloc((long)s->HW * c->C);
    if (c->temporal) {
        s->XK = zalloc(hd * 2 * c->L * c->Tf); s->XV = zalloc(hd * 2 * c->L * c->Tf);
        s->CK = zalloc(hd * c->Lc * c->Tf); s->CV = zalloc(hd * c->Lc * c->Tf);
    }
    if (c->Llrp > 0) {
        s->LK = zalloc(hd * c->Llrp * c->Tf); s->LV = zalloc(hd * c->Llrp * c->Tf);
    }
    if (c->Nc > 0) {
        /* the block-lower-triangular mask on each mixing matrix [in][out]:
         * output group i keeps the rows of input groups 0..i */
        int dc = c->dc, dg = c->dc / c->Nc;
        s->xc = zalloc((long)s->HW * dc);
        for (int l = 0; l < c->Lct; l++) {
            s->ctM[l] = zalloc((long)dc * dc);
            const double *M = w + s->lay.ct_M[l];
            for (int i = 0; i < dc; i++)
                for (int o = 0; o < dc; o++)
                    s->ctM[l][(long)i * dc + o] = (i / dg <= o / dg) ? M[(long)i * dc + o] : 0.0;
        }
    }
    return (s->x1 && s->K1 && s->V1 && s->eh && s->Ka && s->Va && s->x2 && s->K2 && s->V2 &&
            s->q && s->mu && s->sigma) ? 0 : -1;
}

static void state_free(or_state *s)
{
    free(s->x1); free(s->K1); free(s->V1); free(s->eh); free(s->Ka); free(s->Va);
    free(s->x2); free(s->K2); free(s->V2); free(s->q); free(s->mu); free(s->sigma);
    free(s->XK); free(s->XV); free(s->CK); free(s->CV); free(s->LK); free(s->LV);
    free(s->xc);
    for (int l = 0; l < s->c->Lct; l++) free(s->ctM[l]);
}

#define WP(off) (s->w + (off))

/* Token embedding of a latent vector (Sec. 3.1: channel-wise input scaling
 * followed by a linear projection to the model width). */
static void embed_latent(const or_state *s, const int16_t *yv, long g_off, long W_off, long b_off,
                         double *out)
{
    const or_cfg *c = s->c;
    double *t = zalloc(c->C);
    for (int ch = 0; ch < c->C; ch++) t[ch] = WP(g_off)[ch] * (double)yv[ch];
    or_matvec(t, WP(W_off), c->C, c->d, out);
    for (int e = 0; e < c->d; e++) out[e] += WP(b_off)[e];
    free(t);
}

/* Hyperprior tokens (Sec. 3.1, Fig. 1 right: the decoded hyperprior enters
 * the transformer as the accumulator's query and residual).  A transposed
 * convolution with kernel = stride = r: the hyperpixel above (i, j) times the
 * sub-position weight (i mod r, j mod r), plus a bias. */
static void hyper_synthesis(or_state *s, const int16_t *zhat);

static void embed_hyper(or_state *s, const int16_t *zhat)
{
    const or_cfg *c = s->c;
    if (c->hp) { hyper_synthesis(s, zhat); return; }
    for (int p = 0; p < s->HW; p++) {
        int i = p / c->W, j = p % c->W;
        const int16_t *zv = zhat + ((long)(i / c->r) * c->Wh + (j / c->r)) * c->Ch;
        double *t = zalloc(c->Ch);
        for (int ch = 0; ch < c->Ch; ch++) t[ch] = WP(s->lay.gamma_z)[ch] * (double)zv[ch];
        int sub = (i % c->r) * c->r + (j % c->r);
        double *o = s->eh + (long)p * c->d;
        or_matvec(t, WP(s->lay.W_hp) + (long)sub * c->Ch * c->d, c->Ch, c->d, o);
        for (int e = 0; e < c->d; e++) o[e] += WP(s->lay.b_hp)[e];
        free(t);
    }
}

/* ------------------------------------------------------------------------ */
/* Convolutional hyperprior (Fig. 1 right: RB-down x2 -> z -> Q -> AE/AD      */
/* with a factorized prior -> z-hat -> RB-up x2)                              */
/* ------------------------------------------------------------------------ */
/* Grids are channel-last [h][w][C].  The residual blocks follow the down-
 * and upsampling residual blocks of DCVC-DC that the paper cites: a strided
 * (or sub-pixel) 3x3 convolution and LeakyReLU, a 3x3 convolution, and a
 * strided 1x1 (or sub-pixel 3x3) convolution on the skip path. */

static double or_lrelu(double x) { return x >= 0.0 ? x : 0.01 * x; }

/* 3x3 convolution, zero padding 1, stride st: out [ho][wo][Co] with
 * ho = ceil(h / st); W [3][3][Ci][Co]; taps and input channels summed in
 * ascending order after the bias. */
static void or_conv3(const double *x, int h, int w, int Ci, const double *W, const double *b, int Co, int st,
                     double *out)
{
    int ho = (h - 1) / st + 1, wo = (w - 1) / st + 1;
    for (int i = 0; i < ho; i++)
        for (int j = 0; j < wo; j++) {
            double *o = out + ((long)i * wo + j) * Co;
            for (int q = 0; q < Co; q++) o[q] = b[q];
            for (int di = 0; di < 3; di++)
                for (int dj = 0; dj < 3; dj++) {
                    int ii = st * i + di - 1, jj = st * j + dj - 1;
                    if (ii < 0 || ii >= h || jj < 0 || jj >= w) continue;
                    const double *xv = x + ((long)ii * w + jj) * Ci;
                    const double *Wt = W + (long)(di * 3 + dj) * Ci * Co;
                    for (int c = 0; c < Ci; c++)
                        for (int q = 0; q < Co; q++) o[q] += xv[c] * Wt[(long)c * Co + q];
                }
        }
}

/* 1x1 convolution with stride 2: out [ceil(h/2)][ceil(w/2)][Co]. */
static void or_conv1s2(const double *x, int h, int w, int Ci, const double *W, const double *b, int Co, double *out)
{
    int ho = (h + 1) / 2, wo = (w + 1) / 2;
    for (int i = 0; i < ho; i++)
        for (int j = 0; j < wo; j++) {
            double *o = out + ((long)i * wo + j) * Co;
            const double *xv = x + ((long)(2 * i) * w + 2 * j) * Ci;
            for (int q = 0; q < Co; q++) o[q] = b[q];
            for (int c = 0; c < Ci; c++)
                for (int q = 0; q < Co; q++) o[q] += xv[c] * W[(long)c * Co + q];
        }
}

/* Pixel shuffle by 2: u [h][w][4C] -> v [2h][2w][C],
 * v[2i + a][2j + b][c] = u[i][j][(2a + b) C + c]. */
static void or_shuffle(const double *u, int h, int w, int C, double *v)
{
    for (int i = 0; i < h; i++)
        for (int j = 0; j < w; j++)
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++)
                    for (int c = 0; c < C; c++)
                        v[((long)(2 * i + a) * 2 * w + 2 * j + b) * C + c] = u[((long)i * w + j) * 4 * C + (2 * a + b) * C + c];
}

/* RB-down: out = conv3(LReLU(conv3_s2(x) + ba)) + bb + (conv1_s2(x) + bs). */
static double *or_rb_down(const or_state *s, const or_rb *rb, const double *x, int h, int w, int Ci, int Co)
{
    int ho = (h + 1) / 2, wo = (w + 1) / 2;
    long n = (long)ho * wo * Co;
    double *a = zalloc(n), *t = zalloc(n), *k = zalloc(n);
    or_conv3(x, h, w, Ci, WP(rb->Wa), WP(rb->ba), Co, 2, a);
    for (long e = 0; e < n; e++) a[e] = or_lrelu(a[e]);
    or_conv3(a, ho, wo, Co, WP(rb->Wb), WP(rb->bb), Co, 1, t);
    or_conv1s2(x, h, w, Ci, WP(rb->Ws), WP(rb->bs), Co, k);
    for (long e = 0; e < n; e++) t[e] += k[e];
    free(a); free(k);
    return t;
}

/* RB-up: out = conv3(LReLU(shuffle(conv3(x) + ba))) + bb
 *              + shuffle(conv3(x) + bs) (sub-pixel convolutions). */
static double *or_rb_up(const or_state *s, const or_rb *rb, const double *x, int h, int w, int Ci, int Co)
{
    long nl = (long)h * w * 4 * Co, n = nl;
    double *u = zalloc(nl), *a = zalloc(n), *t = zalloc(n), *k = zalloc(n);
    or_conv3(x, h, w, Ci, WP(rb->Wa), WP(rb->ba), 4 * Co, 1, u);
    or_shuffle(u, h, w, Co, a);
    for (long e = 0; e < n; e++) a[e] = or_lrelu(a[e]);
    or_conv3(a, 2 * h, 2 * w, Co, WP(rb->Wb), WP(rb->bb), Co, 1, t);
    or_conv3(x, h, w, Ci, WP(rb->Ws), WP(rb->bs), 4 * Co, 1, u);
    or_shuffle(u, h, w, Co, k);
    for (long e = 0; e < n; e++) t[e] += k[e];
    free(u); free(a); free(k);
    return t;
}

/* Hyperprior synthesis: the channel-scaled z-hat through the RB-up blocks
 * (Ch -> Ch, ..., last Ch -> d) to the grid (Hh r) x (Wh r), cropped to
 * H x W: the hyperprior tokens. */
static void hyper_synthesis(or_state *s, const int16_t *zhat)
{
    const or_cfg *c = s->c;
    int nb = or_hyper_blocks(c), h = c->Hh, w = c->Wh;
    double *x = zalloc((long)h * w * c->Ch);
    for (long p = 0; p < (long)h * w; p++)
        for (int ch = 0; ch < c->Ch; ch++) x[p * c->Ch + ch] = WP(s->lay.gamma_z)[ch] * (double)zhat[p * c->Ch + ch];
    for (int b = 0; b < nb; b++) {
        int Co = b == nb - 1 ? c->d : c->Ch;
        double *y = or_rb_up(s, &s->lay.rbu[b], x, h, w, c->Ch, Co);
        free(x);
        x = y; h *= 2; w *= 2;
    }
    for (int i = 0; i < c->H; i++)
        memcpy(s->eh + (long)i * c->W * c->d, x + (long)i * w * c->d, sizeof(double) * c->W * c->d);
    free(x);
}

/* Hyperprior analysis: RMSNorm of the Spatial Module 1 output at every
 * position through the RB-down blocks (d -> Ch, then Ch -> Ch) to z on the
 * ceil(H/r) x ceil(W/r) grid; z-hat = round-half-even(z), clamped to int16. */
static void hyper_analysis(or_state *s, int16_t *zhat, double *z_out)
{
    const or_cfg *c = s->c;
    int nb = or_hyper_blocks(c), h = c->H, w = c->W, Ci = c->d;
    double *x = zalloc((long)h * w * c->d);
    for (int p = 0; p < s->HW; p++) or_rmsnorm(s->x1 + (long)p * c->d, WP(s->lay.g_za), c->d, x + (long)p * c->d);
    for (int b = 0; b < nb; b++) {
        double *y = or_rb_down(s, &s->lay.rbd[b], x, h, w, Ci, c->Ch);
        free(x);
        x = y; h = (h + 1) / 2; w = (w + 1) / 2; Ci = c->Ch;
    }
    for (long e = 0; e < (long)h * w * c->Ch; e++) {
        double r = nearbyint(x[e]);
        if (r < -32768.0) r = -32768.0;
        if (r > 32767.0) r = 32767.0;
        zhat[e] = (int16_t)r;
        if (z_out) z_out[e] = x[e];
    }
    free(x);
}

/* Temporal cross-attention of one query over the co-located T x k x k
 * windows of the Context Transformer output (Sec. 3.1, Sec. 4.1).  Keys are
 * ordered by frame (oldest first), then raster index. */
static void cross_attend(const or_state *s, int b, int p, const double *qv, double *out)
{
    const or_cfg *c = s->c;
    const or_blk *bw = (b < c->L) ? &s->lay.sm1[b] : &s->lay.sm2[b - c->L];
    int maxk = c->Tf * c->k * c->k;
    const double **K = (const double **)malloc(sizeof(double *) * maxk);
    const double **V = (const double **)malloc(sizeof(double *) * maxk);
    double *bias = zalloc((long)maxk * c->nh);
    int *idx = (int *)malloc(sizeof(int) * c->k * c->k), *off = (int *)malloc(sizeof(int) * c->k * c->k);
    int n = 0, kk = c->k * c->k;
    long hd = (long)s->HW * c->d;
    int f0 = s->frame - c->Tf + 1; if (f0 < 0) f0 = 0;
    int nw = or_window_keys(c, -1, p, idx, off);
    for (int f = f0; f <= s->frame; f++) {
        int slot = f % c->Tf, age = s->frame - f;
        for (int j = 0; j < nw; j++) {
            long base = ((long)b * c->Tf + slot) * hd + (long)idx[j] * c->d;
            K[n] = s->XK + base; V[n] = s->XV + base;
            for (int h = 0; h < c->nh; h++)
                bias[(long)n * c->nh + h] = WP(bw->xbias)[((long)h * c->Tf + age) * kk + off[j]];
            n++;
        }
    }
    or_attend(qv, n, K, V, bias, c->nh, c->d, out);
    free(K); free(V); free(bias); free(idx); free(off);
}

/* Phase 1 of a spatial block for position p: pre-norm and Q/K/V. */
static void block_qkv(or_state *s, const or_blk *bw, double *x, double *Kl, double *Vl, int p)
{
    const or_cfg *c = s->c;
    double *n = zalloc(c->d);
    or_rmsnorm(x + (long)p * c->d, WP(bw->g_attn), c->d, n);
    or_matvec(n, WP(bw->Wq), c->d, c->d, s->q + (long)p * c->d);
    or_matvec(n, WP(bw->Wk), c->d, c->d, Kl + (long)p * c->d);
    or_matvec(n, WP(bw->Wv), c->d, c->d, Vl + (long)p * c->d);
    free(n);
}

/* Phase 2 of a spatial block for position p: masked window self-attention
 * over S(p) with residual, optional temporal cross-attention, SwiGLU FFN. */
static void block_rest(or_state *s, int b, const or_blk *bw, double *x, const double *Kl,
                       const double *Vl, int p)
{
    const or_cfg *c = s->c;
    int d = c->d, kk = c->k * c->k;
    int *idx = (int *)malloc(sizeof(int) * kk), *off = (int *)malloc(sizeof(int) * kk);
    const double **K = (const double **)malloc(sizeof(double *) * kk);
    const double **V = (const double **)malloc(sizeof(double *) * kk);
    double *bias = zalloc((long)kk * c->nh), *o = zalloc(d), *t = zalloc(d), *n = zalloc(d);
    double *xp = x + (long)p * d;
    int nk = or_window_keys(c, 1, p, idx, off);
    for (int j = 0; j < nk; j++) {
        K[j] = Kl + (long)idx[j] * d; V[j] = Vl + (long)idx[j] * d;
        for (int h = 0; h < c->nh; h++) bias[(long)j * c->nh + h] = WP(bw->bias)[(long)h * kk + off[j]];
    }
    or_attend(s->q + (long)p * d, nk, K, V, bias, c->nh, d, o);
    or_matvec(o, WP(bw->Wo), d, d, t);
    for (int e = 0; e < d; e++) xp[e] += t[e];
    if (c->temporal) {
        double *qx = zalloc(d);
        or_rmsnorm(xp, WP(bw->g_x), d, n);
        or_matvec(n, WP(bw->Wxq), d, d, qx);
        cross_attend(s, b, p, qx, o);
        or_matvec(o, WP(bw->Wxo), d, d, t);
        for (int e = 0; e < d; e++) xp[e] += t[e];
        free(qx);
    }
    or_rmsnorm(xp, WP(bw->g_ffn), d, n);
    or_swiglu(n, WP(bw->Wg), WP(bw->Wu), WP(bw->Wd), d, c->F, t);
    for (int e = 0; e < d; e++) xp[e] += t[e];
    free(idx); free(off); free(K); free(V); free(bias); free(o); free(t); free(n);
}

/* Spatial Module 1 on a set of positions whose latents are known, then the
 * accumulator's keys/values from its output (Sec. 3.1). */
static void run_sm1(or_state *s, const int *pos, int n, const int16_t *yvis)
{
    const or_cfg *c = s->c;
    long hd = (long)s->HW * c->d;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < n; a++)
        embed_latent(s, yvis + (long)pos[a] * c->C, s->lay.gamma_in, s->lay.W_in, s->lay.b_in,
                     s->x1 + (long)pos[a] * c->d);
    for (int l = 0; l < c->L; l++) {
        #pragma omp parallel for schedule(dynamic, 1)
        for (int a = 0; a < n; a++) block_qkv(s, &s->lay.sm1[l], s->x1, s->K1 + l * hd, s->V1 + l * hd, pos[a]);
        #pragma omp parallel for schedule(dynamic, 1)
        for (int a = 0; a < n; a++) block_rest(s, l, &s->lay.sm1[l], s->x1, s->K1 + l * hd, s->V1 + l * hd, pos[a]);
    }
    #pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < n; a++) {
        double *m = zalloc(c->d);
        long p = pos[a];
        or_rmsnorm(s->x1 + p * c->d, WP(s->lay.acc.g_kv), c->d, m);
        or_matvec(m, WP(s->lay.acc.Wk), c->d, c->d, s->Ka + p * c->d);
        or_matvec(m, WP(s->lay.acc.Wv), c->d, c->d, s->Va + p * c->d);
        free(m);
    }
}

/* Accumulator for one position: hyperprior token as query and residual,
 * keys/values over A(p) (strictly past positions), then SwiGLU (Sec. 3.1,
 * Fig. 2b).  The result initialises the Spatial Module 2 stream. */
static void run_acc(or_state *s, int p)
{
    const or_cfg *c = s->c;
    const or_accw *aw = &s->lay.acc;
    int d = c->d, kk = c->k * c->k;
    int *idx = (int *)malloc(sizeof(int) * kk), *off = (int *)malloc(sizeof(int) * kk);
    const double **K = (const double **)malloc(sizeof(double *) * kk);
    const double **V = (const double **)malloc(sizeof(double *) * kk);
    double *bias = zalloc((long)kk * c->nh), *n = zalloc(d), *qv = zalloc(d), *o = zalloc(d), *t = zalloc(d);
    double *xp = s->x2 + (long)p * d;
    const double *ep = s->eh + (long)p * d;
    or_rmsnorm(ep, WP(aw->g_q), d, n);
    or_matvec(n, WP(aw->Wq), d, d, qv);
    int nk = or_window_keys(c, 0, p, idx, off);
    for (int j = 0; j < nk; j++) {
        K[j] = s->Ka + (long)idx[j] * d; V[j] = s->Va + (long)idx[j] * d;
        for (int h = 0; h < c->nh; h++) bias[(long)j * c->nh + h] = WP(aw->bias)[(long)h * kk + off[j]];
    }
    or_attend(qv, nk, K, V, bias, c->nh, d, o);
    or_matvec(o, WP(aw->Wo), d, d, t);
    for (int e = 0; e < d; e++) xp[e] = ep[e] + t[e];
    or_rmsnorm(xp, WP(aw->g_ffn), d, n);
    or_swiglu(n, WP(aw->Wg), WP(aw->Wu), WP(aw->Wd), d, c->F, t);
    for (int e = 0; e < d; e++) xp[e] += t[e];
    free(idx); free(off); free(K); free(V); free(bias); free(n); free(qv); free(o); free(t);
}

/* Prediction heads (Sec. 3.1): RMSNorm, then two-layer MLPs with SiLU,
 * channel-wise output scaling; sigma through exp with the scale-table range
 * as clamp. */
static void run_heads(or_state *s, int p)
{
    const or_cfg *c = s->c;
    int d = c->d, C = c->C;
    double *n = zalloc(d), *hid = zalloc(d), *o = zalloc(C);
    or_rmsnorm(s->x2 + (long)p * d, WP(s->lay.g_head), d, n);
    or_matvec(n, WP(s->lay.W1m), d, d, hid);
    for (int e = 0; e < d; e++) hid[e] = or_silu(hid[e] + WP(s->lay.b1m)[e]);
    or_matvec(hid, WP(s->lay.W2m), d, C, o);
    for (int ch = 0; ch < C; ch++)
        s->mu[(long)p * C + ch] = WP(s->lay.gamma_mu)[ch] * o[ch] + WP(s->lay.beta_mu)[ch];
    or_matvec(n, WP(s->lay.W1s), d, d, hid);
    for (int e = 0; e < d; e++) hid[e] = or_silu(hid[e] + WP(s->lay.b1s)[e]);
    or_matvec(hid, WP(s->lay.W2s), d, C, o);
    const double lo = log(0.11), hi = log(256.0);
    for (int ch = 0; ch < C; ch++) {
        double v = WP(s->lay.gamma_sig)[ch] * o[ch] + WP(s->lay.beta_sig)[ch];
        if (v < lo) v = lo;
        if (v > hi) v = hi;
        s->sigma[(long)p * C + ch] = exp(v);
    }
    free(n); free(hid); free(o);
}

/* Accumulator, Spatial Module 2 and heads for a set of positions. */
static void run_acc_sm2_heads(or_state *s, const int *pos, int n)
{
    const or_cfg *c = s->c;
    long hd = (long)s->HW * c->d;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < n; a++) run_acc(s, pos[a]);
    for (int l = 0; l < c->L; l++) {
        #pragma omp parallel for schedule(dynamic, 1)
        for (int a = 0; a < n; a++) block_qkv(s, &s->lay.sm2[l], s->x2, s->K2 + l * hd, s->V2 + l * hd, pos[a]);
        #pragma omp parallel for schedule(dynamic, 1)
        for (int a = 0; a < n; a++) block_rest(s, c->L + l, &s->lay.sm2[l], s->x2, s->K2 + l * hd, s->V2 + l * hd, pos[a]);
    }
    if (c->Nc > 0) return;       /* the Channel Transformer and its grouped heads follow */
    #pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < n; a++) run_heads(s, pos[a]);
}

/* RMSNorm of each of the G groups of x (n values) separately: the
 * statistics of a group never see another group's values. */
static void group_rmsnorm(const double *x, const double *g, int n, int G, double *y)
{
    int w = n / G;
    for (int j = 0; j < G; j++) or_rmsnorm(x + (long)j * w, g + (long)j * w, w, y + (long)j * w);
}

/* Channel Transformer and grouped heads at position p (Sec. 3.1, Channel
 * Transformer paragraph; Sec. 3.2, s spatial steps times N channel groups;
 * Sec. 4.1 sizes), from the Spatial Module 2 output there and the latents
 * yv.  The width-dc stream is N groups of dg = dc / N.  Input: the
 * normalised Spatial Module 2 output projected to dc; with the channel
 * shift, group g >= 1 adds the embedding of the channel-scaled latents of
 * group g - 1, so group 0 holds only the spatio-temporal context.  Each of
 * Lct blocks: group-wise RMSNorm, the mixing layer (a dc x dc projection
 * whose block-lower-triangular mask lets output group i read input groups
 * 0..i only, a masked 1 x 1 convolution over channels) with residual, then
 * group-wise RMSNorm and a SwiGLU of each group's own weights with residual.
 * Heads: group-wise RMSNorm, then for mu and for sigma a two-layer MLP per
 * group (grouped MLPs) giving that group's C / N channels.  So the
 * parameters of group g depend on the latents of groups 0..g-1 only.  The
 * final stream is kept in xc (the LRP Transformer's representation). */
static void run_ct_heads(or_state *s, int p, const int16_t *yv)
{
    const or_cfg *c = s->c;
    int d = c->d, C = c->C, dc = c->dc, G = c->Nc, dg = dc / G, Cg = C / G, Fc = c->Fc;
    double *n = zalloc(d), *h = s->xc + (long)p * dc, *a = zalloc(dc), *t = zalloc(dc);
    double *yc = zalloc(Cg), *hid = zalloc(dg), *o = zalloc(Cg);
    or_rmsnorm(s->x2 + (long)p * d, WP(s->lay.ct_g_in), d, n);
    or_matvec(n, WP(s->lay.ct_W_in), d, dc, h);
    for (int e = 0; e < dc; e++) h[e] += WP(s->lay.ct_b_in)[e];
    for (int g = 1; g < G; g++) {
        for (int ch = 0; ch < Cg; ch++) {
            int cc = (g - 1) * Cg + ch;
            yc[ch] = WP(s->lay.ct_gamma_y)[cc] * (double)yv[(long)p * C + cc];
        }
        or_matvec(yc, WP(s->lay.ct_E) + (long)(g - 1) * Cg * dg, Cg, dg, t);
        for (int e = 0; e < dg; e++) h[(long)g * dg + e] += t[e];
    }
    for (int l = 0; l < c->Lct; l++) {
        group_rmsnorm(h, WP(s->lay.ct_g_mix[l]), dc, G, a);
        or_matvec(a, s->ctM[l], dc, dc, t);
        for (int e = 0; e < dc; e++) h[e] += t[e];
        group_rmsnorm(h, WP(s->lay.ct_g_ffn[l]), dc, G, a);
        for (int g = 0; g < G; g++) {
            or_swiglu(a + (long)g * dg, WP(s->lay.ct_Wg[l]) + (long)g * dg * Fc, WP(s->lay.ct_Wu[l]) + (long)g * dg * Fc,
                      WP(s->lay.ct_Wd[l]) + (long)g * Fc * dg, dg, Fc, t);
            for (int e = 0; e < dg; e++) h[(long)g * dg + e] += t[e];
        }
    }
    group_rmsnorm(h, WP(s->lay.g_head), dc, G, a);
    const double lo = log(0.11), hi = log(256.0);
    for (int g = 0; g < G; g++) {
        const double *ag = a + (long)g * dg;
        or_matvec(ag, WP(s->lay.W1m) + (long)g * dg * dg, dg, dg, hid);
        for (int e = 0; e < dg; e++) hid[e] = or_silu(hid[e] + WP(s->lay.b1m)[(long)g * dg + e]);
        or_matvec(hid, WP(s->lay.W2m) + (long)g * dg * Cg, dg, Cg, o);
        for (int ch = 0; ch < Cg; ch++) {
            int cc = g * Cg + ch;
            s->mu[(long)p * C + cc] = WP(s->lay.gamma_mu)[cc] * o[ch] + WP(s->lay.beta_mu)[cc];
        }
        or_matvec(ag, WP(s->lay.W1s) + (long)g * dg * dg, dg, dg, hid);
        for (int e = 0; e < dg; e++) hid[e] = or_silu(hid[e] + WP(s->lay.b1s)[(long)g * dg + e]);
        or_matvec(hid, WP(s->lay.W2s) + (long)g * dg * Cg, dg, Cg, o);
        for (int ch = 0; ch < Cg; ch++) {
            int cc = g * Cg + ch;
            double v = WP(s->lay.gamma_sig)[cc] * o[ch] + WP(s->lay.beta_sig)[cc];
            if (v < lo) v = lo;
            if (v > hi) v = hi;
            s->sigma[(long)p * C + cc] = exp(v);
        }
    }
    free(n); free(a); free(t); free(yc); free(hid); free(o);
}

static void run_ct_all(or_state *s, const int *pos, int n, const int16_t *yv)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < n; a++) run_ct_heads(s, pos[a], yv);
}

/* Context Transformer for frame f (Sec. 3.1): tokens are the previous frame's
 * latents at the same position (temporal shift) or, for frame 0, the learned
 * padding vector; Lc blocks of time-causal window attention over the last Tf
 * frames at this layer, spatially unmasked; final RMSNorm.  Its output is
 * projected once per spatial block into that block's cross-attention K/V. */
static void run_context(or_state *s, const int16_t *yprev)
{
    const or_cfg *c = s->c;
    int d = c->d, kk = c->k * c->k, HW = s->HW, f = s->frame, slot_f = f % c->Tf;
    long hd = (long)HW * d;
    double *g = zalloc(hd);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int p = 0; p < HW; p++) {
        if (f == 0) memcpy(g + (long)p * d, WP(s->lay.pad), sizeof(double) * d);
        else embed_latent(s, yprev + (long)p * c->C, s->lay.gamma_c, s->lay.W_c, s->lay.b_c, g + (long)p * d);
    }
    int f0 = f - c->Tf + 1; if (f0 < 0) f0 = 0;
    for (int l = 0; l < c->Lc; l++) {
        const or_blk *bw = &s->lay.ctx[l];
        double *CKl = s->CK + (long)l * c->Tf * hd, *CVl = s->CV + (long)l * c->Tf * hd;
        #pragma omp parallel for schedule(dynamic, 4)
        for (int p = 0; p < HW; p++) {
            double *n = zalloc(d);
            or_rmsnorm(g + (long)p * d, WP(bw->g_attn), d, n);
            or_matvec(n, WP(bw->Wq), d, d, s->q + (long)p * d);
            or_matvec(n, WP(bw->Wk), d, d, CKl + slot_f * hd + (long)p * d);
            or_matvec(n, WP(bw->Wv), d, d, CVl + slot_f * hd + (long)p * d);
            free(n);
        }
        #pragma omp parallel for schedule(dynamic, 4)
        for (int p = 0; p < HW; p++) {
            int maxk = c->Tf * kk, nk = 0;
            const double **K = (const double **)malloc(sizeof(double *) * maxk);
            const double **V = (const double **)malloc(sizeof(double *) * maxk);
            double *bias = zalloc((long)maxk * c->nh), *o = zalloc(d), *t = zalloc(d), *n = zalloc(d);
            int *idx = (int *)malloc(sizeof(int) * kk), *off = (int *)malloc(sizeof(int) * kk);
            int nw = or_window_keys(c, -1, p, idx, off);
            for (int ff = f0; ff <= f; ff++) {
                int sl = ff % c->Tf, age = f - ff;
                for (int j = 0; j < nw; j++) {
                    K[nk] = CKl + sl * hd + (long)idx[j] * d;
                    V[nk] = CVl + sl * hd + (long)idx[j] * d;
                    for (int h = 0; h < c->nh; h++)
                        bias[(long)nk * c->nh + h] = WP(bw->bias)[((long)h * c->Tf + age) * kk + off[j]];
                    nk++;
                }
            }
            double *gp = g + (long)p * d;
            or_attend(s->q + (long)p * d, nk, K, V, bias, c->nh, d, o);
            or_matvec(o, WP(bw->Wo), d, d, t);
            for (int e = 0; e < d; e++) gp[e] += t[e];
            or_rmsnorm(gp, WP(bw->g_ffn), d, n);
            or_swiglu(n, WP(bw->Wg), WP(bw->Wu), WP(bw->Wd), d, c->F, t);
            for (int e = 0; e < d; e++) gp[e] += t[e];
            free(K); free(V); free(bias); free(o); free(t); free(n); free(idx); free(off);
        }
    }
    #pragma omp parallel for schedule(dynamic, 4)
    for (int p = 0; p < HW; p++) {
        double *cn = zalloc(d);
        or_rmsnorm(g + (long)p * d, WP(s->lay.g_ctx), d, cn);
        for (int b = 0; b < 2 * c->L; b++) {
            const or_blk *bw = (b < c->L) ? &s->lay.sm1[b] : &s->lay.sm2[b - c->L];
            long base = ((long)b * c->Tf + slot_f) * hd + (long)p * d;
            or_matvec(cn, WP(bw->Wxk), d, d, s->XK + base);
            or_matvec(cn, WP(bw->Wxv), d, d, s->XV + base);
        }
        free(cn);
    }
    free(g);
}

/* LRP Transformer of a coded frame (Sec. 3.1, the latent residual
 * prediction; Sec. 4.3 on its temporal transformer): every position's token
 * concatenates the model's final representation there (the heads' input:
 * the Channel Transformer's stream if the model has one, else the Spatial
 * Module 2 stream), normalised, with the channel-scaled quantised
 * latent, projected to the model width; Llrp blocks of window self-attention
 * and SwiGLU; then RMSNorm and a projection to the C channels give the
 * residual eps.  The window is the whole k x k window of the current frame
 * (spatially unmasked: the frame is fully decoded) and, for the temporal
 * model, the same window in each of the Tf - 1 frames before it, whose keys
 * and values of the same block were kept when their LRP ran (time-causal,
 * relative bias by frame age, like the Context Transformer).  Every block
 * computes the keys and values of all positions before any position is
 * updated. */
static void run_lrp(or_state *s, const int16_t *yf, double *eps)
{
    const or_cfg *c = s->c;
    int d = c->d, C = c->C, kk = c->k * c->k, HW = s->HW, f = s->frame;
    int Tw = c->temporal ? c->Tf : 1, slot_f = f % Tw;
    int f0 = f - Tw + 1; if (f0 < 0) f0 = 0;
    long hd = (long)HW * d;
    double *u = zalloc(hd);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int p = 0; p < HW; p++) {
        double *nr = zalloc(c->Nc > 0 ? c->dc : d), *t = zalloc(d), *yc = zalloc(C), *up = u + (long)p * d;
        if (c->Nc > 0) {
            or_rmsnorm(s->xc + (long)p * c->dc, WP(s->lay.lrp_g_rep), c->dc, nr);
            or_matvec(nr, WP(s->lay.lrp_W_rep), c->dc, d, up);
        } else {
            or_rmsnorm(s->x2 + (long)p * d, WP(s->lay.lrp_g_rep), d, nr);
            or_matvec(nr, WP(s->lay.lrp_W_rep), d, d, up);
        }
        for (int ch = 0; ch < C; ch++) yc[ch] = WP(s->lay.lrp_gamma_y)[ch] * (double)yf[(long)p * C + ch];
        or_matvec(yc, WP(s->lay.lrp_W_y), C, d, t);
        for (int e = 0; e < d; e++) up[e] += t[e] + WP(s->lay.lrp_b_in)[e];
        free(nr); free(t); free(yc);
    }
    for (int l = 0; l < c->Llrp; l++) {
        const or_blk *bw = &s->lay.lrp[l];
        double *LKl = s->LK + (long)l * Tw * hd, *LVl = s->LV + (long)l * Tw * hd;
        #pragma omp parallel for schedule(dynamic, 4)
        for (int p = 0; p < HW; p++) {
            double *n = zalloc(d);
            or_rmsnorm(u + (long)p * d, WP(bw->g_attn), d, n);
            or_matvec(n, WP(bw->Wq), d, d, s->q + (long)p * d);
            or_matvec(n, WP(bw->Wk), d, d, LKl + slot_f * hd + (long)p * d);
            or_matvec(n, WP(bw->Wv), d, d, LVl + slot_f * hd + (long)p * d);
            free(n);
        }
        #pragma omp parallel for schedule(dynamic, 4)
        for (int p = 0; p < HW; p++) {
            int maxk = Tw * kk, nk = 0;
            int *idx = (int *)malloc(sizeof(int) * kk), *off = (int *)malloc(sizeof(int) * kk);
            const double **Kp = (const double **)malloc(sizeof(double *) * maxk);
            const double **Vp = (const double **)malloc(sizeof(double *) * maxk);
            double *bias = zalloc((long)maxk * c->nh), *o = zalloc(d), *t = zalloc(d), *n = zalloc(d);
            double *up = u + (long)p * d;
            int nw = or_window_keys(c, -1, p, idx, off);
            for (int ff = f0; ff <= f; ff++) {
                int sl = ff % Tw, age = f - ff;
                for (int j = 0; j < nw; j++) {
                    Kp[nk] = LKl + sl * hd + (long)idx[j] * d;
                    Vp[nk] = LVl + sl * hd + (long)idx[j] * d;
                    for (int h = 0; h < c->nh; h++)
                        bias[(long)nk * c->nh + h] = WP(bw->bias)[((long)h * Tw + age) * kk + off[j]];
                    nk++;
                }
            }
            or_attend(s->q + (long)p * d, nk, Kp, Vp, bias, c->nh, d, o);
            or_matvec(o, WP(bw->Wo), d, d, t);
            for (int e = 0; e < d; e++) up[e] += t[e];
            or_rmsnorm(up, WP(bw->g_ffn), d, n);
            or_swiglu(n, WP(bw->Wg), WP(bw->Wu), WP(bw->Wd), d, c->F, t);
            for (int e = 0; e < d; e++) up[e] += t[e];
            free(idx); free(off); free(Kp); free(Vp); free(bias); free(o); free(t); free(n);
        }
    }
    #pragma omp parallel for schedule(dynamic, 4)
    for (int p = 0; p < HW; p++) {
        double *n = zalloc(d), *ep = eps + (long)p * C;
        or_rmsnorm(u + (long)p * d, WP(s->lay.lrp_g_out), d, n);
        or_matvec(n, WP(s->lay.lrp_W_eps), d, C, ep);
        for (int ch = 0; ch < C; ch++) ep[ch] += WP(s->lay.lrp_b_eps)[ch];
        free(n);
    }
    free(u);
}

/* ------------------------------------------------------------------------ */
/* Schedules                                                                 */
/* ------------------------------------------------------------------------ */

/* Step sets of a schedule: 0 = wavefront by mask label (positions of one
 * label in raster order), 1 = raster order (one position per step).
 * order[] receives all positions in schedule order; start[t]..start[t+1]-1
 * is step t.  Returns the number of steps. */
int or_schedule(const or_cfg *c, int kind, int *order, int *start)
{
    int HW = c->H * c->W, n = 0, T = 0;
    if (kind == 1) {
        for (int p = 0; p < HW; p++) { start[p] = p; order[p] = p; }
        start[HW] = HW;
        return HW;
    }
    int maxl = 0;
    for (int i = 0; i < c->H; i++)
        for (int j = 0; j < c->W; j++)
            if (or_label(c->mask, i, j) > maxl) maxl = or_label(c->mask, i, j);
    for (int t = 0; t <= maxl; t++) {
        start[T] = n;
        for (int i = 0; i < c->H; i++)
            for (int j = 0; j < c->W; j++)
                if (or_label(c->mask, i, j) == t) order[n++] = i * c->W + j;
        if (n > start[T]) T++;
    }
    start[T] = n;
    return T;
}

/* ------------------------------------------------------------------------ */
/* Scale table, quantisation, CDF tables, rate (Fig. 1: Q, AE/AD)            */
/* ------------------------------------------------------------------------ */
/* E4M3 weights (the FP8 precision form of Sec. 3.2's GEMMs)                  */
/* ------------------------------------------------------------------------ */

/* Nearest E4M3 value, ties to even, saturating at +-448.  The format: sign,
 * 4 exponent bits with bias 7, 3 mantissa bits, no infinities; normal values
 * (1 + m/8) 2^e for e = -6 .. 8 (the all-ones pattern at e = 8 is NaN, so
 * 448 = 1.75 * 2^8 is the largest finite), subnormals (m/8) 2^-6.  Within a
 * binade 2^e .. 2^(e+1) the spacing is 2^(e-3); below 2^-6 it is 2^-9. */
double or_e4m3(double x)
{
    double a = fabs(x);
    if (a == 0.0 || a != a) return x;
    int e2;
    frexp(a, &e2);                         /* a = f 2^e2, f in [0.5, 1) */
    int e = e2 - 1;                        /* a in [2^e, 2^(e+1)) */
    if (e < -6) e = -6;
    double q = ldexp(1.0, e - 3);
    double v = nearbyint(a / q) * q;       /* default rounding: to nearest, ties to even */
    if (v > 448.0) v = 448.0;
    return copysign(v, x);
}

/* One tensor quantised and dequantised as the FP8 weights: with max |x| in
 * [2^e, 2^(e+1)) (e >= -100) the scale is s = 2^(e-7), s = 1 for an
 * all-zero tensor, and out[i] = s E4M3(x[i] / s).  Returns s. */
double or_e4m3_tensor(long n, const double *x, double *out)
{
    double amax = 0.0;
    for (long i = 0; i < n; i++) amax = fmax(amax, fabs(x[i]));
    double s = 1.0;
    if (amax > 0.0) {
        int e2;
        frexp(amax, &e2);
        int e = e2 - 1 < -100 ? -100 : e2 - 1;
        s = ldexp(1.0, e - 7);
    }
    for (long i = 0; i < n; i++) out[i] = s * or_e4m3(x[i] / s);
    return s;
}

/* ------------------------------------------------------------------------ */

#define OR_NSCALES 64
#define OR_PREC 16
#define OR_M (1u << OR_PREC)

/* 64 log-spaced scales from 0.11 to 256, rounded to float. */
void or_scale_table(float *tab)
{
    double lo = log(0.11), hi = log(256.0);
    for (int l = 0; l < OR_NSCALES; l++) tab[l] = (float)exp(lo + l * (hi - lo) / (OR_NSCALES - 1));
}

/* idx = smallest l with table[l] >= sigma (float compare), else 63;
 * m = round-half-even of mu clamped to the int16 range (float). */
void or_quantize(long n, const float *mu, const float *sigma, uint8_t *idx, int32_t *m)
{
    float tab[OR_NSCALES];
    or_scale_table(tab);
    for (long a = 0; a < n; a++) {
        int l = OR_NSCALES - 1;
        for (int t = 0; t < OR_NSCALES; t++)
            if (tab[t] >= sigma[a]) { l = t; break; }
        idx[a] = (uint8_t)l;
        float mc = fminf(fmaxf(mu[a], -32768.0f), 32767.0f);
        m[a] = (int32_t)rintf(mc);
    }
}

/* Support half-width of table l. */
int or_cdf_T(int l)
{
    float tab[OR_NSCALES];
    or_scale_table(tab);
    int T = (int)ceil(7.0 * (double)tab[l]);
    return T < 1 ? 1 : T;
}

/* Integer frequency table for scale l: slots -T..T then ESC (2T+2 slots).
 * pmf of a zero-mean quantised Gaussian from erfc; ESC takes both tails;
 * freq = 1 + floor(pmf * (2^16 - n)); the remainder goes to symbol 0.
 * freq[] needs 2T+2 entries.  Returns n. */
int or_cdf_freq(int l, uint32_t *freq)
{
    float tab[OR_NSCALES];
    or_scale_table(tab);
    double sg = (double)tab[l];
    int T = or_cdf_T(l), n = 2 * T + 2;
    double den = sg * 1.4142135623730951;
    long sum = 0;
    for (int s = -T; s <= T; s++) {
        double u = (double)(s < 0 ? -s : s);
        double pmf = 0.5 * (erfc((u - 0.5) / den) - erfc((u + 0.5) / den));
        freq[s + T] = 1u + (uint32_t)floor(pmf * (double)(OR_M - (uint32_t)n));
        sum += freq[s + T];
    }
    double pesc = erfc(((double)T + 0.5) / den);
    freq[2 * T + 1] = 1u + (uint32_t)floor(pesc * (double)(OR_M - (uint32_t)n));
    sum += freq[2 * T + 1];
    freq[T] = (uint32_t)((long)freq[T] + ((long)OR_M - sum));
    return n;
}

/* Model rate: -sum log2 P(y | mu, sigma) with P the Gaussian mass of
 * [y - 1/2, y + 1/2] (evaluated on |y - mu| through erfc), sigma clamped to
 * [0.11, 256], P floored at 1e-9. */
double or_likelihood(double y, double mu, double sigma)
{
    if (sigma < 0.11) sigma = 0.11;
    if (sigma > 256.0) sigma = 256.0;
    double u = fabs(y - mu), den = sigma * 1.4142135623730951;
    double p = 0.5 * (erfc((u - 0.5) / den) - erfc((u + 0.5) / den));
    return p < 1e-9 ? 1e-9 : p;
}

double or_rate_bits(long n, const int16_t *y, const double *mu, const double *sigma)
{
    double bits = 0.0;
    for (long a = 0; a < n; a++) bits -= log2(or_likelihood((double)y[a], mu[a], sigma[a]));
    return bits;
}

/* ------------------------------------------------------------------------ */
/* Interleaved rANS (32 lanes, 32-bit states, 16-bit words, M = 2^16)         */
/* ------------------------------------------------------------------------ */
/* Container (little endian): u32 magic 'PSW1', u16 version 1, u16 schedule,
 * u16 H, u16 W, u16 C, u16 0, u32 offsets[C+1] (absolute byte offsets of the
 * C channel streams, last = total size).  Stream: u32 state[32], then the
 * renormalisation words in decoding order, padded with one zero word to a
 * multiple of 4 bytes.  Symbol k of a channel stream (schedule order) is
 * coded on lane k mod 32.  Per symbol the decoder: takes the slot from the
 * low 16 bits, advances the state, reads one word if the state fell below
 * 2^16; for ESC it then takes two raw 16-bit digits d0 (low) and d1 of
 * v = 2 (|s| - T - 1) + (s < 0), each followed by one word read. */

#define OR_MAGIC 0x31575350u
#define OR_LOW (1u << 16)

typedef struct { uint32_t *cum, *freq; int *T, *n; } or_tables;

static void tables_alloc(or_tables *tb, int nt)
{
    tb->cum = (uint32_t *)malloc(sizeof(uint32_t) * nt * 4096);
    tb->freq = (uint32_t *)malloc(sizeof(uint32_t) * nt * 4096);
    tb->T = (int *)malloc(sizeof(int) * nt);
    tb->n = (int *)malloc(sizeof(int) * nt);
}

static void tables_cum(or_tables *tb, int l)
{
    uint32_t *f = tb->freq + (long)l * 4096, *cm = tb->cum + (long)l * 4096, acc = 0;
    for (int s = 0; s < tb->n[l]; s++) { cm[s] = acc; acc += f[s]; }
}

static void tables_build(or_tables *tb)
{
    tables_alloc(tb, OR_NSCALES);
    for (int l = 0; l < OR_NSCALES; l++) {
        tb->n[l] = or_cdf_freq(l, tb->freq + (long)l * 4096);
        tb->T[l] = or_cdf_T(l);
        tables_cum(tb, l);
    }
}

/* Factorized prior of z-hat (Fig. 1 right "Factorized Prior"; the
 * univariate non-parametric density of Balle et al. 2018 that the
 * hyperprior literature uses): per channel a cumulative
 * c(x) = sigmoid(f4(f3(f2(f1(x))))) through widths 1 -> 3 -> 3 -> 3 -> 1, with
 * f_k(v) = g_k(softplus(H_k) v + b_k), g_k(t) = t + tanh(a_k) tanh(t) for
 * k < 4 (elementwise), f_4 affine; softplus keeps every matrix entry
 * positive, so c is increasing.  P(z-hat = k) = c(k + 1/2) - c(k - 1/2).
 * Sums run over ascending inputs after the bias. */
static double fp_softplus(double x) { return x > 30.0 ? x : log1p(exp(x)); }

static double prior_cdf(const double *w, const or_layout *L, int ch, double x)
{
    double v1[3], v2[3], v3[3];
    for (int i = 0; i < 3; i++) {
        double t = w[L->fp_b1 + ch * 3 + i] + fp_softplus(w[L->fp_H1 + ch * 3 + i]) * x;
        v1[i] = t + tanh(w[L->fp_a1 + ch * 3 + i]) * tanh(t);
    }
    for (int i = 0; i < 3; i++) {
        double t = w[L->fp_b2 + ch * 3 + i];
        for (int k = 0; k < 3; k++) t += fp_softplus(w[L->fp_H2 + (ch * 3 + i) * 3 + k]) * v1[k];
        v2[i] = t + tanh(w[L->fp_a2 + ch * 3 + i]) * tanh(t);
    }
    for (int i = 0; i < 3; i++) {
        double t = w[L->fp_b3 + ch * 3 + i];
        for (int k = 0; k < 3; k++) t += fp_softplus(w[L->fp_H3 + (ch * 3 + i) * 3 + k]) * v2[k];
        v3[i] = t + tanh(w[L->fp_a3 + ch * 3 + i]) * tanh(t);
    }
    double t = w[L->fp_b4 + ch];
    for (int k = 0; k < 3; k++) t += fp_softplus(w[L->fp_H4 + ch * 3 + k]) * v3[k];
    return 1.0 / (1.0 + exp(-t));
}

#define OR_TZ 31   /* support half-width of every channel's z-hat table */

/* Integer table of channel ch: slots -TZ..TZ then ESC (both tails), with
 * the rule of the scale tables (freq = 1 + floor(pmf (2^16 - n)), the
 * remainder to symbol 0).  Returns n. */
static int prior_freq(const double *w, const or_layout *L, int ch, uint32_t *freq)
{
    int T = OR_TZ, n = 2 * T + 2;
    long sum = 0;
    for (int v = -T; v <= T; v++) {
        double pmf = prior_cdf(w, L, ch, v + 0.5) - prior_cdf(w, L, ch, v - 0.5);
        freq[v + T] = 1u + (uint32_t)floor(pmf * (double)(OR_M - (uint32_t)n));
        sum += freq[v + T];
    }
    double pesc = prior_cdf(w, L, ch, -T - 0.5) + (1.0 - prior_cdf(w, L, ch, T + 0.5));
    freq[2 * T + 1] = 1u + (uint32_t)floor(pesc * (double)(OR_M - (uint32_t)n));
    sum += freq[2 * T + 1];
    freq[T] = (uint32_t)((long)freq[T] + ((long)OR_M - sum));
    return n;
}

static void tables_prior(or_tables *tb, const or_cfg *c, const double *w)
{
    or_layout L;
    make_layout(c, &L);
    tables_alloc(tb, c->Ch);
    for (int ch = 0; ch < c->Ch; ch++) {
        tb->n[ch] = prior_freq(w, &L, ch, tb->freq + (long)ch * 4096);
        tb->T[ch] = OR_TZ;
        tables_cum(tb, ch);
    }
}

int or_prior_freq(const or_cfg *c, const double *w, int ch, uint32_t *freq)
{
    or_layout L;
    if (!c->hp || ch < 0 || ch >= c->Ch) return 0;
    make_layout(c, &L);
    return prior_freq(w, &L, ch, freq);
}

/* -sum log2 P(z-hat) under the factorized prior (P floored at 1e-9). */
double or_hyper_rate(const or_cfg *c, const double *w, const int16_t *zhat)
{
    or_layout L;
    make_layout(c, &L);
    double bits = 0.0;
    for (long a = 0; a < (long)c->Hh * c->Wh * c->Ch; a++) {
        int ch = (int)(a % c->Ch);
        double p = prior_cdf(w, &L, ch, zhat[a] + 0.5) - prior_cdf(w, &L, ch, zhat[a] - 0.5);
        bits -= log2(p < 1e-9 ? 1e-9 : p);
    }
    return bits;
}

static void tables_free(or_tables *tb) { free(tb->cum); free(tb->freq); free(tb->T); free(tb->n); }

static void put16(uint8_t *b, uint16_t v) { b[0] = (uint8_t)v; b[1] = (uint8_t)(v >> 8); }
static void put32(uint8_t *b, uint32_t v) { put16(b, (uint16_t)v); put16(b + 2, (uint16_t)(v >> 16)); }
static uint16_t get16(const uint8_t *b) { return (uint16_t)(b[0] | (b[1] << 8)); }
static uint32_t get32(const uint8_t *b) { return (uint32_t)get16(b) | ((uint32_t)get16(b + 2) << 16); }

/* Encode one frame.  y, idx, m: [HW][C] in raster layout; order: the
 * schedule's position order.  Returns the container size, or -1 if it does
 * not fit in cap bytes, or -2 on an unencodable symbol. */
static long rans_encode_tb(const or_tables *tbp, int H, int W, int C, int schedule, const int *order,
                           const int16_t *y, const uint8_t *idx, const int32_t *m, uint8_t *out, long cap);

long or_rans_encode(int H, int W, int C, int schedule, const int *order, const int16_t *y,
                    const uint8_t *idx, const int32_t *m, uint8_t *out, long cap)
{
    or_tables tb;
    tables_build(&tb);
    long r = rans_encode_tb(&tb, H, W, C, schedule, order, y, idx, m, out, cap);
    tables_free(&tb);
    return r;
}

/* The encoder with a given table set (idx: table of each symbol). */
static long rans_encode_tb(const or_tables *tbp, int H, int W, int C, int schedule, const int *order,
                           const int16_t *y, const uint8_t *idx, const int32_t *m, uint8_t *out, long cap)
{
    const or_tables tb = *tbp;
    int HW = H * W;
    long hdr = 16 + 4L * (C + 1), pos = hdr;
    uint16_t *words = (uint16_t *)malloc(sizeof(uint16_t) * (3L * HW + 2));
    if (hdr > cap) { free(words); return -1; }
    put32(out, OR_MAGIC); put16(out + 4, 1); put16(out + 6, (uint16_t)schedule);
    put16(out + 8, (uint16_t)H); put16(out + 10, (uint16_t)W); put16(out + 12, (uint16_t)C); put16(out + 14, 0);
    for (int c = 0; c < C; c++) {
        uint32_t x[32];
        for (int l = 0; l < 32; l++) x[l] = OR_LOW;
        long nw = 0;
        for (long k = HW - 1; k >= 0; k--) {
            long a = (long)order[k] * C + c;
            int lane = (int)(k % 32), l = idx[a], T = tb.T[l];
            long sv = (long)y[a] - (long)m[a];
            int slot;
            if (sv >= -T && sv <= T) slot = (int)(sv + T);
            else {
                slot = 2 * T + 1;
                long e = (sv < 0 ? -sv : sv) - T - 1;
                long v = 2 * e + (sv < 0 ? 1 : 0);
                if (v < 0 || v >= (1L << 32)) { free(words); return -2; }
                uint32_t dig[2] = { (uint32_t)(v & 0xFFFF), (uint32_t)(v >> 16) };
                if (dig[1] > 0xFFFF) { free(words); return -2; }
                for (int q = 1; q >= 0; q--) {     /* d1 first: decoded last */
                    words[nw++] = (uint16_t)(x[lane] & 0xFFFF);
                    x[lane] >>= 16;
                    x[lane] = (x[lane] << 16) | dig[q];
                }
            }
            uint32_t f = tb.freq[(long)l * 4096 + slot], cm = tb.cum[(long)l * 4096 + slot];
            if (x[lane] >= (f << 16)) { words[nw++] = (uint16_t)(x[lane] & 0xFFFF); x[lane] >>= 16; }
            x[lane] = ((x[lane] / f) << 16) + (x[lane] % f) + cm;
        }
        long sz = 128 + 2 * nw + ((nw & 1) ? 2 : 0);
        if (pos + sz > cap) { free(words); return -1; }
        put32(out + 16 + 4L * c, (uint32_t)pos);
        for (int l = 0; l < 32; l++) put32(out + pos + 4L * l, x[l]);
        for (long q = 0; q < nw; q++) put16(out + pos + 128 + 2 * q, words[nw - 1 - q]);
        if (nw & 1) put16(out + pos + 128 + 2 * nw, 0);
        pos += sz;
    }
    put32(out + 16 + 4L * C, (uint32_t)pos);
    free(words);
    return pos;
}

/* Sequential decoder state for one frame. */
typedef struct {
    const uint8_t *buf; long len;
    int C;
    uint32_t x[4096][32];  /* per channel lane states (C <= 4096) */
    long ptr[4096], end[4096];
    long k;                /* symbols decoded so far per channel */
    int err;
    or_tables tb;
} or_dec;

static int dec_open_hdr(or_dec *D, const uint8_t *buf, long len, int H, int W, int C, int schedule);

static int dec_open(or_dec *D, const uint8_t *buf, long len, int H, int W, int C, int schedule)
{
    if (dec_open_hdr(D, buf, len, H, W, C, schedule)) return -1;
    tables_build(&D->tb);
    return 0;
}

/* Header and stream checks, lane states; no tables. */
static int dec_open_hdr(or_dec *D, const uint8_t *buf, long len, int H, int W, int C, int schedule)
{
    memset(D, 0, sizeof(*D));
    D->buf = buf; D->len = len; D->C = C;
    long hdr = 16 + 4L * (C + 1);
    if (C > 4096 || len < hdr) return -1;
    if (get32(buf) != OR_MAGIC || get16(buf + 4) != 1 || get16(buf + 6) != schedule ||
        get16(buf + 8) != H || get16(buf + 10) != W || get16(buf + 12) != C) return -1;
    for (int c = 0; c < C; c++) {
        long a = get32(buf + 16 + 4L * c), b = get32(buf + 16 + 4L * (c + 1));
        if (a < hdr || b > len || b < a + 128) return -1;
        for (int l = 0; l < 32; l++) D->x[c][l] = get32(buf + a + 4L * l);
        D->ptr[c] = a + 128; D->end[c] = b;
    }
    return 0;
}

static uint32_t dec_word(or_dec *D, int c)
{
    if (D->ptr[c] + 2 > D->end[c]) { D->err = 1; return 0; }
    uint32_t w = get16(D->buf + D->ptr[c]);
    D->ptr[c] += 2;
    return w;
}

/* Decode the symbols of n positions (the next n of the schedule) for every
 * channel.  idx, m: [n][C] for those positions; yout: [n][C]. */
/* The next n symbols of channels [c0, c1) (idx, m, yout: [n][C]); the
 * symbol counter advances with dec_advance once every channel is done. */
static void dec_channels(or_dec *D, int n, int c0, int c1, const uint8_t *idx, const int32_t *m, int16_t *yout)
{
    for (int c = c0; c < c1; c++) {
        for (int a = 0; a < n; a++) {
            long k = D->k + a;
            int lane = (int)(k % 32), l = idx[(long)a * D->C + c], T = D->tb.T[l];
            const uint32_t *cm = D->tb.cum + (long)l * 4096, *fq = D->tb.freq + (long)l * 4096;
            uint32_t x = D->x[c][lane], v = x & 0xFFFF;
            int slot = 0;
            while (slot + 1 < D->tb.n[l] && cm[slot + 1] <= v) slot++;
            x = fq[slot] * (x >> 16) + v - cm[slot];
            if (x < OR_LOW) x = (x << 16) | dec_word(D, c);
            long sv;
            if (slot == 2 * T + 1) {
                uint32_t dig[2];
                for (int q = 0; q < 2; q++) {
                    dig[q] = x & 0xFFFF;
                    x >>= 16;
                    x = (x << 16) | dec_word(D, c);
                }
                uint32_t vv = dig[0] | (dig[1] << 16);
                long mag = (long)T + 1 + (long)(vv >> 1);
                sv = (vv & 1) ? -mag : mag;
            } else {
                sv = slot - T;
            }
            D->x[c][lane] = x;
            long yv = (long)m[(long)a * D->C + c] + sv;
            if (yv < -32768 || yv > 32767) { D->err = 1; yv = 0; }
            yout[(long)a * D->C + c] = (int16_t)yv;
        }
    }
}

static void dec_advance(or_dec *D, int n) { D->k += n; }

static void dec_symbols(or_dec *D, int n, const uint8_t *idx, const int32_t *m, int16_t *yout)
{
    dec_channels(D, n, 0, D->C, idx, m, yout);
    dec_advance(D, n);
}

static int dec_close(or_dec *D)
{
    int bad = D->err;
    for (int c = 0; c < D->C; c++) {
        long rem = D->end[c] - D->ptr[c];
        if (!(rem == 0 || (rem == 2 && get16(D->buf + D->ptr[c]) == 0))) bad = 1;
        for (int l = 0; l < 32; l++) if (D->x[c][l] != OR_LOW) bad = 1;
    }
    tables_free(&D->tb);
    return bad ? -1 : 0;
}

/* z-hat container (the coder's format: raster order over the hyperprior
 * grid, one stream per channel, channel ch coded with its factorized-prior
 * table, mean 0).  Returns the size, -1 if it does not fit, -2 on an
 * unencodable symbol. */
long or_hyper_encode(const or_cfg *c, const double *w, const int16_t *zhat, uint8_t *out, long cap)
{
    long HW = (long)c->Hh * c->Wh, n = HW * c->Ch;
    int *order = (int *)malloc(sizeof(int) * HW);
    uint8_t *idx = (uint8_t *)malloc((size_t)n);
    int32_t *m = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    for (long p = 0; p < HW; p++) order[p] = (int)p;
    for (long a = 0; a < n; a++) idx[a] = (uint8_t)(a % c->Ch);
    or_tables tb;
    tables_prior(&tb, c, w);
    long r = rans_encode_tb(&tb, c->Hh, c->Wh, c->Ch, 1, order, zhat, idx, m, out, cap);
    tables_free(&tb);
    free(order); free(idx); free(m);
    return r;
}

/* Decode a z-hat container: 0, or -1 if it fails validation. */
int or_hyper_decode(const or_cfg *c, const double *w, const uint8_t *buf, long len, int16_t *zhat)
{
    long HW = (long)c->Hh * c->Wh, n = HW * c->Ch;
    or_dec *D = (or_dec *)malloc(sizeof(or_dec));
    if (c->Ch > 256 || dec_open_hdr(D, buf, len, c->Hh, c->Wh, c->Ch, 1)) { free(D); return -1; }
    tables_prior(&D->tb, c, w);
    uint8_t *idx = (uint8_t *)malloc((size_t)n);
    int32_t *m = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    for (long a = 0; a < n; a++) idx[a] = (uint8_t)(a % c->Ch);
    dec_symbols(D, (int)HW, idx, m, zhat);
    int rc = dec_close(D);
    free(D); free(idx); free(m);
    return rc;
}

/* Coder-only decode with known per-symbol (idx, m) (they do not depend on
 * the decoded values in this entry point).  Returns 0 or -1 (corrupt). */
int or_rans_decode(int H, int W, int C, int schedule, const int *order, const int *start, int T,
                   const uint8_t *idx, const int32_t *m, const uint8_t *buf, long len, int16_t *y)
{
    or_dec *D = (or_dec *)malloc(sizeof(or_dec));
    if (dec_open(D, buf, len, H, W, C, schedule)) { free(D); return -1; }
    uint8_t *ib = (uint8_t *)malloc((size_t)H * W * C);
    int32_t *mb = (int32_t *)malloc(sizeof(int32_t) * H * W * C);
    int16_t *yb = (int16_t *)malloc(sizeof(int16_t) * H * W * C);
    for (int t = 0; t < T; t++) {
        int n = start[t + 1] - start[t];
        for (int a = 0; a < n; a++) {
            long p = order[start[t] + a];
            memcpy(ib + (long)a * C, idx + p * C, C);
            memcpy(mb + (long)a * C, m + p * C, sizeof(int32_t) * C);
        }
        dec_symbols(D, n, ib, mb, yb);
        for (int a = 0; a < n; a++) memcpy(y + (long)order[start[t] + a] * C, yb + (long)a * C, sizeof(int16_t) * C);
    }
    int rc = dec_close(D);
    free(D); free(ib); free(mb); free(yb);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Drivers                                                                   */
/* ------------------------------------------------------------------------ */

/* Run the model over a sequence of nf frames.
 *   driver 0: masked parallel pass (every position at once per layer; the
 *             encoder's view and the definition of the parameters);
 *   driver 1: schedule-driven decode: step t runs Spatial Module 1 on the
 *             positions of step t-1 (whose latents were just revealed), then
 *             the accumulator, Spatial Module 2 and heads on step t; the
 *             latents of step t are then revealed.  Latents not yet revealed
 *             hold the poison value 30000, so any read of them shows up.
 *             sched selects the step sets (0 wavefront, 1 raster).
 *   driver 2: like 1, but the latents are decoded from the per-frame
 *             bitstreams (bs[f], lens[f]) with float-rounded parameters
 *             instead of revealed from y; y receives the decoded latents.
 * y: [nf][H][W][C]; z: [nf][Hh][Wh][Ch]; mu, sigma: [nf][H][W][C].
 * Returns 0, -1 on allocation failure, -2 on a corrupt bitstream. */
/* or_run, and for a model with an LRP Transformer (eps non-null) each
 * frame's residual eps [nf][H][W][C] from its coded latents. */
int or_run_lrp(const or_cfg *c, const double *w, int nf, int16_t *y, const int16_t *z,
               int driver, int sched, const uint8_t *const *bs, const long *lens,
               double *mu, double *sigma, double *eps)
{
    or_state st, *s = &st;
    if (c->L > OR_MAXL || c->Lc > OR_MAXL || c->Llrp > OR_MAXL || c->Lct > OR_MAXL) return -1;
    if (c->hp && or_hyper_blocks(c) < 0) return -1;
    if (eps && c->Llrp <= 0) return -1;
    if (state_init(s, c, w)) { state_free(s); return -1; }
    int HW = s->HW, C = c->C;
    int *order = (int *)malloc(sizeof(int) * HW), *start = (int *)malloc(sizeof(int) * (HW + 1));
    int16_t *yvis = (int16_t *)malloc(sizeof(int16_t) * (long)HW * C);
    int T = or_schedule(c, sched, order, start);
    int rc = 0;
    for (int f = 0; f < nf && rc == 0; f++) {
        int16_t *yf = y + (long)f * HW * C;
        s->frame = f;
        memset(s->x1, 0, sizeof(double) * HW * c->d);
        memset(s->x2, 0, sizeof(double) * HW * c->d);
        if (c->temporal) run_context(s, f > 0 ? y + (long)(f - 1) * HW * C : NULL);
        embed_hyper(s, z + (long)f * c->Hh * c->Wh * c->Ch);
        if (driver == 0) {
            int *all = (int *)malloc(sizeof(int) * HW);
            for (int p = 0; p < HW; p++) all[p] = p;
            run_sm1(s, all, HW, yf);
            run_acc_sm2_heads(s, all, HW);
            if (c->Nc > 0) run_ct_all(s, all, HW, yf);
            free(all);
        } else {
            or_dec *D = NULL;
            uint8_t *ib = NULL; int32_t *mb = NULL; int16_t *yb = NULL;
            if (driver == 2) {
                D = (or_dec *)malloc(sizeof(or_dec));
                if (dec_open(D, bs[f], lens[f], c->H, c->W, C, sched)) { free(D); rc = -2; break; }
                ib = (uint8_t *)malloc((size_t)HW * C);
                mb = (int32_t *)malloc(sizeof(int32_t) * HW * C);
                yb = (int16_t *)malloc(sizeof(int16_t) * HW * C);
            }
            for (long a = 0; a < (long)HW * C; a++) yvis[a] = 30000;
            for (int t = 0; t < T; t++) {
                const int *ps = order + start[t];
                int n = start[t + 1] - start[t];
                if (t > 0) run_sm1(s, order + start[t - 1], start[t] - start[t - 1], yvis);
                run_acc_sm2_heads(s, ps, n);
                /* with a Channel Transformer the step's channel groups follow
                 * one another: the parameters of group g (computed with the
                 * latents revealed so far), then that group's latents */
                int G = c->Nc > 0 ? c->Nc : 1, Cg = C / G;
                for (int g = 0; g < G; g++) {
                    int c0 = g * Cg;
                    if (c->Nc > 0) run_ct_all(s, ps, n, yvis);
                    if (driver == 1) {
                        for (int a = 0; a < n; a++)
                            memcpy(yvis + (long)ps[a] * C + c0, yf + (long)ps[a] * C + c0, sizeof(int16_t) * Cg);
                    } else {
                        float *mf = (float *)malloc(sizeof(float) * n * C), *sf = (float *)malloc(sizeof(float) * n * C);
                        for (int a = 0; a < n; a++)
                            for (int ch = 0; ch < C; ch++) {
                                mf[(long)a * C + ch] = (float)s->mu[(long)ps[a] * C + ch];
                                sf[(long)a * C + ch] = (float)s->sigma[(long)ps[a] * C + ch];
                            }
                        or_quantize((long)n * C, mf, sf, ib, mb);
                        dec_channels(D, n, c0, c0 + Cg, ib, mb, yb);
                        for (int a = 0; a < n; a++)
                            memcpy(yvis + (long)ps[a] * C + c0, yb + (long)a * C + c0, sizeof(int16_t) * Cg);
                        free(mf); free(sf);
                    }
                }
                if (driver == 2) dec_advance(D, n);
            }
            if (driver == 2) {
                if (dec_close(D)) rc = -2;
                memcpy(yf, yvis, sizeof(int16_t) * HW * C);
                free(D); free(ib); free(mb); free(yb);
            }
        }
        memcpy(mu + (long)f * HW * C, s->mu, sizeof(double) * HW * C);
        memcpy(sigma + (long)f * HW * C, s->sigma, sizeof(double) * HW * C);
        if (eps && rc == 0) run_lrp(s, yf, eps + (long)f * HW * C);
    }
    free(order); free(start); free(yvis);
    state_free(s);
    return rc;
}

/* The encoder's hyperprior analysis of nf frames (convolutional
 * hyperprior models): per frame the Context Transformer (temporal model)
 * and Spatial Module 1 over every position with the frame's latents, then
 * the RB-down blocks and rounding.  zhat: [nf][Hh][Wh][Ch]; z (optional,
 * may be NULL) receives the unrounded values.  Returns 0 or -1. */
int or_hyper_analysis(const or_cfg *c, const double *w, int nf, const int16_t *y, int16_t *zhat, double *z)
{
    or_state st, *s = &st;
    if (!c->hp || or_hyper_blocks(c) < 0 || c->L > OR_MAXL || c->Lc > OR_MAXL) return -1;
    if (state_init(s, c, w)) { state_free(s); return -1; }
    int HW = s->HW, C = c->C;
    long nz = (long)c->Hh * c->Wh * c->Ch;
    int *all = (int *)malloc(sizeof(int) * HW);
    for (int p = 0; p < HW; p++) all[p] = p;
    for (int f = 0; f < nf; f++) {
        s->frame = f;
        memset(s->x1, 0, sizeof(double) * HW * c->d);
        if (c->temporal) run_context(s, f > 0 ? y + (long)(f - 1) * HW * C : NULL);
        run_sm1(s, all, HW, y + (long)f * HW * C);
        hyper_analysis(s, zhat + f * nz, z ? z + f * nz : NULL);
    }
    free(all);
    state_free(s);
    return 0;
}

int or_run(const or_cfg *c, const double *w, int nf, int16_t *y, const int16_t *z,
           int driver, int sched, const uint8_t *const *bs, const long *lens,
           double *mu, double *sigma)
{
    return or_run_lrp(c, w, nf, y, z, driver, sched, bs, lens, mu, sigma, NULL);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
