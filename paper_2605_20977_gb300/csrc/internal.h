// internal.h -- declarations shared by the library's translation units.
// Not part of the public ABI (include/psw.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/psw.h"

namespace psw {

enum Prec { P_F32 = 0, P_BF16 = 1 };

// Device status bits (OR-ed by kernels into a device word).
enum : int { ST_CORRUPT = 1, ST_TIMEOUT = 2, ST_CAPACITY = 4 };

constexpr int NSCALES = 64;
constexpr int CDF_PREC = 16;
constexpr int MAX_KK = 81;        // largest window (9 x 9)
constexpr int MAX_TF = 4;         // frames in a temporal window
constexpr int MAX_SLOTS = 512;    // frames in one batch (token word: slot << 23 | position)
constexpr int POS_BITS = 23;      // raster positions per frame: below 2^23
constexpr int WIDE_M = 1024;      // tokens from which a projection takes the persistent tensor-core kernel

// One frame in flight.  A device-resident table of these lets one launch
// serve tokens of several frames (of different sequences and grids): a token
// is the word (slot << 23) | raster position.  Caches are [layer][stride][d]
// in the compute type; the hyperprior tokens eh are FP32 [stride][d]; stride
// is the sequence's maximum H*W.  (Residual streams are not per-position
// state: a position's stream lives only while its step runs, in compact
// workspace rows, one row per token of the launch.)
struct Slot {
    int H, W, stride, frame, sched;
    int nfr;                       // temporal: frames in the window (<= Tf)
    int ring[MAX_TF];              // their ring positions, oldest first
    float *eh;
    void *qa, *K1, *V1, *K2, *V2, *Ka, *Va;
    void *CK, *CV, *XK, *XV;
    void *LK, *LV;                 // LRP Transformer keys / values [Llrp (x Tf)][stride][d]
    float *rep;                    // LRP: the Spatial Module 2 stream per position, FP32 [stride][d] (or null)
    float *mu, *sigma;
    uint8_t *idx;
    int32_t *m;
    int16_t *y;                    // this frame's latents (input copy or decoded)
    const int16_t *yprev, *zhat;
    const uint8_t *bs;             // decoder input container
    uint64_t len;
    uint32_t *rstate, *rptr, *rend;
    const int *order;              // positions in schedule order
    int *status;
};

__host__ __device__ inline int tok_slot(int t) { return (int)((unsigned)t >> POS_BITS); }
__host__ __device__ inline int tok_pos(int t) { return t & ((1 << POS_BITS) - 1); }
__host__ __device__ inline int tok_make(int slot, int pos) { return (int)(((unsigned)slot << POS_BITS) | (unsigned)pos); }

// Caches a kernel can name.
enum CacheSel { CS_NONE = -1, CS_K1 = 0, CS_V1, CS_K2, CS_V2, CS_KA, CS_VA, CS_QA, CS_CK, CS_CV, CS_XK, CS_XV,
                CS_LK, CS_LV };

// Launch with programmatic dependent launch allowed: the kernel may begin
// while its predecessor in the stream finishes, and must execute
// griddepcontrol.wait before it reads or writes anything that predecessor
// touches (kernels launched this way do so).
template <typename Kern, typename... Args>
inline cudaError_t launch_pdl(Kern k, dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// ---------------------------------------------------------------- GEMM
// Y[m][n] = sum_k A[m][k] * Wt[n][k]  (A compact token-major, Wt the
// transposed projection, both in the compute type), FP32 accumulation in
// ascending k, then one of the epilogues below.  Every output element's
// arithmetic depends only on its own row of A and column of W, never on M or
// on the tile it falls in, so a token gets bit-identical results whether it
// is processed alone (decoder step) or with the whole frame (encoder).
enum EpiMode {
    EPI_STORE = 0,      // out[m][n] = y, or into cache st_sel at the token's position
    EPI_QKV = 1,        // n < q_cols: out[m][n]; then caches kc_sel, vc_sel at the token's position
    EPI_RESID = 2,      // rows[m][n] += y               (FP32 residual stream rows)
    EPI_RESID_BASE = 3, // rows[m][n] = eh[token position][n] + y
    EPI_SWIGLU = 4,     // dual GEMM: out[m][n] = silu(y_gate) * y_up
    EPI_BIAS_SILU = 5,  // out[m][n] = silu(y + bias[n])
    EPI_SET_BIAS = 6,   // rows[m][n] = y + bias[n]
    EPI_HEADS = 7       // rows 2c / 2c+1 give mu_c / sigma_c of the token: channel-wise
                        // scaling, sigma = exp(clamp(.)), then scale index and rounded mean
};

struct Epi {
    int mode;
    const int *tok;               // packed tokens, one per row m
    const Slot *slots;
    int d;                        // width of a cache / stream row
    int q_cols;
    void *out; int ld_out;        // compact output rows
    int kc_sel, vc_sel, kv_layer; // EPI_QKV caches and their layer index
    int ring, Tf;                 // ring = 1: layer kv_layer * Tf + the slot's current ring position
    int st_sel, st_layer;         // EPI_STORE into a cache (CS_NONE: compact out)
    float *rows;                  // EPI_RESID / EPI_RESID_BASE / EPI_SET_BIAS: FP32 rows [M][N]
    const float *bias;            // EPI_BIAS_SILU, EPI_SET_BIAS
    const float *gmu, *bmu, *gsg, *bsg;   // EPI_HEADS channel-wise scale and offset
    const float *scale;           // EPI_HEADS scale table [64]
    int C;                        // EPI_HEADS channels of a position's mu / sigma row
    int c0;                       // EPI_HEADS first channel this projection writes (its N / 2 channels follow)
    int eh_out;                   // EPI_SET_BIAS into the token's hyperprior-token row of its slot instead of rows
    int hr;                       // A_ZHAT: the hyperprior's upsampling factor
};

// Source of the token operand of a GEMM.
enum ASrc {
    A_DIRECT = 0,       // compact rows A[m][lda] in the compute type
    A_NORM = 1,         // RMSNorm(FP32 rows xrows[m]) * a_gain
    A_EMBED = 2,        // a_gain[c] * latent y[c] of the token (the latent embedding input)
    A_ZHAT = 3          // a_gain[c] * z-hat[c] of the token's hyperlatent (position (i, j) of a frame
                        //    whose hyperprior is r times coarser: hyperlatent (i / r, j / r); r = epi.hr)
};

struct GemmArgs {
    const void *A; int lda;       // A_DIRECT: [M][lda]
    int asrc;
    int f8;                       // 1: E4M3 projection: Wt / Wt2 are E4M3 [N][K] bytes, row f of each
                                  //    dequantised by wsc[f] / wsc2[f]; the token operand is quantised
                                  //    per token with a power-of-two scale
    const float *wsc, *wsc2;
    const float *xrows;           // A_NORM: FP32 rows [M][K]
    const float *a_gain;          // A_NORM gain [K]; A_EMBED channel scaling [K]
    void *prep;                   // compact [M][K] scratch for the SIMT path's operand
    const void *Wt;               // [N][K]
    const void *Wt2;              // second operand of a dual GEMM (EPI_SWIGLU)
    int M, N, K;
    Epi epi;
    int *status;                  // device status word (ST_TIMEOUT from bounded waits)
    int tnb;                      // wide kernel's tokens per tile (0: its cost model; else 64, 128 or 256,
                                  //    capped at the largest its epilogue takes)
    const float *xs;              // f8 with streamed E4M3 rows (A_DIRECT, wide kernel): each row's
                                  //    dequantisation scale
};

// Enqueue one GEMM.  BF16 projections whose N and K tile evenly run on the
// tensor cores (the choice never depends on M); everything else on the SIMT
// kernel.  Launches of at least WIDE_M tokens take the persistent
// warp-specialised tensor-core kernel (a BF16 normalised input is then
// normalised once by launch_norm_rows); the tensor-core kernels give
// bit-identical results, so the choice never changes a value.  Returns
// false if the launch could not be prepared.
bool gemm(int prec, const GemmArgs &g, cudaStream_t s);
// dst[m * ldd + k] = bf16(RMSNorm(X[m]) * gain) for m < M, K <= 512 (a
// multiple of 4; ldd 0 means K, else a multiple of 8 and >= K): the
// normalised token operand of a projection whose tiles then stream it
// (A_DIRECT), bit-identical to the operand an A_NORM tile builds.
bool launch_norm_rows(const float *X, const float *gain, int M, int K, void *dst, cudaStream_t s, int ldd = 0);
// dst[m][k] = bf16(gain[k] * y[k]) of the latents of token tok[m] (m < M, K a
// multiple of 4): the latent embedding's operand as an A_EMBED tile builds
// it, for a projection whose tiles stream it.
bool launch_embed_rows(const Slot *S, const int *tok, int M, const float *gain, int K, void *dst, cudaStream_t s);
// E4M3 token rows dst[m][k] (bytes) and their dequantisation scales xs[m]
// for m < M: of RMSNorm(X[m]) * gain (asrc A_NORM, K <= 512) or of the bf16
// rows A[m][lda] (A_DIRECT, K <= 1024), K a multiple of 128; byte-identical
// to the operand an E4M3 tile builds in shared memory.
bool launch_rows8(int asrc, const float *X, const float *gain, const void *A, int lda, int M, int K, uint8_t *dst,
                  float *xs, cudaStream_t s);
// The persistent warp-specialised kernel for launches with many token tiles
// (gemm_ws.cu): BF16, a streamed token operand (A_DIRECT), the epilogues of
// block projections and heads; bit-identical to the one-tile-per-CTA kernel.
bool gemm_ws_supported(const GemmArgs &g);
// Whether gemm() sends this launch to the persistent kernel.
bool gemm_takes_ws(int prec, const GemmArgs &g);
bool gemm_ws(const GemmArgs &g, cudaStream_t s);
bool gemm_ws_prepare();           // kernel attributes, before any capture
bool gemm_tc_supported(int prec, int N, int K, int asrc);
bool gemm_tc8_supported(int N, int K, int asrc);
// E4M3 weights of one tensor: dst[i] = e4m3_rn(src[i] / s) with the
// power-of-two s = 2^(e - 7), max |src| in [2^e, 2^(e+1)) (s = 1 for an
// all-zero tensor); n FP32 values on the device.  Returns s, or a negative
// value on a CUDA error.  Synchronous.
float quantize_e4m3(const float *src, size_t n, uint8_t *dst);
bool gemm_tc_available();         // driver entry point for tensor maps present
void launch_gather_embed(int prec, const Slot *S, const int *tok, int n, const float *gamma, int C, void *dst,
                         cudaStream_t s);
void launch_convert(int prec, const float *src, size_t n, void *dst, cudaStream_t s);

// Pointer to row `pos` of cache `sel`, layer `layer`, of a slot (device).
template <typename T>
__device__ __forceinline__ T *cache_row(const Slot &s, int sel, int layer, int pos, int d)
{
    void *base;
    switch (sel) {
    case CS_K1: base = s.K1; break;
    case CS_V1: base = s.V1; break;
    case CS_K2: base = s.K2; break;
    case CS_V2: base = s.V2; break;
    case CS_KA: base = s.Ka; break;
    case CS_VA: base = s.Va; break;
    case CS_QA: base = s.qa; break;
    case CS_CK: base = s.CK; break;
    case CS_CV: base = s.CV; break;
    case CS_XK: base = s.XK; break;
    case CS_LK: base = s.LK; break;
    case CS_LV: base = s.LV; break;
    default: base = s.XV; break;
    }
    return (T *)base + ((long)layer * s.stride + pos) * d;
}


// ---------------------------------------------------------------- kernels
// One device-to-device copy of a batch's copy kernel.
struct CopyJob {
    const void *src;
    void *dst;
    unsigned long long bytes;
};
// jobs[0 .. n) (a device array) in one launch: 16-byte words where both
// addresses are 16-byte aligned, bytes otherwise.
void launch_copy_jobs(const CopyJob *jobs, int n, unsigned long long max_bytes, cudaStream_t s);
void launch_transpose_convert(int prec, const float *src, int K, int N, void *dst, int row_off,
                              cudaStream_t s);
// Context Transformer input rows out[m] of each token from the previous
// frame's latents (temporal shift), or the learned pad for frame 0.
void launch_embed_context(const Slot *S, const int *tok, int n, int C, const float *gamma, const float *W,
                          const float *b, const float *pad, int d, float *out, cudaStream_t s);
void launch_embed_hyper(const Slot *S, const int *tok, int n, int H, int W, int Ch, int r, const float *gamma,
                        const float *Whp, const float *b, int d, cudaStream_t s);
// The same for slots 0 .. nslots - 1 of the table in one launch (each slot's
// own grid, at most Hmax x Wmax): every element as launch_embed_hyper
// computes it.
void launch_embed_hyper_batch(const Slot *S, int nslots, int Hmax, int Wmax, int Ch, int r, const float *gamma,
                              const float *Whp, const float *b, int d, cudaStream_t s);
// dst[w * ldd + e] = RMSNorm(X[w]) * g in the compute type (ldd 0: d); the
// SIMT path's operand.
void launch_rmsnorm(int prec, const float *X, int n, const float *g, int d, void *dst, cudaStream_t s, int ldd = 0);
// rep[position * ld + off + e] = X[m * w + e] (e < w; w, ld, off multiples
// of 4) for each token m of a slot whose rep pointer is set: the heads'
// input kept for the LRP Transformer.
void launch_store_rows(const Slot *S, const int *tok, int n, const float *X, int w, int ld, int off, cudaStream_t s);
// Channel Transformer, channel shift: X[m][e] += sum_c (gamma[c] y[c0 + c])
// E[c][e] over the Cg latents of the previous channel group at the token's
// position (FP32, c ascending), e < dg.
void launch_ct_embed(const Slot *S, const int *tok, int n, int C, int c0, int Cg, const float *gamma, const float *E,
                     int dg, float *X, cudaStream_t s);

struct AttnArgs {
    const int *tok; int n;
    const Slot *slots;
    const void *Q; int q_sel;       // compact [n][d], or cache q_sel (CS_QA) at the token's position
    int k_sel, v_sel;               // key / value caches
    int layer;                      // spatial: layer index; temporal: block index (ring layer = layer*Tf + ring)
    int temporal;                   // 1: keys over the slot's frame ring, unmasked windows
    int Tf;
    const float *bias;              // + h * bias_h_stride + age * k*k + window offset
    int bias_h_stride;
    void *O;                        // compact [n][d]
    int d, nh, k;
    int mask;                       // 0: 2i+j with raster clause, 1: cyclic
    int kind;                       // 0: accumulator A(p), 1: self-attention S(p), -1: window
};
void launch_attention(int prec, const AttnArgs &a, cudaStream_t s);
bool attention_prepare();          // kernel attributes, before any capture

void launch_quantize(size_t n, const float *mu, const float *sigma, const float *scale,
                     uint8_t *idx, int32_t *m, cudaStream_t s);
void launch_rate(size_t n, const int16_t *y, const float *mu, const float *sigma, double *partials,
                 double *out, cudaStream_t s);
int rate_partials(size_t n);

// ---------------------------------------------------------------- coding
struct CdfTables {
    float scale[NSCALES];
    int T[NSCALES], n[NSCALES], off[NSCALES];
    int total;                               // slots over all tables
    uint32_t *packed;                        // host: cum | freq << 16
};
void build_scale_table(float *tab);
void build_cdf_tables(CdfTables &t);        // allocates t.packed (free with free_cdf_tables)
void free_cdf_tables(CdfTables &t);

struct CoderDev {
    const uint32_t *cdf;                     // packed slots
    const int *meta;                         // [3][nt]: T, n, off of each table
    int nt = NSCALES;                        // tables (the scale tables; the factorized prior: one per channel)
};
size_t container_capacity(int H, int W, int C);
// Encoder of one slot: symbols y / idx / m and the schedule order from the slot.
void launch_rans_encode(const CoderDev &cd, const Slot *S, int slot, int HW, int C, uint16_t *scratch,
                        int cap_words, uint32_t *nwords, uint32_t *states, cudaStream_t s);
void launch_rans_assemble(int H, int W, int C, int sched, const uint16_t *scratch, int cap_words,
                          const uint32_t *nwords, const uint32_t *states, uint8_t *out, size_t cap,
                          uint64_t *total, int *status, cudaStream_t s);
// Validate each slot's container (bs, len, H, W, sched) and load its states.
void launch_rans_dec_init(const Slot *S, int nslots, int C, cudaStream_t s);
// kn[b] = (first symbol, count) of slot b in this step (count 0: idle).
// Channels [c0, c0 + nc) only (nc = C: every channel).
void launch_rans_dec_step(const CoderDev &cd, const Slot *S, int nslots, const int2 *kn, int C, cudaStream_t s,
                          int c0 = 0, int nc = -1);
void launch_rans_dec_finish(const Slot *S, int nslots, int C, cudaStream_t s);


// ---------------------------------------------------------------- hyperprior (hyper.cu)
// Token operand of a convolution over the FP32 grid src (logical [h][w][C];
// view 1: the pixel-shuffle source of [h/2][w/2] positions ls floats apart,
// ls 0 meaning 4C): ks = 3: every 3 x 3 tap at stride st, zero padded
// (K = 9C, tap-major); ks = 1: the tap (st i, st j) (K = C); LeakyReLU
// (0.01) first when act; rows of ceil(h/st) x ceil(w/st) positions in
// raster order, compute type.
void launch_im2col(int prec, const float *src, int h, int w, int C, int view, int ls, int act, int ks, int st,
                   void *dst, cudaStream_t s);
// dst [2h][2w][C] = pixel shuffle of src ([h][w] positions ls floats apart).
void launch_shuffle(const float *src, int h, int w, int C, int ls, float *dst, cudaStream_t s);
// gamma * z-hat of the slot of tok[0] (n hyperprior positions x Ch) as FP32.
void launch_zhat_grid(const Slot *S, const int *tok, int n, const float *gamma, int Ch, float *dst, cudaStream_t s);
// The slot's hyperprior tokens: the top-left H x W of a grid of row width ws.
void launch_crop_eh(const Slot *S, const int *tok, const float *src, int ws, int H, int W, int d, cudaStream_t s);
// z-hat = round-half-even(z), clamped to int16; zout (may be null) = z.
void launch_round_z(const float *z, long n, int16_t *zhat, float *zout, cudaStream_t s);
// z-hat coder inputs: table index = channel, mean 0, raster order.
void launch_hyper_coder_tables(int HW, int Ch, uint8_t *idx, int32_t *m, int *order, cudaStream_t s);

// ---------------------------------------------------------------- persistent decoder
// One phase of a wavefront step, as the persistent decoder runs it: a
// projection, a window attention or the rANS step.  A phase works either on
// the positions of the current step (the accumulator, Spatial Module 2, the
// heads and the coder) or on those of the previous step (Spatial Module 1 and
// the accumulator keys/values, which need their just-decoded latents); the
// kernel fills in the token list and count of each step (GemmArgs.M and
// epi.tok, AttnArgs.tok and n, kn).
enum OpType { OP_GEMM = 0, OP_ATTN = 1, OP_RANS = 2 };
enum TokSet { TS_CUR = 0, TS_PREV = 1 };

struct Op {
    int type, tokset;
    int dual;                      // OP_GEMM: SwiGLU dual form
    int wmap, wmap2, xmap;         // OP_GEMM: indices into the tensor-map table (-1: none)
    const int2 *kn;                // OP_RANS: this step's (first symbol, count) per slot
    GemmArgs g;                    // OP_GEMM
    AttnArgs a;                    // OP_ATTN
};

struct PersistArgs {
    const Op *ops; int nops;
    const void *maps;              // CUtensorMap table (64-byte aligned)
    int nmaps;
    const int *tok;                // token lists of every step
    const int *step_off, *step_n;  // per global step: offset into tok, count
    const int2 *kn; int nslots;    // per step and slot: (first symbol, count)
    CoderDev cd;
    const Slot *slots;
    int C;
    int t0, t1;                    // global steps to run
    unsigned *bar;                 // grid-barrier counter (zero at launch)
    int *abort_g;                  // set by a CTA whose bounded wait expired
    int *status;                   // context status word
};

// Host-side builder of a decoder program (the phases of one step).
struct ProgramBuilder;
ProgramBuilder *program_new(int ws_rows);
void program_free(ProgramBuilder *b);
bool program_gemm(ProgramBuilder *b, const GemmArgs &g, int tokset);
void program_attn(ProgramBuilder *b, const AttnArgs &a, int tokset);
void program_rans(ProgramBuilder *b);
// Upload the program and its tensor maps; the device arrays stay valid until
// program_free.  Returns false on a CUDA error.
bool program_upload(ProgramBuilder *b, const Op **ops, int *nops, const void **maps, int *nmaps, size_t *smem,
                    bool *f8);
// Kernel attributes and the grid (one CTA per SM, all co-resident) for a
// dynamic shared-memory size; false if that cannot be resident.
bool persist_prepare(size_t smem, bool f8, int *grid);
bool persist_launch(const PersistArgs &a, int grid, size_t smem, bool f8, cudaStream_t s);
// The grid barrier's bounded wait on a count nothing reaches (limit_ns), its
// expiry ORed into *status as ST_TIMEOUT; false on a CUDA error.
bool wait_probe(uint64_t limit_ns, int *status, cudaStream_t s);

}  // namespace psw

// The coder tables of a context (for entry points outside api.cu): channels,
// mask, device CDF slots and table metadata.  False for a null context.
bool psw_coder_view(const psw_ctx *ctx, int *C, int *mask, const uint32_t **cdf, const int **meta);

namespace psw {

}  // namespace psw
