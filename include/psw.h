/*
 * psw.h -- C ABI of the GB300 (sm_103a) implementation of the P-SWA
 * entropy model's hot path: diagonal-wavefront decoding of the
 * sliding-window-attention context model of "Parallel Context Modeling for
 * Sliding Window Attention in Neural Video Coding" (Kopte & Kaup).
 *
 * The library computes, for every latent symbol y(i,j,c) of a frame, the
 * Gaussian parameters (mu, sigma) the context model assigns to it given the
 * decoded hyperprior, the previously decoded positions of the frame and (for
 * the temporal model) previous frames (Sec. 3.1, Fig. 1).  The encoder
 * evaluates every position in one masked parallel pass; the decoder walks the
 * step labels l(i,j) = 2i+j (one diagonal wavefront per step, Sec. 2 and
 * Sec. 3.2) or raster order, predicting all positions of a step together
 * (Sec. 3.2, Fig. 2).  sigma is quantised to a 64-entry log-spaced scale
 * table; integer CDFs of the quantised Gaussian drive 32-lane interleaved
 * rANS, standing in for the "AE/AD" boxes of Fig. 1.
 *
 * Conventions for every call:
 *  - Tensors are channel-last and contiguous: latents y [H][W][C] int16,
 *    hyperlatents z [ceil(H/r)][ceil(W/r)][Ch] int16, mu/sigma [H][W][C]
 *    float32.  Pointers named *_dev are CUDA device pointers; *_host are
 *    host pointers.  The caller owns every pointer it passes; the library
 *    never frees or keeps them beyond the call.
 *  - The library owns its weights, CDF tables, per-sequence caches and all
 *    scratch memory.  Nothing is allocated per call except where stated.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it; calls that return a host-side result (a length, a bit
 *    count, a decode status) synchronise that stream before returning.
 *  - No exception crosses the ABI.  Every call returns a psw_status; the
 *    message of the last failure on a context is psw_last_error(ctx).
 *  - A context may be used by one host thread at a time.
 */
#ifndef PSW_H
#define PSW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct psw_ctx psw_ctx;   /* model weights + tables (opaque) */
typedef struct psw_seq psw_seq;   /* one video sequence's caches (opaque) */

typedef enum {
    PSW_OK = 0,
    PSW_ERR_INVALID = 1,   /* bad argument, shape or descriptor            */
    PSW_ERR_OOM = 2,       /* device allocation failed / budget exceeded   */
    PSW_ERR_CUDA = 3,      /* a CUDA runtime call failed                   */
    PSW_ERR_CORRUPT = 4,   /* bitstream fails validation while decoding    */
    PSW_ERR_TIMEOUT = 5,   /* a bounded device-side wait ran out           */
    PSW_ERR_CAPACITY = 6   /* output buffer too small                      */
} psw_status;

/* PSW_FP8: the projections run on E4M3 operands with FP32 accumulation --
 * weights quantised once per projection with a power-of-two scale, the
 * token operand quantised per token with a power-of-two scale computed from
 * that token's row alone (so a token's result never depends on the other
 * tokens of a launch); everything else (caches, attention, norms, residual
 * streams, heads' epilogue) is as in PSW_BF16. */
typedef enum { PSW_FP32 = 0, PSW_BF16 = 1, PSW_FP8 = 2 } psw_precision;

typedef enum {
    PSW_SCHED_WAVEFRONT = 0,   /* one step per label value, all positions of the step together */
    PSW_SCHED_RASTER = 1       /* one position per step, raster order (same model, same masks) */
} psw_schedule;

/* Model hyper-parameters (Sec. 3.1 block structure; Sec. 4.1 sizes).
 *   C      latent channels            Ch, r  hyperprior channels, upsampling
 *   d, nh  model width, heads         F      SwiGLU hidden width
 *   L      blocks per spatial module (Spatial Module 1 and 2; plus one
 *          accumulator block)          k      spatial window (k x k, odd)
 *   temporal  1 = Context Transformer (Lc blocks) and temporal
 *          cross-attention over Tf frames in every spatial block
 *   mask   0 = label 2i+j with the raster clause (wavefront and raster
 *          schedules valid); 1 = cyclic s = 4 label of Fig. 2a.
 *   Llrp   blocks of the LRP Transformer (Sec. 3.1 latent residual
 *          prediction; 0 = none, at most 64), run by psw_lrp_residual.
 *   Nc     channel groups of the Channel Transformer (Sec. 3.1; Sec. 3.2:
 *          the decoder runs N channel-group sub-steps per spatial step;
 *          0 = none: the heads read Spatial Module 2 directly).  With Nc > 0:
 *          C and dc divisible by Nc, dg = dc / Nc a multiple of 64 and at
 *          most 512;
 *   dc     its width; Lct its blocks (1..16); Fc the SwiGLU hidden width of
 *          each group (a multiple of 64).  All four are 0 without it.
 *   hp     1 = convolutional hyperprior (Fig. 1 right): psw_hyper_encode
 *          computes z-hat from the frame (log2 r downsampling residual
 *          blocks on Spatial Module 1's output) and codes it under a
 *          factorized prior, psw_hyper_decode decodes it, and the
 *          hyperprior tokens come from log2 r upsampling residual blocks
 *          (r a power of two, Ch <= 256); 0 = z-hat is an input embedded by a
 *          transposed convolution. */
typedef struct {
    int C, Ch, r;
    int d, nh, F, L, k;
    int temporal, Lc, Tf;
    int mask;
    int Llrp;
    int Nc, dc, Lct, Fc;
    int hp;
} psw_model_desc;

/* One frame: latent grid H x W (hyperprior grid ceil(H/r) x ceil(W/r)) and
 * the decoding schedule (psw_schedule) the bitstream is ordered by. */
typedef struct {
    int H, W;
    int schedule;
} psw_frame_desc;

/* Number of float32 values in the flat weight vector of a model.
 * Packing order (every projection stored [in][out], used as x . W):
 *   gamma_in[C] W_in[C][d] b_in[d] gamma_z[Ch]
 *   if hp (nb = log2 r residual blocks per direction):
 *          g_za[d]
 *          nb x RB-down { Wa[3][3][Ci][Ch] ba[Ch] Wb[3][3][Ch][Ch] bb[Ch] Ws[Ci][Ch] bs[Ch] }
 *             (Ci = d for the first block, else Ch)
 *          nb x RB-up { Wa[3][3][Ch][4Co] ba[4Co] Wb[3][3][Co][Co] bb[Co]
 *             Ws[3][3][Ch][4Co] bs[4Co] } (Co = d for the last block, else Ch;
 *             the 4Co outputs of a sub-pixel convolution are the 2 x 2
 *             sub-positions a, b at channel (2a + b) Co + c)
 *          factorized prior per channel: H1[Ch][3] b1[Ch][3] a1[Ch][3]
 *             H2[Ch][3][3] b2[Ch][3] a2[Ch][3] H3[Ch][3][3] b3[Ch][3] a3[Ch][3]
 *             H4[Ch][3] b4[Ch]
 *   else   W_hp[r*r][Ch][d] b_hp[d]
 *   if temporal: gamma_c[C] W_c[C][d] b_c[d] pad[d]
 *                Lc x { g_attn[d] Wq Wk Wv Wo [d][d] bias[nh][Tf][k][k]
 *                       g_ffn[d] Wg[d][F] Wu[d][F] Wd[F][d] }  g_ctx[d]
 *   L x Spatial Module 1 block:
 *     { g_attn[d] Wq Wk Wv Wo [d][d] bias[nh][k][k]
 *       if temporal: g_x[d] Wxq Wxk Wxv Wxo [d][d] xbias[nh][Tf][k][k]
 *       g_ffn[d] Wg[d][F] Wu[d][F] Wd[F][d] }
 *   accumulator: g_q[d] g_kv[d] Wq Wk Wv Wo [d][d] bias[nh][k][k]
 *                g_ffn[d] Wg[d][F] Wu[d][F] Wd[F][d]
 *   L x Spatial Module 2 block (as Spatial Module 1)
 *   if Nc (the Channel Transformer; dg = dc/Nc, Cg = C/Nc):
 *          g_in[d] W_in[d][dc] b_in[dc] gamma_y[C] E[Nc-1][Cg][dg]
 *          Lct x { g_mix[dc] M[dc][dc] g_ffn[dc] Wg[Nc][dg][Fc] Wu[Nc][dg][Fc]
 *                  Wd[Nc][Fc][dg] }   (M's entries from a later input group
 *                  than the output group are ignored: the causal mask)
 *     heads: g_head[dc] W1m[Nc][dg][dg] b1m[dc] W2m[Nc][dg][Cg] W1s[Nc][dg][dg]
 *          b1s[dc] W2s[Nc][dg][Cg] gamma_mu[C] beta_mu[C] gamma_sig[C] beta_sig[C]
 *   else heads: g_head[d] W1m[d][d] b1m[d] W2m[d][C] W1s[d][d] b1s[d] W2s[d][C]
 *          gamma_mu[C] beta_mu[C] gamma_sig[C] beta_sig[C]
 *   if Llrp (the LRP Transformer; dh = dc with a Channel Transformer, else d):
 *          g_rep[dh] W_rep[dh][d] gamma_y[C] W_y[C][d] b_in[d]
 *          Llrp x { g_attn[d] Wq Wk Wv Wo [d][d] bias[nh][k][k] (temporal:
 *                   bias[nh][Tf][k][k]) g_ffn[d] Wg[d][F] Wu[d][F] Wd[F][d] }
 *          g_out[d] W_eps[d][C] b_eps[C]
 * Returns 0 for an invalid descriptor. */
size_t psw_weights_count(const psw_model_desc *desc);

/* Create a context: validates the descriptor, uploads the weights (host
 * float32, psw_weights_count values) to the current CUDA device, converts
 * block projections to the compute precision (PSW_FP32 or PSW_BF16,
 * round-to-nearest-even; PSW_FP8: every transformer-block projection whose
 * shape the E4M3 tile takes -- K a multiple of 128, at most 512 for a
 * normalised input and 1024 for the FFN down projection -- as E4M3 bytes,
 * each source tensor with its own power-of-two scale as psw_quantize_e4m3
 * computes it; the latent embedding, the heads, the Channel and LRP
 * Transformers and any other projection in BF16) and builds the scale and
 * CDF tables.
 * hbm_budget bounds the device memory of this context and its sequences
 * (0 = no bound); a sequence that would exceed it fails with PSW_ERR_OOM.
 * On failure *out is NULL. */
psw_status psw_create(const psw_model_desc *desc, const float *weights_host, size_t n_weights,
                      int precision, size_t hbm_budget, psw_ctx **out);
void psw_destroy(psw_ctx *ctx);

/* Message of the last failure on ctx ("" if none).  Valid until the next
 * call on ctx.  psw_last_error(NULL) reports failures of psw_create. */
const char *psw_last_error(const psw_ctx *ctx);

/* Device bytes held by the context (weights, tables) and, for a sequence
 * of the given maximum grid, by one sequence (caches and scratch). */
size_t psw_ctx_bytes(const psw_ctx *ctx);
size_t psw_seq_bytes(const psw_ctx *ctx, int max_H, int max_W);

/* A sequence owns the per-frame caches (window K/V of every layer, residual
 * streams, step scratch) for frames up to max_H x max_W and, for the
 * temporal model, the rings of the last Tf frames' context K/V (Sec. 3.1:
 * the Context Transformer and temporal cross-attention see previous
 * frames).  Frames must be coded in order; psw_encode_params and
 * psw_decode_frame advance it identically.  psw_seq_reset starts a new
 * sequence (the next frame is frame 0, whose temporal context is the learned
 * padding vector).  max_H and max_W are 1..4096 with max_H * max_W < 2^23
 * (PSW_ERR_INVALID otherwise). */
psw_status psw_seq_create(psw_ctx *ctx, int max_H, int max_W, psw_seq **out);
psw_status psw_seq_reset(psw_seq *seq);
void psw_seq_destroy(psw_seq *seq);

/* Upper bound on the container size of one frame (bytes). */
size_t psw_bitstream_capacity(const psw_ctx *ctx, const psw_frame_desc *fd);

/* Encoder (Sec. 3.1: the accumulator's keys are limited to positions
 * decoded earlier; Sec. 3.2): one masked parallel pass over every position of
 * the frame gives (mu, sigma); sigma -> scale index, mu -> rounded mean;
 * symbols y - round(mu) are rANS-coded per channel in the schedule's order.
 *   yhat_dev  [H][W][C] int16 latents of this frame
 *   zhat_dev  [ceil(H/r)][ceil(W/r)][Ch] int16 decoded hyperlatents
 *   mu_dev, sigma_dev  optional [H][W][C] float32 outputs (NULL to skip)
 *   bitstream_dev  optional device buffer of cap bytes for the container
 *                  (NULL: parameters only, *len_out set to 0)
 *   len_out   host: container size in bytes
 * Errors: PSW_ERR_INVALID (shape), PSW_ERR_CAPACITY (cap too small; the
 * sequence still advances), PSW_ERR_CUDA.  Synchronises `stream`. */
psw_status psw_encode_params(psw_ctx *ctx, psw_seq *seq, const psw_frame_desc *fd,
                             const int16_t *yhat_dev, const int16_t *zhat_dev,
                             float *mu_dev, float *sigma_dev,
                             uint8_t *bitstream_dev, size_t cap, size_t *len_out, void *stream);

/* Decoder (Sec. 3.2, Fig. 2): for each step of the schedule, Spatial
 * Module 1 runs on the positions decoded in the previous step, then the
 * accumulator, Spatial Module 2 and heads run on all positions of the step
 * together, their symbols are rANS-decoded and written to yhat.  With a
 * Channel Transformer the step ends in Nc sub-steps: the Channel
 * Transformer and heads of channel group g, then the rANS decode of that
 * group's channels (their latents feed group g + 1).
 *   bitstream_dev  device container of len bytes (from psw_encode_params)
 *   zhat_dev       hyperlatents as for the encoder
 *   yhat_out_dev   [H][W][C] int16 decoded latents
 *   mu_dev, sigma_dev  optional float32 outputs (NULL to skip)
 * Returns PSW_ERR_CORRUPT if the container fails validation (header,
 * offsets, a read past a stream's end, a final state other than the initial
 * one, a latent outside int16); the outputs are then unspecified but every
 * device access stayed in bounds.  Synchronises `stream`. */
psw_status psw_decode_frame(psw_ctx *ctx, psw_seq *seq, const psw_frame_desc *fd,
                            const uint8_t *bitstream_dev, size_t len, const int16_t *zhat_dev,
                            int16_t *yhat_out_dev, float *mu_dev, float *sigma_dev, void *stream);

/* Batched decode: n frames of n different sequences (any mix of grids and
 * schedules up to each sequence's maximum, 1 <= n <= 512) decoded together:
 * step t of every frame runs in global step t, so each launch carries the
 * positions of all frames (Sec. 3.2 parallelism across frames as well as
 * along a wavefront).  Arrays have n entries; mu_dev / sigma_dev may be NULL
 * or hold NULL entries.  Every frame's results are bit-identical to decoding
 * it alone with psw_decode_frame.  status_out (host, n entries, may be NULL)
 * receives each frame's status; the call returns the first failure.  The
 * first call for a given set of sequences and grids records the launches in
 * a CUDA graph that later calls replay. */
psw_status psw_decode_batch(psw_ctx *ctx, int n, psw_seq *const *seqs, const psw_frame_desc *fds,
                            const uint8_t *const *bitstreams_dev, const size_t *lens,
                            const int16_t *const *zhat_dev, int16_t *const *yhat_out_dev,
                            float *const *mu_dev, float *const *sigma_dev,
                            int *status_out, void *stream);

/* Convolutional hyperprior, encoder side (Fig. 1 right; hp = 1): for the
 * next frame of seq (the one psw_encode_params codes next; the sequence
 * does not advance), Spatial Module 1 over every position with the frame's
 * latents (after the Context Transformer for the temporal model), then
 * RMSNorm and nb downsampling residual blocks (a 3 x 3 convolution of
 * stride 2 and LeakyReLU 0.01, a 3 x 3 convolution, plus a 1 x 1
 * convolution of stride 2) give z; z-hat = round-half-even(z) (int16).
 * z-hat is coded by interleaved rANS under the factorized prior: per
 * channel the cumulative c(x) = sigmoid(f4(f3(f2(f1(x))))), f_k(v) =
 * g_k(softplus(H_k) v + b_k), g_k(t) = t + tanh(a_k) tanh(t) (k < 4), f4
 * affine, widths 1-3-3-3-1; the table of channel c holds slots -31..31 and
 * an escape, freq = 1 + floor(P (2^16 - 64)) with the remainder on 0; the
 * container has the latent containers' format (raster order over the
 * ceil(H/r) x ceil(W/r) grid, one stream per hyperprior channel).
 *   yhat_dev   [H][W][C] int16 latents of the frame
 *   zhat_dev   [ceil(H/r)][ceil(W/r)][Ch] int16 output
 *   z_dev      optional float32 output of the unrounded z (NULL to skip)
 *   bitstream_dev  optional device buffer of cap bytes for the z-hat
 *              container (NULL: analysis only, *len_out 0)
 * Errors: PSW_ERR_INVALID (no convolutional hyperprior, shape),
 * PSW_ERR_CAPACITY, PSW_ERR_CUDA.  Synchronises `stream`. */
psw_status psw_hyper_encode(psw_ctx *ctx, psw_seq *seq, const psw_frame_desc *fd, const int16_t *yhat_dev,
                            int16_t *zhat_dev, float *z_dev, uint8_t *bitstream_dev, size_t cap, size_t *len_out,
                            void *stream);

/* Decoder side: z-hat of a frame with grid fd from its container (len
 * bytes, 4-byte aligned device memory) into zhat_dev; PSW_ERR_CORRUPT if the
 * container fails validation (as for the latent containers).  z-hat then
 * goes to psw_decode_frame / psw_decode_batch, whose hyperprior tokens come
 * from the upsampling residual blocks.  Synchronises `stream`. */
psw_status psw_hyper_decode(psw_ctx *ctx, const psw_frame_desc *fd, const uint8_t *bitstream_dev, size_t len,
                            int16_t *zhat_dev, void *stream);

/* Frequency table of hyperprior channel ch of the factorized prior (64
 * slots: -31..31, escape; sum 2^16).  Host output. */
psw_status psw_prior_table(const psw_ctx *ctx, int ch, uint32_t *freq_host, int cap, int *n_out);

/* LRP Transformer (Sec. 3.1 latent residual prediction; Sec. 4.3): the
 * residual eps of the sequence's last coded frame, from the quantised
 * latents of that frame and the model's final representation at every
 * position (the heads' input: the Channel Transformer's stream if the model
 * has one, else the Spatial Module 2 stream; kept per position by
 * psw_encode_params and the decoders of a context with Llrp > 0).
 * Its input token is RMSNorm(representation) . W_rep + (gamma_y * yhat) . W_y
 * + b_in; Llrp blocks of window self-attention over the whole k x k window
 * (no prediction mask: the frame is decoded) and SwiGLU; then
 * eps = RMSNorm(.) . W_eps + b_eps.  For the temporal model the windows also
 * cover the same window of the Tf - 1 previous frames (time-causal; each
 * block's keys and values are kept per sequence in a ring of Tf frames), so
 * the LRP of every coded frame must run, in order: once per frame, after
 * that frame is coded and before the next one is.
 *   fd       the grid of the last coded frame
 *   eps_dev  [H][W][C] float32 output (may be NULL for the temporal model:
 *            the ring advances, nothing is written)
 * The encoder's and the decoder's residuals are bit-identical.
 * Errors: PSW_ERR_INVALID if the model has no LRP Transformer, no frame was
 * coded since the sequence was created or reset, fd's grid is not the last
 * coded frame's, or (temporal model) the LRP of an earlier frame was
 * skipped or that of this frame already ran; PSW_ERR_CUDA.  Synchronises
 * `stream`. */
psw_status psw_lrp_residual(psw_ctx *ctx, psw_seq *seq, const psw_frame_desc *fd, float *eps_dev,
                            void *stream);

/* Model rate of a frame (Fig. 1 rate term): bits = -sum log2 P(y) with
 * P(y) the Gaussian mass of [y - 1/2, y + 1/2] under (mu, sigma), sigma
 * clamped to [0.11, 256], P floored at 1e-9; FP64, fixed reduction order.
 * n symbols; bits_out_host receives the sum.  Synchronises `stream`. */
psw_status psw_rate(psw_ctx *ctx, size_t n, const int16_t *yhat_dev, const float *mu_dev,
                    const float *sigma_dev, double *bits_out_host, void *stream);

/* Quantisation step alone: idx = smallest l with scale[l] >= sigma (float
 * compare; 63 if none), m = round-half-even(clamp(mu, -32768, 32767)).
 * n values; idx_dev uint8, m_dev int32.  Asynchronous. */
psw_status psw_quantize(psw_ctx *ctx, size_t n, const float *mu_dev, const float *sigma_dev,
                        uint8_t *idx_dev, int32_t *m_dev, void *stream);

/* Failure-detection check (not part of the method): runs the persistent
 * decoder's bounded grid-barrier wait on a barrier no block arrives at, with
 * a limit of `seconds` (0 < seconds <= 10) instead of the decoder's ~2 s.
 * The expiry is reported through the context's status word, as a decode
 * reports one.  Returns PSW_ERR_TIMEOUT when the wait expired (the expected
 * outcome) and PSW_OK if it did not; the context stays usable.  Synchronous,
 * default stream. */
psw_status psw_check_wait_timeout(psw_ctx *ctx, double seconds);

/* E4M3 quantisation of one weight tensor as PSW_FP8 contexts store it
 * (Sec. 3.2 precision forms): with max |src| in [2^e, 2^(e+1)) the scale is
 * s = 2^(e-7) (e clamped at -100; s = 1 for an all-zero tensor) and
 * dst[i] = E4M3(src[i] / s), round to nearest even, so |src[i] / s| < 256.
 * src_dev: n float32 on the device (16-byte aligned); dst_dev: n bytes on the
 * device (4-byte aligned).  *scale_out = s (host).  Synchronous.
 * PSW_ERR_INVALID for NaN or Inf among the values. */
psw_status psw_quantize_e4m3(size_t n, const float *src_dev, uint8_t *dst_dev, float *scale_out);

/* The scale table (64 float32) and CDF table l: freq[n] for slots
 * -T..T, ESC (n = 2T+2, sum 2^16).  Host outputs. */
psw_status psw_scale_table(const psw_ctx *ctx, float *table_host);
psw_status psw_cdf_table(const psw_ctx *ctx, int l, uint32_t *freq_host, int cap, int *n_out, int *T_out);

/* Coder alone, with caller-supplied per-symbol scale index and rounded mean
 * ([H][W][C] each): encode y into a container, or decode a container into y.
 * Encoding: *len_out = container size (PSW_ERR_CAPACITY if > cap).
 * Decoding: PSW_ERR_CORRUPT as for psw_decode_frame.  Synchronise `stream`. */
psw_status psw_rans_encode(psw_ctx *ctx, psw_seq *seq, const psw_frame_desc *fd,
                           const int16_t *yhat_dev, const uint8_t *idx_dev, const int32_t *m_dev,
                           uint8_t *bitstream_dev, size_t cap, size_t *len_out, void *stream);
psw_status psw_rans_decode(psw_ctx *ctx, psw_seq *seq, const psw_frame_desc *fd,
                           const uint8_t *bitstream_dev, size_t len, const uint8_t *idx_dev,
                           const int32_t *m_dev, int16_t *yhat_out_dev, void *stream);

/* Coder-only encoder that allocates no device memory (the paper has no
 * counterpart: this is a deployment convenience).  Some callers cannot call
 * cudaMalloc at the point where they encode: processes whose device memory
 * is handed out entirely by another allocator (a framework's caching pool)
 * or capped by a quota, and latency-critical loops that forbid allocation
 * after warm-up.  This entry point does the
 * work of psw_rans_encode (same inputs, same container bytes) without a
 * psw_seq: its scratch (schedule order, word buffers, stream lengths,
 * states) lives in one static device array of about 9.2 MiB that every GPU
 * loading this library holds until the process exits.
 *   Limits: H*W <= 32768, C <= 256, H*W*C <= 1572864 (one 68 x 120 x 192
 *   latent frame); larger frames return PSW_ERR_INVALID.
 *   The first call on a device looks up the array's device address for that
 *   device.
 *   Every call shares the array (the previous call's contents remain; the
 *   call clears what it needs), so calls whose GPU work overlaps -- on two
 *   streams, or from two host threads -- race; serialise them.
 *   Calls no cudaMalloc/cudaFree and no allocating library routine.
 *   Returns PSW_ERR_CAPACITY if the container exceeds cap (len_out still
 *   receives its size, and no byte of bitstream_dev is written).
 *   Each call copies the schedule order and a slot record from host memory
 *   to the array, reads the length and status back into host memory, and
 *   synchronises `stream` before it returns. */
psw_status psw_rans_encode_noalloc(const psw_ctx *ctx, const psw_frame_desc *fd, const int16_t *yhat_dev,
                                   const uint8_t *idx_dev, const int32_t *m_dev, uint8_t *bitstream_dev,
                                   size_t cap, size_t *len_out, void *stream);

/* Decode engine (not in the paper; an implementation choice).  Both engines
 * run the same per-tile arithmetic, so their results are bit-identical.
 *   PSW_ENGINE_GRAPH       every phase of every step is its own kernel, the
 *                          launches recorded once per batch shape in CUDA
 *                          graphs and replayed.
 *   PSW_ENGINE_PERSISTENT  one cooperative launch, one block per SM, walks
 *                          all steps (Sec. 3.2 schedule) with a grid-wide
 *                          barrier between phases; nothing is recorded per
 *                          batch shape, so it suits batches that change
 *                          from call to call; BF16 and FP8 contexts.
 *   PSW_ENGINE_AUTO        the graph engine (the faster of the two on the
 *                          1080p configurations measured; the default).
 * psw_set_engine returns PSW_ERR_INVALID for an unknown engine or for
 * PSW_ENGINE_PERSISTENT on an FP32 context; a decode asked to run
 * persistently on a device that cannot co-schedule the blocks returns
 * PSW_ERR_CUDA; the persistent engine does not run contexts with an LRP or a
 * Channel Transformer (PSW_ERR_INVALID).  psw_last_engine: the engine of the context's last decode
 * (0 = individual launches, as under psw_profile_begin). */
typedef enum { PSW_ENGINE_AUTO = 0, PSW_ENGINE_GRAPH = 1, PSW_ENGINE_PERSISTENT = 2 } psw_engine;
psw_status psw_set_engine(psw_ctx *ctx, int engine);
int psw_last_engine(const psw_ctx *ctx);

/* Tile policy of the persistent warp-specialised projection kernel (not in
 * the paper; an implementation choice the autotuner makes): tokens per tile
 * (64, 128 or 256; 0 = the library's cost model) for each launch class --
 * QKV projections, residual projections (attention output, FFN down,
 * accumulator output), the SwiGLU gate/up pair, and the rest.  A width the
 * class's epilogue cannot take is capped.  Every width gives bit-identical
 * results (one accumulator per output, K in ascending order), so the policy
 * changes only speed.  Setting it synchronises the device and drops the
 * recorded decode graphs.  PSW_ERR_INVALID for an unknown class or width;
 * psw_tile_policy returns the current value (-1 for a bad argument). */
typedef enum { PSW_TILE_QKV = 0, PSW_TILE_RESIDUAL = 1, PSW_TILE_SWIGLU = 2, PSW_TILE_OTHER = 3,
               PSW_TILE_CLASSES = 4 } psw_tile_class;
psw_status psw_set_tile_policy(psw_ctx *ctx, int cls, int tokens);
int psw_tile_policy(const psw_ctx *ctx, int cls);

/* Instrumentation (not in the paper; measurement support).
 * psw_launch_count: kernels this context has launched so far.
 * psw_profile_begin: from now on every kernel launch of this context is
 * bracketed by CUDA events on its stream (adds host overhead; for
 * measurement runs only).  psw_profile_end synchronises the device, stops
 * recording and writes one psw_kernel_stat per kernel class (at most cap;
 * *n_out = number written): launches, summed event time in ms, and the
 * algorithmic FLOPs and bytes of those launches (FLOPs: 2 per multiply-add
 * of the projections and attention; bytes: operands read once plus results
 * written once). */
typedef struct {
    char name[32];
    long launches;
    double ms;
    double flops;
    double bytes;
} psw_kernel_stat;

long psw_launch_count(const psw_ctx *ctx);
psw_status psw_profile_begin(psw_ctx *ctx);
psw_status psw_profile_end(psw_ctx *ctx, psw_kernel_stat *out, int cap, int *n_out);

#ifdef __cplusplus
}
#endif
#endif /* PSW_H */
