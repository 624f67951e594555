// kernels.cu -- elementwise, normalisation, window-attention, head and
// SIMT GEMM kernels of the P-SWA context model (Sec. 3.1 block structure,
// Sec. 3.2 masked window attention).  Every per-token computation has a
// fixed arithmetic order that does not depend on how many tokens a launch
// carries or which other frames share it, so the encoder's masked pass, the
// decoder's wavefront steps and batched decoding produce bit-identical
// parameters.  Tokens are (slot, position) words; per-frame state is reached
// through the slot table.
#include "internal.h"
#include "device_common.cuh"
#include "attn_dev.cuh"
#include "attn_tok.cuh"

#include <math.h>

#include <algorithm>

namespace psw {

static inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------- weights

// dst[(row_off + n) * K + k] = src[k * N + n]: a projection stored [in][out]
// becomes [out][in] (K-major) in the compute type, rounded to nearest even.
template <typename T>
__global__ void k_transpose_convert(const float *__restrict__ src, int K, int N, T *__restrict__ dst,
                                    int row_off)
{
    __shared__ float tile[32][33];
    int k0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int k = k0 + r, n = n0 + threadIdx.x;
        tile[r][threadIdx.x] = (k < K && n < N) ? src[(long)k * N + n] : 0.0f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int n = n0 + r, k = k0 + threadIdx.x;
        if (n < N && k < K) dst[(long)(row_off + n) * K + k] = from_f<T>(tile[threadIdx.x][r]);
    }
}

void launch_transpose_convert(int prec, const float *src, int K, int N, void *dst, int row_off,
                              cudaStream_t s)
{
    dim3 grid(cdiv(N, 32), cdiv(K, 32)), block(32, 8);
    if (prec == P_BF16)
        k_transpose_convert<__nv_bfloat16><<<grid, block, 0, s>>>(src, K, N, (__nv_bfloat16 *)dst, row_off);
    else
        k_transpose_convert<float><<<grid, block, 0, s>>>(src, K, N, (float *)dst, row_off);
}

// ---------------------------------------------------------------- embeddings

// Context Transformer input (Sec. 3.1: temporal shift, channel-wise input
// scaling then a linear map): out[m][e] = b[e] + sum_c (gamma[c] yprev[c])
// W[c][e] from the previous frame's latents at the token's position, or the
// learned padding vector for the first frame of a sequence.  Runs once per
// frame; FP32.
__global__ void k_embed_context(const Slot *__restrict__ S, const int *__restrict__ tok, int C,
                                const float *__restrict__ gamma, const float *__restrict__ W,
                                const float *__restrict__ b, const float *__restrict__ pad, int d,
                                float *__restrict__ out)
{
    extern __shared__ float t[];
    int tk = tok[blockIdx.x];
    const Slot &s = S[tok_slot(tk)];
    int p = tok_pos(tk);
    float *x = out + (long)blockIdx.x * d;
    if (s.frame == 0) {
        for (int e = threadIdx.x; e < d; e += blockDim.x) x[e] = pad[e];
        return;
    }
    const int16_t *y = s.yprev + (long)p * C;
    for (int c = threadIdx.x; c < C; c += blockDim.x) t[c] = gamma[c] * (float)y[c];
    __syncthreads();
    for (int e = threadIdx.x; e < d; e += blockDim.x) {
        float acc = 0.0f;
        for (int c = 0; c < C; c++) acc = fmaf(t[c], W[(long)c * d + e], acc);
        x[e] = acc + b[e];
    }
}

void launch_embed_context(const Slot *S, const int *tok, int n, int C, const float *gamma, const float *W,
                          const float *b, const float *pad, int d, float *out, cudaStream_t s)
{
    if (n <= 0) return;
    k_embed_context<<<n, 128, C * sizeof(float), s>>>(S, tok, C, gamma, W, b, pad, d, out);
}

// Hyperprior tokens (Fig. 1: the decoded hyperprior enters the transformer):
// transposed convolution with kernel = stride = r, for every position of one
// frame.  Position (i, j) takes tap (i mod r, j mod r) of W_hp and the
// hyperlatent (i / r, j / r), so a block takes one tap and up to 32
// hyperlatents of one hyperlatent row: the tap's weights [Ch][d] are read
// once for all of them (not once per position).  Thread e owns output column
// e (and e + blockDim, ...); each output sums over c in ascending order, then
// adds the bias.
constexpr int EH_NB = 32;

__global__ void __launch_bounds__(384) k_embed_hyper(const Slot *__restrict__ S, const int *__restrict__ tok, int nz,
                                                     int Ch, int r, int nbmax, const float *__restrict__ gamma,
                                                     const float *__restrict__ Whp, const float *__restrict__ b, int d)
{
    extern __shared__ float4 t4[];                    // [Ch][nbmax] floats: gamma * zhat, channel-major
    float *t = reinterpret_cast<float *>(t4);
    // one frame (tok[0]'s slot), or (nz > 0) slot blockIdx.z / nz of a batch
    const Slot &s = S[nz > 0 ? (int)(blockIdx.z / nz) : tok_slot(tok[0])];
    const int zb = nz > 0 ? (int)(blockIdx.z % nz) : (int)blockIdx.z;
    const int H = s.H, W = s.W, Wh = (W + r - 1) / r;
    const int ti = blockIdx.x / r, tj = blockIdx.x % r, a = blockIdx.y, b0 = zb * nbmax;
    const int i = a * r + ti;
    if (i >= H || b0 >= Wh) return;                   // uniform over the block
    const int nb = min(nbmax, Wh - b0);
    for (int x = threadIdx.x; x < nb * Ch; x += blockDim.x) {
        const int k = x / Ch, c = x - k * Ch;
        t[c * nbmax + k] = gamma[c] * (float)s.zhat[((long)a * Wh + b0 + k) * Ch + c];
    }
    __syncthreads();
    const float *Ws = Whp + (long)blockIdx.x * Ch * d;
    for (int e = threadIdx.x; e < d; e += blockDim.x) {
        float acc[EH_NB];
#pragma unroll
        for (int k = 0; k < EH_NB; k++) acc[k] = 0.0f;
#pragma unroll 2
        for (int c = 0; c < Ch; c++) {
            const float w = Ws[(long)c * d + e];
            const float4 *tc = t4 + c * (nbmax >> 2);
#pragma unroll
            for (int q = 0; q < EH_NB / 4; q++) {
                if (4 * q < nb) {                      // columns past nb are never stored
                    const float4 v = tc[q];
                    acc[4 * q] = fmaf(v.x, w, acc[4 * q]);
                    acc[4 * q + 1] = fmaf(v.y, w, acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(v.z, w, acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(v.w, w, acc[4 * q + 3]);
                }
            }
        }
        const float be = b[e];
#pragma unroll
        for (int k = 0; k < EH_NB; k++) {
            const int j = (b0 + k) * r + tj;
            if (k < nb && j < W) s.eh[((long)i * W + j) * d + e] = acc[k] + be;
        }
    }
}

// tok: every position of one frame in raster order (the slot is tok[0]'s).
void launch_embed_hyper(const Slot *S, const int *tok, int n, int H, int W, int Ch, int r, const float *gamma,
                        const float *Whp, const float *b, int d, cudaStream_t s)
{
    if (n <= 0) return;
    const int Hh = (H + r - 1) / r, Wh = (W + r - 1) / r;
    const int nbmax = std::max(4, std::min(EH_NB, (12288 / Ch) & ~3));   // staged hyperlatents: <= 64 KB
    const dim3 grid(r * r, Hh, (Wh + nbmax - 1) / nbmax);
    const int threads = d < 384 ? ((d + 31) / 32) * 32 : 384;
    k_embed_hyper<<<grid, threads, (size_t)nbmax * Ch * sizeof(float), s>>>(S, tok, 0, Ch, r, nbmax, gamma, Whp, b,
                                                                            d);
}

void launch_embed_hyper_batch(const Slot *S, int nslots, int Hmax, int Wmax, int Ch, int r, const float *gamma,
                              const float *Whp, const float *b, int d, cudaStream_t s)
{
    if (nslots <= 0) return;
    const int Hh = (Hmax + r - 1) / r, Wh = (Wmax + r - 1) / r;
    const int nbmax = std::max(4, std::min(EH_NB, (12288 / Ch) & ~3));
    const int nz = (Wh + nbmax - 1) / nbmax;
    const dim3 grid(r * r, Hh, nslots * nz);
    const int threads = d < 384 ? ((d + 31) / 32) * 32 : 384;
    k_embed_hyper<<<grid, threads, (size_t)nbmax * Ch * sizeof(float), s>>>(S, nullptr, nz, Ch, r, nbmax, gamma, Whp,
                                                                            b, d);
}

// ---------------------------------------------------------------- batched copies

__global__ void k_copy_jobs(const CopyJob *__restrict__ jobs)
{
    const CopyJob j = jobs[blockIdx.y];
    const size_t stride = (size_t)gridDim.x * blockDim.x, t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((((uintptr_t)j.src | (uintptr_t)j.dst) & 15) == 0) {
        const size_t nw = j.bytes / 16;
        const uint4 *src = (const uint4 *)j.src;
        uint4 *dst = (uint4 *)j.dst;
        for (size_t w = t0; w < nw; w += stride) dst[w] = src[w];
        for (size_t b = nw * 16 + t0; b < j.bytes; b += stride) ((char *)j.dst)[b] = ((const char *)j.src)[b];
    } else {
        for (size_t b = t0; b < j.bytes; b += stride) ((char *)j.dst)[b] = ((const char *)j.src)[b];
    }
}

void launch_copy_jobs(const CopyJob *jobs, int n, unsigned long long max_bytes, cudaStream_t s)
{
    if (n <= 0) return;
    const unsigned long long words = (max_bytes + 15) / 16;
    const int gx = (int)std::max<unsigned long long>(1, std::min<unsigned long long>((words + 255) / 256, 64));
    k_copy_jobs<<<dim3(gx, n), 256, 0, s>>>(jobs);
}

// ---------------------------------------------------------------- RMSNorm

// One warp per row: y = x / sqrt(mean(x^2) + 1e-6) * g, FP32 statistics,
// a fixed lane assignment and butterfly reduction (the SIMT path's operand).
template <typename T>
__global__ void k_rmsnorm(const float *__restrict__ X, int n, const float *__restrict__ g, int d, T *__restrict__ dst,
                          int ldd)
{
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= n) return;
    const float *x = X + (long)w * d;
    float ss = 0.0f;
    for (int e = lane; e < d; e += 32) ss = fmaf(x[e], x[e], ss);
    ss = warp_sum(ss);
    float inv = 1.0f / sqrtf(ss / (float)d + 1e-6f);
    T *y = dst + (long)w * ldd;
    for (int e = lane; e < d; e += 32) y[e] = from_f<T>(x[e] * inv * g[e]);
}

void launch_rmsnorm(int prec, const float *X, int n, const float *g, int d, void *dst, cudaStream_t s, int ldd)
{
    if (n <= 0) return;
    if (ldd <= 0) ldd = d;
    int blocks = cdiv((long)n * 32, 256);
    if (prec == P_BF16) k_rmsnorm<__nv_bfloat16><<<blocks, 256, 0, s>>>(X, n, g, d, (__nv_bfloat16 *)dst, ldd);
    else k_rmsnorm<float><<<blocks, 256, 0, s>>>(X, n, g, d, (float *)dst, ldd);
}

// rep[position][off + e] = X[m][e]: one float4 per thread, tokens of slots
// without a rep buffer skipped.  A plain launch: it starts after its
// predecessor has finished.
__global__ void k_store_rows(const Slot *__restrict__ S, const int *__restrict__ tok, int n,
                             const float *__restrict__ X, int w4, int ld4, int off4)
{
    const long total = (long)n * w4;
    for (long a = blockIdx.x * (long)blockDim.x + threadIdx.x; a < total; a += (long)gridDim.x * blockDim.x) {
        const int m = (int)(a / w4), e = (int)(a - (long)m * w4);
        const int tk = tok[m];
        float *rep = S[tok_slot(tk)].rep;
        if (!rep) continue;
        reinterpret_cast<float4 *>(rep)[(long)tok_pos(tk) * ld4 + off4 + e] = reinterpret_cast<const float4 *>(X)[a];
    }
}

void launch_store_rows(const Slot *S, const int *tok, int n, const float *X, int w, int ld, int off, cudaStream_t s)
{
    if (n <= 0) return;
    long total = (long)n * (w / 4);
    int blocks = (int)std::min<long>(cdiv(total, 256), 152 * 8);
    k_store_rows<<<blocks, 256, 0, s>>>(S, tok, n, X, w / 4, ld / 4, off / 4);
}

// Channel shift of the Channel Transformer: one block per token, the
// channel-scaled latents of the previous group in shared memory, thread e
// owns output column e (and e + blockDim, ...), summing over c in ascending
// order before adding to the row.  A plain launch.
__global__ void k_ct_embed(const Slot *__restrict__ S, const int *__restrict__ tok, int C, int c0, int Cg,
                           const float *__restrict__ gamma, const float *__restrict__ E, int dg, float *__restrict__ X)
{
    extern __shared__ float t[];
    const int tk = tok[blockIdx.x];
    const Slot &s = S[tok_slot(tk)];
    const int16_t *y = s.y + (long)tok_pos(tk) * C + c0;
    for (int c = threadIdx.x; c < Cg; c += blockDim.x) t[c] = gamma[c] * (float)y[c];
    __syncthreads();
    float *x = X + (long)blockIdx.x * dg;
    for (int e = threadIdx.x; e < dg; e += blockDim.x) {
        float acc = 0.0f;
        for (int c = 0; c < Cg; c++) acc = fmaf(t[c], E[(long)c * dg + e], acc);
        x[e] += acc;
    }
}

void launch_ct_embed(const Slot *S, const int *tok, int n, int C, int c0, int Cg, const float *gamma, const float *E,
                     int dg, float *X, cudaStream_t s)
{
    if (n <= 0) return;
    k_ct_embed<<<n, 128, Cg * sizeof(float), s>>>(S, tok, C, c0, Cg, gamma, E, dg, X);
}

// ---------------------------------------------------------------- attention

// Warps per block: shared staging of one warp is CK key and CK value rows of
// a head.
template <typename T, int DH>
__host__ __device__ constexpr int attn_wpb() { return AttnWarp<T, DH>::RB <= 128 ? 4 : (AttnWarp<T, DH>::RB <= 256 ? 2 : 1); }

template <typename T, int DH, int CK, int MAXC>
__global__ void __launch_bounds__(32 * attn_wpb<T, DH>()) k_attention(AttnArgs a)
{
    constexpr int WPB = attn_wpb<T, DH>();
    __shared__ AttnWarp<T, DH, CK, MAXC> sm[WPB];
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * WPB + wib;
    if (gw >= a.n * a.nh) return;                              // warps are independent: no block barrier
    attn_item<T, DH, true, CK, MAXC>(a, gw, sm[wib]);
}

// 64-wide BF16 heads: one warp per token and head group, on the tensor
// cores (attn_tok.cuh); TK_WPB warps per block, each with its own staging.
constexpr int TK_WPB = 4;

__global__ void __launch_bounds__(32 * TK_WPB, 4) k_attn_tok(AttnArgs a)
{
    extern __shared__ __align__(16) unsigned char tk_smem[];
    const int wib = threadIdx.x >> 5, gw = blockIdx.x * TK_WPB + wib;
    if (gw >= a.n * (a.nh / TK_HG)) return;                    // warps are independent: no block barrier
    attn_token<true>(a, gw, tk_smem + (size_t)wib * attn_tok_bytes());
}

// Spatial windows (k * k <= 81 candidates) take the compact staging.
template <typename T, int DH>
static void attention_dh(const AttnArgs &a, cudaStream_t s)
{
    const long warps = (long)a.n * a.nh;
    const dim3 grid(cdiv(warps, attn_wpb<T, DH>())), block(32 * attn_wpb<T, DH>());
    static_assert(MAX_KK <= 96, "spatial candidate list");
    if (a.temporal) launch_pdl(k_attention<T, DH, 32, 256>, grid, block, 0, s, a);
    else if (a.k * a.k <= 64) launch_pdl(k_attention<T, DH, 24, 64>, grid, block, 0, s, a);
    else launch_pdl(k_attention<T, DH, 24, 96>, grid, block, 0, s, a);
}

template <typename T, int DH>
static bool attention_carveout()
{
    // warps of a block are independent: prefer the shared-memory carveout
    // that holds the most blocks
    const int c = cudaSharedmemCarveoutMaxShared;
    return cudaFuncSetAttribute(k_attention<T, DH, 32, 256>, cudaFuncAttributePreferredSharedMemoryCarveout, c) ==
               cudaSuccess &&
           cudaFuncSetAttribute(k_attention<T, DH, 24, 96>, cudaFuncAttributePreferredSharedMemoryCarveout, c) ==
               cudaSuccess &&
           cudaFuncSetAttribute(k_attention<T, DH, 24, 64>, cudaFuncAttributePreferredSharedMemoryCarveout, c) ==
               cudaSuccess;
}

bool attention_prepare()
{
    if (cudaFuncSetAttribute(k_attn_tok, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(TK_WPB * attn_tok_bytes())) != cudaSuccess ||
        cudaFuncSetAttribute(k_attn_tok, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return false;
    if (cudaFuncSetAttribute(k_embed_hyper, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 4096 * 4) != cudaSuccess)
        return false;                                 // 4 staged hyperlatents of 4096 channels
    return attention_carveout<__nv_bfloat16, 32>() && attention_carveout<__nv_bfloat16, 64>() &&
           attention_carveout<__nv_bfloat16, 128>() && attention_carveout<float, 32>() &&
           attention_carveout<float, 64>() && attention_carveout<float, 128>();
}

template <typename T>
static void attention_t(const AttnArgs &a, cudaStream_t s)
{
    switch (a.d / a.nh) {
    case 32: attention_dh<T, 32>(a, s); break;
    case 64: attention_dh<T, 64>(a, s); break;
    case 128: attention_dh<T, 128>(a, s); break;
    default: break;   // rejected at context creation
    }
}

void launch_attention(int prec, const AttnArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return;
    if (attn_tok_ok(prec, a.d, a.nh, a.mask, a.kind)) {
        launch_pdl(k_attn_tok, dim3(cdiv((long)a.n * (a.nh / TK_HG), TK_WPB)), dim3(32 * TK_WPB),
                   TK_WPB * attn_tok_bytes(), s, a);
        return;
    }
    if (prec == P_BF16) attention_t<__nv_bfloat16>(a, s);
    else attention_t<float>(a, s);
}

// ---------------------------------------------------------------- heads

__device__ __forceinline__ void quantize_one(float mu, float sigma, const float *scale, uint8_t &idx,
                                             int32_t &m)
{
    idx = (uint8_t)scale_index(scale, sigma);
    m = (int32_t)rintf(fminf(fmaxf(mu, -32768.0f), 32767.0f));
}

__global__ void k_quantize(size_t n, const float *mu, const float *sigma, const float *scale,
                           uint8_t *idx, int32_t *m)
{
    __shared__ float stab[NSCALES];
    if (threadIdx.x < NSCALES) stab[threadIdx.x] = scale[threadIdx.x];
    __syncthreads();
    for (size_t a = blockIdx.x * (size_t)blockDim.x + threadIdx.x; a < n; a += (size_t)gridDim.x * blockDim.x)
        quantize_one(mu[a], sigma[a], stab, idx[a], m[a]);
}

void launch_quantize(size_t n, const float *mu, const float *sigma, const float *scale, uint8_t *idx,
                     int32_t *m, cudaStream_t s)
{
    if (n == 0) return;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_quantize<<<blocks, 256, 0, s>>>(n, mu, sigma, scale, idx, m);
}

// ---------------------------------------------------------------- rate

// -log2 of the Gaussian mass of [y - 1/2, y + 1/2] (|y - mu| form, sigma
// clamped to [0.11, 256], mass floored at 1e-9), FP64.  Block b sums the
// fixed chunk [b * 4096, (b + 1) * 4096) with a fixed tree; a second pass adds
// the partials in order.
constexpr int RATE_CHUNK = 4096;

__global__ void k_rate_partial(size_t n, const int16_t *y, const float *mu, const float *sigma,
                               double *partials)
{
    __shared__ double red[256];
    size_t base = (size_t)blockIdx.x * RATE_CHUNK;
    double acc = 0.0;
    for (int u = threadIdx.x; u < RATE_CHUNK; u += 256) {
        size_t a = base + u;
        if (a >= n) break;
        double sg = (double)sigma[a];
        sg = sg < 0.11 ? 0.11 : (sg > 256.0 ? 256.0 : sg);
        double uu = fabs((double)y[a] - (double)mu[a]), den = sg * 1.4142135623730951;
        double pr = 0.5 * (erfc((uu - 0.5) / den) - erfc((uu + 0.5) / den));
        if (pr < 1e-9) pr = 1e-9;
        acc -= log2(pr);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_rate_final(int np, const double *partials, double *out)
{
    if (threadIdx.x != 0) return;
    double acc = 0.0;
    for (int b = 0; b < np; b++) acc += partials[b];
    *out = acc;
}

int rate_partials(size_t n) { return (int)((n + RATE_CHUNK - 1) / RATE_CHUNK); }

void launch_rate(size_t n, const int16_t *y, const float *mu, const float *sigma, double *partials,
                 double *out, cudaStream_t s)
{
    int np = rate_partials(n);
    if (np > 0) k_rate_partial<<<np, 256, 0, s>>>(n, y, mu, sigma, partials);
    k_rate_final<<<1, 32, 0, s>>>(np, partials, out);
}

// ---------------------------------------------------------------- SIMT GEMM

// 32 tokens x 64 outputs per block, 256 threads, each 4 tokens x 2 outputs
// (x2 for the dual SwiGLU form); K in chunks of 32 through shared memory,
// FP32 accumulation in ascending k.
template <typename T, bool DUAL>
__global__ void __launch_bounds__(256) k_gemm_simt(GemmArgs g)
{
    __shared__ float As[32][33];
    __shared__ float Ws[64][33];
    __shared__ float Ws2[DUAL ? 64 : 1][33];
    const T *A = (const T *)g.A, *Wt = (const T *)g.Wt, *Wt2 = (const T *)g.Wt2;
    int m0 = blockIdx.y * 32, n0 = blockIdx.x * 64;
    int tn = threadIdx.x & 31, tm = threadIdx.x >> 5;
    float acc[4][2], acc2[4][2];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) { acc[i][j] = 0.0f; acc2[i][j] = 0.0f; }
    for (int k0 = 0; k0 < g.K; k0 += 32) {
        for (int u = threadIdx.x; u < 32 * 32; u += 256) {
            int r = u >> 5, c = u & 31, m = m0 + r, k = k0 + c;
            As[r][c] = (m < g.M && k < g.K) ? to_f<T>(A[(long)m * g.lda + k]) : 0.0f;
        }
        for (int u = threadIdx.x; u < 64 * 32; u += 256) {
            int r = u >> 5, c = u & 31, n = n0 + r, k = k0 + c;
            bool ok = n < g.N && k < g.K;
            Ws[r][c] = ok ? to_f<T>(Wt[(long)n * g.K + k]) : 0.0f;
            if (DUAL) Ws2[r][c] = ok ? to_f<T>(Wt2[(long)n * g.K + k]) : 0.0f;
        }
        __syncthreads();
        int kmax = min(32, g.K - k0);
        for (int kk = 0; kk < kmax; kk++) {
            float a[4], w[2], w2[2];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[tm * 4 + i][kk];
#pragma unroll
            for (int j = 0; j < 2; j++) {
                w[j] = Ws[tn * 2 + j][kk];
                if (DUAL) w2[j] = Ws2[tn * 2 + j][kk];
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 2; j++) {
                    acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
                    if (DUAL) acc2[i][j] = fmaf(a[i], w2[j], acc2[i][j]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int m = m0 + tm * 4 + i;
        if (m >= g.M) continue;
        if (g.epi.mode == EPI_HEADS) {
            int n = n0 + tn * 2;                     // a thread holds the (mu, sigma) rows of one channel
            if (n + 1 < g.N) heads_pair(g.epi, g.epi.scale, m, n, acc[i][0], acc[i][1]);
            continue;
        }
#pragma unroll
        for (int j = 0; j < 2; j++) {
            int n = n0 + tn * 2 + j;
            if (n < g.N) epilogue_store<T>(g.epi, g.N, m, n, acc[i][j], acc2[i][j]);
        }
    }
}

void gemm_simt(int prec, const GemmArgs &g, cudaStream_t s)
{
    dim3 grid(cdiv(g.N, 64), cdiv(g.M, 32));
    bool dual = g.epi.mode == EPI_SWIGLU;
    if (prec == P_BF16) {
        if (dual) k_gemm_simt<__nv_bfloat16, true><<<grid, 256, 0, s>>>(g);
        else k_gemm_simt<__nv_bfloat16, false><<<grid, 256, 0, s>>>(g);
    } else {
        if (dual) k_gemm_simt<float, true><<<grid, 256, 0, s>>>(g);
        else k_gemm_simt<float, false><<<grid, 256, 0, s>>>(g);
    }
}

bool gemm_tc(const GemmArgs &g, cudaStream_t s);

bool gemm(int prec, const GemmArgs &g0, cudaStream_t s)
{
    if (g0.M <= 0 || g0.N <= 0) return true;
    if (gemm_takes_ws(prec, g0)) return gemm_ws(g0, s);
    if (g0.f8 || gemm_tc_supported(prec, g0.N, g0.K, g0.asrc)) return gemm_tc(g0, s);     // E4M3: tensor cores only
    // SIMT path: materialise the token operand first
    GemmArgs g = g0;
    if (g.asrc == A_NORM) {
        launch_rmsnorm(prec, g.xrows, g.M, g.a_gain, g.K, g.prep, s);
        g.A = g.prep; g.lda = g.K;
    } else if (g.asrc == A_EMBED) {
        launch_gather_embed(prec, g.epi.slots, g.epi.tok, g.M, g.a_gain, g.K, g.prep, s);
        g.A = g.prep; g.lda = g.K;
    }
    gemm_simt(prec, g, s);
    return true;
}

// Channel-scaled latents of each token as compact rows (the latent
// embedding's input on the SIMT path).
template <typename T>
__global__ void k_gather_embed(const Slot *__restrict__ S, const int *__restrict__ tok, const float *__restrict__ gamma,
                               int C, T *__restrict__ dst)
{
    int tk = tok[blockIdx.x];
    const Slot &s = S[tok_slot(tk)];
    const int16_t *y = s.y + (long)tok_pos(tk) * C;
    for (int c = threadIdx.x; c < C; c += blockDim.x) dst[(long)blockIdx.x * C + c] = from_f<T>(gamma[c] * (float)y[c]);
}

void launch_gather_embed(int prec, const Slot *S, const int *tok, int n, const float *gamma, int C, void *dst,
                         cudaStream_t s)
{
    if (n <= 0) return;
    if (prec == P_BF16) k_gather_embed<__nv_bfloat16><<<n, 128, 0, s>>>(S, tok, gamma, C, (__nv_bfloat16 *)dst);
    else k_gather_embed<float><<<n, 128, 0, s>>>(S, tok, gamma, C, (float *)dst);
}

template <typename T>
__global__ void k_convert(const float *__restrict__ src, size_t n, T *__restrict__ dst)
{
    for (size_t a = blockIdx.x * (size_t)blockDim.x + threadIdx.x; a < n; a += (size_t)gridDim.x * blockDim.x)
        dst[a] = from_f<T>(src[a]);
}

void launch_convert(int prec, const float *src, size_t n, void *dst, cudaStream_t s)
{
    if (n == 0) return;
    int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
    if (prec == P_BF16) k_convert<__nv_bfloat16><<<blocks, 256, 0, s>>>(src, n, (__nv_bfloat16 *)dst);
    else k_convert<float><<<blocks, 256, 0, s>>>(src, n, (float *)dst);
}

}  // namespace psw
