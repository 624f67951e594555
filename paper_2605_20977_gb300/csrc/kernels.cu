// kernels.cu -- elementwise, normalisation, window-attention, head and
// SIMT GEMM kernels of the P-SWA context model (Sec. 3.1 block structure,
// Sec. 3.2 masked window attention).  Every per-token computation has a
// fixed arithmetic order that does not depend on how many tokens a launch
// carries, so the encoder's masked pass and the decoder's wavefront steps
// produce bit-identical parameters.
#include "internal.h"

#include <math.h>

namespace psw {

// ---------------------------------------------------------------- helpers

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float silu_f(float x) { return x / (1.0f + expf(-x)); }

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

// Latent token embedding (Sec. 3.1, channel-wise input scaling then a
// linear map): x[p][e] = b[e] + sum_c (gamma[c] y[p][c]) W[c][e].
__global__ void k_embed_latent(const int *__restrict__ pos, const int16_t *__restrict__ y, int C,
                               const float *__restrict__ gamma, const float *__restrict__ W,
                               const float *__restrict__ b, int d, float *__restrict__ x)
{
    extern __shared__ float t[];
    int p = pos ? pos[blockIdx.x] : blockIdx.x;
    for (int c = threadIdx.x; c < C; c += blockDim.x) t[c] = gamma[c] * (float)y[(long)p * C + c];
    __syncthreads();
    for (int e = threadIdx.x; e < d; e += blockDim.x) {
        float acc = 0.0f;
        for (int c = 0; c < C; c++) acc = fmaf(t[c], W[(long)c * d + e], acc);
        x[(long)p * d + e] = acc + b[e];
    }
}

void launch_embed_latent(const int *pos, int n, const int16_t *y, int C, const float *gamma,
                         const float *W, const float *b, int d, float *x, cudaStream_t s)
{
    if (n <= 0) return;
    k_embed_latent<<<n, 128, C * sizeof(float), s>>>(pos, y, C, gamma, W, b, d, x);
}

__global__ void k_fill_rows(const float *__restrict__ v, int d, float *__restrict__ x)
{
    for (int e = threadIdx.x; e < d; e += blockDim.x) x[(long)blockIdx.x * d + e] = v[e];
}

void launch_fill_rows(const float *v, int n, int d, float *x, cudaStream_t s)
{
    if (n <= 0) return;
    k_fill_rows<<<n, 128, 0, s>>>(v, d, x);
}

// Hyperprior tokens (Fig. 1: the decoded hyperprior enters the transformer):
// transposed convolution with kernel = stride = r.
__global__ void k_embed_hyper(const int16_t *__restrict__ z, int W, int Wh, int Ch, int r,
                              const float *__restrict__ gamma, const float *__restrict__ Whp,
                              const float *__restrict__ b, int d, float *__restrict__ eh)
{
    extern __shared__ float t[];
    int p = blockIdx.x, i = p / W, j = p % W;
    const int16_t *zv = z + ((long)(i / r) * Wh + (j / r)) * Ch;
    for (int c = threadIdx.x; c < Ch; c += blockDim.x) t[c] = gamma[c] * (float)zv[c];
    __syncthreads();
    const float *Ws = Whp + (long)((i % r) * r + (j % r)) * Ch * d;
    for (int e = threadIdx.x; e < d; e += blockDim.x) {
        float acc = 0.0f;
        for (int c = 0; c < Ch; c++) acc = fmaf(t[c], Ws[(long)c * d + e], acc);
        eh[(long)p * d + e] = acc + b[e];
    }
}

void launch_embed_hyper(const int16_t *z, int H, int W, int Wh, int Ch, int r, const float *gamma,
                        const float *Whp, const float *b, int d, float *eh, cudaStream_t s)
{
    k_embed_hyper<<<H * W, 128, Ch * sizeof(float), s>>>(z, W, Wh, Ch, r, gamma, Whp, b, d, eh);
}

// ---------------------------------------------------------------- RMSNorm

// One warp per token: y = x / sqrt(mean(x^2) + 1e-6) * g, FP32 statistics,
// a fixed lane assignment and butterfly reduction.
template <typename T>
__global__ void k_rmsnorm(const int *__restrict__ pos, int n, const float *__restrict__ src,
                          const float *__restrict__ g, int d, T *__restrict__ dst, int scatter)
{
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= n) return;
    int p = pos ? pos[w] : w;
    const float *x = src + (long)p * d;
    float ss = 0.0f;
    for (int e = lane; e < d; e += 32) ss = fmaf(x[e], x[e], ss);
    ss = warp_sum(ss);
    float inv = 1.0f / sqrtf(ss / (float)d + 1e-6f);
    T *y = dst + (long)(scatter ? p : w) * d;
    for (int e = lane; e < d; e += 32) y[e] = from_f<T>(x[e] * inv * g[e]);
}

void launch_rmsnorm(int prec, const int *pos, int n, const float *src, const float *g, int d, void *dst,
                    int scatter, cudaStream_t s)
{
    if (n <= 0) return;
    int blocks = cdiv((long)n * 32, 256);
    if (prec == P_BF16)
        k_rmsnorm<__nv_bfloat16><<<blocks, 256, 0, s>>>(pos, n, src, g, d, (__nv_bfloat16 *)dst, scatter);
    else
        k_rmsnorm<float><<<blocks, 256, 0, s>>>(pos, n, src, g, d, (float *)dst, scatter);
}

// ---------------------------------------------------------------- attention

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

// One warp per (token, head).  Candidate keys are the window positions of
// each key frame in ascending raster order (frames oldest first); a lane
// scores its candidates, the warp takes max and sum by butterflies, then each
// lane accumulates its output dimensions over the candidates in order.
template <typename T, int DH>
__global__ void k_attention(AttnArgs a)
{
    constexpr int PER = DH / 32;
    __shared__ float qs[4][DH];
    int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int gw = blockIdx.x * 4 + wib;
    if (gw >= a.n * a.nh) return;
    int tok = gw / a.nh, h = gw % a.nh;
    int p = a.pos ? a.pos[tok] : tok;
    int pi = p / a.W, pj = p % a.W, w = (a.k - 1) >> 1, kk = a.k * a.k;
    const T *q = (const T *)a.Q + (long)(a.q_full ? p : tok) * a.d + h * DH;
    for (int e = lane; e < DH; e += 32) qs[wib][e] = to_f<T>(q[e]);
    __syncwarp();
    const float scale = rsqrtf((float)DH);
    int ncand = a.nfr * kk;
    int rounds = (ncand + 31) >> 5;
    // scores of this lane's candidates (at most 8 rounds: 4 frames x 49)
    float sc[8];
    int key[8];
    float mx = -INFINITY;
#pragma unroll
    for (int r = 0; r < 8; r++) {
        sc[r] = -INFINITY; key[r] = -1;
        if (r >= rounds) continue;
        int cidx = r * 32 + lane;
        if (cidx >= ncand) continue;
        int fr = cidx / kk, c = cidx % kk;
        int qi = pi + c / a.k - w, qj = pj + c % a.k - w;
        if (qi < 0 || qi >= a.H || qj < 0 || qj >= a.W) continue;
        if (!visible(a.mask, a.kind, a.W, pi, pj, qi, qj)) continue;
        int qp = qi * a.W + qj;
        const T *kr = (const T *)a.K[fr] + (long)qp * a.d + h * DH;
        float acc = 0.0f;
#pragma unroll 8
        for (int e = 0; e < DH; e++) acc = fmaf(qs[wib][e], to_f<T>(kr[e]), acc);
        sc[r] = acc * scale + a.bias[(long)h * a.bias_h_stride + (long)a.age[fr] * kk + c];
        key[r] = qp;
        mx = fmaxf(mx, sc[r]);
    }
    mx = warp_max(mx);
    float z = 0.0f;
#pragma unroll
    for (int r = 0; r < 8; r++) {
        float e = (key[r] >= 0) ? expf(sc[r] - mx) : 0.0f;
        sc[r] = e;
        z += e;
    }
    z = warp_sum(z);
    float inv = z > 0.0f ? 1.0f / z : 0.0f;
    float o[PER];
#pragma unroll
    for (int u = 0; u < PER; u++) o[u] = 0.0f;
    for (int r = 0; r < rounds; r++) {
        for (int src = 0; src < 32; src++) {
            int kq = __shfl_sync(0xffffffffu, key[r], src);
            float pr = __shfl_sync(0xffffffffu, sc[r] * inv, src);
            if (kq < 0) continue;
            int fr = (r * 32 + src) / kk;
            const T *vr = (const T *)a.V[fr] + (long)kq * a.d + h * DH;
#pragma unroll
            for (int u = 0; u < PER; u++) o[u] = fmaf(pr, to_f<T>(vr[u * 32 + lane]), o[u]);
        }
    }
    T *out = (T *)a.O + (long)tok * a.d + h * DH;
#pragma unroll
    for (int u = 0; u < PER; u++) out[u * 32 + lane] = from_f<T>(o[u]);
}

template <typename T>
static void attention_t(const AttnArgs &a, cudaStream_t s)
{
    int dh = a.d / a.nh;
    int blocks = cdiv((long)a.n * a.nh, 4);
    switch (dh) {
    case 32: k_attention<T, 32><<<blocks, 128, 0, s>>>(a); break;
    case 64: k_attention<T, 64><<<blocks, 128, 0, s>>>(a); break;
    case 128: k_attention<T, 128><<<blocks, 128, 0, s>>>(a); break;
    default: break;   // rejected at context creation
    }
}

void launch_attention(int prec, const AttnArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return;
    if (prec == P_BF16) attention_t<__nv_bfloat16>(a, s);
    else attention_t<float>(a, s);
}

// ---------------------------------------------------------------- heads

__device__ __forceinline__ void quantize_one(float mu, float sigma, const float *scale, uint8_t &idx,
                                             int32_t &m)
{
    int l = NSCALES - 1;
    for (int t = 0; t < NSCALES; t++)
        if (scale[t] >= sigma) { l = t; break; }
    idx = (uint8_t)l;
    m = (int32_t)rintf(fminf(fmaxf(mu, -32768.0f), 32767.0f));
}

// Prediction heads (Sec. 3.1: grouped two-layer MLPs for mu and sigma, with
// channel-wise output scaling), one block per token, FP32; then the scale
// index and rounded mean of every channel.
__global__ void k_heads(HeadsArgs a)
{
    extern __shared__ float sm[];
    float *xn = sm, *hm = sm + a.d, *hs = sm + 2 * a.d;
    __shared__ float red[32];
    __shared__ float stab[NSCALES];
    int p = a.pos ? a.pos[blockIdx.x] : blockIdx.x;
    const float *x = a.x + (long)p * a.d;
    if (threadIdx.x < NSCALES) stab[threadIdx.x] = a.scale[threadIdx.x];
    float ss = 0.0f;
    for (int e = threadIdx.x; e < a.d; e += blockDim.x) ss = fmaf(x[e], x[e], ss);
    ss = warp_sum(ss);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        v = warp_sum(v);
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    float inv = 1.0f / sqrtf(red[0] / (float)a.d + 1e-6f);
    for (int e = threadIdx.x; e < a.d; e += blockDim.x) xn[e] = x[e] * inv * a.g[e];
    __syncthreads();
    for (int e = threadIdx.x; e < a.d; e += blockDim.x) {
        float am = 0.0f, as = 0.0f;
        for (int i = 0; i < a.d; i++) {
            am = fmaf(xn[i], a.W1m[(long)i * a.d + e], am);
            as = fmaf(xn[i], a.W1s[(long)i * a.d + e], as);
        }
        hm[e] = silu_f(am + a.b1m[e]);
        hs[e] = silu_f(as + a.b1s[e]);
    }
    __syncthreads();
    const float lo = logf(0.11f), hi = logf(256.0f);
    for (int c = threadIdx.x; c < a.C; c += blockDim.x) {
        float om = 0.0f, os = 0.0f;
        for (int e = 0; e < a.d; e++) {
            om = fmaf(hm[e], a.W2m[(long)e * a.C + c], om);
            os = fmaf(hs[e], a.W2s[(long)e * a.C + c], os);
        }
        float mu = a.gamma_mu[c] * om + a.beta_mu[c];
        float v = a.gamma_sig[c] * os + a.beta_sig[c];
        float sg = expf(fminf(fmaxf(v, lo), hi));
        long o = (long)p * a.C + c;
        a.mu[o] = mu;
        a.sigma[o] = sg;
        quantize_one(mu, sg, stab, a.idx[o], a.m[o]);
    }
}

void launch_heads(const HeadsArgs &h, cudaStream_t s)
{
    if (h.n <= 0) return;
    k_heads<<<h.n, 256, 3 * h.d * sizeof(float), s>>>(h);
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
    const Epi &e = g.epi;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int m = m0 + tm * 4 + i;
        if (m >= g.M) continue;
        int p = e.pos ? e.pos[m] : m;
#pragma unroll
        for (int j = 0; j < 2; j++) {
            int n = n0 + tn * 2 + j;
            if (n >= g.N) continue;
            float y = acc[i][j];
            switch (e.mode) {
            case EPI_STORE:
                ((T *)e.out)[(long)(e.scatter ? p : m) * e.ld_out + n] = from_f<T>(y);
                break;
            case EPI_QKV:
                if (n < e.q_cols) ((T *)e.out)[(long)m * e.ld_out + n] = from_f<T>(y);
                else if (n < e.q_cols + e.d) ((T *)e.kc)[(long)p * e.d + (n - e.q_cols)] = from_f<T>(y);
                else ((T *)e.vc)[(long)p * e.d + (n - e.q_cols - e.d)] = from_f<T>(y);
                break;
            case EPI_RESID:
                e.resid[(long)p * g.N + n] += y;
                break;
            case EPI_RESID_BASE:
                e.resid[(long)p * g.N + n] = e.base[(long)p * g.N + n] + y;
                break;
            case EPI_SWIGLU:
                ((T *)e.out)[(long)m * e.ld_out + n] = from_f<T>(silu_f(y) * acc2[i][j]);
                break;
            }
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

bool gemm(int prec, const GemmArgs &g, cudaStream_t s)
{
    if (g.M <= 0 || g.N <= 0) return true;
    if (gemm_tc_supported(prec, g.N, g.K)) return gemm_tc(g, s);
    gemm_simt(prec, g, s);
    return true;
}

}  // namespace psw
