// hyper.cu -- data movement of the convolutional hyperprior (Fig. 1 right:
// down- and upsampling residual blocks around z, z-hat coded under a
// factorized prior).  The convolutions themselves are projections: each
// kernel here builds the token operand of one (an im2col gather of 3 x 3
// or strided 1 x 1 taps, with the LeakyReLU of the block and the pixel
// shuffle of a sub-pixel convolution folded into the gather), or moves a
// grid between the layouts the projections write.  Grids are FP32,
// channel-last [h][w][C]; every element's value depends only on its own
// inputs, never on the launch shape.
#include "internal.h"
#include "device_common.cuh"

#include <algorithm>

namespace psw {

static inline int cdiv_l(long a, long b) { return (int)((a + b - 1) / b); }
static inline int grid_of(long n, int tpb) { return (int)std::min<long>(cdiv_l(n, tpb), 152L * 16); }

// Element (i, j, c) of a logical [h][w][C] grid stored plainly, or (view 1)
// as the pixel-shuffle source of a sub-pixel convolution, positions of the
// [h/2][w/2] grid ls floats apart: (i, j, c) = u[i/2][j/2][(2 (i%2) + j%2) C + c].
__device__ __forceinline__ float grid_at(const float *src, int w, int C, int view, int ls, int i, int j, int c)
{
    if (view == 0) return src[((long)i * w + j) * C + c];
    const int wl = w >> 1;
    return src[((long)(i >> 1) * wl + (j >> 1)) * ls + (2 * (i & 1) + (j & 1)) * C + c];
}

// dst[(io * wo + jo) * K + t * C + c] for t over the taps (ks = 3: the 3 x 3
// window at stride st, zero outside the grid, K = 9C; ks = 1: the single tap
// (st io, st jo), K = C), LeakyReLU (slope 0.01) applied to the source
// value when act is set, converted to the compute type.
template <typename T>
__global__ void k_im2col(const float *__restrict__ src, int h, int w, int C, int view, int ls, int act, int ks, int st,
                         int ho, int wo, T *__restrict__ dst)
{
    const int K = ks * ks * C;
    const long total = (long)ho * wo * K;
    for (long a = blockIdx.x * (long)blockDim.x + threadIdx.x; a < total; a += (long)gridDim.x * blockDim.x) {
        const long pos = a / K;
        const int k = (int)(a - pos * K), t = k / C, c = k - t * C;
        const int io = (int)(pos / wo), jo = (int)(pos - (long)io * wo);
        int i = st * io, j = st * jo;
        if (ks == 3) { i += t / 3 - 1; j += t % 3 - 1; }
        float v = 0.0f;
        if (i >= 0 && i < h && j >= 0 && j < w) {
            v = grid_at(src, w, C, view, ls, i, j, c);
            if (act) v = v >= 0.0f ? v : 0.01f * v;
        }
        dst[a] = from_f<T>(v);
    }
}

void launch_im2col(int prec, const float *src, int h, int w, int C, int view, int ls, int act, int ks, int st,
                   void *dst, cudaStream_t s)
{
    const int ho = (h - 1) / st + 1, wo = (w - 1) / st + 1;
    const long total = (long)ho * wo * ks * ks * C;
    if (total <= 0) return;
    if (ls <= 0) ls = 4 * C;
    if (prec == P_BF16)
        k_im2col<__nv_bfloat16><<<grid_of(total, 256), 256, 0, s>>>(src, h, w, C, view, ls, act, ks, st, ho, wo,
                                                                     (__nv_bfloat16 *)dst);
    else
        k_im2col<float><<<grid_of(total, 256), 256, 0, s>>>(src, h, w, C, view, ls, act, ks, st, ho, wo,
                                                             (float *)dst);
}

// dst [2h][2w][C] = pixel shuffle of src (positions of [h][w] ls floats
// apart, 4C values each used).
__global__ void k_shuffle(const float *__restrict__ src, int h, int w, int C, int ls, float *__restrict__ dst)
{
    const long total = (long)4 * h * w * C;
    for (long a = blockIdx.x * (long)blockDim.x + threadIdx.x; a < total; a += (long)gridDim.x * blockDim.x) {
        const long pos = a / C;
        const int c = (int)(a - pos * C);
        const int I = (int)(pos / (2 * w)), J = (int)(pos - (long)I * 2 * w);
        const int sub = 2 * (I & 1) + (J & 1);
        dst[a] = src[((long)(I >> 1) * w + (J >> 1)) * ls + sub * C + c];
    }
}

void launch_shuffle(const float *src, int h, int w, int C, int ls, float *dst, cudaStream_t s)
{
    const long total = (long)4 * h * w * C;
    if (total <= 0) return;
    k_shuffle<<<grid_of(total, 256), 256, 0, s>>>(src, h, w, C, ls, dst);
}

// The synthesis input: gamma[c] * z-hat of the slot of tok[0] as an FP32
// grid [Hh][Wh][Ch].
__global__ void k_zhat_grid(const Slot *__restrict__ S, const int *__restrict__ tok, int n, const float *__restrict__ gamma,
                            int Ch, float *__restrict__ dst)
{
    const Slot &sl = S[tok_slot(tok[0])];
    for (long a = blockIdx.x * (long)blockDim.x + threadIdx.x; a < (long)n * Ch; a += (long)gridDim.x * blockDim.x)
        dst[a] = gamma[a % Ch] * (float)sl.zhat[a];
}

void launch_zhat_grid(const Slot *S, const int *tok, int n, const float *gamma, int Ch, float *dst, cudaStream_t s)
{
    if (n <= 0) return;
    k_zhat_grid<<<grid_of((long)n * Ch, 256), 256, 0, s>>>(S, tok, n, gamma, Ch, dst);
}

// The hyperprior tokens of the slot of tok[0]: rows i < H, j < W of the
// synthesis grid [.][ws][d] copied to eh [H * W][d].
__global__ void k_crop_eh(const Slot *__restrict__ S, const int *__restrict__ tok, const float *__restrict__ src,
                          int ws, int H, int W, int d)
{
    const Slot &sl = S[tok_slot(tok[0])];
    const long total = (long)H * W * d;
    for (long a = blockIdx.x * (long)blockDim.x + threadIdx.x; a < total; a += (long)gridDim.x * blockDim.x) {
        const long p = a / d;
        const int e = (int)(a - p * d), i = (int)(p / W), j = (int)(p - (long)i * W);
        sl.eh[a] = src[((long)i * ws + j) * d + e];
    }
}

void launch_crop_eh(const Slot *S, const int *tok, const float *src, int ws, int H, int W, int d, cudaStream_t s)
{
    const long total = (long)H * W * d;
    if (total <= 0) return;
    k_crop_eh<<<grid_of(total, 256), 256, 0, s>>>(S, tok, src, ws, H, W, d);
}

// z-hat = round-half-even(z) clamped to int16 (the quantiser Q); z
// optionally copied out.
__global__ void k_round_z(const float *__restrict__ z, long n, int16_t *__restrict__ zhat, float *__restrict__ zout)
{
    for (long a = blockIdx.x * (long)blockDim.x + threadIdx.x; a < n; a += (long)gridDim.x * blockDim.x) {
        const float v = z[a];
        zhat[a] = (int16_t)rintf(fminf(fmaxf(v, -32768.0f), 32767.0f));
        if (zout) zout[a] = v;
    }
}

void launch_round_z(const float *z, long n, int16_t *zhat, float *zout, cudaStream_t s)
{
    if (n <= 0) return;
    k_round_z<<<grid_of(n, 256), 256, 0, s>>>(z, n, zhat, zout);
}

// The z-hat coder's per-symbol table index (the channel) and zero means,
// and the identity (raster) order.
__global__ void k_hyper_coder_tables(int HW, int Ch, uint8_t *__restrict__ idx, int32_t *__restrict__ m,
                                     int *__restrict__ order)
{
    for (long a = blockIdx.x * (long)blockDim.x + threadIdx.x; a < (long)HW * Ch; a += (long)gridDim.x * blockDim.x) {
        idx[a] = (uint8_t)(a % Ch);
        m[a] = 0;
        if (a < HW) order[a] = (int)a;
    }
}

void launch_hyper_coder_tables(int HW, int Ch, uint8_t *idx, int32_t *m, int *order, cudaStream_t s)
{
    if (HW <= 0) return;
    k_hyper_coder_tables<<<grid_of((long)HW * Ch, 256), 256, 0, s>>>(HW, Ch, idx, m, order);
}

}  // namespace psw
