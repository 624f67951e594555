// gemm_tc.cu -- the BF16 and E4M3 projection GEMMs as one kernel launch per
// projection: one 128-feature x 64-token tile per CTA (the tile functions of
// gemm_dev.cuh), weights prefetched before the programmatic-dependent-launch
// wait, plus the host side shared with the persistent decoder (tensor maps,
// shared-memory sizes, kernel attributes) and the E4M3 weight quantiser.
#include "gemm_dev.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

namespace psw {

using namespace tc;

namespace {

// LEAN: the single-accumulator tile with the smaller ring, two CTAs per SM
// (one's token build and epilogue overlap the other's copies and MMAs);
// chosen for launches with more tiles than SMs.  Same arithmetic as the
// one-CTA form.
// TN: tokens per tile, 64, or 32 for launches whose 64-token grid leaves SMs
// idle (twice the CTAs, each with half the token build and epilogue).
template <bool DUAL, int MODE, bool F8, bool LEAN = false, int TN = NT>
__global__ void __launch_bounds__(NTHREADS, LEAN ? 2 : 1)
k_gemm_tc(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmW2,
          const __grid_constant__ CUtensorMap tmX, GemmArgs g, int *status)
{
    constexpr uint32_t TCOLS = tile_tcols(DUAL, TN);
    extern __shared__ uint8_t smem_raw[];
    __shared__ GemmShared S;
    uint8_t *ring = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int f0 = blockIdx.x * TM, m0 = blockIdx.y * TN;
    if (threadIdx.x == 0) gemm_shared_init(S);
    if ((threadIdx.x >> 5) == 0) tmem_alloc(&S.tmem_slot, TCOLS);
    __syncthreads();                                   // barriers initialised before any warp issues copies
    pdl_trigger();
    // token lists, the slot table and the scale table are fixed for the
    // whole decode, and the weights for the context's life: read them before
    // waiting for the previous kernel
    GemmPipe pp;
    int first = gemm_tile_pre<DUAL, MODE, F8, LEAN, TN>(S, ring, &tmW, &tmW2, g, f0, m0, pp);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_slot;
    pdl_wait();                                        // activations are ready from here on
    gemm_tile_main<DUAL, MODE, F8, LEAN, TN>(S, ring, tmem, &tmW, &tmW2, &tmX, g, f0, m0, first, pp);
    if (threadIdx.x == 0 && S.abort) atomicOr(status, ST_TIMEOUT);
    if ((threadIdx.x >> 5) == 0) tmem_free(tmem, TCOLS);
}

// RMSNorm rows for a projection whose tiles stream their token operand:
// dst[m] = bf16(RMSNorm(X[m]) * gain), R consecutive rows per warp with all
// their loads issued before the first reduction, eight warps per block, the
// gains staged in shared memory before the wait for the previous kernel
// (norm_row_store: the same values a tile would build, whatever R).
// Blocks per SM the registers are bounded for: the R x CH float4 of a
// warp's rows stay in registers without spilling.
template <int CH, int R>
constexpr int norm_rows_min_blocks() { return R == 1 ? 1 : CH * R <= 6 ? 4 : CH * R <= 12 ? 3 : 2; }

template <int CH, int R>
__global__ void __launch_bounds__(256, norm_rows_min_blocks<CH, R>())
k_norm_rows(const float *__restrict__ X, const float *__restrict__ gain, int M, int K, __nv_bfloat16 *__restrict__ dst,
            int ldd)
{
    __shared__ float4 sg[CH * 32];
    pdl_trigger();
    for (int i = threadIdx.x; i < CH * 32; i += blockDim.x) {
        const int e = 4 * i;
        sg[i] = e < K ? make_float4(gain[e], gain[e + 1], gain[e + 2], gain[e + 3]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const float invK = 1.0f / (float)K;
    const int lane = threadIdx.x & 31;
    const long m0 = ((long)blockIdx.x * 8 + (threadIdx.x >> 5)) * R;
    pdl_wait();
    float4 v[R][CH];
#pragma unroll
    for (int b = 0; b < R; b++) {
        const float *x = m0 + b < M ? X + (m0 + b) * K : nullptr;
#pragma unroll
        for (int c = 0; c < CH; c++) {
            const int e = lane * 4 + c * 128;
            v[b][c] = (x && e < K) ? *(const float4 *)(x + e) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    float4 gh[CH];
#pragma unroll
    for (int c = 0; c < CH; c++) gh[c] = sg[lane + 32 * c];
#pragma unroll
    for (int b = 0; b < R; b++)
        if (m0 + b < M) norm_row_store<CH>(v[b], gh, invK, K, dst + (m0 + b) * ldd);
}

// The latent embedding's operand rows for a projection whose tiles stream
// them: dst[m][k] = bf16(gain[k] * y[k]) of token m's latents, one warp per
// row, eight rows per block (the values embed_rows builds in a tile: lane l
// holds elements 4l + 128c .. +3).
__global__ void __launch_bounds__(256) k_embed_rows(const Slot *__restrict__ S, const int *__restrict__ tok, int M,
                                                    const float *__restrict__ gain, int K,
                                                    __nv_bfloat16 *__restrict__ dst)
{
    pdl_trigger();
    const int m = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    pdl_wait();
    if (m >= M) return;
    const int tk = tok[m];
    const int16_t *y = S[tok_slot(tk)].y + (long)tok_pos(tk) * K;
    for (int e = lane * 4; e < K; e += 128) {
        const short4 q = *(const short4 *)(y + e);
        *(uint2 *)(dst + (long)m * K + e) = pack4(gain[e] * (float)q.x, gain[e + 1] * (float)q.y,
                                                  gain[e + 2] * (float)q.z, gain[e + 3] * (float)q.w);
    }
}

// E4M3 streamed rows: R consecutive rows per warp with all their loads
// issued before the first reduction, eight warps per block; each row's
// arithmetic is norm_row8_store's or quant_row8_store's, whatever R.
template <int CH, int R>
__global__ void __launch_bounds__(256, norm_rows_min_blocks<CH, R>())
k_rows8_norm(const float *__restrict__ X, const float *__restrict__ gain, int M, int K, uint8_t *__restrict__ dst,
             float *__restrict__ xs)
{
    __shared__ float4 sg[CH * 32];
    pdl_trigger();
    for (int i = threadIdx.x; i < CH * 32; i += blockDim.x) {
        const int e = 4 * i;
        sg[i] = e < K ? make_float4(gain[e], gain[e + 1], gain[e + 2], gain[e + 3]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const float invK = 1.0f / (float)K;
    const int lane = threadIdx.x & 31;
    const long m0 = ((long)blockIdx.x * 8 + (threadIdx.x >> 5)) * R;
    pdl_wait();
    float4 v[R][CH];
#pragma unroll
    for (int b = 0; b < R; b++) {
        const float *x = m0 + b < M ? X + (m0 + b) * K : nullptr;
#pragma unroll
        for (int c = 0; c < CH; c++) {
            const int e = lane * 4 + c * 128;
            v[b][c] = (x && e < K) ? *(const float4 *)(x + e) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    float4 gh[CH];
#pragma unroll
    for (int c = 0; c < CH; c++) gh[c] = sg[lane + 32 * c];
#pragma unroll
    for (int b = 0; b < R; b++)
        if (m0 + b < M) norm_row8_store<CH>(v[b], gh, invK, K, dst + (m0 + b) * K, xs + m0 + b);
}

template <int CH, int R>
__global__ void __launch_bounds__(256, norm_rows_min_blocks<CH, R>())
k_rows8_quant(const __nv_bfloat16 *__restrict__ A, int lda, int M, int K, uint8_t *__restrict__ dst,
              float *__restrict__ xs)
{
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const long m0 = ((long)blockIdx.x * 8 + (threadIdx.x >> 5)) * R;
    pdl_wait();
    uint4 q[R][CH];
#pragma unroll
    for (int b = 0; b < R; b++) {
        const __nv_bfloat16 *row = m0 + b < M ? A + (m0 + b) * lda : nullptr;
#pragma unroll
        for (int c = 0; c < CH; c++) {
            const int e = lane * 8 + c * 256;
            q[b][c] = (row && e < K) ? *(const uint4 *)(row + e) : make_uint4(0, 0, 0, 0);
        }
    }
#pragma unroll
    for (int b = 0; b < R; b++)
        if (m0 + b < M) quant_row8_store<CH>(q[b], K, dst + (m0 + b) * K, xs + m0 + b);
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_mu;
EncodeTiledFn g_encode = nullptr;
std::map<std::tuple<const void *, int, int, int, int, bool>, CUtensorMap> g_maps;

EncodeTiledFn encoder()
{
    if (!g_encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (EncodeTiledFn)fn;
    }
    return g_encode;
}

// 2D bf16 [rows][ld] (K used columns) with a box of box_rows x 64 (E4M3,
// f8: box_rows x 128 bytes), 128-byte swizzle; rows past the end read as
// zero.
bool tensor_map(const void *ptr, int rows, int K, int ld, int box_rows, CUtensorMap *out, bool f8 = false)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_tuple(ptr, rows, K, ld, box_rows, f8);
    auto it = g_maps.find(key);
    if (it != g_maps.end()) { *out = it->second; return true; }
    EncodeTiledFn enc = encoder();
    if (!enc) return false;
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * (f8 ? 1 : 2)};
    cuuint32_t box[2] = {(cuuint32_t)kchunk(f8), (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(&m, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    if (g_maps.size() > 65536) g_maps.clear();
    g_maps[key] = m;
    *out = m;
    return true;
}

size_t smem_bytes(bool dual, bool resident, int K, bool f8 = false, bool lean = false, int tn = NT)
{
    return (size_t)tile_smem(dual, resident, K, f8, lean, tn) + 1024;
}


// Multiprocessors of the current device (lean tiles pay off past one wave).
int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// Tokens per tile of a launch: 32 when the 64-token grid fills less than the
// SMs and the 32-token grid still fits in one wave.
int tile_tokens(int nf, int M)
{
    const int t64 = nf * ((M + 63) / 64), t32 = nf * ((M + 31) / 32);
    return t64 < sm_count() && t32 <= sm_count() ? 32 : 64;
}

// Rows per warp of the row producers: the most (1, 2 or 4) that still
// leaves two blocks of eight warps per SM.
int rows_per_warp(int M)
{
    return (M + 31) / 32 >= 2 * sm_count() ? 4 : (M + 15) / 16 >= 2 * sm_count() ? 2 : 1;
}

// ---------------------------------------------------------------- E4M3 weights

__global__ void k_absmax(const float *__restrict__ src, size_t n, unsigned *out)
{
    float a = 0.0f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        a = fmaxf(a, fabsf(src[i]));
    a = warp_max(a);
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(a));     // non-negative: bit order = value order
}

__global__ void k_quant_e4m3(const float *__restrict__ src, size_t n, float qmul, uint8_t *__restrict__ dst)
{
    size_t n4 = n / 4;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        float4 v = reinterpret_cast<const float4 *>(src)[i];
        reinterpret_cast<uint32_t *>(dst)[i] = e4m3x4(v.x * qmul, v.y * qmul, v.z * qmul, v.w * qmul);
    }
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t < n - 4 * n4) {
        size_t i = 4 * n4 + t;
        dst[i] = (uint8_t)(e4m3x4(src[i] * qmul, 0.0f, 0.0f, 0.0f) & 255u);
    }
}

}  // namespace

bool launch_norm_rows(const float *X, const float *gain, int M, int K, void *dst, cudaStream_t s, int ldd)
{
    if (M <= 0) return true;
    if (ldd <= 0) ldd = K;
    if (K > KRES_MAX || K % 4 || ldd < K || ldd % 8 || ((uintptr_t)dst & 15)) return false;
    const int R = rows_per_warp(M);
    dim3 grid((M + 8 * R - 1) / (8 * R)), block(256);
    __nv_bfloat16 *d = (__nv_bfloat16 *)dst;
    cudaError_t e;
    if (K <= 384)
        e = R == 4 ? launch_pdl(k_norm_rows<3, 4>, grid, block, 0, s, X, gain, M, K, d, ldd)
          : R == 2 ? launch_pdl(k_norm_rows<3, 2>, grid, block, 0, s, X, gain, M, K, d, ldd)
                   : launch_pdl(k_norm_rows<3, 1>, grid, block, 0, s, X, gain, M, K, d, ldd);
    else
        e = R == 4 ? launch_pdl(k_norm_rows<4, 4>, grid, block, 0, s, X, gain, M, K, d, ldd)
          : R == 2 ? launch_pdl(k_norm_rows<4, 2>, grid, block, 0, s, X, gain, M, K, d, ldd)
                   : launch_pdl(k_norm_rows<4, 1>, grid, block, 0, s, X, gain, M, K, d, ldd);
    return e == cudaSuccess;
}

bool launch_embed_rows(const Slot *S, const int *tok, int M, const float *gain, int K, void *dst, cudaStream_t s)
{
    if (M <= 0) return true;
    if (K % 4 || ((uintptr_t)dst & 15)) return false;
    return launch_pdl(k_embed_rows, dim3((M + 7) / 8), dim3(256), 0, s, S, tok, M, gain, K, (__nv_bfloat16 *)dst) ==
           cudaSuccess;
}

bool launch_rows8(int asrc, const float *X, const float *gain, const void *A, int lda, int M, int K, uint8_t *dst,
                  float *xs, cudaStream_t s)
{
    if (M <= 0) return true;
    if (K % KC8 || ((uintptr_t)dst & 15)) return false;
    const int R = rows_per_warp(M);
    dim3 grid((M + 8 * R - 1) / (8 * R)), block(256);
    cudaError_t e;
    if (asrc == A_NORM) {
        if (K > KRES_MAX) return false;
        if (K <= 384)
            e = R == 4 ? launch_pdl(k_rows8_norm<3, 4>, grid, block, 0, s, X, gain, M, K, dst, xs)
              : R == 2 ? launch_pdl(k_rows8_norm<3, 2>, grid, block, 0, s, X, gain, M, K, dst, xs)
                       : launch_pdl(k_rows8_norm<3, 1>, grid, block, 0, s, X, gain, M, K, dst, xs);
        else
            e = R == 4 ? launch_pdl(k_rows8_norm<4, 4>, grid, block, 0, s, X, gain, M, K, dst, xs)
              : R == 2 ? launch_pdl(k_rows8_norm<4, 2>, grid, block, 0, s, X, gain, M, K, dst, xs)
                       : launch_pdl(k_rows8_norm<4, 1>, grid, block, 0, s, X, gain, M, K, dst, xs);
    } else {
        if (K > 1024 || lda % 8) return false;
        const __nv_bfloat16 *Ab = (const __nv_bfloat16 *)A;
        if (K <= 512)
            e = R == 4 ? launch_pdl(k_rows8_quant<2, 4>, grid, block, 0, s, Ab, lda, M, K, dst, xs)
              : R == 2 ? launch_pdl(k_rows8_quant<2, 2>, grid, block, 0, s, Ab, lda, M, K, dst, xs)
                       : launch_pdl(k_rows8_quant<2, 1>, grid, block, 0, s, Ab, lda, M, K, dst, xs);
        else
            e = R == 4 ? launch_pdl(k_rows8_quant<4, 4>, grid, block, 0, s, Ab, lda, M, K, dst, xs)
              : R == 2 ? launch_pdl(k_rows8_quant<4, 2>, grid, block, 0, s, Ab, lda, M, K, dst, xs)
                       : launch_pdl(k_rows8_quant<4, 1>, grid, block, 0, s, Ab, lda, M, K, dst, xs);
    }
    return e == cudaSuccess;
}

bool gemm_tensor_map(const void *ptr, int rows, int K, int ld, int box_rows, CUtensorMap *out, bool f8)
{
    return tensor_map(ptr, rows, K, ld, box_rows, out, f8);
}

bool gemm_tc_supported(int prec, int N, int K, int asrc)
{
    return prec == P_BF16 && K % KC == 0 && K >= KC && N >= 1 && (asrc == A_DIRECT || K <= KRES_MAX);
}

// E4M3 projections: whole 128-element chunks, a token operand the CTA can
// build (RMSNorm rows up to 512 wide, bf16 rows up to 1024) and a weight ring
// that fits beside it.
bool gemm_tc8_supported(int N, int K, int asrc)
{
    if (N < 1 || K < KC8 || K % KC8) return false;
    if (!(asrc == A_NORM ? K <= KRES_MAX : asrc == A_DIRECT ? K <= 1024 : false)) return false;
    return tile_smem(true, true, K, true) <= RING_BUDGET;
}

float quantize_e4m3(const float *src, size_t n, uint8_t *dst)
{
    if (n == 0) return 1.0f;
    unsigned *d_max = nullptr, bits = 0;
    if (cudaMalloc(&d_max, sizeof(unsigned)) != cudaSuccess) return -1.0f;
    cudaMemset(d_max, 0, sizeof(unsigned));
    int blocks = (int)std::min<size_t>((n + 255) / 256, 1024);
    k_absmax<<<blocks, 256>>>(src, n, d_max);
    cudaError_t e = cudaMemcpy(&bits, d_max, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(d_max);
    if (e != cudaSuccess) return -1.0f;
    float amax;
    memcpy(&amax, &bits, sizeof amax);
    if (!(amax <= 3.0e38f)) return -1.0f;                              // NaN or Inf among the weights
    int ex = 0;
    if (amax > 0.0f) std::frexp(amax, &ex);                            // amax = f 2^ex, f in [0.5, 1)
    int el = amax > 0.0f ? std::max(ex - 1, -100) : 7;                 // max |w| in [2^el, 2^(el+1))
    float s = std::ldexp(1.0f, el - 7), qmul = std::ldexp(1.0f, 7 - el);
    k_quant_e4m3<<<blocks, 256>>>(src, n, qmul, dst);
    if (cudaDeviceSynchronize() != cudaSuccess) return -1.0f;
    return s;
}

template <bool DUAL, int MODE, bool F8 = false, bool LEAN = false, int TN = NT>
bool set_attr(size_t bytes)
{
    auto k = k_gemm_tc<DUAL, MODE, F8, LEAN, TN>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) return false;
    // lean tiles: room for two CTAs' shared memory on one SM
    return !LEAN || cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared) == cudaSuccess;
}

// Checks for the tensor-map entry point and raises the kernels' dynamic
// shared-memory limit (done before any stream capture).
static bool set_narrow_attrs()
{
    const size_t m = RING_BUDGET + 1024;
    return set_attr<true, EPI_SWIGLU, false, false, 32>(m) && set_attr<false, EPI_STORE, false, false, 32>(m) &&
           set_attr<false, EPI_QKV, false, false, 32>(m) && set_attr<false, EPI_RESID, false, false, 32>(m) &&
           set_attr<false, EPI_RESID_BASE, false, false, 32>(m) && set_attr<false, EPI_BIAS_SILU, false, false, 32>(m) &&
           set_attr<false, EPI_SET_BIAS, false, false, 32>(m) && set_attr<false, EPI_HEADS, false, false, 32>(m) &&
           set_attr<true, EPI_SWIGLU, true, false, 32>(m) && set_attr<false, EPI_STORE, true, false, 32>(m) &&
           set_attr<false, EPI_QKV, true, false, 32>(m) && set_attr<false, EPI_RESID, true, false, 32>(m) &&
           set_attr<false, EPI_RESID_BASE, true, false, 32>(m);
}

static bool set_lean_attrs()
{
    const size_t ml = RING_BUDGET_LEAN + 1024;
    return set_attr<false, EPI_STORE, false, true>(ml) && set_attr<false, EPI_QKV, false, true>(ml) &&
           set_attr<false, EPI_RESID, false, true>(ml) && set_attr<false, EPI_RESID_BASE, false, true>(ml) &&
           set_attr<false, EPI_BIAS_SILU, false, true>(ml) && set_attr<false, EPI_SET_BIAS, false, true>(ml) &&
           set_attr<false, EPI_HEADS, false, true>(ml) && set_attr<false, EPI_STORE, true, true>(ml) &&
           set_attr<false, EPI_QKV, true, true>(ml) && set_attr<false, EPI_RESID, true, true>(ml) &&
           set_attr<false, EPI_RESID_BASE, true, true>(ml);
}

bool gemm_tc_available()
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!encoder()) return false;
    size_t m2 = RING_BUDGET + 1024, m1 = RING_BUDGET + 1024;
    return set_attr<true, EPI_SWIGLU>(m2) && set_attr<false, EPI_STORE>(m1) && set_attr<false, EPI_QKV>(m1) &&
           set_attr<false, EPI_RESID>(m1) && set_attr<false, EPI_RESID_BASE>(m1) &&
           set_attr<false, EPI_BIAS_SILU>(m1) && set_attr<false, EPI_SET_BIAS>(m1) && set_attr<false, EPI_HEADS>(m1) &&
           set_attr<true, EPI_SWIGLU, true>(m2) && set_attr<false, EPI_STORE, true>(m1) &&
           set_attr<false, EPI_QKV, true>(m1) && set_attr<false, EPI_RESID, true>(m1) &&
           set_attr<false, EPI_RESID_BASE, true>(m1) && set_lean_attrs() && set_narrow_attrs();
}

namespace {

// E4M3 projection launch: the five epilogues block projections use.
bool gemm_tc8(const GemmArgs &g, cudaStream_t s)
{
    CUtensorMap tw, tw2;
    bool dual = g.epi.mode == EPI_SWIGLU;
    if (!g.wsc || (dual && !g.wsc2) || !gemm_tc8_supported(g.N, g.K, g.asrc)) return false;
    if (!tensor_map(g.Wt, g.N, g.K, g.K, TM, &tw, true)) return false;
    if (dual && !tensor_map(g.Wt2, g.N, g.K, g.K, TM, &tw2, true)) return false;
    if (!dual) tw2 = tw;
    const int nf = (g.N + TM - 1) / TM, tn = tile_tokens(nf, g.M);
    dim3 grid(nf, (g.M + tn - 1) / tn), block(NTHREADS);
    const bool lean = !dual && tn == NT && (int)(grid.x * grid.y) > sm_count();
    size_t smem = smem_bytes(dual, true, g.K, true, lean, tn);
    int *st = g.status;
    cudaError_t e;
#define F8_CASE(MODE_)                                                                                         \
    case MODE_:                                                                                                \
        e = tn == 32 ? launch_pdl(k_gemm_tc<false, MODE_, true, false, 32>, grid, block, smem, s, tw, tw2, tw, g, st) \
            : lean   ? launch_pdl(k_gemm_tc<false, MODE_, true, true>, grid, block, smem, s, tw, tw2, tw, g, st)      \
                     : launch_pdl(k_gemm_tc<false, MODE_, true, false>, grid, block, smem, s, tw, tw2, tw, g, st);    \
        break;
    switch (g.epi.mode) {
    case EPI_SWIGLU:
        e = tn == 32 ? launch_pdl(k_gemm_tc<true, EPI_SWIGLU, true, false, 32>, grid, block, smem, s, tw, tw2, tw, g, st)
                     : launch_pdl(k_gemm_tc<true, EPI_SWIGLU, true>, grid, block, smem, s, tw, tw2, tw, g, st);
        break;
    F8_CASE(EPI_STORE)
    F8_CASE(EPI_QKV)
    F8_CASE(EPI_RESID)
    F8_CASE(EPI_RESID_BASE)
    default: return false;
    }
#undef F8_CASE
    return e == cudaSuccess;
}

}  // namespace

bool gemm_tc(const GemmArgs &g, cudaStream_t s)
{
    if (g.f8) return gemm_tc8(g, s);
    CUtensorMap tw, tw2, tx;
    bool dual = g.epi.mode == EPI_SWIGLU;
    bool resident = g.asrc != A_DIRECT;
    if (!tensor_map(g.Wt, g.N, g.K, g.K, TM, &tw)) return false;
    if (dual && !tensor_map(g.Wt2, g.N, g.K, g.K, TM, &tw2)) return false;
    if (!dual) tw2 = tw;
    const int nf = (g.N + TM - 1) / TM, tn = tile_tokens(nf, g.M);
    if (!resident) {
        if (!tensor_map(g.A, g.M, g.K, g.lda, tn, &tx)) return false;
    } else {
        tx = tw;
    }
    dim3 grid(nf, (g.M + tn - 1) / tn);
    const bool lean = !dual && tn == NT && (int)(grid.x * grid.y) > sm_count();
    size_t smem = smem_bytes(dual, resident, g.K, false, lean, tn);
    int *st = g.status;
    dim3 block(NTHREADS);
    cudaError_t e;
#define BF_CASE(MODE_)                                                                                            \
    case MODE_:                                                                                                   \
        e = tn == 32 ? launch_pdl(k_gemm_tc<false, MODE_, false, false, 32>, grid, block, smem, s, tw, tw2, tx, g, st) \
            : lean   ? launch_pdl(k_gemm_tc<false, MODE_, false, true>, grid, block, smem, s, tw, tw2, tx, g, st)      \
                     : launch_pdl(k_gemm_tc<false, MODE_, false, false>, grid, block, smem, s, tw, tw2, tx, g, st);    \
        break;
    switch (g.epi.mode) {
    case EPI_SWIGLU:
        e = tn == 32 ? launch_pdl(k_gemm_tc<true, EPI_SWIGLU, false, false, 32>, grid, block, smem, s, tw, tw2, tx, g, st)
                     : launch_pdl(k_gemm_tc<true, EPI_SWIGLU, false>, grid, block, smem, s, tw, tw2, tx, g, st);
        break;
    BF_CASE(EPI_STORE)
    BF_CASE(EPI_QKV)
    BF_CASE(EPI_RESID)
    BF_CASE(EPI_RESID_BASE)
    BF_CASE(EPI_BIAS_SILU)
    BF_CASE(EPI_SET_BIAS)
    BF_CASE(EPI_HEADS)
    default: return false;
    }
#undef BF_CASE
    return e == cudaSuccess;
}

}  // namespace psw
