// gemm_tc.cu -- the BF16 projection GEMM as one kernel launch per
// projection: one 128-feature x 64-token tile per CTA (the tile functions of
// gemm_dev.cuh), weights prefetched before the programmatic-dependent-launch
// wait, plus the host side shared with the persistent decoder (tensor maps,
// shared-memory sizes, kernel attributes).
#include "gemm_dev.cuh"

#include <map>
#include <mutex>
#include <tuple>

namespace psw {

using namespace tc;

namespace {

template <bool DUAL, int MODE>
__global__ void __launch_bounds__(NTHREADS, 1)
k_gemm_tc(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmW2,
          const __grid_constant__ CUtensorMap tmX, GemmArgs g, int *status)
{
    constexpr uint32_t TCOLS = tile_tcols(DUAL);
    extern __shared__ uint8_t smem_raw[];
    __shared__ GemmShared S;
    uint8_t *ring = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int f0 = blockIdx.x * TM, m0 = blockIdx.y * NT;
    if (threadIdx.x == 0) gemm_shared_init(S);
    if ((threadIdx.x >> 5) == 0) tmem_alloc(&S.tmem_slot, TCOLS);
    __syncthreads();                                   // barriers initialised before any warp issues copies
    pdl_trigger();
    // token lists, the slot table and the scale table are fixed for the
    // whole decode, and the weights for the context's life: read them before
    // waiting for the previous kernel
    GemmPipe pp;
    int first = gemm_tile_pre<DUAL, MODE>(S, ring, &tmW, &tmW2, g, f0, m0, pp);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_slot;
    pdl_wait();                                        // activations are ready from here on
    gemm_tile_main<DUAL, MODE>(S, ring, tmem, &tmW, &tmW2, &tmX, g, f0, m0, first, pp);
    if (threadIdx.x == 0 && S.abort) atomicOr(status, ST_TIMEOUT);
    if ((threadIdx.x >> 5) == 0) tmem_free(tmem, TCOLS);
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_mu;
EncodeTiledFn g_encode = nullptr;
std::map<std::tuple<const void *, int, int, int, int>, CUtensorMap> g_maps;

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

// 2D bf16 [rows][ld] (K used columns) with a box of box_rows x 64, 128-byte
// swizzle; rows past the end read as zero.
bool tensor_map(const void *ptr, int rows, int K, int ld, int box_rows, CUtensorMap *out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_tuple(ptr, rows, K, ld, box_rows);
    auto it = g_maps.find(key);
    if (it != g_maps.end()) { *out = it->second; return true; }
    EncodeTiledFn enc = encoder();
    if (!enc) return false;
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    if (g_maps.size() > 65536) g_maps.clear();
    g_maps[key] = m;
    *out = m;
    return true;
}

size_t smem_bytes(bool dual, bool resident, int K) { return (size_t)tile_smem(dual, resident, K) + 1024; }

}  // namespace

bool gemm_tensor_map(const void *ptr, int rows, int K, int ld, int box_rows, CUtensorMap *out)
{
    return tensor_map(ptr, rows, K, ld, box_rows, out);
}

bool gemm_tc_supported(int prec, int N, int K, int asrc)
{
    return prec == P_BF16 && K % KC == 0 && K >= KC && N >= 1 && (asrc == A_DIRECT || K <= KRES_MAX);
}

template <bool DUAL, int MODE>
bool set_attr(size_t bytes)
{
    return cudaFuncSetAttribute(k_gemm_tc<DUAL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
           cudaSuccess;
}

// Checks for the tensor-map entry point and raises the kernels' dynamic
// shared-memory limit (done before any stream capture).
bool gemm_tc_available()
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!encoder()) return false;
    size_t m2 = RING_BUDGET + 1024, m1 = RING_BUDGET + 1024;
    return set_attr<true, EPI_SWIGLU>(m2) && set_attr<false, EPI_STORE>(m1) && set_attr<false, EPI_QKV>(m1) &&
           set_attr<false, EPI_RESID>(m1) && set_attr<false, EPI_RESID_BASE>(m1) &&
           set_attr<false, EPI_BIAS_SILU>(m1) && set_attr<false, EPI_SET_BIAS>(m1) && set_attr<false, EPI_HEADS>(m1);
}

bool gemm_tc(const GemmArgs &g, cudaStream_t s)
{
    CUtensorMap tw, tw2, tx;
    bool dual = g.epi.mode == EPI_SWIGLU;
    bool resident = g.asrc != A_DIRECT;
    if (!tensor_map(g.Wt, g.N, g.K, g.K, TM, &tw)) return false;
    if (dual && !tensor_map(g.Wt2, g.N, g.K, g.K, TM, &tw2)) return false;
    if (!dual) tw2 = tw;
    if (!resident) {
        if (!tensor_map(g.A, g.M, g.K, g.lda, NT, &tx)) return false;
    } else {
        tx = tw;
    }
    dim3 grid((g.N + TM - 1) / TM, (g.M + NT - 1) / NT);
    size_t smem = smem_bytes(dual, resident, g.K);
    int *st = g.status;
    dim3 block(NTHREADS);
    cudaError_t e;
    switch (g.epi.mode) {
    case EPI_SWIGLU: e = launch_pdl(k_gemm_tc<true, EPI_SWIGLU>, grid, block, smem, s, tw, tw2, tx, g, st); break;
    case EPI_STORE: e = launch_pdl(k_gemm_tc<false, EPI_STORE>, grid, block, smem, s, tw, tw2, tx, g, st); break;
    case EPI_QKV: e = launch_pdl(k_gemm_tc<false, EPI_QKV>, grid, block, smem, s, tw, tw2, tx, g, st); break;
    case EPI_RESID: e = launch_pdl(k_gemm_tc<false, EPI_RESID>, grid, block, smem, s, tw, tw2, tx, g, st); break;
    case EPI_RESID_BASE:
        e = launch_pdl(k_gemm_tc<false, EPI_RESID_BASE>, grid, block, smem, s, tw, tw2, tx, g, st);
        break;
    case EPI_BIAS_SILU:
        e = launch_pdl(k_gemm_tc<false, EPI_BIAS_SILU>, grid, block, smem, s, tw, tw2, tx, g, st);
        break;
    case EPI_SET_BIAS: e = launch_pdl(k_gemm_tc<false, EPI_SET_BIAS>, grid, block, smem, s, tw, tw2, tx, g, st); break;
    case EPI_HEADS: e = launch_pdl(k_gemm_tc<false, EPI_HEADS>, grid, block, smem, s, tw, tw2, tx, g, st); break;
    default: return false;
    }
    return e == cudaSuccess;
}

}  // namespace psw
