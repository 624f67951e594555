// gemm_tc.cu -- BF16 projection GEMM on the sm_100-family tensor cores
// (tcgen05.mma, accumulator in tensor memory, operands staged by TMA).
//
// Y[token][feature] = sum_k X[token][k] Wt[feature][k].  The projection is
// the MMA's A operand (M = 128 output features per CTA) and the tokens are
// its B operand (N = 64 tokens per CTA), so a decoder step with a few dozen
// tokens fills one tile and the weights stream through once.  K is consumed
// in 64-element chunks (one 128-byte swizzle atom) through a 4-stage TMA ring;
// one thread issues the MMAs, 128 threads run the epilogue from TMEM
// (thread t holds feature row t of the tile).  Accumulation order is fixed
// (ascending K chunks), so every output element is the same function of its
// row and column whatever the tile or launch it falls in.
//
// Every mbarrier wait is bounded (~2 s of globaltimer); on expiry the CTA
// records ST_TIMEOUT, waits (bounded) for its own copies and MMAs, frees its
// tensor memory and returns.
#include "internal.h"

#include <cuda.h>

#include <map>
#include <mutex>
#include <tuple>

namespace psw {

namespace {

constexpr int TM = 128;        // output features per CTA (MMA M)
constexpr int NT = 64;         // tokens per CTA (MMA N)
constexpr int KC = 64;         // K elements per stage (128 bytes of bf16)
constexpr int STAGES = 4;
constexpr int A_BYTES = TM * KC * 2;
constexpr int B_BYTES = NT * KC * 2;
constexpr uint64_t WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on a phase of an mbarrier; false after ~2 s.
__device__ __noinline__ bool mbar_wait(uint64_t *b, uint32_t parity)
{
    if (mbar_try(b, parity)) return true;
    uint64_t t0 = gtime();
    while (!mbar_try(b, parity))
        if (gtime() - t0 > WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *tm, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(su32(dst)), "l"(tm), "r"(su32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row atoms 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
    d |= (uint64_t)1 << 46;                          // version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: F32 accumulate, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t dt, uint64_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dt), "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t addr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float silu_f(float x) { return x / (1.0f + expf(-x)); }

template <bool DUAL>
__global__ void __launch_bounds__(128, 1)
k_gemm_tc(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmW2,
          const __grid_constant__ CUtensorMap tmX, GemmArgs g, int *status)
{
    constexpr int NACC = DUAL ? 2 : 1;
    constexpr int STAGE = NACC * A_BYTES + B_BYTES;
    constexpr uint32_t TCOLS = DUAL ? 2 * NT : NT;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int f0 = blockIdx.x * TM, m0 = blockIdx.y * NT;
    const int nk = g.K / KC;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: TMA ring
        int issued = 0;
        for (int kc = 0; kc < nk; kc++) {
            int s = kc % STAGES, it = kc / STAGES;
            if (abort_flag) break;
            if (kc >= STAGES && !mbar_wait(&empty[s], (it - 1) & 1)) { abort_flag = 1; break; }
            uint8_t *st = smem + s * STAGE;
            mbar_expect_tx(&full[s], STAGE);
            tma_load(st, &tmW, &full[s], kc * KC, f0);
            if (DUAL) tma_load(st + A_BYTES, &tmW2, &full[s], kc * KC, f0);
            tma_load(st + NACC * A_BYTES, &tmX, &full[s], kc * KC, m0);
            issued = kc + 1;
        }
        if (abort_flag) {
            // let this CTA's copies land before it can exit
            for (int kc = (issued > STAGES ? issued - STAGES : 0); kc < issued; kc++)
                mbar_wait(&full[kc % STAGES], (kc / STAGES) & 1);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t id = idesc_bf16(TM, NT);
        for (int kc = 0; kc < nk; kc++) {
            int s = kc % STAGES, it = kc / STAGES;
            if (abort_flag) break;
            if (!mbar_wait(&full[s], it & 1)) { abort_flag = 1; break; }
            fence_after();
            uint32_t base = su32(smem + s * STAGE);
            uint32_t bb = base + NACC * A_BYTES;
#pragma unroll
            for (int k = 0; k < KC / 16; k++) {
                uint32_t acc = (kc | k) != 0;
                mma(tmem, sdesc(base + k * 32), sdesc(bb + k * 32), id, acc);
                if (DUAL) mma(tmem + NT, sdesc(base + A_BYTES + k * 32), sdesc(bb + k * 32), id, acc);
            }
            mma_commit(&empty[s]);
        }
        mma_commit(&done);
    }
    __syncwarp();
    bool ok = mbar_wait(&done, 0);
    if (!ok) abort_flag = 1;
    fence_after();
    __syncthreads();
    if (abort_flag) {
        if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
    } else {
        const Epi &e = g.epi;
        const int f = f0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < NT; c0 += 16) {
            float v[16], v2[16];
            tmem_ld16(trow + c0, v);
            if (DUAL) tmem_ld16(trow + NT + c0, v2);
            if (f >= g.N) continue;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                int m = m0 + c0 + j;
                if (m >= g.M) break;
                int p = e.pos ? e.pos[m] : m;
                float y = v[j];
                switch (e.mode) {
                case EPI_STORE:
                    ((__nv_bfloat16 *)e.out)[(long)(e.scatter ? p : m) * e.ld_out + f] = __float2bfloat16_rn(y);
                    break;
                case EPI_QKV:
                    if (f < e.q_cols)
                        ((__nv_bfloat16 *)e.out)[(long)m * e.ld_out + f] = __float2bfloat16_rn(y);
                    else if (f < e.q_cols + e.d)
                        ((__nv_bfloat16 *)e.kc)[(long)p * e.d + (f - e.q_cols)] = __float2bfloat16_rn(y);
                    else
                        ((__nv_bfloat16 *)e.vc)[(long)p * e.d + (f - e.q_cols - e.d)] = __float2bfloat16_rn(y);
                    break;
                case EPI_RESID:
                    e.resid[(long)p * g.N + f] += y;
                    break;
                case EPI_RESID_BASE:
                    e.resid[(long)p * g.N + f] = e.base[(long)p * g.N + f] + y;
                    break;
                case EPI_SWIGLU:
                    if (DUAL) ((__nv_bfloat16 *)e.out)[(long)m * e.ld_out + f] = __float2bfloat16_rn(silu_f(y) * v2[j]);
                    break;
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_mu;
EncodeTiledFn g_encode = nullptr;
std::map<std::tuple<const void *, int, int, int>, CUtensorMap> g_maps;

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

// 2D row-major bf16 [rows][K] with a box of box_rows x 64, 128-byte swizzle.
bool tensor_map(const void *ptr, int rows, int K, int box_rows, CUtensorMap *out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_tuple(ptr, rows, K, box_rows);
    auto it = g_maps.find(key);
    if (it != g_maps.end()) { *out = it->second; return true; }
    EncodeTiledFn enc = encoder();
    if (!enc) return false;
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)K * 2};
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

}  // namespace

void gemm_simt(int prec, const GemmArgs &g, cudaStream_t s);

bool gemm_tc_supported(int prec, int N, int K)
{
    return prec == P_BF16 && N % TM == 0 && K % KC == 0 && K >= KC;
}

bool gemm_tc_available()
{
    std::lock_guard<std::mutex> lk(g_mu);
    return encoder() != nullptr;
}

bool gemm_tc(const GemmArgs &g, cudaStream_t s)
{
    int *status = g.status;
    CUtensorMap tw, tw2, tx;
    if (!tensor_map(g.Wt, g.N, g.K, TM, &tw)) return false;
    if (!tensor_map(g.A, g.M, g.K, NT, &tx)) return false;
    bool dual = g.epi.mode == EPI_SWIGLU;
    if (dual && !tensor_map(g.Wt2, g.N, g.K, TM, &tw2)) return false;
    if (!dual) tw2 = tw;
    dim3 grid(g.N / TM, (g.M + NT - 1) / NT);
    if (dual) {
        size_t smem = (size_t)STAGES * (2 * A_BYTES + B_BYTES) + 1024;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_gemm_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = true;
        }
        k_gemm_tc<true><<<grid, 128, smem, s>>>(tw, tw2, tx, g, status);
    } else {
        size_t smem = (size_t)STAGES * (A_BYTES + B_BYTES) + 1024;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_gemm_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = true;
        }
        k_gemm_tc<false><<<grid, 128, smem, s>>>(tw, tw2, tx, g, status);
    }
    return true;
}

}  // namespace psw
