// persist.cu -- the persistent wavefront decoder: one cooperative launch,
// one CTA per SM, walks every global step of a batched decode.
//
// A step is a fixed program of phases (Sec. 3.1 / Fig. 1 model on the step's
// positions, then the rANS step): Spatial Module 1 and the accumulator
// keys/values on the positions decoded at the previous step, the
// accumulator, Spatial Module 2 and the heads on the positions of this step,
// then the coder.  Phases depend on one another through global memory, so a
// grid-wide barrier separates them; within a phase the CTAs share its tiles
// (projections: 128 features x 64 tokens) or warp items ((token, head) of an
// attention, (frame, channel) of the coder) round-robin, starting at a CTA
// that rotates from phase to phase, so that a small phase runs on CTAs the
// previous one left idle.
//
// Each phase runs the same tile and item functions as the one-launch-per-op
// kernels (gemm_dev.cuh, attn_dev.cuh, rans_dev.cuh), so the decoder's
// parameters are bit-identical to the encoder's masked pass.  What the
// persistent form adds: no launch or drain between phases, and the next
// phase's token table and first weight copies are issued early (they do not
// depend on the phase in flight): by CTAs idle in the current phase at its
// start, by the others before they wait at the barrier.
//
// Every wait is bounded: mbarrier waits as in the GEMM engine, the grid
// barrier after ~2 s of globaltimer or once another CTA has raised the
// global abort flag.  A CTA that gives up records ST_TIMEOUT, raises the
// flag, frees its tensor memory and returns; the others leave at their next
// barrier.  Co-residency of all CTAs (which the barrier relies on) is
// guaranteed by the cooperative launch.
#include "gemm_dev.cuh"
#include "attn_dev.cuh"
#include "attn_tok.cuh"
#include "rans_dev.cuh"

#include <map>
#include <tuple>
#include <vector>

namespace psw {

using namespace tc;

namespace {

constexpr int PWARPS = NTHREADS / 32;
constexpr uint32_t PTCOLS = tile_tcols(true);      // tensor-memory columns: the dual form's accumulators
#ifndef PSW_SPIN_NS
#define PSW_SPIN_NS 200
#endif
constexpr unsigned SPIN_NS = PSW_SPIN_NS;          // pause between polls of the grid barrier

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier on a monotone counter: every CTA adds one per barrier and
// waits until the counter reaches (barriers so far) x (CTAs).  Thread 0 only.
// Polls back off (a short sleep between reads) so that idle CTAs do not
// flood the counter's L2 slice while others work.
__device__ __forceinline__ bool grid_wait(const unsigned *bar, unsigned target, const volatile int *abort_g,
                                          uint64_t limit_ns = WAIT_NS)
{
    if (ld_acquire(bar) >= target) return true;
    uint64_t t0 = gtime();
    for (;;) {
        __nanosleep(SPIN_NS);
        if (ld_acquire(bar) >= target) return true;
        if (*abort_g) return false;
        if (gtime() - t0 > limit_ns) return false;
    }
}

// Failure-detection check: one thread runs the grid barrier's bounded wait
// for an arrival count that nothing will reach, with the given limit, and
// reports the expiry into the status word as the decoder does.
__global__ void k_wait_probe(const unsigned *bar, const int *abort_g, uint64_t limit_ns, int *status)
{
    if (threadIdx.x == 0 && !grid_wait(bar, 1u, abort_g, limit_ns)) atomicOr(status, ST_TIMEOUT);
}

// The tokens of the step a phase works on.
__device__ __forceinline__ bool phase_valid(const PersistArgs &P, int t, int i)
{
    int ts = P.ops[i].tokset;
    if (ts == TS_PREV && t == 0) return false;
    return P.step_n[ts == TS_PREV ? t - 1 : t] > 0;
}

// Advance (t, i) to the next phase with work; false past the last step.
__device__ __forceinline__ bool next_phase(const PersistArgs &P, int &t, int &i)
{
    for (;;) {
        if (++i == P.nops) { i = 0; t++; }
        if (t >= P.t1) return false;
        if (phase_valid(P, t, i)) return true;
    }
}

// Copy phase (t, i) into shared memory and fill in its step's tokens.
__device__ __forceinline__ void load_op(const PersistArgs &P, Op &op, int t, int i)
{
    const int *src = reinterpret_cast<const int *>(P.ops + i);
    int *dst = reinterpret_cast<int *>(&op);
    for (int w = threadIdx.x; w < (int)(sizeof(Op) / 4); w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    if (threadIdx.x == 0) {
        int tt = op.tokset == TS_PREV ? t - 1 : t;
        const int *tok = P.tok + P.step_off[tt];
        int n = P.step_n[tt];
        op.g.M = n; op.g.epi.tok = tok;
        op.a.tok = tok; op.a.n = n;
        op.kn = P.kn + (size_t)t * P.nslots;
    }
    __syncthreads();
}

__device__ __forceinline__ int gemm_tiles(const GemmArgs &g, int &nf)
{
    nf = (g.N + TM - 1) / TM;
    return nf * ((g.M + NT - 1) / NT);
}

template <bool DUAL, int MODE, bool F8 = false>
__device__ __forceinline__ int pre_t(GemmShared &S, uint8_t *ring, const CUtensorMap *maps, const Op &op, int j,
                                     GemmPipe &pp)
{
    int nf;
    gemm_tiles(op.g, nf);
    return gemm_tile_pre<DUAL, MODE, F8>(S, ring, maps + op.wmap, maps + (op.wmap2 >= 0 ? op.wmap2 : op.wmap), op.g,
                                         (j % nf) * TM, (j / nf) * NT, pp);
}

// gemm_tile_pre of tile j of a projection phase.  F8: the program has E4M3
// projections (the five epilogues of block projections).
template <bool F8>
__device__ __noinline__ int gemm_pre(GemmShared &S, uint8_t *ring, const CUtensorMap *maps, const Op &op, int j,
                                     GemmPipe &pp)
{
    if constexpr (F8) {
        if (op.g.f8) {
            switch (op.g.epi.mode) {
            case EPI_SWIGLU: return pre_t<true, EPI_SWIGLU, true>(S, ring, maps, op, j, pp);
            case EPI_STORE: return pre_t<false, EPI_STORE, true>(S, ring, maps, op, j, pp);
            case EPI_QKV: return pre_t<false, EPI_QKV, true>(S, ring, maps, op, j, pp);
            case EPI_RESID: return pre_t<false, EPI_RESID, true>(S, ring, maps, op, j, pp);
            default: return pre_t<false, EPI_RESID_BASE, true>(S, ring, maps, op, j, pp);
            }
        }
    }
    switch (op.g.epi.mode) {
    case EPI_SWIGLU: return pre_t<true, EPI_SWIGLU>(S, ring, maps, op, j, pp);
    case EPI_STORE: return pre_t<false, EPI_STORE>(S, ring, maps, op, j, pp);
    case EPI_QKV: return pre_t<false, EPI_QKV>(S, ring, maps, op, j, pp);
    case EPI_RESID: return pre_t<false, EPI_RESID>(S, ring, maps, op, j, pp);
    case EPI_RESID_BASE: return pre_t<false, EPI_RESID_BASE>(S, ring, maps, op, j, pp);
    case EPI_BIAS_SILU: return pre_t<false, EPI_BIAS_SILU>(S, ring, maps, op, j, pp);
    case EPI_SET_BIAS: return pre_t<false, EPI_SET_BIAS>(S, ring, maps, op, j, pp);
    default: return pre_t<false, EPI_HEADS>(S, ring, maps, op, j, pp);
    }
}

// This CTA's tiles of a projection phase (tiles rank, rank + grid, ...); the
// first may have been prepared (gemm_pre) before the barrier.
template <bool DUAL, int MODE, bool F8 = false>
__device__ __noinline__ void gemm_phase(GemmShared &S, uint8_t *ring, uint32_t tmem, const CUtensorMap *maps,
                                        const Op &op, int rank, bool prepared, int first, GemmPipe &pp)
{
    int nf;
    const int ntiles = gemm_tiles(op.g, nf);
    const CUtensorMap *tw = maps + op.wmap, *tw2 = maps + (op.wmap2 >= 0 ? op.wmap2 : op.wmap);
    const CUtensorMap *tx = maps + (op.xmap >= 0 ? op.xmap : op.wmap);
    for (int j = rank; j < ntiles; j += gridDim.x) {
        const int f0 = (j % nf) * TM, m0 = (j / nf) * NT;
        if (!(prepared && j == rank)) {
            first = gemm_tile_pre<DUAL, MODE, F8>(S, ring, tw, tw2, op.g, f0, m0, pp);
            __syncthreads();
        }
        gemm_tile_main<DUAL, MODE, F8>(S, ring, tmem, tw, tw2, tx, op.g, f0, m0, first, pp);
        if (S.abort) return;
    }
}

template <bool F8>
__device__ __noinline__ void run_gemm(GemmShared &S, uint8_t *ring, uint32_t tmem, const CUtensorMap *maps,
                                      const Op &op, int rank, bool prepared, int first, GemmPipe &pp)
{
    if constexpr (F8) {
        if (op.g.f8) {
            switch (op.g.epi.mode) {
            case EPI_SWIGLU: gemm_phase<true, EPI_SWIGLU, true>(S, ring, tmem, maps, op, rank, prepared, first, pp); return;
            case EPI_STORE: gemm_phase<false, EPI_STORE, true>(S, ring, tmem, maps, op, rank, prepared, first, pp); return;
            case EPI_QKV: gemm_phase<false, EPI_QKV, true>(S, ring, tmem, maps, op, rank, prepared, first, pp); return;
            case EPI_RESID: gemm_phase<false, EPI_RESID, true>(S, ring, tmem, maps, op, rank, prepared, first, pp); return;
            default:
                gemm_phase<false, EPI_RESID_BASE, true>(S, ring, tmem, maps, op, rank, prepared, first, pp);
                return;
            }
        }
    }
    switch (op.g.epi.mode) {
    case EPI_SWIGLU: gemm_phase<true, EPI_SWIGLU>(S, ring, tmem, maps, op, rank, prepared, first, pp); break;
    case EPI_STORE: gemm_phase<false, EPI_STORE>(S, ring, tmem, maps, op, rank, prepared, first, pp); break;
    case EPI_QKV: gemm_phase<false, EPI_QKV>(S, ring, tmem, maps, op, rank, prepared, first, pp); break;
    case EPI_RESID: gemm_phase<false, EPI_RESID>(S, ring, tmem, maps, op, rank, prepared, first, pp); break;
    case EPI_RESID_BASE:
        gemm_phase<false, EPI_RESID_BASE>(S, ring, tmem, maps, op, rank, prepared, first, pp);
        break;
    case EPI_BIAS_SILU: gemm_phase<false, EPI_BIAS_SILU>(S, ring, tmem, maps, op, rank, prepared, first, pp); break;
    case EPI_SET_BIAS: gemm_phase<false, EPI_SET_BIAS>(S, ring, tmem, maps, op, rank, prepared, first, pp); break;
    default: gemm_phase<false, EPI_HEADS>(S, ring, tmem, maps, op, rank, prepared, first, pp); break;
    }
}

// 64-wide heads: one warp per token and head group (attn_tok.cuh), the
// same function as the attention kernel's.
__device__ __noinline__ void attn_tok_phase(const AttnArgs &a, uint8_t *dyn, int rank)
{
    const int warp = threadIdx.x >> 5, items = a.n * (a.nh / TK_HG);
    unsigned char *sm = dyn + (size_t)warp * attn_tok_bytes();
    for (int gw = rank * PWARPS + warp; gw < items; gw += gridDim.x * PWARPS) attn_token<false>(a, gw, sm);
}

template <int DH>
__device__ __noinline__ void attn_phase(const AttnArgs &a, uint8_t *dyn, int rank)
{
    AttnWarp<__nv_bfloat16, DH> *sm = reinterpret_cast<AttnWarp<__nv_bfloat16, DH> *>(dyn);
    const int warp = threadIdx.x >> 5, items = a.n * a.nh;
    for (int gw = rank * PWARPS + warp; gw < items; gw += gridDim.x * PWARPS)
        attn_item<__nv_bfloat16, DH, false>(a, gw, sm[warp]);
}

__device__ __noinline__ void rans_phase(const PersistArgs &P, const int2 *kn, int rank)
{
    const int warp = threadIdx.x >> 5, items = P.nslots * P.C;
    for (int wi = rank * PWARPS + warp; wi < items; wi += gridDim.x * PWARPS)
        rans_step_item<false>(P.cd, P.slots, kn, P.C, wi);
}

// Work units of a phase: projection tiles, or CTAs' worth of warp items.
__device__ __forceinline__ int phase_units(const PersistArgs &P, const Op &op)
{
    if (op.type == OP_GEMM) {
        int nf;
        return gemm_tiles(op.g, nf);
    }
    int items = op.type == OP_ATTN ? (attn_tok_ok(P_BF16, op.a.d, op.a.nh, op.a.mask, op.a.kind) ? op.a.n * (op.a.nh / TK_HG) : op.a.n * op.a.nh)
                                   : P.nslots * P.C;
    return (items + PWARPS - 1) / PWARPS;
}

template <bool F8>
__global__ void __launch_bounds__(NTHREADS, 1) k_persist(const __grid_constant__ PersistArgs P)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ GemmShared S;
    __shared__ Op ops[2];                              // this phase and the next
    __shared__ int stop;
    uint8_t *dyn = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const CUtensorMap *maps = (const CUtensorMap *)P.maps;
    const int warp = threadIdx.x >> 5;
    const int G = gridDim.x;
    if (threadIdx.x == 0) { gemm_shared_init(S); stop = 0; }
    // the tensor maps sit in global memory (written before the launch): make
    // them visible to the tensor-map proxy of the threads that issue copies
    if ((threadIdx.x & 31) == 0)
        for (int m = 0; m < P.nmaps; m++)
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(maps + m) : "memory");
    if (warp == 0) tmem_alloc(&S.tmem_slot, PTCOLS);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_slot;
    GemmPipe pp;
    uint32_t nbar = 0;
    int t = P.t0, i = -1, first = 0, cur = 0;
    int base = 0;                                      // CTA where this phase's work starts (rotates)
    bool prepared = false;
    bool have = next_phase(P, t, i);
    if (have) load_op(P, ops[cur], t, i);
    while (have) {
        Op &op = ops[cur];
        Op &nop = ops[cur ^ 1];
        const int units = phase_units(P, op);
        const int rank = (int)((blockIdx.x - base + G) % G);
        const bool busy = rank < units;
        // the next phase: its record, and this CTA's rank in it
        int nt = t, ni = i;
        const bool more = next_phase(P, nt, ni);
        const int nbase = (base + (units < G ? units : G)) % G;
        const int nrank = (int)((blockIdx.x - nbase + G) % G);
        if (more) load_op(P, nop, nt, ni);
        bool nprep = false;
        if (!busy && more && nop.type == OP_GEMM) {
            // idle in this phase: prepare the next phase's first tile now
            int nf;
            if (nrank < gemm_tiles(nop.g, nf)) {
                first = gemm_pre<F8>(S, dyn, maps, nop, nrank, pp);
                nprep = true;
            }
        }
        if (busy) {
            if (op.type == OP_GEMM) run_gemm<F8>(S, dyn, tmem, maps, op, rank, prepared, first, pp);
            else if (op.type == OP_ATTN) {
                const int dh = op.a.d / op.a.nh;
                if (attn_tok_ok(P_BF16, op.a.d, op.a.nh, op.a.mask, op.a.kind)) attn_tok_phase(op.a, dyn, rank);
                else if (dh == 64) attn_phase<64>(op.a, dyn, rank);
                else if (dh == 32) attn_phase<32>(op.a, dyn, rank);
                else attn_phase<128>(op.a, dyn, rank);
            } else {
                rans_phase(P, op.kn, rank);
            }
        }
        // shared staging is free for the next phase's tensor copies; the
        // threads that issue them order their acquire of this phase's global
        // writes before the copies (fence_proxy_global in gemm_tile_main)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (S.abort || !more) break;
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(P.bar, 1u);
        }
        nbar++;
        if (busy && nop.type == OP_GEMM) {
            int nf;
            if (nrank < gemm_tiles(nop.g, nf)) {
                first = gemm_pre<F8>(S, dyn, maps, nop, nrank, pp);
                nprep = true;
            }
        }
        if (threadIdx.x == 0 && !grid_wait(P.bar, nbar * G, P.abort_g)) stop = 1;
        __syncthreads();
        if (stop || S.abort) break;
        t = nt; i = ni; cur ^= 1; base = nbase; prepared = nprep;
    }
    if (threadIdx.x == 0 && (S.abort || stop)) {
        atomicOr(P.status, ST_TIMEOUT);
        atomicExch(P.abort_g, 1);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, PTCOLS);
}

}  // namespace

// ---------------------------------------------------------------- host side

struct ProgramBuilder {
    int ws_rows;
    std::vector<Op> ops;
    std::vector<CUtensorMap> maps;
    std::map<std::tuple<const void *, int, int, int, int, bool>, int> map_idx;
    size_t smem = 0;
    bool f8 = false;                   // some projection is E4M3
    Op *d_ops = nullptr;
    CUtensorMap *d_maps = nullptr;
};

static int map_of(ProgramBuilder *b, const void *ptr, int rows, int K, int ld, int box, bool f8 = false)
{
    auto key = std::make_tuple(ptr, rows, K, ld, box, f8);
    auto it = b->map_idx.find(key);
    if (it != b->map_idx.end()) return it->second;
    CUtensorMap m;
    if (!gemm_tensor_map(ptr, rows, K, ld, box, &m, f8)) return -1;
    b->maps.push_back(m);
    return b->map_idx[key] = (int)b->maps.size() - 1;
}

ProgramBuilder *program_new(int ws_rows)
{
    ProgramBuilder *b = new ProgramBuilder();
    b->ws_rows = ws_rows;
    return b;
}

void program_free(ProgramBuilder *b)
{
    if (!b) return;
    cudaFree(b->d_ops);
    cudaFree(b->d_maps);
    delete b;
}

bool program_gemm(ProgramBuilder *b, const GemmArgs &g, int tokset)
{
    const bool f8 = g.f8 != 0;
    if (f8 ? !gemm_tc8_supported(g.N, g.K, g.asrc) : !gemm_tc_supported(P_BF16, g.N, g.K, g.asrc)) return false;
    Op op{};
    op.type = OP_GEMM; op.tokset = tokset;
    op.dual = g.epi.mode == EPI_SWIGLU;
    op.g = g;
    op.wmap = map_of(b, g.Wt, g.N, g.K, g.K, TM, f8);
    op.wmap2 = op.dual ? map_of(b, g.Wt2, g.N, g.K, g.K, TM, f8) : -1;
    // activation rows: the whole workspace; rows past a step's tokens only
    // feed accumulator columns that are never stored (E4M3 projections
    // build their token operand)
    const bool streamed = !f8 && g.asrc == A_DIRECT;
    op.xmap = streamed ? map_of(b, g.A, b->ws_rows, g.K, g.lda, NT) : -1;
    if (op.wmap < 0 || (op.dual && op.wmap2 < 0) || (streamed && op.xmap < 0)) return false;
    b->ops.push_back(op);
    b->smem = std::max(b->smem, (size_t)tile_smem(op.dual, !streamed, g.K, f8));
    b->f8 = b->f8 || f8;
    return true;
}

void program_attn(ProgramBuilder *b, const AttnArgs &a, int tokset)
{
    Op op{};
    op.type = OP_ATTN; op.tokset = tokset;
    op.wmap = op.wmap2 = op.xmap = -1;
    op.a = a;
    b->ops.push_back(op);
    int dh = a.d / a.nh;
    size_t per = attn_tok_ok(P_BF16, a.d, a.nh, a.mask, a.kind) ? attn_tok_bytes()
                 : dh == 32 ? sizeof(AttnWarp<__nv_bfloat16, 32>)
                 : dh == 64 ? sizeof(AttnWarp<__nv_bfloat16, 64>) : sizeof(AttnWarp<__nv_bfloat16, 128>);
    b->smem = std::max(b->smem, per * PWARPS);
}

void program_rans(ProgramBuilder *b)
{
    Op op{};
    op.type = OP_RANS; op.tokset = TS_CUR;
    op.wmap = op.wmap2 = op.xmap = -1;
    b->ops.push_back(op);
}

bool program_upload(ProgramBuilder *b, const Op **ops, int *nops, const void **maps, int *nmaps, size_t *smem,
                    bool *f8)
{
    if (!b->d_ops) {
        if (cudaMalloc(&b->d_ops, b->ops.size() * sizeof(Op)) != cudaSuccess) return false;
        if (cudaMalloc(&b->d_maps, std::max<size_t>(b->maps.size(), 1) * sizeof(CUtensorMap)) != cudaSuccess)
            return false;
        if (cudaMemcpy(b->d_ops, b->ops.data(), b->ops.size() * sizeof(Op), cudaMemcpyHostToDevice) != cudaSuccess)
            return false;
        if (!b->maps.empty() &&
            cudaMemcpy(b->d_maps, b->maps.data(), b->maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice) !=
                cudaSuccess)
            return false;
    }
    *ops = b->d_ops;
    *nops = (int)b->ops.size();
    *maps = b->d_maps;
    *nmaps = (int)b->maps.size();
    *smem = b->smem + 1024;
    *f8 = b->f8;
    return true;
}

bool persist_prepare(size_t smem, bool f8, int *grid)
{
    auto kern = f8 ? k_persist<true> : k_persist<false>;
    int dev = 0, nsm = 0, coop = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return false;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return false;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NTHREADS, smem) != cudaSuccess || per < 1)
        return false;
    *grid = nsm;
    return true;
}

bool wait_probe(uint64_t limit_ns, int *status, cudaStream_t s)
{
    unsigned *words = nullptr;                         // [0]: barrier counter, [1]: abort flag, both zero
    if (cudaMalloc(&words, 2 * sizeof(unsigned)) != cudaSuccess) return false;
    bool ok = cudaMemsetAsync(words, 0, 2 * sizeof(unsigned), s) == cudaSuccess;
    if (ok) {
        k_wait_probe<<<1, 32, 0, s>>>(words, (const int *)(words + 1), limit_ns, status);
        ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
    }
    cudaFree(words);
    return ok;
}

bool persist_launch(const PersistArgs &a, int grid, size_t smem, bool f8, cudaStream_t s)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, f8 ? k_persist<true> : k_persist<false>, a) == cudaSuccess;
}

}  // namespace psw
