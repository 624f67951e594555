// device_common.cuh -- small device helpers shared by the kernels and both
// GEMMs (type conversion, warp reductions, SiLU, the GEMM epilogues).
#pragma once

#include "internal.h"

namespace psw {

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
// SiLU with the fast exponential and division intrinsics (a few ulp; the
// tensor-core epilogues, where the accurate forms dominated the epilogue's
// instruction count).  For x far below zero the denominator overflows to
// infinity and the quotient is 0, as SiLU's limit.
__device__ __forceinline__ float silu_fast(float x) { return __fdividef(x, 1.0f + __expf(-x)); }

// Programmatic dependent launch: let the next kernel in the stream start its
// prologue now; wait until the previous kernel's results are visible.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ln 0.11 and ln 256: sigma's range (the scale table's end points).
constexpr float LN_SIG_LO = -2.2072749131897207f, LN_SIG_HI = 5.545177444479562f;

// Writes GEMM output (m, n) = y (and, for the dual SwiGLU form, the
// up-projection y2) as the epilogue says.  EPI_HEADS is handled per channel
// pair by heads_pair.
template <typename T>
__device__ __forceinline__ void epilogue_store(const Epi &e, int N, int m, int n, float y, float y2)
{
    switch (e.mode) {
    case EPI_STORE:
        if (e.st_sel == CS_NONE) {
            ((T *)e.out)[(long)m * e.ld_out + n] = from_f<T>(y);
        } else {
            int tk = e.tok[m];
            cache_row<T>(e.slots[tok_slot(tk)], e.st_sel, e.st_layer, tok_pos(tk), e.d)[n] = from_f<T>(y);
        }
        break;
    case EPI_QKV:
        if (n < e.q_cols) {
            ((T *)e.out)[(long)m * e.ld_out + n] = from_f<T>(y);
        } else {
            int tk = e.tok[m];
            const Slot &s = e.slots[tok_slot(tk)];
            int nn = n - e.q_cols;
            int layer = e.ring ? e.kv_layer * e.Tf + s.ring[s.nfr - 1] : e.kv_layer;
            if (nn < e.d) cache_row<T>(s, e.kc_sel, layer, tok_pos(tk), e.d)[nn] = from_f<T>(y);
            else cache_row<T>(s, e.vc_sel, layer, tok_pos(tk), e.d)[nn - e.d] = from_f<T>(y);
        }
        break;
    case EPI_RESID:
        e.rows[(long)m * N + n] += y;
        break;
    case EPI_RESID_BASE: {
        int tk = e.tok[m];
        const Slot &s = e.slots[tok_slot(tk)];
        e.rows[(long)m * N + n] = s.eh[(long)tok_pos(tk) * N + n] + y;
        break;
    }
    case EPI_SWIGLU:
        ((T *)e.out)[(long)m * e.ld_out + n] = from_f<T>(silu_f(y) * y2);
        break;
    case EPI_BIAS_SILU:
        ((T *)e.out)[(long)m * e.ld_out + n] = from_f<T>(silu_f(y + e.bias[n]));
        break;
    case EPI_SET_BIAS:
        e.rows[(long)m * N + n] = y + e.bias[n];
        break;
    default:
        break;
    }
}

// Scale index of sigma: the smallest l with scale[l] >= sigma (float
// compare), 63 if there is none (or sigma is NaN).  The table increases
// strictly, so a binary search gives the index a linear scan would.
__device__ __forceinline__ int scale_index(const float *scale, float sg)
{
    int lo = 0, n = NSCALES;
#pragma unroll
    for (int it = 0; it < 6; it++) {
        int half = n >> 1;
        if (!(scale[lo + half - 1] >= sg)) lo += half;
        n -= half;
    }
    // lo: first index whose entry is >= sg among 0..63, or 63 (the search
    // never moves past the last entry)
    return lo;
}

// Prediction heads' output for channel c = n / 2 of a token (rows 2c and
// 2c+1 of the interleaved second layer): channel-wise scaling of mu, sigma =
// exp of the clamped scaled value, then the scale index (smallest table
// entry not below sigma, float compare) and the rounded mean.
__device__ __forceinline__ void heads_pair(const Epi &e, const float *scale, int m, int n, float ymu, float ysg)
{
    int tk = e.tok[m];
    const Slot &s = e.slots[tok_slot(tk)];
    long o = (long)tok_pos(tk) * e.C + e.c0 + (n >> 1);
    int c = n >> 1;
    float mu = e.gmu[c] * ymu + e.bmu[c];
    float sg = expf(fminf(fmaxf(e.gsg[c] * ysg + e.bsg[c], LN_SIG_LO), LN_SIG_HI));
    s.mu[o] = mu;
    s.sigma[o] = sg;
    s.idx[o] = (uint8_t)scale_index(scale, sg);
    s.m[o] = (int32_t)rintf(fminf(fmaxf(mu, -32768.0f), 32767.0f));
}

}  // namespace psw
