// rans_dev.cuh -- device side of the interleaved rANS decoder shared by the
// coder kernels and the persistent decoder: container constants, byte
// readers, the lane scan, and one schedule step of one channel stream.
#pragma once

#include "internal.h"
#include "device_common.cuh"

namespace psw {

constexpr uint32_t MAGIC = 0x31575350u;    // 'PSW1'
constexpr uint32_t RANS_L = 1u << 16;      // lower bound of the coder state

__device__ __forceinline__ uint32_t lane_exclusive_scan(uint32_t v, uint32_t &total)
{
    int lane = threadIdx.x & 31;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    total = __shfl_sync(0xffffffffu, inc, 31);
    return inc - v;
}

__device__ __forceinline__ uint32_t ld8(const uint8_t *b, size_t o) { return b[o]; }
__device__ __forceinline__ uint32_t ld16le(const uint8_t *b, size_t o) { return ld8(b, o) | (ld8(b, o + 1) << 8); }
__device__ __forceinline__ uint32_t ld32le(const uint8_t *b, size_t o) { return ld16le(b, o) | (ld16le(b, o + 2) << 16); }

// Decode symbols k0 .. k0 + n - 1 of channel c of slot b (one schedule
// step; warp item wi = b * C + c, kn[b] = (k0, n)).  A group of 32 consecutive
// symbols decodes in parallel on its lanes, which then read their words in
// lane order (a warp scan of the words each lane needs).
template <bool PDL>
__device__ __forceinline__ void rans_step_item(const CoderDev &cd, const Slot *__restrict__ S,
                                               const int2 *__restrict__ kn, int C, int wi)
{
    int lane = threadIdx.x & 31;
    int b = wi / C, c = wi % C;
    int2 r = kn[b];
    int k0 = r.x, n = r.y;
    if (PDL) pdl_trigger();
    if (n <= 0) return;
    if (PDL) pdl_wait();                               // this step's scale indices and means are ready
    const Slot &sl = S[b];
    const uint8_t *__restrict__ bs = sl.bs;
    const int *__restrict__ order = sl.order;
    uint32_t x = sl.rstate[(size_t)c * 32 + lane];
    uint32_t p = sl.rptr[c];
    const uint32_t e = sl.rend[c];
    bool bad = false;
    for (int g = k0 / 32; g * 32 < k0 + n; g++) {
        int k = g * 32 + lane;
        bool act = k >= k0 && k < k0 + n;
        uint32_t need = 0;
        long pos = 0;
        int T = 0, slot = 0;
        int32_t mm = 0;
        if (act) {
            pos = order[k];
            long a = pos * C + c;
            int l = sl.idx[a];
            mm = sl.m[a];
            T = cd.meta[l];
            int nsl = cd.meta[cd.nt + l], off = cd.meta[2 * cd.nt + l];
            uint32_t v = x & 0xFFFFu;
            int lo = 0, hi = nsl - 1;                  // last slot with cum <= v
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if ((cd.cdf[off + mid] & 0xFFFFu) <= v) lo = mid; else hi = mid - 1;
            }
            slot = lo;
            uint32_t ent = cd.cdf[off + slot];
            x = (ent >> 16) * (x >> 16) + v - (ent & 0xFFFFu);
            need = (x < RANS_L ? 1u : 0u) + (slot == 2 * T + 1 ? 2u : 0u);
        }
        uint32_t total;
        uint32_t pre = lane_exclusive_scan(need, total);
        uint32_t q = p + 2 * pre;
        auto word = [&](void) -> uint32_t {
            if (q + 2 > e) { bad = true; return 0u; }
            uint32_t wv = ld16le(bs, q);
            q += 2;
            return wv;
        };
        if (act) {
            if (x < RANS_L) x = (x << 16) | word();
            long sv;
            if (slot == 2 * T + 1) {
                uint32_t d0 = x & 0xFFFFu;
                x = (x & 0xFFFF0000u) | word();
                uint32_t d1 = x & 0xFFFFu;
                x = (x & 0xFFFF0000u) | word();
                uint32_t v = d0 | (d1 << 16);
                long mag = (long)T + 1 + (long)(v >> 1);
                sv = (v & 1) ? -mag : mag;
            } else {
                sv = slot - T;
            }
            long yv = (long)mm + sv;
            if (yv < -32768 || yv > 32767) { bad = true; yv = 0; }
            sl.y[pos * C + c] = (int16_t)yv;
        }
        p += 2 * total;
        if (p > e) p = e;
    }
    sl.rstate[(size_t)c * 32 + lane] = x;
    if (lane == 0) sl.rptr[c] = p;
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(sl.status, ST_CORRUPT);
}

}  // namespace psw
