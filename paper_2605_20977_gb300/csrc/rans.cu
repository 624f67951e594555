// rans.cu -- scale table, integer CDF tables and 32-lane interleaved rANS.
//
// The paper draws quantisation and arithmetic coding as "Q", "AE" and "AD"
// (Fig. 1) and names no coder.  This file realises them:
//   * scale table: 64 scales log-spaced from 0.11 to 256 (float);
//   * CDF table per scale: zero-mean quantised Gaussian over -T..T plus an
//     escape slot, T = max(1, ceil(7 sigma)); pmf from erfc; 16-bit
//     frequencies, each at least 1, summing to 2^16;
//   * rANS (32-bit state in [2^16, 2^32), 16-bit renormalisation words,
//     M = 2^16), one stream per channel, symbol k of a stream on lane
//     k mod 32; an escape codes v = 2 (|s| - T - 1) + sign as two raw 16-bit
//     digits on the same lane.
// Container (little endian): u32 magic 'PSW1', u16 version 1, u16 schedule,
// u16 H, u16 W, u16 C, u16 0, u32 offsets[C + 1]; each stream is u32 state[32]
// followed by its words in decoding order, padded to 4 bytes.
#include "internal.h"
#include "device_common.cuh"
#include "rans_dev.cuh"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

namespace psw {


// ---------------------------------------------------------------- tables (host)

void build_scale_table(float *tab)
{
    const double a = log(0.11), b = log(256.0);
    for (int l = 0; l < NSCALES; l++) tab[l] = (float)exp(a + l * (b - a) / (NSCALES - 1));
}

void build_cdf_tables(CdfTables &t)
{
    build_scale_table(t.scale);
    int total = 0;
    for (int l = 0; l < NSCALES; l++) {
        int T = (int)ceil(7.0 * (double)t.scale[l]);
        if (T < 1) T = 1;
        t.T[l] = T;
        t.n[l] = 2 * T + 2;
        t.off[l] = total;
        total += t.n[l];
    }
    t.total = total;
    t.packed = (uint32_t *)malloc(sizeof(uint32_t) * total);
    uint32_t *fr = (uint32_t *)malloc(sizeof(uint32_t) * 4096);
    for (int l = 0; l < NSCALES; l++) {
        const double sg = (double)t.scale[l], den = sg * 1.4142135623730951;
        const int T = t.T[l], n = t.n[l];
        const double room = (double)((1u << CDF_PREC) - (uint32_t)n);
        long sum = 0;
        for (int sl = 0; sl <= 2 * T; sl++) {
            int s = sl - T;
            double u = (double)(s < 0 ? -s : s);
            double pmf = 0.5 * (erfc((u - 0.5) / den) - erfc((u + 0.5) / den));
            fr[sl] = 1u + (uint32_t)floor(pmf * room);
            sum += fr[sl];
        }
        double tail = erfc(((double)T + 0.5) / den);
        fr[2 * T + 1] = 1u + (uint32_t)floor(tail * room);
        sum += fr[2 * T + 1];
        fr[T] = (uint32_t)((long)fr[T] + ((long)(1u << CDF_PREC) - sum));
        uint32_t cum = 0;
        for (int sl = 0; sl < n; sl++) {
            t.packed[t.off[l] + sl] = cum | (fr[sl] << 16);
            cum += fr[sl];
        }
    }
    free(fr);
}

void free_cdf_tables(CdfTables &t)
{
    free(t.packed);
    t.packed = nullptr;
}

size_t container_capacity(int H, int W, int C)
{
    size_t HW = (size_t)H * W;
    return 16 + 4 * (size_t)(C + 1) + (size_t)C * (128 + 6 * HW + 4);
}

// ---------------------------------------------------------------- device helpers

// ---------------------------------------------------------------- encoder

// One warp per channel stream.  Groups of 32 symbols are encoded from the
// last to the first; in a group lane j holds symbol 32 g + j.  Each lane
// produces its renormalisation words in decoding order ([main], [d0, d1]);
// a warp scan places the group's words, in lane order, just before the
// words already written (the scratch region is filled from its end).
__global__ void k_rans_encode(CoderDev cd, const Slot *__restrict__ S, int slot, int HW, int C,
                              uint16_t *__restrict__ scratch, int cap_words, uint32_t *__restrict__ nwords,
                              uint32_t *__restrict__ states)
{
    int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (c >= C) return;
    const Slot &sl = S[slot];
    const int *__restrict__ order = sl.order;
    const int16_t *__restrict__ y = sl.y;
    const uint8_t *__restrict__ idx = sl.idx;
    const int32_t *__restrict__ m = sl.m;
    uint16_t *buf = scratch + (size_t)c * cap_words;
    uint32_t x = RANS_L;
    int wpos = cap_words;
    int ngroups = (HW + 31) / 32;
    for (int g = ngroups - 1; g >= 0; g--) {
        int k = g * 32 + lane;
        uint32_t cnt = 0, w[3] = {0, 0, 0};
        if (k < HW) {
            long a = (long)order[k] * C + c;
            int l = idx[a], T = cd.meta[l], off = cd.meta[2 * cd.nt + l];
            long sv = (long)y[a] - (long)m[a];
            int slot_ = 0;
            bool esc = false;
            uint32_t e0 = 0, e1 = 0;
            if (sv >= -T && sv <= T) {
                slot_ = (int)(sv + T);
            } else {
                slot_ = 2 * T + 1;
                esc = true;
                long mag = sv < 0 ? -sv : sv;
                uint32_t v = (uint32_t)(2 * (mag - T - 1) + (sv < 0 ? 1 : 0));
                uint32_t d0 = v & 0xFFFFu, d1 = v >> 16;
                e1 = x & 0xFFFFu; x = (x & 0xFFFF0000u) | d1;     // d1 encoded first
                e0 = x & 0xFFFFu; x = (x & 0xFFFF0000u) | d0;
            }
            uint32_t ent = cd.cdf[off + slot_];
            uint32_t cm = ent & 0xFFFFu, f = ent >> 16;
            bool ren = x >= (f << 16);
            uint32_t em = x & 0xFFFFu;
            if (ren) x >>= 16;
            x = ((x / f) << 16) + (x % f) + cm;
            if (ren) w[cnt++] = em;
            if (esc) { w[cnt++] = e0; w[cnt++] = e1; }
        }
        uint32_t total;
        uint32_t pre = lane_exclusive_scan(cnt, total);
        int base = wpos - (int)total;
        for (uint32_t j = 0; j < cnt; j++) buf[base + pre + j] = (uint16_t)w[j];
        wpos = base;
    }
    states[(size_t)c * 32 + lane] = x;
    if (lane == 0) nwords[c] = (uint32_t)(cap_words - wpos);
}

void launch_rans_encode(const CoderDev &cd, const Slot *S, int slot, int HW, int C, uint16_t *scratch,
                        int cap_words, uint32_t *nwords, uint32_t *states, cudaStream_t s)
{
    int blocks = (C * 32 + 127) / 128;
    k_rans_encode<<<blocks, 128, 0, s>>>(cd, S, slot, HW, C, scratch, cap_words, nwords, states);
}

// Offsets by a single-block scan over the streams, then the header; the
// total goes to *total.  If it exceeds cap nothing is written and the
// capacity bit is set.
__global__ void k_rans_offsets(int H, int W, int C, int sched, const uint32_t *__restrict__ nwords,
                               uint8_t *__restrict__ out, size_t cap, uint32_t *__restrict__ offs,
                               uint64_t *__restrict__ total, int *__restrict__ status)
{
    __shared__ uint64_t part[1024];
    int per = (C + blockDim.x - 1) / blockDim.x;
    uint64_t acc = 0;
    for (int u = 0; u < per; u++) {
        int c = threadIdx.x * per + u;
        if (c < C) { uint32_t nw = nwords[c]; acc += 128 + 2ull * nw + ((nw & 1) ? 2 : 0); }
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t run = 16 + 4ull * (C + 1);
        for (int t = 0; t < (int)blockDim.x; t++) { uint64_t v = part[t]; part[t] = run; run += v; }
        *total = run;
        if (run > cap || run > 0xFFFFFFFFull) atomicOr(status, ST_CAPACITY);
    }
    __syncthreads();
    uint64_t run = part[threadIdx.x];
    for (int u = 0; u < per; u++) {
        int c = threadIdx.x * per + u;
        if (c < C) {
            offs[c] = (uint32_t)run;
            uint32_t nw = nwords[c];
            run += 128 + 2ull * nw + ((nw & 1) ? 2 : 0);
        }
    }
    if (threadIdx.x == 0) offs[C] = (uint32_t)*total;
}

__global__ void k_rans_write(int H, int W, int C, int sched, const uint16_t *__restrict__ scratch,
                             int cap_words, const uint32_t *__restrict__ nwords,
                             const uint32_t *__restrict__ states, const uint32_t *__restrict__ offs,
                             const uint64_t *__restrict__ total, size_t cap, uint8_t *__restrict__ out)
{
    if (*total > cap) return;
    int c = blockIdx.x;
    if (c == 0) {
        for (int t = threadIdx.x; t < 16 + 4 * (C + 1); t += blockDim.x) {
            uint32_t v;
            if (t < 16) {
                uint32_t h[4] = {MAGIC, 1u | ((uint32_t)sched << 16), (uint32_t)H | ((uint32_t)W << 16),
                                 (uint32_t)C};
                v = h[t >> 2];
            } else {
                v = offs[(t - 16) >> 2];
            }
            out[t] = (uint8_t)(v >> (8 * (t & 3)));
        }
    }
    uint8_t *o = out + offs[c];
    for (int t = threadIdx.x; t < 128; t += blockDim.x)
        o[t] = (uint8_t)(states[(size_t)c * 32 + (t >> 2)] >> (8 * (t & 3)));
    uint32_t nw = nwords[c];
    const uint16_t *src = scratch + (size_t)c * cap_words + (cap_words - nw);
    uint16_t *dst = (uint16_t *)(o + 128);
    for (uint32_t t = threadIdx.x; t < nw; t += blockDim.x) dst[t] = src[t];
    if ((nw & 1) && threadIdx.x == 0) dst[nw] = 0;
}

void launch_rans_assemble(int H, int W, int C, int sched, const uint16_t *scratch, int cap_words,
                          const uint32_t *nwords, const uint32_t *states, uint8_t *out, size_t cap,
                          uint64_t *total, int *status, cudaStream_t s)
{
    // offsets live just after the stream lengths in the same scratch word
    uint32_t *offs = (uint32_t *)(nwords + C);
    k_rans_offsets<<<1, 1024, 0, s>>>(H, W, C, sched, nwords, out, cap, offs, total, status);
    k_rans_write<<<C, 256, 0, s>>>(H, W, C, sched, scratch, cap_words, nwords, states, offs, total, cap, out);
}

// ---------------------------------------------------------------- decoder

// Validate each slot's container and load every stream's 32 states; one
// thread per (slot, channel).  An invalid container sets the corrupt bit and
// leaves every stream empty (ptr = end), so later word reads are refused
// without touching memory.
__global__ void k_rans_dec_init(const Slot *__restrict__ S, int nslots, int C)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nslots * C) return;
    int b = t / C, c = t % C;
    const Slot &sl = S[b];
    const uint8_t *bs = sl.bs;
    size_t len = sl.len, hdr = 16 + 4 * (size_t)(C + 1);
    bool ok = bs != nullptr && len >= hdr;
    if (ok) {
        ok = ld32le(bs, 0) == MAGIC && ld16le(bs, 4) == 1 && (int)ld16le(bs, 6) == sl.sched &&
             (int)ld16le(bs, 8) == sl.H && (int)ld16le(bs, 10) == sl.W && (int)ld16le(bs, 12) == C;
    }
    uint32_t a = 0, e = 0;
    if (ok) {
        a = ld32le(bs, 16 + 4 * (size_t)c);
        e = ld32le(bs, 16 + 4 * (size_t)(c + 1));
        ok = a >= hdr && (a & 3) == 0 && (e & 3) == 0 && e >= a + 128 && e <= len;
    }
    if (!ok) {
        atomicOr(sl.status, ST_CORRUPT);
        for (int l = 0; l < 32; l++) sl.rstate[(size_t)c * 32 + l] = RANS_L;
        sl.rptr[c] = 0; sl.rend[c] = 0;
        return;
    }
    for (int l = 0; l < 32; l++) sl.rstate[(size_t)c * 32 + l] = ld32le(bs, a + 4 * l);
    sl.rptr[c] = a + 128;
    sl.rend[c] = e;
}

void launch_rans_dec_init(const Slot *S, int nslots, int C, cudaStream_t s)
{
    int n = nslots * C;
    if (n <= 0) return;
    k_rans_dec_init<<<(n + 127) / 128, 128, 0, s>>>(S, nslots, C);
}

// One schedule step of every channel of every slot: one warp per (slot,
// channel), see rans_step_item.
// Warp w takes channel c0 + w % nc of slot w / nc.
__global__ void k_rans_dec_step(CoderDev cd, const Slot *__restrict__ S, int nslots,
                                const int2 *__restrict__ kn, int C, int c0, int nc)
{
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nslots * nc) return;
    int b = w / nc, c = c0 + (w - b * nc);
    rans_step_item<true>(cd, S, kn, C, b * C + c);
}

void launch_rans_dec_step(const CoderDev &cd, const Slot *S, int nslots, const int2 *kn, int C, cudaStream_t s,
                          int c0, int nc)
{
    if (nc < 0) nc = C;
    int warps = nslots * nc;
    if (warps <= 0) return;
    launch_pdl(k_rans_dec_step, dim3((warps * 32 + 127) / 128), dim3(128), 0, s, cd, S, nslots, kn, C, c0, nc);
}

// After the last step every lane must be back at the initial state and
// every stream fully consumed (one zero pad word allowed).
__global__ void k_rans_dec_finish(const Slot *__restrict__ S, int nslots, int C)
{
    int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wi >= nslots * C) return;
    int b = wi / C, c = wi % C;
    const Slot &sl = S[b];
    bool bad = sl.rstate[(size_t)c * 32 + lane] != RANS_L;
    if (lane == 0) {
        uint32_t p = sl.rptr[c], e = sl.rend[c];
        if (e == 0) bad = true;
        else if (!(p == e || (p + 2 == e && ld16le(sl.bs, p) == 0))) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(sl.status, ST_CORRUPT);
}

void launch_rans_dec_finish(const Slot *S, int nslots, int C, cudaStream_t s)
{
    int warps = nslots * C;
    if (warps <= 0) return;
    k_rans_dec_finish<<<(warps * 32 + 127) / 128, 128, 0, s>>>(S, nslots, C);
}

}  // namespace psw

// ---------------------------------------------------------------- encoder without allocation
//
// psw_rans_encode_noalloc: the coder-only encoder of psw_rans_encode, but
// with every scratch buffer (schedule order, per-stream word buffers, stream
// lengths and offsets, final states, total, status) carved from one
// file-scope device array instead of a sequence's allocations.  The array
// is part of the loaded module: every GPU that loads this library holds it
// (NOALLOC_BYTES, about 9.2 MiB) until the process exits.

namespace psw {
namespace {

constexpr size_t NOALLOC_MAX_SYMBOLS = 1572864;      // H*W*C of one 68 x 120 x 192 latent frame
constexpr int NOALLOC_MAX_HW = 32768;
constexpr int NOALLOC_MAX_C = 256;
constexpr size_t NA_SLOT = 0;                                             // one Slot
constexpr size_t NA_ORDER = 512;                                          // int[MAX_HW]
constexpr size_t NA_NW = NA_ORDER + 4 * (size_t)NOALLOC_MAX_HW;           // u32[2C + 1]
constexpr size_t NA_STATES = NA_NW + 2304;                                // u32[32 C]
constexpr size_t NA_TOTAL = NA_STATES + 4 * 32 * (size_t)NOALLOC_MAX_C;   // u64
constexpr size_t NA_STATUS = NA_TOTAL + 256;                              // int
constexpr size_t NA_WORDS = NA_STATUS + 256;                              // u16[3 HW C + 64 C]
constexpr size_t NOALLOC_BYTES = NA_WORDS + 2 * (3 * NOALLOC_MAX_SYMBOLS + 64 * (size_t)NOALLOC_MAX_C);

static_assert(sizeof(Slot) <= 512, "slot record must fit its reserved space");

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_na_mu;
std::map<int, unsigned char *> g_na_addr;    // device -> address of g_noalloc_scratch on it

}  // namespace
}  // namespace psw

extern "C" psw_status psw_rans_encode_noalloc(const psw_ctx *ctx, const psw_frame_desc *fd, const int16_t *yhat_dev,
                                              const uint8_t *idx_dev, const int32_t *m_dev, uint8_t *bitstream_dev,
                                              size_t cap, size_t *len_out, void *stream)
{
    using namespace psw;
    int C = 0, mask = 0;
    const uint32_t *cdf = nullptr;
    const int *meta = nullptr;
    if (!psw_coder_view(ctx, &C, &mask, &cdf, &meta)) return PSW_ERR_INVALID;
    if (!fd || !yhat_dev || !idx_dev || !m_dev || !bitstream_dev || !len_out) return PSW_ERR_INVALID;
    if (fd->H < 1 || fd->W < 1 || (fd->schedule != PSW_SCHED_WAVEFRONT && fd->schedule != PSW_SCHED_RASTER))
        return PSW_ERR_INVALID;
    if (fd->schedule == PSW_SCHED_RASTER && mask == 1) return PSW_ERR_INVALID;
    size_t HW = (size_t)fd->H * fd->W;
    if (fd->H > 65535 || fd->W > 65535 || HW > (size_t)NOALLOC_MAX_HW || C > NOALLOC_MAX_C ||
        HW * (size_t)C > NOALLOC_MAX_SYMBOLS)
        return PSW_ERR_INVALID;                       // beyond the static scratch
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PSW_ERR_CUDA;
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        auto it = g_na_addr.find(dev);
        if (it == g_na_addr.end()) {
            // once per device, with that device current: the array's device
            // address (its host-side name is only a stand-in)
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PSW_ERR_CUDA;
            it = g_na_addr.emplace(dev, (unsigned char *)p).first;
        }
        base = it->second;
    }
    // schedule order (host), then the slot record the encoder reads
    std::vector<int> order(HW);
    if (fd->schedule == PSW_SCHED_RASTER) {
        for (size_t p = 0; p < HW; p++) order[p] = (int)p;
    } else {
        auto lab = [&](int i, int j) { return mask == 1 ? ((i % 4) + (j % 4)) % 4 : 2 * i + j; };
        int maxl = 0;
        for (int i = 0; i < fd->H; i++)
            for (int j = 0; j < fd->W; j++) maxl = std::max(maxl, lab(i, j));
        std::vector<int> cnt(maxl + 2, 0);
        for (int i = 0; i < fd->H; i++)
            for (int j = 0; j < fd->W; j++) cnt[lab(i, j) + 1]++;
        for (int t = 1; t <= maxl + 1; t++) cnt[t] += cnt[t - 1];
        for (int i = 0; i < fd->H; i++)
            for (int j = 0; j < fd->W; j++) order[cnt[lab(i, j)]++] = i * fd->W + j;
    }
    Slot sl;
    memset(&sl, 0, sizeof(sl));
    sl.H = fd->H; sl.W = fd->W; sl.stride = (int)HW; sl.sched = fd->schedule;
    sl.y = const_cast<int16_t *>(yhat_dev);
    sl.idx = const_cast<uint8_t *>(idx_dev);
    sl.m = const_cast<int32_t *>(m_dev);
    sl.order = (const int *)(base + NA_ORDER);
    sl.status = (int *)(base + NA_STATUS);
    int cap_words = 3 * (int)HW + 64;
    uint16_t *words = (uint16_t *)(base + NA_WORDS);
    uint32_t *nw = (uint32_t *)(base + NA_NW), *states = (uint32_t *)(base + NA_STATES);
    uint64_t *total = (uint64_t *)(base + NA_TOTAL);
    // the slot record and order are copied from pageable host memory (the
    // copies are complete when cudaMemcpyAsync returns); the status word and
    // total start at zero for every call
    if (cudaMemcpyAsync(base + NA_SLOT, &sl, sizeof(Slot), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(base + NA_ORDER, order.data(), HW * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(base + NA_TOTAL, 0, 512, s) != cudaSuccess)
        return PSW_ERR_CUDA;
    CoderDev cd{cdf, meta};
    launch_rans_encode(cd, (const Slot *)(base + NA_SLOT), 0, (int)HW, C, words, cap_words, nw, states, s);
    launch_rans_assemble(fd->H, fd->W, C, fd->schedule, words, cap_words, nw, states, bitstream_dev, cap, total,
                         (int *)(base + NA_STATUS), s);
    uint64_t h_total = 0;
    int h_status = 0;
    if (cudaMemcpyAsync(&h_total, total, sizeof(h_total), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&h_status, base + NA_STATUS, sizeof(h_status), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PSW_ERR_CUDA;
    *len_out = (size_t)h_total;
    if (h_status & ST_CAPACITY) return PSW_ERR_CAPACITY;
    return PSW_OK;
}
