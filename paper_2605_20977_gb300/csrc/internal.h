// internal.h -- declarations shared by the library's translation units.
// Not part of the public ABI (include/psw.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/psw.h"

namespace psw {

enum Prec { P_F32 = 0, P_BF16 = 1 };

// Device status bits (OR-ed by kernels into a device word).
enum : int { ST_CORRUPT = 1, ST_TIMEOUT = 2, ST_CAPACITY = 4 };

constexpr int NSCALES = 64;
constexpr int CDF_PREC = 16;
constexpr int MAX_KK = 81;        // largest window (9 x 9)
constexpr int MAX_TF = 4;         // frames in a temporal window

// ---------------------------------------------------------------- GEMM
// Y[m][n] = sum_k A[m][k] * Wt[n][k]  (A compact token-major, Wt the
// transposed projection, both in the compute type), FP32 accumulation in
// ascending k, then one of the epilogues below.  Every output element's
// arithmetic depends only on its own row of A and column of W, never on M or
// on the tile it falls in, so a token gets bit-identical results whether it
// is processed alone (decoder step) or with the whole frame (encoder).
enum EpiMode {
    EPI_STORE = 0,      // out[row][n] = y                 (row = m, or pos[m] if scatter)
    EPI_QKV = 1,        // n < q_cols: out[m][n]; then K cache[pos][.], V cache[pos][.]
    EPI_RESID = 2,      // resid[pos[m]][n] += y           (FP32 residual stream)
    EPI_RESID_BASE = 3, // resid[pos[m]][n] = base[pos[m]][n] + y
    EPI_SWIGLU = 4      // dual GEMM: out[m][n] = silu(y_gate) * y_up
};

struct Epi {
    int mode;
    const int *pos;     // token -> raster position (may be NULL = identity)
    int scatter;        // EPI_STORE: write row pos[m] instead of m
    int d;              // width of one K/V cache row
    int q_cols;         // EPI_QKV: leading columns that go to `out`
    void *out; int ld_out;
    void *kc; void *vc; // caches [HW][d]
    float *resid; const float *base;
};

struct GemmArgs {
    const void *A; int lda;       // [M][K]
    const void *Wt;               // [N][K]
    const void *Wt2;              // second operand of a dual GEMM (EPI_SWIGLU)
    int M, N, K;
    Epi epi;
    int *status;                  // device status word (ST_TIMEOUT from bounded waits)
};

// Enqueue one GEMM.  BF16 projections whose N and K tile evenly run on the
// tensor cores (the choice never depends on M); everything else on the SIMT
// kernel.  Returns false if the launch could not be prepared.
bool gemm(int prec, const GemmArgs &g, cudaStream_t s);
bool gemm_tc_supported(int prec, int N, int K);
bool gemm_tc_available();         // driver entry point for tensor maps present

// ---------------------------------------------------------------- kernels
void launch_transpose_convert(int prec, const float *src, int K, int N, void *dst, int row_off,
                              cudaStream_t s);
void launch_embed_latent(const int *pos, int n, const int16_t *y, int C, const float *gamma,
                         const float *W, const float *b, int d, float *x, cudaStream_t s);
void launch_fill_rows(const float *v, int n, int d, float *x, cudaStream_t s);
void launch_embed_hyper(const int16_t *z, int H, int W, int Wh, int Ch, int r, const float *gamma,
                        const float *Whp, const float *b, int d, float *eh, cudaStream_t s);
void launch_rmsnorm(int prec, const int *pos, int n, const float *src, const float *g, int d,
                    void *dst, int scatter, cudaStream_t s);

struct AttnArgs {
    const int *pos; int n;
    const void *Q; int q_full;               // compact [n][d], or full [HW][d] indexed by pos
    const void *K[MAX_TF]; const void *V[MAX_TF];
    int nfr;                                 // frames of keys, oldest first
    const float *bias;                       // + h * bias_h_stride + age * k*k + window offset
    int bias_h_stride;
    int age[MAX_TF];
    void *O;                                 // compact [n][d]
    int H, W, d, nh, k;
    int mask;                                // 0: 2i+j with raster clause, 1: cyclic
    int kind;                                // 0: accumulator A(p), 1: self-attention S(p), -1: window
};
void launch_attention(int prec, const AttnArgs &a, cudaStream_t s);

struct HeadsArgs {
    const int *pos; int n;
    const float *x; int d, C;
    const float *g, *W1m, *b1m, *W2m, *W1s, *b1s, *W2s;
    const float *gamma_mu, *beta_mu, *gamma_sig, *beta_sig;
    const float *scale;                      // device scale table [64]
    float *mu, *sigma; uint8_t *idx; int32_t *m;   // [HW][C]
};
void launch_heads(const HeadsArgs &h, cudaStream_t s);
void launch_quantize(size_t n, const float *mu, const float *sigma, const float *scale,
                     uint8_t *idx, int32_t *m, cudaStream_t s);
void launch_rate(size_t n, const int16_t *y, const float *mu, const float *sigma, double *partials,
                 double *out, cudaStream_t s);
int rate_partials(size_t n);

// ---------------------------------------------------------------- coding
struct CdfTables {
    float scale[NSCALES];
    int T[NSCALES], n[NSCALES], off[NSCALES];
    int total;                               // slots over all tables
    uint32_t *packed;                        // host: cum | freq << 16
};
void build_scale_table(float *tab);
void build_cdf_tables(CdfTables &t);        // allocates t.packed (free with free_cdf_tables)
void free_cdf_tables(CdfTables &t);

struct CoderDev {
    const uint32_t *cdf;                     // packed slots
    const int *meta;                         // [3][64]: T, n, off
};
size_t container_capacity(int H, int W, int C);
void launch_rans_encode(const CoderDev &cd, const int *order, int HW, int C, const int16_t *y,
                        const uint8_t *idx, const int32_t *m, uint16_t *scratch, int cap_words,
                        uint32_t *nwords, uint32_t *states, cudaStream_t s);
void launch_rans_assemble(int H, int W, int C, int sched, const uint16_t *scratch, int cap_words,
                          const uint32_t *nwords, const uint32_t *states, uint8_t *out, size_t cap,
                          uint64_t *total, int *status, cudaStream_t s);
void launch_rans_dec_init(const uint8_t *bs, size_t len, int H, int W, int C, int sched,
                          uint32_t *states, uint32_t *ptr, uint32_t *end, int *status, cudaStream_t s);
void launch_rans_dec_step(const CoderDev &cd, const int *order, int k0, int n, int C,
                          const uint8_t *idx, const int32_t *m, const uint8_t *bs, uint32_t *states,
                          uint32_t *ptr, const uint32_t *end, int16_t *y, int *status, cudaStream_t s);
void launch_rans_dec_finish(const uint8_t *bs, int C, const uint32_t *states, const uint32_t *ptr,
                            const uint32_t *end, int *status, cudaStream_t s);

}  // namespace psw
