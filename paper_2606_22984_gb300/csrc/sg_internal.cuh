// sg_internal.cuh -- internal declarations shared by the libsg translation
// units: device Philox4x32-10, the weight-blob offsets, the model and
// instance objects, and launch helpers.
#pragma once

#include <cuda_bf16.h>

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "sg.h"

#define SG_MAX_LAYERS 16

namespace sg {

// ---------------------------------------------------------------------------
// Error plumbing: every entry point converts failures to sg_status + message.
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
sg_status fail(sg_status code, const std::string &msg);
sg_status check_launch(const char *what);

// Every kernel launch passes its stream through counted(), which bumps the
// library's launch counter (sg_launch_count) and returns the stream.
cudaStream_t counted(cudaStream_t st);

#define SG_CUDA_TRY(expr)                                                              \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            cudaGetLastError(); /* clear a non-sticky error so it cannot leak */       \
            return ::sg::fail(SG_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
        }                                                                              \
    } while (0)

#define SG_TRY(expr)                        \
    do {                                    \
        sg_status s_ = (expr);              \
        if (s_ != SG_OK) return s_;         \
    } while (0)

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): two 32x32 -> 64-bit
// multiplies per round, Weyl key schedule, 10 rounds.  The uniform of word 0
// is ((x0 >> 8) + 0.5) * 2^-24, exactly representable in binary32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ float philox_uniform(uint64_t seed, uint32_t a, uint32_t b,
                                                uint32_t stream, uint32_t e)
{
    const uint4 r = philox4x32_10(make_uint4(a, b, stream, e), (uint32_t)seed,
                                  (uint32_t)(seed >> 32));
    return ((float)(r.x >> 8) + 0.5f) * (1.0f / 16777216.0f);
}

// log(sigmoid(x)) without overflow, FP32.
__device__ __forceinline__ float log_sigmoid_f(float x)
{
    return x >= 0.f ? -log1pf(expf(-x)) : x - log1pf(expf(x));
}

__device__ __forceinline__ float gelu_f(float x)
{
    return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad_f(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f))
           + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// 2^x and 1/x on the special-function unit (relative errors about 2^-22).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// GELU of the BF16 path: gelu(v) = v Phi(v), gelu'(v) = Phi(v) + v phi(v),
// with Phi(v) = (1 + erf(v / sqrt 2)) / 2 from the approximation of
// Abramowitz & Stegun, Handbook of Mathematical Functions, formula 7.1.26
// (after Hastings): erf(z) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5))))
// e^{-z^2}, t = 1 / (1 + p z), z >= 0, |error| <= 1.5e-7, odd in z.  Its
// exponential e^{-v^2/2} is also the normal density phi(v) up to 1/sqrt(2 pi).
// Every caller rounds the result to BF16 (relative step 2^-8), far coarser
// than the approximation; sg_gelu_selfcheck() measures it against erff.
__device__ __forceinline__ float gelu_as(float v, float *dgelu = nullptr)
{
    const float e = ex2_approx(v * v * -0.72134752044448170f);  // e^{-v^2/2} = 2^{-v^2 log2(e) / 2}
    const float z = fabsf(v) * 0.70710678118654752f;
    const float t = rcp_approx(fmaf(0.3275911f, z, 1.0f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
                 0.254829592f);
    const float h = 0.5f * poly * e;  // (1 - erf(z)) / 2
    const float Phi = v >= 0.f ? 1.0f - h : h;
    if (dgelu) *dgelu = fmaf(v * 0.39894228040143268f, e, Phi);
    return v * Phi;
}

// ---------------------------------------------------------------------------
// Weight-blob offsets (floats), blob layout of include/sg.h.
// ---------------------------------------------------------------------------
struct LayerOff {
    int64_t ln1g, ln1b, Wqkv, bqkv, ln2g, ln2b, W1, b1, W2, b2;
};

struct BlobOff {
    int64_t tok, pos;
    LayerOff L[SG_MAX_LAYERS];
    int64_t lnfg, lnfb, Wh, bh, total;
};

BlobOff blob_offsets(const sg_config &c);

// Patching (see sg_config): spins per token, tokens, classes.
__host__ __device__ __forceinline__ int spins_per_token(const sg_config &c)
{
    return c.patch > 1 ? c.patch : 1;
}

// Raster site of bit j of token t (patch map of sg_config).
__host__ __device__ __forceinline__ int patch_site(int t, int j, int P, int latD, int latL)
{
    if (P == 1) return t;
    if (latD == 0) return t * P + j;
    const int M = latL >> 1;
    int site = 0, stride = 1, rem = t;
    for (int k = 0; k < latD; ++k) {
        const int cell = rem % M;
        rem /= M;
        site += (2 * cell + ((j >> k) & 1)) * stride;
        stride *= latL;
    }
    return site;
}

// Offsets of the 16-byte aligned FP32 copies read with vector loads by the
// CUDA-core GEMMs: k-major (transposed) WqkvT [d][3d], W1T [d][d_ff],
// W2T [d_ff][d]; the row-major Wqkv, W1, W2 of the backward; and the biases.
struct PackOff {
    int64_t WqkvT[SG_MAX_LAYERS], W1T[SG_MAX_LAYERS], W2T[SG_MAX_LAYERS];
    int64_t Wqkv[SG_MAX_LAYERS], W1[SG_MAX_LAYERS], W2[SG_MAX_LAYERS];
    int64_t bqkv[SG_MAX_LAYERS], b1[SG_MAX_LAYERS], b2[SG_MAX_LAYERS];
    int64_t total;
};

PackOff pack_offsets(const sg_config &c);

// Everything a kernel needs about the model, passed by value.
struct DevModel {
    int N, L, d, nh, dt, dff, mask, W, S;   // N: tokens (the sequence length)
    int P, K, Nspins, latD, latL;           // patching: spins per token, classes
    const float *w;    // master FP32 blob
    const float *wt;   // transposed FP32 copies
    BlobOff o;
    PackOff p;
};

// Visible-key geometry of query t (mask of include/sg.h):
// keys [0, n_sink) then [band_lo, t].
__host__ __device__ __forceinline__ void visible_ranges(int mask, int W, int S, int t,
                                                        int &n_sink, int &band_lo)
{
    if (mask == SG_MASK_DENSE) {
        n_sink = 0;
        band_lo = 0;
    } else {
        n_sink = S < t + 1 ? S : t + 1;
        const int lo = t - W;
        band_lo = lo > S ? lo : S;
    }
}

__host__ __device__ __forceinline__ int band_count(int t, int band_lo)
{
    return t >= band_lo ? t - band_lo + 1 : 0;
}

__host__ __device__ __forceinline__ bool key_visible(int mask, int W, int S, int t, int k)
{
    if (k > t) return false;
    if (mask == SG_MASK_DENSE) return true;
    return (t - k <= W) || (k < S);
}

}  // namespace sg

// ---------------------------------------------------------------------------
// Library objects (opaque in the ABI).
// ---------------------------------------------------------------------------
struct sg_model {
    sg_config cfg;
    sg_config seq;            // cfg with N = tokens (the sequence the transformer sees)
    int64_t P;                // floats of all models' blobs
    int64_t P1 = 0;           // floats of one model's blob
    int n_models = 1;
    int device;
    sg::BlobOff off;
    sg::PackOff pack;
    float *w = nullptr;       // master FP32 blob
    float *wt = nullptr;      // transposed FP32 copies
    void *bf = nullptr;       // BF16 packed operands (tensor-core path)
    size_t bf_bytes = 0;
    void *kv = nullptr;       // KV-cache workspace
    size_t kv_bytes = 0;
    void *ws = nullptr;       // prefill / backward workspace
    size_t ws_bytes = 0;
    int64_t max_chunk = 0;    // cap on samples per prefill / backward chunk (0: by free memory)
    void *err = nullptr;      // device error word written by kernels (bounded waits, NaN)
    size_t err_bytes = 0;
    // tiled BF16 weights for the tensor-core teacher-forced pass and backward
    // (byte offsets per layer: Wqkv, W1, W2 as forward B operands; W2^T, W1^T,
    // Wqkv^T as backward B operands)
    void *bt = nullptr;
    size_t bt_bytes = 0;
    size_t bt_off[SG_MAX_LAYERS][6] = {};
};

struct sg_instance {
    int32_t kind, N, D, L, periodic;
    bool integer_bonds;
    float *J = nullptr;       // SK: [N][N]; EA: bonds [N][D]
    int8_t *Ji8 = nullptr;    // EA with integer bonds: bonds as int8
    void *Jbf = nullptr;      // SK: BF16 hi/lo split of J, tensor-core layout
    void *ws = nullptr;       // SK tensor-core path: tiled spins
    size_t ws_bytes = 0;
    void *err = nullptr;      // device error word
    size_t err_bytes = 0;
};

namespace sg {
sg_status ensure_buffer(void **ptr, size_t *have, size_t need);

// Launchers implemented in the kernel translation units.
sg_status launch_pack_f32(sg_model *m, cudaStream_t st);
sg_status launch_pack_bf16(sg_model *m, cudaStream_t st);
sg_status launch_pack_tiled_weights(sg_model *m, cudaStream_t st);
bool sk_tc_supported(int N);
sg_status prepare_sk_tc(sg_instance *inst);
sg_status launch_energy_sk_tc(const sg_instance *inst, const int8_t *spins, int64_t B, float *E,
                              void **ws, size_t *ws_bytes, int *err, cudaStream_t st);
sg_status launch_decode_bf16(sg_model *m, int64_t B, uint64_t seed, uint32_t sid, float band,
                             int8_t *spins, float *logq, uint32_t *flags, cudaStream_t st);
sg_status launch_decode_f32(sg_model *m, int64_t B, uint64_t seed, uint32_t sid, float band,
                            int8_t *spins, float *logq, uint32_t *flags, cudaStream_t st);
// KV-cache bytes the decodes need for B samples (sg_model_reserve sizes the
// workspace with these before a launch).
size_t decode_bf16_layout(const sg_model *m, int64_t B, int *rows, int *cpm, int64_t *tiles);
size_t decode_f32_kv_bytes(const sg_model *m, int64_t B);
sg_status launch_logprob_f32(sg_model *m, const int8_t *spins, int64_t B, float *logq,
                             cudaStream_t st);
sg_status launch_grad_f32(sg_model *m, const int8_t *spins, const float *coeff, int64_t B,
                          float *grad, float *logq, cudaStream_t st);
sg_status launch_energy(const sg_instance *inst, const int8_t *spins, int64_t B, int prec,
                        float *E, int32_t *E_int, cudaStream_t st);
sg_status launch_free_energy(const float *E, const float *logq, int64_t B, double beta,
                             double *out, float *coeff, cudaStream_t st);
sg_status launch_loss_coeff(const float *E, const float *logq, int64_t B, double a, double c,
                            double w, double *mean, float *coeff, cudaStream_t st);
sg_status launch_mh(const int8_t *prop, const float *E, const float *logq, int64_t B, int N,
                    int C, double beta, uint64_t seed, int8_t *cs, double *cE, double *cL,
                    int64_t *acc, float *trace, cudaStream_t st);
sg_status launch_metropolis(const sg_instance *inst, int8_t *spins, int64_t R, int sweeps,
                            double beta, uint64_t seed, double *E, float *trace,
                            cudaStream_t st);
sg_status launch_overlap(const int8_t *spins, int64_t B, int N, int64_t *hist, cudaStream_t st);
bool attn_tc_supported(const sg_config &c);
sg_status launch_attn_fwd_tc(const sg_config &c, const float *QKV, const float *Hin, float *O,
                             float *Hmid, float *LSE, int Bc, int *err, cudaStream_t st);
sg_status launch_attn_bwd_tc(const sg_config &c, const float *QKV, const float *O, const float *dO,
                             const float *LSE, float *dQKV, float *Dt, int Bc, int *err,
                             cudaStream_t st);
// Attention of the BF16 teacher-forced pass on warp-level tensor-core MMAs
// (head dims 16 and 32), QKV rows in BF16; O is kept in BF16 for the
// backward (or not written when O is null); the backward writes dQKV as wide
// BF16 and per-sample bias sums bsum [Bc][3 d].
bool attn_mma_supported(const sg_config &c);
sg_status launch_attn_fwd_mma(const sg_config &c, const __nv_bfloat16 *QKVh, const float *Hin,
                              __nv_bfloat16 *O, float *Hmid, float *LSE, int Bc, cudaStream_t st);
sg_status launch_attn_bwd_mma(const sg_config &c, const __nv_bfloat16 *QKVh, const __nv_bfloat16 *O,
                              const float *dO, const float *LSE, unsigned char *dQKVt, float *bsum,
                              int Bc, cudaStream_t st);
// The same contract on tcgen05 (TMEM scores, thread-per-row softmax) for
// d_h = 16 shapes whose queries see many keys; err receives a time-out code.
bool attn_tmem_supported(const sg_config &c);
sg_status launch_attn_fwd_tmem(const sg_config &c, const __nv_bfloat16 *QKVh, const float *Hin,
                               __nv_bfloat16 *O, float *Hmid, float *LSE, int Bc, int *err, cudaStream_t st);
sg_status launch_attn_bwd_tmem(const sg_config &c, const __nv_bfloat16 *QKVh, const __nv_bfloat16 *O,
                               const float *dO, const float *LSE, unsigned char *dQKVt, float *bsum, int Bc,
                               int *err, cudaStream_t st);
// Band masks on sequences too long to stage whole: per-tile tcgen05 kernels
// (d_h 16 or 32) with the same contract.
bool attn_band_supported(const sg_config &c);
sg_status launch_attn_fwd_band(const sg_config &c, const __nv_bfloat16 *QKVh, const float *Hin, __nv_bfloat16 *O,
                               float *Hmid, float *LSE, int Bc, int *err, cudaStream_t st);
sg_status launch_attn_bwd_band(const sg_config &c, const __nv_bfloat16 *QKVh, const __nv_bfloat16 *O,
                               const float *dO, const float *LSE, unsigned char *dQKVt, float *bsum, int Bc,
                               int *err, cudaStream_t st);
sg_status launch_adam(float *w, const float *g, float *m, float *v, int64_t n, float lr,
                      float b1, float b2, float eps, int64_t step, cudaStream_t st);
}  // namespace sg
