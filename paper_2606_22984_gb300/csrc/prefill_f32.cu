// prefill_f32.cu -- teacher-forced log q (Algorithm 1 structure with the
// pre-LayerNorm placement of Algorithm 2) over whole sequences, and the
// hand-written backward of sum_b c_b log q(sigma_b) (REINFORCE, Eq. loss1).
//
// Rows r = b * N + t of a chunk of samples are processed layer by layer:
//   embed -> [LN1 -> QKV GEMM -> masked attention (+residual) -> LN2 ->
//   FFN1 GEMM (GELU) -> FFN2 GEMM (+residual)] x n_layers -> LN_f -> head.
// For the gradient every layer's activations of the chunk are kept and the
// backward runs in reverse; the chunk size bounds memory, so any B fits.
// All arithmetic is FP32 on CUDA cores; weight gradients are reduced over rows
// with per-block partial sums and atomics.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "gemm_tc.cuh"
#include "sg_internal.cuh"

namespace sg {

namespace {

__device__ __forceinline__ float wsum(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Embedding (Eq. concatePE): H[r] = [tok(s_{t-1}); pos(t)], start token 0.
// ---------------------------------------------------------------------------
__global__ void embed_kernel(const int8_t *__restrict__ spins, int64_t R, int N, int D, int dt,
                             const float *__restrict__ tok, const float *__restrict__ pos,
                             float *__restrict__ H)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * D) return;
    const int64_t r = i / D;
    const int j = (int)(i % D), t = (int)(r % N);
    if (j < dt) {
        const int tk = t == 0 ? 0 : (spins[r - 1] + 1) >> 1;
        H[i] = tok[tk * dt + j];
    } else {
        H[i] = pos[(size_t)t * (D - dt) + (j - dt)];
    }
}

// The same embedding, one float4 of a row per thread (D a multiple of 4):
// 256 / (D / 4) rows per block, the row's token read once.
__global__ void embed4_kernel(const int8_t *__restrict__ spins, int64_t R, int N, int D, int dt,
                              const float *__restrict__ tok, const float *__restrict__ pos,
                              float *__restrict__ H)
{
    const int D4 = D >> 2, rpb = blockDim.x / D4;
    const int lr = threadIdx.x / D4, c4 = threadIdx.x - lr * D4;
    if (lr >= rpb) return;
    const int64_t r = (int64_t)blockIdx.x * rpb + lr;
    if (r >= R) return;
    const int t = (int)(r % N);
    const int tk = t == 0 ? 0 : (spins[r - 1] + 1) >> 1;
    const float *prow = pos + (size_t)t * (D - dt) - dt;
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int j = 4 * c4 + k;
        v[k] = j < dt ? tok[tk * dt + j] : prow[j];
    }
    *reinterpret_cast<float4 *>(H + r * D + 4 * c4) = make_float4(v[0], v[1], v[2], v[3]);
}

// ---------------------------------------------------------------------------
// Patched models (sg_config.patch > 1): one token of P spins per position,
// a softmax head over K = 2^P classes.  Rows r = b T + t of a chunk.
// ---------------------------------------------------------------------------
__global__ void spins_to_tokens_kernel(const int8_t *__restrict__ spins, int64_t R, int T, int Ns,
                                       int P, int latD, int latL, uint8_t *__restrict__ tok)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R) return;
    const int64_t b = i / T;
    const int t = (int)(i % T);
    int v = 0;
    for (int j = 0; j < P; ++j) v |= ((spins[b * Ns + patch_site(t, j, P, latD, latL)] + 1) >> 1) << j;
    tok[i] = (uint8_t)v;
}

__global__ void embed_tok_kernel(const uint8_t *__restrict__ tok, int64_t R, int T, int D, int dt,
                                 const float *__restrict__ tokE, const float *__restrict__ pos,
                                 float *__restrict__ H)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * D) return;
    const int64_t r = i / D;
    const int j = (int)(i % D), t = (int)(r % T);
    if (j < dt) H[i] = tokE[(t == 0 ? 0 : tok[r - 1]) * dt + j];
    else H[i] = pos[(size_t)t * (D - dt) + (j - dt)];
}

__global__ void embed_bwd_tok_kernel(const float *__restrict__ dH, const uint8_t *__restrict__ tok,
                                     int Bc, int T, int D, int dt, float *__restrict__ gtok,
                                     float *__restrict__ gpos)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)T * D) return;
    const int t = (int)(i / D), j = (int)(i % D);
    if (j >= dt) {
        float s = 0.f;
        for (int b = 0; b < Bc; ++b) s += dH[((size_t)b * T + t) * D + j];
        atomicAdd(gpos + (size_t)t * (D - dt) + (j - dt), s);
    } else {
        for (int b = 0; b < Bc; ++b) {
            const size_t r = (size_t)b * T + t;
            const int tk = t == 0 ? 0 : tok[r - 1];
            atomicAdd(gtok + tk * dt + j, dH[r * D + j]);
        }
    }
}

// Warp per row: LN_f, the K logits, log-sum-exp; lp = z[tok] - lse.  Saves
// Y, mu, rs and lse for the backward (which recomputes the logits from Y).
__global__ void head_fwd_cat_kernel(const float *__restrict__ H, const float *__restrict__ g,
                                    const float *__restrict__ bb, const float *__restrict__ Wh,
                                    const float *__restrict__ bh, const uint8_t *__restrict__ tok,
                                    float *__restrict__ Y, float *__restrict__ mu,
                                    float *__restrict__ rs, float *__restrict__ lse_out,
                                    float *__restrict__ lp, int64_t R, int D, int K)
{
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= R) return;
    const float *x = H + r * D;
    float s = 0.f;
    for (int j = lane; j < D; j += 32) s += x[j];
    const float mean = wsum(s) / D;
    float q = 0.f;
    for (int j = lane; j < D; j += 32) {
        const float dv = x[j] - mean;
        q += dv * dv;
    }
    const float r_s = 1.0f / sqrtf(wsum(q) / D + 1e-5f);
    float yv[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int j = lane + 32 * i;
        yv[i] = j < D ? (x[j] - mean) * r_s * g[j] + bb[j] : 0.f;
        if (Y && j < D) Y[r * D + j] = yv[i];
    }
    const int tk = tok[r];
    float mx = -INFINITY, se = 0.f, zt = 0.f;
    for (int k = 0; k < K; ++k) {
        float zk = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int j = lane + 32 * i;
            if (j < D) zk += yv[i] * Wh[(size_t)k * D + j];
        }
        zk = wsum(zk) + bh[k];
        const float mn = fmaxf(mx, zk);
        se = se * expf(mx - mn) + expf(zk - mn);
        mx = mn;
        if (k == tk) zt = zk;
    }
    if (lane == 0) {
        const float lse = mx + logf(se);
        if (lse_out) lse_out[r] = lse;
        if (mu) {
            mu[r] = mean;
            rs[r] = r_s;
        }
        lp[r] = zt - lse;
    }
}

// dz_k = c_b (onehot(tok) - softmax(z)_k), then LN_f backward into dH and the
// head / LN_f weight gradients (shared-memory partial sums when K D fits).
__global__ void head_bwd_cat_kernel(const float *__restrict__ H, const float *__restrict__ mu,
                                    const float *__restrict__ rs, const float *__restrict__ Y,
                                    const float *__restrict__ lse, const uint8_t *__restrict__ tok,
                                    const float *__restrict__ coeff, const float *__restrict__ g,
                                    const float *__restrict__ Wh, const float *__restrict__ bh,
                                    float *__restrict__ dH, float *__restrict__ gWh,
                                    float *__restrict__ gbh, float *__restrict__ glnfg,
                                    float *__restrict__ glnfb, int64_t R, int T, int D, int K,
                                    int rows_per_block, int shared_sums)
{
    extern __shared__ float red[];  // [K][D] Wh, [D] lnf_g, [D] lnf_b, [K] bh
    float *rW = red, *rg = red + (size_t)K * D, *rb = rg + D, *rh = rb + D;
    if (shared_sums)
        for (int j = threadIdx.x; j < K * D + 2 * D + K; j += blockDim.x) red[j] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    for (int64_t r = r0 + warp; r < R && r < r0 + rows_per_block; r += nw) {
        const float c = coeff[r / T];
        const int tk = tok[r];
        float yv[16], dy[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int j = lane + 32 * i;
            yv[i] = j < D ? Y[r * D + j] : 0.f;
            dy[i] = 0.f;
        }
        for (int k = 0; k < K; ++k) {
            float zk = 0.f;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int j = lane + 32 * i;
                if (j < D) zk += yv[i] * Wh[(size_t)k * D + j];
            }
            zk = wsum(zk) + bh[k];
            const float dz = c * ((k == tk ? 1.f : 0.f) - expf(zk - lse[r]));
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int j = lane + 32 * i;
                if (j >= D) break;
                dy[i] += dz * Wh[(size_t)k * D + j];
                if (shared_sums) atomicAdd(rW + (size_t)k * D + j, dz * yv[i]);
                else atomicAdd(gWh + (size_t)k * D + j, dz * yv[i]);
            }
            if (lane == 0) {
                if (shared_sums) atomicAdd(rh + k, dz);
                else atomicAdd(gbh + k, dz);
            }
        }
        const float m = mu[r], s = rs[r];
        float m1 = 0.f, m2 = 0.f, xh[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int j = lane + 32 * i;
            xh[i] = j < D ? (H[r * D + j] - m) * s : 0.f;
            if (j < D) {
                const float dxh = dy[i] * g[j];
                m1 += dxh;
                m2 += dxh * xh[i];
                if (shared_sums) {
                    atomicAdd(rg + j, dy[i] * xh[i]);
                    atomicAdd(rb + j, dy[i]);
                } else {
                    atomicAdd(glnfg + j, dy[i] * xh[i]);
                    atomicAdd(glnfb + j, dy[i]);
                }
            }
        }
        m1 = wsum(m1) / D;
        m2 = wsum(m2) / D;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int j = lane + 32 * i;
            if (j < D) dH[r * D + j] = s * (dy[i] * g[j] - m1 - xh[i] * m2);
        }
    }
    if (!shared_sums) return;
    __syncthreads();
    for (int j = threadIdx.x; j < K * D; j += blockDim.x) atomicAdd(gWh + j, rW[j]);
    for (int j = threadIdx.x; j < D; j += blockDim.x) {
        atomicAdd(glnfg + j, rg[j]);
        atomicAdd(glnfb + j, rb[j]);
    }
    for (int j = threadIdx.x; j < K; j += blockDim.x) atomicAdd(gbh + j, rh[j]);
}

// ---------------------------------------------------------------------------
// LayerNorm forward / backward, one warp per row (eps 1e-5, biased variance).
// ---------------------------------------------------------------------------
__global__ void ln_fwd_kernel(const float *__restrict__ X, const float *__restrict__ g,
                              const float *__restrict__ b, float *__restrict__ Y,
                              float *__restrict__ mu, float *__restrict__ rs, int64_t R, int D,
                              unsigned char *__restrict__ At = nullptr)
{
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= R) {  // padding rows of the wide copy's last row block are zero
        if (At && r < tl_blocks(R) * 128)
            for (int j = 2 * lane; j < D; j += 64)
                *reinterpret_cast<__nv_bfloat162 *>(At + wl_offset(r, j, D)) = __floats2bfloat162_rn(0.f, 0.f);
        return;
    }
    const float *x = X + r * D;
    float s = 0.f;
    for (int j = lane; j < D; j += 32) s += x[j];
    const float mean = wsum(s) / D;
    float q = 0.f;
    for (int j = lane; j < D; j += 32) {
        const float dv = x[j] - mean;
        q += dv * dv;
    }
    const float r_s = 1.0f / sqrtf(wsum(q) / D + 1e-5f);
    if (Y)
        for (int j = lane; j < D; j += 32) Y[r * D + j] = (x[j] - mean) * r_s * g[j] + b[j];
    if (At) {  // wide BF16 copy, two columns per lane (D even)
        for (int j = 2 * lane; j < D; j += 64) {
            const __nv_bfloat162 v = __floats2bfloat162_rn((x[j] - mean) * r_s * g[j] + b[j],
                                                           (x[j + 1] - mean) * r_s * g[j + 1] + b[j + 1]);
            *reinterpret_cast<__nv_bfloat162 *>(At + wl_offset(r, j, D)) = v;
        }
    }
    if (lane == 0 && mu) {
        mu[r] = mean;
        rs[r] = r_s;
    }
}

// dX (+)= d LN(X)/dX^T dY; dg += sum_r dY xhat; db += sum_r dY.  D <= 512.
__global__ void ln_bwd_kernel(const float *__restrict__ dY, const float *__restrict__ X,
                              const float *__restrict__ mu, const float *__restrict__ rs,
                              const float *__restrict__ g, float *__restrict__ dX, int accumulate,
                              float *__restrict__ dg, float *__restrict__ db, int64_t R, int D,
                              int rows_per_block)
{
    extern __shared__ float red[];  // [2][D]
    for (int j = threadIdx.x; j < 2 * D; j += blockDim.x) red[j] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    float pg[16], pb[16];
    for (int i = 0; i < 16; ++i) pg[i] = pb[i] = 0.f;
    for (int64_t r = r0 + warp; r < R && r < r0 + rows_per_block; r += nw) {
        const float m = mu[r], s = rs[r];
        float m1 = 0.f, m2 = 0.f;
        int i = 0;
        for (int j = lane; j < D; j += 32, ++i) {
            const float xh = (X[r * D + j] - m) * s, dy = dY[r * D + j];
            const float dxh = dy * g[j];
            m1 += dxh;
            m2 += dxh * xh;
            pg[i] += dy * xh;
            pb[i] += dy;
        }
        m1 = wsum(m1) / D;
        m2 = wsum(m2) / D;
        for (int j = lane; j < D; j += 32) {
            const float xh = (X[r * D + j] - m) * s;
            const float v = s * (dY[r * D + j] * g[j] - m1 - xh * m2);
            if (accumulate) dX[r * D + j] += v;
            else dX[r * D + j] = v;
        }
    }
    int i = 0;
    for (int j = lane; j < D; j += 32, ++i) {
        atomicAdd(red + j, pg[i]);
        atomicAdd(red + D + j, pb[i]);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < D; j += blockDim.x) {
        atomicAdd(dg + j, red[j]);
        atomicAdd(db + j, red[D + j]);
    }
}

// ---------------------------------------------------------------------------
// Row kernels with 8 contiguous columns per lane (D in {32, 64, 128, 256}):
// LPR = D / 8 lanes share a row, a warp covers 32 / LPR rows per pass and
// keeps RPW passes of loads in flight.  Per-row sums reduce over the row's
// lanes with xor shuffles (offsets below LPR stay inside the lane group), and
// a lane's 8 columns are one 16-byte piece of the wide BF16 layout.
// ---------------------------------------------------------------------------
template <int LPR>
__device__ __forceinline__ float gsum(float v)
{
#pragma unroll
    for (int o = LPR / 2; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void ld8(const float *p, float (&v)[8])
{
    const float4 a = *reinterpret_cast<const float4 *>(p);
    const float4 b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// Parameter vectors (LayerNorm affine, head rows) sit at arbitrary float
// offsets of the weight blob: scalar loads.
__device__ __forceinline__ void ld8s(const float *p, float (&v)[8])
{
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __ldg(p + j);
}

__device__ __forceinline__ void st8(float *p, const float (&v)[8])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4 *>(p + 4) = make_float4(v[4], v[5], v[6], v[7]);
}

__device__ __forceinline__ uint4 pack8_bf16(const float (&v)[8])
{
    uint4 q;
    __nv_bfloat162 h;
    h = __floats2bfloat162_rn(v[0], v[1]); q.x = *reinterpret_cast<uint32_t *>(&h);
    h = __floats2bfloat162_rn(v[2], v[3]); q.y = *reinterpret_cast<uint32_t *>(&h);
    h = __floats2bfloat162_rn(v[4], v[5]); q.z = *reinterpret_cast<uint32_t *>(&h);
    h = __floats2bfloat162_rn(v[6], v[7]); q.w = *reinterpret_cast<uint32_t *>(&h);
    return q;
}

bool g8_width(int D) { return D == 32 || D == 64 || D == 128 || D == 256; }

// LayerNorm forward: Y (FP32, optional) and/or the wide BF16 copy At (rows
// past R up to the row-block end zeroed), mean and 1/std per row (optional).
template <int D, int RPW>
__global__ void __launch_bounds__(256)
ln_fwd_g8_kernel(const float *__restrict__ X, const float *__restrict__ g,
                 const float *__restrict__ b, float *__restrict__ Y, float *__restrict__ mu,
                 float *__restrict__ rs, int64_t R, unsigned char *__restrict__ At)
{
    constexpr int LPR = D / 8, RPP = 32 / LPR, RPI = RPW * RPP;
    const int lane = threadIdx.x & 31, sub = lane / LPR, c0 = 8 * (lane % LPR);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t R_end = At ? tl_blocks(R) * 128 : R;
    float gl[8], bl[8];
    ld8s(g + c0, gl);
    ld8s(b + c0, bl);
    for (int64_t r0 = gw * RPI; r0 < R_end; r0 += nw * RPI) {
        float x[RPW][8], mean[RPW], r_s[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int64_t r = r0 + q * RPP + sub;
            if (r < R) ld8(X + r * D + c0, x[q]);
            else
#pragma unroll
                for (int j = 0; j < 8; ++j) x[q][j] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) s += x[q][j];
            mean[q] = gsum<LPR>(s) / D;
        }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            float v = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float dv = x[q][j] - mean[q];
                v += dv * dv;
            }
            r_s[q] = 1.0f / sqrtf(gsum<LPR>(v) / D + 1e-5f);
        }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int64_t r = r0 + q * RPP + sub;
            if (r >= R_end) break;
            float y[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) y[j] = r < R ? (x[q][j] - mean[q]) * r_s[q] * gl[j] + bl[j] : 0.f;
            if (At) *reinterpret_cast<uint4 *>(At + wl_offset(r, c0, D)) = pack8_bf16(y);
            if (r >= R) continue;
            if (Y) st8(Y + r * D + c0, y);
            if (mu && c0 == 0) {
                mu[r] = mean[q];
                rs[r] = r_s[q];
            }
        }
    }
}

// Output head forward (LN_f -> z = Wh y + bh -> l = z1 - z0 -> lp).
template <int D, int RPW>
__global__ void __launch_bounds__(256)
head_fwd_g8_kernel(const float *__restrict__ H, const float *__restrict__ g,
                   const float *__restrict__ bb, const float *__restrict__ Wh,
                   const float *__restrict__ bh, const int8_t *__restrict__ spins,
                   float *__restrict__ mu, float *__restrict__ rs, float *__restrict__ ell,
                   float *__restrict__ lp, int64_t R)
{
    constexpr int LPR = D / 8, RPP = 32 / LPR, RPI = RPW * RPP;
    const int lane = threadIdx.x & 31, sub = lane / LPR, c0 = 8 * (lane % LPR);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float gl[8], bl[8], w0[8], w1[8];
    ld8s(g + c0, gl);
    ld8s(bb + c0, bl);
    ld8s(Wh + c0, w0);
    ld8s(Wh + D + c0, w1);
    const float bh0 = bh[0], bh1 = bh[1];
    for (int64_t r0 = gw * RPI; r0 < R; r0 += nw * RPI) {
        float x[RPW][8];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int64_t r = r0 + q * RPP + sub;
            ld8(H + (r < R ? r : R - 1) * D + c0, x[q]);
        }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int64_t r = r0 + q * RPP + sub;
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) s += x[q][j];
            const float mean = gsum<LPR>(s) / D;
            float v = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float dv = x[q][j] - mean;
                v += dv * dv;
            }
            const float r_s = 1.0f / sqrtf(gsum<LPR>(v) / D + 1e-5f);
            float z0 = 0.f, z1 = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float y = (x[q][j] - mean) * r_s * gl[j] + bl[j];
                z0 += y * w0[j];
                z1 += y * w1[j];
            }
            z0 = gsum<LPR>(z0) + bh0;
            z1 = gsum<LPR>(z1) + bh1;
            if (c0 == 0 && r < R) {
                const float l = z1 - z0;
                if (ell) ell[r] = l;
                if (mu) {
                    mu[r] = mean;
                    rs[r] = r_s;
                }
                lp[r] = log_sigmoid_f((float)spins[r] * l);
            }
        }
    }
}

// Output head backward: dl = c_b s sigmoid(-s l) per row, y recomputed from
// H, mean and 1/std; LN_f backward into dH; Wh, bh, lnf gradients reduced
// per lane, per warp (shuffles over the lanes of a column group), per block
// (shared memory), then one atomic per value and block.
template <int D, int RPW>
__global__ void __launch_bounds__(256)
head_bwd_g8_kernel(const float *__restrict__ H, const float *__restrict__ mu,
                   const float *__restrict__ rs, const float *__restrict__ ell,
                   const int8_t *__restrict__ spins, const float *__restrict__ coeff,
                   const float *__restrict__ g, const float *__restrict__ bb,
                   const float *__restrict__ Wh, float *__restrict__ dH, float *__restrict__ gWh,
                   float *__restrict__ gbh, float *__restrict__ glnfg, float *__restrict__ glnfb,
                   int64_t R, int N, unsigned char *__restrict__ dHt, float *__restrict__ dcol)
{
    constexpr int LPR = D / 8, RPP = 32 / LPR, RPI = RPW * RPP;
    __shared__ float red[5 * D + 2];
    for (int j = threadIdx.x; j < 5 * D + 2; j += blockDim.x) red[j] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, sub = lane / LPR, c0 = 8 * (lane % LPR);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float gl[8], bl[8], w0[8], w1[8];
    ld8s(g + c0, gl);
    ld8s(bb + c0, bl);
    ld8s(Wh + c0, w0);
    ld8s(Wh + D + c0, w1);
    float pw0[8], pw1[8], pg[8], pb[8], pc[8], pz = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) pw0[j] = pw1[j] = pg[j] = pb[j] = pc[j] = 0.f;
    const int64_t R_end = dHt ? tl_blocks(R) * 128 : R;
    for (int64_t r0 = gw * RPI; r0 < R_end; r0 += nw * RPI) {
        float x[RPW][8], s[RPW], dl[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int64_t r = r0 + q * RPP + sub, rr = r < R ? r : R - 1;
            ld8(H + rr * D + c0, x[q]);
            const float m = mu[rr];
            s[q] = rs[rr];
            const float sg = (float)spins[rr];
            dl[q] = r < R ? coeff[rr / N] * sg / (1.0f + expf(sg * ell[rr])) : 0.f;  // c s sigmoid(-s l)
#pragma unroll
            for (int j = 0; j < 8; ++j) x[q][j] = (x[q][j] - m) * s[q];  // xhat
        }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int64_t r = r0 + q * RPP + sub;
            float m1 = 0.f, m2 = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float xh = x[q][j];
                const float y = xh * gl[j] + bl[j];
                const float dy = dl[q] * (w1[j] - w0[j]);  // dz1 = dl, dz0 = -dl
                pw0[j] -= dl[q] * y;
                pw1[j] += dl[q] * y;
                pg[j] += dy * xh;
                pb[j] += dy;
                const float dxh = dy * gl[j];
                m1 += dxh;
                m2 += dxh * xh;
            }
            m1 = gsum<LPR>(m1) / D;
            m2 = gsum<LPR>(m2) / D;
            if (c0 == 0) pz += dl[q];
            float out[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float dxh = dl[q] * (w1[j] - w0[j]) * gl[j];
                out[j] = r < R ? s[q] * (dxh - m1 - x[q][j] * m2) : 0.f;
                pc[j] += out[j];
            }
            if (r < R) st8(dH + r * D + c0, out);
            if (dHt && r < R_end) *reinterpret_cast<uint4 *>(dHt + wl_offset(r, c0, D)) = pack8_bf16(out);
        }
    }
    // lanes with the same column group: offsets LPR, 2 LPR, ..., 16
#pragma unroll
    for (int o = LPR; o < 32; o <<= 1)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            pw0[j] += __shfl_xor_sync(0xffffffffu, pw0[j], o);
            pw1[j] += __shfl_xor_sync(0xffffffffu, pw1[j], o);
            pg[j] += __shfl_xor_sync(0xffffffffu, pg[j], o);
            pb[j] += __shfl_xor_sync(0xffffffffu, pb[j], o);
            pc[j] += __shfl_xor_sync(0xffffffffu, pc[j], o);
        }
    pz = wsum(pz);
    if (sub == 0)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            atomicAdd(red + c0 + j, pw0[j]);
            atomicAdd(red + D + c0 + j, pw1[j]);
            atomicAdd(red + 2 * D + c0 + j, pg[j]);
            atomicAdd(red + 3 * D + c0 + j, pb[j]);
            atomicAdd(red + 4 * D + 2 + c0 + j, pc[j]);
        }
    if (lane == 0) atomicAdd(red + 4 * D, pz);
    __syncthreads();
    for (int j = threadIdx.x; j < D; j += blockDim.x) {
        atomicAdd(gWh + j, red[j]);
        atomicAdd(gWh + D + j, red[D + j]);
        atomicAdd(glnfg + j, red[2 * D + j]);
        atomicAdd(glnfb + j, red[3 * D + j]);
        if (dcol) atomicAdd(dcol + j, red[4 * D + 2 + j]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(gbh, -red[4 * D]);
        atomicAdd(gbh + 1, red[4 * D]);
    }
}

// LayerNorm backward: dX = dres + rs (dY g - m1 - xhat m2) (dres may be
// null), m1 = mean(dY g), m2 = mean(dY g xhat); dg += sum dY xhat, db += sum
// dY.  Optionally the wide BF16 copy dXt of dX (rows past R up to the
// row-block end zeroed) and dcol += sum_r dX (the bias gradient of the layer
// that produced X's input gradient).
template <int D, int RPW>
__global__ void __launch_bounds__(256)
ln_bwd_g8_kernel(const float *__restrict__ dY, const float *__restrict__ X,
                 const float *__restrict__ mu, const float *__restrict__ rs,
                 const float *__restrict__ g, const float *__restrict__ dres,
                 float *__restrict__ dX, float *__restrict__ dg, float *__restrict__ db, int64_t R,
                 unsigned char *__restrict__ dXt, float *__restrict__ dcol)
{
    constexpr int LPR = D / 8, RPP = 32 / LPR, RPI = RPW * RPP;
    __shared__ float red[3][D];
    for (int j = threadIdx.x; j < 3 * D; j += blockDim.x) (&red[0][0])[j] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, sub = lane / LPR, c0 = 8 * (lane % LPR);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t R_end = dXt ? tl_blocks(R) * 128 : R;
    float gl[8], pg[8], pb[8], pc[8];
    ld8s(g + c0, gl);
#pragma unroll
    for (int j = 0; j < 8; ++j) pg[j] = pb[j] = pc[j] = 0.f;
    for (int64_t r0 = gw * RPI; r0 < R_end; r0 += nw * RPI) {
        float x[RPW][8], dy[RPW][8], s[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int64_t r = r0 + q * RPP + sub, rr = r < R ? r : R - 1;
            const float m = mu[rr];
            s[q] = rs[rr];
            ld8(X + rr * D + c0, x[q]);
            ld8(dY + rr * D + c0, dy[q]);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                x[q][j] = (x[q][j] - m) * s[q];  // xhat
                if (r >= R) dy[q][j] = 0.f;      // rows past the end add nothing
            }
        }
        float m1[RPW], m2[RPW];  // all lanes shuffle before any row is skipped
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            float a = 0.f, c = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float dxh = dy[q][j] * gl[j];
                a += dxh;
                c += dxh * x[q][j];
            }
            m1[q] = gsum<LPR>(a) * (1.0f / D);
            m2[q] = gsum<LPR>(c) * (1.0f / D);
        }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int64_t r = r0 + q * RPP + sub;
            if (r >= R_end) break;
            float out[8];
            if (dres && r < R) ld8(dres + r * D + c0, out);
            else
#pragma unroll
                for (int j = 0; j < 8; ++j) out[j] = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (r < R) out[j] += s[q] * (dy[q][j] * gl[j] - m1[q] - x[q][j] * m2[q]);
                pg[j] += dy[q][j] * x[q][j];
                pb[j] += dy[q][j];
                pc[j] += out[j];
            }
            if (r < R) st8(dX + r * D + c0, out);
            if (dXt) *reinterpret_cast<uint4 *>(dXt + wl_offset(r, c0, D)) = pack8_bf16(out);
        }
    }
#pragma unroll
    for (int o = LPR; o < 32; o <<= 1)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            pg[j] += __shfl_xor_sync(0xffffffffu, pg[j], o);
            pb[j] += __shfl_xor_sync(0xffffffffu, pb[j], o);
            pc[j] += __shfl_xor_sync(0xffffffffu, pc[j], o);
        }
    if (sub == 0)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            atomicAdd(&red[0][c0 + j], pg[j]);
            atomicAdd(&red[1][c0 + j], pb[j]);
            atomicAdd(&red[2][c0 + j], pc[j]);
        }
    __syncthreads();
    for (int j = threadIdx.x; j < D; j += blockDim.x) {
        atomicAdd(dg + j, red[0][j]);
        atomicAdd(db + j, red[1][j]);
        if (dcol) atomicAdd(dcol + j, red[2][j]);
    }
}

// Embedding backward over a chunk: thread (t, j) sums dH over the samples of
// its split (grid.y), one atomic per thread.
__global__ void embed_bwd_split_kernel(const float *__restrict__ dH, const int8_t *__restrict__ spins,
                                       int Bc, int N, int D, int dt, int per_split,
                                       float *__restrict__ gtok, float *__restrict__ gpos)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)N * D) return;
    const int t = (int)(i / D), j = (int)(i % D);
    const int b0 = blockIdx.y * per_split, b1 = min(Bc, b0 + per_split);
    if (j >= dt) {
        float s = 0.f;
        for (int b = b0; b < b1; ++b) s += dH[((size_t)b * N + t) * D + j];
        atomicAdd(gpos + (size_t)t * (D - dt) + (j - dt), s);
    } else {
        float s0 = 0.f, s1 = 0.f;
        for (int b = b0; b < b1; ++b) {
            const size_t r = (size_t)b * N + t;
            const float v = dH[r * D + j];
            const int tk = t == 0 ? 0 : (spins[r - 1] + 1) >> 1;
            if (tk) s1 += v; else s0 += v;
        }
        atomicAdd(gtok + j, s0);
        atomicAdd(gtok + dt + j, s1);
    }
}

// LayerNorm backward for D = 32 VPL (VPL values per lane, contiguous, vector
// loads): dX = dres + rs (dY g - m1 - xhat m2) (dres may be null), with
// m1 = mean(dY g), m2 = mean(dY g xhat); dg += sum dY xhat, db += sum dY.
// A warp walks RPW rows at a time so that their loads are in flight together;
// per-lane partials of dg, db are reduced per block and added with atomics.
template <int VPL>
__device__ __forceinline__ void ld_vec(const float *p, float (&v)[VPL])
{
    if (VPL % 4 == 0) {
#pragma unroll
        for (int c = 0; c < VPL / 4; ++c) {
            const float4 x = *reinterpret_cast<const float4 *>(p + 4 * c);
            v[4 * c] = x.x; v[4 * c + 1] = x.y; v[4 * c + 2] = x.z; v[4 * c + 3] = x.w;
        }
    } else if (VPL % 2 == 0) {
#pragma unroll
        for (int c = 0; c < VPL / 2; ++c) {
            const float2 x = *reinterpret_cast<const float2 *>(p + 2 * c);
            v[2 * c] = x.x; v[2 * c + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int c = 0; c < VPL; ++c) v[c] = p[c];
    }
}

template <int VPL>
__device__ __forceinline__ void st_vec(float *p, const float (&v)[VPL])
{
    if (VPL % 4 == 0) {
#pragma unroll
        for (int c = 0; c < VPL / 4; ++c)
            *reinterpret_cast<float4 *>(p + 4 * c) = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    } else if (VPL % 2 == 0) {
#pragma unroll
        for (int c = 0; c < VPL / 2; ++c)
            *reinterpret_cast<float2 *>(p + 2 * c) = make_float2(v[2 * c], v[2 * c + 1]);
    } else {
#pragma unroll
        for (int c = 0; c < VPL; ++c) p[c] = v[c];
    }
}

template <int VPL, int RPW>
__global__ void __launch_bounds__(256)
ln_bwd_rows_kernel(const float *__restrict__ dY, const float *__restrict__ X,
                   const float *__restrict__ mu, const float *__restrict__ rs,
                   const float *__restrict__ g, const float *__restrict__ dres,
                   float *__restrict__ dX, float *__restrict__ dg, float *__restrict__ db, int64_t R)
{
    constexpr int D = 32 * VPL;
    __shared__ float red[2][D];
    for (int j = threadIdx.x; j < 2 * D; j += blockDim.x) (&red[0][0])[j] = 0.f;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float gl[VPL], pg[VPL], pb[VPL];
    ld_vec<VPL>(g + lane * VPL, gl);
#pragma unroll
    for (int j = 0; j < VPL; ++j) pg[j] = pb[j] = 0.f;
    __syncthreads();
    for (int64_t r0 = gw * RPW; r0 < R; r0 += nw * RPW) {
        float x[RPW][VPL], dy[RPW][VPL], m[RPW], s[RPW], m1[RPW], m2[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int64_t r = r0 + q < R ? r0 + q : R - 1;  // duplicate a row past the end, never stored
            m[q] = mu[r];
            s[q] = rs[r];
            ld_vec<VPL>(X + r * D + lane * VPL, x[q]);
            ld_vec<VPL>(dY + r * D + lane * VPL, dy[q]);
        }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            float a = 0.f, b = 0.f;
#pragma unroll
            for (int j = 0; j < VPL; ++j) {
                x[q][j] = (x[q][j] - m[q]) * s[q];  // xhat
                const float dxh = dy[q][j] * gl[j];
                a += dxh;
                b += dxh * x[q][j];
            }
            m1[q] = a;
            m2[q] = b;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1)
#pragma unroll
            for (int q = 0; q < RPW; ++q) {
                m1[q] += __shfl_xor_sync(0xffffffffu, m1[q], o);
                m2[q] += __shfl_xor_sync(0xffffffffu, m2[q], o);
            }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            if (r0 + q >= R) break;
            const int64_t r = r0 + q;
            float out[VPL];
            if (dres) ld_vec<VPL>(dres + r * D + lane * VPL, out);
            else {
#pragma unroll
                for (int j = 0; j < VPL; ++j) out[j] = 0.f;
            }
#pragma unroll
            for (int j = 0; j < VPL; ++j) {
                out[j] += s[q] * (dy[q][j] * gl[j] - m1[q] * (1.0f / D) - x[q][j] * m2[q] * (1.0f / D));
                pg[j] += dy[q][j] * x[q][j];
                pb[j] += dy[q][j];
            }
            st_vec<VPL>(dX + r * D + lane * VPL, out);
        }
    }
#pragma unroll
    for (int j = 0; j < VPL; ++j) {
        atomicAdd(&red[0][lane * VPL + j], pg[j]);
        atomicAdd(&red[1][lane * VPL + j], pb[j]);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < D; j += blockDim.x) {
        atomicAdd(dg + j, red[0][j]);
        atomicAdd(db + j, red[1][j]);
    }
}

// ---------------------------------------------------------------------------
// GEMM C[M][N] = A[M][K] * B[K][N] (+bias) with a fused epilogue.  64x64 block
// tile, 16-deep k tiles, 4x4 outputs per thread.  K, N, lda, ldb multiples of 4.
// ---------------------------------------------------------------------------
enum { G_STORE = 0, G_GELU = 1, G_ADDRES = 2, G_GELU_BWD = 3, G_GELU_ONLY = 4 };

template <int EPI>
__global__ void __launch_bounds__(256)
gemm_nn_kernel(const float *__restrict__ A, int lda, const float *__restrict__ Bm, int ldb,
               const float *__restrict__ bias, float *__restrict__ C, int ldc,
               const float *__restrict__ aux, int ldaux, float *__restrict__ aux_out, int64_t M,
               int N, int K)
{
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    // one-dimensional grid, column tile fastest: consecutive blocks share a
    // row tile of A, and M / 64 may exceed the 65535 limit of grid.y
    const int nt = (N + 63) / 64;
    const int64_t m0 = (int64_t)(blockIdx.x / nt) * 64;
    const int n0 = (int)(blockIdx.x % nt) * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        {   // A tile: 64 rows x 16 k, stored transposed
            const int row = tid >> 2, kq = (tid & 3) * 4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (m0 + row < M && k0 + kq < K)
                v = *reinterpret_cast<const float4 *>(A + (m0 + row) * lda + k0 + kq);
            As[kq + 0][row] = v.x;
            As[kq + 1][row] = v.y;
            As[kq + 2][row] = v.z;
            As[kq + 3][row] = v.w;
        }
        {   // B tile: 16 k x 64 cols
            const int kk = tid >> 4, col = (tid & 15) * 4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k0 + kk < K && n0 + col < N)
                v = *reinterpret_cast<const float4 *>(Bm + (size_t)(k0 + kk) * ldb + n0 + col);
            *reinterpret_cast<float4 *>(&Bs[kk][col]) = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = m0 + ty * 4 + i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = n0 + tx * 4 + j;
            if (c >= N) continue;
            float v = acc[i][j] + (bias ? bias[c] : 0.f);
            if (EPI == G_STORE) {
                C[r * ldc + c] = v;
            } else if (EPI == G_GELU) {
                aux_out[r * ldaux + c] = v;
                C[r * ldc + c] = gelu_f(v);
            } else if (EPI == G_GELU_ONLY) {
                C[r * ldc + c] = gelu_f(v);
            } else if (EPI == G_ADDRES) {
                C[r * ldc + c] = aux[r * ldaux + c] + v;
            } else {  // G_GELU_BWD
                C[r * ldc + c] = v * gelu_grad_f(aux[r * ldaux + c]);
            }
        }
    }
}

// C[N1][N2] += sum_r A[r][i] * B[r][j] over rows [0, M): weight gradients.
__global__ void __launch_bounds__(256)
gemm_tn_acc_kernel(const float *__restrict__ A, int lda, const float *__restrict__ Bm, int ldb,
                   float *__restrict__ C, int64_t M, int N1, int N2, int64_t rows_per_block)
{
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    const int64_t rb = (int64_t)blockIdx.z * rows_per_block;
    const int64_t re = rb + rows_per_block < M ? rb + rows_per_block : M;
    float acc[4][4] = {};
    for (int64_t r0 = rb; r0 < re; r0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            const int rr = e >> 6, cc = e & 63;
            const int64_t r = r0 + rr;
            As[rr][cc] = (r < re && i0 + cc < N1) ? A[r * lda + i0 + cc] : 0.f;
            Bs[rr][cc] = (r < re && j0 + cc < N2) ? Bm[r * ldb + j0 + cc] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            const int ii = i0 + ty * 4 + i, jj = j0 + tx * 4 + j;
            if (ii < N1 && jj < N2) atomicAdd(C + (size_t)ii * N2 + jj, acc[i][j]);
        }
}

// out[j] += sum_r A[r][j]
__global__ void colsum_kernel(const float *__restrict__ A, int lda, int64_t M, int N,
                              float *__restrict__ out, int64_t rows_per_block)
{
    __shared__ float red[8][33];
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int64_t rb = (int64_t)blockIdx.y * rows_per_block;
    const int64_t re = rb + rows_per_block < M ? rb + rows_per_block : M;
    float s = 0.f;
    if (j < N)
        for (int64_t r = rb + threadIdx.y; r < re; r += 8) s += A[r * lda + j];
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && j < N) {
        float t = 0.f;
        for (int y = 0; y < 8; ++y) t += red[y][threadIdx.x];
        atomicAdd(out + j, t);
    }
}

// ---------------------------------------------------------------------------
// Masked attention over a whole sequence.  One warp per (sample, head, tile
// of 32 queries); lane = query.  Keys are read as warp-uniform broadcasts.
// QKV rows: [q | k | v], head-major inside each block of D.
// Writes O (attention output), Hmid = Hin + O, and LSE per (row, head).
// ---------------------------------------------------------------------------
template <int DH>
__global__ void attn_fwd_kernel(const float *__restrict__ QKV, const float *__restrict__ Hin,
                                float *__restrict__ O, float *__restrict__ Hmid,
                                float *__restrict__ LSE, int Bc, int N, int D, int NH, int mask,
                                int W, int S)
{
    const int warp_g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int ntile = (N + 31) >> 5;
    if (warp_g >= Bc * NH * ntile) return;
    const int tile = warp_g % ntile, hh = (warp_g / ntile) % NH, b = warp_g / (ntile * NH);
    const int t = tile * 32 + lane;
    const bool active = t < N;
    const int tq = active ? t : N - 1;
    const size_t rq = (size_t)b * N + tq;
    const float scale = rsqrtf((float)DH);
    float q[DH], acc[DH];
#pragma unroll
    for (int j = 0; j < DH; ++j) {
        q[j] = QKV[rq * 3 * D + hh * DH + j] * scale;
        acc[j] = 0.f;
    }
    float mx = -INFINITY, den = 0.f;
    const int t_first = tile * 32, t_last = min(N - 1, tile * 32 + 31);
    // union of visible keys of the tile: [0, min(S, t_last+1)) U [max(S, t_first-W), t_last]
    int ns, blo_first, ns2, blo2;
    visible_ranges(mask, W, S, t_last, ns, blo2);
    visible_ranges(mask, W, S, t_first, ns2, blo_first);
    if (mask == SG_MASK_DENSE) { ns = 0; blo_first = 0; }
    const int nk = ns + band_count(t_last, blo_first);
    for (int i = 0; i < nk; ++i) {
        const int k = i < ns ? i : blo_first + (i - ns);
        if (i >= ns && k < ns) continue;  // already covered by the sink part
        const float *kp = QKV + ((size_t)b * N + k) * 3 * D + D + hh * DH;
        float sc = 0.f;
#pragma unroll
        for (int j = 0; j < DH; ++j) sc += q[j] * kp[j];
        if (!key_visible(mask, W, S, tq, k)) continue;
        const float mn = fmaxf(mx, sc);
        const float corr = expf(mx - mn), p = expf(sc - mn);
        mx = mn;
        den = den * corr + p;
        const float *vp = kp + D;
#pragma unroll
        for (int j = 0; j < DH; ++j) acc[j] = acc[j] * corr + p * vp[j];
    }
    if (!active) return;
    const float inv = 1.0f / den;
#pragma unroll
    for (int j = 0; j < DH; ++j) {
        const size_t idx = rq * D + hh * DH + j;
        const float o = acc[j] * inv;
        O[idx] = o;
        Hmid[idx] = Hin[idx] + o;
    }
    LSE[rq * NH + hh] = mx + logf(den);
}

// dQ and Dt = dO . O per (row, head); lane = query.
template <int DH>
__global__ void attn_bwd_q_kernel(const float *__restrict__ QKV, const float *__restrict__ O,
                                  const float *__restrict__ dO, const float *__restrict__ LSE,
                                  float *__restrict__ dQKV, float *__restrict__ Dt, int Bc, int N,
                                  int D, int NH, int mask, int W, int S)
{
    const int warp_g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int ntile = (N + 31) >> 5;
    if (warp_g >= Bc * NH * ntile) return;
    const int tile = warp_g % ntile, hh = (warp_g / ntile) % NH, b = warp_g / (ntile * NH);
    const int t = tile * 32 + lane;
    const bool active = t < N;
    const int tq = active ? t : N - 1;
    const size_t rq = (size_t)b * N + tq;
    const float scale = rsqrtf((float)DH);
    float q[DH], dq[DH], go[DH];
    float dd = 0.f;
#pragma unroll
    for (int j = 0; j < DH; ++j) {
        q[j] = QKV[rq * 3 * D + hh * DH + j] * scale;
        go[j] = dO[rq * D + hh * DH + j];
        dd += go[j] * O[rq * D + hh * DH + j];
        dq[j] = 0.f;
    }
    const float lse = LSE[rq * NH + hh];
    const int t_first = tile * 32, t_last = min(N - 1, tile * 32 + 31);
    int ns, blo_first, ns2, blo2;
    visible_ranges(mask, W, S, t_last, ns, blo2);
    visible_ranges(mask, W, S, t_first, ns2, blo_first);
    if (mask == SG_MASK_DENSE) { ns = 0; blo_first = 0; }
    const int nk = ns + band_count(t_last, blo_first);
    for (int i = 0; i < nk; ++i) {
        const int k = i < ns ? i : blo_first + (i - ns);
        if (i >= ns && k < ns) continue;
        const float *kp = QKV + ((size_t)b * N + k) * 3 * D + D + hh * DH;
        const float *vp = kp + D;
        float sc = 0.f, dp = 0.f;
#pragma unroll
        for (int j = 0; j < DH; ++j) {
            sc += q[j] * kp[j];
            dp += go[j] * vp[j];
        }
        if (!key_visible(mask, W, S, tq, k)) continue;
        const float ds = expf(sc - lse) * (dp - dd) * scale;
#pragma unroll
        for (int j = 0; j < DH; ++j) dq[j] += ds * kp[j];
    }
    if (!active) return;
#pragma unroll
    for (int j = 0; j < DH; ++j) dQKV[rq * 3 * D + hh * DH + j] = dq[j];
    Dt[rq * NH + hh] = dd;
}

// dK, dV per (row, head); lane = key; loops over the queries that see the key.
template <int DH>
__global__ void attn_bwd_kv_kernel(const float *__restrict__ QKV, const float *__restrict__ dO,
                                   const float *__restrict__ LSE, const float *__restrict__ Dt,
                                   float *__restrict__ dQKV, int Bc, int N, int D, int NH,
                                   int mask, int W, int S)
{
    const int warp_g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int ntile = (N + 31) >> 5;
    if (warp_g >= Bc * NH * ntile) return;
    const int tile = warp_g % ntile, hh = (warp_g / ntile) % NH, b = warp_g / (ntile * NH);
    const int k = tile * 32 + lane;
    const bool active = k < N;
    const int kk = active ? k : N - 1;
    const size_t rk = (size_t)b * N + kk;
    const float scale = rsqrtf((float)DH);
    float key[DH], val[DH], dk[DH], dv[DH];
#pragma unroll
    for (int j = 0; j < DH; ++j) {
        key[j] = QKV[rk * 3 * D + D + hh * DH + j];
        val[j] = QKV[rk * 3 * D + 2 * D + hh * DH + j];
        dk[j] = dv[j] = 0.f;
    }
    const int k_first = tile * 32, k_last = min(N - 1, tile * 32 + 31);
    // queries that see some key of the tile: t in [k_first, t_hi]
    int t_hi = N - 1;
    if (mask == SG_MASK_BAND_SINK && k_first >= S) t_hi = min(N - 1, k_last + W);
    for (int t = k_first; t <= t_hi; ++t) {
        const size_t rq = (size_t)b * N + t;
        const float *qp = QKV + rq * 3 * D + hh * DH;
        const float *gp = dO + rq * D + hh * DH;
        float sc = 0.f, dp = 0.f;
#pragma unroll
        for (int j = 0; j < DH; ++j) {
            sc += qp[j] * key[j];
            dp += gp[j] * val[j];
        }
        if (!key_visible(mask, W, S, t, kk)) continue;
        const float p = expf(sc * scale - LSE[rq * NH + hh]);
        const float ds = p * (dp - Dt[rq * NH + hh]) * scale;
#pragma unroll
        for (int j = 0; j < DH; ++j) {
            dk[j] += ds * qp[j];
            dv[j] += p * gp[j];
        }
    }
    if (!active) return;
#pragma unroll
    for (int j = 0; j < DH; ++j) {
        dQKV[rk * 3 * D + D + hh * DH + j] = dk[j];
        dQKV[rk * 3 * D + 2 * D + hh * DH + j] = dv[j];
    }
}

// ---------------------------------------------------------------------------
// Output head: LN_f -> z = Wh y + bh -> l = z1 - z0 -> lp = log sigmoid(s l).
// ---------------------------------------------------------------------------
__global__ void head_fwd_kernel(const float *__restrict__ H, const float *__restrict__ g,
                                const float *__restrict__ bb, const float *__restrict__ Wh,
                                const float *__restrict__ bh, const int8_t *__restrict__ spins,
                                float *__restrict__ Y, float *__restrict__ mu,
                                float *__restrict__ rs, float *__restrict__ ell,
                                float *__restrict__ lp, int64_t R, int D)
{
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= R) return;
    const float *x = H + r * D;
    float s = 0.f;
    for (int j = lane; j < D; j += 32) s += x[j];
    const float mean = wsum(s) / D;
    float q = 0.f;
    for (int j = lane; j < D; j += 32) {
        const float dv = x[j] - mean;
        q += dv * dv;
    }
    const float r_s = 1.0f / sqrtf(wsum(q) / D + 1e-5f);
    float z0 = 0.f, z1 = 0.f;
    for (int j = lane; j < D; j += 32) {
        const float y = (x[j] - mean) * r_s * g[j] + bb[j];
        if (Y) Y[r * D + j] = y;
        z0 += y * Wh[j];
        z1 += y * Wh[D + j];
    }
    z0 = wsum(z0) + bh[0];
    z1 = wsum(z1) + bh[1];
    if (lane == 0) {
        const float l = z1 - z0;
        if (ell) ell[r] = l;
        if (mu) {
            mu[r] = mean;
            rs[r] = r_s;
        }
        lp[r] = log_sigmoid_f((float)spins[r] * l);
    }
}

// dY of the head for row r, then LN_f backward into dH; head weight grads.
// Per-warp register partial sums (D <= 512), one shared reduction per block.
__global__ void head_bwd_kernel(const float *__restrict__ H, const float *__restrict__ mu,
                                const float *__restrict__ rs, const float *__restrict__ Y,
                                const float *__restrict__ ell, const int8_t *__restrict__ spins,
                                const float *__restrict__ coeff, const float *__restrict__ g,
                                const float *__restrict__ Wh, float *__restrict__ dH,
                                float *__restrict__ gWh, float *__restrict__ gbh,
                                float *__restrict__ glnfg, float *__restrict__ glnfb, int64_t R,
                                int N, int D, int rows_per_block)
{
    extern __shared__ float red[];  // [4][D] + 2: Wh0, Wh1, lnf_g, lnf_b, bh
    for (int j = threadIdx.x; j < 4 * D + 2; j += blockDim.x) red[j] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    float pw0[16], pw1[16], pg[16], pb[16], pz0 = 0.f, pz1 = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) pw0[i] = pw1[i] = pg[i] = pb[i] = 0.f;
    for (int64_t r = r0 + warp; r < R && r < r0 + rows_per_block; r += nw) {
        const float sg = (float)spins[r];
        const float c = coeff[r / N];
        const float dl = c * sg / (1.0f + expf(sg * ell[r]));  // c s sigmoid(-s l)
        const float dz0 = -dl, dz1 = dl;
        const float m = mu[r], s = rs[r];
        float m1 = 0.f, m2 = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int j = lane + 32 * i;
            if (j >= D) break;
            const float y = Y[r * D + j];
            pw0[i] += dz0 * y;
            pw1[i] += dz1 * y;
            const float dy = dz0 * Wh[j] + dz1 * Wh[D + j];
            const float xh = (H[r * D + j] - m) * s;
            pg[i] += dy * xh;
            pb[i] += dy;
            const float dxh = dy * g[j];
            m1 += dxh;
            m2 += dxh * xh;
        }
        m1 = wsum(m1) / D;
        m2 = wsum(m2) / D;
        for (int j = lane; j < D; j += 32) {
            const float dy = dz0 * Wh[j] + dz1 * Wh[D + j];
            const float xh = (H[r * D + j] - m) * s;
            dH[r * D + j] = s * (dy * g[j] - m1 - xh * m2);
        }
        pz0 += dz0;
        pz1 += dz1;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int j = lane + 32 * i;
        if (j >= D) break;
        atomicAdd(red + j, pw0[i]);
        atomicAdd(red + D + j, pw1[i]);
        atomicAdd(red + 2 * D + j, pg[i]);
        atomicAdd(red + 3 * D + j, pb[i]);
    }
    if (lane == 0) {
        atomicAdd(red + 4 * D, pz0);
        atomicAdd(red + 4 * D + 1, pz1);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < D; j += blockDim.x) {
        atomicAdd(gWh + j, red[j]);
        atomicAdd(gWh + D + j, red[D + j]);
        atomicAdd(glnfg + j, red[2 * D + j]);
        atomicAdd(glnfb + j, red[3 * D + j]);
    }
    if (threadIdx.x < 2) atomicAdd(gbh + threadIdx.x, red[4 * D + threadIdx.x]);
}

// logq[b] = sum_t lp[b*N + t], fixed-order tree reduction per sample.
__global__ void seg_sum_kernel(const float *__restrict__ lp, int N, float *__restrict__ logq)
{
    __shared__ float red[256];
    const int b = blockIdx.x;
    float s = 0.f;
    for (int t = threadIdx.x; t < N; t += blockDim.x) s += lp[(size_t)b * N + t];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) logq[b] = red[0];
}

unsigned blocks_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

// ---------------------------------------------------------------------------
// Host-side orchestration.
// ---------------------------------------------------------------------------
struct LayerBufs {
    float *Hin, *mu1, *rs1, *A1, *QKV, *O, *LSE, *Hmid, *mu2, *rs2, *A2, *F1, *G;
    // tensor-core path: tiled BF16 operands kept for the backward
    unsigned char *A1t, *A2t, *Gt, *F1t;  // F1t holds gelu'(F1), the GELU derivative
};

// The BF16 model runs its teacher-forced GEMMs on tcgen05 (every output
// width a multiple of 32).
bool use_tc(const sg_config &c)
{
    return c.precision == SG_BF16 && c.d % 32 == 0 && c.d_ff % 32 == 0;
}

// out[j] += sum_r T[r][j] over a wide BF16 matrix W(R, F)
__global__ void colsum_tiled_kernel(const unsigned char *__restrict__ T, int64_t R, int F,
                                    float *__restrict__ out, int64_t rows_per_block)
{
    __shared__ float red[8][33];
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int64_t rb0 = (int64_t)blockIdx.y * rows_per_block;
    const int64_t re = rb0 + rows_per_block < R ? rb0 + rows_per_block : R;
    float s = 0.f;
    if (j < F)
        for (int64_t r = rb0 + threadIdx.y; r < re; r += 8) {
            const uint16_t b = *reinterpret_cast<const uint16_t *>(T + wl_offset(r, j, F));
            s += __uint_as_float((uint32_t)b << 16);
        }
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && j < F) {
        float t = 0.f;
        for (int y = 0; y < 8; ++y) t += red[y][threadIdx.x];
        atomicAdd(out + j, t);
    }
}

struct Plan {
    int64_t Bc;       // samples per chunk
    int64_t R;        // rows per chunk
    bool keep;        // keep every layer (backward) or reuse one set
};

// ---------------------------------------------------------------------------
// Shared-memory attention: one CTA per (sample, head) stages the head's rows
// of the sequence in padded shared memory (row stride DH + 4 floats, an odd
// number of 16-byte units, so 16-byte row reads by 32 different rows are
// conflict-free) and walks the visible keys there.
// ---------------------------------------------------------------------------
template <int DH>
__device__ __forceinline__ void stage_rows(float *dst, const float *__restrict__ src, int N,
                                           int stride_src)
{
    constexpr int DP = DH + 4;
    for (int e = threadIdx.x; e < N * (DH / 4); e += blockDim.x) {
        const int t = e / (DH / 4), c = e % (DH / 4);
        *reinterpret_cast<float4 *>(dst + t * DP + 4 * c) =
            *reinterpret_cast<const float4 *>(src + (size_t)t * stride_src + 4 * c);
    }
}

// Shared-memory row (16-byte aligned) into registers with 128-bit loads.
template <int DH>
__device__ __forceinline__ void row_regs(const float *row, float (&r)[DH])
{
#pragma unroll
    for (int c = 0; c < DH / 4; ++c) {
        const float4 x = *reinterpret_cast<const float4 *>(row + 4 * c);
        r[4 * c] = x.x;
        r[4 * c + 1] = x.y;
        r[4 * c + 2] = x.z;
        r[4 * c + 3] = x.w;
    }
}

template <int DH>
__device__ __forceinline__ float dot_regs(const float (&a)[DH], const float (&b)[DH])
{
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int j = 0; j < DH; j += 2) {
        s0 += a[j] * b[j];
        s1 += a[j + 1] * b[j + 1];
    }
    return s0 + s1;
}

// Rows staged in shared memory as FP32 (FP32 model) or BF16 (BF16 model:
// half the shared-memory bytes per row read; values as the tensor-core paths
// see them).  Row pitch in elements: FP32 DH + 4, BF16 DH + 8 (24 for DH = 8),
// so 8 consecutive rows' 16-byte pieces fall in distinct banks.
template <int DH, typename TS>
struct Pitch {
    static constexpr int value = sizeof(TS) == 4 ? DH + 4 : (DH == 8 ? 24 : DH + 8);
};

template <int DH, typename TS>
__device__ __forceinline__ void stage_rows_t(TS *dst, const float *__restrict__ src, int N,
                                             int stride_src)
{
    constexpr int DP = Pitch<DH, TS>::value;
    if constexpr (sizeof(TS) == 4) {
        for (int e = threadIdx.x; e < N * (DH / 4); e += blockDim.x) {
            const int t = e / (DH / 4), c = e % (DH / 4);
            *reinterpret_cast<float4 *>(dst + t * DP + 4 * c) =
                *reinterpret_cast<const float4 *>(src + (size_t)t * stride_src + 4 * c);
        }
    } else {
        for (int e = threadIdx.x; e < N * (DH / 8); e += blockDim.x) {
            const int t = e / (DH / 8), c = e % (DH / 8);
            const float4 a = *reinterpret_cast<const float4 *>(src + (size_t)t * stride_src + 8 * c);
            const float4 b = *reinterpret_cast<const float4 *>(src + (size_t)t * stride_src + 8 * c + 4);
            __nv_bfloat162 h[4] = {__floats2bfloat162_rn(a.x, a.y), __floats2bfloat162_rn(a.z, a.w),
                                   __floats2bfloat162_rn(b.x, b.y), __floats2bfloat162_rn(b.z, b.w)};
            *reinterpret_cast<uint4 *>(dst + t * DP + 8 * c) = *reinterpret_cast<const uint4 *>(h);
        }
    }
}

// Rows copied as they are (BF16 -> BF16 or FP32 -> FP32) by cp.async, 16
// bytes per copy; the caller waits (cp_async_wait<0>) before the barrier.
// Row pitch DPS elements; 16-byte aligned rows on both sides.
template <int DH, int DPS, typename T>
__device__ __forceinline__ void stage_rows_async(T *dst, const T *__restrict__ src, int N, int stride_src)
{
    constexpr int PIECES = DH * (int)sizeof(T) / 16;  // 16-byte pieces per row
    constexpr int PER = 16 / (int)sizeof(T);          // elements per piece
    for (int e = threadIdx.x; e < N * PIECES; e += blockDim.x) {
        const int t = e / PIECES, c = e % PIECES;
        tc::cp_async16(dst + t * DPS + PER * c, src + (size_t)t * stride_src + PER * c);
    }
}

// Rows of a BF16 row-major source (16-byte pieces) into the staged layout:
// copied as they are (BF16 staging) or widened (FP32 staging).
template <int DH, typename TS>
__device__ __forceinline__ void stage_rows_h(TS *dst, const __nv_bfloat16 *__restrict__ src, int N,
                                             int stride_src)
{
    constexpr int DP = sizeof(TS) == 4 ? DH + 4 : Pitch<DH, TS>::value;
    for (int e = threadIdx.x; e < N * (DH / 8); e += blockDim.x) {
        const int t = e / (DH / 8), c = e % (DH / 8);
        const uint4 x = *reinterpret_cast<const uint4 *>(src + (size_t)t * stride_src + 8 * c);
        if constexpr (sizeof(TS) == 2) {
            *reinterpret_cast<uint4 *>(dst + t * DP + 8 * c) = x;
        } else {
            const uint32_t w[4] = {x.x, x.y, x.z, x.w};
            float *d = reinterpret_cast<float *>(dst) + t * DP + 8 * c;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                d[2 * j] = __uint_as_float(w[j] << 16);
                d[2 * j + 1] = __uint_as_float(w[j] & 0xffff0000u);
            }
        }
    }
}

template <int DH>
__device__ __forceinline__ void row_regs_t(const float *row, float (&r)[DH])
{
    row_regs<DH>(row, r);
}

template <int DH>
__device__ __forceinline__ void row_regs_t(const __nv_bfloat16 *row, float (&r)[DH])
{
#pragma unroll
    for (int c = 0; c < DH / 8; ++c) {
        const uint4 x = *reinterpret_cast<const uint4 *>(row + 8 * c);
        const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            r[8 * c + 2 * j] = __uint_as_float(w[j] << 16);
            r[8 * c + 2 * j + 1] = __uint_as_float(w[j] & 0xffff0000u);
        }
    }
}

template <int DH>
__device__ __forceinline__ float dot_row(const float *q, const float *row)
{
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < DH / 4; ++c) {
        const float4 k = *reinterpret_cast<const float4 *>(row + 4 * c);
        s += q[4 * c] * k.x + q[4 * c + 1] * k.y + q[4 * c + 2] * k.z + q[4 * c + 3] * k.w;
    }
    return s;
}

// Packed FP32 arithmetic (fma.rn.f32x2 on sm_100 and later): a row of DH
// values as DH / 2 pairs.  The dot product keeps the even and the odd
// products in the two halves and adds them at the end.
template <int DH>
__device__ __forceinline__ void row_pairs(const float *row, float2 (&r)[DH / 2])
{
#pragma unroll
    for (int c = 0; c < DH / 4; ++c) {
        const float4 x = *reinterpret_cast<const float4 *>(row + 4 * c);
        r[2 * c] = make_float2(x.x, x.y);
        r[2 * c + 1] = make_float2(x.z, x.w);
    }
}

template <int DH>
__device__ __forceinline__ void row_pairs(const __nv_bfloat16 *row, float2 (&r)[DH / 2])
{
#pragma unroll
    for (int c = 0; c < DH / 8; ++c) {
        const uint4 x = *reinterpret_cast<const uint4 *>(row + 8 * c);
        const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
            r[4 * c + j] = make_float2(__uint_as_float(w[j] << 16), __uint_as_float(w[j] & 0xffff0000u));
    }
}

template <int DH>
__device__ __forceinline__ float dot_pairs(const float2 (&a)[DH / 2], const float2 (&b)[DH / 2])
{
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < DH / 2; ++j) s = __ffma2_rn(a[j], b[j], s);
    return s.x + s.y;
}

// acc += w b, pairwise
template <int DH>
__device__ __forceinline__ void axpy_pairs(float2 (&acc)[DH / 2], float w, const float2 (&b)[DH / 2])
{
    const float2 w2 = make_float2(w, w);
#pragma unroll
    for (int j = 0; j < DH / 2; ++j) acc[j] = __ffma2_rn(w2, b[j], acc[j]);
}

template <int DH, typename TS>
__global__ void __launch_bounds__(256)
attn_fwd_smem_kernel(const float *__restrict__ QKV, const float *__restrict__ Hin,
                     float *__restrict__ O, float *__restrict__ Hmid, float *__restrict__ LSE,
                     int N, int D, int NH, int mask, int W, int S,
                     const __nv_bfloat16 *__restrict__ QKVh)
{
    constexpr int DP = DH + 4, DPS = Pitch<DH, TS>::value;
    extern __shared__ float4 sm4[];
    float *Qs = reinterpret_cast<float *>(sm4);  // Q in, attention output out (FP32)
    TS *Ks = reinterpret_cast<TS *>(Qs + N * DP);
    TS *Vs = Ks + N * DPS;
    const int b = blockIdx.x / NH, hh = blockIdx.x % NH;
    if (QKVh) {  // QKV rows in BF16: K, V copied asynchronously, Q widened
        const __nv_bfloat16 *hb = QKVh + (size_t)b * N * 3 * D;
        if constexpr (sizeof(TS) == 2) {
            stage_rows_async<DH, DPS>(Ks, hb + D + hh * DH, N, 3 * D);
            stage_rows_async<DH, DPS>(Vs, hb + 2 * D + hh * DH, N, 3 * D);
            tc::cp_async_commit();
        } else {
            stage_rows_h<DH, TS>(Ks, hb + D + hh * DH, N, 3 * D);
            stage_rows_h<DH, TS>(Vs, hb + 2 * D + hh * DH, N, 3 * D);
        }
        stage_rows_h<DH, float>(Qs, hb + hh * DH, N, 3 * D);
        if constexpr (sizeof(TS) == 2) tc::cp_async_wait<0>();
    } else {
        const float *base = QKV + (size_t)b * N * 3 * D;
        stage_rows<DH>(Qs, base + hh * DH, N, 3 * D);
        stage_rows_t<DH, TS>(Ks, base + D + hh * DH, N, 3 * D);
        stage_rows_t<DH, TS>(Vs, base + 2 * D + hh * DH, N, 3 * D);
    }
    __syncthreads();
    const float scale = rsqrtf((float)DH);
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        const size_t r = (size_t)b * N + t;
        float2 q[DH / 2], acc[DH / 2];
        row_pairs<DH>(Qs + t * DP, q);
#pragma unroll
        for (int j = 0; j < DH / 2; ++j) {
            q[j] = make_float2(q[j].x * scale, q[j].y * scale);
            acc[j] = make_float2(0.f, 0.f);
        }
        int n_sink, band_lo;
        visible_ranges(mask, W, S, t, n_sink, band_lo);
        const int nk = n_sink + band_count(t, band_lo);
        float mx = -INFINITY, den = 0.f;
        for (int i = 0; i < nk; ++i) {
            const int k = i < n_sink ? i : band_lo + (i - n_sink);
            float2 kr[DH / 2], vr[DH / 2];
            row_pairs<DH>(Ks + k * DPS, kr);
            row_pairs<DH>(Vs + k * DPS, vr);
            const float sc = dot_pairs<DH>(q, kr);
            const float mn = fmaxf(mx, sc);
            const float corr = __expf(mx - mn), p = __expf(sc - mn);
            mx = mn;
            den = den * corr + p;
            const float2 c2 = make_float2(corr, corr), p2 = make_float2(p, p);
#pragma unroll
            for (int j = 0; j < DH / 2; ++j) acc[j] = __ffma2_rn(p2, vr[j], __fmul2_rn(acc[j], c2));
        }
        const float inv = 1.0f / den;
#pragma unroll
        for (int j = 0; j < DH / 2; ++j)  // own row only
            *reinterpret_cast<float2 *>(Qs + t * DP + 2 * j) = make_float2(acc[j].x * inv, acc[j].y * inv);
        LSE[r * NH + hh] = mx + logf(den);
    }
    __syncthreads();
    // coalesced float4 writes of O and Hmid = Hin + O for this head's columns
    for (int e = threadIdx.x; e < N * (DH / 4); e += blockDim.x) {
        const int t = e / (DH / 4), c = e % (DH / 4);
        const size_t idx = ((size_t)b * N + t) * D + hh * DH + 4 * c;
        const float4 o = *reinterpret_cast<const float4 *>(Qs + t * DP + 4 * c);
        const float4 hin = *reinterpret_cast<const float4 *>(Hin + idx);
        *reinterpret_cast<float4 *>(O + idx) = o;
        *reinterpret_cast<float4 *>(Hmid + idx) =
            make_float4(hin.x + o.x, hin.y + o.y, hin.z + o.z, hin.w + o.w);
    }
}

// Backward of one (sample, head): dQ by query threads; dK, dV of band keys by
// key threads (each sees at most W + 1 queries); sink keys (and every key of
// a dense mask) by warps, lanes striding over the queries with a shuffle
// reduction.
template <int DH, typename TS>
__global__ void __launch_bounds__(256)
attn_bwd_smem_kernel(const float *__restrict__ QKV, const float *__restrict__ O,
                     const float *__restrict__ dO, const float *__restrict__ LSE,
                     float *__restrict__ dQKV, int N, int D, int NH, int mask, int W, int S,
                     unsigned char *__restrict__ dQKVt, float *__restrict__ bsum,
                     const __nv_bfloat16 *__restrict__ QKVh)
{
    constexpr int DP = DH + 4, DPS = Pitch<DH, TS>::value;
    constexpr bool kF32 = sizeof(TS) == 4;
    extern __shared__ float4 sm4[];
    float *Os = reinterpret_cast<float *>(sm4);  // O in; then the dQ, dK, dV rows out
    float *Ls = Os + N * DP;                     // LSE
    float *Ds = Ls + N;                          // D_t = dO_t . O_t
    // FP32 rows for the dV of sink keys (the FP32 model parks them in Vs)
    float *Pk = Ds + N;
    // the staged rows start 16-byte aligned after the FP32 arrays
    const int f32_floats = (N * DP + 2 * N + (kF32 ? 0 : N * DP) + 3) & ~3;
    TS *Qs = reinterpret_cast<TS *>(reinterpret_cast<float *>(sm4) + f32_floats);
    TS *Ks = Qs + N * DPS;
    TS *Vs = Ks + N * DPS;
    TS *Gs = Vs + N * DPS;  // dO
    const int b = blockIdx.x / NH, hh = blockIdx.x % NH;
    bool async = false;
    if (QKVh) {  // QKV rows in BF16
        const __nv_bfloat16 *hb = QKVh + (size_t)b * N * 3 * D;
        if constexpr (sizeof(TS) == 2) {  // copied asynchronously, with O
            stage_rows_async<DH, DPS>(Qs, hb + hh * DH, N, 3 * D);
            stage_rows_async<DH, DPS>(Ks, hb + D + hh * DH, N, 3 * D);
            stage_rows_async<DH, DPS>(Vs, hb + 2 * D + hh * DH, N, 3 * D);
            stage_rows_async<DH, DP>(Os, O + (size_t)b * N * D + hh * DH, N, D);
            tc::cp_async_commit();
            async = true;
        } else {
            stage_rows_h<DH, TS>(Qs, hb + hh * DH, N, 3 * D);
            stage_rows_h<DH, TS>(Ks, hb + D + hh * DH, N, 3 * D);
            stage_rows_h<DH, TS>(Vs, hb + 2 * D + hh * DH, N, 3 * D);
        }
    } else {
        const float *base = QKV + (size_t)b * N * 3 * D;
        stage_rows_t<DH, TS>(Qs, base + hh * DH, N, 3 * D);
        stage_rows_t<DH, TS>(Ks, base + D + hh * DH, N, 3 * D);
        stage_rows_t<DH, TS>(Vs, base + 2 * D + hh * DH, N, 3 * D);
    }
    stage_rows_t<DH, TS>(Gs, dO + (size_t)b * N * D + hh * DH, N, D);
    if (!async) stage_rows<DH>(Os, O + (size_t)b * N * D + hh * DH, N, D);
    for (int t = threadIdx.x; t < N; t += blockDim.x) Ls[t] = LSE[((size_t)b * N + t) * NH + hh];
    if (async) tc::cp_async_wait<0>();
    __syncthreads();
    const float scale = rsqrtf((float)DH);
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        float2 gr[DH / 2], orr[DH / 2];
        row_pairs<DH>(Gs + t * DPS, gr);
        row_pairs<DH>(Os + t * DP, orr);
        Ds[t] = dot_pairs<DH>(gr, orr);
    }
    __syncthreads();
    // out_part 0/1/2 = q/k/v columns of dQKV, from the rows in Os: FP32 rows
    // (coalesced float4), or 16-byte pieces of the wide BF16 copy plus this
    // (sample, head)'s column sums (a slice of the bias gradient) in bsum
    __shared__ float csum[256];
    auto flush = [&](int part) {
        __syncthreads();
        if (dQKVt) {
            for (int e = threadIdx.x; e < N * (DH / 8); e += blockDim.x) {
                const int t = e / (DH / 8), c = e % (DH / 8);
                float v[8];
                ld8(Os + t * DP + 8 * c, v);
                *reinterpret_cast<uint4 *>(dQKVt + wl_offset((int64_t)b * N + t, part * D + hh * DH + 8 * c, 3 * D)) =
                    pack8_bf16(v);
            }
            constexpr int SL = 256 / DH;  // row slices (blockDim.x = 256)
            const int j = threadIdx.x % DH, sl = threadIdx.x / DH;
            float a = 0.f;
            for (int t = sl; t < N; t += SL) a += Os[t * DP + j];
            csum[threadIdx.x] = a;
            __syncthreads();
            if (threadIdx.x < DH) {
                float tot = 0.f;
                for (int q = 0; q < SL; ++q) tot += csum[q * DH + threadIdx.x];
                bsum[(size_t)b * 3 * D + part * D + hh * DH + threadIdx.x] = tot;
            }
        } else {
            for (int e = threadIdx.x; e < N * (DH / 4); e += blockDim.x) {
                const int t = e / (DH / 4), c = e % (DH / 4);
                *reinterpret_cast<float4 *>(dQKV + ((size_t)b * N + t) * 3 * D + part * D + hh * DH + 4 * c) =
                    *reinterpret_cast<const float4 *>(Os + t * DP + 4 * c);
            }
        }
        __syncthreads();
    };
    // dQ_t = scale * sum_k P_tk (dP_tk - D_t) k_k
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        float2 q[DH / 2], g[DH / 2], dq[DH / 2];
        row_pairs<DH>(Qs + t * DPS, q);
        row_pairs<DH>(Gs + t * DPS, g);
#pragma unroll
        for (int j = 0; j < DH / 2; ++j) {
            q[j] = make_float2(q[j].x * scale, q[j].y * scale);
            dq[j] = make_float2(0.f, 0.f);
        }
        const float lse = Ls[t], dd = Ds[t];
        int n_sink, band_lo;
        visible_ranges(mask, W, S, t, n_sink, band_lo);
        const int nk = n_sink + band_count(t, band_lo);
        for (int i = 0; i < nk; ++i) {
            const int k = i < n_sink ? i : band_lo + (i - n_sink);
            float2 kr[DH / 2], vr[DH / 2];  // each row read once, with 128-bit loads
            row_pairs<DH>(Ks + k * DPS, kr);
            row_pairs<DH>(Vs + k * DPS, vr);
            const float p = __expf(dot_pairs<DH>(q, kr) - lse);
            const float ds = p * (dot_pairs<DH>(g, vr) - dd) * scale;
            axpy_pairs<DH>(dq, ds, kr);
        }
#pragma unroll
        for (int j = 0; j < DH / 2; ++j) *reinterpret_cast<float2 *>(Os + t * DP + 2 * j) = dq[j];  // own row
    }
    flush(0);
    // dK and dV.  Keys seen only through the band: one thread per key, up to
    // W + 1 queries each; keys visible to every later query (sink, or all keys
    // when dense): one warp per key, lanes over queries, shuffle reduction.
    // Each key's dV is parked in registers while dK goes out first.
    const int k_band0 = mask == SG_MASK_DENSE ? N : (S < N ? S : N);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    constexpr int KPT = 2;  // band keys per thread kept in registers (N <= 512)
    float2 dv_keep[KPT][DH / 2];
    int kk_i = 0;
    for (int k = k_band0 + threadIdx.x; k < N; k += blockDim.x, ++kk_i) {
        float2 key[DH / 2], val[DH / 2], dk[DH / 2], dv[DH / 2];
        row_pairs<DH>(Ks + k * DPS, key);
        row_pairs<DH>(Vs + k * DPS, val);
#pragma unroll
        for (int j = 0; j < DH / 2; ++j) {
            key[j] = make_float2(key[j].x * scale, key[j].y * scale);
            dk[j] = dv[j] = make_float2(0.f, 0.f);
        }
        const int t_hi = min(N - 1, k + W);
        for (int t = k; t <= t_hi; ++t) {
            float2 qr[DH / 2], gr[DH / 2];
            row_pairs<DH>(Qs + t * DPS, qr);
            row_pairs<DH>(Gs + t * DPS, gr);
            const float p = __expf(dot_pairs<DH>(key, qr) - Ls[t]);
            const float ds = p * (dot_pairs<DH>(val, gr) - Ds[t]) * scale;
            axpy_pairs<DH>(dk, ds, qr);
            axpy_pairs<DH>(dv, p, gr);
        }
#pragma unroll
        for (int j = 0; j < DH / 2; ++j) {
            *reinterpret_cast<float2 *>(Os + k * DP + 2 * j) = dk[j];
            if (kk_i < KPT) dv_keep[kk_i][j] = dv[j];
        }
    }
    for (int k = warp; k < k_band0; k += nw) {
        float2 key[DH / 2], val[DH / 2], dk2[DH / 2], dv2[DH / 2];
        row_pairs<DH>(Ks + k * DPS, key);
        row_pairs<DH>(Vs + k * DPS, val);
#pragma unroll
        for (int j = 0; j < DH / 2; ++j) {
            key[j] = make_float2(key[j].x * scale, key[j].y * scale);
            dk2[j] = dv2[j] = make_float2(0.f, 0.f);
        }
        for (int t = k + lane; t < N; t += 32) {
            float2 qr[DH / 2], gr[DH / 2];
            row_pairs<DH>(Qs + t * DPS, qr);
            row_pairs<DH>(Gs + t * DPS, gr);
            const float p = __expf(dot_pairs<DH>(key, qr) - Ls[t]);
            const float ds = p * (dot_pairs<DH>(val, gr) - Ds[t]) * scale;
            axpy_pairs<DH>(dk2, ds, qr);
            axpy_pairs<DH>(dv2, p, gr);
        }
        float dk[DH], dv[DH];
#pragma unroll
        for (int j = 0; j < DH / 2; ++j) {
            dk[2 * j] = wsum(dk2[j].x);
            dk[2 * j + 1] = wsum(dk2[j].y);
            dv[2 * j] = wsum(dv2[j].x);
            dv[2 * j + 1] = wsum(dv2[j].y);
        }
        // dK to the output buffer; dV parked in row k of Vs (FP32 model: nothing
        // reads it again, the dQ phase is over and key k is owned by this warp)
        // or of the FP32 rows Pk (BF16 model)
        if (lane == 0)
#pragma unroll
            for (int j = 0; j < DH; ++j) {
                Os[k * DP + j] = dk[j];
                if constexpr (kF32) Vs[k * DPS + j] = dv[j];
                else Pk[k * DP + j] = dv[j];
            }
    }
    flush(1);
    // dV: band keys from registers, sink keys from their parked rows in Vs
    kk_i = 0;
    for (int k = k_band0 + threadIdx.x; k < N; k += blockDim.x, ++kk_i)
#pragma unroll
        for (int j = 0; j < DH / 2; ++j)
            *reinterpret_cast<float2 *>(Os + k * DP + 2 * j) = dv_keep[kk_i < KPT ? kk_i : 0][j];
    for (int k = warp; k < k_band0; k += nw)
        if (lane == 0)
#pragma unroll
            for (int j = 0; j < DH; ++j) {
                if constexpr (kF32) Os[k * DP + j] = Vs[k * DPS + j];
                else Os[k * DP + j] = Pk[k * DP + j];
            }
    flush(2);
}

constexpr size_t kAttnSmemMax = 200 * 1024;

template <int DH, typename TS>
size_t attn_bwd_smem_bytes(int N)
{
    // Q, K, V, dO rows (TS) + O/out rows, LSE, D (+ sink dV rows for BF16).
    // The backward keeps at most two band keys' dV per thread in registers,
    // so it serves N <= 512 (256 threads).
    if (N > 512) return (size_t)1 << 40;
    const size_t f32 = (((size_t)(sizeof(TS) == 4 ? 1 : 2) * N * (DH + 4) + 2 * N + 3) & ~(size_t)3) *
                       sizeof(float);
    return f32 + (size_t)4 * N * Pitch<DH, TS>::value * sizeof(TS);
}

template <int DH, typename TS>
void attn_fwd_t(const float *QKV, const float *Hin, float *O, float *Hmid, float *LSE, int Bc,
                const sg_config &c, cudaStream_t st, const __nv_bfloat16 *QKVh)
{
    const size_t fwd_smem = (size_t)c.N * (DH + 4) * sizeof(float) +
                            (size_t)2 * c.N * Pitch<DH, TS>::value * sizeof(TS);
    cudaFuncSetAttribute(attn_fwd_smem_kernel<DH, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fwd_smem);
    attn_fwd_smem_kernel<DH, TS><<<(unsigned)(Bc * c.n_heads), 256, fwd_smem, ::sg::counted(st)>>>(
        QKV, Hin, O, Hmid, LSE, c.N, c.d, c.n_heads, c.mask_kind, c.W, c.S, QKVh);
}

template <int DH>
void attn_fwd(const float *QKV, const float *Hin, float *O, float *Hmid, float *LSE, int Bc,
              const sg_config &c, cudaStream_t st, const __nv_bfloat16 *QKVh)
{
    if (attn_bwd_smem_bytes<DH, float>(c.N) <= kAttnSmemMax) {
        if (c.precision == SG_BF16) attn_fwd_t<DH, __nv_bfloat16>(QKV, Hin, O, Hmid, LSE, Bc, c, st, QKVh);
        else attn_fwd_t<DH, float>(QKV, Hin, O, Hmid, LSE, Bc, c, st, QKVh);
        return;
    }
    const int warps = Bc * c.n_heads * ((c.N + 31) / 32);
    attn_fwd_kernel<DH><<<blocks_for(warps, 8), 256, 0, ::sg::counted(st)>>>(
        QKV, Hin, O, Hmid, LSE, Bc, c.N, c.d, c.n_heads, c.mask_kind, c.W, c.S);
}

// Returns true when the shared-memory kernel wrote the wide copy dQKVt and
// the per-sample bias sums bsum instead of the FP32 dQKV (dQKVt non-null).
template <int DH>
bool attn_bwd(const float *QKV, const float *O, const float *dO, const float *LSE, float *dQKV,
              float *Dt, int Bc, const sg_config &c, cudaStream_t st, unsigned char *dQKVt,
              float *bsum, const __nv_bfloat16 *QKVh)
{
    if (attn_bwd_smem_bytes<DH, float>(c.N) <= kAttnSmemMax) {
        auto go = [&](auto kern, size_t smem) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kern<<<(unsigned)(Bc * c.n_heads), 256, smem, ::sg::counted(st)>>>(
                QKV, O, dO, LSE, dQKV, c.N, c.d, c.n_heads, c.mask_kind, c.W, c.S, dQKVt, bsum, QKVh);
        };
        if (c.precision == SG_BF16)
            go(attn_bwd_smem_kernel<DH, __nv_bfloat16>, attn_bwd_smem_bytes<DH, __nv_bfloat16>(c.N));
        else
            go(attn_bwd_smem_kernel<DH, float>, attn_bwd_smem_bytes<DH, float>(c.N));
        return dQKVt != nullptr;
    }
    const int warps = Bc * c.n_heads * ((c.N + 31) / 32);
    attn_bwd_q_kernel<DH><<<blocks_for(warps, 8), 256, 0, ::sg::counted(st)>>>(
        QKV, O, dO, LSE, dQKV, Dt, Bc, c.N, c.d, c.n_heads, c.mask_kind, c.W, c.S);
    attn_bwd_kv_kernel<DH><<<blocks_for(warps, 8), 256, 0, ::sg::counted(st)>>>(
        QKV, dO, LSE, Dt, dQKV, Bc, c.N, c.d, c.n_heads, c.mask_kind, c.W, c.S);
    return false;
}

bool dh_supported(int dh) { return dh == 8 || dh == 16 || dh == 32; }

// The BF16 tensor-core pass writes QKV in BF16 (row-major [R][3 D]) where the
// shared-memory attention kernels serve the shape (they stage K and V, and the
// backward also Q, in BF16 anyway); the tcgen05 attention and the
// global-memory kernels read FP32 QKV.
bool qkv_bf16(const sg_config &c)
{
    const int dh = c.d / c.n_heads;
    if (use_tc(c) && (attn_mma_supported(c) || attn_band_supported(c))) return true;
    if (!use_tc(c) || attn_tc_supported(c) || !dh_supported(dh)) return false;
    const size_t need = dh == 8 ? attn_bwd_smem_bytes<8, float>(c.N)
                      : dh == 16 ? attn_bwd_smem_bytes<16, float>(c.N)
                                 : attn_bwd_smem_bytes<32, float>(c.N);
    return need <= kAttnSmemMax;
}

// keep_o: O is read back by the backward (the MMA path keeps it in BF16 in
// O's buffer, and skips it for a forward-only pass).
void attn_fwd_dispatch(int dh, const float *QKV, const float *Hin, float *O, float *Hmid,
                       float *LSE, int Bc, const sg_config &c, cudaStream_t st, int *err,
                       const __nv_bfloat16 *QKVh = nullptr, bool keep_o = true)
{
    if (QKVh && attn_mma_supported(c) && attn_tmem_supported(c)) {  // many keys per query: tcgen05
        launch_attn_fwd_tmem(c, QKVh, Hin, keep_o ? reinterpret_cast<__nv_bfloat16 *>(O) : nullptr, Hmid,
                             LSE, Bc, err, st);
        return;
    }
    if (QKVh && attn_mma_supported(c)) {  // BF16 QKV: warp-level tensor-core MMAs
        launch_attn_fwd_mma(c, QKVh, Hin, keep_o ? reinterpret_cast<__nv_bfloat16 *>(O) : nullptr, Hmid,
                            LSE, Bc, st);
        return;
    }
    if (QKVh && attn_band_supported(c)) {  // long band sequences: per-tile tcgen05 kernels
        launch_attn_fwd_band(c, QKVh, Hin, keep_o ? reinterpret_cast<__nv_bfloat16 *>(O) : nullptr, Hmid, LSE, Bc,
                             err, st);
        return;
    }
    if (attn_tc_supported(c)) {  // BF16 model: tcgen05 attention
        launch_attn_fwd_tc(c, QKV, Hin, O, Hmid, LSE, Bc, err, st);
        return;
    }
    if (dh == 8) attn_fwd<8>(QKV, Hin, O, Hmid, LSE, Bc, c, st, QKVh);
    else if (dh == 16) attn_fwd<16>(QKV, Hin, O, Hmid, LSE, Bc, c, st, QKVh);
    else attn_fwd<32>(QKV, Hin, O, Hmid, LSE, Bc, c, st, QKVh);
}

// dQKV of one layer: FP32 rows, or (returns true) the wide BF16 copy dQKVt
// and per-sample bias sums bsum [Bc][3 D] where the kernel fuses them.
bool attn_bwd_dispatch(int dh, const float *QKV, const float *O, const float *dO,
                       const float *LSE, float *dQKV, float *Dt, int Bc, const sg_config &c,
                       cudaStream_t st, int *err, unsigned char *dQKVt = nullptr,
                       float *bsum = nullptr, const __nv_bfloat16 *QKVh = nullptr)
{
    if (QKVh && dQKVt && attn_band_supported(c)) {
        launch_attn_bwd_band(c, QKVh, reinterpret_cast<const __nv_bfloat16 *>(O), dO, LSE, dQKVt, bsum, Bc, err, st);
        return true;
    }
    if (QKVh && dQKVt && attn_mma_supported(c) && attn_tmem_supported(c)) {
        launch_attn_bwd_tmem(c, QKVh, reinterpret_cast<const __nv_bfloat16 *>(O), dO, LSE, dQKVt, bsum, Bc,
                             err, st);
        return true;
    }
    if (QKVh && dQKVt && attn_mma_supported(c)) {
        launch_attn_bwd_mma(c, QKVh, reinterpret_cast<const __nv_bfloat16 *>(O), dO, LSE, dQKVt, bsum, Bc, st);
        return true;
    }
    if (attn_tc_supported(c)) {
        launch_attn_bwd_tc(c, QKV, O, dO, LSE, dQKV, Dt, Bc, err, st);
        return false;
    }
    if (dh == 8) return attn_bwd<8>(QKV, O, dO, LSE, dQKV, Dt, Bc, c, st, dQKVt, bsum, QKVh);
    if (dh == 16) return attn_bwd<16>(QKV, O, dO, LSE, dQKV, Dt, Bc, c, st, dQKVt, bsum, QKVh);
    return attn_bwd<32>(QKV, O, dO, LSE, dQKV, Dt, Bc, c, st, dQKVt, bsum, QKVh);
}

template <int EPI>
void gemm(const float *A, int lda, const float *Bm, int ldb, const float *bias, float *C, int ldc,
          int64_t M, int N, int K, cudaStream_t st, const float *aux = nullptr, int ldaux = 0,
          float *aux_out = nullptr)
{
    const int64_t blocks = (int64_t)((N + 63) / 64) * ((M + 63) / 64);
    gemm_nn_kernel<EPI><<<(unsigned)blocks, 256, 0, ::sg::counted(st)>>>(A, lda, Bm, ldb, bias, C, ldc, aux, ldaux, aux_out,
                                             M, N, K);
}

void gemm_tn_acc(const float *A, int lda, const float *Bm, int ldb, float *C, int64_t M, int N1,
                 int N2, cudaStream_t st)
{
    const int tiles = ((N1 + 63) / 64) * ((N2 + 63) / 64);
    int64_t splits = std::max<int64_t>(1, std::min<int64_t>((M + 511) / 512, 608 / tiles + 1));
    const int64_t rpb = (M + splits - 1) / splits;
    splits = (M + rpb - 1) / rpb;
    dim3 grid((N2 + 63) / 64, (N1 + 63) / 64, (unsigned)splits);
    gemm_tn_acc_kernel<<<grid, 256, 0, ::sg::counted(st)>>>(A, lda, Bm, ldb, C, M, N1, N2, rpb);
}

void colsum(const float *A, int lda, int64_t M, int N, float *out, cudaStream_t st)
{
    const int64_t splits = std::max<int64_t>(1, std::min<int64_t>((M + 1023) / 1024, 256));
    const int64_t rpb = (M + splits - 1) / splits;
    dim3 grid((N + 31) / 32, (unsigned)((M + rpb - 1) / rpb)), block(32, 8);
    colsum_kernel<<<grid, block, 0, ::sg::counted(st)>>>(A, lda, M, N, out, rpb);
}

int sm_count()
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Blocks of 256 threads for a row kernel of `rows` rows taking `rows_per_warp`
// rows per warp pass, at most `per_sm` blocks per SM (grid-stride beyond).
unsigned row_blocks(int64_t rows, int rows_per_warp, int per_sm)
{
    const int64_t warps = (rows + rows_per_warp - 1) / rows_per_warp;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, (int64_t)sm_count() * per_sm));
}

// LayerNorm forward: Y (FP32) and/or the wide BF16 copy At, mean and 1/std.
void ln_fwd(const float *X, const float *g, const float *b, float *Y, float *mu, float *rs, int64_t R,
            int D, unsigned char *At, cudaStream_t st)
{
    constexpr int RPW = 4;
    const int64_t rows = At ? tl_blocks(R) * 128 : R;
    auto go = [&](auto kern, int lpr) {
        kern<<<row_blocks(rows, RPW * (32 / lpr), 8), 256, 0, ::sg::counted(st)>>>(X, g, b, Y, mu, rs, R, At);
    };
    switch (D) {
    case 32: go(ln_fwd_g8_kernel<32, RPW>, 4); return;
    case 64: go(ln_fwd_g8_kernel<64, RPW>, 8); return;
    case 128: go(ln_fwd_g8_kernel<128, RPW>, 16); return;
    case 256: go(ln_fwd_g8_kernel<256, RPW>, 32); return;
    default: break;
    }
    ln_fwd_kernel<<<blocks_for(rows, 8), 256, 0, ::sg::counted(st)>>>(X, g, b, Y, mu, rs, R, D, At);
}

// dX = dres + LN'(X)^T dY (dres may be null), dg/db accumulated; optionally
// the wide BF16 copy dXt and the column sums dcol += sum_r dX.  Returns false
// (nothing launched for dXt/dcol) where the width has no fused kernel.
bool ln_bwd_res(const float *dY, const float *X, const float *mu, const float *rs, const float *g,
                const float *dres, float *dX, float *dg, float *db, int64_t R, int D, cudaStream_t st,
                unsigned char *dXt = nullptr, float *dcol = nullptr)
{
    if (g8_width(D)) {
        constexpr int RPW = 2;
        const int64_t rows = dXt ? tl_blocks(R) * 128 : R;
        auto go = [&](auto kern, int lpr) {
            kern<<<row_blocks(rows, RPW * (32 / lpr), 8), 256, 0, ::sg::counted(st)>>>(
                dY, X, mu, rs, g, dres, dX, dg, db, R, dXt, dcol);
        };
        switch (D) {
        case 32: go(ln_bwd_g8_kernel<32, RPW>, 4); break;
        case 64: go(ln_bwd_g8_kernel<64, RPW>, 8); break;
        case 128: go(ln_bwd_g8_kernel<128, RPW>, 16); break;
        default: go(ln_bwd_g8_kernel<256, RPW>, 32); break;
        }
        return true;
    }
    constexpr int RPW = 4;
    const int64_t want = (R + 8 * RPW - 1) / (8 * RPW);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * 8));
    auto go = [&](auto kern) { kern<<<blocks, 256, 0, ::sg::counted(st)>>>(dY, X, mu, rs, g, dres, dX, dg, db, R); };
    switch (D) {
    case 96: go(ln_bwd_rows_kernel<3, RPW>); return false;
    default: break;
    }
    // other widths: copy the residual, then the generic kernel accumulates
    if (dres) cudaMemcpyAsync(dX, dres, (size_t)R * D * sizeof(float), cudaMemcpyDeviceToDevice, st);
    const int rpb = 256;
    ln_bwd_kernel<<<blocks_for(R, rpb), 256, 2 * D * sizeof(float), ::sg::counted(st)>>>(
        dY, X, mu, rs, g, dX, dres ? 1 : 0, dg, db, R, D, rpb);
    return false;
}

struct Work {
    std::vector<LayerBufs> layers;
    float *Hfin, *muf, *rsf, *Y, *ell, *lp, *Hping;
    float *dH, *dHmid, *dA, *dQKV, *dF1, *Dt;
    // tensor-core backward scratch (wide BF16)
    unsigned char *dHt, *dF1t, *dQKVt;
    float *bsum;    // per-sample bias sums of dQKV [R / N][3 D]
    uint8_t *tok8;  // patched models: the token class of every row
    int64_t total_floats;
};

Work carve(const sg_config &c, float *base, int64_t R, bool bwd)
{
    Work w{};
    const int64_t D = c.d, F = c.d_ff, NH = c.n_heads;
    const bool tc = use_tc(c);
    int64_t off = 0;  // floats; every buffer starts 16-byte aligned
    auto take = [&](int64_t n) {
        float *q = base ? base + off : nullptr;
        off += (n + 3) & ~int64_t(3);
        return q;
    };
    auto take_t = [&](int64_t rows, int64_t F) {  // wide BF16 W(rows, F)
        return reinterpret_cast<unsigned char *>(take((int64_t)((wl_bytes(rows, (int)F) + 3) / 4)));
    };
    const int nl = bwd ? c.n_layers : 1;
    for (int l = 0; l < nl; ++l) {
        LayerBufs L{};
        L.Hin = take(R * D);
        L.mu1 = take(R);
        L.rs1 = take(R);
        if (!tc) L.A1 = take(R * D);  // FP32 LayerNorm outputs: the FP32 model's GEMMs
        L.QKV = take(R * 3 * D);
        L.O = take(R * D);
        L.LSE = take(R * NH);
        L.Hmid = take(R * D);
        L.mu2 = take(R);
        L.rs2 = take(R);
        if (!tc) L.A2 = take(R * D);
        if (tc) {
            L.A1t = take_t(R, D);
            L.A2t = take_t(R, D);
            L.Gt = take_t(R, F);
            L.F1t = take_t(R, F);
        } else {
            L.F1 = take(R * F);
            L.G = take(R * F);
        }
        w.layers.push_back(L);
    }
    if (tc && bwd) {
        w.dHt = take_t(R, D);
        w.dF1t = take_t(R, F);
        w.dQKVt = take_t(R, 3 * D);
        w.bsum = take((R / c.N + 1) * 3 * D);
    }
    w.Hfin = take(R * D);
    w.Hping = take(R * D);
    w.muf = take(R);
    w.rsf = take(R);
    if (spins_per_token(c) > 1 || !g8_width((int)D)) w.Y = take(R * D);  // patched / generic head
    w.ell = take(R);
    w.lp = take(R);
    if (spins_per_token(c) > 1) w.tok8 = reinterpret_cast<uint8_t *>(take((R + 3) / 4));
    if (bwd) {
        w.dH = take(R * D);
        w.dHmid = take(R * D);
        w.dA = take(R * D);
        // FP32 dQKV only where the attention backward does not write the wide
        // BF16 copy itself (the FP32 model, the tcgen05 flash attention)
        if (!tc || !qkv_bf16(c)) w.dQKV = take(R * 3 * D);
        if (!tc) w.dF1 = take(R * F);
        w.Dt = take(R * NH);
    }
    w.total_floats = off;
    return w;
}

sg_status plan_chunks(sg_model *m, int64_t B, bool bwd, Plan &p, size_t &bytes)
{
    const sg_config &c = m->seq;  // N = tokens
    // floats per sample from a dry run of carve() over one sample's rows
    const size_t per_sample = (size_t)carve(c, nullptr, c.N, bwd).total_floats * sizeof(float);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    // at most a third of the free memory and 64 GB: large enough that a batch of
    // 16384 short sequences is one chunk (launch count and tail effects then
    // stay per layer, not per chunk and layer), small enough that a BF16 and an
    // FP32 model can hold their workspaces side by side on one GPU
    const size_t budget = std::min<size_t>((size_t)64 << 30, free_b / 3 + m->ws_bytes);
    int64_t Bc = std::max<int64_t>(1, (int64_t)(budget / per_sample));
    Bc = std::min<int64_t>(Bc, B);
    if (m->max_chunk > 0) Bc = std::min<int64_t>(Bc, m->max_chunk);
    // keep the warp count of the attention kernels within a 32-bit grid
    Bc = std::min<int64_t>(Bc, (int64_t)((1ll << 30) / ((int64_t)c.N * c.n_heads)));
    p.Bc = Bc;
    p.R = Bc * c.N;
    p.keep = bwd;
    bytes = (size_t)carve(c, nullptr, p.R, bwd).total_floats * sizeof(float);
    return SG_OK;
}

// Forward over one chunk.  Layer l reads H_in (embedding or previous output)
// and writes its output into the next layer's Hin (or Hfin after the last).
void forward_chunk(sg_model *m, const int8_t *spins, int Bc, Work &w, bool keep, cudaStream_t st)
{
    const sg_config &c = m->seq;  // N = tokens
    const int64_t R = (int64_t)Bc * c.N;
    const int P = spins_per_token(c), K = 1 << P;
    const int D = c.d, F = c.d_ff, dh = c.d / c.n_heads;
    const float *W = m->w;
    float *H = keep ? w.layers[0].Hin : w.Hping;
    if (P > 1) {
        spins_to_tokens_kernel<<<blocks_for(R, 256), 256, 0, ::sg::counted(st)>>>(
            spins, R, c.N, m->cfg.N, P, c.lat_D, c.lat_L, w.tok8);
        embed_tok_kernel<<<blocks_for(R * D, 256), 256, 0, ::sg::counted(st)>>>(
            w.tok8, R, c.N, D, c.d_token, W + m->off.tok, W + m->off.pos, H);
    } else if (D % 4 == 0 && D <= 1024) {
        const int rpb = std::max(1, 256 / (D / 4));
        embed4_kernel<<<(unsigned)((R + rpb - 1) / rpb), 256, 0, ::sg::counted(st)>>>(
            spins, R, c.N, D, c.d_token, W + m->off.tok, W + m->off.pos, H);
    } else
    embed_kernel<<<blocks_for(R * D, 256), 256, 0, ::sg::counted(st)>>>(spins, R, c.N, D, c.d_token,
                                                         W + m->off.tok, W + m->off.pos, H);
    for (int l = 0; l < c.n_layers; ++l) {
        LayerBufs &L = w.layers[keep ? l : 0];
        const LayerOff &o = m->off.L[l];
        float *Hin = keep ? L.Hin : H;
        float *Hout = keep ? (l + 1 < c.n_layers ? w.layers[l + 1].Hin : w.Hfin)
                           : (H == w.Hping ? w.Hfin : w.Hping);
        const bool tcp = use_tc(c);
        ln_fwd(Hin, W + o.ln1g, W + o.ln1b, tcp ? nullptr : L.A1, L.mu1, L.rs1, R, D,
               tcp ? L.A1t : nullptr, st);
        if (tcp) {
            // tensor-core GEMMs over tiled BF16 operands; the LayerNorms write
            // the tiled A operands directly
            const unsigned char *bt = (const unsigned char *)m->bt;
            RowGemm g{};
            g.A = L.A1t; g.RB = tl_blocks(R); g.K = D; g.KC = (D + 63) / 64; g.R = R; g.err = (int *)m->err;
            g.Bw = bt + m->bt_off[l][0]; g.NBw = (int)tl_blocks(3 * D); g.N = 3 * D;
            g.bias = m->wt + m->pack.bqkv[l]; g.ld_out = 3 * D;
            const bool hq = qkv_bf16(c);
            __nv_bfloat16 *QKVh = hq ? reinterpret_cast<__nv_bfloat16 *>(L.QKV) : nullptr;
            g.out_f32 = L.QKV; g.out_h = QKVh;
            launch_row_gemm(g, hq ? TE_STORE_BF16 : TE_STORE_F32, st);
            attn_fwd_dispatch(dh, L.QKV, Hin, L.O, L.Hmid, L.LSE, Bc, c, st, (int *)m->err, QKVh, keep);
            ln_fwd(L.Hmid, W + o.ln2g, W + o.ln2b, nullptr, L.mu2, L.rs2, R, D, L.A2t, st);
            g.A = L.A2t; g.Bw = bt + m->bt_off[l][1]; g.NBw = (int)tl_blocks(F); g.N = F;
            // G = gelu(F1) for FFN2, and gelu'(F1) kept for the backward
            g.bias = m->wt + m->pack.b1[l]; g.out_t = L.Gt; g.out_t2 = keep ? L.F1t : nullptr;
            launch_row_gemm(g, TE_GELU_T, st);
            g.A = L.Gt; g.K = F; g.KC = (F + 63) / 64; g.Bw = bt + m->bt_off[l][2]; g.NBw = (int)tl_blocks(D);
            g.N = D; g.bias = m->wt + m->pack.b2[l]; g.out_f32 = Hout; g.ld_out = D;
            g.resid = L.Hmid; g.ld_resid = D;
            launch_row_gemm(g, TE_RESID_F32, st);
            H = Hout;
            continue;
        }
        gemm<G_STORE>(L.A1, D, m->wt + m->pack.WqkvT[l], 3 * D, m->wt + m->pack.bqkv[l], L.QKV, 3 * D, R,
                      3 * D, D, st);
        attn_fwd_dispatch(dh, L.QKV, Hin, L.O, L.Hmid, L.LSE, Bc, c, st, (int *)m->err);
        ln_fwd(L.Hmid, W + o.ln2g, W + o.ln2b, L.A2, L.mu2, L.rs2, R, D, nullptr, st);
        if (keep)
            gemm<G_GELU>(L.A2, D, m->wt + m->pack.W1T[l], F, m->wt + m->pack.b1[l], L.G, F, R, F, D, st,
                         nullptr, F, L.F1);
        else
            gemm<G_GELU_ONLY>(L.A2, D, m->wt + m->pack.W1T[l], F, m->wt + m->pack.b1[l], L.G, F, R, F, D, st);
        gemm<G_ADDRES>(L.G, F, m->wt + m->pack.W2T[l], D, m->wt + m->pack.b2[l], Hout, D, R, D, F, st, L.Hmid,
                       D);
        H = Hout;
    }
    // ensure the final stream lives in Hfin
    if (H != w.Hfin)
        cudaMemcpyAsync(w.Hfin, H, (size_t)R * D * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (P > 1)
        head_fwd_cat_kernel<<<blocks_for(R, 8), 256, 0, ::sg::counted(st)>>>(
            w.Hfin, W + m->off.lnfg, W + m->off.lnfb, W + m->off.Wh, W + m->off.bh, w.tok8,
            keep ? w.Y : nullptr, keep ? w.muf : nullptr, keep ? w.rsf : nullptr,
            keep ? w.ell : nullptr, w.lp, R, D, K);
    else if (g8_width(D)) {
        constexpr int RPW = 2;
        auto go = [&](auto kern, int lpr) {
            kern<<<row_blocks(R, RPW * (32 / lpr), 8), 256, 0, ::sg::counted(st)>>>(
                w.Hfin, W + m->off.lnfg, W + m->off.lnfb, W + m->off.Wh, W + m->off.bh, spins,
                keep ? w.muf : nullptr, keep ? w.rsf : nullptr, keep ? w.ell : nullptr, w.lp, R);
        };
        switch (D) {
        case 32: go(head_fwd_g8_kernel<32, RPW>, 4); break;
        case 64: go(head_fwd_g8_kernel<64, RPW>, 8); break;
        case 128: go(head_fwd_g8_kernel<128, RPW>, 16); break;
        default: go(head_fwd_g8_kernel<256, RPW>, 32); break;
        }
    } else
        head_fwd_kernel<<<blocks_for(R, 8), 256, 0, ::sg::counted(st)>>>(
            w.Hfin, W + m->off.lnfg, W + m->off.lnfb, W + m->off.Wh, W + m->off.bh, spins,
            keep ? w.Y : nullptr, keep ? w.muf : nullptr, keep ? w.rsf : nullptr,
            keep ? w.ell : nullptr, w.lp, R, D);
}

}  // namespace

// Tiled BF16 copies of the weights for the tensor-core teacher-forced pass:
// Wqkv, W1, W2 (forward B operands) and W2^T, W1^T, Wqkv^T (backward).
sg_status launch_pack_tiled_weights(sg_model *m, cudaStream_t st)
{
    const sg_config &c = m->cfg;
    if (!use_tc(c)) return SG_OK;
    const int D = c.d, F = c.d_ff;
    const size_t sizes[6] = {tl_bytes(3 * D, D), tl_bytes(F, D), tl_bytes(D, F),
                             tl_bytes(F, D), tl_bytes(D, F), tl_bytes(D, 3 * D)};
    size_t per_layer = 0;
    for (size_t s : sizes) per_layer += s;
    SG_TRY(ensure_buffer(&m->bt, &m->bt_bytes, per_layer * c.n_layers));
    unsigned char *bt = (unsigned char *)m->bt;
    for (int l = 0; l < c.n_layers; ++l) {
        size_t off = per_layer * l;
        for (int i = 0; i < 6; ++i) {
            m->bt_off[l][i] = off;
            off += sizes[i];
        }
        const LayerOff &o = m->off.L[l];
        const float *W = m->w;
        SG_TRY(launch_pack_tiled(W + o.Wqkv, 3 * D, D, bt + m->bt_off[l][0], false, st));
        SG_TRY(launch_pack_tiled(W + o.W1, F, D, bt + m->bt_off[l][1], false, st));
        SG_TRY(launch_pack_tiled(W + o.W2, D, F, bt + m->bt_off[l][2], false, st));
        SG_TRY(launch_pack_tiled(W + o.W2, D, F, bt + m->bt_off[l][3], true, st));
        SG_TRY(launch_pack_tiled(W + o.W1, F, D, bt + m->bt_off[l][4], true, st));
        SG_TRY(launch_pack_tiled(W + o.Wqkv, 3 * D, D, bt + m->bt_off[l][5], true, st));
    }
    return SG_OK;
}

sg_status launch_logprob_f32(sg_model *m, const int8_t *spins, int64_t B, float *logq,
                             cudaStream_t st)
{
    const sg_config &c = m->seq;  // N = tokens
    if (!dh_supported(c.d / c.n_heads))
        return fail(SG_EUNSUPPORTED, "prefill attention is built for d_h in {8, 16, 32}");
    if (c.d % 4 || c.d_ff % 4) return fail(SG_EUNSUPPORTED, "d and d_ff must be multiples of 4");
    Plan p;
    size_t bytes;
    SG_TRY(plan_chunks(m, B, false, p, bytes));
    SG_TRY(ensure_buffer(&m->ws, &m->ws_bytes, bytes));
    for (int64_t b0 = 0; b0 < B; b0 += p.Bc) {
        const int Bc = (int)std::min<int64_t>(p.Bc, B - b0);
        Work w = carve(c, (float *)m->ws, (int64_t)Bc * c.N, false);
        const int8_t *sp = spins + b0 * m->cfg.N;
        forward_chunk(m, sp, Bc, w, false, st);
        seg_sum_kernel<<<Bc, 256, 0, ::sg::counted(st)>>>(w.lp, c.N, logq + b0);
    }
    return check_launch("teacher-forced log q");
}

sg_status launch_grad_f32(sg_model *m, const int8_t *spins, const float *coeff, int64_t B,
                          float *grad, float *logq, cudaStream_t st)
{
    const sg_config &c = m->seq;  // N = tokens
    if (!dh_supported(c.d / c.n_heads))
        return fail(SG_EUNSUPPORTED, "prefill attention is built for d_h in {8, 16, 32}");
    if (c.d % 4 || c.d_ff % 4) return fail(SG_EUNSUPPORTED, "d and d_ff must be multiples of 4");
    if (c.d > 512) return fail(SG_EUNSUPPORTED, "backward is built for d <= 512");
    const int P = spins_per_token(c), K = 1 << P;
    Plan p;
    size_t bytes;
    SG_TRY(plan_chunks(m, B, true, p, bytes));
    SG_TRY(ensure_buffer(&m->ws, &m->ws_bytes, bytes));
    SG_CUDA_TRY(cudaMemsetAsync(grad, 0, (size_t)m->P * sizeof(float), st));
    const int D = c.d, F = c.d_ff, dh = c.d / c.n_heads;
    const float *W = m->w;
    const BlobOff &O = m->off;
    for (int64_t b0 = 0; b0 < B; b0 += p.Bc) {
        const int Bc = (int)std::min<int64_t>(p.Bc, B - b0);
        const int64_t R = (int64_t)Bc * c.N;
        Work w = carve(c, (float *)m->ws, R, true);
        const int8_t *sp = spins + b0 * m->cfg.N;
        forward_chunk(m, sp, Bc, w, true, st);
        if (logq) seg_sum_kernel<<<Bc, 256, 0, ::sg::counted(st)>>>(w.lp, c.N, logq + b0);
        // head + LN_f
        bool dH_fused = false;  // dHt and the top layer's b2 gradient already written
        if (P > 1) {
            const size_t red = ((size_t)K * D + 2 * D + K) * sizeof(float);
            const int shared = red <= 48 * 1024;
            head_bwd_cat_kernel<<<blocks_for(R, 256), 256, shared ? red : 0, ::sg::counted(st)>>>(
                w.Hfin, w.muf, w.rsf, w.Y, w.ell, w.tok8, coeff + b0, W + O.lnfg, W + O.Wh,
                W + O.bh, w.dH, grad + O.Wh, grad + O.bh, grad + O.lnfg, grad + O.lnfb, R, c.N, D,
                K, 256, shared);
        } else if (g8_width(D)) {
            constexpr int RPW = 2;
            // the tensor-core backward takes the wide copy of dH and b2's gradient here
            unsigned char *dHt = use_tc(c) ? w.dHt : nullptr;
            float *db2 = use_tc(c) ? grad + O.L[c.n_layers - 1].b2 : nullptr;
            dH_fused = use_tc(c);
            auto go = [&](auto kern, int lpr) {
                kern<<<row_blocks(dHt ? tl_blocks(R) * 128 : R, RPW * (32 / lpr), 4), 256, 0,
                       ::sg::counted(st)>>>(
                    w.Hfin, w.muf, w.rsf, w.ell, sp, coeff + b0, W + O.lnfg, W + O.lnfb, W + O.Wh,
                    w.dH, grad + O.Wh, grad + O.bh, grad + O.lnfg, grad + O.lnfb, R, c.N, dHt, db2);
            };
            switch (D) {
            case 32: go(head_bwd_g8_kernel<32, RPW>, 4); break;
            case 64: go(head_bwd_g8_kernel<64, RPW>, 8); break;
            case 128: go(head_bwd_g8_kernel<128, RPW>, 16); break;
            default: go(head_bwd_g8_kernel<256, RPW>, 32); break;
            }
        } else
            head_bwd_kernel<<<blocks_for(R, 256), 256, (4 * D + 2) * sizeof(float), ::sg::counted(st)>>>(
                w.Hfin, w.muf, w.rsf, w.Y, w.ell, sp, coeff + b0, W + O.lnfg, W + O.Wh, w.dH,
                grad + O.Wh, grad + O.bh, grad + O.lnfg, grad + O.lnfb, R, c.N, D, 256);
        for (int l = c.n_layers - 1; l >= 0 && use_tc(c); --l) {
            // tensor-core backward: dX GEMMs by row_gemm, weight gradients by
            // split wgrad reading the wide BF16 activations MN-major
            LayerBufs &L = w.layers[l];
            const LayerOff &o = O.L[l];
            const unsigned char *bt = (const unsigned char *)m->bt;
            const int64_t RB = tl_blocks(R);
            // C (+)= A^T B over the rows; A has the wider feature count
            auto wgrad = [&](const unsigned char *A, int M, const unsigned char *Bm, int N, float *C,
                             int ldc, bool transpose_out) {
                WgradGemm g{};
                g.A = A; g.M = M; g.Bm = Bm; g.N = N; g.RB = RB;
                const int64_t per_split = (int64_t)((M + 127) / 128) * ((N + 255) / 256);
                const int64_t splits = std::max<int64_t>(1, std::min<int64_t>(RB, 304 / per_split));
                g.rb_per_cta = (RB + splits - 1) / splits;
                g.C = C; g.ldc = ldc; g.transpose_out = transpose_out ? 1 : 0; g.err = (int *)m->err;
                launch_wgrad_gemm(g, st);
            };
            RowGemm g{};
            g.RB = RB; g.R = R; g.err = (int *)m->err;
            // FFN: H = Hmid + W2 G + b2, G = gelu(F1), F1 = W1 A2 + b1
            if (!dH_fused) {
                launch_to_wide(w.dH, R, D, w.dHt, st);
                colsum(w.dH, D, R, D, grad + o.b2, st);
            }
            // dF1 = (dH W2) gelu'(F1), its column sums (b1's gradient) fused
            g.A = w.dHt; g.K = D; g.KC = (D + 63) / 64; g.Bw = bt + m->bt_off[l][3];
            g.NBw = (int)tl_blocks(F); g.N = F; g.aux_t = L.F1t; g.out_t = w.dF1t;
            g.colsum = F <= 1024 ? grad + o.b1 : nullptr;
            launch_row_gemm(g, TE_GELU_BWD_T, st);
            g.colsum = nullptr;
            wgrad(L.Gt, F, w.dHt, D, grad + o.W2, F, true);        // dW2[d][f] = sum dH[d] G[f]
            wgrad(w.dF1t, F, L.A2t, D, grad + o.W1, D, false);     // dW1[f][d] = sum dF1[f] A2[d]
            if (F > 1024) {
                const int64_t rpb = 4096;
                dim3 grid((F + 31) / 32, (unsigned)((R + rpb - 1) / rpb)), block(32, 8);
                colsum_tiled_kernel<<<grid, block, 0, ::sg::counted(st)>>>(w.dF1t, R, F, grad + o.b1, rpb);
            }
            // dHmid = dH + LN2'(dF1 W1): the LayerNorm backward in the GEMM epilogue where it fits
            g.A = w.dF1t; g.K = F; g.KC = (F + 63) / 64; g.Bw = bt + m->bt_off[l][4];
            g.NBw = (int)tl_blocks(D); g.N = D; g.ld_out = D;
            if (ln_bwd_fusable(g)) {
                g.out_f32 = w.dHmid;
                g.ln_x = L.Hmid; g.ln_mu = L.mu2; g.ln_rs = L.rs2; g.ln_g = W + o.ln2g; g.ln_dres = w.dH;
                g.ln_dg = grad + o.ln2g; g.ln_db = grad + o.ln2b; g.ln_dcol = nullptr; g.ln_dxt = nullptr;
                launch_row_gemm(g, TE_LN_BWD, st);
            } else {
                g.out_f32 = w.dA;
                launch_row_gemm(g, TE_STORE_F32, st);
                ln_bwd_res(w.dA, L.Hmid, L.mu2, L.rs2, W + o.ln2g, w.dH, w.dHmid, grad + o.ln2g,
                           grad + o.ln2b, R, D, st);
            }
            // attention: Hmid = Hin + O(QKV)
            if (attn_bwd_dispatch(dh, L.QKV, L.O, w.dHmid, L.LSE, w.dQKV, w.Dt, Bc, c, st,
                                  (int *)m->err, w.dQKVt, w.bsum,
                                  qkv_bf16(c) ? reinterpret_cast<const __nv_bfloat16 *>(L.QKV) : nullptr)) {
                if (l == c.n_layers - 1) launch_zero_wide_tail(R, 3 * D, w.dQKVt, st);
                colsum(w.bsum, 3 * D, Bc, 3 * D, grad + o.bqkv, st);
            } else {
                launch_to_wide(w.dQKV, R, 3 * D, w.dQKVt, st);
                colsum(w.dQKV, 3 * D, R, 3 * D, grad + o.bqkv, st);
            }
            wgrad(w.dQKVt, 3 * D, L.A1t, D, grad + o.Wqkv, D, false);  // dWqkv[j][d] = sum dQKV[j] A1[d]
            // dH of layer l - 1 = dHmid + LN1'(dQKV Wqkv), with its wide copy and b2's
            // gradient, the LayerNorm backward in the GEMM epilogue where it fits
            g.A = w.dQKVt; g.K = 3 * D; g.KC = (3 * D + 63) / 64; g.Bw = bt + m->bt_off[l][5];
            g.NBw = (int)tl_blocks(D); g.N = D; g.ld_out = D;
            if (ln_bwd_fusable(g)) {
                g.out_f32 = w.dH;
                g.ln_x = L.Hin; g.ln_mu = L.mu1; g.ln_rs = L.rs1; g.ln_g = W + o.ln1g; g.ln_dres = w.dHmid;
                g.ln_dg = grad + o.ln1g; g.ln_db = grad + o.ln1b;
                g.ln_dcol = l > 0 ? grad + O.L[l - 1].b2 : nullptr;
                g.ln_dxt = l > 0 ? w.dHt : nullptr;
                launch_row_gemm(g, TE_LN_BWD, st);
                dH_fused = true;
            } else {
                g.out_f32 = w.dA;
                launch_row_gemm(g, TE_STORE_F32, st);
                dH_fused = ln_bwd_res(w.dA, L.Hin, L.mu1, L.rs1, W + o.ln1g, w.dHmid, w.dH, grad + o.ln1g,
                                      grad + o.ln1b, R, D, st, l > 0 ? w.dHt : nullptr,
                                      l > 0 ? grad + O.L[l - 1].b2 : nullptr);
            }
        }
        for (int l = c.n_layers - 1; l >= 0 && !use_tc(c); --l) {
            LayerBufs &L = w.layers[l];
            const LayerOff &o = O.L[l];
            // FFN: H = Hmid + W2 G + b2, G = gelu(F1), F1 = W1 A2 + b1
            gemm_tn_acc(w.dH, D, L.G, F, grad + o.W2, R, D, F, st);
            colsum(w.dH, D, R, D, grad + o.b2, st);
            gemm<G_GELU_BWD>(w.dH, D, m->wt + m->pack.W2[l], F, nullptr, w.dF1, F, R, F, D, st, L.F1, F);
            gemm_tn_acc(w.dF1, F, L.A2, D, grad + o.W1, R, F, D, st);
            colsum(w.dF1, F, R, F, grad + o.b1, st);
            gemm<G_STORE>(w.dF1, F, m->wt + m->pack.W1[l], D, nullptr, w.dA, D, R, D, F, st);
            ln_bwd_res(w.dA, L.Hmid, L.mu2, L.rs2, W + o.ln2g, w.dH, w.dHmid, grad + o.ln2g,
                       grad + o.ln2b, R, D, st);
            // attention: Hmid = Hin + O(QKV)
            attn_bwd_dispatch(dh, L.QKV, L.O, w.dHmid, L.LSE, w.dQKV, w.Dt, Bc, c, st, (int *)m->err);
            gemm_tn_acc(w.dQKV, 3 * D, L.A1, D, grad + o.Wqkv, R, 3 * D, D, st);
            colsum(w.dQKV, 3 * D, R, 3 * D, grad + o.bqkv, st);
            gemm<G_STORE>(w.dQKV, 3 * D, m->wt + m->pack.Wqkv[l], D, nullptr, w.dA, D, R, D, 3 * D, st);
            ln_bwd_res(w.dA, L.Hin, L.mu1, L.rs1, W + o.ln1g, w.dHmid, w.dH, grad + o.ln1g,
                       grad + o.ln1b, R, D, st);
        }
        if (P > 1)
            embed_bwd_tok_kernel<<<blocks_for((int64_t)c.N * D, 256), 256, 0, ::sg::counted(st)>>>(
                w.dH, w.tok8, Bc, c.N, D, c.d_token, grad + O.tok, grad + O.pos);
        else {
            // samples split so that about 4 warps per SM-slot are in flight
            const int64_t nd_blocks = blocks_for((int64_t)c.N * D, 256);
            const int64_t splits = std::max<int64_t>(
                1, std::min<int64_t>(Bc, ((int64_t)sm_count() * 8 + nd_blocks - 1) / nd_blocks));
            const int per_split = (int)((Bc + splits - 1) / splits);
            embed_bwd_split_kernel<<<dim3((unsigned)nd_blocks, (unsigned)((Bc + per_split - 1) / per_split)),
                                     256, 0, ::sg::counted(st)>>>(w.dH, sp, Bc, c.N, D, c.d_token,
                                                                  per_split, grad + O.tok, grad + O.pos);
        }
    }
    return check_launch("REINFORCE backward");
}

}  // namespace sg
