// attn_tc.cu -- teacher-forced attention on tcgen05 (BF16 operands, FP32
// accumulation in TMEM), block-sparse over 128 x 128 tiles of (query, key)
// with the band + sink mask of the sampler (SI Sec. I.A) or a dense causal
// mask.  Scores use the scale 1/sqrt(d_h) of the model (no W_O; heads are
// column slices of the QKV rows).
//
//   forward   (per sample, head, 128-query tile; thread = query row):
//             S = Q K^T -> online softmax in registers -> P (BF16, shared)
//             -> O_blk = P V -> O = sum corr * O_blk; writes O, Hmid = Hin + O
//             and the row log-sum-exp.
//   backward  dQ pass (thread = query row): S, dP = dO V^T, dS = P (dP - D)
//             -> dQ += dS K; also writes D = rowsum(dO * O).
//             dK/dV pass (per 128-key block; thread = key row): S^T = K Q^T,
//             dP^T = V dO^T, P^T, dS^T -> dV += P^T dO, dK += dS^T Q.
// Shared-memory operands are in the core-matrix layout of tc.cuh (no swizzle);
// "T" operands are transposed copies ([d_h x 128] with the 128 positions as
// the K dimension).  One mbarrier per CTA orders MMA completion; every wait is
// bounded and sets the model's error word on a timeout.
#include <cuda_bf16.h>

#include <algorithm>

#include "sg_internal.cuh"
#include "tc.cuh"

namespace sg {

namespace {

constexpr int kT = 128;  // queries per tile = keys per block = MMA M

__device__ __forceinline__ uint32_t bf2(float a, float b)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// row `r` of a [128 x DH] operand (K = DH), 8 values per 16-byte store
template <int DH>
__device__ __forceinline__ void put_row(unsigned char *tile, int r, const float (&v)[DH])
{
#pragma unroll
    for (int c = 0; c < DH / 8; ++c) {
        uint4 q;
        q.x = bf2(v[8 * c], v[8 * c + 1]);
        q.y = bf2(v[8 * c + 2], v[8 * c + 3]);
        q.z = bf2(v[8 * c + 4], v[8 * c + 5]);
        q.w = bf2(v[8 * c + 6], v[8 * c + 7]);
        *reinterpret_cast<uint4 *>(tile + tc::cm_offset(r, 8 * c, DH / 8)) = q;
    }
}

// column `r` of a transposed [DH x 128] operand (K = the 128 positions)
template <int DH>
__device__ __forceinline__ void put_col(unsigned char *tile, int r, const float (&v)[DH])
{
#pragma unroll
    for (int j = 0; j < DH; ++j)
        *reinterpret_cast<__nv_bfloat16 *>(tile + tc::cm_offset(j, r, kT / 8)) = __float2bfloat16(v[j]);
}

// 32 values of row r of a [128 x 128] operand starting at column c0
__device__ __forceinline__ void put_row32(unsigned char *tile, int r, int c0, const float (&v)[32])
{
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint4 q;
        q.x = bf2(v[8 * c], v[8 * c + 1]);
        q.y = bf2(v[8 * c + 2], v[8 * c + 3]);
        q.z = bf2(v[8 * c + 4], v[8 * c + 5]);
        q.w = bf2(v[8 * c + 6], v[8 * c + 7]);
        *reinterpret_cast<uint4 *>(tile + tc::cm_offset(r, c0 + 8 * c, kT / 8)) = q;
    }
}

template <int DH>
__device__ __forceinline__ void load_row(const float *src, bool ok, float scale, float (&v)[DH])
{
#pragma unroll
    for (int c = 0; c < DH / 4; ++c) {
        const float4 x = ok ? __ldg(reinterpret_cast<const float4 *>(src) + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[4 * c] = x.x * scale;
        v[4 * c + 1] = x.y * scale;
        v[4 * c + 2] = x.z * scale;
        v[4 * c + 3] = x.w * scale;
    }
}

// D[128 x n] (+)= A[128 x K] B[n x K]^T, K = 16 * ksteps; A, B core-matrix
// operands with KG_a, KG_b core groups along K.
__device__ __forceinline__ void mma_tile(uint32_t d_tmem, const unsigned char *A, int kg_a,
                                         const unsigned char *B, int kg_b, int n, int ksteps,
                                         bool accumulate)
{
    const uint32_t idesc = tc::idesc_bf16(kT, n);
    const uint32_t sa = tc::smem_u32(A), sb = tc::smem_u32(B);
    for (int k = 0; k < ksteps; ++k)
        tc::mma_bf16(d_tmem, tc::smem_desc(sa + 256 * k, 128, kg_a * 128),
                     tc::smem_desc(sb + 256 * k, 128, kg_b * 128), idesc,
                     (accumulate || k > 0) ? 1u : 0u);
}

struct AttnArgs {
    const float *QKV;   // [R][3D]
    const float *Hin;   // [R][D]
    float *O_out;       // [R][D]   forward output
    float *Hmid;        // [R][D]
    float *LSE_out;     // [R][NH]  forward output
    const float *O;     // [R][D]   backward input
    const float *LSE;   // [R][NH]  backward input
    const float *dO;    // [R][D]
    float *Dt;          // [R][NH]
    float *dQKV;        // [R][3D]
    int B, N, D, NH, mask, W, S;
    int *err;
};

// Key block kb holds a key visible to some query of tile qt.
__device__ __forceinline__ bool block_visible(const AttnArgs &a, int qt, int kb)
{
    if (kb > qt) return false;
    if (a.mask == SG_MASK_DENSE) return true;
    if (kb * kT < a.S) return true;
    return kb * kT + kT - 1 >= qt * kT - a.W;
}

// Last query tile that sees key block kb.
__device__ __forceinline__ int last_query_tile(const AttnArgs &a, int kb)
{
    const int nq = (a.N + kT - 1) / kT;
    if (a.mask == SG_MASK_DENSE || kb * kT < a.S) return nq - 1;
    return min(nq - 1, (kb * kT + kT - 1 + a.W) / kT);
}

// Bounded wait on the CTA's MMA barrier; false (and the error word set) on a timeout.
__device__ __forceinline__ bool wait_mma(uint64_t *bar, uint32_t &phase, int *err, int code)
{
    const bool ok = tc::mbar_wait(bar, phase);
    phase ^= 1u;
    if (!ok && (threadIdx.x & 31) == 0) atomicExch(err, code);
    return ok;
}

template <int DH>
__global__ void __launch_bounds__(128) attn_fwd_tc_kernel(const __grid_constant__ AttnArgs a)
{
    constexpr int KG = DH / 8;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Qs = smem;                 // [128 x DH]
    unsigned char *Ks = Qs + kT * DH * 2;     // [128 x DH]
    unsigned char *Vt = Ks + kT * DH * 2;     // [DH x 128]
    unsigned char *Ps = Vt + kT * DH * 2;     // [128 x 128]
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ int s_err;
    const int tid = threadIdx.x;
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
        s_err = 0;
    }
    if (tid < 32) {
        tc::tmem_alloc(&tslot, 128);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tslot, lanes = (uint32_t)(32 * (tid >> 5)) << 16;
    uint32_t phase = 0;
    const float scale = rsqrtf((float)DH);
    const int nq = (a.N + kT - 1) / kT;
    const int64_t units = (int64_t)a.B * a.NH * nq;

    for (int64_t u = blockIdx.x; u < units && !s_err; u += gridDim.x) {
        const int qt = (int)(u % nq);
        const int hh = (int)((u / nq) % a.NH);
        const int64_t b = u / ((int64_t)nq * a.NH);
        const int t = qt * kT + tid;
        const bool vq = t < a.N;
        const int64_t row = b * a.N + t;
        {
            float q[DH];
            load_row<DH>(a.QKV + row * 3 * a.D + hh * DH, vq, scale, q);
            put_row<DH>(Qs, tid, q);
        }
        float m = -INFINITY, l = 0.f, o[DH];
#pragma unroll
        for (int j = 0; j < DH; ++j) o[j] = 0.f;
        for (int kb = 0; kb <= qt; ++kb) {
            if (!block_visible(a, qt, kb)) continue;
            {
                const int k = kb * kT + tid;
                const bool vk = k < a.N;
                const float *src = a.QKV + (b * a.N + k) * 3 * a.D + hh * DH;
                float v[DH];
                load_row<DH>(src + a.D, vk, 1.f, v);
                put_row<DH>(Ks, tid, v);
                load_row<DH>(src + 2 * a.D, vk, 1.f, v);
                put_col<DH>(Vt, tid, v);
            }
            tc::fence_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc::tc_fence_after();
                mma_tile(tmem, Qs, KG, Ks, KG, kT, DH / 16, false);
                tc::mma_commit(&bar);
            }
            __syncwarp();
            if (!wait_mma(&bar, phase, a.err, 31)) s_err = 1;
            tc::tc_fence_after();
            // block maximum of the visible scores of this row
            float mb = -INFINITY;
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                float s[32];
                tc::tmem_ld32(tmem + lanes + 32 * c, s);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int k = kb * kT + 32 * c + j;
                    if (vq && k < a.N && key_visible(a.mask, a.W, a.S, t, k)) mb = fmaxf(mb, s[j]);
                }
            }
            const float mn = fmaxf(m, mb);
            const float corr = mn == -INFINITY ? 1.f : __expf(m - mn);
            float ps = 0.f;
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                float s[32];
                tc::tmem_ld32(tmem + lanes + 32 * c, s);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int k = kb * kT + 32 * c + j;
                    const bool vis = vq && k < a.N && key_visible(a.mask, a.W, a.S, t, k);
                    s[j] = vis ? __expf(s[j] - mn) : 0.f;
                    ps += s[j];
                }
                put_row32(Ps, tid, 32 * c, s);
            }
            m = mn;
            l = l * corr + ps;
            tc::fence_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            if (tid == 0 && !s_err) {
                tc::tc_fence_after();
                mma_tile(tmem, Ps, kT / 8, Vt, kT / 8, DH, kT / 16, false);
                tc::mma_commit(&bar);
            }
            __syncwarp();
            if (!s_err && !wait_mma(&bar, phase, a.err, 32)) s_err = 1;
            tc::tc_fence_after();
            {
                float ob[32];
                if (DH == 16) {
                    float h[16];
                    tc::tmem_ld16(tmem + lanes, h);
#pragma unroll
                    for (int j = 0; j < 16; ++j) ob[j] = h[j];
                } else {
                    tc::tmem_ld32(tmem + lanes, ob);
                }
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < DH; ++j) o[j] = o[j] * corr + ob[j];
            }
            tc::tc_fence_before();
            __syncthreads();  // the next block's MMA overwrites S and reads Ks/Vt
            if (s_err) break;
        }
        if (vq && l > 0.f) {
            const float inv = 1.0f / l;
            const size_t idx = (size_t)row * a.D + hh * DH;
#pragma unroll
            for (int c = 0; c < DH / 4; ++c) {
                const float4 hin = __ldg(reinterpret_cast<const float4 *>(a.Hin + idx) + c);
                const float4 ov = make_float4(o[4 * c] * inv, o[4 * c + 1] * inv, o[4 * c + 2] * inv,
                                              o[4 * c + 3] * inv);
                reinterpret_cast<float4 *>(a.O_out + idx)[c] = ov;
                reinterpret_cast<float4 *>(a.Hmid + idx)[c] =
                    make_float4(hin.x + ov.x, hin.y + ov.y, hin.z + ov.z, hin.w + ov.w);
            }
            a.LSE_out[row * a.NH + hh] = m + logf(l);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (tid < 32) tc::tmem_dealloc(tmem, 128);
}

// dQ pass.  TMEM: S at columns [0, 128), dP at [128, 256); the dQ block
// product reuses columns [0, DH) once S has been consumed.
template <int DH>
__global__ void __launch_bounds__(128) attn_bwd_dq_tc_kernel(const __grid_constant__ AttnArgs a)
{
    constexpr int KG = DH / 8;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Qs = smem;               // [128 x DH]  (scaled q)
    unsigned char *Gs = Qs + kT * DH * 2;   // [128 x DH]  dO
    unsigned char *Ks = Gs + kT * DH * 2;   // [128 x DH]
    unsigned char *Kt = Ks + kT * DH * 2;   // [DH x 128]
    unsigned char *Vs = Kt + kT * DH * 2;   // [128 x DH]
    unsigned char *dS = Vs + kT * DH * 2;   // [128 x 128]
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ int s_err;
    const int tid = threadIdx.x;
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
        s_err = 0;
    }
    if (tid < 32) {
        tc::tmem_alloc(&tslot, 256);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tslot, lanes = (uint32_t)(32 * (tid >> 5)) << 16;
    uint32_t phase = 0;
    const float scale = rsqrtf((float)DH);
    const int nq = (a.N + kT - 1) / kT;
    const int64_t units = (int64_t)a.B * a.NH * nq;

    for (int64_t u = blockIdx.x; u < units && !s_err; u += gridDim.x) {
        const int qt = (int)(u % nq);
        const int hh = (int)((u / nq) % a.NH);
        const int64_t b = u / ((int64_t)nq * a.NH);
        const int t = qt * kT + tid;
        const bool vq = t < a.N;
        const int64_t row = b * a.N + t;
        float dd = 0.f, lse = 0.f;
        {
            float q[DH], g[DH], o[DH];
            load_row<DH>(a.QKV + row * 3 * a.D + hh * DH, vq, scale, q);
            put_row<DH>(Qs, tid, q);
            load_row<DH>(a.dO + row * a.D + hh * DH, vq, 1.f, g);
            put_row<DH>(Gs, tid, g);
            load_row<DH>(a.O + row * a.D + hh * DH, vq, 1.f, o);
#pragma unroll
            for (int j = 0; j < DH; ++j) dd += g[j] * o[j];
            if (vq) {
                a.Dt[row * a.NH + hh] = dd;
                lse = a.LSE[row * a.NH + hh];
            }
        }
        float dq[DH];
#pragma unroll
        for (int j = 0; j < DH; ++j) dq[j] = 0.f;
        for (int kb = 0; kb <= qt; ++kb) {
            if (!block_visible(a, qt, kb)) continue;
            {
                const int k = kb * kT + tid;
                const bool vk = k < a.N;
                const float *src = a.QKV + (b * a.N + k) * 3 * a.D + hh * DH;
                float v[DH];
                load_row<DH>(src + a.D, vk, 1.f, v);
                put_row<DH>(Ks, tid, v);
                put_col<DH>(Kt, tid, v);
                load_row<DH>(src + 2 * a.D, vk, 1.f, v);
                put_row<DH>(Vs, tid, v);
            }
            tc::fence_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc::tc_fence_after();
                mma_tile(tmem, Qs, KG, Ks, KG, kT, DH / 16, false);        // S
                mma_tile(tmem + kT, Gs, KG, Vs, KG, kT, DH / 16, false);   // dP
                tc::mma_commit(&bar);
            }
            __syncwarp();
            if (!wait_mma(&bar, phase, a.err, 33)) s_err = 1;
            tc::tc_fence_after();
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                float s[32], dp[32];
                tc::tmem_ld32(tmem + lanes + 32 * c, s);
                tc::tmem_ld32(tmem + lanes + kT + 32 * c, dp);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int k = kb * kT + 32 * c + j;
                    const bool vis = vq && k < a.N && key_visible(a.mask, a.W, a.S, t, k);
                    const float p = vis ? __expf(s[j] - lse) : 0.f;
                    s[j] = p * (dp[j] - dd);
                }
                put_row32(dS, tid, 32 * c, s);
            }
            tc::fence_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            if (tid == 0 && !s_err) {
                tc::tc_fence_after();
                mma_tile(tmem, dS, kT / 8, Kt, kT / 8, DH, kT / 16, false);  // dS K
                tc::mma_commit(&bar);
            }
            __syncwarp();
            if (!s_err && !wait_mma(&bar, phase, a.err, 34)) s_err = 1;
            tc::tc_fence_after();
            {
                float ob[32];
                if (DH == 16) {
                    float h[16];
                    tc::tmem_ld16(tmem + lanes, h);
#pragma unroll
                    for (int j = 0; j < 16; ++j) ob[j] = h[j];
                } else {
                    tc::tmem_ld32(tmem + lanes, ob);
                }
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < DH; ++j) dq[j] += ob[j];
            }
            tc::tc_fence_before();
            __syncthreads();
            if (s_err) break;
        }
        if (vq) {
            float4 *dst = reinterpret_cast<float4 *>(a.dQKV + row * 3 * a.D + hh * DH);
#pragma unroll
            for (int c = 0; c < DH / 4; ++c)
                dst[c] = make_float4(dq[4 * c] * scale, dq[4 * c + 1] * scale, dq[4 * c + 2] * scale,
                                     dq[4 * c + 3] * scale);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (tid < 32) tc::tmem_dealloc(tmem, 256);
}

// dK/dV pass over key blocks.  TMEM: S^T at [0, 128), dP^T at [128, 256);
// the dV and dK block products reuse [0, DH) and [32, 32 + DH).
template <int DH>
__global__ void __launch_bounds__(128) attn_bwd_dkv_tc_kernel(const __grid_constant__ AttnArgs a)
{
    constexpr int KG = DH / 8;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Ks = smem;               // [128 keys x DH]
    unsigned char *Vs = Ks + kT * DH * 2;   // [128 keys x DH]
    unsigned char *Qs = Vs + kT * DH * 2;   // [128 q x DH] (scaled)
    unsigned char *Qt = Qs + kT * DH * 2;   // [DH x 128 q] (scaled)
    unsigned char *Gs = Qt + kT * DH * 2;   // [128 q x DH] dO
    unsigned char *Gt = Gs + kT * DH * 2;   // [DH x 128 q]
    unsigned char *Pt = Gt + kT * DH * 2;   // [128 keys x 128 q]
    unsigned char *dSt = Pt + kT * kT * 2;  // [128 keys x 128 q]
    float *Ls = reinterpret_cast<float *>(dSt + kT * kT * 2);  // [128]
    float *Ds = Ls + kT;                                       // [128]
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ int s_err;
    const int tid = threadIdx.x;
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
        s_err = 0;
    }
    if (tid < 32) {
        tc::tmem_alloc(&tslot, 256);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tslot, lanes = (uint32_t)(32 * (tid >> 5)) << 16;
    uint32_t phase = 0;
    const float scale = rsqrtf((float)DH);
    const int nkb = (a.N + kT - 1) / kT;
    const int64_t units = (int64_t)a.B * a.NH * nkb;

    for (int64_t u = blockIdx.x; u < units && !s_err; u += gridDim.x) {
        const int kb = (int)(u % nkb);
        const int hh = (int)((u / nkb) % a.NH);
        const int64_t b = u / ((int64_t)nkb * a.NH);
        const int k = kb * kT + tid;
        const bool vk = k < a.N;
        {
            const float *src = a.QKV + (b * a.N + k) * 3 * a.D + hh * DH;
            float v[DH];
            load_row<DH>(src + a.D, vk, 1.f, v);
            put_row<DH>(Ks, tid, v);
            load_row<DH>(src + 2 * a.D, vk, 1.f, v);
            put_row<DH>(Vs, tid, v);
        }
        float dk[DH], dv[DH];
#pragma unroll
        for (int j = 0; j < DH; ++j) dk[j] = dv[j] = 0.f;
        const int qt_hi = last_query_tile(a, kb);
        for (int qt = kb; qt <= qt_hi; ++qt) {
            {
                const int t = qt * kT + tid;
                const bool vq = t < a.N;
                const int64_t row = b * a.N + t;
                float q[DH];
                load_row<DH>(a.QKV + row * 3 * a.D + hh * DH, vq, scale, q);
                put_row<DH>(Qs, tid, q);
                put_col<DH>(Qt, tid, q);
                load_row<DH>(a.dO + row * a.D + hh * DH, vq, 1.f, q);
                put_row<DH>(Gs, tid, q);
                put_col<DH>(Gt, tid, q);
                Ls[tid] = vq ? a.LSE[row * a.NH + hh] : 0.f;
                Ds[tid] = vq ? a.Dt[row * a.NH + hh] : 0.f;
            }
            tc::fence_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc::tc_fence_after();
                mma_tile(tmem, Ks, KG, Qs, KG, kT, DH / 16, false);        // S^T
                mma_tile(tmem + kT, Vs, KG, Gs, KG, kT, DH / 16, false);   // dP^T
                tc::mma_commit(&bar);
            }
            __syncwarp();
            if (!wait_mma(&bar, phase, a.err, 35)) s_err = 1;
            tc::tc_fence_after();
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                float s[32], dp[32];
                tc::tmem_ld32(tmem + lanes + 32 * c, s);
                tc::tmem_ld32(tmem + lanes + kT + 32 * c, dp);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int tq = 32 * c + j, t = qt * kT + tq;
                    const bool vis = vk && t < a.N && key_visible(a.mask, a.W, a.S, t, k);
                    const float p = vis ? __expf(s[j] - Ls[tq]) : 0.f;
                    s[j] = p;
                    dp[j] = p * (dp[j] - Ds[tq]);
                }
                put_row32(Pt, tid, 32 * c, s);
                put_row32(dSt, tid, 32 * c, dp);
            }
            tc::fence_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            if (tid == 0 && !s_err) {
                tc::tc_fence_after();
                mma_tile(tmem, Pt, kT / 8, Gt, kT / 8, DH, kT / 16, false);        // P^T dO
                mma_tile(tmem + 32, dSt, kT / 8, Qt, kT / 8, DH, kT / 16, false);  // dS^T Q
                tc::mma_commit(&bar);
            }
            __syncwarp();
            if (!s_err && !wait_mma(&bar, phase, a.err, 36)) s_err = 1;
            tc::tc_fence_after();
            {
                float xv[32], xk[32];
                if (DH == 16) {
                    float h[16], g[16];
                    tc::tmem_ld16(tmem + lanes, h);
                    tc::tmem_ld16(tmem + lanes + 32, g);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        xv[j] = h[j];
                        xk[j] = g[j];
                    }
                } else {
                    tc::tmem_ld32(tmem + lanes, xv);
                    tc::tmem_ld32(tmem + lanes + 32, xk);
                }
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < DH; ++j) {
                    dv[j] += xv[j];
                    dk[j] += xk[j];
                }
            }
            tc::tc_fence_before();
            __syncthreads();
            if (s_err) break;
        }
        if (vk) {
            float *dst = a.dQKV + (b * a.N + k) * 3 * a.D + hh * DH;
#pragma unroll
            for (int c = 0; c < DH / 4; ++c) {
                reinterpret_cast<float4 *>(dst + a.D)[c] =
                    make_float4(dk[4 * c], dk[4 * c + 1], dk[4 * c + 2], dk[4 * c + 3]);
                reinterpret_cast<float4 *>(dst + 2 * a.D)[c] =
                    make_float4(dv[4 * c], dv[4 * c + 1], dv[4 * c + 2], dv[4 * c + 3]);
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (tid < 32) tc::tmem_dealloc(tmem, 256);
}

// Dynamic shared memory that lets at most n CTAs share an SM, so that every
// resident CTA's TMEM allocation succeeds at once (n CTAs x columns <= 512).
size_t at_most(size_t need, int n)
{
    int dev = 0, per_sm = 228 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    return std::max(need, (size_t)per_sm / (n + 1) + 1);
}

int grid_of(int64_t units, int per_sm)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (int)std::max<int64_t>(1, std::min<int64_t>(units, (int64_t)sms * per_sm));
}

AttnArgs args_of(const sg_config &c, int Bc, int *err)
{
    AttnArgs a{};
    a.B = Bc;
    a.N = c.N;
    a.D = c.d;
    a.NH = c.n_heads;
    a.mask = c.mask_kind;
    a.W = c.W;
    a.S = c.S;
    a.err = err;
    return a;
}

template <int DH>
sg_status fwd_tc(const AttnArgs &a, cudaStream_t st)
{
    const size_t smem = at_most((size_t)3 * kT * DH * 2 + (size_t)kT * kT * 2, 4);
    const int64_t units = (int64_t)a.B * a.NH * ((a.N + kT - 1) / kT);
    SG_CUDA_TRY(cudaFuncSetAttribute(attn_fwd_tc_kernel<DH>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attn_fwd_tc_kernel<DH><<<grid_of(units, 4), 128, smem, ::sg::counted(st)>>>(a);
    return check_launch("attn_fwd_tc_kernel");
}

template <int DH>
sg_status bwd_tc(const AttnArgs &a, cudaStream_t st)
{
    const int nt = (a.N + kT - 1) / kT;
    const int64_t units = (int64_t)a.B * a.NH * nt;
    const size_t smem_dq = at_most((size_t)5 * kT * DH * 2 + (size_t)kT * kT * 2, 2);
    SG_CUDA_TRY(cudaFuncSetAttribute(attn_bwd_dq_tc_kernel<DH>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_dq));
    attn_bwd_dq_tc_kernel<DH><<<grid_of(units, 2), 128, smem_dq, ::sg::counted(st)>>>(a);
    SG_TRY(check_launch("attn_bwd_dq_tc_kernel"));
    const size_t smem_kv =
        at_most((size_t)6 * kT * DH * 2 + (size_t)2 * kT * kT * 2 + 2 * kT * sizeof(float), 2);
    SG_CUDA_TRY(cudaFuncSetAttribute(attn_bwd_dkv_tc_kernel<DH>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_kv));
    attn_bwd_dkv_tc_kernel<DH><<<grid_of(units, 2), 128, smem_kv, ::sg::counted(st)>>>(a);
    return check_launch("attn_bwd_dkv_tc_kernel");
}

}  // namespace

// The BF16 model's teacher-forced attention runs on the tensor cores when
// d_h is 16 or 32 and a query sees many keys (dense, or a band + sink of 64
// keys or more, or N beyond the shared-memory CUDA-core kernels).  Narrow
// bands waste most of a 128 x 128 score tile, and the CUDA-core kernels that
// walk only the visible keys are faster there.
bool attn_tc_supported(const sg_config &c)
{
    const int dh = c.d / c.n_heads;
    if (c.precision != SG_BF16 || (dh != 16 && dh != 32)) return false;
    const int64_t keys = c.mask_kind == SG_MASK_DENSE ? c.N / 2
                                                     : std::min<int64_t>(c.N, (int64_t)c.W + 1 + c.S);
    return c.N > 512 || keys >= 64;
}

sg_status launch_attn_fwd_tc(const sg_config &c, const float *QKV, const float *Hin, float *O,
                             float *Hmid, float *LSE, int Bc, int *err, cudaStream_t st)
{
    AttnArgs a = args_of(c, Bc, err);
    a.QKV = QKV;
    a.Hin = Hin;
    a.O_out = O;
    a.Hmid = Hmid;
    a.LSE_out = LSE;
    return c.d / c.n_heads == 16 ? fwd_tc<16>(a, st) : fwd_tc<32>(a, st);
}

sg_status launch_attn_bwd_tc(const sg_config &c, const float *QKV, const float *O, const float *dO,
                             const float *LSE, float *dQKV, float *Dt, int Bc, int *err,
                             cudaStream_t st)
{
    AttnArgs a = args_of(c, Bc, err);
    a.QKV = QKV;
    a.O = O;
    a.dO = dO;
    a.LSE = LSE;
    a.dQKV = dQKV;
    a.Dt = Dt;
    return c.d / c.n_heads == 16 ? bwd_tc<16>(a, st) : bwd_tc<32>(a, st);
}

}  // namespace sg
