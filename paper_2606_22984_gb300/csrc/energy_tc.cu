// energy_tc.cu -- SK energy (Eq. SKHam) on tcgen05 tensor cores.
//
// E_b = -1/2 sum_i s_bi (J s_b)_i with J symmetric and zero on the diagonal
// (each pair i < j counted once).  The contraction Y = S J runs as a GEMM on
// tiled BF16 operands: S holds the spins (+-1, exact in BF16) and J is split
// into two BF16 terms, J = J_hi + J_lo, both multiplied into the same FP32
// TMEM accumulator, so the product carries about 16 mantissa bits of J.  The
// epilogue forms the row dot with the spins and adds -1/2 of it to E_b.
//
// One CTA per (128-sample block, 256-column block of Y): warp 0 streams the S
// tile and the J_hi / J_lo tiles of each 64-wide K chunk through two
// shared-memory stages, warp 1 issues the MMAs, warps 2-5 run the epilogue.
#include <cuda_bf16.h>

#include "gemm_tc.cuh"

namespace sg {

namespace {

struct SkArgs {
    const unsigned char *S;    // T(B, N) spins as BF16
    int64_t RB;                // row blocks of S
    const unsigned char *Jhi;  // T(N, N)
    const unsigned char *Jlo;  // T(N, N)
    int NRB;                   // row blocks of J
    int KC;                    // K chunks (N / 64)
    int N;
    const int8_t *spins;
    int64_t B;
    float *E;
    int *err;
};

constexpr int kSkStages = 2;
constexpr uint32_t kSkStage = 5 * 16384;  // S tile + 2 J_hi tiles + 2 J_lo tiles

__global__ void __launch_bounds__(192, 1) sk_energy_tc_kernel(const __grid_constant__ SkArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t full[kSkStages], empty[kSkStages], tfull;
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t rb = blockIdx.x / (a.N / 256);
    const int cb = (int)(blockIdx.x % (a.N / 256));
    if (threadIdx.x == 0) {
        for (int s = 0; s < kSkStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(&tfull, 1);
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(&tslot, 256);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tslot;
    if (warp == 0 && lane == 0) {
        for (int kc = 0; kc < a.KC; ++kc) {
            const int s = kc % kSkStages;
            if (kc >= kSkStages &&
                !tc::mbar_wait(&empty[s], (uint32_t)((kc / kSkStages - 1) & 1))) {
                atomicExch(a.err, 31);
                break;
            }
            unsigned char *dst = smem + (size_t)s * kSkStage;
            tc::mbar_arrive_expect_tx(&full[s], kSkStage);
            tc::bulk_g2s(dst, a.S + ((size_t)(kc * a.RB + rb) << 14), 16384, &full[s]);
            const size_t jt = (size_t)(kc * a.NRB + 2 * cb) << 14;  // two adjacent row blocks
            tc::bulk_g2s(dst + 16384, a.Jhi + jt, 32768, &full[s]);
            tc::bulk_g2s(dst + 49152, a.Jlo + jt, 32768, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = tc::idesc_bf16(128, 256);
        bool ok = true;
        for (int kc = 0; kc < a.KC; ++kc) {
            const int s = kc % kSkStages;
            if (!tc::mbar_wait(&full[s], (uint32_t)((kc / kSkStages) & 1))) {
                ok = false;
                break;
            }
            tc::tc_fence_after();
            const uint32_t sa = tc::smem_u32(smem + (size_t)s * kSkStage);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint64_t ad = tc::smem_desc(sa + 256 * ks, 128, 1024);
                tc::mma_bf16(tmem, ad, tc::smem_desc(sa + 16384 + 256 * ks, 128, 1024), idesc,
                             (kc | ks) != 0 ? 1u : 0u);
                tc::mma_bf16(tmem, ad, tc::smem_desc(sa + 49152 + 256 * ks, 128, 1024), idesc, 1u);
            }
            tc::mma_commit(&empty[s]);
        }
        if (!ok) atomicExch(a.err, 32);
        tc::mma_commit(&tfull);
    } else if (warp >= 2) {
        const int q = warp & 3;
        const int64_t b = rb * 128 + 32 * q + lane;
        if (tc::mbar_wait(&tfull, 0)) {
            tc::tc_fence_after();
            float part = 0.f;
            for (int c = 0; c < 8; ++c) {
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 32 * c, v);
                tc::tmem_wait_ld();
                if (b < a.B) {
                    const int8_t *sp = a.spins + b * a.N + 256 * cb + 32 * c;
#pragma unroll
                    for (int j = 0; j < 32; ++j) part += (float)sp[j] * v[j];
                }
            }
            if (b < a.B) atomicAdd(a.E + b, -0.5f * part);
        } else if (lane == 0) {
            atomicExch(a.err, 33);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, 256);
}

// spins int8 [B][N] -> T(B, N) BF16 (+-1; zero padding)
__global__ void spins_to_tiled_kernel(const int8_t *__restrict__ spins, int64_t B, int N,
                                      unsigned char *__restrict__ dst)
{
    const int64_t RB = tl_blocks(B);
    const int groups = ((N + 63) >> 6) * 8;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= RB * 128 * groups) return;
    const int64_t r = i / groups;
    const int kg = (int)(i % groups);
    uint32_t w[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        float v[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int k = kg * 8 + 2 * p + e;
            v[e] = (r < B && k < N) ? (float)spins[r * N + k] : 0.f;
        }
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[0], v[1]);
        w[p] = *reinterpret_cast<const uint32_t *>(&h);
    }
    *reinterpret_cast<uint4 *>(dst + tl_offset(r, kg * 8, RB)) = make_uint4(w[0], w[1], w[2], w[3]);
}

// J [N][N] fp32 -> T(N, N) of bf16(J) and of bf16(J - bf16(J))
__global__ void jsplit_tiled_kernel(const float *__restrict__ J, int N, unsigned char *__restrict__ hi,
                                    unsigned char *__restrict__ lo)
{
    const int64_t RB = tl_blocks(N);
    const int groups = ((N + 63) >> 6) * 8;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= RB * 128 * groups) return;
    const int64_t r = i / groups;
    const int kg = (int)(i % groups);
    uint32_t wh[4], wl[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        float h[2], l[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int k = kg * 8 + 2 * p + e;
            const float x = (r < N && k < N) ? J[r * N + k] : 0.f;
            h[e] = __bfloat162float(__float2bfloat16(x));
            l[e] = x - h[e];
        }
        const __nv_bfloat162 vh = __floats2bfloat162_rn(h[0], h[1]);
        const __nv_bfloat162 vl = __floats2bfloat162_rn(l[0], l[1]);
        wh[p] = *reinterpret_cast<const uint32_t *>(&vh);
        wl[p] = *reinterpret_cast<const uint32_t *>(&vl);
    }
    const size_t off = tl_offset(r, kg * 8, RB);
    *reinterpret_cast<uint4 *>(hi + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
    *reinterpret_cast<uint4 *>(lo + off) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
}

}  // namespace

bool sk_tc_supported(int N) { return N >= 256 && N % 256 == 0; }

sg_status prepare_sk_tc(sg_instance *inst)
{
    if (!sk_tc_supported(inst->N)) return SG_OK;
    const size_t bytes = tl_bytes(inst->N, inst->N);
    size_t have = 0;
    SG_TRY(ensure_buffer(&inst->Jbf, &have, 2 * bytes));
    unsigned char *hi = (unsigned char *)inst->Jbf, *lo = hi + bytes;
    const int64_t n = tl_blocks(inst->N) * 128 * (((inst->N + 63) >> 6) * 8);
    jsplit_tiled_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ::sg::counted(nullptr)>>>(
        inst->J, inst->N, hi, lo);
    SG_TRY(check_launch("jsplit_tiled_kernel"));
    SG_CUDA_TRY(cudaDeviceSynchronize());
    return SG_OK;
}

sg_status launch_energy_sk_tc(const sg_instance *inst, const int8_t *spins, int64_t B, float *E,
                              void **ws, size_t *ws_bytes, int *err, cudaStream_t st)
{
    const int N = inst->N;
    const size_t sbytes = tl_bytes(B, N);
    SG_TRY(ensure_buffer(ws, ws_bytes, sbytes));
    unsigned char *S = (unsigned char *)*ws;
    const int64_t n = tl_blocks(B) * 128 * (((N + 63) >> 6) * 8);
    spins_to_tiled_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ::sg::counted(st)>>>(spins, B, N, S);
    SG_CUDA_TRY(cudaMemsetAsync(E, 0, (size_t)B * sizeof(float), st));
    SkArgs a{};
    a.S = S;
    a.RB = tl_blocks(B);
    a.Jhi = (const unsigned char *)inst->Jbf;
    a.Jlo = a.Jhi + tl_bytes(N, N);
    a.NRB = (int)tl_blocks(N);
    a.KC = N / 64;
    a.N = N;
    a.spins = spins;
    a.B = B;
    a.E = E;
    a.err = err;
    const size_t smem = (size_t)kSkStages * kSkStage;
    SG_CUDA_TRY(cudaFuncSetAttribute(sk_energy_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    sk_energy_tc_kernel<<<(unsigned)(a.RB * (N / 256)), 192, smem, ::sg::counted(st)>>>(a);
    return check_launch("sk_energy_tc_kernel");
}

}  // namespace sg
