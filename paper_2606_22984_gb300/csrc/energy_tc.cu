// energy_tc.cu -- SK energy (Eq. SKHam) on tcgen05 tensor cores.
//
// E_b = -1/2 sum_i s_bi (J s_b)_i with J symmetric and zero on the diagonal
// (each pair i < j counted once).  The contraction Y = S J runs as a GEMM on
// tiled BF16 operands: S holds the spins (+-1, exact in BF16) and J is split
// into two BF16 terms, J = J_hi + J_lo, both multiplied into the same FP32
// TMEM accumulator, so the product carries about 16 mantissa bits of J.  The
// epilogue forms the row dot with the spins and adds -1/2 of it to E_b.
//
// Persistent over the SMs.  A work unit is one 64-wide K chunk of one tile
// (128 samples x 256 columns of Y): unit u = tile * KC + kc with tile =
// rb * CB + cb.  CTA i of G takes the units [U i / G, U (i + 1) / G), so every
// SM does the same number of MMAs whatever the tile count; a tile split
// between two CTAs is summed by both into E_b (the energy is linear in Y).
// Warp 0 streams the S tile and the J_hi / J_lo tiles of each unit through two
// shared-memory stages, warp 1 issues the MMAs into one of two TMEM
// accumulators (alternating per tile segment), and warps 2-5 run the
// epilogue of one segment while the MMAs of the next run.
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
    int CB;                    // column blocks of Y (N / 256)
    int N;
    int64_t U;                 // work units: RB * CB * KC
    const int8_t *spins;
    int64_t B;
    float *E;
    int *err;
};

constexpr int kSkStages = 2;
constexpr uint32_t kSkStage = 5 * 16384;  // S tile + 2 J_hi tiles + 2 J_lo tiles

// VEC: the spin rows are 16-byte aligned (spins pointer aligned, N a multiple
// of 256), so the epilogue fetches a row's 256 spins as 16 vector loads.
template <bool VEC>
__global__ void __launch_bounds__(192, 1) sk_energy_tc_kernel(const __grid_constant__ SkArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t full[kSkStages], empty[kSkStages], acc_full[2], acc_empty[2], done;
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t u0 = a.U * blockIdx.x / gridDim.x, u1 = a.U * (blockIdx.x + 1) / gridDim.x;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kSkStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int x = 0; x < 2; ++x) {
            tc::mbar_init(&acc_full[x], 1);
            tc::mbar_init(&acc_empty[x], 128);
        }
        tc::mbar_init(&done, 1);
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(&tslot, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tslot;
    // Launched as a programmatic dependent of the spin conversion: the setup
    // above overlaps the conversion's tail, and nothing below (S tiles, E)
    // is touched before the conversion has completed and its writes are
    // visible.  Without that launch attribute the wait returns at once.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (warp == 0 && lane == 0) {
        // Chunk j of this CTA uses stage j % 2; its refill waits for the MMAs
        // of chunk j - 2 (completion (j - 2) / 2 of that stage's empty
        // barrier).  (rb, cb, kc) of unit u are stepped without divisions: a
        // refill is issued right after a stage frees, so its address math is
        // on the critical path.
        int64_t rb = (u0 / a.KC) / a.CB;
        int cb = (int)((u0 / a.KC) % a.CB), kc = (int)(u0 % a.KC);
        int64_t j = 0;
        for (int64_t u = u0; u < u1; ++u, ++j) {
            const int s = (int)(j & 1);
            if (j >= kSkStages && !tc::mbar_wait(&empty[s], (uint32_t)(((j >> 1) - 1) & 1))) {
                atomicExch(a.err, 31);
                break;
            }
            unsigned char *dst = smem + (size_t)s * kSkStage;
            tc::mbar_arrive_expect_tx(&full[s], kSkStage);
            tc::bulk_g2s(dst, a.S + ((size_t)(kc * a.RB + rb) << 14), 16384, &full[s]);
            const size_t jt = (size_t)(kc * a.NRB + 2 * cb) << 14;  // two adjacent row blocks
            tc::bulk_g2s(dst + 16384, a.Jhi + jt, 32768, &full[s]);
            tc::bulk_g2s(dst + 49152, a.Jlo + jt, 32768, &full[s]);
            if (++kc == a.KC) {
                kc = 0;
                if (++cb == a.CB) {
                    cb = 0;
                    ++rb;
                }
            }
        }
        // no copy may still be landing when the CTA exits (after a time-out):
        // wait for the last fill of each stage
        for (int s = 0; s < kSkStages; ++s) {
            const int64_t last = (j - 1 - s) >= 0 ? ((j - 1 - s) & ~(int64_t)1) + s : -1;
            if (last >= 0) tc::mbar_wait(&full[s], (uint32_t)((last >> 1) & 1), 1u << 22);
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = tc::idesc_bf16(128, 256);
        bool ok = true;
        int64_t j = 0;
        int seg = 0;
        int kc0 = (int)(u0 % a.KC);  // K chunk of the segment's first unit
        for (int64_t u = u0; u < u1; ++seg, kc0 = 0) {
            const int64_t uend = min(u1, u + (a.KC - kc0));  // this tile's units
            const int acc = seg & 1;
            // the accumulator's previous segment (seg - 2) has been read out
            if (seg >= 2 && !tc::mbar_wait(&acc_empty[acc], (uint32_t)(((seg >> 1) + 1) & 1))) {
                ok = false;
                break;
            }
            tc::tc_fence_after();
            const uint32_t d = tmem + 256 * acc;
            for (bool first = true; u < uend; ++u, ++j, first = false) {
                const int s = (int)(j & 1);
                if (!tc::mbar_wait(&full[s], (uint32_t)((j >> 1) & 1))) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t sa = tc::smem_u32(smem + (size_t)s * kSkStage);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t ad = tc::smem_desc(sa + 256 * ks, 128, 1024);
                    tc::mma_bf16(d, ad, tc::smem_desc(sa + 16384 + 256 * ks, 128, 1024), idesc,
                                 (first && ks == 0) ? 0u : 1u);
                    tc::mma_bf16(d, ad, tc::smem_desc(sa + 49152 + 256 * ks, 128, 1024), idesc, 1u);
                }
                tc::mma_commit(&empty[s]);
            }
            if (!ok) break;
            tc::mma_commit(&acc_full[acc]);
        }
        if (!ok) atomicExch(a.err, 32);
        // every MMA of this thread has completed before TMEM is freed
        tc::mma_commit(&done);
        tc::mbar_wait(&done, 0, 1u << 22);
    } else if (warp >= 2) {
        const int q = warp & 3;
        int seg = 0;
        int64_t tile = u0 / a.KC, rb = tile / a.CB;
        int cb = (int)(tile % a.CB);
        for (int64_t u = u0; u < u1; ++seg) {
            u = min(u1, (tile + 1) * a.KC);
            const int64_t b = rb * 128 + 32 * q + lane;
            // The row's 256 spins of this column block, fetched while the
            // MMAs run.  A warp's load touches 32 rows, so byte loads would
            // cost 32 L1 wavefronts per spin; 16-byte loads cost 16 per row.
            uint4 sv[16];
            if constexpr (VEC) {
                const uint4 *src =
                    reinterpret_cast<const uint4 *>(a.spins + (b < a.B ? b : 0) * a.N + 256 * cb);
#pragma unroll
                for (int x = 0; x < 16; ++x) sv[x] = __ldg(src + x);
            }
            const int acc = seg & 1;
            if (!tc::mbar_wait(&acc_full[acc], (uint32_t)((seg >> 1) & 1))) {
                if (lane == 0) atomicExch(a.err, 33);
                break;
            }
            tc::tc_fence_after();
            float part = 0.f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 256 * acc + 32 * c, v);
                tc::tmem_wait_ld();
                if constexpr (VEC) {
                    const uint32_t w[8] = {sv[2 * c].x,     sv[2 * c].y,     sv[2 * c].z,     sv[2 * c].w,
                                           sv[2 * c + 1].x, sv[2 * c + 1].y, sv[2 * c + 1].z, sv[2 * c + 1].w};
#pragma unroll
                    for (int x = 0; x < 32; ++x)
                        part += (float)(int8_t)(w[x >> 2] >> (8 * (x & 3))) * v[x];
                } else if (b < a.B) {
                    const int8_t *sp = a.spins + b * a.N + 256 * cb + 32 * c;
#pragma unroll
                    for (int x = 0; x < 32; ++x) part += (float)sp[x] * v[x];
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&acc_empty[acc]);
            if (b < a.B) atomicAdd(a.E + b, -0.5f * part);
            ++tile;
            if (++cb == a.CB) {
                cb = 0;
                ++rb;
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// BF16 of two int8 values (given as bytes lo, hi), packed lo | hi << 16, with
// integer and FP32-add operations only: the float with bits
// 0x4B000000 | (b ^ 0x80) is 2^23 + 128 + int8(b), so subtracting 2^23 + 128
// leaves int8(b) exactly; every int8 has at most 8 significant bits, so its
// BF16 is the float's upper half.
__device__ __forceinline__ uint32_t bf16_pair_of_bytes(uint32_t lo, uint32_t hi)
{
    const float fl = __uint_as_float((lo ^ 0x80u) | 0x4B000000u) - 8388736.0f;
    const float fh = __uint_as_float((hi ^ 0x80u) | 0x4B000000u) - 8388736.0f;
    return __byte_perm(__float_as_uint(fl), __float_as_uint(fh), 0x7632);
}

// spins int8 [B][N] -> T(B, N) BF16 (+-1; zero padding), and E[b] = 0 for
// the energy kernel's sums.  Thread (r, kc) converts row r's 64 spins of K
// chunk kc; rows run fastest, so the 8 threads of an 8-row group fill a
// core-matrix column's 128 contiguous bytes with each store.  VEC: 16-byte
// aligned rows (read as 4 vector loads).
template <bool VEC>
__global__ void spins_to_tiled_kernel(const int8_t *__restrict__ spins, int64_t B, int N,
                                      unsigned char *__restrict__ dst, float *__restrict__ E)
{
    // the energy kernel may be scheduled once every block of this grid runs;
    // it waits for this grid's completion before reading S or E
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int64_t RB = tl_blocks(B), rows = RB * 128;
    const int KC = (N + 63) >> 6;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * KC) return;
    const int64_t r = i % rows;
    const int kc = (int)(i / rows);
    if (kc == 0 && r < B) E[r] = 0.f;
    uint32_t w[16];  // the 64 spins, 4 per word
    if (VEC && r < B && 64 * kc + 64 <= N) {
        const uint4 *src = reinterpret_cast<const uint4 *>(spins + r * N + 64 * kc);
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const uint4 v = __ldg(src + x);
            w[4 * x] = v.x;
            w[4 * x + 1] = v.y;
            w[4 * x + 2] = v.z;
            w[4 * x + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int x = 0; x < 16; ++x) {
            uint32_t u = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 64 * kc + 4 * x + e;
                if (r < B && k < N) u |= (uint32_t)(uint8_t)spins[r * N + k] << (8 * e);
            }
            w[x] = u;
        }
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        uint32_t h[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const uint32_t u = w[2 * g + (p >> 1)] >> (16 * (p & 1));
            h[p] = bf16_pair_of_bytes(u & 0xff, (u >> 8) & 0xff);
        }
        *reinterpret_cast<uint4 *>(dst + tl_offset(r, 64 * kc + 8 * g, RB)) = make_uint4(h[0], h[1], h[2], h[3]);
    }
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
    const bool vec = (uintptr_t)spins % 16 == 0;  // N is a multiple of 256
    const int64_t n = tl_blocks(B) * 128 * ((N + 63) >> 6);
    if (vec)
        spins_to_tiled_kernel<true><<<(unsigned)((n + 255) / 256), 256, 0, ::sg::counted(st)>>>(spins, B, N, S, E);
    else
        spins_to_tiled_kernel<false><<<(unsigned)((n + 255) / 256), 256, 0, ::sg::counted(st)>>>(spins, B, N, S, E);
    SG_TRY(check_launch("spins_to_tiled_kernel"));
    SkArgs a{};
    a.S = S;
    a.RB = tl_blocks(B);
    a.Jhi = (const unsigned char *)inst->Jbf;
    a.Jlo = a.Jhi + tl_bytes(N, N);
    a.NRB = (int)tl_blocks(N);
    a.KC = N / 64;
    a.CB = N / 256;
    a.N = N;
    a.U = a.RB * a.CB * a.KC;
    a.spins = spins;
    a.B = B;
    a.E = E;
    a.err = err;
    const size_t smem = (size_t)kSkStages * kSkStage;
    // one CTA per SM (the stages take 160 KB), never more CTAs than units
    int dev = 0, sms = 0;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    SG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)std::min<int64_t>(sms, a.U);
    auto go = [&](auto kern) -> sg_status {
        SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        // may start while the conversion still runs (it waits for it first)
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(192);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = ::sg::counted(st);
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        SG_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, a));
        return check_launch("sk_energy_tc_kernel");
    };
    return vec ? go(sk_energy_tc_kernel<true>) : go(sk_energy_tc_kernel<false>);
}

}  // namespace sg
