// gemm_tc.cu -- tcgen05 GEMMs for the BF16 teacher-forced pass and backward.
//
// row_gemm_kernel: C[R][N] = A[R][K] B[N][K]^T with a fused epilogue.  A
// persistent CTA walks row blocks of 128; warp 0 streams A tiles by bulk copy
// into two shared-memory stages, warp 1 issues the MMAs into one of two TMEM
// accumulators, warps 2-5 drain the other accumulator through the epilogue.
// B (the weights, <= 256 x 256) stays resident in shared memory.  Larger
// weights go through tile_gemm_kernel (column blocks of 256, A and B streamed).
//
// wgrad_kernel: C[M][N] += A[M][Kr] B[N][Kr]^T, a split-K reduction over the
// batch rows for weight gradients: each CTA owns one 128-row block of C and a
// range of K chunks, pipelines them through four stages, and adds its TMEM
// accumulator to C with atomics.
//
// Every wait is bounded; on a timeout the kernel sets the error word and the
// roles stop issuing work.
#include <cuda_bf16.h>

#include <algorithm>

#include "gemm_tc.cuh"

namespace sg {

namespace {

__device__ __forceinline__ uint32_t pk2(float a, float b)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void st8(unsigned char *base, size_t off, const float *v)
{
    uint4 q;
    q.x = pk2(v[0], v[1]);
    q.y = pk2(v[2], v[3]);
    q.z = pk2(v[4], v[5]);
    q.w = pk2(v[6], v[7]);
    *reinterpret_cast<uint4 *>(base + off) = q;
}

__device__ __forceinline__ void ld8(const unsigned char *base, size_t off, float *v)
{
    const uint4 q = *reinterpret_cast<const uint4 *>(base + off);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        v[2 * i] = __uint_as_float(w[i] << 16);
        v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
}

// Column sums of a warp's 32 x 32 block (lane = row): a reduce-scatter
// butterfly leaves lane j with the sum of column j (31 shuffles).
__device__ __forceinline__ float warp_colsum32(float (&y)[32])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const bool upper = lane & o;
#pragma unroll
        for (int j = 0; j < o; ++j) {
            const float send = upper ? y[j] : y[j + o];
            const float recv = __shfl_xor_sync(0xffffffffu, send, o);
            y[j] = (upper ? y[j + o] : y[j]) + recv;
        }
    }
    return y[0];
}

constexpr int kColsumMax = 1024;

// Bulk prefetch of [p, p + bytes) into L2 (one thread; bytes a multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The epilogue inputs of row block rb that are read from global memory (each
// one contiguous range), prefetched into L2 while an earlier block is drained.
template <int EPI>
__device__ __forceinline__ void prefetch_epilogue(const RowGemm &g, int64_t rb)
{
    if (rb >= g.RB) return;
    const int64_t r0 = rb * 128, rows = min((int64_t)128, g.R - r0);
    if (rows <= 0) return;
    if (EPI == TE_LN_BWD) {
        prefetch_l2(g.ln_x + r0 * g.N, (uint32_t)(rows * g.N * 4));
        if (g.ln_dres) prefetch_l2(g.ln_dres + r0 * g.N, (uint32_t)(rows * g.N * 4));
        // whole 16-byte pieces only: the statistics end with the rows
        const uint32_t sb = (uint32_t)((rows * 4) & ~int64_t(15));
        if (sb) {
            prefetch_l2(g.ln_mu + r0, sb);
            prefetch_l2(g.ln_rs + r0, sb);
        }
    } else if (EPI == TE_RESID_F32) {
        if (g.ld_resid == g.N) prefetch_l2(g.resid + r0 * g.N, (uint32_t)(rows * g.N * 4));
    } else if (EPI == TE_GELU_BWD_T) {
        prefetch_l2(g.aux_t + (size_t)rb * wl_block_bytes(g.N), (uint32_t)wl_block_bytes(g.N));
    }
}

template <int EPI>
__device__ __forceinline__ void row_epilogue(const RowGemm &g, const float (&v)[32], int64_t r,
                                             int col0, bool valid, float *s_col)
{
    if (EPI == TE_STORE_F32 || EPI == TE_RESID_F32 || EPI == TE_STORE_F32_T) {
        if (!valid && EPI != TE_STORE_F32_T) return;
        float o[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            o[j] = v[j] + (g.bias ? __ldg(g.bias + col0 + j) : 0.f);
            if (EPI == TE_RESID_F32) o[j] += g.resid[r * g.ld_resid + col0 + j];
        }
        if (valid) {
            float4 *dst = reinterpret_cast<float4 *>(g.out_f32 + r * g.ld_out + col0);
#pragma unroll
            for (int j = 0; j < 8; ++j) dst[j] = make_float4(o[4 * j], o[4 * j + 1], o[4 * j + 2], o[4 * j + 3]);
        }
        if (EPI == TE_STORE_F32_T) {
#pragma unroll
            for (int j = 0; j < 32; ++j) o[j] = valid ? o[j] : 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) st8(g.out_t, wl_offset(r, col0 + 8 * c, g.N), o + 8 * c);
        }
    } else if (EPI == TE_STORE_BF16) {
        if (!valid) return;
        float o[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) o[j] = v[j] + (g.bias ? __ldg(g.bias + col0 + j) : 0.f);
        uint4 *dst = reinterpret_cast<uint4 *>(g.out_h + r * g.ld_out + col0);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint4 q;
            q.x = pk2(o[8 * c], o[8 * c + 1]);
            q.y = pk2(o[8 * c + 2], o[8 * c + 3]);
            q.z = pk2(o[8 * c + 4], o[8 * c + 5]);
            q.w = pk2(o[8 * c + 6], o[8 * c + 7]);
            dst[c] = q;
        }
    } else if (EPI == TE_GELU_T) {
        // gelu(v) and gelu'(v) from one evaluation (gelu_as)
        float y[32], d[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float x = v[j] + __ldg(g.bias + col0 + j);
            float dx;
            const float gx = gelu_as(x, &dx);
            y[j] = valid ? gx : 0.f;
            d[j] = valid ? dx : 0.f;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            st8(g.out_t, wl_offset(r, col0 + 8 * c, g.N), y + 8 * c);
            if (g.out_t2) st8(g.out_t2, wl_offset(r, col0 + 8 * c, g.N), d + 8 * c);
        }
    } else {  // TE_GELU_BWD_T
        float y[32];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float gp[8];
            ld8(g.aux_t, wl_offset(r, col0 + 8 * c, g.N), gp);
#pragma unroll
            for (int j = 0; j < 8; ++j) y[8 * c + j] = valid ? v[8 * c + j] * gp[j] : 0.f;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) st8(g.out_t, wl_offset(r, col0 + 8 * c, g.N), y + 8 * c);
        if (s_col) atomicAdd(s_col + col0 + (threadIdx.x & 31), warp_colsum32(y));
    }
}

constexpr int kEpiWarps = 16;  // four epilogue warps per TMEM lane quadrant
constexpr int kEpiPerQuad = kEpiWarps / 4;

// Barrier among the epilogue warps only (named barrier 1).
__device__ __forceinline__ void epi_sync()
{
    asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
}

// Row-major outputs (FP32 rows, FP32 rows plus residual, BF16 rows) leave
// through a shared-memory tile: the TMEM drain writes acc + bias there (row
// pitch N + 4 floats, so 16-byte writes of 8 consecutive rows hit distinct
// banks), then all epilogue threads read it back with the residual and store
// with consecutive threads on consecutive 16-byte pieces of a row.
template <int EPI>
__device__ __forceinline__ void staged_store(const RowGemm &g, const float *sOut, int64_t rb)
{
    const int et = threadIdx.x - 64;  // epilogue thread 0 .. 511
    const int P = g.N + 4;
    if (EPI == TE_STORE_BF16) {
        // the tile holds BF16 rows (pitch N + 8 elements, see the TMEM drain)
        const unsigned char *sB = reinterpret_cast<const unsigned char *>(sOut);
        const int per_row = g.N / 8, PB = 2 * (g.N + 8);
        for (int e = et; e < 128 * per_row; e += 32 * kEpiWarps) {
            const int row = e / per_row, c8 = e % per_row;
            const int64_t r = rb * 128 + row;
            if (r >= g.R) continue;
            *reinterpret_cast<uint4 *>(g.out_h + r * g.ld_out + 8 * c8) =
                *reinterpret_cast<const uint4 *>(sB + row * PB + 16 * c8);
        }
    } else {
        const int per_row = g.N / 4;
        constexpr int U = EPI == TE_RESID_F32 ? 4 : 1;  // residual loads in flight per thread
        const int step = 32 * kEpiWarps;
        for (int e0 = et; e0 < 128 * per_row; e0 += U * step) {
            float4 h[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * step;
                const int row = e / per_row, c4 = e % per_row;
                const int64_t r = rb * 128 + row;
                h[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (EPI == TE_RESID_F32 && e < 128 * per_row && r < g.R)
                    h[u] = *reinterpret_cast<const float4 *>(g.resid + r * g.ld_resid + 4 * c4);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * step;
                const int row = e / per_row, c4 = e % per_row;
                const int64_t r = rb * 128 + row;
                if (e >= 128 * per_row || r >= g.R) continue;
                float4 v = *reinterpret_cast<const float4 *>(sOut + row * P + 4 * c4);
                v.x += h[u].x;
                v.y += h[u].y;
                v.z += h[u].z;
                v.w += h[u].w;
                *reinterpret_cast<float4 *>(g.out_f32 + r * g.ld_out + 4 * c4) = v;
            }
        }
    }
}

// The LayerNorm backward over a staged tile of dY rows (TE_LN_BWD): LPR =
// N / 8 lanes per row, each lane 8 consecutive columns; per-lane sums of
// dY xhat, dY and dX accumulate in pg, pb, pc across row blocks.
template <int N>
__device__ __forceinline__ void ln_bwd_tile(const RowGemm &g, const float *sOut, int64_t rb,
                                            const float (&gl)[8], float (&pg)[8], float (&pb)[8],
                                            float (&pc)[8])
{
    constexpr int LPR = N / 8, RPP = 32 / LPR, P = N + 4;
    const int lane = threadIdx.x & 31, ew = (threadIdx.x - 64) >> 5;  // epilogue warp 0..15
    const int sub = lane / LPR, c0 = 8 * (lane % LPR);
    const int64_t R_end = g.ln_dxt ? tl_blocks(g.R) * 128 : g.R;
    for (int row = ew * RPP + sub; row < 128; row += kEpiWarps * RPP) {  // same trip count for the warp
        const int64_t r = rb * 128 + row;
        const bool in = r < g.R;
        const int64_t rr = in ? r : g.R - 1;
        float dy[8], x[8];
        const float4 a = *reinterpret_cast<const float4 *>(sOut + row * P + c0);
        const float4 b = *reinterpret_cast<const float4 *>(sOut + row * P + c0 + 4);
        dy[0] = a.x; dy[1] = a.y; dy[2] = a.z; dy[3] = a.w;
        dy[4] = b.x; dy[5] = b.y; dy[6] = b.z; dy[7] = b.w;
        const float4 xa = *reinterpret_cast<const float4 *>(g.ln_x + rr * N + c0);
        const float4 xb = *reinterpret_cast<const float4 *>(g.ln_x + rr * N + c0 + 4);
        x[0] = xa.x; x[1] = xa.y; x[2] = xa.z; x[3] = xa.w;
        x[4] = xb.x; x[5] = xb.y; x[6] = xb.z; x[7] = xb.w;
        const float m = g.ln_mu[rr], s = g.ln_rs[rr];
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (!in) dy[j] = 0.f;
            x[j] = (x[j] - m) * s;  // xhat
            const float dxh = dy[j] * gl[j];
            s1 += dxh;
            s2 += dxh * x[j];
        }
#pragma unroll
        for (int o = LPR / 2; o; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        const float m1 = s1 * (1.0f / N), m2 = s2 * (1.0f / N);
        float out[8];
        if (g.ln_dres && in) {
            const float4 da = *reinterpret_cast<const float4 *>(g.ln_dres + r * N + c0);
            const float4 db = *reinterpret_cast<const float4 *>(g.ln_dres + r * N + c0 + 4);
            out[0] = da.x; out[1] = da.y; out[2] = da.z; out[3] = da.w;
            out[4] = db.x; out[5] = db.y; out[6] = db.z; out[7] = db.w;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) out[j] = 0.f;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (in) out[j] += s * (dy[j] * gl[j] - m1 - x[j] * m2);
            pg[j] += dy[j] * x[j];
            pb[j] += dy[j];
            pc[j] += out[j];
        }
        if (in) {
            float4 *dst = reinterpret_cast<float4 *>(g.out_f32 + r * N + c0);
            dst[0] = make_float4(out[0], out[1], out[2], out[3]);
            dst[1] = make_float4(out[4], out[5], out[6], out[7]);
        }
        if (g.ln_dxt && r < R_end) st8(g.ln_dxt, wl_offset(r, c0, N), out);
    }
}

// Per-lane LayerNorm-backward sums (lanes of one column group added by
// shuffles) into shared memory, then one atomic per column and CTA.
template <int N>
__device__ __forceinline__ void ln_bwd_flush(const RowGemm &g, float *red, float (&pg)[8],
                                             float (&pb)[8], float (&pc)[8])
{
    constexpr int LPR = N / 8;
    const int lane = threadIdx.x & 31, c0 = 8 * (lane % LPR);
#pragma unroll
    for (int o = LPR; o < 32; o <<= 1)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            pg[j] += __shfl_xor_sync(0xffffffffu, pg[j], o);
            pb[j] += __shfl_xor_sync(0xffffffffu, pb[j], o);
            pc[j] += __shfl_xor_sync(0xffffffffu, pc[j], o);
        }
    if (lane < LPR)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            atomicAdd(red + c0 + j, pg[j]);
            atomicAdd(red + N + c0 + j, pb[j]);
            atomicAdd(red + 2 * N + c0 + j, pc[j]);
        }
}

template <int EPI>
__global__ void __launch_bounds__(64 + 32 * kEpiWarps, 1) row_gemm_kernel(const __grid_constant__ RowGemm g)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t stage_bytes = (uint32_t)wl_block_bytes(g.K);  // one row block of A
    unsigned char *Bs = smem;
    unsigned char *As = smem + (size_t)g.NBw * g.KC * kTileBytes;
    __shared__ uint64_t full[2], empty[2], tfull[2], tempty[2], wfull;
    __shared__ uint32_t tslot;
    __shared__ float s_colbuf[EPI == TE_GELU_BWD_T ? kColsumMax : 1];
    float *s_col = EPI == TE_GELU_BWD_T && g.colsum ? s_colbuf : nullptr;
    if (s_col)
        for (int j = threadIdx.x; j < g.N; j += blockDim.x) s_col[j] = 0.f;
    // staged output tile (row-major epilogues); TE_LN_BWD reuses its first 3 N
    // floats for the column sums once the last row block is done
    float *sTile = reinterpret_cast<float *>(As + 2 * (size_t)stage_bytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
            tc::mbar_init(&tfull[s], 1);
            tc::mbar_init(&tempty[s], kEpiWarps);
        }
        tc::mbar_init(&wfull, 1);
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
    const int64_t nblk = g.RB;
    const int64_t my_n = (int64_t)blockIdx.x < nblk ? (nblk - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == 0 && lane == 0) {
        const uint32_t wbytes = (uint32_t)(g.NBw * g.KC) * kTileBytes;
        tc::mbar_arrive_expect_tx(&wfull, wbytes);
        for (int t = 0; t < g.NBw * g.KC; ++t)
            tc::bulk_g2s(Bs + (size_t)t * kTileBytes, g.Bw + (size_t)t * kTileBytes, kTileBytes, &wfull);
        for (int64_t i = 0; i < my_n; ++i) {
            const int s = (int)(i & 1);
            const int64_t rb = blockIdx.x + i * gridDim.x;
            if (i >= 2 && !tc::mbar_wait(&empty[s], (uint32_t)(((i >> 1) - 1) & 1))) {
                atomicExch(g.err, 11);
                break;
            }
            tc::mbar_arrive_expect_tx(&full[s], stage_bytes);
            tc::bulk_g2s(As + (size_t)s * stage_bytes, g.A + (size_t)rb * stage_bytes, stage_bytes,
                         &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        bool ok = tc::mbar_wait(&wfull, 0);
        const uint32_t idesc = tc::idesc_bf16(128, g.N);
        for (int64_t i = 0; i < my_n && ok; ++i) {
            const int s = (int)(i & 1), acc = (int)(i & 1);
            ok = tc::mbar_wait(&full[s], (uint32_t)((i >> 1) & 1));
            if (ok && i >= 2) ok = tc::mbar_wait(&tempty[acc], (uint32_t)(((i >> 1) - 1) & 1));
            if (!ok) break;
            tc::tc_fence_after();
            const uint32_t sa = tc::smem_u32(As + (size_t)s * stage_bytes);
            for (int ks = 0; ks < g.K / 16; ++ks) {
                const uint32_t sb = tc::smem_u32(Bs + (size_t)(ks >> 2) * g.NBw * kTileBytes) + 256 * (ks & 3);
                tc::mma_bf16(tmem + acc * 256, tc::smem_desc(sa + 256 * ks, 128, 16 * g.K),
                             tc::smem_desc(sb, 128, 1024), idesc, ks != 0 ? 1u : 0u);
            }
            tc::mma_commit(&empty[s]);
            tc::mma_commit(&tfull[acc]);
        }
        if (!ok) atomicExch(g.err, 12);
    } else if (warp >= 2) {
        const int q = warp & 3;             // TMEM lane quadrant of this warp
        const int part = (warp - 2) >> 2;   // which interleaved 32-column chunks
        const int row = 32 * q + lane;
        constexpr bool kRowMajor = EPI == TE_STORE_F32 || EPI == TE_RESID_F32 || EPI == TE_STORE_BF16 ||
                                   EPI == TE_LN_BWD;
        const bool staged = kRowMajor && (g.staged || EPI == TE_LN_BWD);
        float *sOut = sTile;
        bool ok = true;
        // TE_LN_BWD: this lane's 8 columns of the LayerNorm gain and its sums
        float gl[8], pg[8], pb[8], pc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            gl[j] = EPI == TE_LN_BWD ? __ldg(g.ln_g + (8 * (lane % (g.N / 8)) + j)) : 0.f;
            pg[j] = pb[j] = pc[j] = 0.f;
        }
        for (int64_t i = 0; i < my_n; ++i) {
            const int acc = (int)(i & 1);
            const int64_t rb = blockIdx.x + i * gridDim.x;
            // every epilogue warp takes part in the barriers below: a timed-out
            // wait records the error and the warp drains nothing further
            if (ok && !tc::mbar_wait(&tfull[acc], (uint32_t)((i >> 1) & 1))) {
                if (lane == 0) atomicExch(g.err, 13);
                ok = false;
            }
            if (!ok && !staged) break;
            tc::tc_fence_after();
            // the next row block's epilogue inputs into L2 while this one drains
            if (warp == 2 && lane == 0) prefetch_epilogue<EPI>(g, rb + gridDim.x);
            const int64_t r = rb * 128 + row;
            const bool valid = r < g.R;
            for (int c = part; ok && c < g.N / 32; c += kEpiPerQuad) {
                float v[32];
                tc::tmem_ld32(tmem + acc * 256 + ((uint32_t)(32 * q) << 16) + 32 * c, v);
                tc::tmem_wait_ld();
                if (staged && EPI == TE_STORE_BF16) {
                    // BF16 rows, pitch N + 8 elements (an odd number of 16-byte
                    // pieces: 16-byte writes of 8 consecutive rows hit distinct banks)
                    uint4 *d = reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(sOut) +
                                                         row * 2 * (g.N + 8) + 64 * c);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float o[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k) o[k] = v[8 * j + k] + (g.bias ? __ldg(g.bias + 32 * c + 8 * j + k) : 0.f);
                        uint4 qv;
                        qv.x = pk2(o[0], o[1]);
                        qv.y = pk2(o[2], o[3]);
                        qv.z = pk2(o[4], o[5]);
                        qv.w = pk2(o[6], o[7]);
                        d[j] = qv;
                    }
                } else if (staged) {
                    float4 *d = reinterpret_cast<float4 *>(sOut + row * (g.N + 4) + 32 * c);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float b[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) b[k] = g.bias ? __ldg(g.bias + 32 * c + 4 * j + k) : 0.f;
                        d[j] = make_float4(v[4 * j] + b[0], v[4 * j + 1] + b[1], v[4 * j + 2] + b[2],
                                           v[4 * j + 3] + b[3]);
                    }
                } else {
                    row_epilogue<EPI>(g, v, r, 32 * c, valid, s_col);
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (ok && lane == 0) tc::mbar_arrive(&tempty[acc]);
            if (staged) {
                epi_sync();  // the tile is complete
                if (EPI == TE_LN_BWD) {
                    if (ok) {
                        if (g.N == 32) ln_bwd_tile<32>(g, sOut, rb, gl, pg, pb, pc);
                        else if (g.N == 64) ln_bwd_tile<64>(g, sOut, rb, gl, pg, pb, pc);
                        else if (g.N == 128) ln_bwd_tile<128>(g, sOut, rb, gl, pg, pb, pc);
                        else ln_bwd_tile<256>(g, sOut, rb, gl, pg, pb, pc);
                    }
                } else if (ok) {
                    staged_store<EPI>(g, sOut, rb);
                }
                epi_sync();  // the tile is free for the next row block
            }
        }
        if (EPI == TE_LN_BWD) {
            // the tile is free (the loop ended on a barrier): zero 3 N sums
            for (int j = threadIdx.x - 64; j < 3 * g.N; j += 32 * kEpiWarps) sOut[j] = 0.f;
            epi_sync();
            if (g.N == 32) ln_bwd_flush<32>(g, sOut, pg, pb, pc);
            else if (g.N == 64) ln_bwd_flush<64>(g, sOut, pg, pb, pc);
            else if (g.N == 128) ln_bwd_flush<128>(g, sOut, pg, pb, pc);
            else ln_bwd_flush<256>(g, sOut, pg, pb, pc);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
    if (s_col)
        for (int j = threadIdx.x; j < g.N; j += blockDim.x) atomicAdd(g.colsum + j, s_col[j]);
    if (EPI == TE_LN_BWD)
        for (int j = threadIdx.x; j < g.N; j += blockDim.x) {
            atomicAdd(g.ln_dg + j, sTile[j]);
            atomicAdd(g.ln_db + j, sTile[g.N + j]);
            if (g.ln_dcol) atomicAdd(g.ln_dcol + j, sTile[2 * g.N + j]);
        }
}

// tile_gemm_kernel: the same product and epilogues for any N (a multiple of
// 32) and any K.  Output tiles of 128 rows x up to 256 columns are walked by
// persistent CTAs (column blocks of one row block consecutively, so the A
// tiles are reused from L2); per K chunk of 64 a stage holds the A tile and
// the one or two B tiles of the column block, through four stages.
constexpr int kTStages = 4;

template <int EPI>
__global__ void __launch_bounds__(64 + 32 * kEpiWarps, 1) tile_gemm_kernel(const __grid_constant__ RowGemm g)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr uint32_t stage_bytes = 3 * kTileBytes;
    __shared__ uint64_t full[kTStages], empty[kTStages], tfull[2], tempty[2];
    __shared__ uint32_t tslot;
    __shared__ float s_colbuf[EPI == TE_GELU_BWD_T ? kColsumMax : 1];
    float *s_col = EPI == TE_GELU_BWD_T && g.colsum ? s_colbuf : nullptr;
    if (s_col)
        for (int j = threadIdx.x; j < g.N; j += blockDim.x) s_col[j] = 0.f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&tfull[s], 1);
            tc::mbar_init(&tempty[s], kEpiWarps);
        }
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
    const int ncb = (g.N + 255) / 256;
    const int64_t ntiles = g.RB * ncb;
    const int64_t my_n = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto cols_of = [&](int cb) { return min(256, g.N - 256 * cb); };

    if (warp == 0 && lane == 0) {
        int64_t j = 0;  // chunks issued
        bool ok = true;
        for (int64_t i = 0; i < my_n && ok; ++i) {
            const int64_t t = blockIdx.x + i * gridDim.x, rb = t / ncb;
            const int cb = (int)(t % ncb), nbc = (cols_of(cb) + 127) / 128;
            for (int kc = 0; kc < g.KC; ++kc) {
                const int s = (int)(j % kTStages);
                if (j >= kTStages && !tc::mbar_wait(&empty[s], (uint32_t)((j / kTStages - 1) & 1))) {
                    atomicExch(g.err, 14);
                    ok = false;
                    break;
                }
                unsigned char *dst = smem + (size_t)s * stage_bytes;
                // K chunk kc of A: in each 8-row group, core groups 8 kc .. of the row block
                const uint32_t kw = (uint32_t)min(64, g.K - 64 * kc);
                tc::mbar_arrive_expect_tx(&full[s], 16u * 16u * kw + (uint32_t)nbc * kTileBytes);
                const unsigned char *arow = g.A + (size_t)rb * wl_block_bytes(g.K) + (size_t)kc * 1024;
                for (int rg = 0; rg < 16; ++rg)
                    tc::bulk_g2s(dst + rg * 1024, arow + (size_t)rg * 16 * g.K, 16u * kw, &full[s]);
                tc::bulk_g2s(dst + kTileBytes, g.Bw + ((size_t)(kc * g.NBw + 2 * cb) << 14),
                             (uint32_t)nbc * kTileBytes, &full[s]);
                ++j;
            }
        }
        // no bulk copy may be in flight when the CTA exits (the last stages'
        // phases complete when their copies land; earlier ones already have)
        for (int64_t jj = j > kTStages ? j - kTStages : 0; jj < j; ++jj)
            if (!tc::mbar_wait(&full[jj % kTStages], (uint32_t)((jj / kTStages) & 1))) break;
    } else if (warp == 1 && lane == 0) {
        int64_t j = 0;
        bool ok = true;
        for (int64_t i = 0; i < my_n && ok; ++i) {
            const int acc = (int)(i & 1);
            const int64_t t = blockIdx.x + i * gridDim.x;
            const int cb = (int)(t % ncb);
            if (i >= 2 && !tc::mbar_wait(&tempty[acc], (uint32_t)(((i >> 1) - 1) & 1))) {
                ok = false;
                break;
            }
            const uint32_t idesc = tc::idesc_bf16(128, cols_of(cb));
            for (int kc = 0; kc < g.KC; ++kc, ++j) {
                const int s = (int)(j % kTStages);
                if (!tc::mbar_wait(&full[s], (uint32_t)((j / kTStages) & 1))) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t sa = tc::smem_u32(smem + (size_t)s * stage_bytes);
                const uint32_t sb = sa + kTileBytes;
                const int nks = min(4, (g.K - 64 * kc) / 16);  // only k-steps inside K
                for (int ks = 0; ks < nks; ++ks)
                    tc::mma_bf16(tmem + acc * 256, tc::smem_desc(sa + 256 * ks, 128, 1024),
                                 tc::smem_desc(sb + 256 * ks, 128, 1024), idesc,
                                 (kc | ks) != 0 ? 1u : 0u);
                tc::mma_commit(&empty[s]);
            }
            if (ok) tc::mma_commit(&tfull[acc]);
        }
        if (!ok) atomicExch(g.err, 15);
    } else if (warp >= 2) {
        const int q = warp & 3, part = (warp - 2) >> 2, row = 32 * q + lane;
        for (int64_t i = 0; i < my_n; ++i) {
            const int acc = (int)(i & 1);
            const int64_t t = blockIdx.x + i * gridDim.x, rb = t / ncb;
            const int cb = (int)(t % ncb);
            if (!tc::mbar_wait(&tfull[acc], (uint32_t)((i >> 1) & 1))) {
                if (lane == 0) atomicExch(g.err, 16);
                break;
            }
            tc::tc_fence_after();
            const int64_t r = rb * 128 + row;
            const bool valid = r < g.R;
            for (int c = part; c < cols_of(cb) / 32; c += kEpiPerQuad) {
                float v[32];
                tc::tmem_ld32(tmem + acc * 256 + ((uint32_t)(32 * q) << 16) + 32 * c, v);
                tc::tmem_wait_ld();
                row_epilogue<EPI>(g, v, r, 256 * cb + 32 * c, valid, s_col);
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[acc]);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
    if (s_col)
        for (int j = threadIdx.x; j < g.N; j += blockDim.x) atomicAdd(g.colsum + j, s_col[j]);
}

// wgrad_kernel: C (+)= A^T B over the rows of two wide activations.  CTA
// (mt, nb, split) owns C rows 128 mt .. (features of A) and columns 256 nb ..
// (features of B) and a range of row blocks.  Per row block a stage holds the
// A window [128 rows x 128 features] and the B window [128 rows x nw
// features], gathered per 8-row group by bulk copies; both are read MN-major
// (instruction-descriptor bits 15 and 16), 8 MMAs of 16 rows each.  The TMEM
// accumulator is added to C with atomics.  A window that overhangs the
// features of A reads the next row group (or the slack tail); those
// accumulator rows are never stored.
__global__ void __launch_bounds__(192, 1) wgrad_kernel(const __grid_constant__ WgradGemm g, int stages)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int nbn = (g.N + 255) / 256, nmt = (g.M + 127) / 128;
    const int mt = (int)(blockIdx.x % nmt), nb = (int)((blockIdx.x / nmt) % nbn);
    const int64_t split = blockIdx.x / nmt / nbn;
    const int nw = min(256, g.N - 256 * nb);
    const uint32_t a_bytes = 128 * 128 * 2, b_bytes = (uint32_t)(128 * nw * 2);
    const uint32_t stage_bytes = a_bytes + b_bytes;
    const int64_t rb0 = split * g.rb_per_cta;
    const int64_t rb1 = rb0 + g.rb_per_cta < g.RB ? rb0 + g.rb_per_cta : g.RB;
    const int64_t n = rb1 > rb0 ? rb1 - rb0 : 0;
    __shared__ uint64_t full[4], empty[4], tfull;
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
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
        // A window: 16 KB... per 8-row group 16 core matrices (2 KB) of A's row group;
        // B window: nw / 8 core matrices of B's row group
        const uint32_t a_row = (uint32_t)min(2048, 16 * (g.M - 128 * mt));
        int64_t j = 0;
        for (; j < n; ++j) {
            const int s = (int)(j % stages);
            if (j >= stages && !tc::mbar_wait(&empty[s], (uint32_t)((j / stages - 1) & 1))) {
                atomicExch(g.err, 21);
                break;
            }
            const int64_t rb = rb0 + j;
            unsigned char *dst = smem + (size_t)s * stage_bytes;
            tc::mbar_arrive_expect_tx(&full[s], 16 * a_row + b_bytes);
            const unsigned char *ab = g.A + (size_t)rb * wl_block_bytes(g.M) + (size_t)mt * 2048;
            const unsigned char *bb = g.Bm + (size_t)rb * wl_block_bytes(g.N) + (size_t)nb * 4096;
            for (int rg = 0; rg < 16; ++rg) {
                tc::bulk_g2s(dst + rg * 2048, ab + (size_t)rg * 16 * g.M, a_row, &full[s]);
                tc::bulk_g2s(dst + a_bytes + rg * 16 * nw, bb + (size_t)rg * 16 * g.N, 16u * nw, &full[s]);
            }
        }
        // no bulk copy may be in flight when the CTA exits
        for (int64_t jj = j > stages ? j - stages : 0; jj < j; ++jj)
            if (!tc::mbar_wait(&full[jj % stages], (uint32_t)((jj / stages) & 1))) break;
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = tc::idesc_bf16(128, nw) | (1u << 15) | (1u << 16);  // A, B MN-major
        bool ok = true;
        for (int64_t j = 0; j < n; ++j) {
            const int s = (int)(j % stages);
            if (!tc::mbar_wait(&full[s], (uint32_t)((j / stages) & 1))) {
                ok = false;
                break;
            }
            tc::tc_fence_after();
            const uint32_t sa = tc::smem_u32(smem + (size_t)s * stage_bytes);
            const uint32_t sb = sa + a_bytes;
#pragma unroll
            for (int ks = 0; ks < 8; ++ks)  // 16 rows = two 8-row groups per MMA
                tc::mma_bf16(tmem, tc::smem_desc(sa + ks * 2 * 2048, 2048, 128),
                             tc::smem_desc(sb + ks * 2 * 16 * nw, 16 * nw, 128), idesc,
                             (j | ks) != 0 ? 1u : 0u);
            tc::mma_commit(&empty[s]);
        }
        if (!ok) atomicExch(g.err, 22);
        tc::mma_commit(&tfull);
    } else if (warp >= 2 && n > 0) {
        const int q = warp & 3;
        const int m = mt * 128 + 32 * q + lane;
        if (tc::mbar_wait(&tfull, 0)) {
            tc::tc_fence_after();
            for (int c = 0; c < nw / 32; ++c) {
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 32 * c, v);
                tc::tmem_wait_ld();
                if (m < g.M) {
                    const int n0 = nb * 256 + 32 * c;
                    if (g.transpose_out)
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) atomicAdd(g.C + (size_t)(n0 + jj) * g.ldc + m, v[jj]);
                    else
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) atomicAdd(g.C + (size_t)m * g.ldc + n0 + jj, v[jj]);
                }
            }
        } else if (lane == 0) {
            atomicExch(g.err, 23);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, 256);
}

// wgrad_rows_kernel: the same product when every feature of A (M <= 512,
// ceil(M / 128) x N <= 512 TMEM columns) and of B (N <= 256) fits one CTA:
// a stage is one row block of A and one of B, each a single bulk copy
// (contiguous in the wide layout), two stages in flight.  Per 16-row k-step
// one MMA per 128 features of A; A's 8-row groups are 16 M bytes apart.  A
// last 128-feature window that overhangs M reads the next row group (or B's
// block); those accumulator rows are never stored.
__global__ void __launch_bounds__(192, 1) wgrad_rows_kernel(const __grid_constant__ WgradGemm g)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int stages = 2;
    const int nmt = (g.M + 127) / 128;
    const uint32_t a_bytes = (uint32_t)wl_block_bytes(g.M), b_bytes = (uint32_t)wl_block_bytes(g.N);
    const uint32_t stage_bytes = a_bytes + b_bytes;
    const int64_t rb0 = (int64_t)blockIdx.x * g.rb_per_cta;
    const int64_t rb1 = rb0 + g.rb_per_cta < g.RB ? rb0 + g.rb_per_cta : g.RB;
    const int64_t n = rb1 > rb0 ? rb1 - rb0 : 0;
    __shared__ uint64_t full[stages], empty[stages], tfull;
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(&tfull, 1);
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
    if (warp == 0 && lane == 0) {
        int64_t j = 0;
        for (; j < n; ++j) {
            const int s = (int)(j % stages);
            if (j >= stages && !tc::mbar_wait(&empty[s], (uint32_t)((j / stages - 1) & 1))) {
                atomicExch(g.err, 24);
                break;
            }
            const int64_t rb = rb0 + j;
            unsigned char *dst = smem + (size_t)s * stage_bytes;
            tc::mbar_arrive_expect_tx(&full[s], stage_bytes);
            tc::bulk_g2s(dst, g.A + (size_t)rb * a_bytes, a_bytes, &full[s]);
            tc::bulk_g2s(dst + a_bytes, g.Bm + (size_t)rb * b_bytes, b_bytes, &full[s]);
        }
        // no bulk copy may be in flight when the CTA exits
        for (int64_t jj = j > stages ? j - stages : 0; jj < j; ++jj)
            if (!tc::mbar_wait(&full[jj % stages], (uint32_t)((jj / stages) & 1))) break;
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = tc::idesc_bf16(128, g.N) | (1u << 15) | (1u << 16);  // A, B MN-major
        bool ok = true;
        for (int64_t j = 0; j < n; ++j) {
            const int s = (int)(j % stages);
            if (!tc::mbar_wait(&full[s], (uint32_t)((j / stages) & 1))) {
                ok = false;
                break;
            }
            tc::tc_fence_after();
            const uint32_t sa = tc::smem_u32(smem + (size_t)s * stage_bytes);
            const uint32_t sb = sa + a_bytes;
#pragma unroll 1
            for (int ks = 0; ks < 8; ++ks)  // 16 rows = two 8-row groups per MMA
                for (int mt = 0; mt < nmt; ++mt)
                    tc::mma_bf16(tmem + (uint32_t)(mt * g.N),
                                 tc::smem_desc(sa + ks * 2 * 16 * g.M + mt * 2048, 16 * g.M, 128),
                                 tc::smem_desc(sb + ks * 2 * 16 * g.N, 16 * g.N, 128), idesc,
                                 (j | ks) != 0 ? 1u : 0u);
            tc::mma_commit(&empty[s]);
        }
        if (!ok) atomicExch(g.err, 25);
        tc::mma_commit(&tfull);
    } else if (warp >= 2 && n > 0) {
        const int q = warp & 3;
        if (tc::mbar_wait(&tfull, 0)) {
            tc::tc_fence_after();
            for (int mt = 0; mt < nmt; ++mt) {
                const int m = mt * 128 + 32 * q + lane;
                for (int c = 0; c < g.N / 32; ++c) {
                    float v[32];
                    tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(mt * g.N + 32 * c), v);
                    tc::tmem_wait_ld();
                    if (m < g.M) {
                        const int n0 = 32 * c;
                        if (g.transpose_out)
#pragma unroll
                            for (int jj = 0; jj < 32; ++jj) atomicAdd(g.C + (size_t)(n0 + jj) * g.ldc + m, v[jj]);
                        else
#pragma unroll
                            for (int jj = 0; jj < 32; ++jj) atomicAdd(g.C + (size_t)m * g.ldc + n0 + jj, v[jj]);
                    }
                }
            }
        } else if (lane == 0) {
            atomicExch(g.err, 26);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// FP32 row-major -> tiled BF16.  Thread = (8-element group along the tiled
// K axis, tiled row); padding is written as zeros.
__global__ void to_tiled_kernel(const float *__restrict__ X, int64_t R, int F, int ldx,
                                unsigned char *__restrict__ dst, int transpose)
{
    // tiled matrix: rows_t x K_t
    const int64_t rows_t = transpose ? F : R;
    const int64_t K_t = transpose ? R : F;
    const int64_t RBt = tl_blocks(rows_t);
    const int64_t groups = ((K_t + 63) >> 6) * 8;  // 8-wide groups along K (padded)
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= RBt * 128 * groups) return;
    int64_t rt, kg;
    if (transpose) {  // consecutive threads take consecutive tiled rows (features)
        rt = i % (RBt * 128);
        kg = i / (RBt * 128);
    } else {
        kg = i % groups;
        rt = i / groups;
    }
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int64_t kt = kg * 8 + j;
        float x = 0.f;
        if (rt < rows_t && kt < K_t)
            x = transpose ? X[kt * ldx + rt] : X[rt * ldx + kt];
        v[j] = x;
    }
    st8(dst, tl_offset(rt, (int)(kg * 8), RBt), v);
}

// Rows R .. the end of the last row block of W(R, F) set to zero.
__global__ void zero_wide_tail_kernel(int64_t R, int F, unsigned char *__restrict__ dst)
{
    const int groups = F >> 3;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = R + i / groups;
    if (r >= tl_blocks(R) * 128) return;
    *reinterpret_cast<uint4 *>(dst + wl_offset(r, 8 * (int)(i % groups), F)) = make_uint4(0, 0, 0, 0);
}

// FP32 row-major [R][F] -> W(R, F).  Thread = (row, 8-wide group); rows past
// R up to the end of the last row block are written as zeros.
__global__ void to_wide_kernel(const float *__restrict__ X, int64_t R, int F,
                               unsigned char *__restrict__ dst)
{
    const int groups = F >> 3;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tl_blocks(R) * 128 * groups) return;
    const int64_t r = i / groups;
    const int kg = (int)(i % groups);
    float v[8];
    if (r < R) {
        const float4 a = *reinterpret_cast<const float4 *>(X + r * F + 8 * kg);
        const float4 b = *reinterpret_cast<const float4 *>(X + r * F + 8 * kg + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = 0.f;
    }
    st8(dst, wl_offset(r, 8 * kg, F), v);
}

unsigned grid_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

sg_status launch_to_tiled(const float *X, int64_t R, int F, int ldx, unsigned char *dst,
                          bool transpose, cudaStream_t st)
{
    const int64_t rows_t = transpose ? F : R, K_t = transpose ? R : F;
    const int64_t n = tl_blocks(rows_t) * 128 * (((K_t + 63) >> 6) * 8);
    to_tiled_kernel<<<grid_for(n, 256), 256, 0, ::sg::counted(st)>>>(X, R, F, ldx, dst,
                                                                     transpose ? 1 : 0);
    return check_launch("to_tiled_kernel");
}

sg_status launch_zero_wide_tail(int64_t R, int F, unsigned char *dst, cudaStream_t st)
{
    const int64_t n = (tl_blocks(R) * 128 - R) * (F >> 3);
    if (n > 0) zero_wide_tail_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ::sg::counted(st)>>>(R, F, dst);
    return check_launch("zero_wide_tail_kernel");
}

sg_status launch_to_wide(const float *X, int64_t R, int F, unsigned char *dst, cudaStream_t st)
{
    const int64_t n = tl_blocks(R) * 128 * (F >> 3);
    to_wide_kernel<<<grid_for(n, 256), 256, 0, ::sg::counted(st)>>>(X, R, F, dst);
    return check_launch("to_wide_kernel");
}

sg_status launch_pack_tiled(const float *W, int rows, int K, unsigned char *dst, bool transpose,
                            cudaStream_t st)
{
    // W[rows][K] row-major; transpose packs W^T (K x rows)
    return launch_to_tiled(W, rows, K, K, dst, transpose, st);
}

bool ln_bwd_fusable(const RowGemm &g)
{
    if (!(g.N == 32 || g.N == 64 || g.N == 128 || g.N == 256) || g.KC > 4 || g.N > g.NBw * 128)
        return false;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, row_gemm_kernel<TE_LN_BWD>) != cudaSuccess) return false;
    const size_t smem = (size_t)g.NBw * g.KC * kTileBytes + 2 * wl_block_bytes(g.K) +
                        (size_t)128 * (g.N + 4) * sizeof(float) + fa.sharedSizeBytes;
    return smem <= (size_t)optin;
}

sg_status launch_row_gemm(const RowGemm &g, int epi, cudaStream_t st)
{
    if (g.N % 32 || g.N < 32 || g.N > g.NBw * 128 || g.KC < 1)
        return fail(SG_EUNSUPPORTED, "tensor-core GEMM needs N a multiple of 32");
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // weights that fit stay resident (row_gemm_kernel); otherwise column
    // blocks of 256 with A and B streamed per K chunk (tile_gemm_kernel)
    if (g.K % 16 || g.KC != (g.K + 63) / 64)
        return fail(SG_EUNSUPPORTED, "tensor-core GEMM needs K a multiple of 16");
    if (g.colsum && (epi != TE_GELU_BWD_T || g.N > kColsumMax))
        return fail(SG_EUNSUPPORTED, "fused column sums need the GELU backward and N <= 1024");
    if (epi == TE_LN_BWD && !ln_bwd_fusable(g))
        return fail(SG_EUNSUPPORTED, "the fused LayerNorm backward needs N in {32, 64, 128, 256} "
                                     "and its output tile in shared memory");
    const bool resident = g.N <= 256 && g.KC <= 4;
    const size_t smem0 = resident ? (size_t)g.NBw * g.KC * kTileBytes + 2 * wl_block_bytes(g.K)
                                  : (size_t)kTStages * 3 * kTileBytes;
    const int64_t units = resident ? g.RB : g.RB * ((g.N + 255) / 256);
    const unsigned grid = (unsigned)std::min<int64_t>(units, sms);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    auto go = [&](auto kern) -> sg_status {
        RowGemm h = g;
        size_t smem = smem0;
        // row-major outputs through a shared-memory tile where it fits
        const bool row_major = epi == TE_STORE_F32 || epi == TE_RESID_F32 || epi == TE_STORE_BF16 ||
                               epi == TE_LN_BWD;
        const size_t tile = (size_t)128 * (g.N + 4) * sizeof(float);
        cudaFuncAttributes fa{};
        SG_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
        h.staged = 0;
        if (resident && row_major && g.ld_out == g.N && (epi != TE_RESID_F32 || g.ld_resid == g.N) &&
            smem0 + tile + fa.sharedSizeBytes <= (size_t)optin) {
            h.staged = 1;
            smem = smem0 + tile;
        }
        if (epi == TE_LN_BWD && !h.staged)
            return fail(SG_EUNSUPPORTED, "the fused LayerNorm backward needs its tile in shared memory");
        SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<grid, 64 + 32 * kEpiWarps, smem, ::sg::counted(st)>>>(h);
        return check_launch(resident ? "row_gemm_kernel" : "tile_gemm_kernel");
    };
    if (resident) {
        switch (epi) {
        case TE_STORE_F32: return go(row_gemm_kernel<TE_STORE_F32>);
        case TE_RESID_F32: return go(row_gemm_kernel<TE_RESID_F32>);
        case TE_GELU_T: return go(row_gemm_kernel<TE_GELU_T>);
        case TE_GELU_BWD_T: return go(row_gemm_kernel<TE_GELU_BWD_T>);
        case TE_STORE_BF16: return go(row_gemm_kernel<TE_STORE_BF16>);
        case TE_LN_BWD: return go(row_gemm_kernel<TE_LN_BWD>);
        default: return go(row_gemm_kernel<TE_STORE_F32_T>);
        }
    }
    switch (epi) {
    case TE_STORE_F32: return go(tile_gemm_kernel<TE_STORE_F32>);
    case TE_RESID_F32: return go(tile_gemm_kernel<TE_RESID_F32>);
    case TE_GELU_T: return go(tile_gemm_kernel<TE_GELU_T>);
    case TE_GELU_BWD_T: return go(tile_gemm_kernel<TE_GELU_BWD_T>);
    case TE_STORE_BF16: return go(tile_gemm_kernel<TE_STORE_BF16>);
    default: return go(tile_gemm_kernel<TE_STORE_F32_T>);
    }
}

sg_status launch_wgrad_gemm(const WgradGemm &g, cudaStream_t st)
{
    if (g.N % 16 || g.M % 16 || g.N < 16 || g.M < 16)
        return fail(SG_EUNSUPPORTED, "weight-gradient GEMM needs feature counts that are multiples of 16");
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nmt = (g.M + 127) / 128;
    const size_t rows_stage = wl_block_bytes(g.M) + wl_block_bytes(g.N);
    if (g.N <= 256 && g.N % 32 == 0 && nmt * g.N <= 512 && 2 * rows_stage <= 200 * 1024) {
        // whole row blocks per stage: one CTA per SM, row blocks split evenly
        WgradGemm h = g;
        const int64_t ctas = std::min<int64_t>(g.RB, sms);
        h.rb_per_cta = (g.RB + ctas - 1) / ctas;
        const size_t smem = 2 * rows_stage;
        SG_CUDA_TRY(cudaFuncSetAttribute(wgrad_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        wgrad_rows_kernel<<<(unsigned)((g.RB + h.rb_per_cta - 1) / h.rb_per_cta), 192, smem,
                            ::sg::counted(st)>>>(h);
        return check_launch("wgrad_rows_kernel");
    }
    const int nw = std::min(256, g.N);
    const size_t stage = (size_t)128 * 128 * 2 + (size_t)128 * nw * 2;
    const int stages = (int)std::min<size_t>(4, (200 * 1024) / stage);
    const int64_t splits = (g.RB + g.rb_per_cta - 1) / g.rb_per_cta;
    const int64_t ctas = (int64_t)((g.M + 127) / 128) * ((g.N + 255) / 256) * splits;
    const size_t smem = stage * stages;
    SG_CUDA_TRY(cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    wgrad_kernel<<<(unsigned)ctas, 192, smem, ::sg::counted(st)>>>(g, stages);
    return check_launch("wgrad_kernel");
}

}  // namespace sg
