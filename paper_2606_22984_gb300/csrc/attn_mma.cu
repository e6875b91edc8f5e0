// attn_mma.cu -- the causal band + sink (or dense) attention of the BF16
// teacher-forced pass (Eq. mask; Algorithm 1) on warp-level tensor-core MMAs.
//
// One CTA per (sample, head) stages the head's rows of Q, K, V (and of dO in
// the backward) in shared memory as BF16.  A row's 16-byte chunks are
// XOR-swizzled by row so that ldmatrix reads of 8 consecutive rows fall in 8
// distinct bank groups.  Warps take 16-row tiles and run mma.sync m16n8k16
// (BF16 operands, FP32 accumulators): the scores of a 16 x 16 block of
// queries and keys come out as accumulator fragments, the softmax (forward)
// or its gradient (backward) runs on them in registers, and the result,
// rounded to BF16, is the A operand of the next product without leaving
// registers.  Only 16-key blocks holding visible keys are visited -- the
// sink [0, S) and the band [t - W, t] -- and elements are masked one by one.
//
// Backward without cross-warp reductions: one warp per 16-query tile forms
// dQ = scale (P o (dP - D)) K; one warp per 16-key tile forms dV = P^T dO and
// dK = scale (P o (dP - D))^T Q over the queries that see its keys, with P
// recomputed from the forward's log-sum-exp.  dQ, dK, dV leave as wide BF16
// pieces, together with this (sample, head)'s column sums (bias gradient).
//
// The tiles are 16 rows by 16 or 32 columns.  A tcgen05 MMA needs 64 or 128
// rows with its accumulator in TMEM; here the fragments stay in registers.
#include <cuda_bf16.h>

#include <algorithm>

#include <type_traits>

#include "gemm_tc.cuh"
#include "sg_internal.cuh"

namespace sg {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t (&r)[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

// d += a b, m16n8k16, BF16 x BF16 -> FP32
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                               uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Bulk prefetch of [p, p + bytes) into L2 (one thread; bytes a multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The softmax runs in base 2 (ex2_approx) with log2(e) folded into its scale
// and into the stored log-sum-exp.
__device__ __forceinline__ float ex2(float x) { return ex2_approx(x); }

constexpr float kLog2e = 1.4426950408889634f;

// Query t sees key k iff 0 <= t - k <= lim(k): lim = W for band keys, and
// unbounded for sink keys (k < S) and under the dense causal mask.
__device__ __forceinline__ uint32_t key_lim(int mask, int W, int S, int k)
{
    return (mask == SG_MASK_DENSE || k < S) ? 0x7fffffffu : (uint32_t)W;
}

// Element masks of a 16 x 16 block: every entry visible (kFull); band keys
// only (k0 >= S) and every row inside the sequence, so that one unsigned
// compare of the offset against W decides (kBand); anything else (kAny).
constexpr int kFull = 0, kBand = 1, kAny = 2;
template <int K>
using kind_t = std::integral_constant<int, K>;

// Every (query, key) of the 16 x 16 block at (t0, k0) is visible.
__device__ __forceinline__ bool block_full(int mask, int W, int S, int N, int t0, int k0)
{
    return t0 >= k0 + 16 && t0 + 16 <= N &&
           (mask == SG_MASK_DENSE || k0 + 16 <= S || t0 + 15 - k0 <= W);
}

// Byte offset of 16-byte chunk c of row r in a [rows][DH] BF16 array.
template <int DH>
__device__ __forceinline__ uint32_t sw_off(int r, int c)
{
    const int sc = DH == 16 ? (c ^ ((r >> 2) & 1)) : (c ^ ((r >> 1) & 3));
    return (uint32_t)(r * DH * 2 + 16 * sc);
}

// The helpers below take row bases that are multiples of 8, so the swizzle
// (bits 1..2 of the row) depends on the lane's row within its 8-row group
// only: address = base + row0 * DH * 2 + a per-lane constant.

// A fragments (16 rows from row0, all DH columns) of a staged array.
template <int DH>
__device__ __forceinline__ void load_a(uint32_t base, int row0, uint32_t (&a)[DH / 16][4])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int ks = 0; ks < DH / 16; ++ks)
        ldsm_x4(base + (uint32_t)(row0 * DH * 2) + sw_off<DH>(lane & 15, 2 * ks + (lane >> 4)), a[ks]);
}

// B fragments for X Y^T with Y's rows y0 .. y0 + 15 (two n-blocks of 8) and
// K = DH: b[ks][0..1] for rows y0 .. y0 + 7, b[ks][2..3] for y0 + 8 .. y0 + 15.
template <int DH>
__device__ __forceinline__ void load_b_rows(uint32_t base, int y0, uint32_t (&b)[DH / 16][4])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int ks = 0; ks < DH / 16; ++ks)
        ldsm_x4(base + (uint32_t)(y0 * DH * 2) +
                    sw_off<DH>((lane & 7) + ((lane >> 4) << 3), 2 * ks + ((lane >> 3) & 1)),
                b[ks]);
}

// acc (16 x DH) += A (16 x 16, rows of the k16 step) Y (16 x DH) with Y's
// rows y0 .. y0 + 15 (the K dimension) staged: B fragments by ldmatrix.trans.
template <int DH>
__device__ __forceinline__ void mma_a_rows(float (&acc)[DH / 8][4], const uint32_t (&a)[4],
                                           uint32_t base, int y0)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int nb = 0; nb < DH / 8; nb += 2) {
        uint32_t t[4];
        ldsm_x4_t(base + (uint32_t)(y0 * DH * 2) +
                      sw_off<DH>((lane & 7) + (((lane >> 3) & 1) << 3), nb + (lane >> 4)), t);
        mma_bf16_16816(acc[nb], a, t[0], t[1]);
        mma_bf16_16816(acc[nb + 1], a, t[2], t[3]);
    }
}

// C fragments of the 16-row block at x0 x the 16 rows of Y at y0 (K = DH).
template <int DH>
__device__ __forceinline__ void scores(float (&s)[2][4], const uint32_t (&a)[DH / 16][4],
                                       uint32_t ybase, int y0)
{
    uint32_t b[DH / 16][4];
    load_b_rows<DH>(ybase, y0, b);
#pragma unroll
    for (int nb = 0; nb < 2; ++nb)
#pragma unroll
        for (int j = 0; j < 4; ++j) s[nb][j] = 0.f;
#pragma unroll
    for (int ks = 0; ks < DH / 16; ++ks) {
        mma_bf16_16816(s[0], a[ks], b[ks][0], b[ks][1]);
        mma_bf16_16816(s[1], a[ks], b[ks][2], b[ks][3]);
    }
}

// The A fragment (16 x 16, BF16) of two accumulator n-blocks.
__device__ __forceinline__ void frag_a(const float (&x)[2][4], uint32_t (&a)[4])
{
    a[0] = pack_bf2(x[0][0], x[0][1]);
    a[1] = pack_bf2(x[0][2], x[0][3]);
    a[2] = pack_bf2(x[1][0], x[1][1]);
    a[3] = pack_bf2(x[1][2], x[1][3]);
}

// Key blocks (16 keys) visible to the query tile [t0, t0 + 16): one or two
// ranges [lo, hi) of 16-aligned keys.
__device__ __forceinline__ int key_ranges(int mask, int W, int S, int t0, int (&lo)[2], int (&hi)[2])
{
    const int top = t0 + 16;
    if (mask == SG_MASK_DENSE) {
        lo[0] = 0; hi[0] = top;
        return 1;
    }
    const int sink_hi = min((S + 15) & ~15, top);
    const int band_lo = max(0, (t0 - W) & ~15);
    if (band_lo <= sink_hi) {  // the sink and the band blocks touch
        lo[0] = 0; hi[0] = top;
        return 1;
    }
    if (sink_hi == 0) {  // no sink
        lo[0] = band_lo; hi[0] = top;
        return 1;
    }
    lo[0] = 0; hi[0] = sink_hi;
    lo[1] = band_lo; hi[1] = top;
    return 2;
}

// Stage Q, K, V (part 0, 1, 2 of the BF16 QKV rows) by cp.async; rows N ..
// Npad zeroed.
template <int DH>
__device__ __forceinline__ void stage_qkv(unsigned char *sq, const __nv_bfloat16 *__restrict__ QKVh,
                                          int b, int hh, int N, int Npad, int D, int nparts_zero)
{
    constexpr int CH = DH / 8;
    const size_t part_bytes = (size_t)Npad * DH * 2;
    for (int e = threadIdx.x; e < N * 3 * CH; e += blockDim.x) {
        const int t = e / (3 * CH), rem = e % (3 * CH), part = rem / CH, c = rem % CH;
        tc::cp_async16(sq + part * part_bytes + sw_off<DH>(t, c),
                       QKVh + ((size_t)b * N + t) * 3 * D + part * D + hh * DH + 8 * c);
    }
    tc::cp_async_commit();
    for (int e = threadIdx.x; e < (Npad - N) * CH * nparts_zero; e += blockDim.x) {
        const int part = e / ((Npad - N) * CH), rem = e % ((Npad - N) * CH);
        *reinterpret_cast<uint4 *>(sq + part * part_bytes + sw_off<DH>(N + rem / CH, rem % CH)) =
            make_uint4(0, 0, 0, 0);
    }
}

// ---------------------------------------------------------------------------
// Forward: O = softmax(scale Q K^T + mask) V, Hmid = Hin + O, LSE per row.
// ---------------------------------------------------------------------------
template <int DH>
__global__ void __launch_bounds__(kThreads)
attn_fwd_mma_kernel(const __nv_bfloat16 *__restrict__ QKVh, const float *__restrict__ Hin,
                    __nv_bfloat16 *__restrict__ O, float *__restrict__ Hmid, float *__restrict__ LSE,
                    int N, int Npad, int D, int NH, int mask, int W, int S, int Bc, int ahead)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int b = blockIdx.x / NH, hh = blockIdx.x % NH;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
    const size_t part_bytes = (size_t)Npad * DH * 2;
    // the rows of the sample whose CTAs start about one wave later, into L2
    if (hh == 0 && threadIdx.x == 0 && b + ahead < Bc) {
        const size_t nb = (size_t)b + ahead;
        prefetch_l2(QKVh + nb * N * 3 * D, (uint32_t)((size_t)N * 3 * D * 2));
        prefetch_l2(Hin + nb * N * D, (uint32_t)((size_t)N * D * 4));
    }
    stage_qkv<DH>(smem, QKVh, b, hh, N, Npad, D, 3);
    tc::cp_async_wait<0>();
    __syncthreads();
    const uint32_t sQ = tc::smem_u32(smem), sK = sQ + (uint32_t)part_bytes,
                   sV = sQ + 2 * (uint32_t)part_bytes;
    const float sc2 = rsqrtf((float)DH) * kLog2e;  // softmax scale in base 2
    for (int tile = warp; tile < Npad / 16; tile += kThreads / 32) {
        const int t0 = 16 * tile;
        const int r_lo = t0 + g, r_hi = t0 + g + 8;
        uint32_t qa[DH / 16][4];
        load_a<DH>(sQ, t0, qa);
        float o[DH / 8][4];
#pragma unroll
        for (int nb = 0; nb < DH / 8; ++nb)
#pragma unroll
            for (int j = 0; j < 4; ++j) o[nb][j] = 0.f;
        float m_lo = -INFINITY, m_hi = -INFINITY, l_lo = 0.f, l_hi = 0.f;
        int lo[2], hi[2];
        const int nr = key_ranges(mask, W, S, t0, lo, hi);
        for (int ri = 0; ri < nr; ++ri)
            for (int k0 = lo[ri]; k0 < hi[ri]; k0 += 16) {
                float s[2][4];
                scores<DH>(s, qa, sK, k0);
                // scores in base 2: x = log2(e) scale s, masked to -inf
                float mx_lo = -INFINITY, mx_hi = -INFINITY;
                auto mask_scores = [&](auto kind) {
                    constexpr int KIND = decltype(kind)::value;
#pragma unroll
                    for (int nb = 0; nb < 2; ++nb)
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int key = k0 + 8 * nb + 2 * q + e;
                            bool ok_lo = true, ok_hi = true;
                            if constexpr (KIND == kBand) {
                                ok_lo = (uint32_t)(r_lo - key) <= (uint32_t)W;
                                ok_hi = (uint32_t)(r_hi - key) <= (uint32_t)W;
                            } else if constexpr (KIND == kAny) {
                                const uint32_t lim = key_lim(mask, W, S, key);
                                ok_lo = (uint32_t)(r_lo - key) <= lim && r_lo < N;
                                ok_hi = (uint32_t)(r_hi - key) <= lim && r_hi < N;
                            }
                            s[nb][e] = ok_lo ? s[nb][e] * sc2 : -INFINITY;
                            s[nb][2 + e] = ok_hi ? s[nb][2 + e] * sc2 : -INFINITY;
                            mx_lo = fmaxf(mx_lo, s[nb][e]);
                            mx_hi = fmaxf(mx_hi, s[nb][2 + e]);
                        }
                };
                if (block_full(mask, W, S, N, t0, k0)) mask_scores(kind_t<kFull>{});
                else if (mask != SG_MASK_DENSE && k0 >= S && t0 + 16 <= N) mask_scores(kind_t<kBand>{});
                else mask_scores(kind_t<kAny>{});
#pragma unroll
                for (int x = 1; x < 4; x <<= 1) {
                    mx_lo = fmaxf(mx_lo, __shfl_xor_sync(0xffffffffu, mx_lo, x));
                    mx_hi = fmaxf(mx_hi, __shfl_xor_sync(0xffffffffu, mx_hi, x));
                }
                const float n_lo = fmaxf(m_lo, mx_lo), n_hi = fmaxf(m_hi, mx_hi);
                // rows with nothing visible yet keep scale 1 and add nothing
                const float c_lo = n_lo == -INFINITY ? 1.f : ex2(m_lo - n_lo);
                const float c_hi = n_hi == -INFINITY ? 1.f : ex2(m_hi - n_hi);
                m_lo = n_lo;
                m_hi = n_hi;
                const float z_lo = n_lo == -INFINITY ? 0.f : n_lo, z_hi = n_hi == -INFINITY ? 0.f : n_hi;
                float p[2][4];
#pragma unroll
                for (int nb = 0; nb < 2; ++nb)
#pragma unroll
                    for (int j = 0; j < 4; ++j) p[nb][j] = ex2(s[nb][j] - (j < 2 ? z_lo : z_hi));  // ex2(-inf) = 0
                l_lo = l_lo * c_lo + p[0][0] + p[0][1] + p[1][0] + p[1][1];
                l_hi = l_hi * c_hi + p[0][2] + p[0][3] + p[1][2] + p[1][3];
#pragma unroll
                for (int nb = 0; nb < DH / 8; ++nb) {
                    o[nb][0] *= c_lo;
                    o[nb][1] *= c_lo;
                    o[nb][2] *= c_hi;
                    o[nb][3] *= c_hi;
                }
                uint32_t pa[4];
                frag_a(p, pa);
                mma_a_rows<DH>(o, pa, sV, k0);
            }
#pragma unroll
        for (int x = 1; x < 4; x <<= 1) {
            l_lo += __shfl_xor_sync(0xffffffffu, l_lo, x);
            l_hi += __shfl_xor_sync(0xffffffffu, l_hi, x);
        }
        const float i_lo = 1.0f / l_lo, i_hi = 1.0f / l_hi;
#pragma unroll
        for (int nb = 0; nb < DH / 8; ++nb) {
            const int col = hh * DH + 8 * nb + 2 * q;
            // O (BF16, kept only for the backward's D_t) and Hmid = Hin + O (FP32)
            if (r_lo < N) {
                const size_t idx = ((size_t)b * N + r_lo) * D + col;
                const float2 ov = make_float2(o[nb][0] * i_lo, o[nb][1] * i_lo);
                const float2 hv = *reinterpret_cast<const float2 *>(Hin + idx);
                if (O) *reinterpret_cast<uint32_t *>(O + idx) = pack_bf2(ov.x, ov.y);
                *reinterpret_cast<float2 *>(Hmid + idx) = make_float2(hv.x + ov.x, hv.y + ov.y);
            }
            if (r_hi < N) {
                const size_t idx = ((size_t)b * N + r_hi) * D + col;
                const float2 ov = make_float2(o[nb][2] * i_hi, o[nb][3] * i_hi);
                const float2 hv = *reinterpret_cast<const float2 *>(Hin + idx);
                if (O) *reinterpret_cast<uint32_t *>(O + idx) = pack_bf2(ov.x, ov.y);
                *reinterpret_cast<float2 *>(Hmid + idx) = make_float2(hv.x + ov.x, hv.y + ov.y);
            }
        }
        if (q == 0) {  // natural log-sum-exp: (m + log2 l) ln 2
            if (r_lo < N) LSE[((size_t)b * N + r_lo) * NH + hh] = (m_lo + log2f(l_lo)) * 0.69314718055994531f;
            if (r_hi < N) LSE[((size_t)b * N + r_hi) * NH + hh] = (m_hi + log2f(l_hi)) * 0.69314718055994531f;
        }
    }
}

// ---------------------------------------------------------------------------
// Backward.
// ---------------------------------------------------------------------------

// A 16 x DH accumulator tile of rows row0 .. as wide BF16 pieces of dQKVt
// (part 0/1/2 = q/k/v columns), and its column sums into csum[part].
template <int DH>
__device__ __forceinline__ void put_tile(const float (&acc)[DH / 8][4], int b, int hh, int N, int D,
                                         int row0, int part, unsigned char *__restrict__ dQKVt,
                                         float *csum)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int nb = 0; nb < DH / 8; ++nb) {
        const uint32_t u_lo = pack_bf2(acc[nb][0], acc[nb][1]);
        const uint32_t u_hi = pack_bf2(acc[nb][2], acc[nb][3]);
        uint32_t v_lo[4], v_hi[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            v_lo[i] = __shfl_sync(0xffffffffu, u_lo, (lane & ~3) | i);
            v_hi[i] = __shfl_sync(0xffffffffu, u_hi, (lane & ~3) | i);
        }
        const int col = part * D + hh * DH + 8 * nb;
        if (q == 0 && row0 + g < N)
            *reinterpret_cast<uint4 *>(dQKVt + wl_offset((int64_t)b * N + row0 + g, col, 3 * D)) =
                make_uint4(v_lo[0], v_lo[1], v_lo[2], v_lo[3]);
        if (q == 1 && row0 + g + 8 < N)
            *reinterpret_cast<uint4 *>(dQKVt + wl_offset((int64_t)b * N + row0 + g + 8, col, 3 * D)) =
                make_uint4(v_hi[0], v_hi[1], v_hi[2], v_hi[3]);
        float c0 = acc[nb][0] + acc[nb][2], c1 = acc[nb][1] + acc[nb][3];
#pragma unroll
        for (int x = 4; x < 32; x <<= 1) {
            c0 += __shfl_xor_sync(0xffffffffu, c0, x);
            c1 += __shfl_xor_sync(0xffffffffu, c1, x);
        }
        if (g == 0) {
            atomicAdd(csum + part * DH + 8 * nb + 2 * q, c0);
            atomicAdd(csum + part * DH + 8 * nb + 2 * q + 1, c1);
        }
    }
}

template <int DH>
__global__ void __launch_bounds__(kThreads)
attn_bwd_mma_kernel(const __nv_bfloat16 *__restrict__ QKVh, const __nv_bfloat16 *__restrict__ O,
                    const float *__restrict__ dO, const float *__restrict__ LSE,
                    unsigned char *__restrict__ dQKVt, float *__restrict__ bsum, int N, int Npad,
                    int D, int NH, int mask, int W, int S, int Bc, int ahead)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ float csum[3 * DH];
    __shared__ int next_task;
    const int b = blockIdx.x / NH, hh = blockIdx.x % NH;
    // the rows of the sample whose CTAs start about one wave later, into L2
    if (hh == 0 && threadIdx.x == 0 && b + ahead < Bc) {
        const size_t nb = (size_t)b + ahead;
        prefetch_l2(QKVh + nb * N * 3 * D, (uint32_t)((size_t)N * 3 * D * 2));
        prefetch_l2(O + nb * N * D, (uint32_t)((size_t)N * D * 2));
        prefetch_l2(dO + nb * N * D, (uint32_t)((size_t)N * D * 4));
        if ((N * NH) % 4 == 0) prefetch_l2(LSE + nb * N * NH, (uint32_t)((size_t)N * NH * 4));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
    const size_t part_bytes = (size_t)Npad * DH * 2;
    unsigned char *sG = smem + 3 * part_bytes;  // dO rows (BF16)
    float *Ls = reinterpret_cast<float *>(smem + 4 * part_bytes);
    float *Ds = Ls + Npad;
    for (int j = threadIdx.x; j < 3 * DH; j += blockDim.x) csum[j] = 0.f;
    if (threadIdx.x == 0) next_task = kThreads / 32;
    stage_qkv<DH>(smem, QKVh, b, hh, N, Npad, D, 3);
    // dO rows to BF16, D_t = dO_t . O_t in FP32, the log-sum-exp; padding zero
    for (int t = threadIdx.x; t < Npad; t += blockDim.x) {
        float dd = 0.f, lse = 0.f;
        if (t < N) {
            const size_t r = (size_t)b * N + t;
            const float4 *gp = reinterpret_cast<const float4 *>(dO + r * D + hh * DH);
            const uint4 *op = reinterpret_cast<const uint4 *>(O + r * D + hh * DH);
#pragma unroll
            for (int c = 0; c < DH / 8; ++c) {
                const float4 g0 = gp[2 * c], g1 = gp[2 * c + 1];
                const uint4 ow = op[c];
                const uint32_t w[4] = {ow.x, ow.y, ow.z, ow.w};
                float ov[8];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    ov[2 * j] = __uint_as_float(w[j] << 16);
                    ov[2 * j + 1] = __uint_as_float(w[j] & 0xffff0000u);
                }
                dd += g0.x * ov[0] + g0.y * ov[1] + g0.z * ov[2] + g0.w * ov[3];
                dd += g1.x * ov[4] + g1.y * ov[5] + g1.z * ov[6] + g1.w * ov[7];
                *reinterpret_cast<uint4 *>(sG + sw_off<DH>(t, c)) =
                    make_uint4(pack_bf2(g0.x, g0.y), pack_bf2(g0.z, g0.w), pack_bf2(g1.x, g1.y),
                               pack_bf2(g1.z, g1.w));
            }
            lse = LSE[r * NH + hh];
        } else {
#pragma unroll
            for (int c = 0; c < DH / 8; ++c)
                *reinterpret_cast<uint4 *>(sG + sw_off<DH>(t, c)) = make_uint4(0, 0, 0, 0);
        }
        Ls[t] = lse * kLog2e;             // base-2 log-sum-exp
        Ds[t] = dd * rsqrtf((float)DH);   // scale D_t
    }
    tc::cp_async_wait<0>();
    __syncthreads();
    const uint32_t sQ = tc::smem_u32(smem), sK = sQ + (uint32_t)part_bytes,
                   sV = sQ + 2 * (uint32_t)part_bytes, sGu = sQ + 3 * (uint32_t)part_bytes;
    const float scale = rsqrtf((float)DH), sc2 = scale * kLog2e;
    const int T = Npad / 16;
    // tasks: key tiles first (those holding sink keys see every later query),
    // then the query tiles; a warp takes the next task when it is done
    for (int task = warp; task < 2 * T;) {
        if (task < T) {
            // ---- dK, dV of keys k0 .. k0 + 15 ----
            const int k0 = 16 * task;
            const int key_lo = k0 + g, key_hi = k0 + g + 8;
            uint32_t ka[DH / 16][4], va[DH / 16][4];
            load_a<DH>(sK, k0, ka);
            load_a<DH>(sV, k0, va);
            float dk[DH / 8][4], dv[DH / 8][4];
#pragma unroll
            for (int nb = 0; nb < DH / 8; ++nb)
#pragma unroll
                for (int j = 0; j < 4; ++j) dk[nb][j] = dv[nb][j] = 0.f;
            const bool all_q = mask == SG_MASK_DENSE || k0 < S;
            const int q_hi = all_q ? Npad : min(Npad, (k0 + 16 + W + 15) & ~15);
            const uint32_t lim_lo = key_lim(mask, W, S, key_lo), lim_hi = key_lim(mask, W, S, key_hi);
            for (int t0 = k0; t0 < q_hi; t0 += 16) {
                float s[2][4], dp[2][4];
                scores<DH>(s, ka, sQ, t0);   // S^T: keys x queries
                scores<DH>(dp, va, sGu, t0); // dP^T = V dO^T
                float p[2][4], ds[2][4];
                auto grads = [&](auto kind) {
                    constexpr int KIND = decltype(kind)::value;
#pragma unroll
                    for (int nb = 0; nb < 2; ++nb) {
                        const int tc0 = t0 + 8 * nb + 2 * q;  // this thread's two query columns
                        const float2 l2 = *reinterpret_cast<const float2 *>(Ls + tc0);
                        const float2 d2 = *reinterpret_cast<const float2 *>(Ds + tc0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int t = tc0 + (j & 1);
                            const int key = j < 2 ? key_lo : key_hi;
                            bool ok = true;
                            if constexpr (KIND == kBand) ok = (uint32_t)(t - key) <= (uint32_t)W;
                            else if constexpr (KIND == kAny)
                                ok = (uint32_t)(t - key) <= (j < 2 ? lim_lo : lim_hi) && t < N;
                            const float pv = ok ? ex2(fmaf(s[nb][j], sc2, -((j & 1) ? l2.y : l2.x))) : 0.f;
                            p[nb][j] = pv;
                            ds[nb][j] = pv * fmaf(dp[nb][j], scale, -((j & 1) ? d2.y : d2.x));
                        }
                    }
                };
                if (block_full(mask, W, S, N, t0, k0)) grads(kind_t<kFull>{});
                else if (mask != SG_MASK_DENSE && k0 >= S && t0 + 16 <= N) grads(kind_t<kBand>{});
                else grads(kind_t<kAny>{});
                uint32_t pa[4], dsa[4];
                frag_a(p, pa);
                frag_a(ds, dsa);
                mma_a_rows<DH>(dv, pa, sGu, t0);  // dV += P^T dO
                mma_a_rows<DH>(dk, dsa, sQ, t0);  // dK += dS^T Q
            }
            put_tile<DH>(dk, b, hh, N, D, k0, 1, dQKVt, csum);
            put_tile<DH>(dv, b, hh, N, D, k0, 2, dQKVt, csum);
        } else {
            // ---- dQ of queries t0 .. t0 + 15 ----
            const int t0 = 16 * (task - T);
            const int r_lo = t0 + g, r_hi = t0 + g + 8;
            const float lse_lo = Ls[r_lo], lse_hi = Ls[r_hi], d_lo = Ds[r_lo], d_hi = Ds[r_hi];
            const bool in_lo = r_lo < N, in_hi = r_hi < N;
            uint32_t qa[DH / 16][4], ga[DH / 16][4];
            load_a<DH>(sQ, t0, qa);
            load_a<DH>(sGu, t0, ga);
            float dq[DH / 8][4];
#pragma unroll
            for (int nb = 0; nb < DH / 8; ++nb)
#pragma unroll
                for (int j = 0; j < 4; ++j) dq[nb][j] = 0.f;
            int lo[2], hi[2];
            const int nr = key_ranges(mask, W, S, t0, lo, hi);
            for (int ri = 0; ri < nr; ++ri)
                for (int k0 = lo[ri]; k0 < hi[ri]; k0 += 16) {
                    float s[2][4], dp[2][4];
                    scores<DH>(s, qa, sK, k0);
                    scores<DH>(dp, ga, sV, k0);
                    float ds[2][4];
                    auto grads = [&](auto kind) {
                        constexpr int KIND = decltype(kind)::value;
#pragma unroll
                        for (int nb = 0; nb < 2; ++nb)
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const int key = k0 + 8 * nb + 2 * q + e;
                                bool ok_lo = true, ok_hi = true;
                                if constexpr (KIND == kBand) {
                                    ok_lo = (uint32_t)(r_lo - key) <= (uint32_t)W;
                                    ok_hi = (uint32_t)(r_hi - key) <= (uint32_t)W;
                                } else if constexpr (KIND == kAny) {
                                    const uint32_t lim = key_lim(mask, W, S, key);
                                    ok_lo = (uint32_t)(r_lo - key) <= lim && in_lo;
                                    ok_hi = (uint32_t)(r_hi - key) <= lim && in_hi;
                                }
                                const float p_lo = ok_lo ? ex2(fmaf(s[nb][e], sc2, -lse_lo)) : 0.f;
                                const float p_hi = ok_hi ? ex2(fmaf(s[nb][2 + e], sc2, -lse_hi)) : 0.f;
                                ds[nb][e] = p_lo * fmaf(dp[nb][e], scale, -d_lo);
                                ds[nb][2 + e] = p_hi * fmaf(dp[nb][2 + e], scale, -d_hi);
                            }
                    };
                    if (block_full(mask, W, S, N, t0, k0)) grads(kind_t<kFull>{});
                    else if (mask != SG_MASK_DENSE && k0 >= S && t0 + 16 <= N) grads(kind_t<kBand>{});
                    else grads(kind_t<kAny>{});
                    uint32_t dsa[4];
                    frag_a(ds, dsa);
                    mma_a_rows<DH>(dq, dsa, sK, k0);  // dQ += dS K
                }
            put_tile<DH>(dq, b, hh, N, D, t0, 0, dQKVt, csum);
        }
        int nt = 0;
        if (lane == 0) nt = atomicAdd(&next_task, 1);
        task = __shfl_sync(0xffffffffu, nt, 0);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < 3 * DH; j += blockDim.x) {
        const int part = j / DH, c = j % DH;
        bsum[(size_t)b * 3 * D + part * D + hh * DH + c] = csum[j];
    }
}

// Samples whose CTAs are resident at once (one CTA per sample and head): the
// distance at which a CTA prefetches a later sample's rows.
template <class K>
int samples_per_wave(K kern, size_t smem, int NH)
{
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    return std::max(1, sms * std::max(per_sm, 1) / NH);
}

size_t mma_smem_bytes(int DH, int N, bool bwd)
{
    const size_t Npad = (size_t)(N + 15) & ~(size_t)15;
    return bwd ? 4 * Npad * DH * 2 + 2 * Npad * sizeof(float) : 3 * Npad * DH * 2;
}

}  // namespace

bool attn_mma_supported(const sg_config &c)
{
    const int dh = c.d / c.n_heads;
    return c.precision == SG_BF16 && (dh == 16 || dh == 32) && c.d % 8 == 0 &&
           mma_smem_bytes(dh, c.N, true) <= 160 * 1024;
}

sg_status launch_attn_fwd_mma(const sg_config &c, const __nv_bfloat16 *QKVh, const float *Hin,
                              __nv_bfloat16 *O, float *Hmid, float *LSE, int Bc, cudaStream_t st)
{
    const int dh = c.d / c.n_heads, Npad = (c.N + 15) & ~15;
    const size_t smem = mma_smem_bytes(dh, c.N, false);
    auto go = [&](auto kern) -> sg_status {
        SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<(unsigned)(Bc * c.n_heads), kThreads, smem, ::sg::counted(st)>>>(
            QKVh, Hin, O, Hmid, LSE, c.N, Npad, c.d, c.n_heads, c.mask_kind, c.W, c.S, Bc,
            samples_per_wave(kern, smem, c.n_heads));
        return check_launch("attn_fwd_mma_kernel");
    };
    return dh == 16 ? go(attn_fwd_mma_kernel<16>) : go(attn_fwd_mma_kernel<32>);
}

sg_status launch_attn_bwd_mma(const sg_config &c, const __nv_bfloat16 *QKVh, const __nv_bfloat16 *O,
                              const float *dO, const float *LSE, unsigned char *dQKVt, float *bsum,
                              int Bc, cudaStream_t st)
{
    const int dh = c.d / c.n_heads, Npad = (c.N + 15) & ~15;
    const size_t smem = mma_smem_bytes(dh, c.N, true);
    auto go = [&](auto kern) -> sg_status {
        SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<(unsigned)(Bc * c.n_heads), kThreads, smem, ::sg::counted(st)>>>(
            QKVh, O, dO, LSE, dQKVt, bsum, c.N, Npad, c.d, c.n_heads, c.mask_kind, c.W, c.S, Bc,
            samples_per_wave(kern, smem, c.n_heads));
        return check_launch("attn_bwd_mma_kernel");
    };
    return dh == 16 ? go(attn_bwd_mma_kernel<16>) : go(attn_bwd_mma_kernel<32>);
}

}  // namespace sg
