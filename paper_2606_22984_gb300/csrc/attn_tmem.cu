// attn_tmem.cu -- the causal band + sink (or dense) attention of the BF16
// teacher-forced pass (Eq. mask; Algorithm 1) and its backward on tcgen05,
// for sequences whose queries see many keys (dense N ~ 1000, wide bands).
//
// One CTA per (sample, head) stages the head's rows of Q, K, V (and of dO in
// the backward) in shared memory as BF16 in the core-matrix layout of tc.cuh.
// The same bytes serve as a K-major operand (rows = M or N, d_h = K) and as
// an MN-major operand (d_h = N, rows = K), so no transposed copy is made.
//
// Rows of a 128-row tile map one to one onto TMEM lanes and threads (a warp
// reads its lane quarter), so row maxima and sums are per thread: no
// shuffles.  Scores land in TMEM; the threads read their row (tcgen05.ld),
// run the softmax (or its gradient) in registers and store the BF16
// probabilities back over the scores they have read, where the next product
// takes them as its A operand straight from TMEM.  A warp skips the 32-key
// chunks that none of its rows can see (it stores zeros there).
//
// Forward  (2 CTAs per SM; per CTA two softmax warpgroups and one MMA warp
//          each): a query tile is a pipeline of 32-key steps -- S = Q K^T
//          into a ring of three TMEM buffers, P over S, O += P V accumulated
//          in TMEM -- with the MMA warp issuing the scores two steps ahead.
// Backward (1 CTA per SM, 4 warpgroups, each issuing its own products), in
//          64-wide steps:
//          key tile (thread = key):   S^T = K Q^T, dP^T = V dO^T ->
//                                     P^T, dS^T -> dV += P^T dO, dK += dS^T Q
//          query tile (thread = query): S = Q K^T, dP = dO V^T -> dS ->
//                                     dQ += dS K
//          P is recomputed from the forward's log-sum-exp; dS carries the
//          1/sqrt(d_h) scale.  dQ, dK, dV leave as wide BF16 pieces with the
//          (sample, head)'s column sums (bias gradient).
// Every mbarrier wait is bounded; a time-out sets the error word and the CTA
// stops issuing work.
#include <cuda_bf16.h>

#include <algorithm>

#include "gemm_tc.cuh"
#include "sg_internal.cuh"
#include "tc.cuh"

namespace sg {

namespace {

constexpr int kT = 128;             // rows per tile = TMEM lanes
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// D[tmem] (+)= A[tmem] * B[smem]^T, kind::f16: A (M = 128 rows = lanes, K
// BF16 values packed two per 32-bit column from column a_tmem) in TMEM.
__device__ __forceinline__ void mma_bf16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                            uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
        ::"r"(d_tmem), "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// registers -> TMEM, 32 lanes x 16 consecutive columns
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
          "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]),
          "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

// DH consecutive FP32 columns of this thread's lane
template <int DH>
__device__ __forceinline__ void tmem_ld_dh(uint32_t taddr, float (&v)[DH])
{
    if constexpr (DH == 16) {
        tc::tmem_ld16(taddr, v);
    } else {
        tc::tmem_ld32(taddr, v);
    }
}

// Barrier over the 128 threads of warpgroup wg (ids 1.. ; 0 is __syncthreads).
__device__ __forceinline__ void wg_sync(int wg)
{
    asm volatile("bar.sync %0, 128;" ::"r"(wg + 1) : "memory");
}

// K-major operand of 128 rows from `row0` of a staged [rows][DH] part, K-step ks.
template <int DH>
__device__ __forceinline__ uint64_t desc_k(uint32_t part, int row0, int ks)
{
    return tc::smem_desc(part + (uint32_t)(row0 * DH * 2 + 256 * ks), 128, 16 * DH);
}

// MN-major operand (N = DH columns, K = 16 rows per step from `row0`).
template <int DH>
__device__ __forceinline__ uint64_t desc_mn(uint32_t part, int row0, int ks)
{
    return tc::smem_desc(part + (uint32_t)(row0 * DH * 2 + ks * 2 * 16 * DH), 16 * DH, 128);
}

// Query t sees key k iff 0 <= t - k <= lim(k): lim = W for band keys, and
// unbounded for sink keys (k < S) and under the dense causal mask.
__device__ __forceinline__ uint32_t key_lim(int mask, int W, int S, int k)
{
    return (mask == SG_MASK_DENSE || k < S) ? 0x7fffffffu : (uint32_t)W;
}

// Visibility of the 32 x 32 block of queries [t0, t0 + 32) and keys
// [k0, k0 + 32): kNone for none of the pairs, kAll for every pair (no element
// mask needed), kSome otherwise.
constexpr int kNone = 0, kAll = 1, kSome = 2;
__device__ __forceinline__ int chunk_kind(int mask, int W, int S, int N, int t0, int k0)
{
    const int t1 = min(t0 + 31, N - 1);
    if (t0 >= N || k0 > t1) return kNone;
    if (mask != SG_MASK_DENSE && k0 >= S && k0 + 31 < t0 - W) return kNone;
    const bool all = k0 + 31 <= t0 && t0 + 31 < N &&
                     (mask == SG_MASK_DENSE || k0 + 32 <= S || t0 + 31 - k0 <= W);
    return all ? kAll : kSome;
}

// Some query of [t0, t0 + nt) sees some key of [k0, k0 + nk).
__device__ __forceinline__ bool range_visible(int mask, int W, int S, int N, int t0, int nt, int k0,
                                              int nk)
{
    const int t1 = min(t0 + nt - 1, N - 1);
    if (t0 >= N || k0 > t1) return false;
    if (mask == SG_MASK_DENSE || k0 < S) return true;
    return k0 + nk - 1 >= t0 - W;
}

// Stage rows [0, N) of `nparts` parts of the BF16 QKV rows (part p at
// smem + p * Npad * DH * 2) in the core-matrix layout; rows N .. Npad zeroed.
template <int DH>
__device__ __forceinline__ void stage_parts(unsigned char *sq, const __nv_bfloat16 *__restrict__ QKVh,
                                            int b, int hh, int N, int Npad, int D, int nparts)
{
    constexpr int CH = DH / 8;
    const size_t part_bytes = (size_t)Npad * DH * 2;
    for (int e = threadIdx.x; e < N * nparts * CH; e += blockDim.x) {
        const int t = e / (nparts * CH), rem = e % (nparts * CH), part = rem / CH, c = rem % CH;
        tc::cp_async16(sq + part * part_bytes + tc::cm_offset(t, 8 * c, CH),
                       QKVh + ((size_t)b * N + t) * 3 * D + part * D + hh * DH + 8 * c);
    }
    tc::cp_async_commit();
    for (int e = threadIdx.x; e < (Npad - N) * CH * nparts; e += blockDim.x) {
        const int part = e / ((Npad - N) * CH), rem = e % ((Npad - N) * CH);
        *reinterpret_cast<uint4 *>(sq + part * part_bytes + tc::cm_offset(N + rem / CH, 8 * (rem % CH), CH)) =
            make_uint4(0, 0, 0, 0);
    }
}

// Bulk prefetch of [p, p + bytes) into L2 (one thread; bytes a multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Bounded wait on an mbarrier phase that suspends the thread (up to about a
// microsecond per probe) instead of spinning, so that waiting warps leave
// their issue slots to the warps that compute; false after about 4 s.
__device__ __forceinline__ bool mwait(uint64_t *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < (1u << 22); ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(tc::smem_u32(bar)), "r"(parity), "r"(1000u)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Bounded wait of the whole warpgroup on its MMA barrier.
__device__ __forceinline__ bool wg_wait(uint64_t *bar, uint32_t &phase, int *err, int code)
{
    const bool ok = mwait(bar, phase);
    phase ^= 1u;
    if (!ok && (threadIdx.x & 127) == 0) atomicExch(err, code);
    tc::tc_fence_after();
    return ok;
}

// registers -> TMEM, 32 lanes x 8 consecutive columns
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
                   "r"(v[6]), "r"(v[7])
                 : "memory");
}

// After a warpgroup stopped on a time-out: wait (bounded) for the MMAs it
// had committed, so that TMEM is not freed under them.
__device__ __forceinline__ void drain_on_error(uint64_t *bar, uint32_t phase, bool erred)
{
    if (erred && (threadIdx.x & 127) == 0) tc::mbar_wait(bar, phase ^ 1u, 1u << 20);
}

__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Row t's key k0 + j is visible (chunks that are only partly visible).
__device__ __forceinline__ bool vis_at(int t, int k, int mask, int W, int S, int N)
{
    return (uint32_t)(t - k) <= key_lim(mask, W, S, k) && t < N;
}

// Maximum of the visible scores of one 32-key chunk of this thread's row.
template <int KIND>
__device__ __forceinline__ float chunk_max(const float (&s)[32], int t, int k0, int mask, int W, int S, int N)
{
    if constexpr (KIND == kAll) {
        float a = fmax3(s[0], s[1], s[2]), b = fmax3(s[3], s[4], s[5]);
#pragma unroll
        for (int j = 6; j < 30; j += 4) {  // s[6] .. s[29]
            a = fmax3(a, s[j], s[j + 1]);
            b = fmax3(b, s[j + 2], s[j + 3]);
        }
        return fmaxf(fmax3(a, s[30], s[31]), b);
    } else {
        float a = -INFINITY;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (vis_at(t, k0 + j, mask, W, S, N)) a = fmaxf(a, s[j]);
        return a;
    }
}

// P = 2^(sc2 s - z) of one chunk (zero where not visible), packed as BF16
// pairs; the FP32 values are added to the row sum (two partial sums).
template <int KIND>
__device__ __forceinline__ void chunk_exp(const float (&s)[32], int t, int k0, int mask, int W, int S, int N,
                                          float sc2, float z, float2 &sum, uint32_t (&pk)[16])
{
    const float2 a2 = make_float2(sc2, sc2), b2 = make_float2(-z, -z);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        float2 x = __ffma2_rn(make_float2(s[2 * j], s[2 * j + 1]), a2, b2);
        if constexpr (KIND == kSome) {
            if (!vis_at(t, k0 + 2 * j, mask, W, S, N)) x.x = -INFINITY;
            if (!vis_at(t, k0 + 2 * j + 1, mask, W, S, N)) x.y = -INFINITY;
        }
        const float2 p = make_float2(ex2_approx(x.x), ex2_approx(x.y));  // 2^-inf = 0
        sum = __fadd2_rn(sum, p);
        pk[j] = pack_bf2(p.x, p.y);
    }
}

// ---------------------------------------------------------------------------
// Forward: O = softmax(scale Q K^T + mask) V, Hmid = Hin + O, LSE per row.
//
// A query tile runs as a pipeline of 32-key steps over its visible keys.
// TMEM per warpgroup: a ring of three score buffers at columns 0, 32, 64
// (S of a step, then its P in BF16 over the first 16 columns) and the output
// accumulator O at column 96.  Each warpgroup (4 softmax warps, one row per
// thread) has its own MMA warp.  Per step the softmax warps wait for the
// step's scores, store P and arrive on the step's "P ready" barrier; the MMA
// warp waits for it, adds P V into O and issues the scores of step i + 2 into
// the buffer step i - 1 used (after the commit that covers step i - 1's P V),
// so the scores of the next two steps are in flight during a softmax.  A row
// keeps its reference maximum m until the running maximum exceeds it by more
// than 8 (base 2): P stays below 2^8, and O (in TMEM) and the row sum are
// rescaled only then, after the pending products have landed.  Query tiles go
// to the two warpgroups in a fixed order (most keys first), which both the
// softmax warps and the MMA warp follow.
// ---------------------------------------------------------------------------
constexpr int kRing = 3;
constexpr uint32_t kOcol = 96;

// The visible 32-key chunks of query tile qt: the sink's [0, ns) and the
// band's [bstart, cend) (all chunks up to the diagonal under the dense mask).
struct TileSteps {
    int n, ns, bstart;
    __device__ __forceinline__ TileSteps(int mask, int W, int S, int N, int qt)
    {
        const int tile0 = qt * kT, tile1 = min(tile0 + kT, N) - 1;
        const int cend = min(4 * (qt + 1), (N + 31) / 32);
        ns = 0;
        bstart = 0;
        if (mask != SG_MASK_DENSE) {
            ns = (min(S, tile1 + 1) + 31) / 32;
            bstart = max(ns, max(0, tile0 - W) / 32);
        }
        n = ns + max(0, cend - bstart);
    }
    __device__ __forceinline__ int key0(int i) const { return 32 * (i < ns ? i : bstart + (i - ns)); }
};

template <int DH>
__global__ void __launch_bounds__(320, 2)
attn_fwd_tmem_kernel(const __nv_bfloat16 *__restrict__ QKVh, const float *__restrict__ Hin,
                     __nv_bfloat16 *__restrict__ O, float *__restrict__ Hmid, float *__restrict__ LSE,
                     int N, int Npad, int D, int NH, int mask, int W, int S, int Bc, int ahead, int *err)
{
    static_assert(DH == 16, "the TMEM layout holds a 16-column O");
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t sbar[2][kRing], pbar[2][kRing], obar[2], dbar[2];
    __shared__ uint32_t tslot;
    __shared__ int s_err;
    const int b = blockIdx.x / NH, hh = blockIdx.x % NH;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // warps 0-3 and 4-7: softmax warpgroups 0 and 1; warps 8 and 9: their MMA warps
    const bool mma_warp = warp >= 8;
    const int wg = mma_warp ? warp - 8 : warp >> 2, r = tid & 127;
    // the rows of the sample whose CTAs start about one wave later, into L2
    if (hh == 0 && tid == 0 && b + ahead < Bc) {
        const size_t nb = (size_t)b + ahead;
        prefetch_l2(QKVh + nb * N * 3 * D, (uint32_t)((size_t)N * 3 * D * 2));
        prefetch_l2(Hin + nb * N * D, (uint32_t)((size_t)N * D * 4));
    }
    if (tid == 0) {
        for (int g = 0; g < 2; ++g) {
            for (int i = 0; i < kRing; ++i) {
                tc::mbar_init(&sbar[g][i], 1);
                tc::mbar_init(&pbar[g][i], 4);
            }
            tc::mbar_init(&obar[g], 4);
            tc::mbar_init(&dbar[g], 1);
        }
        tc::fence_mbar_init();
        s_err = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&tslot, 256);
        tc::tmem_relinquish();
    }
    stage_parts<DH>(smem, QKVh, b, hh, N, Npad, D, 3);
    tc::cp_async_wait<0>();
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t part_bytes = (uint32_t)Npad * DH * 2;
    const uint32_t sQ = tc::smem_u32(smem), sK = sQ + part_bytes, sV = sK + part_bytes;
    const uint32_t tm = tslot + 128u * (uint32_t)wg;  // this warpgroup's columns
    const int nq = Npad / kT;
    uint64_t *sb = sbar[wg], *pb = pbar[wg];
    // completed phases of each ring barrier before the current tile, as parity bits
    uint32_t sbits = 0, pbits = 0;
    auto spar = [&](int j) { return ((sbits >> (j % kRing)) + (uint32_t)(j / kRing)) & 1u; };
    auto advance = [&](int n) {  // commits j = 0 .. n + 1, P phases i = 0 .. n - 1
#pragma unroll
        for (int bb = 0; bb < kRing; ++bb) {
            sbits ^= (uint32_t)(((n + 4 - bb) / kRing) & 1) << bb;
            pbits ^= (uint32_t)(((n + 2 - bb) / kRing) & 1) << bb;
        }
    };
    auto fail = [&](int code) {
        atomicExch(err, code);
        s_err = 1;
    };

    if (mma_warp) {
        if (lane == 0) {
            const uint32_t idesc_s = tc::idesc_bf16(kT, 32);
            const uint32_t idesc_o = tc::idesc_bf16(kT, DH) | (1u << 16);  // V read MN-major
            // descriptors of row 0; a step adds its rows' byte offset (in 16-byte
            // units) to the start-address field, which cannot carry below 256 KB
            const uint64_t dK0 = desc_k<DH>(sK, 0, 0), dV0 = desc_mn<DH>(sV, 0, 0), dV1 = desc_mn<DH>(sV, 0, 1);
            auto rows = [](int row0) { return (uint64_t)((uint32_t)(row0 * DH * 2) >> 4); };
            int tile_no = 0;
            for (int task = wg; task < nq && !s_err; task += 2, ++tile_no) {
                const int qt = nq - 1 - task;  // the later tiles see more keys: they go first
                const TileSteps st(mask, W, S, N, qt);
                const uint64_t dq = desc_k<DH>(sQ, qt * kT, 0);
                auto issue_s = [&](int j, int bj) {  // scores of step j into ring buffer bj = j % 3
                    tc::mma_bf16(tm + 32u * (uint32_t)bj, dq, dK0 + rows(st.key0(j)), idesc_s, 0u);
                };
                tc::tc_fence_after();
                issue_s(0, 0);
                tc::mma_commit(&sb[0]);
                if (st.n > 1) issue_s(1, 1);
                tc::mma_commit(&sb[1]);
                int bi = 0, q = 0;  // i % 3 and i / 3
                for (int i = 0; i < st.n && !s_err; ++i) {
                    const int b1 = bi == 2 ? 0 : bi + 1, b2 = bi == 0 ? 2 : bi - 1;  // (i + 1) % 3, (i + 2) % 3
                    const int q1 = q + (bi == 2);                                    // (i + 1) / 3
                    if (!mwait(&pb[bi], ((pbits >> bi) + (uint32_t)q) & 1u)) fail(43);
                    // step i + 2 reuses step i - 1's buffer: its P V must have landed
                    if (i >= 1 && i + 2 < st.n && !mwait(&sb[b1], ((sbits >> b1) + (uint32_t)q1) & 1u)) fail(44);
                    // the first P V of a tile overwrites O: the previous tile's O must have been read
                    if (i == 0 && tile_no > 0 && !mwait(&obar[wg], (uint32_t)(tile_no - 1) & 1u)) fail(46);
                    tc::tc_fence_after();
                    if (s_err) break;
                    const uint64_t kr = rows(st.key0(i));
                    mma_bf16_ta(tm + kOcol, tm + 32u * (uint32_t)bi, dV0 + kr, idesc_o, i > 0 ? 1u : 0u);
                    mma_bf16_ta(tm + kOcol, tm + 32u * (uint32_t)bi + 8u, dV1 + kr, idesc_o, 1u);
                    if (i + 2 < st.n) issue_s(i + 2, b2);
                    tc::mma_commit(&sb[b2]);  // also marks step i's P V
                    bi = b1;
                    q = q1;
                }
                // the next tile's scores overwrite buffers that this tile's last
                // P V products read: wait for the commit after the last one
                if (!s_err && !mwait(&sb[(st.n + 1) % kRing], spar(st.n + 1))) fail(47);
                advance(st.n);
            }
            // let this thread's MMAs land before TMEM is freed
            tc::mma_commit(&dbar[wg]);
            tc::mbar_wait(&dbar[wg], 0, 1u << 22);
        }
    } else {
        const uint32_t tl = tm + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's lanes
        const float sc2 = rsqrtf((float)DH) * kLog2e;                  // softmax scale in base 2
        for (int task = wg; task < nq && !s_err; task += 2) {
            const int qt = nq - 1 - task;
            const TileSteps st(mask, W, S, N, qt);
            const int t = qt * kT + r, t0w = qt * kT + 32 * (warp & 3);
            float mref = -INFINITY, l = 0.f;
            int bi = 0, q = 0;  // i % 3 and i / 3
            for (int i = 0; i < st.n; ++i) {
                const int b1 = bi == 2 ? 0 : bi + 1, q1 = q + (bi == 2);  // (i + 1) % 3, (i + 1) / 3
                const int k0 = st.key0(i);
                if (!mwait(&sb[bi], ((sbits >> bi) + (uint32_t)q) & 1u)) fail(41);
                tc::tc_fence_after();
                if (s_err) break;
                const int kind = chunk_kind(mask, W, S, N, t0w, k0);
                uint32_t pk[16];
                if (kind == kNone) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) pk[j] = 0u;
                } else {
                    float s[32];
                    tc::tmem_ld32(tl + 32u * (uint32_t)bi, s);
                    tc::tmem_wait_ld();
                    const float mx = kind == kAll ? chunk_max<kAll>(s, t, k0, mask, W, S, N)
                                                  : chunk_max<kSome>(s, t, k0, mask, W, S, N);
                    const float mn = fmaxf(mref, mx * sc2);
                    const bool grow = mn > mref + 8.f;  // also the first visible key (mref = -inf)
                    const bool rescale = grow && mref != -INFINITY;
                    if (__any_sync(0xffffffffu, rescale)) {
                        // O of this warp's rows, once every P V issued so far has
                        // landed (the commit of step i + 1 follows step i - 1's)
                        if (!mwait(&sb[b1], ((sbits >> b1) + (uint32_t)q1) & 1u)) fail(42);
                        tc::tc_fence_after();
                        float o[16];
                        tc::tmem_ld16(tl + kOcol, o);
                        tc::tmem_wait_ld();
                        const float f = rescale ? ex2_approx(mref - mn) : 1.f;
                        uint32_t ou[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) ou[j] = __float_as_uint(o[j] * f);
                        tmem_st16(tl + kOcol, ou);
                    }
                    if (grow) {
                        if (rescale) l *= ex2_approx(mref - mn);
                        mref = mn;
                    }
                    const float z = mref == -INFINITY ? 0.f : mref;
                    float2 ps2 = make_float2(0.f, 0.f);
                    if (kind == kAll) chunk_exp<kAll>(s, t, k0, mask, W, S, N, sc2, z, ps2, pk);
                    else chunk_exp<kSome>(s, t, k0, mask, W, S, N, sc2, z, ps2, pk);
                    l += ps2.x + ps2.y;
                }
                tmem_st16(tl + 32u * (uint32_t)bi, pk);  // P over the scores already read
                tc::tmem_wait_st();
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&pb[bi]);
                bi = b1;
                q = q1;
            }
            if (s_err) break;
            // O is complete once the commit of step n + 1 (after the last P V) lands
            if (!mwait(&sb[(st.n + 1) % kRing], spar(st.n + 1))) fail(45);
            tc::tc_fence_after();
            float o[16];
            tc::tmem_ld16(tl + kOcol, o);
            tc::tmem_wait_ld();
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&obar[wg]);  // O read: the next tile may overwrite it
            if (t < N) {
                const float inv = 1.0f / l;
                const size_t idx = ((size_t)b * N + t) * D + hh * DH;
#pragma unroll
                for (int c = 0; c < DH / 8; ++c) {
                    float ov[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) ov[j] = o[8 * c + j] * inv;
                    const float4 h0 = __ldg(reinterpret_cast<const float4 *>(Hin + idx) + 2 * c);
                    const float4 h1 = __ldg(reinterpret_cast<const float4 *>(Hin + idx) + 2 * c + 1);
                    reinterpret_cast<float4 *>(Hmid + idx)[2 * c] =
                        make_float4(h0.x + ov[0], h0.y + ov[1], h0.z + ov[2], h0.w + ov[3]);
                    reinterpret_cast<float4 *>(Hmid + idx)[2 * c + 1] =
                        make_float4(h1.x + ov[4], h1.y + ov[5], h1.z + ov[6], h1.w + ov[7]);
                    if (O)  // O in BF16, kept only for the backward's D_t
                        *reinterpret_cast<uint4 *>(O + idx + 8 * c) =
                            make_uint4(pack_bf2(ov[0], ov[1]), pack_bf2(ov[2], ov[3]), pack_bf2(ov[4], ov[5]),
                                       pack_bf2(ov[6], ov[7]));
                }
                // natural log-sum-exp: (m + log2 l) ln 2
                LSE[((size_t)b * N + t) * NH + hh] = (mref + log2f(l)) * 0.69314718055994531f;
            }
            advance(st.n);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tslot, 256);
    }
}

// ---------------------------------------------------------------------------
// Backward.  TMEM per warpgroup (128 columns), per 64-wide step (one elected
// thread of the warpgroup issues; two MMA round trips per step):
//   [0, 64)   scores (S or S^T); then P^T (key tiles) or dS (query tiles) in
//             BF16 over [0, 32); the step's dV (key) or dQ (query) at [32, 32 + DH)
//   [64, 128) dP or dP^T; then dS^T in BF16 over [64, 96) and the step's dK
//             at [96, 96 + DH) (key tiles)
// ---------------------------------------------------------------------------

// A tile's rows (this thread's row `row`) as wide BF16 pieces of dQKVt
// (part 0/1/2 = q/k/v columns), and the tile's column sums into csum[part].
template <int DH>
__device__ __forceinline__ void put_rows(const float (&acc)[DH], int64_t b, int hh, int N, int D, int row,
                                         int part, unsigned char *__restrict__ dQKVt, float *csum)
{
    if (row < N) {
#pragma unroll
        for (int c = 0; c < DH / 8; ++c)
            *reinterpret_cast<uint4 *>(dQKVt + wl_offset(b * N + row, part * D + hh * DH + 8 * c, 3 * D)) =
                make_uint4(pack_bf2(acc[8 * c], acc[8 * c + 1]), pack_bf2(acc[8 * c + 2], acc[8 * c + 3]),
                           pack_bf2(acc[8 * c + 4], acc[8 * c + 5]), pack_bf2(acc[8 * c + 6], acc[8 * c + 7]));
    }
    // rows beyond N hold zeros: no visible pair reaches them
#pragma unroll
    for (int j = 0; j < DH; ++j) {
        float v = acc[j];
#pragma unroll
        for (int x = 1; x < 32; x <<= 1) v += __shfl_xor_sync(0xffffffffu, v, x);
        if ((threadIdx.x & 31) == 0) atomicAdd(csum + part * DH + j, v);
    }
}

// Key tile: P^T and dS^T of queries tq .. tq + 15 for this thread's key k
// (Ln, Dn: minus the base-2 log-sum-exp and minus the scaled D_t per query).
template <int KIND>
__device__ __forceinline__ void key_grads16(const float (&s)[16], const float (&dp)[16], const float *Ln,
                                            const float *Dn, int tq, int k, uint32_t lim, int N, float sc2,
                                            float scale, uint32_t (&pp)[8], uint32_t (&dd)[8])
{
    const float2 a2 = make_float2(sc2, sc2), c2 = make_float2(scale, scale);
#pragma unroll
    for (int j4 = 0; j4 < 4; ++j4) {
        const float4 l4 = *reinterpret_cast<const float4 *>(Ln + tq + 4 * j4);
        const float4 d4 = *reinterpret_cast<const float4 *>(Dn + tq + 4 * j4);
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
            const int j = 4 * j4 + 2 * e2;
            float2 x = __ffma2_rn(make_float2(s[j], s[j + 1]), a2,
                                  e2 ? make_float2(l4.z, l4.w) : make_float2(l4.x, l4.y));
            if constexpr (KIND == kSome) {
                const int t = tq + j;
                if (!((uint32_t)(t - k) <= lim && t < N)) x.x = -INFINITY;
                if (!((uint32_t)(t + 1 - k) <= lim && t + 1 < N)) x.y = -INFINITY;
            }
            const float2 p = make_float2(ex2_approx(x.x), ex2_approx(x.y));
            const float2 g = __ffma2_rn(make_float2(dp[j], dp[j + 1]), c2,
                                        e2 ? make_float2(d4.z, d4.w) : make_float2(d4.x, d4.y));
            const float2 ds = __fmul2_rn(p, g);
            pp[j / 2] = pack_bf2(p.x, p.y);
            dd[j / 2] = pack_bf2(ds.x, ds.y);
        }
    }
}

// Query tile: dS of keys k0 .. k0 + 31 for this thread's query t (ln, dn:
// minus its base-2 log-sum-exp and minus its scaled D_t).
template <int KIND>
__device__ __forceinline__ void query_grads32(const float (&s)[32], const float (&dp)[32], int t, int k0,
                                              int mask, int W, int S, int N, float sc2, float scale, float ln,
                                              float dn, uint32_t (&dd)[16])
{
    const float2 a2 = make_float2(sc2, sc2), c2 = make_float2(scale, scale);
    const float2 l2 = make_float2(ln, ln), d2 = make_float2(dn, dn);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        float2 x = __ffma2_rn(make_float2(s[2 * j], s[2 * j + 1]), a2, l2);
        if constexpr (KIND == kSome) {
            if (!vis_at(t, k0 + 2 * j, mask, W, S, N)) x.x = -INFINITY;
            if (!vis_at(t, k0 + 2 * j + 1, mask, W, S, N)) x.y = -INFINITY;
        }
        const float2 p = make_float2(ex2_approx(x.x), ex2_approx(x.y));
        const float2 g = __ffma2_rn(make_float2(dp[2 * j], dp[2 * j + 1]), c2, d2);
        const float2 ds = __fmul2_rn(p, g);
        dd[j] = pack_bf2(ds.x, ds.y);
    }
}

template <int DH>
__global__ void __launch_bounds__(512, 1)
attn_bwd_tmem_kernel(const __nv_bfloat16 *__restrict__ QKVh, const __nv_bfloat16 *__restrict__ O,
                     const float *__restrict__ dO, const float *__restrict__ LSE,
                     unsigned char *__restrict__ dQKVt, float *__restrict__ bsum, int N, int Npad, int D,
                     int NH, int mask, int W, int S, int Bc, int ahead, int *err)
{
    constexpr int NWG = 4;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ float csum[3 * DH];
    __shared__ uint64_t bar[NWG];
    __shared__ uint32_t tslot;
    __shared__ int next_task, wg_task[NWG], s_err[NWG];
    const int b = blockIdx.x / NH, hh = blockIdx.x % NH;
    const int tid = threadIdx.x, wg = tid >> 7, r = tid & 127, warp = tid >> 5;
    if (hh == 0 && tid == 0 && b + ahead < Bc) {
        const size_t nb = (size_t)b + ahead;
        prefetch_l2(QKVh + nb * N * 3 * D, (uint32_t)((size_t)N * 3 * D * 2));
        prefetch_l2(O + nb * N * D, (uint32_t)((size_t)N * D * 2));
        prefetch_l2(dO + nb * N * D, (uint32_t)((size_t)N * D * 4));
        if ((N * NH) % 4 == 0) prefetch_l2(LSE + nb * N * NH, (uint32_t)((size_t)N * NH * 4));
    }
    if (tid == 0) {
        for (int i = 0; i < NWG; ++i) {
            tc::mbar_init(&bar[i], 1);
            s_err[i] = 0;
        }
        tc::fence_mbar_init();
        next_task = NWG;
    }
    for (int j = tid; j < 3 * DH; j += blockDim.x) csum[j] = 0.f;
    if (warp == 0) {
        tc::tmem_alloc(&tslot, 512);
        tc::tmem_relinquish();
    }
    const uint32_t part_bytes = (uint32_t)Npad * DH * 2;
    unsigned char *sGp = smem + 3 * part_bytes;  // dO rows (BF16)
    float *Ls = reinterpret_cast<float *>(smem + 4 * part_bytes);
    float *Ds = Ls + Npad;
    stage_parts<DH>(smem, QKVh, b, hh, N, Npad, D, 3);
    // dO rows to BF16, D_t = dO_t . O_t in FP32, the log-sum-exp; padding zero
    for (int t = tid; t < Npad; t += blockDim.x) {
        float dd = 0.f, lse = 0.f;
        if (t < N) {
            const size_t rr = (size_t)b * N + t;
            const float4 *gp = reinterpret_cast<const float4 *>(dO + rr * D + hh * DH);
            const uint4 *op = reinterpret_cast<const uint4 *>(O + rr * D + hh * DH);
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
                *reinterpret_cast<uint4 *>(sGp + tc::cm_offset(t, 8 * c, DH / 8)) =
                    make_uint4(pack_bf2(g0.x, g0.y), pack_bf2(g0.z, g0.w), pack_bf2(g1.x, g1.y),
                               pack_bf2(g1.z, g1.w));
            }
            lse = LSE[rr * NH + hh];
        } else {
#pragma unroll
            for (int c = 0; c < DH / 8; ++c)
                *reinterpret_cast<uint4 *>(sGp + tc::cm_offset(t, 8 * c, DH / 8)) = make_uint4(0, 0, 0, 0);
        }
        Ls[t] = -lse * kLog2e;            // minus the base-2 log-sum-exp
        Ds[t] = -dd * rsqrtf((float)DH);  // minus the scaled D_t
    }
    tc::cp_async_wait<0>();
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t sQ = tc::smem_u32(smem), sK = sQ + part_bytes, sV = sK + part_bytes, sG = sV + part_bytes;
    const uint32_t tm = tslot + 128u * (uint32_t)wg;
    const uint32_t tl = tm + ((uint32_t)(32 * (warp & 3)) << 16);
    const float scale = rsqrtf((float)DH), sc2 = scale * kLog2e;
    const int nt = Npad / kT;
    const uint32_t idesc_s = tc::idesc_bf16(kT, 64);
    const uint32_t idesc_p = tc::idesc_bf16(kT, DH) | (1u << 16);  // B read MN-major
    uint32_t phase = 0;
    // tasks 2i: key tile i (dK, dV); 2i + 1: query tile nt - 1 - i (dQ), so
    // the tiles that meet the most pairs under the causal mask go first
    for (int task = wg; task < 2 * nt;) {
        if ((task & 1) == 0) {
            // ---- dK, dV of keys kt * 128 + r ----
            const int kt = task >> 1;
            const int k = kt * kT + r, k0w = kt * kT + 32 * (warp & 3);
            const uint32_t lim = key_lim(mask, W, S, k);
            float dk[DH], dv[DH];
#pragma unroll
            for (int j = 0; j < DH; ++j) dk[j] = dv[j] = 0.f;
            for (int q0 = kt * kT; q0 < Npad; q0 += 64) {
                if (!range_visible(mask, W, S, N, q0, 64, kt * kT, kT)) continue;
                if (r == 0) {
#pragma unroll
                    for (int ks = 0; ks < DH / 16; ++ks) {
                        tc::mma_bf16(tm, desc_k<DH>(sK, kt * kT, ks), desc_k<DH>(sQ, q0, ks), idesc_s,
                                     ks > 0 ? 1u : 0u);  // S^T
                        tc::mma_bf16(tm + 64, desc_k<DH>(sV, kt * kT, ks), desc_k<DH>(sG, q0, ks), idesc_s,
                                     ks > 0 ? 1u : 0u);  // dP^T = V dO^T
                    }
                    tc::mma_commit(&bar[wg]);
                }
                __syncwarp();
                if (!wg_wait(&bar[wg], phase, err, 43)) s_err[wg] = 1;
#pragma unroll 1
                for (int c = 0; c < 2; ++c) {
                    const int tq = q0 + 32 * c;  // this chunk's first query
                    const int kind = chunk_kind(mask, W, S, N, tq, k0w);
#pragma unroll 1
                    for (int h = 0; h < 2; ++h) {
                        uint32_t pp[8], dd[8];
                        if (kind == kNone) {
#pragma unroll
                            for (int j = 0; j < 8; ++j) pp[j] = dd[j] = 0u;
                        } else {
                            float s[16], dp[16];
                            tc::tmem_ld16(tl + 32 * c + 16 * h, s);
                            tc::tmem_ld16(tl + 64 + 32 * c + 16 * h, dp);
                            tc::tmem_wait_ld();
                            if (kind == kAll) key_grads16<kAll>(s, dp, Ls, Ds, tq + 16 * h, k, lim, N, sc2, scale, pp, dd);
                            else key_grads16<kSome>(s, dp, Ls, Ds, tq + 16 * h, k, lim, N, sc2, scale, pp, dd);
                        }
                        tmem_st8(tl + 16 * c + 8 * h, pp);       // P^T over S^T already read
                        tmem_st8(tl + 64 + 16 * c + 8 * h, dd);  // dS^T over dP^T already read
                    }
                }
                tc::tmem_wait_st();
                tc::tc_fence_before();
                wg_sync(wg);
                if (s_err[wg]) break;
                if (r == 0) {
                    tc::tc_fence_after();
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        mma_bf16_ta(tm + 32, tm + 8 * ks, desc_mn<DH>(sG, q0, ks), idesc_p,
                                    ks > 0 ? 1u : 0u);  // dV += P^T dO
                        mma_bf16_ta(tm + 96, tm + 64 + 8 * ks, desc_mn<DH>(sQ, q0, ks), idesc_p,
                                    ks > 0 ? 1u : 0u);  // dK += dS^T Q
                    }
                    tc::mma_commit(&bar[wg]);
                }
                __syncwarp();
                if (!wg_wait(&bar[wg], phase, err, 44)) s_err[wg] = 1;
                {
                    float x[DH];
                    tmem_ld_dh<DH>(tl + 32, x);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < DH; ++j) dv[j] += x[j];
                    tmem_ld_dh<DH>(tl + 96, x);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < DH; ++j) dk[j] += x[j];
                }
                tc::tc_fence_before();
                wg_sync(wg);
                if (s_err[wg]) break;
            }
            if (s_err[wg]) break;
            put_rows<DH>(dk, b, hh, N, D, k, 1, dQKVt, csum);
            put_rows<DH>(dv, b, hh, N, D, k, 2, dQKVt, csum);
        } else {
            // ---- dQ of queries qt * 128 + r ----
            const int qt = nt - 1 - (task >> 1);
            const int t = qt * kT + r, t0w = qt * kT + 32 * (warp & 3);
            const float l2 = Ls[t], dt = Ds[t];
            float dq[DH];
#pragma unroll
            for (int j = 0; j < DH; ++j) dq[j] = 0.f;
            for (int k0 = 0; k0 < qt * kT + kT; k0 += 64) {
                if (!range_visible(mask, W, S, N, qt * kT, kT, k0, 64)) continue;
                if (r == 0) {
#pragma unroll
                    for (int ks = 0; ks < DH / 16; ++ks) {
                        tc::mma_bf16(tm, desc_k<DH>(sQ, qt * kT, ks), desc_k<DH>(sK, k0, ks), idesc_s,
                                     ks > 0 ? 1u : 0u);  // S
                        tc::mma_bf16(tm + 64, desc_k<DH>(sG, qt * kT, ks), desc_k<DH>(sV, k0, ks), idesc_s,
                                     ks > 0 ? 1u : 0u);  // dP = dO V^T
                    }
                    tc::mma_commit(&bar[wg]);
                }
                __syncwarp();
                if (!wg_wait(&bar[wg], phase, err, 45)) s_err[wg] = 1;
#pragma unroll 1
                for (int c = 0; c < 2; ++c) {
                    const int kc = k0 + 32 * c;  // this chunk's first key
                    const int kind = chunk_kind(mask, W, S, N, t0w, kc);
                    uint32_t dd[16];
                    if (kind == kNone) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) dd[j] = 0u;
                    } else {
                        float s[32], dp[32];
                        tc::tmem_ld32(tl + 32 * c, s);
                        tc::tmem_ld32(tl + 64 + 32 * c, dp);
                        tc::tmem_wait_ld();
                        if (kind == kAll) query_grads32<kAll>(s, dp, t, kc, mask, W, S, N, sc2, scale, l2, dt, dd);
                        else query_grads32<kSome>(s, dp, t, kc, mask, W, S, N, sc2, scale, l2, dt, dd);
                    }
                    tmem_st16(tl + 16 * c, dd);  // dS over S already read
                }
                tc::tmem_wait_st();
                tc::tc_fence_before();
                wg_sync(wg);
                if (s_err[wg]) break;
                if (r == 0) {
                    tc::tc_fence_after();
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        mma_bf16_ta(tm + 32, tm + 8 * ks, desc_mn<DH>(sK, k0, ks), idesc_p,
                                    ks > 0 ? 1u : 0u);  // dQ += dS K
                    tc::mma_commit(&bar[wg]);
                }
                __syncwarp();
                if (!wg_wait(&bar[wg], phase, err, 46)) s_err[wg] = 1;
                {
                    float x[DH];
                    tmem_ld_dh<DH>(tl + 32, x);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < DH; ++j) dq[j] += x[j];
                }
                tc::tc_fence_before();
                wg_sync(wg);
                if (s_err[wg]) break;
            }
            if (s_err[wg]) break;
            put_rows<DH>(dq, b, hh, N, D, t, 0, dQKVt, csum);
        }
        if (r == 0) wg_task[wg] = atomicAdd(&next_task, 1);
        wg_sync(wg);
        task = wg_task[wg];
        wg_sync(wg);
    }
    drain_on_error(&bar[wg], phase, s_err[wg] != 0);
    tc::tc_fence_before();
    __syncthreads();
    for (int j = tid; j < 3 * DH; j += blockDim.x) {
        const int part = j / DH, c = j % DH;
        bsum[(size_t)b * 3 * D + part * D + hh * DH + c] = csum[j];
    }
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tslot, 512);
    }
}

size_t tmem_smem_bytes(int DH, int N, bool bwd)
{
    const size_t Npad = (size_t)(N + kT - 1) / kT * kT;
    return bwd ? 4 * Npad * DH * 2 + 2 * Npad * sizeof(float) : 3 * Npad * DH * 2;
}

// Samples whose CTAs are resident at once (one CTA per sample and head).
template <class K>
int tmem_samples_per_wave(K kern, int threads, size_t smem, int NH)
{
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    return std::max(1, sms * std::max(per_sm, 1) / NH);
}

}  // namespace

// The tcgen05 attention serves BF16 models with d_h = 16 under the dense
// causal mask from 128 positions on (a query sees on average N / 2 keys).
// Band masks stay on the warp-level MMA kernels: their 16-key blocks follow
// a band's edges more closely than 32-key chunks of 128-key tiles, and the
// two MMA round trips per tile step cost more than the wasted exponentials
// save (measured on the 3D EA L=10 band, W = 100: backward 50 ms against 42 ms
// at B = 2048).  The kernels handle any mask of the sampler.
bool attn_tmem_supported(const sg_config &c)
{
    const int dh = c.d / c.n_heads;
    return c.precision == SG_BF16 && dh == 16 && c.d % 8 == 0 && c.mask_kind == SG_MASK_DENSE &&
           c.N >= kT && tmem_smem_bytes(dh, c.N, true) <= 200 * 1024;
}

sg_status launch_attn_fwd_tmem(const sg_config &c, const __nv_bfloat16 *QKVh, const float *Hin,
                               __nv_bfloat16 *O, float *Hmid, float *LSE, int Bc, int *err, cudaStream_t st)
{
    const int dh = c.d / c.n_heads, Npad = (c.N + kT - 1) / kT * kT;
    const size_t smem = tmem_smem_bytes(dh, c.N, false);
    auto kern = attn_fwd_tmem_kernel<16>;
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)(Bc * c.n_heads), 320, smem, ::sg::counted(st)>>>(
        QKVh, Hin, O, Hmid, LSE, c.N, Npad, c.d, c.n_heads, c.mask_kind, c.W, c.S, Bc,
        tmem_samples_per_wave(kern, 320, smem, c.n_heads), err);
    return check_launch("attn_fwd_tmem_kernel");
}

sg_status launch_attn_bwd_tmem(const sg_config &c, const __nv_bfloat16 *QKVh, const __nv_bfloat16 *O,
                               const float *dO, const float *LSE, unsigned char *dQKVt, float *bsum, int Bc,
                               int *err, cudaStream_t st)
{
    const int dh = c.d / c.n_heads, Npad = (c.N + kT - 1) / kT * kT;
    const size_t smem = tmem_smem_bytes(dh, c.N, true);
    auto kern = attn_bwd_tmem_kernel<16>;
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)(Bc * c.n_heads), 512, smem, ::sg::counted(st)>>>(
        QKVh, O, dO, LSE, dQKVt, bsum, c.N, Npad, c.d, c.n_heads, c.mask_kind, c.W, c.S, Bc,
        tmem_samples_per_wave(kern, 512, smem, c.n_heads), err);
    return check_launch("attn_bwd_tmem_kernel");
}

}  // namespace sg
