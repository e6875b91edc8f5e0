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
// Error-word values of the bounded waits: kWaitCode + 8 * site (bit 2, the
// non-finite-logit flag of the error word, stays clear).
constexpr int kWaitCode = 0x1000;
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
// their issue slots to the warps that compute; false after about 0.26 s
// (every wait here covers microseconds of work).
__device__ __forceinline__ bool mwait(uint64_t *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < (1u << 18); ++i) {
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

// Ring-barrier phases: bit b of the parity words holds the parity of buffer
// b's next phase at the start of a tile; a tile commits j = 0 .. n + 1 (one
// per step and two more) and completes P phases i = 0 .. n - 1.
__device__ __forceinline__ uint32_t ring_parity(uint32_t bits, int j)
{
    return ((bits >> (j % kRing)) + (uint32_t)(j / kRing)) & 1u;
}

__device__ __forceinline__ void ring_advance(uint32_t &sbits, uint32_t &pbits, int n)
{
#pragma unroll
    for (int bb = 0; bb < kRing; ++bb) {
        sbits ^= (uint32_t)(((n + 4 - bb) / kRing) & 1) << bb;
        pbits ^= (uint32_t)(((n + 2 - bb) / kRing) & 1) << bb;
    }
}

// The MMA warp's part of one query tile (lane 0 only).  dq: the Q tile's
// descriptor; dK0, dV0: descriptors of row 0 of the staged K and V arrays;
// krow(i): the row in them of step i's 32 keys.  tile_no > 0 makes the tile
// wait until the previous tile's O has been read (obar).  Returns false
// after a time-out (the error word is set).
template <int DH, class KRow>
__device__ __forceinline__ bool fwd_tile_mma(uint32_t tm, uint64_t dq, uint64_t dK0, uint64_t dV0, int n, KRow krow,
                                             uint64_t *sb, uint64_t *pb, uint64_t *obar, int tile_no, uint32_t sbits,
                                             uint32_t pbits, int *err, volatile int *s_err)
{
    const uint32_t idesc_s = tc::idesc_bf16(kT, 32);
    const uint32_t idesc_o = tc::idesc_bf16(kT, DH) | (1u << 16);  // V read MN-major
    // a step adds its rows' byte offset (in 16-byte units) to the start-address
    // field of the row-0 descriptors, which cannot carry below 256 KB
    auto rows = [](int row0) { return (uint64_t)((uint32_t)(row0 * DH * 2) >> 4); };
    auto issue_s = [&](int j, int bj) {  // scores of step j into ring buffer bj = j % 3
        const uint64_t kr = rows(krow(j));
#pragma unroll
        for (int ks = 0; ks < DH / 16; ++ks)  // K-step: 2 core matrices = 256 bytes
            tc::mma_bf16(tm + 32u * (uint32_t)bj, dq + 16u * ks, dK0 + kr + 16u * ks, idesc_s, ks > 0 ? 1u : 0u);
    };
    auto fail = [&](int code) {
        atomicExch(err, code);
        *s_err = 1;
        return false;
    };
    // A new tile's commits reuse the ring barriers.  Every softmax warp has
    // observed the previous tile's last commit (and read its O) before it
    // arrives on obar, so no warp can still be polling a phase that this
    // tile's commits would complete twice over; and the first P V overwrites O.
    if (tile_no > 0 && !mwait(obar, (uint32_t)(tile_no - 1) & 1u)) return fail(kWaitCode + 8 * 46);
    tc::tc_fence_after();
    issue_s(0, 0);
    tc::mma_commit(&sb[0]);
    if (n > 1) issue_s(1, 1);
    tc::mma_commit(&sb[1]);
    int bi = 0, q = 0;  // i % 3 and i / 3
    for (int i = 0; i < n; ++i) {
        const int b1 = bi == 2 ? 0 : bi + 1, b2 = bi == 0 ? 2 : bi - 1;  // (i + 1) % 3, (i + 2) % 3
        const int q1 = q + (bi == 2);                                    // (i + 1) / 3
        if (!mwait(&pb[bi], ((pbits >> bi) + (uint32_t)q) & 1u)) return fail(kWaitCode + 8 * 43);
        // step i + 2 reuses step i - 1's buffer: its P V must have landed
        if (i >= 1 && i + 2 < n && !mwait(&sb[b1], ((sbits >> b1) + (uint32_t)q1) & 1u)) return fail(kWaitCode + 8 * 44);
        tc::tc_fence_after();
        if (*s_err) return false;
        const uint64_t kr = rows(krow(i));
        // P V: K = 32 keys in two 16-key steps of 2 core-matrix rows (2 * 16 * DH bytes)
        mma_bf16_ta(tm + kOcol, tm + 32u * (uint32_t)bi, dV0 + kr, idesc_o, i > 0 ? 1u : 0u);
        mma_bf16_ta(tm + kOcol, tm + 32u * (uint32_t)bi + 8u, dV0 + kr + (uint64_t)(2 * DH), idesc_o, 1u);
        if (i + 2 < n) issue_s(i + 2, b2);
        tc::mma_commit(&sb[b2]);  // also marks step i's P V
        bi = b1;
        q = q1;
    }
    // the next tile's scores overwrite buffers that this tile's last P V
    // products read: wait for the commit after the last one
    if (!mwait(&sb[(n + 1) % kRing], ring_parity(sbits, n + 1))) return fail(kWaitCode + 8 * 47);
    return true;
}

// The softmax warps' part of one query tile: steps over the n visible chunks
// (keys key0(i) .. + 31) for row t of the warp's rows t0w .. t0w + 31; on
// return o holds the row's unnormalised output, mref its reference maximum
// (base 2) and l its sum.  Returns false after a time-out.
template <int DH, class Key0>
__device__ __forceinline__ bool fwd_tile_softmax(uint32_t tl, int n, Key0 key0, int t, int t0w, int mask, int W, int S,
                                                 int N, uint64_t *sb, uint64_t *pb, uint32_t sbits, int *err,
                                                 volatile int *s_err, float &mref, float &l, float (&o)[DH])
{
    const int lane = threadIdx.x & 31;
    const float sc2 = rsqrtf((float)DH) * kLog2e;  // softmax scale in base 2
    auto fail = [&](int code) {
        atomicExch(err, code);
        *s_err = 1;
        return false;
    };
    mref = -INFINITY;
    l = 0.f;
    int bi = 0, q = 0;  // i % 3 and i / 3
    for (int i = 0; i < n; ++i) {
        const int b1 = bi == 2 ? 0 : bi + 1, q1 = q + (bi == 2);  // (i + 1) % 3, (i + 1) / 3
        const int k0 = key0(i);
        if (!mwait(&sb[bi], ((sbits >> bi) + (uint32_t)q) & 1u)) return fail(kWaitCode + 8 * 41);
        tc::tc_fence_after();
        if (*s_err) return false;
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
                if (!mwait(&sb[b1], ((sbits >> b1) + (uint32_t)q1) & 1u)) return fail(kWaitCode + 8 * 42);
                tc::tc_fence_after();
                float ov[DH];
                tmem_ld_dh<DH>(tl + kOcol, ov);
                tc::tmem_wait_ld();
                const float f = rescale ? ex2_approx(mref - mn) : 1.f;
#pragma unroll
                for (int c = 0; c < DH / 16; ++c) {
                    uint32_t ou[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) ou[j] = __float_as_uint(ov[16 * c + j] * f);
                    tmem_st16(tl + kOcol + 16u * c, ou);
                }
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
    // O is complete once the commit of step n + 1 (after the last P V) lands
    if (!mwait(&sb[(n + 1) % kRing], ring_parity(sbits, n + 1))) return fail(kWaitCode + 8 * 45);
    tc::tc_fence_after();
    tmem_ld_dh<DH>(tl + kOcol, o);
    tc::tmem_wait_ld();
    return true;
}

// Row t's outputs: O (BF16, optional) and Hmid = Hin + O / l (FP32), LSE.
template <int DH>
__device__ __forceinline__ void fwd_row_out(const float (&o)[DH], float mref, float l, int64_t b, int t, int hh, int N,
                                            int D, int NH, const float *__restrict__ Hin, __nv_bfloat16 *__restrict__ O,
                                            float *__restrict__ Hmid, float *__restrict__ LSE)
{
    const float inv = 1.0f / l;
    const size_t idx = ((size_t)b * N + t) * D + hh * DH;
#pragma unroll
    for (int c = 0; c < DH / 8; ++c) {
        float ov[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) ov[j] = o[8 * c + j] * inv;
        const float4 h0 = __ldg(reinterpret_cast<const float4 *>(Hin + idx) + 2 * c);
        const float4 h1 = __ldg(reinterpret_cast<const float4 *>(Hin + idx) + 2 * c + 1);
        reinterpret_cast<float4 *>(Hmid + idx)[2 * c] = make_float4(h0.x + ov[0], h0.y + ov[1], h0.z + ov[2], h0.w + ov[3]);
        reinterpret_cast<float4 *>(Hmid + idx)[2 * c + 1] =
            make_float4(h1.x + ov[4], h1.y + ov[5], h1.z + ov[6], h1.w + ov[7]);
        if (O)  // O in BF16, kept only for the backward's D_t
            *reinterpret_cast<uint4 *>(O + idx + 8 * c) = make_uint4(
                pack_bf2(ov[0], ov[1]), pack_bf2(ov[2], ov[3]), pack_bf2(ov[4], ov[5]), pack_bf2(ov[6], ov[7]));
    }
    // natural log-sum-exp: (m + log2 l) ln 2
    LSE[((size_t)b * N + t) * NH + hh] = (mref + log2f(l)) * 0.69314718055994531f;
}

template <int DH>
__global__ void __launch_bounds__(320, 2)
attn_fwd_tmem_kernel(const __nv_bfloat16 *__restrict__ QKVh, const float *__restrict__ Hin,
                     __nv_bfloat16 *__restrict__ O, float *__restrict__ Hmid, float *__restrict__ LSE,
                     int N, int Npad, int D, int NH, int mask, int W, int S, int Bc, int ahead, int *err)
{
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
    uint32_t sbits = 0, pbits = 0;
    if (mma_warp) {
        if (lane == 0) {
            const uint64_t dK0 = desc_k<DH>(sK, 0, 0), dV0 = desc_mn<DH>(sV, 0, 0);
            int tile_no = 0;
            for (int task = wg; task < nq && !s_err; task += 2, ++tile_no) {
                const int qt = nq - 1 - task;  // the later tiles see more keys: they go first
                const TileSteps st(mask, W, S, N, qt);
                if (!fwd_tile_mma<DH>(tm, desc_k<DH>(sQ, qt * kT, 0), dK0, dV0, st.n,
                                      [&](int i) { return st.key0(i); }, sbar[wg], pbar[wg], &obar[wg], tile_no,
                                      sbits, pbits, err, &s_err))
                    break;
                ring_advance(sbits, pbits, st.n);
            }
            // let this thread's MMAs land before TMEM is freed
            tc::mma_commit(&dbar[wg]);
            tc::mbar_wait(&dbar[wg], 0, 1u << 22);
        }
    } else {
        const uint32_t tl = tm + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's lanes
        for (int task = wg; task < nq && !s_err; task += 2) {
            const int qt = nq - 1 - task;
            const TileSteps st(mask, W, S, N, qt);
            const int t = qt * kT + r, t0w = qt * kT + 32 * (warp & 3);
            float mref, l, o[DH];
            if (!fwd_tile_softmax<DH>(tl, st.n, [&](int i) { return st.key0(i); }, t, t0w, mask, W, S, N, sbar[wg],
                                      pbar[wg], sbits, err, &s_err, mref, l, o))
                break;
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&obar[wg]);  // O read: the next tile may overwrite it
            if (t < N) fwd_row_out<DH>(o, mref, l, b, t, hh, N, D, NH, Hin, O, Hmid, LSE);
            ring_advance(sbits, pbits, st.n);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tslot, 256);
    }
}

// Stage the CTA's query tile (rows qt * 128 .. + 127 of part 0, zero beyond N)
// at sq and the K and V rows of its n visible 32-key chunks compactly (chunk
// i at rows 32 i .. 32 i + 31 of sk, sv; zero beyond N).
template <int DH, class Key0>
__device__ __forceinline__ void stage_tile(unsigned char *sq, unsigned char *sk, unsigned char *sv,
                                           const __nv_bfloat16 *__restrict__ QKVh, int64_t b, int hh, int N, int D,
                                           int qt, int n, Key0 key0)
{
    constexpr int CH = DH / 8;
    for (int e = threadIdx.x; e < kT * CH; e += blockDim.x) {
        const int row = e / CH, c = e % CH, t = qt * kT + row;
        unsigned char *dst = sq + tc::cm_offset(row, 8 * c, CH);
        if (t < N) tc::cp_async16(dst, QKVh + ((size_t)b * N + t) * 3 * D + hh * DH + 8 * c);
        else *reinterpret_cast<uint4 *>(dst) = make_uint4(0, 0, 0, 0);
    }
    const int per_part = n * 32 * CH;
    for (int e = threadIdx.x; e < 2 * per_part; e += blockDim.x) {
        const int part = e / per_part, rem = e % per_part, row = rem / CH, c = rem % CH;
        const int k = key0(row >> 5) + (row & 31);
        unsigned char *dst = (part ? sv : sk) + tc::cm_offset(row, 8 * c, CH);
        if (k < N) tc::cp_async16(dst, QKVh + ((size_t)b * N + k) * 3 * D + (1 + part) * D + hh * DH + 8 * c);
        else *reinterpret_cast<uint4 *>(dst) = make_uint4(0, 0, 0, 0);
    }
    tc::cp_async_commit();
}

// Forward for sequences longer than a CTA can stage whole, under the band +
// sink mask: one CTA per (sample, head, query tile) with one softmax
// warpgroup and one MMA warp (the pipeline above), staging only the tile's
// queries and the keys and values of its visible chunks.
template <int DH>
__global__ void __launch_bounds__(160, 3)
attn_fwd_band_kernel(const __nv_bfloat16 *__restrict__ QKVh, const float *__restrict__ Hin,
                     __nv_bfloat16 *__restrict__ O, float *__restrict__ Hmid, float *__restrict__ LSE, int N, int D,
                     int NH, int mask, int W, int S, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t sbar[kRing], pbar[kRing], obar, dbar;
    __shared__ uint32_t tslot;
    __shared__ int s_err;
    const int nq = (N + kT - 1) / kT;
    const int qt = (int)(blockIdx.x % nq);
    const int64_t bh = blockIdx.x / nq;
    const int64_t b = bh / NH;
    const int hh = (int)(bh % NH);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, r = tid & 127;
    const TileSteps st(mask, W, S, N, qt);
    if (tid == 0) {
        for (int i = 0; i < kRing; ++i) {
            tc::mbar_init(&sbar[i], 1);
            tc::mbar_init(&pbar[i], 4);
        }
        tc::mbar_init(&obar, 4);
        tc::mbar_init(&dbar, 1);
        tc::fence_mbar_init();
        s_err = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&tslot, 128);
        tc::tmem_relinquish();
    }
    unsigned char *sq = smem, *sk = sq + kT * DH * 2, *sv = sk + st.n * 32 * DH * 2;
    stage_tile<DH>(sq, sk, sv, QKVh, b, hh, N, D, qt, st.n, [&](int i) { return st.key0(i); });
    tc::cp_async_wait<0>();
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tm = tslot;
    if (warp == 4) {
        if (lane == 0) {
            fwd_tile_mma<DH>(tm, desc_k<DH>(tc::smem_u32(sq), 0, 0), desc_k<DH>(tc::smem_u32(sk), 0, 0),
                             desc_mn<DH>(tc::smem_u32(sv), 0, 0), st.n, [](int i) { return 32 * i; }, sbar, pbar, &obar,
                             0, 0u, 0u, err, &s_err);
            tc::mma_commit(&dbar);
            tc::mbar_wait(&dbar, 0, 1u << 22);
        }
    } else {
        const uint32_t tl = tm + ((uint32_t)(32 * warp) << 16);
        const int t = qt * kT + r, t0w = qt * kT + 32 * warp;
        float mref, l, o[DH];
        if (fwd_tile_softmax<DH>(tl, st.n, [&](int i) { return st.key0(i); }, t, t0w, mask, W, S, N, sbar, pbar, 0u,
                                 err, &s_err, mref, l, o) &&
            t < N)
            fwd_row_out<DH>(o, mref, l, b, t, hh, N, D, NH, Hin, O, Hmid, LSE);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tslot, 128);
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
                if (!wg_wait(&bar[wg], phase, err, kWaitCode + 8 * 61)) s_err[wg] = 1;
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
                if (!wg_wait(&bar[wg], phase, err, kWaitCode + 8 * 62)) s_err[wg] = 1;
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
                if (!wg_wait(&bar[wg], phase, err, kWaitCode + 8 * 63)) s_err[wg] = 1;
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
                if (!wg_wait(&bar[wg], phase, err, kWaitCode + 8 * 64)) s_err[wg] = 1;
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

// ---------------------------------------------------------------------------
// Backward for long band sequences (the gradient of attn_fwd_band_kernel).
// One CTA (one warpgroup, 128 TMEM columns) per task; the tasks of a
// (sample, head):
//   query tile qt      dQ of queries qt * 128 + r over the tile's visible
//                      32-key chunks (those of the forward)
//   key tile kt        dK, dV of the band keys kt * 128 + r (S <= k < N)
//                      over the queries that see them (k .. k + W)
//   sink tile st       dK, dV of the sink keys st * 128 + r (k < S) over
//                      every query tile from st on (128 queries staged per
//                      tile); these tasks run longest and come first in the
//                      grid.  Every row is summed in one fixed order, so the
//                      gradient does not depend on scheduling (only the bias
//                      column sums are gathered by FP32 atomics).
// Steps are 32 keys (query tiles) or 32 queries wide.  TMEM: scores at
// [0, 32), dP at [32, 64); P^T in BF16 over [0, 16) and dS over [32, 48);
// accumulators at 64 (dQ or dV) and 96 (dK).  Rows whose gradient a task does
// not own (sink keys in a key tile, keys at or past N) compute unused values:
// a row of dK or dV depends only on its own row of P^T and dS^T.
// ---------------------------------------------------------------------------

// Queries t0 .. t0 + cnt - 1 (zero beyond N) at rows 0 .. cnt - 1: Q (by
// cp.async) into sq, dO in BF16 into sg, Ln = -log2(e) LSE and
// Dn = -(dO . O) / sqrt(d_h) into Ln, Dn.
template <int DH>
__device__ __forceinline__ void stage_queries(unsigned char *sq, unsigned char *sg, float *Ln, float *Dn,
                                              const __nv_bfloat16 *__restrict__ QKVh, const __nv_bfloat16 *__restrict__ O,
                                              const float *__restrict__ dO, const float *__restrict__ LSE, int64_t b,
                                              int hh, int N, int D, int NH, int t0, int cnt)
{
    constexpr int CH = DH / 8;
    for (int e = threadIdx.x; e < cnt * CH; e += blockDim.x) {
        const int row = e / CH, c = e % CH, t = t0 + row;
        unsigned char *dst = sq + tc::cm_offset(row, 8 * c, CH);
        if (t < N) tc::cp_async16(dst, QKVh + ((size_t)b * N + t) * 3 * D + hh * DH + 8 * c);
        else *reinterpret_cast<uint4 *>(dst) = make_uint4(0, 0, 0, 0);
    }
    tc::cp_async_commit();
    for (int row = threadIdx.x; row < cnt; row += blockDim.x) {
        const int t = t0 + row;
        float dd = 0.f, lse = 0.f;
        if (t < N) {
            const size_t rr = (size_t)b * N + t;
            const float4 *gp = reinterpret_cast<const float4 *>(dO + rr * D + hh * DH);
            const uint4 *op = reinterpret_cast<const uint4 *>(O + rr * D + hh * DH);
#pragma unroll
            for (int c = 0; c < CH; ++c) {
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
                *reinterpret_cast<uint4 *>(sg + tc::cm_offset(row, 8 * c, CH)) = make_uint4(
                    pack_bf2(g0.x, g0.y), pack_bf2(g0.z, g0.w), pack_bf2(g1.x, g1.y), pack_bf2(g1.z, g1.w));
            }
            lse = LSE[rr * NH + hh];
        } else {
#pragma unroll
            for (int c = 0; c < CH; ++c)
                *reinterpret_cast<uint4 *>(sg + tc::cm_offset(row, 8 * c, CH)) = make_uint4(0, 0, 0, 0);
        }
        Ln[row] = -lse * kLog2e;
        Dn[row] = -dd * rsqrtf((float)DH);
    }
}

// Keys key0(i) + j, i < nchunks, j < 32 (zero at or beyond klim) at rows
// 32 i + j of sk (part 1) and sv (part 2).
template <int DH, class Key0>
__device__ __forceinline__ void stage_keys(unsigned char *sk, unsigned char *sv, const __nv_bfloat16 *__restrict__ QKVh,
                                           int64_t b, int hh, int N, int D, int nchunks, Key0 key0, int klim)
{
    constexpr int CH = DH / 8;
    const int per_part = nchunks * 32 * CH;
    for (int e = threadIdx.x; e < 2 * per_part; e += blockDim.x) {
        const int part = e / per_part, rem = e % per_part, row = rem / CH, c = rem % CH;
        const int k = key0(row >> 5) + (row & 31);
        unsigned char *dst = (part ? sv : sk) + tc::cm_offset(row, 8 * c, CH);
        if (k < klim) tc::cp_async16(dst, QKVh + ((size_t)b * N + k) * 3 * D + (1 + part) * D + hh * DH + 8 * c);
        else *reinterpret_cast<uint4 *>(dst) = make_uint4(0, 0, 0, 0);
    }
    tc::cp_async_commit();
}

// Key rows: P^T and dS^T of 32 queries (compact rows q0 .. q0 + 31 of Ln, Dn;
// query indices tq .. tq + 31) for this thread's key k; kSome chunks mask
// query t by vis(t).
template <int KIND, class Vis>
__device__ __forceinline__ void key_grads32(const float (&s)[32], const float (&dp)[32], const float *Ln,
                                            const float *Dn, int q0, int tq, Vis vis, float sc2, float scale,
                                            uint32_t (&pp)[16], uint32_t (&dd)[16])
{
    const float2 a2 = make_float2(sc2, sc2), c2 = make_float2(scale, scale);
#pragma unroll
    for (int j4 = 0; j4 < 8; ++j4) {
        const float4 l4 = *reinterpret_cast<const float4 *>(Ln + q0 + 4 * j4);
        const float4 d4 = *reinterpret_cast<const float4 *>(Dn + q0 + 4 * j4);
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
            const int j = 4 * j4 + 2 * e2;
            float2 x = __ffma2_rn(make_float2(s[j], s[j + 1]), a2,
                                  e2 ? make_float2(l4.z, l4.w) : make_float2(l4.x, l4.y));
            if constexpr (KIND == kSome) {
                if (!vis(tq + j)) x.x = -INFINITY;
                if (!vis(tq + j + 1)) x.y = -INFINITY;
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

// Largest number of visible 32-key chunks of a query tile (query tasks) and
// of 32-query chunks that see a key tile (key tasks) under the band mask.
__host__ __device__ __forceinline__ int band_query_chunks(int W, int S, int N, int kt)
{
    const int qc0 = 4 * kt, qc1 = min((N + 31) / 32, (kt * kT + kT - 1 + W) / 32 + 1);
    return max(0, qc1 - qc0);
}

template <int DH>
__global__ void __launch_bounds__(128, 3)
attn_bwd_band_kernel(const __nv_bfloat16 *__restrict__ QKVh, const __nv_bfloat16 *__restrict__ O,
                     const float *__restrict__ dO, const float *__restrict__ LSE, unsigned char *__restrict__ dQKVt,
                     float *__restrict__ bsum, int N, int D, int NH, int mask, int W, int S, int nq, int nst,
                     int64_t nbh, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ float csum[3 * DH];
    __shared__ uint64_t bar, dbar;
    __shared__ uint32_t tslot;
    __shared__ int s_err;
    // the sink tasks (one per sample, head and sink tile, each over every
    // query tile from its own on) come first in the grid: they run longest
    const int64_t nsink = nbh * nst;
    int kind_of_task, tile, stile = 0;
    int64_t bh;
    if ((int64_t)blockIdx.x < nsink) {
        kind_of_task = 2;  // sink keys stile * 128 + r
        bh = blockIdx.x / nst;
        stile = (int)(blockIdx.x % nst);
        tile = stile;
    } else {
        const int64_t rr = blockIdx.x - nsink;
        bh = rr / (2 * nq);
        const int task = (int)(rr % (2 * nq));
        kind_of_task = task < nq ? 0 : 1;  // query tile / key tile
        tile = task % nq;
    }
    const int64_t b = bh / NH;
    const int hh = (int)(bh % NH);
    const int tid = threadIdx.x, warp = tid >> 5, r = tid;
    if (kind_of_task == 1 && min(N, tile * kT + kT) <= max(S, tile * kT)) return;  // no band key in the tile
    if (kind_of_task == 2 && stile * kT >= min(S, N)) return;                      // no sink key in the tile
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_init(&dbar, 1);
        tc::fence_mbar_init();
        s_err = 0;
    }
    for (int j = tid; j < 3 * DH; j += blockDim.x) csum[j] = 0.f;
    if (warp == 0) {
        tc::tmem_alloc(&tslot, 128);
        tc::tmem_relinquish();
    }
    // shared memory: the 128-row operand tile(s) first, then the chunked rows
    const TileSteps st(mask, W, S, N, tile);
    int nsteps = 0;
    unsigned char *sA = smem, *sB = sA + kT * DH * 2;  // query task: Q, dO tile; key tasks: K, V tile
    unsigned char *sC = sB + kT * DH * 2;                 // query task: K chunks; key tasks: Q chunks
    unsigned char *sD;                                    // V chunks / dO chunks
    float *Ln, *Dn;
    if (kind_of_task == 0) {
        nsteps = st.n;
        sD = sC + nsteps * 32 * DH * 2;
        Ln = reinterpret_cast<float *>(sD + nsteps * 32 * DH * 2);
        Dn = Ln + kT;
        stage_queries<DH>(sA, sB, Ln, Dn, QKVh, O, dO, LSE, b, hh, N, D, NH, tile * kT, kT);
        stage_keys<DH>(sC, sD, QKVh, b, hh, N, D, nsteps, [&](int i) { return st.key0(i); }, N);
    } else {
        const int k0 = tile * kT;
        stage_keys<DH>(sA, sB, QKVh, b, hh, N, D, 4, [&](int i) { return k0 + 32 * i; },
                       kind_of_task == 1 ? N : min(S, N));
        // key tile: the queries k0 .. k0 + 127 + W in one stage; sink tile:
        // the query tiles from its own on, 128 queries (4 steps) per stage
        const int staged = kind_of_task == 1 ? band_query_chunks(W, S, N, tile) : 4;
        nsteps = kind_of_task == 1 ? staged : 4 * (nq - tile);
        sD = sC + staged * 32 * DH * 2;
        Ln = reinterpret_cast<float *>(sD + staged * 32 * DH * 2);
        Dn = Ln + staged * 32;
        stage_queries<DH>(sC, sD, Ln, Dn, QKVh, O, dO, LSE, b, hh, N, D, NH, k0, staged * 32);
    }
    tc::cp_async_wait<0>();
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tm = tslot, tl = tm + ((uint32_t)(32 * warp) << 16);
    const float scale = rsqrtf((float)DH), sc2 = scale * kLog2e;
    const uint32_t idesc_s = tc::idesc_bf16(kT, 32);
    const uint32_t idesc_p = tc::idesc_bf16(kT, DH) | (1u << 16);  // B read MN-major
    const uint32_t uA = tc::smem_u32(sA), uB = tc::smem_u32(sB), uC = tc::smem_u32(sC), uD = tc::smem_u32(sD);
    uint32_t phase = 0;
    auto wait_mma = [&](int code) {
        if (!mwait(&bar, phase)) {
            if ((tid & 31) == 0) atomicExch(err, code + (kind_of_task << 16));
            s_err = 1;
        }
        phase ^= 1u;
        tc::tc_fence_after();
    };
    for (int i = 0; i < nsteps; ++i) {
        // a sink task restages the next query tile once the previous step's
        // products (which read the staged rows) have landed (checked below)
        if (kind_of_task == 2 && i > 0 && (i & 3) == 0) {
            stage_queries<DH>(sC, sD, Ln, Dn, QKVh, O, dO, LSE, b, hh, N, D, NH, (tile + (i >> 2)) * kT, kT);
            tc::cp_async_wait<0>();
            tc::fence_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            tc::tc_fence_after();
        }
        const int crow = kind_of_task == 2 ? 32 * (i & 3) : 32 * i;  // the step's staged rows
        // scores: query task S = Q K_c^T, dP = dO V_c^T; key tasks S^T = K Q_c^T, dP^T = V dO_c^T
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < DH / 16; ++ks) {
                tc::mma_bf16(tm, desc_k<DH>(uA, 0, ks), desc_k<DH>(uC, crow, ks), idesc_s, ks > 0 ? 1u : 0u);
                tc::mma_bf16(tm + 32, desc_k<DH>(uB, 0, ks), desc_k<DH>(uD, crow, ks), idesc_s, ks > 0 ? 1u : 0u);
            }
            tc::mma_commit(&bar);
        }
        __syncwarp();
        wait_mma(kWaitCode + 8 * 51);
        float sv[32], dp[32];
        uint32_t pp[16], dd[16];
        bool any;
        if (kind_of_task == 0) {
            const int t = tile * kT + r, t0w = tile * kT + 32 * warp, k0 = st.key0(i);
            const int kind = chunk_kind(mask, W, S, N, t0w, k0);
            any = kind != kNone;
            if (any) {
                tc::tmem_ld32(tl, sv);
                tc::tmem_ld32(tl + 32, dp);
                tc::tmem_wait_ld();
                if (kind == kAll) query_grads32<kAll>(sv, dp, t, k0, mask, W, S, N, sc2, scale, Ln[r], Dn[r], dd);
                else query_grads32<kSome>(sv, dp, t, k0, mask, W, S, N, sc2, scale, Ln[r], Dn[r], dd);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) dd[j] = 0u;
            }
            tmem_st16(tl + 32, dd);  // dS over dP already read
        } else {
            const int k = tile * kT + r;
            const int k0w = tile * kT + 32 * warp;
            const int tq = kind_of_task == 1 ? tile * kT + 32 * i : (tile + (i >> 2)) * kT + crow;
            // key tiles: band keys (query t sees key k iff 0 <= t - k <= W);
            // sink tiles: sink keys (t >= k); other rows are not this task's
            const int kind = kind_of_task == 1 ? chunk_kind(mask, W, 0, N, tq, k0w)
                                               : chunk_kind(SG_MASK_DENSE, W, 0, N, tq, k0w);
            any = kind != kNone;
            if (any) {
                tc::tmem_ld32(tl, sv);
                tc::tmem_ld32(tl + 32, dp);
                tc::tmem_wait_ld();
                const uint32_t lim = kind_of_task == 1 ? (uint32_t)W : 0x7fffffffu;
                auto vis = [&](int t) { return (uint32_t)(t - k) <= lim && t < N; };
                if (kind == kAll) key_grads32<kAll>(sv, dp, Ln, Dn, crow, tq, vis, sc2, scale, pp, dd);
                else key_grads32<kSome>(sv, dp, Ln, Dn, crow, tq, vis, sc2, scale, pp, dd);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) pp[j] = dd[j] = 0u;
            }
            tmem_st16(tl, pp);       // P^T over S^T already read
            tmem_st16(tl + 32, dd);  // dS^T over dP^T already read
        }
        tc::tmem_wait_st();
        tc::tc_fence_before();
        wg_sync(0);
        if (s_err) break;
        // products, accumulated in TMEM over the steps (K = 32 in two 16-row steps)
        if (tid == 0) {
            tc::tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
                if (kind_of_task == 0) {
                    mma_bf16_ta(tm + 64, tm + 32 + 8 * ks, desc_mn<DH>(uC, crow, ks), idesc_p, acc);  // dQ += dS K
                } else {
                    mma_bf16_ta(tm + 64, tm + 8 * ks, desc_mn<DH>(uD, crow, ks), idesc_p, acc);       // dV += P^T dO
                    mma_bf16_ta(tm + 96, tm + 32 + 8 * ks, desc_mn<DH>(uC, crow, ks), idesc_p, acc);  // dK += dS^T Q
                }
            }
            tc::mma_commit(&bar);
        }
        // The next step's scores overwrite what these products read.  Thread 0
        // waits for them and issues those scores after the barrier, so no
        // thread can still be polling this phase when the next one completes
        // (a parity wait cannot tell a phase from the one two later).
        if (tid == 0) wait_mma(kWaitCode + 8 * 52);
        else phase ^= 1u;
        tc::tc_fence_before();
        wg_sync(0);
        tc::tc_fence_after();
        if (s_err) break;
    }
    if (!s_err) {
        if (kind_of_task == 0) {
            float x[DH];
            tmem_ld_dh<DH>(tl + 64, x);
            tc::tmem_wait_ld();
            const int t = tile * kT + r;
            if (nsteps == 0 || t >= N) {
#pragma unroll
                for (int j = 0; j < DH; ++j) x[j] = 0.f;
            }
            put_rows<DH>(x, b, hh, N, D, t < N ? t : N, 0, dQKVt, csum);
        } else {
            float xv[DH], xk[DH];
            tmem_ld_dh<DH>(tl + 64, xv);
            tmem_ld_dh<DH>(tl + 96, xk);
            tc::tmem_wait_ld();
            const int k = tile * kT + r;
            const bool own = kind_of_task == 1 ? (k >= S && k < N) : (k < S && k < N);
            if (!own || nsteps == 0) {
#pragma unroll
                for (int j = 0; j < DH; ++j) xv[j] = xk[j] = 0.f;
            }
            put_rows<DH>(xk, b, hh, N, D, own ? k : N, 1, dQKVt, csum);
            put_rows<DH>(xv, b, hh, N, D, own ? k : N, 2, dQKVt, csum);
        }
    }
    if (s_err && tid == 0) {  // let this thread's MMAs land before TMEM is freed
        tc::mma_commit(&dbar);
        tc::mbar_wait(&dbar, 0, 1u << 20);
    }
    tc::tc_fence_before();
    __syncthreads();
    for (int j = tid; j < 3 * DH; j += blockDim.x)
            if (csum[j] != 0.f) atomicAdd(bsum + (size_t)b * 3 * D + (j / DH) * D + hh * DH + j % DH, csum[j]);
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tslot, 128);
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

// Largest number of visible 32-key chunks of a query tile (TileSteps).
static int band_max_tile_chunks(const sg_config &c)
{
    const int nq = (c.N + kT - 1) / kT;
    int best = 0;
    for (int qt = 0; qt < nq; ++qt) {
        const int tile0 = qt * kT, tile1 = std::min(tile0 + kT, c.N) - 1;
        const int cend = std::min(4 * (qt + 1), (c.N + 31) / 32);
        const int ns = (std::min(c.S, tile1 + 1) + 31) / 32;
        const int bstart = std::max(ns, std::max(0, tile0 - c.W) / 32);
        best = std::max(best, ns + std::max(0, cend - bstart));
    }
    return best;
}

static size_t band_fwd_smem(const sg_config &c)
{
    const int dh = c.d / c.n_heads;
    return (size_t)kT * dh * 2 + (size_t)2 * band_max_tile_chunks(c) * 32 * dh * 2;
}

static size_t band_bwd_smem(const sg_config &c)
{
    const int dh = c.d / c.n_heads, nq = (c.N + kT - 1) / kT;
    int nqc = 0;
    for (int kt = 0; kt < nq; ++kt) nqc = std::max(nqc, band_query_chunks(c.W, c.S, c.N, kt));
    const size_t tile = (size_t)2 * kT * dh * 2;
    const size_t q = tile + (size_t)2 * band_max_tile_chunks(c) * 32 * dh * 2 + 2 * kT * sizeof(float);
    const size_t k = tile + (size_t)2 * nqc * 32 * dh * 2 + (size_t)2 * nqc * 32 * sizeof(float);
    const size_t sk = tile + (size_t)2 * 4 * 32 * dh * 2 + 2 * kT * sizeof(float);
    return std::max(q, std::max(k, sk));
}

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

// Band masks on sequences beyond the staged kernels' shared memory: the
// per-tile tcgen05 kernels, where a tile's keys (and a key tile's queries)
// fit in 72 KB.
bool attn_band_supported(const sg_config &c)
{
    const int dh = c.d / c.n_heads;
    return c.precision == SG_BF16 && (dh == 16 || dh == 32) && c.d % 8 == 0 && c.mask_kind != SG_MASK_DENSE &&
           c.N >= 1 && !attn_mma_supported(c) && band_bwd_smem(c) <= 72 * 1024;
}

sg_status launch_attn_fwd_band(const sg_config &c, const __nv_bfloat16 *QKVh, const float *Hin, __nv_bfloat16 *O,
                               float *Hmid, float *LSE, int Bc, int *err, cudaStream_t st)
{
    const int dh = c.d / c.n_heads, nq = (c.N + kT - 1) / kT;
    const size_t smem = band_fwd_smem(c);
    auto go = [&](auto kern) -> sg_status {
        SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<(unsigned)((int64_t)Bc * c.n_heads * nq), 160, smem, ::sg::counted(st)>>>(
            QKVh, Hin, O, Hmid, LSE, c.N, c.d, c.n_heads, c.mask_kind, c.W, c.S, err);
        return check_launch("attn_fwd_band_kernel");
    };
    return dh == 16 ? go(attn_fwd_band_kernel<16>) : go(attn_fwd_band_kernel<32>);
}

sg_status launch_attn_bwd_band(const sg_config &c, const __nv_bfloat16 *QKVh, const __nv_bfloat16 *O,
                               const float *dO, const float *LSE, unsigned char *dQKVt, float *bsum, int Bc,
                               int *err, cudaStream_t st)
{
    const int dh = c.d / c.n_heads, nq = (c.N + kT - 1) / kT, nst = (c.S + kT - 1) / kT;
    const size_t smem = band_bwd_smem(c);
    SG_CUDA_TRY(cudaMemsetAsync(bsum, 0, (size_t)Bc * 3 * c.d * sizeof(float), st));  // gathered by atomics
    const int64_t nbh = (int64_t)Bc * c.n_heads;
    auto go = [&](auto kern) -> sg_status {
        SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<(unsigned)(nbh * (2 * nq + nst)), 128, smem, ::sg::counted(st)>>>(
            QKVh, O, dO, LSE, dQKVt, bsum, c.N, c.d, c.n_heads, c.mask_kind, c.W, c.S, nq, nst, nbh, err);
        return check_launch("attn_bwd_band_kernel");
    };
    return dh == 16 ? go(attn_bwd_band_kernel<16>) : go(attn_bwd_band_kernel<32>);
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
