// decode_bf16.cu -- BF16 ancestral sampler (Algorithm 2, KV-cache sampling)
// with the per-step GEMMs on the 5th-generation tensor cores (tcgen05).
//
// One CTA owns up to 128 samples (one MMA tile of M = 128 rows) for the
// whole sequence.  Thread (row r, half hf) of the 256 threads keeps the FP32
// residual stream h[r][32 hf .. 32 hf + 31] in registers.  Per step and layer:
//   LN1 (row statistics exchanged through shared memory) -> BF16 A tile in
//   shared memory -> tcgen05.mma QKV = A Wqkv^T (TMEM accumulators) ->
//   tcgen05.ld, bias, append (k_t, v_t) in BF16 to the tile's KV ring in HBM
//   -> attention of the thread's two heads over the visible keys, reading the
//   ring straight from HBM with one key prefetched -> residual -> LN2 ->
//   tcgen05.mma FFN1 -> GELU -> BF16 A2 tile -> tcgen05.mma FFN2 -> residual.
// The output head and the draw u < sigmoid(l_t) run in registers.  Weights
// are pre-packed in the operand layout of tc.cuh and streamed per layer into
// three shared-memory buffers by 1D bulk copies (TMA), each refilled as soon
// as the MMA that read it completes.  Every wait is bounded: on a timeout the
// kernel records an error word, stops issuing work, drains what it issued and
// frees its TMEM.
//
// KV ring layout per tile: [layer][slot][K|V][D/8][128 rows][8 bf16]; a warp
// (32 consecutive rows) moves 512 contiguous bytes per 16-byte access.
#include <cuda_bf16.h>

#include <algorithm>

#include "sg_internal.cuh"
#include "tc.cuh"

namespace sg {

namespace {

constexpr int kRows = 128;     // MMA M: samples per CTA tile
constexpr int kThreads = 256;  // two threads per row

struct Bf16Geom {
    int nslots;
    bool ring;
};

__host__ __device__ __forceinline__ Bf16Geom bgeom(int mask, int N, int W, int S)
{
    Bf16Geom g;
    g.ring = mask == SG_MASK_BAND_SINK && (int64_t)S + W + 1 < N;
    g.nslots = g.ring ? S + W + 1 : N;
    return g;
}

__device__ __forceinline__ int bslot(const Bf16Geom &g, int S, int W, int k)
{
    return (!g.ring || k < S) ? k : S + (k - S) % (W + 1);
}

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ uint32_t pack_bf2(float a, float b)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float round_bf(float x) { return __bfloat162float(__float2bfloat16(x)); }

// Pack W[rows][K] (fp32, row-major) into the bf16 core-matrix operand layout.
__global__ void pack_cm_kernel(const float *__restrict__ W, __nv_bfloat16 *__restrict__ dst,
                               int rows, int K)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * K) return;
    const int r = (int)(i / K), k = (int)(i % K);
    dst[tc::cm_offset(r, k, K / 8) >> 1] = __float2bfloat16(W[i]);
}

struct DecodeArgs {
    int N, L, dt, mask, W, S, dff;
    int rows_per_cta;           // active rows per CTA (<= 128)
    const float *w;             // master FP32 blob
    const float *wt;            // packed FP32 (biases)
    const unsigned char *bf;    // packed bf16 operands
    size_t bf_layer_bytes;      // per-layer stride of the packed operands
    BlobOff o;
    PackOff p;
    int64_t B;
    uint64_t seed;
    uint32_t sid;
    float band;
    int8_t *spins;
    float *logq;
    uint32_t *flags;
    unsigned char *kv;          // KV ring workspace
    int *err;                   // device error word
    // grouped models (d = 256 kernel): sample b uses model b / rows_per_model
    int64_t rows_per_model;
    int64_t stride_w, stride_wt;  // floats between consecutive models' blobs
    size_t stride_bf;             // bytes between consecutive models' packed chunks
    int max_keys;                 // capacity of the per-step key-offset table
    int kv_stages;                // d = 64: keys in flight per thread (2 or 3)
    // d = 256 with grouped models: ctas_per_model > 0 splits each model's rows
    // over that many CTAs (row counts differing by at most one); 0: CTA c
    // serves rows c rows_per_cta ..
    int ctas_per_model;
    int P, K, Nspins, latD, latL; // patching (d = 64 decode): spins per token, classes
};

// Element (r, k) of a core-matrix tile as a 16-byte group store of 8 bf16.
__device__ __forceinline__ void store8(unsigned char *tile, int r, int k0, int KG,
                                       const float *v)
{
    uint4 q;
    q.x = pack_bf2(v[0], v[1]);
    q.y = pack_bf2(v[2], v[3]);
    q.z = pack_bf2(v[4], v[5]);
    q.w = pack_bf2(v[6], v[7]);
    *reinterpret_cast<uint4 *>(tile + tc::cm_offset(r, k0, KG)) = q;
}

template <int D, int DFF>
__global__ void __launch_bounds__(kThreads, 1) decode_bf16_kernel(const __grid_constant__ DecodeArgs a)
{
    static_assert(D == 64, "this build of the BF16 decode serves d = 64");
    constexpr int DH = 16, HALF = D / 2, KG = D / 8, KG2 = DFF / 8;
    constexpr uint32_t QKV_COL = 0, FF2_COL = 3 * D, FF1_COL = 256;
    constexpr uint32_t A_BYTES = kRows * D * 2, A2_BYTES = kRows * DFF * 2;
    constexpr uint32_t WQKV_BYTES = 3 * D * D * 2, W1_BYTES = DFF * D * 2, W2_BYTES = D * DFF * 2;
    static_assert(3 * D <= 256 && DFF <= 256, "TMEM column plan");

    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Abuf = smem;
    unsigned char *A2buf = Abuf + A_BYTES;
    unsigned char *Wq = A2buf + A2_BYTES;
    unsigned char *W1s = Wq + WQKV_BYTES;
    unsigned char *W2s = W1s + W1_BYTES;
    float *xln = reinterpret_cast<float *>(W2s + W2_BYTES);  // [2][128][2]
    float *xhd = xln + 2 * kRows * 2;                          // [2][128][2]
    __shared__ uint64_t wbar[3], mbar;
    __shared__ uint32_t tslot;
    __shared__ int s_err;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = 32 * (warp & 3) + lane, hf = warp >> 2;
    const int64_t b = (int64_t)blockIdx.x * a.rows_per_cta + r;
    const bool active = r < a.rows_per_cta && b < a.B;
    const Bf16Geom g = bgeom(a.mask, a.N, a.W, a.S);
    const size_t slot_bytes = (size_t)2 * D * kRows * 2;
    const size_t layer_bytes = slot_bytes * g.nslots;
    unsigned char *kvt = a.kv + (size_t)blockIdx.x * layer_bytes * a.L;
    const int nfw = (a.N + 31) >> 5;
    const uint32_t tq = (uint32_t)(32 * (warp & 3)) << 16;  // TMEM lane base of this warp

    if (tid == 0) {
        tc::mbar_init(&wbar[0], 1);
        tc::mbar_init(&wbar[1], 1);
        tc::mbar_init(&wbar[2], 1);
        tc::mbar_init(&mbar, 1);
        tc::fence_mbar_init();
        s_err = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&tslot, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tslot;

    // weight streaming state (thread 0 only)
    uint32_t wphase[3] = {0, 0, 0}, mphase = 0;
    bool wpending[3] = {false, false, false};
    auto issue = [&](int which, int layer) {
        const unsigned char *src = a.bf + (size_t)layer * a.bf_layer_bytes;
        unsigned char *dst = which == 0 ? Wq : (which == 1 ? W1s : W2s);
        const uint32_t bytes = which == 0 ? WQKV_BYTES : (which == 1 ? W1_BYTES : W2_BYTES);
        const size_t off = which == 0 ? 0 : (which == 1 ? WQKV_BYTES : WQKV_BYTES + W1_BYTES);
        tc::mbar_arrive_expect_tx(&wbar[which], bytes);
        tc::bulk_g2s(dst, src + off, bytes, &wbar[which]);
        wpending[which] = true;
    };
    if (tid == 0) {
        issue(0, 0);
        issue(1, 0);
        issue(2, 0);
    }

    float h[HALF];
    float lq = 0.f;
    int tok = 0;
    const float qscale = 0.25f;  // 1 / sqrt(16)

    // MMA helper run by thread 0: waits for the weights, issues the K steps,
    // commits to mbar.  Every thread then waits on mbar.
    auto gemm = [&](int which, const unsigned char *A, uint32_t a_kg, const unsigned char *Bw,
                    uint32_t n, uint32_t k_total, uint32_t col) {
        if (tid == 0) {
            bool ok = s_err == 0 && tc::mbar_wait(&wbar[which], wphase[which]);
            if (ok) {
                wphase[which] ^= 1u;
                wpending[which] = false;
                tc::tc_fence_after();
                const uint32_t idesc = tc::idesc_bf16(kRows, (int)n);
                const uint32_t sa = tc::smem_u32(A), sb = tc::smem_u32(Bw);
                for (uint32_t s = 0; s < k_total / 16; ++s)
                    tc::mma_bf16(tmem + col, tc::smem_desc(sa + 256 * s, 128, a_kg * 128),
                                 tc::smem_desc(sb + 256 * s, 128, a_kg * 128), idesc, s > 0);
            } else {
                atomicExch(a.err, 1);
                s_err = 1;
            }
            tc::mma_commit(&mbar);
        }
        __syncwarp();
        if (!tc::mbar_wait(&mbar, mphase)) {
            if (lane == 0) atomicExch(a.err, 2);
            s_err = 1;
        }
        mphase ^= 1u;
        __syncthreads();  // makes s_err uniform before anyone branches on it
        tc::tc_fence_after();
    };

    for (int t = 0; t < a.N && !s_err; ++t) {
        // concatenated positional embedding
        {
            const float *pos = a.w + a.o.pos + (size_t)t * (D - a.dt);
#pragma unroll
            for (int j = 0; j < HALF; ++j) {
                const int d = HALF * hf + j;
                h[j] = d < a.dt ? __ldg(a.w + a.o.tok + tok * a.dt + d) : __ldg(pos + d - a.dt);
            }
        }
        int n_sink, band_lo;
        visible_ranges(a.mask, a.W, a.S, t, n_sink, band_lo);
        const int slot_t = bslot(g, a.S, a.W, t);

        for (int l = 0; l < a.L; ++l) {
            const LayerOff &o = a.o.L[l];
            const bool last = (t == a.N - 1) && (l == a.L - 1);
            const int nl = l + 1 < a.L ? l + 1 : 0;  // layer of the next use of each buffer
            // ---- LN1 -> A tile
            auto layernorm_to = [&](const float *gam, const float *bet) {
                float s1 = 0.f, s2 = 0.f;
#pragma unroll
                for (int j = 0; j < HALF; ++j) {
                    s1 += h[j];
                    s2 += h[j] * h[j];
                }
                xln[(hf * kRows + r) * 2] = s1;
                xln[(hf * kRows + r) * 2 + 1] = s2;
                __syncthreads();
                const float t1 = xln[r * 2] + xln[(kRows + r) * 2];
                const float t2 = xln[r * 2 + 1] + xln[(kRows + r) * 2 + 1];
                const float mean = t1 * (1.0f / D);
                const float var = fmaxf(t2 * (1.0f / D) - mean * mean, 0.f);
                const float rs = 1.0f / sqrtf(var + 1e-5f);
#pragma unroll
                for (int c = 0; c < HALF / 8; ++c) {
                    float v[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int d = HALF * hf + 8 * c + j;
                        v[j] = (h[8 * c + j] - mean) * rs * __ldg(gam + d) + __ldg(bet + d);
                    }
                    store8(Abuf, r, HALF * hf + 8 * c, KG, v);
                }
                tc::fence_async_smem();
                tc::tc_fence_before();
                __syncthreads();
            };
            layernorm_to(a.w + o.ln1g, a.w + o.ln1b);
            gemm(0, Abuf, KG, Wq, 3 * D, D, QKV_COL);
            if (tid == 0 && !last && !s_err) issue(0, nl);
            if (s_err) break;
            // ---- QKV epilogue: bias, KV append, attention of heads 2hf, 2hf+1
            {
                float q[HALF], kk[HALF], vv[HALF];
                tc::tmem_ld32(tmem + tq + QKV_COL + HALF * hf, q);
                tc::tmem_ld32(tmem + tq + QKV_COL + D + HALF * hf, kk);
                tc::tmem_ld32(tmem + tq + QKV_COL + 2 * D + HALF * hf, vv);
                tc::tmem_wait_ld();
                const float *bq = a.wt + a.p.bqkv[l];
#pragma unroll
                for (int j = 0; j < HALF; ++j) {
                    q[j] = (q[j] + __ldg(bq + HALF * hf + j)) * qscale;
                    kk[j] = round_bf(kk[j] + __ldg(bq + D + HALF * hf + j));
                    vv[j] = round_bf(vv[j] + __ldg(bq + 2 * D + HALF * hf + j));
                }
                unsigned char *kvl = kvt + (size_t)l * layer_bytes;
                if (active) {
                    uint4 *dk = reinterpret_cast<uint4 *>(kvl + (size_t)slot_t * slot_bytes);
                    uint4 *dv = dk + (D / 8) * kRows;
#pragma unroll
                    for (int c = 0; c < HALF / 8; ++c) {
                        uint4 x, y;
                        x.x = pack_bf2(kk[8 * c], kk[8 * c + 1]);
                        x.y = pack_bf2(kk[8 * c + 2], kk[8 * c + 3]);
                        x.z = pack_bf2(kk[8 * c + 4], kk[8 * c + 5]);
                        x.w = pack_bf2(kk[8 * c + 6], kk[8 * c + 7]);
                        y.x = pack_bf2(vv[8 * c], vv[8 * c + 1]);
                        y.y = pack_bf2(vv[8 * c + 2], vv[8 * c + 3]);
                        y.z = pack_bf2(vv[8 * c + 4], vv[8 * c + 5]);
                        y.w = pack_bf2(vv[8 * c + 6], vv[8 * c + 7]);
                        dk[(4 * hf + c) * kRows + r] = x;
                        dv[(4 * hf + c) * kRows + r] = y;
                    }
                }
                // the current key from registers
                float m0, m1, l0 = 1.f, l1 = 1.f, acc[HALF];
                {
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll
                    for (int j = 0; j < DH; ++j) {
                        s0 += q[j] * kk[j];
                        s1 += q[DH + j] * kk[DH + j];
                    }
                    m0 = s0;
                    m1 = s1;
#pragma unroll
                    for (int j = 0; j < HALF; ++j) acc[j] = vv[j];
                }
                const int nk = active ? n_sink + band_count(t, band_lo) - 1 : 0;  // keys < t
                const uint4 *kb = reinterpret_cast<const uint4 *>(kvl) + (4 * hf) * kRows + r;
                auto key_of = [&](int i) { return i < n_sink ? i : band_lo + (i - n_sink); };
                uint4 ck[4], cv[4];
                if (nk > 0) {
                    const uint4 *p = kb + (size_t)bslot(g, a.S, a.W, key_of(0)) * (slot_bytes / 16);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        ck[c] = __ldcg(p + c * kRows);
                        cv[c] = __ldcg(p + (D / 8) * kRows + c * kRows);
                    }
                }
                for (int i = 0; i < nk; ++i) {
                    uint4 nk4[4], nv4[4];
                    if (i + 1 < nk) {
                        const uint4 *p =
                            kb + (size_t)bslot(g, a.S, a.W, key_of(i + 1)) * (slot_bytes / 16);
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            nk4[c] = __ldcg(p + c * kRows);
                            nv4[c] = __ldcg(p + (D / 8) * kRows + c * kRows);
                        }
                    }
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const uint32_t w0[4] = {ck[c].x, ck[c].y, ck[c].z, ck[c].w};
                        const uint32_t w1[4] = {ck[c + 2].x, ck[c + 2].y, ck[c + 2].z, ck[c + 2].w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            s0 += q[8 * c + 2 * j] * bf_lo(w0[j]) + q[8 * c + 2 * j + 1] * bf_hi(w0[j]);
                            s1 += q[DH + 8 * c + 2 * j] * bf_lo(w1[j]) +
                                  q[DH + 8 * c + 2 * j + 1] * bf_hi(w1[j]);
                        }
                    }
                    const float n0 = fmaxf(m0, s0), n1 = fmaxf(m1, s1);
                    const float c0 = __expf(m0 - n0), p0 = __expf(s0 - n0);
                    const float c1 = __expf(m1 - n1), p1 = __expf(s1 - n1);
                    m0 = n0;
                    m1 = n1;
                    l0 = l0 * c0 + p0;
                    l1 = l1 * c1 + p1;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint32_t wv[4] = {cv[c].x, cv[c].y, cv[c].z, cv[c].w};
                        const float cc = c < 2 ? c0 : c1, pp = c < 2 ? p0 : p1;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            acc[8 * c + 2 * j] = acc[8 * c + 2 * j] * cc + pp * bf_lo(wv[j]);
                            acc[8 * c + 2 * j + 1] = acc[8 * c + 2 * j + 1] * cc + pp * bf_hi(wv[j]);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        ck[c] = nk4[c];
                        cv[c] = nv4[c];
                    }
                }
                const float i0 = 1.0f / l0, i1 = 1.0f / l1;
#pragma unroll
                for (int j = 0; j < DH; ++j) {
                    h[j] += acc[j] * i0;
                    h[DH + j] += acc[DH + j] * i1;
                }
            }
            // ---- LN2 -> A tile -> FFN1 -> GELU -> A2 tile -> FFN2
            layernorm_to(a.w + o.ln2g, a.w + o.ln2b);
            gemm(1, Abuf, KG, W1s, DFF, D, FF1_COL);
            if (tid == 0 && !last && !s_err) issue(1, nl);
            if (s_err) break;
            {
                const float *b1 = a.wt + a.p.b1[l];
#pragma unroll
                for (int c = 0; c < DFF / 2 / 32; ++c) {
                    float v[32];
                    tc::tmem_ld32(tmem + tq + FF1_COL + (DFF / 2) * hf + 32 * c, v);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int g8 = 0; g8 < 4; ++g8) {
                        float x[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int col = (DFF / 2) * hf + 32 * c + 8 * g8 + j;
                            x[j] = gelu_as(v[8 * g8 + j] + __ldg(b1 + col));
                        }
                        store8(A2buf, r, (DFF / 2) * hf + 32 * c + 8 * g8, KG2, x);
                    }
                }
                tc::fence_async_smem();
                tc::tc_fence_before();
                __syncthreads();
            }
            gemm(2, A2buf, KG2, W2s, D, DFF, FF2_COL);
            if (tid == 0 && !last && !s_err) issue(2, nl);
            if (s_err) break;
            {
                float v[32];
                tc::tmem_ld32(tmem + tq + FF2_COL + HALF * hf, v);
                tc::tmem_wait_ld();
                const float *b2 = a.wt + a.p.b2[l];
#pragma unroll
                for (int j = 0; j < HALF; ++j) h[j] += v[j] + __ldg(b2 + HALF * hf + j);
            }
        }
        if (s_err) break;
        // ---- output head and the draw
        {
            float s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int j = 0; j < HALF; ++j) {
                s1 += h[j];
                s2 += h[j] * h[j];
            }
            xln[(hf * kRows + r) * 2] = s1;
            xln[(hf * kRows + r) * 2 + 1] = s2;
            __syncthreads();
            const float mean = (xln[r * 2] + xln[(kRows + r) * 2]) * (1.0f / D);
            const float var = fmaxf((xln[r * 2 + 1] + xln[(kRows + r) * 2 + 1]) * (1.0f / D) -
                                        mean * mean, 0.f);
            const float rs = 1.0f / sqrtf(var + 1e-5f);
            float z0 = 0.f, z1 = 0.f;
#pragma unroll
            for (int j = 0; j < HALF; ++j) {
                const int d = HALF * hf + j;
                const float y = (h[j] - mean) * rs * __ldg(a.w + a.o.lnfg + d) + __ldg(a.w + a.o.lnfb + d);
                z0 += y * __ldg(a.w + a.o.Wh + d);
                z1 += y * __ldg(a.w + a.o.Wh + D + d);
            }
            xhd[(hf * kRows + r) * 2] = z0;
            xhd[(hf * kRows + r) * 2 + 1] = z1;
            __syncthreads();
            if (hf == 0) {
                z0 = xhd[r * 2] + xhd[(kRows + r) * 2] + __ldg(a.w + a.o.bh);
                z1 = xhd[r * 2 + 1] + xhd[(kRows + r) * 2 + 1] + __ldg(a.w + a.o.bh + 1);
                const float ell = z1 - z0;
                const float p = 1.0f / (1.0f + expf(-ell));
                const float u = philox_uniform(a.seed, (uint32_t)b, (uint32_t)t, a.sid, 0u);
                const int sp = u < p ? 1 : -1;
                lq += log_sigmoid_f((float)sp * ell);
                tok = (sp + 1) >> 1;
                if (active) {
                    a.spins[(size_t)b * a.N + t] = (int8_t)sp;
                    if (a.flags && fabsf(p - u) < a.band)
                        a.flags[(size_t)b * nfw + (t >> 5)] |= 1u << (t & 31);
                    if (!isfinite(ell)) atomicOr(a.err, 4);
                }
            }
        }
    }
    if (hf == 0 && active) a.logq[b] = lq;
    // drain: no bulk copy or MMA may be in flight when the CTA exits
    if (tid == 0)
        for (int i = 0; i < 3; ++i)
            if (wpending[i] && !tc::mbar_wait(&wbar[i], wphase[i])) atomicExch(a.err, 3);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Patched head (K = 2^P classes) of the BF16 decodes, for a row whose four
// quarter threads hold its final-LayerNorm output y at dims [Q qr, Q qr + Q)
// (w: this row's model's weight blob).  The classes go through zp, a tile idle
// at the head, in chunks of kHeadChunk: each quarter writes its partial logits
// over its dims ([4][128][chunk] floats) and the row's quarter-0 thread adds
// them.  A first pass keeps the row's running maximum and sum of
// exponentials; a second recomputes each chunk (or, with one chunk, reuses
// it) and walks the cumulative probabilities in class order, drawing the
// first class whose cumulative probability exceeds u.  Its log-probability is
// added to lq and the class is the next token.  A draw within the flag band of
// any cumulative boundary is flagged.  Only `writer` threads store spins,
// flags and the error word.  Every thread of the CTA must call it.
constexpr int kHeadChunk = 32;

template <int Q>
__device__ __forceinline__ void head_partials(const DecodeArgs &a, const float *w, const float (&y)[Q],
                                              int D, int r, int qr, float *zp, int c0, int kc)
{
    for (int k = 0; k < kc; ++k) {
        const float *wh = w + a.o.Wh + (size_t)(c0 + k) * D + Q * qr;
        float zk = 0.f;
#pragma unroll
        for (int j = 0; j < Q; ++j) zk += y[j] * __ldg(wh + j);
        zp[((size_t)qr * kRows + r) * kc + k] = zk;
    }
}

template <int Q>
__device__ __forceinline__ void patched_head(const DecodeArgs &a, const float *w, const float (&y)[Q],
                                             int D, int r, int qr, float *zp, int64_t b, int t,
                                             bool writer, int nfw, float &lq, int &tok)
{
    const int kc = min(a.K, kHeadChunk);
    auto logit = [&](int c0, int k) {
        float zk = __ldg(w + a.o.bh + c0 + k);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) zk += zp[((size_t)q4 * kRows + r) * kc + k];
        return zk;
    };
    // pass 1: the log-sum-exp (with one chunk: the chunk's max, then its sum)
    float mx = -INFINITY, se = 0.f;
    for (int c0 = 0; c0 < a.K; c0 += kc) {
        head_partials<Q>(a, w, y, D, r, qr, zp, c0, kc);
        __syncthreads();
        if (qr == 0) {
            float cm = mx;
            for (int k = 0; k < kc; ++k) cm = fmaxf(cm, logit(c0, k));
            float sc = 0.f;
            for (int k = 0; k < kc; ++k) sc += expf(logit(c0, k) - cm);
            se = se * expf(mx - cm) + sc;  // the first chunk: 0 * 0 + sc
            mx = cm;
        }
        if (c0 + kc < a.K) __syncthreads();  // the next chunk overwrites zp
    }
    const float lse = mx + logf(se);
    // pass 2: the draw
    const float u = qr == 0 ? philox_uniform(a.seed, (uint32_t)b, (uint32_t)t, a.sid, 0u) : 0.f;
    float cdf = 0.f, near = INFINITY, zc = 0.f;
    int cls = a.K - 1;
    bool found = false;
    for (int c0 = 0; c0 < a.K; c0 += kc) {
        if (kc < a.K) {
            __syncthreads();  // quarter 0 has read the previous chunk
            head_partials<Q>(a, w, y, D, r, qr, zp, c0, kc);
            __syncthreads();
        }
        if (qr == 0) {
            for (int k = 0; k < kc; ++k) {
                const float z = logit(c0, k);
                if (c0 + k < a.K - 1) {
                    cdf += expf(z - lse);
                    near = fminf(near, fabsf(u - cdf));
                    if (!found && u < cdf) {
                        cls = c0 + k;
                        zc = z;
                        found = true;
                    }
                } else if (!found) {
                    zc = z;
                }
            }
        }
    }
    if (qr == 0) {
        lq += zc - lse;
        tok = cls;
        if (writer) {
            for (int j = 0; j < a.P; ++j)
                a.spins[(size_t)b * a.Nspins + patch_site(t, j, a.P, a.latD, a.latL)] =
                    (int8_t)(((cls >> j) & 1) ? 1 : -1);
            if (a.flags && near < a.band) a.flags[(size_t)b * nfw + (t >> 5)] |= 1u << (t & 31);
            if (!isfinite(zc - lse)) atomicOr(a.err, 4);
        }
    }
}

// ---------------------------------------------------------------------------
// d = 64 (4 heads of 16, d_ff = 256) with four threads per sample: thread
// (row r, quarter qr) keeps h[r][16 qr .. 16 qr + 15] and serves head qr.
// The 512 threads (16 warps) keep twice as many KV loads in flight as two
// threads per row do, and split the LayerNorm and GELU epilogues four ways.
// Weights stream per layer into three buffers exactly as in the kernel above.
// ---------------------------------------------------------------------------
// NST: keys in flight per thread in the attention (2 or 3); PATCH: K-way head
template <int NST, bool PATCH>
__global__ void __launch_bounds__(512, 1) decode_bf16_d64_kernel(const __grid_constant__ DecodeArgs a)
{
    constexpr int D = 64, DFF = 256, DH = 16, KG = D / 8, KG2 = DFF / 8;
    constexpr uint32_t QKV_COL = 0, FF2_COL = 3 * D, FF1_COL = 256;
    constexpr uint32_t A_BYTES = kRows * D * 2, A2_BYTES = kRows * DFF * 2;
    constexpr uint32_t WQKV_BYTES = 3 * D * D * 2, W1_BYTES = DFF * D * 2, W2_BYTES = D * DFF * 2;

    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Abuf = smem;
    unsigned char *A2buf = Abuf + A_BYTES;
    unsigned char *Wq = A2buf + A2_BYTES;
    unsigned char *W1s = Wq + WQKV_BYTES;
    unsigned char *W2s = W1s + W1_BYTES;
    float *xln = reinterpret_cast<float *>(W2s + W2_BYTES);  // [4][128][2]
    float *xhd = xln + 4 * kRows * 2;                          // [4][128][2]
    uint32_t *koff = reinterpret_cast<uint32_t *>(xhd + 4 * kRows * 2);  // [N]
    // spare 32 KB KV stage after the key table (rounded to 1 KB), when it fits
    unsigned char *kvspare = reinterpret_cast<unsigned char *>(koff) + ((a.N * 4 + 1023) / 1024) * 1024;
    constexpr int nst = NST;
    __shared__ uint64_t wbar[3], mbar;
    __shared__ uint32_t tslot;
    __shared__ int s_err;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = 32 * (warp & 3) + lane, qr = warp >> 2;
    const int64_t b = (int64_t)blockIdx.x * a.rows_per_cta + r;
    const bool active = r < a.rows_per_cta && b < a.B;
    const Bf16Geom g = bgeom(a.mask, a.N, a.W, a.S);
    const size_t slot_bytes = (size_t)2 * D * kRows * 2;
    const size_t layer_bytes = slot_bytes * g.nslots;
    unsigned char *kvt = a.kv + (size_t)blockIdx.x * layer_bytes * a.L;
    const int nfw = (a.N + 31) >> 5;
    const uint32_t tq = (uint32_t)(32 * (warp & 3)) << 16;

    if (tid == 0) {
        tc::mbar_init(&wbar[0], 1);
        tc::mbar_init(&wbar[1], 1);
        tc::mbar_init(&wbar[2], 1);
        tc::mbar_init(&mbar, 1);
        tc::fence_mbar_init();
        s_err = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&tslot, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tslot;

    uint32_t wphase[3] = {0, 0, 0}, mphase = 0;
    bool wpending[3] = {false, false, false};
    auto issue = [&](int which, int layer) {
        const unsigned char *src = a.bf + (size_t)layer * a.bf_layer_bytes;
        unsigned char *dst = which == 0 ? Wq : (which == 1 ? W1s : W2s);
        const uint32_t bytes = which == 0 ? WQKV_BYTES : (which == 1 ? W1_BYTES : W2_BYTES);
        const size_t off = which == 0 ? 0 : (which == 1 ? WQKV_BYTES : WQKV_BYTES + W1_BYTES);
        tc::mbar_arrive_expect_tx(&wbar[which], bytes);
        tc::bulk_g2s(dst, src + off, bytes, &wbar[which]);
        wpending[which] = true;
    };
    if (tid == 0) {
        issue(0, 0);
        issue(1, 0);
        issue(2, 0);
    }

    float h[DH];
    float lq = 0.f;
    int tok = 0;
    const float qscale = 0.25f;  // 1 / sqrt(16)

    auto gemm = [&](int which, const unsigned char *A, uint32_t a_kg, const unsigned char *Bw,
                    uint32_t n, uint32_t k_total, uint32_t col) {
        if (tid == 0) {
            bool ok = s_err == 0 && tc::mbar_wait(&wbar[which], wphase[which]);
            if (ok) {
                wphase[which] ^= 1u;
                wpending[which] = false;
                tc::tc_fence_after();
                const uint32_t idesc = tc::idesc_bf16(kRows, (int)n);
                const uint32_t sa = tc::smem_u32(A), sb = tc::smem_u32(Bw);
                for (uint32_t s = 0; s < k_total / 16; ++s)
                    tc::mma_bf16(tmem + col, tc::smem_desc(sa + 256 * s, 128, a_kg * 128),
                                 tc::smem_desc(sb + 256 * s, 128, a_kg * 128), idesc, s > 0);
            } else {
                atomicExch(a.err, 1);
                s_err = 1;
            }
            tc::mma_commit(&mbar);
        }
        __syncwarp();
        if (!tc::mbar_wait(&mbar, mphase)) {
            if (lane == 0) atomicExch(a.err, 2);
            s_err = 1;
        }
        mphase ^= 1u;
        __syncthreads();
        tc::tc_fence_after();
    };

    // LayerNorm of the row (statistics from the four quarters) into the A tile
    auto layernorm_to = [&](const float *gam, const float *bet) {
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int j = 0; j < DH; ++j) {
            s1 += h[j];
            s2 += h[j] * h[j];
        }
        xln[(qr * kRows + r) * 2] = s1;
        xln[(qr * kRows + r) * 2 + 1] = s2;
        __syncthreads();
        float t1 = 0.f, t2 = 0.f;
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
            t1 += xln[(q4 * kRows + r) * 2];
            t2 += xln[(q4 * kRows + r) * 2 + 1];
        }
        const float mean = t1 * (1.0f / D);
        const float var = fmaxf(t2 * (1.0f / D) - mean * mean, 0.f);
        const float rs = 1.0f / sqrtf(var + 1e-5f);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int d = DH * qr + 8 * c + j;
                v[j] = (h[8 * c + j] - mean) * rs * __ldg(gam + d) + __ldg(bet + d);
            }
            store8(Abuf, r, DH * qr + 8 * c, KG, v);
        }
        tc::fence_async_smem();
        tc::tc_fence_before();
        __syncthreads();
    };

    for (int t = 0; t < a.N && !s_err; ++t) {
        {
            const float *pos = a.w + a.o.pos + (size_t)t * (D - a.dt);
#pragma unroll
            for (int j = 0; j < DH; ++j) {
                const int d = DH * qr + j;
                h[j] = d < a.dt ? __ldg(a.w + a.o.tok + tok * a.dt + d) : __ldg(pos + d - a.dt);
            }
        }
        int n_sink, band_lo;
        visible_ranges(a.mask, a.W, a.S, t, n_sink, band_lo);
        const int slot_t = bslot(g, a.S, a.W, t);
        const int nk_all = n_sink + band_count(t, band_lo) - 1;  // keys < t
        const int nk = active ? nk_all : 0;
        // ring offsets (in 16-byte units) of this step's visible keys, the same
        // for every row and layer: computed once, read as broadcasts
        for (int i = tid; i < nk_all; i += blockDim.x)
            koff[i] = (uint32_t)bslot(g, a.S, a.W, i < n_sink ? i : band_lo + (i - n_sink)) *
                      (uint32_t)(slot_bytes / 16);
        // (the first LayerNorm's barrier orders these writes before any read)

        for (int l = 0; l < a.L; ++l) {
            const LayerOff &o = a.o.L[l];
            const bool last = (t == a.N - 1) && (l == a.L - 1);
            const int nl = l + 1 < a.L ? l + 1 : 0;
            layernorm_to(a.w + o.ln1g, a.w + o.ln1b);
            gemm(0, Abuf, KG, Wq, 3 * D, D, QKV_COL);
            if (tid == 0 && !last && !s_err) issue(0, nl);
            if (s_err) break;
            {
                float q[DH], acc[DH], tmp[DH];
                const float *bq = a.wt + a.p.bqkv[l];
                tc::tmem_ld16(tmem + tq + QKV_COL + DH * qr, q);
                tc::tmem_ld16(tmem + tq + QKV_COL + D + DH * qr, tmp);
                tc::tmem_ld16(tmem + tq + QKV_COL + 2 * D + DH * qr, acc);
                tc::tmem_wait_ld();
                float m0 = 0.f, l0 = 1.f;
#pragma unroll
                for (int j = 0; j < DH; ++j) {
                    q[j] = (q[j] + __ldg(bq + DH * qr + j)) * qscale;
                    tmp[j] = round_bf(tmp[j] + __ldg(bq + D + DH * qr + j));      // k_t
                    acc[j] = round_bf(acc[j] + __ldg(bq + 2 * D + DH * qr + j));  // v_t
                    m0 += q[j] * tmp[j];
                }
                unsigned char *kvl = kvt + (size_t)l * layer_bytes;
                if (active) {
                    uint4 *dk = reinterpret_cast<uint4 *>(kvl + (size_t)slot_t * slot_bytes);
                    uint4 *dv = dk + (D / 8) * kRows;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        uint4 x, y;
                        x.x = pack_bf2(tmp[8 * c], tmp[8 * c + 1]);
                        x.y = pack_bf2(tmp[8 * c + 2], tmp[8 * c + 3]);
                        x.z = pack_bf2(tmp[8 * c + 4], tmp[8 * c + 5]);
                        x.w = pack_bf2(tmp[8 * c + 6], tmp[8 * c + 7]);
                        y.x = pack_bf2(acc[8 * c], acc[8 * c + 1]);
                        y.y = pack_bf2(acc[8 * c + 2], acc[8 * c + 3]);
                        y.z = pack_bf2(acc[8 * c + 4], acc[8 * c + 5]);
                        y.w = pack_bf2(acc[8 * c + 6], acc[8 * c + 7]);
                        dk[(2 * qr + c) * kRows + r] = x;
                        dv[(2 * qr + c) * kRows + r] = y;
                    }
                }
                // keys < t of head qr, staged through shared memory by cp.async:
                // kv_stages keys in flight per thread without holding registers.
                // Stages 0 and 1 are the A2 tile (idle until the GELU epilogue),
                // stage 2 the spare tile; each stage holds, per thread, K pieces
                // at +0, +8 KB and V pieces at +16 KB, +24 KB (conflict-free: the
                // 512 threads' 16-byte pieces are consecutive).
                const uint4 *kb = reinterpret_cast<const uint4 *>(kvl) + (2 * qr) * kRows + r;
                auto stage = [&](int s) { return (s < 2 ? A2buf + s * 32768 : kvspare) + tid * 16; };
                auto fetch = [&](int i, int s) {
                    const uint4 *p = kb + koff[i];
                    unsigned char *dst = stage(s);
                    tc::cp_async16(dst, p);
                    tc::cp_async16(dst + 8192, p + kRows);
                    tc::cp_async16(dst + 16384, p + (D / 8) * kRows);
                    tc::cp_async16(dst + 24576, p + (D / 8) * kRows + kRows);
                    tc::cp_async_commit();
                };
                for (int i = 0; i < nk && i < nst; ++i) fetch(i, i);
                for (int i = 0; i < nk; ++i) {
                    if (nst == 3 && i + 2 < nk) tc::cp_async_wait<2>();
                    else if (i + 1 < nk) tc::cp_async_wait<1>();
                    else tc::cp_async_wait<0>();
                    const int si = i % nst;
                    const unsigned char *src = stage(si);
                    uint4 ck[2], cv[2];
                    ck[0] = *reinterpret_cast<const uint4 *>(src);
                    ck[1] = *reinterpret_cast<const uint4 *>(src + 8192);
                    cv[0] = *reinterpret_cast<const uint4 *>(src + 16384);
                    cv[1] = *reinterpret_cast<const uint4 *>(src + 24576);
                    float s = 0.f;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const uint32_t wk[4] = {ck[c].x, ck[c].y, ck[c].z, ck[c].w};
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            s += q[8 * c + 2 * j] * bf_lo(wk[j]) + q[8 * c + 2 * j + 1] * bf_hi(wk[j]);
                    }
                    const float n0 = fmaxf(m0, s);
                    const float c0 = __expf(m0 - n0), p0 = __expf(s - n0);
                    m0 = n0;
                    l0 = l0 * c0 + p0;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const uint32_t wv[4] = {cv[c].x, cv[c].y, cv[c].z, cv[c].w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            acc[8 * c + 2 * j] = acc[8 * c + 2 * j] * c0 + p0 * bf_lo(wv[j]);
                            acc[8 * c + 2 * j + 1] = acc[8 * c + 2 * j + 1] * c0 + p0 * bf_hi(wv[j]);
                        }
                    }
                    // the stage is refilled only after its data has been consumed
                    if (i + nst < nk) fetch(i + nst, si);
                }
                const float inv = 1.0f / l0;
#pragma unroll
                for (int j = 0; j < DH; ++j) h[j] += acc[j] * inv;
            }
            layernorm_to(a.w + o.ln2g, a.w + o.ln2b);
            gemm(1, Abuf, KG, W1s, DFF, D, FF1_COL);
            if (tid == 0 && !last && !s_err) issue(1, nl);
            if (s_err) break;
            {
                const float *b1 = a.wt + a.p.b1[l];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    float v[32];
                    tc::tmem_ld32(tmem + tq + FF1_COL + 64 * qr + 32 * c, v);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int g8 = 0; g8 < 4; ++g8) {
                        float x[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            x[j] = gelu_as(v[8 * g8 + j] + __ldg(b1 + 64 * qr + 32 * c + 8 * g8 + j));
                        store8(A2buf, r, 64 * qr + 32 * c + 8 * g8, KG2, x);
                    }
                }
                tc::fence_async_smem();
                tc::tc_fence_before();
                __syncthreads();
            }
            gemm(2, A2buf, KG2, W2s, D, DFF, FF2_COL);
            if (tid == 0 && !last && !s_err) issue(2, nl);
            if (s_err) break;
            {
                float v[16];
                tc::tmem_ld16(tmem + tq + FF2_COL + DH * qr, v);
                tc::tmem_wait_ld();
                const float *b2 = a.wt + a.p.b2[l];
#pragma unroll
                for (int j = 0; j < DH; ++j) h[j] += v[j] + __ldg(b2 + DH * qr + j);
            }
        }
        if (s_err) break;
        {
            float s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int j = 0; j < DH; ++j) {
                s1 += h[j];
                s2 += h[j] * h[j];
            }
            xln[(qr * kRows + r) * 2] = s1;
            xln[(qr * kRows + r) * 2 + 1] = s2;
            __syncthreads();
            float t1 = 0.f, t2 = 0.f;
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
                t1 += xln[(q4 * kRows + r) * 2];
                t2 += xln[(q4 * kRows + r) * 2 + 1];
            }
            const float mean = t1 * (1.0f / D);
            const float var = fmaxf(t2 * (1.0f / D) - mean * mean, 0.f);
            const float rs = 1.0f / sqrtf(var + 1e-5f);
            if constexpr (PATCH) {
                // patched: K logits; this quarter's partial sums over its 16
                // dims go through the A2 tile (idle until the next step's attention)
                float y[DH];
#pragma unroll
                for (int j = 0; j < DH; ++j) {
                    const int d = DH * qr + j;
                    y[j] = (h[j] - mean) * rs * __ldg(a.w + a.o.lnfg + d) + __ldg(a.w + a.o.lnfb + d);
                }
                patched_head<DH>(a, a.w, y, D, r, qr, reinterpret_cast<float *>(A2buf), b, t, active, nfw,
                                 lq, tok);
            } else {
            float z0 = 0.f, z1 = 0.f;
#pragma unroll
            for (int j = 0; j < DH; ++j) {
                const int d = DH * qr + j;
                const float y = (h[j] - mean) * rs * __ldg(a.w + a.o.lnfg + d) + __ldg(a.w + a.o.lnfb + d);
                z0 += y * __ldg(a.w + a.o.Wh + d);
                z1 += y * __ldg(a.w + a.o.Wh + D + d);
            }
            xhd[(qr * kRows + r) * 2] = z0;
            xhd[(qr * kRows + r) * 2 + 1] = z1;
            __syncthreads();
            if (qr == 0) {
                z0 = __ldg(a.w + a.o.bh);
                z1 = __ldg(a.w + a.o.bh + 1);
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    z0 += xhd[(q4 * kRows + r) * 2];
                    z1 += xhd[(q4 * kRows + r) * 2 + 1];
                }
                const float ell = z1 - z0;
                const float p = 1.0f / (1.0f + expf(-ell));
                const float u = philox_uniform(a.seed, (uint32_t)b, (uint32_t)t, a.sid, 0u);
                const int sp = u < p ? 1 : -1;
                lq += log_sigmoid_f((float)sp * ell);
                tok = (sp + 1) >> 1;
                if (active) {
                    a.spins[(size_t)b * a.N + t] = (int8_t)sp;
                    if (a.flags && fabsf(p - u) < a.band)
                        a.flags[(size_t)b * nfw + (t >> 5)] |= 1u << (t & 31);
                    if (!isfinite(ell)) atomicOr(a.err, 4);
                }
            }
            }  // two-class head
            // tok lives in the qr == 0 thread, which is the only one that
            // reads it (the token columns are in quarter 0)
        }
    }
    if (qr == 0 && active) a.logq[b] = lq;
    if (tid == 0)
        for (int i = 0; i < 3; ++i)
            if (wpending[i] && !tc::mbar_wait(&wbar[i], wphase[i])) atomicExch(a.err, 3);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// d = 128 variant (8 heads of 16, d_ff = 512).  512 threads: thread (row r,
// quarter qr) keeps h[r][32 qr .. 32 qr + 31] and serves heads 2 qr, 2 qr + 1
// one after the other.  Weights are too large to hold per layer, so every
// layer is streamed as 11 chunks of 32 KB ([128 out rows x 128 K] operands):
// Wq, Wk, Wv, then (W1 rows 128j..) and (W2 K-slice 128j..) for j = 0..3,
// through a 3-stage ring of bulk copies.  TMEM: QKV at columns [0, 384), the
// FFN1 slice at [0, 128), the FFN2 accumulator at [384, 512).
// ---------------------------------------------------------------------------
constexpr int kChunkBytes = 128 * 128 * 2;
constexpr int kChunksPerLayer = 11;
constexpr int kStages = 3;

// chunk c of a layer, element (r, k) of the [128 x 128] operand
__global__ void pack_chunks128_kernel(const float *__restrict__ Wqkv,
                                      const float *__restrict__ W1,
                                      const float *__restrict__ W2, __nv_bfloat16 *__restrict__ dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)kChunksPerLayer * 128 * 128) return;
    const int c = (int)(i / (128 * 128)), r = (int)((i / 128) % 128), k = (int)(i % 128);
    float v;
    if (c < 3) v = Wqkv[(size_t)(128 * c + r) * 128 + k];
    else if ((c - 3) % 2 == 0) v = W1[(size_t)(128 * ((c - 3) / 2) + r) * 128 + k];
    else v = W2[(size_t)r * 512 + 128 * ((c - 4) / 2) + k];
    dst[(size_t)c * (kChunkBytes / 2) + (tc::cm_offset(r, k, 16) >> 1)] = __float2bfloat16(v);
}

__global__ void __launch_bounds__(512, 1) decode_bf16_d128_kernel(const __grid_constant__ DecodeArgs a)
{
    constexpr int D = 128, DH = 16, Q32 = 32, KG = D / 8;
    constexpr uint32_t QKV_COL = 0, FF1_COL = 0, FF2_COL = 384;
    constexpr uint32_t A_BYTES = kRows * D * 2;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Abuf = smem;
    unsigned char *A2buf = Abuf + A_BYTES;
    unsigned char *ring = A2buf + A_BYTES;
    float *xln = reinterpret_cast<float *>(ring + kStages * kChunkBytes);  // [4][128][2]
    float *xhd = xln + 4 * kRows * 2;                                     // [4][128][2]
    uint32_t *koff = reinterpret_cast<uint32_t *>(xhd + 4 * kRows * 2);   // [max_keys]
    // spare 32 KB KV stage after the key table (rounded to 1 KB)
    unsigned char *kvspare = reinterpret_cast<unsigned char *>(koff) + ((a.max_keys * 4 + 1023) / 1024) * 1024;
    __shared__ uint64_t full[kStages], mbar;
    __shared__ uint32_t tslot;
    __shared__ int s_err;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = 32 * (warp & 3) + lane, qr = warp >> 2;
    // With at most 64 rows per CTA, rows 64..127 mirror rows 0..63 (same
    // inputs, so every phase computes identical copies); a row and its mirror
    // (thread tid ^ 64) split the attention's keys and merge their partial
    // softmax states, doubling the KV loads in flight.  Only the row itself
    // writes the KV cache, spins and log q.
    const bool mirror_mode = a.rows_per_cta <= 64;
    const int rr = mirror_mode ? (r & 63) : r;  // the sample row this thread serves
    const bool is_mirror = mirror_mode && r >= 64;
    const int64_t b = (int64_t)blockIdx.x * a.rows_per_cta + rr;
    const bool active = rr < a.rows_per_cta && b < a.B;
    const Bf16Geom g = bgeom(a.mask, a.N, a.W, a.S);
    const size_t slot_bytes = (size_t)2 * D * kRows * 2;
    const size_t layer_bytes = slot_bytes * g.nslots;
    unsigned char *kvt = a.kv + (size_t)blockIdx.x * layer_bytes * a.L;
    const int nfw = (a.N + 31) >> 5;
    const uint32_t tq = (uint32_t)(32 * (warp & 3)) << 16;
    const int64_t total_chunks = (int64_t)a.N * a.L * kChunksPerLayer;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) tc::mbar_init(&full[s], 1);
        tc::mbar_init(&mbar, 1);
        tc::fence_mbar_init();
        s_err = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&tslot, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tslot;

    // chunk stream state (thread 0): chunk gidx lives in stage gidx % kStages
    int64_t next_load = 0, next_use = 0;
    uint32_t fphase[kStages] = {0, 0, 0}, mphase = 0;
    auto load_more = [&]() {
        while (next_load < total_chunks && next_load < next_use + kStages) {
            const int s = (int)(next_load % kStages);
            const int64_t lc = next_load % ((int64_t)a.L * kChunksPerLayer);
            tc::mbar_arrive_expect_tx(&full[s], kChunkBytes);
            tc::bulk_g2s(ring + (size_t)s * kChunkBytes, a.bf + (size_t)lc * kChunkBytes,
                         kChunkBytes, &full[s]);
            ++next_load;
        }
    };
    if (tid == 0) load_more();

    // MMAs of `nchunks` consecutive chunks, chunk i into TMEM column col + i*col_step
    // (accumulating over chunks when col_step == 0), then one commit; all wait.
    auto run_chunks = [&](const unsigned char *A, int nchunks, uint32_t col, uint32_t col_step,
                          bool accumulate_first) {
        if (tid == 0) {
            bool ok = s_err == 0;
            for (int i = 0; i < nchunks && ok; ++i) {
                const int s = (int)(next_use % kStages);
                ok = tc::mbar_wait(&full[s], fphase[s]);
                if (!ok) break;
                fphase[s] ^= 1u;
                tc::tc_fence_after();
                const uint32_t sa = tc::smem_u32(A), sb = tc::smem_u32(ring + (size_t)s * kChunkBytes);
                const uint32_t idesc = tc::idesc_bf16(kRows, 128);
                for (int k = 0; k < 8; ++k)
                    tc::mma_bf16(tmem + col + i * col_step, tc::smem_desc(sa + 256 * k, 128, KG * 128),
                                 tc::smem_desc(sb + 256 * k, 128, KG * 128), idesc,
                                 (k > 0 || (i > 0 && col_step == 0) || accumulate_first) ? 1u : 0u);
                ++next_use;
            }
            if (!ok) {
                atomicExch(a.err, 1);
                s_err = 1;
            }
            tc::mma_commit(&mbar);
        }
        __syncwarp();
        if (!tc::mbar_wait(&mbar, mphase)) {
            if (lane == 0) atomicExch(a.err, 2);
            s_err = 1;
        }
        mphase ^= 1u;
        __syncthreads();
        tc::tc_fence_after();
        if (tid == 0 && !s_err) load_more();  // stages of completed MMAs are free
    };

    float h[Q32];
    auto layernorm_to = [&](const float *gam, const float *bet) {
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int j = 0; j < Q32; ++j) {
            s1 += h[j];
            s2 += h[j] * h[j];
        }
        xln[(qr * kRows + r) * 2] = s1;
        xln[(qr * kRows + r) * 2 + 1] = s2;
        __syncthreads();
        float t1 = 0.f, t2 = 0.f;
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
            t1 += xln[(q4 * kRows + r) * 2];
            t2 += xln[(q4 * kRows + r) * 2 + 1];
        }
        const float mean = t1 * (1.0f / D);
        const float var = fmaxf(t2 * (1.0f / D) - mean * mean, 0.f);
        const float rs = 1.0f / sqrtf(var + 1e-5f);
#pragma unroll
        for (int c = 0; c < Q32 / 8; ++c) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int d = Q32 * qr + 8 * c + j;
                v[j] = (h[8 * c + j] - mean) * rs * __ldg(gam + d) + __ldg(bet + d);
            }
            store8(Abuf, r, Q32 * qr + 8 * c, KG, v);
        }
        tc::fence_async_smem();
        tc::tc_fence_before();
        __syncthreads();
    };

    float lq = 0.f;
    int tok = 0;
    const float qscale = 0.25f;

    for (int t = 0; t < a.N && !s_err; ++t) {
        {
            const float *pos = a.w + a.o.pos + (size_t)t * (D - a.dt);
#pragma unroll
            for (int j = 0; j < Q32; ++j) {
                const int d = Q32 * qr + j;
                h[j] = d < a.dt ? __ldg(a.w + a.o.tok + tok * a.dt + d) : __ldg(pos + d - a.dt);
            }
        }
        int n_sink, band_lo;
        visible_ranges(a.mask, a.W, a.S, t, n_sink, band_lo);
        const int slot_t = bslot(g, a.S, a.W, t);
        const int nk_all = n_sink + band_count(t, band_lo) - 1;  // keys < t
        const int nk = active ? nk_all : 0;
        // ring offsets (16-byte units) of this step's visible keys, the same for
        // every row, head and layer (the first LayerNorm's barrier orders them)
        for (int i = tid; i < nk_all; i += blockDim.x)
            koff[i] = (uint32_t)bslot(g, a.S, a.W, i < n_sink ? i : band_lo + (i - n_sink)) *
                      (uint32_t)(slot_bytes / 16);
        for (int l = 0; l < a.L; ++l) {
            const LayerOff &o = a.o.L[l];
            layernorm_to(a.w + o.ln1g, a.w + o.ln1b);
            run_chunks(Abuf, 3, QKV_COL, 128, false);
            if (s_err) break;
            unsigned char *kvl = kvt + (size_t)l * layer_bytes;
            {
                const float *bq = a.wt + a.p.bqkv[l];
                // append k_t, v_t (this thread's 32 dims) to the ring
                float kk[Q32];
                tc::tmem_ld32(tmem + tq + QKV_COL + D + Q32 * qr, kk);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < Q32; ++j) kk[j] = round_bf(kk[j] + __ldg(bq + D + Q32 * qr + j));
                uint4 *dk = reinterpret_cast<uint4 *>(kvl + (size_t)slot_t * slot_bytes);
                if (active && !is_mirror)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        uint4 x;
                        x.x = pack_bf2(kk[8 * c], kk[8 * c + 1]);
                        x.y = pack_bf2(kk[8 * c + 2], kk[8 * c + 3]);
                        x.z = pack_bf2(kk[8 * c + 4], kk[8 * c + 5]);
                        x.w = pack_bf2(kk[8 * c + 6], kk[8 * c + 7]);
                        dk[(4 * qr + c) * kRows + r] = x;
                    }
                tc::tmem_ld32(tmem + tq + QKV_COL + 2 * D + Q32 * qr, kk);  // now v_t
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < Q32; ++j) kk[j] = round_bf(kk[j] + __ldg(bq + 2 * D + Q32 * qr + j));
                uint4 *dv = dk + (D / 8) * kRows;
                if (active && !is_mirror)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        uint4 x;
                        x.x = pack_bf2(kk[8 * c], kk[8 * c + 1]);
                        x.y = pack_bf2(kk[8 * c + 2], kk[8 * c + 3]);
                        x.z = pack_bf2(kk[8 * c + 4], kk[8 * c + 5]);
                        x.w = pack_bf2(kk[8 * c + 6], kk[8 * c + 7]);
                        dv[(4 * qr + c) * kRows + r] = x;
                    }
                // attention, one head at a time; the current key comes from registers
#pragma unroll 1
                for (int p = 0; p < 2; ++p) {
                    const int hh = 2 * qr + p;
                    float q[DH], acc[DH];
                    __syncwarp();
                    tc::tmem_ld32(tmem + tq + QKV_COL + Q32 * qr, kk);  // q of both heads
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < DH; ++j)
                        q[j] = (kk[DH * p + j] + __ldg(bq + DH * hh + j)) * qscale;
                    // the current key and value, rounded to BF16 as stored
                    tc::tmem_ld32(tmem + tq + QKV_COL + D + Q32 * qr, kk);
                    tc::tmem_wait_ld();
                    float m0 = 0.f, l0 = 1.f;
#pragma unroll
                    for (int j = 0; j < DH; ++j)
                        m0 += q[j] * round_bf(kk[DH * p + j] + __ldg(bq + D + DH * hh + j));
                    tc::tmem_ld32(tmem + tq + QKV_COL + 2 * D + Q32 * qr, kk);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < DH; ++j)
                        acc[j] = round_bf(kk[DH * p + j] + __ldg(bq + 2 * D + DH * hh + j));
                    // The row's keys reduce as two halves, the current key (held
                    // above) with keys [0, half) and keys [half, nk) from the empty
                    // state, merged as (first, second).  In mirror mode the row's
                    // thread takes the first half and its mirror the second;
                    // otherwise one thread runs both and parks the first half's
                    // state.  The arithmetic is the same either way.
                    const int half = (nk + 1) >> 1;
                    const int i0 = mirror_mode && is_mirror ? half : 0;
                    const int i1 = mirror_mode && !is_mirror ? half : nk;
                    float sm = -INFINITY, sl = 0.f, sacc[DH];  // the parked first half
#pragma unroll
                    for (int j = 0; j < DH; ++j) sacc[j] = 0.f;
                    auto park = [&]() {
                        sm = m0;
                        sl = l0;
#pragma unroll
                        for (int j = 0; j < DH; ++j) {
                            sacc[j] = acc[j];
                            acc[j] = 0.f;
                        }
                        m0 = -INFINITY;
                        l0 = 0.f;
                    };
                    if (is_mirror) {  // the second half starts from the empty state
                        m0 = -INFINITY;
                        l0 = 0.f;
#pragma unroll
                        for (int j = 0; j < DH; ++j) acc[j] = 0.f;
                    }
                    // keys < t staged through shared memory by cp.async, three keys
                    // in flight per thread: stages are the A and A2 tiles (idle
                    // during attention) and the spare tile; per thread, K pieces at
                    // +0, +8 KB and V pieces at +16 KB, +24 KB of a stage.
                    const uint4 *kb = reinterpret_cast<const uint4 *>(kvl) + (2 * hh) * kRows + rr;
                    auto stage = [&](int s) {
                        return (s == 0 ? Abuf : (s == 1 ? A2buf : kvspare)) + tid * 16;
                    };
                    auto fetch = [&](int i, int s) {
                        const uint4 *pp = kb + koff[i];
                        unsigned char *dst = stage(s);
                        tc::cp_async16(dst, pp);
                        tc::cp_async16(dst + 8192, pp + kRows);
                        tc::cp_async16(dst + 16384, pp + (D / 8) * kRows);
                        tc::cp_async16(dst + 24576, pp + (D / 8) * kRows + kRows);
                        tc::cp_async_commit();
                    };
                    for (int i = i0; i < i1 && i < i0 + 3; ++i) fetch(i, i - i0);
                    for (int i = i0; i < i1; ++i) {
                        if (!mirror_mode && i == half) park();
                        if (i + 2 < i1) tc::cp_async_wait<2>();
                        else if (i + 1 < i1) tc::cp_async_wait<1>();
                        else tc::cp_async_wait<0>();
                        const int si = (i - i0) % 3;
                        const unsigned char *src = stage(si);
                        uint4 ck[2], cv[2];
                        ck[0] = *reinterpret_cast<const uint4 *>(src);
                        ck[1] = *reinterpret_cast<const uint4 *>(src + 8192);
                        cv[0] = *reinterpret_cast<const uint4 *>(src + 16384);
                        cv[1] = *reinterpret_cast<const uint4 *>(src + 24576);
                        float s = 0.f;
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            const uint32_t wk[4] = {ck[c].x, ck[c].y, ck[c].z, ck[c].w};
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                s += q[8 * c + 2 * j] * bf_lo(wk[j]) + q[8 * c + 2 * j + 1] * bf_hi(wk[j]);
                        }
                        const float n0 = fmaxf(m0, s);
                        const float c0 = __expf(m0 - n0), p0 = __expf(s - n0);
                        m0 = n0;
                        l0 = l0 * c0 + p0;
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            const uint32_t wv[4] = {cv[c].x, cv[c].y, cv[c].z, cv[c].w};
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                acc[8 * c + 2 * j] = acc[8 * c + 2 * j] * c0 + p0 * bf_lo(wv[j]);
                                acc[8 * c + 2 * j + 1] = acc[8 * c + 2 * j + 1] * c0 + p0 * bf_hi(wv[j]);
                            }
                        }
                        // the stage is refilled only after its data has been consumed
                        if (i + 3 < i1) fetch(i + 3, si);
                    }
                    if (!mirror_mode && half >= nk) park();  // nk <= 1: the second half is empty
                    if (mirror_mode) {
                        // exchange partial states through this thread's own stage
                        // slots (its copies are complete): the row's thread parks
                        // its half and takes the mirror's as the second; the
                        // mirror parks the row's half and keeps its own
                        float *mine = reinterpret_cast<float *>(Abuf + tid * 16);
#pragma unroll
                        for (int c = 0; c < DH / 4; ++c)
                            *reinterpret_cast<float4 *>(mine + c * 2048) =
                                make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
                        *reinterpret_cast<float4 *>(A2buf + tid * 16) = make_float4(m0, l0, 0.f, 0.f);
                        __syncthreads();
                        const int ptid = tid ^ 64;
                        const float *other = reinterpret_cast<const float *>(Abuf + ptid * 16);
                        const float4 ox = *reinterpret_cast<const float4 *>(A2buf + ptid * 16);
                        if (!is_mirror) park();
#pragma unroll
                        for (int c = 0; c < DH / 4; ++c) {
                            const float4 v = *reinterpret_cast<const float4 *>(other + c * 2048);
                            const float ov[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                            for (int kq = 0; kq < 4; ++kq) {
                                if (is_mirror) sacc[4 * c + kq] = ov[kq];
                                else acc[4 * c + kq] = ov[kq];
                            }
                        }
                        if (is_mirror) {
                            sm = ox.x;
                            sl = ox.y;
                        } else {
                            m0 = ox.x;
                            l0 = ox.y;
                        }
                        __syncthreads();  // the slots are free again for the next head
                    }
                    {   // merge: parked = first half, current = second half
                        const float mm = fmaxf(sm, m0);
                        const float ca = sm == -INFINITY ? 0.f : __expf(sm - mm);
                        const float cb = m0 == -INFINITY ? 0.f : __expf(m0 - mm);
#pragma unroll
                        for (int j = 0; j < DH; ++j) acc[j] = __fmaf_rn(sacc[j], ca, __fmul_rn(acc[j], cb));
                        l0 = __fmaf_rn(sl, ca, __fmul_rn(l0, cb));
                    }
                    const float inv = 1.0f / l0;
#pragma unroll
                    for (int j = 0; j < DH; ++j) h[DH * p + j] += acc[j] * inv;
                }
            }
            layernorm_to(a.w + o.ln2g, a.w + o.ln2b);
            const float *b1 = a.wt + a.p.b1[l];
            for (int j = 0; j < 4 && !s_err; ++j) {
                run_chunks(Abuf, 1, FF1_COL, 0, false);
                if (s_err) break;
                {
                    float v[32];
                    tc::tmem_ld32(tmem + tq + FF1_COL + Q32 * qr, v);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int g8 = 0; g8 < 4; ++g8) {
                        float x[8];
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj)
                            x[jj] = gelu_as(v[8 * g8 + jj] + __ldg(b1 + 128 * j + Q32 * qr + 8 * g8 + jj));
                        store8(A2buf, r, Q32 * qr + 8 * g8, KG, x);
                    }
                    tc::fence_async_smem();
                    tc::tc_fence_before();
                    __syncthreads();
                }
                run_chunks(A2buf, 1, FF2_COL, 0, j > 0);
            }
            if (s_err) break;
            {
                float v[32];
                tc::tmem_ld32(tmem + tq + FF2_COL + Q32 * qr, v);
                tc::tmem_wait_ld();
                const float *b2 = a.wt + a.p.b2[l];
#pragma unroll
                for (int j = 0; j < Q32; ++j) h[j] += v[j] + __ldg(b2 + Q32 * qr + j);
            }
        }
        if (s_err) break;
        {
            float s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int j = 0; j < Q32; ++j) {
                s1 += h[j];
                s2 += h[j] * h[j];
            }
            xln[(qr * kRows + r) * 2] = s1;
            xln[(qr * kRows + r) * 2 + 1] = s2;
            __syncthreads();
            float t1 = 0.f, t2 = 0.f;
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
                t1 += xln[(q4 * kRows + r) * 2];
                t2 += xln[(q4 * kRows + r) * 2 + 1];
            }
            const float mean = t1 * (1.0f / D);
            const float var = fmaxf(t2 * (1.0f / D) - mean * mean, 0.f);
            const float rs = 1.0f / sqrtf(var + 1e-5f);
            if (a.P > 1) {
                // the A and A2 tiles (64 KB, contiguous) are idle from the last
                // FFN2 of a step to the next step's first LayerNorm
                float y[Q32];
#pragma unroll
                for (int j = 0; j < Q32; ++j) {
                    const int d = Q32 * qr + j;
                    y[j] = (h[j] - mean) * rs * __ldg(a.w + a.o.lnfg + d) + __ldg(a.w + a.o.lnfb + d);
                }
                patched_head<Q32>(a, a.w, y, D, r, qr, reinterpret_cast<float *>(Abuf), b, t,
                                  active && !is_mirror, nfw, lq, tok);
                continue;
            }
            float z0 = 0.f, z1 = 0.f;
#pragma unroll
            for (int j = 0; j < Q32; ++j) {
                const int d = Q32 * qr + j;
                const float y = (h[j] - mean) * rs * __ldg(a.w + a.o.lnfg + d) + __ldg(a.w + a.o.lnfb + d);
                z0 += y * __ldg(a.w + a.o.Wh + d);
                z1 += y * __ldg(a.w + a.o.Wh + D + d);
            }
            xhd[(qr * kRows + r) * 2] = z0;
            xhd[(qr * kRows + r) * 2 + 1] = z1;
            __syncthreads();
            if (qr == 0) {
                z0 = __ldg(a.w + a.o.bh);
                z1 = __ldg(a.w + a.o.bh + 1);
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    z0 += xhd[(q4 * kRows + r) * 2];
                    z1 += xhd[(q4 * kRows + r) * 2 + 1];
                }
                const float ell = z1 - z0;
                const float p = 1.0f / (1.0f + expf(-ell));
                const float u = philox_uniform(a.seed, (uint32_t)b, (uint32_t)t, a.sid, 0u);
                const int sp = u < p ? 1 : -1;
                lq += log_sigmoid_f((float)sp * ell);
                tok = (sp + 1) >> 1;
                if (active && !is_mirror) {
                    a.spins[(size_t)b * a.N + t] = (int8_t)sp;
                    if (a.flags && fabsf(p - u) < a.band)
                        a.flags[(size_t)b * nfw + (t >> 5)] |= 1u << (t & 31);
                    if (!isfinite(ell)) atomicOr(a.err, 4);
                }
            }
        }
    }
    if (qr == 0 && active && !is_mirror) a.logq[b] = lq;
    // drain the bulk copies still in flight before the CTA exits
    if (tid == 0)
        while (next_use < next_load) {
            const int s = (int)(next_use % kStages);
            if (!tc::mbar_wait(&full[s], fphase[s])) {
                atomicExch(a.err, 3);
                break;
            }
            fphase[s] ^= 1u;
            ++next_use;
        }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// d = 256 variant (8 heads of 32, d_ff = 1024).  A row's 256-dim FP32 residual
// stream does not fit in registers, so it lives in TMEM columns [256, 512);
// the accumulators use columns [0, 256).  Per layer:
//   LN1 (h read from TMEM) -> A tile -> MMA k (N = 256) -> ring; MMA v -> ring;
//   MMA q -> TMEM -> attention of the thread's two heads (keys, including
//   t itself, read back from the ring) -> h += o (TMEM ld/st) -> LN2 ->
//   4 x [MMA FFN1 slice -> GELU -> A2 -> MMA FFN2 K-slice accumulated straight
//   into the residual columns] -> h += b2.
// Weights stream as 44 chunks of 32 KB per layer ([256 out rows x 64 K]) through
// a two-stage ring.  Grouped models: each model's rows are split over
// ctas_per_model consecutive CTAs, which read that model's weights.
// ---------------------------------------------------------------------------
constexpr int kChunk256 = 256 * 64 * 2;
constexpr int kChunks256 = 44;
constexpr int kStages256 = 2;

// chunk c of a layer, element (r, k) of the [256 x 64] operand
__global__ void pack_chunks256_kernel(const float *__restrict__ Wqkv,
                                      const float *__restrict__ W1,
                                      const float *__restrict__ W2, __nv_bfloat16 *__restrict__ dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)kChunks256 * 256 * 64) return;
    const int c = (int)(i / (256 * 64)), r = (int)((i / 64) % 256), k = (int)(i % 64);
    float v;
    if (c < 4) v = Wqkv[(size_t)(256 + r) * 256 + 64 * c + k];            // k rows
    else if (c < 8) v = Wqkv[(size_t)(512 + r) * 256 + 64 * (c - 4) + k];  // v rows
    else if (c < 12) v = Wqkv[(size_t)r * 256 + 64 * (c - 8) + k];         // q rows
    else {
        const int f = c - 12, j = f / 8, w = f % 8;
        if (w < 4) v = W1[(size_t)(256 * j + r) * 256 + 64 * w + k];
        else v = W2[(size_t)r * 1024 + 256 * j + 64 * (w - 4) + k];
    }
    dst[(size_t)c * (kChunk256 / 2) + (tc::cm_offset(r, k, 8) >> 1)] = __float2bfloat16(v);
}

__global__ void __launch_bounds__(512, 1) decode_bf16_d256_kernel(const __grid_constant__ DecodeArgs a)
{
    constexpr int D = 256, DH = 32, KG = D / 8;
    constexpr uint32_t ACC = 0, HCOL = 256;
    constexpr uint32_t A_BYTES = kRows * D * 2;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Abuf = smem;
    unsigned char *A2buf = Abuf + A_BYTES;
    unsigned char *ring = A2buf + A_BYTES;
    float *xln = reinterpret_cast<float *>(ring + kStages256 * kChunk256);  // [4][128][2]
    float *xhd = xln + 4 * kRows * 2;                                        // [4][128][2]
    uint32_t *koff = reinterpret_cast<uint32_t *>(xhd + 4 * kRows * 2);     // [max_keys]
    __shared__ uint64_t full[kStages256], empty[kStages256], mbar;
    __shared__ uint32_t tslot;
    __shared__ int s_err;
    __shared__ int stok[kRows];  // token of each row drawn at the previous step

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = 32 * (warp & 3) + lane, qr = warp >> 2;
    // With at most 64 rows per CTA, rows 64..127 mirror rows 0..63 (same
    // inputs, so every phase computes identical copies in TMEM lanes
    // 64..127); a row and its mirror (thread tid ^ 64) split the attention's
    // keys and merge their partial softmax states, doubling the KV loads in
    // flight.  Only the row itself writes the KV cache, spins and log q.
    int64_t row0, mdl;
    int rows;  // rows of this CTA
    if (a.ctas_per_model > 0) {
        mdl = blockIdx.x / a.ctas_per_model;
        const int64_t j = blockIdx.x % a.ctas_per_model;
        const int64_t lo = j * a.rows_per_model / a.ctas_per_model;
        const int64_t hi = (j + 1) * a.rows_per_model / a.ctas_per_model;
        row0 = mdl * a.rows_per_model + lo;
        rows = (int)(hi - lo);
    } else {
        row0 = (int64_t)blockIdx.x * a.rows_per_cta;
        mdl = row0 / a.rows_per_model;
        rows = a.rows_per_cta;
    }
    const bool mirror_mode = rows <= 64;
    const int rr = mirror_mode ? (r & 63) : r;     // the sample row this thread serves
    const bool is_mirror = mirror_mode && r >= 64;
    const int64_t b = row0 + rr;
    const bool active = rr < rows && b < a.B;
    const float *w = a.w + mdl * a.stride_w;
    const float *wt = a.wt + mdl * a.stride_wt;
    const unsigned char *bf = a.bf + mdl * a.stride_bf;
    const Bf16Geom g = bgeom(a.mask, a.N, a.W, a.S);
    const size_t slot_bytes = (size_t)2 * D * kRows * 2;
    const size_t layer_bytes = slot_bytes * g.nslots;
    unsigned char *kvt = a.kv + (size_t)blockIdx.x * layer_bytes * a.L;
    const int nfw = (a.N + 31) >> 5;
    const uint32_t tq = (uint32_t)(32 * (warp & 3)) << 16;
    const int64_t total_chunks = (int64_t)a.N * a.L * kChunks256;

    if (tid == 0) {
        for (int s = 0; s < kStages256; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(&mbar, 1);
        tc::fence_mbar_init();
        s_err = 0;
    }
    if (tid < kRows) stok[tid] = 0;
    if (warp == 0) {
        tc::tmem_alloc(&tslot, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tslot;

    // Chunk stream.  Chunk c (the global count over steps and layers) sits in
    // stage c % kStages256; its full[] and empty[] phases have parity
    // (c / kStages256) & 1.  Two threads share the stream inside a product:
    // thread 0 issues the MMAs of each chunk as soon as it has landed and
    // commits them on empty[] without waiting; thread 32 (otherwise idle
    // there) refills a stage once the MMAs of its previous chunk completed.
    // Loads stop short of load_limit: after a layer's q product the ring stays
    // empty so that the attention can stage keys in it, and its loads go out
    // once the key loop is done.
    constexpr int kProducer = 32;
    int64_t use_ctr = 0;                       // chunks consumed by the products so far (every thread)
    int64_t next_load = 0, load_limit = INT64_MAX;  // thread kProducer
    uint32_t mphase = 0;
    auto parity = [](int64_t c) { return (uint32_t)((c / kStages256) & 1); };
    // thread kProducer: load chunks while they are below `upto`; false when a
    // bounded wait gave up (the error word is set)
    auto produce = [&](int64_t upto) {
        while (next_load < total_chunks && next_load < load_limit && next_load < upto) {
            const int s = (int)(next_load % kStages256);
            if (next_load >= kStages256 && !tc::mbar_wait(&empty[s], parity(next_load - kStages256))) {
                atomicExch(a.err, 4);
                s_err = 1;
                return;
            }
            const int64_t lc = next_load % ((int64_t)a.L * kChunks256);
            tc::mbar_arrive_expect_tx(&full[s], kChunk256);
            tc::bulk_g2s(ring + (size_t)s * kChunk256, bf + (size_t)lc * kChunk256, kChunk256, &full[s]);
            ++next_load;
        }
    };
    if (tid == kProducer) produce(kStages256);

    // MMAs of `nchunks` consecutive K chunks (64 wide) of A x chunk^T into TMEM
    // column col; accumulate onto existing contents when `onto` is set.
    auto run = [&](const unsigned char *A, int nchunks, uint32_t col, bool onto) {
        const int64_t first = use_ctr;
        use_ctr += nchunks;
        if (tid == 0) {
            bool ok = s_err == 0;
            const uint32_t idesc = tc::idesc_bf16(kRows, 256);
            for (int i = 0; i < nchunks && ok; ++i) {
                const int64_t c = first + i;
                const int s = (int)(c % kStages256);
                ok = tc::mbar_wait(&full[s], parity(c));
                if (!ok) break;
                tc::tc_fence_after();
                const uint32_t sa = tc::smem_u32(A) + (uint32_t)(8 * i) * 128;
                const uint32_t sb = tc::smem_u32(ring + (size_t)s * kChunk256);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    tc::mma_bf16(tmem + col, tc::smem_desc(sa + 256 * k, 128, KG * 128),
                                 tc::smem_desc(sb + 256 * k, 128, 8 * 128), idesc,
                                 (onto || i > 0 || k > 0) ? 1u : 0u);
                tc::mma_commit(&empty[s]);
            }
            if (!ok) {
                atomicExch(a.err, 1);
                s_err = 1;
            }
            tc::mma_commit(&mbar);
        } else if (tid == kProducer) {
            // keep the ring full through this product and into the next one
            produce(use_ctr + kStages256);
        }
        __syncwarp();
        if (!tc::mbar_wait(&mbar, mphase)) {
            if (lane == 0) atomicExch(a.err, 2);
            s_err = 1;
        }
        mphase ^= 1u;
        __syncthreads();
        tc::tc_fence_after();
    };

    // this thread's 64 columns of a 256-wide TMEM block at `col`
    auto ld64 = [&](uint32_t col, float (&v0)[32], float (&v1)[32]) {
        tc::tmem_ld32(tmem + tq + col + 64 * qr, v0);
        tc::tmem_ld32(tmem + tq + col + 64 * qr + 32, v1);
        tc::tmem_wait_ld();
    };

    // LayerNorm of h (TMEM) into the BF16 A tile; also returns nothing else
    auto layernorm_to = [&](const float *gam, const float *bet) {
        float v0[32], v1[32];
        ld64(HCOL, v0, v1);
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            s1 += v0[j] + v1[j];
            s2 += v0[j] * v0[j] + v1[j] * v1[j];
        }
        xln[(qr * kRows + r) * 2] = s1;
        xln[(qr * kRows + r) * 2 + 1] = s2;
        __syncthreads();
        float t1 = 0.f, t2 = 0.f;
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
            t1 += xln[(q4 * kRows + r) * 2];
            t2 += xln[(q4 * kRows + r) * 2 + 1];
        }
        const float mean = t1 * (1.0f / D);
        const float var = fmaxf(t2 * (1.0f / D) - mean * mean, 0.f);
        const float rs = 1.0f / sqrtf(var + 1e-5f);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float y[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int d = 64 * qr + 8 * c + j;
                const float x = c < 4 ? v0[8 * c + j] : v1[8 * (c - 4) + j];
                y[j] = (x - mean) * rs * __ldg(gam + d) + __ldg(bet + d);
            }
            store8(Abuf, r, 64 * qr + 8 * c, KG, y);
        }
        tc::fence_async_smem();
        tc::tc_fence_before();
        __syncthreads();
    };

    // append this thread's 64 columns of the accumulator (+bias) to the ring
    auto append = [&](unsigned char *slot, int part, const float *bias) {
        float v0[32], v1[32];
        ld64(ACC, v0, v1);
        if (!active || is_mirror) return;
        uint4 *dst = reinterpret_cast<uint4 *>(slot) + (size_t)part * (D / 8) * kRows;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float x[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                x[j] = (c < 4 ? v0[8 * c + j] : v1[8 * (c - 4) + j]) + __ldg(bias + 64 * qr + 8 * c + j);
            uint4 q;
            q.x = pack_bf2(x[0], x[1]);
            q.y = pack_bf2(x[2], x[3]);
            q.z = pack_bf2(x[4], x[5]);
            q.w = pack_bf2(x[6], x[7]);
            dst[(8 * qr + c) * kRows + r] = q;
        }
    };

    float lq = 0.f;
    const float qscale = 0.17677669529663687f;  // 1 / sqrt(32)

    for (int t = 0; t < a.N && !s_err; ++t) {
        {   // embedding into the residual columns
            const float *pos = w + a.o.pos + (size_t)t * (D - a.dt);
            float v[32];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int d = 64 * qr + 32 * c + j;
                    v[j] = d < a.dt ? __ldg(w + a.o.tok + stok[rr] * a.dt + d) : __ldg(pos + d - a.dt);
                }
                tc::tmem_st32(tmem + tq + HCOL + 64 * qr + 32 * c, v);
            }
            tc::tmem_wait_st();
        }
        int n_sink, band_lo;
        visible_ranges(a.mask, a.W, a.S, t, n_sink, band_lo);
        const int slot_t = bslot(g, a.S, a.W, t);
        const int nk_all = n_sink + band_count(t, band_lo);  // keys <= t
        const int nk = active ? nk_all : 0;
        for (int i = tid; i < nk_all; i += blockDim.x)
            koff[i] = (uint32_t)bslot(g, a.S, a.W, i < n_sink ? i : band_lo + (i - n_sink)) *
                      (uint32_t)(slot_bytes / 16);
        for (int l = 0; l < a.L && !s_err; ++l) {
            const LayerOff &o = a.o.L[l];
            const float *bq = wt + a.p.bqkv[l];
            unsigned char *kvl = kvt + (size_t)l * layer_bytes;
            unsigned char *slot = kvl + (size_t)slot_t * slot_bytes;
            layernorm_to(w + o.ln1g, w + o.ln1b);
            run(Abuf, 4, ACC, false);  // k_t
            if (s_err) break;
            append(slot, 0, bq + D);
            tc::tc_fence_before();
            __syncthreads();  // every thread has drained the accumulator
            run(Abuf, 4, ACC, false);  // v_t
            if (s_err) break;
            append(slot, 1, bq + 2 * D);
            tc::tc_fence_before();
            __syncthreads();
            if (tid == kProducer) load_limit = ((int64_t)t * a.L + l) * kChunks256 + 12;
            run(Abuf, 4, ACC, false);  // q_t stays in TMEM
            if (tid == kProducer) load_limit = INT64_MAX;
            if (s_err) break;
            // attention: heads 2 qr and 2 qr + 1, keys 0..t from the ring
            // (key t of row rr was written before the barriers of the q run)
#pragma unroll 1
            for (int p = 0; p < 2; ++p) {
                const int hh = 2 * qr + p;
                float q[DH], acc[DH];
                __syncwarp();
                tc::tmem_ld32(tmem + tq + ACC + DH * hh, q);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < DH; ++j) {
                    q[j] = (q[j] + __ldg(bq + DH * hh + j)) * qscale;
                    acc[j] = 0.f;
                }
                float m0 = -INFINITY, l0 = 0.f;
                // keys 0..t staged through shared memory by cp.async, three keys
                // in flight per thread: the stages are the A and A2 tiles and the
                // weight ring (all idle during attention); per thread, K pieces
                // at +0..+24 KB and V pieces at +32..+56 KB of a stage, 8 KB
                // apart (conflict-free).
                const uint4 *kb = reinterpret_cast<const uint4 *>(kvl) + (4 * hh) * kRows + rr;
                // Every row reduces its keys as two halves, [0, half) and
                // [half, nk), each an online softmax from the empty state,
                // merged as (first half, second half).  In mirror mode the
                // row's thread takes the first half and its mirror the second;
                // otherwise one thread runs both and parks the first half's
                // state.  The arithmetic is the same either way, so a row's
                // results do not depend on how many rows share its CTA.
                const int half = (nk + 1) >> 1;
                const int i0 = !mirror_mode ? 0 : (is_mirror ? half : 0);
                const int i1 = !mirror_mode ? nk : (is_mirror ? nk : half);
                float sm = -INFINITY, sl = 0.f, sacc[DH];  // the parked first half
#pragma unroll
                for (int j = 0; j < DH; ++j) sacc[j] = 0.f;
                auto park = [&]() {
                    sm = m0;
                    sl = l0;
#pragma unroll
                    for (int j = 0; j < DH; ++j) {
                        sacc[j] = acc[j];
                        acc[j] = 0.f;
                    }
                    m0 = -INFINITY;
                    l0 = 0.f;
                };
                auto stage = [&](int s) { return s == 0 ? Abuf : (s == 1 ? A2buf : ring); };
                auto fetch = [&](int i, int s) {
                    const uint4 *pp = kb + koff[i];
                    unsigned char *dst = stage(s) + tid * 16;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        tc::cp_async16(dst + c * 8192, pp + c * kRows);
                        tc::cp_async16(dst + 32768 + c * 8192, pp + (D / 8) * kRows + c * kRows);
                    }
                    tc::cp_async_commit();
                };
                for (int i = i0; i < i1 && i < i0 + 3; ++i) fetch(i, i - i0);
                for (int i = i0; i < i1; ++i) {
                    if (!mirror_mode && i == half) park();
                    if (i + 2 < i1) tc::cp_async_wait<2>();
                    else if (i + 1 < i1) tc::cp_async_wait<1>();
                    else tc::cp_async_wait<0>();
                    const unsigned char *src = stage((i - i0) % 3) + tid * 16;
                    float s = 0.f;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint4 ck = *reinterpret_cast<const uint4 *>(src + c * 8192);
                        const uint32_t wk[4] = {ck.x, ck.y, ck.z, ck.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            s += q[8 * c + 2 * j] * bf_lo(wk[j]) + q[8 * c + 2 * j + 1] * bf_hi(wk[j]);
                    }
                    const float n0 = fmaxf(m0, s);
                    const float c0 = __expf(m0 - n0), p0 = __expf(s - n0);
                    m0 = n0;
                    l0 = l0 * c0 + p0;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint4 cv = *reinterpret_cast<const uint4 *>(src + 32768 + c * 8192);
                        const uint32_t wv[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            acc[8 * c + 2 * j] = acc[8 * c + 2 * j] * c0 + p0 * bf_lo(wv[j]);
                            acc[8 * c + 2 * j + 1] = acc[8 * c + 2 * j + 1] * c0 + p0 * bf_hi(wv[j]);
                        }
                    }
                    // the stage is refilled only after its data has been consumed
                    if (i + 3 < i1) fetch(i + 3, (i - i0) % 3);
                }
                if (!mirror_mode && half >= nk) park();  // nk <= 1: the second half is empty
                if (mirror_mode) {
                    // exchange partial states through this thread's own stage
                    // slots (its copies are complete); the row's thread parks
                    // the mirror's half, the mirror parks the row's half and
                    // keeps its own as the second
                    float *mine = reinterpret_cast<float *>(Abuf + tid * 16);
                    float *minex = reinterpret_cast<float *>(A2buf + tid * 16);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        *reinterpret_cast<float4 *>(mine + c * 2048) =
                            make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
                    *reinterpret_cast<float4 *>(minex) = make_float4(m0, l0, 0.f, 0.f);
                    __syncthreads();
                    const int ptid = tid ^ 64;
                    const float *other = reinterpret_cast<const float *>(Abuf + ptid * 16);
                    const float4 ox = *reinterpret_cast<const float4 *>(A2buf + ptid * 16);
                    if (!is_mirror) park();  // own half -> parked, partner's -> current
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float4 v = *reinterpret_cast<const float4 *>(other + c * 2048);
                        const float ov[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (is_mirror) sacc[4 * c + k] = ov[k];
                            else acc[4 * c + k] = ov[k];
                        }
                    }
                    if (is_mirror) {
                        sm = ox.x;
                        sl = ox.y;
                    } else {
                        m0 = ox.x;
                        l0 = ox.y;
                    }
                    __syncthreads();  // the slots are free again for the next head
                }
                {   // merge: parked = first half, current = second half
                    const float mm = fmaxf(sm, m0);
                    const float ca = sm == -INFINITY ? 0.f : __expf(sm - mm);
                    const float cb = m0 == -INFINITY ? 0.f : __expf(m0 - mm);
#pragma unroll
                    for (int j = 0; j < DH; ++j) acc[j] = __fmaf_rn(sacc[j], ca, __fmul_rn(acc[j], cb));
                    l0 = __fmaf_rn(sl, ca, __fmul_rn(l0, cb));
                }
                __syncwarp();
                float hv[32];
                tc::tmem_ld32(tmem + tq + HCOL + DH * hh, hv);
                tc::tmem_wait_ld();
                const float inv = active ? 1.0f / l0 : 0.f;
#pragma unroll
                for (int j = 0; j < DH; ++j) hv[j] += acc[j] * inv;
                tc::tmem_st32(tmem + tq + HCOL + DH * hh, hv);
                tc::tmem_wait_st();
            }
            // the ring's key pieces are consumed: order these generic-proxy
            // accesses before the bulk copies that refill it with weights
            tc::fence_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            tc::tc_fence_after();
            if (tid == kProducer) produce(use_ctr + kStages256);
            layernorm_to(w + o.ln2g, w + o.ln2b);
            const float *b1 = wt + a.p.b1[l];
            for (int j = 0; j < 4 && !s_err; ++j) {
                run(Abuf, 4, ACC, false);  // FFN1 slice j
                if (s_err) break;
                {
                    float v0[32], v1[32];
                    ld64(ACC, v0, v1);
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        float x[8];
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            const float z = c < 4 ? v0[8 * c + jj] : v1[8 * (c - 4) + jj];
                            x[jj] = gelu_as(z + __ldg(b1 + 256 * j + 64 * qr + 8 * c + jj));
                        }
                        store8(A2buf, r, 64 * qr + 8 * c, KG, x);
                    }
                    tc::fence_async_smem();
                    tc::tc_fence_before();
                    __syncthreads();
                }
                run(A2buf, 4, HCOL, true);  // FFN2 K-slice j, onto the residual
            }
            if (s_err) break;
            {   // h += b2
                float v0[32], v1[32];
                ld64(HCOL, v0, v1);
                const float *b2 = wt + a.p.b2[l];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    v0[j] += __ldg(b2 + 64 * qr + j);
                    v1[j] += __ldg(b2 + 64 * qr + 32 + j);
                }
                tc::tmem_st32(tmem + tq + HCOL + 64 * qr, v0);
                tc::tmem_st32(tmem + tq + HCOL + 64 * qr + 32, v1);
                tc::tmem_wait_st();
                tc::tc_fence_before();
                __syncthreads();
                tc::tc_fence_after();
            }
        }
        if (s_err) break;
        {   // output head and the draw
            float v0[32], v1[32];
            ld64(HCOL, v0, v1);
            float s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                s1 += v0[j] + v1[j];
                s2 += v0[j] * v0[j] + v1[j] * v1[j];
            }
            xln[(qr * kRows + r) * 2] = s1;
            xln[(qr * kRows + r) * 2 + 1] = s2;
            __syncthreads();
            float t1 = 0.f, t2 = 0.f;
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
                t1 += xln[(q4 * kRows + r) * 2];
                t2 += xln[(q4 * kRows + r) * 2 + 1];
            }
            const float mean = t1 * (1.0f / D);
            const float var = fmaxf(t2 * (1.0f / D) - mean * mean, 0.f);
            const float rs = 1.0f / sqrtf(var + 1e-5f);
            if (a.P > 1) {
                // the A and A2 tiles are idle from the last FFN2 of a step to
                // the next step's first LayerNorm
                float y[64];
#pragma unroll
                for (int j = 0; j < 64; ++j) {
                    const int d = 64 * qr + j;
                    const float x = j < 32 ? v0[j] : v1[j - 32];
                    y[j] = (x - mean) * rs * __ldg(w + a.o.lnfg + d) + __ldg(w + a.o.lnfb + d);
                }
                int tk = 0;
                patched_head<64>(a, w, y, D, r, qr, reinterpret_cast<float *>(Abuf), b, t,
                                 active && !is_mirror, nfw, lq, tk);
                if (qr == 0) stok[r] = tk;
                __syncthreads();  // stok is read by every thread of the row
                continue;
            }
            float z0 = 0.f, z1 = 0.f;
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                const int d = 64 * qr + j;
                const float x = j < 32 ? v0[j] : v1[j - 32];
                const float y = (x - mean) * rs * __ldg(w + a.o.lnfg + d) + __ldg(w + a.o.lnfb + d);
                z0 += y * __ldg(w + a.o.Wh + d);
                z1 += y * __ldg(w + a.o.Wh + D + d);
            }
            xhd[(qr * kRows + r) * 2] = z0;
            xhd[(qr * kRows + r) * 2 + 1] = z1;
            __syncthreads();
            if (qr == 0) {
                z0 = __ldg(w + a.o.bh);
                z1 = __ldg(w + a.o.bh + 1);
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    z0 += xhd[(q4 * kRows + r) * 2];
                    z1 += xhd[(q4 * kRows + r) * 2 + 1];
                }
                const float ell = z1 - z0;
                const float p = 1.0f / (1.0f + expf(-ell));
                const float u = philox_uniform(a.seed, (uint32_t)b, (uint32_t)t, a.sid, 0u);
                const int sp = u < p ? 1 : -1;
                lq += log_sigmoid_f((float)sp * ell);
                stok[r] = (sp + 1) >> 1;
                if (active && !is_mirror) {
                    a.spins[(size_t)b * a.N + t] = (int8_t)sp;
                    if (a.flags && fabsf(p - u) < a.band)
                        a.flags[(size_t)b * nfw + (t >> 5)] |= 1u << (t & 31);
                    if (!isfinite(ell)) atomicOr(a.err, 4);
                }
            }
            __syncthreads();  // stok is read by every thread of the row
        }
    }
    if (qr == 0 && active && !is_mirror) a.logq[b] = lq;
    // no bulk copy may be in flight when the CTA exits: wait for the chunks
    // loaded ahead of the products that did not run
    if (tid == kProducer)
        for (int64_t c = use_ctr; c < next_load; ++c)
            if (!tc::mbar_wait(&full[c % kStages256], parity(c))) {
                atomicExch(a.err, 3);
                break;
            }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

}  // namespace

sg_status launch_pack_bf16(sg_model *m, cudaStream_t st)
{
    const sg_config &c = m->cfg;
    if (c.d == 256) {
        // 44 chunks of 32 KB per layer and model; models follow one another
        const size_t per_layer = (size_t)kChunks256 * kChunk256;
        SG_TRY(ensure_buffer(&m->bf, &m->bf_bytes, per_layer * c.n_layers * m->n_models));
        if (c.d_ff != 1024) return SG_OK;  // the d = 256 decode needs d_ff = 1024
        const int64_t n = (int64_t)kChunks256 * 256 * 64;
        for (int mi = 0; mi < m->n_models; ++mi) {
            const float *w = m->w + (size_t)mi * m->P1;
            for (int l = 0; l < c.n_layers; ++l) {
                const LayerOff &o = m->off.L[l];
                unsigned char *dst =
                    (unsigned char *)m->bf + per_layer * ((size_t)mi * c.n_layers + l);
                pack_chunks256_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ::sg::counted(st)>>>(
                    w + o.Wqkv, w + o.W1, w + o.W2, reinterpret_cast<__nv_bfloat16 *>(dst));
            }
        }
        return check_launch("pack bf16 chunks (d = 256)");
    }
    if (c.d == 128) {
        const size_t per_layer = (size_t)kChunksPerLayer * kChunkBytes;
        SG_TRY(ensure_buffer(&m->bf, &m->bf_bytes, per_layer * c.n_layers));
        if (c.d_ff != 512) return SG_OK;  // the d = 128 decode needs d_ff = 512
        const int64_t n = (int64_t)kChunksPerLayer * 128 * 128;
        for (int l = 0; l < c.n_layers; ++l) {
            const LayerOff &o = m->off.L[l];
            pack_chunks128_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ::sg::counted(st)>>>(
                m->w + o.Wqkv, m->w + o.W1, m->w + o.W2,
                reinterpret_cast<__nv_bfloat16 *>((unsigned char *)m->bf + per_layer * l));
        }
        return check_launch("pack bf16 chunks (d = 128)");
    }
    const size_t per_layer = ((size_t)3 * c.d * c.d + 2 * (size_t)c.d_ff * c.d) * 2;
    SG_TRY(ensure_buffer(&m->bf, &m->bf_bytes, per_layer * c.n_layers));
    for (int l = 0; l < c.n_layers; ++l) {
        __nv_bfloat16 *dst = reinterpret_cast<__nv_bfloat16 *>((unsigned char *)m->bf + per_layer * l);
        const LayerOff &o = m->off.L[l];
        const int64_t n1 = (int64_t)3 * c.d * c.d, n2 = (int64_t)c.d_ff * c.d;
        pack_cm_kernel<<<(unsigned)((n1 + 255) / 256), 256, 0, ::sg::counted(st)>>>(m->w + o.Wqkv, dst, 3 * c.d, c.d);
        pack_cm_kernel<<<(unsigned)((n2 + 255) / 256), 256, 0, ::sg::counted(st)>>>(m->w + o.W1, dst + n1, c.d_ff, c.d);
        pack_cm_kernel<<<(unsigned)((n2 + 255) / 256), 256, 0, ::sg::counted(st)>>>(m->w + o.W2, dst + n1 + n2, c.d, c.d_ff);
    }
    return check_launch("pack bf16 operands");
}

// Launch geometry of the BF16 decode for B samples: rows per CTA, CTAs per
// model (grouped models) and CTAs; returns the bytes of KV cache it needs.
size_t decode_bf16_layout(const sg_model *m, int64_t B, int *rows_out, int *cpm_out,
                          int64_t *tiles_out)
{
    const sg_config &c = m->seq;  // N = tokens
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t rows_per_model = B / m->n_models;
    // spread the batch over every SM: rows per CTA = ceil(B / SMs), at most 128
    int rows = (int)std::min<int64_t>(kRows, (B + sms - 1) / sms);
    rows = std::max(rows, 1);
    // grouped models: a CTA must not straddle two models; each model's rows go
    // to ctas_per_model CTAs (counts differing by at most one), as many as
    // keep all models within one wave over the SMs, at most 128 rows each
    int cpm = 0;
    if (m->n_models > 1) {
        cpm = (int)std::max<int64_t>((rows_per_model + kRows - 1) / kRows,
                                     std::max<int64_t>(1, sms / m->n_models));
        cpm = (int)std::min<int64_t>(cpm, rows_per_model);
        rows = (int)((rows_per_model + cpm - 1) / cpm);
    }
    const int64_t tiles = cpm > 0 ? (int64_t)cpm * m->n_models : (B + rows - 1) / rows;
    const Bf16Geom g = bgeom(c.mask_kind, c.N, c.W, c.S);
    if (rows_out) *rows_out = rows;
    if (cpm_out) *cpm_out = cpm;
    if (tiles_out) *tiles_out = tiles;
    return (size_t)tiles * c.n_layers * g.nslots * 2 * c.d * kRows * 2;
}

sg_status launch_decode_bf16(sg_model *m, int64_t B, uint64_t seed, uint32_t sid, float band,
                             int8_t *spins, float *logq, uint32_t *flags, cudaStream_t st)
{
    const sg_config &c = m->seq;  // N = tokens
    const int P = spins_per_token(c);
    const bool d64 = c.d == 64 && c.n_heads == 4 && c.d_ff == 256 && c.d_token <= 32;
    const bool d128 = c.d == 128 && c.n_heads == 8 && c.d_ff == 512 && c.d_token <= 32;
    const bool d256 = c.d == 256 && c.n_heads == 8 && c.d_ff == 1024 && c.d_token <= 64;
    if (!d64 && !d128 && !d256)
        return fail(SG_EUNSUPPORTED, "BF16 decode is built for (d, heads, d_ff) = (64, 4, 256), "
                                     "(128, 8, 512) and (256, 8, 1024)");
    if (m->n_models > 1 && !d256)
        return fail(SG_EUNSUPPORTED, "grouped models are served by the d = 256 decode");
    if (P > 1 && d64 && c.d_token > 16)
        return fail(SG_EUNSUPPORTED, "patched BF16 decode (d = 64) needs d_token <= 16; use SG_FP32");
    const int64_t rows_per_model = B / m->n_models;
    int rows = 0, cpm = 0;
    int64_t tiles = 0;
    const size_t kv_bytes = decode_bf16_layout(m, B, &rows, &cpm, &tiles);
    const Bf16Geom g = bgeom(c.mask_kind, c.N, c.W, c.S);
    SG_TRY(ensure_buffer(&m->kv, &m->kv_bytes, kv_bytes));
    SG_TRY(ensure_buffer(&m->err, &m->err_bytes, sizeof(int)));
    const size_t smem = (size_t)kRows * c.d * 2 + (size_t)kRows * c.d_ff * 2 +
                        (size_t)3 * c.d * c.d * 2 + 2 * (size_t)c.d_ff * c.d * 2 +
                        4 * kRows * 2 * sizeof(float);
    auto kern = decode_bf16_kernel<64, 256>;
    DecodeArgs a{};
    a.N = c.N;
    a.L = c.n_layers;
    a.dt = c.d_token;
    a.mask = c.mask_kind;
    a.W = c.W;
    a.S = c.S;
    a.dff = c.d_ff;
    a.rows_per_cta = rows;
    a.w = m->w;
    a.wt = m->wt;
    a.bf = (const unsigned char *)m->bf;
    a.bf_layer_bytes = ((size_t)3 * c.d * c.d + 2 * (size_t)c.d_ff * c.d) * 2;
    a.o = m->off;
    a.p = m->pack;
    a.B = B;
    a.seed = seed;
    a.sid = sid;
    a.band = band;
    a.spins = spins;
    a.logq = logq;
    a.flags = flags;
    a.kv = (unsigned char *)m->kv;
    a.err = (int *)m->err;
    a.rows_per_model = rows_per_model;
    a.ctas_per_model = cpm;
    a.stride_w = m->P1;
    a.stride_wt = m->pack.total;
    a.stride_bf = (size_t)kChunks256 * kChunk256 * c.n_layers;
    a.max_keys = g.nslots;
    a.P = P;
    a.K = 1 << P;
    a.Nspins = m->cfg.N;
    a.latD = c.lat_D;
    a.latL = c.lat_L;
    if (d256) {
        const size_t smem256 = 2 * (size_t)kRows * 256 * 2 + (size_t)kStages256 * kChunk256 +
                               8 * kRows * 2 * sizeof(float) + (size_t)g.nslots * sizeof(uint32_t);
        if (smem256 > 227 * 1024)
            return fail(SG_EUNSUPPORTED, "BF16 decode (d = 256) needs at most 6900 visible keys");
        SG_CUDA_TRY(cudaFuncSetAttribute(decode_bf16_d256_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem256));
        decode_bf16_d256_kernel<<<(unsigned)tiles, 512, smem256, ::sg::counted(st)>>>(a);
        return check_launch("decode_bf16_d256_kernel");
    }
    if (d128) {
        const size_t smem128 = 2 * (size_t)kRows * 128 * 2 + (size_t)kStages * kChunkBytes +
                               8 * kRows * 2 * sizeof(float) +
                               (size_t)((g.nslots * 4 + 1023) / 1024) * 1024 + 32768;
        if (smem128 > 227 * 1024)
            return fail(SG_EUNSUPPORTED, "BF16 decode (d = 128) needs at most 12000 visible keys");
        SG_CUDA_TRY(cudaFuncSetAttribute(decode_bf16_d128_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem128));
        decode_bf16_d128_kernel<<<(unsigned)tiles, 512, smem128, ::sg::counted(st)>>>(a);
        return check_launch("decode_bf16_d128_kernel");
    }
    if (c.d_token <= 16) {
        // four threads per sample (16 warps): the default for d = 64
        size_t smem4 = smem + 4 * kRows * 2 * sizeof(float) + (size_t)((c.N * 4 + 1023) / 1024) * 1024;
        if (smem4 > 227 * 1024)
            return fail(SG_EUNSUPPORTED, "BF16 decode (d = 64) needs N <= 11000");
        // a third KV stage (32 KB) when shared memory allows it
        a.kv_stages = smem4 + 32768 <= 227 * 1024 ? 3 : 2;
        if (a.kv_stages == 3) smem4 += 32768;
        auto k64 = P > 1 ? (a.kv_stages == 3 ? decode_bf16_d64_kernel<3, true> : decode_bf16_d64_kernel<2, true>)
                         : (a.kv_stages == 3 ? decode_bf16_d64_kernel<3, false> : decode_bf16_d64_kernel<2, false>);
        SG_CUDA_TRY(cudaFuncSetAttribute(k64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem4));
        k64<<<(unsigned)tiles, 512, smem4, ::sg::counted(st)>>>(a);
        return check_launch("decode_bf16_d64_kernel");
    }
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)tiles, kThreads, smem, ::sg::counted(st)>>>(a);
    return check_launch("decode_bf16_kernel");
}

}  // namespace sg
