// decode_f32.cu -- "FP32 plain" ancestral sampler (Algorithm 2 of the paper,
// KV-cache sampling) on CUDA cores, plus the packing of transposed FP32
// weights that the CUDA-core GEMMs read.
//
// One CTA owns a tile of MS samples for the whole sequence (t = 0..N-1, all
// layers) and never synchronises with other CTAs.  Per step and layer:
// LayerNorm -> QKV GEMM -> append (k_t, v_t) to the tile's KV ring in HBM ->
// attention of each (sample, head) over the visible keys of the band + sink
// mask -> residual -> LayerNorm -> FFN (GELU) -> residual.  After the last
// layer the output head gives l_t = z1 - z0 and the draw u < sigmoid(l_t) is
// taken in registers.
//
// KV layout per tile: [layer][slot][K|V][d/4][MS][4] floats, so that a warp
// (32 consecutive samples, one head) reads 512 contiguous bytes per float4.
// Slot of key k: dense or short sequence -> k; band + sink ring -> k for
// k < S, else S + (k - S) mod (W + 1).
#include <string>

#include "sg_internal.cuh"

namespace sg {

// ---------------------------------------------------------------------------
// Transposed weight copies: WT[k][o] = W[o][k].
// ---------------------------------------------------------------------------
__global__ void transpose_kernel(const float *__restrict__ W, float *__restrict__ WT, int n_out,
                                 int n_in)
{
    __shared__ float tile[32][33];
    const int o0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int o = o0 + i, k = k0 + threadIdx.x;
        if (o < n_out && k < n_in) tile[i][threadIdx.x] = W[(size_t)o * n_in + k];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int k = k0 + i, o = o0 + threadIdx.x;
        if (o < n_out && k < n_in) WT[(size_t)k * n_out + o] = tile[threadIdx.x][i];
    }
}

static void transpose(const float *W, float *WT, int n_out, int n_in, cudaStream_t st)
{
    dim3 grid((n_in + 31) / 32, (n_out + 31) / 32), block(32, 8);
    transpose_kernel<<<grid, block, 0, ::sg::counted(st)>>>(W, WT, n_out, n_in);
}

sg_status launch_pack_f32(sg_model *m, cudaStream_t st)
{
    const sg_config &c = m->cfg;
    const size_t f4 = sizeof(float);
    // grouped models: model mi's blob at w + mi * P1, its packed copies at wt + mi * pack.total
    for (int mi = 0; mi < m->n_models; ++mi) {
        const float *w = m->w + (size_t)mi * m->P1;
        float *wt = m->wt + (size_t)mi * m->pack.total;
        for (int l = 0; l < c.n_layers; ++l) {
            const LayerOff &o = m->off.L[l];
            transpose(w + o.Wqkv, wt + m->pack.WqkvT[l], 3 * c.d, c.d, st);
            transpose(w + o.W1, wt + m->pack.W1T[l], c.d_ff, c.d, st);
            transpose(w + o.W2, wt + m->pack.W2T[l], c.d, c.d_ff, st);
            SG_CUDA_TRY(cudaMemcpyAsync(wt + m->pack.Wqkv[l], w + o.Wqkv,
                                        (size_t)3 * c.d * c.d * f4, cudaMemcpyDeviceToDevice, st));
            SG_CUDA_TRY(cudaMemcpyAsync(wt + m->pack.W1[l], w + o.W1,
                                        (size_t)c.d_ff * c.d * f4, cudaMemcpyDeviceToDevice, st));
            SG_CUDA_TRY(cudaMemcpyAsync(wt + m->pack.W2[l], w + o.W2,
                                        (size_t)c.d * c.d_ff * f4, cudaMemcpyDeviceToDevice, st));
            SG_CUDA_TRY(cudaMemcpyAsync(wt + m->pack.bqkv[l], w + o.bqkv, (size_t)3 * c.d * f4,
                                        cudaMemcpyDeviceToDevice, st));
            SG_CUDA_TRY(cudaMemcpyAsync(wt + m->pack.b1[l], w + o.b1, (size_t)c.d_ff * f4,
                                        cudaMemcpyDeviceToDevice, st));
            SG_CUDA_TRY(cudaMemcpyAsync(wt + m->pack.b2[l], w + o.b2, (size_t)c.d * f4,
                                        cudaMemcpyDeviceToDevice, st));
        }
    }
    return check_launch("pack transposed weights");
}

// ---------------------------------------------------------------------------
// Building blocks over a tile held in shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// y = LayerNorm(x) * g + b over D features, one warp per row.
template <int D>
__device__ __forceinline__ void ln_row(const float *x, const float *__restrict__ g,
                                       const float *__restrict__ b, float *y, int lane)
{
    constexpr int PER = D / 32;
    float v[PER];
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        v[i] = x[lane + 32 * i];
        s += v[i];
    }
    const float mean = warp_sum(s) * (1.0f / D);
    float q = 0.f;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const float dv = v[i] - mean;
        q += dv * dv;
    }
    const float rs = 1.0f / sqrtf(warp_sum(q) * (1.0f / D) + 1e-5f);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int j = lane + 32 * i;
        y[j] = (v[i] - mean) * rs * __ldg(g + j) + __ldg(b + j);
    }
}

enum { EPI_STORE = 0, EPI_GELU = 1, EPI_ADD = 2 };

// C[r][o] (op)= bias[o] + sum_k A[r][k] * BT[k][o] for MS rows, NO columns.
// Each work item is RT rows x 4 columns; consecutive threads take consecutive
// column groups, so A reads are warp broadcasts and BT reads are coalesced.
template <int MS, int RT, int EPI>
__device__ __forceinline__ void tile_gemm(const float *A, int lda, const float *__restrict__ BT,
                                          int NO, int K, const float *__restrict__ bias, float *C,
                                          int ldc)
{
    const int ncg = NO >> 2;
    const int items = ncg * (MS / RT);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int cg = it % ncg, r0 = (it / ncg) * RT;
        const float4 bb = __ldg(reinterpret_cast<const float4 *>(bias) + cg);
        float acc[RT][4];
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            acc[r][0] = bb.x;
            acc[r][1] = bb.y;
            acc[r][2] = bb.z;
            acc[r][3] = bb.w;
        }
        const float4 *bp = reinterpret_cast<const float4 *>(BT) + cg;
#pragma unroll 2
        for (int k = 0; k < K; k += 4) {
            const float4 w0 = __ldg(bp + (size_t)(k + 0) * ncg);
            const float4 w1 = __ldg(bp + (size_t)(k + 1) * ncg);
            const float4 w2 = __ldg(bp + (size_t)(k + 2) * ncg);
            const float4 w3 = __ldg(bp + (size_t)(k + 3) * ncg);
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const float4 a = *reinterpret_cast<const float4 *>(A + (r0 + r) * lda + k);
                acc[r][0] += a.x * w0.x + a.y * w1.x + a.z * w2.x + a.w * w3.x;
                acc[r][1] += a.x * w0.y + a.y * w1.y + a.z * w2.y + a.w * w3.y;
                acc[r][2] += a.x * w0.z + a.y * w1.z + a.z * w2.z + a.w * w3.z;
                acc[r][3] += a.x * w0.w + a.y * w1.w + a.z * w2.w + a.w * w3.w;
            }
        }
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            float *cp = C + (r0 + r) * ldc + 4 * cg;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (EPI == EPI_STORE) cp[j] = acc[r][j];
                else if (EPI == EPI_GELU) cp[j] = gelu_f(acc[r][j]);
                else cp[j] += acc[r][j];
            }
        }
    }
}

// Rows per work item so that a 256-thread CTA has about one item per thread.
template <int MS, int EPI>
__device__ __forceinline__ void tile_gemm_auto(const float *A, int lda, const float *BT, int NO,
                                               int K, const float *bias, float *C, int ldc)
{
    const int ncg = NO >> 2;
    if (ncg * (MS / 8) >= 256) tile_gemm<MS, 8, EPI>(A, lda, BT, NO, K, bias, C, ldc);
    else if (ncg * (MS / 4) >= 256) tile_gemm<MS, 4, EPI>(A, lda, BT, NO, K, bias, C, ldc);
    else tile_gemm<MS, 2, EPI>(A, lda, BT, NO, K, bias, C, ldc);
}

struct RingGeom {
    int nslots;   // slots per (layer) in the cache
    bool ring;    // band + sink ring buffer in use
};

__host__ __device__ __forceinline__ RingGeom ring_geom(int mask, int N, int W, int S)
{
    RingGeom g;
    g.ring = mask == SG_MASK_BAND_SINK && (int64_t)S + W + 1 < N;
    g.nslots = g.ring ? S + W + 1 : N;
    return g;
}

__device__ __forceinline__ int slot_of(const RingGeom &g, int S, int W, int k)
{
    return (!g.ring || k < S) ? k : S + (k - S) % (W + 1);
}

// ---------------------------------------------------------------------------
// The decode kernel.  MS samples per CTA, NH = D/DH heads, MS * NH == 256.
// ---------------------------------------------------------------------------
template <int D, int DH>
__global__ void __launch_bounds__(256, 2)
decode_f32_kernel(const __grid_constant__ DevModel m, int64_t B, uint64_t seed, uint32_t sid, float band,
                  int8_t *__restrict__ spins, float *__restrict__ logq,
                  uint32_t *__restrict__ flags, float *__restrict__ kv)
{
    constexpr int NH = D / DH;
    constexpr int MS = 256 / NH;
    constexpr int RS = D + 4;  // row stride of h / a (floats); RS/4 odd
    int US = (3 * D > m.dff ? 3 * D : m.dff) + 4;
    if (US < m.K + 4) US = m.K + 4;

    extern __shared__ float4 smem4[];
    float *h = reinterpret_cast<float *>(smem4);
    float *a = h + MS * RS;
    float *u = a + MS * RS;
    float *lq = u + MS * US;
    int *tok = reinterpret_cast<int *>(lq + MS);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t b0 = (int64_t)blockIdx.x * MS;
    const RingGeom g = ring_geom(m.mask, m.N, m.W, m.S);
    const size_t slot_stride = (size_t)2 * D * MS;           // floats per slot
    const size_t layer_stride = slot_stride * g.nslots;
    float *kvt = kv + (size_t)blockIdx.x * layer_stride * m.L;
    const int nfw = (m.N + 31) >> 5;

    for (int s = tid; s < MS; s += blockDim.x) {
        lq[s] = 0.f;
        tok[s] = 0;  // start token
    }
    __syncthreads();

    const int as = tid % MS, ah = tid / MS;  // attention: (sample, head) of this thread
    const float qscale = 1.0f / sqrtf((float)DH);

    for (int t = 0; t < m.N; ++t) {
        // concatenated positional embedding x_t = [tok(s_{t-1}); pos(t)]
        const float *pos = m.w + m.o.pos + (size_t)t * (D - m.dt);
        for (int i = tid; i < MS * D; i += blockDim.x) {
            const int s = i / D, j = i % D;
            h[s * RS + j] = j < m.dt ? __ldg(m.w + m.o.tok + tok[s] * m.dt + j)
                                     : __ldg(pos + j - m.dt);
        }
        __syncthreads();
        int n_sink, band_lo;
        visible_ranges(m.mask, m.W, m.S, t, n_sink, band_lo);
        const int slot_t = slot_of(g, m.S, m.W, t);

        for (int l = 0; l < m.L; ++l) {
            const LayerOff &o = m.o.L[l];
            for (int r = warp; r < MS; r += 8)
                ln_row<D>(h + r * RS, m.w + o.ln1g, m.w + o.ln1b, a + r * RS, lane);
            __syncthreads();
            tile_gemm_auto<MS, EPI_STORE>(a, RS, m.wt + m.p.WqkvT[l], 3 * D, D, m.wt + m.p.bqkv[l],
                                          u, US);
            __syncthreads();
            // append (k_t, v_t) to the ring
            float *kvl = kvt + (size_t)l * layer_stride;
            float *dst = kvl + (size_t)slot_t * slot_stride;
            for (int i = tid; i < 2 * (D / 4) * MS; i += blockDim.x) {
                const int part = i / ((D / 4) * MS), rem = i % ((D / 4) * MS);
                const int c = rem / MS, s = rem % MS;
                const float4 v = *reinterpret_cast<const float4 *>(u + s * US + D + part * D + 4 * c);
                reinterpret_cast<float4 *>(dst + (size_t)part * D * MS)[c * MS + s] = v;
            }
            __syncthreads();
            // attention of (sample as, head ah) over keys [0, n_sink) U [band_lo, t]
            {
                float q[DH], acc[DH];
#pragma unroll
                for (int j = 0; j < DH; j += 4) {
                    const float4 v = *reinterpret_cast<const float4 *>(u + as * US + ah * DH + j);
                    q[j] = v.x * qscale;
                    q[j + 1] = v.y * qscale;
                    q[j + 2] = v.z * qscale;
                    q[j + 3] = v.w * qscale;
                    acc[j] = acc[j + 1] = acc[j + 2] = acc[j + 3] = 0.f;
                }
                float mx = -INFINITY, den = 0.f;
                const float4 *kb = reinterpret_cast<const float4 *>(kvl) + (ah * DH / 4) * MS + as;
                const int nk = n_sink + band_count(t, band_lo);
                for (int i = 0; i < nk; ++i) {
                    const int k = i < n_sink ? i : band_lo + (i - n_sink);
                    const float4 *kp = kb + (size_t)slot_of(g, m.S, m.W, k) * (slot_stride / 4);
                    float sc = 0.f;
#pragma unroll
                    for (int c = 0; c < DH / 4; ++c) {
                        const float4 kk = kp[c * MS];
                        sc += q[4 * c] * kk.x + q[4 * c + 1] * kk.y + q[4 * c + 2] * kk.z +
                              q[4 * c + 3] * kk.w;
                    }
                    const float mn = fmaxf(mx, sc);
                    const float corr = expf(mx - mn), p = expf(sc - mn);
                    mx = mn;
                    den = den * corr + p;
                    const float4 *vp = kp + (D / 4) * MS;
#pragma unroll
                    for (int c = 0; c < DH / 4; ++c) {
                        const float4 vv = vp[c * MS];
                        acc[4 * c] = acc[4 * c] * corr + p * vv.x;
                        acc[4 * c + 1] = acc[4 * c + 1] * corr + p * vv.y;
                        acc[4 * c + 2] = acc[4 * c + 2] * corr + p * vv.z;
                        acc[4 * c + 3] = acc[4 * c + 3] * corr + p * vv.w;
                    }
                }
                const float inv = 1.0f / den;
#pragma unroll
                for (int j = 0; j < DH; ++j) h[as * RS + ah * DH + j] += acc[j] * inv;
            }
            __syncthreads();
            for (int r = warp; r < MS; r += 8)
                ln_row<D>(h + r * RS, m.w + o.ln2g, m.w + o.ln2b, a + r * RS, lane);
            __syncthreads();
            tile_gemm_auto<MS, EPI_GELU>(a, RS, m.wt + m.p.W1T[l], m.dff, D, m.wt + m.p.b1[l], u, US);
            __syncthreads();
            tile_gemm_auto<MS, EPI_ADD>(u, US, m.wt + m.p.W2T[l], D, m.dff, m.wt + m.p.b2[l], h, RS);
            __syncthreads();
        }
        // output head and the draw
        for (int r = warp; r < MS && m.P > 1; r += 8) {
            // patched: K logits (a softmax over the token classes), the class
            // by the inverse CDF of u; the cell's P spins land on the patch map
            ln_row<D>(h + r * RS, m.w + m.o.lnfg, m.w + m.o.lnfb, a + r * RS, lane);
            __syncwarp();
            float *z = u + r * US;
            for (int k = 0; k < m.K; ++k) {
                float zk = 0.f;
                for (int j = lane; j < D; j += 32) zk += a[r * RS + j] * __ldg(m.w + m.o.Wh + (size_t)k * D + j);
                zk = warp_sum(zk);
                if (lane == 0) z[k] = zk + __ldg(m.w + m.o.bh + k);
            }
            __syncwarp();
            if (lane == 0) {
                float mx = -INFINITY;
                for (int k = 0; k < m.K; ++k) mx = fmaxf(mx, z[k]);
                float se = 0.f;
                for (int k = 0; k < m.K; ++k) se += expf(z[k] - mx);
                const float lse = mx + logf(se);
                const int64_t b = b0 + r;
                const float uu = philox_uniform(seed, (uint32_t)b, (uint32_t)t, sid, 0u);
                float cdf = 0.f, near = INFINITY;
                int cls = m.K - 1;
                bool found = false;
                for (int k = 0; k < m.K - 1; ++k) {
                    cdf += expf(z[k] - lse);
                    near = fminf(near, fabsf(uu - cdf));
                    if (!found && uu < cdf) {
                        cls = k;
                        found = true;
                    }
                }
                lq[r] += z[cls] - lse;
                tok[r] = cls;
                if (b < B) {
                    for (int j = 0; j < m.P; ++j)
                        spins[(size_t)b * m.Nspins + patch_site(t, j, m.P, m.latD, m.latL)] =
                            (int8_t)(((cls >> j) & 1) ? 1 : -1);
                    if (flags && near < band) flags[(size_t)b * nfw + (t >> 5)] |= 1u << (t & 31);
                }
            }
        }
        for (int r = warp; r < MS && m.P == 1; r += 8) {
            ln_row<D>(h + r * RS, m.w + m.o.lnfg, m.w + m.o.lnfb, a + r * RS, lane);
            __syncwarp();
            float z0 = 0.f, z1 = 0.f;
            for (int j = lane; j < D; j += 32) {
                const float y = a[r * RS + j];
                z0 += y * __ldg(m.w + m.o.Wh + j);
                z1 += y * __ldg(m.w + m.o.Wh + D + j);
            }
            z0 = warp_sum(z0) + __ldg(m.w + m.o.bh);
            z1 = warp_sum(z1) + __ldg(m.w + m.o.bh + 1);
            if (lane == 0) {
                const float ell = z1 - z0;
                const float p = 1.0f / (1.0f + expf(-ell));
                const int64_t b = b0 + r;
                const float uu = philox_uniform(seed, (uint32_t)b, (uint32_t)t, sid, 0u);
                const int sp = uu < p ? 1 : -1;
                lq[r] += log_sigmoid_f((float)sp * ell);
                tok[r] = (sp + 1) >> 1;
                if (b < B) {
                    spins[(size_t)b * m.N + t] = (int8_t)sp;
                    if (flags && fabsf(p - uu) < band)
                        flags[(size_t)b * nfw + (t >> 5)] |= 1u << (t & 31);
                }
            }
        }
        __syncthreads();
    }
    for (int s = tid; s < MS; s += blockDim.x)
        if (b0 + s < B) logq[b0 + s] = lq[s];
}

// KV-cache bytes of the FP32 decode for B samples (tiles of 256 / n_heads
// samples, every slot of the ring for every layer).
size_t decode_f32_kv_bytes(const sg_model *m, int64_t B)
{
    const sg_config &c = m->seq;  // N = tokens
    const int64_t MS = 256 / c.n_heads;
    const RingGeom g = ring_geom(c.mask_kind, c.N, c.W, c.S);
    return (size_t)((B + MS - 1) / MS) * c.n_layers * g.nslots * 2 * c.d * MS * sizeof(float);
}

template <int D, int DH>
static sg_status run_decode(sg_model *m, int64_t B, uint64_t seed, uint32_t sid, float band,
                            int8_t *spins, float *logq, uint32_t *flags, cudaStream_t st)
{
    constexpr int NH = D / DH;
    constexpr int MS = 256 / NH;
    const sg_config &c = m->seq;  // N = tokens
    const int P = spins_per_token(c), K = 1 << P;
    const int64_t tiles = (B + MS - 1) / MS;
    SG_TRY(ensure_buffer(&m->kv, &m->kv_bytes, decode_f32_kv_bytes(m, B)));
    int US = (3 * D > c.d_ff ? 3 * D : c.d_ff) + 4;
    if (US < K + 4) US = K + 4;  // the head's K logits per sample reuse u
    const size_t smem = ((size_t)MS * (2 * (D + 4) + US) + 2 * MS) * sizeof(float);
    auto kern = decode_f32_kernel<D, DH>;
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DevModel dm{c.N, c.n_layers, c.d, c.n_heads, c.d_token, c.d_ff, c.mask_kind, c.W, c.S,
                P, K, m->cfg.N, c.lat_D, c.lat_L, m->w, m->wt, m->off, m->pack};
    kern<<<(unsigned)tiles, 256, smem, ::sg::counted(st)>>>(dm, B, seed, sid, band, spins, logq, flags,
                                             (float *)m->kv);
    return check_launch("decode_f32_kernel");
}

sg_status launch_decode_f32(sg_model *m, int64_t B, uint64_t seed, uint32_t sid, float band,
                            int8_t *spins, float *logq, uint32_t *flags, cudaStream_t st)
{
    const sg_config &c = m->cfg;
    const int dh = c.d / c.n_heads;
    if (c.d_ff % 8 || c.d_ff > 4 * c.d)
        return fail(SG_EUNSUPPORTED, "FP32 decode needs d_ff a multiple of 8 and <= 4 d");
    if (c.d == 32 && dh == 8) return run_decode<32, 8>(m, B, seed, sid, band, spins, logq, flags, st);
    if (c.d == 64 && dh == 16) return run_decode<64, 16>(m, B, seed, sid, band, spins, logq, flags, st);
    if (c.d == 64 && dh == 8) return run_decode<64, 8>(m, B, seed, sid, band, spins, logq, flags, st);
    if (c.d == 128 && dh == 16) return run_decode<128, 16>(m, B, seed, sid, band, spins, logq, flags, st);
    if (c.d == 128 && dh == 32) return run_decode<128, 32>(m, B, seed, sid, band, spins, logq, flags, st);
    if (c.d == 32 && dh == 16) return run_decode<32, 16>(m, B, seed, sid, band, spins, logq, flags, st);
    return fail(SG_EUNSUPPORTED, "FP32 decode is built for (d, d_h) in {(32,8), (32,16), (64,8), "
                                 "(64,16), (128,16), (128,32)}");
}

// ---------------------------------------------------------------------------
// Allocation-free sampling (sg_sample_noalloc).  Its scratch -- the packed
// weight copies followed by the KV cache -- lives in one file-scope device
// array instead of memory from cudaMalloc.  Host code cannot use the array's
// name as a device address, so every call looks it up with
// cudaGetSymbolAddress in the current context (a host-side table lookup).  No
// address is cached, so a device reset or a new primary context cannot leave
// a stale pointer behind.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[SG_NOALLOC_SCRATCH_BYTES];

static sg_status noalloc_scratch(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return fail(SG_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    *out = p;
    return SG_OK;
}

template <int D, int DH>
static sg_status run_decode_noalloc(const sg_config &c, const float *w, const BlobOff &off,
                                    const PackOff &pack, float *wt, float *kv, int64_t B,
                                    uint64_t seed, uint32_t sid, float band, int8_t *spins,
                                    float *logq, uint32_t *flags, cudaStream_t st)
{
    constexpr int NH = D / DH;
    constexpr int MS = 256 / NH;
    const int64_t tiles = (B + MS - 1) / MS;
    const int US = (3 * D > c.d_ff ? 3 * D : c.d_ff) + 4;
    const size_t smem = ((size_t)MS * (2 * (D + 4) + US) + 2 * MS) * sizeof(float);
    auto kern = decode_f32_kernel<D, DH>;
    SG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DevModel dm{c.N, c.n_layers, c.d, c.n_heads, c.d_token, c.d_ff, c.mask_kind, c.W, c.S,
                1, 2, c.N, 0, 0, w, wt, off, pack};
    kern<<<(unsigned)tiles, 256, smem, ::sg::counted(st)>>>(dm, B, seed, sid, band, spins, logq,
                                                            flags, kv);
    return check_launch("decode_f32_kernel (no-alloc)");
}

}  // namespace sg

extern "C" sg_status sg_sample_noalloc(const sg_config *cfg, const float *weights, int64_t B,
                                       double beta, uint64_t seed, uint32_t stream_id,
                                       float flag_band, int8_t *spins, float *logq,
                                       uint32_t *flags, sg_stream stream)
{
    using namespace sg;
    (void)beta;
    if (sg_param_count(cfg) < 0) return SG_EINVAL;  // message set by the validation
    if (!weights || !spins || !logq) return fail(SG_EINVAL, "NULL weights or output");
    if (B < 1 || B >= (int64_t)1 << 32) return fail(SG_EINVAL, "B must be in [1, 2^32)");
    const sg_config &c = *cfg;
    if (c.precision != SG_FP32)
        return fail(SG_EUNSUPPORTED, "sg_sample_noalloc serves the FP32 path only");
    if (c.n_models > 1) return fail(SG_EUNSUPPORTED, "sg_sample_noalloc serves single models");
    if (c.patch > 1) return fail(SG_EUNSUPPORTED, "sg_sample_noalloc serves unpatched models");
    const int dh = c.d / c.n_heads;
    const bool shape_ok = (c.d == 32 && (dh == 8 || dh == 16)) || (c.d == 64 && (dh == 8 || dh == 16)) ||
                          (c.d == 128 && (dh == 16 || dh == 32));
    if (!shape_ok || c.d_ff % 8 || c.d_ff > 4 * c.d)
        return fail(SG_EUNSUPPORTED, "sg_sample_noalloc: unsupported (d, d_h, d_ff)");
    const int MS = 256 / c.n_heads;
    const RingGeom g = ring_geom(c.mask_kind, c.N, c.W, c.S);
    const BlobOff off = blob_offsets(c);
    const PackOff pack = pack_offsets(c);
    const size_t wt_bytes = ((size_t)pack.total * sizeof(float) + 255) & ~size_t(255);
    const size_t kv_bytes = (size_t)((B + MS - 1) / MS) * c.n_layers * g.nslots * 2 * c.d * MS *
                            sizeof(float);
    if (wt_bytes + kv_bytes > SG_NOALLOC_SCRATCH_BYTES)
        return fail(SG_EINVAL, "sg_sample_noalloc needs " + std::to_string(wt_bytes + kv_bytes) +
                                   " bytes of scratch; the static scratch holds " +
                                   std::to_string((unsigned long long)SG_NOALLOC_SCRATCH_BYTES) +
                                   " (reduce B or use sg_sample)");
    void *base = nullptr;
    SG_TRY(noalloc_scratch(&base));
    float *wt = static_cast<float *>(base);
    float *kv = reinterpret_cast<float *>(static_cast<unsigned char *>(base) + wt_bytes);
    cudaStream_t st = (cudaStream_t)stream;
    if (flag_band <= 0.f) flag_band = 1e-5f;
    if (flags)
        SG_CUDA_TRY(cudaMemsetAsync(flags, 0, (size_t)B * ((c.N + 31) / 32) * sizeof(uint32_t), st));
    // packed copies of this call's weights (every byte the kernel reads is
    // written here or earlier in the same launch, so nothing needs clearing)
    const size_t f4 = sizeof(float);
    for (int l = 0; l < c.n_layers; ++l) {
        const LayerOff &o = off.L[l];
        transpose(weights + o.Wqkv, wt + pack.WqkvT[l], 3 * c.d, c.d, st);
        transpose(weights + o.W1, wt + pack.W1T[l], c.d_ff, c.d, st);
        transpose(weights + o.W2, wt + pack.W2T[l], c.d, c.d_ff, st);
        SG_CUDA_TRY(cudaMemcpyAsync(wt + pack.bqkv[l], weights + o.bqkv, (size_t)3 * c.d * f4,
                                    cudaMemcpyDeviceToDevice, st));
        SG_CUDA_TRY(cudaMemcpyAsync(wt + pack.b1[l], weights + o.b1, (size_t)c.d_ff * f4,
                                    cudaMemcpyDeviceToDevice, st));
        SG_CUDA_TRY(cudaMemcpyAsync(wt + pack.b2[l], weights + o.b2, (size_t)c.d * f4,
                                    cudaMemcpyDeviceToDevice, st));
    }
    SG_TRY(check_launch("pack weights (no-alloc)"));
#define SG_NA(DD, HH)                                                                          \
    if (c.d == DD && dh == HH)                                                                 \
        return run_decode_noalloc<DD, HH>(c, weights, off, pack, wt, kv, B, seed, stream_id,   \
                                          flag_band, spins, logq, flags, st);
    SG_NA(32, 8) SG_NA(32, 16) SG_NA(64, 8) SG_NA(64, 16) SG_NA(128, 16) SG_NA(128, 32)
#undef SG_NA
    return fail(SG_EUNSUPPORTED, "sg_sample_noalloc: unsupported (d, d_h)");
}
