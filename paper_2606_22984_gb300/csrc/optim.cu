// optim.cu -- Muon (Methods "Comparison on optimizers"): per weight matrix,
// momentum M = mu M + G, the quintic Newton-Schulz orthogonalisation of
// Jordan et al. (2024) on X = M / (|M|_F + 1e-7) (on M^T when M has more rows
// than columns): X <- a X + (b A + c A A) X, A = X X^T, (a, b, c) =
// (3.4445, -4.7750, 2.0315); then W -= lr (s O + wd W) with the RMS alignment
// s = 0.2 sqrt(max(rows, cols)) and decoupled weight decay of Liu et al.
// (2025).  The other parameters take an AdamW step.
//
// FP32 models: each product of the iteration is a small FP32 GEMM on CUDA
// cores (64 x 64 output tiles), three launches per Newton-Schulz step.
// BF16 models whose matrices have min(rows, cols) <= 128 (d <= 128): one
// launch runs the whole step for every weight matrix of the model, one CTA per
// matrix (muon_ns_tc_kernel): momentum, normalisation, the Newton-Schulz
// iteration on tcgen05 tensor cores with X kept in shared memory as BF16 (the
// operand precision of the BF16 path; the iteration is the usual BF16 practice
// for Muon) and FP32 accumulators in TMEM, and the weight update.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sg_internal.cuh"
#include "tc.cuh"

namespace sg {

namespace {

__global__ void momentum_sumsq_kernel(float *__restrict__ M, const float *__restrict__ G, int64_t n,
                                      float mu, double *__restrict__ ss)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float v = mu * M[i] + G[i];
        M[i] = v;
        acc += (double)v * v;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(ss, red[0]);
}

// X (p x q, p <= q) = M / (|M|_F + 1e-7), transposed when rows > cols
__global__ void ns_init_kernel(const float *__restrict__ M, int rows, int cols,
                               const double *__restrict__ ss, float *__restrict__ X)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * cols) return;
    const int r = (int)(i / cols), c = (int)(i % cols);
    const float inv = (float)(1.0 / (sqrt(*ss) + 1e-7));
    const float v = M[i] * inv;
    if (rows > cols) X[(int64_t)c * rows + r] = v;
    else X[i] = v;
}

// C[M][N] = alpha sum_k A(m, k) B(k, n) + beta D[M][N], operands addressed by
// strides (so transposes are free); 64 x 64 tile per block, 4 x 4 per thread.
__global__ void __launch_bounds__(256)
sgemm_strided_kernel(int M, int N, int K, const float *__restrict__ A, int64_t sam, int64_t sak,
                     const float *__restrict__ B, int64_t sbk, int64_t sbn, float alpha,
                     const float *__restrict__ D, float beta, float *__restrict__ C)
{
    __shared__ float As[16][65], Bs[16][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = tid; e < 64 * 16; e += 256) {
            const int mm = e >> 4, kk = e & 15;
            As[kk][mm] = (m0 + mm < M && k0 + kk < K) ? A[(int64_t)(m0 + mm) * sam + (int64_t)(k0 + kk) * sak] : 0.f;
            const int kb = e >> 6, nn = e & 63;
            Bs[kb][nn] = (k0 + kb < K && n0 + nn < N) ? B[(int64_t)(k0 + kb) * sbk + (int64_t)(n0 + nn) * sbn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty * 4 + i];
                b[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) {
                const int64_t o = (int64_t)m * N + n;
                C[o] = alpha * acc[i][j] + (D ? beta * D[o] : 0.f);
            }
        }
}

// W -= lr (s O + wd W); O is X (p x q) read back in the matrix's orientation
__global__ void muon_apply_kernel(float *__restrict__ W, const float *__restrict__ X, int rows,
                                  int cols, float lr, float s, float wd)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * cols) return;
    const int r = (int)(i / cols), c = (int)(i % cols);
    const float o = rows > cols ? X[(int64_t)c * rows + r] : X[i];
    W[i] -= lr * (s * o + wd * W[i]);
}

__global__ void adamw_kernel(float *__restrict__ w, const float *__restrict__ g,
                             float *__restrict__ m, float *__restrict__ v, int64_t n, float lr,
                             float wd, float bc1, float bc2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * ((mi / bc1) / (sqrtf(vi / bc2) + 1e-8f) + wd * w[i]);
}

struct Seg {
    int64_t off, n;
    int rows, cols;  // rows > 0: a weight matrix
};

// ---------------------------------------------------------------------------
// Newton-Schulz on tcgen05 for one weight matrix per CTA (128 threads; thread
// r owns row r of the iterate X (p x q, p = min(rows, cols) <= 128, rows p ..
// 127 zero) and TMEM lane r).  Per step:
//   A  = X X^T           M = 128, N = p, K = q      -> TMEM columns [0, p)
//   A2 = A A^T (A in BF16) M = 128, N = p, K = p     -> TMEM columns [128, 128 + p)
//   Bm = b A + c A2 (BF16, shared memory)
//   Y  = Bm X            M = 128, N = q (<= 256 per MMA), K = p, X read MN-major
//                                                    -> TMEM columns [0, q)
//   X  = a X + Y (BF16, in place)
// X sits in the core-matrix layout of one 128-row block (8 x 8 BF16 cores of
// 128 bytes, K-adjacent cores 128 bytes apart, 8-row groups q / 8 cores
// apart): K-major for the first product (both operands), MN-major for the
// last (instruction-descriptor bit 16; leading byte offset = the 16 q bytes
// between 8-row groups, stride byte offset = 128 bytes between cores).
// ---------------------------------------------------------------------------
constexpr int kMuonJobs = 3 * SG_MAX_LAYERS;

struct MuonJobs {
    int n;
    int64_t off[kMuonJobs];
    int rows[kMuonJobs], cols[kMuonJobs];
};

__device__ __forceinline__ uint16_t bf16_bits(float v)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t *>(&h);
}

__device__ __forceinline__ float bf16_float(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

__global__ void __launch_bounds__(128, 1)
muon_ns_tc_kernel(const __grid_constant__ MuonJobs jobs, float *__restrict__ W,
                  const float *__restrict__ G, float *__restrict__ Mom, float lr, float mu,
                  float wd, int ns_steps, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ double red[4];
    __shared__ int s_err;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lanes = (uint32_t)(32 * warp) << 16;
    constexpr float ca = 3.4445f, cb = -4.7750f, cc = 2.0315f;
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
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
    uint32_t phase = 0;
    // wait for the MMAs thread 0 committed; a bounded wait that gives up
    // records the error and the remaining steps are skipped
    auto mma_done = [&]() {
        if (tid == 0) tc::mma_commit(&bar);
        __syncwarp();
        if (!tc::mbar_wait(&bar, phase)) {
            if (lane == 0) atomicExch(err, 31);
            s_err = 1;
        }
        phase ^= 1u;
        __syncthreads();
        tc::tc_fence_after();
    };
    for (int job = blockIdx.x; job < jobs.n; job += gridDim.x) {
        const int rows = jobs.rows[job], cols = jobs.cols[job];
        const bool tr = rows > cols;
        const int p = tr ? cols : rows, q = tr ? rows : cols;
        const int64_t n = (int64_t)rows * cols;
        float *w = W + jobs.off[job];
        float *m = Mom + jobs.off[job];
        const float *g = G + jobs.off[job];
        unsigned char *Xs = smem;                              // 128 x q BF16
        unsigned char *Ab = smem + (size_t)128 * q * 2;       // 128 x p BF16 (A, then Bm)
        const uint32_t kgx = (uint32_t)q / 8, kga = (uint32_t)p / 8;
        // momentum and its squared Frobenius norm
        double ss = 0.0;
        for (int64_t i = tid; i < n; i += blockDim.x) {
            const float v = mu * m[i] + g[i];
            m[i] = v;
            ss += (double)v * v;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) red[warp] = ss;
        // zero the rows p .. 127 of X and of the A tile
        for (int i = tid; i < (128 - p) * q; i += blockDim.x) {
            const int r = p + i / q, k = i % q;
            *reinterpret_cast<uint16_t *>(Xs + tc::cm_offset(r, k, kgx)) = 0;
        }
        for (int i = tid; i < (128 - p) * p; i += blockDim.x) {
            const int r = p + i / p, k = i % p;
            *reinterpret_cast<uint16_t *>(Ab + tc::cm_offset(r, k, kga)) = 0;
        }
        __syncthreads();
        const float inv = (float)(1.0 / (sqrt(red[0] + red[1] + red[2] + red[3]) + 1e-7));
        // X = M / (|M|_F + 1e-7), transposed when rows > cols
        for (int64_t i = tid; i < n; i += blockDim.x) {
            const int r = (int)(i / cols), c = (int)(i % cols);
            const int xr = tr ? c : r, xk = tr ? r : c;
            *reinterpret_cast<uint16_t *>(Xs + tc::cm_offset(xr, xk, kgx)) = bf16_bits(m[i] * inv);
        }
        tc::fence_async_smem();
        tc::tc_fence_before();
        __syncthreads();
        tc::tc_fence_after();
        const uint32_t sx = tc::smem_u32(Xs), sab = tc::smem_u32(Ab);
        for (int it = 0; it < ns_steps && !s_err; ++it) {
            // A = X X^T
            if (tid == 0)
                for (int ks = 0; ks < q / 16; ++ks) {
                    const uint64_t d = tc::smem_desc(sx + 256u * ks, 128, kgx * 128);
                    tc::mma_bf16(tmem, d, d, tc::idesc_bf16(128, p), ks > 0);
                }
            mma_done();
            if (s_err) break;
            // A as a BF16 operand
            for (int c0 = 0; c0 < p; c0 += 32) {
                float v[32];
                tc::tmem_ld32(tmem + lanes + (uint32_t)c0, v);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c0 + j < p)
                        *reinterpret_cast<uint16_t *>(Ab + tc::cm_offset(tid, c0 + j, kga)) = bf16_bits(v[j]);
            }
            tc::fence_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            tc::tc_fence_after();
            // A2 = A A^T
            if (tid == 0)
                for (int ks = 0; ks < p / 16; ++ks) {
                    const uint64_t d = tc::smem_desc(sab + 256u * ks, 128, kga * 128);
                    tc::mma_bf16(tmem + 128, d, d, tc::idesc_bf16(128, p), ks > 0);
                }
            mma_done();
            if (s_err) break;
            // Bm = b A + c A2 (BF16, over the A tile)
            for (int c0 = 0; c0 < p; c0 += 32) {
                float va[32], v2[32];
                tc::tmem_ld32(tmem + lanes + (uint32_t)c0, va);
                tc::tmem_ld32(tmem + lanes + 128u + (uint32_t)c0, v2);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c0 + j < p)
                        *reinterpret_cast<uint16_t *>(Ab + tc::cm_offset(tid, c0 + j, kga)) =
                            bf16_bits(cb * va[j] + cc * v2[j]);
            }
            tc::fence_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            tc::tc_fence_after();
            // Y = Bm X: X read MN-major, N blocks of at most 256 columns
            if (tid == 0)
                for (int n0 = 0; n0 < q; n0 += 256) {
                    const int nw = min(256, q - n0);
                    const uint32_t idesc = tc::idesc_bf16(128, nw) | (1u << 16);
                    for (int ks = 0; ks < p / 16; ++ks)
                        tc::mma_bf16(tmem + (uint32_t)n0,
                                     tc::smem_desc(sab + 256u * ks, 128, kga * 128),
                                     tc::smem_desc(sx + (uint32_t)(ks * 2 * 16 * q + (n0 / 8) * 128),
                                                   16u * q, 128),
                                     idesc, ks > 0);
                }
            mma_done();
            if (s_err) break;
            // X = a X + Y (this thread's row, in place)
            for (int c0 = 0; c0 < q; c0 += 32) {
                float y[32];
                tc::tmem_ld32(tmem + lanes + (uint32_t)c0, y);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (tid < p && c0 + j < q) {  // q may end mid-chunk (a multiple of 16)
                        uint16_t *xp = reinterpret_cast<uint16_t *>(Xs + tc::cm_offset(tid, c0 + j, kgx));
                        *xp = bf16_bits(ca * bf16_float(*xp) + y[j]);
                    }
            }
            tc::fence_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            tc::tc_fence_after();
        }
        if (s_err) break;
        // W -= lr (s O + wd W), O = X in the matrix's orientation
        const float scale = 0.2f * sqrtf((float)q);
        for (int64_t i = tid; i < n; i += blockDim.x) {
            const int r = (int)(i / cols), c = (int)(i % cols);
            const int xr = tr ? c : r, xk = tr ? r : c;
            const float o = bf16_float(*reinterpret_cast<const uint16_t *>(Xs + tc::cm_offset(xr, xk, kgx)));
            w[i] -= lr * (scale * o + wd * w[i]);
        }
        __syncthreads();  // X is rewritten by the next job
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

std::vector<Seg> segments(const sg_model *m)
{
    const sg_config &c = m->cfg;
    const int64_t d = c.d, f = c.d_ff;
    std::vector<Seg> out;
    int64_t at = 0;
    auto rest_until = [&](int64_t end) {
        if (end > at) out.push_back({at, end - at, 0, 0});
        at = end;
    };
    auto mat = [&](int64_t off, int r, int cc) {
        rest_until(off);
        out.push_back({off, (int64_t)r * cc, r, cc});
        at = off + (int64_t)r * cc;
    };
    for (int l = 0; l < c.n_layers; ++l) {
        const LayerOff &o = m->off.L[l];
        mat(o.Wqkv, (int)(3 * d), (int)d);
        mat(o.W1, (int)f, (int)d);
        mat(o.W2, (int)d, (int)f);
    }
    rest_until(m->off.total);
    return out;
}

unsigned blocks_of(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

}  // namespace sg

using namespace sg;

extern "C" sg_status sg_muon_step(sg_model *m, float *weights, const float *grad, float *momentum,
                                  float *adam_m, float *adam_v, double lr, double mu,
                                  double weight_decay, int32_t ns_steps, int64_t step,
                                  sg_stream stream)
{
    if (!m || !weights || !grad || !momentum || !adam_m || !adam_v)
        return fail(SG_EINVAL, "NULL model or pointer");
    if (step < 1 || ns_steps < 0 || ns_steps > 32) return fail(SG_EINVAL, "bad step or ns_steps");
    if (!std::isfinite(lr) || !std::isfinite(mu) || !std::isfinite(weight_decay))
        return fail(SG_EINVAL, "lr, mu and weight_decay must be finite");
    if (m->n_models > 1) return fail(SG_EUNSUPPORTED, "sg_muon_step serves single models");
    cudaStream_t st = (cudaStream_t)stream;
    const std::vector<Seg> segs = segments(m);
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)step));
    const float bc2 = (float)(1.0 - std::pow(0.999, (double)step));
    // BF16 models with every matrix within the tensor-core kernel's shapes:
    // one launch for all matrices, AdamW for the rest
    bool tc_ok = m->cfg.precision == SG_BF16;
    MuonJobs jobs{};
    int qmax = 0;
    for (const Seg &s : segs)
        if (s.rows && tc_ok) {
            const int p = std::min(s.rows, s.cols), q = std::max(s.rows, s.cols);
            tc_ok = p <= 128 && p % 16 == 0 && q % 16 == 0 && q <= 512 && jobs.n < kMuonJobs;
            if (tc_ok) {
                jobs.off[jobs.n] = s.off;
                jobs.rows[jobs.n] = s.rows;
                jobs.cols[jobs.n] = s.cols;
                ++jobs.n;
                qmax = std::max(qmax, q);
            }
        }
    if (tc_ok && jobs.n > 0) {
        SG_TRY(ensure_buffer(&m->err, &m->err_bytes, sizeof(int)));
        const size_t smem = (size_t)128 * qmax * 2 + (size_t)128 * 128 * 2;
        SG_CUDA_TRY(cudaFuncSetAttribute(muon_ns_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        muon_ns_tc_kernel<<<(unsigned)jobs.n, 128, smem, counted(st)>>>(
            jobs, weights, grad, momentum, (float)lr, (float)mu, (float)weight_decay, ns_steps,
            (int *)m->err);
        for (const Seg &s : segs)
            if (!s.rows)
                adamw_kernel<<<blocks_of(s.n), 256, 0, counted(st)>>>(
                    weights + s.off, grad + s.off, adam_m + s.off, adam_v + s.off, s.n, (float)lr,
                    (float)weight_decay, bc1, bc2);
        return check_launch("muon step (tensor cores)");
    }
    // scratch: X, Y (p x q), A, Bm (p x p) for the largest matrix, then the norm
    size_t mat_bytes = 0;
    for (const Seg &s : segs)
        if (s.rows) {
            const size_t p = std::min(s.rows, s.cols), q = std::max(s.rows, s.cols);
            mat_bytes = std::max(mat_bytes, (2 * p * q + 2 * p * p) * sizeof(float));
        }
    const size_t ss_off = (mat_bytes + 255) / 256 * 256;
    SG_TRY(ensure_buffer(&m->ws, &m->ws_bytes, ss_off + 256));
    const float a = 3.4445f, b = -4.7750f, c = 2.0315f;
    for (const Seg &s : segs) {
        if (!s.rows) {
            adamw_kernel<<<blocks_of(s.n), 256, 0, counted(st)>>>(
                weights + s.off, grad + s.off, adam_m + s.off, adam_v + s.off, s.n, (float)lr,
                (float)weight_decay, bc1, bc2);
            continue;
        }
        const int p = std::min(s.rows, s.cols), q = std::max(s.rows, s.cols);
        float *X = (float *)m->ws;
        float *Y = X + (size_t)p * q;
        float *A = Y + (size_t)p * q;
        float *Bm = A + (size_t)p * p;
        double *ss = reinterpret_cast<double *>((unsigned char *)m->ws + ss_off);
        SG_CUDA_TRY(cudaMemsetAsync(ss, 0, sizeof(double), st));
        momentum_sumsq_kernel<<<std::min<unsigned>(blocks_of(s.n), 1024), 256, 0, counted(st)>>>(
            momentum + s.off, grad + s.off, s.n, (float)mu, ss);
        ns_init_kernel<<<blocks_of(s.n), 256, 0, counted(st)>>>(momentum + s.off, s.rows, s.cols, ss, X);
        for (int it = 0; it < ns_steps; ++it) {
            // A = X X^T (p x p)
            sgemm_strided_kernel<<<dim3((p + 63) / 64, (p + 63) / 64), 256, 0, counted(st)>>>(
                p, p, q, X, q, 1, X, 1, q, 1.f, nullptr, 0.f, A);
            // Bm = c A A + b A
            sgemm_strided_kernel<<<dim3((p + 63) / 64, (p + 63) / 64), 256, 0, counted(st)>>>(
                p, p, p, A, p, 1, A, p, 1, c, A, b, Bm);
            // Y = Bm X + a X
            sgemm_strided_kernel<<<dim3((q + 63) / 64, (p + 63) / 64), 256, 0, counted(st)>>>(
                p, q, p, Bm, p, 1, X, q, 1, 1.f, X, a, Y);
            std::swap(X, Y);
        }
        const float scale = 0.2f * std::sqrt((float)std::max(s.rows, s.cols));
        muon_apply_kernel<<<blocks_of(s.n), 256, 0, counted(st)>>>(
            weights + s.off, X, s.rows, s.cols, (float)lr, scale, (float)weight_decay);
    }
    return check_launch("muon step");
}
