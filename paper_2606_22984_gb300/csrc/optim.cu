// optim.cu -- Muon (Methods "Comparison on optimizers"): per weight matrix,
// momentum M = mu M + G, the quintic Newton-Schulz orthogonalisation of
// Jordan et al. (2024) on X = M / (|M|_F + 1e-7) (on M^T when M has more rows
// than columns): X <- a X + (b A + c A A) X, A = X X^T, (a, b, c) =
// (3.4445, -4.7750, 2.0315); then W -= lr (s O + wd W) with the RMS alignment
// s = 0.2 sqrt(max(rows, cols)) and decoupled weight decay of Liu et al.
// (2025).  The other parameters take an AdamW step.
//
// The matrices are at most a few hundred by a thousand, so each product of
// the iteration is a small FP32 GEMM on CUDA cores (64 x 64 output tiles);
// the step is bound by launch latency, not by the tensor cores.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sg_internal.cuh"

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
    // scratch: X, Y (p x q), A, Bm (p x p) for the largest matrix, then the norm
    size_t mat_bytes = 0;
    for (const Seg &s : segs)
        if (s.rows) {
            const size_t p = std::min(s.rows, s.cols), q = std::max(s.rows, s.cols);
            mat_bytes = std::max(mat_bytes, (2 * p * q + 2 * p * p) * sizeof(float));
        }
    const size_t ss_off = (mat_bytes + 255) / 256 * 256;
    SG_TRY(ensure_buffer(&m->ws, &m->ws_bytes, ss_off + 256));
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)step));
    const float bc2 = (float)(1.0 - std::pow(0.999, (double)step));
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
