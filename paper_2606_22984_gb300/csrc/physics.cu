// physics.cu -- energies (Eqs. SKHam, EAHam), the FP64 free-energy
// reduction (Eqs. KL_div, free_energy), independence Metropolis-Hastings,
// single-spin-flip Metropolis, the overlap histogram (Eq.
// overlap_distribution) and the Adam update.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sg_internal.cuh"

namespace sg {

namespace {

__device__ __forceinline__ float wsum_f(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int wsum_i(int v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// +mu neighbour of raster site i (x0 fastest) on an L^D lattice; -1 if the
// bond leaves an open lattice.
__device__ __forceinline__ int ea_plus(int i, int mu, int L, int periodic)
{
    int stride = 1;
    for (int k = 0; k < mu; ++k) stride *= L;
    const int x = (i / stride) % L;
    if (x == L - 1) return periodic ? i - (L - 1) * stride : -1;
    return i + stride;
}

__device__ __forceinline__ int ea_minus(int i, int mu, int L, int periodic)
{
    int stride = 1;
    for (int k = 0; k < mu; ++k) stride *= L;
    const int x = (i / stride) % L;
    if (x == 0) return periodic ? i + (L - 1) * stride : -1;
    return i - stride;
}

// ---------------------------------------------------------------------------
// EA energy: one warp per configuration, lanes over sites, coalesced reads of
// the spin row; integer bonds accumulate exactly in int32.
// ---------------------------------------------------------------------------
template <bool INT>
__global__ void ea_energy_kernel(const int8_t *__restrict__ spins, int64_t B, int N, int D,
                                 int L, int periodic, const float *__restrict__ J,
                                 const int8_t *__restrict__ Ji, float *__restrict__ E,
                                 int32_t *__restrict__ Ei)
{
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= B) return;
    const int8_t *s = spins + b * N;
    int ai = 0;
    float af = 0.f;
    for (int i = lane; i < N; i += 32) {
        const int si = s[i];
        for (int mu = 0; mu < D; ++mu) {
            const int j = ea_plus(i, mu, L, periodic);
            if (j < 0) continue;
            if (INT) ai += (int)Ji[(size_t)i * D + mu] * si * s[j];
            else af += J[(size_t)i * D + mu] * (float)(si * s[j]);
        }
    }
    if (INT) {
        const int e = -wsum_i(ai);
        if (lane == 0) {
            E[b] = (float)e;
            if (Ei) Ei[b] = e;
        }
    } else {
        const float e = -wsum_f(af);
        if (lane == 0) E[b] = e;
    }
}

// ---------------------------------------------------------------------------
// SK energy on CUDA cores: Y = S J for a tile of 64 configurations, then
// E_b = -1/2 sum_i s_bi Y_bi.  Each thread owns 4 configurations x 4 columns
// per 64-column block and keeps its partial energies in registers; a fixed
// order block reduction makes the result deterministic.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
sk_energy_f32_kernel(const int8_t *__restrict__ spins, int64_t B, int N,
                     const float *__restrict__ J, float *__restrict__ E)
{
    extern __shared__ int8_t ss[];  // [64][N] spins of the tile
    __shared__ float red[16][64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t b0 = (int64_t)blockIdx.x * 64;
    for (int e = tid; e < 64 * N; e += 256) {
        const int r = e / N, i = e % N;
        ss[e] = (b0 + r < B) ? spins[(b0 + r) * N + i] : (int8_t)0;
    }
    __syncthreads();
    float part[4] = {0.f, 0.f, 0.f, 0.f};
    for (int c0 = 0; c0 < N; c0 += 64) {
        float y[4][4] = {};
        const int col = c0 + 4 * tx;
        for (int j = 0; j < N; ++j) {
            float jv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) jv[q] = col + q < N ? __ldg(J + (size_t)j * N + col + q) : 0.f;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float sj = (float)ss[(4 * ty + r) * N + j];
#pragma unroll
                for (int q = 0; q < 4; ++q) y[r][q] += sj * jv[q];
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (col + q < N) part[r] += (float)ss[(4 * ty + r) * N + col + q] * y[r][q];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) red[tx][4 * ty + r] = part[r];
    __syncthreads();
    if (tid < 64 && b0 + tid < B) {
        float e = 0.f;
        for (int x = 0; x < 16; ++x) e += red[x][tid];
        E[b0 + tid] = -0.5f * e;
    }
}

// ---------------------------------------------------------------------------
// FP64 batch reductions for F_q, F_IS, Kish ESS and REINFORCE weights.
// ---------------------------------------------------------------------------
__device__ double block_reduce(double v, double *sh, bool is_max)
{
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int w = blockDim.x >> 1; w; w >>= 1) {
        if (tid < w) sh[tid] = is_max ? fmax(sh[tid], sh[tid + w]) : sh[tid] + sh[tid + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(1024)
free_energy_kernel(const float *__restrict__ E, const float *__restrict__ lq, int64_t B,
                   double beta, double *__restrict__ out, float *__restrict__ coeff)
{
    __shared__ double sh[1024];
    double mx = -INFINITY, sl = 0.0;
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
        const double L = beta * (double)E[b] + (double)lq[b];
        sl += L;
        mx = fmax(mx, -L);
    }
    mx = block_reduce(mx, sh, true);
    sl = block_reduce(sl, sh, false);
    double sw = 0.0, sw2 = 0.0;
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
        const double L = beta * (double)E[b] + (double)lq[b];
        const double w = exp(-L - mx);
        sw += w;
        sw2 += w * w;
    }
    sw = block_reduce(sw, sh, false);
    sw2 = block_reduce(sw2, sh, false);
    const double mean = sl / (double)B;
    if (threadIdx.x == 0) {
        out[0] = mean / beta;
        out[1] = -(mx + log(sw) - log((double)B)) / beta;
        out[2] = sw * sw / sw2;
    }
    if (coeff)
        for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
            const double L = beta * (double)E[b] + (double)lq[b];
            coeff[b] = (float)((L - mean) / (double)B);
        }
}

// REINFORCE weights of L_b = a E_b + c ln q_b with the likelihood term w:
// coeff_b = (L_b - mean L - w) / B, one block, FP64 sums.
__global__ void __launch_bounds__(1024)
loss_coeff_kernel(const float *__restrict__ E, const float *__restrict__ lq, int64_t B, double a,
                  double c, double w, double *__restrict__ mean, float *__restrict__ coeff)
{
    __shared__ double sh[1024];
    double sl = 0.0, se = 0.0;
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
        sl += a * (double)E[b] + c * (double)lq[b];
        se += (double)E[b];
    }
    sl = block_reduce(sl, sh, false);
    se = block_reduce(se, sh, false);
    const double ml = sl / (double)B;
    if (threadIdx.x == 0 && mean) {
        mean[0] = ml;
        mean[1] = se / (double)B;
    }
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x)
        coeff[b] = (float)((a * (double)E[b] + c * (double)lq[b] - ml - w) / (double)B);
}

// ---------------------------------------------------------------------------
// Independence MH: one thread per chain, proposals consumed in order.  The
// log-acceptance is formed in FP64 with explicitly rounded operations (no
// contraction) so that the same inputs give the same decisions everywhere.
// ---------------------------------------------------------------------------
__global__ void mh_kernel(const int8_t *__restrict__ prop, const float *__restrict__ E,
                          const float *__restrict__ lq, int64_t B, int N, int C, double beta,
                          uint64_t seed, int8_t *__restrict__ cs, double *__restrict__ cE,
                          double *__restrict__ cL, int64_t *__restrict__ acc,
                          float *__restrict__ trace)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int64_t per = B / C;
    double e = cE[c], l = cL[c];
    int64_t idx = -1, na = 0;
    for (int64_t j = 0; j < per; ++j) {
        const int64_t p = j * C + c;
        const double ep = (double)E[p], lp = (double)lq[p];
        const double la = __dsub_rn(__dsub_rn(__dmul_rn(-beta, ep), lp),
                                    __dsub_rn(__dmul_rn(-beta, e), l));
        const float u = philox_uniform(seed, (uint32_t)c, (uint32_t)j, 1u, 0u);
        if (log((double)u) < la) {
            e = ep;
            l = lp;
            idx = p;
            ++na;
        }
        if (trace) trace[j * C + c] = (float)e;
    }
    cE[c] = e;
    cL[c] = l;
    acc[c] = na;
    if (idx >= 0)
        for (int i = 0; i < N; ++i) cs[(size_t)c * N + i] = prop[(size_t)idx * N + i];
}

// ---------------------------------------------------------------------------
// Single-spin-flip Metropolis.  A block holds RPB replicas; its threads visit
// site i together, so coupling reads are warp-uniform.  Spins live in shared
// memory as [site][replica].
// ---------------------------------------------------------------------------
template <bool SK, bool INT>
__global__ void metropolis_kernel(int8_t *__restrict__ spins, int64_t R, int N, int D, int L,
                                  int periodic, const float *__restrict__ J,
                                  const int8_t *__restrict__ Ji, int sweeps, double beta,
                                  uint64_t seed, double *__restrict__ E,
                                  float *__restrict__ trace)
{
    extern __shared__ int8_t sm[];
    const int RPB = blockDim.x;
    const int lr = threadIdx.x;
    const int64_t r = (int64_t)blockIdx.x * RPB + lr;
    const bool active = r < R;
    for (int e = threadIdx.x; e < N * RPB; e += RPB) {
        const int i = e / RPB, rr = e % RPB;
        const int64_t rg = (int64_t)blockIdx.x * RPB + rr;
        sm[e] = rg < R ? spins[rg * N + i] : (int8_t)1;
    }
    __syncthreads();
    double e = active ? E[r] : 0.0;
    for (int w = 0; w < sweeps; ++w) {
        for (int i = 0; i < N; ++i) {
            double h;
            if (SK) {
                float hf = 0.f;
                double hd = 0.0;
                for (int j = 0; j < N; ++j)
                    if (j != i) hd += (double)__ldg(J + (size_t)i * N + j) * sm[j * RPB + lr];
                (void)hf;
                h = hd;
            } else if (INT) {
                int hi = 0;
                for (int mu = 0; mu < D; ++mu) {
                    const int jp = ea_plus(i, mu, L, periodic);
                    if (jp >= 0) hi += (int)__ldg(Ji + (size_t)i * D + mu) * sm[jp * RPB + lr];
                    const int jm = ea_minus(i, mu, L, periodic);
                    if (jm >= 0) hi += (int)__ldg(Ji + (size_t)jm * D + mu) * sm[jm * RPB + lr];
                }
                h = (double)hi;
            } else {
                double hd = 0.0;
                for (int mu = 0; mu < D; ++mu) {
                    const int jp = ea_plus(i, mu, L, periodic);
                    if (jp >= 0) hd += (double)__ldg(J + (size_t)i * D + mu) * sm[jp * RPB + lr];
                }
                for (int mu = 0; mu < D; ++mu) {
                    const int jm = ea_minus(i, mu, L, periodic);
                    if (jm >= 0) hd += (double)__ldg(J + (size_t)jm * D + mu) * sm[jm * RPB + lr];
                }
                h = hd;
            }
            const int si = sm[i * RPB + lr];
            const double dE = __dmul_rn(2.0 * (double)si, h);
            const double a = exp(__dmul_rn(-beta, dE));
            const float u = philox_uniform(seed, (uint32_t)r, (uint32_t)i, 2u, (uint32_t)w);
            if ((double)u < a) {
                sm[i * RPB + lr] = (int8_t)-si;
                e = __dadd_rn(e, dE);
            }
        }
        if (trace && active) trace[(size_t)w * R + r] = (float)e;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < N * RPB; q += RPB) {
        const int i = q / RPB, rr = q % RPB;
        const int64_t rg = (int64_t)blockIdx.x * RPB + rr;
        if (rg < R) spins[rg * N + i] = sm[q];
    }
    if (active) E[r] = e;
}

__global__ void overlap_kernel(const int8_t *__restrict__ s, int64_t B, int N,
                               unsigned long long *__restrict__ hist)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * k + 1 >= B) return;
    const int8_t *a = s + 2 * k * N, *b = a + N;
    int dot = 0;
    for (int i = 0; i < N; ++i) dot += a[i] * b[i];
    atomicAdd(hist + (dot + N) / 2, 1ull);
}

__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float bc1, float bc2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

}  // namespace

sg_status launch_energy(const sg_instance *inst, const int8_t *spins, int64_t B, int prec,
                        float *E, int32_t *E_int, cudaStream_t st)
{
    (void)prec;
    if (inst->kind == SG_EA_LATTICE) {
        const unsigned blocks = (unsigned)((B + 7) / 8);
        if (inst->integer_bonds)
            ea_energy_kernel<true><<<blocks, 256, 0, ::sg::counted(st)>>>(spins, B, inst->N, inst->D, inst->L,
                                                           inst->periodic, inst->J, inst->Ji8, E,
                                                           E_int);
        else
            ea_energy_kernel<false><<<blocks, 256, 0, ::sg::counted(st)>>>(spins, B, inst->N, inst->D, inst->L,
                                                            inst->periodic, inst->J, nullptr, E,
                                                            nullptr);
        return check_launch("ea_energy_kernel");
    }
    if (prec == SG_BF16 && sk_tc_supported(inst->N)) {
        sg_instance *mi = const_cast<sg_instance *>(inst);  // workspace only
        return launch_energy_sk_tc(inst, spins, B, E, &mi->ws, &mi->ws_bytes, (int *)mi->err, st);
    }
    const size_t smem = (size_t)64 * inst->N;
    if (smem > 200 * 1024) return fail(SG_EUNSUPPORTED, "SK energy on CUDA cores needs N <= 3200");
    SG_CUDA_TRY(cudaFuncSetAttribute(sk_energy_f32_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    sk_energy_f32_kernel<<<(unsigned)((B + 63) / 64), 256, smem, ::sg::counted(st)>>>(spins, B, inst->N, inst->J,
                                                                       E);
    return check_launch("sk_energy_f32_kernel");
}

sg_status launch_free_energy(const float *E, const float *logq, int64_t B, double beta,
                             double *out, float *coeff, cudaStream_t st)
{
    free_energy_kernel<<<1, 1024, 0, ::sg::counted(st)>>>(E, logq, B, beta, out, coeff);
    return check_launch("free_energy_kernel");
}

sg_status launch_loss_coeff(const float *E, const float *logq, int64_t B, double a, double c,
                            double w, double *mean, float *coeff, cudaStream_t st)
{
    loss_coeff_kernel<<<1, 1024, 0, ::sg::counted(st)>>>(E, logq, B, a, c, w, mean, coeff);
    return check_launch("loss_coeff_kernel");
}

sg_status launch_mh(const int8_t *prop, const float *E, const float *logq, int64_t B, int N,
                    int C, double beta, uint64_t seed, int8_t *cs, double *cE, double *cL,
                    int64_t *acc, float *trace, cudaStream_t st)
{
    mh_kernel<<<(C + 127) / 128, 128, 0, ::sg::counted(st)>>>(prop, E, logq, B, N, C, beta, seed, cs, cE, cL,
                                               acc, trace);
    return check_launch("mh_kernel");
}

sg_status launch_metropolis(const sg_instance *inst, int8_t *spins, int64_t R, int sweeps,
                            double beta, uint64_t seed, double *E, float *trace, cudaStream_t st)
{
    int rpb = 64;
    while (rpb > 32 && (size_t)rpb * inst->N > 96 * 1024) rpb >>= 1;
    const size_t smem = (size_t)rpb * inst->N;
    if (smem > 200 * 1024) return fail(SG_EUNSUPPORTED, "Metropolis needs N <= 6400");
    const unsigned blocks = (unsigned)((R + rpb - 1) / rpb);
    if (inst->kind == SG_SK_DENSE) {
        auto k = metropolis_kernel<true, false>;
        SG_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<blocks, rpb, smem, ::sg::counted(st)>>>(spins, R, inst->N, 0, 0, 0, inst->J, nullptr, sweeps, beta,
                                     seed, E, trace);
    } else if (inst->integer_bonds) {
        auto k = metropolis_kernel<false, true>;
        SG_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<blocks, rpb, smem, ::sg::counted(st)>>>(spins, R, inst->N, inst->D, inst->L, inst->periodic, inst->J,
                                     inst->Ji8, sweeps, beta, seed, E, trace);
    } else {
        auto k = metropolis_kernel<false, false>;
        SG_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<blocks, rpb, smem, ::sg::counted(st)>>>(spins, R, inst->N, inst->D, inst->L, inst->periodic, inst->J,
                                     nullptr, sweeps, beta, seed, E, trace);
    }
    return check_launch("metropolis_kernel");
}

sg_status launch_overlap(const int8_t *spins, int64_t B, int N, int64_t *hist, cudaStream_t st)
{
    SG_CUDA_TRY(cudaMemsetAsync(hist, 0, (size_t)(N + 1) * sizeof(int64_t), st));
    const int64_t pairs = B / 2;
    overlap_kernel<<<(unsigned)((pairs + 255) / 256), 256, 0, ::sg::counted(st)>>>(
        spins, B, N, reinterpret_cast<unsigned long long *>(hist));
    return check_launch("overlap_kernel");
}

sg_status launch_adam(float *w, const float *g, float *m, float *v, int64_t n, float lr, float b1,
                      float b2, float eps, int64_t step, cudaStream_t st)
{
    const float bc1 = (float)(1.0 - std::pow((double)b1, (double)step));
    const float bc2 = (float)(1.0 - std::pow((double)b2, (double)step));
    adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ::sg::counted(st)>>>(w, g, m, v, n, lr, b1, b2, eps, bc1,
                                                             bc2);
    return check_launch("adam_kernel");
}

}  // namespace sg

// ---------------------------------------------------------------------------
// GELU self-check: the BF16 path's approximation against erff / expf.
// ---------------------------------------------------------------------------
namespace sg {
namespace {

__global__ void gelu_check_kernel(int64_t n, double *__restrict__ eg, double *__restrict__ ed)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = (float)(-12.0 + 24.0 * (double)i / (double)(n - 1));
    float d;
    const float g = gelu_as(v, &d);
    const double Phi = 0.5 * (1.0 + (double)erff(v * 0.70710678118654752f));
    const double gref = (double)v * Phi;
    const double dref = Phi + (double)v * 0.3989422804014327 * (double)expf(-0.5f * v * v);
    eg[i] = fabs((double)g - gref) / fmax(1.0, fabs((double)v));
    ed[i] = fabs((double)d - dref);
}

}  // namespace
}  // namespace sg

extern "C" sg_status sg_gelu_selfcheck(int64_t n, double *max_err_gelu, double *max_err_grad)
{
    using namespace sg;
    if (n < 2 || !max_err_gelu || !max_err_grad) return fail(SG_EINVAL, "n >= 2 and non-NULL outputs");
    double *buf = nullptr;
    SG_CUDA_TRY(cudaMalloc(&buf, 2 * (size_t)n * sizeof(double)));
    gelu_check_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ::sg::counted(nullptr)>>>(n, buf, buf + n);
    std::vector<double> h(2 * (size_t)n);
    const cudaError_t e = cudaMemcpy(h.data(), buf, h.size() * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(SG_ECUDA, cudaGetErrorString(e));
    double mg = 0.0, md = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        mg = std::max(mg, h[(size_t)i]);
        md = std::max(md, h[(size_t)n + (size_t)i]);
    }
    *max_err_gelu = mg;
    *max_err_grad = md;
    return SG_OK;
}
