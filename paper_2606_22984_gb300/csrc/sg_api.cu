// sg_api.cu -- the extern "C" entry points of include/sg.h: argument checks,
// ownership of model / instance memory, and dispatch to the kernel launchers.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sg_internal.cuh"

namespace sg {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void set_error(const std::string &msg) { g_last_error = msg; }

cudaStream_t counted(cudaStream_t st)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return st;
}

sg_status fail(sg_status code, const std::string &msg)
{
    set_error(msg);
    return code;
}

sg_status check_launch(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return SG_OK;
}

sg_status ensure_buffer(void **ptr, size_t *have, size_t need)
{
    if (*have >= need && *ptr) return SG_OK;
    if (*ptr) {
        cudaDeviceSynchronize();
        cudaFree(*ptr);
        *ptr = nullptr;
        *have = 0;
    }
    cudaError_t e = cudaMalloc(ptr, need);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(SG_ENOMEM, "cudaMalloc(" + std::to_string(need) + " bytes) failed: " +
                                   cudaGetErrorString(e));
    }
    *have = need;
    return SG_OK;
}

BlobOff blob_offsets(const sg_config &c)
{
    BlobOff o{};
    const int64_t d = c.d, f = c.d_ff;
    int64_t p = 0;
    const int64_t K = (int64_t)1 << spins_per_token(c), T = c.N / spins_per_token(c);
    o.tok = p; p += K * (int64_t)c.d_token;
    o.pos = p; p += T * (d - c.d_token);
    for (int l = 0; l < c.n_layers; ++l) {
        LayerOff &L = o.L[l];
        L.ln1g = p; p += d;
        L.ln1b = p; p += d;
        L.Wqkv = p; p += 3 * d * d;
        L.bqkv = p; p += 3 * d;
        L.ln2g = p; p += d;
        L.ln2b = p; p += d;
        L.W1 = p; p += f * d;
        L.b1 = p; p += f;
        L.W2 = p; p += d * f;
        L.b2 = p; p += d;
    }
    o.lnfg = p; p += d;
    o.lnfb = p; p += d;
    o.Wh = p; p += K * d;
    o.bh = p; p += K;
    o.total = p;
    return o;
}

PackOff pack_offsets(const sg_config &c)
{
    PackOff o{};
    const int64_t d = c.d, f = c.d_ff;
    int64_t p = 0;
    auto take = [&](int64_t n) { int64_t q = p; p += (n + 3) & ~int64_t(3); return q; };
    for (int l = 0; l < c.n_layers; ++l) {
        o.WqkvT[l] = take(3 * d * d);
        o.W1T[l] = take(d * f);
        o.W2T[l] = take(f * d);
        o.Wqkv[l] = take(3 * d * d);
        o.W1[l] = take(f * d);
        o.W2[l] = take(d * f);
        o.bqkv[l] = take(3 * d);
        o.b1[l] = take(f);
        o.b2[l] = take(d);
    }
    o.total = p;
    return o;
}

static sg_status validate(const sg_config *c)
{
    if (!c) return fail(SG_EINVAL, "config is NULL");
    if (c->N < 1 || c->n_layers < 1 || c->n_layers > SG_MAX_LAYERS || c->d < 4 ||
        c->n_heads < 1 || c->d % c->n_heads || c->d_token < 1 || c->d_token >= c->d ||
        c->d_ff < 1)
        return fail(SG_EINVAL, "invalid model shape (N, n_layers<=16, d, n_heads | d, "
                               "0 < d_token < d, d_ff)");
    if (c->mask_kind != SG_MASK_DENSE && c->mask_kind != SG_MASK_BAND_SINK)
        return fail(SG_EINVAL, "mask_kind must be SG_MASK_DENSE or SG_MASK_BAND_SINK");
    if (c->mask_kind == SG_MASK_BAND_SINK && (c->W < 0 || c->S < 0))
        return fail(SG_EINVAL, "band W and sink S must be >= 0");
    if (c->precision != SG_FP32 && c->precision != SG_BF16)
        return fail(SG_EINVAL, "precision must be SG_FP32 or SG_BF16");
    if (c->n_models < 0 || c->n_models > 64) return fail(SG_EINVAL, "n_models must be in [0, 64]");
    if (c->patch < 0 || c->patch > 8 || (c->patch > 1 && (c->patch & (c->patch - 1))))
        return fail(SG_EINVAL, "patch must be 0, 1, 2, 4 or 8 spins per token");
    const int P = spins_per_token(*c);
    if (P > 1) {
        if (c->lat_D == 0) {
            if (c->N % P) return fail(SG_EINVAL, "N must be a multiple of patch");
        } else {
            int64_t n = 1;
            for (int k = 0; k < c->lat_D; ++k) n *= c->lat_L;
            if (c->lat_D < 1 || c->lat_D > 3 || (1 << c->lat_D) != P || c->lat_L < 2 ||
                c->lat_L % 2 || n != c->N)
                return fail(SG_EINVAL, "patch map needs patch = 2^lat_D, even lat_L, N = lat_L^lat_D");
        }
    }
    return SG_OK;
}

static int models_of(const sg_config &c) { return c.n_models > 1 ? c.n_models : 1; }

// Grouped models in the teacher-forced calls: model mi scores samples
// [mi B/n, (mi+1) B/n).  Each model runs on a view of the group -- its own
// blob and packed FP32 copies, its tiled BF16 weights repacked into the
// group's one buffer -- one after another on the stream, so the repack of
// model mi + 1 is ordered after model mi's kernels.  Buffers a view grows
// belong to the group.
template <class F>
static sg_status for_each_model(sg_model *m, int64_t B, cudaStream_t st, F &&f)
{
    if (m->n_models == 1) return f(m, (int64_t)0, B);
    if (B % m->n_models) return fail(SG_EINVAL, "B must be a multiple of n_models");
    const int64_t Bm = B / m->n_models;
    for (int mi = 0; mi < m->n_models; ++mi) {
        sg_model v = *m;
        v.n_models = 1;
        v.cfg.n_models = 1;
        v.seq.n_models = 1;
        v.P = m->P1;
        v.w = m->w + (size_t)mi * m->P1;
        v.wt = m->wt + (size_t)mi * m->pack.total;
        sg_status s = launch_pack_tiled_weights(&v, st);
        if (s == SG_OK) s = f(&v, mi * Bm, Bm);
        m->ws = v.ws;
        m->ws_bytes = v.ws_bytes;
        m->bt = v.bt;
        m->bt_bytes = v.bt_bytes;
        std::memcpy(m->bt_off, v.bt_off, sizeof(m->bt_off));
        if (s != SG_OK) return s;
    }
    return SG_OK;
}

}  // namespace sg

using namespace sg;

extern "C" {

const char *sg_last_error(void) { return g_last_error.c_str(); }

int64_t sg_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int64_t sg_param_count(const sg_config *cfg)
{
    if (validate(cfg) != SG_OK) return -1;
    return blob_offsets(*cfg).total * models_of(*cfg);
}

sg_status sg_model_create(const sg_config *cfg, const float *weights_host, int64_t n_weights,
                          sg_model **out)
{
    SG_TRY(validate(cfg));
    if (!weights_host || !out) return fail(SG_EINVAL, "NULL weights or out pointer");
    const int64_t P = blob_offsets(*cfg).total * models_of(*cfg);
    if (n_weights != P)
        return fail(SG_EINVAL, "weight blob has " + std::to_string(n_weights) +
                                   " floats, config needs " + std::to_string(P));
    for (int64_t i = 0; i < P; ++i)
        if (!std::isfinite(weights_host[i]))
            return fail(SG_ENUMERIC, "non-finite weight at index " + std::to_string(i));
    sg_model *m = new (std::nothrow) sg_model();
    if (!m) return fail(SG_ENOMEM, "host allocation failed");
    m->cfg = *cfg;
    m->seq = *cfg;
    m->seq.N = cfg->N / spins_per_token(*cfg);
    m->P = P;
    m->n_models = models_of(*cfg);
    m->P1 = P / m->n_models;
    m->off = blob_offsets(*cfg);
    m->pack = pack_offsets(*cfg);
    cudaGetDevice(&m->device);
    size_t have = 0;
    sg_status s = ensure_buffer((void **)&m->w, &have, (size_t)P * sizeof(float));
    have = 0;
    if (s == SG_OK)
        s = ensure_buffer((void **)&m->wt, &have,
                          (size_t)m->pack.total * m->n_models * sizeof(float));
    if (s == SG_OK && cudaMemcpy(m->w, weights_host, (size_t)P * sizeof(float),
                                 cudaMemcpyHostToDevice) != cudaSuccess)
        s = fail(SG_ECUDA, "copying weights to the device failed");
    if (s == SG_OK) s = ensure_buffer(&m->err, &m->err_bytes, sizeof(int));
    if (s == SG_OK && cudaMemset(m->err, 0, sizeof(int)) != cudaSuccess)
        s = fail(SG_ECUDA, "clearing the error word failed");
    if (s == SG_OK) s = sg_model_refresh(m, nullptr);
    if (s == SG_OK && cudaDeviceSynchronize() != cudaSuccess)
        s = fail(SG_ECUDA, "model set-up failed on the device");
    if (s != SG_OK) {
        sg_model_destroy(m);
        return s;
    }
    *out = m;
    return SG_OK;
}

sg_status sg_model_destroy(sg_model *m)
{
    if (!m) return SG_OK;
    cudaDeviceSynchronize();
    cudaFree(m->w);
    cudaFree(m->wt);
    cudaFree(m->bf);
    cudaFree(m->kv);
    cudaFree(m->ws);
    cudaFree(m->err);
    delete m;
    return SG_OK;
}

float *sg_model_weights(sg_model *m) { return m ? m->w : nullptr; }

sg_status sg_model_refresh(sg_model *m, sg_stream stream)
{
    if (!m) return fail(SG_EINVAL, "NULL model");
    SG_TRY(launch_pack_f32(m, (cudaStream_t)stream));
    if (m->cfg.precision == SG_BF16) {
        SG_TRY(launch_pack_bf16(m, (cudaStream_t)stream));
        SG_TRY(launch_pack_tiled_weights(m, (cudaStream_t)stream));
    }
    return SG_OK;
}

sg_status sg_model_check(sg_model *m, sg_stream stream)
{
    if (!m) return fail(SG_EINVAL, "NULL model");
    SG_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int e = 0;
    SG_CUDA_TRY(cudaMemcpy(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!e) return SG_OK;
    SG_CUDA_TRY(cudaMemset(m->err, 0, sizeof(int)));
    if (e & 4) return fail(SG_ENUMERIC, "a kernel produced a non-finite logit");
    return fail(SG_ECUDA, "a kernel gave up a bounded wait (code " + std::to_string(e) +
                              "); its outputs are not valid");
}

sg_status sg_model_set_max_chunk(sg_model *m, int64_t max_samples)
{
    if (!m) return fail(SG_EINVAL, "NULL model");
    if (max_samples < 0) return fail(SG_EINVAL, "max_samples must be >= 0");
    m->max_chunk = max_samples;
    return SG_OK;
}

sg_status sg_model_reserve(sg_model *m, int64_t B)
{
    if (!m) return fail(SG_EINVAL, "NULL model");
    if (B < 1 || B >= (int64_t)1 << 32) return fail(SG_EINVAL, "B must be in [1, 2^32)");
    if (m->n_models > 1 && B % m->n_models)
        return fail(SG_EINVAL, "B must be a multiple of n_models");
    const size_t need = m->cfg.precision == SG_BF16 ? decode_bf16_layout(m, B, nullptr, nullptr, nullptr)
                                                    : decode_f32_kv_bytes(m, B);
    return ensure_buffer(&m->kv, &m->kv_bytes, need);
}

sg_status sg_sample(sg_model *m, int64_t B, double beta, uint64_t seed, uint32_t stream_id,
                    float flag_band, int8_t *spins, float *logq, uint32_t *flags, sg_stream stream)
{
    (void)beta;
    if (!m || !spins || !logq) return fail(SG_EINVAL, "NULL model or output");
    if (B < 1 || B >= (int64_t)1 << 32) return fail(SG_EINVAL, "B must be in [1, 2^32)");
    if (m->n_models > 1 && B % m->n_models)
        return fail(SG_EINVAL, "B must be a multiple of n_models");
    if (m->n_models > 1 && !(m->cfg.precision == SG_BF16 && m->cfg.d == 256))
        return fail(SG_EUNSUPPORTED, "grouped models are served by the BF16 d = 256 decode");
    if (flag_band <= 0.f) flag_band = m->cfg.precision == SG_BF16 ? 1e-2f : 1e-5f;
    cudaStream_t st = (cudaStream_t)stream;
    if (flags)
        SG_CUDA_TRY(cudaMemsetAsync(flags, 0,
                                    (size_t)B * ((m->seq.N + 31) / 32) * sizeof(uint32_t), st));
    if (m->cfg.precision == SG_BF16)
        return launch_decode_bf16(m, B, seed, stream_id, flag_band, spins, logq, flags, st);
    return launch_decode_f32(m, B, seed, stream_id, flag_band, spins, logq, flags, st);
}

sg_status sg_logprob(sg_model *m, const int8_t *spins, int64_t B, float *logq, sg_stream stream)
{
    if (!m || !spins || !logq) return fail(SG_EINVAL, "NULL model or pointer");
    if (B < 1) return fail(SG_EINVAL, "B must be >= 1");
    const cudaStream_t st = (cudaStream_t)stream;
    const int64_t N = m->cfg.N;
    return for_each_model(m, B, st, [&](sg_model *v, int64_t b0, int64_t Bm) {
        return launch_logprob_f32(v, spins + b0 * N, Bm, logq + b0, st);
    });
}

sg_status sg_grad(sg_model *m, const int8_t *spins, const float *coeff, int64_t B, float *grad,
                  float *logq, sg_stream stream)
{
    if (!m || !spins || !coeff || !grad) return fail(SG_EINVAL, "NULL model or pointer");
    if (B < 1) return fail(SG_EINVAL, "B must be >= 1");
    const cudaStream_t st = (cudaStream_t)stream;
    const int64_t N = m->cfg.N;
    return for_each_model(m, B, st, [&](sg_model *v, int64_t b0, int64_t Bm) {
        return launch_grad_f32(v, spins + b0 * N, coeff + b0, Bm, grad + (b0 / Bm) * m->P1,
                               logq ? logq + b0 : nullptr, st);
    });
}

sg_status sg_instance_create(int32_t kind, int32_t N, int32_t D, int32_t L, int32_t periodic,
                             const float *J_host, sg_instance **out)
{
    if (!J_host || !out) return fail(SG_EINVAL, "NULL J or out pointer");
    size_t nJ = 0;
    if (kind == SG_SK_DENSE) {
        if (N < 2) return fail(SG_EINVAL, "SK needs N >= 2");
        nJ = (size_t)N * N;
        for (int i = 0; i < N; ++i) {
            if (J_host[(size_t)i * N + i] != 0.f)
                return fail(SG_EINVAL, "SK coupling matrix must have a zero diagonal");
            for (int j = 0; j < i; ++j)
                if (J_host[(size_t)i * N + j] != J_host[(size_t)j * N + i])
                    return fail(SG_EINVAL, "SK coupling matrix must be symmetric");
        }
    } else if (kind == SG_EA_LATTICE) {
        if (D < 1 || D > 3 || L < 2) return fail(SG_EINVAL, "EA needs 1 <= D <= 3 and L >= 2");
        int64_t n = 1;
        for (int k = 0; k < D; ++k) n *= L;
        if (n != N) return fail(SG_EINVAL, "EA needs N == L^D");
        nJ = (size_t)N * D;
    } else {
        return fail(SG_EINVAL, "kind must be SG_SK_DENSE or SG_EA_LATTICE");
    }
    for (size_t i = 0; i < nJ; ++i)
        if (!std::isfinite(J_host[i])) return fail(SG_ENUMERIC, "non-finite coupling");
    sg_instance *inst = new (std::nothrow) sg_instance();
    if (!inst) return fail(SG_ENOMEM, "host allocation failed");
    inst->kind = kind;
    inst->N = N;
    inst->D = D;
    inst->L = L;
    inst->periodic = periodic ? 1 : 0;
    inst->integer_bonds = false;
    size_t have = 0;
    sg_status s = ensure_buffer((void **)&inst->J, &have, nJ * sizeof(float));
    if (s == SG_OK && cudaMemcpy(inst->J, J_host, nJ * sizeof(float), cudaMemcpyHostToDevice) !=
                          cudaSuccess)
        s = fail(SG_ECUDA, "copying couplings failed");
    if (s == SG_OK && kind == SG_EA_LATTICE) {
        bool integer = true;
        for (size_t i = 0; i < nJ && integer; ++i)
            integer = J_host[i] == std::floor(J_host[i]) && std::fabs(J_host[i]) <= 127.f;
        if (integer) {
            std::vector<int8_t> b(nJ);
            for (size_t i = 0; i < nJ; ++i) b[i] = (int8_t)J_host[i];
            have = 0;
            s = ensure_buffer((void **)&inst->Ji8, &have, nJ);
            if (s == SG_OK &&
                cudaMemcpy(inst->Ji8, b.data(), nJ, cudaMemcpyHostToDevice) != cudaSuccess)
                s = fail(SG_ECUDA, "copying integer bonds failed");
            inst->integer_bonds = s == SG_OK;
        }
    }
    have = 0;
    if (s == SG_OK) s = ensure_buffer(&inst->err, &have, sizeof(int));
    if (s == SG_OK && cudaMemset(inst->err, 0, sizeof(int)) != cudaSuccess)
        s = fail(SG_ECUDA, "clearing the error word failed");
    if (s == SG_OK && kind == SG_SK_DENSE) s = prepare_sk_tc(inst);
    if (s != SG_OK) {
        sg_instance_destroy(inst);
        return s;
    }
    *out = inst;
    return SG_OK;
}

sg_status sg_instance_destroy(sg_instance *inst)
{
    if (!inst) return SG_OK;
    cudaDeviceSynchronize();
    cudaFree(inst->J);
    cudaFree(inst->Ji8);
    cudaFree(inst->Jbf);
    cudaFree(inst->ws);
    cudaFree(inst->err);
    delete inst;
    return SG_OK;
}

sg_status sg_energy(const sg_instance *inst, const int8_t *spins, int64_t B, int32_t precision,
                    float *E, int32_t *E_int, sg_stream stream)
{
    if (!inst || !spins || !E) return fail(SG_EINVAL, "NULL instance or pointer");
    if (B < 1) return fail(SG_EINVAL, "B must be >= 1");
    if (E_int && !(inst->kind == SG_EA_LATTICE && inst->integer_bonds))
        return fail(SG_EINVAL, "integer energies need an EA instance with integer bonds");
    return launch_energy(inst, spins, B, precision, E, E_int, (cudaStream_t)stream);
}

sg_status sg_free_energy(const float *E, const float *logq, int64_t B, double beta, double *out,
                         float *coeff, sg_stream stream)
{
    if (!E || !logq || !out) return fail(SG_EINVAL, "NULL pointer");
    if (B < 1) return fail(SG_EINVAL, "B must be >= 1");
    if (!(beta > 0.0) || !std::isfinite(beta)) return fail(SG_EINVAL, "beta must be > 0");
    return launch_free_energy(E, logq, B, beta, out, coeff, (cudaStream_t)stream);
}

sg_status sg_loss_coeff(const float *E, const float *logq, int64_t B, double a, double c,
                        double w, double *mean, float *coeff, sg_stream stream)
{
    if (!E || !logq || !coeff) return fail(SG_EINVAL, "NULL pointer");
    if (B < 1) return fail(SG_EINVAL, "B must be >= 1");
    if (!std::isfinite(a) || !std::isfinite(c) || !std::isfinite(w))
        return fail(SG_EINVAL, "a, c and w must be finite");
    return launch_loss_coeff(E, logq, B, a, c, w, mean, coeff, (cudaStream_t)stream);
}

sg_status sg_mh_step(const int8_t *prop_spins, const float *E, const float *logq, int64_t B,
                     int32_t N, int32_t C, double beta, uint64_t seed, int8_t *chain_spins,
                     double *chain_E, double *chain_lq, int64_t *accepts, float *trace_E,
                     sg_stream stream)
{
    if (!prop_spins || !E || !logq || !chain_spins || !chain_E || !chain_lq || !accepts)
        return fail(SG_EINVAL, "NULL pointer");
    if (C < 1 || B < C || B % C) return fail(SG_EINVAL, "need C >= 1 and B a multiple of C");
    if (N < 1) return fail(SG_EINVAL, "N must be >= 1");
    return launch_mh(prop_spins, E, logq, B, N, C, beta, seed, chain_spins, chain_E, chain_lq,
                     accepts, trace_E, (cudaStream_t)stream);
}

sg_status sg_metropolis(const sg_instance *inst, int8_t *spins, int64_t R, int32_t sweeps,
                        double beta, uint64_t seed, double *E, float *trace_E, sg_stream stream)
{
    if (!inst || !spins || !E) return fail(SG_EINVAL, "NULL pointer");
    if (R < 1 || sweeps < 0) return fail(SG_EINVAL, "need R >= 1 and sweeps >= 0");
    return launch_metropolis(inst, spins, R, sweeps, beta, seed, E, trace_E,
                             (cudaStream_t)stream);
}

sg_status sg_overlap_hist(const int8_t *spins, int64_t B, int32_t N, int64_t *hist,
                          sg_stream stream)
{
    if (!spins || !hist || B < 2 || N < 1) return fail(SG_EINVAL, "bad overlap arguments");
    return launch_overlap(spins, B, N, hist, (cudaStream_t)stream);
}

sg_status sg_adam_step(float *w, const float *g, float *m, float *v, int64_t n, float lr,
                       float beta1, float beta2, float eps, int64_t step, sg_stream stream)
{
    if (!w || !g || !m || !v || n < 1 || step < 1) return fail(SG_EINVAL, "bad Adam arguments");
    return launch_adam(w, g, m, v, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream);
}

}  // extern "C"
