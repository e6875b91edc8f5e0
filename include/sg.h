/*
 * sg.h -- C ABI of libsg, the GB300 (sm_103a) implementation of the FlashVAN
 * hot path (arXiv 2606.22984, "Scalable Physics-Inspired Transformers for
 * Spin Glasses"): batched ancestral sampling from the autoregressive
 * transformer, teacher-forced log q, Ising energies, variational and
 * importance-weighted free energies, the REINFORCE gradient and neural
 * Metropolis-Hastings.
 *
 * Conventions for every entry point
 *   - Plain pointers and sizes only.  "dev" pointers are CUDA device memory
 *     owned by the caller unless stated otherwise; "host" pointers are host
 *     memory read during the call.
 *   - sg_stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream only enqueue work on it and return
 *     without synchronising, unless stated otherwise.
 *   - Spins are int8 with values -1 / +1, row-major [B][N] (sample-major).
 *   - Every call returns an sg_status; on failure nothing is written to the
 *     outputs that the caller can rely on and sg_last_error() describes the
 *     cause (a per-thread string, valid until the next failing call).  No C++
 *     exception crosses this boundary.
 *   - Random numbers: the counter-based Philox4x32-10 generator (Salmon et
 *     al., SC'11) keyed by the 64-bit seed; the uniform of counter
 *     (a, b, stream, e) is ((x0 >> 8) + 0.5) * 2^-24.
 *
 * Weight blob (sg_param_count floats), row-major, linear maps "out x in";
 * K = 2^P token classes and T = N / P tokens (K = 2, T = N without patching):
 *   tok[K][d_token]  pos[T][d - d_token]
 *   per layer: ln1_g[d] ln1_b[d] Wqkv[3d][d] bqkv[3d] ln2_g[d] ln2_b[d]
 *              W1[d_ff][d] b1[d_ff] W2[d][d_ff] b2[d]
 *   lnf_g[d] lnf_b[d] Wh[K][d] bh[K]
 * Rows of Wqkv: queries, keys, values, each head-major (head h owns
 * columns h*d_h .. h*d_h + d_h - 1 of its block).
 */
#ifndef SG_H
#define SG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void *sg_stream;

typedef enum {
    SG_OK = 0,
    SG_EINVAL = 1,       /* bad argument, shape or configuration            */
    SG_ENOMEM = 2,       /* device or host allocation failed                */
    SG_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed     */
    SG_ENUMERIC = 4,     /* NaN / Inf seen where a finite value is required */
    SG_EUNSUPPORTED = 5  /* valid configuration the library does not serve  */
} sg_status;

typedef enum { SG_MASK_DENSE = 0, SG_MASK_BAND_SINK = 1 } sg_mask_kind;
typedef enum { SG_FP32 = 0, SG_BF16 = 1 } sg_precision;
typedef enum { SG_SK_DENSE = 0, SG_EA_LATTICE = 1 } sg_instance_kind;

/*
 * Model configuration (paper: "Overall architecture", Eq. concatePE,
 * Algorithm 2, SI Sec. I.A; hyper-parameter names of the SI symbol table).
 *   N          spins = sequence length.
 *   n_layers   decoder layers (pre-LayerNorm attention and FFN sublayers,
 *              Algorithm 2).
 *   d          model width, d = d_token + d_pos (Eq. concatePE).
 *   n_heads    heads; d_h = d / n_heads; no output projection W_O.
 *   d_token    token-embedding width (2 in the paper).
 *   d_ff       FFN hidden width (GELU).
 *   mask_kind  SG_MASK_DENSE: causal.  SG_MASK_BAND_SINK: query t sees key k
 *              iff k <= t and (t - k <= W or k < S) -- the sliding window
 *              A_tk = 0 for t - k > W of SI Sec. I.A plus a sink of the first
 *              S keys (start token and first lattice row / plane, reached by
 *              the periodic wrap).
 *   precision  SG_FP32: every step in FP32 on CUDA cores ("FP32 plain").
 *              SG_BF16: GEMMs on tcgen05 tensor cores with BF16 operands and
 *              FP32 accumulation, BF16 KV cache; LayerNorm, softmax, residual
 *              stream and the draw stay FP32.
 *   n_models   0 or 1: one model.  n > 1: a group of n models of this shape
 *              (e.g. one per temperature), weight blobs concatenated; in
 *              sg_sample, sg_logprob and sg_grad, sample b of B (B a multiple
 *              of n) belongs to model b / (B / n).  Grouped sampling is served
 *              by the BF16 decode for d = 256 (other shapes return
 *              SG_EUNSUPPORTED); sg_logprob and sg_grad serve groups of any
 *              shape they serve singly; sg_muon_step does not.
 *   patch      spins per token P (patching, Methods: the EA lattice cut into
 *              cells of 2^D spins, one token per cell).  0 or 1: one spin per
 *              token.  P > 1: the head is a softmax over K = 2^P classes and
 *              the draw is categorical, class k chosen by the inverse CDF of
 *              the uniform (classes in index order); token = sum_j bit_j 2^j,
 *              bit_j = (s + 1) / 2 of the cell's j-th spin.  W, S count tokens.
 *   lat_D, lat_L  the patch map: lat_D = 0: token t holds spins tP .. tP+P-1;
 *              lat_D > 0 (P = 2^lat_D, even lat_L, N = lat_L^lat_D): tokens are
 *              the cells of the lattice in raster order of the cell grid, bit
 *              j at offset (j & 1, (j >> 1) & 1, ...) from the cell's even
 *              corner (x0 fastest).  Spins stay in lattice raster order.
 *              Patched models are served by the FP32 decode, the BF16
 *              decodes (2D and 3D cells, K up to 256; d = 64, 128, 256,
 *              grouped d = 256 included; at d = 64 with d_token <= 16, else
 *              SG_EUNSUPPORTED) and the teacher-forced pass.
 * Key position k holds the token of position k-1; key 0 holds the start token 0.
 */
typedef struct {
    int32_t N, n_layers, d, n_heads, d_token, d_ff;
    int32_t mask_kind, W, S;
    int32_t precision;
    int32_t n_models;
    int32_t patch, lat_D, lat_L;
} sg_config;

typedef struct sg_model sg_model;
typedef struct sg_instance sg_instance;

/* Human-readable description of the last failure on this thread. */
const char *sg_last_error(void);

/* Number of CUDA kernels this library has launched in this process (host
 * counter, all threads and devices); used to report launches per step. */
int64_t sg_launch_count(void);

/* Number of floats in the weight blob of cfg (all n_models blobs), or -1 if
 * cfg is invalid. */
int64_t sg_param_count(const sg_config *cfg);

/*
 * Create a model from a host weight blob of n_weights floats (layout above).
 * The library copies the weights to the current device and owns them, plus
 * the packed per-kernel layouts derived from them and the KV-cache
 * workspace (grown on demand by sg_sample).  Errors: SG_EINVAL (cfg or
 * n_weights), SG_EUNSUPPORTED, SG_ENOMEM, SG_ECUDA.  Synchronous.
 */
sg_status sg_model_create(const sg_config *cfg, const float *weights_host, int64_t n_weights,
                          sg_model **out);

/* Free every device buffer the model owns (synchronises the device). */
sg_status sg_model_destroy(sg_model *m);

/* Device pointer to the model's FP32 master weight blob (sg_param_count
 * floats, layout above).  The caller may update it in place on a stream
 * (e.g. with sg_adam_step) and must then call sg_model_refresh on that
 * stream before the next sampling or scoring call. */
float *sg_model_weights(sg_model *m);

/* Re-derive the packed kernel layouts from the master blob, on stream. */
sg_status sg_model_refresh(sg_model *m, sg_stream stream);

/*
 * Synchronise stream and report the model's device error word, which kernels
 * set instead of hanging or trapping: SG_ECUDA when a bounded wait inside a
 * kernel gave up (the kernel stopped early; its outputs are invalid),
 * SG_ENUMERIC when a non-finite logit was produced.  The word is cleared.
 */
sg_status sg_model_check(sg_model *m, sg_stream stream);

/*
 * Cap the samples per chunk of the teacher-forced pass and its backward
 * (sg_logprob, sg_grad).  Those calls keep every layer's activations of a
 * chunk of samples on the device, which is how batches whose activations
 * outgrow device memory are trained (the paper recomputes activations for
 * its large systems); by default (max_samples = 0) a chunk is sized
 * to a third of the free device memory, at most 64 GB.  A cap bounds the
 * workspace further; results do not depend on the chunking beyond FP32
 * summation order.  Errors: SG_EINVAL (NULL model, max_samples < 0).
 */
sg_status sg_model_set_max_chunk(sg_model *m, int64_t max_samples);

/*
 * Size the model's KV-cache workspace for sampling B configurations now, so
 * that the next sg_sample calls of at most B samples allocate nothing (the
 * workspace of Algorithm 2's KV cache; sg_sample otherwise grows it on
 * demand).  Synchronous; may free and re-allocate the workspace, so no
 * sampling call of this model may be in flight.
 * Errors: SG_EINVAL (NULL model, B outside [1, 2^32), B not a multiple of
 * n_models), SG_ENOMEM.
 */
sg_status sg_model_reserve(sg_model *m, int64_t B);

/*
 * Batched ancestral sampling (Algorithm 2, KV-cache decode) of B
 * configurations in one persistent kernel launch.
 *   spins  dev int8 [B][N]   out: sampled spins.
 *   logq   dev float [B]     out: log q(sigma) = sum_t log sigmoid(sigma_t l_t).
 *   flags  dev uint32 [B][(T+31)/32] or NULL   out: bit t set where the draw
 *          of token position t was flagged, |p+ - u| < flag_band (patched:
 *          u within flag_band of a boundary of the cumulative class
 *          probabilities); flag_band <= 0 selects 1e-5 for FP32 and 1e-2 for
 *          BF16.  T = N / patch (T = N without patching).
 * Sample b, step t uses u = uniform(seed, counter (b, t, stream_id, 0)) and
 * takes sigma_t = +1 iff u < p+ = sigmoid(l_t), l_t = z1 - z0 of the output
 * head.  beta is recorded only (sampling does not depend on it).
 * Errors: SG_EINVAL (B < 1, B >= 2^32, NULL outputs), SG_ENOMEM, SG_ECUDA.
 */
sg_status sg_sample(sg_model *m, int64_t B, double beta, uint64_t seed, uint32_t stream_id,
                    float flag_band, int8_t *spins, float *logq, uint32_t *flags,
                    sg_stream stream);

/*
 * Allocation-free variant of sg_sample (FP32 path).  The paper has no
 * counterpart: this entry point exists for callers that must not let a
 * library allocate device memory -- code embedded in a host framework that
 * owns every device allocation through its own memory pool (memory the pool
 * did not hand out is memory it cannot budget), or latency-sensitive loops in
 * which cudaMalloc / cudaFree would synchronise the device and stall its other
 * streams.  It calls no cudaMalloc, cudaFree or allocating library routine.  Its scratch (packed weight copies followed by
 * the KV cache) is one statically sized device array of
 * SG_NOALLOC_SCRATCH_BYTES inside libsg, which every GPU that loads the
 * library holds until the process exits.
 *   cfg      model configuration (precision must be SG_FP32).
 *   weights  dev float [sg_param_count(cfg)]: the caller's weight blob.
 *   spins, logq, flags, seed, stream_id, flag_band: as for sg_sample.
 * Errors: SG_EINVAL when cfg is invalid or when the packed weights plus the
 * KV cache of B samples exceed SG_NOALLOC_SCRATCH_BYTES (reduce B, or use
 * sg_sample); SG_EUNSUPPORTED for shapes the FP32 decode is not built for.
 * Every call looks up the scratch's address in the current device context
 * (cudaGetSymbolAddress, a host-side lookup), so the entry point stays valid
 * across a cudaDeviceReset.  Every call shares the one scratch array and it
 * keeps the last call's contents; nothing in it needs to start at zero,
 * because each call writes every byte it reads.  Calls whose work overlaps on
 * the GPU (other streams, other host threads) race on the scratch: serialise
 * them.
 */
#define SG_NOALLOC_SCRATCH_BYTES (64ull << 20)
sg_status sg_sample_noalloc(const sg_config *cfg, const float *weights, int64_t B, double beta,
                            uint64_t seed, uint32_t stream_id, float flag_band, int8_t *spins,
                            float *logq, uint32_t *flags, sg_stream stream);

/*
 * Teacher-forced log q (Algorithm 1) of B given configurations, computed over
 * the whole sequence at once (prefill).
 *   spins  dev int8 [B][N] in;  logq dev float [B] out.
 * Grouped models: sample b is scored by model b / (B / n_models).
 * Errors: SG_EINVAL (also B not a multiple of n_models), SG_ENOMEM, SG_ECUDA.
 */
sg_status sg_logprob(sg_model *m, const int8_t *spins, int64_t B, float *logq, sg_stream stream);

/*
 * REINFORCE gradient (Eq. loss1): grad = sum_b coeff[b] * d log q(sigma_b)/d theta,
 * with activations recomputed per chunk of samples.  With
 * coeff[b] = (L_b - Lbar)/B, L = beta E + ln q, this is the paper's
 * estimator of beta * grad F_q.
 *   spins  dev int8 [B][N];  coeff dev float [B];
 *   grad   dev float [sg_param_count] out (overwritten, blob layout);
 *   logq   dev float [B] or NULL: out, the teacher-forced log q.
 * Grouped models: samples [i B/n, (i+1) B/n) belong to model i and their
 * gradient fills model i's block of grad (blobs concatenated like the
 * weights); the models run one after another on the stream.
 * Errors: SG_EINVAL (also B not a multiple of n_models), SG_ENOMEM, SG_ECUDA.
 */
sg_status sg_grad(sg_model *m, const int8_t *spins, const float *coeff, int64_t B, float *grad,
                  float *logq, sg_stream stream);

/*
 * Problem instance (Eqs. SKHam, EAHam).  kind SG_SK_DENSE: J_host is the
 * dense symmetric N x N float matrix with zero diagonal, E = -sum_{i<j} J_ij
 * s_i s_j (the paper's 1/sqrt(N) folded into J).  kind SG_EA_LATTICE: N =
 * L^D, J_host holds bonds[N][D], bonds[i][mu] coupling raster site
 * i = x0 + L x1 + L^2 x2 to its +mu neighbour (periodic wrap, or no bond
 * across the edge when periodic = 0); E = -sum_i sum_mu bonds[i][mu] s_i s_(i+mu).
 * The library copies J to the device and owns it.  Synchronous.
 */
sg_status sg_instance_create(int32_t kind, int32_t N, int32_t D, int32_t L, int32_t periodic,
                             const float *J_host, sg_instance **out);
sg_status sg_instance_destroy(sg_instance *inst);

/*
 * Energies of B configurations.
 *   E      dev float [B] out.
 *   E_int  dev int32 [B] or NULL: exact integer energies, only for EA
 *          instances whose bonds are all integers (else SG_EINVAL).
 *   spins  dev int8 [B][N], values +-1.
 * precision SG_BF16 on an SK instance with N a multiple of 256 runs the
 * s.J.s contraction on tcgen05 tensor cores (J split into two BF16 terms,
 * FP32 accumulation; other N use CUDA cores); SG_FP32 uses CUDA cores.  The
 * tensor-core path adds the partial sums of E_b by FP32 atomics, so E is not
 * bit-reproducible from call to call (FP32 rounding order).  Its spins are
 * read in 16-byte pieces when the pointer is 16-byte aligned; otherwise a
 * BF16 copy of them (2 B N bytes, in the instance's workspace) is written
 * first.  EA is a coalesced neighbour gather either way.
 */
sg_status sg_energy(const sg_instance *inst, const int8_t *spins, int64_t B, int32_t precision,
                    float *E, int32_t *E_int, sg_stream stream);

/*
 * Free energies from one batch (Eqs. KL_div, free_energy), reduced in FP64
 * on the device:  L_b = beta E_b + ln q_b;
 *   out[0] = F_q  = mean(L) / beta,
 *   out[1] = F_IS = -(1/beta) [ln sum_b exp(-L_b) - ln B],
 *   out[2] = Kish ESS = (sum w)^2 / sum w^2, w_b = exp(-L_b - max(-L)).
 *   out    dev double [3].
 *   coeff  dev float [B] or NULL: (L_b - mean L) / B, the REINFORCE weights.
 */
sg_status sg_free_energy(const float *E, const float *logq, int64_t B, double beta, double *out,
                         float *coeff, sg_stream stream);

/*
 * REINFORCE weights of a general per-sample loss, reduced in FP64 on the
 * device:  L_b = a E_b + c ln q_b,  coeff_b = (L_b - mean L - w) / B,
 * so that sg_grad with these weights gives (1/B) sum_b (L_b - mean L) grad ln q
 * - (w/B) sum_b grad ln q.  The cases:
 *   (a, c, w) = (beta, 1, 0)  Eq. loss1, the free energy F_q;
 *   (a, c, w) = (1, T, 0)     the ground-state form of Methods "Variational
 *                             annealing", L = E + T ln q, which stays
 *                             bounded as T -> 0;
 *   w > 0                     Eq. loss2, the likelihood (self-distillation)
 *                             term on configurations refined by local Monte
 *                             Carlo before scoring.
 *   E, logq dev float [B]; coeff dev float [B] out;
 *   mean    dev double [2] out or NULL: mean L, mean E.
 * Errors: SG_EINVAL on NULL inputs, B < 1 or non-finite a, c, w.
 */
sg_status sg_loss_coeff(const float *E, const float *logq, int64_t B, double a, double c,
                        double w, double *mean, float *coeff, sg_stream stream);

/*
 * Independence Metropolis-Hastings with the model as proposal (the paper's
 * Monte Carlo + generative-model combination; not an algorithm it prints).
 * Chain c (of C, B % C == 0) consumes proposals p = j*C + c, j = 0..B/C-1,
 * in order: log alpha = (-beta E_p - ln q_p) - (-beta E_c - ln q_c) in
 * FP64; accept iff ln u < log alpha, u = uniform(seed, (c, j, 1, 0)).
 *   prop_spins dev int8 [B][N]; E, logq dev float [B];
 *   chain_spins dev int8 [C][N], chain_E, chain_lq dev double [C]: in/out state;
 *   accepts dev int64 [C] out (acceptances in this call);
 *   trace_E dev float [B/C][C] or NULL: chain energy after each proposal.
 */
sg_status sg_mh_step(const int8_t *prop_spins, const float *E, const float *logq, int64_t B,
                     int32_t N, int32_t C, double beta, uint64_t seed, int8_t *chain_spins,
                     double *chain_E, double *chain_lq, int64_t *accepts, float *trace_E,
                     sg_stream stream);

/*
 * Single-spin-flip Metropolis (the paper's local Monte Carlo refinement and
 * the classical reference).  Replica r, sweep w visits sites i = 0..N-1 in
 * order; dE = 2 s_i h_i; accept iff u < exp(-beta dE) in FP64,
 * u = uniform(seed, (r, i, 2, w)).
 *   spins dev int8 [R][N] in/out;  E dev double [R] in/out (energy of spins);
 *   trace_E dev float [sweeps][R] or NULL: energy after each sweep.
 */
sg_status sg_metropolis(const sg_instance *inst, int8_t *spins, int64_t R, int32_t sweeps,
                        double beta, uint64_t seed, double *E, float *trace_E, sg_stream stream);

/*
 * Overlap histogram (Eq. overlap_distribution): q = s1.s2 / N for pairs
 * (2k, 2k+1); hist dev int64 [N+1] out, bin (N q + N)/2.
 */
sg_status sg_overlap_hist(const int8_t *spins, int64_t B, int32_t N, int64_t *hist,
                          sg_stream stream);

/*
 * Adam update (the minimal optimiser of the training loop; the paper's Muon
 * is a later addition): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * w -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * All arrays dev float [n]; step >= 1.
 */
sg_status sg_adam_step(float *w, const float *g, float *m, float *v, int64_t n, float lr,
                       float beta1, float beta2, float eps, int64_t step, sg_stream stream);

/*
 * Muon update of a model's weight blob (Methods "Comparison on optimizers":
 * the optimiser of Jordan et al. 2024 with the weight decay and RMS alignment
 * of Liu et al. 2025).  For each weight matrix (per layer Wqkv [3d][d],
 * W1 [d_ff][d], W2 [d][d_ff]) with gradient G:
 *   M = mu M + G;  O = NS(M);  W -= lr (0.2 sqrt(max(rows, cols)) O + wd W),
 * NS = ns_steps quintic Newton-Schulz steps on X = M / (|M|_F + 1e-7), taken
 * on M^T when rows > cols: X <- a X + (b A + c A A) X, A = X X^T,
 * (a, b, c) = (3.4445, -4.7750, 2.0315).  Every other parameter (embeddings,
 * LayerNorm gains and biases, biases, output head) takes an AdamW step
 * (beta1 0.9, beta2 0.999, eps 1e-8, same lr, decoupled decay wd).
 *   weights, grad, momentum, adam_m, adam_v: dev float [sg_param_count];
 *   momentum is used on the matrix entries, adam_m/adam_v on the others;
 *   step >= 1 (AdamW bias correction); 0 <= ns_steps <= 32.
 * Scratch is the model's workspace.  Errors: SG_EINVAL (pointers, values),
 * SG_EUNSUPPORTED (grouped models).  The paper prints no counterpart of the
 * AdamW split; it is the usual practice for the non-matrix parameters.
 */
sg_status sg_muon_step(sg_model *m, float *weights, const float *grad, float *momentum,
                       float *adam_m, float *adam_v, double lr, double mu, double weight_decay,
                       int32_t ns_steps, int64_t step, sg_stream stream);

/*
 * Self-check of the GELU the BF16 path evaluates (the "GELU" of the
 * architecture, Methods "Overall architecture"; erf form): the approximation
 * of erf by Abramowitz & Stegun formula 7.1.26 against CUDA's erff and expf,
 * on the current device, over n points evenly spaced in [-12, 12] (n >= 2).
 *   max_err_gelu: max |gelu_approx(v) - v (1 + erff(v / sqrt 2)) / 2| / max(1, |v|)
 *   max_err_grad: max |gelu'_approx(v) - (Phi(v) + v expf(-v^2 / 2) / sqrt(2 pi))|
 * (host doubles).  Synchronous.  Errors: SG_EINVAL (n < 2 or NULL), SG_ECUDA.
 */
sg_status sg_gelu_selfcheck(int64_t n, double *max_err_gelu, double *max_err_grad);

#ifdef __cplusplus
}
#endif

#endif /* SG_H */
