/*
 * sg_oracle.c -- plain, slow FP64 CPU oracle for the FlashVAN hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the tests, the package smoke check and the benchmark's CPU-baseline
 * leg load it.  It shares no code, header, table or helper with the CUDA
 * library; both sides read the same documented weight-blob layout and the
 * same seeded inputs, and each implements the counter-based Philox4x32-10
 * generator on its own from its published definition.
 *
 * Every function cites the passage of the paper (arXiv 2606.22984,
 * "Scalable Physics-Inspired Transformers for Spin Glasses") it follows.
 * Where the paper is silent the documented reading is stated beside the
 * code.  All floating point is double; no blocking, fusion or reordering
 * beyond the definitions.
 *
 * Philox4x32-10 is pinned word for word against PyTorch's independent
 * header-only engine (at::philox_engine) by the CPU tests, besides its
 * statistical checks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Configuration (mirrors the documented C-ABI config field by field, but is */
/* declared here on its own).                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t N;          /* spins = sequence length                         */
    int32_t n_layers;   /* decoder layers                                  */
    int32_t d;          /* model width d = d_token + d_pos                 */
    int32_t n_heads;    /* attention heads, d_h = d / n_heads              */
    int32_t d_token;    /* token-embedding width (2 in the paper)          */
    int32_t d_ff;       /* FFN hidden width                                */
    int32_t mask_kind;  /* 0 = dense causal, 1 = sliding band + sink       */
    int32_t W;          /* band: key k visible to query t iff t-k <= W     */
    int32_t S;          /* sink: keys k < S always visible                 */
    int32_t patch;      /* spins per token P (0 or 1: one spin per token)  */
    int32_t lat_D;      /* lattice dimension for the patch map (0: chain)  */
    int32_t lat_L;      /* lattice side                                     */
} or_cfg;

/* ------------------------------------------------------------------------ */
/* Patching (Methods / SI: the EA lattice is cut into non-overlapping        */
/* patches of 2^D spins, one token per patch, sequence length (L/2)^D).      */
/* Readings: patches in raster order of the patch grid; bit j of a token is  */
/* the spin at offset delta = (j & 1, (j >> 1) & 1, ...) from the patch's    */
/* even corner (x0 fastest), value (sigma + 1) / 2; token = sum_j bit_j 2^j; */
/* the head is a softmax over K = 2^P classes; without a lattice, token t    */
/* holds spins tP .. tP + P - 1.  P = 1 is the unpatched model.               */
/* ------------------------------------------------------------------------ */
static int n_spt(const or_cfg *c) { return c->patch > 1 ? c->patch : 1; }
static int n_tok(const or_cfg *c) { return c->N / n_spt(c); }
static int n_cls(const or_cfg *c) { return 1 << n_spt(c); }

/* site (raster index) of bit j of token t */
static int patch_site(const or_cfg *c, int t, int j)
{
    const int P = n_spt(c);
    if (P == 1) return t;
    if (c->lat_D == 0) return t * P + j;
    const int D = c->lat_D, L = c->lat_L, M = L / 2;
    int site = 0, stride = 1, rem = t;
    for (int k = 0; k < D; ++k) {
        const int pk = rem % M;
        rem /= M;
        site += (2 * pk + ((j >> k) & 1)) * stride;
        stride *= L;
    }
    return site;
}

static int token_of(const or_cfg *c, const int8_t *s, int t)
{
    int tok = 0;
    for (int j = 0; j < n_spt(c); ++j) tok |= ((s[patch_site(c, t, j)] + 1) / 2) << j;
    return tok;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the       */
/* paper's description: 10 rounds of two 32x32->64 multiplies with a         */
/* Weyl-sequence key schedule.  The sampler's uniform u (Algorithm 2, the    */
/* categorical draw) is ((x0 >> 8) + 0.5) * 2^-24, exact in binary32.        */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* u in (0,1) from word 0 of Philox(key = seed, ctr = (a, b, stream, e)). */
double or_uniform(uint64_t seed, uint32_t a, uint32_t b, uint32_t stream, uint32_t e)
{
    uint32_t ctr[4] = {a, b, stream, e};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox(ctr, key, out);
    return ((double)(out[0] >> 8) + 0.5) * (1.0 / 16777216.0);
}

/* ------------------------------------------------------------------------ */
/* Weight blob: one flat array (float32 on the device, passed here widened). */
/* Order (all row-major, "out x in" for linear maps):                        */
/*   tok[K][d_token]  pos[T][d - d_token]   (K = 2^P classes, T = N / P)     */
/*   per layer: ln1_g[d] ln1_b[d] Wqkv[3d][d] bqkv[3d] ln2_g[d] ln2_b[d]     */
/*              W1[d_ff][d] b1[d_ff] W2[d][d_ff] b2[d]                        */
/*   lnf_g[d] lnf_b[d] Wh[K][d] bh[K]                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    double *ln1g, *ln1b, *Wqkv, *bqkv, *ln2g, *ln2b, *W1, *b1, *W2, *b2;
} or_layer;

typedef struct {
    double *base;
    size_t n;
    double *tok, *pos;
    or_layer *L;
    double *lnfg, *lnfb, *Wh, *bh;
} or_model;

static size_t layer_params(const or_cfg *c)
{
    size_t d = (size_t)c->d, f = (size_t)c->d_ff;
    return 2 * d + 3 * d * d + 3 * d + 2 * d + f * d + f + d * f + d;
}

int64_t or_param_count(const or_cfg *c)
{
    size_t d = (size_t)c->d, K = (size_t)n_cls(c), T = (size_t)n_tok(c);
    return (int64_t)(K * (size_t)c->d_token + T * (d - (size_t)c->d_token)
                     + (size_t)c->n_layers * layer_params(c) + 2 * d + K * d + K);
}

/* Lay views over a double buffer of or_param_count() entries. */
static void model_views(const or_cfg *c, double *p, or_model *m)
{
    size_t d = (size_t)c->d, f = (size_t)c->d_ff;
    m->base = p;
    m->n = (size_t)or_param_count(c);
    m->tok = p; p += (size_t)n_cls(c) * c->d_token;
    m->pos = p; p += (size_t)n_tok(c) * (d - (size_t)c->d_token);
    for (int l = 0; l < c->n_layers; ++l) {
        or_layer *L = &m->L[l];
        L->ln1g = p; p += d;
        L->ln1b = p; p += d;
        L->Wqkv = p; p += 3 * d * d;
        L->bqkv = p; p += 3 * d;
        L->ln2g = p; p += d;
        L->ln2b = p; p += d;
        L->W1 = p; p += f * d;
        L->b1 = p; p += f;
        L->W2 = p; p += d * f;
        L->b2 = p; p += d;
    }
    m->lnfg = p; p += d;
    m->lnfb = p; p += d;
    m->Wh = p; p += (size_t)n_cls(c) * d;
    m->bh = p; p += (size_t)n_cls(c);
}

static int model_load(const or_cfg *c, const double *w, or_model *m)
{
    size_t n = (size_t)or_param_count(c);
    double *p = (double *)malloc(n * sizeof(double));
    m->L = (or_layer *)malloc((size_t)c->n_layers * sizeof(or_layer));
    if (!p || !m->L) { free(p); free(m->L); return -1; }
    memcpy(p, w, n * sizeof(double));
    model_views(c, p, m);
    return 0;
}

static void model_free(or_model *m) { free(m->base); free(m->L); }

/* ------------------------------------------------------------------------ */
/* Building blocks (paper "Overall architecture" and Algorithm 2).           */
/* LayerNorm: affine, biased variance, eps = 1e-5 (paper silent; PyTorch's   */
/* default).  GELU: exact erf form (paper silent).  Attention: softmax of    */
/* q.k / sqrt(d_h), heads concatenated, no output projection W_O.            */
/* ------------------------------------------------------------------------ */
#define LN_EPS 1e-5

static void layernorm(const double *x, const double *g, const double *b, int d,
                      double *y, double *xhat, double *rstd_out)
{
    double mu = 0.0, var = 0.0;
    for (int i = 0; i < d; ++i) mu += x[i];
    mu /= d;
    for (int i = 0; i < d; ++i) var += (x[i] - mu) * (x[i] - mu);
    var /= d;
    double rs = 1.0 / sqrt(var + LN_EPS);
    for (int i = 0; i < d; ++i) {
        double xh = (x[i] - mu) * rs;
        if (xhat) xhat[i] = xh;
        y[i] = xh * g[i] + b[i];
    }
    if (rstd_out) *rstd_out = rs;
}

/* y[o] = b[o] + sum_i W[o][i] x[i] */
static void linear(const double *W, const double *b, const double *x, int n_in, int n_out,
                   double *y)
{
    for (int o = 0; o < n_out; ++o) {
        double s = b ? b[o] : 0.0;
        const double *w = W + (size_t)o * n_in;
        for (int i = 0; i < n_in; ++i) s += w[i] * x[i];
        y[o] = s;
    }
}

static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }

static double gelu_grad(double x)
{
    return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
}

/* log sigmoid(x), evaluated without overflow. */
static double log_sigmoid(double x)
{
    return x >= 0.0 ? -log1p(exp(-x)) : x - log1p(exp(x));
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* Physics-inspired sparse attention (SI Sec. I.A): A_tk = 0 for t - k > W.
 * Reading for periodic lattices: keys k < S (BOS + first row/plane) are
 * always visible, since periodic wrap puts the first row in the ordered
 * Markov boundary of the last row.  Dense causal when mask_kind == 0. */
static int visible(const or_cfg *c, int t, int k)
{
    if (k > t) return 0;
    if (c->mask_kind == 0) return 1;
    return (t - k <= c->W) || (k < c->S);
}

/* Concatenated positional embedding (Eq. concatePE): x_t = [tok(s); pos(t)].
 * Query position t carries the token of spin t-1; position 0 carries the
 * start token 0 (Algorithm 2, "Start token (default: 0)"). */
static void embed(const or_cfg *c, const or_model *m, int t, int tok, double *x)
{
    int dt = c->d_token, dp = c->d - c->d_token;
    for (int i = 0; i < dt; ++i) x[i] = m->tok[tok * dt + i];
    for (int i = 0; i < dp; ++i) x[dt + i] = m->pos[(size_t)t * dp + i];
}

/* Output head (Algorithm 2 "OutputHead", softmax over 2 logits): final
 * LayerNorm then Linear(d -> 2); returns l = z1 - z0 so that
 * q(sigma_t = +1 | past) = softmax(z)_1 = sigmoid(l). */
static double head_logit(const or_cfg *c, const or_model *m, const double *h, double *y,
                         double *xhat, double *rstd)
{
    double z[2];
    layernorm(h, m->lnfg, m->lnfb, c->d, y, xhat, rstd);
    linear(m->Wh, m->bh, y, c->d, 2, z);
    return z[1] - z[0];
}

/* ------------------------------------------------------------------------ */
/* KV-cache decode step (Algorithm 2, one iteration of the t-loop) for one   */
/* sample.  K, V hold [n_layers][N][d]; position t's key and value are       */
/* appended before attention so the query sees its own token.  Returns the   */
/* logit l_t.  work: at least 6*d + d_ff doubles.                            */
/* ------------------------------------------------------------------------ */
static void decode_logits(const or_cfg *c, const or_model *m, double *K, double *V, int t,
                          int tok, double *work, double *z)
{
    int d = c->d, nh = c->n_heads, dh = d / nh, N = n_tok(c);
    double *h = work, *a = h + d, *qkv = a + d, *o = qkv + 3 * d, *f = o + d;
    double inv_sqrt = 1.0 / sqrt((double)dh);
    embed(c, m, t, tok, h);
    for (int l = 0; l < c->n_layers; ++l) {
        const or_layer *L = &m->L[l];
        double *Kl = K + (size_t)l * N * d, *Vl = V + (size_t)l * N * d;
        layernorm(h, L->ln1g, L->ln1b, d, a, NULL, NULL);
        linear(L->Wqkv, L->bqkv, a, d, 3 * d, qkv);
        memcpy(Kl + (size_t)t * d, qkv + d, (size_t)d * sizeof(double));
        memcpy(Vl + (size_t)t * d, qkv + 2 * d, (size_t)d * sizeof(double));
        for (int hh = 0; hh < nh; ++hh) {
            const double *q = qkv + hh * dh;
            double mx = -INFINITY;
            for (int k = 0; k <= t; ++k) {
                if (!visible(c, t, k)) continue;
                double s = 0.0;
                for (int j = 0; j < dh; ++j) s += q[j] * Kl[(size_t)k * d + hh * dh + j];
                s *= inv_sqrt;
                if (s > mx) mx = s;
            }
            double den = 0.0;
            for (int j = 0; j < dh; ++j) o[hh * dh + j] = 0.0;
            for (int k = 0; k <= t; ++k) {
                if (!visible(c, t, k)) continue;
                double s = 0.0;
                for (int j = 0; j < dh; ++j) s += q[j] * Kl[(size_t)k * d + hh * dh + j];
                double p = exp(s * inv_sqrt - mx);
                den += p;
                for (int j = 0; j < dh; ++j) o[hh * dh + j] += p * Vl[(size_t)k * d + hh * dh + j];
            }
            for (int j = 0; j < dh; ++j) o[hh * dh + j] /= den;
        }
        for (int i = 0; i < d; ++i) h[i] += o[i];
        layernorm(h, L->ln2g, L->ln2b, d, a, NULL, NULL);
        linear(L->W1, L->b1, a, d, c->d_ff, f);
        for (int i = 0; i < c->d_ff; ++i) f[i] = gelu(f[i]);
        linear(L->W2, L->b2, f, c->d_ff, d, o);
        for (int i = 0; i < d; ++i) h[i] += o[i];
    }
    layernorm(h, m->lnfg, m->lnfb, d, a, NULL, NULL);
    linear(m->Wh, m->bh, a, d, n_cls(c), z);
}

/* One spin per token: the logit l_t = z1 - z0 of q(+1 | past) = sigmoid(l). */
static double decode_step(const or_cfg *c, const or_model *m, double *K, double *V, int t,
                          int tok, double *work)
{
    double z[2];
    decode_logits(c, m, K, V, t, tok, work, z);
    return z[1] - z[0];
}

/* log softmax of z[K] into lp[K] */
static void log_softmax(const double *z, int K, double *lp)
{
    double mx = -INFINITY, s = 0.0;
    for (int k = 0; k < K; ++k) if (z[k] > mx) mx = z[k];
    for (int k = 0; k < K; ++k) s += exp(z[k] - mx);
    const double lse = mx + log(s);
    for (int k = 0; k < K; ++k) lp[k] = z[k] - lse;
}

/* ------------------------------------------------------------------------ */
/* Ancestral sampling (Algorithm 2).  Sample b, step t draws                 */
/* u = U(Philox(seed, (b, t, stream, 0))) and takes sigma_t = +1 iff         */
/* u < p+ = sigmoid(l_t); log q accumulates log sigmoid(sigma_t * l_t).      */
/* A draw with |p+ - u| < flag_band is "flagged".  If override is non-NULL,  */
/* at every position where override[b*N+t] != 0 the spin is taken from      */
/* override_spins instead (the protocol that replays another                 */
/* implementation's decision on a flagged draw).                             */
/* Outputs (any may be NULL except spins/logq): spins int8 +-1 [B][N],       */
/* logq [B], pplus [B][N], flags uint8 [B][N].  row_ids (may be NULL) gives  */
/* the sample index b used in the counter of output row i (default i).       */
/* cdf_lo [B][N] (may be NULL; patched models only): the cumulative          */
/* probability of the classes before the drawn class, so that the draw's     */
/* class interval is [cdf_lo, cdf_lo + pplus).                               */
/* ------------------------------------------------------------------------ */
int or_sample(const or_cfg *c, const double *weights, int64_t B, const int64_t *row_ids,
              uint64_t seed, uint32_t stream, double flag_band, const uint8_t *override_mask, const int8_t *override_spins,
              int8_t *spins, double *logq, double *pplus, uint8_t *flags, int n_threads,
              double *cdf_lo)
{
    or_model m;
    if (model_load(c, weights, &m)) return -1;
    int N = c->N, d = c->d;
    int err = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel reduction(| : err)
#endif
    {
        size_t kv = (size_t)c->n_layers * N * d;
        double *K = (double *)malloc(kv * sizeof(double));
        double *V = (double *)malloc(kv * sizeof(double));
        double *work = (double *)malloc((size_t)(8 * d + c->d_ff) * sizeof(double));
        if (!K || !V || !work) err = 1;
        else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int64_t b = 0; b < B; ++b) {
              if (n_spt(c) > 1) {
                /* patched: a categorical draw over K classes by the inverse
                 * CDF of u (classes in index order); flagged when u lies
                 * within flag_band of a CDF boundary */
                const int T = n_tok(c), Kc = n_cls(c), P = n_spt(c);
                double z[256], lp[256];
                double lq = 0.0;
                int tok = 0; /* start token */
                for (int t = 0; t < T; ++t) {
                    decode_logits(c, &m, K, V, t, tok, work, z);
                    log_softmax(z, Kc, lp);
                    double u = or_uniform(seed, (uint32_t)(row_ids ? row_ids[b] : b), (uint32_t)t,
                                          stream, 0);
                    /* the first class whose cumulative probability exceeds u */
                    double cdf = 0.0, near = INFINITY;
                    int k = Kc - 1, found = 0;
                    for (int j = 0; j < Kc - 1; ++j) {
                        cdf += exp(lp[j]);
                        if (fabs(u - cdf) < near) near = fabs(u - cdf);
                        if (!found && u < cdf) { k = j; found = 1; }
                    }
                    size_t bt = (size_t)b * N + t;
                    if (override_mask && override_mask[bt])
                        k = token_of(c, override_spins + (size_t)b * N, t);
                    for (int j = 0; j < P; ++j)
                        spins[(size_t)b * N + patch_site(c, t, j)] = (int8_t)(((k >> j) & 1) ? 1 : -1);
                    if (pplus) pplus[bt] = exp(lp[k]);
                    if (cdf_lo) {
                        double below = 0.0;
                        for (int j = 0; j < k; ++j) below += exp(lp[j]);
                        cdf_lo[bt] = below;
                    }
                    if (flags) flags[bt] = (uint8_t)(near < flag_band);
                    lq += lp[k];
                    tok = k;
                }
                logq[b] = lq;
                continue;
              }
              {
                double lq = 0.0;
                int tok = 0; /* start token */
                for (int t = 0; t < N; ++t) {
                    double l = decode_step(c, &m, K, V, t, tok, work);
                    double p = sigmoid(l);
                    double u = or_uniform(seed, (uint32_t)(row_ids ? row_ids[b] : b), (uint32_t)t,
                                          stream, 0);
                    int s = (u < p) ? 1 : -1;
                    int fl = fabs(p - u) < flag_band;
                    size_t bt = (size_t)b * N + t;
                    if (override_mask && override_mask[bt]) s = override_spins[bt];
                    spins[bt] = (int8_t)s;
                    if (pplus) pplus[bt] = p;
                    if (flags) flags[bt] = (uint8_t)fl;
                    lq += log_sigmoid((double)s * l);
                    tok = (s + 1) / 2;
                }
                logq[b] = lq;
              }
            }
        }
        free(K); free(V); free(work);
    }
    model_free(&m);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Teacher-forced forward over the whole sequence (Algorithm 1 structure,    */
/* with Algorithm 2's pre-LayerNorm placement on both sublayers so that the  */
/* sampled and the teacher-forced log q are the same function).  The tape    */
/* keeps what the hand-written backward needs.                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    double *Hin;   /* [L][N][d]  layer input                                 */
    double *X1;    /* [L][N][d]  LN1 normalised (xhat)                        */
    double *R1;    /* [L][N]     LN1 1/std                                    */
    double *A1;    /* [L][N][d]  LN1 output                                   */
    double *QKV;   /* [L][N][3d]                                              */
    double *Hmid;  /* [L][N][d]  after attention residual                     */
    double *X2, *R2, *A2;
    double *F1;    /* [L][N][d_ff] pre-GELU                                   */
    double *G;     /* [L][N][d_ff] post-GELU                                  */
    double *Hfin;  /* [N][d]                                                  */
    double *Xf, *Rf, *Yf;
    double *logit; /* [N]                                                     */
    double *z;     /* [T][K] logits of a patched model (NULL when P = 1)      */
} or_tape;

static int tape_alloc(const or_cfg *c, or_tape *T)
{
    size_t N = (size_t)c->N, d = (size_t)c->d, f = (size_t)c->d_ff, L = (size_t)c->n_layers;
    memset(T, 0, sizeof(*T));
    T->Hin = malloc(L * N * d * sizeof(double));
    T->X1 = malloc(L * N * d * sizeof(double));
    T->R1 = malloc(L * N * sizeof(double));
    T->A1 = malloc(L * N * d * sizeof(double));
    T->QKV = malloc(L * N * 3 * d * sizeof(double));
    T->Hmid = malloc(L * N * d * sizeof(double));
    T->X2 = malloc(L * N * d * sizeof(double));
    T->R2 = malloc(L * N * sizeof(double));
    T->A2 = malloc(L * N * d * sizeof(double));
    T->F1 = malloc(L * N * f * sizeof(double));
    T->G = malloc(L * N * f * sizeof(double));
    T->Hfin = malloc(N * d * sizeof(double));
    T->Xf = malloc(N * d * sizeof(double));
    T->Rf = malloc(N * sizeof(double));
    T->Yf = malloc(N * d * sizeof(double));
    T->logit = malloc(N * sizeof(double));
    T->z = n_spt(c) > 1 ? malloc((size_t)n_tok(c) * n_cls(c) * sizeof(double)) : NULL;
    return (T->Hin && T->X1 && T->R1 && T->A1 && T->QKV && T->Hmid && T->X2 && T->R2 && T->A2
            && T->F1 && T->G && T->Hfin && T->Xf && T->Rf && T->Yf && T->logit
            && (n_spt(c) == 1 || T->z)) ? 0 : -1;
}

static void tape_free(or_tape *T)
{
    free(T->Hin); free(T->X1); free(T->R1); free(T->A1); free(T->QKV); free(T->Hmid);
    free(T->X2); free(T->R2); free(T->A2); free(T->F1); free(T->G); free(T->Hfin);
    free(T->Xf); free(T->Rf); free(T->Yf); free(T->logit); free(T->z);
}

/* Attention probabilities of query t, head hh over keys 0..t (zero where the
 * mask hides a key), from the tape's Q and K of layer l. */
static void attn_probs(const or_cfg *c, const double *QKV, int t, int hh, double *p)
{
    int d = c->d, dh = d / c->n_heads;
    double inv_sqrt = 1.0 / sqrt((double)dh);
    const double *q = QKV + (size_t)t * 3 * d + hh * dh;
    double mx = -INFINITY;
    for (int k = 0; k <= t; ++k) {
        if (!visible(c, t, k)) { p[k] = 0.0; continue; }
        const double *kk = QKV + (size_t)k * 3 * d + d + hh * dh;
        double s = 0.0;
        for (int j = 0; j < dh; ++j) s += q[j] * kk[j];
        p[k] = s * inv_sqrt;
        if (p[k] > mx) mx = p[k];
    }
    double den = 0.0;
    for (int k = 0; k <= t; ++k) {
        if (!visible(c, t, k)) continue;
        p[k] = exp(p[k] - mx);
        den += p[k];
    }
    for (int k = 0; k <= t; ++k) p[k] /= den;
}

/* Returns log q(sigma) = sum_t log sigmoid(sigma_t l_t) (Algorithm 1, last
 * line, with softmax over two logits written as a sigmoid). */
static double tf_forward(const or_cfg *c, const or_model *m, const int8_t *s, or_tape *T,
                         double *prob)
{
    int N = n_tok(c), d = c->d, f = c->d_ff, nh = c->n_heads, dh = d / nh;
    size_t Nd = (size_t)N * d;
    double *H = T->Hfin; /* running residual stream [T][d] */
    for (int t = 0; t < N; ++t) embed(c, m, t, t == 0 ? 0 : token_of(c, s, t - 1), H + (size_t)t * d);
    for (int l = 0; l < c->n_layers; ++l) {
        const or_layer *L = &m->L[l];
        double *Hin = T->Hin + l * Nd, *X1 = T->X1 + l * Nd, *A1 = T->A1 + l * Nd;
        double *QKV = T->QKV + l * 3 * Nd, *Hmid = T->Hmid + l * Nd;
        double *X2 = T->X2 + l * Nd, *A2 = T->A2 + l * Nd;
        double *F1 = T->F1 + (size_t)l * N * f, *G = T->G + (size_t)l * N * f;
        memcpy(Hin, H, Nd * sizeof(double));
        for (int t = 0; t < N; ++t) {
            layernorm(Hin + (size_t)t * d, L->ln1g, L->ln1b, d, A1 + (size_t)t * d,
                      X1 + (size_t)t * d, T->R1 + (size_t)l * N + t);
            linear(L->Wqkv, L->bqkv, A1 + (size_t)t * d, d, 3 * d, QKV + (size_t)t * 3 * d);
        }
        for (int t = 0; t < N; ++t) {
            double *hm = Hmid + (size_t)t * d;
            memcpy(hm, Hin + (size_t)t * d, (size_t)d * sizeof(double));
            for (int hh = 0; hh < nh; ++hh) {
                attn_probs(c, QKV, t, hh, prob);
                for (int j = 0; j < dh; ++j) {
                    double o = 0.0;
                    for (int k = 0; k <= t; ++k)
                        o += prob[k] * QKV[(size_t)k * 3 * d + 2 * d + hh * dh + j];
                    hm[hh * dh + j] += o;
                }
            }
        }
        for (int t = 0; t < N; ++t) {
            layernorm(Hmid + (size_t)t * d, L->ln2g, L->ln2b, d, A2 + (size_t)t * d,
                      X2 + (size_t)t * d, T->R2 + (size_t)l * N + t);
            linear(L->W1, L->b1, A2 + (size_t)t * d, d, f, F1 + (size_t)t * f);
            for (int i = 0; i < f; ++i) G[(size_t)t * f + i] = gelu(F1[(size_t)t * f + i]);
            double *ho = H + (size_t)t * d;
            linear(L->W2, L->b2, G + (size_t)t * f, f, d, ho);
            for (int i = 0; i < d; ++i) ho[i] += Hmid[(size_t)t * d + i];
        }
    }
    double lq = 0.0;
    if (n_spt(c) > 1) {  /* log softmax of the token's class */
        const int Kc = n_cls(c);
        double lp[256];
        for (int t = 0; t < N; ++t) {
            double *z = T->z + (size_t)t * Kc;
            layernorm(H + (size_t)t * d, m->lnfg, m->lnfb, d, T->Yf + (size_t)t * d,
                      T->Xf + (size_t)t * d, T->Rf + t);
            linear(m->Wh, m->bh, T->Yf + (size_t)t * d, d, Kc, z);
            log_softmax(z, Kc, lp);
            lq += lp[token_of(c, s, t)];
        }
        return lq;
    }
    for (int t = 0; t < N; ++t) {
        T->logit[t] = head_logit(c, m, H + (size_t)t * d, T->Yf + (size_t)t * d,
                                 T->Xf + (size_t)t * d, T->Rf + t);
        lq += log_sigmoid((double)s[t] * T->logit[t]);
    }
    return lq;
}

/* Teacher-forced log q for B given configurations (Algorithm 1). */
int or_logprob(const or_cfg *c, const double *weights, int64_t B, const int8_t *spins,
               double *logq, double *pplus, int n_threads)
{
    or_model m;
    if (model_load(c, weights, &m)) return -1;
    int err = 0, N = c->N;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel reduction(| : err)
#endif
    {
        or_tape T;
        double *prob = (double *)malloc((size_t)N * sizeof(double));
        if (tape_alloc(c, &T) || !prob) err = 1;
        else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int64_t b = 0; b < B; ++b) {
                logq[b] = tf_forward(c, &m, spins + (size_t)b * N, &T, prob);
                if (pplus && n_spt(c) > 1) {
                    double lp[256];
                    for (int t = 0; t < n_tok(c); ++t) {
                        log_softmax(T.z + (size_t)t * n_cls(c), n_cls(c), lp);
                        pplus[(size_t)b * N + t] = exp(lp[token_of(c, spins + (size_t)b * N, t)]);
                    }
                } else if (pplus)
                    for (int t = 0; t < N; ++t) pplus[(size_t)b * N + t] = sigmoid(T.logit[t]);
            }
        }
        tape_free(&T);
        free(prob);
    }
    model_free(&m);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Hand-written FP64 backward of the teacher-forced log q.                   */
/* grad = sum_b coeff[b] * d log q(sigma_b) / d theta, the REINFORCE sum of  */
/* Eq. (loss1) with coeff[b] = (L_b - Lbar) / M.  grad has the blob layout.  */
/* ------------------------------------------------------------------------ */
static void layernorm_bwd(const double *dy, const double *xhat, double rstd, const double *g,
                          int d, double *dx_accum, double *dg, double *db)
{
    double m1 = 0.0, m2 = 0.0;
    for (int i = 0; i < d; ++i) {
        double dxh = dy[i] * g[i];
        dg[i] += dy[i] * xhat[i];
        db[i] += dy[i];
        m1 += dxh;
        m2 += dxh * xhat[i];
    }
    m1 /= d; m2 /= d;
    for (int i = 0; i < d; ++i) dx_accum[i] += rstd * (dy[i] * g[i] - m1 - xhat[i] * m2);
}

static void backward_one(const or_cfg *c, const or_model *m, const int8_t *s, double coeff,
                         or_tape *T, or_model *gm, double *prob, double *dprob, double *buf)
{
    int N = n_tok(c), d = c->d, f = c->d_ff, nh = c->n_heads, dh = d / nh;
    size_t Nd = (size_t)N * d;
    double inv_sqrt = 1.0 / sqrt((double)dh);
    double *dH = buf;                    /* [N][d] gradient w.r.t. residual stream */
    double *dHmid = dH + Nd;             /* [N][d] */
    double *dQKV = dHmid + Nd;           /* [N][3d] */
    double *tmp = dQKV + 3 * Nd;         /* [max(d_ff, 3d)] */
    double *dA = tmp + (f > 3 * d ? f : 3 * d); /* [d] */
    memset(dH, 0, Nd * sizeof(double));
    /* patched head: d log softmax(z)[tok] / dz = onehot(tok) - softmax(z) */
    for (int t = 0; t < N && n_spt(c) > 1; ++t) {
        const int Kc = n_cls(c), tok = token_of(c, s, t);
        double lp[256];
        log_softmax(T->z + (size_t)t * Kc, Kc, lp);
        const double *y = T->Yf + (size_t)t * d;
        for (int i = 0; i < d; ++i) dA[i] = 0.0;
        for (int k = 0; k < Kc; ++k) {
            const double dz = coeff * ((k == tok ? 1.0 : 0.0) - exp(lp[k]));
            gm->bh[k] += dz;
            for (int i = 0; i < d; ++i) {
                gm->Wh[(size_t)k * d + i] += dz * y[i];
                dA[i] += dz * m->Wh[(size_t)k * d + i];
            }
        }
        layernorm_bwd(dA, T->Xf + (size_t)t * d, T->Rf[t], m->lnfg, d, dH + (size_t)t * d,
                      gm->lnfg, gm->lnfb);
    }
    /* head: log sigmoid(s l) -> d/dl = s * sigmoid(-s l) */
    for (int t = 0; t < N && n_spt(c) == 1; ++t) {
        double sl = (double)s[t];
        double dl = coeff * sl * sigmoid(-sl * T->logit[t]);
        double dz[2] = {-dl, dl};
        const double *y = T->Yf + (size_t)t * d;
        for (int j = 0; j < 2; ++j) {
            gm->bh[j] += dz[j];
            for (int i = 0; i < d; ++i) gm->Wh[j * d + i] += dz[j] * y[i];
        }
        for (int i = 0; i < d; ++i) dA[i] = dz[0] * m->Wh[i] + dz[1] * m->Wh[d + i];
        layernorm_bwd(dA, T->Xf + (size_t)t * d, T->Rf[t], m->lnfg, d, dH + (size_t)t * d,
                      gm->lnfg, gm->lnfb);
    }
    for (int l = c->n_layers - 1; l >= 0; --l) {
        const or_layer *L = &m->L[l];
        or_layer *GL = &gm->L[l];
        double *X1 = T->X1 + l * Nd, *A1 = T->A1 + l * Nd, *QKV = T->QKV + l * 3 * Nd;
        double *X2 = T->X2 + l * Nd, *A2 = T->A2 + l * Nd;
        double *F1 = T->F1 + (size_t)l * N * f, *G = T->G + (size_t)l * N * f;
        /* FFN sublayer: H = Hmid + W2 gelu(W1 LN2(Hmid) + b1) + b2 */
        memcpy(dHmid, dH, Nd * sizeof(double));
        for (int t = 0; t < N; ++t) {
            const double *dy = dH + (size_t)t * d;
            for (int o = 0; o < d; ++o) {
                GL->b2[o] += dy[o];
                for (int i = 0; i < f; ++i) GL->W2[(size_t)o * f + i] += dy[o] * G[(size_t)t * f + i];
            }
            for (int i = 0; i < f; ++i) {
                double g = 0.0;
                for (int o = 0; o < d; ++o) g += L->W2[(size_t)o * f + i] * dy[o];
                tmp[i] = g * gelu_grad(F1[(size_t)t * f + i]);
            }
            for (int i = 0; i < f; ++i) {
                GL->b1[i] += tmp[i];
                for (int k = 0; k < d; ++k) GL->W1[(size_t)i * d + k] += tmp[i] * A2[(size_t)t * d + k];
            }
            for (int k = 0; k < d; ++k) {
                double a = 0.0;
                for (int i = 0; i < f; ++i) a += L->W1[(size_t)i * d + k] * tmp[i];
                dA[k] = a;
            }
            layernorm_bwd(dA, X2 + (size_t)t * d, T->R2[(size_t)l * N + t], L->ln2g, d,
                          dHmid + (size_t)t * d, GL->ln2g, GL->ln2b);
        }
        /* attention sublayer: Hmid = Hin + concat_h sum_k P_tk v_k */
        memset(dQKV, 0, 3 * Nd * sizeof(double));
        for (int t = 0; t < N; ++t) {
            const double *dout = dHmid + (size_t)t * d;
            for (int hh = 0; hh < nh; ++hh) {
                attn_probs(c, QKV, t, hh, prob);
                double dot = 0.0;
                for (int k = 0; k <= t; ++k) {
                    const double *v = QKV + (size_t)k * 3 * d + 2 * d + hh * dh;
                    double dp = 0.0;
                    for (int j = 0; j < dh; ++j) {
                        dp += dout[hh * dh + j] * v[j];
                        dQKV[(size_t)k * 3 * d + 2 * d + hh * dh + j] += prob[k] * dout[hh * dh + j];
                    }
                    dprob[k] = dp;
                    dot += prob[k] * dp;
                }
                const double *q = QKV + (size_t)t * 3 * d + hh * dh;
                for (int k = 0; k <= t; ++k) {
                    double ds = prob[k] * (dprob[k] - dot) * inv_sqrt;
                    if (ds == 0.0) continue;
                    const double *kk = QKV + (size_t)k * 3 * d + d + hh * dh;
                    for (int j = 0; j < dh; ++j) {
                        dQKV[(size_t)t * 3 * d + hh * dh + j] += ds * kk[j];
                        dQKV[(size_t)k * 3 * d + d + hh * dh + j] += ds * q[j];
                    }
                }
            }
        }
        /* QKV projection and LN1 */
        memcpy(dH, dHmid, Nd * sizeof(double));
        for (int t = 0; t < N; ++t) {
            const double *dq = dQKV + (size_t)t * 3 * d;
            for (int o = 0; o < 3 * d; ++o) {
                GL->bqkv[o] += dq[o];
                for (int k = 0; k < d; ++k) GL->Wqkv[(size_t)o * d + k] += dq[o] * A1[(size_t)t * d + k];
            }
            for (int k = 0; k < d; ++k) {
                double a = 0.0;
                for (int o = 0; o < 3 * d; ++o) a += L->Wqkv[(size_t)o * d + k] * dq[o];
                dA[k] = a;
            }
            layernorm_bwd(dA, X1 + (size_t)t * d, T->R1[(size_t)l * N + t], L->ln1g, d,
                          dH + (size_t)t * d, GL->ln1g, GL->ln1b);
        }
    }
    /* concatenated embedding */
    int dt = c->d_token, dp = d - dt;
    for (int t = 0; t < N; ++t) {
        int tok = t == 0 ? 0 : token_of(c, s, t - 1);
        for (int i = 0; i < dt; ++i) gm->tok[tok * dt + i] += dH[(size_t)t * d + i];
        for (int i = 0; i < dp; ++i) gm->pos[(size_t)t * dp + i] += dH[(size_t)t * d + dt + i];
    }
}

int or_grad(const or_cfg *c, const double *weights, int64_t B, const int8_t *spins,
            const double *coeff, double *grad, double *logq, int n_threads)
{
    or_model m;
    if (model_load(c, weights, &m)) return -1;
    int N = c->N, d = c->d, f = c->d_ff;
    size_t P = (size_t)or_param_count(c);
    memset(grad, 0, P * sizeof(double));
    int err = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel reduction(| : err)
#endif
    {
        or_tape T;
        or_model gm;
        double *gbuf = (double *)calloc(P, sizeof(double));
        gm.L = (or_layer *)malloc((size_t)c->n_layers * sizeof(or_layer));
        double *prob = (double *)malloc((size_t)N * sizeof(double));
        double *dprob = (double *)malloc((size_t)N * sizeof(double));
        size_t nb = (size_t)N * d * 5 + (size_t)(f > 3 * d ? f : 3 * d) + (size_t)d;
        double *buf = (double *)malloc(nb * sizeof(double));
        if (tape_alloc(c, &T) || !gbuf || !gm.L || !prob || !dprob || !buf) err = 1;
        else {
            model_views(c, gbuf, &gm);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int64_t b = 0; b < B; ++b) {
                const int8_t *s = spins + (size_t)b * N;
                double lq = tf_forward(c, &m, s, &T, prob);
                if (logq) logq[b] = lq;
                backward_one(c, &m, s, coeff[b], &T, &gm, prob, dprob, buf);
            }
#ifdef _OPENMP
#pragma omp critical
#endif
            for (size_t i = 0; i < P; ++i) grad[i] += gbuf[i];
        }
        tape_free(&T);
        free(gbuf); free(gm.L); free(prob); free(dprob); free(buf);
    }
    model_free(&m);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Energies.                                                                 */
/* SK (Eq. SKHam): E = -sum_{i<j} J_ij s_i s_j; the 1/sqrt(N) of the paper   */
/* is folded into J ~ N(0, 1/N).  J is a dense N x N array, only i<j read.   */
/* EA (Eq. EAHam): E = -sum over nearest-neighbour pairs, each pair once;    */
/* bonds[i*D + mu] couples site i to its +mu neighbour in raster order       */
/* i = x0 + L x1 + L^2 x2.  Periodic wrap, or no bond across the edge when   */
/* open.                                                                     */
/* ------------------------------------------------------------------------ */
void or_energy_sk(int N, const float *J, int64_t B, const int8_t *spins, double *E)
{
    for (int64_t b = 0; b < B; ++b) {
        const int8_t *s = spins + (size_t)b * N;
        double e = 0.0;
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j) e -= (double)J[(size_t)i * N + j] * s[i] * s[j];
        E[b] = e;
    }
}

static int ea_neighbor(int D, int L, int periodic, int i, int mu)
{
    int stride = 1;
    for (int k = 0; k < mu; ++k) stride *= L;
    int x = (i / stride) % L;
    if (x == L - 1) return periodic ? i - (L - 1) * stride : -1;
    return i + stride;
}

void or_energy_ea(int D, int L, int periodic, const float *bonds, int64_t B,
                  const int8_t *spins, double *E)
{
    int N = 1;
    for (int k = 0; k < D; ++k) N *= L;
    for (int64_t b = 0; b < B; ++b) {
        const int8_t *s = spins + (size_t)b * N;
        double e = 0.0;
        for (int i = 0; i < N; ++i)
            for (int mu = 0; mu < D; ++mu) {
                int j = ea_neighbor(D, L, periodic, i, mu);
                if (j >= 0) e -= (double)bonds[(size_t)i * D + mu] * s[i] * s[j];
            }
        E[b] = e;
    }
}

/* ------------------------------------------------------------------------ */
/* Free energies (Eqs. KL_div and free_energy), from a batch:                 */
/*   L_b = beta E_b + ln q_b,  F_q = mean(L)/beta,                            */
/*   F_IS = -(1/beta) [ln sum_b exp(-L_b) - ln B]  (importance reweighting), */
/*   Kish ESS = (sum w)^2 / sum w^2 with w_b = exp(-L_b - max(-L)).          */
/* out = {F_q, F_IS, ESS}.                                                   */
/* ------------------------------------------------------------------------ */
void or_free_energy(int64_t B, const double *E, const double *logq, double beta, double *out)
{
    long double sumL = 0.0L, mx = -INFINITY;
    for (int64_t b = 0; b < B; ++b) {
        double Lb = beta * E[b] + logq[b];
        sumL += Lb;
        if (-Lb > mx) mx = -Lb;
    }
    long double sw = 0.0L, sw2 = 0.0L;
    for (int64_t b = 0; b < B; ++b) {
        long double w = expl(-(beta * E[b] + logq[b]) - mx);
        sw += w;
        sw2 += w * w;
    }
    out[0] = (double)(sumL / B / beta);
    out[1] = (double)(-(mx + logl(sw) - logl((long double)B)) / beta);
    out[2] = (double)(sw * sw / sw2);
}

/* ------------------------------------------------------------------------ */
/* REINFORCE weights of a per-sample loss L_b = a E_b + c ln q_b (Eq. loss1  */
/* with (a, c) = (beta, 1); the ground-state form L = E + T ln q of Methods  */
/* "Variational annealing" with (1, T)) and the likelihood term of Eq. loss2 */
/* with weight w:  the gradient (1/B) sum (L - mean L) grad ln q - (w/B) sum */
/* grad ln q is sum_b coeff_b grad ln q_b with coeff_b = (L_b - mean L - w)/B. */
/* mean_out = {mean L, mean E}.                                              */
/* ------------------------------------------------------------------------ */
void or_loss_coeff(int64_t B, const double *E, const double *logq, double a, double c, double w,
                   double *mean_out, double *coeff)
{
    long double sumL = 0.0L, sumE = 0.0L;
    for (int64_t b = 0; b < B; ++b) {
        sumL += a * E[b] + c * logq[b];
        sumE += E[b];
    }
    const double meanL = (double)(sumL / B);
    mean_out[0] = meanL;
    mean_out[1] = (double)(sumE / B);
    for (int64_t b = 0; b < B; ++b) coeff[b] = (a * E[b] + c * logq[b] - meanL - w) / (double)B;
}

/* ------------------------------------------------------------------------ */
/* Muon (Methods "Comparison on optimizers"): for each weight matrix         */
/* (Wqkv, W1, W2 of every layer) with gradient G: M = mu M + G; O = k        */
/* quintic Newton-Schulz steps on X = M / (|M|_F + 1e-7), taken on M^T when  */
/* it has more rows than columns: X <- a X + (b A + c A A) X, A = X X^T,     */
/* (a, b, c) = (3.4445, -4.7750, 2.0315) (Jordan et al. 2024); then          */
/* W -= lr (s O + wd W) with the RMS alignment s = 0.2 sqrt(max(r, c)) and   */
/* decoupled weight decay (Liu et al. 2025).  Every other parameter takes an */
/* AdamW step (beta1 0.9, beta2 0.999, eps 1e-8, same lr and wd).            */
/* ------------------------------------------------------------------------ */
static void ns_orthogonalise(const double *M, int rows, int cols, int steps, double *O)
{
    const int tr = rows > cols;
    const int p = tr ? cols : rows, q = tr ? rows : cols;  /* X is p x q, p <= q */
    double *X = (double *)malloc((size_t)p * q * sizeof(double));
    double *Y = (double *)malloc((size_t)p * q * sizeof(double));
    double *A = (double *)malloc((size_t)p * p * sizeof(double));
    double *Bm = (double *)malloc((size_t)p * p * sizeof(double));
    double ss = 0.0;
    for (size_t i = 0; i < (size_t)rows * cols; ++i) ss += M[i] * M[i];
    const double inv = 1.0 / (sqrt(ss) + 1e-7);
    for (int i = 0; i < rows; ++i)
        for (int j = 0; j < cols; ++j) {
            const double v = M[(size_t)i * cols + j] * inv;
            if (tr) X[(size_t)j * q + i] = v;
            else X[(size_t)i * q + j] = v;
        }
    const double a = 3.4445, b = -4.7750, c = 2.0315;
    for (int it = 0; it < steps; ++it) {
        for (int i = 0; i < p; ++i)          /* A = X X^T */
            for (int j = 0; j < p; ++j) {
                double acc = 0.0;
                for (int k = 0; k < q; ++k) acc += X[(size_t)i * q + k] * X[(size_t)j * q + k];
                A[(size_t)i * p + j] = acc;
            }
        for (int i = 0; i < p; ++i)          /* Bm = b A + c A A */
            for (int j = 0; j < p; ++j) {
                double acc = 0.0;
                for (int k = 0; k < p; ++k) acc += A[(size_t)i * p + k] * A[(size_t)k * p + j];
                Bm[(size_t)i * p + j] = b * A[(size_t)i * p + j] + c * acc;
            }
        for (int i = 0; i < p; ++i)          /* Y = a X + Bm X */
            for (int j = 0; j < q; ++j) {
                double acc = 0.0;
                for (int k = 0; k < p; ++k) acc += Bm[(size_t)i * p + k] * X[(size_t)k * q + j];
                Y[(size_t)i * q + j] = a * X[(size_t)i * q + j] + acc;
            }
        double *t = X; X = Y; Y = t;
    }
    for (int i = 0; i < rows; ++i)
        for (int j = 0; j < cols; ++j)
            O[(size_t)i * cols + j] = tr ? X[(size_t)j * q + i] : X[(size_t)i * q + j];
    free(X); free(Y); free(A); free(Bm);
}

void or_newton_schulz(const double *M, int rows, int cols, int steps, double *O)
{
    ns_orthogonalise(M, rows, cols, steps, O);
}

static void adamw_range(double *w, const double *g, double *m, double *v, size_t n, double lr,
                        double wd, double bc1, double bc2)
{
    for (size_t i = 0; i < n; ++i) {
        m[i] = 0.9 * m[i] + 0.1 * g[i];
        v[i] = 0.999 * v[i] + 0.001 * g[i] * g[i];
        w[i] -= lr * ((m[i] / bc1) / (sqrt(v[i] / bc2) + 1e-8) + wd * w[i]);
    }
}

void or_muon_step(const or_cfg *c, double *w, const double *g, double *mom, double *am, double *av,
                  double lr, double mu, double wd, int ns_steps, int64_t step)
{
    const size_t d = (size_t)c->d, f = (size_t)c->d_ff;
    const double bc1 = 1.0 - pow(0.9, (double)step), bc2 = 1.0 - pow(0.999, (double)step);
    size_t off = 0;
    /* walk the blob in layout order: matrices get Muon, the rest AdamW */
#define OR_ADAMW(n) do { adamw_range(w + off, g + off, am + off, av + off, (n), lr, wd, bc1, bc2); off += (n); } while (0)
#define OR_MUON(r, cc) do { \
        const size_t n_ = (size_t)(r) * (cc); \
        for (size_t i_ = 0; i_ < n_; ++i_) mom[off + i_] = mu * mom[off + i_] + g[off + i_]; \
        double *O_ = (double *)malloc(n_ * sizeof(double)); \
        ns_orthogonalise(mom + off, (int)(r), (int)(cc), ns_steps, O_); \
        const double s_ = 0.2 * sqrt((double)((r) > (cc) ? (r) : (cc))); \
        for (size_t i_ = 0; i_ < n_; ++i_) w[off + i_] -= lr * (s_ * O_[i_] + wd * w[off + i_]); \
        free(O_); off += n_; } while (0)
    OR_ADAMW(2 * (size_t)c->d_token);
    OR_ADAMW((size_t)c->N * (d - (size_t)c->d_token));
    for (int l = 0; l < c->n_layers; ++l) {
        OR_ADAMW(2 * d);          /* ln1 gain, bias */
        OR_MUON(3 * d, d);        /* Wqkv */
        OR_ADAMW(3 * d + 2 * d);  /* bqkv, ln2 gain, bias */
        OR_MUON(f, d);            /* W1 */
        OR_ADAMW(f);              /* b1 */
        OR_MUON(d, f);            /* W2 */
        OR_ADAMW(d);              /* b2 */
    }
    OR_ADAMW(2 * d + 2 * d + 2);  /* LN_f, head */
#undef OR_ADAMW
#undef OR_MUON
}

/* ------------------------------------------------------------------------ */
/* Exhaustive enumeration over all 2^N configurations by a prefix-tree walk: */
/* each tree node costs one decode step (Algorithm 2) and its two children   */
/* reuse its KV cache.  Gives sum_sigma q (=1 by construction, Sec.          */
/* "Framework"), ln Z with E from the given instance, F = -ln Z / beta and   */
/* the exact F_q = (1/beta) sum q (beta E + ln q) of Eq. (free_energy).      */
/* kind 0: SK with J [N][N]; kind 1: EA with (D, L, periodic, bonds).        */
/* out = {sum_q, lnZ, F, F_q, E_min}.                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_cfg *c;
    const or_model *m;
    int kind, D, L, periodic;
    const float *J;
    double beta;
    double *K, *V, *work;
    int8_t *s;
    /* accumulators */
    double sum_q, sum_q_c;     /* Kahan */
    double fq, fq_c;           /* Kahan: sum q (beta E + ln q) */
    double lz_max, lz_sum;     /* running log-sum-exp of -beta E */
    double emin;
} enum_ctx;

static double energy_one(const enum_ctx *x)
{
    double e;
    if (x->kind == 0) or_energy_sk(x->c->N, x->J, 1, x->s, &e);
    else or_energy_ea(x->D, x->L, x->periodic, x->J, 1, x->s, &e);
    return e;
}

static void kahan_add(double *sum, double *comp, double v)
{
    double y = v - *comp;
    double t = *sum + y;
    *comp = (t - *sum) - y;
    *sum = t;
}

static void enum_leaf(enum_ctx *x, double lq)
{
    double e = energy_one(x);
    double q = exp(lq);
    kahan_add(&x->sum_q, &x->sum_q_c, q);
    kahan_add(&x->fq, &x->fq_c, q * (x->beta * e + lq));
    double a = -x->beta * e;
    if (a > x->lz_max) {
        x->lz_sum = x->lz_sum * exp(x->lz_max - a) + 1.0;
        x->lz_max = a;
    } else {
        x->lz_sum += exp(a - x->lz_max);
    }
    if (e < x->emin) x->emin = e;
}

static void enum_rec(enum_ctx *x, int t, double lq)
{
    int N = x->c->N;
    if (t == N) { enum_leaf(x, lq); return; }
    int tok = t == 0 ? 0 : (x->s[t - 1] + 1) / 2;
    double l = decode_step(x->c, x->m, x->K, x->V, t, tok, x->work);
    x->s[t] = 1;
    enum_rec(x, t + 1, lq + log_sigmoid(l));
    x->s[t] = -1;
    enum_rec(x, t + 1, lq + log_sigmoid(-l));
}

/* patched models: the tree has K children per token */
static void enum_rec_tok(enum_ctx *x, int t, int tok_prev, double lq)
{
    const or_cfg *c = x->c;
    if (t == n_tok(c)) { enum_leaf(x, lq); return; }
    double z[256], lp[256];
    decode_logits(c, x->m, x->K, x->V, t, tok_prev, x->work, z);
    log_softmax(z, n_cls(c), lp);
    for (int k = 0; k < n_cls(c); ++k) {
        for (int j = 0; j < n_spt(c); ++j)
            x->s[patch_site(c, t, j)] = (int8_t)(((k >> j) & 1) ? 1 : -1);
        enum_rec_tok(x, t + 1, k, lq + lp[k]);
    }
}

int or_enumerate(const or_cfg *c, const double *weights, int kind, int D, int L, int periodic,
                 const float *J, double beta, double *out, int n_threads)
{
    or_model m;
    if (model_load(c, weights, &m)) return -1;
    int N = c->N, d = c->d;
    const int patched = n_spt(c) > 1;
    int split = N < 6 ? N : 6; /* 2^split independent subtrees (K for a patched model) */
    int64_t nsub = patched ? (int64_t)n_cls(c) : (int64_t)1 << split;
    double sum_q = 0.0, fq = 0.0, emin = INFINITY;
    double *lzm = (double *)malloc((size_t)nsub * sizeof(double));
    double *lzs = (double *)malloc((size_t)nsub * sizeof(double));
    double *sq = (double *)malloc((size_t)nsub * sizeof(double));
    double *sf = (double *)malloc((size_t)nsub * sizeof(double));
    double *em = (double *)malloc((size_t)nsub * sizeof(double));
    int err = (!lzm || !lzs || !sq || !sf || !em);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel reduction(| : err)
#endif
    if (!err) {
        enum_ctx x;
        memset(&x, 0, sizeof(x));
        x.c = c; x.m = &m; x.kind = kind; x.D = D; x.L = L; x.periodic = periodic; x.J = J;
        x.beta = beta;
        size_t kv = (size_t)c->n_layers * N * d;
        x.K = (double *)malloc(kv * sizeof(double));
        x.V = (double *)malloc(kv * sizeof(double));
        x.work = (double *)malloc((size_t)(8 * d + c->d_ff) * sizeof(double));
        x.s = (int8_t *)malloc((size_t)N);
        if (!x.K || !x.V || !x.work || !x.s) err = 1;
        else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int64_t sub = 0; sub < nsub; ++sub) {
                x.sum_q = x.sum_q_c = x.fq = x.fq_c = 0.0;
                x.lz_max = -INFINITY; x.lz_sum = 0.0; x.emin = INFINITY;
                if (patched) {  /* subtree: the class of token 0 */
                    double z[256], lp[256];
                    decode_logits(c, &m, x.K, x.V, 0, 0, x.work, z);
                    log_softmax(z, n_cls(c), lp);
                    for (int j = 0; j < n_spt(c); ++j)
                        x.s[patch_site(c, 0, j)] = (int8_t)(((sub >> j) & 1) ? 1 : -1);
                    enum_rec_tok(&x, 1, (int)sub, lp[sub]);
                    lzm[sub] = x.lz_max; lzs[sub] = x.lz_sum;
                    sq[sub] = x.sum_q; sf[sub] = x.fq; em[sub] = x.emin;
                    continue;
                }
                /* walk the prefix of this subtree: bit t of sub = spin t is -1 */
                double lq = 0.0;
                for (int t = 0; t < split; ++t) {
                    int tok = t == 0 ? 0 : (x.s[t - 1] + 1) / 2;
                    double l = decode_step(c, &m, x.K, x.V, t, tok, x.work);
                    int sp = ((sub >> t) & 1) ? -1 : 1;
                    x.s[t] = (int8_t)sp;
                    lq += log_sigmoid(sp * l);
                }
                enum_rec(&x, split, lq);
                lzm[sub] = x.lz_max; lzs[sub] = x.lz_sum;
                sq[sub] = x.sum_q; sf[sub] = x.fq; em[sub] = x.emin;
            }
        }
        free(x.K); free(x.V); free(x.work); free(x.s);
    }
    if (!err) {
        double mx = -INFINITY, s = 0.0;
        for (int64_t i = 0; i < nsub; ++i) if (lzm[i] > mx) mx = lzm[i];
        for (int64_t i = 0; i < nsub; ++i) s += lzs[i] * exp(lzm[i] - mx);
        double cq = 0.0, cf = 0.0;
        for (int64_t i = 0; i < nsub; ++i) {
            kahan_add(&sum_q, &cq, sq[i]);
            kahan_add(&fq, &cf, sf[i]);
            if (em[i] < emin) emin = em[i];
        }
        double lnZ = mx + log(s);
        out[0] = sum_q;
        out[1] = lnZ;
        out[2] = -lnZ / beta;
        out[3] = fq / beta;
        out[4] = emin;
    }
    free(lzm); free(lzs); free(sq); free(sf); free(em);
    model_free(&m);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Independence Metropolis-Hastings with the model as proposal (not in the   */
/* paper; its Monte Carlo + generative-model combination).  Chain c consumes */
/* proposals p = j*C + c, j = 0..B/C-1, in order.  With log weights          */
/* lw = -beta E - ln q, the log acceptance is lw(p) - lw(state); the draw    */
/* u = U(Philox(seed, (c, j, 1, 0))) accepts iff log u < log alpha.          */
/* |log alpha - log u| < flag_band marks a flagged decision; override        */
/* (per proposal, may be NULL) replays the other side's decision there.      */
/* chain_E, chain_lq, chain_idx hold the state in and out (chain_idx = index */
/* of the accepted proposal, -1 = initial state).  trace_E [B/C][C] gets the */
/* chain energy after each proposal.  accept [C] counts acceptances.          */
/* ------------------------------------------------------------------------ */
int or_mh(int64_t B, int C, const double *E, const double *logq, double beta, uint64_t seed,
          double flag_band, const int8_t *override_acc, double *chain_E, double *chain_lq,
          int64_t *chain_idx, double *trace_E, int64_t *accepts, uint8_t *flags)
{
    if (C <= 0 || B % C) return -1;
    int64_t per = B / C;
    for (int c = 0; c < C; ++c) {
        double e = chain_E[c], lq = chain_lq[c];
        int64_t idx = chain_idx[c], acc = 0;
        for (int64_t j = 0; j < per; ++j) {
            int64_t p = j * C + c;
            double la = (-beta * E[p] - logq[p]) - (-beta * e - lq);
            double lu = log(or_uniform(seed, (uint32_t)c, (uint32_t)j, 1, 0));
            int a = lu < la;
            if (flags) flags[p] = fabs(la - lu) < flag_band;
            if (override_acc && override_acc[p] >= 0) a = override_acc[p];
            if (a) { e = E[p]; lq = logq[p]; idx = p; ++acc; }
            if (trace_E) trace_E[j * C + c] = e;
        }
        chain_E[c] = e; chain_lq[c] = lq; chain_idx[c] = idx; accepts[c] = acc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Single-spin-flip Metropolis (the local Monte Carlo of the paper's loss2   */
/* refinement and the classical reference).  Replica r, sweep w visits       */
/* sites i = 0..N-1 in order; dE = 2 s_i h_i with h_i = sum_j J_ij s_j;      */
/* accept iff u < exp(-beta dE), u = U(Philox(seed, (r, i, 2, w))).          */
/* kind 0: SK dense J; kind 1: EA bonds.  trace_E [sweeps][R] gets the       */
/* energy after each sweep (E0 [R] is the initial energy).  flags counts     */
/* decisions with |u - exp(-beta dE)| < 1e-12.                               */
/* ------------------------------------------------------------------------ */
static double local_field(int kind, int N, int D, int L, int periodic, const float *J,
                          const int8_t *s, int i)
{
    double h = 0.0;
    if (kind == 0) {
        for (int j = 0; j < N; ++j)
            if (j != i) h += (double)J[(size_t)i * N + j] * s[j];
        return h;
    }
    /* bonds from i to its +mu neighbours */
    for (int mu = 0; mu < D; ++mu) {
        int j = ea_neighbor(D, L, periodic, i, mu);
        if (j >= 0) h += (double)J[(size_t)i * D + mu] * s[j];
    }
    /* bonds from the -mu neighbours k, whose +mu neighbour is i */
    int stride = 1;
    for (int mu = 0; mu < D; ++mu) {
        int x = (i / stride) % L;
        int k = -1;
        if (x > 0) k = i - stride;
        else if (periodic) k = i + (L - 1) * stride;
        if (k >= 0) h += (double)J[(size_t)k * D + mu] * s[k];
        stride *= L;
    }
    return h;
}

int or_metropolis(int kind, int N, int D, int L, int periodic, const float *J, int64_t R,
                  int sweeps, double beta, uint64_t seed, int8_t *spins, double *E,
                  double *trace_E, int64_t *flags)
{
    int64_t nflag = 0;
    for (int64_t r = 0; r < R; ++r) {
        int8_t *s = spins + (size_t)r * N;
        double e = E[r];
        for (int w = 0; w < sweeps; ++w) {
            for (int i = 0; i < N; ++i) {
                double h = local_field(kind, N, D, L, periodic, J, s, i);
                double dE = 2.0 * s[i] * h;
                double acc = exp(-beta * dE);
                double u = or_uniform(seed, (uint32_t)r, (uint32_t)i, 2, (uint32_t)w);
                if (fabs(u - acc) < 1e-12) ++nflag;
                if (u < acc) { s[i] = (int8_t)-s[i]; e += dE; }
            }
            if (trace_E) trace_E[(size_t)w * R + r] = e;
        }
        E[r] = e;
    }
    if (flags) *flags = nflag;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Overlap distribution (Eq. overlap_distribution): q = s1.s2 / N over       */
/* pairs (2k, 2k+1); hist[(N*q + N)/2] counts, N+1 bins.                     */
/* ------------------------------------------------------------------------ */
void or_overlap_hist(int N, int64_t B, const int8_t *spins, int64_t *hist)
{
    for (int i = 0; i <= N; ++i) hist[i] = 0;
    for (int64_t k = 0; 2 * k + 1 < B; ++k) {
        const int8_t *a = spins + (size_t)(2 * k) * N, *b = spins + (size_t)(2 * k + 1) * N;
        int dot = 0;
        for (int i = 0; i < N; ++i) dot += a[i] * b[i];
        hist[(dot + N) / 2] += 1;
    }
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
