"""Mutation test of the oracle's pins.

Each case plants one plausible mistake in a copy of oracle/sg_oracle.c (an
off-by-one in the band or the sink, an unbiased LayerNorm variance, a dropped
bias, a wrong GELU constant, a flipped head sign, a wrong attention scale, a
wrong lattice neighbour, a double-counted SK bond, wrong LayerNorm, attention,
GELU or head backward, a wrong Metropolis field, a flipped MH ratio, a missing
ln B in F_IS, a shifted token or position index, swapped Philox words or key
constants, a missing half-step in the uniform, a flipped likelihood weight, a
patched draw one class off, a class interval that includes its own class),
builds it, and runs the pins of tests/test_oracle_pins.py against it: at
least one pin must fail for every mistake.  The unmodified source built the
same way must pass them all.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "sg_oracle.c")

# name: [(text in sg_oracle.c, replacement)], every text must occur
MUTANTS = {
    "band_off_by_one": [("return (t - k <= c->W) || (k < c->S);",
                         "return (t - k < c->W) || (k < c->S);")],
    "sink_off_by_one": [("return (t - k <= c->W) || (k < c->S);",
                         "return (t - k <= c->W) || (k <= c->S);")],
    "ln_unbiased_variance": [("    var /= d;\n", "    var /= (d - 1);\n")],
    "dropped_bias": [("double s = b ? b[o] : 0.0;", "double s = 0.0;")],
    "gelu_constant": [("static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }",
                       "static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / 2.0)); }")],
    "head_sign": [("return z[1] - z[0];", "return z[0] - z[1];")],
    "attention_scale": [("double inv_sqrt = 1.0 / sqrt((double)dh);",
                         "double inv_sqrt = 1.0 / (double)dh;")],
    "ea_wrap_neighbour": [("return periodic ? i - (L - 1) * stride : -1;",
                           "return periodic ? i - (L - 2) * stride : -1;")],
    "sk_double_count": [("for (int j = i + 1; j < N; ++j) e -=", "for (int j = 0; j < N; ++j) e -=")],
    "ln_backward": [("dx_accum[i] += rstd * (dy[i] * g[i] - m1 - xhat[i] * m2);",
                     "dx_accum[i] += rstd * (dy[i] * g[i] - m1 + xhat[i] * m2);")],
    "attention_backward": [("double ds = prob[k] * (dprob[k] - dot) * inv_sqrt;",
                            "double ds = prob[k] * dprob[k] * inv_sqrt;")],
    "gelu_backward": [("x * exp(-0.5 * x * x) / sqrt(2.0 * M_PI)", "x * exp(-x * x) / sqrt(2.0 * M_PI)")],
    "head_backward": [("double dl = coeff * sl * sigmoid(-sl * T->logit[t]);",
                       "double dl = coeff * sl * sigmoid(sl * T->logit[t]);")],
    "metropolis_field": [("double dE = 2.0 * s[i] * h;", "double dE = s[i] * h;")],
    "mh_ratio_sign": [("double la = (-beta * E[p] - logq[p]) - (-beta * e - lq);",
                       "double la = (-beta * E[p] + logq[p]) - (-beta * e + lq);")],
    "fis_without_ln_B": [("out[1] = (double)(-(mx + logl(sw) - logl((long double)B)) / beta);",
                          "out[1] = (double)(-(mx + logl(sw)) / beta);")],
    "token_index": [("embed(c, m, t, t == 0 ? 0 : token_of(c, s, t - 1), H + (size_t)t * d);",
                     "embed(c, m, t, token_of(c, s, t), H + (size_t)t * d);")],
    "position_index": [("x[dt + i] = m->pos[(size_t)t * dp + i];",
                        "x[dt + i] = m->pos[(size_t)(t > 0 ? t - 1 : 0) * dp + i];")],
    "philox_word_swap": [("c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;", "c0 = n0; c1 = lo0; c2 = n2; c3 = lo1;")],
    "philox_key_schedule": [("if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }",
                             "if (r > 0) { k0 += PHILOX_W1; k1 += PHILOX_W0; }")],
    "uniform_half_step": [("return ((double)(out[0] >> 8) + 0.5) * (1.0 / 16777216.0);",
                           "return ((double)(out[0] >> 8)) * (1.0 / 16777216.0);")],
    "likelihood_weight_sign": [("coeff[b] = (a * E[b] + c * logq[b] - meanL - w) / (double)B;",
                                "coeff[b] = (a * E[b] + c * logq[b] - meanL + w) / (double)B;")],
    "fq_without_beta": [("out[0] = (double)(sumL / B / beta);", "out[0] = (double)(sumL / B);")],
    "patched_draw_next_class": [("if (!found && u < cdf) { k = j; found = 1; }",
                                 "if (!found && u < cdf) { k = j + 1; found = 1; }")],
    "cdf_lo_includes_class": [("for (int j = 0; j < k; ++j) below += exp(lp[j]);",
                               "for (int j = 0; j <= k; ++j) below += exp(lp[j]);")],
}


def _build(text, out):
    gcc = shutil.which("gcc")
    src = out[:-3] + ".c"
    with open(src, "w") as f:
        f.write(text)
    base = [gcc, "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", src, "-o", out, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base, check=True, capture_output=True)


def _run_pins(libpath):
    env = dict(os.environ, SG_ORACLE_LIB=libpath, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    return r.returncode, r.stdout[-2000:]


def _case(name, tmp):
    with open(SRC) as f:
        text = f.read()
    for old, new in MUTANTS.get(name, []):
        assert old in text, f"{name}: text to mutate not found: {old!r}"
        text = text.replace(old, new)
    lib = os.path.join(tmp, f"lib_{name}.so")
    _build(text, lib)
    return (name,) + _run_pins(lib)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_every_planted_mistake_fails_a_pin():
    tmp = tempfile.mkdtemp(prefix="oracle_mutants_")
    names = ["unmodified"] + list(MUTANTS)
    workers = max(1, min(len(names), (os.cpu_count() or 2)))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = {name: (rc, out) for name, rc, out in ex.map(lambda n: _case(n, tmp), names)}
    rc, out = results.pop("unmodified")
    assert rc == 0, "the unmodified oracle failed its pins:\n" + out
    survived = [n for n, (rc, _) in results.items() if rc != 1]
    assert not survived, "mistakes no pin caught (or that broke collection): " + ", ".join(
        f"{n} (rc {results[n][0]})" for n in survived)
