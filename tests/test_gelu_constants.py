"""The constants of the BF16 path's GELU, read from the CUDA header and
checked on the CPU.

The device code evaluates Phi(v) = (1 + erf(v / sqrt 2)) / 2 by Abramowitz &
Stegun, Handbook of Mathematical Functions, formula 7.1.26: erf(z) = 1 - t
(a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^{-z^2}, t = 1 / (1 + p z), with
|error| <= 1.5e-7 for z >= 0.  Here the formula is evaluated in FP64 with the
numbers as they appear in the header (so a mistyped digit fails), against
scipy's erf, and the header's other constants (1/sqrt 2, log2(e)/2,
1/sqrt(2 pi)) are checked against their definitions.  The device
implementation itself is measured against CUDA's erff by sg_gelu_selfcheck
(GPU test).
"""
import math
import os
import re

import numpy as np
import pytest

HEADER = os.path.join(os.path.dirname(__file__), "..", "paper_2606_22984_gb300", "csrc",
                      "sg_internal.cuh")


def _gelu_as_source():
    src = open(HEADER).read()
    i = src.index("__device__ __forceinline__ float gelu_as(")
    return src[i:src.index("\n}\n", i)]


def _floats(text):
    return [float(x) for x in re.findall(r"-?\d+\.\d+(?:e-?\d+)?(?=f)", text)]


def test_abramowitz_stegun_constants_reach_their_bound():
    scipy_special = pytest.importorskip("scipy.special")
    body = _gelu_as_source()
    # the polynomial line: innermost coefficient first, as written in Horner form
    poly = body[body.index("const float poly"):body.index(";", body.index("const float poly"))]
    a5, a4, a3, a2, a1 = _floats(poly)
    p_line = body[body.index("const float t"):body.index(";", body.index("const float t"))]
    p = _floats(p_line)[0]  # rcp(fmaf(p, z, 1.0))
    z = np.linspace(0.0, 9.0, 200001)
    t = 1.0 / (1.0 + p * z)
    erf_as = 1.0 - t * (a1 + t * (a2 + t * (a3 + t * (a4 + t * a5)))) * np.exp(-z * z)
    err = np.abs(erf_as - scipy_special.erf(z)).max()
    assert err <= 1.5e-7, err
    # and not trivially: a perturbed coefficient breaks the bound
    t2 = 1.0 / (1.0 + p * z)
    bad = 1.0 - t2 * (a1 * 1.001 + t2 * (a2 + t2 * (a3 + t2 * (a4 + t2 * a5)))) * np.exp(-z * z)
    assert np.abs(bad - scipy_special.erf(z)).max() > 1e-5


def test_gelu_scale_constants():
    body = _gelu_as_source()
    e_line = body[body.index("const float e"):body.index(";", body.index("const float e"))]
    (c_exp,) = _floats(e_line)
    assert abs(c_exp - (-0.5 * math.log2(math.e))) < 1e-15  # e^{-v^2/2} = 2^{c v^2}
    z_line = body[body.index("const float z"):body.index(";", body.index("const float z"))]
    (c_z,) = _floats(z_line)
    assert abs(c_z - 1.0 / math.sqrt(2.0)) < 1e-15
    d_line = body[body.index("if (dgelu)"):body.index(";", body.index("if (dgelu)"))]
    (c_phi,) = _floats(d_line)
    assert abs(c_phi - 1.0 / math.sqrt(2.0 * math.pi)) < 1e-15
