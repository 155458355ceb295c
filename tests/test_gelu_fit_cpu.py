"""The BF16 form's GELU coefficients, checked on the CPU against the closed form.

The device GELU is 0.5 x (1 + tanh(x P(x^2))) with a fitted degree-4 P (the logistic form
of the normal CDF).  This reads P's coefficients from the device source, evaluates the
form in FP64 with an exact tanh and compares it with 0.5 x (1 + erf(x / sqrt 2)): the fit
error stays within 5e-6 on [-12, 12], and the form saturates to x and to 0 beyond (u = x
P(x^2) increasing), so that a mistyped constant fails here without a GPU.  The hardware
tanh's own error is covered by the GPU test.
"""
import math
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2509_10466_gb300", "csrc",
                   "common.cuh")


def coefficients():
    body = open(SRC).read()
    body = body[body.index("float gelu_as(float x)"):]
    body = body[:body.index("\n}")]
    c = []
    for lead, const in re.findall(r"fmaf\((?:p|([-+0-9.eE]+)f), x2, ([-+0-9.eE]+)f\)", body):
        if lead:
            c.append(float(lead))
        c.append(float(const))
    assert len(c) == 5, c
    return np.array(c, dtype=np.float32).astype(np.float64)  # highest degree first, as stored


def form(x, c):
    x2 = x * x
    p = c[0]
    for k in c[1:]:
        p = p * x2 + k
    return 0.5 * x * (1.0 + np.tanh(x * p))


def gelu(x):
    return 0.5 * x * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))


def test_fit_within_5e6_on_the_fitted_range():
    c = coefficients()
    x = np.linspace(-12.0, 12.0, 240001)
    assert np.abs(form(x, c) - gelu(x)).max() <= 5e-6


def test_argument_increasing_and_saturation():
    c = coefficients()
    x = np.linspace(0.0, 40.0, 400001)
    x2 = x * x
    p = c[0]
    for k in c[1:]:
        p = p * x2 + k
    u = x * p
    assert np.all(np.diff(u) > 0)  # u(x) = x P(x^2) increasing, so sigmoid(2u) is monotone
    big = np.array([30.0, 100.0, 1e4])
    assert np.allclose(form(big, c), big, rtol=0, atol=0)
    assert np.all(form(-big, c) == 0.0)



def h2_coefficients():
    """The polynomial of the FP16 hidden-activation GELU (gelu_h2), highest degree first."""
    body = open(SRC).read()
    body = body[body.index("__half2 gelu_h2(__half2 x)"):]
    body = body[:body.index("\n}")]
    c = []
    for lead, const in re.findall(
            r"__hfma2\((?:p|__float2half2_rn\(([-+0-9.eE]+)f\)), x2, __float2half2_rn\(([-+0-9.eE]+)f\)\)", body):
        if lead:
            c.append(float(lead))
        c.append(float(const))
    return np.array(c, dtype=np.float32).astype(np.float64)


def test_fp16_form_uses_the_pinned_fit():
    """The FP16 hidden-activation GELU evaluates the same fitted polynomial as the FP32 one
    (whose fit the tests above pin); only the arithmetic differs (covered on the GPU)."""
    assert np.array_equal(h2_coefficients(), coefficients())
