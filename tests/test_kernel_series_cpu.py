"""The FP32 polynomials of the Magnus-4 step, read from the kernel source, against the
functions they stand for on the series range th <= 0.2 (t = th^2 <= 0.04): tan(th)/th
(the tracked-norm series step), cos(th) - 1 and sin(th)/th (the wide-range step).
No GPU: the coefficients are parsed from the header and evaluated in FP64."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = open(os.path.join(ROOT, "paper_1704_08919_gb300", "csrc", "pp_policies.cuh")).read()
T = np.linspace(0.0, 0.04, 4001)
TH = np.sqrt(T)


def body(name, start):
    """The source of the device function `name` after position `start`."""
    i = SRC.index(name, start)
    return SRC[i:SRC.index("}", i)]


def horner_float_constants(src):
    """The float literals of a Horner chain in source order (innermost first)."""
    return [float(x.rstrip("f")) if "/" not in x else eval(x.replace("f", ""))
            for x in re.findall(r"(-?[0-9.]+(?:e-?[0-9]+)?f(?:\s*/\s*[0-9.]+f)?)", src)]


def test_tan_series_matches_tan_over_th():
    c = horner_float_constants(body("float tanc(float t)", SRC.index("struct TanSeries")))
    assert len(c) == 4  # a cubic in t
    r = np.full_like(T, np.float32(c[0]), dtype=np.float64)
    for k in c[1:]:
        r = T * r + np.float32(k)
    ref = np.ones_like(T)
    ref[1:] = np.tan(TH[1:]) / TH[1:]
    assert np.abs(r / ref - 1).max() < 2e-9


def test_trig_series_float_match_cos_and_sinc():
    start = SRC.index("struct TrigSeries<float>")
    cm1_src = body("float cm1(float t)", start)
    sinc_src = body("float sinc(float t)", start)
    # cm1 = t * (-1/2 + t (1/24 - t/720)), sinc = 1 + t (-1/6 + t/120)
    assert re.search(r"-1\.0f\s*/\s*720\.0f", cm1_src) and re.search(r"1\.0f\s*/\s*24\.0f", cm1_src)
    assert re.search(r"1\.0f\s*/\s*120\.0f", sinc_src) and re.search(r"-1\.0f\s*/\s*6\.0f", sinc_src)
    cm1 = T * (T * (T * (-1.0 / 720.0) + 1.0 / 24.0) - 0.5)
    sinc = T * (T * (1.0 / 120.0) - 1.0 / 6.0) + 1.0
    assert np.abs(cm1 - (np.cos(TH) - 1.0)).max() < 1e-10
    s_ref = np.ones_like(T)
    s_ref[1:] = np.sin(TH[1:]) / TH[1:]
    assert np.abs(sinc - s_ref).max() < 2e-8
