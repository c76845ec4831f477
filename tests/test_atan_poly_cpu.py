"""Pins the polynomial atan used by the refinement kernels (indexing.cu) to
np.arctan: the coefficients are read from the CUDA source and evaluated with
FP32 Horner steps, as the kernel does (there with fused multiply-adds)."""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2009_00735_gb300", "csrc", "indexing.cu")


def coefficients():
    src = open(SRC).read()
    body = src[src.index("float atan01(float t)"):]
    body = body[:body.index("return t * p;")]
    vals = [float(v) for v in re.findall(r"(-?\d\.\d+e[-+]\d+)f", body)]
    assert len(vals) == 8
    return [np.float32(v) for v in vals]   # highest power first


def atan01(t):
    c = coefficients()
    t = np.asarray(t, np.float32)
    s = t * t
    p = np.full_like(t, c[0])
    for v in c[1:]:
        p = p * s + v
    return t * p


def atan2_deg(y, x):
    y = np.asarray(y, np.float32)
    x = np.asarray(x, np.float32)
    ax, ay = np.abs(x), np.abs(y)
    a = atan01(np.minimum(ax, ay) / np.maximum(ax, ay))
    a = np.where(ay > ax, np.float32(np.pi / 2) - a, a)
    a = np.where(x < 0, np.float32(np.pi) - a, a)
    a = np.where(y < 0, -a, a)
    return a * np.float32(180.0 / np.pi)


def test_atan01_error_bound():
    t = np.linspace(0.0, 1.0, 1_000_001, dtype=np.float32)
    err = np.abs(atan01(t).astype(np.float64) - np.arctan(t.astype(np.float64)))
    assert err.max() < 2.5e-7


def test_atan2_deg_all_octants():
    rng = np.random.default_rng(5)
    v = rng.standard_normal((200_000, 2)).astype(np.float32)
    got = atan2_deg(v[:, 0], v[:, 1]).astype(np.float64)
    want = np.degrees(np.arctan2(v[:, 0].astype(np.float64), v[:, 1].astype(np.float64)))
    assert np.abs(got - want).max() < 3e-5
    # axes and diagonals
    assert atan2_deg(0.0, 1.0) == 0.0
    assert abs(atan2_deg(1.0, 0.0) - 90.0) < 1e-5
    assert abs(atan2_deg(0.0, -1.0) - 180.0) < 1e-5
    assert abs(atan2_deg(-1.0, -1.0) + 135.0) < 2e-5
