"""The branch-free arg() of the inverse epilogues (csrc/ofa_math.cuh), on the CPU.

Its coefficients must be the ones the generator script derives, and the
formula, evaluated in float32 exactly as the kernel evaluates it, must stay
within 5e-7 rad of atan2 over all quadrants and magnitudes (the fast 2-ulp
division on the GPU adds at most ~2.4e-7 to the 1.2e-7 of the polynomial).
"""
import os
import re
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2206_12661_gb300", "csrc")
sys.path.insert(0, CSRC)


def header_coefficients():
    src = open(os.path.join(CSRC, "ofa_math.cuh")).read()
    first = re.findall(r"float p = ([-0-9.e]+)f;", src)
    rest = re.findall(r"p = fmaf\(p, t, ([-0-9.e]+)f\);", src)
    return np.array(first + rest, dtype=np.float32)


def arg_f32(y, x, c):
    y = y.astype(np.float32)
    x = x.astype(np.float32)
    ax, ay = np.abs(x), np.abs(y)
    hi, lo = np.maximum(ax, ay), np.minimum(ax, ay)
    a = np.where(hi > 0, lo / np.where(hi > 0, hi, 1), 0).astype(np.float32)
    t = (a * a).astype(np.float32)
    p = np.full_like(a, c[0])
    for ci in c[1:]:
        p = (p * t + ci).astype(np.float32)
    r = (a * p).astype(np.float32)
    r = np.where(ay > ax, np.float32(np.pi / 2) - r, r).astype(np.float32)
    r = np.where(x < 0, np.float32(np.pi) - r, r).astype(np.float32)
    return np.copysign(r, y)


def test_coefficients_come_from_the_generator():
    import gen_atan_poly
    assert np.array_equal(header_coefficients(), gen_atan_poly.fit().astype(np.float32))


def test_branch_free_arg_accuracy():
    rng = np.random.default_rng(0)
    c = header_coefficients()
    ang = rng.uniform(-np.pi, np.pi, 400_000)
    mag = 10.0 ** rng.uniform(-6, 4, ang.size)
    x, y = mag * np.cos(ang), mag * np.sin(ang)
    # axes, diagonals and signed zeros
    x = np.concatenate([x, [1, -1, 0, 0, 1, -1, 1, -1, 0.0]])
    y = np.concatenate([y, [0, 0, 1, -1, 1, 1, -1, -1, 0.0]])
    got = arg_f32(y, x, c).astype(np.float64)
    ref = np.arctan2(y.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64))
    err = np.abs(np.angle(np.exp(1j * (got - ref))))
    assert err.max() < 5e-7
    assert got[-1] == 0.0  # arg(0) = 0
