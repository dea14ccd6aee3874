"""Host-side logic of bench.py that needs no GPU.

* fit_power, the power alpha of Table 1 (Section 3: Mvps grows as size^alpha):
  an exact power law returns its exponent with zero error; a perturbed one
  returns the slope of the straight line through its log-log points, whose
  closed form for three points is checked here; per-L alpha is twice the
  per-volume one by construction of size = L^2.
* the default command line times the paper's workload: 10 configurations of a
  256^2 lattice, at least 3 warm-up steps, tolerance 1e-8.
"""
import math
import sys

import pytest

import bench


def test_fit_power_exact_law():
    sizes = [64, 128, 256]
    for alpha in (0.13, 0.25, 0.76):
        mv = [7.0 * (L * L) ** alpha for L in sizes]
        a, se = bench.fit_power(sizes, mv)
        assert abs(a - alpha) <= 1e-12 and se <= 1e-12


def test_fit_power_three_points_closed_form():
    # x = log L^2 at L = 64, 128, 256 is equally spaced (step h = 2 log 2), so the
    # least-squares slope is (y3 - y1) / (2 h) and the middle residual carries all
    # of the scatter: r2 = y2 - (y1 + y3) / 2 with residuals (-r2/3, 2 r2/3, -r2/3)
    sizes = [64, 128, 256]
    y = [math.log(464.0), math.log(498.0), math.log(714.0)]
    a, se = bench.fit_power(sizes, [math.exp(v) for v in y])
    h = 2 * math.log(2.0)
    assert abs(a - (y[2] - y[0]) / (2 * h)) <= 1e-12
    r2 = y[1] - (y[0] + y[2]) / 2
    ssr = (r2 / 3) ** 2 + (2 * r2 / 3) ** 2 + (r2 / 3) ** 2
    assert abs(se - math.sqrt(ssr / 1 / (2 * h * h))) <= 1e-12


def test_default_command_line(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    args = bench.parse()
    assert (args.configs, args.gpus, args.impl, args.coarse_mma) == (10, 1, "native", 1)
    assert args.warmup >= 3 and args.steps >= 1
    assert (bench.L, bench.NCONF, bench.TOL) == (256, 10, 1e-8)
