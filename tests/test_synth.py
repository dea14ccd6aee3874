"""Pins of the seeded input generators (CPU only).

* 2D U(1) lattice gauge theory is exactly solvable: the plaquette average is
  <Re U_P> = I_1(beta) / I_0(beta) (0.912359 at beta = 6.0);
* the topological charge (1/2pi) sum arg U_P of a periodic field is an integer;
* the von Mises sampler has E[cos theta] = I_1(k)/I_0(k), E[cos 2 theta] = I_2(k)/I_0(k);
* the arithmetic-only exponential agrees with libm to a few ulp;
* fields are reproducible and match the fingerprints the m0 table was tuned on.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import iv

import synth


def plaquettes(U):
    return U[:, :, 0] * np.roll(U[:, :, 1], -1, axis=1) * np.conj(np.roll(U[:, :, 0], -1, axis=0)) * np.conj(U[:, :, 1])


def test_plaquette_matches_exact_solution():
    vals = [plaquettes(synth.gauge_field(64, c, cache=False)).real.mean() for c in range(2)]
    exact = iv(1, 6.0) / iv(0, 6.0)
    assert abs(exact - 0.912359) < 1e-6
    assert abs(np.mean(vals) - exact) < 0.004


def test_topological_charge_integer_and_unit_links():
    U = synth.gauge_field(32, 1, cache=False)
    q = np.angle(plaquettes(U)).sum() / (2 * np.pi)
    assert abs(q - round(q)) < 1e-9
    assert np.abs(np.abs(U) - 1).max() < 1e-14


@pytest.mark.parametrize("kappa", [0.3, 3.0, 12.0])
def test_vonmises_moments(kappa):
    cs = synth.vonmises(kappa, 200000, 5)
    th = np.arctan2(cs[:, 1], cs[:, 0])
    assert abs(np.cos(th).mean() - iv(1, kappa) / iv(0, kappa)) < 0.006
    assert abs(np.cos(2 * th).mean() - iv(2, kappa) / iv(0, kappa)) < 0.006
    assert abs(np.sin(th).mean()) < 0.006


def test_arithmetic_exp():
    xs = np.concatenate([np.linspace(-700, 700, 2001), np.linspace(-1, 1, 2001)])
    err = max(abs(synth.det_exp(x) / math.exp(x) - 1) for x in xs)
    assert err < 1e-15


def test_fields_reproducible_and_fingerprinted():
    a = synth.heatbath(16, 16, 6.0, 50, 3)
    b = synth.heatbath(16, 16, 6.0, 50, 3)
    assert np.array_equal(a, b)
    t = synth.m0_table()
    for key in ("16:0", "32:0"):
        L, c = (int(v) for v in key.split(":"))
        assert synth.check_fingerprint(L, c, synth.gauge_field(L, c, cache=False)), key


def test_complex_gaussian_and_z4():
    z = synth.complex_gaussian((200000,), 1, 2)
    assert abs(np.mean(np.abs(z) ** 2) - 1) < 0.01
    assert abs(np.mean(z.real * z.imag)) < 0.01
    q = synth.z4_noise((1000,), 3)
    assert np.allclose(np.abs(q), 1) and set(np.round(q ** 4, 12).real) == {1.0}


def test_m0_table_puts_spectrum_edge_at_target():
    t = synth.m0_table()
    for key, e in t["entries"].items():
        assert abs(e["m0"] + e["lambda_min_re"] - 1e-3) < 1e-12, key
        assert e["min_abs_eig"] >= 1e-3 * (1 - 1e-9), key
