"""The FP64 oracle against what the paper and the mathematics fix (CPU only)."""

import json
import math
import os

import numpy as np
import pytest

import oracle
import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.json")


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle)


def _round_to(x, ref):
    """Round x to the number of decimals printed in ref."""
    s = repr(float(ref))
    dec = len(s.split(".")[1]) if "." in s and not s.endswith(".0") else 0
    return round(x, dec)


def test_printed_values():
    g = json.load(open(GOLDEN))
    sw = g["synthetic_wavelength"]
    lam = oracle.synthetic_wavelength(sw["lambda1_nm"] * 1e-9, sw["lambda2_nm"] * 1e-9)
    assert _round_to(lam * 1e6, sw["value_um"]) == sw["value_um"]
    cl = g["coherence_length"]
    dz = oracle.coherence_length(cl["lambda1_nm"] * 1e-9, cl["lambda2_nm"] * 1e-9)
    assert _round_to(dz * 1e6, cl["value_um"]) == cl["value_um"]
    for e in g["axial_range"]:
        r = oracle.axial_range(e["lambda1_nm"] * 1e-9, e["lambda2_nm"] * 1e-9, e["nz"])
        assert _round_to(r * 1e3, e["value_mm"]) == e["value_mm"], (e, r)
    it = g["input_throughput"]
    gbps = it["fps"] * it["nx"] * it["ny"] * it["bytes_per_px"] / 1e9
    assert round(gbps) == it["value_GBps"]
    ot = g["output_throughput"]
    gv = ot["volumes_per_s"] * ot["nx"] * ot["ny"] * ot["nz"] / 1e9
    assert round(gv) == ot["value_Gvoxel_per_s"]


def test_fresnel_limit_is_chirp_nyquist():
    """z_b = N d^2 / lambda_1 is the distance at which the input chirp's phase step
    between the two outermost samples reaches pi (the sampling limit)."""
    n, d, lam = 1024, 12e-6, 870e-9
    zb = oracle.fresnel_limit(n, d, lam)
    x = n / 2 * d
    step = math.pi * (x ** 2 - (x - d) ** 2) / (lam * zb)
    assert abs(step - math.pi) < 2 * math.pi / n


def test_reconstructed_pixel_eq4():
    """d' N d = lambda z, and d' grows linearly with lambda (the dilation Eq. 5 undoes)."""
    dp1 = oracle.reconstructed_pixel(800e-9, 0.3, 1024, 20e-6)
    dp2 = oracle.reconstructed_pixel(850e-9, 0.3, 1024, 20e-6)
    assert abs(dp1 * 1024 * 20e-6 - 800e-9 * 0.3) < 1e-18
    assert abs(dp2 / dp1 - 850 / 800) < 1e-14


def test_scale_factors():
    lam = np.array([800e-9, 810e-9, 850e-9])
    s = oracle.scale_factors(lam)
    assert s[0] == 1.0 and abs(s[2] - 850 / 800) < 1e-15
    assert oracle.start_wavelength(lam) == 800e-9


def test_cuts_are_orthogonal_slices():
    rng = np.random.default_rng(3)
    p = rng.uniform(size=(6, 5, 7))
    xy, xz, yz = oracle.cuts(p, 2, 3, 4)
    assert xy.shape == (5, 7) and xz.shape == (6, 7) and yz.shape == (6, 5)
    assert xy[3, 2] == p[4, 3, 2] and xz[4, 2] == p[4, 3, 2] and yz[4, 3] == p[4, 3, 2]


def test_fft_and_dense_agree_midsize():
    rng = np.random.default_rng(19)
    fr = rng.integers(0, 4096, size=(6, 96, 128)).astype(np.uint16)
    lam = np.linspace(800e-9, 850e-9, 6)
    a = oracle.reconstruct(fr, 20e-6, 0.3, lam, method="dense", window=(10, 20, 64, 40))
    b = oracle.reconstruct(fr, 20e-6, 0.3, lam, method="fft", window=(10, 20, 64, 40))
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-12
