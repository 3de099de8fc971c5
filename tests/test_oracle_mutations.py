"""Planted mistakes in a copy of the oracle must each fail at least one pin.

Each case edits the oracle's source text (a dropped term, a wrong sign, a
swapped or transposed operand, a wrong reference wavelength), loads the edited
copy as a separate module on the CPU, and runs the pins against it.  The real
oracle is untouched.
"""

import importlib.util
import os
import types

import pytest

import pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "ssoct_oracle.py")

MUTATIONS = {
    "fresnel_dft_sign": ("np.exp(2j * np.pi * np.outer(cx[cols], cx) / nx)",
                         "np.exp(-2j * np.pi * np.outer(cx[cols], cx) / nx)"),
    "fresnel_fft_direction": ("sfft.ifft2(sfft.ifftshift(a)", "sfft.fft2(sfft.ifftshift(a)"),
    "input_chirp_sign": ("a = ip * np.exp(-1j * np.pi * ys[:, None] ** 2 / lz)",
                         "a = ip * np.exp(+1j * np.pi * ys[:, None] ** 2 / lz)"),
    "input_chirp_x_dropped": ("* np.exp(-1j * np.pi * xs[None, :] ** 2 / lz)\n", "\n"),
    "output_chirp_dropped": ("out_chirp = np.exp(-1j * np.pi * yp[rows, None] ** 2 / lz) * np.exp(-1j * np.pi * xm[None, cols] ** 2 / lz)",
                             "out_chirp = 1.0"),
    "pitch_squared_dropped": ("* np.exp(-1j * k1z) * pitch * pitch", "* np.exp(-1j * k1z) * pitch"),
    "dft_operands_transposed": ("s = ey @ a @ ex.T", "s = ex @ a.T @ ey.T"),
    "axial_sign": ("w = np.exp(-2j * np.pi * np.outer(t, t) / n)", "w = np.exp(2j * np.pi * np.outer(t, t) / n)"),
    "axial_fft_inverse": ("return sfft.fft(h, axis=0", "return sfft.ifft(h, axis=0"),
    "rescale_ratio_inverted": ("return lam / lam[0]", "return lam[0] / lam"),
    "rescale_origin_corner": ("    c = n / 2.0\n    u = c + (np.arange(n, dtype=np.float64) - c) * s",
                              "    c = 0.0\n    u = c + (np.arange(n, dtype=np.float64) - c) * s"),
    "rescale_clamp_not_zero": ("w0 = np.where((i0 >= 0) & (i0 < n), 1.0 - a, 0.0)", "w0 = 1.0 - a"),
    "rescale_weights_swapped": ("w0 = np.where((i0 >= 0) & (i0 < n), 1.0 - a, 0.0)\n    w1 = np.where((i1 >= 0) & (i1 < n), a, 0.0)",
                                "w0 = np.where((i0 >= 0) & (i0 < n), a, 0.0)\n    w1 = np.where((i1 >= 0) & (i1 < n), 1.0 - a, 0.0)"),
    "rescale_axes_swapped": ("jx0, jx1, wx0, wx1 = rescale_taps(nx, s)\n    jy0, jy1, wy0, wy1 = rescale_taps(ny, s)",
                             "jx0, jx1, wx0, wx1 = rescale_taps(ny, s)\n    jy0, jy1, wy0, wy1 = rescale_taps(nx, s)"),
    "rescale_skipped": ("ip = rescale(frames[t], s[t])", "ip = np.asarray(frames[t], dtype=np.float64)"),
    "lambda_t_in_fresnel": ("h[t - t0] = fresnel(ip, pitch, z, lam1,", "h[t - t0] = fresnel(ip, pitch, z, lambdas[t],"),
    "reconstructed_pixel_wrong_n": ("return lam * z / (n * pitch)", "return lam * z / pitch"),
    "intensity_imag_dropped": ("return v.real ** 2 + v.imag ** 2", "return v.real ** 2"),
    "intensity_magnitude_not_squared": ("return v.real ** 2 + v.imag ** 2", "return np.sqrt(v.real ** 2 + v.imag ** 2)"),
    "intensity_complex_square": ("return v.real ** 2 + v.imag ** 2", "return (v * v).real"),
    "cuts_xz_yz_swapped": ("p[:, y0, :].copy(), p[:, :, x0].copy()", "p[:, :, x0].copy(), p[:, y0, :].copy()"),
}


def _load_mutant(name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation {name}: pattern not found"
    src = src.replace(old, new, 1)
    mod = types.ModuleType(f"oracle_mutant_{name}")
    mod.__file__ = SRC
    exec(compile(src, f"<mutant {name}>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    mutant = _load_mutant(name, old, new)
    failed = []
    for pin in pins.ALL_PINS:
        try:
            pin(mutant)
        except Exception:  # an assertion or a shape error both count as caught
            failed.append(pin.__name__)
    assert failed, f"planted mistake {name} passed every pin"
