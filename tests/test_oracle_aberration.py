"""Pins of the aberration oracle (Zernike pupil, sharpness loss, adjoint gradient).

What pins it, besides itself:
* orthonormality of Z_1..Z_15 on the unit disk (Gauss-Legendre x trapezoid
  quadrature): a wrong coefficient, power or angular factor breaks it;
* textbook values of single polynomials (Noll 1976);
* coefficients all zero: the pupil reconstruction is the plain one;
* piston (Z_1 = 1) is a global phase: its gradient is zero;
* the adjoint pieces pass the dot-product test <F x, w> = <x, F^H w>;
* the gradient matches central finite differences of the loss as defined
  (sharpness of |V|^2 of the full chain, output chirp and K included), for z
  and for every c_j; h = 1e-3 rad and 1e-3 mm.
Planted mistakes in a copy of the module must each fail one of these.
"""

import types

import numpy as np
import pytest

import oracle
import synth
from oracle import aberration as ab

SRC = ab.__file__


def _case(seed=5, nl=16, n=48, window=None):
    w = synth.workload("custom", nx=n, ny=n, nlambda=nl, kind="points", seed=seed)
    rng = np.random.default_rng(seed)
    coeffs = rng.normal(0.0, 0.5, 15)
    return w, coeffs, window


def pin_orthonormal(m):
    x, wx = np.polynomial.legendre.leggauss(40)
    rho = 0.5 * (x + 1.0)
    wr = 0.5 * wx
    th = np.linspace(0.0, 2.0 * np.pi, 64, endpoint=False)
    R, T = np.meshgrid(rho, th, indexing="ij")
    wgt = (wr * rho)[:, None] * (2.0 * np.pi / th.size) / np.pi     # dA / (area of the disk)
    z = np.stack([m.zernike(j, R, T) for j in range(1, 16)])
    gram = np.einsum("iab,jab,ab->ij", z, z, wgt)
    assert np.allclose(gram, np.eye(15), atol=1e-10), np.abs(gram - np.eye(15)).max()


def pin_textbook_values(m):
    assert m.zernike(1, np.array(0.3), np.array(1.0)) == 1.0
    assert np.isclose(m.zernike(2, np.array(1.0), np.array(0.0)), 2.0)
    assert np.isclose(m.zernike(3, np.array(1.0), np.array(np.pi / 2)), 2.0)
    assert np.isclose(m.zernike(4, np.array(1.0), np.array(0.0)), np.sqrt(3.0))
    assert np.isclose(m.zernike(4, np.array(0.0), np.array(0.0)), -np.sqrt(3.0))
    assert np.isclose(m.zernike(11, np.array(0.0), np.array(0.0)), np.sqrt(5.0))
    assert np.isclose(m.zernike(6, np.array(1.0), np.array(0.0)), np.sqrt(6.0))
    assert np.isclose(m.zernike(10, np.array(1.0), np.array(0.0)), np.sqrt(8.0))
    assert np.isclose(m.zernike(14, np.array(1.0), np.array(0.0)), np.sqrt(10.0))
    rho, th = m.sensor_polar(8, 8, 20e-6)
    assert rho[4, 4] == 0.0 and np.isclose(rho[4, 0], 1.0) and np.isclose(th[4, 0], np.pi)


def pin_zero_pupil_is_plain(m):
    w, _, _ = _case(nl=8, n=32)
    v0 = oracle.reconstruct(w.frames, w.pitch, 0.305, w.lambdas, method="fft")
    v1 = m.reconstruct_pupil(w.frames, w.pitch, 0.305, w.lambdas, np.zeros(15))
    assert np.allclose(v0, v1, rtol=0, atol=1e-12 * np.abs(v0).max())


def pin_piston_gradient_zero(m):
    w, c, _ = _case()
    loss, g = m.sharpness_gradient(w.frames, w.pitch, 0.305, w.lambdas, c)
    assert abs(g[1]) <= 1e-10 * np.linalg.norm(g), (g[1], np.linalg.norm(g))


def pin_dot_product(m):
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 12, 10)) + 1j * rng.normal(size=(2, 12, 10))
    y = rng.normal(size=(2, 12, 10)) + 1j * rng.normal(size=(2, 12, 10))
    lhs = np.vdot(y, m._dft_plus(x))
    rhs = np.vdot(m._dft_minus(y), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def pin_finite_differences(m, window=(6, 10, 30, 26)):
    w, c, _ = _case(window=window)
    z = 0.305
    loss, g = m.sharpness_gradient(w.frames, w.pitch, z, w.lambdas, c, window)
    f = lambda zz, cc: m.sharpness_loss(w.frames, w.pitch, zz, w.lambdas, cc, window)  # noqa: E731
    assert np.isclose(loss, f(z, c), rtol=1e-12, atol=0)
    fd = np.empty(16)
    h = 1e-6
    fd[0] = (f(z + h, c) - f(z - h, c)) / (2 * h)
    for j in range(15):
        e = np.zeros(15)
        e[j] = 1e-3
        fd[j + 1] = (f(z, c + e) - f(z, c - e)) / 2e-3
    err = np.abs(fd - g) / np.linalg.norm(g[1:])
    assert err[1:].max() <= 1e-4, err
    assert abs(fd[0] - g[0]) <= 1e-4 * abs(g[0]), (fd[0], g[0])


ALL = [pin_orthonormal, pin_textbook_values, pin_zero_pupil_is_plain, pin_piston_gradient_zero,
       pin_dot_product, pin_finite_differences]


@pytest.mark.parametrize("pin", ALL, ids=[p.__name__ for p in ALL])
def test_aberration_pin(pin):
    pin(ab)


MUTATIONS = {
    "z8_coefficient": ("np.sqrt(8.0) * (3.0 * r2 - 2.0) * rho * np.cos(theta)",
                       "np.sqrt(6.0) * (3.0 * r2 - 2.0) * rho * np.cos(theta)"),
    "z11_radial": ("6.0 * r2 * r2 - 6.0 * r2 + 1.0", "6.0 * r2 * r2 - 5.0 * r2 + 1.0"),
    "z13_angle": ("(4.0 * r2 - 3.0) * r2 * np.sin(2.0 * theta)", "(4.0 * r2 - 3.0) * r2 * np.sin(theta)"),
    "radius_full_width": ("radius = min(nx, ny) * pitch / 2.0", "radius = min(nx, ny) * pitch"),
    "pupil_sign": ("screen = np.exp(1j * np.tensordot(coeffs", "screen = np.exp(-1j * np.tensordot(coeffs"),
    "dldp_sign": ("dldp = -2.0 * p / (s1 * s1) + 2.0 * s2", "dldp = 2.0 * p / (s1 * s1) + 2.0 * s2"),
    "w_factor": ("w = 2.0 * alpha * alpha * dldp * vt", "w = alpha * alpha * dldp * vt"),
    "adjoint_axial_direction": ("ahw = sfft.ifft(w, axis=0) * nl", "ahw = sfft.fft(w, axis=0)"),
    "adjoint_lateral_direction": ("y = _dft_minus(b)", "y = _dft_plus(b) / (nx * ny)"),
    "m_real_part": ("m = -np.imag(chirp * screen * q)", "m = np.real(chirp * screen * q)"),
    "z_gradient_missing_alpha": ("grad[0] = np.sum(m * np.pi * alpha * r2 / z)", "grad[0] = np.sum(m * np.pi * r2 / z)"),
    "window_ignored": ("b[:, rows, cols] = ahw", "b[:, :ahw.shape[1], :ahw.shape[2]] = ahw"),
}


def _mutant(name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation {name}: pattern not unique"
    src = src.replace(old, new)
    mod = types.ModuleType(f"aberration_mutant_{name}")
    mod.__file__ = SRC
    mod.__package__ = "oracle"
    exec(compile(src, f"<mutant {name}>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    mod = _mutant(name, *MUTATIONS[name])
    failed = []
    for pin in ALL:
        try:
            pin(mod)
        except (AssertionError, ValueError, IndexError):
            failed.append(pin.__name__)
    assert failed, f"mutation {name} passed every pin"
