"""FP64 CPU oracle of the aberration-correction extension: a Zernike pupil phase
screen in the sensor plane, the sharpness of the reconstructed volume, and the
gradient of that sharpness with respect to the reconstruction distance z and the
15 Zernike coefficients.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper names aberration correction in post-processing as one advantage of
the holographic (phase-resolved) volume but gives no method (introduction).  The
reading used here:

* A phase screen exp(i phi(x', y')) multiplies each rescaled interferogram
  together with the input chirp of Eq. 6, phi = sum_j c_j Z_j(rho, theta) with
  Noll-ordered Zernike polynomials (Noll 1976, J. Opt. Soc. Am. 66, 207),
  j = 1..15 (radial order n <= 4), RMS-normalised on the unit disk.  Sensor
  coordinates x'_n = (n - N_x/2) d, rho = r / R with R = min(N_x, N_y) d / 2;
  the polynomials are continued outside the disk, with no mask.
* The sharpness loss of an intensity volume P_v = |V_v|^2 is
  L = - sum_v P_v^2 / (sum_v P_v)^2 (scale invariant, so |K|^2 drops out).
* Its gradient comes from one adjoint pass.  W = 2 |K|^2 (dL/dP) V~ with
  V~ = A F (c P u) (axial DFT A of Eq. 7 after the centred DFT F of Eq. 6, c the
  input chirp, P the pupil factor, u the rescaled frames of Eq. 5).  Y_t = the
  adjoint F^H A^H W, zero outside the window.  Q = sum_t conj(Y_t) u_t.  Then
  M = -Im(c P Q) and
      dL/dc_j = sum_{x',y'} Z_j M,
      dL/dz   = sum_{x',y'} (pi |K| r_pix^2 / z) M,   r_pix^2 = (n-N_x/2)^2 + (l-N_y/2)^2,
  because d(phase of c)/dz = pi d^2 r_pix^2 / (lambda_1 z^2) and neither the
  output chirp nor K changes |V|^2 up to a scale.
"""

from __future__ import annotations

from typing import Optional, Sequence, Tuple

import numpy as np
import scipy.fft as sfft

from .ssoct_oracle import (_centred, axial, fresnel, intensity, rescale, scale_factors,
                           start_wavelength)

N_ZERNIKE = 15


def zernike(j: int, rho: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Z_j(rho, theta), Noll index j = 1..15, normalised so that the mean of Z_j^2
    over the unit disk is 1 (Noll 1976, Table 1)."""
    r2 = rho * rho
    if j == 1:
        return np.ones_like(rho)
    if j == 2:
        return 2.0 * rho * np.cos(theta)
    if j == 3:
        return 2.0 * rho * np.sin(theta)
    if j == 4:
        return np.sqrt(3.0) * (2.0 * r2 - 1.0)
    if j == 5:
        return np.sqrt(6.0) * r2 * np.sin(2.0 * theta)
    if j == 6:
        return np.sqrt(6.0) * r2 * np.cos(2.0 * theta)
    if j == 7:
        return np.sqrt(8.0) * (3.0 * r2 - 2.0) * rho * np.sin(theta)
    if j == 8:
        return np.sqrt(8.0) * (3.0 * r2 - 2.0) * rho * np.cos(theta)
    if j == 9:
        return np.sqrt(8.0) * r2 * rho * np.sin(3.0 * theta)
    if j == 10:
        return np.sqrt(8.0) * r2 * rho * np.cos(3.0 * theta)
    if j == 11:
        return np.sqrt(5.0) * (6.0 * r2 * r2 - 6.0 * r2 + 1.0)
    if j == 12:
        return np.sqrt(10.0) * (4.0 * r2 - 3.0) * r2 * np.cos(2.0 * theta)
    if j == 13:
        return np.sqrt(10.0) * (4.0 * r2 - 3.0) * r2 * np.sin(2.0 * theta)
    if j == 14:
        return np.sqrt(10.0) * r2 * r2 * np.cos(4.0 * theta)
    if j == 15:
        return np.sqrt(10.0) * r2 * r2 * np.sin(4.0 * theta)
    raise ValueError("Noll index 1..15")


def sensor_polar(nx: int, ny: int, pitch: float) -> Tuple[np.ndarray, np.ndarray]:
    """(rho, theta) of every sensor pixel [ny][nx]: x'_n = (n - N_x/2) d, y'_l the
    same along y, rho = r / R with R = min(N_x, N_y) d / 2."""
    xs = _centred(nx) * pitch
    ys = _centred(ny) * pitch
    x, y = np.meshgrid(xs, ys)
    radius = min(nx, ny) * pitch / 2.0
    return np.hypot(x, y) / radius, np.arctan2(y, x)


def zernike_maps(nx: int, ny: int, pitch: float) -> np.ndarray:
    """Z_1..Z_15 on the sensor grid, [15][ny][nx]."""
    rho, theta = sensor_polar(nx, ny, pitch)
    return np.stack([zernike(j, rho, theta) for j in range(1, N_ZERNIKE + 1)])


def pupil_phase(coeffs: Sequence[float], nx: int, ny: int, pitch: float) -> np.ndarray:
    """phi = sum_j c_j Z_j on the sensor grid (radians), [ny][nx]; coeffs[0] is c_1."""
    c = np.asarray(coeffs, dtype=np.float64)
    if c.size > N_ZERNIKE:
        raise ValueError("at most 15 coefficients")
    maps = zernike_maps(nx, ny, pitch)[: c.size]
    return np.tensordot(c, maps, axes=1) if c.size else np.zeros((ny, nx))


def reconstruct_pupil(frames: np.ndarray, pitch: float, z: float, lambdas: Sequence[float],
                      coeffs: Sequence[float], window: Optional[Tuple[int, int, int, int]] = None,
                      method: str = "fft") -> np.ndarray:
    """The chain of ``reconstruct`` (Eq. 5, Eq. 6, window, Eq. 7) with every rescaled
    frame multiplied by exp(i phi) before the Fresnel transform."""
    nl, ny, nx = frames.shape
    x0, y0, wx, wy = window if window else (0, 0, nx, ny)
    lam1 = start_wavelength(lambdas)
    s = scale_factors(lambdas)
    screen = np.exp(1j * pupil_phase(coeffs, nx, ny, pitch))
    h = np.empty((nl, wy, wx), dtype=np.complex128)
    for t in range(nl):
        h[t] = fresnel(rescale(frames[t], s[t]) * screen, pitch, z, lam1, method=method,
                       rows=slice(y0, y0 + wy), cols=slice(x0, x0 + wx))
    return axial(h, method=method)


def sharpness(p: np.ndarray) -> float:
    """L = - sum P^2 / (sum P)^2 of an intensity volume."""
    p = np.asarray(p, dtype=np.float64)
    s1 = p.sum()
    return float(-(p * p).sum() / (s1 * s1))


def sharpness_loss(frames, pitch, z, lambdas, coeffs, window=None, method: str = "fft") -> float:
    """The loss as its definition: sharpness of |V|^2 of the pupil reconstruction."""
    return sharpness(intensity(reconstruct_pupil(frames, pitch, z, lambdas, coeffs, window, method)))


def _dft_plus(a: np.ndarray) -> np.ndarray:
    """sum_n a_n exp(+2 pi i (m - c)(n - c) / N) over both axes (c = N/2), the sum of Eq. 6."""
    ny, nx = a.shape[-2:]
    return sfft.fftshift(sfft.ifft2(sfft.ifftshift(a, axes=(-2, -1))), axes=(-2, -1)) * (nx * ny)


def _dft_minus(b: np.ndarray) -> np.ndarray:
    """The adjoint of ``_dft_plus``: sum_m b_m exp(-2 pi i (m - c)(n - c) / N)."""
    return sfft.fftshift(sfft.fft2(sfft.ifftshift(b, axes=(-2, -1))), axes=(-2, -1))


def sharpness_gradient(frames: np.ndarray, pitch: float, z: float, lambdas: Sequence[float],
                       coeffs: Sequence[float], window: Optional[Tuple[int, int, int, int]] = None):
    """(L, grad) with grad[0] = dL/dz (per metre) and grad[j] = dL/dc_j, j = 1..15,
    by the adjoint pass described in the module docstring."""
    nl, ny, nx = frames.shape
    x0, y0, wx, wy = window if window else (0, 0, nx, ny)
    rows, cols = slice(y0, y0 + wy), slice(x0, x0 + wx)
    lam1 = start_wavelength(lambdas)
    s = scale_factors(lambdas)
    alpha = pitch * pitch / (lam1 * z)                       # |K|
    cx, cy = _centred(nx), _centred(ny)
    chirp = np.exp(-1j * np.pi * alpha * cy[:, None] ** 2) * np.exp(-1j * np.pi * alpha * cx[None, :] ** 2)
    coeffs = np.zeros(N_ZERNIKE) if coeffs is None else np.asarray(coeffs, dtype=np.float64)
    maps = zernike_maps(nx, ny, pitch)
    screen = np.exp(1j * np.tensordot(coeffs, maps[: coeffs.size], axes=1)) if coeffs.size else np.ones((ny, nx))
    u = np.stack([rescale(frames[t], s[t]) for t in range(nl)])          # [nl][ny][nx], real
    vt = axial(_dft_plus(chirp * screen * u)[:, rows, cols], method="fft")  # V~ [nl][wy][wx]
    p = alpha * alpha * intensity(vt)
    s1, s2 = p.sum(), (p * p).sum()
    loss = -s2 / (s1 * s1)
    dldp = -2.0 * p / (s1 * s1) + 2.0 * s2 / (s1 ** 3)
    w = 2.0 * alpha * alpha * dldp * vt
    ahw = sfft.ifft(w, axis=0) * nl                           # sum_q W_q exp(+2 pi i q t / N)
    b = np.zeros((nl, ny, nx), dtype=np.complex128)
    b[:, rows, cols] = ahw
    y = _dft_minus(b)
    q = (np.conj(y) * u).sum(axis=0)
    m = -np.imag(chirp * screen * q)
    r2 = cy[:, None] ** 2 + cx[None, :] ** 2
    grad = np.empty(1 + N_ZERNIKE)
    grad[0] = np.sum(m * np.pi * alpha * r2 / z)
    grad[1:] = np.tensordot(maps, m, axes=([1, 2], [0, 1]))
    return float(loss), grad
