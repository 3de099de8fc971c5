"""FP64 CPU oracle: chromatic rescale (Eq. 5) -> discrete Fresnel transform (Eq. 6)
-> sweep-axis Fourier transform (Eq. 7) -> |.|^2 and three orthogonal cuts.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy/scipy in
float64 / complex128, written from the paper's equations in the paper's order:

* Eq. 3 (axial range), Eq. 4 (reconstructed pixel), the z >= z_b validity bound
  stated under Eq. 6: small closed forms.
* Eq. 5: each interferogram is resampled by linear interpolation onto a grid of
  the same size whose pitch is lambda_t d / lambda_1, i.e. the value at pixel i is
  the input at position c + (i - c) lambda_t / lambda_1.
* Eq. 6: the Fresnel integral with lambda_1, k_1 for every frame, discretised on
  centred grids x'_n = (n - c) d (sensor) and x_m = (m - c) d' (hologram), with d'
  from Eq. 4.  Expanding (x - x')^2 gives prefactor * output chirp *
  sum_n input chirp * exp(+2 pi i (m - c)(n - c) / N): the oracle evaluates that
  sum either with dense DFT matrices (the brute-force sum as a matrix product)
  or with a centred FFT.
* Eq. 7: rectangular gate of N_lambda consecutive frames, transform over the
  frame index with kernel exp(-2 pi i q t / N_lambda), no normalisation.
* The envelope is formed as |.|^2 (the cut formulas printed after Eq. 7).

Readings where the paper is silent are listed in the repository's design notes;
the ones visible in this code: lambda_1 = lambdas[0]; the resampling origin and
the Fresnel grid centre are both the pixel c = N/2; taps that fall outside the
frame read as 0; no 1/N anywhere; dx'dy' -> d^2; depth bins are unshifted.
"""

from __future__ import annotations

import os
from typing import Optional, Sequence, Tuple

import numpy as np
import scipy.fft as sfft


# ----------------------------------------------------------------------------
# closed forms (Eq. 3, Eq. 4, z_b)
# ----------------------------------------------------------------------------

# Threads scipy.fft may use (None: all host cores).  Only the timing of the
# oracle changes with it, never a value.
WORKERS = None


def _workers() -> int:
    return WORKERS or os.cpu_count()


def start_wavelength(lambdas: Sequence[float]) -> float:
    """lambda_1: the wavelength of the first frame of the sweep (Eq. 5, Eq. 6)."""
    return float(lambdas[0])


def scale_factors(lambdas: Sequence[float]) -> np.ndarray:
    """lambda_t / lambda_1, the per-frame resampling ratio of Eq. 5."""
    lam = np.asarray(lambdas, dtype=np.float64)
    return lam / lam[0]


def reconstructed_pixel(lam: float, z: float, n: int, pitch: float) -> float:
    """d' = lambda z / (N d), Eq. 4."""
    return lam * z / (n * pitch)


def fresnel_limit(n: int, pitch: float, lambda1: float) -> float:
    """z_b = N d^2 / lambda_1: Eq. 6 is used for z >= z_b (text under Eq. 6)."""
    return n * pitch * pitch / lambda1


def synthetic_wavelength(lambda1: float, lambda2: float) -> float:
    """Lambda = lambda_1 lambda_2 / |lambda_2 - lambda_1| (text under Eq. 3)."""
    return lambda1 * lambda2 / abs(lambda2 - lambda1)


def axial_range(lambda1: float, lambda2: float, nz: int) -> float:
    """Delta z = N_z Lambda / 2, Eq. 3."""
    return nz * synthetic_wavelength(lambda1, lambda2) / 2.0


def coherence_length(lambda1: float, lambda2: float) -> float:
    """delta z ~ lambda_bar^2 / Delta lambda (text under Eq. 3)."""
    lbar = 0.5 * (lambda1 + lambda2)
    return lbar * lbar / abs(lambda2 - lambda1)


# ----------------------------------------------------------------------------
# Eq. 5: chromatic rescale by linear interpolation
# ----------------------------------------------------------------------------

def rescale_taps(n: int, s: float) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """Linear-interpolation taps along one axis for ratio s = lambda_t / lambda_1.

    Output pixel i reads the input at u = c + (i - c) s, c = n / 2: taps
    floor(u) with weight 1 - frac(u) and floor(u) + 1 with weight frac(u).  A tap
    outside [0, n) contributes 0.  Returns (index0, index1, weight0, weight1)
    with indices clipped into range (their weight is 0 where they were clipped).
    """
    c = n / 2.0
    u = c + (np.arange(n, dtype=np.float64) - c) * s
    i0 = np.floor(u)
    a = u - i0
    i0 = i0.astype(np.int64)
    i1 = i0 + 1
    w0 = np.where((i0 >= 0) & (i0 < n), 1.0 - a, 0.0)
    w1 = np.where((i1 >= 0) & (i1 < n), a, 0.0)
    return np.clip(i0, 0, n - 1), np.clip(i1, 0, n - 1), w0, w1


def rescale(frame: np.ndarray, s: float) -> np.ndarray:
    """Eq. 5: I'(x, y) = I(x lambda/lambda_1, y lambda/lambda_1), bilinear, float64.

    ``frame`` is [ny][nx]; the same ratio s applies along both axes.
    """
    ny, nx = frame.shape
    jx0, jx1, wx0, wx1 = rescale_taps(nx, s)
    jy0, jy1, wy0, wy1 = rescale_taps(ny, s)
    f = np.asarray(frame, dtype=np.float64)
    # sum over the four taps of w_y w_x I(tap_y, tap_x)
    return (wy0[:, None] * (wx0[None, :] * f[np.ix_(jy0, jx0)] + wx1[None, :] * f[np.ix_(jy0, jx1)])
            + wy1[:, None] * (wx0[None, :] * f[np.ix_(jy1, jx0)] + wx1[None, :] * f[np.ix_(jy1, jx1)]))


# ----------------------------------------------------------------------------
# Eq. 6: discrete Fresnel transform
# ----------------------------------------------------------------------------

def fresnel_prefactor(pitch: float, z: float, lambda1: float) -> complex:
    """(i / (lambda_1 z)) exp(-i k_1 z) d^2: the constant of Eq. 6 with dx'dy' -> d^2."""
    k1z = 2.0 * np.pi * z / lambda1
    return (1j / (lambda1 * z)) * np.exp(-1j * k1z) * pitch * pitch


def _centred(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.float64) - n / 2.0


def _fresnel_axes(n: int, pitch: float, z: float, lambda1: float):
    """Sensor coordinates x'_n, hologram coordinates x_m (pitch d' of Eq. 4)."""
    dprime = reconstructed_pixel(lambda1, z, n, pitch)
    return _centred(n) * pitch, _centred(n) * dprime


def fresnel(ip: np.ndarray, pitch: float, z: float, lambda1: float, method: str = "dense",
            rows: Optional[slice] = None, cols: Optional[slice] = None) -> np.ndarray:
    """Eq. 6 on a rescaled frame ``ip`` [ny][nx] -> complex128 hologram.

    H(x_m, y_p) = K exp(-i pi (x_m^2 + y_p^2) / (lambda_1 z))
                  * sum_{n,l} I'(x'_n, y'_l) exp(-i pi (x'_n^2 + y'_l^2) / (lambda_1 z))
                  * exp(+2 pi i [(m - c_x)(n - c_x) / N_x + (p - c_y)(l - c_y) / N_y])
    which is the convolution of Eq. 6 with (x - x')^2 expanded, using
    x_m x'_n / (lambda_1 z) = (m - c)(n - c) / N from Eq. 4.

    method "dense": the double sum as two products with dense DFT matrices built
    from the centred exponent.  method "fft": the same sum with a centred,
    unnormalised inverse-direction FFT (even N only).  ``rows``/``cols`` select an
    output window (hologram-plane pixels).
    """
    ny, nx = ip.shape
    xs, xm = _fresnel_axes(nx, pitch, z, lambda1)
    ys, yp = _fresnel_axes(ny, pitch, z, lambda1)
    lz = lambda1 * z
    a = ip * np.exp(-1j * np.pi * ys[:, None] ** 2 / lz) * np.exp(-1j * np.pi * xs[None, :] ** 2 / lz)
    rows = rows or slice(0, ny)
    cols = cols or slice(0, nx)
    if method == "dense":
        cx, cy = _centred(nx), _centred(ny)
        ex = np.exp(2j * np.pi * np.outer(cx[cols], cx) / nx)     # [wx][nx]
        ey = np.exp(2j * np.pi * np.outer(cy[rows], cy) / ny)     # [wy][ny]
        s = ey @ a @ ex.T
    elif method == "fft":
        if nx % 2 or ny % 2:
            raise ValueError("fft method needs even sizes")
        s = sfft.fftshift(sfft.ifft2(sfft.ifftshift(a), workers=_workers()))
        s = s[rows, cols] * (nx * ny)
    else:
        raise ValueError(method)
    out_chirp = np.exp(-1j * np.pi * yp[rows, None] ** 2 / lz) * np.exp(-1j * np.pi * xm[None, cols] ** 2 / lz)
    return fresnel_prefactor(pitch, z, lambda1) * out_chirp * s


# ----------------------------------------------------------------------------
# Eq. 7: transform over the sweep (one rectangular gate of N_lambda frames)
# ----------------------------------------------------------------------------

def axial(h: np.ndarray, method: str = "dense") -> np.ndarray:
    """V[q] = sum_{t=0}^{N-1} H[t] exp(-2 pi i q t / N), along axis 0, unnormalised."""
    n = h.shape[0]
    if method == "dense":
        t = np.arange(n, dtype=np.float64)
        w = np.exp(-2j * np.pi * np.outer(t, t) / n)
        return (w @ h.reshape(n, -1)).reshape(h.shape)
    if method == "fft":
        return sfft.fft(h, axis=0, workers=_workers())
    raise ValueError(method)


# ----------------------------------------------------------------------------
# whole chain
# ----------------------------------------------------------------------------

def reconstruct(frames: np.ndarray, pitch: float, z: float, lambdas: Sequence[float],
                window: Optional[Tuple[int, int, int, int]] = None, method: str = "dense",
                frame_range: Optional[Tuple[int, int]] = None) -> np.ndarray:
    """uint16 frames [N_lambda][ny][nx] -> complex128 volume V [N_lambda][wy][wx].

    Steps in the paper's order (Fig. 3): Eq. 5 rescale with lambda_t / lambda_1,
    Eq. 6 Fresnel transform with lambda_1 for every frame, crop to the window
    (x0, y0, wx, wy) in hologram-plane pixels, Eq. 7 over the frame index.
    ``frame_range`` (t0, t1) stops after the lateral stage of frames t0..t1-1 and
    returns H for those frames instead (used for sampled timings).
    """
    nl, ny, nx = frames.shape
    if len(lambdas) != nl:
        raise ValueError("one wavelength per frame")
    x0, y0, wx, wy = window if window else (0, 0, nx, ny)
    lam1 = start_wavelength(lambdas)
    s = scale_factors(lambdas)
    t0, t1 = frame_range if frame_range else (0, nl)
    h = np.empty((t1 - t0, wy, wx), dtype=np.complex128)
    for t in range(t0, t1):
        ip = rescale(frames[t], s[t])
        h[t - t0] = fresnel(ip, pitch, z, lam1, method=method,
                            rows=slice(y0, y0 + wy), cols=slice(x0, x0 + wx))
    if frame_range:
        return h
    return axial(h, method=method)


def intensity(v: np.ndarray) -> np.ndarray:
    """|V|^2, the squared envelope whose cuts are printed after Eq. 7."""
    return v.real ** 2 + v.imag ** 2


def cuts(p: np.ndarray, x0: int, y0: int, z0: int):
    """The three orthogonal cuts of the volume P [q][y][x] at (x0, y0, z0):
    P(x, y, z0) [wy][wx], P(x, y0, z) [N_lambda][wx], P(x0, y, z) [N_lambda][wy]."""
    return p[z0, :, :].copy(), p[:, y0, :].copy(), p[:, :, x0].copy()


def pixel_sample(frames: np.ndarray, pitch: float, z: float, lambdas: Sequence[float],
                 pixels: Sequence[Tuple[int, int]]) -> np.ndarray:
    """V[:, y, x] at a few hologram-plane pixels, without forming whole holograms.

    Same chain as ``reconstruct`` (Eq. 5, Eq. 6, Eq. 7) but Eq. 6 is evaluated
    only at the requested output pixels, as the double sum over the sensor, so a
    full-size stack can be checked at sampled voxels.  Returns [len(pixels)][N_lambda].
    """
    nl, ny, nx = frames.shape
    lam1 = start_wavelength(lambdas)
    s = scale_factors(lambdas)
    xs, xm = _fresnel_axes(nx, pitch, z, lam1)
    ys, yp = _fresnel_axes(ny, pitch, z, lam1)
    lz = lam1 * z
    cx, cy = _centred(nx), _centred(ny)
    pix = list(pixels)
    ex = np.stack([np.exp(2j * np.pi * cx[x] * cx / nx) for (x, y) in pix])   # [P][nx]
    ey = np.stack([np.exp(2j * np.pi * cy[y] * cy / ny) for (x, y) in pix])   # [P][ny]
    chirp_in = np.exp(-1j * np.pi * ys[:, None] ** 2 / lz) * np.exp(-1j * np.pi * xs[None, :] ** 2 / lz)
    out = np.exp(-1j * np.pi * np.array([yp[y] ** 2 + xm[x] ** 2 for (x, y) in pix]) / lz)
    kpre = fresnel_prefactor(pitch, z, lam1)
    h = np.empty((nl, len(pix)), dtype=np.complex128)
    for t in range(nl):
        a = rescale(frames[t], s[t]) * chirp_in
        rowsum = a @ ex.T                       # [ny][P]: sum over n for each pixel's x
        h[t] = kpre * out * np.einsum("pl,lp->p", ey, rowsum)
    return axial(h, method="dense").T
