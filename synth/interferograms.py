"""Forward model of an off-axis swept-source recording (test/bench input only).

Recording model (Sec. 2 of the paper, setup paragraph and Fig. 1): the camera
records I = |E + E_LO|^2 for every wavelength of a sweep in which the wavenumber
k = 2 pi / lambda varies linearly with time.  Here

* the local oscillator E_LO is a unit plane wave tilted so that its fringes have
  ``carrier`` cycles across the frame at the first wavelength of the sweep (the
  tilt angle is fixed, so at wavelength lambda_t the fringe count scales as
  lambda_1 / lambda_t);
* the object field E is a sum of paraxial point-source waves,
  a * exp(i [2 k delta + k ((x'-X)^2 + (y'-Y)^2) / (2 z)]), from scatterers at
  lateral position (X, Y) in the object plane a distance z from the sensor and at
  extra round-trip depth delta;
* counts are ``dn * |E + E_LO|^2`` plus read noise (Gaussian) or shot noise
  (Poisson), rounded and clipped to the camera's bit depth, stored as uint16.

Sensor coordinates are x'_n = (n - N/2) d.  Everything is float64 numpy; the
field is built from separable x and y factors so that a 1024 x 1024 x 256 stack
is generated in seconds.  Nothing here reconstructs anything.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Optics shared by every workload: sweep 800 -> 850 nm linear in wavenumber,
# 20 um pixels, 0.3 m object distance, carrier at (N/4, N/4) cycles.
OPTICS = dict(lambda_start=800e-9, lambda_end=850e-9, pitch=20e-6, z=0.3)


def sweep_wavelengths(lambda_start: float, lambda_end: float, n: int) -> np.ndarray:
    """Wavelengths of an n-frame sweep whose wavenumber is linear in time.

    k_t = k_a + t (k_b - k_a) / (n - 1), endpoints included; lambda_t = 2 pi / k_t.
    Frame 0 is at ``lambda_start``.
    """
    ka = 2.0 * np.pi / lambda_start
    kb = 2.0 * np.pi / lambda_end
    if n == 1:
        return np.array([lambda_start])
    k = ka + np.arange(n, dtype=np.float64) * (kb - ka) / (n - 1)
    return 2.0 * np.pi / k


@dataclass
class Scatterer:
    X: float          # object-plane lateral position [m]
    Y: float
    delta: float      # extra round-trip path / 2, i.e. depth [m]
    amp: complex      # complex amplitude relative to |E_LO| = 1


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nlambda: int
    pitch: float
    z: float
    lambdas: np.ndarray
    frames: Optional[np.ndarray]          # uint16 [nlambda][ny][nx]
    scatterers: List[Scatterer] = field(default_factory=list)
    carrier: Tuple[float, float] = (0.0, 0.0)
    window: Tuple[int, int, int, int] = (0, 0, 0, 0)

    @property
    def voxels(self) -> int:
        return self.window[2] * self.window[3] * self.nlambda


def _sensor_axis(n: int, pitch: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) - n / 2.0) * pitch


def _object_field(xs, ys, k, z, scatterers, amps_t):
    """E[y][x] = sum_s A_s u_s(x) v_s(y), built as one (ny x S) @ (S x nx) product."""
    X = np.array([s.X for s in scatterers])
    Y = np.array([s.Y for s in scatterers])
    u = np.exp(1j * k * (xs[None, :] - X[:, None]) ** 2 / (2.0 * z))   # S x nx
    v = np.exp(1j * k * (ys[:, None] - Y[None, :]) ** 2 / (2.0 * z))   # ny x S
    return v @ (amps_t[:, None] * u)


def _record(nx, ny, pitch, z, lambdas, carrier, scatterers, counts_fn, chunk=8):
    """Generic recording loop; counts_fn(intensity, t) -> uint16 frame."""
    xs = _sensor_axis(nx, pitch)
    ys = _sensor_axis(ny, pitch)
    lam0 = lambdas[0]
    # tilt chosen so the fringe count is `carrier` cycles per frame at lam0
    sx = lam0 * carrier[0] / (nx * pitch)
    sy = lam0 * carrier[1] / (ny * pitch)
    amps = np.array([complex(s.amp) for s in scatterers]) if scatterers else None
    deltas = np.array([s.delta for s in scatterers]) if scatterers else None
    out = np.empty((len(lambdas), ny, nx), dtype=np.uint16)
    for t, lam in enumerate(lambdas):
        k = 2.0 * np.pi / lam
        lo_x = np.exp(1j * k * sx * xs)
        lo_y = np.exp(1j * k * sy * ys)
        field_ = lo_y[:, None] * lo_x[None, :]
        if scatterers:
            a_t = amps * np.exp(2j * k * deltas)
            field_ = field_ + _object_field(xs, ys, k, z, scatterers, a_t)
        inten = field_.real ** 2 + field_.imag ** 2
        out[t] = counts_fn(inten, t)
    return out


def point_scatterer_stack(nx, ny, nlambda, scatterers, *, rng, pitch=OPTICS["pitch"],
                          z=OPTICS["z"], lambdas=None, carrier=None, dn=1000.0,
                          read_noise=2.0, bits=12):
    """uint16 stack [nlambda][ny][nx] of point scatterers with Gaussian read noise."""
    if lambdas is None:
        lambdas = sweep_wavelengths(OPTICS["lambda_start"], OPTICS["lambda_end"], nlambda)
    if carrier is None:
        carrier = (nx / 4.0, ny / 4.0)
    top = float(2 ** bits - 1)

    def counts(inten, t):
        c = dn * inten
        if read_noise > 0:
            c = c + rng.normal(0.0, read_noise, size=c.shape)
        return np.clip(np.rint(c), 0.0, top).astype(np.uint16)

    return _record(nx, ny, pitch, z, lambdas, carrier, scatterers, counts), lambdas, carrier


def speckle_stack(nx, ny, nlambda, scatterers, *, rng, pitch=OPTICS["pitch"],
                  z=OPTICS["z"], lambdas=None, carrier=None, mean_dn=2000.0):
    """uint16 stack with Poisson (shot-noise-like) counts around ``mean_dn``."""
    if lambdas is None:
        lambdas = sweep_wavelengths(OPTICS["lambda_start"], OPTICS["lambda_end"], nlambda)
    if carrier is None:
        carrier = (nx / 4.0, ny / 4.0)

    def counts(inten, t):
        c = rng.poisson(mean_dn * inten)
        return np.clip(c, 0, 65535).astype(np.uint16)

    return _record(nx, ny, pitch, z, lambdas, carrier, scatterers, counts), lambdas, carrier


def _random_points(rng, n, nx, pitch, z, lam0, depth_max, amp_lo=1e-3, amp_hi=1.0):
    """n scatterers over the quarter field centred on the object-plane origin.

    The object-plane field of view is lam0 z / pitch (the reconstructed pixel of
    Eq. 4 times N); a quarter of it keeps the +1 order inside the carrier quadrant.
    Amplitudes are log-uniform in [amp_lo, amp_hi] divided by n, which keeps the
    12-bit quantiser out of clipping.
    """
    fov = lam0 * z / pitch
    pts = []
    for _ in range(n):
        X = rng.uniform(-fov / 8.0, fov / 8.0)
        Y = rng.uniform(-fov / 8.0, fov / 8.0)
        d = rng.uniform(0.0, depth_max)
        a = np.exp(rng.uniform(np.log(amp_lo), np.log(amp_hi))) / n
        ph = rng.uniform(0.0, 2.0 * np.pi)
        pts.append(Scatterer(X, Y, d, a * np.exp(1j * ph)))
    return pts


def _speckle_layer(rng, nx, pitch, z, lam0, n_layers=64, per_layer=16, atten=0.3e-3,
                   depth_max=1.2e-3, scale=0.02):
    """Diffuse layer: circular complex-Gaussian scatterers, intensity ~ exp(-delta/atten)."""
    fov = lam0 * z / pitch
    pts = []
    for l in range(n_layers):
        d = (l + 0.5) * depth_max / n_layers
        sigma = scale * np.sqrt(np.exp(-d / atten))
        for _ in range(per_layer):
            X = rng.uniform(-fov / 8.0, fov / 8.0)
            Y = rng.uniform(-fov / 8.0, fov / 8.0)
            a = sigma * (rng.normal() + 1j * rng.normal()) / np.sqrt(2.0)
            pts.append(Scatterer(X, Y, d, a))
    return pts


# name -> (nx, ny, nlambda, kind, seed)
WORKLOADS = {
    "tiny_64x64x32": (64, 64, 32, "points", 1),
    "mid_512x512x128": (512, 512, 128, "speckle", 2),
    "paper_1024x1024x256": (1024, 1024, 256, "points", 3),
}


def workload(name: str, *, seed: Optional[int] = None, frames: bool = True,
             nx: Optional[int] = None, ny: Optional[int] = None,
             nlambda: Optional[int] = None, kind: Optional[str] = None) -> Workload:
    """Build a named workload (or a custom size with ``nx``/``ny``/``nlambda``).

    Named workloads: ``tiny_64x64x32`` (5 points, read noise, 12 bit),
    ``mid_512x512x128`` (50 points + diffuse speckle layer, Poisson around
    2000 DN) and ``paper_1024x1024x256`` (as tiny).  ``frames=False`` skips the
    stack (geometry only).
    """
    if name in WORKLOADS:
        nx0, ny0, nl0, kind0, seed0 = WORKLOADS[name]
    else:
        nx0, ny0, nl0, kind0, seed0 = nx, ny, nlambda, kind or "points", 0
    nx = nx or nx0
    ny = ny or ny0
    nlambda = nlambda or nl0
    kind = kind or kind0
    seed = seed0 if seed is None else seed
    rng = np.random.default_rng(seed)
    pitch, z = OPTICS["pitch"], OPTICS["z"]
    lambdas = sweep_wavelengths(OPTICS["lambda_start"], OPTICS["lambda_end"], nlambda)
    if kind == "points":
        pts = _random_points(rng, 5, nx, pitch, z, lambdas[0], 0.5e-3)
    elif kind == "speckle":
        pts = _random_points(rng, 50, nx, pitch, z, lambdas[0], 0.5e-3)
        pts += _speckle_layer(rng, nx, pitch, z, lambdas[0])
    else:
        raise ValueError(f"unknown workload kind {kind!r}")
    carrier = (nx / 4.0, ny / 4.0)
    stack = None
    if frames:
        if kind == "points":
            stack, _, _ = point_scatterer_stack(nx, ny, nlambda, pts, rng=rng,
                                                lambdas=lambdas, carrier=carrier)
        else:
            stack, _, _ = speckle_stack(nx, ny, nlambda, pts, rng=rng,
                                        lambdas=lambdas, carrier=carrier)
    return Workload(name, nx, ny, nlambda, pitch, z, lambdas, stack, pts, carrier,
                    (0, 0, nx, ny))
