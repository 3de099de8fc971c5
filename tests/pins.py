"""Checks that pin the FP64 oracle to things other than itself.

Each ``pin_*`` function takes an oracle module ``o`` (the real one, or a copy
with a planted mistake) and raises AssertionError when the oracle disagrees with
what the paper or the mathematics fix.  The expected values never come from the
oracle: they are the literal convolution form of Eq. 6 summed term by term,
pure-Python DFT loops, Parseval's identity, the Dirichlet kernel, hand-derived
interpolation values, and the closed-form focus position and depth bin of a
synthetic point scatterer.
"""

from __future__ import annotations

import cmath
import math

import numpy as np

from synth.interferograms import Scatterer, point_scatterer_stack, sweep_wavelengths

PITCH = 20e-6
Z = 0.3


# ---------------------------------------------------------------- Eq. 5 pins

def pin_rescale_identity(o):
    """s = 1 (frame 0 of every sweep) leaves the frame unchanged, exactly."""
    rng = np.random.default_rng(5)
    f = rng.integers(0, 4096, size=(12, 20)).astype(np.uint16)
    out = o.rescale(f, 1.0)
    assert out.shape == f.shape
    assert np.array_equal(out, f.astype(np.float64))


def pin_rescale_affine(o):
    """Linear interpolation reproduces an affine image exactly wherever both taps
    of both axes fall inside the frame (non-square frame, so a swapped axis shows)."""
    ny, nx = 24, 40
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    f = 3.0 * ii + 7.0 * jj + 11.0
    for s in (1.0137, 1.0625, 0.97):
        out = o.rescale(f, s)
        u = nx / 2.0 + (np.arange(nx) - nx / 2.0) * s
        v = ny / 2.0 + (np.arange(ny) - ny / 2.0) * s
        okx = (u >= 0) & (u <= nx - 1)
        oky = (v >= 0) & (v <= ny - 1)
        expect = 3.0 * u[None, :] + 7.0 * v[:, None] + 11.0
        m = oky[:, None] & okx[None, :]
        assert m.sum() > 0.5 * m.size
        assert np.max(np.abs(out[m] - expect[m])) < 1e-9


def pin_rescale_hand_values(o):
    """8 x 8 frame, s = 2, centre 4: output x reads input x' = 2x - 4 (an exact
    sample) for x = 2..5 and lies outside the frame (value 0) for x = 0, 1, 6, 7.
    s = 1.5: x = 5 reads 5.5 -> the mean of samples 5 and 6; x = 1 reads -0.5 ->
    half of sample 0 (the tap at -1 reads 0)."""
    f = np.arange(64, dtype=np.float64).reshape(8, 8) * 10.0 + 1.0
    out = o.rescale(f, 2.0)
    src = {2: 0, 3: 2, 4: 4, 5: 6}
    for y in range(8):
        for x in range(8):
            if x in src and y in src:
                exp = f[src[y], src[x]]
            else:
                exp = 0.0
            assert abs(out[y, x] - exp) < 1e-12, (y, x, out[y, x], exp)
    out = o.rescale(f, 1.5)
    # y = 4 reads row 4 exactly (centre)
    assert abs(out[4, 5] - 0.5 * (f[4, 5] + f[4, 6])) < 1e-12
    assert abs(out[4, 1] - 0.5 * f[4, 0]) < 1e-12


def pin_rescale_zero_outside(o):
    """A constant frame stays constant where the rescaled grid is inside the frame
    and falls to 0 (not to the edge value) where it leaves it."""
    n = 32
    f = np.full((n, n), 100.0)
    out = o.rescale(f, 1.25)
    u = n / 2.0 + (np.arange(n) - n / 2.0) * 1.25
    inside = (u >= 0) & (u <= n - 1)
    far = (u < -1) | (u >= n)
    assert np.allclose(out[np.ix_(inside, inside)], 100.0, atol=1e-12)
    assert np.all(out[np.ix_(far, np.arange(n))] == 0.0)


# ---------------------------------------------------------------- Eq. 6 pins

def eq6_convolution_bruteforce(ip, pitch, z, lam1):
    """Eq. 6 as printed: H(x, y) = (i / (lambda_1 z)) exp(-i k_1 z)
    sum_{x', y'} I'(x', y') exp[-i pi ((x - x')^2 + (y - y')^2) / (lambda_1 z)] d^2,
    with x' = (n - N/2) d on the sensor and x = (m - N/2) d' on the hologram plane,
    d' = lambda_1 z / (N d) (Eq. 4).  Plain loops over output pixels."""
    ny, nx = ip.shape
    lz = lam1 * z
    xs = (np.arange(nx) - nx / 2.0) * pitch
    ys = (np.arange(ny) - ny / 2.0) * pitch
    xh = (np.arange(nx) - nx / 2.0) * (lz / (nx * pitch))
    yh = (np.arange(ny) - ny / 2.0) * (lz / (ny * pitch))
    pre = 1j / lz * cmath.exp(-1j * 2.0 * math.pi * z / lam1) * pitch * pitch
    out = np.empty((ny, nx), dtype=np.complex128)
    for p in range(ny):
        for m in range(nx):
            ker = np.exp(-1j * math.pi * ((xh[m] - xs[None, :]) ** 2 + (yh[p] - ys[:, None]) ** 2) / lz)
            out[p, m] = pre * np.sum(ip * ker)
    return out


def pin_fresnel_convolution(o, shapes=((8, 8), (12, 16), (10, 6)), methods=("dense", "fft")):
    """The oracle's chirp-DFT-chirp evaluation equals the literal convolution of Eq. 6."""
    rng = np.random.default_rng(7)
    for (ny, nx) in shapes:
        ip = rng.uniform(0, 4000, size=(ny, nx))
        lam1 = 812e-9
        ref = eq6_convolution_bruteforce(ip, PITCH, Z, lam1)
        for meth in methods:
            got = o.fresnel(ip, PITCH, Z, lam1, method=meth)
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err < 1e-10, (ny, nx, meth, err)


def pin_fresnel_matched_chirp(o):
    """A field that cancels the input chirp and carries a linear phase that steers
    to hologram pixel (m0, p0) transforms to a single nonzero pixel there (a
    Kronecker delta of height |K| N_x N_y), as Eq. 6 expanded says."""
    nx, ny = 32, 24
    lam1 = 800e-9
    lz = lam1 * Z
    xs = (np.arange(nx) - nx / 2.0) * PITCH
    ys = (np.arange(ny) - ny / 2.0) * PITCH
    m0, p0 = 21, 5
    a = (np.exp(1j * math.pi * (xs[None, :] ** 2 + ys[:, None] ** 2) / lz)
         * np.exp(-2j * math.pi * (m0 - nx / 2.0) * (np.arange(nx)[None, :] - nx / 2.0) / nx)
         * np.exp(-2j * math.pi * (p0 - ny / 2.0) * (np.arange(ny)[:, None] - ny / 2.0) / ny))
    for meth in ("dense", "fft"):
        h = o.fresnel(a, PITCH, Z, lam1, method=meth)
        mag = np.abs(h)
        kmag = PITCH * PITCH / lz
        assert abs(mag[p0, m0] - kmag * nx * ny) < 1e-9 * kmag * nx * ny
        mag[p0, m0] = 0.0
        assert mag.max() < 1e-9 * kmag * nx * ny


def pin_fresnel_parseval(o):
    """sum |H|^2 = |K|^2 N_x N_y sum |I'|^2 (both chirps have unit modulus)."""
    rng = np.random.default_rng(11)
    ip = rng.uniform(0, 4000, size=(48, 64))
    lam1 = 830e-9
    h = o.fresnel(ip, PITCH, Z, lam1, method="fft")
    kmag2 = (PITCH * PITCH / (lam1 * Z)) ** 2
    lhs = np.sum(np.abs(h) ** 2)
    rhs = kmag2 * 48 * 64 * np.sum(ip ** 2)
    assert abs(lhs - rhs) < 1e-10 * rhs


# ---------------------------------------------------------------- Eq. 7 pins

def pin_axial_loops(o):
    """Eq. 7 with a rectangular gate equals the DFT written as plain loops."""
    rng = np.random.default_rng(13)
    n = 12
    h = rng.normal(size=(n, 3, 2)) + 1j * rng.normal(size=(n, 3, 2))
    ref = np.zeros_like(h)
    for q in range(n):
        for t in range(n):
            ref[q] += h[t] * cmath.exp(-2j * math.pi * q * t / n)
    for meth in ("dense", "fft"):
        got = o.axial(h, method=meth)
        assert np.max(np.abs(got - ref)) < 1e-11


def pin_axial_dirichlet(o):
    """A single exponential exp(i theta t) gives the Dirichlet kernel at every bin:
    V_q = exp(i (N-1) phi / 2) sin(N phi / 2) / sin(phi / 2), phi = theta - 2 pi q / N."""
    n = 32
    theta = 2 * math.pi * 5.3 / n
    h = np.exp(1j * theta * np.arange(n))[:, None]
    for meth in ("dense", "fft"):
        v = o.axial(h, method=meth)[:, 0]
        for q in range(n):
            phi = theta - 2 * math.pi * q / n
            ref = cmath.exp(1j * (n - 1) * phi / 2) * math.sin(n * phi / 2) / math.sin(phi / 2)
            assert abs(v[q] - ref) < 1e-10, (q, v[q], ref)


def pin_axial_parseval(o):
    """sum_q |V_q|^2 = N sum_t |H_t|^2."""
    rng = np.random.default_rng(17)
    h = rng.normal(size=(64, 5)) + 1j * rng.normal(size=(64, 5))
    v = o.axial(h, method="fft")
    assert np.allclose(np.sum(np.abs(v) ** 2, axis=0), 64 * np.sum(np.abs(h) ** 2, axis=0), rtol=1e-12)


def pin_intensity(o):
    """The envelope of the cut formulas after Eq. 7 is |V|^2 = Re^2 + Im^2:
    hand values, then Parseval through the axial transform (sum_q |V_q|^2 =
    N sum_t |H_t|^2, the right side summed here from squared real and imaginary
    parts), and the three cuts are plain slices of it."""
    v = np.array([3 + 4j, -1j, 0.5 - 0.5j, -2 + 0j, 0j])
    assert np.array_equal(o.intensity(v), np.array([25.0, 1.0, 0.5, 4.0, 0.0]))
    rng = np.random.default_rng(23)
    h = rng.normal(size=(16, 4, 5)) + 1j * rng.normal(size=(16, 4, 5))
    p = o.intensity(o.axial(h, method="fft"))
    assert p.shape == h.shape and np.isrealobj(p) and (p >= 0).all()
    assert np.isclose(p.sum(), 16 * (h.real ** 2 + h.imag ** 2).sum(), rtol=1e-12)
    xy, xz, yz = o.cuts(p, 3, 1, 7)
    assert np.array_equal(xy, p[7]) and np.array_equal(xz, p[:, 1, :]) and np.array_equal(yz, p[:, :, 3])


# ---------------------------------------------------------------- end to end

def point_case(n=64, nl=32, X_px=3.3, Y_px=-5.2, delta=0.1e-3, ny=None):
    ny = ny or n
    lam = sweep_wavelengths(800e-9, 850e-9, nl)
    dpx = lam[0] * Z / (n * PITCH)
    dpy = lam[0] * Z / (ny * PITCH)
    sc = Scatterer(X_px * dpx, Y_px * dpy, delta, 0.5)
    frames, _, _ = point_scatterer_stack(n, ny, nl, [sc], rng=np.random.default_rng(0), read_noise=0.0)
    return frames, lam, sc, dpx, dpy


def expected_focus(n, ny, nl, lam, sc, dpx, dpy):
    """Closed forms: after Eq. 5 the scatterer's linear phase is independent of the
    frame, so it focuses at (N/2 + X/d'_x + N/4, N/2 + Y/d'_y + N/4) (carrier at N/4
    cycles); its frame-to-frame phase step is Delta k (2 delta + rho^2 / (2 z)),
    so the depth bin is N_lambda Delta k (2 delta + rho^2/(2z)) / (2 pi) mod N_lambda."""
    ex = n / 2.0 + sc.X / dpx + n / 4.0
    ey = ny / 2.0 + sc.Y / dpy + ny / 4.0
    dk = 2 * math.pi / lam[1] - 2 * math.pi / lam[0]
    eq = (nl * dk * (2 * sc.delta + (sc.X ** 2 + sc.Y ** 2) / (2 * Z)) / (2 * math.pi)) % nl
    return ex, ey, eq


def _circ(a, b, n):
    d = abs(a - b) % n
    return min(d, n - d)


def pin_point_scatterer(o, cases=((64, 64, 32, 3.3, -5.2, 0.1e-3), (48, 64, 40, -6.6, 7.1, 0.37e-3)),
                        method="dense"):
    for (n, ny, nl, X, Y, d) in cases:
        frames, lam, sc, dpx, dpy = point_case(n, nl, X, Y, d, ny=ny)
        v = o.reconstruct(frames, PITCH, Z, lam, method=method)
        p = np.abs(v) ** 2
        # search the carrier quadrant only (DC and the twin image live elsewhere)
        qm = np.zeros_like(p, dtype=bool)
        qm[:, ny // 2 + 2:, n // 2 + 2:] = True
        q, y, x = np.unravel_index(np.argmax(np.where(qm, p, 0.0)), p.shape)
        ex, ey, eq = expected_focus(n, ny, nl, lam, sc, dpx, dpy)
        assert abs(x - ex) <= 1.0 and abs(y - ey) <= 1.0, ((x, y), (ex, ey))
        assert _circ(q, eq, nl) <= 1.0, (q, eq)


def pin_chromatic_compensation(o):
    """Eq. 5's purpose: after rescaling, every frame's hologram focuses the same
    off-centre scatterer on the same pixel (with lambda_t d' it would drift)."""
    n, nl = 64, 16
    frames, lam, sc, dpx, dpy = point_case(n, nl, X_px=10.4, Y_px=9.6, delta=0.0)
    h = o.reconstruct(frames, PITCH, Z, lam, frame_range=(0, nl))
    ex, ey, _ = expected_focus(n, n, nl, lam, sc, dpx, dpy)
    for t in range(nl):
        p = np.abs(h[t]) ** 2
        # carrier quadrant, away from the spread-out zero order around N/2
        p[: n // 2 + 8, :] = 0.0
        p[:, : n // 2 + 8] = 0.0
        y, x = np.unravel_index(np.argmax(p), p.shape)
        assert abs(x - ex) <= 1.0 and abs(y - ey) <= 1.0, (t, (x, y), (ex, ey))


def pin_pixel_sample(o):
    """The per-pixel double-sum path agrees with the whole-volume path."""
    frames, lam, sc, dpx, dpy = point_case(32, 16, 2.2, 3.1, 0.2e-3)
    v = o.reconstruct(frames, PITCH, Z, lam, method="fft")
    pix = [(0, 0), (31, 31), (16, 16), (25, 27), (3, 29)]
    vs = o.pixel_sample(frames, PITCH, Z, lam, pix)
    for i, (x, y) in enumerate(pix):
        ref = v[:, y, x]
        assert np.linalg.norm(vs[i] - ref) <= 1e-10 * np.linalg.norm(v) / 4


ALL_PINS = [
    pin_rescale_identity, pin_rescale_affine, pin_rescale_hand_values, pin_rescale_zero_outside,
    pin_fresnel_convolution, pin_fresnel_matched_chirp, pin_fresnel_parseval,
    pin_axial_loops, pin_axial_dirichlet, pin_axial_parseval, pin_intensity,
    pin_point_scatterer, pin_chromatic_compensation, pin_pixel_sample,
]
