"""The seeded synthetic workloads: shapes, types, determinism, value ranges."""

import numpy as np

import synth


def test_tiny_workload_shape_and_determinism():
    a = synth.workload("tiny_64x64x32")
    b = synth.workload("tiny_64x64x32")
    assert a.frames.shape == (32, 64, 64) and a.frames.dtype == np.uint16
    assert np.array_equal(a.frames, b.frames)
    assert a.frames.max() <= 4095 and len(a.scatterers) == 5
    assert a.window == (0, 0, 64, 64) and a.voxels == 64 * 64 * 32
    c = synth.workload("tiny_64x64x32", seed=99)
    assert not np.array_equal(a.frames, c.frames)


def test_sweep_is_linear_in_wavenumber():
    lam = synth.sweep_wavelengths(800e-9, 850e-9, 17)
    k = 2 * np.pi / lam
    assert abs(lam[0] - 800e-9) < 1e-20 and abs(lam[-1] - 850e-9) < 1e-20
    assert np.allclose(np.diff(k), np.diff(k)[0], rtol=1e-10)


def test_custom_speckle_workload():
    w = synth.workload("custom", nx=64, ny=48, nlambda=8, kind="speckle", seed=4)
    assert w.frames.shape == (8, 48, 64)
    m = w.frames.mean()
    assert 1500 < m < 2600       # Poisson counts around a 2000 DN mean
