"""Aberration path on the GPU (SSOCT_FLAG_PUPIL) against the FP64 oracle.

The volume with a Zernike phase screen must match the oracle's pupil
reconstruction (relative L2 <= 2e-5 on |V|^2), the sharpness loss to 1e-5
relative, and the gradient (dL/dz, dL/dc_1..15) to a relative L2 error
<= 1e-4 of the oracle's adjoint gradient, which its own pins tie to finite
differences of the loss.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from oracle import aberration as ab  # noqa: E402
import oracle  # noqa: E402


@pytest.fixture(scope="module")
def ss():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_08960_gb300 import build
    build.build()
    import paper_2003_08960_gb300 as ss
    return ss


def _dev(frames):
    return torch.from_numpy(np.ascontiguousarray(frames).view(np.int16)).cuda()


def _compare(ss, w, coeffs, z, window=None, tol_grad=1e-4):
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, 0.3, w.lambdas, window=window, flags=ss.SSOCT_FLAG_PUPIL)
    loss, grad, vol = plan.sharpness(_dev(w.frames), coeffs, z)
    ref_v = oracle.intensity(ab.reconstruct_pupil(w.frames, w.pitch, z, w.lambdas, coeffs, window))
    err_v = np.linalg.norm(vol.cpu().numpy() - ref_v) / np.linalg.norm(ref_v)
    ref_loss, ref_grad = ab.sharpness_gradient(w.frames, w.pitch, z, w.lambdas, coeffs, window)
    err_l = abs(loss - ref_loss) / abs(ref_loss)
    err_g = np.linalg.norm(grad - ref_grad) / np.linalg.norm(ref_grad)
    print(f"{w.nx}x{w.ny}x{w.nlambda} window={window}: |V|^2 {err_v:.2e}, loss {err_l:.2e}, gradient {err_g:.2e}, "
          f"piston/|g| {abs(grad[1]) / np.linalg.norm(grad):.1e}")
    assert err_v <= 2e-5, err_v
    assert err_l <= 1e-5, (loss, ref_loss)
    assert err_g <= tol_grad, (grad, ref_grad)
    return plan, grad


@pytest.mark.parametrize("shape,window", [((64, 64, 32), None), ((128, 64, 64), (10, 6, 100, 50)),
                                          ((256, 256, 16), (0, 64, 256, 128))])
def test_pupil_volume_loss_and_gradient(ss, shape, window):
    nx, ny, nl = shape
    w = synth.workload("custom", nx=nx, ny=ny, nlambda=nl, kind="points", seed=nx + ny)
    coeffs = np.random.default_rng(nl).normal(0.0, 0.5, 15)
    _compare(ss, w, coeffs, 0.305, window)


def test_zero_pupil_equals_plain_reconstruction(ss):
    w = synth.workload("tiny_64x64x32")
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, 0.3, w.lambdas, flags=ss.SSOCT_FLAG_PUPIL)
    f = _dev(w.frames)
    loss, grad, vol = plan.sharpness(f, [], 0.3)
    plain = plan.reconstruct(f)
    torch.cuda.synchronize()
    assert torch.allclose(vol, plain, rtol=2e-5, atol=1e-6 * float(plain.max()))


def test_config5_speckle_512x512x128(ss):
    """The 512x512x128 speckle workload with 15 coefficients ~ N(0, 0.5 rad),
    reconstructed 5 mm beyond the generating distance."""
    w = synth.workload("mid_512x512x128")
    coeffs = np.random.default_rng(5).normal(0.0, 0.5, 15)
    _compare(ss, w, coeffs, 0.305)


def test_autograd_backward_and_descent(ss):
    from paper_2003_08960_gb300.autograd import sharpness
    w = synth.workload("custom", nx=64, ny=64, nlambda=32, kind="points", seed=11)
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, 0.3, w.lambdas, flags=ss.SSOCT_FLAG_PUPIL)
    f = _dev(w.frames)
    c = torch.tensor(np.random.default_rng(2).normal(0.0, 0.3, 15), dtype=torch.float64, requires_grad=True)
    z = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    loss = sharpness(plan, f, c, z)
    loss.backward()
    _, g, _ = plan.sharpness(f, c.detach().numpy(), 0.3)
    # the FP64 block sums are atomics, so two calls agree to rounding, not bit for bit
    assert np.allclose(c.grad.numpy(), g[1:], rtol=0, atol=1e-9 * np.linalg.norm(g))
    assert abs(z.grad.item() - g[0]) <= 1e-9 * abs(g[0])
    # gradient descent on the coefficients sharpens the volume (the frames carry no aberration)
    opt = torch.optim.SGD([c], lr=0.05 / float(np.linalg.norm(g[1:])))
    first = float(loss)
    for _ in range(8):
        opt.zero_grad()
        loss = sharpness(plan, f, c, z.detach())
        loss.backward()
        opt.step()
    assert float(sharpness(plan, f, c.detach(), z.detach())) < first


def test_config5_gradient_against_finite_differences_of_the_gpu_loss(ss):
    """Central differences of the GPU's own loss (not the oracle's) at the
    512x512x128 speckle workload, 15 coefficients ~ N(0, 0.5 rad), z + 5 mm,
    with the steps h = 1e-3 rad for c_j and 1e-3 mm for z.

    Noise floor of the difference quotient: the loss is reduced in FP64 from the
    FP32 volume with atomics, so two evaluations at the same point differ by
    rounding only; that spread (measured here) divided by h bounds the quotient's
    noise, and the truncation error of a central difference is O(h^2).  Each
    sampled component must agree with the adjoint gradient to 1e-3 of the
    gradient's norm, far above both."""
    w = synth.workload("mid_512x512x128")
    coeffs = np.random.default_rng(5).normal(0.0, 0.5, 15)
    z = 0.305
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, 0.3, w.lambdas, flags=ss.SSOCT_FLAG_PUPIL)
    f = _dev(w.frames)
    vol = plan.empty_volume()[0]

    def loss(c, zz):
        l, _, _ = plan.sharpness(f, c, zz, out=vol)
        return l

    l0, g, _ = plan.sharpness(f, coeffs, z, out=vol)
    noise = max(abs(loss(coeffs, z) - l0) for _ in range(3))
    gnorm = float(np.linalg.norm(g))
    h_c, h_z = 1e-3, 1e-6
    checks = [("z", 0, None)] + [(f"c_{j}", j, j - 1) for j in (1, 2, 4, 7, 11, 15)]
    worst = 0.0
    for name, gi, ci in checks:
        if ci is None:
            fd = (loss(coeffs, z + h_z) - loss(coeffs, z - h_z)) / (2 * h_z)
            scale = gnorm
        else:
            cp, cm = coeffs.copy(), coeffs.copy()
            cp[ci] += h_c
            cm[ci] -= h_c
            fd = (loss(cp, z) - loss(cm, z)) / (2 * h_c)
            scale = float(np.linalg.norm(g[1:]))
        err = abs(fd - g[gi]) / scale
        worst = max(worst, err)
        print(f"{name}: adjoint {g[gi]:+.6e}  central difference {fd:+.6e}  |diff|/|g| {err:.1e}")
        assert err <= 1e-3, (name, fd, g[gi])
    print(f"loss {l0:.6e}; repeat-evaluation spread {noise:.1e} (quotient noise <= {noise / h_c:.1e} per rad, "
          f"{noise / h_z:.1e} per m); worst |diff|/|g| {worst:.1e}")
