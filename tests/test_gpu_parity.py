"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerance: the FP32 path must match the oracle's complex volume V to a relative
L2 error <= 1e-5 per volume (also checked on |V|^2 and, separately, on the +1
order quadrant, where the signal is far below the zero order).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
import pins  # noqa: E402

TOL = 1e-5


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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run(ss, w, window=None, method="dense", flags=0):
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas, window=window, flags=flags)
    vol, cplx = plan.reconstruct(_dev(w.frames), complex_out=True)
    plan.sync()
    ref = oracle.reconstruct(w.frames, w.pitch, w.z, w.lambdas, window=window, method=method)
    return plan, vol.cpu().numpy(), cplx.cpu().numpy(), ref


def _check(vol, cplx, ref, tol=TOL, quadrant=True):
    err_v = _rel(cplx.astype(np.complex128), ref)
    pref = oracle.intensity(ref)
    err_p = _rel(vol.astype(np.float64), pref)
    assert err_v <= tol, f"complex volume rel L2 {err_v:.3e}"
    assert err_p <= 2 * tol, f"|V|^2 rel L2 {err_p:.3e}"
    if quadrant:
        nl, wy, wx = ref.shape
        q = (slice(None), slice(wy // 2 + 2, None), slice(wx // 2 + 2, None))
        err_q = _rel(cplx[q].astype(np.complex128), ref[q])
        assert err_q <= 10 * tol, f"+1-order quadrant rel L2 {err_q:.3e}"
    return err_v


def test_tiny_full_window(ss):
    w = synth.workload("tiny_64x64x32")
    plan, vol, cplx, ref = _run(ss, w)
    _check(vol, cplx, ref)


def test_tiny_ragged_window(ss):
    """Off-axis window whose width is not a multiple of the 32-pixel tile."""
    w = synth.workload("tiny_64x64x32")
    win = (36, 40, 23, 17)
    plan, vol, cplx, ref = _run(ss, w, window=win)
    assert vol.shape == (32, 17, 23)
    _check(vol, cplx, ref, quadrant=False)


@pytest.mark.parametrize("shape", [(128, 64, 16), (64, 128, 64), (128, 128, 128)])
def test_non_square_and_sizes(ss, shape):
    nx, ny, nl = shape
    w = synth.workload("custom", nx=nx, ny=ny, nlambda=nl, kind="points", seed=nx + ny + nl)
    plan, vol, cplx, ref = _run(ss, w)
    _check(vol, cplx, ref)


def test_point_scatterer_focus_on_gpu(ss):
    """The closed-form focus position and depth bin, read off the GPU volume."""
    for case in [(64, 64, 32, 3.3, -5.2, 0.1e-3), (128, 64, 16, -9.6, 7.1, 0.37e-3)]:
        n, ny, nl, X, Y, d = case
        frames, lam, sc, dpx, dpy = pins.point_case(n, nl, X, Y, d, ny=ny)
        plan = ss.Plan(n, ny, nl, pins.PITCH, pins.Z, lam)
        vol = plan.reconstruct(_dev(frames)).cpu().numpy()
        mask = np.zeros_like(vol, dtype=bool)
        mask[:, ny // 2 + 2:, n // 2 + 2:] = True
        q, y, x = np.unravel_index(np.argmax(np.where(mask, vol, 0)), vol.shape)
        ex, ey, eq = pins.expected_focus(n, ny, nl, lam, sc, dpx, dpy)
        assert abs(x - ex) <= 1 and abs(y - ey) <= 1, ((x, y), (ex, ey))
        dq = abs(q - eq) % nl
        assert min(dq, nl - dq) <= 1, (q, eq)


@pytest.mark.parametrize("shape,window", [((64, 64, 256), (5, 3, 37, 11)),      # 22 tiles: fewer than SMs
                                          ((256, 256, 256), None),               # the 3-buffer ring wraps
                                          ((128, 128, 128), (7, 9, 100, 70)),    # 6 buffers, ragged tiles
                                          ((128, 128, 64), None)])               # 8 buffers
def test_streaming_axial_form(ss, shape, window):
    """Sweeps of 64 to 256 frames take the persistent axial kernel (TMA-fed ring
    of stage buffers, two consumer groups): few tiles per SM, many ring wraps
    and ragged last tiles must all match the oracle, and no wait may run out."""
    nx, ny, nl = shape
    w = synth.workload("custom", nx=nx, ny=ny, nlambda=nl, kind="points", seed=5 * nx + ny + nl)
    plan, vol, cplx, ref = _run(ss, w, window=window, method="fft")
    _check(vol, cplx, ref, quadrant=window is None)
    plan.sync()
    # the |V| envelope from the same kernel
    mag = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas, window=window, flags=ss.SSOCT_FLAG_MAGNITUDE)
    m = mag.reconstruct(_dev(w.frames)).cpu().numpy().astype(np.float64)
    mag.sync()
    assert _rel(m * m, vol.astype(np.float64)) <= 1e-6


def test_mid_speckle_512(ss):
    w = synth.workload("mid_512x512x128")
    plan, vol, cplx, ref = _run(ss, w, method="fft")
    _check(vol, cplx, ref)


def test_magnitude_flag_and_determinism(ss):
    w = synth.workload("tiny_64x64x32")
    p1 = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas)
    p2 = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas, flags=ss.SSOCT_FLAG_MAGNITUDE)
    f = _dev(w.frames)
    a = p1.reconstruct(f)
    b = p1.reconstruct(f)
    m = p2.reconstruct(f)
    torch.cuda.synchronize()
    assert torch.equal(a, b), "two runs of the same plan differ"
    assert torch.allclose(m * m, a, rtol=1e-5, atol=0)


def test_ring_path_equals_device_path(ss):
    w = synth.workload("tiny_64x64x32")
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas)
    ref = plan.reconstruct(_dev(w.frames))
    with pytest.raises(ss.SsoctError) as e:
        plan.reconstruct_ring()
    assert e.value.status == ss.SSOCT_ENOTREADY
    # push from the host in two pieces, with sequence numbers
    assert plan.push(w.frames[:10], first_seq=100) == ss.SSOCT_OK
    assert plan.push(w.frames[10:], first_seq=110) == ss.SSOCT_OK
    v1 = plan.reconstruct_ring()
    torch.cuda.synchronize()
    assert torch.equal(v1, ref)
    # a wrapped ring: push 5 stray frames then a whole sweep from the device
    plan.push(_dev(w.frames[:5]), first_seq=142)
    plan.push(_dev(w.frames), first_seq=147)
    v2 = plan.reconstruct_ring()
    torch.cuda.synchronize()
    assert torch.equal(v2, ref)
    # a drop restarts the gate
    assert plan.push(w.frames[:4], first_seq=500) == ss.SSOCT_EDROPPED
    with pytest.raises(ss.SsoctError):
        plan.reconstruct_ring()


def test_cuts_are_slices(ss):
    w = synth.workload("tiny_64x64x32")
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas, window=(8, 4, 50, 40))
    vol = plan.reconstruct(_dev(w.frames))
    xy, xz, yz = plan.cuts(vol, 17, 33, 5)
    torch.cuda.synchronize()
    assert torch.equal(xy, vol[5]) and torch.equal(xz, vol[:, 33, :]) and torch.equal(yz, vol[:, :, 17])
    with pytest.raises(ss.SsoctError):
        plan.cuts(vol, 50, 0, 0)


def test_profile_records_both_kernels(ss):
    w = synth.workload("tiny_64x64x32")
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas)
    assert ss.ssoct_profile(plan.handle, True) == 0
    f = _dev(w.frames)
    for _ in range(3):
        plan.reconstruct(f)
    st, lat, ax, calls = ss.ssoct_profile_read(plan.handle)
    assert st == 0 and calls == 3 and lat > 0 and ax > 0


@pytest.mark.slow
def test_paper_size_1024x1024x256(ss):
    """Full-size volume in the bench's launch configuration, whole-volume parity."""
    w = synth.workload("paper_1024x1024x256")
    plan, vol, cplx, ref = _run(ss, w, method="fft")
    err = _check(vol, cplx, ref)
    print(f"1024x1024x256 complex rel L2 = {err:.3e}")


def test_wait_timeout_is_reported_and_device_recovers(ss):
    """Failure path of the bounded device waits: skipping the first work item
    leaves the column items of frame 0 waiting for a row item that never runs;
    they give up after 50 ms, the kernels return, ssoct_sync reports
    SSOCT_ETIMEOUT, and the next normal call reproduces the volume exactly."""
    w = synth.workload("tiny_64x64x32")
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas)
    f = _dev(w.frames)
    ref = plan.reconstruct(f)
    plan.sync()
    stream = torch.cuda.current_stream().cuda_stream
    assert ss.ssoct_inject_stall(plan.handle, 1, 50_000_000) == ss.SSOCT_OK
    plan.reconstruct(f)
    assert ss.ssoct_sync(plan.handle, stream) == ss.SSOCT_ETIMEOUT
    assert "gave up" in ss.ssoct_last_error(plan.handle)
    assert ss.ssoct_inject_stall(plan.handle, 0, 0) == ss.SSOCT_OK
    again = plan.reconstruct(f)
    plan.sync()
    assert torch.equal(again, ref)


def test_sliding_gate_matches_oracle(ss):
    """Sliding gates over a periodic sweep: after each push the gate is the last
    nlambda frames.  Its |V|^2 equals the oracle's for those frames put in
    slot (= wavelength) order, and the complex output is V in slot order."""
    a = synth.workload("tiny_64x64x32", seed=1)
    b = synth.workload("tiny_64x64x32", seed=7)      # the scene changes between sweeps
    c = synth.workload("tiny_64x64x32", seed=11)
    stream = np.concatenate([a.frames, b.frames, c.frames])   # frame i at lambda[i % 32]
    plan = ss.Plan(a.nx, a.ny, a.nlambda, a.pitch, a.z, a.lambdas)
    nl = a.nlambda
    pushed = 0
    for step in (32, 13, 5, 0, 27, 19):
        if step:
            assert plan.push(_dev(stream[pushed:pushed + step])) == ss.SSOCT_OK
            pushed += step
        vol, cplx = plan.reconstruct_sliding(complex_out=True)
        plan.sync()
        gate = stream[pushed - nl:pushed]
        first = pushed - nl
        slot_order = np.roll(gate, first % nl, axis=0)         # slot r holds the frame with i % nl == r
        ref = oracle.reconstruct(slot_order, a.pitch, a.z, a.lambdas)
        _check(vol.cpu().numpy(), cplx.cpu().numpy(), ref)
    # a full reconstruct in between invalidates the kept holograms; the next
    # sliding call redoes the whole gate and is still exact
    plan.reconstruct(_dev(a.frames))
    vol = plan.reconstruct_sliding()
    plan.sync()
    gate = stream[pushed - nl:pushed]
    ref = oracle.reconstruct(np.roll(gate, (pushed - nl) % nl, axis=0), a.pitch, a.z, a.lambdas)
    assert _rel(vol.cpu().numpy().astype(np.float64), oracle.intensity(ref)) <= 2 * TOL


def test_sliding_gate_mixed_radix_384(ss):
    """Sliding gates on a mixed-radix frame (384 = 16 x 24, stage 2 with idle
    threads) with a window: the lateral pass over the new frames only, then the
    gate in slot order, against the oracle."""
    w = synth.workload("custom", nx=384, ny=384, nlambda=96, kind="points", seed=31)
    v = synth.workload("custom", nx=384, ny=384, nlambda=96, kind="points", seed=32)
    stream = np.concatenate([w.frames, v.frames])   # frame i at lambda[i % 96]
    win = (40, 24, 300, 330)
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas, window=win)
    nl = w.nlambda
    pushed = 0
    for step in (96, 13, 40):
        assert plan.push(_dev(stream[pushed:pushed + step])) == ss.SSOCT_OK
        pushed += step
        vol, cplx = plan.reconstruct_sliding(complex_out=True)
        plan.sync()
        gate = stream[pushed - nl:pushed]
        slot_order = np.roll(gate, (pushed - nl) % nl, axis=0)
        ref = oracle.reconstruct(slot_order, w.pitch, w.z, w.lambdas, window=win, method="fft")
        err = _check(vol.cpu().numpy(), cplx.cpu().numpy(), ref, quadrant=False)
        print(f"sliding 384x384x96 after {pushed} frames: complex rel L2 {err:.3e}")


# Tensor-core axial form (SSOCT_FLAG_TC_AXIAL): BF16 hi + lo operands, FP32
# accumulation.  Bound: relative L2 <= 1e-3 per volume against the FP64 oracle;
# the split-precision arithmetic puts it near 1e-5, checked at 1e-4 as well.
TC_TOL = 1e-3


def _check_tc(vol, cplx, ref):
    err_v = _rel(cplx.astype(np.complex128), ref)
    err_p = _rel(vol.astype(np.float64), oracle.intensity(ref))
    assert err_v <= TC_TOL and err_p <= 2 * TC_TOL, (err_v, err_p)
    assert err_v <= 1e-4, f"tensor-core form rel L2 {err_v:.3e}, expected near 1e-5"
    return err_v, err_p


@pytest.mark.parametrize("shape,window", [((64, 64, 256), None), ((128, 64, 256), (20, 8, 77, 50)),
                                          ((256, 256, 256), None)])
def test_tc_axial_matches_oracle(ss, shape, window):
    nx, ny, nl = shape
    w = synth.workload("custom", nx=nx, ny=ny, nlambda=nl, kind="points", seed=nx + 3 * ny)
    plan, vol, cplx, ref = _run(ss, w, window=window, method="fft", flags=ss.SSOCT_FLAG_TC_AXIAL)
    err_v, err_p = _check_tc(vol, cplx, ref)
    print(f"TC axial {shape} window={window}: complex rel L2 {err_v:.3e}, |V|^2 rel L2 {err_p:.3e}")


def test_tc_axial_speckle_and_point_focus(ss):
    """Speckle frames (fully developed, every bin populated) and the closed-form
    focus of a point scatterer, both through the tensor-core form."""
    w = synth.workload("custom", nx=128, ny=128, nlambda=256, kind="speckle", seed=5)
    plan, vol, cplx, ref = _run(ss, w, method="fft", flags=ss.SSOCT_FLAG_TC_AXIAL)
    _check_tc(vol, cplx, ref)
    frames, lam, sc, dpx, dpy = pins.point_case(64, 256, 3.3, -5.2, 0.4e-3, ny=64)
    plan = ss.Plan(64, 64, 256, pins.PITCH, pins.Z, lam, flags=ss.SSOCT_FLAG_TC_AXIAL)
    vol = plan.reconstruct(_dev(frames)).cpu().numpy()
    mask = np.zeros_like(vol, dtype=bool)
    mask[:, 34:, 34:] = True
    q, y, x = np.unravel_index(np.argmax(np.where(mask, vol, 0)), vol.shape)
    ex, ey, eq = pins.expected_focus(64, 64, 256, lam, sc, dpx, dpy)
    assert abs(x - ex) <= 1 and abs(y - ey) <= 1
    dq = abs(q - eq) % 256
    assert min(dq, 256 - dq) <= 1, (q, eq)


def test_tc_axial_magnitude_and_sliding(ss):
    w = synth.workload("custom", nx=64, ny=64, nlambda=256, kind="points", seed=9)
    f = _dev(w.frames)
    a = ss.Plan(w.nx, w.ny, 256, w.pitch, w.z, w.lambdas, flags=ss.SSOCT_FLAG_TC_AXIAL)
    m = ss.Plan(w.nx, w.ny, 256, w.pitch, w.z, w.lambdas,
                flags=ss.SSOCT_FLAG_TC_AXIAL | ss.SSOCT_FLAG_MAGNITUDE)
    va, vm = a.reconstruct(f), m.reconstruct(f)
    assert a.push(f) == ss.SSOCT_OK
    vs = a.reconstruct_sliding()
    a.sync()
    m.sync()
    assert torch.allclose(vm * vm, va, rtol=1e-5, atol=0)
    assert torch.equal(vs, va)


@pytest.mark.slow
def test_tc_axial_paper_size_1024x1024x256(ss):
    w = synth.workload("paper_1024x1024x256")
    plan, vol, cplx, ref = _run(ss, w, method="fft", flags=ss.SSOCT_FLAG_TC_AXIAL)
    err_v, err_p = _check_tc(vol, cplx, ref)
    print(f"TC axial 1024x1024x256: complex rel L2 {err_v:.3e}, |V|^2 rel L2 {err_p:.3e}")


# Mixed radix (2/3/5): frame sizes 384, 640, 768 take the two-pass lateral path,
# sweep lengths 96, 160, 200 the axial kernel with N1 = 4, 4, 5.
@pytest.mark.parametrize("shape,window", [((384, 384, 96), None), ((640, 640, 160), (100, 60, 400, 300)),
                                          ((640, 384, 32), None), ((256, 256, 200), None),
                                          ((768, 768, 200), (0, 0, 768, 200))])
def test_mixed_radix_sizes(ss, shape, window):
    nx, ny, nl = shape
    w = synth.workload("custom", nx=nx, ny=ny, nlambda=nl, kind="points", seed=nx + ny + nl)
    plan, vol, cplx, ref = _run(ss, w, window=window, method="fft")
    err = _check(vol, cplx, ref, quadrant=window is None)
    print(f"{shape} window={window}: complex rel L2 {err:.3e}")


def test_mixed_radix_ring_path(ss):
    """A frame size outside the persistent lateral kernel's list (640 x 384) takes
    the two-pass path: the ring gives the same volume, sliding gates are refused."""
    w = synth.workload("custom", nx=640, ny=384, nlambda=32, kind="points", seed=4)
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas)
    ref = plan.reconstruct(_dev(w.frames))
    plan.push(_dev(w.frames[:20]), first_seq=0)
    plan.push(_dev(w.frames), first_seq=20)     # the gate (last 32 frames) is the sweep, from ring slot 20
    v = plan.reconstruct_ring()
    torch.cuda.synchronize()
    assert torch.equal(v, ref)
    with pytest.raises(ss.SsoctError) as e:
        plan.reconstruct_sliding()
    assert e.value.status == ss.SSOCT_EUNSUPPORTED


# Axial-first order (SSOCT_FLAG_AXIAL_FIRST): Eq. 5 and Eq. 7 first, then Eq. 6
# per depth bin writing the volume; the same V as the paper's order.
@pytest.mark.parametrize("shape,window", [((64, 64, 32), None), ((64, 64, 32), (36, 40, 23, 17)),
                                          ((128, 64, 16), None), ((64, 128, 64), (10, 20, 40, 90)),
                                          ((128, 128, 128), None), ((256, 256, 256), None)])
def test_axial_first_matches_oracle(ss, shape, window):
    nx, ny, nl = shape
    w = synth.workload("custom", nx=nx, ny=ny, nlambda=nl, kind="points", seed=nx + 2 * ny + nl)
    plan, vol, cplx, ref = _run(ss, w, window=window, method="fft", flags=ss.SSOCT_FLAG_AXIAL_FIRST)
    err = _check(vol, cplx, ref, quadrant=window is None)
    print(f"axial-first {shape} window={window}: complex rel L2 {err:.3e}")


@pytest.mark.parametrize("shape,window", [((384, 384, 96), None), ((640, 640, 160), (100, 60, 400, 300)),
                                          ((768, 768, 200), None), ((384, 384, 64), None),
                                          ((768, 768, 128), None), ((640, 640, 32), (100, 60, 400, 300))])
def test_axial_first_mixed_radix(ss, shape, window):
    """Axial-first order on the persistent kernel's mixed-radix frames (stage 2
    with idle threads in the depth-bin epilogue), with the tiled first pass on
    its own splits of 96, 160, 200 frames (16 x 6, 16 x 10, 20 x 10, stage 2
    with idle threads) and on 64 and 128 frames, and the one-tile-per-CTA pass
    (32 frames), against the oracle."""
    nx, ny, nl = shape
    w = synth.workload("custom", nx=nx, ny=ny, nlambda=nl, kind="points", seed=nx + nl + 5)
    plan, vol, cplx, ref = _run(ss, w, window=window, method="fft", flags=ss.SSOCT_FLAG_AXIAL_FIRST)
    err = _check(vol, cplx, ref, quadrant=window is None)
    print(f"axial-first {shape} window={window}: complex rel L2 {err:.3e}")


@pytest.mark.parametrize("shape,window", [((64, 64, 64), None), ((128, 64, 128), (5, 9, 101, 50))])
def test_axial_first_decreasing_sweep(ss, shape, window):
    """A sweep from long to short wavelengths: every frame is rescaled by a ratio
    below 1 (Eq. 5 shrinks the field instead of widening it), so the tiled first
    pass staggers its taps the other way along each strip."""
    nx, ny, nl = shape
    w = synth.workload("custom", nx=nx, ny=ny, nlambda=nl, kind="points", seed=nx + ny + nl + 1)
    lam = np.ascontiguousarray(w.lambdas[::-1])
    plan = ss.Plan(nx, ny, nl, w.pitch, w.z, lam, window=window, flags=ss.SSOCT_FLAG_AXIAL_FIRST)
    vol, cplx = plan.reconstruct(_dev(w.frames), complex_out=True)
    plan.sync()
    ref = oracle.reconstruct(w.frames, w.pitch, w.z, lam, window=window, method="fft")
    err = _check(vol.cpu().numpy(), cplx.cpu().numpy(), ref, quadrant=False)
    print(f"axial-first, decreasing sweep {shape} window={window}: complex rel L2 {err:.3e}")


def test_axial_first_ring_magnitude_profile(ss):
    w = synth.workload("mid_512x512x128")
    af = ss.SSOCT_FLAG_AXIAL_FIRST
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas, flags=af)
    mag = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas, flags=af | ss.SSOCT_FLAG_MAGNITUDE)
    paper = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas)
    f = _dev(w.frames)
    assert ss.ssoct_profile(plan.handle, True) == 0
    v = plan.reconstruct(f)
    st, lat, ax, calls = ss.ssoct_profile_read(plan.handle)
    assert st == 0 and calls == 1 and lat > 0 and ax > 0
    ss.ssoct_profile(plan.handle, False)
    plan.push(_dev(w.frames[:30]), first_seq=0)
    plan.push(f, first_seq=30)                     # the ring wraps: gate from slot 30
    v_ring = plan.reconstruct_ring()
    m = mag.reconstruct(f)
    p = paper.reconstruct(f)
    torch.cuda.synchronize()
    assert torch.equal(v_ring, v)
    assert torch.allclose(m * m, v, rtol=1e-5, atol=0)
    assert float((v.double() - p.double()).norm() / p.double().norm()) <= 2e-6
    with pytest.raises(ss.SsoctError) as e:
        plan.reconstruct_sliding()
    assert e.value.status == ss.SSOCT_EUNSUPPORTED


@pytest.mark.slow
def test_axial_first_paper_size_1024x1024x256(ss):
    w = synth.workload("paper_1024x1024x256")
    plan, vol, cplx, ref = _run(ss, w, method="fft", flags=ss.SSOCT_FLAG_AXIAL_FIRST)
    err = _check(vol, cplx, ref)
    print(f"axial-first 1024x1024x256 complex rel L2 = {err:.3e}")


def test_sliding_cuts_only(ss):
    """Cuts-only sliding gates give the cuts of the sliding volume: xz and yz bit
    for bit (same transform), xy to FP32 rounding (one-bin sum instead of the
    FFT); a window and a ragged tile are included."""
    a = synth.workload("tiny_64x64x32", seed=1)
    b = synth.workload("tiny_64x64x32", seed=7)
    stream = np.concatenate([a.frames, b.frames])
    win = (6, 10, 50, 37)
    full = ss.Plan(a.nx, a.ny, a.nlambda, a.pitch, a.z, a.lambdas, window=win)
    cuts = ss.Plan(a.nx, a.ny, a.nlambda, a.pitch, a.z, a.lambdas, window=win)
    pushed = 0
    for step, (x0, y0, z0) in zip((32, 13, 5, 0, 14), [(3, 4, 5), (49, 36, 31), (0, 0, 0), (33, 17, 12), (20, 30, 7)]):
        if step:
            f = _dev(stream[pushed:pushed + step])
            assert full.push(f) == ss.SSOCT_OK and cuts.push(f) == ss.SSOCT_OK
            pushed += step
        vol = full.reconstruct_sliding()
        xy_ref, xz_ref, yz_ref = full.cuts(vol, x0, y0, z0)
        xy, xz, yz = cuts.sliding_cuts(x0, y0, z0)
        torch.cuda.synchronize()
        assert torch.equal(xz, xz_ref) and torch.equal(yz, yz_ref)
        assert torch.allclose(xy, xy_ref, rtol=1e-4, atol=1e-6 * float(xy_ref.max()))
    with pytest.raises(ss.SsoctError):
        cuts.sliding_cuts(50, 0, 0)


def test_sliding_cuts_running_xy(ss):
    """The running xy cut of cuts-only sliding gates (the new frames' holograms
    added, the replaced ones subtracted, while z0 stays) against the oracle's
    |V|^2 plane of each gate: the full re-sum after nlambda swapped-in frames, a
    change of z0, a call without xy and a full reconstruct in between all come
    up in the sequence."""
    ws = [synth.workload("tiny_64x64x32", seed=sd) for sd in (3, 5, 9, 13)]
    a = ws[0]
    nl = a.nlambda
    stream = np.concatenate([w.frames for w in ws])
    win = (6, 10, 50, 37)
    plan = ss.Plan(a.nx, a.ny, a.nlambda, a.pitch, a.z, a.lambdas, window=win)
    cuda_stream = torch.cuda.current_stream().cuda_stream
    # (new frames, z0, what else happens before the call)
    seq = [(32, 5, None), (3, 5, None), (7, 5, None), (1, 5, None), (0, 5, None), (13, 5, None),
           (9, 5, None),                       # 33 frames swapped in since the full sum: re-sum
           (6, 21, None), (11, 21, None), (4, 21, None),
           (5, 21, "no-xy"), (8, 21, None),    # a call without xy leaves the running sum stale
           (10, 21, "full"), (12, 21, None), (2, 21, None)]
    pushed = 0
    for step, z0, event in seq:
        if step:
            assert plan.push(_dev(stream[pushed:pushed + step])) == ss.SSOCT_OK
            pushed += step
        if event == "full":
            plan.reconstruct(_dev(a.frames))
        if event == "no-xy":
            xz = torch.empty((nl, win[2]), dtype=torch.float32, device="cuda")
            assert ss.ssoct_sliding_cuts(plan.handle, 1, 2, z0, 0, xz.data_ptr(), 0, cuda_stream) == ss.SSOCT_OK
            plan.sync()
            continue
        xy, xz, yz = plan.sliding_cuts(3, 4, z0)
        plan.sync()
        gate = stream[pushed - nl:pushed]
        ref = oracle.reconstruct(np.roll(gate, (pushed - nl) % nl, axis=0), a.pitch, a.z, a.lambdas,
                                 window=win, method="fft")
        p_ref = oracle.intensity(ref)
        err = _rel(xy.cpu().numpy().astype(np.float64), p_ref[z0])
        assert err <= 2 * TOL, f"xy after {pushed} frames (z0 {z0}): rel L2 {err:.3e}"
        assert _rel(xz.cpu().numpy().astype(np.float64), p_ref[:, 4, :]) <= 2 * TOL
    # the running sum also feeds the |V| envelope
    mag = ss.Plan(a.nx, a.ny, a.nlambda, a.pitch, a.z, a.lambdas, window=win, flags=ss.SSOCT_FLAG_MAGNITUDE)
    assert mag.push(_dev(stream[:nl])) == ss.SSOCT_OK
    mag.sliding_cuts(3, 4, 9)
    assert mag.push(_dev(stream[nl:nl + 7])) == ss.SSOCT_OK
    xy, _, _ = mag.sliding_cuts(3, 4, 9)               # running: 7 frames swapped in
    mag.sync()
    gate = stream[7:nl + 7]
    ref = oracle.reconstruct(np.roll(gate, 7 % nl, axis=0), a.pitch, a.z, a.lambdas, window=win, method="fft")
    err = _rel(xy.cpu().numpy().astype(np.float64), np.sqrt(oracle.intensity(ref)[9]))
    assert err <= 2 * TOL, f"running |V| xy: rel L2 {err:.3e}"
