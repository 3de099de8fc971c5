"""The no-allocation entry point, through the C ABI, against ssoct_reconstruct_frames.

ssoct_reconstruct_frames_noalloc serves callers that cannot allocate device
memory (acquisition loops that must not allocate mid-stream, plug-ins whose host
application owns the device heap).  Its plans get no workspace; its scratch is a
fixed device array inside the library.  Each call must reproduce the workspace
path's volume and complex volume within the parity tolerance used throughout
the tests (relative L2 <= 1e-5), on consecutive calls that switch between plans
of different sizes (the shared array keeps the previous call's contents).
This file is named so that pytest collects it last.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def ss():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_08960_gb300 import build
    build.build()
    import paper_2003_08960_gb300 as ss
    return ss


def _rel(a, b):
    a = a.double().cpu().numpy() if a.dtype != torch.complex64 else a.cpu().numpy().astype(np.complex128)
    b = b.double().cpu().numpy() if b.dtype != torch.complex64 else b.cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(ss, w, window, flags=0):
    """Reference outputs from the workspace path, plus a workspace-less plan."""
    frames = torch.from_numpy(np.ascontiguousarray(w.frames).view(np.int16)).cuda()
    ref_plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas, window=window, flags=flags)
    vol_ref, cplx_ref = ref_plan.reconstruct(frames, complex_out=True)
    st, h = ss.ssoct_create_plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas, window, flags)
    assert st == ss.SSOCT_OK
    vol = torch.empty_like(vol_ref)
    cplx = torch.empty_like(cplx_ref)
    return dict(frames=frames, ref_plan=ref_plan, vol_ref=vol_ref, cplx_ref=cplx_ref, h=h, vol=vol, cplx=cplx)


def _call(ss, c):
    c["vol"].fill_(float("nan"))
    c["cplx"].fill_(float("nan"))
    stream = torch.cuda.current_stream().cuda_stream
    st = ss.ssoct_reconstruct_frames_noalloc(c["h"], c["frames"].data_ptr(), c["vol"].data_ptr(),
                                             c["cplx"].data_ptr(), stream)
    assert st == ss.SSOCT_OK, ss.ssoct_last_error(c["h"])
    torch.cuda.synchronize()
    assert torch.isfinite(c["vol"]).all()
    assert _rel(c["vol"], c["vol_ref"]) <= TOL
    assert _rel(c["cplx"], c["cplx_ref"]) <= TOL


def test_noalloc_matches_workspace_path_on_consecutive_calls(ss):
    import synth
    a = _case(ss, synth.workload("tiny_64x64x32"), None)
    b = _case(ss, synth.workload("custom", nx=128, ny=128, nlambda=16, kind="points", seed=12), (20, 36, 77, 50))
    # 128 frames: the persistent, TMA-fed axial kernel, its error word in the array
    c = _case(ss, synth.workload("custom", nx=64, ny=64, nlambda=128, kind="points", seed=13), (3, 5, 57, 41))
    # the tensor-core axial form: its BF16 DFT operand table is uploaded into the
    # array over whatever the previous plan left there
    d = _case(ss, synth.workload("custom", nx=64, ny=64, nlambda=256, kind="points", seed=14), None,
              flags=ss.SSOCT_FLAG_TC_AXIAL)
    try:
        _call(ss, a)
        _call(ss, a)   # two calls in a row on the same plan
        _call(ss, b)   # a different size and a ragged window over the same array
        _call(ss, c)
        _call(ss, d)
        _call(ss, a)   # and back
        _call(ss, d)
    finally:
        for x in (a, b, c, d):
            ss.ssoct_destroy_plan(x["h"])


def test_noalloc_reports_a_kernel_time_out(ss):
    """A bounded device wait that runs out on this path leaves its error word in
    the shared array; ssoct_sync on the plan reports it, and the next call
    without the injected stall reproduces the workspace path again."""
    import synth
    a = _case(ss, synth.workload("tiny_64x64x32"), None)
    stream = torch.cuda.current_stream().cuda_stream
    try:
        assert ss.ssoct_inject_stall(a["h"], 1, 50_000_000) == ss.SSOCT_OK
        st = ss.ssoct_reconstruct_frames_noalloc(a["h"], a["frames"].data_ptr(), a["vol"].data_ptr(),
                                                 a["cplx"].data_ptr(), stream)
        assert st == ss.SSOCT_OK
        assert ss.ssoct_sync(a["h"], stream) == ss.SSOCT_ETIMEOUT
        assert "no-allocation" in ss.ssoct_last_error(a["h"])
        assert ss.ssoct_inject_stall(a["h"], 0, 0) == ss.SSOCT_OK
        _call(ss, a)
        assert ss.ssoct_sync(a["h"], stream) == ss.SSOCT_OK
    finally:
        ss.ssoct_destroy_plan(a["h"])


def test_noalloc_axial_pass_spans_the_gpu(ss):
    """The persistent axial kernel sizes its grid by the SM count: the path must
    pass the device's, not a plan field it never sets.  At 256 x 256 x 64 the
    axial pass alone on one SM's worth of CTAs would take milliseconds; the whole
    call (table uploads included) must stay within 1 ms of the workspace path."""
    import synth
    a = _case(ss, synth.workload("custom", nx=256, ny=256, nlambda=64, kind="points", seed=15), None)
    stream = torch.cuda.current_stream().cuda_stream
    try:
        def timed(fn):
            best = float("inf")
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            return best
        ws_ms = timed(lambda: a["ref_plan"].reconstruct(a["frames"], out=(a["vol_ref"], None)))
        na_ms = timed(lambda: ss.ssoct_reconstruct_frames_noalloc(a["h"], a["frames"].data_ptr(),
                                                                  a["vol"].data_ptr(), 0, stream))
        print(f"256x256x64: workspace path {ws_ms:.3f} ms, no-allocation path {na_ms:.3f} ms")
        assert na_ms < ws_ms + 1.0
        _call(ss, a)
    finally:
        ss.ssoct_destroy_plan(a["h"])


def test_noalloc_rejects_plans_beyond_its_array(ss):
    lam = np.linspace(800e-9, 850e-9, 32)
    st, h = ss.ssoct_create_plan(512, 512, 32, 20e-6, 0.3, lam)
    assert st == ss.SSOCT_OK
    try:
        vol = torch.empty((32, 512, 512), dtype=torch.float32, device="cuda")
        frames = torch.zeros((32, 512, 512), dtype=torch.int16, device="cuda")
        st = ss.ssoct_reconstruct_frames_noalloc(h, frames.data_ptr(), vol.data_ptr(), 0,
                                                 torch.cuda.current_stream().cuda_stream)
        assert st == ss.SSOCT_EUNSUPPORTED
        assert "64 MiB" in ss.ssoct_last_error(h)
    finally:
        ss.ssoct_destroy_plan(h)
