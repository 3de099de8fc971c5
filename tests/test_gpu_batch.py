"""Batched graph launches of uneven volumes and the autotuner, on the GPU.

A batch runs the same kernels as separate reconstructs, so its volumes must be
bit-identical to them; a relaunch on the same pointers must not recapture.  The
autotuner only changes the schedule (bit-identical volume) or the axial form
(tensor-core rounding, relative L2 <= 1e-4 against the FP32 form), and a second
plan of the same shape must take its choice from the cache file.
"""

import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402


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


# (640, 384) takes the two-pass lateral path, the others the persistent kernel
SHAPES = [(64, 64, 32), (128, 128, 16), (384, 384, 96), (640, 384, 32), (256, 256, 64), (128, 64, 200)]


def test_batch_equals_separate_reconstructs(ss):
    ws = [synth.workload("custom", nx=nx, ny=ny, nlambda=nl, kind="points", seed=i)
          for i, (nx, ny, nl) in enumerate(SHAPES)]
    plans = [ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas) for w in ws]
    frames = [_dev(w.frames) for w in ws]
    refs = [p.reconstruct(f) for p, f in zip(plans, frames)]
    torch.cuda.synchronize()
    batch = ss.Batch(plans, lanes=0)
    vols = [p.empty_volume()[0] for p in plans]
    for _ in range(3):
        for v in vols:
            v.zero_()
        batch.run(frames, vols)
        batch.sync()
        for v, r in zip(vols, refs):
            assert torch.equal(v, r)
    assert batch.captures == 1
    other = [p.empty_volume()[0] for p in plans]
    batch.run(frames, other)
    batch.sync()
    assert batch.captures == 2
    for v, r in zip(other, refs):
        assert torch.equal(v, r)


def test_batch_refuses_duplicate_plans(ss):
    w = synth.workload("tiny_64x64x32")
    p = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas)
    with pytest.raises(ss.SsoctError):
        ss.Batch([p, p])


def test_autotune_choice_and_cache(ss, tmp_path):
    w = synth.workload("custom", nx=256, ny=256, nlambda=256, kind="points", seed=21)
    f = _dev(w.frames)
    ref = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas).reconstruct(f)
    cache = tmp_path / "tune.json"
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas)
    r = plan.autotune(f, cache)
    print("autotune 256x256x256:", r)
    # lateral schedules x (paper order with the FP32 or tensor-core axial pass,
    # axial-first order)
    assert r["from_cache"] == 0 and r["candidates"] % 3 == 0 and r["candidates"] >= 27 and r["ms"] > 0
    assert 1 <= r["lag"] and r["lag"] + 2 <= r["ring_slots"]
    assert not (r["tc_axial"] and r["axial_first"])
    v = plan.reconstruct(f)
    torch.cuda.synchronize()
    if r["tc_axial"]:
        assert float((v.double() - ref.double()).norm() / ref.double().norm()) <= 1e-4
    elif r["axial_first"]:
        assert float((v.double() - ref.double()).norm() / ref.double().norm()) <= 2e-6
    else:
        assert torch.equal(v, ref)
    entries = json.loads(cache.read_text())["entries"]
    assert len(entries) == 1 and entries[0]["lag"] == r["lag"]
    again = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas).autotune(f, cache)
    assert again["from_cache"] == 1
    assert (again["lag"], again["ring_slots"], again["tc_axial"], again["axial_first"]) == \
        (r["lag"], r["ring_slots"], r["tc_axial"], r["axial_first"])
    # a generic-path plan has no lateral schedule to tune; 96 frames have no tensor-core form
    g = synth.workload("custom", nx=640, ny=384, nlambda=96, kind="points", seed=22)
    gp = ss.Plan(g.nx, g.ny, g.nlambda, g.pitch, g.z, g.lambdas)
    rg = gp.autotune(_dev(g.frames), cache)
    assert rg["candidates"] == 1 and rg["tc_axial"] == 0
    assert len(json.loads(cache.read_text())["entries"]) == 2


def test_autotuned_axial_first_order(ss, tmp_path):
    """A plan made without SSOCT_FLAG_AXIAL_FIRST may be tuned to that order
    (here forced through an edited cache entry): whole-volume reconstructions
    then run it (the same V to FP32 rounding), while sliding gates and the
    no-allocation entry point keep the paper's order and give its volume bit
    for bit."""
    w = synth.workload("custom", nx=128, ny=128, nlambda=128, kind="points", seed=23)
    f = _dev(w.frames)
    ref = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas).reconstruct(f)
    cache = tmp_path / "tune.json"
    r = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas).autotune(f, cache)
    assert r["candidates"] % 2 == 0  # lateral schedules x 2 orders; 128 frames have no tensor-core form
    text = cache.read_text().replace('"axial_first": 0', '"axial_first": 1')
    cache.write_text(text)
    plan = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas)
    rf = plan.autotune(f, cache)
    assert rf["from_cache"] == 1 and rf["axial_first"] == 1 and rf["tc_axial"] == 0
    v = plan.reconstruct(f)
    torch.cuda.synchronize()
    err = float((v.double() - ref.double()).norm() / ref.double().norm())
    print(f"autotuned axial-first order vs paper order: rel L2 {err:.2e}")
    assert 0 < err <= 2e-6  # a different order of the same sums, not the same kernels
    assert plan.push(f) == ss.SSOCT_OK
    vs = plan.reconstruct_sliding()
    vn = torch.empty_like(ref)
    st = ss.ssoct_reconstruct_frames_noalloc(plan.handle, f.data_ptr(), vn.data_ptr(), 0,
                                             torch.cuda.current_stream().cuda_stream)
    assert st == ss.SSOCT_OK, ss.ssoct_last_error(plan.handle)
    torch.cuda.synchronize()
    assert ss.ssoct_sync(plan.handle, torch.cuda.current_stream().cuda_stream) == ss.SSOCT_OK
    assert torch.equal(vs, ref) and torch.equal(vn, ref)
    again = plan.reconstruct(f)   # and whole volumes are axial-first again
    torch.cuda.synchronize()
    assert torch.equal(again, v)
