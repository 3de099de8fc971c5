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


SHAPES = [(64, 64, 32), (128, 128, 16), (384, 384, 96), (256, 256, 64), (128, 64, 200)]


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
    assert r["from_cache"] == 0 and r["candidates"] == 18 and r["ms"] > 0
    assert 1 <= r["lag"] <= 3 and r["lag"] + 2 <= r["ring_slots"] <= 6
    v = plan.reconstruct(f)
    torch.cuda.synchronize()
    if r["tc_axial"]:
        assert float((v.double() - ref.double()).norm() / ref.double().norm()) <= 1e-4
    else:
        assert torch.equal(v, ref)
    entries = json.loads(cache.read_text())["entries"]
    assert len(entries) == 1 and entries[0]["lag"] == r["lag"]
    again = ss.Plan(w.nx, w.ny, w.nlambda, w.pitch, w.z, w.lambdas).autotune(f, cache)
    assert again["from_cache"] == 1
    assert (again["lag"], again["ring_slots"], again["tc_axial"]) == (r["lag"], r["ring_slots"], r["tc_axial"])
    # a generic-path plan has no lateral schedule to tune; 96 frames have no tensor-core form
    g = synth.workload("custom", nx=384, ny=384, nlambda=96, kind="points", seed=22)
    gp = ss.Plan(g.nx, g.ny, g.nlambda, g.pitch, g.z, g.lambdas)
    rg = gp.autotune(_dev(g.frames), cache)
    assert rg["candidates"] == 1 and rg["tc_axial"] == 0
    assert len(json.loads(cache.read_text())["entries"]) == 2
