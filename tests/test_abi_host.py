"""The C-ABI library without a GPU: it loads, exports every declared symbol,
validates arguments, and its host-built plan facts agree with the oracle's
closed forms.  No call here reaches CUDA."""

import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from paper_2003_08960_gb300 import build as ssbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ss():
    ssbuild.build()
    import paper_2003_08960_gb300 as ss
    return ss


def _declared_symbols():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"SSOCT_API[^;(]*?\b(ssoct_\w+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(ss):
    lib = ss._abi.lib()
    declared = _declared_symbols()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(ss._abi.SIGNATURES), "binding and header disagree"


LAM = np.linspace(800e-9, 850e-9, 32)


def test_create_plan_validation(ss):
    ok, h = ss.ssoct_create_plan(64, 64, 32, 20e-6, 0.3, LAM)
    assert ok == ss.SSOCT_OK and h
    ss.ssoct_destroy_plan(h)
    bad = [
        (63, 64, 32, 20e-6, 0.3, LAM, None),          # odd size
        (64, 64, 32, -1.0, 0.3, LAM, None),           # pitch
        (64, 64, 32, 20e-6, 0.0, LAM, None),          # z = 0
        (64, 64, 32, 20e-6, 0.3, -LAM, None),         # negative wavelengths
        (64, 64, 32, 20e-6, 0.3, LAM, (40, 0, 30, 10)),  # window outside
        (64, 64, 32, 20e-6, 0.3, LAM, (0, 0, 0, 10)),    # empty window
    ]
    for args in bad:
        st, h = ss.ssoct_create_plan(*args[:6], window=args[6])
        assert st == ss.SSOCT_EINVAL and h is None, args
    st, h = ss.ssoct_create_plan(96, 96, 32, 20e-6, 0.3, LAM)
    assert st == ss.SSOCT_EUNSUPPORTED
    st, h = ss.ssoct_create_plan(64, 64, 24, 20e-6, 0.3, np.linspace(800e-9, 850e-9, 24))
    assert st == ss.SSOCT_EUNSUPPORTED
    # unknown flag bits; the tensor-core axial form exists for nlambda = 256 only
    st, h = ss.ssoct_create_plan(64, 64, 32, 20e-6, 0.3, LAM, flags=0x10)
    assert st == ss.SSOCT_EINVAL
    # axial-first order: persistent-kernel sizes, even sweeps, not with the tensor-core form
    st, h = ss.ssoct_create_plan(64, 64, 32, 20e-6, 0.3, LAM, flags=ss.SSOCT_FLAG_AXIAL_FIRST)
    assert st == ss.SSOCT_OK
    ss.ssoct_destroy_plan(h)
    st, h = ss.ssoct_create_plan(384, 384, 32, 20e-6, 0.3, LAM, flags=ss.SSOCT_FLAG_AXIAL_FIRST)
    assert st == ss.SSOCT_OK
    ss.ssoct_destroy_plan(h)
    st, h = ss.ssoct_create_plan(640, 384, 32, 20e-6, 0.3, LAM, flags=ss.SSOCT_FLAG_AXIAL_FIRST)
    assert st == ss.SSOCT_EUNSUPPORTED
    lam256 = np.linspace(800e-9, 850e-9, 256)
    st, h = ss.ssoct_create_plan(64, 64, 256, 20e-6, 0.3, lam256,
                                 flags=ss.SSOCT_FLAG_AXIAL_FIRST | ss.SSOCT_FLAG_TC_AXIAL)
    assert st == ss.SSOCT_EUNSUPPORTED
    st, h = ss.ssoct_create_plan(64, 64, 32, 20e-6, 0.3, LAM, flags=ss.SSOCT_FLAG_TC_AXIAL)
    assert st == ss.SSOCT_EUNSUPPORTED and h is None
    lam256 = np.linspace(800e-9, 850e-9, 256)
    st, h = ss.ssoct_create_plan(64, 64, 256, 20e-6, 0.3, lam256, flags=ss.SSOCT_FLAG_TC_AXIAL)
    assert st == ss.SSOCT_OK
    st, bytes_tc = ss.ssoct_workspace_size(h)
    ss.ssoct_destroy_plan(h)
    st, h = ss.ssoct_create_plan(64, 64, 256, 20e-6, 0.3, lam256)
    st, bytes_plain = ss.ssoct_workspace_size(h)
    assert ss.ssoct_workspace_bytes(h) == (st, bytes_plain)
    ss.ssoct_destroy_plan(h)
    assert bytes_tc == bytes_plain      # every 256-frame plan keeps the BF16 operand table (the autotuner may switch)


def test_pupil_plan_validation(ss):
    """The aberration path: sizes it compiles, its workspace, and the calls it
    refuses without the flag, without a workspace or with bad coefficients."""
    st, h = ss.ssoct_create_plan(96, 64, 32, 20e-6, 0.3, LAM, flags=ss.SSOCT_FLAG_PUPIL)
    assert st == ss.SSOCT_EUNSUPPORTED
    st, h = ss.ssoct_create_plan(64, 1000, 32, 20e-6, 0.3, LAM, flags=ss.SSOCT_FLAG_PUPIL)
    assert st == ss.SSOCT_EUNSUPPORTED
    st, plain = ss.ssoct_create_plan(64, 64, 32, 20e-6, 0.3, LAM)
    st, h = ss.ssoct_create_plan(64, 64, 32, 20e-6, 0.3, LAM, flags=ss.SSOCT_FLAG_PUPIL)
    assert st == ss.SSOCT_OK
    _, b0 = ss.ssoct_workspace_size(plain)
    _, b1 = ss.ssoct_workspace_size(h)
    # c P table + one complex frame per wavelength + 4 chunks of partial Q + FP64 block, each 256-aligned
    assert b1 - b0 == 64 * 64 * 8 + 32 * 64 * 64 * 8 + 4 * 64 * 64 * 8 + 256
    assert ss.ssoct_set_pupil(plain, [0.1] * 15, 0.3) == ss.SSOCT_EINVAL
    assert ss.ssoct_set_pupil(h, [0.1] * 16, 0.3) == ss.SSOCT_EINVAL
    assert ss.ssoct_set_pupil(h, [float("nan")], 0.3) == ss.SSOCT_EINVAL
    assert ss.ssoct_set_pupil(h, [0.1] * 15, 0.0) == ss.SSOCT_EINVAL
    assert ss.ssoct_set_pupil(h, [0.1] * 15, 0.3) == ss.SSOCT_ENOMEM      # no workspace yet
    st, out = ss.ssoct_sharpness(h, 0, 0, 0)
    assert st == ss.SSOCT_ENOMEM
    ss.ssoct_destroy_plan(plain)
    ss.ssoct_destroy_plan(h)


def test_plan_info_matches_closed_forms(ss):
    lam = np.linspace(800e-9, 850e-9, 256)
    st, h = ss.ssoct_create_plan(1024, 1024, 256, 20e-6, 0.3, lam)
    assert st == 0
    st, info = ss.ssoct_plan_info(h)
    assert st == 0
    assert info.lambda1_m == lam[0]
    assert abs(info.dprime_x_m - oracle.reconstructed_pixel(lam[0], 0.3, 1024, 20e-6)) < 1e-18
    assert abs(info.z_b_m - oracle.fresnel_limit(1024, 20e-6, lam[0])) < 1e-15
    assert info.aliased_chirp == 1            # z = 0.3 m < z_b = 0.512 m
    k = oracle.fresnel_prefactor(20e-6, 0.3, lam[0])
    assert abs(complex(info.prefactor_re, info.prefactor_im) - k) < 1e-9 * abs(k)
    # workspace: tables + ring + scratch + 2 GiB intermediate for a full window
    assert info.workspace_bytes > 1024 * 1024 * 256 * 8
    assert info.window.wx == 1024 and info.window.wy == 1024
    ss.ssoct_destroy_plan(h)
    st, h = ss.ssoct_create_plan(64, 64, 32, 20e-6, 0.3, LAM)
    st, info = ss.ssoct_plan_info(h)
    assert info.aliased_chirp == 0            # z_b = 0.032 m
    ss.ssoct_destroy_plan(h)


def test_calls_without_workspace_or_gpu_fail_cleanly(ss):
    st, h = ss.ssoct_create_plan(64, 64, 32, 20e-6, 0.3, LAM)
    assert ss.ssoct_reconstruct_volume(h, 0, 0, 0) == ss.SSOCT_ENOMEM
    assert ss.ssoct_reconstruct_frames(h, 0, 0, 0, 0) == ss.SSOCT_ENOMEM
    assert ss.ssoct_push_frames(h, 0, 1, True, -1, 0) == ss.SSOCT_ENOMEM
    assert "workspace" in ss.ssoct_last_error(h)
    assert ss.ssoct_get_cuts(h, 0, 0, 0, 0, 0, 0, 0, 0) == ss.SSOCT_EINVAL
    assert ss.ssoct_get_cuts(h, 16, 64, 0, 0, 16, 0, 0, 0) == ss.SSOCT_EINVAL   # x0 out of range
    assert ss.ssoct_get_cuts(h, 16, 0, 0, 32, 16, 0, 0, 0) == ss.SSOCT_EINVAL   # z0 out of range
    assert ss.ssoct_set_workspace(h, 0, 1 << 20) == ss.SSOCT_EINVAL
    assert ss.ssoct_set_workspace(h, 256, 16) == ss.SSOCT_ENOMEM
    assert ss.ssoct_status_string(7) == "SSOCT_ETIMEOUT"
    ss.ssoct_destroy_plan(h)


def test_binding_refuses_without_gpu(ss):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError, match="CUDA device"):
        ss.Plan(64, 64, 32, 20e-6, 0.3, LAM)


def test_mixed_radix_plan_sizes(ss):
    """Square frames of 384, 640 and 768 run on the persistent lateral kernel;
    other mixed-radix sizes take the two-pass lateral path (its frame buffer
    shows in the workspace); sweep lengths 96, 160, 200 are compiled; other
    lengths and sizes are refused."""
    def ws(nx, ny, nl):
        lam = np.linspace(800e-9, 850e-9, nl)
        st, h = ss.ssoct_create_plan(nx, ny, nl, 20e-6, 0.3, lam)
        if st != ss.SSOCT_OK:
            return st, None
        _, b = ss.ssoct_workspace_size(h)
        ss.ssoct_destroy_plan(h)
        return st, b
    for nx, ny, nl in [(384, 384, 96), (640, 640, 160), (768, 768, 200), (640, 384, 32), (256, 256, 96)]:
        st, b = ws(nx, ny, nl)
        assert st == ss.SSOCT_OK, (nx, ny, nl)
    for nx, ny, nl in [(100, 64, 32), (384, 384, 100), (1280, 1280, 32), (256, 256, 48)]:
        st, _ = ws(nx, ny, nl)
        assert st == ss.SSOCT_EUNSUPPORTED, (nx, ny, nl)
    # two-pass plan: no scratch ring, a frame buffer [nl][ny][nx] and a chirp table instead
    _, b_gen = ws(640, 384, 32)
    frames = 32 * 640 * 384
    assert b_gen >= frames * 2 + frames * 8 + 640 * 384 * 8
    # the persistent kernel's plan of the same sweep holds no frame buffer
    _, b_sq = ws(384, 384, 32)
    assert b_sq < 32 * 384 * 384 * (2 + 8 + 8)


def test_batch_and_autotune_refuse_without_workspace(ss):
    st, h = ss.ssoct_create_plan(64, 64, 32, 20e-6, 0.3, LAM)
    assert st == ss.SSOCT_OK
    st, b = ss.ssoct_batch_create([h])
    assert st == ss.SSOCT_ENOMEM and b is None
    st, b = ss.ssoct_batch_create([])
    assert st == ss.SSOCT_EINVAL
    st, r = ss.ssoct_autotune(h, 0, 0, None, 0)
    assert st == ss.SSOCT_ENOMEM
    ss.ssoct_destroy_plan(h)
