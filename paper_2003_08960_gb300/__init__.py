"""Python binding of libssoct: swept-source holographic OCT reconstruction on one GPU.

Thin layer over the C ABI (include/ssoct.h): the functions below carry the C
names and only marshal arguments; every step of the reconstruction runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  If the
library is not built, or no CUDA device is present when a GPU call is made, the
call raises: there is no CPU path.

    plan = Plan(nx, ny, nlambda, pitch, z, lambdas, window=None)
    vol = plan.reconstruct(frames_u16_on_gpu)           # float32 [nlambda][wy][wx]
    xy, xz, yz = plan.cuts(vol, x0, y0, z0)
"""

from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence, Tuple

import numpy as np

from . import _abi
from ._abi import (  # noqa: F401
    SSOCT_EDROPPED, SSOCT_EINVAL, SSOCT_ENOMEM, SSOCT_ENOTREADY, SSOCT_EUNSUPPORTED, SSOCT_ETIMEOUT,
    SSOCT_FLAG_AXIAL_FIRST, SSOCT_FLAG_MAGNITUDE, SSOCT_FLAG_PUPIL, SSOCT_FLAG_TC_AXIAL, SSOCT_OK, ssoct_plan_info_t, ssoct_window,
)


class SsoctError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_abi.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status: int, plan=None, what: str = "") -> int:
    if status != SSOCT_OK:
        msg = _abi.lib().ssoct_last_error(plan).decode() if plan else ""
        raise SsoctError(status, f"{what} {msg}".strip())
    return status


# ---------------------------------------------------------------- C names

def ssoct_create_plan(nx: int, ny: int, nlambda: int, pitch_m: float, z_m: float,
                      lambda_m: Sequence[float], window: Optional[Tuple[int, int, int, int]] = None,
                      flags: int = 0):
    """Returns (status, plan handle or None)."""
    lam = np.ascontiguousarray(lambda_m, dtype=np.float64)
    if lam.shape != (nlambda,):
        return SSOCT_EINVAL, None
    h = _abi.ssoct_plan()
    w = ssoct_window(*window) if window is not None else None
    st = _abi.lib().ssoct_create_plan(nx, ny, nlambda, pitch_m, z_m,
                                      lam.ctypes.data_as(C.POINTER(C.c_double)),
                                      C.byref(w) if w is not None else None, flags, C.byref(h))
    return st, (h if st == SSOCT_OK else None)


def ssoct_plan_info(plan):
    info = ssoct_plan_info_t()
    st = _abi.lib().ssoct_plan_info(plan, C.byref(info))
    return st, info


def ssoct_workspace_size(plan):
    n = C.c_size_t()
    st = _abi.lib().ssoct_workspace_size(plan, C.byref(n))
    return st, n.value


def ssoct_workspace_bytes(plan):
    n = C.c_size_t()
    st = _abi.lib().ssoct_workspace_bytes(plan, C.byref(n))
    return st, n.value


def ssoct_set_workspace(plan, dev_ptr: int, nbytes: int) -> int:
    return _abi.lib().ssoct_set_workspace(plan, C.c_void_p(dev_ptr), nbytes)


def ssoct_push_frames(plan, frames_ptr: int, n: int, frames_on_device: bool, first_seq: int, stream: int) -> int:
    return _abi.lib().ssoct_push_frames(plan, C.c_void_p(frames_ptr), n, int(bool(frames_on_device)),
                                        first_seq, C.c_void_p(stream))


def ssoct_reconstruct_volume(plan, vol_ptr: int, complex_ptr: int, stream: int) -> int:
    return _abi.lib().ssoct_reconstruct_volume(plan, C.c_void_p(vol_ptr), C.c_void_p(complex_ptr or None),
                                               C.c_void_p(stream))


def ssoct_reconstruct_frames(plan, frames_ptr: int, vol_ptr: int, complex_ptr: int, stream: int) -> int:
    return _abi.lib().ssoct_reconstruct_frames(plan, C.c_void_p(frames_ptr), C.c_void_p(vol_ptr),
                                               C.c_void_p(complex_ptr or None), C.c_void_p(stream))


def ssoct_reconstruct_sliding(plan, vol_ptr: int, complex_ptr: int, stream: int) -> int:
    return _abi.lib().ssoct_reconstruct_sliding(plan, C.c_void_p(vol_ptr), C.c_void_p(complex_ptr or None),
                                                C.c_void_p(stream))


def ssoct_reconstruct_frames_noalloc(plan, frames_ptr: int, vol_ptr: int, complex_ptr: int, stream: int) -> int:
    """ssoct_reconstruct_frames without any device allocation (scratch in a fixed
    64 MiB device array inside the library); the plan needs no workspace."""
    return _abi.lib().ssoct_reconstruct_frames_noalloc(plan, C.c_void_p(frames_ptr), C.c_void_p(vol_ptr),
                                                       C.c_void_p(complex_ptr or None), C.c_void_p(stream))


def ssoct_get_cuts(plan, vol_ptr: int, x0: int, y0: int, z0: int, xy_ptr: int, xz_ptr: int, yz_ptr: int,
                   stream: int) -> int:
    return _abi.lib().ssoct_get_cuts(plan, C.c_void_p(vol_ptr), x0, y0, z0, C.c_void_p(xy_ptr or None),
                                     C.c_void_p(xz_ptr or None), C.c_void_p(yz_ptr or None), C.c_void_p(stream))


def ssoct_sync(plan, stream: int) -> int:
    return _abi.lib().ssoct_sync(plan, C.c_void_p(stream))


def ssoct_set_pupil(plan, coeffs: Sequence[float], z_m: float) -> int:
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    return _abi.lib().ssoct_set_pupil(plan, c.ctypes.data_as(C.POINTER(C.c_double)), int(c.size), float(z_m))


def ssoct_sharpness(plan, frames_ptr: int, vol_ptr: int, stream: int):
    """Returns (status, out[17]): loss, dL/dz, dL/dc_1 .. dL/dc_15."""
    out = np.zeros(17, dtype=np.float64)
    st = _abi.lib().ssoct_sharpness(plan, C.c_void_p(frames_ptr), C.c_void_p(vol_ptr),
                                    out.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(stream))
    return st, out


def ssoct_sliding_cuts(plan, x0: int, y0: int, z0: int, xy_ptr: int, xz_ptr: int, yz_ptr: int, stream: int) -> int:
    return _abi.lib().ssoct_sliding_cuts(plan, x0, y0, z0, C.c_void_p(xy_ptr or None), C.c_void_p(xz_ptr or None),
                                         C.c_void_p(yz_ptr or None), C.c_void_p(stream))


def ssoct_inject_stall(plan, skip: int, wait_limit_ns: int) -> int:
    """Test hook: make the next reconstructs skip `skip` work items so that
    dependent items time out after wait_limit_ns (see include/ssoct.h)."""
    return _abi.lib().ssoct_inject_stall(plan, skip, wait_limit_ns)


def ssoct_profile(plan, enable: bool) -> int:
    return _abi.lib().ssoct_profile(plan, int(bool(enable)))


def ssoct_profile_read(plan):
    """Returns (status, lateral_ms, axial_ms, calls)."""
    a, b, n = C.c_double(), C.c_double(), C.c_int()
    st = _abi.lib().ssoct_profile_read(plan, C.byref(a), C.byref(b), C.byref(n))
    return st, a.value, b.value, n.value


def ssoct_last_error(plan) -> str:
    return _abi.lib().ssoct_last_error(plan).decode()


def ssoct_status_string(status: int) -> str:
    return _abi.lib().ssoct_status_string(status).decode()


def ssoct_destroy_plan(plan) -> None:
    _abi.lib().ssoct_destroy_plan(plan)


# ---------------------------------------------------------------- convenience

def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libssoct needs a CUDA device; there is no CPU path")
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Plan:
    """A reconstruction plan with its device workspace (allocated through torch)."""

    def __init__(self, nx: int, ny: int, nlambda: int, pitch_m: float, z_m: float,
                 lambda_m: Sequence[float], window: Optional[Tuple[int, int, int, int]] = None,
                 flags: int = 0, device=None):
        st, h = ssoct_create_plan(nx, ny, nlambda, pitch_m, z_m, lambda_m, window, flags)
        _check(st, None, "create_plan")
        self._h = h
        self.nx, self.ny, self.nlambda = nx, ny, nlambda
        st, info = ssoct_plan_info(h)
        _check(st, h, "plan_info")
        self.info = info
        w = info.window
        self.window = (w.x0, w.y0, w.wx, w.wy)
        self.workspace = None
        torch = _torch()
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        with torch.cuda.device(dev):
            self.workspace = torch.empty(info.workspace_bytes, dtype=torch.uint8, device=dev)
            _check(ssoct_set_workspace(h, self.workspace.data_ptr(), info.workspace_bytes), h, "set_workspace")

    def close(self):
        if getattr(self, "_h", None):
            ssoct_destroy_plan(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def volume_shape(self):
        return (self.nlambda, self.window[3], self.window[2])

    def empty_volume(self, complex_out: bool = False):
        torch = _torch()
        vol = torch.empty(self.volume_shape(), dtype=torch.float32, device=self.device)
        cplx = torch.empty(self.volume_shape(), dtype=torch.complex64, device=self.device) if complex_out else None
        return vol, cplx

    def reconstruct(self, frames, out=None, complex_out: bool = False, stream=None):
        """frames: uint16-valued torch tensor [nlambda][ny][nx] on this device
        (dtype torch.uint16, or int16 holding the same bits)."""
        torch = _torch()
        if frames.device != self.device or not frames.is_contiguous() or frames.element_size() != 2:
            raise ValueError("frames must be a contiguous 16-bit tensor on the plan's device")
        if tuple(frames.shape) != (self.nlambda, self.ny, self.nx):
            raise ValueError(f"frames must be [{self.nlambda}][{self.ny}][{self.nx}]")
        vol, cplx = out if out is not None else self.empty_volume(complex_out)
        _check(ssoct_reconstruct_frames(self._h, frames.data_ptr(), vol.data_ptr(),
                                        cplx.data_ptr() if cplx is not None else 0, _stream_ptr(stream)),
               self._h, "reconstruct_frames")
        return (vol, cplx) if complex_out else vol

    def push(self, frames, first_seq: int = -1, stream=None) -> int:
        """Append frames (torch tensor on this device, or a numpy uint16 array on
        the host) to the plan's ring.  Returns the status (OK or EDROPPED)."""
        if isinstance(frames, np.ndarray):
            if frames.dtype != np.uint16 or not frames.flags.c_contiguous:
                raise ValueError("host frames must be C-contiguous uint16")
            n = frames.shape[0] if frames.ndim == 3 else 1
            st = ssoct_push_frames(self._h, frames.ctypes.data, n, False, first_seq, _stream_ptr(stream))
        else:
            n = frames.shape[0] if frames.dim() == 3 else 1
            st = ssoct_push_frames(self._h, frames.data_ptr(), n, frames.is_cuda, first_seq, _stream_ptr(stream))
        if st not in (SSOCT_OK, SSOCT_EDROPPED):
            _check(st, self._h, "push_frames")
        return st

    def reconstruct_ring(self, out=None, complex_out: bool = False, stream=None):
        vol, cplx = out if out is not None else self.empty_volume(complex_out)
        _check(ssoct_reconstruct_volume(self._h, vol.data_ptr(), cplx.data_ptr() if cplx is not None else 0,
                                        _stream_ptr(stream)), self._h, "reconstruct_volume")
        return (vol, cplx) if complex_out else vol

    def reconstruct_sliding(self, out=None, complex_out: bool = False, stream=None):
        """Volume of the last nlambda pushed frames of a periodic sweep (sliding
        gate); only frames pushed since the previous call are transformed."""
        vol, cplx = out if out is not None else self.empty_volume(complex_out)
        _check(ssoct_reconstruct_sliding(self._h, vol.data_ptr(), cplx.data_ptr() if cplx is not None else 0,
                                         _stream_ptr(stream)), self._h, "reconstruct_sliding")
        return (vol, cplx) if complex_out else vol

    def sliding_cuts(self, x0: int, y0: int, z0: int, stream=None):
        """The three cuts of the sliding gate (see ssoct_sliding_cuts)."""
        torch = _torch()
        nl, wy, wx = self.volume_shape()
        xy = torch.empty((wy, wx), dtype=torch.float32, device=self.device)
        xz = torch.empty((nl, wx), dtype=torch.float32, device=self.device)
        yz = torch.empty((nl, wy), dtype=torch.float32, device=self.device)
        _check(ssoct_sliding_cuts(self._h, x0, y0, z0, xy.data_ptr(), xz.data_ptr(), yz.data_ptr(),
                                  _stream_ptr(stream)), self._h, "sliding_cuts")
        return xy, xz, yz

    def cuts(self, vol, x0: int, y0: int, z0: int, stream=None):
        torch = _torch()
        nl, wy, wx = self.volume_shape()
        xy = torch.empty((wy, wx), dtype=torch.float32, device=self.device)
        xz = torch.empty((nl, wx), dtype=torch.float32, device=self.device)
        yz = torch.empty((nl, wy), dtype=torch.float32, device=self.device)
        _check(ssoct_get_cuts(self._h, vol.data_ptr(), x0, y0, z0, xy.data_ptr(), xz.data_ptr(), yz.data_ptr(),
                              _stream_ptr(stream)), self._h, "get_cuts")
        return xy, xz, yz

    def sync(self, stream=None) -> None:
        _check(ssoct_sync(self._h, _stream_ptr(stream)), self._h, "sync")

    def autotune(self, frames, cache_path=None, stream=None) -> dict:
        """Time this plan's candidate schedules on `frames` and keep the fastest
        (see ssoct_autotune); returns the choice."""
        vol, _ = self.empty_volume()
        st, r = ssoct_autotune(self._h, frames.data_ptr(), vol.data_ptr(), cache_path, _stream_ptr(stream))
        _check(st, self._h, "autotune")
        return r

    def sharpness(self, frames, coeffs: Sequence[float], z_m: float, out=None, stream=None):
        """(loss, grad[16], volume) of the pupil-corrected reconstruction: grad[0] =
        dL/dz, grad[j] = dL/dc_j (needs a plan made with SSOCT_FLAG_PUPIL)."""
        _check(ssoct_set_pupil(self._h, coeffs, z_m), self._h, "set_pupil")
        vol = out if out is not None else self.empty_volume()[0]
        st, res = ssoct_sharpness(self._h, frames.data_ptr(), vol.data_ptr(), _stream_ptr(stream))
        _check(st, self._h, "sharpness")
        return float(res[0]), res[1:].copy(), vol


def ssoct_autotune(plan, frames_ptr: int, vol_ptr: int, cache_path, stream: int):
    """Returns (status, dict with lag, ring_slots, tc_axial, ms, from_cache, candidates, axial_first)."""
    r = _abi.ssoct_tune_t()
    path = None if cache_path is None else str(cache_path).encode()
    st = _abi.lib().ssoct_autotune(plan, C.c_void_p(frames_ptr), C.c_void_p(vol_ptr), path, C.c_void_p(stream),
                                   C.byref(r))
    return st, {k: getattr(r, k) for k, _ in r._fields_}


def ssoct_batch_create(plans, lanes: int = 1):
    """Returns (status, batch handle or None) for a list of plan handles."""
    arr = (_abi.ssoct_plan * len(plans))(*plans)
    out = C.c_void_p()
    st = _abi.lib().ssoct_batch_create(arr, len(plans), lanes, C.byref(out))
    return st, (out.value if st == SSOCT_OK else None)


def ssoct_batch_run(batch, frame_ptrs, vol_ptrs, stream: int) -> int:
    n = len(frame_ptrs)
    fa = (C.c_void_p * n)(*frame_ptrs)
    va = (C.c_void_p * n)(*vol_ptrs)
    return _abi.lib().ssoct_batch_run(batch, fa, va, C.c_void_p(stream))


def ssoct_batch_sync(batch, stream: int) -> int:
    return _abi.lib().ssoct_batch_sync(batch, C.c_void_p(stream))


def ssoct_batch_captures(batch) -> int:
    return _abi.lib().ssoct_batch_captures(batch)


def ssoct_batch_last_error(batch) -> str:
    return _abi.lib().ssoct_batch_last_error(batch).decode()


def ssoct_batch_destroy(batch) -> None:
    _abi.lib().ssoct_batch_destroy(batch)


class Batch:
    """Several plans reconstructed by one CUDA graph launch (see ssoct_batch_run)."""

    def __init__(self, plans, lanes: int = 1):
        self.plans = list(plans)
        st, self._b = ssoct_batch_create([p.handle for p in self.plans], lanes)
        if st != SSOCT_OK:
            raise SsoctError(st, "batch_create")

    def run(self, frames, vols, stream=None) -> None:
        st = ssoct_batch_run(self._b, [f.data_ptr() for f in frames], [v.data_ptr() for v in vols],
                             _stream_ptr(stream))
        if st != SSOCT_OK:
            raise SsoctError(st, "batch_run " + ssoct_batch_last_error(self._b))

    def sync(self, stream=None) -> None:
        st = ssoct_batch_sync(self._b, _stream_ptr(stream))
        if st != SSOCT_OK:
            raise SsoctError(st, "batch_sync " + ssoct_batch_last_error(self._b))

    @property
    def captures(self) -> int:
        return ssoct_batch_captures(self._b)

    def __del__(self):
        if getattr(self, "_b", None):
            ssoct_batch_destroy(self._b)
            self._b = None
