"""Thin ctypes binding of libwavestep (include/wavestep.h), same names as the C ABI.

Argument marshalling only: every computation runs in the library's CUDA
kernels. Arrays may be numpy arrays (host), or torch tensors on the CPU or on
the current CUDA device (float32, contiguous, [nz][ny][nx] for grid arrays).
Every call raises :class:`WaveStepError` when the library returns an error.
There is no fallback: if the library is missing, loading raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

WS_OK = 0
WS_ERR_BADARG = -1
WS_ERR_CFL = -2
WS_ERR_OOM = -3
WS_ERR_CUDA = -4
WS_ERR_TIMEOUT = -5
WS_ERR_STATE = -6

WS_KERNEL_AUTO = 0
WS_KERNEL_DIRECT = 1
WS_KERNEL_STREAM = 2

WS_STORAGE_FP32 = 0
WS_STORAGE_BF16 = 1
WS_STORAGE_FP16 = 2

WS_MAX_SOURCES = 16

WS_ADJ_DATA = 0
WS_ADJ_RESIDUAL = 1


class WaveStepError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"[{code}] {message}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = False):
    """Load libwavestep.so (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise OSError(f"libwavestep.so is not built ({path}); run "
                      "paper_2204_03775_gb300.build.build() or __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "ws_create": (i, [ctypes.POINTER(vp), i, i, i, d, d]),
        "ws_destroy": (i, [vp]),
        "ws_set_stream": (i, [vp, vp]),
        "ws_set_velocity": (i, [vp, vp, i]),
        "ws_set_slowness2": (i, [vp, vp, i]),
        "ws_adjoint_gradient": (i, [vp, vp, i, vp, ctypes.POINTER(d), i]),
        "ws_forward": (i, [vp]),
        "ws_adjoint_gradient_shots": (i, [ctypes.POINTER(vp), i, ctypes.POINTER(vp), i, vp,
                                          ctypes.POINTER(d), ctypes.POINTER(d), i]),
        "ws_set_sponge": (i, [vp, i, d]),
        "ws_add_source": (i, [vp, i, i, i, d, d, d]),
        "ws_clear_sources": (i, [vp]),
        "ws_set_receivers": (i, [vp, i, vp, i]),
        "ws_step": (i, [vp, i]),
        "ws_read_traces": (i, [vp, vp, i]),
        "ws_read_field": (i, [vp, vp, vp, i]),
        "ws_write_field": (i, [vp, vp, vp, ll, i]),
        "ws_get_step": (i, [vp, ctypes.POINTER(ll)]),
        "ws_set_kernel": (i, [vp, i, i, i, i]),
        "ws_set_storage": (i, [vp, i]),
        "ws_synchronize": (i, [vp]),
        "ws_launch_count": (ll, [vp]),
        "ws_energy": (i, [vp, ctypes.POINTER(d)]),
        "ws_energy_noalloc": (i, [vp, vp, vp, i, i, i, d, d, vp, vp]),
        "ws_last_error": (ctypes.c_char_p, []),
        "ws_autotune": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
        "ws_test_stall": (i, [vp, i]),
        "ws_test_fill_padding": (i, [vp]),
        "ws_test_check_padding": (i, [vp, ctypes.POINTER(ll)]),
        "ws_batch_create": (i, [ctypes.POINTER(vp), i, vp]),
        "ws_batch_destroy": (i, [vp]),
        "ws_batch_set_tiling": (i, [vp, i, i, i]),
        "ws_batch_get_tiling": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
        "ws_batch_step": (i, [vp, i]),
        "ws_batch_synchronize": (i, [vp]),
        "ws_batch_launch_count": (ll, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def ws_last_error() -> str:
    return load_library().ws_last_error().decode()


def _check(rc: int, name: str) -> None:
    if rc != WS_OK:
        raise WaveStepError(rc, f"{name}: {ws_last_error()}")


def _ptr(a, shape=None, dtype="float32"):
    """(pointer, on_device) of a host/device array; validates dtype, contiguity, shape."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype) or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {dtype} array")
        if shape is not None and tuple(a.shape) != tuple(shape):
            raise ValueError(f"expected shape {tuple(shape)}, got {a.shape}")
        return a.ctypes.data, 0
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != getattr(torch, dtype) or not a.is_contiguous():
            raise TypeError(f"expected a contiguous torch.{dtype} tensor")
        if shape is not None and tuple(a.shape) != tuple(shape):
            raise ValueError(f"expected shape {tuple(shape)}, got {tuple(a.shape)}")
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError(f"unsupported array type {type(a)}")


class Handle:
    """Owned ws_t; destroyed on garbage collection or by ws_destroy."""

    def __init__(self, ptr: int, shape):
        self.ptr = ctypes.c_void_p(ptr)
        self.shape = shape  # (nz, ny, nx)
        self.nrec = 0
        self.nt_max = 0
        self.batches = 0    # live batches that reference this handle

    def __del__(self):
        if self.ptr and _lib is not None:
            _lib.ws_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(None)


def ws_create(nx: int, ny: int, nz: int, h: float, dt: float) -> Handle:
    lib = load_library()
    out = ctypes.c_void_p()
    _check(lib.ws_create(ctypes.byref(out), nx, ny, nz, h, dt), "ws_create")
    return Handle(out.value, (nz, ny, nx))


def ws_destroy(ws: Handle) -> None:
    if ws.batches:
        raise WaveStepError(WS_ERR_STATE, "ws_destroy: a live batch still references this "
                                          "handle; destroy the batch first")
    if ws.ptr:
        _check(load_library().ws_destroy(ws.ptr), "ws_destroy")
        ws.ptr = ctypes.c_void_p(None)


def ws_set_stream(ws: Handle, stream) -> None:
    """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(load_library().ws_set_stream(ws.ptr, ctypes.c_void_p(raw or None)), "ws_set_stream")


def ws_set_velocity(ws: Handle, v) -> None:
    p, dev = _ptr(v, ws.shape)
    _check(load_library().ws_set_velocity(ws.ptr, ctypes.c_void_p(p), dev), "ws_set_velocity")


def ws_set_slowness2(ws: Handle, m) -> None:
    p, dev = _ptr(m, ws.shape)
    _check(load_library().ws_set_slowness2(ws.ptr, ctypes.c_void_p(p), dev), "ws_set_slowness2")


def ws_adjoint_gradient(ws: Handle, data, mode: int = WS_ADJ_DATA, grad_m=None):
    """(dJ/dm [nz][ny][nx], J) of the trace misfit; data [nrec][nt_max] float32.

    grad_m (optional) receives the gradient; host and device arrays must not
    be mixed. Returns (grad_m, misfit)."""
    pd, dd = _ptr(data, (ws.nrec, ws.nt_max))
    if grad_m is None:
        if dd:
            import torch
            grad_m = torch.empty(ws.shape, dtype=torch.float32, device=data.device)
        else:
            grad_m = np.empty(ws.shape, np.float32)
    pg, dg = _ptr(grad_m, ws.shape)
    if dd != dg:
        raise ValueError("data and grad_m must both be host or both be device arrays")
    j = ctypes.c_double()
    _check(load_library().ws_adjoint_gradient(ws.ptr, ctypes.c_void_p(pd), int(mode),
                                              ctypes.c_void_p(pg), ctypes.byref(j), dd),
           "ws_adjoint_gradient")
    return grad_m, j.value


def ws_adjoint_gradient_shots(shots, data, mode: int = WS_ADJ_DATA, grad_m=None):
    """(sum of dJ_s/dm [nz][ny][nx], summed J, FP64 ||gradient||_2) of several
    shots on grids of one size; data: one [nrec_s][nt_max] float32 array per
    shot, all host or all device arrays (grad_m alike)."""
    shots = list(shots)
    data = list(data)
    if len(shots) != len(data) or not shots:
        raise ValueError("one data array per shot, at least one shot")
    ptrs, devs = zip(*(_ptr(d, (h.nrec, h.nt_max)) for h, d in zip(shots, data)))
    if len(set(devs)) != 1:
        raise ValueError("data arrays must all be host or all be device arrays")
    dd = devs[0]
    if grad_m is None:
        if dd:
            import torch
            grad_m = torch.empty(shots[0].shape, dtype=torch.float32, device=data[0].device)
        else:
            grad_m = np.empty(shots[0].shape, np.float32)
    pg, dg = _ptr(grad_m, shots[0].shape)
    if dd != dg:
        raise ValueError("data and grad_m must both be host or both be device arrays")
    hs = (ctypes.c_void_p * len(shots))(*(h.ptr.value for h in shots))
    ds = (ctypes.c_void_p * len(shots))(*ptrs)
    j, gn = ctypes.c_double(), ctypes.c_double()
    _check(load_library().ws_adjoint_gradient_shots(hs, len(shots), ds, int(mode),
                                                    ctypes.c_void_p(pg), ctypes.byref(j),
                                                    ctypes.byref(gn), dd),
           "ws_adjoint_gradient_shots")
    return grad_m, j.value, gn.value


def ws_forward(ws: Handle) -> None:
    """Forward run from rest over nt_max steps, keeping the adjoint's checkpoints."""
    _check(load_library().ws_forward(ws.ptr), "ws_forward")


def ws_set_sponge(ws: Handle, nb: int, a: float) -> None:
    _check(load_library().ws_set_sponge(ws.ptr, int(nb), float(a)), "ws_set_sponge")


def ws_add_source(ws: Handle, ix: int, iy: int, iz: int, f0: float, t0: float, amp: float) -> None:
    _check(load_library().ws_add_source(ws.ptr, int(ix), int(iy), int(iz), float(f0), float(t0),
                                        float(amp)), "ws_add_source")


def ws_clear_sources(ws: Handle) -> None:
    _check(load_library().ws_clear_sources(ws.ptr), "ws_clear_sources")


def ws_set_receivers(ws: Handle, ijk, nt_max: int) -> None:
    ijk = np.ascontiguousarray(np.asarray(ijk, dtype=np.int32).reshape(-1, 3))
    _check(load_library().ws_set_receivers(ws.ptr, ijk.shape[0], ctypes.c_void_p(ijk.ctypes.data),
                                           int(nt_max)), "ws_set_receivers")
    ws.nrec, ws.nt_max = ijk.shape[0], (int(nt_max) if ijk.shape[0] else 0)


def ws_step(ws: Handle, nsteps: int) -> None:
    _check(load_library().ws_step(ws.ptr, int(nsteps)), "ws_step")


def ws_read_traces(ws: Handle, out=None):
    """Traces [nrec][nt_max] float32 into out (numpy/torch), or a new numpy array."""
    if out is None:
        out = np.zeros((ws.nrec, ws.nt_max), dtype=np.float32)
    p, dev = _ptr(out, (ws.nrec, ws.nt_max))
    if ws.nrec:
        _check(load_library().ws_read_traces(ws.ptr, ctypes.c_void_p(p), dev), "ws_read_traces")
    return out


def ws_read_field(ws: Handle, u=None, u_prev=None, *, new: bool = True):
    """(u^n, u^{n-1}) as [nz][ny][nx] float32; allocates numpy arrays when new=True."""
    if new and u is None and u_prev is None:
        u = np.empty(ws.shape, np.float32)
        u_prev = np.empty(ws.shape, np.float32)
    pu, du = _ptr(u, ws.shape)
    pp, dp = _ptr(u_prev, ws.shape)
    if u is not None and u_prev is not None and du != dp:
        raise ValueError("u and u_prev must both be host or both be device arrays")
    _check(load_library().ws_read_field(ws.ptr, ctypes.c_void_p(pu), ctypes.c_void_p(pp),
                                        du if u is not None else dp), "ws_read_field")
    return u, u_prev


def ws_write_field(ws: Handle, u, u_prev, step: int) -> None:
    pu, du = _ptr(u, ws.shape)
    pp, dp = _ptr(u_prev, ws.shape)
    if u is not None and u_prev is not None and du != dp:
        raise ValueError("u and u_prev must both be host or both be device arrays")
    _check(load_library().ws_write_field(ws.ptr, ctypes.c_void_p(pu), ctypes.c_void_p(pp),
                                         int(step), du if u is not None else dp), "ws_write_field")


def ws_get_step(ws: Handle) -> int:
    s = ctypes.c_longlong()
    _check(load_library().ws_get_step(ws.ptr, ctypes.byref(s)), "ws_get_step")
    return s.value


def ws_set_kernel(ws: Handle, kernel: int, tile_x: int = 0, tile_y: int = 0, zblock: int = 0) -> None:
    _check(load_library().ws_set_kernel(ws.ptr, int(kernel), int(tile_x), int(tile_y), int(zblock)),
           "ws_set_kernel")


def ws_set_storage(ws: Handle, storage: int) -> None:
    _check(load_library().ws_set_storage(ws.ptr, int(storage)), "ws_set_storage")


def ws_synchronize(ws: Handle) -> None:
    _check(load_library().ws_synchronize(ws.ptr), "ws_synchronize")


def ws_energy(ws: Handle) -> float:
    e = ctypes.c_double()
    _check(load_library().ws_energy(ws.ptr, ctypes.byref(e)), "ws_energy")
    return e.value


def ws_energy_noalloc(u, u_prev, v, h: float, dt: float, out, stream=None) -> None:
    """Energy of device arrays [nz][ny][nx] into the device double out[0]; allocates nothing.

    All four tensors must sit on one CUDA device; the call is made with that
    device current, on ``stream`` (default: torch's current stream of that
    device, so the call is ordered after the work that produced the inputs
    and before the work that reads ``out``). It returns without waiting.
    """
    import torch
    for t in (u, u_prev, v):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
                and t.is_contiguous() and t.dim() == 3 and t.shape == u.shape):
            raise TypeError("u, u_prev, v: contiguous float32 CUDA tensors of one [nz][ny][nx] shape")
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64
            and out.numel() >= 1):
        raise TypeError("out: a float64 CUDA tensor")
    dev = u.device
    if any(t.device != dev for t in (u_prev, v, out)):
        raise TypeError("u, u_prev, v and out must be on one CUDA device")
    nz, ny, nx = u.shape
    with torch.cuda.device(dev):
        if stream is None:
            raw = torch.cuda.current_stream(dev).cuda_stream
        else:
            raw = getattr(stream, "cuda_stream", stream)
        _check(load_library().ws_energy_noalloc(
            ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u_prev.data_ptr()),
            ctypes.c_void_p(v.data_ptr()), nx, ny, nz, float(h), float(dt),
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(raw or None)), "ws_energy_noalloc")


def ws_autotune(ws: Handle):
    """Time the streaming kernel's tilings on this grid; returns (tile_x, tile_y, zblock)."""
    tx, ty, zb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load_library().ws_autotune(ws.ptr, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(zb)),
           "ws_autotune")
    return tx.value, ty.value, zb.value


class Batch:
    """Owned ws_batch_t; keeps its shot handles alive; destroyed before them."""

    def __init__(self, ptr: int, shots):
        self.ptr = ctypes.c_void_p(ptr)
        self.shots = list(shots)
        for h in self.shots:
            h.batches += 1

    def _release(self):
        if self.ptr and _lib is not None:
            _lib.ws_batch_destroy(self.ptr)
        if self.ptr:
            for h in self.shots:
                h.batches -= 1
        self.ptr = ctypes.c_void_p(None)

    def __del__(self):
        self._release()


def ws_batch_create(shots) -> Batch:
    shots = list(shots)
    arr = (ctypes.c_void_p * len(shots))(*[h.ptr.value for h in shots])
    out = ctypes.c_void_p()
    _check(load_library().ws_batch_create(ctypes.byref(out), len(shots),
                                          ctypes.cast(arr, ctypes.c_void_p)), "ws_batch_create")
    return Batch(out.value, shots)


def ws_batch_destroy(b: Batch) -> None:
    b._release()


def ws_batch_set_tiling(b: Batch, tile_x: int, tile_y: int, zmul: int = 0) -> None:
    _check(load_library().ws_batch_set_tiling(b.ptr, int(tile_x), int(tile_y), int(zmul)),
           "ws_batch_set_tiling")


def ws_batch_get_tiling(b: Batch):
    tx, ty, zm = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load_library().ws_batch_get_tiling(b.ptr, ctypes.byref(tx), ctypes.byref(ty),
                                              ctypes.byref(zm)), "ws_batch_get_tiling")
    return tx.value, ty.value, zm.value


def ws_batch_step(b: Batch, nsteps: int) -> None:
    _check(load_library().ws_batch_step(b.ptr, int(nsteps)), "ws_batch_step")


def ws_batch_synchronize(b: Batch) -> None:
    _check(load_library().ws_batch_synchronize(b.ptr), "ws_batch_synchronize")


def ws_batch_launch_count(b: Batch) -> int:
    return int(load_library().ws_batch_launch_count(b.ptr))


def ws_test_stall(ws: Handle, item: int) -> None:
    """Test hook: the next streaming step withholds one copy of work item `item` (see header)."""
    _check(load_library().ws_test_stall(ws.ptr, int(item)), "ws_test_stall")


def ws_test_fill_padding(ws: Handle) -> None:
    """Write NaN canaries into the row padding of every field buffer (test hook)."""
    _check(load_library().ws_test_fill_padding(ws.ptr), "ws_test_fill_padding")


def ws_test_check_padding(ws: Handle) -> int:
    """Cells outside the interior that changed since the canaries were written."""
    n = ctypes.c_longlong(0)
    _check(load_library().ws_test_check_padding(ws.ptr, ctypes.byref(n)), "ws_test_check_padding")
    return int(n.value)


def ws_launch_count(ws: Handle) -> int:
    return int(load_library().ws_launch_count(ws.ptr))
