"""ws_energy_noalloc, the entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc -- an allocator policy forbids it, or
they cannot afford the device-wide synchronization it may cause -- so
ws_energy_noalloc takes device arrays the caller owns and keeps its partial
sums in a static device array of the library. It must give exactly what
ws_energy gives for the same state (same terms, same summation order), call
after call, although every call reuses (and leaves behind) the same scratch.
This file is collected last so that a run that stops at the first failure
has run every other test first; it passes both alone in a fresh process and
after the other tests.
"""

import ctypes

import numpy as np
import pytest

import paper_2204_03775_gb300 as wsb
from paper_2204_03775_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _energy_of_handle_state(torch, nx, ny, nz, vel, u, p, h, dt):
    """ws_energy of a handle holding the state (u, p) on the model vel."""
    hd = wsb.ws_create(nx, ny, nz, h, dt)
    wsb.ws_set_velocity(hd, vel)
    wsb.ws_write_field(hd, u, p, 0)
    e = wsb.ws_energy(hd)
    wsb.ws_destroy(hd)
    return e


def test_energy_noalloc_matches_ws_energy_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    wsb.load_library(build_if_missing=True)
    nx, ny, nz = 101, 70, 45
    vel = synthetic.layered_model(nx, ny, nz, seed=5)
    h = 10.0
    dt = synthetic.cfl_dt(vel.max(), h)
    hd = wsb.ws_create(nx, ny, nz, h, dt)
    wsb.ws_set_velocity(hd, vel)
    wsb.ws_add_source(hd, 40, 30, 20, 25.0, 0.03, 1.0)
    v_dev = torch.from_numpy(vel).cuda()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")

    for steps in (60, 25):   # two calls in a row, on two different states
        wsb.ws_step(hd, steps)
        e_ref = wsb.ws_energy(hd)
        u, p = wsb.ws_read_field(hd)
        u_dev = torch.from_numpy(u).cuda()
        p_dev = torch.from_numpy(p).cuda()
        torch.cuda.synchronize()
        wsb.ws_energy_noalloc(u_dev, p_dev, v_dev, h, dt, out)
        torch.cuda.synchronize()
        e = float(out.item())
        assert e_ref != 0.0
        assert e == e_ref, (e, e_ref)   # same terms, same order: bit for bit
    wsb.ws_destroy(hd)


def test_energy_noalloc_fills_the_whole_scratch():
    """ceil(32 / 32) * 32768 = 32768 partial sums: the last slot is used."""
    torch = pytest.importorskip("torch")
    wsb.load_library(build_if_missing=True)
    nx, ny, nz = 8, 32, 32768
    rng = np.random.default_rng(11)
    vel = rng.uniform(1500.0, 4500.0, (nz, ny, nx)).astype(np.float32)
    h = 10.0
    dt = synthetic.cfl_dt(float(vel.max()), h)
    u = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    p = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    # the deepest plane alone carries a large value, so a dropped last partial shows
    u[-1] *= 1e3
    e_ref = _energy_of_handle_state(torch, nx, ny, nz, vel, u, p, h, dt)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    wsb.ws_energy_noalloc(torch.from_numpy(u).cuda(), torch.from_numpy(p).cuda(),
                          torch.from_numpy(vel).cuda(), h, dt, out)
    torch.cuda.synchronize()
    assert float(out.item()) == e_ref


def test_energy_noalloc_on_a_non_default_stream():
    """The binding issues on torch's current stream: the producer of the
    inputs and the reader of out are ordered with the call without any
    explicit synchronization."""
    torch = pytest.importorskip("torch")
    wsb.load_library(build_if_missing=True)
    nx, ny, nz = 96, 64, 40
    vel = synthetic.smooth_random_velocity((nz, ny, nx), seed=21)
    h = 10.0
    dt = synthetic.cfl_dt(float(vel.max()), h)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    p = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    e_ref = _energy_of_handle_state(torch, nx, ny, nz, vel, u, p, h, dt)
    u_host = torch.from_numpy(u).pin_memory()
    p_host = torch.from_numpy(p).pin_memory()
    v_host = torch.from_numpy(vel).pin_memory()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        # long work ahead of the copies, so that an unordered call would read garbage
        big = torch.randn((4096, 4096), device="cuda")
        for _ in range(4):
            big = big @ big
            big /= big.abs().max()
        u_dev = torch.empty_like(u_host, device="cuda")
        p_dev = torch.empty_like(p_host, device="cuda")
        v_dev = torch.empty_like(v_host, device="cuda")
        u_dev.copy_(u_host, non_blocking=True)
        p_dev.copy_(p_host, non_blocking=True)
        v_dev.copy_(v_host, non_blocking=True)
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        wsb.ws_energy_noalloc(u_dev, p_dev, v_dev, h, dt, out)
        res = out.to("cpu", non_blocking=False)
    assert float(res.item()) == e_ref


def test_energy_noalloc_rejects_mixed_devices_on_the_host():
    torch = pytest.importorskip("torch")
    wsb.load_library(build_if_missing=True)
    u = torch.zeros((4, 4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(TypeError):   # out in host memory
        wsb.ws_energy_noalloc(u, u, u, 10.0, 1e-3, torch.zeros(1, dtype=torch.float64))
    if torch.cuda.device_count() < 2:
        pytest.skip("one CUDA device: a second device's tensor cannot be made")
    out1 = torch.zeros((1,), dtype=torch.float64, device="cuda:1")
    with pytest.raises(TypeError):
        wsb.ws_energy_noalloc(u, u, u, 10.0, 1e-3, out1)


def test_energy_noalloc_rejects_a_grid_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    wsb.load_library(build_if_missing=True)
    # ceil(64 / 32) * 16385 = 32770 partial sums > WS_NOALLOC_MAX_PARTIALS = 32768;
    # the sizes are checked before any array is touched, so 1-element tensors do
    u = torch.zeros((1, 1, 1), dtype=torch.float32, device="cuda")
    out = torch.zeros((1,), dtype=torch.float64, device="cuda")
    lib = wsb.load_library()
    rc = lib.ws_energy_noalloc(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                               ctypes.c_void_p(u.data_ptr()), 8, 64, 16385, 10.0, 1e-3,
                               ctypes.c_void_p(out.data_ptr()), None)
    assert rc == wsb.WS_ERR_BADARG
    assert "partial sums" in wsb.ws_last_error()
