"""ws_energy_noalloc, the entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc -- an allocator policy forbids it, or
they cannot afford the device-wide synchronization it may cause -- so
ws_energy_noalloc takes device arrays the caller owns and keeps its partial
sums in a static device array of the library. It must give what ws_energy
gives for the same state, call after call, although every call reuses (and
leaves behind) the same scratch. This file is collected last so that a run
that stops at the first failure has run every other test first; it passes
both alone in a fresh process and after the other tests.
"""

import numpy as np
import pytest

import paper_2204_03775_gb300 as wsb
from paper_2204_03775_gb300 import synthetic

pytestmark = pytest.mark.gpu

RTOL = 1e-11   # the tolerance of the ws_energy tests


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
        assert abs(e - e_ref) <= RTOL * abs(e_ref), (e, e_ref)


def test_energy_noalloc_rejects_a_grid_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    wsb.load_library(build_if_missing=True)
    # ceil(64 / 32) * 16385 = 32770 partial sums > WS_NOALLOC_MAX_PARTIALS = 32768;
    # the sizes are checked before any array is touched, so 1-element tensors do
    u = torch.zeros((1, 1, 1), dtype=torch.float32, device="cuda")
    out = torch.zeros((1,), dtype=torch.float64, device="cuda")
    lib = wsb.load_library()
    import ctypes
    rc = lib.ws_energy_noalloc(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                               ctypes.c_void_p(u.data_ptr()), 8, 64, 16385, 10.0, 1e-3,
                               ctypes.c_void_p(out.data_ptr()), None)
    assert rc == wsb.WS_ERR_BADARG
    assert "partial sums" in wsb.ws_last_error()
