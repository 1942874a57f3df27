"""Failure detection on the GPU without a GPU fault.

ws_test_stall makes the next streaming step withhold one TMA copy, so the
bounded waits of one CTA run out (about one second): the kernel records a
timeout in the handle's status word, every warp of that CTA leaves its
loops, the CTA drains its own copies in flight, and the launch ends.
ws_synchronize must report WS_ERR_TIMEOUT once, the CUDA context must stay
usable, and after a fresh state the handle must step exactly as a new one.
Both streaming kernels: the FP32 one (warps leave together by a warp vote)
and the 16-bit one (its consumer warps meet at a named barrier every plane,
which also ANDs their wait flags, so all of them leave at the same plane).
"""

import time

import numpy as np
import pytest

import paper_2204_03775_gb300 as wsb
from paper_2204_03775_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _handle(w, storage=wsb.WS_STORAGE_FP32):
    h = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
    wsb.ws_set_storage(h, storage)
    wsb.ws_set_velocity(h, w.vel)
    wsb.ws_set_sponge(h, *w.sponge)
    for s in w.sources:
        wsb.ws_add_source(h, *s)
    wsb.ws_set_kernel(h, wsb.WS_KERNEL_STREAM, 64, 8, 0)
    return h


@pytest.mark.parametrize("storage", [wsb.WS_STORAGE_FP32, wsb.WS_STORAGE_FP16])
def test_bounded_wait_timeout_is_reported_and_recoverable(storage):
    wsb.load_library(build_if_missing=True)
    w = synthetic.layered_survey(128, 64, 48, nt=20)
    h = _handle(w, storage)
    wsb.ws_step(h, 3)
    wsb.ws_synchronize(h)
    wsb.ws_test_stall(h, 5)
    t0 = time.perf_counter()
    wsb.ws_step(h, 1)
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_synchronize(h)
    took = time.perf_counter() - t0
    assert e.value.code == wsb.WS_ERR_TIMEOUT
    assert 0.5 < took < 30.0, took
    wsb.ws_synchronize(h)                       # reported once, then cleared
    # the context is usable: restart from rest and compare with a new handle
    wsb.ws_write_field(h, None, None, 0)
    wsb.ws_step(h, 20)
    wsb.ws_synchronize(h)
    ref = _handle(w, storage)
    wsb.ws_step(ref, 20)
    u, up = wsb.ws_read_field(h)
    ur, upr = wsb.ws_read_field(ref)
    np.testing.assert_array_equal(u, ur)
    np.testing.assert_array_equal(up, upr)
    assert np.abs(u).max() > 0


def test_stall_hook_arguments():
    wsb.load_library(build_if_missing=True)
    h = wsb.ws_create(64, 8, 8, 10.0, 1e-3)
    with pytest.raises(wsb.WaveStepError):
        wsb.ws_test_stall(h, -2)
    wsb.ws_test_stall(h, 3)
    wsb.ws_test_stall(h, -1)                    # cleared: the next step runs normally
    wsb.ws_set_velocity(h, np.full((8, 8, 64), 2000.0, np.float32))
    wsb.ws_step(h, 2)
    wsb.ws_synchronize(h)
