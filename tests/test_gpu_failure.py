"""Failure detection on the GPU without a GPU fault.

ws_test_stall makes the next streaming step withhold one TMA copy, so the
bounded waits of one CTA run out (about one second): the kernel records a
timeout in the handle's status word, every warp of that CTA leaves its
loops, the CTA drains its own copies in flight, and the launch ends.
ws_synchronize must report WS_ERR_TIMEOUT once, the CUDA context must stay
usable, and after a fresh state the handle must step exactly as a new one.
All three streaming kernels: the FP32 one (warps leave together by a warp
vote), the 16-bit one (its consumer warps meet at a named barrier every
plane, which also ANDs their wait flags, so all of them leave at the same
plane) and the batched one (the FP32 body over a table of shots).
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


def test_batch_stall_is_reported_and_recoverable():
    """The same hook in a batch: the first launch of the run withholds one
    copy of one shot's item; the batch reports the timeout once, and after
    fresh states every shot steps exactly like a shot stepped alone."""
    wsb.load_library(build_if_missing=True)
    ws = [synthetic.layered_survey(128, 64, 48, nt=20), synthetic.layered_survey(96, 40, 30, nt=20)]
    hs = [_handle(w) for w in ws]
    b = wsb.ws_batch_create(hs)
    wsb.ws_batch_set_tiling(b, 32, 16, 0)
    wsb.ws_batch_step(b, 2)
    wsb.ws_batch_synchronize(b)
    wsb.ws_test_stall(hs[1], 3)
    t0 = time.perf_counter()
    wsb.ws_batch_step(b, 3)
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_batch_synchronize(b)
    took = time.perf_counter() - t0
    assert e.value.code == wsb.WS_ERR_TIMEOUT
    assert 0.5 < took < 30.0, took
    wsb.ws_batch_synchronize(b)                 # reported once, then cleared
    for h in hs:
        wsb.ws_write_field(h, None, None, 0)
    wsb.ws_batch_step(b, 20)
    wsb.ws_batch_synchronize(b)
    for h, w in zip(hs, ws):
        ref = _handle(w)
        wsb.ws_step(ref, 20)
        np.testing.assert_array_equal(wsb.ws_read_field(h)[0], wsb.ws_read_field(ref)[0])
        np.testing.assert_array_equal(wsb.ws_read_field(h)[1], wsb.ws_read_field(ref)[1])
    wsb.ws_batch_destroy(b)


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
