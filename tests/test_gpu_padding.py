"""Memory-safety checks without a sanitizer: NaN canaries in the row padding.

A padded field is the interior, the 4-cell zero halo (the zero-Dirichlet
boundary) and, in x, row padding beyond the halo. ws_test_fill_padding puts a
quiet NaN into every padding cell of every field buffer of a handle (state and
model, 16-bit ones included). Each kernel path then runs on a grid ragged in
x, y and z, with tiles that reach past the grid's edge, sources and receivers
at the edges:
  - the results (field, previous field, traces) must equal, bit for bit, those
    of the same run without canaries: no value beyond the halo reaches a
    result (a NaN would poison it);
  - ws_test_check_padding must find every halo cell still 0 and every padding
    cell still the NaN: no kernel writes outside the interior.
"""

import numpy as np
import pytest

import paper_2204_03775_gb300 as wsb
from paper_2204_03775_gb300 import synthetic

pytestmark = pytest.mark.gpu

NX, NY, NZ, NT = 99, 37, 21, 25


@pytest.fixture(scope="module", autouse=True)
def _library():
    wsb.load_library(build_if_missing=True)


def _handle(storage, kernel, tile, vel, dt):
    h = wsb.ws_create(NX, NY, NZ, 10.0, dt)
    wsb.ws_set_storage(h, storage)
    wsb.ws_set_velocity(h, vel)
    wsb.ws_set_sponge(h, 4, 0.1)
    wsb.ws_set_kernel(h, kernel, *tile, 0)
    wsb.ws_add_source(h, NX - 1, NY // 2, NZ // 2, 25.0, 0.02, 1.0)
    wsb.ws_add_source(h, 2, NY - 1, 0, 18.0, 0.03, 0.5)
    rec = np.array([[0, 0, 0], [NX - 1, NY - 1, NZ - 1], [NX - 2, 1, NZ // 2], [50, NY - 1, 3]],
                   np.int32)
    wsb.ws_set_receivers(h, rec, NT)
    return h


def _result(h):
    u, up = wsb.ws_read_field(h)
    return u, up, wsb.ws_read_traces(h)


CASES = [
    (wsb.WS_STORAGE_FP32, wsb.WS_KERNEL_STREAM, (64, 8)),
    (wsb.WS_STORAGE_FP32, wsb.WS_KERNEL_STREAM, (32, 16)),
    (wsb.WS_STORAGE_FP32, wsb.WS_KERNEL_DIRECT, (0, 0)),
    (wsb.WS_STORAGE_FP16, wsb.WS_KERNEL_STREAM, (0, 0)),
    (wsb.WS_STORAGE_BF16, wsb.WS_KERNEL_STREAM, (0, 0)),
    (wsb.WS_STORAGE_FP16, wsb.WS_KERNEL_STREAM, (64, 16)),
]


@pytest.mark.parametrize("storage,kernel,tile", CASES)
def test_padding_is_neither_read_nor_written(storage, kernel, tile):
    vel = synthetic.smooth_random_velocity((NZ, NY, NX), 21, spacing=4)
    dt = synthetic.cfl_dt(4500.0, 10.0)
    plain = _handle(storage, kernel, tile, vel, dt)
    wsb.ws_step(plain, NT)
    ref = _result(plain)
    h = _handle(storage, kernel, tile, vel, dt)
    assert wsb.ws_test_check_padding(h) > 0       # the padding exists and holds no canary yet
    wsb.ws_test_fill_padding(h)
    assert wsb.ws_test_check_padding(h) == 0
    wsb.ws_step(h, NT)
    got = _result(h)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    assert np.isfinite(got[0]).all() and np.abs(got[0]).max() > 0
    assert wsb.ws_test_check_padding(h) == 0
    # the check sees writes there: ws_write_field rewrites whole buffers
    wsb.ws_write_field(h, None, None, 0)
    assert wsb.ws_test_check_padding(h) > 0


def test_batch_with_padding_canaries():
    vel = synthetic.smooth_random_velocity((NZ, NY, NX), 22, spacing=4)
    dt = synthetic.cfl_dt(4500.0, 10.0)
    other = synthetic.smooth_random_velocity((30, 40, 72), 23, spacing=4)

    def pair():
        a = _handle(wsb.WS_STORAGE_FP32, wsb.WS_KERNEL_STREAM, (64, 8), vel, dt)
        b = wsb.ws_create(72, 40, 30, 10.0, dt)
        wsb.ws_set_velocity(b, other)
        wsb.ws_add_source(b, 71, 0, 29, 20.0, 0.02, 1.0)
        wsb.ws_set_receivers(b, np.array([[71, 39, 29], [0, 0, 0]], np.int32), NT)
        return [a, b]

    ref = pair()
    for h in ref:
        wsb.ws_step(h, NT)
    hs = pair()
    for h in hs:
        wsb.ws_test_fill_padding(h)
    b = wsb.ws_batch_create(hs)
    wsb.ws_batch_set_tiling(b, 32, 16, 0)
    wsb.ws_batch_step(b, NT)
    wsb.ws_batch_synchronize(b)
    for h, r in zip(hs, ref):
        for x, y in zip(_result(h), _result(r)):
            np.testing.assert_array_equal(x, y)
        assert wsb.ws_test_check_padding(h) == 0
    wsb.ws_batch_destroy(b)


def test_adjoint_with_padding_canaries():
    """The gradient (forward with checkpoints, recomputation, adjoint steps,
    imaging) from a handle whose state and model carry padding canaries. The
    gradient restarts the state from rest, re-zeroing both state buffers
    whole (as ws_write_field does), so afterwards exactly those two buffers'
    padding differs from the canaries and the model's canaries must be
    intact; the gradient must be bit for bit the one without canaries."""
    vel = synthetic.smooth_random_velocity((NZ, NY, NX), 24, 2000.0, 3200.0, spacing=4)
    dt = synthetic.cfl_dt(float(vel.max()), 10.0)
    resid = np.random.default_rng(24).standard_normal((4, NT)).astype(np.float32)
    plain = _handle(wsb.WS_STORAGE_FP32, wsb.WS_KERNEL_STREAM, (64, 8), vel, dt)
    g_plain, _ = wsb.ws_adjoint_gradient(plain, resid, wsb.WS_ADJ_RESIDUAL)

    rezeroed = _handle(wsb.WS_STORAGE_FP32, wsb.WS_KERNEL_STREAM, (64, 8), vel, dt)
    wsb.ws_test_fill_padding(rezeroed)
    wsb.ws_write_field(rezeroed, None, None, 0)
    expected = wsb.ws_test_check_padding(rezeroed)
    assert expected > 0

    h = _handle(wsb.WS_STORAGE_FP32, wsb.WS_KERNEL_STREAM, (64, 8), vel, dt)
    wsb.ws_test_fill_padding(h)
    g, _ = wsb.ws_adjoint_gradient(h, resid, wsb.WS_ADJ_RESIDUAL)
    assert wsb.ws_test_check_padding(h) == expected
    np.testing.assert_array_equal(g, g_plain)
    assert np.isfinite(g).all() and np.abs(g).max() > 0
