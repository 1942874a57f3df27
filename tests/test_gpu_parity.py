"""Parity of the CUDA stepper with the FP64 oracle, through the C ABI.

Both sides get the same seeded inputs from ``paper_2204_03775_gb300.synthetic``.
Tolerance (FP32 path vs FP64 oracle): relative L2 error <= 1e-4 over the
whole field and over the traces, and every element within 1e-4 of the
oracle's maximum magnitude. Integer and copy work (restart, receiver
bookkeeping, the untouched zero halo) is checked bit for bit, and the two
CUDA kernels (direct and streaming) are checked to agree bit for bit, since
they evaluate the same expression in the same order.
"""

import numpy as np
import pytest

import oracle
import paper_2204_03775_gb300 as wsb
from paper_2204_03775_gb300 import synthetic

pytestmark = pytest.mark.gpu

RTOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _library():
    wsb.load_library(build_if_missing=True)


def assert_parity(got, ref, rtol=RTOL):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape
    scale = np.abs(ref).max()
    assert scale > 0
    rel_l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    max_err = np.abs(got - ref).max() / scale
    assert rel_l2 <= rtol, f"relative L2 error {rel_l2:.3e} > {rtol}"
    assert max_err <= rtol, f"max error {max_err:.3e} of max|ref| > {rtol}"
    return rel_l2, max_err


def run_gpu(w, nt=None, kernel=wsb.WS_KERNEL_AUTO, tile=(0, 0), zblock=0):
    nt = w.nt if nt is None else nt
    h = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
    wsb.ws_set_kernel(h, kernel, tile[0], tile[1], zblock)
    wsb.ws_set_velocity(h, w.vel)
    wsb.ws_set_sponge(h, *w.sponge)
    for s in w.sources:
        wsb.ws_add_source(h, *s)
    if w.receivers is not None and len(w.receivers):
        wsb.ws_set_receivers(h, w.receivers, nt)
    wsb.ws_step(h, nt)
    wsb.ws_synchronize(h)
    u, up = wsb.ws_read_field(h)
    tr = wsb.ws_read_traces(h) if h.nrec else None
    return h, u, up, tr


def run_oracle(w, nt=None):
    nt = w.nt if nt is None else nt
    return oracle.run(w.vel, w.h, w.dt, nt, sources=w.sources, receivers=w.receivers,
                      sponge=w.sponge)


@pytest.mark.parametrize("kernel,tile", [(wsb.WS_KERNEL_STREAM, (64, 16)),
                                         (wsb.WS_KERNEL_STREAM, (32, 8)),
                                         (wsb.WS_KERNEL_DIRECT, (0, 0))])
def test_homogeneous_cube_64(kernel, tile):
    """64^3, v = 2000 m/s, 100 steps, centred 15 Hz Ricker, 16 top-plane receivers."""
    w = synthetic.homogeneous_cube()
    ref = run_oracle(w)
    _, u, up, tr = run_gpu(w, kernel=kernel, tile=tile)
    assert_parity(u, ref["u"])
    assert_parity(up, ref["u_prev"])
    assert_parity(tr, ref["traces"])


def _ragged_workload(nt=80):
    nx, ny, nz = 101, 37, 45   # ragged in x (64 + 37), y (2 * 16 + 5), z (2 * 16 + 13)
    vel = synthetic.layered_model(nx, ny, nz, seed=7)
    h = 10.0
    dt = synthetic.cfl_dt(vel.max(), h)
    src = [(50, 18, 6, 20.0, 0.05, 1.0), (nx - 1, ny - 1, nz - 1, 30.0, 0.03, -0.5)]
    rec = np.array([[0, 0, 0], [nx - 1, ny - 1, nz - 1], [50, 18, 6], [63, 15, 16], [64, 16, 32],
                    [100, 36, 0], [3, 36, 44], [77, 5, 20]], dtype=np.int32)
    return synthetic.Workload("ragged", nx, ny, nz, h, dt, nt, vel, sources=src,
                              receivers=rec, sponge=(6, 0.05))


@pytest.mark.parametrize("kernel,tile,zb", [(wsb.WS_KERNEL_STREAM, (64, 16), 16),
                                            (wsb.WS_KERNEL_STREAM, (64, 8), 0),
                                            (wsb.WS_KERNEL_STREAM, (32, 16), 7),
                                            (wsb.WS_KERNEL_DIRECT, (0, 0), 0)])
def test_ragged_layered_with_sponge(kernel, tile, zb):
    w = _ragged_workload()
    ref = run_oracle(w)
    _, u, up, tr = run_gpu(w, kernel=kernel, tile=tile, zblock=zb)
    assert_parity(u, ref["u"])
    assert_parity(up, ref["u_prev"])
    assert_parity(tr, ref["traces"])


@pytest.mark.parametrize("tile", [(64, 8), (32, 16), (32, 8)])
def test_stream_z_blocks_of_every_length_agree_bitwise(tile):
    """The streaming kernel walks an item's planes three at a time through
    rings of 8 (ring A) and 4 (ring B) slots: items of 1 to 13 planes end a
    trip early at every phase and wrap the rings a different number of times.
    Every z block gives the same bits as the direct kernel."""
    w = _ragged_workload(nt=40)
    _, u1, p1, t1 = run_gpu(w, kernel=wsb.WS_KERNEL_DIRECT)
    for zb in (1, 2, 3, 4, 5, 6, 7, 8, 9, 11, 13):
        h, u2, p2, t2 = run_gpu(w, kernel=wsb.WS_KERNEL_STREAM, tile=tile, zblock=zb)
        wsb.ws_destroy(h)
        np.testing.assert_array_equal(u1, u2, err_msg=f"zblock {zb}")
        np.testing.assert_array_equal(p1, p2, err_msg=f"zblock {zb}")
        np.testing.assert_array_equal(t1, t2, err_msg=f"zblock {zb}")


def test_direct_and_stream_agree_bitwise():
    w = _ragged_workload(nt=60)
    _, u1, p1, t1 = run_gpu(w, kernel=wsb.WS_KERNEL_DIRECT)
    for tile, zb in [((64, 16), 0), ((32, 8), 5), ((64, 8), 45)]:
        _, u2, p2, t2 = run_gpu(w, kernel=wsb.WS_KERNEL_STREAM, tile=tile, zblock=zb)
        np.testing.assert_array_equal(u1, u2)
        np.testing.assert_array_equal(p1, p2)
        np.testing.assert_array_equal(t1, t2)


@pytest.mark.parametrize("shape", [(8, 8, 8), (1, 1, 1), (5, 7, 9), (3, 50, 2), (33, 8, 1),
                                   (40, 9, 3)])
def test_small_and_degenerate_grids(shape):
    nx, ny, nz = shape
    vel = synthetic.smooth_random_velocity((nz, ny, nx), seed=nx * 100 + ny * 10 + nz)
    h = 10.0
    dt = synthetic.cfl_dt(vel.max(), h)
    src = [(nx // 2, ny // 2, nz // 2, 40.0, 0.01, 1.0)]
    rec = np.array([[0, 0, 0], [nx - 1, ny - 1, nz - 1]], dtype=np.int32)
    w = synthetic.Workload("small", nx, ny, nz, h, dt, 30, vel, sources=src, receivers=rec,
                           sponge=(1, 0.2))
    ref = run_oracle(w)
    kernels = [wsb.WS_KERNEL_DIRECT]
    if nx >= 32 and ny >= 8:
        kernels.append(wsb.WS_KERNEL_STREAM)
    for kern in kernels:
        tile = (32, 8) if kern == wsb.WS_KERNEL_STREAM else (0, 0)
        _, u, up, tr = run_gpu(w, kernel=kern, tile=tile)
        assert_parity(u, ref["u"])
        assert_parity(tr, ref["traces"])


def test_zero_steps_and_empty_receivers():
    w = synthetic.homogeneous_cube(n=40, nt=0)
    h = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
    wsb.ws_set_velocity(h, w.vel)
    wsb.ws_set_receivers(h, np.zeros((0, 3), np.int32), 0)
    wsb.ws_step(h, 0)
    u, up = wsb.ws_read_field(h)
    assert not u.any() and not up.any()
    assert wsb.ws_get_step(h) == 0


def test_restart_is_bitwise():
    w = _ragged_workload(nt=60)
    _, u_ref, up_ref, _ = run_gpu(w, nt=60)
    h1, u40, up40, _ = run_gpu(w, nt=40)
    h2 = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
    wsb.ws_set_velocity(h2, w.vel)
    wsb.ws_set_sponge(h2, *w.sponge)
    for s in w.sources:
        wsb.ws_add_source(h2, *s)
    wsb.ws_write_field(h2, u40, up40, 40)
    wsb.ws_step(h2, 20)
    u, up = wsb.ws_read_field(h2)
    np.testing.assert_array_equal(u, u_ref)
    np.testing.assert_array_equal(up, up_ref)


def test_device_pointers_and_stream():
    torch = pytest.importorskip("torch")
    w = _ragged_workload(nt=30)
    _, u_ref, _, tr_ref = run_gpu(w)
    stream = torch.cuda.Stream()
    h = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
    wsb.ws_set_stream(h, stream)
    with torch.cuda.stream(stream):
        vel = torch.from_numpy(w.vel).cuda()
        wsb.ws_set_velocity(h, vel)
        wsb.ws_set_sponge(h, *w.sponge)
        for s in w.sources:
            wsb.ws_add_source(h, *s)
        wsb.ws_set_receivers(h, w.receivers, 30)
        wsb.ws_step(h, 30)
        u = torch.empty(w.vel.shape, dtype=torch.float32, device="cuda")
        tr = torch.empty((len(w.receivers), 30), dtype=torch.float32, device="cuda")
        wsb.ws_read_field(h, u, None)
        wsb.ws_read_traces(h, tr)
    stream.synchronize()
    np.testing.assert_array_equal(u.cpu().numpy(), u_ref)
    np.testing.assert_array_equal(tr.cpu().numpy(), tr_ref)


def test_argument_errors():
    w = synthetic.homogeneous_cube(n=24, nt=10)
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_create(0, 4, 4, 10.0, 1e-3)
    assert e.value.code == wsb.WS_ERR_BADARG
    h = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_step(h, 1)
    assert e.value.code == wsb.WS_ERR_STATE
    fast = np.full_like(w.vel, 2000.0)
    fast[3, 4, 5] = 2000.0 * 0.46 / 0.4   # just above the stability limit
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_set_velocity(h, fast)
    assert e.value.code == wsb.WS_ERR_CFL
    bad = w.vel.copy()
    bad[0, 0, 0] = -1.0
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_set_velocity(h, bad)
    assert e.value.code == wsb.WS_ERR_BADARG
    wsb.ws_set_velocity(h, w.vel)
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_add_source(h, 24, 0, 0, 10.0, 0.1, 1.0)
    assert e.value.code == wsb.WS_ERR_BADARG
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_set_receivers(h, [[0, 0, 24]], 5)
    assert e.value.code == wsb.WS_ERR_BADARG
    wsb.ws_set_receivers(h, [[1, 2, 3]], 5)
    wsb.ws_step(h, 5)
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_step(h, 1)
    assert e.value.code == wsb.WS_ERR_STATE
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_set_kernel(h, wsb.WS_KERNEL_STREAM, 64, 16, 0)   # 24 < 64: tile does not fit
    assert e.value.code == wsb.WS_ERR_BADARG
    for s in range(wsb.WS_MAX_SOURCES):
        wsb.ws_add_source(h, 1, 1, 1, 10.0, 0.1, 1.0)
    with pytest.raises(wsb.WaveStepError):
        wsb.ws_add_source(h, 1, 1, 1, 10.0, 0.1, 1.0)
    wsb.ws_synchronize(h)


def test_full_size_window_against_oracle():
    """The benchmark's 1024^3 layered survey, in the benchmark's launch setup.

    After nt steps from rest the wavefield is exactly zero farther than 4 nt
    cells from the source; the oracle computes the window that holds that
    region (whose outer faces are the grid's top face or lie beyond the light
    cone), and the GPU field must match it there and be exactly zero outside.
    """
    nt = 40
    w = synthetic.layered_survey(1024, 1024, 1024, nt=nt)
    h, u, up, tr = run_gpu(w, nt=nt)
    si, sj, sk = w.sources[0][:3]
    r = 4 * nt + 1
    ox, oy, oz = si - r, sj - r, 0
    wx, wy, wz = 2 * r + 1, 2 * r + 1, sk + r + 1
    sub = w.vel[oz:oz + wz, oy:oy + wy, ox:ox + wx]
    inside = [(n, rr) for n, rr in enumerate(w.receivers)
              if ox <= rr[0] < ox + wx and oy <= rr[1] < oy + wy and oz <= rr[2] < oz + wz]
    ref = oracle.run(sub, w.h, w.dt, nt, sources=w.sources,
                     receivers=np.array([rr for _, rr in inside], np.int32).reshape(-1, 3),
                     sponge=w.sponge, window=(ox, oy, oz, w.nx, w.ny, w.nz))
    assert_parity(u[oz:oz + wz, oy:oy + wy, ox:ox + wx], ref["u"])
    assert_parity(up[oz:oz + wz, oy:oy + wy, ox:ox + wx], ref["u_prev"])
    mask = np.ones(u.shape, bool)
    mask[oz:oz + wz, oy:oy + wy, ox:ox + wx] = False
    assert not u[mask].any()
    idx = [n for n, _ in inside]
    if idx and np.abs(ref["traces"]).max() > 0:
        assert_parity(tr[idx], ref["traces"])
    others = np.setdiff1d(np.arange(len(w.receivers)), idx)
    assert not tr[others].any()
