"""Batched shots (ws_batch_*) and the tiling autotuner (ws_autotune).

A batch advances shots on grids of different sizes with one persistent
launch per step. Every tiling computes the same FP32 expression per cell, so
a batch must reproduce, bit for bit, each shot stepped on its own with
ws_step (which the parity tests pin to the FP64 oracle); one shot is also
checked against the oracle directly. Covered: online tuning inside the run,
a fixed tiling, runs split at odd step counts (the leapfrog parity), shots
that join at different steps, 32-wide-only grids, receivers and sources in
every shot, and the tuner leaving the state untouched.
"""

import numpy as np
import pytest

import oracle
import paper_2204_03775_gb300 as wsb
from paper_2204_03775_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    wsb.load_library(build_if_missing=True)


SHAPES = [(72, 40, 30), (150, 44, 36), (96, 64, 50), (64, 16, 70), (130, 9, 12)]


def _shot(shape, seed, nt):
    nx, ny, nz = shape
    vel = synthetic.smooth_random_velocity((nz, ny, nx), seed, spacing=5)
    h = 10.0
    dt = synthetic.cfl_dt(4500.0, h)
    rng = np.random.default_rng(seed)
    src = [(int(rng.integers(0, nx)), int(rng.integers(0, ny)), int(rng.integers(0, nz)),
            float(rng.uniform(12, 30)), 0.04, float(rng.uniform(0.5, 2)))]
    cells = rng.choice(nx * ny * nz, 9, replace=False)
    rec = np.stack([cells % nx, cells // nx % ny, cells // (nx * ny)], axis=1).astype(np.int32)
    return dict(vel=vel, h=h, dt=dt, src=src, rec=rec, sponge=(4, 0.1), nt=nt)


def _handle(s, kernel=wsb.WS_KERNEL_AUTO):
    nz, ny, nx = s["vel"].shape
    hd = wsb.ws_create(nx, ny, nz, s["h"], s["dt"])
    wsb.ws_set_velocity(hd, s["vel"])
    wsb.ws_set_sponge(hd, *s["sponge"])
    wsb.ws_set_kernel(hd, kernel)
    for q in s["src"]:
        wsb.ws_add_source(hd, *q)
    wsb.ws_set_receivers(hd, s["rec"], s["nt"])
    return hd


def _state(hd):
    u, up = wsb.ws_read_field(hd)
    return u, up, wsb.ws_read_traces(hd), wsb.ws_get_step(hd)


def _check_equal(a, b):
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_array_equal(x, y)
    assert a[3] == b[3]


@pytest.mark.parametrize("fixed", [None, (64, 8, 2), (32, 16, 0), (32, 8, 8)])
def test_batch_equals_single_shots(fixed):
    nt = 61
    shots = [_shot(sh, 40 + q, nt) for q, sh in enumerate(SHAPES)]
    if fixed is not None:   # only the shots the fixed tile fits
        shots = [s for s in shots if s["vel"].shape[2] >= fixed[0] and s["vel"].shape[1] >= fixed[1]]
    ref = []
    for s in shots:
        hd = _handle(s)
        wsb.ws_step(hd, nt)
        ref.append(_state(hd))
    hs = [_handle(s) for s in shots]
    # one shot joins two steps late: it is stepped on its own first
    wsb.ws_step(hs[1], 2)
    b = wsb.ws_batch_create(hs[:1] + hs[2:])
    if fixed is not None:
        wsb.ws_batch_set_tiling(b, *fixed)
    wsb.ws_batch_step(b, 2)
    b2 = wsb.ws_batch_create(hs)
    if fixed is not None:
        wsb.ws_batch_set_tiling(b2, *fixed)
    for n in (7, 1, 30, 21):                  # odd run lengths flip the leapfrog parity
        wsb.ws_batch_step(b2, n)
    wsb.ws_batch_synchronize(b2)
    assert wsb.ws_batch_launch_count(b2) == nt - 2
    for hd, r in zip(hs, ref):
        _check_equal(_state(hd), r)
    tile = wsb.ws_batch_get_tiling(b2)
    if fixed is not None:
        assert tile == fixed
    else:
        assert wsb.ws_get_step(hs[0]) == nt and tile[0] in (32, 64)


def test_batch_shot_matches_oracle():
    nt = 80
    s = _shot((96, 64, 50), 7, nt)
    other = _shot((72, 40, 30), 8, nt)
    hs = [_handle(s), _handle(other)]
    b = wsb.ws_batch_create(hs)
    wsb.ws_batch_step(b, nt)
    u, _, tr, _ = _state(hs[0])
    ref = oracle.run(s["vel"].astype(np.float64), s["h"], s["dt"], nt, sources=s["src"],
                     receivers=s["rec"], sponge=s["sponge"])
    err = np.linalg.norm(u - ref["u"]) / np.linalg.norm(ref["u"])
    assert err <= 1e-4, err
    assert np.abs(tr - ref["traces"]).max() <= 1e-4 * np.abs(ref["traces"]).max()


def test_autotune_keeps_state_and_results():
    nt = 40
    s = _shot((150, 44, 36), 3, nt)
    a = _handle(s)
    wsb.ws_step(a, 5)
    before = _state(a)
    tx, ty, zb = wsb.ws_autotune(a)
    assert (tx, ty) in [(64, 8), (32, 8), (32, 16), (64, 16), (64, 32)]
    assert 1 <= zb <= 36
    _check_equal(_state(a), before)
    wsb.ws_step(a, nt - 5)
    ref = _handle(s)
    wsb.ws_step(ref, nt)
    _check_equal(_state(a), _state(ref))
    # cached per grid size: a second handle gets the same answer
    assert wsb.ws_autotune(_handle(s)) == (tx, ty, zb)


def test_autotune_cache_persists_across_processes(tmp_path):
    """The tuned tiling is written to the cache file ($WS_TUNE_CACHE) keyed by
    GPU name, storage and grid size; a new process tuning the same grid finds
    it there and times nothing (no kernel launches)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = tmp_path / "tune.txt"
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import numpy as np\n"
        "import paper_2204_03775_gb300 as wsb\n"
        "wsb.load_library(build_if_missing=True)\n"
        "h = wsb.ws_create(130, 40, 30, 10.0, 1e-3)\n"
        "wsb.ws_set_velocity(h, np.full((30, 40, 130), 2000.0, np.float32))\n"
        "n0 = wsb.ws_launch_count(h)\n"
        "t = wsb.ws_autotune(h)\n"
        "print(*t, wsb.ws_launch_count(h) - n0)\n" % root)
    env = dict(os.environ, WS_TUNE_CACHE=str(path))
    runs = [subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=300) for _ in range(2)]
    for r in runs:
        assert r.returncode == 0, r.stderr
    first, second = (list(map(int, r.stdout.split())) for r in runs)
    assert first[3] > 0 and second[3] == 0, (first, second)
    assert first[:3] == second[:3]
    lines = path.read_text().splitlines()
    assert len(lines) == 1
    gpu, storage, nx, ny, nz, tx, ty, zb = lines[0].split("|")
    assert gpu and (int(storage), int(nx), int(ny), int(nz)) == (wsb.WS_STORAGE_FP32, 130, 40, 30)
    assert [int(tx), int(ty), int(zb)] == first[:3]


def test_batch_errors():
    s = _shot((72, 40, 30), 1, 10)
    h = _handle(s)
    with pytest.raises(wsb.WaveStepError):
        wsb.ws_batch_create([h, h])
    small = wsb.ws_create(16, 16, 16, 10.0, 1e-3)
    with pytest.raises(wsb.WaveStepError):
        wsb.ws_batch_create([small])
    b = wsb.ws_batch_create([h])
    with pytest.raises(wsb.WaveStepError) as e:       # receivers hold 10 steps
        wsb.ws_batch_step(b, 11)
    assert e.value.code == wsb.WS_ERR_STATE
    with pytest.raises(wsb.WaveStepError):
        wsb.ws_batch_set_tiling(b, 48, 8, 0)
    h16 = _handle(_shot((72, 40, 30), 2, 10))                # batches need FP32 storage
    wsb.ws_set_storage(h16, wsb.WS_STORAGE_FP16)
    b16 = wsb.ws_batch_create([h16])
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_batch_step(b16, 1)
    assert e.value.code == wsb.WS_ERR_STATE


def test_full_size_batch_equals_single_shots():
    """The benchmark's batch (64 shots, 96^3 .. 320x320x256, 500 steps, online
    tuning, CUDA graph) against each shot stepped alone: every trace, and the
    final fields of four shots, bit for bit."""
    shots = synthetic.batched_shots()
    nt = shots[0].nt
    hs = []
    for w in shots:
        s = dict(vel=w.vel, h=w.h, dt=w.dt, src=w.sources, rec=w.receivers, sponge=w.sponge, nt=nt)
        hs.append(_handle(s))
    b = wsb.ws_batch_create(hs)
    wsb.ws_batch_step(b, nt)
    wsb.ws_batch_synchronize(b)
    assert wsb.ws_batch_launch_count(b) == nt
    probe = [0, 17, 40, 63]
    got_tr = [wsb.ws_read_traces(h) for h in hs]
    got_u = {q: wsb.ws_read_field(hs[q])[0] for q in probe}
    for q, (h, w) in enumerate(zip(hs, shots)):
        wsb.ws_write_field(h, None, None, 0)
        wsb.ws_set_receivers(h, w.receivers, nt)
        wsb.ws_step(h, nt)
        np.testing.assert_array_equal(wsb.ws_read_traces(h), got_tr[q])
        if q in got_u:
            np.testing.assert_array_equal(wsb.ws_read_field(h)[0], got_u[q])


def test_shots_used_alone_between_batch_steps():
    """A shot stepped on its own with another tile and with new receivers
    between batch steps: the batch re-encodes its maps and receiver table."""
    nt = 30
    shots = [_shot(sh, 60 + q, nt) for q, sh in enumerate(SHAPES[:3])]
    ref = []
    for s in shots:
        hd = _handle(s)
        wsb.ws_step(hd, nt)
        ref.append(_state(hd))
    hs = [_handle(s) for s in shots]
    b = wsb.ws_batch_create(hs)
    wsb.ws_batch_set_tiling(b, 64, 8, 2)
    wsb.ws_batch_step(b, 10)
    wsb.ws_set_kernel(hs[0], wsb.WS_KERNEL_STREAM, 32, 16, 0)   # another tile
    wsb.ws_step(hs[0], 5)
    wsb.ws_batch_step(b, 5)        # hs[0] at 20 steps, the others at 15
    wsb.ws_step(hs[1], 5)
    wsb.ws_step(hs[2], 5)
    wsb.ws_batch_step(b, 10)       # every shot at nt = 30
    wsb.ws_batch_synchronize(b)
    for hd, r in zip(hs, ref):     # tiles never change the bits
        _check_equal(_state(hd), r)


def test_binding_keeps_batched_handles_alive():
    s = _shot((72, 40, 30), 2, 10)
    h = _handle(s)
    b = wsb.ws_batch_create([h])
    with pytest.raises(wsb.WaveStepError):
        wsb.ws_destroy(h)                 # the batch still uses it
    wsb.ws_batch_destroy(b)
    wsb.ws_destroy(h)
