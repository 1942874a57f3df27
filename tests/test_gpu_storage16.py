"""16-bit field storage (ws_set_storage): one step against the exact update, stated accuracy.

The 16-bit modes store U = u^n and D = u^n - u^{n-1} (velocity form) and the
model (V dt/h)^2 in FP16.
1. One step: from a state whose u^n and u^n - u^{n-1} are exact in the
   16-bit format, with a model exact in FP16, the kernel computes u~ = u^{n+1}
   and d~ = u^{n+1} - u^n in FP32 and stores their 16-bit roundings. Against
   the FP64 oracle's step from the same state, the stored U' and D' are the
   correctly rounded values (the FP32 arithmetic is ~1e-6 off, far below one
   16-bit unit, so only values within that of a rounding boundary may land
   on the neighbour) and the traces are u~ itself, to FP32 accuracy. The grid
   has tiles inside the taper (the update without taper multiplies) and
   tiles that touch it, ragged edges and a source.
2. Accuracy against the FP64 oracle over many steps: FP32 storage within
   1e-4, FP16 within 1e-2 at every checkpoint up to the configured 1000
   steps; BF16 within 1e-2 where it is claimed (100 steps) -- beyond that its
   8-bit significand does not hold 1e-2 (the rounding errors of the state add
   up like a random walk, ~1.6e-3 sqrt(steps)), and the tests report the
   measured error instead of asserting a bound.
3. Converting FP32 -> 16-bit -> FP32 keeps the state within one 16-bit rounding.
"""

import numpy as np
import pytest

import oracle
import paper_2204_03775_gb300 as wsb
from paper_2204_03775_gb300 import synthetic

pytestmark = pytest.mark.gpu

MODES = [(wsb.WS_STORAGE_BF16, "bf16"), (wsb.WS_STORAGE_FP16, "fp16")]


@pytest.fixture(scope="module", autouse=True)
def _library():
    wsb.load_library(build_if_missing=True)


def round_bf16(x):
    """Round float32 to bfloat16 precision (nearest, ties to even), back to float32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def round_fp16(x, e=0):
    """FP16 rounding of x * 2^e, in units of x."""
    x = np.asarray(x, np.float64) * 2.0 ** e
    return (x.astype(np.float16).astype(np.float64) * 2.0 ** -e)


def ulp_bf16(x):
    """Spacing of BF16 values at |x| (normal range)."""
    _, k = np.frexp(np.abs(np.asarray(x, np.float64)))
    return np.ldexp(1.0, k - 8)


def ulp_fp16(x, e=0):
    """Spacing of FP16 values at |x * 2^e| (subnormals included), in units of x."""
    _, k = np.frexp(np.abs(np.asarray(x, np.float64)) * 2.0 ** e)
    return np.ldexp(1.0, np.maximum(k - 11, -24) - e)


@pytest.mark.parametrize("tile_y", [16, 24, 48])
@pytest.mark.parametrize("shape", [(200, 60, 30), (99, 57, 21)])   # taper-free tiles; ragged x, odd y
@pytest.mark.parametrize("storage,name", MODES)
def test_one_step_is_the_rounded_exact_update(storage, name, shape, tile_y):
    nx, ny, nz = shape
    h, v = 10.0, 2000.0
    dt = 0.25 * h / v                      # (V dt / h)^2 = 1/16, exact everywhere
    vel = np.full((nz, ny, nx), v, np.float32)
    rng = np.random.default_rng(4)
    # u^n and d = u^n - u^{n-1} on a coarse grid (multiples of 2^-7 in +-[0.5, 1)
    # and +-[2^-3, 2^-2)): exact in BF16 and FP16, and u^{n-1} = u^n - d exact in FP32
    sgn = lambda: rng.choice([-1.0, 1.0], (nz, ny, nx))
    u0 = (np.round(rng.uniform(0.5, 1.0, (nz, ny, nx)) * 128) / 128 * sgn()).astype(np.float32)
    d0 = (np.round(rng.uniform(0.125, 0.25, (nz, ny, nx)) * 128) / 128 * sgn()).astype(np.float32)
    assert np.array_equal(round_bf16(u0), u0) and np.array_equal(round_fp16(u0), u0)
    assert np.array_equal(round_bf16(d0), d0) and np.array_equal(round_fp16(d0), d0)
    um1 = (u0 - d0).astype(np.float32)
    # the last cells sit in the partial column quad and the unpaired last row
    rec = np.array([[5, 5, 5], [60, 20, 15], [nx - 1, ny - 1, nz - 1], [nx - 2, ny - 2, 3],
                    [100 % nx, 30, 12]], np.int32)
    src = [(48, 20, 15, 25.0, 0.01, 0.05)]   # small: the field's maximum stays below 1
    sponge = (5, 0.1)

    hd = wsb.ws_create(nx, ny, nz, h, dt)
    wsb.ws_set_kernel(hd, wsb.WS_KERNEL_AUTO, 64, tile_y, 0)
    wsb.ws_set_storage(hd, storage)
    wsb.ws_set_velocity(hd, vel)
    wsb.ws_set_sponge(hd, *sponge)
    for s_ in src:
        wsb.ws_add_source(hd, *s_)
    wsb.ws_write_field(hd, u0, um1, 3)
    wsb.ws_set_receivers(hd, rec, 1)
    wsb.ws_step(hd, 1)
    wsb.ws_synchronize(hd)
    u16, up16 = wsb.ws_read_field(hd)
    tr16 = wsb.ws_read_traces(hd)
    wsb.ws_destroy(hd)

    ref = oracle.run(vel.astype(np.float64), h, dt, 1, sources=src, receivers=rec, sponge=sponge,
                     n0=3, u_init=u0, uprev_init=um1)
    ue = ref["u"]                              # exact u^{n+1}
    de = ue - u0.astype(np.float64)            # exact u^{n+1} - u^n
    d16 = u16.astype(np.float64) - up16.astype(np.float64)   # the stored D' (exact in FP32)
    np.testing.assert_allclose(tr16, ref["traces"], rtol=0, atol=2e-6)   # traces: u~ in FP32
    # the kernel scales the state by 2^e with the field's maximum near 2^12:
    # max(|u^n|, |u^n - u^{n-1}|, source bound) < 1 here, so e = 12
    if name == "bf16":
        rnd, ulp = round_bf16, ulp_bf16
    else:
        rnd, ulp = (lambda x: round_fp16(x, 12)), (lambda x: ulp_fp16(x, 12))
    for got, exact in [(u16.astype(np.float64), ue), (d16, de)]:
        diff = np.abs(got - exact)
        assert (diff <= ulp(exact) + 2e-6).all(), diff.max()        # within one unit
        exact_rounded = got == rnd(exact)
        assert exact_rounded.mean() >= 0.99, exact_rounded.mean()    # correctly rounded


# stated accuracy (relative L2 vs the FP64 oracle) on the layered survey:
# FP32 and FP16 after 200 steps, BF16 after 100 (its claimed range); FP32
# storage is there for contrast
BOUNDS = {"fp32": 1e-5, "fp16": 3e-3, "bf16": 1e-2}
STEPS = {"fp32": 200, "fp16": 200, "bf16": 100}   # BF16: where 1e-2 is claimed


@pytest.mark.parametrize("storage,name", [(wsb.WS_STORAGE_FP32, "fp32")] + MODES)
def test_accuracy_against_oracle(storage, name):
    w = synthetic.layered_survey(96, 80, 72, nt=STEPS[name])
    ref = oracle.run(w.vel, w.h, w.dt, w.nt, sources=w.sources, receivers=w.receivers,
                     sponge=w.sponge)
    hd = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
    wsb.ws_set_storage(hd, storage)
    wsb.ws_set_velocity(hd, w.vel)
    wsb.ws_set_sponge(hd, *w.sponge)
    for s in w.sources:
        wsb.ws_add_source(hd, *s)
    wsb.ws_set_receivers(hd, w.receivers, w.nt)
    wsb.ws_step(hd, w.nt)
    wsb.ws_synchronize(hd)
    u, _ = wsb.ws_read_field(hd)
    err = np.linalg.norm(u - ref["u"]) / np.linalg.norm(ref["u"])
    print(f"{name}: relative L2 error after {w.nt} steps: {err:.3e}")
    assert err <= BOUNDS[name], err


def test_storage_modes_against_oracle_to_1000_steps():
    """The layered survey recipe at 512^3 (the benchmark's model at half the
    size per axis) for the configured 1000 steps: every storage mode against
    the FP64 oracle at steps 100, 500 and 1000 (the oracle continues its own
    state between checkpoints), on the field and on the traces recorded so
    far. Claimed and asserted: FP32 within 1e-4 and FP16 within 1e-2 at every
    checkpoint, BF16 within 1e-2 at 100 steps. Beyond 100 steps BF16 is
    reported, not bounded: it does not hold 1e-2 there."""
    w = synthetic.layered_survey(512, 512, 512, nt=1000)
    checkpoints = (100, 500, 1000)
    hs = {}
    for storage, name in [(wsb.WS_STORAGE_FP32, "fp32")] + MODES:
        hd = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
        wsb.ws_set_storage(hd, storage)
        wsb.ws_set_velocity(hd, w.vel)
        wsb.ws_set_sponge(hd, *w.sponge)
        for s in w.sources:
            wsb.ws_add_source(hd, *s)
        wsb.ws_set_receivers(hd, w.receivers, w.nt)
        hs[name] = hd
    claimed = {"fp32": (1e-4, 1000), "fp16": (1e-2, 1000), "bf16": (1e-2, 100)}
    v64 = w.vel.astype(np.float64)
    ref, done, ref_tr = None, 0, []
    for c in checkpoints:
        kw = {} if ref is None else {"n0": done, "u_init": ref["u"], "uprev_init": ref["u_prev"]}
        ref = oracle.run(v64, w.h, w.dt, c - done, sources=w.sources, receivers=w.receivers,
                         sponge=w.sponge, **kw)
        ref_tr.append(ref["traces"])
        rtr = np.concatenate(ref_tr, axis=1)
        nref, ntr = np.linalg.norm(ref["u"]), np.linalg.norm(rtr)
        for name, hd in hs.items():
            wsb.ws_step(hd, c - done)
            u, _ = wsb.ws_read_field(hd)
            tr = wsb.ws_read_traces(hd)[:, :c]
            err = np.linalg.norm(u - ref["u"]) / nref
            err_tr = np.linalg.norm(tr - rtr) / ntr
            print(f"{name}: 512^3, {c} steps, relative L2 vs the FP64 oracle: field {err:.3e}, "
                  f"traces {err_tr:.3e}")
            bound, upto = claimed[name]
            if c <= upto:
                assert err <= bound and err_tr <= bound, (name, c, err, err_tr)
            else:
                assert np.isfinite(err) and np.isfinite(err_tr), (name, c)
        done = c
    for hd in hs.values():
        wsb.ws_destroy(hd)


@pytest.mark.parametrize("shape", [(64, 16, 1), (64, 16, 3), (70, 17, 6), (128, 16, 2),
                                   (64, 24, 2), (70, 25, 5), (65, 48, 3), (130, 50, 4)])
@pytest.mark.parametrize("storage,name", MODES)
def test_thin_and_minimal_grids(storage, name, shape):
    """The smallest grids 16-bit storage accepts (nx >= 64, ny >= 16), down to
    one plane, ragged in x and y, with each tile height that fits the grid
    (64 x 16 from ny = 16, 64 x 24 from 24, 64 x 48 from 48): 30 steps against
    the FP64 oracle."""
    nx, ny, nz = shape
    vel = synthetic.smooth_random_velocity((nz, ny, nx), 11, spacing=4)
    h, dt = 10.0, synthetic.cfl_dt(4500.0, 10.0)
    src = [(nx // 3, ny // 2, nz // 2, 20.0, 0.04, 1.0)]
    rec = np.array([[0, 0, 0], [nx - 1, ny - 1, nz - 1], [nx // 2, ny // 3, nz // 2]], np.int32)
    hd = wsb.ws_create(nx, ny, nz, h, dt)
    wsb.ws_set_kernel(hd, wsb.WS_KERNEL_AUTO, 64, max(t for t in (16, 24, 48) if t <= ny), 0)
    wsb.ws_set_storage(hd, storage)
    wsb.ws_set_velocity(hd, vel)
    wsb.ws_set_sponge(hd, 3, 0.1)
    for s in src:
        wsb.ws_add_source(hd, *s)
    wsb.ws_set_receivers(hd, rec, 30)
    wsb.ws_step(hd, 30)
    u, _ = wsb.ws_read_field(hd)
    tr = wsb.ws_read_traces(hd)
    ref = oracle.run(vel.astype(np.float64), h, dt, 30, sources=src, receivers=rec, sponge=(3, 0.1))
    bound = {"fp16": 3e-3, "bf16": 1e-2}[name]
    err = np.linalg.norm(u - ref["u"]) / np.linalg.norm(ref["u"])
    assert err <= bound, err
    # traces against the field's scale: a receiver the wave has barely reached
    # sees values below the 16-bit range of this step's scale (FP16 spans
    # ~2^-36 of the field maximum), which the stored state holds as zero
    scale = max(np.abs(ref["traces"]).max(), np.abs(ref["u"]).max())
    assert np.abs(tr - ref["traces"]).max() <= bound * scale


@pytest.mark.parametrize("tile_y", [16, 24])
@pytest.mark.parametrize("storage,name", MODES)
def test_z_blocks_do_not_change_bits(storage, name, tile_y):
    """Items of every length from one plane up: the kernel walks each item's
    planes three at a time around a 9-slot ring, so item lengths that end a
    trip early and items that wrap the ring several times must give the same
    bits as the default blocks (every tiling computes the same expression per
    cell). 25 steps with a source, receivers in and between blocks, and the
    taper."""
    nx, ny, nz = 150, 40, 61
    vel = synthetic.smooth_random_velocity((nz, ny, nx), 23, spacing=4)
    h, dt = 10.0, synthetic.cfl_dt(4500.0, 10.0)
    src = (70, 20, 30, 20.0, 0.04, 1.0)
    rec = np.array([[0, 0, 0], [149, 39, 60], [70, 20, 9], [71, 21, 10], [5, 33, 27],
                    [100, 8, 45]], np.int32)

    def run(zb):
        hd = wsb.ws_create(nx, ny, nz, h, dt)
        wsb.ws_set_kernel(hd, wsb.WS_KERNEL_AUTO, 64, tile_y, zb)
        wsb.ws_set_storage(hd, storage)
        wsb.ws_set_velocity(hd, vel)
        wsb.ws_set_sponge(hd, 4, 0.1)
        wsb.ws_add_source(hd, *src)
        wsb.ws_set_receivers(hd, rec, 25)
        wsb.ws_step(hd, 25)
        out = (*wsb.ws_read_field(hd), wsb.ws_read_traces(hd))
        wsb.ws_destroy(hd)
        return out

    ref = run(0)
    assert np.abs(ref[2]).max() > 0
    for zb in (1, 2, 3, 4, 5, 7, 9, 10, 13, 29, 61):
        got = run(zb)
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b, err_msg=f"zblock {zb}")


@pytest.mark.parametrize("storage,name", MODES)
def test_storage_round_trip(storage, name):
    w = synthetic.layered_survey(80, 64, 48, nt=60)
    hd = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
    wsb.ws_set_velocity(hd, w.vel)
    for s in w.sources:
        wsb.ws_add_source(hd, *s)
    wsb.ws_step(hd, 60)
    u_a, p_a = wsb.ws_read_field(hd)
    wsb.ws_set_storage(hd, storage)
    u_b, p_b = wsb.ws_read_field(hd)
    wsb.ws_set_storage(hd, wsb.WS_STORAGE_FP32)
    u_c, p_c = wsb.ws_read_field(hd)
    tol = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11}[name]
    for a, b, c in [(u_a, u_b, u_c), (p_a, p_b, p_c)]:
        scale = np.abs(a).max()
        assert np.abs(b - a).max() <= tol * scale
        np.testing.assert_array_equal(b, c)
    assert wsb.ws_get_step(hd) == 60


def test_storage_needs_a_64_wide_grid():
    hd = wsb.ws_create(48, 16, 16, 10.0, 1e-3)
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_set_storage(hd, wsb.WS_STORAGE_BF16)
    assert e.value.code == wsb.WS_ERR_BADARG
    hd = wsb.ws_create(64, 30, 16, 10.0, 1e-3)       # a 16-bit tile taller than the grid
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_set_kernel(hd, wsb.WS_KERNEL_AUTO, 64, 48, 0)
    assert e.value.code == wsb.WS_ERR_BADARG
    with pytest.raises(wsb.WaveStepError) as e:      # not a tile of either streaming kernel
        wsb.ws_set_kernel(hd, wsb.WS_KERNEL_AUTO, 64, 40, 0)
    assert e.value.code == wsb.WS_ERR_BADARG


def test_full_size_accuracy_against_fp32_and_oracle():
    """The benchmark's 1024^3 survey, 100 steps: each 16-bit mode against FP32
    storage on the device, and every mode against the FP64 oracle on the
    light cone, in the launch configurations bench.py times (the 16-bit
    kernel's 64 x 16 tile, the FP32 kernel's default 64 x 8, default z
    blocks). Bounds: the claimed 1e-2 for BF16 (measured 6.2e-3), 2e-3 for
    FP16 (measured 7.9e-4)."""
    import torch
    w = synthetic.layered_survey(1024, 1024, 1024, nt=100)
    bound = {"fp32": 0.0, "fp16": 2e-3, "bf16": 1e-2}
    out = {}
    for storage, name in [(wsb.WS_STORAGE_FP32, "fp32")] + MODES:
        hd = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
        wsb.ws_set_storage(hd, storage)
        wsb.ws_set_velocity(hd, w.vel)
        wsb.ws_set_sponge(hd, *w.sponge)
        for s in w.sources:
            wsb.ws_add_source(hd, *s)
        wsb.ws_set_receivers(hd, w.receivers, w.nt)
        wsb.ws_step(hd, w.nt)
        wsb.ws_synchronize(hd)
        u = torch.empty((w.nz, w.ny, w.nx), dtype=torch.float32, device="cuda")
        wsb.ws_read_field(hd, u, None)
        torch.cuda.synchronize()
        out[name] = u
        wsb.ws_destroy(hd)
    ref = out["fp32"].double()
    nref = torch.linalg.vector_norm(ref).item()
    for name in ("fp16", "bf16"):
        err = torch.linalg.vector_norm(out[name].double() - ref).item() / nref
        print(f"{name}: 1024^3, 100 steps, relative L2 vs FP32 storage {err:.3e}")
        assert err <= bound[name], (name, err)

    # and against the FP64 oracle itself: after nt steps from rest the field
    # is exactly zero farther than 4 nt cells from the source, so the oracle
    # steps only the window that holds the light cone (803 x 803 x 422 cells)
    si, sj, sk = w.sources[0][:3]
    r = 4 * w.nt + 1
    ox, oy, wx, wy, wz = si - r, sj - r, 2 * r + 1, 2 * r + 1, sk + r + 1
    sub = np.ascontiguousarray(w.vel[:wz, oy:oy + wy, ox:ox + wx])
    orc = oracle.run(sub, w.h, w.dt, w.nt, sources=w.sources, sponge=w.sponge,
                     window=(ox, oy, 0, w.nx, w.ny, w.nz))["u"]
    norc = np.linalg.norm(orc)
    vs_oracle = {"fp32": 1e-4, "fp16": 2e-3, "bf16": 1e-2}
    for name, bnd in vs_oracle.items():
        u = out[name]
        win = u[:wz, oy:oy + wy, ox:ox + wx].cpu().numpy().astype(np.float64)
        err = np.linalg.norm(win - orc) / norc
        print(f"{name}: 1024^3, 100 steps, relative L2 vs the FP64 oracle {err:.3e}")
        assert err <= bnd, (name, err)
        beyond = u.clone()                        # exactly zero beyond the light cone
        beyond[:wz, oy:oy + wy, ox:ox + wx] = 0
        assert torch.count_nonzero(beyond).item() == 0, name
        del beyond
