"""GPU adjoint gradient (ws_adjoint_gradient) against the FP64 oracle.

The oracle's adjoint is pinned on the CPU by the dot-product test and by
central differences (tests/test_oracle_adjoint.py); here the GPU gradient,
computed by a different route (the step kernels advance rho = W G lambda,
the states come back from sqrt(N) checkpoints), must match it:
1. the whole gradient field, relative to its maximum, within 1e-3 (FP32
   forward and backward passes; the observed error is far smaller), on grids
   that span several streaming tiles with a ragged tail, and on the direct
   kernel. Both sides get the same seeded residual (residual mode; the
   oracle gets d = its traces - r), so the comparison measures the adjoint
   itself. With observed data instead, the residual is a difference of FP32
   traces: at a receiver on the source, |traces| / |r| reaches 1e4 and the
   traces' FP32 rounding alone moves the gradient there by ~1e-3, so the
   data-mode comparison keeps its receivers off the sources;
2. the oracle's FP64 central differences of the misfit at 8 cells (source,
   receiver, taper, interior), within 1e-3 of the gradient's maximum;
3. step counts that exercise the checkpoint layout (1, 2, a perfect square,
   a prime) and a source in the taper;
4. the residual mode gives bit for bit the data mode's gradient when handed
   traces - d (the same FP32 residual), and the handle ends in the state of a
   plain forward run.
"""

import numpy as np
import pytest

import oracle
import paper_2204_03775_gb300 as wsb
from paper_2204_03775_gb300 import synthetic

pytestmark = pytest.mark.gpu

TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _library():
    wsb.load_library(build_if_missing=True)


def _case(nx, ny, nz, nt, seed=5, sponge=(4, 0.12), rec_on_source=True):
    vel = synthetic.smooth_random_velocity((nz, ny, nx), seed, 2000.0, 3200.0, spacing=6)
    h = 10.0
    dt = synthetic.cfl_dt(float(vel.max()), h)
    src = [(nx // 3, ny // 2, 3, 28.0, 0.035, 1.0), (2 * nx // 3, ny // 3, nz - 5, 22.0, 0.05, -0.7)]
    rng = np.random.default_rng(seed)
    cells = rng.choice(nx * ny * nz, 12, replace=False)    # distinct cells
    rec = np.stack([cells % nx, cells // nx % ny, cells // (nx * ny)], axis=1).astype(np.int32)
    if rec_on_source:
        rec[0] = (src[0][0], src[0][1], src[0][2])
    true = vel.astype(np.float64)
    true[nz // 4: nz // 2, ny // 4: 3 * ny // 4, nx // 4: nx // 2] *= 1.07
    d_obs = oracle.run(true, h, dt, nt, sources=src, receivers=rec, sponge=sponge)["traces"]
    return vel, h, dt, src, rec, sponge, d_obs.astype(np.float32)


def _gpu(vel, h, dt, nt, src, rec, sponge, data, kernel=wsb.WS_KERNEL_AUTO, mode=None,
         slowness=False):
    nz, ny, nx = vel.shape
    hd = wsb.ws_create(nx, ny, nz, h, dt)
    if slowness:
        wsb.ws_set_slowness2(hd, (1.0 / vel.astype(np.float64) ** 2).astype(np.float32))
    else:
        wsb.ws_set_velocity(hd, vel)
    wsb.ws_set_sponge(hd, *sponge)
    wsb.ws_set_kernel(hd, kernel)
    for s in src:
        wsb.ws_add_source(hd, *s)
    wsb.ws_set_receivers(hd, rec, nt)
    g, j = wsb.ws_adjoint_gradient(hd, data, wsb.WS_ADJ_DATA if mode is None else mode)
    return hd, g, j


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("shape,nt,kernel", [
    ((150, 40, 36), 80, wsb.WS_KERNEL_STREAM),     # 3 x 5 tiles, ragged in x and y
    ((72, 20, 16), 49, wsb.WS_KERNEL_STREAM),      # N a perfect square
    ((40, 22, 18), 53, wsb.WS_KERNEL_DIRECT),      # N prime
    ((72, 20, 16), 2, wsb.WS_KERNEL_STREAM),
    ((33, 17, 12), 1, wsb.WS_KERNEL_DIRECT),
])
def test_gradient_matches_oracle(shape, nt, kernel):
    nx, ny, nz = shape
    vel, h, dt, src, rec, sponge, _ = _case(nx, ny, nz, nt)
    v64 = vel.astype(np.float64)
    ref_tr = oracle.run(v64, h, dt, nt, sources=src, receivers=rec, sponge=sponge)["traces"]
    r = np.random.default_rng(nt).standard_normal(ref_tr.shape).astype(np.float32)
    ref = oracle.adjoint_gradient(v64, h, dt, nt, ref_tr - r.astype(np.float64), sources=src,
                                  receivers=rec, sponge=sponge)
    hd, g, j = _gpu(vel, h, dt, nt, src, rec, sponge, r, kernel, mode=wsb.WS_ADJ_RESIDUAL)
    err = _rel(g, ref["grad_m"])
    print(f"{shape} nt={nt}: gradient max error / max |g| = {err:.2e}")
    assert err <= TOL, err
    assert j == pytest.approx(ref["misfit"], rel=1e-6)
    tr = wsb.ws_read_traces(hd)
    assert _rel(tr, ref_tr) <= 1e-5
    assert wsb.ws_get_step(hd) == nt


def test_gradient_from_observed_data_matches_oracle():
    nx, ny, nz, nt = 150, 40, 36, 80
    vel, h, dt, src, rec, sponge, d_obs = _case(nx, ny, nz, nt, rec_on_source=False)
    ref = oracle.adjoint_gradient(vel.astype(np.float64), h, dt, nt, d_obs.astype(np.float64),
                                  sources=src, receivers=rec, sponge=sponge)
    _, g, j = _gpu(vel, h, dt, nt, src, rec, sponge, d_obs)
    err = _rel(g, ref["grad_m"])
    print(f"observed data: gradient max error / max |g| = {err:.2e}; misfit {j:.6e} vs "
          f"{ref['misfit']:.6e}")
    assert err <= TOL, err
    assert j == pytest.approx(ref["misfit"], rel=1e-4)


def test_gradient_matches_oracle_central_differences():
    nx, ny, nz, nt = 72, 20, 16, 60
    vel, h, dt, src, rec, sponge, d_obs = _case(nx, ny, nz, nt, seed=8, rec_on_source=False)
    v64 = vel.astype(np.float64)
    d64 = d_obs.astype(np.float64)
    _, g, _ = _gpu(vel, h, dt, nt, src, rec, sponge, d_obs)

    def misfit(m):
        tr = oracle.run(1.0 / np.sqrt(m), h, dt, nt, sources=src, receivers=rec,
                        sponge=sponge)["traces"]
        return 0.5 * np.sum((tr - d64) ** 2)

    m = 1.0 / v64 ** 2
    rng = np.random.default_rng(1)
    cells = [(src[0][2], src[0][1], src[0][0]), (rec[3][2], rec[3][1], rec[3][0]), (1, 2, 3),
             (nz - 1, ny - 2, nx - 1),
             *[tuple(int(x) for x in rng.integers([0, 0, 0], [nz, ny, nx])) for _ in range(4)]]
    scale = np.abs(g).max()
    for (k, j, i) in cells:
        eps = 1e-4 * m[k, j, i]
        mp, mm = m.copy(), m.copy()
        mp[k, j, i] += eps
        mm[k, j, i] -= eps
        fd = (misfit(mp) - misfit(mm)) / (2 * eps)
        assert abs(fd - g[k, j, i]) <= TOL * scale, ((k, j, i), fd, g[k, j, i])


def test_residual_mode_and_slowness_model():
    nx, ny, nz, nt = 72, 24, 20, 40
    vel, h, dt, src, rec, sponge, d_obs = _case(nx, ny, nz, nt, seed=11)
    hd, g_data, j_data = _gpu(vel, h, dt, nt, src, rec, sponge, d_obs)
    tr = wsb.ws_read_traces(hd)
    r = (tr - d_obs).astype(np.float32)
    _, g_res, j_res = _gpu(vel, h, dt, nt, src, rec, sponge, r, mode=wsb.WS_ADJ_RESIDUAL)
    np.testing.assert_array_equal(g_res, g_data)
    assert j_res == j_data
    # the handle ends where a plain forward run ends
    hf = wsb.ws_create(nx, ny, nz, h, dt)
    wsb.ws_set_velocity(hf, vel)
    wsb.ws_set_sponge(hf, *sponge)
    for s in src:
        wsb.ws_add_source(hf, *s)
    wsb.ws_set_receivers(hf, rec, nt)
    wsb.ws_step(hf, nt)
    u_f, p_f = wsb.ws_read_field(hf)
    u_a, p_a = wsb.ws_read_field(hd)
    np.testing.assert_array_equal(u_a, u_f)
    np.testing.assert_array_equal(p_a, p_f)
    np.testing.assert_array_equal(wsb.ws_read_traces(hf), tr)
    # a model given as squared slowness: W differs by float rounding only
    _, g_m, _ = _gpu(vel, h, dt, nt, src, rec, sponge, d_obs, slowness=True)
    assert _rel(g_m, g_data) <= 1e-4


def test_device_arrays():
    torch = pytest.importorskip("torch")
    nx, ny, nz, nt = 72, 20, 16, 30
    vel, h, dt, src, rec, sponge, d_obs = _case(nx, ny, nz, nt, seed=12)
    _, g_host, j_host = _gpu(vel, h, dt, nt, src, rec, sponge, d_obs)
    _, g_dev, j_dev = _gpu(vel, h, dt, nt, src, rec, sponge, torch.from_numpy(d_obs).cuda())
    assert g_dev.is_cuda
    np.testing.assert_array_equal(g_dev.cpu().numpy(), g_host)
    assert j_dev == j_host


def test_errors():
    hd = wsb.ws_create(40, 20, 16, 10.0, 1e-3)
    data = np.zeros((1, 5), np.float32)
    with pytest.raises(wsb.WaveStepError) as e:        # no model
        wsb.ws_set_receivers(hd, [[1, 1, 1]], 5)
        wsb.ws_adjoint_gradient(hd, data)
    assert e.value.code == wsb.WS_ERR_STATE
    wsb.ws_set_velocity(hd, np.full((16, 20, 40), 2000.0, np.float32))
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_adjoint_gradient(hd, data, mode=7)
    assert e.value.code == wsb.WS_ERR_BADARG
    wsb.ws_set_receivers(hd, np.zeros((0, 3), np.int32), 0)
    with pytest.raises(wsb.WaveStepError) as e:        # no receivers
        wsb.ws_adjoint_gradient(hd, np.zeros((0, 0), np.float32))
    assert e.value.code == wsb.WS_ERR_STATE
    with pytest.raises(wsb.WaveStepError) as e:        # non-positive slowness
        wsb.ws_set_slowness2(hd, np.zeros((16, 20, 40), np.float32))
    assert e.value.code == wsb.WS_ERR_BADARG
    with pytest.raises(wsb.WaveStepError) as e:        # too fast for dt
        wsb.ws_set_slowness2(hd, np.full((16, 20, 40), 1e-9, np.float32))
    assert e.value.code == wsb.WS_ERR_CFL
    h16 = wsb.ws_create(64, 16, 8, 10.0, 1e-3)             # the adjoint needs FP32 storage
    wsb.ws_set_storage(h16, wsb.WS_STORAGE_FP16)
    wsb.ws_set_velocity(h16, np.full((8, 16, 64), 2000.0, np.float32))
    wsb.ws_set_receivers(h16, [[1, 1, 1]], 5)
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_adjoint_gradient(h16, data)
    assert e.value.code == wsb.WS_ERR_STATE


def test_autograd_function_two_shots():
    torch = pytest.importorskip("torch")
    from paper_2204_03775_gb300 import autograd as wsa
    nx, ny, nz, nt = 72, 20, 16, 40
    vel, h, dt, src, rec, sponge, d_obs = _case(nx, ny, nz, nt, seed=13)
    shots = [wsa.Shot((nz, ny, nx), h, dt, nt, [s], rec, sponge) for s in src]
    d_each = [oracle.run(vel.astype(np.float64) * 1.03, h, dt, nt, sources=[s], receivers=rec,
                         sponge=sponge)["traces"].astype(np.float32) for s in src]
    m = torch.from_numpy((1.0 / vel.astype(np.float64) ** 2).astype(np.float32)).cuda()
    m.requires_grad_(True)
    loss = sum(0.5 * ((wsa.traces(m, sh) - torch.from_numpy(d).cuda()) ** 2).sum()
               for sh, d in zip(shots, d_each))
    loss.backward()
    ref = np.zeros((nz, ny, nx), np.float32)
    jsum = 0.0
    for s, d in zip(src, d_each):
        _, g, j = _gpu(vel, h, dt, nt, [s], rec, sponge, d, slowness=True)
        ref += g
        jsum += j
    np.testing.assert_allclose(m.grad.cpu().numpy(), ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())
    assert float(loss.detach()) == pytest.approx(jsum, rel=1e-5)


def test_forward_then_residual_gradient_reuses_the_run():
    """ws_forward keeps the checkpoints; a residual-mode gradient right after
    it skips its own forward run and gives the same bits; any change to the
    model in between forces a new forward run (and the right gradient)."""
    nx, ny, nz, nt = 72, 20, 16, 40
    vel, h, dt, src, rec, sponge, _ = _case(nx, ny, nz, nt, seed=21)
    r = np.random.default_rng(3).standard_normal((len(rec), nt)).astype(np.float32)
    hd, g_full, _ = _gpu(vel, h, dt, nt, src, rec, sponge, r, mode=wsb.WS_ADJ_RESIDUAL)
    h2 = wsb.ws_create(nx, ny, nz, h, dt)
    wsb.ws_set_velocity(h2, vel)
    wsb.ws_set_sponge(h2, *sponge)
    for s in src:
        wsb.ws_add_source(h2, *s)
    wsb.ws_set_receivers(h2, rec, nt)
    wsb.ws_forward(h2)
    np.testing.assert_array_equal(wsb.ws_read_traces(h2), wsb.ws_read_traces(hd))
    launches = wsb.ws_launch_count(h2)
    g_reuse, _ = wsb.ws_adjoint_gradient(h2, r, wsb.WS_ADJ_RESIDUAL)
    used = wsb.ws_launch_count(h2) - launches
    np.testing.assert_array_equal(g_reuse, g_full)
    launches = wsb.ws_launch_count(h2)
    wsb.ws_adjoint_gradient(h2, r, wsb.WS_ADJ_RESIDUAL)          # still the same run: reused
    assert wsb.ws_launch_count(h2) - launches == used
    # a new model: the forward run is redone, so more launches, other values
    wsb.ws_set_velocity(h2, (vel * 1.01).astype(np.float32))
    launches = wsb.ws_launch_count(h2)
    g_new, _ = wsb.ws_adjoint_gradient(h2, r, wsb.WS_ADJ_RESIDUAL)
    assert wsb.ws_launch_count(h2) - launches >= used + nt
    _, g_ref, _ = _gpu((vel * 1.01).astype(np.float32), h, dt, nt, src, rec, sponge, r,
                       mode=wsb.WS_ADJ_RESIDUAL)
    np.testing.assert_array_equal(g_new, g_ref)


def test_several_shots_sum_and_norm_against_oracle():
    """ws_adjoint_gradient_shots: three shots on one model (each its own
    sources, receivers and stream) against the FP64 oracle's summed adjoint
    gradient, with the same seeded residuals; the summed misfit; the FP64
    gradient norm against the norm of the oracle's gradient; and each shot
    alone through ws_adjoint_gradient gives the same summed field."""
    torch = pytest.importorskip("torch")
    nx, ny, nz, nt = 150, 40, 36, 64
    vel, h, dt, _, _, sponge, _ = _case(nx, ny, nz, nt)
    v64 = vel.astype(np.float64)
    rng = np.random.default_rng(31)
    shots = []
    for q in range(3):
        src = [(20 + 50 * q, 10 + 9 * q, 3 + q, 25.0 + 2 * q, 0.04, 1.0 - 0.3 * q)]
        cells = rng.choice(nx * ny * nz, 9 + q, replace=False)
        rec = np.stack([cells % nx, cells // nx % ny, cells // (nx * ny)], axis=1).astype(np.int32)
        tr = oracle.run(v64, h, dt, nt, sources=src, receivers=rec, sponge=sponge)["traces"]
        r = rng.standard_normal(tr.shape).astype(np.float32)
        ref = oracle.adjoint_gradient(v64, h, dt, nt, tr - r.astype(np.float64), sources=src,
                                      receivers=rec, sponge=sponge)
        shots.append((src, rec, r, ref))
    g_ref = sum(s[3]["grad_m"] for s in shots)
    j_ref = sum(s[3]["misfit"] for s in shots)

    handles, streams = [], []
    for src, rec, _, _ in shots:
        hd = wsb.ws_create(nx, ny, nz, h, dt)
        st = torch.cuda.Stream()
        wsb.ws_set_stream(hd, st)
        wsb.ws_set_velocity(hd, vel)
        wsb.ws_set_sponge(hd, *sponge)
        for s in src:
            wsb.ws_add_source(hd, *s)
        wsb.ws_set_receivers(hd, rec, nt)
        handles.append(hd)
        streams.append(st)
    g, j, gn = wsb.ws_adjoint_gradient_shots(handles, [s[2] for s in shots], wsb.WS_ADJ_RESIDUAL)
    err = _rel(g, g_ref)
    print(f"3 shots: summed gradient max error / max |g| = {err:.2e}, norm {gn:.6e} vs "
          f"{np.linalg.norm(g_ref):.6e}")
    assert err <= TOL, err
    assert j == pytest.approx(j_ref, rel=1e-6)
    # the norm is the FP64 norm of the returned field, and close to the oracle's
    assert gn == pytest.approx(np.linalg.norm(g.astype(np.float64)), rel=1e-12)
    assert gn == pytest.approx(np.linalg.norm(g_ref), rel=TOL)
    # shot by shot through the single-shot call: the same per-shot fields,
    # summed here in FP64 in shot order
    acc = np.zeros((nz, ny, nx))
    for hd, (_, _, r, _) in zip(handles, shots):
        gq, _ = wsb.ws_adjoint_gradient(hd, r, wsb.WS_ADJ_RESIDUAL)
        acc += gq.astype(np.float64)
    np.testing.assert_array_equal(g, acc.astype(np.float32))


def test_several_shots_reject_mismatched_handles():
    a = wsb.ws_create(40, 20, 16, 10.0, 1e-3)
    b = wsb.ws_create(40, 20, 17, 10.0, 1e-3)
    d = np.zeros((1, 4), np.float32)
    for h in (a, b):
        wsb.ws_set_velocity(h, np.full(h.shape, 2000.0, np.float32))
        wsb.ws_set_receivers(h, np.array([[1, 1, 1]], np.int32), 4)
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_adjoint_gradient_shots([a, b], [d, d])
    assert e.value.code == wsb.WS_ERR_BADARG
    with pytest.raises(wsb.WaveStepError) as e:
        wsb.ws_adjoint_gradient_shots([a, a], [d, d])
    assert e.value.code == wsb.WS_ERR_BADARG
