"""The adjoint gradient on the full gradient workload: 256^3, 16 surface
shots, 128 x 128 receivers, 800 steps, true model = layered background with
a +10% Gaussian blob, start model = the background.

The FP64 oracle cannot take this size (it keeps every state: 800 x 20 M
doubles), so here the gradient is held to what holds at any size: it is the
derivative of the misfit the same library computes. Central differences of
the FP32 forward misfit (four-point, step 1% of m at the cell) at 8 random
cells of the 60 planes under the shots agree with it within 1e-3 of max |g|,
and the derivative along the blob direction within 2e-3 relative. The
oracle comparison of the whole field runs at smaller sizes
(test_gpu_adjoint.py). An opt-in test (WS_ORACLE_FD=1) takes the FP64
oracle's own central differences at full size for one shot, with the same
residual on both sides: the residual of this survey (reflections of the
blob) is ~1e-5 of the traces, so FP32 modelling error in the traces would
otherwise decide the comparison.
"""

import os

import numpy as np
import pytest

import paper_2204_03775_gb300 as wsb
from paper_2204_03775_gb300 import synthetic

pytestmark = pytest.mark.gpu


def test_gradient_against_central_differences_full_size():
    torch = pytest.importorskip("torch")
    wsb.load_library(build_if_missing=True)
    w = synthetic.adjoint_survey()
    dev = torch.device("cuda")
    m_true = torch.from_numpy((1.0 / w.vel_true.astype(np.float64) ** 2).astype(np.float32)).to(dev)
    m0 = torch.from_numpy((1.0 / w.vel_start.astype(np.float64) ** 2).astype(np.float32)).to(dev)
    hs = []
    for shot in w.shots:
        h = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
        wsb.ws_set_sponge(h, *w.sponge)
        for s in shot:
            wsb.ws_add_source(h, *s)
        wsb.ws_set_receivers(h, w.receivers, w.nt)
        wsb.ws_set_slowness2(h, m0)
        wsb.ws_autotune(h)
        hs.append(h)
    nrec = len(w.receivers)

    def forward(m):
        out = []
        for h in hs:
            wsb.ws_set_slowness2(h, m)
            wsb.ws_write_field(h, None, None, 0)
            wsb.ws_set_receivers(h, w.receivers, w.nt)
            wsb.ws_step(h, w.nt)
            t = torch.empty((nrec, w.nt), dtype=torch.float32, device=dev)
            wsb.ws_read_traces(h, t)
            out.append(t)
        return out

    d_obs = forward(m_true)

    def misfit(m):
        return sum(0.5 * float(((a - b).double() ** 2).sum()) for a, b in zip(forward(m), d_obs))

    g = torch.zeros_like(m0)
    gs = torch.empty_like(m0)
    J = 0.0
    for h, d in zip(hs, d_obs):
        wsb.ws_set_slowness2(h, m0)
        _, j = wsb.ws_adjoint_gradient(h, d, wsb.WS_ADJ_DATA, gs)
        g += gs
        J += j
    assert J == pytest.approx(misfit(m0), rel=1e-12)
    gc = g.cpu().numpy()
    gmax = np.abs(gc).max()
    nb = w.sponge[0]
    rng = np.random.default_rng(7)
    # the shots and receivers lie on k = 20: cells in the 60 planes below it
    cells = [tuple(int(x) for x in rng.integers([nb, nb, nb], [nb + 60, w.ny - nb, w.nx - nb]))
             for _ in range(8)]
    for c in cells:
        mc = float(m0[c])
        eps = 1e-2 * mc
        val = {}
        for s in (-2, -1, 1, 2):
            mp = m0.clone()
            mp[c] = mc + s * eps
            val[s] = misfit(mp)
        fd = (8.0 * (val[1] - val[-1]) - (val[2] - val[-2])) / (12.0 * eps)
        print(f"cell {c}: adjoint {gc[c]:.5e}  fd {fd:.5e}  |diff| / max|g| = "
              f"{abs(fd - gc[c]) / gmax:.2e}")
        assert abs(fd - gc[c]) <= 1e-3 * gmax, (c, fd, gc[c], gmax)
    dm = m_true - m0
    e = 0.1
    fd = (misfit(m0 + e * dm) - misfit(m0 - e * dm)) / (2 * e)
    dd = float((g.double() * dm.double()).sum())
    print(f"directional: fd {fd:.6e}  <g, dm> {dd:.6e}")
    assert abs(fd - dd) <= 2e-3 * abs(dd)


@pytest.mark.skipif(os.environ.get("WS_ORACLE_FD") != "1",
                    reason="17 FP64 oracle runs of 256^3 x 800 steps (about 8 minutes on 16 "
                           "host cores); set WS_ORACLE_FD=1")
def test_gradient_against_oracle_central_differences_full_size():
    """One shot of the full workload: the GPU gradient against the FP64
    oracle's central differences of the misfit (the oracle's own forward
    runs, the same observed data) at 8 seeded cells near the shot, where the
    gradient is large, within 1e-3 of max |g|."""
    import oracle

    wsb.load_library(build_if_missing=True)
    w = synthetic.adjoint_survey()
    shot = w.shots[0]
    # receivers within 10 cells of the source record the direct wave 1e3-1e4
    # times larger than the residual; there the FP32 traces' rounding, not
    # the adjoint, would decide the comparison, so they are left out
    si, sj, sk = shot[0][:3]
    far = np.hypot(w.receivers[:, 0] - si, w.receivers[:, 1] - sj) > 10
    rec = np.ascontiguousarray(w.receivers[far])
    true64 = w.vel_true.astype(np.float64)
    d_obs = oracle.run(true64, w.h, w.dt, w.nt, sources=shot, receivers=rec,
                       sponge=w.sponge)["traces"]
    h = wsb.ws_create(w.nx, w.ny, w.nz, w.h, w.dt)
    wsb.ws_set_sponge(h, *w.sponge)
    for s in shot:
        wsb.ws_add_source(h, *s)
    wsb.ws_set_receivers(h, rec, w.nt)
    wsb.ws_set_velocity(h, w.vel_start)
    g_data, _ = wsb.ws_adjoint_gradient(h, d_obs.astype(np.float32))
    # the same residual on both sides: the oracle's traces minus the data (the
    # GPU's FP32 traces differ from them by ~1e-6 of the direct wave, which is
    # not small next to a residual made of weak reflections)
    tr0 = oracle.run(w.vel_start.astype(np.float64), w.h, w.dt, w.nt, sources=shot,
                     receivers=rec, sponge=w.sponge)["traces"]
    r = (tr0 - d_obs).astype(np.float32)
    g, _ = wsb.ws_adjoint_gradient(h, r, wsb.WS_ADJ_RESIDUAL)
    gmax = np.abs(g).max()
    print(f"residual vs traces: |r| / |traces| = {np.linalg.norm(r) / np.linalg.norm(tr0):.2e}; "
          f"data-mode gradient differs from the residual-mode one by "
          f"{np.abs(g_data - g).max() / gmax:.2e} of max |g|")
    m = 1.0 / w.vel_start.astype(np.float64) ** 2
    # 8 seeded cells where this shot's gradient is not negligible: within 40
    # cells of the source laterally and 60 cells below the receiver plane
    rng = np.random.default_rng(11)
    lo = [sk, max(0, sj - 40), max(0, si - 40)]
    hi = [min(w.nz, sk + 60), min(w.ny, sj + 41), min(w.nx, si + 41)]
    cells = [tuple(int(x) for x in rng.integers(lo, hi)) for _ in range(8)]

    def misfit(mm):
        tr = oracle.run(1.0 / np.sqrt(mm), w.h, w.dt, w.nt, sources=shot, receivers=rec,
                        sponge=w.sponge)["traces"]
        return 0.5 * np.sum((tr - d_obs) ** 2)

    for c in cells:
        eps = 1e-4 * m[c]
        mp, mm = m.copy(), m.copy()
        mp[c] += eps
        mm[c] -= eps
        fd = (misfit(mp) - misfit(mm)) / (2 * eps)
        print(f"cell {c}: GPU adjoint {g[c]:.6e} (from FP32 traces {g_data[c]:.6e})  oracle FD "
              f"{fd:.6e}  |diff| / max|g| = {abs(fd - g[c]) / gmax:.2e}")
        assert abs(fd - g[c]) <= 1e-3 * gmax
