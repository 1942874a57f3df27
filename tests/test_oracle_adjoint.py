"""Pins of the oracle's adjoint gradient (FP64, CPU).

The adjoint is the build's extension (the paper has no inversion), so it is
pinned by the facts that define an adjoint rather than by values:
1. dot-product test: for the linear map F from a source's time function to
   the receiver traces, <F s, d> = <s, F^T d>, with F computed by the
   forward stepper and F^T by the adjoint recurrence (two different codes);
2. central finite differences of the misfit with respect to the squared
   slowness of single cells (source cell, receiver cell, taper cell,
   interior cells) equal the adjoint gradient;
3. the misfit it reports equals 1/2 |traces - d_obs|^2 of a forward run.
Planted slips in the model (a missing taper on u^{n-1}) fail the FD check.
"""

import numpy as np
import pytest

import oracle


def _setup(seed=3):
    rng = np.random.default_rng(seed)
    nx, ny, nz, h, dt = 22, 18, 14, 10.0, 1.0e-3
    from scipy.ndimage import gaussian_filter
    vel = 2400.0 + 600.0 * np.tanh(gaussian_filter(rng.standard_normal((nz, ny, nx)), 2.0))
    src = [(8, 9, 4, 30.0, 0.03, 1.0), (15, 6, 9, 22.0, 0.045, -0.6)]
    rec = np.array([[3, 3, 2], [18, 14, 2], [11, 9, 12], [20, 2, 7], [1, 16, 10], [12, 12, 0]],
                   np.int32)
    return nx, ny, nz, h, dt, vel, src, rec


def test_dot_product_source_to_traces():
    nx, ny, nz, h, dt, vel, src, rec = _setup()
    nt = 70
    rng = np.random.default_rng(1)
    s = rng.standard_normal((len(src), nt))
    d = rng.standard_normal((len(rec), nt))
    for sponge in [(0, 0.0), (3, 0.15)]:
        fs = oracle.run(vel, h, dt, nt, sources=src, receivers=rec, sponge=sponge,
                        source_series=s)["traces"]
        adj = oracle.adjoint_gradient(vel, h, dt, nt, -d, sources=src, receivers=rec,
                                      sponge=sponge, source_series=np.zeros_like(s))
        lhs = np.sum(fs * d)
        rhs = np.sum(s * adj["dj_dsrc"])
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs), (lhs, rhs)


def _misfit(vel, h, dt, nt, src, rec, sponge, d_obs):
    tr = oracle.run(vel, h, dt, nt, sources=src, receivers=rec, sponge=sponge)["traces"]
    return 0.5 * np.sum((tr - d_obs) ** 2)


@pytest.mark.parametrize("sponge", [(0, 0.0), (3, 0.15)])
def test_gradient_matches_central_differences(sponge):
    nx, ny, nz, h, dt, vel, src, rec = _setup()
    nt = 60
    # observed data from a perturbed model, so the residual is not zero
    true = vel.copy()
    true[4:9, 6:12, 7:14] *= 1.08
    d_obs = oracle.run(true, h, dt, nt, sources=src, receivers=rec, sponge=sponge)["traces"]
    adj = oracle.adjoint_gradient(vel, h, dt, nt, d_obs, sources=src, receivers=rec,
                                  sponge=sponge)
    assert adj["misfit"] == pytest.approx(_misfit(vel, h, dt, nt, src, rec, sponge, d_obs),
                                          rel=1e-13)
    m = 1.0 / vel ** 2
    rng = np.random.default_rng(2)
    cells = [(4, 9, 8), (9, 12, 11), (2, 3, 3), (0, 1, 1),        # source, receiver, two near faces
             *[tuple(rng.integers([0, 0, 0], [nz, ny, nx])) for _ in range(4)]]
    g = adj["grad_m"]
    scale = np.abs(g).max()
    for (k, j, i) in cells:
        eps = 1e-4 * m[k, j, i]
        mp, mm = m.copy(), m.copy()
        mp[k, j, i] += eps
        mm[k, j, i] -= eps
        fd = (_misfit(1 / np.sqrt(mp), h, dt, nt, src, rec, sponge, d_obs)
              - _misfit(1 / np.sqrt(mm), h, dt, nt, src, rec, sponge, d_obs)) / (2 * eps)
        assert abs(fd - g[k, j, i]) <= 1e-6 * scale + 1e-6 * abs(g[k, j, i]), ((k, j, i), fd, g[k, j, i])


def test_planted_slip_fails_central_differences():
    """Drop the taper from the previous level in the forward model used for the
    finite differences: the adjoint of the true scheme no longer matches."""
    nx, ny, nz, h, dt, vel, src, rec = _setup()
    nt, sponge = 60, (3, 0.15)
    true = vel.copy()
    true[4:9, 6:12, 7:14] *= 1.08
    d_obs = oracle.run(true, h, dt, nt, sources=src, receivers=rec, sponge=sponge)["traces"]
    adj = oracle.adjoint_gradient(vel, h, dt, nt, d_obs, sources=src, receivers=rec,
                                  sponge=sponge)
    # finite differences of a different scheme: no taper at all
    m = 1.0 / vel ** 2
    k, j, i = 1, 2, 2   # inside the taper
    eps = 1e-4 * m[k, j, i]
    mp, mm = m.copy(), m.copy()
    mp[k, j, i] += eps
    mm[k, j, i] -= eps
    fd = (_misfit(1 / np.sqrt(mp), h, dt, nt, src, rec, (0, 0.0), d_obs)
          - _misfit(1 / np.sqrt(mm), h, dt, nt, src, rec, (0, 0.0), d_obs)) / (2 * eps)
    assert abs(fd - adj["grad_m"][k, j, i]) > 1e-3 * np.abs(adj["grad_m"]).max()
