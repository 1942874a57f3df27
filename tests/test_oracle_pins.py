"""Pins of the FP64 oracle against facts the mathematics fixes.

No test here re-types the oracle's formula and compares it with itself: each
one checks the oracle against something independent of its code -- a
published table, an exact polynomial derivative, a convergence rate, the exact
discrete dispersion relation, a conserved energy, reciprocity, cube symmetry,
a Kronecker-product brute force built another way, or the continuum Green's
function -- and is chosen so that a plausible slip (a dropped term, a wrong
sign or axis, a transposed operand) fails at least one of them. A few tests
plant such slips in the oracle's inputs and check that the pins notice.
"""

import os
from fractions import Fraction
from itertools import permutations, product

import numpy as np
import pytest
import scipy.sparse as sp

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _published_coefficients():
    out = {}
    with open(os.path.join(GOLDEN, "fd8_second_derivative.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            m, frac = line.split()
            out[int(m)] = Fraction(frac)
    return [out[m] for m in range(5)]


# --------------------------------------------------------------------------
# Coefficients of the 25-point formula (Section II)
# --------------------------------------------------------------------------

def test_coefficients_equal_published_table():
    assert oracle.fd8_coefficients() == _published_coefficients()


def test_coefficients_order_is_exactly_eight():
    """1D stencil is exact on x^p for p <= 9 and first fails at p = 10.

    (Odd powers are reproduced for every p, by the stencil's symmetry.)
    """
    c = oracle.fd8_coefficients()
    for p in range(0, 12):
        # second difference of x^p at x = 0 with h = 1, exact rationals
        approx = c[0] * (0 ** p) + sum(c[m] * (Fraction(m) ** p + Fraction(-m) ** p)
                                       for m in range(1, 5))
        exact = 2 if p == 2 else 0
        if p <= 9 or p % 2 == 1:
            assert approx == exact, p
        else:
            assert approx != exact, p
    # truncation term: sum_m (m^10 + (-m)^10) c_m, a closed number of the scheme
    assert sum(2 * c[m] * m ** 10 for m in range(1, 5)) == -1152


# --------------------------------------------------------------------------
# Laplacian
# --------------------------------------------------------------------------

def _poly_grid(nx, ny, nz, h, origin):
    """Coordinates of the padded grid (halo included)."""
    H = oracle.HALO
    x = origin[0] + h * np.arange(-H, nx + H)
    y = origin[1] + h * np.arange(-H, ny + H)
    z = origin[2] + h * np.arange(-H, nz + H)
    return x, y, z


@pytest.mark.parametrize("degs", [(9, 0, 0), (0, 9, 0), (0, 0, 9), (9, 9, 9), (4, 7, 2)])
def test_laplacian_exact_on_polynomials(degs):
    rng = np.random.default_rng(11)
    nx, ny, nz, h = 7, 6, 5, 0.125
    x, y, z = _poly_grid(nx, ny, nz, h, origin=(-0.4, 0.3, -0.2))
    px = np.polynomial.Polynomial(rng.uniform(-1, 1, degs[0] + 1))
    py = np.polynomial.Polynomial(rng.uniform(-1, 1, degs[1] + 1))
    pz = np.polynomial.Polynomial(rng.uniform(-1, 1, degs[2] + 1))
    X, Y, Z = px(x), py(y), pz(z)
    u = Z[:, None, None] * Y[None, :, None] * X[None, None, :]
    H = oracle.HALO
    sl = (slice(H, H + nz), slice(H, H + ny), slice(H, H + nx))
    exact = (pz(z)[:, None, None] * py(y)[None, :, None] * px.deriv(2)(x)[None, None, :]
             + pz(z)[:, None, None] * py.deriv(2)(y)[None, :, None] * px(x)[None, None, :]
             + pz.deriv(2)(z)[:, None, None] * py(y)[None, :, None] * px(x)[None, None, :])[sl]
    got = oracle.laplacian(u, h)
    scale = np.abs(u).max() / h ** 2
    assert np.abs(got - exact).max() <= 1e-11 * scale


def test_laplacian_not_exact_for_degree_ten():
    nx, ny, nz, h = 6, 5, 5, 0.25
    x, y, z = _poly_grid(nx, ny, nz, h, origin=(0.0, 0.0, 0.0))
    u = np.broadcast_to((x ** 10)[None, None, :], (nz + 8, ny + 8, nx + 8)).copy()
    H = oracle.HALO
    got = oracle.laplacian(u, h)
    exact = 90 * x[H:H + nx] ** 8
    err = got[0, 0, :] - exact
    # the leading error term of the 8th-order difference is -1152 h^8 / 2 * ... : nonzero
    assert np.abs(err).max() > 1e-6


def _plane_wave_error(n, modes):
    L = 1.0
    h = L / n
    coords = h * np.arange(n)
    kx, ky, kz = (2 * np.pi * m / L for m in modes)
    u = np.sin(kz * coords[:, None, None] + ky * coords[None, :, None] + kx * coords[None, None, :])
    up = oracle.fill_halo(oracle.pad(u), periodic=True)
    lap = oracle.laplacian(up, h)
    return np.abs(lap + (kx ** 2 + ky ** 2 + kz ** 2) * u).max() / (kx ** 2 + ky ** 2 + kz ** 2)


def test_laplacian_eighth_order_convergence():
    ns = [20, 28, 40, 56]
    errs = [_plane_wave_error(n, (1, 2, 1)) for n in ns]
    slope = np.polyfit(np.log(1.0 / np.array(ns)), np.log(errs), 1)[0]
    assert 7.7 <= slope <= 8.3, (slope, errs)


def test_planted_wrong_coefficient_breaks_convergence():
    c = oracle.coefficients_f64().copy()
    c[3] *= -1.0  # a sign slip in one weight
    nx = ny = nz = 6
    h = 0.5
    x, y, z = _poly_grid(nx, ny, nz, h, origin=(0.1, 0.2, 0.3))
    u = np.broadcast_to((x ** 4)[None, None, :], (nz + 8, ny + 8, nx + 8)).copy()
    got = oracle.laplacian(u, h, coeffs=c)
    exact = 12 * x[4:4 + nx] ** 2
    assert np.abs(got[0, 0] - exact).max() > 1e-3


# --------------------------------------------------------------------------
# Stepper (Algorithm 1, Eq. 2)
# --------------------------------------------------------------------------

def _discrete_eigenvalue(kvec, h):
    c = oracle.coefficients_f64()
    return sum(c[0] + 2 * sum(c[m] * np.cos(m * k * h) for m in range(1, 5)) for k in kvec) / h ** 2


def test_exact_discrete_mode():
    """u^n = cos(n theta) sin(k.x) with cos(theta) = 1 + (v dt)^2 lambda_h / 2.

    lambda_h is the eigenvalue of the discrete Laplacian on sin(k.x) (periodic
    grid); the leapfrog recurrence of Eq. 2 then reproduces the mode exactly.
    """
    nx, ny, nz, h = 16, 12, 10, 10.0
    v, dt = 2000.0, 1.5e-3
    modes = (3, 2, 1)
    kvec = [2 * np.pi * m / (n * h) for m, n in zip(modes, (nx, ny, nz))]
    lam = _discrete_eigenvalue(kvec, h)
    theta = np.arccos(1 + 0.5 * (v * dt) ** 2 * lam)
    x, y, z = (h * np.arange(n) for n in (nx, ny, nz))
    s = np.sin(kvec[2] * z[:, None, None] + kvec[1] * y[None, :, None] + kvec[0] * x[None, None, :])
    vel = np.full((nz, ny, nx), v)
    nt = 60
    out = oracle.run(vel, h, dt, nt, u_init=s, uprev_init=np.cos(theta) * s, periodic=True)
    assert np.abs(out["u"] - np.cos(nt * theta) * s).max() < 1e-11
    assert np.abs(out["u_prev"] - np.cos((nt - 1) * theta) * s).max() < 1e-11


def _smooth_random(shape, rng, sigma=1.5):
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(rng.standard_normal(shape), sigma)


def _kron_laplacian(nx, ny, nz, h):
    """Laplacian as a sparse matrix, assembled from 1D banded operators.

    Flattened index k*ny*nx + j*nx + i (x fastest). Zero-Dirichlet outside.
    Built independently of the oracle's loops: Kronecker sums of 1D matrices.
    """
    c = [float(q) for q in _published_coefficients()]

    def d2(n):
        diags = [np.full(n - abs(o), c[abs(o)]) for o in range(-4, 5) if n - abs(o) > 0]
        offs = [o for o in range(-4, 5) if n - abs(o) > 0]
        return sp.diags(diags, offs, shape=(n, n), format="csr")

    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    A = (sp.kron(Iz, sp.kron(Iy, d2(nx))) + sp.kron(Iz, sp.kron(d2(ny), Ix))
         + sp.kron(d2(nz), sp.kron(Iy, Ix)))
    return (A / h ** 2).tocsr()


def test_energy_conserved_without_damping():
    """E^{n+1/2} = sum (u^{n+1}-u^n)^2 / (v dt)^2 - sum u^{n+1} L u^n is constant.

    Multiplying the recurrence M (u^{n+1} - 2u^n + u^{n-1}) = L u^n, M =
    1/(v dt)^2, by u^{n+1} - u^{n-1} telescopes for symmetric L. L is applied
    here through the independently assembled Kronecker matrix.
    """
    rng = np.random.default_rng(5)
    nx, ny, nz, h, dt = 12, 10, 9, 10.0, 1.0e-3
    vel = 2000.0 + 800.0 * np.tanh(_smooth_random((nz, ny, nx), rng))
    assert vel.max() * dt / h < 0.45
    u0 = _smooth_random((nz, ny, nx), rng)
    um1 = u0 + 0.01 * _smooth_random((nz, ny, nx), rng)
    A = _kron_laplacian(nx, ny, nz, h)
    w = (vel * dt).ravel() ** 2
    energies = []
    cur, prev = u0, um1
    for n in range(30):
        out = oracle.run(vel, h, dt, 1, u_init=cur, uprev_init=prev, n0=n)
        nxt = out["u"]
        e = np.sum((nxt - cur).ravel() ** 2 / w) - nxt.ravel() @ (A @ cur.ravel())
        energies.append(e)
        prev, cur = cur, nxt
    energies = np.array(energies)
    assert np.abs(energies - energies[0]).max() <= 1e-10 * abs(energies[0])


def test_planted_sign_slip_breaks_energy():
    """A wrong-sign Laplacian weight set (all negated) is unstable: energy drifts."""
    rng = np.random.default_rng(6)
    nx, ny, nz, h, dt = 10, 9, 8, 10.0, 1.0e-3
    vel = np.full((nz, ny, nx), 2000.0)
    u0 = _smooth_random((nz, ny, nx), rng)
    out = oracle.run(vel, h, dt, 40, u_init=u0, uprev_init=u0, coeffs=-oracle.coefficients_f64())
    assert np.abs(out["u"]).max() > 1e3 * np.abs(u0).max()


@pytest.mark.parametrize("sponge", [(0, 0.0), (3, 0.12)])
def test_reciprocity(sponge):
    """Source at a, receiver at b equals source at b, receiver at a.

    The recurrence is M D2 u = L u + delta_s f with symmetric M and L, so its
    Green's function is symmetric. With the absorbing taper on, the same holds
    for source and receiver cells outside the taper (g = 1 there).
    """
    rng = np.random.default_rng(7)
    nx, ny, nz, h, dt = 18, 16, 14, 10.0, 1.0e-3
    vel = 2500.0 + 900.0 * np.tanh(_smooth_random((nz, ny, nx), rng, 2.0))
    a, b = (5, 6, 4), (12, 9, 10)
    src = lambda p: [(p[0], p[1], p[2], 25.0, 0.04, 1.0)]
    ab = oracle.run(vel, h, dt, 120, sources=src(a), receivers=[b], sponge=sponge)["traces"][0]
    ba = oracle.run(vel, h, dt, 120, sources=src(b), receivers=[a], sponge=sponge)["traces"][0]
    assert np.abs(ab).max() > 0
    assert np.abs(ab - ba).max() <= 1e-12 * np.abs(ab).max()


def test_planted_source_scaling_breaks_reciprocity():
    """Injecting dt^2 f (no per-cell v^2) is not reciprocal in a variable medium."""
    rng = np.random.default_rng(8)
    nx, ny, nz, h, dt = 14, 13, 12, 10.0, 1.0e-3
    vel = 2500.0 + 900.0 * np.tanh(_smooth_random((nz, ny, nx), rng, 2.0))
    a, b = (4, 5, 3), (9, 8, 8)

    def trace(s, r):
        # planted slip: source amplitude divided by the local v^2, i.e. dt^2 f only
        amp = 1.0 / vel[s[2], s[1], s[0]] ** 2
        return oracle.run(vel, h, dt, 100, sources=[(*s, 25.0, 0.04, amp)], receivers=[r])["traces"][0]

    ab, ba = trace(a, b), trace(b, a)
    assert np.abs(ab - ba).max() > 1e-3 * np.abs(ab).max()


def test_cube_symmetry():
    """Constant v, centred source, odd cube: the field has all 48 cube symmetries."""
    n, h, dt = 17, 10.0, 2.0e-3
    vel = np.full((n, n, n), 2000.0)
    c = n // 2
    out = oracle.run(vel, h, dt, 30, sources=[(c, c, c, 15.0, 1 / 15.0, 1.0)], sponge=(3, 0.1))
    u = out["u"]
    scale = np.abs(u).max()
    assert scale > 0
    for perm in permutations(range(3)):
        for flips in product([False, True], repeat=3):
            t = np.transpose(u, perm)
            for ax, f in enumerate(flips):
                if f:
                    t = np.flip(t, ax)
            assert np.abs(t - u).max() <= 1e-13 * scale


def test_bruteforce_kronecker_matches_oracle():
    """Whole run against a Kronecker-matrix stepper on non-cubic tiny grids.

    The brute force applies the absorbing layer in Cerjan's two-level form
    (plain step, then multiply the new and the current level by g), which the
    oracle's one-pass form must equal.
    """
    rng = np.random.default_rng(9)
    for (nx, ny, nz) in [(8, 8, 8), (5, 7, 9), (9, 4, 6)]:
        h, dt = 10.0, 1.0e-3
        vel = 2200.0 + 700.0 * np.tanh(rng.standard_normal((nz, ny, nx)))
        nb, a = 2, 0.3
        sources = [(nx // 2, ny // 2, nz // 2, 30.0, 0.03, 1.5), (1, ny - 2, 2, 20.0, 0.05, -0.7)]
        rec = np.array([[0, 0, 0], [nx - 1, ny // 3, nz - 1], [nx // 2, ny // 2, nz // 2]])
        nt = 25
        got = oracle.run(vel, h, dt, nt, sources=sources, receivers=rec, sponge=(nb, a))

        A = _kron_laplacian(nx, ny, nz, h)
        w = (vel * dt).ravel() ** 2

        def prof(n):
            d = np.minimum(np.arange(n), n - 1 - np.arange(n))
            return np.where(d < nb, np.exp(-(a * (nb - d)) ** 2), 1.0)

        g = (prof(nz)[:, None, None] * prof(ny)[None, :, None] * prof(nx)[None, None, :]).ravel()
        flat = lambda i, j, k: (k * ny + j) * nx + i
        cur = np.zeros(nx * ny * nz)
        prev = np.zeros(nx * ny * nz)
        traces = np.zeros((len(rec), nt))
        for n in range(nt):
            new = 2 * cur - prev + w * (A @ cur)
            new *= g
            cur_t = g * cur
            t = n * dt
            for (i, j, k, f0, t0, amp) in sources:
                tau = t - t0
                x = (np.pi * f0 * tau) ** 2
                new[flat(i, j, k)] += w[flat(i, j, k)] * amp * (1 - 2 * x) * np.exp(-x)
            for r, (i, j, k) in enumerate(rec):
                traces[r, n] = new[flat(i, j, k)]
            prev_raw = cur
            prev, cur = cur_t, new
        scale = np.abs(cur).max()
        assert scale > 0
        assert np.abs(got["u"].ravel() - cur).max() <= 1e-12 * scale
        # the oracle returns the previous level before its taper is applied
        assert np.abs(got["u_prev"].ravel() - prev_raw).max() <= 1e-12 * scale
        assert np.abs(got["traces"] - traces).max() <= 1e-12 * np.abs(traces).max()


def test_window_equals_full_grid_inside_light_cone():
    """A window run matches the full-grid run where the field cannot reach its inner faces."""
    rng = np.random.default_rng(10)
    nx, ny, nz, h, dt = 60, 56, 30, 10.0, 1.5e-3
    vel = 2000.0 + 500.0 * np.tanh(_smooth_random((nz, ny, nx), rng, 2.0))
    s = (30, 28, 5)
    nt = 5
    src = [(*s, 30.0, 0.0, 1.0)]
    rec = [(30, 28, 6), (34, 30, 9)]
    full = oracle.run(vel, h, dt, nt, sources=src, receivers=rec, sponge=(6, 0.05))
    r = 4 * nt + 1
    ox, oy, oz = s[0] - r, s[1] - r, 0
    wx, wy, wz = 2 * r + 1, 2 * r + 1, s[2] + r + 1
    win = oracle.run(vel[oz:oz + wz, oy:oy + wy, ox:ox + wx], h, dt, nt, sources=src,
                     receivers=rec, sponge=(6, 0.05), window=(ox, oy, oz, nx, ny, nz))
    np.testing.assert_array_equal(win["u"], full["u"][oz:oz + wz, oy:oy + wy, ox:ox + wx])
    np.testing.assert_array_equal(win["traces"], full["traces"])


# --------------------------------------------------------------------------
# Source wavelet and taper
# --------------------------------------------------------------------------

def test_ricker_closed_forms():
    f0, t0, amp = 12.0, 0.1, 2.5
    assert oracle.ricker(t0, f0, t0, amp) == pytest.approx(amp, rel=1e-15)
    tz = 1.0 / (np.pi * f0 * np.sqrt(2.0))            # zero crossings
    assert abs(oracle.ricker(t0 + tz, f0, t0, amp)) < 1e-14
    assert abs(oracle.ricker(t0 - tz, f0, t0, amp)) < 1e-14
    tm = np.sqrt(1.5) / (np.pi * f0)                   # side lobes
    assert oracle.ricker(t0 + tm, f0, t0, amp) == pytest.approx(-2 * amp * np.exp(-1.5), rel=1e-13)
    t = np.linspace(t0 - 1.0, t0 + 1.0, 20001)
    vals = oracle.ricker(t, f0, t0, amp)
    assert abs(np.trapezoid(vals, t)) < 1e-9          # zero mean
    spec = np.abs(np.fft.rfft(vals, 1 << 18))
    freqs = np.fft.rfftfreq(1 << 18, t[1] - t[0])
    assert freqs[np.argmax(spec)] == pytest.approx(f0, rel=2e-3)   # peak frequency f0


def test_cerjan_profile_shape():
    n, nb, a = 50, 20, 0.015
    g = oracle.cerjan(n, nb, a)
    assert np.all(g[nb:n - nb] == 1.0)
    assert np.all(g[:nb] < 1.0) and np.all(g[n - nb:] < 1.0)
    np.testing.assert_array_equal(g, g[::-1])
    assert np.all(np.diff(g[:nb + 1]) > 0)
    assert g[0] == pytest.approx(np.exp(-(a * nb) ** 2), rel=1e-15)
    assert np.all(oracle.cerjan(n, 0, a) == 1.0)


# --------------------------------------------------------------------------
# Physics: continuum Green's function of Eq. 1
# --------------------------------------------------------------------------

@pytest.mark.parametrize("r", [10, 15, 20])
def test_far_field_matches_continuum_greens_function(r):
    """Homogeneous medium: u(r, t) -> h^3 s(t - r/v) / (4 pi r).

    The discrete source adds (v dt)^2 f at one cell, i.e. a Dirac of weight
    h^3 in Eq. 1, whose free-space solution is that retarded spherical wave.
    Dispersion and the grid make it approximate: 5 % in L2 over the window,
    which closes before the boundary reflection arrives.
    """
    n, h, v, f0 = 64, 10.0, 2000.0, 15.0
    dt = 0.4 * h / v
    t0 = 1.0 / f0
    c = n // 2
    vel = np.full((n, n, n), v)
    nt = 100
    out = oracle.run(vel, h, dt, nt, sources=[(c, c, c, f0, t0, 1.0)], receivers=[(c + r, c, c)])
    t = (np.arange(nt) + 1) * dt  # trace sample n is u^{n+1}
    expected = h ** 3 * oracle.ricker(t - r * h / v, f0, t0, 1.0) / (4 * np.pi * r * h)
    got = out["traces"][0]
    err = np.linalg.norm(got - expected) / np.linalg.norm(expected)
    assert err < 0.05, err
