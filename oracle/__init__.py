"""FP64 CPU oracle of the 25-point acoustic wave stepper (arXiv 2204.03775).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package. The CUDA
library and its Python binding never import it, and it imports nothing from
them: the two sides share no code, only the seeded inputs that the tests feed
to both.

What is here:

* :func:`fd8_coefficients` -- the 8th-order central second-derivative weights,
  solved in exact rational arithmetic from the Taylor conditions (the paper
  names the weights c_{xm}, c_{ym}, c_{zm} of its 25-point formula in Section II
  but does not print them);
* :func:`laplacian` -- the 25-point star Laplacian of Section II on a padded
  array whose halo the caller chooses;
* :func:`run` -- Algorithm 1 with the update of Eq. 2, plus the build's
  absorbing taper, Ricker source and receivers (C, FP64, OpenMP over z);
* :func:`ricker`, :func:`cerjan` -- the source wavelet and taper profile.

Each function is pinned by ``tests/test_oracle_pins.py`` against facts the
mathematics fixes (published coefficient table, polynomial exactness, 8th-order
convergence, the exact discrete dispersion relation, energy conservation,
reciprocity, cube symmetry, a Kronecker-product brute force, the continuum
Green's function).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wave_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libwave_oracle.so")

HALO = 4


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.or_num_threads.restype = ctypes.c_int
    lib.or_fill_halo.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.or_laplacian.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, dp]
    lib.or_cerjan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double]
    lib.or_cerjan.restype = ctypes.c_double
    lib.or_ricker.argtypes = [ctypes.c_double] * 4
    lib.or_ricker.restype = ctypes.c_double
    lib.or_run.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp,
        dp, ctypes.c_int, ctypes.c_double,
        ctypes.c_int, ip, dp,
        ctypes.c_int, ip, ctypes.c_int, ctypes.c_longlong,
        dp, dp, ctypes.c_int,
        ip, dp,
        dp, dp, dp]
    lib.or_run.restype = ctypes.c_int
    lib.or_adjoint_gradient.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp,
        dp, ctypes.c_int, ctypes.c_double,
        ctypes.c_int, ip, dp, dp,
        ctypes.c_int, ip, ctypes.c_int, dp,
        dp, dp, dp, dp]
    lib.or_adjoint_gradient.restype = ctypes.c_int
    _lib = lib
    return lib


def num_threads() -> int:
    """OpenMP threads the oracle runs on."""
    return int(_load().or_num_threads())


def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def fd8_coefficients() -> list[Fraction]:
    """Weights c_0..c_4 of the 8th-order central second difference.

    The 25-point formula of Section II sums, per axis, c_m (u(+m) + u(-m)) for
    m = 0..4 with weights it leaves to the solver. Expanding u(+m) + u(-m) in
    Taylor series, the second difference c_0 u + sum_m c_m (u(+m) + u(-m))
    equals h^2 u'' + O(h^10) exactly when

        c_0 + 2 sum_m c_m = 0,   sum_m m^2 c_m = 1,   sum_m m^(2q) c_m = 0 (q = 2, 3, 4).

    The 4x4 system in c_1..c_4 is solved by Gaussian elimination over the
    rationals, so the result is exact.
    """
    n = 4
    rows = [[Fraction(m ** (2 * q)) for m in range(1, n + 1)] + [Fraction(1 if q == 1 else 0)]
            for q in range(1, n + 1)]
    for col in range(n):
        piv = next(r for r in range(col, n) if rows[r][col] != 0)
        rows[col], rows[piv] = rows[piv], rows[col]
        for r in range(n):
            if r != col and rows[r][col] != 0:
                f = rows[r][col] / rows[col][col]
                rows[r] = [a - f * b for a, b in zip(rows[r], rows[col])]
    cm = [rows[r][n] / rows[r][r] for r in range(n)]
    c0 = -2 * sum(cm)
    return [c0] + cm


def coefficients_f64() -> np.ndarray:
    return np.array([float(c) for c in fd8_coefficients()], dtype=np.float64)


def pad(u: np.ndarray) -> np.ndarray:
    """Embed an unpadded [nz][ny][nx] array into a zero 4-cell halo."""
    nz, ny, nx = u.shape
    out = np.zeros((nz + 2 * HALO, ny + 2 * HALO, nx + 2 * HALO), dtype=np.float64)
    out[HALO:HALO + nz, HALO:HALO + ny, HALO:HALO + nx] = u
    return out


def fill_halo(u_padded: np.ndarray, periodic: bool) -> np.ndarray:
    """Zero (Dirichlet) or periodic halo, in place on a padded float64 array."""
    u_padded = np.ascontiguousarray(u_padded, dtype=np.float64)
    nz, ny, nx = (s - 2 * HALO for s in u_padded.shape)
    _load().or_fill_halo(_dptr(u_padded), nx, ny, nz, int(bool(periodic)))
    return u_padded


def laplacian(u_padded: np.ndarray, h: float, coeffs=None) -> np.ndarray:
    """25-point Laplacian (Section II) of a padded [nz+8][ny+8][nx+8] field.

    The halo is used as given (the caller fills it). Returns [nz][ny][nx].
    """
    u_padded = np.ascontiguousarray(u_padded, dtype=np.float64)
    nz, ny, nx = (s - 2 * HALO for s in u_padded.shape)
    c = coefficients_f64() if coeffs is None else np.ascontiguousarray(coeffs, dtype=np.float64)
    out = np.empty((nz, ny, nx), dtype=np.float64)
    _load().or_laplacian(_dptr(u_padded), _dptr(out), nx, ny, nz, float(h), _dptr(c))
    return out


def ricker(t, f0: float, t0: float, amp: float = 1.0):
    """Ricker wavelet used as the source time function f^n of Eq. 2."""
    lib = _load()
    t = np.asarray(t, dtype=np.float64)
    return np.vectorize(lambda x: lib.or_ricker(float(x), f0, t0, amp))(t)


def cerjan(n: int, nb: int, a: float) -> np.ndarray:
    """Absorbing-taper profile of one axis of n cells (1 outside the layer)."""
    lib = _load()
    return np.array([lib.or_cerjan(i, n, nb, a) for i in range(n)], dtype=np.float64)


def run(vel: np.ndarray, h: float, dt: float, nt: int, *,
        sources=(), receivers=None, sponge=(0, 0.0), n0: int = 0,
        u_init=None, uprev_init=None, periodic: bool = False,
        window=None, coeffs=None, source_series=None) -> dict:
    """Algorithm 1 / Eq. 2 for nt steps; see ``or_run`` in wave_oracle.c.

    vel        [nz][ny][nx] velocity of the computed box (float64 copy taken)
    sources    sequence of (i, j, k, f0, t0, amp) in global cells
    receivers  [nrec][3] int array of global (i, j, k)
    sponge     (nb, a) Cerjan width and strength; nb = 0 disables it
    window     None, or (ox, oy, oz, NX, NY, NZ): the box is a window of a
               larger grid (exact while the wavefield stays inside it)
    source_series  None, or [nsrc][nt]: each source's f^n, replacing the Ricker
    Returns dict(traces=[nrec][nt], u=u^{n0+nt}, u_prev=u^{n0+nt-1}).
    """
    vel = np.ascontiguousarray(vel, dtype=np.float64)
    nz, ny, nx = vel.shape
    c = coefficients_f64() if coeffs is None else np.ascontiguousarray(coeffs, dtype=np.float64)
    src = list(sources)
    nsrc = len(src)
    src_ijk = np.ascontiguousarray(np.array([s[:3] for s in src], dtype=np.int32).reshape(nsrc, 3))
    src_par = np.ascontiguousarray(np.array([s[3:] for s in src], dtype=np.float64).reshape(nsrc, 3))
    rec = np.zeros((0, 3), np.int32) if receivers is None else np.asarray(receivers, np.int32)
    rec = np.ascontiguousarray(rec.reshape(-1, 3))
    nrec = rec.shape[0]
    traces = np.zeros((nrec, nt), dtype=np.float64)
    u_out = np.zeros((nz, ny, nx), dtype=np.float64)
    up_out = np.zeros((nz, ny, nx), dtype=np.float64)
    ui = None if u_init is None else np.ascontiguousarray(u_init, dtype=np.float64)
    upi = None if uprev_init is None else np.ascontiguousarray(uprev_init, dtype=np.float64)
    win = None if window is None else np.ascontiguousarray(np.array(window, dtype=np.int32))
    ser = None
    if source_series is not None:
        ser = np.ascontiguousarray(np.asarray(source_series, np.float64).reshape(nsrc, nt))
    rc = _load().or_run(nx, ny, nz, float(h), float(dt), _dptr(c),
                        _dptr(vel), int(sponge[0]), float(sponge[1]),
                        nsrc, _iptr(src_ijk), _dptr(src_par),
                        nrec, _iptr(rec), int(nt), int(n0),
                        _dptr(ui), _dptr(upi), int(bool(periodic)),
                        _iptr(win), _dptr(ser),
                        _dptr(traces), _dptr(u_out), _dptr(up_out))
    if rc != 0:
        raise ValueError("oracle run rejected its arguments")
    return {"traces": traces, "u": u_out, "u_prev": up_out}


def adjoint_gradient(vel: np.ndarray, h: float, dt: float, nt: int, d_obs: np.ndarray, *,
                     sources=(), receivers=None, sponge=(0, 0.0), source_series=None,
                     coeffs=None) -> dict:
    """Misfit 1/2 |traces - d_obs|^2 of a run from rest and its gradient with
    respect to the squared slowness m = 1/V^2 (see or_adjoint_gradient).

    Returns dict(misfit, grad_m [nz][ny][nx], traces [nrec][nt],
    dj_dsrc [nsrc][nt] = dJ/d(source function sample)).
    """
    vel = np.ascontiguousarray(vel, dtype=np.float64)
    nz, ny, nx = vel.shape
    c = coefficients_f64() if coeffs is None else np.ascontiguousarray(coeffs, dtype=np.float64)
    src = list(sources)
    nsrc = len(src)
    src_ijk = np.ascontiguousarray(np.array([s[:3] for s in src], dtype=np.int32).reshape(nsrc, 3))
    src_par = np.ascontiguousarray(np.array([s[3:] for s in src], dtype=np.float64).reshape(nsrc, 3))
    rec = np.ascontiguousarray(np.asarray(receivers, np.int32).reshape(-1, 3))
    nrec = rec.shape[0]
    dob = np.ascontiguousarray(np.asarray(d_obs, np.float64).reshape(nrec, nt))
    ser = None
    if source_series is not None:
        ser = np.ascontiguousarray(np.asarray(source_series, np.float64).reshape(nsrc, nt))
    misfit = ctypes.c_double()
    grad = np.zeros((nz, ny, nx), np.float64)
    traces = np.zeros((nrec, nt), np.float64)
    djds = np.zeros((nsrc, nt), np.float64)
    rc = _load().or_adjoint_gradient(nx, ny, nz, float(h), float(dt), _dptr(c), _dptr(vel),
                                     int(sponge[0]), float(sponge[1]), nsrc, _iptr(src_ijk),
                                     _dptr(src_par), _dptr(ser), nrec, _iptr(rec), int(nt),
                                     _dptr(dob), ctypes.byref(misfit), _dptr(grad),
                                     _dptr(traces), _dptr(djds))
    if rc != 0:
        raise ValueError("oracle adjoint rejected its arguments")
    return {"misfit": misfit.value, "grad_m": grad, "traces": traces, "dj_dsrc": djds}
