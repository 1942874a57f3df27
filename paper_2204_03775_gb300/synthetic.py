"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle runs.

This module only builds inputs (velocity models, cell positions, time-step
sizes, sizes of grids); it holds none of the stepper's arithmetic, and it
imports neither the CUDA binding nor the oracle. The same arrays are fed to
both sides.

Workloads (shapes and value ranges of the paper's setting: synthetic grids of
hundreds to a thousand cells per axis, 1000 steps, Section IV):

* ``homogeneous_cube`` -- 64^3, h = 10 m, v = 2000 m/s, dt at CFL 0.4,
  100 steps, 15 Hz Ricker at the centre, 16 receivers (4 x 4) on the top plane,
  no damping.
* ``layered_model`` -- 10 horizontal layers of equal thickness, layer l at
  1500 + l * 3000 / 9 m/s, times (1 + 0.05 n) with n a smooth noise field in
  [-1, 1], clipped to [1500, 4500] m/s. n is seeded N(0, 1) noise on a coarse
  grid of spacing 8 cells, Gaussian-filtered (sigma = 1 coarse cell, i.e.
  8 fine cells) and trilinearly interpolated to the grid.
* ``layered_survey`` -- the layered model with a 20-cell absorbing layer on
  every face, dt at CFL 0.4, one 10 Hz Ricker at (nx/2, ny/2, 20) and a
  32 x 32 receiver grid on the plane k = 20; 1024^3 and 1000 steps is the
  benchmark's workload, smaller sizes are parity cases.
* ``adjoint_survey`` -- gradient workload: the layered model as the start
  (background) model, the true model the background times
  1 + 0.1 exp(-|x - c|^2 / (2 s^2)) (a +10% Gaussian blob, s = 12 cells,
  centre c drawn from the seed: 20 to 40 cells below the plane k = 20 and
  laterally inside the middle half), a 4 x 4 grid of 10 Hz Ricker shots and
  a 128 x 128 receiver grid on the plane k = 20, a 20-cell absorbing layer,
  dt at CFL 0.4 of the faster (true) model; 256^3 with 800 steps is the
  full size.
* ``batched_shots`` -- 64 independent shots on grids whose sizes are drawn
  from the seed (nx, ny uniform in [96, 320], nz in [96, 256]), each with
  its own smooth random model in [1500, 4500] m/s (``smooth_random_velocity``,
  seeded per shot), a 16-cell absorbing layer, dt at CFL 0.4 of 4500 m/s, one
  Ricker source (f0 uniform in [8, 20] Hz) at a random cell of the upper
  quarter and an 8 x 8 receiver grid on the plane k = 16; 500 steps each.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

CFL = 0.4


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    dt: float
    nt: int
    vel: np.ndarray                      # [nz][ny][nx] float32, m/s
    sources: list = field(default_factory=list)   # (i, j, k, f0, t0, amp)
    receivers: np.ndarray = None         # [nrec][3] int32 (i, j, k)
    sponge: tuple = (0, 0.0)             # (nb, a)

    @property
    def points(self) -> int:
        return self.nx * self.ny * self.nz


def cfl_dt(vmax: float, h: float, cfl: float = CFL) -> float:
    """Time step with vmax * dt / h = cfl."""
    return cfl * h / float(vmax)


def homogeneous_cube(n: int = 64, nt: int = 100, h: float = 10.0, v: float = 2000.0,
                     f0: float = 15.0) -> Workload:
    vel = np.full((n, n, n), v, dtype=np.float32)
    c = n // 2
    rec = np.array([[int((p + 0.5) * n / 4), int((q + 0.5) * n / 4), 0]
                    for q in range(4) for p in range(4)], dtype=np.int32)
    return Workload("homogeneous_cube", n, n, n, h, cfl_dt(v, h), nt, vel,
                    sources=[(c, c, c, f0, 1.0 / f0, 1.0)], receivers=rec, sponge=(0, 0.0))


def smooth_noise(shape, seed: int, spacing: int = 8) -> np.ndarray:
    """Smooth field in [-1, 1]: coarse Gaussian-filtered noise, trilinear upsampling."""
    import torch
    from scipy.ndimage import gaussian_filter

    nz, ny, nx = shape
    cshape = tuple(max(2, -(-n // spacing) + 1) for n in (nz, ny, nx))
    rng = np.random.Generator(np.random.PCG64(seed))
    coarse = gaussian_filter(rng.standard_normal(cshape), sigma=1.0, mode="wrap")
    coarse /= np.abs(coarse).max()
    t = torch.from_numpy(coarse.astype(np.float32))[None, None]
    # coarse node c sits at fine cell c * spacing; sample the fine grid inside
    size = tuple((m - 1) * spacing + 1 for m in cshape)
    fine = torch.nn.functional.interpolate(t, size=size, mode="trilinear", align_corners=True)
    return fine[0, 0, :nz, :ny, :nx].contiguous().numpy()


def layered_model(nx: int, ny: int, nz: int, seed: int = 2204, layers: int = 10,
                  vmin: float = 1500.0, vmax: float = 4500.0, noise: float = 0.05) -> np.ndarray:
    k = np.arange(nz)
    layer = np.minimum(k * layers // nz, layers - 1)
    base = (vmin + layer * (vmax - vmin) / (layers - 1)).astype(np.float32)
    n = smooth_noise((nz, ny, nx), seed)
    vel = n
    vel *= np.float32(noise)
    vel += np.float32(1.0)
    vel *= base[:, None, None]
    np.clip(vel, vmin, vmax, out=vel)
    return vel


def surface_receivers(nx: int, ny: int, k: int, side: int, margin: int) -> np.ndarray:
    """side x side grid on plane k, evenly spread inside [margin, n - margin)."""
    ii = [margin + int((p + 0.5) * (nx - 2 * margin) / side) for p in range(side)]
    jj = [margin + int((q + 0.5) * (ny - 2 * margin) / side) for q in range(side)]
    return np.array([[i, j, k] for j in jj for i in ii], dtype=np.int32)


def layered_survey(nx: int = 1024, ny: int = 1024, nz: int = 1024, nt: int = 1000,
                   h: float = 10.0, nb: int = 20, a: float = 0.015, f0: float = 10.0,
                   side: int = 32, seed: int = 2204) -> Workload:
    vel = layered_model(nx, ny, nz, seed=seed)
    dt = cfl_dt(float(vel.max()), h)
    src = [(nx // 2, ny // 2, min(nb, nz - 1), f0, 1.0 / f0, 1.0)]
    rec = surface_receivers(nx, ny, min(nb, nz - 1), min(side, nx, ny), min(nb, nx // 4, ny // 4))
    return Workload(f"layered_survey_{nx}x{ny}x{nz}", nx, ny, nz, h, dt, nt, vel,
                    sources=src, receivers=rec, sponge=(nb, a))


def smooth_random_velocity(shape, seed: int, vmin: float = 1500.0, vmax: float = 4500.0,
                           spacing: int = 4) -> np.ndarray:
    """Smooth random model spanning [vmin, vmax] (per-test or per-shot models)."""
    n = smooth_noise(shape, seed, spacing=spacing)
    v = 0.5 * (vmin + vmax) + 0.5 * (vmax - vmin) * n
    return np.clip(v, vmin, vmax).astype(np.float32)


@dataclass
class AdjointSurvey:
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    dt: float
    nt: int
    vel_true: np.ndarray                 # [nz][ny][nx] float32, m/s
    vel_start: np.ndarray                # the background model
    shots: list                          # per shot: a list of (i, j, k, f0, t0, amp)
    receivers: np.ndarray                # [nrec][3] int32, shared by every shot
    sponge: tuple = (20, 0.015)


def adjoint_survey(n: int = 256, nt: int = 800, shots_side: int = 4, rec_side: int = 128,
                   h: float = 10.0, nb: int = 20, a: float = 0.015, f0: float = 10.0,
                   seed: int = 2204) -> AdjointSurvey:
    bg = layered_model(n, n, n, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    # blob centre (k, j, i): laterally in the middle half, 20 to 40 cells below
    # the shot/receiver plane, so its reflections reach the receivers within
    # the 800 steps (deeper, they would arrive after the recording ends)
    plane = min(nb, n - 1)
    c = np.array([rng.uniform(plane + 20, plane + 40), *rng.uniform(n / 4, 3 * n / 4, 2)])
    s = 12.0
    k, j, i = np.ogrid[:n, :n, :n]
    r2 = (k - c[0]) ** 2 + (j - c[1]) ** 2 + (i - c[2]) ** 2
    true = (bg * (1.0 + 0.1 * np.exp(-r2 / (2.0 * s * s)))).astype(np.float32)
    dt = cfl_dt(float(true.max()), h)
    margin = min(nb, n // 4)
    side = min(rec_side, n - 2 * margin)
    rec = surface_receivers(n, n, plane, side, margin)
    pos = surface_receivers(n, n, plane, shots_side, margin)
    shots = [[(int(p[0]), int(p[1]), int(p[2]), f0, 1.0 / f0, 1.0)] for p in pos]
    return AdjointSurvey(f"adjoint_survey_{n}^3", n, n, n, h, dt, nt, true, bg, shots, rec,
                         sponge=(nb, a))


def batched_shots(nshots: int = 64, nt: int = 500, lo=(96, 96, 96), hi=(320, 320, 256),
                  h: float = 10.0, nb: int = 16, a: float = 0.02, seed: int = 2204) -> list:
    """Workloads of independent shots on uneven grids (sizes (nx, ny, nz) in [lo, hi])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dt = cfl_dt(4500.0, h)
    out = []
    for q in range(nshots):
        nx, ny, nz = (int(rng.integers(lo[d], hi[d] + 1)) for d in range(3))
        vel = smooth_random_velocity((nz, ny, nx), seed + 1000 + q, spacing=8)
        plane = min(nb, nz - 1)
        src = [(int(rng.integers(nb, nx - nb)), int(rng.integers(nb, ny - nb)),
                int(rng.integers(plane, max(plane + 1, nz // 4))), float(rng.uniform(8.0, 20.0)),
                0.1, 1.0)]
        rec = surface_receivers(nx, ny, plane, 8, nb)
        out.append(Workload(f"shot{q}_{nx}x{ny}x{nz}", nx, ny, nz, h, dt, nt, vel, sources=src,
                            receivers=rec, sponge=(nb, a)))
    return out
