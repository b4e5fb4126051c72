"""Seeded synthetic camera set-ups (the inputs of every test and benchmark).

This module only draws and lists inputs; it holds none of the method's
arithmetic, and both the CUDA path and the CPU oracle read their inputs from
it. The workloads stand in for the paper's own figure set-ups (Sec. 3.2 shadow,
Sec. 4.3 lensing, Sec. 5 disk), which use no dataset.

A render is a dict with keys
  a, r_obs, incl_deg, extent=(x_min, x_max, y_min, y_max), nx, ny,
  mode ("shadow" or "disk"), r_in, r_out (disk only; r_in = "isco" means the
  prograde ISCO of spin a, resolved by whoever traces it), tol,
  cell_deg, cell_phase_deg.
"""
import math

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(seed: int) -> int:
    """One output of the SplitMix64 generator (Steele, Lea & Flood 2014) for `seed`."""
    z = (seed + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def checker_phase_deg(seed: int, cell_deg: float = 10.0) -> float:
    """Longitude offset of the seeded celestial checkerboard: cell * u, u in [0, 1)."""
    return cell_deg * (splitmix64(seed) / 2.0 ** 64)


def render(a, r_obs, incl_deg, extent, nx, ny, mode="shadow", r_in=None, r_out=None,
           tol=1e-10, cell_deg=10.0, seed=2202, l0=None, q=None):
    """mode "disk" with l0=None: Keplerian disk; with l0: disk of constant
    specific angular momentum l0. q given: the q-metric (a is ignored)."""
    return dict(a=float(a), r_obs=float(r_obs), incl_deg=float(incl_deg),
                extent=tuple(float(v) for v in extent), nx=int(nx), ny=int(ny), mode=mode,
                r_in=r_in, r_out=r_out, tol=float(tol), cell_deg=float(cell_deg),
                cell_phase_deg=checker_phase_deg(seed, cell_deg),
                l0=None if l0 is None else float(l0), q=None if q is None else float(q))


def schwarzschild_shadow_64():
    """Schwarzschild shadow: a=0, r_obs=1000, 85 deg, 64x64 on [-10,10]^2, tol 1e-10."""
    return render(0.0, 1000.0, 85.0, (-10.0, 10.0, -10.0, 10.0), 64, 64)


KERR_SPINS = (0.0, 0.5, 0.9, 0.998)
KERR_INCLINATIONS = (17.0, 60.0, 90.0)


def kerr_shadow_ring_set(side=1024):
    """Kerr shadow and Einstein ring set: 4 spins x 3 inclinations, r_obs=1000,
    side x side on [-8,8]^2, tol 1e-10, seeded 10-degree checkerboard."""
    return [render(a, 1000.0, inc, (-8.0, 8.0, -8.0, 8.0), side, side)
            for a in KERR_SPINS for inc in KERR_INCLINATIONS]


QMETRIC_QS = (-0.5, 0.1, 0.5)
QMETRIC_INCLINATIONS = (30.0, 90.0)


def qmetric_shadow_set(side=1024):
    """q-metric shadow set (Appendix A): q in {-0.5, 0.1, 0.5} x inclination
    {30, 90} deg, r_obs = 1000, side x side on [-8,8]^2, tol 1e-10."""
    return [render(0.0, 1000.0, inc, (-8.0, 8.0, -8.0, 8.0), side, side, q=q)
            for q in QMETRIC_QS for inc in QMETRIC_INCLINATIONS]


def schwarzschild_disk(side=2048):
    """Thin Keplerian disk around Schwarzschild: r_in=6, r_out=20, 80 deg,
    r_obs=1000, side x side on [-25,25]^2, tol 1e-10."""
    return render(0.0, 1000.0, 80.0, (-25.0, 25.0, -25.0, 25.0), side, side, mode="disk",
                  r_in=6.0, r_out=20.0)


PAPER_DISK_CASES = ((0.0, 2.8), (0.5, 2.8), (0.998, 1.8))


def paper_disk_figure(nx=2048, ny=1024):
    """The thin-disk figure set-up of Sec. 5: a in {0, 0.5, 0.998} with
    l0 = 2.8, 2.8, 1.8, r_obs = 1000, 85 deg, r_in = ISCO(a), r_out = 20,
    x in [-24, 24], y in [-12, 12], 2048 x 1024 pixels."""
    return [render(a, 1000.0, 85.0, (-24.0, 24.0, -12.0, 12.0), nx, ny, mode="disk",
                   r_in="isco", r_out=20.0, l0=l0) for a, l0 in PAPER_DISK_CASES]


def uneven_batch(n=256, seed=4, sides=(128, 256, 512, 1024)):
    """Batched uneven renders: n requests drawn from PCG64(seed). Draw order per
    request: side, a, inclination, r_obs. Even requests are shadow renders on
    [-8,8]^2, odd requests disk renders (r_in = ISCO(a), r_out = 20) on
    [-25,25]^2; tol 1e-10."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for k in range(n):
        side = int(rng.choice(np.asarray(sides)))
        a = float(rng.uniform(0.0, 0.998))
        inc = float(rng.uniform(5.0, 85.0))
        r_obs = float(rng.uniform(500.0, 2000.0))
        if k % 2 == 0:
            reqs.append(render(a, r_obs, inc, (-8.0, 8.0, -8.0, 8.0), side, side))
        else:
            reqs.append(render(a, r_obs, inc, (-25.0, 25.0, -25.0, 25.0), side, side,
                               mode="disk", r_in="isco", r_out=20.0))
    return reqs


def served_stream(rate_hz=50.0, duration_s=60.0, seed=5, side_min=64, side_max=2048):
    """Served render stream: Poisson arrivals from PCG64(seed). Per request the
    draws are: inter-arrival gap, log-uniform side, a, inclination, mode, tol.
    r_obs = 1000. Returns a list of (arrival_time_s, render)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    t = 0.0
    while True:
        t += float(rng.exponential(1.0 / rate_hz))
        if t >= duration_s:
            break
        side = int(round(math.exp(rng.uniform(math.log(side_min), math.log(side_max)))))
        a = float(rng.uniform(0.0, 0.998))
        inc = float(rng.uniform(5.0, 85.0))
        disk = bool(rng.uniform() < 0.5)
        tol = 1e-8 if rng.uniform() < 0.5 else 1e-10
        if disk:
            r = render(a, 1000.0, inc, (-25.0, 25.0, -25.0, 25.0), side, side, mode="disk",
                       r_in="isco", r_out=20.0, tol=tol)
        else:
            r = render(a, 1000.0, inc, (-8.0, 8.0, -8.0, 8.0), side, side, tol=tol)
        out.append((t, r))
    return out
