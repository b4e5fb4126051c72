"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints, closed forms (Bardeen's critical curve moved to finite r0, the
Schwarzschild photon sphere and deflection integral, straight lines in flat
space, Keplerian redshift), invariants of the exact flow (H = 0, Carter
constant), and the Runge-Kutta order conditions. A plausible slip in the
oracle (a dropped term, a wrong sign or index, a transposed operand) fails at
least one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2202_00086_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
R0 = 1000.0


# ---------------------------------------------------------------------------
# Metric (Sec. 4.3): closed-form properties of the Kerr line element
# ---------------------------------------------------------------------------

def _points(seed=0, n=40):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        a = rng.uniform(0.0, 0.999)
        rh = 1.0 + math.sqrt(1.0 - a * a)
        r = rh * 1.05 + rng.uniform(0.0, 30.0)
        th = rng.uniform(0.05, math.pi - 0.05)
        yield a, r, th


def test_metric_closed_forms():
    for a, r, th in _points():
        g = oracle.metric_cov(a, r, th)
        s, c = math.sin(th), math.cos(th)
        Sigma = r * r + a * a * c * c
        # sqrt(-det g) = Sigma sin(theta) for Kerr in Boyer-Lindquist form.
        assert np.linalg.det(g) == pytest.approx(-(Sigma * s) ** 2, rel=1e-11)
        # frame-dragging rate -g_tphi/g_phph = 2 a r / ((r^2+a^2)^2 - a^2 Delta sin^2)
        Delta = r * r - 2 * r + a * a
        omega = 2 * a * r / ((r * r + a * a) ** 2 - a * a * Delta * s * s)
        assert -g[0, 3] / g[3, 3] == pytest.approx(omega, rel=1e-12, abs=1e-300)
        # symmetric, and only (t,phi) mixes
        assert np.allclose(g, g.T, rtol=0, atol=0)
        assert g[0, 1] == g[0, 2] == g[1, 2] == g[1, 3] == g[2, 3] == 0.0
    # Schwarzschild limit
    r, th = 7.3, 1.1
    g = oracle.metric_cov(0.0, r, th)
    expect = np.diag([-(1 - 2 / r), 1 / (1 - 2 / r), r * r, (r * math.sin(th)) ** 2])
    assert np.allclose(g, expect, rtol=1e-15, atol=0)
    # ergosphere: g_tt = 0 at r = 1 + sqrt(1 - a^2 cos^2)
    a, th = 0.9, 0.7
    r_erg = 1 + math.sqrt(1 - (a * math.cos(th)) ** 2)
    assert abs(oracle.metric_cov(a, r_erg, th)[0, 0]) < 1e-14
    # flat space (M = 0): Minkowski in spherical coordinates
    g = oracle.metric_cov(0.0, 5.0, 0.4, M=0.0)
    assert np.allclose(g, np.diag([-1, 1, 25, 25 * math.sin(0.4) ** 2]), rtol=1e-15, atol=0)


def test_inverse_metric_is_inverse():
    for a, r, th in _points(1):
        g = oracle.metric_cov(a, r, th)
        gi = oracle.metric_con(a, r, th)
        assert np.allclose(gi @ g, np.eye(4), rtol=0, atol=1e-12)
    # g^rr vanishes on the horizon
    a = 0.7
    rh = 1 + math.sqrt(1 - a * a)
    assert abs(oracle.metric_con(a, rh, 1.0)[1, 1]) < 1e-15


def _fd(f, x, h):
    # fourth-order central difference
    return (-f(x + 2 * h) + 8 * f(x + h) - 8 * f(x - h) + f(x - 2 * h)) / (12 * h)


def test_inverse_metric_derivatives():
    for a, r, th in _points(2, 25):
        dr, dth = oracle.metric_con_derivs(a, r, th)
        fr = _fd(lambda rr: oracle.metric_con(a, rr, th), r, 1e-3 * r)
        ft = _fd(lambda tt: oracle.metric_con(a, r, tt), th, 1e-3)
        scale_r = np.abs(fr).max()
        scale_t = np.abs(ft).max() + 1e-300
        assert np.abs(dr - fr).max() <= 1e-8 * scale_r
        assert np.abs(dth - ft).max() <= 1e-8 * max(scale_t, 1e-12)


# ---------------------------------------------------------------------------
# Equations of motion (Sec. 2.1): the RHS is the Hamiltonian vector field
# ---------------------------------------------------------------------------

def test_rhs_is_hamiltonian_vector_field():
    rng = np.random.default_rng(3)
    for _ in range(20):
        a = rng.uniform(0, 0.99)
        r = 1.2 * (1 + math.sqrt(1 - a * a)) + rng.uniform(0, 20)
        th = rng.uniform(0.2, math.pi - 0.2)
        y = np.array([0.0, r, th, 0.3, rng.normal(), rng.normal() * 3])
        E, L = rng.uniform(0.5, 1.5), rng.normal() * 4  # off-shell on purpose: H != 0

        def H(yy=y, EE=E, LL=L):
            return oracle.hamiltonian(a, yy, EE, LL)

        def d_state(k, h):
            return _fd(lambda v: H(np.where(np.arange(6) == k, v, y)), y[k], h)

        dy = oracle.rhs(a, y, E, L)
        dH_dE = _fd(lambda v: H(y, v, L), E, 1e-4)
        dH_dL = _fd(lambda v: H(y, E, v), L, 1e-4)
        expect = np.array([
            -dH_dE,                 # t'  = dH/dp_t = -dH/dE
            d_state(4, 1e-4),       # r'  = dH/dp_r
            d_state(5, 1e-4),       # th' = dH/dp_th
            dH_dL,                  # ph' = dH/dp_ph
            -d_state(1, 1e-4 * r),  # p_r'  = -dH/dr
            -d_state(2, 1e-4),      # p_th' = -dH/dth
        ])
        assert np.allclose(dy, expect, rtol=1e-7, atol=1e-9 * np.abs(expect).max())


# ---------------------------------------------------------------------------
# Initial data (Sec. 2.3) against the values the paper prints (Sec. 3.1)
# ---------------------------------------------------------------------------

def _golden_ics():
    with open(os.path.join(GOLDEN, "paper_single_orbit_ics.json")) as f:
        return json.load(f)


def test_printed_initial_conditions():
    gold = _golden_ics()
    a, r0 = gold["spacetime"]["a"], gold["observer"]["r0"]
    for ray in gold["rays"]:
        st = oracle.init_ray(a, r0, 90.0, ray["x"], ray["y"])
        p_t, p_r, p_th, p_ph = -st[6], st[4], st[5], st[7]
        # six printed decimals; p_r printed one unit off in the sixth place
        assert p_t == pytest.approx(ray["p_t"], abs=2e-6)
        assert p_r == pytest.approx(ray["p_r"], abs=2e-6)
        assert p_th == pytest.approx(ray["p_theta"], abs=1e-6)
        assert p_ph == pytest.approx(ray["p_phi"], abs=1e-6)
        assert abs(oracle.hamiltonian(a, st[:6], st[6], st[7])) < 1e-15


def test_initial_data_is_null_everywhere():
    rng = np.random.default_rng(4)
    for _ in range(50):
        a = rng.uniform(0, 0.998)
        inc = rng.uniform(3, 90)
        x, y = rng.uniform(-25, 25, 2)
        st = oracle.init_ray(a, rng.uniform(100, 2000), inc, x, y)
        assert abs(oracle.hamiltonian(a, st[:6], st[6], st[7])) < 1e-14
        assert st[4] < 0  # ingoing


# ---------------------------------------------------------------------------
# Capture flags: Bardeen's critical curve (Sec. 3.2) moved to finite r0
# ---------------------------------------------------------------------------

def _captured_by_radial_potential(a, st):
    """Exact test: the ingoing ray is captured iff R(r) > 0 on [r_H, r0], with
    R = (r^2 + a^2 - a xi)^2 - Delta (eta + (xi - a)^2), xi = L/E,
    eta = Q/E^2, Q the Carter constant."""
    r0, th0, p_th, E, L = st[1], st[2], st[5], st[6], st[7]
    xi = L / E
    eta = (p_th ** 2 + math.cos(th0) ** 2 * (L ** 2 / math.sin(th0) ** 2 - a * a * E * E)) / E ** 2
    # R(r) = r^4 + (a^2 - xi^2 - eta) r^2 + 2 (eta + (xi - a)^2) r - a^2 eta
    coeffs = [1.0, 0.0, a * a - xi * xi - eta, 2.0 * (eta + (xi - a) ** 2), -a * a * eta]
    rh = 1 + math.sqrt(1 - a * a)
    roots = np.roots(coeffs)
    real = [z.real for z in roots if abs(z.imag) < 1e-7 * max(1.0, abs(z))]
    return not any(rh < z < r0 for z in real)


def _band_mask(flags):
    """True where the 3x3 neighbourhood of a pixel has mixed flags."""
    f = flags.astype(int)
    ny, nx = f.shape
    pad = np.pad(f, 1, mode="edge")
    lo = np.full_like(f, 2)
    hi = np.full_like(f, -1)
    for dj in range(3):
        for di in range(3):
            w = pad[dj:dj + ny, di:di + nx]
            lo = np.minimum(lo, w)
            hi = np.maximum(hi, w)
    return lo != hi


@pytest.mark.parametrize("a,inc", [(0.0, 60.0), (0.5, 17.0), (0.9, 90.0), (0.998, 60.0),
                                   (0.998, 90.0)])
def test_capture_flags_match_critical_curve(a, inc):
    n = 24
    ext = (-8.0, 8.0, -8.0, 8.0)
    res = oracle.trace_pixels(a, R0, inc, ext, n, n)
    flags = np.zeros((n, n), bool)
    for j in range(n):
        for i in range(n):
            x = ext[0] + (i + 0.5) * (ext[1] - ext[0]) / n
            y = ext[2] + (j + 0.5) * (ext[3] - ext[2]) / n
            flags[j, i] = _captured_by_radial_potential(a, oracle.init_ray(a, R0, inc, x, y))
    got = (res["status"] == oracle.STATUS_CAPTURED).reshape(n, n)
    assert set(np.unique(res["status"])) <= {oracle.STATUS_CAPTURED, oracle.STATUS_ESCAPED}
    keep = ~_band_mask(flags)
    assert keep.sum() > 0.6 * n * n
    assert np.array_equal(got[keep], flags[keep])


def test_worked_orbits_fates():
    """The two printed initial conditions (Sec. 3.1) end as the equations say."""
    gold = _golden_ics()
    a, r0 = gold["spacetime"]["a"], gold["observer"]["r0"]
    for ray in gold["rays"]:
        st = oracle.init_ray(a, r0, 90.0, ray["x"], ray["y"])
        captured = _captured_by_radial_potential(a, st)
        assert captured == (ray["fate_from_equations"] == "captured")
        res = oracle.trace_states(a, r0, st[None, :6], [st[6]], [st[7]])
        want = oracle.STATUS_CAPTURED if captured else oracle.STATUS_ESCAPED
        assert res["status"][0] == want


def test_schwarzschild_shadow_radius():
    """Config 'Schwarzschild shadow 64x64': captured iff rho < 3 sqrt(3) sqrt(1 - 2/r0)."""
    cam = workloads.schwarzschild_shadow_64()
    n = cam["nx"]
    res = oracle.trace_pixels(cam["a"], cam["r_obs"], cam["incl_deg"], cam["extent"], n, n,
                              tol=cam["tol"])
    x0, x1, y0, y1 = cam["extent"]
    xs = x0 + (np.arange(n) + 0.5) * (x1 - x0) / n
    ys = y0 + (np.arange(n) + 0.5) * (y1 - y0) / n
    rho = np.hypot(xs[None, :], ys[:, None])
    rho_c = 3 * math.sqrt(3) * math.sqrt(1 - 2 / cam["r_obs"])
    expect = rho < rho_c
    got = (res["status"] == oracle.STATUS_CAPTURED).reshape(n, n)
    keep = ~_band_mask(expect)
    assert np.array_equal(got[keep], expect[keep])
    # terminal surfaces located by bisection
    cap = res["status"] == oracle.STATUS_CAPTURED
    esc = res["status"] == oracle.STATUS_ESCAPED
    assert np.allclose(res["r"][cap], 1.01 * 2.0, rtol=1e-12)
    assert np.allclose(res["r"][esc], 1.1 * cam["r_obs"], rtol=1e-12)


def test_schwarzschild_critical_impact_parameter():
    """Bisection in rho on the oracle converges to 3 sqrt(3) sqrt(1 - 2/r0)."""
    inc = 85.0
    lo, hi = 5.0, 5.4
    for _ in range(24):
        mid = 0.5 * (lo + hi)
        st = oracle.init_ray(0.0, R0, inc, -mid, 0.0)
        res = oracle.trace_states(0.0, R0, st[None, :6], [st[6]], [st[7]])
        if res["status"][0] == oracle.STATUS_CAPTURED:
            lo = mid
        else:
            hi = mid
    assert 0.5 * (lo + hi) == pytest.approx(3 * math.sqrt(3) * math.sqrt(1 - 2 / R0), abs=2e-6)


# ---------------------------------------------------------------------------
# Photon sphere and deflection (Schwarzschild), straight lines (flat space)
# ---------------------------------------------------------------------------

def test_photon_sphere_orbit():
    """r = 3, p_r = 0, b = 3 sqrt(3): a circular photon orbit with dphi/dt = 1/(3 sqrt 3)."""
    b = 3 * math.sqrt(3)
    st = np.array([[0.0, 3.0, math.pi / 2, 0.0, 0.0, 0.0]])
    res = oracle.trace_states(0.0, R0, st, [1.0], [b], max_steps=60)
    assert res["status"][0] == oracle.STATUS_MAXSTEP
    assert res["r"][0] == pytest.approx(3.0, abs=1e-8)
    assert res["phi"][0] / res["t"][0] == pytest.approx(1 / b, rel=1e-9)
    assert res["t"][0] > 20.0


def spherical_photon_orbit(a, f):
    """A Kerr spherical photon orbit (Teo 2003): radius r a fraction f of the
    way from the prograde to the retrograde equatorial photon orbit
    r_ph = 2 (1 + cos(2/3 arccos(-+a))); with E = 1 its constants are
    xi = L/E = -(r^3 - 3 r^2 + a^2 r + a^2) / (a (r - 1)),
    eta = Q/E^2 = -r^3 (r^3 - 6 r^2 + 9 r - 4 a^2) / (a^2 (r - 1)^2),
    for which the radial potential and its derivative vanish at r. Returns
    (r, xi, eta, u_plus) with u_plus = cos^2 of the theta turning points."""
    r_pro = 2 * (1 + math.cos(2 / 3 * math.acos(-a)))
    r_retro = 2 * (1 + math.cos(2 / 3 * math.acos(a)))
    r = r_pro + f * (r_retro - r_pro)
    xi = -(r ** 3 - 3 * r ** 2 + a * a * r + a * a) / (a * (r - 1))
    eta = -r ** 3 * (r ** 3 - 6 * r ** 2 + 9 * r - 4 * a * a) / (a * a * (r - 1) ** 2)
    b = eta + xi * xi - a * a
    u_plus = (-b + math.sqrt(b * b + 4 * a * a * eta)) / (2 * a * a)
    return r, xi, eta, u_plus


@pytest.mark.parametrize("a", [0.5, 0.9, 0.998])
@pytest.mark.parametrize("f", [0.25, 0.5, 0.75])
def test_kerr_spherical_photon_orbits(a, f):
    """Started on the equator with p_r = 0 and p_theta = sqrt(eta), a photon
    with the spherical-orbit constants keeps r fixed (the frame-dragging terms
    of dp_r/dlambda must cancel exactly) while theta oscillates between the
    turning points cos^2(theta) = u_plus, and the Carter constant stays eta."""
    r, xi, eta, u_plus = spherical_photon_orbit(a, f)
    st = np.array([[0.0, r, math.pi / 2, 0.0, 0.0, math.sqrt(eta)]])
    res = oracle.trace_states(a, R0, st, [1.0], [xi], max_steps=800, tol=1e-12)
    assert res["status"][0] == oracle.STATUS_MAXSTEP
    assert res["t"][0] > 20.0
    assert abs(res["r"][0] - r) < 1e-8 * r
    assert math.cos(res["theta"][0]) ** 2 <= u_plus * (1 + 1e-9)
    assert res["carter0"][0] == pytest.approx(eta, rel=1e-12)
    assert res["max_carter_drift"][0] < 1e-9
    assert res["max_abs_H"][0] < 1e-10


def _cartesian_frame(th, ph):
    er = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    et = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
    ep = np.array([-math.sin(ph), math.cos(ph), 0.0])
    return er, et, ep


def _initial_direction(x, y, r0, th0):
    """Unit spatial direction of the ray in the observer's orthonormal frame:
    (P^r, P^theta, P^phi) = (-sqrt(1 - (x^2+y^2)/r0^2), y/r0, -x/r0)."""
    er, et, ep = _cartesian_frame(th0, 0.0)
    v = -math.sqrt(1 - (x * x + y * y) / r0 ** 2) * er + (y / r0) * et + (-x / r0) * ep
    return er, v


def _angles(u):
    th = math.acos(max(-1.0, min(1.0, u[2])))
    ph = math.atan2(u[1], u[0]) % (2 * math.pi)
    return th, ph


def _ang_close(got_th, got_ph, th, ph, tol):
    assert abs(got_th - th) < tol
    d = (got_ph - ph + math.pi) % (2 * math.pi) - math.pi
    assert abs(d) < tol


def test_flat_space_straight_lines():
    rng = np.random.default_rng(5)
    r0, inc = 1000.0, 70.0
    th0 = math.radians(inc)
    pts = rng.uniform(-400, 400, size=(12, 2))
    for x, y in pts:
        st = oracle.init_ray(0.0, r0, inc, x, y, M=0.0)
        res = oracle.trace_states(0.0, r0, st[None, :6], [st[6]], [st[7]], M=0.0)
        assert res["status"][0] == oracle.STATUS_ESCAPED
        n0, v = _initial_direction(x, y, r0, th0)
        X0 = r0 * n0
        r_esc = 1.1 * r0
        bdot = X0 @ v
        s = -bdot + math.sqrt(bdot * bdot - r0 * r0 + r_esc * r_esc)
        Xf = X0 + s * v
        th, ph = _angles(Xf / np.linalg.norm(Xf))
        _ang_close(res["theta"][0], res["phi"][0] % (2 * math.pi), th, ph, 1e-9)
        assert res["max_abs_H"][0] < 1e-9  # truncation error at tol 1e-10


def test_checkerboard_cells_from_exact_directions():
    """Celestial cells and parity (Sec. 4.1 set-up, 10-degree cells with a
    longitude phase) of flat-space rays, whose final directions are known
    exactly: straight lines to the escape sphere. The x = 0 rays (L = 0) cross
    the polar axis, so their coordinate theta leaves [0, pi] (above pi and
    below 0) and the fold theta -> -theta or 2 pi - theta, phi -> phi + pi must
    bring them back to the geometric direction."""
    r0, inc, cell_deg, phase_deg = 1000.0, 70.0, 10.0, 3.7
    th0, cell, phase = math.radians(inc), math.radians(cell_deg), math.radians(phase_deg)
    rng = np.random.default_rng(6)
    pts = [tuple(p) for p in rng.uniform(-400, 400, size=(24, 2))]
    pts += [(0.0, 150.0), (0.0, -150.0), (0.0, 420.0), (0.0, -600.0)]
    checked, folded = 0, 0
    for x, y in pts:
        st = oracle.init_ray(0.0, r0, inc, x, y, M=0.0)
        res = oracle.trace_states(0.0, r0, st[None, :6], [st[6]], [st[7]], M=0.0,
                                  cell_deg=cell_deg, cell_phase_deg=phase_deg)
        assert res["status"][0] == oracle.STATUS_ESCAPED
        n0, v = _initial_direction(x, y, r0, th0)
        X0 = r0 * n0
        bdot = X0 @ v
        Xf = X0 + (-bdot + math.sqrt(bdot * bdot - r0 * r0 + (1.1 * r0) ** 2)) * v
        th, ph = _angles(Xf / np.linalg.norm(Xf))
        q = (ph + phase) % (2 * math.pi)
        if min(abs(th / cell - round(th / cell)), abs(q / cell - round(q / cell))) * cell < 1e-6:
            continue  # too close to a cell edge to be decided by the direction alone
        i, j = int(th // cell), int(q // cell)
        assert (res["cell_i"][0], res["cell_j"][0], res["parity"][0]) == (i, j, (i + j) % 2), (x, y)
        checked += 1
        folded += not (0.0 <= res["theta"][0] <= math.pi)
    assert checked >= 24 and folded == 4


def _deflection_sweep(b, r0, r_esc):
    """Swept orbital angle from r0 in to the turning point and out to r_esc
    (Schwarzschild, M = 1): with u = 1/r the orbit equation reads
    (du/dphi)^2 = G(u) = 1/b^2 - u^2 + 2 u^3, so the sweep is the sum of the
    two integrals of du / sqrt(G) from 1/r0 and from 1/r_esc up to the
    turning point u_t, the smallest positive root of G."""
    import mpmath as mp
    mp.mp.dps = 40
    b = mp.mpf(b)
    roots = mp.polyroots([2, -1, 0, 1 / (b * b)], maxsteps=400, extraprec=120)
    u_t = min(mp.re(z) for z in roots if abs(mp.im(z)) < mp.mpf(10) ** -30 and mp.re(z) > 0)

    def f(u):
        return 1 / mp.sqrt(1 / (b * b) - u * u + 2 * u ** 3)

    total = mp.quad(f, [1 / mp.mpf(r0), u_t]) + mp.quad(f, [1 / mp.mpf(r_esc), u_t])
    return float(mp.re(total))


def test_schwarzschild_deflection():
    r0, inc = 1000.0, 85.0
    th0 = math.radians(inc)
    for x, y in [(-6.5, 0.7), (7.0, -3.0), (0.4, 8.9), (-9.0, -9.5), (5.6, 1.1)]:
        st = oracle.init_ray(0.0, r0, inc, x, y)
        res = oracle.trace_states(0.0, r0, st[None, :6], [st[6]], [st[7]])
        assert res["status"][0] == oracle.STATUS_ESCAPED
        b = math.hypot(x, y) / math.sqrt(1 - 2 / r0)
        Phi = _deflection_sweep(b, r0, 1.1 * r0)
        n0, v = _initial_direction(x, y, r0, th0)
        nrm = np.cross(n0, v)
        nrm /= np.linalg.norm(nrm)
        # rotate n0 by Phi about the orbit normal (Rodrigues)
        uf = n0 * math.cos(Phi) + np.cross(nrm, n0) * math.sin(Phi)
        th, ph = _angles(uf)
        _ang_close(res["theta"][0], res["phi"][0] % (2 * math.pi), th, ph, 1e-8)


# ---------------------------------------------------------------------------
# Invariants along oracle rays
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("a,inc", [(0.9, 60.0), (0.998, 17.0), (0.5, 90.0)])
def test_carter_constant_and_H(a, inc):
    n = 16
    res = oracle.trace_pixels(a, R0, inc, (-8, 8, -8, 8), n, n)
    rel = res["max_carter_drift"] / np.maximum(np.abs(res["carter0"]), 1.0)
    assert rel.max() < 1e-8
    esc = res["status"] == oracle.STATUS_ESCAPED
    # |H| of escaped rays stays near the per-step tolerance (1e-10)
    assert res["max_abs_H"][esc].max() < 2e-9


def test_H_scales_with_tolerance():
    cam = workloads.schwarzschild_shadow_64()
    pix = np.arange(0, 64 * 64, 37)
    out = {}
    for tol in (1e-10, 1e-11):
        res = oracle.trace_pixels(0.0, R0, 85.0, cam["extent"], 64, 64, pixels=pix, tol=tol)
        esc = res["status"] == oracle.STATUS_ESCAPED
        out[tol] = res["max_abs_H"][esc].max()
    assert out[1e-11] < 1e-10
    assert out[1e-11] < out[1e-10] / 5


# ---------------------------------------------------------------------------
# Thin Keplerian disk (Sec. 5)
# ---------------------------------------------------------------------------

def test_schwarzschild_disk_redshift_closed_form():
    cam = workloads.schwarzschild_disk(side=40)
    n = cam["nx"]
    res = oracle.trace_pixels(0.0, R0, cam["incl_deg"], cam["extent"], n, n, disk=True,
                              r_in=cam["r_in"], r_out=cam["r_out"],
                              cell_phase_deg=cam["cell_phase_deg"])
    disk = res["status"] == oracle.STATUS_DISK
    assert disk.sum() > 0.1 * n * n
    r = res["r_hit"][disk]
    assert r.min() >= 6.0 and r.max() <= 20.0
    assert np.abs(res["theta"][disk] - math.pi / 2).max() < 1e-12
    E, L = res["E"][disk], res["L"][disk]
    # u^t = 1/sqrt(1 - 3/r), Omega = r^-3/2
    g_expect = np.sqrt(1 - 3 / r) / (E - L * r ** -1.5)
    assert np.allclose(res["g"][disk], g_expect, rtol=1e-13)
    assert np.allclose(res["intensity"][disk], g_expect ** 3 / r ** 2, rtol=1e-12)
    # rays that miss the disk follow exactly the shadow-mode trajectory
    sh = oracle.trace_pixels(0.0, R0, cam["incl_deg"], cam["extent"], n, n,
                             cell_phase_deg=cam["cell_phase_deg"])
    miss = ~disk
    for key in ("status", "r", "theta", "phi", "max_abs_H", "accepted"):
        assert np.array_equal(res[key][miss], sh[key][miss]), key


def test_kerr_disk_redshift_closed_form():
    a = 0.9
    r_in = oracle.isco(a)
    res = oracle.trace_pixels(a, R0, 60.0, (-25, 25, -25, 25), 24, 24, disk=True, r_in=r_in,
                              r_out=20.0)
    disk = res["status"] == oracle.STATUS_DISK
    assert disk.sum() > 50
    r, E, L = res["r_hit"][disk], res["E"][disk], res["L"][disk]
    # Bardeen-Press-Teukolsky prograde circular orbit: u^t and Omega in closed form
    ut = (r ** 1.5 + a) / (r ** 0.75 * np.sqrt(r ** 1.5 - 3 * r ** 0.5 + 2 * a))
    Om = 1 / (r ** 1.5 + a)
    assert np.allclose(res["g"][disk], 1 / (ut * (E - Om * L)), rtol=1e-12)


def test_redshift_special_cases():
    # L = 0 ray hitting a Schwarzschild disk: g = sqrt(1 - 3/r) / E
    for r in (6.0, 9.5, 20.0):
        g, I = oracle.disk_observables(0.0, r, 0.97, 0.0)
        assert g == pytest.approx(math.sqrt(1 - 3 / r) / 0.97, rel=1e-14)
        assert I == pytest.approx(g ** 3 / r ** 2, rel=1e-14)


def test_isco():
    """ISCO closed form: extremum of the circular-orbit energy; a=0 -> 6, a=1 -> 1."""
    from scipy.optimize import minimize_scalar
    assert oracle.isco(0.0) == pytest.approx(6.0, abs=1e-13)
    assert oracle.isco(1.0) == pytest.approx(1.0, abs=1e-6)
    for a in (0.3, 0.5, 0.9, 0.998):
        def energy(r):
            return (r ** 1.5 - 2 * r ** 0.5 + a) / (r ** 0.75 * math.sqrt(r ** 1.5 - 3 * r ** 0.5 + 2 * a))
        rg = oracle.isco(a)
        opt = minimize_scalar(energy, bracket=(rg * 0.9, rg, rg * 1.5), tol=1e-12)
        assert opt.x == pytest.approx(rg, rel=1e-5)


# ---------------------------------------------------------------------------
# Cash-Karp 4(5) (Sec. 3.1)
# ---------------------------------------------------------------------------

def _order_conditions(A, b, c, order):
    """Butcher order conditions up to `order` (17 for order 5); returns residuals."""
    Ac = A @ c
    Ac2 = A @ (c * c)
    AAc = A @ Ac
    conds = [
        (1, b.sum(), 1),
        (2, b @ c, Fraction(1, 2)),
        (3, b @ c ** 2, Fraction(1, 3)), (3, b @ Ac, Fraction(1, 6)),
        (4, b @ c ** 3, Fraction(1, 4)), (4, b @ (c * Ac), Fraction(1, 8)),
        (4, b @ Ac2, Fraction(1, 12)), (4, b @ AAc, Fraction(1, 24)),
        (5, b @ c ** 4, Fraction(1, 5)), (5, b @ (c * c * Ac), Fraction(1, 10)),
        (5, b @ (c * Ac2), Fraction(1, 15)), (5, b @ (c * AAc), Fraction(1, 30)),
        (5, b @ (Ac * Ac), Fraction(1, 20)), (5, b @ (A @ c ** 3), Fraction(1, 20)),
        (5, b @ (A @ (c * Ac)), Fraction(1, 40)), (5, b @ (A @ Ac2), Fraction(1, 60)),
        (5, b @ (A @ AAc), Fraction(1, 120)),
    ]
    return [(o, float(v) - float(t)) for o, v, t in conds if o <= order]


def test_cash_karp_tableau_order_conditions():
    c, A, b5, b4 = oracle.ck_tableau()
    assert np.allclose(A.sum(axis=1), c, atol=1e-15)
    assert np.allclose(np.triu(A), 0.0)
    res5 = _order_conditions(A, b5, c, 5)
    assert len(res5) == 17
    assert max(abs(r) for _, r in res5) < 1e-14
    res4 = _order_conditions(A, b4, c, 5)
    assert max(abs(r) for o, r in res4 if o <= 4) < 1e-14
    assert max(abs(r) for o, r in res4 if o == 5) > 1e-4  # the embedded pair is 4th order


def test_cash_karp_convergence_order():
    """Fixed-step integration of a flat-space ray: global error of the
    propagated solution falls as h^5."""
    r0, th0 = 10.0, 1.0
    x, y = 3.0, -2.0
    st = oracle.init_ray(0.0, r0, math.degrees(th0), x, y, M=0.0)
    n0, v = _initial_direction(x, y, r0, th0)
    lam = 12.0
    Xf = r0 * n0 + lam * v  # E = 1: the affine parameter is the Euclidean length
    r_ex = np.linalg.norm(Xf)
    th_ex, ph_ex = _angles(Xf / r_ex)
    errs = []
    for nsteps in (80, 160, 320):
        yv = st[:6].copy()
        h = lam / nsteps
        for _ in range(nsteps):
            yv, _d = oracle.ck_step(0.0, yv, st[6], st[7], h, M=0.0)
        errs.append(max(abs(yv[1] - r_ex), abs(yv[2] - th_ex),
                        abs((yv[3] - ph_ex + math.pi) % (2 * math.pi) - math.pi)))
    orders = [math.log2(e1 / e2) for e1, e2 in zip(errs, errs[1:])]
    # pre-asymptotic at the coarse end, ~5.0 once h is small enough
    assert 4.6 < orders[0] < 6.2
    assert 4.7 < orders[1] < 5.3


# ---------------------------------------------------------------------------
# Dormand-Prince 5(4) (Sec. 3.1, the paper's preferred integrator)
# ---------------------------------------------------------------------------

def test_dormand_prince_tableau():
    n, c, A, b5, b4 = oracle.tableau(oracle.RKDP45)
    assert n == 7
    assert np.allclose(A.sum(axis=1), c, atol=1e-15)
    # first same as last: the seventh stage is evaluated at the fifth-order solution
    assert np.array_equal(A[6], b5) and c[6] == 1.0 and b5[6] == 0.0
    res5 = _order_conditions(A, b5, c, 5)
    assert max(abs(r) for _, r in res5) < 1e-14
    res4 = _order_conditions(A, b4, c, 5)
    assert max(abs(r) for o, r in res4 if o <= 4) < 1e-14
    assert max(abs(r) for o, r in res4 if o == 5) > 1e-5
    # the Cash-Karp tableau is unchanged by the generic stepper
    nc, cc, Ac, b5c, b4c = oracle.tableau(oracle.RKCK45)
    c0, A0, b50, b40 = oracle.ck_tableau()
    assert nc == 6 and np.array_equal(Ac[:6, :6], A0) and np.array_equal(b5c[:6], b50)


def test_dormand_prince_convergence_order():
    r0, th0 = 10.0, 1.0
    x, y = 3.0, -2.0
    st = oracle.init_ray(0.0, r0, math.degrees(th0), x, y, M=0.0)
    n0, v = _initial_direction(x, y, r0, th0)
    lam = 12.0
    Xf = r0 * n0 + lam * v
    r_ex = np.linalg.norm(Xf)
    th_ex, ph_ex = _angles(Xf / r_ex)
    errs = []
    for nsteps in (80, 160, 320):
        yv = st[:6].copy()
        for _ in range(nsteps):
            yv, _d = oracle.rk_step(oracle.RKDP45, 0.0, yv, st[6], st[7], lam / nsteps, M=0.0)
        errs.append(max(abs(yv[1] - r_ex), abs(yv[2] - th_ex),
                        abs((yv[3] - ph_ex + math.pi) % (2 * math.pi) - math.pi)))
    orders = [math.log2(e1 / e2) for e1, e2 in zip(errs, errs[1:])]
    assert 4.6 < orders[1] < 5.6


def test_dormand_prince_deflection_and_flags():
    """The DP45 path reaches the same exact results: Schwarzschild deflection
    and the finite-r0 critical curve."""
    r0, inc = 1000.0, 85.0
    th0 = math.radians(inc)
    for x, y in [(-6.5, 0.7), (7.0, -3.0)]:
        st = oracle.init_ray(0.0, r0, inc, x, y)
        res = oracle.trace_states(0.0, r0, st[None, :6], [st[6]], [st[7]],
                                  integrator=oracle.RKDP45)
        b = math.hypot(x, y) / math.sqrt(1 - 2 / r0)
        Phi = _deflection_sweep(b, r0, 1.1 * r0)
        n0, v = _initial_direction(x, y, r0, th0)
        nrm = np.cross(n0, v)
        nrm /= np.linalg.norm(nrm)
        uf = n0 * math.cos(Phi) + np.cross(nrm, n0) * math.sin(Phi)
        th, ph = _angles(uf)
        _ang_close(res["theta"][0], res["phi"][0] % (2 * math.pi), th, ph, 1e-8)
    a, inc, n = 0.9, 60.0, 16
    ext = (-8.0, 8.0, -8.0, 8.0)
    res = oracle.trace_pixels(a, R0, inc, ext, n, n, integrator=oracle.RKDP45)
    flags = np.zeros((n, n), bool)
    for j in range(n):
        for i in range(n):
            xx = ext[0] + (i + 0.5) * 16 / n
            yy = ext[2] + (j + 0.5) * 16 / n
            flags[j, i] = _captured_by_radial_potential(a, oracle.init_ray(a, R0, inc, xx, yy))
    got = (res["status"] == oracle.STATUS_CAPTURED).reshape(n, n)
    keep = ~_band_mask(flags)
    assert np.array_equal(got[keep], flags[keep])


def test_dormand_prince_keeps_H_smaller():
    """Sec. 3.1-3.2: Dormand-Prince preserves the constraint better than
    Cash-Karp. At the same tolerance its mean |H| is lower on escaped rays and
    much lower near the horizon."""
    out = {}
    for integ in (oracle.RKCK45, oracle.RKDP45):
        r = oracle.trace_pixels(0.98, R0, 90.0, (-8, 8, -8, 8), 32, 32, integrator=integ)
        esc = r["status"] == oracle.STATUS_ESCAPED
        cap = r["status"] == oracle.STATUS_CAPTURED
        out[integ] = (r["max_abs_H"][esc].mean(), r["max_abs_H"][cap].mean())
    assert out[oracle.RKDP45][0] < out[oracle.RKCK45][0]
    assert out[oracle.RKDP45][1] < out[oracle.RKCK45][1] / 5


# ---------------------------------------------------------------------------
# Disk of constant specific angular momentum l0 (Sec. 5)
# ---------------------------------------------------------------------------

def test_constant_l0_disk_closed_forms():
    # Schwarzschild: Omega = l0 (1 - 2/r) / r^2, u^t = 1/sqrt((1 - 2/r) - Omega^2 r^2)
    for r, l0, E, L in ((6.0, 2.8, 0.97, 1.3), (11.0, 3.5, 1.0, -2.0)):
        g, I = oracle.disk_observables_l0(0.0, r, E, L, l0)
        Om = l0 * (1 - 2 / r) / r ** 2
        g_expect = math.sqrt((1 - 2 / r) - Om ** 2 * r ** 2) / (E - Om * L)
        assert g == pytest.approx(g_expect, rel=1e-13)
        assert I == pytest.approx(g_expect ** 3 / r ** 2, rel=1e-13)
    # l0 equal to the Keplerian l(r) = (r^2 - 2 a sqrt r + a^2) / (r^3/2 - 2 sqrt r + a)
    # at radius r reproduces the Keplerian redshift there (Schwarzschild and Kerr)
    for a, r in ((0.0, 7.5), (0.9, 3.1), (0.998, 1.6)):
        lk = (r * r - 2 * a * math.sqrt(r) + a * a) / (r ** 1.5 - 2 * math.sqrt(r) + a)
        gk, _ = oracle.disk_observables(a, r, 0.93, 2.2)
        gl, _ = oracle.disk_observables_l0(a, r, 0.93, 2.2, lk)
        assert gl == pytest.approx(gk, rel=1e-12)


def test_constant_l0_disk_render():
    rd = workloads.paper_disk_figure(nx=48, ny=24)[2]  # a = 0.998, l0 = 1.8
    res = oracle.trace_pixels(rd["a"], rd["r_obs"], rd["incl_deg"], rd["extent"], rd["nx"],
                              rd["ny"], disk=True, r_in=oracle.isco(rd["a"]), r_out=20.0,
                              disk_model=oracle.DISK_CONSTANT_L, l0=rd["l0"])
    disk = res["status"] == oracle.STATUS_DISK
    assert disk.sum() > 100
    # the l0 model changes only the observables: every other output equals the
    # Keplerian render's
    kep = oracle.trace_pixels(rd["a"], rd["r_obs"], rd["incl_deg"], rd["extent"], rd["nx"],
                              rd["ny"], disk=True, r_in=oracle.isco(rd["a"]), r_out=20.0)
    for key in ("status", "r", "theta", "phi", "accepted"):
        assert np.array_equal(res[key], kep[key]), key
    assert not np.allclose(res["g"][disk], kep["g"][disk])
    assert np.all(res["g"][disk] > 0)


# ---------------------------------------------------------------------------
# q-metric (Appendix A) and time-like geodesics
# ---------------------------------------------------------------------------

def _qmetric_line_element(q, r, th):
    """The q-metric of Appendix A, converted to signature (-,+,+,+)."""
    f = 1 - 2 / r
    X = 1 + math.sin(th) ** 2 / (r * r - 2 * r)
    k = q * (2 + q)
    return np.diag([-f ** (1 + q), f ** (-1 - q) * X ** -k, f ** -q * r * r * X ** -k,
                    f ** -q * (r * math.sin(th)) ** 2])


@pytest.mark.parametrize("q", [0.5, -0.5, 0.2])
def test_qmetric_components_and_derivatives(q):
    for r, th in ((3.5, 1.0), (9.0, 0.4), (25.0, 2.0), (4.2, math.pi / 2)):
        g, gi, dr, dth = oracle.metric_sp(oracle.QMETRIC, r, th, q=q)
        assert np.allclose(g, _qmetric_line_element(q, r, th), rtol=1e-14, atol=0)
        assert np.allclose(gi @ g, np.eye(4), atol=1e-13)
        fr = _fd(lambda rr: oracle.metric_sp(oracle.QMETRIC, rr, th, q=q)[1], r, 1e-3 * r)
        ft = _fd(lambda tt: oracle.metric_sp(oracle.QMETRIC, r, tt, q=q)[1], th, 1e-3)
        scale = np.abs(fr).max()
        assert np.abs(dr - fr).max() <= 1e-8 * scale
        # theta-derivatives vanish on the equator: compare on the r-derivative scale
        assert np.abs(dth - ft).max() <= 1e-8 * max(np.abs(ft).max(), scale)


def test_qmetric_q0_is_schwarzschild():
    for r, th in ((3.0, 0.7), (50.0, 2.2)):
        gq = oracle.metric_sp(oracle.QMETRIC, r, th, q=0.0)
        gk = oracle.metric_sp(oracle.KERR, r, th, a=0.0)
        for A, B in zip(gq, gk):
            assert np.allclose(A, B, rtol=1e-13, atol=1e-300)
    n = 16
    rq = oracle.trace_pixels(0.0, R0, 60.0, (-8, 8, -8, 8), n, n, spacetime=oracle.QMETRIC,
                             q=0.0)
    rk = oracle.trace_pixels(0.0, R0, 60.0, (-8, 8, -8, 8), n, n)
    assert np.array_equal(rq["status"], rk["status"])
    for key in ("r", "theta", "phi"):
        assert np.allclose(rq[key], rk[key], rtol=1e-9, atol=1e-9), key


def _circular_orbit(q, r):
    """Equatorial circular time-like orbit of the static metric from the line
    element alone: Omega^2 = -d_r g_tt / d_r g_phph, u^t from g_ab u^a u^b = -1,
    E = -g_tt u^t, L = g_phph Omega u^t."""
    h = 1e-5 * r
    g = _qmetric_line_element(q, r, math.pi / 2)
    gp = _qmetric_line_element(q, r + h, math.pi / 2)
    gm = _qmetric_line_element(q, r - h, math.pi / 2)
    dgtt = (gp[0, 0] - gm[0, 0]) / (2 * h)
    dgpp = (gp[3, 3] - gm[3, 3]) / (2 * h)
    Om = math.sqrt(-dgtt / dgpp)
    ut = 1 / math.sqrt(-g[0, 0] - g[3, 3] * Om * Om)
    return Om, -g[0, 0] * ut, g[3, 3] * Om * ut


def qmetric_light_ring(q):
    """The equatorial circular photon orbit of the q-metric: b^2 = g_phph / -g_tt
    = r^2 f^-(1+2q) is extremal where 2/r = (1+2q) 2/(r (r-2)), i.e.
    r = 3 + 2q (X does not enter g_tt or g_phph on the equator); dphi/dt = 1/b.
    Exists for q > -1/2."""
    r = 3.0 + 2.0 * q
    b = r * (1.0 - 2.0 / r) ** (-(1.0 + 2.0 * q) / 2.0)
    return r, b


@pytest.mark.parametrize("q", [-0.3, 0.1, 0.5])
def test_qmetric_light_ring(q):
    """Started on r = 3 + 2q with p_r = p_theta = 0 and L/E = b, a photon stays
    on the circle and goes round at dphi/dt = 1/b: fixes the r-equation of the
    q-metric (a wrong term in d g^tt/dr or d g^phph/dr moves or breaks the
    circle)."""
    r, b = qmetric_light_ring(q)
    st = np.array([[0.0, r, math.pi / 2, 0.0, 0.0, 0.0]])
    assert abs(oracle.hamiltonian_sp(oracle.QMETRIC, st[0], 1.0, b, q=q)) < 1e-14
    res = oracle.trace_states(0.0, R0, st, [1.0], [b], spacetime=oracle.QMETRIC, q=q,
                              max_steps=60)
    assert res["status"][0] == oracle.STATUS_MAXSTEP
    assert res["r"][0] == pytest.approx(r, abs=1e-8)
    assert res["phi"][0] / res["t"][0] == pytest.approx(1 / b, rel=1e-9)
    assert res["t"][0] > 10.0
    # off the ring by 1e-3 the same photon leaves it (the ring is unstable)
    st[0, 1] = r * (1 + 1e-3)
    off = oracle.trace_states(0.0, R0, st, [1.0], [b], spacetime=oracle.QMETRIC, q=q,
                              max_steps=400)
    assert off["status"][0] in (oracle.STATUS_ESCAPED, oracle.STATUS_CAPTURED)


@pytest.mark.parametrize("q", [0.0, 0.5, -0.5])
def test_timelike_circular_orbits(q):
    r = 12.0
    Om, E, L = _circular_orbit(q, r)
    if q == 0.0:  # Schwarzschild closed form
        assert E == pytest.approx((1 - 2 / r) / math.sqrt(1 - 3 / r), rel=1e-9)
        assert L == pytest.approx(math.sqrt(r) / math.sqrt(1 - 3 / r), rel=1e-9)
    st = np.array([[0.0, r, math.pi / 2, 0.0, 0.0, 0.0]])
    # the initial data lie on the mass shell H = -1/2
    assert oracle.hamiltonian_sp(oracle.QMETRIC, st[0], E, L, q=q) == pytest.approx(-0.5,
                                                                                   abs=1e-9)
    res = oracle.trace_states(0.0, 1000.0, st, [E], [L], spacetime=oracle.QMETRIC, q=q,
                              mass2=1.0, max_steps=150)
    assert res["status"][0] == oracle.STATUS_MAXSTEP
    assert res["r"][0] == pytest.approx(r, rel=1e-7)
    assert res["phi"][0] / res["t"][0] == pytest.approx(Om, rel=1e-7)
    assert res["max_abs_H"][0] < 1e-8


def bpt_circular_orbit(a, r):
    """Prograde equatorial circular orbit of a unit-mass particle in Kerr
    (Bardeen, Press & Teukolsky 1972, M = 1): energy, angular momentum and
    angular velocity as closed forms in r and a."""
    v = math.sqrt(r)
    den = r ** 0.75 * math.sqrt(r * v - 3.0 * v + 2.0 * a)
    E = (r * v - 2.0 * v + a) / den
    L = (r * r - 2.0 * a * v + a * a) / den
    return E, L, 1.0 / (r * v + a)


@pytest.mark.parametrize("a", [0.5, 0.9, 0.998])
@pytest.mark.parametrize("r_over_isco", [1.2, 3.0])
def test_kerr_timelike_circular_orbits(a, r_over_isco):
    """A unit-mass particle started on the closed-form Kerr circular orbit
    (on the mass shell H = -1/2) stays on it and goes round at
    dphi/dt = 1/(r^(3/2) + a): pins the Kerr equations of motion with mass,
    the H0 = -1/2 bookkeeping and the t and phi equations."""
    r = r_over_isco * oracle.isco(a)
    E, L, Om = bpt_circular_orbit(a, r)
    st = np.array([[0.0, r, math.pi / 2, 0.0, 0.0, 0.0]])
    assert oracle.hamiltonian(a, st[0], E, L) == pytest.approx(-0.5, abs=1e-13)
    res = oracle.trace_states(a, 1000.0, st, [E], [L], mass2=1.0, max_steps=200)
    assert res["status"][0] == oracle.STATUS_MAXSTEP
    assert res["r"][0] == pytest.approx(r, rel=1e-8)
    assert res["theta"][0] == pytest.approx(math.pi / 2, abs=1e-12)
    assert res["phi"][0] / res["t"][0] == pytest.approx(Om, rel=1e-9)
    assert res["max_abs_H"][0] < 1e-10


def test_timelike_radial_escape_and_H_shell():
    """An unbound time-like particle (E > 1) in the q-metric escapes, keeping
    |H + 1/2| near the tolerance; the same ray traced as null data fails the
    null constraint, which is what max_abs_H reports."""
    q = -0.5
    r = 30.0
    g = _qmetric_line_element(q, r, math.pi / 2)
    E, L, pth = 1.2, 4.0, 0.0
    # p_r from the mass shell g^tt E^2 + g^rr p_r^2 + g^phph L^2 = -1
    pr = math.sqrt((-1 + E * E / -g[0, 0] - L * L / g[3, 3]) * g[1, 1])
    st = np.array([[0.0, r, math.pi / 2, 0.0, pr, pth]])
    res = oracle.trace_states(0.0, 100.0, st, [E], [L], spacetime=oracle.QMETRIC, q=q, mass2=1.0)
    assert res["status"][0] == oracle.STATUS_ESCAPED
    assert res["max_abs_H"][0] < 1e-8
    res0 = oracle.trace_states(0.0, 100.0, st, [E], [L], spacetime=oracle.QMETRIC, q=q)
    assert abs(res0["max_abs_H"][0] - 0.5) < 1e-8


# ---------------------------------------------------------------------------
# Generic Kerr end points from the first integrals (Mino-time quadratures,
# oracle/first_integrals.py)
# ---------------------------------------------------------------------------

from oracle.first_integrals import KERR_END_POINT_RAYS, kerr_end_point  # noqa: E402

@pytest.mark.parametrize("a,inc,pixels,captured", KERR_END_POINT_RAYS)
def test_kerr_escape_point_from_first_integrals(a, inc, pixels, captured):
    """Generic Kerr rays (a != 0, off the equator, several passes through the
    polar turning points): the oracle's end point (cos theta, phi) at
    r_esc = 1.1 r0 for escaping rays and at r_cap = 1.01 r_H for captured
    ones, integrated at tol 1e-12, agrees with the quadratures of the first
    integrals to 1e-8. A slip in any derivative of the oracle's equations of
    motion moves the end point by far more."""
    r0 = 1000.0
    r_cap = 1.01 * (1.0 + math.sqrt(1.0 - a * a))
    for (x, y), fate in [(p, oracle.STATUS_ESCAPED) for p in pixels] + \
                        [(p, oracle.STATUS_CAPTURED) for p in captured]:
        st = oracle.init_ray(a, r0, inc, x, y)
        res = oracle.trace_states(a, r0, st[None, :6], [st[6]], [st[7]], tol=1e-12)
        assert res["status"][0] == fate, (a, inc, x, y)
        uf, phif = kerr_end_point(a, 1.1 * r0, st, r_cap=r_cap)
        assert abs(math.cos(res["theta"][0]) - uf) < 1e-8, (x, y, math.cos(res["theta"][0]), uf)
        assert abs(res["phi"][0] - phif) < 1e-8 * max(1.0, abs(phif)), (x, y, res["phi"][0], phif)


def test_golden_kerr_end_points_are_current():
    """tests/golden/kerr_end_points.json (the GPU test's expected values) is
    what its script writes from the quadratures: two entries recomputed."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "kerr_end_points.json")) as f:
        rays = json.load(f)["rays"]
    assert len(rays) == sum(len(e) + len(c) for _, _, e, c in KERR_END_POINT_RAYS)
    for row in (rays[0], rays[-1]):
        a = row["a"]
        st = oracle.init_ray(a, 1000.0, row["incl_deg"], row["x"], row["y"])
        u, phi = kerr_end_point(a, 1100.0, st, r_cap=1.01 * (1.0 + math.sqrt(1.0 - a * a)))
        assert abs(u - row["cos_theta"]) < 1e-14 and abs(phi - row["phi"]) < 1e-13


# ---------------------------------------------------------------------------
# Generic q-metric rays against the geodesic equation of the line element
# ---------------------------------------------------------------------------

def _qmetric_geodesic_end(q, r_obs, st, r_cap):
    """End point of a q-metric null geodesic from the second-order geodesic
    equation x'' = -Gamma(x', x'), with the Christoffel symbols derived by
    sympy from the line element of Appendix A (signature -+++, m = 1:
    g_tt = -f^(1+q), g_rr = f^(-1-q) X^-k, g_thth = f^-q r^2 X^-k,
    g_phph = f^-q r^2 sin^2, f = 1 - 2/r, X = 1 + sin^2 / (r^2 - 2 r),
    k = q (2 + q)), integrated by scipy's DOP853 at rtol 1e-13 from the same
    initial momenta (velocities x'^mu = g^{mu mu} p_mu) to r = 1.1 r_obs or
    r = r_cap. Returns (status, theta, phi)."""
    sp = pytest.importorskip("sympy")
    from scipy.integrate import solve_ivp
    r, th = sp.symbols("r theta", positive=True)
    f = 1 - 2 / r
    X = 1 + sp.sin(th) ** 2 / (r ** 2 - 2 * r)
    k = q * (2 + q)
    g = [-f ** (1 + q), f ** (-1 - q) * X ** (-k), f ** (-q) * r ** 2 * X ** (-k),
         f ** (-q) * r ** 2 * sp.sin(th) ** 2]
    x = [None, r, th, None]  # t and phi are cyclic
    gam = {}
    for a_ in range(4):
        for b_ in range(4):
            for c_ in range(b_, 4):
                # diagonal metric: Gamma^a_bc = (d_b g_ac + d_c g_ab - d_a g_bc) / (2 g_aa)
                term = 0
                if a_ == c_ and x[b_] is not None:
                    term += sp.diff(g[a_], x[b_])
                if a_ == b_ and x[c_] is not None:
                    term += sp.diff(g[a_], x[c_])
                if b_ == c_ and x[a_] is not None:
                    term -= sp.diff(g[b_], x[a_])
                term = sp.simplify(term / (2 * g[a_]))
                if term != 0:
                    gam[(a_, b_, c_)] = sp.lambdify((r, th), term, "math")
    gdiag = [sp.lambdify((r, th), gi, "math") for gi in g]

    def rhs(_, s):
        pos, vel = s[:4], s[4:]
        acc = [0.0, 0.0, 0.0, 0.0]
        for (a_, b_, c_), fn in gam.items():
            v = fn(pos[1], pos[2]) * vel[b_] * vel[c_]
            acc[a_] -= v if b_ == c_ else 2.0 * v
        return list(vel) + acc

    r0, th0, p_r, p_th, E, L = st[1], st[2], st[4], st[5], st[6], st[7]
    gv = [fn(r0, th0) for fn in gdiag]
    v0 = [-E / gv[0], p_r / gv[1], p_th / gv[2], L / gv[3]]
    esc = lambda _, s: s[1] - 1.1 * r_obs
    esc.terminal, esc.direction = True, 1
    cap = lambda _, s: s[1] - r_cap
    cap.terminal, cap.direction = True, -1
    sol = solve_ivp(rhs, (0.0, 1e5), [0.0, r0, th0, 0.0] + v0, method="DOP853", rtol=1e-13,
                    atol=1e-13, events=(esc, cap))
    assert sol.status == 1
    hit = 0 if sol.t_events[0].size else 1
    end = sol.y_events[hit][0]
    return (oracle.STATUS_ESCAPED if hit == 0 else oracle.STATUS_CAPTURED), end[2], end[3]


@pytest.mark.parametrize("q,inc,pixels", [(0.5, 60.0, [(9.0, 3.0), (-7.5, 5.0), (1.0, 0.5)]),
                                          (-0.5, 30.0, [(-5.5, 3.0), (4.0, 4.0),
                                                        (0.5, -1.5)])])
def test_qmetric_rays_against_line_element_geodesics(q, inc, pixels):
    """Generic q-metric rays (no Carter constant, so no quadratures): the
    oracle's end points (Hamilton's equations with hand-derived inverse-metric
    derivatives, Cash-Karp at tol 1e-12) against the second-order geodesic
    equation of the printed line element with symbolic Christoffel symbols,
    integrated by an unrelated high-order method: status identical, theta and
    phi within 1e-8 (measured: 1.6e-10)."""
    r0 = 1000.0
    r_cap = 1.01 * 2.0
    fates = set()
    for x, y in pixels:
        st = oracle.init_ray_sp(oracle.QMETRIC, r0, inc, x, y, q=q)
        res = oracle.trace_states(0.0, r0, st[None, :6], [st[6]], [st[7]],
                                  spacetime=oracle.QMETRIC, q=q, tol=1e-12)
        status, th_f, ph_f = _qmetric_geodesic_end(q, r0, st, r_cap)
        assert res["status"][0] == status, (q, x, y)
        fates.add(status)
        assert abs(res["theta"][0] - th_f) < 1e-8, (q, x, y, res["theta"][0], th_f)
        assert abs(res["phi"][0] - ph_f) < 1e-8 * max(1.0, abs(ph_f)), (q, x, y, res["phi"][0], ph_f)
    assert fates == {oracle.STATUS_ESCAPED, oracle.STATUS_CAPTURED}
