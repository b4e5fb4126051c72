"""Exact end points of Kerr null geodesics from their first integrals.

TEST INFRASTRUCTURE (part of the oracle): only the test suite and the script
that writes tests/golden/kerr_end_points.json call it. It computes what the
oracle's Runge-Kutta integration of Hamilton's equations (Sec. 2.1, on the
Kerr metric of Sec. 4.3, Eq. Kerr) computes for a ray, the point where it
reaches the escape or capture radius, by a different route: Kerr null
geodesics separate (E, L and the Carter constant are conserved), so in Mino
time the motion reduces to one-dimensional quadratures of the radial and
polar potentials. It shares no code with the oracle's integrator and none
with the CUDA library. tests/test_oracle_pins.py pins the oracle to it.
"""
# (a, inclination in degrees, escaping pixels, captured pixels) of the rays
# the pin and the golden end points use; r_obs = 1000
KERR_END_POINT_RAYS = [
    (0.9, 60.0, [(6.5, 1.0), (-7.5, 2.0), (2.0, -6.8)], [(1.0, 0.5), (-2.5, -1.0)]),
    (0.998, 17.0, [(6.0, 1.5), (-4.5, 5.5)], [(0.5, 2.0)]),
    (0.5, 90.0, [(0.8, 6.5), (-6.0, -2.0)], [(-1.5, 3.0)]),
]


def kerr_end_point(a, r_esc, st, r_cap=None):
    """Final (cos theta, phi) at r = r_esc of an escaping Kerr null geodesic
    or, when it has no radial turning point outside r_cap, at r = r_cap where
    it is captured: from its first integrals alone (Carter 1968), with E = 1, xi = L/E and
    eta = Q/E^2, in Mino time tau (d tau = d lambda / Sigma):
      (dr/dtau)^2 = R(r) = (r^2 + a^2 - a xi)^2 - Delta (eta + (xi - a)^2),
      (du/dtau)^2 = U(u) = eta - (eta + xi^2 - a^2) u^2 - a^2 u^4,  u = cos theta,
      dphi/dtau  = a (r^2 + a^2 - a xi) / Delta - a + xi / (1 - u^2).
    The radial leg runs in from r0 to the turning point r_min (largest root of
    R) and out to r_esc (or, captured, from r0 to r_cap); its Mino time is how
    far u travels along its
    oscillation between -u+ and +u+, starting in the direction opposite to the
    sign of p_theta. Every integral is a one-dimensional quadrature (mpmath,
    30 digits) with the potentials factored at their turning points, so the
    endpoint singularities are exact square-root ones."""
    import mpmath as mp
    mp.mp.dps = 30
    r0, th0, p_th, E, L = (mp.mpf(float(v)) for v in (st[1], st[2], st[5], st[6], st[7]))
    a = mp.mpf(a)
    r_esc = mp.mpf(r_esc)
    xi = L / E
    eta = (p_th ** 2 + mp.cos(th0) ** 2 * (L ** 2 / mp.sin(th0) ** 2 - a * a * E * E)) / E ** 2
    # R(r) = r^4 + c2 r^2 + c1 r + c0 and its largest real root
    c2, c1, c0 = a * a - xi * xi - eta, 2 * (eta + (xi - a) ** 2), -a * a * eta
    roots = mp.polyroots([1, 0, c2, c1, c0], maxsteps=400, extraprec=200)
    real = [mp.re(z) for z in roots if abs(mp.im(z)) < mp.mpf(10) ** -20]
    r_min = max(real) if real else None
    if r_min is not None and r_min > (r_cap if r_cap is not None else 1):
        b2 = r_min                   # R = (r - r_min) (r^3 + b2 r^2 + b1 r + b0)
        b1 = c2 + r_min * b2
        b0 = c1 + r_min * b1

        def radial(f):
            g = lambda r: f(r) / mp.sqrt((r - r_min) * (((r + b2) * r + b1) * r + b0))
            return mp.quad(g, [r_min, r0]) + mp.quad(g, [r_min, r_esc])
    else:  # no turning point before the capture radius: one inward leg
        assert r_cap is not None

        def radial(f):
            g = lambda r: f(r) / mp.sqrt((((r * r + c2) * r + c1) * r + c0))
            return mp.quad(g, [mp.mpf(r_cap), r0])

    tau = radial(lambda r: 1)
    phi = radial(lambda r: a * (r * r + a * a - a * xi) / (r * r - 2 * r + a * a) - a)
    # U(u) = a^2 (u+^2 - u^2)(u^2 + m): u^2 roots of a^2 w^2 + (eta + xi^2 - a^2) w - eta
    B = eta + xi * xi - a * a
    disc = mp.sqrt(B * B + 4 * a * a * eta)
    up = mp.sqrt((-B + disc) / (2 * a * a))
    m = (B + disc) / (2 * a * a)
    U = lambda u: a * a * (up - u) * (up + u) * (u * u + m)
    dtau = lambda u: 1 / mp.sqrt(U(u))
    dphi = lambda u: xi / (1 - u * u) / mp.sqrt(U(u))
    u = mp.cos(th0)
    s = -1 if p_th > 0 else 1
    left = tau
    while True:  # one monotone pass of u per iteration; s = sign of du/dtau
        end = s * up
        seg = s * mp.quad(dtau, [u, end])  # Mino time of the pass (> 0)
        if left <= seg:
            uf = mp.findroot(lambda v: s * mp.quad(dtau, [u, v]) - left, (u, end),
                             solver="anderson")
            phi += s * mp.quad(dphi, [u, uf])
            return float(uf), float(phi)
        left -= seg
        phi += s * mp.quad(dphi, [u, end])
        u, s = end, -s
