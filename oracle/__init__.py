"""ctypes front end of the serial FP64 CPU oracle (oracle/osiris_oracle.cpp).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package. It shares no code with
the CUDA library and never calls it.

Every function follows a passage of Velasquez-Cadavid et al., "OSIRIS"
(arXiv:2202.00086); see the header of osiris_oracle.cpp for the list.
Every function is pinned to something other than itself (closed forms,
reductions, first integrals, an independent geodesic integration); the one
quantity with no such pin is the size of the integration error |H| itself.
"""
import ctypes
import os

import numpy as np

from . import build as _build

STATUS_NONE, STATUS_CAPTURED, STATUS_ESCAPED, STATUS_DISK, STATUS_MAXSTEP, STATUS_ERROR = range(6)
RKCK45, RKDP45 = 0, 1
DISK_KEPLERIAN, DISK_CONSTANT_L = 0, 1
KERR, QMETRIC = 0, 1

_P = ctypes.POINTER
_d = ctypes.c_double
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


class OracleOptions(ctypes.Structure):
    _fields_ = [("tol", _d), ("max_steps", _i64), ("r_cap_factor", _d), ("r_esc_factor", _d),
                ("disk", _i32), ("r_in", _d), ("r_out", _d), ("cell_deg", _d),
                ("cell_phase_deg", _d), ("integrator", _i32), ("disk_model", _i32),
                ("l0", _d), ("spacetime", _i32), ("q", _d), ("mass2", _d)]


_OUT_FIELDS = [
    ("status", np.int32), ("t", np.float64), ("r", np.float64), ("theta", np.float64),
    ("phi", np.float64), ("p_r", np.float64), ("p_theta", np.float64), ("E", np.float64),
    ("L", np.float64), ("max_abs_H", np.float64), ("accepted", np.int64),
    ("rejected", np.int64), ("bisection_steps", np.int64), ("cell_i", np.int32),
    ("cell_j", np.int32), ("parity", np.int32), ("g", np.float64), ("intensity", np.float64),
    ("r_hit", np.float64), ("carter0", np.float64), ("max_carter_drift", np.float64),
]
_CT = {np.int32: _i32, np.int64: _i64, np.float64: _d}


class OracleOutputs(ctypes.Structure):
    _fields_ = [(name, _P(_CT[dt])) for name, dt in _OUT_FIELDS]


_lib = None


def lib():
    """Load (building first if needed) liboracle.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_trace_pixels.argtypes = [_d, _d, _d, _d, _d, _d, _d, _d, _i32, _i32,
                                          _P(OracleOptions), _P(_i64), _i64, _i32,
                                          _P(OracleOutputs)]
        L.oracle_trace_pixels.restype = ctypes.c_int
        L.oracle_trace_states.argtypes = [_d, _d, _d, _P(OracleOptions), _P(_d), _P(_d), _P(_d),
                                          _i64, _P(OracleOutputs)]
        L.oracle_trace_states.restype = ctypes.c_int
        L.oracle_init_ray.argtypes = [_d, _d, _d, _d, _d, _d, _P(_d)]
        for fn in ("oracle_metric_cov", "oracle_metric_con"):
            getattr(L, fn).argtypes = [_d, _d, _d, _d, _P(_d)]
        L.oracle_metric_con_derivs.argtypes = [_d, _d, _d, _d, _P(_d), _P(_d)]
        L.oracle_hamiltonian.argtypes = [_d, _d, _P(_d), _d, _d]
        L.oracle_hamiltonian.restype = _d
        L.oracle_rhs.argtypes = [_d, _d, _P(_d), _d, _d, _P(_d)]
        L.oracle_ck_step.argtypes = [_d, _d, _P(_d), _d, _d, _d, _P(_d), _P(_d)]
        L.oracle_ck_tableau.argtypes = [_P(_d)] * 4
        L.oracle_rk_step.argtypes = [_i32, _d, _d, _P(_d), _d, _d, _d, _P(_d), _P(_d)]
        L.oracle_tableau.argtypes = [_i32] + [_P(_d)] * 4
        L.oracle_tableau.restype = _i32
        L.oracle_disk_observables.argtypes = [_d, _d, _d, _d, _d, _P(_d), _P(_d)]
        L.oracle_disk_observables_l0.argtypes = [_d, _d, _d, _d, _d, _d, _P(_d), _P(_d)]
        L.oracle_metric_sp.argtypes = [_i32, _d, _d, _d, _d, _d] + [_P(_d)] * 4
        L.oracle_hamiltonian_sp.argtypes = [_i32, _d, _d, _d, _P(_d), _d, _d]
        L.oracle_hamiltonian_sp.restype = _d
        L.oracle_rhs_sp.argtypes = [_i32, _d, _d, _d, _P(_d), _d, _d, _P(_d)]
        L.oracle_init_ray_sp.argtypes = [_i32, _d, _d, _d, _d, _d, _d, _d, _P(_d)]
        L.oracle_isco.argtypes = [_d, _d]
        L.oracle_isco.restype = _d
        _lib = L
    return _lib


def _ptr(arr, ct):
    return arr.ctypes.data_as(_P(ct))


def options(tol=1e-10, max_steps=1_000_000, r_cap_factor=1.01, r_esc_factor=1.1, disk=False,
            r_in=0.0, r_out=0.0, cell_deg=10.0, cell_phase_deg=0.0, integrator=RKCK45,
            disk_model=DISK_KEPLERIAN, l0=0.0, spacetime=KERR, q=0.0, mass2=0.0):
    """spacetime KERR (the `a` argument of the trace calls is the spin) or
    QMETRIC (quadrupole q, Appendix A); mass2 = 0 null, 1 time-like."""
    return OracleOptions(tol, max_steps, r_cap_factor, r_esc_factor, 1 if disk else 0, r_in,
                         r_out, cell_deg, cell_phase_deg, int(integrator), int(disk_model),
                         float(l0), int(spacetime), float(q), float(mass2))


def _alloc(n):
    arrs = {name: np.zeros(n, dtype=dt) for name, dt in _OUT_FIELDS}
    out = OracleOutputs(**{name: _ptr(arrs[name], _CT[dt]) for name, dt in _OUT_FIELDS})
    return arrs, out


def trace_pixels(a, r_obs, incl_deg, extent, nx, ny, pixels=None, M=1.0, nthreads=None,
                 **opt):
    """Trace image-plane pixels of a camera (Sec. 2.3 set-up, Sec. 3-5 integration).

    extent = (x_min, x_max, y_min, y_max); pixels = linear indices j*nx + i
    (default: the whole image). Returns a dict of numpy arrays, one entry per
    traced pixel. Generic Kerr end points are pinned to the quadratures of
    the first integrals (Mino time); generic q-metric end points (no Carter
    constant, no quadrature) to the second-order geodesic equation of the
    line element, integrated independently. The pins are listed in
    tests/test_oracle_pins.py.
    """
    L = lib()
    if pixels is None:
        pixels = np.arange(nx * ny, dtype=np.int64)
    pixels = np.ascontiguousarray(pixels, dtype=np.int64)
    n = pixels.size
    arrs, out = _alloc(n)
    o = options(**opt)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    x0, x1, y0, y1 = extent
    L.oracle_trace_pixels(M, a, r_obs, incl_deg, x0, x1, y0, y1, nx, ny, ctypes.byref(o),
                          _ptr(pixels, _i64), n, nthreads, ctypes.byref(out))
    return arrs


def trace_states(a, r_obs, states, E, L_z, M=1.0, **opt):
    """Trace rays from explicit initial data rows (t, r, theta, phi, p_r, p_theta)."""
    lb = lib()
    states = np.ascontiguousarray(states, dtype=np.float64).reshape(-1, 6)
    E = np.ascontiguousarray(E, dtype=np.float64).reshape(-1)
    L_z = np.ascontiguousarray(L_z, dtype=np.float64).reshape(-1)
    n = states.shape[0]
    arrs, out = _alloc(n)
    o = options(**opt)
    lb.oracle_trace_states(M, a, r_obs, ctypes.byref(o), _ptr(states, _d), _ptr(E, _d),
                           _ptr(L_z, _d), n, ctypes.byref(out))
    return arrs


def init_ray(a, r_obs, incl_deg, x, y, M=1.0):
    """(t, r, theta, phi, p_r, p_theta, E, L) for image-plane point (x, y) (Sec. 2.3)."""
    out = np.zeros(8)
    lib().oracle_init_ray(M, a, r_obs, incl_deg, x, y, _ptr(out, _d))
    return out


def metric_cov(a, r, th, M=1.0):
    g = np.zeros(16)
    lib().oracle_metric_cov(M, a, r, th, _ptr(g, _d))
    return g.reshape(4, 4)


def metric_con(a, r, th, M=1.0):
    g = np.zeros(16)
    lib().oracle_metric_con(M, a, r, th, _ptr(g, _d))
    return g.reshape(4, 4)


def metric_con_derivs(a, r, th, M=1.0):
    dr = np.zeros(16)
    dth = np.zeros(16)
    lib().oracle_metric_con_derivs(M, a, r, th, _ptr(dr, _d), _ptr(dth, _d))
    return dr.reshape(4, 4), dth.reshape(4, 4)


def hamiltonian(a, y6, E, L_z, M=1.0):
    y6 = np.ascontiguousarray(y6, dtype=np.float64)
    return lib().oracle_hamiltonian(M, a, _ptr(y6, _d), E, L_z)


def rhs(a, y6, E, L_z, M=1.0):
    y6 = np.ascontiguousarray(y6, dtype=np.float64)
    dy = np.zeros(6)
    lib().oracle_rhs(M, a, _ptr(y6, _d), E, L_z, _ptr(dy, _d))
    return dy


def ck_step(a, y6, E, L_z, h, M=1.0):
    y6 = np.ascontiguousarray(y6, dtype=np.float64)
    y5 = np.zeros(6)
    d = np.zeros(6)
    lib().oracle_ck_step(M, a, _ptr(y6, _d), E, L_z, h, _ptr(y5, _d), _ptr(d, _d))
    return y5, d


def rk_step(integrator, a, y6, E, L_z, h, M=1.0):
    """One step of the chosen embedded pair (Sec. 3.1): (y5, y5 - y4)."""
    y6 = np.ascontiguousarray(y6, dtype=np.float64)
    y5 = np.zeros(6)
    d = np.zeros(6)
    lib().oracle_rk_step(int(integrator), M, a, _ptr(y6, _d), E, L_z, h, _ptr(y5, _d),
                         _ptr(d, _d))
    return y5, d


def tableau(integrator):
    """(stages, c, A, b5, b4) of an integrator (7-entry arrays, zero padded)."""
    c = np.zeros(7)
    A = np.zeros(49)
    b5 = np.zeros(7)
    b4 = np.zeros(7)
    n = lib().oracle_tableau(int(integrator), _ptr(c, _d), _ptr(A, _d), _ptr(b5, _d),
                             _ptr(b4, _d))
    return n, c, A.reshape(7, 7), b5, b4


def ck_tableau():
    c = np.zeros(6)
    A = np.zeros(36)
    b5 = np.zeros(6)
    b4 = np.zeros(6)
    lib().oracle_ck_tableau(_ptr(c, _d), _ptr(A, _d), _ptr(b5, _d), _ptr(b4, _d))
    return c, A.reshape(6, 6), b5, b4


def disk_observables(a, r, E, L_z, M=1.0):
    g = _d()
    I = _d()
    lib().oracle_disk_observables(M, a, r, E, L_z, ctypes.byref(g), ctypes.byref(I))
    return g.value, I.value


def disk_observables_l0(a, r, E, L_z, l0, M=1.0):
    """(g, I) on a disk of constant specific angular momentum l0 (Sec. 5)."""
    g = _d()
    I = _d()
    lib().oracle_disk_observables_l0(M, a, r, E, L_z, l0, ctypes.byref(g), ctypes.byref(I))
    return g.value, I.value


def metric_sp(kind, r, th, a=0.0, q=0.0, M=1.0):
    """(g_cov, g_con, d_r g_con, d_theta g_con) for Kerr (kind 0) or the q-metric (1)."""
    out = [np.zeros(16) for _ in range(4)]
    lib().oracle_metric_sp(kind, M, a, q, r, th, *[_ptr(o, _d) for o in out])
    return tuple(o.reshape(4, 4) for o in out)


def hamiltonian_sp(kind, y6, E, L_z, a=0.0, q=0.0, M=1.0):
    y6 = np.ascontiguousarray(y6, dtype=np.float64)
    return lib().oracle_hamiltonian_sp(kind, M, a, q, _ptr(y6, _d), E, L_z)


def rhs_sp(kind, y6, E, L_z, a=0.0, q=0.0, M=1.0):
    y6 = np.ascontiguousarray(y6, dtype=np.float64)
    dy = np.zeros(6)
    lib().oracle_rhs_sp(kind, M, a, q, _ptr(y6, _d), E, L_z, _ptr(dy, _d))
    return dy


def init_ray_sp(kind, r_obs, incl_deg, x, y, a=0.0, q=0.0, M=1.0):
    out = np.zeros(8)
    lib().oracle_init_ray_sp(kind, M, a, q, r_obs, incl_deg, x, y, _ptr(out, _d))
    return out


def isco(a, M=1.0):
    return lib().oracle_isco(M, a)
