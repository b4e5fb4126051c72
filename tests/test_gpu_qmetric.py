"""The q-metric (Appendix A) and time-like geodesics on the GPU, against the
oracle, in FP64 and in double-float (DF64): q-metric shadow renders (q = 0
equal to the Kerr a = 0 render), circular and escaping massive particles,
and the mass-shell error; and q-metric renders in MIXED (FP32 evaluations) at
tol 1e-8 against the oracle at 1e-10, within MIXED's stated bound."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2202_00086_gb300 as osr
from paper_2202_00086_gb300 import workloads

from _parity import assert_parity, compare, gpu_render, oracle_render, oracle_sampled

pytestmark = pytest.mark.gpu


PRECISIONS = [osr.FP64, osr.DF64]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("q", [-0.5, 0.1, 0.5])
@pytest.mark.parametrize("inc", [30.0, 90.0])
def test_qmetric_render_parity(q, inc, precision):
    rd = workloads.render(0.0, 1000.0, inc, (-8, 8, -8, 8), 32, 32, q=q)
    rep = compare(rd, gpu_render(rd, precision=precision), oracle_render(rd),
                  precision=precision)
    print(rep)
    assert_parity(rep)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_qmetric_q0_equals_schwarzschild_on_gpu(precision):
    rq = workloads.render(0.0, 1000.0, 60.0, (-8, 8, -8, 8), 24, 24, q=0.0)
    rk = workloads.render(0.0, 1000.0, 60.0, (-8, 8, -8, 8), 24, 24)
    gq, gk = gpu_render(rq, precision=precision), gpu_render(rk, precision=precision)
    assert np.array_equal(gq["status"], gk["status"])
    for key in ("r", "theta", "phi"):
        assert np.allclose(gq[key], gk[key], rtol=1e-9, atol=1e-9)


def _line_element(q, r):
    """g_tt, g_rr, g_phph of the q-metric on the equator (sin = 1)."""
    f = 1 - 2 / r
    X = 1 + 1 / (r * r - 2 * r)
    k = q * (2 + q)
    return -f ** (1 + q), f ** (-1 - q) * X ** -k, f ** -q * r * r


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("q", [0.0, 0.5, -0.5])
def test_timelike_orbits_parity(q, precision):
    r = 12.0
    # circular orbit from the covariant metric: Omega^2 = -d g_tt / d g_phph
    h = 1e-5 * r
    gp, gm = _line_element(q, r + h), _line_element(q, r - h)
    Om = math.sqrt(-(gp[0] - gm[0]) / (gp[2] - gm[2]))
    g = _line_element(q, r)
    ut = 1 / math.sqrt(-g[0] - g[2] * Om * Om)
    Ec, Lc = -g[0] * ut, g[2] * Om * ut
    # an unbound particle launched outwards from r = 30
    g30 = _line_element(q, 30.0)
    Eu, Lu = 1.2, 4.0
    pru = math.sqrt((-1 + Eu * Eu / -g30[0] - Lu * Lu / g30[2]) * g30[1])
    st = np.array([[0.0, r, math.pi / 2, 0.0, 0.0, 0.0], [0.0, 30.0, math.pi / 2, 0.0, pru, 0.0]])
    E = np.array([Ec, Eu])
    L = np.array([Lc, Lu])
    out = osr.trace_states(0.0, 100.0, torch.tensor(st, device="cuda"),
                           torch.tensor(E, device="cuda"), torch.tensor(L, device="cuda"),
                           q=q, mass2=1.0, max_steps=150, precision=precision)
    torch.cuda.synchronize()
    ref = oracle.trace_states(0.0, 100.0, st, E, L, spacetime=oracle.QMETRIC, q=q, mass2=1.0,
                              max_steps=150)
    got = {k: v.cpu().numpy() for k, v in out.items()}
    assert got["status"].tolist() == ref["status"].tolist() == [osr.STATUS_MAXSTEP,
                                                               osr.STATUS_ESCAPED]
    assert abs(got["r"][0] - r) < 1e-6 * r  # stays on the circular orbit
    for key in ("r", "theta", "phi"):  # the escape point is located exactly
        assert abs(got[key][1] - ref[key][1]) <= 1e-8 * max(1.0, abs(ref[key][1])), key
    assert got["max_abs_H"].max() < 1e-8
    # the DF64 kernels track |H - H0| from double-float sums: the same size,
    # not the same rounding
    rtol = 0.05 if precision == osr.FP64 else 0.5
    assert np.allclose(got["max_abs_H"], ref["max_abs_H"], rtol=rtol, atol=1e-13)


def test_qmetric_rejects_a_disk():
    cam = osr.Camera(0.0, 1000.0, 60.0, (-8, 8, -8, 8), 8, 8, q=0.5)
    with pytest.raises(osr.OsirisError):
        osr.render_disk(cam, 6.0, 20.0)


@pytest.mark.parametrize("q,inc", [(0.5, 60.0), (-0.5, 30.0), (0.1, 90.0)])
def test_qmetric_mixed_error_bound(q, inc):
    rd = dict(workloads.render(0.0, 1000.0, inc, (-8, 8, -8, 8), 32, 32, q=q), tol=1e-8)
    ref = oracle_render(dict(rd, tol=1e-10))
    rep = compare(rd, gpu_render(rd, precision=osr.MIXED), ref, coord_rtol=1e-5,
                  precision=osr.MIXED)
    print(rep)
    assert_parity(rep)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_qmetric_batch_equals_single_calls(precision):
    """q-metric renders in one batched persistent launch give the outputs of
    the same renders traced one by one, and a batch may not mix space-times."""
    rds = [workloads.render(0.0, 1000.0, inc, (-8, 8, -8, 8), 20, 16, q=q)
           for q, inc in ((0.5, 30.0), (-0.5, 60.0), (0.1, 90.0))]
    cams = [osr.Camera.from_render(rd) for rd in rds]
    outs = [osr.alloc_outputs(c.n_rays) for c in cams]
    reqs = [{"camera": c, "out": o, "tol": rd["tol"]} for c, o, rd in zip(cams, outs, rds)]
    ws = torch.empty(osr.workspace_bytes(len(reqs)), dtype=torch.uint8, device="cuda")
    osr.trace_batch(reqs, workspace=ws, cell_deg=rds[0]["cell_deg"],
                    cell_phase_deg=rds[0]["cell_phase_deg"], precision=precision)
    torch.cuda.synchronize()
    for rd, o in zip(rds, outs):
        alone = gpu_render(rd, precision=precision)
        for f in alone:
            assert np.array_equal(o[f].cpu().numpy(), alone[f]), f
    kerr = osr.Camera.from_render(workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 4, 4))
    mixed = reqs[:1] + [{"camera": kerr, "out": osr.alloc_outputs(16), "tol": 1e-10}]
    with pytest.raises(osr.OsirisError) as e:
        osr.trace_batch(mixed, workspace=ws, precision=precision)
    assert e.value.code == osr.EINVAL


@pytest.mark.parametrize("precision", PRECISIONS)
def test_full_size_qmetric_batch_sampled(precision):
    """The six 1024^2 q-metric renders (q in {-0.5, 0.1, 0.5} x inclination
    {30, 90} deg) in one batched launch, as they are timed; 40 sampled pixels
    per render against the oracle."""
    rds = [workloads.render(0.0, 1000.0, inc, (-8, 8, -8, 8), 1024, 1024, q=q)
           for q in (-0.5, 0.1, 0.5) for inc in (30.0, 90.0)]
    cams = [osr.Camera.from_render(rd) for rd in rds]
    outs = [osr.alloc_outputs(c.n_rays) for c in cams]
    ws = torch.empty(osr.workspace_bytes(len(cams)), dtype=torch.uint8, device="cuda")
    osr.trace_batch([{"camera": c, "out": o, "tol": rd["tol"]}
                     for c, o, rd in zip(cams, outs, rds)], workspace=ws, precision=precision,
                    cell_deg=rds[0]["cell_deg"], cell_phase_deg=rds[0]["cell_phase_deg"])
    torch.cuda.synchronize()
    rng = np.random.default_rng(21)
    for rd, o in zip(rds, outs):
        gpu = {k: v.cpu().numpy() for k, v in o.items()}
        pix = np.sort(rng.choice(1024 * 1024, 40, replace=False))
        ref, band = oracle_sampled(rd, pix)
        rep = compare(rd, gpu, ref, pixels=pix, band=band, precision=precision)
        print(rep)
        assert_parity(rep)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("q", [-0.3, 0.1, 0.5])
def test_qmetric_light_ring_on_gpu(q, precision):
    """The equatorial light ring of the q-metric, r = 3 + 2q with
    b = r f^-(1+2q)/2 (the extremum of b^2 = g_phph / -g_tt): a photon started
    on it stays on it through 60 steps."""
    r = 3.0 + 2.0 * q
    b = r * (1.0 - 2.0 / r) ** (-(1.0 + 2.0 * q) / 2.0)
    st = torch.tensor([[0.0, r, math.pi / 2, 0.0, 0.0, 0.0]], device="cuda", dtype=torch.float64)
    out = osr.trace_states(0.0, 1000.0, st, torch.ones(1, device="cuda", dtype=torch.float64),
                           torch.full((1,), b, device="cuda", dtype=torch.float64), q=q,
                           max_steps=60, precision=precision)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    assert got["status"][0] == osr.STATUS_MAXSTEP
    assert abs(got["r"][0] - r) < 1e-8
    assert got["phi"][0] > 1.0  # it went round
    assert got["max_abs_H"][0] < 1e-12


@pytest.mark.parametrize("q", [None, 0.5])
def test_mixed_timelike_particles(q):
    """Unit-mass particles (H = -1/2) in MIXED at tol 1e-8, Kerr a = 0.9 or the
    q-metric, launched outwards from r = 30 with the bench's recipe: the same
    fates as the oracle at 1e-10 and escape points within 1e-5; the end-point
    |H + 1/2| comes from the double-float equations."""
    rng = np.random.default_rng(31)
    n = 64
    a = 0.0 if q is not None else 0.9
    E = np.full(n, 1.2)
    L = rng.uniform(-4.0, 4.0, n)
    # the q-metric particles start on the equator, where _line_element holds
    th = rng.uniform(0.3, math.pi - 0.3, n) if q is None else np.full(n, math.pi / 2)
    r0 = 30.0
    st = np.zeros((n, 6))
    st[:, 1], st[:, 2] = r0, th
    for i in range(n):  # outward p_r on the mass shell H = -1/2, p_theta = 0
        if q is None:
            s2 = math.sin(th[i]) ** 2
            sig = r0 * r0 + a * a * (1 - s2)
            dlt = r0 * r0 - 2 * r0 + a * a
            A = (r0 * r0 + a * a) ** 2 - a * a * dlt * s2
            gtt, gtp = -A / (sig * dlt), -2 * a * r0 / (sig * dlt)
            gpp = (dlt - a * a * s2) / (sig * dlt * s2)
            grr = dlt / sig
            rest = gtt * E[i] ** 2 - 2 * gtp * E[i] * L[i] + gpp * L[i] ** 2 + 1.0
        else:
            g = _line_element(q, r0)
            grr = 1.0 / g[1]
            rest = E[i] ** 2 / g[0] + L[i] ** 2 / (g[2] * math.sin(th[i]) ** 2) + 1.0
        st[i, 4] = math.sqrt(max(0.0, -rest / grr))
    kw = dict(q=q) if q is not None else {}
    dev = [torch.tensor(x, device="cuda") for x in (st, E, L)]
    out = osr.trace_states(a, 100.0, *dev, mass2=1.0, tol=1e-8, precision=osr.MIXED, **kw)
    torch.cuda.synchronize()
    okw = dict(spacetime=oracle.QMETRIC, q=q) if q is not None else {}
    ref = oracle.trace_states(a, 100.0, st, E, L, mass2=1.0, **okw)
    got = {k: v.cpu().numpy() for k, v in out.items()}
    assert got["status"].tolist() == ref["status"].tolist()
    esc = ref["status"] == oracle.STATUS_ESCAPED
    assert esc.sum() > n // 2
    for key in ("r", "theta", "phi"):
        err = np.abs(got[key][esc] - ref[key][esc])
        assert np.all(err <= 1e-5 * np.maximum(1.0, np.abs(ref[key][esc]))), (key, err.max())
    assert np.all(got["max_abs_H"][esc] < 1e-5)

