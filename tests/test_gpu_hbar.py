"""The |H| bar (Sec. 3.1 reports the integration error as |H_num|; the target
asks for |H| below 1e-10) on four of the benchmark's Kerr renders (a = 0.9 and
0.998 at 17 and 60 degrees, 256x256 on [-8, 8]^2), per class of ray, as
measured on the full 12-render set and stated in the design notes:

  Cash-Karp, tol 1e-10
    escaped rays: p99 of max |H| below 1e-9, max below 2e-8;
    captured rays: |H| grows next to the horizon with the terms of 2H
      (P^2 / Delta ~ 1e4 at the 1.01 r_H buffer of a = 0.998), so the bound
      is relative: max |H| Delta Sigma / P^2 at the capture point (|2H|
      over the summed magnitude of its terms, which is 2 P^2 / (Delta Sigma)
      on the constraint surface) below 5e-9;
  Cash-Karp, tol 1e-12: every escaped ray below 1e-10 (the bar);
  Dormand-Prince, tol 1e-12: captured rays' normalised |H| below 5e-11.
|H| scales with tol, and Dormand-Prince keeps it ~10x lower than Cash-Karp
at the same tol (Sec. 3.1-3.2)."""
import numpy as np
import pytest
import torch

import paper_2202_00086_gb300 as osr
from paper_2202_00086_gb300 import workloads

pytestmark = pytest.mark.gpu

BAR = 1e-10


def _renders():
    return [workloads.render(a, 1000.0, inc, (-8, 8, -8, 8), 256, 256)
            for a in (0.9, 0.998) for inc in (17.0, 60.0)]


def _trace(rds, tol, integrator):
    outs = []
    cams = [osr.Camera.from_render(rd) for rd in rds]
    outs = [osr.alloc_outputs(c.n_rays) for c in cams]
    ws = torch.empty(osr.workspace_bytes(len(cams)), dtype=torch.uint8, device="cuda")
    osr.trace_batch([{"camera": c, "out": o} for c, o in zip(cams, outs)], workspace=ws,
                    tol=tol, integrator=integrator, cell_phase_deg=rds[0]["cell_phase_deg"])
    torch.cuda.synchronize()
    return [{k: v.cpu().numpy() for k, v in o.items()} for o in outs]


def _captured_normalised(rd, o):
    """max |H| Delta Sigma / P^2 at the capture point; E and L of each pixel
    from the zero-angular-momentum observer of Sec. 2.3 (Kerr metric at the
    observer)."""
    cap = o["status"] == osr.STATUS_CAPTURED
    a, r0, th0 = rd["a"], rd["r_obs"], np.radians(rd["incl_deg"])
    x0, x1, _, _ = rd["extent"]
    idx = np.flatnonzero(cap)
    x = x0 + (idx % rd["nx"] + 0.5) * (x1 - x0) / rd["nx"]
    s2, c2 = np.sin(th0) ** 2, np.cos(th0) ** 2
    sig0, dlt0 = r0 * r0 + a * a * c2, r0 * r0 - 2 * r0 + a * a
    g_tph = -2 * a * r0 * s2 / sig0
    g_pp = s2 * ((r0 * r0 + a * a) ** 2 - a * a * dlt0 * s2) / sig0
    E = np.sqrt(dlt0 * s2 / g_pp) + x * g_tph / (r0 * np.sqrt(g_pp))
    L = -x * np.sqrt(g_pp) / r0
    r, c = o["r"][idx], np.cos(o["theta"][idx])
    sig, dlt = r * r + a * a * c * c, r * r - 2 * r + a * a
    P = (r * r + a * a) * E - a * L
    return o["max_abs_H"][idx] * dlt * sig / (P * P)


def _by_class(rds, outs):
    st = np.concatenate([o["status"] for o in outs])
    h = np.concatenate([o["max_abs_H"] for o in outs])
    norm = np.concatenate([_captured_normalised(rd, o) for rd, o in zip(rds, outs)])
    return h[st == osr.STATUS_ESCAPED], h[st == osr.STATUS_CAPTURED], norm


def test_hbar_cash_karp_tol_1e10():
    rds = _renders()
    esc, cap, norm = _by_class(rds, _trace(rds, 1e-10, osr.RKCK45))
    assert esc.size > 50000 and cap.size > 20000
    print("CK45 1e-10: escaped p50 %.2e p99 %.2e max %.2e; captured max %.2e, normalised "
          "max %.2e" % (np.median(esc), np.percentile(esc, 99), esc.max(), cap.max(), norm.max()))
    assert np.percentile(esc, 99) < 1e-9 and esc.max() < 2e-8
    assert norm.max() < 5e-9
    assert cap.max() > BAR  # next to the horizon the absolute |H| does not meet the bar


def test_hbar_met_by_escaped_rays_at_tol_1e12():
    rds = _renders()
    esc, cap, norm = _by_class(rds, _trace(rds, 1e-12, osr.RKCK45))
    print("CK45 1e-12: escaped max %.2e; captured max %.2e, normalised max %.2e"
          % (esc.max(), cap.max(), norm.max()))
    assert esc.max() < BAR
    assert norm.max() < 5e-11 * 10  # |H| scales with tol: 1e-2 of the tol-1e-10 bound


def test_hbar_dormand_prince_tol_1e12():
    rds = _renders()
    esc, cap, norm = _by_class(rds, _trace(rds, 1e-12, osr.RKDP45))
    print("DP45 1e-12: escaped max %.2e; captured max %.2e (%.3f below the bar), normalised "
          "max %.2e" % (esc.max(), cap.max(), (cap < BAR).mean(), norm.max()))
    assert esc.max() < BAR
    assert norm.max() < 5e-11
