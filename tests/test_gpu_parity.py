"""GPU-vs-oracle parity of the FP64 path, through the C interface.

Every case runs the same seeded render on the GPU (libosiris.so) and in the
CPU oracle and compares them element by element (rules in tests/_parity.py).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2202_00086_gb300 as osr
from paper_2202_00086_gb300 import workloads

from _parity import assert_parity, band_mask, compare, gpu_render, oracle_render, oracle_sampled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    osr.lib()


def _check(rd, **kw):
    gpu = gpu_render(rd, **kw)
    ref = oracle_render(rd)
    rep = compare(rd, gpu, ref)
    print(rep)
    assert_parity(rep)
    return gpu, ref, rep


def test_schwarzschild_shadow_64_fp64():
    rd = workloads.schwarzschild_shadow_64()
    gpu, ref, rep = _check(rd)
    assert rep["compared"] > 3500
    assert rep["steps_equal_frac"] > 0.95
    # the exact shadow edge rho_c = 3 sqrt(3) sqrt(1 - 2/r0)
    n = rd["nx"]
    xs = -10 + (np.arange(n) + 0.5) * 20 / n
    rho = np.hypot(xs[None, :], xs[:, None]).reshape(-1)
    cap = gpu["status"] == osr.STATUS_CAPTURED
    rho_c = 3 * math.sqrt(3) * math.sqrt(1 - 2 / 1000.0)
    keep = ~band_mask((rho < rho_c).reshape(n, n)).reshape(-1)
    assert np.array_equal(cap[keep], (rho < rho_c)[keep])


def test_persistent_matches_plain_bitwise():
    rd = workloads.render(0.9, 1000.0, 60.0, (-8, 8, -8, 8), 61, 47)
    a = gpu_render(rd, persistent=False)
    b = gpu_render(rd, persistent=True)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("a", workloads.KERR_SPINS)
@pytest.mark.parametrize("inc", workloads.KERR_INCLINATIONS)
def test_kerr_shadow_ring_subsampled(a, inc):
    # same extent and checkerboard as the 1024^2 set, 40x40 cell centres
    rd = workloads.render(a, 1000.0, inc, (-8, 8, -8, 8), 40, 40)
    _check(rd)


def test_kerr_ragged_sizes_and_block_shapes():
    rd = workloads.render(0.998, 1000.0, 17.0, (-8, 8, -8, 8), 37, 29)
    ref = oracle_render(rd)
    for block in (32, 96, 256):
        gpu = gpu_render(rd, block_size=block)
        assert_parity(compare(rd, gpu, ref))


def test_single_pixel_and_odd_grid():
    # 1x1: the ray through the image centre; 5x3 with x = 0 exactly (L = 0)
    for nx, ny in ((1, 1), (5, 3)):
        rd = workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), nx, ny)
        _check(rd)


def test_schwarzschild_disk_subsampled():
    rd = workloads.schwarzschild_disk(side=64)
    gpu, ref, rep = _check(rd)
    assert rep["n_disk"] > 300


def test_kerr_disk_isco():
    rd = workloads.render(0.9, 1000.0, 60.0, (-25, 25, -25, 25), 48, 48, mode="disk",
                          r_in="isco", r_out=20.0)
    gpu, ref, rep = _check(rd)
    assert rep["n_disk"] > 100


def test_max_steps_cap_matches_oracle():
    rd = workloads.render(0.9, 1000.0, 60.0, (-8, 8, -8, 8), 16, 16)
    gpu = gpu_render(rd, max_steps=40)
    ref = oracle_render(rd, max_steps=40)
    assert np.array_equal(gpu["status"], ref["status"])
    ms = ref["status"] == oracle.STATUS_MAXSTEP
    assert ms.sum() > 0
    assert np.array_equal(gpu["steps"][ms].astype(np.int64), ref["accepted"][ms])
    # A capped ray stops wherever its budget ran out: the affine parameter
    # reached is the sum of the step lengths, which the kernel sizes in FP32
    # (relative 1e-7 from the oracle's FP64 controller), so the end points lie
    # on the same curve but not at the same parameter.
    for key in ("r", "theta", "phi"):
        assert np.allclose(gpu[key][ms], ref[key][ms], rtol=1e-5, atol=1e-6)


def test_explicit_states_hook():
    """Printed initial conditions of Sec. 3.1 and the photon-sphere orbit."""
    st = np.array([oracle.init_ray(0.98, 100.0, 90.0, -2.0, 1.87),
                   oracle.init_ray(0.98, 100.0, 90.0, -1.25, 3.75)])
    states = torch.tensor(st[:, :6], device="cuda").contiguous()
    E = torch.tensor(st[:, 6], device="cuda")
    L = torch.tensor(st[:, 7], device="cuda")
    out = osr.trace_states(0.98, 100.0, states, E, L)
    torch.cuda.synchronize()
    ref = oracle.trace_states(0.98, 100.0, st[:, :6], st[:, 6], st[:, 7])
    assert out["status"].cpu().numpy().tolist() == ref["status"].tolist()
    assert ref["status"].tolist() == [oracle.STATUS_CAPTURED, oracle.STATUS_ESCAPED]
    for key in ("r", "theta", "phi"):
        g = out[key].cpu().numpy()
        assert np.allclose(g, ref[key], rtol=1e-8, atol=1e-8), key
    # photon sphere: r stays at 3 while the step cap runs out
    b = 3 * math.sqrt(3)
    s = torch.tensor([[0.0, 3.0, math.pi / 2, 0.0, 0.0, 0.0]], device="cuda", dtype=torch.float64)
    o = osr.trace_states(0.0, 1000.0, s, torch.ones(1, device="cuda", dtype=torch.float64),
                         torch.full((1,), b, device="cuda", dtype=torch.float64), max_steps=60)
    torch.cuda.synchronize()
    assert int(o["status"][0]) == osr.STATUS_MAXSTEP
    assert abs(float(o["r"][0]) - 3.0) < 1e-8


@pytest.mark.parametrize("precision", [osr.FP64, osr.DF64])
def test_kerr_spherical_photon_orbits(precision):
    """Kerr spherical photon orbits (closed-form constants, see the oracle pin
    of the same name) traced on the GPU: r stays fixed to 1e-8 over 800 steps,
    theta stays inside its turning points, |H| stays small, and the final r
    agrees with the oracle's."""
    from test_oracle_pins import spherical_photon_orbit
    rows, E, L, cases = [], [], [], []
    for a in (0.5, 0.9, 0.998):
        for f in (0.25, 0.5, 0.75):
            r, xi, eta, u_plus = spherical_photon_orbit(a, f)
            cases.append((a, r, xi, eta, u_plus))
    for a, r, xi, eta, u_plus in cases:
        st = np.array([[0.0, r, math.pi / 2, 0.0, 0.0, math.sqrt(eta)]])
        o = osr.trace_states(a, 1000.0, torch.tensor(st, device="cuda"),
                             torch.ones(1, device="cuda", dtype=torch.float64),
                             torch.full((1,), xi, device="cuda", dtype=torch.float64),
                             max_steps=800, tol=1e-12, precision=precision)
        torch.cuda.synchronize()
        ref = oracle.trace_states(a, 1000.0, st, [1.0], [xi], max_steps=800, tol=1e-12)
        assert int(o["status"][0]) == osr.STATUS_MAXSTEP
        rg = float(o["r"][0])
        assert abs(rg - r) < 1e-8 * r, (a, r, rg)
        assert abs(rg - ref["r"][0]) < 1e-8 * r
        assert math.cos(float(o["theta"][0])) ** 2 <= u_plus * (1 + 1e-7)
        assert float(o["max_abs_H"][0]) < 1e-9


def test_stats_counters():
    rd = workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 32, 32)
    stats = osr.new_stats()
    gpu = gpu_render(rd, stats=stats)
    s = osr.decode_stats(stats)
    assert s["rays"] == 32 * 32
    counts = np.bincount(gpu["status"], minlength=6)
    assert s["status_captured"] == counts[1] and s["status_escaped"] == counts[2]
    assert s["accepted"] == int(gpu["steps"].astype(np.int64).sum())
    assert s["rhs_evals"] == 6 * (s["accepted"] + s["rejected"] + s["root_steps"]) + s["rays"]
    assert s["max_abs_H"] == pytest.approx(float(gpu["max_abs_H"].max()), rel=0, abs=0)


def test_invalid_arguments_rejected():
    cam = osr.Camera(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 8, 8)
    with pytest.raises(osr.OsirisError) as e:
        osr.trace(cam, tol=0.0)
    assert e.value.code == osr.EINVAL
    with pytest.raises(osr.OsirisError):
        osr.render_disk(cam, 1.0, 20.0)  # r_in inside the capture radius
    with pytest.raises(osr.OsirisError) as e:
        osr.trace(cam, persistent=True)  # no workspace
    assert e.value.code == osr.ENOMEM


def test_full_size_kerr_sampled():
    """1024^2 render (a = 0.998, 60 deg) in the benchmark's launch
    configuration; 600 sampled pixels checked against the oracle one by one."""
    rd = workloads.kerr_shadow_ring_set(1024)[3 * 3 + 1]
    assert rd["a"] == 0.998 and rd["incl_deg"] == 60.0
    gpu = gpu_render(rd, persistent=True)
    rng = np.random.default_rng(11)
    pix = np.sort(rng.choice(1024 * 1024, 600, replace=False))
    ref, band = oracle_sampled(rd, pix)
    rep = compare(rd, gpu, ref, pixels=pix, band=band)
    print(rep)
    assert_parity(rep)


@pytest.mark.parametrize("precision", [osr.FP64, osr.DF64])
def test_full_size_schwarzschild_disk_sampled(precision):
    """The 2048^2 Schwarzschild thin disk (r_in = 6, r_out = 20, 80 deg) in
    one persistent launch; 2000 sampled pixels checked against the oracle one
    by one, over 200 of them disk hits (g, intensity, r_hit)."""
    rd = workloads.schwarzschild_disk()
    assert rd["nx"] == rd["ny"] == 2048
    gpu = gpu_render(rd, precision=precision, persistent=True)
    assert int((gpu["status"] == 0).sum()) == 0
    rng = np.random.default_rng(13)
    pix = np.sort(rng.choice(2048 * 2048, 2000, replace=False))
    ref, band = oracle_sampled(rd, pix)
    rep = compare(rd, gpu, ref, pixels=pix, band=band, precision=precision)
    print(rep)
    assert_parity(rep)
    assert rep["n_disk"] > 200


@pytest.mark.parametrize("precision", [osr.FP64, osr.DF64])
def test_kerr_escape_points_against_first_integrals(precision):
    """The GPU's end points of generic Kerr rays (a = 0.9, 0.998, 0.5;
    inclinations 60, 17, 90 deg; escaping and captured), traced at tol 1e-12
    from the oracle's initial data, against their exact end points from the
    quadratures of the first integrals (tests/golden/kerr_end_points.json,
    written by its script from oracle/first_integrals.py): cos theta and phi
    within 1e-8 (the oracle's own integration agrees to 2.4e-11)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "kerr_end_points.json")) as f:
        rays = json.load(f)["rays"]
    for a in sorted({r["a"] for r in rays}):
        rows = [r for r in rays if r["a"] == a]
        st = np.array([oracle.init_ray(a, 1000.0, r["incl_deg"], r["x"], r["y"]) for r in rows])
        out = osr.trace_states(a, 1000.0, torch.tensor(st[:, :6], device="cuda").contiguous(),
                               torch.tensor(st[:, 6], device="cuda"),
                               torch.tensor(st[:, 7], device="cuda"), tol=1e-12,
                               precision=precision)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        for k, r in enumerate(rows):
            fate = osr.STATUS_ESCAPED if r["fate"] == "escaped" else osr.STATUS_CAPTURED
            assert got["status"][k] == fate, (a, r)
            assert abs(math.cos(got["theta"][k]) - r["cos_theta"]) < 1e-8, (a, r)
            assert abs(got["phi"][k] - r["phi"]) < 1e-8 * max(1.0, abs(r["phi"])), (a, r)
