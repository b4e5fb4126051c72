"""Helpers that run the same seeded render through the CUDA library and the
CPU oracle and compare them element by element.

Comparison rules (the parity bar):
  - status: identical outside the one-pixel band around the critical curve
    and other fate boundaries, i.e. pixels whose 3x3 neighbourhood in the
    reference status image holds more than one status are excluded;
  - final r, theta, phi: |gpu - ref| <= 1e-8 max(1, |ref|) (relative, with a
    unit floor for angles near zero);
  - checkerboard cell: identical where the reference angles are further than
    1e-6 rad from a cell boundary;
  - disk: g, intensity, r_hit within 1e-8 relative;
  - max |H| (Sec. 3.1, Error = |H_num|): |H_gpu - H_ref| <= H_RTOL |H_ref| +
    H_EPS T, where T is the sum of the magnitudes of the terms of 2H at the
    oracle's end point (for Kerr (Delta p_r^2 + p_theta^2 + W^2 + P^2/Delta) /
    Sigma). |H| is the small remainder of terms of size T, so two correct
    integrations whose states agree to a relative d differ in |H| by about
    d T: d ~ 1e-13 for FP64 (a few hundred steps of 2^-53 rounding), ~1e-11
    for the double-float state (2^-48 per operation). Next to the horizon of
    a = 0.998, T reaches 1e4-1e5 while Dormand-Prince keeps |H| near 1e-8,
    so there the second term decides (measured worst over the GPU suite: 0.44 of the
    bound in FP64, 0.31 in double-float);
  - accepted-step counts: the FP64 kernels take the oracle's accept/reject
    decision on every step (their error test is exact in FP64 near the
    threshold), so their counts equal the oracle's on all but a stated share
    of the rays (STEPS_ALLOW); the double-float kernels take a few decisions
    differently (their error estimate has a floor near 1e-12 of 1 + |y|), so
    every ray's count is within 4 + 1% of the oracle's (measured: within 4, 0.58 of
    the bound).

Sampled comparisons at full size take the band from the oracle too: each
sampled pixel's 3x3 neighbourhood is traced by the oracle
(`oracle_sampled`), never read from the GPU image.
"""
import math

import numpy as np
import torch

import oracle
import paper_2202_00086_gb300 as osr

COORD_RTOL = 1e-8
G_RTOL = 1e-8
CELL_MARGIN = 1e-6
# max |H| against the oracle: |dH| <= H_RTOL |H_ref| + H_EPS T (see above)
H_RTOL = {osr.FP64: 1e-3, osr.DF64: 0.25}
H_EPS = {osr.FP64: 1e-12, osr.DF64: 1e-10}
# FP64: rays whose accepted-step count may differ from the oracle's (a share
# of the compared rays plus a fixed count, for small samples); DF64: largest
# difference per ray (a fixed count plus a share of the oracle's count)
STEPS_ALLOW = {osr.FP64: (0.002, 1), osr.DF64: (4, 0.01)}


def band_mask(status_img):
    """True where the 3x3 neighbourhood of a pixel holds more than one status."""
    f = status_img.astype(np.int64)
    ny, nx = f.shape
    pad = np.pad(f, 1, mode="edge")
    lo = np.full_like(f, 1 << 30)
    hi = np.full_like(f, -1)
    for dj in range(3):
        for di in range(3):
            w = pad[dj:dj + ny, di:di + nx]
            lo = np.minimum(lo, w)
            hi = np.maximum(hi, w)
    return lo != hi


def neighbourhood(nx, ny, pixels):
    """(9, n) linear indices of the 3x3 neighbourhood of each pixel; beyond
    the image edge the nearest edge pixel stands in (as in band_mask)."""
    pixels = np.asarray(pixels, dtype=np.int64)
    i, j = pixels % nx, pixels // nx
    rows = []
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            rows.append(np.clip(j + dj, 0, ny - 1) * nx + np.clip(i + di, 0, nx - 1))
    return np.stack(rows)


def terms_of_2H(rd, ref):
    """Sum of the magnitudes of the terms of 2H = g^{mu nu} p_mu p_nu at the
    oracle's end point of each ray (p_t = -E, p_phi = L), the scale of the
    rounding in |H|: Kerr (Sec. 4.3) in the separated form, the q-metric
    (Appendix A) term by term."""
    r, th = ref["r"], ref["theta"]
    pr, pth, E, L = ref["p_r"], ref["p_theta"], ref["E"], ref["L"]
    s, c = np.sin(th), np.cos(th)
    s = np.where(np.abs(s) < 1e-300, 1e-300, s)
    if rd.get("q") is not None:
        q = rd["q"]
        k = q * (2.0 + q)
        f = 1.0 - 2.0 / r
        X = 1.0 + s * s / (r * r - 2.0 * r)
        fa = np.abs(f)
        return (E * E / fa ** (1.0 + q) + fa ** (1.0 + q) * X ** k * pr * pr
                + fa ** q * X ** k * pth * pth / (r * r) + fa ** q * L * L / (r * r * s * s))
    a = rd["a"]
    sig = r * r + a * a * c * c
    dlt = np.abs(r * r - 2.0 * r + a * a)
    P = (r * r + a * a) * E - a * L
    W = L / s - a * E * s
    return (dlt * pr * pr + pth * pth + W * W + P * P / dlt) / sig


def oracle_sampled(rd, pixels, **extra):
    """Oracle outputs at the sampled pixels, and the reference band for a
    sampled comparison: a full-image boolean array that is True at a sampled
    pixel whose 3x3 neighbourhood holds more than one status in the ORACLE
    (the neighbours are traced here as well)."""
    pixels = np.asarray(pixels, dtype=np.int64)
    nb = neighbourhood(rd["nx"], rd["ny"], pixels)
    uniq, inv = np.unique(nb, return_inverse=True)
    ref_all = oracle_render(rd, pixels=uniq, **extra)
    st = ref_all["status"][inv.reshape(nb.shape)]
    band = np.zeros(rd["nx"] * rd["ny"], dtype=bool)
    band[pixels] = st.min(axis=0) != st.max(axis=0)
    pos = np.searchsorted(uniq, pixels)
    ref = {k: v[pos] for k, v in ref_all.items()}
    return ref, band


def gpu_render(rd, precision=osr.FP64, persistent=False, stats=None, fields=None, **extra):
    cam = osr.Camera.from_render(rd)
    disk = rd["mode"] == "disk"
    ws = None
    if persistent:
        ws = torch.empty(osr.workspace_bytes(1), dtype=torch.uint8, device="cuda")
    opts = dict(tol=rd["tol"], precision=precision, persistent=persistent,
                cell_deg=rd["cell_deg"], cell_phase_deg=rd["cell_phase_deg"], stats=stats,
                workspace=ws)
    opts.update(extra)
    if fields is None:
        fields = osr.DISK_FIELDS if disk else osr.SHADOW_FIELDS
    out = osr.alloc_outputs(cam.n_rays, fields=fields)
    if disk:
        osr.render_disk(cam, osr.resolve_r_in(rd), rd["r_out"], out=out, l0=rd.get("l0"), **opts)
    else:
        osr.trace(cam, out=out, **opts)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def oracle_render(rd, pixels=None, **extra):
    disk = rd["mode"] == "disk"
    r_in = oracle.isco(rd["a"]) if rd.get("r_in") == "isco" else (rd.get("r_in") or 0.0)
    opts = dict(tol=rd["tol"], cell_deg=rd["cell_deg"], cell_phase_deg=rd["cell_phase_deg"],
                disk=disk, r_in=r_in, r_out=rd.get("r_out") or 0.0)
    if rd.get("l0") is not None:
        opts.update(disk_model=oracle.DISK_CONSTANT_L, l0=rd["l0"])
    if rd.get("q") is not None:
        opts.update(spacetime=oracle.QMETRIC, q=rd["q"])
    opts.update(extra)
    return oracle.trace_pixels(rd["a"], rd["r_obs"], rd["incl_deg"], rd["extent"], rd["nx"],
                               rd["ny"], pixels=pixels, **opts)


def _cell_boundary_distance(theta, phi, cell_deg, phase_deg):
    t = np.mod(theta, 2 * np.pi)
    p = phi.copy()
    fold = t > np.pi
    t = np.where(fold, 2 * np.pi - t, t)
    p = np.where(fold, p + np.pi, p)
    q = np.mod(p + math.radians(phase_deg), 2 * np.pi)
    cell = math.radians(cell_deg)
    dt = np.abs(t / cell - np.round(t / cell)) * cell
    dq = np.abs(q / cell - np.round(q / cell)) * cell
    return np.minimum(dt, dq)


def compare(rd, gpu, ref, pixels=None, band=None, coord_rtol=COORD_RTOL, g_rtol=G_RTOL,
            precision=osr.FP64):
    """Compare GPU outputs (full image arrays) with oracle outputs (for
    `pixels`, or the whole image). With `pixels`, `band` must come from the
    oracle (oracle_sampled). Returns a report dict; assert_parity asserts."""
    n = rd["nx"] * rd["ny"]
    if pixels is None:
        if band is not None:
            raise ValueError("a whole-image comparison takes its band from the oracle image")
        pixels = np.arange(n)
    elif band is None:
        raise ValueError("a sampled comparison needs the oracle band (oracle_sampled)")
    st_ref = ref["status"].astype(np.int64)
    st_gpu = gpu["status"].astype(np.int64)[pixels]
    if band is None:
        img = np.zeros(n, np.int64)
        img[pixels] = st_ref
        band = band_mask(img.reshape(rd["ny"], rd["nx"])).reshape(-1)
    in_band = band[pixels]
    rep = {"n": len(pixels), "band": int(in_band.sum()), "precision": int(precision)}
    mism = (st_gpu != st_ref) & ~in_band
    rep["status_mismatch"] = int(mism.sum())
    same = (st_gpu == st_ref) & ~in_band
    rep["compared"] = int(same.sum())

    def rel_err(key, floor):
        g = gpu[key][pixels][same].astype(np.float64)
        r = ref[key][same].astype(np.float64)
        return np.abs(g - r) / np.maximum(np.abs(r), floor)

    for key, floor in (("r", 1e-300), ("theta", 1.0), ("phi", 1.0)):
        e = rel_err(key, floor)
        rep[key + "_max_rel"] = float(e.max()) if e.size else 0.0
        rep[key + "_n_over"] = int((e > coord_rtol).sum())
    esc = same & (st_ref == oracle.STATUS_ESCAPED)
    if "cell_i" in gpu and esc.any():
        dist = _cell_boundary_distance(ref["theta"][esc], ref["phi"][esc], rd["cell_deg"],
                                       rd["cell_phase_deg"])
        ok = dist > CELL_MARGIN
        gi = gpu["cell_i"][pixels][esc].astype(np.int64)
        gj = gpu["cell_j"][pixels][esc].astype(np.int64)
        rep["cell_mismatch"] = int(((gi != ref["cell_i"][esc]) | (gj != ref["cell_j"][esc]))[ok].sum())
        rep["parity_mismatch"] = int((gpu["parity"][pixels][esc].astype(np.int64)
                                      != ref["parity"][esc])[ok].sum())
    dk = same & (st_ref == oracle.STATUS_DISK)
    rep["n_disk"] = int(dk.sum())
    if "g" in gpu and dk.any():
        for key in ("g", "intensity", "r_hit"):
            g = gpu[key][pixels][dk]
            r = ref[key][dk]
            e = np.abs(g - r) / np.abs(r)
            rep[key + "_max_rel"] = float(e.max())
            rep[key + "_n_over"] = int((e > g_rtol).sum())
    hg = gpu["max_abs_H"][pixels][same]
    hr = ref["max_abs_H"][same]
    rep["H_gpu_max"] = float(hg.max()) if hg.size else 0.0
    rep["H_ref_max"] = float(hr.max()) if hr.size else 0.0
    sg = gpu["steps"][pixels][same].astype(np.int64)
    sr = ref["accepted"][same]
    rep["steps_equal_frac"] = float((sg == sr).mean()) if hg.size else 1.0
    rep["steps_n_diff"] = int((sg != sr).sum())
    rep["steps_max_diff"] = int(np.abs(sg - sr).max()) if hg.size else 0
    rep["H_nonfinite"] = int((~np.isfinite(hg)).sum())
    if precision in H_RTOL and hg.size:
        T = terms_of_2H(rd, {k: v[same] for k, v in ref.items()})
        dH = np.abs(hg - hr)
        rep["H_bound_ratio"] = float((dH / (H_RTOL[precision] * hr + H_EPS[precision] * T)).max())
        rep["steps_bound_ratio"] = float((np.abs(sg - sr) / (STEPS_ALLOW[osr.DF64][0] +
                                          STEPS_ALLOW[osr.DF64][1] * sr)).max())
    rel = np.abs(hg - hr) / np.maximum(hr, 1e-300)
    rep["H_rel_p50"] = float(np.median(rel)) if rel.size else 0.0
    rep["H_rel_max"] = float(rel.max()) if rel.size else 0.0
    return rep


def assert_parity(rep, allow_coord_outliers=0):
    assert rep["status_mismatch"] == 0, rep
    assert rep["H_nonfinite"] == 0, rep
    prec = rep["precision"]
    if prec in H_RTOL and rep["compared"]:  # MIXED runs at other tolerances than its reference
        assert rep["H_bound_ratio"] <= 1.0, rep
        if prec == osr.FP64:
            share, extra = STEPS_ALLOW[prec]
            assert rep["steps_n_diff"] <= int(share * rep["compared"]) + extra, rep
        else:
            assert rep["steps_bound_ratio"] <= 1.0, rep
    for key in ("r", "theta", "phi"):
        assert rep[key + "_n_over"] <= allow_coord_outliers, rep
    for key in ("cell", "parity"):
        if key + "_mismatch" in rep:
            assert rep[key + "_mismatch"] == 0, rep
    for key in ("g", "intensity", "r_hit"):
        if key + "_n_over" in rep:
            assert rep[key + "_n_over"] <= allow_coord_outliers, rep
