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
  - disk: g, intensity, r_hit within 1e-8 relative.
"""
import math

import numpy as np
import torch

import oracle
import paper_2202_00086_gb300 as osr

COORD_RTOL = 1e-8
G_RTOL = 1e-8
CELL_MARGIN = 1e-6


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


def compare(rd, gpu, ref, pixels=None, band=None, coord_rtol=COORD_RTOL, g_rtol=G_RTOL):
    """Compare GPU outputs (full image arrays) with oracle outputs (for
    `pixels`, or the whole image). Returns a report dict; the caller asserts."""
    n = rd["nx"] * rd["ny"]
    if pixels is None:
        pixels = np.arange(n)
    st_ref = ref["status"].astype(np.int64)
    st_gpu = gpu["status"].astype(np.int64)[pixels]
    if band is None:
        img = np.zeros(n, np.int64)
        img[pixels] = st_ref
        band = band_mask(img.reshape(rd["ny"], rd["nx"])).reshape(-1)
    in_band = band[pixels]
    rep = {"n": len(pixels), "band": int(in_band.sum())}
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
    rep["steps_equal_frac"] = float((gpu["steps"][pixels][same].astype(np.int64)
                                     == ref["accepted"][same]).mean()) if hg.size else 1.0
    return rep


def assert_parity(rep, allow_coord_outliers=0):
    assert rep["status_mismatch"] == 0, rep
    for key in ("r", "theta", "phi"):
        assert rep[key + "_n_over"] <= allow_coord_outliers, rep
    for key in ("cell", "parity"):
        if key + "_mismatch" in rep:
            assert rep[key + "_mismatch"] == 0, rep
    for key in ("g", "intensity", "r_hit"):
        if key + "_n_over" in rep:
            assert rep[key + "_n_over"] <= allow_coord_outliers, rep
