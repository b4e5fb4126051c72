"""Failure paths of the trace kernels, made on the host (no GPU fault).

A ray whose explicit initial data hold NaN or Inf (a corrupt upload, a
division by zero in the caller's set-up) must end with STATUS_ERROR after its
first attempt, and must not disturb the rays beside it: those give exactly
the outputs of the same rays traced without the bad ones. Every table index
the kernels derive from a coordinate is range-checked (NaN and Inf fall back
to the library function), so such a ray reads nothing out of bounds.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2202_00086_gb300 as osr

pytestmark = pytest.mark.gpu


def _rays(a, r_obs, incl, n, seed):
    rng = np.random.default_rng(seed)
    st = np.array([oracle.init_ray(a, r_obs, incl, x, y)
                   for x, y in rng.uniform(-8.0, 8.0, size=(n, 2))])
    return st[:, :6].copy(), st[:, 6].copy(), st[:, 7].copy()


def _trace(states, E, L, **kw):
    dev = [torch.tensor(np.ascontiguousarray(x), device="cuda") for x in (states, E, L)]
    out = osr.trace_states(kw.pop("a", 0.0), 1000.0, *dev, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


# (row, column of the state or "E" / "L", value)
BAD = [(1, 4, float("nan")), (4, "E", float("inf")), (6, 2, float("nan")), (9, 1, -float("inf")),
       (12, "L", float("nan"))]


@pytest.mark.parametrize("precision", [osr.FP64, osr.DF64, osr.MIXED])
@pytest.mark.parametrize("q", [None, 0.5])
@pytest.mark.parametrize("persistent", [False, True])
def test_non_finite_initial_data_end_in_error(precision, q, persistent):
    a = 0.9 if q is None else 0.0
    st, E, L = _rays(a, 1000.0, 60.0, 16, seed=5)
    if q is not None:
        st, E, L = [], [], []
        rng = np.random.default_rng(5)
        for x, y in rng.uniform(-8.0, 8.0, size=(16, 2)):
            row = oracle.init_ray_sp(oracle.QMETRIC, 1000.0, 60.0, x, y, q=q)
            st.append(row[:6])
            E.append(row[6])
            L.append(row[7])
        st, E, L = np.array(st), np.array(E), np.array(L)
    bad_rows = sorted({r for r, _, _ in BAD})
    good = np.setdiff1d(np.arange(16), bad_rows)
    kw = dict(a=a, q=q, precision=precision)
    if precision == osr.MIXED:
        kw["tol"] = 1e-8  # the tolerances MIXED is meant for
    ws = None
    if persistent:
        ws = torch.empty(osr.workspace_bytes(1), dtype=torch.uint8, device="cuda")
        kw.update(persistent=True, workspace=ws)
    clean = _trace(st[good], E[good], L[good], **kw)
    st_b, E_b, L_b = st.copy(), E.copy(), L.copy()
    for row, col, val in BAD:
        if col == "E":
            E_b[row] = val
        elif col == "L":
            L_b[row] = val
        else:
            st_b[row, col] = val
    stats = osr.new_stats()
    got = _trace(st_b, E_b, L_b, stats=stats, **kw)
    assert got["status"][bad_rows].tolist() == [osr.STATUS_ERROR] * len(bad_rows)
    for k in clean:  # the good rays are untouched, bit for bit
        assert np.array_equal(got[k][good], clean[k], equal_nan=True), k
    assert np.all(np.isin(got["status"][good], [osr.STATUS_CAPTURED, osr.STATUS_ESCAPED]))
    # a failed ray stops at its first attempt and reports no accepted step
    assert np.all(got["steps"][bad_rows] == 0)
    s = osr.decode_stats(stats)
    assert s["status_error"] == len(bad_rows) and s["rays"] == 16
    assert math.isfinite(s["max_abs_H"])


def test_stream_wait_is_bounded():
    """osiris_stream_wait returns OSIRIS_ETIMEOUT when the bound runs out
    before the queued render completes (nothing is interrupted: the render
    finishes and a second, longer wait returns OSIRIS_OK)."""
    cam = osr.Camera(0.9, 1000.0, 60.0, (-8, 8, -8, 8), 512, 512)
    out = osr.alloc_outputs(cam.n_rays)
    out["status"].zero_()
    torch.cuda.synchronize()
    osr.trace(cam, out=out)  # ~80 ms of FP64 work
    assert osr.stream_wait(1e-4) == osr.ETIMEOUT
    assert osr.stream_wait(120.0) == osr.OK
    assert int((out["status"] == 0).sum()) == 0
    with pytest.raises(osr.OsirisError) as e:
        osr.stream_wait(-1.0)
    assert e.value.code == osr.EINVAL
