"""CPU-side checks of the C interface: the library builds, loads and exports
every entry point include/osiris.h declares; host-only calls and argument
validation work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def osr():
    from paper_2202_00086_gb300 import build
    build.build()
    import paper_2202_00086_gb300 as m
    return m


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(osiris_\w+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(osr):
    names = _declared_functions()
    assert {"osiris_init_camera", "osiris_trace", "osiris_render_disk"} <= names
    lib = ctypes.CDLL(osr.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_host_helpers(osr):
    import oracle
    for a in (0.0, 0.5, 0.9, 0.998):
        assert osr.isco(a) == pytest.approx(oracle.isco(a), rel=1e-14)
        assert osr.horizon(a) == pytest.approx(1 + (1 - a * a) ** 0.5, rel=1e-15)


@pytest.mark.parametrize("args", [
    (1.0, 1000.0, 60.0, (-8, 8, -8, 8), 8, 8),      # a >= 1
    (0.5, 15.0, 60.0, (-8, 8, -8, 8), 8, 8),        # r_obs <= 10 r_H
    (0.5, 1000.0, 0.0, (-8, 8, -8, 8), 8, 8),       # on the axis
    (0.5, 1000.0, 60.0, (8, -8, -8, 8), 8, 8),      # empty extent
    (0.5, 1000.0, 60.0, (-8, 8, -8, 8), 0, 8),      # no pixels
    (0.5, 30.0, 60.0, (-25, 25, -25, 25), 8, 8),    # corner outside the sky
])
def test_camera_validation(osr, args):
    with pytest.raises(osr.OsirisError) as e:
        osr.Camera(*args)
    assert e.value.code == osr.EINVAL


def test_trace_validation_before_launch(osr):
    cam = osr.Camera(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 8, 8)
    out = osr.Outputs()
    for bad in (dict(tol=-1.0), dict(max_steps=0), dict(precision=7), dict(r_cap_factor=1.0),
                dict(cell_deg=0.0), dict(block_size=48)):
        o = osr.make_opts(**bad)
        rc = osr.lib().osiris_trace(cam.handle, ctypes.byref(o), ctypes.byref(out), None)
        assert rc == osr.EINVAL, bad
    o = osr.make_opts()
    rc = osr.lib().osiris_render_disk(cam.handle, 30.0, 20.0, ctypes.byref(o), ctypes.byref(out),
                                      None)
    assert rc == osr.EINVAL
    rc = osr.lib().osiris_trace_batch(None, 0, ctypes.byref(o), None)
    assert rc == osr.EINVAL
    reqs = (osr.Request * 1)()
    rc = osr.lib().osiris_trace_batch(reqs, 65537, ctypes.byref(o), None)  # above the maximum
    assert rc == osr.EINVAL
    assert osr.workspace_bytes(10) > osr.workspace_bytes(1) >= 256


def test_batch_plan_validation_before_any_cuda_call(osr):
    """Argument errors of the batch-plan entry points are reported before the
    plan touches the device (no workspace, no pinned memory, no graph)."""
    L = osr.lib()
    h = ctypes.c_void_p()
    o = osr.make_opts()
    assert L.osiris_batch_plan_create(ctypes.byref(h), 0, osr.SPACETIME_KERR,
                                      ctypes.byref(o)) == osr.EINVAL
    assert L.osiris_batch_plan_create(ctypes.byref(h), 70000, osr.SPACETIME_KERR,
                                      ctypes.byref(o)) == osr.EINVAL
    assert L.osiris_batch_plan_create(ctypes.byref(h), 4, 7, ctypes.byref(o)) == osr.EINVAL
    o_bad = osr.make_opts()
    o_bad.precision = 7
    assert L.osiris_batch_plan_create(ctypes.byref(h), 4, osr.SPACETIME_QMETRIC,
                                      ctypes.byref(o_bad)) == osr.EINVAL  # no such precision
    assert L.osiris_batch_plan_create(ctypes.byref(h), 4, osr.SPACETIME_KERR,
                                      ctypes.byref(osr.make_opts(tol=0.0))) == osr.EINVAL
    assert L.osiris_batch_plan_create(ctypes.byref(h), 4, osr.SPACETIME_KERR,
                                      ctypes.byref(o)) == osr.ENOMEM  # no workspace
    assert not h.value
    arr = (osr.Request * 1)()
    assert L.osiris_batch_plan_launch(None, arr, 1, None) == osr.EINVAL
    L.osiris_batch_plan_destroy(None)


def test_oracle_library_loads():
    import oracle
    lib = oracle.lib()
    for n in ("oracle_trace_pixels", "oracle_trace_states", "oracle_init_ray"):
        assert hasattr(lib, n)


def test_new_entry_points_validate_before_any_cuda_call(osr):
    """Argument errors of the pipe probes, the bounded stream wait and the
    work-distribution options are refused on the host (no GPU here)."""
    L = osr.lib()
    fl = ctypes.c_double()
    buf = ctypes.c_void_p(1)  # never dereferenced: the arguments are refused first
    for prec, op, n, iters in ((7, 0, 256, 1), (osr.FP64, 5, 256, 1), (osr.FP64, -1, 256, 1),
                               (osr.FP64, 0, 100, 1), (osr.FP64, 0, 256, 0)):
        assert L.osiris_pipe_probe(prec, op, n, iters, buf, ctypes.byref(fl), None) == osr.EINVAL
    assert L.osiris_pipe_probe(osr.FP64, 0, 256, 1, None, ctypes.byref(fl), None) == osr.EINVAL
    assert L.osiris_pipe_probe_threads(7, 0) == osr.EINVAL
    assert L.osiris_pipe_probe_threads(osr.FP64, 9) == osr.EINVAL
    assert L.osiris_stream_wait(None, -1.0) == osr.EINVAL
    assert L.osiris_stream_wait(None, float("nan")) == osr.EINVAL
    cam = osr.Camera(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 8, 8)
    out = osr.Outputs()
    for bad in (dict(rays_per_lane=-1), dict(rays_per_lane=65), dict(refill_lanes=-1),
                dict(refill_lanes=33)):
        o = osr.make_opts(**bad)
        assert osr.lib().osiris_trace(cam.handle, ctypes.byref(o), ctypes.byref(out),
                                      None) == osr.EINVAL, bad
    o = osr.make_opts()
    assert (o.rays_per_lane, o.refill_lanes) == (0, 0)  # 0 = the library default
