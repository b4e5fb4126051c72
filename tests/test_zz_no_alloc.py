"""The allocation-free batched trace (osiris_trace_batch_static) against the
workspace-based one (osiris_trace_batch).

osiris_trace_batch_static serves callers that cannot allocate device memory
themselves (plug-ins whose host application owns the device memory, processes
under a device-memory quota, loops that must not call cudaMalloc/cudaFree).
It keeps its queue counter and request table in a fixed device array inside
the library instead of a caller workspace. This file is collected last so that
a run stopping at the first failure has already run every other test; it
also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2202_00086_gb300 as osr
from paper_2202_00086_gb300 import workloads

pytestmark = pytest.mark.gpu


def _batch(seed):
    """A small uneven batch: shadow and disk renders of different sizes."""
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(5):
        side = int(rng.choice([8, 16, 24]))
        a = float(rng.uniform(0.0, 0.998))
        inc = float(rng.uniform(5.0, 85.0))
        if k % 2:
            rd = workloads.render(a, 1000.0, inc, (-25, 25, -25, 25), side, side + 3,
                                  mode="disk", r_in="isco", r_out=20.0)
        else:
            rd = workloads.render(a, 1000.0, inc, (-8, 8, -8, 8), side + 5, side)
        reqs.append(rd)
    return reqs


def _requests(renders):
    out = []
    for rd in renders:
        cam = osr.Camera.from_render(rd)
        disk = rd["mode"] == "disk"
        fields = osr.DISK_FIELDS if disk else osr.SHADOW_FIELDS
        out.append({"camera": cam, "disk": disk, "r_in": osr.resolve_r_in(rd) if disk else 0.0,
                    "r_out": rd["r_out"] if disk else 0.0, "tol": rd["tol"],
                    "out": osr.alloc_outputs(cam.n_rays, fields=fields)})
    return out


def _host(reqs):
    torch.cuda.synchronize()
    return [{k: v.cpu().numpy() for k, v in q["out"].items()} for q in reqs]


def _assert_same(a, b):
    """Bit-identical outputs: the two entry points run the same kernel on the
    same request table, so any difference means a table or queue that was not
    what the caller asked for."""
    for qa, qb in zip(a, b):
        assert qa.keys() == qb.keys()
        for key in qa:
            assert qa[key].dtype == qb[key].dtype, key
            assert np.array_equal(qa[key].view(np.uint8), qb[key].view(np.uint8)), key


def test_static_batch_matches_workspace_batch_twice():
    assert torch.cuda.is_available()
    phase = workloads.checker_phase_deg(2202)
    for call, seed in enumerate((1, 2)):  # two calls in a row, different batches
        renders = _batch(seed)
        ref = _requests(renders)
        ws = torch.empty(osr.workspace_bytes(len(ref)), dtype=torch.uint8, device="cuda")
        osr.trace_batch(ref, workspace=ws, cell_phase_deg=phase)
        expect = _host(ref)

        got_reqs = _requests(renders)
        for q in got_reqs:  # poison the outputs: every entry must be written
            for t in q["out"].values():
                t.fill_(7 if t.dtype != torch.float64 else float("nan"))
        osr.trace_batch_static(got_reqs, cell_phase_deg=phase)
        got = _host(got_reqs)
        _assert_same(got, expect)
        assert sum(int((g["status"] == 0).sum()) for g in got) == 0, call


def test_static_batch_rejects_too_many_requests():
    lib = osr.lib()
    n = 257  # OSIRIS_STATIC_MAX_REQUESTS + 1
    arr = (osr.Request * n)()
    o = osr.make_opts()
    fn = lib.osiris_trace_batch_static
    fn.argtypes = [ctypes.POINTER(osr.Request), ctypes.c_int32, ctypes.POINTER(osr.TraceOpts),
                   ctypes.c_void_p]
    assert fn(arr, n, ctypes.byref(o), None) == osr.EINVAL
    assert fn(arr, 0, ctypes.byref(o), None) == osr.EINVAL
