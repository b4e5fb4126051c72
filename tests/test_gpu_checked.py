"""The bounds-checked build (libosiris_checked.so: the library compiled with
OSIRIS_CHECKED, which checks each ray's queue, request and pixel or state
index before use and counts failures in the stats array instead of trapping)
on the small and ragged launches where an index slip would show: 1x1, 2x3
and 5x3 renders, a 37x29 render at block sizes 32, 96 and 256, plain and
persistent, FP64 and DF64, a batch of pixel ranges, and explicit initial
data. Every launch must report no failed check and give, bit for bit, the
outputs of the default build."""
import numpy as np
import pytest
import torch

import oracle
import paper_2202_00086_gb300 as osr
from paper_2202_00086_gb300 import workloads

from _parity import gpu_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checked():
    from paper_2202_00086_gb300 import build
    build.build(checked=True)
    return osr.load(osr.LIB_CHECKED_PATH)


def _both(checked, fn):
    a = fn(None)
    stats = osr.new_stats()
    with osr.using_library(checked):
        b = fn(stats)
    s = stats.cpu().numpy()
    assert s[13] == 0 and s[14] == 0, ("failed index checks", int(s[13]), hex(int(s[14])))
    for k in a:
        assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k
    return b


CASES = [(0.5, 60.0, 1, 1), (0.5, 60.0, 2, 3), (0.9, 17.0, 5, 3), (0.998, 60.0, 37, 29)]


@pytest.mark.parametrize("precision", [osr.FP64, osr.DF64])
@pytest.mark.parametrize("a,inc,nx,ny", CASES)
def test_checked_renders(checked, precision, a, inc, nx, ny):
    rd = workloads.render(a, 1000.0, inc, (-8, 8, -8, 8), nx, ny)
    for block in (32, 96, 256):
        for persistent in (False, True):
            _both(checked, lambda st: gpu_render(rd, precision=precision, block_size=block,
                                                 persistent=persistent, stats=st))


def test_checked_disk_and_batch_of_ranges(checked):
    disk = workloads.render(0.9, 1000.0, 60.0, (-25, 25, -25, 25), 23, 17, mode="disk",
                            r_in="isco", r_out=20.0)
    _both(checked, lambda st: gpu_render(disk, persistent=True, block_size=64, stats=st))
    rds = [workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 5, 3),
           workloads.render(0.9, 1000.0, 30.0, (-8, 8, -8, 8), 7, 11)]
    ranges = [(0, 15), (4, 70)]  # a whole render, then pixels [4, 74) of the 7x11 one

    def run(st):
        outs = [osr.alloc_outputs(rd["nx"] * rd["ny"]) for rd in rds]
        for o in outs:
            for t in o.values():
                t.zero_()
        reqs = [{"camera": osr.Camera.from_render(rd), "out": o, "first_ray": f, "n_rays": n}
                for rd, o, (f, n) in zip(rds, outs, ranges)]
        ws = torch.empty(osr.workspace_bytes(2), dtype=torch.uint8, device="cuda")
        osr.trace_batch(reqs, workspace=ws, stats=st, block_size=32)
        torch.cuda.synchronize()
        return {"%d_%s" % (k, f): v.cpu().numpy() for k, o in enumerate(outs)
                for f, v in o.items()}

    out = _both(checked, run)
    assert np.all(out["1_status"][:4] == 0) and np.all(out["1_status"][4:74] > 0)


def test_checked_explicit_states(checked):
    st = np.array([oracle.init_ray(0.9, 1000.0, 60.0, x, y)
                   for x, y in ((-3.0, 1.0), (0.5, 6.0), (7.0, -2.0))])
    dev = [torch.tensor(np.ascontiguousarray(x), device="cuda")
           for x in (st[:, :6], st[:, 6], st[:, 7])]

    def run(stats):
        o = osr.trace_states(0.9, 1000.0, *dev, stats=stats)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in o.items()}

    _both(checked, run)
