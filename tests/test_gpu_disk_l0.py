"""The constant-l0 disk (Sec. 5) on the GPU against the oracle, on the paper's
disk-figure set-up (a in {0, 0.5, 0.998}, l0 = 2.8, 2.8, 1.8, 85 deg,
[-24,24] x [-12,12], r_in = ISCO, r_out = 20)."""
import numpy as np
import pytest
import torch

import paper_2202_00086_gb300 as osr
from paper_2202_00086_gb300 import workloads

from _parity import assert_parity, compare, gpu_render, oracle_render, oracle_sampled

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [osr.FP64, osr.DF64])
@pytest.mark.parametrize("case", [0, 1, 2])
def test_paper_disk_figure_subsampled(precision, case):
    rd = workloads.paper_disk_figure(nx=96, ny=48)[case]
    rep = compare(rd, gpu_render(rd, precision=precision), oracle_render(rd),
                  precision=precision)
    print(rep)
    assert_parity(rep)
    assert rep["n_disk"] > 300


def test_paper_disk_figure_full_size_sampled():
    rd = workloads.paper_disk_figure()[2]  # a = 0.998, l0 = 1.8, 2048 x 1024
    gpu = gpu_render(rd, precision=osr.DF64, persistent=True)
    rng = np.random.default_rng(31)
    pix = np.sort(rng.choice(rd["nx"] * rd["ny"], 300, replace=False))
    ref, band = oracle_sampled(rd, pix)
    rep = compare(rd, gpu, ref, pixels=pix, band=band, precision=osr.DF64)
    print(rep)
    assert_parity(rep)
    assert rep["n_disk"] > 20


def test_l0_batch_equals_single():
    rds = workloads.paper_disk_figure(nx=40, ny=20)
    singles = [gpu_render(rd, precision=osr.DF64) for rd in rds]
    cams = [osr.Camera.from_render(rd) for rd in rds]
    outs = [osr.alloc_outputs(c.n_rays, fields=osr.DISK_FIELDS) for c in cams]
    ws = torch.empty(osr.workspace_bytes(3), dtype=torch.uint8, device="cuda")
    reqs = [{"camera": c, "disk": True, "r_in": osr.resolve_r_in(rd), "r_out": 20.0,
             "l0": rd["l0"], "out": o} for c, o, rd in zip(cams, outs, rds)]
    osr.trace_batch(reqs, workspace=ws, precision=osr.DF64,
                    cell_phase_deg=rds[0]["cell_phase_deg"])
    torch.cuda.synchronize()
    for o, ref in zip(outs, singles):
        for k in ref:
            assert np.array_equal(o[k].cpu().numpy(), ref[k]), k
