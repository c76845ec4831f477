"""Histograms at bin edges, bit-exact on both signature paths: a ROI whose
atoms sit on and one float32 ulp either side of bin edges along the three
coordinate axes (the projection onto an axis is the coordinate itself), plus
random directions, against the FP64 oracle's contract histograms.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2009_00735_gb300 as apt

from test_gpu_plain import torch_cuda  # noqa: F401
from test_oracle_pins import bin_edge_positions

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m, R", [(8, 1.0), (10, 2.0), (10, 2.37), (11, 2.0), (12, 3.1)])
@pytest.mark.parametrize("path", [apt.APTIDX_PATH_PLAIN_FP32, apt.APTIDX_PATH_TC_FP16])
def test_histograms_bit_exact_at_bin_edges(torch_cuda, m, R, path):
    torch = torch_cuda
    xs = bin_edge_positions(m, R)
    rng = np.random.default_rng(2)
    pts = []
    for axis in range(3):
        p = (rng.random((xs.shape[0], 3)) - 0.5) * 0.05
        p[:, axis] = xs
        pts.append(p)
    xyz = np.ascontiguousarray(np.concatenate(pts).astype(np.float32))
    u = rng.standard_normal((61, 3))
    dirs = np.concatenate([np.eye(3), u / np.linalg.norm(u, axis=1, keepdims=True)]).astype(np.float32)
    dirs = np.ascontiguousarray(dirs)
    ctx = apt.Context(0)
    h = ctx.handle
    apt.aptidx_load_positions(h, torch.from_numpy(xyz).cuda())
    apt.aptidx_set_directions(h, torch.from_numpy(dirs).cuda())
    apt.aptidx_set_binning(h, m, 1, 4)
    apt.aptidx_set_rois(h, np.zeros((1, 3)), np.array([R]))
    hg = np.empty((dirs.shape[0], 1 << m), np.uint16)
    apt.aptidx_get_histograms(h, 0, path, hg)
    ctx.close()
    _, xc = oracle.gather(xyz, np.zeros(3), R)
    ho = oracle.histograms(xc, dirs, m, R)
    assert xc.shape[0] > 0.9 * xyz.shape[0]
    assert np.array_equal(hg.astype(np.int64), ho.astype(np.int64))
