"""Indexing at the paper's scale (Section 2.3, supplement "Indexing
algorithm"): 618324 test orientations in the cubic fundamental zone, the
1000 strongest reference nodes, and the 1000 best solutions per ROI.

Checks on 64 ROIs of the b.c.c. box: the top-1000 lists are ascending and
distinct; re-scoring ROI 0's 1000 solutions through a second look-up table
built on just those orientations reproduces their scores bit for bit (the
same FP32 sums); that table's rows equal the oracle's nearest nodes; the
top solution equals the plain argmin; and the best coarse orientations lie
within a few degrees of the box's known orientation.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2009_00735_gb300 as apt

from test_gpu_plain import torch_cuda  # noqa: F401

pytestmark = pytest.mark.gpu

N_G = 618324
TOPK = 1000


def test_paper_scale_orientation_set_top1000(torch_cuda):
    torch = torch_cuda
    w = synth.single_crystal_bcc()
    nroi = 64
    w.centres = np.ascontiguousarray(w.centres[:nroi])
    w.radii = np.ascontiguousarray(w.radii[:nroi])
    R = float(w.radii[0])
    band = oracle.band_for_spacing(*w.d_spacing, R, w.m)
    ctx = apt.Context(0)
    h = ctx.handle
    # reference: perfect b.c.c. at identity, same band
    xyz, _ = synth.perfect_crystal_roi("bcc", 0.287, R + 0.5)
    apt.aptidx_load_positions(h, torch.from_numpy(xyz).cuda())
    apt.aptidx_set_directions(h, torch.from_numpy(w.dirs).cuda())
    apt.aptidx_set_binning(h, w.m, band[0], band[1])
    apt.aptidx_set_rois(h, np.zeros((1, 3)), np.array([R]))
    node = torch.empty((1, w.dirs.shape[0]), dtype=torch.float32, device="cuda")
    apt.aptidx_compute_signatures(h, apt.APTIDX_PATH_TC_FP16, apt.APTIDX_NORMALISE_MAX, node, None, None)
    node = node.reshape(-1).contiguous()
    # measured signatures
    apt.aptidx_load_positions(h, torch.from_numpy(w.xyz).cuda())
    apt.aptidx_set_rois(h, torch.from_numpy(w.centres).cuda(), torch.from_numpy(w.radii).cuda())
    S = torch.empty((nroi, w.dirs.shape[0]), dtype=torch.float32, device="cuda")
    apt.aptidx_compute_signatures(h, apt.APTIDX_PATH_TC_FP16, apt.APTIDX_NORMALISE_MAX, S, None, None)

    Q = synth.so3_halton_fz(N_G)
    apt.aptidx_set_reference(h, 0, node, 1000, None)
    apt.aptidx_build_lut(h, 0, torch.from_numpy(Q).cuda())
    best = torch.empty((nroi, TOPK), dtype=torch.int32, device="cuda")
    score = torch.empty((nroi, TOPK), dtype=torch.float32, device="cuda")
    apt.aptidx_match_topk(h, 0, S, TOPK, best, score)
    b1 = torch.empty(nroi, dtype=torch.int32, device="cuda")
    s1 = torch.empty(nroi, dtype=torch.float32, device="cuda")
    apt.aptidx_match(h, 0, S, b1, s1)
    best, score = best.cpu().numpy(), score.cpu().numpy()
    assert np.array_equal(best[:, 0], b1.cpu().numpy()) and np.array_equal(score[:, 0], s1.cpu().numpy())
    for r in range(nroi):
        assert len(np.unique(best[r])) == TOPK and best[r].min() >= 0 and best[r].max() < N_G
        assert np.all(np.diff(score[r]) >= 0)

    # ROI 0's solutions re-scored through a table on just those orientations
    sub = np.ascontiguousarray(Q[best[0]])
    apt.aptidx_set_reference(h, 1, node, 1000, None)
    apt.aptidx_build_lut(h, 1, torch.from_numpy(sub).cuda())
    b_sub = torch.empty((1, TOPK), dtype=torch.int32, device="cuda")
    s_sub = torch.empty((1, TOPK), dtype=torch.float32, device="cuda")
    apt.aptidx_match_topk(h, 1, S[:1].contiguous(), TOPK, b_sub, s_sub)
    b_sub, s_sub = b_sub.cpu().numpy()[0], s_sub.cpu().numpy()[0]
    assert np.array_equal(s_sub, score[0])                 # same sums, same order of ties
    assert np.array_equal(best[0][b_sub], best[0])         # ties kept in g order in both tables
    L_sub = apt.aptidx_get_lut(h, 1, ng=TOPK)
    top = oracle.top_nodes(node.cpu().numpy(), 1000)
    assert np.array_equal(L_sub[:100], oracle.lut(w.dirs, top, sub[:100]))

    mis = np.array([oracle.disorientation_deg(Q[best[r, 0]], w.truth["quat"]) for r in range(nroi)])
    print(f"\n618324 orientations, top-{TOPK} of {nroi} ROIs: coarse misorientation median {np.median(mis):.2f}, "
          f"max {mis.max():.2f} deg")
    assert np.median(mis) <= 2.0
    ctx.close()
