"""Local ROI grid refinement (Section 3.4): a coarse 2 nm ROI grid over a box
whose left half is a noisy b.c.c. crystal and whose right half holds the same
number density of randomly placed atoms; ROIs whose peak signature reaches
kappa times the largest one get their cell split into 5^3 new ROIs.  The new
centres and parents equal the oracle's (computed from oracle signatures) bit
for bit, the crystal side qualifies and the random side does not, and the
second pass over the new ROIs matches the oracle.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2009_00735_gb300 as apt

from test_gpu_plain import roi_error, torch_cuda  # noqa: F401

pytestmark = pytest.mark.gpu

TOL_TC = 5e-3


def half_crystal_box():
    rng = np.random.default_rng(synth.SEED_BASE + 13)
    q = synth.random_quaternions(rng, 1)[0]
    lo, hi = np.zeros(3), np.array([12.0, 12.0, 6.0])
    xyz, _ = synth.lattice_box("bcc", 0.287, lo, hi, rot=synth.quat_to_matrix(q))
    xyz = xyz[synth.keep_fraction(rng, xyz.shape[0], 0.4)]
    xyz = synth.displace(rng, xyz, (0.05, 0.05, 0.02))
    left = xyz[xyz[:, 0] < 6.0]
    rand = lo + rng.random((int((xyz[:, 0] >= 6.0).sum()), 3)) * np.array([6.0, 12.0, 6.0])
    rand[:, 0] += 6.0
    pos = np.concatenate([left, rand]).astype(np.float32)
    centres = synth.roi_grid((5, 5, 2), 2.0, (lo + hi) / 2)
    return np.ascontiguousarray(pos), centres


def test_roi_grid_refinement(torch_cuda):
    torch = torch_cuda
    pos, centres = half_crystal_box()
    nroi = centres.shape[0]
    radii = np.full(nroi, 2.0)
    dirs = np.ascontiguousarray(synth.icosphere(4))
    m = 10
    band = oracle.band_for_spacing(0.9 * 0.287 / np.sqrt(2), 1.1 * 0.287 / np.sqrt(2), 2.0, m)
    So, _, _ = oracle.signatures(pos, centres, radii, band[0], band[1], dirs, m)
    # the kappa in [0.6, 0.95] farthest from every ROI's relative peak
    peak = So.max(axis=1) / So.max()
    grid = np.arange(0.60, 0.95, 0.0025)
    kappa = float(grid[np.argmax([np.abs(peak - k).min() for k in grid])])
    assert np.abs(peak - kappa).min() >= 0.003
    ctx = apt.Context(0)
    h = ctx.handle
    apt.aptidx_load_positions(h, torch.from_numpy(pos).cuda())
    apt.aptidx_set_directions(h, torch.from_numpy(dirs).cuda())
    apt.aptidx_set_binning(h, m, band[0], band[1])
    apt.aptidx_set_rois(h, centres, radii)
    S = torch.empty((nroi, dirs.shape[0]), dtype=torch.float32, device="cuda")
    apt.aptidx_compute_signatures(h, apt.APTIDX_PATH_TC_FP16, 0, S, None, None)
    c_gpu, p_gpu = apt.aptidx_refine_roi_grid(h, S, float(kappa), 2.0, 5)
    c_orc, p_orc = oracle.refine_roi_grid(So, centres, float(kappa), 2.0, 5)
    assert c_gpu.shape[0] > 0 and np.array_equal(p_gpu, p_orc) and np.array_equal(c_gpu, c_orc)
    # host output buffers give the same
    c_h, p_h = apt.aptidx_refine_roi_grid(h, S.cpu().numpy(), float(kappa), 2.0, 5)
    assert np.array_equal(c_h, c_gpu) and np.array_equal(p_h, p_gpu)
    crystal = centres[np.unique(p_gpu)][:, 0]
    assert crystal.max() < 6.0                           # no ROI of the random half qualifies
    # second pass on the new ROIs
    apt.aptidx_set_rois(h, c_gpu, np.full(c_gpu.shape[0], 2.0))
    S2 = torch.empty((c_gpu.shape[0], dirs.shape[0]), dtype=torch.float32, device="cuda")
    apt.aptidx_compute_signatures(h, apt.APTIDX_PATH_TC_FP16, 0, S2, None, None)
    rng = np.random.default_rng(3)
    pick = rng.choice(c_gpu.shape[0], 8, replace=False)
    So2, _, _ = oracle.signatures(pos, c_gpu[pick], np.full(8, 2.0), band[0], band[1], dirs, m)
    assert roi_error(S2.cpu().numpy()[pick], So2).max() <= TOL_TC
    print(f"\nkappa {kappa:.2f}: {np.unique(p_gpu).size} of {nroi} coarse ROIs refined into {c_gpu.shape[0]}")
    ctx.close()
