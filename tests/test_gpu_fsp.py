"""GPU parity of the reciprocal-space signature (Eq. 2) on tcgen05 against the
FP64 oracle: |F(k)| on the L^3 grid over [-2 pi, 2 pi]^3 nm^-1 (L = 64, and
the larger grids of the paper's benchmark up to L = 512), fp16 operands with
FP32 accumulation; per ROI e = max_k |F_gpu - F_oracle| / max_k F_oracle
<= 5e-3.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2009_00735_gb300 as apt

from test_gpu_plain import torch_cuda  # noqa: F401

pytestmark = pytest.mark.gpu

TOL = 5e-3
L = 64


def fsp_gpu(torch, xyz, centres, radii, types=None, mask=0xFFFFFFFF, kmax=2 * np.pi, L=L):
    ctx = apt.Context(0)
    h = ctx.handle
    apt.aptidx_load_positions(h, torch.from_numpy(xyz).cuda(), None if types is None else torch.from_numpy(types).cuda())
    apt.aptidx_set_directions(h, torch.from_numpy(synth.icosphere(1)).cuda())
    apt.aptidx_set_binning(h, 8, 10, 11)
    apt.aptidx_set_rois(h, centres, radii, type_mask=mask)
    amp = torch.empty((centres.shape[0], L, L, L), dtype=torch.float32, device="cuda")
    apt.aptidx_compute_fsp(h, amp, kmax)
    apt.aptidx_sync(h)
    out = amp.cpu().numpy()
    ctx.close()
    return out


def test_fsp_tiny_full_grid_and_samples(torch_cuda):
    w = synth.tiny_fcc()
    centres = w.centres.copy()
    centres[5] = [100.0, 100.0, 100.0]             # an empty ROI
    F = fsp_gpu(torch_cuda, w.xyz, centres, w.radii)
    assert np.all(F[5] == 0)
    rng = np.random.default_rng(9)
    for r in [0, 1]:                               # every grid point
        _, xc = oracle.gather(w.xyz, centres[r], w.radii[r])
        Fo = oracle.fsp(xc, L).reshape(L, L, L)
        e = np.abs(F[r] - Fo).max() / Fo.max()
        assert e <= TOL, (r, e)
    pts = rng.choice(L ** 3, 3000, replace=False)
    for r in range(centres.shape[0]):
        if r == 5:
            continue
        _, xc = oracle.gather(w.xyz, centres[r], w.radii[r])
        Fo = oracle.fsp(xc, L, points=pts)
        assert np.abs(F[r].reshape(-1)[pts] - Fo).max() / xc.shape[0] <= TOL


def test_fsp_single_crystal_rois_and_type_mask(torch_cuda):
    w = synth.single_crystal_bcc()
    sel = [0, 1000, 4095, 8191]
    centres, radii = w.centres[sel], w.radii[sel]
    F = fsp_gpu(torch_cuda, w.xyz, centres, radii, kmax=5.0)
    rng = np.random.default_rng(10)
    c = np.arange(30, 34)                           # around k = 0, where |F| approaches N_w
    centre = ((c[:, None, None] * L + c[None, :, None]) * L + c[None, None, :]).reshape(-1)
    pts = np.unique(np.concatenate([rng.choice(L ** 3, 4000, replace=False), centre]))
    for i in range(len(sel)):
        _, xc = oracle.gather(w.xyz, centres[i], radii[i])
        Fo = oracle.fsp(xc, L, kmax=5.0, points=pts)
        e = np.abs(F[i].reshape(-1)[pts] - Fo).max() / Fo.max()
        assert e <= TOL, (i, e)
    # atoms of one type only: the mask applies to the gather
    types = (np.arange(w.xyz.shape[0]) % 2).astype(np.uint8)
    Fm = fsp_gpu(torch_cuda, w.xyz, centres[:1], radii[:1], types=types, mask=0b10, kmax=5.0)
    _, xc = oracle.gather(w.xyz, centres[0], radii[0], types=types, type_mask=0b10)
    Fo = oracle.fsp(xc, L, kmax=5.0, points=pts)
    assert np.abs(Fm[0].reshape(-1)[pts] - Fo).max() / Fo.max() <= TOL


def edge_points(L, n, seed):
    """n random flat grid indices plus every combination of the 64-block
    edges (first and last index of each block) along the three axes."""
    rng = np.random.default_rng(seed)
    edge = np.unique(np.concatenate([np.arange(0, L, 64), np.arange(63, L, 64)]))
    ijk = np.stack(np.meshgrid(edge, edge, edge, indexing="ij"), -1).reshape(-1, 3)
    return np.unique(np.concatenate([rng.choice(L ** 3, n, replace=False), (ijk[:, 0] * L + ijk[:, 1]) * L + ijk[:, 2]]))


@pytest.mark.parametrize("Lg", [128, 512])
def test_fsp_larger_grids(torch_cuda, Lg):
    """The larger grids of the paper's benchmark (L_D up to 512): a b.c.c. ROI
    and a small f.c.c. ROI at sampled points, among them every block edge."""
    b = synth.single_crystal_bcc()
    w = synth.tiny_fcc()
    for xyz, centre, radius in [(b.xyz, b.centres[:1], b.radii[:1]), (w.xyz, w.centres[1:2], w.radii[1:2])]:
        F = fsp_gpu(torch_cuda, xyz, centre, radius, L=Lg).reshape(-1)
        pts = edge_points(Lg, 4000, 11)
        _, xc = oracle.gather(xyz, centre[0], radius[0])
        Fo = oracle.fsp(xc, Lg, points=pts)
        assert np.abs(F[pts] - Fo).max() / xc.shape[0] <= TOL, Lg
        del F
