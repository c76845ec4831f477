"""Several signatures per ROI in one call (Section 3.1: per atom type and per
lattice-plane family) on a noisy L1_2 Al3Sc crystal: {111}, {200} and {220}
over all atoms, {100} and {110} over the Sc sub-lattice only (the
superstructure reflections that tell L1_2 from f.c.c.).  Every signature
matches the FP64 oracle with that type mask and band, on both paths; the
interleaved masks land in their own slabs; the context's own band and type
mask are untouched afterwards.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2009_00735_gb300 as apt

from test_gpu_plain import TOL_PLAIN, roi_error, torch_cuda  # noqa: F401

pytestmark = pytest.mark.gpu

TOL_TC = 5e-3
ALL, SC = 0xFFFFFFFF, 0b10


@pytest.fixture(scope="module")
def l12():
    rng = np.random.default_rng(synth.SEED_BASE + 7)
    q = synth.random_quaternions(rng, 1)[0]
    lo, hi = np.zeros(3), np.full(3, 9.0)
    xyz, t = synth.lattice_box("l12", 0.410, lo, hi, rot=synth.quat_to_matrix(q))
    keep = synth.keep_fraction(rng, xyz.shape[0], 0.5)
    xyz = synth.displace(rng, xyz[keep], (0.03, 0.03, 0.03)).astype(np.float32)
    centres = synth.roi_random(rng, 24, lo, hi, 1.6)
    radii = np.full(24, 1.5)
    return np.ascontiguousarray(xyz), np.ascontiguousarray(t[keep]), centres, radii


def spacing_band(d, R, m):
    return oracle.band_for_spacing(0.9 * d, 1.1 * d, R, m)


@pytest.mark.parametrize("path", [apt.APTIDX_PATH_PLAIN_FP32, apt.APTIDX_PATH_TC_FP16])
def test_multi_signatures(torch_cuda, l12, path):
    torch = torch_cuda
    xyz, types, centres, radii = l12
    m = 9
    a = 0.410
    sigs = [(ALL, a / np.sqrt(3)), (SC, a), (ALL, a / 2), (ALL, a / np.sqrt(8)), (SC, a / np.sqrt(2))]
    masks = [s[0] for s in sigs]
    bands = [spacing_band(d, 1.5, m) for _, d in sigs]
    lo = [b[0] for b in bands]
    hi = [b[1] for b in bands]
    dirs = np.ascontiguousarray(synth.icosphere(5))
    ctx = apt.Context(0)
    h = ctx.handle
    apt.aptidx_load_positions(h, torch.from_numpy(xyz).cuda(), torch.from_numpy(types).cuda())
    apt.aptidx_set_directions(h, torch.from_numpy(dirs).cuda())
    own = spacing_band(a / 2, 1.5, m)
    apt.aptidx_set_binning(h, m, own[0], own[1])
    apt.aptidx_set_rois(h, centres, radii)
    nroi, nv = centres.shape[0], dirs.shape[0]
    S0 = torch.empty((nroi, nv), dtype=torch.float32, device="cuda")
    apt.aptidx_compute_signatures(h, path, 0, S0, None, None)
    S = torch.empty((len(sigs), nroi, nv), dtype=torch.float32, device="cuda")
    A = torch.empty((len(sigs), nroi, nv), dtype=torch.uint16, device="cuda")
    N = torch.empty((len(sigs), nroi), dtype=torch.int32, device="cuda")
    apt.aptidx_compute_signatures_multi(h, path, 0, masks, lo, hi, S, A, N)
    S, A, N = S.cpu().numpy(), A.cpu().numpy().astype(np.int64), N.cpu().numpy()
    tol = TOL_PLAIN if path == apt.APTIDX_PATH_PLAIN_FP32 else TOL_TC
    for s in range(len(sigs)):
        So, Ao, No = oracle.signatures(xyz, centres, radii, lo[s], hi[s], dirs, m, types=types, type_mask=masks[s])
        assert np.array_equal(N[s], No), s
        assert np.all((A[s] >= lo[s]) & (A[s] <= hi[s])), s
        keep = No > 0
        assert roi_error(S[s][keep], So[keep]).max() <= tol, s
    assert N[1].max() < N[0].min()                    # the Sc sub-lattice is a quarter of the atoms
    # the context's own band and type mask still apply to a plain call
    S1 = torch.empty((nroi, nv), dtype=torch.float32, device="cuda")
    apt.aptidx_compute_signatures(h, path, 0, S1, None, None)
    assert np.array_equal(S1.cpu().numpy(), S0.cpu().numpy())
    # normalised multi output: every row peaks at 1
    Sn = torch.empty((len(sigs), nroi, nv), dtype=torch.float32, device="cuda")
    apt.aptidx_compute_signatures_multi(h, path, apt.APTIDX_NORMALISE_MAX, masks, lo, hi, Sn)
    assert np.allclose(Sn.cpu().numpy().max(axis=2), 1.0)
    ctx.close()


@pytest.mark.parametrize("path", [apt.APTIDX_PATH_PLAIN_FP32, apt.APTIDX_PATH_TC_FP16])
def test_multi_masks_wider_than_the_context(torch_cuda, l12, path):
    """The ROI set gathers the Sc sub-lattice only; a multi call that also
    asks for all atoms sizes its gather buffer for the union of the masks
    and matches the oracle; afterwards the context still gathers Sc only."""
    torch = torch_cuda
    xyz, types, centres, radii = l12
    m = 9
    a = 0.410
    masks = [ALL, SC, ALL]
    bands = [spacing_band(a / 2, 1.5, m), spacing_band(a, 1.5, m), spacing_band(a / np.sqrt(3), 1.5, m)]
    lo = [b[0] for b in bands]
    hi = [b[1] for b in bands]
    dirs = np.ascontiguousarray(synth.icosphere(4))
    ctx = apt.Context(0)
    h = ctx.handle
    apt.aptidx_load_positions(h, torch.from_numpy(xyz).cuda(), torch.from_numpy(types).cuda())
    apt.aptidx_set_directions(h, torch.from_numpy(dirs).cuda())
    apt.aptidx_set_binning(h, m, lo[1], hi[1])
    apt.aptidx_set_rois(h, centres, radii, type_mask=SC)
    nroi, nv = centres.shape[0], dirs.shape[0]
    S = torch.empty((len(masks), nroi, nv), dtype=torch.float32, device="cuda")
    N = torch.empty((len(masks), nroi), dtype=torch.int32, device="cuda")
    apt.aptidx_compute_signatures_multi(h, path, 0, masks, lo, hi, S, None, N)
    S, N = S.cpu().numpy(), N.cpu().numpy()
    tol = TOL_PLAIN if path == apt.APTIDX_PATH_PLAIN_FP32 else TOL_TC
    for s in range(len(masks)):
        So, _, No = oracle.signatures(xyz, centres, radii, lo[s], hi[s], dirs, m, types=types, type_mask=masks[s])
        assert np.array_equal(N[s], No), s
        keep = No > 0
        assert roi_error(S[s][keep], So[keep]).max() <= tol, s
    S1 = torch.empty((nroi, nv), dtype=torch.float32, device="cuda")
    N1 = torch.empty(nroi, dtype=torch.int32, device="cuda")
    apt.aptidx_compute_signatures(h, path, 0, S1, None, N1)
    assert np.array_equal(N1.cpu().numpy(), N[1])
    assert np.allclose(S1.cpu().numpy(), S[1], rtol=1e-6, atol=0)
    ctx.close()
