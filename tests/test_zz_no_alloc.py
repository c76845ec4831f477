"""The no-allocation entry point, aptidx_signatures_noalloc.

Some callers cannot call cudaMalloc -- code running while a CUDA graph is
captured, a host framework that owns all device memory through its own pool,
a plugin that may not allocate from its callback.  They pass their own input
and output buffers, and the library keeps what the call derives in one fixed
scratch array.  These tests call it through the C ABI:

  - two calls in a row (different ROI order and band the second time, so the
    shared scratch array must be fully rewritten) give bit for bit the
    signatures of aptidx_compute_signatures on the FP32 path (the same kernel
    on the same gathered atoms), and both lie within the FP32 tolerance of the
    FP64 oracle;
  - a wide band (k = 8..128, more frequency groups than warps) takes the
    kernel's other spectrum branch and still matches bit for bit;
  - a call without a status word works; a direction that is not a unit vector
    and a zero radius raise the INVALID status bit, and the zero-radius ROI
    gets a zero row.

The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2009_00735_gb300 as apt
from paper_2009_00735_gb300 import build as B

pytestmark = pytest.mark.gpu

TOL_PLAIN = 1e-3
STATUS_INVALID = 4


def reference(torch, w, centres, radii, band):
    """Signatures and gathered atoms from the context-based entry points."""
    ctx = apt.Context(0)
    h = ctx.handle
    apt.aptidx_load_positions(h, torch.from_numpy(w.xyz).cuda())
    apt.aptidx_set_directions(h, torch.from_numpy(w.dirs).cuda())
    apt.aptidx_set_binning(h, w.m, band[0], band[1])
    apt.aptidx_set_rois(h, torch.from_numpy(centres).cuda(), torch.from_numpy(radii).cuda())
    nroi, nv = centres.shape[0], w.dirs.shape[0]
    S = torch.empty((nroi, nv), dtype=torch.float32, device="cuda")
    apt.aptidx_compute_signatures(h, apt.APTIDX_PATH_PLAIN_FP32, 0, S, None, None)
    apt.aptidx_sync(h)
    atoms = [apt.aptidx_get_roi_atoms(h, r) for r in range(nroi)]
    ctx.close()
    return S.cpu().numpy(), atoms


def packed(torch, atoms):
    n = np.array([a.shape[0] for a in atoms], np.int64)
    off = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
    xc4 = np.zeros((max(int(off[-1]), 1), 4), np.float32)
    for r, a in enumerate(atoms):
        xc4[off[r]:off[r + 1], :3] = a
    return torch.from_numpy(xc4).cuda(), torch.from_numpy(off).cuda()


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    B.build()
    return torch


def test_noalloc_matches_compute_signatures_on_two_calls(torch_cuda):
    torch = torch_cuda
    w = synth.tiny_fcc()
    nv = w.dirs.shape[0]
    u = torch.from_numpy(w.dirs).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    cases = [(w.centres, w.radii, (10, 11)),
             (np.ascontiguousarray(w.centres[::-1]), np.ascontiguousarray(w.radii[::-1] * 0.9), (6, 14))]
    for centres, radii, band in cases:
        S_ref, atoms = reference(torch, w, centres, radii, band)
        xc4, off = packed(torch, atoms)
        S = torch.full((centres.shape[0], nv), -1.0, dtype=torch.float32, device="cuda")
        apt.aptidx_signatures_noalloc(xc4, off, torch.from_numpy(radii).cuda(), u, w.m, band[0], band[1], S, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        S = S.cpu().numpy()
        assert np.array_equal(S, S_ref), "no-allocation signatures differ from aptidx_compute_signatures"
        So, _, _ = oracle.signatures(w.xyz, centres, radii, band[0], band[1], w.dirs, w.m)
        rel = np.abs(S.astype(np.float64) - So).max(axis=1) / So.max(axis=1)
        assert rel.max() <= TOL_PLAIN, rel


def test_noalloc_wide_band_and_no_status_word(torch_cuda):
    """k = 8..128 at 2^8 bins: 31 groups of four frequencies, more than the
    kernel's 16 warps, so the spectrum takes the per-warp band-maximum branch."""
    torch = torch_cuda
    w = synth.tiny_fcc()
    band = (8, 128)
    S_ref, atoms = reference(torch, w, w.centres, w.radii, band)
    xc4, off = packed(torch, atoms)
    S = torch.full((w.centres.shape[0], w.dirs.shape[0]), -1.0, dtype=torch.float32, device="cuda")
    apt.aptidx_signatures_noalloc(xc4, off, torch.from_numpy(w.radii).cuda(), torch.from_numpy(w.dirs).cuda(), w.m,
                                  band[0], band[1], S, None)
    torch.cuda.synchronize()
    assert np.array_equal(S.cpu().numpy(), S_ref)


def test_noalloc_status_flags_invalid_inputs(torch_cuda):
    torch = torch_cuda
    w = synth.tiny_fcc()
    _, atoms = reference(torch, w, w.centres[:3], w.radii[:3], (10, 11))
    xc4, off = packed(torch, atoms)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # one direction of norm 1.1
    u = np.array([[1.1, 0.0, 0.0], [0.0, 1.0, 0.0]], np.float32)
    S = torch.zeros((3, 2), dtype=torch.float32, device="cuda")
    apt.aptidx_signatures_noalloc(xc4, off, torch.from_numpy(w.radii[:3]).cuda(), torch.from_numpy(u).cuda(), w.m,
                                  10, 11, S, status)
    torch.cuda.synchronize()
    assert int(status.item()) == STATUS_INVALID
    # a zero radius: INVALID and a zero row for that ROI, the others computed
    status.zero_()
    radii = np.array([w.radii[0], 0.0, w.radii[2]])
    u = np.ascontiguousarray(w.dirs[:64])
    S = torch.full((3, 64), -1.0, dtype=torch.float32, device="cuda")
    apt.aptidx_signatures_noalloc(xc4, off, torch.from_numpy(radii).cuda(), torch.from_numpy(u).cuda(), w.m, 10, 11,
                                  S, status)
    torch.cuda.synchronize()
    assert int(status.item()) == STATUS_INVALID
    S = S.cpu().numpy()
    assert np.all(S[1] == 0.0) and np.all(S[0] > 0.0) and np.all(S[2] > 0.0)


def test_noalloc_rejects_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    one = torch.zeros(4, dtype=torch.float32, device="cuda")
    off = torch.zeros(2, dtype=torch.int64, device="cuda")
    S = torch.zeros(1, dtype=torch.float32, device="cuda")
    big = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = apt.load()
    rc = lib.aptidx_signatures_noalloc(one.data_ptr(), off.data_ptr(), big.data_ptr(), 65537, one.data_ptr(), 1,
                                       8, 1, 2, S.data_ptr(), None, None)
    assert rc == apt.APTIDX_E_INVALID_ARG
    rc = lib.aptidx_signatures_noalloc(one.data_ptr(), off.data_ptr(), big.data_ptr(), 1, one.data_ptr(), 65537,
                                       8, 1, 2, S.data_ptr(), None, None)
    assert rc == apt.APTIDX_E_INVALID_ARG
    rc = lib.aptidx_signatures_noalloc(one.data_ptr(), off.data_ptr(), big.data_ptr(), 1, one.data_ptr(), 1,
                                       13, 1, 2, S.data_ptr(), None, None)
    assert rc == apt.APTIDX_E_INVALID_ARG
    # the binding checks dtypes before anything reaches the library
    with pytest.raises(TypeError):
        apt.aptidx_signatures_noalloc(one.reshape(1, 4), off.to(torch.int32), big, one[:3].reshape(1, 3), 8, 1, 2,
                                      S.reshape(1, 1))
