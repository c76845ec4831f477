"""GPU parity of steps (a1)-(a5), plain FP32 path, against the FP64 oracle.

Gather: N_w and the centred FP32 coordinates are identical (as sets).
Histograms: bit-exact.  Signatures: per-ROI error
e = max_v |S_gpu - S_oracle| / max_v S_oracle <= 1e-3 (FP32 path).
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2009_00735_gb300 as apt
from paper_2009_00735_gb300 import build as B

pytestmark = pytest.mark.gpu

TOL_PLAIN = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    return torch


def roi_error(S_gpu, S_orc):
    S_gpu = np.asarray(S_gpu, np.float64)
    S_orc = np.asarray(S_orc, np.float64)
    den = np.maximum(S_orc.max(axis=-1), 1e-30)
    return np.abs(S_gpu - S_orc).max(axis=-1) / den


def sorted_rows(x):
    x = np.asarray(x)
    return x[np.lexsort(x.T[::-1])]


def make_ctx(torch, w, band=None, dirs=None, m=None, types=None, type_mask=0xFFFFFFFF):
    ctx = apt.Context(0)
    h = ctx.handle
    apt.aptidx_load_positions(h, torch.from_numpy(w.xyz).cuda(), None if types is None else torch.from_numpy(types).cuda())
    d = w.dirs if dirs is None else dirs
    apt.aptidx_set_directions(h, torch.from_numpy(np.ascontiguousarray(d)).cuda())
    mm = w.m if m is None else m
    if band is None:
        band = oracle.band_for_spacing(*w.d_spacing, float(w.radii[0]), mm)
    apt.aptidx_set_binning(h, mm, band[0], band[1])
    apt.aptidx_set_rois(h, torch.from_numpy(w.centres).cuda(), torch.from_numpy(w.radii).cuda(),
                        type_mask=type_mask)
    return ctx, band, mm, d


def gpu_signatures(torch, ctx, nroi, nv, path=apt.APTIDX_PATH_PLAIN_FP32, flags=0):
    S = torch.empty((nroi, nv), dtype=torch.float32, device="cuda")
    A = torch.empty((nroi, nv), dtype=torch.uint16, device="cuda")
    N = torch.empty(nroi, dtype=torch.int32, device="cuda")
    apt.aptidx_compute_signatures(ctx.handle, path, flags, S, A, N)
    apt.aptidx_sync(ctx.handle)
    return S.cpu().numpy(), A.cpu().numpy().astype(np.int64), N.cpu().numpy()


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_fcc()


def test_gather_parity(torch_cuda, tiny):
    ctx, band, m, d = make_ctx(torch_cuda, tiny)
    for r in range(tiny.centres.shape[0]):
        xc_gpu = apt.aptidx_get_roi_atoms(ctx.handle, r)
        _, xc_orc = oracle.gather(tiny.xyz, tiny.centres[r], tiny.radii[r])
        assert xc_gpu.shape == xc_orc.shape
        assert np.array_equal(sorted_rows(xc_gpu), sorted_rows(xc_orc))
    ctx.close()


@pytest.mark.parametrize("roi", [0, 5, 15])
def test_histograms_bit_exact(torch_cuda, tiny, roi):
    ctx, band, m, d = make_ctx(torch_cuda, tiny)
    nv = d.shape[0]
    h = np.empty((nv, 1 << m), np.uint16)
    apt.aptidx_get_histograms(ctx.handle, roi, apt.APTIDX_PATH_PLAIN_FP32, h)
    _, xc = oracle.gather(tiny.xyz, tiny.centres[roi], tiny.radii[roi])
    ref = oracle.histograms(xc, d, m, tiny.radii[roi])
    assert np.array_equal(h.astype(np.int64), ref.astype(np.int64))
    ctx.close()


def test_signatures_plain_tiny(torch_cuda, tiny):
    ctx, band, m, d = make_ctx(torch_cuda, tiny)
    nroi, nv = tiny.centres.shape[0], d.shape[0]
    S, A, N = gpu_signatures(torch_cuda, ctx, nroi, nv)
    So, Ao, No = oracle.signatures(tiny.xyz, tiny.centres, tiny.radii, band[0], band[1], d, m)
    assert np.array_equal(N, No)
    e = roi_error(S, So)
    assert e.max() <= TOL_PLAIN, e
    # argk: a frequency of the band whose oracle amplitude equals the maximum
    assert np.all((A >= band[0]) & (A <= band[1]))
    agree = (A == Ao).mean()
    assert agree > 0.999
    ctx.close()


def test_host_and_device_outputs_agree(torch_cuda, tiny):
    ctx, band, m, d = make_ctx(torch_cuda, tiny)
    nroi, nv = tiny.centres.shape[0], d.shape[0]
    S, A, N = gpu_signatures(torch_cuda, ctx, nroi, nv)
    Sh = np.empty((nroi, nv), np.float32)
    Ah = np.empty((nroi, nv), np.uint16)
    Nh = np.empty(nroi, np.int32)
    apt.aptidx_compute_signatures(ctx.handle, apt.APTIDX_PATH_PLAIN_FP32, 0, Sh, Ah, Nh)
    assert np.array_equal(S, Sh) and np.array_equal(A, Ah) and np.array_equal(N, Nh)
    S2, _, _ = gpu_signatures(torch_cuda, ctx, nroi, nv)
    assert np.array_equal(S, S2)       # deterministic run to run
    ctx.close()


def test_normalise_flag(torch_cuda, tiny):
    ctx, band, m, d = make_ctx(torch_cuda, tiny)
    nroi, nv = tiny.centres.shape[0], d.shape[0]
    S, _, _ = gpu_signatures(torch_cuda, ctx, nroi, nv)
    Sn, _, _ = gpu_signatures(torch_cuda, ctx, nroi, nv, flags=apt.APTIDX_NORMALISE_MAX)
    ref = oracle.normalise(S.astype(np.float64))
    assert np.allclose(Sn, ref, rtol=1e-6, atol=1e-7)
    assert np.allclose(Sn.max(axis=1), 1.0)
    ctx.close()


@pytest.mark.parametrize("case", ["ragged_nv", "band_one", "band_wide", "m9", "m10", "empty_roi", "typemask"])
def test_plain_edge_cases(torch_cuda, tiny, case):
    w = tiny
    dirs = w.dirs
    m = 8
    band = None
    types = None
    mask = 0xFFFFFFFF
    centres = w.centres.copy()
    if case == "ragged_nv":
        dirs = np.ascontiguousarray(w.dirs[:100])
    elif case == "band_one":
        band = (11, 11)
    elif case == "band_wide":
        band = (0, 128)                 # K = 129 > 64 frequencies: per-warp maximum path
        dirs = np.ascontiguousarray(w.dirs[:700])
    elif case == "m9":
        m = 9
        dirs = np.ascontiguousarray(w.dirs[:1000])
    elif case == "m10":
        m = 10
        dirs = np.ascontiguousarray(w.dirs[:1000])
    elif case == "empty_roi":
        centres[3] = [100.0, 100.0, 100.0]
    elif case == "typemask":
        types = (np.arange(w.xyz.shape[0]) % 3).astype(np.uint8)
        mask = 0b101
    w2 = synth.Workload(w.name, w.xyz, w.types, centres, w.radii, dirs, m, w.d_spacing)
    if band is None:
        band = oracle.band_for_spacing(*w.d_spacing, 1.0, m)
    ctx, band, m, d = make_ctx(torch_cuda, w2, band=band, m=m, types=types, type_mask=mask)
    nroi, nv = centres.shape[0], d.shape[0]
    S, A, N = gpu_signatures(torch_cuda, ctx, nroi, nv)
    So, Ao, No = oracle.signatures(w.xyz, centres, w.radii, band[0], band[1], d, m,
                                   types=types, type_mask=mask)
    assert np.array_equal(N, No)
    if case == "empty_roi":
        assert N[3] == 0 and np.all(S[3] == 0)
        keep = np.arange(nroi) != 3
        assert roi_error(S[keep], So[keep]).max() <= TOL_PLAIN
    else:
        assert roi_error(S, So).max() <= TOL_PLAIN
    ctx.close()


def test_large_roi_chunked_atoms(torch_cuda):
    """More atoms than one shared-memory stage holds (restaged per tile)."""
    xyz, t = synth.perfect_crystal_roi("fcc", 0.404, 2.7)
    rng = np.random.default_rng(1)
    xyz = (xyz.astype(np.float64) + rng.normal(0, 0.02, xyz.shape)).astype(np.float32)
    centres = np.array([[0.0, 0.0, 0.0], [0.1, -0.05, 0.02]])
    radii = np.array([2.6, 2.6])
    dirs = np.ascontiguousarray(synth.icosphere(3))
    w = synth.Workload("big", xyz, t, centres, radii, dirs, 8, synth.band_spacing(0.202))
    ctx, band, m, d = make_ctx(torch_cuda, w)
    S, A, N = gpu_signatures(torch_cuda, ctx, 2, d.shape[0])
    So, Ao, No = oracle.signatures(xyz, centres, radii, band[0], band[1], d, m)
    assert np.array_equal(N, No) and N.min() > 4096
    assert roi_error(S, So).max() <= TOL_PLAIN
    h = np.empty((d.shape[0], 1 << m), np.uint16)
    apt.aptidx_get_histograms(ctx.handle, 1, apt.APTIDX_PATH_PLAIN_FP32, h)
    _, xc = oracle.gather(xyz, centres[1], radii[1])
    assert np.array_equal(h.astype(np.int64), oracle.histograms(xc, d, m, radii[1]).astype(np.int64))
    ctx.close()


def test_invalid_arguments(torch_cuda, tiny):
    ctx = apt.Context(0)
    h = ctx.handle
    with pytest.raises(apt.AptidxError) as ei:
        apt.aptidx_set_rois(h, tiny.centres, tiny.radii)
    assert ei.value.code == apt.APTIDX_E_STATE
    with pytest.raises(apt.AptidxError) as ei:
        bad = tiny.xyz.copy()
        bad[5, 1] = np.nan
        apt.aptidx_load_positions(h, bad)
    assert ei.value.code == apt.APTIDX_E_INVALID_ARG
    apt.aptidx_load_positions(h, tiny.xyz)
    # every non-finite form, also into the buffers of a same-sized set; the
    # context then holds no positions until a good set is loaded
    for i, v in [(0, np.inf), (tiny.xyz.shape[0] - 1, -np.inf), (7, -np.nan)]:
        bad = tiny.xyz.copy()
        bad[i, 2] = v
        with pytest.raises(apt.AptidxError) as ei:
            apt.aptidx_load_positions(h, bad)
        assert ei.value.code == apt.APTIDX_E_INVALID_ARG
        apt.aptidx_set_directions(h, tiny.dirs)
        apt.aptidx_set_binning(h, 8, 10, 11)
        with pytest.raises(apt.AptidxError) as ei:
            apt.aptidx_set_rois(h, tiny.centres, tiny.radii)
        assert ei.value.code == apt.APTIDX_E_STATE
    apt.aptidx_load_positions(h, tiny.xyz)
    with pytest.raises(apt.AptidxError):
        apt.aptidx_set_directions(h, tiny.dirs * 1.01)
    apt.aptidx_set_directions(h, tiny.dirs)
    for m, lo, hi in [(7, 1, 2), (13, 1, 2), (8, 5, 4), (8, 0, 129)]:
        with pytest.raises(apt.AptidxError) as ei:
            apt.aptidx_set_binning(h, m, lo, hi)
        assert ei.value.code == apt.APTIDX_E_INVALID_ARG
    apt.aptidx_set_binning(h, 8, 10, 11)
    with pytest.raises(apt.AptidxError):
        apt.aptidx_set_rois(h, tiny.centres, -tiny.radii)
    with pytest.raises(apt.AptidxError) as ei:
        apt.aptidx_compute_signatures(h, 0, 0, np.empty((16, tiny.dirs.shape[0]), np.float32))
    assert ei.value.code == apt.APTIDX_E_STATE
    apt.aptidx_set_rois(h, tiny.centres, tiny.radii)
    with pytest.raises(apt.AptidxError):
        apt.aptidx_compute_signatures(h, 7, 0, np.empty((16, tiny.dirs.shape[0]), np.float32))
    ctx.close()


def test_roi_atom_limit(torch_cuda):
    """A ROI above APTIDX_MAX_ATOMS_PER_ROI (2^24 - 1) selected atoms is
    refused with OVERFLOW."""
    rng = np.random.default_rng(0)
    xyz = (rng.random((1 << 24, 3), dtype=np.float32) * np.float32(0.5))
    ctx = apt.Context(0)
    h = ctx.handle
    apt.aptidx_load_positions(h, xyz)
    apt.aptidx_set_directions(h, synth.icosphere(1))
    apt.aptidx_set_binning(h, 8, 10, 11)
    with pytest.raises(apt.AptidxError) as ei:
        apt.aptidx_set_rois(h, np.array([[0.25, 0.25, 0.25]]), np.array([2.0]))
    assert ei.value.code == apt.APTIDX_E_OVERFLOW
    ctx.close()


@pytest.fixture(scope="module")
def single_crystal():
    return synth.single_crystal_bcc()


def antipodes(u):
    from scipy.spatial import cKDTree
    t = cKDTree(u.astype(np.float64))
    _, j = t.query(-u.astype(np.float64))
    return j


def test_full_size_single_crystal_sampled(torch_cuda, single_crystal):
    """8192 ROIs x 40962 directions x 1024 bins in the benchmark's launch
    configuration; sampled ROIs and directions against the oracle, and
    properties that hold everywhere: 0 <= S <= N_w and S(-u) = S(u)."""
    w = single_crystal
    ctx, band, m, d = make_ctx(torch_cuda, w)
    nroi, nv = w.centres.shape[0], d.shape[0]
    S, A, N = gpu_signatures(torch_cuda, ctx, nroi, nv)
    rng = np.random.default_rng(3)
    rois = [0, nroi // 2 + 17, nroi - 1] + list(rng.choice(nroi, 3, replace=False))
    vs = np.sort(rng.choice(nv, 700, replace=False))
    vs[:3] = [0, nv // 2, nv - 1]
    vs = np.unique(vs)
    for r in rois:
        _, xc = oracle.gather(w.xyz, w.centres[r], w.radii[r])
        assert N[r] == xc.shape[0]
        So, _ = oracle.roi_signature(xc, d[vs], m, w.radii[r], band[0], band[1])
        assert roi_error(S[r, vs], So) <= TOL_PLAIN
    assert np.all(S >= 0)
    assert np.all(S <= N[:, None].astype(np.float32) * (1 + 1e-5) + 1e-3)
    j = antipodes(d)
    rel = np.abs(S - S[:, j]).max(axis=1) / S.max(axis=1)
    assert rel.max() <= TOL_PLAIN
    ctx.close()
