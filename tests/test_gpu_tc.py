"""GPU parity of the tensor-core path (tcgen05) against the FP64 oracle.

Histograms from the tensor-core kernel's own histogram stage are bit-exact;
signatures satisfy e = max_v |S_gpu - S_oracle| / max_v S_oracle <= 5e-3.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2009_00735_gb300 as apt

from test_gpu_plain import (TOL_PLAIN, antipodes, gpu_signatures, make_ctx, roi_error, single_crystal,  # noqa: F401
                            tiny, torch_cuda)

pytestmark = pytest.mark.gpu

TOL_TC = 5e-3
TC = apt.APTIDX_PATH_TC_FP16


@pytest.fixture(scope="module")
def tc(torch_cuda):
    ctx = apt.Context(0)
    ok = apt.aptidx_path_supported(ctx.handle, TC)
    ctx.close()
    assert ok, "tensor-core path must be available on GB300"
    return torch_cuda


@pytest.mark.parametrize("roi", [0, 7, 15])
def test_tc_histograms_bit_exact(tc, tiny, roi):
    ctx, band, m, d = make_ctx(tc, tiny)
    h = np.empty((d.shape[0], 1 << m), np.uint16)
    apt.aptidx_get_histograms(ctx.handle, roi, TC, h)
    _, xc = oracle.gather(tiny.xyz, tiny.centres[roi], tiny.radii[roi])
    assert np.array_equal(h.astype(np.int64), oracle.histograms(xc, d, m, tiny.radii[roi]).astype(np.int64))
    ctx.close()


def test_tc_signatures_tiny(tc, tiny):
    ctx, band, m, d = make_ctx(tc, tiny)
    nroi, nv = tiny.centres.shape[0], d.shape[0]
    S, A, N = gpu_signatures(tc, ctx, nroi, nv, path=TC)
    So, Ao, No = oracle.signatures(tiny.xyz, tiny.centres, tiny.radii, band[0], band[1], d, m)
    assert np.array_equal(N, No)
    e = roi_error(S, So)
    assert e.max() <= TOL_TC, e
    assert np.all((A >= band[0]) & (A <= band[1]))
    assert (A == Ao).mean() > 0.99
    Sp, _, _ = gpu_signatures(tc, ctx, nroi, nv)
    assert roi_error(S, Sp).max() <= TOL_TC
    S2, _, _ = gpu_signatures(tc, ctx, nroi, nv, path=TC)
    assert np.array_equal(S, S2)          # deterministic run to run
    ctx.close()


@pytest.mark.parametrize("case", ["ragged_nv", "band_one", "band_multi_batch", "m9", "m10", "empty_roi",
                                  "typemask", "per_roi_bands"])
def test_tc_edge_cases(tc, tiny, case):
    w = tiny
    dirs = w.dirs
    m = 8
    band = None
    types = None
    mask = 0xFFFFFFFF
    centres = w.centres.copy()
    blo = bhi = None
    if case == "ragged_nv":
        dirs = np.ascontiguousarray(w.dirs[:100])
    elif case == "band_one":
        band = (11, 11)
    elif case == "band_multi_batch":
        band = (2, 60)                  # 15 frequency groups: two shared-memory batches at m = 8
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
        mask = 0b011
    elif case == "per_roi_bands":
        rng = np.random.default_rng(0)
        blo = rng.integers(3, 20, centres.shape[0]).astype(np.int32)
        bhi = (blo + rng.integers(0, 9, centres.shape[0])).astype(np.int32)
    if band is None:
        band = oracle.band_for_spacing(*w.d_spacing, 1.0, m)
    ctx = apt.Context(0)
    h = ctx.handle
    apt.aptidx_load_positions(h, tc.from_numpy(w.xyz).cuda(), None if types is None else tc.from_numpy(types).cuda())
    apt.aptidx_set_directions(h, tc.from_numpy(np.ascontiguousarray(dirs)).cuda())
    apt.aptidx_set_binning(h, m, band[0], band[1])
    apt.aptidx_set_rois(h, centres, w.radii, blo, bhi, type_mask=mask)
    nroi, nv = centres.shape[0], dirs.shape[0]
    S, A, N = gpu_signatures(tc, ctx, nroi, nv, path=TC)
    lo = blo if blo is not None else band[0]
    hi = bhi if bhi is not None else band[1]
    So, Ao, No = oracle.signatures(w.xyz, centres, w.radii, lo, hi, dirs, m, types=types, type_mask=mask)
    assert np.array_equal(N, No)
    if case == "empty_roi":
        assert N[3] == 0 and np.all(S[3] == 0)
        keep = np.arange(nroi) != 3
        assert roi_error(S[keep], So[keep]).max() <= TOL_TC
    else:
        assert roi_error(S, So).max() <= TOL_TC
    ctx.close()


def test_tc_large_rois_in_atom_blocks(tc):
    """ROIs above 2048 atoms run on the tensor cores in blocks of at most 2048
    atoms (every count of a block exact in fp16), contracted into the same
    accumulators; ROIs of both kinds in one call match the oracle."""
    xyz, t = synth.perfect_crystal_roi("fcc", 0.404, 2.7)
    rng = np.random.default_rng(2)
    xyz = (xyz.astype(np.float64) + rng.normal(0, 0.02, xyz.shape)).astype(np.float32)
    centres = np.array([[0.0, 0.0, 0.0], [0.3, 0.1, -0.2], [0.05, 0.0, 0.1], [-0.2, 0.2, 0.0]])
    radii = np.array([2.6, 1.2, 2.2, 1.0])
    dirs = np.ascontiguousarray(synth.icosphere(3))
    w = synth.Workload("mixed", xyz, t, centres, radii, dirs, 8, synth.band_spacing(0.202))
    band = (8, 30)
    ctx, band, m, d = make_ctx(tc, w, band=band)
    S, A, N = gpu_signatures(tc, ctx, 4, d.shape[0], path=TC)
    So, Ao, No = oracle.signatures(xyz, centres, radii, band[0], band[1], d, m)
    assert np.array_equal(N, No)
    assert N.max() > 2048 and N.min() < 2048
    assert roi_error(S, So).max() <= TOL_TC
    ctx.close()


def test_tc_full_size_single_crystal_sampled(tc, single_crystal):
    w = single_crystal
    ctx, band, m, d = make_ctx(tc, w)
    nroi, nv = w.centres.shape[0], d.shape[0]
    S, A, N = gpu_signatures(tc, ctx, nroi, nv, path=TC)
    rng = np.random.default_rng(4)
    rois = [0, nroi // 3, nroi - 1] + list(rng.choice(nroi, 3, replace=False))
    vs = np.unique(np.concatenate([[0, nv // 2, nv - 1], rng.choice(nv, 700, replace=False)]))
    for r in rois:
        _, xc = oracle.gather(w.xyz, w.centres[r], w.radii[r])
        assert N[r] == xc.shape[0]
        So, _ = oracle.roi_signature(xc, d[vs], m, w.radii[r], band[0], band[1])
        assert roi_error(S[r, vs], So) <= TOL_TC
    assert np.all(S >= 0)
    assert np.all(S <= N[:, None].astype(np.float32) * (1 + 1e-3) + 1e-2)
    j = antipodes(d)
    assert (np.abs(S - S[:, j]).max(axis=1) / S.max(axis=1)).max() <= TOL_TC
    Sp, _, _ = gpu_signatures(tc, ctx, nroi, nv)
    assert roi_error(S, Sp).max() <= TOL_TC
    ctx.close()


def test_autotune_and_graph_replay(tc, tiny, tmp_path, monkeypatch):
    """APTIDX_AUTOTUNE picks a launch configuration (and persists it in
    APTIDX_TUNE_CACHE); APTIDX_GRAPH captures the call once and replays it.
    Results agree with the plain launches of the same path; changing the ROI
    set discards the graph."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("APTIDX_TUNE_CACHE", str(cache))
    ctx, band, m, d = make_ctx(tc, tiny)
    nroi, nv = tiny.centres.shape[0], d.shape[0]
    for path in (apt.APTIDX_PATH_PLAIN_FP32, TC):
        S_ref, _, _ = gpu_signatures(tc, ctx, nroi, nv, path=path)
        flags = apt.APTIDX_AUTOTUNE | apt.APTIDX_GRAPH
        S1, _, _ = gpu_signatures(tc, ctx, nroi, nv, path=path, flags=flags)
        S2, _, _ = gpu_signatures(tc, ctx, nroi, nv, path=path, flags=flags)
        assert np.array_equal(S1, S2)
        assert roi_error(S1, S_ref).max() <= 1e-5
        tpi, iss = apt.aptidx_get_tuning(ctx.handle, path)
        assert tpi in (4, 8, 16, 32)
        assert iss in ((2, 4) if path == TC else (0,))
    assert cache.exists() and len(cache.read_text().splitlines()) == 2
    # a new ROI set discards the captured graphs
    apt.aptidx_set_rois(ctx.handle, tiny.centres[:5], tiny.radii[:5])
    S3 = tc.empty((5, nv), dtype=tc.float32, device="cuda")
    apt.aptidx_compute_signatures(ctx.handle, TC, apt.APTIDX_GRAPH, S3, None, None)
    apt.aptidx_sync(ctx.handle)
    So, _, _ = oracle.signatures(tiny.xyz, tiny.centres[:5], tiny.radii[:5], band[0], band[1], d, m)
    assert roi_error(S3.cpu().numpy(), So).max() <= TOL_TC
    ctx.close()
