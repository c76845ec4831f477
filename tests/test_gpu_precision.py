"""Precision of the band spectrum on the b.c.c. single crystal (4.33 M atoms,
8192 ROIs of R = 2 nm, 40962 directions, 2^10 bins), with the signature taken
over frequency bins 8..128 and over the {110} band (k = 18..21).

Three arithmetic paths of Eq. 1 + the amplitude spectrum are compared per ROI,
e = max_v |S - S_ref| / max_v S_ref:
  tensor cores   fp16 counts x (hi + lo) fp16 twiddles, FP32 accumulate
  CUDA cores     FP32 twiddles and FP32 sums
  oracle         FP64
The test prints max and median of e for each pair and bounds them by the
tolerances the paths are held to elsewhere (5e-3 tensor cores, 1e-3 FP32).
"""
import numpy as np
import pytest

import oracle
import paper_2009_00735_gb300 as apt

from test_gpu_plain import TOL_PLAIN, gpu_signatures, make_ctx, roi_error, single_crystal, torch_cuda  # noqa: F401

pytestmark = pytest.mark.gpu

TOL_TC = 5e-3


@pytest.mark.parametrize("which", ["wide", "110"])
def test_band_precision(torch_cuda, single_crystal, which):
    w = single_crystal
    BAND = (8, 128) if which == "wide" else oracle.band_for_spacing(*w.d_spacing, float(w.radii[0]), w.m)
    ctx, band, m, d = make_ctx(torch_cuda, w, band=BAND)
    nroi, nv = w.centres.shape[0], d.shape[0]
    St, At, Nt = gpu_signatures(torch_cuda, ctx, nroi, nv, path=apt.APTIDX_PATH_TC_FP16)
    Sp, Ap, Np = gpu_signatures(torch_cuda, ctx, nroi, nv)
    ctx.close()
    assert np.array_equal(Nt, Np)
    assert np.all((At >= BAND[0]) & (At <= BAND[1]))
    e_tp = roi_error(St, Sp)
    rng = np.random.default_rng(8)
    rois = np.unique(np.concatenate([[0, nroi - 1], rng.choice(nroi, 46, replace=False)]))
    vs = np.unique(np.concatenate([[0, nv - 1], rng.choice(nv, 1022, replace=False)]))
    dv = np.ascontiguousarray(d[vs])
    e_t, e_p = [], []
    for r in rois:
        _, xc = oracle.gather(w.xyz, w.centres[r], w.radii[r])
        So, _ = oracle.roi_signature(xc, dv, m, w.radii[r], *BAND)
        e_t.append(roi_error(St[r, vs], So))
        e_p.append(roi_error(Sp[r, vs], So))
    e_t, e_p = np.array(e_t), np.array(e_p)
    print(f"\nband {BAND[0]}..{BAND[1]}, {rois.size} ROIs x {vs.size} directions vs FP64 oracle: "
          f"tensor cores max {e_t.max():.3e} median {np.median(e_t):.3e}; "
          f"FP32 max {e_p.max():.3e} median {np.median(e_p):.3e}; "
          f"tensor cores vs FP32 over all {nroi} ROIs x {nv} directions: max {e_tp.max():.3e} "
          f"median {np.median(e_tp):.3e}")
    assert e_t.max() <= TOL_TC
    assert e_p.max() <= TOL_PLAIN
    assert e_tp.max() <= TOL_TC
