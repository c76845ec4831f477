"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a
GPU, and exports every function include/aptidx.h declares."""
import os
import re

import pytest

import paper_2009_00735_gb300 as apt
from paper_2009_00735_gb300 import build as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "aptidx.h")


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(aptidx_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return apt.load()


def test_header_declares_the_hot_path_calls():
    names = declared()
    for n in ["aptidx_create", "aptidx_load_positions", "aptidx_set_directions", "aptidx_set_binning",
              "aptidx_set_rois", "aptidx_compute_signatures", "aptidx_match", "aptidx_refine",
              "aptidx_refine_loss", "aptidx_build_lut", "aptidx_set_reference", "aptidx_sync",
              "aptidx_get_histograms", "aptidx_last_error", "aptidx_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert apt.aptidx_version() >= 100


def test_binding_names_match_header():
    for n in declared():
        assert hasattr(apt, n), n


def test_library_does_not_reference_oracle():
    with open(apt.library_path(), "rb") as fh:
        blob = fh.read()
    assert b"orc_" not in blob and b"liboracle" not in blob


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes as C
    h = C.c_void_p()
    rc = lib.aptidx_create(C.byref(h), 0, None)
    assert rc == apt.APTIDX_E_INVALID_ARG and not h.value


def test_band_for_spacing_matches_oracle(lib):
    """aptidx_band_for_spacing (host code of the library, no GPU) against the
    oracle's band arithmetic, and its argument checks."""
    import oracle
    import synth
    for R, m in [(1.0, 8), (2.0, 10), (1.37, 9), (2.5, 11), (3.1, 12)]:
        for d in [0.2025, 0.2029, 0.25]:
            lo, hi = synth.band_spacing(d)
            assert apt.aptidx_band_for_spacing(lo, hi, R, m) == oracle.band_for_spacing(lo, hi, R, m)
    assert apt.band_for_spacing is apt.aptidx_band_for_spacing
    for bad in [(0.0, 0.2, 2.0, 10), (0.3, 0.2, 2.0, 10), (0.2, 0.3, 0.0, 10), (0.2, 0.3, 2.0, 7),
                (0.2, 0.3, 2.0, 13), (1e-4, 2e-4, 2.0, 8)]:   # the last band exceeds 2^(m-1)
        with pytest.raises(apt.AptidxError):
            apt.aptidx_band_for_spacing(*bad)


def test_binding_constants_match_header():
    """Every numeric #define of include/aptidx.h that a caller passes or
    receives (status codes, memory spaces, paths, flags, limits) exists in the
    binding with the header's value."""
    src = open(HEADER).read()
    defs = dict(re.findall(r"^#define\s+(APTIDX_\w+)\s+\(?([0-9]+)u?\)?", src, re.M))
    assert len(defs) > 20
    must = [n for n in defs if n.startswith(("APTIDX_E_", "APTIDX_MEM_", "APTIDX_PATH_"))] + [
        "APTIDX_OK", "APTIDX_NORMALISE_MAX", "APTIDX_AUTOTUNE", "APTIDX_GRAPH", "APTIDX_DIRECT", "APTIDX_MAX_TOPK",
        "APTIDX_MAX_BANDS"]
    for n in must:
        assert hasattr(apt, n), n
    for n, v in defs.items():
        if hasattr(apt, n):
            assert getattr(apt, n) == int(v), n
