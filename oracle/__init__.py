"""FP64 CPU oracle of the RSP signature method (arXiv 2009.00735) -- TEST
INFRASTRUCTURE.

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import
this package.  The CUDA library never calls it and shares no code with it.
The arithmetic lives in ``aptidx_oracle.c`` (plain C, FP64); this module
compiles it with gcc and exposes numpy-friendly wrappers.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aptidx_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


def build_mutant(k: int) -> str:
    """Test-only: the oracle compiled with planted mistake k (the
    ORC_MUTATION points of the C source), for checking that the pins catch
    it.  Returns the library path."""
    path = os.path.join(os.path.dirname(_LIB), f"liboracle_mut{int(k)}.so")
    if os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(_SRC):
        return path
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                    f"-DORC_MUTATION={int(k)}", "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, path)
    return path


def use_library(path=None):
    """Test-only: route every wrapper to the library at `path` (None: the
    default build)."""
    global _lib
    _lib = C.CDLL(path if path else build())
    _declare(_lib)


_p = C.c_void_p
_i64 = C.c_int64
_i32 = C.c_int32
_d = C.c_double


def _declare(L):
    L.orc_gather.restype = _i64
    L.orc_gather.argtypes = [_p, _i64, _p, C.c_uint32, _p, _d, _p, _p]
    L.orc_bin_eq1.restype = C.c_int
    L.orc_bin_eq1.argtypes = [_p, _p, C.c_int, _d]
    L.orc_bin_contract.restype = C.c_int
    L.orc_bin_contract.argtypes = [_p, _p, C.c_int, _d]
    L.orc_bin_scale.restype = C.c_float
    L.orc_bin_scale.argtypes = [C.c_int, _d]
    L.orc_project_f32.restype = C.c_float
    L.orc_project_f32.argtypes = [_p, _p]
    L.orc_histograms.restype = None
    L.orc_histograms.argtypes = [_p, _i64, _p, _i64, C.c_int, _d, _p]
    L.orc_histograms_eq1.restype = None
    L.orc_histograms_eq1.argtypes = [_p, _i64, _p, _i64, C.c_int, _d, _p]
    L.orc_band_amplitudes.restype = None
    L.orc_band_amplitudes.argtypes = [_p, C.c_int, C.c_int, C.c_int, _p]
    L.orc_roi_signature.restype = None
    L.orc_roi_signature.argtypes = [_p, _i64, _p, _i64, C.c_int, _d, C.c_int, C.c_int, _p, _p]
    L.orc_signatures.restype = C.c_int
    L.orc_signatures.argtypes = [_p, _i64, _p, C.c_uint32, _p, _p, _i64, _p, _p, _p, _i64, C.c_int,
                                 _p, _p, _p, C.c_int]
    L.orc_normalise.restype = None
    L.orc_normalise.argtypes = [_p, _i64, _i64]
    L.orc_band_for_spacing.restype = None
    L.orc_band_for_spacing.argtypes = [_d, _d, _d, C.c_int, _p, _p]
    L.orc_quat_to_matrix.restype = None
    L.orc_quat_to_matrix.argtypes = [_p, _p]
    L.orc_disorientation_deg.restype = _d
    L.orc_disorientation_deg.argtypes = [_p, _p]
    L.orc_top_nodes.restype = None
    L.orc_top_nodes.argtypes = [_p, _i64, C.c_int, _p]
    L.orc_rotate_node.restype = None
    L.orc_rotate_node.argtypes = [_p, _p, _p]
    L.orc_nearest_node.restype = _i32
    L.orc_nearest_node.argtypes = [_p, _i64, _p]
    L.orc_lut.restype = None
    L.orc_lut.argtypes = [_p, _i64, _p, C.c_int, _p, _i64, _p, C.c_int]
    L.orc_match.restype = None
    L.orc_match.argtypes = [_p, _i64, _i64, _p, _p, C.c_int, _p, _i64, _p, _p, _p, C.c_int]
    L.orc_match_phase.restype = None
    L.orc_match_phase.argtypes = [_p, _i64, _i64, C.c_int, _p, _p, _p, _p, C.c_int, _p, _i64, _p, _p, _p, C.c_int]
    L.orc_fsp.restype = None
    L.orc_fsp.argtypes = [_p, _i64, C.c_int, _d, _p, _i64, _p]
    L.orc_bilinear.restype = C.c_int
    L.orc_bilinear.argtypes = [_p, _p, _p, _p, _p]
    L.orc_refine_eval.restype = None
    L.orc_refine_eval.argtypes = [_p, _p, _p, _i64, _p, _p, _p, _p, _p, _p]
    L.orc_refine.restype = None
    L.orc_refine.argtypes = [_p, _p, _p, _i64, _p, C.c_int, _p, _p]
    L.orc_refine_batch.restype = None
    L.orc_refine_batch.argtypes = [_p, _p, _p, _i64, _i64, _p, C.c_int, _p, _p, C.c_int]
    L.orc_openmp_threads.restype = C.c_int
    L.orc_openmp_threads.argtypes = []


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def threads() -> int:
    return int(lib().orc_openmp_threads())


# ---------------------------------------------------------------- signatures

def gather(xyz, centre, R, types=None, type_mask=0xFFFFFFFF):
    """(indices int64 [N_w], centred float32 [N_w, 3]) of atoms with |p - c| <= R."""
    xyz = _c(xyz, np.float32)
    c = _c(centre, np.float64)
    t = None if types is None else _c(types, np.uint8)
    n = xyz.shape[0]
    nw = lib().orc_gather(_ptr(xyz), n, _ptr(t), type_mask, _ptr(c), float(R), None, None)
    idx = np.empty(nw, np.int64)
    xc = np.empty((nw, 3), np.float32)
    lib().orc_gather(_ptr(xyz), n, _ptr(t), type_mask, _ptr(c), float(R), _ptr(idx), _ptr(xc))
    return idx, xc


def bin_contract(u, x, m, R) -> int:
    return int(lib().orc_bin_contract(_ptr(_c(u, np.float32)), _ptr(_c(x, np.float32)), m, float(R)))


def bin_eq1(u, x, m, R) -> int:
    return int(lib().orc_bin_eq1(_ptr(_c(u, np.float64)), _ptr(_c(x, np.float64)), m, float(R)))


def bin_scale(m, R) -> np.float32:
    return np.float32(lib().orc_bin_scale(m, float(R)))


def project_f32(u, x) -> np.float32:
    return np.float32(lib().orc_project_f32(_ptr(_c(u, np.float32)), _ptr(_c(x, np.float32))))


def histograms(xc, dirs, m, R, exact_eq1=False):
    """int32 [N_v, 2^m] SDM counts of centred atoms xc along dirs."""
    xc = _c(xc, np.float32).reshape(-1, 3)
    u = _c(dirs, np.float32).reshape(-1, 3)
    h = np.empty((u.shape[0], 1 << m), np.int32)
    f = lib().orc_histograms_eq1 if exact_eq1 else lib().orc_histograms
    f(_ptr(xc), xc.shape[0], _ptr(u), u.shape[0], m, float(R), _ptr(h))
    return h


def band_amplitudes(h, m, k_lo, k_hi):
    h = _c(h, np.int32)
    amp = np.empty(k_hi - k_lo + 1, np.float64)
    lib().orc_band_amplitudes(_ptr(h), m, k_lo, k_hi, _ptr(amp))
    return amp


def roi_signature(xc, dirs, m, R, k_lo, k_hi):
    xc = _c(xc, np.float32).reshape(-1, 3)
    u = _c(dirs, np.float32).reshape(-1, 3)
    S = np.empty(u.shape[0], np.float64)
    ak = np.empty(u.shape[0], np.int32)
    lib().orc_roi_signature(_ptr(xc), xc.shape[0], _ptr(u), u.shape[0], m, float(R), k_lo, k_hi,
                            _ptr(S), _ptr(ak))
    return S, ak


def signatures(xyz, centres, radii, band_lo, band_hi, dirs, m, types=None, type_mask=0xFFFFFFFF,
               threads=0):
    """(S float64 [N_roi, N_v], argk int32 [N_roi, N_v], N_w int64 [N_roi])."""
    xyz = _c(xyz, np.float32)
    cen = _c(centres, np.float64).reshape(-1, 3)
    rad = _c(radii, np.float64)
    nroi = cen.shape[0]
    blo = _c(np.broadcast_to(band_lo, (nroi,)), np.int32)
    bhi = _c(np.broadcast_to(band_hi, (nroi,)), np.int32)
    u = _c(dirs, np.float32)
    t = None if types is None else _c(types, np.uint8)
    nv = u.shape[0]
    S = np.empty((nroi, nv), np.float64)
    ak = np.empty((nroi, nv), np.int32)
    nw = np.empty(nroi, np.int64)
    lib().orc_signatures(_ptr(xyz), xyz.shape[0], _ptr(t), type_mask, _ptr(cen), _ptr(rad), nroi,
                         _ptr(blo), _ptr(bhi), _ptr(u), nv, m, _ptr(S), _ptr(ak), _ptr(nw), threads)
    return S, ak, nw


def normalise(S):
    S = np.array(S, dtype=np.float64, copy=True, order="C")
    S2 = S.reshape(-1, S.shape[-1])
    lib().orc_normalise(_ptr(S2), S2.shape[0], S2.shape[1])
    return S


def band_for_spacing(d_min, d_max, R, m):
    lo, hi = np.zeros(1, np.int32), np.zeros(1, np.int32)
    lib().orc_band_for_spacing(float(d_min), float(d_max), float(R), m, _ptr(lo), _ptr(hi))
    return int(lo[0]), int(hi[0])


# ---------------------------------------------------------------- rotations

def quat_to_matrix(q):
    M = np.empty(9, np.float64)
    lib().orc_quat_to_matrix(_ptr(_c(q, np.float64)), _ptr(M))
    return M.reshape(3, 3)


def disorientation_deg(q1, q2) -> float:
    return float(lib().orc_disorientation_deg(_ptr(_c(q1, np.float64)), _ptr(_c(q2, np.float64))))


# ---------------------------------------------------------------- indexing (Eq. 3)

def top_nodes(sig, n_hat):
    s = _c(sig, np.float32)
    out = np.empty(n_hat, np.int32)
    lib().orc_top_nodes(_ptr(s), s.shape[0], n_hat, _ptr(out))
    return out


def rotate_node(q, n):
    r = np.empty(3, np.float32)
    lib().orc_rotate_node(_ptr(_c(q, np.float64)), _ptr(_c(n, np.float32)), _ptr(r))
    return r


def nearest_node(dirs, r) -> int:
    u = _c(dirs, np.float32)
    return int(lib().orc_nearest_node(_ptr(u), u.shape[0], _ptr(_c(r, np.float32))))


def lut(dirs, top, quats, threads=0):
    u = _c(dirs, np.float32)
    top = _c(top, np.int32)
    q = _c(quats, np.float64).reshape(-1, 4)
    out = np.empty((q.shape[0], top.shape[0]), np.int32)
    lib().orc_lut(_ptr(u), u.shape[0], _ptr(top), top.shape[0], _ptr(q), q.shape[0], _ptr(out), threads)
    return out


def fsp(xc, L, kmax=2 * np.pi, points=None):
    """|F(k)| of Eq. 2 for centred positions xc on the L^3 grid over
    [-kmax, kmax]^3 (nm^-1), FP64 direct sum.  points: flat indices
    (ix * L + iy) * L + iz (default: all L^3).  Returns float64 [npts]."""
    xc = _c(xc, np.float32).reshape(-1, 3)
    pts = np.arange(L ** 3, dtype=np.int64) if points is None else _c(points, np.int64)
    out = np.empty(pts.shape[0], np.float64)
    lib().orc_fsp(_ptr(xc), xc.shape[0], int(L), float(kmax), _ptr(pts), pts.shape[0], _ptr(out))
    return out


def refine_roi_grid(S, centres, kappa, spacing, split=5):
    """Local refinement of a cubic ROI grid (Section 3.4, aluminium
    bicrystal): ROIs whose largest signature value reaches kappa times the
    largest value over all ROIs qualify; the cubic cell of edge `spacing`
    centred on each is split into split^3 cells and a new ROI goes to every
    cell centre, centre + (i - (split - 1) / 2) * spacing / split per axis.
    New ROIs in order of the qualifying ROI, then cell j = ix + split * (iy +
    split * iz).  Returns (centres float64 [n, 3], parent int32 [n])."""
    S = np.asarray(S, np.float64)
    centres = np.asarray(centres, np.float64).reshape(-1, 3)
    peak = S.max(axis=1)
    g = peak.max() if peak.size else 0.0
    sel = np.nonzero(peak >= np.float32(kappa) * np.float32(g))[0] if g > 0 else np.zeros(0, np.int64)
    h = spacing / split
    i = np.arange(split, dtype=np.float64)
    iz, iy, ix = np.meshgrid(i, i, i, indexing="ij")
    offs = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)
    offs = (offs - (split - 1) * 0.5) * h
    out = (centres[sel][:, None, :] + offs[None, :, :]).reshape(-1, 3)
    return np.ascontiguousarray(out), np.repeat(sel.astype(np.int32), split ** 3)


def match_topk(S_msr, S_ref, top, lut_, k, threads=0):
    """The k best test orientations per ROI under Eq. 3 (supplement "Indexing
    algorithm": the paper keeps up to 1000 solutions per ROI): Delta(g) of
    every g in FP64 (orc_match), then a stable sort by (Delta, g).
    Returns (g int32 [nroi, k], Delta float64 [nroi, k])."""
    _, _, sc = match(S_msr, S_ref, top, lut_, return_scores=True, threads=threads)
    order = np.argsort(sc, axis=1, kind="stable")[:, :k]
    return order.astype(np.int32), np.take_along_axis(sc, order, axis=1)


def match(S_msr, S_ref, top, lut_, return_scores=False, threads=0):
    S = _c(S_msr, np.float32)
    S = S.reshape(-1, S.shape[-1])
    ref = _c(S_ref, np.float32)
    top = _c(top, np.int32)
    L = _c(lut_, np.int32)
    nroi, nv = S.shape
    ng = L.shape[0]
    best = np.empty(nroi, np.int32)
    bs = np.empty(nroi, np.float64)
    sc = np.empty((nroi, ng), np.float64) if return_scores else None
    lib().orc_match(_ptr(S), nroi, nv, _ptr(ref), _ptr(top), top.shape[0], _ptr(L), ng, _ptr(best),
                    _ptr(bs), _ptr(sc), threads)
    return (best, bs, sc) if return_scores else (best, bs)


def match_phase(S, off, sig, refs, tops, luts, threads=0):
    """Phase and orientation from several signatures per candidate (Eq. 3
    of each channel relative to its reference's energy E_j = sum of its
    squared strongest values, averaged over a candidate's channels, FP64).  S: float32 [n_sig, nroi,
    nv] measured signatures; candidate c owns channels off[c] .. off[c+1]-1;
    channel j compares S[sig[j]] with reference refs[j] (float32 [nv]) at its
    strongest nodes tops[j] (int32 [n_hat], one n_hat for all) through its
    look-up table luts[j] (int32 [ng, n_hat], one orientation set).
    Returns (phase int32 [nroi], best int32 [n_cand, nroi], score float64
    [n_cand, nroi])."""
    S = _c(S, np.float32)
    n_sig, nroi, nv = S.shape
    off = _c(off, np.int32)
    sig = _c(sig, np.int32)
    n_cand = off.shape[0] - 1
    refs = _c(np.stack(refs), np.float32)
    tops = _c(np.stack(tops), np.int32)
    luts = _c(np.stack(luts), np.int32)
    n_hat = tops.shape[1]
    ng = luts.shape[1]
    phase = np.empty(nroi, np.int32)
    best = np.empty((n_cand, nroi), np.int32)
    score = np.empty((n_cand, nroi), np.float64)
    lib().orc_match_phase(_ptr(S), nroi, nv, n_cand, _ptr(off), _ptr(sig), _ptr(refs), _ptr(tops), n_hat,
                          _ptr(luts), ng, _ptr(phase), _ptr(best), _ptr(score), threads)
    return phase, best, score


# ---------------------------------------------------------------- refinement

def bilinear(img, c):
    img = _c(img, np.float32)
    val = np.zeros(1)
    grad = np.zeros(3)
    cell = np.zeros(2, np.int32)
    ok = lib().orc_bilinear(_ptr(img), _ptr(_c(c, np.float64)), _ptr(val), _ptr(grad), _ptr(cell))
    return bool(ok), float(val[0]), grad, cell


def refine_eval(img, S_msr, dirs, q, weights=None):
    """(loss, grad wrt left perturbation, J^T J, J^T r) at orientation q."""
    img = _c(img, np.float32)
    S = _c(S_msr, np.float32)
    u = _c(dirs, np.float32)
    w = None if weights is None else _c(weights, np.float64)
    loss = np.zeros(1)
    g = np.zeros(3)
    H = np.zeros(9)
    b = np.zeros(3)
    lib().orc_refine_eval(_ptr(img), _ptr(S), _ptr(u), u.shape[0], _ptr(_c(q, np.float64)), _ptr(w),
                          _ptr(loss), _ptr(g), _ptr(H), _ptr(b))
    return float(loss[0]), g, H.reshape(3, 3), b


def refine(img, S_msr, dirs, q0, iters=20, threads=0):
    """Gauss-Newton refinement of one or more ROIs; returns (q [.., 4], loss [..])."""
    img = _c(img, np.float32)
    u = _c(dirs, np.float32)
    nv = u.shape[0]
    S = _c(S_msr, np.float32).reshape(-1, nv)
    q0 = _c(q0, np.float64).reshape(-1, 4)
    nroi = S.shape[0]
    q = np.empty((nroi, 4))
    loss = np.empty(nroi)
    lib().orc_refine_batch(_ptr(img), _ptr(S), _ptr(u), nv, nroi, _ptr(q0), iters, _ptr(q), _ptr(loss),
                           threads)
    return q, loss
