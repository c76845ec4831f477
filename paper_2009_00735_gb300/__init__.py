"""GB300-native RSP signatures and orientation indexing for atom probe data
(Kuehbach et al., arXiv 2009.00735) -- Python binding of libaptidx.

Thin ctypes marshalling over the C ABI declared in include/aptidx.h: every
function keeps its C name, accepts torch tensors (CUDA -> device pointer,
CPU -> host pointer) or numpy arrays (host), and raises AptidxError on a
non-zero status.  All computation runs in the library's CUDA kernels; there is
no CPU fallback.  Build the library first with
``paper_2009_00735_gb300.build.build()``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build_mod

__all__ = [
    "AptidxError", "load", "Context",
    "aptidx_version", "aptidx_create", "aptidx_destroy", "aptidx_last_error", "aptidx_sync",
    "aptidx_load_positions", "aptidx_set_directions", "aptidx_set_binning", "aptidx_set_rois",
    "aptidx_compute_signatures", "aptidx_get_histograms", "aptidx_get_roi_atoms",
    "aptidx_set_reference", "aptidx_build_lut", "aptidx_get_lut", "aptidx_match", "aptidx_match_topk", "aptidx_match_phase", "aptidx_compute_signatures_multi", "aptidx_refine_roi_grid", "aptidx_compute_fsp", "aptidx_refine_loss", "aptidx_refine",
    "band_for_spacing", "aptidx_band_for_spacing", "aptidx_path_supported", "aptidx_set_profiling", "aptidx_get_profile", "aptidx_probe_l2", "aptidx_probe_smem_atomics",
    "tc_available", "PHASES", "aptidx_signatures_noalloc",
    "APTIDX_MEM_HOST", "APTIDX_MEM_DEVICE", "APTIDX_PATH_PLAIN_FP32", "APTIDX_PATH_TC_FP16",
    "APTIDX_NORMALISE_MAX", "APTIDX_AUTOTUNE", "APTIDX_GRAPH", "APTIDX_DIRECT", "aptidx_get_tuning",
]

APTIDX_OK = 0
APTIDX_MAX_TOPK = 1024
APTIDX_MAX_BANDS = 4
APTIDX_FSP_L_MIN = 64
APTIDX_FSP_L_MAX = 512
APTIDX_E_INVALID_ARG = 1
APTIDX_E_CUDA = 2
APTIDX_E_OOM = 3
APTIDX_E_TIMEOUT = 4
APTIDX_E_OVERFLOW = 5
APTIDX_E_STATE = 6
APTIDX_MEM_HOST = 0
APTIDX_MEM_DEVICE = 1
APTIDX_PATH_PLAIN_FP32 = 0
APTIDX_PATH_TC_FP16 = 1
APTIDX_NORMALISE_MAX = 1
APTIDX_AUTOTUNE = 2
APTIDX_GRAPH = 4
APTIDX_DIRECT = 8

_ERR_NAMES = {1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "TIMEOUT", 5: "OVERFLOW", 6: "STATE"}


class AptidxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"aptidx error {code} ({_ERR_NAMES.get(code, '?')}): {msg}")
        self.code = code


_lib = None
_vp = C.c_void_p
_i64 = C.c_int64
_i32 = C.c_int32
_SIGS = {
    "aptidx_version": (C.c_int, []),
    "aptidx_band_for_spacing": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_int, _vp, _vp]),
    "aptidx_create": (C.c_int, [C.POINTER(_vp), C.c_int, _vp]),
    "aptidx_destroy": (C.c_int, [_vp]),
    "aptidx_last_error": (C.c_char_p, [_vp]),
    "aptidx_sync": (C.c_int, [_vp]),
    "aptidx_load_positions": (C.c_int, [_vp, _vp, _i64, _vp, C.c_int]),
    "aptidx_set_directions": (C.c_int, [_vp, _vp, _i32, C.c_int]),
    "aptidx_set_binning": (C.c_int, [_vp, C.c_int, _i32, _i32, C.c_int]),
    "aptidx_set_rois": (C.c_int, [_vp, _vp, _vp, _i64, _vp, _vp, C.c_uint32, C.c_int]),
    "aptidx_compute_signatures": (C.c_int, [_vp, C.c_int, C.c_uint, _vp, _vp, _vp, C.c_int]),
    "aptidx_get_histograms": (C.c_int, [_vp, _i64, C.c_int, _vp, C.c_int]),
    "aptidx_get_roi_atoms": (C.c_int, [_vp, _i64, _vp, _i64, C.POINTER(_i64), C.c_int]),
    "aptidx_set_reference": (C.c_int, [_vp, _i32, _vp, _i32, _vp, C.c_int]),
    "aptidx_build_lut": (C.c_int, [_vp, _i32, _vp, _i64, C.c_int]),
    "aptidx_get_lut": (C.c_int, [_vp, _i32, _vp, _vp, C.c_int]),
    "aptidx_match": (C.c_int, [_vp, _i32, _vp, _i64, _vp, _vp, C.c_int]),
    "aptidx_match_topk": (C.c_int, [_vp, _i32, _vp, _i64, _i32, _vp, _vp, C.c_int]),
    "aptidx_compute_fsp": (C.c_int, [_vp, C.c_int32, C.c_double, _vp, C.c_int]),
    "aptidx_match_phase": (C.c_int, [_vp, _i32, _vp, _vp, _vp, _i32, _vp, _i64, _vp, _vp, _vp, C.c_int]),
    "aptidx_refine_roi_grid": (C.c_int, [_vp, _vp, _i64, C.c_float, C.c_double, _i32, _vp, _vp, _i64, _vp,
                                         C.c_int]),
    "aptidx_compute_signatures_multi": (C.c_int, [_vp, C.c_int, C.c_uint, _i32, _vp, _vp, _vp, _vp, _vp, _vp,
                                                  C.c_int]),
    "aptidx_refine_loss": (C.c_int, [_vp, _i32, _vp, _vp, _vp, _i64, _vp, _vp, C.c_int]),
    "aptidx_refine": (C.c_int, [_vp, _i32, _vp, _vp, _vp, _i64, _i32, _vp, _vp, C.c_int]),
    "aptidx_path_supported": (C.c_int, [_vp, C.c_int]),
    "aptidx_get_tuning": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "aptidx_set_profiling": (C.c_int, [_vp, C.c_int]),
    "aptidx_get_profile": (C.c_int, [_vp, _vp, _vp, _vp]),
    "aptidx_probe_l2": (C.c_int, [_vp, C.c_int64, C.c_int32, _vp]),
    "aptidx_probe_smem_atomics": (C.c_int, [_vp, C.c_int32, C.c_int32, _vp, _vp]),
    "aptidx_signatures_noalloc": (C.c_int, [_vp, _vp, _vp, _i64, _vp, _i32, C.c_int, _i32, _i32, _vp, _vp, _vp]),
}

APTIDX_N_PHASES = 6
PHASES = ("gather", "order", "signature", "normalise", "match", "refine")


def library_path() -> str:
    return _build_mod.LIB


def load():
    """Load libaptidx.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libaptidx.so is not built ({path}); run paper_2009_00735_gb300.build.build()")
        lib = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            if hasattr(lib, name):
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    lib = load()
    return [n for n in _SIGS if hasattr(lib, n)]


# ---------------------------------------------------------------------------
# marshalling
# ---------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _is_torch(x):
    try:
        import torch
        return isinstance(x, torch.Tensor)
    except ImportError:
        return False


def _arg(x, dtype):
    """(pointer, mem, keep-alive object) of an input array."""
    if x is None:
        return None, None, None
    if _is_torch(x):
        torch = _torch()
        tdt = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32,
               np.uint8: torch.uint8, np.uint16: torch.uint16, np.int64: torch.int64}[dtype]
        if x.dtype != tdt:
            raise TypeError(f"expected {tdt}, got {x.dtype}")
        x = x.contiguous()
        return x.data_ptr(), (APTIDX_MEM_DEVICE if x.is_cuda else APTIDX_MEM_HOST), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, APTIDX_MEM_HOST, a


def _out(x, dtype):
    """(pointer, mem) of an output array; must already be contiguous."""
    if x is None:
        return None, None
    if _is_torch(x):
        torch = _torch()
        if not x.is_contiguous():
            raise ValueError("output tensors must be contiguous")
        return x.data_ptr(), (APTIDX_MEM_DEVICE if x.is_cuda else APTIDX_MEM_HOST)
    if not (isinstance(x, np.ndarray) and x.flags.c_contiguous and x.dtype == dtype):
        raise ValueError(f"output arrays must be C-contiguous {np.dtype(dtype)}")
    return x.ctypes.data, APTIDX_MEM_HOST


def _one_mem(*mems):
    ms = {m for m in mems if m is not None}
    if len(ms) > 1:
        raise ValueError("all arrays of one call must live in the same memory space")
    return ms.pop() if ms else APTIDX_MEM_HOST


def _check(ctx, rc):
    if rc != APTIDX_OK:
        msg = load().aptidx_last_error(ctx).decode() if ctx else ""
        raise AptidxError(rc, msg)


# ---------------------------------------------------------------------------
# the C ABI, one Python function per C function
# ---------------------------------------------------------------------------

def aptidx_version() -> int:
    """Library version, major * 10000 + minor * 100 + patch."""
    return load().aptidx_version()


def aptidx_create(device: int = 0, stream=None):
    """Context on `device`; `stream` is a torch.cuda.Stream, a raw cudaStream_t
    (int) or None for torch's current stream on that device."""
    lib = load()
    if stream is None:
        torch = _torch()
        stream = torch.cuda.current_stream(device).cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    h = _vp()
    rc = lib.aptidx_create(C.byref(h), int(device), _vp(int(stream)) if stream else None)
    if rc != APTIDX_OK:
        raise AptidxError(rc, "aptidx_create failed")
    return h


def aptidx_destroy(ctx):
    """Synchronise and free the context and every buffer it owns."""
    _check(None, load().aptidx_destroy(ctx))


def aptidx_last_error(ctx) -> str:
    """Message of the context's last failing call ("" if none)."""
    return load().aptidx_last_error(ctx).decode()


def aptidx_sync(ctx):
    """Synchronise the context's stream; raises on a device status (TIMEOUT, OVERFLOW)."""
    _check(ctx, load().aptidx_sync(ctx))


def aptidx_load_positions(ctx, xyz, types=None):
    """Atom positions p_i: xyz [n, 3] float32 (nm), types [n] uint8 or None;
    host (numpy) or device (torch) arrays, copied by the library."""
    p, m, k1 = _arg(xyz, np.float32)
    t, mt, k2 = _arg(types, np.uint8)
    n = (k1.numel() if _is_torch(k1) else k1.size) // 3
    _check(ctx, load().aptidx_load_positions(ctx, p, n, t, _one_mem(m, mt)))


def aptidx_set_directions(ctx, u):
    """Projection directions: u [nv, 3] float32 unit vectors."""
    p, m, k = _arg(u, np.float32)
    nv = (k.numel() if _is_torch(k) else k.size) // 3
    _check(ctx, load().aptidx_set_directions(ctx, p, nv, m))


def aptidx_set_binning(ctx, m: int, k_lo: int, k_hi: int, flags: int = 0):
    """2^m histogram bins (Eq. 1) and the default band [k_lo, k_hi] of
    frequency bins whose amplitude maximum is the signature."""
    _check(ctx, load().aptidx_set_binning(ctx, m, k_lo, k_hi, flags))


def aptidx_set_rois(ctx, centres, radii, band_lo=None, band_hi=None, type_mask=0xFFFFFFFF):
    """ROIs: centres [nroi, 3] float64 (nm), radii [nroi] float64, optional
    per-ROI bands (int32 arrays or scalars), atom-type bit mask."""
    pc, mc, kc = _arg(centres, np.float64)
    pr, mr, kr = _arg(radii, np.float64)
    nroi = (kr.numel() if _is_torch(kr) else kr.size)
    if band_lo is not None and not _is_torch(band_lo):
        band_lo = np.broadcast_to(np.asarray(band_lo, np.int32), (nroi,))
        band_hi = np.broadcast_to(np.asarray(band_hi, np.int32), (nroi,))
    pl, ml, kl = _arg(band_lo, np.int32)
    ph, mh, kh = _arg(band_hi, np.int32)
    _check(ctx, load().aptidx_set_rois(ctx, pc, pr, nroi, pl, ph, C.c_uint32(type_mask & 0xFFFFFFFF),
                                       _one_mem(mc, mr, ml, mh)))


def aptidx_compute_signatures(ctx, path: int, flags: int, S=None, argk=None, n_atoms=None):
    """Signatures of every ROI on `path` (APTIDX_PATH_PLAIN_FP32 or
    APTIDX_PATH_TC_FP16): S [nroi, nv] float32, argk [nroi, nv] uint16 and
    n_atoms [nroi] int32 (each optional, host or device); flags:
    APTIDX_NORMALISE_MAX | APTIDX_AUTOTUNE | APTIDX_GRAPH | APTIDX_DIRECT."""
    pS, mS = _out(S, np.float32)
    pA, mA = _out(argk, np.uint16)
    pN, mN = _out(n_atoms, np.int32)
    _check(ctx, load().aptidx_compute_signatures(ctx, path, flags, pS, pA, pN, _one_mem(mS, mA, mN)))


def aptidx_compute_signatures_multi(ctx, path: int, flags: int, type_masks, k_lo, k_hi, S, argk=None, n_atoms=None):
    """Several signatures per ROI: S[s, roi, v] for signature s with atom
    types type_masks[s] and band [k_lo[s], k_hi[s]] (host sequences)."""
    tm = np.ascontiguousarray(np.asarray(type_masks, dtype=np.uint32))
    lo = np.ascontiguousarray(np.asarray(k_lo, dtype=np.int32))
    hi = np.ascontiguousarray(np.asarray(k_hi, dtype=np.int32))
    n_sig = tm.size
    if lo.size != n_sig or hi.size != n_sig:
        raise ValueError("type_masks, k_lo and k_hi need the same length")
    pS, mS = _out(S, np.float32)
    pA, mA = _out(argk, np.uint16)
    pN, mN = _out(n_atoms, np.int32)
    _check(ctx, load().aptidx_compute_signatures_multi(ctx, path, flags, n_sig, tm.ctypes.data_as(_vp),
                                                       lo.ctypes.data_as(_vp), hi.ctypes.data_as(_vp), pS, pA, pN,
                                                       _one_mem(mS, mA, mN)))


def aptidx_refine_roi_grid(ctx, S, kappa: float, spacing: float, split: int = 5):
    """New ROI centres (float64 [n, 3]) and their coarse parents (int32 [n])
    of the local grid refinement; S holds the current ROIs' signatures."""
    pS, mS, kS = _arg(S, np.float32)
    nroi = int(kS.shape[0])
    n = _i64(0)
    _check(ctx, load().aptidx_refine_roi_grid(ctx, pS, nroi, C.c_float(kappa), C.c_double(spacing), int(split), None,
                                              None, 0, C.byref(n), mS))
    cen = np.empty((n.value, 3), np.float64)
    par = np.empty(n.value, np.int32)
    if n.value:
        if mS == APTIDX_MEM_DEVICE:
            import torch
            cd = torch.empty((n.value, 3), dtype=torch.float64, device=kS.device)
            pd = torch.empty(n.value, dtype=torch.int32, device=kS.device)
            _check(ctx, load().aptidx_refine_roi_grid(ctx, pS, nroi, C.c_float(kappa), C.c_double(spacing), int(split),
                                                      C.c_void_p(cd.data_ptr()), C.c_void_p(pd.data_ptr()), n.value,
                                                      C.byref(_i64(0)), mS))
            return cd.cpu().numpy(), pd.cpu().numpy()
        _check(ctx, load().aptidx_refine_roi_grid(ctx, pS, nroi, C.c_float(kappa), C.c_double(spacing), int(split),
                                                  cen.ctypes.data_as(_vp), par.ctypes.data_as(_vp), n.value,
                                                  C.byref(_i64(0)), mS))
    return cen, par


def aptidx_compute_fsp(ctx, amp, k_max: float = 2 * 3.141592653589793):
    """|F(k)| of Eq. 2 on the L^3 grid over [-k_max, k_max]^3 (nm^-1) for
    every ROI: amp [nroi, L, L, L] float32 (ix, iy, iz); L (a multiple of 64
    up to 512) is taken from amp's shape."""
    L = int(amp.shape[1])
    pA, mA = _out(amp, np.float32)
    _check(ctx, load().aptidx_compute_fsp(ctx, C.c_int32(L), C.c_double(k_max), pA, mA))


def aptidx_get_histograms(ctx, roi: int, path: int, h):
    """Debug/parity: the 2^m-bin histograms of ROI `roi` as `path`'s
    histogram stage computes them, h [nv, 2^m] uint16."""
    p, m = _out(h, np.uint16)
    _check(ctx, load().aptidx_get_histograms(ctx, roi, path, p, m))


def aptidx_get_roi_atoms(ctx, roi: int, xc=None, cap: int = 0):
    """Debug/parity: the centred FP32 atoms of ROI `roi` as the gather
    produced them, [n_w, 3] (allocated when xc is None)."""
    n = _i64(0)
    if xc is None:
        rc = load().aptidx_get_roi_atoms(ctx, roi, None, 0, C.byref(n), APTIDX_MEM_HOST)
        if rc not in (APTIDX_OK, APTIDX_E_OVERFLOW):
            _check(ctx, rc)
        xc = np.empty((n.value, 3), np.float32)
        cap = n.value
    p, m = _out(xc, np.float32)
    _check(ctx, load().aptidx_get_roi_atoms(ctx, roi, p, cap, C.byref(n), m))
    return xc[: n.value]


def aptidx_set_reference(ctx, cand: int, node_sig, n_hat: int, img=None):
    """Reference of candidate `cand`: its normalised signature on the
    directions (node_sig [nv] float32, the n_hat strongest nodes enter Eq. 3)
    and optionally its [181, 360] elevation-azimuth image for refinement."""
    p, m, k = _arg(node_sig, np.float32)
    pi, mi, ki = _arg(img, np.float32)
    _check(ctx, load().aptidx_set_reference(ctx, cand, p, n_hat, pi, _one_mem(m, mi)))


def aptidx_build_lut(ctx, cand: int, quats):
    """Look-up table of candidate `cand` for test orientations quats
    [ng, 4] float64 (w, x, y, z; crystal to lab)."""
    p, m, k = _arg(quats, np.float64)
    ng = (k.numel() if _is_torch(k) else k.size) // 4
    _check(ctx, load().aptidx_build_lut(ctx, cand, p, ng, m))


def aptidx_get_lut(ctx, cand: int, ng: int = None):
    """The candidate's look-up table as int32 [ng, n_hat] (host)."""
    nh = np.zeros(1, np.int32)
    _check(ctx, load().aptidx_get_lut(ctx, cand, None, nh.ctypes.data, APTIDX_MEM_HOST))
    if ng is None:
        raise ValueError("pass ng (the number of test orientations of the table)")
    out = np.empty((ng, int(nh[0])), np.int32)
    _check(ctx, load().aptidx_get_lut(ctx, cand, out.ctypes.data, None, APTIDX_MEM_HOST))
    return out


def aptidx_match(ctx, cand: int, S, best, score=None):
    """Eq. 3 for every ROI: best [nroi] int32 = argmin_g Delta(g) (ties:
    lowest g), score [nroi] float32 = Delta(best); S [nroi, nv] normalised."""
    pS, mS, kS = _arg(S, np.float32)
    pb, mb = _out(best, np.int32)
    ps, ms = _out(score, np.float32)
    nroi = best.shape[0]
    _check(ctx, load().aptidx_match(ctx, cand, pS, nroi, pb, ps, _one_mem(mS, mb, ms)))


def aptidx_match_topk(ctx, cand: int, S, topk: int, best, score=None):
    """best, score: [nroi, topk] outputs, ascending by (Delta, g)."""
    pS, mS, kS = _arg(S, np.float32)
    pb, mb = _out(best, np.int32)
    ps, ms = _out(score, np.float32)
    nroi = best.shape[0]
    _check(ctx, load().aptidx_match_topk(ctx, cand, pS, nroi, int(topk), pb, ps, _one_mem(mS, mb, ms)))


def aptidx_match_phase(ctx, cand_off, ref, sig, S, phase=None, best=None, score=None):
    """Phase and orientation from several signatures per candidate: candidate
    c owns channels cand_off[c] .. cand_off[c+1]-1 (host sequences), channel j
    compares S[sig[j]] (S [n_sig, nroi, nv] float32, normalised) with the
    reference of slot ref[j].  Outputs: phase [nroi] int32, best and score
    [n_cand, nroi] (int32, float32); any may be None."""
    off = np.ascontiguousarray(np.asarray(cand_off, dtype=np.int32))
    rf = np.ascontiguousarray(np.asarray(ref, dtype=np.int32))
    sg = np.ascontiguousarray(np.asarray(sig, dtype=np.int32))
    if rf.size != sg.size or off.size < 2 or off[-1] != rf.size:
        raise ValueError("cand_off[-1] must equal the number of channels in ref and sig")
    pS, mS, kS = _arg(S, np.float32)
    if len(kS.shape) != 3:
        raise ValueError("S must be [n_sig, nroi, nv]")
    n_sig, nroi = int(kS.shape[0]), int(kS.shape[1])
    pp, mp = _out(phase, np.int32)
    pb, mb = _out(best, np.int32)
    ps, ms = _out(score, np.float32)
    _check(ctx, load().aptidx_match_phase(ctx, off.size - 1, off.ctypes.data_as(_vp), rf.ctypes.data_as(_vp),
                                          sg.ctypes.data_as(_vp), n_sig, pS, nroi, pp, pb, ps,
                                          _one_mem(mS, mp, mb, ms)))


def aptidx_refine_loss(ctx, cand: int, S, q0, loss, grad=None, omega=None):
    """Refinement loss [nroi] and its gradient [nroi, 3] with respect to
    the axis-angle offset omega [nroi, 3] (None: zero) at q0 [nroi, 4]."""
    pS, mS, kS = _arg(S, np.float32)
    pq, mq, kq = _arg(q0, np.float64)
    pw, mw, kw = _arg(omega, np.float64)
    pl, ml = _out(loss, np.float32)
    pg, mg = _out(grad, np.float32)
    nroi = loss.shape[0]
    _check(ctx, load().aptidx_refine_loss(ctx, cand, pS, pq, pw, nroi, pl, pg, _one_mem(mS, mq, mw, ml, mg)))


def aptidx_refine(ctx, cand: int, S, q0, iters: int, q_out, loss=None, best=None):
    """Gauss-Newton from q0 [nroi, 4], or from the test orientations best
    [nroi] of the candidate's look-up table when `best` is given."""
    pS, mS, kS = _arg(S, np.float32)
    pq, mq, kq = _arg(q0, np.float64)
    pb, mb, kb = _arg(best, np.int32)
    po, mo = _out(q_out, np.float64)
    pl, ml = _out(loss, np.float32)
    nroi = q_out.shape[0]
    _check(ctx, load().aptidx_refine(ctx, cand, pS, pq, pb, nroi, iters, po, pl, _one_mem(mS, mq, mb, mo, ml)))


def aptidx_path_supported(ctx, path: int) -> bool:
    """True if `path` runs on the context's device."""
    return bool(load().aptidx_path_supported(ctx, path))


def aptidx_get_tuning(ctx, path: int):
    """(tiles per work item, MMA issuer warps) the next call on `path` uses."""
    t = np.zeros(1, np.int32)
    i = np.zeros(1, np.int32)
    _check(ctx, load().aptidx_get_tuning(ctx, path, t.ctypes.data, i.ctypes.data))
    return int(t[0]), int(i[0])


def aptidx_probe_l2(ctx, nbytes: int = 32 << 20, iters: int = 200) -> float:
    """Read bandwidth (GB/s) of the device's L2 cache over an nbytes buffer
    read iters times (the roof of the gather-bound kernels)."""
    g = np.zeros(1, np.float64)
    _check(ctx, load().aptidx_probe_l2(ctx, int(nbytes), int(iters), g.ctypes.data))
    return float(g[0])


def aptidx_probe_smem_atomics(ctx, threads: int = 512, iters: int = 4096):
    """Shared-memory atomic add throughput: (lane increments per second over
    the device, 32-lane atomic instructions per SM and SM cycle)."""
    g = np.zeros(2, np.float64)
    _check(ctx, load().aptidx_probe_smem_atomics(ctx, int(threads), int(iters), g.ctypes.data, g.ctypes.data + 8))
    return float(g[0]), float(g[1])


def aptidx_set_profiling(ctx, enable: bool):
    """Record per-phase CUDA-event times and kernel counts of the following
    calls (resets the totals), or stop recording."""
    _check(ctx, load().aptidx_set_profiling(ctx, 1 if enable else 0))


def aptidx_get_profile(ctx):
    """{phase: (total ms, calls)} and the library kernel-launch count."""
    ms = np.zeros(APTIDX_N_PHASES, np.float64)
    calls = np.zeros(APTIDX_N_PHASES, np.int64)
    n = np.zeros(1, np.int64)
    _check(ctx, load().aptidx_get_profile(ctx, ms.ctypes.data, calls.ctypes.data, n.ctypes.data))
    return {PHASES[i]: (float(ms[i]), int(calls[i])) for i in range(APTIDX_N_PHASES)}, int(n[0])


def aptidx_signatures_noalloc(xc4, off, radii, u, m: int, k_lo: int, k_hi: int, S, status=None, stream=None):
    """The no-allocation call: every array is a contiguous CUDA tensor the
    caller owns, all on one device -- xc4 float32 [N, 4], off int64
    [nroi + 1], radii float64 [nroi], u float32 [nv, 3], S float32
    [nroi, nv], status int32 [>= 1] or None.  Queued on `stream` (default:
    torch's current stream of S's device); returns without waiting."""
    torch = _torch()
    named = [("xc4", xc4, torch.float32), ("off", off, torch.int64), ("radii", radii, torch.float64),
             ("u", u, torch.float32), ("S", S, torch.float32)]
    if status is not None:
        named.append(("status", status, torch.int32))
    for name, t, dt in named:
        if not (_is_torch(t) and t.is_cuda and t.is_contiguous()):
            raise ValueError(f"aptidx_signatures_noalloc: {name} must be a contiguous CUDA tensor")
        if t.dtype != dt:
            raise TypeError(f"aptidx_signatures_noalloc: {name} must be {dt}, got {t.dtype}")
        if t.device != S.device:
            raise ValueError(f"aptidx_signatures_noalloc: {name} is on {t.device}, S on {S.device}")
    nroi = radii.numel()
    if xc4.dim() != 2 or xc4.shape[1] != 4:
        raise ValueError("aptidx_signatures_noalloc: xc4 must be [N, 4]")
    if off.numel() != nroi + 1:
        raise ValueError("aptidx_signatures_noalloc: off must hold nroi + 1 offsets")
    if u.dim() != 2 or u.shape[1] != 3:
        raise ValueError("aptidx_signatures_noalloc: u must be [nv, 3]")
    nv = u.shape[0]
    if S.numel() < nroi * nv:
        raise ValueError("aptidx_signatures_noalloc: S must hold nroi x nv values")
    if status is not None and status.numel() < 1:
        raise ValueError("aptidx_signatures_noalloc: status must hold one int32")
    with torch.cuda.device(S.device):
        if stream is None:
            stream = torch.cuda.current_stream(S.device).cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        rc = load().aptidx_signatures_noalloc(xc4.data_ptr(), off.data_ptr(), radii.data_ptr(), nroi, u.data_ptr(),
                                              nv, m, k_lo, k_hi, S.data_ptr(),
                                              status.data_ptr() if status is not None else None,
                                              _vp(int(stream)) if stream else None)
    if rc != APTIDX_OK:
        raise AptidxError(rc, "aptidx_signatures_noalloc: invalid sizes (limits in include/aptidx.h) or CUDA error")


def tc_available(device: int = 0) -> bool:
    ctx = Context(device)
    try:
        return aptidx_path_supported(ctx.handle, APTIDX_PATH_TC_FP16)
    finally:
        ctx.close()


def aptidx_band_for_spacing(d_min: float, d_max: float, R: float, m: int):
    """Frequency-bin band (k_lo, k_hi) holding plane spacings d_min..d_max
    (nm) for a ROI of radius R at 2^m bins (computed by the library)."""
    lo = np.zeros(1, np.int32)
    hi = np.zeros(1, np.int32)
    rc = load().aptidx_band_for_spacing(float(d_min), float(d_max), float(R), int(m), lo.ctypes.data, hi.ctypes.data)
    if rc != APTIDX_OK:
        raise AptidxError(rc, f"aptidx_band_for_spacing({d_min}, {d_max}, {R}, {m}): invalid arguments or band")
    return int(lo[0]), int(hi[0])


band_for_spacing = aptidx_band_for_spacing


class Context:
    """Owning wrapper of an aptidx context (destroyed on close/garbage collection)."""

    def __init__(self, device: int = 0, stream=None):
        self.handle = aptidx_create(device, stream)
        self.device = device

    def close(self):
        if self.handle is not None:
            aptidx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
