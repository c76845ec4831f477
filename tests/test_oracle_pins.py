"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: exact
rational arithmetic, closed forms, numpy's FFT, the paper's worked example
(Fig. 2 caption), crystal symmetry, and brute force on tiny inputs.  A
plausible slip in the oracle (a dropped term, a wrong sign, a transposed
operand, an off-by-one bin) fails at least one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# exact rational helpers (independent of the C code)
# --------------------------------------------------------------------------

def rn32(fr: Fraction) -> Fraction:
    """Round a rational to the nearest float32 (ties to even), exactly."""
    if fr == 0:
        return Fraction(0)
    sign = -1 if fr < 0 else 1
    a = abs(fr)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    if Fraction(2) ** (e + 1) <= a:
        e += 1
    e = max(e, -126)                      # subnormal spacing below 2^-126
    ulp = Fraction(2) ** (e - 23)
    q, r = divmod(a, ulp)
    q = int(q)
    if r * 2 > ulp or (r * 2 == ulp and q % 2 == 1):
        q += 1
    return sign * q * ulp


def contract_bin_exact(u, x, m, R):
    """The documented FP32 binning contract, evaluated in exact arithmetic."""
    U = [Fraction(float(c)) for c in np.asarray(u, np.float32)]
    X = [Fraction(float(c)) for c in np.asarray(x, np.float32)]
    p = rn32(U[0] * X[0])
    a = rn32(U[1] * X[1] + p)
    s = rn32(U[2] * X[2] + a)
    scale = Fraction(float(np.float32(float(Fraction((1 << (m - 1)) - 1) / Fraction(R)))))
    b = (1 << (m - 1)) + math.floor(s * scale)
    return min(max(b, 0), (1 << m) - 1)


def eq1_bin_exact(u, x, m, R):
    """Eq. 1 in exact rational arithmetic (inputs taken as the given floats)."""
    U = [Fraction(float(c)) for c in u]
    X = [Fraction(float(c)) for c in x]
    Rf = Fraction(R)
    dR = Rf / ((1 << (m - 1)) - 1)
    s = U[0] * X[0] + U[1] * X[1] + U[2] * X[2]
    t = (s + Rf + dR) * (1 << m) / (dR + 2 * Rf + dR)
    b = math.floor(t)
    return min(max(b, 0), (1 << m) - 1)


# --------------------------------------------------------------------------
# Eq. 1 binning
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m", [8, 10, 12])
def test_bin_closed_forms(m):
    """With R = 2^(m-1) - 1 the bin width is exactly 1 (dR = 1): an atom at
    s = j lands in bin 2^(m-1) + j, just below j in the bin before, and the
    centre in bin 2^(m-1); s = +R lands in the last bin, s = -R in bin 1."""
    R = float((1 << (m - 1)) - 1)
    u = np.array([1, 0, 0], np.float32)
    c = 1 << (m - 1)
    for j in [-5, -1, 0, 1, 7, 100 % (c - 1)]:
        x = np.array([j, 0, 0], np.float32)
        assert oracle.bin_contract(u, x, m, R) == c + j
        assert oracle.bin_eq1(u.astype(float), x.astype(float), m, R) == c + j
        xm = np.array([np.nextafter(np.float32(j), np.float32(-1e9))], np.float32)
        assert oracle.bin_contract(u, np.array([xm[0], 0, 0], np.float32), m, R) == c + j - 1
        xh = np.array([j + 0.5, 0, 0], np.float32)
        assert oracle.bin_contract(u, xh, m, R) == c + j
    assert oracle.bin_contract(u, np.array([R, 0, 0], np.float32), m, R) == (1 << m) - 1
    assert oracle.bin_contract(u, np.array([-R, 0, 0], np.float32), m, R) == 1
    assert oracle.bin_contract(u, np.zeros(3, np.float32), m, R) == c


def test_bin_contract_brute_force_rational():
    """10-atom ROIs: the oracle's FP32 contract equals the same contract
    evaluated in exact rational arithmetic with explicit float32 rounding."""
    rng = np.random.default_rng(7)
    for trial in range(6):
        m = [8, 10, 12][trial % 3]
        R = [1.0, 2.0, 2.37][trial % 3]
        x = (rng.random((10, 3)) * 2 - 1).astype(np.float32) * np.float32(R / math.sqrt(3))
        u = rng.standard_normal((5, 3))
        u = (u / np.linalg.norm(u, axis=1, keepdims=True)).astype(np.float32)
        h = oracle.histograms(x, u, m, R)
        for v in range(5):
            ref = np.zeros(1 << m, np.int64)
            for i in range(10):
                b = contract_bin_exact(u[v], x[i], m, R)
                assert oracle.bin_contract(u[v], x[i], m, R) == b
                ref[b] += 1
            assert np.array_equal(h[v], ref)
            assert h[v].sum() == 10


def bin_edge_positions(m, R, n=40, seed=0):
    """float32 coordinates on and one ulp either side of bin edges: for
    integers j across the histogram, x0 = the float32 nearest to j / scale
    (s * scale = j is a bin edge of the contract when s = x0), then its two
    float32 neighbours.  |x| <= R except possibly one ulp past it."""
    scale = Fraction(float(np.float32(float(Fraction((1 << (m - 1)) - 1) / Fraction(R)))))
    half = (1 << (m - 1)) - 1
    rng = np.random.default_rng(seed)
    js = np.concatenate([[0, 1, -1, half - 1, -(half - 1)], rng.integers(-half + 1, half, n)])
    xs = []
    for j in js:
        x0 = np.float32(float(Fraction(int(j)) / scale))
        xs += [np.nextafter(x0, np.float32(-np.inf)), x0, np.nextafter(x0, np.float32(np.inf))]
    return np.array(xs, np.float32)


@pytest.mark.parametrize("m, R", [(8, 1.0), (10, 2.0), (10, 2.37), (11, 2.0), (12, 3.1)])
def test_bin_contract_at_bin_edges(m, R):
    """Atoms on and one ulp around bin edges (projection along a coordinate
    axis, so s is the coordinate itself): the oracle's contract equals the
    exact-rational contract, and the bins of x0 - ulp, x0, x0 + ulp never
    decrease and step by at most one."""
    xs = bin_edge_positions(m, R)
    rng = np.random.default_rng(1)
    for axis in range(3):
        u = np.zeros(3, np.float32)
        u[axis] = 1.0
        for t in range(0, xs.shape[0], 3):
            bins = []
            for d in range(3):
                x = (rng.random(3).astype(np.float32) - np.float32(0.5)) * np.float32(0.1)
                x[axis] = xs[t + d]
                b = oracle.bin_contract(u, x, m, R)
                assert b == contract_bin_exact(u, x, m, R)
                bins.append(b)
            # every triple straddles exactly one edge
            assert bins[0] <= bins[1] <= bins[2] and bins[2] - bins[0] == 1


def test_bin_eq1_matches_exact_eq1_and_contract_moves_only_boundary_atoms():
    """The FP64 Eq. 1 oracle equals exact-rational Eq. 1, and the FP32
    contract differs from Eq. 1 only for atoms within a few float ulps of a
    bin edge, which move to the adjacent bin."""
    rng = np.random.default_rng(11)
    m, R = 10, 2.0
    x = ((rng.random((400, 3)) * 2 - 1) * 1.15).astype(np.float32)
    u = rng.standard_normal((40, 3))
    u = (u / np.linalg.norm(u, axis=1, keepdims=True)).astype(np.float32)
    moved = 0
    for v in range(40):
        for i in range(400):
            be = eq1_bin_exact(u[v].astype(float), x[i].astype(float), m, R)
            assert oracle.bin_eq1(u[v].astype(float), x[i].astype(float), m, R) == be
            bc = oracle.bin_contract(u[v], x[i], m, R)
            if bc != be:
                moved += 1
                assert abs(bc - be) == 1
                # boundary atom: exact t within 1e-5 bins of an integer
                s = float(np.dot(u[v].astype(float), x[i].astype(float)))
                t = (1 << (m - 1)) + s * ((1 << (m - 1)) - 1) / R
                assert abs(t - round(t)) < 1e-4
    assert moved <= 3


def test_histogram_counts_sum_and_mirror():
    """Sum over bins is N_w for every direction; reversing the direction
    mirrors the histogram: h_{-u}[n] = h_u[N_b - 1 - n] (no atom on an edge)."""
    w = synth.tiny_fcc()
    _, xc = oracle.gather(w.xyz, w.centres[3], 1.0)
    u = w.dirs[:200]
    h = oracle.histograms(xc, u, 8, 1.0)
    hm = oracle.histograms(xc, -u, 8, 1.0)
    assert np.all(h.sum(1) == xc.shape[0])
    assert np.array_equal(hm, h[:, ::-1])
    # in-ball atoms never reach the outer padding bin on the negative side
    assert h[:, 0].sum() == 0


# --------------------------------------------------------------------------
# membership
# --------------------------------------------------------------------------

def test_gather_matches_kdtree_ball():
    from scipy.spatial import cKDTree
    w = synth.tiny_fcc()
    tree = cKDTree(w.xyz.astype(np.float64))
    for c in w.centres[:6]:
        idx, xc = oracle.gather(w.xyz, c, 1.0)
        ref = np.sort(np.array(tree.query_ball_point(c, 1.0), np.int64))
        d = np.linalg.norm(w.xyz.astype(np.float64) - c, axis=1)
        sym = set(idx.tolist()) ^ set(ref.tolist())
        assert all(abs(d[i] - 1.0) < 1e-12 for i in sym)
        assert np.allclose(xc, (w.xyz[idx].astype(np.float64) - c).astype(np.float32))
        assert np.all(np.diff(idx) > 0)


def test_gather_type_mask():
    xyz, t = synth.perfect_crystal_roi("l12", 0.41, 1.0)
    idx_all, _ = oracle.gather(xyz, np.zeros(3), 1.0, types=t)
    idx_sc, _ = oracle.gather(xyz, np.zeros(3), 1.0, types=t, type_mask=0b10)
    idx_al, _ = oracle.gather(xyz, np.zeros(3), 1.0, types=t, type_mask=0b01)
    assert len(idx_all) == len(idx_sc) + len(idx_al)
    assert np.all(t[idx_sc] == 1) and np.all(t[idx_al] == 0)


# --------------------------------------------------------------------------
# spectrum
# --------------------------------------------------------------------------

def test_spectrum_closed_forms():
    m = 8
    nb = 1 << m
    h = np.zeros(nb, np.int32)
    h[37] = 1
    assert np.allclose(oracle.band_amplitudes(h, m, 0, nb // 2), 1.0, atol=1e-12)
    h[37] = 0
    b1, b2 = 40, 95
    h[b1] = 1
    h[b2] = 1
    k = np.arange(0, nb // 2 + 1)
    expect = np.abs(2 * np.cos(np.pi * k * (b1 - b2) / nb))
    assert np.allclose(oracle.band_amplitudes(h, m, 0, nb // 2), expect, atol=1e-12)
    rng = np.random.default_rng(3)
    h = rng.integers(0, 50, nb).astype(np.int32)
    assert oracle.band_amplitudes(h, m, 0, 0)[0] == pytest.approx(h.sum(), abs=0)


@pytest.mark.parametrize("m", [8, 10])
def test_spectrum_matches_numpy_rfft(m):
    rng = np.random.default_rng(m)
    nb = 1 << m
    h = rng.integers(0, 30, nb).astype(np.int32)
    ref = np.abs(np.fft.rfft(h.astype(np.float64)))
    got = oracle.band_amplitudes(h, m, 0, nb // 2)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-9 * ref.max())
    got2 = oracle.band_amplitudes(h, m, 8, 128)
    assert np.allclose(got2, ref[8:129], rtol=1e-12, atol=1e-9 * ref.max())


def test_signature_is_band_max_with_lowest_argk():
    w = synth.tiny_fcc()
    _, xc = oracle.gather(w.xyz, w.centres[0], 1.0)
    u = w.dirs[:64]
    S, ak = oracle.roi_signature(xc, u, 8, 1.0, 6, 14)
    h = oracle.histograms(xc, u, 8, 1.0)
    for v in range(64):
        a = np.abs(np.fft.rfft(h[v].astype(np.float64)))[6:15]
        assert S[v] == pytest.approx(a.max(), rel=1e-12)
        assert ak[v] == 6 + int(np.argmax(a >= a.max() * (1 - 1e-12)))
    # X(0) = N_w: the peak at the origin counts the atoms (Section 3.1)
    S0, _ = oracle.roi_signature(xc, u, 8, 1.0, 0, 0)
    assert np.allclose(S0, xc.shape[0])
    # exact ties: one atom at the centre sits in bin 2^(m-1), so
    # X(k) = (-1)^k and |X(k)| = 1 at every k; the lowest k of the band wins
    S1, ak1 = oracle.roi_signature(np.zeros((1, 3), np.float32), u[:4], 8, 1.0, 6, 14)
    assert np.all(S1 == 1.0) and np.all(ak1 == 6)


# --------------------------------------------------------------------------
# the paper's verification experiment (Section 3.1, Fig. 2)
# --------------------------------------------------------------------------

def _spectrum_along(kind, a, R, m, direction, types_keep=None):
    xyz, t = synth.perfect_crystal_roi(kind, a, R, types_keep=types_keep)
    _, xc = oracle.gather(xyz, np.zeros(3), R)
    d = np.asarray(direction, float)
    u = (d / np.linalg.norm(d)).astype(np.float32)[None, :]
    h = oracle.histograms(xc, u, m, R)
    return oracle.band_amplitudes(h[0], m, 0, (1 << m) // 2), xc.shape[0]


def test_fig2_worked_example_al_200_bin_19():
    g = json.load(open(os.path.join(GOLDEN, "fig2_peak_position.json")))
    R, m, a = g["R_nm"], g["m"], g["a_nm"]
    dR = R / ((1 << (m - 1)) - 1)
    W = 2 * (R + dR)                        # = L / f_s
    assert math.floor(W / g["plane_spacing_nm"]) == g["expected_bin_floor"]
    amp, nw = _spectrum_along("fcc", a, R, m, g["direction"])
    assert amp[0] == pytest.approx(nw)      # peak at the origin = atom count
    k = 2 + int(np.argmax(amp[2:]))
    assert k in (19, 20)                    # nearest integer frequency of 19.91
    assert amp[k] > 0.3 * nw


@pytest.mark.parametrize("kind,a,m,direction,d", [
    ("fcc", 0.405, 8, [1, 1, 1], 0.405 / math.sqrt(3)),
    ("fcc", 0.405, 8, [1, 1, 0], 0.405 / (2 * math.sqrt(2))),
    ("bcc", 0.287, 10, [1, 1, 0], 0.287 / math.sqrt(2)),
    ("bcc", 0.316, 8, [1, 0, 0], 0.316 / 2),
])
def test_peak_at_plane_spacing(kind, a, m, direction, d):
    """Perfect lattice, ROI centred on a site: the strongest non-zero
    frequency lies within 1 of W / d_hkl for the allowed reflection."""
    R = 2.0
    dR = R / ((1 << (m - 1)) - 1)
    W = 2 * (R + dR)
    amp, nw = _spectrum_along(kind, a, R, m, direction)
    k = 2 + int(np.argmax(amp[2:int(1.3 * W / d) + 2]))
    assert abs(k - W / d) <= 1.0


def test_l12_sublattices_differ_from_fcc():
    """Along [100] the L1_2 Sc sub-lattice (cube corners) repeats every a and
    peaks at W / a, where f.c.c. (and the full L1_2 set of sites) has no peak:
    the two sub-lattice spectra distinguish L1_2 from f.c.c. (Section 3.1)."""
    R, m, a = 2.0, 8, 0.41
    dR = R / ((1 << (m - 1)) - 1)
    W = 2 * (R + dR)
    ka = int(round(W / a))
    sc, nsc = _spectrum_along("l12", a, R, m, [1, 0, 0], types_keep=[1])
    al, nal = _spectrum_along("l12", a, R, m, [1, 0, 0], types_keep=[0])
    fcc, nf = _spectrum_along("fcc", a, R, m, [1, 0, 0])
    assert sc[ka] / nsc > 0.5
    assert fcc[ka] / nf < 0.1
    assert al[ka] / nal > 0.2         # Al planes alternate 1:2 in density
    assert abs((sc[ka] * 1.0) - al[ka] / 2.0) < 0.5 * sc[ka] + 1


def test_band_interval_reproduces_paper_al_200():
    g = json.load(open(os.path.join(GOLDEN, "al_band_interval.json")))
    d = g["al_d200_nm"]
    dmin, dmax = synth.band_spacing(d)
    assert dmin == pytest.approx(g["al_interval_nm"][0], rel=2e-3)
    assert dmax == pytest.approx(g["al_interval_nm"][1], rel=2e-3)
    d2 = g["al3li_d200_nm"]
    assert synth.band_spacing(d2)[0] == pytest.approx(g["al3li_interval_nm"][0], rel=2e-3)
    assert synth.band_spacing(d2)[1] == pytest.approx(g["al3li_interval_nm"][1], rel=2e-3)
    lo, hi = oracle.band_for_spacing(dmin, dmax, g["R_nm"], g["m"])
    R, m = g["R_nm"], g["m"]
    W = 2 * (R + R / ((1 << (m - 1)) - 1))
    assert lo == math.ceil(W / dmax) and hi == math.floor(W / dmin)
    assert lo <= 20 <= hi                   # contains the Al {200} peak of Fig. 2


# --------------------------------------------------------------------------
# symmetry and rotation covariance
# --------------------------------------------------------------------------

def test_cubic_point_group_invariance():
    """Unrotated perfect f.c.c. centred on a site: S(P u) = S(u) for all 48
    signed permutations P (the ball and the crystal are invariant), up to
    atoms that sit on a bin edge."""
    R, m, a = 1.013, 8, 0.405
    xyz, _ = synth.perfect_crystal_roi("fcc", a, R)
    _, xc = oracle.gather(xyz, np.zeros(3), R)
    lo, hi = 8, 14
    rng = np.random.default_rng(5)
    base = rng.standard_normal((6, 3))
    base /= np.linalg.norm(base, axis=1, keepdims=True)
    P = synth.signed_permutation_matrices()
    dirs = np.concatenate([(P @ b) for b in base]).astype(np.float32)
    S, _ = oracle.roi_signature(xc, dirs, m, R, lo, hi)
    S = S.reshape(6, 48)
    rel = np.abs(S - S[:, :1]) / S.max()
    assert np.median(rel) < 1e-9
    assert rel.max() < 0.05


def test_rotation_covariance():
    """Rotating the crystal by g gives S_g(u) = S(g^T u)."""
    R, m, a = 1.5, 8, 0.405
    q = synth.axis_angle_quaternion([1, 2, 3], 0.7)
    G = synth.quat_to_matrix(q)
    xyz, _ = synth.perfect_crystal_roi("fcc", a, R)
    xyz_r = (xyz.astype(np.float64) @ G.T).astype(np.float32)
    _, xc = oracle.gather(xyz, np.zeros(3), R)
    _, xcr = oracle.gather(xyz_r, np.zeros(3), R)
    assert xc.shape == xcr.shape
    u = synth.icosphere(3).astype(np.float64)
    ug = (u @ G).astype(np.float32)          # rows g^T u
    S_rot, _ = oracle.roi_signature(xcr, u.astype(np.float32), m, R, 8, 14)
    S_ref, _ = oracle.roi_signature(xc, ug, m, R, 8, 14)
    rel = np.abs(S_rot - S_ref) / S_ref.max()
    assert np.median(rel) < 1e-6
    assert rel.max() < 0.05


# --------------------------------------------------------------------------
# disorientation
# --------------------------------------------------------------------------

def test_disorientation_textbook_values():
    I = np.array([1.0, 0, 0, 0])
    for ang, exp in [(10, 10), (30, 30), (50, 40), (90, 0), (130, 40)]:
        q = synth.axis_angle_quaternion([1, 0, 0], math.radians(ang))
        assert oracle.disorientation_deg(I, q) == pytest.approx(exp, abs=1e-9)
    q = synth.axis_angle_quaternion([1, 1, 1], math.radians(60))
    assert oracle.disorientation_deg(I, q) == pytest.approx(60, abs=1e-9)
    q = synth.axis_angle_quaternion([1, 1, 1], math.radians(120))
    assert oracle.disorientation_deg(I, q) == pytest.approx(0, abs=1e-6)
    rng = np.random.default_rng(0)
    Q = synth.random_quaternions(rng, 300)
    d = [oracle.disorientation_deg(Q[i], Q[i + 1]) for i in range(299)]
    assert max(d) <= 62.81                  # cubic-cubic maximum (Mackenzie)
    # symmetric equivalents give zero
    for s in synth.cubic_rotation_matrices():
        qs = synth.quat_mul(Q[0], synth.matrix_to_quat(s))
        assert oracle.disorientation_deg(Q[0], qs) == pytest.approx(0, abs=1e-6)


# --------------------------------------------------------------------------
# indexing, Eq. 3
# --------------------------------------------------------------------------

def test_quat_to_matrix_matches_axis_angle_rodrigues():
    ax = np.array([0.3, -0.5, 0.8])
    ax /= np.linalg.norm(ax)
    th = 0.9
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Rr = np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K
    assert np.allclose(oracle.quat_to_matrix(synth.axis_angle_quaternion(ax, th)), Rr, atol=1e-14)


def test_lut_is_nearest_node():
    u = synth.icosphere(3)
    rng = np.random.default_rng(2)
    q = synth.random_quaternions(rng, 7)
    top = np.array([0, 5, 100, 641], np.int32)
    L = oracle.lut(u, top, q)
    for g in range(7):
        M = synth.quat_to_matrix(q[g])
        for k, v in enumerate(top):
            r = M @ u[v].astype(np.float64)
            dots = u.astype(np.float64) @ r
            assert dots[L[g, k]] >= dots.max() - 1e-6


def test_normalise_divides_each_row_by_its_maximum():
    """Normalisation S / max_v S per row (values exact in binary); an
    all-zero row stays zero."""
    S = np.array([[0.5, 2.0, 1.0], [0.0, 0.0, 0.0], [3.0, 3.0, 1.5]])
    assert np.array_equal(oracle.normalise(S), [[0.25, 1.0, 0.5], [0.0, 0.0, 0.0], [1.0, 1.0, 0.5]])


def test_top_nodes_order_and_ties():
    s = np.array([0.5, 0.9, 0.9, 0.1, 0.7], np.float32)
    assert list(oracle.top_nodes(s, 4)) == [1, 2, 4, 0]


def test_match_recovers_planted_orientation():
    """A measured signature holding the reference values at the look-up nodes
    of test orientation g* scores Delta(g*) = 0, the unique minimum."""
    u = synth.icosphere(3)
    ref = synth.bump_values(synth.family_100(), 12.0, u)
    ref = ref / ref.max()
    top = oracle.top_nodes(ref, 60)
    rng = np.random.default_rng(4)
    Q = synth.random_quaternions(rng, 50)
    L = oracle.lut(u, top, Q)
    # plant at an orientation whose look-up row has no two top nodes on the
    # same measured node (otherwise Delta(g*) = 0 is not reachable)
    gstar = next(g for g in range(10, 50) if len(np.unique(L[g])) == len(top))
    msr = np.full((1, u.shape[0]), 0.05, np.float32)
    msr[0, L[gstar]] = ref[top]
    best, bs, sc = oracle.match(msr, ref, top, L, return_scores=True)
    assert best[0] == gstar and bs[0] == 0.0
    assert np.sort(sc[0])[1] > 0.0
    # Eq. 3 by hand for one g
    g = 3
    assert sc[0, g] == pytest.approx(float(np.sum((msr[0, L[g]].astype(float) - ref[top]) ** 2)), rel=1e-12)


def _phase_case():
    """Three references (bumps around <100>, <110>, <111>) on a level-3
    icosphere, 40 strongest nodes each, 60 test orientations."""
    u = synth.icosphere(3)
    fam = [synth.family_100(), synth.family_110(),
           np.array([[1, 1, 1], [1, 1, -1], [1, -1, 1], [-1, 1, 1]], float) / np.sqrt(3)]
    fam[2] = np.concatenate([fam[2], -fam[2]])
    refs = []
    for f in fam:
        r = synth.bump_values(f, 12.0, u)
        refs.append((r / r.max()).astype(np.float32))
    n_hat = 40
    tops = [oracle.top_nodes(r, n_hat) for r in refs]
    rng = np.random.default_rng(9)
    Q = np.concatenate([[[1.0, 0, 0, 0]], synth.random_quaternions(rng, 59)])
    luts = [oracle.lut(u, t, Q) for t in tops]
    return u, refs, tops, luts, rng


def _energy(ref, top):
    r = np.asarray(ref, np.float64)[top]
    return float((r * r).sum())


def test_match_phase_reduces_to_eq3_and_averages_channels():
    """A one-channel candidate gives Eq. 3's argmin and its minimum divided by
    the reference's energy E = sum of its squared strongest values; a
    candidate of two identical channels gives the same score (the channels'
    mean, not their sum); equal candidates resolve to the lower index."""
    u, refs, tops, luts, rng = _phase_case()
    S = rng.random((2, 5, u.shape[0])).astype(np.float32)
    off = [0, 1, 3, 5]
    sig = [0, 1, 1, 1, 1]
    R = [refs[0], refs[1], refs[1], refs[1], refs[1]]
    T = [tops[0], tops[1], tops[1], tops[1], tops[1]]
    L = [luts[0], luts[1], luts[1], luts[1], luts[1]]
    phase, best, score = oracle.match_phase(S, off, sig, R, T, L)
    b0, s0 = oracle.match(S[0], refs[0], tops[0], luts[0])
    b1, s1 = oracle.match(S[1], refs[1], tops[1], luts[1])
    e0, e1 = _energy(refs[0], tops[0]), _energy(refs[1], tops[1])
    assert abs(e0 - e1) > 0.05 * e1    # the references differ in energy: the division shows
    assert np.array_equal(best[0], b0) and np.allclose(score[0], s0 / e0, rtol=1e-12)
    for c in (1, 2):
        assert np.array_equal(best[c], b1) and np.allclose(score[c], s1 / e1, rtol=1e-12)
    assert np.all(phase != 2)          # candidates 1 and 2 tie: the lower index wins
    assert np.array_equal(phase, np.where(score[1] < score[0], 1, 0))


def test_match_phase_empty_signature_scores_one():
    """An empty measured signature differs from every rotated reference by
    exactly the reference's energy (Eq. 3 with S = 0 sums the squared
    strongest reference values), so every candidate scores 1 at every
    orientation, whatever its channels: the lowest g and the lowest
    candidate win the ties."""
    u, refs, tops, luts, rng = _phase_case()
    S = np.zeros((3, 2, u.shape[0]), np.float32)
    phase, best, score = oracle.match_phase(S, [0, 1, 3], [0, 1, 2], [refs[0], refs[1], refs[2]],
                                            [tops[0], tops[1], tops[2]], [luts[0], luts[1], luts[2]])
    assert np.allclose(score, 1.0, rtol=1e-12, atol=0)
    assert np.all(best == 0) and np.all(phase == 0)


def test_match_phase_recovers_planted_candidate():
    """Measured signatures holding candidate 1's references at the look-up
    nodes of g* in both of its channels: candidate 1 scores Delta(g*) = 0 and
    is the phase; candidate 0 (one channel, another reference) scores above 0."""
    u, refs, tops, luts, rng = _phase_case()
    ng = luts[0].shape[0]
    gstar = next(g for g in range(5, ng) if len(np.unique(luts[1][g])) == len(tops[1])
                 and len(np.unique(luts[2][g])) == len(tops[2]))
    S = np.full((3, 4, u.shape[0]), 0.05, np.float32)
    for r in range(4):
        S[1, r, luts[1][gstar]] = refs[1][tops[1]]
        S[2, r, luts[2][gstar]] = refs[2][tops[2]]
    off = [0, 1, 3]
    sig = [0, 1, 2]
    phase, best, score = oracle.match_phase(S, off, sig, [refs[0], refs[1], refs[2]], [tops[0], tops[1], tops[2]],
                                            [luts[0], luts[1], luts[2]])
    assert np.all(best[1] == gstar) and np.all(score[1] == 0.0)
    assert np.all(score[0] > 0.0) and np.all(phase == 1)


def test_match_topk_orders_solutions():
    """Top-k of Eq. 3: the planted orientation first with Delta = 0, then the
    rest ascending by (Delta, g) as a brute-force ranking of the hand-computed
    Delta gives; k = 1 is the plain argmin; equal Delta keeps the lower g."""
    u = synth.icosphere(3)
    ref = synth.bump_values(synth.family_100(), 12.0, u)
    ref = ref / ref.max()
    top = oracle.top_nodes(ref, 60)
    rng = np.random.default_rng(4)
    Q = synth.random_quaternions(rng, 50)
    L = oracle.lut(u, top, Q)
    gstar = next(g for g in range(10, 50) if len(np.unique(L[g])) == len(top))
    msr = np.full((2, u.shape[0]), 0.05, np.float32)
    msr[0, L[gstar]] = ref[top]
    g, d = oracle.match_topk(msr, ref, top, L, 7)
    assert g[0, 0] == gstar and d[0, 0] == 0.0
    hand = [(float(np.sum((msr[0, L[h]].astype(float) - ref[top]) ** 2)), h) for h in range(Q.shape[0])]
    assert [h for _, h in sorted(hand)[:7]] == list(g[0])
    assert np.all(np.diff(d[0]) >= 0)
    best, _ = oracle.match(msr, ref, top, L)
    g1, _ = oracle.match_topk(msr, ref, top, L, 1)
    assert np.array_equal(g1[:, 0], best)
    # a constant measured signature gives every g the same Delta: ties keep g order
    assert list(g[1]) == list(range(7))


def test_refine_roi_grid_geometry_and_threshold():
    """Grid refinement: peaks 1.0, 0.8, 0.5 and kappa = 0.75 keep the first two
    ROIs; each gets 125 new centres on a 5 x 5 x 5 lattice of pitch
    spacing / 5 centred on it, filling its cell (extent spacing - pitch), the
    x index running fastest."""
    S = np.array([[0.2, 1.0, 0.3], [0.8, 0.1, 0.0], [0.5, 0.5, 0.4]])
    centres = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [4.0, 0.0, 0.0]])
    c, par = oracle.refine_roi_grid(S, centres, 0.75, 2.0, 5)
    assert c.shape == (250, 3) and list(np.unique(par)) == [0, 1]
    for r in (0, 1):
        sub = c[par == r]
        assert np.allclose(sub.mean(axis=0), centres[r])
        assert np.allclose(sub.max(axis=0) - sub.min(axis=0), 2.0 - 0.4)
        assert np.allclose(np.unique(np.round(sub[:, 0] - centres[r, 0], 12)), [-0.8, -0.4, 0.0, 0.4, 0.8])
    assert np.allclose(c[1] - c[0], [0.4, 0.0, 0.0]) and np.allclose(c[5] - c[0], [0.0, 0.4, 0.0])
    c2, _ = oracle.refine_roi_grid(S, centres, 0.5, 2.0, 2)     # 0.5 * 1.0: the third ROI just qualifies
    assert c2.shape == (24, 3)


def test_fsp_closed_forms():
    """Eq. 2 closed forms: one atom anywhere gives |F| = 1 on the whole grid;
    at k = 0 (odd L puts it at the centre) |F| = N_w; two atoms d apart along
    x give |F| = |2 cos(pi k_x d)|; grid points follow k = -kmax + i dk."""
    L = 5
    one = oracle.fsp(np.array([[0.3, -0.7, 1.1]], np.float32), L)
    assert np.allclose(one, 1.0, atol=1e-12)
    rng = np.random.default_rng(1)
    xc = rng.uniform(-2, 2, (37, 3)).astype(np.float32)
    c = ((L // 2) * L + L // 2) * L + L // 2
    assert oracle.fsp(xc, L, points=[c])[0] == pytest.approx(37.0, abs=1e-9)
    d = 0.25
    two = np.array([[-d / 2, 0.0, 0.0], [d / 2, 0.0, 0.0]], np.float32)
    F = oracle.fsp(two, L).reshape(L, L, L)
    kx = -2 * np.pi + np.arange(L) * (4 * np.pi / (L - 1))
    assert np.allclose(F[:, 1, 3], np.abs(2 * np.cos(np.pi * kx * np.float64(np.float32(d)))), atol=1e-9)


def test_fsp_matches_brute_force_and_lattice_peaks():
    """Eq. 2 against a numpy evaluation of the same sum on random points, and a
    simple cubic lattice of pitch 0.5 nm peaking at its reciprocal lattice
    points k = (h, k, l) / 0.5 with |F| = N_w."""
    rng = np.random.default_rng(2)
    xc = rng.uniform(-1.5, 1.5, (50, 3)).astype(np.float32)
    L = 7
    F = oracle.fsp(xc, L)
    k = -np.pi * 2 + np.arange(L) * (4 * np.pi / (L - 1))
    K = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3)
    ref = np.abs(np.exp(-2j * np.pi * (K @ xc.astype(np.float64).T)).sum(axis=1))
    assert np.allclose(F, ref, rtol=1e-10, atol=1e-9)
    g = np.arange(-3, 4) * 0.5
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    # kmax = 2 per nm, L = 9: dk = 0.5, k = 2 per nm (= 1 / 0.5) is grid index 8
    F2 = oracle.fsp(lat, 9, kmax=2.0).reshape(9, 9, 9)
    assert F2[8, 4, 4] == pytest.approx(lat.shape[0], rel=1e-9)
    assert F2[4, 4, 4] == pytest.approx(lat.shape[0], rel=1e-9)
    assert F2[6, 4, 4] < 0.2 * lat.shape[0]


def test_match_indexes_rotated_crystal_end_to_end():
    """Signatures of a rotated perfect f.c.c. ROI, matched against the
    unrotated reference over a test-orientation set that contains the true
    orientation, rank the true orientation first (Section 3.2, Fig. 4: the
    lowest image difference has the lowest disorientation)."""
    R, m, a = 1.0, 8, 0.405
    u = synth.icosphere(4)
    lo, hi = oracle.band_for_spacing(*synth.band_spacing(a / 2), R, m)
    xyz, _ = synth.perfect_crystal_roi("fcc", a, R)
    _, xc = oracle.gather(xyz, np.zeros(3), R)
    ref, _ = oracle.roi_signature(xc, u, m, R, lo, hi)
    ref = (ref / ref.max()).astype(np.float32)
    rng = np.random.default_rng(9)
    qt = synth.random_quaternions(rng, 1)[0]
    grid = np.concatenate([synth.so3_grid(6.0), qt[None]])
    G = synth.quat_to_matrix(qt)
    xr = (xyz.astype(np.float64) @ G.T).astype(np.float32)
    _, xcr = oracle.gather(xr, np.zeros(3), R)
    msr, _ = oracle.roi_signature(xcr, u, m, R, lo, hi)
    msr = (msr / msr.max()).astype(np.float32)[None, :]
    top = oracle.top_nodes(ref, 300)
    L = oracle.lut(u, top, grid)
    best, _, sc = oracle.match(msr, ref, top, L, return_scores=True)
    assert best[0] == grid.shape[0] - 1
    # the runner-up orientations are near-misses or symmetry-related ones
    order = np.argsort(sc[0])
    assert oracle.disorientation_deg(grid[order[1]], qt) < 12.0


# --------------------------------------------------------------------------
# refinement
# --------------------------------------------------------------------------

def _ref_image():
    d = synth.elevation_azimuth_grid(1.0)
    img = synth.bump_values(synth.family_100(), 9.0, d)
    return img / img.max()


def test_bilinear_reproduces_grid_values_and_is_linear_inside_cells():
    img = _ref_image()
    for (i, j) in [(30, 40), (90, 0), (150, 359), (100, 200)]:
        al, be = math.radians(-90 + i), math.radians(j)
        c = np.array([math.cos(al) * math.cos(be), math.cos(al) * math.sin(be), math.sin(al)])
        ok, val, _, cell = oracle.bilinear(img, c)
        assert ok and val == pytest.approx(float(img[i, j]), abs=1e-12)
    # midpoint of a cell = mean of its four corners
    al, be = math.radians(-90 + 60.5), math.radians(10.5)
    c = np.array([math.cos(al) * math.cos(be), math.cos(al) * math.sin(be), math.sin(al)])
    ok, val, _, _ = oracle.bilinear(img, c)
    assert val == pytest.approx(float(img[60:62, 10:12].astype(float).mean()), abs=1e-12)
    ok, _, _, _ = oracle.bilinear(img, np.array([0.0, 0.001, 1.0]))
    assert not ok                           # inside the excluded pole cap


def _synthetic_measurement(img, u, qt):
    """S_msr(u) = I(g^T u) for the true orientation (a closed-form minimum)."""
    G = synth.quat_to_matrix(qt)
    out = np.zeros(u.shape[0], np.float32)
    for v in range(u.shape[0]):
        ok, val, _, _ = oracle.bilinear(img, G.T @ u[v].astype(float))
        out[v] = val if ok else 0.0
    return out


def test_refine_gradient_matches_finite_differences():
    img = _ref_image()
    u = synth.icosphere(3)
    qt = synth.axis_angle_quaternion([1, 2, 2], 0.4)
    msr = _synthetic_measurement(img, u, qt)
    q = synth.quat_mul(synth.axis_angle_quaternion([0, 1, 1], math.radians(2.0)), qt)
    h = 1e-4
    G = synth.quat_to_matrix(q)
    # leave out directions whose stencil crosses a cell edge or the pole cap
    w = np.ones(u.shape[0])
    for v in range(u.shape[0]):
        cells = set()
        for ax in range(3):
            for sgn in (-1, 1):
                d = np.zeros(3)
                d[ax] = sgn * h
                E = synth.quat_to_matrix(synth.axis_angle_quaternion(d, np.linalg.norm(d)))
                ok, _, _, cell = oracle.bilinear(img, (E @ G).T @ u[v].astype(float))
                cells.add((ok, int(cell[0]), int(cell[1])))
        ok0, _, _, cell0 = oracle.bilinear(img, G.T @ u[v].astype(float))
        cells.add((ok0, int(cell0[0]), int(cell0[1])))
        if len(cells) > 1:
            w[v] = 0.0
    L0, g, H, b = oracle.refine_eval(img, msr, u, q, weights=w)
    fd = np.zeros(3)
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        qp = synth.quat_mul(synth.axis_angle_quaternion(e, h), q)
        qm = synth.quat_mul(synth.axis_angle_quaternion(-e, h), q)
        fd[ax] = (oracle.refine_eval(img, msr, u, qp, weights=w)[0]
                  - oracle.refine_eval(img, msr, u, qm, weights=w)[0]) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-7 * max(1.0, np.abs(g).max()))
    assert np.allclose(g, 2 * b)
    assert np.allclose(H, H.T) and np.all(np.linalg.eigvalsh(H) >= -1e-12)


def test_refine_converges_to_truth():
    img = _ref_image()
    u = synth.icosphere(4)
    rng = np.random.default_rng(12)
    for trial in range(3):
        qt = synth.random_quaternions(rng, 1)[0]
        msr = _synthetic_measurement(img, u, qt)
        ax = rng.standard_normal(3)
        q0 = synth.quat_mul(synth.axis_angle_quaternion(ax, math.radians(2.5)), qt)
        q, loss = oracle.refine(img, msr, u, q0, iters=20)
        assert oracle.disorientation_deg(q[0], qt) < 0.05
        assert loss[0] < 1e-6
