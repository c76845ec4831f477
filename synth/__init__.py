"""Seeded synthetic inputs for the real-space (RSP) signature path.

Everything here produces plain input arrays: atom positions of perfect and
noisy cubic crystals, icosphere direction sets, ROI centres and radii,
orientation sets and smooth spherical test images.  None of the signature
method's arithmetic (membership, projection, binning, spectrum, band
selection, matching, refinement) lives here; the FP64 oracle and the CUDA
path both consume these arrays unchanged.

The shapes follow the paper's synthetic workloads: single crystals of f.c.c.
Al (a = 0.405 nm), L1_2 Al3Sc (a = 0.410 nm) and b.c.c. W (a = 0.316 nm)
(Section 3.1), random removal of atoms down to a kept fraction eta and
anisotropic Gaussian displacements sigma_x = sigma_y = 2 sigma_z (Section 3.1,
"How robust are signatures"), a Poisson-Voronoi polycrystal (Section 3.3) and
a geodesic-sphere direction set with 40962 nodes (Section 2.2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20200901

# ---------------------------------------------------------------------------
# Direction sets
# ---------------------------------------------------------------------------

_ICO_FACES = np.array(
    [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
     (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
     (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
     (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)], dtype=np.int64)


def icosphere(level: int, return_faces: bool = False):
    """Unit normals of a geodesic (icosphere) mesh with 10*4**level + 2 nodes.

    Level 5 gives 10242 nodes and level 6 gives the paper's N_v = 40962
    (Section 2.2).  Each level splits every triangle into four through edge
    midpoints projected onto the sphere.  Computed in float64, returned as
    float32 [N_v, 3] row-major.
    """
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
                  (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
                  (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = _ICO_FACES.copy()
    for _ in range(level):
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        e.sort(axis=1)
        uniq, inv = np.unique(e, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        mid = v[uniq[:, 0]] + v[uniq[:, 1]]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        base = v.shape[0]
        v = np.concatenate([v, mid], axis=0)
        n = f.shape[0]
        m01 = base + inv[0:n]
        m12 = base + inv[n:2 * n]
        m20 = base + inv[2 * n:3 * n]
        f = np.concatenate([
            np.stack([f[:, 0], m01, m20], axis=1),
            np.stack([f[:, 1], m12, m01], axis=1),
            np.stack([f[:, 2], m20, m12], axis=1),
            np.stack([m01, m12, m20], axis=1)], axis=0)
    out = np.ascontiguousarray(v.astype(np.float32))
    if return_faces:
        return out, f
    return out


def elevation_azimuth_grid(step_deg: float = 1.0):
    """Directions of a regular elevation-azimuth grid (rows = elevation).

    Elevation alpha_i = -90 + i*step (i = 0..180/step), azimuth beta_j = j*step
    (j < 360/step); d = (cos a cos b, cos a sin b, sin a) as in Eq. 1.
    Returns float32 [n_alpha, n_beta, 3].
    """
    na = int(round(180.0 / step_deg)) + 1
    nb = int(round(360.0 / step_deg))
    a = np.deg2rad(-90.0 + step_deg * np.arange(na))[:, None]
    b = np.deg2rad(step_deg * np.arange(nb))[None, :]
    d = np.stack([np.cos(a) * np.cos(b), np.cos(a) * np.sin(b),
                  np.broadcast_to(np.sin(a), (na, nb))], axis=-1)
    return np.ascontiguousarray(d.astype(np.float32))


# ---------------------------------------------------------------------------
# Rotations (input generation only: orienting synthetic crystals)
# ---------------------------------------------------------------------------

def random_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Haar-uniform unit quaternions (w, x, y, z), w >= 0 (Shoemake 1992)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    q = np.stack([np.sqrt(u1) * np.cos(2 * np.pi * u3),
                  np.sqrt(1 - u1) * np.sin(2 * np.pi * u2),
                  np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                  np.sqrt(u1) * np.sin(2 * np.pi * u3)], axis=1)
    q[q[:, 0] < 0] *= -1
    return q


def quat_to_matrix(q) -> np.ndarray:
    """Rotation matrix of a unit quaternion (w, x, y, z); maps crystal -> lab."""
    w, x, y, z = (float(c) for c in q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def axis_angle_quaternion(axis, angle_rad: float) -> np.ndarray:
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    h = 0.5 * angle_rad
    return np.array([math.cos(h), *(math.sin(h) * axis)])


def quat_mul(a, b) -> np.ndarray:
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def bunge_to_matrix(phi1_deg: float, Phi_deg: float, phi2_deg: float) -> np.ndarray:
    """Crystal -> lab rotation for Bunge angles (Z-X-Z), as used for the
    (8, 8, 8) degree single crystals of Section 3.1."""
    p1, P, p2 = np.deg2rad([phi1_deg, Phi_deg, phi2_deg])
    rz1 = np.array([[math.cos(p1), -math.sin(p1), 0], [math.sin(p1), math.cos(p1), 0], [0, 0, 1]])
    rx = np.array([[1, 0, 0], [0, math.cos(P), -math.sin(P)], [0, math.sin(P), math.cos(P)]])
    rz2 = np.array([[math.cos(p2), -math.sin(p2), 0], [math.sin(p2), math.cos(p2), 0], [0, 0, 1]])
    return rz1 @ rx @ rz2


def cubic_rotation_matrices() -> np.ndarray:
    """The 24 proper rotations of the cubic point group m-3m (det = +1 signed
    permutation matrices).  Returned [24, 3, 3] float64, identity first."""
    import itertools
    mats = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            m = np.zeros((3, 3))
            for r, c in enumerate(perm):
                m[r, c] = signs[r]
            if round(np.linalg.det(m)) == 1:
                mats.append(m)
    mats.sort(key=lambda m: (0 if np.allclose(m, np.eye(3)) else 1))
    return np.array(mats)


def signed_permutation_matrices() -> np.ndarray:
    """All 48 signed permutation matrices (the full cubic group incl. inversion)."""
    import itertools
    mats = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            m = np.zeros((3, 3))
            for r, c in enumerate(perm):
                m[r, c] = signs[r]
            mats.append(m)
    return np.array(mats)


# ---------------------------------------------------------------------------
# Crystals
# ---------------------------------------------------------------------------

#: fractional basis and atom-type id per site; L1_2 puts the minority species
#: (Sc, type 1) on the cube corners and Al (type 0) on the face centres.
LATTICES = {
    "sc": (np.array([[0, 0, 0]], float), np.array([0], np.uint8)),
    "bcc": (np.array([[0, 0, 0], [.5, .5, .5]], float), np.array([0, 0], np.uint8)),
    "fcc": (np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], float),
            np.array([0, 0, 0, 0], np.uint8)),
    "l12": (np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], float),
            np.array([1, 0, 0, 0], np.uint8)),
}


def lattice_box(kind: str, a: float, lo, hi, rot=None, origin=None):
    """All sites of a (rotated) cubic lattice inside the half-open box [lo, hi).

    Site positions are origin + a * rot @ (n + basis) with integer n; rot maps
    crystal to lab.  The default origin is the box centre, which is then a
    lattice site.  Returns (xyz float64 [N, 3], types uint8 [N]).
    """
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    rot = np.eye(3) if rot is None else np.asarray(rot, float)
    origin = (lo + hi) / 2 if origin is None else np.asarray(origin, float)
    basis, btypes = LATTICES[kind]
    corners = np.array([[x, y, z] for x in (lo[0], hi[0]) for y in (lo[1], hi[1])
                        for z in (lo[2], hi[2])]) - origin
    cc = corners @ rot / a
    nmin = np.floor(cc.min(0)).astype(np.int64) - 1
    nmax = np.ceil(cc.max(0)).astype(np.int64) + 1
    nx = np.arange(nmin[0], nmax[0] + 1)
    ny = np.arange(nmin[1], nmax[1] + 1)
    gx, gy = np.meshgrid(nx, ny, indexing="ij")
    gx = gx.reshape(-1).astype(float)
    gy = gy.reshape(-1).astype(float)
    step = a * rot[:, 2]
    out_xyz, out_t = [], []
    for b, t in zip(basis, btypes):
        base = origin[None, :] + a * (np.outer(gx + b[0], rot[:, 0]) + np.outer(gy + b[1], rot[:, 1])
                                      + b[2] * rot[:, 2][None, :])
        zlo = np.full(base.shape[0], -np.inf)
        zhi = np.full(base.shape[0], np.inf)
        for j in range(3):
            if abs(step[j]) < 1e-15:
                bad = (base[:, j] < lo[j]) | (base[:, j] >= hi[j])
                zlo[bad] = np.inf
                continue
            l = (lo[j] - base[:, j]) / step[j]
            h = (hi[j] - base[:, j]) / step[j]
            zlo = np.maximum(zlo, np.minimum(l, h))
            zhi = np.minimum(zhi, np.maximum(l, h))
        ok = np.isfinite(zlo) & np.isfinite(zhi) & (zhi >= zlo)
        zl = np.ceil(zlo[ok] - 1e-9).astype(np.int64)
        zh = np.floor(zhi[ok] + 1e-9).astype(np.int64)
        cnt = np.maximum(zh - zl + 1, 0)
        tot = int(cnt.sum())
        if tot == 0:
            continue
        rows = np.repeat(np.nonzero(ok)[0], cnt)
        start = np.repeat(np.cumsum(cnt) - cnt, cnt)
        nz = np.repeat(zl, cnt) + (np.arange(tot) - start)
        p = base[rows] + nz[:, None].astype(float) * step[None, :]
        inside = np.all((p >= lo) & (p < hi), axis=1)
        out_xyz.append(p[inside])
        out_t.append(np.full(int(inside.sum()), t, np.uint8))
    if not out_xyz:
        return np.zeros((0, 3)), np.zeros(0, np.uint8)
    return np.concatenate(out_xyz), np.concatenate(out_t)


def keep_fraction(rng: np.random.Generator, n: int, eta: float) -> np.ndarray:
    """Boolean mask keeping each atom with probability eta (detection efficiency)."""
    return rng.random(n) < eta


def displace(rng: np.random.Generator, xyz: np.ndarray, sigma_xyz) -> np.ndarray:
    """Add independent Gaussian displacements with per-axis standard deviation."""
    s = np.asarray(sigma_xyz, float).reshape(1, 3)
    return xyz + rng.standard_normal(xyz.shape) * s


# ---------------------------------------------------------------------------
# ROI placement
# ---------------------------------------------------------------------------

def roi_grid(shape, pitch: float, centre) -> np.ndarray:
    """ROI centres on a regular grid (Section 2.4: ROIs placed on a 3D grid)."""
    idx = np.stack(np.meshgrid(*[np.arange(s) for s in shape], indexing="ij"), -1).reshape(-1, 3)
    off = (np.asarray(shape, float) - 1) / 2
    return np.ascontiguousarray(np.asarray(centre, float)[None, :] + (idx - off) * pitch)


def roi_random(rng: np.random.Generator, n: int, lo, hi, margin) -> np.ndarray:
    """ROI centres sampled uniformly at least `margin` inside every box face."""
    lo = np.asarray(lo, float) + margin
    hi = np.asarray(hi, float) - margin
    return lo + rng.random((n, 3)) * (hi - lo)


# ---------------------------------------------------------------------------
# Smooth spherical images (inputs for matching/refinement tests)
# ---------------------------------------------------------------------------

def bump_values(peaks, width_deg: float, dirs) -> np.ndarray:
    """Sum of Gaussian bumps exp(-theta^2 / (2 w^2)) around unit vectors `peaks`,
    evaluated at unit vectors `dirs` (theta = angle between them).  A smooth
    stand-in with the shape of an RSP signature (bright spots at one family of
    lattice-plane normals).  Returns float32 with the shape of dirs[..., 0]."""
    d = np.asarray(dirs, float)
    p = np.asarray(peaks, float)
    c = np.clip(np.tensordot(d, p.T, axes=1), -1.0, 1.0)
    th = np.arccos(c)
    w = np.deg2rad(width_deg)
    return np.exp(-(th ** 2) / (2 * w * w)).sum(-1).astype(np.float32)


def family_100() -> np.ndarray:
    return np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)


def family_110() -> np.ndarray:
    v = [[1, 1, 0], [1, -1, 0], [1, 0, 1], [1, 0, -1], [0, 1, 1], [0, 1, -1]]
    v = np.array(v, float) / math.sqrt(2)
    return np.concatenate([v, -v])


def family_111() -> np.ndarray:
    v = np.array([[1, 1, 1], [1, 1, -1], [1, -1, 1], [-1, 1, 1]], float) / math.sqrt(3)
    return np.concatenate([v, -v])


# ---------------------------------------------------------------------------
# Orientation sets
# ---------------------------------------------------------------------------

def _halton(n: int, base: int) -> np.ndarray:
    out = np.zeros(n)
    for i in range(n):
        f, r, k = 1.0, 0.0, i + 1
        while k > 0:
            f /= base
            r += f * (k % base)
            k //= base
        out[i] = r
    return out


def so3_grid(step_deg: float = 5.0, oversample: int = 16) -> np.ndarray:
    """Quasi-equidistant orientations in the cubic (m-3m) fundamental zone.

    Candidates: a Halton point set pushed through Shoemake's volume-preserving
    map [0,1)^3 -> SO(3), each reduced to its symmetry-equivalent quaternion
    with the largest |w| (the fundamental-zone representative).  Greedy
    thinning keeps a candidate only if it lies at least step_deg away from
    every kept orientation, giving a maximal step_deg-separated set (so every
    candidate is within step_deg of a kept one).  Returns float64 [N_g, 4]
    (w, x, y, z) with w > 0.  At 5 degrees N_g is a few thousand, the size the
    paper's 1-degree, 0.62 M orientation set has at 1 degree (Section 2.3).
    """
    from scipy.spatial import cKDTree
    theta = np.deg2rad(step_deg)
    vol_frac = (theta ** 3) / (math.pi ** 2) * 0.5
    n_target = max(64, int(1.0 / vol_frac / 24))
    n = n_target * oversample * 24
    u1, u2, u3 = _halton(n, 2), _halton(n, 3), _halton(n, 5)
    q = np.stack([np.sqrt(u1) * np.cos(2 * np.pi * u3),
                  np.sqrt(1 - u1) * np.sin(2 * np.pi * u2),
                  np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                  np.sqrt(u1) * np.sin(2 * np.pi * u3)], axis=1)
    best = _reduce_cubic_fz(q)
    # greedy thinning in the chordal metric of the 4-vectors (monotone in angle)
    chord = 2 * math.sin(theta / 4)  # |q1 - q2| for rotation angle theta
    tree = cKDTree(best)
    taken = np.zeros(len(best), bool)
    blocked = np.zeros(len(best), bool)
    for i in range(len(best)):
        if blocked[i]:
            continue
        taken[i] = True
        for j in tree.query_ball_point(best[i], chord):
            blocked[j] = True
    return np.ascontiguousarray(best[taken])


def _reduce_cubic_fz(q: np.ndarray) -> np.ndarray:
    """Each quaternion's symmetry-equivalent q * s (s one of the 24 proper
    cubic rotations) with the largest |w|, sign-fixed to w >= 0: the cubic
    fundamental-zone representative."""
    symq = np.array([_matrix_to_quat(m) for m in cubic_rotation_matrices()])
    best = None
    bestw = None
    for s in symq:
        qs = np.stack([q[:, 0] * s[0] - q[:, 1] * s[1] - q[:, 2] * s[2] - q[:, 3] * s[3],
                       q[:, 0] * s[1] + q[:, 1] * s[0] + q[:, 2] * s[3] - q[:, 3] * s[2],
                       q[:, 0] * s[2] - q[:, 1] * s[3] + q[:, 2] * s[0] + q[:, 3] * s[1],
                       q[:, 0] * s[3] + q[:, 1] * s[2] - q[:, 2] * s[1] + q[:, 3] * s[0]], 1)
        w = np.abs(qs[:, 0])
        if best is None:
            best, bestw = qs, w
        else:
            upd = w > bestw
            best[upd] = qs[upd]
            bestw[upd] = w[upd]
    best[best[:, 0] < 0] *= -1
    return best


def so3_halton_fz(n: int, skip: int = 1) -> np.ndarray:
    """n quasi-uniform orientations in the cubic fundamental zone: the Halton
    points (bases 2, 3, 5) from index `skip` on, through Shoemake's
    volume-preserving map [0,1)^3 -> SO(3), reduced to the fundamental zone.
    A fast stand-in at the size of the paper's 1-degree set (n = 618324,
    Section 2.3) where greedy thinning (so3_grid) is too slow; no minimum
    separation is enforced.  float64 [n, 4] (w, x, y, z), w >= 0."""
    idx = np.arange(skip, skip + n)
    u1, u2, u3 = _halton_idx(idx, 2), _halton_idx(idx, 3), _halton_idx(idx, 5)
    q = np.stack([np.sqrt(u1) * np.cos(2 * np.pi * u3),
                  np.sqrt(1 - u1) * np.sin(2 * np.pi * u2),
                  np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                  np.sqrt(u1) * np.sin(2 * np.pi * u3)], axis=1)
    return np.ascontiguousarray(_reduce_cubic_fz(q))


def _halton_idx(idx: np.ndarray, base: int) -> np.ndarray:
    """Radical inverse of the integers idx in `base` (vectorised)."""
    out = np.zeros(idx.shape[0])
    f = 1.0 / base
    i = idx.astype(np.int64).copy()
    while np.any(i > 0):
        out += f * (i % base)
        i //= base
        f /= base
    return out


def _matrix_to_quat(m) -> np.ndarray:
    m = np.asarray(m, float)
    tr = np.trace(m)
    if tr > 0:
        s = math.sqrt(tr + 1.0) * 2
        q = [0.25 * s, (m[2, 1] - m[1, 2]) / s, (m[0, 2] - m[2, 0]) / s, (m[1, 0] - m[0, 1]) / s]
    elif m[0, 0] > m[1, 1] and m[0, 0] > m[2, 2]:
        s = math.sqrt(1.0 + m[0, 0] - m[1, 1] - m[2, 2]) * 2
        q = [(m[2, 1] - m[1, 2]) / s, 0.25 * s, (m[0, 1] + m[1, 0]) / s, (m[0, 2] + m[2, 0]) / s]
    elif m[1, 1] > m[2, 2]:
        s = math.sqrt(1.0 + m[1, 1] - m[0, 0] - m[2, 2]) * 2
        q = [(m[0, 2] - m[2, 0]) / s, (m[0, 1] + m[1, 0]) / s, 0.25 * s, (m[1, 2] + m[2, 1]) / s]
    else:
        s = math.sqrt(1.0 + m[2, 2] - m[0, 0] - m[1, 1]) * 2
        q = [(m[1, 0] - m[0, 1]) / s, (m[0, 2] + m[2, 0]) / s, (m[1, 2] + m[2, 1]) / s, 0.25 * s]
    q = np.array(q)
    q /= np.linalg.norm(q)
    if q[0] < 0:
        q = -q
    return q


matrix_to_quat = _matrix_to_quat


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    """One synthetic reconstruction plus the ROI list and direction set."""
    name: str
    xyz: np.ndarray            # float32 [N, 3] absolute positions (nm)
    types: np.ndarray          # uint8 [N]
    centres: np.ndarray        # float64 [N_roi, 3]
    radii: np.ndarray          # float64 [N_roi]
    dirs: np.ndarray           # float32 [N_v, 3]
    m: int                     # 2**m histogram bins
    d_spacing: tuple           # (d_min, d_max) nm of the signature band
    truth: dict = field(default_factory=dict)


def _lattice_dataset(rng, kind, a, lo, hi, eta, sigma, rot):
    xyz, t = lattice_box(kind, a, lo, hi, rot=rot)
    keep = keep_fraction(rng, xyz.shape[0], eta)
    xyz, t = xyz[keep], t[keep]
    xyz = displace(rng, xyz, sigma)
    return np.ascontiguousarray(xyz.astype(np.float32)), np.ascontiguousarray(t)


def band_spacing(d_hkl: float, rel: float = 0.10):
    """(d_min, d_max) = d_hkl (1 -/+ rel): the paper's Al {200} interval
    1.823-2.230 Angstrom is 2.025 Angstrom -/+ 10 % (supplement, Al bicrystal)."""
    return (d_hkl * (1 - rel), d_hkl * (1 + rel))


def tiny_fcc(seed: int = SEED_BASE + 1, n_roi: int = 16, level: int = 5) -> Workload:
    """Perfect f.c.c. a = 0.404 nm, random orientation, 50 % kept, isotropic
    sigma = 0.03 nm, 8 nm box, 16 ROIs of R = 1.0 nm at random interior
    centres, icosphere level 5 (10242 directions), 2**8 bins."""
    rng = np.random.default_rng(seed)
    q = random_quaternions(rng, 1)[0]
    lo, hi = np.zeros(3), np.full(3, 8.0)
    xyz, t = _lattice_dataset(rng, "fcc", 0.404, lo, hi, 0.5, (0.03, 0.03, 0.03), quat_to_matrix(q))
    centres = roi_random(rng, n_roi, lo, hi, 1.0 + 0.2)
    return Workload("fcc-tiny-16roi-L5-m8", xyz, t, centres, np.full(n_roi, 1.0),
                    icosphere(level), 8, band_spacing(0.404 / 2), {"quat": q, "lattice": "fcc", "a": 0.404})


def single_crystal_bcc(seed: int = SEED_BASE + 2, grid=(16, 16, 32), level: int = 6,
                       box=(40.0, 40.0, 80.0)) -> Workload:
    """b.c.c. a = 0.287 nm in a 40 x 40 x 80 nm box, 40 % kept, sigma_xy = 0.05,
    sigma_z = 0.02 nm, random orientation; 8192 ROIs of R = 2 nm on a 1 nm grid
    centred in the box; icosphere level 6 (40962 directions); 2**10 bins;
    signature band {110} +/- 10 %."""
    rng = np.random.default_rng(seed)
    q = random_quaternions(rng, 1)[0]
    lo, hi = np.zeros(3), np.asarray(box, float)
    xyz, t = _lattice_dataset(rng, "bcc", 0.287, lo, hi, 0.4, (0.05, 0.05, 0.02), quat_to_matrix(q))
    centres = roi_grid(grid, 1.0, (lo + hi) / 2)
    n = centres.shape[0]
    return Workload(f"bcc-{box[0]:.0f}x{box[1]:.0f}x{box[2]:.0f}nm-{n}roi-R2-L{level}-m10",
                    xyz, t, centres, np.full(n, 2.0), icosphere(level), 10,
                    band_spacing(0.287 / math.sqrt(2)), {"quat": q, "lattice": "bcc", "a": 0.287})


def perfect_crystal_roi(kind: str, a: float, R: float, rot=None, types_keep=None):
    """Atoms of a perfect crystal within a sphere of radius R around a lattice
    site at the origin (float32 centred coordinates).  Used for the paper's
    verification experiment (Section 3.1, Fig. 2)."""
    L = R + 2 * a
    xyz, t = lattice_box(kind, a, (-L, -L, -L), (L, L, L), rot=rot, origin=np.zeros(3))
    if types_keep is not None:
        sel = np.isin(t, np.asarray(types_keep))
        xyz, t = xyz[sel], t[sel]
    return np.ascontiguousarray(xyz.astype(np.float32)), t


def polycrystal(seed: int = SEED_BASE + 3, box=(60.0, 60.0, 120.0), n_grains: int = 200, n_roi: int = 100000,
                r_range=(1.0, 2.5), a_matrix: float = 0.405, a_prec: float = 0.410, prec_vol: float = 0.05,
                prec_r=(2.0, 5.0), eta: float = 0.5, sigma: float = 0.04, level: int = 6, m: int = 10) -> Workload:
    """Poisson-Voronoi polycrystal (Section 3.3): `n_grains` f.c.c. Al grains
    (a = 0.405 nm) with uniformly random orientations, spherical L1_2 Al3Sc
    precipitates (a = 0.410 nm, Sc on the cube corners = type 1, coherent with
    their host grain, never overlapping) filling `prec_vol` of the volume, `eta` kept, isotropic
    sigma.  ROIs at random interior centres with radii uniform in r_range
    (uneven atom counts); the signature band is {200} +/- 10 % per ROI."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    lo, hi = np.zeros(3), np.asarray(box, float)
    seeds = lo + rng.random((n_grains, 3)) * (hi - lo)
    quats = random_quaternions(rng, n_grains)
    tree = cKDTree(seeds)
    # grain bounding boxes from a 1 nm voxel sampling (+ margin)
    g = [np.arange(0.5, b, 1.0) for b in hi]
    vox = np.stack(np.meshgrid(*g, indexing="ij"), -1).reshape(-1, 3)
    _, owner = tree.query(vox, workers=-1)
    parts_xyz, parts_t = [], []
    for k in range(n_grains):
        sel = vox[owner == k]
        if sel.shape[0] == 0:
            continue
        blo = np.maximum(sel.min(0) - 1.5, lo)
        bhi = np.minimum(sel.max(0) + 1.5, hi)
        xyz, t = lattice_box("fcc", a_matrix, blo, bhi, rot=quat_to_matrix(quats[k]), origin=seeds[k])
        keep = keep_fraction(rng, xyz.shape[0], eta)
        xyz, t = xyz[keep], t[keep]
        _, o = tree.query(xyz, workers=-1)
        parts_xyz.append(xyz[o == k])
        parts_t.append(t[o == k])
    xyz = np.concatenate(parts_xyz)
    types = np.concatenate(parts_t)
    # precipitates: replace the matrix inside each sphere by the L1_2 lattice
    target = prec_vol * float(np.prod(hi - lo))
    vol = 0.0
    spheres = []
    while vol < target:
        r = rng.uniform(*prec_r)
        c = lo + r + rng.random(3) * (hi - lo - 2 * r)
        if any(np.linalg.norm(c - c2) < r + r2 + a_prec for c2, r2 in spheres):
            continue                    # precipitates do not overlap
        spheres.append((c, r))
        vol += 4.0 / 3.0 * math.pi * r ** 3
    inside = np.zeros(xyz.shape[0], bool)
    ptree = cKDTree(xyz)
    add_xyz, add_t = [], []
    for c, r in spheres:
        idx = ptree.query_ball_point(c, r)
        inside[idx] = True
        _, host = tree.query(c)
        pxyz, pt = lattice_box("l12", a_prec, c - r - a_prec, c + r + a_prec, rot=quat_to_matrix(quats[host]), origin=c)
        sel = np.linalg.norm(pxyz - c, axis=1) <= r
        pxyz, pt = pxyz[sel], pt[sel]
        keep = keep_fraction(rng, pxyz.shape[0], eta)
        add_xyz.append(pxyz[keep])
        add_t.append(pt[keep])
    xyz = np.concatenate([xyz[~inside]] + add_xyz)
    types = np.concatenate([types[~inside]] + add_t)
    xyz = displace(rng, xyz, (sigma, sigma, sigma))
    radii = rng.uniform(r_range[0], r_range[1], n_roi)
    centres = lo + radii[:, None] + rng.random((n_roi, 3)) * (hi - lo - 2 * radii[:, None])
    name = f"polycrystal-{box[0]:.0f}x{box[1]:.0f}x{box[2]:.0f}nm-{n_grains}grains-{n_roi}roi-R{r_range[0]}-{r_range[1]}-L{level}-m{m}"
    return Workload(name, np.ascontiguousarray(xyz.astype(np.float32)), np.ascontiguousarray(types.astype(np.uint8)),
                    np.ascontiguousarray(centres), np.ascontiguousarray(radii), icosphere(level), m,
                    band_spacing(a_matrix / 2), {"grain_seeds": seeds, "grain_quats": quats, "spheres": spheres,
                                                 "lattice": "fcc", "a": a_matrix})
