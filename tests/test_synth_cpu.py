"""The seeded synthetic inputs match the recipe the measurements are quoted
on: sizes, densities, noise, ROI layout and direction and orientation sets
(the b.c.c. single crystal of the timed step, the small f.c.c. parity case,
a reduced polycrystal, the geodesic spheres and the orientation sets), and
the same seed gives the same data.
"""
import numpy as np
from scipy.spatial import cKDTree

import synth


def test_icosphere_counts_and_unit_norm():
    for level, n in [(0, 12), (1, 42), (4, 2562), (5, 10242), (6, 40962)]:
        u = synth.icosphere(level)
        assert u.shape == (n, 3) and u.dtype == np.float32
        assert np.abs(np.linalg.norm(u.astype(np.float64), axis=1) - 1).max() < 1e-6
    # nearest-neighbour spacing at level 6 is about 1.1 degrees, fairly uniform
    u = synth.icosphere(6).astype(np.float64)
    d, _ = cKDTree(u).query(u, k=2)
    ang = np.degrees(2 * np.arcsin(d[:, 1] / 2))
    assert 0.9 < np.median(ang) < 1.3 and ang.max() / ang.min() < 1.6


def test_single_crystal_bcc_recipe():
    w = synth.single_crystal_bcc()
    assert w.centres.shape == (8192, 3) and np.all(w.radii == 2.0) and w.m == 10
    assert w.dirs.shape == (40962, 3)
    # 40 x 40 x 80 nm of b.c.c. a = 0.287 nm at 40 % detection: 2 atoms per cell
    expect = 0.4 * 2 * 40 * 40 * 80 / 0.287 ** 3
    assert abs(w.xyz.shape[0] / expect - 1) < 0.01
    assert np.all(w.xyz.min(0) > -0.5) and np.all(w.xyz.max(0) < np.array([40.5, 40.5, 80.5]))
    # ROIs on a 16 x 16 x 32 grid of 1 nm pitch centred in the box
    c = w.centres
    assert np.allclose(np.sort(np.unique(c[:, 0])), 20 - 7.5 + np.arange(16))
    assert np.allclose(np.sort(np.unique(c[:, 2])), 40 - 15.5 + np.arange(32))
    # about 1134 atoms per ROI of R = 2 nm
    tree = cKDTree(w.xyz.astype(np.float64))
    n = [len(tree.query_ball_point(c[i], 2.0)) for i in range(0, 8192, 97)]
    assert 1100 < np.mean(n) < 1170
    # band {110} +/- 10 %
    assert np.allclose(w.d_spacing, (0.9 * 0.287 / np.sqrt(2), 1.1 * 0.287 / np.sqrt(2)))
    # seeded: a second call gives the same atoms
    w2 = synth.single_crystal_bcc()
    assert np.array_equal(w.xyz[::1000], w2.xyz[::1000]) and np.array_equal(w.truth["quat"], w2.truth["quat"])


def test_tiny_fcc_recipe():
    w = synth.tiny_fcc()
    assert w.centres.shape == (16, 3) and np.all(w.radii == 1.0) and w.m == 8 and w.dirs.shape == (10242, 3)
    expect = 0.5 * 4 * 8 ** 3 / 0.404 ** 3
    assert abs(w.xyz.shape[0] / expect - 1) < 0.03
    tree = cKDTree(w.xyz.astype(np.float64))
    n = [len(tree.query_ball_point(x, 1.0)) for x in w.centres]
    assert 100 < np.mean(n) < 160


def test_reduced_polycrystal_recipe():
    w = synth.polycrystal(box=(24.0, 24.0, 48.0), n_grains=16, n_roi=3000)
    assert w.centres.shape == (3000, 3) and w.m == 10
    assert np.all((w.radii >= 1.0) & (w.radii <= 2.5))
    assert set(np.unique(w.types)) <= {0, 1} and (w.types == 1).any()
    tree = cKDTree(w.xyz.astype(np.float64))
    n = np.array([len(tree.query_ball_point(w.centres[i], w.radii[i])) for i in range(0, 3000, 20)])
    assert n.min() >= 50 and n.max() <= 2300 and 500 < n.mean() < 1100   # uneven atom counts


def test_orientation_sets_in_the_cubic_fundamental_zone():
    rot = synth.cubic_rotation_matrices()
    sym = np.array([synth._matrix_to_quat(m) for m in rot])

    def angle_deg(q):
        return np.degrees(2 * np.arccos(np.clip(np.abs(q[:, 0]), 0, 1)))

    for Q in [synth.so3_grid(5.0), synth.so3_halton_fz(5000)]:
        assert np.abs(np.linalg.norm(Q, axis=1) - 1).max() < 1e-12
        # each member has the smallest rotation angle among its 24 equivalents
        a0 = angle_deg(Q)
        for s in sym:
            w = s[0] * Q[:, 0] - s[1] * Q[:, 1] - s[2] * Q[:, 2] - s[3] * Q[:, 3]
            assert np.all(a0 <= np.degrees(2 * np.arccos(np.clip(np.abs(w), 0, 1))) + 1e-9)
        assert a0.max() <= 62.8 + 1e-6
    assert synth.so3_grid(5.0).shape[0] == 3419
