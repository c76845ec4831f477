"""GPU parity of the general signature paths against the FP64 oracle:

  - 2^11 and 2^12 bins (Section 2.2 gives m in [8, 12]): the kernels build
    each histogram in chunks of 1024 bins; histograms bit-exact on both paths,
    signatures within 1e-3 (FP32) and 5e-3 (tensor cores);
  - ROIs of 2049, about 1e4 and about 7e4 atoms: the tensor-core kernel
    contracts blocks of at most 2048 atoms (every count exact in fp16), the
    FP32 kernel accumulates its spectrum over blocks of at most 65535 atoms;
    atom counts and histograms bit-exact, signatures within tolerance;
  - antipodal pairs: with the direction set closed under negation the
    tensor-core path projects one direction of a pair; its results equal those
    of projecting every direction (APTIDX_DIRECT) within FP32 rounding, the
    pair members carry the same value, and a ROI with atoms whose bin product
    is an exact integer (where the mirror image of the histogram is not the
    histogram of -u) still matches the oracle direction by direction.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2009_00735_gb300 as apt

from test_gpu_plain import TOL_PLAIN, gpu_signatures, make_ctx, roi_error, torch_cuda  # noqa: F401

pytestmark = pytest.mark.gpu

TOL_TC = 5e-3
PLAIN, TC = apt.APTIDX_PATH_PLAIN_FP32, apt.APTIDX_PATH_TC_FP16
PATHS = [(PLAIN, TOL_PLAIN), (TC, TOL_TC)]


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_fcc()


@pytest.mark.parametrize("m", [11, 12])
@pytest.mark.parametrize("path,tol", PATHS)
def test_many_bins(torch_cuda, tiny, m, path, tol):
    dirs = np.ascontiguousarray(tiny.dirs[:1500])
    ctx, band, mm, d = make_ctx(torch_cuda, tiny, dirs=dirs, m=m)
    assert mm == m
    nroi, nv = tiny.centres.shape[0], d.shape[0]
    for roi in (0, 9):
        h = np.empty((nv, 1 << m), np.uint16)
        apt.aptidx_get_histograms(ctx.handle, roi, path, h)
        _, xc = oracle.gather(tiny.xyz, tiny.centres[roi], tiny.radii[roi])
        assert np.array_equal(h.astype(np.int64), oracle.histograms(xc, d, m, tiny.radii[roi]).astype(np.int64))
    S, A, N = gpu_signatures(torch_cuda, ctx, nroi, nv, path=path)
    So, Ao, No = oracle.signatures(tiny.xyz, tiny.centres, tiny.radii, band[0], band[1], d, m)
    assert np.array_equal(N, No)
    assert roi_error(S, So).max() <= tol
    assert (A == Ao).mean() > 0.99
    # a wide band: several frequency-group batches (tensor cores) or rounds (FP32)
    apt.aptidx_set_binning(ctx.handle, m, 5, 100)
    apt.aptidx_set_rois(ctx.handle, tiny.centres[:4], tiny.radii[:4])
    S, _, _ = gpu_signatures(torch_cuda, ctx, 4, nv, path=path)
    So, _, _ = oracle.signatures(tiny.xyz, tiny.centres[:4], tiny.radii[:4], 5, 100, d, m)
    assert roi_error(S, So).max() <= tol
    ctx.close()


def big_rois():
    """A noisy f.c.c. block and three ROIs whose radii fall between the
    distances of consecutive atoms, so that they hold exactly 2049, 10000 and
    70000 atoms."""
    rng = np.random.default_rng(21)
    q = synth.random_quaternions(rng, 1)[0]
    xyz, t = synth.lattice_box("fcc", 0.404, (-7.4, -7.4, -7.4), (7.4, 7.4, 7.4), rot=synth.quat_to_matrix(q),
                               origin=np.zeros(3))
    xyz = (xyz.astype(np.float64) + rng.normal(0.0, 0.03, xyz.shape)).astype(np.float32)
    centres = np.array([[0.11, -0.07, 0.05], [-0.2, 0.13, 0.31], [0.02, 0.04, -0.06]])
    radii = []
    for c, n in zip(centres, (2049, 10000, 70000)):
        d = np.sort(np.sqrt(((xyz.astype(np.float64) - c) ** 2).sum(axis=1)))
        radii.append(0.5 * (d[n - 1] + d[n]))
    return np.ascontiguousarray(xyz), centres, np.array(radii)


@pytest.mark.parametrize("path,tol", PATHS)
def test_large_rois(torch_cuda, path, tol):
    torch = torch_cuda
    xyz, centres, radii = big_rois()
    dirs = np.ascontiguousarray(synth.icosphere(2))    # 162 directions, closed under negation
    m = 10
    band = oracle.band_for_spacing(0.9 * 0.202, 1.1 * 0.202, float(radii[0]), m)
    ctx = apt.Context(0)
    h = ctx.handle
    apt.aptidx_load_positions(h, torch.from_numpy(xyz).cuda())
    apt.aptidx_set_directions(h, torch.from_numpy(dirs).cuda())
    apt.aptidx_set_binning(h, m, band[0], band[1])
    apt.aptidx_set_rois(h, centres, radii)
    nv = dirs.shape[0]
    S, A, N = gpu_signatures(torch, ctx, 3, nv, path=path)
    assert list(N) == [2049, 10000, 70000]
    So, Ao, No = oracle.signatures(xyz, centres, radii, band[0], band[1], dirs, m)
    assert np.array_equal(N, No)
    assert roi_error(S, So).max() <= tol
    for roi in range(3):
        hg = np.empty((nv, 1 << m), np.uint16)
        apt.aptidx_get_histograms(h, roi, path, hg)
        _, xc = oracle.gather(xyz, centres[roi], radii[roi])
        ho = oracle.histograms(xc, dirs, m, radii[roi])
        assert ho.max() < 65536
        assert np.array_equal(hg.astype(np.int64), ho.astype(np.int64))
    ctx.close()


def test_antipodal_pairs_match_direct(torch_cuda, tiny):
    ctx, band, m, d = make_ctx(torch_cuda, tiny)
    nroi, nv = tiny.centres.shape[0], d.shape[0]
    S, A, N = gpu_signatures(torch_cuda, ctx, nroi, nv, path=TC)
    Sd, Ad, _ = gpu_signatures(torch_cuda, ctx, nroi, nv, path=TC, flags=apt.APTIDX_DIRECT)
    assert roi_error(S, Sd).max() <= 1e-5
    assert (A == Ad).mean() > 0.999
    So, _, _ = oracle.signatures(tiny.xyz, tiny.centres, tiny.radii, band[0], band[1], d, m)
    assert roi_error(S, So).max() <= TOL_TC and roi_error(Sd, So).max() <= TOL_TC
    # every node of the icosphere has its exact antipode; for noisy atoms no
    # bin product is an integer, so the pair carries one value
    key = {tuple((d[i] + np.float32(0)).tolist()): i for i in range(nv)}
    j = np.array([key[tuple((-d[i] + np.float32(0)).tolist())] for i in range(nv)])
    assert np.array_equal(S, S[:, j]) and np.array_equal(A, A[:, j])
    ctx.close()


@pytest.mark.parametrize("R", [1.0, 0.97])
def test_antipodal_pairs_with_integer_products(torch_cuda, R):
    """Atoms on the plane x = 0 through the ROI centre project to exactly 0
    along (1, 0, 0), an integer bin product: the histogram along (-1, 0, 0) is
    then not the mirror image of the one along (1, 0, 0), and the kernel must
    project (-1, 0, 0) itself.  Checked against the oracle direction by
    direction, with and without pairing.  R = 1 (scale 127 = 127 x 2^0: atoms
    at |s| = 1 could also give integers) takes the exact count of
    non-integer products; R = 0.97 (a scale with a full significand: only s = 0
    can) takes the zero-product check."""
    torch = torch_cuda
    rng = np.random.default_rng(5)
    yz = (rng.random((40, 2)) - 0.5) * 1.2
    on_plane = np.column_stack([np.zeros(40), yz])
    off_plane = np.column_stack([np.full(25, 0.3), (rng.random((25, 2)) - 0.5) * 1.2])
    rest = (rng.random((300, 3)) - 0.5) * 1.6
    # an atom at |x| = 1 keeps the R = 1 case on the exact count (|s| = 1 gives an integer there)
    xyz = np.ascontiguousarray(np.concatenate([on_plane, off_plane, rest, [[0.0, 0.0, 1.0]]]).astype(np.float32))
    u = rng.standard_normal((40, 3))
    u = u / np.linalg.norm(u, axis=1, keepdims=True)
    half = np.concatenate([[[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]], u]).astype(np.float32)
    dirs = np.ascontiguousarray(np.concatenate([half, -half]))
    m, band = 8, (3, 9)
    ctx = apt.Context(0)
    h = ctx.handle
    apt.aptidx_load_positions(h, torch.from_numpy(xyz).cuda())
    apt.aptidx_set_directions(h, torch.from_numpy(dirs).cuda())
    apt.aptidx_set_binning(h, m, band[0], band[1])
    apt.aptidx_set_rois(h, np.zeros((1, 3)), np.array([R]))
    nv = dirs.shape[0]
    So, Ao, _ = oracle.signatures(xyz, np.zeros((1, 3)), np.array([R]), band[0], band[1], dirs, m)
    # the mirror image would differ along -x: the oracle's -x signature is not the +x one
    assert So[0, 0] != So[0, 42]
    for flags in (0, apt.APTIDX_DIRECT):
        S, A, _ = gpu_signatures(torch, ctx, 1, nv, path=TC, flags=flags)
        assert roi_error(S, So).max() <= TOL_TC
        assert np.abs(S[0] - So[0]).max() <= 1e-5 * So[0].max()
    ctx.close()


@pytest.mark.parametrize("m,band", [(8, (3, 100)), (9, (4, 60)), (10, (2, 126))])
def test_wide_band_stream(torch_cuda, tiny, m, band):
    """Bands wider than one batch of twiddles in shared memory: the tensor-core
    kernel streams the twiddles of all the band's frequency groups through two
    stages per 64-bin block and contracts every group in one MMA per K step
    (25, 15 and 32 groups: odd counts take a zero group of padding)."""
    dirs = np.ascontiguousarray(tiny.dirs[:1200])
    ctx, band, mm, d = make_ctx(torch_cuda, tiny, band=band, dirs=dirs, m=m)
    nroi, nv = tiny.centres.shape[0], d.shape[0]
    S, A, N = gpu_signatures(torch_cuda, ctx, nroi, nv, path=TC)
    Sp, Ap, _ = gpu_signatures(torch_cuda, ctx, nroi, nv, path=PLAIN)
    So, Ao, No = oracle.signatures(tiny.xyz, tiny.centres, tiny.radii, band[0], band[1], d, m)
    assert np.array_equal(N, No)
    assert roi_error(S, So).max() <= TOL_TC
    assert roi_error(Sp, So).max() <= TOL_PLAIN
    assert np.all((A >= band[0]) & (A <= band[1]))
    assert (A == Ao).mean() > 0.99
    ctx.close()


def test_wide_band_large_rois(torch_cuda):
    """The streamed wide-band contraction over several 2048-atom blocks of one
    ROI (2049, 10000 and 70000 atoms), band k = 8..128."""
    torch = torch_cuda
    xyz, centres, radii = big_rois()
    dirs = np.ascontiguousarray(synth.icosphere(2))
    m, band = 10, (8, 128)
    ctx = apt.Context(0)
    h = ctx.handle
    apt.aptidx_load_positions(h, torch.from_numpy(xyz).cuda())
    apt.aptidx_set_directions(h, torch.from_numpy(dirs).cuda())
    apt.aptidx_set_binning(h, m, band[0], band[1])
    apt.aptidx_set_rois(h, centres, radii)
    S, A, N = gpu_signatures(torch, ctx, 3, dirs.shape[0], path=TC)
    So, Ao, No = oracle.signatures(xyz, centres, radii, band[0], band[1], dirs, m)
    assert np.array_equal(N, No)
    assert roi_error(S, So).max() <= TOL_TC
    ctx.close()


def test_probe_l2(torch_cuda):
    """The L2 read-bandwidth probe returns a plausible rate and refuses sizes
    outside [1 MiB, 96 MiB] or not a multiple of 16."""
    ctx = apt.Context(0)
    g = apt.aptidx_probe_l2(ctx.handle, 8 << 20, 20)
    assert 1e3 < g < 1e5, g
    for nbytes in (1 << 19, (96 << 20) + 16, (8 << 20) + 8):
        with pytest.raises(apt.AptidxError) as ei:
            apt.aptidx_probe_l2(ctx.handle, nbytes, 10)
        assert ei.value.code == apt.APTIDX_E_INVALID_ARG
    ctx.close()


def test_probe_smem_atomics(torch_cuda):
    """The shared-memory atomic probe counts every increment (the kernel checks
    its array's sum), returns a rate between 0.05 and 4 32-lane atomics per SM
    and cycle, and refuses thread counts that are not a multiple of 32 in
    [32, 1024]."""
    ctx = apt.Context(0)
    incr, per_cycle = apt.aptidx_probe_smem_atomics(ctx.handle, 512, 256)
    assert 0.05 < per_cycle < 4.0, per_cycle
    assert 1e10 < incr < 1e14, incr
    for threads in (16, 1056, 100):
        with pytest.raises(apt.AptidxError) as ei:
            apt.aptidx_probe_smem_atomics(ctx.handle, threads, 10)
        assert ei.value.code == apt.APTIDX_E_INVALID_ARG
    ctx.close()


@pytest.mark.parametrize("path", [PLAIN, TC])
def test_reload_reuses_blocks(torch_cuda, tiny, path):
    """A reload keeps the ROI and cell-grid blocks it releases for the next set
    of the same sizes.  Loading set A, then a set B of other sizes (half the
    atoms, every other ROI), then A again gives A's signatures, argmax bins and
    atom counts bit for bit, and B's match a context that only ever saw B."""
    torch = torch_cuda
    ctx, band, m, d = make_ctx(torch, tiny)
    h = ctx.handle
    nv = d.shape[0]
    nroi = tiny.centres.shape[0]
    S1, A1, N1 = gpu_signatures(torch, ctx, nroi, nv, path=path)
    xyz_b = np.ascontiguousarray(tiny.xyz[::2])
    cen_b = np.ascontiguousarray(tiny.centres[::2])
    rad_b = np.ascontiguousarray(tiny.radii[::2])
    for _ in range(2):
        apt.aptidx_load_positions(h, torch.from_numpy(xyz_b).cuda())
        apt.aptidx_set_rois(h, torch.from_numpy(cen_b).cuda(), torch.from_numpy(rad_b).cuda())
        Sb, Ab, Nb = gpu_signatures(torch, ctx, cen_b.shape[0], nv, path=path)
        apt.aptidx_load_positions(h, torch.from_numpy(tiny.xyz).cuda())
        apt.aptidx_set_rois(h, torch.from_numpy(tiny.centres).cuda(), torch.from_numpy(tiny.radii).cuda())
        S2, A2, N2 = gpu_signatures(torch, ctx, nroi, nv, path=path)
        assert np.array_equal(N1, N2)
        assert np.array_equal(A1, A2)
        assert np.array_equal(S1.view(np.uint32), S2.view(np.uint32))
    ctx.close()
    fresh = apt.Context(0)
    hf = fresh.handle
    apt.aptidx_load_positions(hf, torch.from_numpy(xyz_b).cuda())
    apt.aptidx_set_directions(hf, torch.from_numpy(np.ascontiguousarray(d)).cuda())
    apt.aptidx_set_binning(hf, m, band[0], band[1])
    apt.aptidx_set_rois(hf, torch.from_numpy(cen_b).cuda(), torch.from_numpy(rad_b).cuda())
    Sf, Af, Nf = gpu_signatures(torch, fresh, cen_b.shape[0], nv, path=path)
    assert np.array_equal(Nb, Nf)
    assert np.array_equal(Ab, Af)
    assert np.array_equal(Sb.view(np.uint32), Sf.view(np.uint32))
    fresh.close()
