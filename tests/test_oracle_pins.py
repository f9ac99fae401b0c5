"""Pins for the CPU oracle: each test checks an oracle function against
something other than itself -- published vectors, a library routine, a closed
form, an invariant or a brute-force definition -- so that a dropped term, a
wrong sign or index, or a transposed operand fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import pfsynth
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ Philox

def test_philox_known_answers(orc):
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v, 16) for v in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = orc.philox(r[0:4], r[4:6])
        assert [int(v) for v in out] == r[6:10]


def test_philox_counter_sensitivity(orc):
    base = orc.philox([1, 2, 3, 4], [5, 6])
    for w in range(4):
        c = [1, 2, 3, 4]
        c[w] ^= 1
        assert not np.array_equal(orc.philox(c, [5, 6]), base)
    # uniformity of the 24-bit draws used by the filter
    u = np.array([orc.philox([i, 0, 1, 0], [0, 0])[0] >> 8 for i in range(4000)]) / 2**24
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1 / 12) < 0.01


# ------------------------------------------------------------ sin / cos

def test_sin_cos_against_libm(orc):
    xs = np.concatenate([np.linspace(-np.pi / 2, np.pi / 2, 2001), [0.0, 1e-8, -1e-300, np.pi / 2]])
    for x in xs:
        s, c = orc.sin(x), orc.cos(x)
        assert abs(s - math.sin(x)) <= 4.5e-16
        assert abs(c - math.cos(x)) <= 4.5e-16
        assert abs(s * s + c * c - 1.0) <= 1e-15
    assert orc.sin(0.0) == 0.0 and orc.cos(0.0) == 1.0


# ------------------------------------------------------------- rotation

def _rand_poses(n, rot=np.pi / 2, tr=10.0, seed=1):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.uniform(-rot, rot, (n, 3)), rng.uniform(-tr, tr, (n, 3))], 1)


def test_rotation_matches_scipy_intrinsic_zxy(orc):
    for pose in _rand_poses(200):
        R = orc.rotation(pose.astype(np.float32))
        Rs = pfsynth.rotation_zxy(pose.astype(np.float32))
        assert np.max(np.abs(R - Rs)) < 2e-15


def test_rotation_single_axis_textbook(orc):
    th = 0.37
    c, s = math.cos(th), math.sin(th)
    Rx = orc.rotation(np.array([th, 0, 0, 0, 0, 0], np.float32))
    Ry = orc.rotation(np.array([0, th, 0, 0, 0, 0], np.float32))
    Rz = orc.rotation(np.array([0, 0, th, 0, 0, 0], np.float32))
    t32 = float(np.float32(th))
    c, s = math.cos(t32), math.sin(t32)
    np.testing.assert_allclose(Rx, [[1, 0, 0], [0, c, -s], [0, s, c]], atol=1e-15)
    np.testing.assert_allclose(Ry, [[c, 0, s], [0, 1, 0], [-s, 0, c]], atol=1e-15)
    np.testing.assert_allclose(Rz, [[c, -s, 0], [s, c, 0], [0, 0, 1]], atol=1e-15)


def test_rotation_composition_and_inverse(orc):
    for pose in _rand_poses(50, seed=3).astype(np.float32):
        R = orc.rotation(pose)
        Rz = orc.rotation(np.array([0, 0, pose[2], 0, 0, 0], np.float32))
        Rx = orc.rotation(np.array([pose[0], 0, 0, 0, 0, 0], np.float32))
        Ry = orc.rotation(np.array([0, pose[1], 0, 0, 0, 0], np.float32))
        np.testing.assert_allclose(R, Rz @ Rx @ Ry, atol=1e-15)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-15)
        assert abs(np.linalg.det(R) - 1.0) < 1e-14
        # single-axis inverse: R(theta) R(-theta) = I
        for ax in range(3):
            p, m = np.zeros(6, np.float32), np.zeros(6, np.float32)
            p[ax], m[ax] = pose[ax], -pose[ax]
            np.testing.assert_allclose(orc.rotation(p) @ orc.rotation(m), np.eye(3), atol=1e-15)


def test_pose_matrix_geometry(orc):
    sd, so, to = (37, 29, 23), np.array([1.5, -2.0, 0.25], np.float32), np.array([4.0, 3.0, -1.0], np.float32)
    td = (21, 18, 11)
    for pose in _rand_poses(20, rot=0.6, tr=5, seed=4).astype(np.float32):
        M, a = orc.pose_matrix(pose, sd, so, to)
        c = so.astype(np.float64) + (np.array(sd) - 1) / 2.0
        np.testing.assert_allclose(a, c - to, rtol=0, atol=1e-6)
        np.testing.assert_allclose(M[[3, 7, 11]], c + pose[3:] - so, atol=1e-5)
        p = bf.target_points(td)
        Mm = M.reshape(3, 4).astype(np.float64)
        q = (p - a) @ Mm[:, :3].T + Mm[:, 3]
        q_ref = bf.source_index_f64(pose, sd, so, td, to)
        assert np.max(np.abs(q - q_ref)) < 2e-4


def test_pose_matrix_geometry_with_spacing(orc):
    """Anisotropic voxels (Table 1 sizes): the matrix maps target voxels to
    source voxels through world positions, checked against scipy's rotation
    applied in world units; unit spacings give the unit-spacing matrix bit
    for bit."""
    sd, so, to = (37, 29, 23), np.array([1.5, -2.0, 0.25], np.float32), np.array([4.0, 3.0, -1.0], np.float32)
    td = (21, 18, 11)
    ss, ts = np.array([0.87, 1.08, 0.73], np.float32), np.array([1.09, 1.30, 0.92], np.float32)
    for pose in _rand_poses(20, rot=0.6, tr=5, seed=5).astype(np.float32):
        M, a = orc.pose_matrix(pose, sd, so, to, ss, ts)
        Mm = M.reshape(3, 4).astype(np.float64)
        q = (bf.target_points(td) - a) @ Mm[:, :3].T + Mm[:, 3]
        q_ref = bf.source_index_f64(pose, sd, so, td, to, ss, ts)
        assert np.max(np.abs(q - q_ref)) < 2e-4
        # the 3x3 block is R scaled column-wise by s_T and row-wise by 1/s_S
        R = pfsynth.rotation_zxy(pose.astype(np.float64))
        np.testing.assert_allclose(Mm[:, :3], R * ts[None, :].astype(np.float64) / ss[:, None], atol=1e-6)
        M1, a1 = orc.pose_matrix(pose, sd, so, to, (1, 1, 1), (1, 1, 1))
        M0, a0 = orc.pose_matrix(pose, sd, so, to)
        assert np.array_equal(M1, M0) and np.array_equal(a1, a0)


# --------------------------------------------------------- measure, mask

def _exact_cases(seed, n=12):
    rng = np.random.default_rng(seed)
    perms = bf.signed_permutations()
    for i in range(n):
        P = perms[rng.integers(len(perms))]
        b = rng.integers(-6, 20, 3)
        yield P, b


def test_mask_counts_integer_maps_exact(orc):
    src = pfsynth.random_mask(11, (19, 14, 12), 0.4)
    tgt = pfsynth.random_mask(12, (13, 17, 15), 0.4)
    a0 = np.zeros(3, np.float32)
    for P, b in _exact_cases(5, 24):
        got = orc.measure_mask(src, tgt, bf.exact_matrix(P, b), a0)[0]
        want = bf.integer_map_counts(src, tgt, P, b)
        assert got.tolist() == want.tolist()


def test_mask_counts_half_voxel_ties_round_up(orc):
    # q = P p + b + h with h_d in {0, 1/2}: every coordinate with h_d = 1/2 sits
    # exactly on a tie of the nearest-neighbour rounding; the reading takes
    # voxel floor(q + 1/2), i.e. rounds the tie up, which is the integer map
    # with b + 1 on those axes (round-half-even or half-down would differ)
    src = pfsynth.random_mask(13, (17, 15, 13), 0.45)
    tgt = pfsynth.random_mask(14, (14, 16, 12), 0.45)
    a0 = np.zeros(3, np.float32)
    rng = np.random.default_rng(8)
    for P, b in _exact_cases(7, 24):
        h = rng.integers(0, 2, 3)
        if not h.any():
            h[rng.integers(3)] = 1
        M = bf.exact_matrix(P, b)
        M[[3, 7, 11]] += 0.5 * h
        got = orc.measure_mask(src, tgt, M, a0)[0]
        want = bf.integer_map_counts(src, tgt, P, b + h)
        assert got.tolist() == want.tolist(), (P.tolist(), b.tolist(), h.tolist())


def test_mask_identity_gives_dice_one(orc):
    m = pfsynth.random_mask(3, (16, 15, 14), 0.35)
    sd = (16, 15, 14)
    M, a = orc.pose_matrix(np.zeros(6, np.float32), sd, np.zeros(3, np.float32), np.zeros(3, np.float32))
    n, A, B, C = (int(v) for v in orc.measure_mask(m, m, M, a)[0])
    assert n == m.size and A == B == C == int(m.sum())
    assert orc.dice_from_counts(n, A, C, int(m.sum())) == 1.0
    assert orc.score("mask_ncc", np.array([0] * 8 + [n, A, B, C], np.uint64)) == 1.0


def test_mask_counts_general_pose_vs_bruteforce(orc):
    src = pfsynth.random_mask(21, (24, 22, 20), 0.4)
    tgt = pfsynth.random_mask(22, (20, 18, 17), 0.4)
    so, to = np.zeros(3, np.float32), np.array([2.0, 1.0, 3.0], np.float32)
    for pose in _rand_poses(10, rot=0.5, tr=4, seed=9).astype(np.float32):
        M, a = orc.pose_matrix(pose, src.shape[::-1], so, to)
        got = orc.measure_mask(src, tgt, M, a)[0].astype(np.int64)
        q = bf.source_index_f64(pose, src.shape[::-1], so, tgt.shape[::-1], to)
        want = bf.nn_counts_f64(src, tgt, q)
        # fp32 vs fp64 coordinates can only flip voxels sitting on a rounding boundary
        assert np.all(np.abs(got - want) <= 3), (got, want)


def test_dice_symmetry_and_definition(orc):
    a = pfsynth.random_mask(31, (14, 13, 12), 0.3)
    b = pfsynth.random_mask(32, (14, 13, 12), 0.3)
    M, off = orc.pose_matrix(np.zeros(6, np.float32), (14, 13, 12), np.zeros(3, np.float32),
                             np.zeros(3, np.float32))
    n1, A1, B1, C1 = (int(v) for v in orc.measure_mask(a, b, M, off)[0])
    n2, A2, B2, C2 = (int(v) for v in orc.measure_mask(b, a, M, off)[0])
    d1 = orc.dice_from_counts(n1, A1, C1, int(b.sum()))
    d2 = orc.dice_from_counts(n2, A2, C2, int(a.sum()))
    want = 2 * np.sum(a & b) / (a.sum() + b.sum())
    assert d1 == d2 and abs(d1 - want) < 1e-15


# -------------------------------------------------------- measure, image

def test_image_moments_integer_maps_exact(orc):
    src = pfsynth.random_image(41, (17, 15, 13))
    tgt = pfsynth.random_image(42, (14, 16, 11))
    a0 = np.zeros(3, np.float32)
    for P, b in _exact_cases(6, 24):
        got = orc.measure_image(src, tgt, bf.exact_matrix(P, b), a0)[0]
        want = bf.integer_map_counts(src, tgt, P, b, image=True)
        assert got.tolist() == want.tolist()


def _ramp(dims, g, c0):
    X, Y, Z = dims
    z, y, x = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    v = g[0] * x + g[1] * y + g[2] * z + c0
    assert v.min() >= 0 and v.max() <= 255
    return v.astype(np.uint8)


def test_image_moments_dyadic_shifts_exact(orc):
    # axis maps shifted by multiples of a quarter voxel: every trilinear
    # fraction is 0, 1/4, 1/2 or 3/4, so the samples and the 15-bit moments
    # are exact rationals -- an exact check of the interpolation (corner
    # order, lerp direction) that integer maps, whose fractions are all 0,
    # cannot give
    src = pfsynth.random_image(43, (13, 12, 11))
    tgt = pfsynth.random_image(44, (11, 12, 10))
    a0 = np.zeros(3, np.float32)
    rng = np.random.default_rng(12)
    cases = 0
    for P, b in _exact_cases(9, 40):
        b = rng.integers(-3, 8, 3)
        h4 = rng.integers(0, 4, 3)
        M = bf.exact_matrix(P, b)
        M[[3, 7, 11]] += 0.25 * h4
        got = orc.measure_image(src, tgt, M, a0)[0][:7]
        want = bf.dyadic_map_moments(src, tgt, P, b, h4)
        assert got.tolist() == want.tolist(), (P.tolist(), b.tolist(), h4.tolist())
        cases += int(want[0]) > 0
    assert cases >= 20   # most cases overlap


def test_image_ncc_linear_ramp_closed_form(orc):
    """Trilinear interpolation reproduces an affine field exactly, so for a
    target box wholly inside the source, NCC^2 = (u.V.h)^2 / (u.V.u h.V.h)
    with u = R^T g and V = diag((n_d^2 - 1)/12) the lattice covariance."""
    sd, td = (32, 32, 32), (16, 15, 14)
    g, h = np.array([3, 2, 1]), np.array([1, 4, 2])
    src = _ramp(sd, g, 5)
    tgt = _ramp(td, h, 7)
    so = np.zeros(3, np.float32)
    to = ((np.array(sd) - np.array(td)) / 2).astype(np.float32)
    V = (np.array(td, np.float64) ** 2 - 1) / 12.0
    for pose in _rand_poses(12, rot=0.35, tr=2.0, seed=13).astype(np.float32):
        M, a = orc.pose_matrix(pose, sd, so, to)
        mom = orc.measure_image(src, tgt, M, a)[0]
        assert int(mom[0]) == tgt.size           # whole target inside
        R = orc.rotation(pose)
        u = R.T @ g
        want = (u * V * h).sum() ** 2 / ((u * V * u).sum() * (h * V * h).sum())
        got = orc.ncc2_from_moments(mom)
        assert abs(got - want) <= 1e-5 * want, (got, want)
        got64 = orc.ncc2_f64(src, tgt, M, a)[0]
        assert abs(got64 - want) <= 2e-6 * want


def test_image_ncc_f64_vs_scipy_pearson(orc):
    src = pfsynth.random_image(51, (26, 24, 22))
    tgt = pfsynth.random_image(52, (20, 19, 18))
    so, to = np.zeros(3, np.float32), np.array([3.0, 2.0, 2.0], np.float32)
    for pose in _rand_poses(6, rot=0.4, tr=3, seed=17).astype(np.float32):
        M, a = orc.pose_matrix(pose, src.shape[::-1], so, to)
        got = orc.ncc2_f64(src, tgt, M, a)[0]
        q = bf.source_index_f64(pose, src.shape[::-1], so, tgt.shape[::-1], to)
        ok, s = bf.trilinear_f64(src, q)
        r = stats.pearsonr(s, tgt.reshape(-1)[ok].astype(np.float64)).statistic
        assert abs(got - r * r) <= 5e-5 * max(r * r, 1e-3), (got, r * r)


def test_fixed_point_ncc_within_1e5_of_fp64(orc):
    src = pfsynth.random_image(61, (30, 28, 26))
    tgt = pfsynth.random_image(62, (24, 22, 20))
    so, to = np.zeros(3, np.float32), np.array([2.0, 3.0, 1.0], np.float32)
    for pose in _rand_poses(10, rot=0.5, tr=4, seed=19).astype(np.float32):
        M, a = orc.pose_matrix(pose, src.shape[::-1], so, to)
        m = orc.measure_image(src, tgt, M, a)[0]
        fixed = orc.ncc2_from_moments(m)
        exact = orc.ncc2_f64(src, tgt, M, a)[0]
        assert abs(fixed - exact) <= 1e-5 * exact, (fixed, exact)


def test_ncc_formula_against_exact_rationals(orc):
    rng = np.random.default_rng(5)
    for _ in range(200):
        n = int(rng.integers(10, 10**7))
        s = rng.integers(0, 65281, 3)
        t = rng.integers(0, 256, 3)
        # consistent moments from a tiny synthetic sample scaled up
        sv = int(s[0]) * 128                      # samples up to 2^23 (15 fractional bits)
        S1, S2, ST = sv * n // 3, sv ** 2 * n // 2, sv * int(t[0]) * n // 4
        T1, T2 = int(t[0]) * n // 3, int(t[0]) ** 2 * n // 2
        m = [n, S1, S2 & (2**64 - 1), S2 >> 64, ST, T1, T2]
        vs, vt = n * S2 - S1 * S1, n * T2 - T1 * T1
        if vs <= 0 or vt <= 0:
            assert orc.ncc2_from_moments(m) == 0.0
            continue
        want = Fraction((n * ST - S1 * T1) ** 2, vs * vt)
        got = orc.ncc2_from_moments(m)
        assert abs(got - float(want)) <= 1e-15 * float(want)


def test_ncc_invariant_to_affine_intensity(orc):
    src = pfsynth.random_image(71, (22, 20, 18))
    tgt = pfsynth.random_image(72, (18, 16, 15)) // 3
    so, to = np.zeros(3, np.float32), np.array([1.0, 2.0, 1.0], np.float32)
    tgt2 = (tgt.astype(np.int32) * 2 + 17).astype(np.uint8)
    for pose in _rand_poses(5, rot=0.4, tr=3, seed=23).astype(np.float32):
        M, a = orc.pose_matrix(pose, src.shape[::-1], so, to)
        s1 = orc.ncc2_from_moments(orc.measure_image(src, tgt, M, a)[0])
        s2 = orc.ncc2_from_moments(orc.measure_image(src, tgt2, M, a)[0])
        assert abs(s1 - s2) <= 1e-12


def test_image_identity_ncc_one(orc):
    v = pfsynth.random_image(81, (15, 14, 13))
    M, a = orc.pose_matrix(np.zeros(6, np.float32), (15, 14, 13), np.zeros(3, np.float32),
                           np.zeros(3, np.float32))
    m = orc.measure_image(v, v, M, a)[0]
    assert int(m[0]) == v.size and int(m[1]) == 32768 * int(v.astype(np.int64).sum())
    assert abs(orc.ncc2_from_moments(m) - 1.0) < 1e-15


def test_mask_ncc_and_combined_scores_against_scipy(orc):
    # mask NCC^2 from the four counts is the squared Pearson correlation of
    # the binary samples over the overlap; the combined score is half the sum
    # of the image NCC^2 (Pearson of the image samples) and the mask Dice
    # over the whole target grid -- each computed here from exact integer-map
    # samples with scipy / numpy
    src = pfsynth.random_image(45, (15, 14, 13))
    tgt = pfsynth.random_image(46, (13, 14, 12))
    smask = pfsynth.random_mask(47, (15, 14, 13), 0.45)
    tmask = pfsynth.random_mask(48, (13, 14, 12), 0.45)
    a0 = np.zeros(3, np.float32)
    sd = np.array([15, 14, 13])
    checked = 0
    for P, b in _exact_cases(11, 30):
        b = np.random.default_rng(int(np.abs(b).sum())).integers(-2, 4, 3)
        p = bf.target_points((13, 14, 12))
        q = p @ P.T + b
        ok = np.all((q >= 0) & (q < sd), axis=1)
        if ok.sum() < 50:
            continue
        qq = q[ok]
        s_img = src[qq[:, 2], qq[:, 1], qq[:, 0]].astype(np.float64)
        t_img = tgt.reshape(-1)[ok].astype(np.float64)
        s_m = (smask[qq[:, 2], qq[:, 1], qq[:, 0]] != 0).astype(np.float64)
        t_m = (tmask.reshape(-1)[ok] != 0).astype(np.float64)
        M = bf.exact_matrix(P, b)
        mom = np.zeros(12, np.uint64)
        mom[:7] = orc.measure_image(src, tgt, M, a0)[0]
        mom[8:] = orc.measure_mask(smask, tmask, M, a0)[0]
        b_full = int((tmask != 0).sum())
        if s_m.std() > 0 and t_m.std() > 0:
            r_m = stats.pearsonr(s_m, t_m)[0]
            assert abs(orc.score("mask_ncc", mom, b_full) - r_m ** 2) < 1e-12
        r_i = stats.pearsonr(s_img, t_img)[0]
        dice = 2.0 * np.sum(s_m * t_m) / (s_m.sum() + b_full)
        assert abs(orc.score("combined", mom, b_full) - 0.5 * (r_i ** 2 + dice)) < 1e-12
        assert abs(orc.score("mask_dice", mom, b_full) - dice) < 1e-15
        checked += 1
    assert checked >= 10


def test_score_zero_cases(orc):
    # overlap below n_min, empty overlap, constant target
    assert orc.ncc2_from_moments([5, 10, 30, 0, 20, 2, 4], n_min=6) == 0.0
    assert orc.ncc2_from_moments([0, 0, 0, 0, 0, 0, 0]) == 0.0
    assert orc.ncc2_from_moments([4, 1000, 400000, 0, 4000, 16, 64]) == 0.0
    assert orc.dice_from_counts(10, 0, 0, 0) == 0.0


def test_min_overlap_boundary(orc):
    # the reading: a score is 0 when the overlap n is BELOW n_min, so n = n_min
    # still scores.  Samples (1, 2, 3, 4) against (1, 2, 3, 5): r^2 = 0.9657...
    m = [4, 10, 30, 0, 34, 11, 39]
    r = np.corrcoef([1, 2, 3, 4], [1, 2, 3, 5])[0, 1]
    assert orc.ncc2_from_moments(m, n_min=4) == pytest.approx(r * r, rel=1e-12)
    assert orc.ncc2_from_moments(m, n_min=5) == 0.0
    assert orc.dice_from_counts(7, 3, 2, 5, n_min=7) == pytest.approx(2 * 2 / (3 + 5))
    assert orc.dice_from_counts(7, 3, 2, 5, n_min=8) == 0.0


# ------------------------------------------------------ weights, resampling

def test_weights_definition(orc):
    rng = np.random.default_rng(7)
    s = rng.uniform(0, 1, 500)
    W = orc.weights(s, 5).astype(np.int64)
    want = np.floor(((s / s.max()) ** 32) * 2**24).astype(np.int64)
    assert np.all(np.abs(W - want) <= 1) and W.max() == 2**24
    assert np.all(orc.weights(np.zeros(10), 5) == 0)


@pytest.mark.parametrize("N", [1, 7, 256, 1000])
def test_resample_matches_bruteforce(orc, N):
    rng = np.random.default_rng(N)
    for trial in range(3):
        W = rng.integers(0, 2**24 + 1, N).astype(np.uint64)
        W[rng.random(N) < 0.5] = 0
        u = int(rng.integers(0, 2**32))
        got = orc.resample(W, u)
        assert np.array_equal(got, bf.systematic_bruteforce(W, u))


def test_resample_closed_forms(orc):
    N = 333
    assert np.array_equal(orc.resample(np.full(N, 12345, np.uint64), 0), np.arange(N))
    assert np.array_equal(orc.resample(np.full(N, 2**24, np.uint64), 2**32 - 1), np.arange(N))
    oh = np.zeros(N, np.uint64)
    oh[101] = 77
    assert np.all(orc.resample(oh, 999) == 101)
    assert np.array_equal(orc.resample(np.zeros(N, np.uint64), 5), np.arange(N))
    rng = np.random.default_rng(3)
    W = rng.integers(0, 1000, N).astype(np.uint64)
    idx = orc.resample(W, int(rng.integers(0, 2**32)))
    counts = np.bincount(idx, minlength=N)
    exp = N * W.astype(np.float64) / W.sum()
    assert np.all(counts >= np.floor(exp) - 1e-9) and np.all(counts <= np.ceil(exp) + 1e-9)
    assert np.all(np.diff(idx) >= 0)


def test_estimate_weighted_mean(orc):
    rng = np.random.default_rng(8)
    x = rng.uniform(-1, 1, (6, 50)).astype(np.float32)
    W = rng.integers(0, 100, 50).astype(np.uint64)
    np.testing.assert_allclose(orc.estimate(x, W), (x.astype(np.float64) * W).sum(1) / W.sum(),
                               rtol=1e-14)
    np.testing.assert_allclose(orc.estimate(x, np.zeros(50, np.uint64)), x.mean(1), rtol=1e-6)


# ------------------------------------------------------ prediction / init

def test_init_and_perturb_statistics(orc):
    lim = np.array([0.5, 0.4, 0.3, 8, 6, 4], np.float32)
    x = orc.init_particles(20000, 3, lim)
    assert np.all(np.abs(x) <= lim[:, None])
    np.testing.assert_allclose(x.mean(1), 0, atol=0.02 * lim.max())
    np.testing.assert_allclose(x.var(1), lim**2 / 3, rtol=0.05)
    z = np.zeros((6, 20000), np.float32)
    sig = np.ones(6, np.float32) * 0.01
    big = np.full(6, 1e3, np.float32)
    e = orc.perturb(z, 3, 1, sig, big) / 0.01
    assert np.all(np.abs(e) <= 2 * math.sqrt(3) + 1e-5)
    np.testing.assert_allclose(e.mean(1), 0, atol=0.03)
    np.testing.assert_allclose(e.var(1), 1.0, rtol=0.05)
    # clamping to the limits
    xc = orc.perturb(np.tile(lim[:, None], (1, 100)), 3, 2, lim, lim)
    assert np.all(np.abs(xc) <= lim[:, None])
    s = orc.sigma(0.25, 0.8, 3, lim)
    np.testing.assert_allclose(s, 0.25 * lim * 0.8**3, rtol=1e-6)


def test_random_draws_independent_across_dofs_iterations_and_particles(orc):
    # Each (particle, iteration, DOF) draws its own counter-based numbers: the
    # initial DOFs are uncorrelated with one another, the perturbation noise
    # of one iteration with that of the next and across DOFs, and the
    # resampling offsets of successive iterations are uniform on [0, 2^32).
    from scipy import stats as st
    N = 20000
    bound = 5 / math.sqrt(N)
    lim = np.array([0.5, 0.4, 0.3, 8, 6, 4], np.float32)
    x = orc.init_particles(N, 11, lim)
    c = np.corrcoef(x)
    assert np.all(np.abs(c[np.triu_indices(6, 1)]) < bound)
    z = np.zeros((6, N), np.float32)
    sig = np.full(6, 0.01, np.float32)
    big = np.full(6, 1e3, np.float32)
    e1 = orc.perturb(z, 11, 1, sig, big)
    e2 = orc.perturb(z, 11, 2, sig, big)
    for d in range(6):
        assert abs(np.corrcoef(e1[d], e2[d])[0, 1]) < bound
    c = np.corrcoef(e1)
    assert np.all(np.abs(c[np.triu_indices(6, 1)]) < bound)
    u = np.array([orc.resample_offset(11, k) for k in range(4096)], np.float64)
    assert len(np.unique(u)) >= 4090
    assert st.kstest(u / 2.0**32, "uniform").pvalue > 1e-4


def test_register_noise_scale_follows_the_schedule_and_the_proposal_spread(orc):
    # One step of the filter from a given cloud: the perturbation of
    # iteration 1 moves each resampled particle by sigma_1 * eps, eps of unit
    # variance, with sigma_1 = sigma0_frac * L * decay by default and
    # sig_base * decay when a proposal's spread is given.
    N, decay = 4096, 0.8
    src = pfsynth.random_mask(4, (9, 9, 9), 0.5)
    lim_r, lim_t = 3.0, 100.0
    rng = np.random.default_rng(3)
    x0 = (rng.uniform(-1, 1, (6, N)) * np.array([0.05] * 3 + [1.0] * 3)[:, None]).astype(np.float32)
    for sig_base, want in ((None, 0.25 * np.array([lim_r] * 3 + [lim_t] * 3) * decay),
                           (np.array([0.01, 0.02, 0.03, 0.4, 0.5, 0.6], np.float32),
                            np.array([0.01, 0.02, 0.03, 0.4, 0.5, 0.6]) * decay)):
        r = orc.register("mask_dice", (9, 9, 9), np.zeros(3, np.float32), (9, 9, 9), np.zeros(3, np.float32),
                         N, 2, lim_r, lim_t, seed=5, src_mask=src, tgt_mask=src, poses=x0.copy(),
                         sigma_decay=decay, sig_base=sig_base)
        moved = r["tr_poses"][1] - r["tr_poses"][0][:, r["tr_idx"][0]]
        np.testing.assert_allclose(moved.std(1), want, rtol=0.05)


# ----------------------------------------------------------------- warp

def test_warp_identity_and_integer_maps(orc):
    src = pfsynth.random_image(91, (13, 12, 11))
    out = orc.warp(src, np.zeros(3, np.float32), (13, 12, 11), np.zeros(3, np.float32),
                   np.zeros(6, np.float32), 1)
    assert np.array_equal(out, src)
    out = orc.warp(src, np.zeros(3, np.float32), (13, 12, 11), np.zeros(3, np.float32),
                   np.zeros(6, np.float32), 0)
    assert np.array_equal(out, src)
    a0 = np.zeros(3, np.float32)
    for P, b in _exact_cases(8, 10):
        for interp in (0, 1):
            got = orc.warp_matrix(src, (9, 14, 10), bf.exact_matrix(P, b), a0, interp)
            assert np.array_equal(got, bf.integer_map_warp(src, (9, 14, 10), P, b))


def test_warp_dyadic_shifts_exact(orc):
    # quarter-voxel shifts of the axis maps: the trilinear samples are exact
    # multiples of 1/64, so the uint8 output is pinned exactly, ties (odd
    # multiples of 1/2 at half-voxel shifts) included: rounded half to even;
    # nearest neighbour rounds its half-voxel ties up
    src = pfsynth.random_image(94, (12, 11, 10))
    a0 = np.zeros(3, np.float32)
    rng = np.random.default_rng(14)
    ties = 0
    for P, b in _exact_cases(10, 24):
        b = rng.integers(-3, 7, 3)
        h4 = rng.integers(0, 4, 3)
        M = bf.exact_matrix(P, b)
        M[[3, 7, 11]] += 0.25 * h4
        for interp in (0, 1):
            got = orc.warp_matrix(src, (10, 12, 9), M, a0, interp)
            want = bf.dyadic_map_warp(src, (10, 12, 9), P, b, h4, interp)
            assert np.array_equal(got, want), (P.tolist(), b.tolist(), h4.tolist(), interp)
        ties += int((h4 == 2).any())
    assert ties >= 8


def test_warp_rot90_equals_numpy(orc):
    src = pfsynth.random_image(92, (11, 9, 7))
    X, Y, Z = 11, 9, 7
    # q = (X-1-y, x, z): target dims (Y, X, Z) holds the source turned by 90 deg about z
    P = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]])
    b = np.array([X - 1, 0, 0])
    got = orc.warp_matrix(src, (Y, X, Z), bf.exact_matrix(P, b), np.zeros(3, np.float32), 1)
    want = np.transpose(src, (0, 2, 1))[:, ::-1, :]
    assert np.array_equal(got, want)


def test_warp_trilinear_vs_scipy(orc):
    src = pfsynth.random_image(93, (24, 22, 20))
    so, to, td = np.zeros(3, np.float32), np.array([2.0, 1.0, 2.0], np.float32), (18, 17, 15)
    pose = np.array([0.2, -0.1, 0.3, 1.5, -0.7, 0.4], np.float32)
    got = orc.warp(src, so, td, to, pose, 1).reshape(-1).astype(np.int32)
    q = bf.source_index_f64(pose, (24, 22, 20), so, td, to)
    ok, s = bf.trilinear_f64(src, q)
    want = np.zeros(len(q), np.int32)
    want[ok] = np.rint(s).astype(np.int32)
    diff = np.abs(got - want)
    assert diff.max() <= 1 and np.mean(diff > 0) < 0.01


def test_fixed_point_ncc_weak_correlation(orc):
    """Near r = 0 the relative error of r^2 is largest (Eq. 2 is squared);
    15 fractional bits keep even these scores within 1e-5 of the fp64 NCC."""
    worst = 0.0
    for seed in range(4):
        src = pfsynth.random_image(100 + seed, (40, 37, 29))
        tgt = pfsynth.random_image(200 + seed, (45, 33, 27))
        so, to = np.array([0.0, 1.5, -2.0], np.float32), np.array([3.0, -1.0, 2.5], np.float32)
        for pose in _rand_poses(10, rot=0.6, tr=8, seed=seed).astype(np.float32):
            M, a = orc.pose_matrix(pose, src.shape[::-1], so, to)
            fixed = orc.ncc2_from_moments(orc.measure_image(src, tgt, M, a)[0])
            exact = orc.ncc2_f64(src, tgt, M, a)[0]
            if exact > 0:
                worst = max(worst, abs(fixed - exact) / exact)
    assert worst <= 1e-5, worst


# --------------------------------------------------- quaternion estimator

def test_quaternion_of_pose_matches_scipy_and_rotation(orc):
    from scipy.spatial.transform import Rotation
    for pose in _rand_poses(30, rot=1.5, tr=5, seed=8):
        q = orc.quaternion(pose)
        rx, ry, rz = pose[:3]
        x, y, z, w = Rotation.from_euler("ZXY", [rz, rx, ry]).as_quat()
        ref = np.array([w, x, y, z])
        assert min(np.max(np.abs(q - ref)), np.max(np.abs(q + ref))) < 1e-14
        np.testing.assert_allclose(orc.quaternion_matrix(q), orc.rotation(pose.astype(np.float32)), atol=1e-6)
        assert abs(np.linalg.norm(q) - 1.0) < 1e-15


def test_quaternion_estimate_closed_forms(orc):
    # two rotations about z with weights w1, w2: the average turns by
    # atan2(w1 sin t1 + w2 sin t2, w1 cos t1 + w2 cos t2) about z
    for t1, t2, w1, w2 in ((0.3, -0.3, 5, 5), (0.1, 0.5, 3, 1), (-0.7, 0.2, 1, 7)):
        poses = np.zeros((6, 2), np.float32)
        poses[2] = (t1, t2)
        poses[3] = (1.0, 3.0)
        est = orc.estimate_quaternion(poses, np.array([w1, w2], np.uint64))
        want = math.atan2(w1 * math.sin(np.float32(t1)) + w2 * math.sin(np.float32(t2)),
                          w1 * math.cos(np.float32(t1)) + w2 * math.cos(np.float32(t2)))
        assert abs(est[2] - want) < 1e-12 and abs(est[0]) < 1e-12 and abs(est[1]) < 1e-12
        assert abs(est[3] - (w1 * 1.0 + w2 * 3.0) / (w1 + w2)) < 1e-12
    # identical rotations give that rotation; all-zero weights average uniformly
    pose = np.array([0.4, -0.2, 1.1, 0, 0, 0], np.float32)
    est = orc.estimate_quaternion(np.repeat(pose[:, None], 5, 1), np.zeros(5, np.uint64))
    np.testing.assert_allclose(est[:3], pose[:3].astype(np.float64), atol=1e-7)


def test_quaternion_estimate_matches_scipy_mean(orc):
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(3)
    centre = np.array([0.3, -0.5, 0.9])
    poses = np.zeros((6, 400), np.float32)
    poses[:3] = (centre[:, None] + rng.normal(0, 0.25, (3, 400))).clip(-1.5, 1.5)
    W = rng.integers(0, 1 << 24, 400).astype(np.uint64)
    est = orc.estimate_quaternion(poses, W)
    p64 = poses.astype(np.float64)
    rot = Rotation.from_euler("ZXY", np.stack([p64[2], p64[0], p64[1]], 1))
    rz, rx, ry = rot.mean(weights=W.astype(np.float64)).as_euler("ZXY")
    np.testing.assert_allclose(est[:3], [rx, ry, rz], atol=1e-9)
    # the angle mean is biased away from it for a wide cloud
    assert np.max(np.abs(orc.estimate(poses, W)[:3] - est[:3])) > 1e-4


def _round_f32(x):
    """Nearest float32 to the exact rational x (ties to even)."""
    from fractions import Fraction
    c = np.float32(float(x))
    best = None
    for cand in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        err = abs(Fraction(float(cand)) - x)
        key = (err, int(np.float32(cand).view(np.uint32)) & 1)
        if best is None or key < best[0]:
            best = (key, cand)
    return np.float32(best[1])


def test_trilinear_lerp_single_rounding(orc):
    """Each lerp of the trilinear sample (Sec. 3.3) rounds a + f*(b - a) once:
    on a volume that varies along x only, the y and z lerps are exact, so the
    sample must be the exact interpolation a + f*(b - a) rounded to fp32 once.
    A separately rounded product (two roundings) differs on some of these."""
    from fractions import Fraction
    rng = np.random.default_rng(41)
    X, Y, Z = 40, 3, 3
    line = rng.integers(0, 256, X).astype(np.uint8)
    src = np.broadcast_to(line[None, None, :], (Z, Y, X)).copy()
    twice = 0
    for _ in range(4000):
        qx = np.float32(rng.uniform(0, X - 1))
        q = np.array([qx, rng.uniform(0, Y - 1), rng.uniform(0, Z - 1)], np.float32)
        got = orc.trilinear(src, q)
        i = min(int(np.floor(qx)), X - 2)
        f = Fraction(float(qx)) - i                 # exact: q - floor(q) is representable
        a, b = int(line[i]), int(line[i + 1])
        want = _round_f32(a + f * (b - a))
        assert np.float32(got) == want, (qx, got, want)
        two = np.float32(np.float32(a) + np.float32(np.float32(f) * np.float32(b - a)))
        twice += int(two != want)
    assert twice > 0   # the case set separates one rounding from two
    assert orc.trilinear(src, np.array([X - 0.5, 1, 1], np.float32)) is None


def test_init_gaussian_statistics(orc):
    """The proposal-seeded cloud: bounded Irwin-Hall draws (|eps| <= 2 sqrt 3)
    of unit variance around the mean, clamped to the limits."""
    N = 20000
    lim = np.array([0.5, 0.5, 0.5, 20, 20, 20], np.float32)
    mean = np.array([0.1, -0.2, 0.05, 3.0, -4.0, 1.0], np.float32)
    std = np.array([0.02, 0.03, 0.01, 1.0, 2.0, 0.5], np.float32)
    x = orc.init_gaussian(N, 7, mean, std, lim)
    eps = (x.astype(np.float64) - mean[:, None]) / std[:, None]
    assert np.all(np.abs(eps) <= 2 * np.sqrt(3) + 1e-4)
    assert np.allclose(eps.mean(1), 0.0, atol=0.03)
    assert np.allclose(eps.std(1), 1.0, atol=0.03)
    assert np.array_equal(x, orc.init_gaussian(N, 7, mean, std, lim))
    assert not np.array_equal(x, orc.init_gaussian(N, 8, mean, std, lim))
    # clamping: a mean outside the limits puts every particle on the limit
    far = mean.copy()
    far[3] = 40.0
    assert np.all(orc.init_gaussian(100, 7, far, std, lim)[3] == 20.0)
    far[3], far[4] = -40.0, -25.0
    x = orc.init_gaussian(100, 7, far, std, lim)
    assert np.all(x[3] == -20.0) and np.all(x[4] == -20.0)
