"""The seeded synthetic inputs follow the recipes the benchmark workloads state
(the paper's data is private): shapes, ground-truth pose ranges, the target
field of view and its overlap with the source, the speckle distribution, and
that each target is the source's shape seen through the ground-truth pose.
CPU only; the oracle serves as the resampler where one is needed.
"""
import numpy as np

import pfsynth
from tests import bruteforce as bf


def _dice(a, b):
    a, b = a != 0, b != 0
    return 2.0 * np.sum(a & b) / (a.sum() + b.sum())


def test_mask_workload_recipe(orc):
    # 64^3 ellipsoid mask, centre 31.5 +- 1, semi-axes 20/14/14 +- 1, target
    # 64x64x45 with origin (0, 0, 19), true pose within 10 deg / 5 voxels
    for seed in (0, 1, 2):
        p = pfsynth.ellipsoid_pair(seed)
        assert p.src.shape == (64, 64, 64) and p.tgt.shape == (45, 64, 64)
        assert p.src.dtype == np.uint8 and set(np.unique(p.src)) <= {0, 1} and set(np.unique(p.tgt)) <= {0, 1}
        assert np.array_equal(p.tgt_origin, [0, 0, 19])
        assert np.all(np.abs(p.true_pose[:3]) <= np.deg2rad(10.0) + 1e-6)
        assert np.all(np.abs(p.true_pose[3:]) <= 5.0 + 1e-6)
        assert np.all(np.abs(p.info["centre"] - 31.5) <= 1.0)
        assert np.all(np.abs(p.info["semi_axes"] - [20, 14, 14]) <= 1.0)
        # the target is the analytic shape under the true pose: the source
        # resampled by it (nearest neighbour) differs only on the boundary
        warped = orc.warp(p.src, p.src_origin, (64, 64, 45), p.tgt_origin, p.true_pose, 0)
        assert _dice(warped, p.tgt) > 0.97
        # and the identity does not line them up as well
        ident = orc.warp(p.src, p.src_origin, (64, 64, 45), p.tgt_origin, np.zeros(6, np.float32), 0)
        assert _dice(ident, p.tgt) < _dice(warped, p.tgt)


def test_image_workload_overlap_and_pose():
    # the target field of view slides along x until the fraction of target
    # voxels that see the source is a draw from U(35 %, 60 %); true pose
    # within 15 deg / 12 voxels (smaller grids than the 224x208x176 workload,
    # same recipe)
    dims = (72, 64, 56)
    for seed in range(4):
        p = pfsynth.speckle_pair(seed, src_dims=dims, with_masks=True)
        assert p.src.shape == p.tgt.shape == dims[::-1]
        assert np.all(np.abs(p.true_pose[:3]) <= np.deg2rad(15.0) + 1e-6)
        assert np.all(np.abs(p.true_pose[3:]) <= 12.0 + 1e-6)
        assert p.tgt_origin[1] == p.tgt_origin[2] == 0.0      # slid along x only
        frac = _overlap(p, dims)
        # the placement estimates the fraction on a stride-4 lattice and
        # rounds the origin to whole voxels, which on grids this small costs
        # up to a few per cent (under 1 % at the workload's size, below)
        assert abs(frac - p.info["overlap_target"]) < 0.05, (frac, p.info["overlap_target"])
        assert 0.35 - 0.05 <= frac <= 0.60 + 0.05
        # LV-cavity masks: binary, inside the field of view, non-empty
        assert set(np.unique(p.src_mask)) <= {0, 1} and p.src_mask.sum() > 0 and p.tgt_mask.sum() > 0


def test_image_workload_pair_at_full_size():
    # the benchmark's own 224x208x176 pair (seed 0): overlap within 1 % of
    # its U(35 %, 60 %) draw, pose within the recipe's ranges
    dims = (224, 208, 176)
    p = pfsynth.cached(pfsynth.speckle_pair, 0, with_masks=True)
    assert p.src.shape == p.tgt.shape == dims[::-1]
    frac = _overlap(p, dims)
    assert abs(frac - p.info["overlap_target"]) < 0.01 and 0.35 <= p.info["overlap_target"] <= 0.60
    assert np.all(np.abs(p.true_pose[:3]) <= np.deg2rad(15.0) + 1e-6)
    assert np.all(np.abs(p.true_pose[3:]) <= 12.0 + 1e-6)


def _overlap(p, dims):
    q = bf.source_index_f64(p.true_pose, dims, p.src_origin, dims, p.tgt_origin)
    return float(np.mean(np.all((q >= 0) & (q <= np.asarray(dims) - 1), axis=1)))


def test_image_target_is_the_source_seen_through_the_true_pose(orc):
    # same tissue and speckle grain in both views (speckle hashed from the
    # rounded world voxel), each view with its own gain: NCC^2 of the source
    # resampled by the true pose against the target is far above that of the
    # identity
    dims = (64, 60, 56)
    p = pfsynth.speckle_pair(3, src_dims=dims, overlap=(0.55, 0.6), max_rot_deg=8, max_trans=4)
    m_true, a = orc.pose_matrix(p.true_pose, dims, p.src_origin, p.tgt_origin)
    m_id, _ = orc.pose_matrix(np.zeros(6, np.float32), dims, p.src_origin, p.tgt_origin)
    s_true = orc.ncc2_f64(p.src, p.tgt, m_true, a)[0]
    s_id = orc.ncc2_f64(p.src, p.tgt, m_id, a)[0]
    assert s_true > 0.3 and s_true > 3 * s_id, (s_true, s_id)


def test_speckle_is_rayleigh_sigma_40():
    # Rayleigh(sigma): mean sigma sqrt(pi/2), variance sigma^2 (4 - pi)/2
    rng = np.random.default_rng(0)
    w = rng.uniform(-500, 500, (3, 400000))
    s = pfsynth._speckle(w[0], w[1], w[2], 40.0, 1234)
    assert abs(s.mean() / (40.0 * np.sqrt(np.pi / 2)) - 1) < 0.01
    assert abs(s.std() / (40.0 * np.sqrt((4 - np.pi) / 2)) - 1) < 0.02
    # one grain per world voxel: the same rounded position gives the same value
    s2 = pfsynth._speckle(np.rint(w[0]) + 0.3, np.rint(w[1]) - 0.2, np.rint(w[2]), 40.0, 1234)
    assert np.array_equal(s, pfsynth._speckle(np.rint(w[0]), np.rint(w[1]), np.rint(w[2]), 40.0, 1234))
    assert np.array_equal(s, s2)
