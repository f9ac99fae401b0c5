"""GPU parity: the sm_103a kernels, called through the C ABI, against the CPU
oracle on the same seeded inputs.

Bars (element by element):
  * Philox words, pose matrices, mask counts, image moments (samples rounded
    to 2^-15), scores, quantised weights, resampled indices, particle clouds
    and warped voxels: bit-exact;
  * image NCC^2 against the fp64 two-pass oracle: within 1e-5 relative;
  * final estimates: within 1e-4 rad and 1e-3 voxel (the fp64 weighted sums
    are reduced in a different order).
"""
import numpy as np
import pytest

import pfsynth
from tests import bruteforce as bf

pytestmark = pytest.mark.gpu

ROT_TOL, TRANS_TOL, NCC_RTOL = 1e-4, 1e-3, 1e-5


@pytest.fixture(scope="module")
def pk():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2504_19930_gb300 as pk
    pk.build()
    pk.load()
    return pk


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _reg(pk, mode, pair, N, lim_r, lim_t, seed, device=True, **kw):
    d = _cuda if device else (lambda a: a)
    args = {}
    if mode in ("image_ncc", "combined"):
        args.update(src=d(pair.src), tgt=d(pair.tgt))
    if mode != "image_ncc":
        args.update(src_mask=d(pair.src_mask), tgt_mask=d(pair.tgt_mask))
    args.update({k: kw.pop(k) for k in ("src_mask", "tgt_mask") if k in kw})
    return pk.Registration(mode, src_origin=pair.src_origin, tgt_origin=pair.tgt_origin, n_particles=N,
                           rot_limit=lim_r, trans_limit=lim_t, seed=seed, **args, **kw)


def _oracle_run(orc, mode, pair, N, K, lim_r, lim_t, seed, **kw):
    return orc.register(mode, pair.src_dims, pair.src_origin, pair.tgt_dims, pair.tgt_origin, N, K, lim_r,
                        lim_t, seed=seed, src=pair.src if mode in ("image_ncc", "combined") else None,
                        tgt=pair.tgt if mode in ("image_ncc", "combined") else None,
                        src_mask=pair.src_mask if mode != "image_ncc" else None,
                        tgt_mask=pair.tgt_mask if mode != "image_ncc" else None, **kw)


def _assert_trajectory(reg, ref, K, k0=0):
    for kk in range(K):
        reg.step(1)
        st = reg.state()
        k = kk
        assert np.array_equal(st["poses_measured"], ref["tr_poses"][k]), f"particles differ at k={k0 + k}"
        assert np.array_equal(st["moments"], ref["tr_mom"][k]), f"moments differ at k={k0 + k}"
        assert np.array_equal(st["scores"], ref["tr_score"][k]), f"scores differ at k={k0 + k}"
        assert np.array_equal(st["weights"], ref["tr_W"][k]), f"weights differ at k={k0 + k}"
        assert np.array_equal(st["resample_idx"], ref["tr_idx"][k]), f"indices differ at k={k0 + k}"
    est, _ = reg.estimate(with_score=False)
    err = np.abs(est.astype(np.float64) - ref["est"])
    assert np.all(err[:3] <= ROT_TOL) and np.all(err[3:] <= TRANS_TOL), err


# --------------------------------------------------------------- primitives

def test_philox_device_matches_known_answers(pk, orc):
    import os
    rows = [l.split() for l in open(os.path.join(os.path.dirname(__file__), "golden",
                                                 "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    for r in rows:
        v = [int(x, 16) for x in r]
        assert [int(x) for x in pk.pf_philox(v[0:4], v[4:6])] == v[6:10]
    rng = np.random.default_rng(0)
    for _ in range(50):
        ctr, key = rng.integers(0, 2**32, 4), rng.integers(0, 2**32, 2)
        assert np.array_equal(pk.pf_philox(ctr, key), orc.philox(ctr, key))


def test_pose_matrix_bit_exact(pk, orc):
    rng = np.random.default_rng(1)
    edge = np.float32(np.pi / 2)
    poses = [np.array([edge, -edge, edge, 3.25, -7.5, 0.0], np.float32), np.zeros(6, np.float32)]
    poses += [np.concatenate([rng.uniform(-1.57, 1.57, 3), rng.uniform(-40, 40, 3)]).astype(np.float32)
              for _ in range(200)]
    for i, pose in enumerate(poses):
        sd = tuple(int(v) for v in rng.integers(2, 300, 3))
        so = rng.uniform(-20, 20, 3).astype(np.float32)
        to = rng.uniform(-20, 20, 3).astype(np.float32)
        Mg, ag = pk.pf_pose_matrix(pose, sd, so, to)
        Mo, ao = orc.pose_matrix(pose, sd, so, to)
        assert np.array_equal(Mg, Mo) and np.array_equal(ag, ao), (i, Mg - Mo)


# ------------------------------------------------------------- measurement

def _measure_ctx(pk, mode, src, tgt, N=1, src_mask=None, tgt_mask=None):
    s, t = _cuda(src), _cuda(tgt)
    if mode == "image_ncc":
        return pk.Registration(mode, src=s, tgt=t, n_particles=N)
    if mode == "combined":
        sm = s if src_mask is None else _cuda(src_mask)
        tm = t if tgt_mask is None else _cuda(tgt_mask)
        return pk.Registration(mode, src=s, tgt=t, src_mask=sm, tgt_mask=tm, n_particles=N)
    return pk.Registration(mode, src_mask=s, tgt_mask=t, n_particles=N)


@pytest.mark.parametrize("mode", ["mask_dice", "image_ncc"])
def test_integer_maps_exact(pk, mode):
    """Grid-aligned 90-degree maps and integer shifts, injected as exact
    matrices: counts and moments equal numpy's exact integer brute force."""
    if mode == "mask_dice":
        src = pfsynth.random_mask(11, (37, 29, 23), 0.4)
        tgt = pfsynth.random_mask(12, (33, 35, 31), 0.4)
    else:
        src = pfsynth.random_image(41, (37, 29, 23))
        tgt = pfsynth.random_image(42, (33, 35, 31))
    rng = np.random.default_rng(5)
    perms = bf.signed_permutations()
    cases = [(perms[rng.integers(len(perms))], rng.integers(-10, 40, 3)) for _ in range(48)]
    mats = np.stack([bf.exact_matrix(P, b) for P, b in cases])
    with _measure_ctx(pk, mode, src, tgt) as reg:
        got = reg.measure(mats, np.zeros(3, np.float32))
    for i, (P, b) in enumerate(cases):
        want = bf.integer_map_counts(src, tgt, P, b, image=(mode == "image_ncc"))
        g = got[i, 8:12] if mode == "mask_dice" else got[i, 0:7]
        assert g.tolist() == want.tolist(), (i, P, b)


@pytest.mark.parametrize("mode,sdims,tdims", [
    ("mask_dice", (40, 37, 29), (45, 33, 27)),          # bit mask in shared memory, ragged rows
    ("mask_dice", (130, 118, 97), (61, 50, 40)),        # bit mask too large for shared memory
    ("image_ncc", (40, 37, 29), (45, 33, 27)),
    ("image_ncc", (70, 66, 60), (97, 31, 20)),          # rows longer than 3 warps, few rows
    ("image_ncc", (30, 40, 36), (20, 45, 40)),          # every row shorter than a pass of 64
    ("image_ncc", (70, 30, 26), (64, 33, 30)),          # rows of exactly one pass at the centre
    ("image_ncc", (300, 40, 20), (290, 36, 16)),        # > 8192 entries per work item
    ("combined", (44, 39, 31), (41, 35, 30)),
])
def test_measure_random_poses_bit_exact(pk, orc, mode, sdims, tdims):
    if mode == "mask_dice":
        src, tgt = pfsynth.random_mask(1, sdims, 0.4), pfsynth.random_mask(2, tdims, 0.4)
    else:
        src, tgt = pfsynth.random_image(1, sdims), pfsynth.random_image(2, tdims)
    so = np.array([0.0, 1.5, -2.0], np.float32)
    to = np.array([3.0, -1.0, 2.5], np.float32)
    rng = np.random.default_rng(3)
    poses = np.concatenate([rng.uniform(-0.6, 0.6, (40, 3)), rng.uniform(-8, 8, (40, 3))], 1).astype(np.float32)
    mats, a = orc.pose_matrices(poses.T, sdims, so, to)
    with _measure_ctx(pk, mode, src, tgt) as reg:
        got = reg.measure(mats, a)
    srcm = (src != 0).astype(np.uint8) if mode == "combined" else src
    tgtm = (tgt != 0).astype(np.uint8) if mode == "combined" else tgt
    if mode in ("mask_dice", "combined"):
        want = orc.measure_mask(srcm, tgtm, mats, a)
        assert np.array_equal(got[:, 8:12], want)
    if mode in ("image_ncc", "combined"):
        want = orc.measure_image(src, tgt, mats, a)
        assert np.array_equal(got[:, 0:7], want)
        f64 = orc.ncc2_f64(src, tgt, mats, a)
        for i in range(len(mats)):
            s = orc.ncc2_from_moments(got[i, 0:7])
            assert abs(s - f64[i]) <= NCC_RTOL * f64[i], (i, s, f64[i])


@pytest.mark.parametrize("mode,sdims,tdims,P", [
    # combined mode with masks drawn independently of the image (not image != 0)
    ("combined", (44, 39, 31), (41, 35, 30), 40),
    # targets of 64 x 40 rows = 80 work items per particle, more than the 64 a
    # CTA takes, so the CTA shares two x-product tables (the per-CTA form) and
    # CTAs straddle two particles; P = 37 leaves the last CTA partial
    ("combined", (50, 46, 40), (41, 64, 40), 37),           # mask bits in shared memory
    ("mask_dice", (130, 118, 97), (41, 64, 40), 37),        # mask bits too large: read from L2
    ("combined", (130, 118, 97), (41, 64, 40), 37),
])
def test_measure_independent_masks_and_cta_tables_bit_exact(pk, orc, mode, sdims, tdims, P):
    src_m, tgt_m = pfsynth.random_mask(21, sdims, 0.45), pfsynth.random_mask(22, tdims, 0.45)
    src_i, tgt_i = pfsynth.random_image(23, sdims), pfsynth.random_image(24, tdims)
    so = np.array([1.0, -2.0, 0.5], np.float32)
    to = np.array([-3.0, 2.0, 1.0], np.float32)
    rng = np.random.default_rng(31)
    poses = np.concatenate([rng.uniform(-0.6, 0.6, (P, 3)), rng.uniform(-9, 9, (P, 3))], 1).astype(np.float32)
    mats, a = orc.pose_matrices(poses.T, sdims, so, to)
    if mode == "combined":
        with _measure_ctx(pk, mode, src_i, tgt_i, src_mask=src_m, tgt_mask=tgt_m) as reg:
            got = reg.measure(mats, a)
        assert np.array_equal(got[:, 0:7], orc.measure_image(src_i, tgt_i, mats, a))
    else:
        with _measure_ctx(pk, mode, src_m, tgt_m) as reg:
            got = reg.measure(mats, a)
    want = orc.measure_mask(src_m, tgt_m, mats, a)
    assert np.array_equal(got[:, 8:12], want)
    # the masks are not trivially full: the counts carry information
    assert np.all(want[:, 1] <= want[:, 0]) and np.any(want[:, 1] < want[:, 0]) and np.any(want[:, 3] < want[:, 1])


def test_image_source_beyond_2p23_voxels_bit_exact(pk, orc):
    """A source of more than 2^23 voxels (256 x 256 x 160): the kernel forms
    the quad index with integer arithmetic instead of fp32 (exact only below
    2^24).  The target sits near the source's far corner, so the indices
    themselves exceed 2^23 (every sample at z >= 128)."""
    sdims, tdims = (256, 256, 160), (60, 50, 40)
    assert np.prod(sdims) > (1 << 23)
    src, tgt = pfsynth.random_image(51, sdims, smooth=False), pfsynth.random_image(52, tdims)
    so = np.zeros(3, np.float32)
    to = np.array([150.0, 180.0, 110.0], np.float32)
    rng = np.random.default_rng(53)
    poses = np.concatenate([rng.uniform(-0.4, 0.4, (24, 3)), rng.uniform(-10, 10, (24, 3))], 1).astype(np.float32)
    mats, a = orc.pose_matrices(poses.T, sdims, so, to)
    with _measure_ctx(pk, "image_ncc", src, tgt) as reg:
        got = reg.measure(mats, a)
    want = orc.measure_image(src, tgt, mats, a)
    assert np.array_equal(got[:, 0:7], want)
    assert np.all(want[:, 0] > 0)
    # samples come from source planes z >= 128, whose voxel indices exceed 2^23
    corners = np.array([[x, y, z] for x in (0, tdims[0] - 1) for y in (0, tdims[1] - 1)
                        for z in (0, tdims[2] - 1)], np.float64) - a
    qz = corners @ mats[:, 8:11].T.astype(np.float64) + mats[:, 11]
    assert np.any((qz >= 129) & (qz <= sdims[2] - 1))


def test_measure_degenerate_cases(pk, orc):
    """No overlap at all, full overlap at identity, and a 2x2x2 source."""
    src = pfsynth.random_image(5, (16, 15, 14))
    far = np.zeros((1, 12), np.float32)
    far[0, [0, 5, 10]] = 1
    far[0, 3] = 1e4
    ident, a = orc.pose_matrix(np.zeros(6, np.float32), (16, 15, 14), np.zeros(3, np.float32),
                               np.zeros(3, np.float32))
    with _measure_ctx(pk, "image_ncc", src, src) as reg:
        got = reg.measure(np.stack([far[0], ident]), a)
    assert np.all(got[0] == 0)
    assert got[1, 0] == src.size and got[1, 1] == 32768 * int(src.astype(np.int64).sum())
    tiny = pfsynth.random_image(6, (2, 2, 2))
    tgt = pfsynth.random_image(7, (5, 4, 3))
    rng = np.random.default_rng(9)
    poses = np.concatenate([rng.uniform(-0.5, 0.5, (20, 3)), rng.uniform(-1, 1, (20, 3))], 1).astype(np.float32)
    mats, a = orc.pose_matrices(poses.T, (2, 2, 2), np.zeros(3, np.float32), np.array([-1.5, -1, -0.5], np.float32))
    with _measure_ctx(pk, "image_ncc", tiny, tgt) as reg:
        got = reg.measure(mats, a)
    assert np.array_equal(got[:, 0:7], orc.measure_image(tiny, tgt, mats, a))


# ---------------------------------------------------------- whole filter

@pytest.mark.parametrize("mode", ["mask_dice", "mask_ncc", "image_ncc", "combined"])
def test_trajectory_bit_exact_small(pk, orc, mode):
    if mode in ("mask_dice", "mask_ncc"):
        pair = pfsynth.ellipsoid_pair(7, src_dims=(30, 28, 26), tgt_dims=(33, 27, 21), tgt_origin=(0, 0, 6),
                                      semi_axes=(10, 7, 6), asymmetric=True, max_rot_deg=8, max_trans=3)
    else:
        pair = pfsynth.speckle_pair(7, src_dims=(36, 34, 30), tgt_dims=(37, 33, 29), overlap=(0.55, 0.7),
                                    max_rot_deg=8, max_trans=3, with_masks=(mode == "combined"))
    N, K, lr, lt = 200, 5, 0.2, 4.0
    ref = _oracle_run(orc, mode, pair, N, K, lr, lt, seed=17)
    with _reg(pk, mode, pair, N, lr, lt, 17) as reg:
        _assert_trajectory(reg, ref, K)


@pytest.mark.parametrize("N", [1, 1024, 1025])
def test_trajectory_at_the_update_kernel_boundary(pk, orc, N):
    """Clouds of up to 1024 particles take the one-CTA update, larger ones
    the three-kernel form; a single particle is the degenerate cloud."""
    pair = pfsynth.ellipsoid_pair(12, src_dims=(26, 24, 22), tgt_dims=(25, 24, 18), tgt_origin=(0, 0, 4),
                                  semi_axes=(9, 6, 5), asymmetric=True, max_rot_deg=8, max_trans=3)
    ref = _oracle_run(orc, "mask_dice", pair, N, 3, 0.2, 3.0, seed=31)
    with _reg(pk, "mask_dice", pair, N, 0.2, 3.0, 31) as reg:
        _assert_trajectory(reg, ref, 3)


def test_host_inputs_equal_device_inputs(pk, orc):
    pair = pfsynth.ellipsoid_pair(8, src_dims=(26, 24, 22), tgt_dims=(25, 24, 18), tgt_origin=(0, 0, 4),
                                  semi_axes=(9, 6, 5))
    ref = _oracle_run(orc, "mask_ncc", pair, 64, 3, 0.2, 3.0, seed=4)
    with _reg(pk, "mask_ncc", pair, 64, 0.2, 3.0, 4, device=False) as reg:
        _assert_trajectory(reg, ref, 3)


def test_checkpoint_resume_bit_exact(pk, orc):
    pair = pfsynth.ellipsoid_pair(9, src_dims=(28, 26, 24), tgt_dims=(28, 26, 20), tgt_origin=(0, 0, 4),
                                  semi_axes=(9, 7, 6), asymmetric=True)
    N = 128
    with _reg(pk, "mask_dice", pair, N, 0.25, 4.0, 21) as full:
        full.step(6)
        st_full = full.state()
        est_full, _ = full.estimate(False)
    with _reg(pk, "mask_dice", pair, N, 0.25, 4.0, 21) as a:
        a.step(3)
        saved, k = a.state()["poses_next"], a.iteration
    assert k == 3
    with _reg(pk, "mask_dice", pair, N, 0.25, 4.0, 21) as b:
        b.set_state(saved, k)
        b.step(3)
        st_b = b.state()
        est_b, _ = b.estimate(False)
    for key in ("poses_measured", "moments", "weights", "resample_idx", "poses_next"):
        assert np.array_equal(st_full[key], st_b[key]), key
    assert np.array_equal(est_full, est_b)


def test_mask64_full_registration_bit_exact(pk, orc):
    """The mask-based workload at full size: 64^3 ellipsoid, 64x64x45 target,
    N=256, 10 iterations, +-15 deg / +-8 voxels, Dice with nearest neighbour."""
    c = pfsynth.MASK64
    pair = pfsynth.ellipsoid_pair(0)
    lr, lt = np.deg2rad(c["rot_limit_deg"]), c["trans_limit"]
    ref = _oracle_run(orc, "mask_dice", pair, c["n_particles"], c["n_iters"], lr, lt, seed=c["seed"])
    with _reg(pk, "mask_dice", pair, c["n_particles"], lr, lt, c["seed"]) as reg:
        _assert_trajectory(reg, ref, c["n_iters"])
        est, score = reg.estimate()
        M, a = orc.pose_matrix(est, pair.src_dims, pair.src_origin, pair.tgt_origin)
        cnt = orc.measure_mask(pair.src, pair.tgt, M, a)[0]
        nmin = int(float(np.float32(0.01)) * pair.tgt.size)
        want = orc.dice_from_counts(cnt[0], cnt[1], cnt[3], int(pair.tgt.sum()), nmin)
        assert score == want
        _, best, ess, evals, _ = reg.log()
        assert len(best) == c["n_iters"] and best[-1] > 0.9 and np.all(ess > 0)
        assert evals[-1] == int(ref["tr_mom"][-1][:, 8].sum())


def test_image224_full_size_sampled(pk, orc):
    """The image-based workload at full size and in the launch configuration
    the bench times (224x208x176 speckle, N=2048, all 50 iterations, tuned
    tile shape): every cheap step (score, weights, resampling, prediction) is
    recomputed by the oracle on the GPU's own state at every iteration, bit
    for bit; at k = 0 and at the last iteration 32 sampled particles are
    re-measured by the oracle (spawned processes), moments bit for bit and
    NCC^2 within 1e-5 of the fp64 oracle."""
    from tests.oracle_pool import measure_image_parallel
    c = pfsynth.IMAGE224
    pair = pfsynth.cached(pfsynth.speckle_pair, 0, with_masks=True)
    N, K, lr, lt, seed = c["n_particles"], c["n_iters"], np.deg2rad(c["rot_limit_deg"]), c["trans_limit"], c["seed"]
    lim = np.array([lr] * 3 + [lt] * 3, np.float32)
    nmin = int(float(np.float32(0.01)) * pair.tgt.size)
    with _reg(pk, "image_ncc", pair, N, lr, lt, seed, autotune=True) as reg:
        prev_next = None
        for k in range(K):
            reg.step(1)
            st = reg.state()
            x = st["poses_measured"]
            if k == 0:
                assert np.array_equal(x, orc.init_particles(N, seed, lim))
            else:
                assert np.array_equal(x, orc.perturb(prev_next, seed, k, orc.sigma(0.25, 0.8, k, lim), lim))
            if k in (0, K - 1):
                sample = np.sort(np.random.default_rng(k).choice(N, 32, replace=False))
                mats, a = orc.pose_matrices(x[:, sample], pair.src_dims, pair.src_origin, pair.tgt_origin)
                mom, f64 = measure_image_parallel(pair.src, pair.tgt, mats, a)
                assert np.array_equal(st["moments"][sample, 0:7], mom), f"moments differ at k={k}"
                for j, i in enumerate(sample):
                    assert abs(st["scores"][i] - f64[j]) <= NCC_RTOL * f64[j], (k, i)
            s = np.array([orc.score("image_ncc", m, 0, nmin) for m in st["moments"]])
            assert np.array_equal(st["scores"], s)
            W = orc.weights(s, 5)
            assert np.array_equal(st["weights"], W)
            idx = orc.resample(W, orc.resample_offset(seed, k))
            assert np.array_equal(st["resample_idx"], idx)
            assert np.array_equal(st["poses_next"], x[:, idx])
            est = orc.estimate(x, W)
            log_est, _, _, log_evals, _ = reg.log()
            assert log_evals[-1] == int(st["moments"][:, 0].sum())
            assert np.all(np.abs(log_est[-1] - est) <= np.array([ROT_TOL] * 3 + [TRANS_TOL] * 3))
            prev_next = st["poses_next"]


def test_image224_small_cloud_trajectory_bit_exact(pk, orc):
    """The whole filter on the full 224x208x176 pair against the oracle's own
    run (N = 64, 3 iterations, +-30 deg / +-25 voxels, tuned tile shape):
    particles, moments, scores, weights and resampled indices bit for bit at
    every iteration, the estimate within 1e-4 rad / 1e-3 voxel."""
    c = pfsynth.IMAGE224
    pair = pfsynth.cached(pfsynth.speckle_pair, 0, with_masks=True)
    N, K, lr, lt, seed = 64, 3, np.deg2rad(c["rot_limit_deg"]), c["trans_limit"], c["seed"]
    ref = _oracle_run(orc, "image_ncc", pair, N, K, lr, lt, seed)
    with _reg(pk, "image_ncc", pair, N, lr, lt, seed, autotune=True) as reg:
        _assert_trajectory(reg, ref, K)


# ------------------------------------------------------------------- warp

@pytest.mark.parametrize("interp", [0, 1])
def test_warp_sequence_bit_exact(pk, orc, interp):
    import torch
    sd, td = (37, 30, 23), (41, 29, 26)
    so, to = np.array([0, 0, 0], np.float32), np.array([4.0, -2.0, 3.0], np.float32)
    frames = np.stack([pfsynth.random_image(s, sd) for s in range(70)])   # > 64: two launches
    fin = [_cuda(f) for f in frames]
    fout = [torch.empty((td[2], td[1], td[0]), dtype=torch.uint8, device="cuda") for _ in frames]
    pose = np.array([0.3, -0.2, 0.4, 2.5, -1.25, 0.75], np.float32)
    pk.warp_sequence(fin, sd, so, fout, td, to, pose, interp)
    torch.cuda.synchronize()
    for i in (0, 1, 63, 64, 69):
        want = orc.warp(frames[i], so, td, to, pose, interp)
        assert np.array_equal(fout[i].cpu().numpy(), want), i


def test_warp_identity_and_rot90(pk):
    import torch
    v = pfsynth.random_image(3, (21, 18, 13))
    out = torch.empty_like(_cuda(v))
    pk.warp_sequence([_cuda(v)], (21, 18, 13), (0, 0, 0), [out], (21, 18, 13), (0, 0, 0), np.zeros(6), 1)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), v)


def test_warp_image224_frame_full_size(pk, orc):
    import torch
    pair = pfsynth.cached(pfsynth.speckle_pair, 0)
    frames = pfsynth.cached(pfsynth.frame_sequence, pair, 3)
    fin = [_cuda(f) for f in frames]
    fout = [torch.empty(pair.tgt.shape, dtype=torch.uint8, device="cuda") for _ in fin]
    pose = pair.true_pose
    pk.warp_sequence(fin, pair.src_dims, pair.src_origin, fout, pair.tgt_dims, pair.tgt_origin, pose, 1)
    torch.cuda.synchronize()
    want = orc.warp(frames[1], pair.src_origin, pair.tgt_dims, pair.tgt_origin, pose, 1)
    assert np.array_equal(fout[1].cpu().numpy(), want)


def test_kernel_launches_are_counted(pk):
    before = pk.pf_kernel_launches()
    pair = pfsynth.ellipsoid_pair(2, src_dims=(16, 16, 16), tgt_dims=(16, 16, 12), tgt_origin=(0, 0, 4),
                                  semi_axes=(6, 4, 4))
    with _reg(pk, "mask_dice", pair, 32, 0.2, 2.0, 1) as reg:
        reg.step(4)
        reg.estimate(False)
    assert pk.pf_kernel_launches() - before >= 12


@pytest.mark.parametrize("mode", ["image_ncc", "mask_dice"])
def test_estimate_dice_trace(pk, orc, mode):
    """Sec. 3.2: the masks are warped with the estimate after every iteration
    and their Dice is logged.  The traced Dice equals the oracle's Dice at the
    same fp32 estimate, and tracing leaves the filter's trajectory unchanged."""
    pair = pfsynth.speckle_pair(11, src_dims=(40, 36, 32), tgt_dims=(39, 35, 30), overlap=(0.6, 0.7),
                                max_rot_deg=8, max_trans=3, with_masks=True)
    N, K, lr, lt = 128, 6, 0.2, 4.0
    ref = _oracle_run(orc, mode, pair, N, K, lr, lt, seed=5)
    with _reg(pk, mode, pair, N, lr, lt, 5, trace_estimate=True,
              **({"src_mask": _cuda(pair.src_mask), "tgt_mask": _cuda(pair.tgt_mask)}
                 if mode == "image_ncc" else {})) as reg:
        _assert_trajectory(reg, ref, K)
        est, _, _, _, dice = reg.log()
    assert len(dice) == K and np.all(dice >= 0)
    bfull = int((pair.tgt_mask != 0).sum())
    for k in range(K):
        M, a = orc.pose_matrix(est[k].astype(np.float32), pair.src_dims, pair.src_origin, pair.tgt_origin)
        c = orc.measure_mask(pair.src_mask, pair.tgt_mask, M, a)[0]
        assert dice[k] == orc.dice_from_counts(c[0], c[1], c[3], bfull, 0), k


def test_combined256_full_size_sampled(pk, orc):
    """The combined stress workload at full size (256^3 image + LV mask,
    N=16384, +-45 deg / +-32 voxels, score 0.5 (NCC^2 + Dice)): one iteration
    on the GPU; the oracle re-measures sampled particles (image moments and
    mask counts) and recomputes every cheap step on the GPU's state."""
    c = pfsynth.COMBINED256
    pair = pfsynth.cached(pfsynth.speckle_pair, 0, src_dims=(256, 256, 256), with_masks=True,
                          max_rot_deg=20.0, max_trans=15.0)
    N, lr, lt, seed = c["n_particles"], np.deg2rad(c["rot_limit_deg"]), c["trans_limit"], c["seed"]
    lim = np.array([lr] * 3 + [lt] * 3, np.float32)
    nmin = int(float(np.float32(0.01)) * pair.tgt.size)
    bfull = int((pair.tgt_mask != 0).sum())
    with _reg(pk, "combined", pair, N, lr, lt, seed) as reg:
        reg.step(1)
        st = reg.state()
        x = st["poses_measured"]
        assert np.array_equal(x, orc.init_particles(N, seed, lim))
        sample = np.random.default_rng(4).choice(N, 3, replace=False)
        mats, a = orc.pose_matrices(x[:, sample], pair.src_dims, pair.src_origin, pair.tgt_origin)
        assert np.array_equal(st["moments"][sample, 0:7], orc.measure_image(pair.src, pair.tgt, mats, a))
        assert np.array_equal(st["moments"][sample, 8:12], orc.measure_mask(pair.src_mask, pair.tgt_mask, mats, a))
        s = np.array([orc.score("combined", m, bfull, nmin) for m in st["moments"]])
        assert np.array_equal(st["scores"], s)
        W = orc.weights(s, 5)
        assert np.array_equal(st["weights"], W)
        idx = orc.resample(W, orc.resample_offset(seed, 0))
        assert np.array_equal(st["resample_idx"], idx)
        assert np.array_equal(st["poses_next"], x[:, idx])


# ------------------------------------------------- anisotropic voxels (Table 1)

SP_SRC, SP_TGT = (0.87, 1.08, 0.73), (1.09, 1.30, 0.92)


def test_pose_matrix_with_spacing_bit_exact(pk, orc):
    rng = np.random.default_rng(11)
    for i in range(100):
        pose = np.concatenate([rng.uniform(-1.5, 1.5, 3), rng.uniform(-30, 30, 3)]).astype(np.float32)
        sd = tuple(int(v) for v in rng.integers(2, 300, 3))
        so, to = rng.uniform(-20, 20, 3).astype(np.float32), rng.uniform(-20, 20, 3).astype(np.float32)
        ss, ts = rng.uniform(0.3, 3.0, 3).astype(np.float32), rng.uniform(0.3, 3.0, 3).astype(np.float32)
        Mg, ag = pk.pf_pose_matrix(pose, sd, so, to, ss, ts)
        Mo, ao = orc.pose_matrix(pose, sd, so, to, ss, ts)
        assert np.array_equal(Mg, Mo) and np.array_equal(ag, ao), i


@pytest.mark.parametrize("mode", ["mask_dice", "image_ncc"])
def test_trajectory_with_spacing_bit_exact(pk, orc, mode):
    if mode == "mask_dice":
        pair = pfsynth.ellipsoid_pair(12, src_dims=(34, 28, 36), tgt_dims=(30, 24, 27), tgt_origin=(0, 0, 6),
                                      semi_axes=(10, 7, 7), asymmetric=True, max_rot_deg=8, max_trans=3,
                                      src_spacing=SP_SRC, tgt_spacing=SP_TGT)
    else:
        pair = pfsynth.speckle_pair(12, src_dims=(36, 34, 30), tgt_dims=(37, 33, 29), overlap=(0.55, 0.7),
                                    max_rot_deg=8, max_trans=3)
    N, K, lr, lt = 160, 4, 0.2, 4.0
    ref = _oracle_run(orc, mode, pair, N, K, lr, lt, seed=21, src_spacing=SP_SRC, tgt_spacing=SP_TGT)
    with _reg(pk, mode, pair, N, lr, lt, 21, src_spacing=SP_SRC, tgt_spacing=SP_TGT) as reg:
        _assert_trajectory(reg, ref, K)


def test_warp_with_spacing_bit_exact(pk, orc):
    import torch
    sd, td = (37, 30, 23), (29, 25, 20)
    so, to = np.zeros(3, np.float32), np.array([3.0, -2.0, 2.5], np.float32)
    frames = [pfsynth.random_image(s, sd) for s in range(3)]
    fout = [torch.empty((td[2], td[1], td[0]), dtype=torch.uint8, device="cuda") for _ in frames]
    pose = np.array([0.2, -0.3, 0.25, 2.5, -1.25, 0.75], np.float32)
    for interp in (0, 1):
        pk.warp_sequence([_cuda(f) for f in frames], sd, so, fout, td, to, pose, interp, src_spacing=SP_SRC,
                         tgt_spacing=SP_TGT)
        torch.cuda.synchronize()
        for i, f in enumerate(frames):
            want = orc.warp(f, so, td, to, pose, interp, SP_SRC, SP_TGT)
            assert np.array_equal(fout[i].cpu().numpy(), want), (interp, i)


# ------------------------------------------------------ quaternion estimator

@pytest.mark.parametrize("mode", ["mask_dice", "image_ncc"])
def test_quaternion_estimator_against_oracle(pk, orc, mode):
    if mode == "mask_dice":
        pair = pfsynth.ellipsoid_pair(14, src_dims=(30, 28, 26), tgt_dims=(33, 27, 21), tgt_origin=(0, 0, 6),
                                      semi_axes=(10, 7, 6), asymmetric=True, max_rot_deg=8, max_trans=3)
    else:
        pair = pfsynth.speckle_pair(14, src_dims=(36, 34, 30), tgt_dims=(37, 33, 29), overlap=(0.55, 0.7),
                                    max_rot_deg=8, max_trans=3)
    N, K, lr, lt = 300, 5, 0.6, 4.0
    ref = _oracle_run(orc, mode, pair, N, K, lr, lt, seed=5)
    with _reg(pk, mode, pair, N, lr, lt, 5, estimator="quaternion") as rq, _reg(pk, mode, pair, N, lr, lt, 5) as rm:
        rq.step(K)
        rm.step(K)
        a, b = rq.state(), rm.state()
        for key in a:   # the estimator does not touch the cloud
            assert np.array_equal(a[key], b[key]), key
        est, _, _, _, _ = rq.log()
    for k in range(K):
        want = orc.estimate_quaternion(ref["tr_poses"][k], ref["tr_W"][k])
        assert np.max(np.abs(est[k] - want)) <= 1e-9, (k, est[k] - want)


# ------------------------------------------------------------- fault paths

def test_allocation_failure_is_reported_and_released(pk):
    """Host-side fault injection: with a cap on a context's device bytes,
    creation fails with PF_ENOMEM (no fault, nothing leaked), and works again
    once the cap is lifted."""
    import torch
    src = pfsynth.random_mask(3, (40, 40, 40), 0.4)
    free0 = torch.cuda.mem_get_info()[0]
    pk.pf_debug_alloc_limit(4096)
    try:
        with pytest.raises(pk.PfError) as ei:
            pk.Registration("mask_dice", src_mask=src, tgt_mask=src, n_particles=256)
        assert ei.value.code == -2
    finally:
        pk.pf_debug_alloc_limit(0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)
    with pk.Registration("mask_dice", src_mask=src, tgt_mask=src, n_particles=256) as r:
        r.step(1)


def test_bounded_wait_reports_instead_of_hanging(pk):
    """A device-side wait that nothing satisfies gives up after its bound and
    sets the flag the host reads; the context stays usable."""
    import torch
    assert pk.nn_status(clear=True) == 0
    pk.nn_wait_selftest()
    torch.cuda.synchronize()
    assert pk.nn_status(clear=True) == 1
    assert pk.nn_status(clear=True) == 0
    x = torch.ones(4, device="cuda")
    assert float((x * 2).sum()) == 8.0
