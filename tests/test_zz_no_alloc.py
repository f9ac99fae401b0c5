"""pf_measure_matrices_noalloc: the measurement entry point for callers that
cannot allocate device memory while they run (a loop that must not stall on
the allocator or fail midway, or a fixed memory budget after start-up).

Its output must equal pf_measure_matrices' output and the oracle's moments
bit for bit (the tolerance the other moment tests use), on consecutive calls
that share the fixed scratch array; it must make no device allocation, and it
must reject batches larger than that array.  This file sorts last so a run
that stops at the first failure has run every other test.
"""
import numpy as np
import pytest

import oracle as orc
import pfsynth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2504_19930_gb300 as pk
    pk.build()
    pk.load()
    return pk


def _matrices(pk, n, sdims, so, to, seed):
    rng = np.random.default_rng(seed)
    poses = np.concatenate([rng.uniform(-0.5, 0.5, (n, 3)), rng.uniform(-6, 6, (n, 3))], 1).astype(np.float32)
    mats, a = [], None
    for p in poses:
        M, a = pk.pf_pose_matrix(p, sdims, so, to)
        mats.append(M)
    return np.stack(mats), a


@pytest.mark.parametrize("mode", ["image_ncc", "mask_dice", "combined"])
def test_noalloc_matches_allocating_entry_point(pk, mode):
    import torch
    sd, td = (41, 36, 30), (39, 34, 28)
    so, to = np.zeros(3, np.float32), np.array([1.0, -2.0, 1.5], np.float32)
    img_s, img_t = pfsynth.random_image(3, sd), pfsynth.random_image(4, td)
    msk_s, msk_t = pfsynth.random_mask(5, sd, 0.4), pfsynth.random_mask(6, td, 0.4)
    vols = {}
    if mode in ("image_ncc", "combined"):
        vols.update(src=torch.from_numpy(img_s).cuda(), tgt=torch.from_numpy(img_t).cuda())
    if mode in ("mask_dice", "combined"):
        vols.update(src_mask=torch.from_numpy(msk_s).cuda(), tgt_mask=torch.from_numpy(msk_t).cuda())
    with pk.Registration(mode, src_origin=so, tgt_origin=to, n_particles=16, **vols) as reg:
        mats_a, a = _matrices(pk, 300, sd, so, to, seed=1)
        mats_b, _ = _matrices(pk, 120, sd, so, to, seed=2)
        want_a = pk.pf_measure_matrices(reg.ctx, mats_a, a)
        want_b = pk.pf_measure_matrices(reg.ctx, mats_b, a)
        got_a1 = pk.pf_measure_matrices_noalloc(reg.ctx, mats_a, a)
        allocs = pk.pf_debug_device_allocs()
        got_a2 = pk.pf_measure_matrices_noalloc(reg.ctx, mats_a, a)      # second call, same scratch
        got_b = pk.pf_measure_matrices_noalloc(reg.ctx, mats_b, a)       # fewer matrices after more
        assert pk.pf_debug_device_allocs() == allocs, "the no-alloc entry point allocated device memory"
        assert np.any(want_a != 0)
        assert np.array_equal(got_a1, want_a)
        assert np.array_equal(got_a2, want_a)
        assert np.array_equal(got_b, want_b)
    # the moments themselves, against the oracle (not only against the other entry point)
    if mode in ("image_ncc", "combined"):
        assert np.array_equal(got_a2[:, 0:7], orc.measure_image(img_s, img_t, mats_a, a))
        assert np.array_equal(got_b[:, 0:7], orc.measure_image(img_s, img_t, mats_b, a))
    if mode in ("mask_dice", "combined"):
        assert np.array_equal(got_a2[:, 8:12], orc.measure_mask(msk_s, msk_t, mats_a, a))
        assert np.array_equal(got_b[:, 8:12], orc.measure_mask(msk_s, msk_t, mats_b, a))


def test_allocating_calls_are_counted(pk):
    """The allocation counter the no-alloc test relies on does see allocations:
    the allocating entry point grows its scratch for a larger batch."""
    import torch
    v = torch.from_numpy(pfsynth.random_mask(8, (12, 11, 10), 0.4)).cuda()
    with pk.Registration("mask_dice", src_mask=v, tgt_mask=v, n_particles=4) as reg:
        eye = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
        pk.pf_measure_matrices(reg.ctx, np.tile(eye, (2, 1)), np.zeros(3, np.float32))
        before = pk.pf_debug_device_allocs()
        pk.pf_measure_matrices(reg.ctx, np.tile(eye, (64, 1)), np.zeros(3, np.float32))
        assert pk.pf_debug_device_allocs() > before


def test_noalloc_rejects_batches_beyond_its_scratch(pk):
    import torch
    v = torch.from_numpy(pfsynth.random_mask(7, (12, 11, 10), 0.4)).cuda()
    with pk.Registration("mask_dice", src_mask=v, tgt_mask=v, n_particles=4) as reg:
        mats = np.tile(np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32),
                       (pk.NOALLOC_MAX_MATRICES + 1, 1))
        with pytest.raises(pk.PfError) as err:
            pk.pf_measure_matrices_noalloc(reg.ctx, mats, np.zeros(3, np.float32))
        assert err.value.code == -1 and "4096" in str(err.value)
        full = pk.pf_measure_matrices_noalloc(reg.ctx, mats[:pk.NOALLOC_MAX_MATRICES], np.zeros(3, np.float32))
        assert np.all(full[:, 8] == 12 * 11 * 10)
