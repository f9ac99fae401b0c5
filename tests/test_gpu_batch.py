"""Batches of registrations (one graph per iteration over all of them) give
bit for bit the results of stepping every registration on its own, which the
single-registration tests tie to the oracle; two members are also checked
against the oracle directly."""
import numpy as np
import pytest

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


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# (mode, pair maker, N, K, seed): uneven sizes, particle counts and iteration counts
def _members():
    return [
        ("mask_dice", pfsynth.ellipsoid_pair(21, src_dims=(30, 28, 26), tgt_dims=(31, 27, 20),
                                             tgt_origin=(0, 0, 6), semi_axes=(10, 7, 6), asymmetric=True),
         96, 5, 1),
        ("image_ncc", pfsynth.speckle_pair(22, src_dims=(41, 37, 33), overlap=(0.55, 0.7), max_rot_deg=6,
                                           max_trans=2), 150, 3, 2),
        ("combined", pfsynth.speckle_pair(23, src_dims=(36, 34, 30), overlap=(0.6, 0.7), max_rot_deg=6,
                                          max_trans=2, with_masks=True), 64, 6, 3),
        ("mask_ncc", pfsynth.ellipsoid_pair(24, src_dims=(26, 24, 22), tgt_dims=(25, 24, 18),
                                            tgt_origin=(0, 0, 4), semi_axes=(9, 6, 5)), 33, 4, 4),
        ("image_ncc", pfsynth.speckle_pair(25, src_dims=(29, 31, 27), overlap=(0.6, 0.7), max_rot_deg=6,
                                           max_trans=2), 200, 0, 5),
        ("mask_dice", pfsynth.ellipsoid_pair(26, src_dims=(70, 66, 60), tgt_dims=(68, 60, 50),
                                             tgt_origin=(0, 0, 10), semi_axes=(22, 15, 14)), 128, 2, 6),
        # members large enough for their own measurement launch inside the batch graph
        ("mask_dice", pfsynth.ellipsoid_pair(27, src_dims=(40, 38, 36), tgt_dims=(40, 38, 30),
                                             tgt_origin=(0, 0, 6), semi_axes=(13, 9, 8), asymmetric=True),
         4096, 3, 7),
        ("combined", pfsynth.speckle_pair(28, src_dims=(40, 36, 34), overlap=(0.6, 0.7), max_rot_deg=6,
                                          max_trans=2, with_masks=True), 4096, 2, 8),
    ]


# a member with at least this many measurement work items (32 target rows of
# one particle each) is measured by its own launch in the batch graph
SOLO_ITEMS = 120000


def _items(pair, N):
    rows = pair.tgt.shape[0] * pair.tgt.shape[1]
    return (rows + 31) // 32 * N


def _make(pk, mode, pair, N, seed, **cfg):
    vols = {}
    if mode in ("image_ncc", "combined"):
        vols.update(src=_cuda(pair.src), tgt=_cuda(pair.tgt))
    if mode != "image_ncc":
        vols.update(src_mask=_cuda(pair.src_mask), tgt_mask=_cuda(pair.tgt_mask))
    return pk.Registration(mode, src_origin=pair.src_origin, tgt_origin=pair.tgt_origin, n_particles=N,
                           rot_limit=0.2, trans_limit=3.0, seed=seed, **vols, **cfg)


def _snapshot(reg):
    st = reg.state()
    est, best, ess, evals, _ = reg.log()
    return st, est, best, evals, reg.iteration


def _assert_same(a, b, tag):
    st_a, est_a, best_a, ev_a, k_a = a
    st_b, est_b, best_b, ev_b, k_b = b
    assert k_a == k_b, tag
    for key in st_a:
        assert np.array_equal(st_a[key], st_b[key]), (tag, key)
    assert np.array_equal(best_a, best_b) and np.array_equal(ev_a, ev_b), tag
    assert np.max(np.abs(est_a - est_b), initial=0.0) <= 1e-9, tag   # fp64 sums: reduction order


def test_batch_equals_individual_registrations(pk):
    members = _members()
    sizes = [_items(pair, N) for mode, pair, N, K, seed in members]
    assert any(n >= SOLO_ITEMS for n in sizes) and any(n < SOLO_ITEMS for n in sizes)   # both launch forms
    singles = []
    for mode, pair, N, K, seed in members:
        with _make(pk, mode, pair, N, seed) as r:
            r.step(K)
            singles.append(_snapshot(r))
    regs = [_make(pk, mode, pair, N, seed) for mode, pair, N, K, seed in members]
    with pk.Batch(regs, [m[3] for m in members]) as b:
        b.run()
    for i, r in enumerate(regs):
        _assert_same(_snapshot(r), singles[i], f"member {i} ({members[i][0]})")
        r.close()


def test_batch_in_parts_and_against_the_oracle(pk, orc):
    members = _members()[:3]
    regs = [_make(pk, mode, pair, N, seed) for mode, pair, N, K, seed in members]
    with pk.Batch(regs, [m[3] for m in members]) as b:
        b.step(2)
        assert [r.iteration for r in regs] == [2, 2, 2]
        b.run()
    assert [r.iteration for r in regs] == [m[3] for m in members]
    for (mode, pair, N, K, seed), r in zip(members, regs):
        kw = {}
        if mode in ("image_ncc", "combined"):
            kw.update(src=pair.src, tgt=pair.tgt)
        if mode != "image_ncc":
            kw.update(src_mask=pair.src_mask, tgt_mask=pair.tgt_mask)
        ref = orc.register(mode, pair.src_dims, pair.src_origin, pair.tgt_dims, pair.tgt_origin, N, K, 0.2, 3.0,
                           seed=seed, **kw)
        st = r.state()
        assert np.array_equal(st["poses_measured"], ref["tr_poses"][-1])
        assert np.array_equal(st["moments"], ref["tr_mom"][-1])
        assert np.array_equal(st["resample_idx"], ref["tr_idx"][-1])
        assert np.array_equal(st["poses_next"], ref["poses"])
        r.close()


def test_batch_rejects_bad_membership(pk):
    pair = _members()[0][1]
    r = _make(pk, "mask_dice", pair, 16, 1)
    with pytest.raises(pk.PfError):
        pk.pf_batch_create([r.ctx, r.ctx], [1, 1])
    with pytest.raises(pk.PfError):
        pk.pf_batch_create([r.ctx], [-1])
    r.close()


CANDIDATES = (1, 2, 4, 8, 16, 32)


def test_autotuned_tile_shape_changes_no_result(pk):
    """The autotuner only picks how work items are spread over warps; every
    registration and every batch member gives the same bits as with the
    default tile shape."""
    members = _members()
    singles = []
    for mode, pair, N, K, seed in members:
        with _make(pk, mode, pair, N, seed) as r:
            assert r.tile_shape() == (32, 8)
            r.step(K)
            singles.append(_snapshot(r))
    for i, (mode, pair, N, K, seed) in enumerate(members):
        with _make(pk, mode, pair, N, seed, autotune=True) as r:
            assert r.tile_shape()[1] in CANDIDATES
            assert r.iteration == 0 and not r.state()["moments"].any()
            r.step(K)
            _assert_same(_snapshot(r), singles[i], f"tuned member {i}")
    regs = [_make(pk, mode, pair, N, seed, autotune=True) for mode, pair, N, K, seed in members]
    with pk.Batch(regs, [m[3] for m in members]) as b:
        assert b.tile_shape() in CANDIDATES
        b.run()
    for i, r in enumerate(regs):
        _assert_same(_snapshot(r), singles[i], f"tuned batch member {i} ({members[i][0]})")
        r.close()
