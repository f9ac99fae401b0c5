"""The two half-iterations of the C ABI (pf_step_measure / pf_step_update) on
the GPU: two contexts standing for two ranks measure disjoint particle
slices, their moment buffers are summed (what the all-reduce does between
processes) and both update; every iteration's state must equal pf_step's on
a third context bit for bit.  Both "ranks" run on one stream in turn: nothing
waits on another launch."""
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


def _make(pk, mode, pair, N, seed, trace=False):
    vols = {}
    if mode in ("image_ncc", "combined"):
        vols.update(src=_cuda(pair.src), tgt=_cuda(pair.tgt))
    if mode != "image_ncc":
        vols.update(src_mask=_cuda(pair.src_mask), tgt_mask=_cuda(pair.tgt_mask))
    return pk.Registration(mode, src_origin=pair.src_origin, tgt_origin=pair.tgt_origin, n_particles=N,
                           rot_limit=0.2, trans_limit=3.0, seed=seed, trace_estimate=trace, **vols)


CASES = [
    ("mask_dice", lambda: pfsynth.ellipsoid_pair(31, src_dims=(30, 28, 26), tgt_dims=(31, 27, 20),
                                                 tgt_origin=(0, 0, 6), semi_axes=(10, 7, 6),
                                                 asymmetric=True), 101, True),
    ("image_ncc", lambda: pfsynth.speckle_pair(32, src_dims=(41, 37, 33), overlap=(0.55, 0.7),
                                               max_rot_deg=6, max_trans=2), 150, False),
    ("combined", lambda: pfsynth.speckle_pair(33, src_dims=(36, 34, 30), overlap=(0.6, 0.7), max_rot_deg=6,
                                              max_trans=2, with_masks=True), 64, True),
]


@pytest.mark.parametrize("mode,maker,N,trace", CASES, ids=[c[0] for c in CASES])
def test_two_slices_summed_equal_pf_step(pk, mode, maker, N, trace):
    import torch
    pair = maker()
    one = _make(pk, mode, pair, N, 9, trace)
    ra, rb = _make(pk, mode, pair, N, 9, trace), _make(pk, mode, pair, N, 9, trace)
    ma, mb = ra.moments(), rb.moments()
    assert ma.dtype == torch.int64 and ma.numel() == 12 * N and ma.is_cuda
    h = N // 3
    for k in range(4):
        ra.step_measure(0, h)
        rb.step_measure(h, N)
        total = ma + mb
        ma.copy_(total)
        mb.copy_(total)
        ra.step_update()
        rb.step_update()
        one.step(1)
        ref = one.state()
        for r in (ra, rb):
            st = r.state()
            for key in ref:
                assert np.array_equal(st[key], ref[key]), (k, key)
    est_ref, best_ref, _, evals_ref, dice_ref = one.log()
    for r in (ra, rb):
        est, best, _, evals, dice = r.log()
        assert np.array_equal(best, best_ref) and np.array_equal(evals, evals_ref)
        assert np.max(np.abs(est - est_ref)) <= 1e-9
        if trace:
            assert np.array_equal(dice, dice_ref)
    for r in (one, ra, rb):
        r.close()


def test_driver_with_one_rank_equals_pf_step(pk):
    from paper_2504_19930_gb300.shard import ShardedRegistration
    pair = CASES[0][1]()
    one = _make(pk, "mask_dice", pair, 77, 4)
    one.step(3)
    r = _make(pk, "mask_dice", pair, 77, 4)
    ShardedRegistration(r, 0, 1, all_reduce_sum=lambda t: None).step(3)
    a, b = one.state(), r.state()
    for key in a:
        assert np.array_equal(a[key], b[key]), key
    one.close()
    r.close()


def test_slice_arguments_are_checked(pk):
    pair = CASES[0][1]()
    r = _make(pk, "mask_dice", pair, 16, 1)
    for lo, hi in ((-1, 4), (5, 4), (0, 17)):
        with pytest.raises(pk.PfError):
            r.step_measure(lo, hi)
    r.step_measure(0, 0)           # an empty slice is allowed
    r.step_update()
    assert r.iteration == 1
    r.close()
