"""The sharded iteration (measurement split over ranks, moment buffers summed,
update repeated on every rank) on CPU: two and three gloo ranks drive
:class:`ShardedRegistration` over a stand-in registration whose two halves
are the oracle's step functions, and every rank must end with the cloud the
oracle's own single-process loop produces."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_slice_bounds_partition_the_particles():
    from paper_2504_19930_gb300.shard import slice_bounds
    for N in (1, 2, 7, 64, 1000, 65536):
        for world in (1, 2, 3, 8):
            b = [slice_bounds(N, r, world) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == N
            assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in b]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slice_bounds(10, 2, 2)


class OracleHalves:
    """A registration whose two half-iterations are the oracle's steps
    (mask Dice mode), with the moment buffer as an int64 CPU tensor."""

    def __init__(self, orc, pair, N, seed, rot, trans):
        import torch
        self.orc, self.pair, self.N, self.seed = orc, pair, N, seed
        self.lim = np.array([rot] * 3 + [trans] * 3, np.float32)
        self.k = 0
        self.x = orc.init_particles(N, seed, self.lim)
        self.mom = torch.zeros(12 * N, dtype=torch.int64)
        nt = int(np.prod(pair.tgt_dims))
        self.n_min = int(np.float64(np.float32(0.01)) * nt)
        self.b_full = int((pair.tgt_mask != 0).sum())

    def moments(self):
        return self.mom

    def step_measure(self, lo, hi):
        import torch
        o, p = self.orc, self.pair
        if self.k > 0:
            self.x = o.perturb(self.x, self.seed, self.k, o.sigma(0.25, 0.8, self.k, self.lim), self.lim)
        mats, a = o.pose_matrices(self.x, p.src_dims, p.src_origin, p.tgt_origin)
        self.mom.zero_()
        if hi > lo:
            counts = o.measure_mask(p.src_mask, p.tgt_mask, mats[lo:hi], a).astype(np.int64)
            self.mom.view(self.N, 12)[lo:hi, 8:12] = torch.from_numpy(counts)

    def step_update(self):
        o = self.orc
        m = self.mom.view(self.N, 12).numpy().astype(np.uint64)
        s = np.array([o.score("mask_dice", m[i], self.b_full, self.n_min) for i in range(self.N)])
        W = o.weights(s, 5)
        idx = o.resample(W, o.resample_offset(self.seed, self.k))
        self.x = np.ascontiguousarray(self.x[:, idx])
        self.k += 1


def _pair():
    import pfsynth
    return pfsynth.ellipsoid_pair(11, src_dims=(20, 18, 16), tgt_dims=(21, 17, 14), tgt_origin=(0, 0, 3),
                                  semi_axes=(7, 5, 4), asymmetric=True)


N_PART, K_ITERS, SEED, ROT, TRANS = 37, 3, 5, 0.2, 3.0


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle
    from paper_2504_19930_gb300.shard import ShardedRegistration
    dist.init_process_group("gloo", rank=rank, world_size=world)
    reg = OracleHalves(oracle, _pair(), N_PART, SEED, ROT, TRANS)
    ShardedRegistration(reg, rank, world).step(K_ITERS)
    dist.destroy_process_group()
    out.put((rank, reg.x.copy()))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_shard_the_measurement(orc, world):
    p = _pair()
    ref = orc.register("mask_dice", p.src_dims, p.src_origin, p.tgt_dims, p.tgt_origin, N_PART, K_ITERS,
                       ROT, TRANS, seed=SEED, src_mask=p.src_mask, tgt_mask=p.tgt_mask, trace=False)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, x in res:
        assert np.array_equal(x, ref["poses"]), rank


def test_single_rank_without_a_process_group(orc):
    p = _pair()
    from paper_2504_19930_gb300.shard import ShardedRegistration
    reg = OracleHalves(orc, p, N_PART, SEED, ROT, TRANS)
    ShardedRegistration(reg, 0, 1, all_reduce_sum=lambda t: None).step(K_ITERS)
    ref = orc.register("mask_dice", p.src_dims, p.src_origin, p.tgt_dims, p.tgt_origin, N_PART, K_ITERS,
                       ROT, TRANS, seed=SEED, src_mask=p.src_mask, tgt_mask=p.tgt_mask, trace=False)
    assert np.array_equal(reg.x, ref["poses"])
