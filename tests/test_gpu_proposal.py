"""The learned proposal network on the GPU against its float64 oracle
(oracle/nn.py), and the proposal-seeded filter against the C oracle."""
import numpy as np
import pytest

from oracle import nn as onn

pytestmark = pytest.mark.gpu

ROT, TRANS = 0.5235988, 25.0
DIMS = (96, 80, 72)   # small synthetic volumes keep the generator quick


@pytest.fixture(scope="module")
def torch_():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def pk():
    import paper_2504_19930_gb300 as pk
    pk.build()
    pk.load()
    return pk


def _bf16_host(torch, t):
    return onn.from_bf16_bits(t.view(torch.int16).cpu().numpy().view(np.uint16))


def _batch(torch, pk, net, B, seed=3, step=0):
    x = torch.zeros((B, 64, 64, 64, 2), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros((B, 6), dtype=torch.float32, device="cuda")
    net.synth(x, y, seed, step, DIMS, ROT, TRANS)
    torch.cuda.synchronize()
    return x, y


def test_synthetic_batch_is_well_formed(torch_, pk):
    torch = torch_
    net = pk.Proposal(max_batch=4, seed=1)
    x, y = _batch(torch, pk, net, 4)
    xs, ys = _bf16_host(torch, x), y.cpu().numpy()
    assert np.all(np.abs(ys) <= 1.0) and np.std(ys) > 0.2
    assert np.all(xs >= 0) and np.all(np.isfinite(xs))
    # the source channel covers the whole box; the target channel, slid along
    # +x by 40-65 % of X, is empty over the first 40 % of the cells in x
    assert np.all(xs[..., 0].mean(axis=(1, 2, 3)) > 0.05)
    assert np.all(xs[:, :, :, : int(0.39 * 64), 1] == 0.0)
    assert np.all(xs[:, :, :, -8:, 1].mean(axis=(1, 2, 3)) > 0.05)
    x2, y2 = _batch(torch, pk, net, 4)
    assert torch.equal(x, x2) and torch.equal(y, y2)           # seeded
    x3, _ = _batch(torch, pk, net, 4, step=1)
    assert not torch.equal(x, x3)


def test_forward_matches_oracle(torch_, pk):
    torch = torch_
    B = 2
    net = pk.Proposal(max_batch=B, seed=5)
    theta = net.params()
    x, _ = _batch(torch, pk, net, B, seed=11)
    out = torch.zeros((B, 12), dtype=torch.float32, device="cuda")
    hid = torch.zeros((B, 128), dtype=torch.float32, device="cuda")
    net.forward(x, out, hid)
    torch.cuda.synchronize()
    want, h_want, _ = onn.net_forward(theta, _bf16_host(torch, x))
    got = out.cpu().numpy()
    scale = np.abs(want).max()
    assert np.max(np.abs(got - want)) <= 2e-2 * scale, (got, want)
    assert np.max(np.abs(hid.cpu().numpy() - h_want)) <= 2e-2 * np.abs(h_want).max()


def test_backward_matches_oracle(torch_, pk):
    torch = torch_
    B = 2
    net = pk.Proposal(max_batch=B, seed=6)
    x, y = _batch(torch, pk, net, B, seed=12)
    out = torch.zeros((B, 12), dtype=torch.float32, device="cuda")
    net.forward(x, out)
    loss = net.backward(y)
    theta, grad = net.params(with_grad=True)
    want_loss, want = onn.net_backward(theta, _bf16_host(torch, x), y.cpu().numpy())
    assert abs(loss - want_loss) <= 2e-2 * abs(want_loss)
    off, _ = onn.layout()
    for k, (o, sh) in off.items():
        n = int(np.prod(sh))
        g, w = grad[o:o + n].astype(np.float64), want[o:o + n]
        rel = np.linalg.norm(g - w) / max(np.linalg.norm(w), 1e-30)
        assert rel < 5e-2, f"{k}: relative gradient error {rel:.3g}"


def test_input_matches_box_average(torch_, pk):
    torch = torch_
    import pfsynth
    src = pfsynth.random_image(5, (70, 66, 67))
    tgt = pfsynth.random_image(6, (60, 72, 50))
    so, to = np.array([0.0, 0.0, 0.0], np.float32), np.array([20.0, -5.0, 3.0], np.float32)
    net = pk.Proposal(max_batch=1, seed=1)
    x = torch.zeros((1, 64, 64, 64, 2), dtype=torch.bfloat16, device="cuda")
    net.input(torch.from_numpy(src).cuda(), tgt, x, so, to)
    torch.cuda.synchronize()
    got = _bf16_host(torch, x)[0]
    h = np.array([70, 66, 67], np.float64) / 64.0
    for c, (v, o) in enumerate(((src, so), (tgt, to))):
        want = onn.box_average(v, o.astype(np.float64), np.ones(3), so.astype(np.float64), h)
        assert np.all(np.abs(got[..., c] - want) <= 2.0 ** -7 * np.abs(want) + 1e-6)   # fp32 mean, then bf16


def test_training_reduces_the_loss(torch_, pk):
    net = pk.Proposal(max_batch=16, seed=7)
    loss = net.train(300, batch=16, lr=1e-3, data_seed=5, vol_dims=DIMS, rot_limit=ROT, trans_limit=TRANS)
    assert np.all(np.isfinite(loss))
    assert pk.nn_status() == 0
    assert loss[-30:].mean() < loss[:30].mean() - 0.5, (loss[:30].mean(), loss[-30:].mean())


def test_seeded_filter_matches_oracle(torch_, pk):
    """pf_seed_gaussian + pf_step follow the oracle bit for bit: the seeded
    cloud, its perturbation scale and every iteration."""
    import oracle
    import pfsynth
    p = pfsynth.ellipsoid_pair(4, src_dims=(26, 24, 22), tgt_dims=(24, 22, 16), tgt_origin=(0, 0, 5),
                               semi_axes=(8, 6, 5), asymmetric=True, max_rot_deg=8, max_trans=2)
    N, K, lr_, lt = 128, 4, 0.3, 4.0
    mean = np.array([0.02, -0.03, 0.01, 0.5, -0.4, 0.2], np.float32)
    std = np.array([0.05, 0.04, 0.06, 1.0, 0.8, 1.2], np.float32)
    reg = pk.Registration("mask_dice", src_mask=p.src, tgt_mask=p.tgt, src_origin=p.src_origin,
                          tgt_origin=p.tgt_origin, n_particles=N, rot_limit=lr_, trans_limit=lt, seed=9)
    reg.seed_gaussian(mean, std)
    lim = np.array([lr_] * 3 + [lt] * 3, np.float32)
    x0 = oracle.init_gaussian(N, 9, mean, std, lim)
    ref = oracle.register("mask_dice", p.src_dims, p.src_origin, p.tgt_dims, p.tgt_origin, N, K, lr_, lt,
                          seed=9, src_mask=p.src, tgt_mask=p.tgt, poses=x0, sig_base=std)
    for k in range(K):
        reg.step(1)
        st = reg.state()
        assert np.array_equal(st["poses_measured"], ref["tr_poses"][k]), f"poses differ at k={k}"
        assert np.array_equal(st["moments"], ref["tr_mom"][k]), f"counts differ at k={k}"
        assert np.array_equal(st["resample_idx"], ref["tr_idx"][k]), f"indices differ at k={k}"
    with pytest.raises(Exception):
        reg.seed_gaussian(mean, std)        # only before the first iteration
    reg.close()


def test_predict_returns_a_finite_proposal(torch_, pk):
    import pfsynth
    net = pk.Proposal(max_batch=8, seed=8)
    net.train(20, batch=8, lr=1e-3, data_seed=2, vol_dims=DIMS, rot_limit=ROT, trans_limit=TRANS)
    p = pfsynth.speckle_pair(3, src_dims=DIMS)
    mean, std = net.predict(p.src, p.tgt, p.src_origin, p.tgt_origin)
    assert np.all(np.isfinite(mean)) and np.all(std > 0)


def test_checkpoint_round_trip_and_continued_training(torch_, pk):
    """Parameters saved from one network and loaded into another give the
    same outputs; training continues across calls with the step counter."""
    torch = torch_
    a = pk.Proposal(max_batch=4, seed=21)
    l1 = a.train(10, batch=4, lr=1e-3, data_seed=3, vol_dims=DIMS, rot_limit=ROT, trans_limit=TRANS)
    l2 = a.train(10, batch=4, lr=1e-3, data_seed=3, vol_dims=DIMS, rot_limit=ROT, trans_limit=TRANS)
    assert len(l1) == len(l2) == 10 and np.all(np.isfinite(l2))
    assert not np.array_equal(l1, l2)                  # new batches (the step counter moved on)
    theta = a.params()
    b = pk.Proposal(max_batch=4, seed=99)
    assert not np.array_equal(b.params(), theta)
    b.params(theta_in=theta)
    assert np.array_equal(b.params(), theta)
    x, _ = _batch(torch, pk, a, 4, seed=13)
    oa = torch.zeros((4, 12), dtype=torch.float32, device="cuda")
    ob = torch.zeros((4, 12), dtype=torch.float32, device="cuda")
    a.forward(x, oa)
    b.forward(x, ob)
    torch.cuda.synchronize()
    assert torch.equal(oa, ob)
    with pytest.raises(pk.PfError):                    # the output units are the training limits
        a.train(1, batch=4, lr=1e-3, data_seed=3, vol_dims=DIMS, rot_limit=ROT / 2, trans_limit=TRANS)
    with pytest.raises(pk.PfError):
        a.train(1, batch=5, lr=1e-3, data_seed=3, vol_dims=DIMS, rot_limit=ROT, trans_limit=TRANS)


def test_gave_up_wait_is_returned_as_timeout(torch_, pk):
    """A bounded device wait that ran out is reported by the next synchronous
    proposal call as PF_ETIMEOUT (and the flag is cleared): the self-test
    kernel waits on an mbarrier nothing arrives on, gives up and sets the flag
    -- nothing faults or hangs."""
    torch = torch_
    net = pk.Proposal(max_batch=2, seed=5)
    x, y = _batch(torch, pk, net, 2)
    out = torch.zeros((2, 12), dtype=torch.float32, device="cuda")
    net.forward(x, out)
    assert pk.nn_status(clear=True) == 0
    pk.nn_wait_selftest()
    with pytest.raises(pk.PfError) as err:
        net.backward(y)
    assert err.value.code == -4 and "PF_ETIMEOUT" in str(err.value)
    assert pk.nn_status(clear=False) == 0        # cleared by the call that reported it
    assert np.isfinite(net.backward(y))          # the next call succeeds
    net.close()


U32 = 2.0 ** -23   # fp32 unit roundoff, doubled: a tensor-core accumulator need not round to nearest


def _bf16_ok(got, ref, bound, what):
    """got = bf16 rounding of an fp32 value within `bound` of ref."""
    tol = 2.0 ** -8 * (np.abs(ref) + bound) + bound + 1e-30
    err = np.abs(np.asarray(got, np.float64) - ref)
    bad = err > tol
    assert not bad.any(), f"{what}: {bad.sum()} of {bad.size} outside the bound, worst {err.max():.3g}"


def _f32_ok(got, ref, bound, what):
    err = np.abs(np.asarray(got, np.float64) - ref)
    bad = err > bound + 1e-30
    assert not bad.any(), f"{what}: {bad.sum()} of {bad.size} outside the bound, worst {err.max():.3g}"


def test_backward_layer_by_layer_element_by_element(torch_, pk):
    """Every tensor of one forward and backward pass, element by element: each
    layer is recomputed in float64 from the GPU's own inputs to that layer
    (so a bf16 rounding that went the other way upstream does not spread),
    against the bound that fp32 arithmetic guarantees for it: a sum of K
    terms accumulated in fp32, in any order, is within (K - 1) u sum|terms| of
    the exact sum (one more u per product rounding and bias add; u = 2^-23,
    doubled for the tensor core), and a bf16 output within half an ulp
    (2^-8 relative) of that.  The loss gradient's bound adds the documented
    error of __expf (2 + 1.16 |x| ulp)."""
    torch = torch_
    B = 2
    net = pk.Proposal(max_batch=B, seed=9)
    x, y = _batch(torch, pk, net, B, seed=13)
    out_t = torch.zeros((B, 12), dtype=torch.float32, device="cuda")
    net.forward(x, out_t)
    net.backward(y)
    theta, grad = net.params(with_grad=True)
    P = onn.unpack(theta)
    off, _ = onn.layout()
    G = {k: np.asarray(grad[o:o + int(np.prod(sh))], np.float64).reshape(sh) for k, (o, sh) in off.items()}
    xin = _bf16_host(torch, x).astype(np.float64)
    yv = y.cpu().numpy().astype(np.float64)
    a = [onn.from_bf16_bits(net.tensor(l, B)).astype(np.float64) for l in range(4)]
    d = [onn.from_bf16_bits(net.tensor(4 + l, B)).astype(np.float64) for l in range(4)]
    h, out, dh, dout = (net.tensor(k, B).astype(np.float64) for k in (8, 9, 10, 11))
    ins = [xin] + a[:3]
    Wb = [onn.bf16_round(P[f"cw{l}"].astype(np.float32)).astype(np.float64) for l in range(4)]

    # forward: the four convolutions (bf16 x bf16 products are exact in fp32)
    for l in range(4):
        K = 64 * onn.CIN[l] + 1
        ref = onn.relu(onn.conv3d_pre(ins[l], Wb[l], P[f"cb{l}"]))
        bound = K * U32 * (onn.conv3d_abs_bound(ins[l], Wb[l]) + np.abs(P[f"cb{l}"]))
        _bf16_ok(a[l], ref, bound, f"conv {l} output")
    flat = a[3].reshape(B, -1)
    _f32_ok(h, onn.relu(flat @ P["f1w"].T + P["f1b"]),
            (2048 + 2) * U32 * (np.abs(flat) @ np.abs(P["f1w"]).T + np.abs(P["f1b"])), "hidden")
    _f32_ok(out, h @ P["f2w"].T + P["f2b"], (128 + 2) * U32 * (np.abs(h) @ np.abs(P["f2w"]).T + np.abs(P["f2b"])),
            "output")

    # the loss gradient from the GPU's output
    mu, s = out[:, :6], out[:, 6:]
    r = yv - mu
    e = np.exp(-s)
    de = (2.0 + 1.16 * np.abs(s) + 2.0) * U32          # __expf, plus its argument's rounding
    want = np.concatenate([-r * e / B, 0.5 * (1.0 - r * r * e) / B], 1)
    bound = np.concatenate([np.abs(r * e / B) * (de + 4 * U32),
                            0.5 * (r * r * e * (de + 4 * U32) + 4 * U32 * (1.0 + r * r * e)) / B], 1)
    _f32_ok(dout, want, bound, "loss gradient")

    # fully connected layers' gradients
    _f32_ok(G["f2w"], dout.T @ h, (B + 1) * U32 * (np.abs(dout).T @ np.abs(h)), "fc2 weight gradient")
    _f32_ok(G["f2b"], dout.sum(0), B * U32 * np.abs(dout).sum(0), "fc2 bias gradient")
    _f32_ok(dh, (dout @ P["f2w"]) * (h > 0), (12 + 1) * U32 * (np.abs(dout) @ np.abs(P["f2w"])), "hidden gradient")
    _f32_ok(G["f1w"], dh.T @ flat, (B + 1) * U32 * (np.abs(dh).T @ np.abs(flat)), "fc1 weight gradient")
    _f32_ok(G["f1b"], dh.sum(0), B * U32 * np.abs(dh).sum(0), "fc1 bias gradient")
    ref = ((dh @ P["f1w"]) * (flat > 0)).reshape(d[3].shape)
    bound = ((128 + 1) * U32 * (np.abs(dh) @ np.abs(P["f1w"]))).reshape(d[3].shape)
    _bf16_ok(d[3], ref, bound, "conv 3 pre-activation gradient")

    # the convolutions' gradients, top down
    for l in range(3, -1, -1):
        Kw = B * (32 >> l) ** 3
        _f32_ok(G[f"cw{l}"], onn.conv3d_backward_weights(ins[l], d[l]),
                (Kw + 1) * U32 * onn.conv3d_backward_weights(np.abs(ins[l]), np.abs(d[l])),
                f"conv {l} weight gradient")
        _f32_ok(G[f"cb{l}"], d[l].reshape(-1, 32).sum(0), Kw * U32 * np.abs(d[l]).reshape(-1, 32).sum(0),
                f"conv {l} bias gradient")
        if l > 0:
            D = 64 >> l
            ref = onn.conv3d_backward_data(d[l], Wb[l], D) * (ins[l] > 0)
            bound = (64 * 32 + 1) * U32 * onn.conv3d_backward_data(np.abs(d[l]), np.abs(Wb[l]), D)
            _bf16_ok(d[l - 1], ref, bound, f"conv {l - 1} pre-activation gradient")
    net.close()
