"""Tensor-core (tcgen05) contractions of the proposal network against the
float64 oracle (oracle/nn.py), through the C ABI.

Inputs are bf16-representable, so every product is exact in fp32; the only
errors are the fp32 accumulation (bounded by (K - 1) u sum|terms| for any
summation order, u = 2^-24 for round-to-nearest; 2^-23 is used, since the
tensor core's accumulator need not round to nearest) and, for bf16 outputs,
the final rounding (half an ulp, <= 2^-8 |value|).  The tolerances below are those bounds."""
import numpy as np
import pytest

from oracle import nn as onn

pytestmark = pytest.mark.gpu

U = 2.0 ** -23   # unit roundoff of fp32 accumulation, doubled: the tensor core need not round to nearest


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


def _bf16(rng, shape, scale=1.0, nonneg=False):
    a = rng.standard_normal(shape).astype(np.float32) * scale
    if nonneg:
        a = np.where(rng.random(shape) < 0.3, 0.0, np.abs(a)).astype(np.float32)
    return onn.bf16_round(a)


def _dev(torch, a):
    """float32 numpy (bf16-representable) -> CUDA bf16 tensor with the same values."""
    return torch.from_numpy(onn.bf16_bits(a).view(np.int16)).cuda().view(torch.bfloat16)


def _host(torch, t):
    return onn.from_bf16_bits(t.view(torch.int16).cpu().numpy().view(np.uint16))


def _check_bf16(got, ref, bound, what):
    # rounding the fp32 result v to bf16 (8 significant bits) moves it by at
    # most 2^-8 |v|, and |v - ref| <= bound
    tol = 2.0 ** -8 * (np.abs(ref) + bound) + bound + 1e-30
    err = np.abs(got.astype(np.float64) - ref)
    bad = err > tol
    assert not bad.any(), f"{what}: {bad.sum()} of {bad.size} outside the bound, worst {err.max():.3g}"


@pytest.mark.parametrize("M,K", [(300, 200), (128, 64), (1, 8), (513, 2048)])
def test_gemm_bf16(torch_, pk, M, K):
    torch = torch_
    rng = np.random.default_rng(M + K)
    A, B = _bf16(rng, (M, K)), _bf16(rng, (32, K))
    C = torch.full((M, 32), np.nan, dtype=torch.float32, device="cuda")
    pk.nn_gemm_bf16(_dev(torch, A), _dev(torch, B), C)
    torch.cuda.synchronize()
    assert pk.nn_status() == 0
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    bound = K * U * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T)
    err = np.abs(C.cpu().numpy() - ref)
    assert np.all(err <= bound + 1e-30), f"worst {err.max():.3g}"


@pytest.mark.parametrize("Bn,D,Cin", [(2, 10, 32), (2, 18, 2), (1, 2, 8), (4, 64, 2), (4, 32, 32), (1, 32, 32),
                                      (2, 64, 32), (1, 32, 2)])
def test_conv_forward(torch_, pk, Bn, D, Cin):
    torch = torch_
    rng = np.random.default_rng(10 * D + Cin)
    x = _bf16(rng, (Bn, D, D, D, Cin), nonneg=True)
    w = _bf16(rng, (32, 64, Cin), scale=0.2)
    b = rng.standard_normal(32).astype(np.float32) * 0.1
    y = torch.full((Bn, D // 2, D // 2, D // 2, 32), 7.0, dtype=torch.bfloat16, device="cuda")
    pk.nn_conv3d_forward(_dev(torch, x), _dev(torch, w), torch.from_numpy(b).cuda(), y)
    torch.cuda.synchronize()
    assert pk.nn_status() == 0
    ref = onn.relu(onn.conv3d_pre(x, w, b))
    bound = 64 * Cin * U * (onn.conv3d_abs_bound(x, w) + np.abs(b))
    _check_bf16(_host(torch, y), ref, bound, "conv forward")


@pytest.mark.parametrize("Bn,D,masked", [(2, 10, True), (1, 8, False), (3, 16, True), (2, 32, True), (1, 64, False)])
def test_conv_backward_data(torch_, pk, Bn, D, masked):
    torch = torch_
    rng = np.random.default_rng(100 + D)
    Do = D // 2
    dy = _bf16(rng, (Bn, Do, Do, Do, 32))
    w = _bf16(rng, (32, 64, 32), scale=0.2)
    act = _bf16(rng, (Bn, D, D, D, 32), nonneg=True) if masked else None
    w_t = np.ascontiguousarray(np.transpose(w, (2, 1, 0)))       # [ci][tap][co]
    dx = torch.full((Bn, D, D, D, 32), 7.0, dtype=torch.bfloat16, device="cuda")
    pk.nn_conv3d_backward_data(_dev(torch, dy), _dev(torch, w_t), None if act is None else _dev(torch, act), dx)
    torch.cuda.synchronize()
    assert pk.nn_status() == 0
    ref = onn.conv3d_backward_data(dy, w, D)
    bound = 2048 * U * onn.conv3d_backward_data(np.abs(dy), np.abs(w), D)
    if masked:
        ref = ref * (act > 0)
        bound = bound * (act > 0)
    _check_bf16(_host(torch, dx), ref, bound, "conv backward data")


@pytest.mark.parametrize("Bn,D,Cin", [(2, 10, 32), (2, 18, 2), (4, 32, 32), (2, 64, 32)])
def test_conv_backward_weights(torch_, pk, Bn, D, Cin):
    torch = torch_
    rng = np.random.default_rng(200 + D + Cin)
    Do = D // 2
    x = _bf16(rng, (Bn, D, D, D, Cin), nonneg=True)
    dy = _bf16(rng, (Bn, Do, Do, Do, 32), scale=0.5)
    init = rng.standard_normal((32, 64, Cin)).astype(np.float32)
    dw = torch.from_numpy(init.copy()).cuda()
    pk.nn_conv3d_backward_weights(_dev(torch, x), _dev(torch, dy), dw)
    torch.cuda.synchronize()
    assert pk.nn_status() == 0
    ref = init.astype(np.float64) + onn.conv3d_backward_weights(x, dy)
    P = Bn * Do ** 3
    bound = (P + 1) * U * (onn.conv3d_backward_weights(np.abs(x), np.abs(dy)) + np.abs(init))
    err = np.abs(dw.cpu().numpy() - ref)
    assert np.all(err <= bound + 1e-30), f"worst {err.max():.3g}"
