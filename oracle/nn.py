"""CPU oracle of the learned proposal network (numpy, float64).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers; the product path never
imports it.

The network (a 3-D CNN predicting the mean and log-variance of the 6-DOF pose
that seeds the particle cloud; the learned approach Sec. 6 names as future
work) is written here from its definitions, one plain step at a time:

* strided convolution, kernel 4^3, stride 2, padding 1 (definition: output
  voxel o sums input voxel 2o + k - 1 times tap k, zero outside), gathered
  tap by tap;
* its data gradient as the scatter (adjoint) of that gather, and its weight
  gradient as the correlation of the input with the output gradient;
* ReLU, fully connected layers, the Gaussian negative log-likelihood with a
  diagonal covariance, Adam (Kingma & Ba 2015, Algorithm 1).

Layouts follow the C ABI: activations (B, D, D, D, C) channel-last; conv
weights (32, 64, Cin) with tap = (kz * 4 + ky) * 4 + kx.

Parity status (pins in tests/test_oracle_nn.py): the convolution against a
pure-Python loop on tiny inputs and against scipy.signal.correlate; both
gradients by the adjoint identities <conv(x), g> = <x, conv^T(g)> =
<w, dW(x, g)> (exact for linear maps); the loss gradient by central finite
differences; Adam against its closed form on a constant gradient.
"""
from __future__ import annotations

import numpy as np

TAPS = [(kz, ky, kx) for kz in range(4) for ky in range(4) for kx in range(4)]


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest, ties to even); returned as float32."""
    a = np.ascontiguousarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)


def bf16_bits(a):
    """bfloat16 bit patterns (uint16) of float values already representable in bf16."""
    a = np.ascontiguousarray(a, np.float32)
    return (a.view(np.uint32) >> np.uint32(16)).astype(np.uint16)


def from_bf16_bits(b):
    return (np.asarray(b, np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32)


def conv3d_pre(x, w, bias=None):
    """Pre-activation of a strided conv: x (B,D,D,D,Cin) -> (B,D/2,D/2,D/2,32), float64."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    B, D, _, _, Cin = x.shape
    Do = D // 2
    xp = np.zeros((B, D + 2, D + 2, D + 2, Cin))
    xp[:, 1:-1, 1:-1, 1:-1, :] = x            # padding 1: padded index = input index + 1
    out = np.zeros((B, Do, Do, Do, w.shape[0]))
    for t, (kz, ky, kx) in enumerate(TAPS):
        # output o reads input 2o + k - 1 = padded 2o + k
        patch = xp[:, kz:kz + 2 * Do:2, ky:ky + 2 * Do:2, kx:kx + 2 * Do:2, :]
        out += patch @ w[:, t, :].T
    if bias is not None:
        out += np.asarray(bias, np.float64)
    return out


def conv3d_abs_bound(x, w):
    """sum over the terms of |x| |w| per output (for rounding-error bounds)."""
    return conv3d_pre(np.abs(np.asarray(x, np.float64)), np.abs(np.asarray(w, np.float64)))


def conv3d_backward_data(dy, w, D):
    """Adjoint of conv3d_pre in x: scatter each tap's contribution back."""
    dy = np.asarray(dy, np.float64)
    w = np.asarray(w, np.float64)
    B, Do = dy.shape[0], dy.shape[1]
    Cin = w.shape[2]
    dxp = np.zeros((B, D + 2, D + 2, D + 2, Cin))
    for t, (kz, ky, kx) in enumerate(TAPS):
        dxp[:, kz:kz + 2 * Do:2, ky:ky + 2 * Do:2, kx:kx + 2 * Do:2, :] += dy @ w[:, t, :]
    return dxp[:, 1:-1, 1:-1, 1:-1, :]


def conv3d_backward_weights(x, dy):
    """dW[co, tap, ci] = sum_{b,o} x[b, 2o + k - 1, ci] dy[b, o, co]."""
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    B, D, _, _, Cin = x.shape
    Do = D // 2
    xp = np.zeros((B, D + 2, D + 2, D + 2, Cin))
    xp[:, 1:-1, 1:-1, 1:-1, :] = x
    g = dy.reshape(-1, dy.shape[-1])
    dw = np.zeros((dy.shape[-1], 64, Cin))
    for t, (kz, ky, kx) in enumerate(TAPS):
        patch = xp[:, kz:kz + 2 * Do:2, ky:ky + 2 * Do:2, kx:kx + 2 * Do:2, :].reshape(-1, Cin)
        dw[:, t, :] = g.T @ patch
    return dw


def conv3d_loop(x, w, bias):
    """Pure-Python loop of the definition (tiny inputs only)."""
    B, D, _, _, Cin = x.shape
    Do = D // 2
    out = np.zeros((B, Do, Do, Do, w.shape[0]))
    for b in range(B):
        for oz in range(Do):
            for oy in range(Do):
                for ox in range(Do):
                    for co in range(w.shape[0]):
                        acc = float(bias[co])
                        for t, (kz, ky, kx) in enumerate(TAPS):
                            iz, iy, ix = 2 * oz + kz - 1, 2 * oy + ky - 1, 2 * ox + kx - 1
                            if 0 <= iz < D and 0 <= iy < D and 0 <= ix < D:
                                for ci in range(Cin):
                                    acc += float(x[b, iz, iy, ix, ci]) * float(w[co, t, ci])
                        out[b, oz, oy, ox, co] = acc
    return out


def relu(a):
    return np.maximum(a, 0.0)


def gaussian_nll(out, y):
    """Mean over the batch of sum_d 0.5 ((y - mu)^2 exp(-s) + s), out = [mu | s]."""
    out = np.asarray(out, np.float64)
    y = np.asarray(y, np.float64)
    mu, s = out[:, :6], out[:, 6:12]
    r2 = (y - mu) ** 2
    loss = 0.5 * np.sum(r2 * np.exp(-s) + s) / out.shape[0]
    g = np.zeros_like(out)
    g[:, :6] = -(y - mu) * np.exp(-s) / out.shape[0]
    g[:, 6:12] = 0.5 * (1.0 - r2 * np.exp(-s)) / out.shape[0]
    return loss, g


def adam(theta, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t = 1, 2, ...); returns the new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------------ the whole network

G, HIDDEN, NOUT, FLAT = 64, 128, 12, 4 * 4 * 4 * 32
CIN = (2, 32, 32, 32)


def layout():
    """Offsets of the flat parameter vector: conv l weight (32, 64, Cin_l) and
    bias (32), fc1 (128, 2048) + (128), fc2 (12, 128) + (12)."""
    off, o = {}, 0
    for l, c in enumerate(CIN):
        off[f"cw{l}"] = (o, (32, 64, c))
        o += 32 * 64 * c
        off[f"cb{l}"] = (o, (32,))
        o += 32
    off["f1w"] = (o, (HIDDEN, FLAT))
    o += HIDDEN * FLAT
    off["f1b"] = (o, (HIDDEN,))
    o += HIDDEN
    off["f2w"] = (o, (NOUT, HIDDEN))
    o += NOUT * HIDDEN
    off["f2b"] = (o, (NOUT,))
    o += NOUT
    return off, o


def unpack(theta):
    off, total = layout()
    assert theta.size == total
    return {k: np.asarray(theta[o:o + int(np.prod(sh))], np.float64).reshape(sh) for k, (o, sh) in off.items()}


def _bf16(a):
    """float64 values rounded to bf16 (through float32, as the device does)."""
    return bf16_round(np.asarray(a, np.float64).astype(np.float32)).astype(np.float64)


def net_forward(theta, x, rnd=_bf16):
    """Forward pass with the bf16 roundings of the device path: conv weights
    and every conv output (after ReLU) rounded to bf16; the fully connected
    layers in float64.  x: (B, 64, 64, 64, 2) bf16 values.  Returns
    (out (B, 12), h (B, 128), acts [a0..a3]).  rnd: the rounding applied
    (identity for the exact-arithmetic network)."""
    P = unpack(theta)
    a, acts = np.asarray(x, np.float64), []
    for l in range(4):
        a = rnd(relu(conv3d_pre(a, rnd(P[f"cw{l}"]), P[f"cb{l}"])))
        acts.append(a)
    flat = a.reshape(a.shape[0], -1)
    h = relu(flat @ P["f1w"].T + P["f1b"])
    out = h @ P["f2w"].T + P["f2b"]
    return out, h, acts


def net_backward(theta, x, y, rnd=_bf16):
    """Loss and gradient (flat, like theta) of the mean Gaussian NLL, with the
    device path's roundings: the gradients wrt the conv pre-activations are
    stored as bf16 before they feed the next layer down."""
    P = unpack(theta)
    out, h, acts = net_forward(theta, x, rnd)
    loss, dout = gaussian_nll(out, y)
    off, total = layout()
    g = np.zeros(total)

    def put(k, v):
        o, sh = off[k]
        g[o:o + int(np.prod(sh))] = np.asarray(v).reshape(-1)

    put("f2w", dout.T @ h)
    put("f2b", dout.sum(0))
    dh = (dout @ P["f2w"]) * (h > 0)
    flat = acts[3].reshape(acts[3].shape[0], -1)
    put("f1w", dh.T @ flat)
    put("f1b", dh.sum(0))
    d = rnd((dh @ P["f1w"]) * (flat > 0)).reshape(acts[3].shape)
    for l in range(3, -1, -1):
        below = np.asarray(x, np.float64) if l == 0 else acts[l - 1]
        put(f"cw{l}", conv3d_backward_weights(below, d))
        put(f"cb{l}", d.reshape(-1, 32).sum(0))
        if l > 0:
            d = rnd(conv3d_backward_data(d, rnd(P[f"cw{l}"]), below.shape[1]) * (below > 0))
    return loss, g


def box_average(vol, origin, spacing, box_o, h, G=64):
    """Network input channel: mean of the voxels of vol (Z, Y, X) whose world
    position origin + spacing * p falls in each cell [box_o + h g, box_o + h (g + 1))
    of a G^3 grid, divided by 64; 0 for cells without a voxel."""
    dims = (vol.shape[2], vol.shape[1], vol.shape[0])
    rng = []
    for d in range(3):
        lo = np.ceil((box_o[d] + h[d] * np.arange(G) - origin[d]) / spacing[d]).astype(np.int64)
        hi = np.ceil((box_o[d] + h[d] * (np.arange(G) + 1) - origin[d]) / spacing[d]).astype(np.int64)
        rng.append((np.clip(lo, 0, dims[d]), np.clip(hi, 0, dims[d])))
    S = np.zeros((vol.shape[0] + 1, vol.shape[1] + 1, vol.shape[2] + 1))
    S[1:, 1:, 1:] = np.cumsum(np.cumsum(np.cumsum(vol.astype(np.float64), 0), 1), 2)
    (xl, xh), (yl, yh), (zl, zh) = rng
    Z0, Y0, X0 = np.meshgrid(zl, yl, xl, indexing="ij")
    Z1, Y1, X1 = np.meshgrid(zh, yh, xh, indexing="ij")
    tot = (S[Z1, Y1, X1] - S[Z0, Y1, X1] - S[Z1, Y0, X1] - S[Z1, Y1, X0]
           + S[Z0, Y0, X1] + S[Z0, Y1, X0] + S[Z1, Y0, X0] - S[Z0, Y0, X0])
    cnt = np.maximum(Z1 - Z0, 0) * np.maximum(Y1 - Y0, 0) * np.maximum(X1 - X0, 0)
    return np.where(cnt > 0, tot / np.maximum(cnt, 1) / 64.0, 0.0)
