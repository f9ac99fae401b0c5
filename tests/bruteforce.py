"""Independent numpy/scipy definitions used to pin the oracle.

Nothing here calls the oracle or the CUDA path.  Geometry is float64 through
scipy's Rotation; trilinear sampling is scipy.ndimage.map_coordinates(order=1);
integer maps (axis permutations with signs plus integer shifts) are applied
with exact integer indexing.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy import ndimage

import pfsynth


def target_points(tgt_dims):
    X, Y, Z = tgt_dims
    z, y, x = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    return np.stack([x, y, z], -1).reshape(-1, 3)


def source_index_f64(pose, src_dims, src_origin, tgt_dims, tgt_origin, src_spacing=(1.0, 1.0, 1.0),
                     tgt_spacing=(1.0, 1.0, 1.0)):
    """Continuous source index of every target voxel (float64, scipy rotation)."""
    w = pfsynth.map_target_to_source(pose, src_dims, src_origin, tgt_origin, target_points(tgt_dims),
                                     src_spacing, tgt_spacing)
    return (w - np.asarray(src_origin, np.float64)) / np.asarray(src_spacing, np.float64)


def nn_counts_f64(src, tgt, q):
    sd = np.array([src.shape[2], src.shape[1], src.shape[0]])
    i = np.floor(q + 0.5).astype(np.int64)
    ok = np.all((i >= 0) & (i < sd), axis=1)
    s = np.zeros(len(q), np.int64)
    ii = i[ok]
    s[ok] = src[ii[:, 2], ii[:, 1], ii[:, 0]] != 0
    t = (tgt.reshape(-1) != 0).astype(np.int64)
    return np.array([ok.sum(), s.sum(), (t * ok).sum(), (s & t).sum()], np.int64)


def trilinear_f64(src, q):
    """(inside mask, samples) with scipy's order-1 spline = trilinear."""
    sd = np.array([src.shape[2], src.shape[1], src.shape[0]], np.float64)
    ok = np.all((q >= 0) & (q <= sd - 1), axis=1)
    coords = np.stack([q[ok, 2], q[ok, 1], q[ok, 0]])   # (z, y, x) order
    s = ndimage.map_coordinates(src.astype(np.float64), coords, order=1, mode="nearest")
    return ok, s


def signed_permutations():
    """All 48 proper and improper axis maps as integer 3x3 matrices."""
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            P = np.zeros((3, 3), np.int64)
            for r, c in enumerate(perm):
                P[r, c] = signs[r]
            out.append(P)
    return out


def integer_map_counts(src, tgt, P, b, image=False):
    """Exact counts/moments for q = P p + b with integer P, b (a = 0)."""
    sd = np.array([src.shape[2], src.shape[1], src.shape[0]])
    tgt_dims = (tgt.shape[2], tgt.shape[1], tgt.shape[0])
    p = target_points(tgt_dims)
    q = p @ P.T + b
    ok = np.all((q >= 0) & (q < sd), axis=1)
    t = tgt.reshape(-1).astype(np.int64)
    s = np.zeros(len(p), np.int64)
    qq = q[ok]
    s[ok] = src[qq[:, 2], qq[:, 1], qq[:, 0]]
    if not image:
        sb, tb = (s != 0).astype(np.int64), (t != 0).astype(np.int64)
        return np.array([ok.sum(), sb.sum(), (tb * ok).sum(), (sb & tb).sum()], np.int64)
    sq = [32768 * int(v) for v in s]          # exact Python ints (S2 needs > 64 bits)
    tt = [int(v) for v in t]
    S2 = sum(v * v for v in sq)
    okl = [int(v) for v in ok]
    return np.array([sum(okl), sum(sq), S2 & (2**64 - 1), S2 >> 64, sum(a * b for a, b in zip(sq, tt)),
                     sum(a * b for a, b in zip(tt, okl)), sum(a * a * b for a, b in zip(tt, okl))],
                    dtype=np.uint64)


def dyadic_map_moments(src, tgt, P, b, h4):
    """Exact image moments for q = P p + b + h4/4 (integer P, b, h4; a = 0).

    Every fraction is a multiple of 1/4, so each trilinear weight, corner
    product and sample is a dyadic rational with at most 6 fractional bits:
    the samples, their 15-bit fixed point values and all sums are exact
    (Python integers in units of 2^-6 for the samples)."""
    sd = np.array([src.shape[2], src.shape[1], src.shape[0]], np.int64)
    tgt_dims = (tgt.shape[2], tgt.shape[1], tgt.shape[0])
    p = target_points(tgt_dims).astype(np.int64)
    q4 = 4 * (p @ P.T + b) + h4                       # 4 q, exact integers
    ok = np.all((q4 >= 0) & (q4 <= 4 * (sd - 1)), axis=1)
    i0 = np.minimum(q4 // 4, sd - 2)                  # min(floor q, D - 2)
    f4 = q4 - 4 * i0                                  # 4 f, in 0..4
    t = tgt.reshape(-1).astype(np.int64)
    srci = src.astype(np.int64)
    n = S1 = S2 = ST = T1 = T2 = 0
    for k in np.nonzero(ok)[0]:
        x0, y0, z0 = (int(v) for v in i0[k])
        fx, fy, fz = (int(v) for v in f4[k])
        acc = 0                                       # 64 s (weights in quarters per axis)
        for dz, wz in ((0, 4 - fz), (1, fz)):
            for dy, wy in ((0, 4 - fy), (1, fy)):
                for dx, wx in ((0, 4 - fx), (1, fx)):
                    if wx and wy and wz:
                        acc += wx * wy * wz * int(srci[z0 + dz, y0 + dy, x0 + dx])
        sq = acc * 512                                # 2^15 s = 2^15 acc / 64
        tk = int(t[k])
        n += 1
        S1 += sq
        S2 += sq * sq
        ST += sq * tk
        T1 += tk
        T2 += tk * tk
    return np.array([n, S1, S2 & (2**64 - 1), S2 >> 64, ST, T1, T2], dtype=np.uint64)


def dyadic_map_warp(src, tgt_dims, P, b, h4, interp):
    """Exact warp for q = P p + b + h4/4 (integer P, b, h4): trilinear samples
    are exact multiples of 1/64, rounded half to even into uint8; nearest
    neighbour takes voxel floor(q + 1/2); 0 outside the source."""
    sd = np.array([src.shape[2], src.shape[1], src.shape[0]], np.int64)
    p = target_points(tgt_dims).astype(np.int64)
    q4 = 4 * (p @ P.T + b) + h4
    out = np.zeros(len(p), np.uint8)
    srci = src.astype(np.int64)
    if interp == 0:
        i = (q4 + 2) // 4                             # floor(q + 1/2)
        ok = np.all((i >= 0) & (i < sd), axis=1)
        ii = i[ok]
        out[ok] = src[ii[:, 2], ii[:, 1], ii[:, 0]]
    else:
        ok = np.all((q4 >= 0) & (q4 <= 4 * (sd - 1)), axis=1)
        i0 = np.minimum(q4 // 4, sd - 2)
        f4 = q4 - 4 * i0
        for k in np.nonzero(ok)[0]:
            x0, y0, z0 = (int(v) for v in i0[k])
            fx, fy, fz = (int(v) for v in f4[k])
            acc = 0                                   # 64 s
            for dz, wz in ((0, 4 - fz), (1, fz)):
                for dy, wy in ((0, 4 - fy), (1, fy)):
                    for dx, wx in ((0, 4 - fx), (1, fx)):
                        if wx and wy and wz:
                            acc += wx * wy * wz * int(srci[z0 + dz, y0 + dy, x0 + dx])
            v, r = divmod(acc, 64)
            v += 1 if (r > 32 or (r == 32 and v % 2 == 1)) else 0
            out[k] = min(v, 255)
    X, Y, Z = tgt_dims
    return out.reshape(Z, Y, X)


def integer_map_warp(src, tgt_dims, P, b):
    sd = np.array([src.shape[2], src.shape[1], src.shape[0]])
    p = target_points(tgt_dims)
    q = p @ P.T + b
    ok = np.all((q >= 0) & (q < sd), axis=1)
    out = np.zeros(len(p), np.uint8)
    qq = q[ok]
    out[ok] = src[qq[:, 2], qq[:, 1], qq[:, 0]]
    X, Y, Z = tgt_dims
    return out.reshape(Z, Y, X)


def exact_matrix(P, b):
    M = np.zeros(12, np.float32)
    for i in range(3):
        M[4 * i:4 * i + 3] = P[i]
        M[4 * i + 3] = b[i]
    return M


def systematic_bruteforce(W, u):
    """a_j = min{i : C_i > T_j}, T_j = floor((j 2^32 + u) S / (N 2^32)), Python ints."""
    W = [int(w) for w in W]
    N = len(W)
    C, run = [], 0
    for w in W:
        run += w
        C.append(run)
    S = run
    if S == 0:
        return np.arange(N, dtype=np.int32)
    out = []
    for j in range(N):
        T = ((j << 32) + int(u)) * S // (N << 32)
        out.append(next(i for i in range(N) if C[i] > T))
    return np.array(out, np.int32)
