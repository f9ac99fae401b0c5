"""CPU oracle for the particle-filter rigid registration hot path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path
(``paper_2504_19930_gb300``) never imports this package.

The arithmetic lives in ``pf_oracle.c`` (single-threaded C, built with
``-O2 -ffp-contract=off``); this module compiles it with gcc on first use and
wraps each function with numpy marshalling.  Volumes are numpy uint8 arrays
of shape (Z, Y, X); dims triples are (X, Y, Z).

Parity status of each function (what pins it, see ``tests/test_oracle_pins.py``):
  philox            Random123 known-answer vectors (published)
  sin / cos         libm within a few ulp; sin^2 + cos^2 = 1
  rotation          scipy Rotation.from_euler('ZXY'); orthonormality; inverse
  measure_mask      numpy brute force; identity; grid-aligned 90-degree maps
  measure_image     linear-ramp closed form; numpy trilinear brute force;
                    the fp64 two-pass NCC within the rounding bound
  ncc2_f64          scipy.stats.pearsonr squared on the same samples
  weights/resample  closed forms (uniform, one-hot, copy counts) and an
                    O(N^2) brute-force definition; offsets uniform over
                    iterations
  init / perturb    bounds, mean and variance, independence across DOFs,
                    particles and iterations; the scheduled step size
  register          recovers the generating pose of a synthetic pair;
                    reaches the exhaustive grid optimum on tiny masks
  warp              identity returns the input; 90-degree maps equal numpy
                    rot90/transpose
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libpforacle.so")
_lock = threading.Lock()
_lib = None

MODES = {"mask_dice": 0, "mask_ncc": 1, "image_ncc": 2, "combined": 3}


def build(force: bool = False) -> str:
    """Compile pf_oracle.c into oracle/_build/libpforacle.so (gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # PF_ORACLE_LIB names another build of pf_oracle.c: the mutation
            # tests load copies with a planted mistake to show that the pins
            # catch it.
            _lib = C.CDLL(os.environ.get("PF_ORACLE_LIB") or build())
            _declare(_lib)
    return _lib


_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_vp = C.c_void_p


def _declare(L):
    L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    L.orc_sin.argtypes = [C.c_double]
    L.orc_sin.restype = C.c_double
    L.orc_cos.argtypes = [C.c_double]
    L.orc_cos.restype = C.c_double
    L.orc_rotation.argtypes = [_f32p, _f64p]
    L.orc_pose_matrix.argtypes = [_f32p, _i32p, _f32p, _f32p, _f32p, _f32p]
    L.orc_pose_matrix_sp.argtypes = [_f32p, _i32p, _f32p, _vp, _f32p, _vp, _f32p, _f32p]
    for name in ("orc_measure_mask", "orc_measure_image"):
        getattr(L, name).argtypes = [_u8p, _i32p, _u8p, _i32p, _f32p, _f32p, C.c_int32, _u64p]
    L.orc_ncc2_f64.argtypes = [_u8p, _i32p, _u8p, _i32p, _f32p, _f32p, C.c_int32, _f64p]
    L.orc_ncc2_from_moments.argtypes = [C.c_uint64] * 8
    L.orc_ncc2_from_moments.restype = C.c_double
    L.orc_dice_from_counts.argtypes = [C.c_uint64] * 5
    L.orc_dice_from_counts.restype = C.c_double
    L.orc_score.argtypes = [C.c_int32, _u64p, C.c_uint64, C.c_uint64]
    L.orc_score.restype = C.c_double
    L.orc_weights.argtypes = [_f64p, C.c_int32, C.c_int32, _u64p]
    L.orc_resample.argtypes = [_u64p, C.c_int32, C.c_uint32, _i32p]
    L.orc_estimate.argtypes = [_f32p, C.c_int32, _u64p, _f64p]
    L.orc_init.argtypes = [_f32p, C.c_int32, C.c_uint64, _f32p]
    L.orc_sigma.argtypes = [C.c_float, C.c_float, C.c_int32, _f32p, _f32p]
    L.orc_perturb.argtypes = [_f32p, C.c_int32, C.c_uint64, C.c_int32, _f32p, _f32p]
    L.orc_resample_offset.argtypes = [C.c_uint64, C.c_int32]
    L.orc_resample_offset.restype = C.c_uint32
    L.orc_register.argtypes = [
        C.c_int32, _vp, _vp, _vp, _vp, _i32p, _f32p, _vp, _i32p, _f32p, _vp, C.c_int32, C.c_int32,
        _f32p, _f32p, C.c_float, C.c_float, C.c_int32, C.c_uint64, C.c_float,
        _f32p, C.c_int32, C.c_int32, _f64p, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.orc_register.restype = C.c_int32
    L.orc_init_gaussian.argtypes = [_f32p, C.c_int32, C.c_uint64, _f32p, _f32p, _f32p]
    L.orc_warp.argtypes = [_u8p, _i32p, _u8p, _i32p, _f32p, _f32p, C.c_int32]
    L.orc_trilinear.argtypes = [_u8p, _i32p, _f32p, _f32p]
    L.orc_trilinear.restype = C.c_int32


def _dims(vol):
    return np.array([vol.shape[2], vol.shape[1], vol.shape[0]], np.int32)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------- primitives

def philox(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_c(ctr, np.uint32), _c(key, np.uint32), out)
    return out


def trilinear(src, q):
    """fp32 trilinear sample of src (Z, Y, X) at q = (qx, qy, qz); None outside."""
    out = np.zeros(1, np.float32)
    ok = lib().orc_trilinear(_c(src, np.uint8), _dims(src), _c(q, np.float32), out)
    return float(out[0]) if ok else None


def sin(x):
    return lib().orc_sin(float(x))


def cos(x):
    return lib().orc_cos(float(x))


def rotation(pose):
    R = np.zeros(9, np.float64)
    lib().orc_rotation(_c(pose, np.float32), R)
    return R.reshape(3, 3)


def _sp(spacing):
    """Spacing argument: None (unit) or float32[3]."""
    return None if spacing is None else _c(np.broadcast_to(np.asarray(spacing, np.float32), (3,)), np.float32)


def pose_matrix(pose, src_dims, src_origin, tgt_origin, src_spacing=None, tgt_spacing=None):
    """(M float32[12], a float32[3]) with q = M3 (p - a) + b (voxel units)."""
    M = np.zeros(12, np.float32)
    a = np.zeros(3, np.float32)
    ss, ts = _sp(src_spacing), _sp(tgt_spacing)
    if ss is None and ts is None:
        lib().orc_pose_matrix(_c(pose, np.float32), _c(src_dims, np.int32), _c(src_origin, np.float32),
                              _c(tgt_origin, np.float32), M, a)
    else:
        ptr = lambda v: None if v is None else v.ctypes.data_as(C.c_void_p)  # noqa: E731
        lib().orc_pose_matrix_sp(_c(pose, np.float32), _c(src_dims, np.int32), _c(src_origin, np.float32),
                                 ptr(ss), _c(tgt_origin, np.float32), ptr(ts), M, a)
    return M, a


def pose_matrices(poses6xN, src_dims, src_origin, tgt_origin, src_spacing=None, tgt_spacing=None):
    poses6xN = np.asarray(poses6xN, np.float32)
    N = poses6xN.shape[1]
    mats = np.zeros((N, 12), np.float32)
    a = None
    for i in range(N):
        mats[i], a = pose_matrix(poses6xN[:, i], src_dims, src_origin, tgt_origin, src_spacing, tgt_spacing)
    return mats, a


def measure_mask(src, tgt, mats, a):
    """counts [M,4] = (n, A, B, C) for each 3x4 matrix."""
    src, tgt = _c(src, np.uint8), _c(tgt, np.uint8)
    mats = _c(np.atleast_2d(mats), np.float32)
    out = np.zeros((mats.shape[0], 4), np.uint64)
    lib().orc_measure_mask(src, _dims(src), tgt, _dims(tgt), mats, _c(a, np.float32),
                           mats.shape[0], out)
    return out


def measure_image(src, tgt, mats, a):
    """moments [M,7] = (n, S1, S2 low, S2 high, ST, T1, T2) for each 3x4 matrix
    (samples rounded to 15 fractional bits; S2 is a 128-bit sum)."""
    src, tgt = _c(src, np.uint8), _c(tgt, np.uint8)
    mats = _c(np.atleast_2d(mats), np.float32)
    out = np.zeros((mats.shape[0], 7), np.uint64)
    lib().orc_measure_image(src, _dims(src), tgt, _dims(tgt), mats, _c(a, np.float32),
                            mats.shape[0], out)
    return out


def ncc2_f64(src, tgt, mats, a):
    src, tgt = _c(src, np.uint8), _c(tgt, np.uint8)
    mats = _c(np.atleast_2d(mats), np.float32)
    out = np.zeros(mats.shape[0], np.float64)
    lib().orc_ncc2_f64(src, _dims(src), tgt, _dims(tgt), mats, _c(a, np.float32),
                       mats.shape[0], out)
    return out


def ncc2_from_moments(m, n_min=0):
    """NCC^2 from the 7 image moments (n, S1, S2 lo, S2 hi, ST, T1, T2)."""
    m = [int(v) for v in m]
    return lib().orc_ncc2_from_moments(*m, int(n_min))


def dice_from_counts(n, A, C_, b_full, n_min=0):
    return lib().orc_dice_from_counts(int(n), int(A), int(C_), int(b_full), int(n_min))


MOM_STRIDE = 12   # [n S1 S2lo S2hi ST T1 T2 0 | n_nn A B C]


def score(mode, mom12, b_full=0, n_min=0):
    mode = MODES.get(mode, mode)
    return lib().orc_score(int(mode), _c(mom12, np.uint64), int(b_full), int(n_min))


def weights(scores, gamma_log2):
    s = _c(scores, np.float64)
    W = np.zeros(s.shape[0], np.uint64)
    lib().orc_weights(s, s.shape[0], int(gamma_log2), W)
    return W


def resample(W, u):
    W = _c(W, np.uint64)
    idx = np.zeros(W.shape[0], np.int32)
    lib().orc_resample(W, W.shape[0], int(u) & 0xFFFFFFFF, idx)
    return idx


def estimate(poses6xN, W):
    p = _c(poses6xN, np.float32)
    est = np.zeros(6, np.float64)
    lib().orc_estimate(p, p.shape[1], _c(W, np.uint64), est)
    return est


def _qmul(a, b):
    """Hamilton product of quaternions (w, x, y, z)."""
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw])


def quaternion(pose):
    """Unit quaternion (w, x, y, z) of R = Rz(rz) Rx(rx) Ry(ry): qz * qx * qy,
    each an axis rotation by its half angle (the oracle's fp64 sin/cos)."""
    rx, ry, rz = (float(v) for v in pose[:3])
    qx = np.array([cos(rx / 2), sin(rx / 2), 0.0, 0.0])
    qy = np.array([cos(ry / 2), 0.0, sin(ry / 2), 0.0])
    qz = np.array([cos(rz / 2), 0.0, 0.0, sin(rz / 2)])
    return _qmul(qz, _qmul(qx, qy))


def quaternion_matrix(q):
    """Rotation matrix of a unit quaternion (w, x, y, z)."""
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def estimate_quaternion(poses6xN, W):
    """Estimate (Fig. 1 "estimation") with the rotation averaged as
    quaternions: translations are the W-weighted mean (uniform when all W are
    0); the rotation is the unit eigenvector of the largest eigenvalue of
    sum_i W_i q_i q_i^T, turned back into (rx, ry, rz) of R = Rz Rx Ry
    (R21 = sin rx, R20 = -cos rx sin ry, R22 = cos rx cos ry,
    R01 = -sin rz cos rx, R11 = cos rz cos rx)."""
    poses6xN = np.asarray(poses6xN, np.float32)
    est = estimate(poses6xN, W)
    w = np.asarray(W, np.uint64).astype(np.float64)
    if w.sum() == 0:
        w = np.ones_like(w)
    Q = np.stack([quaternion(poses6xN[:, i]) for i in range(poses6xN.shape[1])])
    A = (Q * w[:, None]).T @ Q / w.sum()
    vals, vecs = np.linalg.eigh(A)
    R = quaternion_matrix(vecs[:, -1] / np.linalg.norm(vecs[:, -1]))
    est[0] = np.arcsin(np.clip(R[2, 1], -1.0, 1.0))
    est[1] = np.arctan2(-R[2, 0], R[2, 2])
    est[2] = np.arctan2(-R[0, 1], R[1, 1])
    return est


def init_particles(N, seed, lim6):
    x = np.zeros((6, N), np.float32)
    lib().orc_init(x, N, int(seed), _c(lim6, np.float32))
    return x


def init_gaussian(N, seed, mean6, std6, lim6):
    """Initial cloud around a proposal: clamp(mean + std * eps) per DOF."""
    x = np.zeros((6, N), np.float32)
    lib().orc_init_gaussian(x, N, int(seed), _c(mean6, np.float32), _c(std6, np.float32), _c(lim6, np.float32))
    return x


def sigma(sigma0_frac, decay, k, lim6):
    out = np.zeros(6, np.float32)
    lib().orc_sigma(float(sigma0_frac), float(decay), int(k), _c(lim6, np.float32), out)
    return out


def perturb(poses6xN, seed, k, sig6, lim6):
    x = np.array(poses6xN, np.float32, copy=True, order="C")
    lib().orc_perturb(x, x.shape[1], int(seed), int(k), _c(sig6, np.float32), _c(lim6, np.float32))
    return x


def resample_offset(seed, k):
    return lib().orc_resample_offset(int(seed), int(k))


def warp(src, src_origin, tgt_dims, tgt_origin, pose, interp=1, src_spacing=None, tgt_spacing=None):
    """Warp one source-grid volume into the target grid with the pose."""
    src = _c(src, np.uint8)
    M, a = pose_matrix(pose, _dims(src), src_origin, tgt_origin, src_spacing, tgt_spacing)
    X, Y, Z = tgt_dims
    out = np.zeros((Z, Y, X), np.uint8)
    lib().orc_warp(src, _dims(src), out, _c(tgt_dims, np.int32), M, a, int(interp))
    return out


def warp_matrix(src, tgt_dims, M, a, interp=1):
    src = _c(src, np.uint8)
    X, Y, Z = tgt_dims
    out = np.zeros((Z, Y, X), np.uint8)
    lib().orc_warp(src, _dims(src), out, _c(tgt_dims, np.int32), _c(M, np.float32),
                   _c(a, np.float32), int(interp))
    return out


# ------------------------------------------------------------------ the filter

DEFAULTS = dict(sigma0_frac=0.25, sigma_decay=0.8, gamma_log2=5, min_overlap_frac=0.01)


def register(mode, src_dims, src_origin, tgt_dims, tgt_origin, n_particles, n_iters,
             rot_limit, trans_limit, seed=0, src=None, tgt=None, src_mask=None, tgt_mask=None,
             sigma0_frac=0.25, sigma_decay=0.8, gamma_log2=5, min_overlap_frac=0.01,
             poses=None, k0=0, trace=True, src_spacing=None, tgt_spacing=None, sig_base=None):
    """Run the whole filter for ``n_iters`` iterations starting at iteration
    ``k0`` (from ``poses`` [6,N] if given, else the Philox initial cloud).
    ``sig_base`` (6 floats) replaces sigma0_frac * limit as the noise base.

    Returns a dict: est (fp64[6] of the last iteration), poses (the resampled
    cloud after the last iteration) and, with ``trace``, per-iteration arrays
    poses [K,6,N], mom [K,N,12], score [K,N], W [K,N], idx [K,N], est [K,6].
    """
    mode = MODES.get(mode, mode)
    N, K = int(n_particles), int(n_iters)
    rl = np.broadcast_to(np.asarray(rot_limit, np.float32), (3,)).copy()
    tl = np.broadcast_to(np.asarray(trans_limit, np.float32), (3,)).copy()
    have = poses is not None
    x = np.array(poses, np.float32, order="C") if have else np.zeros((6, N), np.float32)
    est = np.zeros(6, np.float64)
    keep = []

    def ptr(a):
        keep.append(a)
        return a.ctypes.data_as(C.c_void_p) if a is not None else None

    need = {MODES["image_ncc"]: (1, 1, 0, 0), MODES["mask_dice"]: (0, 0, 1, 1),
            MODES["mask_ncc"]: (0, 0, 1, 1), MODES["combined"]: (1, 1, 1, 1)}[mode]
    for v, n, name, dims in zip((src, tgt, src_mask, tgt_mask), need, ("src", "tgt", "src_mask", "tgt_mask"),
                                (src_dims, tgt_dims, src_dims, tgt_dims)):
        if n and v is None:
            raise ValueError(f"register: mode needs {name}")
        if v is not None and np.size(v) != int(np.prod(np.asarray(dims, np.int64))):
            raise ValueError(f"register: {name} has {np.size(v)} voxels, dims are {tuple(dims)}")
    vols = [None if v is None else _c(v, np.uint8) for v in (src, tgt, src_mask, tgt_mask)]
    if trace:
        tr = dict(poses=np.zeros((K, 6, N), np.float32), mom=np.zeros((K, N, 12), np.uint64),
                  score=np.zeros((K, N), np.float64), W=np.zeros((K, N), np.uint64),
                  idx=np.zeros((K, N), np.int32), est=np.zeros((K, 6), np.float64))
        trp = [ptr(tr[k]) for k in ("poses", "mom", "score", "W", "idx", "est")]
    else:
        tr, trp = {}, [None] * 6
    rc = lib().orc_register(
        mode, *[ptr(v) for v in vols], _c(src_dims, np.int32), _c(src_origin, np.float32),
        ptr(_sp(src_spacing)), _c(tgt_dims, np.int32), _c(tgt_origin, np.float32), ptr(_sp(tgt_spacing)),
        N, K, rl, tl,
        float(sigma0_frac), float(sigma_decay), int(gamma_log2), int(seed),
        float(min_overlap_frac), x, int(have), int(k0), est, *trp,
        ptr(None if sig_base is None else _c(sig_base, np.float32)))
    if rc != 0:
        raise RuntimeError(f"orc_register failed: {rc}")
    out = dict(est=est, poses=x)
    out.update({"tr_" + k: v for k, v in tr.items()})
    return out
