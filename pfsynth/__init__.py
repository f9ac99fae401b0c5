"""Seeded synthetic inputs for the particle-filter rigid registration.

This module is the only code that both the CPU oracle (``oracle/``) and the
CUDA path (``paper_2504_19930_gb300``) rely on.  It holds none of the
registration method's arithmetic: it draws volumes, binary masks, frame
sequences and ground-truth poses.  Ground-truth rotations come from
``scipy.spatial.transform.Rotation`` (intrinsic z, x', y'' Euler angles), so
neither side's own pose-to-matrix code builds its own test inputs.

Conventions (shared by both sides, stated here so the generator is readable
alone):

* A volume is a numpy ``uint8`` array of shape ``(Z, Y, X)`` (x fastest);
  its dims triple is ``(X, Y, Z)``.
* Every grid carries a world origin ``o`` in voxel units (spacing 1), so
  voxel index ``p`` sits at world position ``p + o``.
* A pose is ``[rx, ry, rz, tx, ty, tz]`` (radians, voxels).  It maps a target
  world point ``w`` to the source world point ``R (w - c) + c + t`` with
  ``R = Rz(rz) Rx(rx) Ry(ry)`` and ``c`` the centre of the source grid,
  ``c = o_S + (dims_S - 1) / 2``.

The stand-ins follow the paper's data description (Sec. 3.2, Table 1): uint8
echo volumes of about 224 x 208 x 176 voxels and binary left-ventricle masks.
The paper's data is private; nothing here reproduces it.
"""
from __future__ import annotations

import hashlib
import os
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial.transform import Rotation

__all__ = [
    "Pair",
    "rotation_zxy",
    "map_target_to_source",
    "ellipsoid_pair",
    "speckle_pair",
    "frame_sequence",
    "random_image",
    "random_mask",
    "MASK64",
    "IMAGE224",
    "COMBINED256",
]


@dataclass
class Pair:
    """A source/target pair with its geometry and the pose that made it."""

    src: np.ndarray                 # (Zs, Ys, Xs) uint8
    tgt: np.ndarray                 # (Zt, Yt, Xt) uint8
    src_origin: np.ndarray          # float32[3], world origin of the source grid
    tgt_origin: np.ndarray          # float32[3], world origin of the target grid
    true_pose: np.ndarray           # float32[6], rx ry rz tx ty tz
    src_mask: np.ndarray | None = None
    tgt_mask: np.ndarray | None = None
    info: dict = field(default_factory=dict)
    src_spacing: np.ndarray = field(default_factory=lambda: np.ones(3, np.float32))   # world units per voxel
    tgt_spacing: np.ndarray = field(default_factory=lambda: np.ones(3, np.float32))

    @property
    def src_dims(self):
        return (self.src.shape[2], self.src.shape[1], self.src.shape[0])

    @property
    def tgt_dims(self):
        return (self.tgt.shape[2], self.tgt.shape[1], self.tgt.shape[0])


def rotation_zxy(pose) -> np.ndarray:
    """Rz(rz) @ Rx(rx) @ Ry(ry) as float64, built by scipy (intrinsic 'ZXY')."""
    rx, ry, rz = (float(v) for v in pose[:3])
    return Rotation.from_euler("ZXY", [rz, rx, ry]).as_matrix()


def _centre(dims, origin, spacing=(1.0, 1.0, 1.0)):
    return np.asarray(origin, np.float64) + np.asarray(spacing, np.float64) * \
        ((np.asarray(dims, np.float64) - 1.0) / 2.0)


def map_target_to_source(pose, src_dims, src_origin, tgt_origin, pts_tgt_index,
                         src_spacing=(1.0, 1.0, 1.0), tgt_spacing=(1.0, 1.0, 1.0)):
    """World-space map of target voxel indices (…,3 as x,y,z) into source world
    (voxel p of a grid sits at origin + spacing * p)."""
    R = rotation_zxy(pose)
    c = _centre(src_dims, src_origin, src_spacing)
    w = np.asarray(pts_tgt_index, np.float64) * np.asarray(tgt_spacing, np.float64) + \
        np.asarray(tgt_origin, np.float64)
    return (w - c) @ R.T + c + np.asarray(pose[3:6], np.float64)


def _grid(dims, origin, dtype=np.float64, spacing=(1.0, 1.0, 1.0)):
    X, Y, Z = dims
    z, y, x = np.meshgrid(
        np.arange(Z, dtype=dtype), np.arange(Y, dtype=dtype), np.arange(X, dtype=dtype),
        indexing="ij",
    )
    o = np.asarray(origin, dtype)
    sp = np.asarray(spacing, dtype)
    return x * sp[0] + o[0], y * sp[1] + o[1], z * sp[2] + o[2]


def _warp_grid(pose, src_dims, src_origin, tgt_dims, tgt_origin, dtype=np.float64,
               src_spacing=(1.0, 1.0, 1.0), tgt_spacing=(1.0, 1.0, 1.0)):
    """Source-world coordinates of every target voxel, each (Zt,Yt,Xt)."""
    R = rotation_zxy(pose).astype(dtype)
    c = _centre(src_dims, src_origin, src_spacing).astype(dtype)
    t = np.asarray(pose[3:6], dtype)
    wx, wy, wz = _grid(tgt_dims, tgt_origin, dtype, tgt_spacing)
    dx, dy, dz = wx - c[0], wy - c[1], wz - c[2]
    sx = R[0, 0] * dx + R[0, 1] * dy + R[0, 2] * dz + c[0] + t[0]
    sy = R[1, 0] * dx + R[1, 1] * dy + R[1, 2] * dz + c[1] + t[1]
    sz = R[2, 0] * dx + R[2, 1] * dy + R[2, 2] * dz + c[2] + t[2]
    return sx, sy, sz


# --------------------------------------------------------------------------
# Binary left-ventricle mask stand-in: ellipsoid (optionally with an
# off-axis sphere that breaks its rotational symmetry).
# --------------------------------------------------------------------------

def _ellipsoid_indicator(wx, wy, wz, centre, axes, bump=None):
    e = ((wx - centre[0]) / axes[0]) ** 2 + ((wy - centre[1]) / axes[1]) ** 2 \
        + ((wz - centre[2]) / axes[2]) ** 2
    m = e <= 1.0
    if bump is not None:
        bc, br = bump
        m |= ((wx - bc[0]) ** 2 + (wy - bc[1]) ** 2 + (wz - bc[2]) ** 2) <= br * br
    return m.astype(np.uint8)


def ellipsoid_pair(seed: int = 0, src_dims=(64, 64, 64), tgt_dims=(64, 64, 45),
                   tgt_origin=(0.0, 0.0, 19.0), semi_axes=(20.0, 14.0, 14.0),
                   max_rot_deg: float = 10.0, max_trans: float = 5.0,
                   asymmetric: bool = False, true_pose=None, src_spacing=(1.0, 1.0, 1.0),
                   tgt_spacing=(1.0, 1.0, 1.0)) -> Pair:
    """Binary mask pair: an ellipsoid and its rigidly moved, cropped copy.

    The source is the ellipsoid sampled on the source grid (origin 0).  The
    target is the same analytic shape evaluated at the ground-truth map of every
    target voxel (no resampling of the source), on a grid whose origin crops
    the field of view.  ``asymmetric`` adds an off-axis sphere so all six
    degrees of freedom are identifiable.  Grids may have anisotropic voxel
    sizes (spacings); centre, semi-axes, origins and translations are then in
    world units.
    """
    rng = np.random.default_rng(seed)
    src_origin = np.zeros(3, np.float32)
    centre = _centre(src_dims, src_origin, src_spacing) + rng.uniform(-1, 1, 3)
    axes = np.asarray(semi_axes, np.float64) + rng.uniform(-1, 1, 3)
    if true_pose is None:
        rot = np.deg2rad(rng.uniform(-max_rot_deg, max_rot_deg, 3))
        tr = rng.uniform(-max_trans, max_trans, 3)
        true_pose = np.concatenate([rot, tr])
    true_pose = np.asarray(true_pose, np.float32)
    bump = None
    if asymmetric:
        bump = (centre + np.array([0.55 * axes[0], 0.75 * axes[1], 0.0]), 0.45 * axes[1])
    sx, sy, sz = _grid(src_dims, src_origin, spacing=src_spacing)
    src = _ellipsoid_indicator(sx, sy, sz, centre, axes, bump)
    wx, wy, wz = _warp_grid(true_pose, src_dims, src_origin, tgt_dims, tgt_origin,
                            src_spacing=src_spacing, tgt_spacing=tgt_spacing)
    tgt = _ellipsoid_indicator(wx, wy, wz, centre, axes, bump)
    return Pair(src=src, tgt=tgt, src_origin=src_origin,
                tgt_origin=np.asarray(tgt_origin, np.float32), true_pose=true_pose,
                src_mask=src, tgt_mask=tgt,
                info={"centre": centre, "semi_axes": axes, "bump": bump},
                src_spacing=np.asarray(src_spacing, np.float32), tgt_spacing=np.asarray(tgt_spacing, np.float32))


# --------------------------------------------------------------------------
# Echo-like image stand-in: Rayleigh speckle over a bright myocardial shell.
# --------------------------------------------------------------------------

_M1 = np.uint64(0x9E3779B97F4A7C15)
_M2 = np.uint64(0xC2B2AE3D27D4EB4F)
_M3 = np.uint64(0x165667B19E3779F9)


def _splitmix(h):
    h = h ^ (h >> np.uint64(30))
    h = h * np.uint64(0xBF58476D1CE4E5B9)
    h = h ^ (h >> np.uint64(27))
    h = h * np.uint64(0x94D049BB133111EB)
    return h ^ (h >> np.uint64(31))


def _speckle(wx, wy, wz, sigma, seed):
    """Rayleigh(sigma) speckle hashed from the rounded world voxel, so two
    views of the same tissue see the same speckle grain."""
    ix = np.rint(wx).astype(np.int64).astype(np.uint64)
    iy = np.rint(wy).astype(np.int64).astype(np.uint64)
    iz = np.rint(wz).astype(np.int64).astype(np.uint64)
    with np.errstate(over="ignore"):
        h = (ix * _M1) ^ (iy * _M2) ^ (iz * _M3) ^ np.uint64(seed * 0x2545F4914F6CDD1D % (1 << 64))
        h = _splitmix(h)
    u = ((h >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
    return sigma * np.sqrt(-2.0 * np.log(u))


@dataclass
class _Heart:
    centre: np.ndarray
    outer: np.ndarray       # outer semi-axes of the myocardial shell
    thickness: float
    base_x: float           # the shell is cut open at x > base_x (the valve plane)


def _tissue(wx, wy, wz, heart: _Heart, scale: float = 1.0):
    """Brightness: myocardium 1.0, blood pool 0.15, background 0.3."""
    outer = heart.outer * scale
    inner = outer - heart.thickness
    ux, uy, uz = wx - heart.centre[0], wy - heart.centre[1], wz - heart.centre[2]
    eo = (ux / outer[0]) ** 2 + (uy / outer[1]) ** 2 + (uz / outer[2]) ** 2
    ei = (ux / inner[0]) ** 2 + (uy / inner[1]) ** 2 + (uz / inner[2]) ** 2
    out = np.full(wx.shape, 0.3, np.float64)
    myo = (eo <= 1.0) & (ei > 1.0) & (ux <= heart.base_x)
    pool = (ei <= 1.0) & (ux <= heart.base_x)
    out[myo] = 1.0
    out[pool] = 0.15
    return out


def _gain(dims, rng, amplitude=0.3):
    """Smooth multiplicative gain 1 + amplitude * (low-frequency cosine field)
    on a view's own voxel grid; amplitude 0.3 gives the +-30 % spread."""
    X, Y, Z = dims
    z, y, x = np.meshgrid(np.arange(Z) / Z, np.arange(Y) / Y, np.arange(X) / X, indexing="ij")
    field_ = np.zeros_like(x)
    for _ in range(3):
        f = rng.uniform(0.3, 1.2, 3)
        ph = rng.uniform(0, 2 * np.pi)
        field_ += np.cos(2 * np.pi * (f[0] * x + f[1] * y + f[2] * z) + ph)
    field_ /= 3.0
    return 1.0 + amplitude * field_


def _make_heart(src_dims, rng):
    c = (np.asarray(src_dims, np.float64) - 1.0) / 2.0 + rng.uniform(-4, 4, 3)
    outer = np.array([0.36 * src_dims[0], 0.26 * src_dims[1], 0.28 * src_dims[2]]) \
        * rng.uniform(0.95, 1.05, 3)
    return _Heart(centre=c, outer=outer, thickness=0.055 * src_dims[0],
                  base_x=0.55 * outer[0])


def _to_u8(v):
    return np.clip(np.rint(v), 0, 255).astype(np.uint8)


def _overlap_fraction(pose, src_dims, tgt_dims, tgt_origin, stride=4):
    """Fraction of (strided) target voxels whose mapped point lies inside the
    source grid; used only to place the target field of view."""
    sub = tuple(max(1, (d + stride - 1) // stride) for d in tgt_dims)
    X, Y, Z = sub
    z, y, x = np.meshgrid(np.arange(Z) * stride, np.arange(Y) * stride,
                          np.arange(X) * stride, indexing="ij")
    pts = np.stack([x, y, z], -1).reshape(-1, 3).astype(np.float64)
    pts = pts[(pts[:, 0] < tgt_dims[0]) & (pts[:, 1] < tgt_dims[1]) & (pts[:, 2] < tgt_dims[2])]
    q = map_target_to_source(pose, src_dims, np.zeros(3), tgt_origin, pts)
    ok = np.all((q >= 0) & (q <= np.asarray(src_dims, np.float64) - 1), axis=1)
    return float(ok.mean())


def speckle_pair(seed: int = 0, src_dims=(224, 208, 176), tgt_dims=None,
                 overlap=(0.35, 0.60), max_rot_deg: float = 15.0, max_trans: float = 12.0,
                 sigma: float = 40.0, gain_amplitude: float = 0.3,
                 with_masks: bool = False, true_pose=None) -> Pair:
    """Echo-like image pair: Rayleigh speckle (sigma 40) over a cut-open
    ellipsoidal myocardial shell, each view with its own smooth gain field.

    The target field of view is shifted along x (through its origin) until the
    fraction of target voxels that see the source reaches a draw from
    ``overlap``.  With ``with_masks`` the left-ventricle cavity masks of both
    views are returned as well.
    """
    if tgt_dims is None:
        tgt_dims = src_dims
    rng = np.random.default_rng(seed)
    src_origin = np.zeros(3, np.float32)
    heart = _make_heart(src_dims, rng)
    if true_pose is None:
        rot = np.deg2rad(rng.uniform(-max_rot_deg, max_rot_deg, 3))
        tr = rng.uniform(-max_trans, max_trans, 3)
        true_pose = np.concatenate([rot, tr])
    true_pose = np.asarray(true_pose, np.float32)
    want = rng.uniform(*overlap)
    # Target origin: centre the target on the source, then slide it along x.
    base = (np.asarray(src_dims, np.float64) - np.asarray(tgt_dims, np.float64)) / 2.0
    lo, hi = 0.0, float(src_dims[0])
    for _ in range(30):
        mid = 0.5 * (lo + hi)
        o = base + np.array([mid, 0.0, 0.0])
        if _overlap_fraction(true_pose, src_dims, tgt_dims, o) > want:
            lo = mid
        else:
            hi = mid
    tgt_origin = np.round(base + np.array([0.5 * (lo + hi), 0.0, 0.0])).astype(np.float32)
    speckle_seed = int(rng.integers(0, 2**31))
    g_src = _gain(src_dims, rng, gain_amplitude)
    g_tgt = _gain(tgt_dims, rng, gain_amplitude)
    sx, sy, sz = _grid(src_dims, src_origin)
    src = _to_u8(_tissue(sx, sy, sz, heart) * _speckle(sx, sy, sz, sigma, speckle_seed) * g_src)
    wx, wy, wz = _warp_grid(true_pose, src_dims, src_origin, tgt_dims, tgt_origin)
    tgt = _to_u8(_tissue(wx, wy, wz, heart) * _speckle(wx, wy, wz, sigma, speckle_seed) * g_tgt)
    pair = Pair(src=src, tgt=tgt, src_origin=src_origin, tgt_origin=tgt_origin,
                true_pose=true_pose,
                info={"overlap_target": want, "speckle_seed": speckle_seed,
                      "heart": heart, "sigma": sigma})
    if with_masks:
        pair.src_mask = _cavity(sx, sy, sz, heart)
        pair.tgt_mask = _cavity(wx, wy, wz, heart)
    return pair


def _cavity(wx, wy, wz, heart: _Heart, scale: float = 1.0):
    inner = heart.outer * scale - heart.thickness
    ux, uy, uz = wx - heart.centre[0], wy - heart.centre[1], wz - heart.centre[2]
    ei = (ux / inner[0]) ** 2 + (uy / inner[1]) ** 2 + (uz / inner[2]) ** 2
    return ((ei <= 1.0) & (ux <= heart.base_x)).astype(np.uint8)


def frame_sequence(pair: Pair, n_frames: int = 20, dilation: float = 0.08,
                   seed: int = 0) -> np.ndarray:
    """Source-view cardiac cycle: frame f scales the shell by
    1 + dilation * sin(2 pi f / n_frames).  Returns (F, Zs, Ys, Xs) uint8."""
    heart = pair.info["heart"]
    rng = np.random.default_rng(seed + 7919)
    g = _gain(pair.src_dims, rng, 0.3)
    sx, sy, sz = _grid(pair.src_dims, pair.src_origin)
    speck = _speckle(sx, sy, sz, pair.info["sigma"], pair.info["speckle_seed"]) * g
    out = np.empty((n_frames,) + pair.src.shape, np.uint8)
    for f in range(n_frames):
        scale = 1.0 + dilation * np.sin(2.0 * np.pi * f / n_frames)
        out[f] = _to_u8(_tissue(sx, sy, sz, heart, scale) * speck)
    return out


# --------------------------------------------------------------------------
# Small random volumes for unit and parity tests.
# --------------------------------------------------------------------------

def random_image(seed: int, dims, smooth: bool = True) -> np.ndarray:
    """uint8 (Z,Y,X) volume: smooth random blobs plus noise (or pure noise)."""
    rng = np.random.default_rng(seed)
    X, Y, Z = dims
    if not smooth:
        return rng.integers(0, 256, (Z, Y, X), dtype=np.uint8)
    z, y, x = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    v = np.zeros((Z, Y, X))
    for _ in range(6):
        c = rng.uniform(0, 1, 3) * np.array([X, Y, Z])
        r = rng.uniform(0.15, 0.4) * min(X, Y, Z) + 1.0
        v += rng.uniform(40, 120) * np.exp(-(((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
                                          / (2 * r * r)))
    v += rng.normal(0, 12, v.shape)
    return _to_u8(v + 20)


def random_mask(seed: int, dims, fill: float = 0.5) -> np.ndarray:
    """Binary uint8 (Z,Y,X) mask: union of random balls (fill is approximate)."""
    rng = np.random.default_rng(seed)
    X, Y, Z = dims
    z, y, x = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    m = np.zeros((Z, Y, X), bool)
    while m.mean() < fill:
        c = rng.uniform(0, 1, 3) * np.array([X, Y, Z])
        r = rng.uniform(0.1, 0.35) * min(X, Y, Z) + 1.0
        m |= ((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) <= r * r
    return m.astype(np.uint8)


# --------------------------------------------------------------------------
# Named workloads (sizes and PF settings of the three single-GPU cases).
# --------------------------------------------------------------------------

MASK64 = dict(  # mask-based, 64^3 ellipsoid, N=256, 10 iterations
    name="mask64_dice_n256_k10", mode="mask_dice", n_particles=256, n_iters=10,
    rot_limit_deg=15.0, trans_limit=8.0, seed=0)
IMAGE224 = dict(  # image-based, 224x208x176 speckle, N=2048, 50 iterations, 20-frame warp
    name="speckle224x208x176_ncc_n2048_k50_warp20", mode="image_ncc", n_particles=2048,
    n_iters=50, rot_limit_deg=30.0, trans_limit=25.0, seed=0, n_frames=20)
COMBINED256 = dict(  # combined image+mask, 256^3, N=16384, 40 iterations, 30-frame warp
    name="stress256_combined_n16384_k40_warp30", mode="combined", n_particles=16384,
    n_iters=40, rot_limit_deg=45.0, trans_limit=32.0, seed=0, n_frames=30)


def cached(fn, *args, cache_dir=None, **kwargs):
    """Memoise a generator call on disk (keyed by its arguments)."""
    import pickle
    cache_dir = cache_dir or os.environ.get("PFSYNTH_CACHE", "/tmp/pfsynth_cache")
    key = hashlib.sha1(pickle.dumps((fn.__name__, args, sorted(kwargs.items())),
                                    protocol=4)).hexdigest()[:16]
    path = os.path.join(cache_dir, f"{fn.__name__}_{key}.pkl")
    if os.path.exists(path):
        try:
            with open(path, "rb") as f:
                return pickle.load(f)
        except Exception:
            pass
    obj = fn(*args, **kwargs)
    try:
        os.makedirs(cache_dir, exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "wb") as f:
            pickle.dump(obj, f, protocol=pickle.HIGHEST_PROTOCOL)
        os.replace(tmp, path)
    except OSError:
        pass
    return obj
