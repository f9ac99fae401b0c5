"""GB300-native particle-filter 3D-3D rigid registration.

Thin Python binding of ``libpfreg.so`` (C ABI in ``include/pfreg.h``).  It only
marshals arguments: every step of the registration runs in the library's
sm_103a kernels.  PyTorch provides device memory and streams.  There is no
CPU fallback: when the library is missing or no GPU is present the calls
raise.

Functions carry the C names (``pf_register_init``, ``pf_step``,
``pf_estimate``, ``warp_sequence``, ...).  :class:`Registration` wraps one
context for convenience.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from ._build import LIB as _LIB_RELEASE
from ._build import LIB_DEBUG as _LIB_DEBUG
from ._build import build as _build_lib

# PFREG_DEBUG=1 loads the bounds-checked build (libpfreg_debug.so) instead.
_DEBUG = os.environ.get("PFREG_DEBUG", "0") == "1"
_LIB_PATH = _LIB_DEBUG if _DEBUG else _LIB_RELEASE

__all__ = [
    "PF_MASK_DICE", "PF_MASK_NCC", "PF_IMAGE_NCC", "PF_COMBINED", "PfError", "load",
    "pf_config_default", "pf_register_init", "pf_step", "pf_estimate", "pf_register_destroy",
    "warp_sequence", "pf_get_iteration", "pf_get_state", "pf_set_state", "pf_get_log",
    "pf_measure_matrices", "pf_pose_matrix", "pf_philox", "pf_kernel_launches", "pf_last_error",
    "pf_profile_begin", "pf_profile_end", "register_sequence", "pf_measure_matrices_noalloc",
    "pf_step_measure", "pf_step_update", "pf_moments_device", "pf_debug_device_allocs", "pf_probe_read", "pf_debug_bounds",
    "Batch", "pf_batch_create", "pf_batch_step", "pf_batch_run", "pf_batch_destroy",
    "Registration", "MODES", "build", "library_path",
]

PF_MASK_DICE, PF_MASK_NCC, PF_IMAGE_NCC, PF_COMBINED = 0, 1, 2, 3
MODES = {"mask_dice": 0, "mask_ncc": 1, "image_ncc": 2, "combined": 3}
MOM_STRIDE = 12   # [n S1 S2lo S2hi ST T1 T2 0 | n_nn A B C]
_ERRORS = {-1: "PF_EINVAL", -2: "PF_ENOMEM", -3: "PF_ECUDA", -4: "PF_ETIMEOUT", -5: "PF_ESTATE"}


class PfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class pf_volume(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dims", C.c_int32 * 3), ("origin", C.c_float * 3),
                ("is_device", C.c_int32), ("spacing", C.c_float * 3)]


class pf_config(C.Structure):
    _fields_ = [("mode", C.c_int32), ("n_particles", C.c_int32), ("rot_limit", C.c_float * 3),
                ("trans_limit", C.c_float * 3), ("sigma0_frac", C.c_float),
                ("sigma_decay", C.c_float), ("gamma_log2", C.c_int32), ("seed", C.c_uint64),
                ("min_overlap_frac", C.c_float), ("trace_estimate", C.c_int32), ("estimator", C.c_int32),
                ("autotune", C.c_int32)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _LIB_PATH


def build(force: bool = False, debug: bool = None) -> str:
    """Build the release library (and the debug one when debug is True or the
    process runs with PFREG_DEBUG=1); returns the path this process loads."""
    _build_lib(force=force, debug=_DEBUG if debug is None else debug)
    return _LIB_PATH


def load():
    """Load libpfreg.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(
                    f"{os.path.basename(_LIB_PATH)} not found at {_LIB_PATH}; build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(_LIB_PATH)
            _declare(L)
            _lib = L
    return _lib


def _declare(L):
    vp, i32, u64 = C.c_void_p, C.c_int32, C.c_uint64
    L.pf_config_default.argtypes = [C.POINTER(pf_config)]
    L.pf_config_default.restype = None
    L.pf_register_init.argtypes = [C.POINTER(vp), C.POINTER(pf_volume), C.POINTER(pf_volume),
                                   C.POINTER(pf_volume), C.POINTER(pf_volume), C.POINTER(pf_config), vp]
    L.pf_step.argtypes = [vp, i32]
    L.pf_estimate.argtypes = [vp, vp, vp]
    L.pf_register_destroy.argtypes = [vp]
    L.warp_sequence.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp]
    L.pf_get_iteration.argtypes = [vp, vp]
    L.pf_get_state.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.pf_set_state.argtypes = [vp, vp, i32]
    L.pf_get_log.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.pf_measure_matrices.argtypes = [vp, vp, i32, vp, vp]
    L.pf_pose_matrix.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.pf_philox.argtypes = [vp, vp, vp]
    L.pf_measure_matrices_noalloc.argtypes = [vp, vp, i32, vp, vp]
    L.pf_batch_create.argtypes = [C.POINTER(vp), vp, i32, vp]
    L.pf_batch_step.argtypes = [vp, i32]
    L.pf_batch_run.argtypes = [vp]
    L.pf_batch_destroy.argtypes = [vp]
    L.pf_profile_begin.argtypes = [vp, i32]
    L.pf_profile_end.argtypes = [vp, vp, vp]
    L.pf_step_measure.argtypes = [vp, i32, i32]
    L.pf_step_update.argtypes = [vp]
    L.pf_moments_device.argtypes = [vp, vp, vp]
    L.pf_kernel_launches.argtypes = []
    L.pf_kernel_launches.restype = u64
    L.pf_debug_device_allocs.argtypes = []
    L.pf_debug_device_allocs.restype = u64
    L.pf_probe_read.argtypes = [vp, C.c_int64, i32, vp, vp]
    L.pf_probe_read.restype = C.c_int
    L.pf_debug_bounds.argtypes = [i32, vp, vp, vp]
    L.pf_debug_bounds.restype = C.c_int
    L.pf_last_error.argtypes = []
    L.pf_last_error.restype = C.c_char_p
    L.pf_nn_gemm_bf16.argtypes = [vp, vp, vp, i32, i32, vp]
    L.pf_nn_conv3d_forward.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp]
    L.pf_nn_conv3d_backward_data.argtypes = [vp, i32, i32, vp, vp, vp, vp]
    L.pf_nn_conv3d_backward_weights.argtypes = [vp, i32, i32, i32, vp, vp, vp]
    L.pf_nn_status.argtypes = [i32, vp]
    L.pf_seed_gaussian.argtypes = [vp, vp, vp]
    L.pf_tile_shape.argtypes = [vp, vp, vp]
    L.pf_debug_alloc_limit.argtypes = [C.c_int64]
    L.pf_nn_wait_selftest.argtypes = [vp]
    L.pf_batch_tile_shape.argtypes = [vp, vp]
    L.pf_proposal_create.argtypes = [C.POINTER(vp), i32, u64, vp]
    L.pf_proposal_destroy.argtypes = [vp]
    L.pf_proposal_train.argtypes = [vp, i32, i32, C.c_float, u64, vp, C.c_float, C.c_float, vp]
    L.pf_proposal_predict.argtypes = [vp, C.POINTER(pf_volume), C.POINTER(pf_volume), vp, vp]
    L.pf_proposal_params.argtypes = [vp, vp, vp, vp, vp]
    L.pf_proposal_forward.argtypes = [vp, vp, i32, vp, vp]
    L.pf_proposal_backward.argtypes = [vp, vp, i32, vp]
    L.pf_proposal_synth.argtypes = [vp, i32, u64, i32, vp, C.c_float, C.c_float, vp, vp]
    L.pf_proposal_input.argtypes = [vp, C.POINTER(pf_volume), C.POINTER(pf_volume), vp]
    L.pf_proposal_tensor.argtypes = [vp, i32, i32, vp]
    for name in ("pf_nn_gemm_bf16", "pf_nn_conv3d_forward", "pf_nn_conv3d_backward_data",
                 "pf_nn_conv3d_backward_weights", "pf_nn_status", "pf_seed_gaussian", "pf_proposal_create",
                 "pf_proposal_destroy", "pf_proposal_train", "pf_proposal_predict", "pf_proposal_params",
                 "pf_proposal_forward", "pf_proposal_backward", "pf_proposal_synth", "pf_proposal_input",
                 "pf_proposal_tensor",
                 "pf_tile_shape", "pf_batch_tile_shape", "pf_debug_alloc_limit", "pf_nn_wait_selftest"):
        getattr(L, name).restype = C.c_int
    for name in ("pf_register_init", "pf_step", "pf_estimate", "pf_register_destroy", "warp_sequence",
                 "pf_get_iteration", "pf_get_state", "pf_set_state", "pf_get_log",
                 "pf_measure_matrices", "pf_pose_matrix", "pf_philox", "pf_profile_begin",
                 "pf_profile_end", "pf_measure_matrices_noalloc", "pf_batch_create", "pf_batch_step",
                 "pf_batch_run", "pf_batch_destroy"):
        getattr(L, name).restype = C.c_int


def pf_last_error() -> str:
    return load().pf_last_error().decode()


def _check(rc):
    if rc != 0:
        raise PfError(rc, pf_last_error())
    return rc


def _ptr(a):
    """ctypes pointer of a numpy array (host) or torch tensor (host or device).
    The caller keeps ``a`` alive for the duration of the C call."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return C.c_void_p(a.ctypes.data)
    return C.c_void_p(a.data_ptr())


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def make_volume(vol, origin=(0.0, 0.0, 0.0), dims=None, spacing=(1.0, 1.0, 1.0)):
    """pf_volume from a (Z,Y,X) uint8 numpy array or torch tensor (CPU or CUDA);
    origin and spacing (x, y, z) in world units."""
    if vol is None:
        return None
    is_dev = 0
    if isinstance(vol, np.ndarray):
        if vol.dtype != np.uint8 or vol.ndim != 3 or not vol.flags.c_contiguous:
            raise ValueError("volume must be a C-contiguous (Z,Y,X) uint8 array")
        shape = vol.shape
    else:
        import torch
        if vol.dtype != torch.uint8 or vol.dim() != 3 or not vol.is_contiguous():
            raise ValueError("volume must be a contiguous (Z,Y,X) uint8 tensor")
        shape = tuple(vol.shape)
        is_dev = 1 if vol.is_cuda else 0
    v = pf_volume()
    v.data = _ptr(vol).value
    d = dims if dims is not None else (shape[2], shape[1], shape[0])
    v.dims[:] = [int(x) for x in d]
    v.origin[:] = [float(x) for x in origin]
    v.is_device = is_dev
    v.spacing[:] = [float(x) for x in np.broadcast_to(np.asarray(spacing, np.float32), (3,))]
    return v


def pf_config_default() -> pf_config:
    cfg = pf_config()
    load().pf_config_default(C.byref(cfg))
    return cfg


ESTIMATORS = {"mean": 0, "quaternion": 1}


def make_config(mode="mask_dice", n_particles=256, rot_limit=0.2617994, trans_limit=8.0,
                sigma0_frac=0.25, sigma_decay=0.8, gamma_log2=5, seed=0, min_overlap_frac=0.01,
                trace_estimate=False, estimator="mean", autotune=False):
    cfg = pf_config_default()
    cfg.mode = MODES.get(mode, mode)
    cfg.n_particles = int(n_particles)
    cfg.rot_limit[:] = [float(v) for v in np.broadcast_to(np.asarray(rot_limit, np.float32), (3,))]
    cfg.trans_limit[:] = [float(v) for v in np.broadcast_to(np.asarray(trans_limit, np.float32), (3,))]
    cfg.sigma0_frac = float(sigma0_frac)
    cfg.sigma_decay = float(sigma_decay)
    cfg.gamma_log2 = int(gamma_log2)
    cfg.seed = int(seed)
    cfg.min_overlap_frac = float(min_overlap_frac)
    cfg.trace_estimate = int(bool(trace_estimate))
    cfg.estimator = ESTIMATORS.get(estimator, estimator)
    cfg.autotune = int(bool(autotune))
    return cfg


def pf_register_init(src, tgt, src_mask, tgt_mask, cfg, stream=None):
    """Create a context; volumes are pf_volume structures (or None)."""
    ctx = C.c_void_p()
    ref = lambda v: C.byref(v) if v is not None else None  # noqa: E731
    _check(load().pf_register_init(C.byref(ctx), ref(src), ref(tgt), ref(src_mask), ref(tgt_mask),
                                   C.byref(cfg), _stream_handle(stream)))
    return ctx


def pf_step(ctx, n_iters):
    _check(load().pf_step(ctx, int(n_iters)))


def pf_step_measure(ctx, p_begin, p_end):
    _check(load().pf_step_measure(ctx, int(p_begin), int(p_end)))


def pf_step_update(ctx):
    _check(load().pf_step_update(ctx))


def pf_moments_device(ctx):
    """(device address, number of uint64 words) of the context's moment buffer."""
    ptr = C.c_void_p()
    n = C.c_int64()
    _check(load().pf_moments_device(ctx, C.byref(ptr), C.byref(n)))
    return ptr.value, n.value


class _DeviceWords:
    """A device buffer of int64 words seen through ``__cuda_array_interface__``."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<i8", "data": (int(ptr), False),
                                         "version": 3, "strides": None, "stream": None}


def pf_estimate(ctx, with_score=True):
    pose = np.zeros(6, np.float32)
    score = C.c_double()
    _check(load().pf_estimate(ctx, _ptr(pose), C.byref(score) if with_score else None))
    return pose, (score.value if with_score else None)


def pf_register_destroy(ctx):
    _check(load().pf_register_destroy(ctx))


def _spacing3(sp):
    return _np(np.broadcast_to(np.asarray(sp, np.float32), (3,)), np.float32)


def warp_sequence(frames_in, src_dims, src_origin, frames_out, tgt_dims, tgt_origin, pose,
                  interp=1, stream=None, src_spacing=(1.0, 1.0, 1.0), tgt_spacing=(1.0, 1.0, 1.0)):
    """frames_in / frames_out: sequences of CUDA uint8 tensors (one per frame)."""
    n = len(frames_in)
    if len(frames_out) != n:
        raise ValueError("frames_in and frames_out differ in length")
    fin = (C.c_void_p * max(n, 1))(*[f.data_ptr() for f in frames_in])
    fout = (C.c_void_p * max(n, 1))(*[f.data_ptr() for f in frames_out])
    sd, so, ss = _np(src_dims, np.int32), _np(src_origin, np.float32), _spacing3(src_spacing)
    td, to, ts = _np(tgt_dims, np.int32), _np(tgt_origin, np.float32), _spacing3(tgt_spacing)
    ps = _np(pose, np.float32)
    _check(load().warp_sequence(fin, n, _ptr(sd), _ptr(so), _ptr(ss), fout, _ptr(td), _ptr(to), _ptr(ts),
                                _ptr(ps), int(interp), _stream_handle(stream)))


def pf_get_iteration(ctx) -> int:
    k = C.c_int32()
    _check(load().pf_get_iteration(ctx, C.byref(k)))
    return k.value


def pf_get_state(ctx, n_particles):
    N = int(n_particles)
    out = dict(poses_measured=np.zeros((6, N), np.float32),
               moments=np.zeros((N, MOM_STRIDE), np.uint64), scores=np.zeros(N, np.float64),
               weights=np.zeros(N, np.uint64), resample_idx=np.zeros(N, np.int32),
               poses_next=np.zeros((6, N), np.float32))
    _check(load().pf_get_state(ctx, *[_ptr(out[k]) for k in ("poses_measured", "moments", "scores",
                                                              "weights", "resample_idx", "poses_next")]))
    return out


def pf_set_state(ctx, poses6xN, k):
    p = _np(poses6xN, np.float32)
    _check(load().pf_set_state(ctx, _ptr(p), int(k)))


def pf_get_log(ctx, capacity=4096):
    """(est [n,6], best [n], ess [n], evals [n], est_dice [n]) for the last n
    iterations (est_dice is -1 unless the context traces the estimate)."""
    est = np.zeros((capacity, 6), np.float64)
    best = np.zeros(capacity, np.float64)
    ess = np.zeros(capacity, np.float64)
    evals = np.zeros(capacity, np.uint64)
    dice = np.zeros(capacity, np.float64)
    n = C.c_int32(capacity)
    _check(load().pf_get_log(ctx, _ptr(est), _ptr(best), _ptr(ess), _ptr(evals), _ptr(dice), C.byref(n)))
    k = n.value
    return est[:k], best[:k], ess[:k], evals[:k], dice[:k]


def pf_measure_matrices(ctx, mats, a):
    m = _np(np.atleast_2d(mats), np.float32)
    out = np.zeros((m.shape[0], MOM_STRIDE), np.uint64)
    av = _np(a, np.float32)
    _check(load().pf_measure_matrices(ctx, _ptr(m), m.shape[0], _ptr(av), _ptr(out)))
    return out


NOALLOC_MAX_MATRICES = 4096


def pf_measure_matrices_noalloc(ctx, mats, a):
    """pf_measure_matrices without device allocation (fixed shared scratch of
    NOALLOC_MAX_MATRICES matrices; for callers that cannot allocate while
    running).  Calls that overlap on the GPU race on that scratch."""
    m = _np(np.atleast_2d(mats), np.float32)
    out = np.zeros((m.shape[0], MOM_STRIDE), np.uint64)
    av = _np(a, np.float32)
    _check(load().pf_measure_matrices_noalloc(ctx, _ptr(m), m.shape[0], _ptr(av), _ptr(out)))
    return out


def pf_pose_matrix(pose, src_dims, src_origin, tgt_origin, src_spacing=(1.0, 1.0, 1.0),
                   tgt_spacing=(1.0, 1.0, 1.0)):
    M = np.zeros(12, np.float32)
    a = np.zeros(3, np.float32)
    ps, sd = _np(pose, np.float32), _np(src_dims, np.int32)
    so, to = _np(src_origin, np.float32), _np(tgt_origin, np.float32)
    ss, ts = _spacing3(src_spacing), _spacing3(tgt_spacing)
    _check(load().pf_pose_matrix(_ptr(ps), _ptr(sd), _ptr(so), _ptr(ss), _ptr(to), _ptr(ts),
                                 _ptr(M), _ptr(a)))
    return M, a


def pf_philox(ctr, key):
    out = np.zeros(4, np.uint32)
    c, k = _np(ctr, np.uint32), _np(key, np.uint32)
    _check(load().pf_philox(_ptr(c), _ptr(k), _ptr(out)))
    return out


def pf_profile_begin(ctx, capacity):
    _check(load().pf_profile_begin(ctx, int(capacity)))


def pf_profile_end(ctx):
    """(summed measurement-kernel ms, number of timed iterations)."""
    tot = C.c_double()
    n = C.c_int32()
    _check(load().pf_profile_end(ctx, C.byref(tot), C.byref(n)))
    return tot.value, n.value


def pf_kernel_launches() -> int:
    return int(load().pf_kernel_launches())


def pf_debug_device_allocs() -> int:
    """Device allocations the library has made in this process (test hook)."""
    return int(load().pf_debug_device_allocs())


def pf_probe_read(buf, reps, sink, stream=None):
    """Launch the read-bandwidth probe over the device tensor ``buf`` (L1
    bypassed); the caller times it.  ``sink``: a device uint64/int64 tensor."""
    _check(load().pf_probe_read(_ptr(buf), int(buf.numel() * buf.element_size()), int(reps), _ptr(sink),
                                _stream_handle(stream)))


def pf_debug_bounds(clear=True):
    """(checks_on, hits, first_bad) of the debug build's gather bounds checks
    (synchronises the device; checks_on is False in the release build)."""
    on, hits, first = C.c_int32(0), C.c_uint64(0), C.c_int64(0)
    _check(load().pf_debug_bounds(1 if clear else 0, C.byref(on), C.byref(hits), C.byref(first)))
    return bool(on.value), int(hits.value), int(first.value)


class Registration:
    """One registration context.

    Volumes are (Z,Y,X) uint8 numpy arrays (host) or torch tensors (host or
    CUDA); the library copies them into its own device memory.
    """

    def __init__(self, mode, src=None, tgt=None, src_mask=None, tgt_mask=None,
                 src_origin=(0, 0, 0), tgt_origin=(0, 0, 0), stream=None, src_spacing=(1.0, 1.0, 1.0),
                 tgt_spacing=(1.0, 1.0, 1.0), **cfg):
        self.cfg = make_config(mode, **cfg)
        self.N = self.cfg.n_particles
        self.stream = stream
        vols = [make_volume(src, src_origin, spacing=src_spacing), make_volume(tgt, tgt_origin, spacing=tgt_spacing),
                make_volume(src_mask, src_origin, spacing=src_spacing),
                make_volume(tgt_mask, tgt_origin, spacing=tgt_spacing)]
        self.ctx = pf_register_init(*vols, self.cfg, stream)

    def step(self, n_iters=1):
        pf_step(self.ctx, n_iters)
        return self

    def tile_shape(self):
        """(rows per work item, work items per warp) of the measurement."""
        r, i = C.c_int32(0), C.c_int32(0)
        _check(load().pf_tile_shape(self.ctx, C.byref(r), C.byref(i)))
        return r.value, i.value

    def seed_gaussian(self, mean, std):
        """Seed the cloud around a proposal (before the first step)."""
        m, sd = _np(mean, np.float32), _np(std, np.float32)
        _check(load().pf_seed_gaussian(self.ctx, _ptr(m), _ptr(sd)))
        return self

    def estimate(self, with_score=True):
        return pf_estimate(self.ctx, with_score)

    @property
    def iteration(self):
        return pf_get_iteration(self.ctx)

    def state(self):
        return pf_get_state(self.ctx, self.N)

    def set_state(self, poses6xN, k):
        pf_set_state(self.ctx, poses6xN, k)

    def log(self):
        return pf_get_log(self.ctx)

    def measure(self, mats, a):
        return pf_measure_matrices(self.ctx, mats, a)

    # one iteration in two halves (the measurement sharded over processes)
    def step_measure(self, p_begin, p_end):
        pf_step_measure(self.ctx, p_begin, p_end)

    def step_update(self):
        pf_step_update(self.ctx)

    def moments(self):
        """The moment buffer as a CUDA int64 tensor [12 N] (a view, not a copy)."""
        import torch
        ptr, n = pf_moments_device(self.ctx)
        return torch.as_tensor(_DeviceWords(ptr, n), device="cuda")

    def close(self):
        if self.ctx is not None:
            pf_register_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _to_cuda(a, stream=None):
    import torch
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(a))
    if a.is_cuda:
        return a
    return a.cuda(non_blocking=True)


def register_sequence(mode, src=None, tgt=None, frames=(), n_iters=1, src_origin=(0, 0, 0),
                      tgt_origin=(0, 0, 0), src_mask=None, tgt_mask=None, interp=1, out=None,
                      with_score=False, src_spacing=(1.0, 1.0, 1.0), tgt_spacing=(1.0, 1.0, 1.0), **cfg):
    """Register source to target, then warp every source frame by the estimate.

    The whole user-facing path: volumes (host numpy / host or pinned torch /
    CUDA tensors) go to the device, ``n_iters`` filter iterations run, the
    estimate comes back, and all frames are warped into the target grid.
    ``frames`` is a sequence (or (F,Z,Y,X) array) of source-grid frames.
    ``out``: optional list of host (pinned) uint8 tensors for the warped frames;
    when given they are filled and returned, else CUDA tensors are returned.

    Returns (pose float32[6], score or None, warped frames).
    """
    import torch
    reg = Registration(mode, src=src, tgt=tgt, src_mask=src_mask, tgt_mask=tgt_mask,
                       src_origin=src_origin, tgt_origin=tgt_origin, src_spacing=src_spacing,
                       tgt_spacing=tgt_spacing, **cfg)
    try:
        reg.step(n_iters)
        pose, score = reg.estimate(with_score)
    finally:
        reg.close()
    ref = src if src is not None else src_mask
    tgt_ref = tgt if tgt is not None else tgt_mask
    sdims = (ref.shape[2], ref.shape[1], ref.shape[0])
    tshape = tuple(tgt_ref.shape)
    fin = [_to_cuda(f) for f in frames]
    fout = [torch.empty(tshape, dtype=torch.uint8, device="cuda") for _ in fin]
    warp_sequence(fin, sdims, src_origin, fout, (tshape[2], tshape[1], tshape[0]), tgt_origin, pose,
                  interp, src_spacing=src_spacing, tgt_spacing=tgt_spacing)
    if out is not None:
        for o, f in zip(out, fout):
            o.copy_(f, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return pose, score, out
    return pose, score, fout


def pf_batch_create(ctxs, n_iters):
    """Batch of contexts (c_void_p handles) with per-registration counts."""
    arr = (C.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    its = _np(n_iters, np.int32)
    b = C.c_void_p()
    _check(load().pf_batch_create(C.byref(b), arr, len(ctxs), _ptr(its)))
    return b


def pf_batch_step(b, n_iters):
    _check(load().pf_batch_step(b, int(n_iters)))


def pf_batch_run(b):
    _check(load().pf_batch_run(b))


def pf_batch_destroy(b):
    _check(load().pf_batch_destroy(b))


class Batch:
    """Several Registration objects (same stream) stepped together."""

    def __init__(self, registrations, n_iters):
        self.regs = list(registrations)
        self.handle = pf_batch_create([r.ctx for r in self.regs], n_iters)

    def run(self):
        pf_batch_run(self.handle)
        return self

    def tile_shape(self):
        """Work items per warp of the batch's measurement launches."""
        i = C.c_int32(0)
        _check(load().pf_batch_tile_shape(self.handle, C.byref(i)))
        return i.value

    def step(self, n_iters=1):
        pf_batch_step(self.handle, n_iters)
        return self

    def close(self):
        if self.handle is not None:
            pf_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ proposal network contractions
# Thin wrappers over the pf_nn_* exports (tensor-core kernels); tensors are
# torch CUDA tensors, bf16 in NDHWC layout, shapes as in include/pfreg.h.

def _need(t, dtype, shape=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"expected a contiguous CUDA tensor of {dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")


def nn_gemm_bf16(A, B, C, stream=None):
    """C[M][32] = A[M][K] @ B[32][K]^T on the tensor cores (fp32 out)."""
    import torch
    M, K = A.shape
    _need(A, torch.bfloat16), _need(B, torch.bfloat16, (32, K)), _need(C, torch.float32, (M, 32))
    _check(load().pf_nn_gemm_bf16(_ptr(A), _ptr(B), _ptr(C), int(M), int(K), _stream_handle(stream)))


def nn_conv3d_forward(x, w, bias, y, stream=None):
    """y = relu(conv3d(x, w, stride 2, padding 1) + bias); x (B,D,D,D,Cin), y (B,D/2,D/2,D/2,32)."""
    import torch
    Bn, D, _, _, Cin = x.shape
    _need(x, torch.bfloat16), _need(w, torch.bfloat16, (32, 64, Cin)), _need(bias, torch.float32, (32,))
    _need(y, torch.bfloat16, (Bn, D // 2, D // 2, D // 2, 32))
    _check(load().pf_nn_conv3d_forward(_ptr(x), int(Bn), int(D), int(Cin), _ptr(w), _ptr(bias), _ptr(y),
                                       _stream_handle(stream)))


def nn_conv3d_backward_data(dy, w_t, act, dx, stream=None):
    """dx = mask(act) * conv3d-transpose(dy, w); w_t is w as [ci][tap][co]; act may be None."""
    import torch
    Bn, D = dx.shape[0], dx.shape[1]
    _need(dy, torch.bfloat16, (Bn, D // 2, D // 2, D // 2, 32)), _need(w_t, torch.bfloat16, (32, 64, 32))
    _need(dx, torch.bfloat16, (Bn, D, D, D, 32))
    if act is not None:
        _need(act, torch.bfloat16, (Bn, D, D, D, 32))
    _check(load().pf_nn_conv3d_backward_data(_ptr(dy), int(Bn), int(D), _ptr(w_t), _ptr(act), _ptr(dx),
                                             _stream_handle(stream)))


def nn_conv3d_backward_weights(x, dy, dw, stream=None):
    """dw[co][tap][ci] += sum_{b,o} x[b, 2o+k-1, ci] dy[b, o, co] (fp32)."""
    import torch
    Bn, D, _, _, Cin = x.shape
    _need(x, torch.bfloat16), _need(dy, torch.bfloat16, (Bn, D // 2, D // 2, D // 2, 32))
    _need(dw, torch.float32, (32, 64, Cin))
    _check(load().pf_nn_conv3d_backward_weights(_ptr(x), int(Bn), int(D), int(Cin), _ptr(dy), _ptr(dw),
                                                _stream_handle(stream)))


def nn_status(clear=True) -> int:
    """1 when a tensor-core kernel's bounded wait ran out since the last clear."""
    v = C.c_int32(0)
    _check(load().pf_nn_status(1 if clear else 0, C.byref(v)))
    return int(v.value)


# ------------------------------------------------------------------ learned proposal network

class Proposal:
    """The learned proposal network (pf_proposal_*): trains on synthetic
    pairs generated on the GPU and predicts a pose mean and spread that seed
    a registration's particle cloud."""

    N_PARAMS = 464652

    def __init__(self, max_batch=32, seed=0, stream=None):
        self.stream = stream
        h = C.c_void_p()
        _check(load().pf_proposal_create(C.byref(h), int(max_batch), int(seed), _stream_handle(stream)))
        self.h = h
        self.max_batch = int(max_batch)

    def train(self, n_steps, batch=32, lr=1e-3, data_seed=1, vol_dims=(224, 208, 176),
              rot_limit=0.5235988, trans_limit=25.0, with_loss=True):
        loss = np.zeros(max(int(n_steps), 1), np.float32) if with_loss else None
        dims = _np(vol_dims, np.int32)
        _check(load().pf_proposal_train(self.h, int(n_steps), int(batch), float(lr), int(data_seed), _ptr(dims),
                                        float(rot_limit), float(trans_limit), _ptr(loss)))
        return loss[:int(n_steps)] if with_loss else None

    def predict(self, src, tgt, src_origin=(0, 0, 0), tgt_origin=(0, 0, 0), src_spacing=(1, 1, 1),
                tgt_spacing=(1, 1, 1)):
        vs, vt = make_volume(src, src_origin, spacing=src_spacing), make_volume(tgt, tgt_origin, spacing=tgt_spacing)
        mean, std = np.zeros(6, np.float32), np.zeros(6, np.float32)
        _check(load().pf_proposal_predict(self.h, C.byref(vs), C.byref(vt), _ptr(mean), _ptr(std)))
        return mean, std

    def params(self, theta_in=None, with_grad=False):
        n = C.c_int64(0)
        _check(load().pf_proposal_params(self.h, None, None, None, C.byref(n)))
        theta = np.zeros(n.value, np.float32)
        grad = np.zeros(n.value, np.float32) if with_grad else None
        tin = None if theta_in is None else _np(theta_in, np.float32)
        _check(load().pf_proposal_params(self.h, _ptr(theta), _ptr(grad), _ptr(tin), C.byref(n)))
        return (theta, grad) if with_grad else theta

    def forward(self, x, out, hidden=None):
        _check(load().pf_proposal_forward(self.h, _ptr(x), int(x.shape[0]), _ptr(out), _ptr(hidden)))

    def backward(self, y):
        loss = C.c_float(0.0)
        _check(load().pf_proposal_backward(self.h, _ptr(y), int(y.shape[0]), C.byref(loss)))
        return float(loss.value)

    def synth(self, x, y, seed, step, vol_dims=(224, 208, 176), rot_limit=0.5235988, trans_limit=25.0):
        dims = _np(vol_dims, np.int32)
        _check(load().pf_proposal_synth(self.h, int(x.shape[0]), int(seed), int(step), _ptr(dims),
                                        float(rot_limit), float(trans_limit), _ptr(x), _ptr(y)))

    def input(self, src, tgt, x, src_origin=(0, 0, 0), tgt_origin=(0, 0, 0), src_spacing=(1, 1, 1),
              tgt_spacing=(1, 1, 1)):
        vs, vt = make_volume(src, src_origin, spacing=src_spacing), make_volume(tgt, tgt_origin, spacing=tgt_spacing)
        _check(load().pf_proposal_input(self.h, C.byref(vs), C.byref(vt), _ptr(x)))

    def tensor(self, which, batch):
        """Host copy of a device tensor of the last pass (pf_proposal_tensor):
        0..3 conv outputs a_l, 4..7 pre-activation gradients d_l (bf16 bit
        patterns, uint16), 8 h, 9 out, 10 dh, 11 dout (float32)."""
        if 0 <= which < 8:
            D = 64 >> ((which & 3) + 1)
            out = np.zeros((batch, D, D, D, 32), np.uint16)
        elif which in (8, 10):
            out = np.zeros((batch, 128), np.float32)
        else:
            out = np.zeros((batch, 12), np.float32)
        _check(load().pf_proposal_tensor(self.h, int(which), int(batch), _ptr(out)))
        return out

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().pf_proposal_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pf_debug_alloc_limit(nbytes):
    """Cap the device bytes a context may allocate (0 = no cap); test fault injection."""
    _check(load().pf_debug_alloc_limit(int(nbytes)))


def nn_wait_selftest(stream=None):
    """Run the bounded-wait self-test kernel (sets the nn_status flag)."""
    _check(load().pf_nn_wait_selftest(_stream_handle(stream)))
