"""The C-ABI library builds, loads and exports every function that
include/*.h declares; argument validation works without a GPU (no compute
call is made here)."""
import ctypes as C
import glob
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def pk():
    import paper_2504_19930_gb300 as pk
    pk.build()
    pk.load()
    return pk


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, re.M):
            name = m.group(1)
            if name not in ("defined", "sizeof"):
                names.add(name)
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("pf_register_init", "pf_step", "pf_estimate", "warp_sequence", "pf_register_destroy",
                 "pf_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(pk):
    lib = C.CDLL(pk.library_path())
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_config_default(pk):
    cfg = pk.pf_config_default()
    assert cfg.mode == pk.PF_MASK_DICE and cfg.n_particles == 256 and cfg.gamma_log2 == 5
    assert abs(cfg.rot_limit[0] - np.deg2rad(15)) < 1e-6 and cfg.trans_limit[2] == 8.0
    assert cfg.sigma0_frac == 0.25 and abs(cfg.sigma_decay - 0.8) < 1e-7


def _init_rc(pk, cfg, vols):
    lib = pk.load()
    ctx = C.c_void_p(123)
    ref = lambda v: C.byref(v) if v is not None else None  # noqa: E731
    rc = lib.pf_register_init(C.byref(ctx), *[ref(v) for v in vols], C.byref(cfg), None)
    return rc, ctx.value


@pytest.mark.parametrize("field,value", [
    ("n_particles", 0), ("n_particles", 65537), ("mode", 7), ("gamma_log2", 11),
    ("sigma0_frac", 0.0), ("sigma_decay", 1.5), ("min_overlap_frac", -0.1), ("autotune", 2)])
def test_invalid_config_is_rejected(pk, field, value):
    cfg = pk.make_config("mask_dice")
    setattr(cfg, field, value)
    m = np.zeros((4, 4, 4), np.uint8)
    v = pk.make_volume(m)
    rc, ctx = _init_rc(pk, cfg, [None, None, v, v])
    assert rc == -1 and ctx is None
    assert pk.pf_last_error()


def test_invalid_limits_and_volumes_are_rejected(pk):
    m = np.zeros((4, 4, 4), np.uint8)
    v = pk.make_volume(m)
    for rot in (0.0, 1.6, float("nan")):
        cfg = pk.make_config("mask_dice", rot_limit=rot)
        assert _init_rc(pk, cfg, [None, None, v, v])[0] == -1
    cfg = pk.make_config("mask_dice")
    assert _init_rc(pk, cfg, [None, None, None, v])[0] == -1          # missing mask
    small = pk.make_volume(np.zeros((1, 4, 4), np.uint8))
    assert _init_rc(pk, cfg, [None, None, small, v])[0] == -1         # dims < 2
    cfg = pk.make_config("image_ncc")
    assert _init_rc(pk, cfg, [None, None, v, v])[0] == -1             # images missing
    cfg = pk.make_config("combined")
    other = pk.make_volume(np.zeros((4, 4, 5), np.uint8))
    assert _init_rc(pk, cfg, [v, v, other, v])[0] == -1               # mask off its image grid
    assert "combined" in pk.pf_last_error()


def test_null_arguments_are_rejected(pk):
    lib = pk.load()
    assert lib.pf_step(None, 1) == -1
    assert lib.pf_estimate(None, None, None) == -1
    assert lib.pf_register_destroy(None) == 0
    assert lib.warp_sequence(None, 1, None, None, None, None, None, None, None, None, 1, None) == -1
    assert lib.pf_measure_matrices(None, None, 1, None, None) == -1
    assert lib.pf_step_measure(None, 0, 1) == -1 and lib.pf_step_update(None) == -1
    assert lib.pf_moments_device(None, None, None) == -1


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    import paper_2504_19930_gb300 as pk
    monkeypatch.setattr(pk, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pk, "_lib", None)
    with pytest.raises(RuntimeError, match="missing.so not found at"):
        pk.load()


def test_trace_without_masks_is_rejected(pk):
    v = pk.make_volume(np.zeros((4, 4, 4), np.uint8))
    cfg = pk.make_config("image_ncc", trace_estimate=True)
    rc, ctx = _init_rc(pk, cfg, [v, v, None, None])
    assert rc == -1 and ctx is None and "trace_estimate" in pk.pf_last_error()


def test_batch_arguments_are_validated(pk):
    lib = pk.load()
    out = C.c_void_p(7)
    assert lib.pf_batch_create(C.byref(out), None, 0, None) == -1 and out.value is None
    assert lib.pf_batch_step(None, 1) == -1 and lib.pf_batch_run(None) == -1
    assert lib.pf_batch_destroy(None) == 0


def test_volume_and_config_marshalling(pk):
    # (Z, Y, X) arrays become pf_volume dims {X, Y, Z}; origin and spacing are
    # passed through per axis; malformed arrays are refused before any C call
    vol = np.zeros((5, 6, 7), np.uint8)
    v = pk.make_volume(vol, origin=(1.5, -2.0, 3.0), spacing=(0.8, 1.0, 1.2))
    assert list(v.dims) == [7, 6, 5] and v.is_device == 0 and v.data == vol.ctypes.data
    assert list(v.origin) == [1.5, -2.0, 3.0]
    np.testing.assert_allclose(list(v.spacing), [0.8, 1.0, 1.2], rtol=1e-7)
    assert list(pk.make_volume(vol, spacing=2.0).spacing) == [2.0, 2.0, 2.0]
    assert pk.make_volume(None) is None
    for bad in (np.zeros((5, 6, 7), np.float32), np.zeros((5, 6), np.uint8),
                np.zeros((7, 6, 5), np.uint8).transpose(2, 1, 0)):
        with pytest.raises(ValueError):
            pk.make_volume(bad)
    cfg = pk.make_config("combined", n_particles=100, rot_limit=(0.1, 0.2, 0.3), trans_limit=4.0,
                         seed=2**40 + 3, trace_estimate=True, estimator="quaternion", autotune=True)
    assert cfg.mode == pk.PF_COMBINED and cfg.n_particles == 100 and cfg.seed == 2**40 + 3
    np.testing.assert_allclose(list(cfg.rot_limit), [0.1, 0.2, 0.3], rtol=1e-7)
    assert list(cfg.trans_limit) == [4.0, 4.0, 4.0]
    assert (cfg.trace_estimate, cfg.estimator, cfg.autotune) == (1, 1, 1)
