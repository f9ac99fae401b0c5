"""Spawned processes running the oracle's image measurement on chunks of
matrices (test infrastructure only: the full-size parity checks re-measure
dozens of particles of a 224x208x176 pair, ~0.1 s of single-core oracle time
per particle).  The pool is started with `spawn`, so it is safe after the
test process has initialised CUDA."""
import multiprocessing as mp
import os

import numpy as np

_VOL = {}


def _init(src, tgt):
    import oracle
    oracle.build()
    _VOL["src"], _VOL["tgt"] = src, tgt


def _image(task):
    import oracle
    mats, a = task
    return (oracle.measure_image(_VOL["src"], _VOL["tgt"], mats, a),
            oracle.ncc2_f64(_VOL["src"], _VOL["tgt"], mats, a))


def measure_image_parallel(src, tgt, mats, a, procs=None):
    """(moments [M,7], fp64 NCC^2 [M]) of the oracle for each matrix."""
    mats = np.ascontiguousarray(np.atleast_2d(mats), np.float32)
    procs = max(1, min(len(mats), procs or (os.cpu_count() or 1)))
    chunks = [c for c in np.array_split(np.arange(len(mats)), procs) if len(c)]
    with mp.get_context("spawn").Pool(len(chunks), initializer=_init, initargs=(src, tgt)) as pool:
        res = pool.map(_image, [(mats[c], a) for c in chunks])
    return np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res])
