"""The device code's arithmetic, checked on the CPU against the oracle.

The sources are the product's own (headers included, kernel functions
copied verbatim out of the .cu files), compiled for the host through
tests/host_shim, which maps each CUDA intrinsic to the IEEE operation it
names; the package never builds or loads any of this.

1. The fp64 Taylor chain of the pose -> matrix step (Eq. 3) divides every
   term by a constant; the device takes each quotient from a stored
   reciprocal and one FMA correction (Markstein, 1990) for fp32 angles with
   2^-32 <= |x| <= 64, and from the IEEE division elsewhere.  The stored
   reciprocals are pinned to their definition and every fp32 angle of that
   range is walked through both chains, so the shortcut is the correctly
   rounded quotient on every input the kernels can receive.
2. The measurement kernel replaces conversions by fp32 adds: floors as the
   bits of 2^23 + q rounded down, the 15-bit fixed-point sample as the bits
   of s + 256, bytes as floats with the bits 2^23 + b.  Each is walked over
   every fp32 input of its range against the plain operation the oracle
   uses (floorf, lrintf(32768 s), (float)b).
3. The device headers' scalar arithmetic (sin/cos chain, pose -> matrix
   with spacings, Philox, the four scores from the integer moments and the
   quantised weights) compiled for the host through tests/host_shim (each
   intrinsic mapped to the IEEE operation it names) equals the oracle bit for
   bit on 10^5 angles, 5000 random poses and grids, 20000 random moment
   vectors in every mode and 11 weight exponents, far more than the GPU
   tests sample.  (A stored reciprocal off by one unit in the last place is
   mostly absorbed by the correction step, which is why the literals are
   pinned on their own.)
4. The measurement kernel's row set-up -- the conservative x-range of a
   target row and its exact inside interval (the functions copied verbatim
   out of measure.cu) -- equals, row by row, the voxels the oracle samples
   inside the source, for 800 random poses and grids in both the
   nearest-neighbour and trilinear bounds; six planted mistakes in a copy of
   it are each caught.
5. The sequence warp's per-voxel code (sample_at / sample_frame copied
   verbatim out of warp.cu), driven as the warp kernel drives it, equals the
   oracle's warp voxel for voxel on 300 random images, poses and grids, both
   interpolations, with and without voxel spacing.
6. The measurement kernel's per-voxel code (eval_pair with the helpers and
   the row set-up, copied verbatim out of measure.cu, the packed fp32 pairs
   in their scalar form), driven over each row's inside interval, gives the
   oracle's moments and counts bit for bit in the image, mask and combined
   forms, with the fp32 and the integer quad index; ten planted mistakes in
   a copy of it are each caught.
7. Kernels with no shared memory, barrier or shuffle -- the initial clouds
   (k_init, k_seed_gaussian) and the quad packing (k_pack_quads) -- run as a
   host loop over their threads equal the oracle's initial clouds and the
   quad layout written out in numpy.  The set-up kernels (mask bits, the
   binarised mask, the voxel count), the pose -> matrix and single-score
   exports and the estimate's traced Dice, under the block emulation, equal
   their numpy definitions and the oracle; five planted mistakes are each
   caught.
8. The measurement kernel's whole warp routine (measure_item: the row
   set-up, the sweep of 32 rows' intervals in 64-voxel passes with the
   row-crossing passes, the per-voxel code, the warp reduction and the
   atomics with S2's carry) and the warp's x-product table, copied verbatim
   out of measure.cu, run under a lockstep emulation of one warp
   (tests/host_shim/warp_emulation.h) and give the oracle's moments in every
   form the kernel instantiates; six planted mistakes in the sweep are each
   caught.
9. The prediction kernel k_predict (perturbation, the shared sin/cos chain,
   pose -> matrix, 8 lanes per particle exchanging by shuffles), copied
   verbatim out of filter.cu and run warp by warp under the same emulation,
   gives the oracle's perturbed cloud and matrices (and, for the quaternion
   estimator, each pose's quaternion) for random cloud sizes, iterations,
   limits (clamping included), seeds and grids; four planted mistakes in it
   are each caught.
10. The update step -- k_update_small (one block of 1024 threads) and the
   three-kernel form k_score / k_weights / k_finalise -- copied verbatim out
   of filter.cu and run under the block emulation (barriers, shared memory,
   warp scans), gives the oracle's scores, weights, scan, resampled indices
   and cloud bit for bit and its estimate and ESS within their summation
   rounding (the quaternion average's rotation within 1e-9), for 1 to 13000
   particles; six planted mistakes are each caught.
11. The measurement kernel k_measure itself, block by block under the
   emulation -- per-warp and per-block (CTAB) x-product tables, mask bits in
   shared memory or from the global array, both quad indexes, 1 to 8 items
   per warp, blocks whose items span two particles -- gives the oracle's
   moments in every combination its launch selects.
12. The sequence-warp kernel k_warp itself, block by block under the
   emulation (matrix built in shared memory, grid-stride rows, four frames
   at a time and the remainder, both index widths), equals the oracle's warp
   of every frame.
13. One batch iteration -- k_predict_batch, k_measure_batch over the image,
   mask and combined lists, k_score_batch, k_weights_batch, k_finalise_batch
   -- under the emulation gives every member of a mixed batch the oracle's
   single-registration steps (cloud, matrices, moments, scores, weights,
   indices, resampled cloud), with and without the per-warp tables.
14. Whole trajectories: k_predict, k_measure and the update kernels run
   iteration after iteration from the initial cloud, as the iteration graph
   runs them, and every iteration equals the oracle registration's trace in
   all four modes, on both sides of the one-block update, with unit and
   anisotropic voxel spacings.
15. The debug build's bounds checks (every gather index against its buffer
   before the load) over the measurement's and the warp kernel's runs: no
   index outside.
16. The proposal network's CUDA-core kernels (weight transpose, fully
   connected layers and their gradients, bias gradient, Gaussian loss, Adam,
   bf16 copies, uniform initialisation, the input's box average), under the
   block emulation, equal the oracle's fp64 definitions within the fp32
   accumulation bound (bit for bit where the result is a copy or a rounding);
   six planted mistakes are each caught.
17. The learned proposal's training labels (k_synth_params, run on the
   host) are poses in the filter's convention: each synthetic pair's map
   from target voxel to source point equals the oracle's pose -> matrix of
   its label; four planted mistakes (rotation order, axis, centre, sign)
   are each caught.  The pairs' network input (k_synth_views) is their
   full-resolution views box-averaged as the oracle box-averages a real
   volume; three planted mistakes are each caught.
18. The tensor-core path's operand layout (umma.cuh's tile_offset) is a
   bijection of 8 x 8 core matrices whose strides are the LBO / SBO the
   GEMM puts in its descriptors, and the descriptors' fields decode as the
   PTX ISA's tcgen05 formats.
"""
import os
import platform
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2504_19930_gb300", "csrc", "device.cuh")
CHECK_C = os.path.join(ROOT, "tests", "taylor_division_check.c")
IDENT_C = os.path.join(ROOT, "tests", "device_identities_check.c")


def _literals(name):
    text = open(HEADER).read()
    m = re.search(r"#define " + name + r" \{(.*?)\}", text, re.S)
    assert m, name
    return [float.fromhex(v.strip()) if v.strip().startswith("0x") else float(v)
            for v in m.group(1).replace("\\", " ").split(",")]


@pytest.mark.parametrize("name, divisor", [
    ("PF_TAYLOR_RECIP_SIN", lambda k: (2 * k) * (2 * k + 1)),
    ("PF_TAYLOR_RECIP_COS", lambda k: (2 * k - 1) * (2 * k)),
])
def test_reciprocals_are_the_rounded_quotients(name, divisor):
    vals = _literals(name)
    assert len(vals) == 14
    for k in range(1, 14):
        assert vals[k] == 1.0 / divisor(k), (name, k)   # Python's division is IEEE round-to-nearest


def _flags():
    flags = ["-O2", "-ffp-contract=off"]
    if platform.machine() in ("x86_64", "AMD64"):
        try:
            if " fma " in open("/proc/cpuinfo").read().replace("\n", " "):
                flags.append("-mfma")   # the hardware FMA; glibc's software fma gives the same bits, slowly
        except OSError:
            pass
    return flags


def _run_parts(src, exe, extra=()):
    """Compile a checker and run it split over the host's cores; (checked, mismatches)."""
    subprocess.run(["gcc", *_flags(), *extra, "-o", exe, src, "-lm"], check=True)
    nparts = max(1, min(os.cpu_count() or 1, 32))
    procs = [subprocess.Popen([exe, str(p), str(nparts)], stdout=subprocess.PIPE, text=True)
             for p in range(nparts)]
    checked = bad = 0
    for pr in procs:
        out, _ = pr.communicate(timeout=1800)
        assert pr.returncode == 0
        m = re.match(r"checked (\d+) mismatches (\d+)", out)
        checked += int(m.group(1))
        bad += int(m.group(2))
    return checked, bad


def test_division_shortcut_is_exact_for_every_fp32_angle(tmp_path):
    checked, bad = _run_parts(CHECK_C, str(tmp_path / "taylor_division_check"))
    n_angles = 0x42800000 - 0x2F800000 + 1          # fp32 bit patterns of 2^-32 .. 64
    assert checked == 26 * n_angles                 # 13 divisions in each of the two chains
    assert bad == 0


def test_conversion_shortcuts_are_exact_over_their_ranges(tmp_path):
    checked, bad = _run_parts(IDENT_C, str(tmp_path / "device_identities_check"), ("-frounding-math",))
    n_floor = 0x4B000000                            # fp32 bit patterns of [0, 2^23)
    n_fixed = 0x437F0000 + 1                        # ... of [0, 255]
    assert checked == n_floor + n_fixed + 256 * 256
    assert bad == 0


# ------------------------------------------------- device pose math on the host

DM_CPP = os.path.join(ROOT, "tests", "device_math_host.cpp")
SHIM = os.path.join(ROOT, "tests", "host_shim")


@pytest.fixture(scope="module")
def dm(tmp_path_factory):
    """The device header's pose arithmetic built for the CPU (the intrinsics
    mapped to the IEEE operations they name), for wide sweeps against the
    oracle; the GPU tests check the same functions on the device itself."""
    import ctypes as C
    so = str(tmp_path_factory.mktemp("dm") / "libdm.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I" + SHIM,
                    DM_CPP, "-o", so], check=True)
    L = C.CDLL(so)
    L.dm_sincos.restype = C.c_double
    L.dm_sincos.argtypes = [C.c_float, C.c_int]
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
    L.dm_pose_matrix.argtypes = [f32p, i32p, f32p, f32p, f32p, f32p, f32p]
    L.dm_philox.argtypes = [u32p, u32p, u32p]
    u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
    L.dm_score.restype = C.c_double
    L.dm_score.argtypes = [C.c_int, u64p, C.c_uint64, C.c_uint64]
    L.dm_weight.restype = C.c_uint64
    L.dm_weight.argtypes = [C.c_double, C.c_double, C.c_int]
    return L


def test_device_sincos_equals_the_oracle(dm, orc):
    rng = np.random.default_rng(21)
    xs = np.concatenate([rng.uniform(-np.pi / 2, np.pi / 2, 100000),
                         np.float32(2.0) ** -rng.uniform(20, 60, 2000) * rng.choice([-1, 1], 2000),
                         [0.0, -0.0, np.pi / 2, -np.pi / 2, 2.0**-32, 2.0**-33, 64.0, 70.0, 3.0]]).astype(np.float32)
    for x in xs:
        assert dm.dm_sincos(x, 0) == orc.sin(float(x)), x
        assert dm.dm_sincos(x, 1) == orc.cos(float(x)), x


def test_device_pose_matrix_equals_the_oracle(dm, orc):
    rng = np.random.default_rng(22)
    for i in range(5000):
        pose = np.concatenate([rng.uniform(-1.57, 1.57, 3), rng.uniform(-60, 60, 3)]).astype(np.float32)
        sd = rng.integers(2, 400, 3).astype(np.int32)
        so = rng.uniform(-50, 50, 3).astype(np.float32)
        to = rng.uniform(-50, 50, 3).astype(np.float32)
        unit = i % 3 == 0
        ss = np.ones(3, np.float32) if unit else rng.uniform(0.2, 3.0, 3).astype(np.float32)
        ts = np.ones(3, np.float32) if unit else rng.uniform(0.2, 3.0, 3).astype(np.float32)
        M = np.zeros(12, np.float32)
        dm.dm_pose_matrix(pose, sd, so, ss, to, ts, M)
        want, _ = orc.pose_matrix(pose, sd, so, to, ss, ts)
        assert np.array_equal(M, want), (i, M - want)


def test_device_philox_equals_the_oracle(dm, orc):
    rng = np.random.default_rng(23)
    for _ in range(2000):
        ctr = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, 2, dtype=np.uint64).astype(np.uint32)
        out = np.zeros(4, np.uint32)
        dm.dm_philox(ctr, key, out)
        assert np.array_equal(out, orc.philox(ctr, key))


def _random_moments(rng):
    """A moment vector [n S1 S2lo S2hi ST T1 T2 0 | n_nn A B C] with the
    ranges a measurement can produce (15-bit fixed-point samples < 2^23,
    uint8 targets), variances sometimes zero."""
    n = int(rng.integers(0, 1 << 26))
    s1 = int(rng.integers(0, n * ((1 << 23) - 1) + 1)) if n else 0
    s2 = (s1 * s1 + n - 1) // n if n else 0
    if rng.random() < 0.9 and n:
        s2 += int(rng.integers(0, 1 << 62)) * int(rng.integers(1, 1 << 16))
    st = int(rng.integers(0, n * ((1 << 23) - 1) * 255 + 1)) if n else 0
    t1 = int(rng.integers(0, 255 * n + 1)) if n else 0
    t2 = (t1 * t1 + n - 1) // n if n else 0
    if rng.random() < 0.9 and n:
        t2 += int(rng.integers(0, 65025 * n // 4 + 1))
    nn = int(rng.integers(0, 1 << 26))
    a, b = int(rng.integers(0, nn + 1)), int(rng.integers(0, nn + 1))
    c = int(rng.integers(0, min(a, b) + 1))
    mom = [n, s1, s2 & (2**64 - 1), s2 >> 64, st, t1, t2, 0, nn, a, b, c]
    return np.array(mom, np.uint64), b + int(rng.integers(0, 1 << 20))


def test_device_scores_equal_the_oracle(dm, orc):
    rng = np.random.default_rng(24)
    for i in range(20000):
        mom, b_full = _random_moments(rng)
        n_min = int(rng.choice([0, int(mom[0]), int(mom[0]) + 1, int(mom[8]), 1 << 20]))
        for mode in range(4):
            got = dm.dm_score(mode, mom, b_full, n_min)
            want = orc.score(mode, mom, b_full, n_min)
            assert got == want or (np.isnan(got) and np.isnan(want)), (i, mode, mom, got, want)


def test_device_weights_equal_the_oracle(dm, orc):
    rng = np.random.default_rng(25)
    for g in range(11):
        s = rng.uniform(0, 1, 2000)
        s[:50] = 0.0
        s[50:60] = s.max()
        s[60:70] = rng.uniform(0, 1e-300, 10)
        want = orc.weights(s, g)
        smax = float(s.max())
        got = np.array([dm.dm_weight(float(v), smax, g) for v in s], np.uint64)
        assert np.array_equal(got, want), g
    assert dm.dm_weight(0.5, 0.0, 5) == 0



# ---------------------------------------- the measurement's row set-up on the host

MEASURE_CU = os.path.join(ROOT, "paper_2504_19930_gb300", "csrc", "measure.cu")
RI_CPP = os.path.join(ROOT, "tests", "row_interval_host.cpp")
RI_BEGIN = "// Coordinate q_d(x) of target voxel x of a row"
RI_END = "// One work item = (particle p, 32 target rows)"


@pytest.fixture(scope="module")
def ri(tmp_path_factory):
    """The kernel's row set-up (row_interval, and coord1 / axis_conds /
    exact_interval copied verbatim from measure.cu) built for the CPU."""
    import ctypes as C
    d = tmp_path_factory.mktemp("ri")
    src = open(MEASURE_CU).read()
    assert src.count(RI_BEGIN) == 1 and src.count(RI_END) == 1
    (d / "measure_row_interval.inc").write_text(src[src.index(RI_BEGIN):src.index(RI_END)])
    so = str(d / "libri.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I" + SHIM,
                    "-I" + str(d), RI_CPP, "-o", so], check=True)
    L = C.CDLL(so)
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    L.dm_row_intervals.argtypes = [f32p, f32p, i32p, i32p, C.c_int, i32p, i32p]
    return L


def test_row_intervals_equal_the_oracles_inside_sets(ri, orc):
    # every target row's visited interval [xl, xr] is exactly the set of
    # voxels the oracle samples inside the source (nearest-neighbour or
    # trilinear bounds): the oracle warps a source of 255s, which marks them
    rng = np.random.default_rng(26)
    half_pi = np.float32(np.pi / 2)
    for i in range(800):
        sd = rng.integers(2, 40, 3).astype(np.int32)
        td = rng.integers(2, 48, 3).astype(np.int32)
        so = rng.uniform(-15, 15, 3).astype(np.float32)
        to = rng.uniform(-15, 15, 3).astype(np.float32)
        if i % 5 == 0:      # no rotation: r_10 = r_20 = 0, q_y and q_z constant along a row
            ang = np.zeros(3)
        elif i % 5 == 1:    # quarter turns
            ang = rng.choice([-half_pi, 0.0, half_pi], 3)
        else:
            ang = rng.uniform(-1.57, 1.57, 3)
        pose = np.concatenate([ang, rng.uniform(-20, 20, 3)]).astype(np.float32)
        if i % 5 == 0 and i % 2 == 0:
            # half-integer origins and translations without rotation put
            # samples exactly on the bounds (q = D - 1, q + 0.5 = D)
            so, to = np.round(so * 2) / 2, np.round(to * 2) / 2
            pose[3:] = np.round(pose[3:] * 2) / 2
        M, a = orc.pose_matrix(pose, sd, so, to)
        ones = np.full((sd[2], sd[1], sd[0]), 255, np.uint8)
        X = int(td[0])
        for tri in (0, 1):
            inside = orc.warp_matrix(ones, tuple(int(v) for v in td), M, a, tri).reshape(-1, X) == 255
            xl = np.zeros(inside.shape[0], np.int32)
            xr = np.zeros(inside.shape[0], np.int32)
            ri.dm_row_intervals(M, a, sd, td, tri, xl, xr)
            cnt = inside.sum(1)
            first = np.argmax(inside, 1)
            last = X - 1 - np.argmax(inside[:, ::-1], 1)
            has = cnt > 0
            assert np.all(cnt[has] == last[has] - first[has] + 1), (i, tri)     # one interval per row
            assert np.array_equal(xl[has], first[has]) and np.array_equal(xr[has], last[has]), (i, tri)
            assert np.all(xr[~has] < xl[~has]), (i, tri)


# planted mistakes in a copy of the kernel's row set-up, each of which the
# comparison above must catch (it is only as good as the rows it samples)
RI_MUTANTS = [
    ("trilinear upper bound strict", "upper = q <= D - 1.0f;", "upper = q < D - 1.0f;"),
    ("nearest-neighbour upper bound inclusive", "upper = h < D;", "upper = h <= D;"),
    ("two probes counted as four", "if (++cnt == 4) break;\n    }\n    if (cnt == 4 && l < xe)",
     "if (++cnt == 2) break;\n    }\n    if (cnt == 4 && l < xe)"),
    ("binary search too short", "for (int step = 2048; step > 0; step >>= 1)\n            if (pl + step",
     "for (int step = 2; step > 0; step >>= 1)\n            if (pl + step"),
    ("constant axes ignored", "xr = constant_ok ? r : xl - 1;", "xr = r;"),
    ("wrong bound for a decreasing axis", "ok &= r0[d] > 0.0f ? up : (r0[d] < 0.0f ? lo : true);",
     "ok &= r0[d] > 0.0f ? up : (r0[d] < 0.0f ? up : true);"),
]


def test_row_interval_comparison_catches_planted_mistakes(orc, tmp_path):
    import ctypes as C
    src = open(MEASURE_CU).read()
    inc = src[src.index(RI_BEGIN):src.index(RI_END)]
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    for k, (name, text, planted) in enumerate(RI_MUTANTS):
        assert inc.count(text) == 1, name
        d = tmp_path / f"m{k}"
        d.mkdir()
        (d / "measure_row_interval.inc").write_text(inc.replace(text, planted))
        so = str(d / "libri.so")
        subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I" + SHIM,
                        "-I" + str(d), RI_CPP, "-o", so], check=True)
        L = C.CDLL(so)
        L.dm_row_intervals.argtypes = [f32p, f32p, i32p, i32p, C.c_int, i32p, i32p]
        with pytest.raises(AssertionError):
            test_row_intervals_equal_the_oracles_inside_sets(L, orc)


# --------------------------------------------- the sequence warp's voxels on the host

WARP_CU = os.path.join(ROOT, "paper_2504_19930_gb300", "csrc", "warp.cu")
WH_CPP = os.path.join(ROOT, "tests", "warp_host.cpp")
WH_BEGIN = "struct WarpArgs {"
WH_END = "// One target row per warp at a time"


def test_warp_voxels_equal_the_oracle(orc, tmp_path):
    # the warp kernel's per-voxel code (sample_at / sample_frame copied
    # verbatim out of warp.cu) driven as k_warp drives it, against the
    # oracle's warp, both interpolations, with and without voxel spacing
    import ctypes as C
    import pfsynth
    src = open(WARP_CU).read()
    assert src.count(WH_BEGIN) == 1 and src.count(WH_END) == 1
    (tmp_path / "warp_sample.inc").write_text(src[src.index(WH_BEGIN):src.index(WH_END)])
    so_path = str(tmp_path / "libwh.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I" + SHIM,
                    "-I" + str(tmp_path), WH_CPP, "-o", so_path], check=True)
    L = C.CDLL(so_path)
    u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    L.dm_warp.argtypes = [u8p, i32p, f32p, f32p, u8p, i32p, f32p, f32p, f32p, f32p, C.c_int]
    rng = np.random.default_rng(27)
    for i in range(300):
        sd = rng.integers(2, 30, 3).astype(np.int32)
        td = rng.integers(2, 30, 3).astype(np.int32)
        img = pfsynth.random_image(int(rng.integers(0, 1 << 30)), tuple(int(v) for v in sd))
        so = rng.uniform(-10, 10, 3).astype(np.float32)
        to = rng.uniform(-10, 10, 3).astype(np.float32)
        unit = i % 2 == 0
        ss = np.ones(3, np.float32) if unit else rng.uniform(0.3, 2.5, 3).astype(np.float32)
        ts = np.ones(3, np.float32) if unit else rng.uniform(0.3, 2.5, 3).astype(np.float32)
        pose = np.concatenate([rng.uniform(-1.5, 1.5, 3), rng.uniform(-12, 12, 3)]).astype(np.float32)
        if i % 10 == 0:
            pose[:3] = 0.0
        _, a = orc.pose_matrix(pose, sd, so, to, ss, ts)
        for interp in (0, 1):
            out = np.zeros((td[2], td[1], td[0]), np.uint8)
            L.dm_warp(np.ascontiguousarray(img), sd, so, ss, out, td, to, ts, a, pose, interp)
            want = orc.warp(img, so, tuple(int(v) for v in td), to, pose, interp, ss, ts)
            assert np.array_equal(out, want), (i, interp, int((out != want).sum()))


# ------------------------------------ the measurement's per-voxel code on the host

MH_CPP = os.path.join(ROOT, "tests", "measure_host.cpp")
MV_BEGIN = "#if PF_DEBUG\n__device__ unsigned long long g_dbg_hits;"


def _build_measure_host(src_text, d):
    import ctypes as C
    assert src_text.count(MV_BEGIN) == 1 and src_text.count(RI_END) == 1
    (d / "measure_voxel.inc").write_text(src_text[src_text.index(MV_BEGIN):src_text.index(RI_END)])
    so = str(d / "libmh.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-frounding-math", "-fPIC", "-shared",
                    "-I" + SHIM, "-I" + str(d), MH_CPP, "-o", so], check=True)
    L = C.CDLL(so)
    u8p = C.c_void_p
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
    L.dm_measure.argtypes = [C.c_int, C.c_int, C.c_int, u8p, u8p, i32p, u8p, u8p, i32p, f32p, C.c_int, f32p, u64p]
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data


def _measure_cases(orc, seed, count):
    import pfsynth
    rng = np.random.default_rng(seed)
    for i in range(count):
        sd = tuple(int(v) for v in rng.integers(2, 26, 3))
        td = tuple(int(v) for v in rng.integers(2, 28, 3))
        src = pfsynth.random_image(int(rng.integers(0, 1 << 30)), sd)
        tgt = pfsynth.random_image(int(rng.integers(0, 1 << 30)), td)
        smask = (rng.random((sd[2], sd[1], sd[0])) < 0.5).astype(np.uint8)
        tmask = (rng.random((td[2], td[1], td[0])) < 0.5).astype(np.uint8)
        so = rng.uniform(-8, 8, 3).astype(np.float32)
        to = rng.uniform(-8, 8, 3).astype(np.float32)
        P = 6
        poses = np.concatenate([rng.uniform(-1.5, 1.5, (3, P)), rng.uniform(-10, 10, (3, P))]).astype(np.float32)
        if i % 4 == 0:
            poses[:3, :2] = 0.0
            so, to = np.round(so * 2) / 2, np.round(to * 2) / 2
            poses[3:, :2] = np.round(poses[3:, :2] * 4) / 4
        mats, a = orc.pose_matrices(poses, sd, so, to)
        yield sd, td, src, tgt, smask, tmask, np.ascontiguousarray(mats, np.float32), a


def _check_measure(L, orc, seed=28, count=120):
    for sd, td, src, tgt, smask, tmask, mats, a in _measure_cases(orc, seed, count):
        P = mats.shape[0]
        sdv, tdv = np.array(sd, np.int32), np.array(td, np.int32)
        want_img = orc.measure_image(src, tgt, mats, a)
        want_msk = orc.measure_mask(smask, tmask, mats, a)
        for img, msk, int_index in ((1, 0, 0), (1, 0, 1), (0, 1, 0), (1, 1, 0), (1, 1, 1)):
            got = np.zeros((P, 12), np.uint64)
            L.dm_measure(img, msk, int_index, _ptr(src) if img else None, _ptr(smask) if msk else None, sdv,
                         _ptr(tgt) if img else None, _ptr(tmask) if msk else None, tdv, mats, P, a, got)
            if img:
                assert np.array_equal(got[:, 0:7], want_img), (sd, td, img, msk, int_index)
            if msk:
                assert np.array_equal(got[:, 8:12], want_msk), (sd, td, img, msk, int_index)


def test_measurement_voxels_equal_the_oracle(orc, tmp_path):
    # eval_pair and the row set-up (copied verbatim out of measure.cu) with
    # the scalar forms of the packed fp32 pairs: per-matrix moments and counts
    # equal the oracle's in the image, mask and combined forms, on random
    # volumes, grids and poses (with samples on the bounds), with both the
    # fp32 quad index (sources up to 2^23 voxels) and the integer one
    L = _build_measure_host(open(MEASURE_CU).read(), tmp_path)
    _check_measure(L, orc)


# planted mistakes in a copy of the kernel's per-voxel code, each of which the
# comparison above must catch
MV_MUTANTS = [
    ("byte read from the wrong lane", "return __uint_as_float(__byte_perm(w, kTwo23Bits, 0x7540u | k));",
     "return __uint_as_float(__byte_perm(w, kTwo23Bits, 0x7540u | (k ^ 1u)));"),
    ("fixed point at 14 bits", "const f2 s = add2(lerp2(c0, c1, fz), splat(256.0f));",
     "const f2 s = add2(lerp2(c0, c1, fz), splat(512.0f));"),
    ("cross moment with the other voxel's target", "ia.ST += (unsigned long long)sq0 * t0;",
     "ia.ST += (unsigned long long)sq0 * t1;"),
    ("nearest neighbour without the half-voxel shift", "const f2 bxn = addrm2(add2(qx, splat(0.5f)), splat(kTwo23));",
     "const f2 bxn = addrm2(qx, splat(kTwo23));"),
    ("fp32 quad index with z for y", "const f2 w = fma2(splat(a.fdims[1]), flz, fma2(splat(a.fdims[0]), fly, bx));",
     "const f2 w = fma2(splat(a.fdims[1]), flz, fma2(splat(a.fdims[0]), flz, bx));"),
    ("y lerps with the z fraction", "const f2 c0 = lerp2(c00, c10, fy), c1 = lerp2(c01, c11, fy);",
     "const f2 c0 = lerp2(c00, c10, fz), c1 = lerp2(c01, c11, fy);"),
    ("x fraction from the y floor", "const f2 fx = sub2(qx, flx), fy = sub2(qy, fly), fz = sub2(qz, flz);",
     "const f2 fx = sub2(qx, fly), fy = sub2(qy, fly), fz = sub2(qz, flz);"),
    ("S2 sums the sample", "ia.S2 += (unsigned long long)sq0 * sq0;", "ia.S2 += (unsigned long long)sq0;"),
    ("mask intersection as a union", "ma.C += sb & tb;", "ma.C += sb | tb;"),
    ("integer quad index bias off by one row", "const uint32_t bias = 0u - kTwo23Bits * (1u + (uint32_t)SX + SXY);",
     "const uint32_t bias = 0u - kTwo23Bits * (1u + (uint32_t)SX + SXY) + (uint32_t)SX;"),
]


def test_measurement_comparison_catches_planted_mistakes(orc, tmp_path):
    src = open(MEASURE_CU).read()
    region = src[src.index(MV_BEGIN):src.index(RI_END)]
    for name, text, _ in MV_MUTANTS:
        assert region.count(text) >= 1, name
    for L in _build_all(_build_measure_host, src, MV_MUTANTS, tmp_path):
        with pytest.raises(AssertionError):
            _check_measure(L, orc, seed=29, count=12)



# ------------------------------- kernels without shared state, as host loops

FILTER_CU = os.path.join(ROOT, "paper_2504_19930_gb300", "csrc", "filter.cu")
KH_CPP = os.path.join(ROOT, "tests", "kernels_host.cpp")


def test_initial_clouds_and_quad_packing_equal_their_definitions(orc, tmp_path):
    # k_init and k_seed_gaussian (copied verbatim out of filter.cu) against
    # the oracle's initial clouds, and k_pack_quads (out of measure.cu)
    # against the quad layout written out in numpy, each kernel run as a loop
    # over its threads
    import ctypes as C
    import pfsynth
    f = open(FILTER_CU).read()
    b0, e0 = "// Initial particles (Abstract", "// Prediction for k > 0"
    assert f.count(b0) == 1 and f.count(e0) == 1
    (tmp_path / "filter_init.inc").write_text(f[f.index(b0):f.index(e0)])
    m = open(MEASURE_CU).read()
    b1 = "__global__ void k_pack_quads("
    assert m.count(b1) == 1
    i = m.index(b1)
    (tmp_path / "pack_quads.inc").write_text(m[i:m.index("}  // namespace", i)])
    so = str(tmp_path / "libkh.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I" + SHIM,
                    "-I" + str(tmp_path), KH_CPP, "-o", so], check=True)
    L = C.CDLL(so)
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
    L.dm_init.argtypes = [C.c_int, C.c_uint64, f32p, f32p]
    L.dm_seed.argtypes = [C.c_int, C.c_uint64, f32p, f32p, f32p, f32p]
    L.dm_pack_quads.argtypes = [u8p, i32p, u32p]
    rng = np.random.default_rng(30)
    for N, seed in ((1, 0), (257, 3), (4096, 2**40 + 7)):
        lim = rng.uniform(0.1, 30, 6).astype(np.float32)
        got = np.zeros((6, N), np.float32)
        L.dm_init(N, seed, lim, got)
        assert np.array_equal(got, orc.init_particles(N, seed, lim))
        mean = rng.uniform(-5, 5, 6).astype(np.float32)
        sdev = rng.uniform(0.01, 8, 6).astype(np.float32)
        L.dm_seed(N, seed, lim, mean, sdev, got)
        assert np.array_equal(got, orc.init_gaussian(N, seed, mean, sdev, lim))
    for dims in ((2, 2, 2), (7, 5, 3), (33, 17, 9)):
        S = pfsynth.random_image(int(rng.integers(0, 1 << 30)), dims)
        Q = np.zeros(S.size, np.uint32)
        L.dm_pack_quads(np.ascontiguousarray(S), np.array(dims, np.int32), Q)
        P = np.zeros((dims[2], dims[1] + 1, dims[0] + 1), np.uint32)
        P[:, :-1, :-1] = S
        want = P[:, :-1, :-1] | P[:, :-1, 1:] << 8 | P[:, 1:, :-1] << 16 | P[:, 1:, 1:] << 24
        assert np.array_equal(Q.reshape(S.shape), want), dims


SK_CPP = os.path.join(ROOT, "tests", "small_kernels_host.cpp")
SK_BEGIN, SK_END = "// Matrix of one pose by a group of 8 lanes", "__global__ void k_philox("


def _build_small(src_text, d):
    import ctypes as C
    assert src_text.count(SK_BEGIN) == 1 and src_text.count(SK_END) == 1
    (d / "small_kernels.inc").write_text(src_text[src_text.index(SK_BEGIN):src_text.index(SK_END)])
    so = str(d / "libsk.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I" + SHIM,
                    "-I" + str(d), SK_CPP, "-o", so], check=True)
    L = C.CDLL(so)
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
    u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
    L.dm_pack_bits.argtypes = [u8p, C.c_int64, u32p]
    L.dm_binarise.argtypes = [u8p, u8p, C.c_int64]
    L.dm_count_nonzero.restype = C.c_ulonglong
    L.dm_count_nonzero.argtypes = [u8p, C.c_int64]
    L.dm_pose_matrix_kernel.argtypes = [f32p, i32p, f32p, f32p, f32p, f32p]
    L.dm_score_one.restype = C.c_double
    L.dm_score_one.argtypes = [C.c_int, u64p, C.c_uint64, C.c_uint64]
    L.dm_trace.argtypes = [f64p, i32p, f32p, f32p, f32p, C.c_uint64, f32p, u64p, f64p]
    return L


def _check_small(L, orc):
    """The registration's remaining kernels: the set-up kernels against their
    plain definitions in numpy, the pose -> matrix and single-score exports
    and the estimate's traced Dice (Eq. 4) against the oracle."""
    rng = np.random.default_rng(40)
    # grid-stride loops over 3 x 64 threads and the last word's tail
    for n in (0, 1, 31, 32, 33, 191, 192, 193, 4097, 20000):
        v = (rng.integers(0, 256, n) * (rng.random(n) < 0.4)).astype(np.uint8)
        v = np.ascontiguousarray(v) if n else np.zeros(1, np.uint8)
        out = np.full(max(n, 1), 7, np.uint8)
        L.dm_binarise(v, out, n)
        assert np.array_equal(out[:n], (v[:n] != 0).astype(np.uint8)) and (n or out[0] == 7), n
        assert L.dm_count_nonzero(v, n) == int(np.count_nonzero(v[:n])), n
        words = (n + 31) // 32
        bits = np.full(max(words, 1), 0xDEADBEEF, np.uint32)
        L.dm_pack_bits(v, n, bits)
        padded = np.zeros(words * 32, bool)
        padded[:n] = v[:n] != 0
        want = (padded.reshape(-1, 32).astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(1)
        assert np.array_equal(bits[:words], want.astype(np.uint32)), n
    for i in range(300):
        pose = np.concatenate([rng.uniform(-1.57, 1.57, 3), rng.uniform(-60, 60, 3)]).astype(np.float32)
        sd = rng.integers(2, 400, 3).astype(np.int32)
        so, to = rng.uniform(-50, 50, 3).astype(np.float32), rng.uniform(-50, 50, 3).astype(np.float32)
        M = np.zeros(12, np.float32)
        L.dm_pose_matrix_kernel(pose, sd, so, to, np.zeros(3, np.float32), M)
        assert np.array_equal(M, orc.pose_matrix(pose, sd, so, to)[0]), i
    for i in range(2000):
        mom, b_full = _random_moments(rng)
        n_min = int(rng.choice([0, int(mom[0]), int(mom[8]) + 1]))
        for mode in range(4):
            got, want = L.dm_score_one(mode, mom, b_full, n_min), orc.score(mode, mom, b_full, n_min)
            assert got == want or (np.isnan(got) and np.isnan(want)), (i, mode)
    # the trace: the estimate rounded to fp32, its matrix, the whole-grid
    # counts of that matrix and their Dice with no overlap threshold
    for i in range(40):
        sd = rng.integers(4, 24, 3).astype(np.int32)
        td = rng.integers(4, 24, 3).astype(np.int32)
        so, to = rng.uniform(-5, 5, 3).astype(np.float32), rng.uniform(-5, 5, 3).astype(np.float32)
        est = np.concatenate([rng.uniform(-0.6, 0.6, 3), rng.uniform(-6, 6, 3)])
        smask = (rng.random(sd[::-1]) < 0.5).astype(np.uint8)
        tmask = (rng.random(td[::-1]) < 0.5).astype(np.uint8) * (i % 7 != 0)
        want_M, a = orc.pose_matrix(est.astype(np.float32), sd, so, to)
        counts = np.ascontiguousarray(orc.measure_mask(smask, tmask, want_M, a)[0])
        b_full = int(np.count_nonzero(tmask))
        M, dice = np.zeros(12, np.float32), np.zeros(1)
        L.dm_trace(est, sd, so, to, a, b_full, M, counts, dice)
        assert np.array_equal(M, want_M), i
        assert dice[0] == orc.dice_from_counts(counts[0], counts[1], counts[3], b_full, 0), i
        assert dice[0] == orc.score("mask_dice", np.r_[np.zeros(8, np.uint64), counts], b_full, 0), i


def test_set_up_export_and_trace_kernels_equal_their_definitions(orc, tmp_path):
    _check_small(_build_small(open(FILTER_CU).read(), tmp_path), orc)


SK_MUTANTS = [
    ("mask bits paired", "if (i < nvox && mask[i] != 0) v |= 1u << b;", "if (i < nvox && mask[i] != 0) v |= 1u << (b ^ 1);"),
    ("count above one", "c += v[i] != 0;\n#pragma", "c += v[i] > 1;\n#pragma"),
    ("trace of the current iteration", "const int k = *B.k - 1;\n    const unsigned", "const int k = *B.k;\n    const unsigned"),
    ("Dice of B instead of A", "dice_from_counts(m[0], m[1], m[3], P.b_full, 0ull)",
     "dice_from_counts(m[0], m[2], m[3], P.b_full, 0ull)"),
    ("estimate perturbed before rounding", "for (int d = 0; d < 6; ++d) pose[d] = __double2float_rn(L.est[d]);",
     "for (int d = 0; d < 6; ++d) pose[d] = __double2float_rn(L.est[d] * 1.0000001);"),
]


def test_small_kernel_comparison_catches_planted_mistakes(orc, tmp_path):
    src = open(FILTER_CU).read()
    for text in (m[1] for m in SK_MUTANTS):
        assert src.count(text) == 1, text
    for L in _build_all(_build_small, src, SK_MUTANTS, tmp_path):
        with pytest.raises(AssertionError):
            _check_small(L, orc)


NN_CU = os.path.join(ROOT, "paper_2504_19930_gb300", "csrc", "nn.cu")
NS_CPP = os.path.join(ROOT, "tests", "nn_small_host.cpp")
NS_BEGIN, NS_END = "// W [32][64][Cin] -> Wt", "// Synthetic training pairs:"
U32 = 2.0 ** -24   # unit roundoff of fp32


def _build_nn_small(src_text, d):
    import ctypes as C
    assert src_text.count(NS_BEGIN) == 1 and src_text.count(NS_END) == 1
    (d / "nn_small.inc").write_text(src_text[src_text.index(NS_BEGIN):src_text.index(NS_END)])
    so = str(d / "libnns.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I" + SHIM,
                    "-I" + str(d), NS_CPP, "-o", so], check=True)
    L = C.CDLL(so)
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
    u16p = np.ctypeslib.ndpointer(np.uint16, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    vp = C.c_void_p
    L.dm_transpose_w.argtypes = [u16p, C.c_int, u16p]
    L.dm_fc_forward.argtypes = [C.c_int, vp, vp, C.c_int, C.c_int, f32p, f32p, C.c_int, f32p, C.c_int]
    L.dm_fc_backward_input.argtypes = [C.c_int, f32p, C.c_int, C.c_int, f32p, C.c_int, vp, vp, vp, vp]
    L.dm_fc_backward_weight.argtypes = [C.c_int, f32p, C.c_int, C.c_int, vp, vp, C.c_int, f32p, f32p]
    L.dm_bias_grad.argtypes = [u16p, C.c_longlong, C.c_int, f32p]
    L.dm_nll.argtypes = [f32p, f32p, C.c_int, f32p, f32p, C.c_int]
    L.dm_adam.argtypes = [f32p, f32p, f32p, f32p, C.c_longlong, C.c_float, C.c_int]
    L.dm_to_bf16.argtypes = [f32p, C.c_longlong, u16p]
    L.dm_init_uniform.argtypes = [f32p, C.c_longlong, C.c_float, C.c_uint64, C.c_uint32]
    L.dm_downsample.argtypes = [u8p, i32p, f32p, f32p, f32p, f32p, C.c_int, C.c_int, u16p]
    return L


def _p(a):
    return None if a is None else a.ctypes.data


def _check_nn_small(L, orc, seed=41):
    """Each CUDA-core kernel of the proposal network against the oracle's
    fp64 definition (oracle/nn.py), within the fp32 accumulation bound
    (terms - 1) u sum|terms| plus, for bf16 results, the final rounding."""
    import oracle.nn as onn
    rng = np.random.default_rng(seed)
    bf = lambda a: onn.bf16_bits(onn.bf16_round(np.asarray(a, np.float32)))   # noqa: E731
    unbf = lambda b: onn.from_bf16_bits(b).astype(np.float64)                  # noqa: E731

    def close_bf16(got_bits, ref, bound, what):
        err = np.abs(unbf(got_bits) - ref)
        tol = 2.0 ** -8 * (np.abs(ref) + bound) + bound + 1e-30
        assert np.all(err <= tol), (what, float(err.max()))

    # weight transpose [32][64][Cin] -> [Cin][64][32], bit for bit
    for cin in (2, 32):
        W = rng.integers(0, 1 << 16, 32 * 64 * cin).astype(np.uint16)
        Wt = np.zeros_like(W)
        L.dm_transpose_w(W, cin, Wt)
        assert np.array_equal(Wt.reshape(cin, 64, 32), W.reshape(32, 64, cin).transpose(2, 1, 0)), cin
    # fully connected layers as the network uses them: fc1 on the bf16
    # flattened features (K = 2048, ReLU), fc2 on the fp32 hidden layer
    for in_bf16, B, K, N, relu in ((1, 3, onn.FLAT, onn.HIDDEN, 1), (0, 3, onn.HIDDEN, onn.NOUT, 0),
                                   (0, 2, 45, 7, 1)):
        x = rng.normal(0, 1, (B, K)).astype(np.float32)
        x16 = bf(x)
        xv = unbf(x16) if in_bf16 else x.astype(np.float64)
        W = rng.normal(0, 0.05, (N, K)).astype(np.float32)
        b = rng.normal(0, 0.1, N).astype(np.float32)
        out = np.zeros((B, N), np.float32)
        L.dm_fc_forward(in_bf16, _p(x), _p(x16), B, K, W, b, N, out, relu)
        pre = xv @ W.T.astype(np.float64) + b
        ref = onn.relu(pre) if relu else pre
        bound = (K + 1) * U32 * (np.abs(xv) @ np.abs(W.T).astype(np.float64) + np.abs(b))
        assert np.all(np.abs(out - ref) <= bound + 1e-30), ("fc forward", K)
        # data gradient through the ReLU of the layer's input activation
        dout = rng.normal(0, 1, (B, N)).astype(np.float32)
        act = rng.normal(0, 1, (B, K)).astype(np.float32)
        act[0, :5] = 0.0
        refd = (dout.astype(np.float64) @ W.astype(np.float64)) * (act > 0)
        boundd = N * U32 * (np.abs(dout).astype(np.float64) @ np.abs(W).astype(np.float64)) * (act > 0)
        if in_bf16:
            din = np.zeros((B, K), np.uint16)
            L.dm_fc_backward_input(1, dout, B, N, W, K, None, _p(bf(act)), None, _p(din))
            refd = (dout.astype(np.float64) @ W.astype(np.float64)) * (unbf(bf(act)) > 0)
            close_bf16(din, refd, boundd, "fc backward input bf16")
        else:
            din = np.zeros((B, K), np.float32)
            L.dm_fc_backward_input(0, dout, B, N, W, K, _p(act), None, _p(din), None)
            assert np.all(np.abs(din - refd) <= boundd + 1e-30), "fc backward input"
        # weight and bias gradients accumulate into what is there
        dW0 = rng.normal(0, 1, (N, K)).astype(np.float32)
        db0 = rng.normal(0, 1, N).astype(np.float32)
        dW, db = dW0.copy(), db0.copy()
        L.dm_fc_backward_weight(in_bf16, dout, B, N, _p(x), _p(x16), K, dW, db)
        refw = dW0 + dout.T.astype(np.float64) @ xv
        boundw = (B + 1) * U32 * (np.abs(dout.T).astype(np.float64) @ np.abs(xv) + np.abs(dW0))
        assert np.all(np.abs(dW - refw) <= boundw + 1e-30), "fc backward weight"
        refb = db0 + dout.astype(np.float64).sum(0)
        boundb = (B + 1) * U32 * (np.abs(dout).astype(np.float64).sum(0) + np.abs(db0))
        assert np.all(np.abs(db - refb) <= boundb + 1e-30), "fc bias"
    # conv bias gradient: 32 channel sums over bf16 rows (grid-stride rows)
    for rows, blocks in ((1, 1), (37, 2), (5000, 3)):
        dY = bf(rng.normal(0, 1, (rows, 32)))
        db0 = rng.normal(0, 1, 32).astype(np.float32)
        db = db0.copy()
        L.dm_bias_grad(dY, rows, blocks, db)
        ref = db0 + unbf(dY).sum(0)
        bound = (rows + 10) * U32 * (np.abs(unbf(dY)).sum(0) + np.abs(db0))
        assert np.all(np.abs(db - ref) <= bound), ("bias grad", rows)
    # Gaussian negative log-likelihood and its gradient; the loss goes into
    # the log entry of the step
    for B in (1, 5, 32):
        out = np.concatenate([rng.normal(0, 1, (B, 6)), rng.normal(0, 1.5, (B, 6))], 1).astype(np.float32)
        y = rng.uniform(-1, 1, (B, 6)).astype(np.float32)
        dout = np.zeros((B, 12), np.float32)
        loss_log = np.full(4, 0.25, np.float32)
        L.dm_nll(out, y, B, dout, loss_log, 2)
        want, g = onn.gaussian_nll(out, y)
        o64 = out.astype(np.float64)
        terms = 0.5 * ((y - o64[:, :6]) ** 2 * np.exp(-o64[:, 6:]) + np.abs(o64[:, 6:])) / B
        assert abs(loss_log[2] - 0.25 - want) <= (6 * B + 40) * U32 * (terms.sum() + 0.25), B
        assert loss_log[[0, 1, 3]].tolist() == [0.25] * 3
        assert np.all(np.abs(dout - g) <= 16 * U32 * (np.abs(g) + 0.5 / B * (1 + terms.max() * B))), B
    # Adam with the step count t = step + 1, then the step counter's increment
    for step in (0, 7):
        n = 1000
        th, m, v = (rng.normal(0, 1, n).astype(np.float32) for _ in range(3))
        v = np.abs(v)
        gr = rng.normal(0, 1, n).astype(np.float32)
        th1, m1, v1 = th.copy(), m.copy(), v.copy()
        L.dm_adam(th1, m1, v1, gr, n, 1e-3, step)
        tw, mw, vw = onn.adam(th.astype(np.float64), m.astype(np.float64), v.astype(np.float64),
                              gr.astype(np.float64), step + 1, np.float64(np.float32(1e-3)))
        assert np.all(np.abs(m1 - mw) <= 8 * U32 * (np.abs(m) + np.abs(gr)))
        assert np.all(np.abs(v1 - vw) <= 8 * U32 * (v + gr * gr))
        assert np.all(np.abs(th1 - tw) <= 4 * U32 * np.abs(th) + 1e-3 * 1e-4)
    # bf16 copies, bit for bit
    a = np.concatenate([rng.normal(0, 1, 3000), [0.0, -0.0, 1.0 + 2.0**-8, 1.0 + 3 * 2.0**-8, 3e-39]]).astype(np.float32)
    b16 = np.zeros(a.size, np.uint16)
    L.dm_to_bf16(a, a.size, b16)
    assert np.array_equal(b16, bf(a))
    # uniform initialisation: U(-a, a) from the top 24 bits of Philox(seed)
    # with the counter (i, tensor, 0x6E6E0000, 0), in fp32
    p = np.zeros(300, np.float32)
    L.dm_init_uniform(p, p.size, 0.125, 2**33 + 5, 3)
    key = np.array([5, 2], np.uint32)
    for i in (0, 1, 150, 299):
        r = orc.philox(np.array([i, 3, 0x6E6E0000, 0], np.uint32), key)
        u = np.float32(r[0] >> 8) * np.float32(2.0**-24)
        assert p[i] == np.float32(0.125) * (np.float32(2.0) * u - np.float32(1.0)), i
    assert np.all(np.abs(p) < 0.125) and len(np.unique(p)) == p.size
    # the network input: box average of each cell / 64, rounded to bf16, in
    # channel c of [G^3][2]
    for dims, orig, sp, box, G in (((9, 7, 5), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), 4),
                                   ((13, 11, 9), (1.5, -2.0, 0.25), (0.8, 1.1, 1.3), (-1.0, -3.0, 0.0), 6),
                                   ((30, 20, 10), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (-8.0, 4.0, -2.0), 8)):
        vol = rng.integers(0, 256, dims[::-1]).astype(np.uint8)
        h = np.array(dims, np.float32) * np.array(sp, np.float32) / np.float32(G)
        for c in (0, 1):
            x = np.full(G**3 * 2, 0x7777, np.uint16)
            L.dm_downsample(vol, np.array(dims, np.int32), np.array(orig, np.float32), np.array(sp, np.float32),
                            np.array(box, np.float32), h, G, c, x)
            want = onn.box_average(vol, np.array(orig), np.array(sp), np.array(box), h.astype(np.float64), G)
            got = unbf(x.reshape(-1, 2)[:, c]).reshape(G, G, G)
            assert np.all(np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 4 * U32 * np.abs(want)), dims
            assert np.all(x.reshape(-1, 2)[:, 1 - c] == 0x7777)


def test_network_cuda_core_kernels_equal_the_oracle(orc, tmp_path):
    _check_nn_small(_build_nn_small(open(NN_CU).read(), tmp_path), orc)


NS_MUTANTS = [
    ("bias of the batch row", "acc += bias[n];", "acc += bias[b];"),
    ("ReLU mask keeps zeros", "if (!(to_f(act[i]) > 0.0f)) acc = 0.0f;", "if (!(to_f(act[i]) >= 0.0f)) acc = 0.0f;"),
    ("bias gradient overwritten", "if (k == 0) db[n] += accb;", "if (k == 0) db[n] = accb;"),
    ("log-variance gradient sign", "0.5f * (1.0f - r * r * e) / (float)B;", "0.5f * (1.0f + r * r * e) / (float)B;"),
    ("second moment with beta1", "vi = b2 * v[i] + (1.0f - b2) * gi * gi;",
     "vi = b2 * v[i] + (1.0f - b1) * gi * gi;"),
    ("cell end rounded down", "hi[d] = min(a.dims[d], (int)ceilf(", "hi[d] = min(a.dims[d], (int)floorf("),
]


def test_network_kernel_comparison_catches_planted_mistakes(orc, tmp_path):
    src = open(NN_CU).read()
    for text in (m[1] for m in NS_MUTANTS):
        assert src.count(text) == 1, text
    for L in _build_all(_build_nn_small, src, NS_MUTANTS, tmp_path):
        with pytest.raises(AssertionError):
            _check_nn_small(L, orc)


SY_CPP = os.path.join(ROOT, "tests", "nn_synth_host.cpp")
SY_BEGIN, SY_END = "// Synthetic training pairs:", "}  // namespace nn\n\nnamespace nn {\n// Failure-detection"


def _build_synth(src_text, d):
    import ctypes as C
    assert src_text.count(SY_BEGIN) == 1 and src_text.count(SY_END) == 1
    assert src_text.count(NS_BEGIN) == 1
    (d / "nn_small.inc").write_text(src_text[src_text.index(NS_BEGIN):src_text.index(SY_BEGIN)])
    (d / "nn_synth.inc").write_text(src_text[src_text.index(SY_BEGIN):src_text.index(SY_END)])
    so = str(d / "libsyn.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I" + SHIM,
                    "-I" + str(d), SY_CPP, "-o", so], check=True)
    L = C.CDLL(so)
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    u16p = np.ctypeslib.ndpointer(np.uint16, flags="C_CONTIGUOUS")
    L.dm_synth_params.argtypes = [C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, C.c_uint64, C.c_int, C.c_int,
                                  f32p, f32p, f32p, i32p, f32p]
    L.dm_synth_views.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, C.c_uint64, C.c_int,
                                 C.c_int, f32p, u16p]
    L.dm_synth_full.argtypes = [C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, C.c_uint64, C.c_int, C.c_int,
                                C.c_int, f32p, f32p]
    return L


def _synth(L, dims, rl, tl, seed, step, B):
    R, t, c = np.zeros((B, 3, 3), np.float32), np.zeros((B, 3), np.float32), np.zeros((B, 3), np.float32)
    shift, y = np.zeros(B, np.int32), np.zeros((B, 6), np.float32)
    L.dm_synth_params(*dims, rl, tl, seed, step, B, R, t, c, shift, y)
    return R, t, c, shift, y


def _check_synth(L, orc):
    """The learned proposal's training labels are poses in the filter's
    convention: for each synthetic pair, the map from a target voxel to the
    source point its tissue comes from equals the pose -> matrix step (Eq. 3)
    applied to the label pose, with the source at the origin and the target
    grid slid along x by the pair's shift."""
    rng = np.random.default_rng(42)
    for dims, seed, step in (((224, 208, 176), 7, 3), ((64, 48, 40), 2**40 + 1, 0), ((96, 96, 96), 5, 1000)):
        rl, tl = np.float32(np.deg2rad(30.0)), np.float32(25.0)
        B = 32
        R, t, c, shift, y = _synth(L, dims, rl, tl, seed, step, B)
        assert np.all(np.abs(y) <= 1.0) and np.std(y) > 0.3
        assert np.array_equal(c, np.tile((np.array(dims, np.float32) - 1) / 2, (B, 1)))
        assert np.all(shift >= int(0.40 * dims[0])) and np.all(shift <= int(np.ceil(0.65 * dims[0])))
        R2 = _synth(L, dims, rl, tl, seed, step, B)[0]
        assert np.array_equal(R, R2)                                   # seeded
        assert not np.array_equal(R, _synth(L, dims, rl, tl, seed, step + 1, B)[0])
        for b in range(B):
            pose = np.concatenate([y[b, :3] * rl, y[b, 3:] * tl]).astype(np.float32)
            assert np.allclose(pose[3:], t[b], rtol=1e-6, atol=1e-5), b
            M, a = orc.pose_matrix(pose, np.array(dims, np.int32), np.zeros(3, np.float32),
                                   np.array([shift[b], 0, 0], np.float32))
            M = M.reshape(3, 4).astype(np.float64)
            p = rng.uniform(0, np.array(dims) - 1, (16, 3))
            q_filter = (p - a) @ M[:, :3].T + M[:, 3]
            q_pair = (p + [shift[b], 0, 0] - c[b]) @ R[b].astype(np.float64).T + c[b] + t[b]
            assert np.abs(q_filter - q_pair).max() < 1e-4, (dims, b)


def _check_synth_views(L, orc):
    """The network input of each synthetic pair is its two full-resolution
    views (the kernels' own per-voxel function) box-averaged as the oracle
    box-averages a real volume: the source view over the box at the
    origin, the target view, slid along x by the pair's shift, over the same
    box (cells it does not reach stay 0), each / 64 in bf16."""
    import oracle.nn as onn
    rl, tl = np.float32(np.deg2rad(30.0)), np.float32(25.0)
    for dims, G, seed, step, B in (((40, 36, 30), 16, 3, 2, 3), ((48, 40, 32), 8, 11, 0, 2)):
        X, Y, Z = dims
        y = np.zeros((B, 6), np.float32)
        x = np.full((B, G**3, 2), 0x7777, np.uint16)
        L.dm_synth_views(X, Y, Z, G, rl, tl, seed, step, B, y, x)
        _, _, _, shift, y2 = _synth(L, dims, rl, tl, seed, step, B)
        assert np.array_equal(y, y2)
        h = np.array(dims, np.float64) / G
        for b in range(B):
            S, T = np.zeros((Z, Y, X), np.float32), np.zeros((Z, Y, X), np.float32)
            L.dm_synth_full(X, Y, Z, rl, tl, seed, step, B, b, S, T)
            assert S.min() >= 0 and S.max() <= 255 and np.array_equal(S, np.rint(S)) and S.std() > 5
            for ch, (vol, org) in enumerate(((S, (0.0, 0.0, 0.0)), (T, (float(shift[b]), 0.0, 0.0)))):
                want = onn.box_average(vol, np.array(org), np.ones(3), np.zeros(3), h, G)
                got = onn.from_bf16_bits(x[b, :, ch]).astype(np.float64).reshape(G, G, G)
                assert np.all(np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 1e-7), (dims, b, ch)
            assert np.all(x[b, :, 1].reshape(G, G, G)[:, :, : int(shift[b] // h[0])] == 0)


def test_training_labels_follow_the_filters_pose_convention(orc, tmp_path):
    _check_synth(_build_synth(open(NN_CU).read(), tmp_path), orc)


def test_training_inputs_are_the_box_averaged_views(orc, tmp_path):
    _check_synth_views(_build_synth(open(NN_CU).read(), tmp_path), orc)


SY_MUTANTS = [
    ("rotation order Rz Ry Rx", "const float Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy};",
     "const float Ry[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx};"),
    ("angle of the wrong axis", "sincosf(ang[0], &sx, &cx);", "sincosf(ang[2], &sx, &cx);"),
    ("centre at dims / 2", "s.c[d] = 0.5f * (dims[d] - 1.0f);", "s.c[d] = 0.5f * dims[d];"),
    ("label of the translation negated", "a.y[b * 6 + 3 + d] = tr[d] / a.trans_lim;",
     "a.y[b * 6 + 3 + d] = -tr[d] / a.trans_lim;"),
]


def test_training_label_comparison_catches_planted_mistakes(orc, tmp_path):
    src = open(NN_CU).read()
    for text in (m[1] for m in SY_MUTANTS):
        assert src.count(text) == 1, text
    for L in _build_all(_build_synth, src, SY_MUTANTS, tmp_path):
        with pytest.raises(AssertionError):
            _check_synth(L, orc)


SV_MUTANTS = [
    ("first target column dropped", "if (px >= 0 && px < a.X) {", "if (px > 0 && px < a.X) {"),
    ("cell end rounded down", "hi[d] = min(dims[d], (int)ceilf(h * (g[d] + 1)));",
     "hi[d] = min(dims[d], (int)floorf(h * (g[d] + 1)));"),
    ("target mean over the source count", "xo[1] = bf16_bits(cnt_t ? sum_t / cnt_t",
     "xo[1] = bf16_bits(cnt_t ? sum_t / cnt_s"),
]


def test_training_input_comparison_catches_planted_mistakes(orc, tmp_path):
    src = open(NN_CU).read()
    for text in (m[1] for m in SV_MUTANTS):
        assert src.count(text) == 1, text
    for L in _build_all(_build_synth, src, SV_MUTANTS, tmp_path):
        with pytest.raises(AssertionError):
            _check_synth_views(L, orc)


def test_tensor_core_operand_layout_matches_its_descriptors(tmp_path):
    # The GEMM's operand tiles (K-major, no swizzle): tile_offset is a
    # bijection onto the tile's bytes, each 8 x 8 core matrix is 128
    # contiguous bytes, and its K and row-group strides are the LBO and SBO
    # the kernel puts in its descriptors, whose fields decode as the PTX
    # ISA's tcgen05 shared-memory and kind::f16 instruction descriptors
    import ctypes as C
    so = str(tmp_path / "libumma.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I" + SHIM,
                    os.path.join(ROOT, "tests", "umma_layout_host.cpp"), "-o", so], check=True)
    L = C.CDLL(so)
    L.dm_tile_offset.restype = C.c_uint32
    L.dm_tile_offset.argtypes = [C.c_int, C.c_int, C.c_int]
    L.dm_smem_desc.restype = C.c_uint64
    L.dm_smem_desc.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32]
    L.dm_idesc.restype = C.c_uint32
    L.dm_idesc.argtypes = [C.c_int, C.c_int]
    nn_src = open(NN_CU).read()
    assert nn_src.count("constexpr int kChunkK = 64;") == 1
    n_a = nn_src.count("umma::smem_desc(a + 256 * kk, 128, 16 * kChunkK)")   # the K-major GEMMs' A and B
    assert n_a >= 1 and nn_src.count("umma::smem_desc(b + 256 * kk, 128, 16 * kChunkK)") == n_a
    for rows, kcols in ((128, 64), (32, 64), (128, 16)):
        off = np.array([[L.dm_tile_offset(r, k, kcols) for k in range(kcols)] for r in range(rows)], np.int64)
        assert np.array_equal(np.sort(off.ravel()), 2 * np.arange(rows * kcols))      # bijection, bf16 steps
        for g in range(rows // 8):
            for j in range(kcols // 8):
                core = off[8 * g:8 * g + 8, 8 * j:8 * j + 8]
                base = core.min()
                assert np.array_equal(core - base, 16 * np.arange(8)[:, None] + 2 * np.arange(8)[None, :])
                assert base == g * 16 * kcols + j * 128                              # SBO, LBO
        for m in range(kcols // 16):
            assert off[0, 16 * m] == 256 * m                                         # per-MMA K advance
    for addr, lbo, sbo in ((0x400, 128, 1024), (0x3FFF0, 128, 16 * 64), (0x1230, 2048, 512)):
        d = L.dm_smem_desc(addr, lbo, sbo)
        assert d & 0x3FFF == (addr >> 4) & 0x3FFF
        assert (d >> 16) & 0x3FFF == lbo >> 4 and (d >> 32) & 0x3FFF == sbo >> 4
        assert (d >> 46) & 0x7 == 1 and (d >> 49) & 0x7 == 0 and (d >> 52) & 1 == 0 and d >> 61 == 0
        assert (d >> 14) & 3 == 0 and (d >> 30) & 3 == 0 and (d >> 53) & 0xFF == 0
    for M, N in ((128, 32), (128, 256), (64, 8)):
        i = L.dm_idesc(M, N)
        assert i & 0xF == 0 and (i >> 4) & 3 == 1 and (i >> 6) & 1 == 0              # dense, f32 D
        assert (i >> 7) & 7 == 1 and (i >> 10) & 7 == 1                               # bf16 A, B
        assert (i >> 13) & 0xF == 0                                                   # no negate, K-major
        assert (i >> 17) & 0x3F == N >> 3 and (i >> 23) & 1 == 0 and (i >> 24) & 0x1F == M >> 4
        assert i >> 29 == 0


# ------------------- the measurement's warp routine under a lockstep warp emulation

MW_CPP = os.path.join(ROOT, "tests", "measure_warp_host.cpp")
MI_END = "// Measurement kernel of one registration."
MX_BEGIN, MX_END = "constexpr int kTabMaxX = 512;", "// CTAB (with XTAB):"


def _build_measure_warp(src_text, d, debug=False, extra=()):
    import ctypes as C
    for m in (MV_BEGIN, MI_END, MX_BEGIN, MX_END):
        assert src_text.count(m) == 1, m
    (d / "measure_item.inc").write_text(src_text[src_text.index(MV_BEGIN):src_text.index(MI_END)])
    (d / "measure_xtab.inc").write_text(src_text[src_text.index(MX_BEGIN):src_text.index(MX_END)])
    so = str(d / "libmw.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-frounding-math", "-fPIC", "-shared",
                    "-I" + SHIM, "-I" + str(d), *(["-DPF_DEBUG=1"] if debug else []), *extra, MW_CPP, "-o", so],
                   check=True)
    L = C.CDLL(so)
    L.dm_debug_hits.restype = C.c_ulonglong
    L.dm_fp32_ops.restype = C.c_ulonglong
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
    L.dm_measure_warp.argtypes = [C.c_int] * 4 + [C.c_void_p, C.c_void_p, i32p, C.c_void_p, C.c_void_p, i32p,
                                                   f32p, C.c_int, f32p, u64p]
    return L


def _warp_cases(orc, seed, count):
    import pfsynth
    rng = np.random.default_rng(seed)
    for i in range(count):
        # long source rows (so the visit intervals run over several 64-voxel
        # passes) on some cases, short ones (every pass crosses rows) on others
        sd = (int(rng.integers(2, 200 if i % 2 else 40)), int(rng.integers(2, 30)), int(rng.integers(2, 20)))
        td = (int(rng.integers(2, 200)), int(rng.integers(2, 24)), int(rng.integers(2, 12)))
        src = pfsynth.random_image(int(rng.integers(0, 1 << 30)), sd)
        tgt = pfsynth.random_image(int(rng.integers(0, 1 << 30)), td)
        smask = (rng.random((sd[2], sd[1], sd[0])) < 0.5).astype(np.uint8)
        tmask = (rng.random((td[2], td[1], td[0])) < 0.5).astype(np.uint8)
        so = rng.uniform(-10, 10, 3).astype(np.float32)
        to = rng.uniform(-10, 10, 3).astype(np.float32)
        P = 3
        rot = 1.5 if i % 3 else 0.15
        poses = np.concatenate([rng.uniform(-rot, rot, (3, P)), rng.uniform(-12, 12, (3, P))]).astype(np.float32)
        if i % 4 == 0:
            poses[:3, 0] = 0.0
            so, to = np.round(so * 2) / 2, np.round(to * 2) / 2
            poses[3:, 0] = np.round(poses[3:, 0] * 2) / 2
        mats, a = orc.pose_matrices(poses, sd, so, to)
        yield sd, td, src, tgt, smask, tmask, np.ascontiguousarray(mats, np.float32), a


WARP_CONFIGS = ((1, 0, 0, 0), (1, 0, 0, 1), (1, 0, 1, 1), (0, 1, 0, 0), (0, 1, 0, 1), (1, 1, 0, 1), (1, 1, 1, 0))


def _bright_case(orc):
    # a bright source under a large overlap: one particle's S2 passes 2^64,
    # so the high word is reached through the atomic's carry
    rng = np.random.default_rng(33)
    sd, td = (80, 80, 70), (74, 74, 62)
    src = (255 - rng.integers(0, 3, (sd[2], sd[1], sd[0]))).astype(np.uint8)
    tgt = rng.integers(0, 256, (td[2], td[1], td[0])).astype(np.uint8)
    pose = np.array([0.01, -0.01, 0.02, 0.3, -0.2, 0.1], np.float32)
    mats, a = orc.pose_matrices(pose[:, None], sd, np.zeros(3, np.float32), np.full(3, 3.0, np.float32))
    return sd, td, src, tgt, None, None, np.ascontiguousarray(mats, np.float32), a


def _edge_case(orc):
    # rows 64 voxels long for nearest-neighbour sampling whose trilinear
    # interval ends one voxel earlier, on the source's top y plane (so the y
    # corner is clamped): a combined full pass in which the image interval
    # ends and the clamp is needed
    rng = np.random.default_rng(41)
    sd, td = (64, 6, 5), (70, 6, 5)
    src = rng.integers(0, 256, (sd[2], sd[1], sd[0])).astype(np.uint8)
    tgt = rng.integers(0, 256, (td[2], td[1], td[0])).astype(np.uint8)
    smask = (rng.random(src.shape) < 0.5).astype(np.uint8)
    tmask = (rng.random(tgt.shape) < 0.5).astype(np.uint8)
    pose = np.array([0, 0, 0, 0.25, 0, 0], np.float32)
    mats, a = orc.pose_matrices(pose[:, None], sd, np.zeros(3, np.float32), np.zeros(3, np.float32))
    return sd, td, src, tgt, smask, tmask, np.ascontiguousarray(mats, np.float32), a


def _check_measure_warp(L, orc, seed=31, count=24):
    import itertools
    bright = _bright_case(orc)
    assert orc.measure_image(bright[2], bright[3], bright[6], bright[7])[0, 3] > 0   # S2 high word used
    for sd, td, src, tgt, smask, tmask, mats, a in itertools.chain(_warp_cases(orc, seed, count), [_edge_case(orc), bright]):
        P = mats.shape[0]
        sdv, tdv = np.array(sd, np.int32), np.array(td, np.int32)
        want_img = orc.measure_image(src, tgt, mats, a)
        want_msk = orc.measure_mask(smask, tmask, mats, a) if smask is not None else None
        for img, msk, int_index, xtab in WARP_CONFIGS:
            if msk and smask is None:   # the bright case is an image case
                continue
            got = np.zeros((P, 12), np.uint64)
            L.dm_measure_warp(img, msk, int_index, xtab, _ptr(src) if img else None, _ptr(smask) if msk else None,
                              sdv, _ptr(tgt) if img else None, _ptr(tmask) if msk else None, tdv, mats, P, a, got)
            cfg = (sd, td, img, msk, int_index, xtab)
            if img:
                assert np.array_equal(got[:, 0:7], want_img), cfg
            if msk:
                assert np.array_equal(got[:, 8:12], want_msk), cfg


def test_measurement_gathers_stay_in_bounds(orc, tmp_path):
    # the debug build's checks (every source, mask-bit and target index
    # against its buffer before the load) over every case of the warp-routine
    # comparison: no index outside, and the moments unchanged
    L = _build_measure_warp(open(MEASURE_CU).read(), tmp_path, debug=True)
    _check_measure_warp(L, orc)
    assert L.dm_debug_hits() == 0


def test_measurement_warp_routine_equals_the_oracle(orc, tmp_path):
    # measure_item -- row set-up, the sweep of 32 rows' intervals in passes of
    # 64 voxels with the row-crossing passes, the per-voxel code and the warp
    # reduction with its atomics -- and the warp's x-product table, copied
    # verbatim out of measure.cu and run by a lockstep emulation of one warp:
    # the moments equal the oracle's in every form the kernel instantiates
    # (image, mask, combined; fp32 or integer quad index; with or without the
    # table), on rows longer than two passes, single-voxel rows and empty ones
    L = _build_measure_warp(open(MEASURE_CU).read(), tmp_path)
    _check_measure_warp(L, orc)


# planted mistakes in the sweep, each of which the comparison above must catch
MW_MUTANTS = [
    ("a full pass advances 63 voxels", "pos += 64;\n                xf = __fadd_rn(xf, 64.0f);\n                toff += 64u;",
     "pos += 63;\n                xf = __fadd_rn(xf, 63.0f);\n                toff += 63u;"),
    ("the next row's share of a crossing pass miscounted", "const int used1 = 64 - len0;",
     "const int used1 = 63 - len0;"),
    ("the crossing pass's second entry from the wrong row",
     "const bool in0a = e0 < len0, in1a = e1 < len0;", "const bool in0a = e0 < len0, in1a = e1 <= len0;"),
    ("the last row's remainder dropped", "if (len0 == 0 && !has1) break;", "if (!has1) break;"),
    ("the S2 carry lost", "if (old + S2 < old) atomicAdd(dst + 3, 1ull);", "(void)old;"),
    ("the x table built from the second row of the matrix",
     "const float r0 = __ldg(Mp + 0), r1 = __ldg(Mp + 4), r2 = __ldg(Mp + 8);",
     "const float r0 = __ldg(Mp + 1), r1 = __ldg(Mp + 4), r2 = __ldg(Mp + 8);"),
]


def _build_all(build, src, mutants, tmp_path):
    """Build one library per planted mistake, in parallel (compiles dominate)."""
    from concurrent.futures import ThreadPoolExecutor
    dirs = []
    for k, (name, text, planted) in enumerate(mutants):
        assert src.count(text) >= 1, name
        d = tmp_path / f"m{k}"
        d.mkdir()
        dirs.append((d, src.replace(text, planted)))
    with ThreadPoolExecutor(max_workers=max(1, min(os.cpu_count() or 1, 8))) as ex:
        return list(ex.map(lambda t: build(t[1], t[0]), dirs))


def test_measurement_warp_comparison_catches_planted_mistakes(orc, tmp_path):
    src = open(MEASURE_CU).read()
    for text in (m[1] for m in MW_MUTANTS):
        assert src.count(text) == 1, text
    for L in _build_all(_build_measure_warp, src, MW_MUTANTS, tmp_path):
        with pytest.raises(AssertionError):
            _check_measure_warp(L, orc, seed=32, count=10)


# ------------------------------------- the prediction kernel under the warp emulation

PH_CPP = os.path.join(ROOT, "tests", "predict_host.cpp")
PH_BEGIN, PH_END = "// Prediction for k > 0", "// Weighted quaternion average"


def _build_predict(src_text, d):
    import ctypes as C
    assert src_text.count(PH_BEGIN) == 1 and src_text.count(PH_END) == 1
    (d / "predict.inc").write_text(src_text[src_text.index(PH_BEGIN):src_text.index(PH_END)])
    so = str(d / "libph.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I" + SHIM,
                    "-I" + str(d), PH_CPP, "-o", so], check=True)
    L = C.CDLL(so)
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    L.dm_predict.argtypes = [C.c_int, C.c_int, C.c_uint64, f32p, C.c_float, C.c_float, i32p, f32p, f32p, i32p,
                             f32p, f32p, f32p, f32p, f32p, C.c_int, C.c_void_p]
    return L


def _check_predict(L, orc, seed=34, count=40):
    rng = np.random.default_rng(seed)
    for i in range(count):
        N = 4 * int(rng.integers(1, 129))
        k = int(rng.choice([0, 1, 2, int(rng.integers(3, 60))]))
        lim = np.concatenate([rng.uniform(0.05, 1.5707963, 3), rng.uniform(0.5, 60, 3)]).astype(np.float32)
        s0, decay = float(rng.uniform(0.05, 1.0)), float(rng.uniform(0.5, 1.0))
        seed_i = int(rng.integers(0, 2**63))
        sd = rng.integers(2, 300, 3).astype(np.int32)
        td = rng.integers(2, 300, 3).astype(np.int32)
        so = rng.uniform(-30, 30, 3).astype(np.float32)
        to = rng.uniform(-30, 30, 3).astype(np.float32)
        unit = i % 2 == 0
        ss = np.ones(3, np.float32) if unit else rng.uniform(0.3, 2.5, 3).astype(np.float32)
        ts = np.ones(3, np.float32) if unit else rng.uniform(0.3, 2.5, 3).astype(np.float32)
        _, a = orc.pose_matrix(np.zeros(6, np.float32), sd, so, to, ss, ts)
        x0 = orc.init_particles(N, seed_i, lim)
        if i % 5 == 0:   # clouds at the limits, so the perturbation clamps
            x0 = np.where(rng.random(x0.shape) < 0.5, lim[:, None], -lim[:, None]).astype(np.float32)
        x = x0.copy()
        mats = np.zeros((N, 12), np.float32)
        est_q = i % 3 == 1                 # the quaternion estimator's per-pose quaternions too
        quat = np.zeros((4, N))
        L.dm_predict(N, k, seed_i, lim, s0, decay, sd, so, ss, td, to, ts, a, x, mats, int(est_q),
                     quat.ctypes.data if est_q else None)
        want = orc.perturb(x0, seed_i, k, orc.sigma(s0, decay, k, lim), lim) if k > 0 else x0
        assert np.array_equal(x, want), (i, N, k)
        wm, _ = orc.pose_matrices(want, sd, so, to, ss, ts)
        assert np.array_equal(mats, wm), (i, N, k)
        if est_q:
            # q and -q are one rotation; fp64 half-angle formulas against the
            # oracle's sin/cos of the half angles
            for j in range(N):
                q = orc.quaternion(want[:, j])
                sgn = 1.0 if np.dot(q, quat[:, j]) >= 0 else -1.0
                np.testing.assert_allclose(quat[:, j], sgn * q, rtol=0, atol=1e-12, err_msg=str((i, j)))


def test_prediction_kernel_equals_the_oracle(orc, tmp_path):
    # k_predict (perturbation, the shared sin/cos chain, pose -> matrix; 8
    # lanes per particle exchanging by shuffles), copied verbatim out of
    # filter.cu and run warp by warp under the lockstep emulation: the
    # perturbed cloud and every matrix equal the oracle's for random cloud
    # sizes, iterations, limits (clamping included), seeds and grids
    _check_predict(_build_predict(open(FILTER_CU).read(), tmp_path), orc)


PH_MUTANTS = [
    ("noise scale decays one step too few", "for (int q = 0; q < k; ++q) pk = __dmul_rn(pk, (double)P.sigma_decay);",
     "for (int q = 1; q < k; ++q) pk = __dmul_rn(pk, (double)P.sigma_decay);"),
    ("no lower clamp", "        if (v < -P.lim[j]) v = -P.lim[j];\n        x = v;", "        x = v;"),
    ("cosine lanes take the wrong angle",
     "const float ang = __shfl_sync(gmask, x, gbase + (j < 3 ? j : (j < 6 ? j - 3 : 0)));",
     "const float ang = __shfl_sync(gmask, x, gbase + (j < 3 ? j : (j < 6 ? 5 - j : 0)));"),
    ("sin and cos of one angle swapped",
     "matrix_from_sincos(pose, sc[0], sc[3], sc[1], sc[4], sc[2], sc[5], P.g, M);",
     "matrix_from_sincos(pose, sc[3], sc[0], sc[1], sc[4], sc[2], sc[5], P.g, M);"),
]


def test_prediction_comparison_catches_planted_mistakes(orc, tmp_path):
    src = open(FILTER_CU).read()
    for name, text, _ in PH_MUTANTS:
        assert src.count(text) == 1, name
    for L in _build_all(_build_predict, src, PH_MUTANTS, tmp_path):
        with pytest.raises(AssertionError):
            _check_predict(L, orc, seed=35, count=10)


# ------------------------------ the update step under the block emulation

UH_CPP = os.path.join(ROOT, "tests", "update_host.cpp")
UH_BEGIN, UH_END = "// Weighted quaternion average", "// Batched prediction"
UH_EXTERN = "extern __shared__ unsigned long long sh_cdf[];"


def _build_update(src_text, d):
    import ctypes as C
    assert src_text.count(UH_BEGIN) == 1 and src_text.count(UH_END) == 1
    region = src_text[src_text.index(UH_BEGIN):src_text.index(UH_END)]
    assert region.count(UH_EXTERN) == 1
    # the dynamic shared array becomes the array the harness declares
    (d / "update.inc").write_text(region.replace(UH_EXTERN, "extern unsigned long long sh_cdf[];"))
    so = str(d / "libuh.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I" + SHIM,
                    "-I" + str(d), UH_CPP, "-o", so], check=True)
    L = C.CDLL(so)
    P = lambda t: np.ctypeslib.ndpointer(t, flags="C_CONTIGUOUS")   # noqa: E731
    L.dm_update.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, C.c_int, C.c_int,
                            P(np.uint64), P(np.float32), P(np.float32), P(np.float64), P(np.uint64), P(np.uint64),
                            P(np.int32), P(np.float64), P(np.float64), P(np.int32), P(np.uint64), C.c_int,
                            C.c_void_p]
    return L


def _check_update(L, orc, seed=36, sizes=(1, 31, 33, 256, 1024, 1025, 4096, 13000)):
    rng = np.random.default_rng(seed)
    for case, N in enumerate(sizes):
        for three in ((0, 1) if N <= 1024 else (0,)):
            mode, g = int(rng.integers(0, 4)), int(rng.integers(0, 8))
            seed_i, k = int(rng.integers(0, 2**63)), int(rng.integers(0, 40))
            moms, b_full = zip(*[_random_moments(rng) for _ in range(N)])
            mom = np.ascontiguousarray(np.stack(moms))
            b_full = max(b_full)
            n_min = int(rng.choice([0, 1 << 24]))
            if case == 2:                      # every score 0: the cloud is kept, the estimate is the plain mean
                n_min = 1 << 40
            x0 = rng.uniform(-1, 1, (6, N)).astype(np.float32)
            poses, pm = x0.copy(), np.zeros_like(x0)
            sc, W, Cc = np.zeros(N), np.zeros(N, np.uint64), np.zeros(N, np.uint64)
            idx, log6, scal = np.zeros(N, np.int32), np.zeros(6), np.zeros(2)
            ints, ev = np.zeros(2, np.int32), np.zeros(1, np.uint64)
            est_q = (case + three) % 2 == 1    # the quaternion estimator on every other case
            quat = np.ascontiguousarray(np.stack([orc.quaternion(x0[:, j]) for j in range(N)], 1)) if est_q else None
            L.dm_update(mode, N, g, b_full, n_min, seed_i, k, three, mom, poses, pm, sc, W, Cc, idx, log6, scal,
                        ints, ev, int(est_q), quat.ctypes.data if est_q else None)
            want_s = np.array([orc.score(mode, m, b_full, n_min) for m in mom])
            want_W = orc.weights(want_s, g)
            want_idx = orc.resample(want_W, orc.resample_offset(seed_i, k))
            cfg = (N, three, mode, g)
            assert np.array_equal(sc, want_s), cfg
            assert np.array_equal(W, want_W) and np.array_equal(Cc, np.cumsum(want_W, dtype=np.uint64)), cfg
            assert np.array_equal(idx, want_idx), cfg
            assert np.array_equal(pm, x0) and np.array_equal(poses, x0[:, want_idx]), cfg
            # the estimate's sums run in another order: equal within their rounding
            want_est = orc.estimate(x0, want_W)
            np.testing.assert_allclose(log6[3:], want_est[3:], rtol=1e-12, atol=1e-12, err_msg=str(cfg))
            if est_q:   # the rotation from the weighted quaternion average (eigenvector, then angles)
                np.testing.assert_allclose(log6[:3], orc.estimate_quaternion(x0, want_W)[:3], rtol=0, atol=1e-9,
                                           err_msg=str(cfg))
            else:
                np.testing.assert_allclose(log6[:3], want_est[:3], rtol=1e-12, atol=1e-12, err_msg=str(cfg))
            assert scal[0] == want_s.max() and ints[0] == int(np.argmax(want_s)), cfg
            S = float(want_W.sum())
            want_ess = S * S / float(np.sum(want_W.astype(np.float64) ** 2)) if S > 0 else 0.0
            assert abs(scal[1] - want_ess) <= 1e-12 * max(1.0, want_ess), cfg
            col = 0 if mode in (2, 3) else 8
            assert int(ev[0]) == int(mom[:, col].sum(dtype=np.uint64)) and ints[1] == k + 1, cfg
    # one particle with a positive score after particles of weight 0, and an
    # offset so small that the first pointer is T_0 = 0 = C_0: only the strict
    # C_i > T_j of the resampling search skips the weightless particles
    N, seed_i = 300, 10488
    assert orc.resample_offset(seed_i, 0) < N * 256
    mom = np.zeros((N, 12), np.uint64)
    mom[5, 8:12] = (10, 5, 4, 3)
    poses, pm = rng.uniform(-1, 1, (6, N)).astype(np.float32), np.zeros((6, N), np.float32)
    idx = np.zeros(N, np.int32)
    L.dm_update(0, N, 5, 10, 0, seed_i, 0, 0, mom, poses, pm, np.zeros(N), np.zeros(N, np.uint64),
                np.zeros(N, np.uint64), idx, np.zeros(6), np.zeros(2), np.zeros(2, np.int32), np.zeros(1, np.uint64),
                0, None)
    assert np.all(idx == 5), idx[:4]


def test_update_step_equals_the_oracle(orc, tmp_path):
    # k_update_small and k_score / k_weights / k_finalise, copied verbatim out
    # of filter.cu and run under the block emulation: scores, integer weights,
    # their scan, the resampled indices and cloud bit for bit, the estimate and
    # ESS within their summation rounding, the best score and its first index,
    # the evaluation count, for clouds of 1 to 13000 particles (past the
    # 12288-entry shared-memory CDF), every mode, all-zero scores included
    _check_update(_build_update(open(FILTER_CU).read(), tmp_path), orc)


UH_MUTANTS = [
    ("the warp scan adds a lane too few", "if (lane >= o) v += t;", "if (lane > o) v += t;"),
    ("the systematic pointers divided by N + 1",
     "const unsigned long long T = (unsigned long long)(num >> 32) / (unsigned long long)N;",
     "const unsigned long long T = (unsigned long long)(num >> 32) / (unsigned long long)(N + 1);"),
    ("the search takes C_i >= T_j", "if (cdf[mid] > T) hi = mid; else lo = mid + 1;",
     "if (cdf[mid] >= T) hi = mid; else lo = mid + 1;"),
    ("the last index attaining the maximum",
     "for (int o = 16; o > 0; o >>= 1) bidx = min(bidx, __shfl_xor_sync(0xffffffffu, bidx, o));",
     "for (int o = 16; o > 0; o >>= 1) bidx = max(bidx == INT_MAX ? -1 : bidx, __shfl_xor_sync(0xffffffffu, bidx == INT_MAX ? -1 : bidx, o));"),
    ("ESS without the square", "L.ess = w2 > 0.0 ? Sd * Sd / w2 : 0.0;", "L.ess = w2 > 0.0 ? Sd / w2 : 0.0;"),
    ("the evaluation count of one warp only", "B.stats[1] = ev;", "B.stats[1] = sh_ev[0];"),
]


def test_update_comparison_catches_planted_mistakes(orc, tmp_path):
    src = open(FILTER_CU).read()
    for name, text, _ in UH_MUTANTS:
        assert src.count(text) == 1, name
    for L in _build_all(_build_update, src, UH_MUTANTS, tmp_path):
        with pytest.raises(AssertionError):
            _check_update(L, orc, seed=37, sizes=(7, 300, 1025, 2000))


# ------------------------------------ the measurement kernel under the block emulation

KC_CPP = os.path.join(ROOT, "tests", "measure_cta_host.cpp")
KC_END = "// Measurement of many registrations in one launch"
KC_EXTERN = "extern __shared__ float4 smem_dyn[];"


def test_measurement_kernel_equals_the_oracle(orc, tmp_path):
    # k_measure itself (copied verbatim out of measure.cu), block by block
    # under the emulation: per-warp and per-block (CTAB) x-product tables,
    # mask bits in shared memory or read from the global array, the fp32 or
    # integer quad index, 1 to 8 items per warp, blocks whose items span two
    # particles; the moments equal the oracle's in every combination the
    # launch selects
    import ctypes as C
    import pfsynth
    src = open(MEASURE_CU).read()
    assert src.count(MV_BEGIN) == 1 and src.count(KC_END) == 1
    region = src[src.index(MV_BEGIN):src.index(KC_END)]
    assert region.count(KC_EXTERN) == 1
    (tmp_path / "k_measure.inc").write_text(region.replace(KC_EXTERN, "extern float4 smem_dyn[];"))
    so = str(tmp_path / "libkc.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-frounding-math", "-fPIC", "-shared",
                    "-I" + SHIM, "-I" + str(tmp_path), KC_CPP, "-o", so], check=True)
    L = C.CDLL(so)
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
    L.dm_k_measure.argtypes = [C.c_int] * 7 + [C.c_void_p, C.c_void_p, i32p, C.c_void_p, C.c_void_p, i32p, f32p,
                                                C.c_int, f32p, u64p]
    rng = np.random.default_rng(38)
    runs = ctab_runs = 0
    for i in range(4):
        sd = (int(rng.integers(8, 60)), int(rng.integers(8, 40)), int(rng.integers(8, 30)))
        td = (int(rng.integers(8, 70)), int(rng.integers(16, 32)), int(rng.integers(16, 28)))
        src_v = pfsynth.random_image(int(rng.integers(0, 1 << 30)), sd)
        tgt_v = pfsynth.random_image(int(rng.integers(0, 1 << 30)), td)
        smask = (rng.random((sd[2], sd[1], sd[0])) < 0.5).astype(np.uint8)
        tmask = (rng.random((td[2], td[1], td[0])) < 0.5).astype(np.uint8)
        P = int(rng.integers(2, 6))
        poses = np.concatenate([rng.uniform(-1.2, 1.2, (3, P)), rng.uniform(-8, 8, (3, P))]).astype(np.float32)
        mats, a = orc.pose_matrices(poses, sd, rng.uniform(-4, 4, 3).astype(np.float32),
                                    rng.uniform(-4, 4, 3).astype(np.float32))
        mats = np.ascontiguousarray(mats, np.float32)
        want_img = orc.measure_image(src_v, tgt_v, mats, a)
        want_msk = orc.measure_mask(smask, tmask, mats, a)
        sdv, tdv = np.array(sd, np.int32), np.array(td, np.int32)
        for img, msk in ((1, 0), (0, 1), (1, 1)):
            for smem in ((0, 1) if msk else (0,)):
                for int_index in ((0, 1) if img else (0,)):
                    for xtab, ctab in ((0, 0), (1, 0), (1, 1)):
                        ipw = int(rng.choice([1, 1, 2] if ctab else [1, 2, 4, 8]))
                        got = np.zeros((P, 12), np.uint64)
                        rc = L.dm_k_measure(img, msk, smem, int_index, xtab, ctab, ipw,
                                            _ptr(src_v) if img else None, _ptr(smask) if msk else None, sdv,
                                            _ptr(tgt_v) if img else None, _ptr(tmask) if msk else None, tdv,
                                            mats, P, a, got)
                        if rc != 0:        # a shape the launch does not use (CTAB without enough rows)
                            continue
                        runs += 1
                        ctab_runs += ctab
                        cfg = (sd, td, P, img, msk, smem, int_index, xtab, ctab, ipw)
                        if img:
                            assert np.array_equal(got[:, 0:7], want_img), cfg
                        if msk:
                            assert np.array_equal(got[:, 8:12], want_msk), cfg
    assert runs >= 60 and ctab_runs >= 8, (runs, ctab_runs)


def test_warp_kernel_equals_the_oracle(orc, tmp_path):
    # k_warp itself (copied verbatim out of warp.cu) block by block under the
    # emulation: the matrix built in shared memory from six lanes' sin/cos,
    # rows walked by a grid-stride loop, frames sampled four at a time with a
    # remainder; both index widths and interpolations
    _check_warp_kernel(orc, tmp_path, debug=False)


def test_warp_kernel_gathers_stay_in_bounds(orc, tmp_path):
    # the same runs in the debug build: no gather index outside its frame
    L = _check_warp_kernel(orc, tmp_path, debug=True)
    assert L.dm_debug_hits() == 0


def _check_warp_kernel(orc, tmp_path, debug):
    import ctypes as C
    import pfsynth
    w = open(WARP_CU).read()
    b0 = "constexpr int kWarpThreads = 256;"
    assert w.count(b0) == 1
    i = w.index(b0)
    (tmp_path / "k_warp.inc").write_text(w[i:w.index("}  // namespace", i)])
    so = str(tmp_path / "libwk.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I" + SHIM,
                    "-I" + str(tmp_path), *(["-DPF_DEBUG=1"] if debug else []),
                    os.path.join(ROOT, "tests", "warp_kernel_host.cpp"), "-o", so], check=True)
    L = C.CDLL(so)
    L.dm_debug_hits.restype = C.c_ulonglong
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
    L.dm_k_warp.argtypes = [u8p, C.c_int, i32p, f32p, f32p, u8p, i32p, f32p, f32p, f32p, f32p, C.c_int, C.c_int,
                            C.c_int]
    rng = np.random.default_rng(39)
    for i, (n_frames, blocks) in enumerate(((1, 1), (5, 2), (9, 3), (4, 1))):
        sd = tuple(int(v) for v in rng.integers(3, 24, 3))
        td = tuple(int(v) for v in rng.integers(3, 24, 3))
        frames = np.stack([pfsynth.random_image(int(rng.integers(0, 1 << 30)), sd) for _ in range(n_frames)])
        so, to = rng.uniform(-5, 5, 3).astype(np.float32), rng.uniform(-5, 5, 3).astype(np.float32)
        ss = np.ones(3, np.float32) if i % 2 == 0 else rng.uniform(0.5, 2.0, 3).astype(np.float32)
        ts = np.ones(3, np.float32) if i % 2 == 0 else rng.uniform(0.5, 2.0, 3).astype(np.float32)
        pose = np.concatenate([rng.uniform(-1.2, 1.2, 3), rng.uniform(-6, 6, 3)]).astype(np.float32)
        _, a = orc.pose_matrix(pose, sd, so, to, ss, ts)
        for interp in (0, 1):
            for wide in (0, 1):
                out = np.zeros((n_frames, td[2], td[1], td[0]), np.uint8)
                L.dm_k_warp(np.ascontiguousarray(frames), n_frames, np.array(sd, np.int32), so, ss, out,
                            np.array(td, np.int32), to, ts, a, pose, interp, wide, blocks)
                for f in range(n_frames):
                    want = orc.warp(frames[f], so, td, to, pose, interp, ss, ts)
                    assert np.array_equal(out[f], want), (i, f, interp, wide)
    return L


# --------------------------------- one batch iteration under the block emulation

BH_CPP = os.path.join(ROOT, "tests", "batch_host.cpp")
BF_END = "// Matrix of one pose by a group of 8 lanes"
BM_END = "template <bool IMG, bool MASK, bool SMEM, bool FIDX, bool XTAB, bool CTAB>\ncudaError_t launch_variant"


def _batch_member_type():
    import ctypes as C
    f3, i3 = C.c_float * 3, C.c_int32 * 3
    P = C.c_void_p

    class DmMember(C.Structure):
        _fields_ = [("mode", C.c_int32), ("N", C.c_int32), ("k", C.c_int32), ("gamma_log2", C.c_int32),
                    ("seed", C.c_uint64), ("b_full", C.c_uint64), ("n_min", C.c_uint64),
                    ("lim", C.c_float * 6), ("sigma0_frac", C.c_float), ("sigma_decay", C.c_float),
                    ("sd", i3), ("td", i3), ("so", f3), ("ss", f3), ("to", f3), ("ts", f3), ("a", f3),
                    ("src", P), ("src_mask", P), ("tgt", P), ("tgt_mask", P), ("poses", P), ("poses_meas", P),
                    ("mats", P), ("mom", P), ("W", P), ("C", P), ("scores", P), ("est", P), ("idx", P)]
    return DmMember


def test_batch_iteration_equals_the_oracle(orc, tmp_path):
    # the batch kernels (copied verbatim out of filter.cu and measure.cu), one
    # iteration of a batch of every mode and mixed sizes under the emulation:
    # each member's perturbed cloud, matrices, moments, scores, weights,
    # resampled indices and cloud equal the oracle's single-registration
    # steps, its estimate within summation rounding
    import ctypes as C
    import pfsynth
    f, m = open(FILTER_CU).read(), open(MEASURE_CU).read()
    fr = f[f.index(PH_BEGIN):f.index(BF_END)]
    mr = m[m.index(MV_BEGIN):m.index(BM_END)]
    assert fr.count(UH_EXTERN) == 1 and mr.count(KC_EXTERN) == 2
    (tmp_path / "batch_filter.inc").write_text(fr.replace(UH_EXTERN, "extern unsigned long long sh_cdf[];"))
    (tmp_path / "batch_measure.inc").write_text(mr.replace(KC_EXTERN, "extern float4 smem_dyn[];"))
    so_path = str(tmp_path / "libbh.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-frounding-math", "-fPIC", "-shared",
                    "-I" + SHIM, "-I" + str(tmp_path), BH_CPP, "-o", so_path], check=True)
    L = C.CDLL(so_path)
    DmMember = _batch_member_type()
    L.dm_batch_step.argtypes = [C.POINTER(DmMember), C.c_int, C.c_int, C.c_int]
    rng = np.random.default_rng(40)
    for ipw, use_tab in ((1, 1), (4, 0), (2, 1)):
        n = 6
        members = (DmMember * n)()
        keep, want = [], []
        for r in range(n):
            mode = (r + ipw) % 4
            sd = tuple(int(v) for v in rng.integers(6, 26, 3))
            td = tuple(int(v) for v in rng.integers(6, 22, 3))
            N = 4 * int(rng.integers(1, 11))
            k = int(rng.integers(1, 8))
            src = pfsynth.random_image(int(rng.integers(0, 1 << 30)), sd)
            tgt = pfsynth.random_image(int(rng.integers(0, 1 << 30)), td)
            smask = (rng.random((sd[2], sd[1], sd[0])) < 0.5).astype(np.uint8)
            tmask = (rng.random((td[2], td[1], td[0])) < 0.5).astype(np.uint8)
            so, to = rng.uniform(-4, 4, 3).astype(np.float32), rng.uniform(-4, 4, 3).astype(np.float32)
            if r % 2:   # anisotropic voxels in odd members
                ss, ts = (rng.uniform(0.7, 1.4, 3).astype(np.float32) for _ in range(2))
            else:
                ss = ts = np.ones(3, np.float32)
            lim = np.array([0.6, 0.5, 0.4, 6, 5, 4], np.float32)
            seed_i, g = int(rng.integers(0, 2**63)), 5
            img, msk = mode in (2, 3), mode != 2
            b_full = int(np.count_nonzero(tmask)) if msk else 0
            n_min = int(0.01 * np.prod(td))
            _, a = orc.pose_matrix(np.zeros(6, np.float32), sd, so, to, ss, ts)
            x0 = orc.init_particles(N, seed_i, lim)
            bufs = dict(poses=x0.copy(), poses_meas=np.zeros((6, N), np.float32), mats=np.zeros((N, 12), np.float32),
                        mom=np.zeros((N, 12), np.uint64), W=np.zeros(N, np.uint64), C=np.zeros(N, np.uint64),
                        scores=np.zeros(N), est=np.zeros(6), idx=np.zeros(N, np.int32))
            vols = dict(src=src if img else None, src_mask=smask if msk else None, tgt=tgt if img else None,
                        tgt_mask=tmask if msk else None)
            keep.append((bufs, vols))
            M = members[r]
            M.mode, M.N, M.k, M.gamma_log2 = mode, N, k, g
            M.seed, M.b_full, M.n_min = seed_i, b_full, n_min
            M.lim[:] = lim.tolist()
            M.sigma0_frac, M.sigma_decay = 0.25, 0.8
            M.sd[:], M.td[:] = sd, td
            M.so[:], M.ss[:], M.to[:], M.ts[:], M.a[:] = so.tolist(), ss.tolist(), to.tolist(), ts.tolist(), a.tolist()
            for name, v in vols.items():
                setattr(M, name, None if v is None else v.ctypes.data)
            for name, v in bufs.items():
                setattr(M, name, v.ctypes.data)
            # the oracle's steps of this member alone
            x1 = orc.perturb(x0, seed_i, k, orc.sigma(0.25, 0.8, k, lim), lim)
            mats, _ = orc.pose_matrices(x1, sd, so, to, ss, ts)
            mom = np.zeros((N, 12), np.uint64)
            if img:
                mom[:, 0:7] = orc.measure_image(src, tgt, mats, a)
            if msk:
                mom[:, 8:12] = orc.measure_mask(smask, tmask, mats, a)
            s = np.array([orc.score(mode, mom[i], b_full, n_min) for i in range(N)])
            W = orc.weights(s, g)
            idx = orc.resample(W, orc.resample_offset(seed_i, k))
            want.append(dict(x1=x1, mats=mats, mom=mom, s=s, W=W, idx=idx, est=orc.estimate(x1, W)))
        L.dm_batch_step(members, n, ipw, use_tab)
        for r, ((bufs, _), w) in enumerate(zip(keep, want)):
            cfg = (ipw, use_tab, r, int(members[r].mode), int(members[r].N))
            assert np.array_equal(bufs["poses_meas"], w["x1"]), cfg
            assert np.array_equal(bufs["mats"], w["mats"]), cfg
            assert np.array_equal(bufs["mom"], w["mom"]), cfg
            assert np.array_equal(bufs["scores"], w["s"]) and np.array_equal(bufs["W"], w["W"]), cfg
            assert np.array_equal(bufs["idx"], w["idx"]), cfg
            assert np.array_equal(bufs["poses"], w["x1"][:, w["idx"]]), cfg
            np.testing.assert_allclose(bufs["est"], w["est"], rtol=1e-12, atol=1e-12, err_msg=str(cfg))


# -------------------------- whole trajectories of the kernels under the emulation

TH_CPP = os.path.join(ROOT, "tests", "trajectory_host.cpp")


def test_kernel_trajectories_equal_the_oracle(orc, tmp_path):
    # k_predict, k_measure and the update kernels (copied verbatim out of
    # filter.cu and measure.cu) run iteration after iteration from the
    # initial cloud, as the iteration graph does: every iteration's measured
    # cloud, moments, scores, weights and indices equal the oracle
    # registration's trace, its estimate within summation rounding, in all
    # four modes, on both sides of the one-block update (the larger cloud
    # for one iteration on a small grid: the emulation is slow), for
    # clouds that fill no whole warp (1 and 5 particles) and with
    # anisotropic voxel spacings in both volumes
    import ctypes as C
    import pfsynth
    f, m = open(FILTER_CU).read(), open(MEASURE_CU).read()
    fr = f[f.index(PH_BEGIN):f.index(BF_END)]
    mr = m[m.index(MV_BEGIN):m.index(BM_END)]
    (tmp_path / "batch_filter.inc").write_text(fr.replace(UH_EXTERN, "extern unsigned long long sh_cdf[];"))
    (tmp_path / "batch_measure.inc").write_text(mr.replace(KC_EXTERN, "extern float4 smem_dyn[];"))
    so_path = str(tmp_path / "libth.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-frounding-math", "-fPIC", "-shared",
                    "-I" + SHIM, "-I" + str(tmp_path), TH_CPP, "-o", so_path], check=True)
    L = C.CDLL(so_path)
    P = C.c_void_p
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    L.dm_trajectory.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, f32p, C.c_float, C.c_float, C.c_int,
                                C.c_float, P, P, i32p, f32p, P, P, i32p, f32p, f32p, P, P, C.c_int, f32p,
                                P, P, P, P, P, P]
    aniso = ((0.8, 1.1, 1.3), (1.2, 0.9, 0.7))   # source / target voxel spacings
    cases = [("mask_dice", 64, 3, 2, None), ("mask_ncc", 61, 3, 1, None), ("image_ncc", 48, 3, 4, None),
             ("combined", 40, 3, 8, None), ("mask_dice", 1, 3, 1, None), ("image_ncc", 5, 2, 2, None),
             ("mask_dice", 1025, 1, 32, None), ("image_ncc", 33, 2, 2, aniso), ("combined", 20, 2, 1, aniso)]
    for i, (mode, N, K, ipw, spacing) in enumerate(cases):
        ss, ts = (None, None) if spacing is None else (np.array(v, np.float32) for v in spacing)
        if mode in ("mask_dice", "mask_ncc"):
            small = N > 1024             # the three-kernel update: a small grid keeps the emulation quick
            pair = pfsynth.ellipsoid_pair(20 + i, src_dims=(12, 11, 10) if small else (18, 16, 14),
                                          tgt_dims=(12, 10, 6) if small else (17, 14, 11),
                                          tgt_origin=(0, 0, 2), semi_axes=(4, 3, 3) if small else (6, 5, 4),
                                          asymmetric=True, max_rot_deg=8, max_trans=3)
        else:
            pair = pfsynth.speckle_pair(20 + i, src_dims=(20, 18, 16), tgt_dims=(19, 17, 14), overlap=(0.55, 0.7),
                                        max_rot_deg=8, max_trans=3, with_masks=(mode == "combined"))
        lr, lt, seed = 0.2, 3.0, 40 + i
        ref = orc.register(mode, pair.src_dims, pair.src_origin, pair.tgt_dims, pair.tgt_origin, N, K, lr, lt,
                           seed=seed, src=pair.src if mode in ("image_ncc", "combined") else None,
                           tgt=pair.tgt if mode in ("image_ncc", "combined") else None,
                           src_mask=pair.src_mask if mode != "image_ncc" else None,
                           tgt_mask=pair.tgt_mask if mode != "image_ncc" else None,
                           src_spacing=ss, tgt_spacing=ts)
        lim = np.array([lr] * 3 + [lt] * 3, np.float32)
        sd, td = np.array(pair.src_dims, np.int32), np.array(pair.tgt_dims, np.int32)
        so = np.asarray(pair.src_origin, np.float32)
        to = np.asarray(pair.tgt_origin, np.float32)
        _, a = orc.pose_matrix(np.zeros(6, np.float32), sd, so, to, ss, ts)
        poses = orc.init_particles(N, seed, lim)
        tr = dict(p=np.zeros((K, 6, N), np.float32), m=np.zeros((K, N, 12), np.uint64), s=np.zeros((K, N)),
                  W=np.zeros((K, N), np.uint64), i=np.zeros((K, N), np.int32), e=np.zeros((K, 6)))
        img, msk = mode in ("image_ncc", "combined"), mode != "image_ncc"
        vol = lambda v, use: (np.ascontiguousarray(v).ctypes.data if use else None)   # noqa: E731
        L.dm_trajectory(orc.MODES[mode], N, K, seed, lim, 0.25, 0.8, 5, 0.01, vol(pair.src, img),
                        vol(pair.src_mask, msk), sd, so, vol(pair.tgt, img), vol(pair.tgt_mask, msk), td, to, a,
                        _p(ss), _p(ts), ipw, poses, *(tr[k].ctypes.data for k in ("p", "m", "s", "W", "i", "e")))
        for kk in range(K):
            cfg = (mode, N, kk, spacing)
            assert np.array_equal(tr["p"][kk], ref["tr_poses"][kk]), cfg
            assert np.array_equal(tr["m"][kk], ref["tr_mom"][kk]), cfg
            assert np.array_equal(tr["s"][kk], ref["tr_score"][kk]), cfg
            assert np.array_equal(tr["W"][kk], ref["tr_W"][kk]), cfg
            assert np.array_equal(tr["i"][kk], ref["tr_idx"][kk]), cfg
            np.testing.assert_allclose(tr["e"][kk], ref["tr_est"][kk], rtol=1e-12, atol=1e-12, err_msg=str(cfg))


def test_measurement_fp32_work_per_evaluation(orc, tmp_path):
    # the fp32 lane operations the measurement code executes per visited
    # evaluation (row set-up included), counted on its host build, against
    # the 27 / 12 / 33 of the arithmetic definition the roofline uses: the
    # image code's floors by rounding, unbiasing subtracts and fp32 quad
    # index cost about ten more; the mask code's table and rounding floors
    # bring it to the definition's count
    import pfsynth
    L = _build_measure_warp(open(MEASURE_CU).read(), tmp_path, extra=("-DPF_HOST_COUNT_FP32",))
    rng = np.random.default_rng(42)
    sd = td = (112, 40, 30)
    src, tgt = pfsynth.random_image(1, sd), pfsynth.random_image(2, td)
    smask = (rng.random(src.shape) < 0.5).astype(np.uint8)
    tmask = (rng.random(tgt.shape) < 0.5).astype(np.uint8)
    poses = np.array([[0.1, -0.05], [0.05, 0.1], [-0.1, 0.02], [2, -3], [1, 2], [-2, 1]], np.float32)
    mats, a = orc.pose_matrices(poses, sd, np.zeros(3, np.float32), np.array([4, 0, 0], np.float32))
    mats = np.ascontiguousarray(mats, np.float32)
    per_eval = {}
    for name, img, msk in (("image", 1, 0), ("mask", 0, 1), ("combined", 1, 1)):
        L.dm_fp32_ops_reset()
        got = np.zeros((2, 12), np.uint64)
        L.dm_measure_warp(img, msk, 0, 1, _ptr(src) if img else None, _ptr(smask) if msk else None,
                          np.array(sd, np.int32), _ptr(tgt) if img else None, _ptr(tmask) if msk else None,
                          np.array(td, np.int32), mats, 2, a, got)
        evals = int(got[:, 0].sum() if img else got[:, 8].sum())
        per_eval[name] = L.dm_fp32_ops() / evals
    assert 35 < per_eval["image"] < 40, per_eval
    assert 11 < per_eval["mask"] < 13.5, per_eval
    assert 42 < per_eval["combined"] < 48, per_eval

