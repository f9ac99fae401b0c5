"""Planted mistakes in the oracle, each of which its pins must catch.

The oracle is trusted because tests that do not share its arithmetic pin it
(known-answer vectors, scipy, brute force, closed forms, exact rationals).
This file checks that those pins have teeth: it copies ``oracle/pf_oracle.c``,
plants one plausible mistake (a dropped term, a wrong sign or index, a
transposed operand, an off-by-one), builds the copy, and runs the CPU pin
suites against it through ``PF_ORACLE_LIB``.  Every mutant must make at least
one pin fail.  The CUDA path is not involved.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pf_oracle.c")
PINS = [os.path.join(ROOT, "tests", f) for f in ("test_oracle_pins.py", "test_oracle_filter.py")]
NN_SRC = os.path.join(ROOT, "oracle", "nn.py")
NN_PINS = [os.path.join(ROOT, "tests", "test_oracle_nn.py")]

# (name, where in the paper the correct form comes from, text, planted text)
MUTANTS = [
    ("philox_multipliers", "RNG (Philox4x32-10, SC'11)",
     "uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;\n        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;",
     "uint64_t p0 = (uint64_t)0xCD9E8D57u * (uint64_t)c0;\n        uint64_t p1 = (uint64_t)0xD2511F53u * (uint64_t)c2;"),
    ("philox_rounds", "RNG (Philox4x32-10, SC'11)",
     "for (int round = 0; round < 10; ++round) {", "for (int round = 0; round < 9; ++round) {"),
    ("sin_divisors", "Eq. 3 (sin/cos reading)",
     "t[k] = (t[k - 1] * (-x2)) / (double)((2 * k) * (2 * k + 1));",
     "t[k] = (t[k - 1] * (-x2)) / (double)((2 * k) * (2 * k + 2));"),
    ("cos_sign", "Eq. 3 (sin/cos reading)",
     "t[k] = (t[k - 1] * (-x2)) / (double)((2 * k - 1) * (2 * k));",
     "t[k] = (t[k - 1] * (x2)) / (double)((2 * k - 1) * (2 * k));"),
    ("rotation_order", "Eq. 3 (R = Rz Rx Ry)", "matmul3(Rx, Ry, XY);", "matmul3(Ry, Rx, XY);"),
    ("rotation_sign", "Eq. 3",
     "double Rx[3][3] = {{1.0, 0.0, 0.0}, {0.0, ca, -sa}, {0.0, sa, ca}};",
     "double Rx[3][3] = {{1.0, 0.0, 0.0}, {0.0, ca, sa}, {0.0, -sa, ca}};"),
    ("rotation_centre", "Eq. 3 (centre reading)",
     "double c = (double)sorigin[i] + ss[i] * ((double)(sdims[i] - 1) / 2.0);",
     "double c = (double)sorigin[i] + ss[i] * ((double)sdims[i] / 2.0);"),
    ("spacing_index", "Eq. 3 in world units (Table 1 spacings)",
     "M[4 * i + j] = (float)((R[3 * i + j] * ts[j]) / ss[i]);",
     "M[4 * i + j] = (float)((R[3 * i + j] * ts[i]) / ss[i]);"),
    ("translation_sign", "Eq. 3",
     "double b = ((c + (double)pose[3 + i]) - (double)sorigin[i]) / ss[i];",
     "double b = ((c - (double)pose[3 + i]) - (double)sorigin[i]) / ss[i];"),
    ("coordinate_axis", "Eq. 3 applied per voxel", "q[i] = M[4 * i + 0] * dx + K;", "q[i] = M[4 * i + 0] * dy + K;"),
    ("nn_truncates", "Sec. 3.3 (nearest-neighbour reading)",
     "float h0 = q[0] + 0.5f, h1 = q[1] + 0.5f, h2 = q[2] + 0.5f;", "float h0 = q[0], h1 = q[1], h2 = q[2];"),
    ("nn_inside", "Sec. 3.3 (nearest-neighbour reading)",
     "if (!(h0 >= 0.0f && h0 < (float)sd[0])) return 0;", "if (!(h0 >= 0.0f && h0 < (float)(sd[0] - 1))) return 0;"),
    ("lerp_direction", "Sec. 3.3 (trilinear)", "return fmaf(f, b - a, a);", "return fmaf(f, a - b, b);"),
    ("trilinear_inside", "Sec. 3.3 (trilinear)",
     "if (!(q[d] >= 0.0f && q[d] <= (float)(sd[d] - 1))) return 0;",
     "if (!(q[d] >= 0.0f && q[d] < (float)(sd[d] - 1))) return 0;"),
    ("trilinear_corner", "Sec. 3.3 (trilinear)",
     "float v010 = S[base + sx], v110 = S[base + sx + 1];", "float v010 = S[base + sxy], v110 = S[base + sxy + 1];"),
    ("fixed_point_bits", "Eq. 2 (fixed-point reading)",
     "uint64_t sq = (uint64_t)lrintf(s * 32768.0f);", "uint64_t sq = (uint64_t)lrintf(s * 16384.0f);"),
    ("moment_t2", "Eq. 2", "T2 += t * t;", "T2 += t;"),
    ("ncc_unsquared", "Eq. 2",
     "return (c * c) / (u128_to_f64(vs) * u128_to_f64(vt));", "return c / (u128_to_f64(vs) * u128_to_f64(vt));"),
    ("dice_factor", "Eq. 4",
     "return (double)(2 * C) / (double)(A + b_full);", "return (double)C / (double)(A + b_full);"),
    ("dice_overlap_only", "Eq. 4 (whole-grid |T| reading)",
     "return orc_dice_from_counts(mk[0], mk[1], mk[3], b_full, n_min);",
     "return orc_dice_from_counts(mk[0], mk[1], mk[3], mk[2], n_min);"),
    ("gamma_squarings", "Fig. 1 update (likelihood reading)",
     "for (int32_t j = 0; j < g; ++j) r = r * r;", "for (int32_t j = 0; j <= g; ++j) r = r * r;"),
    ("weight_scale", "Fig. 1 update (quantised weights)",
     "W[i] = (uint64_t)(r * 16777216.0);", "W[i] = (uint64_t)(r * 8388608.0);"),
    ("resample_ge", "Fig. 1 resampling (systematic reading)",
     "while (!(C[i] > T)) ++i;", "while (!(C[i] >= T)) ++i;"),
    ("resample_offset", "Fig. 1 resampling (systematic reading)",
     "u128 num = (u128)((((uint64_t)j) << 32) + (uint64_t)u) * (u128)S;",
     "u128 num = (u128)(((uint64_t)j) << 32) * (u128)S;"),
    ("estimate_unweighted", "Fig. 1 estimation (weighted-mean reading)",
     "for (int32_t i = 0; i < N; ++i) acc = acc + (double)W[i] * (double)x[i];\n            est[d] = acc / (double)S;",
     "for (int32_t i = 0; i < N; ++i) acc = acc + (double)x[i];\n            est[d] = acc / (double)N;"),
    ("init_one_sided", "Abstract (limits); init reading",
     "poses[(int64_t)d * N + i] = lim[d] * (2.0f * unit24(u[d]) - 1.0f);",
     "poses[(int64_t)d * N + i] = lim[d] * unit24(u[d]);"),
    ("perturb_biased", "Fig. 1 prediction (noise reading)",
     "- 2.0f) * sqrt3;\n            float *x = poses", "- 1.0f) * sqrt3;\n            float *x = poses"),
    ("perturb_unclamped", "Fig. 1 prediction (clamp to the limits)",
     "            float v = *x + sigma[d] * e;\n            if (v > lim[d]) v = lim[d];",
     "            float v = *x + sigma[d] * e;\n            if (v > 2 * lim[d]) v = lim[d];"),
    ("sigma_decay", "Fig. 1 prediction (noise schedule reading)",
     "for (int32_t j = 0; j < k; ++j) p = p * (double)decay;\n    for (int d = 0; d < 6; ++d) sigma[d]",
     "for (int32_t j = 1; j < k; ++j) p = p * (double)decay;\n    for (int d = 0; d < 6; ++d) sigma[d]"),
    ("warp_truncates", "Abstract / Sec. 3.3 (sequence warp)", "long r = lrintf(s);", "long r = (long)s;"),
    ("warp_nn_binarised", "Abstract / Sec. 3.3 (sequence warp)",
     "if (nn_inside(q, sd, &si)) v = src[si];", "if (nn_inside(q, sd, &si)) v = src[si] ? 255 : 0;"),
    ("min_overlap_boundary", "Eq. 2 / Eq. 4 (minimum-overlap reading)",
     "if (n == 0 || n < n_min) return 0.0;", "if (n == 0 || n <= n_min) return 0.0;"),
    ("ncc_covariance_sign", "Eq. 2",
     "u128 cv = nST >= S1T1 ? nST - S1T1 : S1T1 - nST;", "u128 cv = nST - S1T1;"),
    ("ncc_zero_variance", "Eq. 2 (zero-variance reading)",
     "if (nS2 <= S1S1 || nT2 <= T1T1) return 0.0;", "if (nS2 < S1S1 || nT2 < T1T1) return 0.0;"),
    ("u128_low_word", "Eq. 2 (128-bit brackets)",
     "return (double)hi * 18446744073709551616.0 + (double)lo;", "return (double)hi * 18446744073709551616.0;"),
    ("s2_words_swapped", "Eq. 2 (moment layout)",
     "o[2] = (uint64_t)S2; o[3] = (uint64_t)(S2 >> 64);", "o[3] = (uint64_t)S2; o[2] = (uint64_t)(S2 >> 64);"),
    ("mask_count_b", "Eq. 4 (counts)", "                    B += t;\n", "                    B += s;\n"),
    ("mask_count_c", "Eq. 4 (counts)", "C += s & t;", "C += s | t;"),
    ("combined_weight", "combined score reading",
     "return 0.5 * (orc_ncc2_from_moments", "return 1.0 * (orc_ncc2_from_moments"),
    ("target_offset_sign", "Eq. 3",
     "a[i] = (float)((c - (double)torigin[i]) / ts[i]);", "a[i] = (float)((c + (double)torigin[i]) / ts[i]);"),
    ("f64_check_uncentred", "Eq. 2 (fp64 check)",
     "double ds = sv[i] - ms, dt = tv[i] - mt;", "double ds = sv[i] - ms, dt = tv[i];"),
    ("resample_zero_sum", "Fig. 1 resampling (S = 0 reading)",
     "if (S == 0) { idx[j] = j; continue; }", "if (S == 0) { idx[j] = 0; continue; }"),
    ("resample_offset_fixed", "Fig. 1 resampling (one offset per iteration)",
     "philox_seeded(seed, 0u, (uint32_t)k, ORC_STREAM_RESAMPLE, 0u, r);",
     "philox_seeded(seed, 0u, 0u, ORC_STREAM_RESAMPLE, 0u, r);"),
    ("estimate_zero_sum", "Fig. 1 estimation (S = 0 reading)",
     "est[d] = acc / (double)N;\n        }", "est[d] = acc / (double)(N + 1);\n        }"),
    ("init_stream_reuse", "RNG streams (init reading)",
     "philox_seeded(seed, (uint32_t)i, 0u, ORC_STREAM_INIT, 1u, r1);",
     "philox_seeded(seed, (uint32_t)i, 0u, ORC_STREAM_INIT, 0u, r1);"),
    ("perturb_same_each_iteration", "RNG streams (noise reading)",
     "philox_seeded(seed, (uint32_t)i, (uint32_t)k, ORC_STREAM_PERTURB, (uint32_t)d, r);",
     "philox_seeded(seed, (uint32_t)i, 0u, ORC_STREAM_PERTURB, (uint32_t)d, r);"),
    ("perturb_same_each_dof", "RNG streams (noise reading)",
     "philox_seeded(seed, (uint32_t)i, (uint32_t)k, ORC_STREAM_PERTURB, (uint32_t)d, r);",
     "philox_seeded(seed, (uint32_t)i, (uint32_t)k, ORC_STREAM_PERTURB, 0u, r);"),
    ("register_skips_first_prediction", "Fig. 1 cycle (iteration order reading)",
     "        if (k > 0) {\n            float sig[6];", "        if (k > 1) {\n            float sig[6];"),
    ("register_ignores_proposal_spread", "Sec. 6 seeding (noise base reading)",
     "for (int d = 0; d < 6; ++d) sig[d] = (float)((double)sig_base[d] * p);",
     "for (int d = 0; d < 6; ++d) sig[d] = sig[d];"),
    ("seed_mean_ignored", "Sec. 6 seeding",
     "float v = mean[d] + std[d] * e;", "float v = std[d] * e;"),
    ("seed_lower_clamp_missing", "Sec. 6 seeding (clamp to the limits)",
     "            float v = mean[d] + std[d] * e;\n            if (v > lim[d]) v = lim[d];\n            if (v < -lim[d]) v = -lim[d];",
     "            float v = mean[d] + std[d] * e;\n            if (v > lim[d]) v = lim[d];"),
]


# The proposal network's oracle (oracle/nn.py, numpy) and its pins.
NN_MUTANTS = [
    ("conv_taps_transposed", "convolution (4^3 taps, stride 2, padding 1)",
     "patch = xp[:, kz:kz + 2 * Do:2, ky:ky + 2 * Do:2, kx:kx + 2 * Do:2, :]\n        out += patch",
     "patch = xp[:, kz:kz + 2 * Do:2, kx:kx + 2 * Do:2, ky:ky + 2 * Do:2, :]\n        out += patch"),
    ("conv_bias_dropped", "convolution", "        out += np.asarray(bias, np.float64)\n", "        out += 0.0\n"),
    ("dgrad_tap_flipped", "data gradient (adjoint of the convolution)",
     "+= dy @ w[:, t, :]", "+= dy @ w[:, 63 - t, :]"),
    ("wgrad_operands", "weight gradient", "dw[:, t, :] = g.T @ patch", "dw[:, t, :] = g.T @ np.roll(patch, 1, axis=0)"),
    ("nll_mean_gradient_sign", "loss (Gaussian NLL)",
     "g[:, :6] = -(y - mu) * np.exp(-s) / out.shape[0]", "g[:, :6] = (y - mu) * np.exp(-s) / out.shape[0]"),
    ("nll_variance_gradient_half", "loss (Gaussian NLL)",
     "g[:, 6:12] = 0.5 * (1.0 - r2 * np.exp(-s)) / out.shape[0]", "g[:, 6:12] = (1.0 - r2 * np.exp(-s)) / out.shape[0]"),
    ("adam_no_bias_correction", "Adam", "mh = m / (1.0 - beta1 ** t)", "mh = m"),
    ("adam_second_moment", "Adam", "v = beta2 * v + (1.0 - beta2) * g * g", "v = beta2 * v + (1.0 - beta2) * np.abs(g)"),
    ("fc_relu_mask_dropped", "network backward", "dh = (dout @ P[\"f2w\"]) * (h > 0)", "dh = dout @ P[\"f2w\"]"),
    ("conv_relu_mask_dropped", "network backward",
     "d = rnd(conv3d_backward_data(d, rnd(P[f\"cw{l}\"]), below.shape[1]) * (below > 0))",
     "d = rnd(conv3d_backward_data(d, rnd(P[f\"cw{l}\"]), below.shape[1]))"),
    ("bias_gradient_scaled", "network backward", "put(f\"cb{l}\", d.reshape(-1, 32).sum(0))",
     "put(f\"cb{l}\", d.reshape(-1, 32).mean(0))"),
    ("bf16_ties_away", "bf16 rounding (nearest, ties to even)",
     "r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)",
     "r = ((u + np.uint64(0x8000)) >> np.uint64(16)) << np.uint64(16)"),
    ("box_average_scale", "network input (box average / 64)",
     "return np.where(cnt > 0, tot / np.maximum(cnt, 1) / 64.0, 0.0)",
     "return np.where(cnt > 0, tot / np.maximum(cnt, 1), 0.0)"),
    ("box_average_edge", "network input (box average)",
     "lo = np.ceil((box_o[d] + h[d] * np.arange(G) - origin[d]) / spacing[d]).astype(np.int64)",
     "lo = np.floor((box_o[d] + h[d] * np.arange(G) - origin[d]) / spacing[d]).astype(np.int64)"),
]

# Runs the network pins with a mutant module standing in for oracle.nn.
_NN_RUNNER = """
import importlib.util, sys
sys.path.insert(0, sys.argv[1])
import oracle
spec = importlib.util.spec_from_file_location("oracle.nn", sys.argv[2])
mod = importlib.util.module_from_spec(spec)
sys.modules["oracle.nn"] = mod
oracle.nn = mod
spec.loader.exec_module(mod)
import pytest
sys.exit(pytest.main(sys.argv[3:]))
"""


def _build(name, text, planted, outdir):
    src = open(SRC).read()
    assert src.count(text) == 1, f"{name}: the text to replace must occur exactly once"
    path = os.path.join(outdir, f"{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(text, planted))
    so = os.path.join(outdir, f"lib{name}.so")
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    path, "-o", so, "-lm"], check=True)
    return so


def _run_pins(so):
    env = dict(os.environ, PF_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    failed = [ln.split(" ")[1] for ln in r.stdout.splitlines() if ln.startswith("FAILED ")]
    return r.returncode, failed


def _write_nn(name, text, planted, outdir):
    src = open(NN_SRC).read()
    assert src.count(text) == 1, f"{name}: the text to replace must occur exactly once"
    path = os.path.join(outdir, f"nn_{name}.py")
    with open(path, "w") as f:
        f.write(src.replace(text, planted))
    return path


def _run_nn_pins(path):
    r = subprocess.run([sys.executable, "-c", _NN_RUNNER, ROOT, path, *NN_PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    failed = [ln.split(" ")[1] for ln in r.stdout.splitlines() if ln.startswith("FAILED ")]
    return r.returncode, failed


def test_mutant_table_is_well_formed():
    for table, path in ((MUTANTS, SRC), (NN_MUTANTS, NN_SRC)):
        names = [m[0] for m in table]
        assert len(names) == len(set(names))
        src = open(path).read()
        for name, _, text, planted in table:
            assert src.count(text) == 1, name
            assert text != planted, name


def test_every_planted_mistake_fails_a_pin(tmp_path):
    sos = [(m[0], _build(m[0], m[2], m[3], str(tmp_path))) for m in MUTANTS]
    with ThreadPoolExecutor(max_workers=max(1, min(os.cpu_count() or 1, 16))) as ex:
        results = list(ex.map(lambda t: (t[0],) + _run_pins(t[1]), sos))
    survivors = [name for name, rc, _ in results if rc == 0]
    assert not survivors, f"planted mistakes no pin caught: {survivors}"
    for name, rc, failed in results:
        assert rc == 1, f"{name}: the pin run ended with {rc} (a crash, not a failing pin)"


def test_every_planted_network_mistake_fails_a_pin(tmp_path):
    paths = [(m[0], _write_nn(m[0], m[2], m[3], str(tmp_path))) for m in NN_MUTANTS]
    with ThreadPoolExecutor(max_workers=max(1, min(os.cpu_count() or 1, 16))) as ex:
        results = list(ex.map(lambda t: (t[0],) + _run_nn_pins(t[1]), paths))
    survivors = [name for name, rc, _ in results if rc == 0]
    assert not survivors, f"planted mistakes no pin caught: {survivors}"
    for name, rc, failed in results:
        assert rc == 1, f"{name}: the pin run ended with {rc} (a crash, not a failing pin)"
