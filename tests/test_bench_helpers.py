"""Host-side helpers of bench.py (no GPU)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_settled_iteration():
    f = bench.settled_iteration
    assert f([0.5, 0.9, 0.99, 0.99], 0.985) == 3          # first iteration of the final run above target
    assert f([0.99, 0.95, 0.99, 0.99], 0.985) == 3        # a dip resets the count
    assert f([0.99, 0.99], 0.985) == 1
    assert f([0.99, 0.97], 0.985) is None                 # never settles: the last one is below
    assert f([], 0.5) is None
    assert f(np.array([0.2, 0.6]), 0.6) == 2              # >= target counts


def test_workloads_name_sizes_not_indices():
    for key, w in bench.WORKLOADS.items():
        assert not key.startswith("config"), key
        assert "name" in w


def test_kernel_code_hash_ignores_comments_only(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("// header\n__global__ void k(int *p) {\n    p[0] = 1;   // store\n}\n")
    b.write_text("/* another\n header */\n__global__ void k(int *p) {\n  p[0] = 1;\n}\n")
    c.write_text("__global__ void k(int *p) {\n    p[0] = 2;\n}\n")
    h = bench.kernel_code_hash
    assert h([str(a)]) == h([str(b)])
    assert h([str(a)]) != h([str(c)])
    assert h([str(a), str(c)]) != h([str(c), str(a)])   # file order and boundaries count



def test_cpu_sample_size():
    import types
    f = bench.cpu_sample_size
    none = types.SimpleNamespace(cpu_sample_particles=None, cpu_sample_iters=None)
    assert f(none, bench.WORKLOADS["image224"]) == (64, 2)
    assert f(none, bench.WORKLOADS["combined256"]) == (64, 2)
    assert f(none, bench.WORKLOADS["mask64"]) == (256, 10)            # the whole small registration
    given = types.SimpleNamespace(cpu_sample_particles=8, cpu_sample_iters=1)
    assert f(given, bench.WORKLOADS["image224"]) == (8, 1)
    assert f(types.SimpleNamespace(), bench.WORKLOADS["mask64"]) == (256, 10)


def test_secondary_lines_summarised_and_failures_kept_out_of_the_main_line(monkeypatch):
    import json
    import subprocess
    import types

    good = {"metric": "m", "value": 2.5, "unit": "u", "steps": 1500, "ms_per_step": 1.8,
            "config": {"workload": "mask64_dice_n256_k10"},
            "roofline": {"bound": "alu", "frac": 0.12, "l2": {"frac": 0.03}},
            "clocks": {"sm_mhz": 2070.0}, "e2e": None}

    def fake_run(cmd, **kw):
        if "mask64" in cmd:
            return types.SimpleNamespace(returncode=0, stdout="noise\n" + json.dumps(good) + "\n", stderr="")
        return types.SimpleNamespace(returncode=3, stdout="", stderr="boom\nlast line")

    monkeypatch.setattr(subprocess, "run", fake_run)
    out = bench.run_secondary()
    assert out["mask64"]["value"] == 2.5 and out["mask64"]["roofline"]["frac"] == 0.12
    assert out["mask64"]["l2_frac"] == 0.03 and out["mask64"]["clocks"]["sm_mhz"] == 2070.0
    assert "exit 3" in out["conv32"]["missing"] and "last line" in out["conv32"]["missing"]
    json.dumps(out)   # the summary is JSON-serialisable
