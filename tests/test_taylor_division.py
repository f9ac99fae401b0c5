"""The device sin/cos chain's division shortcut, checked on the CPU.

The fp64 Taylor chain of the pose -> matrix step (Eq. 3) divides every term
by a constant; the device takes each quotient from a stored reciprocal and
one FMA correction (Markstein, 1990) for fp32 angles with
2^-32 <= |x| <= 64, and from the IEEE division elsewhere.  These tests pin
the stored reciprocals to their definition and walk every fp32 angle of that
range through both chains, so the shortcut is the correctly rounded quotient
on every input the kernels can receive.
"""
import os
import platform
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2504_19930_gb300", "csrc", "device.cuh")
CHECK_C = os.path.join(ROOT, "tests", "taylor_division_check.c")


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


def test_division_shortcut_is_exact_for_every_fp32_angle(tmp_path):
    exe = str(tmp_path / "taylor_division_check")
    subprocess.run(["gcc", *_flags(), "-o", exe, CHECK_C], check=True)
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
    n_angles = 0x42800000 - 0x2F800000 + 1          # fp32 bit patterns of 2^-32 .. 64
    assert checked == 26 * n_angles                 # 13 divisions in each of the two chains
    assert bad == 0
