"""CPU check of the integer-unit FP64 <-> FP32 conversions the metric and
transformation kernels use (csrc/fp_convert.h), compiled for the host: every
result in the binary32 normal range equals numpy's round-to-nearest-even
conversion bit for bit (random values over many decades, exact halfway
cases with both parities, values next to powers of two and to the overflow
threshold), subnormal results flush to signed zero, and the way back is
exact."""
import os
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1803_07822_gb300", "csrc")


def run(x, tmp_path):
    exe = tmp_path / "conv"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I" + CSRC, os.path.join(ROOT, "tests", "fp_convert_check.cpp"),
                           "-o", str(exe)])
    fi, f1, f2 = tmp_path / "in.bin", tmp_path / "o32.bin", tmp_path / "o64.bin"
    x.astype(np.float64).tofile(fi)
    subprocess.check_call([str(exe), str(fi), str(f1), str(f2)])
    return np.fromfile(f1, dtype=np.float32), np.fromfile(f2, dtype=np.float64)


def test_f64_to_f32_round_to_nearest_even(tmp_path):
    rng = np.random.default_rng(0)
    vals = [rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000)]
    # exact halfway cases: a binary32 value plus half an ulp, kept and dropped bit patterns both ways
    f = rng.standard_normal(4000).astype(np.float32).astype(np.float64)
    ulp = np.spacing(np.abs(f).astype(np.float32)).astype(np.float64)
    vals += [f + 0.5 * ulp, f - 0.5 * ulp, f + 0.5 * ulp * (1 + 2.0 ** -20), f + 0.5 * ulp * (1 - 2.0 ** -20)]
    vals += [np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** 127, 2.0 ** -126, 3.4028234663852886e38,
                       3.4028235677973366e38, 1.0 - 2.0 ** -25, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24])]
    x = np.concatenate(vals)
    got, back = run(x, tmp_path)
    ref = x.astype(np.float32)
    normal = (np.abs(ref) >= np.finfo(np.float32).tiny) & np.isfinite(ref)
    assert normal.sum() > 20000
    assert np.array_equal(got[normal].view(np.uint32), ref[normal].view(np.uint32))
    # above the range: infinity of the same sign
    big = ~np.isfinite(ref)
    assert np.array_equal(got[big], ref[big])
    # below the normal range: signed zero
    small = (np.abs(ref) < np.finfo(np.float32).tiny)
    assert np.all(got[small] == 0.0) and np.array_equal(np.signbit(got[small]), np.signbit(x[small]))
    # and back, exactly
    fin = np.isfinite(got)
    assert np.array_equal(back[fin], got[fin].astype(np.float64))
