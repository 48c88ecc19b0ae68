"""Host helpers of bench.py: the memory-bound FastConv summary picks the batched 16 x 1080p
rows of the direct path with kernels up to 5 x 5 and the separable rows (never typed
inputs or compute-bound kernels), and the host CPU record is well formed."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def _row(kernel, **kw):
    r = {"input": [16, 1080, 1920], "kernel": kernel, "us": 50.0, "GBps": 5000.0, "hbm_frac": 0.7}
    r.update(kw)
    return r


def test_conv_hbm_summary_selects_memory_bound_batched_rows():
    rows = [
        _row([1, 2, 2]), _row([1, 3, 3]), _row([1, 5, 5]), _row([1, 7, 7]), _row([1, 15, 15]),
        _row([1, 3, 3], input_dtype="uint8"), _row([1, 15, 15], path="separable"),
        {"input": [1080, 1920], "kernel": [3, 3], "us": 10.0, "GBps": 1600.0, "hbm_frac": 0.24},
        {"input": [1080, 1920], "crossover_direct_vs_fft": []},
    ]
    out = bench.conv_hbm_summary(rows, 6800.3)
    assert out["peak"] == 6800.3 and out["unit"] == "GB/s"
    names = [r["workload"] for r in out["rows"]]
    assert names == ["16 x 1080 x 1920 FP32 * 1 x 2 x 2", "16 x 1080 x 1920 FP32 * 1 x 3 x 3",
                     "16 x 1080 x 1920 FP32 * 1 x 5 x 5", "16 x 1080 x 1920 FP32 * 1 x 15 x 15 (separable)"]
    assert all(r["frac"] == 0.7 for r in out["rows"])


def test_host_cpu_record():
    info = bench.host_cpu()
    assert info["nproc"] == (os.cpu_count() or 1)
    assert isinstance(info["model"], str) and info["model"]
