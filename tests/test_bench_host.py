"""Host logic of bench.py that needs no GPU: the comment-insensitive source
hash that gates the committed ncu traffic figures, and the per-view error
summary of the accuracy report."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_only_ignores_comments_and_layout():
    a = "int f(int x) {\n    // the answer\n    return x + 42; /* inline */\n}\n"
    b = "int f(int x)\n{\n  return x + 42;\n}"
    assert bench._code_only(a) == bench._code_only(b)
    # a change of code is seen, a change inside a string literal too
    assert bench._code_only(a) != bench._code_only(a.replace("42", "43"))
    s = 'const char* m = "a // not a comment /* nor this */";'
    assert "not a comment" in bench._code_only(s) and "nor this" in bench._code_only(s)
    # escaped quotes inside literals do not end them
    e = 'const char* m = "say \\"hi\\" // still text"; // gone'
    out = bench._code_only(e)
    assert "still text" in out and "gone" not in out


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    files = ("lf_raster.cu", "lf_internal.cuh")
    good = bench._source_hash(files)
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {"k": (123, files, good), "stale": (456, files, "0" * 16)})
    assert bench._traffic("k") == 123
    assert bench._traffic("stale") is None
    assert bench._traffic("missing") is None


def test_view_errors():
    rng = np.random.default_rng(0)
    ref = rng.uniform(0, 1, (3, 4, 5, 4))
    gpu = ref.astype(np.float32).copy()
    gpu[1, 2, 3, 0] += 0.25
    r = bench.view_errors(gpu, ref)
    assert r["max_abs"] == pytest.approx(0.25, abs=1e-6)
    assert r["per_view_max_abs"][1] == pytest.approx(0.25, abs=1e-6)
    assert r["per_view_max_abs"][0] < 1e-6
    mse = 0.25 ** 2 / ref[1].size
    assert r["per_view_psnr_db"][1] == pytest.approx(10 * math.log10(1 / mse), abs=0.01)
    assert r["min_psnr_db"] == r["per_view_psnr_db"][1]
